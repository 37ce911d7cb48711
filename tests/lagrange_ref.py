"""Independent restatement of serial-chain dynamics for pinning the oracle.

Nothing here is shared with the oracle or the CUDA path. Poses come from
scipy's matrix exponential of the 4x4 twist matrix, link twists from the
matrix identity G^-1 dG/dt (no 6x6 adjoint), kinetic energy from the
textbook rigid-body formula 1/2 m |v + w x c|^2 + 1/2 w^T I_c w, and the
joint torques from Lagrange's equations

    tau = M(q) qdd + Mdot(q, qd) qd - d/dq (1/2 qd^T M qd) + d/dq PE(q),

with M(q) obtained from the kinetic energy by polarisation (exact for a
quadratic form) and the q-derivatives by central differences.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import expm


def hat(w):
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def vee_twist(X):
    """4x4 twist matrix -> (v, w)."""
    return np.array([X[0, 3], X[1, 3], X[2, 3], X[2, 1], X[0, 2], X[1, 0]])


def twist_matrix(S):
    X = np.zeros((4, 4))
    X[:3, :3] = hat(S[3:])
    X[:3, 3] = S[:3]
    return X


def home(Mrow):
    T = np.eye(4)
    T[:3, :3] = Mrow[:9].reshape(3, 3)
    T[:3, 3] = Mrow[9:12]
    return T


def poses(chain, q):
    """G_k (base -> link k) for k = 1..n, via expm of the twist matrices."""
    G = np.eye(4)
    out = []
    for i in range(chain.n):
        G = G @ home(chain.M[i]) @ expm(twist_matrix(chain.S[i]) * q[i])
        out.append(G.copy())
    return out


def link_twists(chain, q, qd):
    """Body twist of each link: [V_k] = G_k^-1 dG_k/dt, with
    dG_k/dq_j = G_j [S_j] G_j^-1 G_k for j <= k."""
    Gs = poses(chain, q)
    out = []
    for k in range(chain.n):
        Gk_inv = np.linalg.inv(Gs[k])
        X = np.zeros((4, 4))
        for j in range(k + 1):
            X += Gk_inv @ Gs[j] @ twist_matrix(chain.S[j]) @ np.linalg.inv(Gs[j]) @ Gs[k] * qd[j]
        out.append(vee_twist(X))
    return out


def _Ic(row):
    return np.array([[row[4], row[7], row[8]], [row[7], row[5], row[9]], [row[8], row[9], row[6]]])


def body_kinetic(row, V):
    """1/2 m |v + w x c|^2 + 1/2 w^T I_c w for one body with twist V."""
    m, c = row[0], row[1:4]
    v, w = V[:3], V[3:]
    vc = v + np.cross(w, c)
    return 0.5 * m * vc @ vc + 0.5 * w @ _Ic(row) @ w


def kinetic(chain, q, qd):
    return sum(body_kinetic(chain.inertia[k], V) for k, V in enumerate(link_twists(chain, q, qd)))


def potential(chain, q, g=9.81):
    """Gravity along -z with magnitude g."""
    pe = 0.0
    for k, G in enumerate(poses(chain, q)):
        c = np.append(chain.inertia[k, 1:4], 1.0)
        pe += chain.inertia[k, 0] * g * (G @ c)[2]
    return pe


def mass_matrix(chain, q):
    n = chain.n
    E = np.eye(n)
    ke = [kinetic(chain, q, E[i]) for i in range(n)]
    Mq = np.empty((n, n))
    for i in range(n):
        Mq[i, i] = 2.0 * ke[i]
        for j in range(i + 1, n):
            Mq[i, j] = Mq[j, i] = kinetic(chain, q, E[i] + E[j]) - ke[i] - ke[j]
    return Mq


def spatial_inertia(row):
    """6x6 J with V^T J V = 2 KE(V), by polarisation of the kinetic energy."""
    E = np.eye(6)
    J = np.empty((6, 6))
    ke = [body_kinetic(row, E[a]) for a in range(6)]
    for a in range(6):
        J[a, a] = 2.0 * ke[a]
        for b in range(a + 1, 6):
            J[a, b] = J[b, a] = body_kinetic(row, E[a] + E[b]) - ke[a] - ke[b]
    return J


def torques(chain, q, qd, qdd, g=9.81, h=1e-5):
    """Lagrange's equations; base at rest, gravity g along -z, no external wrench."""
    n = chain.n
    q, qd, qdd = (np.asarray(x, dtype=np.float64) for x in (q, qd, qdd))
    Mq = mass_matrix(chain, q)
    Mdot = (mass_matrix(chain, q + h * qd) - mass_matrix(chain, q - h * qd)) / (2 * h)
    dK = np.empty(n)
    dP = np.empty(n)
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        dK[i] = (kinetic(chain, q + e, qd) - kinetic(chain, q - e, qd)) / (2 * h)
        dP[i] = (potential(chain, q + e, g) - potential(chain, q - e, g)) / (2 * h)
    return Mq @ qdd + Mdot @ qd - dK + dP, Mq


def tip_jacobian(chain, q):
    """Body Jacobian of the last link: column j = twist of link n per unit qd_j."""
    n = chain.n
    cols = []
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        cols.append(link_twists(chain, q, e)[-1])
    return np.stack(cols, axis=1)


# ----- the paper's scan operands, written out for the bracketing pins -----

def Ad(T):
    R, p = T[:3, :3], T[:3, 3]
    A = np.zeros((6, 6))
    A[:3, :3] = R
    A[:3, 3:] = hat(p) @ R
    A[3:, 3:] = R
    return A


def ad(xi):
    A = np.zeros((6, 6))
    A[:3, :3] = hat(xi[3:])
    A[:3, 3:] = hat(xi[:3])
    A[3:, 3:] = hat(xi[3:])
    return A


def link_transforms(chain, q):
    return [home(chain.M[i]) @ expm(twist_matrix(chain.S[i]) * q[i]) for i in range(chain.n)]
