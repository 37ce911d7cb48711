"""Pins of the FP64 oracle against facts that do not come from the oracle.

Closed forms (pendulum, planar two-link arm), an independent Lagrangian
restatement (tests/lagrange_ref.py), invariants of the equations of motion,
and brute-force bracketings of the paper's scan operators. Each check is
chosen so that a dropped term, a flipped sign, a wrong index or a transposed
operand in the oracle fails at least one of them.
"""
import itertools
from functools import lru_cache

import numpy as np
import pytest

import chaingen
import oracle
import lagrange_ref as L

G = 9.81


def base(V0=None, dV0=None, F=None):
    b = np.zeros(18)
    if V0 is not None:
        b[0:6] = V0
    b[6:12] = dV0 if dV0 is not None else [0, 0, G, 0, 0, 0]
    if F is not None:
        b[12:18] = F
    return b


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("Ixx", [0.0, 0.03])
def test_pendulum_closed_form(Ixx):
    m, l = 1.7, 0.45
    ch = chaingen.pendulum(m, l, Ixx)
    rng = np.random.default_rng(3)
    q = rng.uniform(-np.pi, np.pi, (64, 1))
    qd = rng.normal(0, 1, (64, 1))
    qdd = rng.normal(0, 2, (64, 1))
    tau = oracle.rnea(ch, q, qd, qdd)
    expect = (m * l * l + Ixx) * qdd + m * G * l * np.sin(q)
    assert np.max(np.abs(tau - expect)) < 1e-13 * max(1.0, np.max(np.abs(expect)))
    # gravity torque flips sign with q; the velocity does not enter
    t_neg = oracle.rnea(ch, -q, qd, np.zeros_like(q))
    t_pos = oracle.rnea(ch, q, -qd, np.zeros_like(q))
    assert np.allclose(t_neg, -t_pos, atol=1e-13)


def test_planar_two_link_closed_form():
    m1, m2, l1, lc1, lc2, I1, I2 = 1.3, 0.9, 0.6, 0.25, 0.31, 0.021, 0.013
    ch = chaingen.planar_two_link(m1, m2, l1, lc1, lc2, I1, I2)
    rng = np.random.default_rng(5)
    B = 50
    q = rng.uniform(-np.pi, np.pi, (B, 2))
    qd = rng.normal(0, 1, (B, 2))
    qdd = rng.normal(0, 2, (B, 2))
    # gravity along -y: base acceleration +g along y, angles from the x axis
    tau = oracle.rnea(ch, q, qd, qdd, base(dV0=[0, G, 0, 0, 0, 0]))
    q1, q2 = q[:, 0], q[:, 1]
    M11 = I1 + I2 + m1 * lc1**2 + m2 * (l1**2 + lc2**2 + 2 * l1 * lc2 * np.cos(q2))
    M12 = I2 + m2 * (lc2**2 + l1 * lc2 * np.cos(q2))
    M22 = I2 + m2 * lc2**2
    h = m2 * l1 * lc2 * np.sin(q2)
    t1 = (M11 * qdd[:, 0] + M12 * qdd[:, 1] - h * (2 * qd[:, 0] * qd[:, 1] + qd[:, 1] ** 2)
          + (m1 * lc1 + m2 * l1) * G * np.cos(q1) + m2 * lc2 * G * np.cos(q1 + q2))
    t2 = M12 * qdd[:, 0] + M22 * qdd[:, 1] + h * qd[:, 0] ** 2 + m2 * lc2 * G * np.cos(q1 + q2)
    assert np.max(np.abs(tau[:, 0] - t1)) < 1e-12
    assert np.max(np.abs(tau[:, 1] - t2)) < 1e-12


# --------------------------------------------------- Lagrangian restatement

@lru_cache(maxsize=None)
def chain_n(n, seed=chaingen.BASE_SEED):
    return chaingen.make_chain(n, seed=seed)


def states(B, n, seed=11):
    return chaingen.make_states(B, n, seed=seed)


@pytest.mark.parametrize("n", [1, 2, 3, 7])
def test_oracle_matches_lagrange(n):
    ch = chain_n(n)
    st = states(4, n)
    tau = oracle.rnea(ch, st["q"], st["qd"], st["qdd"])
    for b in range(4):
        t_ref, _ = L.torques(ch, st["q"][b], st["qd"][b], st["qdd"][b])
        scale = max(1.0, np.max(np.abs(t_ref)))
        assert np.max(np.abs(tau[b] - t_ref)) < 2e-7 * scale, (b, tau[b], t_ref)


@pytest.mark.parametrize("n", [2, 7])
def test_mass_matrix_matches_kinetic_energy(n):
    ch = chain_n(n)
    q = states(3, n)["q"]
    Mo = oracle.mass_matrix(ch, q)
    for b in range(3):
        Mref = L.mass_matrix(ch, q[b])
        assert np.max(np.abs(Mo[b] - Mref)) < 1e-12 * np.max(np.abs(Mref))


def test_link_twists_match_lagrange():
    ch = chain_n(5)
    st = states(1, 5)
    _, V, _, _ = oracle.rnea_trace(ch, st["q"][0], st["qd"][0], st["qdd"][0])
    Vref = np.stack(L.link_twists(ch, st["q"][0], st["qd"][0]))
    assert np.max(np.abs(V - Vref)) < 1e-12 * max(1, np.max(np.abs(Vref)))


def test_external_wrench_is_jacobian_transpose():
    n = 5
    ch = chain_n(n)
    st = states(2, n)
    F = np.array([3.0, -1.5, 2.0, 0.4, -0.7, 0.25])
    t0 = oracle.rnea(ch, st["q"], st["qd"], st["qdd"], base())
    t1 = oracle.rnea(ch, st["q"], st["qd"], st["qdd"], base(F=F))
    for b in range(2):
        Jt = L.tip_jacobian(ch, st["q"][b])
        assert np.allclose(t1[b] - t0[b], Jt.T @ F, atol=1e-12, rtol=0)


def test_base_twist_equals_virtual_first_joint():
    """A moving base (V_0, dV_0) acts like a massless first joint at rest pose."""
    n = 4
    ch = chain_n(n)
    S1 = ch.S[0]
    st = states(3, n)
    Mz = np.zeros((1, 12))
    Mz[0, [0, 4, 8]] = 1.0
    virt = chaingen.Chain(np.vstack([Mz, ch.M]), np.vstack([S1, ch.S]),
                          np.vstack([np.zeros((1, 10)), ch.inertia]))
    qd1, qdd1 = 0.8, -1.3
    q_ext = np.hstack([np.zeros((3, 1)), st["q"]])
    qd_ext = np.hstack([np.full((3, 1), qd1), st["qd"]])
    qdd_ext = np.hstack([np.full((3, 1), qdd1), st["qdd"]])
    t_ext = oracle.rnea(virt, q_ext, qd_ext, qdd_ext)
    bs = base(V0=S1 * qd1, dV0=S1 * qdd1 + np.array([0, 0, G, 0, 0, 0]))
    t_sub = oracle.rnea(ch, st["q"], st["qd"], st["qdd"], bs)
    assert np.max(np.abs(t_ext[:, 1:] - t_sub)) < 1e-12 * np.max(np.abs(t_sub))


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("n", [1, 2, 7, 32, 100])
def test_mass_matrix_symmetric_positive_definite(n):
    ch = chain_n(n)
    q = states(3, n)["q"]
    Mq = oracle.mass_matrix(ch, q)
    for b in range(3):
        assert np.max(np.abs(Mq[b] - Mq[b].T)) < 1e-12 * np.max(np.abs(Mq[b]))
        assert np.linalg.eigvalsh(Mq[b]).min() > 0.0


@pytest.mark.parametrize("n", [2, 7, 32, 100])
def test_affine_in_qdd_quadratic_in_qd(n):
    ch = chain_n(n)
    st = states(3, n)
    z = np.zeros_like(st["q"])
    t_full = oracle.rnea(ch, st["q"], st["qd"], st["qdd"])
    t_bias = oracle.rnea(ch, st["q"], st["qd"], z)
    Mq = oracle.mass_matrix(ch, st["q"])
    lin = np.einsum("bij,bj->bi", Mq, st["qdd"])
    scale = np.max(np.abs(t_full))
    assert np.max(np.abs(t_full - t_bias - lin)) < 1e-11 * scale
    s = 1.7
    t_g = oracle.rnea(ch, st["q"], z, z)
    t_s = oracle.rnea(ch, st["q"], s * st["qd"], z)
    assert np.max(np.abs((t_s - t_g) - s * s * (t_bias - t_g))) < 1e-11 * scale


@pytest.mark.parametrize("n", [2, 7, 32])
def test_power_identity(n):
    """qd^T tau = d/dt (KE + PE) along q(t) = q + qd t + qdd t^2 / 2."""
    ch = chain_n(n)
    st = states(2, n)
    tau = oracle.rnea(ch, st["q"], st["qd"], st["qdd"])
    Mq = None
    h = 1e-4
    for b in range(2):
        q, qd, qdd = st["q"][b], st["qd"][b], st["qdd"][b]

        def energy(t):
            qt = q + qd * t + 0.5 * qdd * t * t
            qdt = qd + qdd * t
            Mt = oracle.mass_matrix(ch, qt[None])[0]
            return 0.5 * qdt @ Mt @ qdt + L.potential(ch, qt)

        dE = (energy(h) - energy(-h)) / (2 * h)
        power = qd @ tau[b]
        assert abs(power - dE) < 1e-6 * max(1.0, abs(power), np.max(np.abs(tau[b])))
    del Mq


# ------------------------------------------------- scan operators (Sec. III)

def fwd_operands(ch, q, qd, qdd, V0, dV0):
    """Compact operands (g, xi1, xi2) = (f^-1, S qdd, S qd) with A_0 = (I, dV0, V0)."""
    ops = [(np.eye(4), np.array(dV0, float), np.array(V0, float))]
    for i, f in enumerate(L.link_transforms(ch, q)):
        ops.append((np.linalg.inv(f), ch.S[i] * qdd[i], ch.S[i] * qd[i]))
    return ops


def oplus(a, b):
    """(g,x1,x2) (+) (g',x1',x2') = (g g', Ad_g x1' + x1 - ad_{x2} Ad_g x2', Ad_g x2' + x2)."""
    g, x1, x2 = a
    g2, y1, y2 = b
    A = L.Ad(g)
    return (g @ g2, A @ y1 + x1 - L.ad(x2) @ (A @ y2), A @ y2 + x2)


def A13(op):
    """The 13x13 matrix A_i of Eq. (scan-id-vel-acc)."""
    g, x1, x2 = op
    A = L.Ad(g)
    M = np.zeros((13, 13))
    M[0:6, 0:6] = A
    M[0:6, 6:12] = -L.ad(x2) @ A
    M[0:6, 12] = x1
    M[6:12, 6:12] = A
    M[6:12, 12] = x2
    M[12, 12] = 1.0
    return M


def all_bracketings(items, op):
    if len(items) == 1:
        yield items[0]
        return
    for k in range(1, len(items)):
        for left in all_bracketings(items[:k], op):
            for right in all_bracketings(items[k:], op):
                yield op(left, right)


def test_oplus_identity_and_inverse():
    ch = chain_n(3)
    st = states(1, 3)
    ops = fwd_operands(ch, st["q"][0], st["qd"][0], st["qdd"][0], np.zeros(6), np.zeros(6))
    e = (np.eye(4), np.zeros(6), np.zeros(6))
    for a in ops[1:]:
        g, x1, x2 = a
        gi = np.linalg.inv(g)
        inv = (gi, -L.Ad(gi) @ x1, -L.Ad(gi) @ x2)
        for lhs, rhs in ((oplus(a, e), a), (oplus(e, a), a), (oplus(a, inv), e), (oplus(inv, a), e)):
            for u, v in zip(lhs, rhs):
                assert np.allclose(u, v, atol=1e-13)


@pytest.mark.parametrize("n", [1, 2, 4, 6])
def test_forward_scan_all_bracketings_equal_serial(n):
    ch = chain_n(n)
    st = states(1, n, seed=21)
    q, qd, qdd = st["q"][0], st["qd"][0], st["qdd"][0]
    V0 = np.array([0.1, -0.2, 0.05, 0.3, -0.1, 0.2])
    dV0 = np.array([0.0, 0.4, G, -0.2, 0.1, 0.05])
    _, V, dV, _ = oracle.rnea_trace(ch, q, qd, qdd, base(V0=V0, dV0=dV0))
    ops = fwd_operands(ch, q, qd, qdd, V0, dV0)
    # the later link is the left operand: P_i = A_i (+) ... (+) A_1 (+) A_0
    seq = ops[::-1]
    count = 0
    for res in all_bracketings(seq, oplus):
        count += 1
        assert np.allclose(res[1], dV[-1], atol=1e-12)
        assert np.allclose(res[2], V[-1], atol=1e-12)
    catalan = [1, 1, 2, 5, 14, 42, 132, 429]
    assert count == catalan[n]
    # the 13x13 product gives every prefix
    P = np.eye(13)
    for i in range(n + 1):
        P = A13(ops[i]) @ P
        if i >= 1:
            x = P @ np.append(np.zeros(12), 1.0)
            assert np.allclose(x[0:6], dV[i - 1], atol=1e-12)
            assert np.allclose(x[6:12], V[i - 1], atol=1e-12)


@pytest.mark.parametrize("n", [1, 3, 6])
def test_backward_scan_matches_serial(n):
    """8x8 operands of Eq. (id-bkwd-scan) with F_hat from the twists; every bracketing."""
    ch = chain_n(n)
    st = states(1, n, seed=23)
    q, qd, qdd = st["q"][0], st["qd"][0], st["qdd"][0]
    Fext = np.array([0.5, 0.1, -0.3, 0.2, 0.0, -0.1])
    tau, V, dV, F = oracle.rnea_trace(ch, q, qd, qdd, base(F=Fext))
    fs = L.link_transforms(ch, q)
    Fhat = [L.spatial_inertia(ch.inertia[i]) @ dV[i]
            - L.ad(V[i]).T @ (L.spatial_inertia(ch.inertia[i]) @ V[i]) for i in range(n)]

    def op(i):  # (T, b): F_i = T F_{i+1} + b, T = Ad^T_{f_{i,i+1}^-1}
        T = np.eye(6) if i == n - 1 else L.Ad(np.linalg.inv(fs[i + 1])).T
        return (T, Fhat[i])

    def compose(a, b):  # a for the lower index
        return (a[0] @ b[0], a[0] @ b[1] + a[1])

    for i in range(n):
        seq = [op(k) for k in range(i, n)]
        for res in all_bracketings(seq, compose):
            Fi = res[0] @ Fext + res[1]
            assert np.allclose(Fi, F[i], atol=1e-11)
            assert abs(ch.S[i] @ Fi - tau[i]) < 1e-11


# ------------------------------------------------------- forward dynamics

@pytest.mark.parametrize("n", [1, 2, 7, 16])
def test_fd_aba_equals_jsiia_and_lagrange_solve(n):
    ch = chain_n(n)
    st = chaingen.make_states(4, n, seed=31, kinds=("q", "qd", "tau"))
    qa = oracle.fd_aba(ch, st["q"], st["qd"], st["tau"])
    qj, status = oracle.fd_jsiia(ch, st["q"], st["qd"], st["tau"])
    assert np.all(status == 0)
    assert oracle.rel_err(qa, qj) < 1e-9
    if n <= 7:
        z = np.zeros(n)
        for b in range(2):
            bias = oracle.rnea(ch, st["q"][b][None], st["qd"][b][None], z[None])[0]
            Mref = L.mass_matrix(ch, st["q"][b])
            ref = np.linalg.solve(Mref, st["tau"][b] - bias)
            assert np.max(np.abs(qa[b] - ref)) < 1e-9 * max(1, np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [2, 16, 64])
def test_fd_round_trip(n):
    ch = chain_n(n)
    st = chaingen.make_states(3, n, seed=37, kinds=("q", "qd", "tau"))
    qa = oracle.fd_aba(ch, st["q"], st["qd"], st["tau"])
    back = oracle.rnea(ch, st["q"], st["qd"], qa)
    assert oracle.rel_err(back, st["tau"]) < 1e-9


def test_abi_tip_and_omega():
    """hat J_n = J_n; Omega_i = S_i^T hat J_i S_i > 0; hat J symmetric PSD."""
    ch = chain_n(6)
    q = states(1, 6)["q"][0]
    Jh, Om = oracle.abi_trace(ch, q)
    assert np.allclose(Jh[-1], L.spatial_inertia(ch.inertia[-1]), atol=1e-13)
    assert np.all(Om > 0)
    for i in range(6):
        assert np.allclose(Jh[i], Jh[i].T, atol=1e-12)
        assert np.linalg.eigvalsh(Jh[i]).min() > -1e-12
        assert abs(ch.S[i] @ Jh[i] @ ch.S[i] - Om[i]) < 1e-12


@pytest.mark.parametrize("n", [1, 2, 5, 9])
def test_abi_omega_is_the_schur_complement_of_the_mass_matrix(n):
    """Omega_i of Eq. (abi) is the inertia joint i feels with the joints above it
    free and those below it locked: the Schur complement of M[i+1:, i+1:] in
    M[i:, i:] (the pivots of M's factorisation eliminated tip first). M(q) comes
    from unit-acceleration IDs, pinned against the Lagrangian restatement."""
    ch = chain_n(n)
    for q in states(3, n)["q"]:
        _, Om = oracle.abi_trace(ch, q)
        Mq = oracle.mass_matrix(ch, q)[0]
        for i in range(n):
            a = Mq[i, i]
            if i + 1 < n:
                c = Mq[i + 1:, i]
                a -= c @ np.linalg.solve(Mq[i + 1:, i + 1:], c)
            assert abs(Om[i] - a) <= 1e-11 * Mq[i, i], (n, i, Om[i], a)


def test_fd_single_link_closed_form():
    m, l, Ixx = 1.7, 0.45, 0.03
    ch = chaingen.pendulum(m, l, Ixx)
    q = np.array([[0.4], [-1.1]])
    qd = np.array([[0.3], [2.0]])
    tau = np.array([[1.0], [-3.0]])
    qdd = oracle.fd_aba(ch, q, qd, tau)
    expect = (tau - m * G * l * np.sin(q)) / (m * l * l + Ixx)
    assert np.allclose(qdd, expect, atol=1e-13)


# ------------------------------------------------------------- gradients

@pytest.mark.parametrize("n", [1, 3, 7])
def test_complex_step_gradient_vs_central_difference(n):
    ch = chain_n(n)
    st = chaingen.make_states(2, n, seed=41, kinds=("q", "qd", "qdd", "w"))
    gq, gqd, gqdd = oracle.rnea_grad(ch, st["q"], st["qd"], st["qdd"], st["w"])
    h = 1e-6
    for k, g in (("q", gq), ("qd", gqd), ("qdd", gqdd)):
        fd = np.empty_like(g)
        for j in range(n):
            plus = {x: st[x].copy() for x in ("q", "qd", "qdd")}
            minus = {x: st[x].copy() for x in ("q", "qd", "qdd")}
            plus[k][:, j] += h
            minus[k][:, j] -= h
            tp = oracle.rnea(ch, plus["q"], plus["qd"], plus["qdd"])
            tm = oracle.rnea(ch, minus["q"], minus["qd"], minus["qdd"])
            fd[:, j] = np.sum(st["w"] * (tp - tm), axis=1) / (2 * h)
        scale = max(1.0, np.max(np.abs(g)))
        assert np.max(np.abs(g - fd)) < 1e-7 * scale, k


@pytest.mark.parametrize("n", [2, 7, 32])
def test_gradient_wrt_qdd_is_mass_matrix_times_w(n):
    ch = chain_n(n)
    st = chaingen.make_states(2, n, seed=43, kinds=("q", "qd", "qdd", "w"))
    _, _, gqdd = oracle.rnea_grad(ch, st["q"], st["qd"], st["qdd"], st["w"])
    Mq = oracle.mass_matrix(ch, st["q"])
    ref = np.einsum("bij,bj->bi", Mq, st["w"])
    assert np.max(np.abs(gqdd - ref)) < 1e-12 * np.max(np.abs(ref))


def test_gradient_wrt_qd_from_lagrange_qd_only():
    """For qdd = 0 and no gravity, w^T tau = w^T C(q,qd) qd is quadratic in qd:
    d/dqd (w^T tau) . qd = 2 w^T tau (Euler's theorem for homogeneous functions)."""
    n = 5
    ch = chain_n(n)
    st = chaingen.make_states(2, n, seed=47, kinds=("q", "qd", "w"))
    z = np.zeros_like(st["q"])
    b = base(dV0=np.zeros(6))
    _, gqd, _ = oracle.rnea_grad(ch, st["q"], st["qd"], z, st["w"], b)
    tau = oracle.rnea(ch, st["q"], st["qd"], z, b)
    lhs = np.sum(gqd * st["qd"], axis=1)
    rhs = 2 * np.sum(st["w"] * tau, axis=1)
    assert np.allclose(lhs, rhs, rtol=1e-11, atol=1e-12)
