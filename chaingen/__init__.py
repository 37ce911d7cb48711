"""Seeded synthetic serial chains and joint states.

This module only draws random numbers and packs them into arrays. It holds
none of the dynamics arithmetic: both the CUDA path and the FP64 oracle take
its arrays as inputs, and neither imports the other.

The recipe follows the random-robot set-up of the experiments (Sec. V: joint
twists drawn at random, joint inputs randomised on every repetition):

* home transform M_i (frame i -> frame i-1): rotation uniform on SO(3)
  (normalised Gaussian quaternion), translation U[0.1, 0.5] m per axis;
* joint twist S_i = (v, w) expressed in frame i, linear part first:
  w uniform on the unit sphere, a point r ~ U[-0.1, 0.1]^3 m on the axis,
  v = -w x r (a pure revolute joint through r);
* link inertia: mass U[0.5, 5] kg, centre of mass c ~ U[-0.1, 0.1]^3 m in
  frame i, rotational inertia about the centre of mass
  R diag(d2+d3, d1+d3, d1+d2) R^T with d_k ~ U[0.001, 0.05] * m and R uniform
  on SO(3), so the principal moments satisfy the triangle inequality;
* joint states: q ~ U[-pi, pi], qd ~ N(0, 1), qdd ~ N(0, 2), tau ~ N(0, 10),
  adjoint weights w ~ N(0, 1) (second argument = standard deviation).

Array layouts (all float64, C order):

* ``M``: [n, 12] = row-major 3x3 rotation then the translation (3);
* ``S``: [n, 6] = (v_x, v_y, v_z, w_x, w_y, w_z);
* ``inertia``: [n, 10] = (m, c_x, c_y, c_z, I_xx, I_yy, I_zz, I_xy, I_xz,
  I_yz), the rotational inertia taken about the centre of mass in frame i;
* joint states: [B, n].
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 1609

__all__ = [
    "BASE_SEED",
    "Chain",
    "make_chain",
    "make_states",
    "uniform_rotation",
    "pendulum",
    "planar_two_link",
    "uneven_requests",
]


class Chain:
    """Model arrays of one serial chain of n revolute joints."""

    def __init__(self, M, S, inertia):
        self.M = np.ascontiguousarray(M, dtype=np.float64)
        self.S = np.ascontiguousarray(S, dtype=np.float64)
        self.inertia = np.ascontiguousarray(inertia, dtype=np.float64)
        self.n = int(self.M.shape[0])
        assert self.M.shape == (self.n, 12)
        assert self.S.shape == (self.n, 6)
        assert self.inertia.shape == (self.n, 10)

    def sub(self, lo, hi):
        return Chain(self.M[lo:hi], self.S[lo:hi], self.inertia[lo:hi])


def uniform_rotation(rng, count):
    """Rotations uniform on SO(3): normalised Gaussian quaternions."""
    qv = rng.standard_normal((count, 4))
    qv /= np.linalg.norm(qv, axis=1, keepdims=True)
    w, x, y, z = qv[:, 0], qv[:, 1], qv[:, 2], qv[:, 3]
    R = np.empty((count, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def make_chain(n, seed=BASE_SEED, rng=None):
    """Random n-link chain drawn from ``rng`` (or a fresh PCG64 at ``seed``)."""
    if rng is None:
        rng = np.random.default_rng(seed)
    n = int(n)
    RM = uniform_rotation(rng, n)
    pM = rng.uniform(0.1, 0.5, size=(n, 3))
    M = np.concatenate([RM.reshape(n, 9), pM], axis=1)

    w = rng.standard_normal((n, 3))
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    r = rng.uniform(-0.1, 0.1, size=(n, 3))
    v = -np.cross(w, r)
    S = np.concatenate([v, w], axis=1)

    m = rng.uniform(0.5, 5.0, size=n)
    c = rng.uniform(-0.1, 0.1, size=(n, 3))
    d = rng.uniform(0.001, 0.05, size=(n, 3)) * m[:, None]
    principal = np.stack([d[:, 1] + d[:, 2], d[:, 0] + d[:, 2], d[:, 0] + d[:, 1]], axis=1)
    RI = uniform_rotation(rng, n)
    Ic = np.einsum("nij,nj,nkj->nik", RI, principal, RI)
    inertia = np.stack(
        [m, c[:, 0], c[:, 1], c[:, 2],
         Ic[:, 0, 0], Ic[:, 1, 1], Ic[:, 2, 2], Ic[:, 0, 1], Ic[:, 0, 2], Ic[:, 1, 2]],
        axis=1)
    return Chain(M, S, inertia)


def make_states(B, n, seed=BASE_SEED + 7919, rng=None, kinds=("q", "qd", "qdd")):
    """Joint-state batch [B, n] per requested kind, float64."""
    if rng is None:
        rng = np.random.default_rng(seed)
    out = {}
    for k in kinds:
        if k == "q":
            out[k] = rng.uniform(-np.pi, np.pi, size=(B, n))
        elif k == "qd":
            out[k] = rng.normal(0.0, 1.0, size=(B, n))
        elif k == "qdd":
            out[k] = rng.normal(0.0, 2.0, size=(B, n))
        elif k == "tau":
            out[k] = rng.normal(0.0, 10.0, size=(B, n))
        elif k == "w":
            out[k] = rng.normal(0.0, 1.0, size=(B, n))
        else:
            raise ValueError(f"unknown state kind {k!r}")
    return out


def pendulum(mass, length, Ixx=0.0):
    """One link on a joint about x through the origin, centre of mass at (0,0,-l).

    Hangs straight down at q = 0 when gravity points along -z.
    """
    M = np.zeros((1, 12))
    M[0, [0, 4, 8]] = 1.0
    S = np.array([[0.0, 0.0, 0.0, 1.0, 0.0, 0.0]])
    inertia = np.array([[mass, 0.0, 0.0, -length, Ixx, 0.0, 0.0, 0.0, 0.0, 0.0]])
    return Chain(M, S, inertia)


def planar_two_link(m1, m2, l1, lc1, lc2, I1, I2):
    """Two links on parallel z axes; link 2's joint sits l1 along link 1's x axis."""
    M = np.zeros((2, 12))
    M[:, [0, 4, 8]] = 1.0
    M[1, 9] = l1
    S = np.array([[0.0, 0.0, 0.0, 0.0, 0.0, 1.0]] * 2)
    inertia = np.array([
        [m1, lc1, 0.0, 0.0, I1, I1, I1, 0.0, 0.0, 0.0],
        [m2, lc2, 0.0, 0.0, I2, I2, I2, 0.0, 0.0, 0.0],
    ])
    return Chain(M, S, inertia)


def uneven_requests(count, n_lo=6, n_hi=100, fd_fraction=0.2, seed=BASE_SEED):
    """Mixed request list: per request its own chain from seed ``seed + k``.

    Returns a list of dicts {n, chain, kind ('id'|'fd')}; the request kinds and
    link counts are drawn from a separate PCG64 stream at ``seed``.
    """
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    kinds = np.where(rng.random(count) < fd_fraction, "fd", "id")
    reqs = []
    for k in range(count):
        reqs.append({"n": int(ns[k]), "chain": make_chain(int(ns[k]), seed=seed + k),
                     "kind": str(kinds[k])})
    return reqs
