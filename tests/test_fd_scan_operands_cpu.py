"""The scan form of forward dynamics (Sec. III-D), pinned on the host before
any kernel uses it.

With links 0..n-1, X_k = Ad_{f_{k-1,k}^-1}, the articulated inertias hat J_k
and Omega_k = S_k^T hat J_k S_k of Eq. (abi), and
    Y_k  = X_{k+1}^T (I - hat J_{k+1} S_{k+1} S_{k+1}^T / Omega_{k+1}),
    Pi_k = X_{k+1}^T hat J_{k+1} S_{k+1} / Omega_{k+1}
(Sec. II-B; for k = -1 they use link 0's transform X_0), the recursions of
Eq. (recursive-fd) are the products of these operands:

* backward, Eq. (fd-bkwd-scan), state (z_k, c_{k+1}, 1), 8 x 8:
      [[Y_k, 0, Pi_k tau_hat_{k+1}],
       [-S_{k+1}^T / Omega_{k+1}, 0, tau_hat_{k+1} / Omega_{k+1}],
       [0, 0, 1]]
  applied from (z_{n-1}, c_n) = 0, for k = n-2 .. -1 (the factor on the tau_hat
  column is Omega^-1: the printed Omega is read as its inverse, since
  c_hat = Omega^-1 (tau_hat - S^T z_hat));
* forward, Eq. (fd-fwd-scan), state (lambda_k, qdd_k, 1), 8 x 8:
      [[Y_{k-1}^T, 0, S_k c_k], [-Pi_{k-1}^T, 0, c_k], [0, 0, 1]]
  applied from (lambda_{-1}, qdd_{-1}) = 0, for k = 0 .. n-1;
* the fused backward, Eq. (fd-bkwd-scan-large), state (F_{k-1}, tau_hat_k,
  z_k, c_{k+1}, 1), 15 x 15:
      [[X_k^T, 0, 0, 0, F_hat_{k-1}],
       [-S_k^T, 0, 0, 0, tau_k],
       [0, Pi_k, Y_k, 0, 0],
       [0, 1 / Omega_{k+1}, -S_{k+1}^T / Omega_{k+1}, 0, 0],
       [0, 0, 0, 0, 1]]
  applied from (F_{n-1}, 0, 0, 0, 1), for k = n-1 .. -1 (the blocks that name
  link n, or F_hat_{-1}, are zero).

Pins: the serial application of these operands reproduces the oracle's
forward dynamics (fd_aba), its bias wrenches and tau_hat = tau - tau_bias;
every bracketing of the products gives the same states; and the segmented
scan the GPU kernel uses (affine maps z -> M z + v, K links per lane, a suffix
or prefix combine across lanes, then a replay) equals the serial values.
Y, Pi, X and the bias wrenches are formed here from lagrange_ref's Ad, ad and
matrix-exponential poses; hat J and Omega come from the oracle.
"""
import numpy as np
import pytest

import chaingen
import lagrange_ref as L
import oracle

BASE = np.array([0.1, -0.2, 0.05, 0.3, -0.1, 0.2, 0.2, 0.4, 9.81, -0.2, 0.1, 0.05,
                 0.5, 0.1, -0.3, 0.2, 0.0, -0.1])


def _instance(n, seed, base=BASE):
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED + 13 * n + seed)
    st = chaingen.make_states(1, n, seed=seed, kinds=("q", "qd", "tau"))
    q, qd, tau = (st[k][0] for k in ("q", "qd", "tau"))
    X = [L.Ad(np.linalg.inv(f)) for f in L.link_transforms(ch, q)]
    Jh, Om = oracle.abi_trace(ch, q)
    S = [np.asarray(ch.S[k], dtype=np.float64) for k in range(n)]
    tau_bias, V, dV, F = oracle.rnea_trace(ch, q, qd, np.zeros(n), base)
    J = [L.spatial_inertia(ch.inertia[k]) for k in range(n)]
    Fhat = [J[k] @ dV[k] - L.ad(V[k]).T @ (J[k] @ V[k]) for k in range(n)]
    Y, Pi = {}, {}
    for k in range(-1, n - 1):
        U = Jh[k + 1] @ S[k + 1]
        Y[k] = X[k + 1].T @ (np.eye(6) - np.outer(U, S[k + 1]) / Om[k + 1])
        Pi[k] = X[k + 1].T @ U / Om[k + 1]
    return dict(ch=ch, n=n, q=q, qd=qd, tau=tau, X=X, Jh=Jh, Om=Om, S=S, F=F, Fhat=Fhat,
                That=tau - tau_bias, Y=Y, Pi=Pi, base=base)


def _bwd8(d, k):
    A = np.zeros((8, 8))
    A[:6, :6] = d["Y"][k]
    A[:6, 7] = d["Pi"][k] * d["That"][k + 1]
    A[6, :6] = -d["S"][k + 1] / d["Om"][k + 1]
    A[6, 7] = d["That"][k + 1] / d["Om"][k + 1]
    A[7, 7] = 1.0
    return A


def _fwd8(d, k, chat):
    B = np.zeros((8, 8))
    B[:6, :6] = d["Y"][k - 1].T
    B[:6, 7] = d["S"][k] * chat[k]
    B[6, :6] = -d["Pi"][k - 1]
    B[6, 7] = chat[k]
    B[7, 7] = 1.0
    return B


def _bwd15(d, k):
    n = d["n"]
    C = np.zeros((15, 15))
    if k >= 0:
        C[0:6, 0:6] = d["X"][k].T
        C[0:6, 14] = d["Fhat"][k - 1] if k >= 1 else 0.0
        C[6, 0:6] = -d["S"][k]
        C[6, 14] = d["tau"][k]
    if k + 1 < n:
        C[7:13, 6] = d["Pi"][k]
        C[7:13, 7:13] = d["Y"][k]
        C[13, 6] = 1.0 / d["Om"][k + 1]
        C[13, 7:13] = -d["S"][k + 1] / d["Om"][k + 1]
    C[14, 14] = 1.0
    return C


def _serial_fd(d):
    """c_hat and qdd from the 8 x 8 operands applied one at a time."""
    n = d["n"]
    s = np.zeros(8)
    s[7] = 1.0
    chat = np.zeros(n)
    for k in range(n - 2, -2, -1):
        s = _bwd8(d, k) @ s
        chat[k + 1] = s[6]
    chat[n - 1] = d["That"][n - 1] / d["Om"][n - 1]
    t = np.zeros(8)
    t[7] = 1.0
    qdd = np.zeros(n)
    for k in range(n):
        t = _fwd8(d, k, chat) @ t
        qdd[k] = t[6]
    return chat, qdd


def _last_wrench(d):
    """F_{n-1} = F_hat_{n-1} + the end wrench (given in frame n-1)."""
    return d["Fhat"][d["n"] - 1] + d["base"][12:18]


def _all_products(ms):
    """Every bracketing of the product ms[0] @ ms[1] @ ... (recursive split)."""
    if len(ms) == 1:
        return [ms[0]]
    out = []
    for cut in range(1, len(ms)):
        for a in _all_products(ms[:cut]):
            for b in _all_products(ms[cut:]):
                out.append(a @ b)
    return out


@pytest.mark.parametrize("n,seed", [(1, 1), (2, 2), (3, 3), (7, 4), (16, 5)])
def test_8x8_operands_reproduce_the_oracles_forward_dynamics(n, seed):
    d = _instance(n, seed)
    _, qdd = _serial_fd(d)
    ref = oracle.fd_aba(d["ch"], d["q"][None], d["qd"][None], d["tau"][None], base=d["base"])[0]
    assert np.max(np.abs(qdd - ref)) <= 1e-10 * np.max(np.abs(ref))


@pytest.mark.parametrize("n,seed", [(1, 1), (2, 2), (5, 3), (16, 6)])
def test_15x15_operand_reproduces_bias_wrenches_tau_hat_and_c_hat(n, seed):
    d = _instance(n, seed)
    chat, _ = _serial_fd(d)
    r = np.zeros(15)
    r[0:6] = _last_wrench(d)
    r[14] = 1.0
    for k in range(n - 1, -2, -1):
        r = _bwd15(d, k) @ r
        if k >= 1:  # F_{k-1}
            assert np.allclose(r[0:6], d["F"][k - 1], rtol=0, atol=1e-10 * np.max(np.abs(d["F"])))
        if k >= 0:
            assert abs(r[6] - d["That"][k]) <= 1e-10 * np.max(np.abs(d["That"]))
        if k + 1 < n:
            assert abs(r[13] - chat[k + 1]) <= 1e-10 * np.max(np.abs(chat))


@pytest.mark.parametrize("n", [3, 5])
def test_every_bracketing_of_the_8x8_products_agrees(n):
    d = _instance(n, 7)
    chat, qdd = _serial_fd(d)
    s0 = np.zeros(8)
    s0[7] = 1.0
    bwd = [_bwd8(d, k) for k in range(-1, n - 1)]  # A_{-1} A_0 ... A_{n-2}
    for P in _all_products(bwd):
        assert abs((P @ s0)[6] - chat[0]) <= 1e-12 * np.max(np.abs(chat))
    fwd = [_fwd8(d, k, chat) for k in range(n - 1, -1, -1)]  # B_{n-1} ... B_0
    for P in _all_products(fwd):
        assert abs((P @ s0)[6] - qdd[n - 1]) <= 1e-12 * np.max(np.abs(qdd))


def test_every_bracketing_of_the_15x15_product_agrees():
    n = 4
    d = _instance(n, 8)
    chat, _ = _serial_fd(d)
    r0 = np.zeros(15)
    r0[0:6] = _last_wrench(d)
    r0[14] = 1.0
    ops = [_bwd15(d, k) for k in range(-1, n)]  # C_{-1} C_0 ... C_{n-1}
    for P in _all_products(ops):
        r = P @ r0
        assert abs(r[13] - chat[0]) <= 1e-12 * np.max(np.abs(chat))
        assert abs(r[6]) <= 1e-12 * np.max(np.abs(d["That"]))  # tau_hat_{-1} = 0


def _step_z(d, k, z):
    """z_{k-1} from z_k with link k's data: X_k^T (z + U_k (tau_hat_k - S_k^T z) / Omega_k)."""
    U = d["Jh"][k] @ d["S"][k]
    return d["X"][k].T @ (z + U * (d["That"][k] - d["S"][k] @ z) / d["Om"][k])


def _affine_of_segment(d, lo, hi):
    """(M, v) with z_{lo-1} = M z_{hi-1} + v, links hi-1 .. lo applied."""
    M, v = np.eye(6), np.zeros(6)
    for k in range(hi - 1, lo - 1, -1):
        U = d["Jh"][k] @ d["S"][k]
        Lk = d["X"][k].T @ (np.eye(6) - np.outer(U, d["S"][k]) / d["Om"][k])
        ck = d["X"][k].T @ U * d["That"][k] / d["Om"][k]
        M, v = Lk @ M, Lk @ v + ck
    return M, v


@pytest.mark.parametrize("n,K,lanes", [(7, 1, 8), (16, 2, 8), (29, 4, 8), (32, 1, 32),
                                       (64, 2, 32), (100, 4, 32)])
def test_segmented_z_scan_equals_the_serial_recursion(n, K, lanes):
    """The kernel's backward scan: lane l owns links [l K, l K + K); its element
    is the affine map of its segment, z_{lK-1} = M z_{lK+K-1} + v; an inclusive
    suffix combine across lanes ((M, v) o (M', v') = (M M', M v' + v), lower
    o upper) gives each lane the value z_{e-1} entering it from above (that of
    lane l+1's suffix); a replay gives c_hat_k = (tau_hat_k - S_k^T z_k) /
    Omega_k for its links."""
    d = _instance(n, 9)
    chat_ref, _ = _serial_fd(d)
    elems = []
    for l in range(lanes):
        lo, hi = min(l * K, n), min(l * K + K, n)
        elems.append(_affine_of_segment(d, lo, hi))
    suffix = [None] * lanes
    acc = (np.eye(6), np.zeros(6))
    for l in range(lanes - 1, -1, -1):
        M, v = elems[l]
        acc = (M @ acc[0], M @ acc[1] + v)
        suffix[l] = acc
    chat = np.zeros(n)
    for l in range(lanes):
        lo, hi = min(l * K, n), min(l * K + K, n)
        z = suffix[l + 1][1] if l + 1 < lanes else np.zeros(6)  # z_{n-1} = 0 at the tip
        for k in range(hi - 1, lo - 1, -1):
            chat[k] = (d["That"][k] - d["S"][k] @ z) / d["Om"][k]
            z = _step_z(d, k, z)
    assert np.max(np.abs(chat - chat_ref)) <= 1e-10 * np.max(np.abs(chat_ref))


@pytest.mark.parametrize("n,K,lanes", [(7, 1, 8), (29, 4, 8), (64, 2, 32), (100, 4, 32)])
def test_segmented_lambda_scan_equals_the_serial_recursion(n, K, lanes):
    """The kernel's forward scan: a_k = X_k lambda_{k-1}, qdd_k = c_hat_k -
    U_k^T a_k / Omega_k, lambda_k = a_k + S_k qdd_k, as affine maps lambda ->
    N lambda + u per segment; an inclusive prefix combine ((N, u) after
    (N', u'): (N N', N u' + u), later on the left) and a replay."""
    d = _instance(n, 10)
    chat, qdd_ref = _serial_fd(d)

    def step(k, lam):
        a = d["X"][k] @ lam
        U = d["Jh"][k] @ d["S"][k]
        qk = chat[k] - U @ a / d["Om"][k]
        return a + d["S"][k] * qk, qk

    elems = []
    for l in range(lanes):
        lo, hi = min(l * K, n), min(l * K + K, n)
        N, u = np.eye(6), np.zeros(6)
        for k in range(lo, hi):
            U = d["Jh"][k] @ d["S"][k]
            Lk = (np.eye(6) - np.outer(d["S"][k], U) / d["Om"][k]) @ d["X"][k]
            N, u = Lk @ N, Lk @ u + d["S"][k] * chat[k]
        elems.append((N, u))
    prefix = []
    acc = (np.eye(6), np.zeros(6))
    for l in range(lanes):
        N, u = elems[l]
        acc = (N @ acc[0], N @ acc[1] + u)
        prefix.append(acc)
    qdd = np.zeros(n)
    for l in range(lanes):
        lo, hi = min(l * K, n), min(l * K + K, n)
        lam = prefix[l - 1][1] if l > 0 else np.zeros(6)
        for k in range(lo, hi):
            lam, qdd[k] = step(k, lam)
    assert np.max(np.abs(qdd - qdd_ref)) <= 1e-10 * np.max(np.abs(qdd_ref))
