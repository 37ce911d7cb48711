"""The algebra of a lane-parallel adjoint of inverse dynamics, checked on the
host before any kernel uses it.

Reverse mode through Eqs. (id-forward) and (id-backward), with G_i = Ad_{f_i^-1}
(f_i maps frame i to frame i-1) and the loss w^T tau:

* forward, base -> tip, beside V and dV: Fb_i = G_i Fb_{i-1} + S_i w_i;
* backward, tip -> base, the state y_i = (F_i, dVbar_i, Vbar_i) is affine in
  y_{i+1}: y_i = M(G_{i+1}, S_{i+1} qd_{i+1}) y_{i+1} + c_i with
  M(A, X) = [[A^T, 0, 0], [0, A^T, 0], [0, -A^T ad_X^T, A^T]] and the local
  seeds c_i = (F_hat_i, J Fb_i, ad_Fb^T J V - J ad_V Fb);
* gradients: gqdd = S^T dVbar, gqd = S^T Vbar - <dVbar, ad_S V>,
  gq = -<Vbar, ad_S V> - <dVbar, ad_S dV> - <F, ad_S Fb>.

A segment of consecutive links is one element (A, X, c): M(A_lo, X_lo) M(A_hi,
X_hi) = M(A_hi A_lo, A_hi X_lo + X_hi), because Ad_g ad_x Ad_g^-1 = ad_{Ad_g x},
and c = M(A_lo, X_lo) c_hi + c_lo. The forward side carries Fb as a third
channel of the scan element of Sec. III-B that composes like V without the ad
term. The tests check the serial formulas against the oracle's complex-step
gradient, the closed form of the composition against 18 x 18 products, and
that every bracketing of both scans reproduces the serial values.
"""
import numpy as np
import pytest

import chaingen
import lagrange_ref as L
import oracle

G0 = 9.81


def _setup(n, seed):
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED + 11 * n)
    st = chaingen.make_states(1, n, seed=seed, kinds=("q", "qd", "qdd", "w"))
    V0 = np.array([0.1, -0.2, 0.05, 0.3, -0.1, 0.2])
    dV0 = np.array([0.2, 0.4, G0, -0.2, 0.1, 0.05])
    Fext = np.array([0.5, 0.1, -0.3, 0.2, 0.0, -0.1])
    base = np.concatenate([V0, dV0, Fext])
    return ch, {k: v[0] for k, v in st.items()}, base


def _serial(ch, s, base):
    n = ch.n
    G = [L.Ad(np.linalg.inv(f)) for f in L.link_transforms(ch, s["q"])]
    J = [L.spatial_inertia(ch.inertia[i]) for i in range(n)]
    V, dV, Fb = [], [], []
    v, a, fb = base[0:6], base[6:12], np.zeros(6)
    for i in range(n):
        u = ch.S[i] * s["qd"][i]
        gv = G[i] @ v
        a = G[i] @ a + ch.S[i] * s["qdd"][i] - L.ad(u) @ gv
        v = gv + u
        fb = G[i] @ fb + ch.S[i] * s["w"][i]
        V.append(v), dV.append(a), Fb.append(fb)
    c = []
    for i in range(n):
        Fhat = J[i] @ dV[i] - L.ad(V[i]).T @ (J[i] @ V[i])
        dVl = J[i] @ Fb[i]
        Vl = L.ad(Fb[i]).T @ (J[i] @ V[i]) - J[i] @ (L.ad(V[i]) @ Fb[i])
        c.append(np.concatenate([Fhat, dVl, Vl]))
    elems = []
    for i in range(n):
        if i == n - 1:
            A, X = np.eye(6), np.zeros(6)
        else:
            A, X = G[i + 1], ch.S[i + 1] * s["qd"][i + 1]
        elems.append((A, X, c[i]))
    y_top = np.concatenate([base[12:18], np.zeros(12)])
    ys = [None] * n
    y = y_top
    for i in range(n - 1, -1, -1):
        A, X, ci = elems[i]
        y = M18(A, X) @ y + ci
        ys[i] = y
    return G, V, dV, Fb, elems, y_top, ys


def M18(A, X):
    M = np.zeros((18, 18))
    M[0:6, 0:6] = A.T
    M[6:12, 6:12] = A.T
    M[12:18, 6:12] = -A.T @ L.ad(X).T
    M[12:18, 12:18] = A.T
    return M


def compose(lo, hi):
    """One element for the links of lo followed (above) by those of hi."""
    A_lo, X_lo, c_lo = lo
    A_hi, X_hi, c_hi = hi
    return (A_hi @ A_lo, A_hi @ X_lo + X_hi, M18(A_lo, X_lo) @ c_hi + c_lo)


def _gradients(ch, V, dV, Fb, ys):
    n = ch.n
    gq, gqd, gqdd = np.empty(n), np.empty(n), np.empty(n)
    for i in range(n):
        S = ch.S[i]
        F, dVb, Vb = ys[i][0:6], ys[i][6:12], ys[i][12:18]
        gqdd[i] = S @ dVb
        gqd[i] = S @ Vb - dVb @ (L.ad(S) @ V[i])
        gq[i] = -(Vb @ (L.ad(S) @ V[i])) - dVb @ (L.ad(S) @ dV[i]) - F @ (L.ad(S) @ Fb[i])
    return gq, gqd, gqdd


def _all_bracketings(items, op):
    if len(items) == 1:
        yield items[0]
        return
    for k in range(1, len(items)):
        for left in _all_bracketings(items[:k], op):
            for right in _all_bracketings(items[k:], op):
                yield op(left, right)


@pytest.mark.parametrize("n", [1, 2, 5, 9])
def test_serial_adjoint_formulas_match_the_oracle_gradient(n):
    ch, s, base = _setup(n, seed=61)
    _, V, dV, Fb, _, _, ys = _serial(ch, s, base)
    tau, Vo, dVo, Fo = oracle.rnea_trace(ch, s["q"], s["qd"], s["qdd"], base)
    assert np.allclose(np.array(V), Vo, atol=1e-12) and np.allclose(np.array(dV), dVo, atol=1e-12)
    assert np.allclose(np.array([y[0:6] for y in ys]), Fo, atol=1e-11)
    got = np.concatenate(_gradients(ch, V, dV, Fb, ys))
    ref = np.concatenate([g[0] for g in oracle.rnea_grad(
        ch, s["q"][None], s["qd"][None], s["qdd"][None], s["w"][None], base=base)])
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_structured_composition_equals_the_matrix_product():
    ch, s, base = _setup(4, seed=62)
    _, _, _, _, elems, _, _ = _serial(ch, s, base)
    for lo, hi in ((elems[0], elems[1]), (elems[1], elems[2]), (elems[2], elems[3])):
        A, X, _ = compose(lo, hi)
        lhs = M18(A, X)
        rhs = M18(lo[0], lo[1]) @ M18(hi[0], hi[1])
        assert np.allclose(lhs, rhs, atol=1e-12)


@pytest.mark.parametrize("n", [1, 3, 5])
def test_backward_segments_every_bracketing_gives_the_serial_state(n):
    ch, s, base = _setup(n, seed=63)
    _, _, _, _, elems, y_top, ys = _serial(ch, s, base)
    for i in range(n):
        count = 0
        for A, X, c in _all_bracketings(elems[i:], compose):
            y = M18(A, X) @ y_top + c
            assert np.allclose(y, ys[i], atol=1e-10 * max(1.0, np.max(np.abs(ys[i]))))
            count += 1
        assert count == [1, 1, 2, 5, 14, 42][n - i - 1]  # Catalan(k - 1) for k elements


def oplus3(a, b):
    """The forward element of Sec. III-B with Fb as a third channel:
    (g, x1, x2, x3) (+) (g', y1, y2, y3) =
    (g g', Ad_g y1 + x1 - ad_x2 Ad_g y2, Ad_g y2 + x2, Ad_g y3 + x3)."""
    g, x1, x2, x3 = a
    g2, y1, y2, y3 = b
    A = L.Ad(g)
    return (g @ g2, A @ y1 + x1 - L.ad(x2) @ (A @ y2), A @ y2 + x2, A @ y3 + x3)


@pytest.mark.parametrize("n", [1, 3, 5])
def test_forward_scan_with_the_adjoint_weight_channel(n):
    ch, s, base = _setup(n, seed=64)
    _, V, dV, Fb, _, _, _ = _serial(ch, s, base)
    fs = L.link_transforms(ch, s["q"])
    ops = [(np.eye(4), base[6:12].copy(), base[0:6].copy(), np.zeros(6))]
    for i, f in enumerate(fs):
        ops.append((np.linalg.inv(f), ch.S[i] * s["qdd"][i], ch.S[i] * s["qd"][i],
                    ch.S[i] * s["w"][i]))
    seq = ops[::-1]  # the later link is the left operand
    for res in _all_bracketings(seq, oplus3):
        assert np.allclose(res[1], dV[-1], atol=1e-11)
        assert np.allclose(res[2], V[-1], atol=1e-12)
        assert np.allclose(res[3], Fb[-1], atol=1e-12)
