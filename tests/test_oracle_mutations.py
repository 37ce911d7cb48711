"""The oracle's pins catch plausible mistakes.

Each case compiles a copy of the oracle with one planted mistake (a dropped
term, a flipped sign, an off-by-one index, a transposed operand) into a
temporary folder, routes the oracle module to it, and requires that at least
one of the independent pin checks fails. The unmodified oracle must pass all
of them. Mistakes are planted only in the CPU oracle.
"""
import numpy as np
import pytest

import chaingen
import oracle
import lagrange_ref as L

G = 9.81


def _chain(n):
    return chaingen.make_chain(n, seed=chaingen.BASE_SEED)


def check_pendulum():
    m, l, Ixx = 1.7, 0.45, 0.03
    ch = chaingen.pendulum(m, l, Ixx)
    q = np.array([[0.4], [-1.1]])
    qd = np.array([[0.3], [2.0]])
    qdd = np.array([[1.5], [-0.5]])
    tau = oracle.rnea(ch, q, qd, qdd)
    return np.allclose(tau, (m * l * l + Ixx) * qdd + m * G * l * np.sin(q), atol=1e-12)


def check_lagrange():
    ch = _chain(3)
    st = chaingen.make_states(2, 3, seed=11)
    tau = oracle.rnea(ch, st["q"], st["qd"], st["qdd"])
    for b in range(2):
        ref, _ = L.torques(ch, st["q"][b], st["qd"][b], st["qdd"][b])
        if np.max(np.abs(tau[b] - ref)) > 2e-7 * max(1, np.max(np.abs(ref))):
            return False
    return True


def check_external_wrench():
    ch = _chain(3)
    st = chaingen.make_states(1, 3, seed=13)
    F = np.array([3.0, -1.5, 2.0, 0.4, -0.7, 0.25])
    b0 = oracle.default_base()
    b1 = b0.copy()
    b1[12:] = F
    t0 = oracle.rnea(ch, st["q"], st["qd"], st["qdd"], b0)
    t1 = oracle.rnea(ch, st["q"], st["qd"], st["qdd"], b1)
    return np.allclose(t1[0] - t0[0], L.tip_jacobian(ch, st["q"][0]).T @ F, atol=1e-11)


def check_fd():
    ch = _chain(4)
    st = chaingen.make_states(2, 4, seed=31, kinds=("q", "qd", "tau"))
    qa = oracle.fd_aba(ch, st["q"], st["qd"], st["tau"])
    qj, status = oracle.fd_jsiia(ch, st["q"], st["qd"], st["tau"])
    if np.any(status != 0) or not np.all(np.isfinite(qa)):
        return False
    z = np.zeros(4)
    for b in range(2):
        bias = oracle.rnea(ch, st["q"][b][None], st["qd"][b][None], z[None])[0]
        ref = np.linalg.solve(L.mass_matrix(ch, st["q"][b]), st["tau"][b] - bias)
        if np.max(np.abs(qa[b] - ref)) > 1e-8 * max(1, np.max(np.abs(ref))):
            return False
        if np.max(np.abs(qj[b] - ref)) > 1e-8 * max(1, np.max(np.abs(ref))):
            return False
    return True


def check_gradient():
    ch = _chain(3)
    st = chaingen.make_states(1, 3, seed=41, kinds=("q", "qd", "qdd", "w"))
    grads = oracle.rnea_grad(ch, st["q"], st["qd"], st["qdd"], st["w"])
    h = 1e-6
    for k, g in zip(("q", "qd", "qdd"), grads):
        for j in range(3):
            p = {x: st[x].copy() for x in ("q", "qd", "qdd")}
            m = {x: st[x].copy() for x in ("q", "qd", "qdd")}
            p[k][:, j] += h
            m[k][:, j] -= h
            d = np.sum(st["w"] * (oracle.rnea(ch, p["q"], p["qd"], p["qdd"])
                                  - oracle.rnea(ch, m["q"], m["qd"], m["qdd"]))) / (2 * h)
            if abs(g[0, j] - d) > 1e-6 * max(1, abs(d)):
                return False
    return True


def check_abi_schur():
    ch = _chain(4)
    q = chaingen.make_states(1, 4, seed=43, kinds=("q",))["q"][0]
    _, Om = oracle.abi_trace(ch, q)
    Mq = L.mass_matrix(ch, q)
    for i in range(4):
        a = Mq[i, i]
        if i + 1 < 4:
            a -= Mq[i + 1:, i] @ np.linalg.solve(Mq[i + 1:, i + 1:], Mq[i + 1:, i])
        if not abs(Om[i] - a) <= 1e-9 * Mq[i, i]:
            return False
    return True


CHECKS = [check_pendulum, check_lagrange, check_external_wrench, check_fd, check_gradient,
          check_abi_schur]

MUTATIONS = {
    "drop_coriolis_ad_term": {"dyn_body.h": [
        ("dV[i][k] = Sqdd[k] + AdV[k] - corr[k];", "dV[i][k] = Sqdd[k] + AdV[k];")]},
    "flip_sign_adT_in_bias": {"dyn_body.h": [
        ("F[k] = carried[k] + JdV[k] - adT[k];", "F[k] = carried[k] + JdV[k] + adT[k];")]},
    "backward_transform_off_by_one": {"dyn_body.h": [
        ("PREFIX(mat6T_vec)(Adinv[i + 1], Fnext, carried);",
         "PREFIX(mat6T_vec)(Adinv[i], Fnext, carried);")]},
    "backward_transform_not_transposed": {"dyn_body.h": [
        ("PREFIX(mat6T_vec)(Adinv[i + 1], Fnext, carried);",
         "PREFIX(mat6_vec)(Adinv[i + 1], Fnext, carried);")]},
    "forward_uses_f_not_f_inverse": {"dyn_body.h": [
        ("PREFIX(Ad_matrix)(Ri, pi, Adinv[i]);", "PREFIX(Ad_matrix)(R, p, Adinv[i]);")]},
    "exp_translation_drops_third_term": {"dyn_body.h": [
        ("G[i][j] = Id * t + (1.0 - ct) * W[i][j] + (t - st) * W2[i][j];",
         "G[i][j] = Id * t + (1.0 - ct) * W[i][j];")]},
    "inertia_no_parallel_axis_shift": {"dyn_body.h": [
        ("J[3 + i][3 + j] = Ic[i][j] - m * CC[i][j];", "J[3 + i][3 + j] = Ic[i][j];")]},
    "inertia_transposed_coupling": {"dyn_body.h": [
        ("J[i][3 + j] = -m * C[i][j];", "J[i][3 + j] = m * C[i][j];")]},
    "Ad_translation_sign": {"dyn_body.h": [
        ("A[i][3 + j] = PR[i][j];", "A[i][3 + j] = -PR[i][j];")]},
    "ad_blocks_swapped": {"dyn_body.h": [
        ("A[i][3 + j] = Vh[i][j];", "A[i][3 + j] = Wh[i][j];")]},
    "external_wrench_ignored": {"dyn_body.h": [
        ("for (int k = 0; k < 6; ++k) Fnext[k] = base[12 + k];",
         "for (int k = 0; k < 6; ++k) Fnext[k] = 0.0;")]},
    "aba_wrong_omega_index": {"oracle_real.c": [
        ("for (int k = 0; k < 6; ++k) Pi[i][k] = t[k] / Om[i];",
         "for (int k = 0; k < 6; ++k) Pi[i][k] = t[k] / Om[i - 1];")]},
    "aba_rank_one_term_dropped": {"oracle_real.c": [
        ("Jh[i][a][b2] = J[a][b2] + XTJX[a][b2] - T2[a][b2];",
         "Jh[i][a][b2] = J[a][b2] + XTJX[a][b2];")]},
    "aba_lambda_missing_Y": {"oracle_real.c": [
        ("for (int k = 0; k < 6; ++k) lam[k] = lnew[k] + S[6 * i + k] * ch[i];",
         "for (int k = 0; k < 6; ++k) lam[k] = S[6 * i + k] * ch[i];")]},
    "aba_congruence_not_transposed": {"oracle_real.c": [
        ("mat6_mul(XT, Jh[i + 1], T1);    /* X^T hat J */",
         "mat6_mul(X[i + 1], Jh[i + 1], T1);    /* X^T hat J */")]},
    "abi_trace_rank_one_term_dropped": {"oracle_real.c": [
        ("Jh[i][a][b2] = J[a][b2] + XTJX[a][b2] - u[a] * u[b2] / Om1;",
         "Jh[i][a][b2] = J[a][b2] + XTJX[a][b2];")]},
    "jsiia_bias_not_subtracted": {"oracle_real.c": [
        ("double s = tau[o + i] - bias[i];", "double s = tau[o + i];")]},
    "complex_step_reads_real_part": {"oracle_cs.c": [
        ("g += w[o + i] * cimag(tau[i]);", "g += w[o + i] * creal(tau[i]);")]},
}


def test_unmodified_oracle_passes_all_checks():
    for chk in CHECKS:
        assert chk(), chk.__name__


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    so = oracle.build_variant(str(tmp_path / name), MUTATIONS[name])
    failed = []
    with oracle.swapped_library(so):
        for chk in CHECKS:
            try:
                ok = chk()
            except Exception:
                ok = False
            if not ok:
                failed.append(chk.__name__)
    assert failed, f"mutation {name} slipped through every pin"
