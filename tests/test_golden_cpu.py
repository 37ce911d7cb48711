"""The golden fixtures under tests/golden/ against the generator and the oracle.

Each fixture stores seeded inputs and the oracle's FP64 outputs, with the
passage of the paper it follows. These tests check that

* the seeded generator still draws exactly the stored inputs;
* the oracle still reproduces the stored outputs (a later change to its
  arithmetic shows up here and must come with a rewritten fixture);
* the stored values satisfy what the mathematics fixes between them: the two
  forward-dynamics algorithms agree, ID(FD(tau)) = tau, M(q) is symmetric
  positive definite, the per-link trace ends in the stored torques, and
  d(w^T tau)/d qdd = M(q) w.
"""
import numpy as np
import pytest

import chaingen
import golden
import oracle

# the oracle runs the same C code here and on other hosts; only libm's sin
# and cos may round differently in the last place
REPRO = 1e-13

KINDS = {
    "rnea": ("q", "qd", "qdd"),
    "fd": ("q", "qd", "tau"),
    "vjp": ("q", "qd", "qdd", "w"),
    "mass_matrix": ("q",),
}


def _chain(fx):
    return chaingen.Chain(fx["M"], fx["S"], fx["inertia"])


@pytest.fixture(params=golden.FIXTURES)
def fx(request):
    return golden.load(request.param)


def test_fixture_set_is_complete():
    import os

    stored = sorted(f for f in os.listdir(golden.HERE) if f.endswith(".txt"))
    assert stored == sorted(golden.FIXTURES)


def test_fixture_cites_the_paper_and_the_oracle(fx):
    text = " ".join(fx.header)
    assert "Sec." in text, fx.name
    assert "oracle" in text, fx.name
    for key in ("kind", "n", "B", "chain_seed", "state_seed"):
        assert key in fx.scalars, (fx.name, key)


def test_generator_draws_the_stored_inputs(fx):
    n, B = fx.scalars["n"], fx.scalars["B"]
    ch = chaingen.make_chain(n, seed=fx.scalars["chain_seed"])
    assert np.array_equal(ch.M, fx["M"])
    assert np.array_equal(ch.S, fx["S"])
    assert np.array_equal(ch.inertia, fx["inertia"])
    kinds = KINDS[fx.scalars["kind"]]
    st = chaingen.make_states(B, n, seed=fx.scalars["state_seed"], kinds=kinds)
    for k in kinds:
        assert np.array_equal(st[k].astype(np.float32).astype(np.float64), fx[k]), (fx.name, k)


def test_parser_round_trips_the_writer():
    a = np.array([[0.1, -2.5e-300, 3.0], [np.pi, 1.0 / 3.0, -0.0]])
    text = golden.format_fixture("t", ["Sec. I"], {"kind": "x", "n": 3}, [("a", a), ("b", a[0])])
    back = golden.parse(text)
    assert back.scalars == {"kind": "x", "n": 3}
    assert np.array_equal(back["a"], a) and np.array_equal(back["b"], a[0])
    assert np.signbit(back["a"][1, 2])


def _close(x, ref, tol):
    err = oracle.rel_err(np.atleast_2d(x), np.atleast_2d(ref))
    assert err <= tol, err


def test_oracle_reproduces_rnea_fixtures():
    for name in ("rnea_n7.txt", "rnea_n5_moving_base.txt"):
        fx = golden.load(name)
        ch = _chain(fx)
        tau = oracle.rnea(ch, fx["q"], fx["qd"], fx["qdd"], base=fx["base"])
        _close(tau, fx["tau"], REPRO)


def test_oracle_reproduces_the_trace():
    fx = golden.load("rnea_n7.txt")
    t0, V, dV, F = oracle.rnea_trace(_chain(fx), fx["q"][0], fx["qd"][0], fx["qdd"][0],
                                     base=fx["base"])
    for got, key in ((V, "trace_V"), (dV, "trace_dV"), (F, "trace_F")):
        _close(got.reshape(1, -1), fx[key].reshape(1, -1), REPRO)
    _close(t0, fx["tau"][0], REPRO)


def test_oracle_reproduces_fd_fixture():
    fx = golden.load("fd_n6.txt")
    ch = _chain(fx)
    _close(oracle.fd_aba(ch, fx["q"], fx["qd"], fx["tau"], base=fx["base"]), fx["qdd_aba"], REPRO)
    qdd, st = oracle.fd_jsiia(ch, fx["q"], fx["qd"], fx["tau"], base=fx["base"])
    assert np.all(st == 0)
    _close(qdd, fx["qdd_jsiia"], REPRO)
    _, om = oracle.abi_trace(ch, fx["q"][0])
    _close(om, fx["omega"], REPRO)


def test_oracle_reproduces_vjp_fixture():
    fx = golden.load("vjp_n4.txt")
    g = oracle.rnea_grad(_chain(fx), fx["q"], fx["qd"], fx["qdd"], fx["w"], base=fx["base"])
    for got, key in zip(g, ("gq", "gqd", "gqdd")):
        _close(got, fx[key], REPRO)


def test_oracle_reproduces_mass_matrix_fixture():
    fx = golden.load("mass_matrix_n5.txt")
    n, B = fx.scalars["n"], fx.scalars["B"]
    Mq = oracle.mass_matrix(_chain(fx), fx["q"])
    _close(Mq.reshape(B, -1), fx["Mq"].reshape(B, -1), REPRO)


# ---- relations between the stored values


def test_stored_fd_algorithms_agree_and_invert_id():
    fx = golden.load("fd_n6.txt")
    _close(fx["qdd_aba"], fx["qdd_jsiia"], 1e-11)
    tau = oracle.rnea(_chain(fx), fx["q"], fx["qd"], fx["qdd_aba"], base=fx["base"])
    _close(tau, fx["tau"], 1e-11)
    assert np.all(fx["omega"] > 0)


def test_stored_mass_matrix_is_symmetric_positive_definite():
    fx = golden.load("mass_matrix_n5.txt")
    n, B = fx.scalars["n"], fx.scalars["B"]
    for Mb in fx["Mq"].reshape(B, n, n):
        assert np.max(np.abs(Mb - Mb.T)) <= 1e-14 * np.max(np.abs(Mb))
        assert np.all(np.linalg.eigvalsh(Mb) > 0)


def test_stored_trace_ends_in_the_stored_torques():
    fx = golden.load("rnea_n7.txt")
    # tau_i = S_i^T F_i (Eq. id-backward), S_i in frame i, linear part first
    tau0 = np.einsum("ij,ij->i", fx["S"], fx["trace_F"])
    _close(tau0, fx["tau"][0], 1e-13)


def test_stored_qdd_gradient_is_mass_matrix_times_w():
    fx = golden.load("vjp_n4.txt")
    Mq = oracle.mass_matrix(_chain(fx), fx["q"])
    _close(np.einsum("bij,bi->bj", Mq, fx["w"]), fx["gqdd"], 1e-12)
