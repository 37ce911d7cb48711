"""Write the golden fixtures of this folder from the FP64 oracle.

Run from the repository root:  python tests/golden/make_golden.py

Inputs come from the seeded generator (``chaingen``); joint states are rounded
to float32 first, so that an FP32 and an FP64 run of the CUDA path see the same
values as the oracle did. Expected values come from ``oracle`` only. Rewriting
a fixture after a change to the oracle's arithmetic is a deliberate step: the
commit that does it names the passage of the paper that justifies the change.
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
for p in (ROOT, os.path.dirname(HERE)):
    if p not in sys.path:
        sys.path.insert(0, p)

import chaingen  # noqa: E402
import oracle  # noqa: E402
from golden import format_fixture  # noqa: E402

# a moving base with an external wrench on the last link: (V_0, dV_0, F_{n+1})
MOVING_BASE = np.array([0.2, -0.1, 0.3, 0.5, -0.4, 0.25,
                        0.3, 1.1, 9.81, -0.2, 0.4, 0.1,
                        2.0, -1.0, 0.5, 0.3, 0.2, -0.6])


def _inputs(n, B, chain_seed, state_seed, kinds):
    ch = chaingen.make_chain(n, seed=chain_seed)
    st = chaingen.make_states(B, n, seed=state_seed, kinds=kinds)
    st = {k: v.astype(np.float32).astype(np.float64) for k, v in st.items()}
    return ch, st


def _chain_arrays(ch):
    return [("M", ch.M), ("S", ch.S), ("inertia", ch.inertia)]


def rnea_n7():
    n, B, cs, ss = 7, 4, chaingen.BASE_SEED + 7, 101
    ch, st = _inputs(n, B, cs, ss, ("q", "qd", "qdd"))
    base = oracle.default_base()
    tau = oracle.rnea(ch, st["q"], st["qd"], st["qdd"], base=base)
    t0, V, dV, F = oracle.rnea_trace(ch, st["q"][0], st["qd"][0], st["qdd"][0], base=base)
    return format_fixture(
        "inverse dynamics, n = 7, B = 4, base at rest under gravity",
        ["Sec. II-A, Eqs. (id-forward) and (id-backward): tau = ID(q, qd, qdd, V_0, dV_0, F_{n+1})",
         "gravity enters as dV_0 = (0, 0, g, 0, 0, 0), g = 9.81 (linear part first)",
         "trace_V, trace_dV, trace_F: the per-link V_i, dV_i, F_i of instance 0",
         "(the outputs of the forward scan of Eq. (scan-id-vel-acc) and of the backward scan)"],
        {"kind": "rnea", "n": n, "B": B, "chain_seed": cs, "state_seed": ss},
        _chain_arrays(ch) + [("base", base), ("q", st["q"]), ("qd", st["qd"]),
                             ("qdd", st["qdd"]), ("tau", tau), ("trace_V", V),
                             ("trace_dV", dV), ("trace_F", F)])


def rnea_n5_moving_base():
    n, B, cs, ss = 5, 3, chaingen.BASE_SEED + 5, 102
    ch, st = _inputs(n, B, cs, ss, ("q", "qd", "qdd"))
    tau = oracle.rnea(ch, st["q"], st["qd"], st["qdd"], base=MOVING_BASE)
    return format_fixture(
        "inverse dynamics, n = 5, B = 3, moving base and external wrench",
        ["Sec. II-A, Eqs. (id-forward) and (id-backward) with the boundary conditions",
         "V_0, dV_0 (base twist and its derivative) and F_{n+1} (wrench on the last link)"],
        {"kind": "rnea", "n": n, "B": B, "chain_seed": cs, "state_seed": ss},
        _chain_arrays(ch) + [("base", MOVING_BASE), ("q", st["q"]), ("qd", st["qd"]),
                             ("qdd", st["qdd"]), ("tau", tau)])


def fd_n6():
    n, B, cs, ss = 6, 4, chaingen.BASE_SEED + 6, 103
    ch, st = _inputs(n, B, cs, ss, ("q", "qd", "tau"))
    base = oracle.default_base()
    qdd_aba = oracle.fd_aba(ch, st["q"], st["qd"], st["tau"], base=base)
    qdd_jsiia, status = oracle.fd_jsiia(ch, st["q"], st["qd"], st["tau"], base=base)
    assert np.all(status == 0)
    _, omega = oracle.abi_trace(ch, st["q"][0])
    return format_fixture(
        "forward dynamics, n = 6, B = 4, base at rest under gravity",
        ["Sec. II-B: qdd_aba by the articulated-body recursion, Eqs. (abi) and (recursive-fd);",
         "qdd_jsiia = M(q)^-1 (tau - tau_bias), Eqs. (tau-bias) and (JSIinv)",
         "omega: Omega_i = S_i^T J_hat_i S_i of Eq. (abi) for instance 0"],
        {"kind": "fd", "n": n, "B": B, "chain_seed": cs, "state_seed": ss},
        _chain_arrays(ch) + [("base", base), ("q", st["q"]), ("qd", st["qd"]),
                             ("tau", st["tau"]), ("qdd_aba", qdd_aba),
                             ("qdd_jsiia", qdd_jsiia), ("omega", omega)])


def vjp_n4():
    n, B, cs, ss = 4, 3, chaingen.BASE_SEED + 4, 104
    ch, st = _inputs(n, B, cs, ss, ("q", "qd", "qdd", "w"))
    base = oracle.default_base()
    gq, gqd, gqdd = oracle.rnea_grad(ch, st["q"], st["qd"], st["qdd"], st["w"], base=base)
    return format_fixture(
        "adjoint of inverse dynamics, n = 4, B = 3",
        ["gradient of w^T tau with respect to q, qd, qdd, tau from Sec. II-A, Eqs. (id-forward)",
         "and (id-backward); the adjoint the conclusion (Sec. VI) names as future work;",
         "taken by the complex step, exact to rounding"],
        {"kind": "vjp", "n": n, "B": B, "chain_seed": cs, "state_seed": ss},
        _chain_arrays(ch) + [("base", base), ("q", st["q"]), ("qd", st["qd"]),
                             ("qdd", st["qdd"]), ("w", st["w"]), ("gq", gq), ("gqd", gqd),
                             ("gqdd", gqdd)])


def mass_matrix_n5():
    n, B, cs, ss = 5, 2, chaingen.BASE_SEED + 15, 105
    ch, st = _inputs(n, B, cs, ss, ("q",))
    Mq = oracle.mass_matrix(ch, st["q"])
    return format_fixture(
        "joint-space inertia, n = 5, B = 2",
        ["Sec. II-B: the joint-space inertia M(q) of Eq. (fd); column j = ID(q, 0, e_j)",
         "with the base at rest and no gravity, the n unit-acceleration IDs of Sec. III-C"],
        {"kind": "mass_matrix", "n": n, "B": B, "chain_seed": cs, "state_seed": ss},
        _chain_arrays(ch) + [("q", st["q"]), ("Mq", Mq.reshape(B * n, n))])


WRITERS = {
    "rnea_n7.txt": rnea_n7,
    "rnea_n5_moving_base.txt": rnea_n5_moving_base,
    "fd_n6.txt": fd_n6,
    "vjp_n4.txt": vjp_n4,
    "mass_matrix_n5.txt": mass_matrix_n5,
}


def main():
    for name, fn in WRITERS.items():
        with open(os.path.join(HERE, name), "w") as f:
            f.write(fn())
        print("wrote", name)


if __name__ == "__main__":
    main()
