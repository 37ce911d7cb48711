"""The hand-over protocol of rnea_vjp_pair_kernel (csrc/rnea_vjp_pair.cuh),
modelled on the host: two warps, a two-slot ring and four named barriers, each
completing when both warps have arrived (bar.sync waits for completion,
bar.arrive does not).

For every chain length the kernel accepts (n % 4 == 0, n <= 128) and many
interleavings of the two warps, the model checks that the warps never wait on
each other forever, that the consumer reads each link's slot after the
producer wrote that link into it, that the producer never overwrites a slot
the consumer has not read, that no warp arrives twice at one barrier phase, and
that every barrier ends complete (no half-arrived barrier at kernel exit).
"""
import random

import pytest

FULL, EMPTY = 1, 3  # barrier ids of slot 0; slot s uses id + s


def warp_programs(n):
    """The two warps' sweep-2 operations in program order, as the kernel issues
    them: the links run tip to base in chunks of 4 with j = 3..0, and the slot
    is (j + 1) & 1."""
    prod, cons = [], []
    for i0 in range(n - 4, -1, -4):
        for j in (3, 2, 1, 0):
            i = i0 + j
            t = n - 1 - i
            slot = (j + 1) & 1
            assert slot == t & 1
            if t >= 2:
                prod.append(("sync", EMPTY + slot, None))
            prod.append(("write", slot, t))
            prod.append(("arrive", FULL + slot, None))
            cons.append(("sync", FULL + slot, None))
            cons.append(("read", slot, t))
            if t + 2 <= n - 1:
                cons.append(("arrive", EMPTY + slot, None))
    return prod, cons


def simulate(n, pick, programs=None):
    prog = dict(zip("PC", programs or warp_programs(n)))
    pc = {"P": 0, "C": 0}
    arrived = {k: set() for k in (1, 2, 3, 4)}
    waiting = {"P": None, "C": None}
    holds = {0: None, 1: None}
    unread = {0: False, 1: False}
    while pc["P"] < len(prog["P"]) or pc["C"] < len(prog["C"]):
        ready = [w for w in "PC" if waiting[w] is None and pc[w] < len(prog[w])]
        assert ready, f"n={n}: both warps wait (P at {pc['P']}, C at {pc['C']})"
        w = pick(ready)
        op, a, t = prog[w][pc[w]]
        if op in ("sync", "arrive"):
            assert w not in arrived[a], f"n={n}: warp {w} arrives twice at barrier {a}"
            arrived[a].add(w)
            if len(arrived[a]) == 2:
                arrived[a] = set()
                for v in "PC":
                    if waiting[v] == a:
                        waiting[v] = None
            elif op == "sync":
                waiting[w] = a
        elif op == "write":
            assert not unread[a], f"n={n}: slot {a} overwritten before it was read"
            holds[a], unread[a] = t, True
        else:
            assert unread[a] and holds[a] == t, f"n={n}: read of link {t} found {holds[a]}"
            unread[a] = False
        pc[w] += 1
    assert all(not s for s in arrived.values()), f"n={n}: barrier left half-arrived"
    assert waiting == {"P": None, "C": None}


@pytest.mark.parametrize("n", list(range(4, 129, 4)))
def test_pair_protocol_completes_and_orders_the_ring(n):
    simulate(n, lambda ready: ready[0])    # producer first whenever it can run
    simulate(n, lambda ready: ready[-1])   # consumer first whenever it can run
    rng = random.Random(n)
    for _ in range(50):
        simulate(n, rng.choice)


def test_model_catches_a_missing_wait():
    """The model is not vacuous: without the producer's EMPTY waits it
    overwrites a slot the consumer has not read; without the consumer's EMPTY
    arrivals the producer waits forever."""
    prod, cons = warp_programs(8)
    no_wait = [op for op in prod if op[0] != "sync"]
    with pytest.raises(AssertionError, match="overwritten"):
        simulate(8, lambda ready: ready[0], (no_wait, cons))
    no_arrive = [op for op in cons if op[0] != "arrive"]
    with pytest.raises(AssertionError, match="both warps wait"):
        simulate(8, lambda ready: ready[0], (prod, no_arrive))
