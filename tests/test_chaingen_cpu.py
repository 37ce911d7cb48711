"""The seeded input generator against the recipe of the random-robot
experiments (Sec. V): valid rigid bodies and revolute joints, the stated
distributions, reproducibility, and the mixed-request workload (link counts
uniform in 6..100, each robot from its own seed, a 20% share of forward
dynamics)."""
import numpy as np

import chaingen


def test_chain_is_a_valid_serial_chain_of_revolute_joints():
    ch = chaingen.make_chain(64, seed=5)
    R = ch.M[:, :9].reshape(-1, 3, 3)
    assert np.allclose(np.einsum("nij,nkj->nik", R, R), np.eye(3), atol=1e-12)
    assert np.allclose(np.linalg.det(R), 1.0, atol=1e-12)
    assert np.all((ch.M[:, 9:] >= 0.1) & (ch.M[:, 9:] <= 0.5))
    w, v = ch.S[:, 3:], ch.S[:, :3]
    assert np.allclose(np.linalg.norm(w, axis=1), 1.0, atol=1e-12)
    assert np.allclose(np.einsum("ij,ij->i", w, v), 0.0, atol=1e-12)  # zero pitch
    m = ch.inertia[:, 0]
    assert np.all((m >= 0.5) & (m <= 5.0))
    assert np.all(np.abs(ch.inertia[:, 1:4]) <= 0.1)
    for row in ch.inertia:
        Ic = np.array([[row[4], row[7], row[8]], [row[7], row[5], row[9]], [row[8], row[9], row[6]]])
        d = np.linalg.eigvalsh(Ic)
        assert d[0] > 0
        assert d[2] <= d[0] + d[1] + 1e-12  # triangle inequality of principal moments


def test_generator_is_reproducible_and_seed_dependent():
    a, b = chaingen.make_chain(7, seed=11), chaingen.make_chain(7, seed=11)
    c = chaingen.make_chain(7, seed=12)
    assert np.array_equal(a.M, b.M) and np.array_equal(a.inertia, b.inertia)
    assert not np.array_equal(a.M, c.M)
    s1 = chaingen.make_states(5, 7, seed=3, kinds=("q", "tau"))
    s2 = chaingen.make_states(5, 7, seed=3, kinds=("q", "tau"))
    assert np.array_equal(s1["q"], s2["q"]) and np.array_equal(s1["tau"], s2["tau"])


def test_state_distributions():
    st = chaingen.make_states(20000, 10, seed=9, kinds=("q", "qd", "qdd", "tau", "w"))
    assert np.all(np.abs(st["q"]) <= np.pi)
    assert abs(np.std(st["q"]) - np.pi / np.sqrt(3)) < 0.02
    for k, sd in (("qd", 1.0), ("qdd", 2.0), ("tau", 10.0), ("w", 1.0)):
        assert abs(np.mean(st[k])) < 0.03 * sd, k
        assert abs(np.std(st[k]) / sd - 1.0) < 0.02, k


def test_mixed_requests_follow_the_workload_recipe():
    reqs = chaingen.uneven_requests(4000, n_lo=6, n_hi=100, fd_fraction=0.2, seed=77)
    ns = np.array([r["n"] for r in reqs])
    assert ns.min() >= 6 and ns.max() <= 100
    assert set(np.unique(ns)) == set(range(6, 101))  # every length occurs at this count
    fd = np.mean([r["kind"] == "fd" for r in reqs])
    assert abs(fd - 0.2) < 0.02
    for k in (0, 1, 2, 3999):
        assert reqs[k]["chain"].n == reqs[k]["n"]
        own = chaingen.make_chain(reqs[k]["n"], seed=77 + k)
        assert np.array_equal(reqs[k]["chain"].M, own.M)
    assert not np.array_equal(reqs[0]["chain"].S[:6], reqs[1]["chain"].S[:6])
