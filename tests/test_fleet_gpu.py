"""GPU parity of fleet_batch: mixed inverse / forward dynamics requests over
many chains of different lengths, each request with its own robot, in one
persistent launch or one launch per (kind, n) group, against the FP64 oracle.
Bars as for rnea_batch (ID) and aba_batch (FD)."""
import numpy as np
import pytest

import chaingen
import oracle

pytestmark = pytest.mark.gpu
TOL_ID = {"float32": 1e-4, "float64": 1e-10}
TOL_FD = {"float32": 1e-3, "float64": 1e-8}


def build(rd, count, n_lo, n_hi, dtype, seed=7, fd_fraction=0.2):
    import torch

    reqs = chaingen.uneven_requests(count, n_lo=n_lo, n_hi=n_hi, fd_fraction=fd_fraction, seed=seed)
    fleet = rd.Fleet([r["chain"] for r in reqs])
    kinds = np.array([1 if r["kind"] == "fd" else 0 for r in reqs], dtype=np.int32)
    plan = rd.Plan(fleet, np.arange(count, dtype=np.int32), kinds, dtype=dtype)
    J = plan.total_joints
    rng = np.random.default_rng(seed + 1)
    q = rng.uniform(-np.pi, np.pi, J)
    qd = rng.normal(0, 1, J)
    in2 = np.where(np.repeat(kinds, plan.lengths) == 1, rng.normal(0, 10, J), rng.normal(0, 2, J))
    npdt = np.float32 if dtype == "float32" else np.float64
    host = [x.astype(npdt) for x in (q, qd, in2)]
    dev = [torch.from_numpy(x).cuda() for x in host]
    return reqs, fleet, plan, kinds, [x.astype(np.float64) for x in host], dev


def check(reqs, plan, kinds, host, out, dtype, sample=None):
    idx = range(len(reqs)) if sample is None else sample
    worst_id = worst_fd = 0.0
    for r in idx:
        o, n = plan.offsets[r], plan.lengths[r]
        sl = slice(o, o + n)
        ch = reqs[r]["chain"]
        if kinds[r] == 0:
            ref = oracle.rnea(ch, host[0][sl][None], host[1][sl][None], host[2][sl][None])
            worst_id = max(worst_id, oracle.rel_err(out[sl][None], ref))
        else:
            ref = oracle.fd_aba(ch, host[0][sl][None], host[1][sl][None], host[2][sl][None])
            worst_fd = max(worst_fd, oracle.rel_err(out[sl][None], ref))
    assert worst_id <= TOL_ID[dtype], worst_id
    assert worst_fd <= TOL_FD[dtype], worst_fd


@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("schedule", [0, 1])
def test_fleet_mixed_requests(cuda_lib, dtype, schedule):
    reqs, fleet, plan, kinds, host, dev = build(cuda_lib, 400, 1, 40, dtype, fd_fraction=0.3)
    out = cuda_lib.fleet_batch(plan, *dev, schedule=schedule).cpu().numpy().astype(np.float64)
    check(reqs, plan, kinds, host, out, dtype)


def test_fleet_schedules_and_shapes_agree_exactly(cuda_lib):
    reqs, fleet, plan, kinds, host, dev = build(cuda_lib, 300, 6, 60, "float32", seed=9)
    ref = cuda_lib.fleet_batch(plan, *dev, schedule=1).cpu().numpy()
    for tune in (0, cuda_lib.RD_FLEET_TUNE(5, 1), cuda_lib.RD_FLEET_TUNE(8, 2)):
        out = cuda_lib.fleet_batch(plan, *dev, schedule=0, tune=tune).cpu().numpy()
        assert np.array_equal(out, ref)


def test_fleet_uneven_workload_sampled(cuda_lib):
    """5000 requests, n uniform in 6..100, 80% ID / 20% FD, FP32: a sample of 250
    requests checked against the oracle."""
    reqs, fleet, plan, kinds, host, dev = build(cuda_lib, 5000, 6, 100, "float32", seed=1609)
    out = cuda_lib.fleet_batch(plan, *dev).cpu().numpy().astype(np.float64)
    check(reqs, plan, kinds, host, out, "float32", sample=range(0, 5000, 20))


def test_fleet_base_motion_and_wrench(cuda_lib):
    import torch

    base = np.array([0.2, -0.1, 0.3, 0.5, -0.4, 0.25, 0.3, 1.1, 9.81, -0.2, 0.4, 0.1,
                     2.0, -1.0, 0.5, 0.3, 0.2, -0.6])
    reqs, fleet, plan, kinds, host, dev = build(cuda_lib, 60, 2, 20, "float64", seed=5, fd_fraction=0.5)
    out = cuda_lib.fleet_batch(plan, *dev, base=base).cpu().numpy()
    for r in range(60):
        o, n = plan.offsets[r], plan.lengths[r]
        sl = slice(o, o + n)
        fn = oracle.rnea if kinds[r] == 0 else oracle.fd_aba
        ref = fn(reqs[r]["chain"], host[0][sl][None], host[1][sl][None], host[2][sl][None], base=base)
        assert oracle.rel_err(out[sl][None], ref) <= (TOL_ID if kinds[r] == 0 else TOL_FD)["float64"]


def test_fleet_status_flags_singular_forward_request(cuda_lib):
    import torch

    chains = [chaingen.pendulum(1.0, 0.0, 0.0), chaingen.make_chain(5)]
    fleet = cuda_lib.Fleet(chains)
    plan = cuda_lib.Plan(fleet, [0, 1, 1], [1, 1, 0], dtype="float64")
    J = plan.total_joints
    x = torch.zeros(J, dtype=torch.float64, device="cuda")
    status = torch.full((3,), -1, dtype=torch.int32, device="cuda")
    cuda_lib.fleet_batch(plan, x, x, x + 1.0, status=status)
    assert status.cpu().tolist()[:2] == [1, 0]


def test_autotuner_picks_a_working_configuration(cuda_lib, tmp_path, monkeypatch):
    import torch

    from paper_1609_04493_gb300 import autotune

    monkeypatch.setenv("RDYN_TUNE_CACHE", str(tmp_path / "tune.json"))
    reqs, fleet, plan, kinds, host, dev = build(cuda_lib, 200, 6, 30, "float32", seed=3)
    (sched, tune), times = autotune.tune_fleet(plan, *dev, use_cache=False)
    assert (sched, tune) in times and len(times) == len(autotune.fleet_candidates())
    again, _ = autotune.tune_fleet(plan, *dev)  # from the cache now
    assert again == (sched, tune)
    ch = chaingen.make_chain(16)
    model = cuda_lib.Model(ch)
    st = chaingen.make_states(2048, 16, seed=4)
    x = [torch.from_numpy(st[k]).float().cuda() for k in ("q", "qd", "qdd")]
    v, t = autotune.tune_rnea(model, *x, use_cache=False)
    tau = cuda_lib.rnea(model, *x, variant=v).cpu().numpy()
    ref = oracle.rnea(ch, *(a.cpu().double().numpy() for a in x))
    assert oracle.rel_err(tau, ref) <= 1e-4


@pytest.mark.parametrize("schedule", [0, 1])
def test_fleet_fp64_update_flag(cuda_lib, schedule):
    """FP32 plan with RD_FLEET_FP64_UPDATE: the forward-dynamics requests run
    their inertia updates and solves in FP64; same bars, and inverse-dynamics
    outputs identical to the default call (the flag touches only forward
    dynamics)."""
    reqs, fleet, plan, kinds, host, dev = build(cuda_lib, 600, 4, 90, "float32", seed=21,
                                                fd_fraction=0.4)
    out = cuda_lib.fleet_batch(plan, *dev, schedule=schedule | cuda_lib.RD_FLEET_FP64_UPDATE)
    out = out.cpu().numpy()
    check(reqs, plan, kinds, host, out.astype(np.float64), "float32")
    ref = cuda_lib.fleet_batch(plan, *dev, schedule=schedule).cpu().numpy()
    id_mask = np.repeat(kinds, plan.lengths) == 0
    assert np.array_equal(out[id_mask], ref[id_mask])
    # the two update precisions agree to far below the FP32 bar
    fd = ~id_mask
    scale = np.max(np.abs(ref[fd]))
    assert np.max(np.abs(out[fd] - ref[fd])) <= 1e-4 * scale


def _stratified(kinds, lengths, per_group, seed=0):
    """Up to `per_group` requests of every (kind, n) pair, drawn at random."""
    rng = np.random.default_rng(seed)
    pick = []
    for kind in (0, 1):
        for n in np.unique(lengths):
            idx = np.flatnonzero((kinds == kind) & (lengths == n))
            if len(idx):
                pick.extend(rng.choice(idx, size=min(per_group, len(idx)), replace=False))
    return np.sort(np.array(pick))


def test_fleet_uneven_workload_at_full_size(cuda_lib):
    """The bench's uneven workload exactly (100000 requests from seed 1609,
    its inputs, FP32): the persistent launch with FP64 inertia updates and
    solves, one launch per (kind, n) group with the same, the persistent launch
    with the double-float default, and both precisions with two warps per 32
    forward-dynamics requests from 33 links. 11 requests of every (kind, n) pair,
    n = 6..100 (2090 requests), checked against the oracle on the FP32 bars."""
    import torch

    import bench

    rd = cuda_lib
    reqs, fleet, plan, kinds, host = bench.uneven_workload(rd, 100000)
    lengths = np.asarray(plan.lengths)
    assert set(np.unique(lengths)) == set(range(6, 101))
    sample = _stratified(kinds, lengths, 11, seed=1)
    assert len(sample) >= 2000
    assert {int(n) for n in lengths[sample[kinds[sample] == 1]]} == set(range(6, 101))
    assert {int(n) for n in lengths[sample[kinds[sample] == 0]]} == set(range(6, 101))
    x = [torch.from_numpy(a).cuda() for a in host]
    h64 = [a.astype(np.float64) for a in host]
    refs = {}
    for r in sample:
        o, n = plan.offsets[r], plan.lengths[r]
        sl = slice(o, o + n)
        fn = oracle.rnea if kinds[r] == 0 else oracle.fd_aba
        refs[r] = fn(reqs[r]["chain"], h64[0][sl][None], h64[1][sl][None], h64[2][sl][None])
    f64 = rd.RD_FLEET_FP64_UPDATE
    pair = rd.RD_FLEET_TUNE(7, 2) | rd.RD_FLEET_TWO_WARPS(33)
    tri = rd.RD_FLEET_TUNE(7, 2) | rd.RD_FLEET_THREE_WARPS(65)
    for schedule, tune in ((0 | f64, 0), (rd.RD_SCHED_PER_GROUP | f64, 0), (0, 0), (0 | f64, pair),
                           (0, pair), (0 | f64, tri)):
        out = rd.fleet_batch(plan, *x, schedule=schedule, tune=tune).cpu().numpy().astype(np.float64)
        worst = {0: 0.0, 1: 0.0}
        for r in sample:
            o, n = plan.offsets[r], plan.lengths[r]
            e = oracle.rel_err(out[o:o + n][None], refs[r])
            worst[int(kinds[r])] = max(worst[int(kinds[r])], e)
        assert worst[0] <= TOL_ID["float32"], (schedule, tune, worst)
        assert worst[1] <= TOL_FD["float32"], (schedule, tune, worst)


@pytest.mark.parametrize("warps", [2, 3])
@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("min_links", [1, 33, 65])
def test_fleet_two_warp_forward_dynamics(cuda_lib, dtype, min_links, warps):
    """RD_FLEET_TWO_WARPS / RD_FLEET_THREE_WARPS: forward-dynamics groups from a
    length on run two or three warps per 32 requests; every request against the
    oracle, and against the one-thread-per-request schedule (FP64 to rounding,
    FP32 to a few ulps)."""
    reqs, fleet, plan, kinds, host, dev = build(cuda_lib, 700, 2, 100, dtype, seed=31,
                                                fd_fraction=0.4)
    split = cuda_lib.RD_FLEET_TWO_WARPS if warps == 2 else cuda_lib.RD_FLEET_THREE_WARPS
    tune = cuda_lib.RD_FLEET_TUNE(7, 2) | split(min_links)
    out = cuda_lib.fleet_batch(plan, *dev, tune=tune).cpu().numpy().astype(np.float64)
    check(reqs, plan, kinds, host, out, dtype)
    ref = cuda_lib.fleet_batch(plan, *dev).cpu().numpy().astype(np.float64)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(out - ref)) <= (1e-10 if dtype == "float64" else 1e-5) * scale


@pytest.mark.parametrize("warps", [2, 3])
def test_fleet_two_warps_fp64_update_and_status(cuda_lib, warps):
    import torch

    reqs, fleet, plan, kinds, host, dev = build(cuda_lib, 300, 40, 100, "float32", seed=33,
                                                fd_fraction=0.5)
    status = torch.full((300,), -1, dtype=torch.int32, device="cuda")
    split = cuda_lib.RD_FLEET_TWO_WARPS if warps == 2 else cuda_lib.RD_FLEET_THREE_WARPS
    tune = cuda_lib.RD_FLEET_TUNE(6, 4) | split(6)
    out = cuda_lib.fleet_batch(plan, *dev, status=status, tune=tune,
                               schedule=cuda_lib.RD_FLEET_FP64_UPDATE)
    check(reqs, plan, kinds, host, out.cpu().numpy().astype(np.float64), "float32")
    st = status.cpu().numpy()
    assert np.all(st[kinds == 1] == 0)


def test_fleet_two_warps_rejects_bad_shapes(cuda_lib):
    reqs, fleet, plan, kinds, host, dev = build(cuda_lib, 50, 4, 20, "float32", seed=35)
    for tune in (cuda_lib.RD_FLEET_TUNE(5, 1) | cuda_lib.RD_FLEET_TWO_WARPS(6),
                 cuda_lib.RD_FLEET_TUNE(9, 1) | cuda_lib.RD_FLEET_TWO_WARPS(6)):
        with pytest.raises(cuda_lib.RdError):
            cuda_lib.fleet_batch(plan, *dev, tune=tune)
    with pytest.raises(cuda_lib.RdError):
        cuda_lib.fleet_batch(plan, *dev, schedule=cuda_lib.RD_SCHED_PER_GROUP,
                             tune=cuda_lib.RD_FLEET_TWO_WARPS(6))
    # three warps: one or two triples per block (tune threads 64 or 128), a
    # chain length, the persistent schedule
    for tune in (cuda_lib.RD_FLEET_TUNE(8, 1) | cuda_lib.RD_FLEET_THREE_WARPS(6),
                 cuda_lib.RD_FLEET_TUNE(5, 1) | cuda_lib.RD_FLEET_THREE_WARPS(6),
                 cuda_lib.RD_FLEET_TUNE(7, 1) | (1 << 24)):
        with pytest.raises(cuda_lib.RdError):
            cuda_lib.fleet_batch(plan, *dev, tune=tune)
    with pytest.raises(cuda_lib.RdError):
        cuda_lib.fleet_batch(plan, *dev, schedule=cuda_lib.RD_SCHED_PER_GROUP,
                             tune=cuda_lib.RD_FLEET_THREE_WARPS(6))
