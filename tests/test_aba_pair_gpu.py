"""GPU parity of forward dynamics with two warps per 32 instances
(RD_ABA_TWO_WARPS): one warp runs the articulated-inertia recursion of
Eq. (abi), the other the bias sweeps, tau_hat, z_hat and c_hat beside it and
then lambda / qdd (Sec. II-B); and with three (RD_ABA_THREE_WARPS), the
articulated-inertia recursion split over two warps by block. Every test runs
both mappings. Against the FP64 oracle's fd_aba, through the C ABI. Bars as in
test_aba_gpu.py: FP32 data 1e-3, FP64 data 1e-8.
"""
import numpy as np
import pytest

import chaingen
import oracle

pytestmark = pytest.mark.gpu
TOL = {"float32": 1e-3, "float64": 1e-8}
BASE = np.array([0.2, -0.1, 0.3, 0.5, -0.4, 0.25, 0.3, 1.1, 9.81, -0.2, 0.4, 0.1,
                 2.0, -1.0, 0.5, 0.3, 0.2, -0.6])


@pytest.fixture(params=["two", "three"])
def mapping(request, cuda_lib):
    return {"two": cuda_lib.RD_ABA_TWO_WARPS, "three": cuda_lib.RD_ABA_THREE_WARPS}[request.param]


def run(rd, n, B, dtype, seed=73, base=None, flags=0, status=None, mapping=None):
    import torch

    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED + 9 * n)
    st = chaingen.make_states(B, n, seed=seed, kinds=("q", "qd", "tau"))
    npdt = np.float32 if dtype == "float32" else np.float64
    host = {k: st[k].astype(npdt) for k in st}
    dev = {k: torch.from_numpy(v).cuda() for k, v in host.items()}
    model = rd.Model(ch)
    qdd = rd.aba(model, dev["q"], dev["qd"], dev["tau"], base=base, status=status,
                 flags=flags | (rd.RD_ABA_TWO_WARPS if mapping is None else mapping))
    torch.cuda.synchronize()
    h64 = {k: v.astype(np.float64) for k, v in host.items()}
    return qdd.cpu().double().numpy(), ch, h64, model


@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("n", [1, 2, 7, 16, 33, 64, 65, 100, 128])
def test_pair_fd_matches_oracle(cuda_lib, mapping, n, dtype):
    qdd, ch, h, _ = run(cuda_lib, n, 70, dtype, mapping=mapping)
    ref = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"])
    assert oracle.rel_err(qdd, ref) <= TOL[dtype], f"n={n} {dtype}"


@pytest.mark.parametrize("n", [7, 64, 100])
def test_pair_fd_fp64_update_matches_oracle(cuda_lib, mapping, n):
    qdd, ch, h, _ = run(cuda_lib, n, 45, "float32", flags=cuda_lib.RD_ABA_FP64_UPDATE,
                        mapping=mapping)
    ref = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"])
    assert oracle.rel_err(qdd, ref) <= TOL["float32"]


@pytest.mark.parametrize("B", [1, 31, 33, 300])
def test_pair_fd_ragged_batches(cuda_lib, mapping, B):
    """Batches that leave lanes of the last block idle."""
    qdd, ch, h, _ = run(cuda_lib, 21, B, "float64", seed=4, mapping=mapping)
    ref = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"])
    assert oracle.rel_err(qdd, ref) <= TOL["float64"]


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_pair_fd_base_motion_and_wrench(cuda_lib, mapping, dtype):
    for n in (6, 40, 90):
        qdd, ch, h, _ = run(cuda_lib, n, 37, dtype, base=BASE, mapping=mapping)
        ref = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"], base=BASE)
        assert oracle.rel_err(qdd, ref) <= TOL[dtype], f"n={n}"


def test_pair_fd_agrees_with_thread_per_instance(cuda_lib, mapping):
    """FP64 data: one result to rounding; FP32 data: the same operations in the
    same precisions, so equal to a few ulps."""
    import torch

    for n in (12, 64, 97):
        a, ch, h, model = run(cuda_lib, n, 64, "float64", seed=9, mapping=mapping)
        x = [torch.from_numpy(h[k]).cuda() for k in ("q", "qd", "tau")]
        b = cuda_lib.aba(model, *x, flags=cuda_lib.RD_ABA_THREAD_PER_INSTANCE).cpu().numpy()
        assert oracle.rel_err(a, b) <= 1e-10
        a32, _, h32, _ = run(cuda_lib, n, 64, "float32", seed=9, mapping=mapping)
        x32 = [torch.from_numpy(h32[k].astype(np.float32)).cuda() for k in ("q", "qd", "tau")]
        b32 = cuda_lib.aba(model, *x32, flags=cuda_lib.RD_ABA_THREAD_PER_INSTANCE).cpu().numpy()
        assert oracle.rel_err(a32, b32) <= 1e-5


def test_pair_fd_status_word(cuda_lib, mapping):
    """A point mass on the last axis: Omega_n = 0 sets RD_WARN_SINGULAR and
    nothing else; a regular chain reports 0 (no wait ran out)."""
    import torch

    ch = chaingen.make_chain(4, seed=5)
    ch.S[3] = [0.0, 0.0, 0.0, 0.0, 0.0, 1.0]
    ch.inertia[3] = [1.0, 0.0, 0.0, 0.2, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0]
    model = cuda_lib.Model(ch)
    x = torch.zeros((6, 4), dtype=torch.float32, device="cuda")
    status = torch.full((6,), -7, dtype=torch.int32, device="cuda")
    cuda_lib.aba(model, x, x, x + 1.0, status=status, flags=mapping)
    assert torch.all(status == cuda_lib.RD_WARN_SINGULAR)
    ok = torch.full((40,), -7, dtype=torch.int32, device="cuda")
    qdd, _, _, _ = run(cuda_lib, 80, 40, "float32", status=ok, mapping=mapping)
    assert torch.all(ok == 0)


@pytest.mark.parametrize("n", [64, 100])
def test_pair_fd_workload_batch_sampled(cuda_lib, mapping, n):
    """B = 16384 in FP32 (double-float updates): every 64th instance against the
    oracle."""
    qdd, ch, h, _ = run(cuda_lib, n, 16384, "float32", seed=1609, mapping=mapping)
    idx = np.arange(0, 16384, 64)
    ref = oracle.fd_aba(ch, h["q"][idx], h["qd"][idx], h["tau"][idx])
    assert oracle.rel_err(qdd[idx], ref) <= TOL["float32"]


def test_pair_fd_rejects_conflicting_flags(cuda_lib, mapping):
    import torch

    model = cuda_lib.Model(chaingen.make_chain(6))
    x = torch.zeros((4, 6), device="cuda")
    other_map = cuda_lib.RD_ABA_THREE_WARPS if mapping == cuda_lib.RD_ABA_TWO_WARPS \
        else cuda_lib.RD_ABA_TWO_WARPS
    for other in (cuda_lib.RD_ABA_WARP_PER_INSTANCE, cuda_lib.RD_ABA_THREAD_PER_INSTANCE,
                  cuda_lib.RD_ABA_JOINT_FRAMES, cuda_lib.RD_ABA_SCANS_IN_DTYPE, other_map):
        with pytest.raises(cuda_lib.RdError):
            cuda_lib.aba(model, x, x, x, flags=mapping | other)


@pytest.mark.parametrize("flags", [0, 0x4, 0x8])
def test_three_warps_agree_with_two(cuda_lib, flags):
    """The split inertia update performs the two-warp kernel's operations on the
    same operands: FP64 data agree to rounding, FP32 data (double-float, FP64 or
    extended-bias updates) to an ulp or two of the output."""
    import torch

    for n in (1, 5, 31, 64, 77):
        for dtype, tol in (("float64", 1e-12), ("float32", 2e-6)):
            if dtype == "float64" and flags:
                continue
            a, ch, h, model = run(cuda_lib, n, 96, dtype, seed=17, flags=flags,
                                  mapping=cuda_lib.RD_ABA_THREE_WARPS)
            b, _, _, _ = run(cuda_lib, n, 96, dtype, seed=17, flags=flags,
                             mapping=cuda_lib.RD_ABA_TWO_WARPS)
            assert np.max(np.abs(a - b)) <= tol * max(np.max(np.abs(b)), 1.0), (n, dtype, flags)


@pytest.mark.parametrize("n,B,prec,expect", [(64, 1024, 0, "three"), (64, 8192, 0, "two"),
                                              (32, 4096, 0x4, "three"), (32, 16384, 0x4, "two"),
                                              (80, 1536, 0, "two")])
def test_auto_picks_the_measured_mapping(cuda_lib, n, B, prec, expect):
    """Without a mapping flag the library takes three warps up to the measured
    crossover (double-float updates: B <= 2048 with FP32 bias sweeps; FP64
    updates: B <= 4096) and two beyond it: the AUTO result equals that
    mapping's bit for bit."""
    import torch

    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED + 9 * n)
    st = chaingen.make_states(B, n, seed=23, kinds=("q", "qd", "tau"))
    x = [torch.from_numpy(st[k].astype(np.float32)).cuda() for k in ("q", "qd", "tau")]
    model = cuda_lib.Model(ch)
    auto = cuda_lib.aba(model, *x, flags=prec)
    flag = {"two": cuda_lib.RD_ABA_TWO_WARPS, "three": cuda_lib.RD_ABA_THREE_WARPS}[expect]
    pick = cuda_lib.aba(model, *x, flags=prec | flag)
    assert torch.equal(auto, pick)


def test_bounded_wait_runs_out_and_reports(cuda_lib):
    """RD_ABA_TEST_WITHHOLD: warp J announces nothing, so warp Z's bounded wait
    runs out once per instance; the call returns, every status word carries
    RD_WARN_TIMEOUT, and the context stays usable (the next call matches the
    oracle). No wait in the library is unbounded."""
    import torch

    ch = chaingen.make_chain(8, seed=3)
    model = cuda_lib.Model(ch)
    st = chaingen.make_states(40, 8, seed=2, kinds=("q", "qd", "tau"))
    x = [torch.from_numpy(st[k].astype(np.float32)).cuda() for k in ("q", "qd", "tau")]
    status = torch.full((40,), -7, dtype=torch.int32, device="cuda")
    cuda_lib.aba(model, *x, status=status,
                 flags=cuda_lib.RD_ABA_TWO_WARPS | cuda_lib.RD_ABA_TEST_WITHHOLD)
    torch.cuda.synchronize()
    assert torch.all((status & cuda_lib.RD_WARN_TIMEOUT) != 0)
    ok = torch.full((40,), -7, dtype=torch.int32, device="cuda")
    qdd = cuda_lib.aba(model, *x, status=ok, flags=cuda_lib.RD_ABA_TWO_WARPS).cpu().double().numpy()
    assert torch.all(ok == 0)
    h = {k: st[k].astype(np.float32).astype(np.float64) for k in ("q", "qd", "tau")}
    ref = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"])
    assert oracle.rel_err(qdd, ref) <= TOL["float32"]


def test_withhold_hook_needs_two_warps(cuda_lib):
    import torch

    model = cuda_lib.Model(chaingen.make_chain(6))
    x = torch.zeros((4, 6), device="cuda")
    for other in (0, cuda_lib.RD_ABA_THREE_WARPS, cuda_lib.RD_ABA_THREAD_PER_INSTANCE):
        with pytest.raises(cuda_lib.RdError):
            cuda_lib.aba(model, x, x, x, flags=cuda_lib.RD_ABA_TEST_WITHHOLD | other)


@pytest.mark.parametrize("prec", [0, 0x4])
@pytest.mark.parametrize("n", [16, 64])
def test_bench_fd_configuration_sampled(cuda_lib, n, prec):
    """The bench's forward-dynamics lines as launched: FP32 data, B = 16384, no
    mapping flag (the library picks two warps per 32 instances at this batch),
    double-float or FP64 updates (RD_ABA_FP64_UPDATE); every 64th instance
    against the oracle, the rest finite."""
    qdd, ch, h, _ = run(cuda_lib, n, 16384, "float32", seed=6000, flags=prec, mapping=0)
    assert np.all(np.isfinite(qdd))
    idx = np.arange(0, 16384, 64)
    ref = oracle.fd_aba(ch, h["q"][idx], h["qd"][idx], h["tau"][idx])
    assert oracle.rel_err(qdd[idx], ref) <= TOL["float32"]


def test_empty_batch(cuda_lib, mapping):
    """B = 0 with the mapping flag set: nothing launches, the call succeeds."""
    import torch

    model = cuda_lib.Model(chaingen.make_chain(12))
    x = torch.zeros((0, 12), device="cuda")
    qdd = cuda_lib.aba(model, x, x, x, flags=mapping)
    assert qdd.shape == (0, 12)
