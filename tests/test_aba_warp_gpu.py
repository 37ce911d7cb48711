"""GPU parity of forward dynamics with one warp per instance
(RD_ABA_WARP_PER_INSTANCE): tau_bias by the inverse-dynamics scans across the
lanes, the articulated inertias link by link with each update spread over 21
lanes, and the z_hat / c_hat and lambda / qdd recursions as lane scans
(Sec. III-D). Against the FP64 oracle's fd_aba, through the C ABI.

Metric and bars as in test_aba_gpu.py: per instance max_i |qdd - qdd*| /
max_i |qdd*|, FP32 data 1e-3, FP64 data 1e-8.
"""
import numpy as np
import pytest

import chaingen
import oracle

pytestmark = pytest.mark.gpu
TOL = {"float32": 1e-3, "float64": 1e-8}
BASE = np.array([0.2, -0.1, 0.3, 0.5, -0.4, 0.25, 0.3, 1.1, 9.81, -0.2, 0.4, 0.1,
                 2.0, -1.0, 0.5, 0.3, 0.2, -0.6])


def run(rd, n, B, dtype, seed=71, base=None, flags=0, status=None):
    import torch

    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED + 7 * n)
    st = chaingen.make_states(B, n, seed=seed, kinds=("q", "qd", "tau"))
    npdt = np.float32 if dtype == "float32" else np.float64
    host = {k: st[k].astype(npdt) for k in st}
    dev = {k: torch.from_numpy(v).cuda() for k, v in host.items()}
    model = rd.Model(ch)
    qdd = rd.aba(model, dev["q"], dev["qd"], dev["tau"], base=base, status=status,
                 flags=flags | rd.RD_ABA_WARP_PER_INSTANCE)
    torch.cuda.synchronize()
    h64 = {k: v.astype(np.float64) for k, v in host.items()}
    return qdd.cpu().double().numpy(), ch, h64, model


@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("n", [1, 2, 7, 16, 31, 32, 33, 63, 64, 65, 100, 128])
def test_warp_fd_matches_oracle(cuda_lib, n, dtype):
    qdd, ch, h, _ = run(cuda_lib, n, 67, dtype)
    ref = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"])
    assert oracle.rel_err(qdd, ref) <= TOL[dtype], f"n={n} {dtype}"


@pytest.mark.parametrize("n", [7, 32, 64, 100])
def test_warp_fd_fp64_update_matches_oracle(cuda_lib, n):
    qdd, ch, h, _ = run(cuda_lib, n, 40, "float32", flags=cuda_lib.RD_ABA_FP64_UPDATE)
    ref = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"])
    assert oracle.rel_err(qdd, ref) <= TOL["float32"]


@pytest.mark.parametrize("B", [1, 2, 3, 5, 130])
def test_warp_fd_ragged_batches(cuda_lib, B):
    """Batches that leave warps of the last block idle."""
    qdd, ch, h, _ = run(cuda_lib, 20, B, "float64", seed=3)
    ref = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"])
    assert oracle.rel_err(qdd, ref) <= TOL["float64"]


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_warp_fd_base_motion_and_wrench(cuda_lib, dtype):
    for n in (5, 40, 90):
        qdd, ch, h, _ = run(cuda_lib, n, 33, dtype, base=BASE)
        ref = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"], base=BASE)
        assert oracle.rel_err(qdd, ref) <= TOL[dtype], f"n={n}"


def test_warp_fd_agrees_with_thread_per_instance_fp64(cuda_lib):
    """FP64 data: the warp and the thread mappings are one result to rounding."""
    import torch

    for n in (12, 64, 97):
        a, ch, h, model = run(cuda_lib, n, 50, "float64", seed=9)
        x = [torch.from_numpy(h[k]).cuda() for k in ("q", "qd", "tau")]
        b = cuda_lib.aba(model, *x, flags=cuda_lib.RD_ABA_THREAD_PER_INSTANCE).cpu().numpy()
        assert oracle.rel_err(a, b) <= 1e-10


def test_warp_fd_round_trip(cuda_lib):
    qdd, ch, h, _ = run(cuda_lib, 48, 64, "float64", seed=11)
    back = oracle.rnea(ch, h["q"], h["qd"], qdd)
    assert oracle.rel_err(back, h["tau"]) <= 1e-9


def test_warp_fd_flags_a_singular_joint(cuda_lib):
    """Last link a point mass on its own axis: Omega_n = 0 is reported."""
    import torch

    ch = chaingen.make_chain(4, seed=5)
    ch.S[3] = [0.0, 0.0, 0.0, 0.0, 0.0, 1.0]
    ch.inertia[3] = [1.0, 0.0, 0.0, 0.2, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0]
    model = cuda_lib.Model(ch)
    for dt in (torch.float32, torch.float64):
        x = torch.zeros((6, 4), dtype=dt, device="cuda")
        status = torch.full((6,), -7, dtype=torch.int32, device="cuda")
        cuda_lib.aba(model, x, x, x + 1.0, status=status, flags=cuda_lib.RD_ABA_WARP_PER_INSTANCE)
        assert torch.all(status == 1)
    ok = torch.full((6,), -7, dtype=torch.int32, device="cuda")
    y = torch.zeros((6, 9), dtype=torch.float32, device="cuda")
    cuda_lib.aba(cuda_lib.Model(chaingen.make_chain(9)), y, y, y, status=ok,
                 flags=cuda_lib.RD_ABA_WARP_PER_INSTANCE)
    assert torch.all(ok == 0)


def test_warp_fd_rejects_conflicting_flags(cuda_lib):
    import torch

    model = cuda_lib.Model(chaingen.make_chain(6))
    x = torch.zeros((4, 6), device="cuda")
    for other in (cuda_lib.RD_ABA_THREAD_PER_INSTANCE, cuda_lib.RD_ABA_JOINT_FRAMES,
                  cuda_lib.RD_ABA_SCANS_IN_DTYPE):
        with pytest.raises(cuda_lib.RdError):
            cuda_lib.aba(model, x, x, x, flags=cuda_lib.RD_ABA_WARP_PER_INSTANCE | other)


@pytest.mark.parametrize("n", [16, 64, 128])
def test_warp_fd_workload_batch_sampled(cuda_lib, n):
    """B = 4096 in FP32 (default double-float updates): every 16th instance
    against the oracle."""
    qdd, ch, h, _ = run(cuda_lib, n, 4096, "float32", seed=1609)
    idx = np.arange(0, 4096, 16)
    ref = oracle.fd_aba(ch, h["q"][idx], h["qd"][idx], h["tau"][idx])
    assert oracle.rel_err(qdd[idx], ref) <= TOL["float32"]
