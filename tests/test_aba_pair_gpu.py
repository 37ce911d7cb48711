"""GPU parity of forward dynamics with two warps per 32 instances
(RD_ABA_TWO_WARPS): one warp runs the articulated-inertia recursion of
Eq. (abi), the other the bias sweeps, tau_hat, z_hat and c_hat beside it and
then lambda / qdd (Sec. II-B). Against the FP64 oracle's fd_aba, through the
C ABI. Bars as in test_aba_gpu.py: FP32 data 1e-3, FP64 data 1e-8.
"""
import numpy as np
import pytest

import chaingen
import oracle

pytestmark = pytest.mark.gpu
TOL = {"float32": 1e-3, "float64": 1e-8}
BASE = np.array([0.2, -0.1, 0.3, 0.5, -0.4, 0.25, 0.3, 1.1, 9.81, -0.2, 0.4, 0.1,
                 2.0, -1.0, 0.5, 0.3, 0.2, -0.6])


def run(rd, n, B, dtype, seed=73, base=None, flags=0, status=None):
    import torch

    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED + 9 * n)
    st = chaingen.make_states(B, n, seed=seed, kinds=("q", "qd", "tau"))
    npdt = np.float32 if dtype == "float32" else np.float64
    host = {k: st[k].astype(npdt) for k in st}
    dev = {k: torch.from_numpy(v).cuda() for k, v in host.items()}
    model = rd.Model(ch)
    qdd = rd.aba(model, dev["q"], dev["qd"], dev["tau"], base=base, status=status,
                 flags=flags | rd.RD_ABA_TWO_WARPS)
    torch.cuda.synchronize()
    h64 = {k: v.astype(np.float64) for k, v in host.items()}
    return qdd.cpu().double().numpy(), ch, h64, model


@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("n", [1, 2, 7, 16, 33, 64, 65, 100, 128])
def test_pair_fd_matches_oracle(cuda_lib, n, dtype):
    qdd, ch, h, _ = run(cuda_lib, n, 70, dtype)
    ref = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"])
    assert oracle.rel_err(qdd, ref) <= TOL[dtype], f"n={n} {dtype}"


@pytest.mark.parametrize("n", [7, 64, 100])
def test_pair_fd_fp64_update_matches_oracle(cuda_lib, n):
    qdd, ch, h, _ = run(cuda_lib, n, 45, "float32", flags=cuda_lib.RD_ABA_FP64_UPDATE)
    ref = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"])
    assert oracle.rel_err(qdd, ref) <= TOL["float32"]


@pytest.mark.parametrize("B", [1, 31, 33, 300])
def test_pair_fd_ragged_batches(cuda_lib, B):
    """Batches that leave lanes of the last block idle."""
    qdd, ch, h, _ = run(cuda_lib, 21, B, "float64", seed=4)
    ref = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"])
    assert oracle.rel_err(qdd, ref) <= TOL["float64"]


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_pair_fd_base_motion_and_wrench(cuda_lib, dtype):
    for n in (6, 40, 90):
        qdd, ch, h, _ = run(cuda_lib, n, 37, dtype, base=BASE)
        ref = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"], base=BASE)
        assert oracle.rel_err(qdd, ref) <= TOL[dtype], f"n={n}"


def test_pair_fd_agrees_with_thread_per_instance(cuda_lib):
    """FP64 data: one result to rounding; FP32 data: the same operations in the
    same precisions, so equal to a few ulps."""
    import torch

    for n in (12, 64, 97):
        a, ch, h, model = run(cuda_lib, n, 64, "float64", seed=9)
        x = [torch.from_numpy(h[k]).cuda() for k in ("q", "qd", "tau")]
        b = cuda_lib.aba(model, *x, flags=cuda_lib.RD_ABA_THREAD_PER_INSTANCE).cpu().numpy()
        assert oracle.rel_err(a, b) <= 1e-10
        a32, _, h32, _ = run(cuda_lib, n, 64, "float32", seed=9)
        x32 = [torch.from_numpy(h32[k].astype(np.float32)).cuda() for k in ("q", "qd", "tau")]
        b32 = cuda_lib.aba(model, *x32, flags=cuda_lib.RD_ABA_THREAD_PER_INSTANCE).cpu().numpy()
        assert oracle.rel_err(a32, b32) <= 1e-5


def test_pair_fd_status_word(cuda_lib):
    """A point mass on the last axis: Omega_n = 0 sets RD_WARN_SINGULAR and
    nothing else; a regular chain reports 0 (no wait ran out)."""
    import torch

    ch = chaingen.make_chain(4, seed=5)
    ch.S[3] = [0.0, 0.0, 0.0, 0.0, 0.0, 1.0]
    ch.inertia[3] = [1.0, 0.0, 0.0, 0.2, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0]
    model = cuda_lib.Model(ch)
    x = torch.zeros((6, 4), dtype=torch.float32, device="cuda")
    status = torch.full((6,), -7, dtype=torch.int32, device="cuda")
    cuda_lib.aba(model, x, x, x + 1.0, status=status, flags=cuda_lib.RD_ABA_TWO_WARPS)
    assert torch.all(status == cuda_lib.RD_WARN_SINGULAR)
    ok = torch.full((40,), -7, dtype=torch.int32, device="cuda")
    qdd, _, _, _ = run(cuda_lib, 80, 40, "float32", status=ok)
    assert torch.all(ok == 0)


@pytest.mark.parametrize("n", [64, 100])
def test_pair_fd_workload_batch_sampled(cuda_lib, n):
    """B = 16384 in FP32 (double-float updates): every 64th instance against the
    oracle."""
    qdd, ch, h, _ = run(cuda_lib, n, 16384, "float32", seed=1609)
    idx = np.arange(0, 16384, 64)
    ref = oracle.fd_aba(ch, h["q"][idx], h["qd"][idx], h["tau"][idx])
    assert oracle.rel_err(qdd[idx], ref) <= TOL["float32"]


def test_pair_fd_rejects_conflicting_flags(cuda_lib):
    import torch

    model = cuda_lib.Model(chaingen.make_chain(6))
    x = torch.zeros((4, 6), device="cuda")
    for other in (cuda_lib.RD_ABA_WARP_PER_INSTANCE, cuda_lib.RD_ABA_THREAD_PER_INSTANCE,
                  cuda_lib.RD_ABA_JOINT_FRAMES, cuda_lib.RD_ABA_SCANS_IN_DTYPE):
        with pytest.raises(cuda_lib.RdError):
            cuda_lib.aba(model, x, x, x, flags=cuda_lib.RD_ABA_TWO_WARPS | other)
