"""GPU parity of the partial-state inverse dynamics (RD_VARIANT_SERIAL_HYBRID:
state kept for the first K links, the rest re-derived in the backward sweep)
against the FP64 oracle, through the C ABI. Bars as for the other kernels:
FP64 <= 1e-10, FP32 <= 1e-4 of max|tau|."""
import numpy as np
import pytest

import chaingen
import oracle
from test_rnea_gpu import TOL, run_case

pytestmark = pytest.mark.gpu


def _v(rd, K, block=0):
    v = rd.RD_VARIANT_SERIAL_HYBRID | rd.RD_TUNE_STORED_LINKS(K)
    if block:
        v |= rd.RD_TUNE_BLOCK(block)
    return v


@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("n,K", [(1, 4), (2, 4), (7, 4), (7, 8), (16, 4), (16, 12), (16, 16),
                                 (31, 8), (31, 28), (32, 16), (32, 28), (33, 32), (64, 16),
                                 (100, 20), (128, 8)])
def test_hybrid_parity(cuda_lib, n, K, dtype):
    tau, ref = run_case(cuda_lib, n, 1000, dtype, _v(cuda_lib, K))
    err = oracle.rel_err(tau, ref)
    assert err <= TOL[dtype], f"n={n} K={K} {dtype}: rel err {err:.3e}"


@pytest.mark.parametrize("block", [32, 64, 128])
def test_hybrid_block_sizes(cuda_lib, block):
    for dtype in ("float32", "float64"):
        tau, ref = run_case(cuda_lib, 20, 777, dtype, _v(cuda_lib, 8, block))
        assert oracle.rel_err(tau, ref) <= TOL[dtype]


def test_hybrid_K_beyond_chain_is_the_stored_kernel(cuda_lib):
    """K >= n keeps every link's state: the arithmetic of RD_VARIANT_SERIAL."""
    a, _ = run_case(cuda_lib, 12, 500, "float64", _v(cuda_lib, 64))
    b, _ = run_case(cuda_lib, 12, 500, "float64", cuda_lib.RD_VARIANT_SERIAL)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))


@pytest.mark.parametrize("B", [1, 31, 33, 65, 257])
def test_hybrid_ragged_batches(cuda_lib, B):
    tau, ref = run_case(cuda_lib, 10, B, "float32", _v(cuda_lib, 4))
    assert oracle.rel_err(tau, ref) <= TOL["float32"]


def test_hybrid_base_motion_and_external_wrench(cuda_lib):
    base = np.array([0.2, -0.1, 0.3, 0.5, -0.4, 0.25,
                     0.3, 1.1, 9.81, -0.2, 0.4, 0.1,
                     2.0, -1.0, 0.5, 0.3, 0.2, -0.6])
    for dtype in ("float32", "float64"):
        tau, ref = run_case(cuda_lib, 9, 333, dtype, _v(cuda_lib, 4), base=base)
        assert oracle.rel_err(tau, ref) <= TOL[dtype]


def test_hybrid_unaligned_rows(cuda_lib):
    torch = pytest.importorskip("torch")
    n, B = 12, 300
    ch = chaingen.make_chain(n)
    st = chaingen.make_states(B, n, seed=3)
    model = cuda_lib.Model(ch)
    bufs = []
    for k in ("q", "qd", "qdd"):
        flat = torch.zeros(B * n + 1, dtype=torch.float32, device="cuda")
        flat[1:] = torch.from_numpy(st[k].astype(np.float32).ravel()).cuda()
        bufs.append(flat[1:].view(B, n))
    out_flat = torch.zeros(B * n + 1, dtype=torch.float32, device="cuda")
    tau = cuda_lib.rnea(model, *bufs, out=out_flat[1:].view(B, n),
                        variant=_v(cuda_lib, 4)).cpu().numpy()
    ref = oracle.rnea(ch, *(st[k].astype(np.float32).astype(np.float64) for k in ("q", "qd", "qdd")))
    assert oracle.rel_err(tau, ref) <= TOL["float32"]


@pytest.mark.parametrize("n", [8, 32])
def test_hybrid_fast_trig(cuda_lib, n):
    v = _v(cuda_lib, 4) | cuda_lib.RD_FLAG_FAST_TRIG
    tau, ref = run_case(cuda_lib, n, 1000, "float32", v)
    assert oracle.rel_err(tau, ref) <= TOL["float32"]


def test_hybrid_state_too_large_is_an_error(cuda_lib):
    """FP64 state of 128 links for 128 threads cannot fit in shared memory."""
    with pytest.raises(cuda_lib.RdError):
        run_case(cuda_lib, 128, 200, "float64", _v(cuda_lib, 128, 128))
