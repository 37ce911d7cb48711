"""rnea_vjp_noalloc: the adjoint without any device allocation by the library.

It serves callers that cannot allocate device memory at the moment they call,
for example a real-time control loop that forbids allocation, or a plug-in
whose host framework owns the memory pool. These tests call the entry point
directly through the C ABI, on two calls in a row with different inputs:
* against the FP64 oracle's gradient, on sampled rows that include the last
  rows of the batch (the tail of the fixed scratch array);
* bit for bit against rnea_vjp in store mode with a caller workspace, which
  runs the same kernel;
* at the largest batch the scratch holds, and one state beyond it, which must
  be rejected.
Collected last on purpose; they pass alone or after the rest.
"""
import ctypes

import numpy as np
import pytest

import chaingen
import oracle
from gradcheck import grad_err

pytestmark = pytest.mark.gpu
TOL = {"float32": 1e-3, "float64": 1e-9}
SCRATCH = 32 << 20
N = 32


def _fn(lib):
    fn = lib.rnea_vjp_noalloc
    P, I = ctypes.c_void_p, ctypes.c_int
    fn.argtypes = [P, I, I, P, P, P, P, P, P, P, ctypes.POINTER(ctypes.c_double), P]
    fn.restype = I
    return fn


def _max_batch(dtype):
    return SCRATCH // (N * 20 * (4 if dtype == "float32" else 8))


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_noalloc_vjp_matches_oracle_and_store_mode_on_two_calls(cuda_lib, dtype):
    import torch

    lib = cuda_lib.load()
    fn = _fn(lib)
    tdt = torch.float32 if dtype == "float32" else torch.float64
    ch = chaingen.make_chain(N, seed=chaingen.BASE_SEED)
    model = cuda_lib.Model(ch)
    stream = torch.cuda.current_stream()
    bmax = _max_batch(dtype)  # 13107 in FP32, 6553 in FP64
    for call, (seed, B) in enumerate(((101, 4096), (202, bmax))):
        st = chaingen.make_states(B, N, seed=seed, kinds=("q", "qd", "qdd", "w"))
        x = [torch.from_numpy(st[k]).to("cuda", tdt) for k in ("q", "qd", "qdd", "w")]
        out = [torch.full_like(x[0], float("nan")) for _ in range(3)]
        rc = fn(model.handle, B, 0 if dtype == "float32" else 1, *(t.data_ptr() for t in x),
                *(t.data_ptr() for t in out), None, ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.rd_last_error().decode()
        ref = cuda_lib.rnea_vjp(model, *x, mode=cuda_lib.RD_VJP_STORE)
        torch.cuda.synchronize()
        got = [t.cpu().numpy() for t in out]
        same = [t.cpu().numpy() for t in ref]
        for a, b in zip(got, same):
            assert np.array_equal(a, b), f"call {call}: differs from store mode"
        idx = np.unique(np.concatenate([np.arange(0, 32), np.arange(0, B, 97),
                                        np.arange(B - 64, B)]))
        h = [x_.cpu().double().numpy()[idx] for x_ in x]
        want = oracle.rnea_grad(ch, *h)
        err = grad_err([a[idx] for a in got], want)
        assert err <= TOL[dtype], f"call {call} (B = {B}): {err:.3e}"


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_noalloc_vjp_rejects_one_state_beyond_the_scratch(cuda_lib, dtype):
    """B = max + 1 on real, correctly sized buffers: the call returns
    RD_ERR_RANGE and leaves the outputs untouched."""
    import torch

    lib = cuda_lib.load()
    fn = _fn(lib)
    tdt = torch.float32 if dtype == "float32" else torch.float64
    model = cuda_lib.Model(chaingen.make_chain(N))
    big = _max_batch(dtype) + 1
    x = [torch.zeros((big, N), dtype=tdt, device="cuda") for _ in range(4)]
    out = [torch.full_like(x[0], float("nan")) for _ in range(3)]
    stream = torch.cuda.current_stream()
    rc = fn(model.handle, big, 0 if dtype == "float32" else 1, *(t.data_ptr() for t in x),
            *(t.data_ptr() for t in out), None, ctypes.c_void_p(stream.cuda_stream))
    assert rc == -3  # RD_ERR_RANGE
    assert "scratch" in lib.rd_last_error().decode()
    torch.cuda.synchronize()
    assert all(bool(torch.isnan(t).all()) for t in out)
