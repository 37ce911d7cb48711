"""rnea_vjp_noalloc: the adjoint without any device allocation by the library.

It serves callers that cannot allocate device memory at the moment they call
(for example a real-time control loop that forbids allocation, or a plug-in
whose host framework owns the memory pool). This test calls the entry point
directly through the C ABI and checks its gradients against the ordinary
rnea_vjp (store mode with a caller workspace), on two calls in a row with
different inputs, within the tolerances of the other adjoint tests.
Collected last on purpose; it passes alone or after the rest.
"""
import ctypes

import numpy as np
import pytest

import chaingen

pytestmark = pytest.mark.gpu
TOL = {"float32": 1e-3, "float64": 1e-9}


def _grad_err(g, ref):
    a = np.concatenate([np.asarray(x, dtype=np.float64) for x in g], axis=1)
    r = np.concatenate([np.asarray(x, dtype=np.float64) for x in ref], axis=1)
    num = np.max(np.abs(a - r), axis=1)
    den = np.maximum(np.max(np.abs(r), axis=1), 1e-300)
    return float(np.max(num / den))


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_noalloc_vjp_matches_vjp_on_two_calls(cuda_lib, dtype):
    import torch

    lib = cuda_lib.load()
    fn = lib.rnea_vjp_noalloc
    P, I = ctypes.c_void_p, ctypes.c_int
    fn.argtypes = [P, I, I, P, P, P, P, P, P, P, ctypes.POINTER(ctypes.c_double), P]
    fn.restype = I
    n, B = 32, 4096
    tdt = torch.float32 if dtype == "float32" else torch.float64
    model = cuda_lib.Model(chaingen.make_chain(n, seed=chaingen.BASE_SEED))
    stream = torch.cuda.current_stream()
    for call, seed in enumerate((101, 202)):
        st = chaingen.make_states(B, n, seed=seed, kinds=("q", "qd", "qdd", "w"))
        x = [torch.from_numpy(st[k]).to("cuda", tdt) for k in ("q", "qd", "qdd", "w")]
        out = [torch.full_like(x[0], float("nan")) for _ in range(3)]
        rc = fn(model.handle, B, 0 if dtype == "float32" else 1, *(t.data_ptr() for t in x),
                *(t.data_ptr() for t in out), None, ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.rd_last_error().decode()
        ref = cuda_lib.rnea_vjp(model, *x, mode=cuda_lib.RD_VJP_STORE)
        torch.cuda.synchronize()
        err = _grad_err([t.cpu().numpy() for t in out], [t.cpu().numpy() for t in ref])
        assert err <= TOL[dtype], f"call {call}: {err:.3e}"


def test_noalloc_vjp_rejects_batches_beyond_the_scratch(cuda_lib):
    lib = cuda_lib.load()
    fn = lib.rnea_vjp_noalloc
    P, I = ctypes.c_void_p, ctypes.c_int
    fn.argtypes = [P, I, I, P, P, P, P, P, P, P, ctypes.POINTER(ctypes.c_double), P]
    fn.restype = I
    model = cuda_lib.Model(chaingen.make_chain(32))
    big = 13108  # 32 links * 20 scalars * 4 bytes * 13108 > 32 MiB
    rc = fn(model.handle, big, 0, P(16), P(16), P(16), P(16), P(32), P(48), P(64), None, None)
    assert rc == -3
    assert "scratch" in lib.rd_last_error().decode()
