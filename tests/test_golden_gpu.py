"""The CUDA path, through the C ABI, against the stored golden fixtures.

The fixtures hold float32-representable joint states, so an FP32 and an FP64
run see exactly the inputs the oracle saw. Bars as the parity tests of each
entry point: inverse dynamics 1e-10 (FP64) / 1e-4 (FP32); forward dynamics
1e-8 / 1e-3; adjoint 1e-9 / 1e-3; error per instance relative to the
instance's largest stored value.
"""
import numpy as np
import pytest

import chaingen
import golden
import oracle

pytestmark = pytest.mark.gpu

RNEA_TOL = {"float32": 1e-4, "float64": 1e-10}
FD_TOL = {"float32": 1e-3, "float64": 1e-8}
VJP_TOL = {"float32": 1e-3, "float64": 1e-9}


def _dev(fx, keys, dtype):
    import torch

    dt = torch.float32 if dtype == "float32" else torch.float64
    return [torch.from_numpy(np.ascontiguousarray(fx[k])).to(dtype=dt, device="cuda") for k in keys]


def _model(rd, fx):
    return rd.Model(chaingen.Chain(fx["M"], fx["S"], fx["inertia"]))


def _host(t):
    import torch

    torch.cuda.synchronize()
    return t.cpu().double().numpy()


@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("variant", ["auto", "serial"])
@pytest.mark.parametrize("name", ["rnea_n7.txt", "rnea_n5_moving_base.txt"])
def test_rnea_matches_golden(cuda_lib, name, variant, dtype):
    rd = cuda_lib
    fx = golden.load(name)
    q, qd, qdd = _dev(fx, ("q", "qd", "qdd"), dtype)
    v = rd.RD_VARIANT_AUTO if variant == "auto" else rd.RD_VARIANT_SERIAL
    tau = rd.rnea(_model(rd, fx), q, qd, qdd, base=fx["base"], variant=v)
    err = oracle.rel_err(_host(tau), fx["tau"])
    assert err <= RNEA_TOL[dtype], f"{name} {variant} {dtype}: {err:.3e}"


@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("flags", [0, "fp64_update"])
def test_aba_matches_golden(cuda_lib, flags, dtype):
    rd = cuda_lib
    fx = golden.load("fd_n6.txt")
    q, qd, tau = _dev(fx, ("q", "qd", "tau"), dtype)
    f = rd.RD_ABA_FP64_UPDATE if flags == "fp64_update" else 0
    qdd = rd.aba(_model(rd, fx), q, qd, tau, base=fx["base"], flags=f)
    err = oracle.rel_err(_host(qdd), fx["qdd_aba"])
    assert err <= FD_TOL[dtype], f"{flags} {dtype}: {err:.3e}"


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_jsiia_matches_golden(cuda_lib, dtype):
    rd = cuda_lib
    fx = golden.load("fd_n6.txt")
    q, qd, tau = _dev(fx, ("q", "qd", "tau"), dtype)
    qdd = rd.jsiia(_model(rd, fx), q, qd, tau, base=fx["base"])
    err = oracle.rel_err(_host(qdd), fx["qdd_jsiia"])
    assert err <= FD_TOL[dtype], f"{dtype}: {err:.3e}"


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_vjp_matches_golden(cuda_lib, dtype):
    rd = cuda_lib
    fx = golden.load("vjp_n4.txt")
    q, qd, qdd, w = _dev(fx, ("q", "qd", "qdd", "w"), dtype)
    g = rd.rnea_vjp(_model(rd, fx), q, qd, qdd, w, base=fx["base"])
    got = np.concatenate([_host(x) for x in g], axis=1)
    ref = np.concatenate([fx[k] for k in ("gq", "gqd", "gqdd")], axis=1)
    err = oracle.rel_err(got, ref)
    assert err <= VJP_TOL[dtype], f"{dtype}: {err:.3e}"
