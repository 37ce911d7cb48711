"""GPU parity of jsiia_batch (forward dynamics by joint-space-inertia inversion,
Algorithm 2) against the FP64 oracle, through the C ABI. Bars as aba_batch."""
import numpy as np
import pytest

import chaingen
import oracle

pytestmark = pytest.mark.gpu
TOL = {"float32": 1e-3, "float64": 1e-8}


def run(rd, n, B, dtype, seed=41, base=None, chain=None, status=None):
    import torch

    ch = chain or chaingen.make_chain(n, seed=chaingen.BASE_SEED + 7 * n)
    st = chaingen.make_states(B, n, seed=seed, kinds=("q", "qd", "tau"))
    npdt = np.float32 if dtype == "float32" else np.float64
    host = {k: st[k].astype(npdt) for k in st}
    dev = {k: torch.from_numpy(v).cuda() for k, v in host.items()}
    model = rd.Model(ch)
    qdd = rd.jsiia(model, dev["q"], dev["qd"], dev["tau"], base=base, status=status)
    torch.cuda.synchronize()
    return qdd.cpu().double().numpy(), ch, {k: v.astype(np.float64) for k, v in host.items()}, model, dev


@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("n", [1, 2, 7, 16, 31, 32])
def test_jsiia_matches_oracle(cuda_lib, n, dtype):
    qdd, ch, h, _, _ = run(cuda_lib, n, 130, dtype)
    ref, st = oracle.fd_jsiia(ch, h["q"], h["qd"], h["tau"])
    assert np.all(st == 0)
    assert oracle.rel_err(qdd, ref) <= TOL[dtype], f"n={n} {dtype}"
    ref2 = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"])
    assert oracle.rel_err(qdd, ref2) <= TOL[dtype]


def test_jsiia_equals_aba_on_the_gpu_fp64(cuda_lib):
    qdd, ch, h, model, dev = run(cuda_lib, 20, 300, "float64", seed=3)
    other = cuda_lib.aba(model, dev["q"], dev["qd"], dev["tau"]).cpu().numpy()
    assert oracle.rel_err(qdd, other) <= 1e-9


def test_jsiia_base_motion_and_wrench(cuda_lib):
    base = np.array([0.2, -0.1, 0.3, 0.5, -0.4, 0.25, 0.3, 1.1, 9.81, -0.2, 0.4, 0.1,
                     2.0, -1.0, 0.5, 0.3, 0.2, -0.6])
    qdd, ch, h, _, _ = run(cuda_lib, 9, 70, "float64", base=base)
    ref, _ = oracle.fd_jsiia(ch, h["q"], h["qd"], h["tau"], base=base)
    assert oracle.rel_err(qdd, ref) <= TOL["float64"]


def test_jsiia_flags_a_singular_inertia(cuda_lib):
    import torch

    model = cuda_lib.Model(chaingen.pendulum(1.0, 0.0, 0.0))
    x = torch.zeros((6, 1), dtype=torch.float64, device="cuda")
    status = torch.full((6,), -1, dtype=torch.int32, device="cuda")
    cuda_lib.jsiia(model, x, x, x + 1.0, status=status)
    assert torch.all(status == 1)


def test_jsiia_rejects_long_chains(cuda_lib):
    import torch

    model = cuda_lib.Model(chaingen.make_chain(33))
    x = torch.zeros((4, 33), device="cuda")
    with pytest.raises(cuda_lib.RdError):
        cuda_lib.jsiia(model, x, x, x)


def test_forward_dynamics_auto_dispatch(cuda_lib):
    import torch

    for n, B in ((8, 512), (40, 256), (8, 8192)):
        ch = chaingen.make_chain(n, seed=11)
        st = chaingen.make_states(B, n, seed=12, kinds=("q", "qd", "tau"))
        x = [torch.from_numpy(st[k].astype(np.float32)).cuda() for k in ("q", "qd", "tau")]
        model = cuda_lib.Model(ch)
        auto = cuda_lib.forward_dynamics(model, *x)
        assert torch.equal(auto, cuda_lib.aba(model, *x))  # auto takes the ABA
        ref = oracle.fd_aba(ch, *(a.cpu().double().numpy() for a in x))
        assert oracle.rel_err(auto.cpu().double().numpy(), ref) <= TOL["float32"]
