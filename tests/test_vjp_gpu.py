"""GPU parity of rnea_vjp (the adjoint of the two scans) against the oracle's
complex-step gradient and FP64 central differences, through the C ABI.

Metric (tests/gradcheck.py): per instance, each of gq, gqd and gqdd on its own
scale, max|g - g*| / max|g*|, with a floor of 0.1% of the instance's largest
gradient (a single gradient can vanish identically, d tau / d qd of one
revolute joint); the largest over the outputs and the batch.
Bars: FP64 1e-9, FP32 1e-3.
"""
import numpy as np
import pytest

import chaingen
import oracle
from gradcheck import grad_err

pytestmark = pytest.mark.gpu
TOL = {"float32": 1e-3, "float64": 1e-9}


def run(rd, n, B, dtype, mode, seed=3, base=None, chain=None):
    import torch

    ch = chain or chaingen.make_chain(n, seed=chaingen.BASE_SEED + 3 * n)
    st = chaingen.make_states(B, n, seed=seed, kinds=("q", "qd", "qdd", "w"))
    npdt = np.float32 if dtype == "float32" else np.float64
    host = {k: st[k].astype(npdt) for k in st}
    dev = {k: torch.from_numpy(v).cuda() for k, v in host.items()}
    model = rd.Model(ch)
    g = rd.rnea_vjp(model, dev["q"], dev["qd"], dev["qdd"], dev["w"], base=base, mode=mode)
    torch.cuda.synchronize()
    ref = oracle.rnea_grad(ch, *(host[k].astype(np.float64) for k in ("q", "qd", "qdd", "w")),
                           base=base)
    return [x.cpu().double().numpy() for x in g], ref, ch, host


@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("n", [1, 2, 7, 16, 33])
def test_vjp_matches_complex_step(cuda_lib, n, dtype, mode):
    g, ref, _, _ = run(cuda_lib, n, 150, dtype, mode)
    err = grad_err(g, ref)
    assert err <= TOL[dtype], f"n={n} {dtype} mode={mode}: {err:.3e}"


@pytest.mark.parametrize("mode", [1, 2])
def test_vjp_n32_fp32_and_fp64(cuda_lib, mode):
    for dt in ("float32", "float64"):
        g, ref, _, _ = run(cuda_lib, 32, 64, dt, mode, seed=8)
        assert grad_err(g, ref) <= TOL[dt]


def test_vjp_against_central_differences_fp64(cuda_lib):
    n, B, h = 6, 20, 1e-6
    g, _, ch, host = run(cuda_lib, n, B, "float64", 2, seed=21)
    fds = []
    for kidx, k in enumerate(("q", "qd", "qdd")):
        fd = np.empty((B, n))
        for j in range(n):
            p = {x: host[x].copy() for x in ("q", "qd", "qdd")}
            m = {x: host[x].copy() for x in ("q", "qd", "qdd")}
            p[k][:, j] += h
            m[k][:, j] -= h
            tp = oracle.rnea(ch, p["q"], p["qd"], p["qdd"])
            tm = oracle.rnea(ch, m["q"], m["qd"], m["qdd"])
            fd[:, j] = np.sum(host["w"] * (tp - tm), axis=1) / (2 * h)
        fds.append(fd)
    assert grad_err(g, fds) <= 1e-7


def test_vjp_qdd_gradient_is_mass_matrix_times_w(cuda_lib):
    g, _, ch, host = run(cuda_lib, 12, 40, "float64", 1, seed=5)
    Mq = oracle.mass_matrix(ch, host["q"])
    ref = np.einsum("bij,bj->bi", Mq, host["w"])
    assert oracle.rel_err(g[2], ref) <= 1e-10


def test_vjp_base_motion_and_wrench(cuda_lib):
    base = np.array([0.2, -0.1, 0.3, 0.5, -0.4, 0.25, 0.3, 1.1, 9.81, -0.2, 0.4, 0.1,
                     2.0, -1.0, 0.5, 0.3, 0.2, -0.6])
    for mode in (1, 2):
        g, ref, _, _ = run(cuda_lib, 9, 50, "float64", mode, base=base)
        assert grad_err(g, ref) <= TOL["float64"]


def test_vjp_store_equals_recompute(cuda_lib):
    a, _, _, _ = run(cuda_lib, 40, 300, "float64", 1, seed=4)
    b, _, _, _ = run(cuda_lib, 40, 300, "float64", 2, seed=4)
    for x, y in zip(a, b):
        assert np.max(np.abs(x - y)) <= 1e-10 * np.max(np.abs(x))


def test_vjp_store_rejects_small_workspace(cuda_lib):
    import torch

    model = cuda_lib.Model(chaingen.make_chain(5))
    x = torch.zeros((8, 5), device="cuda")
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(cuda_lib.RdError):
        cuda_lib.rnea_vjp(model, x, x, x, x, mode=cuda_lib.RD_VJP_STORE, workspace=ws)


def test_autograd_function_matches_vjp(cuda_lib):
    import torch

    n, B = 10, 64
    ch = chaingen.make_chain(n)
    st = chaingen.make_states(B, n, seed=2, kinds=("q", "qd", "qdd", "w"))
    model = cuda_lib.Model(ch)
    q, qd, qdd = (torch.from_numpy(st[k]).cuda().requires_grad_(True) for k in ("q", "qd", "qdd"))
    w = torch.from_numpy(st["w"]).cuda()
    tau = cuda_lib.rnea_autograd(model, q, qd, qdd)
    (tau * w).sum().backward()
    ref = oracle.rnea_grad(ch, st["q"], st["qd"], st["qdd"], st["w"])
    assert grad_err([t.cpu().numpy() for t in (q.grad, qd.grad, qdd.grad)], ref) <= 1e-9


def test_vjp_full_size_sampled(cuda_lib):
    """n = 32, B = 8192 FP32 (the adjoint workload), every 64th instance checked."""
    import torch

    n, B = 32, 8192
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED)
    st = chaingen.make_states(B, n, seed=99, kinds=("q", "qd", "qdd", "w"))
    host = {k: st[k].astype(np.float32) for k in st}
    dev = {k: torch.from_numpy(v).cuda() for k, v in host.items()}
    model = cuda_lib.Model(ch)
    for mode in (1, 2):
        g = cuda_lib.rnea_vjp(model, dev["q"], dev["qd"], dev["qdd"], dev["w"], mode=mode)
        idx = np.arange(0, B, 64)
        ref = oracle.rnea_grad(ch, *(host[k][idx].astype(np.float64) for k in ("q", "qd", "qdd", "w")))
        assert grad_err([a.cpu().numpy()[idx] for a in g], ref) <= TOL["float32"]


# ---- common-normal frames (rows with n % 4 == 0 and 16-byte alignment)

@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("mode", [1, 2, 2 | 0x400])
@pytest.mark.parametrize("n", [4, 8, 12, 64, 100, 128])
def test_vjp_common_normal_frames_match_complex_step(cuda_lib, n, dtype, mode):
    """Store, recompute (the library's mapping for this batch) and recompute
    with one thread per instance (RD_VJP_FLAG_ONE_THREAD = 0x400)."""
    g, ref, _, _ = run(cuda_lib, n, 150, dtype, mode, seed=13)
    err = grad_err(g, ref)
    assert err <= TOL[dtype], f"n={n} {dtype} mode={mode}: {err:.3e}"


def test_vjp_common_normal_base_motion_and_wrench(cuda_lib):
    """V_0, dV_0 and F_{n+1} converted into the recursion's frames on the host."""
    base = np.array([0.2, -0.1, 0.3, 0.5, -0.4, 0.25, 0.3, 1.1, 9.81, -0.2, 0.4, 0.1,
                     2.0, -1.0, 0.5, 0.3, 0.2, -0.6])
    for mode in (1, 2):
        g, ref, _, _ = run(cuda_lib, 8, 50, "float64", mode, base=base)
        assert grad_err(g, ref) <= TOL["float64"]


def test_vjp_frames_agree_fp64(cuda_lib):
    """The common-normal and joint-frame kernels give one gradient to rounding."""
    flag = cuda_lib.RD_VJP_FLAG_JOINT_FRAMES
    for mode in (1, 2):
        a, _, _, _ = run(cuda_lib, 24, 200, "float64", mode, seed=6)
        b, _, _, _ = run(cuda_lib, 24, 200, "float64", mode | flag, seed=6)
        for x, y in zip(a, b):
            assert np.max(np.abs(x - y)) <= 1e-10 * np.max(np.abs(x))


def test_vjp_common_normal_fast_trig(cuda_lib):
    g, ref, _, _ = run(cuda_lib, 32, 200, "float32", 2 | cuda_lib.RD_FLAG_FAST_TRIG, seed=17)
    assert grad_err(g, ref) <= TOL["float32"]


def test_vjp_recompute_large_batch_sampled(cuda_lib):
    """n = 32, B = 262144 FP32 in recompute mode (the large-batch adjoint
    workload): every 512th instance against the oracle's gradient."""
    import torch

    n, B = 32, 262144
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED)
    st = chaingen.make_states(B, n, seed=101, kinds=("q", "qd", "qdd", "w"))
    host = {k: st[k].astype(np.float32) for k in st}
    dev = {k: torch.from_numpy(v).cuda() for k, v in host.items()}
    g = cuda_lib.rnea_vjp(cuda_lib.Model(ch), dev["q"], dev["qd"], dev["qdd"], dev["w"],
                          mode=cuda_lib.RD_VJP_RECOMPUTE)
    idx = np.arange(0, B, 512)
    ref = oracle.rnea_grad(ch, *(host[k][idx].astype(np.float64) for k in ("q", "qd", "qdd", "w")))
    assert grad_err([a.cpu().numpy()[idx] for a in g], ref) <= TOL["float32"]


# ---- FP32 recompute with each instance split between two warps

@pytest.mark.parametrize("B", [1, 31, 33, 150])
@pytest.mark.parametrize("n", [4, 8, 32, 64, 100, 128])
def test_vjp_two_warps_match_complex_step(cuda_lib, n, B):
    mode = cuda_lib.RD_VJP_RECOMPUTE | cuda_lib.RD_VJP_FLAG_TWO_WARPS
    g, ref, _, _ = run(cuda_lib, n, B, "float32", mode, seed=19)
    err = grad_err(g, ref)
    assert err <= TOL["float32"], f"n={n} B={B}: {err:.3e}"


def test_vjp_two_warps_agree_with_one_thread(cuda_lib):
    """The split kernel and the one-thread kernel evaluate the same formulas."""
    rec = cuda_lib.RD_VJP_RECOMPUTE
    for n in (16, 32):
        a, ref, _, _ = run(cuda_lib, n, 3000, "float32", rec | cuda_lib.RD_VJP_FLAG_TWO_WARPS, seed=21)
        b, _, _, _ = run(cuda_lib, n, 3000, "float32", rec | cuda_lib.RD_VJP_FLAG_ONE_THREAD, seed=21)
        assert grad_err(a, ref) <= TOL["float32"] and grad_err(b, ref) <= TOL["float32"]
        assert grad_err(a, b) <= 1e-4


def test_vjp_two_warps_base_motion_wrench_and_fast_trig(cuda_lib):
    base = np.array([0.2, -0.1, 0.3, 0.5, -0.4, 0.25, 0.3, 1.1, 9.81, -0.2, 0.4, 0.1,
                     2.0, -1.0, 0.5, 0.3, 0.2, -0.6])
    mode = cuda_lib.RD_VJP_RECOMPUTE | cuda_lib.RD_VJP_FLAG_TWO_WARPS
    g, ref, _, _ = run(cuda_lib, 8, 70, "float32", mode, base=base, seed=23)
    assert grad_err(g, ref) <= TOL["float32"]
    g, ref, _, _ = run(cuda_lib, 32, 200, "float32", mode | cuda_lib.RD_FLAG_FAST_TRIG, seed=17)
    assert grad_err(g, ref) <= TOL["float32"]


@pytest.mark.parametrize("n, flag", [(32, "two"), (100, "auto")])
def test_vjp_two_warps_full_workload_sampled(cuda_lib, n, flag):
    """B = 8192 FP32 recompute split over two warps: forced at n = 32 (the
    adjoint workload's size), the library's own choice at n = 100. Every 32nd
    instance against the oracle."""
    import torch

    B = 8192
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED)
    st = chaingen.make_states(B, n, seed=5000, kinds=("q", "qd", "qdd", "w"))
    host = {k: st[k].astype(np.float32) for k in st}
    dev = {k: torch.from_numpy(v).cuda() for k, v in host.items()}
    mode = cuda_lib.RD_VJP_RECOMPUTE
    if flag == "two":
        mode |= cuda_lib.RD_VJP_FLAG_TWO_WARPS
    g = cuda_lib.rnea_vjp(cuda_lib.Model(ch), dev["q"], dev["qd"], dev["qdd"], dev["w"], mode=mode)
    idx = np.arange(0, B, 32)
    ref = oracle.rnea_grad(ch, *(host[k][idx].astype(np.float64) for k in ("q", "qd", "qdd", "w")))
    assert grad_err([a.cpu().numpy()[idx] for a in g], ref) <= TOL["float32"]


def test_vjp_split_flags_conflict(cuda_lib):
    import torch

    x = torch.zeros(4, 8, device="cuda")
    model = cuda_lib.Model(chaingen.make_chain(8, seed=3))
    mode = (cuda_lib.RD_VJP_RECOMPUTE | cuda_lib.RD_VJP_FLAG_TWO_WARPS |
            cuda_lib.RD_VJP_FLAG_ONE_THREAD)
    with pytest.raises(cuda_lib.RdError):
        cuda_lib.rnea_vjp(model, x, x, x, x, mode=mode)


# ---- lanes per instance (RD_VJP_FLAG_LANES): forward and reverse sweeps as
# scans across the lanes of each instance

def _lane_flag(rd, lanes):
    return rd.RD_VJP_RECOMPUTE | (rd.RD_VJP_FLAG_LANES4 if lanes == 4 else rd.RD_VJP_FLAG_LANES)


@pytest.mark.parametrize("lanes", [4, 8])
@pytest.mark.parametrize("n", [4, 8, 16, 32, 64, 100, 128])
@pytest.mark.parametrize("B", [1, 31])
def test_vjp_lanes_match_complex_step(cuda_lib, n, B, lanes):
    g, ref, _, _ = run(cuda_lib, n, B, "float32", _lane_flag(cuda_lib, lanes), seed=17)
    err = grad_err(g, ref)
    assert err <= TOL["float32"], f"n={n} B={B} lanes={lanes}: {err:.3e}"


@pytest.mark.parametrize("lanes", [4, 8])
def test_vjp_lanes_workload_sampled(cuda_lib, lanes):
    """n = 32, B = 8192 (the adjoint workload): every 32nd instance against the
    oracle, and all of them within 1e-4 of one thread per instance."""
    import torch

    n, B = 32, 8192
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED)
    st = chaingen.make_states(B, n, seed=5000, kinds=("q", "qd", "qdd", "w"))
    x = [torch.from_numpy(st[k]).float().cuda() for k in ("q", "qd", "qdd", "w")]
    model = cuda_lib.Model(ch)
    g = cuda_lib.rnea_vjp(model, *x, mode=_lane_flag(cuda_lib, lanes))
    h = cuda_lib.rnea_vjp(model, *x, mode=cuda_lib.RD_VJP_RECOMPUTE | cuda_lib.RD_VJP_FLAG_ONE_THREAD)
    torch.cuda.synchronize()
    idx = np.arange(0, B, 32)
    ref = oracle.rnea_grad(ch, *(a.cpu().double().numpy()[idx] for a in x))
    assert grad_err([a.cpu().numpy()[idx] for a in g], ref) <= TOL["float32"]
    assert grad_err([a.cpu().numpy() for a in g], [b.cpu().numpy() for b in h]) <= 1e-4


def test_vjp_lanes_large_batch_sampled(cuda_lib):
    """B = 262144 at n = 32 with 8 lanes per instance: sampled against the oracle."""
    import torch

    n, B = 32, 262144
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED)
    st = chaingen.make_states(B, n, seed=5001, kinds=("q", "qd", "qdd", "w"))
    x = [torch.from_numpy(st[k]).float().cuda() for k in ("q", "qd", "qdd", "w")]
    g = cuda_lib.rnea_vjp(cuda_lib.Model(ch), *x, mode=_lane_flag(cuda_lib, 8))
    torch.cuda.synchronize()
    idx = np.concatenate([np.arange(0, B, 1024), np.arange(B - 8, B)])
    ref = oracle.rnea_grad(ch, *(a.cpu().double().numpy()[idx] for a in x))
    assert grad_err([a.cpu().numpy()[idx] for a in g], ref) <= TOL["float32"]


@pytest.mark.parametrize("lanes", [4, 8])
def test_vjp_lanes_base_motion_wrench_and_fast_trig(cuda_lib, lanes):
    base = np.array([0.2, -0.1, 0.3, 0.5, -0.4, 0.25, 0.3, 1.1, 9.81, -0.2, 0.4, 0.1,
                     2.0, -1.0, 0.5, 0.3, 0.2, -0.6])
    for n in (12, 32):
        g, ref, _, _ = run(cuda_lib, n, 45, "float32", _lane_flag(cuda_lib, lanes), seed=23,
                           base=base)
        assert grad_err(g, ref) <= TOL["float32"], n
    g, ref, _, _ = run(cuda_lib, 32, 45, "float32",
                       _lane_flag(cuda_lib, lanes) | cuda_lib.RD_FLAG_FAST_TRIG, seed=24)
    assert grad_err(g, ref) <= TOL["float32"]


def test_vjp_lanes_reject_what_they_do_not_cover(cuda_lib):
    import torch

    lanes = cuda_lib.RD_VJP_FLAG_LANES
    model = cuda_lib.Model(chaingen.make_chain(6))  # n % 4 != 0
    x = torch.zeros((4, 6), device="cuda")
    with pytest.raises(cuda_lib.RdError):
        cuda_lib.rnea_vjp(model, x, x, x, x, mode=cuda_lib.RD_VJP_RECOMPUTE | lanes)
    model8 = cuda_lib.Model(chaingen.make_chain(8))
    y = torch.zeros((4, 8), device="cuda", dtype=torch.float64)
    with pytest.raises(cuda_lib.RdError):
        cuda_lib.rnea_vjp(model8, y, y, y, y, mode=cuda_lib.RD_VJP_RECOMPUTE | lanes)
    z = torch.zeros((4, 8), device="cuda")
    with pytest.raises(cuda_lib.RdError):
        cuda_lib.rnea_vjp(model8, z, z, z, z, mode=cuda_lib.RD_VJP_STORE | lanes)
    with pytest.raises(cuda_lib.RdError):
        cuda_lib.rnea_vjp(model8, z, z, z, z,
                          mode=cuda_lib.RD_VJP_RECOMPUTE | lanes | cuda_lib.RD_VJP_FLAG_TWO_WARPS)


# ---- one thread per instance with the forward state in shared memory
# (RD_VJP_FLAG_SHARED_STATE)

@pytest.mark.parametrize("n", [4, 16, 32, 64])
@pytest.mark.parametrize("B", [1, 31, 300])
def test_vjp_shared_state_matches_complex_step(cuda_lib, n, B):
    mode = cuda_lib.RD_VJP_RECOMPUTE | cuda_lib.RD_VJP_FLAG_SHARED_STATE
    g, ref, _, _ = run(cuda_lib, n, B, "float32", mode, seed=19)
    assert grad_err(g, ref) <= TOL["float32"], f"n={n} B={B}"


def test_vjp_shared_state_workload_equals_store_mode(cuda_lib):
    """n = 32, B = 8192: the same arithmetic as the workspace store mode, so
    the same result to the last bit; sampled against the oracle."""
    import torch

    n, B = 32, 8192
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED)
    st = chaingen.make_states(B, n, seed=5002, kinds=("q", "qd", "qdd", "w"))
    x = [torch.from_numpy(st[k]).float().cuda() for k in ("q", "qd", "qdd", "w")]
    model = cuda_lib.Model(ch)
    g = cuda_lib.rnea_vjp(model, *x, mode=cuda_lib.RD_VJP_RECOMPUTE | cuda_lib.RD_VJP_FLAG_SHARED_STATE)
    h = cuda_lib.rnea_vjp(model, *x, mode=cuda_lib.RD_VJP_STORE)
    torch.cuda.synchronize()
    for a, b in zip(g, h):
        assert torch.equal(a, b)
    idx = np.arange(0, B, 64)
    ref = oracle.rnea_grad(ch, *(a.cpu().double().numpy()[idx] for a in x))
    assert grad_err([a.cpu().numpy()[idx] for a in g], ref) <= TOL["float32"]


def test_vjp_shared_state_rejects_what_it_does_not_cover(cuda_lib):
    import torch

    flag = cuda_lib.RD_VJP_FLAG_SHARED_STATE
    m100 = cuda_lib.Model(chaingen.make_chain(100))
    x = torch.zeros((4, 100), device="cuda")
    with pytest.raises(cuda_lib.RdError):
        cuda_lib.rnea_vjp(m100, x, x, x, x, mode=cuda_lib.RD_VJP_RECOMPUTE | flag)
    m8 = cuda_lib.Model(chaingen.make_chain(8))
    z = torch.zeros((4, 8), device="cuda")
    with pytest.raises(cuda_lib.RdError):
        cuda_lib.rnea_vjp(m8, z, z, z, z, mode=cuda_lib.RD_VJP_STORE | flag)
    with pytest.raises(cuda_lib.RdError):
        cuda_lib.rnea_vjp(m8, z, z, z, z, mode=cuda_lib.RD_VJP_RECOMPUTE | flag |
                          cuda_lib.RD_VJP_FLAG_LANES)


# ---- two warps per 32 instances with the state in shared memory
# (RD_VJP_FLAG_TWO_WARPS_SHARED): motion, wrench and dVbar on one warp, the
# adjoint weight and Vbar (with its own dVbar carry) on the other

def _duo(rd):
    return rd.RD_VJP_RECOMPUTE | rd.RD_VJP_FLAG_TWO_WARPS_SHARED


@pytest.mark.parametrize("n", [4, 8, 16, 32, 36, 64])
@pytest.mark.parametrize("B", [1, 31, 33, 300])
def test_vjp_duo_matches_complex_step(cuda_lib, n, B):
    g, ref, _, _ = run(cuda_lib, n, B, "float32", _duo(cuda_lib), seed=29)
    assert grad_err(g, ref) <= TOL["float32"], f"n={n} B={B}"


def test_vjp_duo_base_motion_wrench_and_fast_trig(cuda_lib):
    base = np.array([0.2, -0.1, 0.3, 0.5, -0.4, 0.25, 0.3, 1.1, 9.81, -0.2, 0.4, 0.1,
                     2.0, -1.0, 0.5, 0.3, 0.2, -0.6])
    g, ref, _, _ = run(cuda_lib, 12, 70, "float32", _duo(cuda_lib), base=base, seed=23)
    assert grad_err(g, ref) <= TOL["float32"]
    g, ref, _, _ = run(cuda_lib, 32, 200, "float32", _duo(cuda_lib) | cuda_lib.RD_FLAG_FAST_TRIG,
                       seed=17)
    assert grad_err(g, ref) <= TOL["float32"]


def test_vjp_duo_workload_agrees_with_shared_state(cuda_lib):
    """n = 32, B = 8192 (the adjoint workload): the same formulas as the
    one-thread kernel with its state in shared memory, split over two warps;
    gqdd and the terms agree to the last bits (the two warps evaluate the same
    operations, the compiler may contract a sum differently), and a sample
    matches the oracle."""
    import torch

    n, B = 32, 8192
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED)
    st = chaingen.make_states(B, n, seed=5003, kinds=("q", "qd", "qdd", "w"))
    x = [torch.from_numpy(st[k]).float().cuda() for k in ("q", "qd", "qdd", "w")]
    model = cuda_lib.Model(ch)
    g = cuda_lib.rnea_vjp(model, *x, mode=_duo(cuda_lib))
    h = cuda_lib.rnea_vjp(model, *x, mode=cuda_lib.RD_VJP_RECOMPUTE |
                          cuda_lib.RD_VJP_FLAG_SHARED_STATE)
    torch.cuda.synchronize()
    for a, b in zip(g, h):
        scale = float(b.abs().max())
        assert float((a - b).abs().max()) <= 1e-5 * scale
    idx = np.arange(0, B, 64)
    ref = oracle.rnea_grad(ch, *(a.cpu().double().numpy()[idx] for a in x))
    assert grad_err([a.cpu().numpy()[idx] for a in g], ref) <= TOL["float32"]


def test_vjp_duo_rejects_what_it_does_not_cover(cuda_lib):
    import torch

    flag = cuda_lib.RD_VJP_FLAG_TWO_WARPS_SHARED
    m100 = cuda_lib.Model(chaingen.make_chain(100))
    x = torch.zeros((4, 100), device="cuda")
    with pytest.raises(cuda_lib.RdError):
        cuda_lib.rnea_vjp(m100, x, x, x, x, mode=cuda_lib.RD_VJP_RECOMPUTE | flag)
    m8 = cuda_lib.Model(chaingen.make_chain(8))
    z = torch.zeros((4, 8), device="cuda")
    for other in (cuda_lib.RD_VJP_FLAG_LANES, cuda_lib.RD_VJP_FLAG_TWO_WARPS,
                  cuda_lib.RD_VJP_FLAG_ONE_THREAD, cuda_lib.RD_VJP_FLAG_SHARED_STATE,
                  cuda_lib.RD_VJP_FLAG_JOINT_FRAMES):
        with pytest.raises(cuda_lib.RdError):
            cuda_lib.rnea_vjp(m8, z, z, z, z, mode=cuda_lib.RD_VJP_RECOMPUTE | flag | other)
    with pytest.raises(cuda_lib.RdError):
        cuda_lib.rnea_vjp(m8, z, z, z, z, mode=cuda_lib.RD_VJP_STORE | flag)
    m7 = cuda_lib.Model(chaingen.make_chain(7))
    y = torch.zeros((4, 7), device="cuda")
    with pytest.raises(cuda_lib.RdError):
        cuda_lib.rnea_vjp(m7, y, y, y, y, mode=cuda_lib.RD_VJP_RECOMPUTE | flag)


@pytest.mark.parametrize("n,B,flag", [(48, 2048, "duo"), (64, 4096, "duo"), (64, 8192, "pair"),
                                      (32, 8192, "shared")])
def test_vjp_auto_picks_the_measured_mapping(cuda_lib, n, B, flag):
    """FP32 recompute without a mapping flag follows the measured crossover:
    the AUTO result equals the chosen mapping's bit for bit."""
    import torch

    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED)
    st = chaingen.make_states(B, n, seed=41, kinds=("q", "qd", "qdd", "w"))
    x = [torch.from_numpy(st[k]).float().cuda() for k in ("q", "qd", "qdd", "w")]
    model = cuda_lib.Model(ch)
    rec = cuda_lib.RD_VJP_RECOMPUTE
    pick = {"duo": cuda_lib.RD_VJP_FLAG_TWO_WARPS_SHARED, "pair": cuda_lib.RD_VJP_FLAG_TWO_WARPS,
            "shared": cuda_lib.RD_VJP_FLAG_SHARED_STATE}[flag]
    a = cuda_lib.rnea_vjp(model, *x, mode=rec)
    b = cuda_lib.rnea_vjp(model, *x, mode=rec | pick)
    for u, v in zip(a, b):
        assert torch.equal(u, v)


def test_vjp_duo_empty_batch(cuda_lib):
    import torch

    model = cuda_lib.Model(chaingen.make_chain(16))
    x = torch.zeros((0, 16), device="cuda")
    g = cuda_lib.rnea_vjp(model, x, x, x, x, mode=_duo(cuda_lib))
    assert all(t.shape == (0, 16) for t in g)
