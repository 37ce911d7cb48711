"""GPU parity of aba_batch (forward dynamics, articulated-body algorithm)
against the FP64 oracle's ABA and JSIIA, through the C ABI; round trip
ID(FD(tau)) = tau.

Metric: per instance max_i |qdd - qdd*| / max_i |qdd*|, max over the batch.
Bars: FP32 data 1e-3 (inertia update and Omega solves in double-float
arithmetic by default, or FP64); FP64 1e-8 (FD amplifies rounding by the
conditioning of M(q)).
"""
import numpy as np
import pytest

import chaingen
import oracle

pytestmark = pytest.mark.gpu
TOL = {"float32": 1e-3, "float64": 1e-8}
AUTO = 1 << 40  # test-only marker (stripped before the call): leave the mapping to the library


def run(rd, n, B, dtype, seed=31, base=None, chain=None, status=None, flags=0):
    import torch

    ch = chain or chaingen.make_chain(n, seed=chaingen.BASE_SEED + 5 * n)
    st = chaingen.make_states(B, n, seed=seed, kinds=("q", "qd", "tau"))
    npdt = np.float32 if dtype == "float32" else np.float64
    host = {k: st[k].astype(npdt) for k in st}
    dev = {k: torch.from_numpy(v).cuda() for k, v in host.items()}
    model = rd.Model(ch)
    # this file covers the thread-per-instance kernels (test_aba_warp_gpu.py the
    # warp ones): pin the mapping unless the test asks for AUTO
    if not flags & AUTO:
        flags |= rd.RD_ABA_THREAD_PER_INSTANCE
    qdd = rd.aba(model, dev["q"], dev["qd"], dev["tau"], base=base, status=status,
                 flags=flags & ~AUTO)
    torch.cuda.synchronize()
    h64 = {k: v.astype(np.float64) for k, v in host.items()}
    return qdd.cpu().double().numpy(), ch, h64, model


def test_aba_auto_mapping_matches_oracle(cuda_lib):
    """Without a mapping flag the library takes one warp per instance for long
    chains in small batches and one thread per instance otherwise; both agree
    with the oracle."""
    for n, B in ((64, 256), (100, 1024), (64, 2048), (16, 256)):
        qdd, ch, h, _ = run(cuda_lib, n, B, "float32", seed=5, flags=AUTO)
        idx = np.arange(0, B, max(1, B // 128))
        ref = oracle.fd_aba(ch, h["q"][idx], h["qd"][idx], h["tau"][idx])
        assert oracle.rel_err(qdd[idx], ref) <= TOL["float32"], (n, B)


@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("n", [1, 2, 7, 16, 33, 64, 100])
def test_aba_matches_oracle(cuda_lib, n, dtype):
    qdd, ch, h, _ = run(cuda_lib, n, 300, dtype)
    ref = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"], base=None)
    assert oracle.rel_err(qdd, ref) <= TOL[dtype], f"n={n} {dtype}"


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_aba_matches_jsiia_and_round_trip(cuda_lib, dtype):
    qdd, ch, h, _ = run(cuda_lib, 24, 120, dtype, seed=3)
    ref, status = oracle.fd_jsiia(ch, h["q"], h["qd"], h["tau"])
    assert np.all(status == 0)
    assert oracle.rel_err(qdd, ref) <= TOL[dtype]
    back = oracle.rnea(ch, h["q"], h["qd"], qdd)
    assert oracle.rel_err(back, h["tau"]) <= (1e-3 if dtype == "float32" else 1e-9)


def test_aba_gpu_round_trip_through_rnea_fp64(cuda_lib):
    """FD on the GPU, then ID on the GPU, recovers tau."""
    import torch

    qdd, ch, h, model = run(cuda_lib, 40, 200, "float64", seed=17)
    dev = [torch.from_numpy(h[k]).cuda() for k in ("q", "qd")]
    tau = cuda_lib.rnea(model, dev[0], dev[1], torch.from_numpy(qdd).cuda())
    assert oracle.rel_err(tau.cpu().numpy(), h["tau"]) <= 1e-9


def test_aba_base_motion_and_wrench(cuda_lib):
    base = np.array([0.2, -0.1, 0.3, 0.5, -0.4, 0.25, 0.3, 1.1, 9.81, -0.2, 0.4, 0.1,
                     2.0, -1.0, 0.5, 0.3, 0.2, -0.6])
    qdd, ch, h, _ = run(cuda_lib, 11, 90, "float64", base=base)
    ref = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"], base=base)
    assert oracle.rel_err(qdd, ref) <= TOL["float64"]


def test_aba_single_link_closed_form(cuda_lib):
    import torch

    m, l, Ixx = 1.7, 0.45, 0.03
    model = cuda_lib.Model(chaingen.pendulum(m, l, Ixx))
    q = torch.tensor([[0.4], [-1.1], [2.5]], dtype=torch.float64, device="cuda")
    qd = torch.tensor([[0.3], [2.0], [-1.0]], dtype=torch.float64, device="cuda")
    tau = torch.tensor([[1.0], [-3.0], [0.5]], dtype=torch.float64, device="cuda")
    qdd = cuda_lib.aba(model, q, qd, tau).cpu().numpy()
    qh, th = q.cpu().numpy(), tau.cpu().numpy()
    assert np.allclose(qdd, (th - m * 9.81 * l * np.sin(qh)) / (m * l * l + Ixx), atol=1e-13)


def test_aba_flags_a_singular_joint(cuda_lib):
    """A point mass on the joint axis gives Omega = 0: the status word reports it."""
    import torch

    ch = chaingen.pendulum(1.0, 0.0, 0.0)  # centre of mass on the axis, no inertia
    model = cuda_lib.Model(ch)
    x = torch.zeros((5, 1), dtype=torch.float64, device="cuda")
    status = torch.full((5,), -7, dtype=torch.int32, device="cuda")
    cuda_lib.aba(model, x, x, x + 1.0, status=status)
    assert torch.all(status == 1)  # RD_WARN_SINGULAR
    ch2 = chaingen.make_chain(4)
    st2 = torch.full((5,), -7, dtype=torch.int32, device="cuda")
    y = torch.zeros((5, 4), dtype=torch.float64, device="cuda")
    cuda_lib.aba(cuda_lib.Model(ch2), y, y, y, status=st2)
    assert torch.all(st2 == 0)


@pytest.mark.parametrize("n", [16, 64])
def test_aba_full_batch_sampled(cuda_lib, n):
    """B = 16384 in FP32 (the forward-dynamics workload): every 32nd instance
    checked against the oracle; round trip on the same sample.

    Round-trip scale: the bias inverse dynamics runs in FP32, and with n = 64
    links under gravity the bias torques near the base are about 1e3 times the
    applied tau ~ N(0, 10); its rounding is relative to those torques. So the
    residual is measured per instance against max(max|tau|, max|tau_bias|),
    the magnitude of the terms that cancel in tau_hat = tau - tau_bias."""
    qdd, ch, h, _ = run(cuda_lib, n, 16384, "float32", seed=1609)
    idx = np.arange(0, 16384, 32)
    ref = oracle.fd_aba(ch, h["q"][idx], h["qd"][idx], h["tau"][idx])
    assert oracle.rel_err(qdd[idx], ref) <= TOL["float32"]
    back = oracle.rnea(ch, h["q"][idx], h["qd"][idx], qdd[idx])
    bias = oracle.rnea(ch, h["q"][idx], h["qd"][idx], np.zeros_like(qdd[idx]))
    scale = np.maximum(np.max(np.abs(h["tau"][idx]), axis=1), np.max(np.abs(bias), axis=1))
    err = np.max(np.abs(back - h["tau"][idx]), axis=1) / scale
    assert err.max() <= 1e-4, err.max()


@pytest.mark.parametrize("n", [16, 64])
def test_aba_round_trip_on_max_tau_with_extended_bias(cuda_lib, n):
    """ID(FD(tau)) = tau relative to max|tau| itself, B = 16384 (the
    forward-dynamics workload), with the bias sweeps in double-float
    (RD_ABA_EXTENDED_BIAS). Rounding qdd to FP32 alone moves ID(qdd) by
    M(q) delta qdd, which on heavy 64-link chains is about 1e-3 of max|tau|.
    So the bar is 1e-3 or twice the residual of the oracle's own qdd rounded
    to FP32, whichever is larger (n = 16: 1e-3; n = 64: the rounding floor)."""
    B = 16384
    qdd, ch, h, _ = run(cuda_lib, n, B, "float32", seed=1609, flags=cuda_lib.RD_ABA_EXTENDED_BIAS)
    idx = np.arange(0, B, 32)
    ref = oracle.fd_aba(ch, h["q"][idx], h["qd"][idx], h["tau"][idx])
    assert oracle.rel_err(qdd[idx], ref) <= TOL["float32"]
    back = oracle.rnea(ch, h["q"][idx], h["qd"][idx], qdd[idx])
    floor_back = oracle.rnea(ch, h["q"][idx], h["qd"][idx],
                             ref.astype(np.float32).astype(np.float64))
    got, floor = oracle.rel_err(back, h["tau"][idx]), oracle.rel_err(floor_back, h["tau"][idx])
    print(f"n = {n}: round trip {got:.3e} of max|tau|; FP32-rounded oracle qdd {floor:.3e}")
    assert got <= max(1e-3, 2 * floor)
    if n == 16:
        assert got <= 1e-3


def test_aba_rejects_small_workspace(cuda_lib):
    import torch

    model = cuda_lib.Model(chaingen.make_chain(5))
    x = torch.zeros((8, 5), device="cuda")
    with pytest.raises(cuda_lib.RdError):
        cuda_lib.aba(model, x, x, x, workspace=torch.empty(8, dtype=torch.uint8, device="cuda"))


@pytest.mark.parametrize("n", [7, 16, 64])
def test_aba_fp32_scans_flag(cuda_lib, n):
    """RD_ABA_SCANS_IN_DTYPE: z_hat / lambda in FP32 (inertia update and Omega
    solves still FP64) meets the FP32 bar on qdd."""
    B = 16384 if n == 64 else 300
    qdd, ch, h, _ = run(cuda_lib, n, B, "float32", seed=1609, flags=cuda_lib.RD_ABA_SCANS_IN_DTYPE)
    idx = np.arange(0, B, max(1, B // 512))
    ref = oracle.fd_aba(ch, h["q"][idx], h["qd"][idx], h["tau"][idx])
    assert oracle.rel_err(qdd[idx], ref) <= TOL["float32"]


# ---- common-normal frames (n % 4 == 0, n <= 64, aligned rows)

@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("n", [4, 8, 12, 32, 48])
def test_aba_common_normal_frames_match_oracle(cuda_lib, n, dtype):
    qdd, ch, h, _ = run(cuda_lib, n, 300, dtype, seed=41)
    ref = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"], base=None)
    assert oracle.rel_err(qdd, ref) <= TOL[dtype], f"n={n} {dtype}"


def test_aba_common_normal_base_motion_and_wrench(cuda_lib):
    base = np.array([0.2, -0.1, 0.3, 0.5, -0.4, 0.25, 0.3, 1.1, 9.81, -0.2, 0.4, 0.1,
                     2.0, -1.0, 0.5, 0.3, 0.2, -0.6])
    qdd, ch, h, _ = run(cuda_lib, 12, 90, "float64", base=base)
    ref = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"], base=base)
    assert oracle.rel_err(qdd, ref) <= TOL["float64"]


@pytest.mark.parametrize("n", [8, 32, 64])
def test_aba_frames_agree_fp64(cuda_lib, n):
    """Common-normal and joint-frame kernels, one FP64 result to rounding."""
    a, _, _, _ = run(cuda_lib, n, 200, "float64", seed=43)
    b, _, _, _ = run(cuda_lib, n, 200, "float64", seed=43, flags=cuda_lib.RD_ABA_JOINT_FRAMES)
    assert oracle.rel_err(a, b) <= 1e-9


def test_aba_common_normal_flags_a_singular_joint(cuda_lib):
    """Last link a point mass on its own axis: Omega_n = 0 is reported."""
    import torch

    ch = chaingen.make_chain(4, seed=5)
    # last joint about z through its frame's origin, centre of mass exactly on it
    ch.S[3] = [0.0, 0.0, 0.0, 0.0, 0.0, 1.0]
    ch.inertia[3] = [1.0, 0.0, 0.0, 0.2, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0]
    model = cuda_lib.Model(ch)
    x = torch.zeros((6, 4), dtype=torch.float64, device="cuda")
    status = torch.full((6,), -7, dtype=torch.int32, device="cuda")
    cuda_lib.aba(model, x, x, x + 1.0, status=status)
    assert torch.all(status == 1)


# ---- FP32 data: double-float (default) and FP64 (RD_ABA_FP64_UPDATE) inertia
# updates and solves in the common-normal kernel

@pytest.mark.parametrize("n", [4, 8, 32, 48, 64])
def test_aba_fp64_update_matches_oracle(cuda_lib, n):
    qdd, ch, h, _ = run(cuda_lib, n, 300, "float32", seed=41, flags=cuda_lib.RD_ABA_FP64_UPDATE)
    ref = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"], base=None)
    assert oracle.rel_err(qdd, ref) <= TOL["float32"], f"n={n}"


@pytest.mark.parametrize("n", [8, 32, 64])
def test_aba_double_float_agrees_with_fp64_update(cuda_lib, n):
    """The double-float and FP64 inertia updates differ by a few units of 2^-48
    relative per operation, far below the FP32 rounding of qdd: the two FP32
    outputs agree to a few FP32 ulps."""
    a, _, _, _ = run(cuda_lib, n, 512, "float32", seed=47, flags=cuda_lib.RD_ABA_FP64_UPDATE)
    b, _, _, _ = run(cuda_lib, n, 512, "float32", seed=47)
    assert oracle.rel_err(a, b) <= 1e-5


def test_aba_fp64_update_full_batch_sampled(cuda_lib):
    """B = 16384, n = 64 with the FP64 update: the bars of
    test_aba_full_batch_sampled (which runs the double-float default)."""
    n = 64
    qdd, ch, h, _ = run(cuda_lib, n, 16384, "float32", seed=1609,
                        flags=cuda_lib.RD_ABA_FP64_UPDATE)
    idx = np.arange(0, 16384, 32)
    ref = oracle.fd_aba(ch, h["q"][idx], h["qd"][idx], h["tau"][idx])
    assert oracle.rel_err(qdd[idx], ref) <= TOL["float32"]
    back = oracle.rnea(ch, h["q"][idx], h["qd"][idx], qdd[idx])
    bias = oracle.rnea(ch, h["q"][idx], h["qd"][idx], np.zeros_like(qdd[idx]))
    scale = np.maximum(np.max(np.abs(h["tau"][idx]), axis=1), np.max(np.abs(bias), axis=1))
    err = np.max(np.abs(back - h["tau"][idx]), axis=1) / scale
    assert err.max() <= 1e-4, err.max()


def test_aba_fp64_update_with_fp32_scans(cuda_lib):
    flags = cuda_lib.RD_ABA_FP64_UPDATE | cuda_lib.RD_ABA_SCANS_IN_DTYPE
    qdd, ch, h, _ = run(cuda_lib, 16, 300, "float32", seed=53, flags=flags)
    ref = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"], base=None)
    assert oracle.rel_err(qdd, ref) <= TOL["float32"]


@pytest.mark.parametrize("fp64_update", [False, True])
def test_aba_fp32_base_motion_and_wrench(cuda_lib, fp64_update):
    flags = cuda_lib.RD_ABA_FP64_UPDATE if fp64_update else 0
    base = np.array([0.2, -0.1, 0.3, 0.5, -0.4, 0.25, 0.3, 1.1, 9.81, -0.2, 0.4, 0.1,
                     2.0, -1.0, 0.5, 0.3, 0.2, -0.6])
    qdd, ch, h, _ = run(cuda_lib, 12, 90, "float32", base=base, flags=flags)
    ref = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"], base=base)
    assert oracle.rel_err(qdd, ref) <= TOL["float32"]


def test_aba_double_float_flags_a_singular_joint(cuda_lib):
    """The exact Omega_n = 0 of test_aba_common_normal_flags_a_singular_joint,
    in FP32 data with the double-float solves."""
    import torch

    ch = chaingen.make_chain(4, seed=5)
    ch.S[3] = [0.0, 0.0, 0.0, 0.0, 0.0, 1.0]
    ch.inertia[3] = [1.0, 0.0, 0.0, 0.2, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0]
    model = cuda_lib.Model(ch)
    x = torch.zeros((6, 4), dtype=torch.float32, device="cuda")
    status = torch.full((6,), -7, dtype=torch.int32, device="cuda")
    cuda_lib.aba(model, x, x, x + 1.0, status=status)
    assert torch.all(status == 1)


# ---- FP32 data beyond the parameter-constant kernel: constants and double-float
# records in global memory (n > 64, n % 4 != 0, unaligned rows)

@pytest.mark.parametrize("n", [3, 5, 65, 100])
def test_aba_global_constant_kernel_matches_oracle(cuda_lib, n):
    qdd, ch, h, _ = run(cuda_lib, n, 400, "float32", seed=59)
    ref = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"], base=None)
    assert oracle.rel_err(qdd, ref) <= TOL["float32"], f"n={n}"


def test_aba_long_chain_n128(cuda_lib):
    """n = 128 in FP32 data, the longest chain the library takes, on the FP32
    bar 1e-3: beyond RD_ABA_EXTENDED_BIAS_LINKS the bias sweeps run in
    double-float by default (with either precision of the inertia update).
    Their FP32 version, printed beside it, misses the bar here: the bias
    torques reach about 1e4 max|tau|, and their FP32 rounding, amplified by
    the conditioning of M(q), sets the error of qdd."""
    n, B = 128, 2048
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED + 5 * n)
    a, ch, h, _ = run(cuda_lib, n, B, "float32", seed=59, chain=ch)
    b, _, _, _ = run(cuda_lib, n, B, "float32", seed=59, chain=ch, flags=cuda_lib.RD_ABA_FP64_UPDATE)
    c, _, _, _ = run(cuda_lib, n, B, "float32", seed=59, chain=ch, flags=cuda_lib.RD_ABA_FP32_BIAS)
    idx = np.arange(0, B, 4)
    ref = oracle.fd_aba(ch, h["q"][idx], h["qd"][idx], h["tau"][idx], base=None)
    ea, eb, ec = (oracle.rel_err(x[idx], ref) for x in (a, b, c))
    print(f"n = 128 FP32: extended bias {ea:.3e} (FP64 update {eb:.3e}); FP32 bias {ec:.3e}")
    assert ea <= TOL["float32"]
    assert eb <= TOL["float32"]


@pytest.mark.parametrize("n", [65, 80, 100, 112, 128])
def test_aba_extended_bias_full_batch_sampled(cuda_lib, n):
    """B = 16384 beyond 64 links (the default double-float bias sweeps):
    every 64th instance against the oracle, and the round trip on the scale of
    test_aba_full_batch_sampled."""
    B = 16384
    qdd, ch, h, _ = run(cuda_lib, n, B, "float32", seed=1609)
    idx = np.arange(0, B, 64)
    ref = oracle.fd_aba(ch, h["q"][idx], h["qd"][idx], h["tau"][idx])
    assert oracle.rel_err(qdd[idx], ref) <= TOL["float32"]
    back = oracle.rnea(ch, h["q"][idx], h["qd"][idx], qdd[idx])
    bias = oracle.rnea(ch, h["q"][idx], h["qd"][idx], np.zeros_like(qdd[idx]))
    scale = np.maximum(np.max(np.abs(h["tau"][idx]), axis=1), np.max(np.abs(bias), axis=1))
    err = np.max(np.abs(back - h["tau"][idx]), axis=1) / scale
    assert err.max() <= 1e-4, err.max()


@pytest.mark.parametrize("n", [16, 64])
def test_aba_extended_bias_flag_short_chains(cuda_lib, n):
    """RD_ABA_EXTENDED_BIAS at n <= 64 (the global-constant kernel with
    double-float bias sweeps) agrees with the oracle, with FP64 or
    double-float inertia updates."""
    for fl in (0, cuda_lib.RD_ABA_FP64_UPDATE):
        qdd, ch, h, _ = run(cuda_lib, n, 300, "float32", seed=61,
                            flags=fl | cuda_lib.RD_ABA_EXTENDED_BIAS)
        ref = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"], base=None)
        assert oracle.rel_err(qdd, ref) <= TOL["float32"]


def test_aba_joint_frames_fp32_rejects_long_chains(cuda_lib):
    """The joint-frame comparison kernel keeps FP32 bias sweeps, so for FP32
    data it takes at most RD_ABA_EXTENDED_BIAS_LINKS links."""
    import torch

    model = cuda_lib.Model(chaingen.make_chain(65))
    x = torch.zeros((4, 65), device="cuda")
    with pytest.raises(cuda_lib.RdError):
        cuda_lib.aba(model, x, x, x, flags=cuda_lib.RD_ABA_JOINT_FRAMES)


def test_aba_global_constant_kernel_unaligned_rows_and_base(cuda_lib):
    """Rows off a 16-byte boundary (element loads), with base motion and an end
    wrench."""
    import torch

    n, B = 8, 300
    base = np.array([0.2, -0.1, 0.3, 0.5, -0.4, 0.25, 0.3, 1.1, 9.81, -0.2, 0.4, 0.1,
                     2.0, -1.0, 0.5, 0.3, 0.2, -0.6])
    ch = chaingen.make_chain(n, seed=77)
    st = chaingen.make_states(B, n, seed=78, kinds=("q", "qd", "tau"))
    model = cuda_lib.Model(ch)
    bufs = []
    for k in ("q", "qd", "tau"):
        flat = torch.zeros(B * n + 1, dtype=torch.float32, device="cuda")
        flat[1:] = torch.from_numpy(st[k].astype(np.float32).ravel()).cuda()
        bufs.append(flat[1:].view(B, n))
    out = torch.zeros(B * n + 1, dtype=torch.float32, device="cuda")[1:].view(B, n)
    qdd = cuda_lib.aba(model, *bufs, base=base, out=out).cpu().double().numpy()
    h = {k: st[k].astype(np.float32).astype(np.float64) for k in st}
    ref = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"], base=base)
    assert oracle.rel_err(qdd, ref) <= TOL["float32"]


def test_aba_global_constant_kernel_full_batch_n100(cuda_lib):
    """B = 16384, n = 100: every 64th instance against the oracle, and the
    round-trip residual on the scale of test_aba_full_batch_sampled."""
    n, B = 100, 16384
    qdd, ch, h, _ = run(cuda_lib, n, B, "float32", seed=1609)
    idx = np.arange(0, B, 64)
    ref = oracle.fd_aba(ch, h["q"][idx], h["qd"][idx], h["tau"][idx])
    assert oracle.rel_err(qdd[idx], ref) <= TOL["float32"]
    back = oracle.rnea(ch, h["q"][idx], h["qd"][idx], qdd[idx])
    bias = oracle.rnea(ch, h["q"][idx], h["qd"][idx], np.zeros_like(qdd[idx]))
    scale = np.maximum(np.max(np.abs(h["tau"][idx]), axis=1), np.max(np.abs(bias), axis=1))
    err = np.max(np.abs(back - h["tau"][idx]), axis=1) / scale
    assert err.max() <= 1e-4, err.max()


@pytest.mark.parametrize("dtype,flags", [("float64", 0), ("float32", 4)])
def test_aba_global_constant_kernel_fp64_update_agrees_with_joint_frames(cuda_lib, dtype, flags):
    """The common-normal kernel with constants and FP64 records in global
    memory (FP64 data, n = 100; FP32 data with RD_ABA_FP64_UPDATE, n = 63: a
    length that is not a multiple of 4, within the 64 links the joint-frame
    kernel takes for FP32 data) against the
    joint-frame kernel on the same data (FP64: one result to rounding; FP32:
    each against the oracle, since the FP32 sweeps round differently in the
    two frames)."""
    n = 100 if dtype == "float64" else 63
    a, ch, h, _ = run(cuda_lib, n, 300, dtype, seed=83, flags=flags)
    b, _, _, _ = run(cuda_lib, n, 300, dtype, seed=83, flags=flags | cuda_lib.RD_ABA_JOINT_FRAMES)
    ref = oracle.fd_aba(ch, h["q"], h["qd"], h["tau"], base=None)
    if dtype == "float64":
        assert oracle.rel_err(a, b) <= 1e-9
    assert oracle.rel_err(a, ref) <= TOL[dtype]
    assert oracle.rel_err(b, ref) <= TOL[dtype]
