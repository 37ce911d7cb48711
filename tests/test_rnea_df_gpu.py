"""GPU parity of inverse dynamics for FP64 data in double-float arithmetic
(RD_VARIANT_SERIAL_DF) against the FP64 oracle, through the C ABI, and of its
double-float sine and cosine (rd_joint_trig_df) against numpy.

Every value of the kernel is a pair of FP32 numbers (about 48 significand
bits), so it meets the FP64 bar of 1e-10 (max_i |tau - tau*| / max_i |tau*|
per instance, max over the batch). A lost low part would leave FP32 accuracy
(~1e-7): the tighter agreement with the FP64 kernels (1e-11) and the trig bar
(1e-14 absolute) catch that.
"""
import numpy as np
import pytest

import chaingen
import oracle

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _torch():
    import torch

    return torch


def run(rd, ch, B, variant, seed=11, base=None, block=0):
    torch = _torch()
    n = ch.M.shape[0]
    st = chaingen.make_states(B, n, seed=seed)
    host = {k: st[k].astype(np.float64) for k in ("q", "qd", "qdd")}
    dev = {k: torch.from_numpy(v).cuda() for k, v in host.items()}
    model = rd.Model(ch)
    v = variant | (rd.RD_TUNE_BLOCK(block) if block else 0)
    tau = rd.rnea(model, dev["q"], dev["qd"], dev["qdd"], base=base, variant=v)
    torch.cuda.synchronize()
    ref = oracle.rnea(ch, host["q"], host["qd"], host["qdd"], base=base)
    return tau.cpu().numpy(), ref


# ---- sine and cosine

@pytest.mark.parametrize("scale", [1.0, np.pi, 10.0, 1000.0])
def test_df_trig_matches_numpy(cuda_lib, scale):
    torch = _torch()
    rng = np.random.default_rng(5)
    x = rng.uniform(-scale, scale, 200000)
    s, c = cuda_lib.joint_trig_df(torch.from_numpy(x).cuda())
    s, c = s.cpu().numpy(), c.cpu().numpy()
    assert np.max(np.abs(s - np.sin(x))) <= 1e-14
    assert np.max(np.abs(c - np.cos(x))) <= 1e-14


def test_df_trig_special_points(cuda_lib):
    """Quadrant boundaries (k pi/4, where |r| is largest, and k pi/2, where the
    quadrant changes), zero, negative zero and tiny angles."""
    torch = _torch()
    k = np.arange(-64, 65)
    x = np.concatenate([k * np.pi / 4, k * np.pi / 2, np.nextafter(k * np.pi / 4, np.inf),
                        [0.0, -0.0, 1e-300, -1e-20, 1e-8, 3e-5]])
    s, c = cuda_lib.joint_trig_df(torch.from_numpy(x).cuda())
    s, c = s.cpu().numpy(), c.cpu().numpy()
    assert np.max(np.abs(s - np.sin(x))) <= 1e-14
    assert np.max(np.abs(c - np.cos(x))) <= 1e-14
    assert s[-6] == 0.0 and c[-6] == 1.0
    # small angles inside the FP32 exponent range: relative accuracy of sin
    # (1e-300 lies below it and flushes to 0, within the absolute bar above)
    small = x[-3:]
    assert np.all(np.abs(s[-3:] - np.sin(small)) <= 4e-15 * np.abs(np.sin(small))), s[-3:] - np.sin(small)


def test_df_trig_pythagorean(cuda_lib):
    torch = _torch()
    x = np.linspace(-20, 20, 100001)
    s, c = cuda_lib.joint_trig_df(torch.from_numpy(x).cuda())
    s, c = s.cpu().numpy(), c.cpu().numpy()
    assert np.max(np.abs(s * s + c * c - 1.0)) <= 2e-14


# ---- inverse dynamics

@pytest.mark.parametrize("n", [1, 2, 3, 7, 16, 31, 32, 33, 48, 64])
def test_df_parity(cuda_lib, n):
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED + n)
    tau, ref = run(cuda_lib, ch, 1000, cuda_lib.RD_VARIANT_SERIAL_DF)
    err = oracle.rel_err(tau, ref)
    assert err <= TOL, f"n={n}: rel err {err:.3e}"


@pytest.mark.parametrize("n", [7, 32, 64])
def test_df_agrees_with_fp64_kernels(cuda_lib, n):
    """Same data through the FP64 kernels (AUTO) and the double-float one."""
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED + 2 * n)
    a, _ = run(cuda_lib, ch, 2000, cuda_lib.RD_VARIANT_AUTO, seed=19)
    b, _ = run(cuda_lib, ch, 2000, cuda_lib.RD_VARIANT_SERIAL_DF, seed=19)
    assert oracle.rel_err(b, a) <= 1e-11


@pytest.mark.parametrize("block", [32, 64])
def test_df_block_sizes(cuda_lib, block):
    ch = chaingen.make_chain(20)
    tau, ref = run(cuda_lib, ch, 777, cuda_lib.RD_VARIANT_SERIAL_DF, block=block)
    assert oracle.rel_err(tau, ref) <= TOL


def test_df_base_motion_and_external_wrench(cuda_lib):
    base = np.array([0.2, -0.1, 0.3, 0.5, -0.4, 0.25,
                     0.3, 1.1, 9.81, -0.2, 0.4, 0.1,
                     2.0, -1.0, 0.5, 0.3, 0.2, -0.6])
    ch = chaingen.make_chain(9)
    tau, ref = run(cuda_lib, ch, 333, cuda_lib.RD_VARIANT_SERIAL_DF, base=base)
    assert oracle.rel_err(tau, ref) <= TOL


def test_df_pendulum_closed_form(cuda_lib):
    torch = _torch()
    m, l, Ixx = 1.7, 0.45, 0.03
    model = cuda_lib.Model(chaingen.pendulum(m, l, Ixx))
    q = torch.linspace(-3, 3, 97, dtype=torch.float64, device="cuda").reshape(-1, 1)
    qd = torch.full_like(q, 0.7)
    qdd = torch.cos(q)
    tau = cuda_lib.rnea(model, q, qd, qdd, variant=cuda_lib.RD_VARIANT_SERIAL_DF).cpu().numpy()
    qh, qddh = q.cpu().numpy(), qdd.cpu().numpy()
    expect = (m * l * l + Ixx) * qddh + m * 9.81 * l * np.sin(qh)
    assert np.max(np.abs(tau - expect)) < 1e-12


def test_df_unaligned_rows(cuda_lib):
    """Element loads: rows at any 8-byte offset."""
    torch = _torch()
    n, B = 6, 300
    ch = chaingen.make_chain(n)
    st = chaingen.make_states(B, n, seed=3)
    model = cuda_lib.Model(ch)
    bufs = []
    for k in ("q", "qd", "qdd"):
        flat = torch.zeros(B * n + 1, dtype=torch.float64, device="cuda")
        flat[1:] = torch.from_numpy(st[k].ravel()).cuda()
        bufs.append(flat[1:].view(B, n))
    ref = oracle.rnea(ch, st["q"], st["qd"], st["qdd"])
    out_flat = torch.zeros(B * n + 1, dtype=torch.float64, device="cuda")
    tau = cuda_lib.rnea(model, *bufs, out=out_flat[1:].view(B, n),
                        variant=cuda_lib.RD_VARIANT_SERIAL_DF).cpu().numpy()
    assert oracle.rel_err(tau, ref) <= TOL


@pytest.mark.parametrize("B", [1, 31, 33, 65])
def test_df_edge_batches(cuda_lib, B):
    ch = chaingen.make_chain(5)
    tau, ref = run(cuda_lib, ch, B, cuda_lib.RD_VARIANT_SERIAL_DF)
    assert oracle.rel_err(tau, ref) <= TOL


def test_df_degenerate_geometries(cuda_lib):
    """Parallel axes (planar arm) and nearly parallel ones (1e-7 rad)."""
    I3 = np.eye(3)
    ref = chaingen.make_chain(5, seed=3)

    def twist(r):
        return np.concatenate([-np.cross([0, 0, 1.0], r), [0, 0, 1.0]])

    c, s = np.cos(1e-7), np.sin(1e-7)
    Rx = np.array([[1, 0, 0], [0, c, -s], [0, s, c]])
    for rots in ([I3] * 5, [I3, Rx, Rx.T, I3, I3]):
        M = np.concatenate([np.asarray(rots).reshape(5, 9),
                            [[0.3, 0.1 * k, 0.05 * k] for k in range(5)]], axis=1)
        ch = chaingen.Chain(M, np.array([twist([0.05, 0, 0])] * 5), ref.inertia)
        tau, r = run(cuda_lib, ch, 400, cuda_lib.RD_VARIANT_SERIAL_DF)
        assert oracle.rel_err(tau, r) <= TOL


def test_df_full_batch_sampled(cuda_lib):
    """B = 65536, n = 32 (the inverse-dynamics workload) in FP64 data: every
    64th instance against the oracle."""
    torch = _torch()
    n, B = 32, 65536
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED + n)
    st = chaingen.make_states(B, n, seed=23)
    dev = {k: torch.from_numpy(st[k]).cuda() for k in ("q", "qd", "qdd")}
    tau = cuda_lib.rnea(cuda_lib.Model(ch), dev["q"], dev["qd"], dev["qdd"],
                        variant=cuda_lib.RD_VARIANT_SERIAL_DF).cpu().numpy()
    idx = np.arange(0, B, 64)
    ref = oracle.rnea(ch, *(st[k][idx] for k in ("q", "qd", "qdd")))
    assert oracle.rel_err(tau[idx], ref) <= TOL
    assert cuda_lib.rnea_last_config()[0] == cuda_lib.RD_VARIANT_SERIAL_DF


def test_df_rejects_fp32_data_and_long_chains(cuda_lib):
    torch = _torch()
    model = cuda_lib.Model(chaingen.make_chain(8))
    z = torch.zeros((4, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(cuda_lib.RdError):
        cuda_lib.rnea(model, z, z, z, variant=cuda_lib.RD_VARIANT_SERIAL_DF)
    long_model = cuda_lib.Model(chaingen.make_chain(65))
    z = torch.zeros((4, 65), dtype=torch.float64, device="cuda")
    with pytest.raises(cuda_lib.RdError, match="n <= 64"):
        cuda_lib.rnea(long_model, z, z, z, variant=cuda_lib.RD_VARIANT_SERIAL_DF)
