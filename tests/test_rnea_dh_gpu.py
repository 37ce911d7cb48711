"""GPU parity of the common-normal-frame RNEA kernels (RD_VARIANT_SERIAL_DH,
RD_VARIANT_SERIAL_DH_RECOMPUTE) against the FP64 oracle, through the C ABI.

rd_model_create re-expresses every link in a frame whose x axis lies along the
common normal of consecutive joint axes, so each link rotation is
Rx(alpha_i) Rz(theta0_i + q_i). The torques are the same physical quantities;
these tests check that on random chains and on the geometries where the common
normal degenerates (parallel, intersecting, nearly parallel and coincident
axes). Bars and error metric as in test_rnea_gpu.py.
"""
import numpy as np
import pytest

import chaingen
import oracle

pytestmark = pytest.mark.gpu

TOL = {"float32": 1e-4, "float64": 1e-10}


def _torch():
    import torch

    return torch


def run(rd, ch, B, dtype, variant, seed=11, base=None):
    torch = _torch()
    n = ch.M.shape[0]
    st = chaingen.make_states(B, n, seed=seed)
    np_dt = np.float32 if dtype == "float32" else np.float64
    host = {k: st[k].astype(np_dt) for k in ("q", "qd", "qdd")}
    dev = {k: torch.from_numpy(v).cuda() for k, v in host.items()}
    model = rd.Model(ch)
    tau = rd.rnea(model, dev["q"], dev["qd"], dev["qdd"], base=base, variant=variant)
    torch.cuda.synchronize()
    ref = oracle.rnea(ch, *(host[k].astype(np.float64) for k in ("q", "qd", "qdd")), base=base)
    return tau.cpu().numpy().astype(np.float64), ref


def _variants(rd):
    return {"dh": rd.RD_VARIANT_SERIAL_DH, "dh_recompute": rd.RD_VARIANT_SERIAL_DH_RECOMPUTE}


@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("variant", ["dh", "dh_recompute"])
@pytest.mark.parametrize("n", [1, 2, 3, 7, 16, 31, 32, 33, 64, 100, 128])
def test_dh_parity(cuda_lib, n, dtype, variant):
    if variant == "dh" and dtype == "float64" and n > 100:
        pytest.skip("per-link state of this chain exceeds shared memory")
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED + n)
    tau, ref = run(cuda_lib, ch, 1000, dtype, _variants(cuda_lib)[variant])
    err = oracle.rel_err(tau, ref)
    assert err <= TOL[dtype], f"n={n} {dtype} {variant}: rel err {err:.3e}"


@pytest.mark.parametrize("block", [32, 64, 128])
@pytest.mark.parametrize("variant", ["dh", "dh_recompute"])
def test_dh_block_sizes(cuda_lib, block, variant):
    """Every built block size, several blocks and a ragged tail (B = 2000)."""
    ch = chaingen.make_chain(32)
    v = _variants(cuda_lib)[variant] | cuda_lib.RD_TUNE_BLOCK(block)
    tau, ref = run(cuda_lib, ch, 2000, "float32", v)
    assert oracle.rel_err(tau, ref) <= TOL["float32"]


@pytest.mark.parametrize("variant", ["dh", "dh_recompute"])
def test_dh_fast_trig(cuda_lib, variant):
    ch = chaingen.make_chain(32)
    v = _variants(cuda_lib)[variant] | cuda_lib.RD_FLAG_FAST_TRIG
    tau, ref = run(cuda_lib, ch, 1000, "float32", v)
    assert oracle.rel_err(tau, ref) <= TOL["float32"]


@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("variant", ["dh", "dh_recompute"])
def test_dh_base_motion_and_external_wrench(cuda_lib, dtype, variant):
    """V_0, dV_0 move to the recursion's base frame and F_{n+1} to the last
    link's frame on the host; both conversions are exercised here."""
    base = np.array([0.2, -0.1, 0.3, 0.5, -0.4, 0.25,
                     0.3, 1.1, 9.81, -0.2, 0.4, 0.1,
                     2.0, -1.0, 0.5, 0.3, 0.2, -0.6])
    ch = chaingen.make_chain(9)
    tau, ref = run(cuda_lib, ch, 333, dtype, _variants(cuda_lib)[variant], base=base)
    assert oracle.rel_err(tau, ref) <= TOL[dtype]


def _chain_from_axes(R_list, p_list, S_list, seed=3):
    """Chain with given home rotations/offsets M_i and twists S_i, random inertias."""
    n = len(R_list)
    ref = chaingen.make_chain(n, seed=seed)
    M = np.concatenate([np.asarray(R_list).reshape(n, 9), np.asarray(p_list)], axis=1)
    return chaingen.Chain(M, np.asarray(S_list, dtype=float), ref.inertia)


def _rot_x(t):
    c, s = np.cos(t), np.sin(t)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])


def _twist(w, r):
    w = np.asarray(w, dtype=float)
    w = w / np.linalg.norm(w)
    return np.concatenate([-np.cross(w, r), w])


def _special_chains():
    I3 = np.eye(3)
    chains = {}
    # planar arm: every axis parallel (z), offsets in the plane
    chains["parallel"] = _chain_from_axes([I3] * 6, [[0.3, 0.1 * k, 0.0] for k in range(6)],
                                          [_twist([0, 0, 1], [0.05, 0, 0])] * 6)
    # spherical wrist: three axes through one point, then an offset link
    chains["intersecting"] = _chain_from_axes(
        [I3, I3, I3, I3], [[0.2, 0.1, 0.3], [0, 0, 0], [0, 0, 0], [0.1, 0.0, 0.2]],
        [_twist([1, 0, 0], [0, 0, 0]), _twist([0, 1, 0], [0, 0, 0]),
         _twist([0, 0, 1], [0, 0, 0]), _twist([1, 1, 0], [0.02, 0, 0])])
    # nearly parallel consecutive axes (1e-7 rad apart), and coincident axes
    chains["nearly_parallel"] = _chain_from_axes(
        [I3, _rot_x(1e-7), _rot_x(-2e-7), I3, I3],
        [[0.1, 0.2, 0.3], [0.25, 0.0, 0.1], [0.2, 0.1, 0.0], [0.0, 0.0, 0.3], [0.3, 0.0, 0.0]],
        [_twist([0, 0, 1], [0, 0, 0])] * 5)
    return chains


@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("variant", ["dh", "dh_recompute"])
@pytest.mark.parametrize("geometry", ["parallel", "intersecting", "nearly_parallel"])
def test_dh_degenerate_geometries(cuda_lib, geometry, dtype, variant):
    ch = _special_chains()[geometry]
    tau, ref = run(cuda_lib, ch, 500, dtype, _variants(cuda_lib)[variant])
    assert oracle.rel_err(tau, ref) <= TOL[dtype], geometry


def test_dh_pendulum_closed_form(cuda_lib):
    torch = _torch()
    m, l, Ixx = 1.7, 0.45, 0.03
    model = cuda_lib.Model(chaingen.pendulum(m, l, Ixx))
    q = torch.linspace(-3, 3, 97, dtype=torch.float64, device="cuda").reshape(-1, 1)
    qd = torch.full_like(q, 0.7)
    qdd = torch.cos(q)
    for v in _variants(cuda_lib).values():
        tau = cuda_lib.rnea(model, q, qd, qdd, variant=v).cpu().numpy()
        qh, qddh = q.cpu().numpy(), qdd.cpu().numpy()
        expect = (m * l * l + Ixx) * qddh + m * 9.81 * l * np.sin(qh)
        assert np.max(np.abs(tau - expect)) < 1e-12


def test_dh_matches_joint_frame_kernels_fp64(cuda_lib):
    """Two frame choices, one result: FP64 agreement to rounding."""
    ch = chaingen.make_chain(24)
    a, _ = run(cuda_lib, ch, 500, "float64", cuda_lib.RD_VARIANT_SERIAL)
    for v in _variants(cuda_lib).values():
        b, _ = run(cuda_lib, ch, 500, "float64", v)
        assert np.max(np.abs(a - b)) <= 1e-11 * np.max(np.abs(a))


def test_dh_unaligned_rows(cuda_lib):
    """Rows not 16-byte aligned take the element-load path."""
    torch = _torch()
    n, B = 8, 300
    ch = chaingen.make_chain(n)
    st = chaingen.make_states(B, n, seed=3)
    model = cuda_lib.Model(ch)
    bufs = []
    for k in ("q", "qd", "qdd"):
        flat = torch.zeros(B * n + 1, dtype=torch.float32, device="cuda")
        flat[1:] = torch.from_numpy(st[k].astype(np.float32).ravel()).cuda()
        bufs.append(flat[1:].view(B, n))
    ref = oracle.rnea(ch, *(st[k].astype(np.float32).astype(np.float64) for k in ("q", "qd", "qdd")))
    for v in _variants(cuda_lib).values():
        out_flat = torch.zeros(B * n + 1, dtype=torch.float32, device="cuda")
        tau = cuda_lib.rnea(model, *bufs, out=out_flat[1:].view(B, n), variant=v).cpu().numpy()
        assert oracle.rel_err(tau, ref) <= TOL["float32"]


@pytest.mark.parametrize("B", [1, 31, 33, 65])
def test_dh_edge_batches(cuda_lib, B):
    ch = chaingen.make_chain(5)
    for v in _variants(cuda_lib).values():
        tau, ref = run(cuda_lib, ch, B, "float64", v)
        assert oracle.rel_err(tau, ref) <= TOL["float64"]


@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("n,K", [(8, 4), (8, 8), (32, 4), (32, 12), (32, 24), (32, 32),
                                 (64, 12), (64, 40), (100, 8), (128, 4)])
def test_dh_stored_prefix_lengths(cuda_lib, n, K, dtype):
    """Full state for the first K links, cos/sin only for the rest
    (RD_TUNE_STORED_LINKS(K)); every split point, FP32 and FP64."""
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED + n)
    v = cuda_lib.RD_VARIANT_SERIAL_DH | cuda_lib.RD_TUNE_STORED_LINKS(K)
    if dtype == "float64" and n >= 100:
        v |= cuda_lib.RD_TUNE_BLOCK(32)
    tau, ref = run(cuda_lib, ch, 1000, dtype, v)
    assert oracle.rel_err(tau, ref) <= TOL[dtype], f"n={n} K={K} {dtype}"


@pytest.mark.parametrize("B", [1, 31, 4865, 8192])
def test_dh_default_split_across_batch_sizes(cuda_lib, B):
    """The library's K depends on B (one resident wave or not); parity at each."""
    ch = chaingen.make_chain(32)
    tau, ref = run(cuda_lib, ch, B, "float32", cuda_lib.RD_VARIANT_SERIAL_DH)
    assert oracle.rel_err(tau, ref) <= TOL["float32"]
    tau, ref = run(cuda_lib, ch, B, "float32", cuda_lib.RD_VARIANT_AUTO)
    assert oracle.rel_err(tau, ref) <= TOL["float32"]


def test_dh_auto_full_batch_n64_sampled(cuda_lib):
    """B = 65536, n = 64 in FP32 through AUTO (the common-normal kernel with a
    stored prefix): every 32nd instance against the oracle."""
    torch = _torch()
    n, B = 64, 65536
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED + n)
    st = chaingen.make_states(B, n, seed=21)
    host = {k: st[k].astype(np.float32) for k in ("q", "qd", "qdd")}
    dev = {k: torch.from_numpy(v).cuda() for k, v in host.items()}
    tau = cuda_lib.rnea(cuda_lib.Model(ch), dev["q"], dev["qd"], dev["qdd"]).cpu().numpy()
    idx = np.arange(0, B, 32)
    ref = oracle.rnea(ch, *(host[k][idx].astype(np.float64) for k in ("q", "qd", "qdd")))
    assert oracle.rel_err(tau[idx], ref) <= TOL["float32"]


def test_dh_rejects_state_beyond_shared_memory(cuda_lib):
    """An explicit K whose state cannot fit is refused on the host."""
    torch = _torch()
    n, B = 128, 64
    model = cuda_lib.Model(chaingen.make_chain(n))
    z = torch.zeros((B, n), dtype=torch.float64, device="cuda")
    v = (cuda_lib.RD_VARIANT_SERIAL_DH | cuda_lib.RD_TUNE_STORED_LINKS(128)
         | cuda_lib.RD_TUNE_BLOCK(128))
    with pytest.raises(cuda_lib.RdError, match="shared"):
        cuda_lib.rnea(model, z, z, z, variant=v)


# ---- state of the first 16 links in tensor memory (RD_VARIANT_SERIAL_DH_TMEM)

@pytest.mark.parametrize("n", [4, 8, 12, 16, 20, 24, 28, 32])
def test_tmem_state_parity(cuda_lib, n):
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED + n)
    tau, ref = run(cuda_lib, ch, 1000, "float32", cuda_lib.RD_VARIANT_SERIAL_DH_TMEM)
    err = oracle.rel_err(tau, ref)
    assert err <= TOL["float32"], f"n={n}: rel err {err:.3e}"


@pytest.mark.parametrize("K", [4, 8, 16, 20, 24])
def test_tmem_state_split_points(cuda_lib, K):
    """K links with full state: the first min(K, 16) in TMEM, the rest in shared
    memory, cos/sin only beyond K."""
    ch = chaingen.make_chain(32)
    v = cuda_lib.RD_VARIANT_SERIAL_DH_TMEM | cuda_lib.RD_TUNE_STORED_LINKS(K)
    tau, ref = run(cuda_lib, ch, 777, "float32", v)
    assert oracle.rel_err(tau, ref) <= TOL["float32"]


@pytest.mark.parametrize("B", [1, 127, 129, 4097])
def test_tmem_state_ragged_batches(cuda_lib, B):
    """Threads past the batch run the last row and store nothing."""
    ch = chaingen.make_chain(32)
    tau, ref = run(cuda_lib, ch, B, "float32", cuda_lib.RD_VARIANT_SERIAL_DH_TMEM)
    assert oracle.rel_err(tau, ref) <= TOL["float32"]


def test_tmem_state_base_and_fast_trig(cuda_lib):
    base = np.array([0.2, -0.1, 0.3, 0.5, -0.4, 0.25,
                     0.3, 1.1, 9.81, -0.2, 0.4, 0.1,
                     2.0, -1.0, 0.5, 0.3, 0.2, -0.6])
    ch = chaingen.make_chain(16)
    tau, ref = run(cuda_lib, ch, 500, "float32", cuda_lib.RD_VARIANT_SERIAL_DH_TMEM, base=base)
    assert oracle.rel_err(tau, ref) <= TOL["float32"]
    v = cuda_lib.RD_VARIANT_SERIAL_DH_TMEM | cuda_lib.RD_FLAG_FAST_TRIG
    tau, ref = run(cuda_lib, ch, 500, "float32", v)
    assert oracle.rel_err(tau, ref) <= TOL["float32"]


def test_tmem_state_full_batch_sampled(cuda_lib):
    """n = 32, B = 65536: every instance of the batch in one wave; every 16th
    instance against the oracle, and back-to-back launches agree bit for bit."""
    torch = _torch()
    n, B = 32, 65536
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED)
    st = chaingen.make_states(B, n, seed=31)
    host = {k: st[k].astype(np.float32) for k in ("q", "qd", "qdd")}
    dev = {k: torch.from_numpy(v).cuda() for k, v in host.items()}
    model = cuda_lib.Model(ch)
    v = cuda_lib.RD_VARIANT_SERIAL_DH_TMEM
    t1 = cuda_lib.rnea(model, dev["q"], dev["qd"], dev["qdd"], variant=v)
    t2 = cuda_lib.rnea(model, dev["q"], dev["qd"], dev["qdd"], variant=v)
    torch.cuda.synchronize()
    assert torch.equal(t1, t2)
    idx = np.arange(0, B, 16)
    ref = oracle.rnea(ch, *(host[k][idx].astype(np.float64) for k in ("q", "qd", "qdd")))
    assert oracle.rel_err(t1.cpu().numpy()[idx], ref) <= TOL["float32"]


def test_tmem_state_rejects_unsupported_rows(cuda_lib):
    torch = _torch()
    model = cuda_lib.Model(chaingen.make_chain(36))
    z = torch.zeros((64, 36), dtype=torch.float32, device="cuda")
    with pytest.raises(cuda_lib.RdError, match="TMEM"):
        cuda_lib.rnea(model, z, z, z, variant=cuda_lib.RD_VARIANT_SERIAL_DH_TMEM)


# ---- the first stored links' state in registers (RD_TUNE_REG_STATE_LINKS)

@pytest.mark.parametrize("n,K,R", [(4, 4, 4), (8, 8, 4), (8, 8, 8), (12, 12, 4), (16, 16, 8),
                                   (20, 20, 4), (20, 12, 8), (24, 24, 8), (28, 28, 4),
                                   (32, 32, 8), (32, 24, 12), (32, 32, 16), (32, 16, 16)])
def test_register_state_parity_and_bits(cuda_lib, n, K, R):
    """Against the oracle, and bit for bit against the same K held in shared
    memory (the arithmetic is the same; only where the state sits changes)."""
    torch = _torch()
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED + n)
    v = cuda_lib.RD_VARIANT_SERIAL_DH | cuda_lib.RD_TUNE_BLOCK(32) | cuda_lib.RD_TUNE_STORED_LINKS(K)
    tau, ref = run(cuda_lib, ch, 1000, "float32", v | cuda_lib.RD_TUNE_REG_STATE_LINKS(R))
    assert oracle.rel_err(tau, ref) <= TOL["float32"], f"n={n} K={K} R={R}"
    assert cuda_lib.rnea_last_state_layout() == (R, 3)
    tau0, _ = run(cuda_lib, ch, 1000, "float32", v)
    assert np.array_equal(tau, tau0)


@pytest.mark.parametrize("B", [1, 31, 33, 4097])
def test_register_state_ragged_batches_base_and_fast_trig(cuda_lib, B):
    base = np.array([0.2, -0.1, 0.3, 0.5, -0.4, 0.25, 0.3, 1.1, 9.81, -0.2, 0.4, 0.1,
                     2.0, -1.0, 0.5, 0.3, 0.2, -0.6])
    ch = chaingen.make_chain(32, seed=chaingen.BASE_SEED + 1)
    v = (cuda_lib.RD_VARIANT_SERIAL_DH | cuda_lib.RD_TUNE_BLOCK(32) |
         cuda_lib.RD_TUNE_STORED_LINKS(32) | cuda_lib.RD_TUNE_REG_STATE_LINKS(8))
    tau, ref = run(cuda_lib, ch, B, "float32", v, base=base)
    assert oracle.rel_err(tau, ref) <= TOL["float32"]
    tau, ref = run(cuda_lib, ch, B, "float32", v | cuda_lib.RD_FLAG_FAST_TRIG)
    assert oracle.rel_err(tau, ref) <= TOL["float32"]


@pytest.mark.parametrize("n,B,K,R,S", [(32, 65536, 32, 8, 3), (32, 16384, 32, 4, 2),
                                       (24, 65536, 24, 8, 3), (20, 65536, 20, 8, 2),
                                       (16, 65536, 16, 8, 2), (16, 16384, 16, 4, 2),
                                       (8, 65536, 8, 8, 3)])
def test_auto_register_state_choice(cuda_lib, n, B, K, R, S):
    """AUTO for FP32 n <= 32 (past the scan kernel's batches) stores every link,
    keeps the measured number of them in registers and stages through the
    measured ring depth."""
    torch = _torch()
    model = cuda_lib.Model(chaingen.make_chain(n))
    z = torch.zeros((B, n), dtype=torch.float32, device="cuda")
    cuda_lib.rnea(model, z, z, z)
    kern, block, stored = cuda_lib.rnea_last_config()
    assert kern == cuda_lib.RD_RNEA_KERNEL_DH_PARAM and block == 32
    assert (stored,) + cuda_lib.rnea_last_state_layout() == (K, R, S)


@pytest.mark.parametrize("n,R", [(12, 8), (16, 0), (16, 4), (20, 8), (32, 8)])
def test_two_stage_ring_parity_and_bits(cuda_lib, n, R):
    """RD_TUNE_TWO_STAGE_RING: the same arithmetic with a shallower staging
    ring; bit for bit the three-chunk result, and the oracle's within the bar."""
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED + n)
    v = (cuda_lib.RD_VARIANT_SERIAL_DH | cuda_lib.RD_TUNE_BLOCK(32) |
         cuda_lib.RD_TUNE_STORED_LINKS(n) | cuda_lib.RD_TUNE_REG_STATE_LINKS(R))
    tau2, ref = run(cuda_lib, ch, 3000, "float32", v | cuda_lib.RD_TUNE_TWO_STAGE_RING)
    assert cuda_lib.rnea_last_state_layout() == (R, 2)
    assert oracle.rel_err(tau2, ref) <= TOL["float32"]
    tau3, _ = run(cuda_lib, ch, 3000, "float32", v)
    assert np.array_equal(tau2, tau3)


def test_register_state_rejections(cuda_lib):
    torch = _torch()
    m48 = cuda_lib.Model(chaingen.make_chain(48))
    x48 = torch.zeros((64, 48), device="cuda")
    base_v = cuda_lib.RD_VARIANT_SERIAL_DH | cuda_lib.RD_TUNE_BLOCK(32)
    with pytest.raises(cuda_lib.RdError):  # n > 32
        cuda_lib.rnea(m48, x48, x48, x48, variant=base_v | cuda_lib.RD_TUNE_STORED_LINKS(48) |
                      cuda_lib.RD_TUNE_REG_STATE_LINKS(8))
    m16 = cuda_lib.Model(chaingen.make_chain(16))
    x16 = torch.zeros((64, 16), device="cuda")
    for v in (base_v | cuda_lib.RD_TUNE_STORED_LINKS(4) | cuda_lib.RD_TUNE_REG_STATE_LINKS(8),
              cuda_lib.RD_VARIANT_SERIAL_DH | cuda_lib.RD_TUNE_BLOCK(64) |
              cuda_lib.RD_TUNE_STORED_LINKS(16) | cuda_lib.RD_TUNE_REG_STATE_LINKS(8),
              cuda_lib.RD_VARIANT_SERIAL_DH_RECOMPUTE | cuda_lib.RD_TUNE_REG_STATE_LINKS(8)):
        with pytest.raises(cuda_lib.RdError):
            cuda_lib.rnea(m16, x16, x16, x16, variant=v)
    x16d = torch.zeros((64, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(cuda_lib.RdError):  # FP64
        cuda_lib.rnea(m16, x16d, x16d, x16d, variant=base_v | cuda_lib.RD_TUNE_STORED_LINKS(16) |
                      cuda_lib.RD_TUNE_REG_STATE_LINKS(8))


def test_register_state_empty_batch(cuda_lib):
    torch = _torch()
    model = cuda_lib.Model(chaingen.make_chain(32))
    z = torch.zeros((0, 32), device="cuda")
    v = (cuda_lib.RD_VARIANT_SERIAL_DH | cuda_lib.RD_TUNE_BLOCK(32) | cuda_lib.RD_TUNE_STORED_LINKS(32)
         | cuda_lib.RD_TUNE_REG_STATE_LINKS(8) | cuda_lib.RD_TUNE_TWO_STAGE_RING)
    assert cuda_lib.rnea(model, z, z, z, variant=v).shape == (0, 32)
