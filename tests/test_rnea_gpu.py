"""GPU parity of rnea_batch against the FP64 oracle, through the C ABI.

Error metric (per instance, maximised over the batch):
    max_i |tau_i - tau*_i| / max_i |tau*_i|.
Bars: FP64 GPU <= 1e-10; FP32 GPU <= 1e-4. The oracle always sees exactly the
values the GPU saw (FP32 inputs widened to FP64), so the measured error is
arithmetic error only.
"""
import numpy as np
import pytest

import chaingen
import oracle

pytestmark = pytest.mark.gpu

TOL = {"float32": 1e-4, "float64": 1e-10}
VARIANTS = {"auto": 0, "serial": 1, "recompute": 2}


def _torch():
    import torch

    return torch


def run_case(rd, n, B, dtype, variant, seed=5, base=None, chain=None):
    torch = _torch()
    ch = chain or chaingen.make_chain(n, seed=chaingen.BASE_SEED + n)
    st = chaingen.make_states(B, n, seed=seed)
    np_dt = np.float32 if dtype == "float32" else np.float64
    host = {k: st[k].astype(np_dt) for k in ("q", "qd", "qdd")}
    dev = {k: torch.from_numpy(v).cuda() for k, v in host.items()}
    model = rd.Model(ch)
    tau = rd.rnea(model, dev["q"], dev["qd"], dev["qdd"], base=base, variant=variant)
    torch.cuda.synchronize()
    ref = oracle.rnea(ch, *(host[k].astype(np.float64) for k in ("q", "qd", "qdd")), base=base)
    return tau.cpu().numpy().astype(np.float64), ref


@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("variant", ["auto", "serial", "recompute"])
@pytest.mark.parametrize("n", [1, 2, 7, 16, 31, 32, 33, 48, 64, 100, 128])
def test_rnea_parity(cuda_lib, n, dtype, variant):
    B = 1000  # several blocks and a ragged tail
    if variant == "serial" and dtype == "float64" and n > 100:
        pytest.skip("per-link state of this chain exceeds shared memory; recompute covers it")
    tau, ref = run_case(cuda_lib, n, B, dtype, VARIANTS[variant])
    err = oracle.rel_err(tau, ref)
    assert err <= TOL[dtype], f"n={n} {dtype} {variant}: rel err {err:.3e}"


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_rnea_base_motion_and_external_wrench(cuda_lib, dtype):
    base = np.array([0.2, -0.1, 0.3, 0.5, -0.4, 0.25,      # V_0
                     0.3, 1.1, 9.81, -0.2, 0.4, 0.1,       # dV_0
                     2.0, -1.0, 0.5, 0.3, 0.2, -0.6])      # F_{n+1}
    tau, ref = run_case(cuda_lib, 9, 333, dtype, 0, base=base)
    assert oracle.rel_err(tau, ref) <= TOL[dtype]


@pytest.mark.parametrize("B", [0, 1, 31, 63, 65, 257])
def test_rnea_edge_batches(cuda_lib, B):
    torch = _torch()
    n = 5
    if B == 0:
        model = cuda_lib.Model(chaingen.make_chain(n))
        z = torch.empty((0, n), device="cuda")
        out = cuda_lib.rnea(model, z, z, z)
        assert out.shape == (0, n)
        return
    tau, ref = run_case(cuda_lib, n, B, "float64", 0)
    assert oracle.rel_err(tau, ref) <= TOL["float64"]


def test_rnea_closed_form_pendulum(cuda_lib):
    torch = _torch()
    m, l, Ixx = 1.7, 0.45, 0.03
    ch = chaingen.pendulum(m, l, Ixx)
    model = cuda_lib.Model(ch)
    q = torch.linspace(-3, 3, 97, dtype=torch.float64, device="cuda").reshape(-1, 1)
    qd = torch.full_like(q, 0.7)
    qdd = torch.cos(q)
    tau = cuda_lib.rnea(model, q, qd, qdd).cpu().numpy()
    qh, qddh = q.cpu().numpy(), qdd.cpu().numpy()
    expect = (m * l * l + Ixx) * qddh + m * 9.81 * l * np.sin(qh)
    assert np.max(np.abs(tau - expect)) < 1e-12


@pytest.mark.parametrize("n", [8, 32, 100])
@pytest.mark.parametrize("variant", [1, 2])
def test_rnea_fast_trig_flag(cuda_lib, n, variant):
    """RD_FLAG_FAST_TRIG (SFU sine/cosine after a 2*pi reduction) on chains with
    several links stays within the FP32 bar."""
    tau, ref = run_case(cuda_lib, n, 1000, "float32", variant | cuda_lib.RD_FLAG_FAST_TRIG)
    assert oracle.rel_err(tau, ref) <= TOL["float32"]


def test_rnea_unaligned_rows_fall_back_to_element_loads(cuda_lib):
    """Rows that are not 16-byte aligned (a tensor view offset by one element)."""
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
    out_flat = torch.zeros(B * n + 1, dtype=torch.float32, device="cuda")
    tau = cuda_lib.rnea(model, *bufs, out=out_flat[1:].view(B, n)).cpu().numpy()
    ref = oracle.rnea(ch, *(st[k].astype(np.float32).astype(np.float64) for k in ("q", "qd", "qdd")))
    assert oracle.rel_err(tau, ref) <= TOL["float32"]


def test_rnea_variants_agree_fp64(cuda_lib):
    a, _ = run_case(cuda_lib, 24, 500, "float64", 1)
    b, _ = run_case(cuda_lib, 24, 500, "float64", 2)
    assert np.max(np.abs(a - b)) <= 1e-11 * np.max(np.abs(a))


def test_rnea_full_size_fp32_n32(cuda_lib):
    """n = 32, B = 65536 in FP32 with the launch the benchmark times; the oracle
    checks every instance (about a second of CPU)."""
    tau, ref = run_case(cuda_lib, 32, 65536, "float32", 0, seed=1609)
    assert oracle.rel_err(tau, ref) <= TOL["float32"]


@pytest.mark.parametrize("n", [16, 100])
def test_rnea_full_batch_other_lengths_sampled(cuda_lib, n):
    """B = 65536 at n = 16 and 100: every 64th instance checked against the oracle."""
    torch = _torch()
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED + n)
    st = chaingen.make_states(65536, n, seed=77)
    host = {k: st[k].astype(np.float32) for k in ("q", "qd", "qdd")}
    dev = {k: torch.from_numpy(v).cuda() for k, v in host.items()}
    model = cuda_lib.Model(ch)
    tau = cuda_lib.rnea(model, dev["q"], dev["qd"], dev["qdd"]).cpu().numpy()
    idx = np.arange(0, 65536, 64)
    ref = oracle.rnea(ch, *(host[k][idx].astype(np.float64) for k in ("q", "qd", "qdd")))
    assert oracle.rel_err(tau[idx], ref) <= TOL["float32"]


def test_rnea_host_entry_point(cuda_lib):
    torch = _torch()
    n, B = 12, 700
    ch = chaingen.make_chain(n)
    st = chaingen.make_states(B, n, seed=9)
    model = cuda_lib.Model(ch)
    args = [torch.from_numpy(st[k]).pin_memory() for k in ("q", "qd", "qdd")]
    tau = cuda_lib.rnea_host(model, *args).numpy()
    ref = oracle.rnea(ch, st["q"], st["qd"], st["qdd"])
    assert oracle.rel_err(tau, ref) <= TOL["float64"]


def test_rnea_host_entry_point_pageable_and_fp32(cuda_lib):
    """Pageable host arrays take the staged-copy path; pinned FP32 the in-place path."""
    torch = _torch()
    n, B = 16, 513
    ch = chaingen.make_chain(n)
    st = chaingen.make_states(B, n, seed=10)
    model = cuda_lib.Model(ch)
    for pin in (False, True):
        args = [torch.from_numpy(st[k].astype(np.float32)) for k in ("q", "qd", "qdd")]
        if pin:
            args = [a.pin_memory() for a in args]
        tau = cuda_lib.rnea_host(model, *args).numpy()
        ref = oracle.rnea(ch, *(a.numpy().astype(np.float64) for a in args))
        assert oracle.rel_err(tau, ref) <= TOL["float32"], pin


@pytest.mark.parametrize("B", [8192 * 3 + 77, 300001])
def test_rnea_host_pipeline_chunks(cuda_lib, B):
    """Host arrays spanning several pipeline chunks (ragged last chunk; more rows
    than the chunk cap, so chunks grow): every instance against the device-array
    entry point, which is itself checked against the oracle elsewhere, and a
    sample against the oracle."""
    torch = _torch()
    n = 7
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED + n)
    st = chaingen.make_states(B, n, seed=12)
    model = cuda_lib.Model(ch)
    args = [torch.from_numpy(st[k].astype(np.float32)).pin_memory() for k in ("q", "qd", "qdd")]
    tau = cuda_lib.rnea_host(model, *args).numpy()
    dev = cuda_lib.rnea(model, *(a.cuda() for a in args)).cpu().numpy()
    assert np.array_equal(tau, dev)
    idx = np.arange(0, B, 97)
    ref = oracle.rnea(ch, *(a.numpy()[idx].astype(np.float64) for a in args))
    assert oracle.rel_err(tau[idx].astype(np.float64), ref) <= TOL["float32"]


def test_rnea_host_repeated_calls_use_current_data(cuda_lib):
    """Repeated calls with the same pinned buffers through the staged copies
    (RD_FLAG_HOST_COPY; the device staging buffers are reused): new contents in
    the same buffers, a new boundary state and a new batch size all give the
    fresh result, identical to the device path."""
    torch = _torch()
    n, B = 8, 3 * 8192 + 5
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED + n)
    model = cuda_lib.Model(ch)
    bufs = [torch.empty((B, n), dtype=torch.float32).pin_memory() for _ in range(3)]
    out = torch.empty((B, n), dtype=torch.float32).pin_memory()
    base2 = np.array([0, 0, 0, 0, 0, 0, 0, 0, 9.81, 0, 0, 0, 1.0, 0.5, -0.5, 0.1, 0.2, 0.3])
    for step, (seed, base, rows) in enumerate([(1, None, B), (1, None, B), (2, None, B),
                                               (3, base2, B), (3, base2, B), (4, None, B - 8192)]):
        st = chaingen.make_states(B, n, seed=seed)
        for bf, k in zip(bufs, ("q", "qd", "qdd")):
            bf.copy_(torch.from_numpy(st[k].astype(np.float32)))
        args = [bf[:rows] for bf in bufs]
        tau = cuda_lib.rnea_host(model, *args, out=out[:rows], base=base,
                                 variant=cuda_lib.RD_FLAG_HOST_COPY).numpy().copy()
        dev = cuda_lib.rnea(model, *(a.cuda() for a in args), base=base).cpu().numpy()
        assert np.array_equal(tau, dev), step
        idx = np.arange(0, rows, 211)
        ref = oracle.rnea(ch, *(a.numpy()[idx].astype(np.float64) for a in args), base=base)
        assert oracle.rel_err(tau[idx].astype(np.float64), ref) <= TOL["float32"], step


def test_rnea_rejects_wrong_shapes(cuda_lib):
    torch = _torch()
    model = cuda_lib.Model(chaingen.make_chain(6))
    x = torch.zeros((10, 5), device="cuda")
    with pytest.raises(ValueError):
        cuda_lib.rnea(model, x, x, x)
    y = torch.zeros((10, 6), device="cuda", dtype=torch.float16)
    with pytest.raises(TypeError):
        cuda_lib.rnea(model, y, y, y)


# ---------------------------------------------- lane-parallel scan variant

SCAN_CASES = [(L, n) for L in (2, 4, 8, 16, 32) for n in (1, 2, 5, 7, 16, 31, 32, 33, 64, 100, 128)
              if n <= 8 * L]


@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("L,n", SCAN_CASES)
def test_rnea_scan_parity(cuda_lib, L, n, dtype):
    B = 77  # ragged: instances do not fill the last warp
    tau, ref = run_case(cuda_lib, n, B, dtype, cuda_lib.RD_VARIANT_SCAN(L), seed=11)
    assert oracle.rel_err(tau, ref) <= TOL[dtype], f"L={L} n={n} {dtype}"


@pytest.mark.parametrize("L", [4, 32])
def test_rnea_scan_equals_serial_fp64(cuda_lib, L):
    """The scan reaches the serial recursion's result (Sec. III): FP64 to 1e-12."""
    a, _ = run_case(cuda_lib, 20, 300, "float64", 1, seed=13)
    b, _ = run_case(cuda_lib, 20, 300, "float64", cuda_lib.RD_VARIANT_SCAN(L), seed=13)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


def test_rnea_scan_base_and_wrench(cuda_lib):
    base = np.array([0.2, -0.1, 0.3, 0.5, -0.4, 0.25, 0.3, 1.1, 9.81, -0.2, 0.4, 0.1,
                     2.0, -1.0, 0.5, 0.3, 0.2, -0.6])
    for L in (2, 8, 32):
        tau, ref = run_case(cuda_lib, 13, 100, "float64", cuda_lib.RD_VARIANT_SCAN(L), base=base)
        assert oracle.rel_err(tau, ref) <= TOL["float64"], L


def test_rnea_scan_rejects_too_many_links(cuda_lib):
    torch = _torch()
    model = cuda_lib.Model(chaingen.make_chain(20))
    x = torch.zeros((4, 20), device="cuda")
    with pytest.raises(cuda_lib.RdError):
        cuda_lib.rnea(model, x, x, x, variant=cuda_lib.RD_VARIANT_SCAN(2))


@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("reglinks,block", [(8, 32), (16, 32), (8, 64), (16, 64)])
@pytest.mark.parametrize("n", [4, 8, 12, 16, 20, 32, 64, 100])
def test_rnea_register_state_parity(cuda_lib, n, reglinks, block, dtype):
    """Register-plus-shared-memory state kernel, with chains shorter and longer
    than the register part."""
    v = cuda_lib.RD_VARIANT_SERIAL_REGSTATE | cuda_lib.RD_TUNE_REGLINKS(reglinks) | \
        cuda_lib.RD_TUNE_BLOCK(block)
    tau, ref = run_case(cuda_lib, n, 333, dtype, v, seed=17)
    assert oracle.rel_err(tau, ref) <= TOL[dtype]


# ---- rnea_batch_host reading and writing mapped pinned arrays in place

def _pinned_states(B, n, seed):
    torch = _torch()
    st = chaingen.make_states(B, n, seed=seed)
    return [torch.from_numpy(st[k].astype(np.float32)).pin_memory() for k in ("q", "qd", "qdd")]


@pytest.mark.parametrize("n,B", [(4, 1), (8, 33), (12, 1000), (32, 4097), (64, 2500)])
def test_rnea_host_in_place(cuda_lib, n, B):
    """Pinned FP32 arrays: the kernel reads the rows from host memory and writes
    tau back (ragged last block included); against the oracle, and against the
    device path within the FP32 bar (a different kernel, same recursion: both
    carry FP32 rounding, worst case about 1e-5 of max|tau| at B = 65536)."""
    torch = _torch()
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED + 3 * n)
    model = cuda_lib.Model(ch)
    args = _pinned_states(B, n, seed=30 + n)
    out = torch.full((B, n), float("nan"), dtype=torch.float32).pin_memory()
    tau = cuda_lib.rnea_host(model, *args, out=out).numpy()
    assert cuda_lib.rnea_last_config()[0] == cuda_lib.RD_RNEA_KERNEL_DH_HOST
    ref = oracle.rnea(ch, *(a.numpy().astype(np.float64) for a in args))
    assert oracle.rel_err(tau.astype(np.float64), ref) <= TOL["float32"]
    dev = cuda_lib.rnea(model, *(a.cuda() for a in args)).cpu().numpy()
    assert oracle.rel_err(tau.astype(np.float64), dev.astype(np.float64)) <= TOL["float32"]


def test_rnea_host_in_place_full_batch_and_base(cuda_lib):
    """B = 65536, n = 32 with a moving base and an end wrench: a sample against
    the oracle; the staged-copy path on the same arrays agrees within the FP32
    bar."""
    torch = _torch()
    n, B = 32, 65536
    base = np.array([0.2, -0.1, 0.3, 0.5, -0.4, 0.25, 0.3, 1.1, 9.81, -0.2, 0.4, 0.1,
                     2.0, -1.0, 0.5, 0.3, 0.2, -0.6])
    ch = chaingen.make_chain(n, seed=chaingen.BASE_SEED + n)
    model = cuda_lib.Model(ch)
    args = _pinned_states(B, n, seed=41)
    tau = cuda_lib.rnea_host(model, *args, base=base).numpy().copy()
    idx = np.arange(0, B, 128)
    ref = oracle.rnea(ch, *(a.numpy()[idx].astype(np.float64) for a in args), base=base)
    assert oracle.rel_err(tau[idx].astype(np.float64), ref) <= TOL["float32"]
    staged = cuda_lib.rnea_host(model, *args, base=base, variant=cuda_lib.RD_FLAG_HOST_COPY).numpy()
    assert cuda_lib.rnea_last_config()[0] != cuda_lib.RD_RNEA_KERNEL_DH_HOST
    assert oracle.rel_err(tau.astype(np.float64), staged.astype(np.float64)) <= TOL["float32"]


def test_rnea_host_in_place_needs_every_array_pinned_and_aligned(cuda_lib):
    """A pageable output, or rows that start off a 16-byte boundary, take the
    staged copies; the result is right either way."""
    torch = _torch()
    n, B = 8, 300
    ch = chaingen.make_chain(n)
    model = cuda_lib.Model(ch)
    args = _pinned_states(B, n, seed=5)
    ref = oracle.rnea(ch, *(a.numpy().astype(np.float64) for a in args))
    tau = cuda_lib.rnea_host(model, *args, out=torch.empty((B, n), dtype=torch.float32)).numpy()
    assert cuda_lib.rnea_last_config()[0] != cuda_lib.RD_RNEA_KERNEL_DH_HOST
    assert oracle.rel_err(tau.astype(np.float64), ref) <= TOL["float32"]
    flat = torch.empty(B * n + 1, dtype=torch.float32).pin_memory()
    flat[1:] = args[0].reshape(-1)
    shifted = [flat[1:].view(B, n), args[1], args[2]]
    tau = cuda_lib.rnea_host(model, *shifted).numpy()
    assert cuda_lib.rnea_last_config()[0] != cuda_lib.RD_RNEA_KERNEL_DH_HOST
    assert oracle.rel_err(tau.astype(np.float64), ref) <= TOL["float32"]
