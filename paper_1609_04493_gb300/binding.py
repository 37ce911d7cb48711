"""ctypes binding of librdyn.so (include/rdyn.h). Marshalling only."""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

RD_F32 = 0
RD_F64 = 1
RD_MAX_LINKS = 128
RD_VARIANT_AUTO = 0
RD_VARIANT_SERIAL = 1
RD_VARIANT_SERIAL_RECOMPUTE = 2
RD_VARIANT_SERIAL_RECOMPUTE_CS = 3
RD_VARIANT_SERIAL_REGSTATE = 4
RD_VARIANT_SERIAL_HYBRID = 5
RD_VARIANT_SERIAL_DH = 6
RD_VARIANT_SERIAL_DH_RECOMPUTE = 7
RD_VARIANT_SERIAL_DH_TMEM = 8
RD_VARIANT_SERIAL_DF = 9
RD_FLAG_HOST_COPY = 0x4000
RD_RNEA_KERNEL_DH_HOST = 0x209


RD_FLAG_FAST_TRIG = 0x1000
RD_VJP_AUTO = 0
RD_VJP_STORE = 1
RD_VJP_RECOMPUTE = 2
RD_VJP_FLAG_JOINT_FRAMES = 0x2000
RD_VJP_FLAG_TWO_WARPS = 0x800
RD_VJP_FLAG_ONE_THREAD = 0x400
RD_VJP_FLAG_LANES = 0x100
RD_VJP_FLAG_LANES4 = 0x200
RD_VJP_FLAG_SHARED_STATE = 0x4000
RD_VJP_FLAG_TWO_WARPS_SHARED = 0x8000


def RD_VARIANT_SCAN(lanes):
    return 0x100 | int(lanes)


def RD_TUNE_BLOCK(threads):
    return {32: 5 << 16, 64: 6 << 16, 128: 7 << 16}.get(int(threads), 0)


def RD_TUNE_REGLINKS(links):
    return (int(links) // 4) << 20


def RD_TUNE_STORED_LINKS(links):
    return (int(links) // 4) << 20


_ERRORS = {-1: "RD_ERR_ARG", -2: "RD_ERR_DTYPE", -3: "RD_ERR_RANGE", -4: "RD_ERR_CUDA",
           -5: "RD_ERR_TIMEOUT", -6: "RD_ERR_ALLOC"}

_lock = threading.Lock()
_lib = None


class RdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code


def library_path():
    return _build.SO


def load(build_if_missing=True):
    """Load librdyn.so (building it in-tree first if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and _build.stale():
            _build.build()
        if not os.path.exists(_build.SO):
            raise RuntimeError(f"librdyn.so not found at {_build.SO}; run the build first")
        lib = ctypes.CDLL(_build.SO)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.POINTER(ctypes.c_double)
        lib.rd_model_create.argtypes = [I, D, D, D, ctypes.POINTER(P)]
        lib.rd_model_create.restype = I
        lib.rd_model_destroy.argtypes = [P]
        lib.rd_model_destroy.restype = None
        lib.rd_model_links.argtypes = [P]
        lib.rd_model_links.restype = I
        lib.rnea_batch.argtypes = [P, I, I, P, P, P, P, D, I, P]
        lib.rnea_batch.restype = I
        lib.rnea_batch_host.argtypes = [P, I, I, P, P, P, P, D, I, P]
        lib.rnea_batch_host.restype = I
        lib.rd_last_error.argtypes = []
        lib.rd_last_error.restype = ctypes.c_char_p
        lib.rd_version.argtypes = []
        lib.rd_version.restype = I
        lib.rnea_vjp.argtypes = [P, I, I, P, P, P, P, P, P, P, D, I, P, ctypes.c_size_t, P]
        lib.rnea_vjp.restype = I
        lib.rnea_vjp_workspace_size.argtypes = [P, I, I, ctypes.POINTER(ctypes.c_size_t)]
        lib.rnea_vjp_workspace_size.restype = I
        lib.aba_batch.argtypes = [P, I, I, P, P, P, P, D, P, I, P, ctypes.c_size_t, P]
        lib.aba_batch.restype = I
        lib.aba_workspace_size.argtypes = [P, I, I, I, ctypes.POINTER(ctypes.c_size_t)]
        lib.aba_workspace_size.restype = I
        IPt = ctypes.POINTER(ctypes.c_int)
        LLP = ctypes.POINTER(ctypes.c_longlong)
        lib.rd_fleet_create.argtypes = [I, IPt, D, D, D, ctypes.POINTER(P)]
        lib.rd_fleet_create.restype = I
        lib.rd_fleet_destroy.argtypes = [P]
        lib.rd_fleet_destroy.restype = None
        lib.rd_plan_create.argtypes = [P, I, IPt, IPt, I, ctypes.POINTER(P)]
        lib.rd_plan_create.restype = I
        lib.rd_plan_destroy.argtypes = [P]
        lib.rd_plan_destroy.restype = None
        lib.rd_plan_total_joints.argtypes = [P]
        lib.rd_plan_total_joints.restype = ctypes.c_longlong
        lib.rd_plan_offsets.argtypes = [P, LLP]
        lib.rd_plan_offsets.restype = I
        lib.rd_plan_groups.argtypes = [P]
        lib.rd_plan_groups.restype = I
        lib.fleet_batch.argtypes = [P, P, P, P, P, D, P, I, I, P]
        lib.fleet_batch.restype = I
        lib.jsiia_batch.argtypes = [P, I, I, P, P, P, P, D, P, P]
        lib.jsiia_batch.restype = I
        lib.rd_measure_fma_peak.argtypes = [I, D, P]
        lib.rd_measure_fma_peak.restype = I
        lib.rd_joint_trig.argtypes = [I, P, P, P, I, P]
        lib.rd_joint_trig.restype = I
        lib.rd_joint_trig_df.argtypes = [P, P, P, I, P]
        lib.rd_joint_trig_df.restype = I
        IP = ctypes.POINTER(ctypes.c_int)
        lib.rd_rnea_last_config.argtypes = [IP, IP, IP]
        lib.rd_rnea_last_config.restype = I
        lib.rd_rnea_last_state_layout.argtypes = [IP, IP]
        lib.rd_rnea_last_state_layout.restype = I
        _lib = lib
        return lib


def _check(rc):
    if rc != 0:
        raise RdError(rc, _lib.rd_last_error().decode(errors="replace"))


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def measure_fma_peak(dtype="float32", stream=None):
    """Measured FMA throughput of the current GPU in TFLOP/s (diagnostic)."""
    import torch

    lib = load()
    out = ctypes.c_double()
    st = stream or torch.cuda.current_stream()
    _check(lib.rd_measure_fma_peak(RD_F32 if dtype == "float32" else RD_F64, ctypes.byref(out),
                                   ctypes.c_void_p(st.cuda_stream)))
    return out.value


RD_RNEA_KERNEL_DH_PARAM = 0x206
RD_RNEA_KERNEL_DH_TMEM = 0x208


def rnea_last_config():
    """(kernel, block, stored_links) of this thread's last rnea_batch launch."""
    lib = load()
    k, b, s = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib.rd_rnea_last_config(ctypes.byref(k), ctypes.byref(b), ctypes.byref(s)))
    return k.value, b.value, s.value


def rnea_last_state_layout():
    """(register links, ring chunks) of this thread's last rnea_batch launch of
    the stored-state common-normal kernel (rd_rnea_last_state_layout)."""
    lib = load()
    r, c = ctypes.c_int(), ctypes.c_int()
    _check(lib.rd_rnea_last_state_layout(ctypes.byref(r), ctypes.byref(c)))
    return r.value, c.value


def rnea_last_register_links():
    """Of the stored links of this thread's last rnea_batch launch, how many the
    kernel kept in registers."""
    return rnea_last_state_layout()[0]


def joint_trig(x, fast=False, stream=None):
    """(sin x, cos x) as the FP32 common-normal-frame kernels evaluate them
    (rd_joint_trig; diagnostic). x: contiguous float32 CUDA tensor."""
    import torch

    lib = load()
    if not (x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()):
        raise ValueError("joint_trig expects a contiguous float32 CUDA tensor")
    s, c = torch.empty_like(x), torch.empty_like(x)
    st = stream or torch.cuda.current_stream(x.device)
    _check(lib.rd_joint_trig(RD_FLAG_FAST_TRIG if fast else 0, x.data_ptr(), s.data_ptr(),
                             c.data_ptr(), x.numel(), ctypes.c_void_p(st.cuda_stream)))
    return s, c


def joint_trig_df(x, stream=None):
    """(sin x, cos x) as the double-float kernel of FP64 data evaluates them
    (rd_joint_trig_df; diagnostic). x: contiguous float64 CUDA tensor."""
    import torch

    lib = load()
    if not (x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
        raise ValueError("joint_trig_df expects a contiguous float64 CUDA tensor")
    s, c = torch.empty_like(x), torch.empty_like(x)
    st = stream or torch.cuda.current_stream(x.device)
    _check(lib.rd_joint_trig_df(x.data_ptr(), s.data_ptr(), c.data_ptr(), x.numel(),
                                ctypes.c_void_p(st.cuda_stream)))
    return s, c


def default_base(gravity=9.81):
    """{V_0, dV_0, F_{n+1}} for a base at rest under gravity along -z."""
    b = np.zeros(18)
    b[8] = gravity
    return b


class Model:
    """A serial chain resident on the current CUDA device (rd_model_create)."""

    def __init__(self, M, S=None, inertia=None):
        if S is None and inertia is None:  # a chain object with .M, .S, .inertia
            M, S, inertia = M.M, M.S, M.inertia
        lib = load()
        self._M = np.ascontiguousarray(M, dtype=np.float64).reshape(-1, 12)
        self._S = np.ascontiguousarray(S, dtype=np.float64).reshape(-1, 6)
        self._J = np.ascontiguousarray(inertia, dtype=np.float64).reshape(-1, 10)
        n = self._M.shape[0]
        if self._S.shape[0] != n or self._J.shape[0] != n:
            raise ValueError("M, S and inertia must describe the same number of links")
        h = ctypes.c_void_p()
        _check(lib.rd_model_create(n, _dptr(self._M), _dptr(self._S), _dptr(self._J),
                                   ctypes.byref(h)))
        self._h = h
        self.n = n

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.rd_model_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _dtype_code(t):
    import torch

    if t.dtype == torch.float32:
        return RD_F32
    if t.dtype == torch.float64:
        return RD_F64
    raise TypeError(f"dtype {t.dtype} not supported (float32 or float64)")


def _base_arg(base):
    if base is None:
        return None, None
    b = np.ascontiguousarray(base, dtype=np.float64).reshape(18)
    return b, _dptr(b)


def _check_batch(model, *ts):
    import torch

    ref = ts[0]
    for t in ts:
        if not isinstance(t, torch.Tensor):
            raise TypeError("expected torch tensors")
        if not t.is_cuda:
            raise ValueError("tensors must be on a CUDA device (use rnea_host for host arrays)")
        if t.dtype != ref.dtype or t.shape != ref.shape:
            raise ValueError("all batch tensors must share dtype and shape")
        if not t.is_contiguous():
            raise ValueError("batch tensors must be contiguous [B, n]")
    if ref.dim() != 2 or ref.shape[1] != model.n:
        raise ValueError(f"expected shape [B, {model.n}], got {tuple(ref.shape)}")


def rnea(model, q, qd, qdd, out=None, base=None, variant=RD_VARIANT_AUTO, stream=None):
    """tau = ID(q, qd, qdd, V_0, dV_0, F_{n+1}) on the GPU (rnea_batch)."""
    import torch

    _check_batch(model, q, qd, qdd)
    if out is None:
        out = torch.empty_like(q)
    else:
        _check_batch(model, q, out)
    if stream is None:
        stream = torch.cuda.current_stream(q.device)
    keep, bp = _base_arg(base)
    _check(_lib.rnea_batch(model.handle, q.shape[0], _dtype_code(q), q.data_ptr(), qd.data_ptr(),
                           qdd.data_ptr(), out.data_ptr(), bp, int(variant),
                           ctypes.c_void_p(stream.cuda_stream)))
    del keep
    return out


def rnea_host(model, q, qd, qdd, out=None, base=None, variant=RD_VARIANT_AUTO, stream=None):
    """Inverse dynamics on host arrays (rnea_batch_host); returns when tau is on
    the host. Pinned FP32 arrays (n % 4 == 0, n <= 64) are read and written in
    place by the kernel; other arrays are staged through device buffers with
    the copy engines (variant | RD_FLAG_HOST_COPY forces that). Accepts CPU
    torch tensors or numpy arrays; pinned tensors move fastest."""
    import torch

    arrs = [q, qd, qdd]
    if isinstance(q, np.ndarray):
        arrs = [torch.from_numpy(np.ascontiguousarray(a)) for a in arrs]
    for a in arrs:
        if a.is_cuda or not a.is_contiguous() or a.shape != arrs[0].shape or a.dtype != arrs[0].dtype:
            raise ValueError("rnea_host expects contiguous host arrays of one shape and dtype")
    if arrs[0].dim() != 2 or arrs[0].shape[1] != model.n:
        raise ValueError(f"expected shape [B, {model.n}]")
    if out is None:  # pinned when the inputs are, so the recorded pipeline can serve it
        out = torch.empty(arrs[0].shape, dtype=arrs[0].dtype,
                          pin_memory=bool(arrs[0].is_pinned()))
    if stream is None:
        stream = torch.cuda.current_stream()
    keep, bp = _base_arg(base)
    load()
    _check(_lib.rnea_batch_host(model.handle, arrs[0].shape[0], _dtype_code(arrs[0]),
                                arrs[0].data_ptr(), arrs[1].data_ptr(), arrs[2].data_ptr(),
                                out.data_ptr(), bp, int(variant),
                                ctypes.c_void_p(stream.cuda_stream)))
    del keep
    return out


def vjp_workspace_bytes(model, B, dtype_code):
    """Workspace bytes rnea_vjp needs in store mode for B states."""
    lib = load()
    out = ctypes.c_size_t()
    _check(lib.rnea_vjp_workspace_size(model.handle, int(B), int(dtype_code), ctypes.byref(out)))
    return out.value


def rnea_vjp(model, q, qd, qdd, w, base=None, mode=RD_VJP_AUTO, workspace=None, stream=None,
             out=None):
    """(gq, gqd, gqdd) = d(w^T tau)/d(q, qd, qdd) on the GPU (rnea_vjp).

    ``mode`` is RD_VJP_AUTO, RD_VJP_STORE or RD_VJP_RECOMPUTE, optionally OR-ed
    with RD_FLAG_FAST_TRIG, RD_VJP_FLAG_JOINT_FRAMES, and for FP32 recompute
    RD_VJP_FLAG_TWO_WARPS or RD_VJP_FLAG_ONE_THREAD (each instance split between
    two warps, or not; by default split for chains over 64 links at B <= 8192).
    In store mode (or AUTO with a workspace) the caller may pass a preallocated
    uint8 CUDA tensor as ``workspace``; for RD_VJP_STORE without one, a tensor of
    the required size is allocated here (torch's allocator), never in the library."""
    import torch

    _check_batch(model, q, qd, qdd, w)
    gq, gqd, gqdd = out if out is not None else (torch.empty_like(q) for _ in range(3))
    code = _dtype_code(q)
    ws_ptr, ws_bytes = None, 0
    if workspace is None and (mode & 0xff) == RD_VJP_STORE:
        workspace = torch.empty(vjp_workspace_bytes(model, q.shape[0], code), dtype=torch.uint8,
                                device=q.device)
    if workspace is not None:
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    if stream is None:
        stream = torch.cuda.current_stream(q.device)
    keep, bp = _base_arg(base)
    _check(_lib.rnea_vjp(model.handle, q.shape[0], code, q.data_ptr(), qd.data_ptr(),
                         qdd.data_ptr(), w.data_ptr(), gq.data_ptr(), gqd.data_ptr(),
                         gqdd.data_ptr(), bp, int(mode), ws_ptr, ws_bytes,
                         ctypes.c_void_p(stream.cuda_stream)))
    del keep
    return gq, gqd, gqdd


def _make_function():
    import torch

    class RNEAFunction(torch.autograd.Function):
        """tau = ID(q, qd, qdd) with a backward pass through the adjoint kernel."""

        @staticmethod
        def forward(ctx, model, q, qd, qdd, base=None, vjp_mode=RD_VJP_RECOMPUTE):
            q, qd, qdd = q.contiguous(), qd.contiguous(), qdd.contiguous()
            ctx.model = model
            ctx.base = base
            ctx.vjp_mode = vjp_mode
            ctx.save_for_backward(q, qd, qdd)
            return rnea(model, q, qd, qdd, base=base)

        @staticmethod
        def backward(ctx, grad_tau):
            q, qd, qdd = ctx.saved_tensors
            gq, gqd, gqdd = rnea_vjp(ctx.model, q, qd, qdd, grad_tau.contiguous(), base=ctx.base,
                                     mode=ctx.vjp_mode)
            return None, gq, gqd, gqdd, None, None

    return RNEAFunction


_RNEAFunction = None


def rnea_autograd(model, q, qd, qdd, base=None, vjp_mode=RD_VJP_RECOMPUTE):
    """Differentiable inverse dynamics: a torch.autograd.Function whose backward
    is the library's adjoint kernel."""
    global _RNEAFunction
    if _RNEAFunction is None:
        _RNEAFunction = _make_function()
    return _RNEAFunction.apply(model, q, qd, qdd, base, vjp_mode)


RD_ABA_SCANS_IN_DTYPE = 0x1
RD_ABA_JOINT_FRAMES = 0x2
RD_ABA_FP64_UPDATE = 0x4
RD_ABA_EXTENDED_BIAS = 0x8
RD_ABA_FP32_BIAS = 0x10
RD_ABA_EXTENDED_BIAS_LINKS = 64
RD_ABA_WARP_PER_INSTANCE = 0x20
RD_ABA_THREAD_PER_INSTANCE = 0x40
RD_ABA_TWO_WARPS = 0x80
RD_ABA_THREE_WARPS = 0x100
RD_ABA_TEST_WITHHOLD = 0x40000000
RD_WARN_SINGULAR = 1
RD_WARN_TIMEOUT = 2


def aba_workspace_bytes(model, B, dtype_code, flags=0):
    """Workspace bytes aba_batch needs for B states."""
    lib = load()
    out = ctypes.c_size_t()
    _check(lib.aba_workspace_size(model.handle, int(B), int(dtype_code), int(flags),
                                  ctypes.byref(out)))
    return out.value


def aba(model, q, qd, tau, base=None, workspace=None, status=None, out=None, stream=None,
        flags=0):
    """qdd = FD(q, qd, tau) on the GPU (aba_batch). A workspace (uint8 CUDA tensor)
    of aba_workspace_bytes() is taken from torch's allocator when not given; pass a
    preallocated one (and ``out``) for allocation-free repeated calls. ``status``:
    optional int32 CUDA tensor [B] receiving per-instance warnings."""
    import torch

    _check_batch(model, q, qd, tau)
    qdd = out if out is not None else torch.empty_like(q)
    code = _dtype_code(q)
    if workspace is None:
        workspace = torch.empty(aba_workspace_bytes(model, q.shape[0], code, flags),
                                dtype=torch.uint8, device=q.device)
    if stream is None:
        stream = torch.cuda.current_stream(q.device)
    keep, bp = _base_arg(base)
    st_ptr = None
    if status is not None:
        if status.dtype != torch.int32 or not status.is_cuda or status.numel() < q.shape[0]:
            raise ValueError("status must be an int32 CUDA tensor with B entries")
        st_ptr = status.data_ptr()
    _check(_lib.aba_batch(model.handle, q.shape[0], code, q.data_ptr(), qd.data_ptr(),
                          tau.data_ptr(), qdd.data_ptr(), bp, st_ptr, int(flags), workspace.data_ptr(),
                          workspace.numel() * workspace.element_size(),
                          ctypes.c_void_p(stream.cuda_stream)))
    del keep
    return qdd


RD_REQ_ID = 0
RD_REQ_FD = 1
RD_SCHED_PERSISTENT = 0
RD_SCHED_PER_GROUP = 1
RD_FLEET_FP64_UPDATE = 0x10


RD_TUNE_TWO_STAGE_RING = 0x8000


def RD_TUNE_REG_STATE_LINKS(links):
    return (int(links) // 4) << 28


def RD_FLEET_TUNE(log2_threads, ctas_per_sm):
    return (int(log2_threads) << 8) | int(ctas_per_sm)


def RD_FLEET_TWO_WARPS(min_links):
    return int(min_links) << 16


def RD_FLEET_THREE_WARPS(min_links):
    return (int(min_links) << 16) | (1 << 24)


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


class Fleet:
    """Many chains of different lengths on the current device (rd_fleet_create)."""

    def __init__(self, chains):
        lib = load()
        self.n = np.ascontiguousarray([c.n for c in chains], dtype=np.int32)
        self._M = np.ascontiguousarray(np.concatenate([c.M for c in chains]), dtype=np.float64)
        self._S = np.ascontiguousarray(np.concatenate([c.S for c in chains]), dtype=np.float64)
        self._J = np.ascontiguousarray(np.concatenate([c.inertia for c in chains]), dtype=np.float64)
        h = ctypes.c_void_p()
        _check(lib.rd_fleet_create(len(chains), _iptr(self.n), _dptr(self._M), _dptr(self._S),
                                   _dptr(self._J), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.rd_fleet_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """A fixed request set on a fleet (rd_plan_create): robots[R], kinds[R] (RD_REQ_*)."""

    def __init__(self, fleet, robots, kinds, dtype="float32"):
        lib = load()
        self.fleet = fleet
        self.robots = np.ascontiguousarray(robots, dtype=np.int32)
        self.kinds = np.ascontiguousarray(kinds, dtype=np.int32)
        self.R = int(self.robots.shape[0])
        self.dtype = dtype
        h = ctypes.c_void_p()
        _check(lib.rd_plan_create(fleet.handle, self.R, _iptr(self.robots), _iptr(self.kinds),
                                  RD_F32 if dtype == "float32" else RD_F64, ctypes.byref(h)))
        self._h = h
        self.total_joints = int(lib.rd_plan_total_joints(h))
        self.offsets = np.empty(self.R, dtype=np.int64)
        _check(lib.rd_plan_offsets(h, self.offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))))
        self.groups = int(lib.rd_plan_groups(h))
        self.lengths = fleet.n[self.robots]

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.rd_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fleet_batch(plan, q, qd, in2, out=None, base=None, status=None,
                schedule=RD_SCHED_PERSISTENT, tune=0, stream=None):
    """Evaluate every request of ``plan`` (fleet_batch). q, qd, in2: 1-D CUDA tensors
    of plan.total_joints elements, request r at [offsets[r], offsets[r] + n_r);
    in2 holds qdd for inverse and tau for forward dynamics requests; returns out
    (tau, resp. qdd, in the same layout)."""
    import torch

    for t in (q, qd, in2):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
            raise ValueError("fleet_batch expects contiguous CUDA tensors")
        if t.numel() != plan.total_joints:
            raise ValueError(f"expected {plan.total_joints} joint values, got {t.numel()}")
        want = torch.float32 if plan.dtype == "float32" else torch.float64
        if t.dtype != want:
            raise TypeError(f"plan dtype is {plan.dtype}")
    if out is None:
        out = torch.empty_like(q)
    if stream is None:
        stream = torch.cuda.current_stream(q.device)
    keep, bp = _base_arg(base)
    st_ptr = status.data_ptr() if status is not None else None
    _check(_lib.fleet_batch(plan.handle, q.data_ptr(), qd.data_ptr(), in2.data_ptr(),
                            out.data_ptr(), bp, st_ptr, int(schedule), int(tune),
                            ctypes.c_void_p(stream.cuda_stream)))
    del keep
    return out


def jsiia(model, q, qd, tau, base=None, status=None, out=None, stream=None):
    """qdd = FD(q, qd, tau) by joint-space-inertia inversion (jsiia_batch), n <= 32."""
    import torch

    _check_batch(model, q, qd, tau)
    qdd = out if out is not None else torch.empty_like(q)
    if stream is None:
        stream = torch.cuda.current_stream(q.device)
    keep, bp = _base_arg(base)
    st_ptr = status.data_ptr() if status is not None else None
    _check(_lib.jsiia_batch(model.handle, q.shape[0], _dtype_code(q), q.data_ptr(), qd.data_ptr(),
                            tau.data_ptr(), qdd.data_ptr(), bp, st_ptr,
                            ctypes.c_void_p(stream.cuda_stream)))
    del keep
    return qdd


def forward_dynamics(model, q, qd, tau, method="auto", base=None, status=None, workspace=None,
                     out=None, stream=None):
    """qdd = FD(q, qd, tau) by the articulated-body algorithm (aba_batch) or the
    joint-space-inertia solve (jsiia_batch). ``auto`` takes the articulated-body
    algorithm, which on GB300 leads at every size measured once small batches
    run with three warps per 32 instances (FP32, µs, JSIIA / ABA: n = 8, B = 256:
    30.3 / 19.8; n = 16: 62.2 / 39.0; n = 32, B = 32 / 256 / 1024: 108 / 78.5,
    108.5 / 78.8, 162 / 79.8; larger batches and FP64: ABA by a wider margin).
    ``jsiia`` stays available (n <= 32)."""
    if method == "auto":
        method = "aba"
    if method == "jsiia":
        return jsiia(model, q, qd, tau, base=base, status=status, out=out, stream=stream)
    if method == "aba":
        return aba(model, q, qd, tau, base=base, workspace=workspace, status=status, out=out,
                   stream=stream)
    raise ValueError(f"unknown method {method!r}")
