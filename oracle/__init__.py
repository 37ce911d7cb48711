"""FP64 CPU oracle for batched robot dynamics -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The CUDA library never links or calls
it, and the two share no code: the oracle is plain sequential C written with
dense 6x6 matrices straight from the recursions of Sec. II (Eqs. id-forward,
id-backward, tau-bias, JSIinv, abi, recursive-fd), compiled with
``-ffp-contract=off``.

Parity status: every function here is pinned by independent tests
(closed forms, a Lagrangian restatement built on scipy's matrix
exponential, invariants, brute-force scan bracketings); none is
"parity unpinned".

The library is built with gcc into ``oracle/_build/liboracle.so`` on first
use (or by ``build()``), on whatever host runs it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["oracle_real.c", "oracle_cs.c"]
_lock = threading.Lock()
_lib = None

DEFAULT_GRAVITY = 9.81


def _stale():
    if not os.path.exists(_SO):
        return True
    t = os.path.getmtime(_SO)
    deps = _SOURCES + ["dyn_body.h"]
    return any(os.path.getmtime(os.path.join(_HERE, d)) > t for d in deps)


def build(force=False):
    """Compile the oracle with gcc (plain C11, -O2, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and not _stale():
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp] + [os.path.join(_HERE, s) for s in _SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            D = ctypes.POINTER(ctypes.c_double)
            I = ctypes.c_int
            IP = ctypes.POINTER(ctypes.c_int)
            lib.oracle_rnea.argtypes = [I, D, D, D, I, D, D, D, D, D]
            lib.oracle_rnea_trace.argtypes = [I, D, D, D, D, D, D, D, D, D, D, D]
            lib.oracle_mass_matrix.argtypes = [I, D, D, D, I, D, D]
            lib.oracle_fd_jsiia.argtypes = [I, D, D, D, I, D, D, D, D, D, IP]
            lib.oracle_fd_aba.argtypes = [I, D, D, D, I, D, D, D, D, D]
            lib.oracle_abi_trace.argtypes = [I, D, D, D, D, D, D]
            lib.oracle_rnea_grad_cs.argtypes = [I, D, D, D, I, D, D, D, D, D, D, D, D]
            for f in ("oracle_rnea", "oracle_rnea_trace", "oracle_mass_matrix",
                      "oracle_fd_jsiia", "oracle_fd_aba", "oracle_abi_trace",
                      "oracle_rnea_grad_cs"):
                getattr(lib, f).restype = None
            _lib = lib
    return _lib


class swapped_library:
    """Context manager: route this module's calls to another build of the
    oracle (used by the mutation tests, which compile deliberately broken
    copies in a temporary folder to show that the pins catch them)."""

    def __init__(self, so_path):
        self.so_path = so_path
        self.saved = None

    def __enter__(self):
        global _lib
        _load()
        self.saved = _lib
        lib = ctypes.CDLL(self.so_path)
        for name in ("oracle_rnea", "oracle_rnea_trace", "oracle_mass_matrix",
                     "oracle_fd_jsiia", "oracle_fd_aba", "oracle_abi_trace",
                     "oracle_rnea_grad_cs"):
            fn = getattr(lib, name)
            fn.argtypes = getattr(self.saved, name).argtypes
            fn.restype = None
        with _lock:
            _lib = lib
        return lib

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self.saved
        return False


def build_variant(out_dir, replacements):
    """Compile a copy of the oracle sources with textual replacements
    {file: [(old, new), ...]} into out_dir; returns the .so path."""
    os.makedirs(out_dir, exist_ok=True)
    for src in _SOURCES + ["dyn_body.h"]:
        text = open(os.path.join(_HERE, src)).read()
        for old, new in replacements.get(src, []):
            if old not in text:
                raise ValueError(f"mutation anchor not found in {src}: {old!r}")
            text = text.replace(old, new, 1)
        with open(os.path.join(out_dir, src), "w") as fh:
            fh.write(text)
    so = os.path.join(out_dir, "liboracle_variant.so")
    cmd = ["gcc", "-std=gnu11", "-O1", "-ffp-contract=off", "-fPIC", "-shared", "-w", "-o", so] + \
        [os.path.join(out_dir, s) for s in _SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    return so


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def default_base(gravity=DEFAULT_GRAVITY):
    """{V_0, dV_0, F_{n+1}}: base at rest, dV_0 = (0, 0, g, 0, 0, 0) (gravity along -z)."""
    b = np.zeros(18)
    b[8] = gravity
    return b


def _model(chain):
    return _f64(chain.M), _f64(chain.S), _f64(chain.inertia), int(chain.n)


def _base(base):
    return default_base() if base is None else _f64(base, (18,))


def rnea(chain, q, qd, qdd, base=None):
    """tau = ID(q, qd, qdd, V_0, dV_0, F_{n+1}) for a batch [B, n]."""
    M, S, J, n = _model(chain)
    q, qd, qdd = (_f64(x).reshape(-1, n) for x in (q, qd, qdd))
    B = q.shape[0]
    tau = np.empty((B, n))
    bs = _base(base)
    _load().oracle_rnea(n, _d(M), _d(S), _d(J), B, _d(q), _d(qd), _d(qdd), _d(bs), _d(tau))
    return tau


def rnea_threaded(chain, q, qd, qdd, base=None, threads=1):
    """Same as :func:`rnea`, the batch split statically over ``threads`` host threads."""
    M, S, J, n = _model(chain)
    q, qd, qdd = (_f64(x).reshape(-1, n) for x in (q, qd, qdd))
    B = q.shape[0]
    tau = np.empty((B, n))
    bs = _base(base)
    lib = _load()
    bounds = np.linspace(0, B, threads + 1).astype(int)

    def work(lo, hi):
        if hi > lo:
            lib.oracle_rnea(n, _d(M), _d(S), _d(J), hi - lo, _d(q[lo:hi]), _d(qd[lo:hi]),
                            _d(qdd[lo:hi]), _d(bs), _d(tau[lo:hi]))

    ts = [threading.Thread(target=work, args=(bounds[k], bounds[k + 1])) for k in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    return tau


def rnea_trace(chain, q, qd, qdd, base=None):
    """One instance: (tau [n], V [n,6], dV [n,6], F [n,6])."""
    M, S, J, n = _model(chain)
    q, qd, qdd = (_f64(x, (n,)) for x in (q, qd, qdd))
    tau = np.empty(n)
    V = np.empty((n, 6))
    dV = np.empty((n, 6))
    F = np.empty((n, 6))
    _load().oracle_rnea_trace(n, _d(M), _d(S), _d(J), _d(q), _d(qd), _d(qdd), _d(_base(base)),
                              _d(tau), _d(V), _d(dV), _d(F))
    return tau, V, dV, F


def mass_matrix(chain, q):
    """Joint-space inertia M(q), [B, n, n], one unit-acceleration ID per column."""
    M, S, J, n = _model(chain)
    q = _f64(q).reshape(-1, n)
    B = q.shape[0]
    out = np.empty((B, n, n))
    _load().oracle_mass_matrix(n, _d(M), _d(S), _d(J), B, _d(q), _d(out))
    return out


def fd_jsiia(chain, q, qd, tau, base=None):
    """Forward dynamics by Cholesky of M(q); returns (qdd [B,n], status [B])."""
    M, S, J, n = _model(chain)
    q, qd, tau = (_f64(x).reshape(-1, n) for x in (q, qd, tau))
    B = q.shape[0]
    qdd = np.empty((B, n))
    st = np.zeros(B, dtype=np.int32)
    _load().oracle_fd_jsiia(n, _d(M), _d(S), _d(J), B, _d(q), _d(qd), _d(tau), _d(_base(base)),
                            _d(qdd), st.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return qdd, st


def fd_aba(chain, q, qd, tau, base=None):
    """Forward dynamics by the articulated-body recursion; returns qdd [B, n]."""
    M, S, J, n = _model(chain)
    q, qd, tau = (_f64(x).reshape(-1, n) for x in (q, qd, tau))
    B = q.shape[0]
    qdd = np.empty((B, n))
    _load().oracle_fd_aba(n, _d(M), _d(S), _d(J), B, _d(q), _d(qd), _d(tau), _d(_base(base)),
                          _d(qdd))
    return qdd


def abi_trace(chain, q):
    """Articulated-body inertias hat J_i [n,6,6] and Omega_i [n] for one state."""
    M, S, J, n = _model(chain)
    q = _f64(q, (n,))
    Jh = np.empty((n, 6, 6))
    Om = np.empty(n)
    _load().oracle_abi_trace(n, _d(M), _d(S), _d(J), _d(q), _d(Jh), _d(Om))
    return Jh, Om


def rnea_grad(chain, q, qd, qdd, w, base=None):
    """Complex-step gradient of sum_b w_b^T tau_b wrt (q, qd, qdd), each [B, n]."""
    M, S, J, n = _model(chain)
    q, qd, qdd, w = (_f64(x).reshape(-1, n) for x in (q, qd, qdd, w))
    B = q.shape[0]
    gq, gqd, gqdd = (np.empty((B, n)) for _ in range(3))
    _load().oracle_rnea_grad_cs(n, _d(M), _d(S), _d(J), B, _d(q), _d(qd), _d(qdd), _d(w),
                                _d(_base(base)), _d(gq), _d(gqd), _d(gqdd))
    return gq, gqd, gqdd


def rel_err(x, ref):
    """Per instance max_i |x - ref| / max_i |ref|, maximised over the batch."""
    x = np.asarray(x, dtype=np.float64).reshape(np.shape(ref)[0], -1)
    ref = np.asarray(ref, dtype=np.float64).reshape(x.shape)
    num = np.max(np.abs(x - ref), axis=1)
    den = np.maximum(np.max(np.abs(ref), axis=1), 1e-300)
    return float(np.max(num / den)) if x.shape[0] else 0.0
