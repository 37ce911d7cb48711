"""Batched serial-chain dynamics on one GB300 GPU.

A thin Python binding over the C ABI of ``librdyn.so`` (include/rdyn.h):
argument marshalling only. Every step of the computation runs in the
library's CUDA kernels; there is no CPU or PyTorch fallback, and calls fail
loudly when the library or a CUDA device is missing. PyTorch supplies
device memory and streams.
"""
from .binding import (  # noqa: F401
    RD_F32,
    RD_F64,
    RD_MAX_LINKS,
    RD_VARIANT_AUTO,
    RD_VARIANT_SERIAL,
    RD_VARIANT_SERIAL_RECOMPUTE,
    RD_VARIANT_SERIAL_RECOMPUTE_CS,
    RD_TUNE_BLOCK,
    RD_TUNE_REGLINKS,
    RD_TUNE_STORED_LINKS,
    RD_VARIANT_SERIAL_REGSTATE,
    RD_VARIANT_SERIAL_HYBRID,
    RD_VARIANT_SERIAL_DH,
    RD_VARIANT_SERIAL_DH_RECOMPUTE,
    RD_VARIANT_SCAN,
    RD_FLAG_FAST_TRIG,
    RdError,
    Model,
    load,
    library_path,
    rnea,
    rnea_host,
    rnea_vjp,
    aba,
    jsiia,
    forward_dynamics,
    aba_workspace_bytes,
    RD_ABA_SCANS_IN_DTYPE,
    rnea_autograd,
    vjp_workspace_bytes,
    RD_VJP_AUTO,
    RD_VJP_STORE,
    RD_VJP_RECOMPUTE,
    default_base,
    measure_fma_peak,
    joint_trig,
    Fleet,
    Plan,
    fleet_batch,
    RD_REQ_ID,
    RD_REQ_FD,
    RD_SCHED_PERSISTENT,
    RD_SCHED_PER_GROUP,
    RD_FLEET_TUNE,
)
