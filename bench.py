#!/usr/bin/env python3
"""Benchmark: batched inverse dynamics (RNEA) on GB300.

Headline workload: one 32-link serial chain (the seeded random-robot recipe
of the experiments, Sec. V), B = 65536 joint states per step, FP32 arithmetic;
one step = one rnea_batch call over the batch (forward scan + backward scan,
Algorithm 1). Beside it, on the same GPU and run: the same workload in FP64,
and the host-array entry point (copies in the timed region).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). With N > 1 (torchrun), every rank times its own
B = 65536 batch on its own GPU (instances are independent: no collective on
the data path); value = all ranks' evaluations / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_LINKS = 32
BATCH = 65536
METRIC = "RNEA evals/s at n=32,B=65536 FP32 vs FP64; adjoint evals/s; % of roofline"
UNIT = "evals/s"
WORKLOAD = "rnea_n32_B65536"
ROTATE = 8  # input sets cycled between steps; 8 x 33.5 MB > 2 x L2 (129 MB)
# Algorithmic arithmetic of one link of the recursion of Sec. II-A with general
# link transforms, FMA = 2: transform f = M exp(S q) by the Rodrigues formula and
# a 3x4 compose (~135), forward step (~150), bias wrench (~125), backward step
# (~50), torque (~11). The roofline's "achieved" divides this fixed count by
# the measured time; the kernel's own count is reported beside it.
ALGO_FLOP_PER_LINK = 470
# Executed arithmetic of the joint-frame kernels per link (FMA = 2): rotation 18
# + forward step 94 + bias wrench 93 + carry 60.
JOINT_FRAME_FLOP_PER_LINK = 265


def dh_param_flops(n, K):
    """Executed arithmetic (FMA = 2) of one instance in the common-normal kernel
    with full state for links 0..K-1: a stored link costs sin/cos 26 + rotation
    products 4 + forward step 86 + bias wrench 93 + backward carry 44 + products 4;
    a link without full state adds the re-derivation of its motion (86) and
    moves its bias wrench to the backward sweep; the top link adds instead of
    carrying (-38) and the lowest re-derived link needs no inverse step (-86)."""
    stored, rederived = 257, 343
    total = K * stored + (n - K) * rederived - 38
    if K < n:
        total -= 86
    return total


# adjoint arithmetic per link of the common-normal kernel the bench runs (FMA = 2):
# sweep 1 155 (sin/cos 26, rotation products 4, motion step 86, wrench-adjoint
# step 39); sweep 2 466 (products 4, bias wrench 93, carry 44, three inertia
# products 126, ad terms 30, seeds 42, two adjoint carries 88 and their coupling
# 8, gradients 31); recompute mode adds 151 (sin/cos 26, inverse motion step 86,
# inverse wrench-adjoint step 39)
VJP_FLOP_PER_LINK = {1: 621, 2: 772}
# algorithmic arithmetic of the adjoint per link: about three inverse-dynamics
# passes of the general formulation above
VJP_ALGO_FLOP_PER_LINK = 1400
# forward dynamics per link (articulated-body algorithm), FMA = 2: ~720 FP32
# flop (bias motion and wrenches, backward wrench carry, z_hat / lambda
# transforms) and ~800 FP64 flop (articulated-inertia congruence, the rank-one
# update and the Omega solves), the split of the design's precision plan (the
# latter in FP64 or double-float arithmetic)
FD_FLOP32_PER_LINK = 720
FD_FLOP64_PER_LINK = 800
# executed arithmetic of the common-normal forward-dynamics kernel per link with
# the FP64 update: FP32 257 (sin/cos 26, products 4, bias motion 86, bias wrench
# 93, wrench carry 44, products 4); FP64 400 (projected inertia 35, two plane
# rotations and the shift of the articulated-inertia update 235, z_hat carry
# 60, Omega solve 12, lambda step 56)
FD_EXEC_FLOP32_PER_LINK = 257
FD_EXEC_FLOP64_PER_LINK = 400
# the default for FP32 data carries those FP64 operations in double-float
# arithmetic on the FP32 pipe: FP32-pipe instructions executed per link, from
# the FMA-pipe count of an ncu capture at n = 64, B = 16384 (99.7 M warp
# instructions, 94% of all)
FD_DF_EXEC_FP32_INST_PER_LINK = 3043
# FP32-pipe instructions per link of the double-float kernel for FP64 data
# (RD_VARIANT_SERIAL_DF), from the FMA-pipe count of an ncu capture at n = 32,
# B = 65536 (166.2 M warp instructions, 92% of all)
RNEA_DF_EXEC_FP32_INST_PER_LINK = 2535
# bytes an inverse-dynamics link of the uneven workload moves: q, qd, qdd, tau
# (16) plus its robot's constants streamed per request (112)
UNEVEN_ID_BYTES_PER_LINK = 128
# Peaks: FP32 lanes and FP64 fused multiply-adds per SM per clock (GB300:
# 1.25 TFLOP/s FP64 nominal at 152 SMs and 2.07 GHz). The bench multiplies them
# by the device's SM count and the median SM clock sampled while it ran.
SM_COUNT_NOMINAL = 152
SM_MAX_MHZ = 2070.0
FP32_LANES_PER_SM = 128
FP64_FMA_PER_SM_CLK = 2


def fp32_peak_tflops(sm_count=SM_COUNT_NOMINAL, mhz=SM_MAX_MHZ):
    return sm_count * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


def fp64_peak_tflops(sm_count=SM_COUNT_NOMINAL, mhz=SM_MAX_MHZ):
    return sm_count * FP64_FMA_PER_SM_CLK * 2 * mhz * 1e6 / 1e12


def fp32_inst_rate(sm_count=SM_COUNT_NOMINAL, mhz=SM_MAX_MHZ):
    """FP32-pipe thread instructions per second."""
    return sm_count * FP32_LANES_PER_SM * mhz * 1e6


def rnd(x, digits=4):
    """Round every float in a nested structure to `digits` significant digits
    (keeps the printed line short)."""
    if isinstance(x, float):
        return float(f"{x:.{digits}g}") if x == x and abs(x) != float("inf") else x
    if isinstance(x, dict):
        return {k: rnd(v, digits) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [rnd(v, digits) for v in x]
    return x


def short_us(t):
    """Three significant digits; whole numbers from 100 on (a shorter line)."""
    v = float(f"{t:.3g}")
    return int(v) if v >= 100 else v


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--quick", action="store_true", help="skip auxiliary measurements")
    p.add_argument("--no-uneven", action="store_true", help="skip the 100000-request workload")
    p.add_argument("--kernel-only",
                   choices=["f32", "f64", "f64df", "host", "vjp", "vjplane", "vjppair", "vjpsmem",
                            "aba", "aba64",
                            "abawarp", "abapair", "abatri", "abatri1k", "fleet", "fleetpair",
                            "fleettri64"],
                   default=None,
                   help="profiling case: W + K plain launches of one kernel, no JSON "
                        "(f32/f64: RNEA n=32 B=65536; f64df: the same FP64 data in double-float "
                        "arithmetic; host: rnea_batch_host on pinned FP32 arrays, the same "
                        "size; vjp: adjoint n=32 B=8192; vjplane: adjoint n=32 B=4096, 8 lanes "
                        "per instance; vjppair / vjpsmem: adjoint n=32 B=8192, two warps per 32 "
                        "instances / state in shared memory; aba: forward dynamics n=64 B=16384 (double-float updates; "
                        "aba64: FP64 updates); abawarp: forward dynamics n=64 B=1024, one warp per "
                        "instance; abapair / abatri: forward dynamics n=64 B=16384, two / three "
                        "warps per 32 instances; abatri1k: three warps at B=1024; fleet: 20000 "
                        "mixed requests; fleetpair: the same "
                        "with warp pairs for forward-dynamics chains from 65 links; fleettri64: "
                        "warp triples from 65 links, FP64 updates)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def init_dist(world):
    if world <= 1:
        return None
    import torch.distributed as dist

    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group("gloo")
    return dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x):
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples (every 100 ms) stamped on arrival; regions marked by wall time."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.samples = []
        self.regions = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._reader, daemon=True).start()
        except OSError:
            self.proc = None

    def _reader(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            if self.uuid and parts[0] != self.uuid:
                continue
            try:
                sm, smax = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            active = [r for r, v in zip(self.REASONS, parts[5:9]) if v.lower() == "active"]
            self.samples.append((time.time(), sm, smax, active))

    def region(self, t0, t1):
        self.regions.append((t0, t1))

    def stop(self):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        inside = [s for s in self.samples if any(a - 0.05 <= s[0] <= b + 0.05 for a, b in self.regions)]
        use = inside if inside else self.samples
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        reasons = sorted({r for s in use for r in s[3]})
        return {"sm_mhz": statistics.median(s[1] for s in use),
                "sm_max_mhz": max(s[2] for s in use), "reasons": reasons,
                "samples": len(use), "samples_in_timed_regions": len(inside)}


# ---------------------------------------------------------------- profiles

def recorded_traffic(kernel_tag):
    """Per-launch DRAM bytes from the committed ncu summary for this kernel, if it
    was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    h = re.search(r"kernel_sources_sha256:\s*([0-9a-f]+)", text)
    if not m or not h or h.group(1) != kernel_sources_hash():
        return None
    return float(m.group(1))


# Sources that define the headline kernel's code: a profile summary is matched
# to them, so its counters go stale when the kernel changes.
RNEA_KERNEL_SOURCES = ("spatial.cuh", "spatial_dh.cuh", "rnea_serial.cuh", "rnea_dh.cuh",
                       "rnea_dhp.cuh", "trig_poly.cuh")


def kernel_sources_hash(files=RNEA_KERNEL_SOURCES):
    d = os.path.join(ROOT, "paper_1609_04493_gb300", "csrc")
    hs = hashlib.sha256()
    for f in files:
        hs.update(f.encode())
        hs.update(open(os.path.join(d, f), "rb").read())
    return hs.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            return json.load(open(path))
        except ValueError:
            return {}
    return {}


# --------------------------------------------------------------- our arm

def make_inputs(torch, dev, dtype, sets, seed0):
    import chaingen

    out = []
    for r in range(sets):
        st = chaingen.make_states(BATCH, N_LINKS, seed=seed0 + r)
        d = {k: torch.from_numpy(st[k]).to(device=dev, dtype=dtype) for k in ("q", "qd", "qdd")}
        d["tau"] = torch.empty_like(d["q"])
        out.append(d)
    return out


def capture(torch, rd, model, sets, count, variant=0):
    """CUDA graph of `count` rnea_batch launches cycling through the input sets."""
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        rd.rnea(model, sets[0]["q"], sets[0]["qd"], sets[0]["qdd"], out=sets[0]["tau"],
                variant=variant)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            for k in range(count):
                x = sets[k % len(sets)]
                rd.rnea(model, x["q"], x["qd"], x["qdd"], out=x["tau"], variant=variant)
    torch.cuda.synchronize()
    return g


def capture_calls(torch, fn, count):
    """CUDA graph of `count` calls of fn(k)."""
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn(0)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            for k in range(count):
                fn(k)
    torch.cuda.synchronize()
    return g


def time_calls(torch, fn, steps, warmup, dist, sampler):
    gw = capture_calls(torch, fn, max(warmup, 1))
    gw.replay()
    torch.cuda.synchronize()
    g = capture_calls(torch, fn, steps)
    return max_over_ranks(dist, timed_graph(torch, g, dist, sampler))


class Peaks:
    """Roofline denominators for the device and the clock it ran at."""

    def __init__(self, sm_count, mhz):
        self.sm, self.mhz = sm_count, mhz
        self.f32 = fp32_peak_tflops(sm_count, mhz) * 1e12  # flop/s
        self.f64 = fp64_peak_tflops(sm_count, mhz) * 1e12
        self.i32 = fp32_inst_rate(sm_count, mhz)           # FP32-pipe instructions/s
        self.hbm = measured_peaks().get("hbm_gbs", 6800.0) * 1e9  # B/s


def adjoint_section(torch, rd, chaingen, model, dev, dist, sampler, K):
    """Seconds per rnea_vjp call at n = 32 FP32: recompute (the library's
    mapping) at B = 4096, 8192 and 262144, store at 8192 and 262144 (the
    workspace then holds 671 MB of forward state), and at 8192 each
    mapping by flag: one thread, shared-memory state, 8 lanes, two warps, two
    warps with shared-memory state."""
    raw = {}
    R = rd.RD_VJP_RECOMPUTE
    for B, mode in ((4096, R), (8192, R), (262144, R), (8192, rd.RD_VJP_STORE),
                    (262144, rd.RD_VJP_STORE)):
        sets = []
        nsets = 2 if B > 100000 else 8
        for r in range(nsets):
            st = chaingen.make_states(B, N_LINKS, seed=5000 + r, kinds=("q", "qd", "qdd", "w"))
            x = [torch.from_numpy(st[k]).to(dev, torch.float32) for k in ("q", "qd", "qdd", "w")]
            sets.append((x, tuple(torch.empty_like(x[0]) for _ in range(3))))
        ws = None
        if mode == rd.RD_VJP_STORE:
            ws = torch.empty(rd.vjp_workspace_bytes(model, B, 0), dtype=torch.uint8, device=dev)
        steps = max(3, min(K, 200 if B < 100000 else 50))

        def timed(md):
            def call(k):
                x, o = sets[k % len(sets)]
                rd.rnea_vjp(model, *x, mode=md, workspace=ws, out=o)
            return time_calls(torch, call, steps, 3, dist, sampler) / steps

        name = f"B{B}_{'store' if mode == rd.RD_VJP_STORE else 'recompute'}"
        raw[name] = {"B": B, "mode": mode, "t": timed(mode)}
        if B == 8192 and mode == R:
            raw[name]["alt"] = {
                nm: timed(R | fl) for nm, fl in (("one_us", rd.RD_VJP_FLAG_ONE_THREAD),
                                                 ("smem_us", rd.RD_VJP_FLAG_SHARED_STATE),
                                                 ("lanes_us", rd.RD_VJP_FLAG_LANES),
                                                 ("pair_us", rd.RD_VJP_FLAG_TWO_WARPS),
                                                 ("duo_us", rd.RD_VJP_FLAG_TWO_WARPS_SHARED))}
    return raw


def adjoint_report(raw, pk):
    """frac: the adjoint's work per link, the 621 flop (FMA = 2) of the
    store-mode kernel that re-derives nothing, over the FP32 peak; re-deriving
    the state (772 per link) or scanning across lanes costs more than that."""
    out = {}
    for name, r in raw.items():
        fpl = VJP_FLOP_PER_LINK[1]
        out[name] = {"us": r["t"] * 1e6, "frac": r["B"] * N_LINKS * fpl / r["t"] / pk.f32}
        for k, t in r.get("alt", {}).items():
            out[name][k] = t * 1e6
    out["flop_per_link"] = VJP_FLOP_PER_LINK[1]
    return out


def fd_section(torch, rd, chaingen, dev, dist, sampler, K):
    """Seconds per aba_batch call, FP32 data, B = 16384, n = 16 and 64: FP64
    inertia updates and solves (the workload's precision plan) and the
    library's double-float default."""
    raw = {}
    B = 16384
    for n in (16, 64):
        model = rd.Model(chaingen.make_chain(n, seed=chaingen.BASE_SEED))
        sets = []
        for r in range(4):
            st = chaingen.make_states(B, n, seed=6000 + r, kinds=("q", "qd", "tau"))
            sets.append([torch.from_numpy(st[k]).to(dev, torch.float32) for k in ("q", "qd", "tau")])
        nbytes = max(rd.aba_workspace_bytes(model, B, 0),
                     rd.aba_workspace_bytes(model, B, 0, rd.RD_ABA_FP64_UPDATE))
        ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        o = torch.empty_like(sets[0][0])
        steps = max(3, min(K, 50))

        def timed(flags):
            def call(k):
                x = sets[k % len(sets)]
                rd.aba(model, *x, workspace=ws, out=o, flags=flags)
            return time_calls(torch, call, steps, 3, dist, sampler) / steps

        raw[f"n{n}_B{B}"] = {"n": n, "B": B, "t64": timed(rd.RD_ABA_FP64_UPDATE), "tdf": timed(0)}
    # the four mappings across batch sizes: microseconds [thread per instance,
    # warp per instance (Sec. III-D scans), two warps per 32 instances, three
    # warps per 32 instances, AUTO]; double-float updates at n = 16 and 64, FP64
    # updates ("f64u") at n = 64
    xo = {}
    cases = [(n, Bx, 0) for n in (16, 64) for Bx in (256, 1024, 4096, 16384)]
    cases += [(64, Bx, rd.RD_ABA_FP64_UPDATE) for Bx in (256, 1024, 4096)]
    for n, Bx, prec in cases:
        model = rd.Model(chaingen.make_chain(n, seed=chaingen.BASE_SEED))
        st = chaingen.make_states(Bx, n, seed=6100, kinds=("q", "qd", "tau"))
        x = [torch.from_numpy(st[k]).to(dev, torch.float32) for k in ("q", "qd", "tau")]
        ws = torch.empty(rd.aba_workspace_bytes(model, Bx, 0, prec), dtype=torch.uint8,
                         device=dev)
        o = torch.empty_like(x[0])
        steps = max(3, min(K, 20))
        row = []
        for fl in (rd.RD_ABA_THREAD_PER_INSTANCE, rd.RD_ABA_WARP_PER_INSTANCE,
                   rd.RD_ABA_TWO_WARPS, rd.RD_ABA_THREE_WARPS, 0):
            t = time_calls(torch, lambda k: rd.aba(model, *x, workspace=ws, out=o, flags=fl | prec),
                           steps, 3, dist, sampler)
            row.append(t / steps * 1e6)
        xo[f"{'f64u_' if prec else ''}n{n}_B{Bx}"] = [short_us(t) for t in row]
    raw["crossover_us"] = xo
    return raw


def fd_report(raw, pk):
    """frac: the kernel's executed FP32 and FP64 arithmetic at the two peaks
    (combined time) over the measured time; frac_alg: the same with the
    formulation's count (the method's work: 720 FP32 + 800 FP64 flop per link);
    df_frac: FP32-pipe issue time of the double-float kernel's instructions."""
    out = {}
    for name, r in raw.items():
        if name == "crossover_us":
            out[name] = r
            continue
        nb = r["n"] * r["B"]
        t_exec = nb * (FD_EXEC_FLOP32_PER_LINK / pk.f32 + FD_EXEC_FLOP64_PER_LINK / pk.f64)
        t_alg = nb * (FD_FLOP32_PER_LINK / pk.f32 + FD_FLOP64_PER_LINK / pk.f64)
        t_df = nb * FD_DF_EXEC_FP32_INST_PER_LINK / pk.i32
        out[name] = {"us": r["t64"] * 1e6, "frac": t_exec / r["t64"],
                     "frac_alg": t_alg / r["t64"], "df_us": r["tdf"] * 1e6,
                     "df_frac": t_df / r["tdf"]}
    return out


def crossover_section(torch, rd, chaingen, dev, dist, sampler, K):
    """The inverse-dynamics workload's other sizes: n = 16 and 100 at the same
    batch (AUTO), and AUTO / the serial recursion / the 16-lane scan at n = 32
    across small batches (4 input sets rotated; small batches stay in L2, as
    they do in use)."""
    raw = {}

    def case(n, B, variant):
        model = rd.Model(chaingen.make_chain(n, seed=chaingen.BASE_SEED))
        sets = []
        for r in range(4):
            st = chaingen.make_states(B, n, seed=8000 + r)
            sets.append([torch.from_numpy(st[k]).to(dev, torch.float32) for k in ("q", "qd", "qdd")])
        o = torch.empty_like(sets[0][0])
        steps = max(3, min(K, 100))

        def call(k):
            rd.rnea(model, *sets[k % len(sets)], out=o, variant=variant)

        return time_calls(torch, call, steps, 3, dist, sampler) / steps

    for n in (16, 100):
        raw[f"n{n}_B{BATCH}"] = {"n": n, "t": case(n, BATCH, rd.RD_VARIANT_AUTO)}
    for B in (1024, 2048, 4096, 8192):
        raw[f"n{N_LINKS}_B{B}_us"] = [float(f"{case(N_LINKS, B, v) * 1e6:.3g}") for v in
                                      (rd.RD_VARIANT_AUTO, rd.RD_VARIANT_SERIAL_DH,
                                       rd.RD_VARIANT_SCAN(16))]
    return raw


def crossover_report(raw, pk):
    """n16/n100: algorithmic fraction of the FP32 peak; n32_B*_us: microseconds
    per call as [AUTO, serial, 16-lane scan]."""
    out = {}
    for name, r in raw.items():
        if isinstance(r, dict):
            out[name] = {"us": r["t"] * 1e6,
                         "frac": BATCH * r["n"] * ALGO_FLOP_PER_LINK / r["t"] / pk.f32}
        else:
            out[name] = r
    return out


def uneven_workload(rd, count=100000, seed=None):
    """The uneven-batch workload: `count` requests, each with its own robot
    (seed base + k), n uniform in 6..100, 20% forward dynamics, and its joint
    inputs (FP32; tau ~ N(0, 10) for forward, qdd ~ N(0, 2) for inverse
    dynamics). Returns (requests, fleet, plan, kinds, [q, qd, in2])."""
    import chaingen

    seed = chaingen.BASE_SEED if seed is None else seed
    reqs = chaingen.uneven_requests(count, n_lo=6, n_hi=100, fd_fraction=0.2, seed=seed)
    fleet = rd.Fleet([r["chain"] for r in reqs])
    kinds = np.array([1 if r["kind"] == "fd" else 0 for r in reqs], dtype=np.int32)
    plan = rd.Plan(fleet, np.arange(count, dtype=np.int32), kinds, dtype="float32")
    J = plan.total_joints
    rng = np.random.default_rng(77)
    fd_mask = np.repeat(kinds, plan.lengths) == 1
    in2 = np.where(fd_mask, rng.normal(0, 10, J), rng.normal(0, 2, J))
    host = [a.astype(np.float32) for a in (rng.uniform(-np.pi, np.pi, J), rng.normal(0, 1, J), in2)]
    return reqs, fleet, plan, kinds, host


def uneven_section(torch, rd, chaingen, dev, dist, sampler, K, count=100000):
    from paper_1609_04493_gb300 import autotune

    reqs, fleet, plan, kinds, host = uneven_workload(rd, count)
    x = [torch.from_numpy(a).to(dev) for a in host]
    o = torch.empty_like(x[0])
    f64 = rd.RD_FLEET_FP64_UPDATE
    (sched, tune), _ = autotune.tune_fleet(plan, *x, out=o, flags=f64)
    (sched_df, tune_df), _ = autotune.tune_fleet(plan, *x, out=o)
    steps = max(3, min(K, 20))
    raw = {"count": count, "joints": plan.total_joints, "groups": plan.groups,
           "fd_joints": int(np.sum(np.where(kinds == 1, plan.lengths, 0)))}
    for name, (sc, tu) in (("persistent", (sched | f64, tune)),
                           ("per_group", (rd.RD_SCHED_PER_GROUP | f64, 0)),
                           ("df_persistent", (sched_df, tune_df))):
        t = time_calls(torch, lambda k: rd.fleet_batch(plan, *x, out=o, schedule=sc, tune=tu),
                       steps, 3, dist, sampler)
        raw[name] = {"t": t / steps, "schedule": sc, "tune": tu}
    return raw


def uneven_report(raw, pk):
    """frac: inverse-dynamics links at the larger of their FP32 time (470 flop)
    and HBM time (128 B), plus forward-dynamics links at the combined time of
    the kernel's executed FP32 + FP64 flop (df: FP32-pipe issue time of the
    double-float instructions), over the measured time."""
    n_fd = raw["fd_joints"]
    n_id = raw["joints"] - n_fd
    t_id = n_id * max(ALGO_FLOP_PER_LINK / pk.f32, UNEVEN_ID_BYTES_PER_LINK / pk.hbm)
    t_fd = n_fd * (FD_EXEC_FLOP32_PER_LINK / pk.f32 + FD_EXEC_FLOP64_PER_LINK / pk.f64)
    t_df = n_fd * FD_DF_EXEC_FP32_INST_PER_LINK / pk.i32
    out = {}
    for name in ("persistent", "per_group", "df_persistent"):
        r = raw[name]
        floor = t_id + (t_df if name == "df_persistent" else t_fd)
        out[name] = {"us": r["t"] * 1e6, "value": raw["count"] / r["t"], "frac": floor / r["t"]}
    return out


def timed_graph(torch, g, dist, sampler):
    barrier(dist)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.time()
    e0.record()
    g.replay()
    e1.record()
    torch.cuda.synchronize()
    t1 = time.time()
    barrier(dist)
    if sampler is not None:
        sampler.region(t0, t1)
    return e0.elapsed_time(e1) / 1e3


def run_ours(args):
    import torch

    import chaingen
    import paper_1609_04493_gb300 as rd

    rank, world, local = dist_env()
    dist = init_dist(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rd.load()
    props = torch.cuda.get_device_properties(dev)
    sm_count = props.multi_processor_count
    uuid = getattr(props, "uuid", None)
    sampler = ClockSampler(f"GPU-{uuid}" if uuid is not None else None) if rank == 0 else None

    chain = chaingen.make_chain(N_LINKS, seed=chaingen.BASE_SEED)
    model = rd.Model(chain)
    K, W = args.steps, args.warmup

    # ---- FP32 headline
    sets32 = make_inputs(torch, dev, torch.float32, ROTATE, 1000 + 100 * rank)
    gw = capture(torch, rd, model, sets32, max(W, 1))
    gw.replay()
    torch.cuda.synchronize()
    g32 = capture(torch, rd, model, sets32, K)
    t32 = max_over_ranks(dist, timed_graph(torch, g32, dist, sampler))
    value = world * BATCH * K / t32
    kern_id, kern_block, kern_stored = rd.rnea_last_config()
    kern_reg, kern_ring = rd.rnea_last_state_layout()
    del g32, gw

    raw = {}
    if not args.quick:
        # ---- FP64 on the same GPU, IEEE FP64 and double-float arithmetic
        K64 = max(3, min(K, 200))
        sets64 = make_inputs(torch, dev, torch.float64, 4, 2000 + 100 * rank)
        t64 = {}
        for name, v in (("fp64", rd.RD_VARIANT_AUTO), ("df", rd.RD_VARIANT_SERIAL_DF)):
            gw64 = capture(torch, rd, model, sets64, 3, variant=v)
            gw64.replay()
            torch.cuda.synchronize()
            g64 = capture(torch, rd, model, sets64, K64, variant=v)
            t64[name] = max_over_ranks(dist, timed_graph(torch, g64, dist, sampler)) / K64
            del g64, gw64
        x0 = sets64[0]
        ref64 = rd.rnea(model, x0["q"], x0["qd"], x0["qdd"])
        got = rd.rnea(model, x0["q"], x0["qd"], x0["qdd"], variant=rd.RD_VARIANT_SERIAL_DF)
        scale = ref64.abs().amax(dim=1).clamp_min(1e-300)
        t64["df_diff"] = float(((got - ref64).abs().amax(dim=1) / scale).max())
        raw["fp64"] = t64
        del sets64

        # ---- end to end through the host-array entry point: two sets of
        # pinned host inputs alternate, so no step reads the previous one's
        hosts = []
        for r in range(2):
            st = chaingen.make_states(BATCH, N_LINKS, seed=3000 + 10 * rank + r)
            hosts.append(([torch.from_numpy(st[k].astype(np.float32)).pin_memory()
                           for k in ("q", "qd", "qdd")],
                          torch.empty((BATCH, N_LINKS), dtype=torch.float32).pin_memory()))
        Ke = max(4, min(K, 200))
        e2e = {}
        for name, v in (("inplace", rd.RD_VARIANT_AUTO), ("staged", rd.RD_FLAG_HOST_COPY)):
            for k in range(3):
                rd.rnea_host(model, *hosts[k % 2][0], out=hosts[k % 2][1], variant=v)
            barrier(dist)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for k in range(Ke):
                rd.rnea_host(model, *hosts[k % 2][0], out=hosts[k % 2][1], variant=v)
            te = max_over_ranks(dist, time.perf_counter() - t0)
            barrier(dist)
            if sampler is not None:
                sampler.region(t0, t0 + te)
            e2e[name] = te / Ke
        raw["e2e"] = e2e
        raw["e2e_steps"] = Ke

        raw["adjoint"] = adjoint_section(torch, rd, chaingen, model, dev, dist, sampler, K)
        raw["forward_dynamics"] = fd_section(torch, rd, chaingen, dev, dist, sampler, K)
        raw["crossover"] = crossover_section(torch, rd, chaingen, dev, dist, sampler, K)
        if not args.no_uneven:
            raw["uneven"] = uneven_section(torch, rd, chaingen, dev, dist, sampler, K)

    clocks = sampler.stop() if sampler is not None else None
    mhz = (clocks or {}).get("sm_mhz") or SM_MAX_MHZ
    pk = Peaks(sm_count, mhz)

    res = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
           "warmup": W, "ms_per_step": t32 / K * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n_links": N_LINKS, "batch": BATCH,
                      "global_batch": BATCH * world, "parallelism": f"replicas{world}",
                      "l2": f"{ROTATE} rotating input sets "
                            f"({ROTATE * BATCH * N_LINKS * 16 / 1e6:.0f} MB) > L2",
                      "seed": chaingen.BASE_SEED},
           "gpu_launches": K}

    # roofline of the dominant kernel (one FP32 RNEA launch per step)
    if kern_id == rd.RD_RNEA_KERNEL_DH_PARAM:
        kname = f"rnea_dhp_kernel<float,{kern_block}>,K={kern_stored},R={kern_reg},S={kern_ring}"
        exec_fpl = dh_param_flops(N_LINKS, kern_stored) / N_LINKS
    else:
        kname = f"rnea family {kern_id:#x},{kern_block}"
        exec_fpl = JOINT_FRAME_FLOP_PER_LINK
    avg_launch = t32 / K
    achieved = ALGO_FLOP_PER_LINK * N_LINKS * BATCH / avg_launch / 1e12
    executed = exec_fpl * N_LINKS * BATCH / avg_launch / 1e12
    peak = pk.f32 / 1e12
    res["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                       "frac": achieved / peak,
                       "traffic": recorded_traffic("rnea_fp32_n32_B65536"),
                       "kernel": kname, "avg_launch_us": avg_launch * 1e6,
                       "flop_per_link": ALGO_FLOP_PER_LINK,
                       "executed_flop_per_link": exec_fpl, "executed_frac": executed / peak,
                       "peak_src": f"{sm_count}SMx128x2x{mhz:.0f}MHz",
                       "hbm_frac": BATCH * N_LINKS * 16 / avg_launch / pk.hbm}
    if clocks is not None:
        res["clocks"] = {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons", "samples")}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(target_s=10.0)
    if "e2e" in raw:
        # (timed over raw["e2e_steps"] steps, two pinned host input sets alternating)
        te = raw["e2e"]
        res["e2e"] = {"value": world * BATCH / te["inplace"], "unit": UNIT,
                      "h2d_bytes_per_step": 3 * BATCH * N_LINKS * 4,
                      "d2h_bytes_per_step": BATCH * N_LINKS * 4,
                      "link_gbs": 4 * BATCH * N_LINKS * 4 / te["inplace"] / 1e9,
                      "staged_value": world * BATCH / te["staged"]}
    if "crossover" in raw:
        res["crossover"] = crossover_report(raw["crossover"], pk)
    if "uneven" in raw:
        res["uneven"] = uneven_report(raw["uneven"], pk)
    if "fp64" in raw:
        t = raw["fp64"]
        nb = N_LINKS * BATCH
        res["fp64"] = {"us": t["fp64"] * 1e6, "value": world * BATCH / t["fp64"],
                       "frac": nb * JOINT_FRAME_FLOP_PER_LINK / t["fp64"] / pk.f64,
                       "df_us": t["df"] * 1e6, "df_value": world * BATCH / t["df"],
                       "df_frac": nb * RNEA_DF_EXEC_FP32_INST_PER_LINK / pk.i32 / t["df"],
                       "df_diff": t["df_diff"]}
    if "forward_dynamics" in raw:
        res["forward_dynamics"] = fd_report(raw["forward_dynamics"], pk)
    if "adjoint" in raw:
        res["adjoint"] = adjoint_report(raw["adjoint"], pk)
    if dist is not None:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(rnd(res)), flush=True)


# -------------------------------------------------------- CPU (oracle) arm

def _cpu_threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(target_s=10.0, threads=None):
    """The FP64 oracle, as it stands, on the host cores: a bounded sample of the
    headline workload (same chain, fresh states, the batch split over
    threads), evaluated in passes until about `target_s` seconds of work."""
    import chaingen
    import oracle

    threads = threads or _cpu_threads()
    chain = chaingen.make_chain(N_LINKS, seed=chaingen.BASE_SEED)
    st = chaingen.make_states(BATCH, N_LINKS, seed=4343)
    passes, t0 = 0, time.perf_counter()
    while True:
        oracle.rnea_threaded(chain, st["q"], st["qd"], st["qdd"], threads=threads)
        passes += 1
        dt = time.perf_counter() - t0
        if dt >= target_s:
            break
    return {"value": passes * BATCH / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{passes}x{BATCH} states n=32, FP64 oracle, {threads} threads, {dt:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import chaingen
    import oracle

    threads = _cpu_threads()
    chain = chaingen.make_chain(N_LINKS, seed=chaingen.BASE_SEED)
    probe = chaingen.make_states(256 * threads, N_LINKS, seed=4242)
    t0 = time.perf_counter()
    oracle.rnea_threaded(chain, probe["q"], probe["qd"], probe["qdd"], threads=threads)
    rate = 256 * threads / max(time.perf_counter() - t0, 1e-6)
    total_budget = 90.0
    per_step = int(max(64, min(BATCH, rate * total_budget / (args.steps + args.warmup))))
    st = chaingen.make_states(per_step, N_LINKS, seed=4343)
    for _ in range(args.warmup):
        oracle.rnea_threaded(chain, st["q"], st["qd"], st["qdd"], threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.rnea_threaded(chain, st["q"], st["qd"], st["qdd"], threads=threads)
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    sample = (f"{per_step} of the {BATCH} states per step, n=32 chain, FP64 oracle on "
              f"{threads} host threads")
    res = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "n_links": N_LINKS, "batch": BATCH,
                      "global_batch": BATCH * world, "parallelism": f"replicas{world}",
                      "seed": chaingen.BASE_SEED},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res), flush=True)


def run_kernel_only(args):
    """Small profiling cases for ncu: W + K plain launches of one kernel, no graph."""
    import torch

    import chaingen
    import paper_1609_04493_gb300 as rd

    rd.load()
    dev = torch.device("cuda", 0)
    calls = args.warmup + args.steps
    if args.kernel_only in ("f32", "f64", "f64df"):
        dt = torch.float32 if args.kernel_only == "f32" else torch.float64
        v = rd.RD_VARIANT_SERIAL_DF if args.kernel_only == "f64df" else rd.RD_VARIANT_AUTO
        model = rd.Model(chaingen.make_chain(N_LINKS, seed=chaingen.BASE_SEED))
        x = make_inputs(torch, dev, dt, 1, 1000)[0]
        for _ in range(calls):
            rd.rnea(model, x["q"], x["qd"], x["qdd"], out=x["tau"], variant=v)
        res = x["tau"]
    elif args.kernel_only == "host":
        model = rd.Model(chaingen.make_chain(N_LINKS, seed=chaingen.BASE_SEED))
        st = chaingen.make_states(BATCH, N_LINKS, seed=3000)
        host = [torch.from_numpy(st[k].astype(np.float32)).pin_memory() for k in ("q", "qd", "qdd")]
        res = torch.empty_like(host[0]).pin_memory()
        for _ in range(calls):
            rd.rnea_host(model, *host, out=res)
    elif args.kernel_only in ("vjp", "vjplane", "vjppair", "vjpsmem"):
        lanes = args.kernel_only == "vjplane"
        Bv = 4096 if lanes else 8192
        mode = rd.RD_VJP_RECOMPUTE | {"vjp": rd.RD_VJP_FLAG_ONE_THREAD,
                                      "vjplane": rd.RD_VJP_FLAG_LANES,
                                      "vjppair": rd.RD_VJP_FLAG_TWO_WARPS,
                                      "vjpsmem": rd.RD_VJP_FLAG_SHARED_STATE}[args.kernel_only]
        model = rd.Model(chaingen.make_chain(N_LINKS, seed=chaingen.BASE_SEED))
        st = chaingen.make_states(Bv, N_LINKS, seed=5000, kinds=("q", "qd", "qdd", "w"))
        x = [torch.from_numpy(st[k]).to(dev, torch.float32) for k in ("q", "qd", "qdd", "w")]
        for _ in range(calls):
            res = rd.rnea_vjp(model, *x, mode=mode)[0]
    elif args.kernel_only in ("aba", "aba64", "abawarp", "abapair", "abatri", "abatri1k"):
        flags = {"aba": rd.RD_ABA_THREAD_PER_INSTANCE,
                 "aba64": rd.RD_ABA_FP64_UPDATE | rd.RD_ABA_THREAD_PER_INSTANCE,
                 "abawarp": rd.RD_ABA_WARP_PER_INSTANCE,
                 "abapair": rd.RD_ABA_TWO_WARPS,
                 "abatri": rd.RD_ABA_THREE_WARPS,
                 "abatri1k": rd.RD_ABA_THREE_WARPS}[args.kernel_only]
        Ba = 1024 if args.kernel_only in ("abawarp", "abatri1k") else 16384
        model = rd.Model(chaingen.make_chain(64, seed=chaingen.BASE_SEED))
        st = chaingen.make_states(Ba, 64, seed=6000, kinds=("q", "qd", "tau"))
        x = [torch.from_numpy(st[k]).to(dev, torch.float32) for k in ("q", "qd", "tau")]
        ws = torch.empty(rd.aba_workspace_bytes(model, Ba, 0, flags), dtype=torch.uint8,
                         device=dev)
        for _ in range(calls):
            res = rd.aba(model, *x, workspace=ws, flags=flags)
    else:
        count = 20000
        reqs = chaingen.uneven_requests(count, 6, 100, 0.2, seed=chaingen.BASE_SEED)
        fleet = rd.Fleet([r["chain"] for r in reqs])
        kinds = np.array([1 if r["kind"] == "fd" else 0 for r in reqs], dtype=np.int32)
        plan = rd.Plan(fleet, np.arange(count, dtype=np.int32), kinds, "float32")
        rng = np.random.default_rng(77)
        J = plan.total_joints
        x = [torch.from_numpy(a.astype(np.float32)).to(dev)
             for a in (rng.uniform(-np.pi, np.pi, J), rng.normal(0, 1, J), rng.normal(0, 5, J))]
        sched, tune = {"fleet": (0, rd.RD_FLEET_TUNE(7, 1)),
                       "fleetpair": (0, rd.RD_FLEET_TUNE(7, 2) | rd.RD_FLEET_TWO_WARPS(65)),
                       "fleettri64": (rd.RD_FLEET_FP64_UPDATE,
                                      rd.RD_FLEET_TUNE(7, 2) | rd.RD_FLEET_THREE_WARPS(65)),
                       }[args.kernel_only]
        for _ in range(calls):
            res = rd.fleet_batch(plan, *x, schedule=sched, tune=tune)
    torch.cuda.synchronize()
    print(f"kernel-only {args.kernel_only}: {calls} launches, max|out| = "
          f"{float(res.abs().max()):.4g}")


def main():
    args = parse_args()
    if args.kernel_only:
        run_kernel_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
