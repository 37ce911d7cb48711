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
SM_COUNT = 152
FP32_LANES_PER_SM = 128
FP64_NOMINAL_TFLOPS = 1.25


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
                   choices=["f32", "f64", "f64df", "host", "vjp", "aba", "aba64", "fleet"],
                   default=None,
                   help="profiling case: W + K plain launches of one kernel, no JSON "
                        "(f32/f64: RNEA n=32 B=65536; f64df: the same FP64 data in double-float "
                        "arithmetic; host: rnea_batch_host on pinned FP32 arrays, the same "
                        "size; vjp: adjoint n=32 B=8192; "
                        "aba: forward dynamics n=64 B=16384 (double-float updates; aba64: "
                        "FP64 updates); fleet: 20000 mixed requests)")
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


def fp32_peak_tflops():
    return SM_COUNT * FP32_LANES_PER_SM * 2 * 2.070e9 / 1e12


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


def adjoint_section(torch, rd, chaingen, model, dev, dist, sampler, K):
    out = {}
    for B, mode in ((8192, rd.RD_VJP_RECOMPUTE), (262144, rd.RD_VJP_RECOMPUTE),
                    (8192, rd.RD_VJP_STORE)):
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

        def call(k):
            x, o = sets[k % len(sets)]
            rd.rnea_vjp(model, *x, mode=mode, workspace=ws, out=o)

        t = time_calls(torch, call, steps, 3, dist, sampler)
        name = f"B{B}_{'store' if mode == rd.RD_VJP_STORE else 'recompute'}"
        fpl = VJP_FLOP_PER_LINK[mode]
        tf = B * N_LINKS * VJP_ALGO_FLOP_PER_LINK / (t / steps) / 1e12
        tx = B * N_LINKS * fpl / (t / steps) / 1e12
        peak32 = SM_COUNT * FP32_LANES_PER_SM * 2 * 2.070e9 / 1e12
        out[name] = {"value": B * steps / t, "unit": UNIT, "ms_per_step": t / steps * 1e3,
                     "steps": steps, "flop_per_link": fpl, "achieved_tflops": tx,
                     "frac_of_fp32_peak": tx / peak32,
                     "algorithmic_flop_per_link": VJP_ALGO_FLOP_PER_LINK,
                     "algorithmic_tflops": tf, "algorithmic_frac_of_fp32_peak": tf / peak32}
        if B == 8192 and mode == rd.RD_VJP_RECOMPUTE:
            # each instance split between two warps (RD_VJP_FLAG_TWO_WARPS)
            def call2(k):
                x, o = sets[k % len(sets)]
                rd.rnea_vjp(model, *x, mode=mode | rd.RD_VJP_FLAG_TWO_WARPS, out=o)

            t2 = time_calls(torch, call2, steps, 3, dist, sampler)
            out[name]["two_warps"] = {"value": B * steps / t2, "ms_per_step": t2 / steps * 1e3}
    out["metric"] = "RNEA adjoint d(w^T tau)/d(q, qd, qdd) evals/s, n=32 FP32"
    return out


def fd_section(torch, rd, chaingen, dev, dist, sampler, K):
    out = {}
    B = 16384
    for n in (16, 64):
        model = rd.Model(chaingen.make_chain(n, seed=chaingen.BASE_SEED))
        sets = []
        for r in range(4):
            st = chaingen.make_states(B, n, seed=6000 + r, kinds=("q", "qd", "tau"))
            sets.append([torch.from_numpy(st[k]).to(dev, torch.float32) for k in ("q", "qd", "tau")])
        ws = torch.empty(rd.aba_workspace_bytes(model, B, 0), dtype=torch.uint8, device=dev)
        o = torch.empty_like(sets[0][0])
        steps = max(3, min(K, 50))
        inst_rate = SM_COUNT * FP32_LANES_PER_SM * 2.070e9  # FP32-pipe thread instructions/s

        def timed(flags):
            def call(k):
                x = sets[k % len(sets)]
                rd.aba(model, *x, workspace=ws, out=o, flags=flags)
            return time_calls(torch, call, steps, 3, dist, sampler)

        t64 = timed(rd.RD_ABA_FP64_UPDATE)
        tdf = timed(0)
        t_exec64 = B * n * (FD_EXEC_FLOP32_PER_LINK / (fp32_peak_tflops() * 1e12)
                            + FD_EXEC_FLOP64_PER_LINK / (FP64_NOMINAL_TFLOPS * 1e12))
        t_floor = B * n * FD_EXEC_FLOP64_PER_LINK / (FP64_NOMINAL_TFLOPS * 1e12)
        t_exec = B * n * FD_DF_EXEC_FP32_INST_PER_LINK / inst_rate
        out[f"n{n}_B{B}"] = {"value": B * steps / t64, "unit": UNIT,
                             "ms_per_step": t64 / steps * 1e3, "steps": steps,
                             "roofline_ms": t_exec64 * 1e3,
                             "roofline_frac": t_exec64 / (t64 / steps),
                             "fp64_pipe_floor_ms": t_floor * 1e3,
                             "double_float": {"value": B * steps / tdf,
                                              "ms_per_step": tdf / steps * 1e3,
                                              "roofline_ms": t_exec * 1e3,
                                              "roofline_frac": t_exec / (tdf / steps)}}
    out["algorithmic_flop_per_link"] = {"fp32": FD_FLOP32_PER_LINK,
                                         "extended_precision": FD_FLOP64_PER_LINK}
    out["metric"] = ("forward dynamics (articulated-body, FP32 data, FP64 inertia updates and "
                     "solves as the workload specifies; beside it the library's default, the "
                     "same in double-float arithmetic) evals/s")
    out["roofline"] = (f"FP64 updates: combined FP32 + FP64 time of the kernel's "
                       f"{FD_EXEC_FLOP32_PER_LINK} FP32 and {FD_EXEC_FLOP64_PER_LINK} FP64 flop "
                       f"per link at the derived FP32 and nominal FP64 peaks, divided by the "
                       f"measured time; fp64_pipe_floor_ms: the FP64 part alone; double_float: "
                       f"FP32-pipe issue time of its {FD_DF_EXEC_FP32_INST_PER_LINK} FP32 "
                       f"instructions per link at {SM_COUNT} x {FP32_LANES_PER_SM} lanes x "
                       f"2.07 GHz")
    return out


def crossover_section(torch, rd, chaingen, dev, dist, sampler, K):
    """The inverse-dynamics workload's other sizes: n = 16 and 100 at the same
    batch (AUTO), and the lane-parallel scan against the serial recursion at
    n = 32 across small batches."""
    out = {}

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

        t = time_calls(torch, call, steps, 3, dist, sampler)
        return t / steps, rd.rnea_last_config()

    for n in (16, 100):
        t, fam = case(n, BATCH, rd.RD_VARIANT_AUTO)
        out[f"n{n}_B{BATCH}"] = {
            "value": BATCH / t, "unit": UNIT, "ms_per_step": t * 1e3, "kernel_family": fam[0],
            "stored_links": fam[2],
            "algorithmic_frac_of_fp32_peak":
                BATCH * n * ALGO_FLOP_PER_LINK / t / (fp32_peak_tflops() * 1e12)}
    for B in (1024, 2048, 4096, 8192):
        row = {}
        for name, v in (("auto", rd.RD_VARIANT_AUTO), ("serial", rd.RD_VARIANT_SERIAL_DH),
                        ("scan16", rd.RD_VARIANT_SCAN(16))):
            t, fam = case(N_LINKS, B, v)
            row[name] = t * 1e6
            if name == "auto":
                row["auto_kernel_family"] = fam[0]
        out[f"n{N_LINKS}_B{B}_us"] = row
    out["metric"] = ("RNEA FP32: evals/s at n = 16 and 100 (B = 65536, AUTO); microseconds per "
                     "call at n = 32 for small B: AUTO, the serial common-normal recursion and the "
                     "16-lane scan")
    out["inputs"] = "4 input sets rotated; the small batches are L2-resident, as they are in use"
    return out


def uneven_section(torch, rd, chaingen, dev, dist, sampler, K, count=100000):
    from paper_1609_04493_gb300 import autotune

    reqs = chaingen.uneven_requests(count, n_lo=6, n_hi=100, fd_fraction=0.2, seed=chaingen.BASE_SEED)
    fleet = rd.Fleet([r["chain"] for r in reqs])
    kinds = np.array([1 if r["kind"] == "fd" else 0 for r in reqs], dtype=np.int32)
    plan = rd.Plan(fleet, np.arange(count, dtype=np.int32), kinds, dtype="float32")
    J = plan.total_joints
    rng = np.random.default_rng(77)
    fd_mask = np.repeat(kinds, plan.lengths) == 1
    in2 = np.where(fd_mask, rng.normal(0, 10, J), rng.normal(0, 2, J))
    x = [torch.from_numpy(a.astype(np.float32)).to(dev)
         for a in (rng.uniform(-np.pi, np.pi, J), rng.normal(0, 1, J), in2)]
    o = torch.empty_like(x[0])
    f64 = rd.RD_FLEET_FP64_UPDATE
    (sched, tune), _ = autotune.tune_fleet(plan, *x, out=o, flags=f64)
    (sched_df, tune_df), _ = autotune.tune_fleet(plan, *x, out=o)
    steps = max(3, min(K, 20))
    res = {}
    for name, (sc, tu) in (("persistent_tuned", (sched | f64, tune)),
                           ("per_group_launches", (rd.RD_SCHED_PER_GROUP | f64, 0)),
                           ("double_float_persistent_tuned", (sched_df, tune_df))):
        t = time_calls(torch, lambda k: rd.fleet_batch(plan, *x, out=o, schedule=sc, tune=tu),
                       steps, 3, dist, sampler)
        res[name] = {"value": count * steps / t, "unit": "requests/s",
                     "ms_per_step": t / steps * 1e3, "steps": steps,
                     "schedule": sc, "tune": tu}
    n_fd = int(np.sum(np.where(kinds == 1, plan.lengths, 0)))
    n_id = J - n_fd
    t_id = n_id * max(ALGO_FLOP_PER_LINK / (fp32_peak_tflops() * 1e12),
                      UNEVEN_ID_BYTES_PER_LINK / (measured_peaks().get("hbm_gbs", 6800.0) * 1e9))
    t_alg = t_id + n_fd * (FD_EXEC_FLOP32_PER_LINK / (fp32_peak_tflops() * 1e12)
                           + FD_EXEC_FLOP64_PER_LINK / (FP64_NOMINAL_TFLOPS * 1e12))
    t_alg_df = t_id + n_fd * FD_DF_EXEC_FP32_INST_PER_LINK / (SM_COUNT * FP32_LANES_PER_SM * 2.070e9)
    for name in ("persistent_tuned", "per_group_launches"):
        res[name]["roofline_frac"] = t_alg / (res[name]["ms_per_step"] * 1e-3)
    res["double_float_persistent_tuned"]["roofline_frac"] = t_alg_df / (
        res["double_float_persistent_tuned"]["ms_per_step"] * 1e-3)
    res["roofline_ms"] = t_alg * 1e3
    res["roofline"] = (f"inverse dynamics links at the larger of {ALGO_FLOP_PER_LINK} flop / FP32 "
                       f"peak and {UNEVEN_ID_BYTES_PER_LINK} B (joint values, torque, streamed "
                       f"constants) / measured HBM bandwidth, plus forward dynamics links at the "
                       f"combined FP32 + FP64 time of {FD_EXEC_FLOP32_PER_LINK} FP32 and "
                       f"{FD_EXEC_FLOP64_PER_LINK} FP64 flop per link (double-float line: the "
                       f"FP32-pipe issue time of {FD_DF_EXEC_FP32_INST_PER_LINK} instructions "
                       f"per link); divided by the measured time")
    res["workload"] = (f"{count} requests, own robot each, n uniform in 6..100 "
                       f"({J} joints), {int(kinds.sum())} forward / {count - int(kinds.sum())} "
                       f"inverse dynamics, FP32 with FP64 inertia updates and solves (the "
                       f"double-float line: the library's default)")
    res["launches_per_group_schedule"] = plan.groups
    return res


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
    ms_step = t32 / K * 1e3

    res = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
           "warmup": W, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n_links": N_LINKS, "batch": BATCH,
                      "global_batch": BATCH * world, "parallelism": f"replicas{world}",
                      "l2": f"{ROTATE} rotating input sets "
                            f"({ROTATE * BATCH * N_LINKS * 16 / 1e6:.0f} MB) > L2",
                      "seed": chaingen.BASE_SEED},
           "gpu_launches": K}

    # roofline of the dominant kernel (the FP32 RNEA kernel: one launch per step)
    kern_id, kern_block, kern_stored = rd.rnea_last_config()
    if kern_id == rd.RD_RNEA_KERNEL_DH_PARAM:
        kname = (f"rnea_dhp_kernel<float, {kern_block} threads>, common-normal frames, "
                 f"constants as a kernel parameter, full state for {kern_stored} of "
                 f"{N_LINKS} links, polynomial sin/cos")
        exec_fpl = dh_param_flops(N_LINKS, kern_stored) / N_LINKS
    else:
        kname = f"rnea kernel family {kern_id:#x}, {kern_block} threads"
        exec_fpl = JOINT_FRAME_FLOP_PER_LINK
    avg_launch = t32 / K
    peak32 = SM_COUNT * FP32_LANES_PER_SM * 2 * 2.070e9 / 1e12
    achieved = ALGO_FLOP_PER_LINK * N_LINKS * BATCH / avg_launch / 1e12
    executed = exec_fpl * N_LINKS * BATCH / avg_launch / 1e12
    traffic = recorded_traffic("rnea_fp32_n32_B65536")
    try:
        fma32 = rd.measure_fma_peak("float32")
        fma64 = rd.measure_fma_peak("float64")
    except Exception:  # diagnostic only
        fma32 = fma64 = None
    res["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak32, "unit": "TFLOP/s",
                       "frac": achieved / peak32, "traffic": traffic,
                       "kernel": kname, "avg_launch_us": avg_launch * 1e6,
                       "flop_per_link": ALGO_FLOP_PER_LINK,
                       "flop_count": "algorithmic: the recursion of Sec. II-A with general link "
                                     "transforms (Rodrigues exponential and 3x4 compose), FMA = 2",
                       "executed_flop_per_link": exec_fpl,
                       "executed_tflops": executed, "executed_frac": executed / peak32,
                       "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                       "measured_fma_tflops": {"fp32": fma32, "fp64": fma64},
                       "hbm": {"algorithmic_bytes_per_launch": BATCH * N_LINKS * 16,
                               "achieved_gbs": BATCH * N_LINKS * 16 / avg_launch / 1e9,
                               "peak_gbs": measured_peaks().get("hbm_gbs", 6800.0),
                               "peak_source": "MEASURED_PEAKS.json hbm_gbs"}}

    if not args.quick:
        # ---- FP64 on the same GPU
        K64 = max(3, min(K, 200))
        del g32, gw
        sets64 = make_inputs(torch, dev, torch.float64, 4, 2000 + 100 * rank)
        gw64 = capture(torch, rd, model, sets64, 3)
        gw64.replay()
        torch.cuda.synchronize()
        g64 = capture(torch, rd, model, sets64, K64)
        t64 = max_over_ranks(dist, timed_graph(torch, g64, dist, sampler))
        k64 = rd.rnea_last_config()
        fp64_flops = ALGO_FLOP_PER_LINK * N_LINKS * BATCH / (t64 / K64) / 1e12
        fp64_exec = JOINT_FRAME_FLOP_PER_LINK * N_LINKS * BATCH / (t64 / K64) / 1e12
        res["fp64"] = {"value": world * BATCH * K64 / t64, "unit": UNIT, "steps": K64,
                       "ms_per_step": t64 / K64 * 1e3, "kernel_family": k64[0],
                       "flop_per_link": JOINT_FRAME_FLOP_PER_LINK,
                       "achieved_tflops": fp64_exec, "peak_tflops_nominal": FP64_NOMINAL_TFLOPS,
                       "frac_of_nominal": fp64_exec / FP64_NOMINAL_TFLOPS,
                       "frac_of_measured_fma": (fp64_exec / fma64) if fma64 else None,
                       "algorithmic_tflops": fp64_flops,
                       "algorithmic_frac_of_nominal": fp64_flops / FP64_NOMINAL_TFLOPS,
                       "fp32_over_fp64": value / (world * BATCH * K64 / t64)}
        # the same FP64 data in double-float arithmetic on the FP32 pipe
        vdf = rd.RD_VARIANT_SERIAL_DF
        gwdf = capture(torch, rd, model, sets64, 3, variant=vdf)
        gwdf.replay()
        torch.cuda.synchronize()
        gdf = capture(torch, rd, model, sets64, K64, variant=vdf)
        tdf = max_over_ranks(dist, timed_graph(torch, gdf, dist, sampler))
        x0 = sets64[0]
        ref64 = rd.rnea(model, x0["q"], x0["qd"], x0["qdd"])
        got = rd.rnea(model, x0["q"], x0["qd"], x0["qdd"], variant=vdf)
        scale = ref64.abs().amax(dim=1).clamp_min(1e-300)
        diff = float(((got - ref64).abs().amax(dim=1) / scale).max())
        t_issue = N_LINKS * BATCH * RNEA_DF_EXEC_FP32_INST_PER_LINK / (
            SM_COUNT * FP32_LANES_PER_SM * 2.070e9)
        t_floor = N_LINKS * BATCH * JOINT_FRAME_FLOP_PER_LINK / (FP64_NOMINAL_TFLOPS * 1e12)
        res["fp64"]["double_float"] = {
            "value": world * BATCH * K64 / tdf, "unit": UNIT, "steps": K64,
            "ms_per_step": tdf / K64 * 1e3, "variant": "RD_VARIANT_SERIAL_DF",
            "fp32_inst_per_link": RNEA_DF_EXEC_FP32_INST_PER_LINK,
            "roofline_ms": t_issue * 1e3, "roofline_frac": t_issue / (tdf / K64),
            "fp64_pipe_floor_ms": t_floor * 1e3,
            "max_rel_diff_vs_fp64": diff,
            "roofline": ("FP32-pipe issue time of the kernel's FP32 instructions per link at "
                         f"{SM_COUNT} x {FP32_LANES_PER_SM} lanes x 2.07 GHz over the measured "
                         "time; fp64_pipe_floor_ms: the FP64 kernel's executed "
                         f"{JOINT_FRAME_FLOP_PER_LINK} flop per link at the nominal FP64 peak")}
        del g64, gw64, gdf, gwdf, sets64

        # ---- end to end through the host-array entry point
        st = chaingen.make_states(BATCH, N_LINKS, seed=3000 + rank)
        host = [torch.from_numpy(st[k].astype(np.float32)).pin_memory() for k in ("q", "qd", "qdd")]
        out = torch.empty_like(host[0]).pin_memory()
        for _ in range(3):
            rd.rnea_host(model, *host, out=out)
        Ke = max(3, min(K, 200))
        barrier(dist)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(Ke):
            rd.rnea_host(model, *host, out=out)
        te = max_over_ranks(dist, time.perf_counter() - t0)
        barrier(dist)
        if sampler is not None:
            sampler.region(t0, t0 + te)
        res["e2e"] = {"value": world * BATCH * Ke / te, "unit": UNIT, "steps": Ke,
                      "h2d_bytes_per_step": 3 * BATCH * N_LINKS * 4,
                      "d2h_bytes_per_step": BATCH * N_LINKS * 4,
                      "api": "rnea_batch_host, pinned host arrays, FP32: the kernel reads "
                             "the rows from host memory and writes tau back itself (16-byte "
                             "slab transfers; RD_RNEA_KERNEL_DH_HOST)"}
        # the staged path on the same arrays: copy engines, row chunks pipelined
        # over three streams
        for _ in range(3):
            rd.rnea_host(model, *host, out=out, variant=rd.RD_FLAG_HOST_COPY)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(Ke):
            rd.rnea_host(model, *host, out=out, variant=rd.RD_FLAG_HOST_COPY)
        ts = max_over_ranks(dist, time.perf_counter() - t0)
        res["e2e"]["staged_copies"] = {"value": world * BATCH * Ke / ts, "unit": UNIT,
                                       "ms_per_step": ts / Ke * 1e3}
        link_bytes = 4 * BATCH * N_LINKS * 4
        res["e2e"]["link_gbs"] = link_bytes / (te / Ke) / 1e9

        # ---- adjoint (rnea_vjp), n = 32 FP32
        res["adjoint"] = adjoint_section(torch, rd, chaingen, model, dev, dist, sampler, K)
        # ---- forward dynamics (aba_batch), n = 16 and 64, B = 16384 FP32
        res["forward_dynamics"] = fd_section(torch, rd, chaingen, dev, dist, sampler, K)
        # ---- the inverse-dynamics workload's other sizes and the scan / serial crossover
        res["crossover"] = crossover_section(torch, rd, chaingen, dev, dist, sampler, K)
        # ---- uneven batching: 100000 mixed requests (fleet_batch)
        if not args.no_uneven:
            res["uneven"] = uneven_section(torch, rd, chaingen, dev, dist, sampler, K)

    if sampler is not None:
        res["clocks"] = sampler.stop()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(target_s=10.0)
    if dist is not None:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(res), flush=True)


# -------------------------------------------------------- CPU (oracle) arm

def _cpu_threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(target_s=10.0, threads=None):
    """The FP64 oracle, as it stands, on the host cores: a bounded sample of the
    headline workload (same chain, fresh states), batch split over threads."""
    import chaingen
    import oracle

    threads = threads or _cpu_threads()
    chain = chaingen.make_chain(N_LINKS, seed=chaingen.BASE_SEED)
    probe = chaingen.make_states(256 * threads, N_LINKS, seed=4242)
    t0 = time.perf_counter()
    oracle.rnea_threaded(chain, probe["q"], probe["qd"], probe["qdd"], threads=threads)
    rate = 256 * threads / max(time.perf_counter() - t0, 1e-6)
    sample = int(min(max(rate * target_s / threads, 1024), 4 * BATCH))
    st = chaingen.make_states(sample, N_LINKS, seed=4343)
    t0 = time.perf_counter()
    oracle.rnea_threaded(chain, st["q"], st["qd"], st["qdd"], threads=threads)
    dt = time.perf_counter() - t0
    return {"value": sample / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{sample} states of the n=32 chain (FP64 oracle, {threads} threads, "
                      f"{dt:.1f} s)"}


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
    elif args.kernel_only == "vjp":
        model = rd.Model(chaingen.make_chain(N_LINKS, seed=chaingen.BASE_SEED))
        st = chaingen.make_states(8192, N_LINKS, seed=5000, kinds=("q", "qd", "qdd", "w"))
        x = [torch.from_numpy(st[k]).to(dev, torch.float32) for k in ("q", "qd", "qdd", "w")]
        for _ in range(calls):
            res = rd.rnea_vjp(model, *x, mode=rd.RD_VJP_RECOMPUTE)[0]
    elif args.kernel_only in ("aba", "aba64"):
        flags = rd.RD_ABA_FP64_UPDATE if args.kernel_only == "aba64" else 0
        model = rd.Model(chaingen.make_chain(64, seed=chaingen.BASE_SEED))
        st = chaingen.make_states(16384, 64, seed=6000, kinds=("q", "qd", "tau"))
        x = [torch.from_numpy(st[k]).to(dev, torch.float32) for k in ("q", "qd", "tau")]
        ws = torch.empty(rd.aba_workspace_bytes(model, 16384, 0, flags), dtype=torch.uint8,
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
        for _ in range(calls):
            res = rd.fleet_batch(plan, *x, tune=rd.RD_FLEET_TUNE(7, 1))
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
