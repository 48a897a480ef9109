#!/usr/bin/env python3
"""Benchmark of the correlated-pair walker propagation (one JSON line on rank 0).

Workload (default): the M=128 synthetic pair -- Nchol=768, neutral 16/16 vs ion 16/15,
4096 walkers per system, dt=0.005, 11 repeats, shared Philox field stream.  One
benchmark step = one measurement block of the method for BOTH systems: 5
propagation steps (force bias, fields, V_HS, split propagator with Taylor
exponential, overlap/ratio/phaseless weight), one modified Gram-Schmidt pass and
one mixed-energy evaluation (Coulomb + exchange), i.e. every stage of the path.
Metric: correlated-pair walker-steps per second = walkers x propagation steps / s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores (a bounded walker
sample per step; the reference arm).  Under torchrun each rank runs an independent
replica on its own walker range (weak scaling; no collective on the data path).
"""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

STEPS_PER_BLOCK = 5
WORKLOADS = {
    "C1": dict(cfg="C1", n_walkers=128, dt=0.01, repeats=11,
               desc="synthetic pair M=8, Nchol=24, neutral 2/2 vs ion 2/1, 128 walkers per "
                    "system, dt=0.01, energy+MGS every 5 steps, 11 repeats"),
    "C2": dict(cfg="C2", n_walkers=2048, dt=0.005, repeats=11,
               desc="synthetic pair M=64, Nchol=320, neutral 8/8 vs ion 8/7, 2048 walkers per "
                    "system, dt=0.005, energy+MGS every 5 steps, 11 repeats"),
    "C3": dict(cfg="C3", n_walkers=4096, dt=0.005, repeats=11,
               desc="synthetic pair M=128, Nchol=768, neutral 16/16 vs ion 16/15, 4096 walkers "
                    "per system, dt=0.005, energy+MGS every 5 steps, 11 repeats"),
    "C4": dict(cfg="C4", n_walkers=2048, dt=0.005, repeats=11,
               desc="uneven synthetic pair A: M=200, Nchol=1000, 9/9; B: M=190, Nchol=950, 8/8 "
                    "(own Hamiltonian), 2048 walkers per system, dt=0.005, 11 repeats"),
}
FP64_NOMINAL_TFLOPS = 1.25   # GB300 nominal FP64 (no tcgen05 FP64 kind; DFMA/DMMA pipe)


def _measured_bf16_peak():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except Exception:
        return 1900.0   # recipe fallback (burst)


BF16_PEAK_TFLOPS = _measured_bf16_peak()


def _measured_hbm_peak():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        return 6800.0   # recipe fallback


HBM_PEAK_GBS = _measured_hbm_peak()
# FP32 SIMT peak derived from the unit counts: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


# oracle pair indices timed for cpu_baseline (about 10-30 s of host work per workload)
CPU_SAMPLE = {"C1": 128, "C2": 96, "C3": 16, "C4": 8}
# pair indices per step of the reference arm (the oracle)
REF_SAMPLE = {"C1": 128, "C2": 16, "C3": 4, "C4": 2}


def working_set_gb(wl, d):
    """Bytes one propagation step of both systems streams at least: the FP64 walkers (read and
    written) and the V_HS matrices (FP32, written and read)."""
    M, N, nw = d["M"], d["n_up"] + d["n_dn"], wl["n_walkers"]
    return 2 * nw * (2 * 2 * M * N * 8 + 2 * 2 * M * M * 4) / 1e9


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="C3", choices=sorted(WORKLOADS))
    ap.add_argument("--coupling", default="moderate", choices=["literal", "moderate"])
    ap.add_argument("--precision", default="bf16x3", choices=["fp64", "bf16x3"])
    ap.add_argument("--mode", default="phaseless", choices=["phaseless", "free"],
                    help="free: correlated free projection (x_bar = 0, complex weights)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--pair-form", type=int, choices=[0, 1], default=1,
                    help="1: each pair call is one graph launch looping over the measurement "
                         "blocks on the device (default); 0: the block graph is launched once per "
                         "block (same kernels and results; a profiler sees every kernel node)")
    ap.add_argument("--no-multidet", action="store_true",
                    help="skip the multi-determinant-trial pair measurement")
    ap.add_argument("--autotune-cache", default=None,
                    help="kernel-variant cache file: read if present, else written after tuning "
                         "(lets a profiled run reuse the choices of an unprofiled one)")
    ap.add_argument("--kernel", choices=["vhs", "force_bias", "taylor", "energy", "overlap",
                                         "overlap_update", "mgs"],
                    help="profiling aid: set up the workload, take one step, then launch only "
                         "this kernel --reps times (no JSON line)")
    ap.add_argument("--study", choices=["correlation", "pes"],
                    help="correlation: sigma_dE of correlated against independent fields for "
                         "6..192 walkers per repeat (one JSON line per population); pes: the "
                         "correlated run from the trial against the same run after the "
                         "preliminary equilibration scheme (one JSON line); no benchmark line")
    ap.add_argument("--walkers", type=int, default=None, help="override walkers per system")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--compare-steps", type=int, default=None,
                    help="blocks of the FP64-against-split comparison (default: --steps at M <= 64, "
                         "else at most 10)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def systems(wl, coupling):
    from synthetic import CONFIGS, build_system
    cfg = CONFIGS[wl["cfg"]]
    c = 1.0 if coupling == "literal" else "moderate"
    return [build_system(**dict(cfg[w], coupling=c)) for w in ("A", "B")]


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def time_oracle_sample(wl, coupling, n_walkers, blocks=1):
    """Oracle (CPU, FP64) on n_walkers pair indices for `blocks` measurement blocks of both systems."""
    from oracle import afqmc as orc
    from oracle.philox import gaussian_fields
    dA, dB = systems(wl, coupling)
    osys = [orc.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], wl["dt"]) for d in (dA, dB)]
    k = np.arange(n_walkers)
    wks = [orc.Walkers(s, n_walkers) for s in osys]
    t0 = time.perf_counter()
    t = 0
    for _ in range(blocks):
        for _ in range(STEPS_PER_BLOCK):
            for s, wk in zip(osys, wks):
                orc.propagate(s, wk, gaussian_fields(1, t, k, s.X))
            t += 1
        for s, wk in zip(osys, wks):
            orc.orthonormalise(s, wk)
            orc.local_energy(s, wk.phi)
    return time.perf_counter() - t0


def host_description():
    """The host the oracle baseline ran on: machine, logical CPUs, and the CPU model when the
    kernel reports one."""
    import platform
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if model is None:   # aarch64 kernels report no model name in /proc/cpuinfo
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.strip().lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"machine": platform.machine(), "nproc": os.cpu_count(), "cpu_model": model}


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(v):
            return int(os.environ[v])
    return os.cpu_count()


def device_code_sha256(text):
    """sha256 of a CUDA source's __global__ and __device__ functions (from the start of the
    declaring line to the closing brace of the body), so that host-side edits in the same file
    leave the recorded traffic of unchanged kernels valid."""
    parts = []
    for m in re.finditer(r"__(?:global|device)__", text):
        brace, semi = text.find("{", m.end()), text.find(";", m.end())
        if brace < 0 or 0 <= semi < brace:
            continue    # a declaration or a __device__ variable
        depth, i = 0, brace
        while i < len(text):
            depth += {"{": 1, "}": -1}.get(text[i], 0)
            if depth == 0:
                break
            i += 1
        parts.append(text[text.rfind("\n", 0, m.start()) + 1:i + 1])
    return hashlib.sha256("\n".join(parts).encode()).hexdigest()


def traffic_for(kernel_file, name):
    """dram bytes per launch from the committed ncu summary, if the kernel is unchanged: the
    file's device code hashes as it did when the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        data = json.load(open(path))
        ent = data[name]
        src = open(os.path.join(ROOT, "paper_1703_01545_gb300", "csrc", kernel_file)).read()
        if "device_sha256" in ent:
            return ent if ent["device_sha256"] == device_code_sha256(src) else None
        return ent if ent.get("source_sha256") == hashlib.sha256(src.encode()).hexdigest() else None
    except Exception:
        return None


def step_hbm_report(precision, workload, propagation_variant, ms_per_block):
    """DRAM rate of one measurement block of the split-precision step at the M=64 workload:
    the recorded ncu DRAM bytes of each kernel captured there (system A's capture stands for
    both systems), times its launches per block, over the block's CUDA-event time.  Kernels
    without a current capture count zero, so this is a lower bound on the step's traffic.
    None for other workloads and precisions."""
    if precision != "bf16x3" or workload != "C2" or not ms_per_block > 0:
        return None
    steps = 2 * STEPS_PER_BLOCK            # propagation steps of both systems in one block
    items = [("walker_fast.cu", "overlap_fast_C2", steps), ("gemm_tc.cu", "vhs_tc_C2", steps),
             ("energy_tc.cu", "energy_tc_C2", 2), ("walker_fast.cu", "mgs_reg_C2", 2)]
    if propagation_variant == 3:
        items.insert(0, ("propagate_tc.cu", "propagate_tc_C2", steps))
    counted, total = {}, 0.0
    for kernel_file, name, launches in items:
        t = traffic_for(kernel_file, name)
        if t:
            counted[t["kernel"]] = launches
            total += launches * float(t["dram_bytes_per_launch"])
    if not counted:
        return None
    gbs = total / (ms_per_block / 1e3) / 1e9
    return {"bound": "hbm", "achieved": gbs, "peak": HBM_PEAK_GBS, "unit": "GB/s",
            "frac": gbs / HBM_PEAK_GBS, "dram_bytes_per_block": total,
            "launches_per_block": counted,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs",
            "note": "recorded ncu DRAM bytes of the captured kernels only (a lower bound)"}


def measure_fp64_peak():
    """Measured FP64 rate of this GPU: the best of three cuBLAS DGEMMs (4096^3, through torch),
    in TFLOP/s; the nominal rate if the measurement fails."""
    import torch
    try:
        n = 4096
        a = torch.randn(n, n, dtype=torch.float64, device="cuda")
        b = torch.randn(n, n, dtype=torch.float64, device="cuda")
        torch.matmul(a, b)
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        del a, b
        return 2.0 * n ** 3 / (best / 1e3) / 1e12, "measured: cuBLAS DGEMM 4096^3, best of 3 (burst)"
    except Exception:
        return FP64_NOMINAL_TFLOPS, "GB300 nominal FP64 (measurement failed)"


def measure_kernels(afq, A, dA, nw, precision, workload, stream):
    """Each kernel of one propagation step (and of the measurement's Gram-Schmidt and local
    energy) timed alone with CUDA events, with its algorithmic work from the method's flop
    counts per walker (real flops; complex x real MAC = 4, complex x complex = 8):
      force bias 4 X N M;  V_HS 4 P X, P = M (M + 1) / 2 (packed symmetric L; the full count
      4 M^2 X beside it);  propagator (8 order + 8) M^2 N (Taylor terms and the two one-body
      half steps);  overlap (split path, all FP32: the overlap sums 4 M sum N_s^2, the LU
      8/3 sum N_s^3 and the Theta solves 8 M sum N_s^2);  orthonormalisation 8 M sum N_s^2
      (Gram-Schmidt and Cholesky QR alike);  local energy 4 X M sum N_s^2 + 8 X sum N_s^2.
    Tensor-core kernels also give the split-BF16 MMA work they issue (3 products per product,
    padded tiles) as mma_flops.  Launches per block: 5 propagation steps, one Gram-Schmidt and
    one energy, for one system (system A)."""
    M, X, nu, nd = dA["M"], dA["X"], dA["n_up"], dA["n_dn"]
    N, N2, N3 = nu + nd, nu * nu + nd * nd, nu ** 3 + nd ** 3
    P = M * (M + 1) // 2
    order = 6
    f64_peak, f64_src = measure_fp64_peak()
    bf16 = ("MEASURED_PEAKS.json bf16_tflops (burst; kernel timed alone)", BF16_PEAK_TFLOPS)
    f32 = ("derived FP32 SIMT peak: 152 SMs x 128 lanes x 2 x 2.07 GHz", FP32_PEAK_TFLOPS)
    f64 = (f64_src, f64_peak)
    split = precision != "fp64"
    pv = A.info().tuned_taylor_smem if split else -1
    pad = lambda x, m: (x + m - 1) // m * m
    nb2 = 2 * pad(N, 8)

    def entry(which, launches, flops, bound, peak, name, mma=None, traffic=None, **extra):
        ms = afq.afqmc_time_kernel(A.h, which, 5, stream.cuda_stream)
        ach = flops / (ms / 1e3) / 1e12
        e = {"bound": bound, "achieved": ach, "peak": peak[1], "unit": "TFLOP/s",
             "frac": ach / peak[1], "traffic": traffic, "kernel": name,
             "algorithmic_flops_per_launch": flops, "ms_per_launch": ms,
             "launches_per_block": launches, "ms_per_block": ms * launches,
             "peak_source": peak[0]}
        if mma is not None:
            e["mma_flops_per_launch"] = mma
            e["mma_tflops"] = mma / (ms / 1e3) / 1e12
            e["mma_frac"] = e["mma_tflops"] / peak[1]
        e.update(extra)
        return e

    def tr(kfile, key):
        t = traffic_for(kfile, f"{key}_{workload}")
        return t["dram_bytes_per_launch"] if t else None

    out = {}
    fb = 4.0 * X * N * M * nw
    vhs = 4.0 * P * X * nw
    vhs_full = 4.0 * M * M * X * nw
    prop = (8.0 * order + 8.0) * M * M * N * nw
    mgs = 8.0 * M * N2 * nw
    en = (4.0 * X * M * N2 + 8.0 * X * N2) * nw
    if split:
        out["force_bias"] = entry(afq.K_FORCE_BIAS, STEPS_PER_BLOCK, fb, "tensor", bf16,
                                  "k_gemm_bf16x3_tc (force bias, split-BF16 tcgen05)",
                                  mma=3 * 2.0 * pad(X, 128) * pad(N * M, 64) * 2 * nw,
                                  traffic=tr("gemm_tc.cu", "force_bias_tc"))
        # with the large-M tensor-core propagator the contraction covers only the
        # lower-triangle 16 x 16 blocks of index pairs (two 128-row tiles each), when the
        # persistent kernel runs it (at least 2 x 152 tiles of 128 x 256)
        nb = (M + 15) // 16
        tri_rows = nb * (nb + 1) // 2 * 256
        tri = pv == 4 and (tri_rows // 128) * -(-2 * nw // 256) >= 2 * 152 and pad(2 * nw, 128) % 256 == 0
        vhs_rows = tri_rows if tri else pad(M * M, 128)
        out["vhs"] = entry(afq.K_VHS, STEPS_PER_BLOCK, vhs, "tensor", bf16,
                           "k_gemm_bf16x3_tc_persist (V_HS, split-BF16 tcgen05, "
                           + ("lower-triangle 16 x 16 blocks of the M^2 rows, mirror written "
                              "transposed)" if tri else "full M^2 rows)"),
                           mma=3 * 2.0 * vhs_rows * pad(X, 64) * 2 * nw,
                           traffic=tr("gemm_tc.cu", "vhs_tc"),
                           full_count_flops_per_launch=vhs_full)
        out["vhs"]["frac_full_count"] = out["vhs"]["frac"] * vhs_full / vhs
        if pv == 3:
            out["propagator"] = entry(
                afq.K_TAYLOR, STEPS_PER_BLOCK, prop, "tensor", bf16,
                "k_propagate_tc (split-BF16 tcgen05 one-body + Taylor rounds, M <= 64)",
                mma=nw * (order + 2) * 3.0 * 2.0 * 128 * nb2 * 64,
                traffic=tr("propagate_tc.cu", "propagate_tc"), variant=pv)
        elif pv == 4:
            # per 128-row tile of orbitals and 16-wide K step holding orbitals: 3 products per
            # one-body round, 6 per Taylor round (A_re and A_im), each 2 x 128 x 2 Np x 16 flops
            mt = (M + 127) // 128
            ks = sum(min(4, (M - 64 * kb + 15) // 16) for kb in range((M + 63) // 64))
            mma4 = nw * mt * ks * (2 * 3 + order * 6) * 2.0 * 128 * nb2 * 16
            out["propagator"] = entry(
                afq.K_TAYLOR, STEPS_PER_BLOCK, prop, "tensor", bf16,
                "k_propagate_tcl (split-BF16 tcgen05 one-body + Taylor rounds, V_HS streamed by TMA)",
                mma=mma4, traffic=tr("propagate_tcl.cu", "propagate_tcl"), variant=pv)
        else:
            name = {2: "k_propagate_f32 (fused one-body half steps + Taylor exponential, FP32)"}.get(
                pv, "k_gemm_tn_f32 + k_taylor_f32 + k_gemm_tn_f32 (FP32)")
            out["propagator"] = entry(afq.K_TAYLOR, STEPS_PER_BLOCK, prop, "alu", f32, name,
                                      traffic=tr("propagate_f32.cu", "propagate_f32") if pv == 2 else None,
                                      variant=pv)
        ov = 4.0 * M * N2 * nw + 8.0 / 3.0 * N3 * nw + 8.0 * M * N2 * nw
        out["overlap"] = entry(afq.K_OVERLAP_UPDATE, STEPS_PER_BLOCK, ov, "alu", f32,
                               "k_overlap_fast (update form: overlap sums, LU and Theta in FP32, "
                               "log det accumulated with a power-of-two exponent)",
                               traffic=tr("walker_fast.cu", "overlap_fast"),
                               flops_note="overlap sums 4 M sum N_s^2, LU 8/3 sum N_s^3, Theta "
                                          "solves 8 M sum N_s^2")
        if A.info().tuned_orthonormalise == 1:
            out["mgs"] = entry(afq.K_MGS, 1, mgs, "alu", f32,
                               "k_mgs_chol (Cholesky QR: Gram matrix and Q in FP32, FP64 factor "
                               "and log det)",
                               traffic=tr("walker_fast.cu", "mgs_chol"))
        else:
            out["mgs"] = entry(afq.K_MGS, 1, mgs, "alu", f64,
                               "k_mgs_reg / k_mgs_warp (FP64 Gram-Schmidt)",
                               traffic=tr("walker_fast.cu", "mgs_reg"))
        p2 = 4
        while p2 < max(nu, nd):
            p2 *= 2
        NPp = 2 * p2
        if pad(M, 64) > 64:
            # one product per spin block: rows (g, a < P2) and columns (w, re/im, b < P2) of
            # each spin, padded to whole 128 x 256 tiles
            emma = 3.0 * 2.0 * 2 * pad(X * p2, 128) * pad(2 * p2 * nw, 256) * pad(M, 64)
        else:
            emma = 3.0 * 2.0 * pad(X * NPp, 128) * pad(2 * NPp * nw, 256) * pad(M, 64)
        out["energy"] = entry(afq.K_EXCHANGE, 1, en, "tensor", bf16,
                              "k_energy_B + k_energy_tc (split-BF16 tcgen05 local energy)",
                              mma=emma, traffic=tr("energy_tc.cu", "energy_tc"))
    else:
        out["force_bias"] = entry(afq.K_FORCE_BIAS, STEPS_PER_BLOCK, fb, "alu", f64,
                                  "k_gemm_f64_force_bias (FP64)")
        out["vhs"] = entry(afq.K_VHS, STEPS_PER_BLOCK, vhs, "alu", f64,
                           "k_gemm_f64_vhs (V_HS, packed symmetric L, FP64)",
                           traffic=tr("gemm_f64.cu", "vhs_gemm"))
        out["propagator"] = entry(afq.K_TAYLOR, STEPS_PER_BLOCK, 8.0 * order * M * M * N * nw, "alu",
                                  f64, "k_taylor (Taylor exponential, FP64; the one-body half steps "
                                  "run as separate FP64 GEMMs)", traffic=tr("walker_kernels.cu", "taylor_f64"))
        out["overlap"] = entry(afq.K_OVERLAP, STEPS_PER_BLOCK,
                               (12.0 * M * N2 + 8.0 * N3) * nw, "alu", f64,
                               "k_overlap (FP64 overlap, Gauss-Jordan inverse, Theta; refresh form)")
        out["mgs"] = entry(afq.K_MGS, 1, mgs, "alu", f64, "k_mgs + overlap refresh (FP64)")
        out["energy"] = entry(afq.K_EXCHANGE, 1, en, "alu", f64, "k_energy (FP64 local energy)")
    return out


def multidet_pair(afq, torch, stream, coupling, blocks=2, warm=1):
    """Correlated pair with multi-determinant trials (CASCI over 9 canonical orbitals, CI
    coefficients >= 0.01) at the M=64 shape, FP64: pair walker-steps/s over `blocks` timed
    measurement blocks, the determinant counts and the per-launch times of the determinant
    overlaps and the local energy."""
    from synthetic.multidet import cas_trial
    wl = WORKLOADS["C2"]
    ds = systems(wl, coupling)
    nw, dt, R = wl["n_walkers"], wl["dt"], wl["repeats"]
    hs, ndet = [], []
    for d in ds:
        dets, c, start, _ = cas_trial(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], 9)
        ndet.append(len(c))
        hs.append(afq.System(d["h1"], d["L"], None, d["n_up"], d["n_dn"], dt=dt, n_walkers=nw,
                             seed=1, n_repeats=R, dets=dets, coeffs=c, start=start))
    afq.pair_delta_E(hs[0], hs[1], warm * STEPS_PER_BLOCK, STEPS_PER_BLOCK, STEPS_PER_BLOCK,
                     raise_on_dead=False)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    res = afq.pair_delta_E(hs[0], hs[1], blocks * STEPS_PER_BLOCK, STEPS_PER_BLOCK,
                           STEPS_PER_BLOCK, raise_on_dead=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out = {"workload": wl["desc"].split(",")[0] + " (M=64 pair), CASCI trials over 9 orbitals",
           "precision": "fp64", "n_det": ndet, "walker_steps_per_s": nw * blocks * STEPS_PER_BLOCK / (ms / 1e3),
           "ms_per_block": ms / blocks, "dE_last_Ha": float(np.mean(res["E"][-1, 1] - res["E"][-1, 0])),
           "overlap_ms_per_launch": afq.afqmc_time_kernel(hs[0].h, afq.K_OVERLAP, 3, stream.cuda_stream),
           "energy_ms_per_launch": afq.afqmc_time_kernel(hs[0].h, afq.K_EXCHANGE, 3, stream.cuda_stream),
           "alive_walkers": [h.info().n_alive for h in hs]}
    for h in hs:
        h.close()
    return out


def run_reference(args, wl, rank, world):
    if rank != 0:
        return
    n_sample = REF_SAMPLE[wl["cfg"]]
    for _ in range(args.warmup):
        time_oracle_sample(wl, args.coupling, n_sample)
    tot = 0.0
    for _ in range(args.steps):
        tot += time_oracle_sample(wl, args.coupling, n_sample)
    value = n_sample * STEPS_PER_BLOCK * args.steps / tot
    cores = blas_threads()
    line = {
        "impl": "reference", "metric": "correlated-pair walker-steps/s", "value": value,
        "unit": "walker-steps/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["desc"], "coupling": args.coupling,
                   "sample": f"{n_sample} of {wl['n_walkers']} pair indices per step"},
        "cpu_baseline": {"value": value, "unit": "walker-steps/s", "cores": cores, "kind": "oracle",
                         "sample": f"{n_sample} pair indices x {STEPS_PER_BLOCK} steps + MGS + "
                                   "energy, both systems, per step",
                         "host": host_description()},
        "e2e": {"value": value, "unit": "walker-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_kernel(args, wl):
    """Launch one step kernel in isolation (for a small, bounded ncu capture)."""
    import torch
    import paper_1703_01545_gb300 as afq
    afq.build()
    d = systems(wl, args.coupling)[0]
    nw = args.walkers or wl["n_walkers"]
    A = afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=wl["dt"], n_walkers=nw,
                   precision={"fp64": afq.FP64, "bf16x3": afq.BF16X3}[args.precision],
                   autotune_cache=args.autotune_cache)
    A.propagate(1)
    which = {"vhs": afq.K_VHS, "force_bias": afq.K_FORCE_BIAS, "taylor": afq.K_TAYLOR,
             "energy": afq.K_EXCHANGE, "overlap": afq.K_OVERLAP,
             "overlap_update": afq.K_OVERLAP_UPDATE, "mgs": afq.K_MGS}[args.kernel]
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("kernel_only")   # lets a profiler skip the setup launches
    ms = afq.afqmc_time_kernel(A.h, which, args.reps)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(f"{args.kernel}: {ms:.3f} ms per launch ({nw} walkers)")
    A.close()


def run_study(args, wl):
    """Efficiency of correlated sampling (Sec. III): for each population, the pair run with
    shared fields and again with independent_fields (B keyed by its own seed), each started,
    run once for --steps blocks to equilibrate and capture its graph, then run and timed for
    --steps more blocks. Both runs at one population cost the same per step, so the GPU time
    to reach a given sigma_dE scales with sigma^2 x t. One JSON line per population."""
    import torch
    import paper_1703_01545_gb300 as afq

    afq.build()
    dt, R = wl["dt"], wl["repeats"]
    n_steps = args.steps * STEPS_PER_BLOCK
    tau_eq = 0.25 * n_steps * dt
    prec = {"fp64": afq.FP64, "bf16x3": afq.BF16X3}[args.precision]
    dA, dB = systems(wl, args.coupling)
    stream = torch.cuda.current_stream()
    for per in (6, 12, 24, 48, 96, 192):
        nw = per * R
        row = {"study": "correlated_vs_independent", "workload": wl["cfg"],
               "coupling": args.coupling, "precision": args.precision, "mode": args.mode,
               "repeats": R,
               "walkers_per_repeat": per, "walkers_per_system": nw,
               "propagation_steps": n_steps, "tau_eq": tau_eq}
        for key, indep in (("correlated", False), ("independent", True)):
            hs = [afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=dt,
                             n_walkers=nw, seed=seed, n_repeats=R, precision=prec,
                             autotune_cache=args.autotune_cache, independent_fields=indep,
                             mode=afq.FREE if args.mode == "free" else afq.PHASELESS)
                  for d, seed in ((dA, 1), (dB, 2 if indep else 1))]
            afq.pair_delta_E(hs[0], hs[1], n_steps, STEPS_PER_BLOCK, STEPS_PER_BLOCK,
                             raise_on_dead=False)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            res = afq.pair_delta_E(hs[0], hs[1], n_steps, STEPS_PER_BLOCK, STEPS_PER_BLOCK,
                                   tau_eq=tau_eq, raise_on_dead=False)
            e1.record(stream)
            torch.cuda.synchronize()
            row[key] = {"dE_mean_Ha": res["dE_mean"], "dE_sigma_Ha": res["dE_sigma"],
                        "ms": e0.elapsed_time(e1), "alive": [h.info().n_alive for h in hs]}
            for h in hs:
                h.close()
        c, i = row["correlated"], row["independent"]
        row["gpu_time_ratio_at_equal_sigma"] = (
            (i["dE_sigma_Ha"] ** 2 * i["ms"]) / (c["dE_sigma_Ha"] ** 2 * c["ms"])
            if c["dE_sigma_Ha"] > 0 else None)
        print(json.dumps(row), flush=True)


def run_pes_study(args, wl):
    """Preliminary equilibration scheme (Sec. II.C) against starting both systems at their
    trials. Plain: the pair from the trials for --steps blocks, tau_eq = tau / 4. PES: the
    primary system alone for --steps blocks of [5 steps, orthonormalisation, comb of every
    repeat], the secondary seeded from its walkers (weights by the overlap ratio), then the
    pair for --steps blocks from there with tau_eq = 0. sigma_dE and Delta E of both, and
    the GPU time of each part."""
    import numpy as np
    import torch
    import paper_1703_01545_gb300 as afq

    afq.build()
    dt, R, nw = wl["dt"], wl["repeats"], args.walkers or wl["n_walkers"]
    n_steps = args.steps * STEPS_PER_BLOCK
    prec = {"fp64": afq.FP64, "bf16x3": afq.BF16X3}[args.precision]
    dA, dB = systems(wl, args.coupling)
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(1703)

    def make():
        return [afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=dt,
                           n_walkers=nw, seed=1, n_repeats=R, precision=prec,
                           autotune_cache=args.autotune_cache) for d in (dA, dB)]

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    row = {"study": "pes", "workload": wl["cfg"], "coupling": args.coupling,
           "precision": args.precision, "repeats": R, "walkers_per_system": nw,
           "propagation_steps": n_steps}
    A, B = make()
    res, ms = timed(lambda: afq.pair_delta_E(A, B, n_steps, STEPS_PER_BLOCK, STEPS_PER_BLOCK,
                                             tau_eq=0.25 * n_steps * dt, raise_on_dead=False))
    row["from_trial"] = {"dE_mean_Ha": res["dE_mean"], "dE_sigma_Ha": res["dE_sigma"],
                         "tau_eq": 0.25 * n_steps * dt, "ms": ms}
    A.close()
    B.close()
    A, B = make()

    def equilibrate():
        for _ in range(args.steps):
            A.propagate(STEPS_PER_BLOCK)
            A.orthonormalise()
            A.population_control(rng.random(R))
        B.seed_from(A)

    _, ms_eq = timed(equilibrate)
    res, ms = timed(lambda: afq.pair_delta_E(A, B, n_steps, STEPS_PER_BLOCK, STEPS_PER_BLOCK,
                                             tau_eq=0.0, raise_on_dead=False))
    row["pes"] = {"dE_mean_Ha": res["dE_mean"], "dE_sigma_Ha": res["dE_sigma"], "tau_eq": 0.0,
                  "ms_equilibration": ms_eq, "ms": ms,
                  "alive": [h.info().n_alive for h in (A, B)]}
    A.close()
    B.close()
    print(json.dumps(row), flush=True)


def run_ours(args, wl, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    import paper_1703_01545_gb300 as afq

    from paper_1703_01545_gb300.replicas import walker_offset as replica_offset

    torch.cuda.set_device(local_rank)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    afq.build()
    nw, dt, R = wl["n_walkers"], wl["dt"], wl["repeats"]
    K, W = args.steps, args.warmup
    n_steps = K * STEPS_PER_BLOCK
    tau_eq = 0.25 * n_steps * dt
    stream = torch.cuda.current_stream()
    prec_id = {"fp64": afq.FP64, "bf16x3": afq.BF16X3}

    def make(d, prec, seed=1, independent=False):
        return afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=dt, n_walkers=nw,
                          seed=seed, n_repeats=R, walker_offset=replica_offset(rank, nw), precision=prec_id[prec],
                          autotune_cache=args.autotune_cache, independent_fields=independent,
                          mode=afq.FREE if args.mode == "free" else afq.PHASELESS)

    def timed(prec, coupling, clocks=None, independent=False, blocks=None, form=1):
        """Pair run of `blocks` (default K) timed measurement blocks after W warm-up blocks;
        independent=True gives B its own field key (uncorrelated sampling); form 1 runs the
        call as one graph launch, form 0 launches the block graph once per block."""
        n_steps_run = (K if blocks is None else blocks) * STEPS_PER_BLOCK
        dA, dB = systems(wl, coupling)
        A = make(dA, prec, 1, independent)
        B = make(dB, prec, 2 if independent else 1, independent)
        A.select_kernel(afq.K_PAIR_LOOP, form)
        afq.pair_delta_E(A, B, W * STEPS_PER_BLOCK, STEPS_PER_BLOCK, STEPS_PER_BLOCK,
                         raise_on_dead=False)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        if clocks:
            clocks.start()
            time.sleep(0.3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        if clocks:   # the timed region of the headline run, for a profiler's NVTX filter
            torch.cuda.nvtx.range_push("timed_region")
        e0.record(stream)
        res = afq.pair_delta_E(A, B, n_steps_run, STEPS_PER_BLOCK, STEPS_PER_BLOCK,
                               tau_eq=0.25 * n_steps_run * dt, raise_on_dead=False)
        e1.record(stream)
        torch.cuda.synchronize()
        if clocks:
            torch.cuda.nvtx.range_pop()
        ck = clocks.stop() if clocks else None
        ms = e0.elapsed_time(e1)
        if world > 1:
            t = torch.tensor([ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        alive = [A.info().n_alive, B.info().n_alive]
        return dict(ms=ms, res=res, alive=alive, clocks=ck, A=A, B=B, dA=dA,
                    graph_kernels=afq.pair_graph_kernels(A), steps=n_steps_run,
                    form=afq.pair_run_form(A))

    main = timed(args.precision, args.coupling, ClockSampler(torch.cuda.current_device()),
                 form=args.pair_form)
    ms = main["ms"]
    # Delta E over the repeats of every replica (gathered after the timed region)
    replicas = None
    if world > 1:
        from paper_1703_01545_gb300.replicas import gather_series, merged_delta_E
        E_all = gather_series(main["res"]["E"])
        m_, s_, t_ = merged_delta_E(E_all, main["res"]["taus"], tau_eq)
        replicas = {"dE_mean_Ha": m_, "dE_sigma_Ha": s_, "tau_at_min": t_,
                    "repeats": int(E_all.shape[2])}
    value = world * nw * n_steps / (ms / 1e3)

    # every kernel of the step timed alone on this stream with CUDA events; the one with the
    # largest time per measurement block is the dominant kernel reported as `roofline`
    A, dA = main["A"], main["dA"]
    kernels = measure_kernels(afq, A, dA, nw, args.precision, args.workload, stream)
    dom = max(kernels, key=lambda k: kernels[k]["ms_per_block"])
    roofline = dict(kernels[dom])
    roofline["kernel_key"] = dom
    main["A"].close()
    main["B"].close()

    # the FP64 path on the same fields: throughput and sigma_dE * sqrt(GPU seconds), both paths
    # over the same number of blocks (fewer than K where the FP64 path is slow: M >= 128)
    other_prec = "fp64" if args.precision != "fp64" else None
    cmp_blocks = args.compare_steps or (K if wl["cfg"] in ("C1", "C2") else min(K, 10))
    comp = {}
    runs = {}
    if other_prec and world == 1:
        runs[args.precision] = main
        if cmp_blocks != K:
            r_ = timed(args.precision, args.coupling, blocks=cmp_blocks)
            r_["A"].close()
            r_["B"].close()
            runs[args.precision] = r_
        o = timed(other_prec, args.coupling, blocks=cmp_blocks)
        o["A"].close()
        o["B"].close()
        runs[other_prec] = o
    for p_, r_ in runs.items():
        sig = r_["res"]["dE_sigma"]
        comp[p_] = {"walker_steps_per_s": world * nw * r_["steps"] / (r_["ms"] / 1e3),
                    "gpu_s": r_["ms"] / 1e3, "propagation_steps": r_["steps"],
                    "dE_mean_Ha": r_["res"]["dE_mean"], "dE_sigma_Ha": sig,
                    "sigma_sqrt_gpu_s": sig * (r_["ms"] / 1e3) ** 0.5,
                    "alive_walkers": r_["alive"]}
    if "fp64" in comp and "bf16x3" in comp:
        comp["gpu_time_ratio_at_equal_sigma"] = (comp["fp64"]["sigma_sqrt_gpu_s"] /
                                                 comp["bf16x3"]["sigma_sqrt_gpu_s"]) ** 2
        comp["dE_difference_mHa"] = 1e3 * (comp["bf16x3"]["dE_mean_Ha"] - comp["fp64"]["dE_mean_Ha"])

    # end to end through the public API: host inputs -> setup -> pair run -> results on host
    dA, dB = systems(wl, args.coupling)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    A2 = make(dA, args.precision)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    B2 = make(dB, args.precision)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    res2 = afq.pair_delta_E(A2, B2, n_steps, STEPS_PER_BLOCK, STEPS_PER_BLOCK, raise_on_dead=False)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    e2e_s = t3 - t0
    A2.close()
    B2.close()
    h2d = sum(8 * (d["h1"].size + d["L"].size + d["trial"].size) for d in (dA, dB))
    d2h = 8 * res2["E"].size
    e2e = {"value": world * nw * n_steps / e2e_s, "unit": "walker-steps/s",
           "h2d_bytes_per_step": h2d / K, "d2h_bytes_per_step": d2h / K,
           "seconds": {"setup_A": t1 - t0, "setup_B": t2 - t1, "pair_run": t3 - t2},
           "note": "setup of both systems from host arrays (H2D copies, setup kernels and the "
                   "kernel-variant autotuning inside) + the same pair run + energy series to host"}

    # the same run with the block graph launched once per measurement block instead of one
    # launch looping on the device (identical kernels and results)
    launch = None
    if world == 1:
        r0 = timed(args.precision, args.coupling, form=1 - args.pair_form)
        r0["A"].close()
        r0["B"].close()
        one, per = (main, r0) if main["form"] == 1 else (r0, main)
        launch = {"form": main["form"], "ms_per_block_one_launch": one["ms"] / K,
                  "ms_per_block_launch_per_block": per["ms"] / K,
                  "kernels_per_block": main["graph_kernels"],
                  "identical_dE": bool(r0["res"]["dE_mean"] == main["res"]["dE_mean"]),
                  "note": "one graph launch per pair call (device-side while loop over the "
                          "measurement blocks) against one block-graph launch per block"}

    # correlated against independent fields at the same workload and precision (Sec. III):
    # GPU time to reach a given sigma_dE scales as sigma^2 * t
    corr = None
    if world == 1:
        ri = timed(args.precision, args.coupling, independent=True)
        ri["A"].close()
        ri["B"].close()
        sc, si = main["res"]["dE_sigma"], ri["res"]["dE_sigma"]
        corr = {"dE_mean_correlated_Ha": main["res"]["dE_mean"], "dE_sigma_correlated_Ha": sc,
                "dE_mean_independent_Ha": ri["res"]["dE_mean"], "dE_sigma_independent_Ha": si,
                "ms_correlated": ms, "ms_independent": ri["ms"],
                "gpu_time_ratio_at_equal_sigma": (si * si * ri["ms"]) / (sc * sc * ms)
                if sc > 0 else None,
                "repeats": R, "note": "independent: system B keyed by its own seed"}

    # multi-determinant trial (Sec. II.D): the M=64 pair with truncated CASCI trials, FP64
    md = None
    if world == 1 and not args.no_multidet:
        md = multidet_pair(afq, torch, stream, args.coupling)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n_s = CPU_SAMPLE[wl["cfg"]]
        ts = time_oracle_sample(wl, args.coupling, n_s)
        cpu = {"value": n_s * STEPS_PER_BLOCK / ts, "unit": "walker-steps/s", "cores": blas_threads(),
               "kind": "oracle",
               "sample": f"{n_s} pair indices x {STEPS_PER_BLOCK} steps + MGS + energy, both systems",
               "host": host_description()}
    # kernel nodes of the captured measurement block (both systems), replayed once per block
    per_block = main["graph_kernels"]
    if rank == 0:
        line = {
            "metric": "correlated-pair walker-steps/s", "value": value, "unit": "walker-steps/s",
            "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": ms / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "bf16x3+f32 (f64 determinants/weights/MGS)",
            "data": "synthetic",
            "config": {"workload": wl["desc"], "coupling": args.coupling, "precision": args.precision,
                       "mode": args.mode,
                       "step": "one measurement block (5 propagation steps + MGS + energy) of both systems",
                       "l2": f"inputs larger than L2 (walkers and V_HS alone: "
                             f"{working_set_gb(wl, dA):.2f} GB per step against 0.13 GB of L2)",
                       "fp64_comparison_blocks": cmp_blocks,
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": main["clocks"],
            "gpu_launches": per_block * K + (1 if main["form"] == 1 else 0),
            "alive_walkers": main["alive"],
            "pair_launch": launch,
            "sigma_sqrt_t": comp, "correlated_vs_independent": corr, "kernels": kernels,
            "multidet": md,
            "replicas_dE": replicas,
            "step_hbm": step_hbm_report(args.precision, args.workload,
                                        kernels["propagator"].get("variant"), ms / K),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    rank, world, local_rank = dist_env()
    wl = WORKLOADS[args.workload]
    if args.kernel:
        run_kernel(args, wl)
    elif args.study == "pes":
        run_pes_study(args, wl)
    elif args.study:
        run_study(args, wl)
    elif args.impl == "reference":
        run_reference(args, wl, rank, world)
    else:
        run_ours(args, wl, rank, world, local_rank)


if __name__ == "__main__":
    main()
