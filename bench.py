#!/usr/bin/env python3
"""Benchmark of the correlated-pair walker propagation (one JSON line on rank 0).

Workload (default): the M=64 synthetic pair -- Nchol=320, neutral 8/8 vs ion 8/7,
2048 walkers per system, dt=0.005, 11 repeats, shared Philox field stream.  One
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
FP64_PEAK_TFLOPS = 1.25   # GB300 nominal FP64 (no tcgen05 FP64 kind; DFMA/DMMA pipe)


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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="C2", choices=sorted(WORKLOADS))
    ap.add_argument("--coupling", default="moderate", choices=["literal", "moderate"])
    ap.add_argument("--precision", default="bf16x3", choices=["fp64", "bf16x3"])
    ap.add_argument("--mode", default="phaseless", choices=["phaseless", "free"],
                    help="free: correlated free projection (x_bar = 0, complex weights)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune-cache", default=None,
                    help="kernel-variant cache file: read if present, else written after tuning "
                         "(lets a profiled run reuse the choices of an unprofiled one)")
    ap.add_argument("--kernel", choices=["vhs", "force_bias", "taylor", "energy", "overlap",
                                         "overlap_update"],
                    help="profiling aid: set up the workload, take one step, then launch only "
                         "this kernel --reps times (no JSON line)")
    ap.add_argument("--study", choices=["correlation"],
                    help="correlation: sigma_dE of correlated against independent fields for "
                         "6..192 walkers per repeat (one JSON line per population, no "
                         "benchmark line)")
    ap.add_argument("--walkers", type=int, default=None, help="override walkers per system")
    ap.add_argument("--reps", type=int, default=2)
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


def run_reference(args, wl, rank, world):
    if rank != 0:
        return
    n_sample = 16
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
             "overlap_update": afq.K_OVERLAP_UPDATE}[args.kernel]
    ms = afq.afqmc_time_kernel(A.h, which, args.reps)
    torch.cuda.synchronize()
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

    def timed(prec, coupling, clocks=None, independent=False):
        """Pair run; independent=True gives B its own field key (uncorrelated sampling)."""
        dA, dB = systems(wl, coupling)
        A = make(dA, prec, 1, independent)
        B = make(dB, prec, 2 if independent else 1, independent)
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
        e0.record(stream)
        res = afq.pair_delta_E(A, B, n_steps, STEPS_PER_BLOCK, STEPS_PER_BLOCK, tau_eq=tau_eq,
                               raise_on_dead=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ck = clocks.stop() if clocks else None
        ms = e0.elapsed_time(e1)
        if world > 1:
            t = torch.tensor([ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        alive = [A.info().n_alive, B.info().n_alive]
        return dict(ms=ms, res=res, alive=alive, clocks=ck, A=A, B=B, dA=dA,
                    graph_kernels=afq.pair_graph_kernels(A))

    main = timed(args.precision, args.coupling, ClockSampler(torch.cuda.current_device()))
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

    # kernels timed alone on this stream with CUDA events: the path's time-dominant kernel
    # (by its share of the step in the ncu launch list) and the dominant contraction, V_HS
    A, dA = main["A"], main["dA"]
    M, X, nu, nd = dA["M"], dA["X"], dA["n_up"], dA["n_dn"]
    N, N2 = nu + nd, nu * nu + nd * nd
    P = M * (M + 1) // 2
    vhs_ms = afq.afqmc_time_kernel(A.h, afq.K_VHS, 5, stream.cuda_stream)
    if args.precision == "fp64":
        vflops = 2.0 * P * X * (2 * nw)
        tr = traffic_for("gemm_f64.cu", "vhs_gemm_C2")
        contraction = {"bound": "alu", "achieved": vflops / (vhs_ms / 1e3) / 1e12,
                       "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                       "kernel": "k_gemm_f64_vhs (V_HS, packed symmetric L, FP64)",
                       "algorithmic_flops_per_launch": vflops, "ms_per_launch": vhs_ms,
                       "traffic": tr["dram_bytes_per_launch"] if tr else None}
        # time-dominant kernel of the FP64 step: the Taylor exponential
        t_ms = afq.afqmc_time_kernel(A.h, afq.K_TAYLOR, 5, stream.cuda_stream)
        tflops = 6 * 8.0 * M * M * N * nw
        ach = tflops / (t_ms / 1e3) / 1e12
        trt = traffic_for("walker_kernels.cu", "taylor_f64_C2")
        roofline = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": ach / FP64_PEAK_TFLOPS,
                    "traffic": trt["dram_bytes_per_launch"] if trt else None,
                    "kernel": "k_taylor (Taylor exponential, FP64; largest share of the FP64 step)",
                    "algorithmic_flops_per_launch": tflops, "ms_per_launch": t_ms,
                    "peak_source": "GB300 nominal FP64 1.25 TFLOP/s (recipe table); cuBLAS DGEMM measured 1.10"}
    else:
        useful = 2.0 * M * M * X * (2 * nw)
        vflops = 3.0 * useful     # hi*hi + hi*lo + lo*hi BF16 products
        tr = traffic_for("gemm_tc.cu", "vhs_tc_C2")
        contraction = {"bound": "tensor", "achieved": vflops / (vhs_ms / 1e3) / 1e12,
                       "peak": BF16_PEAK_TFLOPS, "unit": "TFLOP/s",
                       "kernel": "k_gemm_bf16x3_tc (V_HS, split-BF16 tcgen05, full M^2 rows)",
                       "algorithmic_flops_per_launch": vflops, "useful_flops_per_launch": useful,
                       "ms_per_launch": vhs_ms,
                       "traffic": tr["dram_bytes_per_launch"] if tr else None,
                       "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst, kernel timed alone)"}
        # time-dominant kernel of the split-precision step: the propagator
        # e^{-dt K/2} e^A e^{-dt K/2} (largest share in the launch list) in the variant the
        # autotuner chose; its algorithmic work is `order` complex products A T plus two
        # real-by-complex one-body products per walker
        order = 6
        pv = A.info().tuned_taylor_smem
        p_ms = afq.afqmc_time_kernel(A.h, afq.K_TAYLOR, 5, stream.cuda_stream)
        pflops = (8.0 * order + 8.0) * M * M * N * nw
        if pv == 3:
            # tensor cores: per walker (order + 2) rounds of 3 split-BF16 MMAs, M = 128 rows
            # ([A_re; A_im] or E - I over 64 padded orbitals), N = 2 pad8(N), K = 64
            nb = 2 * ((N + 7) // 8 * 8)
            mflops = nw * (order + 2) * 3.0 * 2.0 * 128 * nb * 64
            roofline = {"bound": "tensor", "achieved": mflops / (p_ms / 1e3) / 1e12,
                        "peak": BF16_PEAK_TFLOPS, "unit": "TFLOP/s",
                        "frac": mflops / (p_ms / 1e3) / 1e12 / BF16_PEAK_TFLOPS,
                        "kernel": "k_propagate_tc (split-BF16 tcgen05 one-body + Taylor rounds; "
                                  "largest share of the split-precision step)",
                        "algorithmic_flops_per_launch": mflops, "useful_flops_per_launch": pflops,
                        "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst, kernel timed alone)"}
            trp = traffic_for("propagate_tc.cu", "propagate_tc_C2")
        else:
            name = {2: "k_propagate_f32 (fused one-body half steps + Taylor exponential, FP32"}.get(
                pv, "k_gemm_tn_f32 + k_taylor_f32 + k_gemm_tn_f32 (FP32")
            ach = pflops / (p_ms / 1e3) / 1e12
            roofline = {"bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                        "frac": ach / FP32_PEAK_TFLOPS,
                        "kernel": name + "; largest share of the split-precision step)",
                        "algorithmic_flops_per_launch": pflops,
                        "peak_source": "derived FP32 SIMT peak: 152 SMs x 128 lanes x 2 x 2.07 GHz"}
            trp = traffic_for("propagate_f32.cu", "propagate_f32_C2") if pv == 2 else None
        roofline["ms_per_launch"] = p_ms
        roofline["traffic"] = trp["dram_bytes_per_launch"] if trp else None
        roofline["variant"] = pv
        # the overlap / LU / log det / Theta kernel in the form every step runs (Psi^T Phi as
        # FP32 pairs from the FP32 walkers, FP64 LU, FP32 triangular solves for Theta); its
        # algorithmic work counted as FP64: the overlap contraction and the LU
        o_ms = afq.afqmc_time_kernel(A.h, afq.K_OVERLAP_UPDATE, 5, stream.cuda_stream)
        oflops = (4.0 * M * N2 + 8.0 / 3.0 * (nu ** 3 + nd ** 3)) * nw
        tro = traffic_for("walker_fast.cu", "overlap_fast_C2")
        overlap = {
            "bound": "alu", "achieved": oflops / (o_ms / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s", "frac": oflops / (o_ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
            "traffic": tro["dram_bytes_per_launch"] if tro else None,
            "kernel": "k_overlap_fast (overlap as FP32 pairs, FP64 LU and log det, FP32 Theta; update form)",
            "algorithmic_flops_per_launch": oflops, "ms_per_launch": o_ms,
            "flops_note": "Psi^T Phi (4 M sum N_s^2) and LU (8/3 sum N_s^3) counted as FP64 work",
            "peak_source": "GB300 nominal FP64 1.25 TFLOP/s (recipe table)"}
        # the time-dominant kernel of the step: per measurement block both kernels run once per
        # step; the larger is reported as `roofline`, the other beside it
        if o_ms > p_ms:
            roofline["kernel"] = roofline["kernel"].replace("; largest share of the split-precision step", "")
            overlap["kernel"] += "; largest share of the split-precision step"
            overlap["propagator"] = roofline
            roofline = overlap
        else:
            roofline["overlap_fp64"] = overlap
        # the tensor-core local energy: split-BF16 GEMM of Psi^T L_g Theta over (g, w) with the
        # exchange reduction in the epilogue; MMA work counts the orbital padding to P2 per spin
        e_ms = afq.afqmc_time_kernel(A.h, afq.K_EXCHANGE, 5, stream.cuda_stream)
        p2 = 4
        while p2 < max(nu, nd):
            p2 *= 2
        NPp, Kp = 2 * p2, (M + 63) // 64 * 64
        eflops = 3.0 * 2.0 * (X * NPp) * (2 * NPp * nw) * Kp
        useful_e = 2.0 * X * (nu * nu + nd * nd) * M * 2 * nw
        tre = traffic_for("energy_tc.cu", "energy_tc_C2")
        roofline["energy_tc"] = {
            "bound": "tensor", "achieved": eflops / (e_ms / 1e3) / 1e12, "peak": BF16_PEAK_TFLOPS,
            "unit": "TFLOP/s", "frac": eflops / (e_ms / 1e3) / 1e12 / BF16_PEAK_TFLOPS,
            "traffic": tre["dram_bytes_per_launch"] if tre else None,
            "kernel": "k_energy_B + k_energy_tc + k_energy_tc_reduce (split-BF16 tcgen05 local energy)",
            "algorithmic_flops_per_launch": eflops, "useful_flops_per_launch": useful_e,
            "ms_per_launch": e_ms,
            "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst, kernel timed alone)"}
    contraction["frac"] = contraction["achieved"] / contraction["peak"]
    roofline["contraction_vhs"] = contraction
    main["A"].close()
    main["B"].close()

    # the FP64 path on the same fields: throughput and sigma_dE * sqrt(GPU seconds)
    other_prec = "fp64" if args.precision != "fp64" else None
    comp = {}
    runs = {args.precision: main}
    if other_prec and world == 1:
        o = timed(other_prec, args.coupling)
        o["A"].close()
        o["B"].close()
        runs[other_prec] = o
    for p_, r_ in runs.items():
        sig = r_["res"]["dE_sigma"]
        comp[p_] = {"walker_steps_per_s": world * nw * n_steps / (r_["ms"] / 1e3),
                    "gpu_s": r_["ms"] / 1e3, "dE_mean_Ha": r_["res"]["dE_mean"],
                    "dE_sigma_Ha": sig, "sigma_sqrt_gpu_s": sig * (r_["ms"] / 1e3) ** 0.5}
    if "fp64" in comp and "bf16x3" in comp:
        comp["gpu_time_ratio_at_equal_sigma"] = (comp["fp64"]["sigma_sqrt_gpu_s"] /
                                                 comp["bf16x3"]["sigma_sqrt_gpu_s"]) ** 2
        comp["dE_difference_mHa"] = 1e3 * (comp["bf16x3"]["dE_mean_Ha"] - comp["fp64"]["dE_mean_Ha"])

    # end to end through the public API: host inputs -> setup -> pair run -> results on host
    dA, dB = systems(wl, args.coupling)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    A2, B2 = make(dA, args.precision), make(dB, args.precision)
    res2 = afq.pair_delta_E(A2, B2, n_steps, STEPS_PER_BLOCK, STEPS_PER_BLOCK, raise_on_dead=False)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    A2.close()
    B2.close()
    h2d = sum(8 * (d["h1"].size + d["L"].size + d["trial"].size) for d in (dA, dB))
    d2h = 8 * res2["E"].size
    e2e = {"value": world * nw * n_steps / e2e_s, "unit": "walker-steps/s",
           "h2d_bytes_per_step": h2d / K, "d2h_bytes_per_step": d2h / K,
           "note": "setup of both systems from host arrays + pair run + energy series to host"}

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

    other = None
    if world == 1:
        oc = "literal" if args.coupling == "moderate" else "moderate"
        r3 = timed(args.precision, oc)
        other = {"coupling": oc, "value": nw * n_steps / (r3["ms"] / 1e3), "alive_walkers": r3["alive"]}
        r3["A"].close()
        r3["B"].close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n_s = 96
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
                       "l2": "inputs larger than L2 (per-step working set ~0.5 GB)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": main["clocks"],
            "gpu_launches": per_block * K, "alive_walkers": main["alive"],
            "sigma_sqrt_t": comp, "correlated_vs_independent": corr, "other_coupling": other,
            "replicas_dE": replicas,
            "step_hbm": step_hbm_report(args.precision, args.workload,
                                        roofline.get("variant"), ms / K),
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
    elif args.study:
        run_study(args, wl)
    elif args.impl == "reference":
        run_reference(args, wl, rank, world)
    else:
        run_ours(args, wl, rank, world, local_rank)


if __name__ == "__main__":
    main()
