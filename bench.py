#!/usr/bin/env python
"""Benchmark of the parallel proximal mean-field solve on one GB300 (or N replicas).

Workload: the segmentation-shaped grid CRF -- 512 x 512 pixels, L = 21
labels, 8-connected, unaries -log softmax(N(0, 2^2) logits), symmetric mu
U(-1,1) with zero diagonal, colour-contrast edge weights -- solved with 100
parallel proximal iterations at the step eta = 1/(1+Lambda) (Sec. 3.2).

A step is one full solve: q^0 = softmax(-U), 100 fused iterations (messages,
proximal step, renormalisation, free energy of each iterate) and the free
energy of the final iterate, with the model (and its step-size constant)
already resident in HBM.  The metric counts variable-label updates:
N * L * iterations per solve.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own instance (replicas, weak scaling);
the reported time is the maximum over ranks.  --impl reference times the
FP64 CPU oracle on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "mean-field updates/s (vars·labels·iters); p50/p99 solve latency; vs FP32 plain"
UNIT = "updates/s"
H, W, L, CONN, ITERS = 512, 512, 21, 8, 100
SEED = 1
L2_FLUSH_BYTES = 256 << 20
WORKLOAD = ("segmentation-shaped grid CRF 512x512, L=21, 8-connected, 100 parallel proximal "
            "iterations, FP32 messages and state")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-dense", action="store_true",
                   help="skip the fully connected (N=9216, L=21) FP32 / BF16 measurements")
    p.add_argument("--dense-only", action="store_true",
                   help="run only the fully connected measurements (profiling captures)")
    p.add_argument("--serve-requests", type=int, default=4096,
                   help="requests of the serving measurement (0 skips it)")
    p.add_argument("--serve-only", action="store_true")
    p.add_argument("--no-denoising", action="store_true",
                   help="skip the 64x64 binary denoising measurement")
    p.add_argument("--denoising-only", action="store_true")
    p.add_argument("--no-sparse", action="store_true", help="skip the edge-list graph measurements")
    p.add_argument("--sparse-only", action="store_true")
    p.add_argument("--no-eta-sweep", action="store_true",
                   help="skip the step-parameter sensitivity sweep")
    p.add_argument("--eta-sweep-only", action="store_true")
    p.add_argument("--no-grid-bf16", action="store_true",
                   help="skip the BF16 tensor-core form of the segmentation workload")
    p.add_argument("--grid-bf16-only", action="store_true")
    p.add_argument("--no-unrolled", action="store_true",
                   help="skip the unrolled-inference (forward + reverse) measurement")
    p.add_argument("--unrolled-only", action="store_true")
    p.add_argument("--setup-only", action="store_true",
                   help="time only the step-size constant of the benchmark instance (profiling)")
    p.add_argument("--batch", type=int, default=1,
                   help="instances per GPU (1 = the benchmark workload; >1 for profiling captures)")
    return p.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replica_seeds(rank: int, batch: int) -> list[int]:
    """Seeds of the instances a rank solves: replicas draw disjoint instances
    of the same recipe (weak scaling: the work per rank is fixed)."""
    return [SEED + rank * batch + b for b in range(batch)]


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The slowest rank's time (the job finishes when it does)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, seconds: float, world: int) -> float:
    """Whole-job rate: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / seconds


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# -- clocks ------------------------------------------------------------------

CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="proxmf_clocks_", suffix=".csv")
        os.close(fd)

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={CLOCK_QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "25", "-i", str(self.gpu)], stdout=self.f, stderr=subprocess.DEVNULL)
            # start timing only once the sampler is producing lines
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < 5.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.01)
        except Exception:  # noqa: BLE001 - clocks are best effort
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:  # noqa: BLE001
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# -- oracle baselines ----------------------------------------------------------

def oracle_model(side: int, seed: int = SEED):
    """The FP64 oracle's model of a side x side instance of the timed recipe."""
    import oracle
    from paper_1511_06103_gb300 import synth
    d = synth.segmentation_grid(H=side, W=side, L=L, conn=CONN, seed=seed)
    return oracle.Model.grid(d["U"].astype(np.float64), d["mu"].astype(np.float64),
                             d["w"].astype(np.float64), side, side, CONN)


def oracle_solve_rate(side: int, iters: int, seed: int = SEED, model=None) -> tuple[float, float, dict]:
    """Time the FP64 oracle's parallel proximal solve (q^0, iters steps, F at
    every step) on a side x side instance of the same recipe."""
    m = oracle_model(side, seed) if model is None else model
    eta = 0.04
    t0 = time.perf_counter()
    m.parallel_prox(eta, iters)
    dt = time.perf_counter() - t0
    units = side * side * L * iters
    return units / dt, dt, {"side": side, "iters": iters}


def run_reference(args, world, rank):
    """The oracle timed as it stands on the host cores, on the benchmark's own
    workload: every step is one full 512 x 512 solve of 100 iterations (about
    8.5 s on 16 cores)."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    side, iters = H, ITERS
    m = oracle_model(side)
    for _ in range(args.warmup):
        oracle_solve_rate(side, iters, model=m)
    times = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, dt, _ = oracle_solve_rate(side, iters, model=m)
        times.append(dt)
    wall = time.perf_counter() - t0
    units = side * side * L * iters * args.steps
    value = units / sum(times)
    cores = oracle.num_threads()
    sample = (f"the full workload: one {side}x{side} instance of the same recipe (L=21, 8-connected, seed {SEED}) "
              f"per step, {iters} iterations, F evaluated every iteration")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "H": H, "W": W, "L": L, "conn": CONN, "iters": ITERS,
                   "reference": "FP64 CPU oracle (plain C, OpenMP)", "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


# -- our arm -------------------------------------------------------------------

# dram__bytes_read.sum + dram__bytes_write.sum of the headline step kernel per
# instance-launch, from the ncu capture summarised in the named profile (4
# instances per launch, larger than L2, divided by 4), with the SHA-256 of the
# kernel's source files the counters were taken on.  Once a source changes the
# line reports traffic null (the counters no longer describe the kernel).
GRID_KERNEL = "grid_tma2_step_kernel<21,8>"
GRID_TRAFFIC = {"per_instance": (218290176 + 71568640) // 4,
                "sources": ["paper_1511_06103_gb300/csrc/grid_tma.cuh",
                            "paper_1511_06103_gb300/csrc/grid_step.cuh",
                            "paper_1511_06103_gb300/csrc/f32x2.cuh",
                            "paper_1511_06103_gb300/csrc/tc_common.cuh",
                            "paper_1511_06103_gb300/csrc/dfloat.cuh"],
                "sha256": "73dd5eb780e0ef8ff218d6c5f1e5923be40c39961b95d05ad1a1945407eb6218",
                "profile": "profiles/grid_prox_step_seg512_L21_conn8.md"}


def grid_sources_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in GRID_TRAFFIC["sources"]:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def grid_traffic(batch: int):
    """(traffic per launch or None, note) for the roofline object."""
    if GRID_TRAFFIC["per_instance"] is None or grid_sources_sha() != GRID_TRAFFIC["sha256"]:
        return None, (f"null: the step kernel's sources changed since the ncu capture of "
                      f"{GRID_TRAFFIC['profile']}")
    return batch * GRID_TRAFFIC["per_instance"], (
        f"dram read+write of one launch per instance from the ncu capture in {GRID_TRAFFIC['profile']} "
        "(4 instances per launch, larger than L2, divided by 4); kernel sources unchanged since (SHA-256)")


def algorithmic_bytes_per_launch() -> int:
    """One grid-step launch reads log q and U and writes log q (4 B each per
    variable-label) and reads the n_dirs edge-weight planes (4 B per pixel each)."""
    nd = 4 if CONN == 8 else 2
    return 12 * H * W * L + 4 * nd * H * W


DENSE_SIDE, DENSE_L, DENSE_ITERS = 96, 21, 30


# Exponentials per second of the special-function unit: 16 results per clock
# per SM (CUDA's throughput table for the base-2 exponential) x 152 SMs x the
# 2070 MHz maximum SM clock.  The bound of the dense step that computes K in
# the kernel (one exponential per weight).
EX2_PEAK_G = 16 * 152 * 2070e6 / 1e9


def run_dense(args, dev, precision, peak, fly=False):
    """Fully connected Gaussian CRF, N = 96 x 96 = 9216, L = 21, 30 iterations:
    device-timed solves (q^0, 30 steps, final F) with the model resident.
    fly: the BF16 tensor-core steps compute K in the kernel (no K bytes read)."""
    import torch

    from paper_1511_06103_gb300 import binding, synth
    d = synth.dense_gaussian(side=DENSE_SIDE, L=DENSE_L)
    stream = torch.cuda.current_stream(dev)
    crf = binding.CRF(binding.CRF_DENSE_GAUSS, DENSE_L, DENSE_SIDE, DENSE_SIDE, precision=precision,
                      stream=stream.cuda_stream)
    if fly:
        crf.dense_on_the_fly(True)
    crf.set_unary(torch.from_numpy(d["U"]).to(dev))
    crf.set_pairwise(torch.from_numpy(d["mu"]).to(dev), torch.from_numpy(d["feats"]).to(dev),
                     theta=np.array(d["theta"], np.float32))
    lam, eta = crf.lipschitz()
    # the BF16 form spends the last `refine` of the 30 iterations in FP32
    refine = 2 if precision == binding.CRF_BF16 else 0
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step():
        crf.iterate(DENSE_ITERS - refine, eta=0.0, reset=True, final_free_energy=True, refine_fp32=refine)

    for _ in range(max(1, args.warmup)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    crf.profile(True)
    times, kern = [], []
    n = max(3, min(args.steps, 10))
    for _ in range(n):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        ms, launches = crf.profile_read()
        kern.append(ms / launches)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    crf.profile(False)
    F = float(crf.free_energy()[0])
    q = crf.marginals()
    # the step kernel of this form alone (no FP32 refinement launches in the
    # average): the roofline's launch time
    kern_only = []
    if refine:
        crf.profile(True)
        for _ in range(n):
            flush.zero_()
            crf.iterate(DENSE_ITERS, eta=0.0, reset=True, refine_fp32=0)
            ms, launches = crf.profile_read()
            kern_only.append(ms / launches)
        crf.profile(False)
    crf.close()
    N = DENSE_SIDE * DENSE_SIDE
    ms_step = float(np.mean(times))
    iters = DENSE_ITERS
    kbytes = N * N * (2 if precision == binding.CRF_BF16 else 4)
    kms_all = float(np.mean(kern))
    kms = float(np.mean(kern_only)) if kern_only else kms_all
    if fly:
        # N^2 weights, one exponential each, per launch
        gexp = N * N / (kms / 1000.0) / 1e9
        roof = {"bound": "alu", "achieved": gexp, "peak": EX2_PEAK_G, "unit": "Gexp/s",
                "frac": gexp / EX2_PEAK_G, "exp_per_launch": N * N, "hbm_bytes_of_K": 0,
                "note": "K computed in the kernel: bound by the base-2 exponentials of the special-function "
                        "unit (peak: 16 per clock per SM x 152 SMs x 2070 MHz); launch time of the step kernel "
                        "alone"}
        return {"value": N * DENSE_L * iters / (ms_step / 1000.0), "unit": UNIT, "ms_per_solve": ms_step,
                "iters": DENSE_ITERS, "refine_fp32": refine, "avg_launch_ms": kms,
                "avg_launch_ms_with_refine": kms_all, "roofline": roof, "final_F": F, "eta": float(eta[0]),
                "Lambda": float(lam[0]), "q": q}
    return {"value": N * DENSE_L * iters / (ms_step / 1000.0), "unit": UNIT, "ms_per_solve": ms_step,
            "iters": DENSE_ITERS, "refine_fp32": refine, "avg_launch_ms": kms, "avg_launch_ms_with_refine": kms_all,
            "roofline": {"bound": "hbm", "achieved": kbytes / (kms / 1000.0) / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": kbytes / (kms / 1000.0) / 1e9 / peak,
                         "bytes_per_launch": kbytes,
                         "note": "K streamed once per iteration; launch time of this form's step kernel "
                                 "alone (the BF16 form's FP32 refinement launches are timed apart)"},
            "final_F": F, "eta": float(eta[0]), "Lambda": float(lam[0]), "q": q}


def run_grid_precision(args, dev, peak):
    """The segmentation workload solved by the FP32 form (100 steps) and by
    the BF16 tensor-core form (98 tensor-core steps + 2 FP32 refinement
    steps) at the same step size; device-timed solves, L2 flushed before
    each, average step launch from the profiled loop."""
    import torch

    from paper_1511_06103_gb300 import binding, synth
    d = synth.segmentation_grid(H=H, W=W, L=L, conn=CONN, seed=SEED)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    out = {}
    for name, prec, iters, refine in (("f32", binding.CRF_FP32, ITERS, 0),
                                      ("bf16_tc", binding.CRF_BF16, ITERS - 2, 2)):
        crf = binding.CRF(binding.CRF_GRID8, L, H, W, precision=prec, stream=stream.cuda_stream)
        crf.set_unary(torch.from_numpy(d["U"]).to(dev))
        crf.set_pairwise(torch.from_numpy(d["mu"]).to(dev), torch.from_numpy(d["w"]).to(dev))
        crf.lipschitz()

        def solve():
            crf.iterate(iters, eta=0.0, reset=True, final_free_energy=True, refine_fp32=refine)

        for _ in range(max(3, args.warmup)):
            flush.zero_()
            solve()
        torch.cuda.synchronize()
        times, kern = [], []
        crf.profile(True)
        for _ in range(max(3, min(args.steps, 10))):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solve()
            e1.record(stream)
            ms, n = crf.profile_read()
            kern.append(ms / n)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        crf.profile(False)
        ms = float(np.mean(times))
        kms = float(np.mean(kern))
        bl = algorithmic_bytes_per_launch()
        out[name] = {"value": H * W * L * ITERS / (ms / 1000.0), "unit": UNIT, "ms_per_solve": ms,
                     "tc_steps": iters if refine else 0, "fp32_steps": refine if refine else iters,
                     "avg_launch_ms": kms,
                     "roofline": {"bound": "hbm", "achieved": bl / (kms / 1000.0) / 1e9, "peak": peak,
                                  "unit": "GB/s", "frac": bl / (kms / 1000.0) / 1e9 / peak,
                                  "bytes_per_launch": bl},
                     "final_F": float(crf.free_energy()[0]), "q": crf.marginals()}
        crf.close()
    # the same comparison across label counts (step launch time, 100 steps)
    sweep = {}
    for Ls in (8, 16, 24, 32):
        ds = synth.segmentation_grid(H=H, W=W, L=Ls, conn=CONN, seed=SEED)
        row = {}
        for name, prec, iters, refine in (("f32", binding.CRF_FP32, ITERS, 0), ("bf16_tc", binding.CRF_BF16, ITERS - 2, 2)):
            crf = binding.CRF(binding.CRF_GRID8, Ls, H, W, precision=prec, stream=stream.cuda_stream)
            crf.set_unary(torch.from_numpy(ds["U"]).to(dev))
            crf.set_pairwise(torch.from_numpy(ds["mu"]).to(dev), torch.from_numpy(ds["w"]).to(dev))
            crf.lipschitz()
            for _ in range(2):
                crf.iterate(iters, eta=0.0, reset=True, refine_fp32=refine)
            crf.profile(True)
            ks = []
            for _ in range(3):
                flush.zero_()
                crf.iterate(iters, eta=0.0, reset=True, refine_fp32=refine)
                ms, n = crf.profile_read()
                ks.append(ms / n)
            crf.profile(False)
            row[name + "_launch_us"] = 1000.0 * float(np.mean(ks))
            crf.close()
        row["bf16_speedup"] = row["f32_launch_us"] / row["bf16_tc_launch_us"]
        sweep[str(Ls)] = row
    out["label_sweep"] = sweep
    q32, q16 = out["f32"].pop("q"), out["bf16_tc"].pop("q")
    return {"workload": WORKLOAD + "; FP32 form vs BF16 tensor-core messages (98 + 2 FP32 refinement steps)",
            **out, "bf16_speedup": out["bf16_tc"]["value"] / out["f32"]["value"],
            "final_F_rel_diff": abs(out["bf16_tc"]["final_F"] - out["f32"]["final_F"]) / abs(out["f32"]["final_F"]),
            "q_max_abs_diff": float(np.abs(q32 - q16).max())}


def run_denoising(args, dev):
    """Binary denoising CRF, 64 x 64, L = 2, 4-connected, 50 steps at the
    step-size constant: device time per solve with the whole loop in one
    cluster launch (the default), with one launch per step replayed as a
    CUDA graph, and with launches issued one by one."""
    import torch

    from paper_1511_06103_gb300 import binding, synth
    d = synth.binary_denoising()
    stream = torch.cuda.current_stream(dev)
    out = {}
    for mode in ("resident", "graph", "eager"):
        crf = binding.CRF(binding.CRF_GRID4, 2, 64, 64, stream=stream.cuda_stream)
        crf.use_resident(mode == "resident")
        crf.use_graphs(mode == "graph")
        crf.set_unary(torch.from_numpy(d["U"]).to(dev))
        crf.set_pairwise(torch.from_numpy(d["mu"]).to(dev), torch.from_numpy(d["w"]).to(dev))
        _, eta = crf.lipschitz()

        def solve():
            crf.iterate(50, eta=0.0, reset=True, final_free_energy=True)

        for _ in range(max(3, args.warmup)):
            solve()
        torch.cuda.synchronize()
        n = 50
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        for _ in range(n):
            solve()
        e1.record(stream)
        torch.cuda.synchronize()
        wall = (time.perf_counter() - t0) / n
        ms = e0.elapsed_time(e1) / n
        out[mode] = {"us_per_solve": 1000.0 * ms, "host_us_per_solve": 1e6 * wall,
                     "value": 64 * 64 * 2 * 50 / (ms / 1000.0), "unit": UNIT,
                     "final_F": float(crf.free_energy()[0])}
        crf.close()
    return {"workload": "binary denoising CRF 64x64, L=2, 4-connected, 50 parallel proximal steps at "
                        "eta = 1/(1+Lambda) (0.2383), back-to-back solves", "eta": float(eta[0]), **out}


ETA_GRID = [float(x) for x in np.logspace(-2.5, 0.0, 11)]


def run_eta_sweep(args, dev):
    """Sensitivity to the step parameter (the synthetic counterpart of the
    paper's comparison of OURS-FIXED / OURS-ADAPTIVE with ADHOC over
    eta = 1/(1+d)): final F after a fixed number of steps for each eta of a
    log grid, on the binary denoising model and on the segmentation grid.
    Lower F (= KL up to log Z) is better."""
    import torch

    from paper_1511_06103_gb300 import binding, synth
    stream = torch.cuda.current_stream(dev)
    out = {"eta": ETA_GRID}
    cases = (("denoising_64x64_L2", synth.binary_denoising(), binding.CRF_GRID4, 50),
             ("segmentation_512x512_L21", synth.segmentation_grid(H=H, W=W, L=L, conn=CONN, seed=SEED),
              binding.CRF_GRID8, ITERS))
    for name, d, topo, iters in cases:
        crf = binding.CRF(topo, d["L"], d["H"], d["W"], stream=stream.cuda_stream)
        crf.set_unary(torch.from_numpy(d["U"]).to(dev))
        crf.set_pairwise(torch.from_numpy(d["mu"]).to(dev), torch.from_numpy(d["w"]).to(dev))
        lam, eta_c = crf.lipschitz()
        res = {"iters": iters, "eta_constant": float(eta_c[0]), "fixed": [], "adhoc": []}
        if d["L"] == 2:
            res["adaptive"] = []
        for e in ETA_GRID:
            crf.iterate(iters, eta=e, reset=True, final_free_energy=True)
            res["fixed"].append(float(crf.free_energy()[0]))
            crf.iterate(iters, eta=e, reset=True, final_free_energy=True, rule=binding.MF_RULE_ADHOC)
            res["adhoc"].append(float(crf.free_energy()[0]))
            if d["L"] == 2:
                crf.iterate(iters, reset=True, final_free_energy=True, rule=binding.MF_RULE_ADAPTIVE,
                            d=max(1.0 / e - 1.0, 1e-6))
                res["adaptive"].append(float(crf.free_energy()[0]))
        crf.iterate(iters, eta=0.0, reset=True, final_free_energy=True)
        res["F_at_eta_constant"] = float(crf.free_energy()[0])
        for k in ("fixed", "adhoc", "adaptive"):
            if k in res:
                res[k + "_spread"] = max(res[k]) - min(res[k])
        out[name] = res
        crf.close()
    return out


def run_sparse(args, dev, peak):
    """General pairwise graphs from edge lists: a random graph with the
    segmentation grid's size and degree (N = 262144, 4N edges, L = 21,
    symmetric mu) and DBN-shaped bipartite layers (4096 + 8192 variables,
    fan-out 64, L = 2); 100 steps at the automatic (degree-bound) step,
    device-timed solves, average step launch from the profiled loop."""
    import torch

    from paper_1511_06103_gb300 import binding, synth
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    out = {}
    for name, d in (("random_N262144_E1048576_L21", synth.random_graph(262144, 4 * 262144, 21, seed=31)),
                    ("dbn_4096x8192_fan64_L2", synth.dbn_layers(4096, 8192, 64, 2, seed=32))):
        crf = binding.CRF(binding.CRF_SPARSE, d["L"], d["N"], 1, stream=stream.cuda_stream)
        crf.set_unary(torch.from_numpy(d["U"]).to(dev))
        crf.set_graph(d["mu"], d["src"], d["dst"], d["w"])
        lam, eta = crf.lipschitz()

        def solve():
            crf.iterate(ITERS, eta=0.0, reset=True, final_free_energy=True)

        for _ in range(max(3, args.warmup)):
            flush.zero_()
            solve()
        torch.cuda.synchronize()
        times, kern = [], []
        crf.profile(True)
        for _ in range(max(3, min(args.steps, 10))):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solve()
            e1.record(stream)
            ms, n = crf.profile_read()
            kern.append(ms / n)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        crf.profile(False)
        N, Lc = d["N"], d["L"]
        adj = 2 * d["src"].size          # adjacency entries (both directions)
        # per step: own log q, U, q read + log q, q written (5 x 4L per
        # variable); per adjacency entry: column and weight (8 B) and the
        # neighbour's q row (4L)
        bl = N * 20 * Lc + adj * (8 + 4 * Lc)
        ms = float(np.mean(times))
        kms = float(np.mean(kern))
        out[name] = {"value": N * Lc * ITERS / (ms / 1000.0), "unit": UNIT, "ms_per_solve": ms,
                     "avg_launch_ms": kms, "Lambda_bound": float(lam[0]), "eta": float(eta[0]),
                     "roofline": {"bound": "hbm", "achieved": bl / (kms / 1000.0) / 1e9, "peak": peak,
                                  "unit": "GB/s", "frac": bl / (kms / 1000.0) / 1e9 / peak, "bytes_per_launch": bl,
                                  "kernel": "sparse_step_kernel"},
                     "final_F": float(crf.free_energy()[0])}
        crf.close()
    return out


UNR_B, UNR_SIDE, UNR_L, UNR_CONN, UNR_K = 16, 256, 21, 4, 10


def run_unrolled(args, dev, peak, precision=0):
    """Training step through K = 10 unrolled proximal steps on a batch of 16
    4-connected 256 x 256 grids, L = 21: forward with per-step checkpoints,
    export of log q^K, cross-entropy gradient, reverse pass to dU, dmu, dw.
    Inputs resident on the device; the 1.1 GB of checkpoints exceed L2."""
    import torch

    from paper_1511_06103_gb300 import binding, synth
    d = synth.unrolled_batch(B=UNR_B, H=UNR_SIDE, W=UNR_SIDE, L=UNR_L, conn=UNR_CONN)
    B, N, L, K = UNR_B, UNR_SIDE * UNR_SIDE, UNR_L, UNR_K
    stream = torch.cuda.current_stream(dev)
    crf = binding.CRF(binding.CRF_GRID4, L, UNR_SIDE, UNR_SIDE, batch=B, precision=precision,
                      stream=stream.cuda_stream)
    crf.set_unary(torch.from_numpy(d["U"]).to(dev))
    crf.set_pairwise(torch.from_numpy(d["mu"]).to(dev), torch.from_numpy(d["w"]).to(dev))
    lam, eta_b = crf.lipschitz()
    eta = float(np.min(eta_b))         # one step for the batch
    ckpt = torch.empty(crf.checkpoint_floats(K), dtype=torch.float32, device=dev)
    logq = torch.empty((B, N, L), dtype=torch.float32, device=dev)
    y = torch.from_numpy(d["y"].astype(np.int64)).to(dev)
    g = torch.empty_like(logq)
    dU = torch.empty_like(logq)
    dmu = torch.empty((L, L), dtype=torch.float32, device=dev)
    dw = torch.empty((B, 2, UNR_SIDE, UNR_SIDE), dtype=torch.float32, device=dev)
    scale = -1.0 / (B * N)

    def step(prof=None):
        crf.unrolled_forward(K, eta, ckpt)
        if prof is not None:
            prof.append(crf.profile_read())
        crf.log_marginals(logq)
        g.zero_()
        g.scatter_(2, y[:, :, None], scale)
        crf.unrolled_backward(K, eta, ckpt, g, dU, dmu, dw)
        if prof is not None:
            prof.append(crf.profile_read())

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    times = []
    n = max(3, min(args.steps, 10))
    for _ in range(n):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    # per-step device times of the two loops (a separate pass: reading the
    # loop events waits on the host between forward and reverse)
    crf.profile(True)
    fwd, bwd = [], []
    for _ in range(n):
        prof = []
        step(prof)
        fwd.append(prof[0][0] / prof[0][1])
        bwd.append(prof[1][0] / prof[1][1])
    crf.profile(False)
    loss = float(-(logq.gather(2, y[:, :, None])).mean().item())
    launches = crf.launch_count()
    crf.close()
    ms = float(np.mean(times))
    fwd_ms, bwd_ms = float(np.mean(fwd)), float(np.mean(bwd))
    # algorithmic bytes of one reverse step, per pixel: read d/ds^{t+1},
    # log q^{t+1}, log q^t, dU, w, dw; write d/ds^t, dU, dw
    bwd_bytes = B * N * (24 * L + 12 * 2)
    fwd_bytes = B * N * (12 * L + 4 * 2)
    return {"workload": "unrolled inference, batch 16 of 4-connected 256x256 grids, L=21, K=10, "
                        + ("BF16 tensor-core messages" if precision else "FP32 messages")
                        + "; forward with per-step checkpoints + cross-entropy gradient + "
                        "reverse pass to dU, dmu, dw (FP32)",
            "value": B * N * L * K / (ms / 1000.0), "unit": "updates/s (forward + reverse per update)",
            "train_steps_per_s": 1000.0 / ms, "ms_per_train_step": ms,
            "forward_step_ms": fwd_ms, "reverse_step_ms": bwd_ms, "eta": eta, "loss": loss,
            "roofline_reverse": {"bound": "hbm", "achieved": bwd_bytes / (bwd_ms / 1000.0) / 1e9,
                                 "peak": peak, "unit": "GB/s",
                                 "frac": bwd_bytes / (bwd_ms / 1000.0) / 1e9 / peak,
                                 "bytes_per_step": bwd_bytes,
                                 "kernel": "adj_step_kernel<21,4,sym>"},
            "roofline_forward": {"bound": "hbm", "achieved": fwd_bytes / (fwd_ms / 1000.0) / 1e9,
                                 "peak": peak, "unit": "GB/s",
                                 "frac": fwd_bytes / (fwd_ms / 1000.0) / 1e9 / peak,
                                 "bytes_per_step": fwd_bytes, "kernel": "grid_tma2_step_kernel<21,4>"},
            "launches_total": int(launches)}


SERVE_SIZES = (64, 86, 116, 156, 210, 283, 380, 512)   # log-uniform sides in [64, 512], quantised


def serving_requests(n, seed=7, variants=4):
    """n requests: square side log-uniform in [64, 512] (quantised to 8 sizes
    so edge weights can be reused), L in {2, 8, 21}; L = 2 uses the binary
    denoising recipe, L = 8 and 21 the segmentation recipe.  Unaries are drawn
    `variants` times per (side, L) class and reused in turn (every request is
    still solved in full; the cap only bounds host memory and set-up time)."""
    from paper_1511_06103_gb300 import synth
    rng = np.random.default_rng(seed)
    cache, unaries, turn = {}, {}, {}
    out = []
    for _ in range(n):
        side = SERVE_SIZES[int(rng.integers(0, len(SERVE_SIZES)))]
        L = int(rng.choice([2, 8, 21]))
        key = (side, L)
        if key not in cache:
            if L == 2:
                cache[key] = synth.binary_denoising(H=side, W=side, seed=1000 + side)
            else:
                cache[key] = synth.segmentation_grid(H=side, W=side, L=L, conn=8, seed=2000 + side + L)
            unaries[key] = []
            turn[key] = 0
        base = cache[key]
        if L == 2:
            U = base["U"]
        else:
            k = turn[key] % variants
            turn[key] += 1
            if k == len(unaries[key]):
                unaries[key].append(np.ascontiguousarray(
                    synth.unary_from_logits(rng.normal(0.0, 2.0, size=(side * side, L))), np.float32))
            U = unaries[key][k]
        out.append(dict(base, U=U))
    return out


def run_serving(n_req, max_iters=1000, rel_tol=1e-6, sample=1024):
    """Continuous batching with Poisson arrivals at 0.8x (and 0.5x) the
    saturated rate; p50/p99 latency (arrival to result) and throughput over
    all n_req requests.  The saturated rate and the one-at-a-time comparison
    are measured on the first `sample` requests (sizes and label counts are
    drawn independently, so the sample has the stream's mix)."""
    from paper_1511_06103_gb300 import binding
    reqs = serving_requests(n_req)
    budget = 16 << 30
    sample = min(sample, len(reqs))

    def drive(srv, subset, arrivals, iters_per_step=4):
        t0 = time.perf_counter()
        sub, lat, done_iters = {}, {}, {}
        pending = []
        i = 0
        while len(lat) < len(subset):
            now = time.perf_counter() - t0
            while i < len(subset) and arrivals[i] <= now:
                d = subset[i]
                t = srv.submit(d["U"], d["mu"], d["w"], d["H"], d["W"], d["conn"], eta=0.0, max_iters=max_iters,
                               rel_tol=rel_tol)
                sub[t] = time.perf_counter()
                pending.append((t, i))
                i += 1
            srv.step(iters_per_step)
            still = []
            for t, k in pending:
                st, _, it, _ = srv.poll(t)
                if st == 2:
                    lat[t] = time.perf_counter() - sub[t]
                    done_iters[k] = it
                else:
                    still.append((t, k))
            pending = still
            if i < len(subset) and not pending:
                time.sleep(max(0.0, min(0.001, arrivals[i] - (time.perf_counter() - t0))))
        srv.sync()
        return time.perf_counter() - t0, lat, done_iters

    head = reqs[:sample]
    with binding.Server(budget, max_slots=128) as srv:          # saturated: all at once
        t_sat, _, _ = drive(srv, head, [0.0] * len(head))
    sat_rps = len(head) / t_sat
    rate = 0.8 * sat_rps
    arrivals = np.cumsum(np.random.default_rng(11).exponential(1.0 / rate, size=len(reqs)))
    with binding.Server(budget, max_slots=128) as srv:
        t_run, lat, iters_run = drive(srv, reqs, arrivals)
    # the same requests at half the saturated rate
    rate_half = 0.5 * sat_rps
    arrivals_half = np.cumsum(np.random.default_rng(12).exponential(1.0 / rate_half, size=len(reqs)))
    with binding.Server(budget, max_slots=128) as srv:
        t_half, lat_half, _ = drive(srv, reqs, arrivals_half)
    ms_half = np.array(sorted(lat_half.values())) * 1000
    upd = sum(r["H"] * r["W"] * r["L"] * iters_run[k] for k, r in enumerate(reqs))
    upd_head = sum(r["H"] * r["W"] * r["L"] * iters_run[k] for k, r in enumerate(head))
    t1 = time.perf_counter()
    with binding.Server(budget, max_slots=1) as srv:           # one at a time
        for d in head:
            t = srv.submit(d["U"], d["mu"], d["w"], d["H"], d["W"], d["conn"], eta=0.0, max_iters=max_iters,
                           rel_tol=rel_tol)
            while srv.poll(t)[0] != 2:
                srv.step(8)
        srv.sync()
    t_one = time.perf_counter() - t1
    ms = np.array(sorted(lat.values())) * 1000
    return {"workload": f"{len(reqs)} grid-CRF requests, square side log-uniform in [64,512] (8 sizes), "
                        "L in {2,8,21}, Poisson arrivals at 0.8x (and 0.5x) the saturated rate, retirement at "
                        "dF/|F| <= 1e-6 or 1000 steps, step size from the degree bound; one launch per iteration "
                        "advances every request in flight; 4 unary draws per (side, L) class, reused in turn",
            "requests": len(reqs), "arrival_rate_rps": rate, "run_s": t_run,
            "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)),
                           "mean": float(ms.mean())},
            "throughput_rps": len(reqs) / t_run, "updates_per_s": upd / t_run,
            "saturated": {"requests": len(head), "s": t_sat, "throughput_rps": sat_rps,
                          "updates_per_s": upd_head / t_sat},
            "one_at_a_time": {"requests": len(head), "s": t_one, "throughput_rps": len(head) / t_one,
                              "updates_per_s": upd_head / t_one},
            "half_load": {"arrival_rate_rps": rate_half, "run_s": t_half,
                          "latency_ms": {"p50": float(np.percentile(ms_half, 50)),
                                         "p99": float(np.percentile(ms_half, 99)), "mean": float(ms_half.mean())},
                          "throughput_rps": len(reqs) / t_half},
            "mean_iters": float(np.mean(list(iters_run.values())))}


def run_setup(args, dev, stream):
    """The step-size constant of the benchmark instance alone (step a7), as a
    user pays it for every new pairwise term; warmup + steps repetitions."""
    import torch

    from paper_1511_06103_gb300 import binding, synth
    d = synth.segmentation_grid(H=H, W=W, L=L, conn=CONN, seed=SEED)
    crf = binding.CRF(binding.CRF_GRID8, L, H, W, stream=stream.cuda_stream)
    crf.set_unary(torch.from_numpy(d["U"][None]).to(dev))
    mu_d = torch.from_numpy(d["mu"]).to(dev)
    w_d = torch.from_numpy(d["w"][None]).to(dev)
    times, launches = [], []
    lam = None
    for i in range(args.warmup + args.steps):
        crf.set_pairwise(mu_d, w_d)
        torch.cuda.synchronize()
        n0 = crf.launch_count()
        t0 = time.perf_counter()
        lam, _ = crf.lipschitz()     # returns host values: synchronises
        if i >= args.warmup:
            times.append(1000 * (time.perf_counter() - t0))
            launches.append(crf.launch_count() - n0)
    crf.close()
    return {"workload": "step-size constant (Lanczos on the 512x512 8-connected weights, label-space "
                        "eigen-solve of mu, L=21)", "ms_median": statistics.median(times),
            "ms_min": min(times), "launches": launches[-1], "Lambda": float(lam[0]), "reps": len(times)}


def run_ours(args, world, rank, local):
    import torch
    import torch.distributed as dist

    from paper_1511_06103_gb300 import binding, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    torch.cuda.init()
    stream = torch.cuda.current_stream(dev)
    if args.serve_only:
        print(json.dumps({"serving": run_serving(max(1, args.serve_requests))}), flush=True)
        return
    if args.sparse_only:
        peak, _ = measured_peaks()
        print(json.dumps({"sparse": run_sparse(args, dev, peak)}), flush=True)
        return
    if args.eta_sweep_only:
        print(json.dumps({"eta_sweep": run_eta_sweep(args, dev)}), flush=True)
        return
    if args.denoising_only:
        print(json.dumps({"denoising": run_denoising(args, dev)}), flush=True)
        return
    if args.grid_bf16_only:
        peak, _ = measured_peaks()
        print(json.dumps({"grid_precision": run_grid_precision(args, dev, peak)}), flush=True)
        return
    if args.unrolled_only:
        peak, _ = measured_peaks()
        print(json.dumps({"unrolled": {"f32": run_unrolled(args, dev, peak),
                                       "bf16_tc": run_unrolled(args, dev, peak, 1)}}), flush=True)
        return
    if args.setup_only:
        print(json.dumps({"setup": run_setup(args, dev, stream)}), flush=True)
        return
    if args.dense_only:
        peak, _ = measured_peaks()
        for prec, fly in ((binding.CRF_FP32, False), (binding.CRF_BF16, False), (binding.CRF_BF16, True)):
            r = run_dense(args, dev, prec, peak, fly)
            r.pop("q")
            print(json.dumps({"dense_precision": ("bf16" if prec else "f32") + ("_K_in_kernel" if fly else ""),
                              **r}), flush=True)
        return
    B = args.batch
    ds = [synth.segmentation_grid(H=H, W=W, L=L, conn=CONN, seed=sd) for sd in replica_seeds(rank, B)]
    d = ds[0]
    U = torch.from_numpy(np.stack([x["U"] for x in ds])).to(dev)
    mu = torch.from_numpy(d["mu"]).to(dev)
    wts = torch.from_numpy(np.stack([x["w"] for x in ds])).to(dev)
    crf = binding.CRF(binding.CRF_GRID8, L, H, W, batch=B, stream=stream.cuda_stream)
    crf.set_unary(U)
    crf.set_pairwise(mu, wts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n0 = crf.launch_count()
    lam, eta = crf.lipschitz()           # a7: step-size constant, once per model
    setup_ms = 1000 * (time.perf_counter() - t0)
    setup_launches = crf.launch_count() - n0
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step():
        crf.iterate(ITERS, eta=0.0, reset=True, final_free_energy=True)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    crf.profile(True)
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    loop_ms = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = crf.launch_count()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
    gpu_index = int(vis[local]) if len(vis) > local and vis[local].isdigit() else local
    with ClockSampler(gpu_index) as clk:
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            ev_s[k].record(stream)
            step()
            ev_e[k].record(stream)
            ms, n = crf.profile_read()
            loop_ms.append(ms / n)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        wall1 = time.perf_counter()
    launches = crf.launch_count() - launches0
    crf.profile(False)
    step_ms = [ev_s[k].elapsed_time(ev_e[k]) for k in range(args.steps)]
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    units_per_step = B * H * W * L * ITERS
    value = job_throughput(units_per_step * args.steps, total_ms / 1000.0, world)
    F_final = float(crf.free_energy()[0])
    kern_ms = float(np.mean(loop_ms))
    peak, peak_kind = measured_peaks()
    bytes_launch = B * algorithmic_bytes_per_launch()
    achieved = bytes_launch / (kern_ms / 1000.0) / 1e9

    # end to end through the public API with host buffers: upload U and the
    # pairwise term, solve (the step-size constant is recomputed because the
    # pairwise term changed), download q and F.
    e2e = None
    if not args.no_e2e:
        U_h = U.cpu().pin_memory()
        mu_h = mu.cpu().pin_memory()
        w_h = wts.cpu().pin_memory()
        q_h = torch.empty((B, H * W, L), dtype=torch.float32).pin_memory()
        n_e2e = max(3, min(args.steps, 10))

        def e2e_step():
            crf.set_unary(U_h)
            crf.set_pairwise(mu_h, w_h)
            crf.iterate(ITERS, eta=0.0, final_free_energy=True)
            crf.marginals(q_h)
            return crf.free_energy()

        e2e_step()
        times = []
        for _ in range(n_e2e):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_step()
            times.append(time.perf_counter() - t0)
        e2e_s = max_over_ranks(float(np.mean(times)), world, dev)

        # one more pass, synchronised between its phases (outside the timed loop)
        def phase_ms(f):
            torch.cuda.synchronize()
            t = time.perf_counter()
            f()
            torch.cuda.synchronize()
            return 1000 * (time.perf_counter() - t)

        flush.zero_()
        phases = {"upload_unary": phase_ms(lambda: crf.set_unary(U_h)),
                  "upload_pairwise": phase_ms(lambda: crf.set_pairwise(mu_h, w_h)),
                  "step_size_setup": phase_ms(lambda: crf.lipschitz()),
                  "iterations": phase_ms(lambda: crf.iterate(ITERS, eta=0.0, final_free_energy=True)),
                  "download": phase_ms(lambda: (crf.marginals(q_h), crf.free_energy()))}
        e2e = {"value": job_throughput(units_per_step, e2e_s, world), "unit": UNIT,
               "h2d_bytes_per_step": int(U_h.numel() * 4 + mu_h.numel() * 4 + w_h.numel() * 4),
               "d2h_bytes_per_step": int(q_h.numel() * 4 + 8),
               "ms_per_step": 1000 * e2e_s,
               "includes": "H2D of U and w, step-size constant (Lanczos), 100 iterations, D2H of q and F",
               "phases_ms": phases}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        # the whole instance of the timed workload (one solve, about 10 s of CPU work)
        side, iters = H, ITERS
        rate, dt, _ = oracle_solve_rate(side, iters)
        cpu = {"value": rate, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"one full {side}x{side} instance of the same recipe (L=21, 8-connected, seed {SEED}), "
                         f"{iters} iterations, F every iteration; {dt:.1f} s of CPU work"}

    clocks = clk.summary()
    dense = None
    if not args.no_dense and world == 1:
        r32 = run_dense(args, dev, binding.CRF_FP32, peak)
        r16 = run_dense(args, dev, binding.CRF_BF16, peak)
        rfly = run_dense(args, dev, binding.CRF_BF16, peak, fly=True)
        dq_fly = float(np.abs(r32["q"] - rfly.pop("q")).max())
        dq = float(np.abs(r32.pop("q") - r16.pop("q")).max())
        dense = {"workload": "fully connected Gaussian CRF, N=96x96=9216, L=21, 30 iterations "
                             "(theta_pos=3, theta_rgb=13), model resident; the BF16 form runs 28 "
                             "tensor-core steps and 2 FP32 refinement steps",
                 "f32": r32, "bf16_tc": r16, "bf16_speedup": r16["value"] / r32["value"],
                 "final_F_rel_diff": abs(r16["final_F"] - r32["final_F"]) / abs(r32["final_F"]),
                 "q_max_abs_diff": dq,
                 "bf16_tc_K_in_kernel": {**rfly,
                                         "speedup_vs_f32": rfly["value"] / r32["value"],
                                         "final_F_rel_diff_vs_f32": abs(rfly["final_F"] - r32["final_F"]) /
                                         abs(r32["final_F"]),
                                         "q_max_abs_diff_vs_f32": dq_fly}}
    denoise = None
    if not args.no_denoising and world == 1:
        denoise = run_denoising(args, dev)
    sparse = None
    if not args.no_sparse and world == 1:
        sparse = run_sparse(args, dev, peak)
    eta_sweep = None
    if not args.no_eta_sweep and world == 1:
        eta_sweep = run_eta_sweep(args, dev)
    grid_prec = None
    if not args.no_grid_bf16 and world == 1:
        grid_prec = run_grid_precision(args, dev, peak)
    unrolled = None
    if not args.no_unrolled and world == 1:
        unrolled = {"f32": run_unrolled(args, dev, peak), "bf16_tc": run_unrolled(args, dev, peak, 1)}
    serving = None
    if args.serve_requests > 0 and world == 1:
        serving = run_serving(args.serve_requests)
    traffic, traffic_note = grid_traffic(B)
    if rank == 0:
        srt = sorted(step_ms)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "H": H, "W": W, "L": L, "conn": CONN, "iters": ITERS,
                       "batch_per_gpu": B, "seed": SEED, "parallelism": "replicas" if world > 1 else "single",
                       "eta": float(eta[0]), "Lambda": float(lam[0]),
                       "l2": "flushed before every step (256 MiB write); within a solve the 70 MB working "
                             "set stays L2-resident across its 100 iterations"},
            "latency_ms": {"p50": float(np.percentile(srt, 50)), "p99": float(np.percentile(srt, 99))},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "traffic_note": traffic_note,
                         "kernel": GRID_KERNEL,
                         "bytes_per_launch": bytes_launch, "avg_launch_ms": kern_ms,
                         "peak_kind": peak_kind},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks,
            "setup_ms": setup_ms,
            "setup_launches": int(setup_launches),
            "final_F": F_final,
            "wall_ms_timed": 1000 * (wall1 - wall0),
            "dense": dense,
            "denoising": denoise,
            "eta_sweep": eta_sweep,
            "sparse": sparse,
            "grid_precision": grid_prec,
            "unrolled": unrolled,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    crf.close()


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    try:
        run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
