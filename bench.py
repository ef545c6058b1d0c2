"""Benchmark: the whole hot path of the semi-coherent track statistic on the
one-year workload (365 daily SFTs x 8641 bins, FP32 table, K = 6 power-law
basis, +-1-bin neighbours, 10^7 candidate tracks, top-128).

One step = rebuild the power table from device-resident strain (windowed
SFT + PSD normalisation), evaluate the statistic of every track, select the
top-k (and, on several GPUs, merge the per-rank top-k lists).  Prints one
JSON line.  ``--impl reference`` times the FP64 CPU oracle on the host cores
instead (a bounded sample of tracks per step).

Launch: ``python bench.py [--steps K --warmup W]`` or under torchrun with
``--gpus N`` (one rank per GPU; each rank evaluates its own 10^7 tracks).
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import multiprocessing as mp
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2510_20891_gb300 import synth  # noqa: E402

METRIC = "track-statistic evals/s (1-yr data) + % of L2/HBM gather roofline; served p50/p99"
UNIT = "evals/s"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="oneyear_daily_fp32")
    ap.add_argument("--tracks", type=int, default=0, help="override the track count per rank")
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "f16", "f8e4m3"])
    ap.add_argument("--topk", type=int, default=128)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=1 << 18)
    return ap.parse_args()


# --------------------------------------------------------------------------- inputs
def make_inputs(w, rank: int, n_tracks: int):
    """Seeded synthetic inputs of the workload (the same dataset on every rank,
    a different batch of candidate tracks per rank)."""
    rng = np.random.default_rng(w.seed)
    x, inj = synth.make_strain(w, rng)
    psd = synth.psd_bins(w.psd_fn(), w.n_bin, w.T_sft)
    F = synth.make_training_tracks(w, rng)
    return x, psd, F, inj, np.random.default_rng(1000 + rank)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", FALLBACK_HBM_GBS)), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("eval_kernel.cuh", "tfs_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2510_20891_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str, dtype: str):
    """DRAM bytes per launch of the statistic kernel from the committed ncu summary,
    if it was taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", f"eval_stat_kernel_{workload}_{dtype}.md")
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    mh = re.search(r"kernel source hash:\s*([0-9a-f]+)", txt)
    mt = re.search(r"dram bytes per full launch:\s*([0-9.e+]+)", txt)
    if not mh or not mt or mh.group(1) != kernel_source_hash():
        return None
    return float(mt.group(1))


class ClockSampler:
    """nvidia-smi samples of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                out, _ = self.p.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        else:
            self.lines = []

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except (ValueError, IndexError):
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- CPU oracle arm
_W = {}


def _oracle_init(P, V, T_sft, m):
    _W.update(P=P, V=V, T=T_sft, m=m)


def _oracle_chunk(coeffs):
    import oracle.tfstat_oracle as O

    S, *_ = O.eval_stat(_W["P"], _W["V"], coeffs, np.zeros(len(coeffs)), _W["T"], _W["m"], 0)
    return float(S.sum())


class OracleArm:
    """The oracle as it stands on the host cores: its FP64 SFT of the whole strain
    (one process) plus its statistic of a sample of tracks split over a spawn pool;
    the rate is the batch's tracks over (SFT time + batch x per-track time)."""

    def __init__(self, x, psd, w, V, ncores):
        import oracle.tfstat_oracle as O

        self.O, self.x, self.psd, self.w, self.V, self.ncores = O, x, psd, w, V, ncores
        P = O.power_table(x, w.dt, w.T_sft, psd)
        self.pool = mp.get_context("spawn").Pool(ncores, initializer=_oracle_init, initargs=(P, V, w.T_sft, w.m))
        self.pool.map(_oracle_chunk, [np.zeros((1, V.shape[0]))] * ncores)   # warm the workers

    def step(self, coeffs):
        w = self.w
        t0 = time.perf_counter()
        self.O.power_table(self.x, w.dt, w.T_sft, self.psd)
        t_sft = time.perf_counter() - t0
        t1 = time.perf_counter()
        self.pool.map(_oracle_chunk, np.array_split(coeffs, self.ncores * 4))
        return t_sft, time.perf_counter() - t1

    def close(self):
        self.pool.close()
        self.pool.join()


# --------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = synth.WORKLOADS[args.workload]
    N = args.tracks or w.n_tracks
    x, psd, F, inj, rng = make_inputs(w, 0, N)
    import oracle.tfstat_oracle as O

    V, s, cmin, cmax = O.svd_basis(F, w.K)
    ncores = os.cpu_count() or 1
    sample = min(args.cpu_sample, N)
    coeffs = synth.uniform_coeffs(sample, cmin, cmax, rng)
    arm = OracleArm(x, psd, w, V, ncores)
    rates = []
    for i in range(args.warmup + args.steps):
        t_sft, t_eval = arm.step(coeffs)
        step_s = t_sft + N * (t_eval / sample)
        if i >= args.warmup:
            rates.append(N / step_s)
    arm.close()
    value = float(statistics.median(rates))
    ms = 1e3 * N / value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "tracks_per_step": N, "n_seg": w.n_seg, "n_bin": w.n_bin,
                       "K": w.K, "m": w.m, "topk": args.topk},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncores, "kind": "oracle",
                             "sample": f"per step: FP64 SFT of the full strain + statistic of {sample} tracks "
                                       f"on {ncores} processes, scaled to {N} tracks"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    w = synth.WORKLOADS[args.workload]
    N = args.tracks or w.n_tracks

    ncores = os.cpu_count() or 1
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2510_20891_gb300 import build as B

    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    import paper_2510_20891_gb300 as T
    from paper_2510_20891_gb300.dist import allgather_topk

    L = T.lib()
    x, psd, F, inj, rng = make_inputs(w, rank, N)
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)

    x_d = torch.from_numpy(x).cuda()
    table = T.build_sfts(x_d, w.dt, w.T_sft, psd, "hann", args.dtype)
    basis = T.build_basis(F, w.K)
    U, sig, cmin, cmax = basis.to_host()
    coeffs_h = synth.uniform_coeffs(N, cmin, cmax, rng)
    coeffs_d = torch.from_numpy(coeffs_h).cuda()
    stat = torch.empty(N, dtype=torch.float32, device="cuda")
    kk = min(args.topk, N)
    top_i = torch.empty(kk, dtype=torch.int64, device="cuda")
    top_v = torch.empty(kk, dtype=torch.float32, device="cuda")

    def step(evs=None):
        if evs is not None:
            evs[0].record(stream)
        T.check(L.tfs_table_rebuild(table.handle, x_d.data_ptr(), x_d.numel(), 1, sp))
        if evs is not None:
            evs[1].record(stream)
        T.check(L.tfs_eval_stat(table.handle, basis.handle, coeffs_d.data_ptr(), None, N, w.m, 0,
                                stat.data_ptr(), None, None, None, 1, sp))
        if evs is not None:
            evs[2].record(stream)
        T.check(L.tfs_topk(stat.data_ptr(), N, kk, top_i.data_ptr(), top_v.data_ptr(), 1, sp))
        if evs is not None:
            evs[3].record(stream)
        if world > 1:
            allgather_topk(top_i, top_v, kk, rank * N)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = L.tfs_kernel_launches()
    with ClockSampler(local) as clk:
        start.record(stream)
        for i in range(args.steps):
            step(evs[i])
        end.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches = L.tfs_kernel_launches() - launches0
    total_ms = start.elapsed_time(end)
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    sft_ms = sum(e[0].elapsed_time(e[1]) for e in evs) / args.steps
    eval_ms = sum(e[1].elapsed_time(e[2]) for e in evs) / args.steps
    topk_ms = sum(e[2].elapsed_time(e[3]) for e in evs) / args.steps
    ms_per_step = total_ms / args.steps
    value = world * N / (ms_per_step / 1e3)

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    x_pin = torch.from_numpy(x).pin_memory()
    c_pin = torch.from_numpy(coeffs_h).pin_memory()
    e_top_i = np.empty(kk, np.int64)
    e_top_v = np.empty(kk, np.float32)

    def e2e_step():
        T.check(L.tfs_table_rebuild(table.handle, x_pin.data_ptr(), x_pin.numel(), 0, None))
        T.check(L.tfs_eval_stat(table.handle, basis.handle, c_pin.data_ptr(), None, N, w.m, kk, None,
                                e_top_i.ctypes.data, e_top_v.ctypes.data, None, 0, None))

    e2e_step()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        e2e_step()
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    if world > 1:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    h2d = x.nbytes + coeffs_h.nbytes
    d2h = kk * 12

    # roofline of the dominant kernel (the fused statistic kernel)
    esize = {"f32": 4, "bf16": 2, "f16": 2, "f8e4m3": 1}[args.dtype]
    bytes_per_track = w.n_seg * (2 * w.m + 1) * esize + w.K * 8 + 4
    achieved = N * bytes_per_track / (eval_ms / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    traffic = profiled_traffic(args.workload, args.dtype)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = min(args.cpu_sample, N)
        arm = OracleArm(x, psd, w, U, ncores)
        t_sft, t_eval = arm.step(coeffs_h[:sample])
        arm.close()
        cpu_val = N / (t_sft + N * (t_eval / sample))
        cpu = {"value": cpu_val, "unit": UNIT, "cores": ncores, "kind": "oracle",
               "sample": f"FP64 SFT of the full strain ({t_sft:.2f} s, 1 process) + statistic of {sample} tracks "
                         f"on {ncores} processes ({t_eval:.2f} s), scaled to {N} tracks per step"}
    if rank != 0:
        return
    clocks = clk.summary()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": args.workload, "tracks_per_rank": N, "n_seg": w.n_seg, "n_bin": w.n_bin,
                       "K": w.K, "m": w.m, "topk": kk, "table_dtype": args.dtype,
                       "l2": "inputs larger than L2 (coefficients %.0f MB per step); the table itself is reused "
                             "from L2 within a step" % (coeffs_h.nbytes / 1e6),
                       "parallelism": f"tracks sharded over {world} GPU(s)"},
            "breakdown_ms": {"sft_rebuild": sft_ms, "eval_stat": eval_ms, "topk": topk_ms},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": f"{peak_kind} hbm_gbs",
                         "bytes_per_track": bytes_per_track, "kernel": "eval_stat_kernel"},
            "e2e": {"value": world * N / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
