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
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 200 for the one-year workload, about 1 s, so that the clocks are sampled several times; 20 otherwise)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="oneyear_daily_fp32")
    ap.add_argument("--tracks", type=int, default=0, help="override the track count per rank")
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "f16", "f8e4m3"])
    ap.add_argument("--topk", type=int, default=128)
    ap.add_argument("--e2e-steps", type=int, default=9)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=1 << 18)
    ap.add_argument("--stat-error", type=int, default=20000,
                    help="report the statistic's error against the FP64 oracle on the exact table over this "
                         "many sampled tracks, outside the timed region (0: skip)")
    ap.add_argument("--statistic", default="nearest", choices=["nearest", "chirp"],
                    help="plunge-time search: the nearest-bin statistic or the paper's linear-chirp statistic")
    ap.add_argument("--segment-cuts", action="store_true",
                    help="apply the segment exclusions (second-order, low-frequency and low-fdot cuts)")
    ap.add_argument("--batch-jobs", type=int, default=64, help="datasets of the batched workload")
    ap.add_argument("--no-autotune", action="store_true", help="batched workload: keep the default launch shape")
    ap.add_argument("--requests", type=int, default=2000, help="requests of the served workload")
    ap.add_argument("--rate", type=float, default=200.0, help="request arrival rate (Hz) of the served workload")
    ap.add_argument("--datasets", type=int, default=32, help="resident datasets of the served workload")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="device-memory budget of the served workload")
    ap.add_argument("--budget-small-gb", type=float, default=2.0,
                    help="served workload: also serve the first --small-requests requests under this budget "
                         "(evictions and reloads; 0 skips)")
    ap.add_argument("--small-requests", type=int, default=300)
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 200 if (args.impl == "ours" and args.workload == "oneyear_daily_fp32") else 20
    return args


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


GATHER_NOTE = ("algorithmic bytes per track: 2m+1 table elements per segment, the coefficients, the offset "
               "and the result; the kernel reads one FP32 window sum per (track, segment) from shared memory, "
               "staged once per tile of up to 4608 tracks, so its DRAM and L2 traffic are far smaller and a "
               "fraction above 1 measures that reuse")


def gather_roofline(alg_bytes, ms, resident_bytes, L, kernel):
    """Roofline of a gather launch: algorithmic bytes over its time, against the L2 read bandwidth
    (measured now) when what it gathers from stays in L2, else against the measured HBM copy rate."""
    hbm, kind = measured_peaks()
    l2 = ctypes.c_double()
    rc = L.tfs_measure_l2_read(48 << 20, 40, ctypes.byref(l2))
    achieved = alg_bytes / (ms / 1e3) / 1e9
    bound = "l2" if resident_bytes <= 63e6 and rc == 0 else "hbm"
    peak = l2.value if bound == "l2" else hbm
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None,
            "peak_source": ("tfs_measure_l2_read in this run: 16-byte L1-bypassing loads over a 48 MB buffer, "
                            "40 passes") if bound == "l2" else f"{kind} hbm_gbs (MEASURED_PEAKS.json)",
            "resident_bytes": int(resident_bytes), "hbm_peak_gbs": hbm, "frac_of_hbm": achieved / hbm,
            "l2_peak_gbs": l2.value, "frac_of_l2": achieved / l2.value if l2.value else None, "kernel": kernel,
            "note": GATHER_NOTE}


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("eval_kernel.cuh", "eval_host.cu", "wsum.cu", "tfs_internal.cuh"):
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


def chirp_flops_pair(M: int, P: int) -> int:
    """FP32 work of the chirp statistic per (track, segment) pair: the M-point complex FFT of the
    template (5 M log2 M), its M windowed samples (6 flops each) and the 2P + 1 complex products
    with the data and norms (8 + 4 flops per bin)."""
    return 5 * M * int(math.log2(M)) + 6 * M + 12 * (2 * P + 1)


# --------------------------------------------------------------------------- CPU oracle arm
_W = {}
_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _oracle_init(P, V, T_sft, m, cuts=False):
    _W.update(P=P, V=V, T=T_sft, m=m, cuts=cuts)


def _oracle_chunk(coeffs):
    import oracle.tfstat_oracle as O

    if _W["cuts"]:
        S, _ = O.eval_stat_masked(_W["P"], _W["V"], coeffs, np.zeros(len(coeffs)), _W["T"], _W["m"])
    else:
        S, *_ = O.eval_stat(_W["P"], _W["V"], coeffs, np.zeros(len(coeffs)), _W["T"], _W["m"], 0)
    return float(S.sum())


class OracleArm:
    """The oracle as it stands on the host cores: its FP64 SFT of the whole strain
    (one process) plus its statistic of a sample of tracks split over a spawn pool;
    the rate is the batch's tracks over (SFT time + batch x per-track time)."""

    def __init__(self, x, psd, w, V, ncores, cuts=False):
        import oracle.tfstat_oracle as O

        self.O, self.x, self.psd, self.w, self.V, self.ncores = O, x, psd, w, V, ncores
        P = O.power_table(x, w.dt, w.T_sft, psd)
        # one thread per worker process (numpy's BLAS would otherwise start a thread per core in
        # each of them), so that `ncores` is the number of cores the oracle actually uses
        saved = {k: os.environ.get(k) for k in _THREAD_VARS}
        os.environ.update({k: "1" for k in _THREAD_VARS})
        try:
            self.pool = mp.get_context("spawn").Pool(ncores, initializer=_oracle_init,
                                                     initargs=(P, V, w.T_sft, w.m, cuts))
            self.pool.map(_oracle_chunk, [np.zeros((1, V.shape[0]))] * ncores)   # warm the workers
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

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
    steps_s = []
    for i in range(args.warmup + args.steps):
        t_sft, t_eval = arm.step(coeffs)
        if i >= args.warmup:
            steps_s.append(t_sft + t_eval)
    arm.close()
    # what was timed: one step is the FP64 SFT of the whole strain plus the statistic of `sample`
    # tracks of the workload (not scaled up to the full batch)
    step_s = float(statistics.median(steps_s))
    value = sample / step_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * step_s, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "tracks_per_step": sample, "n_seg": w.n_seg, "n_bin": w.n_bin,
                       "K": w.K, "m": w.m, "topk": args.topk},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncores, "kind": "oracle",
                             "sample": f"per step: FP64 SFT of the full strain + statistic of {sample} of the "
                                       f"workload's tracks on {ncores} single-threaded processes"},
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
    cut_job = None
    if args.segment_cuts:
        # the exclusions are a flag of the batched entry point: one job, asynchronous
        cut_status = torch.zeros(1, dtype=torch.int32, device="cuda")
        cut_job = T.Job(table, basis, coeffs_d, None, m=w.m, stat=stat, segment_cuts=True)

    def eval_call():
        if cut_job is None:
            T.check(L.tfs_eval_stat(table.handle, basis.handle, coeffs_d.data_ptr(), None, N, w.m, 0,
                                    stat.data_ptr(), None, None, None, 1, sp))
        else:
            T.eval_batch([cut_job], dev_status=cut_status, stream=stream.cuda_stream)

    def step(evs=None):
        if evs is not None:
            evs[0].record(stream)
        T.check(L.tfs_table_rebuild(table.handle, x_d.data_ptr(), x_d.numel(), 1, sp))
        if evs is not None:
            evs[1].record(stream)
        eval_call()
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
    if cut_job is not None:
        assert int(cut_status.item()) == 0, "a bounded device wait gave up"
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
    s_pin = torch.empty(N, dtype=torch.float32).pin_memory()   # statistic[N] comes back every step
    e_top_i = np.empty(kk, np.int64)
    e_top_v = np.empty(kk, np.float32)

    if cut_job is not None:
        c_e2e = torch.empty_like(coeffs_d)
        e2e_job = T.Job(table, basis, c_e2e, None, m=w.m, topk=kk, stat=stat, segment_cuts=True)

    # one stream of its own: the rebuild returns once the strain is up and its transform
    # overlaps the upload of the first coefficients; the statistic call returns with the
    # top-k in host memory
    e2e_stream = torch.cuda.Stream()
    e2e_sp = ctypes.c_void_p(e2e_stream.cuda_stream)

    def e2e_step():
        T.check(L.tfs_table_rebuild(table.handle, x_pin.data_ptr(), x_pin.numel(), 0, e2e_sp))
        if cut_job is None:
            T.check(L.tfs_eval_stat(table.handle, basis.handle, c_pin.data_ptr(), None, N, w.m, kk,
                                    s_pin.data_ptr(), e_top_i.ctypes.data, e_top_v.ctypes.data, None, 0, e2e_sp))
        else:
            # host coefficients uploaded on the stream, the batched entry point, top-k read back
            with torch.cuda.stream(e2e_stream):
                c_e2e.copy_(c_pin, non_blocking=True)
                T.eval_batch([e2e_job], stream=e2e_stream.cuda_stream)
                s_pin.copy_(stat, non_blocking=True)
                e_top_i[:] = e2e_job.top_idx.cpu().numpy()
                e_top_v[:] = e2e_job.top_val.cpu().numpy()

    e2e_step()
    e2e_step()
    if world > 1:
        dist.barrier()
    # each step timed on its own (the call returns with its results in host memory); the median
    # step, so that one step held up by something else on the host does not set the figure
    e2e_steps_s = []
    for _ in range(args.e2e_steps):
        t0 = time.perf_counter()
        e2e_step()
        e2e_steps_s.append(time.perf_counter() - t0)
    e2e_s = float(statistics.median(e2e_steps_s))
    if world > 1:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    h2d = x.nbytes + coeffs_h.nbytes
    d2h = N * 4 + kk * 12

    # roofline of the dominant kernel (the fused statistic kernel)
    esize = {"f32": 4, "bf16": 2, "f16": 2, "f8e4m3": 1}[args.dtype]
    bytes_per_track = w.n_seg * (2 * w.m + 1) * esize + w.K * 8 + 4
    achieved = N * bytes_per_track / (eval_ms / 1e3) / 1e9
    hbm_peak, peak_kind = measured_peaks()
    traffic = profiled_traffic(args.workload, args.dtype)
    # L2 read bandwidth, measured in this run (MEASURED_PEAKS.json has no L2 figure)
    l2_gbs = ctypes.c_double()
    T.check(L.tfs_measure_l2_read(48 << 20, 40, ctypes.byref(l2_gbs)))
    # the kernel gathers from the table's FP32 window sums; when they and the table fit in half of
    # the 126 MB L2 (the rest holds the streamed coefficients), the applicable bound is L2, else HBM
    pad32 = lambda n: (n + 31) // 32 * 32  # noqa: E731
    resident = w.n_seg * (pad32(w.n_bin + 2 * w.m) * 4 + pad32(w.n_bin) * esize)
    bound = "l2" if resident <= 63e6 else "hbm"
    peak = l2_gbs.value if bound == "l2" else hbm_peak
    peak_source = ("tfs_measure_l2_read in this run: 16-byte L1-bypassing loads over a 48 MB buffer, 40 passes"
                   if bound == "l2" else f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = min(args.cpu_sample, N)
        arm = OracleArm(x, psd, w, U, ncores, cuts=args.segment_cuts)
        t_sft, t_eval = arm.step(coeffs_h[:sample])
        arm.close()
        cpu_val = N / (t_sft + N * (t_eval / sample))
        cpu = {"value": cpu_val, "unit": UNIT, "cores": ncores, "kind": "oracle",
               "sample": f"FP64 SFT of the full strain ({t_sft:.2f} s, 1 process) + statistic of {sample} tracks "
                         f"on {ncores} processes ({t_eval:.2f} s), scaled to {N} tracks per step"}
        # the same oracle on one core (one single-threaded process), on a smaller sample
        sample1 = max(1, sample // 16)
        arm1 = OracleArm(x, psd, w, U, 1, cuts=args.segment_cuts)
        t_sft1, t_eval1 = arm1.step(coeffs_h[:sample1])
        arm1.close()
        cpu["single_core"] = {"value": N / (t_sft1 + N * (t_eval1 / sample1)), "unit": UNIT, "cores": 1,
                              "sample": f"FP64 SFT of the full strain ({t_sft1:.2f} s) + statistic of {sample1} "
                                        f"tracks ({t_eval1:.2f} s) in one single-threaded process, scaled to {N} "
                                        f"tracks per step"}
    stat_err = None
    if rank == 0 and args.stat_error > 0:
        import oracle.tfstat_oracle as O

        n_s = min(args.stat_error, N)
        P64 = O.power_table(x, w.dt, w.T_sft, psd)
        eval_call()
        got = stat[:n_s].double().cpu().numpy()
        if cut_job is None:
            ref, *_ = O.eval_stat(P64, U, coeffs_h[:n_s], np.zeros(n_s), w.T_sft, w.m, 0)
        else:
            ref, valid = O.eval_stat_masked(P64, U, coeffs_h[:n_s], np.zeros(n_s), w.T_sft, w.m)
        rel = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)
        stat_err = {"max_rel": float(rel.max()), "mean_rel": float(rel.mean()), "tracks": n_s,
                    "against": "FP64 oracle statistic of the exact FP64 table (no quantisation)"}
        if cut_job is not None:
            stat_err["excluded_fraction"] = float(1.0 - valid.mean())
    if rank != 0:
        return
    clocks = clk.summary()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": args.workload, "tracks_per_rank": N, "n_seg": w.n_seg, "n_bin": w.n_bin,
                       "K": w.K, "m": w.m, "topk": kk, "table_dtype": args.dtype,
                       "segment_cuts": bool(args.segment_cuts),
                       "l2": "inputs larger than L2 (coefficients %.0f MB per step); the table itself is reused "
                             "from L2 within a step" % (coeffs_h.nbytes / 1e6),
                       "parallelism": f"tracks sharded over {world} GPU(s)"},
            "breakdown_ms": {"sft_rebuild": sft_ms, "eval_stat": eval_ms, "topk": topk_ms},
            "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_source": peak_source,
                         "bytes_per_track": bytes_per_track, "kernel": "eval_stat_kernel",
                         "resident_bytes": resident,
                         "hbm_peak_gbs": hbm_peak, "frac_of_hbm": achieved / hbm_peak,
                         "l2_peak_gbs": l2_gbs.value, "frac_of_l2": achieved / l2_gbs.value,
                         "note": GATHER_NOTE},
            "e2e": {"value": world * N / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * e2e_s,
                    "mean_ms": 1e3 * sum(e2e_steps_s) / len(e2e_steps_s),
                    "steps_ms": [round(1e3 * t, 3) for t in e2e_steps_s],
                    "timing": "median of the steps, each timed from the call to its results in host memory"},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "cpu_baseline": cpu}
    if stat_err is not None:
        line["stat_error"] = stat_err
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# --------------------------------------------------------------------------- linear-chirp statistic
def _chirp_oracle_sample(x, psd, w, U, coeffs):
    """The oracle's linear-chirp statistic of a few tracks (its own SFT of the strain included)."""
    import oracle.tfstat_oracle as O

    t0 = time.perf_counter()
    d = O.sft(x, w.dt, w.T_sft)
    t_sft = time.perf_counter() - t0
    t1 = time.perf_counter()
    F = O.track_freqs(U, coeffs, np.zeros(len(coeffs)))
    S = O.chirp_statistic(d, psd, w.dt, w.T_sft, F)
    return t_sft, time.perf_counter() - t1, S


def run_chirp(args):
    """The paper's full statistic (the linear-chirp template over 2P + 1 = 201 bins per segment)
    on the one-year data: tracks/s, with the kernel against the FP32 pipe's peak."""
    import torch

    from paper_2510_20891_gb300 import build as B

    B.build()
    import paper_2510_20891_gb300 as T

    L = T.lib()
    w = synth.WORKLOADS["oneyear_daily_fp32"]
    N = args.tracks or 200_000
    x, psd, F, inj, rng = make_inputs(w, 0, N)
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    x_d = torch.from_numpy(x).cuda()
    ct = T.build_chirp_table(x_d, w.dt, w.T_sft, psd)
    basis = T.build_basis(F, w.K)
    U, sig, cmin, cmax = basis.to_host()
    coeffs_h = synth.uniform_coeffs(N, cmin, cmax, rng)
    coeffs_d = torch.from_numpy(coeffs_h).cuda()
    stat = torch.empty(N, dtype=torch.float32, device="cuda")
    kk = min(args.topk, N)
    top_i = torch.empty(kk, dtype=torch.int64, device="cuda")
    top_v = torch.empty(kk, dtype=torch.float32, device="cuda")
    P = T.CHIRP_P

    def step(evs=None):
        if evs is not None:
            evs[0].record(stream)
        T.eval_chirp_stat(ct, basis, coeffs_d, None, P=P, segment_cuts=args.segment_cuts, stat=stat,
                          stream=stream.cuda_stream)
        if evs is not None:
            evs[1].record(stream)
        T.check(L.tfs_topk(stat.data_ptr(), N, kk, top_i.data_ptr(), top_v.data_ptr(), 1, sp))
        if evs is not None:
            evs[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = L.tfs_kernel_launches()
    with ClockSampler(0) as clk:
        start.record(stream)
        for i in range(args.steps):
            step(evs[i])
        end.record(stream)
        torch.cuda.synchronize()
    launches = L.tfs_kernel_launches() - launches0
    ms_per_step = start.elapsed_time(end) / args.steps
    kern_ms = sum(e[0].elapsed_time(e[1]) for e in evs) / args.steps
    topk_ms = sum(e[1].elapsed_time(e[2]) for e in evs) / args.steps

    # end to end: host coefficients (pinned) up, statistic and top-k, top-k back to the host
    c_pin = torch.from_numpy(coeffs_h).pin_memory()
    c_dev = torch.empty_like(coeffs_d)

    def e2e_step():
        c_dev.copy_(c_pin, non_blocking=True)
        _, ti, tv = T.eval_chirp_stat(ct, basis, c_dev, None, P=P, segment_cuts=args.segment_cuts, stat=stat,
                                      topk=kk, stream=stream.cuda_stream)
        return ti.cpu().numpy(), tv.cpu().numpy()

    e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        e2e_step()
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps

    # roofline: FP32 work per (track, segment) pair = the M-point complex FFT of the template
    # (5 M log2 M), the windowed samples (6 flops each) and the 2P + 1 complex products and norms
    # (8 + 4 flops per bin); peak = 152 SMs x 128 FP32 lanes x 2 flops x the sampled SM clock
    flops_pair = chirp_flops_pair(T.CHIRP_M, P)
    achieved = N * w.n_seg * flops_pair / (kern_ms / 1e3) / 1e12
    clocks = clk.summary()
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    cpu = None
    stat_err = None
    if not args.no_cpu_baseline:
        n_s = 16
        t_sft, t_eval, S_ref = _chirp_oracle_sample(x, psd, w, U, coeffs_h[:n_s])
        cpu = {"value": N / (t_sft + N * t_eval / n_s), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"FP64 SFT of the full strain ({t_sft:.2f} s) + linear-chirp statistic of {n_s} tracks "
                         f"({t_eval:.2f} s), one process, scaled to {N} tracks per step"}
        if args.segment_cuts:
            S_ref = None
        else:
            got = stat[:n_s].double().cpu().numpy()
            stat_err = {"max_rel": float(np.max(np.abs(got - S_ref) / np.maximum(np.abs(S_ref), 1e-300))),
                        "tracks": n_s, "against": "FP64 oracle linear-chirp statistic (L-point template SFT)"}
    line = {"metric": "linear-chirp track-statistic evals/s (1-yr data, 2P+1 = 201 bins per segment)",
            "value": N / (ms_per_step / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "oneyear_daily_fp32 linear-chirp statistic", "tracks": N, "n_seg": w.n_seg,
                       "n_bin": w.n_bin, "K": w.K, "P": P, "segment_cuts": bool(args.segment_cuts),
                       "l2": "the 25 MB complex table stays in L2; coefficients %.0f MB per step" %
                             (coeffs_h.nbytes / 1e6)},
            "breakdown_ms": {"chirp_stat": kern_ms, "topk": topk_ms},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops x sampled SM clock",
                         "flops_per_pair": flops_pair, "kernel": "chirp_stat_kernel"},
            "e2e": {"value": N / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(coeffs_h.nbytes),
                    "d2h_bytes_per_step": kk * 12},
            "gpu_launches": int(launches), "clocks": clocks, "cpu_baseline": cpu}
    if stat_err is not None:
        line["stat_error"] = stat_err
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- plunge-time search
def run_tpl_search(args):
    """The paper's whole search (Sec. II.D) on one year of data in 631 SFTs of 5e4 s: 48 chunks of
    growing duration, 1024 initial candidates per chunk, the best 512 kept, then DE iterations,
    each one graph-replayed batched launch over all chunks.  Value: statistic evaluations/s of the
    whole search, host included (the random draws, uploads and the search driver are inside)."""
    import torch

    from paper_2510_20891_gb300 import build as B

    B.build()
    import paper_2510_20891_gb300 as T
    from paper_2510_20891_gb300 import search

    L = T.lib()
    w = synth.WORKLOADS["oneyear_5e4_631"]
    x, psd, F, inj, rng = make_inputs(w, 0, 0)
    chirp = args.statistic == "chirp"
    x_d = torch.from_numpy(x).cuda()
    table = T.build_sfts(x_d, w.dt, w.T_sft, psd, "hann", args.dtype)
    ct = T.build_chirp_table(x_d, w.dt, w.T_sft, psd) if chirp else None
    basis = T.build_basis(F, w.K)
    U, sig, cmin, cmax = basis.to_host()
    cs = search.ChunkSearch(table, basis, chirp_table=ct)
    n_iter = args.steps
    W = 512
    shape = None
    if not args.no_autotune and not chirp:
        # launch shape for one iteration's batch (48 chunk jobs of 512 walkers, with the cuts)
        tune_c = [torch.tensor(cmin + (cmax - cmin) * rng.random((W, w.K)), device="cuda") for _ in cs.sizes]
        shape, _, _ = T.autotune(cs.jobs(tune_c, m=w.m, segment_cuts=True), reps=3)
    # warm-up: a short search builds the cached per-chunk data and the graph machinery
    search.DESearch(cs, cmin, cmax, m=w.m, seed=1, segment_cuts=True,
                    statistic=args.statistic).run(n_iter=max(1, args.warmup), U_full=U)
    torch.cuda.synchronize()
    launches0 = L.tfs_kernel_launches()
    with ClockSampler(0) as clk:
        de = search.DESearch(cs, cmin, cmax, m=w.m, seed=2, segment_cuts=True, statistic=args.statistic)
        res = de.run(n_iter=n_iter, U_full=U)
    # the captured iteration is counted once by the library; its other replays are added here
    launches = L.tfs_kernel_launches() - launches0 + de.uncounted_launches
    # device time of one iteration's batched statistic launch (events around an uncaptured call) on
    # the trial walkers of the search's last iteration (uniform draws from the prior box leave many
    # tracks outside the band, whose pairs cost far less, and the converged population shares its
    # bands more than the proposals do)
    jobs = de.trial_jobs
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    cs.launch(jobs, args.statistic, dev_status=status)
    # replayed from a CUDA graph, as in the search, so that no host time falls between launches
    # (its kernels are not added to gpu_launches: they run after the timed search)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            cs.launch(jobs, args.statistic, dev_status=status, stream=side.cuda_stream)
    torch.cuda.current_stream().wait_stream(side)
    g.replay()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    batch_ms = e0.elapsed_time(e1) / 20
    pairs = W * sum(cs.sizes)
    bytes_batch = sum(W * (n * (2 * w.m + 1) * 4 + 8 * w.K + 4) for n in cs.sizes)
    if chirp:
        flops_pair = chirp_flops_pair(T.CHIRP_M, T.CHIRP_P)
        achieved = pairs * flops_pair / (batch_ms / 1e3) / 1e12
        sm_mhz = 2070.0
        roof = {"bound": "alu", "achieved": achieved, "peak": 152 * 128 * 2 * sm_mhz * 1e6 / 1e12, "unit": "TFLOP/s",
                "traffic": None, "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz",
                "flops_per_pair": flops_pair, "kernel": "chirp_stat_kernel (48 chunk jobs)"}
    else:
        pad32 = lambda n: (n + 31) // 32 * 32  # noqa: E731
        resident = w.n_seg * (pad32(w.n_bin) * 4 + pad32(w.n_bin + 2 * w.m) * 4)
        roof = gather_roofline(bytes_batch, batch_ms, resident, L, "eval_stat_kernel (48 chunk jobs)")
        roof["bytes_per_iteration"] = bytes_batch
    roof["frac"] = roof["achieved"] / roof["peak"]
    cpu = None
    if not args.no_cpu_baseline and chirp:
        import oracle.tfstat_oracle as O

        d = O.sft(x, w.dt, w.T_sft)
        n = cs.sizes[-1]
        c_s = cmin + (cmax - cmin) * rng.random((4, w.K))
        t0 = time.perf_counter()
        Fs = O.track_freqs(U[:, w.n_seg - n:], c_s, np.zeros(4))
        O.chirp_statistic(d[:n], psd, w.dt, w.T_sft, Fs, valid=O.segment_validity(Fs, w.T_sft))
        t_s = time.perf_counter() - t0
        per_pair = t_s / (4 * n)
        cpu = {"value": res.evaluations / (per_pair * (pairs * (n_iter + 2))), "unit": "evals/s", "cores": 1,
               "kind": "oracle", "sample": f"masked linear-chirp statistic of 4 walkers of the {n}-segment chunk "
                                           f"({t_s:.2f} s, one process), scaled by track-segment pairs"}
    elif not args.no_cpu_baseline:
        import oracle.tfstat_oracle as O

        P64 = O.power_table(x, w.dt, w.T_sft, psd)
        sample = [cmin + (cmax - cmin) * rng.random((W, w.K)) for _ in range(4)]
        sizes = cs.sizes[-4:]
        t0 = time.perf_counter()
        for c_s, n in zip(sample, sizes):  # the chunk's data prefix and shifted basis, with the cuts
            O.eval_stat_masked(P64[:n], U[:, w.n_seg - n:], c_s, np.zeros(W), w.T_sft, w.m)
        t_s = time.perf_counter() - t0
        per_pair = t_s / (W * sum(sizes))
        cpu = {"value": res.evaluations / (per_pair * (pairs * (n_iter + 2))), "unit": "evals/s", "cores": 1,
               "kind": "oracle", "sample": f"masked statistic of 4 chunks x {W} walkers ({t_s:.2f} s, one process), "
                                           "scaled by track-segment pairs to the whole search"}
    best = int(np.argmax(res.stat if chirp else res.normalised))
    line = {"metric": "plunge-time search statistic evaluations/s (48 chunks x (1024 + iterations x 512))"
                      + (", linear-chirp statistic" if chirp else ""),
            "value": res.evaluations / res.seconds, "unit": "evals/s", "n_gpus": 1, "steps": n_iter,
            "warmup": args.warmup, "ms_per_step": res.seconds / max(1, n_iter) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": "oneyear_5e4_631 plunge-time search", "n_seg": w.n_seg, "n_bin": w.n_bin,
                       "K": w.K, "m": w.m, "chunks": len(cs.sizes), "chunk_segments": [cs.sizes[0], cs.sizes[-1]],
                       "walkers": W, "initial": 1024, "iterations": n_iter, "table_dtype": args.dtype,
                       "launch_shape": shape, "statistic": args.statistic,
                       "l2": "the 12.6 MB table and every chunk's walkers stay in L2"},
            "search": {"evaluations": res.evaluations, "seconds": res.seconds, "setup_s": de.t_setup,
                       "iterations_s": de.t_iter, "segment_cuts": True,
                       "best_chunk_segments": cs.sizes[best], "best_stat": float(res.stat[best]),
                       "best_normalised": None if chirp else float(res.normalised[best]),
                       "injection": {k: float(v) for k, v in inj.items() if k != "kind"}},
            "breakdown_ms": {"batched_statistic_per_iteration": batch_ms,
                             "iteration": 1e3 * de.t_iter / max(1, n_iter)},
            "roofline": roof,
            "e2e": {"value": res.evaluations / res.seconds, "unit": "evals/s",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                    "note": "the whole search is host-driven; its random draws are uploaded once before the "
                            "iterations and the results read back once after them"},
            "gpu_launches": int(launches), "clocks": clk.summary(), "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- batched datasets
def run_batched(args):
    """64 uneven datasets (durations, T_SFT, K, track counts) evaluated by one persistent
    launch per step, replayed from a CUDA graph; compared with one tfs_eval_stat per dataset."""
    from concurrent.futures import ProcessPoolExecutor

    items = synth.batched_workloads(args.batch_jobs)
    ncores = os.cpu_count() or 1
    with ProcessPoolExecutor(ncores, mp_context=mp.get_context("spawn")) as ex:  # before any CUDA call
        data = list(ex.map(synth.make_batched_inputs, items))
    import torch
    from paper_2510_20891_gb300 import build as B

    B.build()
    import paper_2510_20891_gb300 as T

    L = T.lib()
    stream = torch.cuda.current_stream()
    jobs, keep = [], []
    for (w, snr), (x, psd, F) in zip(items, data):
        x_d = torch.from_numpy(x).cuda()
        table = T.build_sfts(x_d, w.dt, w.T_sft, psd, "hann", args.dtype)
        del x_d
        basis = T.build_basis(F, w.K)
        U, sig, cmin, cmax = basis.to_host()
        c = torch.from_numpy(synth.uniform_coeffs(w.n_tracks, cmin, cmax, np.random.default_rng(1000 + w.seed))).cuda()
        jobs.append(T.Job(table, basis, c, None, m=w.m, topk=min(args.topk, w.n_tracks)))
        keep.append((table, basis))
    n_tracks = sum(w.n_tracks for w, _ in items)
    pairs = sum(w.n_tracks * w.n_seg for w, _ in items)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    T.eval_batch(jobs, dev_status=status)
    torch.cuda.synchronize()
    ms_default = None
    tuned = None
    if not args.no_autotune:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            T.eval_batch(jobs, dev_status=status)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_default = e0.elapsed_time(e1) / 3
        tuned, _, _ = T.autotune(jobs, reps=3)   # untimed: picks the launch shape used below
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            T.eval_batch(jobs, dev_status=status, stream=side.cuda_stream)
    torch.cuda.synchronize()

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    launches0 = L.tfs_kernel_launches()
    with ClockSampler(0) as clk:
        ms = timed(g.replay, args.steps)
    assert int(status.item()) == 0
    # graph launches do not pass through the library's counter: count one replay's kernels
    k0 = L.tfs_kernel_launches()
    T.eval_batch(jobs, dev_status=status)
    torch.cuda.synchronize()
    per_batch = L.tfs_kernel_launches() - k0
    ms_uncaptured = timed(lambda: T.eval_batch(jobs, dev_status=status), max(3, args.steps // 4))

    def sequential():
        for j in jobs:
            T.eval_stat(j.table, j.basis, j.coeffs, None, m=j.m, topk=j.topk, stat=j.stat, top_idx=j.top_idx,
                        top_val=j.top_val)

    ms_seq = timed(sequential, max(3, args.steps // 4))
    del launches0
    esize = {"f32": 4, "bf16": 2, "f16": 2, "f8e4m3": 1}[args.dtype]
    bytes_all = sum(w.n_tracks * (w.n_seg * (2 * w.m + 1) * esize + w.K * 8 + 4) for w, _ in items)
    pad32 = lambda n: (n + 31) // 32 * 32  # noqa: E731
    resident = sum(w.n_seg * (pad32(w.n_bin) * esize + pad32(w.n_bin + 2 * w.m) * 4) for w, _ in items)
    roof = gather_roofline(bytes_all, ms, resident, L, "eval_stat_kernel (all datasets)")
    value = n_tracks / (ms / 1e3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": f"batched{args.batch_jobs}", "datasets": len(items), "tracks": n_tracks,
                       "pairs": pairs, "T_sft_s": sorted({w.T_sft for w, _ in items}),
                       "K": sorted({w.K for w, _ in items}), "n_seg_range": [min(w.n_seg for w, _ in items),
                                                                            max(w.n_seg for w, _ in items)],
                       "m": 1, "topk_per_dataset": args.topk, "table_dtype": args.dtype,
                       "launch": "one tfs_eval_batch per step (one persistent launch per table dtype, "
                                 "per-dataset top-k), replayed from a CUDA graph",
                       "l2": "coefficients %.0f MB per step (larger than L2)" % (n_tracks * 6 * 8 / 1e6)},
            "uncaptured_ms_per_step": ms_uncaptured,
            "autotuned_shape": tuned, "default_shape_ms_per_step": ms_default,
            "sequential_ms_per_step": ms_seq,
            "sequential_value": n_tracks / (ms_seq / 1e3),
            "roofline": roof,
            "e2e": None,
            "gpu_launches": int(per_batch) * args.steps,
            "clocks": clk.summary(),
            "cpu_baseline": None}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- served requests
def run_served(args):
    """Poisson requests (a dataset and 10^3-10^6 tracks, BF16 or FP32 table) against resident
    datasets of the 1577 x 20001 shape, served with continuous batching under a budget;
    compared with the plain FP32 path that runs one request at a time."""
    import queue
    import threading

    import torch
    from paper_2510_20891_gb300 import build as B

    B.build()
    import paper_2510_20891_gb300 as T

    w = synth.WORKLOADS["oneyear_fine_1577x20001"]
    rng = np.random.default_rng(0)
    basis = T.build_basis(synth.make_training_tracks(w, rng), w.K)
    U, sig, cmin, cmax = basis.to_host()
    reqs = synth.served_requests(args.requests, args.rate, args.datasets, seed=0)
    bank = synth.uniform_coeffs(int(max(r[2] for r in reqs)), cmin, cmax, np.random.default_rng(1))
    offs = np.random.default_rng(2).integers(0, 1 << 20, len(reqs))
    budget = int(args.budget_gb * (1 << 30))
    psd = synth.psd_bins(w.psd_fn(), w.n_bin, w.T_sft)

    def dataset_tables(d, dtypes):
        """Dataset d's tables: the fine one-year generator's strain (noise of the one-year PSD and one
        power-law harmonic at SNR 30, seed 100 + d), drawn and transformed on the device."""
        x, _ = synth.make_strain_device(w, 100 + d)
        out = [T.build_sfts(x, w.dt, w.T_sft, psd, "hann", dt) for dt in dtypes]
        del x
        torch.cuda.empty_cache()
        return out

    srv = T.Server(budget, max_batch_jobs=64)
    ids, f32_tables = {}, []
    for d in range(args.datasets):
        tf, tb = dataset_tables(d, ("f32", "bf16"))
        ids[(d, "f32")] = srv.add_dataset(tf, basis)
        ids[(d, "bf16")] = srv.add_dataset(tb, basis)
        # the plain path's own FP32 table of every dataset (the same data; its window sums and L2
        # state are its own)
        f32_tables.append(dataset_tables(d, ("f32",))[0])
    torch.cuda.synchronize()

    def coeffs_of(i):
        N = reqs[i][2]
        o = int(offs[i]) % max(1, bank.shape[0] - N + 1)
        return bank[o:o + N]

    # warm-up: one small request per table (builds each table's window sums and the per-segment
    # data, as the plain path's tables get theirs in its saturated run before its paced one)
    for d in range(args.datasets):
        for dt in ("f32", "bf16"):
            srv.wait(srv.submit(ids[(d, dt)], coeffs_of(0)[:1000], None, m=w.m, topk=16))
    s0 = srv.stats()
    tickets = [None] * len(reqs)
    done_t = [0.0] * len(reqs)
    t_start = time.perf_counter()

    # collectors block on a queue and enter the server's wait as soon as a ticket exists (a
    # collector that polled for its ticket could enter late, and the server's latency, which
    # runs from submit to results in host memory, would count that)
    todo = queue.Queue()

    def collect():
        out = np.zeros(max(r[2] for r in reqs), np.float32)  # this collector's result buffer, reused
        while True:
            i = todo.get()
            if i is None:
                return
            srv.wait(tickets[i], 600000, stat=out)
            done_t[i] = time.perf_counter()

    n_coll = 16
    coll = [threading.Thread(target=collect) for _ in range(n_coll)]
    for t in coll:
        t.start()
    with ClockSampler(0) as clk:
        for i, (ta, d, N, dt) in enumerate(reqs):
            now = time.perf_counter() - t_start
            if ta > now:
                time.sleep(ta - now)
            tickets[i] = srv.submit(ids[(d, dt)], coeffs_of(i), None, m=w.m, topk=16)
            todo.put(i)
        for _ in coll:
            todo.put(None)
        for t in coll:
            t.join()
    t_end = max(done_t)
    st = srv.stats()
    n_tracks = sum(r[2] for r in reqs)
    served_lat = st["p50_ms"], st["p99_ms"]
    value = n_tracks / (t_end - t_start)

    # saturation: every request submitted at once (no pacing): the server's throughput
    t_sat0 = time.perf_counter()
    sat = [srv.submit(ids[(d, dt)], coeffs_of(i), None, m=w.m, topk=16) for i, (ta, d, N, dt) in enumerate(reqs)]
    for tk in sat:
        srv.wait(tk, 600000)
    sat_s = time.perf_counter() - t_sat0
    st_sat = srv.stats()

    # accuracy of the BF16 path against FP32 on the same tracks (a few requests)
    errs = []
    for i in range(4):
        c = coeffs_of(i)[:20000]
        a = srv.wait(srv.submit(ids[(i, "bf16")], c, None, m=w.m))[0].astype(np.float64)
        b = T.eval_stat(f32_tables[i], basis, c, None, m=w.m).stat.astype(np.float64)
        errs.append(float(np.max(np.abs(a - b) / np.abs(b))))
    srv.close()

    # a budget that holds a few datasets only: admission waits for room and idle tables are
    # evicted (least recently used) and reloaded; the first requests of the same stream, paced
    small = None
    if args.budget_small_gb > 0:
        n_small = min(len(reqs), args.small_requests)
        srv2 = T.Server(int(args.budget_small_gb * (1 << 30)), max_batch_jobs=64)
        ids2 = {}
        for d in sorted({r[1] for r in reqs[:n_small]}):
            tf, tb = dataset_tables(d, ("f32", "bf16"))
            ids2[(d, "f32")] = srv2.add_dataset(tf, basis)
            ids2[(d, "bf16")] = srv2.add_dataset(tb, basis)
        torch.cuda.synchronize()
        s20 = srv2.stats()
        t2 = time.perf_counter()
        tk2 = []
        for i, (ta, d, N, dt) in enumerate(reqs[:n_small]):
            now = time.perf_counter() - t2
            if ta > now:
                time.sleep(ta - now)
            tk2.append(srv2.submit(ids2[(d, dt)], coeffs_of(i), None, m=w.m, topk=16))
        for tk in tk2:
            srv2.wait(tk, 600000)
        t2e = time.perf_counter() - t2
        s2 = srv2.stats()
        small = {"budget_gb": args.budget_small_gb, "requests": n_small, "datasets": len(ids2) // 2,
                 "value": sum(r[2] for r in reqs[:n_small]) / t2e, "p50_ms": s2["p50_ms"], "p99_ms": s2["p99_ms"],
                 "evictions": s2["evictions"] - s20["evictions"], "loads": s2["loads"] - s20["loads"],
                 "failed": s2["failed"], "mean_jobs_per_batch": s2["mean_jobs_per_batch"]}
        srv2.close()

    # the plain FP32 path: one request at a time, in arrival order, through tfs_eval_stat
    t_b0 = time.perf_counter()
    for i, (ta, d, N, dt) in enumerate(reqs):
        T.eval_stat(f32_tables[d], basis, coeffs_of(i), None, m=w.m, topk=16)
    base_sat_s = time.perf_counter() - t_b0
    lat = []
    t0 = time.perf_counter()
    for i, (ta, d, N, dt) in enumerate(reqs):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        tb = f32_tables[d]
        T.eval_stat(tb, basis, coeffs_of(i), None, m=w.m, topk=16)
        lat.append((time.perf_counter() - t0 - ta) * 1e3)
    t1 = time.perf_counter() - t0
    lat.sort()
    base = {"value": n_tracks / t1, "saturated_value": n_tracks / base_sat_s, "p50_ms": lat[len(lat) // 2],
            "p99_ms": lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)],
            "path": "tfs_eval_stat on FP32 tables, host buffers, one request at a time in arrival order"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": len(reqs), "warmup": 2,
            "ms_per_step": (t_end - t_start) * 1e3 / len(reqs), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16+f32", "data": "synthetic",
            "config": {"workload": f"served{args.datasets}", "requests": len(reqs), "rate_hz": args.rate,
                       "tracks": n_tracks, "tracks_per_request": "log-uniform 1e3..1e6", "n_seg": w.n_seg,
                       "n_bin": w.n_bin, "K": w.K, "m": w.m, "topk": 16, "tables": "BF16 or FP32 per request, from the fine one-year generator (strain drawn on the device)",
                       "budget_gb": args.budget_gb},
            "served": {"p50_ms": served_lat[0], "p99_ms": served_lat[1], "mean_ms": st["mean_ms"],
                       "batches": st["batches"] - s0["batches"], "mean_jobs_per_batch": st["mean_jobs_per_batch"],
                       "evictions": st["evictions"], "loads": st["loads"], "failed": st["failed"],
                       "bf16_vs_f32_max_rel_err": max(errs),
                       "saturated_value": n_tracks / sat_s,
                       "saturated_mean_jobs_per_batch": (st_sat["mean_jobs_per_batch"] * st_sat["batches"] -
                                                         st["mean_jobs_per_batch"] * st["batches"]) /
                                                        max(1, st_sat["batches"] - st["batches"])},
            "reduced_budget": small,
            "baseline_fp32_one_at_a_time": base,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": int(n_tracks * w.K * 8 / len(reqs)),
                    "d2h_bytes_per_step": int(n_tracks * 4 / len(reqs))},
            "gpu_launches": None,
            "clocks": clk.summary(),
            "cpu_baseline": None}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "served":
        run_served(args)
    elif args.workload == "chirp":
        run_chirp(args)
    elif args.workload == "tpl_search":
        run_tpl_search(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
