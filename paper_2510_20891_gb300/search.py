"""The paper's plunge-time search (Sec. II.D) as a client of the batched statistic.

* ``ChunkSearch``: data chunks of growing duration (0.1 yr, then 12 SFTs more per chunk,
  48 chunks), each the first n_obs rows of one table (a view, no copy) with the basis
  shifted by an integer number of segments so that its plunge falls at the chunk's end;
  the populations of all chunks are evaluated by one ``eval_batch`` call (one persistent
  launch per table dtype).  ``noise_moments`` gives the mean and standard deviation of the
  nearest-bin statistic under noise that normalise each duration.
* ``DESearch``: the population driver: 1024 candidates per chunk drawn uniformly in the
  prior box with the initial frequency drawn uniformly in [5e-4, 1e-2] Hz, the best 512
  kept, then iterations of track-space differential evolution without crossover
  (Eq. de_step, F_DE ~ U[0.3, 1.5]) with greedy acceptance inside the prior, every
  iteration one batched statistic launch plus the proposal and acceptance kernels.
  The gradient (Adam) half of the paper's iterations is not reproduced: the nearest-bin
  statistic is piecewise constant in the coefficients.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import (CHIRP_P, ChirpJob, Job, basis_view, check, ctable_view, eval_batch, eval_chirp_batch, lib,
               table_view, topk)

JULIAN_YEAR_S = 365.25 * 86400.0


def chunk_sizes(n_seg: int, T_sft: float, t_min_yr: float = 0.1, step: int = 12, n_chunks: int = 48):
    """Segments of each chunk: floor(0.1 yr / T_SFT) + 12 c, c = 0..47, those that fit."""
    n0 = int(math.floor(t_min_yr * JULIAN_YEAR_S / T_sft))
    return [n0 + step * c for c in range(n_chunks) if 1 <= n0 + step * c <= n_seg]


def noise_moments(n_segments: int, m: int, window: str = "hann"):
    """(mean, std) of the nearest-bin statistic over n_segments of Gaussian noise: per bin
    chi^2_2 (mean 2, variance 4), bins of one segment covarying by 4 |rho_d|^2 (periodic
    Hann: |rho_1|^2 = 4/9, |rho_2|^2 = 1/36; rectangular: 0), segments independent."""
    corr = (0.0, 4.0 / 9.0, 1.0 / 36.0) if window == "hann" else (0.0, 0.0, 0.0)
    width = 2 * m + 1
    var = float(width)
    for d in range(1, min(width, 3)):
        var += 2.0 * (width - d) * corr[d]
    return 2.0 * width * n_segments, math.sqrt(4.0 * var * n_segments)


class ChunkSearch:
    """Chunks of one table (views) with their shifted bases.  With a chirp table (the same
    strain's linear-chirp table) the chunks can also be evaluated with the paper's
    linear-chirp statistic (``statistic="chirp"``)."""

    def __init__(self, table, basis, sizes=None, chirp_table=None, P: int = CHIRP_P):
        self.table, self.basis = table, basis
        ref = table if table is not None else chirp_table
        self.sizes = list(sizes) if sizes is not None else chunk_sizes(ref.n_seg, ref.T_sft)
        self.tables = [table_view(table, 0, n) for n in self.sizes] if table is not None else None
        self.ctables = [ctable_view(chirp_table, 0, n) for n in self.sizes] if chirp_table is not None else None
        self.bases = [basis_view(basis, basis.n_seg - n, n) for n in self.sizes]
        self.P = P

    def jobs(self, coeffs, f_ref=None, m: int = 0, topk: int = 0, segment_cuts: bool = False, stats=None,
             statistic: str = "nearest"):
        """One job per chunk; coeffs (and f_ref, stats) are per-chunk CUDA tensors."""
        out = []
        for i, c in enumerate(coeffs):
            fr = f_ref[i] if f_ref is not None else None
            st = stats[i] if stats is not None else None
            if statistic == "chirp":
                out.append(ChirpJob(self.ctables[i], self.bases[i], c, fr, P=self.P, segment_cuts=segment_cuts,
                                    stat=st))
            else:
                out.append(Job(self.tables[i], self.bases[i], c, fr, m=m, topk=topk, stat=st,
                               segment_cuts=segment_cuts))
        return out

    def evaluate(self, coeffs, f_ref=None, m: int = 0, topk: int = 0, segment_cuts: bool = False, stats=None,
                 dev_status=None, stream=None, statistic: str = "nearest"):
        """All chunks' statistics in one batched call; returns the jobs (their .stat; .top_* for the
        nearest-bin statistic).  The linear-chirp statistic ignores m, topk and dev_status."""
        jobs = self.jobs(coeffs, f_ref, m, topk, segment_cuts, stats, statistic)
        if statistic == "chirp":
            eval_chirp_batch(jobs, stream=stream)
        else:
            eval_batch(jobs, dev_status=dev_status, stream=stream)
        return jobs

    def launch(self, jobs, statistic: str, dev_status=None, stream=None):
        if statistic == "chirp":
            eval_chirp_batch(jobs, stream=stream)
        else:
            eval_batch(jobs, dev_status=dev_status, stream=stream)

    def moments(self, m: int, window: str = "hann"):
        return [noise_moments(n, m, window) for n in self.sizes]


@dataclasses.dataclass
class DEResult:
    coeffs: list            # per chunk: best walker's coefficients [K] (numpy)
    stat: np.ndarray        # per chunk: its statistic
    normalised: np.ndarray  # per chunk: (stat - mean) / std under noise
    evaluations: int        # statistic evaluations made
    seconds: float          # wall time of the whole search (device synchronised)


class DESearch:
    """Differential-evolution population search over the chunks of a ChunkSearch."""

    def __init__(self, search: ChunkSearch, lo, hi, m: int = 0, n_init: int = 1024, n_walkers: int = 512,
                 f_start=(5e-4, 1e-2), seed: int = 0, graph: bool = True, segment_cuts: bool = False,
                 statistic: str = "nearest"):
        self.s, self.m = search, m
        self.lo, self.hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
        self.n_init, self.n_walkers = n_init, n_walkers
        self.f_start = f_start
        self.rng = np.random.default_rng(seed)
        self.K = self.lo.size
        self.graph = graph
        self.cuts = segment_cuts  # the paper's exclusions (Sec. II.B, II.D)
        self.statistic = statistic  # "nearest" (nearest-bin power sums) or "chirp" (the paper's S_alpha)
        self.uncounted_launches = 0  # kernels of graph replays beyond the captured one (set by run)
        self.t_setup = self.t_iter = 0.0  # wall seconds of the last run's set-up and iterations
        self.population = None  # the last run's walkers [n_chunks * n_walkers, K] (device)
        self.trial_jobs = None  # the last run's batch of trial walkers (its last iteration's proposals)

    def _initial(self, U_chunk):
        """n_init candidates uniform in the prior box, each track shifted by a constant so that
        its first-segment frequency is uniform in f_start, then projected back onto the
        chunk's basis (least squares)."""
        c = self.lo + (self.hi - self.lo) * self.rng.random((self.n_init, self.K))
        f0 = c @ U_chunk[:, 0]
        target = self.rng.uniform(*self.f_start, self.n_init)
        ones_c = np.linalg.lstsq(U_chunk.T, np.ones(U_chunk.shape[1]), rcond=None)[0]
        return c + (target - f0)[:, None] * ones_c[None, :]

    def run(self, n_iter: int = 525, stream=None, U_full=None):
        import time

        import torch

        s, K, W = self.s, self.K, self.n_walkers
        n_ch = len(s.sizes)
        if U_full is None:
            U_full, *_ = s.basis.to_host()
        dev = torch.device("cuda")
        L = lib()
        t0 = time.perf_counter()
        # initial population, best n_walkers per chunk
        init = [torch.tensor(self._initial(U_full[:, U_full.shape[1] - n:]), device=dev) for n in s.sizes]
        if self.statistic == "chirp":
            jobs = s.evaluate(init, segment_cuts=self.cuts, stream=stream, statistic="chirp")
            tops = [topk(j.stat, W, stream=stream) for j in jobs]
        else:
            jobs = s.evaluate(init, m=self.m, topk=W, segment_cuts=self.cuts, stream=stream)
            tops = [(j.top_idx, j.top_val) for j in jobs]
        c = torch.cat([init[i][tops[i][0]] for i in range(n_ch)])               # [n_ch W, K]
        st = torch.cat([tops[i][1] for i in range(n_ch)]).contiguous()
        evals = n_ch * self.n_init
        lo = torch.tensor(self.lo, device=dev)
        hi = torch.tensor(self.hi, device=dev)
        ct = torch.empty_like(c)
        s_trial = torch.empty_like(st)
        inp = torch.empty(n_ch * W, dtype=torch.int32, device=dev)
        views = [ct[i * W:(i + 1) * W] for i in range(n_ch)]
        stats = [s_trial[i * W:(i + 1) * W] for i in range(n_ch)]
        trial_jobs = s.jobs(views, m=self.m, stats=stats, segment_cuts=self.cuts, statistic=self.statistic)
        self.trial_jobs = trial_jobs
        # the random draws of every iteration (r1 != r2 != t within the walker's own chunk,
        # F_DE ~ U[0.3, 1.5]) come from a counter-based generator on the device, keyed by one
        # seed and an iteration number that each draw advances
        n = n_ch * W
        seed = int(self.rng.integers(0, 1 << 63))
        it_d = torch.zeros(1, dtype=torch.int32, device=dev)
        r1_b = torch.empty(n, dtype=torch.int32, device=dev)
        r2_b = torch.empty(n, dtype=torch.int32, device=dev)
        F_b = torch.empty(n, dtype=torch.float32, device=dev)
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        side = torch.cuda.Stream() if stream is None else stream

        def iteration(strm):
            sp = strm.cuda_stream
            check(L.tfs_de_draw(seed, it_d.data_ptr(), n_ch, W, 0.3, 1.5, r1_b.data_ptr(), r2_b.data_ptr(),
                                F_b.data_ptr(), sp))
            check(L.tfs_de_propose(c.data_ptr(), n, K, r1_b.data_ptr(), r2_b.data_ptr(), F_b.data_ptr(),
                                   lo.data_ptr(), hi.data_ptr(), ct.data_ptr(), inp.data_ptr(), sp))
            s.launch(trial_jobs, self.statistic, dev_status=status, stream=sp)
            check(L.tfs_de_accept(c.data_ptr(), st.data_ptr(), ct.data_ptr(), s_trial.data_ptr(), inp.data_ptr(),
                                  n, K, sp))

        self.t_setup = time.perf_counter() - t0  # initial population, its selection, buffers
        t_it = time.perf_counter()
        if n_iter > 0:
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                graph = None
                if self.graph:
                    # one draw + propose + batched statistic + accept, captured once and replayed
                    # (the library counts the captured kernels once; replays pass it by)
                    graph = torch.cuda.CUDAGraph()
                    k0 = L.tfs_kernel_launches()
                    with torch.cuda.graph(graph, stream=side):
                        iteration(side)
                    per_iter = L.tfs_kernel_launches() - k0
                    self.uncounted_launches = per_iter * (n_iter - 1)
                for it in range(n_iter):
                    if graph is not None:
                        graph.replay()
                    else:
                        iteration(side)
                    evals += n
            torch.cuda.current_stream().wait_stream(side)
            torch.cuda.synchronize()
            if int(status.item()) != 0:
                raise RuntimeError("a bounded device wait gave up during the search")
        torch.cuda.synchronize()
        self.t_iter = time.perf_counter() - t_it  # the iterations (capture included), synchronised
        secs = time.perf_counter() - t0
        self.population = c
        st_h = st.cpu().numpy().reshape(n_ch, W)
        c_h = c.cpu().numpy().reshape(n_ch, W, K)
        best = st_h.argmax(axis=1)
        stat = st_h[np.arange(n_ch), best].astype(np.float64)
        if self.statistic == "chirp":
            norm = np.full(n_ch, np.nan)  # no closed form for the linear-chirp statistic's noise moments
        else:
            mom = np.array(s.moments(self.m))
            norm = (stat - mom[:, 0]) / mom[:, 1]
        return DEResult([c_h[i, best[i]] for i in range(n_ch)], stat, norm, evals, secs)
