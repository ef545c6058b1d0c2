// Host side of the fused statistic kernel: tiling of the jobs, window sums, launch shape
// (staging slots, segments per slot, band capacity, tile size) and shared-memory layout, and
// the ordered sum of partial statistics when a launch splits its segments over several tiles.
#include <algorithm>
#include <atomic>

#include "eval_kernel.cuh"

namespace tfs {

static std::atomic<unsigned long long> g_wait_ns{2000000000ull};
static std::atomic<int> g_hold{0};
uint64_t eval_wait_ns() { return g_wait_ns.load(); }
int eval_hold() { return g_hold.load(); }
void set_eval_wait(uint64_t ns, int hold) {
  g_wait_ns.store(ns);
  g_hold.store(hold);
}

// Partial sums of tiles that cover a segment range, added in range order into the statistic.
struct PartJob {
  const double* part;  // [S][N]
  float* stat;        // [N]
  long long N;
  int S;
};
struct PartArgs {
  PartJob jobs[kMaxJobs];
  long long start[kMaxJobs + 1];
  int n;
};
static __global__ void sum_parts_kernel(const __grid_constant__ PartArgs p) {
  const long long total = p.start[p.n];
  int j = 0;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    while (g >= p.start[j + 1]) ++j;
    const PartJob& J = p.jobs[j];
    const long long t = g - p.start[j];
    double v = 0.0;
    for (int q = 0; q < J.S; ++q) v += J.part[(size_t)q * J.N + t];
    J.stat[t] = (float)v;
  }
}

// Tracks that one round of full tiles over all SMs holds (a single job's launch cuts its
// tracks into whole rounds of equal tiles of at most this many tracks per SM).
long long eval_round_tracks(int KP, bool cuts, int tile_div) {
  const long long R = r_of(KP, cuts, false);
  return (long long)kCons * R / std::max(1, std::min(tile_div, 8)) * sm_count();
}

template <int MJ>
static int launch_eval_jobs(const EvalLaunch& L, const EvalTuning& tune, cudaStream_t st) {
  int KP = 0;
  for (int i = 0; i < L.n_jobs; ++i) KP = std::max(KP, L.jobs[i].sp->KP);
  const bool cuts = L.jobs[0].cuts != 0;
  // tracks per consumer thread: the small class when the launch holds less than one round of
  // large tiles (tuning: 1 large, 2 small, 0 automatic); the verification launch keeps the large
  bool bins = false;
  long long n_all = 0;
  for (int i = 0; i < L.n_jobs; ++i) {
    bins = bins || L.jobs[i].bins_out != nullptr;
    n_all += L.jobs[i].N;
  }
  const bool small = !bins && (tune.rsel == 2 ||
                               (tune.rsel == 0 && n_all < (long long)sm_count() * kCons * r_of(KP, cuts, false)));
  const int R = r_of(KP, cuts, small);
  const int nsp = segrow_floats(KP, cuts);

  EvalArgs<MJ> a{};
  a.tie_count = L.tie_count;
  a.tie_track = reinterpret_cast<long long*>(L.tie_track);
  a.tie_seg = L.tie_seg;
  a.tie_cap = L.tie_cap;
  a.status = L.status;
  a.dbg = L.dbg;
  a.wait_ns = eval_wait_ns();
  a.hold = eval_hold();
  a.nsp = nsp;
  const long long tile = (long long)kCons * R / std::max(1, std::min(tune.tile_div, 8));
  // A single job of more than one round of tiles whose last round would run on few SMs: its last
  // tiles' segments are split over several tiles (whole 32-segment blocks each, partial sums
  // added in segment order), so that the last round's work spreads over the SMs.  Two jobs of one
  // launch: the full rounds, then the tail.  (Not with tie reports, whose track indices are those
  // of one job, nor for the verification launch.)
  if (MJ == 1 && L.n_jobs == 1 && !bins && L.tie_cap == 0 && L.jobs[0].split == 0) {
    const EvalJob& E = L.jobs[0];
    const long long sms = sm_count();
    const long long ntj = (E.N + tile - 1) / tile;
    const long long full = ntj / sms * sms, rem = ntj - full;
    const int n_seg = (int)E.table->n_seg;
    if (full > 0 && rem > 0) {
      const int S = (int)std::min<long long>(8, sms / rem);
      const int chunk = ((n_seg + S - 1) / std::max(S, 1) + kSegTile - 1) / kSegTile * kSegTile;
      const int S2 = S >= 2 ? (n_seg + chunk - 1) / chunk : 1;
      if (S2 >= 2) {
        EvalJob J2[2] = {E, E};
        const int64_t nA = full * tile;
        J2[0].N = nA;
        J2[1].N = E.N - nA;
        J2[1].coeffs = E.coeffs + nA * E.basis->K;
        J2[1].f_ref = E.f_ref ? E.f_ref + nA : nullptr;
        J2[1].stat = E.stat + nA;
        J2[1].split = S2;
        J2[0].split = 1;
        EvalLaunch L2 = L;
        L2.jobs = J2;
        L2.n_jobs = 2;
        return launch_eval_jobs<kMaxJobs>(L2, tune, st);
      }
    }
  }
  long long nt = 0;
  int seg_max = 0, qpitch_max = 0;
  size_t part_floats = 0;
  bool split_jobs = false;
  for (int i = 0; i < L.n_jobs; ++i) split_jobs = split_jobs || L.jobs[i].split > 1;
  for (int i = 0; i < L.n_jobs; ++i) {
    const EvalJob& E = L.jobs[i];
    const tfs_table* tb = E.table;
    if (E.sp->KP != KP || E.sp->nsp != nsp) {
      set_error("internal: job %d has %d coefficient slots, launch %d", i, E.sp->KP, KP);
      return TFS_ERR_INVALID_ARG;
    }
    if ((E.cuts != 0) != cuts || (cuts && !E.sp->cuts)) {
      set_error("internal: jobs with and without segment cuts in one launch");
      return TFS_ERR_INVALID_ARG;
    }
    JobDesc& D = a.jobs[i];
    int rc = wsum_get(tb, E.m, st, &D.q, &D.qpitch);
    if (rc) return rc;
    D.U = E.basis->U;
    D.segp = E.sp->segp;
    D.dmax = E.sp->dmax;
    D.umax = E.sp->umax;
    D.coeffs = E.coeffs;
    D.f_ref = E.f_ref;
    D.stat = E.stat;
    D.bins_out = E.bins_out;
    D.N = E.N;
    D.T = tb->T_sft;
    D.n_seg = (int)tb->n_seg;
    D.n_bin = (int)tb->n_bin;
    D.m = E.m;
    D.K = E.basis->K;
    D.alpha_mid = E.sp->alpha_mid;
    D.emax = E.sp->emax;
    D.gmax = E.sp->gmax;
    // tiles of equal size; a single job gets a whole number of rounds over the SMs (or, when
    // small, one tile per SM), so that no round runs on a few SMs alone
    long long ntj = (E.N + tile - 1) / tile;
    if (L.n_jobs == 1 && E.N > 0) {
      const long long sms = sm_count();
      if (ntj < sms) ntj = std::min<long long>(sms, (E.N + 255) / 256);
      else ntj = (ntj + sms - 1) / sms * sms;
    }
    const long long tt = ntj > 0 ? (E.N + ntj - 1) / ntj : tile;
    D.tile_tracks = (int)tt;
    D.seg_split = 1;
    D.seg_chunk = (int)tb->n_seg;
    D.part = nullptr;
    if (E.split > 1) {
      D.seg_chunk = ((D.n_seg + E.split - 1) / E.split + kSegTile - 1) / kSegTile * kSegTile;
      D.seg_split = (D.n_seg + D.seg_chunk - 1) / D.seg_chunk;
      if (D.seg_split > 1) part_floats += (size_t)D.seg_split * D.N;
    }
    a.tile_start[i] = (int)nt;
    nt += (tt > 0 ? (E.N + tt - 1) / tt : 0) * D.seg_split;
    seg_max = std::max(seg_max, (int)tb->n_seg);
    qpitch_max = std::max(qpitch_max, D.qpitch);
  }
  if (nt == 0) return TFS_OK;
  // Few track tiles (small jobs): split the jobs' segments over several tiles so that every
  // SM gets work; the tiles' partial sums are added in segment order by a second small kernel.
  // A tile's time grows with its segments, so the split balances them: the longest tile gets
  // the fewest whole 32-segment blocks for which all tiles still fit one per SM (so a job of
  // many segments takes more tiles than a short one), and no tile has fewer than 16 segments.
  const long long sms_all = sm_count();
  if (!bins && nt < sms_all && !split_jobs) {
    long long work = 0;  // track tiles x segments
    int seg_max_all = 1;
    for (int i = 0; i < L.n_jobs; ++i) {
      const JobDesc& D = a.jobs[i];
      const long long ntj = D.N > 0 ? (D.N + D.tile_tracks - 1) / D.tile_tracks : 0;
      work += ntj * D.n_seg;
      seg_max_all = std::max(seg_max_all, D.n_seg);
    }
    const auto split_of = [](int n_seg, long long cap) {
      return (int)std::max<long long>(1, std::min<long long>((n_seg + cap - 1) / cap, n_seg / 16));
    };
    long long cap = std::max<long long>(kSegTile, (work + sms_all - 1) / sms_all);
    cap = (cap + kSegTile - 1) / kSegTile * kSegTile;
    for (; cap < seg_max_all; cap += kSegTile) {
      long long units = 0;
      for (int i = 0; i < L.n_jobs; ++i) {
        const JobDesc& D = a.jobs[i];
        const long long ntj = D.N > 0 ? (D.N + D.tile_tracks - 1) / D.tile_tracks : 0;
        const int Sj = split_of(D.n_seg, cap);
        const int chunk = ((D.n_seg + Sj - 1) / Sj + kSegTile - 1) / kSegTile * kSegTile;
        units += ntj * ((D.n_seg + chunk - 1) / chunk);
      }
      if (units <= sms_all) break;
    }
    if (cap < seg_max_all) {
      nt = 0;
      part_floats = 0;
      for (int i = 0; i < L.n_jobs; ++i) {
        JobDesc& D = a.jobs[i];
        const long long ntj = D.N > 0 ? (D.N + D.tile_tracks - 1) / D.tile_tracks : 0;
        const int Sj = split_of(D.n_seg, cap);
        // chunks of whole 32-segment blocks: the FP32 block sums are those of an unsplit launch
        D.seg_chunk = ((D.n_seg + Sj - 1) / Sj + kSegTile - 1) / kSegTile * kSegTile;
        D.seg_split = (D.n_seg + D.seg_chunk - 1) / D.seg_chunk;
        if (D.seg_split > 1) part_floats += (size_t)D.seg_split * D.N;
        a.tile_start[i] = (int)nt;
        nt += ntj * D.seg_split;
      }
    }
  }
  if (nt > 0x7fffffffLL) {
    set_error("too many tracks for one launch");
    return TFS_ERR_INVALID_ARG;
  }
  a.n_jobs = L.n_jobs;
  a.tile_start[L.n_jobs] = (int)nt;
  a.n_tiles = (int)nt;

  // launch shape: slots (ring depth), segments per slot, band capacity
  const int NS = tune.slots > 0 ? std::max(2, std::min(tune.slots, kMaxSlots)) : 2;
  const int group = tune.group > 0 ? std::min(tune.group, kMaxGroup) : kMaxGroup;
  int pcap = tune.cap > 0 ? tune.cap : 2048;
  pcap = std::max(64, std::min(pcap, qpitch_max));
  pcap = (pcap + 3) / 4 * 4;
  // shared-memory layout
  const int BW = 2 * KP + 2;
  const int bcap = std::min(seg_max, kBandCap);
  a.bcap = bcap;
  size_t off = 8 * (2 * kMaxSlots + 8);  // mbarriers
  off = (off + 15) & ~(size_t)15;
  a.off_hdr = (int)off;   off += (size_t)NS * sizeof(SlotHdr);
  off = (off + 15) & ~(size_t)15;
  a.off_info = (int)off;  off += sizeof(WarpInfo) * kConsWarps + (size_t)kCons * 4 + (size_t)kConsWarps * BW * 4;
  off = (off + 15) & ~(size_t)15;
  a.off_flags = (int)off; off += 16 + kMaxSlots * 4 + (size_t)2 * BW * 4;
  off = (off + 15) & ~(size_t)15;
  a.off_band = (int)off;  off += (size_t)2 * 2 * bcap * 4;
  off = (off + 15) & ~(size_t)15;
  a.off_queue = (int)off; off += (size_t)kQT * kCons * 4;
  off = (off + 15) & ~(size_t)15;
  a.off_acc = (int)off;   off += (size_t)R * kCons * 4 * 4;  // corr, its error, tot, its error
  off = (off + 127) & ~(size_t)127;
  a.off_slots = (int)off;
  const size_t smem_cap = 227 * 1024;
  const long long avail = ((long long)smem_cap - (long long)off) / 4 / NS / 4 * 4;  // floats per slot
  const long long seg_need = pcap + kSent + nsp;
  long long scap = std::min<long long>(avail, (long long)group * seg_need);
  if (scap < seg_need) {
    // fit one segment of the largest band per slot
    const long long p2 = (scap - kSent - nsp) / 4 * 4;
    if (p2 < 64) {
      set_error("statistic kernel: %d staging slots do not fit in shared memory", NS);
      return TFS_ERR_INVALID_ARG;
    }
    pcap = (int)p2;
  }
  a.pcap = pcap;
  a.scap = (int)scap;
  a.nslots = NS;
  a.group = group;
  const size_t smem = off + (size_t)NS * scap * 4;
  a.smem_bytes = (int)smem;
  if (smem > smem_cap) {
    set_error("statistic kernel needs %zu bytes of shared memory", smem);
    return TFS_ERR_INVALID_ARG;
  }
  const int grid = (int)std::min<long long>(nt, (long long)sm_count());
  // the tile counter, then the helper warps' prologue columns, one block per CTA (stream-ordered
  // scratch)
  char* scratch = nullptr;
  TFS_CUDA(cudaMallocAsync((void**)&scratch, 256 + (size_t)grid * (KP + 1) * kCons * R * sizeof(float), st));
  a.tile_ctr = reinterpret_cast<int*>(scratch);
  a.cbuf = reinterpret_cast<float*>(scratch + 256);
  {
    const cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(int), st);
    if (e != cudaSuccess) {
      cudaFreeAsync(scratch, st);
      return cuda_fail(e, "tile counter");
    }
  }
  double* parts = nullptr;
  if (part_floats) {
    const cudaError_t e = cudaMallocAsync((void**)&parts, part_floats * sizeof(double), st);
    if (e != cudaSuccess) {
      cudaFreeAsync(scratch, st);
      return cuda_fail(e, "partial sums");
    }
    size_t o = 0;
    for (int i = 0; i < L.n_jobs; ++i) {
      JobDesc& D = a.jobs[i];
      if (D.seg_split > 1) {
        D.part = parts + o;
        o += (size_t)D.seg_split * D.N;
      }
    }
  }
  int rc;
  switch (KP) {
    case 2: rc = launch_kp<2, MJ>(a, bins, cuts, small, grid, smem, st); break;
    case 4: rc = launch_kp<4, MJ>(a, bins, cuts, small, grid, smem, st); break;
    case 6: rc = launch_kp<6, MJ>(a, bins, cuts, small, grid, smem, st); break;
    case 8: rc = launch_kp<8, MJ>(a, bins, cuts, small, grid, smem, st); break;
    case 16: rc = launch_kp<16, MJ>(a, bins, cuts, small, grid, smem, st); break;
    case 32: rc = launch_kp<32, MJ>(a, bins, cuts, small, grid, smem, st); break;
    default:
      set_error("unsupported coefficient slot count %d", KP);
      rc = TFS_ERR_INVALID_ARG;
  }
  if (rc == TFS_OK && parts) {
    PartArgs pa;
    pa.n = 0;
    pa.start[0] = 0;
    for (int i = 0; i < L.n_jobs; ++i) {
      const JobDesc& D = a.jobs[i];
      if (D.seg_split <= 1) continue;
      pa.jobs[pa.n] = PartJob{D.part, D.stat, D.N, D.seg_split};
      pa.start[pa.n + 1] = pa.start[pa.n] + D.N;
      ++pa.n;
    }
    const long long total = pa.start[pa.n];
    const int blocks = (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, sm_count() * 8));
    sum_parts_kernel<<<blocks, 256, 0, st>>>(pa);
    count_launch();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "partial sums");
  }
  if (parts) cudaFreeAsync(parts, st);
  cudaFreeAsync(scratch, st);
  return rc;
}

int launch_eval_shape(const EvalLaunch& L, const EvalTuning& tune, cudaStream_t st) {
  if (L.n_jobs <= 0) return TFS_OK;
  if (L.n_jobs == 1) return launch_eval_jobs<1>(L, tune, st);
  if (L.n_jobs > kMaxJobs) {
    set_error("at most %d jobs per launch", kMaxJobs);
    return TFS_ERR_INVALID_ARG;
  }
  return launch_eval_jobs<kMaxJobs>(L, tune, st);
}

}  // namespace tfs
