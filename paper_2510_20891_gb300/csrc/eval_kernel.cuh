// Fused track evaluation + gather + reduction for the semi-coherent statistic
// (paper Sec. II.B Eq. det_stat, nearest-bin reading with +-m neighbours;
// tracks from the SVD basis of Sec. II.C).
//
// Persistent, warp-specialised kernel.  One CTA per SM walks a list of tiles
// (static round-robin); a tile is 256*R tracks of one job, a job is one
// dataset (table, basis, batch of tracks), so datasets of different shapes
// run in one launch.  Three warpgroups:
//
//   producer warpgroup (128 threads, registers lowered with setmaxnreg)
//     * at a tile start, all 128 threads compute, from the tile's coefficient
//       box, a rigorous interval of the bins the tile can touch in every
//       segment (the "band");
//     * warp 0 (the stager) stages, segment after segment, the band of table
//       row alpha into a staging slot with a 1-D bulk copy (cp.async.bulk)
//       completing on an mbarrier;
//     * warps 1-3 (the builders) turn staged bands into window sums
//           Q[b] = sum_{j=-m..m} P[alpha][b+j]      (FP32, fixed order)
//       with 16-byte vector loads and lane shuffles and signal the Q slot;
//       builder warp w takes segments w, w+3, ..., so each warp's per-segment
//       synchronisation latency hides behind the other two warps' work;
//   three consumer warpgroups (384 threads, registers raised with setmaxnreg)
//     per segment, each thread evaluates x = f T_SFT for its R tracks in FP32,
//           y = (x_mid - Bw) + sum_k c_k D_k,alpha,    b = Bw + rint(y),
//     (B = rint(x_mid), x_mid an FP64 per-track constant) and adds Q[b] with a
//     single shared load.  Pairs within a warp-uniform error bound g of a
//     half-integer, and pairs whose centre falls outside the staged band, go
//     to the thread's own queue and are recomputed at the end of the tile in
//     the FP64 operation order of the oracle (separately rounded products and
//     sums): every bin equals the FP64 bin exactly, ties included.
//
// Inside a tile the roles meet only on mbarriers (staging ring full/empty,
// Q ring full/empty, per-tile box hand-off); the consumer warps run up to kNQ
// segments apart.  FP32 sums are flushed to a second accumulator every 32
// segments; fix-up contributions accumulate separately in segment order.  The
// result is deterministic for a given launch; which pairs take the fix-up path
// depends on the warp's base bin and decision limit and on the tile's band, so
// a track's FP32 rounding (never its bins) can change with its tile neighbours.
// Every wait is bounded (2 s) and warp-uniform; after a timeout every role
// keeps iterating without work (so barriers stay matched) and the call
// returns TFS_ERR_TIMEOUT.
#pragma once

#include "tfs_internal.cuh"

namespace tfs {

template <int DT>
struct Store;
template <>
struct Store<TFS_F32> {
  using T = float;
  static constexpr int esize = 4;
  static constexpr bool scaled = false;
  __device__ static float ld(const T* p) { return *p; }
};
template <>
struct Store<TFS_BF16> {
  using T = __nv_bfloat16;
  static constexpr int esize = 2;
  static constexpr bool scaled = false;
  __device__ static float ld(const T* p) { return __bfloat162float(*p); }
};
template <>
struct Store<TFS_F16> {
  using T = __half;
  static constexpr int esize = 2;
  static constexpr bool scaled = false;
  __device__ static float ld(const T* p) { return __half2float(*p); }
};
template <>
struct Store<TFS_F8E4M3> {
  using T = __nv_fp8_e4m3;
  static constexpr int esize = 1;
  static constexpr bool scaled = true;
  __device__ static float ld(const T* p) { return static_cast<float>(*p); }
};

constexpr int kProd = 128;            // producer warpgroup: stager warp + 3 builder warps
constexpr int kBuildWarps = kProd / 32 - 1;  // builder warps; warp w builds segments w, w+3, ...
constexpr int kCons = 384;            // three consumer warpgroups
constexpr int kThreads = kProd + kCons;
constexpr int kConsWarps = kCons / 32;
constexpr int kLaunchRegs = (65536 / kThreads) & ~7;  // 128 registers per thread at launch
constexpr int kProdRegs = 64;         // setmaxnreg targets: 128*64 + 384*144 <= 512*128
constexpr int kConsRegs = 144;
static_assert(kProd * kProdRegs + kCons * kConsRegs <= kThreads * kLaunchRegs, "register split exceeds the launch");
constexpr int kNQ = 4;                // window-sum (Q) slots
constexpr int kNP = 4;                // staging slots
constexpr int kQT = 24;               // fix-up queue entries per consumer thread
constexpr int kPadL = 16;             // zero elements before the staged band in a staging slot
constexpr int kSegTile = 32;          // FP32 partial sums are flushed every kSegTile segments
constexpr int kBandCap = 2048;        // segments whose bands are precomputed per tile
constexpr int kTrunc = 1 << 30;       // flag in a band length: the band was cut to the slot capacity

struct JobDesc {
  const void* table;
  const float* scales;
  const double* U;      // [K][n_seg]
  const float* segp;    // [n_seg][nsp]
  const float* dmax;    // [KP]
  const float* umax;    // [KP]
  const double* coeffs;
  const double* f_ref;
  float* stat;
  int* bins_out;        // [N][n_seg] (BINS instantiations); INT_MIN / INT_MAX: window wholly below / above
  long long N;
  double T;
  int n_seg, n_bin, row_stride, m, K, alpha_mid;
  int seg_resident;     // segp (and scales) copied to shared memory for this job's tiles
  int tile_tracks;      // tracks per tile (<= consumer threads * R); the last tile may hold fewer
  const float* emax;    // [KP] segment-cut launches: max |E_k|, max |G_k| (see SegParams)
  const float* gmax;
  int seg_split;        // tiles per track range, each over seg_chunk consecutive segments
  int seg_chunk;
  float* part;          // [seg_split][N] partial sums when seg_split > 1 (summed in order afterwards)
};


constexpr double kFLowHz = 0x1.4b96be9c2da2cp-12;  // 10^-3.5 Hz, the nearest double
constexpr double kFdotLow = 1e-13;                 // Hz/s

template <int MJ>
struct EvalArgs {
  unsigned long long* tie_count;
  long long* tie_track;
  int* tie_seg;
  int tie_cap;
  int* status;
  unsigned long long* dbg;  // self-check record (TFS_DEBUG_CHECKS builds)
  int smem_bytes;
  int nsp;       // floats per segment row of segp (launch-wide)
  int qcap;      // floats per Q slot (>= kPadL + pcap + vector tail)
  int pcap;      // table elements of band per staging slot (multiple of 16 bytes)
  int n_tiles;
  int n_jobs;
  // shared-memory carve-up (byte offsets)
  int off_qhdr, off_red, off_flags, off_band, off_seg, off_queue, off_acc, off_q, off_p;
  int tile_start[MJ + 1];  // first tile of each job (prefix sums), tile_start[n_jobs] = n_tiles
  JobDesc jobs[MJ];
};

// The tracks [tile0, tile0 + tile_tracks) and segments [s0, s1) of a tile of job j.
template <int MJ>
__device__ __forceinline__ void tile_range(const EvalArgs<MJ>& a, const JobDesc& J, int tile, int j,
                                           long long* tile0, int* sp, int* s0, int* s1) {
  const int local = tile - a.tile_start[j];
  const int tt = local / J.seg_split;
  *sp = local - tt * J.seg_split;
  *tile0 = (long long)tt * J.tile_tracks;
  *s0 = *sp * J.seg_chunk;
  *s1 = min(J.n_seg, *s0 + J.seg_chunk);
}

struct QHdr {
  int qbase;     // window centre held at q[ws_lo]
  int qn;        // valid centres from there on; q[ws_lo + qn] holds 0
  int ws_lo;     // first valid window start in the slot
  int complete;  // every reachable centre whose window overlaps the table has its sum in Q
};

// Packed pairs of FP32 values (two tracks at once): each lane of fma/add/sub.rn.f32x2 is one
// IEEE round-to-nearest operation, the same as the scalar instruction on that value.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 f2pack(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2split(f32x2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 f2fma(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ f32x2 f2add(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f32x2 f2sub(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
// Two packed pairs (16 bytes) from shared memory.  The _v form is volatile: it is re-issued
// at every use instead of being hoisted into registers held across the loop.
__device__ __forceinline__ void lds_pair2(uint32_t addr, f32x2& lo, f32x2& hi) {
  asm("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(lo), "=l"(hi) : "r"(addr));
}
__device__ __forceinline__ void lds_pair2_v(uint32_t addr, f32x2& lo, f32x2& hi) {
  asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(lo), "=l"(hi) : "r"(addr));
}
__device__ __forceinline__ f32x2 lds_pair_v(uint32_t addr) {
  f32x2 v;
  asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(addr));
  return v;
}

#ifdef TFS_DEBUG_CHECKS
__device__ __forceinline__ bool dbg_ok(unsigned long long* dbg, bool cond, int where, long long i0, long long i1) {
  if (!cond && dbg) {
    if (atomicAdd(&dbg[0], 1ull) == 0ull) {
      dbg[1] = (unsigned long long)where;
      dbg[2] = (unsigned long long)i0;
      dbg[3] = (unsigned long long)i1;
    }
  }
  return cond;
}
#else
__device__ __forceinline__ bool dbg_ok(unsigned long long*, bool, int, long long, long long) { return true; }
#endif

// Window sum from the table in global memory; elements outside [0, n_bin) are 0.
// The additions run in the same order as the shared-memory window sums.
template <int DT>
__device__ __forceinline__ float window_global(const JobDesc& J, int seg, int lo, int W, float scale) {
  using S = Store<DT>;
  const typename S::T* row = static_cast<const typename S::T*>(J.table) + (size_t)seg * J.row_stride;
  float v = 0.f;
  for (int j = 0; j < W; ++j) {
    const int k = lo + j;
    const float p = (k >= 0 && k < J.n_bin) ? S::ld(row + k) : 0.f;
    v += S::scaled ? p * scale : p;
  }
  return v;
}

template <int MJ>
__device__ __forceinline__ void report_tie(const EvalArgs<MJ>& a, long long t, int seg) {
  const unsigned long long i = atomicAdd(a.tie_count, 1ull);
  if (i < (unsigned long long)a.tie_cap) {
    a.tie_track[i] = t;
    a.tie_seg[i] = seg;
  }
}

// FP64 frequency of track t at segment seg in the oracle's operation order.
__device__ __forceinline__ double track_freq(const JobDesc& J, long long t, int seg) {
  double f = J.f_ref ? J.f_ref[t] : 0.0;
  const double* c = J.coeffs + t * (long long)J.K;
  for (int k = 0; k < J.K; ++k) f = __dadd_rn(f, __dmul_rn(c[k], J.U[(size_t)k * J.n_seg + seg]));
  return f;
}

// Segment exclusions of (track t, segment seg) in FP64, in the oracle's operation order
// (finite differences of the track at the segment midpoints; see segment_validity there).
static __device__ __noinline__ bool segment_excluded(const JobDesc& J, long long t, int seg, double f) {
  const int n = J.n_seg;
  const double T = J.T;
  double fd = 0.0, z = 0.0;
  if (n >= 2) {
    if (seg == 0) fd = __ddiv_rn(__dsub_rn(track_freq(J, t, 1), f), T);
    else if (seg == n - 1) fd = __ddiv_rn(__dsub_rn(f, track_freq(J, t, n - 2)), T);
    else fd = __ddiv_rn(__dsub_rn(track_freq(J, t, seg + 1), track_freq(J, t, seg - 1)), __dmul_rn(2.0, T));
  }
  if (n >= 3) {
    const int cc = seg == 0 ? 1 : (seg == n - 1 ? n - 2 : seg);
    const double fc = cc == seg ? f : track_freq(J, t, cc);
    const double dd = __dadd_rn(__dsub_rn(track_freq(J, t, cc + 1), __dmul_rn(2.0, fc)), track_freq(J, t, cc - 1));
    z = __dmul_rn(dd, __ddiv_rn(T, 6.0));
  }
  return z > 1.0 || f < kFLowHz || fd < kFdotLow;
}

// FP64 bin of (track t, segment seg) of job J in the oracle's operation order,
// and its window sum from global memory (0 for an excluded segment when CUTS).
template <int DT, bool BINS, bool CUTS, int MJ>
__device__ float exact_pair(const EvalArgs<MJ>& a, const JobDesc& J, long long t, int seg) {
  if (!dbg_ok(a.dbg, t >= 0 && t < J.N && seg >= 0 && seg < J.n_seg, 1, t, seg)) return 0.f;
  const double f = track_freq(J, t, seg);
  if (CUTS && segment_excluded(J, t, seg, f)) return 0.f;
  const double x = __dmul_rn(f, J.T);
  int* bo = BINS ? J.bins_out + t * (long long)J.n_seg + seg : nullptr;
  if (!isfinite(x)) {
    if (BINS) *bo = 0x7fffffff;
    return 0.f;
  }
  const double fl = floor(x);
  if (fabs(__dsub_rn(__dsub_rn(x, fl), 0.5)) <= 1e-9) report_tie(a, t, seg);
  const double z = __dadd_rn(x, 0.5);
  const int m = J.m;
  if (z < -(double)m || z >= (double)J.n_bin + (double)m) {
    if (BINS) *bo = z < 0.0 ? (int)0x80000000 : 0x7fffffff;
    return 0.f;
  }
  const int b = (int)floor(z);
  if (BINS) *bo = b;
  const float scale = Store<DT>::scaled ? J.scales[seg] : 1.f;
  return window_global<DT>(J, seg, b - m, 2 * m + 1, scale);
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ uint32_t mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done;
}
// Warp-uniform bounded wait.  Lane 0 alone polls (32 lanes polling one barrier flood the
// shared-memory pipe that the working warps need); once it sees the phase complete, every
// lane observes it too (acquire).  The timeout and abort decisions are lane 0's, broadcast
// to the warp.  Returns false at once after an abort.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* flags) {
  if (__any_sync(0xffffffffu, flags[0] != 0)) return false;
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    uint32_t done = 1;
    if ((threadIdx.x & 31) == 0) done = mbar_try(bar, parity);
    if (__shfl_sync(0xffffffffu, done, 0)) {
      (void)mbar_try(bar, parity);  // the phase cannot move on before this warp's own next arrival
      return true;
    }
    if ((it & 31) == 0) {
      int stop = 0;
      if ((threadIdx.x & 31) == 0) {
        const uint64_t now = global_ns();
        if (it == 0) t0 = now;
        stop = flags[0] != 0 || (it != 0 && now - t0 > kWaitLimitNs);
      }
      if (__shfl_sync(0xffffffffu, stop, 0)) {
        flags[0] = 1;
        return false;
      }
    }
  }
}
// Single-thread bounded wait.
__device__ __forceinline__ bool thread_wait(uint64_t* bar, uint32_t parity, volatile int* flags) {
  if (flags[0]) return false;
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 31) == 0) {
      const uint64_t now = global_ns();
      if (it == 0) t0 = now;
      else if (flags[0] != 0 || now - t0 > kWaitLimitNs) {
        flags[0] = 1;
        return false;
      }
    }
  }
}
__device__ __forceinline__ void prod_bar() {  // named barrier 1 among the producer warpgroup (warps may be diverged)
  asm volatile("barrier.sync 1, %0;" ::"n"(kProd) : "memory");
}
template <int N>
__device__ __forceinline__ void setmaxnreg_inc() {
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(N));
}
template <int N>
__device__ __forceinline__ void setmaxnreg_dec() {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(N));
}

// Convert the EPV table elements of one 16-byte vector to FP32 (dequantised).
template <int DT>
__device__ __forceinline__ void unpack16(const uint4 raw, float scale, float* out) {
  using S = Store<DT>;
  constexpr int EPV = 16 / S::esize;
  const typename S::T* e = reinterpret_cast<const typename S::T*>(&raw);
#pragma unroll
  for (int i = 0; i < EPV; ++i) {
    const float p = S::ld(e + i);
    out[i] = S::scaled ? p * scale : p;
  }
}

template <int MJ>
__device__ __forceinline__ int job_of(const EvalArgs<MJ>& a, int tile) {
  int j = 0;
  while (j + 1 < a.n_jobs && tile >= a.tile_start[j + 1]) ++j;
  return j;
}

// Band of staged table elements [blo, blo + blen) for segment row d of a tile whose
// coefficient box is [lo_k, hi_k] and base bins [bm, bx] (FP32 with a margin covering
// its rounding: the band only steers staging, bins outside it take the exact path).
// blen carries kTrunc when the band had to be cut to pcap elements.
template <int KP, int EALIGN>
__device__ __forceinline__ void band_of(const float* d, const float* blo_k, const float* bhi_k, int bm, int bx,
                                        int m, int n_bin, int row_stride, int pcap, int* out_lo, int* out_len) {
  int blo = 0, blen = 0;
  if (bm <= bx) {
    float lo = 0.f, hi = 0.f, mag = 0.f;
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      const float p1 = blo_k[k] * d[k], p2 = bhi_k[k] * d[k];
      lo += fminf(p1, p2);
      hi += fmaxf(p1, p2);
      mag += fmaxf(fabsf(p1), fabsf(p2));
    }
    const float fm = 4.f + 1e-5f * mag + 1e-6f * fmaxf(fabsf((float)bm), fabsf((float)bx));
    const float bl = fmaxf(floorf((float)bm + lo - fm) - 2 * m, 0.f);
    const float bh = fminf(floorf((float)bx + 1.f + hi + fm) + 2 * m, (float)(n_bin - 1));
    if (bl <= bh) {
      const int il = ((int)bl) & ~(EALIGN - 1);
      int ih = ((int)bh + EALIGN) & ~(EALIGN - 1);
      ih = min(ih, row_stride);
      blo = il;
      blen = ih - il > pcap ? (pcap | kTrunc) : ih - il;
    }
  }
  *out_lo = blo;
  *out_len = blen;
}

template <int DT, int KP, int R, bool BINS, bool CUTS, int MJ>
__global__ void __launch_bounds__(kThreads, 1) eval_stat_kernel(const __grid_constant__ EvalArgs<MJ> a) {
  constexpr bool kCutRegs = CUTS && KP <= 8;  // segment-cut forms held in registers
  using S = Store<DT>;
  using T = typename S::T;
  constexpr int EALIGN = 16 / S::esize;  // table elements per 16 bytes (= EPV)
  constexpr int RW = 2 * KP + 2;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  uint64_t* full_p = bars;                           // [kNP] staged copy landed (tx)
  uint64_t* empty_p = bars + kNP;                    // [kNP] its builder warp is done with the slot
  uint64_t* full_q = bars + 2 * kNP;                 // [kNQ] window sums ready (32 lanes of a builder warp)
  uint64_t* empty_q = bars + 2 * kNP + kNQ;          // [kNQ] consumers done with the slot (8 warps)
  uint64_t* tile_ready = bars + 2 * kNP + 2 * kNQ;   // [2] a tile's coefficient box is ready (8 warps)
  QHdr* qhdr = reinterpret_cast<QHdr*>(smem + a.off_qhdr);  // [kNQ], then [kNQ][nsp] floats of D
  float* qdseg = reinterpret_cast<float*>(smem + a.off_qhdr + kNQ * sizeof(QHdr));
  float* red = reinterpret_cast<float*>(smem + a.off_red);  // [2][kConsWarps][RW]
  volatile int* flags = reinterpret_cast<volatile int*>(smem + a.off_flags);  // [0] abort
  int* plo_s = reinterpret_cast<int*>(smem + a.off_flags) + 4;  // [kNP] band start per staging slot
  int* plen_s = plo_s + kNP;                                    // [kNP] band length
  float* box = reinterpret_cast<float*>(plen_s + kNP);          // [2*KP] floats, then 2 ints
  int* band = reinterpret_cast<int*>(smem + a.off_band);        // [kBandCap][2]
  float* segs = reinterpret_cast<float*>(smem + a.off_seg);     // resident segp [n_seg][nsp], scales [n_seg]
  uint32_t* queue = reinterpret_cast<uint32_t*>(smem + a.off_queue);  // [kQT][kCons]
  float* corr = reinterpret_cast<float*>(smem + a.off_acc);           // [R][kCons]
  float* tot = corr + R * kCons;                                      // [R][kCons]
  float* qslots = reinterpret_cast<float*>(smem + a.off_q);           // [kNQ][qcap]
  unsigned char* pslots = smem + a.off_p;                             // [kNP][pslot_bytes]
  const int pslot_bytes = (kPadL + a.pcap + EALIGN) * S::esize + a.nsp * 4;

  const int tid = threadIdx.x;
  const int lane = tid & 31;

  if (tid < 4) flags[tid] = 0;
  if (tid == 0) {
    for (int i = 0; i < kNP; ++i) {
      mbar_init(&full_p[i], 1);
      mbar_init(&empty_p[i], 1);
    }
    for (int i = 0; i < kNQ; ++i) {
      mbar_init(&full_q[i], 32);
      mbar_init(&empty_q[i], kConsWarps);
    }
    for (int i = 0; i < 2; ++i) mbar_init(&tile_ready[i], kConsWarps);
    fence_mbar_init();
  }
  // zero the left pads of the staging slots (they stand for bins < 0 when a band starts at bin 0)
  for (int s = 0; s < kNP; ++s) {
    T* sd = reinterpret_cast<T*>(pslots + (size_t)s * pslot_bytes);
    for (int i = tid; i < kPadL; i += kThreads) sd[i] = T(0.f);
  }
  __syncthreads();

  if (tid < kProd) {
    // ================================================================ producer warpgroup
    setmaxnreg_dec<kProdRegs>();
    const int pw = tid >> 5;  // 0: stager, 1..3: builders
    uint32_t p_seq = 0, b_base = 0;
    int cur_job = -1;
    int ltile = 0;
    for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++ltile) {
      const int j = job_of(a, tile);
      const JobDesc& J = a.jobs[j];
      const int n_seg = J.n_seg, m = J.m, W = 2 * m + 1;
      long long tile0_unused;
      int sp_unused, s0, s1;
      tile_range(a, J, tile, j, &tile0_unused, &sp_unused, &s0, &s1);
      const int ns = s1 - s0;  // this tile's segments
      // -------------------------------------------------------------- tile set-up (all 128)
      if (tid == 0) {
        if (thread_wait(&tile_ready[ltile & 1], (uint32_t)((ltile >> 1) & 1), flags)) {
          const float* rb = red + (ltile & 1) * kConsWarps * RW;
          int bm = 0x7fffffff, bx = -0x7fffffff;
          for (int k = 0; k < KP; ++k) {
            float lo = __int_as_float(0x7f800000), hi = -__int_as_float(0x7f800000);
            for (int w = 0; w < kConsWarps; ++w) {
              lo = fminf(lo, rb[w * RW + k]);
              hi = fmaxf(hi, rb[w * RW + KP + k]);
            }
            box[k] = lo;
            box[KP + k] = hi;
          }
          for (int w = 0; w < kConsWarps; ++w) {
            bm = min(bm, reinterpret_cast<const int*>(rb)[w * RW + 2 * KP]);
            bx = max(bx, reinterpret_cast<const int*>(rb)[w * RW + 2 * KP + 1]);
          }
          reinterpret_cast<int*>(box)[2 * KP] = bm;
          reinterpret_cast<int*>(box)[2 * KP + 1] = bx;
        }
      }
      __syncwarp();
      if (j != cur_job && J.seg_resident) {
        prod_bar();  // no producer thread still reads the previous job's resident rows or scales
        for (int i = tid; i < n_seg * a.nsp; i += kProd) segs[i] = J.segp[i];
        if (S::scaled)
          for (int i = tid; i < n_seg; i += kProd) segs[n_seg * a.nsp + i] = J.scales[i];
      }
      cur_job = j;
      prod_bar();
      const float* segrows = J.seg_resident ? segs : J.segp;
      const float* sscales = J.seg_resident ? segs + n_seg * a.nsp : J.scales;
      const int bm = reinterpret_cast<const int*>(box)[2 * KP];
      const int bx = reinterpret_cast<const int*>(box)[2 * KP + 1];
      if (ns <= kBandCap) {  // (band_of gives an in-range band for any box, even after an abort)
        for (int i = tid; i < ns; i += kProd) {
          int lo, len;
          band_of<KP, EALIGN>(segrows + (size_t)(s0 + i) * a.nsp, box, box + KP, bm, bx, m, J.n_bin,
                              J.row_stride, a.pcap, &lo, &len);
          band[2 * i] = lo;
          band[2 * i + 1] = len;
        }
      }
      prod_bar();
      if (pw == 0) {
        // ------------------------------------------------------------ stager warp
        for (int sg = s0; sg < s1; ++sg) {
          const int ps = (int)(p_seq % kNP);
          bool go = true;
          if (p_seq >= kNP) go = warp_wait(&empty_p[ps], ((p_seq / kNP) - 1u) & 1u, flags);
          else go = !__any_sync(0xffffffffu, flags[0] != 0);
          if (go && lane == 0) {
            int blo, blen;
            if (ns <= kBandCap) {
              blo = band[2 * (sg - s0)];
              blen = band[2 * (sg - s0) + 1];
            } else {
              band_of<KP, EALIGN>(segrows + (size_t)sg * a.nsp, box, box + KP, bm, bx, m, J.n_bin, J.row_stride,
                                  a.pcap, &blo, &blen);
            }
            plo_s[ps] = blo;
            plen_s[ps] = blen;
            blen &= kTrunc - 1;
            unsigned char* dst = pslots + (size_t)ps * pslot_bytes;
            uint32_t dbytes = (uint32_t)blen * S::esize;
            {
              const long long src_el = (long long)sg * J.row_stride + blo;
              const bool ok =
                  dbg_ok(a.dbg, (long long)a.off_p + (long long)(ps + 1) * pslot_bytes <= a.smem_bytes, 7, ps,
                         pslot_bytes) &&
                  dbg_ok(a.dbg, blo >= 0 && src_el + blen <= (long long)n_seg * J.row_stride, 8, src_el, blen) &&
                  dbg_ok(a.dbg,
                         ((a.off_p + (long long)ps * pslot_bytes) & 15) == 0 && (dbytes & 15) == 0 &&
                             ((src_el * S::esize) & 15) == 0 && ((pslot_bytes & 15) == 0),
                         9, ps, src_el);
              if (!ok) dbytes = 0;
            }
            fence_proxy_async_smem();  // the slot's previous contents were read through the generic proxy
            mbar_arrive_expect_tx(&full_p[ps], dbytes + (uint32_t)a.nsp * 4u);
            if (dbytes > 0)
              bulk_g2s(dst + kPadL * S::esize, static_cast<const T*>(J.table) + (size_t)sg * J.row_stride + blo,
                       dbytes, &full_p[ps]);
            bulk_g2s(dst + (size_t)(kPadL + a.pcap + EALIGN) * S::esize, J.segp + (size_t)sg * a.nsp,
                     (uint32_t)a.nsp * 4u, &full_p[ps]);
          }
          __syncwarp();
          ++p_seq;
        }
      } else {
        // ------------------------------------------------------------ builder warps
        // builder warp w builds the window sums of segments w, w + 3, w + 6, ...: the latency of
        // each warp's per-segment waits and set-up overlaps the other two warps' work
        for (int sg = s0 + pw - 1; sg < s1; sg += kBuildWarps) {
          const uint32_t gs = b_base + (uint32_t)(sg - s0);  // launch-wide segment sequence number
          const int ps = (int)(gs % kNP), qs = (int)(gs % kNQ);
          bool go = warp_wait(&full_p[ps], (gs / kNP) & 1u, flags);
          if (go && gs >= kNQ) go = warp_wait(&empty_q[qs], ((gs / kNQ) - 1u) & 1u, flags);
          if (go) {
            const int plo = plo_s[ps], plv = plen_s[ps];
            const int plen = plv & (kTrunc - 1);
            const unsigned char* src = pslots + (size_t)ps * pslot_bytes;
            // Window starts (slot coordinates) with a sum in Q: inside the staged band, plus the
            // windows that reach beyond the table, whose missing elements count as 0: into the
            // zero pad when the band starts at bin 0 (centres down to -m if 2m <= kPadL), and past
            // the band's end when it reaches the end of the table (centres up to n_bin - 1 + m).
            // Elements past the band always read as 0.  The band is "complete" when every centre
            // whose window overlaps the table and that the tile's tracks can reach has its sum in
            // Q; then a centre outside Q always has a window wholly outside the table.
            const bool at_end = plo + plen >= J.n_bin;
            const int ws_lo = plo == 0 ? max(kPadL - 2 * m, 0) : kPadL;
            const int ws_hi = kPadL + plen - (W - 1) + (at_end ? 2 * m : 0);
            const int qn = plen == 0 ? 0 : max(0, min(ws_hi, a.qcap - EALIGN) - ws_lo);
            const bool complete = !(plv & kTrunc) && (plo > 0 || 2 * m <= kPadL) && ws_hi <= a.qcap - EALIGN;
            const int nband = (kPadL + plen) / EALIGN;  // vectors of pad + band (plen is a multiple of EALIGN)
            float* q = qslots + (size_t)qs * a.qcap;
            const float scale = S::scaled ? sscales[sg] : 1.f;
            if (m <= 2) {
              // vector path: thread j sums the windows starting at its EPV elements, taking the next
              // 2m elements from the next lane (or, on a warp's last lane, from shared memory)
              const int nvec = (ws_lo + qn + EALIGN - 1) / EALIGN;
              const int nload = min((ws_lo + qn + 4 + EALIGN - 1) / EALIGN, kPadL / EALIGN + a.pcap / EALIGN + 1);
              // each pass: UV vectors (16 table elements) per thread, all loads issued first
              constexpr int UV = 16 / EALIGN;
              for (int v0 = 0; v0 < nvec; v0 += 32 * UV) {
                uint4 raw[UV];
#pragma unroll
                for (int u = 0; u < UV; ++u) {
                  const int vi = v0 + u * 32 + lane;
                  raw[u] = vi < nload && vi < nband ? reinterpret_cast<const uint4*>(src)[vi]
                                                    : make_uint4(0u, 0u, 0u, 0u);
                }
#pragma unroll
                for (int u = 0; u < UV; ++u) {
                  const int vi = v0 + u * 32 + lane;
                  float e[EALIGN + 4];
                  unpack16<DT>(raw[u], scale, e);
                  float nx[4];
#pragma unroll
                  for (int k = 0; k < 4; ++k) nx[k] = __shfl_down_sync(0xffffffffu, e[k], 1);
                  if (lane == 31) {
                    // the next vector belongs to the next pass: read it from shared memory, or
                    // take zeros past the band (the shuffle above returned this lane's own values)
                    const bool in_band = vi < nvec && vi + 1 < nband;
                    const T* tail = reinterpret_cast<const T*>(src) + (size_t)(in_band ? vi + 1 : 0) * EALIGN;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                      const float p = in_band ? S::ld(tail + k) : 0.f;
                      nx[k] = S::scaled ? p * scale : p;
                    }
                  }
#pragma unroll
                  for (int k = 0; k < 4; ++k) e[EALIGN + k] = nx[k];
                  if (vi < nvec) {
                    // compile-time window widths keep e[] in registers; same order: ((0 + e0) + e1) + ...
                    float out[EALIGN];
                    if (W == 1) {
#pragma unroll
                      for (int i = 0; i < EALIGN; ++i) out[i] = 0.f + e[i];
                    } else if (W == 3) {
#pragma unroll
                      for (int i = 0; i < EALIGN; ++i) out[i] = ((0.f + e[i]) + e[i + 1]) + e[i + 2];
                    } else {
#pragma unroll
                      for (int i = 0; i < EALIGN; ++i)
                        out[i] = ((((0.f + e[i]) + e[i + 1]) + e[i + 2]) + e[i + 3]) + e[i + 4];
                    }
                    float4* qv = reinterpret_cast<float4*>(q + (size_t)vi * EALIGN);
#pragma unroll
                    for (int i4 = 0; i4 < EALIGN / 4; ++i4)
                      qv[i4] = make_float4(out[4 * i4], out[4 * i4 + 1], out[4 * i4 + 2], out[4 * i4 + 3]);
                  }
                }
              }
            } else {
              const T* pb = reinterpret_cast<const T*>(src);
              for (int ws = ws_lo + lane; ws < ws_lo + qn; ws += 32) {
                float s = 0.f;
                for (int k = 0; k < W; ++k) {
                  const float p = ws + k < kPadL + plen ? S::ld(pb + ws + k) : 0.f;
                  s += S::scaled ? p * scale : p;
                }
                q[ws] = s;
              }
            }
            for (int i = lane; i < a.nsp; i += 32)
              qdseg[qs * a.nsp + i] =
                  reinterpret_cast<const float*>(src + (size_t)(kPadL + a.pcap + EALIGN) * S::esize)[i];
            __syncwarp();
            if (lane == 0) {
              q[ws_lo + qn] = 0.f;  // the sum every centre outside Q reads in the complete case
              QHdr h;
              h.ws_lo = ws_lo;
              h.qn = qn;
              h.qbase = plo - kPadL + ws_lo + m;  // centre of the window starting at ws_lo
              h.complete = complete ? 1 : 0;
              qhdr[qs] = h;
            }
            mbar_arrive(&full_q[qs]);  // every lane releases its own writes
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty_p[ps]);
          }
        }
      }
      b_base += (uint32_t)ns;
    }
  } else {
    // ================================================================ consumer warpgroups
    setmaxnreg_inc<kConsRegs>();
    const int ctid = tid - kProd;
    const int cwarp = ctid >> 5;
    uint32_t q_seq = 0;
    int ltile = 0;
    for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++ltile) {
      const int j = job_of(a, tile);
      const JobDesc& J = a.jobs[j];
      const int n_seg = J.n_seg, m = J.m, K = J.K;
      long long tile0;
      int sp, s0, s1;
      tile_range(a, J, tile, j, &tile0, &sp, &s0, &s1);
      const long long tend = min(J.N, tile0 + J.tile_tracks);
      const bool live = !__any_sync(0xffffffffu, flags[0] != 0);  // warp-uniform
      // -------------------------------------------------------------- tile prologue
      // Each track is evaluated relative to a warp-uniform base bin Bw (the FP64 mid-segment bin
      // of the warp's first track): y = (x_mid - Bw) + sum_k c_k D_k,alpha in FP32, and the bin
      // is Bw + rint(y).  One base per warp keeps a register per track free.
      // tracks in pairs for the packed FP32x2 arithmetic (an odd R gets an inactive partner):
      // track r is half (r & 1) of c2[r / 2][k] and y02[r / 2]
      constexpr int R2 = (R + 1) / 2;
      f32x2 c2[R2][KP];
      f32x2 y02[R2];
      float acc[R];
#pragma unroll
      for (int p = 0; p < R2; ++p) {
        y02[p] = f2pack(4194303.0f, 4194303.0f);
#pragma unroll
        for (int k = 0; k < KP; ++k) c2[p][k] = f2pack(0.f, 0.f);
      }
      // set half (r & 1) of a packed pair (r is a compile-time index after unrolling)
      auto put = [](f32x2& v, int half, float x) {
        float lo, hi;
        f2split(v, lo, hi);
        v = half ? f2pack(lo, x) : f2pack(x, hi);
      };
      auto get = [](f32x2 v, int half) {
        float lo, hi;
        f2split(v, lo, hi);
        return half ? hi : lo;
      };
      int Bw = 0;
      // warp-uniform decision limit: min over the warp's tracks of 1/2 - g; at most 1/2, so the
      // tracks that take the FP64 path for every pair (y = 1/2) are never decided in FP32
      float wlim = 0.5f;
      // segment cuts: warp-uniform margins of the second-order test (mz), the fdot test (mw)
      // and the low-frequency test (mf, against ylo = 10^-3.5 T_SFT - Bw in bin units)
      float mz = 0.f, mw = 0.f, mf = 0.f, ylo = 0.f;
      // ... as thresholds: included below zin / above win, fin; excluded above zex / below wex, fex
      float zin = 0.f, zex = 0.f, win = 0.f, wex = 0.f, fin = 0.f, fex = 0.f;
      unsigned cutm = 0u;  // tracks whose cuts are decided in FP32 (the others are always pending)
      bool zt = false;     // some track of the warp may reach the second-order cut
      int nq = 0;        // entries in this thread's fix-up queue
      if (live) {
        int bmin = 0x7fffffff, bmax = -0x7fffffff;
        unsigned inbox = 0u;  // tracks that enter the coefficient box (decided in FP32)
#pragma unroll
        for (int r = 0; r < R; ++r) {
          acc[r] = 0.f;
          put(y02[r / 2], r & 1, 0.f);
          corr[r * kCons + ctid] = 0.f;
          tot[r * kCons + ctid] = 0.f;
          const long long t = tile0 + ctid + r * kCons;
          const bool active = t < tend;
          double xm = 0.0;
          float eb = 0.f, ezt = 0.f, ewt = 0.f, zbt = 0.f;
          bool exact = false;
          if (active) {
            const double fr = J.f_ref ? J.f_ref[t] : 0.0;
            double f = fr;
            float A = 0.f, Um = fabsf((float)fr), Az = 0.f, Aw = 0.f;
            const double* cp = J.coeffs + t * (long long)K;
#pragma unroll
            for (int k = 0; k < KP; ++k) {
              const double cd = (k < K) ? cp[k] : 0.0;
              if (k < K) f = fma(cd, J.U[(size_t)k * n_seg + J.alpha_mid], f);
              const float cf = (float)cd;
              put(c2[r / 2][k], r & 1, cf);
              A = fmaf(fabsf(cf), J.dmax[k], A);
              Um = fmaf(fabsf(cf), J.umax[k], Um);
              if (CUTS) {
                Az = fmaf(fabsf(cf), J.emax[k], Az);
                Aw = fmaf(fabsf(cf), J.gmax[k], Aw);
              }
            }
            A *= 1.0001f;  // covers the FP32 rounding of the bounds (|fl32(c)| <= |c| (1 + 2^-24))
            Um *= 1.0001f;
            if (CUTS) {
              // z = fddot T^3/6 and w = fdot are linear in c: z = sum_k c_k E_k, w = sum_k c_k G_k.
              // |fp32 z - oracle z| <= 2^-24 (K+2) sum|c_k| max|E_k| (c, E and the K FMAs rounded)
              // + (4K+40) 2^-53 Um T/6 (the oracle's rounded frequencies, its second difference
              // and the FP64 rounding of E); |fp32 w - oracle w| likewise with G and
              // (2K+12) 2^-53 Um / T_SFT, plus the FP32 rounding of the 1e-13 threshold
              ezt = 1.25f * (5.9604644775390625e-08f * (K + 2.001f) * Az * 1.0001f +
                             (4.f * K + 40.f) * 1.1102230246251565e-16f * Um * (float)(J.T / 6.0)) + 1e-12f;
              ewt = 1.25f * (5.9604644775390625e-08f * (K + 2.001f) * Aw * 1.0001f +
                             (2.f * K + 12.f) * 1.1102230246251565e-16f * Um / (float)J.T) + 1e-20f;
              zbt = Az * 1.0001f + ezt;  // bounds |oracle z| in every segment
            }
            xm = f * J.T;
            // |fp32 y - (x - Bw)| <= err = 2^-24 ((K+1) |y0| + (K+2.001) A) + e64: y0 rounded to
            // FP32, K rounded FMAs on partial sums below |y0| + A, and the FP32 roundings of c and
            // D; e64 = 2^-47 T (|f_ref| + sum_k |c_k| max|U_k|) bounds every FP64 rounding (x_mid,
            // the deltas D, and the oracle's own evaluation).  With g = 1.25 (err + e64) + 4e-9,
            // pairs closer than g to a half-integer are resolved in FP64; outside that band the
            // exact, the oracle's and this bin coincide and none of them is a 1e-9 tie.
            const float e64 = 7.105427357601002e-15f * (float)J.T * Um;
            eb = 1.25f * (5.9604644775390625e-08f * ((K + 2.001f) * A) + 2.f * e64) + 4e-9f;
            exact = !(fabs(xm) < 1073741824.0) || !(A < 1048576.0f);
          }
          if (r == 0) {
            // the warp's base bin: from the first lane whose first track is usable
            const unsigned ok = __ballot_sync(0xffffffffu, active && !exact);
            const int src = ok ? __ffs(ok) - 1 : 0;
            Bw = __shfl_sync(0xffffffffu, (active && !exact) ? (int)rint(xm) : 0, src);
          }
          if (!active) {
            // inactive slot: c = 0 and y far from the table (|y| < 2^22), never pending
            put(y02[r / 2], r & 1, Bw >= 0 ? 4194303.0f : -4194303.0f);
            continue;
          }
          if (!exact) {
            const double yd = xm - (double)Bw;
            const float yf = (float)yd;
            const float g = eb + 1.25f * 5.9604644775390625e-08f * (float)(K + 1) * fabsf(yf) * 1.0001f;
            exact = !(fabs(yd) < 2097152.0) || !(g < 0.25f);
            if (!exact) {
              put(y02[r / 2], r & 1, yf);
              wlim = fminf(wlim, __fsub_rd(0.5f, g));
              if (CUTS) {
                mz = fmaxf(mz, ezt);
                mw = fmaxf(mw, ewt);
                zt = zt || !(zbt < 1.f);
              }
              const int Bd = (int)rint(xm);
              bmin = min(bmin, Bd);
              bmax = max(bmax, Bd);
              inbox |= 1u << r;
            }
          }
          if (exact) {
            // every pair of this track takes the FP64 path: y = 1/2 exactly is never decided
            put(y02[r / 2], r & 1, 0.5f);
#pragma unroll
            for (int k = 0; k < KP; ++k) put(c2[r / 2][k], r & 1, 0.f);
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wlim = fminf(wlim, __shfl_xor_sync(0xffffffffu, wlim, o));
        if (CUTS) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            mz = fmaxf(mz, __shfl_xor_sync(0xffffffffu, mz, o));
            mw = fmaxf(mw, __shfl_xor_sync(0xffffffffu, mw, o));
          }
          const double ylo64 = kFLowHz * J.T - (double)Bw;
          ylo = (float)ylo64;
          // 1/2 - wlim bounds |y - (f T_SFT - Bw)| for every decided track of the warp; add the
          // roundings of ylo (FP32, and FP64 below 1e-6 for |10^-3.5 T_SFT| < 2^29)
          mf = (0.5f - wlim) + fabsf(ylo) * 2.4e-7f + 1e-6f;
          cutm = inbox;
          zt = __any_sync(0xffffffffu, zt);
          zin = __fsub_rd(1.f, mz);
          zex = __fadd_ru(1.f, mz);
          win = __fadd_ru(1e-13f, mw);
          wex = __fsub_rd(1e-13f, mw);
          fin = __fadd_ru(ylo, mf);
          fex = __fsub_rd(ylo, mf);
        }
        // the warp's coefficient box, one coefficient at a time (few live registers)
        float* rb = red + (ltile & 1) * kConsWarps * RW + cwarp * RW;
#pragma unroll
        for (int k = 0; k < KP; ++k) {
          float lo = __int_as_float(0x7f800000), hi = -__int_as_float(0x7f800000);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            if ((inbox >> r) & 1u) {
              lo = fminf(lo, get(c2[r / 2][k], r & 1));
              hi = fmaxf(hi, get(c2[r / 2][k], r & 1));
            }
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
          }
          if (lane == 0) {
            rb[k] = lo;
            rb[KP + k] = hi;
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          bmin = min(bmin, __shfl_xor_sync(0xffffffffu, bmin, o));
          bmax = max(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
        }
        if (lane == 0) {
          reinterpret_cast<int*>(rb)[2 * KP] = bmin;
          reinterpret_cast<int*>(rb)[2 * KP + 1] = bmax;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&tile_ready[ltile & 1]);
      }
      const f32x2 kC2 = f2pack(12582912.0f, 12582912.0f);  // 1.5 * 2^23 in both lanes
      // -------------------------------------------------------------- segments
      const unsigned nin = (unsigned)(J.n_bin + 2 * m);
      for (int sg = s0; sg < s1; ++sg) {
        const int qs = (int)(q_seq % kNQ);
        ++q_seq;
        if (!live || !warp_wait(&full_q[qs], ((q_seq - 1u) / kNQ) & 1u, flags)) continue;
        if (nq > kQT - R) {
          // not enough queue room for this segment: resolve the queue now, in (segment) order
          for (int i = 0; i < nq; ++i) {
            const uint32_t e = queue[i * kCons + ctid];
            const int r2 = (int)(e & 31u), s2 = (int)(e >> 5);
            corr[r2 * kCons + ctid] += exact_pair<DT, BINS, CUTS>(a, J, tile0 + ctid + r2 * kCons, s2);
          }
          nq = 0;
        }
        const QHdr h = qhdr[qs];
        const float* q = qslots + (size_t)qs * a.qcap + h.ws_lo;
        float d[KP];
        {
          const float4* dp = reinterpret_cast<const float4*>(qdseg + (size_t)qs * a.nsp);
#pragma unroll
          for (int k4 = 0; k4 < (KP + 3) / 4; ++k4) {
            const float4 v = dp[k4];
            if (4 * k4 + 0 < KP) d[4 * k4 + 0] = v.x;
            if (4 * k4 + 1 < KP) d[4 * k4 + 1] = v.y;
            if (4 * k4 + 2 < KP) d[4 * k4 + 2] = v.z;
            if (4 * k4 + 3 < KP) d[4 * k4 + 3] = v.w;
          }
        }
        // one straight-line pass over the R tracks: slot offset, FP32 decision, masked gather.
        // off = b - qbase = Bw + (bits(tt) - bits(1.5 * 2^23)) - qbase; the window of b overlaps
        // the table iff 0 <= b + m < n_bin + 2m, i.e. (unsigned)(off + qbase + m) < n_bin + 2m.
        // A pair is pending (queued for the FP64 path) when FP32 cannot decide its bin, or when
        // its window overlaps the table but its centre lies outside the staged band.
        // (unsigned arithmetic: the offsets wrap modulo 2^32 and only b - qbase matters)
        const unsigned koff = (unsigned)Bw - 0x4B400000u - (unsigned)h.qbase;
        const unsigned kin = (unsigned)(h.qbase + m);
        const unsigned qn = (unsigned)h.qn;
        f32x2 d2[KP];
#pragma unroll
        for (int k = 0; k < KP; ++k) d2[k] = f2pack(d[k], d[k]);
        // segment-cut forms, each stored twice (E, E, G, G per coefficient): G held in registers
        // for up to 8 coefficients; E (used only when a track of the warp may reach the
        // second-order cut), and G above 8 coefficients, re-read from shared memory per pair
        const uint32_t egs = smem_u32(qdseg + (size_t)qs * a.nsp + cut_col(KP));
        f32x2 g2[kCutRegs ? KP : 1];
        if (kCutRegs) {
#pragma unroll
          for (int k = 0; k < KP; ++k) g2[k] = lds_pair_v(egs + 16u * k + 8u);
        }
        unsigned pend = 0u;
        // one straight-line pass over the track pairs.  COMPLETE: the band holds every reachable
        // centre (a centre outside Q reads the 0 at q[qn]; only FP32-undecided pairs are
        // pending); otherwise pairs whose window overlaps the table but whose centre lies outside
        // Q are pending too.  ZT: evaluate the second-order cut (off when no track of the warp
        // can reach it).
        auto pairs = [&](auto complete_c, auto zt_c) {
          constexpr bool COMPLETE = decltype(complete_c)::value;
          constexpr bool ZT = CUTS && decltype(zt_c)::value;
          // y of every pair, coefficient by coefficient (R2 independent FMA chains in flight)
          f32x2 yv[R2];
#pragma unroll
          for (int p = 0; p < R2; ++p) yv[p] = y02[p];
#pragma unroll
          for (int k = 0; k < KP; ++k)
#pragma unroll
            for (int p = 0; p < R2; ++p) yv[p] = f2fma(c2[p][k], d2[k], yv[p]);
          if constexpr (COMPLETE && !CUTS && !BINS) {
            // the hot path in three passes: every slot offset and decision, every gather, every sum
            // the decisions are first OR-ed into one flag; only when a pair of the thread is
            // undecided (a few in 10^4 pairs) are they taken one by one, y recomputed as above
            unsigned offs[2 * R2];
            bool und = false;
#pragma unroll
            for (int p = 0; p < R2; ++p) {
              const f32x2 tt2 = f2add(yv[p], kC2);
              const f32x2 dd2 = f2sub(yv[p], f2sub(tt2, kC2));
              float tts[2], dds[2];
              f2split(tt2, tts[0], tts[1]);
              f2split(dd2, dds[0], dds[1]);
#pragma unroll
              for (int hh = 0; hh < 2; ++hh) {
                offs[2 * p + hh] = min((unsigned)__float_as_int(tts[hh]) + koff, qn);
                und |= !(fabsf(dds[hh]) < wlim);
              }
            }
            float vals[2 * R2];
#pragma unroll
            for (int r = 0; r < R; ++r) vals[r] = q[offs[r]];
            if (!und) {
#pragma unroll
              for (int r = 0; r < R; ++r) acc[r] += vals[r];
              return;
            }
            unsigned undm = 0u;
#pragma unroll
            for (int p = 0; p < R2; ++p) {
              f32x2 y2 = y02[p];
#pragma unroll
              for (int k = 0; k < KP; ++k) y2 = f2fma(c2[p][k], d2[k], y2);
              const f32x2 tt2 = f2add(y2, kC2);
              const f32x2 dd2 = f2sub(y2, f2sub(tt2, kC2));
              float dds[2];
              f2split(dd2, dds[0], dds[1]);
#pragma unroll
              for (int hh = 0; hh < 2; ++hh) undm |= (unsigned)!(fabsf(dds[hh]) < wlim) << (2 * p + hh);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] += ((undm >> r) & 1u) ? 0.f : vals[r];
            pend |= undm & ((R >= 32) ? 0xffffffffu : ((1u << R) - 1u));
            return;
          }
#pragma unroll
          for (int p = 0; p < R2; ++p) {
            // tt = y + 1.5 * 2^23 rounds y to an integer (|y| < 2^22); dd = y - rint(y), exact
            const f32x2 y2 = yv[p];
            const f32x2 tt2 = f2add(y2, kC2);
            const f32x2 dd2 = f2sub(y2, f2sub(tt2, kC2));
            float tts[2], dds[2], ys[2], zs[2], ws[2];
            f2split(tt2, tts[0], tts[1]);
            f2split(dd2, dds[0], dds[1]);
            if (CUTS) {
              f32x2 z2 = f2pack(0.f, 0.f), w2 = f2pack(0.f, 0.f);
#pragma unroll
              for (int k = 0; k < KP; ++k) {
                f32x2 ek, gk;
                if (kCutRegs) {
                  gk = g2[k];
                  if (ZT) ek = lds_pair_v(egs + 16u * k);
                } else if (ZT) {
                  lds_pair2_v(egs + 16u * k, ek, gk);
                } else {
                  gk = lds_pair_v(egs + 16u * k + 8u);
                }
                if (ZT) z2 = f2fma(c2[p][k], ek, z2);
                w2 = f2fma(c2[p][k], gk, w2);
              }
              f2split(y2, ys[0], ys[1]);
              f2split(z2, zs[0], zs[1]);
              f2split(w2, ws[0], ws[1]);
            }
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
              const int r = 2 * p + hh;
              if (r >= R) continue;
              const unsigned off = (unsigned)__float_as_int(tts[hh]) + koff;
              bool und = !(fabsf(dds[hh]) < wlim);
              bool excl = false;
              if (CUTS) {
                // included when every test clears its margin, excluded when one fails by more
                // than its margin; anything between is a close call for the FP64 path
                const bool inc = (!ZT || zs[hh] < zin) && ws[hh] > win && ys[hh] > fin;
                excl = (ZT && zs[hh] > zex) || ws[hh] < wex || ys[hh] < fex;
                und = und || (((cutm >> r) & 1u) && !inc && !excl);
              }
              if (COMPLETE) {
                const float v = q[min(off, qn)];
                acc[r] += (und || excl) ? 0.f : v;
                pend |= (unsigned)und << r;
                if (BINS) {
                  const int b = (int)off + h.qbase;
                  const long long t = tile0 + ctid + r * kCons;
                  if (t < tend && !und)
                    J.bins_out[t * n_seg + sg] =
                        (b + m < 0) ? (int)0x80000000 : (b - m >= J.n_bin ? 0x7fffffff : b);
                }
              } else {
                const bool inq = off < qn;
                const bool outside = !inq && off + kin < nin && !excl;
                pend |= (unsigned)(und || outside) << r;
                const bool use = inq && !und && !excl;
                const float v = q[use ? off : 0u];  // the address is always valid
                acc[r] += use ? v : 0.f;
                if (BINS) {
                  const int b = (int)off + h.qbase;
                  const long long t = tile0 + ctid + r * kCons;
                  if (t < tend && !(und || outside))
                    J.bins_out[t * n_seg + sg] =
                        (b + m < 0) ? (int)0x80000000 : (b - m >= J.n_bin ? 0x7fffffff : b);
                }
              }
            }
          }
        };
        using kT = std::true_type;
        using kF = std::false_type;
        if (h.complete) {
          if (!CUTS || zt) pairs(kT{}, kT{});
          else pairs(kT{}, kF{});
        } else {
          if (!CUTS || zt) pairs(kF{}, kT{});
          else pairs(kF{}, kF{});
        }
        // (rare) queue the pending pairs
        if (pend) {
          for (unsigned mk = pend; mk; mk &= mk - 1u) {
            const int r = __ffs(mk) - 1;
            queue[nq * kCons + ctid] = ((uint32_t)sg << 5) | (uint32_t)r;
            ++nq;
          }
        }
        if ((sg % kSegTile) == kSegTile - 1) {
#pragma unroll
          for (int r = 0; r < R; ++r) {
            tot[r * kCons + ctid] += acc[r];
            acc[r] = 0.f;
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty_q[qs]);
      }
      // -------------------------------------------------------------- tile epilogue
      if (live && !__any_sync(0xffffffffu, flags[0] != 0)) {
        for (int i = 0; i < nq; ++i) {
          const uint32_t e = queue[i * kCons + ctid];
          const int r2 = (int)(e & 31u), s2 = (int)(e >> 5);
          corr[r2 * kCons + ctid] += exact_pair<DT, BINS, CUTS>(a, J, tile0 + ctid + r2 * kCons, s2);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const long long t = tile0 + ctid + r * kCons;
          if (t < tend) {
            const float v = (tot[r * kCons + ctid] + acc[r]) + corr[r * kCons + ctid];
            if (J.seg_split > 1) J.part[(size_t)sp * J.N + t] = v;
            else J.stat[t] = v;
          }
        }
      }
    }
  }
  __syncthreads();
  if (flags[0] && tid == 0) {
    // a bounded wait gave up: let every staging copy still in flight land before leaving
    for (int i = 0; i < kNP; ++i) {
      (void)mbar_wait_bounded(&full_p[i], 0u, kWaitLimitNs / 4);
      (void)mbar_wait_bounded(&full_p[i], 1u, kWaitLimitNs / 4);
    }
    atomicExch(a.status, DEV_TIMEOUT);
  }
}

// ---------------------------------------------------------------- host side
template <int DT, int KP, int R, bool BINS, bool CUTS, int MJ>
int launch_one(const EvalArgs<MJ>& a0, int grid, size_t smem, cudaStream_t st) {
  auto kern = eval_stat_kernel<DT, KP, R, BINS, CUTS, MJ>;
  static int configured = -1;
  if (configured < (int)smem) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(eval)");
    configured = (int)smem;
  }
  kern<<<grid, kThreads, smem, st>>>(a0);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "eval_stat_kernel launch");
  return TFS_OK;
}

inline int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// Partial sums of tiles that cover a segment range, added in range order into the statistic.
struct PartJob {
  const float* part;  // [S][N]
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
    float v = 0.f;
    for (int q = 0; q < J.S; ++q) v += J.part[(size_t)q * J.N + t];
    J.stat[t] = v;
  }
}

inline int r_of_kp(int KP) { return KP <= 6 ? 12 : (KP <= 8 ? 9 : (KP <= 16 ? 4 : 2)); }
// with segment cuts each track also carries the two cut forms: fewer tracks per thread
inline int r_of_kp_cuts(int KP) { return KP <= 6 ? 8 : (KP <= 8 ? 6 : 2); }

template <int DT, int MJ>
int launch_eval_jobs(const EvalLaunch& L, const EvalTuning& tune, cudaStream_t st) {
  constexpr int esize = Store<DT>::esize;
  constexpr int EPV = 16 / esize;
  int KP = 0;
  for (int i = 0; i < L.n_jobs; ++i) KP = std::max(KP, L.jobs[i].sp->KP);
  const bool cuts = L.jobs[0].cuts != 0;
  const int R = cuts ? r_of_kp_cuts(KP) : r_of_kp(KP);
  const int nsp = segrow_floats(KP, cuts);

  EvalArgs<MJ> a{};
  a.tie_count = L.tie_count;
  a.tie_track = reinterpret_cast<long long*>(L.tie_track);
  a.tie_seg = L.tie_seg;
  a.tie_cap = L.tie_cap;
  a.status = L.status;
  a.dbg = L.dbg;
  a.nsp = nsp;
  const long long tile = (long long)kCons * R / std::max(1, std::min(tune.tile_div, 8));
  long long nt = 0;
  int row_max = 0, seg_max = 0;
  bool bins = false;
  for (int i = 0; i < L.n_jobs; ++i) {
    const EvalJob& E = L.jobs[i];
    const tfs_table* tb = E.table;
    if (E.sp->KP != KP || E.sp->nsp != nsp) {
      set_error("internal: job %d has %d coefficient slots, launch %d", i, E.sp->KP, KP);
      return TFS_ERR_INVALID_ARG;
    }
    JobDesc& D = a.jobs[i];
    D.table = tb->data;
    D.scales = tb->scales;
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
    D.row_stride = (int)tb->row_stride;
    D.m = E.m;
    D.K = E.basis->K;
    D.alpha_mid = E.sp->alpha_mid;
    D.emax = E.sp->emax;
    D.gmax = E.sp->gmax;
    if ((E.cuts != 0) != cuts || (cuts && !E.sp->cuts)) {
      set_error("internal: jobs with and without segment cuts in one launch");
      return TFS_ERR_INVALID_ARG;
    }
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
    a.tile_start[i] = (int)nt;
    nt += tt > 0 ? (E.N + tt - 1) / tt : 0;
    row_max = std::max(row_max, (int)tb->row_stride);
    seg_max = std::max(seg_max, (int)tb->n_seg);
    bins = bins || E.bins_out != nullptr;
  }
  if (nt == 0) return TFS_OK;
  // Few track tiles (small jobs): split each job's segments over several tiles so that every
  // SM gets work, at least 16 segments per tile; the tiles' partial sums are added in segment
  // order by a second small kernel.
  size_t part_floats = 0;
  const long long sms_all = sm_count();
  if (!bins && nt < sms_all) {
    const int S = (int)std::min<long long>(8, sms_all / nt);
    if (S > 1) {
      nt = 0;
      for (int i = 0; i < L.n_jobs; ++i) {
        JobDesc& D = a.jobs[i];
        const long long ntj = D.N > 0 ? (D.N + D.tile_tracks - 1) / D.tile_tracks : 0;
        const int Sj = std::max(1, std::min(S, D.n_seg / 16));
        D.seg_chunk = (D.n_seg + Sj - 1) / Sj;
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

  // staging slots hold up to pcap band elements; Q slots the window sums of a whole slot
  int pcap = tune.cap > 0 ? tune.cap : 2048;
  pcap = std::max(64, std::min(pcap, row_max));
  pcap = (pcap + 31) / 32 * 32;
  if (pcap > row_max) pcap = row_max;
  a.pcap = pcap;
  a.qcap = kPadL + pcap + 2 * EPV;
  const int RW = 2 * KP + 2;
  const size_t pslot_bytes = (size_t)(kPadL + pcap + EPV) * esize + nsp * 4;
  size_t off = 8 * (2 * kNP + 2 * kNQ + 2);
  off = (off + 15) & ~(size_t)15;
  a.off_qhdr = (int)off;  off += kNQ * sizeof(QHdr) + (size_t)kNQ * nsp * 4;
  off = (off + 15) & ~(size_t)15;
  a.off_red = (int)off;   off += (size_t)2 * kConsWarps * RW * 4;
  off = (off + 15) & ~(size_t)15;
  a.off_flags = (int)off; off += 16 + 2 * kNP * 4 + (size_t)(2 * KP + 2) * 4;
  off = (off + 15) & ~(size_t)15;
  a.off_band = (int)off;  off += (size_t)2 * std::min(seg_max, kBandCap) * 4;
  off = (off + 15) & ~(size_t)15;
  a.off_queue = (int)off; off += (size_t)kQT * kCons * 4;
  a.off_acc = (int)off;   off += (size_t)2 * R * kCons * 4;
  off = (off + 127) & ~(size_t)127;
  a.off_q = (int)off;     off += (size_t)kNQ * a.qcap * 4;
  off = (off + 127) & ~(size_t)127;
  a.off_p = (int)off;     off += (size_t)kNP * pslot_bytes;
  off = (off + 15) & ~(size_t)15;
  a.off_seg = (int)off;
  size_t seg_bytes = (size_t)seg_max * (nsp + 1) * 4;
  const bool resident = off + seg_bytes <= 200 * 1024;  // resident per-segment data when it fits
  if (!resident) seg_bytes = 0;
  for (int i = 0; i < L.n_jobs; ++i) a.jobs[i].seg_resident = resident ? 1 : 0;
  off += seg_bytes;
  const size_t smem = off;
  a.smem_bytes = (int)smem;
  if (smem > 227 * 1024) {
    set_error("statistic kernel needs %zu bytes of shared memory", smem);
    return TFS_ERR_INVALID_ARG;
  }
  const int grid = (int)std::min<long long>(nt, (long long)sm_count());
  float* parts = nullptr;
  if (part_floats) {
    TFS_CUDA(cudaMallocAsync((void**)&parts, part_floats * sizeof(float), st));
    size_t o = 0;
    for (int i = 0; i < L.n_jobs; ++i) {
      JobDesc& D = a.jobs[i];
      if (D.seg_split > 1) {
        D.part = parts + o;
        o += (size_t)D.seg_split * D.N;
      }
    }
  }
  auto dispatch = [&]() -> int {
#define TFS_LAUNCH_KP(KPV, RV, RCV)                                                     \
  if (KP == KPV) {                                                                      \
    if (cuts) return launch_one<DT, KPV, RCV, false, true, MJ>(a, grid, smem, st);       \
    if constexpr (MJ == 1) {                                                            \
      if (bins) return launch_one<DT, KPV, RV, true, false, MJ>(a, grid, smem, st);     \
    }                                                                                   \
    return launch_one<DT, KPV, RV, false, false, MJ>(a, grid, smem, st);                 \
  }
    TFS_LAUNCH_KP(2, 12, 8)
    TFS_LAUNCH_KP(4, 12, 8)
    TFS_LAUNCH_KP(6, 12, 8)
    TFS_LAUNCH_KP(8, 9, 6)
    TFS_LAUNCH_KP(16, 4, 2)
    TFS_LAUNCH_KP(32, 2, 2)
#undef TFS_LAUNCH_KP
    set_error("unsupported coefficient slot count %d", KP);
    return TFS_ERR_INVALID_ARG;
  };
  (void)R;
  int rc = dispatch();
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
  return rc;
}

template <int DT>
int launch_eval_dt(const EvalLaunch& L, const EvalTuning& tune, cudaStream_t st) {
  if (L.n_jobs <= 0) return TFS_OK;
  if (L.n_jobs == 1) return launch_eval_jobs<DT, 1>(L, tune, st);
  if (L.n_jobs > kMaxJobs) {
    set_error("at most %d jobs per launch", kMaxJobs);
    return TFS_ERR_INVALID_ARG;
  }
  return launch_eval_jobs<DT, kMaxJobs>(L, tune, st);
}

}  // namespace tfs
