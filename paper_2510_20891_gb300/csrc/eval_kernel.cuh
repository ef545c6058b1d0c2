// Fused track evaluation + gather + reduction for the semi-coherent statistic
// (paper Sec. II.B Eq. det_stat, nearest-bin reading with +-m neighbours;
// tracks from the SVD basis of Sec. II.C).
//
// The table is read through its window sums W[alpha][c] = sum_{|j|<=m} P[alpha][c+j] (wsum.cu),
// so a (track, segment) pair gathers one FP32 value.  Persistent, warp-specialised kernel: one
// CTA per SM walks a list of tiles (static round-robin); a tile is up to 384 R tracks of one
// job, a job is one dataset (window sums, basis, batch of tracks), so datasets of different
// shapes run in one launch.  Two roles:
//
//   producer warpgroup (128 threads, registers lowered with setmaxnreg)
//     * at a tile start, all 128 threads compute, from the tile's coefficient box, a rigorous
//       interval of the window centres the tile can reach in every segment (the "band");
//     * warp 0 (the stager) fills staging slots: each slot carries the bands of as many
//       consecutive segments as fit (at most `group`), each followed by 4 zero floats and the
//       segment's FP32 basis deltas, all moved by 1-D bulk copies (cp.async.bulk) completing
//       on the slot's mbarrier; the slot's header (segments, offsets, band bases) is written
//       before the arrival that arms the barrier;
//   three consumer warpgroups (384 threads, registers raised with setmaxnreg)
//     wait once per slot; per segment each thread evaluates x = f T_SFT for its R tracks in FP32,
//           y = (x_mid - Bw) + sum_k c_k D_k,alpha,    b = Bw + rint(y),
//     (Bw a warp base bin, x_mid an FP64 per-track constant) and adds W[b] with one shared
//     load.  Pairs within a warp-uniform error bound g of a half-integer, and pairs whose
//     centre falls outside a staged band that had to be cut, go to the thread's own queue and
//     are recomputed at the end of the tile in the FP64 operation order of the oracle
//     (separately rounded products and sums): every bin equals the FP64 bin exactly, ties
//     included.
//
// The roles meet only on mbarriers (slot full/empty, per-tile box hand-off).  FP32 sums of 32
// segments (blocks aligned to the segment index) are added with a compensated (two-sum) FP32
// accumulator, and fix-up contributions likewise in segment order: how a job's segments and
// tracks are grouped barely changes its last bits.  The consumers use no FP64 arithmetic on any
// per-track path (GB300's FP64 rate is 1/64 of FP32): only the fix-ups and split jobs' partials.  The result is deterministic for a given launch; which pairs
// take the fix-up path depends on the warp's base bin and decision limit and on the tile's
// band, so a track's FP32 rounding (never its bins) can change with its tile neighbours.
// Every wait is bounded (a launch argument, 2 s by default) and warp-uniform; after a timeout
// every role leaves its loops, thread 0 lets the copies still in flight land, and the call
// returns TFS_ERR_TIMEOUT.
#pragma once

#include "tfs_internal.cuh"

namespace tfs {

constexpr int kProd = 128;            // producer warpgroup: stager warp + 3 band helpers
constexpr int kCons = 384;            // three consumer warpgroups
constexpr int kThreads = kProd + kCons;
constexpr int kConsWarps = kCons / 32;
constexpr int kLaunchRegs = (65536 / kThreads) & ~7;  // 128 registers per thread at launch
constexpr int kProdRegs = 72;         // setmaxnreg targets: 128*72 + 384*144 <= 512*128
constexpr int kConsRegs = 144;
static_assert(kProd * kProdRegs + kCons * kConsRegs <= kThreads * kLaunchRegs, "register split exceeds the launch");
constexpr int kMaxSlots = 8;          // staging slots at most
constexpr int kMaxGroup = 32;         // segments per staging slot at most (one per lane of the stager)
constexpr int kSent = 4;              // zero floats staged after each band (the sum of centres outside it)
constexpr int kQT = 24;               // fix-up queue entries per consumer thread (a queue that fills
                                      // mid-tile stalls its warp on FP64 work: keep it rare)
constexpr int kSegTile = 32;          // FP32 partial sums are flushed every kSegTile segments
constexpr int kBandCap = 1024;        // segments whose bands are precomputed per tile (two buffers)
constexpr int kTrunc = 1 << 30;       // flag in a band length: the band was cut to the capacity
constexpr uint64_t kDrainNs = 1000000000ull;  // wait for in-flight copies after a timeout (1 s)

struct JobDesc {
  const float* q;       // window sums [n_seg][qpitch]; centre c at index c + m
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
  int n_seg, n_bin, qpitch, m, K, alpha_mid;
  int tile_tracks;      // tracks per tile (<= consumer threads * R); the last tile may hold fewer
  const float* emax;    // [KP] segment-cut launches: max |E_k|, max |G_k| (see SegParams)
  const float* gmax;
  int seg_split;        // tiles per track range, each over seg_chunk consecutive segments
  int seg_chunk;
  double* part;         // [seg_split][N] partial sums when seg_split > 1 (summed in order afterwards)
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
  unsigned long long wait_ns;  // limit of every wait
  int hold;      // the stager first waits for an arrival that never comes (timeout tests)
  int smem_bytes;
  int nsp;       // floats per segment row of segp (launch-wide)
  int pcap;      // window sums staged per segment at most (multiple of 4)
  int scap;      // floats per staging slot (>= pcap + kSent + nsp)
  int nslots;    // staging slots (<= kMaxSlots)
  int group;     // segments per slot at most (<= kMaxGroup)
  int bcap;      // segments whose bands are precomputed per tile (<= kBandCap); longer tiles compute them as they stage
  float* cbuf;   // [grid][KP + 1][consumer threads * R] prologue columns (FP32 coefficients, then y0)
  int* tile_ctr; // tiles claimed beyond each CTA's first (zero at launch)
  int n_tiles;
  int n_jobs;
  // shared-memory carve-up (byte offsets)
  int off_hdr, off_info, off_flags, off_band, off_queue, off_acc, off_slots;
  int tile_start[MJ + 1];  // first tile of each job (prefix sums), tile_start[n_jobs] = n_tiles
  JobDesc jobs[MJ];
};

// Header of a staging slot: its segments in order, each {float offset of its window sums from
// the first slot, centre of the first sum, number of sums, complete (every reachable centre whose window
// overlaps the table has its sum staged)}; the deltas follow the sums after kSent zeros.
struct SlotHdr {
  int nseg, pad0, pad1, pad2;
  int4 seg[kMaxGroup];
};

// 16 zero bytes: the source of the zeros staged after each band.
static __device__ __align__(16) float g_zero4[4];

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

template <int MJ>
__device__ __forceinline__ void report_tie(const EvalArgs<MJ>& a, long long t, int seg) {
  const unsigned long long i = atomicAdd(a.tie_count, 1ull);
  if (i < (unsigned long long)a.tie_cap) {
    a.tie_track[i] = t;
    a.tie_seg[i] = seg;
  }
}

// FP64 bin of (track t, segment seg) of job J in the oracle's operation order, and its window
// sum from the window-sum array in global memory.  With CUTS the segment exclusions are decided
// first, in FP64 in the oracle's operation order, from the track's frequencies at the segments its
// finite differences use (0 for an excluded segment).  (Loading every operand up front and keeping
// the function out of line made the pair loop spill: 2.84 -> 5.4 ms on the one-year launch.)
template <int KP, bool BINS, bool CUTS, int MJ>
__device__ float exact_pair(const EvalArgs<MJ>& a, const JobDesc& J, long long t, int seg) {
  if (!dbg_ok(a.dbg, t >= 0 && t < J.N && seg >= 0 && seg < J.n_seg, 1, t, seg)) return 0.f;
  double f;
  if (!CUTS) {
    f = J.f_ref ? J.f_ref[t] : 0.0;
    const double* c = J.coeffs + t * (long long)J.K;
    for (int k = 0; k < J.K; ++k) f = __dadd_rn(f, __dmul_rn(c[k], J.U[(size_t)k * J.n_seg + seg]));
  } else {
    // the frequencies at the (at most three) segments s0 .. s0 + 2 that the finite differences
    // use, in one pass over the coefficients (each sum in the oracle's order: f_ref, then the K
    // products left to right): one memory wait per coefficient rather than per segment
    const int n = J.n_seg;
    const double T = J.T;
    const int s0 = n >= 3 ? min(max(seg - 1, 0), n - 3) : 0;
    const int n3 = min(n, 3);
    const double fr = J.f_ref ? J.f_ref[t] : 0.0;
    double fs[3] = {fr, fr, fr};
    const double* c = J.coeffs + t * (long long)J.K;
    for (int k = 0; k < J.K; ++k) {
      const double ck = c[k];
      const double* u = J.U + (size_t)k * n + s0;
#pragma unroll
      for (int i = 0; i < 3; ++i)
        if (i < n3) fs[i] = __dadd_rn(fs[i], __dmul_rn(ck, u[i]));
    }
    auto F = [&](int s) { return fs[s - s0]; };
    f = F(seg);
    double fd = 0.0, z = 0.0;
    if (n >= 2) {
      if (seg == 0) fd = __ddiv_rn(__dsub_rn(F(1), f), T);
      else if (seg == n - 1) fd = __ddiv_rn(__dsub_rn(f, F(n - 2)), T);
      else fd = __ddiv_rn(__dsub_rn(F(seg + 1), F(seg - 1)), __dmul_rn(2.0, T));
    }
    if (n >= 3) {
      const int cc = seg == 0 ? 1 : (seg == n - 1 ? n - 2 : seg);
      const double dd = __dadd_rn(__dsub_rn(F(cc + 1), __dmul_rn(2.0, F(cc))), F(cc - 1));
      z = __dmul_rn(dd, __ddiv_rn(T, 6.0));
    }
    if (z > 1.0 || f < kFLowHz || fd < kFdotLow) return 0.f;
  }
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
  return J.q[(size_t)seg * J.qpitch + (b + m)];
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
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* flags, uint64_t limit) {
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
        stop = flags[0] != 0 || (it != 0 && now - t0 > limit);
      }
      if (__shfl_sync(0xffffffffu, stop, 0)) {
        flags[0] = 1;
        return false;
      }
    }
  }
}
// Single-thread bounded wait.
__device__ __forceinline__ bool thread_wait(uint64_t* bar, uint32_t parity, volatile int* flags, uint64_t limit) {
  if (flags[0]) return false;
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 31) == 0) {
      const uint64_t now = global_ns();
      if (it == 0) t0 = now;
      else if (flags[0] != 0 || now - t0 > limit) {
        flags[0] = 1;
        return false;
      }
    }
  }
}
// Named barrier 1 among the three helper warps that also ORs a predicate over their threads:
// every helper gets the same answer, so all of them leave their loop at the same barrier.
__device__ __forceinline__ bool help_bar_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n barrier.cta.red.or.pred q, 1, 96, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}
template <int N>
__device__ __forceinline__ void setmaxnreg_inc() {
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(N));
}
template <int N>
__device__ __forceinline__ void setmaxnreg_dec() {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(N));
}

template <int MJ>
__device__ __forceinline__ int job_of(const EvalArgs<MJ>& a, int tile) {
  int j = 0;
  while (j + 1 < a.n_jobs && tile >= a.tile_start[j + 1]) ++j;
  return j;
}

// Staged window sums [ilo, ilo + len) (indices c + m, ilo and len multiples of 4) for segment
// row d of a tile whose coefficient box is [lo_k, hi_k] and base bins [bm, bx]: every centre
// that a track of the box can reach and whose window overlaps the table, computed in FP32 with a
// margin covering its rounding (the band only steers staging; a pair outside a cut band takes
// the exact path).  len carries kTrunc when the band had to be cut to pcap sums.
template <int KP>
__device__ __forceinline__ void band_of(const float* d, const float* blo_k, const float* bhi_k, int bm, int bx,
                                        int m, int n_bin, int pcap, int* out_lo, int* out_len) {
  int ilo = 0, len = 0;
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
    const float cl = fmaxf(floorf((float)bm + lo - fm), (float)(-m));
    const float ch = fminf(floorf((float)bx + 1.f + hi + fm), (float)(n_bin - 1 + m));
    if (cl <= ch) {
      ilo = ((int)cl + m) & ~3;
      const int ihi = ((int)ch + m + 4) & ~3;  // exclusive, <= the row pitch (a multiple of 32)
      len = ihi - ilo > pcap ? (pcap | kTrunc) : ihi - ilo;
    }
  }
  *out_lo = ilo;
  *out_len = len;
}

// Per consumer warp, the values its tile prologue needs (prepared by the helper warps).
struct WarpInfo {
  int Bw;       // base bin: the FP64 mid-segment bin of the warp's first usable track
  float wlim;   // decision limit: min over the warp's tracks decided in FP32 of 1/2 - g (1/2 if none)
  float mz;     // segment cuts: margin of the second-order test
  float mw;     // segment cuts: margin of the fdot test
  float ylo;    // segment cuts: 10^-3.5 T_SFT - Bw (bin units, FP32)
  int zt;       // segment cuts: some track of the warp may reach the second-order cut
  int pad0, pad1;
};

// ---------------------------------------------------------------- tile prologue (FP64 where the
// bin decision needs it).  Run by the helper warps one tile ahead of the consumers, and by the
// consumers themselves for a CTA's first tile, which no earlier tile hides.

// The base bin of consumer warp w of a tile: the FP64 mid-segment bin of its first lane whose first
// track is usable (one warp).
template <int KP, bool CUTS>
__device__ __forceinline__ void prologue_base(const JobDesc& J, long long tile0, long long tend, int w, int lane,
                                              WarpInfo* winfo) {
  const int n_seg = J.n_seg, K = J.K;
  const long long t = tile0 + w * 32 + lane;
  const bool active = t < tend;
  double xm = 0.0;
  bool ex = false;
  if (active) {
    double f = J.f_ref ? J.f_ref[t] : 0.0;
    float A = 0.f;
    const double* cp = J.coeffs + t * (long long)K;
    for (int k = 0; k < K; ++k) {
      const double cd = cp[k];
      f = fma(cd, J.U[(size_t)k * n_seg + J.alpha_mid], f);
      A = fmaf(fabsf((float)cd), J.dmax[k], A);
    }
    A *= 1.0001f;
    xm = f * J.T;
    ex = !(fabs(xm) < 1073741824.0) || !(A < 1048576.0f);
  }
  const unsigned ok = __ballot_sync(0xffffffffu, active && !ex);
  const int src = ok ? __ffs(ok) - 1 : 0;
  const int Bw = __shfl_sync(0xffffffffu, (active && !ex) ? (int)rint(xm) : 0, src);
  if (lane == 0) {
    winfo[w].Bw = Bw;
    winfo[w].ylo = CUTS ? (float)(kFLowHz * J.T - (double)Bw) : 0.f;
  }
}

// The R tracks of consumer thread ctid (one warp: the 32 lanes of one consumer warp, whose base bin
// is set): their FP32 coefficients and offsets y0 in the prologue columns, which of them FP32
// decides, the warp's decision limits, and the range of their FP64 mid bins (bmin, bmax).
template <int KP, int R, bool CUTS>
__device__ __forceinline__ void prologue_tracks(const JobDesc& J, long long tile0, long long tend, int ctid, int lane,
                                                float* cbuf, WarpInfo* winfo, uint32_t* inboxm, int& bmin, int& bmax) {
  constexpr int kCR = kCons * R;
  const int n_seg = J.n_seg, K = J.K;
  const int w = ctid >> 5;
  const int Bw = winfo[w].Bw;
  float wl = 0.5f, mzl = 0.f, mwl = 0.f;
  bool ztl = false;
  uint32_t ib = 0u;
  for (int r = 0; r < R; ++r) {
    const long long t = tile0 + ctid + r * kCons;
    float* col = cbuf + r * kCons + ctid;  // coefficient k at col[k * kCR], y0 at col[KP * kCR]
    if (!(t < tend)) {
      // inactive slot: c = 0 and y far from the table (|y| < 2^22), never pending
      for (int k = 0; k < KP; ++k) col[k * kCR] = 0.f;
      col[KP * kCR] = Bw >= 0 ? 4194303.0f : -4194303.0f;
      continue;
    }
    const double fr = J.f_ref ? J.f_ref[t] : 0.0;
    double f = fr;
    float A = 0.f, Um = fabsf((float)fr), Az = 0.f, Aw = 0.f;
    const double* cp = J.coeffs + t * (long long)K;
    for (int k = 0; k < KP; ++k) {
      const double cd = (k < K) ? cp[k] : 0.0;
      if (k < K) f = fma(cd, J.U[(size_t)k * n_seg + J.alpha_mid], f);
      const float cf = (float)cd;
      col[k * kCR] = cf;
      A = fmaf(fabsf(cf), J.dmax[k], A);
      Um = fmaf(fabsf(cf), J.umax[k], Um);
      if (CUTS) {
        Az = fmaf(fabsf(cf), J.emax[k], Az);
        Aw = fmaf(fabsf(cf), J.gmax[k], Aw);
      }
    }
    A *= 1.0001f;  // covers the FP32 rounding of the bounds (|fl32(c)| <= |c| (1 + 2^-24))
    Um *= 1.0001f;
    float ezt = 0.f, ewt = 0.f, zbt = 0.f;
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
    const double xm = f * J.T;
    // |fp32 y - (x - Bw)| <= err = 2^-24 ((K+1) |y0| + (K+2.001) A) + e64: y0 rounded to
    // FP32, K rounded FMAs on partial sums below |y0| + A, and the FP32 roundings of c and
    // D; e64 = 2^-47 T (|f_ref| + sum_k |c_k| max|U_k|) bounds every FP64 rounding (x_mid,
    // the deltas D, and the oracle's own evaluation).  With g = 1.25 (err + e64) + 4e-9,
    // pairs closer than g to a half-integer are resolved in FP64; outside that band the
    // exact, the oracle's and this bin coincide and none of them is a 1e-9 tie.
    const float e64 = 7.105427357601002e-15f * (float)J.T * Um;
    const float eb = 1.25f * (5.9604644775390625e-08f * ((K + 2.001f) * A) + 2.f * e64) + 4e-9f;
    bool exact = !(fabs(xm) < 1073741824.0) || !(A < 1048576.0f);
    float y0 = 0.5f;
    if (!exact) {
      const double yd = xm - (double)Bw;
      const float yf = (float)yd;
      const float g = eb + 1.25f * 5.9604644775390625e-08f * (float)(K + 1) * fabsf(yf) * 1.0001f;
      exact = !(fabs(yd) < 2097152.0) || !(g < 0.25f);
      if (!exact) {
        y0 = yf;
        wl = fminf(wl, __fsub_rd(0.5f, g));
        if (CUTS) {
          mzl = fmaxf(mzl, ezt);
          mwl = fmaxf(mwl, ewt);
          ztl = ztl || !(zbt < 1.f);
        }
        const int Bd = (int)rint(xm);
        bmin = min(bmin, Bd);
        bmax = max(bmax, Bd);
        ib |= 1u << r;
      }
    }
    if (exact) {
      // every pair of this track takes the FP64 path: y = 1/2 exactly is never decided
      for (int k = 0; k < KP; ++k) col[k * kCR] = 0.f;
    }
    col[KP * kCR] = y0;
  }
  inboxm[ctid] = ib;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    wl = fminf(wl, __shfl_xor_sync(0xffffffffu, wl, o));
    if (CUTS) {
      mzl = fmaxf(mzl, __shfl_xor_sync(0xffffffffu, mzl, o));
      mwl = fmaxf(mwl, __shfl_xor_sync(0xffffffffu, mwl, o));
    }
  }
  ztl = __any_sync(0xffffffffu, ztl);
  if (lane == 0) {
    winfo[w].wlim = wl;
    winfo[w].mz = mzl;
    winfo[w].mw = mwl;
    winfo[w].zt = ztl ? 1 : 0;
  }
}

// One warp's partial of the tile's coefficient box over the tracks decided in FP32 among consumer
// threads ctid0 + 96 q, q < nq: per coefficient the lowest and highest FP32 value, then the range
// of the FP64 mid bins, in bp[0..2 KP + 1].
template <int KP, int R>
__device__ __forceinline__ void prologue_box_part(const float* cbuf, const uint32_t* inboxm, int ctid0, int nq,
                                                  int lane, int bmin, int bmax, float* bp) {
  constexpr int kCR = kCons * R;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    bmin = min(bmin, __shfl_xor_sync(0xffffffffu, bmin, o));
    bmax = max(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
  }
  if (lane == 0) {
    reinterpret_cast<int*>(bp)[2 * KP] = bmin;
    reinterpret_cast<int*>(bp)[2 * KP + 1] = bmax;
  }
  for (int k = 0; k < KP; ++k) {
    float lo = __int_as_float(0x7f800000), hi = -__int_as_float(0x7f800000);
    for (int q = 0; q < nq; ++q) {
      const int ctid = ctid0 + 96 * q;
      const uint32_t ib = inboxm[ctid];
      for (int r = 0; r < R; ++r) {
        if ((ib >> r) & 1u) {
          const float v = cbuf[k * kCR + r * kCons + ctid];
          lo = fminf(lo, v);
          hi = fmaxf(hi, v);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
      bp[k] = lo;
      bp[KP + k] = hi;
    }
  }
}

template <int KP, int R, bool BINS, bool CUTS, int MJ>
__global__ void __launch_bounds__(kThreads, 1) eval_stat_kernel(const __grid_constant__ EvalArgs<MJ> a) {
  constexpr bool kCutRegs = CUTS && KP <= 8;  // segment-cut forms held in registers
  constexpr int kCR = kCons * R;              // track slots of a tile (slot r * kCons + ctid)
  constexpr int BW = 2 * KP + 2;              // a box: KP minima, KP maxima, then bm, bx (ints)
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  uint64_t* full = bars;                      // [kMaxSlots] a slot's copies landed (tx)
  uint64_t* empty = bars + kMaxSlots;         // [kMaxSlots] consumers done with the slot (12 warps)
  uint64_t* pro_full = bars + 2 * kMaxSlots;  // the next tile's prologue data is ready (helpers)
  uint64_t* pro_free = pro_full + 1;          // the consumers have read it (12 warps)
  uint64_t* band_ready = pro_full + 2;        // [2] a tile's box and bands are ready (helpers)
  uint64_t* band_free = pro_full + 4;         // [2] the stager is done with them
  uint64_t* hold_bar = pro_full + 6;          // nothing arrives on it (timeout tests)
  uint64_t* parts_ready = pro_full + 7;       // the consumers' box partials of their first tile (12 warps)
  SlotHdr* hdr = reinterpret_cast<SlotHdr*>(smem + a.off_hdr);                // [nslots]
  WarpInfo* winfo = reinterpret_cast<WarpInfo*>(smem + a.off_info);          // [kConsWarps]
  uint32_t* inboxm = reinterpret_cast<uint32_t*>(winfo + kConsWarps);         // [kCons] tracks decided in FP32
  float* bpart = reinterpret_cast<float*>(inboxm + kCons);                    // [12][BW] box partials
  // [0] abort, [1] the tile the helpers claimed, [2 + b] the tile of parity b for the stager and
  // the consumers (n_tiles or more: no more tiles)
  volatile int* flags = reinterpret_cast<volatile int*>(smem + a.off_flags);
  uint32_t* issued = reinterpret_cast<uint32_t*>(smem + a.off_flags) + 4;    // [kMaxSlots] last use + 1
  float* boxes = reinterpret_cast<float*>(issued + kMaxSlots);                // [2][BW]
  int* bands = reinterpret_cast<int*>(smem + a.off_band);                     // [2][bcap][2]
  uint32_t* queue = reinterpret_cast<uint32_t*>(smem + a.off_queue);          // [kQT][kCons]
  float* corr = reinterpret_cast<float*>(smem + a.off_acc);                  // [R][kCons] sum of FP64-path values
  float* corrl = corr + R * kCons;                                            // [R][kCons] its rounding error
  float* tot = corrl + R * kCons;                                             // [R][kCons] sum of 32-segment blocks
  float* comp = tot + R * kCons;                                              // [R][kCons] its rounding error
  float* slots = reinterpret_cast<float*>(smem + a.off_slots);                // [nslots][scap]
  // this CTA's prologue columns in global memory: FP32 coefficients [KP][kCR], then y0 [kCR]
  float* cbuf = a.cbuf + (size_t)blockIdx.x * (KP + 1) * kCR;
  const int NS = a.nslots;

  const int tid = threadIdx.x;
  const int lane = tid & 31;

  if (tid < 4) flags[tid] = 0;
  if (tid < kMaxSlots) issued[tid] = 0u;
  if (tid == 0) {
    for (int i = 0; i < kMaxSlots; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kConsWarps);
    }
    mbar_init(pro_full, 1);
    mbar_init(pro_free, kConsWarps);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&band_ready[i], 1);
      mbar_init(&band_free[i], 1);
    }
    mbar_init(hold_bar, 1);
    mbar_init(parts_ready, kConsWarps);
    fence_mbar_init();
  }
  __syncthreads();

  if (tid < kProd) {
    // ================================================================ producer warpgroup
    setmaxnreg_dec<kProdRegs>();
    if (tid < 32) {
      // ------------------------------------------------------------ stager warp
      // per tile: wait for its bands, then fill slots; lane g stages segment sg + g of a slot,
      // the slot taking the leading segments that fit
      uint32_t seq = 0;  // slots filled so far in this launch
      if (a.hold) (void)warp_wait(hold_bar, 0u, flags, a.wait_ns);
      for (int ltile = 0;; ++ltile) {
        const int b = ltile & 1;
        if (!warp_wait(&band_ready[b], (uint32_t)((ltile >> 1) & 1), flags, a.wait_ns)) break;
        const int tile = reinterpret_cast<const int*>(const_cast<const int*>(flags))[2 + b];
        if (tile >= a.n_tiles) break;
        const int j = job_of(a, tile);
        const JobDesc& J = a.jobs[j];
        const int m = J.m;
        long long tile0_unused;
        int sp_unused, s0, s1;
        tile_range(a, J, tile, j, &tile0_unused, &sp_unused, &s0, &s1);
        const int ns = s1 - s0;
        const float* box = boxes + b * BW;
        const int* band = bands + b * 2 * a.bcap;
        const int bm = reinterpret_cast<const int*>(box)[2 * KP];
        const int bx = reinterpret_cast<const int*>(box)[2 * KP + 1];
        bool go = true;
        for (int sg = s0; sg < s1 && go;) {
          const int s = (int)(seq % (uint32_t)NS);
          if (seq >= (uint32_t)NS) go = warp_wait(&empty[s], ((seq / NS) - 1u) & 1u, flags, a.wait_ns);
          else go = !__any_sync(0xffffffffu, flags[0] != 0);
          if (!go) break;
          // a slot never crosses a 32-segment block boundary, so that the consumers add a finished
          // block's FP32 sums after the slot instead of testing every segment
          const bool has = lane < a.group && sg + lane < s1 && lane < kSegTile - (sg % kSegTile);
          int ilo = 0, len = 0, need = 0;
          if (has) {
            if (ns <= a.bcap) {
              ilo = band[2 * (sg + lane - s0)];
              len = band[2 * (sg + lane - s0) + 1];
            } else {
              band_of<KP>(J.segp + (size_t)(sg + lane) * a.nsp, box, box + KP, bm, bx, m, J.n_bin, a.pcap, &ilo,
                          &len);
            }
            need = (len & (kTrunc - 1)) + kSent + a.nsp;
          }
          int incl = need;  // inclusive prefix sum of the floats each segment takes
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
          }
          const unsigned fit = __ballot_sync(0xffffffffu, has && incl <= a.scap);  // a prefix of the lanes
          const int n = __popc(fit);
          const int total = __shfl_sync(0xffffffffu, incl, max(n - 1, 0));
          const int off = incl - need;
          const int ql = len & (kTrunc - 1);
          if (lane < n) hdr[s].seg[lane] = make_int4(s * a.scap + off, ilo - m, ql, (len & kTrunc) ? 0 : 1);
          if (lane == 0) hdr[s].nseg = n;
          __syncwarp();
          // the slot's previous contents were read through the generic proxy
          fence_proxy_async_smem();
          if (lane == 0) mbar_arrive_expect_tx(&full[s], (uint32_t)total * 4u);
          __syncwarp();
          if (lane < n) {
            const int seg = sg + lane;
            float* dst = slots + (size_t)s * a.scap + off;
            const bool ok =
                dbg_ok(a.dbg, n >= 1 && off + need <= a.scap && ((off & 3) == 0) && ((a.scap & 3) == 0), 7, off,
                       need) &&
                dbg_ok(a.dbg, ilo >= 0 && (ilo & 3) == 0 && (ql & 3) == 0 && ilo + ql <= J.qpitch, 8, ilo, ql) &&
                dbg_ok(a.dbg, (long long)a.off_slots + ((long long)s + 1) * a.scap * 4 <= a.smem_bytes, 9, s, a.scap);
            if (ok) {
              if (ql > 0) bulk_g2s(dst, J.q + (size_t)seg * J.qpitch + ilo, (uint32_t)ql * 4u, &full[s]);
              bulk_g2s(dst + ql, g_zero4, (uint32_t)kSent * 4u, &full[s]);
              bulk_g2s(dst + ql + kSent, J.segp + (size_t)seg * a.nsp, (uint32_t)a.nsp * 4u, &full[s]);
            } else {
              // a self-check failed (debug builds): complete the transaction without copying
              asm volatile("mbarrier.complete_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[s])),
                           "r"((uint32_t)need * 4u)
                           : "memory");
            }
          }
          if (lane == 0) issued[s] = seq + 1u;
          __syncwarp();
          sg += n;
          ++seq;
        }
        if (!go) break;
        if (lane == 0) mbar_arrive(&band_free[b]);
      }
    } else {
      // ------------------------------------------------------------ helper warps (3)
      // One tile ahead of the consumers, in FP64 where the bin decision needs it: each track's
      // FP32 coefficients and offset y0 = x_mid - Bw, whether FP32 decides its bins, each
      // consumer warp's base bin and decision limit, the tile's coefficient box and its bands.
      const int hid = tid - 32;  // 0..95
      const int hw = hid >> 5;   // 0..2
      // Tiles are handed out as CTAs get to them: each CTA's first is its own index, every later
      // one is claimed from a launch-wide counter when the helpers start its prologue (one tile
      // ahead of the consumers), so that faster SMs take more tiles and the launch ends together.
      for (int ltile = 0;; ++ltile) {
        const int b = ltile & 1;
        // the consumers have read the previous tile's data
        if (ltile > 0) (void)warp_wait(pro_free, (uint32_t)((ltile - 1) & 1), flags, a.wait_ns);
        if (ltile > 0 && hid == 0) flags[1] = (int)gridDim.x + atomicAdd(a.tile_ctr, 1);
        if (help_bar_or(flags[0] != 0)) break;
        const int tile = ltile == 0 ? (int)blockIdx.x : flags[1];
        if (tile >= a.n_tiles) {
          // no more tiles: tell the stager and the consumers (once the stager is done with this
          // parity's slot of the tile ids)
          if (ltile >= 2) (void)warp_wait(&band_free[b], (uint32_t)(((ltile - 2) >> 1) & 1), flags, a.wait_ns);
          if (hid == 0) {
            flags[2 + b] = tile;
            mbar_arrive(pro_full);
            mbar_arrive(&band_ready[b]);
          }
          break;
        }
        const int j = job_of(a, tile);
        const JobDesc& J = a.jobs[j];
        const int n_seg = J.n_seg, m = J.m, K = J.K;
        long long tile0;
        int sp_unused, s0, s1;
        tile_range(a, J, tile, j, &tile0, &sp_unused, &s0, &s1);
        const int ns = s1 - s0;
        const long long tend = min(J.N, tile0 + J.tile_tracks);
        if (ltile > 0) {
          // the base bin of each consumer warp, then every track: the helper lanes of round q
          // hold the 32 lanes of consumer warp hw + 3q
          for (int w = hw; w < kConsWarps; w += 3) prologue_base<KP, CUTS>(J, tile0, tend, w, lane, winfo);
          if (help_bar_or(flags[0] != 0)) break;
          int bmin = 0x7fffffff, bmax = -0x7fffffff;
          for (int q = 0; q < 4; ++q)
            prologue_tracks<KP, R, CUTS>(J, tile0, tend, hid + 96 * q, lane, cbuf, winfo, inboxm, bmin, bmax);
          // the coefficient box of the tracks decided in FP32 (a partial per helper warp)
          prologue_box_part<KP, R>(cbuf, inboxm, hid, 4, lane, bmin, bmax, bpart + hw * BW);
        } else {
          // the consumers prepare their first tile themselves: wait for their partials
          (void)warp_wait(parts_ready, 0u, flags, a.wait_ns);
        }
        __threadfence_block();  // the columns in global memory, before the consumers are told
        if (help_bar_or(flags[0] != 0)) break;
        // this parity's box and bands are free once the stager is done with tile ltile - 2
        if (ltile >= 2) (void)warp_wait(&band_free[b], (uint32_t)(((ltile - 2) >> 1) & 1), flags, a.wait_ns);
        float* box = boxes + b * BW;
        if (hid == 0) {
          flags[2 + b] = tile;
          int bm = 0x7fffffff, bx = -0x7fffffff;
          const int nparts = ltile == 0 ? kConsWarps : 3;
          for (int k = 0; k < KP; ++k) {
            float lo = __int_as_float(0x7f800000), hi = -__int_as_float(0x7f800000);
            for (int h = 0; h < nparts; ++h) {
              lo = fminf(lo, bpart[h * BW + k]);
              hi = fmaxf(hi, bpart[h * BW + KP + k]);
            }
            box[k] = lo;
            box[KP + k] = hi;
          }
          for (int h = 0; h < nparts; ++h) {
            bm = min(bm, reinterpret_cast<const int*>(bpart + h * BW)[2 * KP]);
            bx = max(bx, reinterpret_cast<const int*>(bpart + h * BW)[2 * KP + 1]);
          }
          reinterpret_cast<int*>(box)[2 * KP] = bm;
          reinterpret_cast<int*>(box)[2 * KP + 1] = bx;
        }
        if (help_bar_or(flags[0] != 0)) break;
        if (ns <= a.bcap) {
          const int bm = reinterpret_cast<const int*>(box)[2 * KP];
          const int bx = reinterpret_cast<const int*>(box)[2 * KP + 1];
          int* band = bands + b * 2 * a.bcap;
          for (int i = hid; i < ns; i += 96) {
            int lo, len;
            band_of<KP>(J.segp + (size_t)(s0 + i) * a.nsp, box, box + KP, bm, bx, m, J.n_bin, a.pcap, &lo, &len);
            band[2 * i] = lo;
            band[2 * i + 1] = len;
          }
        }
        if (help_bar_or(flags[0] != 0)) break;
        if (hid == 0) {
          if (ltile > 0) mbar_arrive(pro_full);  // the consumers prepared their first tile
          mbar_arrive(&band_ready[b]);
        }
      }
    }
  } else {
    // ================================================================ consumer warpgroups
    setmaxnreg_inc<kConsRegs>();
    const int ctid = tid - kProd;
    const int cwarp = ctid >> 5;
    uint32_t seq = 0;
    bool dead = false;
    for (int ltile = 0; !dead; ++ltile) {
      // -------------------------------------------------------------- tile prologue
      // Each track is evaluated relative to a warp-uniform base bin Bw (the FP64 mid-segment bin
      // of the warp's first track): y = (x_mid - Bw) + sum_k c_k D_k,alpha in FP32, and the bin
      // is Bw + rint(y).  One base per warp keeps a register per track free.  The helper warps
      // prepared y0 = x_mid - Bw, the FP32 coefficients (0 for a track that FP32 cannot decide,
      // whose y0 is 1/2), the warp's base and decision limit, and named the tile.
      // The first tile is this CTA's own and its consumers prepare it themselves (no earlier tile
      // hides that prologue, and twelve warps do it four times as fast as three); each later one
      // comes from the helpers, named in the tile ids (a plain load: the wait acquired the write).
      int tile = (int)blockIdx.x;
      if (ltile > 0) {
        if (!warp_wait(pro_full, (uint32_t)((ltile - 1) & 1), flags, a.wait_ns)) break;
        tile = reinterpret_cast<const int*>(const_cast<const int*>(flags))[2 + (ltile & 1)];
        if (tile >= a.n_tiles) break;
      }
      const int j = job_of(a, tile);
      const JobDesc& J = a.jobs[j];
      const int n_seg = J.n_seg, m = J.m;
      long long tile0;
      int sp, s0, s1;
      tile_range(a, J, tile, j, &tile0, &sp, &s0, &s1);
      const long long tend = min(J.N, tile0 + J.tile_tracks);
      if (ltile == 0) {
        prologue_base<KP, CUTS>(J, tile0, tend, cwarp, lane, winfo);
        __syncwarp();
        int bmin = 0x7fffffff, bmax = -0x7fffffff;
        prologue_tracks<KP, R, CUTS>(J, tile0, tend, ctid, lane, cbuf, winfo, inboxm, bmin, bmax);
        prologue_box_part<KP, R>(cbuf, inboxm, ctid, 1, lane, bmin, bmax, bpart + cwarp * BW);
        __syncwarp();
        if (lane == 0) mbar_arrive(parts_ready);
      }
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
      const WarpInfo wi = winfo[cwarp];
      const int Bw = wi.Bw;
      const float wlim = wi.wlim;  // at most 1/2: the tracks that FP32 cannot decide (y = 1/2) never are
      int nq = 0;                  // entries in this thread's fix-up queue
#pragma unroll
      for (int r = 0; r < R; ++r) {
        acc[r] = 0.f;
        corr[r * kCons + ctid] = 0.f;
        corrl[r * kCons + ctid] = 0.f;
        tot[r * kCons + ctid] = 0.f;
        comp[r * kCons + ctid] = 0.f;
        const float* col = cbuf + r * kCons + ctid;
#pragma unroll
        for (int k = 0; k < KP; ++k) put(c2[r / 2][k], r & 1, col[k * kCR]);
        put(y02[r / 2], r & 1, col[KP * kCR]);
      }
      // segment cuts: warp-uniform margins of the second-order test (mz), the fdot test (mw)
      // and the low-frequency test (mf, against ylo = 10^-3.5 T_SFT - Bw in bin units), as
      // thresholds: included below zin / above win, fin; excluded above zex / below wex, fex
      float zin = 0.f, zex = 0.f, win = 0.f, wex = 0.f, fin = 0.f, fex = 0.f;
      unsigned cutm = 0u;  // tracks whose cuts are decided in FP32 (the others are always pending)
      bool zt = false;     // some track of the warp may reach the second-order cut
      if (CUTS) {
        const float mz = wi.mz, mw = wi.mw, ylo = wi.ylo;
        // 1/2 - wlim bounds |y - (f T_SFT - Bw)| for every decided track of the warp; add the
        // roundings of ylo (FP32, and FP64 below 1e-6 for |10^-3.5 T_SFT| < 2^29)
        const float mf = (0.5f - wlim) + fabsf(ylo) * 2.4e-7f + 1e-6f;
        cutm = inboxm[ctid];
        zt = wi.zt != 0;
        zin = __fsub_rd(1.f, mz);
        zex = __fadd_ru(1.f, mz);
        win = __fadd_ru(1e-13f, mw);
        wex = __fsub_rd(1e-13f, mw);
        fin = __fadd_ru(ylo, mf);
        fex = __fsub_rd(ylo, mf);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(pro_free);
      const f32x2 kC2 = f2pack(12582912.0f, 12582912.0f);  // 1.5 * 2^23 in both lanes
      // -------------------------------------------------------------- segments, a slot at a time
      const unsigned nin = (unsigned)(J.n_bin + 2 * m);
      for (int sg = s0; sg < s1;) {
        const int s = (int)(seq % (uint32_t)NS);
        const uint32_t par = (seq / (uint32_t)NS) & 1u;
        ++seq;
        if (!warp_wait(&full[s], par, flags, a.wait_ns)) {
          dead = true;
          break;
        }
        const int se = sg + min(hdr[s].nseg, s1 - sg);
        const int4* hp = hdr[s].seg;
        for (; sg < se; ++sg, ++hp) {
          if (nq > kQT - R) {
            // not enough queue room for this segment: resolve the queue now, in (segment) order
            for (int i = 0; i < nq; ++i) {
              const uint32_t e = queue[i * kCons + ctid];
              const int r2 = (int)(e & 31u), s2 = (int)(e >> 5);
              {
              const float y = exact_pair<KP, BINS, CUTS>(a, J, tile0 + ctid + r2 * kCons, s2);
              const float x = corr[r2 * kCons + ctid];
              const float sm = x + y, yv = sm - x;
              corrl[r2 * kCons + ctid] += (x - (sm - yv)) + (y - yv);
              corr[r2 * kCons + ctid] = sm;
            }
            }
            nq = 0;
          }
          const int4 h = *hp;  // offset in the slots, centre of the first sum, sums, complete
          const float* q = slots + h.x;
          const float* dsm = q + h.z + kSent;
          float d[KP];
          {
            const float4* dp = reinterpret_cast<const float4*>(dsm);
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
          // its window overlaps the table but its centre lies outside a cut band.
          // (unsigned arithmetic: the offsets wrap modulo 2^32 and only b - qbase matters)
          const int qbase = h.y;
          const unsigned koff = (unsigned)Bw - 0x4B400000u - (unsigned)qbase;
          const unsigned kin = (unsigned)(qbase + m);
          const unsigned qn = (unsigned)h.z;
          f32x2 d2[KP];
#pragma unroll
          for (int k = 0; k < KP; ++k) d2[k] = f2pack(d[k], d[k]);
          // segment-cut forms, each stored twice (E, E, G, G per coefficient): G held in registers
          // for up to 8 coefficients; E (used only when a track of the warp may reach the
          // second-order cut), and G above 8 coefficients, re-read from shared memory per pair
          const uint32_t egs = smem_u32(dsm + cut_col(KP));
          f32x2 g2[kCutRegs ? KP : 1];
          if (kCutRegs) {
#pragma unroll
            for (int k = 0; k < KP; ++k) g2[k] = lds_pair_v(egs + 16u * k + 8u);
          }
          unsigned pend = 0u;
          // one straight-line pass over the track pairs.  COMPLETE: the band holds every reachable
          // centre (a centre outside it reads the zero after it; only FP32-undecided pairs are
          // pending); otherwise pairs whose window overlaps the table but whose centre lies outside
          // the band are pending too.  ZT: evaluate the second-order cut (off when no track of the
          // warp can reach it).
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
                    const int b = (int)off + qbase;
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
                    const int b = (int)off + qbase;
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
          if (h.w) {
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
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if ((sg % kSegTile) == 0) {
          // a 32-segment block is complete: tot + comp holds the sum of the block sums exactly to
          // second order (the error of each FP32 addition, by the two-sum of Knuth, goes into comp)
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const float x = tot[r * kCons + ctid], y = acc[r];
            const float sum = x + y, yv = sum - x;
            const float err = (x - (sum - yv)) + (y - yv);
            tot[r * kCons + ctid] = sum;
            comp[r * kCons + ctid] += err;
            acc[r] = 0.f;
          }
        }
      }
      if (dead) break;
      // -------------------------------------------------------------- tile epilogue
      for (int i = 0; i < nq; ++i) {
        const uint32_t e = queue[i * kCons + ctid];
        const int r2 = (int)(e & 31u), s2 = (int)(e >> 5);
        {
              const float y = exact_pair<KP, BINS, CUTS>(a, J, tile0 + ctid + r2 * kCons, s2);
              const float x = corr[r2 * kCons + ctid];
              const float sm = x + y, yv = sm - x;
              corrl[r2 * kCons + ctid] += (x - (sm - yv)) + (y - yv);
              corr[r2 * kCons + ctid] = sm;
            }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const long long t = tile0 + ctid + r * kCons;
        if (t < tend) {
          const float x = tot[r * kCons + ctid], e = comp[r * kCons + ctid];
          const float ch = corr[r * kCons + ctid], cl = corrl[r * kCons + ctid];
          if (J.seg_split > 1) {
            J.part[(size_t)sp * J.N + t] = ((((double)x + (double)e) + (double)acc[r]) + (double)ch) + (double)cl;
          } else {
            const float sm = x + ch, yv = sm - x;
            const float e1 = (x - (sm - yv)) + (ch - yv);
            J.stat[t] = sm + (((e + acc[r]) + cl) + e1);
          }
        }
      }
    }
  }
  __syncthreads();
  if (flags[0] && tid == 0) {
    // a bounded wait gave up: let the copies of every slot's last filling land before leaving
    // (a slot whose last phase already completed passes at once)
    for (int s = 0; s < NS; ++s) {
      if (issued[s] == 0u) continue;
      const uint32_t use = issued[s] - 1u;
      (void)mbar_wait_bounded(&full[s], (use / (uint32_t)NS) & 1u, kDrainNs);
    }
    atomicExch(a.status, DEV_TIMEOUT);
  }
}

// ---------------------------------------------------------------- host side
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

// Tracks per consumer thread: the large classes fill the registers (no spills at any K); the small
// class (4 for K <= 8) serves launches with fewer tracks than one round of large tiles, whose large
// tiles would be mostly empty slots that still cost their per-segment arithmetic.
constexpr int r_big(int KP) { return KP <= 6 ? 12 : (KP <= 8 ? 9 : (KP <= 16 ? 4 : 2)); }
constexpr int r_big_cuts(int KP) { return KP <= 6 ? 8 : (KP <= 8 ? 6 : 2); }
constexpr int r_small(int KP) { return KP <= 8 ? 4 : r_big(KP); }
constexpr int r_small_cuts(int KP) { return KP <= 8 ? 4 : r_big_cuts(KP); }
inline int r_of(int KP, bool cuts, bool small) {
  return small ? (cuts ? r_small_cuts(KP) : r_small(KP)) : (cuts ? r_big_cuts(KP) : r_big(KP));
}

template <int KP, int R, bool BINS, bool CUTS, int MJ>
int launch_one(const EvalArgs<MJ>& a0, int grid, size_t smem, cudaStream_t st) {
  auto kern = eval_stat_kernel<KP, R, BINS, CUTS, MJ>;
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

// Launch the kernel instantiation for KP coefficient slots (one translation unit per KP pair).
template <int KP, int MJ>
int launch_kp(const EvalArgs<MJ>& a, bool bins, bool cuts, bool small, int grid, size_t smem, cudaStream_t st) {
  if (small && r_small(KP) != r_big(KP)) {
    if (cuts) return launch_one<KP, r_small_cuts(KP), false, true, MJ>(a, grid, smem, st);
    return launch_one<KP, r_small(KP), false, false, MJ>(a, grid, smem, st);
  }
  if (cuts) return launch_one<KP, r_big_cuts(KP), false, true, MJ>(a, grid, smem, st);
  if constexpr (MJ == 1) {
    if (bins) return launch_one<KP, r_big(KP), true, false, MJ>(a, grid, smem, st);
  }
  return launch_one<KP, r_big(KP), false, false, MJ>(a, grid, smem, st);
}

#define TFS_DECLARE_KP(KPV)                                                                            \
  extern template int launch_kp<KPV, 1>(const EvalArgs<1>&, bool, bool, bool, int, size_t, cudaStream_t);  \
  extern template int launch_kp<KPV, kMaxJobs>(const EvalArgs<kMaxJobs>&, bool, bool, bool, int, size_t, cudaStream_t);
TFS_DECLARE_KP(2)
TFS_DECLARE_KP(4)
TFS_DECLARE_KP(6)
TFS_DECLARE_KP(8)
TFS_DECLARE_KP(16)
TFS_DECLARE_KP(32)
#undef TFS_DECLARE_KP

#define TFS_INSTANTIATE_KP(KPV)                                                                 \
  template int launch_kp<KPV, 1>(const EvalArgs<1>&, bool, bool, bool, int, size_t, cudaStream_t); \
  template int launch_kp<KPV, kMaxJobs>(const EvalArgs<kMaxJobs>&, bool, bool, bool, int, size_t, cudaStream_t);

}  // namespace tfs
