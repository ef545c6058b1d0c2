// Fused track evaluation + gather + reduction for the semi-coherent statistic
// (paper Sec. II.B Eq. det_stat, nearest-bin reading with +-m neighbours;
// tracks from the SVD basis of Sec. II.C).
//
// Persistent, warp-specialised kernel: one CTA per SM walks tiles of 256*R
// tracks (static round-robin).  Three warpgroups:
//
//   producer warpgroup (128 threads, registers lowered with setmaxnreg) --
//     thread 0 stages, for every segment alpha of the tile, the band of table
//     row alpha the tile can touch (a rigorous interval bound from the tile's
//     coefficient box) with a 1-D bulk copy (cp.async.bulk) completing on an
//     mbarrier; the warpgroup then turns the staged band into window sums
//         Q[b] = sum_{j=-m..m} P[alpha][b+j]       (FP32, fixed order)
//     with 16-byte vector loads and lane shuffles, and signals the Q slot's
//     "full" barrier;
//   two consumer warpgroups (256 threads, registers raised with setmaxnreg) --
//     per segment, each thread evaluates x = f T_SFT for its R tracks in FP32,
//         y = (x_mid - B) + sum_k c_k D_k,alpha,    b = B + rint(y),
//     (B = rint(x_mid), x_mid an FP64 per-track constant) and adds Q[b] with a
//     single shared load, then its warp arrives on the slot's "empty" barrier.
//     Pairs within a warp-uniform error bound g of a half-integer, and pairs
//     whose centre falls outside the staged band, go to the thread's own queue
//     and are recomputed at the end of the tile in the FP64 operation order
//     of the oracle (separately rounded products and sums): every bin equals
//     the FP64 bin exactly, ties included.
//
// No CTA-wide barrier runs inside the segment loop: producer and consumers
// meet only on mbarriers (Q ring, staging ring, per-tile box hand-off), so the
// consumer warps run up to kNQ segments apart.  FP32 sums are flushed to a
// second accumulator every 32 segments; fix-up contributions accumulate
// separately in segment order, so a track's result does not depend on its
// tile neighbours.  Every wait is bounded (2 s) and warp-uniform; a timeout
// makes every role leave its loops and the call return TFS_ERR_TIMEOUT.
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

constexpr int kProd = 128;            // producer warpgroup
constexpr int kCons = 256;            // two consumer warpgroups
constexpr int kThreads = kProd + kCons;
constexpr int kConsWarps = kCons / 32;
constexpr int kProdRegs = 72;         // setmaxnreg targets: 128*72 + 256*216 = 384*168
constexpr int kConsRegs = 216;
static_assert(kProd * kProdRegs + kCons * kConsRegs <= kThreads * 168, "register split exceeds the launch");
constexpr int kNQ = 4;                // window-sum (Q) slots
constexpr int kNP = 4;                // staging slots
constexpr int kQT = 32;               // fix-up queue entries per consumer thread
constexpr int kPadL = 16;             // zero elements before the staged band in a staging slot
constexpr int kSegTile = 32;          // FP32 partial sums are flushed every kSegTile segments

struct EvalArgs {
  const void* table;
  const float* scales;
  int n_seg, n_bin, row_stride;
  double T;
  const double* U;  // [K][n_seg]
  int K, alpha_mid;
  const float* segp;  // [n_seg][nsp]
  int nsp;
  const float* dmax;  // [KP]
  const float* umax;  // [KP]
  const double* coeffs;
  const double* f_ref;
  long long N;
  int m;
  float* stat;
  unsigned long long* tie_count;
  long long* tie_track;
  int* tie_seg;
  int tie_cap;
  int* status;
  int* bins_out;  // [N][n_seg] (BINS instantiations); INT_MIN / INT_MAX: window wholly below / above
  unsigned long long* dbg;  // self-check record (TFS_DEBUG_CHECKS builds)
  int smem_bytes;
  int qcap;      // floats per Q slot (>= kPadL + pcap + vector tail)
  int pcap;      // table elements of band per staging slot (multiple of 16 bytes)
  int n_tiles;
  // shared-memory carve-up (byte offsets)
  int off_qhdr, off_red, off_flags, off_queue, off_acc, off_q, off_p;
  int off_seg;  // resident copy of segp [n_seg][nsp] and scales [n_seg] (-1: read from global)
};

struct QHdr {
  int qbase;  // window centre held at q[ws_lo]
  int qn;     // valid centres from there on
  int ws_lo;  // first valid window start in the slot
  int pad;
};

#ifdef TFS_DEBUG_CHECKS
__device__ __forceinline__ bool dbg_ok(const EvalArgs& a, bool cond, int where, long long i0, long long i1) {
  if (!cond && a.dbg) {
    if (atomicAdd(&a.dbg[0], 1ull) == 0ull) {
      a.dbg[1] = (unsigned long long)where;
      a.dbg[2] = (unsigned long long)i0;
      a.dbg[3] = (unsigned long long)i1;
    }
  }
  return cond;
}
#else
__device__ __forceinline__ bool dbg_ok(const EvalArgs&, bool, int, long long, long long) { return true; }
#endif

// Window sum from the table in global memory; elements outside [0, n_bin) are 0.
// The additions run in the same order as the shared-memory window sums.
template <int DT>
__device__ __forceinline__ float window_global(const EvalArgs& a, int seg, int lo, int W, float scale) {
  using S = Store<DT>;
  const typename S::T* row = static_cast<const typename S::T*>(a.table) + (size_t)seg * a.row_stride;
  float v = 0.f;
  for (int j = 0; j < W; ++j) {
    const int k = lo + j;
    const float p = (k >= 0 && k < a.n_bin) ? S::ld(row + k) : 0.f;
    v += S::scaled ? p * scale : p;
  }
  return v;
}

__device__ __forceinline__ void report_tie(const EvalArgs& a, long long t, int seg) {
  const unsigned long long i = atomicAdd(a.tie_count, 1ull);
  if (i < (unsigned long long)a.tie_cap) {
    a.tie_track[i] = t;
    a.tie_seg[i] = seg;
  }
}

// FP64 bin of (track t, segment seg) in the oracle's operation order, and its
// window sum from global memory.
template <int DT, bool BINS>
__device__ float exact_pair(const EvalArgs& a, long long t, int seg) {
  if (!dbg_ok(a, t >= 0 && t < a.N && seg >= 0 && seg < a.n_seg, 1, t, seg)) return 0.f;
  double f = a.f_ref ? a.f_ref[t] : 0.0;
  const double* c = a.coeffs + t * (long long)a.K;
  for (int k = 0; k < a.K; ++k) f = __dadd_rn(f, __dmul_rn(c[k], a.U[(size_t)k * a.n_seg + seg]));
  const double x = __dmul_rn(f, a.T);
  int* bo = BINS ? a.bins_out + t * (long long)a.n_seg + seg : nullptr;
  if (!isfinite(x)) {
    if (BINS) *bo = 0x7fffffff;
    return 0.f;
  }
  const double fl = floor(x);
  if (fabs(__dsub_rn(__dsub_rn(x, fl), 0.5)) <= 1e-9) report_tie(a, t, seg);
  const double z = __dadd_rn(x, 0.5);
  const int m = a.m;
  if (z < -(double)m || z >= (double)a.n_bin + (double)m) {
    if (BINS) *bo = z < 0.0 ? (int)0x80000000 : 0x7fffffff;
    return 0.f;
  }
  const int b = (int)floor(z);
  if (BINS) *bo = b;
  const float scale = Store<DT>::scaled ? a.scales[seg] : 1.f;
  return window_global<DT>(a, seg, b - m, 2 * m + 1, scale);
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
// Warp-uniform bounded wait: every lane observes the phase (acquire); the timeout and
// abort decisions are lane 0's, broadcast to the warp.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* flags) {
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    const uint32_t done = mbar_try(bar, parity);
    if (__all_sync(0xffffffffu, done)) return true;
    if ((it & 31) == 0) {
      int stop = 0;
      if ((threadIdx.x & 31) == 0) {
        const uint64_t now = global_ns();
        if (it == 0) t0 = now;
        stop = flags[0] != 0 || (it != 0 && now - t0 > kWaitLimitNs);
      }
      if (__shfl_sync(0xffffffffu, stop, 0)) return false;
    }
  }
}
// Single-thread bounded wait (producer thread 0).
__device__ __forceinline__ bool thread_wait(uint64_t* bar, uint32_t parity, volatile int* flags) {
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 31) == 0) {
      const uint64_t now = global_ns();
      if (it == 0) t0 = now;
      else if (flags[0] != 0 || now - t0 > kWaitLimitNs) return false;
    }
  }
}
__device__ __forceinline__ void prod_bar() {  // named barrier 1 among the producer warpgroup
  asm volatile("bar.sync 1, %0;" ::"n"(kProd) : "memory");
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

template <int DT, int KP, int R, bool BINS>
__global__ void __launch_bounds__(kThreads, 1) eval_stat_kernel(const EvalArgs a) {
  using S = Store<DT>;
  using T = typename S::T;
  constexpr int EALIGN = 16 / S::esize;  // table elements per 16 bytes (= EPV)
  constexpr int RW = 2 * KP + 2;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  uint64_t* full_p = bars;                     // [kNP] staging copies landed (tx)
  uint64_t* full_q = bars + kNP;               // [kNQ] window sums ready (producer threads)
  uint64_t* empty_q = bars + kNP + kNQ;        // [kNQ] consumers done with the slot (consumer warps)
  uint64_t* tile_ready = bars + kNP + 2 * kNQ; // [2] a tile's coefficient box is ready (consumer warps)
  QHdr* qhdr = reinterpret_cast<QHdr*>(smem + a.off_qhdr);     // [kNQ], then [kNQ][nsp] floats of D
  float* qdseg = reinterpret_cast<float*>(smem + a.off_qhdr + kNQ * sizeof(QHdr));
  float* red = reinterpret_cast<float*>(smem + a.off_red);     // [2][kConsWarps][RW]
  volatile int* flags = reinterpret_cast<volatile int*>(smem + a.off_flags);  // [0] abort, [1] producer go
  uint32_t* queue = reinterpret_cast<uint32_t*>(smem + a.off_queue);          // [kQT][kCons]
  float* corr = reinterpret_cast<float*>(smem + a.off_acc);                   // [R][kCons]
  float* tot = corr + R * kCons;                                              // [R][kCons]
  float* qslots = reinterpret_cast<float*>(smem + a.off_q);                   // [kNQ][qcap]
  unsigned char* pslots = smem + a.off_p;                                     // [kNP][pslot_bytes]
  const int pslot_bytes = (kPadL + a.pcap + EALIGN) * S::esize + a.nsp * 4;

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int m = a.m;
  const int W = 2 * m + 1;
  const int n_seg = a.n_seg;

  if (tid < 4) flags[tid] = 0;
  if (tid == 0) {
    for (int i = 0; i < kNP; ++i) mbar_init(&full_p[i], 1);
    for (int i = 0; i < kNQ; ++i) {
      mbar_init(&full_q[i], kProd);
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
  // the per-segment basis deltas (and FP8 scales) stay resident for the whole launch
  const float* segp = a.segp;
  const float* scales = a.scales;
  if (a.off_seg >= 0) {
    float* ss = reinterpret_cast<float*>(smem + a.off_seg);
    for (int i = tid; i < n_seg * a.nsp; i += kThreads) ss[i] = a.segp[i];
    if (S::scaled)
      for (int i = tid; i < n_seg; i += kThreads) ss[n_seg * a.nsp + i] = a.scales[i];
    segp = ss;
    scales = ss + n_seg * a.nsp;
  }
  __syncthreads();

  if (tid < kProd) {
    // ================================================================ producer warpgroup
    setmaxnreg_dec<kProdRegs>();
    uint32_t p_issue = 0, p_use = 0, q_seq = 0;
    int* plo_s = reinterpret_cast<int*>(smem + a.off_flags) + 4;  // [kNP] band start per staging slot
    int* plen_s = plo_s + kNP;                                     // [kNP] band length
    float bx_lo[KP], bx_hi[KP];   // the current tile's coefficient box (thread 0)
    int bm = 0, bxm = -1;
    auto stage = [&](int sg) {  // thread 0
      const int ps = (int)(p_issue % kNP);
      const float* dr = segp + (size_t)sg * a.nsp;
      const float* drg = a.segp + (size_t)sg * a.nsp;  // the bulk copy's source stays global
      int blo = 0, blen = 0;
      if (bm <= bxm) {
        float lo = 0.f, hi = 0.f, mag = 0.f;
        for (int k = 0; k < KP; ++k) {
          const float d = dr[k];
          const float p1 = bx_lo[k] * d, p2 = bx_hi[k] * d;
          lo += fminf(p1, p2);
          hi += fmaxf(p1, p2);
          mag += fmaxf(fabsf(p1), fabsf(p2));
        }
        // FP32 with a margin that covers its rounding: the band only steers staging
        const float fm = 4.f + 1e-5f * mag + 1e-6f * fmaxf(fabsf((float)bm), fabsf((float)bxm));
        const float bl = fmaxf(floorf((float)bm + lo - fm) - 2 * m, 0.f);
        const float bh = fminf(floorf((float)bxm + 1.f + hi + fm) + 2 * m, (float)(a.n_bin - 1));
        if (bl <= bh) {
          const int il = ((int)bl) & ~(EALIGN - 1);
          int ih = ((int)bh + EALIGN) & ~(EALIGN - 1);
          ih = min(ih, a.row_stride);
          blo = il;
          blen = min(ih - il, a.pcap);
        }
      }
      plo_s[ps] = blo;
      plen_s[ps] = blen;
      unsigned char* dst = pslots + (size_t)ps * pslot_bytes;
      uint32_t dbytes = (uint32_t)blen * S::esize;
      {
        const long long src_el = (long long)sg * a.row_stride + blo;
        const bool ok =
            dbg_ok(a, (long long)a.off_p + (long long)(ps + 1) * pslot_bytes <= a.smem_bytes, 7, ps, pslot_bytes) &&
            dbg_ok(a, blo >= 0 && src_el + blen <= (long long)a.n_seg * a.row_stride, 8, src_el, blen) &&
            dbg_ok(a, ((a.off_p + (long long)ps * pslot_bytes) & 15) == 0 && (dbytes & 15) == 0 &&
                          ((src_el * S::esize) & 15) == 0 && ((pslot_bytes & 15) == 0), 9, ps, src_el);
        if (!ok) dbytes = 0;
      }
      fence_proxy_async_smem();  // the slot's previous contents were read through the generic proxy
      mbar_arrive_expect_tx(&full_p[ps], dbytes + (uint32_t)a.nsp * 4u);
      if (dbytes > 0)
        bulk_g2s(dst + kPadL * S::esize, static_cast<const T*>(a.table) + (size_t)sg * a.row_stride + blo, dbytes,
                 &full_p[ps]);
      bulk_g2s(dst + (size_t)(kPadL + a.pcap + EALIGN) * S::esize, drg, (uint32_t)a.nsp * 4u, &full_p[ps]);
      ++p_issue;
    };
    int ltile = 0;
    bool stop = false;
    for (int tile = blockIdx.x; tile < a.n_tiles && !stop; tile += gridDim.x, ++ltile) {
      // the consumers' coefficient box of this tile
      if (tid == 0) {
        int go = thread_wait(&tile_ready[ltile & 1], (uint32_t)((ltile >> 1) & 1), flags);
        if (go) {
          const float* rb = red + (ltile & 1) * kConsWarps * RW;
          bm = 0x7fffffff;
          bxm = -0x7fffffff;
          for (int k = 0; k < KP; ++k) {
            bx_lo[k] = __int_as_float(0x7f800000);
            bx_hi[k] = -__int_as_float(0x7f800000);
          }
          for (int w = 0; w < kConsWarps; ++w) {
            for (int k = 0; k < KP; ++k) {
              bx_lo[k] = fminf(bx_lo[k], rb[w * RW + k]);
              bx_hi[k] = fmaxf(bx_hi[k], rb[w * RW + KP + k]);
            }
            bm = min(bm, reinterpret_cast<const int*>(rb)[w * RW + 2 * KP]);
            bxm = max(bxm, reinterpret_cast<const int*>(rb)[w * RW + 2 * KP + 1]);
          }
          for (int sg = 0; sg < kNP && sg < n_seg; ++sg) stage(sg);
        } else {
          flags[0] = 1;
        }
      }
      for (int sg = 0; sg < n_seg; ++sg) {
        const int ps = (int)(p_use % kNP), qs = (int)(q_seq % kNQ);
        if (tid == 0) {
          int go = !flags[0] && thread_wait(&full_p[ps], (p_use / kNP) & 1u, flags);
          if (go && q_seq >= kNQ) go = thread_wait(&empty_q[qs], ((q_seq / kNQ) - 1u) & 1u, flags);
          flags[1] = go ? plo_s[ps] : 0;
          flags[2] = go ? plen_s[ps] : 0;
          flags[3] = go;
          if (!go) flags[0] = 1;
        }
        prod_bar();
        if (!flags[3]) {
          stop = true;
          break;
        }
        const int plo = flags[1], plen = flags[2];
        const unsigned char* src = pslots + (size_t)ps * pslot_bytes;
        // valid window starts (slot coordinates): wholly inside the staged band, or in the zero
        // pad when the band starts at bin 0
        // (windows reaching further below bin 0 than the pad covers are left to the FP64 queue)
        const int ws_lo = plo == 0 ? max(kPadL - m, 0) : kPadL;
        const int ws_hi = kPadL + plen - (W - 1);
        const int qn = plen == 0 ? 0 : max(0, min(ws_hi, a.qcap - EALIGN) - ws_lo);
        float* q = qslots + (size_t)qs * a.qcap;
        const float scale = S::scaled ? scales[sg] : 1.f;
        if (m <= 2) {
          // vector path: thread j sums the windows starting at its EPV elements, taking the
          // next 2m elements from the next lane (or, on a warp's last lane, from memory)
          // vectors holding valid window starts, and (up to 4 elements further) the ones their
          // windows reach into; both stay inside the slot (band + one vector of tail)
          const int nvec = (ws_lo + qn + EALIGN - 1) / EALIGN;
          const int nload = min((ws_lo + qn + 4 + EALIGN - 1) / EALIGN, kPadL / EALIGN + a.pcap / EALIGN + 1);
          for (int v0 = 0; v0 < nvec; v0 += kProd) {
            const int vi = v0 + tid;
            float e[EALIGN + 4];
            uint4 raw = make_uint4(0u, 0u, 0u, 0u);
            if (vi < nload) raw = reinterpret_cast<const uint4*>(src)[vi];
            unpack16<DT>(raw, scale, e);
            float nx[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) nx[j] = __shfl_down_sync(0xffffffffu, e[j], 1);
            if (lane == 31 && vi < nvec) {
              const T* tail = reinterpret_cast<const T*>(src) + (size_t)(vi + 1) * EALIGN;
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const float p = S::ld(tail + j);
                nx[j] = S::scaled ? p * scale : p;
              }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) e[EALIGN + j] = nx[j];
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
                for (int i = 0; i < EALIGN; ++i) out[i] = ((((0.f + e[i]) + e[i + 1]) + e[i + 2]) + e[i + 3]) + e[i + 4];
              }
              float4* qv = reinterpret_cast<float4*>(q + (size_t)vi * EALIGN);
#pragma unroll
              for (int i4 = 0; i4 < EALIGN / 4; ++i4)
                qv[i4] = make_float4(out[4 * i4], out[4 * i4 + 1], out[4 * i4 + 2], out[4 * i4 + 3]);
            }
          }
        } else {
          const T* pb = reinterpret_cast<const T*>(src);
          for (int ws = ws_lo + tid; ws < ws_lo + qn; ws += kProd) {
            float s = 0.f;
            for (int j = 0; j < W; ++j) {
              const float p = S::ld(pb + ws + j);
              s += S::scaled ? p * scale : p;
            }
            q[ws] = s;
          }
        }
        if (tid < a.nsp)
          qdseg[qs * a.nsp + tid] =
              reinterpret_cast<const float*>(src + (size_t)(kPadL + a.pcap + EALIGN) * S::esize)[tid];
        if (tid == 0) {
          QHdr h;
          h.ws_lo = ws_lo;
          h.qn = qn;
          h.qbase = plo - kPadL + ws_lo + m;  // centre of the window starting at ws_lo
          h.pad = 0;
          qhdr[qs] = h;
        }
        mbar_arrive(&full_q[qs]);  // every producer thread releases its own writes
        prod_bar();                // the staging slot has been read by the whole warpgroup
        ++p_use;
        ++q_seq;
        if (tid == 0 && sg + kNP < n_seg) stage(sg + kNP);
      }
    }
  } else {
    // ================================================================ consumer warpgroups
    setmaxnreg_inc<kConsRegs>();
    const int ctid = tid - kProd;
    const int cwarp = ctid >> 5;
    uint32_t q_seq = 0;
    int ltile = 0;
    for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++ltile) {
      if (__any_sync(0xffffffffu, flags[0] != 0)) break;  // warp-uniform
      const long long tile0 = (long long)tile * (kCons * R);
      // -------------------------------------------------------------- tile prologue
      float c[R][KP];
      int B[R];
      float y0[R], acc[R];
      float wlim = 2.f;  // warp-uniform decision limit: min over the warp's tracks of 1/2 - g
      int nq = 0;        // entries in this thread's fix-up queue
      {
        float cmn[KP], cmx[KP];
        int bmin = 0x7fffffff, bmax = -0x7fffffff;
#pragma unroll
        for (int k = 0; k < KP; ++k) {
          cmn[k] = __int_as_float(0x7f800000);
          cmx[k] = -__int_as_float(0x7f800000);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
          acc[r] = 0.f;
          B[r] = -(1 << 29);  // inactive slot: y = 0 is never queued and b is always out of range
          y0[r] = 0.f;
#pragma unroll
          for (int k = 0; k < KP; ++k) c[r][k] = 0.f;
          corr[r * kCons + ctid] = 0.f;
          tot[r * kCons + ctid] = 0.f;
          const long long t = tile0 + ctid + r * kCons;
          if (t < a.N) {
            const double fr = a.f_ref ? a.f_ref[t] : 0.0;
            double f = fr;
            float A = 0.f, Um = fabsf((float)fr);
            const double* cp = a.coeffs + t * (long long)a.K;
            float cf[KP];
#pragma unroll
            for (int k = 0; k < KP; ++k) {
              const double cd = (k < a.K) ? cp[k] : 0.0;
              if (k < a.K) f = fma(cd, a.U[(size_t)k * n_seg + a.alpha_mid], f);
              cf[k] = (float)cd;
              A = fmaf(fabsf(cf[k]), a.dmax[k], A);
              Um = fmaf(fabsf(cf[k]), a.umax[k], Um);
            }
            A *= 1.0001f;  // covers the FP32 rounding of the bounds (|fl32(c)| <= |c| (1 + 2^-24))
            Um *= 1.0001f;
            const double xm = f * a.T;
            // |fp32 estimate - exact x| <= err = 2^-24 ((K+1)/2 + (K+2.001) A) + e64, where
            // e64 = 2^-47 T (|f_ref| + sum_k |c_k| max|U_k|) bounds every FP64 rounding (x_mid, the
            // deltas D, and the oracle's own evaluation).  Pairs closer than g to a half-integer
            // are resolved in FP64; outside that band the exact, the oracle's and this bin
            // coincide and none of them is within the 1e-9 tie band.
            const float e64 = 7.105427357601002e-15f * (float)a.T * Um;
            const float err = 5.9604644775390625e-08f * (0.5f * (a.K + 1) + (a.K + 2.001f) * A) + e64;
            const float g = 1.25f * (err + e64) + 4e-9f;
            const bool exact = !(fabs(xm) < 1073741824.0) || !(g < 0.25f) || !(A < 1048576.0f);
            if (!exact) {
              const double Bd = rint(xm);
              B[r] = (int)Bd;
              y0[r] = (float)(xm - Bd);
              wlim = fminf(wlim, __fsub_rd(0.5f, g));
#pragma unroll
              for (int k = 0; k < KP; ++k) {
                c[r][k] = cf[k];
                cmn[k] = fminf(cmn[k], c[r][k]);
                cmx[k] = fmaxf(cmx[k], c[r][k]);
              }
              bmin = min(bmin, B[r]);
              bmax = max(bmax, B[r]);
            } else {
              // every pair of this track takes the FP64 path: y = 1/2 exactly is never decided
              B[r] = 0;
              y0[r] = 0.5f;
            }
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wlim = fminf(wlim, __shfl_xor_sync(0xffffffffu, wlim, o));
#pragma unroll
        for (int k = 0; k < KP; ++k) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            cmn[k] = fminf(cmn[k], __shfl_xor_sync(0xffffffffu, cmn[k], o));
            cmx[k] = fmaxf(cmx[k], __shfl_xor_sync(0xffffffffu, cmx[k], o));
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          bmin = min(bmin, __shfl_xor_sync(0xffffffffu, bmin, o));
          bmax = max(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
        }
        if (lane == 0) {
          float* rb = red + (ltile & 1) * kConsWarps * RW + cwarp * RW;
#pragma unroll
          for (int k = 0; k < KP; ++k) {
            rb[k] = cmn[k];
            rb[KP + k] = cmx[k];
          }
          reinterpret_cast<int*>(rb)[2 * KP] = bmin;
          reinterpret_cast<int*>(rb)[2 * KP + 1] = bmax;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&tile_ready[ltile & 1]);
      }
      // -------------------------------------------------------------- segments
      bool ok = true;
      for (int sg = 0; sg < n_seg; ++sg) {
        const int qs = (int)(q_seq % kNQ);
        if (nq > kQT - R) {
          // not enough queue room for this segment: resolve the queue now, in (segment) order
          for (int i = 0; i < nq; ++i) {
            const uint32_t e = queue[i * kCons + ctid];
            const int r2 = (int)(e & 31u), s2 = (int)(e >> 5);
            corr[r2 * kCons + ctid] += exact_pair<DT, BINS>(a, tile0 + ctid + r2 * kCons, s2);
          }
          nq = 0;
        }
        if (!warp_wait(&full_q[qs], (q_seq / kNQ) & 1u, flags)) {
          flags[0] = 1;
          ok = false;
          break;
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
        // pass 1 (straight-line over the R tracks): slot offsets and FP32 decisions.
        // off = b - qbase = B + (bits(tt) - bits(1.5 * 2^23)) - qbase; the window of b overlaps
        // the table iff 0 <= b + m < n_bin + 2m, i.e. (unsigned)(off + qbase + m) < n_bin + 2m.
        const int koff = -0x4B400000 - h.qbase;
        const int kin = h.qbase + m;
        const unsigned nin = (unsigned)(a.n_bin + 2 * m);
        const unsigned qn = (unsigned)h.qn;
        unsigned offv[R];
        unsigned undecided = 0u, outside = 0u;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          float y = y0[r];
#pragma unroll
          for (int k = 0; k < KP; ++k) y = fmaf(c[r][k], d[k], y);
          const float tt = y + 12582912.0f;  // 1.5 * 2^23: rounds y to an integer (|y| < 2^22)
          const float dd = y - (tt - 12582912.0f);
          const unsigned off = (unsigned)(B[r] + __float_as_int(tt) + koff);
          offv[r] = off;
          if (!(fabsf(dd) < wlim)) undecided |= 1u << r;
          if (off >= qn && (unsigned)((int)off + kin) < nin) outside |= 1u << r;
        }
        const unsigned pend = undecided | outside;
        // pass 2 (straight-line): one shared load per track, masked; the address is always valid
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const unsigned off = offv[r];
          const bool use = off < qn && !((pend >> r) & 1u);
          const float v = q[use ? off : 0u];
          acc[r] += use ? v : 0.f;
        }
        // pass 3 (rare): queue the undecided pairs and those whose window lies outside the band
        if (pend) {
          for (unsigned mk = pend; mk; mk &= mk - 1u) {
            const int r = __ffs(mk) - 1;
            queue[nq * kCons + ctid] = ((uint32_t)sg << 5) | (uint32_t)r;
            ++nq;
          }
        }
        if (BINS) {
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int b = (int)offv[r] + h.qbase;
            const long long t = tile0 + ctid + r * kCons;
            if (t < a.N && !((pend >> r) & 1u))
              a.bins_out[t * n_seg + sg] = (b + m < 0) ? (int)0x80000000 : (b - m >= a.n_bin ? 0x7fffffff : b);
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
        ++q_seq;
      }
      if (!ok) break;
      // -------------------------------------------------------------- tile epilogue
      for (int i = 0; i < nq; ++i) {
        const uint32_t e = queue[i * kCons + ctid];
        const int r2 = (int)(e & 31u), s2 = (int)(e >> 5);
        corr[r2 * kCons + ctid] += exact_pair<DT, BINS>(a, tile0 + ctid + r2 * kCons, s2);
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const long long t = tile0 + ctid + r * kCons;
        if (t < a.N) a.stat[t] = (tot[r * kCons + ctid] + acc[r]) + corr[r * kCons + ctid];
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
template <int DT, int KP, int R, bool BINS>
int launch_one(const EvalArgs& a0, int grid, size_t smem, cudaStream_t st) {
  auto kern = eval_stat_kernel<DT, KP, R, BINS>;
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

template <int DT>
int launch_eval_dt(const EvalLaunch& L, const EvalTuning& tune, cudaStream_t st) {
  constexpr int esize = Store<DT>::esize;
  constexpr int EPV = 16 / esize;
  const tfs_table* tb = L.table;
  const SegParams* sp = L.sp;
  const int KP = sp->KP;
  const int R = KP <= 8 ? 16 : (KP <= 16 ? 8 : 4);  // must match the instantiations below
  if (L.N <= 0) return TFS_OK;

  EvalArgs a{};
  a.table = tb->data;
  a.scales = tb->scales;
  a.n_seg = (int)tb->n_seg;
  a.n_bin = (int)tb->n_bin;
  a.row_stride = (int)tb->row_stride;
  a.T = tb->T_sft;
  a.U = L.basis->U;
  a.K = L.basis->K;
  a.alpha_mid = sp->alpha_mid;
  a.segp = sp->segp;
  a.nsp = sp->nsp;
  a.dmax = sp->dmax;
  a.umax = sp->umax;
  a.coeffs = L.coeffs;
  a.f_ref = L.f_ref;
  a.N = L.N;
  a.m = L.m;
  a.stat = L.stat;
  a.tie_count = L.tie_count;
  a.tie_track = reinterpret_cast<long long*>(L.tie_track);
  a.tie_seg = L.tie_seg;
  a.tie_cap = L.tie_cap;
  a.status = L.status;
  a.bins_out = L.bins_out;
  a.dbg = L.dbg;

  // staging slots hold up to pcap band elements; Q slots the window sums of a whole slot
  int pcap = tune.cap > 0 ? tune.cap : 2048;
  pcap = std::max(64, std::min(pcap, (int)tb->row_stride));
  pcap = (pcap + 31) / 32 * 32;
  if (pcap > (int)tb->row_stride) pcap = (int)tb->row_stride;
  a.pcap = pcap;
  a.qcap = kPadL + pcap + 2 * EPV;
  const int RW = 2 * KP + 2;
  const size_t pslot_bytes = (size_t)(kPadL + pcap + EPV) * esize + sp->nsp * 4;
  size_t off = 8 * (kNP + 2 * kNQ + 2);
  off = (off + 15) & ~(size_t)15;
  a.off_qhdr = (int)off;  off += kNQ * sizeof(QHdr) + (size_t)kNQ * sp->nsp * 4;
  off = (off + 15) & ~(size_t)15;
  a.off_red = (int)off;   off += (size_t)2 * kConsWarps * RW * 4;
  off = (off + 15) & ~(size_t)15;
  a.off_flags = (int)off; off += 16 + 2 * kNP * 4;  // flags, then the staging slots' band records
  a.off_queue = (int)off; off += (size_t)kQT * kCons * 4;
  a.off_acc = (int)off;   off += (size_t)2 * R * kCons * 4;
  off = (off + 127) & ~(size_t)127;
  a.off_q = (int)off;     off += (size_t)kNQ * a.qcap * 4;
  off = (off + 127) & ~(size_t)127;
  a.off_p = (int)off;     off += (size_t)kNP * pslot_bytes;
  off = (off + 15) & ~(size_t)15;
  const size_t seg_bytes = (size_t)tb->n_seg * (sp->nsp + 1) * 4;
  a.off_seg = -1;
  if (off + seg_bytes <= 200 * 1024) {  // resident per-segment data when it fits
    a.off_seg = (int)off;
    off += seg_bytes;
  }
  const size_t smem = off;
  a.smem_bytes = (int)smem;
  if (smem > 227 * 1024) {
    set_error("statistic kernel needs %zu bytes of shared memory", smem);
    return TFS_ERR_INVALID_ARG;
  }

  const long long tile = (long long)kCons * R;
  const long long nt = (L.N + tile - 1) / tile;
  if (nt > 0x7fffffffLL) {
    set_error("too many tracks for one launch");
    return TFS_ERR_INVALID_ARG;
  }
  a.n_tiles = (int)nt;
  const int grid = (int)std::min<long long>(nt, (long long)sm_count());
  const bool bins = L.bins_out != nullptr;

#define TFS_LAUNCH_KP(KPV, RV)                                                          \
  if (KP == KPV) {                                                                      \
    return bins ? launch_one<DT, KPV, RV, true>(a, grid, smem, st)                      \
                : launch_one<DT, KPV, RV, false>(a, grid, smem, st);                    \
  }
  TFS_LAUNCH_KP(2, 16)
  TFS_LAUNCH_KP(4, 16)
  TFS_LAUNCH_KP(6, 16)
  TFS_LAUNCH_KP(8, 16)
  TFS_LAUNCH_KP(16, 8)
  TFS_LAUNCH_KP(32, 4)
#undef TFS_LAUNCH_KP
  (void)R;
  set_error("unsupported basis size K=%d", L.basis->K);
  return TFS_ERR_INVALID_ARG;
}

}  // namespace tfs
