// Fused track evaluation + gather + reduction for the semi-coherent statistic
// (paper Sec. II.B Eq. det_stat, nearest-bin reading with +-m neighbours;
// tracks from the SVD basis of Sec. II.C).
//
// One CTA of 256 threads owns a tile of 256 * R tracks (R per thread, in
// registers) and walks the segments alpha in order:
//
//   * thread 0 stages, three segments ahead, the band of table row alpha that
//     the tile can touch (a rigorous interval bound from the tile's coefficient
//     box) with a 1-D bulk copy (cp.async.bulk) completing on an mbarrier;
//   * all threads turn the staged band into window sums
//         Q[b] = sum_{j=-m..m} P[alpha][b+j]        (FP32, fixed order)
//     in one of two Q buffers, then meet at one CTA barrier per segment;
//   * each thread evaluates x = f T_SFT for its tracks in FP32,
//         y = (x_mid - B) + sum_k c_k D_k,alpha,    b = B + rint(y),
//     (B = rint(x_mid), x_mid an FP64 per-track constant) and adds Q[b] with a
//     single shared load.  Pairs within a warp-uniform error bound g of a
//     half-integer go to the thread's own queue and are recomputed later in
//     the FP64 operation order of the oracle (separately rounded products and
//     sums), so every bin equals the FP64 bin exactly, ties included.
//
// FP32 sums are flushed to a second accumulator every 32 segments; fix-up
// contributions accumulate separately in segment order, so a track's result
// does not depend on its tile neighbours.  Every wait is bounded (2 s); a
// timeout makes the CTA leave together and the call return TFS_ERR_TIMEOUT.
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

constexpr int kThreads = 256;
constexpr int kNP = 3;        // staging slots (copies run up to kNP segments ahead)
constexpr int kQT = 12;       // fix-up queue entries per thread (flushed when fewer than R remain)
constexpr int kSegTile = 32;  // FP32 partial sums are flushed every kSegTile segments

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
  int qcap;  // window centres per Q buffer
  int pcap;  // table elements per staging slot (multiple of 16 bytes)
  // shared-memory carve-up (byte offsets)
  int off_phdr, off_red, off_bnd, off_flags, off_queue, off_acc, off_q, off_p;
};

struct PHdr {
  int plo;   // first staged table bin
  int plen;  // staged elements
  int pad0, pad1;
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

template <int DT, int KP, int R, bool BINS>
__global__ void __launch_bounds__(kThreads, 2) eval_stat_kernel(const EvalArgs a) {
  using S = Store<DT>;
  using T = typename S::T;
  constexpr int EALIGN = 16 / S::esize;  // table elements per 16 bytes
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full_p = reinterpret_cast<uint64_t*>(smem);                // [kNP]
  PHdr* phdr = reinterpret_cast<PHdr*>(smem + a.off_phdr);             // [kNP]
  float* red = reinterpret_cast<float*>(smem + a.off_red);
  float* bnd = reinterpret_cast<float*>(smem + a.off_bnd);
  volatile int* flags = reinterpret_cast<volatile int*>(smem + a.off_flags);  // [0]: abort
  uint32_t* queue = reinterpret_cast<uint32_t*>(smem + a.off_queue);  // [kQT][kThreads]
  float* corr = reinterpret_cast<float*>(smem + a.off_acc);           // [R][kThreads] fix-up sums
  float* tot = corr + R * kThreads;                                   // [R][kThreads] flushed sums
  float* qbuf = reinterpret_cast<float*>(smem + a.off_q);             // [2][qcap]
  unsigned char* pslots = smem + a.off_p;                             // [kNP][pcap * esize + nsp * 4]
  const int pslot_bytes = a.pcap * S::esize + a.nsp * 4;

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const long long tile0 = (long long)blockIdx.x * (kThreads * R);
  const int K = a.K;
  const int m = a.m;
  const int W = 2 * m + 1;
  const int n_seg = a.n_seg;
  constexpr int RW = 2 * KP + 2;

  // ---------------------------------------------------------------- prologue
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
      corr[r * kThreads + tid] = 0.f;
      tot[r * kThreads + tid] = 0.f;
      const long long t = tile0 + tid + r * kThreads;
      if (t < a.N) {
        const double fr = a.f_ref ? a.f_ref[t] : 0.0;
        double f = fr;
        float A = 0.f, Um = fabsf((float)fr);
        const double* cp = a.coeffs + t * (long long)K;
        float cf[KP];
#pragma unroll
        for (int k = 0; k < KP; ++k) {
          const double cd = (k < K) ? cp[k] : 0.0;
          if (k < K) f = fma(cd, a.U[(size_t)k * n_seg + a.alpha_mid], f);
          cf[k] = (float)cd;
          // bounds in FP32, rounded up generously (|fl32(c)| <= |c| (1 + 2^-24))
          A = fmaf(fabsf(cf[k]), a.dmax[k], A);
          Um = fmaf(fabsf(cf[k]), a.umax[k], Um);
        }
        A *= 1.0001f;
        Um *= 1.0001f;
        const double xm = f * a.T;
        // |fp32 estimate - exact x| <= err = 2^-24 ((K+1)/2 + (K+2.001) A) + e64, where
        // e64 = 2^-47 T (|f_ref| + sum_k |c_k| max|U_k|) bounds every FP64 rounding (x_mid, the
        // deltas D, and the oracle's own evaluation).  Pairs closer than g to a half-integer
        // are resolved in FP64; outside that band the exact, the oracle's and this bin
        // coincide and none of them is within the 1e-9 tie band.  (FP32 arithmetic here: the
        // 1.0001 and 1.25 factors cover its rounding.)
        const float e64 = 7.105427357601002e-15f * (float)a.T * Um;
        const float err = 5.9604644775390625e-08f * (0.5f * (K + 1) + (K + 2.001f) * A) + e64;
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
          // every pair of this track goes through the FP64 path: y = 1/2 exactly is never decided
          B[r] = 0;
          y0[r] = 0.5f;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wlim = fminf(wlim, __shfl_xor_sync(0xffffffffu, wlim, o));
    // tile box of the coefficients and of B (for the staged band)
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
#pragma unroll
      for (int k = 0; k < KP; ++k) {
        red[warp * RW + k] = cmn[k];
        red[warp * RW + KP + k] = cmx[k];
      }
      reinterpret_cast<int*>(red)[warp * RW + 2 * KP] = bmin;
      reinterpret_cast<int*>(red)[warp * RW + 2 * KP + 1] = bmax;
    }
  }
  if (tid < 4) flags[tid] = 0;
  if (tid == 0) {
    for (int i = 0; i < kNP; ++i) mbar_init(&full_p[i], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    int bm = 0x7fffffff, bx = -0x7fffffff;
    for (int k = 0; k < KP; ++k) {
      float lo = __int_as_float(0x7f800000), hi = -__int_as_float(0x7f800000);
      for (int w = 0; w < kThreads / 32; ++w) {
        lo = fminf(lo, red[w * RW + k]);
        hi = fmaxf(hi, red[w * RW + KP + k]);
      }
      bnd[k] = lo;
      bnd[KP + k] = hi;
    }
    for (int w = 0; w < kThreads / 32; ++w) {
      bm = min(bm, reinterpret_cast<int*>(red)[w * RW + 2 * KP]);
      bx = max(bx, reinterpret_cast<int*>(red)[w * RW + 2 * KP + 1]);
    }
    reinterpret_cast<int*>(bnd)[2 * KP] = bm;
    reinterpret_cast<int*>(bnd)[2 * KP + 1] = bx;
  }
  __syncthreads();

  // stage the band of segment sg into slot sg % kNP (thread 0 only)
  auto stage = [&](int sg) {
    const int ps = sg % kNP;
    const float* dr = a.segp + (size_t)sg * a.nsp;
    const int bm = reinterpret_cast<const int*>(bnd)[2 * KP];
    const int bx = reinterpret_cast<const int*>(bnd)[2 * KP + 1];
    int blo = 0, blen = 0;
    if (bm <= bx) {
      float lo = 0.f, hi = 0.f, mag = 0.f;
      for (int k = 0; k < KP; ++k) {
        const float d = dr[k];
        const float p1 = bnd[k] * d, p2 = bnd[KP + k] * d;
        lo += fminf(p1, p2);
        hi += fmaxf(p1, p2);
        mag += fmaxf(fabsf(p1), fabsf(p2));
      }
      // FP32 with a margin that covers its rounding: the band only steers staging (bins outside
      // it are read from global memory), so it needs to be generous, not exact
      const float fm = 4.f + 1e-5f * mag + 1e-6f * fmaxf(fabsf((float)bm), fabsf((float)bx));
      const float xl = (float)bm - 0.5f + lo - fm;
      const float xh = (float)bx + 0.5f + hi + fm;
      const float bl = fmaxf(floorf(xl + 0.5f) - 2 * m, 0.f);
      const float bh = fminf(floorf(xh + 0.5f) + 2 * m, (float)(a.n_bin - 1));
      if (bl <= bh) {
        const int il = ((int)bl) & ~(EALIGN - 1);
        int ih = ((int)bh + EALIGN) & ~(EALIGN - 1);
        ih = min(ih, a.row_stride);
        blo = il;
        blen = min(ih - il, a.pcap);
      }
    }
    PHdr h;
    h.plo = blo;
    h.plen = blen;
    h.pad0 = h.pad1 = 0;
    phdr[ps] = h;
    unsigned char* dst = pslots + (size_t)ps * pslot_bytes;
    uint32_t dbytes = (uint32_t)blen * S::esize;
    {
      const long long src_el = (long long)sg * a.row_stride + blo;
      const bool ok =
          dbg_ok(a, (long long)a.off_p + (long long)(ps + 1) * pslot_bytes <= a.smem_bytes, 7, ps, pslot_bytes) &&
          dbg_ok(a, blo >= 0 && src_el + blen <= (long long)a.n_seg * a.row_stride, 8, src_el, blen) &&
          dbg_ok(a, ((a.off_p + (long long)ps * pslot_bytes) & 15) == 0 && (dbytes & 15) == 0 &&
                        ((src_el * S::esize) & 15) == 0, 9, ps, src_el);
      if (!ok) dbytes = 0;
    }
    fence_proxy_async_smem();  // the slot's previous contents were read through the generic proxy
    mbar_arrive_expect_tx(&full_p[ps], dbytes + (uint32_t)a.nsp * 4u);
    if (dbytes > 0)
      bulk_g2s(dst, static_cast<const T*>(a.table) + (size_t)sg * a.row_stride + blo, dbytes, &full_p[ps]);
    bulk_g2s(dst + (size_t)a.pcap * S::esize, dr, (uint32_t)a.nsp * 4u, &full_p[ps]);
  };
  if (tid == 0)
    for (int sg = 0; sg < kNP && sg < n_seg; ++sg) stage(sg);

  // ---------------------------------------------------------------- segments
  int last_waited = -1;
  for (int sg = 0; sg < n_seg; ++sg) {
    const int ps = sg % kNP;
    const bool filled = mbar_wait_bounded(&full_p[ps], (uint32_t)((sg / kNP) & 1), kWaitLimitNs);
    float* q = qbuf + (size_t)(sg & 1) * a.qcap;
    float d[KP];
    int qlo = 0, qn = 0;
    if (filled) {
      last_waited = sg;
      const PHdr h = phdr[ps];
      const unsigned char* src = pslots + (size_t)ps * pslot_bytes;
      const int plo = h.plo, phi = h.plo + h.plen;
      qlo = (plo == 0) ? -m : plo + m;
      const int qhi = (phi >= a.n_bin) ? a.n_bin + m : phi - m;
      qn = h.plen == 0 ? 0 : min(max(0, qhi - qlo), a.qcap);
      // window sums of the staged band, all threads
      const T* pb = reinterpret_cast<const T*>(src);
      const float scale = S::scaled ? a.scales[sg] : 1.f;
      for (int i = tid; i < qn; i += kThreads) {
        const int lo = qlo + i - m;
        float v = 0.f;
        for (int j = 0; j < W; ++j) {
          const int k = lo + j;  // staged when plo <= k < phi
          float p = 0.f;
          if (k >= 0 && k < a.n_bin && dbg_ok(a, k >= plo && k < phi, 11, k, plo)) p = S::ld(pb + (k - plo));
          v += S::scaled ? p * scale : p;
        }
        q[i] = v;
      }
      const float4* dp = reinterpret_cast<const float4*>(src + (size_t)a.pcap * S::esize);
#pragma unroll
      for (int k4 = 0; k4 < (KP + 3) / 4; ++k4) {
        const float4 v = dp[k4];
        if (4 * k4 + 0 < KP) d[4 * k4 + 0] = v.x;
        if (4 * k4 + 1 < KP) d[4 * k4 + 1] = v.y;
        if (4 * k4 + 2 < KP) d[4 * k4 + 2] = v.z;
        if (4 * k4 + 3 < KP) d[4 * k4 + 3] = v.w;
      }
    } else {
      flags[0] = 1;  // the slot never filled: touch none of it; the CTA leaves after the barrier
      atomicExch(a.status, DEV_TIMEOUT);
    }
    __syncthreads();
    if (flags[0]) break;
    // slot ps has been read by every thread: refill it with segment sg + kNP
    if (tid == 0 && sg + kNP < n_seg) stage(sg + kNP);
    if (nq > kQT - R) {
      // not enough queue room for this segment: resolve the queue now, in (segment) order
      for (int i = 0; i < nq; ++i) {
        const uint32_t e = queue[i * kThreads + tid];
        const int r2 = (int)(e & 7u), s2 = (int)(e >> 3);
        corr[r2 * kThreads + tid] += exact_pair<DT, BINS>(a, tile0 + tid + r2 * kThreads, s2);
      }
      nq = 0;
    }
    // pass 1 (straight-line over the R tracks): bins and FP32 decisions
    int bq[R];
    unsigned undecided = 0u, outside = 0u;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float y = y0[r];
#pragma unroll
      for (int k = 0; k < KP; ++k) y = fmaf(c[r][k], d[k], y);
      const float tt = y + 12582912.0f;  // 1.5 * 2^23: rounds y to an integer (|y| < 2^22)
      const float rr = tt - 12582912.0f;
      const float dd = y - rr;
      const int b = B[r] + (__float_as_int(tt) - 0x4B400000);
      bq[r] = b;
      if (!(fabsf(dd) < wlim)) undecided |= 1u << r;
      if ((unsigned)(b - qlo) >= (unsigned)qn) outside |= 1u << r;
    }
    // pass 2 (straight-line): one shared load per track, masked; the address is always in bounds
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const unsigned off = (unsigned)(bq[r] - qlo);
      const float v = q[off < (unsigned)qn ? off : 0u];
      acc[r] += ((undecided | outside) >> r) & 1u ? 0.f : v;
    }
    // pass 3 (rare, warp-uniform branch): queue undecided pairs, read windows outside the Q band
    if (__any_sync(0xffffffffu, (undecided | outside) != 0u)) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int b = bq[r];
        if ((undecided >> r) & 1u) {
          queue[nq * kThreads + tid] = ((uint32_t)sg << 3) | (uint32_t)r;
          ++nq;
        } else if (((outside >> r) & 1u) && b + m >= 0 && b - m < a.n_bin) {
          acc[r] += window_global<DT>(a, sg, b - m, W, S::scaled ? a.scales[sg] : 1.f);
        }
      }
    }
    if (BINS) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int b = bq[r];
        const long long t = tile0 + tid + r * kThreads;
        if (t < a.N && !((undecided >> r) & 1u))
          a.bins_out[t * n_seg + sg] = (b + m < 0) ? (int)0x80000000 : (b - m >= a.n_bin ? 0x7fffffff : b);
      }
    }
    if ((sg % kSegTile) == kSegTile - 1) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        tot[r * kThreads + tid] += acc[r];
        acc[r] = 0.f;
      }
    }
  }
  __syncthreads();
  if (flags[0]) {
    // a bounded wait gave up: drain the bulk copies still in flight into this CTA, then leave
    if (tid == 0) {
      for (int sg = last_waited + 1; sg < n_seg && sg <= last_waited + kNP; ++sg)
        (void)mbar_wait_bounded(&full_p[sg % kNP], (uint32_t)((sg / kNP) & 1), kWaitLimitNs);
    }
    return;
  }
  // remaining fix-ups, in queue (segment) order per thread
  for (int i = 0; i < nq; ++i) {
    const uint32_t e = queue[i * kThreads + tid];
    const int r2 = (int)(e & 7u), s2 = (int)(e >> 3);
    corr[r2 * kThreads + tid] += exact_pair<DT, BINS>(a, tile0 + tid + r2 * kThreads, s2);
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const long long t = tile0 + tid + r * kThreads;
    if (t < a.N) a.stat[t] = (tot[r * kThreads + tid] + acc[r]) + corr[r * kThreads + tid];
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

template <int DT>
int launch_eval_dt(const EvalLaunch& L, const EvalTuning& tune, cudaStream_t st) {
  constexpr int esize = Store<DT>::esize;
  const tfs_table* tb = L.table;
  const SegParams* sp = L.sp;
  const int KP = sp->KP;
  const int R = KP <= 8 ? 8 : (KP <= 16 ? 4 : 2);  // must match the instantiations below
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

  // a Q buffer holds up to qcap window centres; a staging slot the band plus 2m and alignment
  int qcap = tune.cap > 0 ? tune.cap : 2048;
  qcap = std::max(32, std::min(qcap, (int)tb->row_stride + 2 * L.m + 32));
  qcap = (qcap + 31) / 32 * 32;
  int pcap = qcap + 2 * L.m + 32;
  pcap = (pcap + 15) / 16 * 16;
  if (pcap > (int)tb->row_stride) pcap = (int)tb->row_stride;
  a.qcap = qcap;
  a.pcap = pcap;
  const int RW = 2 * KP + 2;
  size_t off = 8 * kNP;
  off = (off + 15) & ~(size_t)15;
  a.off_phdr = (int)off;  off += kNP * sizeof(PHdr);
  a.off_red = (int)off;   off += (size_t)(kThreads / 32) * RW * 4;
  a.off_bnd = (int)off;   off += (size_t)RW * 4;
  off = (off + 15) & ~(size_t)15;
  a.off_flags = (int)off; off += 16;
  a.off_queue = (int)off; off += (size_t)kQT * kThreads * 4;
  a.off_acc = (int)off;   off += (size_t)2 * R * kThreads * 4;
  off = (off + 127) & ~(size_t)127;
  a.off_q = (int)off;     off += (size_t)2 * qcap * 4;
  off = (off + 127) & ~(size_t)127;
  a.off_p = (int)off;     off += (size_t)kNP * ((size_t)pcap * esize + sp->nsp * 4);
  const size_t smem = off;
  a.smem_bytes = (int)smem;

  const long long tile = (long long)kThreads * R;
  const long long gl = (L.N + tile - 1) / tile;
  if (gl > 0x7fffffffLL) {
    set_error("too many tracks for one launch");
    return TFS_ERR_INVALID_ARG;
  }
  const int grid = (int)gl;
  const bool bins = L.bins_out != nullptr;

#define TFS_LAUNCH_KP(KPV, RV)                                                          \
  if (KP == KPV) {                                                                      \
    return bins ? launch_one<DT, KPV, RV, true>(a, grid, smem, st)                      \
                : launch_one<DT, KPV, RV, false>(a, grid, smem, st);                    \
  }
  TFS_LAUNCH_KP(2, 8)
  TFS_LAUNCH_KP(4, 8)
  TFS_LAUNCH_KP(6, 8)
  TFS_LAUNCH_KP(8, 8)
  TFS_LAUNCH_KP(16, 4)
  TFS_LAUNCH_KP(32, 2)
#undef TFS_LAUNCH_KP
  (void)R;
  set_error("unsupported basis size K=%d", L.basis->K);
  return TFS_ERR_INVALID_ARG;
}

}  // namespace tfs
