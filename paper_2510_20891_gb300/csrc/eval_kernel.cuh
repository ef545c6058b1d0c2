// Fused track evaluation + gather + reduction for the semi-coherent statistic
// (paper Sec. II.B Eq. det_stat, nearest-bin reading with +-m neighbours;
// tracks from the SVD basis of Sec. II.C).
//
// One CTA owns a tile of NT*R tracks (R per thread, in registers) and walks
// the segments alpha in order.  For each segment:
//   * the band of bins its tracks can touch (a rigorous interval bound from
//     the tile's coefficient box) is staged from the table into a shared
//     memory ring slot by a 1-D bulk copy (cp.async.bulk) completing on an
//     mbarrier, together with the segment's FP32 basis deltas;
//   * each thread evaluates x = f T_SFT for its tracks in FP32,
//        y = (x_mid - B) + sum_k c_k D_k,alpha,  b = B + rint(y),
//     where B = rint(x_mid) and x_mid are FP64 per-track constants.  A
//     per-track error bound g decides whether rint(y) is certainly the FP64
//     bin; pairs with |y - rint(y)| >= 1/2 - g are queued;
//   * after a CTA barrier, queued pairs are recomputed with the oracle's
//     FP64 operation order (separately rounded products and sums) and their
//     window sums are added to a per-track correction in shared memory;
//   * the +-m window is summed from the staged band (or, outside it, from
//     global memory) and accumulated in FP32, flushed every 32 segments.
// The bins therefore equal the FP64 bins exactly, ties included.
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
  int* bins_out;  // [N][n_seg] or null; INT_MIN / INT_MAX mark windows wholly below / above the table
  unsigned long long* dbg;  // self-check record (builds with TFS_DEBUG_CHECKS only), else unused
  int smem_bytes;
  // launch shape
  int nst, cap, padl, slot_elems, qcap;
  // shared-memory carve-up (byte offsets)
  int off_hdr, off_segp, off_red, off_bnd, off_qcnt, off_qent, off_corr, off_data, slot_bytes;
};

struct SlotHdr {
  int blo;    // first staged bin (aligned), data begins at slot index padl
  int vlo;    // lowest bin whose window start may be read from the slot
  int span1;  // window starts lo with 0 <= lo - vlo < span1 are fully inside the slot
  int pad;
};

constexpr int kSegTile = 32;  // FP32 partial sums are flushed every kSegTile segments

// Self-checks of every shared and global index (compiled in with TFS_DEBUG_CHECKS): a failing
// check records (site, two values) once and the caller skips the access.
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

template <int DT>
__device__ __forceinline__ float window_global(const EvalArgs& a, int seg, int lo, int W) {
  using S = Store<DT>;
  const typename S::T* row = static_cast<const typename S::T*>(a.table) + (size_t)seg * a.row_stride;
  float v = 0.f;
  for (int j = 0; j < W; ++j) {
    const int k = lo + j;
    if (k >= 0 && k < a.n_bin) v += S::ld(row + k);
  }
  return v;
}

template <int DT, int WT>
__device__ __forceinline__ float window_smem(const typename Store<DT>::T* p, int W) {
  using S = Store<DT>;
  float v = 0.f;
  if (WT > 0) {
#pragma unroll
    for (int j = 0; j < WT; ++j) v += S::ld(p + j);
  } else {
    for (int j = 0; j < W; ++j) v += S::ld(p + j);
  }
  return v;
}

// FP64 bin of (track t, segment seg) in the oracle's operation order, and its window sum.
template <int DT, int WT>
__device__ float exact_pair(const EvalArgs& a, long long t, int seg, const typename Store<DT>::T* slot,
                            const SlotHdr& h, float scale, bool* tie) {
  if (!dbg_ok(a, t >= 0 && t < a.N && seg >= 0 && seg < a.n_seg, 1, t, seg)) {
    *tie = false;
    return 0.f;
  }
  double f = a.f_ref ? a.f_ref[t] : 0.0;
  const double* c = a.coeffs + t * (long long)a.K;
  for (int k = 0; k < a.K; ++k) f = __dadd_rn(f, __dmul_rn(c[k], a.U[(size_t)k * a.n_seg + seg]));
  const double x = __dmul_rn(f, a.T);
  *tie = false;
  int* bo = a.bins_out ? a.bins_out + t * (long long)a.n_seg + seg : nullptr;
  if (!isfinite(x)) {
    if (bo) *bo = 0x7fffffff;
    return 0.f;
  }
  const double fl = floor(x);
  *tie = fabs(__dsub_rn(__dsub_rn(x, fl), 0.5)) <= 1e-9;
  const double z = __dadd_rn(x, 0.5);
  const int m = a.m;
  if (z < -(double)m || z >= (double)a.n_bin + (double)m) {
    if (bo) *bo = z < 0.0 ? (int)0x80000000 : 0x7fffffff;
    return 0.f;
  }
  const int b = (int)floor(z);
  if (bo) *bo = b;
  const int lo = b - m;
  const int W = 2 * m + 1;
  float v = 0.f;
  if ((unsigned)(lo - h.vlo) < (unsigned)h.span1) {
    const int ix = a.padl + (lo - h.blo);
    if (dbg_ok(a, ix >= 0 && ix + W <= a.slot_elems, 3, ix, lo)) v = window_smem<DT, WT>(slot + ix, W);
  } else {
    v = window_global<DT>(a, seg, lo, W);
  }
  return Store<DT>::scaled ? v * scale : v;
}

__device__ __forceinline__ void report_tie(const EvalArgs& a, long long t, int seg) {
  const unsigned long long i = atomicAdd(a.tie_count, 1ull);
  if (i < (unsigned long long)a.tie_cap) {
    a.tie_track[i] = t;
    a.tie_seg[i] = seg;
  }
}

template <int DT, int KP, int R, int WT, int NT>
__global__ void __launch_bounds__(NT) eval_stat_kernel(const EvalArgs a) {
  using S = Store<DT>;
  using T = typename S::T;
  constexpr int EALIGN = 16 / S::esize;  // elements per 16 bytes
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem);
  SlotHdr* hdr = reinterpret_cast<SlotHdr*>(smem + a.off_hdr);
  float* sseg = reinterpret_cast<float*>(smem + a.off_segp);
  float* red = reinterpret_cast<float*>(smem + a.off_red);
  float* bnd = reinterpret_cast<float*>(smem + a.off_bnd);  // [2*KP] cmin,cmax then (int) Bmin,Bmax, abort
  int* qcnt = reinterpret_cast<int*>(smem + a.off_qcnt);    // [4]: 3 queue counters + abort flag
  uint16_t* qent = reinterpret_cast<uint16_t*>(smem + a.off_qent);
  float* corr = reinterpret_cast<float*>(smem + a.off_corr);
  unsigned char* sdata = smem + a.off_data;

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const long long tile0 = (long long)blockIdx.x * (NT * R);
  const int K = a.K;
  const int m = WT > 0 ? (WT - 1) / 2 : a.m;
  const int W = 2 * m + 1;
  const int n_seg = a.n_seg;

  // ---------------------------------------------------------------- prologue
  float c[R][KP];
  int B[R];
  float y0[R], lim[R], acc[R], acct[R];
  float cmn[KP], cmx[KP];
  int bmin = 0x7fffffff, bmax = -0x7fffffff;
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    cmn[k] = __int_as_float(0x7f800000);
    cmx[k] = -__int_as_float(0x7f800000);
  }
  const double mid_T = a.T;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    acc[r] = 0.f;
    acct[r] = 0.f;
    const long long t = tile0 + tid + r * NT;
    corr[tid + r * NT] = 0.f;
#pragma unroll
    for (int k = 0; k < KP; ++k) c[r][k] = 0.f;
    if (t < a.N) {
      const double fr = a.f_ref ? a.f_ref[t] : 0.0;
      double f = fr, A = 0.0, Um = fabs(fr);
      const double* cp = a.coeffs + t * (long long)K;
      double cd[KP];
#pragma unroll
      for (int k = 0; k < KP; ++k) {
        cd[k] = (k < K) ? cp[k] : 0.0;
        if (k < K) f = fma(cd[k], a.U[(size_t)k * n_seg + a.alpha_mid], f);
        A = fma(fabs(cd[k]), (double)a.dmax[k], A);
        Um = fma(fabs(cd[k]), (double)a.umax[k], Um);
      }
      const double xm = f * mid_T;
      // |fp32 estimate - exact x| <= err = 2^-24 ((K+1)/2 + (K+2.001) A) + e64, where
      // e64 = 2^-47 T (|f_ref| + sum_k |c_k| max|U_k|) bounds every FP64 rounding (x_mid, the
      // deltas D, and the oracle's own evaluation).  Pairs closer than g to a half-integer are
      // resolved in FP64; outside that band the exact, the oracle's and this bin coincide and
      // none of them is within the 1e-9 tie band.
      const double e64 = 7.105427357601002e-15 * mid_T * Um;
      const double err = 5.9604644775390625e-08 * (0.5 * (K + 1) + (K + 2.001) * A) + e64;
      const double g = 1.25 * (err + e64) + 4e-9;
      const bool exact = !(fabs(xm) < 1073741824.0) || !(g < 0.25) || !(A < 1048576.0);
      if (!exact) {
        const double Bd = rint(xm);
        B[r] = (int)Bd;
        y0[r] = (float)(xm - Bd);
        lim[r] = __double2float_rd(0.5 - g);
#pragma unroll
        for (int k = 0; k < KP; ++k) {
          c[r][k] = (float)cd[k];
          cmn[k] = fminf(cmn[k], c[r][k]);
          cmx[k] = fmaxf(cmx[k], c[r][k]);
        }
        bmin = min(bmin, B[r]);
        bmax = max(bmax, B[r]);
      } else {
        B[r] = 0;
        y0[r] = 0.f;
        lim[r] = -1.f;  // every pair goes through the FP64 path
      }
    } else {
      B[r] = -(1 << 29);  // inactive slot: always out of range, never queued
      y0[r] = 0.f;
      lim[r] = 2.f;
    }
  }
  // tile bounds of the coefficients and of B (for the staged band)
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
  const int RW = 2 * KP + 2;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      red[warp * RW + k] = cmn[k];
      red[warp * RW + KP + k] = cmx[k];
    }
    reinterpret_cast<int*>(red)[warp * RW + 2 * KP] = bmin;
    reinterpret_cast<int*>(red)[warp * RW + 2 * KP + 1] = bmax;
  }
  if (tid < 8) qcnt[tid] = 0;  // 3 queue counters, the abort flag, two per-parity timeout flags
  // zero the left pads of every slot (they stand for bins < 0 when a band starts at bin 0)
  for (int s = 0; s < a.nst; ++s) {
    T* sd = reinterpret_cast<T*>(sdata + (size_t)s * a.slot_bytes);
    for (int i = tid; i < a.padl; i += NT) sd[i] = T(0.f);
  }
  if (tid == 0) {
    for (int s = 0; s < a.nst; ++s) mbar_init(&mbar[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    int bm = 0x7fffffff, bx = -0x7fffffff;
    for (int k = 0; k < KP; ++k) {
      float lo = __int_as_float(0x7f800000), hi = -__int_as_float(0x7f800000);
      for (int w = 0; w < NT / 32; ++w) {
        lo = fminf(lo, red[w * RW + k]);
        hi = fmaxf(hi, red[w * RW + KP + k]);
      }
      bnd[k] = lo;
      bnd[KP + k] = hi;
    }
    for (int w = 0; w < NT / 32; ++w) {
      bm = min(bm, reinterpret_cast<int*>(red)[w * RW + 2 * KP]);
      bx = max(bx, reinterpret_cast<int*>(red)[w * RW + 2 * KP + 1]);
    }
    reinterpret_cast<int*>(bnd)[2 * KP] = bm;
    reinterpret_cast<int*>(bnd)[2 * KP + 1] = bx;
  }
  __syncthreads();

  // producer: stage the band of segment `sg` into slot `s` (thread 0 only)
  auto issue = [&](int sg, int s) {
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
      const double margin = 4.0 + 1e-5 * (double)mag;
      const double xl = (double)bm - 0.5 + (double)lo - margin;
      const double xh = (double)bx + 0.5 + (double)hi + margin;
      double bl = floor(xl + 0.5) - m, bh = floor(xh + 0.5) + m;
      bl = fmax(bl, 0.0);
      bh = fmin(bh, (double)(a.n_bin - 1));
      if (bl <= bh) {
        const int il = ((int)bl) & ~(EALIGN - 1);
        int ih = ((int)bh + EALIGN) & ~(EALIGN - 1);
        ih = min(ih, a.row_stride);
        blo = il;
        blen = min(ih - il, a.cap);
      }
    }
    const int vlo = (blo == 0) ? -a.padl : blo;
    const int vhi = blo + blen;
    SlotHdr h;
    h.blo = blo;
    h.vlo = vlo;
    h.span1 = max(0, vhi - vlo - W + 1);
    h.pad = 0;
    hdr[s] = h;
    uint32_t dbytes = (uint32_t)blen * S::esize;
    {
      const long long dst_off = (long long)a.off_data + (long long)s * a.slot_bytes + (long long)a.padl * S::esize;
      const long long src_el = (long long)sg * a.row_stride + blo;
      const bool ok = dbg_ok(a, s >= 0 && s < a.nst && dst_off + dbytes <= a.smem_bytes, 7, dst_off, dbytes) &&
                      dbg_ok(a, blo >= 0 && src_el + blen <= (long long)a.n_seg * a.row_stride, 8, src_el, blen) &&
                      dbg_ok(a, ((dst_off | (long long)dbytes | (src_el * S::esize)) & 15) == 0, 9, dst_off, src_el) &&
                      dbg_ok(a, (long long)a.off_segp + (long long)(s + 1) * a.nsp * 4 <= a.off_red, 10, s, a.nsp);
      if (!ok) dbytes = 0;
    }
    mbar_arrive_expect_tx(&mbar[s], dbytes + (uint32_t)a.nsp * 4u);
    if (dbytes > 0)
      bulk_g2s(sdata + (size_t)s * a.slot_bytes + (size_t)a.padl * S::esize,
               static_cast<const T*>(a.table) + (size_t)sg * a.row_stride + blo, dbytes, &mbar[s]);
    bulk_g2s(sseg + (size_t)s * a.nsp, dr, (uint32_t)a.nsp * 4u, &mbar[s]);
  };

  if (tid == 0) {
    for (int sg = 0; sg < a.nst && sg < n_seg; ++sg) issue(sg, sg);
  }

  // ---------------------------------------------------------------- segments
  int last_waited = -1;
  for (int sg = 0; sg < n_seg; ++sg) {
    const int s = sg % a.nst;
    const bool filled = mbar_wait_bounded(&mbar[s], (uint32_t)((sg / a.nst) & 1), kWaitLimitNs);
    if (!filled) {
      // the slot never filled: touch none of it; the CTA leaves together after the barrier below
      qcnt[4 + (sg & 1)] = 1;  // per-parity flag: a thread already in the next segment cannot flip this one
      atomicExch(a.status, DEV_TIMEOUT);
    } else {
      last_waited = sg;
    }
    SlotHdr h = {0, 0, 0, 0};
    if (filled) h = hdr[s];
    const T* slot = reinterpret_cast<const T*>(sdata + (size_t)s * a.slot_bytes);
    float d[KP];
    {
      const float4* dp = reinterpret_cast<const float4*>(sseg + (size_t)s * a.nsp);
#pragma unroll
      for (int k4 = 0; k4 < (KP + 3) / 4; ++k4) {
        const float4 v = dp[k4];
        if (4 * k4 + 0 < KP) d[4 * k4 + 0] = v.x;
        if (4 * k4 + 1 < KP) d[4 * k4 + 1] = v.y;
        if (4 * k4 + 2 < KP) d[4 * k4 + 2] = v.z;
        if (4 * k4 + 3 < KP) d[4 * k4 + 3] = v.w;
      }
    }
    const float scale = S::scaled ? __ldg(a.scales + sg) : 1.f;
    const int q = sg % 3;
    if (filled) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float y = y0[r];
#pragma unroll
      for (int k = 0; k < KP; ++k) y = fmaf(c[r][k], d[k], y);
      const float tt = y + 12582912.0f;  // 1.5 * 2^23: rounds y to an integer (|y| < 2^22)
      const float rr = tt - 12582912.0f;
      const float dd = y - rr;
      const int b = B[r] + (__float_as_int(tt) - 0x4B400000);
      if (!(fabsf(dd) < lim[r])) {
        const int pos = atomicAdd(&qcnt[q], 1);
        if (pos < a.qcap) {
          qent[q * a.qcap + pos] = (uint16_t)(tid + r * NT);
        } else {
          bool tie;
          const long long t = tile0 + tid + r * NT;
          acc[r] += exact_pair<DT, WT>(a, t, sg, slot, h, scale, &tie);
          if (tie) report_tie(a, t, sg);
        }
        continue;
      }
      const int lo = b - m;
      float v = 0.f;
      if ((unsigned)(lo - h.vlo) < (unsigned)h.span1) {
        const int ix = a.padl + (lo - h.blo);
        if (dbg_ok(a, ix >= 0 && ix + W <= a.slot_elems, 5, ix, lo)) v = window_smem<DT, WT>(slot + ix, W);
      } else if (b + m < 0 || lo >= a.n_bin)
        v = 0.f;
      else
        v = window_global<DT>(a, sg, lo, W);
      acc[r] += S::scaled ? v * scale : v;
      if (a.bins_out) {
        const long long t = tile0 + tid + r * NT;
        if (t < a.N)
          a.bins_out[t * n_seg + sg] = (b + m < 0) ? (int)0x80000000 : (lo >= a.n_bin ? 0x7fffffff : b);
      }
    }
    }  // filled
    if ((sg % kSegTile) == kSegTile - 1) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        acct[r] += acc[r];
        acc[r] = 0.f;
      }
    }
    __syncthreads();
    if (qcnt[4 + (sg & 1)]) {  // a bounded wait gave up somewhere in the CTA (uniform after the barrier)
      qcnt[3] = 1;
      break;
    }
    if (tid == 0) {
      qcnt[(sg + 2) % 3] = 0;  // that queue was drained before this barrier
      const int nx = sg - 1 + a.nst;
      if (sg >= 1 && nx < n_seg) issue(nx, (sg - 1) % a.nst);
    }
    // resolve the queued pairs of this segment in FP64
    const int cnt = min(qcnt[q], a.qcap);
    for (int i = tid; i < cnt; i += NT) {
      const int lt = qent[q * a.qcap + i];
      if (!dbg_ok(a, lt < NT * R, 6, lt, i)) continue;
      const long long t = tile0 + lt;
      bool tie;
      corr[lt] += exact_pair<DT, WT>(a, t, sg, slot, h, scale, &tie);
      if (tie) report_tie(a, t, sg);
    }
  }
  __syncthreads();
  if (qcnt[3]) {
    // drain copies still in flight into this CTA's shared memory before exiting
    if (tid == 0) {
      for (int sg = last_waited + 1; sg < n_seg && sg <= last_waited + a.nst; ++sg)
        (void)mbar_wait_bounded(&mbar[sg % a.nst], (uint32_t)((sg / a.nst) & 1), kWaitLimitNs);
    }
    return;
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const long long t = tile0 + tid + r * NT;
    if (t < a.N) a.stat[t] = (acct[r] + acc[r]) + corr[tid + r * NT];
  }
}

// ---------------------------------------------------------------- host side
template <int DT, int KP, int R, int WT, int NT>
int launch_one(const EvalArgs& a0, int grid, size_t smem, cudaStream_t st) {
  auto kern = eval_stat_kernel<DT, KP, R, WT, NT>;
  static int configured = -1;
  if (configured < (int)smem) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(eval)");
    configured = (int)smem;
  }
  kern<<<grid, NT, smem, st>>>(a0);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "eval_stat_kernel launch");
  return TFS_OK;
}

template <int DT>
int launch_eval_dt(const EvalLaunch& L, const EvalTuning& tune, cudaStream_t st) {
  constexpr int NT = 256;
  constexpr int esize = Store<DT>::esize;
  constexpr int EALIGN = 16 / esize;
  const tfs_table* tb = L.table;
  const SegParams* sp = L.sp;
  const int KP = sp->KP;
  const int R = KP <= 8 ? 8 : 4;
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

  const int W = 2 * L.m + 1;
  a.nst = tune.stages > 0 ? tune.stages : 3;
  if (a.nst < 2) a.nst = 2;
  if (a.nst > 4) a.nst = 4;
  a.qcap = tune.qcap > 0 ? tune.qcap : 256;
  a.padl = ((W + EALIGN - 1) / EALIGN) * EALIGN;
  // staged band capacity: whole row when it fits the budget, else what fits
  const int budget = 88 * 1024;
  int cap = tune.cap > 0 ? tune.cap : (int)tb->row_stride;
  const int per_slot_max = budget / a.nst - 2 * a.padl * esize;
  if (cap * esize > per_slot_max) cap = per_slot_max / esize;
  cap = (cap / 32) * 32;
  if (cap < 32) cap = 32;
  if (cap > (int)tb->row_stride) cap = (int)tb->row_stride;
  a.cap = cap;
  a.slot_elems = a.padl + cap + a.padl;
  a.slot_bytes = ((a.slot_elems * esize + 127) / 128) * 128;

  const int RW = 2 * KP + 2;
  size_t off = 64;                                   // 4 mbarriers (8 B each) fit in the first 64 bytes
  a.off_hdr = (int)off;  off += 4 * sizeof(SlotHdr);
  a.off_segp = (int)off; off += (size_t)4 * sp->nsp * 4;
  off = (off + 15) & ~(size_t)15;
  a.off_red = (int)off;  off += (size_t)(NT / 32) * RW * 4;
  a.off_bnd = (int)off;  off += (size_t)RW * 4;
  off = (off + 15) & ~(size_t)15;
  a.off_qcnt = (int)off; off += 32;
  a.off_qent = (int)off; off += (size_t)3 * a.qcap * 2;
  off = (off + 15) & ~(size_t)15;
  a.off_corr = (int)off; off += (size_t)NT * R * 4;
  off = (off + 127) & ~(size_t)127;
  a.off_data = (int)off; off += (size_t)a.nst * a.slot_bytes;
  const size_t smem = off;
  a.smem_bytes = (int)smem;

  const long long tile = (long long)NT * R;
  const long long gl = (L.N + tile - 1) / tile;
  if (gl > 0x7fffffffLL) {
    set_error("too many tracks for one launch");
    return TFS_ERR_INVALID_ARG;
  }
  const int grid = (int)gl;
  const int wt = (L.m == 0) ? 1 : (L.m == 1 ? 3 : 0);

#define TFS_LAUNCH_KP(KPV, RV)                                                        \
  if (KP == KPV) {                                                                    \
    if (wt == 1) return launch_one<DT, KPV, RV, 1, NT>(a, grid, smem, st);            \
    if (wt == 3) return launch_one<DT, KPV, RV, 3, NT>(a, grid, smem, st);            \
    return launch_one<DT, KPV, RV, 0, NT>(a, grid, smem, st);                         \
  }
  TFS_LAUNCH_KP(2, 8)
  TFS_LAUNCH_KP(4, 8)
  TFS_LAUNCH_KP(6, 8)
  TFS_LAUNCH_KP(8, 8)
  TFS_LAUNCH_KP(16, 4)
  TFS_LAUNCH_KP(32, 4)
#undef TFS_LAUNCH_KP
  (void)R;
  set_error("unsupported basis size K=%d", L.basis->K);
  return TFS_ERR_INVALID_ARG;
}

}  // namespace tfs
