// The paper's linear-chirp statistic (Sec. II.B, Eq. det_stat with the chirping local template).
//
// For every (track, segment) pair the local waveform is the linear chirp
// exp(i [2 pi f (t - t_a) + pi fdot (t - t_a)^2]) with f the track's frequency at the segment
// midpoint t_a and fdot its finite difference; S_alpha is |sum_k d~*_k h~_k / S_k|^2 over
// sum_k |h~_k|^2 / S_k on the 2P + 1 bins around the nearest bin b, times 4 / (dt sum w^2).
//
// GB300 layout: one warp per track at a time.  The track's frequency, derivatives and bin
// are evaluated in FP64 in the oracle's operation order, 32 segments at a time with one
// segment per lane (GB300's FP64 rate is a small fraction of FP32), so b is bit-identical.
// The template is the Fourier integral of the Hann-windowed chirp over the segment, sampled
// at 256 points and transformed by a 256-point FFT on each half of the warp (16 samples per
// lane, a lane-local 16-point DFT, twiddles, a transpose through shared memory and a second
// lane-local 16-point DFT), so that the two halves take two segments of the track at once
// (the segments the exclusions keep, packed in pairs).  With the Hann window the sampled
// transform equals the sampled SFT of the template within aliasing of order
// 1 / (2 pi (256 - P - beta / 2)^3) of its peak.  The scaled complex table (L2-resident)
// supplies the data bins; sums in FP32, S_alpha summed over segments in FP64 (each half its
// own segments, the two sums added at the end).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "tfs_internal.cuh"

namespace tfs {
namespace {

constexpr int kM = 256;           // template samples per segment
constexpr int kCW = 8;            // warps per block
constexpr int kCThreads = 32 * kCW;
constexpr int kChirpPMax = 111;   // the outputs kept cover -112 <= j <= 111
constexpr double kFLow = 0x1.4b96be9c2da2cp-12;  // 10^-3.5 Hz, the nearest double

constexpr int kChirpMaxJobs = 64;  // jobs per launch

struct ChirpJob {
  const float2* z;      // [n_seg][n_bin]
  const float* wt;      // [n_bin]
  int n_seg, n_bin;
  const double* U;      // [K][n_seg]
  int K;
  const double* coeffs; // [N][K]
  const double* f_ref;  // [N] or null
  long long N;
  double T;
  int P, cuts;
  float* stat;          // [N]
};

struct ChirpBatch {
  ChirpJob jobs[kChirpMaxJobs];
  long long start[kChirpMaxJobs + 1];  // first track of each job in the launch's numbering
  int n_jobs;
};

__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 c_mi(float2 a) { return make_float2(a.y, -a.x); }  // times -i

// e^{-2 pi i e / 16} and e^{-2 pi i k / 32}
__device__ __forceinline__ float2 w16(int e) {
  switch (e & 15) {
    case 0: return make_float2(1.f, 0.f);
    case 1: return make_float2(0.9238795325112867f, -0.3826834323650898f);
    case 2: return make_float2(0.7071067811865476f, -0.7071067811865475f);
    case 3: return make_float2(0.38268343236508984f, -0.9238795325112867f);
    case 4: return make_float2(0.f, -1.f);
    case 6: return make_float2(-0.7071067811865475f, -0.7071067811865476f);
    case 9: return make_float2(-0.9238795325112868f, 0.38268343236508967f);
    default: return make_float2(0.f, 0.f);  // not used by dft16
  }
}
__device__ __forceinline__ float2 w32(int k) {
  switch (k) {
    case 0: return make_float2(1.f, 0.f);
    case 1: return make_float2(0.9807852804032304f, -0.19509032201612825f);
    case 2: return make_float2(0.9238795325112867f, -0.3826834323650898f);
    case 3: return make_float2(0.8314696123025452f, -0.5555702330196022f);
    case 4: return make_float2(0.7071067811865476f, -0.7071067811865475f);
    case 5: return make_float2(0.5555702330196023f, -0.8314696123025452f);
    case 6: return make_float2(0.38268343236508984f, -0.9238795325112867f);
    case 9: return make_float2(-0.1950903220161282f, -0.9807852804032304f);
    case 10: return make_float2(-0.3826834323650897f, -0.9238795325112867f);
    case 11: return make_float2(-0.555570233019602f, -0.8314696123025455f);
    case 12: return make_float2(-0.7071067811865475f, -0.7071067811865476f);
    case 13: return make_float2(-0.8314696123025453f, -0.5555702330196022f);
    case 14: return make_float2(-0.9238795325112867f, -0.3826834323650899f);
    case 15: return make_float2(-0.9807852804032304f, -0.1950903220161286f);
    default: return make_float2(0.f, 0.f);  // 7, 8: not used by the exchange
  }
}

// 4-point DFT in place (W4 = -i).
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  const float2 a = c_add(x0, x2), b = c_sub(x0, x2), c = c_add(x1, x3), d = c_mi(c_sub(x1, x3));
  x0 = c_add(a, c);
  x2 = c_sub(a, c);
  x1 = c_add(b, d);
  x3 = c_sub(b, d);
}

// 16-point DFT X[k] = sum_n v[n] W16^{nk} by 4 x 4 (n = 4 n1 + n2, k = k1 + 4 k2);
// X[k1 + 4 k2] ends in v[4 k1 + k2] (read it through at16).
__device__ __forceinline__ void dft16(float2 (&v)[16]) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
#pragma unroll
  for (int k1 = 1; k1 < 4; ++k1)
#pragma unroll
    for (int n2 = 1; n2 < 4; ++n2) v[4 * k1 + n2] = c_mul(v[4 * k1 + n2], w16(n2 * k1));
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
}
__device__ __forceinline__ int at16(int k) { return 4 * (k & 3) + (k >> 2); }

__device__ __forceinline__ double track_f(const ChirpJob& a, const double* c, double fr, int seg) {
  double f = fr;
  for (int k = 0; k < a.K; ++k) f = __dadd_rn(f, __dmul_rn(c[k], a.U[(size_t)k * a.n_seg + seg]));
  return f;
}

__global__ void __launch_bounds__(kCThreads, 2) chirp_stat_kernel(const __grid_constant__ ChirpBatch B) {
  __shared__ __align__(16) float2 s_buf[kCW][2][16][18];  // per half-warp transpose (rows padded to 16 B)
  __shared__ double s_c[kCW][32];             // the warp's track coefficients
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int hf = lane >> 4, l16 = lane & 15;  // half of the warp, lane within it
  // the window at this lane's samples m = l16 + 16 i (held in registers: read from shared memory
  // they cost 48 wavefronts per pair, half of them bank conflicts), and y at i = 0, exact
  float wreg[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const float s = sinpif((float)(l16 + 16 * i) / (float)kM);
    wreg[i] = s * s;
  }
  const float y0 = (float)(l16 - kM / 2) * (1.f / kM);
  // e^{-2 pi i l16 j0 / 256}, j0 = 1..15 (exact arguments; j0 = 0 is 1)
  float2 tw[16];
  tw[0] = make_float2(1.f, 0.f);
#pragma unroll
  for (int j0 = 1; j0 < 16; ++j0) {
    float sn, cs;
    sincospif(-(float)(2 * l16 * j0) / (float)kM, &sn, &cs);
    tw[j0] = make_float2(cs, sn);
  }
  __syncthreads();
  const long long nw = (long long)gridDim.x * kCW;
  int jb = 0;  // the job of the current track (tracks are visited in increasing order)
  for (long long gt = (long long)blockIdx.x * kCW + w; gt < B.start[B.n_jobs]; gt += nw) {
    while (gt >= B.start[jb + 1]) ++jb;
    const ChirpJob a = B.jobs[jb];  // by value: the inner loops read registers, not indexed parameters
    const long long t = gt - B.start[jb];
    const int n = a.n_seg;
    const double T = a.T;
    const double T6 = __ddiv_rn(T, 6.0);
    const double invT = 1.0 / T;
    __syncwarp();
    if (lane < a.K) s_c[w][lane] = a.coeffs[t * a.K + lane];
    __syncwarp();
    const double* c = s_c[w];
    const double fr = a.f_ref ? a.f_ref[t] : 0.0;
    // outputs j1 of this lane (j = l16 + 16 j1, less 256 from j1 = 9) with |j| <= P
    unsigned pmask = 0u;
#pragma unroll
    for (int j1 = 0; j1 < 16; ++j1) {
      const int jj = l16 + 16 * j1 - (j1 >= 9 ? kM : 0);
      if (j1 != 7 && j1 != 8 && jj >= -a.P && jj <= a.P) pmask |= 1u << j1;
    }
    double sacc = 0.0;  // this half's segments
    for (int al0 = 0; al0 < n; al0 += 32) {
      // lane s prepares segment al0 + s in FP64, in the oracle's operation order: its frequency
      // and neighbours, fdot by finite differences (one-sided at the ends), the bin, the cuts,
      // and the FP32 phase parameters; the halves then take the kept segments two at a time
      const int sg = al0 + lane;
      bool p_skip = true;
      int p_b = 0;
      float p_d2 = 0.f, p_bh = 0.f, p_bl = 0.f;
      // each lane its segment's frequency, the neighbours' from the adjacent lanes (the edge
      // lanes evaluate theirs): the same FP64 operations whichever lane does them
      const double F0 = sg < n ? track_f(a, c, fr, sg) : 0.0;
      double Fm = __shfl_up_sync(0xffffffffu, F0, 1);
      double Fp = __shfl_down_sync(0xffffffffu, F0, 1);
      if (lane == 0) Fm = (sg > 0 && sg < n) ? track_f(a, c, fr, sg - 1) : 0.0;
      if (lane == 31) Fp = sg + 1 < n ? track_f(a, c, fr, sg + 1) : 0.0;
      if (sg < n) {
        double fd = 0.0;
        if (n >= 2) {
          const double dF = sg == 0 ? __dsub_rn(Fp, F0) : (sg == n - 1 ? __dsub_rn(F0, Fm) : __dsub_rn(Fp, Fm));
          if (a.cuts) {
            // the exclusion compares fdot with its threshold: the oracle's division, exactly
            fd = (sg == 0 || sg == n - 1) ? __ddiv_rn(dF, T) : __ddiv_rn(dF, __dmul_rn(2.0, T));
          } else {
            fd = dF * ((sg == 0 || sg == n - 1) ? invT : 0.5 * invT);  // only the template's beta
          }
        }
        const double x = __dmul_rn(F0, T);
        const double bz = floor(__dadd_rn(x, 0.5));
        // the track's own bin must lie in the table (else only far template tails would remain)
        bool skip = !isfinite(x) || bz < 0.0 || bz >= (double)a.n_bin;
        if (a.cuts && !skip) {
          double z = 0.0;
          if (n >= 3) {
            double fa, fb, fc;  // F at c + 1, c, c - 1 with c the nearest inner segment
            if (sg == 0) {
              fa = track_f(a, c, fr, 2);
              fb = Fp;
              fc = F0;
            } else if (sg == n - 1) {
              fa = F0;
              fb = Fm;
              fc = track_f(a, c, fr, n - 3);
            } else {
              fa = Fp;
              fb = F0;
              fc = Fm;
            }
            z = __dmul_rn(__dadd_rn(__dsub_rn(fa, __dmul_rn(2.0, fb)), fc), T6);
          }
          skip = z > 1.0 || F0 < kFLow || fd < 1e-13;
        }
        if (!skip) {
          p_b = (int)bz;
          p_d2 = (float)(2.0 * __dsub_rn(x, bz));  // 2 delta0, delta0 in [-1/2, 1/2]
          // beta = fdot T^2 split so that beta_hi * y^2 is exact in FP32 (7 + 14 significant bits)
          const double beta = fd * T * T;
          double bh64 = 0.0;
          if (beta != 0.0 && isfinite(beta)) {
            int e;
            frexp(beta, &e);
            bh64 = ldexp(rint(ldexp(beta, 7 - e)), e - 7);
          }
          p_bh = (float)bh64;
          p_bl = (float)(beta - bh64);
        }
        p_skip = skip;
      }
      unsigned todo = __ballot_sync(0xffffffffu, !p_skip);  // the kept segments (warp-uniform)
      while (todo) {
        const int s0 = __ffs(todo) - 1;
        todo &= todo - 1;
        const int s1 = todo ? __ffs(todo) - 1 : -1;
        if (s1 >= 0) todo &= todo - 1;
        // half 0 takes segment s0, half 1 segment s1 (or repeats s0 without counting it)
        const bool live = hf == 0 || s1 >= 0;
        const int src = (hf && s1 >= 0) ? s1 : s0;
        const int al = al0 + src;
        const int b = __shfl_sync(0xffffffffu, p_b, src);
        const float d2 = __shfl_sync(0xffffffffu, p_d2, src);
        const float bh = __shfl_sync(0xffffffffu, p_bh, src);
        const float bl = __shfl_sync(0xffffffffu, p_bl, src);
        // samples m = l16 + 16 i of g(y) = w(y) e^{i pi (2 delta0 y + beta y^2)}, y = m / 256 - 1/2,
        // with the hardware sine and cosine on [-pi, pi] (absolute error about 2^-21.4: far below
        // the FP32 rounding of the template's sums)
        float2 v[16];
        const float bs = bh + bl;
        // the phases first (in v[i].x, radians in [-pi, pi]), then sine and cosine
        if (__all_sync(0xffffffffu, fabsf(bs) <= 2.f)) {
          // |beta| <= 2: pi (2 delta0 y + beta y^2) lies in [-pi, pi] as it is
          const float bsp = 3.14159265358979f * bs, d2p = 3.14159265358979f * d2;
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float y = y0 + 0.0625f * i, q = y * y;  // exact
            v[i].x = fmaf(bsp, q, d2p * y);
          }
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float y = y0 + 0.0625f * i, q = y * y;             // y and y^2, exact
            const float p1 = bh * q;                               // exact
            const float r1 = p1 - 2.f * rintf(0.5f * p1);          // exact reduction modulo 2
            const float ph = r1 + fmaf(bl, q, d2 * y);
            v[i].x = 3.14159265358979f * (ph - 2.f * rintf(0.5f * ph));
          }
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float wv = wreg[i];
          float sn, cs;
          __sincosf(v[i].x, &sn, &cs);
          v[i] = make_float2(wv * cs, wv * sn);
        }
        // 256 = 16 (lane-local, i) x 16 (across the half's lanes): output j0 + 16 j1 is
        // sum_l W16^{l j1} W256^{l j0} sum_i v_l[i] W16^{i j0}
        dft16(v);
#pragma unroll
        for (int j0 = 0; j0 < 16; ++j0) s_buf[w][hf][j0][l16] = j0 ? c_mul(v[at16(j0)], tw[j0]) : v[0];
        __syncwarp();
#pragma unroll
        for (int l = 0; l < 16; l += 2) {  // two at a time: 16-byte loads
          const float4 p = *reinterpret_cast<const float4*>(&s_buf[w][hf][l16][l]);
          v[l] = make_float2(p.x, p.y);
          v[l + 1] = make_float2(p.z, p.w);
        }
        __syncwarp();
        dft16(v);  // lane j0 = l16 now holds G[j0 + 16 j1] in v[at16(j1)]
        // kept outputs: j1 = 0..6 (j = j0 + 16 j1 <= 111) and j1 = 9..15 (j - 256 >= -112), those
        // with |j| <= P (the lane's mask) and, near the table's edges, inside it
        const unsigned use = live ? pmask : 0u;
        const float2* zb = a.z + (size_t)al * a.n_bin + b + l16;  // bin b + l16 of the segment's row
        const float* wb = a.wt + b + l16;
        float re = 0.f, im = 0.f, nr = 0.f;
        const auto acc = [&](const float2 G, const float2 zz, const float wv) {
          re = fmaf(zz.x, G.x, fmaf(zz.y, G.y, re));
          im = fmaf(zz.x, G.y, fmaf(-zz.y, G.x, im));
          nr = fmaf(wv, fmaf(G.x, G.x, G.y * G.y), nr);
        };
        if (b >= 112 && b + 111 < a.n_bin) {  // every kept output lies in the table
#pragma unroll
          for (int j1 = 0; j1 < 16; ++j1) {
            if (j1 == 7 || j1 == 8) continue;
            const int o = 16 * j1 - (j1 >= 9 ? kM : 0);
            if (use >> j1 & 1u) acc(v[at16(j1)], zb[o], wb[o]);
          }
        } else {
#pragma unroll
          for (int j1 = 0; j1 < 16; ++j1) {
            if (j1 == 7 || j1 == 8) continue;
            const int o = 16 * j1 - (j1 >= 9 ? kM : 0);
            const int kb = b + l16 + o;
            if ((use >> j1 & 1u) && kb >= 0 && kb < a.n_bin) acc(v[at16(j1)], zb[o], wb[o]);
          }
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {  // within the half
          re += __shfl_xor_sync(0xffffffffu, re, o);
          im += __shfl_xor_sync(0xffffffffu, im, o);
          nr += __shfl_xor_sync(0xffffffffu, nr, o);
        }
        if (nr > 0.f) sacc += (double)(fmaf(re, re, im * im) / nr);
      }
    }
    const double tot = __shfl_sync(0xffffffffu, sacc, 0) + __shfl_sync(0xffffffffu, sacc, 16);
    if (lane == 0) a.stat[t] = (float)tot;
  }
}

}  // namespace
}  // namespace tfs

using namespace tfs;

// Launches the kernel over up to kChirpMaxJobs jobs (tracks numbered job after job).
static int launch_chirp(const ChirpJob* jobs, int n_jobs, cudaStream_t st) {
  ChirpBatch B;
  B.n_jobs = n_jobs;
  B.start[0] = 0;
  for (int i = 0; i < n_jobs; ++i) {
    B.jobs[i] = jobs[i];
    B.start[i + 1] = B.start[i] + jobs[i].N;
  }
  for (int i = n_jobs; i < kChirpMaxJobs; ++i) B.start[i + 1] = B.start[n_jobs];
  const long long total = B.start[n_jobs];
  if (total == 0) return TFS_OK;
  int dev = 0, n_sm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chirp_stat_kernel, kCThreads, 0);
  const long long want = (total + kCW - 1) / kCW;
  const int grid =
      (int)std::max<long long>(1, std::min<long long>(want, (long long)std::max(1, n_sm) * std::max(1, per_sm)));
  chirp_stat_kernel<<<grid, kCThreads, 0, st>>>(B);
  count_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TFS_OK : cuda_fail(e, "chirp statistic");
}

static ChirpJob make_chirp_job(const tfs_ctable* ct, const tfs_basis* basis, const double* coeffs,
                               const double* f_ref, int64_t N, int P, int flags, float* stat) {
  ChirpJob a;
  a.z = ct->z;
  a.wt = ct->wt;
  a.n_seg = (int)ct->n_seg;
  a.n_bin = (int)ct->n_bin;
  a.U = basis->U;
  a.K = basis->K;
  a.coeffs = coeffs;
  a.f_ref = f_ref;
  a.N = N;
  a.T = ct->T_sft;
  a.P = P;
  a.cuts = (flags & TFS_JOB_SEGMENT_CUTS) ? 1 : 0;
  a.stat = stat;
  return a;
}

extern "C" int tfs_eval_chirp_stat(const tfs_ctable* ct, const tfs_basis* basis, const double* coeffs,
                                   const double* f_ref, int64_t N, int P, int flags, float* stat, int topk,
                                   int64_t* top_idx, float* top_val, void* stream) {
  clear_error();
  NvtxRange nvtx("tfs_eval_chirp_stat");
  TFS_CHECK(ct && basis, TFS_ERR_INVALID_ARG, "null table or basis");
  TFS_CHECK(basis->n_seg == ct->n_seg, TFS_ERR_INVALID_ARG, "basis has %lld segments, table %lld",
            (long long)basis->n_seg, (long long)ct->n_seg);
  TFS_CHECK(basis->K >= 1 && basis->K <= 32, TFS_ERR_INVALID_ARG, "basis size must be in [1, 32]");
  TFS_CHECK(N >= 0 && N < ((int64_t)1 << 31), TFS_ERR_INVALID_ARG, "N must be in [0, 2^31)");
  TFS_CHECK(P >= 0 && P <= kChirpPMax, TFS_ERR_INVALID_ARG, "P must be in [0, %d]", kChirpPMax);
  TFS_CHECK((flags & ~TFS_JOB_SEGMENT_CUTS) == 0, TFS_ERR_INVALID_ARG, "unknown flags");
  TFS_CHECK(topk >= 0 && topk <= 1024, TFS_ERR_INVALID_ARG, "topk must be in [0, 1024]");
  TFS_CHECK(N == 0 || coeffs, TFS_ERR_INVALID_ARG, "null coeffs");
  TFS_CHECK(stat || topk > 0 || N == 0, TFS_ERR_INVALID_ARG, "need stat or topk > 0");
  TFS_CHECK(topk == 0 || N == 0 || (top_idx && top_val), TFS_ERR_INVALID_ARG, "null top-k outputs");
  if (N == 0) return TFS_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float* d_stat = stat;
  void* ws = nullptr;
  const int kk = (int)std::min<int64_t>(topk, N);
  size_t need = (stat ? 0 : (((size_t)N * 4 + 255) & ~(size_t)255)) + (kk ? topk_workspace_bytes(N) : 0);
  char* scratch = nullptr;
  if (need) TFS_CUDA(cudaMallocAsync((void**)&scratch, need, st));
  if (!stat) d_stat = reinterpret_cast<float*>(scratch);
  if (kk) ws = scratch + (stat ? 0 : (((size_t)N * 4 + 255) & ~(size_t)255));
  const ChirpJob a = make_chirp_job(ct, basis, coeffs, f_ref, N, P, flags, d_stat);
  int rc = launch_chirp(&a, 1, st);
  if (rc == TFS_OK && kk) rc = topk_device(d_stat, N, kk, top_idx, top_val, ws, st);
  if (scratch) cudaFreeAsync(scratch, st);
  return rc;
}

extern "C" int tfs_ctable_view(const tfs_ctable* t, int64_t seg0, int64_t n_seg, tfs_ctable** out) {
  clear_error();
  TFS_CHECK(t && out, TFS_ERR_INVALID_ARG, "null argument");
  TFS_CHECK(seg0 >= 0 && n_seg >= 1 && seg0 + n_seg <= t->n_seg, TFS_ERR_INVALID_ARG,
            "rows [%lld, %lld) outside the table's %lld", (long long)seg0, (long long)(seg0 + n_seg),
            (long long)t->n_seg);
  tfs_ctable* v = new tfs_ctable();
  *v = *t;
  v->n_seg = n_seg;
  v->z = t->z + (size_t)seg0 * t->n_bin;
  v->sft_plan = nullptr;
  v->owns = false;
  *out = v;
  return TFS_OK;
}

extern "C" int tfs_eval_chirp_batch(const tfs_chirp_job* jobs, int n_jobs, void* stream) {
  clear_error();
  NvtxRange nvtx("tfs_eval_chirp_batch");
  TFS_CHECK(jobs && n_jobs >= 1 && n_jobs <= 4096, TFS_ERR_INVALID_ARG, "need 1 <= n_jobs <= 4096 jobs");
  std::vector<ChirpJob> cj;
  for (int i = 0; i < n_jobs; ++i) {
    const tfs_chirp_job& j = jobs[i];
    TFS_CHECK(j.table && j.basis, TFS_ERR_INVALID_ARG, "job %d: null table or basis", i);
    TFS_CHECK(j.basis->n_seg == j.table->n_seg, TFS_ERR_INVALID_ARG, "job %d: basis and table segment counts differ",
              i);
    TFS_CHECK(j.basis->K >= 1 && j.basis->K <= 32, TFS_ERR_INVALID_ARG, "job %d: basis size must be in [1, 32]", i);
    TFS_CHECK(j.N >= 0 && j.N < ((int64_t)1 << 31), TFS_ERR_INVALID_ARG, "job %d: N must be in [0, 2^31)", i);
    TFS_CHECK(j.P >= 0 && j.P <= kChirpPMax, TFS_ERR_INVALID_ARG, "job %d: P must be in [0, %d]", i, kChirpPMax);
    TFS_CHECK((j.flags & ~TFS_JOB_SEGMENT_CUTS) == 0, TFS_ERR_INVALID_ARG, "job %d: unknown flags", i);
    TFS_CHECK(j.N == 0 || (j.coeffs && j.stat), TFS_ERR_INVALID_ARG, "job %d: null coeffs or stat", i);
    if (j.N > 0) cj.push_back(make_chirp_job(j.table, j.basis, j.coeffs, j.f_ref, j.N, j.P, j.flags, j.stat));
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (size_t g0 = 0; g0 < cj.size(); g0 += kChirpMaxJobs) {
    const int n = (int)std::min<size_t>(kChirpMaxJobs, cj.size() - g0);
    const int rc = launch_chirp(cj.data() + g0, n, st);
    if (rc) return rc;
  }
  return TFS_OK;
}
