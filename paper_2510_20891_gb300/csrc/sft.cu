// Steps 1-2 of the method: strain -> windowed SFTs -> PSD-normalised power
// table (paper Sec. II.B: d~_{alpha,k} and 4 Delta f |d~|^2 / S_n with
// Delta f = 1/T_SFT; Sec. II.E: known PSD).
//
// All arithmetic is FP64: the red-noise PSDs of the one-year workloads put
// almost all of a segment's energy in its lowest bins (a dynamic range of
// ~1e6 in amplitude), which FP32 rounding would leak into the band.
//
// Each segment of L = T_SFT/dt real samples is transformed as N = L/2
// complex points z[j] = w[2j] x[2j] + i w[2j+1] x[2j+1] by a four-step FFT
// N = N1 x N2 (column FFTs of length N1 with the inter-step twiddles
// W_N^{n2 k1}, then row FFTs of length N2), each small FFT a mixed-radix
// (4, 2, 3, 5) self-sorting Stockham pass sequence in shared memory.  The
// real spectrum follows from X_k = (Z_k + Z*_{N-k})/2 - i e^{-2 pi i k/L}
// (Z_k - Z*_{N-k})/2, and P_k = 4 dt |X_k|^2 / (sum w^2 S_n(k/T_SFT)).
#include <algorithm>
#include <cmath>
#include <vector>

#include "tfs_internal.cuh"

namespace tfs {

namespace {

struct FftPlan {
  int n;
  int nr;
  int radix[20];
};

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 mul_mi(double2 a) { return make_double2(a.y, -a.x); }  // -i * a

struct RadixConsts {
  double h3, c1, c2, s1, s2;  // sqrt(3)/2, cos(2pi/5), cos(4pi/5), sin(2pi/5), sin(4pi/5)
};

__device__ __forceinline__ void dft_r(double2* v, int R, const RadixConsts& K) {
  if (R == 2) {
    const double2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if (R == 4) {
    const double2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    const double2 t2 = cadd(v[1], v[3]), t3 = csub(v[1], v[3]);
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, mul_mi(t3));
    v[3] = csub(t1, mul_mi(t3));
  } else if (R == 3) {
    const double2 a = v[0], s = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    const double2 t = csub(a, cscale(s, 0.5));
    const double2 mid = mul_mi(cscale(d, K.h3));
    v[0] = cadd(a, s);
    v[1] = cadd(t, mid);
    v[2] = csub(t, mid);
  } else {  // R == 5
    const double2 a = v[0];
    const double2 p1 = cadd(v[1], v[4]), m1 = csub(v[1], v[4]);
    const double2 p2 = cadd(v[2], v[3]), m2 = csub(v[2], v[3]);
    const double2 A1 = cadd(a, cadd(cscale(p1, K.c1), cscale(p2, K.c2)));
    const double2 B1 = cadd(cscale(m1, K.s1), cscale(m2, K.s2));
    const double2 A2 = cadd(a, cadd(cscale(p1, K.c2), cscale(p2, K.c1)));
    const double2 B2 = csub(cscale(m1, K.s2), cscale(m2, K.s1));
    v[0] = cadd(a, cadd(p1, p2));
    v[1] = cadd(A1, mul_mi(B1));
    v[4] = csub(A1, mul_mi(B1));
    v[2] = cadd(A2, mul_mi(B2));
    v[3] = csub(A2, mul_mi(B2));
  }
}

// ncol independent length-n FFTs on shared-memory columns d0[col*n + i];
// tw[i] = W_n^i.  Returns the buffer that holds the result (d0 or d1).
__device__ double2* small_fft(double2* d0, double2* d1, int ncol, const FftPlan& p, const double2* tw,
                              const RadixConsts& K) {
  const int n = p.n;
  int Ns = 1;
  for (int s = 0; s < p.nr; ++s) {
    const int R = p.radix[s];
    const int nb = n / R;
    const int step = n / (Ns * R);
    for (int idx = threadIdx.x; idx < ncol * nb; idx += blockDim.x) {
      const int col = idx / nb;
      const int j = idx - col * nb;
      const double2* in = d0 + (size_t)col * n;
      double2* out = d1 + (size_t)col * n;
      const int k = j % Ns;
      double2 v[5];
      for (int r = 0; r < R; ++r) v[r] = in[j + r * nb];
      if (Ns > 1)  // the first stage's twiddles are all 1
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[r * k * step]);
      dft_r(v, R, K);
      const int o = (j / Ns) * Ns * R + k;
      for (int r = 0; r < R; ++r) out[o + r * Ns] = v[r];
    }
    __syncthreads();
    double2* t = d0;
    d0 = d1;
    d1 = t;
    Ns *= R;
  }
  return d0;
}

__device__ RadixConsts make_consts() {
  RadixConsts K;
  const double r5 = sqrt(5.0);
  K.h3 = 0.5 * sqrt(3.0);
  K.c1 = 0.25 * (r5 - 1.0);
  K.c2 = -0.25 * (r5 + 1.0);
  K.s1 = sqrt((5.0 + r5) / 8.0);
  K.s2 = sqrt((5.0 - r5) / 8.0);
  return K;
}

// Step 1: column FFTs of length N1 over CB consecutive columns n2, input straight from the strain.
__global__ void sft_cols(const double* __restrict__ strain, const double* __restrict__ win, int L, int N1, int N2,
                         int CB, FftPlan p1, const double2* __restrict__ tw1, const double2* __restrict__ twN,
                         double2* __restrict__ Y) {
  extern __shared__ __align__(16) double2 sm[];
  double2* b0 = sm;
  double2* b1 = sm + (size_t)CB * N1;
  double2* tws = sm + (size_t)2 * CB * N1;
  const int seg = blockIdx.y;
  const int c0 = blockIdx.x * CB;
  const int N = N1 * N2;
  for (int i = threadIdx.x; i < N1; i += blockDim.x) tws[i] = tw1[i];
  const double* x = strain + (size_t)seg * L;
  for (int idx = threadIdx.x; idx < CB * N1; idx += blockDim.x) {
    const int col = idx % CB, n1 = idx / CB;
    const int n2 = c0 + col;
    double2 z = make_double2(0.0, 0.0);
    if (n2 < N2) {
      const int j = N2 * n1 + n2;
      z = make_double2(x[2 * j] * win[2 * j], x[2 * j + 1] * win[2 * j + 1]);
    }
    b0[(size_t)col * N1 + n1] = z;
  }
  __syncthreads();
  const RadixConsts K = make_consts();
  const double2* res = small_fft(b0, b1, CB, p1, tws, K);
  double2* y = Y + (size_t)seg * N;
  for (int idx = threadIdx.x; idx < CB * N1; idx += blockDim.x) {
    const int col = idx % CB, k1 = idx / CB;
    const int n2 = c0 + col;
    if (n2 < N2) {
      double2 v = res[(size_t)col * N1 + k1];
      if (N2 > 1) v = cmul(v, twN[(size_t)n2 * k1]);
      y[(size_t)k1 * N2 + n2] = v;
    }
  }
}

// Step 2: row FFTs of length N2 over RB consecutive rows k1; Z[k1 + N1 k2].
__global__ void sft_rows(const double2* __restrict__ Y, int N1, int N2, int RB, FftPlan p2,
                         const double2* __restrict__ tw2, double2* __restrict__ Z) {
  extern __shared__ __align__(16) double2 sm[];
  double2* b0 = sm;
  double2* b1 = sm + (size_t)RB * N2;
  double2* tws = sm + (size_t)2 * RB * N2;
  const int seg = blockIdx.y;
  const int r0 = blockIdx.x * RB;
  const int N = N1 * N2;
  for (int i = threadIdx.x; i < N2; i += blockDim.x) tws[i] = tw2[i];
  const double2* y = Y + (size_t)seg * N;
  for (int idx = threadIdx.x; idx < RB * N2; idx += blockDim.x) {
    const int row = idx / N2, n2 = idx - row * N2;
    const int k1 = r0 + row;
    b0[idx] = k1 < N1 ? y[(size_t)k1 * N2 + n2] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const RadixConsts K = make_consts();
  const double2* res = small_fft(b0, b1, RB, p2, tws, K);
  double2* z = Z + (size_t)seg * N;
  for (int idx = threadIdx.x; idx < RB * N2; idx += blockDim.x) {
    const int row = idx % RB, k2 = idx / RB;
    const int k1 = r0 + row;
    if (k1 < N1) z[(size_t)k1 + (size_t)N1 * k2] = res[(size_t)row * N2 + k2];
  }
}

// Step 3: real spectrum and normalised power, FP64, P [n_seg][n_bin].  With E = z_k + conj(z_{N-k})
// and O = z_k - conj(z_{N-k}), X_k = (E - i W_L^k O) / 2: the halving is exact, so it is left to the
// per-bin scale (pscale4 = pscale / 4 for |X_k|^2), which gives the same bits.
__device__ __forceinline__ double power_bin(const double2* __restrict__ Z, int N, const double2* __restrict__ twU,
                                            const double* __restrict__ pscale4, int seg, int k) {
  const double2* z = Z + (size_t)seg * N;
  const double2 zk = z[k == N ? 0 : k];
  const double2 zn0 = z[k == 0 ? 0 : N - k];
  const double2 zn = make_double2(zn0.x, -zn0.y);
  const double2 X2 = cadd(cadd(zk, zn), mul_mi(cmul(twU[k], csub(zk, zn))));  // 2 X_k
  return (X2.x * X2.x + X2.y * X2.y) * pscale4[k];
}

__global__ void sft_power(const double2* __restrict__ Z, int N, const double2* __restrict__ twU,
                          const double* __restrict__ pscale4, double* __restrict__ P) {
  const int seg = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > N) return;
  P[(size_t)seg * (N + 1) + k] = power_bin(Z, N, twU, pscale4, seg, k);
}

// Step 3 for the linear-chirp table: the complex spectrum scaled per bin, FP32 pairs
// z [n_seg][n_bin] = X_k zscale_k, computed as 2 X_k times zscale2 = zscale / 2 (the same bits).
__global__ void sft_cspec(const double2* __restrict__ Z, int N, const double2* __restrict__ twU,
                          const double* __restrict__ zscale2, float2* __restrict__ zout) {
  const int seg = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > N) return;
  const double2* z = Z + (size_t)seg * N;
  const double2 zk = z[k == N ? 0 : k];
  const double2 zn0 = z[k == 0 ? 0 : N - k];
  const double2 zn = make_double2(zn0.x, -zn0.y);
  const double2 X2 = cadd(cadd(zk, zn), mul_mi(cmul(twU[k], csub(zk, zn))));  // 2 X_k
  zout[(size_t)seg * (N + 1) + k] = make_float2((float)(X2.x * zscale2[k]), (float)(X2.y * zscale2[k]));
}

}  // namespace

// ---------------------------------------------------------------- quantisation into a table
template <int DT>
__device__ __forceinline__ void store_q(void* row, int k, double v, double inv_s) {
  if (DT == TFS_F32) static_cast<float*>(row)[k] = (float)v;
  if (DT == TFS_BF16) static_cast<__nv_bfloat16*>(row)[k] = __double2bfloat16(v);
  if (DT == TFS_F16) static_cast<__half*>(row)[k] = __double2half(v);
  if (DT == TFS_F8E4M3) {
    __nv_fp8_storage_t q = __nv_cvt_double_to_fp8(v * inv_s, __NV_SATFINITE, __NV_E4M3);
    static_cast<__nv_fp8_storage_t*>(row)[k] = q;
  }
}

template <int DT>
__global__ void quantise_rows(const double* __restrict__ P, long long ld, int n_bin, int row_stride,
                             void* __restrict__ data, float* __restrict__ scales) {
  const int seg = blockIdx.x;
  const double* p = P + (size_t)seg * ld;
  void* row = static_cast<char*>(data) + (size_t)seg * row_stride * (DT == TFS_F32 ? 4 : (DT == TFS_F8E4M3 ? 1 : 2));
  double inv_s = 1.0;
  if (DT == TFS_F8E4M3) {
    // M = min(max P, 256 * 2^e*), e* the lower median of floor(log2 P) over P > 0; s = fp32(M / 448)
    constexpr int kEmin = -1100, kEbins = 2201;  // floor(log2) of any positive double, offset
    __shared__ unsigned int hist[kEbins];
    __shared__ double wm[32];
    __shared__ unsigned int npos_s[32];
    __shared__ int estar;
    for (int i = threadIdx.x; i < kEbins; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    double mx = 0.0;
    unsigned int npos = 0;
    for (int k = threadIdx.x; k < n_bin; k += blockDim.x) {
      const double v = p[k];
      if (v > 0.0) {
        mx = fmax(mx, v);
        ++npos;
        const int e = ilogb(v);  // floor(log2 v), exact for every positive double
        atomicAdd(&hist[min(max(e, kEmin), kEmin + kEbins - 1) - kEmin], 1u);
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      npos += __shfl_xor_sync(0xffffffffu, npos, o);
    }
    if ((threadIdx.x & 31) == 0) {
      wm[threadIdx.x >> 5] = mx;
      npos_s[threadIdx.x >> 5] = npos;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned int n = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        mx = fmax(mx, wm[w]);
        n += npos_s[w];
      }
      wm[0] = mx;
      const unsigned int need = (n + 1) / 2;
      unsigned int run = 0;
      int es = 0;
      for (int i = 0; i < kEbins && n > 0; ++i) {
        run += hist[i];
        if (run >= need) {
          es = i + kEmin;
          break;
        }
      }
      estar = n > 0 ? es : 0;
      npos_s[0] = n;
    }
    __syncthreads();
    mx = wm[0];
    const double M = npos_s[0] > 0 ? fmin(mx, 256.0 * ldexp(1.0, estar)) : 0.0;
    const float s = M > 0.0 ? __double2float_rn(M / 448.0) : 1.0f;
    if (threadIdx.x == 0) scales[seg] = s;
    for (int k = threadIdx.x; k < n_bin; k += blockDim.x) {
      const double q = p[k] / (double)s;
      store_q<DT>(row, k, q, 1.0);
    }
    return;
  }
  for (int k = threadIdx.x; k < n_bin; k += blockDim.x) store_q<DT>(row, k, p[k], inv_s);
}

template <int DT>
__device__ __forceinline__ double load_q(const void* row, int k) {
  if (DT == TFS_F32) return (double)static_cast<const float*>(row)[k];
  if (DT == TFS_BF16) return (double)__bfloat162float(static_cast<const __nv_bfloat16*>(row)[k]);
  if (DT == TFS_F16) return (double)__half2float(static_cast<const __half*>(row)[k]);
  return (double)static_cast<float>(static_cast<const __nv_fp8_e4m3*>(row)[k]);
}

// dequantised FP64 copy of a table (FP8: the FP32 product q * s_alpha)
template <int DT>
__global__ void dequantise_rows(const void* __restrict__ data, const float* __restrict__ scales, int n_bin,
                                int row_stride, double* __restrict__ P) {
  const int seg = blockIdx.x;
  const void* row = static_cast<const char*>(data) + (size_t)seg * row_stride * (DT == TFS_F32 ? 4 : (DT == TFS_F8E4M3 ? 1 : 2));
  const float s = DT == TFS_F8E4M3 ? scales[seg] : 1.0f;
  for (int k = threadIdx.x; k < n_bin; k += blockDim.x) {
    const double v = load_q<DT>(row, k);
    P[(size_t)seg * n_bin + k] = DT == TFS_F8E4M3 ? (double)((float)v * s) : v;
  }
}

// Step 3 straight into an FP32, BF16 or FP16 table: the elementwise rounding that quantise_rows
// would store from sft_power's output (FP8 needs each row's scale first: it keeps both passes).
template <int DT>
__global__ void sft_power_store(const double2* __restrict__ Z, int N, const double2* __restrict__ twU,
                                const double* __restrict__ pscale4, void* __restrict__ data, int row_stride) {
  const int seg = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > N) return;
  void* row = static_cast<char*>(data) + (size_t)seg * row_stride * (DT == TFS_F32 ? 4 : 2);
  store_q<DT>(row, k, power_bin(Z, N, twU, pscale4, seg, k), 1.0);
}

int quantise_into(const double* P, int64_t ld, tfs_table* t, cudaStream_t st) {
  const int ns = (int)t->n_seg;
  switch (t->dtype) {
    case TFS_F32: quantise_rows<TFS_F32><<<ns, 256, 0, st>>>(P, ld, (int)t->n_bin, (int)t->row_stride, t->data, t->scales); break;
    case TFS_BF16: quantise_rows<TFS_BF16><<<ns, 256, 0, st>>>(P, ld, (int)t->n_bin, (int)t->row_stride, t->data, t->scales); break;
    case TFS_F16: quantise_rows<TFS_F16><<<ns, 256, 0, st>>>(P, ld, (int)t->n_bin, (int)t->row_stride, t->data, t->scales); break;
    case TFS_F8E4M3: quantise_rows<TFS_F8E4M3><<<ns, 256, 0, st>>>(P, ld, (int)t->n_bin, (int)t->row_stride, t->data, t->scales); break;
    default: set_error("bad dtype"); return TFS_ERR_INVALID_ARG;
  }
  count_launch();
  TFS_CUDA(cudaGetLastError());
  return TFS_OK;
}

// ---------------------------------------------------------------- host planning
static bool smooth235(int64_t n) {
  for (int r : {2, 3, 5})
    while (n % r == 0) n /= r;
  return n == 1;
}

static FftPlan make_plan(int n) {
  FftPlan p{};
  p.n = n;
  int m = n;
  // radix 4 while possible (leaving a single 2 when the power of two is odd), then 2, 3, 5
  while (m % 4 == 0) {
    p.radix[p.nr++] = 4;
    m /= 4;
  }
  while (m % 2 == 0) {
    p.radix[p.nr++] = 2;
    m /= 2;
  }
  while (m % 3 == 0) {
    p.radix[p.nr++] = 3;
    m /= 3;
  }
  while (m % 5 == 0) {
    p.radix[p.nr++] = 5;
    m /= 5;
  }
  return p;
}

static void twiddles(int n, std::vector<double2>& out) {
  out.resize(n);
  for (int i = 0; i < n; ++i) {
    const double a = 2.0 * M_PI * (double)i / (double)n;
    out[i] = make_double2(std::cos(a), -std::sin(a));
  }
}

}  // namespace tfs

using namespace tfs;

extern "C" int tfs_table_to_host(const tfs_table* t, double* P, float* scales) {
  clear_error();
  TFS_CHECK(t && P, TFS_ERR_INVALID_ARG, "null argument");
  double* d = nullptr;
  const size_t bytes = (size_t)t->n_seg * t->n_bin * 8;
  TFS_CUDA(cudaMalloc(&d, bytes));
  const int ns = (int)t->n_seg, nb = (int)t->n_bin, rs = (int)t->row_stride;
  switch (t->dtype) {
    case TFS_F32: dequantise_rows<TFS_F32><<<ns, 256>>>(t->data, t->scales, nb, rs, d); break;
    case TFS_BF16: dequantise_rows<TFS_BF16><<<ns, 256>>>(t->data, t->scales, nb, rs, d); break;
    case TFS_F16: dequantise_rows<TFS_F16><<<ns, 256>>>(t->data, t->scales, nb, rs, d); break;
    default: dequantise_rows<TFS_F8E4M3><<<ns, 256>>>(t->data, t->scales, nb, rs, d); break;
  }
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(P, d, bytes, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && scales && t->scales) e = cudaMemcpy(scales, t->scales, (size_t)t->n_seg * 4, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "tfs_table_to_host");
  return TFS_OK;
}

extern "C" int tfs_table_export(const tfs_table* t, void* data, float* scales) {
  clear_error();
  TFS_CHECK(t && data, TFS_ERR_INVALID_ARG, "null argument");
  TFS_CHECK(t->data, TFS_ERR_INVALID_ARG, "table has no device data");
  const size_t bytes = (size_t)t->n_seg * t->row_stride * esize_of(t->dtype);
  TFS_CUDA(cudaMemcpy(data, t->data, bytes, cudaMemcpyDeviceToHost));
  if (scales && t->scales) TFS_CUDA(cudaMemcpy(scales, t->scales, (size_t)t->n_seg * 4, cudaMemcpyDeviceToHost));
  return TFS_OK;
}

extern "C" int tfs_table_import(const void* data, const float* scales, int64_t n_seg, int64_t n_bin, double T_sft,
                                int dtype, tfs_table** out) {
  clear_error();
  TFS_CHECK(data && out, TFS_ERR_INVALID_ARG, "null argument");
  TFS_CHECK(n_seg >= 1 && n_seg <= (1 << 24) && n_bin >= 1 && n_bin <= (1 << 24), TFS_ERR_INVALID_ARG,
            "bad table shape");
  TFS_CHECK(dtype >= TFS_F32 && dtype <= TFS_F8E4M3, TFS_ERR_INVALID_ARG, "bad dtype");
  TFS_CHECK(dtype != TFS_F8E4M3 || scales, TFS_ERR_INVALID_ARG, "an FP8 table needs its scales");
  TFS_CHECK(T_sft > 0 && std::isfinite(T_sft), TFS_ERR_INVALID_ARG, "bad T_sft");
  tfs_table* t = nullptr;
  int rc = alloc_table(n_seg, n_bin, dtype, T_sft, &t);
  if (rc) return rc;
  const size_t bytes = (size_t)n_seg * t->row_stride * esize_of(dtype);
  cudaError_t e = cudaMemcpy(t->data, data, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && t->scales) e = cudaMemcpy(t->scales, scales, (size_t)n_seg * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    tfs_table_free(t);
    return cuda_fail(e, "table import");
  }
  *out = t;
  return TFS_OK;
}

extern "C" int tfs_table_from_power(const double* P, int64_t n_seg, int64_t n_bin, double T_sft, int dtype, int mem,
                                    void* stream, tfs_table** out) {
  clear_error();
  TFS_CHECK(P && out, TFS_ERR_INVALID_ARG, "null argument");
  TFS_CHECK(n_seg >= 1 && n_seg <= (1 << 24) && n_bin >= 1 && n_bin <= (1 << 24), TFS_ERR_INVALID_ARG,
            "bad table shape");
  TFS_CHECK(dtype >= TFS_F32 && dtype <= TFS_F8E4M3, TFS_ERR_INVALID_ARG, "bad dtype");
  TFS_CHECK(mem == TFS_MEM_HOST || mem == TFS_MEM_DEVICE, TFS_ERR_INVALID_ARG, "bad mem kind");
  TFS_CHECK(T_sft > 0 && std::isfinite(T_sft), TFS_ERR_INVALID_ARG, "bad T_sft");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  tfs_table* t = nullptr;
  int rc = alloc_table(n_seg, n_bin, dtype, T_sft, &t);
  if (rc) return rc;
  const double* dP = P;
  double* tmp = nullptr;
  if (mem == TFS_MEM_HOST) {
    cudaError_t e = cudaMalloc(&tmp, (size_t)n_seg * n_bin * 8);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, P, (size_t)n_seg * n_bin * 8, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      if (tmp) cudaFree(tmp);
      tfs_table_free(t);
      return cuda_fail(e, "table upload");
    }
    dP = tmp;
  }
  rc = quantise_into(dP, n_bin, t, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (tmp) cudaFree(tmp);
  if (rc == TFS_OK && e != cudaSuccess) rc = cuda_fail(e, "quantise");
  if (rc) {
    tfs_table_free(t);
    return rc;
  }
  *out = t;
  return TFS_OK;
}

namespace tfs {

struct SftPlan {
  int64_t L = 0;
  int N = 0, N1 = 0, N2 = 0, CB = 1, RB = 1;
  FftPlan p1{}, p2{};
  double* win = nullptr;      // [L]
  double* pscale = nullptr;   // [n_bin]: 4 dt / (sum w^2 S_n) / 4, 0 where unusable (scales |2 X_k|^2)
  double* zscale = nullptr;   // [n_bin]: sqrt(4 dt / (sum w^2 S_ref)) S_ref / S_n / 2, 0 where unusable
  float* wt = nullptr;        // [n_bin]: S_ref / S_n, 0 where unusable
  double s_ref = 1.0;         // median of the usable S_n (keeps the chirp table's values near 1)
  double2* tw1 = nullptr;     // [N1]
  double2* tw2 = nullptr;     // [N2]
  double2* twN = nullptr;     // [N] (N2 > 1)
  double2* twU = nullptr;     // [n_bin]
  size_t sm1 = 0, sm2 = 0;
};

void free_sft_plan(void* p) {
  SftPlan* s = static_cast<SftPlan*>(p);
  if (!s) return;
  for (void* q : {(void*)s->win, (void*)s->pscale, (void*)s->zscale, (void*)s->wt, (void*)s->tw1, (void*)s->tw2,
                  (void*)s->twN, (void*)s->twU})
    if (q) cudaFree(q);
  delete s;
}

static int make_sft_plan(int64_t L, double dt, int window, const double* psd, int mem, SftPlan** out) {
  const int N = (int)(L / 2);
  const int64_t n_bin = N + 1;
  int N1 = N, N2 = 1;
  if (N > 1024) {
    for (int d = (int)std::sqrt((double)N); d >= 2; --d)
      if (N % d == 0) {
        N1 = d;
        N2 = N / d;
        break;
      }
  }
  TFS_CHECK(N1 <= 4096 && N2 <= 4096, TFS_ERR_INVALID_ARG, "segment length has no usable factorisation");
  std::vector<double> win(L), pscale(n_bin), psd_h(n_bin);
  double sw2 = 0.0;
  for (int64_t i = 0; i < L; ++i) {
    const double sn = std::sin(M_PI * (double)i / (double)L);
    win[i] = window == TFS_WINDOW_HANN ? sn * sn : 1.0;
    sw2 += win[i] * win[i];
  }
  if (mem == TFS_MEM_DEVICE)
    TFS_CUDA(cudaMemcpy(psd_h.data(), psd, n_bin * 8, cudaMemcpyDeviceToHost));
  else
    for (int64_t k = 0; k < n_bin; ++k) psd_h[k] = psd[k];
  std::vector<double> usable;
  for (int64_t k = 0; k < n_bin; ++k) {
    const double S = psd_h[k];
    const bool ok = std::isfinite(S) && S > 0 && k > 0;
    pscale[k] = ok ? 4.0 * dt / (sw2 * S) : 0.0;
    if (ok) usable.push_back(S);
  }
  double s_ref = 1.0;
  if (!usable.empty()) {
    std::nth_element(usable.begin(), usable.begin() + usable.size() / 2, usable.end());
    s_ref = usable[usable.size() / 2];
  }
  std::vector<double> zscale(n_bin);
  std::vector<float> wt(n_bin);
  for (int64_t k = 0; k < n_bin; ++k) {
    const bool ok = pscale[k] > 0.0;
    zscale[k] = ok ? std::sqrt(4.0 * dt / (sw2 * s_ref)) * (s_ref / psd_h[k]) : 0.0;
    wt[k] = ok ? (float)(s_ref / psd_h[k]) : 0.f;
  }
  std::vector<double2> tw1, tw2, twN, twU(n_bin);
  twiddles(N1, tw1);
  twiddles(N2, tw2);
  if (N2 > 1) twiddles(N, twN);
  for (int64_t k = 0; k < n_bin; ++k) {
    const double a = 2.0 * M_PI * (double)k / (double)L;
    twU[k] = make_double2(std::cos(a), -std::sin(a));
  }
  SftPlan* s = new SftPlan();
  s->L = L;
  s->N = N;
  s->N1 = N1;
  s->N2 = N2;
  s->p1 = make_plan(N1);
  s->p2 = make_plan(N2);
  const int smem_cap = 96 * 1024;
  s->CB = std::max(1, std::min(16, smem_cap / (32 * N1)));
  s->RB = std::max(1, std::min(16, smem_cap / (32 * N2)));
  s->sm1 = ((size_t)2 * s->CB * N1 + N1) * 16;
  s->sm2 = ((size_t)2 * s->RB * N2 + N2) * 16;
  cudaError_t e = cudaSuccess;
  auto up = [&](void** dst, const void* src, size_t bytes) {
    if (e != cudaSuccess || bytes == 0) return;
    e = cudaMalloc(dst, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
  };
  up((void**)&s->win, win.data(), L * 8);
  // on the device the scales take the untangling's exact factor 1/2 of X_k (sft_power, sft_cspec)
  std::vector<double> pscale4(n_bin), zscale2(n_bin);
  for (int k = 0; k < n_bin; ++k) {
    pscale4[k] = 0.25 * pscale[k];
    zscale2[k] = 0.5 * zscale[k];
  }
  up((void**)&s->pscale, pscale4.data(), n_bin * 8);
  up((void**)&s->zscale, zscale2.data(), n_bin * 8);
  up((void**)&s->wt, wt.data(), n_bin * 4);
  s->s_ref = s_ref;
  up((void**)&s->tw1, tw1.data(), (size_t)N1 * 16);
  up((void**)&s->tw2, tw2.data(), (size_t)N2 * 16);
  if (N2 > 1) up((void**)&s->twN, twN.data(), (size_t)N * 16);
  up((void**)&s->twU, twU.data(), n_bin * 16);
  if (e == cudaSuccess && s->sm1 > 48 * 1024)
    e = cudaFuncSetAttribute(sft_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->sm1);
  if (e == cudaSuccess && s->sm2 > 48 * 1024)
    e = cudaFuncSetAttribute(sft_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->sm2);
  if (e != cudaSuccess) {
    free_sft_plan(s);
    return cuda_fail(e, "SFT plan");
  }
  *out = s;
  return TFS_OK;
}

// The column and row FFT passes of every segment: returns the half-length spectra (Y or Z).
static int run_fft_passes(const SftPlan* p, const double* d_x, int64_t n_seg, double2** Y, double2** Z,
                          const double2** out, cudaStream_t st) {
  const size_t nz = (size_t)n_seg * p->N;
  TFS_CUDA(cudaMallocAsync((void**)Y, nz * 16, st));
  if (p->N2 > 1) TFS_CUDA(cudaMallocAsync((void**)Z, nz * 16, st));
  dim3 g1((p->N2 + p->CB - 1) / p->CB, (unsigned)n_seg);
  sft_cols<<<g1, 256, p->sm1, st>>>(d_x, p->win, (int)p->L, p->N1, p->N2, p->CB, p->p1, p->tw1, p->twN, *Y);
  count_launch();
  *out = *Y;
  if (p->N2 > 1) {
    dim3 g2((p->N1 + p->RB - 1) / p->RB, (unsigned)n_seg);
    sft_rows<<<g2, 256, p->sm2, st>>>(*Y, p->N1, p->N2, p->RB, p->p2, p->tw2, *Z);
    count_launch();
    *out = *Z;
  }
  return TFS_OK;
}

// Strain -> linear-chirp table (complex spectra scaled per bin) on `st`.
static int run_sft_complex(const SftPlan* p, const double* d_x, tfs_ctable* t, cudaStream_t st) {
  double2 *Y = nullptr, *Z = nullptr;
  const double2* Zp = nullptr;
  int rc = run_fft_passes(p, d_x, t->n_seg, &Y, &Z, &Zp, st);
  if (rc == TFS_OK) {
    dim3 g3((unsigned)((t->n_bin + 255) / 256), (unsigned)t->n_seg);
    sft_cspec<<<g3, 256, 0, st>>>(Zp, p->N, p->twU, p->zscale, t->z);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "SFT kernels");
  }
  if (Y) cudaFreeAsync(Y, st);
  if (Z) cudaFreeAsync(Z, st);
  return rc;
}

// Enqueue the whole strain -> table computation on `st` (device strain; scratch is stream-ordered).
static int run_sft(const SftPlan* p, const double* d_x, tfs_table* t, cudaStream_t st) {
  const int64_t n_seg = t->n_seg, n_bin = t->n_bin;
  const size_t nz = (size_t)n_seg * p->N;
  double2 *Y = nullptr, *Z = nullptr;
  double* P = nullptr;
  TFS_CUDA(cudaMallocAsync((void**)&Y, nz * 16, st));
  if (p->N2 > 1) TFS_CUDA(cudaMallocAsync((void**)&Z, nz * 16, st));
  const bool f8 = t->dtype == TFS_F8E4M3;
  if (f8) TFS_CUDA(cudaMallocAsync((void**)&P, (size_t)n_seg * n_bin * 8, st));
  dim3 g1((p->N2 + p->CB - 1) / p->CB, (unsigned)n_seg);
  sft_cols<<<g1, 256, p->sm1, st>>>(d_x, p->win, (int)p->L, p->N1, p->N2, p->CB, p->p1, p->tw1, p->twN, Y);
  count_launch();
  const double2* Zp = Y;
  if (p->N2 > 1) {
    dim3 g2((p->N1 + p->RB - 1) / p->RB, (unsigned)n_seg);
    sft_rows<<<g2, 256, p->sm2, st>>>(Y, p->N1, p->N2, p->RB, p->p2, p->tw2, Z);
    count_launch();
    Zp = Z;
  }
  dim3 g3((unsigned)((n_bin + 255) / 256), (unsigned)n_seg);
  const int rs = (int)t->row_stride;
  switch (t->dtype) {
    case TFS_F32: sft_power_store<TFS_F32><<<g3, 256, 0, st>>>(Zp, p->N, p->twU, p->pscale, t->data, rs); break;
    case TFS_BF16: sft_power_store<TFS_BF16><<<g3, 256, 0, st>>>(Zp, p->N, p->twU, p->pscale, t->data, rs); break;
    case TFS_F16: sft_power_store<TFS_F16><<<g3, 256, 0, st>>>(Zp, p->N, p->twU, p->pscale, t->data, rs); break;
    case TFS_F8E4M3: sft_power<<<g3, 256, 0, st>>>(Zp, p->N, p->twU, p->pscale, P); break;
    default:
      cudaFreeAsync(Y, st);
      if (Z) cudaFreeAsync(Z, st);
      set_error("bad dtype");
      return TFS_ERR_INVALID_ARG;
  }
  count_launch();
  cudaError_t e = cudaGetLastError();
  int rc = e == cudaSuccess ? (f8 ? quantise_into(P, n_bin, t, st) : TFS_OK) : cuda_fail(e, "SFT kernels");
  cudaFreeAsync(Y, st);
  if (Z) cudaFreeAsync(Z, st);
  if (P) cudaFreeAsync(P, st);
  return rc;
}

}  // namespace tfs

extern "C" int tfs_build_sfts(const double* strain, int64_t n, double dt, double T_sft, int window,
                              const double* psd, int dtype, int mem, void* stream, tfs_table** out) {
  clear_error();
  NvtxRange nvtx("tfs_build_sfts");
  TFS_CHECK(strain && psd && out, TFS_ERR_INVALID_ARG, "null argument");
  TFS_CHECK(dt > 0 && T_sft > 0 && std::isfinite(dt) && std::isfinite(T_sft), TFS_ERR_INVALID_ARG,
            "dt and T_sft must be positive");
  TFS_CHECK(window == TFS_WINDOW_RECT || window == TFS_WINDOW_HANN, TFS_ERR_INVALID_ARG, "bad window");
  TFS_CHECK(dtype >= TFS_F32 && dtype <= TFS_F8E4M3, TFS_ERR_INVALID_ARG, "bad dtype");
  TFS_CHECK(mem == TFS_MEM_HOST || mem == TFS_MEM_DEVICE, TFS_ERR_INVALID_ARG, "bad mem kind");
  const double Lf = T_sft / dt;
  const int64_t L = (int64_t)std::llround(Lf);
  TFS_CHECK(L >= 4 && L <= (1 << 20) && std::fabs(Lf - (double)L) <= 1e-9 * Lf, TFS_ERR_INVALID_ARG,
            "T_sft/dt must be an integer in [4, 2^20]");
  TFS_CHECK(L % 2 == 0 && smooth235(L), TFS_ERR_INVALID_ARG,
            "T_sft/dt = %lld must be even with prime factors 2, 3, 5 only", (long long)L);
  const int64_t n_seg = n / L;
  TFS_CHECK(n_seg >= 1 && n_seg <= 65535, TFS_ERR_INVALID_ARG, "need 1 <= n/L <= 65535 segments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SftPlan* plan = nullptr;
  int rc = make_sft_plan(L, dt, window, psd, mem, &plan);
  if (rc) return rc;
  tfs_table* t = nullptr;
  rc = alloc_table(n_seg, L / 2 + 1, dtype, T_sft, &t);
  if (rc) {
    free_sft_plan(plan);
    return rc;
  }
  t->sft_plan = plan;
  t->dt = dt;
  rc = tfs_table_rebuild(t, strain, n, mem, stream);
  if (rc == TFS_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "build_sfts");
  }
  if (rc) {
    tfs_table_free(t);
    return rc;
  }
  *out = t;
  return TFS_OK;
}

extern "C" int tfs_table_rebuild(tfs_table* t, const double* strain, int64_t n, int mem, void* stream) {
  clear_error();
  NvtxRange nvtx("tfs_table_rebuild");
  TFS_CHECK(t && strain, TFS_ERR_INVALID_ARG, "null argument");
  TFS_CHECK(t->sft_plan, TFS_ERR_INVALID_ARG, "table was not made by tfs_build_sfts");
  TFS_CHECK(mem == TFS_MEM_HOST || mem == TFS_MEM_DEVICE, TFS_ERR_INVALID_ARG, "bad mem kind");
  const SftPlan* p = static_cast<const SftPlan*>(t->sft_plan);
  TFS_CHECK(n / p->L == t->n_seg, TFS_ERR_INVALID_ARG, "strain gives %lld segments, table has %lld",
            (long long)(n / p->L), (long long)t->n_seg);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double* d_x = strain;
  double* tmp = nullptr;
  const size_t xbytes = (size_t)t->n_seg * p->L * 8;
  cudaEvent_t copied = nullptr;  // host strain with a stream: wait for the upload only
  if (mem == TFS_MEM_HOST) {
    if (st != nullptr) TFS_CUDA(cudaEventCreateWithFlags(&copied, cudaEventDisableTiming));
    cudaError_t e = cudaMallocAsync((void**)&tmp, xbytes, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, strain, xbytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && copied) e = cudaEventRecord(copied, st);
    if (e != cudaSuccess) {
      if (copied) cudaEventDestroy(copied);
      if (tmp) cudaFreeAsync(tmp, st);
      cudaStreamSynchronize(st);
      return cuda_fail(e, "strain upload");
    }
    d_x = tmp;
  }
  int rc = run_sft(p, d_x, t, st);
  if (rc == TFS_OK) rc = wsum_refresh(t, st);  // window sums kept with the table follow its new values
  if (tmp) cudaFreeAsync(tmp, st);
  if (copied) {
    // the caller may reuse the host strain once it has been copied; the transform keeps
    // running on the stream
    const cudaError_t e = cudaEventSynchronize(copied);
    cudaEventDestroy(copied);
    if (rc == TFS_OK && e != cudaSuccess) rc = cuda_fail(e, "strain upload");
  }
  if (rc) return rc;
  if (st == nullptr) TFS_CUDA(cudaStreamSynchronize(st));
  return TFS_OK;
}

// ---------------------------------------------------------------- linear-chirp table
extern "C" int tfs_build_chirp_table(const double* strain, int64_t n, double dt, double T_sft, const double* psd,
                                     int mem, void* stream, tfs_ctable** out) {
  clear_error();
  NvtxRange nvtx("tfs_build_chirp_table");
  TFS_CHECK(strain && psd && out, TFS_ERR_INVALID_ARG, "null argument");
  TFS_CHECK(dt > 0 && T_sft > 0 && std::isfinite(dt) && std::isfinite(T_sft), TFS_ERR_INVALID_ARG,
            "dt and T_sft must be positive");
  TFS_CHECK(mem == TFS_MEM_HOST || mem == TFS_MEM_DEVICE, TFS_ERR_INVALID_ARG, "bad mem kind");
  const double Lf = T_sft / dt;
  const int64_t L = (int64_t)std::llround(Lf);
  TFS_CHECK(L >= 512 && L <= (1 << 20) && std::fabs(Lf - (double)L) <= 1e-9 * Lf, TFS_ERR_INVALID_ARG,
            "T_sft/dt must be an integer in [512, 2^20]");
  TFS_CHECK(L % 2 == 0 && smooth235(L), TFS_ERR_INVALID_ARG,
            "T_sft/dt = %lld must be even with prime factors 2, 3, 5 only", (long long)L);
  const int64_t n_seg = n / L;
  TFS_CHECK(n_seg >= 1 && n_seg <= 65535, TFS_ERR_INVALID_ARG, "need 1 <= n/L <= 65535 segments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SftPlan* plan = nullptr;
  int rc = make_sft_plan(L, dt, TFS_WINDOW_HANN, psd, mem, &plan);
  if (rc) return rc;
  tfs_ctable* t = new tfs_ctable();
  cudaGetDevice(&t->device);
  t->n_seg = n_seg;
  t->n_bin = L / 2 + 1;
  t->T_sft = T_sft;
  t->dt = dt;
  t->L = L;
  t->s_ref = plan->s_ref;
  t->wt = plan->wt;
  t->sft_plan = plan;
  cudaError_t e = cudaMalloc(&t->z, (size_t)n_seg * t->n_bin * sizeof(float2));
  if (e != cudaSuccess) {
    tfs_ctable_free(t);
    return cuda_fail(e, "chirp table");
  }
  const double* d_x = strain;
  double* tmp = nullptr;
  const size_t xbytes = (size_t)n_seg * L * 8;
  if (mem == TFS_MEM_HOST) {
    e = cudaMallocAsync((void**)&tmp, xbytes, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, strain, xbytes, cudaMemcpyHostToDevice, st);
    d_x = tmp;
  }
  rc = e == cudaSuccess ? run_sft_complex(plan, d_x, t, st) : cuda_fail(e, "strain upload");
  if (tmp) cudaFreeAsync(tmp, st);
  if (rc == TFS_OK) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "build_chirp_table");
  }
  if (rc) {
    tfs_ctable_free(t);
    return rc;
  }
  *out = t;
  return TFS_OK;
}

extern "C" int tfs_ctable_free(tfs_ctable* t) {
  if (!t) return TFS_OK;
  if (t->owns) {
    if (t->z) cudaFree(t->z);
    free_sft_plan(t->sft_plan);  // owns wt
  }
  delete t;
  return TFS_OK;
}

extern "C" int tfs_ctable_info(const tfs_ctable* t, int64_t* n_seg, int64_t* n_bin, double* T_sft, double* dt,
                               double* s_ref) {
  clear_error();
  TFS_CHECK(t, TFS_ERR_INVALID_ARG, "null table");
  if (n_seg) *n_seg = t->n_seg;
  if (n_bin) *n_bin = t->n_bin;
  if (T_sft) *T_sft = t->T_sft;
  if (dt) *dt = t->dt;
  if (s_ref) *s_ref = t->s_ref;
  return TFS_OK;
}

extern "C" int tfs_ctable_to_host(const tfs_ctable* t, float* z, float* wt) {
  clear_error();
  TFS_CHECK(t, TFS_ERR_INVALID_ARG, "null table");
  if (z) TFS_CUDA(cudaMemcpy(z, t->z, (size_t)t->n_seg * t->n_bin * sizeof(float2), cudaMemcpyDeviceToHost));
  if (wt) TFS_CUDA(cudaMemcpy(wt, t->wt, (size_t)t->n_bin * sizeof(float), cudaMemcpyDeviceToHost));
  return TFS_OK;
}
