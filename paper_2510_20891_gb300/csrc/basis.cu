// Track basis (paper Sec. II.C): the uncentred truncated SVD of training
// frequency tracks, f_{i,alpha} = sum_p U_{i,p} S_p V_{p,alpha}; the basis is
// the first K rows of V^T.
//
// Randomised range finder with power iterations (Halko, Martinsson & Tropp,
// SIAM Review 53 (2011), Algorithms 4.4 and 5.1): the products with the large
// M x n training matrix run as FP64 GPU kernels; the thin factors (M x b and
// n x b, b <= 128) are orthonormalised on the host by Gram-Schmidt applied
// twice, and the final small SVD is a one-sided (Hestenes) Jacobi iteration.
// The choice of K for a tolerance evaluates every candidate K's worst
// relative reconstruction error on the GPU.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "tfs_internal.cuh"

namespace tfs {

namespace {

// C[i][j] = sum_l A(i,l) B(l,j), A(i,l) = A[i*sa0 + l*sa1], B(l,j) = B[l*sb0 + j*sb1], C row-major [rows][cols]
__global__ void dgemm_strided(const double* __restrict__ A, long long sa0, long long sa1, const double* __restrict__ Bm,
                              long long sb0, long long sb1, double* __restrict__ C, int rows, int cols, int inner) {
  __shared__ double As[32][33];
  __shared__ double Bs[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 256 threads: ty in [0, 8)
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int l0 = 0; l0 < inner; l0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      const int i = i0 + r, l = l0 + tx;
      As[r][tx] = (i < rows && l < inner) ? A[i * sa0 + l * sa1] : 0.0;
      const int lb = l0 + r, j = j0 + tx;
      Bs[r][tx] = (lb < inner && j < cols) ? Bm[lb * sb0 + j * sb1] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int l = 0; l < 32; ++l) {
      const double b = Bs[l][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fma(As[ty + 8 * q][l], b, acc[q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + ty + 8 * q, j = j0 + tx;
    if (i < rows && j < cols) C[(size_t)i * cols + j] = acc[q];
  }
}

// For track i: err[i][k] = max_alpha |F - sum_{j<=k} C_ij V_j,alpha| / max_alpha |F|, k < b.
__global__ void recon_err(const double* __restrict__ F, const double* __restrict__ C, const double* __restrict__ V,
                          int M, int n, int b, double* __restrict__ err) {
  __shared__ double part[128];
  const int i = blockIdx.x;
  const int k = threadIdx.x;
  const double cik = (k < b) ? C[(size_t)i * b + k] : 0.0;
  double emax = 0.0, fmax_ = 0.0;
  for (int a = 0; a < n; ++a) {
    part[k] = (k < b) ? cik * V[(size_t)k * n + a] : 0.0;
    __syncthreads();
    for (int o = 1; o < 128; o <<= 1) {  // inclusive prefix sum over k
      const double add = k >= o ? part[k - o] : 0.0;
      __syncthreads();
      part[k] += add;
      __syncthreads();
    }
    const double f = F[(size_t)i * n + a];
    fmax_ = fmax(fmax_, fabs(f));
    emax = fmax(emax, fabs(f - part[k]));
    __syncthreads();
  }
  if (k < b) err[(size_t)i * b + k] = fmax_ > 0 ? emax / fmax_ : emax;
}

int gemm(const double* A, long long sa0, long long sa1, const double* Bm, long long sb0, long long sb1, double* C,
         int rows, int cols, int inner, cudaStream_t st) {
  dim3 g((cols + 31) / 32, (rows + 31) / 32);
  dgemm_strided<<<g, 256, 0, st>>>(A, sa0, sa1, Bm, sb0, sb1, C, rows, cols, inner);
  count_launch();
  TFS_CUDA(cudaGetLastError());
  return TFS_OK;
}

// counter-based standard normals: splitmix64 -> two uniforms -> Box-Muller
uint64_t splitmix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}
double normal_at(uint64_t i) {
  const double u1 = ((splitmix64(2 * i) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  const double u2 = ((splitmix64(2 * i + 1) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
}

// Orthonormalise the b columns of the row-major rows x b matrix X in place
// (classical Gram-Schmidt, applied twice per column; a column that vanishes
// is replaced by a fresh pseudo-random direction).
void orth_columns(std::vector<double>& X, int rows, int b, uint64_t seed) {
  std::vector<double> col(rows), dots(b);
  for (int j = 0; j < b; ++j) {
    for (int r = 0; r < rows; ++r) col[r] = X[(size_t)r * b + j];
    double n0 = 0;
    for (double v : col) n0 += v * v;
    n0 = std::sqrt(n0);
    for (int attempt = 0; attempt < 4; ++attempt) {
      for (int pass = 0; pass < 2; ++pass) {
        for (int q = 0; q < j; ++q) {
          double d = 0;
          for (int r = 0; r < rows; ++r) d += X[(size_t)r * b + q] * col[r];
          dots[q] = d;
        }
        for (int q = 0; q < j; ++q)
          for (int r = 0; r < rows; ++r) col[r] -= dots[q] * X[(size_t)r * b + q];
      }
      double nn = 0;
      for (double v : col) nn += v * v;
      nn = std::sqrt(nn);
      if (nn > 1e-12 * n0 && nn > 0) {
        for (int r = 0; r < rows; ++r) X[(size_t)r * b + j] = col[r] / nn;
        break;
      }
      for (int r = 0; r < rows; ++r) col[r] = normal_at(seed * 1000003ull + (uint64_t)j * 7919ull * rows + r + attempt * 104729ull);
      n0 = 0;
      for (double v : col) n0 += v * v;
      n0 = std::sqrt(n0);
    }
  }
}

// One-sided Jacobi on the columns of A (rows x b, row-major): on return the
// columns are orthogonal; sv[j] = column norms.
void hestenes(std::vector<double>& A, int rows, int b, std::vector<double>& sv) {
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < b - 1; ++p)
      for (int q = p + 1; q < b; ++q) {
        double al = 0, be = 0, ga = 0;
        for (int r = 0; r < rows; ++r) {
          const double x = A[(size_t)r * b + p], y = A[(size_t)r * b + q];
          al += x * x;
          be += y * y;
          ga += x * y;
        }
        if (ga == 0.0) continue;
        const double rel = std::fabs(ga) / std::sqrt(al * be);
        off = std::max(off, rel);
        if (rel < 1e-15) continue;
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
        for (int r = 0; r < rows; ++r) {
          const double x = A[(size_t)r * b + p], y = A[(size_t)r * b + q];
          A[(size_t)r * b + p] = c * x - s * y;
          A[(size_t)r * b + q] = s * x + c * y;
        }
      }
    if (off < 1e-15) break;
  }
  sv.assign(b, 0.0);
  for (int j = 0; j < b; ++j) {
    double nn = 0;
    for (int r = 0; r < rows; ++r) nn += A[(size_t)r * b + j] * A[(size_t)r * b + j];
    sv[j] = std::sqrt(nn);
  }
}

}  // namespace
}  // namespace tfs

using namespace tfs;

extern "C" int tfs_build_basis(const double* tracks, int64_t M, int64_t n_seg, int K, double tol, int mem,
                               void* stream, tfs_basis** out) {
  clear_error();
  NvtxRange nvtx("tfs_build_basis");
  TFS_CHECK(tracks && out, TFS_ERR_INVALID_ARG, "null argument");
  TFS_CHECK(M >= 1 && n_seg >= 1 && M <= (1 << 24) && n_seg <= (1 << 20), TFS_ERR_INVALID_ARG, "bad shape");
  TFS_CHECK(K >= 0 && K <= 32 && K <= std::min<int64_t>(M, n_seg), TFS_ERR_INVALID_ARG,
            "K must be in [0, min(M, n_seg, 32)]");
  TFS_CHECK(K > 0 || (tol > 0 && std::isfinite(tol)), TFS_ERR_INVALID_ARG, "K = 0 needs tol > 0");
  TFS_CHECK(mem == TFS_MEM_HOST || mem == TFS_MEM_DEVICE, TFS_ERR_INVALID_ARG, "bad mem kind");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n = (int)n_seg;
  const int Mi = (int)M;
  const int kmax = K > 0 ? K : 32;
  const int b = (int)std::min<int64_t>(std::min<int64_t>(M, n_seg), (int64_t)kmax + 10);
  const int q_iters = 3;

  double *dF = nullptr, *dO = nullptr, *dY = nullptr, *dZ = nullptr, *dC = nullptr, *dV = nullptr, *dE = nullptr;
  auto cleanup = [&]() {
    if (mem == TFS_MEM_HOST && dF) cudaFree(dF);
    for (double* p : {dO, dY, dZ, dC, dV, dE})
      if (p) cudaFree(p);
  };
  cudaError_t e = cudaSuccess;
#define TFS_B_TRY(x)            \
  do {                          \
    e = (x);                    \
    if (e != cudaSuccess) {     \
      cleanup();                \
      return cuda_fail(e, #x);  \
    }                           \
  } while (0)
#define TFS_B_RC(x)   \
  do {                \
    int rc_ = (x);    \
    if (rc_) {        \
      cleanup();      \
      return rc_;     \
    }                 \
  } while (0)
  if (mem == TFS_MEM_HOST) {
    TFS_B_TRY(cudaMalloc(&dF, (size_t)M * n * 8));
    TFS_B_TRY(cudaMemcpyAsync(dF, tracks, (size_t)M * n * 8, cudaMemcpyHostToDevice, st));
  } else {
    dF = const_cast<double*>(tracks);
  }
  TFS_B_TRY(cudaMalloc(&dO, (size_t)n * b * 8));
  TFS_B_TRY(cudaMalloc(&dY, (size_t)M * b * 8));
  TFS_B_TRY(cudaMalloc(&dZ, (size_t)n * b * 8));

  // Omega [n][b] standard normals
  std::vector<double> Om((size_t)n * b), Yh((size_t)M * b), Zh((size_t)n * b);
  for (size_t i = 0; i < Om.size(); ++i) Om[i] = normal_at(i);
  TFS_B_TRY(cudaMemcpyAsync(dO, Om.data(), Om.size() * 8, cudaMemcpyHostToDevice, st));
  // Y = F Omega
  TFS_B_RC(gemm(dF, n, 1, dO, b, 1, dY, Mi, b, n, st));
  TFS_B_TRY(cudaMemcpyAsync(Yh.data(), dY, Yh.size() * 8, cudaMemcpyDeviceToHost, st));
  TFS_B_TRY(cudaStreamSynchronize(st));
  orth_columns(Yh, Mi, b, 1);
  for (int it = 0; it < q_iters; ++it) {
    // Z = F^T Q, orthonormalise; Y = F Z, orthonormalise
    TFS_B_TRY(cudaMemcpyAsync(dY, Yh.data(), Yh.size() * 8, cudaMemcpyHostToDevice, st));
    TFS_B_RC(gemm(dF, 1, n, dY, b, 1, dZ, n, b, Mi, st));
    TFS_B_TRY(cudaMemcpyAsync(Zh.data(), dZ, Zh.size() * 8, cudaMemcpyDeviceToHost, st));
    TFS_B_TRY(cudaStreamSynchronize(st));
    orth_columns(Zh, n, b, 2 + it);
    TFS_B_TRY(cudaMemcpyAsync(dZ, Zh.data(), Zh.size() * 8, cudaMemcpyHostToDevice, st));
    TFS_B_RC(gemm(dF, n, 1, dZ, b, 1, dY, Mi, b, n, st));
    TFS_B_TRY(cudaMemcpyAsync(Yh.data(), dY, Yh.size() * 8, cudaMemcpyDeviceToHost, st));
    TFS_B_TRY(cudaStreamSynchronize(st));
    orth_columns(Yh, Mi, b, 100 + it);
  }
  // B^T = F^T Q  [n][b]; its one-sided Jacobi gives V Sigma
  TFS_B_TRY(cudaMemcpyAsync(dY, Yh.data(), Yh.size() * 8, cudaMemcpyHostToDevice, st));
  TFS_B_RC(gemm(dF, 1, n, dY, b, 1, dZ, n, b, Mi, st));
  TFS_B_TRY(cudaMemcpyAsync(Zh.data(), dZ, Zh.size() * 8, cudaMemcpyDeviceToHost, st));
  TFS_B_TRY(cudaStreamSynchronize(st));
  std::vector<double> sv;
  hestenes(Zh, n, b, sv);
  std::vector<int> order(b);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return sv[x] > sv[y]; });
  // V rows [b][n], sign-fixed (largest-magnitude entry positive)
  std::vector<double> V((size_t)b * n), sig(b);
  for (int r = 0; r < b; ++r) {
    const int j = order[r];
    sig[r] = sv[j];
    const double inv = sv[j] > 0 ? 1.0 / sv[j] : 0.0;
    int amax = 0;
    double vmax = -1.0;
    for (int a = 0; a < n; ++a) {
      const double v = Zh[(size_t)a * b + j] * inv;
      V[(size_t)r * n + a] = v;
      if (std::fabs(v) > vmax) {
        vmax = std::fabs(v);
        amax = a;
      }
    }
    if (V[(size_t)r * n + amax] < 0)
      for (int a = 0; a < n; ++a) V[(size_t)r * n + a] = -V[(size_t)r * n + a];
  }
  // projections C = F V^T [M][b] and (for K = 0) reconstruction errors per K
  TFS_B_TRY(cudaMalloc(&dV, (size_t)b * n * 8));
  TFS_B_TRY(cudaMalloc(&dC, (size_t)M * b * 8));
  TFS_B_TRY(cudaMemcpyAsync(dV, V.data(), V.size() * 8, cudaMemcpyHostToDevice, st));
  TFS_B_RC(gemm(dF, n, 1, dV, 1, n, dC, Mi, b, n, st));
  int Kf = K;
  if (K == 0) {
    TFS_B_TRY(cudaMalloc(&dE, (size_t)M * b * 8));
    recon_err<<<Mi, 128, 0, st>>>(dF, dC, dV, Mi, n, b, dE);
    count_launch();
    TFS_B_TRY(cudaGetLastError());
    std::vector<double> E((size_t)M * b);
    TFS_B_TRY(cudaMemcpyAsync(E.data(), dE, E.size() * 8, cudaMemcpyDeviceToHost, st));
    TFS_B_TRY(cudaStreamSynchronize(st));
    Kf = std::min(b, 32);
    for (int k = 0; k < std::min(b, 32); ++k) {
      double worst = 0;
      for (int i = 0; i < Mi; ++i) worst = std::max(worst, E[(size_t)i * b + k]);
      if (worst <= tol) {
        Kf = k + 1;
        break;
      }
    }
  }
  std::vector<double> Ch((size_t)M * b);
  TFS_B_TRY(cudaMemcpyAsync(Ch.data(), dC, Ch.size() * 8, cudaMemcpyDeviceToHost, st));
  TFS_B_TRY(cudaStreamSynchronize(st));
  tfs_basis* bs = new tfs_basis();
  cudaGetDevice(&bs->device);
  bs->K = Kf;
  bs->n_seg = n;
  bs->sigma.assign(sig.begin(), sig.begin() + Kf);
  bs->cmin.assign(Kf, INFINITY);
  bs->cmax.assign(Kf, -INFINITY);
  for (int i = 0; i < Mi; ++i)
    for (int k = 0; k < Kf; ++k) {
      const double c = Ch[(size_t)i * b + k];
      bs->cmin[k] = std::min(bs->cmin[k], c);
      bs->cmax[k] = std::max(bs->cmax[k], c);
    }
  e = cudaMalloc(&bs->U, (size_t)Kf * n * 8);
  if (e == cudaSuccess) e = cudaMemcpy(bs->U, V.data(), (size_t)Kf * n * 8, cudaMemcpyHostToDevice);
  cleanup();
#undef TFS_B_TRY
#undef TFS_B_RC
  if (e != cudaSuccess) {
    if (bs->U) cudaFree(bs->U);
    delete bs;
    return cuda_fail(e, "basis upload");
  }
  *out = bs;
  return TFS_OK;
}
