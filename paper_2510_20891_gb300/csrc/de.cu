// Track-space differential evolution without crossover (Sec. II.D, Eq. de_step): the
// proposal f_trial = f + F_DE (f_r1 - f_r2) for every walker and the greedy acceptance.
// Tracks are linear in the coefficients (f = f_ref + sum_k c_k U_k), so the proposal's
// projection back onto the basis through its pseudo-inverse is exactly
// c + F_DE (c_r1 - c_r2); both steps therefore run on the coefficients.  The random draws
// (r1, r2, F_DE) are inputs.
#include <cstdint>

#include "tfs_internal.cuh"

namespace tfs {
namespace {

__global__ void de_propose_kernel(const double* __restrict__ c, int64_t N, int K, const int32_t* __restrict__ r1,
                                  const int32_t* __restrict__ r2, const float* __restrict__ F,
                                  const double* __restrict__ lo, const double* __restrict__ hi,
                                  double* __restrict__ ct, int32_t* __restrict__ in_prior) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  const int64_t a = r1[t], b = r2[t];
  const double f = (double)F[t];
  int ok = 1;
  for (int k = 0; k < K; ++k) {
    // each operation rounded on its own (no contraction): c + F (c_r1 - c_r2)
    const double v = __dadd_rn(c[t * K + k], __dmul_rn(f, __dsub_rn(c[a * K + k], c[b * K + k])));
    ct[t * K + k] = v;
    ok &= (v >= lo[k] && v <= hi[k]) ? 1 : 0;
  }
  in_prior[t] = ok;
}

__global__ void de_accept_kernel(double* __restrict__ c, float* __restrict__ s, const double* __restrict__ ct,
                                 const float* __restrict__ st, const int32_t* __restrict__ in_prior, int64_t N,
                                 int K) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  if (in_prior[t] && st[t] > s[t]) {
    for (int k = 0; k < K; ++k) c[t * K + k] = ct[t * K + k];
    s[t] = st[t];
  }
}

}  // namespace
}  // namespace tfs

using namespace tfs;

extern "C" int tfs_de_propose(const double* c, int64_t N, int K, const int32_t* r1, const int32_t* r2, const float* F,
                              const double* lo, const double* hi, double* c_trial, int32_t* in_prior,
                              void* stream) {
  clear_error();
  TFS_CHECK(N >= 0 && N < ((int64_t)1 << 31), TFS_ERR_INVALID_ARG, "N must be in [0, 2^31)");
  TFS_CHECK(K >= 1 && K <= 32, TFS_ERR_INVALID_ARG, "K must be in [1, 32]");
  if (N == 0) return TFS_OK;
  TFS_CHECK(c && r1 && r2 && F && lo && hi && c_trial && in_prior, TFS_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  de_propose_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(c, N, K, r1, r2, F, lo, hi, c_trial, in_prior);
  count_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TFS_OK : cuda_fail(e, "de_propose");
}

extern "C" int tfs_de_accept(double* c, float* s, const double* c_trial, const float* s_trial, const int32_t* in_prior,
                             int64_t N, int K, void* stream) {
  clear_error();
  TFS_CHECK(N >= 0 && N < ((int64_t)1 << 31), TFS_ERR_INVALID_ARG, "N must be in [0, 2^31)");
  TFS_CHECK(K >= 1 && K <= 32, TFS_ERR_INVALID_ARG, "K must be in [1, 32]");
  if (N == 0) return TFS_OK;
  TFS_CHECK(c && s && c_trial && s_trial && in_prior, TFS_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  de_accept_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(c, s, c_trial, s_trial, in_prior, N, K);
  count_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TFS_OK : cuda_fail(e, "de_accept");
}
