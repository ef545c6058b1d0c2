// Track-space differential evolution without crossover (Sec. II.D, Eq. de_step): the
// proposal f_trial = f + F_DE (f_r1 - f_r2) for every walker and the greedy acceptance.
// Tracks are linear in the coefficients (f = f_ref + sum_k c_k U_k), so the proposal's
// projection back onto the basis through its pseudo-inverse is exactly
// c + F_DE (c_r1 - c_r2); both steps therefore run on the coefficients.  The random draws
// (r1, r2, F_DE) are inputs, or come from tfs_de_draw: the counter-based SplitMix64 generator
// (Steele, Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014)
// keyed by a seed and an iteration number kept on the device, so that a captured graph of one
// iteration draws afresh on every replay.
#include <algorithm>
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

// SplitMix64: the output for the state after `k` steps from `seed`, the golden-gamma increment
// added k times (mod 2^64) and the 64-bit finaliser applied.
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + k * kGamma;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Every block reads the iteration number and draws for its walkers; a second one-thread kernel
// advances the number afterwards (stream order), so that a replayed graph draws afresh each time.
__global__ void de_draw_kernel(uint64_t seed, const int32_t* __restrict__ iter, int64_t n, int W, float f_lo,
                               float f_hi, int32_t* __restrict__ r1, int32_t* __restrict__ r2, float* __restrict__ F) {
  const uint64_t it = (uint64_t)(uint32_t)iter[0];
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = 3u * (it * (uint64_t)n + (uint64_t)g);
    const uint64_t z0 = splitmix64_at(seed, k + 1u), z1 = splitmix64_at(seed, k + 2u), z2 = splitmix64_at(seed, k + 3u);
    const int64_t c0 = g - g % W, t = g % W;
    const int64_t a = 1 + (int64_t)(((z0 >> 32) * (uint64_t)(W - 1)) >> 32);  // 1 .. W-1
    int64_t b = 1 + (int64_t)(((z1 >> 32) * (uint64_t)(W - 2)) >> 32);        // 1 .. W-2, then skip a
    b += (b >= a) ? 1 : 0;
    r1[g] = (int32_t)(c0 + (t + a) % W);
    r2[g] = (int32_t)(c0 + (t + b) % W);
    const float u = (float)(uint32_t)(z2 >> 40) * 0x1p-24f;  // [0, 1), exact
    F[g] = __fadd_rn(f_lo, __fmul_rn(__fsub_rn(f_hi, f_lo), u));
  }
}
__global__ void de_advance_kernel(int32_t* __restrict__ iter) { iter[0] = (int32_t)((uint32_t)iter[0] + 1u); }
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

extern "C" int tfs_de_draw(uint64_t seed, int32_t* iter, int64_t n_chunks, int W, float f_lo, float f_hi, int32_t* r1,
                           int32_t* r2, float* F, void* stream) {
  clear_error();
  TFS_CHECK(W >= 3, TFS_ERR_INVALID_ARG, "need at least 3 walkers per chunk");
  TFS_CHECK(n_chunks >= 0 && n_chunks * (int64_t)W < ((int64_t)1 << 31), TFS_ERR_INVALID_ARG,
            "n_chunks * W must be in [0, 2^31)");
  TFS_CHECK(f_lo <= f_hi, TFS_ERR_INVALID_ARG, "f_lo must not exceed f_hi");
  TFS_CHECK(iter, TFS_ERR_INVALID_ARG, "null iteration counter");
  const int64_t n = n_chunks * (int64_t)W;
  TFS_CHECK(n == 0 || (r1 && r2 && F), TFS_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 1024));
  de_draw_kernel<<<blocks, 256, 0, st>>>(seed, iter, n, W, f_lo, f_hi, r1, r2, F);
  de_advance_kernel<<<1, 1, 0, st>>>(iter);
  count_launch(2);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TFS_OK : cuda_fail(e, "de_draw");
}
