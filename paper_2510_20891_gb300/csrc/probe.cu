// Measurement support: the device's L2 read bandwidth, measured the way the statistic kernel
// would use it (a buffer that stays in L2, read repeatedly with 16-byte loads that bypass L1).
// The statistic's one-year table fits in L2, so this is the roofline its gather is held to
// beside the HBM copy bandwidth.
#include <algorithm>
#include <cstdint>

#include "tfs_internal.cuh"

namespace tfs {
namespace {

__global__ void l2_read_kernel(const float4* __restrict__ p, size_t n4, int reps, float* __restrict__ out) {
  float acc = 0.f;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; ++r)
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
      const float4 v = __ldcg(p + i);
      acc += v.x + v.y + v.z + v.w;
    }
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;  // keeps the loads
}

}  // namespace
}  // namespace tfs

using namespace tfs;

extern "C" int tfs_measure_l2_read(int64_t buffer_bytes, int reps, double* gbs) {
  clear_error();
  TFS_CHECK(gbs && buffer_bytes >= (1 << 20) && buffer_bytes <= ((int64_t)1 << 30) && reps >= 1 && reps <= 1000,
            TFS_ERR_INVALID_ARG, "need 1 MB <= buffer_bytes <= 1 GB, 1 <= reps <= 1000");
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = std::max(1, n_sm) * 8, threads = 256;
  const size_t n4 = (size_t)buffer_bytes / 16;
  float4* p = nullptr;
  float* out = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaMalloc(&p, n4 * 16);
  if (e == cudaSuccess) e = cudaMalloc(&out, (size_t)blocks * threads * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(p, 0, n4 * 16);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  float ms = 0.f;
  if (e == cudaSuccess) {
    l2_read_kernel<<<blocks, threads>>>(p, n4, 2, out);  // warm: the buffer settles in L2
    count_launch();
    cudaEventRecord(a);
    l2_read_kernel<<<blocks, threads>>>(p, n4, reps, out);
    count_launch();
    cudaEventRecord(b);
    e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (p) cudaFree(p);
  if (out) cudaFree(out);
  if (e != cudaSuccess) return cuda_fail(e, "L2 read probe");
  *gbs = (double)n4 * 16.0 * reps / (ms / 1e3) / 1e9;
  return TFS_OK;
}
