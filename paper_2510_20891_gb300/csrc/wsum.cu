// Window sums of a power table: W_m[alpha][c] = sum_{j=-m..m} P[alpha][c + j] for every centre
// c whose window overlaps the table (c in [-m, n_bin - 1 + m]), elements outside [0, n_bin)
// counting 0 (paper Sec. II.B Eq. det_stat with +-m neighbours, nearest-bin reading).
//
// The statistic of a track is the sum over segments of W_m[alpha][b_alpha]: one gathered
// value per (track, segment) instead of 2m + 1.  The sums are formed in FP32 from the stored
// (dequantised) values in a fixed order, ((0 + P[c-m]) + P[c-m+1]) + ..., so every reader of
// a window sum (the staged gather of the statistic kernel and its FP64 fix-up path) sees the
// same value.  A table keeps one array per m that it was evaluated with (held by the table
// that owns the storage; views read their rows of it), rebuilt on the rebuild's stream
// whenever the table is recomputed from strain.
#include <algorithm>

#include "tfs_internal.cuh"

namespace tfs {

namespace {

template <int DT>
__device__ __forceinline__ float stored(const void* row, int k, float scale) {
  if (DT == TFS_F32) return static_cast<const float*>(row)[k];
  if (DT == TFS_BF16) return __bfloat162float(static_cast<const __nv_bfloat16*>(row)[k]);
  if (DT == TFS_F16) return __half2float(static_cast<const __half*>(row)[k]);
  return static_cast<float>(static_cast<const __nv_fp8_e4m3*>(row)[k]) * scale;
}

// One thread per output element: index i = c + m of rows blockIdx.y, blockIdx.y + gridDim.y, ...
template <int DT>
__global__ void wsum_kernel(const void* __restrict__ data, const float* __restrict__ scales, int n_seg, int n_bin,
                            int row_stride, int m, int pitch, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pitch) return;
  for (int seg = blockIdx.y; seg < n_seg; seg += gridDim.y) {
    const void* row = static_cast<const char*>(data) + (size_t)seg * row_stride * esize_of(DT);
    const float scale = DT == TFS_F8E4M3 ? scales[seg] : 1.f;
    float v = 0.f;
    if (i < n_bin + 2 * m) {
      const int c = i - m;
      for (int j = -m; j <= m; ++j) {
        const int k = c + j;
        v += (k >= 0 && k < n_bin) ? stored<DT>(row, k, scale) : 0.f;
      }
    }
    out[(size_t)seg * pitch + i] = v;
  }
}

int launch_wsum(const tfs_table* t, int m, int64_t pitch, float* out, cudaStream_t st) {
  dim3 grid((unsigned)((pitch + 255) / 256), (unsigned)std::min<int64_t>(t->n_seg, 65535));
  const int ns = (int)t->n_seg, nb = (int)t->n_bin, rs = (int)t->row_stride, p = (int)pitch;
  switch (t->dtype) {
    case TFS_F32: wsum_kernel<TFS_F32><<<grid, 256, 0, st>>>(t->data, t->scales, ns, nb, rs, m, p, out); break;
    case TFS_BF16: wsum_kernel<TFS_BF16><<<grid, 256, 0, st>>>(t->data, t->scales, ns, nb, rs, m, p, out); break;
    case TFS_F16: wsum_kernel<TFS_F16><<<grid, 256, 0, st>>>(t->data, t->scales, ns, nb, rs, m, p, out); break;
    case TFS_F8E4M3: wsum_kernel<TFS_F8E4M3><<<grid, 256, 0, st>>>(t->data, t->scales, ns, nb, rs, m, p, out); break;
    default: set_error("bad table dtype"); return TFS_ERR_INVALID_ARG;
  }
  count_launch();
  TFS_CUDA(cudaGetLastError());
  return TFS_OK;
}

const tfs_table* owner_of(const tfs_table* t) { return t->owner ? t->owner : t; }

}  // namespace

int64_t wsum_pitch(int64_t n_bin, int m) { return (n_bin + 2 * m + 31) / 32 * 32; }

int64_t wsum_bytes(const tfs_table* t, int m) {
  const tfs_table* o = owner_of(t);
  return o->n_seg * wsum_pitch(o->n_bin, m) * (int64_t)sizeof(float);
}

bool wsum_cached(const tfs_table* t, int m) {
  const tfs_table* o = owner_of(t);
  std::lock_guard<std::mutex> lk(o->wmu);
  for (const WSum& w : o->wsums)
    if (w.m == m) return true;
  return false;
}

int64_t wsum_cached_bytes(const tfs_table* t) {
  const tfs_table* o = owner_of(t);
  std::lock_guard<std::mutex> lk(o->wmu);
  int64_t b = 0;
  for (const WSum& w : o->wsums) b += w.bytes;
  return b;
}

int wsum_get(const tfs_table* t, int m, cudaStream_t st, const float** q, int* pitch) {
  tfs_table* o = const_cast<tfs_table*>(owner_of(t));
  TFS_CHECK(o->data, TFS_ERR_INVALID_ARG, "table has no device data");
  const int64_t seg0 = t->owner ? t->seg0 : 0;
  std::lock_guard<std::mutex> lk(o->wmu);
  for (const WSum& w : o->wsums)
    if (w.m == m) {
      *q = w.q + seg0 * w.pitch;
      *pitch = (int)w.pitch;
      return TFS_OK;
    }
  WSum w;
  w.m = m;
  w.pitch = wsum_pitch(o->n_bin, m);
  w.bytes = o->n_seg * w.pitch * (int64_t)sizeof(float);
  TFS_CHECK(w.pitch < (1 << 30), TFS_ERR_INVALID_ARG, "table row too wide");
  retain_pool_memory();
  TFS_CUDA(cudaMallocAsync((void**)&w.q, (size_t)w.bytes, st));
  int rc = launch_wsum(o, m, w.pitch, w.q, st);
  // one-off per (table, m): later calls may run on other streams without waiting for this one
  if (rc == TFS_OK) {
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "window sums");
  }
  if (rc) {
    cudaFreeAsync(w.q, st);
    return rc;
  }
  o->wsums.push_back(w);
  *q = w.q + seg0 * w.pitch;
  *pitch = (int)w.pitch;
  return TFS_OK;
}

int wsum_refresh(tfs_table* t, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(t->wmu);
  for (const WSum& w : t->wsums) {
    const int rc = launch_wsum(t, w.m, w.pitch, w.q, st);
    if (rc) return rc;
  }
  return TFS_OK;
}

// Work of any stream may still read the sums: wait for the device, then return them to the pool.
void wsum_free(tfs_table* t) {
  std::lock_guard<std::mutex> lk(t->wmu);
  if (t->wsums.empty()) return;
  cudaDeviceSynchronize();
  for (const WSum& w : t->wsums) cudaFreeAsync(w.q, 0);
  t->wsums.clear();
}

// The caller knows that nothing reads the sums any more (a served table with no request in
// flight): freed in the order of `st`, without waiting for the device.
void wsum_free_idle(tfs_table* t, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(t->wmu);
  for (const WSum& w : t->wsums) cudaFreeAsync(w.q, st);
  t->wsums.clear();
}

}  // namespace tfs
