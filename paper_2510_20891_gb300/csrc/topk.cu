// Top-k selection over a float array (step 5 of the method: keep the best
// tracks, paper Sec. II.D).  Exact and deterministic: the k largest values,
// equal values ordered by lower index, -0.0 == +0.0, NaN below every number.
//
// Radix select on a monotone 32-bit key: four histogram passes of 8 bits
// each fix the k-th largest key K*; one counting pass and one scan give each
// chunk of the input the rank of its first element equal to K*, so the
// (k - #{key > K*}) lowest-indexed equal elements are taken; a bitonic sort
// of the <= 1024 selected (key, index) pairs orders the output.
#include "tfs_internal.cuh"

namespace tfs {

namespace {

constexpr int kChunk = 4096;     // elements per chunk in the counting / collecting passes
constexpr int kChunkThreads = 256;
constexpr int kPer = kChunk / kChunkThreads;

struct TopkState {
  uint32_t prefix, mask, krem, ngt;
};

__device__ __forceinline__ uint32_t mono_key(float v) {
  if (v != v) return 0u;  // NaN: lowest
  uint32_t u = __float_as_uint(v);
  if (u == 0x80000000u) u = 0u;  // -0.0 == +0.0
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void topk_init(TopkState* s, uint32_t* hist, uint32_t k) {
  if (threadIdx.x == 0) {
    s->prefix = 0;
    s->mask = 0;
    s->krem = k;
    s->ngt = 0;
  }
  hist[threadIdx.x] = 0;
}

__global__ void topk_hist(const float* __restrict__ v, long long N, const TopkState* __restrict__ s,
                          uint32_t* __restrict__ hist, int shift) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t prefix = s->prefix, mask = s->mask;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const uint32_t key = mono_key(v[i]);
    if ((key & mask) == prefix) atomicAdd(&h[(key >> shift) & 255u], 1u);
  }
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

// one CTA of 256 threads: pick the digit that holds the k_rem-th largest key
__global__ void topk_select(TopkState* s, uint32_t* hist, int shift) {
  __shared__ uint32_t suf[257];
  const int d = threadIdx.x;
  suf[d] = hist[d];
  if (d == 0) suf[256] = 0;
  __syncthreads();
  // inclusive suffix sums (Hillis-Steele over 256 entries)
  for (int o = 1; o < 256; o <<= 1) {
    const uint32_t add = (d + o < 256) ? suf[d + o] : 0u;
    __syncthreads();
    suf[d] += add;
    __syncthreads();
  }
  const uint32_t krem = s->krem;
  const uint32_t above = suf[d + 1];  // keys with a larger digit
  __syncthreads();
  if (above < krem && krem <= suf[d]) {
    s->prefix |= (uint32_t)d << shift;
    s->mask |= 255u << shift;
    s->krem = krem - above;
  }
  hist[d] = 0;  // ready for the next pass
}

__global__ void topk_eqcount(const float* __restrict__ v, long long N, const TopkState* __restrict__ s,
                             uint32_t* __restrict__ cnt) {
  __shared__ uint32_t tot;
  if (threadIdx.x == 0) tot = 0;
  __syncthreads();
  const uint32_t kstar = s->prefix;
  const long long base = (long long)blockIdx.x * kChunk;
  uint32_t c = 0;
  for (int j = threadIdx.x; j < kChunk; j += blockDim.x) {
    const long long i = base + j;
    if (i < N && mono_key(v[i]) == kstar) ++c;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(&tot, c);
  __syncthreads();
  if (threadIdx.x == 0) cnt[blockIdx.x] = tot;
}

// exclusive scan of cnt[0..n) in place, one CTA of 1024 threads
__global__ void topk_scan(uint32_t* cnt, int n) {
  __shared__ uint32_t part[1024];
  const int per = (n + 1023) / 1024;
  const int b0 = threadIdx.x * per;
  uint32_t sum = 0;
  for (int i = 0; i < per; ++i)
    if (b0 + i < n) sum += cnt[b0 + i];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const uint32_t add = threadIdx.x >= o ? part[threadIdx.x - o] : 0u;
    __syncthreads();
    part[threadIdx.x] += add;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - sum;
  for (int i = 0; i < per; ++i)
    if (b0 + i < n) {
      const uint32_t c = cnt[b0 + i];
      cnt[b0 + i] = run;
      run += c;
    }
}

__global__ void topk_collect(const float* __restrict__ v, long long N, TopkState* s,
                             const uint32_t* __restrict__ eqbase, unsigned long long* __restrict__ cand, int k) {
  __shared__ uint32_t wsum[kChunkThreads / 32];
  const uint32_t kstar = s->prefix;
  const uint32_t need = s->krem;       // equal keys to take
  const uint32_t ngt = (uint32_t)k - need;
  const long long base = (long long)blockIdx.x * kChunk + (long long)threadIdx.x * kPer;
  // contiguous run of kPer elements per thread keeps index order within the chunk
  uint32_t myeq = 0;
  for (int j = 0; j < kPer; ++j) {
    const long long i = base + j;
    if (i < N && mono_key(v[i]) == kstar) ++myeq;
  }
  // exclusive block scan of myeq
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = myeq;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  uint32_t woff = 0;
  for (int w = 0; w < warp; ++w) woff += wsum[w];
  uint32_t rank = eqbase[blockIdx.x] + woff + x - myeq;
  for (int j = 0; j < kPer; ++j) {
    const long long i = base + j;
    if (i >= N) break;
    const uint32_t key = mono_key(v[i]);
    const unsigned long long comp = ((unsigned long long)key << 32) | (0xffffffffull - (unsigned long long)i);
    if (key > kstar) {
      const uint32_t pos = atomicAdd(&s->ngt, 1u);
      if (pos < ngt) cand[pos] = comp;
    } else if (key == kstar) {
      if (rank < need) cand[ngt + rank] = comp;
      ++rank;
    }
  }
}

// one CTA of 1024 threads: bitonic sort of the k candidates, descending
__global__ void topk_sort(const float* __restrict__ v, long long N, const unsigned long long* __restrict__ cand, int k,
                          int64_t* __restrict__ idx_out, float* __restrict__ val_out) {
  __shared__ unsigned long long a[1024];
  const int t = threadIdx.x;
  a[t] = t < k ? cand[t] : 0ull;
  __syncthreads();
  for (int size = 2; size <= 1024; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const int p = t ^ stride;
      if (p > t) {
        const bool desc = (t & size) == 0;
        const unsigned long long x = a[t], y = a[p];
        if (desc ? (x < y) : (x > y)) {
          a[t] = y;
          a[p] = x;
        }
      }
      __syncthreads();
    }
  }
  if (t < k) {
    const long long i = (long long)(0xffffffffull - (a[t] & 0xffffffffull));
    const bool ok = i >= 0 && i < N;  // every slot is written by construction; never read out of range
    idx_out[t] = ok ? i : -1;
    val_out[t] = ok ? v[i] : __int_as_float(0x7fc00000);
  }
}

}  // namespace

size_t topk_workspace_bytes(int64_t N) {
  const int64_t nch = (N + kChunk - 1) / kChunk;
  return 256 * 4 + 256 + (size_t)(nch > 0 ? nch : 1) * 4 + 1024 * 8 + 256;
}

int topk_device(const float* v, int64_t N, int k, int64_t* idx_out, float* val_out, void* ws, cudaStream_t st) {
  if (N <= 0 || k <= 0) return TFS_OK;
  char* w = static_cast<char*>(ws);
  uint32_t* hist = reinterpret_cast<uint32_t*>(w);
  TopkState* s = reinterpret_cast<TopkState*>(w + 1024);
  unsigned long long* cand = reinterpret_cast<unsigned long long*>(w + 1024 + 256);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(w + 1024 + 256 + 1024 * 8);
  const int nch = (int)((N + kChunk - 1) / kChunk);
  topk_init<<<1, 256, 0, st>>>(s, hist, (uint32_t)k);
  int grid = (int)std::min<int64_t>((N + 255) / 256, 152 * 8);
  for (int shift = 24; shift >= 0; shift -= 8) {
    topk_hist<<<grid, 256, 0, st>>>(v, N, s, hist, shift);
    topk_select<<<1, 256, 0, st>>>(s, hist, shift);
  }
  topk_eqcount<<<nch, kChunkThreads, 0, st>>>(v, N, s, cnt);
  topk_scan<<<1, 1024, 0, st>>>(cnt, nch);
  topk_collect<<<nch, kChunkThreads, 0, st>>>(v, N, s, cnt, cand, k);
  topk_sort<<<1, 1024, 0, st>>>(v, N, cand, k, idx_out, val_out);
  count_launch(13);
  TFS_CUDA(cudaGetLastError());
  return TFS_OK;
}

}  // namespace tfs

// ---------------------------------------------------------------- top-k without allocation
// Scratch for tfs_topk_noalloc: a file-scope device array sized for kNoAllocMaxN
// inputs, held by every device that loads the library until the process exits.
namespace tfs {
namespace {
constexpr int64_t kNoAllocMaxN = (int64_t)1 << 26;
constexpr size_t kNoAllocBytes = 256 * 4 + 256 + (size_t)((kNoAllocMaxN + 4095) / 4096) * 4 + 1024 * 8 + 256;
}  // namespace
}  // namespace tfs

static __device__ __align__(256) unsigned char g_topk_noalloc_ws[tfs::kNoAllocBytes];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[128] = {nullptr};  // device address of the array, per device ordinal
}  // namespace

extern "C" int tfs_topk_noalloc(const float* val_in, int64_t N, int k, int64_t* idx, float* val, void* stream) {
  using namespace tfs;
  clear_error();
  TFS_CHECK(val_in && idx && val, TFS_ERR_INVALID_ARG, "null argument");
  TFS_CHECK(N >= 1 && N <= kNoAllocMaxN, TFS_ERR_INVALID_ARG,
            "tfs_topk_noalloc handles 1 <= N <= %lld (got %lld)", (long long)kNoAllocMaxN, (long long)N);
  TFS_CHECK(k >= 1 && k <= 1024, TFS_ERR_INVALID_ARG, "k must be in [1, 1024]");
  TFS_CHECK(kNoAllocBytes >= topk_workspace_bytes(N), TFS_ERR_INVALID_ARG, "scratch too small");
  int dev = 0;
  TFS_CUDA(cudaGetDevice(&dev));
  TFS_CHECK(dev >= 0 && dev < 128, TFS_ERR_INVALID_ARG, "device ordinal out of range");
  void* ws = nullptr;
  {
    // one-time set-up per device, with that device current: the array's device address
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_topk_noalloc_ws);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(top-k scratch)");
      g_noalloc_ptr[dev] = p;
    }
    ws = g_noalloc_ptr[dev];
  }
  const int kk = (int)std::min<int64_t>(k, N);
  return topk_device(val_in, N, kk, idx, val, ws, static_cast<cudaStream_t>(stream));
}
