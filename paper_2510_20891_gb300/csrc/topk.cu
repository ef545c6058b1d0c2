// Top-k selection over a float array (step 5 of the method: keep the best
// tracks, paper Sec. II.D).  Exact and deterministic: the k largest values,
// equal values ordered by lower index, -0.0 == +0.0, NaN below every number.
//
// Radix select on a monotone 32-bit key: four histogram passes of 8 bits
// each fix the k-th largest key K* (the last CTA of each pass picks the digit).
// When every element equal to K* is among the k (the usual case: no tie at the
// boundary), one pass collects the k elements with key >= K*.  Otherwise one
// counting pass and one scan give each chunk of the input the rank of its
// first element equal to K*, so the (k - #{key > K*}) lowest-indexed equal
// elements are taken.  A bitonic sort of the <= 1024 selected (key, index)
// pairs orders the output.
#include "tfs_internal.cuh"

namespace tfs {

namespace {

constexpr int kChunk = 4096;     // elements per chunk in the counting / collecting passes
constexpr int kChunkThreads = 256;
constexpr int kPer = kChunk / kChunkThreads;

struct TopkState {
  uint32_t prefix, mask, krem, ngt;
  uint32_t done;  // CTAs of the current histogram pass that have merged their counts
  uint32_t fast;  // every element equal to K* is taken: no ordering among them is needed
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
    s->done = 0;
    s->fast = 0;
  }
  hist[threadIdx.x] = 0;
}

// After a CTA has added its counts to `hist`: the last CTA of the pass (of `n_cta`) picks the digit
// that holds the k_rem-th largest key, records whether all keys equal to K* are taken (last pass),
// and clears the histogram and the counter for the next pass.  256 threads.
__device__ void merge_done_select(TopkState* s, uint32_t* hist, int shift, unsigned n_cta) {
  __shared__ uint32_t suf[257];
  __shared__ bool last;
  __threadfence();  // this thread's histogram atomics before the counter
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&s->done, 1u) == n_cta - 1u;
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int d = threadIdx.x;
  suf[d] = __ldcg(&hist[d]);
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
    // in the last pass suf[d] - above keys equal K*: all of them are taken when that is k_rem
    if (shift == 0) s->fast = suf[d] == krem ? 1u : 0u;
  }
  hist[d] = 0;  // ready for the next pass
  if (d == 0) s->done = 0;
}

// 256 threads per CTA; the pass's last CTA selects the digit
__global__ void topk_hist(const float* __restrict__ v, long long N, TopkState* s, uint32_t* hist, int shift) {
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
  merge_done_select(s, hist, shift, gridDim.x);
}

__global__ void topk_eqcount(const float* __restrict__ v, long long N, const TopkState* __restrict__ s,
                             uint32_t* __restrict__ cnt) {
  __shared__ uint32_t tot;
  if (s->fast) return;  // the collecting pass needs no ranks
  if (threadIdx.x == 0) tot = 0;
  __syncthreads();
  const uint32_t kstar = s->prefix;
  const long long base = (long long)blockIdx.x * kChunk;
  uint32_t c = 0;
  for (int j = threadIdx.x; j < kChunk; j += kChunkThreads) {
    const long long i = base + j;
    if (i < N && mono_key(v[i]) == kstar) ++c;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(&tot, c);
  __syncthreads();
  if (threadIdx.x == 0) cnt[blockIdx.x] = tot;
}

// exclusive scan of cnt[0..n) in place, one CTA of 1024 threads
__global__ void topk_scan(const TopkState* s, uint32_t* cnt, int n) {
  __shared__ uint32_t part[1024];
  if (s->fast) return;
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
  if (s->fast) {
    // exactly k keys are >= K*: take them in any order (the sort orders them)
    for (int t = threadIdx.x; t < kChunk; t += kChunkThreads) {
      const long long i = (long long)blockIdx.x * kChunk + t;
      if (i >= N) break;
      const uint32_t key = mono_key(v[i]);
      if (key >= kstar) {
        const uint32_t pos = atomicAdd(&s->ngt, 1u);
        if (pos < (uint32_t)k) cand[pos] = ((unsigned long long)key << 32) | (0xffffffffull - (unsigned long long)i);
      }
    }
    return;
  }
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
  int kp = 1;
  while (kp < k) kp <<= 1;
  __syncthreads();
  for (int size = 2; size <= kp; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const int p = t ^ stride;
      if (p > t && p < kp) {
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
  for (int shift = 24; shift >= 0; shift -= 8) topk_hist<<<grid, 256, 0, st>>>(v, N, s, hist, shift);
  topk_eqcount<<<nch, kChunkThreads, 0, st>>>(v, N, s, cnt);
  topk_scan<<<1, 1024, 0, st>>>(s, cnt, nch);
  topk_collect<<<nch, kChunkThreads, 0, st>>>(v, N, s, cnt, cand, k);
  topk_sort<<<1, 1024, 0, st>>>(v, N, cand, k, idx_out, val_out);
  count_launch(9);
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

// ---------------------------------------------------------------- segmented top-k over many jobs
// The same selection for up to kTkJobs independent arrays at once (the per-chunk top-k of a batched
// statistic launch, paper Sec. II.D keeping the best walkers of every chunk): every pass covers all
// jobs, so a batch takes 9 launches whatever its number of jobs, and each job's result is that of
// topk_device on the job alone (same passes, same order), bit for bit.
namespace tfs {
namespace {

struct TkJob {
  const float* v;
  long long N;
  int64_t* idx;
  float* val;
  int k;
  int nch;  // chunks of kChunk elements
};
struct TkArgs {
  TkJob jobs[kTkJobs];
  long long chunk0[kTkJobs + 1];  // first chunk of each job in the flattened chunk list
  int n;
  // scratch: hist [n][256], state [n], cand [n][1024], cnt [total chunks]
  uint32_t* hist;
  TopkState* state;
  unsigned long long* cand;
  uint32_t* cnt;
};

__device__ __forceinline__ int tk_job_of(const TkArgs& a, long long chunk) {
  int lo = 0, hi = a.n - 1;  // the last job whose first chunk is <= chunk
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.chunk0[mid] <= chunk) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void tkb_init(const __grid_constant__ TkArgs a) {
  const int j = blockIdx.x;
  if (threadIdx.x == 0) {
    TopkState& s = a.state[j];
    s.prefix = 0;
    s.mask = 0;
    s.krem = (uint32_t)a.jobs[j].k;
    s.ngt = 0;
    s.done = 0;
    s.fast = 0;
  }
  a.hist[j * 256 + threadIdx.x] = 0;
}

// one CTA per chunk of one job (flattened over all jobs); the job's last CTA selects its digit
__global__ void tkb_hist(const __grid_constant__ TkArgs a, int shift) {
  __shared__ uint32_t h[256];
  const int j = tk_job_of(a, blockIdx.x);
  const TkJob& J = a.jobs[j];
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t prefix = a.state[j].prefix, mask = a.state[j].mask;
  const long long base = (long long)(blockIdx.x - a.chunk0[j]) * kChunk;
  for (int t = threadIdx.x; t < kChunk; t += kChunkThreads) {
    const long long i = base + t;
    if (i < J.N) {
      const uint32_t key = mono_key(J.v[i]);
      if ((key & mask) == prefix) atomicAdd(&h[(key >> shift) & 255u], 1u);
    }
  }
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(&a.hist[j * 256 + threadIdx.x], h[threadIdx.x]);
  merge_done_select(a.state + j, a.hist + j * 256, shift, (unsigned)J.nch);
}

__global__ void tkb_eqcount(const __grid_constant__ TkArgs a) {
  __shared__ uint32_t tot;
  const int j = tk_job_of(a, blockIdx.x);
  const TkJob& J = a.jobs[j];
  if (a.state[j].fast) return;  // the collecting pass needs no ranks
  if (threadIdx.x == 0) tot = 0;
  __syncthreads();
  const uint32_t kstar = a.state[j].prefix;
  const long long base = (long long)(blockIdx.x - a.chunk0[j]) * kChunk;
  uint32_t c = 0;
  for (int t = threadIdx.x; t < kChunk; t += kChunkThreads) {
    const long long i = base + t;
    if (i < J.N && mono_key(J.v[i]) == kstar) ++c;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(&tot, c);
  __syncthreads();
  if (threadIdx.x == 0) a.cnt[blockIdx.x] = tot;
}

// one CTA of 1024 threads per job: exclusive scan of the job's chunk counts
__global__ void tkb_scan(const __grid_constant__ TkArgs a) {
  __shared__ uint32_t part[1024];
  const int j = blockIdx.x;
  if (a.state[j].fast) return;
  uint32_t* cnt = a.cnt + a.chunk0[j];
  const int n = a.jobs[j].nch;
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

__global__ void tkb_collect(const __grid_constant__ TkArgs a) {
  __shared__ uint32_t wsum[kChunkThreads / 32];
  const int j = tk_job_of(a, blockIdx.x);
  const TkJob& J = a.jobs[j];
  TopkState* s = a.state + j;
  unsigned long long* cand = a.cand + (size_t)j * 1024;
  const uint32_t kstar = s->prefix;
  const long long chunk = blockIdx.x - a.chunk0[j];
  if (s->fast) {
    // exactly k keys are >= K*: take them in any order (the sort orders them)
    for (int t = threadIdx.x; t < kChunk; t += kChunkThreads) {
      const long long i = chunk * kChunk + t;
      if (i >= J.N) break;
      const uint32_t key = mono_key(J.v[i]);
      if (key >= kstar) {
        const uint32_t pos = atomicAdd(&s->ngt, 1u);
        if (pos < (uint32_t)J.k) cand[pos] = ((unsigned long long)key << 32) | (0xffffffffull - (unsigned long long)i);
      }
    }
    return;
  }
  const uint32_t need = s->krem;
  const uint32_t ngt = (uint32_t)J.k - need;
  const long long base = chunk * kChunk + (long long)threadIdx.x * kPer;
  uint32_t myeq = 0;
  for (int q = 0; q < kPer; ++q) {
    const long long i = base + q;
    if (i < J.N && mono_key(J.v[i]) == kstar) ++myeq;
  }
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
  uint32_t rank = a.cnt[blockIdx.x] + woff + x - myeq;
  for (int q = 0; q < kPer; ++q) {
    const long long i = base + q;
    if (i >= J.N) break;
    const uint32_t key = mono_key(J.v[i]);
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

// one CTA of 1024 threads per job: bitonic sort of its k candidates, descending
__global__ void tkb_sort(const __grid_constant__ TkArgs a) {
  __shared__ unsigned long long x[1024];
  const int j = blockIdx.x;
  const TkJob& J = a.jobs[j];
  const unsigned long long* cand = a.cand + (size_t)j * 1024;
  const int t = threadIdx.x;
  x[t] = t < J.k ? cand[t] : 0ull;
  int kp = 1;
  while (kp < J.k) kp <<= 1;
  __syncthreads();
  for (int size = 2; size <= kp; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const int p = t ^ stride;
      if (p > t && p < kp) {
        const bool desc = (t & size) == 0;
        const unsigned long long u = x[t], w = x[p];
        if (desc ? (u < w) : (u > w)) {
          x[t] = w;
          x[p] = u;
        }
      }
      __syncthreads();
    }
  }
  if (t < J.k) {
    const long long i = (long long)(0xffffffffull - (x[t] & 0xffffffffull));
    const bool ok = i >= 0 && i < J.N;
    J.idx[t] = ok ? i : -1;
    J.val[t] = ok ? J.v[i] : __int_as_float(0x7fc00000);
  }
}

}  // namespace

size_t topk_batch_workspace_bytes(const TopkTask* tasks, int n) {
  size_t chunks = 0;
  for (int i = 0; i < n; ++i) chunks += (size_t)((tasks[i].N + kChunk - 1) / kChunk);
  const size_t per_group = (size_t)kTkJobs * (256 * 4 + sizeof(TopkState) + 1024 * 8);
  return per_group + chunks * 4 + 256;
}

int topk_batch_device(const TopkTask* tasks, int n, void* ws, cudaStream_t st) {
  // groups of up to kTkJobs jobs; the scratch of one group is reused by the next (stream order)
  char* w = static_cast<char*>(ws);
  uint32_t* hist = reinterpret_cast<uint32_t*>(w);
  TopkState* state = reinterpret_cast<TopkState*>(w + (size_t)kTkJobs * 256 * 4);
  unsigned long long* cand =
      reinterpret_cast<unsigned long long*>(w + (size_t)kTkJobs * (256 * 4 + sizeof(TopkState)));
  uint32_t* cnt = reinterpret_cast<uint32_t*>(w + (size_t)kTkJobs * (256 * 4 + sizeof(TopkState) + 1024 * 8));
  int g0 = 0;
  while (g0 < n) {
    TkArgs a;
    a.n = 0;
    a.chunk0[0] = 0;
    a.hist = hist;
    a.state = state;
    a.cand = cand;
    a.cnt = cnt;
    int g = g0;
    for (; g < n && a.n < kTkJobs; ++g) {
      const TopkTask& T = tasks[g];
      if (T.N <= 0 || T.k <= 0) continue;
      TkJob& J = a.jobs[a.n];
      J.v = T.val;
      J.N = T.N;
      J.idx = T.idx_out;
      J.val = T.val_out;
      J.k = (int)std::min<int64_t>(T.k, T.N);
      J.nch = (int)((T.N + kChunk - 1) / kChunk);
      a.chunk0[a.n + 1] = a.chunk0[a.n] + J.nch;
      ++a.n;
    }
    g0 = g;
    if (a.n == 0) continue;
    const unsigned chunks = (unsigned)a.chunk0[a.n];
    tkb_init<<<a.n, 256, 0, st>>>(a);
    for (int shift = 24; shift >= 0; shift -= 8) tkb_hist<<<chunks, kChunkThreads, 0, st>>>(a, shift);
    tkb_eqcount<<<chunks, kChunkThreads, 0, st>>>(a);
    tkb_scan<<<a.n, 1024, 0, st>>>(a);
    tkb_collect<<<chunks, kChunkThreads, 0, st>>>(a);
    tkb_sort<<<a.n, 1024, 0, st>>>(a);
    count_launch(9);
    TFS_CUDA(cudaGetLastError());
  }
  return TFS_OK;
}

}  // namespace tfs
