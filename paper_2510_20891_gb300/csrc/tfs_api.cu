// C-ABI entry points of libtfstat: error model, table and basis handles,
// the statistic call (steps 3-5 of the method, paper Sec. II.B-II.D) and
// the stand-alone top-k.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "tfs_internal.cuh"

namespace tfs {

static thread_local char g_err[512] = "";
static std::atomic<long long> g_launches{0};
#ifdef TFS_DEBUG_CHECKS
static unsigned long long g_dbg_last[4] = {0, 0, 0, 0};
#endif
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
void clear_error() { g_err[0] = 0; }

int cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? TFS_ERR_OOM : TFS_ERR_CUDA;
}

// ---------------------------------------------------------------- tables
int alloc_table(int64_t n_seg, int64_t n_bin, int dtype, double T_sft, tfs_table** out) {
  tfs_table* t = new tfs_table();
  cudaGetDevice(&t->device);
  t->n_seg = n_seg;
  t->n_bin = n_bin;
  t->row_stride = ((n_bin + 31) / 32) * 32;
  t->dtype = dtype;
  t->T_sft = T_sft;
  const size_t bytes = (size_t)n_seg * t->row_stride * esize_of(dtype);
  cudaError_t e = cudaMalloc(&t->data, bytes);
  if (e != cudaSuccess) {
    delete t;
    return cuda_fail(e, "cudaMalloc(table)");
  }
  e = cudaMemset(t->data, 0, bytes);
  if (e == cudaSuccess && dtype == TFS_F8E4M3) {
    e = cudaMalloc(&t->scales, (size_t)n_seg * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(t->scales, 0, (size_t)n_seg * sizeof(float));
  }
  if (e != cudaSuccess) {
    cudaFree(t->data);
    if (t->scales) cudaFree(t->scales);
    delete t;
    return cuda_fail(e, "table allocation");
  }
  t->bytes = (int64_t)bytes + (t->scales ? n_seg * 4 : 0);
  *out = t;
  return TFS_OK;
}

// ---------------------------------------------------------------- basis segment parameters
// D_k,alpha = fl32(T U_k,alpha - T U_k,mid), and max_alpha |D|, max_alpha |U| per k (rounded up).
__global__ void segparams_kernel(const double* __restrict__ U, int K, int KP, int n_seg, int nsp, int mid,
                                 double T, float* __restrict__ segp, float* __restrict__ dmax,
                                 float* __restrict__ umax) {
  const int k = blockIdx.x;  // one CTA per padded coefficient slot
  __shared__ float sd[32], su[32];
  float md = 0.f, mu = 0.f;
  if (k < K) {
    const double wmid = T * U[(size_t)k * n_seg + mid];
    for (int a = threadIdx.x; a < n_seg; a += blockDim.x) {
      const double u = U[(size_t)k * n_seg + a];
      const double dd = __dsub_rn(__dmul_rn(T, u), wmid);
      const float df = (float)dd;
      segp[(size_t)a * nsp + k] = df;
      md = fmaxf(md, fabsf(df));
      mu = fmaxf(mu, __double2float_ru(fabs(u)));
    }
  } else {
    for (int a = threadIdx.x; a < n_seg; a += blockDim.x) segp[(size_t)a * nsp + k] = 0.f;
  }
  for (int o = 16; o > 0; o >>= 1) {
    md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
    mu = fmaxf(mu, __shfl_xor_sync(0xffffffffu, mu, o));
  }
  if ((threadIdx.x & 31) == 0) {
    sd[threadIdx.x >> 5] = md;
    su[threadIdx.x >> 5] = mu;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      md = fmaxf(md, sd[w]);
      mu = fmaxf(mu, su[w]);
    }
    md = fmaxf(md, sd[0]);
    mu = fmaxf(mu, su[0]);
    dmax[k] = md * (1.0f + 1.0f / 1048576.0f);
    umax[k] = mu * (1.0f + 1.0f / 1048576.0f);
  }
}

// Segment-cut forms per (k, alpha): E = (T/6) x the second difference of U_k (the nearest
// inner value at the ends, 0 below three segments) and G = the first difference of U_k over
// the segment spacing (central inside, one-sided at the ends, 0 for one segment), both
// computed in FP64 and stored in FP32 at columns KP + k and 2 KP + k; max |E|, max |G| per k.
__global__ void cutparams_kernel(const double* __restrict__ U, int K, int KP, int n_seg, int nsp, double T,
                                 float* __restrict__ segp, float* __restrict__ emax, float* __restrict__ gmax) {
  const int k = blockIdx.x;
  __shared__ float se[32], sg[32];
  float me = 0.f, mg = 0.f;
  const double* u = U + (size_t)k * n_seg;
  for (int a = threadIdx.x; a < n_seg; a += blockDim.x) {
    double e = 0.0, g = 0.0;
    if (k < K) {
      if (n_seg >= 3) {
        const int c = a == 0 ? 1 : (a == n_seg - 1 ? n_seg - 2 : a);
        e = __dmul_rn(__dadd_rn(__dsub_rn(u[c + 1], __dmul_rn(2.0, u[c])), u[c - 1]), T / 6.0);
      }
      if (n_seg >= 2) {
        if (a == 0) g = __dsub_rn(u[1], u[0]) / T;
        else if (a == n_seg - 1) g = __dsub_rn(u[n_seg - 1], u[n_seg - 2]) / T;
        else g = __dsub_rn(u[a + 1], u[a - 1]) / (2.0 * T);
      }
    }
    const float ef = (float)e, gf = (float)g;
    float* row = segp + (size_t)a * nsp + cut_col(KP) + 4 * k;
    row[0] = ef;
    row[1] = ef;
    row[2] = gf;
    row[3] = gf;
    me = fmaxf(me, fabsf(ef));
    mg = fmaxf(mg, fabsf(gf));
  }
  for (int o = 16; o > 0; o >>= 1) {
    me = fmaxf(me, __shfl_xor_sync(0xffffffffu, me, o));
    mg = fmaxf(mg, __shfl_xor_sync(0xffffffffu, mg, o));
  }
  if ((threadIdx.x & 31) == 0) {
    se[threadIdx.x >> 5] = me;
    sg[threadIdx.x >> 5] = mg;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      me = fmaxf(me, se[w]);
      mg = fmaxf(mg, sg[w]);
    }
    emax[k] = me * (1.0f + 1.0f / 1048576.0f);
    gmax[k] = mg * (1.0f + 1.0f / 1048576.0f);
  }
}

int pick_kp(int K) {
  const int opts[] = {2, 4, 6, 8, 16, 32};
  for (int v : opts)
    if (K <= v) return v;
  return -1;
}

static void free_segparams(SegParams* s) {
  if (!s) return;
  if (s->segp) cudaFree(s->segp);
  if (s->dmax) cudaFree(s->dmax);
  if (s->umax) cudaFree(s->umax);
  if (s->emax) cudaFree(s->emax);
  if (s->gmax) cudaFree(s->gmax);
  delete s;
}

int get_segparams(tfs_basis* b, double T, int kp_min, cudaStream_t st, SegParams** out, int cuts) {
  std::lock_guard<std::mutex> lk(b->mu);
  const int KP = pick_kp(std::max(b->K, kp_min));
  TFS_CHECK(KP > 0, TFS_ERR_INVALID_ARG, "basis size K=%d exceeds 32", std::max(b->K, kp_min));
  cuts = cuts ? 1 : 0;
  for (SegParams* s : b->sps)
    if (s->T == T && s->KP == KP && s->cuts == cuts) {
      *out = s;
      return TFS_OK;
    }
  SegParams* s = new SegParams();
  s->T = T;
  s->KP = KP;
  s->cuts = cuts;
  s->nsp = segrow_floats(KP, cuts != 0);
  s->alpha_mid = (int)(b->n_seg / 2);
  cudaError_t e = cudaMalloc(&s->segp, (size_t)b->n_seg * s->nsp * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&s->dmax, 32 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&s->umax, 32 * sizeof(float));
  if (e == cudaSuccess) e = cudaMemsetAsync(s->segp, 0, (size_t)b->n_seg * s->nsp * sizeof(float), st);
  if (e == cudaSuccess) {
    segparams_kernel<<<KP, 256, 0, st>>>(b->U, b->K, KP, (int)b->n_seg, s->nsp, s->alpha_mid, T, s->segp,
                                         s->dmax, s->umax);
    count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && cuts) {
    e = cudaMalloc(&s->emax, 32 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&s->gmax, 32 * sizeof(float));
    if (e == cudaSuccess) {
      cutparams_kernel<<<KP, 256, 0, st>>>(b->U, b->K, KP, (int)b->n_seg, s->nsp, T, s->segp, s->emax, s->gmax);
      count_launch();
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // one-off per (basis, T, KP): later calls may use other streams
  if (e != cudaSuccess) {
    free_segparams(s);
    return cuda_fail(e, "segment parameters");
  }
  b->sps.push_back(s);
  *out = s;
  return TFS_OK;
}

// ---------------------------------------------------------------- launch tuning
// Launch shapes chosen by tfs_autotune_batch, keyed by what decides them: table dtype,
// coefficient slots, the widest row and the longest job (powers of two), single job or batch.
static std::mutex g_tune_mu;
static std::map<std::string, tfs_tuning> g_tune;
thread_local const EvalTuning* g_force_tuning = nullptr;  // set while the tuner times a candidate

static int ceil_log2(int64_t x) {
  int k = 0;
  while (((int64_t)1 << k) < x) ++k;
  return k;
}

static std::string tuning_key(int dtype, int KP, int64_t row_max, int64_t seg_max, bool multi) {
  char buf[96];
  snprintf(buf, sizeof(buf), "%d:%d:%d:%d:%d", dtype, KP, ceil_log2(row_max), ceil_log2(seg_max), multi ? 1 : 0);
  return buf;
}

static std::string launch_key(const EvalLaunch& L) {
  int KP = 0;
  int64_t row_max = 1, seg_max = 1;
  for (int i = 0; i < L.n_jobs; ++i) {
    KP = std::max(KP, L.jobs[i].sp->KP);
    row_max = std::max<int64_t>(row_max, L.jobs[i].table->row_stride);
    seg_max = std::max<int64_t>(seg_max, L.jobs[i].table->n_seg);
  }
  std::string k = tuning_key(L.jobs[0].table->dtype, KP, row_max, seg_max, L.n_jobs > 1);
  if (L.jobs[0].cuts) k += ":c";
  return k;
}

static std::vector<std::string> g_last_keys;  // keys of the launches of the last tfs_eval_batch (tuner only)

int launch_eval(const EvalLaunch& L, const EvalTuning& tune_in, cudaStream_t st) {
  if (L.n_jobs <= 0) return TFS_OK;
  EvalTuning tune = tune_in;
  const std::string key = launch_key(L);
  if (g_force_tuning) {
    tune = *g_force_tuning;
    g_last_keys.push_back(key);
  } else if (tune.cap == 0 && tune.tile_div == 0 && tune.slots == 0 && tune.group == 0 && tune.rsel == 0) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      tune.cap = it->second.pcap;
      tune.tile_div = it->second.tile_div;
      tune.slots = it->second.slots;
      tune.group = it->second.group;
      tune.rsel = it->second.tile_class;
    }
  }
  return launch_eval_shape(L, tune, st);
}

// Stream-ordered scratch comes from the device's default memory pool, which by default
// returns all freed memory to the system at every synchronisation, so that the next call
// maps its scratch afresh (hundreds of MB for host inputs).  Keep up to 8 GB reserved
// (never lowering a larger threshold set by the application).
void retain_pool_memory() {
  static std::mutex mu;
  static std::vector<int> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> lk(mu);
  if (std::find(done.begin(), done.end(), dev) != done.end()) return;
  done.push_back(dev);
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
  uint64_t cur = 0, want = (uint64_t)8 << 30;
  if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &cur) == cudaSuccess && cur < want)
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &want);
}

// A small device arena for one call: one cudaMallocAsync, freed stream-ordered.
struct Arena {
  char* base = nullptr;
  size_t used = 0, size = 0;
  cudaStream_t st = nullptr;
  ~Arena() {
    if (base) cudaFreeAsync(base, st);
  }
  int init(size_t bytes, cudaStream_t s) {
    st = s;
    size = bytes;
    if (bytes == 0) return TFS_OK;
    retain_pool_memory();
    TFS_CUDA(cudaMallocAsync((void**)&base, bytes, s));
    return TFS_OK;
  }
  template <class T>
  T* take(size_t n) {
    used = (used + 255) & ~(size_t)255;
    T* p = reinterpret_cast<T*>(base + used);
    used += n * sizeof(T);
    return p;
  }
};

static size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }


// Host inputs of tfs_eval_stat are uploaded in chunks on a side stream, each chunk
// evaluated by its own launch as soon as it has arrived, so that the upload of chunk c+1
// overlaps the statistic of chunk c.  A chunk is a whole number of rounds of full tiles
// over the SMs (so that the chunks' launches together take no more rounds than one launch
// over all the tracks), at least 64 MB of coefficients, at most 6 chunks (a launch costs about
// 0.1 ms of start-up and drain, partly hidden by alternating the launches over two streams:
// 10^7 one-year tracks from host buffers ran 3.91 ms per step in 4 chunks, 3.80 in 5 (3 rounds
// each, the most this cap allows), 3.92 in 8; 4.01 in 4 chunks on one stream).  Returns the
// tracks per chunk (N: no chunking).
static int64_t host_chunk_tracks(const EvalLaunch& L, int64_t N, int K) {
  int div = 1;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(launch_key(L));
    if (it != g_tune.end() && it->second.tile_div > 0) div = it->second.tile_div;
  }
  const int64_t round = eval_round_tracks(L.jobs[0].sp->KP, L.jobs[0].cuts != 0, div);
  const int64_t min_tracks = ((int64_t)64 << 20) / (8 * (int64_t)K);
  const int64_t r = std::max<int64_t>({1, (min_tracks + round - 1) / round, (N + 6 * round - 1) / (6 * round)});
  return r * round >= N ? N : r * round;
}

// Device memory allocated on one stream and freed on another (after its last use there).
struct CrossBuf {
  char* p = nullptr;
  cudaStream_t free_on = nullptr;
  int init(size_t bytes, cudaStream_t alloc_on, cudaStream_t free_st) {
    free_on = free_st;
    retain_pool_memory();
    TFS_CUDA(cudaMallocAsync((void**)&p, bytes, alloc_on));
    return TFS_OK;
  }
  ~CrossBuf() {
    if (p) cudaFreeAsync(p, free_on);
  }
};

// Side streams of one call, drained before the call's scratch is freed (declare after the
// Arena and any CrossBuf so that this is destroyed first) and on every early return.
struct SideStreams {
  cudaStream_t s[3] = {nullptr, nullptr, nullptr};
  std::vector<cudaEvent_t> ev;
  int init() {
    // created once per host thread and device and kept (creating three streams per call cost
    // 0.02 ms of the 3.8 ms host-input step); one thread's calls use them one call at a time.
    // A stream that no longer answers (a reset device) is made again.
    thread_local cudaStream_t cache[64][3] = {};
    int dev = 0;
    TFS_CUDA(cudaGetDevice(&dev));
    TFS_CHECK(dev >= 0 && dev < 64, TFS_ERR_INVALID_ARG, "device ordinal out of range");
    for (int i = 0; i < 3; ++i) {
      if (cache[dev][i]) {
        const cudaError_t q = cudaStreamQuery(cache[dev][i]);
        if (q != cudaSuccess && q != cudaErrorNotReady) {
          cudaGetLastError();
          cache[dev][i] = nullptr;
        }
      }
      if (!cache[dev][i]) TFS_CUDA(cudaStreamCreateWithFlags(&cache[dev][i], cudaStreamNonBlocking));
      s[i] = cache[dev][i];
    }
    return TFS_OK;
  }
  int event(cudaEvent_t* e) {
    TFS_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    ev.push_back(*e);
    return TFS_OK;
  }
  // `to` waits for the work enqueued so far on `from`
  int order(cudaStream_t from, cudaStream_t to) {
    cudaEvent_t e;
    int rc = event(&e);
    if (rc) return rc;
    TFS_CUDA(cudaEventRecord(e, from));
    TFS_CUDA(cudaStreamWaitEvent(to, e, 0));
    return TFS_OK;
  }
  ~SideStreams() {
    for (auto x : s)
      if (x) cudaStreamSynchronize(x);
    for (auto e : ev) cudaEventDestroy(e);
  }
};

}  // namespace tfs

using namespace tfs;

extern "C" {

int tfs_version(void) { return 10000; }

const char* tfs_last_error(void) { return tfs::g_err; }

int tfs_table_info(const tfs_table* t, int64_t* n_seg, int64_t* n_bin, int* dtype, double* T_sft,
                   int64_t* row_stride) {
  TFS_CHECK(t, TFS_ERR_INVALID_ARG, "null table");
  if (n_seg) *n_seg = t->n_seg;
  if (n_bin) *n_bin = t->n_bin;
  if (dtype) *dtype = t->dtype;
  if (T_sft) *T_sft = t->T_sft;
  if (row_stride) *row_stride = t->row_stride;
  return TFS_OK;
}

int64_t tfs_table_bytes(const tfs_table* t) { return t ? t->bytes + (t->owns ? wsum_cached_bytes(t) : 0) : 0; }

int tfs_set_wait_limit(int64_t limit_ns, int hold) {
  clear_error();
  TFS_CHECK(hold == 0 || hold == 1, TFS_ERR_INVALID_ARG, "hold must be 0 or 1");
  set_eval_wait(limit_ns > 0 ? (uint64_t)limit_ns : 2000000000ull, hold);
  return TFS_OK;
}

long long tfs_kernel_launches(void) { return tfs::g_launches.load(); }

#ifdef TFS_DEBUG_CHECKS
// Self-check record of the last statistic call (debug builds only): count, site, two values.
void tfs_debug_last(unsigned long long* out) {
  for (int i = 0; i < 4; ++i) out[i] = tfs::g_dbg_last[i];
}
#endif

int tfs_table_free(tfs_table* t) {
  if (!t) return TFS_OK;
  if (t->sft_plan) free_sft_plan(t->sft_plan);
  if (t->owns) {
    wsum_free(t);
    if (t->data) cudaFree(t->data);
    if (t->scales) cudaFree(t->scales);
  }
  delete t;
  return TFS_OK;
}

int tfs_table_view(const tfs_table* t, int64_t seg0, int64_t n_seg, tfs_table** out) {
  clear_error();
  TFS_CHECK(t && out, TFS_ERR_INVALID_ARG, "null argument");
  TFS_CHECK(t->data, TFS_ERR_INVALID_ARG, "table has no device data");
  TFS_CHECK(seg0 >= 0 && n_seg >= 1 && seg0 + n_seg <= t->n_seg, TFS_ERR_INVALID_ARG,
            "rows [%lld, %lld) outside the table's %lld", (long long)seg0, (long long)(seg0 + n_seg),
            (long long)t->n_seg);
  tfs_table* v = new tfs_table();
  v->device = t->device;
  v->n_seg = n_seg;
  v->n_bin = t->n_bin;
  v->row_stride = t->row_stride;
  v->dtype = t->dtype;
  v->T_sft = t->T_sft;
  v->dt = t->dt;
  v->data = static_cast<char*>(t->data) + (size_t)seg0 * t->row_stride * esize_of(t->dtype);
  v->scales = t->scales ? t->scales + seg0 : nullptr;
  v->bytes = 0;
  v->owns = false;
  v->owner = t->owner ? t->owner : t;
  v->seg0 = (t->owner ? t->seg0 : 0) + seg0;
  *out = v;
  return TFS_OK;
}

int tfs_basis_view(const tfs_basis* b, int64_t seg0, int64_t n_seg, tfs_basis** out) {
  clear_error();
  TFS_CHECK(b && out, TFS_ERR_INVALID_ARG, "null argument");
  TFS_CHECK(seg0 >= 0 && n_seg >= 1 && seg0 + n_seg <= b->n_seg, TFS_ERR_INVALID_ARG,
            "segments [%lld, %lld) outside the basis's %lld", (long long)seg0, (long long)(seg0 + n_seg),
            (long long)b->n_seg);
  tfs_basis* v = new tfs_basis();
  v->device = b->device;
  v->K = b->K;
  v->n_seg = n_seg;
  cudaError_t e = cudaMalloc(&v->U, (size_t)b->K * n_seg * sizeof(double));
  if (e == cudaSuccess)
    e = cudaMemcpy2D(v->U, (size_t)n_seg * sizeof(double), b->U + seg0, (size_t)b->n_seg * sizeof(double),
                     (size_t)n_seg * sizeof(double), (size_t)b->K, cudaMemcpyDeviceToDevice);
  if (e != cudaSuccess) {
    if (v->U) cudaFree(v->U);
    delete v;
    return cuda_fail(e, "basis view");
  }
  v->sigma = b->sigma;
  v->cmin = b->cmin;
  v->cmax = b->cmax;
  *out = v;
  return TFS_OK;
}

int tfs_basis_from_host(const double* U, int K, int64_t n_seg, tfs_basis** out) {
  clear_error();
  TFS_CHECK(U && out, TFS_ERR_INVALID_ARG, "null argument");
  TFS_CHECK(K >= 1 && K <= 32, TFS_ERR_INVALID_ARG, "K must be in [1, 32] (got %d)", K);
  TFS_CHECK(n_seg >= 1 && n_seg <= (1 << 24), TFS_ERR_INVALID_ARG, "bad n_seg");
  for (int64_t i = 0; i < (int64_t)K * n_seg; ++i)
    TFS_CHECK(std::isfinite(U[i]), TFS_ERR_INVALID_ARG, "basis has a non-finite entry");
  tfs_basis* b = new tfs_basis();
  cudaGetDevice(&b->device);
  b->K = K;
  b->n_seg = n_seg;
  cudaError_t e = cudaMalloc(&b->U, (size_t)K * n_seg * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(b->U, U, (size_t)K * n_seg * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (b->U) cudaFree(b->U);
    delete b;
    return cuda_fail(e, "basis upload");
  }
  b->sigma.assign(K, 0.0);
  b->cmin.assign(K, 0.0);
  b->cmax.assign(K, 0.0);
  *out = b;
  return TFS_OK;
}

int tfs_basis_info(const tfs_basis* b, int* K, int64_t* n_seg) {
  TFS_CHECK(b, TFS_ERR_INVALID_ARG, "null basis");
  if (K) *K = b->K;
  if (n_seg) *n_seg = b->n_seg;
  return TFS_OK;
}

int tfs_basis_to_host(const tfs_basis* b, double* U, double* sigma, double* cmin, double* cmax) {
  clear_error();
  TFS_CHECK(b, TFS_ERR_INVALID_ARG, "null basis");
  if (U) TFS_CUDA(cudaMemcpy(U, b->U, (size_t)b->K * b->n_seg * sizeof(double), cudaMemcpyDeviceToHost));
  for (int k = 0; k < b->K; ++k) {
    if (sigma) sigma[k] = b->sigma[k];
    if (cmin) cmin[k] = b->cmin[k];
    if (cmax) cmax[k] = b->cmax[k];
  }
  return TFS_OK;
}

int tfs_basis_free(tfs_basis* b) {
  if (!b) return TFS_OK;
  if (b->U) cudaFree(b->U);
  for (SegParams* s : b->sps) free_segparams(s);
  delete b;
  return TFS_OK;
}

int tfs_eval_stat(const tfs_table* table, const tfs_basis* basis_c, const double* coeffs, const double* f_ref,
                  int64_t N, int m, int topk, float* stat, int64_t* top_idx, float* top_val, tfs_tie_report* ties,
                  int mem, void* stream) {
  clear_error();
  NvtxRange nvtx("tfs_eval_stat");
  TFS_CHECK(table && basis_c, TFS_ERR_INVALID_ARG, "null table or basis");
  tfs_basis* basis = const_cast<tfs_basis*>(basis_c);
  TFS_CHECK(mem == TFS_MEM_HOST || mem == TFS_MEM_DEVICE, TFS_ERR_INVALID_ARG, "bad mem kind");
  TFS_CHECK(basis->n_seg == table->n_seg, TFS_ERR_INVALID_ARG,
            "basis has %lld segments, table %lld", (long long)basis->n_seg, (long long)table->n_seg);
  TFS_CHECK(N >= 0 && N < ((int64_t)1 << 40), TFS_ERR_INVALID_ARG, "bad N");
  TFS_CHECK(m >= 0 && m <= 64, TFS_ERR_INVALID_ARG, "m must be in [0, 64]");
  TFS_CHECK(topk >= 0 && topk <= 1024, TFS_ERR_INVALID_ARG, "topk must be in [0, 1024]");
  TFS_CHECK(N == 0 || coeffs, TFS_ERR_INVALID_ARG, "null coeffs");
  TFS_CHECK(stat || topk > 0 || N == 0, TFS_ERR_INVALID_ARG, "need stat or topk > 0");
  TFS_CHECK(topk == 0 || N == 0 || (top_idx && top_val), TFS_ERR_INVALID_ARG, "null top-k outputs");
  TFS_CHECK(topk == 0 || N < ((int64_t)1 << 31), TFS_ERR_INVALID_ARG, "top-k needs N < 2^31");
  TFS_CHECK(!ties || ties->capacity == 0 || (ties->track && ties->seg), TFS_ERR_INVALID_ARG,
            "tie report arrays missing");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int K = basis->K;
  const bool host = (mem == TFS_MEM_HOST);
  const int tie_cap = ties ? ties->capacity : 0;
  const int kk = (int)std::min<int64_t>(topk, N);

  SegParams* sp = nullptr;
  int rc = get_segparams(basis, table->T_sft, 0, st, &sp);
  if (rc) return rc;

  // host inputs go up in chunks (tie reports carry track indices of one launch: not with them)
  int64_t per = N;
  if (host && !ties && N > 0) {
    EvalJob J0{table, basis, sp, nullptr, nullptr, N, m, nullptr, nullptr};
    EvalLaunch L0{&J0, 1, nullptr, nullptr, nullptr, 0, nullptr};
    per = host_chunk_tracks(L0, N, K);
  }
  const bool chunked = per < N;
  const size_t up_bytes = host ? round256((size_t)N * K * 8) + (f_ref ? round256((size_t)N * 8) : 0) : 0;

  // one arena for everything this call needs on the device
  size_t need = 0;
  need += round256(sizeof(unsigned long long)) + round256(sizeof(int));
  need += round256((size_t)std::max(tie_cap, 1) * 8) + round256((size_t)std::max(tie_cap, 1) * 4);
  if (host && !chunked) need += up_bytes;
  if (host || !stat) need += round256((size_t)N * 4);
  if (kk > 0) need += round256((size_t)kk * 12) + round256(topk_workspace_bytes(N));
  Arena ar;
  rc = ar.init(need, st);
  if (rc) return rc;
  unsigned long long* d_tc = ar.take<unsigned long long>(1);
  int* d_status = ar.take<int>(1);
  int64_t* d_tt = ar.take<int64_t>(std::max(tie_cap, 1));
  int* d_ts = ar.take<int>(std::max(tie_cap, 1));
  // chunked uploads: their buffer is allocated on side stream 0, so that they need not wait
  // for earlier work on `stream` (a table rebuild, say), and freed on `stream`
  CrossBuf upb;
  SideStreams side;
  double* up_c = nullptr;  // device copies of host inputs
  double* up_f = nullptr;
  if (chunked) {
    rc = side.init();
    if (rc) return rc;
    rc = upb.init(up_bytes, side.s[0], st);
    if (rc) return rc;
    up_c = reinterpret_cast<double*>(upb.p);
    if (f_ref) up_f = reinterpret_cast<double*>(upb.p + round256((size_t)N * K * 8));
  } else if (host) {
    up_c = ar.take<double>((size_t)N * K);
    if (f_ref) up_f = ar.take<double>((size_t)N);
  }
  const double* d_c = host ? up_c : coeffs;
  const double* d_f = host ? up_f : f_ref;
  float* d_stat = (host || !stat) ? ar.take<float>((size_t)N) : stat;
  TFS_CUDA(cudaMemsetAsync(d_tc, 0, sizeof(unsigned long long), st));
  TFS_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), st));

  EvalJob J{table, basis, sp, d_c, d_f, N, m, d_stat, nullptr};
  EvalLaunch L{&J, 1, d_tc, d_tt, d_ts, tie_cap, d_status};
  if (!chunked) {
    if (host) {
      TFS_CUDA(cudaMemcpyAsync(up_c, coeffs, (size_t)N * K * 8, cudaMemcpyHostToDevice, st));
      if (f_ref) TFS_CUDA(cudaMemcpyAsync(up_f, f_ref, (size_t)N * 8, cudaMemcpyHostToDevice, st));
    }
#ifdef TFS_DEBUG_CHECKS
    unsigned long long* d_dbg = nullptr;
    TFS_CUDA(cudaMallocAsync((void**)&d_dbg, 32, st));
    TFS_CUDA(cudaMemsetAsync(d_dbg, 0, 32, st));
    L.dbg = d_dbg;
#endif
    rc = launch_eval(L, EvalTuning(), st);
    if (rc) return rc;
#ifdef TFS_DEBUG_CHECKS
    TFS_CUDA(cudaMemcpyAsync(g_dbg_last, d_dbg, 32, cudaMemcpyDeviceToHost, st));
    TFS_CUDA(cudaStreamSynchronize(st));
    cudaFreeAsync(d_dbg, st);
    TFS_CHECK(g_dbg_last[0] == 0, TFS_ERR_CUDA, "debug self-check failed %llu times, first at site %llu (%lld, %lld)",
              g_dbg_last[0], g_dbg_last[1], (long long)g_dbg_last[2], (long long)g_dbg_last[3]);
#endif
  } else {
    // uploads on side stream 0; the launches, each as soon as its chunk has arrived, alternate
    // between `stream` and side stream 2 (after everything enqueued on `stream` so far), so that
    // a launch's first tile and its last CTAs overlap its neighbours' (no CTA of the kernel waits
    // for another, so two launches may share the SMs in any way); the per-track values are read
    // back on side stream 1 as each launch ends.  The read-backs are enqueued after every upload
    // and launch: a copy into pageable memory returns only once it is done, and enqueued inside
    // the loop it would hold back the next chunk's upload.
    rc = side.order(st, side.s[2]);
    if (rc) return rc;
    std::vector<cudaEvent_t> ran;
    int ci = 0;
    for (int64_t t0 = 0; t0 < N; t0 += per, ++ci) {
      const int64_t n = std::min(per, N - t0);
      cudaStream_t xs = (ci & 1) ? side.s[2] : st;
      TFS_CUDA(cudaMemcpyAsync(up_c + t0 * K, coeffs + t0 * K, (size_t)n * K * 8,
                               cudaMemcpyHostToDevice, side.s[0]));
      if (f_ref)
        TFS_CUDA(cudaMemcpyAsync(up_f + t0, f_ref + t0, (size_t)n * 8, cudaMemcpyHostToDevice,
                                 side.s[0]));
      rc = side.order(side.s[0], xs);
      if (rc) return rc;
      EvalJob Jc{table, basis, sp, d_c + t0 * K, d_f ? d_f + t0 : nullptr, n, m, d_stat + t0, nullptr};
      EvalLaunch Lc{&Jc, 1, d_tc, d_tt, d_ts, 0, d_status};
      rc = launch_eval(Lc, EvalTuning(), xs);
      if (rc) return rc;
      if (stat) {
        cudaEvent_t e;
        rc = side.event(&e);
        if (rc) return rc;
        TFS_CUDA(cudaEventRecord(e, xs));
        ran.push_back(e);
      }
    }
    rc = side.order(side.s[2], st);
    if (rc) return rc;
    for (size_t c = 0; c < ran.size(); ++c) {
      const int64_t t0 = (int64_t)c * per, n = std::min(per, N - t0);
      TFS_CUDA(cudaStreamWaitEvent(side.s[1], ran[c], 0));
      TFS_CUDA(cudaMemcpyAsync(stat + t0, d_stat + t0, (size_t)n * 4, cudaMemcpyDeviceToHost, side.s[1]));
    }
    rc = side.order(side.s[1], st);
    if (rc) return rc;
  }

  int64_t* d_ti = nullptr;
  float* d_tv = nullptr;
  if (kk > 0) {
    d_ti = ar.take<int64_t>(kk);
    d_tv = ar.take<float>(kk);
    void* ws = ar.take<char>(topk_workspace_bytes(N));
    rc = topk_device(d_stat, N, kk, host ? d_ti : top_idx, host ? d_tv : top_val, ws, st);
    if (rc) return rc;
  }
  if (host) {
    if (stat && N > 0 && !chunked)
      TFS_CUDA(cudaMemcpyAsync(stat, d_stat, (size_t)N * 4, cudaMemcpyDeviceToHost, st));
    if (kk > 0) {
      TFS_CUDA(cudaMemcpyAsync(top_idx, d_ti, (size_t)kk * 8, cudaMemcpyDeviceToHost, st));
      TFS_CUDA(cudaMemcpyAsync(top_val, d_tv, (size_t)kk * 4, cudaMemcpyDeviceToHost, st));
    }
  }
  const bool wait = host || ties || st == nullptr;
  int h_status = 0;
  if (wait) {
    TFS_CUDA(cudaMemcpyAsync(&h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    unsigned long long tc = 0;
    if (ties) TFS_CUDA(cudaMemcpyAsync(&tc, d_tc, sizeof(tc), cudaMemcpyDeviceToHost, st));
    TFS_CUDA(cudaStreamSynchronize(st));
    if (ties) {
      ties->count = (int64_t)tc;
      ties->n_stored = (int32_t)std::min<unsigned long long>(tc, (unsigned long long)tie_cap);
      if (ties->n_stored > 0) {
        TFS_CUDA(cudaMemcpy(ties->track, d_tt, (size_t)ties->n_stored * 8, cudaMemcpyDeviceToHost));
        TFS_CUDA(cudaMemcpy(ties->seg, d_ts, (size_t)ties->n_stored * 4, cudaMemcpyDeviceToHost));
      }
    }
    TFS_CHECK(h_status == 0, TFS_ERR_TIMEOUT, "a bounded device wait gave up (status %d)", h_status);
  }
  return TFS_OK;
}

int tfs_eval_bins(const tfs_table* table, const tfs_basis* basis_c, const double* coeffs, const double* f_ref,
                  int64_t N, int m, int32_t* bins, int mem, void* stream) {
  clear_error();
  TFS_CHECK(table && basis_c && bins && (coeffs || N == 0), TFS_ERR_INVALID_ARG, "null argument");
  tfs_basis* basis = const_cast<tfs_basis*>(basis_c);
  TFS_CHECK(mem == TFS_MEM_HOST || mem == TFS_MEM_DEVICE, TFS_ERR_INVALID_ARG, "bad mem kind");
  TFS_CHECK(basis->n_seg == table->n_seg, TFS_ERR_INVALID_ARG, "basis and table segment counts differ");
  TFS_CHECK(N >= 0 && N * table->n_seg < ((int64_t)1 << 34), TFS_ERR_INVALID_ARG, "bad N");
  TFS_CHECK(m >= 0 && m <= 64, TFS_ERR_INVALID_ARG, "m must be in [0, 64]");
  if (N == 0) return TFS_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SegParams* sp = nullptr;
  int rc = get_segparams(basis, table->T_sft, 0, st, &sp);
  if (rc) return rc;
  const bool host = mem == TFS_MEM_HOST;
  const int K = basis->K;
  const size_t nb = (size_t)N * table->n_seg;
  Arena ar;
  size_t need = round256(8) + round256(4) + round256(8) + round256(4) + round256((size_t)N * 4);
  if (host) need += round256((size_t)N * K * 8) + round256((size_t)N * 8) + round256(nb * 4);
  rc = ar.init(need, st);
  if (rc) return rc;
  unsigned long long* d_tc = ar.take<unsigned long long>(1);
  int* d_status = ar.take<int>(1);
  int64_t* d_tt = ar.take<int64_t>(1);
  int* d_ts = ar.take<int>(1);
  float* d_stat = ar.take<float>(N);
  const double* d_c = coeffs;
  const double* d_f = f_ref;
  int* d_b = bins;
  if (host) {
    double* c = ar.take<double>((size_t)N * K);
    TFS_CUDA(cudaMemcpyAsync(c, coeffs, (size_t)N * K * 8, cudaMemcpyHostToDevice, st));
    d_c = c;
    if (f_ref) {
      double* f = ar.take<double>(N);
      TFS_CUDA(cudaMemcpyAsync(f, f_ref, (size_t)N * 8, cudaMemcpyHostToDevice, st));
      d_f = f;
    }
    d_b = ar.take<int>(nb);
  }
  TFS_CUDA(cudaMemsetAsync(d_tc, 0, 8, st));
  TFS_CUDA(cudaMemsetAsync(d_status, 0, 4, st));
  EvalJob J{table, basis, sp, d_c, d_f, N, m, d_stat, d_b};
  EvalLaunch L{&J, 1, d_tc, d_tt, d_ts, 0, d_status};
  rc = launch_eval(L, EvalTuning(), st);
  if (rc) return rc;
  if (host) TFS_CUDA(cudaMemcpyAsync(bins, d_b, nb * 4, cudaMemcpyDeviceToHost, st));
  int h_status = 0;
  TFS_CUDA(cudaMemcpyAsync(&h_status, d_status, 4, cudaMemcpyDeviceToHost, st));
  TFS_CUDA(cudaStreamSynchronize(st));
  TFS_CHECK(h_status == 0, TFS_ERR_TIMEOUT, "a bounded device wait gave up (status %d)", h_status);
  return TFS_OK;
}

int tfs_eval_batch(const tfs_job* jobs, int n_jobs, int* dev_status, void* stream) {
  clear_error();
  NvtxRange nvtx("tfs_eval_batch");
  TFS_CHECK(jobs && n_jobs >= 1 && n_jobs <= 4096, TFS_ERR_INVALID_ARG, "need 1 <= n_jobs <= 4096 jobs");
  for (int i = 0; i < n_jobs; ++i) {
    const tfs_job& j = jobs[i];
    TFS_CHECK(j.table && j.basis, TFS_ERR_INVALID_ARG, "job %d: null table or basis", i);
    TFS_CHECK(j.basis->n_seg == j.table->n_seg, TFS_ERR_INVALID_ARG, "job %d: basis and table segment counts differ",
              i);
    TFS_CHECK(j.N >= 0 && j.N < ((int64_t)1 << 31), TFS_ERR_INVALID_ARG, "job %d: N must be in [0, 2^31)", i);
    TFS_CHECK(j.m >= 0 && j.m <= 64, TFS_ERR_INVALID_ARG, "job %d: m must be in [0, 64]", i);
    TFS_CHECK(j.topk >= 0 && j.topk <= 1024, TFS_ERR_INVALID_ARG, "job %d: topk must be in [0, 1024]", i);
    TFS_CHECK(j.N == 0 || j.coeffs, TFS_ERR_INVALID_ARG, "job %d: null coeffs", i);
    TFS_CHECK(j.stat || j.topk > 0 || j.N == 0, TFS_ERR_INVALID_ARG, "job %d: need stat or topk > 0", i);
    TFS_CHECK(j.topk == 0 || j.N == 0 || (j.top_idx && j.top_val), TFS_ERR_INVALID_ARG, "job %d: null top-k outputs",
              i);
    TFS_CHECK(pick_kp(j.basis->K) > 0, TFS_ERR_INVALID_ARG, "job %d: basis size exceeds 32", i);
    TFS_CHECK((j.flags & ~TFS_JOB_SEGMENT_CUTS) == 0 && j.reserved == 0, TFS_ERR_INVALID_ARG,
              "job %d: unknown flags or nonzero reserved field", i);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // one launch per (table dtype, segment cuts), with the widest coefficient slot count among its jobs
  int kp_of[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
  auto cut_of = [&](int i) { return (jobs[i].flags & TFS_JOB_SEGMENT_CUTS) ? 1 : 0; };
  for (int i = 0; i < n_jobs; ++i) {
    int& kp = kp_of[jobs[i].table->dtype][cut_of(i)];
    kp = std::max(kp, pick_kp(jobs[i].basis->K));
  }
  std::vector<SegParams*> sps(n_jobs);
  for (int i = 0; i < n_jobs; ++i) {
    int rc = get_segparams(const_cast<tfs_basis*>(jobs[i].basis), jobs[i].table->T_sft,
                           kp_of[jobs[i].table->dtype][cut_of(i)], st, &sps[i], cut_of(i));
    if (rc) return rc;
  }
  size_t need = round256(8) + round256(4) + round256(8) + round256(4);
  std::vector<TopkTask> tasks;  // every job's top-k, selected together after the statistic
  for (int i = 0; i < n_jobs; ++i) {
    if (!jobs[i].stat) need += round256((size_t)jobs[i].N * 4);
    if (jobs[i].topk > 0 && jobs[i].N > 0)
      tasks.push_back(TopkTask{nullptr, jobs[i].N, (int)std::min<int64_t>(jobs[i].topk, jobs[i].N), jobs[i].top_idx,
                               jobs[i].top_val});
  }
  const size_t ws_max = tasks.empty() ? 0 : topk_batch_workspace_bytes(tasks.data(), (int)tasks.size());
  need += round256(ws_max);
  Arena ar;
  int rc = ar.init(need, st);
  if (rc) return rc;
  unsigned long long* d_tc = ar.take<unsigned long long>(1);
  int* d_status = dev_status ? dev_status : ar.take<int>(1);
  int64_t* d_tt = ar.take<int64_t>(1);
  int* d_ts = ar.take<int>(1);
  void* ws = ws_max ? ar.take<char>(ws_max) : nullptr;
  std::vector<EvalJob> ej(n_jobs);
  for (int i = 0; i < n_jobs; ++i) {
    const tfs_job& j = jobs[i];
    float* stat = j.stat ? j.stat : ar.take<float>((size_t)j.N);
    ej[i] = EvalJob{j.table, j.basis, sps[i], j.coeffs, j.f_ref, j.N, j.m, stat, nullptr, cut_of(i)};
  }
  TFS_CUDA(cudaMemsetAsync(d_tc, 0, 8, st));
  TFS_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), st));
  unsigned long long* d_dbg = nullptr;
#ifdef TFS_DEBUG_CHECKS
  TFS_CUDA(cudaMallocAsync((void**)&d_dbg, 32, st));
  TFS_CUDA(cudaMemsetAsync(d_dbg, 0, 32, st));
#endif
  for (int g = 0; g < 8; ++g) {
    const int dt = g >> 1, cu = g & 1;
    if (!kp_of[dt][cu]) continue;
    std::vector<EvalJob> group;
    for (int i = 0; i < n_jobs; ++i)
      if (jobs[i].table->dtype == dt && cut_of(i) == cu && jobs[i].N > 0) group.push_back(ej[i]);
    for (size_t g0 = 0; g0 < group.size(); g0 += kMaxJobs) {
      const int n = (int)std::min<size_t>(kMaxJobs, group.size() - g0);
      EvalLaunch L{group.data() + g0, n, d_tc, d_tt, d_ts, 0, d_status, d_dbg};
      rc = launch_eval(L, EvalTuning(), st);
      if (rc) return rc;
    }
  }
#ifdef TFS_DEBUG_CHECKS
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  TFS_CUDA(cudaStreamIsCapturing(st, &cap));
  if (cap != cudaStreamCaptureStatusNone) {
    cudaFreeAsync(d_dbg, st);  // inside a capture the self-check record cannot be read back
    g_dbg_last[0] = 0;
  } else {
    TFS_CUDA(cudaMemcpyAsync(g_dbg_last, d_dbg, 32, cudaMemcpyDeviceToHost, st));
    TFS_CUDA(cudaStreamSynchronize(st));
    cudaFreeAsync(d_dbg, st);
  }
  TFS_CHECK(g_dbg_last[0] == 0, TFS_ERR_CUDA, "debug self-check failed %llu times, first at site %llu (%lld, %lld)",
            g_dbg_last[0], g_dbg_last[1], (long long)g_dbg_last[2], (long long)g_dbg_last[3]);
#endif
  // every job's top-k in one set of passes (kTkJobs jobs per set)
  if (!tasks.empty()) {
    size_t ti = 0;
    for (int i = 0; i < n_jobs; ++i)
      if (jobs[i].topk > 0 && jobs[i].N > 0) tasks[ti++].val = ej[i].stat;
    rc = topk_batch_device(tasks.data(), (int)tasks.size(), ws, st);
    if (rc) return rc;
  }
  if (!dev_status) {
    int h_status = 0;
    TFS_CUDA(cudaMemcpyAsync(&h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    TFS_CUDA(cudaStreamSynchronize(st));
    TFS_CHECK(h_status == 0, TFS_ERR_TIMEOUT, "a bounded device wait gave up (status %d)", h_status);
  }
  return TFS_OK;
}

int tfs_autotune_batch(const tfs_job* jobs, int n_jobs, int reps, tfs_tuning* best, double* best_ms,
                       double* default_ms, void* stream) {
  clear_error();
  TFS_CHECK(best && reps >= 1 && reps <= 100, TFS_ERR_INVALID_ARG, "need best and 1 <= reps <= 100");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* d_status = nullptr;
  TFS_CUDA(cudaMalloc(&d_status, sizeof(int)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // validation, per-segment data and window sums, and a warm start with the current choice
  int rc = tfs_eval_batch(jobs, n_jobs, d_status, stream);
  if (rc == TFS_OK) {
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "autotune warm-up");
  }
  // time one launch shape on the caller's jobs (ms per call; < 0 if it does not fit)
  std::vector<std::string> keys;
  auto time_shape = [&](const EvalTuning& t, std::vector<std::string>* k_out) -> double {
    g_force_tuning = &t;
    g_last_keys.clear();
    int r = tfs_eval_batch(jobs, n_jobs, d_status, stream);  // shape check (shared memory), warm
    if (r == TFS_OK) {
      cudaEventRecord(e0, st);
      for (int k = 0; k < reps && r == TFS_OK; ++k) r = tfs_eval_batch(jobs, n_jobs, d_status, stream);
      cudaEventRecord(e1, st);
    }
    g_force_tuning = nullptr;
    if (r != TFS_OK) {
      clear_error();
      return -1.0;  // this shape does not fit (e.g. shared memory): skip it
    }
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = cuda_fail(cudaGetLastError(), "autotune timing");
      return -1.0;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (k_out) *k_out = g_last_keys;
    return (double)ms / reps;
  };
  // coordinate descent over the five axes from the default shape, two passes; a move must gain
  // at least 0.5% so that timing noise does not wander
  EvalTuning cur;
  cur.cap = 2048;
  cur.tile_div = 1;
  cur.slots = 2;
  cur.group = 32;
  double cur_t = rc == TFS_OK ? time_shape(cur, &keys) : -1.0;
  const double def_t = cur_t;
  if (rc == TFS_OK && cur_t < 0) rc = TFS_ERR_INVALID_ARG;
  static const int groups[] = {1, 4, 8, 16, 32};
  static const int slots[] = {2, 3, 4, 6, 8};
  static const int caps[] = {512, 1024, 2048, 3072, 4096};
  static const int divs[] = {1, 2, 4, 8};
  static const int classes[] = {1, 2};
  for (int pass = 0; pass < 2 && rc == TFS_OK; ++pass) {
    bool moved = false;
    for (int axis = 0; axis < 5 && rc == TFS_OK; ++axis) {
      const int* vals = axis == 0 ? groups : axis == 1 ? slots : axis == 2 ? caps : axis == 3 ? divs : classes;
      const int nv = axis == 3 ? 4 : (axis == 4 ? 2 : 5);
      for (int i = 0; i < nv && rc == TFS_OK; ++i) {
        EvalTuning t = cur;
        int& f = axis == 0 ? t.group : axis == 1 ? t.slots : axis == 2 ? t.cap : axis == 3 ? t.tile_div : t.rsel;
        if (f == vals[i]) continue;
        f = vals[i];
        std::vector<std::string> k2;
        const double tt = time_shape(t, &k2);
        if (tt > 0 && tt < cur_t * 0.995) {
          cur = t;
          cur_t = tt;
          keys = k2;
          moved = true;
        }
      }
    }
    if (!moved) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d_status);
  if (rc == TFS_ERR_INVALID_ARG) set_error("the default launch shape does not fit these jobs");
  if (rc != TFS_OK) return rc;
  const tfs_tuning win{cur.cap, cur.tile_div, cur.slots, cur.group, cur.rsel};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const std::string& k : keys) g_tune[k] = win;
  }
  *best = win;
  if (best_ms) *best_ms = cur_t;
  if (default_ms) *default_ms = def_t;
  return TFS_OK;
}

int tfs_tuning_save(const char* path) {
  clear_error();
  TFS_CHECK(path, TFS_ERR_INVALID_ARG, "null path");
  FILE* f = fopen(path, "w");
  TFS_CHECK(f, TFS_ERR_INVALID_ARG, "cannot write %s", path);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  fprintf(f, "{\n");
  size_t i = 0;
  for (const auto& kv : g_tune)
    fprintf(f, "  \"%s\": [%d, %d, %d, %d, %d]%s\n", kv.first.c_str(), kv.second.pcap, kv.second.tile_div,
            kv.second.slots, kv.second.group, kv.second.tile_class, ++i < g_tune.size() ? "," : "");
  fprintf(f, "}\n");
  fclose(f);
  return TFS_OK;
}

int tfs_tuning_load(const char* path) {
  clear_error();
  TFS_CHECK(path, TFS_ERR_INVALID_ARG, "null path");
  FILE* f = fopen(path, "r");
  TFS_CHECK(f, TFS_ERR_NOT_FOUND, "cannot read %s", path);
  std::string txt;
  char buf[4096];
  size_t n;
  while ((n = fread(buf, 1, sizeof(buf), f)) > 0) txt.append(buf, n);
  fclose(f);
  std::map<std::string, tfs_tuning> got;
  size_t pos = 0;
  while ((pos = txt.find('"', pos)) != std::string::npos) {
    const size_t end = txt.find('"', pos + 1);
    if (end == std::string::npos) break;
    const std::string key = txt.substr(pos + 1, end - pos - 1);
    int cap = 0, div = 0, ns = 0, grp = 0, cls = 0;
    const int got_n = sscanf(txt.c_str() + end + 1, " : [%d , %d , %d , %d , %d]", &cap, &div, &ns, &grp, &cls);
    if (got_n != 5 || cap < 0 || cap > (1 << 20) || div < 0 || div > 8 || ns < 0 || ns > 8 || grp < 0 || grp > 32 ||
        cls < 0 || cls > 2) {
      set_error("malformed tuning entry for %s", key.c_str());
      return TFS_ERR_INVALID_ARG;
    }
    got[key] = tfs_tuning{cap, div, ns, grp, cls};
    pos = txt.find(']', end);
    if (pos == std::string::npos) break;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (const auto& kv : got) g_tune[kv.first] = kv.second;
  return TFS_OK;
}

int tfs_tuning_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
  return TFS_OK;
}

int tfs_topk_batch(const float* const* vals, const int64_t* Ns, const int* ks, int n, int64_t* const* idx,
                   float* const* val, void* stream) {
  clear_error();
  TFS_CHECK(n >= 0 && n <= 65536, TFS_ERR_INVALID_ARG, "need 0 <= n <= 65536 arrays");
  if (n == 0) return TFS_OK;
  TFS_CHECK(vals && Ns && ks && idx && val, TFS_ERR_INVALID_ARG, "null argument");
  std::vector<TopkTask> tasks;
  for (int i = 0; i < n; ++i) {
    TFS_CHECK(Ns[i] >= 0 && Ns[i] < ((int64_t)1 << 31), TFS_ERR_INVALID_ARG, "array %d: N must be in [0, 2^31)", i);
    TFS_CHECK(ks[i] >= 0 && ks[i] <= 1024, TFS_ERR_INVALID_ARG, "array %d: k must be in [0, 1024]", i);
    if (Ns[i] == 0 || ks[i] == 0) continue;
    TFS_CHECK(vals[i] && idx[i] && val[i], TFS_ERR_INVALID_ARG, "array %d: null pointer", i);
    tasks.push_back(TopkTask{vals[i], Ns[i], (int)std::min<int64_t>(ks[i], Ns[i]), idx[i], val[i]});
  }
  if (tasks.empty()) return TFS_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Arena ar;
  const size_t wsb = topk_batch_workspace_bytes(tasks.data(), (int)tasks.size());
  int rc = ar.init(round256(wsb), st);
  if (rc) return rc;
  rc = topk_batch_device(tasks.data(), (int)tasks.size(), ar.take<char>(wsb), st);
  if (rc) return rc;
  if (st == nullptr) TFS_CUDA(cudaStreamSynchronize(st));
  return TFS_OK;
}

int tfs_topk(const float* val_in, int64_t N, int k, int64_t* idx, float* val, int mem, void* stream) {
  clear_error();
  TFS_CHECK(val_in && idx && val, TFS_ERR_INVALID_ARG, "null argument");
  TFS_CHECK(N >= 1 && N < ((int64_t)1 << 31), TFS_ERR_INVALID_ARG, "N must be in [1, 2^31)");
  TFS_CHECK(k >= 1 && k <= 1024, TFS_ERR_INVALID_ARG, "k must be in [1, 1024]");
  TFS_CHECK(mem == TFS_MEM_HOST || mem == TFS_MEM_DEVICE, TFS_ERR_INVALID_ARG, "bad mem kind");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int kk = (int)std::min<int64_t>(k, N);
  const bool host = mem == TFS_MEM_HOST;
  Arena ar;
  size_t need = round256(topk_workspace_bytes(N));
  if (host) need += round256((size_t)N * 4) + round256((size_t)kk * 8) + round256((size_t)kk * 4);
  int rc = ar.init(need, st);
  if (rc) return rc;
  void* ws = ar.take<char>(topk_workspace_bytes(N));
  const float* d_in = val_in;
  int64_t* d_i = idx;
  float* d_v = val;
  if (host) {
    float* p = ar.take<float>(N);
    TFS_CUDA(cudaMemcpyAsync(p, val_in, (size_t)N * 4, cudaMemcpyHostToDevice, st));
    d_in = p;
    d_i = ar.take<int64_t>(kk);
    d_v = ar.take<float>(kk);
  }
  rc = topk_device(d_in, N, kk, d_i, d_v, ws, st);
  if (rc) return rc;
  if (host) {
    TFS_CUDA(cudaMemcpyAsync(idx, d_i, (size_t)kk * 8, cudaMemcpyDeviceToHost, st));
    TFS_CUDA(cudaMemcpyAsync(val, d_v, (size_t)kk * 4, cudaMemcpyDeviceToHost, st));
  }
  if (host || st == nullptr) TFS_CUDA(cudaStreamSynchronize(st));
  return TFS_OK;
}

}  // extern "C"
