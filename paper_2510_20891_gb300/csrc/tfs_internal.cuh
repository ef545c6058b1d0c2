// Internal declarations shared by the CUDA translation units of libtfstat.
// Nothing here is part of the C ABI (include/tfstat.h is).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/tfstat.h"

namespace tfs {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
void clear_error();
int cuda_fail(cudaError_t e, const char* what);  // records the message, returns TFS_ERR_CUDA

#define TFS_CUDA(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return ::tfs::cuda_fail(e_, #call); \
  } while (0)

#define TFS_CHECK(cond, code, ...)     \
  do {                                 \
    if (!(cond)) {                     \
      ::tfs::set_error(__VA_ARGS__);   \
      return (code);                   \
    }                                  \
  } while (0)

// Device status word values written by kernels (0 = ok).
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_BAD = 2 };

// An NVTX range over an entry point (seen by profilers that record NVTX; free otherwise).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Process-wide count of kernel launches made by this library.
void count_launch(int n = 1);
void free_sft_plan(void* p);

// ---------------------------------------------------------------- handles
// Floats per segment row of segp, and the first column of the segment-cut forms (16-byte aligned).
__host__ __device__ constexpr int cut_col(int KP) { return ((KP + 3) / 4) * 4; }
inline int segrow_floats(int KP, bool cuts) { return cut_col(KP) + (cuts ? 4 * KP : 0); }

struct SegParams {          // per (basis, T_sft) data for the FP32 filter of the track evaluation
  double T = 0.0;
  int KP = 0;               // coefficient slots in the kernel (>= K, zero padded)
  int nsp = 0;              // floats per segment row of `segp` (multiple of 4, >= KP)
  int alpha_mid = 0;
  float* segp = nullptr;    // device [n_seg][nsp]: D_k,alpha = fl32(T U_k,alpha - T U_k,mid) at k;
                            // with cuts also E, E, G, G (each of E_k,alpha and G_k,alpha twice,
                            // the operand pair of a packed two-track FMA) from cut_col(KP) + 4k
  float* dmax = nullptr;    // device [KP]: max_alpha |D_k,alpha| (rounded up)
  float* umax = nullptr;    // device [KP]: max_alpha |U_k,alpha| (rounded up)
  int cuts = 0;             // rows carry the segment-cut forms E (second difference) and G (first)
  float* emax = nullptr;    // device [KP]: max_alpha |E_k,alpha| (rounded up), cuts only
  float* gmax = nullptr;    // device [KP]: max_alpha |G_k,alpha| (rounded up), cuts only
};

// Window sums of a table for one neighbour half-width m (see wsum.cu): [n_seg][pitch] FP32,
// centre c at index c + m; zeros past the last centre whose window overlaps the table.
struct WSum {
  int m = 0;
  int64_t pitch = 0;
  int64_t bytes = 0;
  float* q = nullptr;   // from the device's stream-ordered pool
};

}  // namespace tfs

struct tfs_table {
  int device = 0;
  int64_t n_seg = 0, n_bin = 0, row_stride = 0;
  int dtype = TFS_F32;
  double T_sft = 0.0;
  void* data = nullptr;     // device [n_seg][row_stride], zero padded beyond n_bin
  float* scales = nullptr;  // device [n_seg] (FP8 only)
  int64_t bytes = 0;
  double dt = 0.0;
  void* sft_plan = nullptr; // cached SFT plan (window, twiddles, PSD normalisation) when built from strain
  bool owns = true;         // false for a view: data and scales belong to another table
  const tfs_table* owner = nullptr;  // a view: the table that owns the rows (and their window sums)
  int64_t seg0 = 0;         // a view: its first row in the owner
  mutable std::mutex wmu;   // guards wsums
  mutable std::vector<tfs::WSum> wsums;  // window sums per m used so far (owning tables only)
};

struct tfs_ctable {          // linear-chirp table: scaled complex spectra of a Hann-windowed strain
  int device = 0;
  int64_t n_seg = 0, n_bin = 0, L = 0;
  double T_sft = 0.0, dt = 0.0;
  double s_ref = 1.0;       // reference PSD of the scaling (median of the usable S_n)
  float2* z = nullptr;      // device [n_seg][n_bin]: sqrt(4 dt / (sum w^2 S_ref)) X_k S_ref / S_k
  float* wt = nullptr;      // device [n_bin]: S_ref / S_k (owned by the plan)
  void* sft_plan = nullptr; // the SFT plan (window, twiddles, scales)
  bool owns = true;         // false for a view: z and wt belong to another table
};

struct tfs_basis {
  int device = 0;
  int K = 0;
  int64_t n_seg = 0;
  double* U = nullptr;      // device [K][n_seg]
  std::vector<double> sigma, cmin, cmax;
  std::mutex mu;            // guards the cached segment parameters
  std::vector<tfs::SegParams*> sps;  // one per (T_sft, slot count) used so far; freed with the basis
};

namespace tfs {

__host__ __device__ constexpr int esize_of(int dtype) { return dtype == TFS_F32 ? 4 : (dtype == TFS_F8E4M3 ? 1 : 2); }

// Window sums (wsum.cu).  wsum_get returns the rows of t's window sums for m (built on first
// use, then kept with the owning table; the first build synchronises `st`, so it must not be
// inside a stream capture); wsum_refresh recomputes every kept m on `st` after the table's
// data changed; wsum_free releases them.
int64_t wsum_pitch(int64_t n_bin, int m);
int64_t wsum_bytes(const tfs_table* t, int m);
int64_t wsum_cached_bytes(const tfs_table* t);
bool wsum_cached(const tfs_table* t, int m);
int wsum_get(const tfs_table* t, int m, cudaStream_t st, const float** q, int* pitch);
// Keeps up to 8 GB of freed stream-ordered memory reserved in the device's pool (tfs_api.cu).
void retain_pool_memory();
int wsum_refresh(tfs_table* t, cudaStream_t st);
void wsum_free(tfs_table* t);
void wsum_free_idle(tfs_table* t, cudaStream_t st);  // no kernel of any stream reads them any more

// Cached FP32 filter parameters of a basis for a given T_sft, with at least kp_min coefficient
// slots (built on first use; rebuilt for another T_sft or a wider slot count).
int get_segparams(tfs_basis* b, double T, int kp_min, cudaStream_t st, SegParams** out, int cuts = 0);
int pick_kp(int K);

// ---------------------------------------------------------------- kernels (host launchers)
struct EvalJob {          // one dataset's part of a statistic launch
  const tfs_table* table;
  const tfs_basis* basis;
  const SegParams* sp;    // built with the launch's coefficient slot count
  const double* coeffs;   // device [N][K]
  const double* f_ref;    // device [N] or null
  int64_t N;
  int m;
  float* stat;            // device [N]
  int* bins_out = nullptr;  // device [N][n_seg] or null: the bin of every pair (verification only)
  int cuts = 0;           // apply the segment exclusions (TFS_JOB_SEGMENT_CUTS)
  int split = 0;          // > 1: split every track tile's segments over this many tiles (a launch's tail)
};
struct EvalLaunch {
  const EvalJob* jobs;    // host array
  int n_jobs;
  unsigned long long* tie_count;  // device
  int64_t* tie_track;     // device [tie_cap]
  int* tie_seg;
  int tie_cap;
  int* status;            // device
  unsigned long long* dbg = nullptr;  // self-check record (TFS_DEBUG_CHECKS builds)
};
struct EvalTuning {       // launch shape; zeros select defaults
  int cap = 0;            // window sums staged per segment at most (a band cut to it takes the slower path)
  int tile_div = 0;       // tiles of (consumer threads x R) / tile_div tracks at most
  int slots = 0;          // staging slots (ring depth)
  int group = 0;          // segments per staging slot at most (one hand-off per slot)
  int rsel = 0;           // tracks per consumer thread: 0 automatic, 1 the large class, 2 the small class
};
constexpr int kMaxJobs = 64;  // jobs per statistic launch (larger batches are split)
int launch_eval(const EvalLaunch& L, const EvalTuning& tune, cudaStream_t st);
// the statistic kernel for a shape already chosen (eval_host.cu)
int launch_eval_shape(const EvalLaunch& L, const EvalTuning& tune, cudaStream_t st);
// tracks that one round of full tiles over all SMs holds
long long eval_round_tracks(int KP, bool cuts, int tile_div);
// limit of the statistic kernel's waits (ns) and whether its stager first waits for an arrival
// that never comes (timeout tests); tfs_set_wait_limit sets them process-wide
uint64_t eval_wait_ns();
int eval_hold();
void set_eval_wait(uint64_t ns, int hold);

// top-k over device floats; scratch from `ws` (size from topk_workspace_bytes) or allocated.
size_t topk_workspace_bytes(int64_t N);
int topk_device(const float* val, int64_t N, int k, int64_t* idx_out, float* val_out, void* ws, cudaStream_t st);

// top-k of many arrays at once (one set of passes over all of them; each result equals
// topk_device on that array alone); scratch from topk_batch_workspace_bytes
constexpr int kTkJobs = 64;  // arrays per pass set (more are done in groups)
struct TopkTask {
  const float* val;
  int64_t N;
  int k;
  int64_t* idx_out;
  float* val_out;
};
size_t topk_batch_workspace_bytes(const TopkTask* tasks, int n);
int topk_batch_device(const TopkTask* tasks, int n, void* ws, cudaStream_t st);

// quantise an FP64 device table P [n_seg][n_bin] (row pitch `ld`) into a table's storage
int quantise_into(const double* P, int64_t ld, tfs_table* t, cudaStream_t st);

// allocate a zeroed table of the given shape/dtype (data + scales)
int alloc_table(int64_t n_seg, int64_t n_bin, int dtype, double T_sft, tfs_table** out);

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// 1-D bulk copy global -> shared, completing `bytes` of transaction count on `bar`.
// dst, src 16-byte aligned; bytes a positive multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase `parity` of an mbarrier to complete; gives up after ~limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  const uint32_t a = smem_u32(bar);
  uint32_t done = 0;
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63) == 0) {
      const uint64_t now = global_ns();
      if (it == 0) t0 = now;
      else if (now - t0 > limit_ns) return false;
    }
  }
}

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s

}  // namespace tfs
