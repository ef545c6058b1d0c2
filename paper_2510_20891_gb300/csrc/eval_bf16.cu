// Instantiations of the fused statistic kernel for tables stored as BF16.
#include "eval_kernel.cuh"

namespace tfs {
int launch_eval_bf16(const EvalLaunch& L, const EvalTuning& t, cudaStream_t st) { return launch_eval_dt<TFS_BF16>(L, t, st); }
}  // namespace tfs
