// Instantiations of the fused statistic kernel for tables stored as F8E4M3.
#include "eval_kernel.cuh"

namespace tfs {
int launch_eval_f8(const EvalLaunch& L, const EvalTuning& t, cudaStream_t st) { return launch_eval_dt<TFS_F8E4M3>(L, t, st); }
}  // namespace tfs
