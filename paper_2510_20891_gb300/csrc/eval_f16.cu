// Instantiations of the fused statistic kernel for tables stored as F16.
#include "eval_kernel.cuh"

namespace tfs {
int launch_eval_f16(const EvalLaunch& L, const EvalTuning& t, cudaStream_t st) { return launch_eval_dt<TFS_F16>(L, t, st); }
}  // namespace tfs
