// Instantiations of the fused statistic kernel for tables stored as F32.
#include "eval_kernel.cuh"

namespace tfs {
int launch_eval_f32(const EvalLaunch& L, const EvalTuning& t, cudaStream_t st) { return launch_eval_dt<TFS_F32>(L, t, st); }
}  // namespace tfs
