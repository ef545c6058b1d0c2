// Instantiations of the fused statistic kernel for 16 and 32 coefficient slots (one translation
// unit per pair, so that the instantiations compile in parallel).
#include "eval_kernel.cuh"

namespace tfs {
TFS_INSTANTIATE_KP(16)
TFS_INSTANTIATE_KP(32)
}  // namespace tfs
