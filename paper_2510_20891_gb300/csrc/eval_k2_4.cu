// Instantiations of the fused statistic kernel for 2 and 4 coefficient slots (one translation
// unit per pair, so that the instantiations compile in parallel).
#include "eval_kernel.cuh"

namespace tfs {
TFS_INSTANTIATE_KP(2)
TFS_INSTANTIATE_KP(4)
}  // namespace tfs
