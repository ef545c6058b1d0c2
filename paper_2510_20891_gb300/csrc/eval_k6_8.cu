// Instantiations of the fused statistic kernel for 6 and 8 coefficient slots (one translation
// unit per pair, so that the instantiations compile in parallel).
#include "eval_kernel.cuh"

namespace tfs {
TFS_INSTANTIATE_KP(6)
TFS_INSTANTIATE_KP(8)
}  // namespace tfs
