// Instantiations of the fused statistic kernel for tables stored as F32.
#include "eval_kernel.cuh"

namespace tfs {
int launch_eval_f32(const EvalLaunch& L, const EvalTuning& t, cudaStream_t st) { return launch_eval_dt<TFS_F32>(L, t, st); }

// Tracks that one round of full tiles over all SMs holds (a single job's launch cuts its
// tracks into whole rounds of equal tiles of at most this many tracks per SM).
long long eval_round_tracks(int KP, bool cuts, int tile_div) {
  const long long R = cuts ? r_of_kp_cuts(KP) : r_of_kp(KP);
  return (long long)kCons * R / std::max(1, std::min(tile_div, 8)) * sm_count();
}
}  // namespace tfs
