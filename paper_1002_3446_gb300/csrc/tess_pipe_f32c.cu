// Instantiations of the two-kernel pipeline (float currents, n = 11..12).
#include "tess_pipe_launch.cuh"

namespace tess {

int plan_pipeline_f32c(int n, int sm_count, uint64_t n_events, int hist_bins, int form, int sched,
                          unsigned caps, PipePlan *pl) {
  switch (n) {
    case 11: return plan_pipeline_t<11, float>(sm_count, n_events, hist_bins, form, sched, caps, pl);
    case 12: return plan_pipeline_t<12, float>(sm_count, n_events, hist_bins, form, sched, caps, pl);
    default: return -1;
  }
}

cudaError_t run_pipeline_f32c(int n, const EventParams &P, const PipePlan &pl, char *ws, cudaStream_t s,
                                 const StageHook *hook, const OverlapRes *ov) {
  switch (n) {
    case 11: return run_pipeline_t<11, float>(P, pl, ws, s, hook, ov);
    case 12: return run_pipeline_t<12, float>(P, pl, ws, s, hook, ov);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tess
