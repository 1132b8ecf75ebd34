// Instantiations of the two-kernel pipeline (float currents, n = 4..7).
#include "tess_pipe_launch.cuh"

namespace tess {

int plan_pipeline_f32a(int n, int sm_count, uint64_t n_events, int hist_bins, int form, int sched,
                          unsigned caps, PipePlan *pl) {
  switch (n) {
    case 4: return plan_pipeline_t<4, float>(sm_count, n_events, hist_bins, form, sched, caps, pl);
    case 5: return plan_pipeline_t<5, float>(sm_count, n_events, hist_bins, form, sched, caps, pl);
    case 6: return plan_pipeline_t<6, float>(sm_count, n_events, hist_bins, form, sched, caps, pl);
    case 7: return plan_pipeline_t<7, float>(sm_count, n_events, hist_bins, form, sched, caps, pl);
    default: return -1;
  }
}

cudaError_t run_pipeline_f32a(int n, const EventParams &P, const PipePlan &pl, char *ws, cudaStream_t s,
                                 const StageHook *hook, const OverlapRes *ov) {
  switch (n) {
    case 4: return run_pipeline_t<4, float>(P, pl, ws, s, hook, ov);
    case 5: return run_pipeline_t<5, float>(P, pl, ws, s, hook, ov);
    case 6: return run_pipeline_t<6, float>(P, pl, ws, s, hook, ov);
    case 7: return run_pipeline_t<7, float>(P, pl, ws, s, hook, ov);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tess
