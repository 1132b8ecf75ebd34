// Instantiations of the two-kernel pipeline (double currents, n = 4..12).
#include "tess_pipe_launch.cuh"

namespace tess {

int plan_pipeline_f64(int n, int sm_count, uint64_t n_events, int hist_bins, int form, int sched,
                          unsigned caps, PipePlan *pl) {
  switch (n) {
    case 4: return plan_pipeline_t<4, double>(sm_count, n_events, hist_bins, form, sched, caps, pl);
    case 5: return plan_pipeline_t<5, double>(sm_count, n_events, hist_bins, form, sched, caps, pl);
    case 6: return plan_pipeline_t<6, double>(sm_count, n_events, hist_bins, form, sched, caps, pl);
    case 7: return plan_pipeline_t<7, double>(sm_count, n_events, hist_bins, form, sched, caps, pl);
    case 8: return plan_pipeline_t<8, double>(sm_count, n_events, hist_bins, form, sched, caps, pl);
    case 9: return plan_pipeline_t<9, double>(sm_count, n_events, hist_bins, form, sched, caps, pl);
    case 10: return plan_pipeline_t<10, double>(sm_count, n_events, hist_bins, form, sched, caps, pl);
    case 11: return plan_pipeline_t<11, double>(sm_count, n_events, hist_bins, form, sched, caps, pl);
    case 12: return plan_pipeline_t<12, double>(sm_count, n_events, hist_bins, form, sched, caps, pl);
    default: return -1;
  }
}

cudaError_t run_pipeline_f64(int n, const EventParams &P, const PipePlan &pl, char *ws, cudaStream_t s,
                                 const StageHook *hook, const OverlapRes *ov) {
  switch (n) {
    case 4: return run_pipeline_t<4, double>(P, pl, ws, s, hook, ov);
    case 5: return run_pipeline_t<5, double>(P, pl, ws, s, hook, ov);
    case 6: return run_pipeline_t<6, double>(P, pl, ws, s, hook, ov);
    case 7: return run_pipeline_t<7, double>(P, pl, ws, s, hook, ov);
    case 8: return run_pipeline_t<8, double>(P, pl, ws, s, hook, ov);
    case 9: return run_pipeline_t<9, double>(P, pl, ws, s, hook, ov);
    case 10: return run_pipeline_t<10, double>(P, pl, ws, s, hook, ov);
    case 11: return run_pipeline_t<11, double>(P, pl, ws, s, hook, ov);
    case 12: return run_pipeline_t<12, double>(P, pl, ws, s, hook, ov);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tess
