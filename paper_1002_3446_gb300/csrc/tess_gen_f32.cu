// Instantiations of the fused event kernel with float currents.
#include "tess_launch.cuh"

namespace tess {

cudaError_t launch_generate_f32(int n, bool sum, const EventParams &P, double *partials, int grid,
                                   cudaStream_t s) {
  if (sum) {
    switch (n) {
      case 4: return launch_event<4, float, true>(P, partials, grid, s);
      case 5: return launch_event<5, float, true>(P, partials, grid, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (n) {
    case 4: return launch_event<4, float, false>(P, partials, grid, s);
    case 5: return launch_event<5, float, false>(P, partials, grid, s);
    case 6: return launch_event<6, float, false>(P, partials, grid, s);
    case 7: return launch_event<7, float, false>(P, partials, grid, s);
    case 8: return launch_event<8, float, false>(P, partials, grid, s);
    case 9: return launch_event<9, float, false>(P, partials, grid, s);
    case 10: return launch_event<10, float, false>(P, partials, grid, s);
    case 11: return launch_event<11, float, false>(P, partials, grid, s);
    case 12: return launch_event<12, float, false>(P, partials, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

int grid_generate_f32(int n, bool sum, int sm_count, uint64_t n_events, int hist_bins) {
  if (sum) {
    switch (n) {
      case 4: return event_grid<4, float, true>(sm_count, n_events, hist_bins);
      case 5: return event_grid<5, float, true>(sm_count, n_events, hist_bins);
      default: return 1;
    }
  }
  switch (n) {
    case 4: return event_grid<4, float, false>(sm_count, n_events, hist_bins);
    case 5: return event_grid<5, float, false>(sm_count, n_events, hist_bins);
    case 6: return event_grid<6, float, false>(sm_count, n_events, hist_bins);
    case 7: return event_grid<7, float, false>(sm_count, n_events, hist_bins);
    case 8: return event_grid<8, float, false>(sm_count, n_events, hist_bins);
    case 9: return event_grid<9, float, false>(sm_count, n_events, hist_bins);
    case 10: return event_grid<10, float, false>(sm_count, n_events, hist_bins);
    case 11: return event_grid<11, float, false>(sm_count, n_events, hist_bins);
    case 12: return event_grid<12, float, false>(sm_count, n_events, hist_bins);
    default: return 1;
  }
}

cudaError_t launch_me2_f32(int n, uint64_t n_events, const double *k, const uint8_t *order, const uint32_t *hel,
                              double *me2, cudaStream_t s, bool gauge) {
  switch (n) {
    case 4: return launch_me2_t<4, float>(n_events, k, order, hel, me2, s, gauge);
    case 5: return launch_me2_t<5, float>(n_events, k, order, hel, me2, s, gauge);
    case 6: return launch_me2_t<6, float>(n_events, k, order, hel, me2, s, gauge);
    case 7: return launch_me2_t<7, float>(n_events, k, order, hel, me2, s, gauge);
    case 8: return launch_me2_t<8, float>(n_events, k, order, hel, me2, s, gauge);
    case 9: return launch_me2_t<9, float>(n_events, k, order, hel, me2, s, gauge);
    case 10: return launch_me2_t<10, float>(n_events, k, order, hel, me2, s, gauge);
    case 11: return launch_me2_t<11, float>(n_events, k, order, hel, me2, s, gauge);
    case 12: return launch_me2_t<12, float>(n_events, k, order, hel, me2, s, gauge);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tess
