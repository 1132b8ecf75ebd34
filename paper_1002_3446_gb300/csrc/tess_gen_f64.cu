// Instantiations of the fused event kernel with double currents.
#include "tess_launch.cuh"

namespace tess {

cudaError_t launch_generate_f64(int n, bool sum, const EventParams &P, double *partials, int grid,
                                   cudaStream_t s) {
  if (sum) {
    switch (n) {
      case 4: return launch_event<4, double, true>(P, partials, grid, s);
      case 5: return launch_event<5, double, true>(P, partials, grid, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (n) {
    case 4: return launch_event<4, double, false>(P, partials, grid, s);
    case 5: return launch_event<5, double, false>(P, partials, grid, s);
    case 6: return launch_event<6, double, false>(P, partials, grid, s);
    case 7: return launch_event<7, double, false>(P, partials, grid, s);
    case 8: return launch_event<8, double, false>(P, partials, grid, s);
    case 9: return launch_event<9, double, false>(P, partials, grid, s);
    case 10: return launch_event<10, double, false>(P, partials, grid, s);
    case 11: return launch_event<11, double, false>(P, partials, grid, s);
    case 12: return launch_event<12, double, false>(P, partials, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

int grid_generate_f64(int n, bool sum, int sm_count, uint64_t n_events, int hist_bins) {
  if (sum) {
    switch (n) {
      case 4: return event_grid<4, double, true>(sm_count, n_events, hist_bins);
      case 5: return event_grid<5, double, true>(sm_count, n_events, hist_bins);
      default: return 1;
    }
  }
  switch (n) {
    case 4: return event_grid<4, double, false>(sm_count, n_events, hist_bins);
    case 5: return event_grid<5, double, false>(sm_count, n_events, hist_bins);
    case 6: return event_grid<6, double, false>(sm_count, n_events, hist_bins);
    case 7: return event_grid<7, double, false>(sm_count, n_events, hist_bins);
    case 8: return event_grid<8, double, false>(sm_count, n_events, hist_bins);
    case 9: return event_grid<9, double, false>(sm_count, n_events, hist_bins);
    case 10: return event_grid<10, double, false>(sm_count, n_events, hist_bins);
    case 11: return event_grid<11, double, false>(sm_count, n_events, hist_bins);
    case 12: return event_grid<12, double, false>(sm_count, n_events, hist_bins);
    default: return 1;
  }
}

cudaError_t launch_me2_f64(int n, uint64_t n_events, const double *k, const uint8_t *order, const uint32_t *hel,
                              double *me2, cudaStream_t s, bool gauge) {
  switch (n) {
    case 4: return launch_me2_t<4, double>(n_events, k, order, hel, me2, s, gauge);
    case 5: return launch_me2_t<5, double>(n_events, k, order, hel, me2, s, gauge);
    case 6: return launch_me2_t<6, double>(n_events, k, order, hel, me2, s, gauge);
    case 7: return launch_me2_t<7, double>(n_events, k, order, hel, me2, s, gauge);
    case 8: return launch_me2_t<8, double>(n_events, k, order, hel, me2, s, gauge);
    case 9: return launch_me2_t<9, double>(n_events, k, order, hel, me2, s, gauge);
    case 10: return launch_me2_t<10, double>(n_events, k, order, hel, me2, s, gauge);
    case 11: return launch_me2_t<11, double>(n_events, k, order, hel, me2, s, gauge);
    case 12: return launch_me2_t<12, double>(n_events, k, order, hel, me2, s, gauge);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tess
