// Smoothed-aggregation AMG hierarchy on the device (placeholder).
#include "eb_solver.cuh"

namespace ebk {

struct Hierarchy {};

void amg_build(Solver& S, cudaStream_t) {
  (void)S;
  throw Failure{EB_ERR_NOT_IMPLEMENTED, "amg_setup: AMG hierarchy not built yet; use max_levels = 0"};
}
void amg_free(Solver& S) { S.H = nullptr; }
void amg_vcycle_grid(Solver&, const double*, double*, cudaStream_t) {
  throw Failure{EB_ERR_NOT_IMPLEMENTED, "amg_vcycle: no hierarchy"};
}
void amg_fill_info(const Solver&, amg_info_t* out) { out->num_levels = 0; }
void amg_copy_level(const Solver&, int, int, int32_t*, int32_t*, double*, cudaStream_t) {
  throw Failure{EB_ERR_INVALID, "amg_level_copy: no hierarchy"};
}

}  // namespace ebk
