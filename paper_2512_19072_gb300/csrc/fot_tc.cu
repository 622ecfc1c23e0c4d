// Tensor-core (tcgen05) axis passes: not available in this build yet.
#include "fot_common.cuh"

namespace fot {

bool tc_supported(int, int) { return false; }
int tc_create(fot_ctx*) { return 1; }
void tc_destroy(fot_ctx*) {}
void half_step_tc(fot_ctx*, const float*, const float*, double, float*, float*) {}

}  // namespace fot
