// Sweep kernels with D and F staged as int32_t (see pdit_sweep.cuh).
#include "pdit_sweep.cuh"

namespace pdit {
PDIT_INSTANTIATE_SWEEP(int32_t, false, PDIT_SWEEP_SHAPES_ALL)
}  // namespace pdit
