// Sweep kernels with D and F staged as int16_t (see pdit_sweep.cuh).
#include "pdit_sweep.cuh"

namespace pdit {
PDIT_INSTANTIATE_SWEEP(int16_t, false, PDIT_SWEEP_SHAPES_ALL)
}  // namespace pdit
