// Sweep kernels of the general form (D or F not symmetric) with D and F
// staged as int8_t (see pdit_sweep.cuh).
#include "pdit_sweep.cuh"

namespace pdit {
PDIT_INSTANTIATE_SWEEP(int8_t, true, PDIT_SWEEP_SHAPES_ALL)
}  // namespace pdit
