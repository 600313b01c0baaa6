// Working-precision instantiation (float) of the V-cycle's Vanka sweep kernels.
#include "cycle_inst.cuh"

namespace hz {
namespace cyc {
HZ_CYC_SMOOTH(, float)
}  // namespace cyc
}  // namespace hz
