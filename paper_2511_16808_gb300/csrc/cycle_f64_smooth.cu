// Working-precision instantiation (double) of the V-cycle's Vanka sweep kernels.
#include "cycle_inst.cuh"

namespace hz {
namespace cyc {
HZ_CYC_SMOOTH(, double)
}  // namespace cyc
}  // namespace hz
