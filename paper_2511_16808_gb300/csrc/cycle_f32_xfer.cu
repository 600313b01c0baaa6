// Working-precision instantiation (float) of the V-cycle's restriction and prolongation kernels (and the 2D fused prolongation tiles).
#include "cycle_inst.cuh"

namespace hz {
namespace cyc {
HZ_CYC_XFER(, float)
}  // namespace cyc
}  // namespace hz
