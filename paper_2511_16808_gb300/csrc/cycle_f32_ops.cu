// Working-precision instantiation (float) of the V-cycle's residual kernels (plain and fused with a diagonal sweep).
#include "cycle_inst.cuh"

namespace hz {
namespace cyc {
HZ_CYC_OPS(, float)
}  // namespace cyc
}  // namespace hz
