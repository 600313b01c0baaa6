// Working-precision instantiation (float) of the V-cycle itself (Algorithm 1,
// recursive) and of the coarsest solve; the operator, smoother and transfer
// drivers it calls are instantiated by cycle_f32_ops.cu, cycle_f32_smooth.cu
// and cycle_f32_xfer.cu.
#include "cycle_inst.cuh"

namespace hz {
namespace cyc {
HZ_CYC_OPS(extern, float)
HZ_CYC_SMOOTH(extern, float)
HZ_CYC_XFER(extern, float)
HZ_CYC_TOP(, float)
}  // namespace cyc
}  // namespace hz
