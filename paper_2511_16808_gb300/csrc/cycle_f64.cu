// Working-precision instantiation (double) of the V-cycle itself (Algorithm 1,
// recursive) and of the coarsest solve; the operator, smoother and transfer
// drivers it calls are instantiated by cycle_f64_ops.cu, cycle_f64_smooth.cu
// and cycle_f64_xfer.cu.
#include "cycle_inst.cuh"

namespace hz {
namespace cyc {
HZ_CYC_OPS(extern, double)
HZ_CYC_SMOOTH(extern, double)
HZ_CYC_XFER(extern, double)
HZ_CYC_TOP(, double)
}  // namespace cyc
}  // namespace hz
