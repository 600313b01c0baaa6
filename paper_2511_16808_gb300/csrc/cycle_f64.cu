// Working-precision instantiation (double) of the V-cycle kernels and drivers
// defined in cycle_impl.cuh; compiled as its own translation unit so the
// single- and double-precision kernels build in parallel.
#include "cycle_impl.cuh"

namespace hz {
namespace cyc {
template void resid<double>(Ctx&, int, const void*, const void*, void*, const int*, cudaStream_t);
template void sweep_out<double>(Ctx&, int, const void*, const void*, void*, const int*, cudaStream_t);
template void sweep0<double>(Ctx&, int, const void*, void*, const int*, cudaStream_t);
template void restrict_t<double>(Ctx&, int, const void*, void*, const int*, cudaStream_t);
template void prolong_t<double>(Ctx&, int, const void*, const void*, void*, const int*, cudaStream_t);
template void coarse_t<double>(Ctx&, const void*, void*, const int*, cudaStream_t);
template void vcycle_t<double>(Ctx&, int, const void*, void*, const int*, cudaStream_t);
}  // namespace cyc
}  // namespace hz
