// Working-precision instantiation (float) of the V-cycle kernels and drivers
// defined in cycle_impl.cuh; compiled as its own translation unit so the
// single- and double-precision kernels build in parallel.
#include "cycle_impl.cuh"

namespace hz {
namespace cyc {
template void resid<float>(Ctx&, int, const void*, const void*, void*, const int*, cudaStream_t);
template void sweep_out<float>(Ctx&, int, const void*, const void*, void*, const int*, cudaStream_t);
template void sweep0<float>(Ctx&, int, const void*, void*, const int*, cudaStream_t);
template void restrict_t<float>(Ctx&, int, const void*, void*, const int*, cudaStream_t);
template void prolong_t<float>(Ctx&, int, const void*, const void*, void*, const int*, cudaStream_t);
template void coarse_t<float>(Ctx&, const void*, void*, const int*, cudaStream_t);
template void vcycle_t<float>(Ctx&, int, const void*, void*, const int*, cudaStream_t);
}  // namespace cyc
}  // namespace hz
