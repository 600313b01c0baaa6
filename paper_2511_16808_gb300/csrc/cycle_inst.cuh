// Explicit instantiation lists of the V-cycle drivers (cycle_impl.cuh).  The
// kernels are instantiated by the driver that launches them, so the drivers
// are spread over several translation units per precision (operator,
// smoother, transfers, the cycle itself) that nvcc compiles in parallel;
// every other unit declares them extern.
#pragma once
#include "cycle_impl.cuh"

#define HZ_CYC_OPS(EXT, T)                                                                                        \
  EXT template void resid<T>(Ctx&, int, const void*, const void*, void*, const int*, cudaStream_t);              \
  EXT template void sweep0_resid_diag<T>(Ctx&, int, const void*, void*, void*, const int*, cudaStream_t);        \
  EXT template void resid_sweep_diag<T>(Ctx&, int, const void*, const void*, void*, const int*, cudaStream_t);
#define HZ_CYC_SMOOTH(EXT, T)                                                                                     \
  EXT template void sweep_out<T>(Ctx&, int, const void*, const void*, void*, const int*, cudaStream_t);          \
  EXT template void sweep0<T>(Ctx&, int, const void*, void*, const int*, cudaStream_t);
#define HZ_CYC_XFER(EXT, T)                                                                                       \
  EXT template void restrict_t<T>(Ctx&, int, const void*, void*, const int*, cudaStream_t);                      \
  EXT template void prolong_t<T>(Ctx&, int, const void*, const void*, void*, const int*, cudaStream_t);          \
  EXT template void prolong_fused_2d<T, true>(Ctx&, int, const void*, const void*, const void*, void*, void*,     \
                                              const int*, cudaStream_t);                                          \
  EXT template void prolong_fused_2d<T, false>(Ctx&, int, const void*, const void*, const void*, void*, void*,    \
                                               const int*, cudaStream_t);                                         \
  EXT template void fine_down_diag<T>(Ctx&, const void*, void*, const int*, cudaStream_t);                       \
  EXT template void fine_up_diag<T>(Ctx&, const void*, const void*, void*, const int*, cudaStream_t);       \
  EXT template void level_down_2d<T>(Ctx&, int, const void*, void*, void*, const int*, cudaStream_t);            \
  EXT template void level_up_2d<T>(Ctx&, int, const void*, const void*, const void*, void*, const int*,         \
                                   cudaStream_t);
#define HZ_CYC_TOP(EXT, T)                                                                                        \
  EXT template void coarse_t<T>(Ctx&, const void*, void*, const int*, cudaStream_t);                             \
  EXT template void vcycle_t<T>(Ctx&, int, const void*, void*, const int*, cudaStream_t);
#define HZ_CYC_ALL(EXT, T) HZ_CYC_OPS(EXT, T) HZ_CYC_SMOOTH(EXT, T) HZ_CYC_XFER(EXT, T) HZ_CYC_TOP(EXT, T)
