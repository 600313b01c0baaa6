// Measured arithmetic peak of the current device: the denominator of the
// roofline fraction reported for the FP64 Krylov passes (and, for reference,
// the FP32 rate that the V-cycle arithmetic runs at).  A measurement hook;
// the paper has no counterpart.
//
// Every thread runs CH independent multiply-add chains a = a*b + c for ITER
// steps (no loads or stores in the loop), so the only limit is the issue rate
// of the FMA pipe of that precision.  Two forms are timed and the faster one
// kept: 8 chains sharing b and c, and 16 chains with their own b and c (other
// operand registers, so a register-bank pattern of one form cannot hold the
// rate down).  The grid is a whole number of waves: blocks = SMs x the
// resident blocks per SM.  Timed with CUDA events on a stream of its own,
// best of several launches of about 20 ms after two warm-up launches.
#include "common.cuh"

namespace hz {
namespace {

template <typename T, int CH, bool OWN>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T b0, T c0, T* out) {
  T a[CH], b[CH], c[CH];
#pragma unroll
  for (int k = 0; k < CH; ++k) {
    a[k] = (T)(threadIdx.x + k) * (T)1e-3;
    // OWN: per-chain operands that differ from b0, c0 by less than 1e-9
    // relative, so every chain still converges to about 100
    b[k] = OWN ? b0 - (T)(k + 1) * (T)1e-12 : b0;
    c[k] = OWN ? c0 + (T)(threadIdx.x & 7) * (T)1e-16 : c0;
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < CH; ++k) a[k] = fma(a[k], b[k], c[k]);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < CH; ++k) s += a[k];
  // never true for the inputs used (|a| stays below 1e3); keeps the chains live
  if (s == (T)-12345.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T, int CH, bool OWN>
double measure(int iters, int repeats, double* best_ms) {
  constexpr int kCh = CH;
  int dev = 0, sms = 0, per_sm = 0;
  HZ_CUDA(cudaGetDevice(&dev));
  HZ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  HZ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<T, CH, OWN>, 256, 0));
  const int blocks = sms * std::max(per_sm, 1);
  cudaStream_t s;
  HZ_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  HZ_CUDA(cudaEventCreate(&e0));
  HZ_CUDA(cudaEventCreate(&e1));
  T* out = nullptr;   // written only if the chains ever hit the sentinel
  HZ_CUDA(counted_malloc_async(&out, sizeof(T) * blocks * 256, s));
  const T b = (T)0.999999, c = (T)1e-4;      // a converges to c / (1 - b) = 100
  float best = 1e30f;
  for (int r = 0; r < repeats + 2; ++r) {     // the first two launches warm up
    HZ_CUDA(cudaEventRecord(e0, s));
    k_fma_chains<T, CH, OWN><<<blocks, 256, 0, s>>>(iters, b, c, out);
    HZ_CUDA(cudaGetLastError());
    HZ_CUDA(cudaEventRecord(e1, s));
    HZ_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    HZ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (r >= 2) best = std::min(best, ms);
  }
  HZ_CUDA(cudaFreeAsync(out, s));
  HZ_CUDA(cudaStreamSynchronize(s));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  *best_ms = best;
  const double flops = 2.0 * kCh * (double)iters * blocks * 256.0;
  return flops / (best / 1e3) / 1e12;
}

}  // namespace
}  // namespace hz

using namespace hz;

extern "C" hz_status hz_measure_peak(int kind, double* tflops, double* ms) {
  return guarded([&] {
    require(tflops != nullptr, "null output");
    require(kind == 0 || kind == 1, "kind must be 0 (FP64) or 1 (FP32)");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) throw Error(HZ_ERR_NO_DEVICE, "no CUDA device");
    double t1 = 0, t2 = 0;
    // about 20 ms per launch at the expected rates
    double r1, r2;
    if (kind == 0) {
      r1 = measure<double, 8, false>(4096, 5, &t1);
      r2 = measure<double, 16, true>(2048, 5, &t2);
    } else {
      r1 = measure<float, 8, false>(131072, 5, &t1);
      r2 = measure<float, 16, true>(65536, 5, &t2);
    }
    *tflops = std::max(r1, r2);
    if (ms) *ms = r1 >= r2 ? t1 : t2;
  });
}
