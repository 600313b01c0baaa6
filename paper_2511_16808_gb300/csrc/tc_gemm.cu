// Coarsest-level solve of a multi-RHS V-cycle on the tensor cores (Algorithm
// 1 step 3, exact solve by the dense inverse from setup): U = Ainv F with R
// right-hand sides (R = 16, 32 or 64), complex FP32 data, as one real GEMM
//
//   C' (2n x R) = A' (2n x 2n) F' (2n x R),   A'[2i+a][2j+b] = [[Ar, -Ai], [Ai, Ar]]_ab,
//                                             F'[2j+b][r] = (Fr, Fi)_b,  C'[2i+a][r] = (Ur, Ui)_a
//
// on tcgen05 (kind::tf32, FP32 accumulation in tensor memory) with the
// 3xTF32 split: x = x_hi + x_lo with both parts tf32, x y ~ x_hi y_hi +
// x_hi y_lo + x_lo y_hi (relative error about 2^-22, at the level of the
// FP32 CUDA-core product it replaces).  A CTA of 128 threads owns 128 rows of
// C' (64 complex rows) and all R columns; K is walked in chunks of 32 (16
// complex columns) staged by all threads in shared memory (double buffered:
// the next chunk is loaded while the tensor core works on the current one);
// one thread issues the 12 MMAs of a chunk and commits them to the buffer's
// mbarrier.  With a split of K over S CTAs per row tile, each writes FP32
// partial sums and a second kernel adds them in split order (deterministic).
#include "common.cuh"
#include "tc_ops.cuh"

namespace hz {
namespace {

constexpr int kTcThreads = 128, kTcM = 128, kTcK = 32;
constexpr long long kTcWaitPolls = 20000000LL;    // ~a second or more of polling: far beyond any MMA

__host__ __device__ inline size_t tc_buffer_bytes(int R) { return 2 * (size_t)kTcM * kTcK * 4 + 2 * (size_t)R * kTcK * 4; }

__global__ void __launch_bounds__(kTcThreads) k_coarse_gemm_tc(int n, int R, int split, const float2* __restrict__ A,
                                                               const float2* __restrict__ F, float* __restrict__ part,
                                                               float2* __restrict__ U, int* err, const int* active) {
  extern __shared__ unsigned char smraw[];
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t taddr_s;
  pdl_enter();
  if (active && !*active) return;
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const size_t BUF = tc_buffer_bytes(R);
  const uint32_t cols = R < 32 ? 32u : (uint32_t)R;
  const int tile = blockIdx.x, sidx = blockIdx.y;
  const int nch = (n + 15) / 16;                       // chunks of 16 complex columns
  const int per = (nch + split - 1) / split;
  const int c0 = min(sidx * per, nch), c1 = min(c0 + per, nch);
  if (warp == 0) tc::tmem_alloc(&taddr_s, cols);
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = taddr_s;
  const uint32_t idesc = tc::idesc_tf32(kTcM, R < 16 ? 16 : R);
  const int i0 = tile * (kTcM / 2);                     // first complex row of the tile
  bool ok = true;
  int issued = 0;                                        // chunks whose MMAs were committed
  for (int c = c0; c < c1; ++c) {
    const int L = c - c0, b = L & 1;
    unsigned char* buf = sm + b * BUF;
    float* a_hi = (float*)buf;
    float* a_lo = (float*)(buf + kTcM * kTcK * 4);
    float* b_hi = (float*)(buf + 2 * kTcM * kTcK * 4);
    float* b_lo = (float*)(buf + 2 * kTcM * kTcK * 4 + R * kTcK * 4);
    const int j0 = c * 16;
    // this chunk's A (64 x 16 complex) and F (16 x R complex) values
    float2 av[8], fv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + q * kTcThreads, li = e >> 4, lj = e & 15;
      const int i = i0 + li, j = j0 + lj;
      av[q] = (i < n && j < n) ? A[(long long)i * n + j] : make_float2(0.f, 0.f);
    }
    const int nf = 16 * R / kTcThreads;                 // 2, 4 or 8
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (q < nf) {
        const int e = tid + q * kTcThreads, lj = e / R, r = e - lj * R, j = j0 + lj;
        fv[q] = j < n ? F[(long long)j * R + r] : make_float2(0.f, 0.f);
      }
    }
    // the buffer is free once the MMAs of chunk c - 2 completed (the
    // decision is made by all threads together, so they leave the loop alike)
    if (L >= 2 && !__syncthreads_and(tc::mbar_wait(&mbar[b], ((L - 2) >> 1) & 1, kTcWaitPolls))) {
      ok = false;
      break;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + q * kTcThreads, li = e >> 4, lj = e & 15;
      const float ar = av[q].x, ai = av[q].y;
      const float rh = tc::tf32_rna(ar), rl = tc::tf32_rna(ar - rh);
      const float ih = tc::tf32_rna(ai), il = tc::tf32_rna(ai - ih);
      const int m0 = 2 * li, k0 = 2 * lj;
      *(float*)((unsigned char*)a_hi + tc::kmajor_offset<kTcK>(m0, k0)) = rh;
      *(float*)((unsigned char*)a_hi + tc::kmajor_offset<kTcK>(m0, k0 + 1)) = -ih;
      *(float*)((unsigned char*)a_hi + tc::kmajor_offset<kTcK>(m0 + 1, k0)) = ih;
      *(float*)((unsigned char*)a_hi + tc::kmajor_offset<kTcK>(m0 + 1, k0 + 1)) = rh;
      *(float*)((unsigned char*)a_lo + tc::kmajor_offset<kTcK>(m0, k0)) = rl;
      *(float*)((unsigned char*)a_lo + tc::kmajor_offset<kTcK>(m0, k0 + 1)) = -il;
      *(float*)((unsigned char*)a_lo + tc::kmajor_offset<kTcK>(m0 + 1, k0)) = il;
      *(float*)((unsigned char*)a_lo + tc::kmajor_offset<kTcK>(m0 + 1, k0 + 1)) = rl;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (q < nf) {
        const int e = tid + q * kTcThreads, lj = e / R, r = e - lj * R;
        const float fr = fv[q].x, fi = fv[q].y;
        const float rh = tc::tf32_rna(fr), ih = tc::tf32_rna(fi);
        *(float*)((unsigned char*)b_hi + tc::kmajor_offset<kTcK>(r, 2 * lj)) = rh;
        *(float*)((unsigned char*)b_hi + tc::kmajor_offset<kTcK>(r, 2 * lj + 1)) = ih;
        *(float*)((unsigned char*)b_lo + tc::kmajor_offset<kTcK>(r, 2 * lj)) = tc::tf32_rna(fr - rh);
        *(float*)((unsigned char*)b_lo + tc::kmajor_offset<kTcK>(r, 2 * lj + 1)) = tc::tf32_rna(fi - ih);
      }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
      const uint32_t sbo_a = 128 * kTcK / 4, sbo_b = 128 * kTcK / 4;
#pragma unroll
      for (int k = 0; k < kTcK / 8; ++k) {
        const uint64_t ah = tc::smem_desc(tc::smem_u32(a_hi) + 256 * k, 128, sbo_a);
        const uint64_t al = tc::smem_desc(tc::smem_u32(a_lo) + 256 * k, 128, sbo_a);
        const uint64_t bh = tc::smem_desc(tc::smem_u32(b_hi) + 256 * k, 128, sbo_b);
        const uint64_t bl = tc::smem_desc(tc::smem_u32(b_lo) + 256 * k, 128, sbo_b);
        tc::mma_tf32(taddr, ah, bh, idesc, L > 0 || k > 0);
        tc::mma_tf32(taddr, ah, bl, idesc, true);
        tc::mma_tf32(taddr, al, bh, idesc, true);
      }
      tc::mma_commit(&mbar[b]);
    }
    ++issued;
  }
  // the last commit completes after every earlier MMA of the CTA
  const int nl = c1 - c0;
  if (ok && issued > 0)
    ok = __syncthreads_and(tc::mbar_wait(&mbar[(issued - 1) & 1], ((issued - 1) >> 1) & 1, kTcWaitPolls));
  // a wait that gave up: record it, wait once more (bounded) for the MMAs in
  // flight before the tensor memory is released, and leave the result alone
  if (!ok) {
    if (lane == 0) atomicExch(err, 1);
    if (issued > 0) tc::mbar_wait(&mbar[(issued - 1) & 1], ((issued - 1) >> 1) & 1, kTcWaitPolls);
  }
  const int mrow = tile * kTcM + 32 * warp + lane;     // row of C' held by this thread
  const bool rowok = mrow < 2 * n;
  tc::fence_after_sync();
  if (ok) {
    for (int c = 0; c < R; c += 16) {
      float v[16];
      if (nl > 0) tc::tmem_ld16(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, v);
      else {
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = 0.f;
      }
      if (!rowok) continue;
      if (split == 1) {
        float* u = (float*)U;
        const int i = mrow >> 1, a = mrow & 1;
#pragma unroll
        for (int q = 0; q < 16; ++q) u[((long long)i * R + c + q) * 2 + a] = v[q];
      } else {
        float* pp = part + ((long long)sidx * 2 * n + mrow) * R + c;
#pragma unroll
        for (int q = 0; q < 16; ++q) pp[q] = v[q];
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, cols);
}

// U[i][r] = sum over the splits, in split order
__global__ void k_coarse_gemm_reduce(int n, int R, int split, const float* __restrict__ part, float2* __restrict__ U,
                                     const int* active) {
  pdl_enter();
  if (active && !*active) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // complex output index i * R + r
  if (e >= (long long)n * R) return;
  const long long i = e / R, r = e - i * R;
  float re = 0.f, im = 0.f;
  for (int s = 0; s < split; ++s) {
    re += part[((long long)s * 2 * n + 2 * i) * R + r];
    im += part[((long long)s * 2 * n + 2 * i + 1) * R + r];
  }
  U[e] = make_float2(re, im);
}

template <typename... KArgs, typename... Args>
void launch_smem(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  HZ_CUDA(cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...));
}

}  // namespace

size_t smem_max_tc() { return 1024 + 2 * tc_buffer_bytes(64); }

bool coarse_tc_supported(const Ctx& c, int nrhs) {
  return c.mixed && (nrhs == 16 || nrhs == 32 || nrhs == 64) && c.tc_err != nullptr;
}

void coarse_gemm_tc(Ctx& c, const void* f, void* u, const int* active, cudaStream_t s, int split) {
  const Level& L = c.L.back();
  const int n = (int)L.g.N, R = c.nrhs;
  require(coarse_tc_supported(c, R), "tensor-core coarsest solve: mixed precision, 16/32/64 right-hand sides");
  require(split >= 1 && split <= kTcMaxSplit, "tensor-core split out of range");
  require(split == 1 || c.tc_partial != nullptr, "tensor-core split needs the partial-sum buffer");
  const size_t smem = 1024 + 2 * tc_buffer_bytes(R);
  static bool attr_set[256] = {};
  if (!attr_set[c.dev & 255]) {
    HZ_CUDA(cudaFuncSetAttribute(k_coarse_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max_tc()));
    attr_set[c.dev & 255] = true;
  }
  const dim3 grid((unsigned)((2 * n + kTcM - 1) / kTcM), (unsigned)split);
  launch_smem(k_coarse_gemm_tc, grid, dim3(kTcThreads), smem, s, n, R, split, (const float2*)L.Ainvw,
              (const float2*)f, c.tc_partial, (float2*)u, c.tc_err, active);
  if (split > 1)
    launch_smem(k_coarse_gemm_reduce, dim3((unsigned)(((long long)n * R + 255) / 256)), dim3(256), 0, s, n, R, split,
                (const float*)c.tc_partial, (float2*)u, active);
  HZ_LAUNCHED();
}

}  // namespace hz
