// Coarsest-level solve of a multi-RHS V-cycle on the tensor cores (Algorithm
// 1 step 3, exact solve by the dense inverse from setup): U = Ainv F with R
// right-hand sides (R = 16, 32 or 64), complex FP32 data, as one real GEMM
// with the complex structure on the small operand:
//
//   [Ur | Ui] (n x 2R) = [Ar Ai interleaved] (n x 2n) B (2n x 2R),
//   B[2j][r] = Fr, B[2j][R+r] = Fi, B[2j+1][r] = -Fi, B[2j+1][R+r] = Fr   (F = F[j][r])
//
// so the inverse enters as it is stored (each complex entry two reals, no
// duplication), on tcgen05 (kind::tf32, FP32 accumulation in tensor memory)
// with the 3xTF32 split: x = x_hi + x_lo with both parts tf32, x y ~ x_hi y_hi
// + x_hi y_lo + x_lo y_hi (relative error about 2^-22, at the level of the
// FP32 CUDA-core product it replaces).
//
// Operand images.  The inverse never changes after setup, so its split halves
// are written once, tile by tile, in the exact shared-memory layout the MMA
// reads (K-major, no swizzle; tc_ops.cuh): block (row tile t, K chunk c) =
// 128 rows x 32 real columns of hi, then of lo, 32 KB contiguous.  B is
// written the same way by a small kernel before each product (2R rows x 32
// columns per chunk).  The product kernel moves whole blocks with bulk
// copies (the TMA's non-tensor form) into a ring of shared-memory stages,
// counted on one mbarrier per stage; one thread drives the ring and issues the
// 12 MMAs of a chunk (4 K-steps x 3 split products), whose commit frees the
// stage.  A CTA owns one tile of 128 complex rows and all 2R columns; with K
// split s ways the CTAs of a tile write FP32 partial sums that a second kernel
// adds in split order (deterministic).
#include "common.cuh"
#include "tc_ops.cuh"

namespace hz {
namespace {

constexpr int kTcThreads = 128, kTcM = 128, kTcK = 32, kStages = 3;
constexpr int kTileFloats = kTcM * kTcK;                       // one 16 KB operand tile of the inverse
constexpr long long kTcWaitPolls = 20000000LL;                 // seconds of polling: far beyond any copy or MMA
constexpr int kTcMaxN = 4096;                                  // coarsest sizes given an image (<= 134 MB)

__host__ __device__ inline int tc_chunks(int n) { return (n + 15) / 16; }      // 32 real columns = 16 complex
__host__ __device__ inline int tc_tiles(int n) { return (n + kTcM - 1) / kTcM; }
__host__ __device__ inline uint32_t tc_fblock_bytes(int R) { return 2u * (uint32_t)(2 * R) * kTcK * 4u; }
__host__ __device__ inline uint32_t tc_stage_bytes(int R) { return 2u * kTileFloats * 4u + tc_fblock_bytes(R); }

// the split image of the inverse viewed as n x 2n reals: one thread per
// (tile, chunk, row, column)
__global__ void k_build_a_image(int n, const float2* __restrict__ A, float* __restrict__ img) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)kTcM * kTcK;
  const long long total = (long long)tc_tiles(n) * tc_chunks(n) * per;
  if (e >= total) return;
  const long long blk = e / per;
  const int w = (int)(e - blk * per), m = w / kTcK, k = w - m * kTcK;
  const int t = (int)(blk / tc_chunks(n)), c = (int)(blk - (long long)t * tc_chunks(n));
  const int i = t * kTcM + m, gk = c * kTcK + k, j = gk >> 1;
  float x = 0.f;
  if (i < n && j < n) {
    const float2 v = A[(long long)i * n + j];
    x = (gk & 1) ? v.y : v.x;
  }
  const float hi = tc::tf32_rna(x), lo = tc::tf32_rna(x - hi);
  float* base = img + blk * 2 * per;
  const int off = tc::kmajor_offset<kTcK>(m, k) / 4;
  base[off] = hi;
  base[per + off] = lo;
}

// the split image of B for R right-hand sides: one thread per (chunk, output
// column nn < 2R, K column k); row k = 2 lj + b of chunk c multiplies the
// real (b = 0) or imaginary (b = 1) part of the inverse's column j = 16 c + lj
__global__ void k_build_f_image(int n, int R, const float2* __restrict__ F, float* __restrict__ img,
                                const int* active) {
  pdl_enter();
  if (active && !*active) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)2 * R * kTcK;
  if (e >= (long long)tc_chunks(n) * per) return;
  const int c = (int)(e / per), w = (int)(e - (long long)c * per), nn = w / kTcK, k = w - nn * kTcK;
  const int j = c * 16 + (k >> 1), b = k & 1, r = nn < R ? nn : nn - R;
  const float2 v = j < n ? F[(long long)j * R + r] : make_float2(0.f, 0.f);
  // b = 0: (Fr | Fi); b = 1: (-Fi | Fr)
  const float x = nn < R ? (b ? -v.y : v.x) : (b ? v.x : v.y);
  const float hi = tc::tf32_rna(x), lo = tc::tf32_rna(x - hi);
  float* base = img + (long long)c * 2 * per;
  const int off = tc::kmajor_offset<kTcK>(nn, k) / 4;
  base[off] = hi;
  base[per + off] = lo;
}

__global__ void __launch_bounds__(kTcThreads) k_coarse_gemm_tc(int n, int R, int split, const float* __restrict__ aimg,
                                                               const float* __restrict__ fimg,
                                                               float* __restrict__ part, float2* __restrict__ U,
                                                               int* err, const int* active) {
  extern __shared__ unsigned char smraw[];
  __shared__ uint64_t full[kStages], empty[kStages];
  __shared__ uint32_t taddr_s;
  __shared__ int ok_s;
  pdl_enter();
  if (active && !*active) return;
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t SB = tc_stage_bytes(R), FB = tc_fblock_bytes(R);
  const uint32_t cols = (uint32_t)(2 * R);                // 32, 64 or 128 accumulator columns
  const int tile = blockIdx.x, sidx = blockIdx.y;
  const int nch = tc_chunks(n);
  const int per = (nch + split - 1) / split;
  const int c0 = min(sidx * per, nch), c1 = min(c0 + per, nch), nl = c1 - c0;
  if (warp == 0) tc::tmem_alloc(&taddr_s, cols);
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    ok_s = 1;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = taddr_s;
  if (tid == 0 && nl > 0) {
    const uint32_t idesc = tc::idesc_tf32(kTcM, 2 * R);
    const uint32_t sbo_a = 128 * kTcK / 4, sbo_b = 128 * kTcK / 4;
    auto load = [&](int L) {                          // chunk c0 + L into stage L % kStages
      const int st = L % kStages, c = c0 + L;
      unsigned char* dst = sm + st * SB;
      tc::mbar_expect_tx(&full[st], SB);
      const long long ab = HZ_AT((long long)tile * nch + c, (long long)tc_tiles(n) * nch);   // image block
      tc::bulk_g2s(dst, aimg + ab * 2 * kTileFloats, 2 * kTileFloats * 4, &full[st]);
      tc::bulk_g2s(dst + 2 * kTileFloats * 4, fimg + (long long)HZ_AT(c, nch) * (FB / 4), FB, &full[st]);
    };
    int loaded = 0;                                   // chunks whose copies were issued
    for (; loaded < kStages && loaded < nl; ++loaded) load(loaded);
    bool ok = true;
    int issued = 0;                                   // chunks whose MMAs were committed
    for (int L = 0; L < nl && ok; ++L) {
      const int st = L % kStages;
      const uint32_t ph = (uint32_t)(L / kStages) & 1;
      if (!tc::mbar_wait(&full[st], ph, kTcWaitPolls)) {
        ok = false;
        break;
      }
      tc::fence_after_sync();
      const uint32_t a_hi = tc::smem_u32(sm + st * SB), a_lo = a_hi + kTileFloats * 4;
      const uint32_t b_hi = a_hi + 2 * kTileFloats * 4, b_lo = b_hi + FB / 2;
#pragma unroll
      for (int k = 0; k < kTcK / 8; ++k) {
        const uint64_t ah = tc::smem_desc(a_hi + 256 * k, 128, sbo_a);
        const uint64_t al = tc::smem_desc(a_lo + 256 * k, 128, sbo_a);
        const uint64_t bh = tc::smem_desc(b_hi + 256 * k, 128, sbo_b);
        const uint64_t bl = tc::smem_desc(b_lo + 256 * k, 128, sbo_b);
        tc::mma_tf32(taddr, ah, bh, idesc, L > 0 || k > 0);
        tc::mma_tf32(taddr, ah, bl, idesc, true);
        tc::mma_tf32(taddr, al, bh, idesc, true);
      }
      tc::mma_commit(&empty[st]);
      issued = L + 1;
      if (L + kStages < nl) {
        // the stage is refilled once its MMAs have read it
        if (!tc::mbar_wait(&empty[st], ph, kTcWaitPolls)) {
          ok = false;
          break;
        }
        load(L + kStages);
        ++loaded;
      }
    }
    // every MMA done: the last commit completes after all earlier ones; a
    // wait that gave up is recorded (after one more bounded wait for the
    // MMAs in flight) and the result is left alone
    if (ok && !tc::mbar_wait(&empty[(issued - 1) % kStages], (uint32_t)((issued - 1) / kStages) & 1, kTcWaitPolls))
      ok = false;
    if (!ok) {
      atomicExch(err, 1);
      if (issued > 0)
        tc::mbar_wait(&empty[(issued - 1) % kStages], (uint32_t)((issued - 1) / kStages) & 1, kTcWaitPolls);
      // copies issued but not yet consumed must land before the CTA leaves
      for (int L = issued; L < loaded; ++L)
        tc::mbar_wait(&full[L % kStages], (uint32_t)(L / kStages) & 1, kTcWaitPolls);
      ok_s = 0;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (ok_s) {
    const int i = tile * kTcM + 32 * warp + lane;     // complex row held by this thread
    const bool rowok = i < n;
    // columns c < R are Re U[i][c], columns R + c are Im U[i][c]
    for (int c = 0; c < R; c += 16) {
      float re[16], im[16];
      if (nl > 0) {
        tc::tmem_ld16(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, re);
        tc::tmem_ld16(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)(R + c), im);
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) re[q] = im[q] = 0.f;
      }
      if (!rowok) continue;
      if (split == 1) {
#pragma unroll
        for (int q = 0; q < 16; ++q) U[HZ_AT((long long)i * R + c + q, (long long)n * R)] = make_float2(re[q], im[q]);
      } else {
        float* pp = part + HZ_AT(((long long)sidx * n + i) * 2 * R, (long long)split * n * 2 * R);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          pp[c + q] = re[q];
          pp[R + c + q] = im[q];
        }
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
    const float* pp = part + ((long long)s * n + i) * 2 * R;
    re += pp[r];
    im += pp[R + r];
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

size_t tc_smem(int R) { return 1024 + (size_t)kStages * tc_stage_bytes(R); }

}  // namespace

// The bounded wait of the tensor-core kernels on its own: one thread waits
// `polls` times for phase 0 of a fresh mbarrier (count 1) and records in
// *err whether it gave up; with arrive != 0 it first arrives itself, so the
// phase completes and the wait succeeds at once.
__global__ void k_wait_probe(long long polls, int arrive, int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  tc::mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (arrive) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(tc::smem_u32(&bar))
                 : "memory");
  }
  *err = tc::mbar_wait(&bar, 0, polls) ? 0 : 1;
}

bool coarse_tc_supported(const Ctx& c, int nrhs) {
  return c.mixed && (nrhs == 16 || nrhs == 32 || nrhs == 64) && c.tc_err != nullptr && c.tc_image != nullptr &&
         nrhs <= c.opts.nrhs_max;
}

size_t coarse_tc_bytes(long long n, int nrhs_max) {
  if (n > kTcMaxN || nrhs_max < 16) return 0;
  const size_t img = sizeof(float) * 2 * (size_t)kTileFloats * tc_tiles((int)n) * tc_chunks((int)n);
  const size_t fimg = (size_t)tc_chunks((int)n) * tc_fblock_bytes(nrhs_max);
  const size_t part = sizeof(float) * kTcMaxSplit * (size_t)n * 2 * nrhs_max;
  return img + fimg + part + 256;
}

void coarse_tc_alloc(Ctx& c) {
  const Level& L = c.L.back();
  const int R = c.opts.nrhs_max;
  if (!c.mixed || R < 16 || L.g.N > kTcMaxN) return;
  const int n = (int)L.g.N;
  const long long elems = (long long)tc_tiles(n) * tc_chunks(n) * kTileFloats;
  c.tc_image = (float*)ctx_alloc(c, sizeof(float) * 2 * elems);
  c.tc_fimg = (float*)ctx_alloc(c, (size_t)tc_chunks(n) * tc_fblock_bytes(R));
  c.tc_partial = (float*)ctx_alloc(c, sizeof(float) * kTcMaxSplit * 2 * (size_t)n * R);
  c.tc_err = (int*)ctx_alloc(c, sizeof(int));
  HZ_CUDA(cudaMemsetAsync(c.tc_err, 0, sizeof(int), c.alloc_stream));
  k_build_a_image<<<(unsigned)((elems + 255) / 256), 256, 0, c.alloc_stream>>>(n, (const float2*)L.Ainvw, c.tc_image);
  HZ_CUDA(cudaGetLastError());
}

void coarse_gemm_tc(Ctx& c, const void* f, void* u, const int* active, cudaStream_t s, int split) {
  const Level& L = c.L.back();
  const int n = (int)L.g.N, R = c.nrhs;
  require(coarse_tc_supported(c, R), "tensor-core coarsest solve: mixed precision, 16/32/64 right-hand sides");
  require(split >= 1 && split <= kTcMaxSplit, "tensor-core split out of range");
  static bool attr_set[256] = {};
  if (!attr_set[c.dev & 255]) {
    HZ_CUDA(cudaFuncSetAttribute(k_coarse_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem(64)));
    attr_set[c.dev & 255] = true;
  }
  const long long fe = (long long)tc_chunks(n) * 2 * R * kTcK;
  launch_smem(k_build_f_image, dim3((unsigned)((fe + 255) / 256)), dim3(256), 0, s, n, R, (const float2*)f, c.tc_fimg,
              active);
  const dim3 grid((unsigned)tc_tiles(n), (unsigned)split);
  launch_smem(k_coarse_gemm_tc, grid, dim3(kTcThreads), tc_smem(R), s, n, R, split, (const float*)c.tc_image,
              (const float*)c.tc_fimg, c.tc_partial, (float2*)u, c.tc_err, active);
  if (split > 1)
    launch_smem(k_coarse_gemm_reduce, dim3((unsigned)(((long long)n * R + 255) / 256)), dim3(256), 0, s, n, R, split,
                (const float*)c.tc_partial, (float2*)u, active);
  HZ_LAUNCHED();
}

}  // namespace hz

using namespace hz;

extern "C" hz_status hz_check_wait_timeout(long long polls, int arrive, int* timed_out) {
  return guarded([&] {
    require(timed_out != nullptr, "null output");
    require(polls >= 1 && polls <= (1ll << 24), "polls must be in 1..2^24");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) throw Error(HZ_ERR_NO_DEVICE, "no CUDA device");
    cudaStream_t s;
    HZ_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    int* err = nullptr;
    HZ_CUDA(counted_malloc_async(&err, sizeof(int), s));
    HZ_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    k_wait_probe<<<1, 32, 0, s>>>(polls, arrive, err);
    HZ_CUDA(cudaGetLastError());
    int h = 0;
    HZ_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    HZ_CUDA(cudaFreeAsync(err, s));
    HZ_CUDA(cudaStreamSynchronize(s));
    cudaStreamDestroy(s);
    *timed_out = h;
    if (h) throw Error(HZ_ERR_TIMEOUT, "the bounded device wait gave up (no arrival on the barrier)");
  });
}
