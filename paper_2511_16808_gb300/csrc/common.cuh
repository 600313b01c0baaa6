// Internal definitions shared by the CUDA translation units of libhz.
//
// Layout in HBM (one context):
//   level fields       interleaved complex, node-major, x fastest; with R
//                      right-hand sides the RHS index is innermost
//   stencils           plane-major ("SoA"): entry s of node p at [s*N + p], so a
//                      warp reading one entry of 32 consecutive nodes issues one
//                      coalesced 256 B (c64) / 512 B (c128) request
//   fine level         only the complex diagonal of A_s is stored; the 2d
//                      off-diagonal couplings -prod_{a'!=a} w_a'/h^2 follow from
//                      the node's coordinates (half-cell weights of Section 2.1)
//   coarse levels      full box stencils of radius rho (Galerkin products)
//   Vanka smoother     the assembled sum M = sum_i V_i^T W_i H_i^{-1} V_i as a
//                      per-node stencil over the offsets d_l - d_k of the patch
//                      (Eq. smoother); a sweep is a gather, conflict-free
#pragma once
#include <cstring>
#include <utility>
#include <new>
#include <stdexcept>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <array>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <mutex>
#include <vector>

#include "hz.h"

namespace hz {

struct Error : std::runtime_error {
  hz_status code;
  Error(hz_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define HZ_CUDA(call)                                                                        \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      (void)cudaGetLastError();                                                              \
      throw ::hz::Error(e_ == cudaErrorMemoryAllocation ? HZ_ERR_OOM : HZ_ERR_CUDA,          \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                 \
    }                                                                                        \
  } while (0)

#define HZ_LAUNCHED() HZ_CUDA(cudaGetLastError())

inline void require(bool ok, const std::string& what) {
  if (!ok) throw Error(HZ_ERR_INVALID_ARG, what);
}

// ---------------------------------------------------------------- checked build
// Built with -DHZ_CHECKED (build.py --checked: libhz_checked.so), every
// instrumented global access of the solve's kernels tests its element index
// against the extent of the array it reads or writes.  An index outside
// [0, n) is counted in a device word of the translation unit, the first one
// is recorded (source line, index), and the access is moved to element 0, so
// it stays inside the array: the kernel runs on and never traps.
// hz_check_status reads (and may clear) the words of every translation unit.
// Without HZ_CHECKED, HZ_AT(i, n) is i and HZ_EXT(n) is empty: no cost.
void check_register(int (*read)(unsigned long long* words, int clear));
#ifdef HZ_CHECKED
static __device__ unsigned long long hz_chk_words[2];   // failures; first (line << 40 | index bits)
__device__ __forceinline__ long long hz_chk(long long i, long long n, unsigned line) {
  if (i >= 0 && i < n) return i;
  if (atomicAdd(&hz_chk_words[0], 1ull) == 0ull)
    hz_chk_words[1] = ((unsigned long long)line << 40) | ((unsigned long long)i & 0xffffffffffull);
  return 0;
}
#define HZ_AT(i, n) ::hz::hz_chk((long long)(i), (long long)(n), __LINE__)
#define HZ_EXT(n) , hz_ext = (long long)(n)
static int hz_chk_read(unsigned long long* w, int clear) {
  if (cudaMemcpyFromSymbol(w, hz_chk_words, sizeof(hz_chk_words)) != cudaSuccess) return -1;
  if (clear) {
    const unsigned long long z[2] = {0ull, 0ull};
    if (cudaMemcpyToSymbol(hz_chk_words, z, sizeof(z)) != cudaSuccess) return -1;
  }
  return 0;
}
static const int hz_chk_registered = (check_register(hz_chk_read), 0);
#else
#define HZ_AT(i, n) (i)
#define HZ_EXT(n)
#endif

// ---------------------------------------------------------------- complex
template <typename T> struct cplx;
template <> struct cplx<float> { using t = float2; };
template <> struct cplx<double> { using t = double2; };
template <typename T> using c_t = typename cplx<T>::t;

template <typename V> __host__ __device__ __forceinline__ V cmk(double re, double im);
template <> __host__ __device__ __forceinline__ float2 cmk<float2>(double re, double im) {
  return make_float2((float)re, (float)im);
}
template <> __host__ __device__ __forceinline__ double2 cmk<double2>(double re, double im) {
  return make_double2(re, im);
}

__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }

__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc + a*b
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
  return acc;
}
// conj(a)*b
__host__ __device__ __forceinline__ double2 cconjmul(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

__device__ __forceinline__ double2 to_c128(double2 a) { return a; }
__device__ __forceinline__ double2 to_c128(float2 a) { return make_double2(a.x, a.y); }
template <typename V> __device__ __forceinline__ V from_c128(double2 a);
template <> __device__ __forceinline__ double2 from_c128<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 from_c128<float2>(double2 a) {
  return make_float2((float)a.x, (float)a.y);
}

// float <-> double on the integer pipe.  GB300 executes FP64 instructions,
// conversions included, at 1/64 of the FP32 rate, and converting the FP32
// preconditioned vectors for the FP64 Krylov passes saturated that pipe.
// These repack sign / exponent / mantissa with integer operations only (no
// hardware conversion on any path, so none is issued speculatively either)
// and give exactly the IEEE results: f2d_exact is the exact widening
// (subnormals normalised, infinities and NaN payloads kept), d2f_rn the
// narrowing with round to nearest even, including subnormal results and
// overflow to infinity.  Host-callable so that they can be checked bit for bit
// against the host's conversions.
__host__ __device__ __forceinline__ unsigned f_bits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  unsigned u;
  memcpy(&u, &f, 4);
  return u;
#endif
}
__host__ __device__ __forceinline__ float bits_f(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}
__host__ __device__ __forceinline__ double hilo_d(unsigned hi, unsigned lo) {
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  const unsigned long long b = ((unsigned long long)hi << 32) | lo;
  double d;
  memcpy(&d, &b, 8);
  return d;
#endif
}
__host__ __device__ __forceinline__ void d_hilo(double d, unsigned& hi, unsigned& lo) {
#ifdef __CUDA_ARCH__
  hi = (unsigned)__double2hiint(d);
  lo = (unsigned)__double2loint(d);
#else
  unsigned long long b;
  memcpy(&b, &d, 8);
  hi = (unsigned)(b >> 32);
  lo = (unsigned)b;
#endif
}
__host__ __device__ __forceinline__ int clz32(unsigned m) {
#ifdef __CUDA_ARCH__
  return __clz((int)m);
#else
  return m ? __builtin_clz(m) : 32;
#endif
}

__host__ __device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = f_bits(f);
  const unsigned e = (u >> 23) & 0xffu;
  unsigned m = u & 0x7fffffu;
  unsigned E;                                   // double exponent field
  if (e == 0u) {
    // zero or subnormal m * 2^-149: leading one at bit k -> 1.frac * 2^(k-149)
    const int k = 31 - clz32(m);
    E = m ? (unsigned)(k + 874) : 0u;
    m = m ? (m << (23 - k)) & 0x7fffffu : 0u;
  } else {
    E = e == 0xffu ? 0x7ffu : e + 896u;
  }
  return hilo_d((u & 0x80000000u) | (E << 20) | (m >> 3), m << 29);
}

__host__ __device__ __forceinline__ float d2f_rn(double d) {
  unsigned hi, lo;
  d_hilo(d, hi, lo);
  const unsigned sign = hi & 0x80000000u;
  const int E = (int)((hi >> 20) & 0x7ffu);
  const unsigned mh = hi & 0xfffffu;
  if (E == 0x7ff) {                             // infinity / NaN (quiet, payload kept)
    const unsigned nan = (mh | lo) ? (0x400000u | (mh << 3) | (lo >> 29)) : 0u;
    return bits_f(sign | 0x7f800000u | nan);
  }
  const int e = E - 896;                        // float exponent field
  if (e >= 255) return bits_f(sign | 0x7f800000u);
  if (e >= 1) {
    const unsigned m = (mh << 3) | (lo >> 29);  // 23-bit mantissa
    const unsigned rem = lo & 0x1fffffffu;      // 29 dropped bits
    unsigned bits = ((unsigned)e << 23) | m;
    bits += (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;   // carry may reach exponent
    return bits_f(sign | bits);
  }
  // subnormal (or zero) result: drop 30 - e bits of the 53-bit significand
  const int shift = 30 - e;
  if (E == 0 || shift >= 54) return bits_f(sign);
  const unsigned long long M = ((unsigned long long)(mh | 0x100000u) << 32) | lo;
  const unsigned q = (unsigned)(M >> shift);
  const unsigned long long rem = M & ((1ull << shift) - 1ull), half = 1ull << (shift - 1);
  const unsigned up = (rem > half || (rem == half && (q & 1u))) ? 1u : 0u;
  return bits_f(sign | (q + up));               // a carry gives the smallest normal
}

// ---------------------------------------------------------------- grid
struct GridDev {
  int dim;
  int nx, ny, nz;     // nz = 1 in 2D
  long long N;
};

inline GridDev make_grid(int dim, const int n[3]) {
  GridDev g;
  g.dim = dim;
  g.nx = n[0];
  g.ny = n[1];
  g.nz = dim == 3 ? n[2] : 1;
  g.N = (long long)g.nx * g.ny * g.nz;
  return g;
}

// Half-cell weight of index i on an axis of n nodes (Section 2.1 boundary rows).
__host__ __device__ __forceinline__ double wgt(int i, int n) { return (i == 0 || i == n - 1) ? 0.5 : 1.0; }

// 1D prolongation weight P(j, J): fine node j, coarse node J (fine node 2J),
// kind 0 = linear (Eq. biliniearIntergrid), 1 = cubic (Eq. bicubicIntergrid),
// with P = 2 R^T per axis.  The cubic rule needs c_{-1} and c_{nc} at the two
// ends; they are mirrored (c_{-1} := c_1, c_{nc} := c_{nc-2}).
__host__ __device__ __forceinline__ double p1(int kind, int nf, int nc, int j, int J) {
  int d = j - 2 * J;
  int ad = d < 0 ? -d : d;
  double w;
  if (kind == 0) {
    w = ad == 0 ? 1.0 : (ad == 1 ? 0.5 : 0.0);
  } else {
    w = ad == 0 ? 0.75 : (ad == 1 ? 0.5 : (ad == 2 ? 0.125 : 0.0));
    if (j == 0 && J == 1) w += 0.125;
    if (j == nf - 1 && J == nc - 2) w += 0.125;
  }
  return w;
}
// 1D restriction weight R(J, j) = P(j, J) / 2.
__host__ __device__ __forceinline__ double r1(int kind, int nf, int nc, int J, int j) {
  return 0.5 * p1(kind, nf, nc, j, J);
}
__host__ __device__ __forceinline__ int transfer_radius(int kind) { return kind ? 2 : 1; }

// ---------------------------------------------------------------- stencils
constexpr int kLutR = 3;                       // offsets in [-3, 3]^3
constexpr int kLutW = 2 * kLutR + 1;
constexpr int kLutN = kLutW * kLutW * kLutW;   // 343

__host__ __device__ __forceinline__ int lut_index(int dx, int dy, int dz) {
  return ((dz + kLutR) * kLutW + (dy + kLutR)) * kLutW + (dx + kLutR);
}

// Offsets of a stencil, passed by value to kernels (lives in parameter space).
struct StencilOff {
  int n;
  int rho;                                     // max |offset| over axes
  signed char d[HZ_MAX_STENCIL][3];
};
// Offsets plus an offset -> entry lookup, for setup kernels.
struct StencilLut {
  StencilOff off;
  short lut[kLutN];
};

StencilLut make_lut(const std::vector<std::array<int, 3>>& offs);
std::vector<std::array<int, 3>> fine_offsets(int dim);
std::vector<std::array<int, 3>> box_offsets(int dim, int rho);
std::vector<std::array<int, 3>> patch_offsets(int dim, hz_patch kind);
std::vector<std::array<int, 3>> patch_difference_offsets(int dim, hz_patch kind);

// ---------------------------------------------------------------- dependent launch
// Programmatic dependent launch (Blackwell / Hopper): the kernels of the
// solver's chains (V-cycle steps, Gram-Schmidt passes) are launched with
// programmatic stream serialization, so the next kernel is launched and its
// blocks become resident while the previous one drains; every such kernel
// first waits for its predecessor's completion and memory (griddepcontrol.wait,
// a hardware dependency, returning at once when there is none), then allows
// its own successor to start launching.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// L2 prefetch of elements [e0, e1] of a (one request per 128-byte line, every
// address inside the run).  Kernels issue it before pdl_enter() for operands
// written at setup (stencil planes, the coarsest inverse): with programmatic
// dependent launch the block is often resident while its predecessor still
// runs, so those lines travel from HBM to L2 during the predecessor instead
// of after it.
template <typename V>
__device__ __forceinline__ void prefetch_l2_run(const V* a, long long e0, long long e1) {
  const char* p0 = reinterpret_cast<const char*>(a + e0);
  const char* p1 = reinterpret_cast<const char*>(a + e1);
  const char* q = p0;
  for (; q <= p1; q += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(q));
  if (((uintptr_t)(q - 128) >> 7) != ((uintptr_t)p1 >> 7)) asm volatile("prefetch.global.L2 [%0];" ::"l"(p1));
}

// elements [e0, e1] of a, the lines spread over nth threads
template <typename V>
__device__ __forceinline__ void prefetch_l2_span(const V* a, long long e0, long long e1, int tid, int nth) {
  const char* p0 = reinterpret_cast<const char*>(a + e0);
  const char* p1 = reinterpret_cast<const char*>(a + e1);
  const long long lines = ((long long)(p1 - p0) >> 7) + 1;
  for (long long k = tid; k < lines; k += nth) asm volatile("prefetch.global.L2 [%0];" ::"l"(p0 + (k << 7)));
  if (tid == 0) asm volatile("prefetch.global.L2 [%0];" ::"l"(p1));
}

// The rows [y0, y0 + ny) x columns [x0, x0 + nx) of np planes of an nxg x nyg
// grid (plane stride N elements), clipped to the grid, one (plane, row) per
// thread step.
// Element run [e0, e1] (from P) of task `task` = (plane s, row y0 + r) of a
// plane-row prefetch, clipped to the grid; false when the row or the columns
// lie outside it.  Host-callable so the clipping can be checked on the CPU.
__host__ __device__ inline bool plane_row_run(int task, long long N, int nxg, int nyg, int x0, int nx, int y0, int ny,
                                              long long& e0, long long& e1) {
  const int xa = x0 > 0 ? x0 : 0, xb = (x0 + nx < nxg ? x0 + nx : nxg) - 1;
  const int s = task / ny, y = y0 + (task - s * ny);
  if (xb < xa || y < 0 || y >= nyg) return false;
  const long long row = (long long)s * N + (long long)y * nxg;
  e0 = row + xa;
  e1 = row + xb;
  return true;
}

template <typename V>
__device__ __forceinline__ void prefetch_l2_planes(const V* P, int np, long long N, int nxg, int nyg, int x0, int nx,
                                                   int y0, int ny, int tid, int nth) {
  for (int task = tid; task < np * ny; task += nth) {
    long long e0, e1;
    if (plane_row_run(task, N, nxg, nyg, x0, nx, y0, ny, e0, e1)) prefetch_l2_run(P, e0, e1);
  }
}

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  HZ_CUDA(cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...));
}

// ---------------------------------------------------------------- errors at the ABI
// The message of the calling thread's last failed call (api.cu).
void set_last_error(const char* msg);

// Runs f; converts exceptions into a status and the thread's last message.
template <typename F>
hz_status guarded(F&& f) {
  try {
    f();
    set_last_error(nullptr);
    return HZ_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    return HZ_ERR_OOM;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return HZ_ERR_CUDA;
  } catch (...) {
    set_last_error("unknown error");
    return HZ_ERR_CUDA;
  }
}

// ---------------------------------------------------------------- compact stencil
// Coefficients of the compact fourth-order stencils (Section 2.1) by the
// number m of nonzero offset components: L (times 1/h^2) and the mass M.
//   2D (Eq. disc4thCompact):   L = 10/3, -2/3, -1/6;      M = 2/3, 1/12, 0
//   3D (Eq. disc4thCompact3D): L = 4, -1/3, -1/6, 0;      M = 1/2, 1/12, 0, 0
__host__ __device__ __forceinline__ double compact_L(int dim, int m) {
  if (dim == 2) return m == 0 ? 10.0 / 3.0 : (m == 1 ? -2.0 / 3.0 : -1.0 / 6.0);
  return m == 0 ? 4.0 : (m == 1 ? -1.0 / 3.0 : (m == 2 ? -1.0 / 6.0 : 0.0));
}
__host__ __device__ __forceinline__ double compact_M(int dim, int m) {
  if (m == 0) return dim == 2 ? 2.0 / 3.0 : 0.5;
  return m == 1 ? 1.0 / 12.0 : 0.0;
}

// The compact operator at node p = (x, y, z) in FP64 with a variable medium
// (reading: L - (Sigma M + M Sigma)/2, neighbours outside the grid dropped):
//   (A v)_p = (1/h^2) (L v)_p - (s_p (M v)_p + (M (s v))_p) / 2,  s = sig + dsig
// (dsig = -i alpha omega^2 gives the shifted operator).  ld(q) returns v at node q.
template <typename LD>
__device__ __forceinline__ double2 compact_Av(int nx, int ny, int nz, int dim, double invh2,
                                              const double2* __restrict__ sig, double2 dsig, const LD& ld,
                                              long long p, int x, int y, int z) {
  double2 Lv = make_double2(0, 0), Mv = make_double2(0, 0), Msv = make_double2(0, 0);
  const int zr = dim == 3 ? 1 : 0;
  for (int dz = -zr; dz <= zr; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int m = (dx != 0) + (dy != 0) + (dz != 0);
        const double cl = compact_L(dim, m), cm = compact_M(dim, m);
        if (cl == 0.0 && cm == 0.0) continue;
        const int xx = x + dx, yy = y + dy, zz = z + dz;
        if (xx < 0 || xx >= nx || yy < 0 || yy >= ny || zz < 0 || zz >= nz) continue;
        const long long q = p + dx + (long long)dy * nx + (long long)dz * nx * ny;
        const double2 v = ld(q);
        Lv.x = fma(cl, v.x, Lv.x);
        Lv.y = fma(cl, v.y, Lv.y);
        if (cm != 0.0) {
          const double2 sq = make_double2(sig[q].x + dsig.x, sig[q].y + dsig.y);
          Mv.x = fma(cm, v.x, Mv.x);
          Mv.y = fma(cm, v.y, Mv.y);
          const double2 sv = make_double2(sq.x * v.x - sq.y * v.y, sq.x * v.y + sq.y * v.x);
          Msv.x = fma(cm, sv.x, Msv.x);
          Msv.y = fma(cm, sv.y, Msv.y);
        }
      }
  const double2 sp = make_double2(sig[p].x + dsig.x, sig[p].y + dsig.y);
  const double2 sMv = make_double2(sp.x * Mv.x - sp.y * Mv.y, sp.x * Mv.y + sp.y * Mv.x);
  return make_double2(invh2 * Lv.x - 0.5 * (sMv.x + Msv.x), invh2 * Lv.y - 0.5 * (sMv.y + Msv.y));
}

// ---------------------------------------------------------------- context
struct Level {
  GridDev g;
  bool fine = false;            // the analytic 5-/7-point fine operator (level 0 without the compact stencil)
  bool coarsest = false;
  bool a_sym = false;           // A_s of this level is complex symmetric
  bool a_half = false;          // working copy Aw holds the planes s >= 0 only (symmetric box)
  // operator A_s at this level
  StencilLut A;                 // fine: the 2d+1 point offsets; coarse: box of radius rho
  double2* A64 = nullptr;       // FP64 planes [A.n][N] (setup; kept for export when asked)
  void* Aw = nullptr;           // working precision: fine = diag of A_s [N]; coarse = planes
  // smoother
  hz_patch patch = HZ_PATCH_JACOBI;
  double damping = 1.0;
  StencilLut M;                 // offsets of the assembled Vanka sum (zero planes dropped)
  double2* M64 = nullptr;       // FP64 planes [M.n][N]
  void* Mw = nullptr;           // working precision planes (diagonal M only)
  // M in half form: every patch weight is 1/count of its node, so M = D^{-1} M'
  // with M' = sum_i V_i^T H_i^{-1} V_i, complex symmetric where A_s is (then
  // H_i = H_i^T; Section 3.2).  Stored: 1/count per node and the planes of M'
  // at the offsets s >= 0 (lexicographic, z then y then x), M'(p, p - s) being
  // read as M'(p - s, p) at node p - s; on levels whose operator is not
  // symmetric the planes of M itself are kept (no weights, nothing mirrored).
  StencilLut Mh;                // offsets of the stored half
  unsigned char mh_mirror[HZ_MAX_STENCIL] = {};   // 1: offset -s is stored as s
  void* Mhw = nullptr;          // working precision planes [Mh.n][N]
  void* wcw = nullptr;          // working precision 1/count per node [N] (real); null: Mhw holds M
  // transfers to the next coarser level (0 = linear, 1 = cubic)
  int rkind = 0, pkind = 0;
  // work vectors, working precision, N * nrhs_max
  void* u = nullptr;             // cycle output on coarse levels
  void* f = nullptr;             // right-hand side
  void* r = nullptr;             // residual
  void* t = nullptr;             // pre-smoothed iterate (the post-smoothing writes the output)
  bool m_diag = false;           // assembled Vanka sum is diagonal (Jacobi / RB on 2d+1 points)
  // kernel choices set by the autotuner (hz_autotune / hz_tune_set); the
  // defaults follow fixed rules (batch width, level size)
  int tune_vr = 0;               // RHS pack: 0 rule, 1 one value per thread, 2 packs of 32 bytes
  int tune_mb = -1;              // one-RHS register budget: -1 rule, 0 occupancy, 2 two blocks per SM
  int tune_fuse = -1;            // fused tile passes of a small 2D level: -1 rule, 0 off, 1 on
  // coarsest level: dense inverse [N][N] row-major
  double2* Ainv64 = nullptr;
  void* Ainvw = nullptr;
};

struct KrylovState;              // device-side FGMRES state, krylov.cu

// NVTX range for the life of a scope (setup levels, solves, restart cycles);
// header-only NVTX3, a no-op unless a tool (nsys, ncu --nvtx) is attached
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct Ctx {
  hz_grid grid;
  hz_opts opts;
  double setup_seconds = 0;     // wall time of hz_setup (host, including the device work)
  // per status read of the last single-RHS solve (start, then every restart
  // cycle): iterations so far, true relative residual, Arnoldi estimate
  std::vector<std::array<double, 3>> history;
  std::mutex history_mu;        // hz_solve_history may read while a solve appends
  double omega = 0, alpha = 0, h = 0;
  int dev = 0;
  bool mixed = true;
  bool compact = false;         // compact fourth-order fine stencil (hz_opts.stencil = 1)
  int nrhs = 1;                 // right-hand sides of the current call (V-cycle batch width)
  std::vector<Level> L;
  double2* diagA64 = nullptr;   // fine, unshifted A diagonal (FGMRES matvec), c128 [N];
                                // with the compact stencil: sigma = kappa^2 omega^2 (1 - i gamma/omega) per node
  double* wmass = nullptr;      // fine prod_a w_a per node (q_hat = wmass * q) [N]
  // Krylov workspace (c128 unless noted), nrhs_max wide
  double2* V = nullptr;         // (m+1) vectors
  void* Z = nullptr;            // m vectors, working precision
  double2* qhat = nullptr;
  double2* p = nullptr;         // solution accumulator (copied to the caller's buffer)
  double2* qstage = nullptr;    // source staging for host sources
  double2* partials = nullptr;  // reduction partials [vector][block]
  KrylovState* ks = nullptr;    // device state, one per RHS
  void* ks_host = nullptr;      // pinned host copy of the status
  int red_blocks = 0;
  std::vector<void*> allocations;
  cudaStream_t alloc_stream = nullptr;   // stream of hz_setup: orders the context's allocations
  std::atomic<int> busy{0};
  cudaGraphExec_t cycle_graph = nullptr;
  cudaGraphExec_t batch_graph = nullptr;   // restart cycle for nrhs > 1
  int batch_graph_nrhs = 0, batch_graph_kernels = 0;
  int* n_active = nullptr;                 // right-hand sides still iterating (batched solve)
  int cycle_graph_nrhs = 0;
  cudaStream_t graph_stream = nullptr;   // library stream the solve runs on (graph capture needs one)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // status copies of the queued restart cycles: two slots (event, pinned
  // host copy) used in turn, so the next cycle can be queued before the
  // status of the one before it has been read
  cudaEvent_t ev_status = nullptr, ev_status_b = nullptr;
  int as_state = 0;                        // asynchronous solve: 0 idle, 1 in flight, 2 finished
  int as_before = 0;                       // iterations before the oldest queued cycle (profiling)
  int as_head = 0, as_pending = 0;         // slot of the oldest unread status; statuses queued
  int as_done_slot = 0;                    // slot whose status ended the solve
  bool as_replayed = false;
  int graph_kernels = 0;        // kernel nodes in the captured restart cycle
  // measurement hooks (hz_profile_select / hz_profile_read): CUDA events around
  // the launches of one kernel class inside the captured cycle
  int prof_class = 0;
  std::vector<cudaEvent_t> prof_ev;            // 2 per bracketed launch
  std::vector<int> prof_j;                     // inner iteration of each bracketed launch
  std::vector<double> prof_b, prof_f;          // algorithmic bytes / flops of each launch
  double prof_ms = 0, prof_bytes = 0, prof_flops = 0;
  long long prof_launches = 0;
  long long launches = 0;       // kernels launched by hz_solve on this context
  // coarsest solve of a batched cycle on the tensor cores (tc_gemm.cu):
  // FP32 partial sums of a split K [kTcMaxSplit][n][2 nrhs_max], operand
  // images, a device error word (set if a bounded wait gave up), and the
  // chosen variant per batch width: 0 CUDA-core GEMM, s >= 1 tensor cores
  // with K split s ways
  float* tc_partial = nullptr;
  float* tc_image = nullptr;    // split tf32 image of the real form of the coarsest inverse
  float* tc_fimg = nullptr;     // split image of the right-hand sides of one product
  int* tc_err = nullptr;
  int coarse_variant[7] = {-1, -1, -1, -1, -1, -1, -1};   // by log2(nrhs); -1: default rule
};

// Whether a cycle from zero at level l runs the fine level as two fused
// passes (cycle_impl.cuh k_fine_down_diag_*, k_fine_up_diag_*): level 0 with
// a diagonal smoother, one pre- and one post-sweep, one right-hand side.
inline bool fine_two_pass(const Ctx& c, int l) {
  const Level& L = c.L[l];
  return l == 0 && L.fine && !L.coarsest && L.m_diag && c.opts.nu1 == 1 && c.opts.nu2 == 1 && c.nrhs == 1 &&
         L.g.dim == 2;
}

// Whether a cycle from zero at coarse 2D level l runs as two fused tile
// passes (cycle_impl.cuh k_level_down_2d, k_level_up_2d): a small level
// (where launch and memory latency, not bandwidth, set the time), a stored operator
// of radius <= 3, a non-diagonal smoother of reach <= 2, one pre- and one
// post-sweep, one right-hand side.
inline bool level_two_pass_2d(const Ctx& c, int l) {
  const Level& L = c.L[l];
  return (L.tune_fuse >= 0 ? L.tune_fuse == 1 : L.g.N <= 70000) && !L.fine && !L.coarsest && !L.m_diag && L.g.dim == 2 && c.opts.nu1 == 1 && c.opts.nu2 == 1 &&
         c.nrhs == 1 && L.A.off.rho <= (L.a_half ? 2 : 3) && L.Mh.off.rho <= 2;
}

// Every device allocation of the library goes through counted_malloc_async,
// which counts them process-wide (hz_memory_stats reports the count).
std::atomic<unsigned long long>& device_alloc_count();
inline cudaError_t counted_malloc_async(void** p, size_t bytes, cudaStream_t s) {
  device_alloc_count().fetch_add(1);
  return cudaMallocAsync(p, bytes, s);
}
template <typename P>
inline cudaError_t counted_malloc_async(P** p, size_t bytes, cudaStream_t s) {
  return counted_malloc_async(reinterpret_cast<void**>(p), bytes, s);
}

// One host thread at a time per context: a second concurrent call gets HZ_ERR_BUSY.
struct BusyGuard {
  Ctx* c;
  explicit BusyGuard(Ctx* ctx) : c(ctx) {
    int expected = 0;
    if (!c->busy.compare_exchange_strong(expected, 1)) throw Error(HZ_ERR_BUSY, "context in use");
  }
  ~BusyGuard() { c->busy.store(0); }
  BusyGuard(const BusyGuard&) = delete;
  BusyGuard& operator=(const BusyGuard&) = delete;
};

// allocation helpers (all device memory of a context goes through these)
void* ctx_alloc(Ctx& c, size_t bytes);          // stream-ordered, on c.alloc_stream
void* ctx_alloc(Ctx& c, size_t bytes, cudaStream_t s);
void* pinned_small_alloc(size_t bytes);         // <= 4 KB pinned host block (shared arena)
void pinned_small_free(void* p);
void ctx_free_all(Ctx& c);

// tc_gemm.cu: coarsest multi-RHS solve on the tensor cores
constexpr int kTcMaxSplit = 16;
bool coarse_tc_supported(const Ctx& c, int nrhs);
void coarse_gemm_tc(Ctx& c, const void* f, void* u, const int* active, cudaStream_t s, int split);
void coarse_tc_alloc(Ctx& c);                       // buffers and the inverse's image (mixed, nrhs_max >= 16)
size_t coarse_tc_bytes(long long n, int nrhs_max);  // their size, for admission
// variant of the coarsest solve for the context's current batch width
// (0: CUDA-core GEMM; s >= 1: tensor cores, K split s ways)
inline int coarse_variant_for(const Ctx& c, int nrhs) {
  int lg = 0;
  while ((1 << lg) < nrhs) ++lg;
  const int v = lg < 7 ? c.coarse_variant[lg] : -1;
  if (v >= 0) return v;
  return coarse_tc_supported(c, nrhs) ? 4 : 0;
}

// setup.cu
void build_hierarchy(Ctx& c, const double* kappa_dev, const double* gamma_dev, double gamma0,
                     cudaStream_t s);
size_t hierarchy_bytes(const hz_grid& g, const hz_opts& o);

// cycle.cu (working-precision V-cycle pieces; `active` may be null)
void level_residual(Ctx& c, int l, const void* u, const void* f, void* r, const int* active, cudaStream_t s);
void level_smooth(Ctx& c, int l, void* u, const void* f, bool u_is_zero, const int* active, cudaStream_t s);
void level_restrict(Ctx& c, int l, const void* r, void* fc, const int* active, cudaStream_t s);
void level_prolong_add(Ctx& c, int l, const void* ec, void* u, const int* active, cudaStream_t s);
void coarse_solve(Ctx& c, const void* f, void* u, const int* active, cudaStream_t s);
void level_vanka_apply(Ctx& c, int l, const void* r, void* u, cudaStream_t s);   // u += w M r
void vcycle(Ctx& c, const void* f, void* u, const int* active, cudaStream_t s);   // level 0: f -> u
void fine_apply_f64(Ctx& c, const void* v, bool v_single, double2* w, bool shifted, cudaStream_t s);

// krylov.cu
size_t krylov_bytes(const hz_grid& g, const hz_opts& o);
void krylov_alloc(Ctx& c);
void fgmres_solve(Ctx& c, const double2* q_dev, double2* p_dev, hz_info* info, cudaStream_t s);
// asynchronous single-RHS solve (krylov.cu): step returns 1 once finished
void solve_begin(Ctx& c, const double2* q_dev, cudaStream_t s);
int solve_step(Ctx& c, bool block);
void solve_end(Ctx& c, double2* p_dev, hz_info* info, cudaStream_t s);
void fgmres_solve_batch(Ctx& c, const double2* q_dev, double2* p_dev, int nrhs, hz_info* info, cudaStream_t s);
void precond_apply_c128(Ctx& c, const double2* r, double2* z, int nrhs, cudaStream_t s);
// Eq. cf convergence factor of the cycle as a stationary solver (tune.cu)
void cycle_factor(Ctx& c, const double2* f, double2* u, int warmup, double target, int max_iter, double* factor,
                  int* iters, cudaStream_t s);
void profile_select(Ctx& c, int cls);

}  // namespace hz
