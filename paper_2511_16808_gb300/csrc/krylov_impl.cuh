// FGMRES state and device helpers shared by the single- and multi-RHS drivers
// (krylov.cu, krylov_batch.cu).
#pragma once
#include <cmath>
#include <cstddef>
#include <type_traits>

#include "common.cuh"

namespace hz {

constexpr int kMaxM = 128;      // longest restart cycle (one RHS; kMaxNV with several)
constexpr int kMaxNV = 16;      // vectors per Gram-Schmidt launch: longer passes run in chunks
constexpr int kRedBlock = 256;
constexpr int BX = 32, BY = 8;
constexpr int kRows = 4;        // y rows per thread in the 2D passes
constexpr int kPerThread = 4;   // nodes per thread in the 1D passes

struct KrylovStatus {       // first bytes of KrylovState, copied to the host each cycle
  int iters;
  int done;
  int converged;
  int breakdown;
  double relres_est;
  double relres_true;
};

struct KrylovState {
  KrylovStatus st;
  int active;               // iteration kernels run while 1
  int kcyc;                 // iterations done in the current cycle
  int m, max_iter;
  double tol, bnorm;
  double2 H[kMaxM + 1][kMaxM];
  double cs[kMaxM];
  double2 sn[kMaxM];
  double2 g[kMaxM + 1];
  double scale[kMaxM + 1];  // v_i = scale[i] * V[i]
  double2 y[kMaxM];
  double2 c[kMaxM];         // scale[i] * y[i]: the update coefficients of z'_i
  double2 h1[kMaxM + 2];    // raw dots conj(V_i) . w of the Gram-Schmidt passes
  double2 nrm2;             // .x = ||w||^2 after orthogonalisation
  unsigned counter;         // blocks finished in the current reduction (last block resets it)
};


inline unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

// k with v == 2^k exactly and 0 <= k <= 120, else -1.  When 1/h^2 is such a
// power of two the FP32 neighbour sums of the operator take the factor in
// their exact widening (an add to the exponent field), which leaves the
// interior rows' two FP64 multiplies out with bit-identical results: scaling
// by 2^k commutes with every rounding on the way (no FP64 overflow or
// underflow is reachable from FP32 inputs and k <= 120).
inline int pow2_exponent(double v) {
  int e = 0;
  const double m = std::frexp(v, &e);
  return (m == 0.5 && e - 1 >= 0 && e - 1 <= 120) ? e - 1 : -1;
}

struct Geo {
  int nx, ny, nz, sxy, N, dim;
  int compact;              // the fine operator is the compact fourth-order stencil (diag = sigma)
  int p2;                   // 1/h^2 == 2^p2 (second-order stencil only), else -1
};
inline Geo geo(const GridDev& g, bool compact = false, double invh2 = 0.0) {
  return Geo{g.nx, g.ny, g.nz, g.nx * g.ny, (int)g.N, g.dim, compact ? 1 : 0,
             (!compact && invh2 > 0.0) ? pow2_exponent(invh2) : -1};
}
// 2D grid of 32 x 8 blocks over (x, y), kRows rows per thread; blockIdx.z strides over z
inline dim3 grid_xy(const Geo& g) {
  return dim3((g.nx + BX - 1) / BX, (g.ny + BY * kRows - 1) / (BY * kRows), g.nz < 8 ? g.nz : 8);
}
inline unsigned grid_1d(long long N) { return nblk(N, kRedBlock * kPerThread); }

// Tiles of the persistent stencil passes: 32 x 8 nodes of one z plane (one
// node per thread), small enough that striding blocks end within one tile of
// each other.
inline long long tiles_xy(const Geo& g) {
  return (long long)((g.nx + BX - 1) / BX) * ((g.ny + BY - 1) / BY) * g.nz;
}
// Resident blocks of `threads` threads of `kernel` on the whole device (SMs x
// blocks per SM, cached per kernel): persistent passes launch at most this
// many blocks and stride over their tiles, so no partial last wave idles SMs.
int resident_slots(const void* kernel, int threads);
// At most this many blocks are launched by a persistent pass (8 blocks of 256
// threads per SM), which bounds the reduction partials.
int max_slots();
inline int grid_blocks(const Geo& g) {
  const dim3 d = grid_xy(g);
  return (int)(d.x * d.y * d.z);
}

// w - c v with two DFMA per component
__device__ __forceinline__ double2 axmy(double2 w, double2 c, double2 v) {
  return make_double2(fma(c.y, v.y, fma(-c.x, v.x, w.x)), fma(-c.y, v.x, fma(-c.x, v.y, w.y)));
}
// acc + conj(v) w with two DFMA per component
__device__ __forceinline__ double2 dot_acc(double2 acc, double2 v, double2 w) {
  return make_double2(fma(v.y, w.y, fma(v.x, w.x, acc.x)), fma(-v.y, w.x, fma(v.x, w.y, acc.y)));
}
// acc + |w|^2
__device__ __forceinline__ double nrm_acc(double acc, double2 w) { return fma(w.y, w.y, fma(w.x, w.x, acc)); }

__device__ __forceinline__ double2 ld64(const double2* __restrict__ a, int i) { return a[i]; }
__device__ __forceinline__ double2 ld64(const float2* __restrict__ a, int i) {
  const float2 v = a[i];
  return make_double2(f2d_exact(v.x), f2d_exact(v.y));
}

// Sum of the 2d neighbour values of an FP32 vector for the FP64 operator:
// error-free FP32 two-sums (Knuth: s + e == a + b exactly, IEEE round to
// nearest, no contraction) leave the sum as hi + lo with lo the FP32 sum of
// the rounding errors; one FP64 add of the exactly widened parts then gives
// the neighbour sum with error <= (2d-1)^2 2^-48 times the largest partial sum,
// far below the FP32 storage error of the values themselves.  This replaces
// 2(2d-1) FP64 adds per node by FP32 adds (64x the FP64 rate on GB300).
__host__ __device__ __forceinline__ float fadd_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  volatile float r = a + b;
  return r;
#endif
}
__host__ __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = fadd_rn(a, b);
  const float bb = fadd_rn(s, -a);
  e = fadd_rn(fadd_rn(a, -fadd_rn(s, -bb)), fadd_rn(b, -bb));
}
template <int NN>
__host__ __device__ __forceinline__ double fsum_wide(const float (&v)[NN]) {
  float s = v[0], e = 0.0f;
#pragma unroll
  for (int i = 1; i < NN; ++i) {
    float t;
    two_sum(s, v[i], s, t);
    e = fadd_rn(e, t);
  }
  return f2d_exact(s) + f2d_exact(e);
}
template <int NN>
__device__ __forceinline__ double2 nbr_sum(const float2 (&n)[NN]) {
  float xs[NN], ys[NN];
#pragma unroll
  for (int i = 0; i < NN; ++i) {
    xs[i] = n[i].x;
    ys[i] = n[i].y;
  }
  return make_double2(fsum_wide<NN>(xs), fsum_wide<NN>(ys));
}
// exact widening of f * 2^k (0 <= k <= 120): zero, infinities and NaN pass
// unchanged, every other value moves up k binades
__host__ __device__ __forceinline__ double f2d_exact_pow2(float f, int k) {
  unsigned hi, lo;
  d_hilo(f2d_exact(f), hi, lo);
  const unsigned E = (hi >> 20) & 0x7ffu;
  if (E != 0u && E != 0x7ffu) hi += (unsigned)k << 20;
  return hilo_d(hi, lo);
}
// fsum_wide times 2^k, exactly (the scaling commutes with the final FP64 add)
template <int NN>
__host__ __device__ __forceinline__ double fsum_wide_pow2(const float (&v)[NN], int k) {
  float s = v[0], e = 0.0f;
#pragma unroll
  for (int i = 1; i < NN; ++i) {
    float t;
    two_sum(s, v[i], s, t);
    e = fadd_rn(e, t);
  }
  return f2d_exact_pow2(s, k) + f2d_exact_pow2(e, k);
}
template <int NN>
__device__ __forceinline__ double2 nbr_sum_pow2(const float2 (&n)[NN], int k) {
  float xs[NN], ys[NN];
#pragma unroll
  for (int i = 0; i < NN; ++i) {
    xs[i] = n[i].x;
    ys[i] = n[i].y;
  }
  return make_double2(fsum_wide_pow2<NN>(xs, k), fsum_wide_pow2<NN>(ys, k));
}
// d v - s for a neighbour sum s already scaled by 1/h^2
__device__ __forceinline__ double2 diag_minus(double2 d, double2 vp, double2 s) {
  return make_double2(fma(d.x, vp.x, fma(-d.y, vp.y, -s.x)), fma(d.x, vp.y, fma(d.y, vp.x, -s.y)));
}

// FP64 fine-level (A v)_p, 5-/7-point with half-cell weights
template <typename U>
__device__ __forceinline__ double2 apply_A(const Geo& g, double invh2, const double2* __restrict__ diag,
                                           const U* __restrict__ v, int p, int x, int y, int z) {
  if (g.compact) {
    // the compact stencil (diag holds sigma): FP64 throughout
    auto ld = [v](long long q) { return ld64(v, (int)q); };
    return compact_Av(g.nx, g.ny, g.nz, g.dim, invh2, diag, make_double2(0, 0), ld, p, x, y, z);
  }
  const double2 d = diag[p], vp = ld64(v, p);
  const bool inx = x > 0 && x < g.nx - 1, iny = y > 0 && y < g.ny - 1;
  const bool inz = g.dim == 2 || (z > 0 && z < g.nz - 1);
  if (inx && iny && inz) {
    double2 s;
    if constexpr (std::is_same<U, float2>::value) {
      if (g.dim == 3) {
        const float2 n[6] = {v[HZ_AT(p - 1, g.N)], v[HZ_AT(p + 1, g.N)], v[HZ_AT(p - g.nx, g.N)],
                             v[HZ_AT(p + g.nx, g.N)], v[HZ_AT(p - g.sxy, g.N)], v[HZ_AT(p + g.sxy, g.N)]};
        if (g.p2 >= 0) return diag_minus(d, vp, nbr_sum_pow2<6>(n, g.p2));
        s = nbr_sum<6>(n);
      } else {
        const float2 n[4] = {v[HZ_AT(p - 1, g.N)], v[HZ_AT(p + 1, g.N)], v[HZ_AT(p - g.nx, g.N)],
                             v[HZ_AT(p + g.nx, g.N)]};
        if (g.p2 >= 0) return diag_minus(d, vp, nbr_sum_pow2<4>(n, g.p2));
        s = nbr_sum<4>(n);
      }
    } else {
      s = ld64(v, (int)HZ_AT(p - 1, g.N)) + ld64(v, (int)HZ_AT(p + 1, g.N)) + ld64(v, (int)HZ_AT(p - g.nx, g.N)) +
          ld64(v, (int)HZ_AT(p + g.nx, g.N));
      if (g.dim == 3) s = s + ld64(v, (int)HZ_AT(p - g.sxy, g.N)) + ld64(v, (int)HZ_AT(p + g.sxy, g.N));
    }
    // d v - invh2 s, with FMAs
    return make_double2(fma(d.x, vp.x, fma(-d.y, vp.y, -invh2 * s.x)), fma(d.x, vp.y, fma(d.y, vp.x, -invh2 * s.y)));
  }
  double2 acc = cmul(d, vp);
  const double wx = inx ? 1.0 : 0.5, wy = iny ? 1.0 : 0.5;
  const double wz = (g.dim == 3 && !inz) ? 0.5 : 1.0;
  double2 sx = make_double2(0, 0), sy = make_double2(0, 0);
  if (x > 0) sx = sx + ld64(v, p - 1);
  if (x < g.nx - 1) sx = sx + ld64(v, p + 1);
  if (y > 0) sy = sy + ld64(v, p - g.nx);
  if (y < g.ny - 1) sy = sy + ld64(v, p + g.nx);
  const double cx = wy * wz * invh2, cy = wx * wz * invh2;
  acc.x -= cx * sx.x + cy * sy.x;
  acc.y -= cx * sx.y + cy * sy.y;
  if (g.dim == 3) {
    double2 sz = make_double2(0, 0);
    if (z > 0) sz = sz + ld64(v, p - g.sxy);
    if (z < g.nz - 1) sz = sz + ld64(v, p + g.sxy);
    const double cz = wx * wy * invh2;
    acc.x -= cz * sz.x;
    acc.y -= cz * sz.y;
  }
  return acc;
}

__device__ inline void givens(double2 a, double2 b, double& c, double2& s) {
  const double ab = sqrt(cabs2(b));
  if (ab == 0.0) {
    c = 1.0;
    s = make_double2(0, 0);
    return;
  }
  const double aa = sqrt(cabs2(a));
  if (aa == 0.0) {
    c = 0.0;
    s = make_double2(b.x / ab, -b.y / ab);     // conj(b)/|b|
    return;
  }
  const double t = hypot(aa, ab);
  c = aa / t;
  const double2 ph = make_double2(a.x / aa, a.y / aa);
  s = (1.0 / t) * cmul(ph, make_double2(b.x, -b.y));
}

// Column j of the Hessenberg matrix, Givens rotations, residual estimate
// (one thread, in the last block of the final Gram-Schmidt pass).
// sj: scale of the preconditioned vector when z_j = sj * (V-cycle of the
// unnormalised V_j) was used (the Gram-Schmidt dots and norm are then those
// of A z_j / sj), 1 when z_j came from the normalised v_j.
__device__ inline void arnoldi_update(KrylovState* st, int j, int* n_active = nullptr, double sj = 1.0) {
  for (int i = 0; i <= j; ++i) st->H[i][j] = (sj * st->scale[i]) * st->h1[i];
  const double hn = sqrt(st->nrm2.x);
  st->H[j + 1][j] = make_double2(sj * hn, 0.0);
  for (int i = 0; i < j; ++i) {
    const double2 a = st->H[i][j], b = st->H[i + 1][j];
    const double c = st->cs[i];
    const double2 s = st->sn[i];
    st->H[i][j] = c * a + cmul(s, b);
    st->H[i + 1][j] = cmul(make_double2(-s.x, s.y), a) + c * b;      // -conj(s) a + c b
  }
  double c;
  double2 s;
  givens(st->H[j][j], st->H[j + 1][j], c, s);
  st->cs[j] = c;
  st->sn[j] = s;
  st->H[j][j] = c * st->H[j][j] + cmul(s, st->H[j + 1][j]);
  st->H[j + 1][j] = make_double2(0, 0);
  const double2 gj = st->g[j];
  st->g[j + 1] = cmul(make_double2(-s.x, s.y), gj);
  st->g[j] = c * gj;
  st->st.iters += 1;
  st->kcyc = j + 1;
  st->st.relres_est = sqrt(cabs2(st->g[j + 1])) / st->bnorm;
  if (!(hn > 0.0)) {
    st->st.breakdown = 1;
    st->scale[j + 1] = 0.0;
  } else {
    st->scale[j + 1] = 1.0 / hn;
  }
  if (st->st.relres_est < st->tol || st->st.iters >= st->max_iter || st->st.breakdown || st->kcyc >= st->m) {
    st->active = 0;
    if (n_active) atomicSub(n_active, 1);
  }
}

// arnoldi_update for one right-hand side, called by every thread of the last
// block of a reduction: the block first stages the column's inputs (scales
// and raw inner products, the previous rotations) in shared memory, then one
// thread runs the same sequential chain on the staged values, so its steps
// wait on shared memory instead of a global-memory round trip each.  Same
// operations in the same order as arnoldi_update: bit-identical state.
__device__ inline void arnoldi_update_staged(KrylovState* st, int j, double sj) {
  __shared__ double2 hc[kMaxM + 1];
  __shared__ double2 sn[kMaxM];
  __shared__ double cs[kMaxM];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  for (int i = tid; i <= j; i += nt) hc[i] = (sj * st->scale[i]) * st->h1[i];
  for (int i = tid; i < j; i += nt) {
    cs[i] = st->cs[i];
    sn[i] = st->sn[i];
  }
  __syncthreads();
  if (tid != 0) return;
  const double hn = sqrt(st->nrm2.x);
  double2 below = make_double2(sj * hn, 0.0);               // H[j+1][j]
  for (int i = 0; i < j; ++i) {
    const double2 a = hc[i], b = hc[i + 1];
    const double c = cs[i];
    const double2 sv = sn[i];
    hc[i] = c * a + cmul(sv, b);
    hc[i + 1] = cmul(make_double2(-sv.x, sv.y), a) + c * b;  // -conj(s) a + c b
  }
  double c;
  double2 sv;
  givens(hc[j], below, c, sv);
  st->cs[j] = c;
  st->sn[j] = sv;
  hc[j] = c * hc[j] + cmul(sv, below);
  for (int i = 0; i <= j; ++i) st->H[i][j] = hc[i];
  st->H[j + 1][j] = make_double2(0, 0);
  const double2 gj = st->g[j];
  st->g[j + 1] = cmul(make_double2(-sv.x, sv.y), gj);
  st->g[j] = c * gj;
  st->st.iters += 1;
  st->kcyc = j + 1;
  st->st.relres_est = sqrt(cabs2(st->g[j + 1])) / st->bnorm;
  if (!(hn > 0.0)) {
    st->st.breakdown = 1;
    st->scale[j + 1] = 0.0;
  } else {
    st->scale[j + 1] = 1.0 / hn;
  }
  if (st->st.relres_est < st->tol || st->st.iters >= st->max_iter || st->st.breakdown || st->kcyc >= st->m)
    st->active = 0;
}

__device__ inline void restart_update(KrylovState* st, int* n_active = nullptr) {
  const double beta = sqrt(st->nrm2.x);
  st->st.relres_true = beta / st->bnorm;
  st->active = 0;
  if (st->st.relres_true < st->tol) {
    st->st.converged = 1;
    st->st.done = 1;
    return;
  }
  if (st->st.iters >= st->max_iter) {
    st->st.done = 1;
    return;
  }
  st->st.breakdown = 0;
  st->scale[0] = 1.0 / beta;
  st->g[0] = make_double2(beta, 0.0);
  for (int i = 1; i <= kMaxM; ++i) st->g[i] = make_double2(0, 0);
  st->kcyc = 0;
  st->active = 1;
  if (n_active) atomicAdd(n_active, 1);
}

// NV = 1..kMaxNV as a compile-time constant
template <typename F>
void with_nv(int nv, F&& f) {
  switch (nv) {
#define HZ_NV(K) \
  case K: f(std::integral_constant<int, K>{}); return;
    HZ_NV(1) HZ_NV(2) HZ_NV(3) HZ_NV(4) HZ_NV(5) HZ_NV(6) HZ_NV(7) HZ_NV(8)
    HZ_NV(9) HZ_NV(10) HZ_NV(11) HZ_NV(12) HZ_NV(13) HZ_NV(14) HZ_NV(15) HZ_NV(16)
#undef HZ_NV
    default: throw Error(HZ_ERR_INVALID_ARG, "more than 16 vectors in one Gram-Schmidt launch");
  }
}

// Measurement hooks (krylov.cu): CUDA events around the launches of the
// selected class (1 = Gram-Schmidt update passes, 2 = first pass with the FP64
// operator, 3 = whole V-cycle), recorded inside the captured restart cycle.
int prof_begin(Ctx& c, int cls, int j, double bytes, double flops, cudaStream_t s);
void prof_end(Ctx& c, int k, cudaStream_t s);
void prof_collect(Ctx& c, int ran, const int* ran_r, int R);
double vcycle_bytes(const Ctx& c);

}  // namespace hz
