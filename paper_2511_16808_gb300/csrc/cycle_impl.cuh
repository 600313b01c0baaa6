// V-cycle kernels in the working precision T (float for the mixed path,
// double for the plain FP64 path) and the recursive driver (Algorithm 1).
//
//   residual    r = f - A_s u          fine: diagonal + index weights (5/7-point);
//                                      coarse: stored Galerkin planes (box radius rho)
//   sweep       u += w M r             M = assembled Vanka sum (Eq. smoother) in its
//                                      symmetric half form; the first sweep from
//                                      u = 0 is u = w M f
//   restrict    f_c = R r              Eqs. biliniearIntergrid / bicubicIntergrid (gather)
//   prolong     u += P e_c             P = 2^d R^T of the same kind (gather)
//   coarse      u = A_L^{-1} f         dense inverse from setup, one warp per row
//
// Fused forms (one HBM pass instead of two or three):
//   sweep0+residual   when M is diagonal (Jacobi; RB on a 2d+1-point stencil):
//                     u = w m0 f and r = f - A(w m0 f) in one kernel
//   prolong+residual  2D: u' = t + P e_c on a shared-memory tile with halo, then
//                     r = f - A u' from the tile
//   prolong+sweep     2D with diagonal M: u = u' + w m0 (f - A u') from the tile
// Batched right-hand sides: with R (a power of two <= 64) right-hand sides the
// RHS index is innermost (field index node*R + r); every kernel then sees a
// grid whose x extent is nx*R (x neighbours at +-R, y at +-nx*R), reads each
// coefficient once per node (broadcast across the warp's RHS), and the fused
// shared-memory tile kernels are used only for R = 1.
// Thread mapping: 32 x 8 threads per block over (x*R + r, y), blockIdx.z = z,
// one thread per output value, 32-bit indices; blocks whose stencil reach stays
// inside the grid take an unchecked path (block-uniform branch).  Kernels take
// an optional device flag `active`: when it reads 0 they return at once (a
// captured FGMRES cycle uses it to skip the iterations after convergence).
#pragma once
#include <type_traits>

#include "common.cuh"

namespace hz {
namespace cyc {

constexpr int BX = 32, BY = 8;
constexpr int kMaxM = 125;

struct Geo {
  int nx, ny, nz, sxy, N;     // nodes
  int R, lr;                  // right-hand sides (R = 1 << lr)
  int nxR, sxyR;              // field strides in y and z
  int lv, nxV;                // each thread handles VR = 1 << lv consecutive RHS; threads per row
};
inline Geo geo(const GridDev& g, int R = 1, int VR = 1) {
  int lr = 0, lv = 0;
  while ((1 << lr) < R) ++lr;
  while ((1 << lv) < VR) ++lv;
  require((1 << lr) == R && R <= 64, "nrhs must be a power of two <= 64");
  require((1 << lv) == VR && VR <= R, "bad RHS pack");
  return Geo{g.nx, g.ny, g.nz, g.nx * g.ny, (int)g.N, R, lr, g.nx * R, g.nx * g.ny * R, lv, (g.nx * R) >> lv};
}
inline dim3 grid_of(const Geo& g) { return dim3((g.nxV + BX - 1) / BX, (g.ny + BY - 1) / BY, g.nz); }

// RHS pack per thread: with many right-hand sides each thread handles VR
// consecutive ones (32 bytes: 4 complex floats or 2 complex doubles), so a
// stencil coefficient is loaded once for VR values and the fields move in
// 16-byte vector accesses.  VR = 1 is the plain complex value.
template <typename T, int VR>
struct PkS {
  c_t<T> v[VR];
};
template <typename T, int VR>
using pk_t = std::conditional_t<VR == 1, c_t<T>, PkS<T, VR>>;
template <typename T> constexpr int kVRMax = 32 / (int)sizeof(c_t<T>);
inline int vr_for(int R, int vmax) { return R >= vmax ? vmax : 1; }

// the complex-value versions from namespace hz stay visible beside the pack ones
using ::hz::cfma;
using ::hz::cmul;
using ::hz::operator+;
using ::hz::operator-;
using ::hz::operator*;

template <typename T, int VR>
__device__ __forceinline__ PkS<T, VR> operator+(PkS<T, VR> a, const PkS<T, VR>& b) {
#pragma unroll
  for (int i = 0; i < VR; ++i) a.v[i] = a.v[i] + b.v[i];
  return a;
}
template <typename T, int VR>
__device__ __forceinline__ PkS<T, VR> operator-(PkS<T, VR> a, const PkS<T, VR>& b) {
#pragma unroll
  for (int i = 0; i < VR; ++i) a.v[i] = a.v[i] - b.v[i];
  return a;
}
template <typename T, int VR>
__device__ __forceinline__ PkS<T, VR> operator*(T s, PkS<T, VR> a) {
#pragma unroll
  for (int i = 0; i < VR; ++i) a.v[i] = s * a.v[i];
  return a;
}
template <typename T, int VR>
__device__ __forceinline__ PkS<T, VR> cmul(c_t<T> c, PkS<T, VR> a) {
#pragma unroll
  for (int i = 0; i < VR; ++i) a.v[i] = cmul(c, a.v[i]);
  return a;
}
template <typename T, int VR>
__device__ __forceinline__ PkS<T, VR> cfma(c_t<T> c, const PkS<T, VR>& a, PkS<T, VR> acc) {
#pragma unroll
  for (int i = 0; i < VR; ++i) acc.v[i] = cfma(c, a.v[i], acc.v[i]);
  return acc;
}
template <typename V>
__device__ __forceinline__ V pk_zero() {
  V z;
  if constexpr (std::is_same<V, float2>::value || std::is_same<V, double2>::value) {
    z.x = 0;
    z.y = 0;
  } else {
#pragma unroll
    for (int i = 0; i < (int)(sizeof(V) / sizeof(z.v[0])); ++i) {
      z.v[i].x = 0;
      z.v[i].y = 0;
    }
  }
  return z;
}
// pack load / store at field index q (q a multiple of VR: 16-byte aligned chunks)
template <typename T, int VR>
__device__ __forceinline__ pk_t<T, VR> ldp(const c_t<T>* a, int q) {
  if constexpr (VR == 1) {
    return a[q];
  } else {
    PkS<T, VR> r;
    const uint4* src = reinterpret_cast<const uint4*>(a + q);
    uint4* dst = reinterpret_cast<uint4*>(&r);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(r) / 16); ++i) dst[i] = src[i];
    return r;
  }
}
template <typename T, int VR>
__device__ __forceinline__ void stp(c_t<T>* a, int q, const pk_t<T, VR>& v) {
  if constexpr (VR == 1) {
    a[q] = v;
  } else {
    uint4* dst = reinterpret_cast<uint4*>(a + q);
    const uint4* src = reinterpret_cast<const uint4*>(&v);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(v) / 16); ++i) dst[i] = src[i];
  }
}
inline unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

// Offsets of a stored Vanka sum that is applied as it is (no mirroring), with
// their flat field index offsets (kept small: the list travels in the kernel
// parameters of every sweep launch).
struct MList {
  int n, rho;
  int flat[kMaxM];
  signed char d[kMaxM][3];
};

inline MList mlist(const Level& L, int R = 1) {
  require(L.Mh.off.n <= kMaxM, "Vanka stencil too large");
  MList m;
  m.n = L.Mh.off.n;
  m.rho = L.Mh.off.rho;
  for (int s = 0; s < m.n; ++s) {
    for (int a = 0; a < 3; ++a) m.d[s][a] = L.Mh.off.d[s][a];
    m.flat[s] = (L.Mh.off.d[s][0] + L.Mh.off.d[s][1] * L.g.nx + L.Mh.off.d[s][2] * L.g.nx * L.g.ny) * R;
  }
  return m;
}

// The stored half of a symmetric Vanka sum (setup: L.Mh, L.mh_mirror):
// offsets with node and field index offsets, and whether -s is applied too.
struct SList {
  int n, rho;
  int flat[kMaxM];              // field index offset (node offset x R)
  int nflat[kMaxM];             // node index offset
  signed char d[kMaxM][3];
  unsigned char mirror[kMaxM];
};

inline SList slist(const Level& L, int R = 1) {
  require(L.Mh.off.n <= kMaxM, "Vanka stencil too large");
  SList m;
  m.n = L.Mh.off.n;
  m.rho = L.Mh.off.rho;
  for (int s = 0; s < m.n; ++s) {
    for (int a = 0; a < 3; ++a) m.d[s][a] = L.Mh.off.d[s][a];
    m.nflat[s] = L.Mh.off.d[s][0] + L.Mh.off.d[s][1] * L.g.nx + L.Mh.off.d[s][2] * L.g.nx * L.g.ny;
    m.flat[s] = m.nflat[s] * R;
    m.mirror[s] = L.mh_mirror[s];
  }
  return m;
}

// Thread -> (node x, y, z), node index p and field index q; false past the edge.
__device__ __forceinline__ bool node_xyz(const Geo& g, int& x, int& y, int& z, int& p, int& q) {
  const int X = blockIdx.x * BX + threadIdx.x;
  y = blockIdx.y * BY + threadIdx.y;
  z = blockIdx.z;
  if (X >= g.nxV || y >= g.ny) return false;
  x = X >> (g.lr - g.lv);
  const int row = z * g.ny + y;
  p = row * g.nx + x;
  q = row * g.nxR + (X << g.lv);
  return true;
}

// true when every node of this block and its neighbours within r lie in the grid
template <int DIM>
__device__ __forceinline__ bool interior_block(const Geo& g, int r) {
  const int x0 = (blockIdx.x * BX) >> (g.lr - g.lv), x1 = (blockIdx.x * BX + BX - 1) >> (g.lr - g.lv);
  const int y0 = blockIdx.y * BY;
  bool ok = x0 >= r && x1 + r < g.nx && y0 >= r && y0 + BY - 1 + r < g.ny;
  if (DIM == 3) ok = ok && (int)blockIdx.z >= r && (int)blockIdx.z + r < g.nz;
  return ok;
}

template <typename V>
__device__ __forceinline__ V scale(V a, decltype(a.x) s) {
  a.x *= s;
  a.y *= s;
  return a;
}

// The stencil helpers work on the value type of `ld` (a complex value, or a
// pack of VR right-hand sides sharing the node's coefficients).

// A u at node p for the fine 5-/7-point operator (diag d at p).
template <typename T, int DIM, bool CHECK, typename LD>
__device__ __forceinline__ auto fine_Au(const Geo& g, T invh2, c_t<T> d, const LD& ld, int q, int x, int y, int z) {
  using V = decltype(ld(0));
  V acc = cmul(d, ld(q));
  if (!CHECK) {
    V s = ld(q - g.R) + ld(q + g.R) + ld(q - g.nxR) + ld(q + g.nxR);
    if (DIM == 3) s = s + ld(q - g.sxyR) + ld(q + g.sxyR);
    return acc - invh2 * s;
  }
  const T wx = (x == 0 || x == g.nx - 1) ? T(0.5) : T(1);
  const T wy = (y == 0 || y == g.ny - 1) ? T(0.5) : T(1);
  const T wz = (DIM == 3 && (z == 0 || z == g.nz - 1)) ? T(0.5) : T(1);
  V sx = pk_zero<V>(), sy = pk_zero<V>();
  if (x > 0) sx = sx + ld(q - g.R);
  if (x < g.nx - 1) sx = sx + ld(q + g.R);
  if (y > 0) sy = sy + ld(q - g.nxR);
  if (y < g.ny - 1) sy = sy + ld(q + g.nxR);
  const T cx = wy * wz * invh2, cy = wx * wz * invh2;
  acc = acc - (cx * sx + cy * sy);
  if (DIM == 3) {
    V sz = pk_zero<V>();
    if (z > 0) sz = sz + ld(q - g.sxyR);
    if (z < g.nz - 1) sz = sz + ld(q + g.sxyR);
    const T cz = wx * wy * invh2;
    acc = acc - cz * sz;
  }
  return acc;
}

// A u at node p for a stored box stencil of radius RHO (planes [s][N]).
template <typename T, int DIM, int RHO, bool CHECK, typename LD>
__device__ __forceinline__ auto box_Au(const Geo& g, const c_t<T>* __restrict__ P, const LD& ld, int p, int q, int x,
                                       int y, int z) {
  using V = decltype(ld(0));
  V acc = pk_zero<V>();
  constexpr int RZ = DIM == 3 ? RHO : 0;
  constexpr int W = 2 * RHO + 1;
#pragma unroll
  for (int dz = -RZ; dz <= RZ; ++dz)
#pragma unroll
    for (int dy = -RHO; dy <= RHO; ++dy)
#pragma unroll
      for (int dx = -RHO; dx <= RHO; ++dx) {
        const int s = ((dz + RZ) * W + (dy + RHO)) * W + (dx + RHO);
        int qq = q + dx * g.R + dy * g.nxR + dz * g.sxyR;
        if (CHECK) {
          // branch-free: a neighbour outside the grid has a zero plane entry,
          // so it is read at the node itself (a valid address) and adds 0
          const bool ok = x + dx >= 0 && x + dx < g.nx && y + dy >= 0 && y + dy < g.ny &&
                          (DIM == 2 || (z + dz >= 0 && z + dz < g.nz));
          qq = ok ? qq : q;
        }
        acc = cfma(P[HZ_AT(s * g.N + p, (long long)W * W * (DIM == 3 ? W : 1) * g.N)], ld(qq), acc);
      }
  return acc;
}

// A u at node p for a symmetric stored box stencil of radius RHO kept as its
// half: planes of the offsets s >= 0 (the upper half of the box's (z, y, x)
// order, centre first), A(p, p+s) at node p; A(p, p-s) = A(p-s, p) is read at
// node p-s.  Half the coefficient bytes of box_Au; the mirrored loads are the
// neighbouring nodes' own entries.
template <typename T, int DIM, int RHO, bool CHECK, typename LD>
__device__ __forceinline__ auto box_Au_half(const Geo& g, const c_t<T>* __restrict__ P, const LD& ld, int p, int q,
                                            int x, int y, int z) {
  using V = decltype(ld(0));
  V acc = pk_zero<V>();
  constexpr int RZ = DIM == 3 ? RHO : 0;
  constexpr int W = 2 * RHO + 1;
  constexpr int C = ((2 * RZ + 1) * W * W - 1) / 2;             // box index of the centre
#pragma unroll
  for (int dz = -RZ; dz <= RZ; ++dz)
#pragma unroll
    for (int dy = -RHO; dy <= RHO; ++dy)
#pragma unroll
      for (int dx = -RHO; dx <= RHO; ++dx) {
        const int s = ((dz + RZ) * W + (dy + RHO)) * W + (dx + RHO);
        if (s < C) continue;
        const int k = s - C;
        const int fo = dx * g.R + dy * g.nxR + dz * g.sxyR;
        const int no = dx + dy * g.nx + dz * g.sxy;
        int qp = q + fo;
        if (CHECK) {
          // branch-free: an out-of-grid + neighbour has a zero stored entry (read at q)
          const bool ok = x + dx >= 0 && x + dx < g.nx && y + dy >= 0 && y + dy < g.ny &&
                          (DIM == 2 || (z + dz >= 0 && z + dz < g.nz));
          qp = ok ? qp : q;
        }
        [[maybe_unused]] constexpr long long NH = (long long)(2 * RZ + 1) * W * W - C;   // half planes stored
        acc = cfma(P[HZ_AT(k * g.N + p, NH * g.N)], ld(qp), acc);
        if (s == C) continue;
        if (CHECK) {
          // the mirrored entry lives at node p - s: outside the grid the address
          // is replaced by p and the coefficient by 0
          const bool ok = x - dx >= 0 && x - dx < g.nx && y - dy >= 0 && y - dy < g.ny &&
                          (DIM == 2 || (z - dz >= 0 && z - dz < g.nz));
          c_t<T> cm = P[HZ_AT(k * g.N + (ok ? p - no : p), NH * g.N)];
          cm = ok ? cm : cmk<c_t<T>>(0, 0);
          acc = cfma(cm, ld(ok ? q - fo : q), acc);
        } else {
          acc = cfma(P[HZ_AT(k * g.N + p - no, NH * g.N)], ld(q - fo), acc);
        }
      }
  return acc;
}

// AK = 0: fine analytic operator; AK = rho > 0: stored box stencil;
// AK = 10 + rho: symmetric box stencil stored as its half (box_Au_half).
template <typename T, int DIM, int AK, bool CHECK, typename LD>
__device__ __forceinline__ auto apply_A(const Geo& g, T invh2, const c_t<T>* __restrict__ A, const LD& ld, int p, int q,
                                        int x, int y, int z) {
  if constexpr (AK == 0)
    return fine_Au<T, DIM, CHECK>(g, invh2, A[HZ_AT(p, g.N)], ld, q, x, y, z);
  else if constexpr (AK > 10)
    return box_Au_half<T, DIM, AK - 10, CHECK>(g, A, ld, p, q, x, y, z);
  else
    return box_Au<T, DIM, AK, CHECK>(g, A, ld, p, q, x, y, z);
}

template <typename T, int DIM, bool CHECK, typename LD>
__device__ __forceinline__ auto list_Au(const Geo& g, const MList& m, const c_t<T>* __restrict__ P, const LD& ld, int p,
                                        int q, int x, int y, int z) {
  using V = decltype(ld(0));
  V acc = pk_zero<V>();
  for (int s = 0; s < m.n; ++s) {
    int qq = q + m.flat[s];
    if (CHECK) {
      // branch-free: the plane entry of a neighbour outside the grid is zero
      const int xx = x + m.d[s][0], yy = y + m.d[s][1], zz = z + m.d[s][2];
      const bool ok = xx >= 0 && xx < g.nx && yy >= 0 && yy < g.ny && (DIM == 2 || (zz >= 0 && zz < g.nz));
      qq = ok ? qq : q;
    }
    acc = cfma(P[HZ_AT(s * g.N + p, (long long)m.n * g.N)], ld(qq), acc);
  }
  return acc;
}

// (M v)_p from the stored form: symmetric half (M = D^{-1} M', M'(p, p+s)
// stored at node p for the half offsets, M'(p, p-s) = M'(p-s, p) read at node
// p-s, then the weight 1/count_p), or all planes of M itself (wc null).
template <typename T, int DIM, bool CHECK, bool SYM, typename LST, typename LD>
__device__ __forceinline__ auto sym_Au(const Geo& g, const LST& m, const c_t<T>* __restrict__ P,
                                       const T* __restrict__ wc, const LD& ld, int p, int q, int x, int y, int z) {
  using V = decltype(ld(0));
  V acc = pk_zero<V>();
  for (int s = 0; s < m.n; ++s) {
    if (CHECK) {
      // branch-free: out-of-grid terms read valid addresses and add 0 (the
      // + entry is stored as zero; the mirrored coefficient is selected to 0)
      const int dx = m.d[s][0], dy = m.d[s][1], dz = m.d[s][2];
      const bool okp = x + dx >= 0 && x + dx < g.nx && y + dy >= 0 && y + dy < g.ny &&
                       (DIM == 2 || (z + dz >= 0 && z + dz < g.nz));
      acc = cfma(P[HZ_AT(s * g.N + p, (long long)m.n * g.N)], ld(okp ? q + m.flat[s] : q), acc);
      if constexpr (SYM) {
        const bool okm = m.mirror[s] && x - dx >= 0 && x - dx < g.nx && y - dy >= 0 && y - dy < g.ny &&
                         (DIM == 2 || (z - dz >= 0 && z - dz < g.nz));
        const c_t<T> cm = P[HZ_AT(s * g.N + (okm ? p - m.nflat[s] : p), (long long)m.n * g.N)];
        acc = cfma(okm ? cm : cmk<c_t<T>>(0, 0), ld(okm ? q - m.flat[s] : q), acc);
      }
    } else {
      acc = cfma(P[HZ_AT(s * g.N + p, (long long)m.n * g.N)], ld(q + m.flat[s]), acc);
      if constexpr (SYM)
        if (m.mirror[s])
          acc = cfma(P[HZ_AT(s * g.N + p - m.nflat[s], (long long)m.n * g.N)], ld(q - m.flat[s]), acc);
    }
  }
  if constexpr (SYM) return wc[p] * acc;
  else return acc;                           // the planes hold M itself
}

// planes of the operator's stored form: the fine diagonal (AK = 0), a full
// box of radius rho (AK = rho) or its symmetric half (AK = 10 + rho)
template <int DIM, int AK>
constexpr int a_planes() {
  constexpr int W = 2 * (AK % 10) + 1, BOX = DIM == 3 ? W * W * W : W * W;
  return AK == 0 ? 1 : (AK > 10 ? (BOX + 1) / 2 : BOX);
}

// L2 prefetch of the stencil planes a block of the one-RHS node kernels reads
// (its 32 x 8 nodes of one z plane and their reach rho in x and y), issued
// before pdl_enter() like the tile passes do: the planes are setup data
template <typename T>
__device__ __forceinline__ void prefetch_block_planes(const Geo& g, const c_t<T>* P, int np, int rho) {
  if (g.R != 1) return;
  const int x0 = (int)blockIdx.x * BX - rho, y0 = (int)blockIdx.y * BY - rho;
  prefetch_l2_planes(P + (long long)blockIdx.z * g.sxy, np, g.N, g.nx, g.ny, x0, BX + 2 * rho, y0, BY + 2 * rho,
                     (int)(threadIdx.y * BX + threadIdx.x), BX * BY);
}

// ------------------------------------------------------------------ kernels

// r = f - A u
template <typename T, int DIM, int AK, int VR, int MB>
__global__ void __launch_bounds__(BX* BY, MB) k_resid(Geo g, T invh2, const c_t<T>* __restrict__ A,
                                                  const c_t<T>* __restrict__ u, const c_t<T>* __restrict__ f,
                                                  c_t<T>* __restrict__ r, const int* active) {
  prefetch_block_planes<T>(g, A, a_planes<DIM, AK>(), AK == 0 ? 0 : AK % 10);
  pdl_enter();
  if (active && !*active) return;
  constexpr int RA = AK == 0 ? 1 : AK % 10;
  const bool in = interior_block<DIM>(g, RA);
  int x, y, z, p, q;
  if (!node_xyz(g, x, y, z, p, q)) return;
  auto ld = [u HZ_EXT((long long)g.N * g.R)](int i) { return ldp<T, VR>(u, HZ_AT(i, hz_ext)); };
  const pk_t<T, VR> a = in ? apply_A<T, DIM, AK, false>(g, invh2, A, ld, p, q, x, y, z)
                           : apply_A<T, DIM, AK, true>(g, invh2, A, ld, p, q, x, y, z);
  stp<T, VR>(r, q, ldp<T, VR>(f, q) - a);
}

// u = w M f  (first sweep from u = 0)
template <typename T, int DIM, int VR, int MB>
__global__ void __launch_bounds__(BX* BY, MB) k_sweep0(Geo g, MList m, const c_t<T>* __restrict__ M, T w,
                                                   const c_t<T>* __restrict__ f, c_t<T>* __restrict__ u,
                                                   const int* active) {
  prefetch_block_planes<T>(g, M, m.n, 0);
  pdl_enter();
  if (active && !*active) return;
  const bool in = interior_block<DIM>(g, m.rho);
  int x, y, z, p, q;
  if (!node_xyz(g, x, y, z, p, q)) return;
  auto ld = [f HZ_EXT((long long)g.N * g.R)](int i) { return ldp<T, VR>(f, HZ_AT(i, hz_ext)); };
  const pk_t<T, VR> v = in ? list_Au<T, DIM, false>(g, m, M, ld, p, q, x, y, z)
                           : list_Au<T, DIM, true>(g, m, M, ld, p, q, x, y, z);
  stp<T, VR>(u, q, w * v);
}

// symmetric half form: u = w D^{-1} M' f
template <typename T, int DIM, int VR, int MB>
__global__ void __launch_bounds__(BX* BY, MB) k_sweep0_sym(Geo g, SList m, const c_t<T>* __restrict__ M,
                                                   const T* __restrict__ wc, T w, const c_t<T>* __restrict__ f,
                                                   c_t<T>* __restrict__ u, const int* active) {
  prefetch_block_planes<T>(g, M, m.n, m.rho);
  pdl_enter();
  if (active && !*active) return;
  const bool in = interior_block<DIM>(g, m.rho);
  int x, y, z, p, q;
  if (!node_xyz(g, x, y, z, p, q)) return;
  auto ld = [f HZ_EXT((long long)g.N * g.R)](int i) { return ldp<T, VR>(f, HZ_AT(i, hz_ext)); };
  const pk_t<T, VR> v = in ? sym_Au<T, DIM, false, true>(g, m, M, wc, ld, p, q, x, y, z)
                           : sym_Au<T, DIM, true, true>(g, m, M, wc, ld, p, q, x, y, z);
  stp<T, VR>(u, q, w * v);
}

// diagonal M: u = w m0 f and r = f - A u in one pass
template <typename T, int DIM, int AK, int VR, int MB>
__global__ void __launch_bounds__(BX* BY, MB) k_sweep0_resid_diag(Geo g, T invh2, const c_t<T>* __restrict__ A,
                                                              const c_t<T>* __restrict__ m0, T w,
                                                              const c_t<T>* __restrict__ f, c_t<T>* __restrict__ u,
                                                              c_t<T>* __restrict__ r, const int* active) {
  prefetch_block_planes<T>(g, m0, 1, 0);
  prefetch_block_planes<T>(g, A, a_planes<DIM, AK>(), AK == 0 ? 0 : AK % 10);
  pdl_enter();
  if (active && !*active) return;
  constexpr int RA = AK == 0 ? 1 : AK % 10;
  const bool in = interior_block<DIM>(g, RA);
  int x, y, z, p, q;
  if (!node_xyz(g, x, y, z, p, q)) return;
  const int lr = g.lr;
  auto ld = [m0, f, w, lr HZ_EXT((long long)g.N * g.R)](int i) {
    const int j = (int)HZ_AT(i, hz_ext);
    return w * cmul(m0[j >> lr], ldp<T, VR>(f, j));
  };
  const pk_t<T, VR> a = in ? apply_A<T, DIM, AK, false>(g, invh2, A, ld, p, q, x, y, z)
                           : apply_A<T, DIM, AK, true>(g, invh2, A, ld, p, q, x, y, z);
  const pk_t<T, VR> fp = ldp<T, VR>(f, q);
  stp<T, VR>(u, q, w * cmul(m0[p], fp));
  stp<T, VR>(r, q, fp - a);
}

// out = in + w M r  (out may alias in)
template <typename T, int DIM, int VR, int MB>
__global__ void __launch_bounds__(BX* BY, MB) k_sweep_out(Geo g, MList m, const c_t<T>* __restrict__ M, T w,
                                                      const c_t<T>* __restrict__ r, const c_t<T>* in, c_t<T>* out,
                                                      const int* active) {
  prefetch_block_planes<T>(g, M, m.n, 0);
  pdl_enter();
  if (active && !*active) return;
  const bool inb = interior_block<DIM>(g, m.rho);
  int x, y, z, p, q;
  if (!node_xyz(g, x, y, z, p, q)) return;
  auto ld = [r HZ_EXT((long long)g.N * g.R)](int i) { return ldp<T, VR>(r, HZ_AT(i, hz_ext)); };
  const pk_t<T, VR> v = inb ? list_Au<T, DIM, false>(g, m, M, ld, p, q, x, y, z)
                            : list_Au<T, DIM, true>(g, m, M, ld, p, q, x, y, z);
  stp<T, VR>(out, q, ldp<T, VR>(in, q) + w * v);
}

// symmetric half form: out = in + w D^{-1} M' r
template <typename T, int DIM, int VR, int MB>
__global__ void __launch_bounds__(BX* BY, MB) k_sweep_out_sym(Geo g, SList m, const c_t<T>* __restrict__ M,
                                                      const T* __restrict__ wc, T w, const c_t<T>* __restrict__ r,
                                                      const c_t<T>* in, c_t<T>* out, const int* active) {
  prefetch_block_planes<T>(g, M, m.n, m.rho);
  pdl_enter();
  if (active && !*active) return;
  const bool inb = interior_block<DIM>(g, m.rho);
  int x, y, z, p, q;
  if (!node_xyz(g, x, y, z, p, q)) return;
  auto ld = [r HZ_EXT((long long)g.N * g.R)](int i) { return ldp<T, VR>(r, HZ_AT(i, hz_ext)); };
  const pk_t<T, VR> v = inb ? sym_Au<T, DIM, false, true>(g, m, M, wc, ld, p, q, x, y, z)
                            : sym_Au<T, DIM, true, true>(g, m, M, wc, ld, p, q, x, y, z);
  stp<T, VR>(out, q, ldp<T, VR>(in, q) + w * v);
}

// diagonal M: out = in + w m0 (f - A in)   (out != in)
template <typename T, int DIM, int AK, int VR, int MB>
__global__ void __launch_bounds__(BX* BY, MB) k_resid_sweep_diag(Geo g, T invh2, const c_t<T>* __restrict__ A,
                                                             const c_t<T>* __restrict__ m0, T w,
                                                             const c_t<T>* __restrict__ f, const c_t<T>* __restrict__ in,
                                                             c_t<T>* __restrict__ out, const int* active) {
  prefetch_block_planes<T>(g, m0, 1, 0);
  prefetch_block_planes<T>(g, A, a_planes<DIM, AK>(), AK == 0 ? 0 : AK % 10);
  pdl_enter();
  if (active && !*active) return;
  constexpr int RA = AK == 0 ? 1 : AK % 10;
  const bool inb = interior_block<DIM>(g, RA);
  int x, y, z, p, q;
  if (!node_xyz(g, x, y, z, p, q)) return;
  auto ld = [in HZ_EXT((long long)g.N * g.R)](int i) { return ldp<T, VR>(in, HZ_AT(i, hz_ext)); };
  const pk_t<T, VR> a = inb ? apply_A<T, DIM, AK, false>(g, invh2, A, ld, p, q, x, y, z)
                            : apply_A<T, DIM, AK, true>(g, invh2, A, ld, p, q, x, y, z);
  stp<T, VR>(out, q, ldp<T, VR>(in, q) + w * cmul(m0[p], ldp<T, VR>(f, q) - a));
}

// 1D prolongation weight P(j, J) in single precision (the same exact dyadic
// values as p1; computed with integer tests and float constants only, since
// FP64 arithmetic and conversions are slow on this GPU)
__device__ __forceinline__ float p1f(int kind, int nf, int nc, int j, int J) {
  const int d = j - 2 * J;
  const int ad = d < 0 ? -d : d;
  if (kind == 0) return ad == 0 ? 1.0f : (ad == 1 ? 0.5f : 0.0f);
  float w = ad == 0 ? 0.75f : (ad == 1 ? 0.5f : (ad == 2 ? 0.125f : 0.0f));
  if (j == 0 && J == 1) w += 0.125f;
  if (j == nf - 1 && J == nc - 2) w += 0.125f;
  return w;
}

// f_c = R r, one thread per coarse node (and RHS pack)
template <typename T, int DIM, int KIND, int VR, int MB>
__global__ void __launch_bounds__(BX* BY, MB) k_restrict(Geo gf, Geo gc, const c_t<T>* __restrict__ r,
                                                     c_t<T>* __restrict__ fc, const int* active) {
  pdl_enter();
  if (active && !*active) return;
  int X, Y, Z, pc, qc;
  if (!node_xyz(gc, X, Y, Z, pc, qc)) return;
  const int rr = qc & (gc.R - 1);
  constexpr int RAD = KIND ? 2 : 1;
  constexpr int RZ = DIM == 3 ? RAD : 0;
  // weights are zero outside the fine grid; those terms read a clamped (valid)
  // index, so the loops carry no branches and the loads issue together
  T wx[2 * RAD + 1], wy[2 * RAD + 1], wz[2 * RZ + 1];
  int ix[2 * RAD + 1], iy[2 * RAD + 1], iz[2 * RZ + 1];
#pragma unroll
  for (int k = 0; k <= 2 * RAD; ++k) {
    const int jx = 2 * X - RAD + k, jy = 2 * Y - RAD + k;
    const bool okx = jx >= 0 && jx < gf.nx, oky = jy >= 0 && jy < gf.ny;
    wx[k] = okx ? (T)(0.5f * p1f(KIND, gf.nx, gc.nx, jx, X)) : T(0);
    wy[k] = oky ? (T)(0.5f * p1f(KIND, gf.ny, gc.ny, jy, Y)) : T(0);
    ix[k] = okx ? jx : 2 * X;
    iy[k] = oky ? jy : 2 * Y;
  }
#pragma unroll
  for (int k = 0; k <= 2 * RZ; ++k) {
    const int jz = 2 * Z - RZ + k;
    const bool okz = DIM == 2 || (jz >= 0 && jz < gf.nz);
    wz[k] = DIM == 3 ? (okz ? (T)(0.5f * p1f(KIND, gf.nz, gc.nz, jz, Z)) : T(0)) : T(1);
    iz[k] = okz ? jz : 2 * Z;
  }
  pk_t<T, VR> acc = pk_zero<pk_t<T, VR>>();
#pragma unroll
  for (int kz = 0; kz <= 2 * RZ; ++kz) {
#pragma unroll
    for (int ky = 0; ky <= 2 * RAD; ++ky) {
      const T wyz = wy[ky] * wz[kz];
      const int row = (iz[kz] * gf.ny + iy[ky]) * gf.nx;
#pragma unroll
      for (int kx = 0; kx <= 2 * RAD; ++kx)
        acc = acc + (wyz * wx[kx]) * ldp<T, VR>(r, (int)HZ_AT((row + ix[kx]) * gf.R + rr, (long long)gf.N * gf.R));
    }
  }
  stp<T, VR>(fc, (int)HZ_AT(qc, (long long)gc.N * gc.R), acc);
}

// 1D prolongation stencil of fine index j: coarse nodes J0, J0+1, J0+2 with
// weights w[0..2] (zero where unused).  Odd j = 2J+1: (c_J + c_{J+1})/2 for both
// kinds; even j = 2J: c_J (linear) or (c_{J-1} + 6 c_J + c_{J+1})/8 (cubic), the
// two end nodes using the mirrored ghost (3/4, 1/4).  Same values as p1.
template <int KIND>
__device__ __forceinline__ int p1_stencil(int j, int nf, int nc, float (&w)[3]) {
  const int J = j >> 1;
  if (j & 1) {
    w[0] = 0.5f; w[1] = 0.5f; w[2] = 0.0f;
    return J;
  }
  if (KIND == 0) {
    w[0] = 1.0f; w[1] = 0.0f; w[2] = 0.0f;
    return J;
  }
  if (j == 0) {
    w[0] = 0.75f; w[1] = 0.25f; w[2] = 0.0f;
    return 0;
  }
  if (j == nf - 1) {
    w[0] = 0.25f; w[1] = 0.75f; w[2] = 0.0f;
    return nc - 2;
  }
  w[0] = 0.125f; w[1] = 0.75f; w[2] = 0.125f;
  return J - 1;
}

// (P e_c) at fine node (x, y, z), RHS pack starting at rr
template <typename T, int DIM, int KIND, int VR = 1>
__device__ __forceinline__ pk_t<T, VR> prolong_at(const Geo& gf, const Geo& gc, const c_t<T>* __restrict__ ec, int x,
                                                  int y, int z, int rr = 0) {
  float wx[3], wy[3], wz[3] = {1.0f, 0.0f, 0.0f};
  const int X0 = p1_stencil<KIND>(x, gf.nx, gc.nx, wx);
  const int Y0 = p1_stencil<KIND>(y, gf.ny, gc.ny, wy);
  const int Z0 = DIM == 3 ? p1_stencil<KIND>(z, gf.nz, gc.nz, wz) : 0;
  pk_t<T, VR> acc = pk_zero<pk_t<T, VR>>();
#pragma unroll
  for (int c = 0; c < (DIM == 3 ? 3 : 1); ++c) {
    if (wz[c] == 0.0f) continue;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float wyz = wz[c] * wy[b];
      if (wyz == 0.0f) continue;
      const int row = (((Z0 + c) * gc.ny + Y0 + b) * gc.nx + X0) * gc.R + rr;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (wx[a] == 0.0f) continue;
        acc = acc + (T)(wyz * wx[a]) * ldp<T, VR>(ec, (int)HZ_AT(row + a * gc.R, (long long)gc.N * gc.R));
      }
    }
  }
  return acc;
}

// out = in + P e_c (pointwise; out may alias in)
template <typename T, int DIM, int KIND, int VR, int MB>
__global__ void __launch_bounds__(BX* BY, MB) k_prolong(Geo gf, Geo gc, const c_t<T>* __restrict__ ec, const c_t<T>* in,
                                                    c_t<T>* out, const int* active) {
  pdl_enter();
  if (active && !*active) return;
  int x, y, z, p, q;
  if (!node_xyz(gf, x, y, z, p, q)) return;
  stp<T, VR>(out, q, ldp<T, VR>(in, q) + prolong_at<T, DIM, KIND, VR>(gf, gc, ec, x, y, z, q & (gf.R - 1)));
}

// 2D: u' = t + P e_c on a tile with halo RA in shared memory, then
//   DIAG = false: out = u', r = f - A u'
//   DIAG = true : out = u' + w m0 (f - A u')
template <typename T, int AK, int KIND, bool DIAG, int MB>
__global__ void __launch_bounds__(BX* BY, MB) k_prolong_fused_2d(Geo gf, Geo gc, T invh2, const c_t<T>* __restrict__ A,
                                                             const c_t<T>* __restrict__ ec, const c_t<T>* __restrict__ t,
                                                             const c_t<T>* __restrict__ f, const c_t<T>* __restrict__ m0,
                                                             T w, c_t<T>* __restrict__ out, c_t<T>* __restrict__ r,
                                                             const int* active) {
  prefetch_block_planes<T>(gf, A, a_planes<2, AK>(), AK == 0 ? 0 : AK % 10);
  if (DIAG) prefetch_block_planes<T>(gf, m0, 1, 0);
  pdl_enter();
  if (active && !*active) return;
  constexpr int RA = AK == 0 ? 1 : AK % 10;
  constexpr int TX = BX + 2 * RA, TY = BY + 2 * RA;
  __shared__ c_t<T> sm[TY][TX];
  const int x0 = blockIdx.x * BX - RA, y0 = blockIdx.y * BY - RA;
  const int tid = threadIdx.y * BX + threadIdx.x;
  for (int i = tid; i < TX * TY; i += BX * BY) {
    const int ty = i / TX, tx = i - ty * TX;
    const int gx = x0 + tx, gy = y0 + ty;
    c_t<T> v = cmk<c_t<T>>(0, 0);
    if (gx >= 0 && gx < gf.nx && gy >= 0 && gy < gf.ny)
      v = t[HZ_AT(gy * gf.nx + gx, gf.N)] + prolong_at<T, 2, KIND>(gf, gc, ec, gx, gy, 0);
    sm[ty][tx] = v;
  }
  __syncthreads();
  int x, y, z, p, q;
  if (!node_xyz(gf, x, y, z, p, q)) return;
  const int lx = threadIdx.x + RA, ly = threadIdx.y + RA;
  const c_t<T> up = sm[ly][lx];
  c_t<T> a;
  if constexpr (AK == 0) {
    // zeros outside the grid in the tile: the neighbour sums are the in-grid sums
    const T wx = (x == 0 || x == gf.nx - 1) ? T(0.5) : T(1);
    const T wy = (y == 0 || y == gf.ny - 1) ? T(0.5) : T(1);
    const c_t<T> sx = sm[ly][lx - 1] + sm[ly][lx + 1];
    const c_t<T> sy = sm[ly - 1][lx] + sm[ly + 1][lx];
    a = cmul(A[p], up);
    a.x -= invh2 * (wy * sx.x + wx * sy.x);
    a.y -= invh2 * (wy * sx.y + wx * sy.y);
  } else if constexpr (AK > 10) {
    // symmetric half (box_Au_half): the tile holds zeros outside the grid, and
    // a mirrored entry whose node p - s is outside is read at p instead
    a = cmk<c_t<T>>(0, 0);
    constexpr int R0 = AK - 10, W = 2 * R0 + 1, C = (W * W - 1) / 2;
#pragma unroll
    for (int dy = -R0; dy <= R0; ++dy)
#pragma unroll
      for (int dx = -R0; dx <= R0; ++dx) {
        const int s = (dy + R0) * W + (dx + R0);
        if (s < C) continue;
        a = cfma(A[HZ_AT((s - C) * gf.N + p, (long long)(C + 1) * gf.N)], sm[ly + dy][lx + dx], a);
        if (s == C) continue;
        const bool ok = x - dx >= 0 && x - dx < gf.nx && y - dy >= 0 && y - dy < gf.ny;
        a = cfma(A[HZ_AT((s - C) * gf.N + (ok ? p - dx - dy * gf.nx : p), (long long)(C + 1) * gf.N)],
                 sm[ly - dy][lx - dx], a);
      }
  } else {
    // coefficients reaching outside the grid are stored as zeros
    a = cmk<c_t<T>>(0, 0);
    constexpr int W = 2 * AK + 1;
#pragma unroll
    for (int dy = -AK; dy <= AK; ++dy)
#pragma unroll
      for (int dx = -AK; dx <= AK; ++dx)
        a = cfma(A[HZ_AT(((dy + AK) * W + (dx + AK)) * gf.N + p, (long long)W * W * gf.N)], sm[ly + dy][lx + dx], a);
  }
  const c_t<T> res = f[p] - a;
  if (DIAG) {
    out[p] = up + scale(cmul(m0[p], res), w);
  } else {
    out[p] = up;
    r[p] = res;
  }
}

// ---- fine level with a diagonal smoother, one right-hand side --------------
// With M diagonal (damped Jacobi, or RB patches on the 2d+1-point fine
// stencil) and nu1 = nu2 = 1 the fine level of a V-cycle is two passes:
//   down:  t = w m0 f,  r = f - A t,  f_c = R r      (t, r in shared memory only)
//   up:    u' = w m0 f + P e_c,  out = u' + w m0 (f - A u')
// t = w m0 f is recomputed by the upward pass from f and m0, which it reads
// for the post-smoothing anyway, so neither t nor r ever goes to HBM: per
// fine node the level moves f, m0, A twice and out once (plus the coarse
// vectors), against the five separate reads/writes of t and r otherwise.
// Out-of-grid tile entries are zero, so the neighbour sums are the in-grid
// sums; the operator uses the half-cell boundary weights of the fine stencil.

// fine 2D operator at tile position (ly, lx) of a tile holding u with zeros
// outside the grid: A u = d u - (1/h^2)(wy (u_W + u_E) + wx (u_S + u_N))
template <typename T, int W>
__device__ __forceinline__ c_t<T> fine_tile_Au_2d(const c_t<T> (*su)[W], int ly, int lx, c_t<T> d, T invh2, int x,
                                                  int y, const Geo& g) {
  const T wx = (x == 0 || x == g.nx - 1) ? T(0.5) : T(1);
  const T wy = (y == 0 || y == g.ny - 1) ? T(0.5) : T(1);
  const c_t<T> up = su[ly][lx];
  const c_t<T> sx = su[ly][lx - 1] + su[ly][lx + 1];
  const c_t<T> sy = su[ly - 1][lx] + su[ly + 1][lx];
  c_t<T> a = cmul(d, up);
  a.x -= invh2 * (wy * sx.x + wx * sy.x);
  a.y -= invh2 * (wy * sx.y + wx * sy.y);
  return a;
}

// down pass, 2D: one block = CX x CY coarse nodes (32 x 8 threads).  The
// restriction is applied separably: first along x for every fine row of the
// residual region, then along y.
template <typename T, int RK, int MB>
__global__ void __launch_bounds__(BX* BY, MB ? MB : 4) k_fine_down_diag_2d(Geo gf, Geo gc, T invh2, const c_t<T>* __restrict__ A,
                                                                  const c_t<T>* __restrict__ m0, T w,
                                                                  const c_t<T>* __restrict__ f,
                                                                  c_t<T>* __restrict__ fc, const int* active) {
  constexpr int CX = 32, CY = sizeof(T) == 4 ? 8 : 4;
  constexpr int RR = RK ? 2 : 1;                       // restriction reach in fine nodes
  constexpr int RX = 2 * CX - 1 + 2 * RR, RY = 2 * CY - 1 + 2 * RR;   // residual region
  constexpr int TX = RX + 2, TY = RY + 2;             // t region (residual region + operator halo)
  constexpr int NTH = BX * BY;
  __shared__ c_t<T> st[TY][TX];
  __shared__ c_t<T> sr[RY][RX];
  __shared__ c_t<T> sh[RY][CX];                       // residual rows restricted along x
  const int tid = threadIdx.y * BX + threadIdx.x;
  const int X0 = blockIdx.x * CX, Y0 = blockIdx.y * CY;
  const int rx0 = 2 * X0 - RR, ry0 = 2 * Y0 - RR;
  // the diagonals of the smoother and the operator (setup data) over the t region
  prefetch_l2_planes(m0, 1, gf.N, gf.nx, gf.ny, rx0 - 1, TX, ry0 - 1, TY, tid, NTH);
  prefetch_l2_planes(A, 1, gf.N, gf.nx, gf.ny, rx0, RX, ry0, RY, tid, NTH);
  pdl_enter();
  if (active && !*active) return;
  // every entry's loads of a phase are issued before any is used (fixed,
  // unrolled trip counts): one memory round trip per phase
  constexpr int NT = (TX * TY + NTH - 1) / NTH, NR = (RX * RY + NTH - 1) / NTH;
  {
    c_t<T> mv[NT], fv[NT];
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      const int i = tid + k * NTH, ty = i / TX, tx = i - ty * TX;
      const int gx = rx0 - 1 + tx, gy = ry0 - 1 + ty;
      const bool in = i < TX * TY && gx >= 0 && gx < gf.nx && gy >= 0 && gy < gf.ny;
      const int p = (int)HZ_AT(in ? gy * gf.nx + gx : 0, gf.N);
      mv[k] = in ? m0[p] : cmk<c_t<T>>(0, 0);
      fv[k] = in ? f[p] : cmk<c_t<T>>(0, 0);
    }
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      const int i = tid + k * NTH, ty = i / TX, tx = i - ty * TX;
      if (i < TX * TY) st[ty][tx] = w * cmul(mv[k], fv[k]);
    }
  }
  __syncthreads();
  {
    c_t<T> av[NR], fv[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      const int i = tid + k * NTH, ry = i / RX, rx = i - ry * RX;
      const int gx = rx0 + rx, gy = ry0 + ry;
      const bool in = i < RX * RY && gx >= 0 && gx < gf.nx && gy >= 0 && gy < gf.ny;
      const int p = (int)HZ_AT(in ? gy * gf.nx + gx : 0, gf.N);
      av[k] = in ? A[p] : cmk<c_t<T>>(0, 0);
      fv[k] = in ? f[p] : cmk<c_t<T>>(0, 0);
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      const int i = tid + k * NTH, ry = i / RX, rx = i - ry * RX;
      const int gx = rx0 + rx, gy = ry0 + ry;
      if (i >= RX * RY) continue;
      const bool in = gx >= 0 && gx < gf.nx && gy >= 0 && gy < gf.ny;
      sr[ry][rx] = in ? fv[k] - fine_tile_Au_2d<T, TX>(st, ry + 1, rx + 1, av[k], invh2, gx, gy, gf)
                      : cmk<c_t<T>>(0, 0);
    }
  }
  __syncthreads();
  // R r = Ry (Rx r): weights 0.5 * P(j, J) per axis, zero outside the fine grid
  const int cx = threadIdx.x, X = X0 + cx;
  {
    T wx[2 * RR + 1];
#pragma unroll
    for (int k = 0; k <= 2 * RR; ++k) {
      const int jx = 2 * X - RR + k;
      wx[k] = (jx >= 0 && jx < gf.nx && X < gc.nx) ? (T)(0.5f * p1f(RK, gf.nx, gc.nx, jx, X)) : T(0);
    }
    for (int ry = threadIdx.y; ry < RY; ry += BY) {
      c_t<T> acc = cmk<c_t<T>>(0, 0);
#pragma unroll
      for (int k = 0; k <= 2 * RR; ++k) acc = acc + wx[k] * sr[ry][2 * cx + k];
      sh[ry][cx] = acc;
    }
  }
  __syncthreads();
  const int cy = threadIdx.y, Y = Y0 + cy;
  if (cy >= CY || X >= gc.nx || Y >= gc.ny) return;
  c_t<T> acc = cmk<c_t<T>>(0, 0);
#pragma unroll
  for (int k = 0; k <= 2 * RR; ++k) {
    const int jy = 2 * Y - RR + k;
    const T wy = (jy >= 0 && jy < gf.ny) ? (T)(0.5f * p1f(RK, gf.ny, gc.ny, jy, Y)) : T(0);
    acc = acc + wy * sh[2 * cy + k][cx];
  }
  fc[HZ_AT(Y * gc.nx + X, gc.N)] = acc;
}

// up pass, 2D: one block = 64 x FY fine nodes (2 x FY/8 per thread).  The
// coarse correction's tile is staged in shared memory and prolongated
// separably: along x for each coarse row the tile needs (weights and first
// coarse index per fine column and row computed once per block), then along y.
template <typename T, int PK, int MB>
__global__ void __launch_bounds__(BX* BY, MB ? MB : 4) k_fine_up_diag_2d(Geo gf, Geo gc, T invh2, const c_t<T>* __restrict__ A,
                                                                const c_t<T>* __restrict__ m0, T w,
                                                                const c_t<T>* __restrict__ f,
                                                                const c_t<T>* __restrict__ ec, c_t<T>* __restrict__ out,
                                                                const int* active) {
  constexpr int FX = 64, FY = sizeof(T) == 4 ? 16 : 8;
  constexpr int UX = FX + 2, UY = FY + 2;            // u' tile with the operator halo
  constexpr int EX = FX / 2 + 4, EY = FY / 2 + 4;    // coarse values the tile's prolongation reads
  constexpr int NTH = BX * BY;
  __shared__ c_t<T> su[UY][UX];
  __shared__ c_t<T> sf[UY][UX];
  __shared__ c_t<T> sm[UY][UX];
  __shared__ c_t<T> se[EY][EX];
  __shared__ c_t<T> sh[EY][UX];                      // coarse rows prolongated along x
  __shared__ float wcx[UX][3], wcy[UY][3];
  __shared__ int icx[UX], icy[UY];
  const int tid = threadIdx.y * BX + threadIdx.x;
  const int x0 = blockIdx.x * FX, y0 = blockIdx.y * FY;
  // the diagonals of the smoother and the operator (setup data) over the tile
  prefetch_l2_planes(m0, 1, gf.N, gf.nx, gf.ny, x0 - 1, UX, y0 - 1, UY, tid, NTH);
  prefetch_l2_planes(A, 1, gf.N, gf.nx, gf.ny, x0, FX, y0, FY, tid, NTH);
  pdl_enter();
  if (active && !*active) return;
  const int ex0 = ((x0 - 1) >> 1) - 1, ey0 = ((y0 - 1) >> 1) - 1;   // coarse origin (floor division)
  constexpr int NE = (EX * EY + NTH - 1) / NTH, NU = (UX * UY + NTH - 1) / NTH;
  c_t<T> fvs[NU], mvs[NU];
  {
    c_t<T> ev[NE];
#pragma unroll
    for (int k = 0; k < NE; ++k) {
      const int i = tid + k * NTH, ey = i / EX, exx = i - ey * EX;
      const int gx = ex0 + exx, gy = ey0 + ey;
      const bool in = i < EX * EY && gx >= 0 && gx < gc.nx && gy >= 0 && gy < gc.ny;
      ev[k] = in ? ec[HZ_AT(gy * gc.nx + gx, gc.N)] : cmk<c_t<T>>(0, 0);
    }
#pragma unroll
    for (int k = 0; k < NU; ++k) {
      const int i = tid + k * NTH, uy = i / UX, ux = i - uy * UX;
      const int gx = x0 - 1 + ux, gy = y0 - 1 + uy;
      const bool in = i < UX * UY && gx >= 0 && gx < gf.nx && gy >= 0 && gy < gf.ny;
      const int p = (int)HZ_AT(in ? gy * gf.nx + gx : 0, gf.N);
      fvs[k] = in ? f[p] : cmk<c_t<T>>(0, 0);
      mvs[k] = in ? m0[p] : cmk<c_t<T>>(0, 0);
    }
#pragma unroll
    for (int k = 0; k < NE; ++k) {
      const int i = tid + k * NTH, ey = i / EX, exx = i - ey * EX;
      if (i < EX * EY) se[ey][exx] = ev[k];
    }
  }
  // per fine column / row of the tile: first coarse index (tile-local) and weights
  if (tid < UX) {
    const int gx = min(max(x0 - 1 + tid, 0), gf.nx - 1);
    float wv[3];
    icx[tid] = p1_stencil<PK>(gx, gf.nx, gc.nx, wv) - ex0;
    wcx[tid][0] = wv[0];
    wcx[tid][1] = wv[1];
    wcx[tid][2] = wv[2];
  } else if (tid >= 128 && tid < 128 + UY) {
    const int t = tid - 128, gy = min(max(y0 - 1 + t, 0), gf.ny - 1);
    float wv[3];
    icy[t] = p1_stencil<PK>(gy, gf.ny, gc.ny, wv) - ey0;
    wcy[t][0] = wv[0];
    wcy[t][1] = wv[1];
    wcy[t][2] = wv[2];
  }
  __syncthreads();
  for (int i = tid; i < EY * UX; i += NTH) {
    const int ey = i / UX, ux = i - ey * UX;
    const int c0 = icx[ux];
    sh[ey][ux] = (T)wcx[ux][0] * se[ey][c0] + (T)wcx[ux][1] * se[ey][c0 + 1] + (T)wcx[ux][2] * se[ey][c0 + 2];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NU; ++k) {
    const int i = tid + k * NTH, uy = i / UX, ux = i - uy * UX;
    if (i >= UX * UY) continue;
    const int gx = x0 - 1 + ux, gy = y0 - 1 + uy;
    c_t<T> v = cmk<c_t<T>>(0, 0);
    if (gx >= 0 && gx < gf.nx && gy >= 0 && gy < gf.ny) {
      const int r0 = icy[uy];
      const c_t<T> pe = (T)wcy[uy][0] * sh[r0][ux] + (T)wcy[uy][1] * sh[r0 + 1][ux] + (T)wcy[uy][2] * sh[r0 + 2][ux];
      v = w * cmul(mvs[k], fvs[k]) + pe;
    }
    su[uy][ux] = v;
    sf[uy][ux] = fvs[k];
    sm[uy][ux] = mvs[k];
  }
  __syncthreads();
  constexpr int NO = (FY / BY) * (FX / BX);
  c_t<T> dv[NO];
#pragma unroll
  for (int k = 0; k < NO; ++k) {
    const int lx = threadIdx.x + (k % (FX / BX)) * BX, ly = threadIdx.y + (k / (FX / BX)) * BY;
    const int x = x0 + lx, y = y0 + ly;
    const bool in = x < gf.nx && y < gf.ny;
    dv[k] = in ? A[HZ_AT(y * gf.nx + x, gf.N)] : cmk<c_t<T>>(0, 0);
  }
#pragma unroll
  for (int k = 0; k < NO; ++k) {
    const int lx = threadIdx.x + (k % (FX / BX)) * BX, ly = threadIdx.y + (k / (FX / BX)) * BY;
    const int x = x0 + lx, y = y0 + ly;
    if (x >= gf.nx || y >= gf.ny) continue;
    const c_t<T> a = fine_tile_Au_2d<T, UX>(su, ly + 1, lx + 1, dv[k], invh2, x, y, gf);
    out[HZ_AT(y * gf.nx + x, gf.N)] = su[ly + 1][lx + 1] + w * cmul(sm[ly + 1][lx + 1], sf[ly + 1][lx + 1] - a);
  }
}

// ---- coarse levels in 2D, one right-hand side: two fused passes -----------
// A coarse level of a V(1,1)-cycle from zero is, as separate launches,
// sweep0 -> residual -> restriction down and prolongation + residual ->
// sweep up: five dependent kernels, each paying launch and memory latency
// (on the small levels that latency, not bandwidth, sets the time).  Here
// each direction is one kernel over shared-memory tiles with the halos the
// chained stencils need, recomputed by every block:
//   down:  t = w M f  (tile + R reach + A reach),  r = f - A t  (tile + R reach),
//          f_c = R r;  t is written for the block's own fine nodes
//   up:    u' = t + P e_c  (tile + M reach + A reach),  r = f - A u'  (tile + M
//          reach),  out = u' + w M r
// The stencil coefficients are read from their planes in HBM / L2 as in the
// separate kernels (same terms in the same order, so t and the residuals are
// the separate kernels' values); only field values go through the tiles.
// Tiles hold zeros outside the grid; an out-of-grid neighbour always has a
// zero coefficient.  The smoother's stencil reach is at most 2 in 2D.

constexpr int kTileRM = 2;
// one block of 1024 threads per tile, so every phase has at most one tile
// point per thread (a phase then waits for about one round of loads)
constexpr int kTileThreads = 1024;

// (M v) at node p from a tile of v (row pitch W; (lx, ly) = p's position):
// the stored half of M' with mirrored entries read at the neighbour, then
// the weight 1/count (SYM), or the planes of M itself
template <typename T, bool SYM, typename LST>
__device__ __forceinline__ c_t<T> tile_Mv(const Geo& g, const LST& m, const c_t<T>* __restrict__ P,
                                          const T* __restrict__ wc, const c_t<T>* tile, int W, int lx, int ly, int p,
                                          int x, int y) {
  c_t<T> acc = cmk<c_t<T>>(0, 0);
#pragma unroll 8
  for (int s = 0; s < m.n; ++s) {
    const int dx = m.d[s][0], dy = m.d[s][1];
    acc = cfma(P[HZ_AT(s * g.N + p, (long long)m.n * g.N)], tile[(ly + dy) * W + lx + dx], acc);
    if constexpr (SYM) {
      if (m.mirror[s]) {
        const bool okm = x - dx >= 0 && x - dx < g.nx && y - dy >= 0 && y - dy < g.ny;
        const c_t<T> cm = okm ? P[HZ_AT(s * g.N + p - m.nflat[s], (long long)m.n * g.N)] : cmk<c_t<T>>(0, 0);
        acc = cfma(cm, tile[(ly - dy) * W + lx - dx], acc);
      }
    }
  }
  if constexpr (SYM) return wc[p] * acc;
  else return acc;
}

// (A v) at node p for a stored box stencil (AK = rho) or its symmetric half
// (AK = 10 + rho), from a tile of v
template <typename T, int AK>
__device__ __forceinline__ c_t<T> tile_Av(const Geo& g, const c_t<T>* __restrict__ A, const c_t<T>* tile, int W, int lx,
                                          int ly, int p, int x, int y) {
  constexpr int RHO = AK % 10, WB = 2 * RHO + 1, C = (WB * WB - 1) / 2;
  c_t<T> acc = cmk<c_t<T>>(0, 0);
#pragma unroll
  for (int dy = -RHO; dy <= RHO; ++dy)
#pragma unroll
    for (int dx = -RHO; dx <= RHO; ++dx) {
      const int s = (dy + RHO) * WB + (dx + RHO);
      if constexpr (AK > 10) {
        if (s < C) continue;
        acc = cfma(A[HZ_AT((s - C) * g.N + p, (long long)(C + 1) * g.N)], tile[(ly + dy) * W + lx + dx], acc);
        if (s == C) continue;
        const bool ok = x - dx >= 0 && x - dx < g.nx && y - dy >= 0 && y - dy < g.ny;
        const c_t<T> cm = ok ? A[HZ_AT((s - C) * g.N + p - dx - dy * g.nx, (long long)(C + 1) * g.N)] : cmk<c_t<T>>(0, 0);
        acc = cfma(cm, tile[(ly - dy) * W + lx - dx], acc);
      } else {
        acc = cfma(A[HZ_AT(s * g.N + p, (long long)WB * WB * g.N)], tile[(ly + dy) * W + lx + dx], acc);
      }
    }
  return acc;
}

template <typename T, int AK, bool SYM, int RK, int MB, typename LST>
__global__ void __launch_bounds__(kTileThreads, 1) k_level_down_2d(Geo gf, Geo gc, const c_t<T>* __restrict__ A,
                                                               LST m, const c_t<T>* __restrict__ M,
                                                               const T* __restrict__ wc, T w,
                                                               const c_t<T>* __restrict__ f, c_t<T>* __restrict__ t,
                                                               c_t<T>* __restrict__ fc, const int* active) {
  constexpr int CX = 16, CY = sizeof(T) == 4 ? 8 : 4;
  constexpr int RR = RK ? 2 : 1, RA = AK % 10, RM = kTileRM;
  constexpr int RX = 2 * CX - 1 + 2 * RR, RY = 2 * CY - 1 + 2 * RR;   // residual region
  constexpr int TX = RX + 2 * RA, TY = RY + 2 * RA;                   // t region
  constexpr int FX = TX + 2 * RM, FY = TY + 2 * RM;                   // f region
  constexpr int NTH = kTileThreads;
  __shared__ c_t<T> sf[FY * FX];
  __shared__ c_t<T> st[TY * TX];
  __shared__ c_t<T> sr[RY * RX];
  __shared__ c_t<T> sh[RY * CX];
  const int tid = threadIdx.x;
  const int X0 = blockIdx.x * CX, Y0 = blockIdx.y * CY;
  const int rx0 = 2 * X0 - RR, ry0 = 2 * Y0 - RR;
  const int tx0 = rx0 - RA, ty0 = ry0 - RA, fx0 = tx0 - RM, fy0 = ty0 - RM;
  // the smoother's planes over the t region (mirrored entries up to RM
  // further) and the operator's over the residual region (mirrored up to RA)
  prefetch_l2_planes(M, m.n, gf.N, gf.nx, gf.ny, fx0, FX, fy0, FY, tid, NTH);
  prefetch_l2_planes(A, AK > 10 ? (2 * RA + 1) * (2 * RA + 1) / 2 + 1 : (2 * RA + 1) * (2 * RA + 1), gf.N, gf.nx,
                     gf.ny, tx0, TX, ty0, TY, tid, NTH);
  pdl_enter();
  if (active && !*active) return;
  constexpr int NF = (FX * FY + NTH - 1) / NTH;
  {
    c_t<T> v[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      const int i = tid + k * NTH, ly = i / FX, lx = i - ly * FX;
      const int gx = fx0 + lx, gy = fy0 + ly;
      const bool in = i < FX * FY && gx >= 0 && gx < gf.nx && gy >= 0 && gy < gf.ny;
      v[k] = in ? f[HZ_AT(gy * gf.nx + gx, gf.N)] : cmk<c_t<T>>(0, 0);
    }
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      const int i = tid + k * NTH;
      if (i < FX * FY) sf[i] = v[k];
    }
  }
  __syncthreads();
  // t = w M f on the t region; written out for the block's own fine nodes
  for (int i = tid; i < TX * TY; i += NTH) {
    const int ly = i / TX, lx = i - ly * TX;
    const int gx = tx0 + lx, gy = ty0 + ly;
    c_t<T> v = cmk<c_t<T>>(0, 0);
    if (gx >= 0 && gx < gf.nx && gy >= 0 && gy < gf.ny) {
      const int p = (int)HZ_AT(gy * gf.nx + gx, gf.N);
      v = w * tile_Mv<T, SYM>(gf, m, M, wc, sf, FX, lx + RM, ly + RM, p, gx, gy);
      if (gx >= 2 * X0 && gx < 2 * X0 + 2 * CX && gy >= 2 * Y0 && gy < 2 * Y0 + 2 * CY) t[p] = v;
    }
    st[i] = v;
  }
  __syncthreads();
  for (int i = tid; i < RX * RY; i += NTH) {
    const int ly = i / RX, lx = i - ly * RX;
    const int gx = rx0 + lx, gy = ry0 + ly;
    c_t<T> v = cmk<c_t<T>>(0, 0);
    if (gx >= 0 && gx < gf.nx && gy >= 0 && gy < gf.ny) {
      const int p = (int)HZ_AT(gy * gf.nx + gx, gf.N);
      v = sf[(ly + RA + RM) * FX + lx + RA + RM] - tile_Av<T, AK>(gf, A, st, TX, lx + RA, ly + RA, p, gx, gy);
    }
    sr[i] = v;
  }
  __syncthreads();
  // f_c = Ry (Rx r)
  for (int i = tid; i < RY * CX; i += NTH) {
    const int ly = i / CX, cx = i - ly * CX, X = X0 + cx;
    c_t<T> acc = cmk<c_t<T>>(0, 0);
    if (X < gc.nx) {
#pragma unroll
      for (int k = 0; k <= 2 * RR; ++k) {
        const int jx = 2 * X - RR + k;
        const T wx = (jx >= 0 && jx < gf.nx) ? (T)(0.5f * p1f(RK, gf.nx, gc.nx, jx, X)) : T(0);
        acc = acc + wx * sr[ly * RX + 2 * cx + k];
      }
    }
    sh[i] = acc;
  }
  __syncthreads();
  for (int i = tid; i < CX * CY; i += NTH) {
    const int cy = i / CX, cx = i - cy * CX, X = X0 + cx, Y = Y0 + cy;
    if (X >= gc.nx || Y >= gc.ny) continue;
    c_t<T> acc = cmk<c_t<T>>(0, 0);
#pragma unroll
    for (int k = 0; k <= 2 * RR; ++k) {
      const int jy = 2 * Y - RR + k;
      const T wy = (jy >= 0 && jy < gf.ny) ? (T)(0.5f * p1f(RK, gf.ny, gc.ny, jy, Y)) : T(0);
      acc = acc + wy * sh[(2 * cy + k) * CX + cx];
    }
    fc[HZ_AT(Y * gc.nx + X, gc.N)] = acc;
  }
}

template <typename T, int AK, bool SYM, int PK, int MB, typename LST>
__global__ void __launch_bounds__(kTileThreads, 1) k_level_up_2d(Geo gf, Geo gc, const c_t<T>* __restrict__ A,
                                                             LST m, const c_t<T>* __restrict__ M,
                                                             const T* __restrict__ wc, T w,
                                                             const c_t<T>* __restrict__ f, const c_t<T>* __restrict__ t,
                                                             const c_t<T>* __restrict__ ec, c_t<T>* __restrict__ out,
                                                             const int* active) {
  constexpr int OX = 32, OY = sizeof(T) == 4 ? 16 : 8;                 // owned fine nodes
  constexpr int RA = AK % 10, RM = kTileRM;
  constexpr int RX = OX + 2 * RM, RY = OY + 2 * RM;                   // residual region
  constexpr int UX = RX + 2 * RA, UY = RY + 2 * RA;                   // u' region
  constexpr int EX = UX / 2 + 4, EY = UY / 2 + 4;                     // coarse values P reads
  constexpr int NTH = kTileThreads;
  __shared__ c_t<T> su[UY * UX];
  __shared__ c_t<T> sr[RY * RX];
  __shared__ c_t<T> se[EY * EX];
  __shared__ c_t<T> sh[EY * UX];
  __shared__ float wcx[UX][3], wcy[UY][3];
  __shared__ int icx[UX], icy[UY];
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * OX, y0 = blockIdx.y * OY;
  const int ux0 = x0 - RM - RA, uy0 = y0 - RM - RA;
  // the operator's planes over the u' region, the smoother's over the
  // residual region (each with its mirrored reach)
  prefetch_l2_planes(A, AK > 10 ? (2 * RA + 1) * (2 * RA + 1) / 2 + 1 : (2 * RA + 1) * (2 * RA + 1), gf.N, gf.nx,
                     gf.ny, ux0, UX, uy0, UY, tid, NTH);
  prefetch_l2_planes(M, m.n, gf.N, gf.nx, gf.ny, ux0, UX, uy0, UY, tid, NTH);
  pdl_enter();
  if (active && !*active) return;
  const int ex0 = (ux0 >> 1) - 1, ey0 = (uy0 >> 1) - 1;             // floor division
  constexpr int NE = (EX * EY + NTH - 1) / NTH, NU = (UX * UY + NTH - 1) / NTH;
  c_t<T> tv[NU];
  {
    c_t<T> ev[NE];
#pragma unroll
    for (int k = 0; k < NE; ++k) {
      const int i = tid + k * NTH, ly = i / EX, lx = i - ly * EX;
      const int gx = ex0 + lx, gy = ey0 + ly;
      const bool in = i < EX * EY && gx >= 0 && gx < gc.nx && gy >= 0 && gy < gc.ny;
      ev[k] = in ? ec[HZ_AT(gy * gc.nx + gx, gc.N)] : cmk<c_t<T>>(0, 0);
    }
#pragma unroll
    for (int k = 0; k < NU; ++k) {
      const int i = tid + k * NTH, ly = i / UX, lx = i - ly * UX;
      const int gx = ux0 + lx, gy = uy0 + ly;
      const bool in = i < UX * UY && gx >= 0 && gx < gf.nx && gy >= 0 && gy < gf.ny;
      tv[k] = in ? t[HZ_AT(gy * gf.nx + gx, gf.N)] : cmk<c_t<T>>(0, 0);
    }
#pragma unroll
    for (int k = 0; k < NE; ++k) {
      const int i = tid + k * NTH;
      if (i < EX * EY) se[i] = ev[k];
    }
  }
  if (tid < UX) {
    const int gx = min(max(ux0 + tid, 0), gf.nx - 1);
    float wv[3];
    icx[tid] = p1_stencil<PK>(gx, gf.nx, gc.nx, wv) - ex0;
    wcx[tid][0] = wv[0];
    wcx[tid][1] = wv[1];
    wcx[tid][2] = wv[2];
  } else if (tid >= 128 && tid < 128 + UY) {
    const int k = tid - 128, gy = min(max(uy0 + k, 0), gf.ny - 1);
    float wv[3];
    icy[k] = p1_stencil<PK>(gy, gf.ny, gc.ny, wv) - ey0;
    wcy[k][0] = wv[0];
    wcy[k][1] = wv[1];
    wcy[k][2] = wv[2];
  }
  __syncthreads();
  for (int i = tid; i < EY * UX; i += NTH) {
    const int ly = i / UX, lx = i - ly * UX;
    const int c0 = icx[lx];
    sh[i] = (T)wcx[lx][0] * se[ly * EX + c0] + (T)wcx[lx][1] * se[ly * EX + c0 + 1] +
            (T)wcx[lx][2] * se[ly * EX + c0 + 2];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NU; ++k) {
    const int i = tid + k * NTH, ly = i / UX, lx = i - ly * UX;
    if (i >= UX * UY) continue;
    const int gx = ux0 + lx, gy = uy0 + ly;
    c_t<T> v = cmk<c_t<T>>(0, 0);
    if (gx >= 0 && gx < gf.nx && gy >= 0 && gy < gf.ny) {
      const int r0 = icy[ly];
      v = tv[k] + ((T)wcy[ly][0] * sh[r0 * UX + lx] + (T)wcy[ly][1] * sh[(r0 + 1) * UX + lx] +
                   (T)wcy[ly][2] * sh[(r0 + 2) * UX + lx]);
    }
    su[i] = v;
  }
  __syncthreads();
  for (int i = tid; i < RX * RY; i += NTH) {
    const int ly = i / RX, lx = i - ly * RX;
    const int gx = x0 - RM + lx, gy = y0 - RM + ly;
    c_t<T> v = cmk<c_t<T>>(0, 0);
    if (gx >= 0 && gx < gf.nx && gy >= 0 && gy < gf.ny) {
      const int p = (int)HZ_AT(gy * gf.nx + gx, gf.N);
      v = f[p] - tile_Av<T, AK>(gf, A, su, UX, lx + RA, ly + RA, p, gx, gy);
    }
    sr[i] = v;
  }
  __syncthreads();
  for (int i = tid; i < OX * OY; i += NTH) {
    const int ly = i / OX, lx = i - ly * OX;
    const int gx = x0 + lx, gy = y0 + ly;
    if (gx >= gf.nx || gy >= gf.ny) continue;
    const int p = (int)HZ_AT(gy * gf.nx + gx, gf.N);
    out[p] = su[(ly + RM + RA) * UX + lx + RM + RA] + w * tile_Mv<T, SYM>(gf, m, M, wc, sr, RX, lx + RM, ly + RM, p, gx, gy);
  }
}

// u = Ainv f: TPR threads per row (256 / TPR rows per block of 256), four
// independent accumulators per thread so that several row loads are in flight
// (the matrix is streamed once per cycle); warp shuffles, then the row's warps
// added in a fixed order through shared memory (deterministic).
template <typename T, int TPR>
__global__ void __launch_bounds__(256) k_dense_gemv(int n, const c_t<T>* __restrict__ A, const c_t<T>* __restrict__ f,
                                                    c_t<T>* __restrict__ u, const int* active) {
  {
    // this block's rows of the inverse (setup data) into L2 while the
    // previous kernel runs
    constexpr int RPB = 256 / TPR;
    const int r0 = blockIdx.x * RPB, r1 = (r0 + RPB < n ? r0 + RPB : n) - 1;
    if (r0 <= r1) prefetch_l2_span(A, (long long)r0 * n, (long long)r1 * n + n - 1, threadIdx.x, 256);
  }
  pdl_enter();
  if (active && !*active) return;
  using V = c_t<T>;
  constexpr int RPB = 256 / TPR, WPR = TPR / 32;
  __shared__ V part[RPB][WPR];
  const int tr = threadIdx.x % TPR, rb = threadIdx.x / TPR;
  const int row = blockIdx.x * RPB + rb;
  V acc[4] = {cmk<V>(0, 0), cmk<V>(0, 0), cmk<V>(0, 0), cmk<V>(0, 0)};
  if (row < n) {
    const V* a = A + (long long)row * n;
    int j = tr;
    for (; j + 3 * TPR < n; j += 4 * TPR) {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        acc[k] = cfma(a[HZ_AT(j + k * TPR, n)], f[HZ_AT(j + k * TPR, n)], acc[k]);
    }
    for (int k = 0; j < n; j += TPR, ++k) acc[k] = cfma(a[HZ_AT(j, n)], f[HZ_AT(j, n)], acc[k]);
  }
  V t = (acc[0] + acc[1]) + (acc[2] + acc[3]);
  for (int o = 16; o > 0; o >>= 1) {
    t.x += __shfl_xor_sync(0xffffffffu, t.x, o);
    t.y += __shfl_xor_sync(0xffffffffu, t.y, o);
  }
  if ((tr & 31) == 0) part[rb][tr >> 5] = t;
  __syncthreads();
  if (tr == 0 && row < n) {
    V s = part[rb][0];
#pragma unroll
    for (int w = 1; w < WPR; ++w) s = s + part[rb][w];
    u[row] = s;
  }
}

// u[i][r] = sum_j Ainv[i][j] f[j][r] for R >= 8 right-hand sides (a plain
// complex GEMM): 256 threads per block, each computing rows i0, i0+1 of one
// RHS; a block covers TM = 512/R <= 64 rows x all R right-hand sides.  K is
// walked in chunks (32 complex floats / 16 complex doubles): the chunk of the
// block's Ainv rows and of f are staged in shared memory (the next one already
// loading into registers), then every thread does two complex FMAs per staged
// column, in a fixed order.
template <typename T>
__global__ void __launch_bounds__(256) k_dense_gemm_rhs(int n, int R, const c_t<T>* __restrict__ A,
                                                        const c_t<T>* __restrict__ f, c_t<T>* __restrict__ u,
                                                        const int* active) {
  pdl_enter();
  if (active && !*active) return;
  using V = c_t<T>;
  constexpr int KC = sizeof(T) == 4 ? 32 : 16;
  constexpr int PA = 2 * KC / 8, PF = KC * 64 / 256;   // staged values per thread at most (R >= 8)
  __shared__ V As[64][KC + 1];
  __shared__ V Fs[KC * 64];
  const int TM = 512 / R;
  const int tid = threadIdx.x;
  const int rhs = tid & (R - 1), rg = tid / R;
  const int row0 = blockIdx.x * TM;
  const int i0 = row0 + 2 * rg, i1 = i0 + 1;
  const int na = TM * KC, nf = KC * R;                 // staged values per chunk
  V ra[PA], rf[PF];
  // the next chunk is read into registers while the current one is multiplied
  auto fetch = [&](int k0) {
    const int kc = min(KC, n - k0);
#pragma unroll
    for (int t = 0; t < PA; ++t) {
      const int e = tid + t * 256;
      if (e < na) {
        const int r = e / KC, k = e - r * KC;
        ra[t] = (row0 + r < n && k < kc) ? A[(long long)(row0 + r) * n + k0 + k] : cmk<V>(0, 0);
      }
    }
#pragma unroll
    for (int t = 0; t < PF; ++t) {
      const int e = tid + t * 256;
      if (e < nf) rf[t] = (e / R < kc) ? f[(long long)k0 * R + e] : cmk<V>(0, 0);
    }
  };
  V acc0 = cmk<V>(0, 0), acc1 = cmk<V>(0, 0);
  fetch(0);
  for (int k0 = 0; k0 < n; k0 += KC) {
    __syncthreads();
#pragma unroll
    for (int t = 0; t < PA; ++t) {
      const int e = tid + t * 256;
      if (e < na) As[e / KC][e % KC] = ra[t];
    }
#pragma unroll
    for (int t = 0; t < PF; ++t) {
      const int e = tid + t * 256;
      if (e < nf) Fs[e] = rf[t];
    }
    __syncthreads();
    if (k0 + KC < n) fetch(k0 + KC);
#pragma unroll 8
    for (int k = 0; k < KC; ++k) {
      const V fv = Fs[k * R + rhs];
      acc0 = cfma(As[2 * rg][k], fv, acc0);
      acc1 = cfma(As[2 * rg + 1][k], fv, acc1);
    }
  }
  if (i0 < n) u[(long long)i0 * R + rhs] = acc0;
  if (i1 < n) u[(long long)i1 * R + rhs] = acc1;
}

// the same product for R = 2 or 4: one block per row, one thread per RHS
template <typename T>
__global__ void k_dense_gemm_rhs_small(int n, int R, const c_t<T>* __restrict__ A, const c_t<T>* __restrict__ f,
                                       c_t<T>* __restrict__ u, const int* active) {
  pdl_enter();
  if (active && !*active) return;
  const int i = blockIdx.x, r = threadIdx.x;
  if (r >= R) return;
  c_t<T> acc = cmk<c_t<T>>(0, 0);
  const c_t<T>* row = A + (long long)i * n;
  for (int j = 0; j < n; ++j) acc = cfma(row[j], f[(long long)j * R + r], acc);
  u[(long long)i * R + r] = acc;
}

// ------------------------------------------------------------------ dispatch
template <typename F>
void with_dim_ak(int dim, int ak, F&& f) {
#define HZ_DA(D, K) \
  if (dim == D && ak == K) return f(std::integral_constant<int, D>{}, std::integral_constant<int, K>{});
  HZ_DA(2, 0) HZ_DA(2, 1) HZ_DA(2, 2) HZ_DA(2, 3) HZ_DA(3, 0) HZ_DA(3, 1) HZ_DA(3, 2)
  HZ_DA(2, 11) HZ_DA(2, 12) HZ_DA(3, 11)
#undef HZ_DA
  throw Error(HZ_ERR_INVALID_ARG, "unsupported stencil radius");
}

inline int akind(const Level& L) { return L.fine ? 0 : (L.a_half ? 10 : 0) + L.A.off.rho; }

// dimension and stored form of a level's smoother (symmetric half or M itself)
template <typename F>
void dispatch_dim_sym(const Level& L, F&& f) {
  using I2 = std::integral_constant<int, 2>;
  using I3 = std::integral_constant<int, 3>;
  using ST = std::integral_constant<bool, true>;
  using SF = std::integral_constant<bool, false>;
  const bool sym = L.wcw != nullptr;
  if (L.g.dim == 2) sym ? f(I2{}, ST{}) : f(I2{}, SF{});
  else sym ? f(I3{}, ST{}) : f(I3{}, SF{});
}

// RHS pack width for nrhs right-hand sides: 32 bytes per thread once there
// are enough of them, else one value
template <typename T, typename F>
void with_vr(int nrhs, F&& f) {
  if (vr_for(nrhs, kVRMax<T>) == kVRMax<T>) f(std::integral_constant<int, kVRMax<T>>{});
  else f(std::integral_constant<int, 1>{});
}

// Register budget of a launch (the MB template argument: minimum resident
// blocks per SM in the launch bounds).  MB = 0 leaves ptxas its default
// target of full occupancy (32 registers a thread), which suits the
// bandwidth-bound large levels: many warps hide the latency.  On a small level
// (one right-hand side, at most kIlpNodes nodes: a few blocks per SM at most)
// occupancy cannot hide it, and with 32 registers the stencil loads go out in
// small dependent batches (measured on a 65^2 level: ~9 us per launch in L2
// round trips); MB = 2 allows up to 128 registers, so every coefficient and
// neighbour load of a node is issued before the first use.
constexpr long long kIlpNodes = 20000;
// the two-blocks-per-SM register budget for a one-RHS kernel of level L
inline bool ilp_level(const Level& L) { return L.tune_mb >= 0 ? L.tune_mb == 2 : L.g.N <= kIlpNodes; }

template <typename T, typename F>
void with_vr_mb(const Level& L, int nrhs, long long nodes, F&& f) {
  // RHS pack: the level's autotuned choice (hz_autotune), else packs of 32
  // bytes per thread once there are enough right-hand sides
  const bool pack = L.tune_vr > 0 ? (L.tune_vr == 2 && vr_for(nrhs, kVRMax<T>) == kVRMax<T>)
                                  : vr_for(nrhs, kVRMax<T>) == kVRMax<T>;
  // register budget (one right-hand side): the autotuned choice, else by size
  const bool ilp = nrhs == 1 && (L.tune_mb >= 0 ? L.tune_mb == 2 : nodes <= kIlpNodes);
  if (pack) f(std::integral_constant<int, kVRMax<T>>{}, std::integral_constant<int, 0>{});
  else if (ilp) f(std::integral_constant<int, 1>{}, std::integral_constant<int, 2>{});
  else f(std::integral_constant<int, 1>{}, std::integral_constant<int, 0>{});
}

template <typename T>
void resid(Ctx& c, int l, const void* u, const void* f, void* r, const int* active, cudaStream_t s) {
  Level& L = c.L[l];
  const T invh2 = (T)(1.0 / (c.h * c.h));
  with_vr_mb<T>(L, c.nrhs, L.g.N, [&](auto V, auto MBc) {
    constexpr int VR = decltype(V)::value;
    constexpr int MB = decltype(MBc)::value;
    const Geo g = geo(L.g, c.nrhs, VR);
    with_dim_ak(L.g.dim, akind(L), [&](auto D, auto K) {
      launch_pdl(k_resid<T, D, K, VR, MB>, grid_of(g), dim3(BX, BY), s, g, invh2, (const c_t<T>*)L.Aw, (const c_t<T>*)u,
                                                               (const c_t<T>*)f, (c_t<T>*)r, active);
    });
  });
  HZ_LAUNCHED();
}

template <typename T>
void sweep_out(Ctx& c, int l, const void* r, const void* in, void* out, const int* active, cudaStream_t s) {
  Level& L = c.L[l];
  with_vr_mb<T>(L, c.nrhs, L.g.N, [&](auto V, auto MBc) {
    constexpr int VR = decltype(V)::value;
    constexpr int MB = decltype(MBc)::value;
    const Geo g = geo(L.g, c.nrhs, VR);
    auto go = [&](auto D, auto S) {
      constexpr int DIM = decltype(D)::value;
      if constexpr (decltype(S)::value)
        launch_pdl(k_sweep_out_sym<T, DIM, VR, MB>, grid_of(g), dim3(BX, BY), s, g, slist(L, c.nrhs),
                   (const c_t<T>*)L.Mhw, (const T*)L.wcw, (T)L.damping, (const c_t<T>*)r, (const c_t<T>*)in,
                   (c_t<T>*)out, active);
      else
        launch_pdl(k_sweep_out<T, DIM, VR, MB>, grid_of(g), dim3(BX, BY), s, g, mlist(L, c.nrhs),
                   (const c_t<T>*)L.Mhw, (T)L.damping, (const c_t<T>*)r, (const c_t<T>*)in, (c_t<T>*)out, active);
    };
    dispatch_dim_sym(L, go);
  });
  HZ_LAUNCHED();
}

template <typename T>
void sweep0(Ctx& c, int l, const void* f, void* u, const int* active, cudaStream_t s) {
  Level& L = c.L[l];
  with_vr_mb<T>(L, c.nrhs, L.g.N, [&](auto V, auto MBc) {
    constexpr int VR = decltype(V)::value;
    constexpr int MB = decltype(MBc)::value;
    const Geo g = geo(L.g, c.nrhs, VR);
    auto go = [&](auto D, auto S) {
      constexpr int DIM = decltype(D)::value;
      if constexpr (decltype(S)::value)
        launch_pdl(k_sweep0_sym<T, DIM, VR, MB>, grid_of(g), dim3(BX, BY), s, g, slist(L, c.nrhs),
                   (const c_t<T>*)L.Mhw, (const T*)L.wcw, (T)L.damping, (const c_t<T>*)f, (c_t<T>*)u, active);
      else
        launch_pdl(k_sweep0<T, DIM, VR, MB>, grid_of(g), dim3(BX, BY), s, g, mlist(L, c.nrhs), (const c_t<T>*)L.Mhw,
                   (T)L.damping, (const c_t<T>*)f, (c_t<T>*)u, active);
    };
    dispatch_dim_sym(L, go);
  });
  HZ_LAUNCHED();
}

template <typename T>
void sweep0_resid_diag(Ctx& c, int l, const void* f, void* u, void* r, const int* active, cudaStream_t s) {
  Level& L = c.L[l];
  const T invh2 = (T)(1.0 / (c.h * c.h));
  with_vr_mb<T>(L, c.nrhs, L.g.N, [&](auto V, auto MBc) {
    constexpr int VR = decltype(V)::value;
    constexpr int MB = decltype(MBc)::value;
    const Geo g = geo(L.g, c.nrhs, VR);
    with_dim_ak(L.g.dim, akind(L), [&](auto D, auto K) {
      launch_pdl(k_sweep0_resid_diag<T, D, K, VR, MB>, grid_of(g), dim3(BX, BY), s, g, invh2, (const c_t<T>*)L.Aw, (const c_t<T>*)L.Mw, (T)L.damping, (const c_t<T>*)f, (c_t<T>*)u,
          (c_t<T>*)r, active);
    });
  });
  HZ_LAUNCHED();
}

template <typename T>
void resid_sweep_diag(Ctx& c, int l, const void* f, const void* in, void* out, const int* active, cudaStream_t s) {
  Level& L = c.L[l];
  const T invh2 = (T)(1.0 / (c.h * c.h));
  with_vr_mb<T>(L, c.nrhs, L.g.N, [&](auto V, auto MBc) {
    constexpr int VR = decltype(V)::value;
    constexpr int MB = decltype(MBc)::value;
    const Geo g = geo(L.g, c.nrhs, VR);
    with_dim_ak(L.g.dim, akind(L), [&](auto D, auto K) {
      launch_pdl(k_resid_sweep_diag<T, D, K, VR, MB>, grid_of(g), dim3(BX, BY), s, g, invh2, (const c_t<T>*)L.Aw, (const c_t<T>*)L.Mw, (T)L.damping, (const c_t<T>*)f, (const c_t<T>*)in,
          (c_t<T>*)out, active);
    });
  });
  HZ_LAUNCHED();
}

template <typename T>
void restrict_t(Ctx& c, int l, const void* r, void* fc, const int* active, cudaStream_t s) {
  Level& L = c.L[l];
  Level& C = c.L[l + 1];
  with_vr_mb<T>(L, c.nrhs, C.g.N, [&](auto V, auto MBc) {
    constexpr int VR = decltype(V)::value;
    constexpr int MB = decltype(MBc)::value;
    const Geo gf = geo(L.g, c.nrhs, VR), gc = geo(C.g, c.nrhs, VR);
    auto go = [&](auto D, auto KIND) {
      launch_pdl(k_restrict<T, D, KIND, VR, MB>, grid_of(gc), dim3(BX, BY), s, gf, gc, (const c_t<T>*)r, (c_t<T>*)fc,
                                                                      active);
    };
    using I2 = std::integral_constant<int, 2>;
    using I3 = std::integral_constant<int, 3>;
    using K0 = std::integral_constant<int, 0>;
    using K1 = std::integral_constant<int, 1>;
    if (L.g.dim == 2) L.rkind ? go(I2{}, K1{}) : go(I2{}, K0{});
    else L.rkind ? go(I3{}, K1{}) : go(I3{}, K0{});
  });
  HZ_LAUNCHED();
}

template <typename T>
void prolong_t(Ctx& c, int l, const void* ec, const void* in, void* out, const int* active, cudaStream_t s) {
  Level& L = c.L[l];
  Level& C = c.L[l + 1];
  with_vr_mb<T>(L, c.nrhs, L.g.N, [&](auto V, auto MBc) {
    constexpr int VR = decltype(V)::value;
    constexpr int MB = decltype(MBc)::value;
    const Geo gf = geo(L.g, c.nrhs, VR), gc = geo(C.g, c.nrhs, VR);
    auto go = [&](auto D, auto KIND) {
      launch_pdl(k_prolong<T, D, KIND, VR, MB>, grid_of(gf), dim3(BX, BY), s, gf, gc, (const c_t<T>*)ec, (const c_t<T>*)in,
                                                                     (c_t<T>*)out, active);
    };
    using I2 = std::integral_constant<int, 2>;
    using I3 = std::integral_constant<int, 3>;
    using K0 = std::integral_constant<int, 0>;
    using K1 = std::integral_constant<int, 1>;
    if (L.g.dim == 2) L.pkind ? go(I2{}, K1{}) : go(I2{}, K0{});
    else L.pkind ? go(I3{}, K1{}) : go(I3{}, K0{});
  });
  HZ_LAUNCHED();
}

// 2D fused prolongation + residual (DIAG: + diagonal sweep)
template <typename T, bool DIAG>
void prolong_fused_2d(Ctx& c, int l, const void* ec, const void* t, const void* f, void* out, void* r,
                      const int* active, cudaStream_t s) {
  Level& L = c.L[l];
  Level& C = c.L[l + 1];
  require(c.nrhs == 1, "fused tile kernels take one right-hand side");
  const Geo gf = geo(L.g), gc = geo(C.g);
  const T invh2 = (T)(1.0 / (c.h * c.h));
  auto go = [&](auto K, auto KIND) {
    auto launch = [&](auto MBc) {
      launch_pdl(k_prolong_fused_2d<T, K, KIND, DIAG, decltype(MBc)::value>, grid_of(gf), dim3(BX, BY), s, gf, gc,
                 invh2, (const c_t<T>*)L.Aw, (const c_t<T>*)ec, (const c_t<T>*)t, (const c_t<T>*)f,
                 (const c_t<T>*)L.Mw, (T)L.damping, (c_t<T>*)out, (c_t<T>*)r, active);
    };
    if (ilp_level(L)) launch(std::integral_constant<int, 2>{});
    else launch(std::integral_constant<int, 0>{});
  };
  using K0 = std::integral_constant<int, 0>;
  using K1 = std::integral_constant<int, 1>;
  auto kind = [&](auto K) { L.pkind ? go(K, K1{}) : go(K, K0{}); };
  switch (akind(L)) {
    case 0: kind(std::integral_constant<int, 0>{}); break;
    case 1: kind(std::integral_constant<int, 1>{}); break;
    case 2: kind(std::integral_constant<int, 2>{}); break;
    case 3: kind(std::integral_constant<int, 3>{}); break;
    case 11: kind(std::integral_constant<int, 11>{}); break;
    case 12: kind(std::integral_constant<int, 12>{}); break;
    default: throw Error(HZ_ERR_INVALID_ARG, "unsupported stencil radius");
  }
  HZ_LAUNCHED();
}

template <typename T>
void fine_down_diag(Ctx& c, const void* f, void* fc, const int* active, cudaStream_t s) {
  Level& L = c.L[0];
  Level& C = c.L[1];
  const Geo gf = geo(L.g), gc = geo(C.g);
  const T invh2 = (T)(1.0 / (c.h * c.h));
  constexpr int CY = sizeof(T) == 4 ? 8 : 4;
  const dim3 grid(nblk(gc.nx, 32), nblk(gc.ny, CY));
  auto go = [&](auto RK, auto MBc) {
    launch_pdl(k_fine_down_diag_2d<T, decltype(RK)::value, decltype(MBc)::value>, grid, dim3(BX, BY), s, gf, gc,
               invh2, (const c_t<T>*)L.Aw, (const c_t<T>*)L.Mw, (T)L.damping, (const c_t<T>*)f, (c_t<T>*)fc, active);
  };
  auto mb = [&](auto RK) {
    if (ilp_level(L)) go(RK, std::integral_constant<int, 2>{});
    else go(RK, std::integral_constant<int, 0>{});
  };
  if (L.rkind) mb(std::integral_constant<int, 1>{});
  else mb(std::integral_constant<int, 0>{});
  HZ_LAUNCHED();
}

template <typename T>
void fine_up_diag(Ctx& c, const void* ec, const void* f, void* out, const int* active, cudaStream_t s) {
  Level& L = c.L[0];
  Level& C = c.L[1];
  const Geo gf = geo(L.g), gc = geo(C.g);
  const T invh2 = (T)(1.0 / (c.h * c.h));
  constexpr int FY = sizeof(T) == 4 ? 16 : 8;
  const dim3 grid(nblk(gf.nx, 64), nblk(gf.ny, FY));
  auto go = [&](auto PK, auto MBc) {
    launch_pdl(k_fine_up_diag_2d<T, decltype(PK)::value, decltype(MBc)::value>, grid, dim3(BX, BY), s, gf, gc, invh2,
               (const c_t<T>*)L.Aw, (const c_t<T>*)L.Mw, (T)L.damping, (const c_t<T>*)f, (const c_t<T>*)ec,
               (c_t<T>*)out, active);
  };
  auto mb = [&](auto PK) {
    if (ilp_level(L)) go(PK, std::integral_constant<int, 2>{});
    else go(PK, std::integral_constant<int, 0>{});
  };
  if (L.pkind) mb(std::integral_constant<int, 1>{});
  else mb(std::integral_constant<int, 0>{});
  HZ_LAUNCHED();
}

// operator kind of a coarse 2D level as a compile-time constant
template <typename F>
void with_ak_2d(int ak, F&& f) {
  switch (ak) {
    case 1: return f(std::integral_constant<int, 1>{});
    case 2: return f(std::integral_constant<int, 2>{});
    case 3: return f(std::integral_constant<int, 3>{});
    case 11: return f(std::integral_constant<int, 11>{});
    case 12: return f(std::integral_constant<int, 12>{});
    default: throw Error(HZ_ERR_INVALID_ARG, "unsupported stencil radius");
  }
}

template <typename T>
void level_down_2d(Ctx& c, int l, const void* f, void* t, void* fc, const int* active, cudaStream_t s) {
  Level& L = c.L[l];
  Level& C = c.L[l + 1];
  const Geo gf = geo(L.g), gc = geo(C.g);
  constexpr int CY = sizeof(T) == 4 ? 8 : 4;
  const dim3 grid(nblk(gc.nx, 16), nblk(gc.ny, CY));
  with_ak_2d(akind(L), [&](auto K) {
    auto go = [&](auto SYMc, auto RK, auto MBc, const auto& lst) {
      launch_pdl(k_level_down_2d<T, decltype(K)::value, decltype(SYMc)::value, decltype(RK)::value,
                                 decltype(MBc)::value, std::decay_t<decltype(lst)>>,
                 grid, dim3(kTileThreads), s, gf, gc, (const c_t<T>*)L.Aw, lst, (const c_t<T>*)L.Mhw,
                 (const T*)L.wcw, (T)L.damping, (const c_t<T>*)f, (c_t<T>*)t, (c_t<T>*)fc, active);
    };
    auto rk = [&](auto SYMc, auto MBc, const auto& lst) {
      if (L.rkind) go(SYMc, std::integral_constant<int, 1>{}, MBc, lst);
      else go(SYMc, std::integral_constant<int, 0>{}, MBc, lst);
    };
    auto mb = [&](auto SYMc, const auto& lst) { rk(SYMc, std::integral_constant<int, 0>{}, lst); };
    if (L.wcw) mb(std::true_type{}, slist(L));
    else mb(std::false_type{}, mlist(L));
  });
  HZ_LAUNCHED();
}

template <typename T>
void level_up_2d(Ctx& c, int l, const void* ec, const void* t, const void* f, void* out, const int* active,
                 cudaStream_t s) {
  Level& L = c.L[l];
  Level& C = c.L[l + 1];
  const Geo gf = geo(L.g), gc = geo(C.g);
  constexpr int OY = sizeof(T) == 4 ? 16 : 8;
  const dim3 grid(nblk(gf.nx, 32), nblk(gf.ny, OY));
  with_ak_2d(akind(L), [&](auto K) {
    auto go = [&](auto SYMc, auto PK, auto MBc, const auto& lst) {
      launch_pdl(k_level_up_2d<T, decltype(K)::value, decltype(SYMc)::value, decltype(PK)::value,
                               decltype(MBc)::value, std::decay_t<decltype(lst)>>,
                 grid, dim3(kTileThreads), s, gf, gc, (const c_t<T>*)L.Aw, lst, (const c_t<T>*)L.Mhw,
                 (const T*)L.wcw, (T)L.damping, (const c_t<T>*)f, (const c_t<T>*)t, (const c_t<T>*)ec,
                 (c_t<T>*)out, active);
    };
    auto pk = [&](auto SYMc, auto MBc, const auto& lst) {
      if (L.pkind) go(SYMc, std::integral_constant<int, 1>{}, MBc, lst);
      else go(SYMc, std::integral_constant<int, 0>{}, MBc, lst);
    };
    auto mb = [&](auto SYMc, const auto& lst) { pk(SYMc, std::integral_constant<int, 0>{}, lst); };
    if (L.wcw) mb(std::true_type{}, slist(L));
    else mb(std::false_type{}, mlist(L));
  });
  HZ_LAUNCHED();
}

template <typename T>
void coarse_t(Ctx& c, const void* f, void* u, const int* active, cudaStream_t s) {
  Level& L = c.L.back();
  const int n = (int)L.g.N;
  if (c.nrhs == 1) {
    if (n <= 512)
      launch_pdl(k_dense_gemv<T, 32>, nblk(n, 8), 256, s, n, (const c_t<T>*)L.Ainvw, (const c_t<T>*)f, (c_t<T>*)u,
                 active);
    else
      launch_pdl(k_dense_gemv<T, 128>, nblk(n, 2), 256, s, n, (const c_t<T>*)L.Ainvw, (const c_t<T>*)f, (c_t<T>*)u,
                 active);
  }
  else if (c.nrhs >= 16 && std::is_same<T, float>::value && coarse_variant_for(c, c.nrhs) > 0)
    coarse_gemm_tc(c, f, u, active, s, coarse_variant_for(c, c.nrhs));
  else if (c.nrhs >= 8)
    launch_pdl(k_dense_gemm_rhs<T>, nblk(n, 512 / c.nrhs), 256, s, n, c.nrhs, (const c_t<T>*)L.Ainvw, (const c_t<T>*)f,
                                                               (c_t<T>*)u, active);
  else
    launch_pdl(k_dense_gemm_rhs_small<T>, n, 32, s, n, c.nrhs, (const c_t<T>*)L.Ainvw, (const c_t<T>*)f, (c_t<T>*)u,
                                               active);
  HZ_LAUNCHED();
}

// One V(nu1, nu2) cycle at level l for A_l u = f from u = u0 (0 when u0 is
// null); result in `out`.  Step 3 of Algorithm 1 is opts.cycle_visits cycles
// on the next level (1: V-cycle, 2: W-cycle, Section 2.2).
template <typename T>
void cycle_rec(Ctx& c, int l, const void* f, const void* u0, void* out, const int* active, cudaStream_t s) {
  Level& L = c.L[l];
  if (L.coarsest) {
    coarse_t<T>(c, f, out, active, s);
    return;
  }
  if (u0 == nullptr && level_two_pass_2d(c, l)) {
    Level& C = c.L[l + 1];
    level_down_2d<T>(c, l, f, L.t, C.f, active, s);
    cycle_rec<T>(c, l + 1, C.f, nullptr, C.u, active, s);
    for (int v = 1; v < c.opts.cycle_visits && !C.coarsest; ++v) cycle_rec<T>(c, l + 1, C.f, C.u, C.u, active, s);
    level_up_2d<T>(c, l, C.u, L.t, f, out, active, s);
    return;
  }
  if (u0 == nullptr && fine_two_pass(c, l)) {
    Level& C = c.L[l + 1];
    fine_down_diag<T>(c, f, C.f, active, s);
    cycle_rec<T>(c, l + 1, C.f, nullptr, C.u, active, s);
    for (int v = 1; v < c.opts.cycle_visits && !C.coarsest; ++v) cycle_rec<T>(c, l + 1, C.f, C.u, C.u, active, s);
    fine_up_diag<T>(c, C.u, f, out, active, s);
    return;
  }
  const int nu1 = c.opts.nu1, nu2 = c.opts.nu2;
  const bool d2 = L.g.dim == 2 && c.nrhs == 1;     // shared-memory tile kernels: one RHS
  // steps 1-2: pre-relaxation into t, residual into r
  const void* rr = L.r;
  if (u0) {
    // from the initial guess u0 (the second coarse-level cycle of a W-cycle);
    // u0 may be `out`, which is written only by the post-relaxation
    if (nu1 == 0) {
      HZ_CUDA(cudaMemcpyAsync(L.t, u0, sizeof(c_t<T>) * L.g.N * c.nrhs, cudaMemcpyDeviceToDevice, s));
    } else if (L.m_diag) {
      resid_sweep_diag<T>(c, l, f, u0, L.t, active, s);
    } else {
      resid<T>(c, l, u0, f, L.r, active, s);
      sweep_out<T>(c, l, L.r, u0, L.t, active, s);
    }
    for (int i = 1; i < nu1; ++i) {
      resid<T>(c, l, L.t, f, L.r, active, s);
      sweep_out<T>(c, l, L.r, L.t, L.t, active, s);
    }
    resid<T>(c, l, L.t, f, L.r, active, s);
  } else if (nu1 == 0) {
    HZ_CUDA(cudaMemsetAsync(L.t, 0, sizeof(c_t<T>) * L.g.N * c.nrhs, s));
    rr = f;
  } else if (L.m_diag && nu1 == 1) {
    sweep0_resid_diag<T>(c, l, f, L.t, L.r, active, s);
  } else {
    sweep0<T>(c, l, f, L.t, active, s);
    for (int i = 1; i < nu1; ++i) {
      resid<T>(c, l, L.t, f, L.r, active, s);
      sweep_out<T>(c, l, L.r, L.t, L.t, active, s);
    }
    resid<T>(c, l, L.t, f, L.r, active, s);
  }
  Level& C = c.L[l + 1];
  restrict_t<T>(c, l, rr, C.f, active, s);
  cycle_rec<T>(c, l + 1, C.f, nullptr, C.u, active, s);         // step 3 (recursive)
  // W-cycle: a second coarse-level cycle from the first one's result; on the
  // coarsest level a cycle is the exact solve, so it would repeat the first
  for (int v = 1; v < c.opts.cycle_visits && !C.coarsest; ++v)
    cycle_rec<T>(c, l + 1, C.f, C.u, C.u, active, s);
  // steps 4-5: coarse-grid correction and post-relaxation into out
  if (nu2 == 0) {
    prolong_t<T>(c, l, C.u, L.t, out, active, s);
    return;
  }
  if (d2 && L.m_diag && nu2 == 1) {
    prolong_fused_2d<T, true>(c, l, C.u, L.t, f, out, nullptr, active, s);
    return;
  }
  if (d2) {
    prolong_fused_2d<T, false>(c, l, C.u, L.t, f, out, L.r, active, s);
    sweep_out<T>(c, l, L.r, out, out, active, s);
  } else {
    prolong_t<T>(c, l, C.u, L.t, L.t, active, s);
    if (L.m_diag && nu2 == 1) {
      resid_sweep_diag<T>(c, l, f, L.t, out, active, s);
      return;
    }
    resid<T>(c, l, L.t, f, L.r, active, s);
    sweep_out<T>(c, l, L.r, L.t, out, active, s);
  }
  for (int i = 1; i < nu2; ++i) {
    resid<T>(c, l, out, f, L.r, active, s);
    sweep_out<T>(c, l, L.r, out, out, active, s);
  }
}

template <typename T>
void vcycle_t(Ctx& c, int l, const void* f, void* out, const int* active, cudaStream_t s) {
  cycle_rec<T>(c, l, f, nullptr, out, active, s);
}

}  // namespace cyc
}  // namespace hz
