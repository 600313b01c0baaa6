// Hierarchy setup on the device, all arithmetic in FP64.
//
//   a1  fine coefficients: diagonal of A (Eq. 1 discretised, Section 2.1) and of
//       A_s = A + i alpha omega^2 M (Eq. shift, M the lumped mass)
//   a3  Galerkin coarse operators A_{l+1} = R_l A_l P_l (Section 3.1), one
//       thread per (coarse node, coarse offset)
//   a4  Vanka patches (Sections 3.2-3.3): for every node j and every patch i
//       containing it, H_i = V_i A_s V_i^T is inverted by Gauss-Jordan with
//       partial pivoting and row (j) of W_i H_i^{-1} is gathered into the
//       per-node stencil of M = sum_i V_i^T W_i H_i^{-1} V_i
//   a8  coarsest level: dense inverse by Gauss-Jordan with partial pivoting
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>

#include "common.cuh"

namespace hz {

// ------------------------------------------------------------------ offsets
StencilLut make_lut(const std::vector<std::array<int, 3>>& offs) {
  require(offs.size() <= HZ_MAX_STENCIL, "stencil too large");
  StencilLut s;
  std::memset(&s, 0, sizeof(s));
  s.off.n = (int)offs.size();
  s.off.rho = 0;
  for (int i = 0; i < kLutN; ++i) s.lut[i] = -1;
  for (size_t k = 0; k < offs.size(); ++k) {
    for (int a = 0; a < 3; ++a) {
      require(std::abs(offs[k][a]) <= kLutR, "stencil offset out of range");
      s.off.d[k][a] = (signed char)offs[k][a];
      s.off.rho = std::max(s.off.rho, std::abs(offs[k][a]));
    }
    s.lut[lut_index(offs[k][0], offs[k][1], offs[k][2])] = (short)k;
  }
  return s;
}

std::vector<std::array<int, 3>> fine_offsets(int dim) {
  std::vector<std::array<int, 3>> o = {{0, 0, 0}, {-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}};
  if (dim == 3) {
    o.push_back({0, 0, -1});
    o.push_back({0, 0, 1});
  }
  return o;
}

std::vector<std::array<int, 3>> box_offsets(int dim, int rho) {
  std::vector<std::array<int, 3>> o;
  int rz = dim == 3 ? rho : 0;
  for (int dz = -rz; dz <= rz; ++dz)
    for (int dy = -rho; dy <= rho; ++dy)
      for (int dx = -rho; dx <= rho; ++dx) o.push_back({dx, dy, dz});
  return o;
}

// Patch offsets about the anchor (Section 3.2).
std::vector<std::array<int, 3>> patch_offsets(int dim, hz_patch kind) {
  std::vector<std::array<int, 3>> o;
  int rz = dim == 3 ? 1 : 0;
  if (kind == HZ_PATCH_ELEMENT) {
    for (int dz = 0; dz <= rz; ++dz)
      for (int dy = 0; dy <= 1; ++dy)
        for (int dx = 0; dx <= 1; ++dx) o.push_back({dx, dy, dz});
    return o;
  }
  for (int dz = -rz; dz <= rz; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int m = std::abs(dx) + std::abs(dy) + std::abs(dz);
        bool take = false;
        switch (kind) {
          case HZ_PATCH_JACOBI: take = m == 0; break;
          case HZ_PATCH_PLUS: take = m <= 1; break;
          case HZ_PATCH_RB: take = (m % 2) == 0; break;
          case HZ_PATCH_FULL: take = true; break;
          default: break;
        }
        if (take) o.push_back({dx, dy, dz});
      }
  return o;
}

// All differences d_l - d_k of a patch's offsets: the entries of the assembled
// Vanka sum at one node, in z-y-x lexicographic order.
std::vector<std::array<int, 3>> patch_difference_offsets(int dim, hz_patch kind) {
  auto p = patch_offsets(dim, kind);
  std::map<std::array<int, 3>, int> seen;
  for (auto& a : p)
    for (auto& b : p) seen[{b[2] - a[2], b[1] - a[1], b[0] - a[0]}] = 1;
  std::vector<std::array<int, 3>> o;
  for (auto& kv : seen) o.push_back({kv.first[2], kv.first[1], kv.first[0]});
  return o;
}

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ void node_coords(const GridDev& g, long long p, int& x, int& y, int& z) {
  x = (int)(p % g.nx);
  long long t = p / g.nx;
  y = (int)(t % g.ny);
  z = (int)(t / g.ny);
}
__device__ __forceinline__ bool in_grid(const GridDev& g, int x, int y, int z) {
  return x >= 0 && x < g.nx && y >= 0 && y < g.ny && z >= 0 && z < g.nz;
}
__device__ __forceinline__ long long flat(const GridDev& g, int x, int y, int z) {
  return ((long long)z * g.ny + y) * g.nx + x;
}

// ------------------------------------------------------------------ a1
// diagA: unshifted diagonal of A (Laplacian diagonal part included);
// planes: the fine A_s as 2d+1 planes (setup only); wmass = prod_a w_a.
__global__ void k_fine_coeffs(GridDev g, double h, double omega, double alpha,
                              const double* __restrict__ kappa, const double* __restrict__ gamma,
                              double gamma0, double2* __restrict__ diagA, double* __restrict__ wmass,
                              StencilOff off, double2* __restrict__ planes) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.N) return;
  int x, y, z;
  node_coords(g, p, x, y, z);
  const double wx = wgt(x, g.nx), wy = wgt(y, g.ny);
  const double wz = g.dim == 3 ? wgt(z, g.nz) : 1.0;
  const double bx = (x == 0 || x == g.nx - 1) ? 1.0 : 0.0;
  const double by = (y == 0 || y == g.ny - 1) ? 1.0 : 0.0;
  const double bz = (g.dim == 3 && (z == 0 || z == g.nz - 1)) ? 1.0 : 0.0;
  const double W = wx * wy * wz;
  const double ox = wy * wz, oy = wx * wz, oz = wx * wy;      // weights of the other axes
  const double invh2 = 1.0 / (h * h);
  double lapd = ox * ((x > 0) + (x < g.nx - 1)) + oy * ((y > 0) + (y < g.ny - 1));
  if (g.dim == 3) lapd += oz * ((z > 0) + (z < g.nz - 1));
  const double kap = kappa[p];
  const double gam = gamma ? gamma[p] : gamma0;
  // c = -omega^2 kappa^2 (1 - i gamma/omega)
  const double cre = -omega * omega * kap * kap;
  const double cim = omega * kap * kap * gam;
  const double abc = bx * ox + by * oy + bz * oz;
  double2 d = make_double2(lapd * invh2 + W * cre, W * cim + (omega * kap / h) * abc);
  diagA[p] = d;
  wmass[p] = W;
  double2 ds = make_double2(d.x, d.y + alpha * omega * omega * W);
  for (int s = 0; s < off.n; ++s) {
    int dx = off.d[s][0], dy = off.d[s][1], dz = off.d[s][2];
    double2 v = make_double2(0.0, 0.0);
    if (dx == 0 && dy == 0 && dz == 0) {
      v = ds;
    } else if (in_grid(g, x + dx, y + dy, z + dz)) {
      double o = dx ? ox : (dy ? oy : oz);
      v = make_double2(-o * invh2, 0.0);
    }
    planes[(long long)s * g.N + p] = v;
  }
}

// compact fine operator (Eqs. disc4thCompact, disc4thCompact3D): sigma per
// node (the FGMRES operator's coefficient) and the planes of the shifted
// operator over the radius-1 box, A_s(p, q) = L(q-p)/h^2 - M(q-p) (s_p + s_q)/2
// with s = sigma - i alpha omega^2, zero where q leaves the grid
__global__ void k_fine_coeffs_compact(GridDev g, double h, double omega, double alpha,
                                      const double* __restrict__ kappa, const double* __restrict__ gamma,
                                      double gamma0, double2* __restrict__ sig, double* __restrict__ wmass,
                                      StencilOff off, double2* __restrict__ planes) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.N) return;
  int x, y, z;
  node_coords(g, p, x, y, z);
  auto sigma_at = [&](long long q) {
    const double kap = kappa[q], gam = gamma ? gamma[q] : gamma0;
    return make_double2(omega * omega * kap * kap, -omega * kap * kap * gam);
  };
  const double2 sp = sigma_at(p);
  sig[p] = sp;
  wmass[p] = 1.0;
  const double invh2 = 1.0 / (h * h), shift = alpha * omega * omega;
  for (int s = 0; s < off.n; ++s) {
    const int dx = off.d[s][0], dy = off.d[s][1], dz = off.d[s][2];
    double2 v = make_double2(0.0, 0.0);
    if (in_grid(g, x + dx, y + dy, z + dz)) {
      const int m = (dx != 0) + (dy != 0) + (dz != 0);
      const double2 sq = sigma_at(flat(g, x + dx, y + dy, z + dz));
      const double cm = compact_M(g.dim, m);
      // (s_p + s_q)/2 with s = sigma - i alpha omega^2
      const double2 savg = make_double2(0.5 * (sp.x + sq.x), 0.5 * (sp.y + sq.y) - shift);
      v = make_double2(compact_L(g.dim, m) * invh2 - cm * savg.x, -cm * savg.y);
    }
    planes[(long long)s * g.N + p] = v;
  }
}

// ------------------------------------------------------------------ a3
// Ac(I, I+D) = sum_i R(I,i) sum_s Af(i, off_s) P(i + off_s, I + D)
__global__ void k_galerkin(GridDev gf, StencilOff sf, const double2* __restrict__ Af, GridDev gc,
                           StencilOff sc, double2* __restrict__ Ac, int rk, int pk) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= gc.N * sc.n) return;
  const int e = (int)(t / gc.N);
  const long long I = t - (long long)e * gc.N;
  int X, Y, Z;
  node_coords(gc, I, X, Y, Z);
  const int JX = X + sc.d[e][0], JY = Y + sc.d[e][1], JZ = Z + sc.d[e][2];
  double2 acc = make_double2(0.0, 0.0);
  if (in_grid(gc, JX, JY, JZ)) {
    const int rr = transfer_radius(rk), rp = transfer_radius(pk);
    const int rz = gf.dim == 3 ? rr : 0;
    for (int iz = 2 * Z - rz; iz <= 2 * Z + rz; ++iz) {
      if (iz < 0 || iz >= gf.nz) continue;
      const double wz = gf.dim == 3 ? r1(rk, gf.nz, gc.nz, Z, iz) : 1.0;
      if (wz == 0.0) continue;
      for (int iy = 2 * Y - rr; iy <= 2 * Y + rr; ++iy) {
        if (iy < 0 || iy >= gf.ny) continue;
        const double wy = r1(rk, gf.ny, gc.ny, Y, iy);
        if (wy == 0.0) continue;
        for (int ix = 2 * X - rr; ix <= 2 * X + rr; ++ix) {
          if (ix < 0 || ix >= gf.nx) continue;
          const double wx = r1(rk, gf.nx, gc.nx, X, ix);
          if (wx == 0.0) continue;
          const double wr = wx * wy * wz;
          const long long i = flat(gf, ix, iy, iz);
          for (int s = 0; s < sf.n; ++s) {
            const int jx = ix + sf.d[s][0], jy = iy + sf.d[s][1], jz = iz + sf.d[s][2];
            if (!in_grid(gf, jx, jy, jz)) continue;
            if (abs(jx - 2 * JX) > rp + 1 || abs(jy - 2 * JY) > rp + 1 || abs(jz - 2 * JZ) > rp + 1) continue;
            double pw = p1(pk, gf.nx, gc.nx, jx, JX) * p1(pk, gf.ny, gc.ny, jy, JY);
            if (gf.dim == 3) pw *= p1(pk, gf.nz, gc.nz, jz, JZ);
            if (pw == 0.0) continue;
            const double2 a = Af[(long long)s * gf.N + i];
            acc.x += wr * pw * a.x;
            acc.y += wr * pw * a.y;
          }
        }
      }
    }
  }
  Ac[(long long)e * gc.N + I] = acc;
}

// ------------------------------------------------------------------ a4
struct PatchDesc {
  int np;
  int element;                 // 1: anchors are cells (never clipped)
  signed char d[27][3];
};

// In-place Gauss-Jordan inversion with partial (row) pivoting of an m x m
// complex matrix stored row-major with leading dimension ld; the column
// interchanges that undo the row pivoting are applied at the end.  Returns
// false for an exactly singular pivot.
__host__ __device__ inline bool gj_invert(double2* H, int m, int ld, int* piv) {
  for (int k = 0; k < m; ++k) {
    int p = k;
    double best = cabs2(H[k * ld + k]);
    for (int i = k + 1; i < m; ++i) {
      double v = cabs2(H[i * ld + k]);
      if (v > best) {
        best = v;
        p = i;
      }
    }
    piv[k] = p;
    if (best == 0.0) return false;
    if (p != k)
      for (int c = 0; c < m; ++c) {
        double2 t = H[k * ld + c];
        H[k * ld + c] = H[p * ld + c];
        H[p * ld + c] = t;
      }
    const double2 inv = cdiv(make_double2(1.0, 0.0), H[k * ld + k]);
    H[k * ld + k] = make_double2(1.0, 0.0);
    for (int c = 0; c < m; ++c) H[k * ld + c] = cmul(H[k * ld + c], inv);
    for (int i = 0; i < m; ++i) {
      if (i == k) continue;
      const double2 f = H[i * ld + k];
      if (f.x == 0.0 && f.y == 0.0) continue;
      H[i * ld + k] = make_double2(0.0, 0.0);
      for (int c = 0; c < m; ++c) H[i * ld + c] = H[i * ld + c] - cmul(f, H[k * ld + c]);
    }
  }
  for (int k = m - 1; k >= 0; --k) {
    const int p = piv[k];
    if (p != k)
      for (int i = 0; i < m; ++i) {
        double2 t = H[i * ld + k];
        H[i * ld + k] = H[i * ld + p];
        H[i * ld + p] = t;
      }
  }
  return true;
}

// Anchor test of a patch: element patches are anchored at cells (never
// clipped), the others at nodes.
__device__ __forceinline__ bool anchor_ok(const GridDev& g, const PatchDesc& pd, int ax, int ay, int az) {
  if (pd.element)
    return ax >= 0 && ax < g.nx - 1 && ay >= 0 && ay < g.ny - 1 &&
           (g.dim == 2 ? az == 0 : (az >= 0 && az < g.nz - 1));
  return in_grid(g, ax, ay, az);
}

// In-grid members of the patch anchored at (ax, ay, az): slot[m] = member
// index, idx[m] = node; returns m.
template <int NP>
__device__ __forceinline__ int patch_members(const GridDev& g, const PatchDesc& pd, int ax, int ay, int az,
                                             int (&slot)[NP], long long (&idx)[NP]) {
  int m = 0;
  for (int l = 0; l < pd.np; ++l) {
    const int nx = ax + pd.d[l][0], ny = ay + pd.d[l][1], nz = az + pd.d[l][2];
    if (!in_grid(g, nx, ny, nz)) continue;
    slot[m] = l;
    idx[m] = flat(g, nx, ny, nz);
    ++m;
  }
  return m;
}

// Phase 1 of the Vanka sum (Section 3.2): the inverse of every patch matrix
// H_i (the rows / columns of A_s on the patch's in-grid nodes), once per
// patch.  Anchors are taken along the slow axis (z in 3D, y in 2D) from s0 to
// s1; Hinv[(anchor - first anchor of s0) * NP*NP + a*m + b].
template <int NP>
__global__ void k_patch_inverse(GridDev g, StencilLut A, const double2* __restrict__ Ap, PatchDesc pd, int s0,
                                int s1, double2* __restrict__ Hinv, int* __restrict__ singular) {
  const long long per = g.dim == 3 ? (long long)g.nx * g.ny : g.nx;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * (s1 - s0)) return;
  int ax, ay, az;
  if (g.dim == 3) {
    az = s0 + (int)(t / per);
    const int r = (int)(t % per);
    ay = r / g.nx;
    ax = r % g.nx;
  } else {
    az = 0;
    ay = s0 + (int)(t / per);
    ax = (int)(t % per);
  }
  if (!anchor_ok(g, pd, ax, ay, az)) return;
  int slot[NP], piv[NP];
  long long idx[NP];
  const int m = patch_members<NP>(g, pd, ax, ay, az, slot, idx);
  double2 H[NP * NP];
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) {
      const int dx = pd.d[slot[b]][0] - pd.d[slot[a]][0];
      const int dy = pd.d[slot[b]][1] - pd.d[slot[a]][1];
      const int dz = pd.d[slot[b]][2] - pd.d[slot[a]][2];
      const int e = A.lut[lut_index(dx, dy, dz)];
      H[a * m + b] = e >= 0 ? Ap[(long long)e * g.N + idx[a]] : make_double2(0.0, 0.0);
    }
  if (!gj_invert(H, m, m, piv)) {
    atomicAdd(singular, 1);
    return;
  }
  double2* out = Hinv + t * (NP * NP);
  for (int k = 0; k < m * m; ++k) out[k] = H[k];
}

// Phase 2: node j (slow-axis coordinate in [n0, n1)) adds, patch by patch in
// the order of the patch offsets, its weighted row of each H_i^{-1} (weight
// 1/count, count = patches containing j) to the planes of M at offsets
// d_l - d_k.  The patches' anchors must lie in the slab [s0, s1) of Hinv.
template <int NP>
__global__ void k_vanka_gather(GridDev g, PatchDesc pd, StencilLut Ml, const double2* __restrict__ Hinv, int s0,
                               int n0, int n1, double2* __restrict__ Mp) {
  const long long per = g.dim == 3 ? (long long)g.nx * g.ny : g.nx;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * (n1 - n0)) return;
  const long long j = (long long)n0 * per + t;
  int x, y, z;
  node_coords(g, j, x, y, z);
  int count = 0;
  for (int k = 0; k < pd.np; ++k)
    if (anchor_ok(g, pd, x - pd.d[k][0], y - pd.d[k][1], z - pd.d[k][2])) ++count;
  if (count == 0) return;
  const double W = 1.0 / count;
  int slot[NP];
  long long idx[NP];
  for (int k = 0; k < pd.np; ++k) {
    const int ax = x - pd.d[k][0], ay = y - pd.d[k][1], az = z - pd.d[k][2];
    if (!anchor_ok(g, pd, ax, ay, az)) continue;
    const int m = patch_members<NP>(g, pd, ax, ay, az, slot, idx);
    int kk = 0;
    while (slot[kk] != k) ++kk;
    const int sa = g.dim == 3 ? az : ay;
    const long long at = (long long)(sa - s0) * per + (g.dim == 3 ? (long long)ay * g.nx + ax : ax);
    const double2* Hi = Hinv + at * (NP * NP);
    for (int b = 0; b < m; ++b) {
      const int l = slot[b];
      const int e = Ml.lut[lut_index(pd.d[l][0] - pd.d[k][0], pd.d[l][1] - pd.d[k][1], pd.d[l][2] - pd.d[k][2])];
      double2* dst = Mp + (long long)e * g.N + j;
      *dst = *dst + W * Hi[kk * m + b];
    }
  }
}

// M' planes at the stored half offsets and 1/count per node: M'[s](p) =
// count_p M[s](p) (count_p = patches containing p, the inverse of the weight
// the gather applied), wc(p) = 1/count_p (0 where no patch contains p).
__global__ void k_sym_half(GridDev g, PatchDesc pd, const double2* __restrict__ M64, int nh,
                           const short* __restrict__ src, double2* __restrict__ Mh, double* __restrict__ wc) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  int x, y, z;
  node_coords(g, j, x, y, z);
  int count = 0;
  for (int k = 0; k < pd.np; ++k)
    if (anchor_ok(g, pd, x - pd.d[k][0], y - pd.d[k][1], z - pd.d[k][2])) ++count;
  wc[j] = count ? 1.0 / count : 0.0;
  for (int h = 0; h < nh; ++h) Mh[(long long)h * g.N + j] = (double)count * M64[(long long)src[h] * g.N + j];
}

// 1 in out[e] when plane e of `planes` has a non-zero entry (block-wide OR,
// one atomic per block)
__global__ void k_plane_nonzero(const double2* __restrict__ planes, long long N, unsigned long long* __restrict__ out) {
  const int e = blockIdx.y;
  const double2* pl = planes + (long long)e * N;
  int nz = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = pl[i];
    nz |= (v.x != 0.0 || v.y != 0.0);
  }
  nz = __syncthreads_or(nz);
  if (nz && threadIdx.x == 0) atomicOr(out + e, 1ull);
}

// ------------------------------------------------------------------ casts
template <typename V>
__global__ void k_cast(const double2* __restrict__ in, V* __restrict__ out, long long n) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = from_c128<V>(in[t]);
}

// ------------------------------------------------------------------ a8
__global__ void k_dense_from_planes(GridDev g, StencilOff so, const double2* __restrict__ planes,
                                    double2* __restrict__ D) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.N) return;
  int x, y, z;
  node_coords(g, p, x, y, z);
  for (int s = 0; s < so.n; ++s) {
    const int xx = x + so.d[s][0], yy = y + so.d[s][1], zz = z + so.d[s][2];
    if (!in_grid(g, xx, yy, zz)) continue;
    D[p * g.N + flat(g, xx, yy, zz)] = planes[(long long)s * g.N + p];
  }
}

// pivot search for column k (one block)
__global__ void k_gj_pivot(double2* __restrict__ D, int n, int k, int* __restrict__ piv,
                           int* __restrict__ singular) {
  __shared__ double bv[1024];
  __shared__ int bi[1024];
  double best = -1.0;
  int arg = k;
  for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
    const double v = cabs2(D[(long long)i * n + k]);
    if (v > best) {
      best = v;
      arg = i;
    }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = arg;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double o = bv[threadIdx.x + s];
      const int oi = bi[threadIdx.x + s];
      if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
        bv[threadIdx.x] = o;
        bi[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    piv[k] = bi[0];
    if (bv[0] <= 0.0) atomicAdd(singular, 1);
  }
}

// swap rows k and piv[k], scale the pivot row, save column k
__global__ void k_gj_swap_scale(double2* __restrict__ D, int n, int k, const int* __restrict__ piv,
                                double2* __restrict__ col) {
  const int p = piv[k];
  __shared__ double2 inv;
  if (threadIdx.x == 0) {
    const double2 a = D[(long long)p * n + k];
    inv = (a.x == 0.0 && a.y == 0.0) ? make_double2(0.0, 0.0) : cdiv(make_double2(1.0, 0.0), a);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    double2 rk = D[(long long)k * n + c];
    double2 rp = D[(long long)p * n + c];
    if (p != k) D[(long long)p * n + c] = rk;
    if (c == k) rp = make_double2(1.0, 0.0);
    D[(long long)k * n + c] = cmul(rp, inv);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = D[(long long)i * n + k];
}

// H[i][c] = (c == k ? 0 : H[i][c]) - col[i] * H[k][c] for all i != k
__global__ void k_gj_eliminate(double2* __restrict__ D, int n, int k, const double2* __restrict__ col) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (c >= n || i == k) return;
  const double2 f = col[i];
  if (f.x == 0.0 && f.y == 0.0) return;
  double2 v = c == k ? make_double2(0.0, 0.0) : D[(long long)i * n + c];
  D[(long long)i * n + c] = v - cmul(f, D[(long long)k * n + c]);
}

// undo the row pivoting: column swaps in reverse order, composed into one
// permutation (single thread), then a gather
__global__ void k_gj_compose(const int* __restrict__ piv, int n, int* __restrict__ perm) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int c = 0; c < n; ++c) perm[c] = c;
  for (int k = n - 1; k >= 0; --k) {
    const int p = piv[k];
    const int t = perm[k];
    perm[k] = perm[p];
    perm[p] = t;
  }
}
__global__ void k_gj_permute_cols(const double2* __restrict__ X, int n, const int* __restrict__ perm,
                                  double2* __restrict__ Y) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (c >= n) return;
  Y[(long long)i * n + c] = X[(long long)i * n + perm[c]];
}

// ------------------------------------------------------------------ host
static inline unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

static void invert_dense(Ctx& c, Level& L, cudaStream_t s) {
  const long long n = L.g.N;
  require(n <= 20000, "coarsest level too large for a dense inverse (use more levels)");
  double2* D = (double2*)ctx_alloc(c, sizeof(double2) * n * n);
  HZ_CUDA(cudaMemsetAsync(D, 0, sizeof(double2) * n * n, s));
  k_dense_from_planes<<<nblk(n, 256), 256, 0, s>>>(L.g, L.A.off, L.A64, D);
  HZ_LAUNCHED();
  double2* col = nullptr;
  int *piv = nullptr, *perm = nullptr, *sing = nullptr;
  HZ_CUDA(counted_malloc_async(&col, sizeof(double2) * n, s));
  HZ_CUDA(counted_malloc_async(&piv, sizeof(int) * n, s));
  HZ_CUDA(counted_malloc_async(&perm, sizeof(int) * n, s));
  HZ_CUDA(counted_malloc_async(&sing, sizeof(int), s));
  HZ_CUDA(cudaMemsetAsync(sing, 0, sizeof(int), s));
  for (int k = 0; k < n; ++k) {
    k_gj_pivot<<<1, 1024, 0, s>>>(D, (int)n, k, piv, sing);
    k_gj_swap_scale<<<1, 1024, 0, s>>>(D, (int)n, k, piv, col);
    dim3 gr(nblk(n, 256), (unsigned)n);
    k_gj_eliminate<<<gr, 256, 0, s>>>(D, (int)n, k, col);
  }
  HZ_LAUNCHED();
  k_gj_compose<<<1, 1, 0, s>>>(piv, (int)n, perm);
  L.Ainv64 = (double2*)ctx_alloc(c, sizeof(double2) * n * n);
  dim3 gr(nblk(n, 256), (unsigned)n);
  k_gj_permute_cols<<<gr, 256, 0, s>>>(D, (int)n, perm, L.Ainv64);
  HZ_LAUNCHED();
  int hsing = 0;
  HZ_CUDA(cudaMemcpyAsync(&hsing, sing, sizeof(int), cudaMemcpyDeviceToHost, s));
  HZ_CUDA(cudaStreamSynchronize(s));
  cudaFreeAsync(col, s);
  cudaFreeAsync(piv, s);
  cudaFreeAsync(perm, s);
  cudaFreeAsync(sing, s);
  if (hsing) throw Error(HZ_ERR_INVALID_ARG, "coarsest-level operator is singular");
}

// Both phases over slabs of the slow axis, with at most kSlabBytes of patch
// inverses alive at a time.
constexpr size_t kSlabBytes = 256u << 20;
template <int NP>
static void launch_vanka(Level& L, const PatchDesc& pd, const StencilLut& Mfull, double2* Mp, int* sing,
                         cudaStream_t s) {
  const GridDev& g = L.g;
  const int ns = g.dim == 3 ? g.nz : g.ny;                    // slow-axis extent
  const long long per = g.dim == 3 ? (long long)g.nx * g.ny : g.nx;
  const int ax = g.dim == 3 ? 2 : 1;
  int dmin = 0, dmax = 0;                                      // patch extent along the slow axis
  for (int k = 0; k < pd.np; ++k) {
    dmin = std::min(dmin, (int)pd.d[k][ax]);
    dmax = std::max(dmax, (int)pd.d[k][ax]);
  }
  const size_t per_plane = (size_t)per * NP * NP * sizeof(double2);
  const int chunk = (int)std::max<size_t>(1, kSlabBytes / per_plane);     // node planes per slab
  const int span = std::min(ns, chunk + dmax - dmin);
  double2* Hinv = nullptr;
  HZ_CUDA(counted_malloc_async(&Hinv, per_plane * span, s));
  for (int n0 = 0; n0 < ns; n0 += chunk) {
    const int n1 = std::min(ns, n0 + chunk);
    // anchors of the patches of nodes n0..n1-1: node - d
    const int s0 = std::max(0, n0 - dmax), s1 = std::min(ns, n1 - dmin);
    k_patch_inverse<NP><<<nblk(per * (s1 - s0), 128), 128, 0, s>>>(g, L.A, L.A64, pd, s0, s1, Hinv, sing);
    HZ_LAUNCHED();
    k_vanka_gather<NP><<<nblk(per * (n1 - n0), 128), 128, 0, s>>>(g, pd, Mfull, Hinv, s0, n0, n1, Mp);
    HZ_LAUNCHED();
  }
  HZ_CUDA(cudaFreeAsync(Hinv, s));
}

template <typename V>
__global__ void k_cast_real(const double* __restrict__ in, V* __restrict__ out, long long n) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = (V)in[t];
}

static void* working_copy_real(Ctx& c, const double* src, long long n, cudaStream_t s) {
  if (!c.mixed) return (void*)src;
  float* dst = (float*)ctx_alloc(c, sizeof(float) * n);
  k_cast_real<float><<<nblk(n, 256), 256, 0, s>>>(src, dst, n);
  HZ_LAUNCHED();
  return dst;
}

static void* working_copy(Ctx& c, const double2* src, long long n, cudaStream_t s) {
  if (!c.mixed) return (void*)src;             // FP64 path works on the setup arrays
  float2* dst = (float2*)ctx_alloc(c, sizeof(float2) * n);
  k_cast<float2><<<nblk(n, 256), 256, 0, s>>>(src, dst, n);
  HZ_LAUNCHED();
  return dst;
}

static void assemble_smoother(Ctx& c, Level& L, cudaStream_t s) {
  const int dim = c.grid.dim;
  auto po = patch_offsets(dim, L.patch);
  PatchDesc pd;
  std::memset(&pd, 0, sizeof(pd));
  pd.np = (int)po.size();
  pd.element = L.patch == HZ_PATCH_ELEMENT;
  for (int k = 0; k < pd.np; ++k)
    for (int a = 0; a < 3; ++a) pd.d[k][a] = (signed char)po[k][a];
  auto moffs = patch_difference_offsets(dim, L.patch);
  StencilLut Mfull = make_lut(moffs);
  const long long N = L.g.N;
  double2* Mp = nullptr;
  HZ_CUDA(counted_malloc_async(&Mp, sizeof(double2) * N * Mfull.off.n, s));
  HZ_CUDA(cudaMemsetAsync(Mp, 0, sizeof(double2) * N * Mfull.off.n, s));
  int* sing = nullptr;
  unsigned long long* amax = nullptr;
  HZ_CUDA(counted_malloc_async(&sing, sizeof(int), s));
  HZ_CUDA(cudaMemsetAsync(sing, 0, sizeof(int), s));
  HZ_CUDA(counted_malloc_async(&amax, sizeof(unsigned long long) * Mfull.off.n, s));
  HZ_CUDA(cudaMemsetAsync(amax, 0, sizeof(unsigned long long) * Mfull.off.n, s));
  switch (pd.np) {
    case 1: launch_vanka<1>(L, pd, Mfull, Mp, sing, s); break;
    case 4: launch_vanka<4>(L, pd, Mfull, Mp, sing, s); break;
    case 5: launch_vanka<5>(L, pd, Mfull, Mp, sing, s); break;
    case 7: launch_vanka<7>(L, pd, Mfull, Mp, sing, s); break;
    case 8: launch_vanka<8>(L, pd, Mfull, Mp, sing, s); break;
    case 9: launch_vanka<9>(L, pd, Mfull, Mp, sing, s); break;
    case 13: launch_vanka<13>(L, pd, Mfull, Mp, sing, s); break;
    case 27: launch_vanka<27>(L, pd, Mfull, Mp, sing, s); break;
    default: throw Error(HZ_ERR_INVALID_ARG, "unsupported patch size");
  }
  k_plane_nonzero<<<dim3((unsigned)std::min<long long>(nblk(N, 256 * 8), 1216), Mfull.off.n), 256, 0, s>>>(Mp, N, amax);
  HZ_LAUNCHED();
  std::vector<unsigned long long> hmax(Mfull.off.n);
  int hsing = 0;
  HZ_CUDA(cudaMemcpyAsync(hmax.data(), amax, sizeof(unsigned long long) * Mfull.off.n,
                          cudaMemcpyDeviceToHost, s));
  HZ_CUDA(cudaMemcpyAsync(&hsing, sing, sizeof(int), cudaMemcpyDeviceToHost, s));
  HZ_CUDA(cudaStreamSynchronize(s));
  if (hsing) {
    cudaFreeAsync(Mp, s);
    throw Error(HZ_ERR_INVALID_ARG, "a Vanka patch matrix is singular");
  }
  // drop planes that are identically zero (e.g. the RB patch on a 5-point
  // stencil, whose patch matrices are diagonal: the sum is damped Jacobi)
  std::vector<std::array<int, 3>> keep;
  std::vector<int> src;
  for (int e = 0; e < Mfull.off.n; ++e)
    if (hmax[e] != 0ull) {
      keep.push_back({Mfull.off.d[e][0], Mfull.off.d[e][1], Mfull.off.d[e][2]});
      src.push_back(e);
    }
  L.M = make_lut(keep);
  L.m_diag = keep.size() == 1 && keep[0][0] == 0 && keep[0][1] == 0 && keep[0][2] == 0;
  L.M64 = (double2*)ctx_alloc(c, sizeof(double2) * N * keep.size());
  for (size_t k = 0; k < src.size(); ++k)
    HZ_CUDA(cudaMemcpyAsync(L.M64 + (long long)k * N, Mp + (long long)src[k] * N, sizeof(double2) * N,
                            cudaMemcpyDeviceToDevice, s));
  if (!L.a_sym) {
    // operator not symmetric: the weighted planes of M as they are (working
    // copy made by the caller)
    L.Mh = L.M;
    L.wcw = nullptr;
  } else {
    // half set: s >= 0 lexicographically (z, y, x), mirrored when -s is in the set too
    std::vector<std::array<int, 3>> half;
    std::vector<short> hsrc;
    std::vector<unsigned char> mirror;
    for (size_t k = 0; k < keep.size(); ++k) {
      const auto& d = keep[k];
      const bool pos = d[2] > 0 || (d[2] == 0 && (d[1] > 0 || (d[1] == 0 && d[0] >= 0)));
      const bool has_neg = L.M.lut[lut_index(-d[0], -d[1], -d[2])] >= 0;
      const bool zero = d[0] == 0 && d[1] == 0 && d[2] == 0;
      if (pos || !has_neg) {            // a negative offset without its mirror is stored as it is
        half.push_back(d);
        hsrc.push_back((short)k);
        mirror.push_back((unsigned char)(pos && has_neg && !zero));
      }
    }
    L.Mh = make_lut(half);
    for (size_t k = 0; k < half.size(); ++k) L.mh_mirror[k] = mirror[k];
    short* dsrc = nullptr;
    HZ_CUDA(counted_malloc_async(&dsrc, sizeof(short) * hsrc.size(), s));
    HZ_CUDA(cudaMemcpyAsync(dsrc, hsrc.data(), sizeof(short) * hsrc.size(), cudaMemcpyHostToDevice, s));
    double2* Mh64 = (double2*)ctx_alloc(c, sizeof(double2) * N * half.size());
    double* wc64 = (double*)ctx_alloc(c, sizeof(double) * N);
    k_sym_half<<<nblk(N, 256), 256, 0, s>>>(L.g, pd, L.M64, (int)half.size(), dsrc, Mh64, wc64);
    HZ_LAUNCHED();
    HZ_CUDA(cudaStreamSynchronize(s));  // hsrc (host) and dsrc are released below
    HZ_CUDA(cudaFreeAsync(dsrc, s));
    L.Mhw = working_copy(c, Mh64, N * (long long)half.size(), s);
    L.wcw = working_copy_real(c, wc64, N, s);
  }
  cudaFreeAsync(Mp, s);
  cudaFreeAsync(sing, s);
  cudaFreeAsync(amax, s);
}


static int rkind_of(hz_intergrid ig, int level) {
  switch (ig) {
    case HZ_IG_LINEAR: return 0;
    case HZ_IG_CUBIC: return 1;
    case HZ_IG_MIXED: return 0;
    case HZ_IG_LEVELDEP: return level == 0 ? 1 : 0;
  }
  return 0;
}
static int pkind_of(hz_intergrid ig, int level) {
  (void)level;
  return ig == HZ_IG_LINEAR ? 0 : 1;
}

void build_hierarchy(Ctx& c, const double* kappa, const double* gamma, double gamma0, cudaStream_t s) {
  const int dim = c.grid.dim;
  const int levels = c.opts.levels;
  const size_t vb = c.mixed ? sizeof(float2) : sizeof(double2);
  const int R = std::max(1, c.opts.nrhs_max);
  c.L.assign(levels, Level());
  int n[3] = {c.grid.n[0], c.grid.n[1], dim == 3 ? c.grid.n[2] : 1};
  for (int l = 0; l < levels; ++l) {
    Level& L = c.L[l];
    L.g = make_grid(dim, n);
    L.fine = l == 0 && !c.compact;       // the compact fine level is a stored-stencil level
    L.coarsest = l == levels - 1;
    L.patch = c.opts.patch[l];
    L.damping = c.opts.damping[l];
    L.rkind = rkind_of(c.opts.intergrid, l);
    L.pkind = pkind_of(c.opts.intergrid, l);
    // A_s is complex symmetric on the fine level; R A P keeps that when R is a
    // scaled P^T (same kind of both transfers), not for linear R / cubic P
    L.a_sym = l == 0 || (c.L[l - 1].a_sym && c.L[l - 1].rkind == c.L[l - 1].pkind);
    for (int a = 0; a < dim; ++a) n[a] = (n[a] - 1) / 2 + 1;
  }
  // a1: fine coefficients
  {
    Level& L = c.L[0];
    const long long N = L.g.N;
    L.A = make_lut(c.compact ? box_offsets(dim, 1) : fine_offsets(dim));
    L.A64 = (double2*)ctx_alloc(c, sizeof(double2) * N * L.A.off.n);
    c.diagA64 = (double2*)ctx_alloc(c, sizeof(double2) * N);
    c.wmass = (double*)ctx_alloc(c, sizeof(double) * N);
    if (c.compact)
      k_fine_coeffs_compact<<<nblk(N, 256), 256, 0, s>>>(L.g, c.h, c.omega, c.alpha, kappa, gamma, gamma0,
                                                          c.diagA64, c.wmass, L.A.off, L.A64);
    else
      k_fine_coeffs<<<nblk(N, 256), 256, 0, s>>>(L.g, c.h, c.omega, c.alpha, kappa, gamma, gamma0,
                                                  c.diagA64, c.wmass, L.A.off, L.A64);
    HZ_LAUNCHED();
  }
  static const char* kLevelRange[] = {"hz setup level 0", "hz setup level 1", "hz setup level 2",
                                      "hz setup level 3", "hz setup level 4", "hz setup level 5",
                                      "hz setup level 6", "hz setup level 7", "hz setup level 8",
                                      "hz setup level 9", "hz setup level 10", "hz setup level 11"};
  for (int l = 0; l < levels; ++l) {
    Level& L = c.L[l];
    const long long N = L.g.N;
    NvtxRange range(kLevelRange[l < 12 ? l : 11]);
    if (L.coarsest) {
      invert_dense(c, L, s);
      L.Ainvw = working_copy(c, L.Ainv64, N * N, s);
    } else {
      assemble_smoother(c, L, s);
      // a3: Galerkin operator of the next level
      Level& C = c.L[l + 1];
      const int rho = (transfer_radius(L.rkind) + L.A.off.rho + transfer_radius(L.pkind)) / 2;
      C.A = make_lut(box_offsets(dim, std::min(rho, kLutR)));
      C.A64 = (double2*)ctx_alloc(c, sizeof(double2) * C.g.N * C.A.off.n);
      const long long T = C.g.N * C.A.off.n;
      k_galerkin<<<nblk(T, 128), 128, 0, s>>>(L.g, L.A.off, L.A64, C.g, C.A.off, C.A64, L.rkind, L.pkind);
      HZ_LAUNCHED();
      if (L.m_diag) L.Mw = working_copy(c, L.M64, N, s);
      if (!L.a_sym) L.Mhw = working_copy(c, L.M64, N * (long long)L.M.off.n, s);
    }
    // working operator: fine = diagonal of A_s (plane 0), coarse = all planes;
    // a symmetric full box of radius 1 or 2 (2D) / 1 (3D) keeps only the
    // planes s >= 0, the second half of the box order (centre first)
    const int rho = L.A.off.rho, W = 2 * rho + 1;
    const int box = dim == 3 ? W * W * W : W * W;
    L.a_half = !L.fine && !L.coarsest && L.a_sym && L.A.off.n == box &&
               ((dim == 2 && (rho == 1 || rho == 2)) || (dim == 3 && rho == 1));
    if (L.a_half) {
      const int c0 = (box - 1) / 2;
      L.Aw = working_copy(c, L.A64 + (long long)c0 * N, N * (long long)(box - c0), s);
    } else {
      L.Aw = working_copy(c, L.A64, L.fine ? N : N * L.A.off.n, s);
    }
    L.u = ctx_alloc(c, vb * N * R);
    L.f = ctx_alloc(c, vb * N * R);
    L.r = ctx_alloc(c, vb * N * R);
    L.t = ctx_alloc(c, vb * N * R);
    require(N * (long long)std::max(L.A.off.n, L.coarsest ? 1 : L.M.off.n) < (1ll << 31),
            "level too large for 32-bit plane indexing");
  }
  HZ_CUDA(cudaStreamSynchronize(s));
}

size_t hierarchy_bytes(const hz_grid& g, const hz_opts& o) {
  const int dim = g.dim;
  const size_t vb = o.precision == HZ_PREC_MIXED ? 8 : 16;
  const int R = std::max(1, o.nrhs_max);
  long long n[3] = {g.n[0], g.n[1], dim == 3 ? g.n[2] : 1};
  size_t total = 0;
  int rho = 1;
  for (int l = 0; l < o.levels; ++l) {
    const long long N = n[0] * n[1] * n[2];
    const int sA = l == 0 ? (o.stencil == 1 ? (int)std::pow(3, dim) : 2 * dim + 1) : (int)std::pow(2 * rho + 1, dim);
    total += 16ull * N * sA;                                   // FP64 operator planes
    if (l == 0) total += 16ull * N + 8ull * N + vb * N * (o.stencil == 1 ? sA : 1);   // diag A / sigma, wmass, working operator
    else if (vb == 8) total += 8ull * N * sA;
    if (l == o.levels - 1) {
      total += 16ull * N * N * 2 + (vb == 8 ? 8ull * N * N : 0);   // dense work + inverse
    } else {
      const int sM = (int)patch_difference_offsets(dim, o.patch[l]).size();
      total += (16ull + (vb == 8 ? 8 : 0)) * N * sM;
      const int rk = rkind_of(o.intergrid, l), pk = pkind_of(o.intergrid, l);
      rho = (transfer_radius(rk) + (l == 0 ? 1 : rho) + transfer_radius(pk)) / 2;
    }
    total += 3ull * vb * N * R;
    for (int a = 0; a < dim; ++a) n[a] = (n[a] - 1) / 2 + 1;
  }
  return total;
}

}  // namespace hz
