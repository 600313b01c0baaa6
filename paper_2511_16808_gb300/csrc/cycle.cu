// V-cycle kernels in the working precision T (float for the mixed path,
// double for the plain FP64 path) and the recursive driver (Algorithm 1).
//
//   residual   r = f - A_s u                       (fine: diagonal + index weights;
//                                                   coarse: stored Galerkin planes)
//   sweep      u += w M r, M the assembled Vanka sum (Eq. smoother); the first
//              sweep from u = 0 is u = w M f
//   restrict   f_c = R r   (Eqs. biliniearIntergrid / bicubicIntergrid, gather)
//   prolong    u += P e_c  (P = 2^d R^T of the same kind, gather)
//   coarse     u = A_L^{-1} f (dense inverse from setup; one warp per row)
//
// Every kernel is one thread per output node, HBM-bound; neighbour reads hit
// L1/L2 because consecutive threads are consecutive x.  Kernels take an
// optional device flag `active`: when it reads 0 they return at once, which
// lets a captured FGMRES cycle skip the iterations after convergence.
#include "common.cuh"

namespace hz {

namespace {

constexpr int kBlock = 256;

inline unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

__device__ __forceinline__ void coords(const GridDev& g, long long p, int& x, int& y, int& z) {
  x = (int)(p % g.nx);
  long long t = p / g.nx;
  y = (int)(t % g.ny);
  z = (int)(t / g.ny);
}

// (A u)_p on the fine level: diag_p u_p - sum_a W_other(a)/h^2 * sum_{q = p +- e_a} u_q
template <typename T, typename U>
__device__ __forceinline__ c_t<T> fine_apply_at(const GridDev& g, T invh2, c_t<T> diag, const U* __restrict__ u,
                                                long long p, int x, int y, int z) {
  using V = c_t<T>;
  const T wx = (T)wgt(x, g.nx), wy = (T)wgt(y, g.ny);
  const T wz = g.dim == 3 ? (T)wgt(z, g.nz) : (T)1;
  auto ld = [&](long long q) -> V {
    const U v = u[q];
    V o;
    o.x = (T)v.x;
    o.y = (T)v.y;
    return o;
  };
  V acc = cmul(diag, ld(p));
  V sx = cmk<V>(0, 0), sy = cmk<V>(0, 0), sz = cmk<V>(0, 0);
  if (x > 0) sx = sx + ld(p - 1);
  if (x < g.nx - 1) sx = sx + ld(p + 1);
  if (y > 0) sy = sy + ld(p - g.nx);
  if (y < g.ny - 1) sy = sy + ld(p + g.nx);
  const T cx = wy * wz * invh2, cy = wx * wz * invh2;
  acc.x -= cx * sx.x + cy * sy.x;
  acc.y -= cx * sx.y + cy * sy.y;
  if (g.dim == 3) {
    const long long pl = (long long)g.nx * g.ny;
    if (z > 0) sz = sz + ld(p - pl);
    if (z < g.nz - 1) sz = sz + ld(p + pl);
    const T cz = wx * wy * invh2;
    acc.x -= cz * sz.x;
    acc.y -= cz * sz.y;
  }
  return acc;
}

template <typename T>
__global__ void k_fine_residual(GridDev g, T invh2, const c_t<T>* __restrict__ diag, const c_t<T>* __restrict__ u,
                                const c_t<T>* __restrict__ f, c_t<T>* __restrict__ r, const int* active) {
  if (active && !*active) return;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.N) return;
  int x, y, z;
  coords(g, p, x, y, z);
  const c_t<T> a = fine_apply_at<T>(g, invh2, diag[p], u, p, x, y, z);
  r[p] = f[p] - a;
}

// FP64 operator apply on the fine level, input in float2 or double2.
template <typename U>
__global__ void k_fine_apply64(GridDev g, double invh2, const double2* __restrict__ diag, const U* __restrict__ v,
                               double2* __restrict__ w) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.N) return;
  int x, y, z;
  coords(g, p, x, y, z);
  w[p] = fine_apply_at<double>(g, invh2, diag[p], v, p, x, y, z);
}

template <typename T>
__device__ __forceinline__ c_t<T> stencil_at(const GridDev& g, const StencilOff& so, const c_t<T>* __restrict__ planes,
                                             const c_t<T>* __restrict__ u, long long p, int x, int y, int z) {
  c_t<T> acc = cmk<c_t<T>>(0, 0);
  const long long pl = (long long)g.nx * g.ny;
  for (int s = 0; s < so.n; ++s) {
    const int dx = so.d[s][0], dy = so.d[s][1], dz = so.d[s][2];
    const int xx = x + dx, yy = y + dy, zz = z + dz;
    if (xx < 0 || xx >= g.nx || yy < 0 || yy >= g.ny || zz < 0 || zz >= g.nz) continue;
    acc = cfma(planes[(long long)s * g.N + p], u[p + dx + (long long)dy * g.nx + dz * pl], acc);
  }
  return acc;
}

template <typename T>
__global__ void k_stencil_residual(GridDev g, StencilOff so, const c_t<T>* __restrict__ planes,
                                   const c_t<T>* __restrict__ u, const c_t<T>* __restrict__ f,
                                   c_t<T>* __restrict__ r, const int* active) {
  if (active && !*active) return;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.N) return;
  int x, y, z;
  coords(g, p, x, y, z);
  r[p] = f[p] - stencil_at<T>(g, so, planes, u, p, x, y, z);
}

// ACCUM = 0: out = w * M in ; ACCUM = 1: out += w * M in
template <typename T, int ACCUM>
__global__ void k_vanka_apply(GridDev g, StencilOff so, const c_t<T>* __restrict__ planes, T w,
                              const c_t<T>* __restrict__ in, c_t<T>* __restrict__ out, const int* active) {
  if (active && !*active) return;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.N) return;
  int x, y, z;
  coords(g, p, x, y, z);
  c_t<T> m = stencil_at<T>(g, so, planes, in, p, x, y, z);
  m.x *= w;
  m.y *= w;
  out[p] = ACCUM ? out[p] + m : m;
}

template <typename T>
__global__ void k_restrict(GridDev gf, GridDev gc, int kind, const c_t<T>* __restrict__ r, c_t<T>* __restrict__ fc,
                           const int* active) {
  if (active && !*active) return;
  const long long I = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= gc.N) return;
  int X, Y, Z;
  coords(gc, I, X, Y, Z);
  const int rad = transfer_radius(kind);
  const int rz = gf.dim == 3 ? rad : 0;
  c_t<T> acc = cmk<c_t<T>>(0, 0);
  for (int iz = 2 * Z - rz; iz <= 2 * Z + rz; ++iz) {
    if (iz < 0 || iz >= gf.nz) continue;
    const T wz = gf.dim == 3 ? (T)r1(kind, gf.nz, gc.nz, Z, iz) : (T)1;
    for (int iy = 2 * Y - rad; iy <= 2 * Y + rad; ++iy) {
      if (iy < 0 || iy >= gf.ny) continue;
      const T wyz = wz * (T)r1(kind, gf.ny, gc.ny, Y, iy);
      const long long row = ((long long)iz * gf.ny + iy) * gf.nx;
      for (int ix = 2 * X - rad; ix <= 2 * X + rad; ++ix) {
        if (ix < 0 || ix >= gf.nx) continue;
        const T wgt3 = wyz * (T)r1(kind, gf.nx, gc.nx, X, ix);
        const c_t<T> v = r[row + ix];
        acc.x += wgt3 * v.x;
        acc.y += wgt3 * v.y;
      }
    }
  }
  fc[I] = acc;
}

template <typename T>
__global__ void k_prolong_add(GridDev gf, GridDev gc, int kind, const c_t<T>* __restrict__ ec, c_t<T>* __restrict__ u,
                              const int* active) {
  if (active && !*active) return;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= gf.N) return;
  int x, y, z;
  coords(gf, p, x, y, z);
  const int rad = transfer_radius(kind);
  auto lo = [&](int j, int nc) { return max(0, (j - rad + 1) >> 1); };
  auto hi = [&](int j, int nc) { return min(nc - 1, (j + rad) >> 1); };
  int zlo = 0, zhi = 0;
  if (gf.dim == 3) {
    zlo = lo(z, gc.nz);
    zhi = hi(z, gc.nz);
  }
  c_t<T> acc = cmk<c_t<T>>(0, 0);
  for (int Z = zlo; Z <= zhi; ++Z) {
    const T wz = gf.dim == 3 ? (T)p1(kind, gf.nz, gc.nz, z, Z) : (T)1;
    if (wz == (T)0) continue;
    for (int Y = lo(y, gc.ny); Y <= hi(y, gc.ny); ++Y) {
      const T wyz = wz * (T)p1(kind, gf.ny, gc.ny, y, Y);
      if (wyz == (T)0) continue;
      const long long row = ((long long)Z * gc.ny + Y) * gc.nx;
      for (int X = lo(x, gc.nx); X <= hi(x, gc.nx); ++X) {
        const T w3 = wyz * (T)p1(kind, gf.nx, gc.nx, x, X);
        if (w3 == (T)0) continue;
        const c_t<T> v = ec[row + X];
        acc.x += w3 * v.x;
        acc.y += w3 * v.y;
      }
    }
  }
  u[p] = u[p] + acc;
}

// u = Ainv f, one warp per row
template <typename T>
__global__ void k_dense_gemv(int n, const c_t<T>* __restrict__ A, const c_t<T>* __restrict__ f, c_t<T>* __restrict__ u,
                             const int* active) {
  if (active && !*active) return;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  c_t<T> acc = cmk<c_t<T>>(0, 0);
  const c_t<T>* row = A + (long long)warp * n;
  for (int j = lane; j < n; j += 32) acc = cfma(row[j], f[j], acc);
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) u[warp] = acc;
}

template <typename T>
void residual_t(Ctx& c, int l, const void* u, const void* f, void* r, const int* active, cudaStream_t s) {
  Level& L = c.L[l];
  const long long N = L.g.N;
  if (L.fine) {
    k_fine_residual<T><<<nblk(N, kBlock), kBlock, 0, s>>>(L.g, (T)(1.0 / (c.h * c.h)), (const c_t<T>*)L.Aw,
                                                          (const c_t<T>*)u, (const c_t<T>*)f, (c_t<T>*)r, active);
  } else {
    k_stencil_residual<T><<<nblk(N, kBlock), kBlock, 0, s>>>(L.g, L.A.off, (const c_t<T>*)L.Aw, (const c_t<T>*)u,
                                                             (const c_t<T>*)f, (c_t<T>*)r, active);
  }
  HZ_LAUNCHED();
}

template <typename T>
void smooth_t(Ctx& c, int l, void* u, const void* f, bool u_is_zero, const int* active, cudaStream_t s) {
  Level& L = c.L[l];
  const long long N = L.g.N;
  const T w = (T)L.damping;
  if (u_is_zero) {
    k_vanka_apply<T, 0><<<nblk(N, kBlock), kBlock, 0, s>>>(L.g, L.M.off, (const c_t<T>*)L.Mw, w, (const c_t<T>*)f,
                                                           (c_t<T>*)u, active);
  } else {
    residual_t<T>(c, l, u, f, L.r, active, s);
    k_vanka_apply<T, 1><<<nblk(N, kBlock), kBlock, 0, s>>>(L.g, L.M.off, (const c_t<T>*)L.Mw, w,
                                                           (const c_t<T>*)L.r, (c_t<T>*)u, active);
  }
  HZ_LAUNCHED();
}

template <typename T>
void restrict_t(Ctx& c, int l, const void* r, void* fc, const int* active, cudaStream_t s) {
  Level& L = c.L[l];
  Level& C = c.L[l + 1];
  k_restrict<T><<<nblk(C.g.N, kBlock), kBlock, 0, s>>>(L.g, C.g, L.rkind, (const c_t<T>*)r, (c_t<T>*)fc, active);
  HZ_LAUNCHED();
}

template <typename T>
void prolong_t(Ctx& c, int l, const void* ec, void* u, const int* active, cudaStream_t s) {
  Level& L = c.L[l];
  Level& C = c.L[l + 1];
  k_prolong_add<T><<<nblk(L.g.N, kBlock), kBlock, 0, s>>>(L.g, C.g, L.pkind, (const c_t<T>*)ec, (c_t<T>*)u, active);
  HZ_LAUNCHED();
}

template <typename T>
void coarse_t(Ctx& c, const void* f, void* u, const int* active, cudaStream_t s) {
  Level& L = c.L.back();
  const int n = (int)L.g.N;
  k_dense_gemv<T><<<nblk((long long)n * 32, kBlock), kBlock, 0, s>>>(n, (const c_t<T>*)L.Ainvw, (const c_t<T>*)f,
                                                                   (c_t<T>*)u, active);
  HZ_LAUNCHED();
}

template <typename T>
void vcycle_t(Ctx& c, int l, const void* f, void* u, const int* active, cudaStream_t s) {
  Level& L = c.L[l];
  if (L.coarsest) {
    coarse_t<T>(c, f, u, active, s);
    return;
  }
  const int nu1 = c.opts.nu1, nu2 = c.opts.nu2;
  const size_t vb = sizeof(c_t<T>);
  if (nu1 > 0) {
    smooth_t<T>(c, l, u, f, true, active, s);                   // step 1 from u = 0
    for (int i = 1; i < nu1; ++i) smooth_t<T>(c, l, u, f, false, active, s);
  } else {
    HZ_CUDA(cudaMemsetAsync(u, 0, vb * L.g.N, s));
  }
  residual_t<T>(c, l, u, f, L.r, active, s);                    // step 2
  Level& C = c.L[l + 1];
  restrict_t<T>(c, l, L.r, C.f, active, s);
  vcycle_t<T>(c, l + 1, C.f, C.u, active, s);                   // step 3 (recursive)
  prolong_t<T>(c, l, C.u, u, active, s);                        // step 4
  for (int i = 0; i < nu2; ++i) smooth_t<T>(c, l, u, f, false, active, s);   // step 5
}

}  // namespace

void level_residual(Ctx& c, int l, const void* u, const void* f, void* r, const int* active, cudaStream_t s) {
  if (c.mixed) residual_t<float>(c, l, u, f, r, active, s);
  else residual_t<double>(c, l, u, f, r, active, s);
}
void level_smooth(Ctx& c, int l, void* u, const void* f, bool u_is_zero, const int* active, cudaStream_t s) {
  if (c.mixed) smooth_t<float>(c, l, u, f, u_is_zero, active, s);
  else smooth_t<double>(c, l, u, f, u_is_zero, active, s);
}
void level_restrict(Ctx& c, int l, const void* r, void* fc, const int* active, cudaStream_t s) {
  if (c.mixed) restrict_t<float>(c, l, r, fc, active, s);
  else restrict_t<double>(c, l, r, fc, active, s);
}
void level_prolong_add(Ctx& c, int l, const void* ec, void* u, const int* active, cudaStream_t s) {
  if (c.mixed) prolong_t<float>(c, l, ec, u, active, s);
  else prolong_t<double>(c, l, ec, u, active, s);
}
void level_vanka_apply(Ctx& c, int l, const void* r, void* u, cudaStream_t s) {
  Level& L = c.L[l];
  const long long N = L.g.N;
  if (c.mixed)
    k_vanka_apply<float, 1><<<nblk(N, kBlock), kBlock, 0, s>>>(L.g, L.M.off, (const float2*)L.Mw, (float)L.damping,
                                                               (const float2*)r, (float2*)u, nullptr);
  else
    k_vanka_apply<double, 1><<<nblk(N, kBlock), kBlock, 0, s>>>(L.g, L.M.off, (const double2*)L.Mw, L.damping,
                                                                (const double2*)r, (double2*)u, nullptr);
  HZ_LAUNCHED();
}
void coarse_solve(Ctx& c, const void* f, void* u, const int* active, cudaStream_t s) {
  if (c.mixed) coarse_t<float>(c, f, u, active, s);
  else coarse_t<double>(c, f, u, active, s);
}
void vcycle(Ctx& c, const void* f, void* u, const int* active, cudaStream_t s) {
  if (c.mixed) vcycle_t<float>(c, 0, f, u, active, s);
  else vcycle_t<double>(c, 0, f, u, active, s);
}
void fine_apply_f64(Ctx& c, const void* v, bool v_single, double2* w, bool shifted, cudaStream_t s) {
  Level& L = c.L[0];
  const double2* diag = shifted ? L.A64 : c.diagA64;    // plane 0 of the FP64 fine planes is diag(A_s)
  const double invh2 = 1.0 / (c.h * c.h);
  if (v_single)
    k_fine_apply64<float2><<<nblk(L.g.N, kBlock), kBlock, 0, s>>>(L.g, invh2, diag, (const float2*)v, w);
  else
    k_fine_apply64<double2><<<nblk(L.g.N, kBlock), kBlock, 0, s>>>(L.g, invh2, diag, (const double2*)v, w);
  HZ_LAUNCHED();
}

}  // namespace hz
