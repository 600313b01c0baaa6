// Tuning tools of Section 5.2 on the GPU.
//
// 1. Local Fourier analysis of additive Vanka (Section 4) for a constant
//    stencil, for many damping values in one sweep: the smoothing factor
//    mu_loc (Definition 2.1: sup over high frequencies of |S~|, the scalar
//    symbol of Eq. smoother_symbol) and the two-grid factor rho_loc
//    (Definition 2.2: sup over low frequencies of the spectral radius of the
//    2^d x 2^d symbol TG~ of Eq. symbolTG).  One thread per frequency sample;
//    every damping value is evaluated from the same per-sample symbols.
// 2. The convergence factor of Eq. cf of the cycle used as a stationary solver
//    u <- u + B(f - A_s u) on a set-up hierarchy (the shift and per-level
//    damping searches run it once per candidate).
#include "krylov_impl.cuh"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <vector>

namespace hz {
namespace {

constexpr int kMaxPatch = 27;
constexpr int kMaxHarm = 8;
constexpr double kPi = 3.14159265358979323846;

struct LfaParams {
  int dim, np, nw, samples, nu;            // nu = nu1 + nu2
  int rk, pk;                              // 0 linear, 1 cubic
  double2 st[27];                          // stencil, index (dz+1)*9 + (dy+1)*3 + (dx+1)
  signed char off[kMaxPatch][3];           // patch offsets d_k
};

__host__ __device__ inline double2 cexp_i(double t) {
  double s, c;
  sincos(t, &s, &c);
  return make_double2(c, s);
}

__device__ inline double cabs1(double2 a) { return fabs(a.x) + fabs(a.y); }

__device__ inline double2 csqrt_(double2 z) {
  const double r = hypot(z.x, z.y);
  if (r == 0.0) return make_double2(0.0, 0.0);
  const double t = sqrt(0.5 * (r + fabs(z.x)));
  if (z.x >= 0.0) return make_double2(t, z.y / (2.0 * t));
  return make_double2(fabs(z.y) / (2.0 * t), copysign(t, z.y));
}

// Gauss-Jordan inverse of the constant patch matrix (H_i)_{kl} = s_{d_l - d_k}
// with partial pivoting, one thread (n <= 27).
__global__ void k_lfa_patch_inverse(LfaParams P, double2* __restrict__ inv, int* __restrict__ flag) {
  __shared__ double2 a[kMaxPatch][2 * kMaxPatch];
  if (threadIdx.x != 0) return;
  const int n = P.np;
  for (int k = 0; k < n; ++k)
    for (int l = 0; l < n; ++l) {
      int d[3], inside = 1;
      for (int c = 0; c < 3; ++c) {
        d[c] = P.off[l][c] - P.off[k][c];
        inside &= d[c] >= -1 && d[c] <= 1;
      }
      a[k][l] = inside ? P.st[(d[2] + 1) * 9 + (d[1] + 1) * 3 + (d[0] + 1)] : make_double2(0.0, 0.0);
      a[k][n + l] = make_double2(k == l ? 1.0 : 0.0, 0.0);
    }
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (cabs2(a[r][c]) > cabs2(a[piv][c])) piv = r;
    if (cabs2(a[piv][c]) == 0.0) {
      *flag = 1;
      return;
    }
    if (piv != c)
      for (int j = 0; j < 2 * n; ++j) {
        const double2 t = a[c][j];
        a[c][j] = a[piv][j];
        a[piv][j] = t;
      }
    const double2 ip = cdiv(make_double2(1.0, 0.0), a[c][c]);
    for (int j = 0; j < 2 * n; ++j) a[c][j] = cmul(a[c][j], ip);
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double2 f = a[r][c];
      for (int j = 0; j < 2 * n; ++j) a[r][j] = a[r][j] - cmul(f, a[c][j]);
    }
  }
  for (int k = 0; k < n; ++k)
    for (int l = 0; l < n; ++l) inv[k * n + l] = a[k][n + l];
}

// H~(theta) = sum_d s_d e^{i theta.d} over the 3^dim box.
__device__ double2 stencil_symbol(const LfaParams& P, const double* th) {
  double2 h = make_double2(0.0, 0.0);
  const int zr = P.dim == 3 ? 1 : 0;
  for (int dz = -zr; dz <= zr; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const double2 s = P.st[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)];
        if (s.x == 0.0 && s.y == 0.0) continue;
        h = h + cmul(s, cexp_i(th[0] * dx + th[1] * dy + th[2] * dz));
      }
  return h;
}

// (1/N) phi^H H_i^{-1} phi with phi_k = e^{i theta.d_k}: the scalar factor of
// Eq. smoother_symbol for equal weights 1/N.
__device__ double2 patch_factor(const LfaParams& P, const double2* __restrict__ inv, const double* th) {
  double2 phi[kMaxPatch];
  for (int k = 0; k < P.np; ++k) phi[k] = cexp_i(th[0] * P.off[k][0] + th[1] * P.off[k][1] + th[2] * P.off[k][2]);
  double2 m = make_double2(0.0, 0.0);
  for (int k = 0; k < P.np; ++k) {
    double2 row = make_double2(0.0, 0.0);
    for (int l = 0; l < P.np; ++l) row = row + cmul(inv[k * P.np + l], phi[l]);
    m = m + cconjmul(phi[k], row);
  }
  return (1.0 / P.np) * m;
}

// Per-axis transfer symbol of Section 4.2: (1 + cos t)/2 (linear) or
// (3 + 4 cos t + cos 2t)/8 (cubic); the product over the axes.
__device__ double transfer_symbol(int kind, const double* th, int dim) {
  double out = 1.0;
  for (int a = 0; a < dim; ++a) {
    const double c = cos(th[a]);
    out *= kind == 0 ? 0.5 * (1.0 + c) : (3.0 + 4.0 * c + cos(2.0 * th[a])) / 8.0;
  }
  return out;
}

// Eigenvalue moduli of a complex n x n matrix (n <= 8): Givens similarity
// rotations to upper Hessenberg form, then the single-shift QR iteration with
// Wilkinson shifts and deflation from the bottom (Golub & Van Loan, Matrix
// Computations, Secs. 7.4-7.5).  Only the active diagonal block is updated,
// which is all the eigenvalues need.  Returns max |lambda|, or NaN if an
// eigenvalue has not converged after 60 iterations.
struct Rot {
  double c;
  double2 s;
};
__device__ Rot givens(double2 a, double2 b) {
  const double na = hypot(a.x, a.y), nb = hypot(b.x, b.y);
  if (nb == 0.0) return {1.0, make_double2(0.0, 0.0)};
  if (na == 0.0) return {0.0, make_double2(b.x / nb, -b.y / nb)};
  const double nr = hypot(na, nb);
  const double2 al = make_double2(a.x / na, a.y / na);
  return {na / nr, (1.0 / nr) * cmul(al, make_double2(b.x, -b.y))};
}
__device__ inline void rot_rows(double2 (&A)[kMaxHarm][kMaxHarm], int i, int j, Rot g, int c0, int c1) {
  for (int c = c0; c <= c1; ++c) {
    const double2 x = A[i][c], y = A[j][c];
    A[i][c] = g.c * x + cmul(g.s, y);
    A[j][c] = g.c * y - cconjmul(g.s, x);
  }
}
__device__ inline void rot_cols(double2 (&A)[kMaxHarm][kMaxHarm], int i, int j, Rot g, int r0, int r1) {
  for (int r = r0; r <= r1; ++r) {
    const double2 x = A[r][i], y = A[r][j];
    A[r][i] = g.c * x + cconjmul(g.s, y);
    A[r][j] = g.c * y - cmul(g.s, x);
  }
}
__device__ double spectral_radius(double2 (&A)[kMaxHarm][kMaxHarm], int n) {
  for (int j = 0; j + 2 < n; ++j)
    for (int i = n - 1; i >= j + 2; --i) {
      const Rot g = givens(A[i - 1][j], A[i][j]);
      rot_rows(A, i - 1, i, g, j, n - 1);
      rot_cols(A, i - 1, i, g, 0, n - 1);
      A[i][j] = make_double2(0.0, 0.0);
    }
  const double eps = 2.220446049250313e-16;
  double rho = 0.0;
  int hi = n - 1, iter = 0;
  while (hi >= 0) {
    int l = hi;
    while (l > 0) {
      if (cabs1(A[l][l - 1]) <= eps * (cabs1(A[l - 1][l - 1]) + cabs1(A[l][l]))) {
        A[l][l - 1] = make_double2(0.0, 0.0);
        break;
      }
      --l;
    }
    if (l == hi) {
      rho = fmax(rho, hypot(A[hi][hi].x, A[hi][hi].y));
      --hi;
      iter = 0;
      continue;
    }
    if (++iter > 60) return nan("");
    double2 mu;
    const double2 a = A[hi - 1][hi - 1], b = A[hi - 1][hi], c = A[hi][hi - 1], d = A[hi][hi];
    if (iter % 11 == 10) {
      mu = d + make_double2(0.75 * hypot(c.x, c.y), 0.0);        // exceptional shift
    } else {
      const double2 half = 0.5 * (a - d);
      const double2 disc = csqrt_(cmul(half, half) + cmul(b, c));
      const double2 m1 = 0.5 * (a + d) + disc, m2 = 0.5 * (a + d) - disc;
      mu = cabs2(m1 - d) <= cabs2(m2 - d) ? m1 : m2;
    }
    for (int k = l; k <= hi; ++k) A[k][k] = A[k][k] - mu;
    Rot g[kMaxHarm];
    for (int k = l; k < hi; ++k) {
      g[k] = givens(A[k][k], A[k + 1][k]);
      rot_rows(A, k, k + 1, g[k], k, hi);
      A[k + 1][k] = make_double2(0.0, 0.0);
    }
    for (int k = l; k < hi; ++k) rot_cols(A, k, k + 1, g[k], l, min(k + 2, hi));
    for (int k = l; k <= hi; ++k) A[k][k] = A[k][k] + mu;
  }
  return rho;
}

__device__ inline void max_bits(unsigned long long* out, double v) {
  // non-negative doubles (and NaN) order like their bit patterns
  atomicMax(out, (unsigned long long)__double_as_longlong(v));
}

// mode 0: mu_loc over the high-frequency samples; mode 1: rho_loc over the
// low-frequency samples.  out[w] holds the running max as bits.
__global__ void __launch_bounds__(128) k_lfa_sweep(LfaParams P, const double2* __restrict__ inv_g,
                                                   const double* __restrict__ ws, int mode,
                                                   unsigned long long* __restrict__ out) {
  __shared__ double2 inv[kMaxPatch * kMaxPatch];
  for (int i = threadIdx.x; i < P.np * P.np; i += blockDim.x) inv[i] = inv_g[i];
  __syncthreads();
  long long total = 1;
  for (int a = 0; a < P.dim; ++a) total *= P.samples;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  double th[3] = {0.0, 0.0, 0.0};
  long long rem = i;
  bool high = false;
  for (int a = 0; a < P.dim; ++a) {
    const int ia = (int)(rem % P.samples);
    rem /= P.samples;
    th[a] = mode == 0 ? -kPi / 2 + 2 * kPi * ia / P.samples : -kPi / 2 + kPi * ia / P.samples;
    high |= th[a] >= kPi / 2;
  }
  if (mode == 0) {
    if (!high) return;
    const double2 h = stencil_symbol(P, th);
    const double2 mh = cmul(patch_factor(P, inv, th), h);
    for (int k = 0; k < P.nw; ++k) {
      const double2 s = make_double2(1.0, 0.0) - ws[k] * mh;
      max_bits(&out[k], hypot(s.x, s.y));
    }
    return;
  }
  const int K = 1 << P.dim;
  double2 mh[kMaxHarm], h[kMaxHarm];
  double rs[kMaxHarm], ps[kMaxHarm];
  double2 hc = make_double2(0.0, 0.0);
  for (int k = 0; k < K; ++k) {
    double tk[3] = {th[0], th[1], th[2]};
    for (int a = 0; a < P.dim; ++a)
      if ((k >> (P.dim - 1 - a)) & 1) tk[a] += kPi;
    h[k] = stencil_symbol(P, tk);
    mh[k] = cmul(patch_factor(P, inv, tk), h[k]);
    rs[k] = transfer_symbol(P.rk, tk, P.dim);
    ps[k] = transfer_symbol(P.pk, tk, P.dim);
    hc = hc + (rs[k] * ps[k]) * h[k];                         // Galerkin coarse symbol
  }
  for (int w = 0; w < P.nw; ++w) {
    // eig(S^nu2 C S^nu1) = eig(C S^(nu1+nu2)), C = I - P~ Hc^{-1} R~ H~
    double2 A[kMaxHarm][kMaxHarm];
    for (int j = 0; j < K; ++j) {
      const double2 s = make_double2(1.0, 0.0) - ws[w] * mh[j];
      double2 dj = make_double2(1.0, 0.0);
      for (int e = 0; e < P.nu; ++e) dj = cmul(dj, s);
      const double2 q = cdiv(rs[j] * h[j], hc);                // (R~ H~)_j / Hc
      for (int r = 0; r < K; ++r) {
        const double2 cij = (r == j ? make_double2(1.0, 0.0) : make_double2(0.0, 0.0)) - ps[r] * q;
        A[r][j] = cmul(cij, dj);
      }
    }
    max_bits(&out[w], spectral_radius(A, K));
  }
}

// Patch offsets of Section 3.2 around the patch's anchor, for the symbol.
std::vector<std::array<int, 3>> lfa_patch(int dim, hz_patch kind) {
  std::vector<std::array<int, 3>> out;
  const int zr = dim == 3 ? 1 : 0;
  if (kind == HZ_PATCH_ELEMENT) {
    for (int z = 0; z <= zr; ++z)
      for (int y = 0; y <= 1; ++y)
        for (int x = 0; x <= 1; ++x) out.push_back({x, y, z});
    return out;
  }
  for (int z = -zr; z <= zr; ++z)
    for (int y = -1; y <= 1; ++y)
      for (int x = -1; x <= 1; ++x) {
        const int l1 = std::abs(x) + std::abs(y) + std::abs(z);
        const bool in = kind == HZ_PATCH_FULL || (kind == HZ_PATCH_PLUS && l1 <= 1) ||
                        (kind == HZ_PATCH_RB && l1 % 2 == 0) || (kind == HZ_PATCH_JACOBI && l1 == 0);
        if (in) out.push_back({x, y, z});
      }
  return out;
}

__global__ void k_cf_residual(long long n, const double2* __restrict__ f, const double2* __restrict__ au,
                              double2* __restrict__ r, double* __restrict__ part, unsigned* __restrict__ count,
                              double* __restrict__ norm_out) {
  // r = f - A_s u and ||r||: block partial sums, the last block adds them in
  // block order (deterministic)
  __shared__ double sh[256];
  __shared__ bool last;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = f[i] - au[i];
    r[i] = v;
    acc += cabs2(v);
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x] = sh[0];
    __threadfence();
    last = atomicAdd(count, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double t = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) t += ((volatile double*)part)[b];
    *norm_out = sqrt(t);
    *count = 0;
  }
}

__global__ void k_cf_axpy(long long n, const double2* __restrict__ z, double2* __restrict__ u) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    u[i] = u[i] + z[i];
}

}  // namespace

void cycle_factor(Ctx& c, const double2* f, double2* u, int warmup, double target, int max_iter, double* factor,
                  int* iters, cudaStream_t s) {
  const long long N = c.L[0].g.N;
  // scratch: the first two FGMRES basis vectors (free outside a solve) and the
  // reduction partials
  double2* r = c.V;
  double2* w = c.V + N;
  const int G = std::max(1, max_slots() / 2);      // 4 blocks of 256 per SM (max_slots = 8 per SM)
  double* part = (double*)c.partials;
  double* norm = part + G;
  unsigned* count = (unsigned*)(norm + 1);
  HZ_CUDA(cudaMemsetAsync(count, 0, sizeof(unsigned), s));
  double h_norm = 0.0;
  auto residual = [&]() {
    fine_apply_f64(c, u, false, w, true, s);
    k_cf_residual<<<G, 256, 0, s>>>(N, f, w, r, part, count, norm);
    HZ_LAUNCHED();
    HZ_CUDA(cudaMemcpyAsync(&h_norm, norm, sizeof(double), cudaMemcpyDeviceToHost, s));
    HZ_CUDA(cudaStreamSynchronize(s));
    return h_norm;
  };
  auto step = [&]() {
    precond_apply_c128(c, r, w, 1, s);
    k_cf_axpy<<<G, 256, 0, s>>>(N, w, u);
    HZ_LAUNCHED();
  };
  const double rinit = residual();
  for (int i = 0; i < warmup; ++i) {
    step();
    residual();
  }
  const double r0 = h_norm;
  double rk = r0;
  int k = 0;
  while (k < max_iter && rk / rinit > target) {
    step();
    rk = residual();
    ++k;
  }
  *iters = k;
  *factor = k > 0 ? std::pow(rk / r0, 1.0 / k) : 0.0;
}

}  // namespace hz

extern "C" hz_status hz_lfa_factors(int dim, const double* stencil, hz_patch patch, const double* w, int nw,
                                    hz_intergrid rk, hz_intergrid pk, int nu1, int nu2, int samples, double* mu,
                                    double* rho) {
  using namespace hz;
  return guarded([&] {
    require(dim == 2 || dim == 3, "dim must be 2 or 3");
    require(stencil && w, "null argument");
    require(nw >= 1 && nw <= 1024, "nw must be in 1..1024");
    require(patch >= HZ_PATCH_JACOBI && patch <= HZ_PATCH_FULL, "bad patch");
    require((rk == HZ_IG_LINEAR || rk == HZ_IG_CUBIC) && (pk == HZ_IG_LINEAR || pk == HZ_IG_CUBIC),
            "rk/pk must be HZ_IG_LINEAR or HZ_IG_CUBIC");
    require(nu1 >= 0 && nu2 >= 0 && nu1 + nu2 <= 16, "nu1/nu2 out of range");
    require(samples >= 2 && samples <= (dim == 2 ? 4096 : 256), "samples out of range");
    for (int k = 0; k < nw; ++k) require(std::isfinite(w[k]), "non-finite damping");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) throw Error(HZ_ERR_NO_DEVICE, "no CUDA device");
    LfaParams P{};
    P.dim = dim;
    P.nw = nw;
    P.samples = samples;
    P.nu = nu1 + nu2;
    P.rk = rk == HZ_IG_CUBIC;
    P.pk = pk == HZ_IG_CUBIC;
    const int nst = dim == 3 ? 27 : 9;
    for (int i = 0; i < 27; ++i) P.st[i] = make_double2(0.0, 0.0);
    const int plane0 = dim == 3 ? 0 : 9;                        // 2D: the dz = 0 plane
    for (int i = 0; i < nst; ++i) {
      require(std::isfinite(stencil[2 * i]) && std::isfinite(stencil[2 * i + 1]), "non-finite stencil");
      P.st[plane0 + i] = make_double2(stencil[2 * i], stencil[2 * i + 1]);
    }
    const auto offs = lfa_patch(dim, patch);
    P.np = (int)offs.size();
    for (int k = 0; k < P.np; ++k)
      for (int a = 0; a < 3; ++a) P.off[k][a] = (signed char)offs[k][a];
    cudaStream_t s;
    HZ_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    struct Bufs {
      cudaStream_t s;
      void* p = nullptr;
      ~Bufs() {
        if (p) cudaFreeAsync(p, s);
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
      }
    } b{s};
    const size_t inv_b = sizeof(double2) * kMaxPatch * kMaxPatch;
    const size_t bytes = inv_b + sizeof(double) * nw + 2 * sizeof(unsigned long long) * nw + 16;
    HZ_CUDA(counted_malloc_async(&b.p, bytes, s));
    char* base = (char*)b.p;
    double2* inv = (double2*)base;
    double* wd = (double*)(base + inv_b);
    unsigned long long* out = (unsigned long long*)(wd + nw);
    int* flag = (int*)(out + 2 * nw);
    HZ_CUDA(cudaMemsetAsync(out, 0, 2 * sizeof(unsigned long long) * nw + sizeof(int), s));
    HZ_CUDA(cudaMemcpyAsync(wd, w, sizeof(double) * nw, cudaMemcpyHostToDevice, s));
    k_lfa_patch_inverse<<<1, 32, 0, s>>>(P, inv, flag);
    HZ_LAUNCHED();
    long long total = 1;
    for (int a = 0; a < dim; ++a) total *= samples;
    const unsigned blocks = (unsigned)((total + 127) / 128);
    if (mu) k_lfa_sweep<<<blocks, 128, 0, s>>>(P, inv, wd, 0, out);
    if (rho) k_lfa_sweep<<<blocks, 128, 0, s>>>(P, inv, wd, 1, out + nw);
    HZ_LAUNCHED();
    std::vector<unsigned long long> h(2 * nw);
    int hflag = 0;
    HZ_CUDA(cudaMemcpyAsync(h.data(), out, sizeof(unsigned long long) * 2 * nw, cudaMemcpyDeviceToHost, s));
    HZ_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    HZ_CUDA(cudaStreamSynchronize(s));
    require(hflag == 0, "the patch matrix is singular");
    for (int k = 0; k < nw; ++k) {
      double v;
      if (mu) {
        std::memcpy(&v, &h[k], sizeof v);
        mu[k] = v;
      }
      if (rho) {
        std::memcpy(&v, &h[nw + k], sizeof v);
        rho[k] = v;
      }
    }
  });
}
