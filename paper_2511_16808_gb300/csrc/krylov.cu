// Flexible GMRES(m) in FP64 around the multigrid V-cycle (Section 2.3; m = 5
// in Section 5.2), right preconditioned, zero initial guess (Section 5).
//
// Per inner iteration j (one preconditioner application):
//   f0 = cast(v_j)                 c128 -> working precision
//   z_j = V-cycle(f0)              stored in the working precision (the
//                                  Arnoldi relation A Z = V H holds for the
//                                  stored z_j, so FP32 storage loses nothing)
//   w = A z_j  fused with  h1 = V^H w               (one pass)
//   w -= V h1  fused with  h2 = V^H w, ||w||^2      (classical Gram-Schmidt,
//   w -= V h2  fused with  ||w||^2                    applied twice: CGS2)
//   H(:, j) = h1 + h2, H(j+1, j) = ||w||, complex Givens update of H and g,
//   residual estimate |g_{j+1}| / ||q_hat|| and the stop flag: all on the
//   device, no host synchronisation inside a restart cycle.
// v_{j+1} is stored unnormalised with its scale 1/||w|| (deferred
// normalisation).  At the end of a cycle: y = H^{-1} g (back substitution),
// p += Z y, true residual q_hat - A p in FP64, restart.  The host reads one
// small status record per restart cycle.
//
// Reductions are two-stage and deterministic: each pass kernel writes one
// partial per block, a second kernel sums the partials in a fixed order.
#include <cstddef>
#include <type_traits>

#include "common.cuh"

namespace hz {

constexpr int kMaxM = 16;
constexpr int kRedBlock = 256;

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
  double2 h1[kMaxM + 1];    // raw dots conj(V_i) . w of the two CGS passes
  double2 h2[kMaxM + 2];
  double2 nrm2;             // .x = ||w||^2
};

namespace {

inline unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

__device__ __forceinline__ void coords(const GridDev& g, long long p, int& x, int& y, int& z) {
  x = (int)(p % g.nx);
  long long t = p / g.nx;
  y = (int)(t % g.ny);
  z = (int)(t / g.ny);
}

template <typename U>
__device__ __forceinline__ double2 ld64(const U* __restrict__ a, long long i) {
  const U v = a[i];
  return make_double2((double)v.x, (double)v.y);
}

// FP64 fine-level A v at node p (5-/7-point, half-cell weights)
template <typename U>
__device__ __forceinline__ double2 apply_A(const GridDev& g, double invh2, const double2* __restrict__ diag,
                                           const U* __restrict__ v, long long p) {
  int x, y, z;
  coords(g, p, x, y, z);
  const double wx = wgt(x, g.nx), wy = wgt(y, g.ny);
  const double wz = g.dim == 3 ? wgt(z, g.nz) : 1.0;
  double2 acc = cmul(diag[p], ld64(v, p));
  double2 sx = make_double2(0, 0), sy = make_double2(0, 0);
  if (x > 0) sx = sx + ld64(v, p - 1);
  if (x < g.nx - 1) sx = sx + ld64(v, p + 1);
  if (y > 0) sy = sy + ld64(v, p - g.nx);
  if (y < g.ny - 1) sy = sy + ld64(v, p + g.nx);
  const double cx = wy * wz * invh2, cy = wx * wz * invh2;
  acc.x -= cx * sx.x + cy * sy.x;
  acc.y -= cx * sx.y + cy * sy.y;
  if (g.dim == 3) {
    const long long pl = (long long)g.nx * g.ny;
    double2 sz = make_double2(0, 0);
    if (z > 0) sz = sz + ld64(v, p - pl);
    if (z < g.nz - 1) sz = sz + ld64(v, p + pl);
    const double cz = wx * wy * invh2;
    acc.x -= cz * sz.x;
    acc.y -= cz * sz.y;
  }
  return acc;
}

// Block-reduce K double2 accumulators; thread 0 writes partials[k*nb + block].
template <int K>
__device__ __forceinline__ void block_store(double2 (&acc)[K], double2* __restrict__ partials, int nb) {
  __shared__ double2 sm[K][kRedBlock / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double2 v = acc[k];
    for (int o = 16; o > 0; o >>= 1) {
      v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    if (lane == 0) sm[k][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double2 s = make_double2(0, 0);
    for (int w = 0; w < kRedBlock / 32; ++w) s = s + sm[threadIdx.x][w];
    partials[(long long)threadIdx.x * nb + blockIdx.x] = s;
  }
}

// w = A z_j -> V[NV]; partial dots conj(V_i) . w, i < NV
template <int NV, typename TZ>
__global__ void __launch_bounds__(kRedBlock) k_matvec_dots(GridDev g, double invh2, const double2* __restrict__ diag,
                                                           const TZ* __restrict__ z, double2* __restrict__ V,
                                                           double2* __restrict__ partials, int nb,
                                                           const KrylovState* __restrict__ st) {
  if (!st->active) return;
  double2 acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = make_double2(0, 0);
  const long long N = g.N;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
    const double2 w = apply_A(g, invh2, diag, z, p);
    V[(long long)NV * N + p] = w;
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = acc[i] + cconjmul(V[(long long)i * N + p], w);
  }
  block_store<NV>(acc, partials, nb);
}

// w -= sum_i c_i V_i with c_i = raw_i * scale_i^2; FIRST: partial dots of the
// result with V_i (i < NV) and ||w||^2 (slot NV); else only ||w||^2 (slot 0).
template <int NV, bool FIRST>
__global__ void __launch_bounds__(kRedBlock) k_orth(long long N, double2* __restrict__ V, double2* __restrict__ partials,
                                                    int nb, const KrylovState* __restrict__ st) {
  if (!st->active) return;
  double2 c[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const double s = st->scale[i];
    const double2 raw = FIRST ? st->h1[i] : st->h2[i];
    c[i] = (s * s) * raw;
  }
  constexpr int K = FIRST ? NV + 1 : 1;
  double2 acc[K];
#pragma unroll
  for (int i = 0; i < K; ++i) acc[i] = make_double2(0, 0);
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
    double2 w = V[(long long)NV * N + p];
    double2 vi[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      vi[i] = V[(long long)i * N + p];
      w = w - cmul(c[i], vi[i]);
    }
    V[(long long)NV * N + p] = w;
    if (FIRST) {
#pragma unroll
      for (int i = 0; i < NV; ++i) acc[i] = acc[i] + cconjmul(vi[i], w);
    }
    acc[K - 1].x += cabs2(w);
  }
  block_store<K>(acc, partials, nb);
}

// out[v] = sum_b partials[v*nb + b], one block per v; runs when *flag != 0
__global__ void k_reduce(const double2* __restrict__ partials, int nb, double2* __restrict__ out, const int* flag,
                         int flag_value) {
  if (flag && *flag != flag_value) return;
  __shared__ double2 sm[kRedBlock];
  const int v = blockIdx.x;
  double2 s = make_double2(0, 0);
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s = s + partials[(long long)v * nb + b];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) sm[threadIdx.x] = sm[threadIdx.x] + sm[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[v] = sm[0];
}

__device__ void givens(double2 a, double2 b, double& c, double2& s) {
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

// Column j of the Hessenberg matrix, Givens rotations, residual estimate.
__global__ void k_arnoldi(KrylovState* __restrict__ st, int j) {
  if (!st->active) return;
  for (int i = 0; i <= j; ++i) st->H[i][j] = st->scale[i] * (st->h1[i] + st->h2[i]);
  const double hn = sqrt(st->nrm2.x);
  st->H[j + 1][j] = make_double2(hn, 0.0);
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
  if (st->st.relres_est < st->tol || st->st.iters >= st->max_iter || st->st.breakdown || st->kcyc >= st->m)
    st->active = 0;
}

template <typename V>
__global__ void k_cast_in(long long N, const double2* __restrict__ v, const KrylovState* __restrict__ st, int j,
                          V* __restrict__ f) {
  if (!st->active) return;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  f[p] = from_c128<V>(st->scale[j] * v[p]);
}

__global__ void k_solve_y(KrylovState* __restrict__ st) {
  if (st->st.done) return;
  const int k = st->kcyc;
  for (int i = k - 1; i >= 0; --i) {
    double2 acc = st->g[i];
    for (int l = i + 1; l < k; ++l) acc = acc - cmul(st->H[i][l], st->y[l]);
    st->y[i] = cdiv(acc, st->H[i][i]);
  }
}

template <typename TZ>
__global__ void k_update_p(long long N, const TZ* __restrict__ Z, const KrylovState* __restrict__ st,
                           double2* __restrict__ p) {
  if (st->st.done) return;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N) return;
  const int k = st->kcyc;
  double2 acc = p[q];
  for (int i = 0; i < k; ++i) acc = acc + cmul(st->y[i], ld64(Z, (long long)i * N + q));
  p[q] = acc;
}

// r = q_hat - A p -> V_0; partial ||r||^2
__global__ void __launch_bounds__(kRedBlock) k_true_residual(GridDev g, double invh2, const double2* __restrict__ diag,
                                                             const double2* __restrict__ p,
                                                             const double2* __restrict__ qhat, double2* __restrict__ r,
                                                             double2* __restrict__ partials, int nb,
                                                             const KrylovState* __restrict__ st) {
  if (st->st.done) return;
  double2 acc[1] = {make_double2(0, 0)};
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < g.N; q += (long long)gridDim.x * blockDim.x) {
    const double2 v = qhat[q] - apply_A(g, invh2, diag, p, q);
    r[q] = v;
    acc[0].x += cabs2(v);
  }
  block_store<1>(acc, partials, nb);
}

__global__ void k_restart(KrylovState* __restrict__ st) {
  if (st->st.done) return;
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
}

// q_hat = wmass * q; partial ||q_hat||^2
__global__ void __launch_bounds__(kRedBlock) k_scale_rhs(long long N, const double* __restrict__ wmass,
                                                         const double2* __restrict__ q, double2* __restrict__ qhat,
                                                         double2* __restrict__ partials, int nb) {
  double2 acc[1] = {make_double2(0, 0)};
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
    const double2 v = wmass[p] * q[p];
    qhat[p] = v;
    acc[0].x += cabs2(v);
  }
  block_store<1>(acc, partials, nb);
}

__global__ void k_init(KrylovState* __restrict__ st, double tol, int max_iter, int m) {
  const double bn = sqrt(st->nrm2.x);
  st->bnorm = bn;
  st->tol = tol;
  st->max_iter = max_iter;
  st->m = m;
  st->st.iters = 0;
  st->st.breakdown = 0;
  st->st.relres_est = bn > 0 ? 1.0 : 0.0;
  st->st.relres_true = bn > 0 ? 1.0 : 0.0;
  st->st.done = bn > 0 ? 0 : 1;
  st->st.converged = bn > 0 ? 0 : 1;
  st->active = 0;
  st->kcyc = 0;
}

template <typename V>
__global__ void k_cast_vec(long long N, const double2* __restrict__ in, V* __restrict__ out) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < N) out[p] = from_c128<V>(in[p]);
}
template <typename V>
__global__ void k_widen_vec(long long N, const V* __restrict__ in, double2* __restrict__ out) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < N) out[p] = ld64(in, p);
}

template <typename F>
void dispatch_nv(int nv, F&& f) {
  switch (nv) {
#define HZ_NV(k) case k: f(std::integral_constant<int, k>{}); break;
    HZ_NV(1) HZ_NV(2) HZ_NV(3) HZ_NV(4) HZ_NV(5) HZ_NV(6) HZ_NV(7) HZ_NV(8)
    HZ_NV(9) HZ_NV(10) HZ_NV(11) HZ_NV(12) HZ_NV(13) HZ_NV(14) HZ_NV(15) HZ_NV(16)
#undef HZ_NV
    default: throw Error(HZ_ERR_INVALID_ARG, "restart length out of range");
  }
}

template <typename TZ>
void run_cycle(Ctx& c, double2* p, cudaStream_t s) {
  Level& L0 = c.L[0];
  const long long N = L0.g.N;
  const int m = c.opts.restart_m;
  const int nb = c.red_blocks;
  const double invh2 = 1.0 / (c.h * c.h);
  KrylovState* st = c.ks;
  const int* active = &st->active;
  TZ* Z = (TZ*)c.Z;
  for (int j = 0; j < m; ++j) {
    k_cast_in<TZ><<<nblk(N, 256), 256, 0, s>>>(N, c.V + (long long)j * N, st, j, (TZ*)L0.f);
    vcycle(c, L0.f, Z + (long long)j * N, active, s);
    dispatch_nv(j + 1, [&](auto nvc) {
      constexpr int NV = decltype(nvc)::value;
      k_matvec_dots<NV, TZ><<<nb, kRedBlock, 0, s>>>(L0.g, invh2, c.diagA64, Z + (long long)j * N, c.V,
                                                     c.partials, nb, st);
      k_reduce<<<NV, kRedBlock, 0, s>>>(c.partials, nb, st->h1, active, 1);
      k_orth<NV, true><<<nb, kRedBlock, 0, s>>>(N, c.V, c.partials, nb, st);
      k_reduce<<<NV + 1, kRedBlock, 0, s>>>(c.partials, nb, st->h2, active, 1);
      k_orth<NV, false><<<nb, kRedBlock, 0, s>>>(N, c.V, c.partials, nb, st);
      k_reduce<<<1, kRedBlock, 0, s>>>(c.partials, nb, &st->nrm2, active, 1);
    });
    k_arnoldi<<<1, 1, 0, s>>>(st, j);
  }
  HZ_LAUNCHED();
  const int* done = &st->st.done;
  k_solve_y<<<1, 1, 0, s>>>(st);
  k_update_p<TZ><<<nblk(N, 256), 256, 0, s>>>(N, Z, st, p);
  k_true_residual<<<nb, kRedBlock, 0, s>>>(L0.g, invh2, c.diagA64, p, c.qhat, c.V, c.partials, nb, st);
  k_reduce<<<1, kRedBlock, 0, s>>>(c.partials, nb, &st->nrm2, done, 0);
  k_restart<<<1, 1, 0, s>>>(st);
  HZ_LAUNCHED();
}

template <typename TZ>
void solve_t(Ctx& c, const double2* q, double2* p, hz_info* info, cudaStream_t s) {
  Level& L0 = c.L[0];
  const long long N = L0.g.N;
  const int nb = c.red_blocks;
  const double invh2 = 1.0 / (c.h * c.h);
  KrylovState* st = c.ks;
  KrylovStatus* hs = (KrylovStatus*)c.ks_host;
  k_scale_rhs<<<nb, kRedBlock, 0, s>>>(N, c.wmass, q, c.qhat, c.partials, nb);
  k_reduce<<<1, kRedBlock, 0, s>>>(c.partials, nb, &st->nrm2, nullptr, 0);
  k_init<<<1, 1, 0, s>>>(st, c.opts.tol, c.opts.max_iter, c.opts.restart_m);
  HZ_CUDA(cudaMemsetAsync(p, 0, sizeof(double2) * N, s));
  k_true_residual<<<nb, kRedBlock, 0, s>>>(L0.g, invh2, c.diagA64, p, c.qhat, c.V, c.partials, nb, st);
  k_reduce<<<1, kRedBlock, 0, s>>>(c.partials, nb, &st->nrm2, &st->st.done, 0);
  k_restart<<<1, 1, 0, s>>>(st);
  HZ_LAUNCHED();
  for (;;) {
    HZ_CUDA(cudaMemcpyAsync(hs, &st->st, sizeof(KrylovStatus), cudaMemcpyDeviceToHost, s));
    HZ_CUDA(cudaStreamSynchronize(s));
    if (hs->done) break;
    run_cycle<TZ>(c, p, s);
  }
  info->iters = hs->iters;
  info->converged = hs->converged;
  info->relres_est = hs->relres_est;
  info->relres_true = hs->relres_true;
}

}  // namespace

size_t krylov_bytes(const hz_grid& g, const hz_opts& o) {
  long long N = (long long)g.n[0] * g.n[1] * (g.dim == 3 ? g.n[2] : 1);
  const size_t vb = o.precision == HZ_PREC_MIXED ? 8 : 16;
  const int m = o.restart_m;
  return 16ull * N * (m + 1) + vb * N * m + 16ull * N * 3 + 16ull * (kMaxM + 2) * 2048 + sizeof(KrylovState);
}

void krylov_alloc(Ctx& c) {
  const long long N = c.L[0].g.N;
  const int m = c.opts.restart_m;
  const size_t vb = c.mixed ? sizeof(float2) : sizeof(double2);
  require(m >= 1 && m <= kMaxM, "restart_m must be in 1..16");
  c.V = (double2*)ctx_alloc(c, sizeof(double2) * N * (m + 1));
  c.Z = ctx_alloc(c, vb * N * m);
  c.qhat = (double2*)ctx_alloc(c, sizeof(double2) * N);
  c.red_blocks = (int)std::min<long long>(nblk(N, kRedBlock), 1216);
  c.partials = (double2*)ctx_alloc(c, sizeof(double2) * (kMaxM + 2) * c.red_blocks);
  c.ks = (KrylovState*)ctx_alloc(c, sizeof(KrylovState));
  HZ_CUDA(cudaMemset(c.ks, 0, sizeof(KrylovState)));
  HZ_CUDA(cudaMallocHost(&c.ks_host, sizeof(KrylovStatus)));
}

void fgmres_solve(Ctx& c, const double2* q, double2* p, hz_info* info, cudaStream_t s) {
  if (c.mixed) solve_t<float2>(c, q, p, info, s);
  else solve_t<double2>(c, q, p, info, s);
}

void precond_apply_c128(Ctx& c, const double2* r, double2* z, cudaStream_t s) {
  Level& L0 = c.L[0];
  const long long N = L0.g.N;
  if (c.mixed) {
    k_cast_vec<float2><<<nblk(N, 256), 256, 0, s>>>(N, r, (float2*)L0.f);
    vcycle(c, L0.f, L0.u, nullptr, s);
    k_widen_vec<float2><<<nblk(N, 256), 256, 0, s>>>(N, (const float2*)L0.u, z);
  } else {
    HZ_CUDA(cudaMemcpyAsync(L0.f, r, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s));
    vcycle(c, L0.f, L0.u, nullptr, s);
    HZ_CUDA(cudaMemcpyAsync(z, L0.u, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s));
  }
  HZ_LAUNCHED();
}

}  // namespace hz
