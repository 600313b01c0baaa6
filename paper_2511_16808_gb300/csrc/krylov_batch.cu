// FGMRES(m) for R right-hand sides at once (R a power of two <= 64) sharing one
// hierarchy: the same algorithm as krylov.cu (two-pass classical Gram-Schmidt,
// unnormalised V-cycle inputs with the scales folded into H and the update),
// per right-hand side, with the V-cycle applied to all R right-hand sides in
// one batched pass (RHS index innermost, field index node*R + r).  The FP64
// passes are persistent 1D sweeps over the fields in block ranges that are
// multiples of 256, so a thread always serves the same right-hand side.
//
// Every right-hand side has its own Krylov state (basis scales, Hessenberg
// column, Givens rotations, residual estimate, convergence): a right-hand side
// that has converged stops updating, so its iteration count is the one it has
// when solved alone.  Inner products are reduced per right-hand side in two
// deterministic stages (one partial per block and RHS, then one block per RHS
// that sums them in index order and runs that RHS's Arnoldi / restart step).
// A device counter of active right-hand sides gates the batched V-cycle and
// the iteration kernels; one restart cycle is one captured CUDA graph.
#include "krylov_impl.cuh"

#include <algorithm>
#include <vector>

namespace hz {

namespace {

constexpr int kB = 256;            // threads per block
constexpr int kPerB = 8;           // values per thread in the 1D passes

struct GeoB {
  int nx, ny, nz, N, dim;
  int R, lr, nxR, sxyR, NR;
  int p2;                  // 1/h^2 == 2^p2, else -1 (see pow2_exponent)
};
GeoB geob(const GridDev& g, int R, double invh2) {
  int lr = 0;
  while ((1 << lr) < R) ++lr;
  return GeoB{g.nx, g.ny, g.nz, (int)g.N, g.dim, R, lr, g.nx * R, g.nx * g.ny * R, (int)g.N * R,
              pow2_exponent(invh2)};
}
unsigned grid1(const GeoB& g) { return nblk(g.NR, kB * kPerB); }

// FP64 (A v) at node p, field index q (R right-hand sides, RHS innermost)
template <typename U>
__device__ __forceinline__ double2 apply_A_b(const GeoB& g, double invh2, const double2* __restrict__ diag,
                                             const U* v, int p, int q, int x, int y, int z) {
  const double2 d = diag[p], vp = ld64(v, q);
  const bool inx = x > 0 && x < g.nx - 1, iny = y > 0 && y < g.ny - 1;
  const bool inz = g.dim == 2 || (z > 0 && z < g.nz - 1);
  if (inx && iny && inz) {
    double2 s;
    if constexpr (std::is_same<U, float2>::value) {
      if (g.dim == 3) {
        const float2 n[6] = {v[q - g.R], v[q + g.R], v[q - g.nxR], v[q + g.nxR], v[q - g.sxyR], v[q + g.sxyR]};
        if (g.p2 >= 0) return diag_minus(d, vp, nbr_sum_pow2<6>(n, g.p2));
        s = nbr_sum<6>(n);
      } else {
        const float2 n[4] = {v[q - g.R], v[q + g.R], v[q - g.nxR], v[q + g.nxR]};
        if (g.p2 >= 0) return diag_minus(d, vp, nbr_sum_pow2<4>(n, g.p2));
        s = nbr_sum<4>(n);
      }
    } else {
      s = ld64(v, q - g.R) + ld64(v, q + g.R) + ld64(v, q - g.nxR) + ld64(v, q + g.nxR);
      if (g.dim == 3) s = s + ld64(v, q - g.sxyR) + ld64(v, q + g.sxyR);
    }
    return make_double2(fma(d.x, vp.x, fma(-d.y, vp.y, -invh2 * s.x)), fma(d.x, vp.y, fma(d.y, vp.x, -invh2 * s.y)));
  }
  double2 acc = cmul(d, vp);
  const double wx = inx ? 1.0 : 0.5, wy = iny ? 1.0 : 0.5;
  const double wz = (g.dim == 3 && !inz) ? 0.5 : 1.0;
  double2 sx = make_double2(0, 0), sy = make_double2(0, 0);
  if (x > 0) sx = sx + ld64(v, q - g.R);
  if (x < g.nx - 1) sx = sx + ld64(v, q + g.R);
  if (y > 0) sy = sy + ld64(v, q - g.nxR);
  if (y < g.ny - 1) sy = sy + ld64(v, q + g.nxR);
  const double cx = wy * wz * invh2, cy = wx * wz * invh2;
  acc.x -= cx * sx.x + cy * sy.x;
  acc.y -= cx * sx.y + cy * sy.y;
  if (g.dim == 3) {
    double2 sz = make_double2(0, 0);
    if (z > 0) sz = sz + ld64(v, q - g.sxyR);
    if (z < g.nz - 1) sz = sz + ld64(v, q + g.sxyR);
    const double cz = wx * wy * invh2;
    acc.x -= cz * sz.x;
    acc.y -= cz * sz.y;
  }
  return acc;
}


// Per-RHS block partials: thread t holds (acc, r); partials[r*nb + block] =
// the sum over the block's threads with that r (zero if none), in a fixed
// order.  Within a warp the lanes of one RHS are those congruent mod R (every
// layout here puts r = (32*k + lane) mod R), so a shuffle tree over offsets
// 16..R leaves lane l < min(R, 32) holding its RHS's warp sum; thread t < R
// then adds the 8 warps' sums for RHS t.
__device__ __forceinline__ void block_store_r(double2 acc, int r, int R, double2* __restrict__ partials, int nb,
                                              int block) {
  __shared__ double2 sv[kB / 32][32];
  __shared__ int sr0[kB / 32];
  __syncthreads();                          // the arrays may still be read by a previous call
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  for (int off = 16; off >= R; off >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
  }
  const int W = R < 32 ? R : 32;
  if (lane < W) sv[warp][lane] = acc;
  if (lane == 0) sr0[warp] = r;
  __syncthreads();
  if (tid < R) {
    double2 s = make_double2(0, 0);
#pragma unroll
    for (int w = 0; w < kB / 32; ++w) {
      const int l = (tid - sr0[w]) & (R - 1);
      if (l < W) s = s + sv[w][l];
    }
    partials[tid * nb + block] = s;
  }
}

// q_hat = wmass * q; partial ||q_hat||^2 per RHS
__global__ void __launch_bounds__(kB) k_scale_rhs_b(GeoB g, const double* __restrict__ wmass,
                                                    const double2* __restrict__ q, double2* __restrict__ qhat,
                                                    double2* __restrict__ partials) {
  pdl_enter();
  const int r = threadIdx.x & (g.R - 1);
  double2 acc = make_double2(0, 0);
  const int base = blockIdx.x * (kB * kPerB) + threadIdx.x;
#pragma unroll
  for (int k = 0; k < kPerB; ++k) {
    const int i = base + k * kB;
    if (i < g.NR) {
      const double2 v = wmass[i >> g.lr] * q[i];
      qhat[i] = v;
      acc.x = nrm_acc(acc.x, v);
    }
  }
  block_store_r(acc, r, g.R, partials, gridDim.x, blockIdx.x);
}

enum { kInit = 0, kDots = 1, kArnoldi = 2, kRestart = 3 };

// One block per RHS: sum its partials, then the RHS's state update.
// kDots: idx inner products (partials [(i*R + r)*nb + b]) -> h1[i];
// kArnoldi: the squared norm -> the Arnoldi column of iteration idx.
__global__ void k_reduce_b(const double2* __restrict__ partials, int nb, int R, int mode, int idx, KrylovState* st,
                           int* n_active, double tol, int max_iter, int m) {
  pdl_enter();
  if ((mode == kDots || mode == kArnoldi) && *n_active == 0) return;
  const int r = blockIdx.x;
  KrylovState* s = st + r;
  __shared__ double2 sm[kB];
  const int nsum = mode == kDots ? idx : 1;
  for (int i = 0; i < nsum; ++i) {
    const double2* pp = partials + ((long long)i * R + r) * nb;
    double2 acc = make_double2(0, 0);
    for (int b = threadIdx.x; b < nb; b += kB) acc = acc + pp[b];
    __syncthreads();
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int k = kB / 2; k > 0; k >>= 1) {
      if (threadIdx.x < k) sm[threadIdx.x] = sm[threadIdx.x] + sm[threadIdx.x + k];
      __syncthreads();
    }
    if (threadIdx.x == 0 && mode == kDots && s->active) s->h1[i] = sm[0];
  }
  if (threadIdx.x != 0 || mode == kDots) return;
  const double2 sum = sm[0];
  switch (mode) {
    case kInit: {
      const double bn = sqrt(sum.x);
      s->bnorm = bn;
      s->tol = tol;
      s->max_iter = max_iter;
      s->m = m;
      s->st.iters = 0;
      s->st.breakdown = 0;
      s->st.relres_est = bn > 0 ? 1.0 : 0.0;
      s->st.relres_true = bn > 0 ? 1.0 : 0.0;
      s->st.done = bn > 0 ? 0 : 1;
      s->st.converged = bn > 0 ? 0 : 1;
      s->active = 0;
      s->kcyc = 0;
      break;
    }
    case kArnoldi:
      if (s->active) {
        s->nrm2 = sum;
        arnoldi_update(s, idx, n_active, s->scale[idx]);
      }
      break;
    case kRestart:
      if (!s->st.done) {
        s->nrm2 = sum;
        restart_update(s, n_active);
      }
      break;
  }
}

// Persistent 1D sweep: this block's share of the NR field elements, in a
// range starting at a multiple of kB so that thread t always sees RHS t mod R.
__device__ __forceinline__ void block_range_b(int NR, int& e0, int& e1) {
  const int chunks = (NR + kB - 1) / kB;
  const int per = (chunks + gridDim.x - 1) / gridDim.x;
  e0 = min(NR, blockIdx.x * per * kB);
  e1 = min(NR, e0 + per * kB);
}

// node coordinates of field element e
__device__ __forceinline__ void coords_b(const GeoB& g, int e, int& p, int& x, int& y, int& z) {
  p = e >> g.lr;
  const int row = p / g.nx;
  x = p - row * g.nx;
  z = row / g.ny;
  y = row - z * g.ny;
}

// pass A: w = A z'_j -> V[j+1]; d_i = conj(V_i) . w per RHS, i < NV = j + 1
template <typename TZ, int NV>
__global__ void __launch_bounds__(kB) k_gs_dots_b(GeoB g, double invh2, const double2* __restrict__ diag,
                                                  const TZ* __restrict__ z, double2* __restrict__ V,
                                                  double2* __restrict__ partials, const KrylovState* __restrict__ st,
                                                  const int* n_active) {
  pdl_enter();
  if (*n_active == 0) return;
  const int r = threadIdx.x & (g.R - 1);
  double2 acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = make_double2(0, 0);
  if (st[r].active) {
    double2* w = V + (long long)NV * g.NR;
    int e0, e1;
    block_range_b(g.NR, e0, e1);
    for (int e = e0 + threadIdx.x; e < e1; e += kB) {
      int p, x, y, zz;
      coords_b(g, e, p, x, y, zz);
      const double2 a = apply_A_b(g, invh2, diag, z, p, e, x, y, zz);
      w[e] = a;
#pragma unroll
      for (int i = 0; i < NV; ++i) acc[i] = dot_acc(acc[i], V[(long long)i * g.NR + e], a);
    }
  }
#pragma unroll
  for (int i = 0; i < NV; ++i) block_store_r(acc[i], r, g.R, partials + (long long)i * g.R * gridDim.x, gridDim.x,
                                             blockIdx.x);
}

// pass B: w -= sum_{i < NV} scale_i^2 d_i V_i; ||w||^2 per RHS; f = w in the
// working precision (the next V-cycle input)
template <typename TF, int NV>
__global__ void __launch_bounds__(kB) k_gs_update_b(GeoB g, double2* __restrict__ V, TF* __restrict__ f,
                                                    double2* __restrict__ partials,
                                                    const KrylovState* __restrict__ st, const int* n_active) {
  pdl_enter();
  if (*n_active == 0) return;
  const int r = threadIdx.x & (g.R - 1);
  const KrylovState* s = st + r;
  double acc = 0.0;
  if (s->active) {
    double2 c[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const double sc = s->scale[i];
      c[i] = (sc * sc) * s->h1[i];
    }
    double2* w = V + (long long)NV * g.NR;
    int e0, e1;
    block_range_b(g.NR, e0, e1);
    for (int e = e0 + threadIdx.x; e < e1; e += kB) {
      double2 ww = w[e];
#pragma unroll
      for (int i = 0; i < NV; ++i) ww = axmy(ww, c[i], V[(long long)i * g.NR + e]);
      w[e] = ww;
      if constexpr (std::is_same<TF, float2>::value) f[e] = make_float2(d2f_rn(ww.x), d2f_rn(ww.y));
      else f[e] = ww;
      acc = nrm_acc(acc, ww);
    }
  }
  block_store_r(make_double2(acc, 0.0), r, g.R, partials, gridDim.x, blockIdx.x);
}

__global__ void k_solve_y_b(KrylovState* st, int R) {
  pdl_enter();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  KrylovState* s = st + r;
  if (s->st.done) return;
  const int k = s->kcyc;
  for (int i = k - 1; i >= 0; --i) {
    double2 acc = s->g[i];
    for (int l = i + 1; l < k; ++l) acc = acc - cmul(s->H[i][l], s->y[l]);
    s->y[i] = cdiv(acc, s->H[i][i]);
    s->c[i] = s->scale[i] * s->y[i];
  }
}

// p += sum_i y_i scale_i z'_i
template <typename TZ>
__global__ void k_update_p_b(GeoB g, const TZ* __restrict__ Z, const KrylovState* __restrict__ st,
                             double2* __restrict__ p) {
  pdl_enter();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= g.NR) return;
  const KrylovState* s = st + (q & (g.R - 1));
  if (s->st.done) return;
  const int k = s->kcyc;
  double2 acc = p[q];
  for (int i = 0; i < k; ++i) {
    const double2 yi = s->c[i], zi = ld64(Z, i * g.NR + q);
    acc = make_double2(fma(yi.x, zi.x, fma(-yi.y, zi.y, acc.x)), fma(yi.x, zi.y, fma(yi.y, zi.x, acc.y)));
  }
  p[q] = acc;
}

// r = q_hat - A p -> V_0 and f; partial ||r||^2 per RHS (RHS already done: skipped)
template <typename TF>
__global__ void __launch_bounds__(kB) k_true_residual_b(GeoB g, double invh2, const double2* __restrict__ diag,
                                                        const double2* __restrict__ pv,
                                                        const double2* __restrict__ qhat, double2* __restrict__ rv,
                                                        TF* __restrict__ f, double2* __restrict__ partials,
                                                        const KrylovState* __restrict__ st) {
  pdl_enter();
  const int r = threadIdx.x & (g.R - 1);
  double2 acc = make_double2(0, 0);
  if (!st[r].st.done) {
    int e0, e1;
    block_range_b(g.NR, e0, e1);
    for (int e = e0 + threadIdx.x; e < e1; e += kB) {
      int p, x, y, zz;
      coords_b(g, e, p, x, y, zz);
      const double2 v = qhat[e] - apply_A_b(g, invh2, diag, pv, p, e, x, y, zz);
      rv[e] = v;
      if constexpr (std::is_same<TF, float2>::value) f[e] = make_float2(d2f_rn(v.x), d2f_rn(v.y));
      else f[e] = v;
      acc.x = nrm_acc(acc.x, v);
    }
  }
  block_store_r(acc, r, g.R, partials, gridDim.x, blockIdx.x);
}

template <typename K>
unsigned persistent_grid(K kern, const GeoB& g) {
  return (unsigned)std::max(1, std::min<int>(nblk(g.NR, kB), resident_slots((const void*)kern, kB)));
}

template <typename TZ>
void run_cycle_b(Ctx& c, const GeoB& g, cudaStream_t s) {
  Level& L0 = c.L[0];
  const int m = c.opts.restart_m, R = g.R;
  const double invh2 = 1.0 / (c.h * c.h);
  KrylovState* st = c.ks;
  int* na = c.n_active;
  TZ* Z = (TZ*)c.Z;
  const double tol = c.opts.tol;
  const int mi = c.opts.max_iter;
  const double NR = g.NR;
  for (int j = 0; j < m; ++j) {
    const int nv = j + 1;
    int pk = prof_begin(c, 3, j, vcycle_bytes(c), 0.0, s);
    vcycle(c, L0.f, Z + (long long)j * g.NR, na, s);
    prof_end(c, pk, s);
    // pass A: z and diag read, w written, nv vectors read; A z 16 (3D: 20) flops + 8 per dot
    pk = prof_begin(c, 2, j, NR * (sizeof(TZ) + 16 + 16.0 * nv) + 16.0 * g.N,
                    ((g.dim == 3 ? 20.0 : 16.0) + 8.0 * nv) * NR, s);
    unsigned G = 0;
    with_nv(nv, [&](auto NV) {
      auto kern = k_gs_dots_b<TZ, decltype(NV)::value>;
      G = persistent_grid(kern, g);
      launch_pdl(kern, G, kB, s, g, invh2, c.diagA64, Z + (long long)j * g.NR, c.V, c.partials, st, na);
    });
    prof_end(c, pk, s);
    launch_pdl(k_reduce_b, R, kB, s, c.partials, G, R, kDots, nv, st, na, tol, mi, m);
    // pass B: w and nv vectors read, w and f written; 8 flops per vector + 4 for the norm
    pk = prof_begin(c, 1, j, NR * (32 + 16.0 * nv + sizeof(TZ)), (8.0 * nv + 4.0) * NR, s);
    with_nv(nv, [&](auto NV) {
      auto kern = k_gs_update_b<TZ, decltype(NV)::value>;
      G = persistent_grid(kern, g);
      launch_pdl(kern, G, kB, s, g, c.V, (TZ*)L0.f, c.partials, st, na);
    });
    prof_end(c, pk, s);
    launch_pdl(k_reduce_b, R, kB, s, c.partials, G, R, kArnoldi, j, st, na, tol, mi, m);
  }
  HZ_LAUNCHED();
  launch_pdl(k_solve_y_b, 1, 64, s, st, R);
  launch_pdl(k_update_p_b<TZ>, nblk(g.NR, 256), 256, s, g, Z, st, c.p);
  const unsigned Gt = persistent_grid(k_true_residual_b<TZ>, g);
  launch_pdl(k_true_residual_b<TZ>, Gt, kB, s, g, invh2, c.diagA64, c.p, c.qhat, c.V, (TZ*)L0.f, c.partials, st);
  launch_pdl(k_reduce_b, R, kB, s, c.partials, Gt, R, kRestart, 0, st, na, tol, mi, m);
  HZ_LAUNCHED();
}

template <typename TZ>
void ensure_graph_b(Ctx& c, const GeoB& g) {
  if (c.batch_graph && c.batch_graph_nrhs == g.R) return;
  if (c.batch_graph) cudaGraphExecDestroy(c.batch_graph);
  c.batch_graph = nullptr;
  // the two captured cycles share the event list: one profiled graph at a time
  if (c.prof_class && c.cycle_graph) {
    cudaGraphExecDestroy(c.cycle_graph);
    c.cycle_graph = nullptr;
  }
  c.prof_j.clear();
  c.prof_b.clear();
  c.prof_f.clear();
  cudaGraph_t graph = nullptr;
  HZ_CUDA(cudaStreamBeginCapture(c.graph_stream, cudaStreamCaptureModeThreadLocal));
  try {
    run_cycle_b<TZ>(c, g, c.graph_stream);
  } catch (...) {
    cudaStreamEndCapture(c.graph_stream, &graph);
    if (graph) cudaGraphDestroy(graph);
    throw;
  }
  HZ_CUDA(cudaStreamEndCapture(c.graph_stream, &graph));
  size_t nn = 0;
  HZ_CUDA(cudaGraphGetNodes(graph, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  HZ_CUDA(cudaGraphGetNodes(graph, nodes.data(), &nn));
  c.batch_graph_kernels = 0;
  for (auto n : nodes) {
    cudaGraphNodeType t;
    HZ_CUDA(cudaGraphNodeGetType(n, &t));
    if (t == cudaGraphNodeTypeKernel) ++c.batch_graph_kernels;
  }
  const cudaError_t e = cudaGraphInstantiate(&c.batch_graph, graph, 0);
  cudaGraphDestroy(graph);
  HZ_CUDA(e);
  c.batch_graph_nrhs = g.R;
}

template <typename TZ>
void solve_b(Ctx& c, const double2* q, double2* p, int R, hz_info* info, cudaStream_t user) {
  const GeoB g = geob(c.L[0].g, R, 1.0 / (c.h * c.h));
  c.nrhs = R;
  ensure_graph_b<TZ>(c, g);
  cudaStream_t s = c.graph_stream;
  KrylovState* st = c.ks;
  const int n1 = (int)grid1(g);
  const double invh2 = 1.0 / (c.h * c.h);
  HZ_CUDA(cudaEventRecord(c.ev_in, user));
  HZ_CUDA(cudaStreamWaitEvent(s, c.ev_in, 0));
  HZ_CUDA(cudaMemsetAsync(c.n_active, 0, sizeof(int), s));
  launch_pdl(k_scale_rhs_b, n1, kB, s, g, c.wmass, q, c.qhat, c.partials);
  launch_pdl(k_reduce_b, R, kB, s, c.partials, n1, R, kInit, 0, st, c.n_active, c.opts.tol, c.opts.max_iter,
                              c.opts.restart_m);
  HZ_CUDA(cudaMemsetAsync(c.p, 0, sizeof(double2) * g.NR, s));
  const unsigned Gt = persistent_grid(k_true_residual_b<TZ>, g);
  launch_pdl(k_true_residual_b<TZ>, Gt, kB, s, g, invh2, c.diagA64, c.p, c.qhat, c.V, (TZ*)c.L[0].f, c.partials, st);
  launch_pdl(k_reduce_b, R, kB, s, c.partials, Gt, R, kRestart, 0, st, c.n_active, c.opts.tol, c.opts.max_iter,
                              c.opts.restart_m);
  HZ_LAUNCHED();
  c.launches += 4;
  KrylovStatus* hs = (KrylovStatus*)c.ks_host;
  std::vector<int> before(R, 0), ran(R, 0);
  bool replayed = false;
  for (;;) {
    HZ_CUDA(cudaMemcpy2DAsync(hs, sizeof(KrylovStatus), st, sizeof(KrylovState), sizeof(KrylovStatus), R,
                              cudaMemcpyDeviceToHost, s));
    HZ_CUDA(cudaStreamSynchronize(s));
    if (replayed && c.prof_class) {
      int mx = 0;
      for (int r = 0; r < R; ++r) {
        ran[r] = hs[r].iters - before[r];
        mx = std::max(mx, ran[r]);
      }
      prof_collect(c, mx, ran.data(), R);
    }
    bool all = true;
    for (int r = 0; r < R; ++r) {
      all = all && hs[r].done;
      before[r] = hs[r].iters;
    }
    if (all) break;
    HZ_CUDA(cudaGraphLaunch(c.batch_graph, s));
    replayed = true;
    c.launches += c.batch_graph_kernels;
  }
  if (p != c.p) HZ_CUDA(cudaMemcpyAsync(p, c.p, sizeof(double2) * g.NR, cudaMemcpyDeviceToDevice, s));
  HZ_CUDA(cudaEventRecord(c.ev_out, s));
  HZ_CUDA(cudaStreamWaitEvent(user, c.ev_out, 0));
  c.nrhs = 1;
  for (int r = 0; r < R; ++r) {
    info[r].iters = hs[r].iters;
    info[r].converged = hs[r].converged;
    info[r].relres_est = hs[r].relres_est;
    info[r].relres_true = hs[r].relres_true;
  }
}

}  // namespace

void fgmres_solve_batch(Ctx& c, const double2* q, double2* p, int nrhs, hz_info* info, cudaStream_t s) {
  NvtxRange range("hz batched solve");
  {
    std::lock_guard<std::mutex> lk(c.history_mu);
    c.history.clear();
  }
  if (c.mixed) solve_b<float2>(c, q, p, nrhs, info, s);
  else solve_b<double2>(c, q, p, nrhs, info, s);
  if (c.tc_err) {
    // a bounded wait of the tensor-core coarsest solve that gave up leaves its
    // output untouched: report it instead of a result built on it
    int e = 0;
    HZ_CUDA(cudaMemcpy(&e, c.tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
      HZ_CUDA(cudaMemset(c.tc_err, 0, sizeof(int)));
      throw Error(HZ_ERR_TIMEOUT, "tensor-core coarsest solve: a bounded wait for the MMAs gave up");
    }
  }
}

}  // namespace hz
