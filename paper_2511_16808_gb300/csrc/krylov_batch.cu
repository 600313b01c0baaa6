// FGMRES(m) for R right-hand sides at once (R a power of two <= 64) sharing one
// hierarchy: the same algorithm as krylov.cu, per right-hand side, with the
// V-cycle applied to all R right-hand sides in one batched pass (RHS index
// innermost, field index node*R + r).
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
constexpr int kRowsB = 8;          // y rows per thread in the 2D passes
constexpr int kPerB = 8;           // values per thread in the 1D passes

struct GeoB {
  int nx, ny, nz, N, dim;
  int R, lr, nxR, sxyR, NR;
};
GeoB geob(const GridDev& g, int R) {
  int lr = 0;
  while ((1 << lr) < R) ++lr;
  return GeoB{g.nx, g.ny, g.nz, (int)g.N, g.dim, R, lr, g.nx * R, g.nx * g.ny * R, (int)g.N * R};
}
dim3 grid2(const GeoB& g) {
  return dim3((g.nxR + BX - 1) / BX, (g.ny + BY * kRowsB - 1) / (BY * kRowsB), g.nz < 8 ? g.nz : 8);
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
    double2 s = ld64(v, q - g.R) + ld64(v, q + g.R) + ld64(v, q - g.nxR) + ld64(v, q + g.nxR);
    if (g.dim == 3) s = s + ld64(v, q - g.sxyR) + ld64(v, q + g.sxyR);
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

__device__ __forceinline__ int block_lin() { return (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x; }

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

enum { kInit = 0, kH1 = 1, kArnoldi = 2, kRestart = 3 };

// One block per RHS: sum its partials, then the RHS's state update.
__global__ void k_reduce_b(const double2* __restrict__ partials, int nb, int mode, int idx, KrylovState* st,
                           int* n_active, double tol, int max_iter, int m) {
  if ((mode == kH1 || mode == kArnoldi) && *n_active == 0) return;
  const int r = blockIdx.x;
  KrylovState* s = st + r;
  __shared__ double2 sm[kB];
  double2 acc = make_double2(0, 0);
  for (int b = threadIdx.x; b < nb; b += kB) acc = acc + partials[r * nb + b];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int k = kB / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) sm[threadIdx.x] = sm[threadIdx.x] + sm[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
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
    case kH1:
      if (s->active) s->h1[idx] = sum;
      break;
    case kArnoldi:
      if (s->active) {
        s->nrm2 = sum;
        arnoldi_update(s, idx, n_active);
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

template <typename V>
__global__ void k_cast_in_b(GeoB g, const double2* __restrict__ v, const KrylovState* __restrict__ st, int j,
                            V* __restrict__ f, const int* n_active) {
  if (*n_active == 0) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.NR) return;
  const KrylovState* s = st + (i & (g.R - 1));
  if (!s->active) return;
  const double2 a = v[i];
  if constexpr (std::is_same<V, float2>::value) {
    const float sc = d2f_rn(s->scale[j]);
    f[i] = make_float2(d2f_rn(a.x) * sc, d2f_rn(a.y) * sc);
  } else {
    f[i] = s->scale[j] * a;
  }
}

// pass 0: w = A z_j -> V[j+1]; partial conj(V_0) . w per RHS
template <typename TZ>
__global__ void __launch_bounds__(kB) k_mgs_first_b(GeoB g, double invh2, const double2* __restrict__ diag,
                                                    const TZ* __restrict__ z, double2* __restrict__ V, int j,
                                                    double2* __restrict__ partials, const KrylovState* __restrict__ st,
                                                    const int* n_active) {
  if (*n_active == 0) return;
  const int X = blockIdx.x * BX + threadIdx.x;
  const int r = X & (g.R - 1);
  const bool act = X < g.nxR && st[r].active;
  double2 acc = make_double2(0, 0);
  double2* w = V + (long long)(j + 1) * g.NR;
  if (act) {
    const int x = X >> g.lr;
    for (int zz = blockIdx.z; zz < g.nz; zz += gridDim.z) {
#pragma unroll
      for (int k = 0; k < kRowsB; ++k) {
        const int y = (blockIdx.y * kRowsB + k) * BY + threadIdx.y;
        if (y >= g.ny) break;
        const int row = zz * g.ny + y;
        const int p = row * g.nx + x, q = row * g.nxR + X;
        const double2 a = apply_A_b(g, invh2, diag, z, p, q, x, y, zz);
        w[q] = a;
        acc = dot_acc(acc, V[q], a);
      }
    }
  }
  block_store_r(acc, r, g.R, partials, gridDim.x * gridDim.y * gridDim.z, block_lin());
}

// pass i: w -= h_{i-1} v_{i-1}; partial conj(V_i) . w (LAST: ||w||^2) per RHS
template <bool LAST>
__global__ void __launch_bounds__(kB) k_mgs_step_b(GeoB g, double2* __restrict__ V, int j, int i,
                                                   double2* __restrict__ partials,
                                                   const KrylovState* __restrict__ st, const int* n_active) {
  if (*n_active == 0) return;
  const int r = threadIdx.x & (g.R - 1);
  const KrylovState* s = st + r;
  double2 acc = make_double2(0, 0);
  if (s->active) {
    const double sc = s->scale[i - 1];
    const double2 c = (sc * sc) * s->h1[i - 1];
    const double2* vp = V + (long long)(i - 1) * g.NR;
    const double2* vi = V + (long long)i * g.NR;
    double2* w = V + (long long)(j + 1) * g.NR;
    const int base = blockIdx.x * (kB * kPerB) + threadIdx.x;
#pragma unroll
    for (int k = 0; k < kPerB; ++k) {
      const int p = base + k * kB;
      if (p < g.NR) {
        const double2 ww = axmy(w[p], c, vp[p]);
        w[p] = ww;
        if (LAST) acc.x = nrm_acc(acc.x, ww);
        else acc = dot_acc(acc, vi[p], ww);
      }
    }
  }
  block_store_r(acc, r, g.R, partials, gridDim.x, blockIdx.x);
}

__global__ void k_solve_y_b(KrylovState* st, int R) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  KrylovState* s = st + r;
  if (s->st.done) return;
  const int k = s->kcyc;
  for (int i = k - 1; i >= 0; --i) {
    double2 acc = s->g[i];
    for (int l = i + 1; l < k; ++l) acc = acc - cmul(s->H[i][l], s->y[l]);
    s->y[i] = cdiv(acc, s->H[i][i]);
  }
}

template <typename TZ>
__global__ void k_update_p_b(GeoB g, const TZ* __restrict__ Z, const KrylovState* __restrict__ st,
                             double2* __restrict__ p) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= g.NR) return;
  const KrylovState* s = st + (q & (g.R - 1));
  if (s->st.done) return;
  const int k = s->kcyc;
  double2 acc = p[q];
  for (int i = 0; i < k; ++i) {
    const double2 yi = s->y[i], zi = ld64(Z, i * g.NR + q);
    acc = make_double2(fma(yi.x, zi.x, fma(-yi.y, zi.y, acc.x)), fma(yi.x, zi.y, fma(yi.y, zi.x, acc.y)));
  }
  p[q] = acc;
}

// r = q_hat - A p -> V_0; partial ||r||^2 per RHS (RHS already done: skipped)
__global__ void __launch_bounds__(kB) k_true_residual_b(GeoB g, double invh2, const double2* __restrict__ diag,
                                                        const double2* __restrict__ pv,
                                                        const double2* __restrict__ qhat, double2* __restrict__ rv,
                                                        double2* __restrict__ partials,
                                                        const KrylovState* __restrict__ st) {
  const int X = blockIdx.x * BX + threadIdx.x;
  const int r = X & (g.R - 1);
  const bool act = X < g.nxR && !st[r].st.done;
  double2 acc = make_double2(0, 0);
  if (act) {
    const int x = X >> g.lr;
    for (int zz = blockIdx.z; zz < g.nz; zz += gridDim.z) {
#pragma unroll
      for (int k = 0; k < kRowsB; ++k) {
        const int y = (blockIdx.y * kRowsB + k) * BY + threadIdx.y;
        if (y >= g.ny) break;
        const int row = zz * g.ny + y;
        const int p = row * g.nx + x, q = row * g.nxR + X;
        const double2 v = qhat[q] - apply_A_b(g, invh2, diag, pv, p, q, x, y, zz);
        rv[q] = v;
        acc.x = nrm_acc(acc.x, v);
      }
    }
  }
  block_store_r(acc, r, g.R, partials, gridDim.x * gridDim.y * gridDim.z, block_lin());
}

int nb2(const GeoB& g) {
  const dim3 d = grid2(g);
  return (int)(d.x * d.y * d.z);
}

template <typename TZ>
void run_cycle_b(Ctx& c, const GeoB& g, cudaStream_t s) {
  Level& L0 = c.L[0];
  const int m = c.opts.restart_m, R = g.R;
  const double invh2 = 1.0 / (c.h * c.h);
  KrylovState* st = c.ks;
  int* na = c.n_active;
  TZ* Z = (TZ*)c.Z;
  const int n2 = nb2(g), n1 = (int)grid1(g);
  const double tol = c.opts.tol;
  const int mi = c.opts.max_iter;
  const double NR = g.NR;
  for (int j = 0; j < m; ++j) {
    k_cast_in_b<TZ><<<nblk(g.NR, 256), 256, 0, s>>>(g, c.V + (long long)j * g.NR, st, j, (TZ*)L0.f, na);
    int pk = prof_begin(c, 3, j, vcycle_bytes(c), 0.0, s);
    vcycle(c, L0.f, Z + (long long)j * g.NR, na, s);
    prof_end(c, pk, s);
    // z (sizeof TZ), v_0 read, w written; diag once; 24 flops (A z: 16, dot: 8)
    pk = prof_begin(c, 2, j, NR * (sizeof(TZ) + 32) + 16.0 * g.N, 24.0 * NR, s);
    k_mgs_first_b<TZ><<<grid2(g), dim3(BX, BY), 0, s>>>(g, invh2, c.diagA64, Z + (long long)j * g.NR, c.V, j,
                                                         c.partials, st, na);
    prof_end(c, pk, s);
    k_reduce_b<<<R, kB, 0, s>>>(c.partials, n2, kH1, 0, st, na, tol, mi, m);
    for (int i = 1; i <= j; ++i) {
      // w, v_{i-1}, v_i read, w written; 8 flops update + 8 flops dot
      pk = prof_begin(c, 1, j, 64.0 * NR, 16.0 * NR, s);
      k_mgs_step_b<false><<<n1, kB, 0, s>>>(g, c.V, j, i, c.partials, st, na);
      prof_end(c, pk, s);
      k_reduce_b<<<R, kB, 0, s>>>(c.partials, n1, kH1, i, st, na, tol, mi, m);
    }
    // w, v_j read, w written; 8 flops update + 4 flops norm
    pk = prof_begin(c, 1, j, 48.0 * NR, 12.0 * NR, s);
    k_mgs_step_b<true><<<n1, kB, 0, s>>>(g, c.V, j, j + 1, c.partials, st, na);
    prof_end(c, pk, s);
    k_reduce_b<<<R, kB, 0, s>>>(c.partials, n1, kArnoldi, j, st, na, tol, mi, m);
  }
  HZ_LAUNCHED();
  k_solve_y_b<<<1, 64, 0, s>>>(st, R);
  k_update_p_b<TZ><<<nblk(g.NR, 256), 256, 0, s>>>(g, Z, st, c.p);
  k_true_residual_b<<<grid2(g), dim3(BX, BY), 0, s>>>(g, invh2, c.diagA64, c.p, c.qhat, c.V, c.partials, st);
  k_reduce_b<<<R, kB, 0, s>>>(c.partials, n2, kRestart, 0, st, na, tol, mi, m);
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
  const GeoB g = geob(c.L[0].g, R);
  c.nrhs = R;
  ensure_graph_b<TZ>(c, g);
  cudaStream_t s = c.graph_stream;
  KrylovState* st = c.ks;
  const int n1 = (int)grid1(g), n2 = nb2(g);
  const double invh2 = 1.0 / (c.h * c.h);
  HZ_CUDA(cudaEventRecord(c.ev_in, user));
  HZ_CUDA(cudaStreamWaitEvent(s, c.ev_in, 0));
  HZ_CUDA(cudaMemsetAsync(c.n_active, 0, sizeof(int), s));
  k_scale_rhs_b<<<n1, kB, 0, s>>>(g, c.wmass, q, c.qhat, c.partials);
  k_reduce_b<<<R, kB, 0, s>>>(c.partials, n1, kInit, 0, st, c.n_active, c.opts.tol, c.opts.max_iter,
                              c.opts.restart_m);
  HZ_CUDA(cudaMemsetAsync(c.p, 0, sizeof(double2) * g.NR, s));
  k_true_residual_b<<<grid2(g), dim3(BX, BY), 0, s>>>(g, invh2, c.diagA64, c.p, c.qhat, c.V, c.partials, st);
  k_reduce_b<<<R, kB, 0, s>>>(c.partials, n2, kRestart, 0, st, c.n_active, c.opts.tol, c.opts.max_iter,
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
  if (c.mixed) solve_b<float2>(c, q, p, nrhs, info, s);
  else solve_b<double2>(c, q, p, nrhs, info, s);
}

}  // namespace hz
