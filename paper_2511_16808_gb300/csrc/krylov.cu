// Flexible GMRES(m) in FP64 around the multigrid V-cycle (Section 2.3; m = 5
// in Section 5.2), right preconditioned, zero initial guess (Section 5).
//
// Per inner iteration j (one preconditioner application), two FP64 passes of
// classical Gram-Schmidt:
//   z'_j = V-cycle(f)      f = V_j cast to the working precision, V_j stored
//                          unnormalised with v_j = scale_j V_j, so z_j =
//                          scale_j z'_j (the cycle is linear); z'_j is stored
//                          in the working precision (the Arnoldi relation
//                          A Z = V H holds for the stored vectors)
//   pass A   w = A z'_j -> V_{j+1};  d_i = V_i^H w, i = 0..j (one sweep)
//   pass B   w -= sum_i scale_i^2 d_i V_i;  ||w||^2;  f = cast(w) for the
//            next cycle;  then (last block) H(i, j) = scale_j scale_i d_i,
//            H(j+1, j) = scale_j ||w||, complex Givens update of H and g,
//            residual estimate |g_{j+1}| / ||q_hat|| and the stop flag.
// Two passes and two reductions per iteration whatever j (modified
// Gram-Schmidt needs j + 2 dependent ones) with the same FP64 operation count;
// in FP64 with m = 5 the orthogonality lost by one classical pass stays at
// rounding level.  At the end of a cycle: y = H^{-1} g, p += sum y_i scale_i
// z'_i, true residual q_hat - A p in FP64 (also cast into f), restart.  One
// restart cycle is captured once as a CUDA graph and replayed; the host reads
// one small status record per cycle.  GB300's FP64 rate is 1/64 of FP32, so
// the passes are organised to minimise FP64 operations and launches.
//
// Reductions are two-stage and deterministic: each pass kernel writes one
// partial per block, a second kernel sums the partials in a fixed order.
#include <cstddef>
#include <map>
#include <mutex>
#include <type_traits>

#include "krylov_impl.cuh"

namespace hz {

namespace {

// Block sums of C double2 values per thread by a shared-memory tree (256 ->
// 32 values, then the shuffles of one warp).  The Krylov passes are bound by
// the FP64 pipe, and this takes 7 + 5 FP64 add steps per component against 5
// in every one of the 8 warps for a shuffle tree alone.  CPLX = false sums the
// real parts only.  The result is in v of thread 0 (all of warp 0).
template <int C, bool CPLX>
__device__ __forceinline__ void block_sums(double2 (&v)[C], double2 (&sm)[C][kRedBlock], int tid) {
#pragma unroll
  for (int c = 0; c < C; ++c) sm[c][tid] = v[c];
  __syncthreads();
#pragma unroll
  for (int k = kRedBlock / 2; k >= 32; k >>= 1) {
    if (tid < k) {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        sm[c][tid].x += sm[c][tid + k].x;
        if (CPLX) sm[c][tid].y += sm[c][tid + k].y;
      }
    }
    __syncthreads();
  }
  if (tid < 32) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
      double2 a = sm[c][tid];
      for (int o = 16; o > 0; o >>= 1) {
        a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
        if (CPLX) a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
      }
      v[c] = a;
    }
  }
}

// Block-reduce the real accumulator of each thread; thread 0 writes partials[block].
__device__ __forceinline__ void block_store(double2 acc, double2* __restrict__ partials, int block) {
  __shared__ double2 sm[1][kRedBlock];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  double2 v[1] = {make_double2(acc.x, 0.0)};
  block_sums<1, false>(v, sm, tid);
  if (tid == 0) partials[block] = make_double2(v[0].x, 0.0);
}

// Two-stage deterministic reduction finished by the last block to arrive:
// every block stores its partial, the last one sums all partials in index
// order into *out and returns true (in all its threads).
__device__ __forceinline__ bool reduce_last(double2 acc, double2* __restrict__ partials, int nb, int block,
                                            unsigned* counter, double2* out) {
  block_store(acc, partials, block);
  __threadfence();
  __syncthreads();
  __shared__ int is_last;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if (tid == 0) is_last = atomicAdd(counter, 1u) == (unsigned)(nb - 1);
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  __shared__ double2 red[1][kRedBlock];
  double s = 0.0;
  int b = tid;
  for (; b + 3 * kRedBlock < nb; b += 4 * kRedBlock) {
    const double a0 = __ldcg(partials + b).x, a1 = __ldcg(partials + b + kRedBlock).x;
    const double a2 = __ldcg(partials + b + 2 * kRedBlock).x, a3 = __ldcg(partials + b + 3 * kRedBlock).x;
    s = s + ((a0 + a1) + (a2 + a3));
  }
  for (; b < nb; b += kRedBlock) s = s + __ldcg(partials + b).x;
  double2 v[1] = {make_double2(s, 0.0)};
  block_sums<1, false>(v, red, tid);
  if (tid == 0) {
    *out = make_double2(v[0].x, 0.0);
    *counter = 0u;
  }
  return true;
}



// Per-block partials of NV complex accumulators (block_sums, up to 4 vectors
// per round), then (last block to arrive) NV deterministic sums: warp w sums
// vectors w, w+8, ... over the blocks in index order.  Returns true in the
// last block.
template <int NV>
__device__ __forceinline__ bool reduce_last_multi(const double2 (&acc)[NV], double2* __restrict__ partials, int nb,
                                                  int block, unsigned* counter, double2* out) {
  constexpr int CH = NV < 4 ? NV : 4;            // vectors per shared-memory round
  __shared__ double2 sm[CH][kRedBlock];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
#pragma unroll
  for (int i0 = 0; i0 < NV; i0 += CH) {
    double2 v[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) v[c] = i0 + c < NV ? acc[i0 + c < NV ? i0 + c : NV - 1] : make_double2(0, 0);
    block_sums<CH, true>(v, sm, tid);
    if (tid == 0) {
#pragma unroll
      for (int c = 0; c < CH; ++c)
        if (i0 + c < NV) partials[(i0 + c) * nb + block] = v[c];
    }
    __syncthreads();                               // sm is restaged by the next round
  }
  __threadfence();
  __syncthreads();
  __shared__ int is_last;
  if (tid == 0) is_last = atomicAdd(counter, 1u) == (unsigned)(nb - 1);
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  // thread t sums partials t, t + kRedBlock, ... of each vector (four blocks'
  // loads issued before their adds, which keep the index order), then the
  // block sums the threads' values in a fixed tree: deterministic
#pragma unroll
  for (int i0 = 0; i0 < NV; i0 += CH) {
    double2 v[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) v[c] = make_double2(0, 0);
    int b = tid;
    for (; b + 3 * kRedBlock < nb; b += 4 * kRedBlock) {
      double2 q[CH][4];
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int u = 0; u < 4; ++u)
          q[c][u] = i0 + c < NV ? __ldcg(partials + (long long)(i0 + c) * nb + b + u * kRedBlock) : make_double2(0, 0);
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int u = 0; u < 4; ++u) v[c] = v[c] + q[c][u];
    }
    for (; b < nb; b += kRedBlock) {
#pragma unroll
      for (int c = 0; c < CH; ++c)
        if (i0 + c < NV) v[c] = v[c] + __ldcg(partials + (long long)(i0 + c) * nb + b);
    }
    block_sums<CH, true>(v, sm, tid);
    if (tid == 0) {
#pragma unroll
      for (int c = 0; c < CH; ++c)
        if (i0 + c < NV) out[i0 + c] = v[c];
    }
    __syncthreads();                               // sm is restaged by the next round
  }
  if (tid == 0) *counter = 0u;
  return true;
}

// Persistent stride over the tiles (32 x 8 threads, one node each, one z
// plane per tile): f(p, x, y, z) for every node of the block's tiles.
template <typename F>
__device__ __forceinline__ void for_tiles(const Geo& g, F&& f) {
  const int tnx = (g.nx + BX - 1) / BX, tny = (g.ny + BY - 1) / BY;
  const int tiles = tnx * tny * g.nz;
  for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int tz = t / (tnx * tny), r = t - tz * (tnx * tny);
    const int tyi = r / tnx, txi = r - tyi * tnx;
    const int x = txi * BX + threadIdx.x, y = tyi * BY + threadIdx.y;
    if (x < g.nx && y < g.ny) f((tz * g.ny + y) * g.nx + x, x, y, tz);
  }
}

// Contiguous, equal share [b0, b1) of N elements for this block of a
// persistent 1D pass.
__device__ __forceinline__ void block_range(int N, int& b0, int& b1) {
  const long long per = ((long long)N + gridDim.x - 1) / gridDim.x;
  b0 = (int)std::min<long long>((long long)blockIdx.x * per, N);
  b1 = (int)std::min<long long>(b0 + per, N);
}

// pass A: w = A z'_j (w = V[j+1]); d_i = conj(V_i) . w for i < NV (the first
// chunk of the j + 1 inner products, all of them when j < kMaxNV)
template <typename TZ, int NV>
__global__ void __launch_bounds__(kRedBlock) k_gs_dots(Geo g, double invh2, const double2* __restrict__ diag,
                                                       const TZ* __restrict__ z, const double2* __restrict__ V,
                                                       double2* __restrict__ w, double2* __restrict__ partials,
                                                       KrylovState* st) {
  pdl_enter();
  if (!st->active) return;
  double2 acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = make_double2(0, 0);
  for_tiles(g, [&](int p, int x, int y, int zz) {
    const double2 a = apply_A(g, invh2, diag, z, p, x, y, zz);
    w[p] = a;
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = dot_acc(acc[i], V[HZ_AT((long long)i * g.N + p, (long long)NV * g.N)], a);
  });
  reduce_last_multi<NV>(acc, partials, gridDim.x, blockIdx.x, &st->counter, st->h1);
}

// pass A, further chunks: d_{base+i} = conj(V_{base+i}) . w for i < NV
template <int NV>
__global__ void __launch_bounds__(kRedBlock) k_gs_dots_more(int N, const double2* __restrict__ Vb,
                                                            const double2* __restrict__ w,
                                                            double2* __restrict__ partials, KrylovState* st,
                                                            int base) {
  pdl_enter();
  if (!st->active) return;
  double2 acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = make_double2(0, 0);
  int b0, b1;
  block_range(N, b0, b1);
  for (int p = b0 + threadIdx.x; p < b1; p += kRedBlock) {
    const double2 a = w[p];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = dot_acc(acc[i], Vb[HZ_AT((long long)i * N + p, (long long)NV * N)], a);
  }
  reduce_last_multi<NV>(acc, partials, gridDim.x, blockIdx.x, &st->counter, st->h1 + base);
}

// pass B: w -= sum_{i < NV} scale_{base+i}^2 d_{base+i} V_{base+i}.  The last
// chunk also forms ||w||^2 and f = w in the working precision, then (last
// block) the Arnoldi column j.
template <typename TF, int NV, bool LAST>
__global__ void __launch_bounds__(kRedBlock) k_gs_update(int N, const double2* __restrict__ Vb,
                                                         double2* __restrict__ w, TF* __restrict__ f,
                                                         double2* __restrict__ partials, KrylovState* st, int base,
                                                         int j) {
  pdl_enter();
  if (!st->active) return;
  double2 c[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const double s = st->scale[base + i];
    c[i] = (s * s) * st->h1[base + i];
  }
  double acc = 0.0;
  int b0, b1;
  block_range(N, b0, b1);
  for (int p = b0 + threadIdx.x; p < b1; p += kRedBlock) {
    double2 ww = w[p];
#pragma unroll
    for (int i = 0; i < NV; ++i) ww = axmy(ww, c[i], Vb[HZ_AT((long long)i * N + p, (long long)NV * N)]);
    w[HZ_AT(p, N)] = ww;
    if constexpr (LAST) {
      if constexpr (std::is_same<TF, float2>::value) f[p] = make_float2(d2f_rn(ww.x), d2f_rn(ww.y));
      else f[p] = ww;
      acc = nrm_acc(acc, ww);
    }
  }
  if constexpr (LAST) {
    const bool last = reduce_last(make_double2(acc, 0.0), partials, gridDim.x, blockIdx.x, &st->counter, &st->nrm2);
    if (last) arnoldi_update_staged(st, j, st->scale[j]);
  }
}


// y = H^{-1} g (upper triangular, k columns of the cycle) and the update
// coefficients c_i = scale_i y_i.  For cycles of up to kSolveYStage columns
// the block stages H, g and the scales in shared memory first, so the one
// thread that runs the back substitution reads on-chip values; longer cycles
// read them from global memory.  The same operations in the same order.
constexpr int kSolveYThreads = 128, kSolveYStage = 32;
__global__ void __launch_bounds__(kSolveYThreads) k_solve_y(KrylovState* __restrict__ st) {
  __shared__ double2 hs[kSolveYStage][kSolveYStage + 1];
  __shared__ double2 gs[kSolveYStage], ys[kSolveYStage];
  __shared__ double sc[kSolveYStage];
  pdl_enter();
  if (st->st.done) return;
  const int k = st->kcyc;
  if (k > kSolveYStage) {
    if (threadIdx.x != 0) return;
    for (int i = k - 1; i >= 0; --i) {
      double2 acc = st->g[i];
      for (int l = i + 1; l < k; ++l) acc = acc - cmul(st->H[i][l], st->y[l]);
      st->y[i] = cdiv(acc, st->H[i][i]);
      st->c[i] = st->scale[i] * st->y[i];
    }
    return;
  }
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int i = e / k, l = e - i * k;
    if (l >= i) hs[i][l] = st->H[i][l];
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    gs[i] = st->g[i];
    sc[i] = st->scale[i];
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double2 acc = gs[i];
    for (int l = i + 1; l < k; ++l) acc = acc - cmul(hs[i][l], ys[l]);
    ys[i] = cdiv(acc, hs[i][i]);
    st->y[i] = ys[i];
    st->c[i] = sc[i] * ys[i];                     // once here instead of at every node
  }
}

template <typename TZ>
__global__ void k_update_p(int N, const TZ* __restrict__ Z, const KrylovState* __restrict__ st,
                           double2* __restrict__ p) {
  pdl_enter();
  if (st->st.done) return;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N) return;
  const int k = st->kcyc;
  double2 acc = p[q];
  for (int i = 0; i < k; ++i) {
    const double2 yi = st->c[i], zi = ld64(Z, i * N + q);
    acc = make_double2(fma(yi.x, zi.x, fma(-yi.y, zi.y, acc.x)), fma(yi.x, zi.y, fma(yi.y, zi.x, acc.y)));
  }
  p[q] = acc;
}


// r = q_hat - A p -> V_0 and f (working precision, the next cycle's first
// V-cycle input); ||r||^2, then (last block) the restart decision
template <typename TF>
__global__ void __launch_bounds__(kRedBlock) k_true_residual(Geo g, double invh2, const double2* __restrict__ diag,
                                                             const double2* __restrict__ p,
                                                             const double2* __restrict__ qhat, double2* __restrict__ r,
                                                             TF* __restrict__ f, double2* __restrict__ partials,
                                                             KrylovState* st) {
  pdl_enter();
  if (st->st.done) return;
  double2 acc = make_double2(0, 0);
  for_tiles(g, [&](int q, int x, int y, int zz) {
    const double2 v = qhat[q] - apply_A(g, invh2, diag, p, q, x, y, zz);
    r[q] = v;
    if constexpr (std::is_same<TF, float2>::value) f[q] = make_float2(d2f_rn(v.x), d2f_rn(v.y));
    else f[q] = v;
    acc.x = nrm_acc(acc.x, v);
  });
  const bool last = reduce_last(acc, partials, gridDim.x, blockIdx.x, &st->counter, &st->nrm2);
  if (last && threadIdx.x == 0 && threadIdx.y == 0) restart_update(st);
}

// q_hat = wmass * q; ||q_hat||^2, then (last block) the solver state
// (compact stencil: q_hat = M q with the compact mass stencil, neighbours
// outside the grid dropped)
__global__ void __launch_bounds__(kRedBlock) k_scale_rhs(Geo g, const double* __restrict__ wmass,
                                                         const double2* __restrict__ q, double2* __restrict__ qhat,
                                                         double2* __restrict__ partials, KrylovState* st, double tol,
                                                         int max_iter, int m) {
  pdl_enter();
  double2 acc = make_double2(0, 0);
  const int N = g.N;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < N) {
    double2 v;
    if (g.compact) {
      const int x = p % g.nx, t = p / g.nx, y = t % g.ny, z = t / g.ny;
      v = make_double2(0, 0);
      const int zr = g.dim == 3 ? 1 : 0;
      for (int dz = -zr; dz <= zr; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const int mm = (dx != 0) + (dy != 0) + (dz != 0);
            const double cm = compact_M(g.dim, mm);
            if (cm == 0.0) continue;
            const int xx = x + dx, yy = y + dy, zz = z + dz;
            if (xx < 0 || xx >= g.nx || yy < 0 || yy >= g.ny || zz < 0 || zz >= g.nz) continue;
            const double2 qq = q[p + dx + dy * g.nx + dz * g.sxy];
            v.x = fma(cm, qq.x, v.x);
            v.y = fma(cm, qq.y, v.y);
          }
    } else {
      v = wmass[p] * q[p];
    }
    qhat[p] = v;
    acc.x = cabs2(v);
  }
  const bool last = reduce_last(acc, partials, gridDim.x, blockIdx.x, &st->counter, &st->nrm2);
  if (last && threadIdx.x == 0) {
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
}

template <typename V>
__global__ void k_cast_vec(int N, const double2* __restrict__ in, V* __restrict__ out) {
  pdl_enter();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < N) out[p] = from_c128<V>(in[p]);
}
template <typename V>
__global__ void k_widen_vec(int N, const V* __restrict__ in, double2* __restrict__ out) {
  pdl_enter();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < N) out[p] = ld64(in, p);
}

// One restart cycle: m inner iterations (skipped on the device once stopped),
// the solution update and the true residual; solution accumulates in c.p.
template <typename TZ>
void run_cycle(Ctx& c, cudaStream_t s) {
  Level& L0 = c.L[0];
  const Geo g = geo(L0.g, c.compact, 1.0 / (c.h * c.h));
  const int N = g.N;
  const int m = c.opts.restart_m;
  const double invh2 = 1.0 / (c.h * c.h);
  KrylovState* st = c.ks;
  const int* active = &st->active;
  TZ* Z = (TZ*)c.Z;
  for (int j = 0; j < m; ++j) {
    const int nv = j + 1;
    int pk = prof_begin(c, 3, j, vcycle_bytes(c), 0.0, s);
    vcycle(c, L0.f, Z + (long long)j * N, active, s);
    prof_end(c, pk, s);
    // pass A: z (b) and diag read, w written, nv vectors read; A z 16 flops
    // (2D; 20 in 3D: two more neighbour sums) + 8 per dot
    pk = prof_begin(c, 2, j, (double)N * (sizeof(TZ) + 32 + 16.0 * nv), ((g.dim == 3 ? 20.0 : 16.0) + 8.0 * nv) * N, s);
    double2* w = c.V + (long long)nv * N;
    // more than kMaxNV inner products (restarts longer than 16) run in chunks
    for (int b = 0; b < nv; b += kMaxNV) {
      with_nv(std::min(kMaxNV, nv - b), [&](auto NV) {
        if (b == 0) {
          auto kern = k_gs_dots<TZ, decltype(NV)::value>;
          const unsigned G = (unsigned)std::min<long long>(tiles_xy(g), resident_slots((const void*)kern, kRedBlock));
          launch_pdl(kern, G, dim3(BX, BY), s, g, invh2, c.diagA64, Z + (long long)j * N, (const double2*)c.V, w,
                     c.partials, st);
        } else {
          auto kern = k_gs_dots_more<decltype(NV)::value>;
          const unsigned G = (unsigned)std::min<long long>(grid_1d(N), resident_slots((const void*)kern, kRedBlock));
          launch_pdl(kern, G, kRedBlock, s, N, (const double2*)(c.V + (long long)b * N), (const double2*)w,
                     c.partials, st, b);
        }
      });
    }
    prof_end(c, pk, s);
    // pass B: w and nv vectors read, w and f written; 8 flops per vector + 4 for the norm
    pk = prof_begin(c, 1, j, (double)N * (32 + 16.0 * nv + sizeof(TZ)), (8.0 * nv + 4.0) * N, s);
    for (int b = 0; b < nv; b += kMaxNV) {
      const int cnt = std::min(kMaxNV, nv - b);
      with_nv(cnt, [&](auto NV) {
        auto go = [&](auto kern) {
          const unsigned G = (unsigned)std::min<long long>(grid_1d(N), resident_slots((const void*)kern, kRedBlock));
          launch_pdl(kern, G, kRedBlock, s, N, (const double2*)(c.V + (long long)b * N), w, (TZ*)L0.f, c.partials,
                     st, b, j);
        };
        if (b + cnt >= nv) go(k_gs_update<TZ, decltype(NV)::value, true>);
        else go(k_gs_update<TZ, decltype(NV)::value, false>);
      });
    }
    prof_end(c, pk, s);
  }
  HZ_LAUNCHED();
  launch_pdl(k_solve_y, 1, kSolveYThreads, s, st);
  launch_pdl(k_update_p<TZ>, nblk(N, 256), 256, s, N, Z, st, c.p);
  {
    auto kern = k_true_residual<TZ>;
    const unsigned G = (unsigned)std::min<long long>(tiles_xy(g), resident_slots((const void*)kern, kRedBlock));
    launch_pdl(kern, G, dim3(BX, BY), s, g, invh2, c.diagA64, c.p, c.qhat, c.V, (TZ*)L0.f, c.partials, st);
  }
  HZ_LAUNCHED();
}

template <typename TZ>
void ensure_graph(Ctx& c) {
  if (c.cycle_graph) return;
  // the two captured cycles share the event list: one profiled graph at a time
  if (c.prof_class && c.batch_graph) {
    cudaGraphExecDestroy(c.batch_graph);
    c.batch_graph = nullptr;
  }
  c.prof_j.clear();
  c.prof_b.clear();
  c.prof_f.clear();
  cudaGraph_t graph = nullptr;
  HZ_CUDA(cudaStreamBeginCapture(c.graph_stream, cudaStreamCaptureModeThreadLocal));
  try {
    run_cycle<TZ>(c, c.graph_stream);
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
  c.graph_kernels = 0;
  for (auto n : nodes) {
    cudaGraphNodeType t;
    HZ_CUDA(cudaGraphNodeGetType(n, &t));
    if (t == cudaGraphNodeTypeKernel) ++c.graph_kernels;
  }
  const cudaError_t e = cudaGraphInstantiate(&c.cycle_graph, graph, 0);
  cudaGraphDestroy(graph);
  HZ_CUDA(e);
}

// Asynchronous single-RHS solve: begin queues the start-up work, each step
// reads the status of the last restart cycle (once its event has completed)
// and queues the next cycle, end hands out the solution.  The blocking solve
// and the serving loop are both built from these.
// Queues one restart cycle (the captured graph) and the copy of its status
// into the next free slot.  A cycle queued after the solve has stopped does
// nothing: every kernel of the cycle returns at once once the device state
// says done (the V-cycle and the passes test `active`, the per-restart
// kernels `done`).
void queue_cycle(Ctx& c) {
  const int slot = (c.as_head + c.as_pending) & 1;
  cudaStream_t s = c.graph_stream;
  NvtxRange range("hz restart cycle");
  HZ_CUDA(cudaGraphLaunch(c.cycle_graph, s));
  c.as_replayed = true;
  c.launches += c.graph_kernels;
  HZ_CUDA(cudaMemcpyAsync((KrylovStatus*)c.ks_host + slot, &c.ks->st, sizeof(KrylovStatus), cudaMemcpyDeviceToHost,
                          s));
  HZ_CUDA(cudaEventRecord(slot ? c.ev_status_b : c.ev_status, s));
  ++c.as_pending;
}

template <typename TZ>
void solve_begin_t(Ctx& c, const double2* q, cudaStream_t user) {
  Level& L0 = c.L[0];
  const Geo g = geo(L0.g, c.compact, 1.0 / (c.h * c.h));
  const int N = g.N;
  const double invh2 = 1.0 / (c.h * c.h);
  KrylovState* st = c.ks;
  KrylovStatus* hs = (KrylovStatus*)c.ks_host;
  c.nrhs = 1;
  ensure_graph<TZ>(c);
  // the work runs on the library's stream, ordered after the caller's stream
  cudaStream_t s = c.graph_stream;
  HZ_CUDA(cudaEventRecord(c.ev_in, user));
  HZ_CUDA(cudaStreamWaitEvent(s, c.ev_in, 0));
  HZ_CUDA(cudaMemsetAsync(&st->counter, 0, sizeof(unsigned), s));
  launch_pdl(k_scale_rhs, nblk(N, kRedBlock), kRedBlock, s, g, c.wmass, q, c.qhat, c.partials, st, c.opts.tol,
                                                       c.opts.max_iter, c.opts.restart_m);
  HZ_CUDA(cudaMemsetAsync(c.p, 0, sizeof(double2) * N, s));
  {
    auto kern = k_true_residual<TZ>;
    const unsigned G = (unsigned)std::min<long long>(tiles_xy(g), resident_slots((const void*)kern, kRedBlock));
    launch_pdl(kern, G, dim3(BX, BY), s, g, invh2, c.diagA64, c.p, c.qhat, c.V, (TZ*)c.L[0].f, c.partials, st);
  }
  HZ_LAUNCHED();
  c.launches += 2;
  HZ_CUDA(cudaMemcpyAsync(hs, &st->st, sizeof(KrylovStatus), cudaMemcpyDeviceToHost, s));
  HZ_CUDA(cudaEventRecord(c.ev_status, s));
  {
    std::lock_guard<std::mutex> lk(c.history_mu);
    c.history.clear();
  }
  c.as_before = 0;
  c.as_replayed = false;
  c.as_head = 0;
  c.as_pending = 1;
  c.as_state = 1;
  if (!c.prof_class) queue_cycle(c);   // the first cycle, before the initial status is read
}

}  // namespace

// Reads the oldest queued status; unless the solve has stopped, keeps two
// restart cycles queued (one while profiling, whose events are rewritten by
// every replay), so the device goes on with the next cycle while the host
// reads the status of the previous one.
int solve_step(Ctx& c, bool block) {
  if (c.as_state != 1) return 1;
  const int k = c.as_head;
  cudaEvent_t ev = k ? c.ev_status_b : c.ev_status;
  if (block) {
    HZ_CUDA(cudaEventSynchronize(ev));
  } else {
    const cudaError_t e = cudaEventQuery(ev);
    if (e == cudaErrorNotReady) return 0;
    HZ_CUDA(e);
  }
  const KrylovStatus* hs = (const KrylovStatus*)c.ks_host + k;
  if (c.as_replayed && c.prof_class) prof_collect(c, hs->iters - c.as_before, nullptr, 1);
  {
    std::lock_guard<std::mutex> lk(c.history_mu);
    c.history.push_back({(double)hs->iters, hs->relres_true, hs->relres_est});
  }
  c.as_head ^= 1;
  --c.as_pending;
  if (hs->done) {
    c.as_done_slot = k;
    c.as_state = 2;
    return 1;
  }
  c.as_before = hs->iters;
  const int depth = c.prof_class ? 1 : 2;
  while (c.as_pending < depth) queue_cycle(c);
  return 0;
}

void solve_begin(Ctx& c, const double2* q, cudaStream_t user) {
  require(c.as_state != 1, "an asynchronous solve is already in flight on this context");
  if (c.mixed) solve_begin_t<float2>(c, q, user);
  else solve_begin_t<double2>(c, q, user);
}

void solve_end(Ctx& c, double2* p, hz_info* info, cudaStream_t user) {
  require(c.as_state == 2, "the solve has not finished");
  const int N = (int)c.L[0].g.N;
  cudaStream_t s = c.graph_stream;
  if (p != c.p) HZ_CUDA(cudaMemcpyAsync(p, c.p, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s));
  HZ_CUDA(cudaEventRecord(c.ev_out, s));
  HZ_CUDA(cudaStreamWaitEvent(user, c.ev_out, 0));
  const KrylovStatus* hs = (const KrylovStatus*)c.ks_host + c.as_done_slot;
  info->iters = hs->iters;
  info->converged = hs->converged;
  info->relres_est = hs->relres_est;
  info->relres_true = hs->relres_true;
  c.as_state = 0;
}

namespace {

}  // namespace

int max_slots() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  (void)cudaGetLastError();
  return std::max(1, sms) * 8;
}

int resident_slots(const void* kernel, int threads) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> cache;
  int dev = 0;
  HZ_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_pair(kernel, dev * 4096 + threads);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int per_sm = 0, sms = 0;
  HZ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0));
  HZ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int slots = std::max(1, std::min(per_sm, 2048 / threads)) * sms;
  cache[key] = slots;
  return slots;
}

// ---- measurement hooks: events around the launches of the selected class
// (1 = Gram-Schmidt update passes, 2 = the pass with the FP64 operator and the
// inner products, 3 = whole V-cycle preconditioner application)
int prof_begin(Ctx& c, int cls, int j, double bytes, double flops, cudaStream_t s) {
  if (c.prof_class != cls) return -1;
  const int k = (int)c.prof_j.size();
  if ((int)c.prof_ev.size() < 2 * (k + 1)) {
    cudaEvent_t a, b;
    HZ_CUDA(cudaEventCreate(&a));
    HZ_CUDA(cudaEventCreate(&b));
    c.prof_ev.push_back(a);
    c.prof_ev.push_back(b);
  }
  c.prof_j.push_back(j);
  c.prof_b.push_back(bytes);
  c.prof_f.push_back(flops);
  HZ_CUDA(cudaEventRecordWithFlags(c.prof_ev[2 * k], s, cudaEventRecordExternal));
  return k;
}
void prof_end(Ctx& c, int k, cudaStream_t s) {
  if (k >= 0) HZ_CUDA(cudaEventRecordWithFlags(c.prof_ev[2 * k + 1], s, cudaEventRecordExternal));
}
// After a replayed cycle in which `ran` inner iterations did work.  Batched
// (ran_r: the inner iterations each of the R right-hand sides did): a bracketed
// launch of inner iteration j counts the bytes / flops of the right-hand sides
// still active there (prof_b / prof_f hold the all-active figures).
void prof_collect(Ctx& c, int ran, const int* ran_r, int R) {
  for (size_t k = 0; k < c.prof_j.size(); ++k) {
    if (c.prof_j[k] >= ran) continue;
    double frac = 1.0;
    if (ran_r) {
      int act = 0;
      for (int r = 0; r < R; ++r) act += ran_r[r] > c.prof_j[k];
      frac = (double)act / R;
    }
    float ms = 0.f;
    HZ_CUDA(cudaEventElapsedTime(&ms, c.prof_ev[2 * k], c.prof_ev[2 * k + 1]));
    c.prof_ms += ms;
    c.prof_bytes += frac * c.prof_b[k];
    c.prof_flops += frac * c.prof_f[k];
    c.prof_launches += 1;
  }
}

// Algorithmic (compulsory) bytes of one V-cycle with the kernels of
// cycle_impl.cuh.  Single right-hand side: the fused 2D kernels' reads and
// writes.  R > 1 right-hand sides: per level the field traffic of V(1,1)
// (pre-smooth f -> u, residual, restriction, prolongation-add, residual,
// post-smooth: 14 + 2 rc field passes, rc the coarse/fine node ratio) times R,
// plus the stencil planes of A and M read twice each, shared by all R.
double vcycle_bytes(const Ctx& c) {
  const double b = c.mixed ? 8.0 : 16.0;
  const double R = c.nrhs;
  double tot = 0;
  // visits of each level per cycle: 1 for a V-cycle; a W-cycle visits level
  // l >= 1 twice per visit of level l-1 (the coarsest once per visit of its
  // parent).  Every visit is counted like a first one (zero initial guess).
  double vis = 1.0;
  const double per = std::max(1, c.opts.cycle_visits);
  for (size_t l = 0; l < c.L.size(); ++l) {
    const Level& L = c.L[l];
    const double N = (double)L.g.N;
    const double t0 = tot;
    if (l > 0 && !L.coarsest) vis *= per;
    if (L.coarsest) {
      tot += vis * (N * N * b + 2 * N * b * R);
      continue;
    }
    // stored smoother planes: the diagonal, or the half / full planes (+ a real weight per node)
    const double sMst = L.m_diag ? 1.0 : L.Mh.off.n + (L.wcw ? 0.5 : 0.0);
    if (c.nrhs > 1) {
      const double sA = L.fine ? 1.0 : (L.a_half ? (L.A.off.n + 1) / 2 : L.A.off.n), sM = sMst;
      const double rc = L.g.dim == 3 ? 0.125 : 0.25;
      tot += N * b * R * (14 + 2 * rc) + N * b * 2 * (sA + sM);
    } else {
      const double sA = L.fine ? 1.0 : (L.a_half ? (L.A.off.n + 1) / 2 : L.A.off.n), sM = sMst;
      const double rc = L.g.dim == 3 ? 0.125 : 0.25;
      if (fine_two_pass(c, (int)l)) tot += N * b * (7 + 2 * rc);   // f, m0, A twice, out; coarse
      else if (L.m_diag) tot += N * b * (5 + (1 + rc) + (5 + rc)) + (sA - 1) * 2 * N * b;   // sweep0+resid, restrict, prolong+sweep
      else if (level_two_pass_2d(c, (int)l)) tot += N * b * (5 + 2 * rc) + 2 * (sA + sM) * N * b;   // fused tiles
      else tot += N * b * (2 * sM + 2 * sA + 13 + 2 * rc);
    }
    tot = t0 + vis * (tot - t0);
  }
  return tot;
}

size_t krylov_bytes(const hz_grid& g, const hz_opts& o) {
  long long N = (long long)g.n[0] * g.n[1] * (g.dim == 3 ? g.n[2] : 1);
  const size_t vb = o.precision == HZ_PREC_MIXED ? 8 : 16;
  const int m = o.restart_m;
  const long long R = std::max(1, o.nrhs_max);
  const long long nb = nblk(N * R, kRedBlock) * 2 * R + (long long)m * (nblk(N, BX * BY * kRows) + 2048) +
                       (R > 1 ? (long long)m * R * 2048 : 0);
  size_t tc = 0;                 // partial sums of the tensor-core coarsest solve (mixed, R >= 16)
  if (o.precision == HZ_PREC_MIXED && R >= 16) {
    long long nc = 1;
    for (int a = 0; a < g.dim; ++a) nc *= (g.n[a] - 1) / (1 << (o.levels - 1)) + 1;
    tc = coarse_tc_bytes(nc, (int)R);
  }
  return (16ull * N * (m + 1) + vb * N * m + 16ull * N * 4) * R + 16ull * nb + sizeof(KrylovState) * R + tc;
}

void krylov_alloc(Ctx& c) {
  const long long N = c.L[0].g.N;
  const int m = c.opts.restart_m;
  const long long R = std::max(1, c.opts.nrhs_max);
  const size_t vb = c.mixed ? sizeof(float2) : sizeof(double2);
  require(m >= 1 && m <= kMaxM, "restart_m must be in 1..128");
  require(R == 1 || m <= kMaxNV, "restart_m must be in 1..16 with several right-hand sides");
  require(N * R * (m + 1) < (1ll << 31), "grid too large for 32-bit Krylov indexing");
  c.V = (double2*)ctx_alloc(c, sizeof(double2) * N * R * (m + 1));
  c.Z = ctx_alloc(c, vb * N * R * m);
  c.qhat = (double2*)ctx_alloc(c, sizeof(double2) * N * R);
  c.p = (double2*)ctx_alloc(c, sizeof(double2) * N * R);
  const Geo g = geo(c.L[0].g);
  // single RHS: the operator pass keeps up to m partials per block (one per
  // inner product), the 1D passes one per block; batched: one per block and
  // RHS (blocks of at least 8 values per thread, see krylov_batch.cu)
  const long long nb1 = std::max<long long>((long long)max_slots() * m, nblk(N, kRedBlock));
  const long long nbR = R > 1 ? std::max<long long>(R * nblk(N * R, kRedBlock * 8), (long long)m * R * max_slots()) : 0;
  c.partials = (double2*)ctx_alloc(c, sizeof(double2) * std::max(nb1, nbR));
  c.ks = (KrylovState*)ctx_alloc(c, sizeof(KrylovState) * R);
  HZ_CUDA(cudaMemsetAsync(c.ks, 0, sizeof(KrylovState) * R, c.alloc_stream));
  c.n_active = (int*)ctx_alloc(c, sizeof(int));
  coarse_tc_alloc(c);
  c.ks_host = pinned_small_alloc(sizeof(KrylovStatus) * std::max<long long>(R, 2));   // >= 2 status slots
  HZ_CUDA(cudaStreamCreateWithFlags(&c.graph_stream, cudaStreamNonBlocking));
  HZ_CUDA(cudaEventCreateWithFlags(&c.ev_in, cudaEventDisableTiming));
  HZ_CUDA(cudaEventCreateWithFlags(&c.ev_out, cudaEventDisableTiming));
  HZ_CUDA(cudaEventCreateWithFlags(&c.ev_status, cudaEventDisableTiming));
  HZ_CUDA(cudaEventCreateWithFlags(&c.ev_status_b, cudaEventDisableTiming));
}

void profile_select(Ctx& c, int cls) {
  if (c.cycle_graph) cudaGraphExecDestroy(c.cycle_graph);
  c.cycle_graph = nullptr;
  if (c.batch_graph) cudaGraphExecDestroy(c.batch_graph);
  c.batch_graph = nullptr;
  c.prof_class = cls;
  c.prof_ms = c.prof_bytes = c.prof_flops = 0;
  c.prof_launches = 0;
}

void fgmres_solve(Ctx& c, const double2* q, double2* p, hz_info* info, cudaStream_t s) {
  NvtxRange range("hz solve");
  solve_begin(c, q, s);
  while (!solve_step(c, true)) {
  }
  solve_end(c, p, info, s);
}

void precond_apply_c128(Ctx& c, const double2* r, double2* z, int nrhs, cudaStream_t s) {
  Level& L0 = c.L[0];
  const int NR = (int)L0.g.N * nrhs;
  c.nrhs = nrhs;
  if (c.mixed) {
    launch_pdl(k_cast_vec<float2>, nblk(NR, 256), 256, s, NR, r, (float2*)L0.f);
    vcycle(c, L0.f, L0.u, nullptr, s);
    launch_pdl(k_widen_vec<float2>, nblk(NR, 256), 256, s, NR, (const float2*)L0.u, z);
  } else {
    HZ_CUDA(cudaMemcpyAsync(L0.f, r, sizeof(double2) * NR, cudaMemcpyDeviceToDevice, s));
    vcycle(c, L0.f, L0.u, nullptr, s);
    HZ_CUDA(cudaMemcpyAsync(z, L0.u, sizeof(double2) * NR, cudaMemcpyDeviceToDevice, s));
  }
  HZ_LAUNCHED();
  c.nrhs = 1;
}

}  // namespace hz
