// Autotuner of the V-cycle's kernel choices for one context and batch width.
// No counterpart in the paper: the choices change how a step runs, never what
// it computes.  Each knob is timed on the context's own level vectors (a few
// repetitions between CUDA events on a private stream after one untimed run),
// every candidate is reported, and the fastest is kept on the level:
//   kind 0  coarsest product for R right-hand sides: CUDA-core GEMM (0) or the
//           tcgen05 tensor-core GEMM with K split s ways (s = 1, 2, 4, 8, 16)
//   kind 1  RHS pack of a level's kernels (R >= 4): one value per thread (1) or
//           packs of 32 bytes (2); timed on one residual + one Vanka sweep
//   kind 2  one-RHS register budget of a level's kernels: full occupancy (0) or
//           two blocks per SM (2); timed on one residual + one Vanka sweep
//   kind 3  a small 2D level as the two fused tile passes (1) or as the five
//           separate kernels (0); timed on one down and one up pass
// Captured restart-cycle graphs are dropped, so the next solve captures the
// chosen kernels.
#include <vector>

#include "cycle_inst.cuh"

namespace hz {
namespace cyc {
HZ_CYC_ALL(extern, float)
HZ_CYC_ALL(extern, double)
}  // namespace cyc

namespace {

using namespace cyc;

struct Timer {
  cudaStream_t s;
  cudaEvent_t e0, e1;
  explicit Timer(cudaStream_t st) : s(st) {
    HZ_CUDA(cudaEventCreate(&e0));
    HZ_CUDA(cudaEventCreate(&e1));
  }
  ~Timer() {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  // microseconds per repetition of f, after one untimed run
  template <typename F>
  double us(int reps, F&& f) {
    f();
    HZ_CUDA(cudaEventRecord(e0, s));
    for (int i = 0; i < reps; ++i) f();
    HZ_CUDA(cudaEventRecord(e1, s));
    HZ_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    HZ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    return 1e3 * ms / reps;
  }
};

void drop_graphs(Ctx& c) {
  if (c.cycle_graph) cudaGraphExecDestroy(c.cycle_graph);
  c.cycle_graph = nullptr;
  if (c.batch_graph) cudaGraphExecDestroy(c.batch_graph);
  c.batch_graph = nullptr;
}

int log2i(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

// whether level l could run as the fused tile passes whatever its size
bool fuse_eligible(const Ctx& c, int l) {
  const Level& L = c.L[l];
  return !L.fine && !L.coarsest && !L.m_diag && L.g.dim == 2 && c.opts.nu1 == 1 && c.opts.nu2 == 1 &&
         c.nrhs == 1 && L.A.off.rho <= (L.a_half ? 2 : 3) && L.Mh.off.rho <= 2;
}

template <typename T>
void tune_t(Ctx& c, int reps, cudaStream_t s, std::vector<hz_tune_entry>& out) {
  Timer tm(s);
  const int R = c.nrhs;
  auto add = [&](int kind, int level, int cand, double us) {
    hz_tune_entry e;
    e.kind = kind;
    e.level = level;
    e.nrhs = R;
    e.candidate = cand;
    e.us = us;
    e.chosen = 0;
    out.push_back(e);
  };
  // keep the fastest candidate of the entries from index first on, unless the
  // fixed rule's choice `rule` is within 5% of it (timing noise must not move a
  // choice the rule already gets right); returns the kept candidate
  auto pick = [&](size_t first, int rule) {
    size_t best = first;
    for (size_t i = first; i < out.size(); ++i)
      if (out[i].us < out[best].us) best = i;
    for (size_t i = first; i < out.size(); ++i)
      if (out[i].candidate == rule && out[i].us <= 1.05 * out[best].us) best = i;
    out[best].chosen = 1;
    return out[best].candidate;
  };
  const int nl = (int)c.L.size();
  for (int l = 0; l + 1 < nl; ++l) {
    Level& L = c.L[l];
    Level& C = c.L[l + 1];
    auto resid_sweep = [&]() {
      resid<T>(c, l, L.t, L.f, L.r, nullptr, s);
      sweep_out<T>(c, l, L.r, L.t, L.t, nullptr, s);
    };
    if (R >= kVRMax<T>) {
      const size_t first = out.size();
      for (int cand : {1, 2}) {
        L.tune_vr = cand;
        add(1, l, cand, tm.us(reps, resid_sweep));
      }
      L.tune_vr = pick(first, vr_for(R, kVRMax<T>) == kVRMax<T> ? 2 : 1);
    }
    if (R == 1) {
      const size_t first = out.size();
      for (int cand : {0, 2}) {
        L.tune_mb = cand;
        add(2, l, cand, tm.us(reps, resid_sweep));
      }
      L.tune_mb = pick(first, L.g.N <= kIlpNodes ? 2 : 0);
    }
    if (fuse_eligible(c, l)) {
      const size_t first = out.size();
      L.tune_fuse = 0;
      add(3, l, 0, tm.us(reps, [&]() {
            sweep0<T>(c, l, L.f, L.t, nullptr, s);
            resid<T>(c, l, L.t, L.f, L.r, nullptr, s);
            restrict_t<T>(c, l, L.r, C.f, nullptr, s);
            prolong_fused_2d<T, false>(c, l, C.u, L.t, L.f, L.u, L.r, nullptr, s);
            sweep_out<T>(c, l, L.r, L.u, L.u, nullptr, s);
          }));
      L.tune_fuse = 1;
      add(3, l, 1, tm.us(reps, [&]() {
            level_down_2d<T>(c, l, L.f, L.t, C.f, nullptr, s);
            level_up_2d<T>(c, l, C.u, L.t, L.f, L.u, nullptr, s);
          }));
      L.tune_fuse = pick(first, L.g.N <= 70000 ? 1 : 0);
    }
  }
  if (coarse_tc_supported(c, R)) {
    const int lg = log2i(R);
    const size_t first = out.size();
    Level& Lc = c.L.back();
    for (int cand : {0, 1, 2, 4, 8, 16}) {
      c.coarse_variant[lg] = cand;
      add(0, nl - 1, cand, tm.us(reps, [&]() { coarse_t<T>(c, Lc.f, Lc.u, nullptr, s); }));
    }
    c.coarse_variant[lg] = -1;
    const int rule = coarse_variant_for(c, R);
    c.coarse_variant[lg] = pick(first, rule);
  }
}

}  // namespace
}  // namespace hz

using namespace hz;

struct hz_ctx {
  Ctx c;
};

extern "C" hz_status hz_autotune(hz_ctx* ctx, int nrhs, int reps, hz_tune_entry* entries, int cap, int* n) {
  return guarded([&] {
    require(ctx && n && cap >= 0 && (entries || cap == 0), "null argument");
    Ctx& c = ctx->c;
    require(nrhs >= 1 && nrhs <= c.opts.nrhs_max && (nrhs & (nrhs - 1)) == 0,
            "nrhs must be a power of two <= nrhs_max (and <= 64)");
    require(reps >= 1 && reps <= 1000, "reps must be in 1..1000");
    BusyGuard bg(&c);
    int prev = -1;
    HZ_CUDA(cudaGetDevice(&prev));
    if (prev != c.dev) HZ_CUDA(cudaSetDevice(c.dev));
    cudaStream_t s;
    HZ_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    std::vector<hz_tune_entry> out;
    c.nrhs = nrhs;
    try {
      // the level vectors are scratch between solves: start them from zero
      const size_t vb = c.mixed ? sizeof(float2) : sizeof(double2);
      for (Level& L : c.L)
        for (void* v : {L.f, L.u, L.r, L.t})
          if (v) HZ_CUDA(cudaMemsetAsync(v, 0, vb * L.g.N * nrhs, s));
      if (c.mixed) tune_t<float>(c, reps, s, out);
      else tune_t<double>(c, reps, s, out);
      HZ_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
      c.nrhs = 1;
      cudaStreamDestroy(s);
      if (prev != c.dev) cudaSetDevice(prev);
      throw;
    }
    c.nrhs = 1;
    cudaStreamDestroy(s);
    drop_graphs(c);
    if (prev != c.dev) HZ_CUDA(cudaSetDevice(prev));
    *n = (int)out.size();
    for (int i = 0; i < cap && i < (int)out.size(); ++i) entries[i] = out[i];
  });
}

extern "C" hz_status hz_tune_set(hz_ctx* ctx, int kind, int level, int nrhs, int candidate) {
  return guarded([&] {
    require(ctx != nullptr, "null context");
    Ctx& c = ctx->c;
    require(level >= 0 && level < (int)c.L.size(), "level out of range");
    require(nrhs >= 1 && nrhs <= 64 && (nrhs & (nrhs - 1)) == 0, "nrhs must be a power of two <= 64");
    BusyGuard bg(&c);
    Level& L = c.L[level];
    switch (kind) {
      case 0:
        require(L.coarsest, "kind 0 applies to the coarsest level");
        require(candidate == 0 || ((candidate == 1 || candidate == 2 || candidate == 4 || candidate == 8 ||
                                    candidate == 16) &&
                                   coarse_tc_supported(c, nrhs)),
                "coarsest variant must be 0 or a supported tensor-core split 1, 2, 4, 8, 16");
        c.coarse_variant[log2i(nrhs)] = candidate;
        break;
      case 1:
        require(!L.coarsest && (candidate == 1 || candidate == 2), "RHS pack must be 1 or 2");
        L.tune_vr = candidate;
        break;
      case 2:
        require(!L.coarsest && (candidate == 0 || candidate == 2), "register budget must be 0 or 2");
        L.tune_mb = candidate;
        break;
      case 3:
        require(!L.coarsest && !L.fine && L.g.dim == 2 && (candidate == 0 || candidate == 1),
                "fused tile passes apply to coarse 2D levels (candidate 0 or 1)");
        L.tune_fuse = candidate;
        break;
      default:
        throw Error(HZ_ERR_INVALID_ARG, "kind must be 0..3");
    }
    drop_graphs(c);
  });
}
