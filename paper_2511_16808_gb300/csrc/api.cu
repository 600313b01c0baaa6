// C ABI of libhz (declarations and contracts in include/hz.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>

#include "common.cuh"

#include <chrono>

namespace hz {

static thread_local std::string g_last_error;

std::atomic<unsigned long long>& device_alloc_count() {
  static std::atomic<unsigned long long> n{0};
  return n;
}

void set_last_error(const char* msg) {
  if (msg) g_last_error = msg;
  else g_last_error.clear();
}

// readers of the checked-index words, one per translation unit of the
// checked build (registered during static initialisation)
std::vector<int (*)(unsigned long long*, int)>& check_readers() {
  static std::vector<int (*)(unsigned long long*, int)> v;
  return v;
}
void check_register(int (*read)(unsigned long long* words, int clear)) { check_readers().push_back(read); }

// Scratch of the allocation-free sweep (hz_level_smooth_noalloc): the
// residual of one level, c64 or c128, at most HZ_NOALLOC_MAX_NODES nodes.
// It lives in the module's static device memory, so every GPU that loads the
// library holds these 4 MiB until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[(size_t)HZ_NOALLOC_MAX_NODES * 16];

// Device memory of a context comes from the device's stream-ordered pool
// (cudaMallocAsync on the context's allocation stream), so that building and
// freeing hierarchies while other contexts solve does not synchronize the
// device; freed blocks stay in the pool for the next context.
static void keep_pool_memory(int dev) {
  static std::mutex mu;
  static std::vector<int> done;
  std::lock_guard<std::mutex> lk(mu);
  if (std::find(done.begin(), done.end(), dev) != done.end()) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  (void)cudaGetLastError();
  done.push_back(dev);
}

void* ctx_alloc(Ctx& c, size_t bytes, cudaStream_t s) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  keep_pool_memory(c.dev);
  cudaError_t e = counted_malloc_async(&p, bytes, s);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    throw Error(e == cudaErrorMemoryAllocation ? HZ_ERR_OOM : HZ_ERR_CUDA,
                std::string("cudaMallocAsync(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  c.allocations.push_back(p);
  return p;
}

void* ctx_alloc(Ctx& c, size_t bytes) { return ctx_alloc(c, bytes, c.alloc_stream); }

// Small pinned host blocks (the per-context status copies) from a shared
// arena: pinned allocations are slow and synchronizing, and a served request
// needs one per context.
namespace {
constexpr size_t kPinBlock = 4096, kPinChunk = 256;
std::mutex g_pin_mu;
std::vector<void*> g_pin_free;
}  // namespace

void* pinned_small_alloc(size_t bytes) {
  require(bytes <= kPinBlock, "pinned status block too large");
  std::lock_guard<std::mutex> lk(g_pin_mu);
  if (g_pin_free.empty()) {
    void* chunk = nullptr;
    HZ_CUDA(cudaMallocHost(&chunk, kPinBlock * kPinChunk));
    for (size_t i = 0; i < kPinChunk; ++i) g_pin_free.push_back((char*)chunk + i * kPinBlock);
  }
  void* p = g_pin_free.back();
  g_pin_free.pop_back();
  return p;
}

void pinned_small_free(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_free.push_back(p);
}

void ctx_free_all(Ctx& c) {
  if (c.cycle_graph) cudaGraphExecDestroy(c.cycle_graph);
  c.cycle_graph = nullptr;
  if (c.batch_graph) cudaGraphExecDestroy(c.batch_graph);
  c.batch_graph = nullptr;
  for (auto e : c.prof_ev) cudaEventDestroy(e);
  c.prof_ev.clear();
  if (c.ev_in) cudaEventDestroy(c.ev_in);
  if (c.ev_out) cudaEventDestroy(c.ev_out);
  if (c.ev_status) cudaEventDestroy(c.ev_status);
  if (c.ev_status_b) cudaEventDestroy(c.ev_status_b);
  c.ev_in = c.ev_out = c.ev_status = c.ev_status_b = nullptr;
  // frees are ordered after the context's own stream; the caller has
  // synchronized every stream that used the context
  cudaStream_t fs = c.graph_stream ? c.graph_stream : c.alloc_stream;
  for (void* p : c.allocations) cudaFreeAsync(p, fs);
  c.allocations.clear();
  if (c.graph_stream) cudaStreamDestroy(c.graph_stream);
  c.graph_stream = nullptr;
  pinned_small_free(c.ks_host);
  c.ks_host = nullptr;
  (void)cudaGetLastError();
}

namespace {


bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

long long grid_nodes(const hz_grid& g) {
  return (long long)g.n[0] * g.n[1] * (g.dim == 3 ? g.n[2] : 1);
}

void validate(const hz_grid* g, const hz_opts* o) {
  require(g && o, "null grid or options");
  require(g->dim == 2 || g->dim == 3, "dim must be 2 or 3");
  require(g->h > 0 && std::isfinite(g->h), "h must be positive");
  require(o->levels >= 1 && o->levels <= HZ_MAX_LEVELS, "levels out of range");
  for (int a = 0; a < g->dim; ++a) {
    require(g->n[a] >= 3, "need at least 3 nodes per axis");
    const int div = 1 << (o->levels - 1);
    require((g->n[a] - 1) % div == 0, "n-1 must be divisible by 2^(levels-1) on every axis");
    require((g->n[a] - 1) / div >= 2, "coarsest grid needs at least 3 nodes per axis");
  }
  require(o->nu1 >= 0 && o->nu2 >= 0 && o->nu1 + o->nu2 <= 16, "nu1/nu2 out of range");
  require(o->restart_m >= 1 && o->restart_m <= 128, "restart_m out of range (1..128)");
  require(o->nrhs_max <= 1 || o->restart_m <= 16, "restart_m must be <= 16 when nrhs_max > 1");
  require(o->tol > 0 && o->max_iter >= 1, "tol/max_iter out of range");
  require(o->nrhs_max >= 1 && o->nrhs_max <= 64, "nrhs_max must be in 1..64");
  require(o->cycle_visits >= 0 && o->cycle_visits <= 2, "cycle_visits must be 0, 1 (V) or 2 (W)");
  require(o->stencil == 0 || o->stencil == 1, "stencil must be 0 (5/7-point) or 1 (compact)");
  require(o->stencil == 0 || o->nrhs_max == 1, "the compact stencil takes one right-hand side (nrhs_max 1)");
  require(o->precision == HZ_PREC_FP64 || o->precision == HZ_PREC_MIXED, "bad precision");
  require(o->intergrid >= HZ_IG_LINEAR && o->intergrid <= HZ_IG_LEVELDEP, "bad intergrid");
  require(!(g->dim == 3 && o->intergrid == HZ_IG_CUBIC && o->levels >= 3),
          "cubic intergrid in 3D is limited to 2 levels (7x7x7 Galerkin stencils beyond); use leveldep");
  for (int l = 0; l < o->levels - 1; ++l) {
    require(o->patch[l] >= HZ_PATCH_JACOBI && o->patch[l] <= HZ_PATCH_FULL, "bad patch");
    require(std::isfinite(o->damping[l]), "bad damping");
  }
}

// Table relaxParam (Section 5.2) damping per level; rows: fine, 1st, 2nd and
// 3rd coarse level; deeper levels reuse the last row; patches with no column
// use the plus-patch column.
double default_damping(int dim, hz_patch p, int level) {
  static const double d2[4][4] = {{0.89, 0.9, 0.3, 0.71},      // Jacobi
                                  {0.97, 0.66, 0.48, 0.88},    // Element
                                  {0.87, 0.57, 0.55, 0.74},    // Plus
                                  {0.83, 0.5, 0.4, 0.65}};     // RB
  static const double d3[3][4] = {{0.6, 0.4, 0.3, 0.5},        // Jacobi
                                  {1.1, 0.7, 0.45, 0.6},       // Element
                                  {0.92, 0.55, 0.45, 0.55}};   // Plus
  const int r = level < 3 ? level : 3;
  if (dim == 2) {
    int col = p == HZ_PATCH_JACOBI ? 0 : p == HZ_PATCH_ELEMENT ? 1 : p == HZ_PATCH_RB ? 3 : 2;
    return d2[col][r];
  }
  int col = p == HZ_PATCH_JACOBI ? 0 : p == HZ_PATCH_ELEMENT ? 1 : 2;
  return d3[col][r];
}

// Makes `dev` current for the life of a scope and restores the caller's
// device on every exit path (exceptions included).
struct DeviceGuard {
  int prev = -1;
  bool switched = false;
  explicit DeviceGuard(int dev) {
    HZ_CUDA(cudaGetDevice(&prev));
    if (prev != dev) {
      HZ_CUDA(cudaSetDevice(dev));
      switched = true;
    }
  }
  ~DeviceGuard() {
    if (switched) cudaSetDevice(prev);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
};

// Device address of g_noalloc_scratch on `dev`.  Host code only sees a
// host-side stand-in under the array's name, so the address is looked up once
// per device, with that device current, and cached.
void* noalloc_scratch(int dev) {
  static std::mutex mu;
  static void* addr[256] = {};
  require(dev >= 0 && dev < 256, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    cudaError_t e;
    {
      DeviceGuard dg(dev);
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    }
    if (e != cudaSuccess || p == nullptr) {
      (void)cudaGetLastError();
      throw Error(HZ_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    }
    addr[dev] = p;
  }
  return addr[dev];
}

}  // namespace
}  // namespace hz

using namespace hz;

struct hz_ctx {
  Ctx c;
};

extern "C" {

int hz_abi_version(void) { return HZ_ABI_VERSION; }

const char* hz_status_string(hz_status s) {
  switch (s) {
    case HZ_OK: return "ok";
    case HZ_ERR_INVALID_ARG: return "invalid argument";
    case HZ_ERR_OOM: return "out of device memory";
    case HZ_ERR_CUDA: return "CUDA error";
    case HZ_ERR_NOT_CONVERGED: return "not converged";
    case HZ_ERR_BREAKDOWN: return "Krylov breakdown";
    case HZ_ERR_TIMEOUT: return "device wait timed out";
    case HZ_ERR_BUSY: return "context busy";
    case HZ_ERR_NO_DEVICE: return "no suitable CUDA device";
  }
  return "unknown status";
}

const char* hz_last_error(void) { return g_last_error.c_str(); }

hz_status hz_check_status(int* enabled, uint64_t* failures, uint64_t* first, int clear) {
  return guarded([&] {
    require(enabled && failures && first, "null output");
#ifdef HZ_CHECKED
    *enabled = 1;
#else
    *enabled = 0;
#endif
    *failures = 0;
    *first = 0;
    for (auto read : check_readers()) {
      unsigned long long w[2] = {0ull, 0ull};
      if (read(w, clear) != 0) throw Error(HZ_ERR_CUDA, "reading the checked-index words failed");
      if (w[0] && !*failures) *first = w[1];
      *failures += w[0];
    }
  });
}

hz_status hz_opts_default(int dim, hz_opts* out) {
  return guarded([&] {
    require(out != nullptr, "null output");
    require(dim == 2 || dim == 3, "dim must be 2 or 3");
    std::memset(out, 0, sizeof(*out));
    out->levels = 4;
    const hz_patch p = dim == 2 ? HZ_PATCH_RB : HZ_PATCH_ELEMENT;
    for (int l = 0; l < HZ_MAX_LEVELS; ++l) {
      out->patch[l] = p;
      out->damping[l] = default_damping(dim, p, l);
    }
    out->nu1 = 1;
    out->nu2 = 1;
    out->intergrid = dim == 2 ? HZ_IG_LEVELDEP : HZ_IG_LINEAR;
    out->precision = HZ_PREC_MIXED;
    out->restart_m = 5;
    out->tol = 1e-6;
    out->max_iter = 2000;
    out->nrhs_max = 1;
    out->cycle_visits = 1;
    out->stencil = 0;
  });
}

double hz_default_damping(int dim, hz_patch patch, int level) {
  if ((dim != 2 && dim != 3) || level < 0) return std::nan("");
  return default_damping(dim, patch, level);
}

hz_status hz_setup_bytes(const hz_grid* g, const hz_opts* opts, size_t* bytes) {
  return guarded([&] {
    validate(g, opts);
    require(bytes != nullptr, "null output");
    *bytes = hierarchy_bytes(*g, *opts) + krylov_bytes(*g, *opts);
  });
}

hz_status hz_setup(const hz_grid* g, const double* kappa, double omega, const double* gamma, double gamma0,
                   double shift_alpha, const hz_opts* opts, void* cuda_stream, hz_ctx** out) {
  hz_ctx* h = nullptr;
  hz_status st = guarded([&] {
    validate(g, opts);
    require(out != nullptr && kappa != nullptr, "null kappa or output");
    require(omega > 0 && std::isfinite(omega), "omega must be positive");
    require(shift_alpha >= 0 && std::isfinite(shift_alpha), "shift must be >= 0");
    require(std::isfinite(gamma0), "gamma0 must be finite");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
      (void)cudaGetLastError();
      throw Error(HZ_ERR_NO_DEVICE, "no CUDA device");
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    NvtxRange range("hz_setup");
    const auto t0 = std::chrono::steady_clock::now();
    h = new hz_ctx();
    Ctx& c = h->c;
    c.grid = *g;
    if (g->dim == 2) c.grid.n[2] = 1;
    c.opts = *opts;
    c.omega = omega;
    c.alpha = shift_alpha;
    c.h = g->h;
    c.mixed = opts->precision == HZ_PREC_MIXED;
    c.compact = opts->stencil == 1;
    c.alloc_stream = s;
    HZ_CUDA(cudaGetDevice(&c.dev));
    const long long N = grid_nodes(c.grid);
    // stage kappa / gamma on the device and check kappa
    double* dk = (double*)ctx_alloc(c, sizeof(double) * N);
    double* dg = gamma ? (double*)ctx_alloc(c, sizeof(double) * N) : nullptr;
    HZ_CUDA(cudaMemcpyAsync(dk, kappa, sizeof(double) * N, cudaMemcpyDefault, s));
    if (gamma) HZ_CUDA(cudaMemcpyAsync(dg, gamma, sizeof(double) * N, cudaMemcpyDefault, s));
    if (!is_device_ptr(kappa)) {
      for (long long i = 0; i < N; ++i)
        require(std::isfinite(kappa[i]) && kappa[i] > 0, "kappa must be finite and positive");
    }
    build_hierarchy(c, dk, dg, gamma0, s);
    krylov_alloc(c);
    HZ_CUDA(cudaStreamSynchronize(s));
    c.setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  });
  if (st != HZ_OK) {
    if (h) {
      ctx_free_all(h->c);
      delete h;
    }
    return st;
  }
  *out = h;
  return HZ_OK;
}

hz_status hz_destroy(hz_ctx* ctx) {
  return guarded([&] {
    if (!ctx) return;
    // the context's own work runs on its library stream; other streams that
    // used it are the caller's to synchronize before destroying it
    if (ctx->c.graph_stream) cudaStreamSynchronize(ctx->c.graph_stream);
    ctx_free_all(ctx->c);
    delete ctx;
  });
}

hz_status hz_solve(hz_ctx* ctx, const void* q, void* p, int nrhs, hz_info* info, void* cuda_stream) {
  return guarded([&] {
    require(ctx && q && p && info, "null argument");
    Ctx& c = ctx->c;
    require(nrhs >= 1 && nrhs <= c.opts.nrhs_max && (nrhs & (nrhs - 1)) == 0,
            "nrhs must be a power of two <= nrhs_max (and <= 64)");
    BusyGuard bg(&c);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const long long N = c.L[0].g.N * nrhs;
    const double2* qd = (const double2*)q;
    double2* pd = (double2*)p;
    const bool q_host = !is_device_ptr(q), p_host = !is_device_ptr(p);
    if (q_host) {
      if (!c.qstage) c.qstage = (double2*)ctx_alloc(c, sizeof(double2) * c.L[0].g.N * c.opts.nrhs_max, s);
      HZ_CUDA(cudaMemcpyAsync(c.qstage, q, sizeof(double2) * N, cudaMemcpyHostToDevice, s));
      qd = c.qstage;
    }
    if (p_host) pd = c.p;
    if (nrhs == 1) fgmres_solve(c, qd, pd, info, s);
    else fgmres_solve_batch(c, qd, pd, nrhs, info, s);
    if (p_host) {
      HZ_CUDA(cudaMemcpyAsync(p, pd, sizeof(double2) * N, cudaMemcpyDeviceToHost, s));
      HZ_CUDA(cudaStreamSynchronize(s));
    }
    for (int r = 0; r < nrhs; ++r)
      if (!info[r].converged) throw Error(HZ_ERR_NOT_CONVERGED, "FGMRES did not reach tol within max_iter");
  });
}

hz_status hz_solve_begin(hz_ctx* ctx, const void* q, void* cuda_stream) {
  return guarded([&] {
    require(ctx && q, "null argument");
    Ctx& c = ctx->c;
    BusyGuard bg(&c);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const double2* qd = (const double2*)q;
    if (!is_device_ptr(q)) {
      if (!c.qstage) c.qstage = (double2*)ctx_alloc(c, sizeof(double2) * c.L[0].g.N * c.opts.nrhs_max, s);
      HZ_CUDA(cudaMemcpyAsync(c.qstage, q, sizeof(double2) * c.L[0].g.N, cudaMemcpyHostToDevice, s));
      qd = c.qstage;
    }
    solve_begin(c, qd, s);
  });
}

hz_status hz_solve_step(hz_ctx* ctx, int block, int* done) {
  return guarded([&] {
    require(ctx && done, "null argument");
    BusyGuard bg(&ctx->c);
    require(ctx->c.as_state != 0, "no asynchronous solve in flight");
    *done = solve_step(ctx->c, block != 0);
  });
}

hz_status hz_solve_end(hz_ctx* ctx, void* p, hz_info* info, void* cuda_stream) {
  return guarded([&] {
    require(ctx && p && info, "null argument");
    Ctx& c = ctx->c;
    BusyGuard bg(&c);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const bool p_host = !is_device_ptr(p);
    solve_end(c, p_host ? c.p : (double2*)p, info, s);
    if (p_host) {
      HZ_CUDA(cudaMemcpyAsync(p, c.p, sizeof(double2) * c.L[0].g.N, cudaMemcpyDeviceToHost, s));
      HZ_CUDA(cudaStreamSynchronize(s));
    }
    if (!info->converged) throw Error(HZ_ERR_NOT_CONVERGED, "FGMRES did not reach tol within max_iter");
  });
}

hz_status hz_precond_apply(hz_ctx* ctx, const void* r, void* z, int nrhs, void* cuda_stream) {
  return guarded([&] {
    require(ctx && r && z, "null argument");
    require(nrhs >= 1 && nrhs <= ctx->c.opts.nrhs_max && (nrhs & (nrhs - 1)) == 0,
            "nrhs must be a power of two <= nrhs_max (and <= 64)");
    BusyGuard bg(&ctx->c);
    precond_apply_c128(ctx->c, (const double2*)r, (double2*)z, nrhs, (cudaStream_t)cuda_stream);
  });
}

hz_status hz_apply_operator(hz_ctx* ctx, const void* v, void* w, int nrhs, int shifted, void* cuda_stream) {
  return guarded([&] {
    require(ctx && v && w, "null argument");
    require(nrhs >= 1 && nrhs <= ctx->c.opts.nrhs_max && (nrhs & (nrhs - 1)) == 0,
            "nrhs must be a power of two <= nrhs_max (and <= 64)");
    BusyGuard bg(&ctx->c);
    ctx->c.nrhs = nrhs;
    fine_apply_f64(ctx->c, v, false, (double2*)w, shifted != 0, (cudaStream_t)cuda_stream);
    ctx->c.nrhs = 1;
  });
}

hz_status hz_kernel_launches(const hz_ctx* ctx, int64_t* count) {
  return guarded([&] {
    require(ctx && count, "null argument");
    *count = ctx->c.launches;
  });
}

hz_status hz_profile_select(hz_ctx* ctx, int kernel_class) {
  return guarded([&] {
    require(ctx != nullptr, "null context");
    require(kernel_class >= 0 && kernel_class <= 3, "unknown kernel class");
    BusyGuard bg(&ctx->c);
    profile_select(ctx->c, kernel_class);
  });
}

hz_status hz_profile_read(const hz_ctx* ctx, double* total_ms, int64_t* launches, double* bytes, double* flops) {
  return guarded([&] {
    require(ctx && total_ms && launches && bytes && flops, "null argument");
    const Ctx& c = ctx->c;
    *total_ms = c.prof_ms;
    *launches = c.prof_launches;
    *bytes = c.prof_bytes;
    *flops = c.prof_flops;
  });
}

hz_status hz_memory_stats(int device, uint64_t* pool_used_bytes, uint64_t* device_allocations) {
  return guarded([&] {
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
      (void)cudaGetLastError();
      throw Error(HZ_ERR_NO_DEVICE, "no CUDA device");
    }
    require(device >= 0 && device < n, "device ordinal out of range");
    if (pool_used_bytes) {
      cudaMemPool_t pool;
      HZ_CUDA(cudaDeviceGetDefaultMemPool(&pool, device));
      uint64_t used = 0;
      HZ_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
      *pool_used_bytes = used;
    }
    if (device_allocations) *device_allocations = device_alloc_count().load();
  });
}

hz_status hz_context_info(const hz_ctx* ctx, int* device, int* precision, int* nrhs_max) {
  return guarded([&] {
    require(ctx != nullptr, "null context");
    if (device) *device = ctx->c.dev;
    if (precision) *precision = ctx->c.mixed ? HZ_PREC_MIXED : HZ_PREC_FP64;
    if (nrhs_max) *nrhs_max = ctx->c.opts.nrhs_max;
  });
}

hz_status hz_level_count(const hz_ctx* ctx, int* levels) {
  return guarded([&] {
    require(ctx && levels, "null argument");
    *levels = (int)ctx->c.L.size();
  });
}

hz_status hz_level_describe(const hz_ctx* ctx, int level, hz_level_desc* out) {
  return guarded([&] {
    require(ctx && out, "null argument");
    const Ctx& c = ctx->c;
    require(level >= 0 && level < (int)c.L.size(), "level out of range");
    const Level& L = c.L[level];
    std::memset(out, 0, sizeof(*out));
    out->n[0] = L.g.nx;
    out->n[1] = L.g.ny;
    out->n[2] = L.g.nz;
    out->nodes = L.g.N;
    out->stencil_size = L.A.off.n;
    for (int k = 0; k < L.A.off.n; ++k)
      for (int a = 0; a < 3; ++a) out->stencil_off[k][a] = L.A.off.d[k][a];
    out->smoother_size = L.coarsest ? 0 : L.M.off.n;
    for (int k = 0; k < out->smoother_size; ++k)
      for (int a = 0; a < 3; ++a) out->smoother_off[k][a] = L.M.off.d[k][a];
    out->patch = L.patch;
    out->damping = L.damping;
    out->is_coarsest = L.coarsest ? 1 : 0;
  });
}

hz_status hz_level_export(const hz_ctx* ctx, int level, int what, void* host_out) {
  return guarded([&] {
    require(ctx && host_out, "null argument");
    const Ctx& c = ctx->c;
    require(level >= 0 && level < (int)c.L.size(), "level out of range");
    const Level& L = c.L[level];
    require(what == 0 || (what == 1 && !L.coarsest), "nothing to export");
    const double2* src = what == 0 ? L.A64 : L.M64;
    const int n = what == 0 ? L.A.off.n : L.M.off.n;
    HZ_CUDA(cudaMemcpy(host_out, src, sizeof(double2) * L.g.N * n, cudaMemcpyDeviceToHost));
  });
}

static void check_level(const hz_ctx* ctx, int level, bool need_next) {
  require(ctx != nullptr, "null context");
  require(level >= 0 && level < (int)ctx->c.L.size(), "level out of range");
  if (need_next) require(level + 1 < (int)ctx->c.L.size(), "no coarser level");
}

hz_status hz_level_residual(hz_ctx* ctx, int level, const void* u, const void* f, void* r, void* cuda_stream) {
  return guarded([&] {
    check_level(ctx, level, false);
    require(u && f && r, "null argument");
    BusyGuard bg(&ctx->c);
    ctx->c.nrhs = 1;
    level_residual(ctx->c, level, u, f, r, nullptr, (cudaStream_t)cuda_stream);
  });
}

hz_status hz_level_smooth(hz_ctx* ctx, int level, void* u, const void* f, void* cuda_stream) {
  return guarded([&] {
    check_level(ctx, level, false);
    require(u && f, "null argument");
    require(!ctx->c.L[level].coarsest, "the coarsest level has no smoother");
    BusyGuard bg(&ctx->c);
    ctx->c.nrhs = 1;
    level_smooth(ctx->c, level, u, f, false, nullptr, (cudaStream_t)cuda_stream);
  });
}

hz_status hz_level_smooth_noalloc(hz_ctx* ctx, int level, void* u, const void* f, void* cuda_stream) {
  return guarded([&] {
    check_level(ctx, level, false);
    require(u && f, "null argument");
    Ctx& c = ctx->c;
    const Level& L = c.L[level];
    require(!L.coarsest, "the coarsest level has no smoother");
    if (L.g.N > HZ_NOALLOC_MAX_NODES)
      throw Error(HZ_ERR_INVALID_ARG, "level has " + std::to_string(L.g.N) +
                                          " nodes; the allocation-free sweep handles at most " +
                                          std::to_string(HZ_NOALLOC_MAX_NODES));
    BusyGuard bg(&c);
    void* r = noalloc_scratch(c.dev);
    c.nrhs = 1;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    DeviceGuard dg(c.dev);
    // every scratch entry is written by the residual before it is read: no clearing needed
    level_residual(c, level, u, f, r, nullptr, s);
    level_vanka_apply(c, level, r, u, s);
  });
}

hz_status hz_level_restrict(hz_ctx* ctx, int level, const void* r, void* fc, void* cuda_stream) {
  return guarded([&] {
    check_level(ctx, level, true);
    require(r && fc, "null argument");
    BusyGuard bg(&ctx->c);
    ctx->c.nrhs = 1;
    level_restrict(ctx->c, level, r, fc, nullptr, (cudaStream_t)cuda_stream);
  });
}

hz_status hz_level_prolong_add(hz_ctx* ctx, int level, const void* ec, void* u, void* cuda_stream) {
  return guarded([&] {
    check_level(ctx, level, true);
    require(ec && u, "null argument");
    BusyGuard bg(&ctx->c);
    ctx->c.nrhs = 1;
    level_prolong_add(ctx->c, level, ec, u, nullptr, (cudaStream_t)cuda_stream);
  });
}

hz_status hz_coarse_solve(hz_ctx* ctx, const void* f, void* u, void* cuda_stream) {
  return guarded([&] {
    require(ctx && f && u, "null argument");
    BusyGuard bg(&ctx->c);
    ctx->c.nrhs = 1;
    coarse_solve(ctx->c, f, u, nullptr, (cudaStream_t)cuda_stream);
  });
}

hz_status hz_coarse_solve_batch(hz_ctx* ctx, const void* f, void* u, int nrhs, int variant, void* cuda_stream) {
  return guarded([&] {
    require(ctx && f && u, "null argument");
    Ctx& c = ctx->c;
    require(nrhs >= 1 && nrhs <= c.opts.nrhs_max && (nrhs & (nrhs - 1)) == 0,
            "nrhs must be a power of two <= nrhs_max (and <= 64)");
    require(variant >= -1 && variant <= kTcMaxSplit, "variant must be -1, 0 or a split of 1..16");
    require(variant <= 0 || coarse_tc_supported(c, nrhs),
            "tensor-core variant: mixed precision and 16, 32 or 64 right-hand sides");
    BusyGuard bg(&c);
    int lg = 0;
    while ((1 << lg) < nrhs) ++lg;
    const int keep = c.coarse_variant[lg];
    if (variant >= 0) c.coarse_variant[lg] = variant;
    c.nrhs = nrhs;
    try {
      coarse_solve(c, f, u, nullptr, (cudaStream_t)cuda_stream);
    } catch (...) {
      c.coarse_variant[lg] = keep;
      c.nrhs = 1;
      throw;
    }
    c.coarse_variant[lg] = keep;
    c.nrhs = 1;
  });
}

hz_status hz_setup_seconds(const hz_ctx* ctx, double* seconds) {
  return guarded([&] {
    require(ctx && seconds, "null argument");
    *seconds = ctx->c.setup_seconds;
  });
}

hz_status hz_solve_history(const hz_ctx* ctx, int cap, int* iters, double* relres_true, double* relres_est,
                           int* n) {
  return guarded([&] {
    require(ctx && n && cap >= 0, "null argument or negative capacity");
    std::lock_guard<std::mutex> lk(const_cast<hz_ctx*>(ctx)->c.history_mu);
    const auto& hst = ctx->c.history;
    *n = (int)hst.size();
    for (int i = 0; i < cap && i < (int)hst.size(); ++i) {
      if (iters) iters[i] = (int)hst[i][0];
      if (relres_true) relres_true[i] = hst[i][1];
      if (relres_est) relres_est[i] = hst[i][2];
    }
  });
}

hz_status hz_cycle_factor(hz_ctx* ctx, const void* f, void* u, int warmup, double target, int max_iter,
                          double* factor, int* iters, void* cuda_stream) {
  return guarded([&] {
    require(ctx && f && u && factor && iters, "null argument");
    require(warmup >= 0 && max_iter >= 1, "warmup >= 0 and max_iter >= 1 required");
    require(target > 0.0 && target < 1.0, "target must be in (0, 1)");
    BusyGuard bg(&ctx->c);
    ctx->c.nrhs = 1;
    cycle_factor(ctx->c, (const double2*)f, (double2*)u, warmup, target, max_iter, factor, iters,
                 (cudaStream_t)cuda_stream);
  });
}

}  // extern "C"
