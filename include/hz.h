/*
 * hz.h — C ABI of the GB300 (sm_103a) Vanka-smoothed shifted-Laplacian
 * multigrid / FGMRES solver for the finite-difference Helmholtz equation.
 *
 * Method: Yovel, He & Treister, "Vanka-smoothed Shifted Laplacian multigrid
 * preconditioners for the Helmholtz equations" (arXiv 2511.16808).
 *
 *   Eq. (1)        -Lap p - omega^2 kappa^2 (1 - i gamma/omega) p = q
 *   Eq. (shift)    H_s = H + i alpha omega^2 M   (shift adds damping)
 *   Section 3.1    Galerkin coarse operators R H P, level-dependent intergrid
 *   Section 3.2/3  additive Vanka smoother, Eq. (smoother), boundary patches
 *   Algorithm 1    two-grid cycle, applied recursively as a V-cycle
 *   Section 2.3    flexible GMRES(m) with the cycle as right preconditioner
 *
 * Discretisation (Section 2.1, second-order variant): 5-point (2D) or
 * 7-point (3D) stencil on a nodal grid with spacing h; boundary nodes carry
 * the first-order absorbing condition dp/dn = -i omega kappa p through a
 * ghost point, and every boundary row is halved once per boundary axis, so
 * the matrix is complex symmetric.  The right-hand side is scaled the same
 * way (q_hat = prod_a w_a * q, w_a = 1/2 on the two end nodes of axis a).
 *
 * Conventions for every entry point
 *  - Fields are interleaved complex (re, im) arrays, node-major with x
 *    fastest: node index (k*n_y + j)*n_x + i.  With nrhs > 1 the right-hand
 *    side index is innermost: element (node*nrhs + r).
 *  - "c128" fields are double pairs, "c64" fields float pairs.
 *  - Pointers documented "host or device" may be either; the library finds
 *    out with cudaPointerGetAttributes and stages host data itself.  All other
 *    field pointers are device pointers.
 *  - The caller owns every buffer it passes.  hz_setup copies kappa and gamma;
 *    the context owns the hierarchy and the Krylov workspace.
 *  - Every call returns an hz_status; no C++ exception crosses the ABI and
 *    nothing aborts.  hz_last_error() gives the last message of this thread.
 *  - One context per stream: a context used concurrently from two host threads
 *    returns HZ_ERR_BUSY to the second.
 *  - Inputs are never modified.
 */
#ifndef HZ_H
#define HZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HZ_ABI_VERSION 4
#define HZ_MAX_LEVELS 10
#define HZ_MAX_STENCIL 343   /* 7^3: cubic Galerkin stencils in 3D */

typedef enum {
  HZ_OK = 0,
  HZ_ERR_INVALID_ARG = 1,
  HZ_ERR_OOM = 2,
  HZ_ERR_CUDA = 3,
  HZ_ERR_NOT_CONVERGED = 4,   /* max_iter reached; info and the last iterate are filled */
  HZ_ERR_BREAKDOWN = 5,       /* FGMRES breakdown with a non-converged residual */
  HZ_ERR_TIMEOUT = 6,         /* a bounded device-side wait gave up */
  HZ_ERR_BUSY = 7,            /* context in use by another host thread */
  HZ_ERR_NO_DEVICE = 8        /* no CUDA device or no sm_103 device */
} hz_status;

/* Vanka patches, Section 3.2 (HZ_PATCH_JACOBI: a 1x1 patch = damped Jacobi). */
typedef enum {
  HZ_PATCH_JACOBI = 0,
  HZ_PATCH_ELEMENT = 1,  /* 2^d vertices of a cell                        */
  HZ_PATCH_PLUS = 2,     /* node + 2d nearest neighbours                  */
  HZ_PATCH_RB = 3,       /* node + same red-black colour in the 3^d box   */
  HZ_PATCH_FULL = 4      /* the 3^d box                                    */
} hz_patch;

/* Intergrid schemes, Section 3.1 (Eqs. biliniearIntergrid, bicubicIntergrid,
 * level1Intergrid, levelDepIntergrid; trilinear/tricubic in 3D). */
typedef enum {
  HZ_IG_LINEAR = 0,      /* linear R and P on every level                 */
  HZ_IG_CUBIC = 1,       /* cubic R and P on every level                  */
  HZ_IG_MIXED = 2,       /* linear R, cubic P on every level              */
  HZ_IG_LEVELDEP = 3     /* cubic/cubic for 1->2, linear R / cubic P below */
} hz_intergrid;

typedef enum {
  HZ_PREC_FP64 = 0,      /* V-cycle in complex FP64                        */
  HZ_PREC_MIXED = 1      /* V-cycle in complex FP32 inside FP64 FGMRES     */
} hz_precision;

typedef struct {
  int dim;               /* 2 or 3                                        */
  int n[3];              /* nodes per axis (x, y, z); n[2] = 1 in 2D       */
  double h;              /* uniform grid spacing                           */
} hz_grid;

typedef struct {
  int levels;                        /* multigrid levels, 1..HZ_MAX_LEVELS;
                                        (n[a]-1) divisible by 2^(levels-1) */
  hz_patch patch[HZ_MAX_LEVELS];     /* smoother per level, [0] = finest   */
  double damping[HZ_MAX_LEVELS];     /* damping w per level                */
  int nu1, nu2;                      /* pre- / post-relaxations            */
  hz_intergrid intergrid;
  hz_precision precision;
  int restart_m;                     /* FGMRES restart length, 1..128 (1..16
                                        when nrhs_max > 1); a length at
                                        least the iteration count gives
                                        non-restarted FGMRES (Section 5.2) */
  double tol;                        /* relative residual ||q_hat - A p|| / ||q_hat|| */
  int max_iter;                      /* max preconditioner applications    */
  int nrhs_max;                      /* largest nrhs any call will pass    */
  int cycle_visits;                  /* cycles on the next level per visit of a
                                        level, Section 2.2: 1 = V-cycle,
                                        2 = W-cycle (the coarsest level, solved
                                        exactly, is solved once); 0 means 1  */
  int stencil;                       /* fine-level discretisation, Section 2.1:
                                        0 = second-order 5-point (2D) / 7-point
                                        (3D) with the first-order absorbing
                                        boundary (default);
                                        1 = compact fourth-order 9-point /
                                        19-point stencils (Eqs. disc4thCompact,
                                        disc4thCompact3D) with a variable medium
                                        as L - (Sigma M + M Sigma)/2, neighbours
                                        outside the grid dropped, right-hand side
                                        M q, shift i alpha omega^2 M; one
                                        right-hand side per solve (nrhs_max 1) */
} hz_opts;

typedef struct hz_ctx hz_ctx;        /* opaque, owned by the library */

typedef struct {
  int iters;                         /* preconditioner applications        */
  int converged;                     /* 1 if relres_true < tol             */
  double relres_est;                 /* last Arnoldi residual estimate     */
  double relres_true;                /* ||q_hat - A p|| / ||q_hat||, FP64  */
} hz_info;

/* Per-level description (component entry points below). */
typedef struct {
  int n[3];                          /* nodes per axis                     */
  int64_t nodes;
  int stencil_size;                  /* entries of the level's shifted operator */
  int stencil_off[HZ_MAX_STENCIL][3];
  int smoother_size;                 /* entries of the assembled Vanka sum */
  int smoother_off[HZ_MAX_STENCIL][3];
  hz_patch patch;
  double damping;
  int is_coarsest;
} hz_level_desc;

/* ---- library ---------------------------------------------------------- */

int hz_abi_version(void);
const char* hz_status_string(hz_status s);
/* Message of the last failing call on this host thread ("" if none). */
const char* hz_last_error(void);

/* Defaults for dim = 2 or 3: levels 4, RB patch (2D) / element patch (3D)
 * on every level with the damping of Table relaxParam (levels beyond the
 * table reuse its last row), V(1,1), level-dependent intergrid (2D) /
 * linear (3D), mixed precision, GMRES(5) (Section 5.2), tol 1e-6,
 * max_iter 2000, nrhs_max 1. */
hz_status hz_opts_default(int dim, hz_opts* out);

/* Damping of Table relaxParam for a patch on a level (0 = finest); levels
 * beyond the table reuse its last row, patches without a column (2D full,
 * 3D RB and full) use the plus-patch column.  Returns NaN for a bad dim. */
double hz_default_damping(int dim, hz_patch patch, int level);

/* Device bytes a context for this grid and options will hold (for admission
 * by an HBM budget).  Does not touch the GPU. */
hz_status hz_setup_bytes(const hz_grid* g, const hz_opts* opts, size_t* bytes);

/* Build the hierarchy (Sections 3.1-3.3) for A_s = A + i alpha omega^2 M.
 *   kappa  slowness per node, double, host or device, n_x*n_y*n_z values
 *   gamma  attenuation per node, double, host or device; NULL = gamma0 everywhere
 *   omega  angular frequency (> 0); shift_alpha >= 0
 * Errors: HZ_ERR_INVALID_ARG for bad sizes / non-finite or non-positive kappa,
 * HZ_ERR_OOM when device memory runs out (nothing is leaked), HZ_ERR_CUDA.
 * Work is queued on cuda_stream (a cudaStream_t, NULL = default stream); the
 * call returns after setup has finished on the device. */
hz_status hz_setup(const hz_grid* g, const double* kappa, double omega, const double* gamma,
                   double gamma0, double shift_alpha, const hz_opts* opts, void* cuda_stream,
                   hz_ctx** out);

hz_status hz_destroy(hz_ctx* ctx);

/* Solve A p = q_hat with FGMRES(m) preconditioned by one V(nu1,nu2)-cycle
 * (zero initial guess, Section 5).  q: unscaled source, c128, host or device,
 * nodes*nrhs values; p: c128 output, host or device; info: nrhs entries
 * (host).  nrhs is a power of two <= opts.nrhs_max (<= 64); with nrhs > 1 the
 * right-hand sides share each batched V-cycle launch (RHS index innermost)
 * while each keeps its own Krylov state and convergence, so its iteration
 * count is the one it has alone.  Returns HZ_ERR_NOT_CONVERGED (with p and
 * info filled) when any right-hand side misses tol within max_iter. */
hz_status hz_solve(hz_ctx* ctx, const void* q, void* p, int nrhs, hz_info* info, void* cuda_stream);

/* Asynchronous single-right-hand-side solve: the same FGMRES(m) as hz_solve,
 * split so that one host thread can keep several contexts' solves in flight
 * (the serving loop below is built on it; the paper has no counterpart).
 *   hz_solve_begin  queues the start-up work after the work already queued on
 *                   cuda_stream.  q: unscaled source, c128, host (copied before
 *                   the call returns) or device (read by the queued work: keep it
 *                   unchanged until the solve has finished).
 *   hz_solve_step   looks at the status of the oldest queued restart cycle;
 *                   if it has not completed yet (block = 0) or the solve goes
 *                   on, it sets *done = 0 (in the second case queuing cycles so
 *                   that two stay in flight: the device runs the next cycle
 *                   while the host reads a status; a cycle queued after the
 *                   solve has stopped does no work); *done = 1 once converged
 *                   or out of iterations.  block = 1 waits for the status first.
 *                   (While a kernel class is profiled, hz_profile_select, one
 *                   cycle is queued at a time.)
 *   hz_solve_end    after *done = 1: p (c128, host or device) receives the
 *                   solution, ordered before later work on cuda_stream; info as
 *                   for hz_solve, HZ_ERR_NOT_CONVERGED likewise.
 * A context holds one asynchronous solve at a time (HZ_ERR_INVALID_ARG for a
 * second begin); the other calls on the context must not run in between. */
hz_status hz_solve_begin(hz_ctx* ctx, const void* q, void* cuda_stream);
hz_status hz_solve_step(hz_ctx* ctx, int block, int* done);
hz_status hz_solve_end(hz_ctx* ctx, void* p, hz_info* info, void* cuda_stream);

/* ---------------------------------------------------------------- serving
 * Continuous batching of independent solves on one GPU (the paper has no
 * counterpart).  A request is a whole problem: grid, medium, frequency,
 * shift, solver options (nrhs_max = 1) and one source.  The server admits
 * queued requests in arrival order while their estimated device bytes fit the
 * budget and a slot is free, builds each hierarchy on the request's own
 * stream, keeps every admitted solve's restart cycles in flight at once (they
 * overlap on the device), writes each solution to the caller's buffer and
 * frees the hierarchy, which admits the next request.  Requests are
 * independent: one that fails records its status and releases its slot.
 * Results do not depend on what else runs: each request's kernels and
 * reductions are the ones hz_solve runs, in the same order.
 *
 * Grouping (group_max >= 2): requests of the same problem (the same grid,
 * medium, frequency, shift and solver options; only the source differs)
 * that wait in the queue together are solved together: when the first of
 * them is admitted, the later ones (in arrival order, up to group_max, and
 * only as many as the budget allows) join it, share its hierarchy and run
 * as the right-hand sides of one multi-RHS solve (hz_solve with nrhs = the
 * group's size rounded up to a power of two, the extra right-hand sides
 * zero), so every V-cycle of the group is one batched V-cycle over the same
 * levels.  A grouped request's solution is that of the batched solve: its
 * iteration count and its solution agree with its solve alone within the
 * solver's tolerance, not bit for bit (the batched kernels sum in another
 * order).  The group's solve runs in a setup thread, which it holds until the
 * group finishes.  Requests with the compact stencil or with restarts longer
 * than 16 are never grouped (the batched solve does not take them). */
typedef struct hz_server hz_server;

typedef struct {
  size_t hbm_budget;   /* device bytes the admitted requests may hold; 0 = 80% of free memory */
  int max_active;      /* requests admitted at once (set up or solving); 0 = 32 */
  int device;          /* CUDA device ordinal; -1 = the calling thread's current device */
  int setup_threads;   /* host threads building hierarchies concurrently (1..8); 0 = 2 */
  int group_max;       /* requests of the same problem solved together, at most
                          (a power of two 2..64); 0 or 1 = every request alone */
} hz_server_opts;

typedef struct {
  hz_grid grid;
  const double* kappa;   /* host, nodes values (copied at submission) */
  const double* gamma;   /* host, nodes values or NULL = gamma0 (copied) */
  double gamma0;
  double omega;
  double shift_alpha;
  hz_opts opts;          /* nrhs_max must be 1 */
  const void* q;         /* host c128 source, nodes values (copied) */
  void* p;               /* host c128 solution buffer, written when the request
                            finishes; keep it alive until then */
} hz_request;

enum { HZ_REQ_QUEUED = 0, HZ_REQ_SETUP = 1, HZ_REQ_SOLVING = 2, HZ_REQ_DONE = 3, HZ_REQ_FAILED = 4 };

typedef struct {
  int state;             /* HZ_REQ_* */
  hz_status status;      /* HZ_OK, HZ_ERR_NOT_CONVERGED (p filled) or the failure */
  hz_info info;
  double t_submit, t_admit, t_start, t_done;   /* seconds since hz_server_create */
  size_t bytes;          /* admission estimate */
  char message[128];     /* failure message, empty otherwise */
  int group_size;        /* requests solved together with this one, itself
                            included (1 = alone) */
} hz_ticket_info;

typedef struct {
  int queued, setting_up, solving, done, failed;
  size_t bytes_in_use, peak_bytes, budget;
  int max_active;
  double elapsed_s;          /* since hz_server_create */
  int64_t kernel_launches;   /* kernels launched for the requests finished so far */
  int groups;                /* solves that served two or more requests together */
  int grouped;               /* requests served in those solves */
} hz_server_counters;

/* Starts the server's host threads on the device.  opts may be NULL. */
hz_status hz_server_create(const hz_server_opts* opts, hz_server** out);
/* Validates and copies the request and queues it; *ticket identifies it.
 * HZ_ERR_OOM when its estimate exceeds the whole budget, HZ_ERR_INVALID_ARG
 * for bad sizes or options (the medium is checked later, at setup). */
hz_status hz_server_submit(hz_server* srv, const hz_request* req, uint64_t* ticket);
/* Current state of a request (non-blocking). */
hz_status hz_server_poll(hz_server* srv, uint64_t ticket, hz_ticket_info* out);
/* Waits until the request has finished or failed (timeout_s < 0: no limit);
 * HZ_ERR_TIMEOUT, with out filled, when the time ran out first. */
hz_status hz_server_wait(hz_server* srv, uint64_t ticket, double timeout_s, hz_ticket_info* out);
hz_status hz_server_stats(hz_server* srv, hz_server_counters* out);
/* Finishes every submitted request, then stops the threads and frees all. */
hz_status hz_server_destroy(hz_server* srv);

/* The server's admission policy on its own (host only, no device): FIFO
 * under a byte budget and a slot limit.  offer queues (accepted = 0 when the
 * bytes exceed the whole budget); next admits the head if it fits (admitted =
 * 0 otherwise, nothing overtakes it); release returns a finished request's
 * bytes and slot. */
typedef struct hz_sched hz_sched;
hz_status hz_sched_create(size_t budget, int max_active, hz_sched** out);
hz_status hz_sched_offer(hz_sched* s, uint64_t ticket, size_t bytes, int* accepted);
hz_status hz_sched_next(hz_sched* s, uint64_t* ticket, int* admitted);
hz_status hz_sched_release(hz_sched* s, size_t bytes);
hz_status hz_sched_state(const hz_sched* s, size_t* in_use, size_t* peak, int* active, int* queued);
hz_status hz_sched_destroy(hz_sched* s);

/* z = V-cycle(r) with zero initial guess (Algorithm 1, recursive).
 * r, z: c128 device arrays of nodes*nrhs values (r in the row-scaled space);
 * nrhs as for hz_solve. */
hz_status hz_precond_apply(hz_ctx* ctx, const void* r, void* z, int nrhs, void* cuda_stream);

/* w = A v (shifted = 0) or w = A_s v (shifted = 1), FP64; c128 device arrays. */
hz_status hz_apply_operator(hz_ctx* ctx, const void* v, void* w, int nrhs, int shifted,
                            void* cuda_stream);

/* Number of kernels hz_solve has launched on this context so far (direct
 * launches plus the kernel nodes of every replayed restart-cycle graph;
 * kernels of an iteration skipped on the device after convergence count). */
hz_status hz_kernel_launches(const hz_ctx* ctx, int64_t* count);

/* Measurement hooks.  hz_profile_select makes every later hz_solve on this
 * context record CUDA events around each launch of one kernel class:
 *   0 none, 1 the Gram-Schmidt update passes, 2 the Gram-Schmidt pass with the
 *   FP64 operator apply and the inner products, 3 the whole V-cycle.
 * Only launches of inner iterations that did work are counted.  The restart
 * cycle graph is re-captured with the events; the overhead is two event
 * records per bracketed launch.  hz_profile_read returns the accumulated
 * device time, launch count, and the algorithmic bytes and FP64 flops of
 * those launches (per-node counts documented with each kernel).  Selecting a
 * class resets the accumulators. */
hz_status hz_profile_select(hz_ctx* ctx, int kernel_class);
hz_status hz_profile_read(const hz_ctx* ctx, double* total_ms, int64_t* launches, double* bytes, double* flops);

/* Checked-index debug build (no counterpart in the paper; the stand-in for
 * a memory checker, which this library's test machines do not offer).
 * libhz_checked.so is the same library compiled with every instrumented
 * global access of the solve's kernels testing its element index against
 * the array's extent; an index outside the array is counted, the first one
 * recorded (source line << 40 | low 40 bits of the index in *first), and the
 * access moved to element 0 of the array, so a kernel never traps.
 * hz_check_status: *enabled = 1 in that build (0 in the normal one, where
 * the counts stay 0), *failures the out-of-extent accesses since the last
 * clear, summed over the library's translation units; clear != 0 resets
 * them.  Call it with no kernel of the library in flight. */
hz_status hz_check_status(int* enabled, uint64_t* failures, uint64_t* first, int clear);

/* The bounded device wait on its own (no counterpart in the paper; the test
 * of the failure path that every spin-wait of the tensor-core kernels
 * takes).  One thread waits up to `polls` (1..2^24) times for a phase of a
 * fresh mbarrier; with arrive = 0 nothing arrives, so the wait gives up:
 * *timed_out = 1 and HZ_ERR_TIMEOUT, the status the coarsest product returns
 * when its copies or MMAs do not complete.  arrive != 0: the thread arrives
 * first, *timed_out = 0, HZ_OK.  Synchronizes a private stream; the device
 * stays usable either way. */
hz_status hz_check_wait_timeout(long long polls, int arrive, int* timed_out);

/* Measured arithmetic peak of the current device, the denominator of the
 * roofline fraction of the FP64 Krylov passes.  No counterpart in the paper:
 * a measurement hook.  kind 0: FP64 fused multiply-add (DFMA); kind 1: FP32
 * (FFMA).  Every thread of a whole number of waves (SMs x resident blocks of
 * 256 threads) runs independent multiply-add chains with no memory traffic,
 * in two forms (8 chains sharing their operands; 16 chains with their own);
 * the best of five launches of either form (about 20 ms each), timed with
 * CUDA events after two warm-up launches, gives *tflops (2 flops per FMA) and
 * *ms (that launch's time; may be NULL).  Allocates and frees a small device buffer on a private stream
 * and synchronizes it.  HZ_ERR_INVALID_ARG for another kind or a NULL
 * tflops; HZ_ERR_NO_DEVICE without a device. */
hz_status hz_measure_peak(int kind, double* tflops, double* ms);

/* ---- component entry points (one row of the method each) ---------------
 * Level fields are device arrays in the context's V-cycle precision (c128
 * for HZ_PREC_FP64, c64 for HZ_PREC_MIXED) of the level's node count. */

/* Device memory in use, for tests and monitoring (no counterpart in the
 * paper).  *pool_used_bytes: bytes currently in use in the default
 * stream-ordered pool of `device` (every context allocates from it);
 * *device_allocations: device allocations the library has made in this
 * process so far, all devices.  Either output may be NULL.
 * HZ_ERR_INVALID_ARG for a bad ordinal; HZ_ERR_NO_DEVICE without a device. */
hz_status hz_memory_stats(int device, uint64_t* pool_used_bytes, uint64_t* device_allocations);

/* The context's CUDA device ordinal, V-cycle precision (so the element type
 * of level fields: c64 for HZ_PREC_MIXED, c128 for HZ_PREC_FP64) and the
 * widest batch it was set up for; any output pointer may be NULL. */
hz_status hz_context_info(const hz_ctx* ctx, int* device, int* precision, int* nrhs_max);

hz_status hz_level_count(const hz_ctx* ctx, int* levels);
hz_status hz_level_describe(const hz_ctx* ctx, int level, hz_level_desc* out);

/* Copy a level's stencil planes to host as c128 [size][nodes] (plane-major):
 * what = 0: shifted Galerkin operator A_s^level (Section 3.1); what = 1: the
 * assembled Vanka sum sum_i V_i^T W_i H_i^{-1} V_i (Eq. smoother, no damping).
 * The FP64 values computed at setup are returned for both precisions. */
hz_status hz_level_export(const hz_ctx* ctx, int level, int what, void* host_out);

/* r = f - A_s^level u. */
hz_status hz_level_residual(hz_ctx* ctx, int level, const void* u, const void* f, void* r,
                            void* cuda_stream);
/* One additive Vanka relaxation (Eq. smoother): u += w M (f - A_s u). */
hz_status hz_level_smooth(hz_ctx* ctx, int level, void* u, const void* f, void* cuda_stream);
/* Allocation-free variant of hz_level_smooth.  The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory
 * on the call path, e.g. code whose device memory is fully reserved up
 * front by another allocator or by a fixed per-process budget, where a
 * cudaMalloc could fail or fragment that reservation.  It computes the same
 * sweep, u += w M (f - A_s u), but keeps the level residual in scratch that
 * the library holds in static device memory (4 MiB per GPU that loads the
 * library, held until the process exits) instead of the context's buffer;
 * it calls no cudaMalloc, cudaFree or other allocating routine.
 *   - The level may have at most HZ_NOALLOC_MAX_NODES nodes; larger levels
 *     return HZ_ERR_INVALID_ARG with a message.
 *   - The scratch address is looked up on the first call on each device
 *     (with that device made current); make that first call before any
 *     stream capture.
 *   - All calls share the one scratch array and it keeps the last call's
 *     contents.  Nothing in it needs clearing (the residual overwrites it
 *     before use), but calls whose work overlaps on the GPU race on it:
 *     order them on one stream or synchronise between them. */
#define HZ_NOALLOC_MAX_NODES 262144
hz_status hz_level_smooth_noalloc(hz_ctx* ctx, int level, void* u, const void* f, void* cuda_stream);
/* fc = R_level r (to level+1). */
hz_status hz_level_restrict(hz_ctx* ctx, int level, const void* r, void* fc, void* cuda_stream);
/* u += P_level ec (from level+1). */
hz_status hz_level_prolong_add(hz_ctx* ctx, int level, const void* ec, void* u, void* cuda_stream);
/* u = (A_s^L)^{-1} f on the coarsest level L (dense inverse from setup). */
hz_status hz_coarse_solve(hz_ctx* ctx, const void* f, void* u, void* cuda_stream);
/* U = (A_s^L)^{-1} F for nrhs right-hand sides (a power of two <= nrhs_max;
 * fields node-major, RHS innermost, in the V-cycle precision) with a chosen
 * variant of the product (Algorithm 1 step 3 at a batch width):
 *   variant 0   CUDA-core complex GEMM;
 *   variant s   (1 <= s <= 8) tcgen05 tensor cores, tf32 with the 3xTF32 split
 *               and FP32 accumulation, K split over s CTAs per row tile
 *               (mixed precision and nrhs = 16, 32 or 64 only);
 *   variant -1  the context's current choice (hz_autotune, else the default).
 * HZ_ERR_INVALID_ARG for a variant the context cannot run. */
hz_status hz_coarse_solve_batch(hz_ctx* ctx, const void* f, void* u, int nrhs, int variant, void* cuda_stream);

/* ---- autotuning of kernel choices --------------------------------------
 * No counterpart in the paper: these choose how V-cycle steps run on this
 * GPU, never what they compute.  hz_autotune times every candidate of every
 * knob of the context for batch width nrhs (a few repetitions between CUDA
 * events on the context's own level vectors, which it overwrites: call it
 * between solves), keeps the fastest on the context and reports them all.
 * Knobs (kind, candidate values = what hz_tune_set takes):
 *   0  coarsest product (level = coarsest): 0 CUDA-core GEMM, or the tcgen05
 *      tensor-core GEMM with K split 1, 2, 4, 8 or 16 ways (mixed, nrhs 16..64)
 *   1  RHS pack of a level's kernels (nrhs >= 4): 1 one value per thread,
 *      2 packs of 32 bytes per thread
 *   2  register budget of a level's one-RHS kernels: 0 full occupancy,
 *      2 two blocks per SM (all of a node's stencil loads in flight)
 *   3  a small coarse 2D level as two fused tile passes (1) or as five
 *      separate kernels (0)
 * Without tuning, fixed rules decide (batch width, level size).  Captured
 * restart-cycle graphs are dropped so the next solve uses the choices.
 *   reps      repetitions per candidate (1..1000)
 *   entries   host array of cap entries (may be NULL when cap = 0)
 *   n         out: entries produced (may exceed cap) */
typedef struct {
  int kind;       /* 0..3 as above */
  int level;      /* level the knob belongs to */
  int nrhs;       /* batch width it was timed at */
  int candidate;  /* candidate value */
  double us;      /* device time per repetition, microseconds */
  int chosen;     /* 1 for the candidate kept */
} hz_tune_entry;
hz_status hz_autotune(hz_ctx* ctx, int nrhs, int reps, hz_tune_entry* entries, int cap, int* n);
/* Applies one stored choice (e.g. from a cache of an earlier hz_autotune of
 * the same level shapes); HZ_ERR_INVALID_ARG for a knob or value that does not
 * apply to the level. */
hz_status hz_tune_set(hz_ctx* ctx, int kind, int level, int nrhs, int candidate);

/* ---- per-solve metrics -------------------------------------------------- */

/* Wall time of hz_setup for this context, seconds (host clock around the whole
 * call, device work included). */
hz_status hz_setup_seconds(const hz_ctx* ctx, double* seconds);

/* Convergence history of the last single-RHS solve on the context (hz_solve
 * with nrhs = 1, or hz_solve_begin/step/end): one entry per status read, that
 * is the start and the end of every restart cycle, each with the iteration
 * count so far, the true relative residual ||q_hat - A p|| / ||q_hat|| (FP64,
 * formed at restarts) and the Arnoldi estimate.  A batched solve clears it.
 *   cap        capacity of the output arrays (host); entries beyond it are dropped
 *   iters, relres_true, relres_est   host arrays of cap values, each may be NULL
 *   n          out: entries recorded (may exceed cap)
 * Call it from the thread that drives the context, or when no solve is in
 * flight on it (hz_solve_step appends to the history). */
hz_status hz_solve_history(const hz_ctx* ctx, int cap, int* iters, double* relres_true, double* relres_est,
                           int* n);

/* ---- tuning tools (Section 5.2) ---------------------------------------- */

/* Convergence factor of Eq. cf (Section 5.1) of the context's cycle used as a
 * stationary solver for the shifted fine operator, u <- u + B(f - A_s u):
 * after `warmup` iterations, iterate until ||r_k|| / ||r_init|| <= target or
 * max_iter iterations; factor = (||r_k|| / ||r_warmup||)^(1/k), 0 if k = 0.
 *   f, u     device, complex128, one value per fine node; u holds the initial
 *            guess on entry and the last iterate on return
 *   iters    out: k
 * The residual norm is read back after every iteration (synchronous on the
 * stream).  In a mixed-precision context the cycle runs in complex FP32, so
 * the residual stalls near FP32 rounding: use HZ_PREC_FP64 for targets below
 * about 1e-6.  Uses the context's Krylov buffers as scratch: no solve may be in
 * flight on the context.  Errors: HZ_ERR_INVALID_ARG (null pointers,
 * warmup < 0, max_iter < 1, target not in (0, 1)), HZ_ERR_BUSY. */
hz_status hz_cycle_factor(hz_ctx* ctx, const void* f, void* u, int warmup, double target, int max_iter,
                          double* factor, int* iters, void* cuda_stream);

/* Local Fourier analysis of additive Vanka for a constant stencil (Section 4),
 * for nw damping values in one sweep on the current device:
 *   stencil  host, 3^dim complex values (re, im interleaved) of the stencil on
 *            the box {-1,0,1}^dim, entry (dx, dy[, dz]) at
 *            (dz+1)*9 + (dy+1)*3 + (dx+1) (no dz term in 2D); its symbol is
 *            H~(θ) = Σ_d s_d e^{iθ·d}
 *   patch    the Vanka patch (Section 3.2), equal weights 1/N (Eq. smoother_symbol)
 *   w, nw    host, damping values, 1 <= nw <= 1024
 *   rk, pk   HZ_IG_LINEAR ((1 + cos t)/2 per axis) or HZ_IG_CUBIC
 *            ((3 + 4 cos t + cos 2t)/8 per axis) restriction / prolongation
 *            symbols (Section 4.2); the coarse symbol is Galerkin
 *   nu1, nu2 relaxations in the two-grid symbol (Eq. symbolTG)
 *   samples  points per axis: mu is the max of |S~| over the mesh
 *            θ_a = -π/2 + 2π i/samples restricted to high frequencies (some
 *            θ_a >= π/2), Definition 2.1; rho the max spectral radius of TG~
 *            over the mesh θ_a = -π/2 + π i/samples (low frequencies),
 *            Definition 2.2; 2 <= samples <= 4096 (2D) / 256 (3D)
 *   mu, rho  host out, nw values each; either may be NULL; rho is NaN where
 *            the eigenvalue iteration did not converge
 * Synchronous.  Errors: HZ_ERR_INVALID_ARG (sizes, kinds, non-finite input,
 * singular patch matrix), HZ_ERR_NO_DEVICE, HZ_ERR_CUDA. */
hz_status hz_lfa_factors(int dim, const double* stencil, hz_patch patch, const double* w, int nw, hz_intergrid rk,
                         hz_intergrid pk, int nu1, int nu2, int samples, double* mu, double* rho);

#ifdef __cplusplus
}
#endif
#endif /* HZ_H */
