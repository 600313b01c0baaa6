// Serving loop: continuous batching of independent Helmholtz solves on one GPU
// (the paper has no counterpart; it serves many sources / frequencies / media
// through the same solver).
//
// A request carries a full problem (grid, medium, frequency, shift, solver
// options, one source).  hz_server_submit copies it and queues it; three
// host threads then run it through the C ABI:
//   setup   (one or more threads) admits queued requests in arrival order
//           while the HBM budget and the slot count allow (Admission below),
//           builds each hierarchy on the request's own stream (hz_setup) and
//           starts its solve (hz_solve_begin); several setups overlap;
//   step    keeps every started solve going: each pass polls the status event
//           of each request's last restart cycle and queues its next cycle (a
//           captured graph) as soon as the previous one has finished, so the
//           cycles of all admitted requests overlap on the device;
//   retire  copies finished solutions to the caller's buffers (hz_solve_end),
//           frees the hierarchy (hz_destroy) and returns its bytes to the
//           budget, which lets the setup thread admit the next request.
// Requests are independent: a request that fails (bad medium, out of memory,
// no convergence) records its status and releases its slot; the others go on.
//
// Grouping (group_max >= 2): when a request is admitted, the queued requests
// of the same problem (same grid, medium, frequency, shift and options; only
// the source differs) join it up to a power of two; the group shares one
// hierarchy and is solved as one multi-RHS solve (one batched V-cycle per
// FGMRES iteration for all of them) in the setup thread, and the retire
// thread hands every member its solution.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "server_policy.h"

namespace hz {
namespace {

// FIFO admission under a byte budget and a slot limit.  Arrival order is kept
// (no overtaking), so a large request cannot be starved by small ones; a
// request larger than the whole budget is refused at submission.
struct Admission {
  size_t budget = 0, in_use = 0, peak = 0;
  int max_active = 1, active = 0;
  std::deque<std::pair<uint64_t, size_t>> queue;

  bool offer(uint64_t ticket, size_t bytes) {
    if (bytes > budget) return false;
    queue.emplace_back(ticket, bytes);
    return true;
  }
  bool next(uint64_t* ticket) {
    if (queue.empty() || active >= max_active || in_use + queue.front().second > budget) return false;
    *ticket = queue.front().first;
    in_use += queue.front().second;
    peak = std::max(peak, in_use);
    ++active;
    queue.pop_front();
    return true;
  }
  void release(size_t bytes) {
    in_use -= std::min(in_use, bytes);
    if (active > 0) --active;
  }
};

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  hz_grid grid{};
  hz_opts opts{};
  double omega = 0, alpha = 0, gamma0 = 0;
  std::vector<double> kappa, gamma;
  std::vector<double2> q;
  void* p_out = nullptr;
  size_t bytes = 0;
  int state = HZ_REQ_QUEUED;
  hz_status status = HZ_OK;
  hz_info info{};
  std::string message;
  double t_submit = 0, t_admit = 0, t_start = 0, t_done = 0;
  hz_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  // grouping of requests of the same problem
  uint64_t key = 0;                 // identity of the problem without its source (0: never grouped)
  Request* lead = nullptr;          // a grouped request: the request whose solve serves it
  std::vector<Request*> members;    // the lead of a group: every member, itself first
  int group_size = 1;
  size_t held = 0;                  // bytes held in the admission (a lead: the group's)
  bool solved = false;              // solved in the setup thread (a group): no hz_solve_end
};

long long grid_nodes(const hz_grid& g) {
  return (long long)g.n[0] * g.n[1] * (g.dim == 3 ? g.n[2] : 1);
}

bool opts_equal(const hz_opts& a, const hz_opts& b) {
  if (a.levels != b.levels || a.nu1 != b.nu1 || a.nu2 != b.nu2 || a.intergrid != b.intergrid ||
      a.precision != b.precision || a.restart_m != b.restart_m || a.tol != b.tol || a.max_iter != b.max_iter ||
      a.cycle_visits != b.cycle_visits || a.stencil != b.stencil)
    return false;
  for (int l = 0; l < HZ_MAX_LEVELS; ++l)
    if (a.patch[l] != b.patch[l] || a.damping[l] != b.damping[l]) return false;
  return true;
}

// Identity of a request's problem apart from its source: grid, frequency,
// shift, solver options and every value of the medium (a multiply-xor hash;
// equal keys are confirmed value by value before two requests share a solve).
uint64_t problem_key(const Request& r) {
  uint64_t h = 0x243f6a8885a308d3ull;
  auto word = [&](uint64_t w) {
    h = (h ^ w) * 0x9e3779b97f4a7c15ull;
    h ^= h >> 31;
  };
  auto real = [&](double d) {
    uint64_t w;
    std::memcpy(&w, &d, sizeof w);
    word(w);
  };
  word((uint64_t)r.grid.dim);
  for (int a = 0; a < 3; ++a) word((uint64_t)r.grid.n[a]);
  real(r.grid.h);
  real(r.omega);
  real(r.alpha);
  real(r.gamma0);
  const hz_opts& o = r.opts;
  for (int v : {o.levels, o.nu1, o.nu2, (int)o.intergrid, (int)o.precision, o.restart_m, o.max_iter, o.cycle_visits,
                o.stencil})
    word((uint64_t)(uint32_t)v);
  real(o.tol);
  for (int l = 0; l < HZ_MAX_LEVELS; ++l) {
    word((uint64_t)o.patch[l]);
    real(o.damping[l]);
  }
  for (double v : r.kappa) real(v);
  word(r.gamma.size());
  for (double v : r.gamma) real(v);
  return h ? h : 1;
}

bool same_problem(const Request& a, const Request& b) {
  return a.key == b.key && a.grid.dim == b.grid.dim && a.grid.n[0] == b.grid.n[0] && a.grid.n[1] == b.grid.n[1] &&
         a.grid.n[2] == b.grid.n[2] && a.grid.h == b.grid.h && a.omega == b.omega && a.alpha == b.alpha &&
         a.gamma0 == b.gamma0 && opts_equal(a.opts, b.opts) && a.kappa == b.kappa && a.gamma == b.gamma;
}

}  // namespace
}  // namespace hz

using namespace hz;

struct hz_sched {
  Admission a;
};

struct hz_server {
  int dev = 0;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_setup, cv_step, cv_retire, cv_done;
  Admission adm;
  uint64_t next_ticket = 1;
  std::map<uint64_t, std::unique_ptr<Request>> reqs;
  std::vector<Request*> running;           // started solves (step thread)
  std::deque<Request*> retiring;           // finished or failed after admission (retire thread)
  int setting_up = 0;
  bool stop = false;
  std::atomic<int64_t> launches{0};        // kernels launched by finished requests
  int group_max = 0;                       // >= 2: requests of the same problem solved together
  int groups = 0, grouped = 0;             // solves serving several requests, and those requests
  std::vector<std::thread> t_setup;
  std::thread t_step, t_retire;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

hz_status record(Request* r, hz_status st) {
  r->status = st;
  if (st != HZ_OK && st != HZ_ERR_NOT_CONVERGED) r->message = hz_last_error();
  return st;
}

// Device bytes of a request's context for nrhs_max right-hand sides: the
// hierarchy and Krylov workspace, the staged medium, the staged sources and
// slack for graphs.
size_t request_bytes(const hz_grid& g, const hz_opts& o, int nrhs_max) {
  hz_opts oo = o;
  oo.nrhs_max = nrhs_max;
  size_t bytes = 0;
  const hz_status sb = hz_setup_bytes(&g, &oo, &bytes);
  if (sb != HZ_OK) throw Error(sb, hz_last_error());
  const long long N = grid_nodes(g);
  return bytes + (size_t)N * (2 * sizeof(double) + sizeof(double2) * nrhs_max) + (8u << 20);
}

// Called with the server's lock held, for the request r just admitted: the
// queued requests of the same problem (arrival order) join it, as many as
// make a power of two with r, at most group_max, whose host staging (N x size
// c128 sources and solutions) stays within 1 GiB and whose bytes fit the
// budget.  They leave the queue, hold no slot and no bytes of their own; r
// holds the group's bytes.
void form_group(hz_server* S, Request* r) {
  if (S->group_max < 2 || r->key == 0) return;
  const int cap = group_cap(S->group_max, grid_nodes(r->grid));
  std::vector<Request*> cand;
  for (const auto& e : S->adm.queue) {
    if ((int)cand.size() + 1 >= cap) break;
    Request* m = S->reqs[e.first].get();
    if (m->key == r->key && same_problem(*r, *m)) cand.push_back(m);
  }
  size_t bytes = 0;
  const int k = group_size_for((int)cand.size(), S->adm.in_use, r->held, S->adm.budget,
                               [&](int kk) { return request_bytes(r->grid, r->opts, kk); }, &bytes);
  if (k < 2) return;                                // kept alone
  cand.resize(k - 1);
  r->members.assign(1, r);
  for (Request* m : cand) {
    for (auto it = S->adm.queue.begin(); it != S->adm.queue.end(); ++it)
      if (it->first == m->ticket) {
        S->adm.queue.erase(it);
        break;
      }
    m->lead = r;
    m->state = HZ_REQ_SETUP;
    m->t_admit = S->now();
    m->held = 0;
    r->members.push_back(m);
  }
  S->adm.in_use = S->adm.in_use - r->held + bytes;
  S->adm.peak = std::max(S->adm.peak, S->adm.in_use);
  r->held = bytes;
  for (Request* m : r->members) m->group_size = k;
  ++S->groups;
  S->grouped += k;
}

// The group of r as one multi-RHS solve on the context r->ctx (set up for
// r->members.size() right-hand sides): sources interleaved RHS-innermost,
// solutions and infos handed back to each member.
hz_status solve_group(hz_server* S, Request* r) {
  const int R = (int)r->members.size();
  const long long N = grid_nodes(r->grid);
  std::vector<double2> Q((size_t)N * R), P((size_t)N * R);
  for (int k = 0; k < R; ++k) {
    const double2* q = r->members[k]->q.data();
    for (long long p = 0; p < N; ++p) Q[(size_t)p * R + k] = q[p];
  }
  std::vector<hz_info> info(R);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    const double t = S->now();
    for (Request* m : r->members) {
      m->state = HZ_REQ_SOLVING;
      m->t_start = t;
    }
  }
  const hz_status st = hz_solve(r->ctx, Q.data(), P.data(), R, info.data(), r->stream);
  if (st != HZ_OK && st != HZ_ERR_NOT_CONVERGED) return st;
  for (int k = 0; k < R; ++k) {
    double2* out = (double2*)r->members[k]->p_out;
    for (long long p = 0; p < N; ++p) out[p] = P[(size_t)p * R + k];
  }
  // statuses under the lock, as hz_server_poll reads them
  std::lock_guard<std::mutex> lk(S->mu);
  for (int k = 0; k < R; ++k) {
    Request* m = r->members[k];
    m->info = info[k];
    m->status = info[k].converged ? HZ_OK : HZ_ERR_NOT_CONVERGED;
  }
  return HZ_OK;
}

void setup_loop(hz_server* S) {
  cudaSetDevice(S->dev);
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      uint64_t t = 0;
      S->cv_setup.wait(lk, [&] { return S->stop || S->adm.next(&t); });
      if (t == 0) {
        // stop requested: drain what is still admissible, then leave
        if (!S->adm.next(&t)) {
          if (S->adm.queue.empty()) return;
          S->cv_setup.wait_for(lk, std::chrono::milliseconds(1));
          continue;
        }
      }
      r = S->reqs[t].get();
      r->state = HZ_REQ_SETUP;
      r->t_admit = S->now();
      r->held = r->bytes;
      form_group(S, r);
      ++S->setting_up;
    }
    const bool group = r->members.size() > 1;
    hz_opts o = r->opts;
    if (group) o.nrhs_max = (int)r->members.size();
    hz_status st = HZ_OK;
    if (cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) != cudaSuccess) {
      (void)cudaGetLastError();
      r->stream = nullptr;
      r->message = "cudaStreamCreate failed";
      st = HZ_ERR_CUDA;
    }
    if (st == HZ_OK)
      st = record(r, hz_setup(&r->grid, r->kappa.data(), r->omega, r->gamma.empty() ? nullptr : r->gamma.data(),
                              r->gamma0, r->alpha, &o, r->stream, &r->ctx));
    if (st == HZ_OK && group) {
      // the whole group is solved here; the retire thread hands it out
      const hz_status gs = solve_group(S, r);      // sets each member's own status
      if (gs != HZ_OK) record(r, gs);
      std::lock_guard<std::mutex> lk(S->mu);
      --S->setting_up;
      r->solved = true;
      if (gs != HZ_OK) r->state = HZ_REQ_FAILED;
      S->retiring.push_back(r);
      S->cv_retire.notify_one();
      continue;
    }
    if (st == HZ_OK) st = record(r, hz_solve_begin(r->ctx, r->q.data(), r->stream));
    std::lock_guard<std::mutex> lk(S->mu);
    --S->setting_up;
    r->status = st;
    if (st == HZ_OK) {
      r->state = HZ_REQ_SOLVING;
      r->t_start = S->now();
      S->running.push_back(r);
      S->cv_step.notify_one();
    } else {
      r->state = HZ_REQ_FAILED;
      S->retiring.push_back(r);
      S->cv_retire.notify_one();
    }
  }
}

void step_loop(hz_server* S) {
  cudaSetDevice(S->dev);
  std::vector<Request*> mine;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_step.wait(lk, [&] {
        return !S->running.empty() || !mine.empty() ||
               (S->stop && S->adm.queue.empty() && S->setting_up == 0);
      });
      for (Request* r : S->running) mine.push_back(r);
      S->running.clear();
      if (mine.empty() && S->stop && S->adm.queue.empty() && S->setting_up == 0) return;
    }
    std::vector<Request*> finished;
    for (size_t i = 0; i < mine.size();) {
      Request* r = mine[i];
      int done = 0;
      const hz_status st = hz_solve_step(r->ctx, 0, &done);
      if (st != HZ_OK) {
        record(r, st);
        r->state = HZ_REQ_FAILED;
        done = 1;
      }
      if (done) {
        finished.push_back(r);
        mine[i] = mine.back();
        mine.pop_back();
      } else {
        ++i;
      }
    }
    if (!finished.empty()) {
      std::lock_guard<std::mutex> lk(S->mu);
      for (Request* r : finished) S->retiring.push_back(r);
      S->cv_retire.notify_one();
    } else if (!mine.empty()) {
      // every in-flight cycle is still running: poll again shortly
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  }
}

void retire_loop(hz_server* S) {
  cudaSetDevice(S->dev);
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_retire.wait(lk, [&] {
        return !S->retiring.empty() ||
               (S->stop && S->adm.queue.empty() && S->setting_up == 0 && S->running.empty() && S->adm.active == 0);
      });
      if (S->retiring.empty()) return;
      r = S->retiring.front();
      S->retiring.pop_front();
    }
    if (r->state == HZ_REQ_SOLVING && !r->solved) {
      const hz_status st = hz_solve_end(r->ctx, r->p_out, &r->info, r->stream);
      if (st != HZ_OK && st != HZ_ERR_NOT_CONVERGED) record(r, st);
      else r->status = st;
    }
    int64_t nl = 0;
    if (r->ctx && hz_kernel_launches(r->ctx, &nl) == HZ_OK) S->launches.fetch_add(nl);
    if (r->ctx) hz_destroy(r->ctx);
    r->ctx = nullptr;
    if (r->stream) cudaStreamDestroy(r->stream);
    r->stream = nullptr;
    // a group's members share the lead's outcome (a failure) or carry their
    // own status from the batched solve
    for (Request* m : r->members) {
      if (m == r) continue;
      if (r->state == HZ_REQ_FAILED) {
        m->status = r->status;
        m->message = r->message;
        m->state = HZ_REQ_FAILED;
      }
      std::vector<double>().swap(m->kappa);
      std::vector<double>().swap(m->gamma);
      std::vector<double2>().swap(m->q);
    }
    std::vector<double>().swap(r->kappa);
    std::vector<double>().swap(r->gamma);
    std::vector<double2>().swap(r->q);
    std::lock_guard<std::mutex> lk(S->mu);
    r->t_done = S->now();
    if (r->state != HZ_REQ_FAILED) r->state = HZ_REQ_DONE;
    for (Request* m : r->members) {
      if (m == r) continue;
      m->t_done = r->t_done;
      if (m->state != HZ_REQ_FAILED) m->state = HZ_REQ_DONE;
    }
    S->adm.release(r->held);
    S->cv_setup.notify_one();
    S->cv_step.notify_one();
    S->cv_retire.notify_one();
    S->cv_done.notify_all();
  }
}

void fill(const Request& r, hz_ticket_info* out) {
  out->state = r.state;
  out->status = r.status;
  out->info = r.info;
  out->t_submit = r.t_submit;
  out->t_admit = r.t_admit;
  out->t_start = r.t_start;
  out->t_done = r.t_done;
  out->bytes = r.bytes;
  std::memset(out->message, 0, sizeof(out->message));
  std::strncpy(out->message, r.message.c_str(), sizeof(out->message) - 1);
  out->group_size = r.group_size;
}

bool finished(int state) { return state == HZ_REQ_DONE || state == HZ_REQ_FAILED; }

}  // namespace

extern "C" {

// ---- admission policy alone (host logic, no device)
hz_status hz_sched_create(size_t budget, int max_active, hz_sched** out) {
  return guarded([&] {
    require(out && max_active >= 1, "bad scheduler arguments");
    *out = new hz_sched();
    (*out)->a.budget = budget;
    (*out)->a.max_active = max_active;
  });
}
hz_status hz_sched_offer(hz_sched* s, uint64_t ticket, size_t bytes, int* accepted) {
  return guarded([&] {
    require(s && accepted, "null argument");
    *accepted = s->a.offer(ticket, bytes) ? 1 : 0;
  });
}
hz_status hz_sched_next(hz_sched* s, uint64_t* ticket, int* admitted) {
  return guarded([&] {
    require(s && ticket && admitted, "null argument");
    *admitted = s->a.next(ticket) ? 1 : 0;
  });
}
hz_status hz_sched_release(hz_sched* s, size_t bytes) {
  return guarded([&] {
    require(s, "null argument");
    s->a.release(bytes);
  });
}
hz_status hz_sched_state(const hz_sched* s, size_t* in_use, size_t* peak, int* active, int* queued) {
  return guarded([&] {
    require(s && in_use && peak && active && queued, "null argument");
    *in_use = s->a.in_use;
    *peak = s->a.peak;
    *active = s->a.active;
    *queued = (int)s->a.queue.size();
  });
}
hz_status hz_sched_destroy(hz_sched* s) {
  delete s;
  return HZ_OK;
}

// ---- server
hz_status hz_server_create(const hz_server_opts* opts, hz_server** out) {
  hz_server* S = nullptr;
  hz_status st = guarded([&] {
    require(out != nullptr, "null output");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
      (void)cudaGetLastError();
      throw Error(HZ_ERR_NO_DEVICE, "no CUDA device");
    }
    S = new hz_server();
    S->t0 = Clock::now();
    if (opts && opts->device >= 0) {
      require(opts->device < ndev, "device out of range");
      S->dev = opts->device;
    } else {
      HZ_CUDA(cudaGetDevice(&S->dev));
    }
    HZ_CUDA(cudaSetDevice(S->dev));
    size_t fr = 0, tot = 0;
    HZ_CUDA(cudaMemGetInfo(&fr, &tot));
    S->adm.budget = (opts && opts->hbm_budget) ? opts->hbm_budget : (size_t)(0.8 * (double)fr);
    S->adm.max_active = (opts && opts->max_active > 0) ? opts->max_active : 32;
    const int gm = opts ? opts->group_max : 0;
    require(gm <= 1 || (gm <= 64 && (gm & (gm - 1)) == 0), "group_max must be 0, 1 or a power of two <= 64");
    S->group_max = gm >= 2 ? gm : 0;
    const int nsetup = (opts && opts->setup_threads > 0) ? std::min(opts->setup_threads, 8) : 2;
    for (int i = 0; i < nsetup; ++i) S->t_setup.emplace_back(setup_loop, S);
    S->t_step = std::thread(step_loop, S);
    S->t_retire = std::thread(retire_loop, S);
  });
  if (st != HZ_OK) {
    delete S;
    return st;
  }
  *out = S;
  return HZ_OK;
}

hz_status hz_server_submit(hz_server* S, const hz_request* req, uint64_t* ticket) {
  return guarded([&] {
    require(S && req && ticket, "null argument");
    require(req->kappa && req->q && req->p, "request needs kappa, q and p");
    size_t bytes = 0;
    const hz_status sb = hz_setup_bytes(&req->grid, &req->opts, &bytes);
    if (sb != HZ_OK) throw Error(sb, hz_last_error());
    require(req->opts.nrhs_max == 1, "served requests carry one right-hand side");
    const long long N = (long long)req->grid.n[0] * req->grid.n[1] * (req->grid.dim == 3 ? req->grid.n[2] : 1);
    // hierarchy + Krylov workspace, the staged medium and source, graph and slack
    bytes += (size_t)N * (2 * sizeof(double) + sizeof(double2)) + (8u << 20);
    auto r = std::make_unique<Request>();
    r->grid = req->grid;
    r->opts = req->opts;
    r->omega = req->omega;
    r->alpha = req->shift_alpha;
    r->gamma0 = req->gamma0;
    r->kappa.assign(req->kappa, req->kappa + N);
    if (req->gamma) r->gamma.assign(req->gamma, req->gamma + N);
    const double2* q = (const double2*)req->q;
    r->q.assign(q, q + N);
    r->p_out = req->p;
    r->bytes = bytes;
    // grouped solves run batched: one right-hand side stencils and restarts
    // longer than 16 stay alone
    if (S->group_max >= 2 && req->opts.stencil != 1 && req->opts.restart_m <= 16) r->key = problem_key(*r);
    std::lock_guard<std::mutex> lk(S->mu);
    require(!S->stop, "server is shutting down");
    r->ticket = S->next_ticket++;
    r->t_submit = S->now();
    if (!S->adm.offer(r->ticket, bytes))
      throw Error(HZ_ERR_OOM, "request needs " + std::to_string(bytes) + " bytes, more than the server's budget");
    *ticket = r->ticket;
    S->reqs[r->ticket] = std::move(r);
    S->cv_setup.notify_one();
  });
}

hz_status hz_server_poll(hz_server* S, uint64_t ticket, hz_ticket_info* out) {
  return guarded([&] {
    require(S && out, "null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    require(it != S->reqs.end(), "unknown ticket");
    fill(*it->second, out);
  });
}

hz_status hz_server_wait(hz_server* S, uint64_t ticket, double timeout_s, hz_ticket_info* out) {
  return guarded([&] {
    require(S && out, "null argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    require(it != S->reqs.end(), "unknown ticket");
    Request* r = it->second.get();
    const auto pred = [&] { return finished(r->state); };
    if (timeout_s < 0) S->cv_done.wait(lk, pred);
    else S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred);
    fill(*r, out);
    if (!finished(r->state)) throw Error(HZ_ERR_TIMEOUT, "request still running");
  });
}

hz_status hz_server_stats(hz_server* S, hz_server_counters* out) {
  return guarded([&] {
    require(S && out, "null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(out, 0, sizeof(*out));
    for (auto& kv : S->reqs) {
      switch (kv.second->state) {
        case HZ_REQ_QUEUED: ++out->queued; break;
        case HZ_REQ_SETUP: ++out->setting_up; break;
        case HZ_REQ_SOLVING: ++out->solving; break;
        case HZ_REQ_DONE: ++out->done; break;
        default: ++out->failed; break;
      }
    }
    out->bytes_in_use = S->adm.in_use;
    out->peak_bytes = S->adm.peak;
    out->budget = S->adm.budget;
    out->max_active = S->adm.max_active;
    out->elapsed_s = S->now();
    out->kernel_launches = S->launches.load();
    out->groups = S->groups;
    out->grouped = S->grouped;
  });
}

hz_status hz_server_destroy(hz_server* S) {
  if (!S) return HZ_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_setup.notify_all();
  S->cv_step.notify_all();
  S->cv_retire.notify_all();
  // the threads drain every submitted request before they leave
  for (auto& t : S->t_setup)
    if (t.joinable()) t.join();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->cv_step.notify_all();
  }
  if (S->t_step.joinable()) S->t_step.join();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->cv_retire.notify_all();
  }
  if (S->t_retire.joinable()) S->t_retire.join();
  delete S;
  return HZ_OK;
}

}  // extern "C"
