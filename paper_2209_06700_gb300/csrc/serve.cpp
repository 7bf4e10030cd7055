// Continuous-batching request loop of libirk (irk_serve, declared in include/irk.h).
//
// Arrived requests wait.  A free slot (a host worker thread) takes the smallest waiting request
// (fewest stage-DoFs, the oldest among equals; or the oldest, by option) together with the other
// waiting requests of the same shape (dim, cells, degree, Q), up to the group limit, and runs them
// as one group: one handle whose stage-operator and
// V-cycle launches cover every member's stage vectors and blocks, with one FGMRES per member
// (irk_create_group / irk_step_group).  Handles are kept per shape and group size when idle and
// reused for later groups with irk_set_tau, which rebuilds only what depends on the step tau
// (Chebyshev intervals, coarse inverses); idle handles are evicted, least recently used first, when
// a new handle needs their memory.  Every handle has its own CUDA stream, so groups that arrive
// while others are on the GPU start as soon as a slot and memory are free and their kernels
// overlap on the device.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <list>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "irk.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

constexpr int kMaxGroupStages = 16;  // R Q of one group handle

// Device memory a request reserves: Krylov bases, stage vectors, multigrid levels and the
// transient Chebyshev-interval work vectors, with a 15% margin.
double estimate_bytes(const irk_request& r, const irk_options& o) {
  const double n1 = (double)r.degree * r.cells + 1.0;
  const double n = std::pow(n1, r.dim);
  const double ld = std::ceil(n / 64.0) * 64.0;
  const double Q = r.Q, ns = std::max(r.Q, 2);
  // mg_precision 0: FP64 from Q = 6 on, where the basis change of the preconditioner needs it
  const double eb = (o.mg_precision == 64 || (o.mg_precision == 0 && r.Q >= 6)) ? 8.0 : 4.0;
  double b = (2.0 * o.restart + 2.0) * Q * ld * 8.0;              // V, Z, work vector
  b += (5.0 * ns + 1.0) * ld * 8.0;                               // rhs, stages, M u, K u, T^{-1} rhs, K y
  b += 4.75 * Q * ld * eb * 8.0 / 7.0;                            // multigrid levels and transfer grids
  b += 4.0 * Q * ld * 8.0;                                        // Lanczos work vectors during setup
  if (o.variant == IRK_VARIANT_DIAG) b += (2.0 * o.restart + 2.0) * 2.0 * ld * 8.0 + 4.75 * Q * ld * eb;
  b += ld * 8.0;                                                  // y
  return 1.15 * b + (1 << 20);
}

bool same_shape(const irk_request& a, const irk_request& b) {
  return a.dim == b.dim && a.cells == b.cells && a.degree == b.degree && a.Q == b.Q;
}

// A handle of the cache: the shape of its requests (by a representative request), its group size,
// its stream and the memory charged for it.
struct Cached {
  irk_request shape{};
  int R = 0;
  irk_handle h = nullptr;
  cudaStream_t st = nullptr;
  double bytes = 0.0;
  long long last_use = 0;
  bool busy = false;
};

void release(Cached& c) {
  if (c.h) irk_destroy(c.h);
  if (c.st) {
    cudaStreamSynchronize(c.st);
    cudaStreamDestroy(c.st);
  }
  c.h = nullptr;
  c.st = nullptr;
}

}  // namespace

extern "C" void irk_default_serve_options(irk_serve_options* o) {
  if (!o) return;
  o->max_active = 16;
  o->mem_budget_bytes = 0.0;
  o->realtime = 1;
  irk_default_options(&o->solver);
  o->solver.restart = 16;
  // requests run concurrently: launch-shape timings taken while other requests' kernels share
  // the device would be noise, so served handles keep the cost model's shapes (or shapes tuned
  // earlier in the process)
  o->solver.autotune = 0;
  o->max_group = 0;
  o->reuse_handles = 1;
  o->smallest_first = 1;
}

extern "C" irk_status irk_serve(const irk_request* reqs, int count, const irk_serve_options* opt_in,
                                irk_result* results, double** out_host) {
  if (count < 0 || (count > 0 && (!reqs || !results))) return IRK_EINVAL;
  if (count == 0) return IRK_OK;
  irk_serve_options opt;
  if (opt_in) opt = *opt_in; else irk_default_serve_options(&opt);
  const int nslots = std::max(1, std::min(opt.max_active, 64));
  double budget = opt.mem_budget_bytes;
  if (!(budget > 0)) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return IRK_ECUDA;
    budget = 0.8 * (double)fr;
  }
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return IRK_ECUDA;
  // groups need the LU variant on the Cartesian mesh; handles are reusable with the LU variant
  const bool groups_ok = opt.solver.variant == IRK_VARIANT_LU && !(opt.solver.deform > 0);
  const bool reuse = opt.reuse_handles != 0 && opt.solver.variant == IRK_VARIANT_LU;

  std::vector<double> est(count), work(count);
  for (int i = 0; i < count; ++i) {
    work[i] = reqs[i].Q * std::pow((double)reqs[i].degree * reqs[i].cells - 1.0, reqs[i].dim);
    results[i] = irk_result();
    results[i].status = IRK_OK;
    est[i] = estimate_bytes(reqs[i], opt.solver);
    results[i].mem_bytes = est[i];
  }

  std::mutex mu;
  std::condition_variable cv;
  std::deque<int> pending;       // arrived, waiting for a slot
  std::list<Cached> cache;       // handles: busy ones and idle ones kept for reuse (stable addresses)
  double used = 0.0;             // memory charged for the handles in the cache
  int finished = 0, running = 0;
  long long clock_tick = 0;
  bool closing = false;
  std::vector<Clock::time_point> arrival(count);
  const Clock::time_point start = Clock::now();

  auto worker = [&]() {
    cudaSetDevice(device);
    for (;;) {
      std::vector<int> members;
      Cached* slot = nullptr;
      bool reused = false;
      double need = 0.0;
      std::vector<Cached> victims;
      {
        std::unique_lock<std::mutex> lock(mu);
        cv.wait(lock, [&] { return closing || !pending.empty(); });
        if (pending.empty()) break;
        // the oldest request (or the smallest, oldest among equals) and the waiting requests of its
        // shape, up to the group limit
        auto pick = pending.begin();
        if (opt.smallest_first)
          for (auto it = pending.begin(); it != pending.end(); ++it)
            if (work[*it] < work[*pick]) pick = it;
        const int i0 = *pick;
        pending.erase(pick);
        members.push_back(i0);
        const irk_request& sh = reqs[i0];
        int rmax = groups_ok ? std::max(1, kMaxGroupStages / std::max(1, sh.Q)) : 1;
        if (opt.max_group > 0) rmax = std::min(rmax, opt.max_group);
        for (auto it = pending.begin(); it != pending.end() && (int)members.size() < rmax;) {
          if (same_shape(reqs[*it], sh) && need + est[*it] <= budget) {
            members.push_back(*it);
            it = pending.erase(it);
          } else {
            ++it;
          }
        }
        for (int i : members) need += est[i];
        // shrink the group until it fits the whole budget (every member fits alone)
        while ((int)members.size() > 1 && need > budget) {
          need -= est[members.back()];
          pending.push_front(members.back());
          members.pop_back();
        }
        // an idle handle of this shape for fewer requests is reused rather than a new one created:
        // the group is cut to its size (the largest such handle)
        if (reuse) {
          int best = 0;
          for (const Cached& c : cache)
            if (!c.busy && same_shape(c.shape, sh) && c.R <= (int)members.size()) best = std::max(best, c.R);
          while (best > 0 && (int)members.size() > best) {
            need -= est[members.back()];
            pending.push_front(members.back());
            members.pop_back();
          }
        }
        const int R = (int)members.size();
        for (;;) {
          if (reuse)
            for (Cached& c : cache)
              if (!c.busy && c.R == R && same_shape(c.shape, sh)) {
                slot = &c;
                break;
              }
          if (slot) {
            reused = true;
            break;
          }
          if (used + need <= budget) break;
          // evict the least recently used idle handle, or wait for running groups to finish
          auto lru = cache.end();
          for (auto it = cache.begin(); it != cache.end(); ++it)
            if (!it->busy && (lru == cache.end() || it->last_use < lru->last_use)) lru = it;
          if (lru != cache.end()) {
            used -= lru->bytes;
            victims.push_back(*lru);
            cache.erase(lru);
            continue;
          }
          cv.wait(lock);
        }
        if (!slot) {
          cache.emplace_back();
          slot = &cache.back();
          slot->shape = sh;
          slot->R = R;
          slot->bytes = need;
          used += need;
        }
        slot->busy = true;
        ++running;
      }
      for (Cached& v : victims) release(v);
      const Clock::time_point t_admit = Clock::now();
      const int R = (int)members.size();
      const irk_request& sh = reqs[members[0]];
      std::vector<double> taus(R);
      for (int r = 0; r < R; ++r) taus[r] = reqs[members[r]].tau;
      irk_status s = IRK_OK;
      if (!reused) {
        if (cudaStreamCreateWithFlags(&slot->st, cudaStreamNonBlocking) != cudaSuccess) {
          cudaGetLastError();
          slot->st = nullptr;
          s = IRK_ECUDA;
        }
        irk_mesh mesh{sh.dim, sh.cells};
        if (s == IRK_OK)
          s = groups_ok ? irk_create_group(&mesh, sh.degree, sh.Q, R, taus.data(), &opt.solver, slot->st, &slot->h)
                        : irk_create(&mesh, sh.degree, sh.Q, taus[0], &opt.solver, slot->st, &slot->h);
      } else {
        s = irk_set_tau(slot->h, taus.data());
      }
      cudaStream_t st = slot->st;
      std::vector<double*> ys(R, nullptr);
      long long nd = 0, ni = 0;
      if (s == IRK_OK) {
        nd = irk_ndofs(slot->h);
        ni = irk_ninterior(slot->h);
        for (int r = 0; r < R && s == IRK_OK; ++r) {
          if (cudaMallocAsync((void**)&ys[r], (size_t)nd * sizeof(double), st) != cudaSuccess) {
            cudaGetLastError();
            ys[r] = nullptr;
            s = IRK_ENOMEM;
          }
          if (s == IRK_OK) s = irk_interpolate_initial(slot->h, ys[r], reqs[members[r]].t0);
        }
      }
      if (s == IRK_OK && cudaStreamSynchronize(st) != cudaSuccess) s = IRK_ECUDA;
      const Clock::time_point t_setup = Clock::now();
      std::vector<irk_status> per(R, s);
      std::vector<irk_stats> stats(R);
      if (s == IRK_OK) {
        std::vector<double> t0(R);
        for (int r = 0; r < R; ++r) t0[r] = reqs[members[r]].t0;
        if (groups_ok) {
          irk_step_group(slot->h, ys.data(), t0.data(), stats.data(), per.data());
        } else {
          per[0] = irk_step(slot->h, ys[0], t0[0], nullptr, &stats[0]);
        }
      }
      for (int r = 0; r < R; ++r) {
        const int i = members[r];
        if (per[r] == IRK_OK && out_host && out_host[i]) {
          if (cudaMemcpyAsync(out_host[i], ys[r], (size_t)nd * sizeof(double), cudaMemcpyDeviceToHost, st) !=
                  cudaSuccess ||
              cudaStreamSynchronize(st) != cudaSuccess)
            per[r] = IRK_ECUDA;
        }
      }
      const Clock::time_point t_done = Clock::now();
      for (int r = 0; r < R; ++r) {
        const int i = members[r];
        irk_result& res = results[i];
        res.queue_ms = ms_since(arrival[i], t_admit);
        res.setup_ms = ms_since(t_admit, t_setup);
        res.solve_ms = ms_since(t_setup, t_done);
        res.latency_ms = ms_since(arrival[i], t_done);
        res.iterations = stats[r].iterations;
        res.ndofs = nd;
        res.ninterior = ni;
        res.status = per[r];
        res.group_size = R;
        res.handle_reused = reused ? 1 : 0;
        if (ys[r]) cudaFreeAsync(ys[r], st);
      }
      bool drop = !reuse || s != IRK_OK;
      Cached gone;
      {
        std::lock_guard<std::mutex> lock(mu);
        --running;
        finished += R;
        slot->busy = false;
        slot->last_use = ++clock_tick;
        if (drop) {
          for (auto it = cache.begin(); it != cache.end(); ++it)
            if (&*it == slot) {
              used -= it->bytes;
              gone = *it;
              cache.erase(it);
              break;
            }
        }
      }
      if (drop) release(gone);
      cv.notify_all();
    }
  };

  std::vector<std::thread> pool;
  for (int w = 0; w < nslots; ++w) pool.emplace_back(worker);

  // arrivals: in real time one by one; otherwise all at time 0, queued together (so the groups
  // formed do not depend on thread timing)
  auto arrive = [&](int i) {
    if (est[i] > budget) {
      results[i].status = IRK_EBUSY;
      ++finished;
    } else {
      pending.push_back(i);
    }
  };
  if (opt.realtime) {
    for (int i = 0; i < count; ++i) {
      arrival[i] = start + std::chrono::duration_cast<Clock::duration>(
                               std::chrono::duration<double>(std::max(0.0, reqs[i].arrival_s)));
      std::this_thread::sleep_until(arrival[i]);
      std::lock_guard<std::mutex> lock(mu);
      arrive(i);
      cv.notify_all();
    }
  } else {
    std::lock_guard<std::mutex> lock(mu);
    for (int i = 0; i < count; ++i) {
      arrival[i] = start;
      arrive(i);
    }
    cv.notify_all();
  }
  {
    std::unique_lock<std::mutex> lock(mu);
    cv.wait(lock, [&] { return finished == count; });
    closing = true;
  }
  cv.notify_all();
  for (auto& t : pool) t.join();
  for (Cached& c : cache) release(c);
  for (int i = 0; i < count; ++i)
    if (results[i].status != IRK_OK) return results[i].status;
  return IRK_OK;
}
