// Continuous-batching request loop of libirk (irk_serve, declared in include/irk.h).
//
// A dispatcher admits requests in arrival order as soon as a slot and enough
// of the device-memory budget are free.  Each slot is a host worker thread with
// its own CUDA stream: it builds the request's handle (multigrid hierarchy,
// Chebyshev intervals, Krylov space) with stream-ordered allocations, takes one
// Radau IIA step from the interpolant, copies the result out and releases the
// memory without synchronising the device, so requests that arrive while others
// are running start at once and their kernels overlap on the GPU.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
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

  std::vector<double> est(count);
  for (int i = 0; i < count; ++i) {
    results[i] = irk_result();
    results[i].status = IRK_OK;
    est[i] = estimate_bytes(reqs[i], opt.solver);
    results[i].mem_bytes = est[i];
  }

  std::mutex mu;
  std::condition_variable cv;
  std::deque<int> ready;
  int active = 0, finished = 0;
  double used = 0.0;
  bool closing = false;
  std::vector<Clock::time_point> arrival(count);
  const Clock::time_point start = Clock::now();

  auto worker = [&](int slot) {
    cudaSetDevice(device);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
    (void)slot;
    for (;;) {
      int i;
      {
        std::unique_lock<std::mutex> lock(mu);
        cv.wait(lock, [&] { return closing || !ready.empty(); });
        if (ready.empty()) break;
        i = ready.front();
        ready.pop_front();
      }
      const irk_request& r = reqs[i];
      irk_result& res = results[i];
      const Clock::time_point t_admit = Clock::now();
      res.queue_ms = ms_since(arrival[i], t_admit);
      irk_mesh mesh{r.dim, r.cells};
      irk_handle h = nullptr;
      double* y = nullptr;
      irk_status s = irk_create(&mesh, r.degree, r.Q, r.tau, &opt.solver, st, &h);
      if (s == IRK_OK) {
        res.ndofs = irk_ndofs(h);
        res.ninterior = irk_ninterior(h);
        if (cudaMallocAsync((void**)&y, (size_t)res.ndofs * sizeof(double), st) != cudaSuccess) {
          cudaGetLastError();
          s = IRK_ENOMEM;
        }
      }
      if (s == IRK_OK) s = irk_interpolate_initial(h, y, r.t0);
      if (s == IRK_OK && cudaStreamSynchronize(st) != cudaSuccess) s = IRK_ECUDA;
      const Clock::time_point t_setup = Clock::now();
      res.setup_ms = ms_since(t_admit, t_setup);
      if (s == IRK_OK) {
        irk_stats stats{};
        s = irk_step(h, y, r.t0, nullptr, &stats);
        res.iterations = stats.iterations;
      }
      if (s == IRK_OK && out_host && out_host[i]) {
        if (cudaMemcpyAsync(out_host[i], y, (size_t)res.ndofs * sizeof(double), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
          s = IRK_ECUDA;
      }
      const Clock::time_point t_done = Clock::now();
      res.solve_ms = ms_since(t_setup, t_done);
      res.latency_ms = ms_since(arrival[i], t_done);
      res.status = s;
      if (y) cudaFreeAsync(y, st);
      irk_destroy(h);
      {
        std::lock_guard<std::mutex> lock(mu);
        --active;
        used -= est[i];
        ++finished;
      }
      cv.notify_all();
    }
    if (st) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
  };

  std::vector<std::thread> pool;
  for (int w = 0; w < nslots; ++w) pool.emplace_back(worker, w);

  for (int i = 0; i < count; ++i) {
    const double at = opt.realtime ? std::max(0.0, reqs[i].arrival_s) : 0.0;
    arrival[i] = start + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(at));
    if (opt.realtime) std::this_thread::sleep_until(arrival[i]);
    std::unique_lock<std::mutex> lock(mu);
    if (est[i] > budget) {
      results[i].status = IRK_EBUSY;
      ++finished;
      continue;
    }
    cv.wait(lock, [&] { return active < nslots && used + est[i] <= budget; });
    ++active;
    used += est[i];
    ready.push_back(i);
    cv.notify_all();
  }
  {
    std::unique_lock<std::mutex> lock(mu);
    cv.wait(lock, [&] { return finished == count; });
    closing = true;
  }
  cv.notify_all();
  for (auto& t : pool) t.join();
  for (int i = 0; i < count; ++i)
    if (results[i].status != IRK_OK) return results[i].status;
  return IRK_OK;
}
