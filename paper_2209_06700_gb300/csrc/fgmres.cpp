// Right-preconditioned flexible GMRES in FP64 (the outer Krylov solver of
// arXiv 2209.06700, Sec. 2 and Sec. 5: GMRES on Eq. (irk:A) with the block
// preconditioner of Eq. (irk:P)).  The flexible variant stores the
// preconditioned vectors Z because the preconditioner (one mixed-precision
// V-cycle per block) is not a fixed linear map in floating point.
// Classical Gram-Schmidt with a second pass where one pass would leave the
// basis orthogonal to worse than 2^-16 (decided on the device by the reduction
// that finishes the first pass's coefficients, from the cancellation
// |w - V h| / |w| and the loss carried over from earlier steps); the dot
// products are deterministic device reductions, finished inside each
// Gram-Schmidt kernel by its last block, and the Hessenberg/Givens update runs
// on the host with one device->host transfer per iteration.  The vectors are
// FP64 or float-float (ff), chosen by the caller.
#include <cmath>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "profiler.h"
#include "solver.h"

namespace irk {

// Small pinned host blocks (256 doubles) shared by all handles of the process.  They are never
// handed back to the driver: releasing pinned memory synchronises the device, which would stall
// the streams of other requests in flight.
namespace {
std::mutex g_pin_mu;
std::vector<double*> g_pin_free;
}  // namespace

double* pinned_block_acquire() {
  std::lock_guard<std::mutex> lock(g_pin_mu);
  if (g_pin_free.empty()) {
    double* chunk = nullptr;
    if (cudaMallocHost((void**)&chunk, 64 * 256 * sizeof(double)) != cudaSuccess) return nullptr;
    for (int i = 0; i < 64; ++i) g_pin_free.push_back(chunk + (size_t)i * 256);
  }
  double* p = g_pin_free.back();
  g_pin_free.pop_back();
  return p;
}

void pinned_block_release(double* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lock(g_pin_mu);
  g_pin_free.push_back(p);
}

Status fgmres_alloc(FGMRESWork& w, int ns, long long ld, int m, DeviceArena& arena, cudaStream_t stream) {
  if (m < 1 || m > 60) return Status::Err(IRK_EINVAL, "restart must be in 1..60");
  static_assert(sizeof(ff) == sizeof(double), "ff vectors share the FP64 layout");
  w.ns = ns;
  w.m = m;
  w.ld = ld;
  w.len = (long long)ns * ld;
  w.nb = reduction_blocks(w.len);
  IRK_TRY(arena.alloc((void**)&w.V, (size_t)(m + 1) * w.len * sizeof(double)));
  IRK_TRY(arena.alloc((void**)&w.Z, (size_t)m * w.len * sizeof(double)));
  IRK_TRY(arena.alloc((void**)&w.tmp, (size_t)w.len * sizeof(double)));
  IRK_TRY(arena.alloc((void**)&w.partial, (size_t)66 * w.nb * sizeof(double)));
  IRK_TRY(arena.alloc((void**)&w.dvals, 256 * sizeof(double)));
  IRK_TRY(arena.alloc((void**)&w.fvals, 256 * sizeof(ff)));
  IRK_TRY(arena.alloc((void**)&w.count, 64 * sizeof(unsigned)));
  IRK_CUDA(cudaMemsetAsync(w.count, 0, 64 * sizeof(unsigned), stream));
  if (!w.hvals) {
    w.hvals = pinned_block_acquire();
    if (!w.hvals) return Status::Err(IRK_ENOMEM, "pinned host allocation failed");
  }
  if (!w.hvals2) {
    w.hvals2 = pinned_block_acquire();
    if (!w.hvals2) return Status::Err(IRK_ENOMEM, "pinned host allocation failed");
  }
  for (int i = 0; i < 2; ++i)
    if (!w.ev[i]) IRK_CUDA(cudaEventCreateWithFlags(&w.ev[i], cudaEventDisableTiming));
  // the constant 1 (restart residual b - A x) in both forms
  const ff one{1.0f, 0.0f};
  w.hvals[255] = 1.0;
  std::memcpy(&w.hvals[254], &one, sizeof(ff));
  IRK_CUDA(cudaMemcpyAsync(w.dvals + 255, w.hvals + 255, sizeof(double), cudaMemcpyHostToDevice, stream));
  IRK_CUDA(cudaMemcpyAsync(w.fvals + 255, w.hvals + 254, sizeof(ff), cudaMemcpyHostToDevice, stream));
  IRK_CUDA(cudaStreamSynchronize(stream));
  return Status::Ok();
}

void fgmres_release(FGMRESWork& w) {
  pinned_block_release(w.hvals);
  pinned_block_release(w.hvals2);
  w.hvals = w.hvals2 = nullptr;
  for (int i = 0; i < 2; ++i)
    if (w.ev[i]) cudaEventDestroy(w.ev[i]);
  w.ev[0] = w.ev[1] = nullptr;
}

namespace {

// layout of dvals / fvals / hvals
constexpr int kH1 = 0, kH2 = 65, kNrm = 130, kRedo = 132, kInv = 133, kDelta = 134, kY = 160, kOne = 255;

// The second classical Gram-Schmidt pass is taken only where one pass would leave the basis
// orthogonal to worse than 2^-16 (estimated loss of orthogonality).  With the Gram matrix of the
// m + 1 basis vectors within m 2^-16 <= 1e-3 of the identity (m <= 60), its singular values lie
// within 1 +- 5e-4: the Hessenberg least-squares residual equals the true residual |b - A x| of the
// computed x, and GMRES's residuals the optimal ones over the same space, to within 0.1 %, so the
// stopping test and the iteration count are those of a fully orthogonal basis; the estimate itself
// runs about 100 times above the actual loss.  Rounding of one pass: about 100 units of roundoff of
// the vectors' arithmetic (the blocked length-n dot products; ff: 2^-48).
constexpr double kOrthTol = 1.52587890625e-5;  // 2^-16
template <typename S> constexpr double pass_rounding();
template <> constexpr double pass_rounding<double>() { return 100.0 * 1.1102230246251565e-16; }
template <> constexpr double pass_rounding<ff>() { return 100.0 * 3.552713678800501e-15; }

// The extras of the three Gram-Schmidt reductions of Arnoldi step nv - 1 on the scalars dv / fv:
// pass 1 decides the second pass (flag kRedo, loss estimate kDelta); pass 2 writes |w'| and 1/|w'|
// when no second pass follows; pass 3 writes them after the second pass.
// (always_two: the second pass at every step, classical Gram-Schmidt twice.)
template <typename S>
void gs_sinks(double* dv, ff* fv, unsigned* count, int nv, bool always_two, RowSink& r1, RowSink& r2, RowSink& r3) {
  r1.out = dv + kH1;
  r1.count = count;
  r1.X.out_ff = fv + kH1;
  r1.X.sel_flag = dv + kRedo;
  r1.X.sel_delta = dv + kDelta;
  r1.X.sel_nv = nv;
  r1.X.sel_round = pass_rounding<S>();
  r1.X.sel_tol = always_two ? -1.0 : kOrthTol;
  r2.out = dv + kH2;
  r2.count = count;
  r2.X.out_ff = fv + kH2;
  r2.X.clear_flag = dv + kRedo;
  r2.X.clear_row = nv;
  r2.X.clear_norm = dv + kNrm;
  r2.X.clear_inv = dv + kInv;
  r2.X.clear_inv_ff = fv + kInv;
  r3.out = dv + kNrm;
  r3.count = count;
  r3.take_sqrt = 1;
  r3.X.inv = dv + kInv;
  r3.X.inv_ff = fv + kInv;
}

template <typename S> typename Coef<S>::type* coefs(FGMRESWork& w);
template <> double* coefs<double>(FGMRESWork& w) { return w.dvals; }
template <> ff* coefs<ff>(FGMRESWork& w) { return w.fvals; }

// y (host, FP64) -> device coefficients of the vector type, through the pinned block
template <typename S> Status upload_y(FGMRESWork& w, const std::vector<double>& y, int kk, cudaStream_t st);
template <> Status upload_y<double>(FGMRESWork& w, const std::vector<double>& y, int kk, cudaStream_t st) {
  for (int i = 0; i < kk; ++i) w.hvals[kY + i] = y[i];
  IRK_CUDA(cudaMemcpyAsync(w.dvals + kY, w.hvals + kY, kk * sizeof(double), cudaMemcpyHostToDevice, st));
  return Status::Ok();
}
template <> Status upload_y<ff>(FGMRESWork& w, const std::vector<double>& y, int kk, cudaStream_t st) {
  for (int i = 0; i < kk; ++i) {
    ff v;
    split_double(y[i], &v.hi, &v.lo);
    std::memcpy(&w.hvals[kY + i], &v, sizeof(ff));
  }
  IRK_CUDA(cudaMemcpyAsync(w.fvals + kY, w.hvals + kY, kk * sizeof(ff), cudaMemcpyHostToDevice, st));
  return Status::Ok();
}

template <typename S>
Status norm(FGMRESWork& w, const S* v, cudaStream_t st, double& out) {
  int nb = w.nb;
  RowSink R;
  R.out = w.dvals + kNrm;
  R.count = w.count;
  R.take_sqrt = 1;
  IRK_LAUNCH(PROF_KRYLOV, launch_norm2_partial<S>(v, w.len, w.partial, nb, R, st));
  IRK_CUDA(cudaMemcpyAsync(w.hvals + kNrm, w.dvals + kNrm, sizeof(double), cudaMemcpyDeviceToHost, st));
  IRK_CUDA(cudaStreamSynchronize(st));
  out = w.hvals[kNrm];
  return Status::Ok();
}

}  // namespace

template <typename S>
Status fgmres_solve(FGMRESWork& w, const ApplyFn<S>& op, const ApplyFn<S>& prec, const S* b, S* x, double rtol,
                    int max_it, cudaStream_t st, FGMRESResult& res) {
  res = FGMRESResult();
  const long long len = w.len;
  const int m = w.m;
  S* V = reinterpret_cast<S*>(w.V);
  S* Z = reinterpret_cast<S*>(w.Z);
  S* tmp = reinterpret_cast<S*>(w.tmp);
  typename Coef<S>::type* cf = coefs<S>(w);
  IRK_CUDA(cudaMemsetAsync(x, 0, (size_t)len * sizeof(S), st));
  IRK_CUDA(cudaMemsetAsync(w.count, 0, sizeof(unsigned), st));  // in case a failed launch left it
  double bnorm;
  IRK_TRY(norm<S>(w, b, st, bnorm));
  if (!std::isfinite(bnorm)) return Status::Err(IRK_ENUMERIC, "non-finite right-hand side");
  if (bnorm == 0.0) { res.converged = true; return Status::Ok(); }
  const double target = rtol * bnorm;
  // first cycle: r = b (x0 = 0)
  double beta = bnorm;
  IRK_LAUNCH(PROF_KRYLOV, launch_scale<S>(b, 1.0 / beta, V, len, st));
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  int total = 0;
  // One Arnoldi step j: preconditioner, operator, the Gram-Schmidt passes, the read-back of their
  // scalars into pinned block j % 2 (event ev[j % 2]) and the normalisation by the device-computed
  // 1/|w''| (0 when |w''| = 0).  Nothing in step j + 1 needs the host's Givens update of step j,
  // so step j + 1 is enqueued before the host waits for step j: the GPU does not idle while the
  // host reads the scalars, updates the Hessenberg matrix and tests convergence.  Near the
  // expected convergence the host waits first, so that no step is computed in vain.
  auto launch_step = [&](int j) -> Status {
    S* Vj = V + (size_t)j * len;
    S* Zj = Z + (size_t)j * len;
    S* wv = V + (size_t)(j + 1) * len;
    IRK_TRY(prec(Vj, Zj));
    IRK_TRY(op(Zj, wv));
    // classical Gram-Schmidt; the second pass only where one pass would lose orthogonality
    const int nv = j + 1;
    RowSink r1, r2, r3;
    gs_sinks<S>(w.dvals, w.fvals, w.count, nv, w.always_two_passes != 0, r1, r2, r3);
    // pass 1: h1 = V^T w and |w|^2; its last block decides on the second pass
    int nb = w.nb;  // row capacity of w.partial in, blocks used out
    IRK_LAUNCH(PROF_KRYLOV, launch_gs_dot<S>(V, len, nv, wv, len, w.partial, nb, r1, st));
    // w' = w - V h1 and |w'|^2 (in place up to 16 basis vectors), h2 = V^T w' for the second pass
    S* w2 = (nv <= 16) ? wv : tmp;
    nb = w.nb;
    IRK_LAUNCH(PROF_KRYLOV, launch_gs_axpy_dot<S>(V, len, nv, cf + kH1, wv, w2, len, w.partial, nb, r2,
                                                  w.dvals + kRedo, st));
    // second pass w'' = w' - V h2, |w''| and 1 / |w''| (nothing to do in place without it)
    nb = w.nb;
    IRK_LAUNCH(PROF_KRYLOV, launch_gs_reorth<S>(V, len, nv, cf + kH2, w.dvals + kRedo, w2, wv, len, w.partial,
                                                nb, r3, st));
    double* hb = (j % 2 == 0) ? w.hvals : w.hvals2;
    IRK_CUDA(cudaMemcpyAsync(hb, w.dvals, (kRedo + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
    IRK_CUDA(cudaEventRecord(w.ev[j % 2], st));
    IRK_LAUNCH(PROF_KRYLOV, launch_scale_dev<S>(wv, cf + kInv, wv, len, st));
    return Status::Ok();
  };
  while (true) {
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jlast = -1;
    bool stop = false;
    double prev_resid = -1.0, prev2_resid = -1.0;
    IRK_TRY(launch_step(0));
    for (int j = 0; j < m; ++j) {
      // enqueue step j + 1 ahead unless step j is expected to be the last one
      bool ahead = false;
      if (j + 1 < m && total + 1 < max_it) {
        const bool expect_last = prev_resid > 0.0 && prev2_resid > 0.0 &&
                                 prev_resid * (prev_resid / prev2_resid) <= 2.0 * target;
        if (!expect_last) {
          IRK_TRY(launch_step(j + 1));
          ahead = true;
        }
      }
      IRK_CUDA(cudaEventSynchronize(w.ev[j % 2]));
      const double* hv = (j % 2 == 0) ? w.hvals : w.hvals2;
      const double hn = hv[kNrm];
      if (!std::isfinite(hn)) {
        IRK_CUDA(cudaStreamSynchronize(st));
        return Status::Err(IRK_ENUMERIC, "non-finite value in the Arnoldi process");
      }
      const bool redo = hv[kRedo] != 0.0;
      res.reorth += redo ? 1 : 0;
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hv[kH1 + i] + (redo ? hv[kH2 + i] : 0.0);
      H[(size_t)(j + 1) * m + j] = hn;
      // Givens rotations
      for (int i = 0; i < j; ++i) {
        const double a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * bb;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      const double a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
      const double r = std::hypot(a, bb);
      cs[j] = (r == 0.0) ? 1.0 : a / r;
      sn[j] = (r == 0.0) ? 0.0 : bb / r;
      H[(size_t)j * m + j] = r;
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++total;
      jlast = j;
      const double resid = std::fabs(g[j + 1]);
      res.rel_residual = resid / bnorm;
      prev2_resid = prev_resid;
      prev_resid = resid;
      if (resid <= target) { res.converged = true; stop = true; break; }
      if (total >= max_it || hn == 0.0) { stop = true; break; }
      if (!ahead && j + 1 < m) IRK_TRY(launch_step(j + 1));
    }
    // y = H^{-1} g, x += Z y
    const int kk = jlast + 1;
    for (int i = kk - 1; i >= 0; --i) {
      double s = g[i];
      for (int c = i + 1; c < kk; ++c) s -= H[(size_t)i * m + c] * y[c];
      y[i] = s / H[(size_t)i * m + i];
    }
    IRK_TRY(upload_y<S>(w, y, kk, st));
    IRK_LAUNCH(PROF_KRYLOV, launch_multi_axpy<S>(Z, len, kk, cf + kY, 1.0, x, len, st));
    if (stop) break;
    // restart with the explicit residual
    IRK_TRY(op(x, tmp));
    IRK_LAUNCH(PROF_KRYLOV, launch_scale<S>(tmp, -1.0, tmp, len, st));
    // tmp = b - A x  (coefficient slot kOne holds the constant 1)
    IRK_LAUNCH(PROF_KRYLOV, launch_multi_axpy<S>(b, 0, 1, cf + kOne, 1.0, tmp, len, st));
    IRK_TRY(norm<S>(w, tmp, st, beta));
    if (!std::isfinite(beta)) return Status::Err(IRK_ENUMERIC, "non-finite restart residual");
    if (beta <= target) { res.converged = true; res.rel_residual = beta / bnorm; break; }
    IRK_LAUNCH(PROF_KRYLOV, launch_scale<S>(tmp, 1.0 / beta, V, len, st));
  }
  IRK_CUDA(cudaStreamSynchronize(st));
  res.iterations = total;
  return Status::Ok();
}

Status group_scalars_alloc(GroupScalars& g, int R, DeviceArena& arena, cudaStream_t st) {
  IRK_TRY(arena.alloc((void**)&g.dvals, (size_t)R * 256 * sizeof(double)));
  IRK_TRY(arena.alloc((void**)&g.fvals, (size_t)R * 256 * sizeof(ff)));
  IRK_TRY(arena.alloc((void**)&g.count, (size_t)R * 64 * sizeof(unsigned)));
  IRK_CUDA(cudaMemsetAsync(g.count, 0, (size_t)R * 64 * sizeof(unsigned), st));
  const ff one{1.0f, 0.0f};
  for (int r = 0; r < R; ++r) {
    double* hv = pinned_block_acquire();
    if (!hv) return Status::Err(IRK_ENOMEM, "pinned host allocation failed");
    g.hvals.push_back(hv);
    hv[kOne] = 1.0;
    std::memcpy(&hv[kOne - 1], &one, sizeof(ff));
    IRK_CUDA(cudaMemcpyAsync(g.dvals + (size_t)r * 256 + kOne, hv + kOne, sizeof(double), cudaMemcpyHostToDevice, st));
    IRK_CUDA(cudaMemcpyAsync(g.fvals + (size_t)r * 256 + kOne, hv + kOne - 1, sizeof(ff), cudaMemcpyHostToDevice, st));
  }
  IRK_CUDA(cudaStreamSynchronize(st));
  return Status::Ok();
}

void group_scalars_release(GroupScalars& g) {
  for (double* p : g.hvals) pinned_block_release(p);
  g.hvals.clear();
}

namespace {

// One request's view of the group scalars in the layout of FGMRESWork (coefficients, norms, counter).
FGMRESWork request_view(const FGMRESWork& w, const GroupScalars& gs, int r, int R) {
  FGMRESWork v = w;
  v.len = w.len / R;
  v.nb = reduction_blocks(v.len);
  v.dvals = gs.dvals + (size_t)r * 256;
  v.fvals = gs.fvals + (size_t)r * 256;
  v.hvals = gs.hvals[r];
  v.count = gs.count + (size_t)r * 64;
  return v;
}

}  // namespace

template <typename S>
Status fgmres_solve_group(FGMRESWork& w, int R, GroupScalars& gs, const ApplyFn<S>& op, const ApplyFn<S>& prec,
                          const S* b, S* x, double rtol, int max_it, cudaStream_t st,
                          std::vector<FGMRESResult>& res, std::vector<Status>& st_out) {
  const long long all = w.len, len = w.len / R;
  const int m = w.m;
  S* V = reinterpret_cast<S*>(w.V);
  S* Z = reinterpret_cast<S*>(w.Z);
  S* tmp = reinterpret_cast<S*>(w.tmp);
  res.assign(R, FGMRESResult());
  st_out.assign(R, Status::Ok());
  std::vector<FGMRESWork> wv(R);
  for (int r = 0; r < R; ++r) wv[r] = request_view(w, gs, r, R);
  auto cf = [&](int r) { return coefs<S>(wv[r]); };
  IRK_CUDA(cudaMemsetAsync(x, 0, (size_t)all * sizeof(S), st));
  IRK_CUDA(cudaMemsetAsync(gs.count, 0, (size_t)R * 64 * sizeof(unsigned), st));
  // norms of every request's vector at once (one read-back): out[r] = |v_r|
  auto norms = [&](const S* v, const std::vector<bool>& which, std::vector<double>& out) -> Status {
    for (int r = 0; r < R; ++r) {
      if (!which[r]) continue;
      int nb = wv[r].nb;
      RowSink Rk;
      Rk.out = wv[r].dvals + kNrm;
      Rk.count = wv[r].count;
      Rk.take_sqrt = 1;
      IRK_LAUNCH(PROF_KRYLOV, launch_norm2_partial<S>(v + (size_t)r * len, len, w.partial, nb, Rk, st));
      IRK_CUDA(cudaMemcpyAsync(wv[r].hvals + kNrm, wv[r].dvals + kNrm, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    IRK_CUDA(cudaStreamSynchronize(st));
    for (int r = 0; r < R; ++r)
      if (which[r]) out[r] = wv[r].hvals[kNrm];
    return Status::Ok();
  };
  std::vector<bool> live(R, true);     // still iterating
  std::vector<double> bnorm(R, 0.0), beta(R, 0.0), target(R, 0.0);
  IRK_TRY(norms(b, live, bnorm));
  for (int r = 0; r < R; ++r) {
    if (!std::isfinite(bnorm[r])) {
      st_out[r] = Status::Err(IRK_ENUMERIC, "non-finite right-hand side");
      live[r] = false;
    } else if (bnorm[r] == 0.0) {
      res[r].converged = true;
      live[r] = false;
    }
    target[r] = rtol * bnorm[r];
    beta[r] = bnorm[r];
  }
  // first cycle: r = b (x0 = 0); stopped requests get zero slices
  for (int r = 0; r < R; ++r) {
    if (live[r]) IRK_LAUNCH(PROF_KRYLOV, launch_scale<S>(b + (size_t)r * len, 1.0 / beta[r], V + (size_t)r * len, len, st));
    else IRK_CUDA(cudaMemsetAsync(V + (size_t)r * len, 0, (size_t)len * sizeof(S), st));
  }
  std::vector<std::vector<double>> H(R, std::vector<double>((size_t)(m + 1) * m)), cs(R, std::vector<double>(m)),
      sn(R, std::vector<double>(m)), g(R, std::vector<double>(m + 1)), y(R, std::vector<double>(m));
  std::vector<int> total(R, 0), jlast(R, -1);
  while (true) {
    std::vector<bool> cyc = live;  // requests iterating in this cycle
    for (int r = 0; r < R; ++r) {
      std::fill(g[r].begin(), g[r].end(), 0.0);
      g[r][0] = beta[r];
      jlast[r] = -1;
    }
    for (int j = 0; j < m; ++j) {
      if (std::none_of(cyc.begin(), cyc.end(), [](bool v) { return v; })) break;
      S* Vj = V + (size_t)j * all;
      S* Zj = Z + (size_t)j * all;
      S* W = V + (size_t)(j + 1) * all;
      IRK_TRY(prec(Vj, Zj));
      IRK_TRY(op(Zj, W));
      const int nv = j + 1;
      for (int r = 0; r < R; ++r) {
        if (!cyc[r]) continue;
        FGMRESWork& q = wv[r];
        const S* Vr = V + (size_t)r * len;
        S* wr = W + (size_t)r * len;
        S* tr = tmp + (size_t)r * len;
        RowSink r1, r2, r3;
        gs_sinks<S>(q.dvals, q.fvals, q.count, nv, w.always_two_passes != 0, r1, r2, r3);
        int nb = q.nb;
        IRK_LAUNCH(PROF_KRYLOV, launch_gs_dot<S>(Vr, all, nv, wr, len, w.partial, nb, r1, st));
        S* w2 = (nv <= 16) ? wr : tr;
        nb = q.nb;
        IRK_LAUNCH(PROF_KRYLOV, launch_gs_axpy_dot<S>(Vr, all, nv, cf(r) + kH1, wr, w2, len, w.partial, nb, r2,
                                                      q.dvals + kRedo, st));
        nb = q.nb;
        IRK_LAUNCH(PROF_KRYLOV, launch_gs_reorth<S>(Vr, all, nv, cf(r) + kH2, q.dvals + kRedo, w2, wr, len, w.partial,
                                                    nb, r3, st));
        IRK_CUDA(cudaMemcpyAsync(q.hvals, q.dvals, (kRedo + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
      }
      IRK_CUDA(cudaStreamSynchronize(st));
      for (int r = 0; r < R; ++r) {
        if (!cyc[r]) continue;
        FGMRESWork& q = wv[r];
        const double hn = q.hvals[kNrm];
        S* wr = W + (size_t)r * len;
        if (!std::isfinite(hn)) {
          st_out[r] = Status::Err(IRK_ENUMERIC, "non-finite value in the Arnoldi process");
          cyc[r] = live[r] = false;
          jlast[r] = -1;  // no update of x
          IRK_CUDA(cudaMemsetAsync(wr, 0, (size_t)len * sizeof(S), st));
          continue;
        }
        const bool redo = q.hvals[kRedo] != 0.0;
        res[r].reorth += redo ? 1 : 0;
        std::vector<double>& Hr = H[r];
        for (int i = 0; i <= j; ++i) Hr[(size_t)i * m + j] = q.hvals[kH1 + i] + (redo ? q.hvals[kH2 + i] : 0.0);
        Hr[(size_t)(j + 1) * m + j] = hn;
        for (int i = 0; i < j; ++i) {
          const double a = Hr[(size_t)i * m + j], bb = Hr[(size_t)(i + 1) * m + j];
          Hr[(size_t)i * m + j] = cs[r][i] * a + sn[r][i] * bb;
          Hr[(size_t)(i + 1) * m + j] = -sn[r][i] * a + cs[r][i] * bb;
        }
        const double a = Hr[(size_t)j * m + j], bb = Hr[(size_t)(j + 1) * m + j];
        const double rr = std::hypot(a, bb);
        cs[r][j] = (rr == 0.0) ? 1.0 : a / rr;
        sn[r][j] = (rr == 0.0) ? 0.0 : bb / rr;
        Hr[(size_t)j * m + j] = rr;
        Hr[(size_t)(j + 1) * m + j] = 0.0;
        g[r][j + 1] = -sn[r][j] * g[r][j];
        g[r][j] = cs[r][j] * g[r][j];
        ++total[r];
        jlast[r] = j;
        const double resid = std::fabs(g[r][j + 1]);
        res[r].rel_residual = resid / bnorm[r];
        bool stop = false;
        if (resid <= target[r]) { res[r].converged = true; stop = true; }
        if (total[r] >= max_it || hn == 0.0) stop = true;
        if (stop) {
          cyc[r] = live[r] = false;
          IRK_CUDA(cudaMemsetAsync(wr, 0, (size_t)len * sizeof(S), st));  // later shared launches see zeros
        } else if (hn > 0.0) {
          IRK_LAUNCH(PROF_KRYLOV, launch_scale_dev<S>(wr, cf(r) + kInv, wr, len, st));
        }
      }
    }
    // y = H^{-1} g, x += Z y for every request that iterated in this cycle
    for (int r = 0; r < R; ++r) {
      const int kk = jlast[r] + 1;
      if (kk <= 0) continue;
      for (int i = kk - 1; i >= 0; --i) {
        double t = g[r][i];
        for (int c = i + 1; c < kk; ++c) t -= H[r][(size_t)i * m + c] * y[r][c];
        y[r][i] = t / H[r][(size_t)i * m + i];
      }
      IRK_TRY(upload_y<S>(wv[r], y[r], kk, st));
      IRK_LAUNCH(PROF_KRYLOV, launch_multi_axpy<S>(Z + (size_t)r * len, all, kk, cf(r) + kY, 1.0, x + (size_t)r * len, len, st));
    }
    if (std::none_of(live.begin(), live.end(), [](bool v) { return v; })) break;
    // restart the live requests with their explicit residuals (one shared operator launch)
    IRK_TRY(op(x, tmp));
    for (int r = 0; r < R; ++r) {
      if (!live[r]) continue;
      S* tr = tmp + (size_t)r * len;
      IRK_LAUNCH(PROF_KRYLOV, launch_scale<S>(tr, -1.0, tr, len, st));
      IRK_LAUNCH(PROF_KRYLOV, launch_multi_axpy<S>(b + (size_t)r * len, 0, 1, cf(r) + kOne, 1.0, tr, len, st));
    }
    std::vector<double> nb(R, 0.0);
    IRK_TRY(norms(tmp, live, nb));
    for (int r = 0; r < R; ++r) {
      if (!live[r]) {
        IRK_CUDA(cudaMemsetAsync(V + (size_t)r * len, 0, (size_t)len * sizeof(S), st));
        continue;
      }
      beta[r] = nb[r];
      if (!std::isfinite(beta[r])) {
        st_out[r] = Status::Err(IRK_ENUMERIC, "non-finite restart residual");
        live[r] = false;
      } else if (beta[r] <= target[r]) {
        res[r].converged = true;
        res[r].rel_residual = beta[r] / bnorm[r];
        live[r] = false;
      }
      if (live[r]) IRK_LAUNCH(PROF_KRYLOV, launch_scale<S>(tmp + (size_t)r * len, 1.0 / beta[r], V + (size_t)r * len, len, st));
      else IRK_CUDA(cudaMemsetAsync(V + (size_t)r * len, 0, (size_t)len * sizeof(S), st));
    }
    if (std::none_of(live.begin(), live.end(), [](bool v) { return v; })) break;
  }
  IRK_CUDA(cudaStreamSynchronize(st));
  for (int r = 0; r < R; ++r) res[r].iterations = total[r];
  return Status::Ok();
}

template Status fgmres_solve_group<double>(FGMRESWork&, int, GroupScalars&, const ApplyFn<double>&,
                                           const ApplyFn<double>&, const double*, double*, double, int, cudaStream_t,
                                           std::vector<FGMRESResult>&, std::vector<Status>&);
template Status fgmres_solve_group<ff>(FGMRESWork&, int, GroupScalars&, const ApplyFn<ff>&, const ApplyFn<ff>&,
                                       const ff*, ff*, double, int, cudaStream_t, std::vector<FGMRESResult>&,
                                       std::vector<Status>&);

template Status fgmres_solve<double>(FGMRESWork&, const ApplyFn<double>&, const ApplyFn<double>&, const double*,
                                     double*, double, int, cudaStream_t, FGMRESResult&);
template Status fgmres_solve<ff>(FGMRESWork&, const ApplyFn<ff>&, const ApplyFn<ff>&, const ff*, ff*, double, int,
                                 cudaStream_t, FGMRESResult&);

}  // namespace irk
