// Right-preconditioned flexible GMRES in FP64 (the outer Krylov solver of
// arXiv 2209.06700, Sec. 2 and Sec. 5: GMRES on Eq. (irk:A) with the block
// preconditioner of Eq. (irk:P)).  The flexible variant stores the
// preconditioned vectors Z because the preconditioner (one mixed-precision
// V-cycle per block) is not a fixed linear map in floating point.
// Classical Gram-Schmidt with a conditional second pass (Kahan-Parlett "twice
// is enough", decided on the device by the reduction that finishes |w'|^2);
// the dot products are deterministic device reductions, finished inside each
// Gram-Schmidt kernel by its last block, and the Hessenberg/Givens update runs
// on the host with one device->host transfer per iteration.  The vectors are FP64 or float-float (ff), chosen by the caller.
#include <cmath>
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
  // the constant 1 (restart residual b - A x) in both forms
  const ff one{1.0f, 0.0f};
  w.hvals[255] = 1.0;
  std::memcpy(&w.hvals[254], &one, sizeof(ff));
  IRK_CUDA(cudaMemcpyAsync(w.dvals + 255, w.hvals + 255, sizeof(double), cudaMemcpyHostToDevice, stream));
  IRK_CUDA(cudaMemcpyAsync(w.fvals + 255, w.hvals + 254, sizeof(ff), cudaMemcpyHostToDevice, stream));
  IRK_CUDA(cudaStreamSynchronize(stream));
  return Status::Ok();
}

namespace {

// layout of dvals / fvals / hvals
constexpr int kH1 = 0, kH2 = 65, kNrm = 130, kN0 = 131, kRedo = 132, kInv = 133, kY = 160, kOne = 255;
constexpr double kEta = 0.7;  // Kahan-Parlett threshold of the conditional second pass

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
  while (true) {
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jlast = -1;
    bool stop = false;
    for (int j = 0; j < m; ++j) {
      S* Vj = V + (size_t)j * len;
      S* Zj = Z + (size_t)j * len;
      S* wv = V + (size_t)(j + 1) * len;
      IRK_TRY(prec(Vj, Zj));
      IRK_TRY(op(Zj, wv));
      // classical Gram-Schmidt, second pass only when the first one cancelled ("twice is enough")
      const int nv = j + 1;
      // pass 1: h1 = V^T w and |w|^2 (row nv, kept aside in kN0 before pass 2 overwrites row nv)
      RowSink r1;
      r1.out = w.dvals + kH1;
      r1.count = w.count;
      r1.X.out_ff = w.fvals + kH1;
      r1.X.copy_out = w.dvals + kN0;
      r1.X.copy_row = nv;
      int nb = w.nb;  // row capacity of w.partial in, blocks used out
      IRK_LAUNCH(PROF_KRYLOV, launch_gs_dot<S>(V, len, nv, wv, len, w.partial, nb, r1, st));
      // w' = w - V h1, h2 = V^T w', |w'|^2; second pass when |w'|^2 < eta^2 |w|^2
      RowSink r2;
      r2.out = w.dvals + kH2;
      r2.count = w.count;
      r2.X.out_ff = w.fvals + kH2;
      r2.X.decide_flag = w.dvals + kRedo;
      r2.X.decide_ref = w.dvals + kN0;
      r2.X.decide_row = nv;
      r2.X.eta2 = kEta * kEta;
      nb = w.nb;
      IRK_LAUNCH(PROF_KRYLOV, launch_gs_axpy_dot<S>(V, len, nv, cf + kH1, wv, tmp, len, w.partial, nb, r2, st));
      // w'' = w' - V h2 (if decided), |w''| and 1 / |w''|
      RowSink r3;
      r3.out = w.dvals + kNrm;
      r3.count = w.count;
      r3.take_sqrt = 1;
      r3.X.inv = w.dvals + kInv;
      r3.X.inv_ff = w.fvals + kInv;
      nb = w.nb;
      IRK_LAUNCH(PROF_KRYLOV, launch_gs_reorth<S>(V, len, nv, cf + kH2, w.dvals + kRedo, tmp, wv, len, w.partial,
                                                  nb, r3, st));
      IRK_CUDA(cudaMemcpyAsync(w.hvals, w.dvals, (kRedo + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
      IRK_CUDA(cudaStreamSynchronize(st));
      const double hn = w.hvals[kNrm];
      if (!std::isfinite(hn)) return Status::Err(IRK_ENUMERIC, "non-finite value in the Arnoldi process");
      const bool redo = w.hvals[kRedo] != 0.0;
      res.reorth += redo ? 1 : 0;
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = w.hvals[kH1 + i] + (redo ? w.hvals[kH2 + i] : 0.0);
      H[(size_t)(j + 1) * m + j] = hn;
      if (hn > 0.0) IRK_LAUNCH(PROF_KRYLOV, launch_scale_dev<S>(wv, cf + kInv, wv, len, st));
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
      if (resid <= target) { res.converged = true; stop = true; break; }
      if (total >= max_it || hn == 0.0) { stop = true; break; }
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

template Status fgmres_solve<double>(FGMRESWork&, const ApplyFn<double>&, const ApplyFn<double>&, const double*,
                                     double*, double, int, cudaStream_t, FGMRESResult&);
template Status fgmres_solve<ff>(FGMRESWork&, const ApplyFn<ff>&, const ApplyFn<ff>&, const ff*, ff*, double, int,
                                 cudaStream_t, FGMRESResult&);

}  // namespace irk
