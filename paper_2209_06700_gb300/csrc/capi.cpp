// C ABI of libirk (declared in include/irk.h).
//
// One Radau IIA step of M u' + K u = g (arXiv 2209.06700, Sec. 2):
//   LU variant  : FGMRES on Eq. (irk:A) preconditioned by Eq. (irk:P), the Q
//                 blocks (lambda~_i M + tau K) approximated by one V-cycle each,
//                 all blocks batched into the same launches;
//   DIAG variant: Eq. (irk:Ainv) in the real 2x2-block form of Sec. 6,
//                 one FGMRES per block: the real block (gamma M + tau K) with a
//                 V-cycle, each pair [[alpha M + tau K, -beta M], [beta M,
//                 alpha M + tau K]] with PRESB (Eq. presb:p: two sequential
//                 V-cycles on (alpha + beta) M + tau K).
// Then y_{n+1} = y_n + tau sum_i b_i k_i (Sec. 1).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "deform.h"
#include "deform_kernels.h"
#include "profiler.h"
#include "solver.h"

using namespace irk;

struct irk_problem {
  int dim = 0, k = 0, N = 0, Q = 0;
  double tau = 0;
  irk_options opt{};
  cudaStream_t st = nullptr;
  int device = 0;
  Tableau tab;
  Element1D el;
  LevelGeom fine{};
  DeviceArena arena;
  std::unique_ptr<MGBase> mg;                       // LU blocks
  std::vector<std::unique_ptr<MGBase>> mg_diag;     // DIAG blocks (one per real/pair block)
  FGMRESWork fw;                                    // LU: ns = Q
  FGMRESWork fwd;                                   // DIAG: ns = 2
  double *Ky = nullptr, *rhs = nullptr, *kst = nullptr, *Mu = nullptr, *Ku = nullptr, *G1 = nullptr,
         *x1d = nullptr, *tq = nullptr;
  int nslots = 0;                                   // stage slots of Mu/Ku
  // requests batched in this handle (irk_create_group): R problems of the same shape, each with its
  // own tau; stage vectors [R][Q][stride], hierarchy blocks [R][Q], Krylov vectors interleaved
  int R = 1;
  std::vector<double> taus;                         // tau of each request
  double* Yg = nullptr;                             // y_n of the requests side by side [R][stride]
  GroupScalars gsc;                                 // per-request Krylov scalars of group steps
  int mg_sel = 0;                                   // hierarchy of the irk_mg_* entry points (irk_mg_select)
  // curved mesh (opt.deform > 0): mapping data, cell-wise buffers, full load vector
  bool deformed = false;
  DeformGeom dgeom;
  DeformDevice<double> dd;
  double* Gv = nullptr;
  Profiler prof;
  std::string last_err;
  ~irk_problem() {
    group_scalars_release(gsc);
    fgmres_release(fw);
    fgmres_release(fwd);
  }
};

namespace {

irk_status fail(irk_problem* h, const Status& s) {
  if (h) h->last_err = s.msg;
  return s.code;
}

CombineParams combine_params(int nout, int nin, const double* Da, const double* Db = nullptr, int ninb = 0) {
  CombineParams C;
  std::memset(&C, 0, sizeof(C));
  C.nout = nout;
  C.nina = nin;
  C.ninb = ninb;
  for (int i = 0; i < nout; ++i)
    for (int j = 0; j < nin; ++j) C.Da[i * kMaxQ + j] = Da[i * nin + j];
  if (Db)
    for (int i = 0; i < nout; ++i)
      for (int j = 0; j < ninb; ++j) C.Db[i * kMaxQ + j] = Db[i * ninb + j];
  return C;
}

// The outer solver's stage vectors are ff (float-float pairs, default: every FP64-accurate
// operation on the FP32 pipe) or FP64 (op_ff = 0, the plain FP64 path).  Buffers are allocated
// as 8-byte elements and viewed with the handle's storage type.
template <typename S> S* as(double* p) { return reinterpret_cast<S*>(p); }

// FP64-accurate operator launch on the fine mesh.  cat: PROF_APPLY64 for the stage operator,
// PROF_RHS for K y_n.
template <typename S>
Status launch_apply64(irk_problem* h, const S* u, int ns, const double* cm, const double* ck, int epi, S* out,
                      S* out2, int cat = PROF_APPLY64) {
  if constexpr (std::is_same<S, double>::value) {
    if (h->deformed) {  // curved mesh: mapping data per Gauss point, all ns stages in one cell loop
      // K y_n of the stage right-hand side always in native FP64: on a smooth y_n the stiffness
      // terms cancel strongly, and float-float's 48 bits would miss the 1e-12 operator bar there
      DeformDevice<double> dd = h->dd;
      if (cat == PROF_RHS) dd.ff = false;
      IRK_LAUNCH(cat, launch_deformed<double>(dd, ns, u, h->fine.ld, epi, cm, ck, out, out2, h->st));
      return Status::Ok();
    }
  } else {
    if (h->deformed) return Status::Err(IRK_EINVAL, "curved meshes use FP64 stage vectors");
  }
  using T = typename std::conditional<std::is_same<S, ff>::value, ff, double>::type;
  OpParams<T> P = make_op_params<T>(h->fine, ns, cm, ck);
  // a launch over the stage vectors of several requests takes the launch shape of one request's
  P.shape_ns = (h->R > 1 && ns % h->R == 0) ? ns / h->R : 0;
  EpiParams<S> E;
  std::memset(&E, 0, sizeof(E));
  E.out = out;
  E.out2 = out2;
  IRK_LAUNCH(cat, launch_op<T>(h->dim, h->k, ns, u, P, epi, E, h->st));
  return Status::Ok();
}

// v = (Cm (x) M + Ck (x) K) u on the fine mesh, FP64-accurate, ns stage vectors
template <typename S>
Status apply_general(irk_problem* h, const S* u, S* v, int ns, const double* Cm, const double* Ck) {
  if (ns > h->nslots) return Status::Err(IRK_EINVAL, "too many stage vectors for this handle");
  S* Mu = as<S>(h->Mu);
  S* Ku = as<S>(h->Ku);
  IRK_TRY(launch_apply64<S>(h, u, ns, nullptr, nullptr, EPI_DUAL, Mu, Ku));
  CombineParams C = combine_params(ns, ns, Cm, Ck, ns);
  IRK_LAUNCH(PROF_COMBINE, launch_combine<S, S, S>(Mu, Ku, v, h->fine.n, h->fine.ld, C, h->st));
  return Status::Ok();
}

template <typename S>
Status apply_calA(irk_problem* h, const S* u, S* v) {
  const int Q = h->Q;
  std::vector<double> Ck((size_t)Q * Q, 0.0);
  for (int i = 0; i < Q; ++i) Ck[(size_t)i * Q + i] = h->tau;
  return apply_general<S>(h, u, v, Q, h->tab.Ainv.data(), Ck.data());
}

// copy-with-combination between the solver's stage vectors and an MG's fine buffers:
// mg_b = (D (x) I) in (+ Db in2), out = (D (x) I) mg_x (+ Db add), cast to the MG precision
template <typename S>
Status to_mg_combine(irk_problem* h, MGBase* mg, const S* in, const S* in2, const CombineParams& C) {
  const LevelGeom& g = h->fine;
  if (mg->elem_size() == 4)
    IRK_LAUNCH(PROF_COMBINE, launch_combine<S, S, float>(in, in2, (float*)mg->fine_b(), g.n, g.ld, C, h->st));
  else
    IRK_LAUNCH(PROF_COMBINE, launch_combine<S, S, double>(in, in2, (double*)mg->fine_b(), g.n, g.ld, C, h->st));
  return Status::Ok();
}
template <typename S>
Status from_mg_combine(irk_problem* h, MGBase* mg, S* out, const S* add, const CombineParams& C) {
  const LevelGeom& g = h->fine;
  if (mg->elem_size() == 4)
    IRK_LAUNCH(PROF_COMBINE, launch_combine<float, S, S>((const float*)mg->fine_x(), add, out, g.n, g.ld, C, h->st));
  else
    IRK_LAUNCH(PROF_COMBINE,
               launch_combine<double, S, S>((const double*)mg->fine_x(), add, out, g.n, g.ld, C, h->st));
  return Status::Ok();
}

// z = P^{-1} r (Eq. irk:P) with the configured MG precision
template <typename S>
Status precondition_lu(irk_problem* h, const S* r, S* z) {
  const int Q = h->Q;
  CombineParams Cin = combine_params(Q, Q, h->tab.Sinv.data());
  CombineParams Cout = combine_params(Q, Q, h->tab.S.data());
  IRK_TRY(to_mg_combine<S>(h, h->mg.get(), r, nullptr, Cin));
  IRK_TRY(h->mg->vcycle_top(h->st, h->opt.use_graph != 0));
  return from_mg_combine<S>(h, h->mg.get(), z, nullptr, Cout);
}

CombineParams scale_pair(double sa, bool with_b, double sb) {
  CombineParams C;
  std::memset(&C, 0, sizeof(C));
  C.nout = 1;
  C.nina = 1;
  C.Da[0] = sa;
  C.ninb = with_b ? 1 : 0;
  C.Db[0] = sb;
  return C;
}

// mg_b = sa in (+ sb in2)  /  out = sa mg_x (+ sb add), one vector
template <typename S>
Status to_mg(irk_problem* h, MGBase* mg, const S* in, double sa, const S* in2, double sb) {
  return to_mg_combine<S>(h, mg, in, in2, scale_pair(sa, in2 != nullptr, sb));
}
template <typename S>
Status from_mg(irk_problem* h, MGBase* mg, S* out, double sa, const S* add, double sb) {
  return from_mg_combine<S>(h, mg, out, add, scale_pair(sa, add != nullptr, sb));
}

// rhs = (A^{-1} (x) I)(g - 1 (x) K y_n), y_n FP64 (the caller's vector)
template <typename S>
Status stage_rhs(irk_problem* h, const double* y, double t_n, const double* loads, S* rhs) {
  const LevelGeom& g = h->fine;
  double zero = 0.0, one = 1.0;
  const S* yin;
  if constexpr (std::is_same<S, ff>::value) {
    IRK_LAUNCH(PROF_RHS, launch_to_ff(y, as<ff>(h->Mu), g.ld, h->st));
    yin = as<ff>(h->Mu);
  } else {
    yin = y;
  }
  IRK_TRY(launch_apply64<S>(h, yin, 1, &zero, &one, EPI_STORE, as<S>(h->Ky), nullptr, PROF_RHS));
  RhsParams R;
  std::memset(&R, 0, sizeof(R));
  R.Q = h->Q;
  for (int i = 0; i < h->Q; ++i)
    for (int j = 0; j < h->Q; ++j) R.Ainv[i * kMaxQ + j] = h->tab.Ainv[i * h->Q + j];
  const double pi = 3.14159265358979323846;
  for (int j = 0; j < h->Q; ++j) {
    const double t = t_n + h->tab.c[j] * h->tau;
    R.phi[j] = h->dim * pi * pi * std::cos(t) - std::sin(t);
  }
  IRK_LAUNCH(PROF_RHS, launch_stage_rhs<S>(g.grid(), R, as<S>(h->Ky), h->G1, h->Gv, loads, rhs, h->st));
  return Status::Ok();
}

template <typename S>
Status step_lu(irk_problem* h, double* y, double t_n, const double* loads, irk_stats* stats) {
  S* rhs = as<S>(h->rhs);
  S* kst = as<S>(h->kst);
  IRK_TRY(stage_rhs<S>(h, y, t_n, loads, rhs));
  ApplyFn<S> op = [h](const S* in, S* out) { return apply_calA<S>(h, in, out); };
  ApplyFn<S> prec = [h](const S* in, S* out) { return precondition_lu<S>(h, in, out); };
  FGMRESResult res;
  IRK_TRY(fgmres_solve<S>(h->fw, op, prec, rhs, kst, h->opt.rtol, h->opt.max_it, h->st, res));
  if (stats) {
    stats->iterations = res.iterations;
    stats->vcycles = res.iterations;
    stats->rel_residual = res.rel_residual;
    stats->reorth_passes = res.reorth;
  }
  if (!res.converged) return Status::Err(IRK_ENOTCONV, "FGMRES did not converge");
  IRK_LAUNCH(PROF_RHS, launch_update<S>(h->fine.grid(), h->Q, kst, h->tab.b.data(), h->tau, y, h->st));
  return Status::Ok();
}

template <typename S>
Status step_diag(irk_problem* h, double* y, double t_n, const double* loads, irk_stats* stats) {
  const int Q = h->Q;
  const LevelGeom& g = h->fine;
  S* rhs = as<S>(h->rhs);
  S* tq = as<S>(h->tq);
  S* kst = as<S>(h->kst);
  IRK_TRY(stage_rhs<S>(h, y, t_n, loads, rhs));
  // rtilde = (T^{-1} (x) I) rhs  -> tq
  CombineParams Cin = combine_params(Q, Q, h->tab.Tinv.data());
  IRK_LAUNCH(PROF_COMBINE, launch_combine<S, S, S>(rhs, nullptr, tq, g.n, g.ld, Cin, h->st));
  int iters = 0, vc = 0, reo = 0;
  double worst = 0.0;
  for (size_t bi = 0; bi < h->tab.blocks.size(); ++bi) {
    const auto& blk = h->tab.blocks[bi];
    MGBase* mg = h->mg_diag[bi].get();
    const int ns = blk.pair ? 2 : 1;
    FGMRESWork w = h->fwd;
    w.ns = ns;
    w.len = (long long)ns * g.ld;
    w.nb = reduction_blocks(w.len);
    S* bvec = tq + (size_t)blk.offset * g.ld;
    S* xvec = kst + (size_t)blk.offset * g.ld;
    ApplyFn<S> op, prec;
    const double al = blk.alpha, be = blk.beta, tau = h->tau;
    if (!blk.pair) {
      op = [h, al](const S* in, S* out) {
        const double Cm[1] = {al}, Ck[1] = {h->tau};
        return apply_general<S>(h, in, out, 1, Cm, Ck);
      };
      prec = [h, mg](const S* in, S* out) {
        IRK_TRY(to_mg<S>(h, mg, in, 1.0, nullptr, 0.0));
        IRK_TRY(mg->vcycle_top(h->st, h->opt.use_graph != 0));
        return from_mg<S>(h, mg, out, 1.0, nullptr, 0.0);
      };
    } else if (h->opt.pair_precond == 1) {
      op = [h, al, be, tau](const S* in, S* out) {
        const double Cm[4] = {al, -be, be, al}, Ck[4] = {tau, 0.0, 0.0, tau};
        return apply_general<S>(h, in, out, 2, Cm, Ck);
      };
      // one V-cycle on the coupled system [[alpha M + tau K, -beta M], [beta M, alpha M + tau K]]
      prec = [h, mg](const S* in, S* out) {
        const double I2[4] = {1.0, 0.0, 0.0, 1.0};
        const CombineParams C = combine_params(2, 2, I2);
        IRK_TRY(to_mg_combine<S>(h, mg, in, nullptr, C));
        IRK_TRY(mg->vcycle_top(h->st, h->opt.use_graph != 0));
        return from_mg_combine<S>(h, mg, out, nullptr, C);
      };
    } else {
      op = [h, al, be, tau](const S* in, S* out) {
        const double Cm[4] = {al, -be, be, al}, Ck[4] = {tau, 0.0, 0.0, tau};
        return apply_general<S>(h, in, out, 2, Cm, Ck);
      };
      // PRESB (Eq. presb:p): a = f + g; w1 = H^{-1} a; w2 = H^{-1}(g - beta M w1); out = (w1 - w2, w2)
      prec = [h, mg, be](const S* in, S* out) {
        const LevelGeom& gg = h->fine;
        const S* f = in;
        const S* gv = in + gg.ld;
        S* o1 = out;
        S* o2 = out + gg.ld;
        IRK_TRY(to_mg<S>(h, mg, f, 1.0, gv, 1.0));
        IRK_TRY(mg->vcycle_top(h->st, h->opt.use_graph != 0));
        IRK_TRY(from_mg<S>(h, mg, o1, 1.0, nullptr, 0.0));        // o1 = w1
        // b2 = g - beta M w1: M w1 FP64-accurate through the fine operator (ns = 1)
        const double Cm[1] = {be}, Ck[1] = {0.0};
        IRK_TRY(apply_general<S>(h, o1, o2, 1, Cm, Ck));          // o2 = beta M w1
        IRK_TRY(to_mg<S>(h, mg, gv, 1.0, o2, -1.0));
        IRK_TRY(mg->vcycle_top(h->st, h->opt.use_graph != 0));
        IRK_TRY(from_mg<S>(h, mg, o2, 1.0, nullptr, 0.0));        // o2 = w2
        return from_mg<S>(h, mg, o1, -1.0, o1, 1.0);              // o1 = w1 - w2
      };
    }
    FGMRESResult res;
    IRK_TRY(fgmres_solve<S>(w, op, prec, bvec, xvec, h->opt.rtol, h->opt.max_it, h->st, res));
    iters += res.iterations;
    reo += res.reorth;
    vc += res.iterations * ((blk.pair && h->opt.pair_precond == 0) ? 2 : 1);
    worst = std::max(worst, res.rel_residual);
    if (!res.converged) {
      if (stats) { stats->iterations = iters; stats->vcycles = vc; stats->rel_residual = worst; stats->reorth_passes = reo; }
      return Status::Err(IRK_ENOTCONV, "FGMRES did not converge on a diagonal block");
    }
  }
  // k = (T (x) I) x~
  CombineParams Cout = combine_params(Q, Q, h->tab.T.data());
  IRK_LAUNCH(PROF_COMBINE, launch_combine<S, S, S>(kst, nullptr, tq, g.n, g.ld, Cout, h->st));
  if (stats) { stats->iterations = iters; stats->vcycles = vc; stats->rel_residual = worst; stats->reorth_passes = reo; }
  IRK_LAUNCH(PROF_RHS, launch_update<S>(g.grid(), Q, tq, h->tab.b.data(), h->tau, y, h->st));
  return Status::Ok();
}

// ---- groups of requests (irk_create_group): shared launches, one FGMRES per request ----

// v_r = (A^{-1} (x) M + tau_r I (x) K) u_r for every request r: M and K of all R Q stage vectors in
// one launch, then each request's combination with its own tau
template <typename S>
Status apply_calA_group(irk_problem* h, const S* u, S* v) {
  const int Q = h->Q, R = h->R;
  const LevelGeom& g = h->fine;
  const long long len = (long long)Q * g.ld;
  S* Mu = as<S>(h->Mu);
  S* Ku = as<S>(h->Ku);
  IRK_TRY(launch_apply64<S>(h, u, R * Q, nullptr, nullptr, EPI_DUAL, Mu, Ku));
  std::vector<double> Ck((size_t)Q * Q, 0.0);
  for (int r = 0; r < R; ++r) {
    for (int i = 0; i < Q; ++i) Ck[(size_t)i * Q + i] = h->taus[r];
    CombineParams C = combine_params(Q, Q, h->tab.Ainv.data(), Ck.data(), Q);
    IRK_LAUNCH(PROF_COMBINE, launch_combine<S, S, S>(Mu + r * len, Ku + r * len, v + r * len, g.n, g.ld, C, h->st));
  }
  return Status::Ok();
}

// z_r = P^{-1} r_r (Eq. irk:P) for every request: basis changes per request, one V-cycle over all
// R Q blocks
template <typename S>
Status precondition_group(irk_problem* h, const S* r_all, S* z_all) {
  const int Q = h->Q, R = h->R;
  const LevelGeom& g = h->fine;
  const long long len = (long long)Q * g.ld;
  MGBase* mg = h->mg.get();
  CombineParams Cin = combine_params(Q, Q, h->tab.Sinv.data());
  CombineParams Cout = combine_params(Q, Q, h->tab.S.data());
  for (int r = 0; r < R; ++r) {
    if (mg->elem_size() == 4)
      IRK_LAUNCH(PROF_COMBINE, launch_combine<S, S, float>(r_all + r * len, nullptr, (float*)mg->fine_b() + r * len,
                                                         g.n, g.ld, Cin, h->st));
    else
      IRK_LAUNCH(PROF_COMBINE, launch_combine<S, S, double>(r_all + r * len, nullptr, (double*)mg->fine_b() + r * len,
                                                          g.n, g.ld, Cin, h->st));
  }
  IRK_TRY(mg->vcycle_top(h->st, h->opt.use_graph != 0));
  for (int r = 0; r < R; ++r) {
    if (mg->elem_size() == 4)
      IRK_LAUNCH(PROF_COMBINE, launch_combine<float, S, S>((const float*)mg->fine_x() + r * len, nullptr, z_all + r * len,
                                                         g.n, g.ld, Cout, h->st));
    else
      IRK_LAUNCH(PROF_COMBINE, launch_combine<double, S, S>((const double*)mg->fine_x() + r * len, nullptr,
                                                          z_all + r * len, g.n, g.ld, Cout, h->st));
  }
  return Status::Ok();
}

// One step of every request: ys[r] (device) y_n -> y_{n+1} from t_ns[r].  Per-request results in
// stats / sts; a request that fails keeps its y.
template <typename S>
Status step_group_t(irk_problem* h, double* const* ys, const double* t_ns, std::vector<FGMRESResult>& res,
                    std::vector<Status>& sts) {
  const int Q = h->Q, R = h->R;
  const LevelGeom& g = h->fine;
  const long long len = (long long)Q * g.ld;
  double* Y = (R > 1) ? h->Yg : ys[0];
  if (R > 1)
    for (int r = 0; r < R; ++r)
      IRK_CUDA(cudaMemcpyAsync(Y + (size_t)r * g.ld, ys[r], (size_t)g.n * sizeof(double), cudaMemcpyDeviceToDevice,
                               h->st));
  // K y_n of every request in one launch
  const S* yin;
  if constexpr (std::is_same<S, ff>::value) {
    IRK_LAUNCH(PROF_RHS, launch_to_ff(Y, as<ff>(h->Mu), (long long)R * g.ld, h->st));
    yin = as<ff>(h->Mu);
  } else {
    yin = Y;
  }
  std::vector<double> zero(R, 0.0), one(R, 1.0);
  IRK_TRY(launch_apply64<S>(h, yin, R, zero.data(), one.data(), EPI_STORE, as<S>(h->Ky), nullptr, PROF_RHS));
  S* rhs = as<S>(h->rhs);
  S* kst = as<S>(h->kst);
  const double pi = 3.14159265358979323846;
  for (int r = 0; r < R; ++r) {
    RhsParams Rp;
    std::memset(&Rp, 0, sizeof(Rp));
    Rp.Q = Q;
    for (int i = 0; i < Q; ++i)
      for (int j = 0; j < Q; ++j) Rp.Ainv[i * kMaxQ + j] = h->tab.Ainv[i * Q + j];
    for (int j = 0; j < Q; ++j) {
      const double t = t_ns[r] + h->tab.c[j] * h->taus[r];
      Rp.phi[j] = h->dim * pi * pi * std::cos(t) - std::sin(t);
    }
    IRK_LAUNCH(PROF_RHS, launch_stage_rhs<S>(g.grid(), Rp, as<S>(h->Ky) + r * g.ld, h->G1, h->Gv, nullptr,
                                             rhs + r * len, h->st));
  }
  ApplyFn<S> op = [h](const S* in, S* out) { return apply_calA_group<S>(h, in, out); };
  ApplyFn<S> prec = [h](const S* in, S* out) { return precondition_group<S>(h, in, out); };
  IRK_TRY(fgmres_solve_group<S>(h->fw, R, h->gsc, op, prec, rhs, kst, h->opt.rtol, h->opt.max_it, h->st, res, sts));
  for (int r = 0; r < R; ++r) {
    if (sts[r].ok() && !res[r].converged) sts[r] = Status::Err(IRK_ENOTCONV, "FGMRES did not converge");
    if (sts[r].ok())
      IRK_LAUNCH(PROF_RHS, launch_update<S>(g.grid(), Q, kst + r * len, h->tab.b.data(), h->taus[r], ys[r], h->st));
  }
  return Status::Ok();
}

Status step(irk_problem* h, double* y, double t_n, const double* loads, irk_stats* stats) {
  const bool diag = (h->opt.variant == IRK_VARIANT_DIAG);
  if (h->opt.op_ff) return diag ? step_diag<ff>(h, y, t_n, loads, stats) : step_lu<ff>(h, y, t_n, loads, stats);
  return diag ? step_diag<double>(h, y, t_n, loads, stats) : step_lu<double>(h, y, t_n, loads, stats);
}

// The entry points below take FP64 vectors; with ff storage they go through the handle's
// stage buffers tq (input) and kst (output), which irk_step uses only inside a step.
template <typename F>
Status with_ff_io(irk_problem* h, const double* in, long long nin, double* out, long long nout, F&& f) {
  ff* a = as<ff>(h->tq);
  ff* b = as<ff>(h->kst);
  IRK_LAUNCH(PROF_COMBINE, launch_to_ff(in, a, nin, h->st));
  IRK_TRY(f(a, b));
  IRK_LAUNCH(PROF_COMBINE, launch_from_ff(b, out, nout, h->st));
  return Status::Ok();
}

// Launch shapes of the FP64-accurate fine-mesh operator: the stage operator (DUAL epilogue, Q
// stages, or the DIAG blocks' 1 and 2) and K y_n (STORE, 1 stage), timed on the handle's stage
// buffers before they hold data.
template <typename S>
Status autotune_stage_operator_t(irk_problem* h) {
  using T = typename std::conditional<std::is_same<S, ff>::value, ff, double>::type;
  const LevelGeom& g = h->fine;
  std::vector<int> counts{h->Q};
  if (h->opt.variant == IRK_VARIANT_DIAG) counts = {1, 2};
  std::vector<double> one(kMaxStages, 1.0);
  for (int ns : counts) {
    OpParams<T> P = make_op_params<T>(g, ns, one.data(), one.data());
    EpiParams<S> E;
    std::memset(&E, 0, sizeof(E));
    E.out = as<S>(h->Mu);
    E.out2 = as<S>(h->Ku);
    IRK_CUDA(tune_op<T>(h->dim, h->k, ns, as<S>(h->kst), P, EPI_DUAL, E, h->st));
  }
  OpParams<T> P1 = make_op_params<T>(g, 1, one.data(), one.data());
  EpiParams<S> E1;
  std::memset(&E1, 0, sizeof(E1));
  E1.out = as<S>(h->Ky);
  IRK_CUDA(tune_op<T>(h->dim, h->k, 1, as<S>(h->kst), P1, EPI_STORE, E1, h->st));
  return Status::Ok();
}

Status autotune_stage_operator(irk_problem* h) {
  return h->opt.op_ff ? autotune_stage_operator_t<ff>(h) : autotune_stage_operator_t<double>(h);
}

// Multigrid precision of mg_precision = 0: the preconditioner of Eq. (irk:P) maps the V-cycle's
// result back through the basis S~ (the real Jordan basis T in the DIAG variant), which magnifies
// the FP32 rounding of the V-cycle by up to cond(S~).  FP32 while cond_F(S~) 2^-24 stays about two
// orders below the V-cycle's own error contraction (cond_F <= 2e5: Q <= 5), FP64 above.
int auto_mg_precision(const Tableau& t, int variant) {
  const std::vector<double>& B = (variant == IRK_VARIANT_DIAG) ? t.T : t.S;
  const std::vector<double>& Bi = (variant == IRK_VARIANT_DIAG) ? t.Tinv : t.Sinv;
  double f = 0.0, fi = 0.0;
  for (double v : B) f += v * v;
  for (double v : Bi) fi += v * v;
  return std::sqrt(f * fi) <= 2e5 ? 32 : 64;
}

Status create(const irk_mesh* mesh, int degree, int Q, double tau, const irk_options* opt, void* stream,
              irk_problem* h, int R = 1, const double* taus = nullptr) {
  if (!mesh) return Status::Err(IRK_EINVAL, "mesh is NULL");
  if (mesh->dim != 2 && mesh->dim != 3) return Status::Err(IRK_EINVAL, "dim must be 2 or 3");
  if (mesh->cells_per_axis < 1 || mesh->cells_per_axis > 4096) return Status::Err(IRK_EINVAL, "cells_per_axis out of range");
  if (degree < 1 || degree > 4) return Status::Err(IRK_EINVAL, "degree must be in 1..4");
  if (Q < 1 || Q > 9) return Status::Err(IRK_EINVAL, "Q must be in 1..9");
  if (!(tau > 0) || !std::isfinite(tau)) return Status::Err(IRK_EINVAL, "tau must be positive");
  if (degree * mesh->cells_per_axis < 2) return Status::Err(IRK_EINVAL, "mesh has no interior node");
  irk_default_options(&h->opt);
  if (opt) h->opt = *opt;
  const irk_options& o = h->opt;
  if (!(o.rtol > 0) || o.max_it < 1 || o.restart < 1 || o.restart > 60 || o.cheb_degree < 1 || o.cheb_degree > 16 ||
      (o.mg_precision != 0 && o.mg_precision != 32 && o.mg_precision != 64) || (o.variant != IRK_VARIANT_LU && o.variant != IRK_VARIANT_DIAG) ||
      o.eig_steps < 2 || !(o.smoothing_range > 1) || !(o.eig_safety >= 1) ||
      (o.pair_precond != 0 && o.pair_precond != 1) || !(o.deform >= 0) || (o.gs_reorth != 0 && o.gs_reorth != 1) ||
      (o.deform > 0 && !deform_valid(mesh->dim, o.deform)))
    return Status::Err(IRK_EINVAL, "invalid options");
  if (o.variant == IRK_VARIANT_DIAG && Q < 2) return Status::Err(IRK_EINVAL, "DIAG variant needs Q >= 2");
  if (R < 1 || R * Q > kMaxStages) return Status::Err(IRK_EINVAL, "a group holds 1..16/Q requests");
  if (R > 1 && (o.variant != IRK_VARIANT_LU || o.deform > 0))
    return Status::Err(IRK_EINVAL, "groups of requests use the LU variant on the Cartesian mesh");
  h->R = R;
  h->taus.assign(R, tau);
  if (taus)
    for (int r = 0; r < R; ++r) {
      if (!(taus[r] > 0) || !std::isfinite(taus[r])) return Status::Err(IRK_EINVAL, "tau must be positive");
      h->taus[r] = taus[r];
    }
  tau = h->taus[0];
  // curved mesh: FP64 stage vectors; op_ff picks the operator's arithmetic (float-float or FP64)
  const int deform_ff = o.op_ff;
  if (o.deform > 0) h->opt.op_ff = 0;
  h->dim = mesh->dim;
  h->N = mesh->cells_per_axis;
  h->k = degree;
  h->Q = Q;
  h->tau = tau;
  h->st = (cudaStream_t)stream;
  h->prof.st = h->st;
  h->arena.set_stream(h->st);
  IRK_CUDA(cudaGetDevice(&h->device));
  std::string err;
  if (!build_tableau(Q, h->tab, err)) return Status::Err(IRK_EINVAL, err);
  if (o.mg_precision == 0) h->opt.mg_precision = auto_mg_precision(h->tab, o.variant);
  if (!build_element1d(degree, h->el, err)) return Status::Err(IRK_EINVAL, err);
  h->fine = make_level(h->dim, degree, h->N, h->el);
  const LevelGeom& g = h->fine;
  h->nslots = std::max(R * Q, 2);
  const size_t vq = (size_t)h->nslots * g.ld * sizeof(double);
  IRK_TRY(h->arena.alloc((void**)&h->Ky, (size_t)R * g.ld * sizeof(double)));
  if (R > 1) IRK_TRY(h->arena.alloc((void**)&h->Yg, (size_t)R * g.ld * sizeof(double)));
  IRK_TRY(h->arena.alloc((void**)&h->rhs, vq));
  IRK_TRY(h->arena.alloc((void**)&h->kst, vq));
  IRK_TRY(h->arena.alloc((void**)&h->Mu, vq));
  IRK_TRY(h->arena.alloc((void**)&h->Ku, vq));
  IRK_TRY(h->arena.alloc((void**)&h->tq, vq));
  // 1D load vector G1[j] = int sin(pi x) phi_j (Gauss k+1 per cell) and node coordinates
  {
    const int n1 = g.n1, p = degree + 1;
    std::vector<long double> G1(n1, 0.0L), xn(n1, 0.0L);
    // Gauss rule on [0,1]
    std::vector<long double> gq(p), gw(p);
    for (int i = 0; i < p; ++i) {
      long double s = std::cos(3.14159265358979323846264338327950288L * (i + 0.75L) / (p + 0.5L));
      for (int it = 0; it < 100; ++it) {
        long double p0 = 1, p1 = s;
        for (int jj = 1; jj < p; ++jj) { long double p2 = ((2 * jj + 1) * s * p1 - jj * p0) / (jj + 1); p0 = p1; p1 = p2; }
        long double dp = p * (s * p1 - p0) / (s * s - 1);
        long double ds = p1 / dp;
        s -= ds;
        if (std::fabs((double)ds) < 1e-30) break;
      }
      long double p0 = 1, p1 = s;
      for (int jj = 1; jj < p; ++jj) { long double p2 = ((2 * jj + 1) * s * p1 - jj * p0) / (jj + 1); p0 = p1; p1 = p2; }
      long double dp = p * (s * p1 - p0) / (s * s - 1);
      gq[i] = 0.5L * (s + 1);
      gw[i] = 1.0L / ((1 - s * s) * dp * dp);
    }
    const long double hh = 1.0L / h->N, pil = 3.14159265358979323846264338327950288L;
    for (int c = 0; c < h->N; ++c) {
      for (int r = 0; r <= degree; ++r) xn[degree * c + r] = (c + (long double)h->el.nodes[r]) * hh;
      for (int q = 0; q < p; ++q) {
        const long double xq = (c + gq[q]) * hh;
        const long double sv = std::sin(pil * xq) * gw[q] * hh;
        for (int i = 0; i < p; ++i) {
          long double li = 1;
          for (int m = 0; m < p; ++m)
            if (m != i) li *= (gq[q] - h->el.nodes[m]) / ((long double)h->el.nodes[i] - h->el.nodes[m]);
          G1[degree * c + i] += sv * li;
        }
      }
    }
    G1[0] = 0;
    G1[n1 - 1] = 0;
    std::vector<double> G1d(G1.begin(), G1.end()), xd(xn.begin(), xn.end());
    IRK_TRY(h->arena.alloc((void**)&h->G1, n1 * sizeof(double)));
    IRK_TRY(h->arena.alloc((void**)&h->x1d, n1 * sizeof(double)));
    IRK_CUDA(cudaMemcpyAsync(h->G1, G1d.data(), n1 * sizeof(double), cudaMemcpyHostToDevice, h->st));
    IRK_CUDA(cudaMemcpyAsync(h->x1d, xd.data(), n1 * sizeof(double), cudaMemcpyHostToDevice, h->st));
    IRK_CUDA(cudaStreamSynchronize(h->st));
  }
  if (o.deform > 0) {  // curved mesh: mapping data per cell and Gauss point, load vector
    h->deformed = true;
    if (!build_deform_geometry(h->dim, h->N, h->el, o.deform, h->dgeom, err)) return Status::Err(IRK_EINVAL, err);
    const DeformGeom& dg = h->dgeom;
    double *geo = nullptr, *eM = nullptr, *eK = nullptr;
    const size_t ecell = (size_t)dg.ncell * h->nslots * dg.nq * sizeof(double);
    IRK_TRY(h->arena.alloc((void**)&geo, dg.geo.size() * sizeof(double)));
    IRK_TRY(h->arena.alloc((void**)&eM, ecell));
    IRK_TRY(h->arena.alloc((void**)&eK, ecell));
    IRK_TRY(h->arena.alloc((void**)&h->Gv, g.ld * sizeof(double)));
    std::vector<double> Gload;
    deform_load_vector(dg, h->el, Gload);
    IRK_CUDA(cudaMemcpyAsync(geo, dg.geo.data(), dg.geo.size() * sizeof(double), cudaMemcpyHostToDevice, h->st));
    IRK_CUDA(cudaMemcpyAsync(h->Gv, Gload.data(), Gload.size() * sizeof(double), cudaMemcpyHostToDevice, h->st));
    IRK_CUDA(cudaStreamSynchronize(h->st));
    h->dgeom.geo.clear();
    h->dgeom.geo.shrink_to_fit();
    h->dd.dim = h->dim;
    h->dd.N = h->N;
    h->dd.k = degree;
    h->dd.max_ns = h->nslots;
    h->dd.ff = deform_ff;
    h->dd.ncell = dg.ncell;
    h->dd.geo = geo;
    h->dd.eM = eM;
    h->dd.eK = eK;
    h->dd.B = h->el.B.data();
    h->dd.D = h->el.D.data();
  }
  MGConfig mc;
  mc.dim = h->dim; mc.k = degree; mc.N = h->N; mc.tau = tau;
  mc.cheb_degree = o.cheb_degree; mc.eig_steps = o.eig_steps;
  mc.smoothing_range = o.smoothing_range; mc.eig_safety = o.eig_safety;
  mc.shared_cheb = o.shared_cheb; mc.batched = o.batched; mc.precision = o.mg_precision;
  mc.autotune = o.autotune;
  // LU blocks (also used by the per-step entry points of the C ABI); a group's blocks are [R][Q]
  mc.nb = R * Q;
  mc.cm.clear();
  for (int r = 0; r < R; ++r) mc.cm.insert(mc.cm.end(), h->tab.lam.begin(), h->tab.lam.end());
  if (R > 1)
    for (int r = 0; r < R; ++r) mc.taus.insert(mc.taus.end(), Q, h->taus[r]);
  mc.shape_ns = Q;
  IRK_TRY(make_mg(mc, h->el, h->arena, h->st, h->mg));
  IRK_TRY(fgmres_alloc(h->fw, R * Q, g.ld, o.restart, h->arena, h->st));
  h->fw.always_two_passes = o.gs_reorth;
  IRK_TRY(group_scalars_alloc(h->gsc, R, h->arena, h->st));
  if (o.variant == IRK_VARIANT_DIAG) {
    for (const auto& blk : h->tab.blocks) {
      MGConfig md = mc;
      md.shape_ns = 0;
      md.nb = 1;
      md.shared_cheb = 0;
      md.cm = {blk.pair ? blk.alpha + blk.beta : blk.alpha};
      if (blk.pair && o.pair_precond == 1) {  // one V-cycle on the coupled 2x2 block
        md.nb = 2;
        md.batched = 1;
        md.cm = {blk.alpha, blk.alpha};
        md.coupled_beta = blk.beta;
      }
      std::unique_ptr<MGBase> m;
      IRK_TRY(make_mg(md, h->el, h->arena, h->st, m));
      h->mg_diag.push_back(std::move(m));
    }
    IRK_TRY(fgmres_alloc(h->fwd, 2, g.ld, o.restart, h->arena, h->st));
    h->fwd.always_two_passes = o.gs_reorth;
  }
  if (o.autotune && !h->deformed) IRK_TRY(autotune_stage_operator(h));
  IRK_CUDA(cudaStreamSynchronize(h->st));
  return Status::Ok();
}

// Makes the handle's GPU current for one call and restores the caller's device afterwards: kernels
// can only be launched into a stream of the current device, and a process may drive several GPUs.
struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(int dev) {
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != dev && cudaSetDevice(dev) == cudaSuccess) prev = cur;
    cudaGetLastError();
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

template <typename F>
irk_status guarded(irk_problem* h, F&& f) {
  if (!h) return IRK_EINVAL;
  DeviceScope dev(h->device);
  ProfBind bind(&h->prof);
  try {
    Status s = f();
    if (!s.ok()) return fail(h, s);
    return IRK_OK;
  } catch (const std::bad_alloc&) {
    return fail(h, Status::Err(IRK_ENOMEM, "host allocation failed"));
  } catch (...) {
    return fail(h, Status::Err(IRK_ECUDA, "unexpected exception"));
  }
}

// the hierarchy the irk_mg_* entry points act on: the LU blocks, or one DIAG block (irk_mg_select)
MGBase* lu_mg(irk_problem* h) { return h->mg_sel == 0 ? h->mg.get() : h->mg_diag[h->mg_sel - 1].get(); }

}  // namespace

// Restriction into library-owned scratch, for the allocation-free entry point (noalloc.cu).  The
// kernels run on the handle's stream, on the GPU the handle was created on, so the scratch address
// is looked up for that device with that device current; the caller's current device is restored
// afterwards.  `resolve` returns the array's device address and size for a device index, or a
// status and a one-line reason that become the handle's last error.
using ScratchResolver = irk_status (*)(int device, void** addr, size_t* bytes, const char** why);
irk_status irk_restrict_scratch_impl(irk_handle h, int level, const void* r, void* bc, ScratchResolver resolve) {
  return guarded(h, [&]() -> Status {
    if (!r || !bc || level < 0 || level + 1 >= lu_mg(h)->levels())
      return Status::Err(IRK_EINVAL, "bad arguments");
    int cur = -1;
    IRK_CUDA(cudaGetDevice(&cur));
    if (cur != h->device) IRK_CUDA(cudaSetDevice(h->device));
    void* scratch = nullptr;
    size_t bytes = 0;
    const char* why = "";
    const irk_status rs = resolve(h->device, &scratch, &bytes, &why);
    if (cur != h->device) IRK_CUDA(cudaSetDevice(cur));
    if (rs != IRK_OK) return Status::Err(rs, std::string("scratch array: ") + why);
    return lu_mg(h)->restrict_in_scratch(level, r, bc, scratch, bytes, h->st);
  });
}

extern "C" {

void irk_default_options(irk_options* o) {
  if (!o) return;
  o->rtol = 1e-10;
  o->max_it = 200;
  o->restart = 30;
  o->cheb_degree = 3;
  o->variant = IRK_VARIANT_LU;
  o->mg_precision = 0;
  o->batched = 1;
  o->use_graph = 1;
  o->eig_steps = 20;
  o->smoothing_range = 10.0;
  o->eig_safety = 1.2;
  o->shared_cheb = 0;
  o->op_ff = 0;
  o->autotune = 1;
  o->pair_precond = 0;
  o->deform = 0.0;
  o->gs_reorth = 0;
}

irk_status irk_create(const irk_mesh* mesh, int degree, int Q, double tau, const irk_options* opt,
                      void* cuda_stream, irk_handle* out) {
  if (!out) return IRK_EINVAL;
  *out = nullptr;
  irk_problem* h = nullptr;
  try {
    h = new irk_problem();
  } catch (...) {
    return IRK_ENOMEM;
  }
  Status s;
  try {
    s = create(mesh, degree, Q, tau, opt, cuda_stream, h);
  } catch (const std::bad_alloc&) {
    s = Status::Err(IRK_ENOMEM, "host allocation failed");
  } catch (...) {
    s = Status::Err(IRK_ECUDA, "unexpected exception");
  }
  if (!s.ok()) {
    cudaStreamSynchronize((cudaStream_t)cuda_stream);
    delete h;
    return s.code;
  }
  *out = h;
  return IRK_OK;
}

irk_status irk_create_group(const irk_mesh* mesh, int degree, int Q, int R, const double* taus,
                            const irk_options* opt, void* cuda_stream, irk_handle* out) {
  if (!out) return IRK_EINVAL;
  *out = nullptr;
  if (!taus || R < 1) return IRK_EINVAL;
  irk_problem* h = nullptr;
  try {
    h = new irk_problem();
  } catch (...) {
    return IRK_ENOMEM;
  }
  Status s;
  try {
    s = create(mesh, degree, Q, taus[0], opt, cuda_stream, h, R, taus);
  } catch (const std::bad_alloc&) {
    s = Status::Err(IRK_ENOMEM, "host allocation failed");
  } catch (...) {
    s = Status::Err(IRK_ECUDA, "unexpected exception");
  }
  if (!s.ok()) {
    cudaStreamSynchronize((cudaStream_t)cuda_stream);
    delete h;
    return s.code;
  }
  *out = h;
  return IRK_OK;
}

int irk_group_size(irk_handle h) { return h ? h->R : -1; }

irk_status irk_step_group(irk_handle h, double* const* ys, const double* t_ns, irk_stats* stats,
                          irk_status* per_item) {
  return guarded(h, [&]() -> Status {
    if (!ys || !t_ns) return Status::Err(IRK_EINVAL, "ys or t_ns is NULL");
    for (int r = 0; r < h->R; ++r)
      if (!ys[r]) return Status::Err(IRK_EINVAL, "ys holds a NULL vector");
    if (h->opt.variant != IRK_VARIANT_LU || h->deformed)
      return Status::Err(IRK_EINVAL, "group steps use the LU variant on the Cartesian mesh");
    auto t0 = std::chrono::steady_clock::now();
    std::vector<FGMRESResult> res;
    std::vector<Status> sts;
    Status s = h->opt.op_ff ? step_group_t<ff>(h, ys, t_ns, res, sts) : step_group_t<double>(h, ys, t_ns, res, sts);
    IRK_CUDA(cudaStreamSynchronize(h->st));
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (!s.ok()) return s;
    Status first = Status::Ok();
    for (int r = 0; r < h->R; ++r) {
      if (stats) {
        stats[r].iterations = res[r].iterations;
        stats[r].vcycles = res[r].iterations;
        stats[r].rel_residual = res[r].rel_residual;
        stats[r].reorth_passes = res[r].reorth;
        stats[r].ms_total = ms;
      }
      if (per_item) per_item[r] = sts[r].code;
      if (!sts[r].ok() && first.ok()) first = sts[r];
    }
    return first;
  });
}

irk_status irk_set_tau(irk_handle h, const double* taus) {
  return guarded(h, [&]() -> Status {
    if (!taus) return Status::Err(IRK_EINVAL, "taus is NULL");
    if (h->opt.variant != IRK_VARIANT_LU) return Status::Err(IRK_EINVAL, "irk_set_tau needs the LU variant");
    for (int r = 0; r < h->R; ++r)
      if (!(taus[r] > 0) || !std::isfinite(taus[r])) return Status::Err(IRK_EINVAL, "tau must be positive");
    std::vector<double> blocks;
    for (int r = 0; r < h->R; ++r) blocks.insert(blocks.end(), h->Q, taus[r]);
    IRK_TRY(h->mg->retau(blocks, h->st));
    for (int r = 0; r < h->R; ++r) h->taus[r] = taus[r];
    h->tau = taus[0];
    return Status::Ok();
  });
}

irk_status irk_step(irk_handle h, double* y, double t_n, const double* stage_load, irk_stats* stats) {
  return guarded(h, [&]() -> Status {
    if (!y) return Status::Err(IRK_EINVAL, "y is NULL");
    if (h->R > 1) return Status::Err(IRK_EINVAL, "a group handle steps with irk_step_group");
    auto t0 = std::chrono::steady_clock::now();
    Status s = step(h, y, t_n, stage_load, stats);
    IRK_CUDA(cudaStreamSynchronize(h->st));
    if (stats) stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return s;
  });
}

irk_status irk_solve_batch(irk_handle* hs, double** ys, const double* t_ns, int count, irk_status* per_item) {
  if (count < 0 || (count > 0 && (!hs || !ys || !t_ns))) return IRK_EINVAL;
  if (count == 0) return IRK_OK;
  // Items of one handle run in order on one host thread (a handle is not thread-safe); distinct
  // handles run on their own threads, so their streams' kernels overlap and each thread's
  // per-iteration residual read-back waits only for its own stream.
  std::vector<std::vector<int>> groups;
  {
    std::map<irk_handle, int> gid;
    for (int i = 0; i < count; ++i) {
      auto it = gid.find(hs[i]);
      if (it == gid.end()) {
        it = gid.emplace(hs[i], (int)groups.size()).first;
        groups.emplace_back();
      }
      groups[it->second].push_back(i);
    }
  }
  std::vector<irk_status> st(count, IRK_OK);
  auto run_group = [&](int g) {
    const std::vector<int>& items = groups[g];
    if (hs[items[0]]) cudaSetDevice(hs[items[0]]->device);
    for (int i : items) st[i] = irk_step(hs[i], ys[i], t_ns[i], nullptr, nullptr);
  };
  const int nthreads = (int)std::min<size_t>(groups.size(), 64);
  if (nthreads <= 1) {
    for (size_t g = 0; g < groups.size(); ++g) run_group((int)g);
  } else {
    std::atomic<int> next{0};
    int device = 0;
    cudaGetDevice(&device);
    std::vector<std::thread> pool;
    try {
      for (int t = 0; t < nthreads; ++t)
        pool.emplace_back([&]() {
          cudaSetDevice(device);
          for (int g; (g = next.fetch_add(1)) < (int)groups.size();) run_group(g);
        });
    } catch (...) {
      // could not start every thread: the started ones (or this thread) take the remaining groups
    }
    for (int g; (g = next.fetch_add(1)) < (int)groups.size();) run_group(g);
    for (auto& th : pool) th.join();
  }
  irk_status first = IRK_OK;
  for (int i = 0; i < count; ++i) {
    if (per_item) per_item[i] = st[i];
    if (st[i] != IRK_OK && first == IRK_OK) first = st[i];
  }
  return first;
}

irk_status irk_destroy(irk_handle h) {
  if (!h) return IRK_OK;
  {
    DeviceScope dev(h->device);  // the handle's memory, graphs and events are freed on its GPU
    cudaStreamSynchronize(h->st);
    delete h;
  }
  return IRK_OK;
}

long long irk_ndofs(irk_handle h) { return h ? h->fine.n : -1; }
long long irk_ninterior(irk_handle h) {
  if (!h) return -1;
  long long m = 1;
  for (int a = 0; a < h->dim; ++a) m *= (h->fine.n1 - 2);
  return m;
}
long long irk_stage_stride(irk_handle h) { return h ? h->fine.ld : -1; }
int irk_num_levels(irk_handle h) { return h ? h->mg->levels() : -1; }

const char* irk_strerror(irk_status s) {
  switch (s) {
    case IRK_OK: return "ok";
    case IRK_EINVAL: return "invalid argument";
    case IRK_ENOMEM: return "out of device memory";
    case IRK_ENOTCONV: return "FGMRES did not converge";
    case IRK_ENUMERIC: return "non-finite value";
    case IRK_ETIMEOUT: return "device wait timed out";
    case IRK_ECUDA: return "CUDA runtime error";
    case IRK_EBUSY: return "admission refused";
  }
  return "unknown status";
}

const char* irk_last_error(irk_handle h) { return h ? h->last_err.c_str() : "NULL handle"; }

int irk_autotune_report(char* buf, int len) { return tune_report(buf, len); }

irk_status irk_op_shape_force(int elem_bytes, int cxs, int zc, int cluster) {
  if (elem_bytes != 4 && elem_bytes != 8) return IRK_EINVAL;
  if (cxs != 0 && ((cxs != 8 && cxs != 16 && cxs != 32) || zc < 1 || zc > 4096 || (cluster != 0 && cluster != 1)))
    return IRK_EINVAL;
  op_shape_force(elem_bytes, cxs, zc, cluster);
  return IRK_OK;
}

irk_status irk_op_shape_last(int elem_bytes, int* out4) {
  if ((elem_bytes != 4 && elem_bytes != 8) || !out4) return IRK_EINVAL;
  if (!op_shape_last(elem_bytes, out4))
    for (int i = 0; i < 4; ++i) out4[i] = -1;
  return IRK_OK;
}

irk_status irk_interpolate_initial(irk_handle h, double* y, double t) {
  return guarded(h, [&]() -> Status {
    if (!y) return Status::Err(IRK_EINVAL, "y is NULL");
    if (h->deformed) {  // interpolant at the mapped nodes, built on the host
      std::vector<double> y0;
      deform_initial_value(h->dgeom, h->el, t, y0);
      IRK_CUDA(cudaMemcpyAsync(y, y0.data(), y0.size() * sizeof(double), cudaMemcpyHostToDevice, h->st));
      IRK_CUDA(cudaStreamSynchronize(h->st));
      return Status::Ok();
    }
    IRK_LAUNCH(PROF_RHS, launch_interpolate(h->fine.grid(), h->x1d, std::cos(t), y, h->st));
    return Status::Ok();
  });
}

namespace {
// factor `which` of irk_get_tableau / irk_tableau_factors (nullptr: unknown)
const std::vector<double>* tableau_field(const Tableau& t, int which) {
  switch (which) {
    case 0: return &t.A;
    case 1: return &t.b;
    case 2: return &t.c;
    case 3: return &t.Ainv;
    case 4: return &t.L;
    case 5: return &t.U;
    case 6: return &t.S;
    case 7: return &t.Sinv;
    case 8: return &t.lam;
    case 9: return &t.T;
    case 10: return &t.Tinv;
    case 11: return &t.J;
    default: return nullptr;
  }
}
}  // namespace

irk_status irk_get_tableau(irk_handle h, int which, double* out) {
  return guarded(h, [&]() -> Status {
    if (!out) return Status::Err(IRK_EINVAL, "out is NULL");
    const std::vector<double>* src = tableau_field(h->tab, which);
    if (!src) return Status::Err(IRK_EINVAL, "unknown tableau factor");
    std::memcpy(out, src->data(), src->size() * sizeof(double));
    return Status::Ok();
  });
}

irk_status irk_tableau_factors(int Q, int which, double* out) {
  if (!out || Q < 1 || Q > kMaxQ) return IRK_EINVAL;
  try {
    Tableau t;
    std::string err;
    if (!build_tableau(Q, t, err)) return IRK_ENUMERIC;
    const std::vector<double>* src = tableau_field(t, which);
    if (!src) return IRK_EINVAL;
    std::memcpy(out, src->data(), src->size() * sizeof(double));
    return IRK_OK;
  } catch (const std::bad_alloc&) {
    return IRK_ENOMEM;
  } catch (...) {
    return IRK_ENUMERIC;
  }
}

irk_status irk_element_factors(int k, int which, double* out) {
  if (!out || k < 1 || k > kMaxDeg) return IRK_EINVAL;
  try {
    Element1D e;
    std::string err;
    if (!build_element1d(k, e, err)) return IRK_ENUMERIC;
    const std::vector<double>* src = nullptr;
    switch (which) {
      case 0: src = &e.nodes; break;
      case 1: src = &e.Me; break;
      case 2: src = &e.Ke; break;
      case 3: src = &e.Pc; break;
      case 4: src = &e.gq; break;
      case 5: src = &e.gw; break;
      case 6: src = &e.B; break;
      case 7: src = &e.D; break;
      default: return IRK_EINVAL;
    }
    std::memcpy(out, src->data(), src->size() * sizeof(double));
    return IRK_OK;
  } catch (const std::bad_alloc&) {
    return IRK_ENOMEM;
  } catch (...) {
    return IRK_ENUMERIC;
  }
}

irk_status irk_get_cheb_interval(irk_handle h, int level, int block, double* out) {
  return guarded(h, [&]() -> Status {
    const int nb = h->mg_sel == 0 ? h->Q : (h->tab.blocks[h->mg_sel - 1].pair && h->opt.pair_precond == 1 ? 2 : 1);
    if (!out || level < 0 || level + 1 >= lu_mg(h)->levels() || block < 0 || block >= nb)
      return Status::Err(IRK_EINVAL, "bad level/block");
    lu_mg(h)->interval(level, block, &out[0], &out[1]);
    return Status::Ok();
  });
}

irk_status irk_apply_op(irk_handle h, const double* u, double* v, int ns, const double* Cm, const double* Ck) {
  return guarded(h, [&]() -> Status {
    if (!u || !v || !Cm || !Ck || ns < 1 || ns > kMaxQ) return Status::Err(IRK_EINVAL, "bad arguments");
    if (ns > h->nslots) return Status::Err(IRK_EINVAL, "too many stage vectors for this handle");
    if (!h->opt.op_ff) return apply_general<double>(h, u, v, ns, Cm, Ck);
    const long long len = (long long)ns * h->fine.ld;
    return with_ff_io(h, u, len, v, len, [&](const ff* a, ff* b) { return apply_general<ff>(h, a, b, ns, Cm, Ck); });
  });
}

irk_status irk_apply(irk_handle h, const double* u, double* v) {
  return guarded(h, [&]() -> Status {
    if (!u || !v) return Status::Err(IRK_EINVAL, "bad arguments");
    if (h->R > 1) {  // every request's stage vectors, [R][Q][stride]
      if (!h->opt.op_ff) return apply_calA_group<double>(h, u, v);
      const long long len = (long long)h->R * h->Q * h->fine.ld;
      return with_ff_io(h, u, len, v, len, [&](const ff* a, ff* b) { return apply_calA_group<ff>(h, a, b); });
    }
    if (!h->opt.op_ff) return apply_calA<double>(h, u, v);
    const long long len = (long long)h->Q * h->fine.ld;
    return with_ff_io(h, u, len, v, len, [&](const ff* a, ff* b) { return apply_calA<ff>(h, a, b); });
  });
}

irk_status irk_stage_rhs(irk_handle h, const double* y, double t_n, double* rhs) {
  return guarded(h, [&]() -> Status {
    if (!y || !rhs) return Status::Err(IRK_EINVAL, "bad arguments");
    if (h->R > 1) return Status::Err(IRK_EINVAL, "a group handle forms its right-hand sides in irk_step_group");
    if (!h->opt.op_ff) return stage_rhs<double>(h, y, t_n, nullptr, rhs);
    IRK_TRY(stage_rhs<ff>(h, y, t_n, nullptr, as<ff>(h->kst)));
    IRK_LAUNCH(PROF_RHS, launch_from_ff(as<ff>(h->kst), rhs, (long long)h->Q * h->fine.ld, h->st));
    return Status::Ok();
  });
}

irk_status irk_precondition(irk_handle h, const double* r, double* z) {
  return guarded(h, [&]() -> Status {
    if (!r || !z) return Status::Err(IRK_EINVAL, "bad arguments");
    if (h->R > 1) {  // every request's stage vectors, [R][Q][stride]
      if (!h->opt.op_ff) return precondition_group<double>(h, r, z);
      const long long len = (long long)h->R * h->Q * h->fine.ld;
      return with_ff_io(h, r, len, z, len, [&](const ff* a, ff* b) { return precondition_group<ff>(h, a, b); });
    }
    if (!h->opt.op_ff) return precondition_lu<double>(h, r, z);
    const long long len = (long long)h->Q * h->fine.ld;
    return with_ff_io(h, r, len, z, len, [&](const ff* a, ff* b) { return precondition_lu<ff>(h, a, b); });
  });
}

irk_status irk_basis_to_mg(irk_handle h, const double* r, void* b) {
  return guarded(h, [&]() -> Status {
    if (!r || !b) return Status::Err(IRK_EINVAL, "bad arguments");
    if (h->opt.variant != IRK_VARIANT_LU || h->R > 1)
      return Status::Err(IRK_EINVAL, "the basis changes of the LU variant, one request per handle");
    const LevelGeom& g = h->fine;
    const CombineParams C = combine_params(h->Q, h->Q, h->tab.Sinv.data());
    if (h->mg->elem_size() == 4)
      IRK_LAUNCH(PROF_COMBINE, launch_combine<double, double, float>(r, nullptr, (float*)b, g.n, g.ld, C, h->st));
    else
      IRK_LAUNCH(PROF_COMBINE, launch_combine<double, double, double>(r, nullptr, (double*)b, g.n, g.ld, C, h->st));
    return Status::Ok();
  });
}

irk_status irk_basis_from_mg(irk_handle h, const void* x, double* z) {
  return guarded(h, [&]() -> Status {
    if (!x || !z) return Status::Err(IRK_EINVAL, "bad arguments");
    if (h->opt.variant != IRK_VARIANT_LU || h->R > 1)
      return Status::Err(IRK_EINVAL, "the basis changes of the LU variant, one request per handle");
    const LevelGeom& g = h->fine;
    const CombineParams C = combine_params(h->Q, h->Q, h->tab.S.data());
    if (h->mg->elem_size() == 4)
      IRK_LAUNCH(PROF_COMBINE,
                 launch_combine<float, double, double>((const float*)x, nullptr, z, g.n, g.ld, C, h->st));
    else
      IRK_LAUNCH(PROF_COMBINE,
                 launch_combine<double, double, double>((const double*)x, nullptr, z, g.n, g.ld, C, h->st));
    return Status::Ok();
  });
}

long long irk_level_ndofs(irk_handle h, int level) {
  if (!h || level < 0 || level >= h->mg->levels()) return -1;
  return h->mg->geom(level).n;
}
long long irk_level_stride(irk_handle h, int level) {
  if (!h || level < 0 || level >= h->mg->levels()) return -1;
  return h->mg->geom(level).ld;
}

irk_status irk_mg_smooth(irk_handle h, int level, const void* b, void* x, int x_is_zero) {
  return guarded(h, [&]() -> Status {
    if (!b || !x || level < 0 || level + 1 >= lu_mg(h)->levels()) return Status::Err(IRK_EINVAL, "bad arguments");
    return lu_mg(h)->smooth(level, b, x, x_is_zero, h->st);
  });
}
irk_status irk_mg_residual(irk_handle h, int level, const void* b, const void* x, void* r) {
  return guarded(h, [&]() -> Status {
    if (!b || !x || !r || level < 0 || level >= lu_mg(h)->levels()) return Status::Err(IRK_EINVAL, "bad arguments");
    return lu_mg(h)->residual(level, b, x, r, h->st);
  });
}
irk_status irk_mg_restrict(irk_handle h, int level, const void* r, void* bc) {
  return guarded(h, [&]() -> Status {
    if (!r || !bc || level < 0 || level + 1 >= lu_mg(h)->levels()) return Status::Err(IRK_EINVAL, "bad arguments");
    return lu_mg(h)->restrict_to(level, r, bc, h->st);
  });
}
irk_status irk_mg_prolongate(irk_handle h, int level, const void* ec, void* x) {
  return guarded(h, [&]() -> Status {
    if (!ec || !x || level < 0 || level + 1 >= lu_mg(h)->levels()) return Status::Err(IRK_EINVAL, "bad arguments");
    return lu_mg(h)->prolongate_add(level, ec, x, h->st);
  });
}
irk_status irk_mg_coarse_solve(irk_handle h, const void* b, void* x) {
  return guarded(h, [&]() -> Status {
    if (!b || !x) return Status::Err(IRK_EINVAL, "bad arguments");
    return lu_mg(h)->coarse_solve(b, x, h->st);
  });
}
irk_status irk_mg_select(irk_handle h, int which) {
  return guarded(h, [&]() -> Status {
    if (which < 0 || which > (int)h->mg_diag.size()) return Status::Err(IRK_EINVAL, "no such multigrid hierarchy");
    h->mg_sel = which;
    return Status::Ok();
  });
}

irk_status irk_mg_vcycle(irk_handle h, int level, const void* b, void* x) {
  return guarded(h, [&]() -> Status {
    if (!b || !x || level < 0 || level >= lu_mg(h)->levels()) return Status::Err(IRK_EINVAL, "bad arguments");
    return lu_mg(h)->vcycle_io(level, b, x, h->st);
  });
}

irk_status irk_stage_combine(irk_handle h, const double* u, int nin, double* v, int nout, const double* D) {
  return guarded(h, [&]() -> Status {
    if (!u || !v || !D || nin < 1 || nin > kMaxQ || nout < 1 || nout > kMaxQ)
      return Status::Err(IRK_EINVAL, "bad arguments");
    CombineParams C = combine_params(nout, nin, D);
    IRK_LAUNCH(PROF_COMBINE,
               launch_combine<double, double, double>(u, nullptr, v, h->fine.n, h->fine.ld, C, h->st));
    return Status::Ok();
  });
}

irk_status irk_profile(irk_handle h, unsigned mask) {
  return guarded(h, [&]() -> Status {
    IRK_CUDA(cudaStreamSynchronize(h->st));
    h->prof.reset(mask);
    return Status::Ok();
  });
}

irk_status irk_profile_read(irk_handle h, int category, double* ms, long long* launches, long long* timed) {
  return guarded(h, [&]() -> Status {
    if (category < 0 || category >= PROF_NCAT) return Status::Err(IRK_EINVAL, "unknown category");
    IRK_CUDA(cudaStreamSynchronize(h->st));
    h->prof.read(category, ms, launches, timed);
    return Status::Ok();
  });
}

irk_status irk_synchronize(irk_handle h) {
  return guarded(h, [&]() -> Status {
    IRK_CUDA(cudaStreamSynchronize(h->st));
    return Status::Ok();
  });
}

}  // extern "C"
