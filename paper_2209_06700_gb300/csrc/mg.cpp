// Geometric multigrid of libirk: one V-cycle per block (lambda_i M + tau K),
// the block solver of Eq. (irk:P) (arXiv 2209.06700, Sec. 2) with the
// smoother/coarse-solver pairing of Sec. 5: Chebyshev iteration around
// point-Jacobi; the coarsest level is solved exactly with a dense FP64
// inverse.  All blocks of a level are processed by the same launches
// (blockIdx.z = block), the batched form of Sec. 3.4, including the transfers.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "coarse_cycle.h"
#include "profiler.h"
#include "solver.h"

namespace irk {

// Stream-ordered allocations from the device's default memory pool: releasing a handle does not
// synchronise the device, so concurrent requests on other streams keep running.
DeviceArena::~DeviceArena() {
  for (auto it = ptrs_.rbegin(); it != ptrs_.rend(); ++it) cudaFreeAsync(*it, st_);
}

static void keep_pool_memory() {
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    unsigned long long keep = ~0ull;  // freed blocks stay cached in the pool for the next handle
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  done[dev] = true;
}

Status DeviceArena::alloc(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 256;
  keep_pool_memory();
  cudaError_t e = cudaMallocAsync(p, bytes, st_);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return Status::Err(IRK_ENOMEM, "allocation of " + std::to_string(bytes) + " bytes failed");
  }
  ptrs_.push_back(*p);
  total_ += bytes;
  e = cudaMemsetAsync(*p, 0, bytes, st_);
  if (e != cudaSuccess) return Status::Err(IRK_ECUDA, "cudaMemsetAsync failed");
  return Status::Ok();
}

long long round_ld(long long n) { return (n + 63) / 64 * 64; }

LevelGeom make_level(int dim, int k, int N, const Element1D& e) {
  LevelGeom g;
  g.dim = dim; g.k = k; g.N = N; g.n1 = k * N + 1;
  g.n = 1;
  for (int a = 0; a < dim; ++a) g.n *= g.n1;
  g.ld = round_ld(g.n);
  g.h = 1.0 / N;
  const int p = k + 1;
  for (int i = 0; i <= kMaxDeg; ++i)
    for (int j = 0; j <= kMaxDeg; ++j) {
      g.me[i][j] = (i < p && j < p) ? e.Me[i * p + j] * g.h : 0.0;
      g.ke[i][j] = (i < p && j < p) ? e.Ke[i * p + j] / g.h : 0.0;
    }
  for (int r = 0; r < kMaxDeg; ++r) { g.dmr[r] = 0; g.dkr[r] = 0; }
  g.dmr[0] = g.me[0][0] + g.me[k][k];
  g.dkr[0] = g.ke[0][0] + g.ke[k][k];
  for (int r = 1; r < k; ++r) { g.dmr[r] = g.me[r][r]; g.dkr[r] = g.ke[r][r]; }
  return g;
}

namespace {
template <typename T> T from_double(double d) { return (T)d; }
template <> ff from_double<ff>(double d) {
  const float hi = (float)d;
  return ff{hi, (float)(d - (double)hi)};
}
}  // namespace

template <typename T>
OpParams<T> make_op_params(const LevelGeom& g, int nstage, const double* cm, const double* ck) {
  OpParams<T> P;
  std::memset(&P, 0, sizeof(P));
  P.N = g.N; P.n1 = g.n1; P.ld = g.ld;
  P.zc = 0;  // chosen by the launcher from the occupancy
  P.ntile_y = 1;
  const int k = g.k;
  for (int i = 0; i <= kMaxDeg; ++i)
    for (int j = 0; j <= kMaxDeg; ++j) {
      P.me[i][j] = from_double<T>(g.me[i][j]);
      P.ke[i][j] = from_double<T>(g.ke[i][j]);
    }
  // a vertex row couples to the k nodes of the cell below and above: taps -k..k
  for (int o = -k; o <= k; ++o) {
    double a = 0.0, b = 0.0;
    if (o >= 0) { a += g.me[0][o]; b += g.ke[0][o]; }
    if (o <= 0) { a += g.me[k][k + o]; b += g.ke[k][k + o]; }
    P.yvm[o + k] = from_double<T>(a);
    P.yvk[o + k] = from_double<T>(b);
  }
  for (int s = 0; s < nstage && s < kMaxStages; ++s) {
    P.cm[s] = from_double<T>(cm ? cm[s] : 0.0);
    P.ck[s] = from_double<T>(ck ? ck[s] : 0.0);
  }
  return P;
}
template OpParams<float> make_op_params<float>(const LevelGeom&, int, const double*, const double*);
template OpParams<double> make_op_params<double>(const LevelGeom&, int, const double*, const double*);
template OpParams<ff> make_op_params<ff>(const LevelGeom&, int, const double*, const double*);

template <typename T>
DiagParams<T> make_diag_params(const LevelGeom& g, int nstage, const double* cm, const double* ck, const double* c) {
  DiagParams<T> D;
  std::memset(&D, 0, sizeof(D));
  for (int s = 0; s < nstage && s < kMaxStages; ++s) {
    D.cm[s] = (T)cm[s]; D.ck[s] = (T)ck[s]; D.c[s] = (T)(c ? c[s] : 1.0);
  }
  for (int r = 0; r < kMaxDeg; ++r) { D.dmr[r] = (T)g.dmr[r]; D.dkr[r] = (T)g.dkr[r]; }
  return D;
}
template DiagParams<float> make_diag_params<float>(const LevelGeom&, int, const double*, const double*, const double*);
template DiagParams<double> make_diag_params<double>(const LevelGeom&, int, const double*, const double*,
                                                     const double*);

namespace {

// Largest eigenvalue of the symmetric tridiagonal (alpha, beta) by Sturm bisection.
double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b) {
  const int n = (int)a.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < n; ++i) {
    double r = (i > 0 ? std::fabs(b[i - 1]) : 0) + (i + 1 < n ? std::fabs(b[i]) : 0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  auto count_below = [&](double x) {
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < n; ++i) {
      double bb = (i > 0) ? b[i - 1] * b[i - 1] : 0.0;
      d = a[i] - x - (i > 0 ? bb / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d < 0) ++cnt;
    }
    return cnt;
  };
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (count_below(mid) >= n) hi = mid; else lo = mid;
    if (hi - lo <= 1e-14 * std::max(1.0, std::fabs(hi))) break;
  }
  return hi;
}

// Dense SPD inverse by Cholesky (FP64).
bool spd_inverse(int n, std::vector<double>& A) {
  std::vector<double> L(A);
  for (int j = 0; j < n; ++j) {
    double s = L[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    if (s <= 0) return false;
    const double d = std::sqrt(s);
    L[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = L[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      L[(size_t)i * n + j] = t / d;
    }
  }
  // inverse of L (lower), then A^{-1} = L^{-T} L^{-1}
  std::vector<double> Li((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    Li[(size_t)j * n + j] = 1.0 / L[(size_t)j * n + j];
    for (int i = j + 1; i < n; ++i) {
      double s = 0;
      for (int k = j; k < i; ++k) s += L[(size_t)i * n + k] * Li[(size_t)k * n + j];
      Li[(size_t)i * n + j] = -s / L[(size_t)i * n + i];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = 0;
      for (int k = i; k < n; ++k) s += Li[(size_t)k * n + i] * Li[(size_t)k * n + j];
      A[(size_t)i * n + j] = s;
      A[(size_t)j * n + i] = s;
    }
  return true;
}

// Symmetric eigen-decomposition A = W diag(w) W^T by cyclic Jacobi rotations (A destroyed).
void jacobi_eigen(int n, std::vector<double>& A, std::vector<double>& W, std::vector<double>& w) {
  W.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) W[(size_t)i * n + i] = 1.0;
  auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
  double norm = 0.0;
  for (double x : A) norm += x * x;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += a(i, j) * a(i, j);
    if (off <= 1e-32 * norm) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a(p, q);
        if (std::fabs(apq) < 1e-300) continue;
        const double theta = (a(q, q) - a(p, p)) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = a(k, p), akq = a(k, q);
          a(k, p) = c * akp - sn * akq;
          a(k, q) = sn * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = a(p, k), aqk = a(q, k);
          a(p, k) = c * apk - sn * aqk;
          a(q, k) = sn * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double wkp = W[(size_t)k * n + p], wkq = W[(size_t)k * n + q];
          W[(size_t)k * n + p] = c * wkp - sn * wkq;
          W[(size_t)k * n + q] = sn * wkp + c * wkq;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = a(i, i);
}

template <typename T>
class MG final : public MGBase {
 public:
  struct Lvl {
    LevelGeom g;
    T *b = nullptr, *xa = nullptr, *xb = nullptr, *r = nullptr, *t1 = nullptr, *t2 = nullptr;
    T *mx = nullptr, *kx = nullptr;  // coupled mode: M x and K x of both components
    long long ld1 = 0, ld2 = 0;   // strides of t1, t2
    T* cur = nullptr;             // buffer holding the level's current iterate
    std::vector<double> lo, hi;   // Chebyshev interval per block
    std::vector<std::vector<double>> c1, c2;  // [step][block]
  };

  MG(const MGConfig& c, const Element1D& e, DeviceArena& a) : cfg_(c), el_(e), arena_(a) {}

  // level-operator parameters with the launch-shape key of one request's blocks
  template <typename U>
  OpParams<U> opp(const LevelGeom& g, int nstage, const double* cm, const double* ck) const {
    OpParams<U> P = make_op_params<U>(g, nstage, cm, ck);
    P.shape_ns = (cfg_.shape_ns > 0 && nstage == cfg_.nb) ? cfg_.shape_ns : 0;
    return P;
  }

  // Coupled mode: the two blocks are the components of [[A, -beta M], [beta M, A]] (a 2x2 block of
  // the real form of Eq. irk:Ainv, Sec. 6) and one V-cycle acts on the coupled system.
  bool coupled() const { return cfg_.coupled_beta != 0.0; }

  Status setup(cudaStream_t st) {
    st_ = st;
    if (coupled() && (cfg_.nb != 2 || !cfg_.batched || cfg_.cm.size() != 2 || cfg_.cm[0] != cfg_.cm[1]))
      return Status::Err(IRK_EINVAL, "coupled multigrid needs two batched components with one mass coefficient");
    // level sizes: N, N/2, ... while even and the coarse mesh keeps an interior node
    std::vector<int> sizes{cfg_.N};
    const int nmin = (cfg_.k == 1) ? 2 : 1;
    while (sizes.back() % 2 == 0 && sizes.back() / 2 >= nmin) sizes.push_back(sizes.back() / 2);
    const int nb = cfg_.nb;
    if (!cfg_.taus.empty() && (int)cfg_.taus.size() != nb) return Status::Err(IRK_EINVAL, "one tau per block");
    ck_.assign(nb, cfg_.tau);
    if (!cfg_.taus.empty()) ck_ = cfg_.taus;
    for (size_t l = 0; l < sizes.size(); ++l) {
      Lvl L;
      L.g = make_level(cfg_.dim, cfg_.k, sizes[l], el_);
      const size_t vb = (size_t)nb * L.g.ld * sizeof(T);
      IRK_TRY(arena_.alloc((void**)&L.b, vb));
      IRK_TRY(arena_.alloc((void**)&L.xa, vb));
      IRK_TRY(arena_.alloc((void**)&L.xb, vb));
      IRK_TRY(arena_.alloc((void**)&L.r, vb));
      if (coupled()) {
        IRK_TRY(arena_.alloc((void**)&L.mx, vb));
        IRK_TRY(arena_.alloc((void**)&L.kx, vb));
      }
      L.cur = L.xa;
      if (l + 1 < sizes.size()) {
        const long long nf = L.g.n1, nc = (long long)cfg_.k * sizes[l + 1] + 1;
        long long s1 = (cfg_.dim == 3) ? nc * nf * nf : nc * nf;
        long long s2 = (cfg_.dim == 3) ? nc * nc * nf : nc * nc;
        L.ld1 = round_ld(s1);
        L.ld2 = round_ld(s2);
        IRK_TRY(arena_.alloc((void**)&L.t1, (size_t)nb * L.ld1 * sizeof(T)));
        IRK_TRY(arena_.alloc((void**)&L.t2, (size_t)nb * L.ld2 * sizeof(T)));
      }
      lv_.push_back(std::move(L));
    }
    IRK_TRY(setup_coarse());
    IRK_TRY(setup_chebyshev(st));
    IRK_TRY(setup_fused());
    if (cfg_.autotune) IRK_TRY(autotune(st));
    IRK_CUDA(cudaStreamSynchronize(st));
    return Status::Ok();
  }

  // Launch shapes of the level operators (Chebyshev step and residual, batched blocks), timed on
  // the levels' own buffers before they hold data (process-wide cache; see tune_op).
  Status autotune(cudaStream_t st) {
    if (!cfg_.batched || coupled()) return Status::Ok();
    const int nb = cfg_.nb;
    const int last = fused_ ? lc_ : levels() - 1;
    for (int l = 0; l < last; ++l) {
      Lvl& L = lv_[l];
      OpParams<T> P = opp<T>(L.g, nb, cfg_.cm.data(), ck_.data());
      EpiParams<T> E;
      std::memset(&E, 0, sizeof(E));
      E.out = L.xb;
      E.b = L.b;
      E.xj = L.xa;
      for (int s = 0; s < nb; ++s) { E.c1[s] = (T)L.c1[cfg_.cheb_degree > 1 ? 1 : 0][s]; E.c2[s] = (T)L.c2[0][s]; }
      for (int r = 0; r < kMaxDeg; ++r) { E.dmr[r] = (T)L.g.dmr[r]; E.dkr[r] = (T)L.g.dkr[r]; }
      IRK_CUDA(tune_op<T>(cfg_.dim, cfg_.k, nb, L.xa, P, EPI_CHEB, E, st));
      IRK_CUDA(tune_op<T>(cfg_.dim, cfg_.k, nb, L.xa, P, EPI_RESID, E, st));
    }
    // the buffers used as scratch above start from zero again
    for (int l = 0; l < last; ++l) {
      const size_t vb = (size_t)nb * lv_[l].g.ld * sizeof(T);
      IRK_CUDA(cudaMemsetAsync(lv_[l].xb, 0, vb, st));
    }
    return Status::Ok();
  }

  int levels() const override { return (int)lv_.size(); }
  int elem_size() const override { return sizeof(T); }
  void* fine_b() override { return lv_[0].b; }
  void* fine_x() override { return lv_[0].cur; }
  const LevelGeom& geom(int l) const override { return lv_[l].g; }
  void interval(int l, int b, double* lo, double* hi) const override { *lo = lv_[l].lo[b]; *hi = lv_[l].hi[b]; }

  Status vcycle(int l, cudaStream_t st) override {
    Lvl& L = lv_[l];
    if (fused_ && l == lc_) {  // the whole sub-cycle below in one launch
      fparams_.b_in = L.b;
      fparams_.x_out = L.xa;
      IRK_LAUNCH(PROF_COARSE, launch_coarse_cycle<float>(fparams_, cfg_.dim, cfg_.k, st));
      L.cur = L.xa;
      return Status::Ok();
    }
    if (l == levels() - 1) {
      IRK_TRY(coarse_solve(L.b, L.xa, st));
      L.cur = L.xa;
      return Status::Ok();
    }
    IRK_TRY(cheb(l, L.b, /*from_zero=*/true, st));
    IRK_TRY(residual(l, L.b, L.cur, L.r, st));
    IRK_TRY(restrict_to(l, L.r, lv_[l + 1].b, st));
    IRK_TRY(vcycle(l + 1, st));
    IRK_TRY(prolongate_add(l, lv_[l + 1].cur, L.cur, st));
    IRK_TRY(cheb(l, L.b, /*from_zero=*/false, st));
    return Status::Ok();
  }

  Status retau(const std::vector<double>& taus, cudaStream_t st) override {
    if ((int)taus.size() != cfg_.nb) return Status::Err(IRK_EINVAL, "one tau per block");
    for (double t : taus)
      if (!(t > 0) || !std::isfinite(t)) return Status::Err(IRK_EINVAL, "tau must be positive");
    if (coupled()) return Status::Err(IRK_EINVAL, "the coupled hierarchy keeps its tau");
    st_ = st;
    ck_ = taus;
    cfg_.taus = taus;
    if (use_fd_) {
      for (int s = 0; s < cfg_.nb && s < kMaxStages; ++s) fd_params_.taus[s] = ck_[s];
    } else {
      IRK_TRY(setup_coarse());
    }
    IRK_TRY(setup_chebyshev(st));
    IRK_TRY(setup_fused());
    if (gexec_) cudaGraphExecDestroy(gexec_);
    if (graph_) cudaGraphDestroy(graph_);
    gexec_ = nullptr;
    graph_ = nullptr;
    IRK_CUDA(cudaStreamSynchronize(st));
    return Status::Ok();
  }

  ~MG() override {
    if (gexec_) cudaGraphExecDestroy(gexec_);
    if (graph_) cudaGraphDestroy(graph_);
  }

  Status vcycle_top(cudaStream_t st, bool allow_graph) override {
    const unsigned mg_mask = (1u << PROF_MG_OP) | (1u << PROF_MG_OP_FINE) | (1u << PROF_MG_POINT) |
                             (1u << PROF_TRANSFER) | (1u << PROF_COARSE);
    const bool timing = g_prof && (g_prof->mask & mg_mask);
    if (!allow_graph || st == nullptr || timing || eager_runs_ < 1) {
      ++eager_runs_;
      return vcycle(0, st);
    }
    if (!gexec_) {
      Profiler counter;  // counts the captured launches per category
      counter.st = st;
      ProfBind bind(&counter);
      IRK_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
      Status s = vcycle(0, st);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(st, &g);
      if (!s.ok()) {
        if (g) cudaGraphDestroy(g);
        return s;
      }
      IRK_CUDA(e);
      graph_ = g;
      IRK_CUDA(cudaGraphInstantiate(&gexec_, graph_, 0));
      for (int c = 0; c < PROF_NCAT; ++c) gcounts_[c] = counter.launches[c];
    }
    IRK_CUDA(cudaGraphLaunch(gexec_, st));
    if (g_prof)
      for (int c = 0; c < PROF_NCAT; ++c) g_prof->launches[c] += gcounts_[c];
    return Status::Ok();
  }

  Status vcycle_io(int l, const void* b, void* x, cudaStream_t st) override {
    Lvl& L = lv_[l];
    const size_t bytes = (size_t)cfg_.nb * L.g.ld * sizeof(T);
    IRK_CUDA(cudaMemcpyAsync(L.b, b, bytes, cudaMemcpyDeviceToDevice, st));
    IRK_TRY(vcycle(l, st));
    IRK_CUDA(cudaMemcpyAsync(x, L.cur, bytes, cudaMemcpyDeviceToDevice, st));
    return Status::Ok();
  }

  Status smooth(int l, const void* b, void* x, int x_is_zero, cudaStream_t st) override {
    Lvl& L = lv_[l];
    const size_t bytes = (size_t)cfg_.nb * L.g.ld * sizeof(T);
    if (!x_is_zero) IRK_CUDA(cudaMemcpyAsync(L.xa, x, bytes, cudaMemcpyDeviceToDevice, st));
    L.cur = L.xa;
    IRK_TRY(cheb(l, (const T*)b, x_is_zero != 0, st));
    IRK_CUDA(cudaMemcpyAsync(x, L.cur, bytes, cudaMemcpyDeviceToDevice, st));
    return Status::Ok();
  }

  // coupled level operator: M x and K x of both components in one launch, then the pointwise
  // coupling fused with the residual (cheb = 0) or the Chebyshev step (cheb = 1, step j; cheb = 2,
  // the first step from zero, needs no operator)
  Status coupled_apply(int l, const T* x, const T* b, T* out, int cheb, int j, bool xold_zero, cudaStream_t st) {
    Lvl& L = lv_[l];
    EpiParams<T> E;
    std::memset(&E, 0, sizeof(E));
    E.out = L.mx;
    E.out2 = L.kx;
    OpParams<T> P = opp<T>(L.g, 2, cfg_.cm.data(), ck_.data());
    if (cheb != 2)
      IRK_LAUNCH(l == 0 ? PROF_MG_OP_FINE : PROF_MG_OP, launch_op<T>(cfg_.dim, cfg_.k, 2, x, P, EPI_DUAL, E, st));
    CoupledParams C;
    std::memset(&C, 0, sizeof(C));
    C.cm = cfg_.cm[0];
    C.ck = ck_[0];
    C.beta = cfg_.coupled_beta;
    C.cheb = cheb;
    C.xold_zero = xold_zero ? 1 : 0;
    if (cheb) { C.c1 = L.c1[j][0]; C.c2 = L.c2[j][0]; }
    for (int r = 0; r < kMaxDeg; ++r) { C.dmr[r] = L.g.dmr[r]; C.dkr[r] = L.g.dkr[r]; }
    IRK_LAUNCH(PROF_MG_POINT, launch_coupled_update<T>(L.g.grid(), L.mx, L.kx, x, b, out, C, st));
    return Status::Ok();
  }

  Status residual(int l, const void* b, const void* x, void* r, cudaStream_t st) override {
    if (coupled()) return coupled_apply(l, (const T*)x, (const T*)b, (T*)r, 0, 0, false, st);
    Lvl& L = lv_[l];
    EpiParams<T> E;
    std::memset(&E, 0, sizeof(E));
    E.out = (T*)r;
    E.b = (const T*)b;
    return op(l, (const T*)x, EPI_RESID, E, st);
  }

  Status restrict_to(int l, const void* rin, void* bc, cudaStream_t st) override {
    Lvl& L = lv_[l];
    const Lvl& C = lv_[l + 1];
    TransferParams P = transfer_params(C.g.N);
    const int nf = L.g.n1, nc = C.g.n1;
    if (cfg_.dim == 3) {
      int d0[3] = {nf, nf, nf}, d1[3] = {nc, nf, nf}, d2[3] = {nc, nc, nf}, d3[3] = {nc, nc, nc};
      IRK_LAUNCH(PROF_TRANSFER, launch_transfer_axis<T>((const T*)rin, L.t1, cfg_.nb, L.g.ld, L.ld1, d0, d1, 0, 1, 0, P, st));
      IRK_LAUNCH(PROF_TRANSFER, launch_transfer_axis<T>(L.t1, L.t2, cfg_.nb, L.ld1, L.ld2, d1, d2, 1, 1, 0, P, st));
      IRK_LAUNCH(PROF_TRANSFER, launch_transfer_axis<T>(L.t2, (T*)bc, cfg_.nb, L.ld2, C.g.ld, d2, d3, 2, 1, 0, P, st));
    } else {
      int d0[3] = {nf, nf, 1}, d1[3] = {nc, nf, 1}, d2[3] = {nc, nc, 1};
      IRK_LAUNCH(PROF_TRANSFER, launch_transfer_axis<T>((const T*)rin, L.t1, cfg_.nb, L.g.ld, L.ld1, d0, d1, 0, 1, 0, P, st));
      IRK_LAUNCH(PROF_TRANSFER, launch_transfer_axis<T>(L.t1, (T*)bc, cfg_.nb, L.ld1, C.g.ld, d1, d2, 1, 1, 0, P, st));
    }
    return Status::Ok();
  }

  Status restrict_in_scratch(int l, const void* rin, void* bc, void* scratch, size_t bytes,
                             cudaStream_t st) override {
    Lvl& L = lv_[l];
    const Lvl& C = lv_[l + 1];
    const size_t need = (size_t)cfg_.nb * (size_t)(L.ld1 + L.ld2) * sizeof(T);
    if (need > bytes)
      return Status::Err(IRK_EINVAL, "restriction of level " + std::to_string(l) + " needs " + std::to_string(need) +
                                         " bytes of scratch, more than the " + std::to_string(bytes) + " available");
    // the passes leave the coarse-boundary entries of their outputs unwritten: start from zero
    IRK_CUDA(cudaMemsetAsync(scratch, 0, need, st));
    T* t1 = static_cast<T*>(scratch);
    T* t2 = t1 + (size_t)cfg_.nb * L.ld1;
    TransferParams P = transfer_params(C.g.N);
    const int nf = L.g.n1, nc = C.g.n1;
    if (cfg_.dim == 3) {
      int d0[3] = {nf, nf, nf}, d1[3] = {nc, nf, nf}, d2[3] = {nc, nc, nf}, d3[3] = {nc, nc, nc};
      IRK_LAUNCH(PROF_TRANSFER, launch_transfer_axis<T>((const T*)rin, t1, cfg_.nb, L.g.ld, L.ld1, d0, d1, 0, 1, 0, P, st));
      IRK_LAUNCH(PROF_TRANSFER, launch_transfer_axis<T>(t1, t2, cfg_.nb, L.ld1, L.ld2, d1, d2, 1, 1, 0, P, st));
      IRK_LAUNCH(PROF_TRANSFER, launch_transfer_axis<T>(t2, (T*)bc, cfg_.nb, L.ld2, C.g.ld, d2, d3, 2, 1, 0, P, st));
    } else {
      int d0[3] = {nf, nf, 1}, d1[3] = {nc, nf, 1}, d2[3] = {nc, nc, 1};
      IRK_LAUNCH(PROF_TRANSFER, launch_transfer_axis<T>((const T*)rin, t1, cfg_.nb, L.g.ld, L.ld1, d0, d1, 0, 1, 0, P, st));
      IRK_LAUNCH(PROF_TRANSFER, launch_transfer_axis<T>(t1, (T*)bc, cfg_.nb, L.ld1, C.g.ld, d1, d2, 1, 1, 0, P, st));
    }
    return Status::Ok();
  }

  Status prolongate_add(int l, const void* ec, void* x, cudaStream_t st) override {
    Lvl& L = lv_[l];
    const Lvl& C = lv_[l + 1];
    TransferParams P = transfer_params(C.g.N);
    const int nf = L.g.n1, nc = C.g.n1;
    if (cfg_.dim == 3) {
      int d3[3] = {nc, nc, nc}, d2[3] = {nc, nc, nf}, d1[3] = {nc, nf, nf}, d0[3] = {nf, nf, nf};
      IRK_LAUNCH(PROF_TRANSFER, launch_transfer_axis<T>((const T*)ec, L.t2, cfg_.nb, C.g.ld, L.ld2, d3, d2, 2, 0, 0, P, st));
      IRK_LAUNCH(PROF_TRANSFER, launch_transfer_axis<T>(L.t2, L.t1, cfg_.nb, L.ld2, L.ld1, d2, d1, 1, 0, 0, P, st));
      IRK_LAUNCH(PROF_TRANSFER, launch_transfer_axis<T>(L.t1, (T*)x, cfg_.nb, L.ld1, L.g.ld, d1, d0, 0, 0, 1, P, st));
    } else {
      int d2[3] = {nc, nc, 1}, d1[3] = {nc, nf, 1}, d0[3] = {nf, nf, 1};
      IRK_LAUNCH(PROF_TRANSFER, launch_transfer_axis<T>((const T*)ec, L.t1, cfg_.nb, C.g.ld, L.ld1, d2, d1, 1, 0, 0, P, st));
      IRK_LAUNCH(PROF_TRANSFER, launch_transfer_axis<T>(L.t1, (T*)x, cfg_.nb, L.ld1, L.g.ld, d1, d0, 0, 0, 1, P, st));
    }
    return Status::Ok();
  }

  Status coarse_solve(const void* b, void* x, cudaStream_t st) override {
    const LevelGeom& g = lv_.back().g;
    if (!use_fd_) {
      IRK_LAUNCH(PROF_COARSE, launch_coarse_solve<T>((const T*)b, (T*)x, cfg_.nb, g.ld, dAinv_, dmap_, nci_, st));
      return Status::Ok();
    }
    // W^T along every axis, diagonal scaling, W along every axis
    const int nb = cfg_.nb, n1 = g.n1, dim = g.dim, ni = n1 - 2;
    double* t[2] = {fd_t1_, fd_t2_};
    int cur = 0;
    IRK_LAUNCH(PROF_COARSE, launch_fd_axis<T, double>((const T*)b, t[0], nb, g.ld, n1, dim, 0, fd_Vt_, ni, st));
    for (int a = 1; a < dim; ++a) {
      IRK_LAUNCH(PROF_COARSE, launch_fd_axis<double, double>(t[cur], t[1 - cur], nb, g.ld, n1, dim, a, fd_Vt_, ni, st));
      cur = 1 - cur;
    }
    if (coupled())
      IRK_LAUNCH(PROF_COARSE, launch_fd_scale_coupled(t[cur], g.ld, n1, dim, fd_mu_, fd_params_, st));
    else
      IRK_LAUNCH(PROF_COARSE, launch_fd_scale(t[cur], nb, g.ld, n1, dim, fd_mu_, fd_params_, st));
    for (int a = 0; a + 1 < dim; ++a) {
      IRK_LAUNCH(PROF_COARSE, launch_fd_axis<double, double>(t[cur], t[1 - cur], nb, g.ld, n1, dim, a, fd_V_, ni, st));
      cur = 1 - cur;
    }
    IRK_LAUNCH(PROF_COARSE, launch_fd_axis<double, T>(t[cur], (T*)x, nb, g.ld, n1, dim, dim - 1, fd_V_, ni, st));
    return Status::Ok();
  }

  Status apply_mass(int l, const void* x, void* y, double scale, cudaStream_t st) override {
    std::vector<double> cm(cfg_.nb, scale), ck(cfg_.nb, 0.0);
    EpiParams<T> E;
    std::memset(&E, 0, sizeof(E));
    E.out = (T*)y;
    OpParams<T> P = opp<T>(lv_[l].g, cfg_.nb, cm.data(), ck.data());
    IRK_LAUNCH(PROF_MG_OP, launch_op<T>(cfg_.dim, cfg_.k, cfg_.nb, (const T*)x, P, EPI_STORE, E, st));
    return Status::Ok();
  }

 private:
  TransferParams transfer_params(int Nc) const {
    TransferParams P;
    std::memset(&P, 0, sizeof(P));
    P.k = cfg_.k;
    P.Nc = Nc;
    for (size_t i = 0; i < el_.Pc.size(); ++i) {
      P.Pc[i] = el_.Pc[i];
      P.Pcf[i] = (float)el_.Pc[i];
    }
    return P;
  }

  // operator launch over all blocks (batched) or block by block
  Status op(int l, const T* u, int epi, const EpiParams<T>& E, cudaStream_t st) {
    Lvl& L = lv_[l];
    const int nb = cfg_.nb;
    if (cfg_.batched) {
      OpParams<T> P = opp<T>(L.g, nb, cfg_.cm.data(), ck_.data());
      IRK_LAUNCH(l == 0 ? PROF_MG_OP_FINE : PROF_MG_OP, launch_op<T>(cfg_.dim, cfg_.k, nb, u, P, epi, E, st));
      return Status::Ok();
    }
    for (int s = 0; s < nb; ++s) {
      OpParams<T> P = opp<T>(L.g, 1, &cfg_.cm[s], &ck_[s]);
      EpiParams<T> Es = E;
      const long long off = (long long)s * L.g.ld;
      Es.out = E.out ? E.out + off : nullptr;
      Es.out2 = E.out2 ? E.out2 + off : nullptr;
      Es.b = E.b ? E.b + off : nullptr;
      Es.xj = E.xj ? E.xj + off : nullptr;
      Es.c1[0] = E.c1[s];
      Es.c2[0] = E.c2[s];
      IRK_LAUNCH(l == 0 ? PROF_MG_OP_FINE : PROF_MG_OP, launch_op<T>(cfg_.dim, cfg_.k, 1, u + off, P, epi, Es, st));
    }
    return Status::Ok();
  }

  // degree-m Chebyshev iteration on level l; result in L.cur
  Status cheb(int l, const T* b, bool from_zero, cudaStream_t st) {
    Lvl& L = lv_[l];
    const int nb = cfg_.nb, m = cfg_.cheb_degree;
    T* cur = from_zero ? L.xa : L.cur;
    T* oth = (cur == L.xa) ? L.xb : L.xa;
    int j0 = 0;
    if (from_zero) {
      if (coupled()) {
        IRK_TRY(coupled_apply(l, nullptr, b, cur, 2, 0, true, st));
      } else {
        std::vector<double> c(nb);
        for (int s = 0; s < nb; ++s) c[s] = L.c2[0][s];
        DiagParams<T> D = make_diag_params<T>(L.g, nb, cfg_.cm.data(), ck_.data(), c.data());
        IRK_LAUNCH(PROF_MG_POINT, launch_cheb_first<T>(L.g.grid(), nb, b, cur, D, st));
      }
      j0 = 1;
    }
    for (int j = j0; j < m; ++j) {
      EpiParams<T> E;
      std::memset(&E, 0, sizeof(E));
      E.out = oth;
      E.b = b;
      E.xj = cur;
      for (int s = 0; s < nb; ++s) { E.c1[s] = (T)L.c1[j][s]; E.c2[s] = (T)L.c2[j][s]; }
      for (int r = 0; r < kMaxDeg; ++r) { E.dmr[r] = (T)L.g.dmr[r]; E.dkr[r] = (T)L.g.dkr[r]; }
      // x_{j-1} is zero only for the second step of a smoothing that started from zero
      E.xold_zero = (from_zero && j == 1) || j == 0;
      if (coupled()) IRK_TRY(coupled_apply(l, cur, b, oth, 1, j, E.xold_zero != 0, st));
      else IRK_TRY(op(l, cur, EPI_CHEB, E, st));
      std::swap(cur, oth);
    }
    L.cur = cur;
    return Status::Ok();
  }

  Status setup_coarse() {
    const Lvl& C = lv_.back();
    const int dim = cfg_.dim, n1 = C.g.n1, ni = n1 - 2;
    nci_ = 1;
    for (int a = 0; a < dim; ++a) nci_ *= ni;
    if (nci_ < 1) return Status::Err(IRK_EINVAL, "coarsest mesh has no interior node");
    use_fd_ = nci_ > kDenseCoarseMax || coupled();  // the coupled system is solved mode by mode
    // 1D assembled interior matrices on the coarsest mesh
    const int k = cfg_.k, p = k + 1;
    std::vector<double> M1((size_t)n1 * n1, 0.0), K1((size_t)n1 * n1, 0.0);
    for (int c = 0; c < C.g.N; ++c)
      for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j) {
          M1[(size_t)(k * c + i) * n1 + k * c + j] += C.g.me[i][j];
          K1[(size_t)(k * c + i) * n1 + k * c + j] += C.g.ke[i][j];
        }
    if (use_fd_) return setup_coarse_fd(M1, K1);
    std::vector<int> map(nci_);
    for (int q = 0; q < nci_; ++q) {
      int t = q, node = 0, stride = 1;
      for (int a = 0; a < dim; ++a) {
        const int ia = t % ni + 1;
        t /= ni;
        node += ia * stride;
        stride *= n1;
      }
      map[q] = node;
    }
    std::vector<double> Ainv_all((size_t)cfg_.nb * nci_ * nci_);
    for (int s = 0; s < cfg_.nb; ++s) {
      std::vector<double> A((size_t)nci_ * nci_);
      for (int q = 0; q < nci_; ++q)
        for (int r = 0; r < nci_; ++r) {
          int tq = q, tr = r;
          double mprod = 1.0;
          double mv[3], kv[3];
          for (int a = 0; a < dim; ++a) {
            const int iq = tq % ni + 1, ir = tr % ni + 1;
            tq /= ni; tr /= ni;
            mv[a] = M1[(size_t)iq * n1 + ir];
            kv[a] = K1[(size_t)iq * n1 + ir];
            mprod *= mv[a];
          }
          double kterm = 0.0;
          for (int a = 0; a < dim; ++a) {
            double t = kv[a];
            for (int b = 0; b < dim; ++b) if (b != a) t *= mv[b];
            kterm += t;
          }
          A[(size_t)q * nci_ + r] = cfg_.cm[s] * mprod + ck_[s] * kterm;
        }
      if (!spd_inverse(nci_, A)) return Status::Err(IRK_ENUMERIC, "coarse operator not SPD");
      std::copy(A.begin(), A.end(), Ainv_all.begin() + (size_t)s * nci_ * nci_);
    }
    ainv_host_ = Ainv_all;
    if (!dAinv_) IRK_TRY(arena_.alloc((void**)&dAinv_, Ainv_all.size() * sizeof(double)));
    if (!dmap_) IRK_TRY(arena_.alloc((void**)&dmap_, map.size() * sizeof(int)));
    IRK_CUDA(cudaMemcpyAsync(dAinv_, Ainv_all.data(), Ainv_all.size() * sizeof(double), cudaMemcpyHostToDevice, st_));
    IRK_CUDA(cudaMemcpyAsync(dmap_, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice, st_));
    return Status::Ok();
  }

  // Fused coarse cycle: the lowest levels with at most kFusedMaxNodes3D (2D) nodes per block run in
  // one launch (FP32 multigrid, batched blocks, dense coarsest solve, at least two fused levels).
  Status setup_fused() {
    fused_ = false;
    if (sizeof(T) != 4 || !cfg_.batched || use_fd_ || coupled() || cfg_.cheb_degree > kMaxChebDegree ||
        cfg_.nb > kMaxStages)
      return Status::Ok();
    int lc = levels() - 1;
    const long long maxn = (cfg_.dim == 3) ? kFusedMaxNodes3D : kFusedMaxNodes2D;
    // the lowest levels that fit, at most kMaxFusedLevels of them (a hierarchy with more small levels
    // fuses its lowest ones and runs the others level by level)
    while (lc > 0 && lv_[lc - 1].g.n <= maxn && levels() - (lc - 1) <= kMaxFusedLevels) --lc;
    const int nlev = levels() - lc;
    if (nlev < 2 || nlev > kMaxFusedLevels) return Status::Ok();
    CoarseParams& P = fparams_;
    std::memset(&P, 0, sizeof(P));
    P.nlev = nlev;
    P.nb = cfg_.nb;
    P.m = cfg_.cheb_degree;
    P.nci = nci_;
    for (int s = 0; s < cfg_.nb; ++s) {
      P.cm[s] = (float)cfg_.cm[s];
      P.taus[s] = (float)ck_[s];
    }
    for (int i = 0; i < nlev; ++i) {
      const Lvl& L = lv_[lc + i];
      CoarseLevel& C = P.lv[i];
      C.N = L.g.N;
      C.n1 = L.g.n1;
      C.n = (int)L.g.n;
      C.magic = coarse_cycle_magic(C.n1);
      for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b) { C.me[a][b] = (float)L.g.me[a][b]; C.ke[a][b] = (float)L.g.ke[a][b]; }
      for (int r = 0; r < kMaxDeg; ++r) { C.dmr[r] = (float)L.g.dmr[r]; C.dkr[r] = (float)L.g.dkr[r]; }
      if (lc + i + 1 < levels())
        for (int j = 0; j < cfg_.cheb_degree; ++j)
          for (int s = 0; s < cfg_.nb; ++s) { C.c1[j][s] = (float)L.c1[j][s]; C.c2[j][s] = (float)L.c2[j][s]; }
    }
    for (size_t i = 0; i < el_.Pc.size(); ++i) P.pc[i] = (float)el_.Pc[i];
    if (coarse_cycle_smem(P, sizeof(float)) > kCoarseCycleMaxSmem) return Status::Ok();
    P.ainv = dAinv_;  // the FP64 inverses of setup_coarse
    P.map = dmap_;
    P.ld = lv_[lc].g.ld;
    lc_ = lc;
    fused_ = true;
    return Status::Ok();
  }

  // Generalised 1D eigenproblem on the interior nodes: K1 v = mu M1 v, V^T M1 V = I.
  Status setup_coarse_fd(const std::vector<double>& M1, const std::vector<double>& K1) {
    const LevelGeom& g = lv_.back().g;
    const int n1 = g.n1, ni = n1 - 2;
    std::vector<double> Mi((size_t)ni * ni), Ki((size_t)ni * ni);
    for (int i = 0; i < ni; ++i)
      for (int j = 0; j < ni; ++j) {
        Mi[(size_t)i * ni + j] = M1[(size_t)(i + 1) * n1 + j + 1];
        Ki[(size_t)i * ni + j] = K1[(size_t)(i + 1) * n1 + j + 1];
      }
    // Cholesky Mi = L L^T
    std::vector<double> L((size_t)ni * ni, 0.0);
    for (int j = 0; j < ni; ++j) {
      double d = Mi[(size_t)j * ni + j];
      for (int k = 0; k < j; ++k) d -= L[(size_t)j * ni + k] * L[(size_t)j * ni + k];
      if (d <= 0) return Status::Err(IRK_ENUMERIC, "1D mass matrix not SPD");
      d = std::sqrt(d);
      L[(size_t)j * ni + j] = d;
      for (int i = j + 1; i < ni; ++i) {
        double t = Mi[(size_t)i * ni + j];
        for (int k = 0; k < j; ++k) t -= L[(size_t)i * ni + k] * L[(size_t)j * ni + k];
        L[(size_t)i * ni + j] = t / d;
      }
    }
    // C = L^{-1} Ki L^{-T}: solve column by column
    auto fwd = [&](std::vector<double>& x) {  // x <- L^{-1} x
      for (int i = 0; i < ni; ++i) {
        double t = x[i];
        for (int k = 0; k < i; ++k) t -= L[(size_t)i * ni + k] * x[k];
        x[i] = t / L[(size_t)i * ni + i];
      }
    };
    std::vector<double> Y((size_t)ni * ni), C((size_t)ni * ni), col(ni);
    for (int j = 0; j < ni; ++j) {  // Y = L^{-1} Ki
      for (int i = 0; i < ni; ++i) col[i] = Ki[(size_t)i * ni + j];
      fwd(col);
      for (int i = 0; i < ni; ++i) Y[(size_t)i * ni + j] = col[i];
    }
    for (int i = 0; i < ni; ++i) {  // C = Y L^{-T} = (L^{-1} Y^T)^T
      for (int j = 0; j < ni; ++j) col[j] = Y[(size_t)i * ni + j];
      fwd(col);
      for (int j = 0; j < ni; ++j) C[(size_t)i * ni + j] = col[j];
    }
    for (int i = 0; i < ni; ++i)
      for (int j = i + 1; j < ni; ++j) {
        const double a = 0.5 * (C[(size_t)i * ni + j] + C[(size_t)j * ni + i]);
        C[(size_t)i * ni + j] = C[(size_t)j * ni + i] = a;
      }
    std::vector<double> W, mu;
    jacobi_eigen(ni, C, W, mu);
    // V = L^{-T} W (back substitution per column)
    std::vector<double> V((size_t)ni * ni), Vt((size_t)ni * ni);
    for (int j = 0; j < ni; ++j) {
      for (int i = ni - 1; i >= 0; --i) {
        double t = W[(size_t)i * ni + j];
        for (int k = i + 1; k < ni; ++k) t -= L[(size_t)k * ni + i] * V[(size_t)k * ni + j];
        V[(size_t)i * ni + j] = t / L[(size_t)i * ni + i];
      }
    }
    for (int i = 0; i < ni; ++i)
      for (int j = 0; j < ni; ++j) Vt[(size_t)i * ni + j] = V[(size_t)j * ni + i];
    IRK_TRY(arena_.alloc((void**)&fd_V_, V.size() * sizeof(double)));
    IRK_TRY(arena_.alloc((void**)&fd_Vt_, Vt.size() * sizeof(double)));
    IRK_TRY(arena_.alloc((void**)&fd_mu_, mu.size() * sizeof(double)));
    const size_t vb = (size_t)cfg_.nb * g.ld * sizeof(double);
    IRK_TRY(arena_.alloc((void**)&fd_t1_, vb));
    IRK_TRY(arena_.alloc((void**)&fd_t2_, vb));
    IRK_CUDA(cudaMemcpyAsync(fd_V_, V.data(), V.size() * sizeof(double), cudaMemcpyHostToDevice, st_));
    IRK_CUDA(cudaMemcpyAsync(fd_Vt_, Vt.data(), Vt.size() * sizeof(double), cudaMemcpyHostToDevice, st_));
    IRK_CUDA(cudaMemcpyAsync(fd_mu_, mu.data(), mu.size() * sizeof(double), cudaMemcpyHostToDevice, st_));
    std::memset(&fd_params_, 0, sizeof(fd_params_));
    fd_params_.ni = ni;
    for (int s = 0; s < cfg_.nb && s < kMaxStages; ++s) {
      fd_params_.cm[s] = cfg_.cm[s];
      fd_params_.taus[s] = ck_[s];
    }
    fd_params_.beta = cfg_.coupled_beta;
    return Status::Ok();
  }

  // Lanczos on D^{-1/2} A D^{-1/2} (FP64) per level and block -> Chebyshev intervals.
  Status setup_chebyshev(cudaStream_t st) {
    const int nb = cfg_.nb;
    const LevelGeom& g0 = lv_[0].g;
    const size_t len = (size_t)nb * g0.ld;
    const int steps = std::max(2, cfg_.eig_steps);
    DeviceArena tmp(st);  // Lanczos work vectors, released when the setup returns
    // the operator of the estimate in the smoother's own arithmetic for an FP32 hierarchy (it needs
    // a few digits of lambda_max, and the FP32 level kernels are several times faster than the
    // float-float ones on the large fine levels), float-float for an FP64 hierarchy (FP32 pipe);
    // Lanczos vectors and reductions in FP64, the diagonal scalings convert between the two
    using LT = typename std::conditional<sizeof(T) == 4, float, ff>::type;
    double *v0, *v1, *w, *partial, *ab;
    LT *t, *wf;
    IRK_TRY(tmp.alloc((void**)&v0, len * sizeof(double)));
    IRK_TRY(tmp.alloc((void**)&v1, len * sizeof(double)));
    IRK_TRY(tmp.alloc((void**)&w, len * sizeof(double)));
    IRK_TRY(tmp.alloc((void**)&t, len * sizeof(LT)));
    IRK_TRY(tmp.alloc((void**)&wf, len * sizeof(LT)));
    const int nbred = std::min(reduction_blocks((long long)g0.ld), 1024);
    IRK_TRY(tmp.alloc((void**)&partial, (size_t)nbred * nb * sizeof(double)));
    // per level: alpha[step][block], beta[step][block], norm[block], zeros[block]; every level's
    // recurrence is enqueued back to back and read back once
    const int nlev = levels() - 1;
    const size_t per_level = (size_t)(2 * steps + 2) * nb;
    IRK_TRY(tmp.alloc((void**)&ab, std::max<size_t>(1, nlev) * per_level * sizeof(double)));
    std::vector<double> hab(std::max<size_t>(1, nlev) * per_level);
    for (int l = 0; l < nlev; ++l) {
      double* alpha = ab + (size_t)l * per_level;
      double* beta = alpha + (size_t)steps * nb;
      double* nrm0 = alpha + (size_t)2 * steps * nb;
      double* zeros = nrm0 + nb;  // beta_0 = 0 (allocation is zero-initialised)
      Lvl& L = lv_[l];
      const LevelGeom& g = L.g;
      const long long n = g.n, ldl = g.ld;
      const int nbl = std::min(reduction_blocks(n), nbred);
      // deterministic start vector on interior nodes (hash-based), same for every block
      IRK_CUDA(launch_hash_fill(g.grid(), nb, w, st));
      IRK_CUDA(cudaMemsetAsync(v0, 0, (size_t)nb * ldl * sizeof(double), st));
      IRK_CUDA(launch_block_dot(w, w, nb, n, ldl, partial, nbl, st));
      IRK_CUDA(launch_reduce_partials(partial, nb, nbl, nrm0, st, 1));
      IRK_CUDA(launch_block_shift(nullptr, v1, w, nrm0, nb, n, ldl, st));
      std::vector<double> one(nb, 1.0);
      DiagParams<double> D = make_diag_params<double>(g, nb, cfg_.cm.data(), ck_.data(), one.data());
      OpParams<LT> P = opp<LT>(g, nb, cfg_.cm.data(), ck_.data());
      EpiParams<LT> E;
      std::memset(&E, 0, sizeof(E));
      E.out = wf;
      // symmetric form D^{-1/2} A D^{-1/2}; every block advances together, no host round trip
      for (int it = 0; it < steps; ++it) {
        IRK_CUDA(launch_diag_scale<double, LT>(g.grid(), nb, v1, t, D, 1, st));
        IRK_CUDA(launch_op<LT>(g.dim, g.k, nb, t, P, EPI_STORE, E, st));
        IRK_CUDA(launch_diag_scale<LT, double>(g.grid(), nb, wf, w, D, 1, st));
        double* a_it = alpha + (size_t)it * nb;
        double* b_it = beta + (size_t)it * nb;
        const double* b_prev = (it == 0) ? zeros : beta + (size_t)(it - 1) * nb;
        IRK_CUDA(launch_block_dot(w, v1, nb, n, ldl, partial, nbl, st));
        IRK_CUDA(launch_reduce_partials(partial, nb, nbl, a_it, st));
        IRK_CUDA(launch_block_axpy2(w, v1, v0, a_it, b_prev, nb, n, ldl, st));
        IRK_CUDA(launch_block_dot(w, w, nb, n, ldl, partial, nbl, st));
        IRK_CUDA(launch_reduce_partials(partial, nb, nbl, b_it, st, 1));
        IRK_CUDA(launch_block_shift(v0, v1, w, b_it, nb, n, ldl, st));
      }
    }
    if (nlev > 0) {
      IRK_CUDA(cudaMemcpyAsync(hab.data(), ab, (size_t)nlev * per_level * sizeof(double), cudaMemcpyDeviceToHost, st));
      IRK_CUDA(cudaStreamSynchronize(st));
    }
    for (int l = 0; l < nlev; ++l) {
      Lvl& L = lv_[l];
      const double* hl = hab.data() + (size_t)l * per_level;
      std::vector<std::vector<double>> alpha_h(nb), beta_h(nb);
      for (int s = 0; s < nb; ++s) {
        for (int it = 0; it < steps; ++it) {
          const double a = hl[(size_t)it * nb + s], bb = hl[(size_t)(steps + it) * nb + s];
          alpha_h[s].push_back(a);
          if (!(bb > 1e-12 * std::fabs(a))) break;  // invariant subspace found
          if (it + 1 < steps) beta_h[s].push_back(bb);
        }
      }
      L.lo.resize(nb);
      L.hi.resize(nb);
      for (int s = 0; s < nb; ++s) {
        std::vector<double> b2(beta_h[s].begin(), beta_h[s].end());
        b2.resize(alpha_h[s].size() > 0 ? alpha_h[s].size() - 1 : 0);
        const double lmax = tridiag_max_eig(alpha_h[s], b2);
        L.hi[s] = cfg_.eig_safety * lmax;
        L.lo[s] = L.hi[s] / cfg_.smoothing_range;
      }
      if (cfg_.shared_cheb) {
        const double hmax = *std::max_element(L.hi.begin(), L.hi.end());
        for (int s = 0; s < nb; ++s) { L.hi[s] = hmax; L.lo[s] = hmax / cfg_.smoothing_range; }
      }
      // coefficients of the three-term recurrence
      const int m = cfg_.cheb_degree;
      L.c1.assign(m, std::vector<double>(nb, 0.0));
      L.c2.assign(m, std::vector<double>(nb, 0.0));
      for (int s = 0; s < nb; ++s) {
        const double theta = 0.5 * (L.hi[s] + L.lo[s]), delta = 0.5 * (L.hi[s] - L.lo[s]);
        double rho = delta / theta;
        L.c1[0][s] = 0.0;
        L.c2[0][s] = 1.0 / theta;
        for (int j = 1; j < m; ++j) {
          const double rn = 1.0 / (2.0 * theta / delta - rho);
          L.c1[j][s] = rn * rho;
          L.c2[j][s] = 2.0 * rn / delta;
          rho = rn;
        }
      }
    }
    IRK_CUDA(cudaStreamSynchronize(st));
    return Status::Ok();
  }

  MGConfig cfg_;
  Element1D el_;
  DeviceArena& arena_;
  std::vector<Lvl> lv_;
  std::vector<double> ck_;
  double* dAinv_ = nullptr;
  int* dmap_ = nullptr;
  int nci_ = 0;
  cudaStream_t st_ = nullptr;
  std::vector<double> ainv_host_;
  bool fused_ = false;
  int lc_ = -1;
  CoarseParams fparams_{};
  cudaGraph_t graph_ = nullptr;
  cudaGraphExec_t gexec_ = nullptr;
  long long gcounts_[PROF_NCAT] = {};
  int eager_runs_ = 0;
  static constexpr int kDenseCoarseMax = 729;  // dense inverse up to 9^3 unknowns, else fast diagonalisation
  bool use_fd_ = false;
  double *fd_V_ = nullptr, *fd_Vt_ = nullptr, *fd_mu_ = nullptr, *fd_t1_ = nullptr, *fd_t2_ = nullptr;
  FdParams fd_params_{};
};

}  // namespace

Status make_mg(const MGConfig& cfg, const Element1D& e, DeviceArena& arena, cudaStream_t st,
               std::unique_ptr<MGBase>& out) {
  if (cfg.precision == 64) {
    auto mg = std::make_unique<MG<double>>(cfg, e, arena);
    IRK_TRY(mg->setup(st));
    out = std::move(mg);
  } else {
    auto mg = std::make_unique<MG<float>>(cfg, e, arena);
    IRK_TRY(mg->setup(st));
    out = std::move(mg);
  }
  return Status::Ok();
}

}  // namespace irk
