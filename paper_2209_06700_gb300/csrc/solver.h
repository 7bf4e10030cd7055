// Host solver of libirk: multigrid hierarchy, FGMRES, IRK step (internal).
#pragma once
#include <cuda_runtime.h>

#include <functional>
#include <memory>
#include <string>
#include <vector>

#include "host_math.h"
#include "irk.h"
#include "kernels.h"

namespace irk {

struct Status {
  irk_status code = IRK_OK;
  std::string msg;
  bool ok() const { return code == IRK_OK; }
  static Status Ok() { return Status(); }
  static Status Err(irk_status c, std::string m) { Status s; s.code = c; s.msg = std::move(m); return s; }
};

#define IRK_CUDA(...)                                                                            \
  do {                                                                                           \
    cudaError_t e_ = (__VA_ARGS__);                                                              \
    if (e_ != cudaSuccess)                                                                       \
      return ::irk::Status::Err(IRK_ECUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_)); \
  } while (0)
#define IRK_TRY(...)                   \
  do {                                 \
    ::irk::Status s_ = (__VA_ARGS__);  \
    if (!s_.ok()) return s_;           \
  } while (0)

// Device allocation owned by the handle (freed in reverse order).
class DeviceArena {
 public:
  explicit DeviceArena(cudaStream_t st = nullptr) : st_(st) {}
  ~DeviceArena();
  DeviceArena(const DeviceArena&) = delete;
  DeviceArena& operator=(const DeviceArena&) = delete;
  void set_stream(cudaStream_t st) { st_ = st; }
  Status alloc(void** p, size_t bytes);  // zero-initialised, stream-ordered
  size_t bytes() const { return total_; }
 private:
  cudaStream_t st_;
  std::vector<void*> ptrs_;
  size_t total_ = 0;
};

long long round_ld(long long n);

// One mesh level of the hierarchy.
struct LevelGeom {
  int dim, k, N, n1;
  long long n, ld;
  double h;
  double me[kMaxDeg + 1][kMaxDeg + 1], ke[kMaxDeg + 1][kMaxDeg + 1];
  double dmr[kMaxDeg], dkr[kMaxDeg];
  GridInfo grid() const { return GridInfo{dim, k, N, n1, n, ld}; }
};

LevelGeom make_level(int dim, int k, int N, const Element1D& e);

template <typename T>
OpParams<T> make_op_params(const LevelGeom& g, int nstage, const double* cm, const double* ck);
template <typename T>
DiagParams<T> make_diag_params(const LevelGeom& g, int nstage, const double* cm, const double* ck, const double* c);

// Geometric multigrid for nb independent blocks (cm_i M + tau K), element type T.
class MGBase {
 public:
  virtual ~MGBase() = default;
  virtual int levels() const = 0;
  virtual int elem_size() const = 0;
  // finest-level rhs / solution buffers ([nb][ld0], element type T)
  virtual void* fine_b() = 0;
  virtual void* fine_x() = 0;          // result of the last vcycle on level 0
  virtual Status vcycle(int level, cudaStream_t st) = 0;  // b_level -> x_level
  // V-cycle from the finest level; replayed from a captured CUDA graph when allowed (non-default
  // stream, no per-kernel timing requested), after one eager run.
  virtual Status vcycle_top(cudaStream_t st, bool allow_graph) = 0;
  virtual Status vcycle_io(int level, const void* b, void* x, cudaStream_t st) = 0;
  virtual Status smooth(int level, const void* b, void* x, int x_is_zero, cudaStream_t st) = 0;
  virtual Status residual(int level, const void* b, const void* x, void* r, cudaStream_t st) = 0;
  virtual Status restrict_to(int level, const void* r, void* bc, cudaStream_t st) = 0;
  // The same restriction with its two intermediate axis-pass grids placed in caller-provided
  // device scratch of `bytes` bytes (cleared here before use); EINVAL if it does not fit.
  virtual Status restrict_in_scratch(int level, const void* r, void* bc, void* scratch, size_t bytes,
                                     cudaStream_t st) = 0;
  virtual Status prolongate_add(int level, const void* ec, void* x, cudaStream_t st) = 0;
  virtual Status coarse_solve(const void* b, void* x, cudaStream_t st) = 0;
  virtual Status apply_mass(int level, const void* x, void* y, double scale, cudaStream_t st) = 0;
  virtual const LevelGeom& geom(int level) const = 0;
  // New per-block stiffness coefficients (nb values): rebuilds what depends on them (level operator
  // coefficients, Chebyshev intervals, coarse inverses, fused-cycle parameters) on the existing buffers
  // and drops the captured V-cycle graph.
  virtual Status retau(const std::vector<double>& taus, cudaStream_t st) = 0;
  virtual void interval(int level, int block, double* lo, double* hi) const = 0;
};

struct MGConfig {
  int dim, k, N;
  int nb;                    // blocks
  std::vector<double> cm;    // per-block mass coefficient lambda_i
  double tau;
  int cheb_degree;
  int eig_steps;
  double smoothing_range, eig_safety;
  int shared_cheb;
  int batched;
  int precision;             // 32 or 64
  int autotune = 1;          // time the level operators' launch shapes at setup
  double coupled_beta = 0.0; // != 0: nb = 2 components of [[A, -beta M], [beta M, A]], A = cm M + tau K
  std::vector<double> taus;  // per-block stiffness coefficient (blocks of several requests); empty: tau for all
  int shape_ns = 0;          // blocks per request: level-operator launches take that count's launch shape
};

Status make_mg(const MGConfig& cfg, const Element1D& e, DeviceArena& arena, cudaStream_t st,
               std::unique_ptr<MGBase>& out);

// Right-preconditioned flexible GMRES on ns stage vectors of stride ld.  The vectors are stored
// as 8-byte elements of type S: double (plain FP64 path) or ff (float-float, FP32 pipe); the
// Hessenberg matrix, Givens rotations and small solves run on the host in FP64.
struct FGMRESWork {
  int ns = 0, m = 0;
  long long ld = 0, len = 0;  // len = ns * ld
  double* V = nullptr;        // (m+1) x len elements of S
  double* Z = nullptr;        // m x len
  double* tmp = nullptr;      // len (restart residual, second Gram-Schmidt pass)
  double* partial = nullptr;  // 66 x nb
  double* dvals = nullptr;    // device scalars: h1[65], h2[65], norms, decision, y[64], 1
  ff* fvals = nullptr;        // the same scalars split into ff (the ff kernels' coefficients)
  double* hvals = nullptr;    // pinned host mirror
  double* hvals2 = nullptr;   // second pinned block: iteration j's scalars land in block j % 2
  cudaEvent_t ev[2] = {nullptr, nullptr};  // recorded after the read-back of iteration j into block j % 2
  unsigned* count = nullptr;  // arrival counter of the fused reductions (0 between kernels)
  int nb = 0;
  int always_two_passes = 0;  // 1: second Gram-Schmidt pass at every step (else where needed)
};
// Releases the pinned blocks and events of fgmres_alloc.
void fgmres_release(FGMRESWork& w);

Status fgmres_alloc(FGMRESWork& w, int ns, long long ld, int m, DeviceArena& arena, cudaStream_t stream);
double* pinned_block_acquire();
void pinned_block_release(double* p);

struct FGMRESResult { int iterations = 0; int reorth = 0; double rel_residual = 0; bool converged = false; };

template <typename S>
using ApplyFn = std::function<Status(const S* in, S* out)>;

template <typename S>
Status fgmres_solve(FGMRESWork& w, const ApplyFn<S>& op, const ApplyFn<S>& prec, const S* b, S* x, double rtol,
                    int max_it, cudaStream_t st, FGMRESResult& res);

// Lockstep flexible GMRES for R independent systems (one per request of a group handle), stored
// interleaved in w's arrays: vector j of request r at base + (j R + r) len, len = w.len / R.  op and
// prec act on the R requests' vectors at once (shared launches); the Gram-Schmidt passes, norms,
// Hessenberg matrices, Givens rotations and convergence tests are per request, with one device->host
// transfer per iteration for all of them.  A request that has stopped (converged, failed or out of
// iterations) keeps its result; its later slices are zero.  Scalars: per-request blocks of 256
// values in dvals / fvals and one pinned host block per request; status per request in st_out.
struct GroupScalars {
  double* dvals = nullptr;     // R x 256 device FP64 scalars
  ff* fvals = nullptr;         // R x 256 device ff scalars
  std::vector<double*> hvals;  // R pinned host blocks of 256 (from the process-wide pool)
  unsigned* count = nullptr;   // R arrival counters of the fused reductions
};
Status group_scalars_alloc(GroupScalars& g, int R, DeviceArena& arena, cudaStream_t st);
void group_scalars_release(GroupScalars& g);
template <typename S>
Status fgmres_solve_group(FGMRESWork& w, int R, GroupScalars& gs, const ApplyFn<S>& op, const ApplyFn<S>& prec,
                          const S* b, S* x, double rtol, int max_it, cudaStream_t st,
                          std::vector<FGMRESResult>& res, std::vector<Status>& st_out);

}  // namespace irk
