// Launch interface between the host solver and the sm_103a kernels of libirk.
// Host-only declarations: parameter structs passed by value to kernels, and
// launcher functions (defined in op_f32.cu, op_f64.cu, vec.cu).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace irk {

constexpr int kMaxStages = 16;   // per-launch stage slots (Q <= 9, 2x2 DIAG blocks use 2)
constexpr int kMaxDeg = 4;       // Q_k degree k <= 4

// Float-float value hi + lo (|lo| <= ulp(hi) / 2): about 48 significant bits computed on the
// FP32 pipe.  The FP64-accurate stage operator and the Krylov vectors use it; a vector of ff is
// stored as pairs (8 bytes per value, 8-byte aligned, the size of FP64).
struct alignas(8) ff {
  float hi, lo;
};
template <typename T> struct Storage { using type = T; };

// Geometry and coefficients of one tensor-product operator launch
//   v_s = cm[s] M u_s + ck[s] K u_s          (s = blockIdx.z, one stage per CTA)
// M = Mz (x) My (x) Mx, K = Kz My Mx + Mz Ky Mx + Mz My Kx on the uniform mesh;
// me/ke are the 1D element matrices already scaled by h and 1/h.
template <typename T>
struct OpParams {
  int N, n1;           // cells per axis, nodes per axis (k N + 1)
  long long ld;        // elements between stage vectors
  int zc;              // streaming chunk, in cells (0: chosen by the launcher)
  int ntile_y;         // 3D: number of y tiles (grid.y = ntile_y * nch, chunk index fastest)
  int nch;             // 3D: number of z chunks (set by the launcher)
  int cluster;         // 3D: 1 = the nch chunks of a tile form a thread-block cluster (set by the launcher)
  int shape_ns;        // 3D: stage count whose launch shape this launch takes (0: nstage).  Launches that
                       // batch the stages of several requests use the shape of one request's stages, so
                       // each stage's arithmetic (chunk-boundary summation order) is the same as alone
  T me[kMaxDeg + 1][kMaxDeg + 1];
  T ke[kMaxDeg + 1][kMaxDeg + 1];
  T yvm[2 * kMaxDeg + 1], yvk[2 * kMaxDeg + 1];  // banded taps of a vertex row, offsets -k..k
  T cm[kMaxStages], ck[kMaxStages];
};

enum EpiKind { EPI_STORE = 0, EPI_DUAL = 1, EPI_RESID = 2, EPI_CHEB = 3 };

// Fused epilogue of an operator launch, evaluated once per interior output node.
//  STORE: out = v                      DUAL: out = M u, out2 = K u (cm/ck ignored)
//  RESID: out = b - v
//  CHEB : out(x_{j-1} in, x_{j+1} out) = x_j + c1 (x_j - x_{j-1}) + c2 D^{-1} (b - v)
//         with D = diag(cm M + ck K) from the 1D diagonals dmr/dkr (indexed by node mod k).
template <typename T>
struct EpiParams {
  T* out;
  T* out2;
  const T* b;
  const T* xj;
  T c1[kMaxStages], c2[kMaxStages];
  T dmr[kMaxDeg], dkr[kMaxDeg];
  int xold_zero;
};

// Launch v = op(u) with the given epilogue; dim in {2,3}, k in 1..4, nstage <= kMaxStages.
// T is the arithmetic type (float, double, ff); vectors are stored as Storage<T>::type.
template <typename T>
cudaError_t launch_op(int dim, int k, int nstage, const typename Storage<T>::type* u, const OpParams<T>& P,
                      int epi, const EpiParams<typename Storage<T>::type>& E, cudaStream_t st);

// Tile shape used by launch_op (cells per CTA in x and y) for a degree k.
void op_tile_shape(int dim, int k, int* cx, int* cy);

// Autotuning of a 3D operator launch: times the candidate launch shapes (warp-segment width,
// z chunk, thread-block cluster) on this call's arguments and keeps the fastest for every later
// launch of the same kernel with the same cells per axis and stage count (process-wide).  The
// call's outputs must be scratch: the candidates run repeatedly.  Returns at once when the
// shape is known, for 2D, during stream capture, and for small launches (model shape kept).
template <typename T>
cudaError_t tune_op(int dim, int k, int nstage, const typename Storage<T>::type* u, const OpParams<T>& P,
                    int epi, const EpiParams<typename Storage<T>::type>& E, cudaStream_t st);
// Registry of the tuned shapes (tune.cpp): one line per tuned kernel and size.
void tune_record(const char* kernel, int k, int epi, int N, int nstage, int cxs, int zc, int cluster,
                 double us, double us_model, int model_cxs, int model_zc, int model_cluster);
int tune_report(char* buf, int len);
// Test support: a launch shape forced on every later 3D streaming operator launch of one element
// size (elem 4: the FP32 multigrid kernels, 8: the FP64-accurate kernels; cxs = 0 clears it), and
// the shape (cxs, zc, cluster, z chunks) of the last such launch.
void op_shape_force(int elem, int cxs, int zc, int cluster);
bool op_shape_forced(int elem, int* cxs, int* zc, int* cluster);
void op_shape_record(int elem, int cxs, int zc, int cluster, int nch);
bool op_shape_last(int elem, int* out4);

// ---------------- pointwise / vector kernels (vec.cu) ----------------

constexpr int kMaxQ = 9;  // stage-combination matrices are at most 9 x 9

struct CombineParams {  // out_i = sum_j Da[i][j] a_j (+ sum_j Db[i][j] b_j)
  int nout, nina, ninb;
  double Da[kMaxQ * kMaxQ];
  double Db[kMaxQ * kMaxQ];
  unsigned nza[kMaxQ], nzb[kMaxQ];  // bit j of row i: coefficient (i, j) is nonzero (set by the launcher)
  float Dah[kMaxQ * kMaxQ], Dal[kMaxQ * kMaxQ], Dbh[kMaxQ * kMaxQ], Dbl[kMaxQ * kMaxQ];  // ff split (launcher)
};

// Storage types of the outer solver's stage vectors: double (plain FP64 path) or ff.  Coef<S> is
// the type of the device-side coefficients those kernels read (h of Gram-Schmidt, 1/norm, y).
template <typename S> struct Coef { using type = double; };
template <> struct Coef<ff> { using type = ff; };

// hi + lo split of an FP64 coefficient on the host
void split_double(double d, float* hi, float* lo);

// a [nina][ld] of Ta, b [ninb][ld] of Tb (may be null), out [nout][ld] of Tout; n elements per vector.
// Arithmetic in ff when any of the three is ff, else FP64.
template <typename Ta, typename Tb, typename Tout>
cudaError_t launch_combine(const Ta* a, const Tb* b, Tout* out, long long n, long long ld,
                           const CombineParams& C, cudaStream_t st);

struct GridInfo {      // node grid of one level
  int dim, k, N, n1;
  long long n, ld;
};

// Per-stage diagonal data of a level operator cm M + ck K, and a per-stage scalar c.
template <typename T>
struct DiagParams {
  T cm[kMaxStages], ck[kMaxStages], c[kMaxStages];
  T dmr[kMaxDeg], dkr[kMaxDeg];
};

// x = c[s] D^{-1} b (first Chebyshev step from x0 = 0), interior nodes, all stages.
template <typename T>
cudaError_t launch_cheb_first(const GridInfo& g, int nstage, const T* b, T* x, const DiagParams<T>& D,
                              cudaStream_t st);
// Deterministic start vector of the Lanczos estimate: 0.5 + hash(node) / 2^53 on interior nodes, zero
// elsewhere, identical for every block.
cudaError_t launch_hash_fill(const GridInfo& g, int nstage, double* x, cudaStream_t st);
// out = x * D^{-1/2} (inv_sqrt = 1) or out = x * D (inv_sqrt = 0), interior nodes; the factor in
// FP32, the product in FP64 (Tin, Tout in {float, double, ff}: float with float only).
template <typename Tin, typename Tout>
cudaError_t launch_diag_scale(const GridInfo& g, int nstage, const Tin* x, Tout* out, const DiagParams<double>& D,
                              int inv_sqrt, cudaStream_t st);

struct RhsParams {
  int Q;
  double Ainv[kMaxQ * kMaxQ];
  double phi[kMaxQ];
  float Ainvh[kMaxQ * kMaxQ], Ainvl[kMaxQ * kMaxQ], phih[kMaxQ], phil[kMaxQ];  // ff split (launcher)
};
// rhs_i = sum_j Ainv[i][j] (load_j - Ky); load_j = phi_j (G1 (x) G1 (x) G1) (built-in source; phi_j Gv
// with the full load vector Gv when Gv != nullptr) or the user stage loads (device [Q][ld], FP64)
// when loads != nullptr.  Ky, rhs of type S.
template <typename S>
cudaError_t launch_stage_rhs(const GridInfo& g, const RhsParams& R, const S* Ky, const double* G1, const double* Gv,
                             const double* loads, S* rhs, cudaStream_t st);
// y += tau sum_i b_i k_i  (k of type S, y FP64)
template <typename S>
cudaError_t launch_update(const GridInfo& g, int Q, const S* kst, const double* bw, double tau,
                          double* y, cudaStream_t st);
// FP64 <-> ff copies of n values
cudaError_t launch_to_ff(const double* in, ff* out, long long n, cudaStream_t st);
cudaError_t launch_from_ff(const ff* in, double* out, long long n, cudaStream_t st);
// y = prod sin(pi x_a) * ct at nodes (x1d: node coordinates of one grid line, device)
cudaError_t launch_interpolate(const GridInfo& g, const double* x1d, double ct, double* y,
                               cudaStream_t st);

// Deterministic reductions over long vectors of length n (fixed block count from n).
int reduction_blocks(long long n);
// partial[i][nb] = partial dot(V_i, w), V_i = V + i * vstride, i < nv (FP64 vectors)
cudaError_t launch_multidot(const double* V, long long vstride, int nv, const double* w, long long n,
                            double* partial, int nb, cudaStream_t st);
// Optional outputs of a reduction, written by the block that finishes the row.
struct ReduceExtra {
  ff* out_ff = nullptr;               // ff copy of each row result
  double* inv = nullptr;              // 1 / (row 0 result), 0 when the result is 0
  ff* inv_ff = nullptr;               // the same in ff
  // Second Gram-Schmidt pass or not, decided once every row is final (rows 0 .. sel_nv - 1: the
  // coefficients h = V^T w; row sel_nv: |w|^2).  sel_flag[0] = 1.0 when the new basis vector would
  // lose orthogonality beyond sel_tol after one pass, else 0.0; sel_delta[0] carries the basis's estimated
  // loss of orthogonality from one Arnoldi step to the next (taken as 0 when sel_nv == 1);
  // sel_round is the rounding of one pass and sel_tol the loss allowed.
  double* sel_flag = nullptr;
  double* sel_delta = nullptr;
  int sel_nv = -1;
  double sel_round = 0.0, sel_tol = 0.0;
  // Norm of a Gram-Schmidt result that gets no second pass (clear_flag[0] == 0): sqrt of row
  // clear_row into clear_norm[0], its inverse (0 for 0) into clear_inv[0] and clear_inv_ff[0].
  const double* clear_flag = nullptr;
  int clear_row = -1;
  double* clear_norm = nullptr;
  double* clear_inv = nullptr;
  ff* clear_inv_ff = nullptr;
};
// Rows finished inside the kernel that produced their partials: every block adds its partials,
// and the block that arrives last on *count sums each row over the blocks in a fixed order, writes
// out[i] (sqrt with take_sqrt) and the extras, and resets *count to 0.
struct RowSink {
  double* out = nullptr;
  unsigned* count = nullptr;
  int take_sqrt = 0;
  ReduceExtra X;
};
// out[i] = sum_b partial[i][b] (fixed order); with take_sqrt, out[i] = sqrt(sum)
cudaError_t launch_reduce_partials(const double* partial, int nv, int nb, double* out, cudaStream_t st,
                                   int take_sqrt = 0, const ReduceExtra* extra = nullptr);
// Vector work of FGMRES on stage vectors of type S (double or ff); reductions produce FP64
// partial sums per block (rows of nb), finished by the kernel's last block into the RowSink.  nb is
// in-out: at most nb blocks (the row capacity of partial), the blocks used (one full wave of the
// kernel) on return.
//  norm2_partial: partial[0] = |w|^2
//  multi_axpy   : w += sign sum_i h[i] V_i          (h on the device, Coef<S>)
//  scale_dev    : out = inv[0] w                    (inv on the device, Coef<S>; out may alias w)
//  scale        : out = a x                         (a from the host)
//  gs_dot       : partial[i] = dot(V_i, w) (i < nv), partial[nv] = |w|^2
//  gs_axpy_dot  : w_out = w_in - sum_i h[i] V_i; partial[i] = dot(V_i, w_out) when *dots_flag != 0
//                 (or dots_flag is null; else 0), partial[nv] = |w_out|^2.  w_out may be w_in for
//                 nv <= 16 (element-wise in place)
//  gs_reorth    : w_out = w_in - sum_i h[i] V_i if *redo_flag != 0 (second pass of classical
//                 Gram-Schmidt), else w_out = w_in; partial[0] = |w_out|^2.  w_out may be w_in;
//                 then nothing runs when *redo_flag == 0 (the norm comes from gs_axpy_dot)
template <typename S>
cudaError_t launch_norm2_partial(const S* w, long long n, double* partial, int& nb, const RowSink& R,
                                 cudaStream_t st);
template <typename S>
cudaError_t launch_multi_axpy(const S* V, long long vstride, int nv, const typename Coef<S>::type* h, double sign,
                              S* w, long long n, cudaStream_t st);
template <typename S>
cudaError_t launch_scale_dev(const S* w, const typename Coef<S>::type* inv, S* out, long long n, cudaStream_t st);
template <typename S>
cudaError_t launch_scale(const S* x, double a, S* out, long long n, cudaStream_t st);
template <typename S>
cudaError_t launch_gs_dot(const S* V, long long vstride, int nv, const S* w, long long n, double* partial, int& nb,
                          const RowSink& R, cudaStream_t st);
template <typename S>
cudaError_t launch_gs_axpy_dot(const S* V, long long vstride, int nv, const typename Coef<S>::type* h,
                               const S* w_in, S* w_out, long long n, double* partial, int& nb, const RowSink& R,
                               const double* dots_flag, cudaStream_t st);
template <typename S>
cudaError_t launch_gs_reorth(const S* V, long long vstride, int nv, const typename Coef<S>::type* h,
                             const double* redo_flag, const S* w_in, S* w_out, long long n, double* partial, int& nb,
                             const RowSink& R, cudaStream_t st);

// Block-wise helpers (ns vectors of n elements at stride ld), coefficients on the device:
//  block_dot:   partial[s][nb] = partial sums of a_s . b_s
//  block_axpy2: w_s -= alpha[s] v1_s + beta[s] v0_s
//  block_shift: v0_s = v1_s; v1_s = w_s / nrm[s] (0 where nrm[s] == 0); with v0 = nullptr: v1_s = w_s / nrm[s]
cudaError_t launch_block_dot(const double* a, const double* b, int ns, long long n, long long ld, double* partial,
                             int nb, cudaStream_t st);
cudaError_t launch_block_axpy2(double* w, const double* v1, const double* v0, const double* alpha, const double* beta,
                               int ns, long long n, long long ld, cudaStream_t st);
cudaError_t launch_block_shift(double* v0, double* v1, const double* w, const double* nrm, int ns, long long n,
                               long long ld, cudaStream_t st);

// ---------------- intergrid transfer (Q_k embedding) ----------------
struct TransferParams {
  int k, Nc;                 // degree, coarse cells per axis
  double Pc[(2 * kMaxDeg + 1) * (kMaxDeg + 1)];  // (2k+1) x (k+1)
  float Pcf[(2 * kMaxDeg + 1) * (kMaxDeg + 1)];  // the same in FP32 (arithmetic of the FP32 multigrid)
};
// One 1D pass along `axis` of a 3D (or 2D, d2 = 1) array; in/out dims (x fastest).
// restrict: out[.. c ..] = sum_f P1[f][c] in[.. f ..]; prolong: out[.. f ..] (+)= sum_c P1[f][c] in[.. c ..]
template <typename T>
cudaError_t launch_transfer_axis(const T* in, T* out, int nstage, long long ld_in, long long ld_out,
                                 const int din[3], const int dout[3], int axis, int restrict_mode,
                                 int accumulate, const TransferParams& P, cudaStream_t st);

// Exact coarse solve by fast diagonalisation: (cm_s M + tau_s K)^{-1} = W diag(1/(cm_s + tau_s mu)) W^T,
// W = V (x) V (x) V with V^T M1 V = I, V^T K1 V = diag(mu1) on the interior 1D nodes.
struct FdParams {
  int ni;                   // interior nodes per axis
  double taus[kMaxStages];  // stiffness coefficient tau of each block
  double cm[kMaxStages];
  double beta;              // coupled 2x2 systems (launch_fd_scale_coupled): coupling coefficient
};
// out = transform of `in` along `axis` on the interior grid: out[..i..] = sum_j Mt[i][j] in[..j..]
template <typename Tin, typename Tout>
cudaError_t launch_fd_axis(const Tin* in, Tout* out, int nstage, long long ld, int n1, int dim, int axis,
                           const double* Mt, int ni, cudaStream_t st);
// t[interior] *= 1 / (cm_s + tau_s (mu_a + mu_b (+ mu_c)))
cudaError_t launch_fd_scale(double* t, int nstage, long long ld, int n1, int dim, const double* mu,
                            const FdParams& P, cudaStream_t st);
// The coupled 2x2 system [[A, -beta M], [beta M, A]], A = cm[0] M + tau K, in modal coordinates:
// per mode (t0, t1) <- [[a, -beta], [beta, a]]^{-1} (t0, t1), a = cm[0] + tau mu; t0 at t, t1 at t + ld.
cudaError_t launch_fd_scale_coupled(double* t, long long ld, int n1, int dim, const double* mu, const FdParams& P,
                                    cudaStream_t st);

// Level operator of the coupled 2x2 system [[A, -beta M], [beta M, A]] (A = cm M + ck K; a 2x2
// block of Eq. complex:twobytwo) from the products M x_s, K x_s of its two components (s = 0, 1,
// at stride ld), fused with the residual or the Chebyshev step around point-Jacobi, the point
// being a node with its two components: D2 = [[d, -beta m], [beta m, d]], d = diag(A), m = diag(M):
//   cheb = 0: out = b - A2 x
//   cheb = 1: out = x + c1 (x - xold) + c2 D2^{-1} (b - A2 x), xold read from out (zero when xold_zero)
//   cheb = 2: out = c2 D2^{-1} b (first step from x = 0; mx, kx, x unused).  Interior nodes only.
struct CoupledParams {
  double cm, ck, beta, c1, c2;
  double dmr[kMaxDeg], dkr[kMaxDeg];
  int cheb, xold_zero;
};
template <typename T>
cudaError_t launch_coupled_update(const GridInfo& g, const T* mx, const T* kx, const T* x, const T* b, T* out,
                                  const CoupledParams& C, cudaStream_t st);

// Dense coarse solve per stage: x[map] = Ainv_s b[map] (FP64 inverse), zero elsewhere untouched.
template <typename T>
cudaError_t launch_coarse_solve(const T* b, T* x, int nstage, long long ld, const double* Ainv,
                                const int* map, int nci, cudaStream_t st);

}  // namespace irk
