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
// FP32 pipe.  Used for the FP64-accurate operator apply; stored in memory as FP64.
struct ff {
  float hi, lo;
};
template <typename T> struct Storage { using type = T; };
template <> struct Storage<ff> { using type = double; };

// Geometry and coefficients of one tensor-product operator launch
//   v_s = cm[s] M u_s + ck[s] K u_s          (s = blockIdx.z, one stage per CTA)
// M = Mz (x) My (x) Mx, K = Kz My Mx + Mz Ky Mx + Mz My Kx on the uniform mesh;
// me/ke are the 1D element matrices already scaled by h and 1/h.
template <typename T>
struct OpParams {
  int N, n1;           // cells per axis, nodes per axis (k N + 1)
  long long ld;        // elements between stage vectors
  int zc;              // streaming chunk, in cells (0: chosen by the launcher)
  int ntile_y;         // 3D: number of y tiles (grid.y = ntile_y * chunks)
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

// ---------------- pointwise / vector kernels (vec.cu) ----------------

constexpr int kMaxQ = 9;  // stage-combination matrices are at most 9 x 9

struct CombineParams {  // out_i = sum_j Da[i][j] a_j (+ sum_j Db[i][j] b_j)
  int nout, nina, ninb;
  double Da[kMaxQ * kMaxQ];
  double Db[kMaxQ * kMaxQ];
  unsigned nza[kMaxQ], nzb[kMaxQ];  // bit j of row i: coefficient (i, j) is nonzero (set by the launcher)
};
// Tin/Tout in {float,double}; a [nina][ld], b [ninb][ld] (may be null), out [nout][ld];
// n elements per vector are processed.
template <typename Tin, typename Tout>
cudaError_t launch_combine(const Tin* a, const double* b, Tout* out, long long n, long long ld,
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
// out = x * D^{-1/2} (inv_sqrt = 1) or out = x * D (inv_sqrt = 0), interior nodes.
template <typename T>
cudaError_t launch_diag_scale(const GridInfo& g, int nstage, const T* x, T* out, const DiagParams<T>& D,
                              int inv_sqrt, cudaStream_t st);

struct RhsParams {
  int Q;
  double Ainv[kMaxQ * kMaxQ];
  double phi[kMaxQ];
};
// rhs_i = sum_j Ainv[i][j] (load_j - Ky); load_j = phi_j (G1 (x) G1 (x) G1) (built-in source)
// or the user stage loads (device [Q][ld]) when loads != nullptr.
cudaError_t launch_stage_rhs(const GridInfo& g, const RhsParams& R, const double* Ky, const double* G1,
                             const double* loads, double* rhs, cudaStream_t st);
// y += tau sum_i b_i k_i
cudaError_t launch_update(const GridInfo& g, int Q, const double* kst, const double* bw, double tau,
                          double* y, cudaStream_t st);
// y = prod sin(pi x_a) * ct at nodes (x1d: node coordinates of one grid line, device)
cudaError_t launch_interpolate(const GridInfo& g, const double* x1d, double ct, double* y,
                               cudaStream_t st);

// Deterministic reductions over long vectors of length n (fixed block count from n).
int reduction_blocks(long long n);
// partial[i][nb] = partial dot(V_i, w), V_i = V + i * vstride, i < nv
cudaError_t launch_multidot(const double* V, long long vstride, int nv, const double* w, long long n,
                            double* partial, int nb, cudaStream_t st);
// out[i] = sum_b partial[i][b] (fixed order); with take_sqrt, out[i] = sqrt(sum)
cudaError_t launch_reduce_partials(const double* partial, int nv, int nb, double* out, cudaStream_t st,
                                   int take_sqrt = 0);
// partial[0][nb] = partial sum of w^2
cudaError_t launch_norm2_partial(const double* w, long long n, double* partial, int nb, cudaStream_t st);
// w -= sum_i h[i] V_i   (h on the device)
cudaError_t launch_multi_axpy(const double* V, long long vstride, int nv, const double* h, double sign,
                              double* w, long long n, cudaStream_t st);
// out = w * (1 / nrm[0])
cudaError_t launch_scale_inv(const double* w, const double* nrm, double* out, long long n, cudaStream_t st);
// out = a * x
cudaError_t launch_scale(const double* x, double a, double* out, long long n, cudaStream_t st);
// Fused Gram-Schmidt passes (classical Gram-Schmidt with the "twice is enough" test of Kahan
// and Parlett); partial has rows [0, nv] x nb:
//  gs_dot      : partial[i] = dot(V_i, w) (i < nv), partial[nv] = |w|^2
//  gs_axpy_dot : w_out = w_in - sum_i h[i] V_i; partial[i] = dot(V_i, w_out), partial[nv] = |w_out|^2
//  gs_reorth   : if |w_mid|^2 < eta^2 |w|^2 (device scalars norm2_mid, norm2_in): w_out = w_in - sum h[i] V_i,
//                else w_out = w_in; partial[0] = |w_out|^2
cudaError_t launch_gs_dot(const double* V, long long vstride, int nv, const double* w, long long n, double* partial,
                          int nb, cudaStream_t st);
cudaError_t launch_gs_axpy_dot(const double* V, long long vstride, int nv, const double* h, const double* w_in,
                               double* w_out, long long n, double* partial, int nb, cudaStream_t st);
cudaError_t launch_gs_reorth(const double* V, long long vstride, int nv, const double* h, const double* w_in,
                             double* w_out, long long n, const double* norm2_in, const double* norm2_mid, double eta,
                             double* partial, int nb, cudaStream_t st);

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

// Exact coarse solve by fast diagonalisation: (cm_s M + tau K)^{-1} = W diag(1/(cm_s + tau mu)) W^T,
// W = V (x) V (x) V with V^T M1 V = I, V^T K1 V = diag(mu1) on the interior 1D nodes.
struct FdParams {
  int ni;                   // interior nodes per axis
  double tau;
  double cm[kMaxStages];
};
// out = transform of `in` along `axis` on the interior grid: out[..i..] = sum_j Mt[i][j] in[..j..]
template <typename Tin, typename Tout>
cudaError_t launch_fd_axis(const Tin* in, Tout* out, int nstage, long long ld, int n1, int dim, int axis,
                           const double* Mt, int ni, cudaStream_t st);
// t[interior] *= 1 / (cm_s + tau (mu_a + mu_b (+ mu_c)))
cudaError_t launch_fd_scale(double* t, int nstage, long long ld, int n1, int dim, const double* mu,
                            const FdParams& P, cudaStream_t st);

// Dense coarse solve per stage: x[map] = Ainv_s b[map] (FP64 inverse), zero elsewhere untouched.
template <typename T>
cudaError_t launch_coarse_solve(const T* b, T* x, int nstage, long long ld, const double* Ainv,
                                const int* map, int nci, cudaStream_t st);

}  // namespace irk
