// Pointwise, reduction, transfer and coarse-solve kernels of libirk (sm_103a).
//
// * Stage combination v_i = sum_j D_ij u_j: the "generalized matrix-vector
//   product" (D (x) I) u of arXiv 2209.06700, Sec. 2, used for A^{-1}, S~^{-1},
//   S~ (Eq. irk:A, irk:P) and T, T^{-1} (Eq. irk:Ainv, real form).  On one GPU
//   all stages of a node sit in the same memory, so the combination is an
//   elementwise kernel reading the Q stage values of each node.
// * Stage right-hand side and solution update (Sec. 1 and Sec. 2).
// * Deterministic reductions for FGMRES (fixed block counts, fixed order).
// * Intergrid transfer: the Q_k embedding P = P1 (x) P1 (x) P1 and its transpose,
//   applied one axis at a time.
// * Dense coarse-grid solve with a precomputed FP64 inverse.
#include <algorithm>
#include <cstdint>

#include "kernels.h"

namespace irk {

namespace {

constexpr int kThreads = 256;

inline int blocks_for(long long n, int per_thread = 1) {
  long long b = (n + (long long)kThreads * per_thread - 1) / ((long long)kThreads * per_thread);
  if (b < 1) b = 1;
  if (b > 152 * 32) b = 152 * 32;
  return (int)b;
}

// 32-bit index arithmetic: a stage vector has fewer than 2^31 nodes
__device__ __forceinline__ void coords(int idx, int dim, int n1, int& x, int& y, int& z) {
  x = idx % n1;
  const int r = idx / n1;
  y = r % n1;
  z = (dim == 3) ? r / n1 : 0;
}

__device__ __forceinline__ bool interior(int dim, int n1, int x, int y, int z) {
  bool ok = x >= 1 && x <= n1 - 2 && y >= 1 && y <= n1 - 2;
  if (dim == 3) ok = ok && z >= 1 && z <= n1 - 2;
  return ok;
}

template <typename T>
__device__ __forceinline__ T diag_at(const DiagParams<T>& D, int s, int dim, int k, int x, int y, int z) {
  const int rx = x % k, ry = y % k;
  T dmx = D.dmr[rx], dmy = D.dmr[ry], dkx = D.dkr[rx], dky = D.dkr[ry];
  if (dim == 3) {
    const int rz = z % k;
    T dmz = D.dmr[rz], dkz = D.dkr[rz];
    return D.cm[s] * (dmx * dmy * dmz) + D.ck[s] * (dkx * dmy * dmz + dmx * dky * dmz + dmx * dmy * dkz);
  }
  return D.cm[s] * (dmx * dmy) + D.ck[s] * (dkx * dmy + dmx * dky);
}

// ------------------------------------------------------------ stage combination
// NMAX: compile-time bound on the number of input/output stage vectors (keeps the
// per-thread arrays in registers at a register count that allows full occupancy).
template <typename Tin, typename Tout, int NMAX>
__global__ void __launch_bounds__(kThreads) combine_kernel(const Tin* __restrict__ a, const double* __restrict__ b,
                                                           Tout* __restrict__ out, int n, long long ld,
                                                           const CombineParams C) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    double av[NMAX], bv[NMAX];
#pragma unroll
    for (int j = 0; j < NMAX; ++j) {
      av[j] = (j < C.nina) ? (double)a[j * ld + e] : 0.0;
      bv[j] = (j < C.ninb) ? b[j * ld + e] : 0.0;
    }
#pragma unroll
    for (int i = 0; i < NMAX; ++i) {
      if (i < C.nout) {
        double acc = 0.0;
        // zero coefficients (triangular S~, diagonal stiffness coupling) are skipped through
        // host-built integer masks: FP64 instructions, compares included, are scarce on this part
#pragma unroll
        for (int j = 0; j < NMAX; ++j) {
          if ((C.nza[i] >> j) & 1u) acc += C.Da[i * kMaxQ + j] * av[j];
          if ((C.nzb[i] >> j) & 1u) acc += C.Db[i * kMaxQ + j] * bv[j];
        }
        out[i * ld + e] = (Tout)acc;
      }
    }
  }
}

// Structured combinations with compile-time stage count Q (no dead FP64 instructions: on this
// part every FP64 instruction, predicated or not, occupies the narrow FP64 pipe).
//  UNIT_LOWER: out_i = a_i + sum_{j<i} Da[i][j] a_j          (S~ and S~^{-1}, unit lower triangular)
//  FULL_DIAGB: out_i = sum_j Da[i][j] a_j + Db[i][i] b_i      (A^{-1} (x) M + tau I (x) K combination)
enum CombineStructure { CS_UNIT_LOWER = 1, CS_FULL_DIAGB = 2 };
template <typename Tin, typename Tout, int Q, int CS>
__global__ void __launch_bounds__(kThreads) combine_struct_kernel(const Tin* __restrict__ a,
                                                                  const double* __restrict__ b,
                                                                  Tout* __restrict__ out, int n, long long ld,
                                                                  const CombineParams C) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    double av[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) av[j] = (double)a[j * ld + e];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      double acc;
      if constexpr (CS == CS_UNIT_LOWER) {
        acc = av[i];
#pragma unroll
        for (int j = 0; j < i; ++j) acc = fma(C.Da[i * kMaxQ + j], av[j], acc);
      } else {
        acc = C.Db[i * kMaxQ + i] * b[i * ld + e];
#pragma unroll
        for (int j = 0; j < Q; ++j) acc = fma(C.Da[i * kMaxQ + j], av[j], acc);
      }
      out[i * ld + e] = (Tout)acc;
    }
  }
}

// ------------------------------------------------------------ Chebyshev start, diag scaling
template <typename T>
__global__ void cheb_first_kernel(GridInfo g, const T* __restrict__ b, T* __restrict__ x, const DiagParams<T> D) {
  const int s = blockIdx.y;
  const int n = (int)g.n;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    int ix, iy, iz;
    coords(e, g.dim, g.n1, ix, iy, iz);
    if (!interior(g.dim, g.n1, ix, iy, iz)) continue;
    const long long o = s * g.ld + e;
    x[o] = D.c[s] * b[o] / diag_at(D, s, g.dim, g.k, ix, iy, iz);
  }
}

template <typename T>
__global__ void diag_scale_kernel(GridInfo g, const T* __restrict__ x, T* __restrict__ out, const DiagParams<T> D,
                                  int inv_sqrt) {
  const int s = blockIdx.y;
  const int n = (int)g.n;
  // the diagonal factor in FP32 (this scaling only feeds the Chebyshev-interval estimate): the
  // 1D diagonals are converted once per block into shared memory, only the multiply by x uses
  // the type of x
  __shared__ float sdm[kMaxDeg], sdk[kMaxDeg];
  if (threadIdx.x < kMaxDeg) {
    sdm[threadIdx.x] = (float)D.dmr[threadIdx.x];
    sdk[threadIdx.x] = (float)D.dkr[threadIdx.x];
  }
  __syncthreads();
  const float cm = (float)D.cm[s], ck = (float)D.ck[s];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    int ix, iy, iz;
    coords(e, g.dim, g.n1, ix, iy, iz);
    if (!interior(g.dim, g.n1, ix, iy, iz)) continue;
    const long long o = s * g.ld + e;
    const int rx = ix % g.k, ry = iy % g.k;
    const float mx = sdm[rx], my = sdm[ry], kx = sdk[rx], ky = sdk[ry];
    float d;
    if (g.dim == 3) {
      const int rz = iz % g.k;
      const float mz = sdm[rz], kz = sdk[rz];
      d = cm * (mx * my * mz) + ck * (kx * my * mz + mx * ky * mz + mx * my * kz);
    } else {
      d = cm * (mx * my) + ck * (kx * my + mx * ky);
    }
    out[o] = x[o] * (T)(inv_sqrt ? rsqrtf(d) : d);
  }
}

__global__ void hash_fill_kernel(GridInfo g, double* __restrict__ x) {
  const int s = blockIdx.y;
  const int n = (int)g.n;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    int ix, iy, iz;
    coords(e, g.dim, g.n1, ix, iy, iz);
    double v = 0.0;
    if (interior(g.dim, g.n1, ix, iy, iz)) {
      unsigned long long h = (unsigned long long)(e + 1) * 0x9E3779B97F4A7C15ULL;
      h ^= h >> 29;
      h *= 0xBF58476D1CE4E5B9ULL;
      h ^= h >> 32;
      v = 0.5 + (double)(h >> 11) * (1.0 / 9007199254740992.0);
    }
    x[s * g.ld + e] = v;
  }
}

// ------------------------------------------------------------ RHS, update, interpolation
__global__ void stage_rhs_kernel(GridInfo g, const RhsParams R, const double* __restrict__ Ky,
                                 const double* __restrict__ G1, const double* __restrict__ loads,
                                 double* __restrict__ rhs) {
  const int n = (int)g.n;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    int ix, iy, iz;
    coords(e, g.dim, g.n1, ix, iy, iz);
    if (!interior(g.dim, g.n1, ix, iy, iz)) continue;
    const double ky = Ky[e];
    double G = G1[ix] * G1[iy];
    if (g.dim == 3) G *= G1[iz];
    double f[kMaxQ];
#pragma unroll
    for (int j = 0; j < kMaxQ; ++j)
      if (j < R.Q) f[j] = (loads ? loads[j * g.ld + e] : R.phi[j] * G) - ky;
#pragma unroll
    for (int i = 0; i < kMaxQ; ++i) {
      if (i >= R.Q) break;
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j < kMaxQ; ++j)
        if (j < R.Q) acc += R.Ainv[i * kMaxQ + j] * f[j];
      rhs[i * g.ld + e] = acc;
    }
  }
}

struct UpdateParams { int Q; double bw[kMaxQ]; double tau; };

__global__ void update_kernel(GridInfo g, const UpdateParams U, const double* __restrict__ kst, double* __restrict__ y) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.n; e += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < U.Q; ++i) acc += U.bw[i] * kst[i * g.ld + e];
    y[e] += U.tau * acc;
  }
}

__global__ void interpolate_kernel(GridInfo g, const double* __restrict__ x1d, double ct, double* __restrict__ y) {
  const double pi = 3.14159265358979323846;
  const int n = (int)g.n;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    int ix, iy, iz;
    coords(e, g.dim, g.n1, ix, iy, iz);
    if (!interior(g.dim, g.n1, ix, iy, iz)) { y[e] = 0.0; continue; }
    double v = sin(pi * x1d[ix]) * sin(pi * x1d[iy]);
    if (g.dim == 3) v *= sin(pi * x1d[iz]);
    y[e] = v * ct;
  }
}

// ------------------------------------------------------------ reductions
template <int G>
__global__ void multidot_kernel(const double* __restrict__ V, long long vstride, int nv, const double* __restrict__ w,
                                long long n, double* __restrict__ partial, int nb) {
  const int i0 = blockIdx.y * G;
  double acc[G];
#pragma unroll
  for (int g = 0; g < G; ++g) acc[g] = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double we = w[e];
#pragma unroll
    for (int g = 0; g < G; ++g)
      if (i0 + g < nv) acc[g] += V[(i0 + g) * vstride + e] * we;
  }
  __shared__ double red[G][kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int g = 0; g < G; ++g) {
    double v = acc[g];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[g][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < G && i0 + (int)threadIdx.x < nv) {
    double v = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) v += red[threadIdx.x][q];
    partial[(long long)(i0 + threadIdx.x) * nb + blockIdx.x] = v;
  }
}

// Fused Gram-Schmidt kernels (see kernels.h).  Each block reduces its partial sums in a fixed order.
// Basis vectors are taken in groups of 8 (blockIdx.y); the last group also reduces |w|^2 into row nv.
template <int MODE>  // 0: dots of w_in;  1: w_out = w_in - V h, then dots of w_out
__global__ void __launch_bounds__(kThreads) gs_kernel(const double* __restrict__ V, long long vstride, int nv,
                                                      const double* __restrict__ h, const double* __restrict__ w_in,
                                                      double* __restrict__ w_out, int n, double* __restrict__ partial,
                                                      int nb) {
  constexpr int G = 8;
  const int i0 = blockIdx.y * G;
  const bool last = (i0 + G >= nv);
  __shared__ double hs[64];
  if (MODE == 1) {
    for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = h[i];
    __syncthreads();
  }
  double acc[G + 1];
#pragma unroll
  for (int g = 0; g <= G; ++g) acc[g] = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    double we = w_in[e];
    if (MODE == 1) {
      for (int i = 0; i < nv; ++i) we -= hs[i] * V[i * vstride + e];
      if (blockIdx.y == 0) w_out[e] = we;
    }
#pragma unroll
    for (int g = 0; g < G; ++g)
      if (i0 + g < nv) acc[g] += V[(i0 + g) * vstride + e] * we;
    acc[G] += we * we;
  }
  const int cnt = min(G, nv - i0);
  __shared__ double sred[G + 1][kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int g = 0; g <= G; ++g) {
    double v = acc[g];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) sred[g][warp] = v;
  }
  __syncthreads();
  if ((int)threadIdx.x <= G) {
    const int g = threadIdx.x;
    double v = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) v += sred[g][q];
    if (g < cnt) partial[(long long)(i0 + g) * nb + blockIdx.x] = v;
    if (g == G && last) partial[(long long)nv * nb + blockIdx.x] = v;
  }
}

// w_out = w_in - V h when the first pass cancelled more than 1 - eta of |w| ("twice is enough"),
// else w_out = w_in; partial = |w_out|^2 per block.
__global__ void __launch_bounds__(kThreads) gs_reorth_kernel(const double* __restrict__ V, long long vstride, int nv,
                                                             const double* __restrict__ h,
                                                             const double* __restrict__ w_in,
                                                             double* __restrict__ w_out, int n,
                                                             const double* __restrict__ norm2_in,
                                                             const double* __restrict__ norm2_mid, double eta,
                                                             double* __restrict__ partial) {
  const bool redo = norm2_mid[0] < eta * eta * norm2_in[0];
  __shared__ double hs[64];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = redo ? h[i] : 0.0;
  __syncthreads();
  double acc = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    double we = w_in[e];
    if (redo)
      for (int i = 0; i < nv; ++i) we -= hs[i] * V[i * vstride + e];
    w_out[e] = we;
    acc += we * we;
  }
  __shared__ double red[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) v += red[q];
    partial[blockIdx.x] = v;
  }
}

// Basis sizes up to 16: fully unrolled, one pass over the basis per kernel; in MODE 1 the
// basis values loaded for the update are reused for the dot products.
template <int MODE, int NV>
__global__ void __launch_bounds__(kThreads) gs_small_kernel(const double* __restrict__ V, long long vstride,
                                                            const double* __restrict__ h,
                                                            const double* __restrict__ w_in,
                                                            double* __restrict__ w_out, int n,
                                                            double* __restrict__ partial, int nb) {
  double hr[NV];
  if (MODE == 1) {
#pragma unroll
    for (int i = 0; i < NV; ++i) hr[i] = h[i];
  }
  double acc[NV + 1];
#pragma unroll
  for (int i = 0; i <= NV; ++i) acc[i] = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    double vv[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) vv[i] = V[i * vstride + e];
    double we = w_in[e];
    if (MODE == 1) {
#pragma unroll
      for (int i = 0; i < NV; ++i) we -= hr[i] * vv[i];
      w_out[e] = we;
    }
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] += vv[i] * we;
    acc[NV] += we * we;
  }
  __shared__ double sred[NV + 1][kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int g = 0; g <= NV; ++g) {
    double x = acc[g];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    if (lane == 0) sred[g][warp] = x;
  }
  __syncthreads();
  if ((int)threadIdx.x <= NV) {
    double x = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) x += sred[threadIdx.x][q];
    partial[(long long)threadIdx.x * nb + blockIdx.x] = x;
  }
}

template <int NV>
__global__ void __launch_bounds__(kThreads) gs_reorth_small_kernel(const double* __restrict__ V, long long vstride,
                                                                   const double* __restrict__ h,
                                                                   const double* __restrict__ w_in,
                                                                   double* __restrict__ w_out, int n,
                                                                   const double* __restrict__ norm2_in,
                                                                   const double* __restrict__ norm2_mid, double eta,
                                                                   double* __restrict__ partial) {
  const bool redo = norm2_mid[0] < eta * eta * norm2_in[0];
  double hr[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) hr[i] = redo ? h[i] : 0.0;
  double acc = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    double we = w_in[e];
    if (redo) {
#pragma unroll
      for (int i = 0; i < NV; ++i) we -= hr[i] * V[i * vstride + e];
    }
    w_out[e] = we;
    acc += we * we;
  }
  __shared__ double red[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) x += red[q];
    partial[blockIdx.x] = x;
  }
}

__global__ void __launch_bounds__(kThreads) block_dot_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                                             int n, long long ld, double* __restrict__ partial) {
  const int s = blockIdx.y;
  const double* as = a + s * ld;
  const double* bs = b + s * ld;
  double acc = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) acc += as[e] * bs[e];
  __shared__ double red[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) x += red[q];
    partial[(long long)s * gridDim.x + blockIdx.x] = x;
  }
}

__global__ void block_axpy2_kernel(double* __restrict__ w, const double* __restrict__ v1, const double* __restrict__ v0,
                                   const double* __restrict__ alpha, const double* __restrict__ beta, int n,
                                   long long ld) {
  const int s = blockIdx.y;
  const double a = alpha[s], bt = beta[s];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const long long o = s * ld + e;
    w[o] -= a * v1[o] + bt * v0[o];
  }
}

__global__ void block_shift_kernel(double* __restrict__ v0, double* __restrict__ v1, const double* __restrict__ w,
                                   const double* __restrict__ nrm, int n, long long ld) {
  const int s = blockIdx.y;
  const double f = (nrm[s] > 0.0) ? 1.0 / nrm[s] : 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const long long o = s * ld + e;
    if (v0) v0[o] = v1[o];
    v1[o] = w[o] * f;
  }
}

__global__ void norm2_kernel(const double* __restrict__ w, long long n, double* __restrict__ partial) {
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double v = w[e];
    acc += v * v;
  }
  __shared__ double red[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) v += red[q];
    partial[blockIdx.x] = v;
  }
}

__global__ void reduce_partials_kernel(const double* __restrict__ partial, int nb, double* __restrict__ out,
                                       int take_sqrt) {
  const int i = blockIdx.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += partial[(long long)i * nb + b];
  __shared__ double red[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) v += red[q];
    out[i] = take_sqrt ? sqrt(v) : v;
  }
}

__global__ void multi_axpy_kernel(const double* __restrict__ V, long long vstride, int nv, const double* __restrict__ h,
                                  double sign, double* __restrict__ w, long long n) {
  __shared__ double hs[64];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = sign * h[i];
  __syncthreads();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    double acc = w[e];
    for (int i = 0; i < nv; ++i) acc += hs[i] * V[i * vstride + e];
    w[e] = acc;
  }
}

__global__ void scale_inv_kernel(const double* __restrict__ w, const double* __restrict__ nrm, double* __restrict__ out,
                                 long long n) {
  const double f = 1.0 / nrm[0];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    out[e] = w[e] * f;
}

__global__ void scale_kernel(const double* __restrict__ x, double a, double* __restrict__ out, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    out[e] = a * x[e];
}

// ------------------------------------------------------------ transfers
// One 1D pass of the Q_k nodal embedding P (restriction applies P^T) along AXIS, one thread per
// coarse cell of a grid line.  On a coarse cell cc the fine nodes 2Kcc + m (m = 0..2K) take
// sum_i Pc[m][i] u_c(Kcc + i) (i = 0..K); the coarse vertex Kcc collects from the fine nodes of
// both cells that share it.  K and AXIS are compile-time, so every Pc coefficient is a uniform
// constant operand and each thread's loads along the line are unrolled.
template <typename T, int K, int AXIS>
struct LineMap {
  // thread t -> (coarse cell cc, line bases in and out, stride along the axis in and out)
  __device__ __forceinline__ static void map(int t, int Nc, int din0, int din1, int dout0, int dout1, int& cc,
                                              long long& bin, long long& bout, int& sin_, int& sout) {
    if (AXIS == 0) {
      cc = t % Nc;
      const int r = t / Nc;  // row (o1, o2), the same in both arrays
      bin = (long long)r * din0;
      bout = (long long)r * dout0;
      sin_ = sout = 1;
    } else if (AXIS == 1) {
      const int o0 = t % din0;  // din0 == dout0
      const int t2 = t / din0;
      cc = t2 % Nc;
      const int o2 = t2 / Nc;
      bin = o0 + (long long)o2 * din0 * din1;
      bout = o0 + (long long)o2 * dout0 * dout1;
      sin_ = sout = din0;
    } else {
      const int plane = din0 * din1;  // == dout0 * dout1
      const int pidx = t % plane;
      cc = t / plane;
      bin = bout = pidx;
      sin_ = sout = plane;
    }
  }
};

template <typename T, int K, int AXIS, bool RESTRICT>
__global__ void __launch_bounds__(kThreads) transfer_cell_kernel(const T* __restrict__ in, T* __restrict__ out,
                                                                 long long ld_in, long long ld_out, int din0, int din1,
                                                                 int dout0, int dout1, int nthreads, int accumulate,
                                                                 const TransferParams P) {
  constexpr int KP = K + 1;
  const int s = blockIdx.y;
  const int Nc = P.Nc;
  const T* __restrict__ src0 = in + s * ld_in;
  T* __restrict__ dst0 = out + s * ld_out;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nthreads; t += gridDim.x * blockDim.x) {
    int cc, si, so;
    long long bi, bo;
    LineMap<T, K, AXIS>::map(t, Nc, din0, din1, dout0, dout1, cc, bi, bo, si, so);
    const T* src = src0 + bi;
    T* dst = dst0 + bo;
    // arithmetic in the element type (FP32 for the FP32 multigrid)
#define IRK_PC(m, i) ((sizeof(T) == 4) ? (T)P.Pcf[(m) * KP + (i)] : (T)P.Pc[(m) * KP + (i)])
    if (RESTRICT) {
      T f[4 * K + 1];  // fine nodes 2K(cc-1) .. 2K(cc+1); the first 2K only for the vertex, cc > 0
#pragma unroll
      for (int j = 0; j < 2 * K; ++j) f[j] = (cc > 0) ? src[(long long)(2 * K * (cc - 1) + j) * si] : T(0);
#pragma unroll
      for (int j = 2 * K; j <= 4 * K; ++j) f[j] = src[(long long)(2 * K * (cc - 1) + j) * si];
      T r[K];
      {
        T acc = T(0);
        if (cc > 0) {
#pragma unroll
          for (int m = 0; m < 2 * K; ++m) acc += IRK_PC(m, K) * f[m];
#pragma unroll
          for (int m = 0; m <= 2 * K; ++m) acc += IRK_PC(m, 0) * f[2 * K + m];
        }
        r[0] = acc;  // coarse boundary node 0 stays zero
      }
#pragma unroll
      for (int i = 1; i < K; ++i) {
        T acc = T(0);
#pragma unroll
        for (int m = 0; m <= 2 * K; ++m) acc += IRK_PC(m, i) * f[2 * K + m];
        r[i] = acc;
      }
#pragma unroll
      for (int i = 0; i < K; ++i) {
        T* d = dst + (long long)(K * cc + i) * so;
        if (accumulate) *d += r[i];
        else *d = r[i];
      }
      if (cc == Nc - 1 && !accumulate) dst[(long long)(K * Nc) * so] = T(0);  // coarse boundary node
    } else {
      T c[KP];
#pragma unroll
      for (int i = 0; i <= K; ++i) c[i] = src[(long long)(K * cc + i) * si];
      const int mend = (cc == Nc - 1) ? 2 * K : 2 * K - 1;  // the last cell also owns the end node
#pragma unroll
      for (int m = 0; m <= 2 * K; ++m) {
        if (m > mend) break;
        T acc = T(0);
#pragma unroll
        for (int i = 0; i <= K; ++i) acc += IRK_PC(m, i) * c[i];
        T* d = dst + (long long)(2 * K * cc + m) * so;
        if (accumulate) *d += acc;
        else *d = acc;
      }
    }
#undef IRK_PC
  }
}

// ------------------------------------------------------------ coarse solve
template <typename T>
__global__ void coarse_solve_kernel(const T* __restrict__ b, T* __restrict__ x, long long ld,
                                    const double* __restrict__ Ainv, const int* __restrict__ map, int nci) {
  extern __shared__ double sb[];
  const int s = blockIdx.x;
  for (int i = threadIdx.x; i < nci; i += blockDim.x) sb[i] = (double)b[s * ld + map[i]];
  __syncthreads();
  const double* A = Ainv + (long long)s * nci * nci;
  for (int r = threadIdx.x; r < nci; r += blockDim.x) {
    double acc = 0.0;
    for (int c = 0; c < nci; ++c) acc += A[(long long)r * nci + c] * sb[c];
    x[s * ld + map[r]] = (T)acc;
  }
}

// ------------------------------------------------------------ fast-diagonalisation coarse solve
template <typename Tin, typename Tout>
__global__ void fd_axis_kernel(const Tin* __restrict__ in, Tout* __restrict__ out, long long ld, int n1, int dim,
                               int axis, const double* __restrict__ Mt, int ni) {
  const int s = blockIdx.y;
  const int total = (dim == 3) ? ni * ni * ni : ni * ni;
  const int stride[3] = {1, n1, n1 * n1};
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    int a[3];
    a[0] = e % ni;
    a[1] = (e / ni) % ni;
    a[2] = (dim == 3) ? e / (ni * ni) : 0;
    int base = 0;
    for (int d = 0; d < dim; ++d)
      if (d != axis) base += (a[d] + 1) * stride[d];
    const int i = a[axis];
    const Tin* src = in + s * ld + base + stride[axis];
    double acc = 0.0;
    for (int j = 0; j < ni; ++j) acc += Mt[i * ni + j] * (double)src[j * stride[axis]];
    out[s * ld + base + (i + 1) * stride[axis]] = (Tout)acc;
  }
}

__global__ void fd_scale_kernel(double* __restrict__ t, long long ld, int n1, int dim, const double* __restrict__ mu,
                                const FdParams P) {
  const int s = blockIdx.y;
  const int ni = P.ni;
  const int total = (dim == 3) ? ni * ni * ni : ni * ni;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int a0 = e % ni, a1 = (e / ni) % ni, a2 = (dim == 3) ? e / (ni * ni) : 0;
    double m = mu[a0] + mu[a1];
    int idx = (a0 + 1) + (a1 + 1) * n1;
    if (dim == 3) { m += mu[a2]; idx += (a2 + 1) * n1 * n1; }
    t[s * ld + idx] /= (P.cm[s] + P.tau * m);
  }
}

}  // namespace

// ============================================================ launchers
template <typename Tin, typename Tout>
cudaError_t launch_combine(const Tin* a, const double* b, Tout* out, long long n, long long ld, const CombineParams& C,
                           cudaStream_t st) {
  const int nmax = std::max(C.nout, std::max(C.nina, C.ninb));
  const int grid = blocks_for(n, 2);
  CombineParams Cz = C;
  for (int i = 0; i < kMaxQ; ++i) {
    Cz.nza[i] = Cz.nzb[i] = 0u;
    for (int j = 0; j < kMaxQ; ++j) {
      if (i < C.nout && j < C.nina && C.Da[i * kMaxQ + j] != 0.0) Cz.nza[i] |= 1u << j;
      if (i < C.nout && j < C.ninb && C.Db[i * kMaxQ + j] != 0.0) Cz.nzb[i] |= 1u << j;
    }
  }
  // structure detection: unit lower triangular Da (no Db), or full Da with diagonal Db
  bool unit_lower = (C.ninb == 0 && C.nina == C.nout);
  bool diag_b = (C.ninb == C.nout && C.nina == C.nout && b != nullptr);
  for (int i = 0; i < C.nout; ++i)
    for (int j = 0; j < C.nina; ++j) {
      const double d = C.Da[i * kMaxQ + j];
      if ((j > i && d != 0.0) || (j == i && d != 1.0)) unit_lower = false;
      if (j != i && j < C.ninb && C.Db[i * kMaxQ + j] != 0.0) diag_b = false;
    }
  const int q = C.nout;
#define IRK_CS(QQ, CSV) combine_struct_kernel<Tin, Tout, QQ, CSV><<<grid, kThreads, 0, st>>>(a, b, out, (int)n, ld, Cz)
#define IRK_CS_Q(CSV)                         \
  switch (q) {                                \
    case 1: IRK_CS(1, CSV); break;            \
    case 2: IRK_CS(2, CSV); break;            \
    case 3: IRK_CS(3, CSV); break;            \
    case 4: IRK_CS(4, CSV); break;            \
    case 5: IRK_CS(5, CSV); break;            \
    default: break;                           \
  }
  if (q <= 5 && unit_lower) {
    IRK_CS_Q(CS_UNIT_LOWER);
    return cudaGetLastError();
  }
  if (q <= 5 && diag_b) {
    IRK_CS_Q(CS_FULL_DIAGB);
    return cudaGetLastError();
  }
#undef IRK_CS_Q
#undef IRK_CS
  if (nmax <= 1) combine_kernel<Tin, Tout, 1><<<grid, kThreads, 0, st>>>(a, b, out, (int)n, ld, Cz);
  else if (nmax <= 2) combine_kernel<Tin, Tout, 2><<<grid, kThreads, 0, st>>>(a, b, out, (int)n, ld, Cz);
  else if (nmax <= 3) combine_kernel<Tin, Tout, 3><<<grid, kThreads, 0, st>>>(a, b, out, (int)n, ld, Cz);
  else if (nmax <= 5) combine_kernel<Tin, Tout, 5><<<grid, kThreads, 0, st>>>(a, b, out, (int)n, ld, Cz);
  else combine_kernel<Tin, Tout, kMaxQ><<<grid, kThreads, 0, st>>>(a, b, out, (int)n, ld, Cz);
  return cudaGetLastError();
}
template cudaError_t launch_combine<double, double>(const double*, const double*, double*, long long, long long,
                                                    const CombineParams&, cudaStream_t);
template cudaError_t launch_combine<double, float>(const double*, const double*, float*, long long, long long,
                                                   const CombineParams&, cudaStream_t);
template cudaError_t launch_combine<float, double>(const float*, const double*, double*, long long, long long,
                                                   const CombineParams&, cudaStream_t);

template <typename T>
cudaError_t launch_cheb_first(const GridInfo& g, int nstage, const T* b, T* x, const DiagParams<T>& D, cudaStream_t st) {
  dim3 grid(blocks_for(g.n, 2), nstage);
  cheb_first_kernel<T><<<grid, kThreads, 0, st>>>(g, b, x, D);
  return cudaGetLastError();
}
template cudaError_t launch_cheb_first<float>(const GridInfo&, int, const float*, float*, const DiagParams<float>&,
                                              cudaStream_t);
template cudaError_t launch_cheb_first<double>(const GridInfo&, int, const double*, double*, const DiagParams<double>&,
                                               cudaStream_t);

template <typename T>
cudaError_t launch_diag_scale(const GridInfo& g, int nstage, const T* x, T* out, const DiagParams<T>& D, int inv_sqrt,
                              cudaStream_t st) {
  dim3 grid(blocks_for(g.n, 2), nstage);
  diag_scale_kernel<T><<<grid, kThreads, 0, st>>>(g, x, out, D, inv_sqrt);
  return cudaGetLastError();
}
template cudaError_t launch_diag_scale<float>(const GridInfo&, int, const float*, float*, const DiagParams<float>&, int,
                                              cudaStream_t);
template cudaError_t launch_diag_scale<double>(const GridInfo&, int, const double*, double*, const DiagParams<double>&,
                                               int, cudaStream_t);

cudaError_t launch_hash_fill(const GridInfo& g, int nstage, double* x, cudaStream_t st) {
  dim3 grid(blocks_for(g.n, 2), nstage);
  hash_fill_kernel<<<grid, kThreads, 0, st>>>(g, x);
  return cudaGetLastError();
}

cudaError_t launch_stage_rhs(const GridInfo& g, const RhsParams& R, const double* Ky, const double* G1,
                             const double* loads, double* rhs, cudaStream_t st) {
  stage_rhs_kernel<<<blocks_for(g.n, 2), kThreads, 0, st>>>(g, R, Ky, G1, loads, rhs);
  return cudaGetLastError();
}

cudaError_t launch_update(const GridInfo& g, int Q, const double* kst, const double* bw, double tau, double* y,
                          cudaStream_t st) {
  UpdateParams U;
  U.Q = Q;
  for (int i = 0; i < kMaxQ; ++i) U.bw[i] = (i < Q) ? bw[i] : 0.0;
  U.tau = tau;
  update_kernel<<<blocks_for(g.n, 2), kThreads, 0, st>>>(g, U, kst, y);
  return cudaGetLastError();
}

cudaError_t launch_interpolate(const GridInfo& g, const double* x1d, double ct, double* y, cudaStream_t st) {
  interpolate_kernel<<<blocks_for(g.n, 2), kThreads, 0, st>>>(g, x1d, ct, y);
  return cudaGetLastError();
}

int reduction_blocks(long long n) { return blocks_for(n, 8); }

cudaError_t launch_multidot(const double* V, long long vstride, int nv, const double* w, long long n, double* partial,
                            int nb, cudaStream_t st) {
  dim3 grid(nb, (nv + 7) / 8);
  multidot_kernel<8><<<grid, kThreads, 0, st>>>(V, vstride, nv, w, n, partial, nb);
  return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const double* partial, int nv, int nb, double* out, cudaStream_t st,
                                   int take_sqrt) {
  reduce_partials_kernel<<<nv, kThreads, 0, st>>>(partial, nb, out, take_sqrt);
  return cudaGetLastError();
}

#define IRK_GSC(MODE, NVV, ...) \
  case NVV: gs_small_kernel<MODE, NVV><<<nb, kThreads, 0, st>>>(__VA_ARGS__); break;
#define IRK_GS_SMALL(MODE, ...)                                                                            \
  switch (nv) {                                                                                           \
    IRK_GSC(MODE, 1, __VA_ARGS__) IRK_GSC(MODE, 2, __VA_ARGS__) IRK_GSC(MODE, 3, __VA_ARGS__)            \
    IRK_GSC(MODE, 4, __VA_ARGS__) IRK_GSC(MODE, 5, __VA_ARGS__) IRK_GSC(MODE, 6, __VA_ARGS__)            \
    IRK_GSC(MODE, 7, __VA_ARGS__) IRK_GSC(MODE, 8, __VA_ARGS__) IRK_GSC(MODE, 9, __VA_ARGS__)            \
    IRK_GSC(MODE, 10, __VA_ARGS__) IRK_GSC(MODE, 11, __VA_ARGS__) IRK_GSC(MODE, 12, __VA_ARGS__)         \
    IRK_GSC(MODE, 13, __VA_ARGS__) IRK_GSC(MODE, 14, __VA_ARGS__) IRK_GSC(MODE, 15, __VA_ARGS__)         \
    default: gs_small_kernel<MODE, 16><<<nb, kThreads, 0, st>>>(__VA_ARGS__); break;                      \
  }

cudaError_t launch_gs_dot(const double* V, long long vstride, int nv, const double* w, long long n, double* partial,
                          int nb, cudaStream_t st) {
  if (nv > 64) return cudaErrorInvalidValue;
  if (nv <= 16) {
    IRK_GS_SMALL(0, V, vstride, nullptr, w, nullptr, (int)n, partial, nb);
    return cudaGetLastError();
  }
  dim3 grid(nb, (nv + 7) / 8);
  gs_kernel<0><<<grid, kThreads, 0, st>>>(V, vstride, nv, nullptr, w, nullptr, (int)n, partial, nb);
  return cudaGetLastError();
}

cudaError_t launch_gs_axpy_dot(const double* V, long long vstride, int nv, const double* h, const double* w_in,
                               double* w_out, long long n, double* partial, int nb, cudaStream_t st) {
  if (nv > 64 || w_in == w_out) return cudaErrorInvalidValue;
  if (nv <= 16) {
    IRK_GS_SMALL(1, V, vstride, h, w_in, w_out, (int)n, partial, nb);
    return cudaGetLastError();
  }
  // group 0 writes w_out; the other groups recompute it for their dots
  dim3 grid(nb, (nv + 7) / 8);
  gs_kernel<1><<<grid, kThreads, 0, st>>>(V, vstride, nv, h, w_in, w_out, (int)n, partial, nb);
  return cudaGetLastError();
}

cudaError_t launch_gs_reorth(const double* V, long long vstride, int nv, const double* h, const double* w_in,
                             double* w_out, long long n, const double* norm2_in, const double* norm2_mid, double eta,
                             double* partial, int nb, cudaStream_t st) {
  if (nv > 64) return cudaErrorInvalidValue;
  switch (nv) {
#define IRK_GSR(NVV)                                                                                          \
  case NVV:                                                                                                   \
    gs_reorth_small_kernel<NVV><<<nb, kThreads, 0, st>>>(V, vstride, h, w_in, w_out, (int)n, norm2_in, norm2_mid, \
                                                         eta, partial);                                       \
    return cudaGetLastError();
    IRK_GSR(1) IRK_GSR(2) IRK_GSR(3) IRK_GSR(4) IRK_GSR(5) IRK_GSR(6) IRK_GSR(7) IRK_GSR(8)
    IRK_GSR(9) IRK_GSR(10) IRK_GSR(11) IRK_GSR(12) IRK_GSR(13) IRK_GSR(14) IRK_GSR(15) IRK_GSR(16)
#undef IRK_GSR
    default: break;
  }
  gs_reorth_kernel<<<nb, kThreads, 0, st>>>(V, vstride, nv, h, w_in, w_out, (int)n, norm2_in, norm2_mid, eta, partial);
  return cudaGetLastError();
}

cudaError_t launch_block_dot(const double* a, const double* b, int ns, long long n, long long ld, double* partial,
                             int nb, cudaStream_t st) {
  dim3 grid(nb, ns);
  block_dot_kernel<<<grid, kThreads, 0, st>>>(a, b, (int)n, ld, partial);
  return cudaGetLastError();
}

cudaError_t launch_block_axpy2(double* w, const double* v1, const double* v0, const double* alpha, const double* beta,
                               int ns, long long n, long long ld, cudaStream_t st) {
  dim3 grid(blocks_for(n, 2), ns);
  block_axpy2_kernel<<<grid, kThreads, 0, st>>>(w, v1, v0, alpha, beta, (int)n, ld);
  return cudaGetLastError();
}

cudaError_t launch_block_shift(double* v0, double* v1, const double* w, const double* nrm, int ns, long long n,
                               long long ld, cudaStream_t st) {
  dim3 grid(blocks_for(n, 2), ns);
  block_shift_kernel<<<grid, kThreads, 0, st>>>(v0, v1, w, nrm, (int)n, ld);
  return cudaGetLastError();
}

cudaError_t launch_norm2_partial(const double* w, long long n, double* partial, int nb, cudaStream_t st) {
  norm2_kernel<<<nb, kThreads, 0, st>>>(w, n, partial);
  return cudaGetLastError();
}

cudaError_t launch_multi_axpy(const double* V, long long vstride, int nv, const double* h, double sign, double* w,
                              long long n, cudaStream_t st) {
  if (nv > 64) return cudaErrorInvalidValue;
  multi_axpy_kernel<<<blocks_for(n, 2), kThreads, 0, st>>>(V, vstride, nv, h, sign, w, n);
  return cudaGetLastError();
}

cudaError_t launch_scale_inv(const double* w, const double* nrm, double* out, long long n, cudaStream_t st) {
  scale_inv_kernel<<<blocks_for(n, 2), kThreads, 0, st>>>(w, nrm, out, n);
  return cudaGetLastError();
}

cudaError_t launch_scale(const double* x, double a, double* out, long long n, cudaStream_t st) {
  scale_kernel<<<blocks_for(n, 2), kThreads, 0, st>>>(x, a, out, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_transfer_axis(const T* in, T* out, int nstage, long long ld_in, long long ld_out, const int din[3],
                                 const int dout[3], int axis, int restrict_mode, int accumulate,
                                 const TransferParams& P, cudaStream_t st) {
  if (P.k < 1 || P.k > kMaxDeg || axis < 0 || axis > 2) return cudaErrorInvalidValue;
  // threads: one per coarse cell of every grid line along `axis`
  const long long others = (long long)dout[0] * dout[1] * dout[2] / (axis == 0 ? dout[0] : axis == 1 ? dout[1] : dout[2]);
  const long long nthreads = others * P.Nc;
  if (nthreads <= 0) return cudaSuccess;
  if (nthreads > INT32_MAX) return cudaErrorInvalidValue;
  dim3 grid(blocks_for(nthreads), nstage);
#define IRK_TR(KK, AX, R)                                                                                  \
  transfer_cell_kernel<T, KK, AX, R><<<grid, kThreads, 0, st>>>(in, out, ld_in, ld_out, din[0], din[1], dout[0], \
                                                                dout[1], (int)nthreads, accumulate, P)
#define IRK_TR_AX(KK)                                                          \
  if (restrict_mode) {                                                         \
    if (axis == 0) IRK_TR(KK, 0, true);                                        \
    else if (axis == 1) IRK_TR(KK, 1, true);                                   \
    else IRK_TR(KK, 2, true);                                                  \
  } else {                                                                     \
    if (axis == 0) IRK_TR(KK, 0, false);                                       \
    else if (axis == 1) IRK_TR(KK, 1, false);                                  \
    else IRK_TR(KK, 2, false);                                                 \
  }
  switch (P.k) {
    case 1: IRK_TR_AX(1); break;
    case 2: IRK_TR_AX(2); break;
    case 3: IRK_TR_AX(3); break;
    default: IRK_TR_AX(4); break;
  }
#undef IRK_TR_AX
#undef IRK_TR
  return cudaGetLastError();
}
template cudaError_t launch_transfer_axis<float>(const float*, float*, int, long long, long long, const int[3],
                                                 const int[3], int, int, int, const TransferParams&, cudaStream_t);
template cudaError_t launch_transfer_axis<double>(const double*, double*, int, long long, long long, const int[3],
                                                  const int[3], int, int, int, const TransferParams&, cudaStream_t);

template <typename Tin, typename Tout>
cudaError_t launch_fd_axis(const Tin* in, Tout* out, int nstage, long long ld, int n1, int dim, int axis,
                           const double* Mt, int ni, cudaStream_t st) {
  const long long total = (dim == 3) ? (long long)ni * ni * ni : (long long)ni * ni;
  dim3 grid(blocks_for(total), nstage);
  fd_axis_kernel<Tin, Tout><<<grid, kThreads, 0, st>>>(in, out, ld, n1, dim, axis, Mt, ni);
  return cudaGetLastError();
}
template cudaError_t launch_fd_axis<float, double>(const float*, double*, int, long long, int, int, int,
                                                   const double*, int, cudaStream_t);
template cudaError_t launch_fd_axis<double, double>(const double*, double*, int, long long, int, int, int,
                                                    const double*, int, cudaStream_t);
template cudaError_t launch_fd_axis<double, float>(const double*, float*, int, long long, int, int, int,
                                                   const double*, int, cudaStream_t);

cudaError_t launch_fd_scale(double* t, int nstage, long long ld, int n1, int dim, const double* mu, const FdParams& P,
                            cudaStream_t st) {
  const long long total = (dim == 3) ? (long long)P.ni * P.ni * P.ni : (long long)P.ni * P.ni;
  dim3 grid(blocks_for(total), nstage);
  fd_scale_kernel<<<grid, kThreads, 0, st>>>(t, ld, n1, dim, mu, P);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarse_solve(const T* b, T* x, int nstage, long long ld, const double* Ainv, const int* map, int nci,
                                cudaStream_t st) {
  const size_t smem = (size_t)nci * sizeof(double);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  static size_t granted = 48 * 1024;  // opt-in dynamic shared memory, raised once when needed
  if (smem > granted) {
    cudaError_t e = cudaFuncSetAttribute(coarse_solve_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    granted = smem;
  }
  coarse_solve_kernel<T><<<nstage, kThreads, smem, st>>>(b, x, ld, Ainv, map, nci);
  return cudaGetLastError();
}
template cudaError_t launch_coarse_solve<float>(const float*, float*, int, long long, const double*, const int*, int,
                                                cudaStream_t);
template cudaError_t launch_coarse_solve<double>(const double*, double*, int, long long, const double*, const int*, int,
                                                 cudaStream_t);

}  // namespace irk
