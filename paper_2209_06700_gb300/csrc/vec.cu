// Multigrid-side pointwise, reduction, transfer and coarse-solve kernels of libirk (sm_103a).
//
// * Chebyshev start and diagonal scalings of the level operators (Sec. 5 smoother), the
//   deterministic Lanczos helpers of the Chebyshev-interval estimate.
// * Initial interpolant of the manufactured solution.
// * Intergrid transfer: the Q_k embedding P = P1 (x) P1 (x) P1 and its transpose,
//   applied one axis at a time.
// * Dense coarse-grid solve with a precomputed FP64 inverse, and the exact coarse solve by
//   fast diagonalisation.
#include <algorithm>
#include <cstdint>

#include "ffmath.cuh"
#include "kernels.h"
#include "pdl.cuh"

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

// ------------------------------------------------------------ Chebyshev start, diag scaling
// One warp per grid row (y, z) of one block, eight rows per CTA: the row's K values c / diag by
// in-cell x position are formed once per warp, then x = (c / D) b along the row (interior nodes).
template <typename T>
__global__ void cheb_first_kernel(GridInfo g, const T* __restrict__ b, T* __restrict__ x, const DiagParams<T> D) {
  dev::pdl_enter();
  const int s = blockIdx.y;
  const int n1 = g.n1, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nrows = (g.dim == 3) ? n1 * n1 : n1;
  const int r = blockIdx.x * (blockDim.x >> 5) + w;
  if (r >= nrows) return;
  const int iy = (g.dim == 3) ? r % n1 : r, iz = (g.dim == 3) ? r / n1 : 1;
  if (iy < 1 || iy > n1 - 2 || (g.dim == 3 && (iz < 1 || iz > n1 - 2))) return;
  T sc = T(0);  // lane rx < k holds c / diag for in-cell x position rx
  if (lane < g.k) {
    const int rx = lane, ry = iy % g.k, rz = iz % g.k;
    const T mx = D.dmr[rx], kx = D.dkr[rx], my = D.dmr[ry], ky = D.dkr[ry];
    T d;
    if (g.dim == 3) {
      const T mz = D.dmr[rz], kz = D.dkr[rz];
      d = D.cm[s] * (mx * my * mz) + D.ck[s] * (kx * my * mz + mx * ky * mz + mx * my * kz);
    } else {
      d = D.cm[s] * (mx * my) + D.ck[s] * (kx * my + mx * ky);
    }
    sc = D.c[s] / d;
  }
  const long long o = s * g.ld + (long long)r * n1;
  for (int x0 = 1; x0 <= n1 - 2; x0 += 32) {  // uniform trip count: every lane takes part in the shuffle
    const int ix = x0 + lane;
    const T f = __shfl_sync(0xffffffffu, sc, ix % g.k);
    if (ix <= n1 - 2) x[o + ix] = f * b[o + ix];
  }
}

template <typename Tin, typename Tout>
__global__ void diag_scale_kernel(GridInfo g, const Tin* __restrict__ x, Tout* __restrict__ out,
                                  const DiagParams<double> D, int inv_sqrt) {
  dev::pdl_enter();
  const int s = blockIdx.y;
  const int n = (int)g.n;
  // the diagonal factor in FP32 (this scaling only feeds the Chebyshev-interval estimate): the
  // 1D diagonals are converted once per block into shared memory; the product is formed in FP64
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
    const double f = (double)(inv_sqrt ? rsqrtf(d) : d);
    out[o] = dev::convert<Tout>(dev::to_double(x[o]) * f);
  }
}

__global__ void hash_fill_kernel(GridInfo g, double* __restrict__ x) {
  dev::pdl_enter();
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
__global__ void interpolate_kernel(GridInfo g, const double* __restrict__ x1d, double ct, double* __restrict__ y) {
  dev::pdl_enter();
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
  dev::pdl_enter();
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

__global__ void __launch_bounds__(kThreads) block_dot_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                                             int n, long long ld, double* __restrict__ partial) {
  dev::pdl_enter();
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
  dev::pdl_enter();
  const int s = blockIdx.y;
  const double a = alpha[s], bt = beta[s];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const long long o = s * ld + e;
    w[o] -= a * v1[o] + bt * v0[o];
  }
}

__global__ void block_shift_kernel(double* __restrict__ v0, double* __restrict__ v1, const double* __restrict__ w,
                                   const double* __restrict__ nrm, int n, long long ld) {
  dev::pdl_enter();
  const int s = blockIdx.y;
  const double f = (nrm[s] > 0.0) ? 1.0 / nrm[s] : 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const long long o = s * ld + e;
    if (v0) v0[o] = v1[o];
    v1[o] = w[o] * f;
  }
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
  dev::pdl_enter();
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

// x-axis passes (the contiguous axis) by rows: one warp per grid row stages the row in shared
// memory with coalesced loads and writes its outputs consecutively; coefficients from shared
// memory (they differ from lane to lane).  Rows up to row_max<T>() nodes (4 KB per warp).
template <typename T> struct RowMax { static constexpr int value = 4096 / (int)sizeof(T); };
template <typename T, int K, bool RESTRICT>
__global__ void __launch_bounds__(kThreads) transfer_x_rows_kernel(const T* __restrict__ in, T* __restrict__ out,
                                                                   long long ld_in, long long ld_out, int nin,
                                                                   int nout, int rows, int accumulate,
                                                                   const TransferParams P) {
  dev::pdl_enter();
  constexpr int KP = K + 1, NW = kThreads / 32;
  __shared__ T srow[NW][RowMax<T>::value];
  __shared__ T spc[(2 * K + 1) * KP];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < (2 * K + 1) * KP; i += blockDim.x)
    spc[i] = (sizeof(T) == 4) ? (T)P.Pcf[i] : (T)P.Pc[i];
  __syncthreads();
  const int s = blockIdx.y;
  const int row = blockIdx.x * NW + w;
  if (row >= rows) return;
  const T* src = in + s * ld_in + (long long)row * nin;
  T* dst = out + s * ld_out + (long long)row * nout;
  T* f = srow[w];
  for (int j = lane; j < nin; j += 32) f[j] = src[j];
  __syncwarp();
  const int Nc = P.Nc;
  for (int o = lane; o < nout; o += 32) {
    T acc = T(0);
    if (RESTRICT) {  // coarse node o
      if (o > 0 && o < nout - 1) {
        const int cc = o / K, i = o - cc * K;
        if (i != 0) {
#pragma unroll
          for (int m = 0; m <= 2 * K; ++m) acc += spc[m * KP + i] * f[2 * K * cc + m];
        } else {
#pragma unroll
          for (int m = 0; m < 2 * K; ++m) acc += spc[m * KP + K] * f[2 * K * (cc - 1) + m];
#pragma unroll
          for (int m = 0; m <= 2 * K; ++m) acc += spc[m * KP] * f[2 * K * cc + m];
        }
      }
    } else {  // fine node o
      int cc = o / (2 * K);
      if (cc > Nc - 1) cc = Nc - 1;
      const int m = o - 2 * K * cc;
#pragma unroll
      for (int i = 0; i <= K; ++i) acc += spc[m * KP + i] * f[K * cc + i];
    }
    if (accumulate) dst[o] += acc;
    else dst[o] = acc;
  }
}

// ------------------------------------------------------------ coarse solve
template <typename T>
__global__ void coarse_solve_kernel(const T* __restrict__ b, T* __restrict__ x, long long ld,
                                    const double* __restrict__ Ainv, const int* __restrict__ map, int nci) {
  dev::pdl_enter();
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
  dev::pdl_enter();
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
  dev::pdl_enter();
  const int s = blockIdx.y;
  const int ni = P.ni;
  const int total = (dim == 3) ? ni * ni * ni : ni * ni;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int a0 = e % ni, a1 = (e / ni) % ni, a2 = (dim == 3) ? e / (ni * ni) : 0;
    double m = mu[a0] + mu[a1];
    int idx = (a0 + 1) + (a1 + 1) * n1;
    if (dim == 3) { m += mu[a2]; idx += (a2 + 1) * n1 * n1; }
    t[s * ld + idx] /= (P.cm[s] + P.taus[s] * m);
  }
}

__global__ void fd_scale_coupled_kernel(double* __restrict__ t, long long ld, int n1, int dim,
                                        const double* __restrict__ mu, const FdParams P) {
  dev::pdl_enter();
  const int ni = P.ni;
  const int total = (dim == 3) ? ni * ni * ni : ni * ni;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int a0 = e % ni, a1 = (e / ni) % ni, a2 = (dim == 3) ? e / (ni * ni) : 0;
    double m = mu[a0] + mu[a1];
    int idx = (a0 + 1) + (a1 + 1) * n1;
    if (dim == 3) { m += mu[a2]; idx += (a2 + 1) * n1 * n1; }
    const double a = P.cm[0] + P.taus[0] * m, bt = P.beta;
    const double den = a * a + bt * bt;
    const double t0 = t[idx], t1 = t[ld + idx];
    t[idx] = (a * t0 + bt * t1) / den;
    t[ld + idx] = (a * t1 - bt * t0) / den;
  }
}

template <typename T>
__global__ void coupled_update_kernel(GridInfo g, const T* __restrict__ mx, const T* __restrict__ kx,
                                      const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ out,
                                      const CoupledParams C) {
  dev::pdl_enter();
  const int n = (int)g.n;
  const T cm = (T)C.cm, ck = (T)C.ck, beta = (T)C.beta, c1 = (T)C.c1, c2 = (T)C.c2;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    int ix, iy, iz;
    coords(e, g.dim, g.n1, ix, iy, iz);
    if (!interior(g.dim, g.n1, ix, iy, iz)) continue;
    const long long o0 = e, o1 = g.ld + e;
    T r0, r1;
    if (C.cheb == 2) {  // first step from x = 0: the residual is b
      r0 = b[o0];
      r1 = b[o1];
    } else {
      const T m0 = mx[o0], m1 = mx[o1];
      const T a0 = cm * m0 + ck * kx[o0] - beta * m1;
      const T a1 = cm * m1 + ck * kx[o1] + beta * m0;
      r0 = b[o0] - a0;
      r1 = b[o1] - a1;
    }
    if (C.cheb == 0) {
      out[o0] = r0;
      out[o1] = r1;
      continue;
    }
    // nodal 2x2 block of the coupled system: [[d, -beta m], [beta m, d]], d = diag(A), m = diag(M)
    const int rx = ix % g.k, ry = iy % g.k, rz = iz % g.k;
    double md, kd;
    if (g.dim == 3) {
      md = C.dmr[rx] * C.dmr[ry] * C.dmr[rz];
      kd = C.dkr[rx] * C.dmr[ry] * C.dmr[rz] + C.dmr[rx] * C.dkr[ry] * C.dmr[rz] + C.dmr[rx] * C.dmr[ry] * C.dkr[rz];
    } else {
      md = C.dmr[rx] * C.dmr[ry];
      kd = C.dkr[rx] * C.dmr[ry] + C.dmr[rx] * C.dkr[ry];
    }
    const T d = (T)(C.cm * md + C.ck * kd), bm = (T)(C.beta * md);
    const T den = d * d + bm * bm;
    const T z0 = (d * r0 + bm * r1) / den, z1 = (d * r1 - bm * r0) / den;
    if (C.cheb == 2) {
      out[o0] = c2 * z0;
      out[o1] = c2 * z1;
      continue;
    }
    const T x0 = x[o0], x1 = x[o1];
    const T p0 = C.xold_zero ? T(0) : out[o0], p1 = C.xold_zero ? T(0) : out[o1];
    out[o0] = x0 + c1 * (x0 - p0) + c2 * z0;
    out[o1] = x1 + c1 * (x1 - p1) + c2 * z1;
  }
}

}  // namespace

// ============================================================ launchers
template <typename T>
cudaError_t launch_cheb_first(const GridInfo& g, int nstage, const T* b, T* x, const DiagParams<T>& D, cudaStream_t st) {
  const int rows = (g.dim == 3) ? g.n1 * g.n1 : g.n1;
  dim3 grid((rows + 7) / 8, nstage);
  launch_pdl(cheb_first_kernel<T>, grid, 256, 0, st, g, b, x, D);
  return cudaGetLastError();
}
template cudaError_t launch_cheb_first<float>(const GridInfo&, int, const float*, float*, const DiagParams<float>&,
                                              cudaStream_t);
template cudaError_t launch_cheb_first<double>(const GridInfo&, int, const double*, double*, const DiagParams<double>&,
                                               cudaStream_t);

template <typename Tin, typename Tout>
cudaError_t launch_diag_scale(const GridInfo& g, int nstage, const Tin* x, Tout* out, const DiagParams<double>& D,
                              int inv_sqrt, cudaStream_t st) {
  dim3 grid(blocks_for(g.n, 2), nstage);
  launch_pdl(diag_scale_kernel<Tin, Tout>, grid, kThreads, 0, st, g, x, out, D, inv_sqrt);
  return cudaGetLastError();
}
template cudaError_t launch_diag_scale<double, double>(const GridInfo&, int, const double*, double*,
                                                       const DiagParams<double>&, int, cudaStream_t);
template cudaError_t launch_diag_scale<double, ff>(const GridInfo&, int, const double*, ff*, const DiagParams<double>&,
                                                   int, cudaStream_t);
template cudaError_t launch_diag_scale<ff, double>(const GridInfo&, int, const ff*, double*, const DiagParams<double>&,
                                                   int, cudaStream_t);
template cudaError_t launch_diag_scale<double, float>(const GridInfo&, int, const double*, float*,
                                                      const DiagParams<double>&, int, cudaStream_t);
template cudaError_t launch_diag_scale<float, double>(const GridInfo&, int, const float*, double*,
                                                      const DiagParams<double>&, int, cudaStream_t);

cudaError_t launch_hash_fill(const GridInfo& g, int nstage, double* x, cudaStream_t st) {
  dim3 grid(blocks_for(g.n, 2), nstage);
  launch_pdl(hash_fill_kernel, grid, kThreads, 0, st, g, x);
  return cudaGetLastError();
}

cudaError_t launch_interpolate(const GridInfo& g, const double* x1d, double ct, double* y, cudaStream_t st) {
  launch_pdl(interpolate_kernel, blocks_for(g.n, 2), kThreads, 0, st, g, x1d, ct, y);
  return cudaGetLastError();
}

cudaError_t launch_multidot(const double* V, long long vstride, int nv, const double* w, long long n, double* partial,
                            int nb, cudaStream_t st) {
  dim3 grid(nb, (nv + 7) / 8);
  launch_pdl(multidot_kernel<8>, grid, kThreads, 0, st, V, vstride, nv, w, n, partial, nb);
  return cudaGetLastError();
}

cudaError_t launch_block_dot(const double* a, const double* b, int ns, long long n, long long ld, double* partial,
                             int nb, cudaStream_t st) {
  dim3 grid(nb, ns);
  launch_pdl(block_dot_kernel, grid, kThreads, 0, st, a, b, (int)n, ld, partial);
  return cudaGetLastError();
}

cudaError_t launch_block_axpy2(double* w, const double* v1, const double* v0, const double* alpha, const double* beta,
                               int ns, long long n, long long ld, cudaStream_t st) {
  dim3 grid(blocks_for(n, 2), ns);
  launch_pdl(block_axpy2_kernel, grid, kThreads, 0, st, w, v1, v0, alpha, beta, (int)n, ld);
  return cudaGetLastError();
}

cudaError_t launch_block_shift(double* v0, double* v1, const double* w, const double* nrm, int ns, long long n,
                               long long ld, cudaStream_t st) {
  dim3 grid(blocks_for(n, 2), ns);
  launch_pdl(block_shift_kernel, grid, kThreads, 0, st, v0, v1, w, nrm, (int)n, ld);
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
  if (axis == 0 && !restrict_mode && din[0] <= RowMax<T>::value) {  // prolongation rows via shared memory
    const int rows = dout[1] * dout[2];
    dim3 rgrid((rows + kThreads / 32 - 1) / (kThreads / 32), nstage);
#define IRK_TX(KK, R)                                                                                          \
  launch_pdl(transfer_x_rows_kernel<T, KK, R>, rgrid, kThreads, 0, st, in, out, ld_in, ld_out, din[0], dout[0], rows, \
                                                                accumulate, P)
#define IRK_TX_K(KK) \
  if (restrict_mode) IRK_TX(KK, true); else IRK_TX(KK, false);
    switch (P.k) {
      case 1: IRK_TX_K(1); break;
      case 2: IRK_TX_K(2); break;
      case 3: IRK_TX_K(3); break;
      default: IRK_TX_K(4); break;
    }
#undef IRK_TX_K
#undef IRK_TX
    return cudaGetLastError();
  }
  dim3 grid(blocks_for(nthreads), nstage);
#define IRK_TR(KK, AX, R)                                                                                  \
  launch_pdl(transfer_cell_kernel<T, KK, AX, R>, grid, kThreads, 0, st, in, out, ld_in, ld_out, din[0], din[1], dout[0], \
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
  launch_pdl(fd_axis_kernel<Tin, Tout>, grid, kThreads, 0, st, in, out, ld, n1, dim, axis, Mt, ni);
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
  launch_pdl(fd_scale_kernel, grid, kThreads, 0, st, t, ld, n1, dim, mu, P);
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
  launch_pdl(coarse_solve_kernel<T>, nstage, kThreads, smem, st, b, x, ld, Ainv, map, nci);
  return cudaGetLastError();
}
template cudaError_t launch_coarse_solve<float>(const float*, float*, int, long long, const double*, const int*, int,
                                                cudaStream_t);
template cudaError_t launch_coarse_solve<double>(const double*, double*, int, long long, const double*, const int*, int,
                                                 cudaStream_t);

cudaError_t launch_fd_scale_coupled(double* t, long long ld, int n1, int dim, const double* mu, const FdParams& P,
                                    cudaStream_t st) {
  const long long total = (dim == 3) ? (long long)P.ni * P.ni * P.ni : (long long)P.ni * P.ni;
  launch_pdl(fd_scale_coupled_kernel, blocks_for(total), kThreads, 0, st, t, ld, n1, dim, mu, P);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coupled_update(const GridInfo& g, const T* mx, const T* kx, const T* x, const T* b, T* out,
                                  const CoupledParams& C, cudaStream_t st) {
  launch_pdl(coupled_update_kernel<T>, blocks_for(g.n, 2), kThreads, 0, st, g, mx, kx, x, b, out, C);
  return cudaGetLastError();
}
template cudaError_t launch_coupled_update<float>(const GridInfo&, const float*, const float*, const float*,
                                                  const float*, float*, const CoupledParams&, cudaStream_t);
template cudaError_t launch_coupled_update<double>(const GridInfo&, const double*, const double*, const double*,
                                                   const double*, double*, const CoupledParams&, cudaStream_t);

}  // namespace irk
