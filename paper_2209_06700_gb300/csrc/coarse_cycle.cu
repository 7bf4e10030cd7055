// Fused coarse-grid V-cycle of libirk (sm_103a).
//
// The lower levels of the geometric multigrid of Eq. (irk:P)'s blocks (arXiv
// 2209.06700, Sec. 5: one V-cycle per block, Chebyshev/point-Jacobi
// smoother; exact coarse solve here) hold only a few thousand nodes per block,
// where a launch per smoothing step is all latency.  This kernel runs the whole
// sub-cycle from level lc down to the coarsest and back in one launch: one CTA
// per block (blockIdx.x), every vector of every fused level resident in shared
// memory, operator applications by sum factorisation in three axis passes over
// the shared grid, Q_k restriction/prolongation by axis passes, and the dense
// coarse inverse read from global memory.  The arithmetic is the same as the
// level-by-level path (same operator, same Chebyshev recurrence and interval).
#include "coarse_cycle.h"

namespace irk {
namespace {

constexpr int kCT = 512;  // threads per CTA

// 1D banded apply along one axis of an n1-node line: out = sum_taps c * in, for mass (me) and
// stiffness (ke) element matrices; position i on the line, stride between line neighbours.
template <typename T, int K>
__device__ __forceinline__ void band2(const T* src, int i, int n1, int stride, const float (&me)[5][5],
                                      const float (&ke)[5][5], T& om, T& ok) {
  const int r = i % K;
  T am = T(0), ak = T(0);
  if (r != 0) {
    const int base = i - r;
#pragma unroll
    for (int m = 0; m <= K; ++m) {
      const T v = src[(base + m - i) * stride];
      am += (T)me[r][m] * v;
      ak += (T)ke[r][m] * v;
    }
  } else {
#pragma unroll
    for (int o = -K; o <= K; ++o) {
      const int j = i + o;
      if (j < 0 || j >= n1) continue;
      T cm = T(0), ck = T(0);
      if (o >= 0) { cm += (T)me[0][o]; ck += (T)ke[0][o]; }
      if (o <= 0) { cm += (T)me[K][K + o]; ck += (T)ke[K][K + o]; }
      const T v = src[o * stride];
      am += cm * v;
      ak += ck * v;
    }
  }
  om = am;
  ok = ak;
}

template <typename T, int K>
__device__ __forceinline__ T band1(const T* src, int i, int n1, int stride, const float (&me)[5][5]) {
  const int r = i % K;
  T a = T(0);
  if (r != 0) {
    const int base = i - r;
#pragma unroll
    for (int m = 0; m <= K; ++m) a += (T)me[r][m] * src[(base + m - i) * stride];
  } else {
#pragma unroll
    for (int o = -K; o <= K; ++o) {
      const int j = i + o;
      if (j < 0 || j >= n1) continue;
      T c = T(0);
      if (o >= 0) c += (T)me[0][o];
      if (o <= 0) c += (T)me[K][K + o];
      a += c * src[o * stride];
    }
  }
  return a;
}

template <typename T, int DIM>
__device__ __forceinline__ bool interior(int q, int n1, int& ix, int& iy, int& iz) {
  ix = q % n1;
  iy = (q / n1) % n1;
  iz = (DIM == 3) ? q / (n1 * n1) : 1;
  return ix > 0 && ix < n1 - 1 && iy > 0 && iy < n1 - 1 && (DIM == 2 || (iz > 0 && iz < n1 - 1));
}

// A u on one level into t3 (interior nodes; boundary left untouched), with t1, t2 scratch of n nodes.
// 3D: p1 = Mx u, p2 = Kx u; q1 = My p1, q2 = Ky p1 + My p2; A u = Mz (cm q1 + ck q2) + ck Kz q1.
template <typename T, int K, int DIM>
__device__ void apply_level(const CoarseLevel& L, T cm, T ck, const T* u, T* p1, T* p2, T* q1, T* q2, T* out) {
  const int n1 = L.n1, n = L.n;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const int ix = q % n1;
    T a, b;
    band2<T, K>(u + q, ix, n1, 1, L.me, L.ke, a, b);
    p1[q] = a;
    p2[q] = b;
  }
  __syncthreads();
  if constexpr (DIM == 2) {
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      int ix, iy, iz;
      if (!interior<T, 2>(q, n1, ix, iy, iz)) continue;
      T m1, k1;
      band2<T, K>(p1 + q, iy, n1, n1, L.me, L.ke, m1, k1);
      const T m2 = band1<T, K>(p2 + q, iy, n1, n1, L.me);
      out[q] = cm * m1 + ck * (k1 + m2);
    }
    __syncthreads();
    return;
  } else {
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const int iy = (q / n1) % n1;
    T m1, k1;
    band2<T, K>(p1 + q, iy, n1, n1, L.me, L.ke, m1, k1);
    q1[q] = m1;
    q2[q] = k1 + band1<T, K>(p2 + q, iy, n1, n1, L.me);
  }
  __syncthreads();
  const int pl = n1 * n1;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    int ix, iy, iz;
    if (!interior<T, 3>(q, n1, ix, iy, iz)) continue;
    // Mz (cm q1 + ck q2) + ck Kz q1
    const int r = iz % K;
    T acc = T(0);
    if (r != 0) {
      const int base = iz - r;
#pragma unroll
      for (int m = 0; m <= K; ++m) {
        const int o = (base + m - iz) * pl;
        acc += (T)L.me[r][m] * (cm * q1[q + o] + ck * q2[q + o]) + ck * (T)L.ke[r][m] * q1[q + o];
      }
    } else {
#pragma unroll
      for (int o = -K; o <= K; ++o) {
        const int j = iz + o;
        if (j < 0 || j >= n1) continue;
        T cmz = T(0), ckz = T(0);
        if (o >= 0) { cmz += (T)L.me[0][o]; ckz += (T)L.ke[0][o]; }
        if (o <= 0) { cmz += (T)L.me[K][K + o]; ckz += (T)L.ke[K][K + o]; }
        const T a = q1[q + o * pl], b = q2[q + o * pl];
        acc += cmz * (cm * a + ck * b) + ck * ckz * a;
      }
    }
    out[q] = acc;
  }
  __syncthreads();
  }
}

template <typename T, int K, int DIM>
__device__ __forceinline__ T inv_diag(const CoarseLevel& L, T cm, T ck, int ix, int iy, int iz) {
  const int rx = ix % K, ry = iy % K, rz = iz % K;
  const T dmx = L.dmr[rx], dmy = L.dmr[ry], dkx = L.dkr[rx], dky = L.dkr[ry];
  if (DIM == 3) {
    const T dmz = L.dmr[rz], dkz = L.dkr[rz];
    return T(1) / (cm * (dmx * dmy * dmz) + ck * (dkx * dmy * dmz + dmx * dky * dmz + dmx * dmy * dkz));
  }
  return T(1) / (cm * (dmx * dmy) + ck * (dkx * dmy + dmx * dky));
}

// degree-m Chebyshev smoothing on level L of block s (from zero or from x)
template <typename T, int K, int DIM>
__device__ void smooth(const CoarseLevel& L, const CoarseParams& P, int s, T* x, T* xo, const T* b, T* t1, T* t2,
                       T* t3, T* t4, T* av, bool from_zero) {
  const T cm = (T)P.cm[s], ck = (T)P.tau;
  const int n1 = L.n1, n = L.n;
  int j0 = 0;
  if (from_zero) {
    const T c2 = (T)L.c2[0][s];
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      int ix, iy, iz;
      x[q] = interior<T, DIM>(q, n1, ix, iy, iz) ? c2 * b[q] * inv_diag<T, K, DIM>(L, cm, ck, ix, iy, iz) : T(0);
      xo[q] = T(0);
    }
    __syncthreads();
    j0 = 1;
  }
  for (int j = j0; j < P.m; ++j) {
    apply_level<T, K, DIM>(L, cm, ck, x, t1, t2, t3, t4, av);
    const T c1 = (T)L.c1[j][s], c2 = (T)L.c2[j][s];
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      int ix, iy, iz;
      if (!interior<T, DIM>(q, n1, ix, iy, iz)) continue;
      const T xv = x[q];
      const T prev = (j == 0) ? xv : xo[q];  // step 0 from a given x has no momentum term
      const T xn = xv + c1 * (xv - prev) + c2 * (b[q] - av[q]) * inv_diag<T, K, DIM>(L, cm, ck, ix, iy, iz);
      xo[q] = xv;
      x[q] = xn;
    }
    __syncthreads();
  }
}

// one axis pass of the Q_k embedding between a fine line of nf nodes and a coarse one of nc
// nodes (restriction: fine -> coarse, transposed interpolation; prolongation: coarse -> fine).
// src/dst grids: d0 x d1 x d2 with the pass axis changing size; pc = (2k+1) x (k+1), Nc cells.
template <typename T, int K, bool RESTRICT>
__device__ void transfer_pass(const T* src, T* dst, int axis, const int (&ds)[3], const int (&dd)[3], int Nc,
                              const float* pc, bool accumulate) {
  const int nout = dd[0] * dd[1] * dd[2];
  const int ss[3] = {1, ds[0], ds[0] * ds[1]};
  for (int e = threadIdx.x; e < nout; e += blockDim.x) {
    int o[3];
    o[0] = e % dd[0];
    o[1] = (e / dd[0]) % dd[1];
    o[2] = e / (dd[0] * dd[1]);
    int base = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (a != axis) base += o[a] * ss[a];
    const int st = ss[axis];
    const int ca = o[axis];
    T acc = T(0);
    if (RESTRICT) {
      const int ndc = dd[axis];
      if (ca == 0 || ca == ndc - 1) {
        dst[e] = T(0);
        continue;
      }
      const int cc = ca / K, i = ca - cc * K;
      if (i != 0) {
#pragma unroll
        for (int m = 0; m <= 2 * K; ++m) acc += (T)pc[m * (K + 1) + i] * src[base + (2 * K * cc + m) * st];
      } else {
#pragma unroll
        for (int m = 0; m < 2 * K; ++m) acc += (T)pc[m * (K + 1) + K] * src[base + (2 * K * (cc - 1) + m) * st];
#pragma unroll
        for (int m = 0; m <= 2 * K; ++m) acc += (T)pc[m * (K + 1)] * src[base + (2 * K * cc + m) * st];
      }
    } else {
      int cc = ca / (2 * K);
      if (cc > Nc - 1) cc = Nc - 1;
      const int m = ca - 2 * K * cc;
#pragma unroll
      for (int i = 0; i <= K; ++i) acc += (T)pc[m * (K + 1) + i] * src[base + (K * cc + i) * st];
    }
    if (accumulate) dst[e] += acc;
    else dst[e] = acc;
  }
  __syncthreads();
}

template <typename T, int K, int DIM>
__global__ void __launch_bounds__(kCT) coarse_cycle_kernel(const CoarseParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int s = blockIdx.x;
  const int nlev = P.nlev;
  // arena: per level x, xo, b, r; then four scratch grids of the largest level
  T* x[kMaxFusedLevels];
  T* xo[kMaxFusedLevels];
  T* b[kMaxFusedLevels];
  T* r[kMaxFusedLevels];
  int off = 0;
  for (int l = 0; l < nlev; ++l) {
    const int n = P.lv[l].n;
    x[l] = sm + off; off += n;
    xo[l] = sm + off; off += n;
    b[l] = sm + off; off += n;
    r[l] = sm + off; off += n;
  }
  const int nmax = P.lv[0].n;
  T* t1 = sm + off; off += nmax;
  T* t2 = sm + off; off += nmax;
  T* t3 = sm + off; off += nmax;
  T* t4 = sm + off; off += nmax;
  T* t5 = sm + off;
  for (int i = threadIdx.x; i < off + nmax; i += blockDim.x) sm[i] = T(0);
  __syncthreads();
  const T* bin = reinterpret_cast<const T*>(P.b_in) + (long long)s * P.ld;
  for (int q = threadIdx.x; q < P.lv[0].n; q += blockDim.x) b[0][q] = bin[q];
  __syncthreads();
  // down: pre-smooth, residual, restrict
  for (int l = 0; l + 1 < nlev; ++l) {
    const CoarseLevel& L = P.lv[l];
    smooth<T, K, DIM>(L, P, s, x[l], xo[l], b[l], t1, t2, t3, t4, t5, true);
    apply_level<T, K, DIM>(L, (T)P.cm[s], (T)P.tau, x[l], t1, t2, t3, t4, t5);
    for (int q = threadIdx.x; q < L.n; q += blockDim.x) {
      int ix, iy, iz;
      r[l][q] = interior<T, DIM>(q, L.n1, ix, iy, iz) ? b[l][q] - t5[q] : T(0);
    }
    __syncthreads();
    const int nf = L.n1, nc = P.lv[l + 1].n1, Nc = P.lv[l + 1].N;
    if (DIM == 3) {
      const int d0[3] = {nf, nf, nf}, d1[3] = {nc, nf, nf}, d2[3] = {nc, nc, nf}, d3[3] = {nc, nc, nc};
      transfer_pass<T, K, true>(r[l], t1, 0, d0, d1, Nc, P.pc, false);
      transfer_pass<T, K, true>(t1, t2, 1, d1, d2, Nc, P.pc, false);
      transfer_pass<T, K, true>(t2, b[l + 1], 2, d2, d3, Nc, P.pc, false);
    } else {
      const int d0[3] = {nf, nf, 1}, d1[3] = {nc, nf, 1}, d2[3] = {nc, nc, 1};
      transfer_pass<T, K, true>(r[l], t1, 0, d0, d1, Nc, P.pc, false);
      transfer_pass<T, K, true>(t1, b[l + 1], 1, d1, d2, Nc, P.pc, false);
    }
  }
  // coarsest: dense inverse (float copy of the FP64 inverse)
  {
    const int lc = nlev - 1;
    const float* A = P.ainv + (long long)s * P.nci * P.nci;
    for (int rr = threadIdx.x; rr < P.nci; rr += blockDim.x) {
      T acc = T(0);
      for (int c = 0; c < P.nci; ++c) acc += (T)A[(long long)rr * P.nci + c] * b[lc][P.map[c]];
      x[lc][P.map[rr]] = acc;
    }
    __syncthreads();
  }
  // up: prolongate and post-smooth
  for (int l = nlev - 2; l >= 0; --l) {
    const CoarseLevel& L = P.lv[l];
    const int nf = L.n1, nc = P.lv[l + 1].n1, Nc = P.lv[l + 1].N;
    if (DIM == 3) {
      const int d3[3] = {nc, nc, nc}, d2[3] = {nc, nc, nf}, d1[3] = {nc, nf, nf}, d0[3] = {nf, nf, nf};
      transfer_pass<T, K, false>(x[l + 1], t2, 2, d3, d2, Nc, P.pc, false);
      transfer_pass<T, K, false>(t2, t1, 1, d2, d1, Nc, P.pc, false);
      transfer_pass<T, K, false>(t1, x[l], 0, d1, d0, Nc, P.pc, true);
    } else {
      const int d2[3] = {nc, nc, 1}, d1[3] = {nc, nf, 1}, d0[3] = {nf, nf, 1};
      transfer_pass<T, K, false>(x[l + 1], t1, 1, d2, d1, Nc, P.pc, false);
      transfer_pass<T, K, false>(t1, x[l], 0, d1, d0, Nc, P.pc, true);
    }
    smooth<T, K, DIM>(L, P, s, x[l], xo[l], b[l], t1, t2, t3, t4, t5, false);
  }
  T* xout = reinterpret_cast<T*>(P.x_out) + (long long)s * P.ld;
  for (int q = threadIdx.x; q < P.lv[0].n; q += blockDim.x) xout[q] = x[0][q];
}

template <typename T, int K, int DIM>
cudaError_t launch_kd(const CoarseParams& P, size_t smem, cudaStream_t st) {
  static size_t granted = 48 * 1024;
  if (smem > granted) {
    cudaError_t e = cudaFuncSetAttribute(coarse_cycle_kernel<T, K, DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    granted = smem;
  }
  coarse_cycle_kernel<T, K, DIM><<<P.nb, kCT, smem, st>>>(P);
  return cudaGetLastError();
}

}  // namespace

size_t coarse_cycle_smem(const CoarseParams& P, int elem_size) {
  size_t n = 0;
  for (int l = 0; l < P.nlev; ++l) n += 4 * (size_t)P.lv[l].n;
  n += 5 * (size_t)P.lv[0].n;
  return n * elem_size;
}

template <typename T>
cudaError_t launch_coarse_cycle(const CoarseParams& P, int dim, int k, cudaStream_t st) {
  const size_t smem = coarse_cycle_smem(P, sizeof(T));
  if (P.nlev < 1 || P.nlev > kMaxFusedLevels || smem > kCoarseCycleMaxSmem) return cudaErrorInvalidValue;
#define IRK_CC(KK)                                                                             \
  case KK:                                                                                     \
    return (dim == 3) ? launch_kd<T, KK, 3>(P, smem, st) : launch_kd<T, KK, 2>(P, smem, st);
  switch (k) {
    IRK_CC(1) IRK_CC(2) IRK_CC(3) IRK_CC(4)
    default: return cudaErrorInvalidValue;
  }
#undef IRK_CC
}
template cudaError_t launch_coarse_cycle<float>(const CoarseParams&, int, int, cudaStream_t);

}  // namespace irk
