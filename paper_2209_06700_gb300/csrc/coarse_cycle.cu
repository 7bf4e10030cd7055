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
#include "pdl.cuh"

namespace irk {
namespace {

constexpr int kCT = 1024;  // threads per CTA (one CTA per block owns the SM: shared memory bound)

// q / n for the small node counts of the fused levels: umulhi with the magic ceil(2^32 / n) is
// exact while q * (magic * n - 2^32) < 2^32, i.e. for every q below 2^32 / n.
__device__ __forceinline__ int udiv(int q, unsigned magic) { return (int)__umulhi((unsigned)q, magic); }

template <int DIM>
__device__ __forceinline__ bool node(const CoarseLevel& L, int q, int& ix, int& iy, int& iz) {
  const int n1 = L.n1;
  const int r1 = udiv(q, L.magic);
  ix = q - r1 * n1;
  if (DIM == 3) {
    iz = udiv(r1, L.magic);
    iy = r1 - iz * n1;
  } else {
    iy = r1;
    iz = 1;
  }
  return ix > 0 && ix < n1 - 1 && iy > 0 && iy < n1 - 1 && (DIM == 2 || (iz > 0 && iz < n1 - 1));
}

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

// A u on one level, handed node by node (interior nodes only) to out(q, ix, iy, iz, (A u)_q);
// p1, p2, q1, q2 are scratch grids of n nodes.
// 3D: p1 = Mx u, p2 = Kx u; q1 = My p1, q2 = Ky p1 + My p2; A u = Mz (cm q1 + ck q2) + ck Kz q1.
template <typename T, int K, int DIM, class Out>
__device__ __forceinline__ void apply_level(const CoarseLevel& L, T cm, T ck, const T* u, T* p1, T* p2, T* q1,
                                            T* q2, Out&& out) {
  const int n1 = L.n1, n = L.n;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const int ix = q - udiv(q, L.magic) * n1;
    T a, b;
    band2<T, K>(u + q, ix, n1, 1, L.me, L.ke, a, b);
    p1[q] = a;
    p2[q] = b;
  }
  __syncthreads();
  if constexpr (DIM == 2) {
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      int ix, iy, iz;
      if (!node<2>(L, q, ix, iy, iz)) continue;
      T m1, k1;
      band2<T, K>(p1 + q, iy, n1, n1, L.me, L.ke, m1, k1);
      const T m2 = band1<T, K>(p2 + q, iy, n1, n1, L.me);
      out(q, ix, iy, 0, cm * m1 + ck * (k1 + m2));
    }
    __syncthreads();
  } else {
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      const int r1 = udiv(q, L.magic);
      const int iy = r1 - udiv(r1, L.magic) * n1;
      T m1, k1;
      band2<T, K>(p1 + q, iy, n1, n1, L.me, L.ke, m1, k1);
      q1[q] = m1;
      q2[q] = k1 + band1<T, K>(p2 + q, iy, n1, n1, L.me);
    }
    __syncthreads();
    const int pl = n1 * n1;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      int ix, iy, iz;
      if (!node<3>(L, q, ix, iy, iz)) continue;
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
      out(q, ix, iy, iz, acc);
    }
    __syncthreads();
  }
}

// 1 / diag(cm M + ck K) by in-cell position (x, y, z) mod k, the formula of the level operator
template <typename T, int K, int DIM>
__device__ __forceinline__ T inv_diag(const CoarseLevel& L, T cm, T ck, int rx, int ry, int rz) {
  const T dmx = L.dmr[rx], dmy = L.dmr[ry], dkx = L.dkr[rx], dky = L.dkr[ry];
  if (DIM == 3) {
    const T dmz = L.dmr[rz], dkz = L.dkr[rz];
    return T(1) / (cm * (dmx * dmy * dmz) + ck * (dkx * dmy * dmz + dmx * dky * dmz + dmx * dmy * dkz));
  }
  return T(1) / (cm * (dmx * dmy) + ck * (dkx * dmy + dmx * dky));
}

template <int K, int DIM>
__device__ __forceinline__ int dslot(int ix, int iy, int iz) {
  return (DIM == 3) ? ((iz % K) * K + (iy % K)) * K + (ix % K) : (iy % K) * K + (ix % K);
}

// degree-m Chebyshev smoothing on level L of block s (from zero or from x); each step's update is
// applied in the last pass of its operator application.  invd: 1/D by in-cell position.
template <typename T, int K, int DIM>
__device__ void smooth(const CoarseLevel& L, const CoarseParams& P, int s, T* x, T* xo, const T* b, T* t1, T* t2,
                       T* t3, T* t4, const T* invd, bool from_zero) {
  const T cm = (T)P.cm[s], ck = (T)P.taus[s];
  const int n = L.n;
  int j0 = 0;
  if (from_zero) {
    const T c2 = (T)L.c2[0][s];
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      int ix, iy, iz;
      x[q] = node<DIM>(L, q, ix, iy, iz) ? c2 * b[q] * invd[dslot<K, DIM>(ix, iy, iz)] : T(0);
      xo[q] = T(0);
    }
    __syncthreads();
    j0 = 1;
  }
  for (int j = j0; j < P.m; ++j) {
    const T c1 = (T)L.c1[j][s], c2 = (T)L.c2[j][s];
    const bool first = (j == 0);  // step 0 from a given x has no momentum term
    apply_level<T, K, DIM>(L, cm, ck, x, t1, t2, t3, t4, [&](int q, int ix, int iy, int iz, T av) {
      const T xv = x[q];
      const T prev = first ? xv : xo[q];
      xo[q] = xv;
      x[q] = xv + c1 * (xv - prev) + c2 * (b[q] - av) * invd[dslot<K, DIM>(ix, iy, iz)];
    });
  }
}

// One axis pass of the Q_k embedding between a fine line of 2K Nc + 1 nodes and a coarse one of
// K Nc + 1 nodes, one thread per coarse cell of every line (restriction: fine -> coarse with the
// transposed interpolation; prolongation: coarse -> fine).  Grids d0 x d1 x d2, x fastest; the
// pass axis changes size between src (ds) and dst (dd).  pc = (2K+1) x (K+1).
template <typename T, int K, int AXIS, bool RESTRICT>
__device__ void tpass(const T* src, T* dst, const int (&ds)[3], const int (&dd)[3], int Nc, const float* pc,
                      bool accumulate) {
  constexpr int KP = K + 1;
  const int others = (AXIS == 0) ? dd[1] * dd[2] : (AXIS == 1) ? dd[0] * dd[2] : dd[0] * dd[1];
  const int total = others * Nc;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    int cc, bi, bo, si, so;
    if (AXIS == 0) {
      cc = t % Nc;
      const int r = t / Nc;
      bi = r * ds[0];
      bo = r * dd[0];
      si = so = 1;
    } else if (AXIS == 1) {
      const int o0 = t % ds[0];
      const int t2 = t / ds[0];
      cc = t2 % Nc;
      const int o2 = t2 / Nc;
      bi = o0 + o2 * ds[0] * ds[1];
      bo = o0 + o2 * dd[0] * dd[1];
      si = so = ds[0];
    } else {
      const int plane = ds[0] * ds[1];
      bi = bo = t % plane;
      cc = t / plane;
      si = so = plane;
    }
    const T* in = src + bi;
    T* out = dst + bo;
    if (RESTRICT) {
      T f[4 * K + 1];
#pragma unroll
      for (int j = 0; j < 2 * K; ++j) f[j] = (cc > 0) ? in[(2 * K * (cc - 1) + j) * si] : T(0);
#pragma unroll
      for (int j = 2 * K; j <= 4 * K; ++j) f[j] = in[(2 * K * (cc - 1) + j) * si];
      T r0 = T(0);
      if (cc > 0) {
#pragma unroll
        for (int m = 0; m < 2 * K; ++m) r0 += (T)pc[m * KP + K] * f[m];
#pragma unroll
        for (int m = 0; m <= 2 * K; ++m) r0 += (T)pc[m * KP] * f[2 * K + m];
      }
      out[(K * cc) * so] = accumulate ? out[(K * cc) * so] + r0 : r0;
#pragma unroll
      for (int i = 1; i < K; ++i) {
        T acc = T(0);
#pragma unroll
        for (int m = 0; m <= 2 * K; ++m) acc += (T)pc[m * KP + i] * f[2 * K + m];
        out[(K * cc + i) * so] = accumulate ? out[(K * cc + i) * so] + acc : acc;
      }
      if (cc == Nc - 1 && !accumulate) out[(K * Nc) * so] = T(0);  // coarse boundary node
    } else {
      T c[KP];
#pragma unroll
      for (int i = 0; i <= K; ++i) c[i] = in[(K * cc + i) * si];
      const int mend = (cc == Nc - 1) ? 2 * K : 2 * K - 1;
#pragma unroll
      for (int m = 0; m <= 2 * K; ++m) {
        if (m > mend) break;
        T acc = T(0);
#pragma unroll
        for (int i = 0; i <= K; ++i) acc += (T)pc[m * KP + i] * c[i];
        out[(2 * K * cc + m) * so] = accumulate ? out[(2 * K * cc + m) * so] + acc : acc;
      }
    }
  }
  __syncthreads();
}

template <typename T, int K, int DIM>
__global__ void __launch_bounds__(kCT) coarse_cycle_kernel(const CoarseParams P) {
  dev::pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  constexpr int KD = (DIM == 3) ? K * K * K : K * K;
  __shared__ T sinv[kMaxFusedLevels][KD];  // 1/D per level by in-cell position
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
  for (int i = threadIdx.x; i < off; i += blockDim.x) sm[i] = T(0);
  for (int i = threadIdx.x; i < nlev * KD; i += blockDim.x) {
    const int l = i / KD, t = i - l * KD;
    const int rx = t % K, ry = (t / K) % K, rz = (DIM == 3) ? t / (K * K) : 0;
    sinv[l][t] = inv_diag<T, K, DIM>(P.lv[l], (T)P.cm[s], (T)P.taus[s], rx, ry, rz);
  }
  __syncthreads();
  const T* bin = reinterpret_cast<const T*>(P.b_in) + (long long)s * P.ld;
  for (int q = threadIdx.x; q < P.lv[0].n; q += blockDim.x) b[0][q] = bin[q];
  __syncthreads();
  // down: pre-smooth, residual, restrict
  for (int l = 0; l + 1 < nlev; ++l) {
    const CoarseLevel& L = P.lv[l];
    smooth<T, K, DIM>(L, P, s, x[l], xo[l], b[l], t1, t2, t3, t4, sinv[l], true);
    T* rl = r[l];
    const T* bl = b[l];
    apply_level<T, K, DIM>(L, (T)P.cm[s], (T)P.taus[s], x[l], t1, t2, t3, t4,
                           [&](int q, int, int, int, T av) { rl[q] = bl[q] - av; });
    const int nf = L.n1, nc = P.lv[l + 1].n1, Nc = P.lv[l + 1].N;
    if (DIM == 3) {
      const int d0[3] = {nf, nf, nf}, d1[3] = {nc, nf, nf}, d2[3] = {nc, nc, nf}, d3[3] = {nc, nc, nc};
      tpass<T, K, 0, true>(rl, t1, d0, d1, Nc, P.pc, false);
      tpass<T, K, 1, true>(t1, t2, d1, d2, Nc, P.pc, false);
      tpass<T, K, 2, true>(t2, b[l + 1], d2, d3, Nc, P.pc, false);
    } else {
      const int d0[3] = {nf, nf, 1}, d1[3] = {nc, nf, 1}, d2[3] = {nc, nc, 1};
      tpass<T, K, 0, true>(rl, t1, d0, d1, Nc, P.pc, false);
      tpass<T, K, 1, true>(t1, b[l + 1], d1, d2, Nc, P.pc, false);
    }
  }
  // coarsest: the dense FP64 inverse applied in FP64 (the coarse-grid solve stays FP64 inside the
  // FP32 V-cycle)
  {
    const int lc = nlev - 1;
    const double* A = P.ainv + (long long)s * P.nci * P.nci;
    for (int rr = threadIdx.x; rr < P.nci; rr += blockDim.x) {
      double acc = 0.0;
      for (int c = 0; c < P.nci; ++c) acc += A[(long long)rr * P.nci + c] * (double)b[lc][P.map[c]];
      x[lc][P.map[rr]] = (T)acc;
    }
    __syncthreads();
  }
  // up: prolongate and post-smooth
  for (int l = nlev - 2; l >= 0; --l) {
    const CoarseLevel& L = P.lv[l];
    const int nf = L.n1, nc = P.lv[l + 1].n1, Nc = P.lv[l + 1].N;
    if (DIM == 3) {
      const int d3[3] = {nc, nc, nc}, d2[3] = {nc, nc, nf}, d1[3] = {nc, nf, nf}, d0[3] = {nf, nf, nf};
      tpass<T, K, 2, false>(x[l + 1], t2, d3, d2, Nc, P.pc, false);
      tpass<T, K, 1, false>(t2, t1, d2, d1, Nc, P.pc, false);
      tpass<T, K, 0, false>(t1, x[l], d1, d0, Nc, P.pc, true);
    } else {
      const int d2[3] = {nc, nc, 1}, d1[3] = {nc, nf, 1}, d0[3] = {nf, nf, 1};
      tpass<T, K, 1, false>(x[l + 1], t1, d2, d1, Nc, P.pc, false);
      tpass<T, K, 0, false>(t1, x[l], d1, d0, Nc, P.pc, true);
    }
    smooth<T, K, DIM>(L, P, s, x[l], xo[l], b[l], t1, t2, t3, t4, sinv[l], false);
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
  launch_pdl(coarse_cycle_kernel<T, K, DIM>, P.nb, kCT, smem, st, P);
  return cudaGetLastError();
}

}  // namespace

unsigned coarse_cycle_magic(int n) { return (unsigned)(0xFFFFFFFFull / (unsigned long long)n + 1ull); }

size_t coarse_cycle_smem(const CoarseParams& P, int elem_size) {
  size_t n = 0;
  for (int l = 0; l < P.nlev; ++l) n += 4 * (size_t)P.lv[l].n;
  n += 4 * (size_t)P.lv[0].n;
  return n * elem_size;
}

template <typename T>
cudaError_t launch_coarse_cycle(const CoarseParams& P, int dim, int k, cudaStream_t st) {
  const size_t smem = coarse_cycle_smem(P, sizeof(T));
  if (P.nlev < 1 || P.nlev > kMaxFusedLevels || smem > kCoarseCycleMaxSmem) return cudaErrorInvalidValue;
  for (int l = 0; l < P.nlev; ++l)  // udiv exactness (q < n1^2 <= 2^32 / n1) and the magic itself
    if (P.lv[l].n1 < 2 || P.lv[l].n1 > 1024 || P.lv[l].magic != coarse_cycle_magic(P.lv[l].n1))
      return cudaErrorInvalidValue;
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
