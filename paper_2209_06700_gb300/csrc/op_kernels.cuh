// Matrix-free tensor-product operator kernels of libirk (sm_103a).
//
// Computes v_s = cm_s M u_s + ck_s K u_s for continuous Q_k elements on the
// uniform mesh of [0,1]^d with Gauss (k+1)^d quadrature (arXiv 2209.06700,
// Sec. 5: tensor-product Lagrange elements, consistent Gauss rule; Sec. 2:
// "generalized vector scaling" (I (x) C) u applied stage by stage).  On an
// affine Cartesian cell the Gauss rule factorises, so the cell matrices are
// Kronecker products of the 1D element matrices me (mass, x h) and ke
// (stiffness, / h) and
//   M u = Mz (My (Mx u)),   K u = Mz (My (Kx u) + Ky (Mx u)) + Kz (My (Mx u)),
// i.e. sum factorisation with dense (k+1) x (k+1) 1D contractions per cell.
//
// GPU mapping (2.5D streaming, one stage per CTA):
//  * a CTA owns 32 cells in x (one per lane) and CY cells in y (k*CY rows,
//    one warp per row) and streams through a chunk of z cells;
//  * each input z-plane (x-y tile + halo: k nodes below, 1 above) is
//    prefetched into registers one plane ahead and staged in shared memory
//    in a cell-interleaved layout [m][cell], m = node index inside the cell,
//    so that lanes (= cells) touch consecutive words;
//  * y contraction: banded form with warp-uniform row position r = y mod k;
//  * x contraction: cell-wise dense (k+1)^2 products per lane, the shared
//    vertex node merged with the left neighbour by __shfl_up_sync;
//  * z contraction: cell-wise "push" into k+1 register accumulators per
//    owned node; a z-cell's k planes are complete, and emitted through the
//    fused epilogue, once its upper vertex plane has been pushed.
// Boundary nodes (homogeneous Dirichlet) are read as zero and never written.
#pragma once
#include "kernels.h"

namespace irk {
namespace dev {

template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// Epilogue for one interior output node (stage s, linear index idx in the stage vector).
template <typename T, int EPI, int K, int DIM>
__device__ __forceinline__ void epilogue(const EpiParams<T>& E, long long o, int x, int y, int z,
                                         T cm, T ck, int s, T va, T vb) {
  if constexpr (EPI == EPI_STORE) {
    E.out[o] = va;
  } else if constexpr (EPI == EPI_DUAL) {
    E.out[o] = va;
    E.out2[o] = vb;
  } else if constexpr (EPI == EPI_RESID) {
    E.out[o] = E.b[o] - va;
  } else {  // EPI_CHEB
    const int rx = x % K, ry = y % K;
    T dmx = E.dmr[rx], dmy = E.dmr[ry], dkx = E.dkr[rx], dky = E.dkr[ry];
    T D;
    if constexpr (DIM == 3) {
      const int rz = z % K;
      T dmz = E.dmr[rz], dkz = E.dkr[rz];
      D = cm * (dmx * dmy * dmz) + ck * (dkx * dmy * dmz + dmx * dky * dmz + dmx * dmy * dkz);
    } else {
      D = cm * (dmx * dmy) + ck * (dkx * dmy + dmx * dky);
    }
    const T xv = E.xj[o];
    const T xo = E.xold_zero ? T(0) : E.out[o];
    const T c1 = E.c1[s];
    const T upd = (c1 != T(0)) ? c1 * (xv - xo) : T(0);
    E.out[o] = xv + upd + E.c2[s] * (E.b[o] - va) / D;
  }
}

// y-direction banded taps for output row position R (compile time); col points at
// the output row in the staged input column, stride = row stride.
template <typename T, int K, int R>
__device__ __forceinline__ void ytaps(const T* col, int stride, const OpParams<T>& P, T& g, T& h) {
  if constexpr (R == 0) {
#pragma unroll
    for (int o = -K; o <= K; ++o) {
      T a = T(0), b = T(0);
      if (o >= 0) { a += P.me[0][o]; b += P.ke[0][o]; }
      if (o <= 0) { a += P.me[K][K + o]; b += P.ke[K][K + o]; }
      const T v = col[o * stride];
      g += a * v;
      h += b * v;
    }
  } else {
#pragma unroll
    for (int m = 0; m <= K; ++m) {
      const T v = col[(m - R) * stride];
      g += P.me[R][m] * v;
      h += P.ke[R][m] * v;
    }
  }
}

template <typename T, int K, int R = 0>
__device__ __forceinline__ void ytaps_dispatch(int r, const T* col, int stride, const OpParams<T>& P,
                                               T& g, T& h) {
  if constexpr (R < K) {
    if (r == R) ytaps<T, K, R>(col, stride, P, g, h);
    else ytaps_dispatch<T, K, R + 1>(r, col, stride, P, g, h);
  }
}

// Cell-wise x contraction for one lane's cell (staged columns cl, cl+1 of slots [m][cell]).
// MODE3: g = My u, h = Ky u given -> R = Mx g, Pp = Kx g + Mx h.  MODE2: u given -> R = Mx u, Pp = Kx u.
template <typename T, int K, bool MODE3, int CW>
__device__ __forceinline__ void xcell(const T* g, const T* h, int cl, const OpParams<T>& P,
                                      T (&r)[K + 1], T (&p)[K + 1]) {
  T gv[K + 1], hv[K + 1];
#pragma unroll
  for (int m = 0; m < K; ++m) {
    gv[m] = g[m * CW + cl];
    if constexpr (MODE3) hv[m] = h[m * CW + cl];
  }
  gv[K] = g[cl + 1];
  if constexpr (MODE3) hv[K] = h[cl + 1];
#pragma unroll
  for (int mo = 0; mo <= K; ++mo) {
    T a = T(0), b = T(0);
#pragma unroll
    for (int m = 0; m <= K; ++m) {
      a += P.me[mo][m] * gv[m];
      b += P.ke[mo][m] * gv[m];
      if constexpr (MODE3) b += P.me[mo][m] * hv[m];
    }
    r[mo] = a;
    p[mo] = b;
  }
}

// Top-vertex outputs (local node K) of the cell at staged column cl.
template <typename T, int K, bool MODE3, int CW>
__device__ __forceinline__ void xcell_top(const T* g, const T* h, int cl, const OpParams<T>& P, T& r, T& p) {
  T a = T(0), b = T(0);
#pragma unroll
  for (int m = 0; m <= K; ++m) {
    const int slot = (m < K) ? (m * CW + cl) : (cl + 1);
    const T gv = g[slot];
    a += P.me[K][m] * gv;
    b += P.ke[K][m] * gv;
    if constexpr (MODE3) b += P.me[K][m] * h[slot];
  }
  r = a;
  p = b;
}

// z push of column RZ (compile time) into the accumulators of the owned nodes.
template <typename T, int K, int RZ, bool DUAL>
__device__ __forceinline__ void zpush(const OpParams<T>& P, T cm, T ck, const T (&R)[K], const T (&Pp)[K],
                                      T (&accA)[K][K + 1], T (&accB)[K][K + 1]) {
#pragma unroll
  for (int m = 0; m < K; ++m) {
    if constexpr (DUAL) {
#pragma unroll
      for (int mo = 0; mo <= K; ++mo) {
        accA[m][mo] += P.me[mo][RZ] * R[m];
        accB[m][mo] += P.me[mo][RZ] * Pp[m] + P.ke[mo][RZ] * R[m];
      }
    } else {
      const T F = cm * R[m] + ck * Pp[m];
      const T Ez = ck * R[m];
#pragma unroll
      for (int mo = 0; mo <= K; ++mo) accA[m][mo] += P.me[mo][RZ] * F + P.ke[mo][RZ] * Ez;
    }
  }
}

template <typename T, int K, bool DUAL>
__device__ __forceinline__ void carry(T (&accA)[K][K + 1], T (&accB)[K][K + 1]) {
#pragma unroll
  for (int m = 0; m < K; ++m) {
    accA[m][0] = accA[m][K];
    if constexpr (DUAL) accB[m][0] = accB[m][K];
#pragma unroll
    for (int mo = 1; mo <= K; ++mo) {
      accA[m][mo] = T(0);
      if constexpr (DUAL) accB[m][mo] = T(0);
    }
  }
}

}  // namespace dev

template <int K> struct Tile3D { static constexpr int CY = (K == 1) ? 8 : (K == 2) ? 4 : 2; };

// ---------------------------------------------------------------- 3D kernel
template <typename T, int K, int EPI>
__global__ void __launch_bounds__(32 * K * Tile3D<K>::CY)
op3d_kernel(const T* __restrict__ u, const OpParams<T> P, const EpiParams<T> E) {
  constexpr int CY = Tile3D<K>::CY;
  constexpr int CX = 32, TY = K * CY, NT = 32 * TY;
  constexpr int CW = CX + 2, SL = K * CW;
  constexpr int HY = TY + K + 1, HX = K * CX + K + 1;
  constexpr int NLD = HY * HX;
  constexpr int PF = (NLD + NT - 1) / NT;
  constexpr bool DUAL = (EPI == EPI_DUAL);
  __shared__ T su[HY * SL];
  __shared__ T sg[TY * SL];
  __shared__ T sh[TY * SL];

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int N = P.N, n1 = P.n1;
  const int cx0 = blockIdx.x * CX;
  const int ty = blockIdx.y % P.ntile_y, zchunk = blockIdx.y / P.ntile_y;
  const int y0 = K * CY * ty, x0 = K * cx0;
  const int s = blockIdx.z;
  const T* __restrict__ us = u + (long long)s * P.ld;
  const T cm = P.cm[s], ck = P.ck[s];
  const int c0 = zchunk * P.zc;
  if (c0 >= N) return;
  const int c1 = min(N, c0 + P.zc);
  const int cstart = max(c0 - 1, 0);
  const long long plane = (long long)n1 * n1;

  for (int i = tid; i < HY * SL; i += NT) su[i] = T(0);  // padding slots stay zero

  // per-thread load slots: global offset within a plane (or -1) and shared slot
  int goff[PF], soff[PF];
#pragma unroll
  for (int q = 0; q < PF; ++q) {
    const int i = tid + q * NT;
    goff[q] = -1;
    soff[q] = -1;
    if (i < NLD) {
      const int yl = i / HX, xl = i - yl * HX;
      const int yg = y0 - K + yl, xg = x0 - K + xl;
      const int cl = xl / K, m = xl - cl * K;
      soff[q] = yl * SL + m * CW + cl;
      if (yg >= 0 && yg < n1 && xg >= 0 && xg < n1) goff[q] = yg * n1 + xg;
    }
  }
  T pf[PF];
  auto load_plane = [&](int zp) {
    const T* base = us + zp * plane;
#pragma unroll
    for (int q = 0; q < PF; ++q) pf[q] = (goff[q] >= 0) ? dev::ldg(base + goff[q]) : T(0);
  };
  auto store_plane = [&]() {
#pragma unroll
    for (int q = 0; q < PF; ++q)
      if (soff[q] >= 0) su[soff[q]] = pf[q];
  };
  auto ypass = [&]() {
    const int ro = w % K;
    const T* colbase = su + (w + K) * SL;
    for (int sl = lane; sl < SL; sl += 32) {
      T g = T(0), h = T(0);
      dev::ytaps_dispatch<T, K>(ro, colbase + sl, SL, P, g, h);
      sg[w * SL + sl] = g;
      sh[w * SL + sl] = h;
    }
  };
  auto xpass = [&](T (&R)[K], T (&Pp)[K]) {
    const T* g = sg + w * SL;
    const T* h = sh + w * SL;
    T r[K + 1], p[K + 1];
    dev::xcell<T, K, true, CW>(g, h, lane + 1, P, r, p);
    T rl = __shfl_up_sync(0xffffffffu, r[K], 1);
    T pl = __shfl_up_sync(0xffffffffu, p[K], 1);
    if (lane == 0) dev::xcell_top<T, K, true, CW>(g, h, 0, P, rl, pl);
    r[0] += rl;
    p[0] += pl;
#pragma unroll
    for (int m = 0; m < K; ++m) { R[m] = r[m]; Pp[m] = p[m]; }
  };
  const int yrow = y0 + w;
  const int cell = cx0 + lane;
  const bool row_ok = (yrow >= 1 && yrow <= n1 - 2) && (cell < N);
  T accA[K][K + 1], accB[K][K + 1];
#pragma unroll
  for (int m = 0; m < K; ++m)
#pragma unroll
    for (int mo = 0; mo <= K; ++mo) { accA[m][mo] = T(0); accB[m][mo] = T(0); }

  auto emit = [&](int cz) {
    if (!row_ok) return;
#pragma unroll
    for (int mo = 0; mo < K; ++mo) {
      const int z = K * cz + mo;
      if (z < 1) continue;
#pragma unroll
      for (int m = 0; m < K; ++m) {
        const int x = K * cell + m;
        if (x < 1) continue;
        const long long idx = ((long long)z * n1 + yrow) * n1 + x;
        dev::epilogue<T, EPI, K, 3>(E, (long long)s * P.ld + idx, x, yrow, z, cm, ck, s, accA[m][mo],
                                    accB[m][mo]);
      }
    }
  };

  __syncthreads();
  load_plane(K * cstart);
  for (int c = cstart; c < c1; ++c) {
#pragma unroll
    for (int r = 0; r < K; ++r) {
      const int zp = K * c + r;
      store_plane();
      __syncthreads();
      load_plane(zp + 1);
      ypass();
      __syncthreads();
      T R[K], Pp[K];
      xpass(R, Pp);
      if (r == 0) {
        if (c > cstart) {
          dev::zpush<T, K, K, DUAL>(P, cm, ck, R, Pp, accA, accB);
          if (c - 1 >= c0) emit(c - 1);
          dev::carry<T, K, DUAL>(accA, accB);
        }
        dev::zpush<T, K, 0, DUAL>(P, cm, ck, R, Pp, accA, accB);
      } else {
        // r is a compile-time constant after unrolling
        if (r == 1) dev::zpush<T, K, (1 < K ? 1 : 0), DUAL>(P, cm, ck, R, Pp, accA, accB);
        if constexpr (K > 2) if (r == 2) dev::zpush<T, K, (2 < K ? 2 : 0), DUAL>(P, cm, ck, R, Pp, accA, accB);
        if constexpr (K > 3) if (r == 3) dev::zpush<T, K, (3 < K ? 3 : 0), DUAL>(P, cm, ck, R, Pp, accA, accB);
      }
    }
  }
  // upper vertex plane of the last cell
  store_plane();
  __syncthreads();
  ypass();
  __syncthreads();
  {
    T R[K], Pp[K];
    xpass(R, Pp);
    dev::zpush<T, K, K, DUAL>(P, cm, ck, R, Pp, accA, accB);
    if (c1 - 1 >= c0) emit(c1 - 1);
  }
}

// ---------------------------------------------------------------- 2D kernel
// Plane = one x row; streaming along y.  NW warps, 32*NW cells per tile in x.
template <typename T, int K, int EPI>
__global__ void __launch_bounds__(64)
op2d_kernel(const T* __restrict__ u, const OpParams<T> P, const EpiParams<T> E) {
  constexpr int NW = 2, NT = 32 * NW;
  constexpr int CX = 32 * NW, CW = CX + 2, SL = K * CW;
  constexpr int HX = K * CX + K + 1;
  constexpr int PF = (HX + NT - 1) / NT;
  constexpr bool DUAL = (EPI == EPI_DUAL);
  __shared__ T su[SL];

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int N = P.N, n1 = P.n1;
  const int cx0 = blockIdx.x * CX, x0 = K * cx0;
  const int s = blockIdx.z;
  const T* __restrict__ us = u + (long long)s * P.ld;
  const T cm = P.cm[s], ck = P.ck[s];
  const int c0 = blockIdx.y * P.zc;
  if (c0 >= N) return;
  const int c1 = min(N, c0 + P.zc);
  const int cstart = max(c0 - 1, 0);

  for (int i = tid; i < SL; i += NT) su[i] = T(0);
  int goff[PF], soff[PF];
#pragma unroll
  for (int q = 0; q < PF; ++q) {
    const int xl = tid + q * NT;
    goff[q] = -1;
    soff[q] = -1;
    if (xl < HX) {
      const int xg = x0 - K + xl;
      const int cl = xl / K, m = xl - cl * K;
      soff[q] = m * CW + cl;
      if (xg >= 0 && xg < n1) goff[q] = xg;
    }
  }
  T pf[PF];
  auto load_row = [&](int yp) {
    const T* base = us + (long long)yp * n1;
#pragma unroll
    for (int q = 0; q < PF; ++q) pf[q] = (goff[q] >= 0) ? dev::ldg(base + goff[q]) : T(0);
  };
  auto store_row = [&]() {
#pragma unroll
    for (int q = 0; q < PF; ++q)
      if (soff[q] >= 0) su[soff[q]] = pf[q];
  };
  const int cl = w * 32 + lane + 1;
  auto xpass = [&](T (&R)[K], T (&Pp)[K]) {
    T r[K + 1], p[K + 1];
    dev::xcell<T, K, false, CW>(su, su, cl, P, r, p);
    T rl = __shfl_up_sync(0xffffffffu, r[K], 1);
    T pl = __shfl_up_sync(0xffffffffu, p[K], 1);
    if (lane == 0) dev::xcell_top<T, K, false, CW>(su, su, cl - 1, P, rl, pl);
    r[0] += rl;
    p[0] += pl;
#pragma unroll
    for (int m = 0; m < K; ++m) { R[m] = r[m]; Pp[m] = p[m]; }
  };
  const int cell = cx0 + w * 32 + lane;
  const bool col_ok = cell < N;
  T accA[K][K + 1], accB[K][K + 1];
#pragma unroll
  for (int m = 0; m < K; ++m)
#pragma unroll
    for (int mo = 0; mo <= K; ++mo) { accA[m][mo] = T(0); accB[m][mo] = T(0); }
  auto emit = [&](int cyc) {
    if (!col_ok) return;
#pragma unroll
    for (int mo = 0; mo < K; ++mo) {
      const int y = K * cyc + mo;
      if (y < 1) continue;
#pragma unroll
      for (int m = 0; m < K; ++m) {
        const int x = K * cell + m;
        if (x < 1) continue;
        const long long idx = (long long)y * n1 + x;
        dev::epilogue<T, EPI, K, 2>(E, (long long)s * P.ld + idx, x, y, 0, cm, ck, s, accA[m][mo],
                                    accB[m][mo]);
      }
    }
  };
  __syncthreads();
  load_row(K * cstart);
  for (int c = cstart; c < c1; ++c) {
#pragma unroll
    for (int r = 0; r < K; ++r) {
      const int yp = K * c + r;
      __syncthreads();
      store_row();
      __syncthreads();
      load_row(yp + 1);
      T R[K], Pp[K];
      xpass(R, Pp);
      if (r == 0) {
        if (c > cstart) {
          dev::zpush<T, K, K, DUAL>(P, cm, ck, R, Pp, accA, accB);
          if (c - 1 >= c0) emit(c - 1);
          dev::carry<T, K, DUAL>(accA, accB);
        }
        dev::zpush<T, K, 0, DUAL>(P, cm, ck, R, Pp, accA, accB);
      } else {
        if (r == 1) dev::zpush<T, K, (1 < K ? 1 : 0), DUAL>(P, cm, ck, R, Pp, accA, accB);
        if constexpr (K > 2) if (r == 2) dev::zpush<T, K, (2 < K ? 2 : 0), DUAL>(P, cm, ck, R, Pp, accA, accB);
        if constexpr (K > 3) if (r == 3) dev::zpush<T, K, (3 < K ? 3 : 0), DUAL>(P, cm, ck, R, Pp, accA, accB);
      }
    }
  }
  __syncthreads();
  store_row();
  __syncthreads();
  {
    T R[K], Pp[K];
    xpass(R, Pp);
    dev::zpush<T, K, K, DUAL>(P, cm, ck, R, Pp, accA, accB);
    if (c1 - 1 >= c0) emit(c1 - 1);
  }
}

inline void op_tile_shape_impl(int dim, int k, int* cx, int* cy) {
  if (dim == 2) { *cx = 64; *cy = 1; return; }
  *cx = 32;
  *cy = (k == 1) ? 8 : (k == 2) ? 4 : 2;
}

inline int device_sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    n = v > 0 ? v : 1;
  }
  return n;
}

// Streaming chunk (cells per CTA along the streaming axis): minimise
// waves(CTAs) x planes per CTA, where a chunk that does not start at the
// bottom also streams the k planes of the cell below it.
inline int pick_zc(int N, long long base_ctas, long long slots, int K) {
  int best = N;
  long long best_cost = -1;
  for (int zc = 1; zc <= N; ++zc) {
    const long long nch = (N + zc - 1) / zc;
    const long long waves = (base_ctas * nch + slots - 1) / slots;
    const long long planes = (long long)K * (zc + (nch > 1 ? 1 : 0)) + 1;
    const long long cost = waves * planes;
    if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = zc; }
  }
  return best;
}

template <typename T, int K, int EPI>
cudaError_t launch_op_k(int dim, int nstage, const T* u, const OpParams<T>& P, const EpiParams<T>& E,
                        cudaStream_t st) {
  int cx, cy;
  op_tile_shape_impl(dim, K, &cx, &cy);
  const int ntx = (P.N + cx - 1) / cx;
  OpParams<T> Q = P;
  if (dim == 3) {
    const int threads = 32 * K * cy;
    static int occ = 0;
    if (occ == 0) {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, op3d_kernel<T, K, EPI>, threads, 0);
      if (occ < 1) occ = 1;
    }
    Q.ntile_y = (P.N + cy - 1) / cy;
    if (Q.zc <= 0) Q.zc = pick_zc(P.N, (long long)ntx * Q.ntile_y * nstage, (long long)occ * device_sm_count(), K);
    const int nch = (P.N + Q.zc - 1) / Q.zc;
    dim3 grid(ntx, Q.ntile_y * nch, nstage);
    op3d_kernel<T, K, EPI><<<grid, threads, 0, st>>>(u, Q, E);
  } else {
    static int occ = 0;
    if (occ == 0) {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, op2d_kernel<T, K, EPI>, 64, 0);
      if (occ < 1) occ = 1;
    }
    if (Q.zc <= 0) Q.zc = pick_zc(P.N, (long long)ntx * nstage, (long long)occ * device_sm_count(), K);
    const int nch = (P.N + Q.zc - 1) / Q.zc;
    dim3 grid(ntx, nch, nstage);
    op2d_kernel<T, K, EPI><<<grid, 64, 0, st>>>(u, Q, E);
  }
  return cudaGetLastError();
}

template <typename T, int EPI>
cudaError_t launch_op_e(int dim, int k, int nstage, const T* u, const OpParams<T>& P, const EpiParams<T>& E,
                        cudaStream_t st) {
  switch (k) {
    case 1: return launch_op_k<T, 1, EPI>(dim, nstage, u, P, E, st);
    case 2: return launch_op_k<T, 2, EPI>(dim, nstage, u, P, E, st);
    case 3: return launch_op_k<T, 3, EPI>(dim, nstage, u, P, E, st);
    case 4: return launch_op_k<T, 4, EPI>(dim, nstage, u, P, E, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace irk
