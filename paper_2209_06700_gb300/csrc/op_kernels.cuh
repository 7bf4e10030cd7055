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
//    vertex node merged with the left neighbour by a warp shuffle;
//  * z contraction: cell-wise "push" into k+1 register accumulators per
//    owned node; a z-cell's k planes are complete, and emitted through the
//    fused epilogue, once its upper vertex plane has been pushed;
//  * z chunks: the vertex plane between two chunks takes contributions from
//    the cells on both sides.  When the chunks of a tile run as one thread-
//    block cluster, each CTA streams only its own cells, keeps its bottom
//    vertex plane back, and adds the lower chunk's top contributions read from
//    that CTA's shared memory (distributed shared memory) after a cluster
//    barrier; otherwise a chunk re-streams the cell below it.
// Boundary nodes (homogeneous Dirichlet) are read as zero and never written.
//
// Arithmetic goes through dev::mad / mul / add so that one body serves FP32
// (multigrid), FP64 and float-float (T = ff: FP64-accurate apply on the FP32
// pipe, vectors stored as ff pairs).
#pragma once
#include <cooperative_groups.h>

#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

#include "ffmath.cuh"
#include "kernels.h"
#include "pdl.cuh"

namespace irk {
namespace dev {

// 4-byte asynchronous copy global -> shared (completes at cp_async_wait_all in the same thread)
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
template <typename A, typename B> __device__ __forceinline__ void cp_async4(A*, const B*) {}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// load from storage and store back (ff vectors are stored as ff pairs, 8 bytes per value)
template <typename T> __device__ __forceinline__ T load(const typename Storage<T>::type* p) { return ldg<T>(p); }
__device__ __forceinline__ float to_storage(float v) { return v; }
__device__ __forceinline__ double to_storage(double v) { return v; }
__device__ __forceinline__ ff to_storage(ff v) { return v; }

// ---------------------------------------------------------------- epilogues
// One interior output node (stage s, flat offset o).  CHEB needs invD = 1/diag(cm M + ck K).
template <typename T, int EPI>
__device__ __forceinline__ void epilogue(const EpiParams<typename Storage<T>::type>& E, long long o, int s, T va,
                                         T vb, typename Storage<T>::type invD) {
  if constexpr (EPI == EPI_STORE) {
    E.out[o] = to_storage(va);
  } else if constexpr (EPI == EPI_DUAL) {
    E.out[o] = to_storage(va);
    E.out2[o] = to_storage(vb);
  } else if constexpr (EPI == EPI_RESID) {
    E.out[o] = E.b[o] - to_storage(va);
  } else {  // EPI_CHEB (float / double)
    using S = typename Storage<T>::type;
    const S xv = E.xj[o];
    const S bv = E.b[o];
    const S c1 = E.c1[s];
    S upd = S(0);  // momentum c1 (x_j - x_{j-1}); x_{j-1} = 0 when xold_zero
    if (c1 != S(0)) upd = c1 * (xv - (E.xold_zero ? S(0) : E.out[o]));
    E.out[o] = xv + upd + E.c2[s] * (bv - to_storage(va)) * invD;
  }
}

// The same epilogues with the operands' addresses already at the node (the streaming kernel keeps
// per-thread pointers to its row, so no 64-bit index arithmetic runs per node); c1, c2: the
// stage's Chebyshev coefficients.
template <typename T, int EPI>
__device__ __forceinline__ void epilogue_at(typename Storage<T>::type* out, typename Storage<T>::type* out2,
                                            const typename Storage<T>::type* b, const typename Storage<T>::type* xj,
                                            int xold_zero, typename Storage<T>::type c1,
                                            typename Storage<T>::type c2, T va, T vb,
                                            typename Storage<T>::type invD) {
  using S = typename Storage<T>::type;
  if constexpr (EPI == EPI_STORE) {
    *out = to_storage(va);
  } else if constexpr (EPI == EPI_DUAL) {
    *out = to_storage(va);
    *out2 = to_storage(vb);
  } else if constexpr (EPI == EPI_RESID) {
    *out = *b - to_storage(va);
  } else {  // EPI_CHEB (float / double)
    const S xv = *xj;
    const S bv = *b;
    S upd = S(0);  // momentum c1 (x_j - x_{j-1}); x_{j-1} = 0 when xold_zero
    if (c1 != S(0)) upd = c1 * (xv - (xold_zero ? S(0) : *out));
    *out = xv + upd + c2 * (bv - to_storage(va)) * invD;
  }
}

// 1 / diag(cm M + ck K) at a node with positions (rx, ry, rz) = (x, y, z) mod k inside the cell.
template <typename S, int DIM>
__device__ __forceinline__ S inv_diag(const EpiParams<S>& E, S cm, S ck, int rx, int ry, int rz) {
  const S dmx = E.dmr[rx], dmy = E.dmr[ry], dkx = E.dkr[rx], dky = E.dkr[ry];
  if constexpr (DIM == 3) {
    const S dmz = E.dmr[rz], dkz = E.dkr[rz];
    return S(1) / (cm * (dmx * dmy * dmz) + ck * (dkx * dmy * dmz + dmx * dky * dmz + dmx * dmy * dkz));
  } else {
    return S(1) / (cm * (dmx * dmy) + ck * (dkx * dmy + dmx * dky));
  }
}

// ---------------------------------------------------------------- 1D contractions
// y-direction banded taps for output row position R (compile time); col points at the
// output row in the staged input column, stride = row stride.
// (a, b) += (ca va, cb vb): a packed pair when PK, else two scalar multiply-adds (same result)
template <bool PK, typename T>
__device__ __forceinline__ void mad2p(T& a, T& b, T ca, T cb, T va, T vb) {
  if constexpr (PK) {
    mad2(a, b, ca, cb, va, vb);
  } else {
    a = mad(a, ca, va);
    b = mad(b, cb, vb);
  }
}

template <typename T, int K, int R, bool PK>
__device__ __forceinline__ void ytaps(const T* col, int stride, const OpParams<T>& P, T& g, T& h) {
  if constexpr (R == 0) {
#pragma unroll
    for (int o = -K; o <= K; ++o) {
      const T v = col[o * stride];
      mad2p<PK>(g, h, P.yvm[o + K], P.yvk[o + K], v, v);
    }
  } else {
#pragma unroll
    for (int m = 0; m <= K; ++m) {
      const T v = col[(m - R) * stride];
      mad2p<PK>(g, h, P.me[R][m], P.ke[R][m], v, v);
    }
  }
}

// y pass of one tile row with output row position R (compile time): the row's SL staged columns,
// 32 per step with this lane's column first (col, g, h point at it), every offset a constant;
// only the last step, when SL is not a multiple of 32, checks the lane.  FP32 unrolls every step;
// FP64 two at a time, which gives the FP64 pipe independent chains without the registers (and
// resident CTAs) that a full unroll costs.
template <typename T, int K, int R, bool PK, int SL>
__device__ __forceinline__ void yrow(const T* col, T* g, T* h, int lane, const OpParams<T>& P) {
  constexpr int IT = (SL + 31) / 32;
  constexpr int UNR = sizeof(T) == 8 ? 2 : IT;
#pragma unroll (UNR)
  for (int i = 0; i < IT; ++i) {
    if ((i + 1) * 32 <= SL || lane + 32 * i < SL) {
      T a = zero<T>(), b = zero<T>();
      ytaps<T, K, R, PK>(col + 32 * i, SL, P, a, b);
      g[32 * i] = a;
      h[32 * i] = b;
    }
  }
}

template <typename T, int K, bool PK, int SL, int R = 0>
__device__ __forceinline__ void yrow_dispatch(int r, const T* col, T* g, T* h, int lane, const OpParams<T>& P) {
  if constexpr (R < K) {
    if (r == R) yrow<T, K, R, PK, SL>(col, g, h, lane, P);
    else yrow_dispatch<T, K, PK, SL, R + 1>(r, col, g, h, lane, P);
  }
}

template <typename T, int K, bool PK, int R = 0>
__device__ __forceinline__ void ytaps_dispatch(int r, const T* col, int stride, const OpParams<T>& P,
                                               T& g, T& h) {
  if constexpr (R < K) {
    if (r == R) ytaps<T, K, R, PK>(col, stride, P, g, h);
    else ytaps_dispatch<T, K, PK, R + 1>(r, col, stride, P, g, h);
  }
}

// Cell-wise x contraction for one lane's cell (staged columns cl, cl+1 of slots [m][cell]).
// MODE3: g = My u, h = Ky u given -> R = Mx g, Pp = Kx g + Mx h.  MODE2: u given -> R = Mx u, Pp = Kx u.
template <typename T, int K, bool MODE3, int CW, bool PK>
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
    T a = zero<T>(), b = zero<T>();
#pragma unroll
    for (int m = 0; m <= K; ++m) {
      mad2p<PK>(a, b, P.me[mo][m], P.ke[mo][m], gv[m], gv[m]);
      if constexpr (MODE3) b = mad(b, P.me[mo][m], hv[m]);
    }
    r[mo] = a;
    p[mo] = b;
  }
}

// Top-vertex outputs (local node K) of the cell at staged column cl.
template <typename T, int K, bool MODE3, int CW, bool PK>
__device__ __forceinline__ void xcell_top(const T* g, const T* h, int cl, const OpParams<T>& P, T& r, T& p) {
  T a = zero<T>(), b = zero<T>();
#pragma unroll
  for (int m = 0; m <= K; ++m) {
    const int slot = (m < K) ? (m * CW + cl) : (cl + 1);
    const T gv = g[slot];
    mad2p<PK>(a, b, P.me[K][m], P.ke[K][m], gv, gv);
    if constexpr (MODE3) b = mad(b, P.me[K][m], h[slot]);
  }
  r = a;
  p = b;
}

// z push of column RZ (compile time) into the accumulators of the owned nodes.
template <typename T, int K, int RZ, bool DUAL, bool PK>
__device__ __forceinline__ void zpush(const OpParams<T>& P, T cm, T ck, const T (&R)[K], const T (&Pp)[K],
                                      T (&accA)[K][K + 1], T (&accB)[K][K + 1]) {
  if constexpr (PK && !DUAL) {
    T F[K], Ez[K];
#pragma unroll
    for (int m = 0; m < K; ++m) {
      F[m] = mad(mul(cm, R[m]), ck, Pp[m]);
      Ez[m] = mul(ck, R[m]);
    }
    // nodes m and m + 1 share the coefficients: one pair of multiply-adds per tap
#pragma unroll
    for (int m = 0; m + 1 < K; m += 2) {
#pragma unroll
      for (int mo = 0; mo <= K; ++mo) {
        mad2(accA[m][mo], accA[m + 1][mo], P.me[mo][RZ], P.me[mo][RZ], F[m], F[m + 1]);
        mad2(accA[m][mo], accA[m + 1][mo], P.ke[mo][RZ], P.ke[mo][RZ], Ez[m], Ez[m + 1]);
      }
    }
    if constexpr (K % 2 == 1) {
#pragma unroll
      for (int mo = 0; mo <= K; ++mo)
        accA[K - 1][mo] = mad(mad(accA[K - 1][mo], P.me[mo][RZ], F[K - 1]), P.ke[mo][RZ], Ez[K - 1]);
    }
  } else {
#pragma unroll
    for (int m = 0; m < K; ++m) {
      if constexpr (DUAL) {
#pragma unroll
        for (int mo = 0; mo <= K; ++mo) {
          if constexpr (PK) {
            mad2(accA[m][mo], accB[m][mo], P.me[mo][RZ], P.me[mo][RZ], R[m], Pp[m]);
            accB[m][mo] = mad(accB[m][mo], P.ke[mo][RZ], R[m]);
          } else {
            accA[m][mo] = mad(accA[m][mo], P.me[mo][RZ], R[m]);
            accB[m][mo] = mad(mad(accB[m][mo], P.me[mo][RZ], Pp[m]), P.ke[mo][RZ], R[m]);
          }
        }
      } else {
        const T F = mad(mul(cm, R[m]), ck, Pp[m]);
        const T Ez = mul(ck, R[m]);
#pragma unroll
        for (int mo = 0; mo <= K; ++mo) accA[m][mo] = mad(mad(accA[m][mo], P.me[mo][RZ], F), P.ke[mo][RZ], Ez);
      }
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
      accA[m][mo] = zero<T>();
      if constexpr (DUAL) accB[m][mo] = zero<T>();
    }
  }
}

// push of the plane with in-cell position r (0..K-1) into the accumulators; at a vertex plane
// (r = 0) the cell below is completed first (column K), emitted, and its top vertex carried.
template <typename T, int K, bool DUAL, bool PK, class Emit>
__device__ __forceinline__ void zstep(int r, int c, int cstart, int c0, const OpParams<T>& P, T cm, T ck,
                                      const T (&R)[K], const T (&Pp)[K], T (&accA)[K][K + 1], T (&accB)[K][K + 1],
                                      Emit&& emit) {
  if (r == 0) {
    if (c > cstart) {
      zpush<T, K, K, DUAL, PK>(P, cm, ck, R, Pp, accA, accB);
      if (c - 1 >= c0) emit(c - 1);
      carry<T, K, DUAL>(accA, accB);
    }
    zpush<T, K, 0, DUAL, PK>(P, cm, ck, R, Pp, accA, accB);
  } else if (r == 1) {
    zpush<T, K, (1 < K ? 1 : 0), DUAL, PK>(P, cm, ck, R, Pp, accA, accB);
  } else if (r == 2) {
    zpush<T, K, (2 < K ? 2 : 0), DUAL, PK>(P, cm, ck, R, Pp, accA, accB);
  } else {
    zpush<T, K, (3 < K ? 3 : 0), DUAL, PK>(P, cm, ck, R, Pp, accA, accB);
  }
}

}  // namespace dev

// Tile of a 3D CTA: CXS cells in x per warp segment (32, or 16 / 8 on meshes with fewer cells, so
// that no lane idles), 32 / CXS node rows per warp, K * CY node rows in y; the thread count is the
// same for every CXS.  FP32 CTAs hold 8 warps (K = 3: 6) and run 3 per SM; the FP64-accurate
// kernels, limited to one 8-warp CTA per SM by their register use, use CTAs of half the rows so
// that two of them share an SM and one computes while the other waits at its barrier.
template <typename T, int K> struct Warps3D {
  static constexpr int value = K * ((K == 1) ? 8 : (K == 2) ? 4 : 2) / (sizeof(T) == 4 ? 1 : 2);
};
template <typename T, int K, int CXS> struct Tile3D {
  static constexpr int CY = Warps3D<T, K>::value * (32 / CXS) / K;
};
// resident CTAs per SM requested from the register allocator: FP32 3 (24 warps per SM), at
// degree 3 4 CTAs of 6 warps (the kernel waits on loads: 24 warps hide more of that than 18)
template <typename T, int K> struct MinBlocks {
  static constexpr int value = (sizeof(T) == 4) ? (K == 3 ? 4 : 3) : 2;
};

// Shared-memory layout of the 3D kernel (dynamic): two staged planes, two y-pass outputs (g, h),
// the held bottom plane of a cluster chunk, and the 1/D table of the Chebyshev epilogue.
template <typename T, int K, int EPI, int CXS>
struct Op3dSmem {
  static constexpr int CY = Tile3D<T, K, CXS>::CY, TY = K * CY, NT = 32 * Warps3D<T, K>::value;
  static constexpr int CW = CXS + 2, SL = K * CW, HY = TY + K + 1;
  static constexpr int SU = HY * SL, SG = TY * SL, SHOLD = (EPI == EPI_DUAL ? 2 : 1) * K * NT;
  static constexpr int SINV = (EPI == EPI_CHEB) ? K * K * K : 1;
  // FP32 Chebyshev step and residual at degrees 2..3: the epilogue's operands of a z-cell (b; x_j,
  // x_{j-1}), fetched asynchronously while the cell streams (at degree 4 the extra shared memory
  // would cost a resident CTA)
  static constexpr bool PRE =
      std::is_same<T, float>::value && K >= 2 && K <= 3 && (EPI == EPI_CHEB || EPI == EPI_RESID);
  static constexpr int NPRE = (EPI == EPI_CHEB) ? 3 : 1;
  static constexpr int SPRE = PRE ? NPRE * K * K * NT : 0;
  static constexpr size_t bytes = (size_t)(2 * SU + 4 * SG + SHOLD) * sizeof(T) +
                                  (size_t)(SINV + SPRE) * sizeof(typename Storage<T>::type);
};

// ---------------------------------------------------------------- 3D kernel
template <typename T, int K, int EPI, int CXS>
__global__ void __launch_bounds__(32 * Warps3D<T, K>::value, MinBlocks<T, K>::value)
op3d_kernel(const typename Storage<T>::type* __restrict__ u, const OpParams<T> P,
            const EpiParams<typename Storage<T>::type> E) {
  dev::pdl_enter();
  using S = typename Storage<T>::type;
  constexpr int RPW = 32 / CXS;  // node rows per warp
  constexpr int CY = Tile3D<T, K, CXS>::CY;
  constexpr int CX = CXS, TY = K * CY, NT = 32 * Warps3D<T, K>::value;
  constexpr int CW = CX + 2, SL = K * CW;
  constexpr int HY = TY + K + 1, HX = K * CX + K + 1;
  constexpr int NLD = HY * HX;
  constexpr int PF = (NLD + NT - 1) / NT;
  constexpr bool DUAL = (EPI == EPI_DUAL);
  // packed pairs of multiply-adds, except FP32 DUAL (only on the coupled-block path), where the
  // pairing constraints on the allocator raise the spills at this kernel's register cap
  constexpr bool PK = !(DUAL && sizeof(T) == 4);
  using L = Op3dSmem<T, K, EPI, CXS>;
  extern __shared__ __align__(16) unsigned char op_smem[];
  T* const su2 = reinterpret_cast<T*>(op_smem);  // two staged planes (double buffer)
  T* const sg2 = su2 + 2 * L::SU;                 // two y-pass outputs g
  T* const sh2 = sg2 + 2 * L::SG;                 // two y-pass outputs h
  T* const shold = sh2 + 2 * L::SG;               // bottom plane held for the cluster exchange
  S* const sinvd = reinterpret_cast<S*>(shold + L::SHOLD);  // 1/D by (x, y, z) mod k
  S* const spre = sinvd + L::SINV;                          // prefetched epilogue operands
  T* const sg = sg2;  // buffer 0 doubles as the cluster exchange area
  T* const sh = sh2;

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int N = P.N, n1 = P.n1;
  const int cx0 = blockIdx.x * CX;
  const int zchunk = blockIdx.y % P.nch, ty = blockIdx.y / P.nch;
  const int y0 = K * CY * ty, x0 = K * cx0;
  const int s = blockIdx.z;
  const S* __restrict__ us = u + (long long)s * P.ld;
  const T cm = P.cm[s], ck = P.ck[s];
  const bool clustered = P.cluster != 0;
  const int c0 = zchunk * P.zc;
  if (!clustered && c0 >= N) return;  // a cluster's chunks are all non-empty (launcher)
  const int c1 = min(N, c0 + P.zc);
  const int cstart = clustered ? c0 : max(c0 - 1, 0);
  const bool hold_bottom = clustered && c0 > 0;  // bottom vertex plane waits for the lower chunk
  const long long plane = (long long)n1 * n1;

  for (int i = tid; i < 2 * HY * SL; i += NT) su2[i] = dev::zero<T>();  // padding slots stay zero
  if constexpr (EPI == EPI_CHEB) {
    if (tid < K * K * K) {
      const int rx = tid % K, ry = (tid / K) % K, rz = tid / (K * K);
      sinvd[tid] = dev::inv_diag<S, 3>(E, (S)P.cm[s], (S)P.ck[s], rx, ry, rz);
    }
  }

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
    const S* base = us + zp * plane;
#pragma unroll
    for (int q = 0; q < PF; ++q) pf[q] = (goff[q] >= 0) ? dev::load<T>(base + goff[q]) : dev::zero<T>();
  };
  auto store_plane = [&](int buf) {
    T* su = su2 + buf * L::SU;
#pragma unroll
    for (int q = 0; q < PF; ++q)
      if ((q + 1) * NT <= NLD || soff[q] >= 0) su[soff[q]] = pf[q];  // only the last slot can be empty
  };
  // FP32 levels (F32; not the dual products at degree 4, which would spill) and FP64: the warp's
  // rows with every offset a constant (this lane's first output slot; the input column sits K rows
  // lower); float-float keeps the rolled loop
  constexpr bool F32 = std::is_same<T, float>::value && (K <= 3 || EPI != EPI_DUAL);
  constexpr bool YCONST = F32 || std::is_same<T, double>::value;
  const int yout0 = w * RPW * SL + lane;
  auto ypass = [&](int buf) {
    const T* su = su2 + buf * L::SU;
    T* sgb = sg2 + buf * L::SG;
    T* shb = sh2 + buf * L::SG;
    if constexpr (YCONST) {
#pragma unroll 1
      for (int rr = 0; rr < RPW; ++rr) {  // the warp's rows one at a time (warp-uniform tap row)
        const int o = yout0 + rr * SL;
        dev::yrow_dispatch<T, K, PK, SL>((w * RPW + rr) % K, su + K * SL + o, sgb + o, shb + o, lane, P);
      }
    } else {
#pragma unroll 1
      for (int rr = 0; rr < RPW; ++rr) {  // the warp's rows, one at a time (warp-uniform tap row)
        const int yr = w * RPW + rr;
        const int ro = yr % K;
        const T* colbase = su + (yr + K) * SL;
        for (int sl = lane; sl < SL; sl += 32) {
          T g = dev::zero<T>(), h = dev::zero<T>();
          dev::ytaps_dispatch<T, K, PK>(ro, colbase + sl, SL, P, g, h);
          sgb[yr * SL + sl] = g;
          shb[yr * SL + sl] = h;
        }
      }
    }
  };
  const int seg = lane / CXS, lx = lane - seg * CXS;
  const int trow = w * RPW + seg;  // this thread's node row in the tile
  auto xpass = [&](int buf, T (&R)[K], T (&Pp)[K]) {
    const T* g = sg2 + buf * L::SG + trow * SL;
    const T* h = sh2 + buf * L::SG + trow * SL;
    T r[K + 1], p[K + 1];
    dev::xcell<T, K, true, CW, PK>(g, h, lx + 1, P, r, p);
    T rl = dev::shfl_up(r[K]);
    T pl = dev::shfl_up(p[K]);
    if (lx == 0) {  // the cell left of the tile: none at the domain's left boundary
      if (cx0 > 0) {
        dev::xcell_top<T, K, true, CW, PK>(g, h, 0, P, rl, pl);
      } else {
        rl = dev::zero<T>();
        pl = dev::zero<T>();
      }
    }
    r[0] = dev::add(r[0], rl);
    p[0] = dev::add(p[0], pl);
#pragma unroll
    for (int m = 0; m < K; ++m) { R[m] = r[m]; Pp[m] = p[m]; }
  };
  const int yrow = y0 + trow;
  const int cell = cx0 + lx;
  const bool row_ok = (yrow >= 1 && yrow <= n1 - 2) && (cell < N);
  T accA[K][K + 1], accB[K][K + 1];
#pragma unroll
  for (int m = 0; m < K; ++m)
#pragma unroll
    for (int mo = 0; mo <= K; ++mo) { accA[m][mo] = dev::zero<T>(); accB[m][mo] = dev::zero<T>(); }

  // the thread's output nodes (z, yrow, K cell + m) sit at rowbase + z * n1^2 + m in stage s
  // (32-bit offsets within a stage vector; the stage offset is uniform across the CTA).  F32: the
  // row start, the stage's Chebyshev coefficients and this row's part of the 1/D table are fixed
  // for the kernel, and the operands' addresses are formed once per plane.
  const int rowbase = yrow * n1 + K * cell;
  const int plane32 = n1 * n1;
  const long long sbase = (long long)s * P.ld;
  const long long rowstart = sbase + rowbase;
  S ec1{}, ec2{};
  if constexpr (F32 && EPI == EPI_CHEB) {
    ec1 = E.c1[s];
    ec2 = E.c2[s];
  }
  const int sinv_row = (yrow % K) * K;
  // prefetch slots: operand a (b, x_j, x_{j-1}) of node (mo, m) of this thread at
  // spre[((a K + mo) K + m) NT + tid]; x_{j-1} only when the momentum term reads it
  constexpr bool PRE = L::PRE;
  bool need_old = false;
  if constexpr (PRE && EPI == EPI_CHEB) need_old = ec1 != 0.0f && !E.xold_zero;
  auto prefetch = [&](int cz) {  // the operands of cell cz's emitted nodes (emit below)
    if constexpr (PRE) {
      if (!row_ok) return;
#pragma unroll
      for (int mo = 0; mo < K; ++mo) {
        const int z = K * cz + mo;
        if (z < 1 || (mo == 0 && hold_bottom && cz == c0)) continue;
        const long long o = rowstart + (long long)(z * plane32);
#pragma unroll
        for (int m = 0; m < K; ++m) {
          if (m == 0 && cell == 0) continue;
          const int slot = (mo * K + m) * NT + tid;
          dev::cp_async4(spre + slot, (E.b + o) + m);
          if constexpr (EPI == EPI_CHEB) {
            dev::cp_async4(spre + K * K * NT + slot, (E.xj + o) + m);
            if (need_old) dev::cp_async4(spre + 2 * K * K * NT + slot, (E.out + o) + m);
          }
        }
      }
    }
  };
  auto emit_node = [&](int z, int m, int mo, T va, T vb, bool pre = false) {
    if (m == 0 && cell == 0) return;  // x = 0: boundary node
    S invD{};
    if constexpr (PRE) {
      if (pre) {
        const int slot = (mo * K + m) * NT + tid;
        const long long o = rowstart + (long long)(z * plane32);
        const S bv = spre[slot];
        if constexpr (EPI == EPI_RESID) {
          (E.out + o)[m] = bv - dev::to_storage(va);
        } else {
          const S xv = spre[K * K * NT + slot];
          S upd = S(0);
          if (ec1 != S(0)) upd = ec1 * (xv - (need_old ? spre[2 * K * K * NT + slot] : S(0)));
          invD = sinvd[sinv_row + mo * K * K + m];
          (E.out + o)[m] = xv + upd + ec2 * (bv - dev::to_storage(va)) * invD;
        }
        return;
      }
    }
    if constexpr (F32) {
      if constexpr (EPI == EPI_CHEB) invD = sinvd[sinv_row + mo * K * K + m];
      const long long o = rowstart + (long long)(z * plane32);
      dev::epilogue_at<T, EPI>((E.out + o) + m, EPI == EPI_DUAL ? (E.out2 + o) + m : nullptr,
                               (EPI == EPI_RESID || EPI == EPI_CHEB) ? (E.b + o) + m : nullptr,
                               EPI == EPI_CHEB ? (E.xj + o) + m : nullptr, E.xold_zero, ec1, ec2, va, vb, invD);
    } else {
      if constexpr (EPI == EPI_CHEB) invD = sinvd[(mo * K + (yrow % K)) * K + m];
      dev::epilogue<T, EPI>(E, sbase + (rowbase + z * plane32 + m), s, va, vb, invD);
    }
  };
  auto emit = [&](int cz) {
    if (!row_ok) return;
    if constexpr (PRE) dev::cp_async_wait_all();  // this thread's prefetched operands of cell cz
#pragma unroll
    for (int mo = 0; mo < K; ++mo) {
      const int z = K * cz + mo;
      if (z < 1) continue;
      if (mo == 0 && hold_bottom && cz == c0) {  // completed after the cluster exchange
#pragma unroll
        for (int m = 0; m < K; ++m) {
          shold[m * NT + tid] = accA[m][0];
          if constexpr (DUAL) shold[(K + m) * NT + tid] = accB[m][0];
        }
        continue;
      }
#pragma unroll
      for (int m = 0; m < K; ++m) emit_node(z, m, mo, accA[m][mo], accB[m][mo], true);
    }
  };

  // Two-stage pipeline over the planes z0 .. zlast with one barrier per plane: in the interval of
  // plane zp the y pass of zp, the x pass and z push of zp - 1, the store of zp + 1 (prefetched one
  // plane earlier) and the load of zp + 2 run together; planes alternate between two buffers.
  const int z0 = K * cstart, zlast = K * c1;
  __syncthreads();
  load_plane(z0);
  store_plane(0);
  load_plane(z0 + 1);
  __syncthreads();
  ypass(0);
  store_plane(1);
  if (z0 + 2 <= zlast) load_plane(z0 + 2);
  __syncthreads();
  for (int c = cstart; c < c1; ++c) {
#pragma unroll
    for (int r = 0; r < K; ++r) {
      const int zp = K * c + r + 1;  // plane of this interval's y pass; x pass and z push: zp - 1
      const int buf = (zp - z0) & 1;
      ypass(buf);
      T R[K], Pp[K];
      xpass(buf ^ 1, R, Pp);
      dev::zstep<T, K, DUAL, PK>(r, c, cstart, c0, P, cm, ck, R, Pp, accA, accB, emit);
      // cell c's operands, one barrier after emit(c - 1) read the slots: K - 1 planes ahead
      if (PRE && r == 1 && c >= c0) prefetch(c);
      if (zp + 1 <= zlast) {
        store_plane(buf ^ 1);
        if (zp + 2 <= zlast) load_plane(zp + 2);
      }
      __syncthreads();
    }
  }
  {  // upper vertex plane of the last cell
    T R[K], Pp[K];
    xpass((zlast - z0) & 1, R, Pp);
    dev::zpush<T, K, K, DUAL, PK>(P, cm, ck, R, Pp, accA, accB);
    if (c1 - 1 >= c0) emit(c1 - 1);
  }
  if (clustered) {
    // accA[.][K] (accB) now hold the last cell's contributions to the vertex plane above the
    // chunk: publish them in this CTA's (now idle) staging buffers for the chunk above
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    __syncthreads();
#pragma unroll
    for (int m = 0; m < K; ++m) {
      sg[m * NT + tid] = accA[m][K];
      if constexpr (DUAL) sh[m * NT + tid] = accB[m][K];
    }
    cluster.sync();
    if (hold_bottom && row_ok) {
      const unsigned below = cluster.block_rank() - 1;
      const T* ca = cluster.map_shared_rank(sg, below);
      const T* cb = DUAL ? cluster.map_shared_rank(sh, below) : nullptr;
      const int z = K * c0;
#pragma unroll
      for (int m = 0; m < K; ++m) {
        const T va = dev::add(shold[m * NT + tid], ca[m * NT + tid]);
        T vb = dev::zero<T>();
        if constexpr (DUAL) vb = dev::add(shold[(K + m) * NT + tid], cb[m * NT + tid]);
        emit_node(z, m, 0, va, vb);
      }
    }
    cluster.sync();  // the chunk above has read this CTA's shared memory
  }
}

// ---------------------------------------------------------------- 2D kernel
// Plane = one x row; streaming along y.  NW warps, 32*NW cells per tile in x.
template <typename T, int K, int EPI>
__global__ void __launch_bounds__(64)
op2d_kernel(const typename Storage<T>::type* __restrict__ u, const OpParams<T> P,
            const EpiParams<typename Storage<T>::type> E) {
  dev::pdl_enter();
  using S = typename Storage<T>::type;
  constexpr int NW = 2, NT = 32 * NW;
  constexpr int CX = 32 * NW, CW = CX + 2, SL = K * CW;
  constexpr int HX = K * CX + K + 1;
  constexpr int PF = (HX + NT - 1) / NT;
  constexpr bool DUAL = (EPI == EPI_DUAL);
  constexpr bool PK = false;  // scalar multiply-adds: the packed pairs spill the degree-4 kernels here
  __shared__ T su[SL];

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int N = P.N, n1 = P.n1;
  const int cx0 = blockIdx.x * CX, x0 = K * cx0;
  const int s = blockIdx.z;
  const S* __restrict__ us = u + (long long)s * P.ld;
  const T cm = P.cm[s], ck = P.ck[s];
  const int c0 = blockIdx.y * P.zc;
  if (c0 >= N) return;
  const int c1 = min(N, c0 + P.zc);
  const int cstart = max(c0 - 1, 0);

  for (int i = tid; i < SL; i += NT) su[i] = dev::zero<T>();
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
    const S* base = us + (long long)yp * n1;
#pragma unroll
    for (int q = 0; q < PF; ++q) pf[q] = (goff[q] >= 0) ? dev::load<T>(base + goff[q]) : dev::zero<T>();
  };
  auto store_row = [&]() {
#pragma unroll
    for (int q = 0; q < PF; ++q)
      if (soff[q] >= 0) su[soff[q]] = pf[q];
  };
  const int cl = w * 32 + lane + 1;
  auto xpass = [&](T (&R)[K], T (&Pp)[K]) {
    T r[K + 1], p[K + 1];
    dev::xcell<T, K, false, CW, PK>(su, su, cl, P, r, p);
    T rl = dev::shfl_up(r[K]);
    T pl = dev::shfl_up(p[K]);
    if (lane == 0) dev::xcell_top<T, K, false, CW, PK>(su, su, cl - 1, P, rl, pl);
    r[0] = dev::add(r[0], rl);
    p[0] = dev::add(p[0], pl);
#pragma unroll
    for (int m = 0; m < K; ++m) { R[m] = r[m]; Pp[m] = p[m]; }
  };
  const int cell = cx0 + w * 32 + lane;
  const bool col_ok = cell < N;
  T accA[K][K + 1], accB[K][K + 1];
#pragma unroll
  for (int m = 0; m < K; ++m)
#pragma unroll
    for (int mo = 0; mo <= K; ++mo) { accA[m][mo] = dev::zero<T>(); accB[m][mo] = dev::zero<T>(); }
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
        S invD{};
        if constexpr (EPI == EPI_CHEB) invD = dev::inv_diag<S, 2>(E, (S)P.cm[s], (S)P.ck[s], m, mo, 0);
        dev::epilogue<T, EPI>(E, (long long)s * P.ld + idx, s, accA[m][mo], accB[m][mo], invD);
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
      dev::zstep<T, K, DUAL, PK>(r, c, cstart, c0, P, cm, ck, R, Pp, accA, accB, emit);
    }
  }
  __syncthreads();
  store_row();
  __syncthreads();
  {
    T R[K], Pp[K];
    xpass(R, Pp);
    dev::zpush<T, K, K, DUAL, PK>(P, cm, ck, R, Pp, accA, accB);
    if (c1 - 1 >= c0) emit(c1 - 1);
  }
}

template <typename T> const char* tune_kernel_name();
template <> inline const char* tune_kernel_name<float>() { return "op3d<float>"; }
template <> inline const char* tune_kernel_name<double>() { return "op3d<double>"; }
template <> inline const char* tune_kernel_name<ff>() { return "op3d<ff>"; }

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

constexpr int kMaxClusterChunks = 16;  // z chunks per thread-block cluster (above 8: non-portable size)

// Clusters of nch CTAs of this kernel that fit on the device at once (0: not launchable as a cluster).
template <typename Kern>
int max_active_clusters(Kern kern, int nch, int threads, dim3 grid, size_t smem) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = nch;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (nch > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// Launch shape of the 3D kernel: warp-segment width (cells), z chunk (cells), cluster mode.
struct OpShape {
  int cxs = 32, zc = 1, cluster = 0;
};

// Per kernel instantiation: dynamic shared memory (opted in once above the 48 KB default),
// occupancy and cluster fit, queried once.
template <typename T, int K, int EPI, int CXS>
struct Op3dInfo {
  static constexpr size_t smem = Op3dSmem<T, K, EPI, CXS>::bytes;
  static bool smem_ready() {
    static int ok = -1;
    if (ok < 0) {
      ok = 1;
      if (smem > 48 * 1024 &&
          cudaFuncSetAttribute(op3d_kernel<T, K, EPI, CXS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem) != cudaSuccess) {
        cudaGetLastError();
        ok = 0;
      }
    }
    return ok == 1;
  }
  static int occ() {
    static int o = 0;
    if (o == 0) {
      smem_ready();
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, op3d_kernel<T, K, EPI, CXS>, 32 * Warps3D<T, K>::value, smem);
      if (o < 1) o = 1;
    }
    return o;
  }
  // clusters of nch chunks that fit on the device at once (0: not launchable as a cluster)
  static int clusters_fit(int nch, dim3 grid) {
    static int fit[kMaxClusterChunks + 1] = {-1, -1, -1, -1, -1, -1, -1, -1, -1,
                                             -1, -1, -1, -1, -1, -1, -1, -1};
    if (nch < 2 || nch > kMaxClusterChunks) return 0;
    if (fit[nch] < 0) {
      smem_ready();
      fit[nch] = max_active_clusters(op3d_kernel<T, K, EPI, CXS>, nch, 32 * Warps3D<T, K>::value, grid, smem);
    }
    return fit[nch];
  }
};

// Cost model: waves x planes streamed per CTA (a chunk off the bottom re-streams the cell below it
// unless its tile's chunks form a cluster).
template <typename T, int K, int EPI, int CXS>
OpShape model_shape(int N, int nstage) {
  using I = Op3dInfo<T, K, EPI, CXS>;
  const int ntx = (N + CXS - 1) / CXS, nty = (N + Tile3D<T, K, CXS>::CY - 1) / Tile3D<T, K, CXS>::CY;
  const long long base = (long long)ntx * nty * nstage;
  const long long slots = (long long)I::occ() * device_sm_count();
  OpShape best;
  best.cxs = CXS;
  long long best_cost = -1;
  for (int zc = 1; zc <= N; ++zc) {
    const int nch = (N + zc - 1) / zc;
    const long long waves = (base * nch + slots - 1) / slots;
    const long long cost = waves * ((long long)K * (zc + (nch > 1 ? 1 : 0)) + 1);
    if (best_cost < 0 || cost < best_cost) { best_cost = cost; best.zc = zc; best.cluster = 0; }
    const int fit = I::clusters_fit(nch, dim3(ntx, nty * nch, nstage));
    if (fit > 0) {
      const long long cw = (base + fit - 1) / fit;
      const long long ccost = cw * ((long long)K * zc + 1);
      if (ccost < best_cost) { best_cost = ccost; best.zc = zc; best.cluster = 1; }
    }
  }
  return best;
}

template <typename T, int K, int EPI, int CXS>
cudaError_t launch_shape(int nstage, const typename Storage<T>::type* u, const OpParams<T>& P,
                         const EpiParams<typename Storage<T>::type>& E, cudaStream_t st, const OpShape& sh) {
  using I = Op3dInfo<T, K, EPI, CXS>;
  auto kern = op3d_kernel<T, K, EPI, CXS>;
  const int threads = 32 * Warps3D<T, K>::value;
  if (!I::smem_ready()) return cudaErrorInvalidValue;
  OpParams<T> Q = P;
  const int ntx = (P.N + CXS - 1) / CXS;
  Q.ntile_y = (P.N + Tile3D<T, K, CXS>::CY - 1) / Tile3D<T, K, CXS>::CY;
  Q.zc = sh.zc;
  Q.nch = (P.N + Q.zc - 1) / Q.zc;
  Q.cluster = sh.cluster;
  dim3 grid(ntx, Q.ntile_y * Q.nch, nstage);
  op_shape_record(sizeof(T) == 4 ? 4 : 8, CXS, Q.zc, Q.cluster, Q.nch);
  if (!Q.cluster) {
    kern<<<grid, threads, I::smem, st>>>(u, Q, E);  // a plain launch (pdl.cuh)
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = I::smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = Q.nch;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, u, Q, E);
}

// Process-wide autotuned shapes per kernel instantiation, keyed by (cells per axis, stages).
template <typename T, int K, int EPI>
struct OpTuned {
  static std::mutex& mu() { static std::mutex m; return m; }
  static std::map<long long, OpShape>& table() { static std::map<long long, OpShape> t; return t; }
  static long long key(int N, int ns) { return ((long long)N << 8) | ns; }
  static bool find(int N, int ns, OpShape& out) {
    std::lock_guard<std::mutex> lock(mu());
    auto it = table().find(key(N, ns));
    if (it == table().end()) return false;
    out = it->second;
    return true;
  }
  static void put(int N, int ns, const OpShape& sh) {
    std::lock_guard<std::mutex> lock(mu());
    table()[key(N, ns)] = sh;
  }
};

template <typename T> constexpr bool narrow_tiles() { return sizeof(T) == 4; }  // FP32 levels only
inline int default_cxs(int N) { return N <= 8 ? 8 : (N <= 16 ? 16 : 32); }

template <typename T, int K, int EPI>
OpShape default_shape(int N, int nstage) {
  if constexpr (narrow_tiles<T>()) {
    const int c = default_cxs(N);
    if (c == 8) return model_shape<T, K, EPI, 8>(N, nstage);
    if (c == 16) return model_shape<T, K, EPI, 16>(N, nstage);
  }
  return model_shape<T, K, EPI, 32>(N, nstage);
}

template <typename T, int K, int EPI>
cudaError_t launch_by_shape(int nstage, const typename Storage<T>::type* u, const OpParams<T>& P,
                            const EpiParams<typename Storage<T>::type>& E, cudaStream_t st, const OpShape& sh) {
  if constexpr (narrow_tiles<T>()) {
    if (sh.cxs == 8) return launch_shape<T, K, EPI, 8>(nstage, u, P, E, st, sh);
    if (sh.cxs == 16) return launch_shape<T, K, EPI, 16>(nstage, u, P, E, st, sh);
  }
  return launch_shape<T, K, EPI, 32>(nstage, u, P, E, st, sh);
}

template <typename T, int K, int EPI>
cudaError_t launch_op_k(int dim, int nstage, const typename Storage<T>::type* u, const OpParams<T>& P,
                        const EpiParams<typename Storage<T>::type>& E, cudaStream_t st) {
  if (dim == 3) {
    OpShape sh;
    if (op_shape_forced(sizeof(T) == 4 ? 4 : 8, &sh.cxs, &sh.zc, &sh.cluster)) {
      // a forced shape (test support) runs only where this kernel supports it
      if (sh.cxs != 32 && !(narrow_tiles<T>() && (sh.cxs == 8 || sh.cxs == 16))) return cudaErrorInvalidValue;
      if (sh.zc < 1) return cudaErrorInvalidValue;
      if (sh.cluster) {
        const int nch = (P.N + sh.zc - 1) / sh.zc;
        const int cy = (sh.cxs == 8) ? Tile3D<T, K, 8>::CY : (sh.cxs == 16) ? Tile3D<T, K, 16>::CY : Tile3D<T, K, 32>::CY;
        const dim3 grid((P.N + sh.cxs - 1) / sh.cxs, ((P.N + cy - 1) / cy) * nch, nstage);
        int fit = 0;
        if constexpr (narrow_tiles<T>()) {
          fit = (sh.cxs == 8) ? Op3dInfo<T, K, EPI, 8>::clusters_fit(nch, grid)
                : (sh.cxs == 16) ? Op3dInfo<T, K, EPI, 16>::clusters_fit(nch, grid)
                                 : Op3dInfo<T, K, EPI, 32>::clusters_fit(nch, grid);
        } else {
          fit = Op3dInfo<T, K, EPI, 32>::clusters_fit(nch, grid);
        }
        if (fit <= 0) return cudaErrorInvalidConfiguration;
      }
    } else {
      const int key = P.shape_ns > 0 ? P.shape_ns : nstage;
      if (!OpTuned<T, K, EPI>::find(P.N, key, sh)) sh = default_shape<T, K, EPI>(P.N, key);
    }
    return launch_by_shape<T, K, EPI>(nstage, u, P, E, st, sh);
  }
  int cx, cy;
  op_tile_shape_impl(dim, K, &cx, &cy);
  const int ntx = (P.N + cx - 1) / cx;
  OpParams<T> Q = P;
  static int occ = 0;
  if (occ == 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, op2d_kernel<T, K, EPI>, 64, 0);
    if (occ < 1) occ = 1;
  }
  if (Q.zc <= 0) Q.zc = pick_zc(P.N, (long long)ntx * nstage, (long long)occ * device_sm_count(), K);
  const int nch = (P.N + Q.zc - 1) / Q.zc;
  dim3 grid(ntx, nch, nstage);
  launch_pdl(op2d_kernel<T, K, EPI>, grid, 64, 0, st, u, Q, E);
  return cudaGetLastError();
}

// Autotuner of the 3D launch shape: times the candidate shapes (segment width, z chunk, cluster
// mode) of this kernel on the call's own arguments and keeps the fastest for every later launch
// of the same kernel, cells per axis and stage count.  The call's outputs must be scratch (the
// candidates run repeatedly); levels below kTuneMinNodes stage-nodes keep the model's shape.
constexpr long long kTuneMinNodes = 1 << 18;

template <typename T, int K, int EPI>
cudaError_t tune_op_k(int dim, int nstage, const typename Storage<T>::type* u, const OpParams<T>& P,
                      const EpiParams<typename Storage<T>::type>& E, cudaStream_t st) {
  if (dim != 3) return cudaSuccess;
  const int key = P.shape_ns > 0 ? P.shape_ns : nstage;  // the shape is kept per stage count of a request
  OpShape known;
  if (OpTuned<T, K, EPI>::find(P.N, key, known)) return cudaSuccess;
  const long long nodes = (long long)P.n1 * P.n1 * P.n1 * nstage;
  const OpShape model = default_shape<T, K, EPI>(P.N, key);
  if (nodes < kTuneMinNodes) {
    OpTuned<T, K, EPI>::put(P.N, key, model);
    return cudaSuccess;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return cudaSuccess;
  // one tuning at a time per kernel: a second thread waits, then finds the shape cached
  static std::mutex tune_mu;
  std::lock_guard<std::mutex> tune_lock(tune_mu);
  if (OpTuned<T, K, EPI>::find(P.N, key, known)) return cudaSuccess;
  // candidates: the model's segment width (and 32 for FP32 levels), every distinct chunk count,
  // with and without a cluster where one fits
  std::vector<OpShape> cands;
  std::vector<int> widths = {model.cxs};
  if (model.cxs != 32) widths.push_back(32);
  for (int cxs : widths) {
    int last_nch = -1;
    for (int zc = 1; zc <= P.N; ++zc) {
      const int nch = (P.N + zc - 1) / zc;
      if (nch == last_nch) continue;
      last_nch = nch;
      OpShape c;
      c.cxs = cxs;
      c.zc = zc;
      c.cluster = 0;
      cands.push_back(c);
      if (nch >= 2 && nch <= kMaxClusterChunks) {
        c.cluster = 1;
        cands.push_back(c);
      }
    }
  }
  // drop the cluster shapes the device cannot hold
  std::vector<OpShape> ok;
  for (const OpShape& c : cands) {
    if (c.cluster) {
      const int cy = (c.cxs == 8) ? Tile3D<T, K, 8>::CY : (c.cxs == 16) ? Tile3D<T, K, 16>::CY : Tile3D<T, K, 32>::CY;
      const int nch = (P.N + c.zc - 1) / c.zc;
      const dim3 grid((P.N + c.cxs - 1) / c.cxs, ((P.N + cy - 1) / cy) * nch, nstage);
      int fit = 0;
      if constexpr (narrow_tiles<T>()) {
        fit = (c.cxs == 8) ? Op3dInfo<T, K, EPI, 8>::clusters_fit(nch, grid)
              : (c.cxs == 16) ? Op3dInfo<T, K, EPI, 16>::clusters_fit(nch, grid)
                              : Op3dInfo<T, K, EPI, 32>::clusters_fit(nch, grid);
      } else {
        fit = Op3dInfo<T, K, EPI, 32>::clusters_fit(nch, grid);
      }
      if (fit <= 0) continue;
    }
    ok.push_back(c);
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cudaGetLastError();
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return cudaGetLastError(); }
  // warm-up: bring the clocks to their working point on the model shape (about 2 ms of launches)
  {
    float ms = 0.f;
    for (int r = 0; r < 200 && ms < 2.f; ++r) {
      cudaEventRecord(e0, st);
      launch_by_shape<T, K, EPI>(nstage, u, P, E, st, model);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) break;
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      ms += t;
    }
  }
  // three rounds over all candidates (interleaved, so a slow moment hits every shape), best of
  // three per shape, each sample the mean of three launches
  std::vector<float> best_of(ok.size(), -1.f);
  for (int round = 0; round < 3; ++round) {
    for (size_t i = 0; i < ok.size(); ++i) {
      if (round > 0 && best_of[i] < 0.f) continue;  // failed to launch
      if (launch_by_shape<T, K, EPI>(nstage, u, P, E, st, ok[i]) != cudaSuccess) {  // warm-up
        cudaGetLastError();
        continue;
      }
      cudaEventRecord(e0, st);
      for (int r = 0; r < 3; ++r) launch_by_shape<T, K, EPI>(nstage, u, P, E, st, ok[i]);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= 3.f;
      if (best_of[i] < 0.f || ms < best_of[i]) best_of[i] = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the model's shape stays unless a candidate beats it by more than 3 %
  OpShape best = model;
  float best_ms = -1.f, model_ms = -1.f;
  for (size_t i = 0; i < ok.size(); ++i)
    if (ok[i].cxs == model.cxs && ok[i].zc == model.zc && ok[i].cluster == model.cluster) model_ms = best_of[i];
  best_ms = model_ms;
  for (size_t i = 0; i < ok.size(); ++i) {
    if (best_of[i] < 0.f) continue;
    if (best_ms < 0.f || best_of[i] < 0.97f * best_ms) { best_ms = best_of[i]; best = ok[i]; }
  }
  const cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  OpTuned<T, K, EPI>::put(P.N, key, best);
  tune_record(tune_kernel_name<T>(), K, EPI, P.N, key, best.cxs, best.zc, best.cluster, 1e3 * best_ms,
              model_ms < 0.f ? -1.0 : 1e3 * model_ms, model.cxs, model.zc, model.cluster);
  return cudaSuccess;
}

template <typename T, int EPI>
cudaError_t launch_op_e(int dim, int k, int nstage, const typename Storage<T>::type* u, const OpParams<T>& P,
                        const EpiParams<typename Storage<T>::type>& E, cudaStream_t st) {
  switch (k) {
    case 1: return launch_op_k<T, 1, EPI>(dim, nstage, u, P, E, st);
    case 2: return launch_op_k<T, 2, EPI>(dim, nstage, u, P, E, st);
    case 3: return launch_op_k<T, 3, EPI>(dim, nstage, u, P, E, st);
    case 4: return launch_op_k<T, 4, EPI>(dim, nstage, u, P, E, st);
    default: return cudaErrorInvalidValue;
  }
}


template <typename T, int EPI>
cudaError_t tune_op_e(int dim, int k, int nstage, const typename Storage<T>::type* u, const OpParams<T>& P,
                      const EpiParams<typename Storage<T>::type>& E, cudaStream_t st) {
  switch (k) {
    case 1: return tune_op_k<T, 1, EPI>(dim, nstage, u, P, E, st);
    case 2: return tune_op_k<T, 2, EPI>(dim, nstage, u, P, E, st);
    case 3: return tune_op_k<T, 3, EPI>(dim, nstage, u, P, E, st);
    case 4: return tune_op_k<T, 4, EPI>(dim, nstage, u, P, E, st);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace irk
