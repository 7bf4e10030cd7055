// 3D level operator for meshes of few cells per axis (the coarse multigrid levels, sm_103a).
//
// The z-streaming operator kernel (op_kernels.cuh) walks a chunk of planes one after the other;
// on a level of 4 or 8 cells per axis each CTA streams a handful of planes and spends the launch
// waiting for one plane load after another.  Here one CTA per (cell, stage) computes the outputs
// at the k^3 nodes the cell owns (local index 0..k-1 on each axis; the last node of every axis is
// a boundary node) from the (2k+1)^3 block of nodes around them (the cell and its three lower
// neighbours), so that every load of the launch is in flight at once.  The operator is the same
// tensor-product form cm M + ck K with the assembled 1D rows (a vertex row couples 2k+1 nodes
// through both adjacent cells, an inner row the k+1 nodes of its cell), applied by sum
// factorisation in three axis passes over the block in shared memory, with the same fused
// epilogues (store, residual, Chebyshev step) as the streaming kernel.
#pragma once
#include "op_kernels.cuh"

namespace irk {

// levels with at most this many cells per axis take the cell kernel (FP32 multigrid levels)
constexpr int kCellKernelMaxN = 8;

namespace dev {

// 1D row of the assembled operator at owned position r (0..B K - 1) of a block of B cells whose
// node block starts K nodes below the first owned node: returns sum_taps (mass, stiffness) of
// src[local * stride], local in 0..(B+1) K.
template <typename T, int K>
__device__ __forceinline__ void cell_row(const T* src, int stride, int r, const OpParams<T>& P, T& m, T& k) {
  T a = zero<T>(), b = zero<T>();
  const int rr = r % K;
  if (rr == 0) {  // vertex row: offsets -K..K around local K + r
#pragma unroll
    for (int o = 0; o <= 2 * K; ++o) {
      const T v = src[(r + o) * stride];
      mad2(a, b, P.yvm[o], P.yvk[o], v, v);
    }
  } else {  // inner row rr of its cell: the K+1 nodes of the cell
    const T* c = src + (K + r - rr) * stride;
#pragma unroll
    for (int q = 0; q <= K; ++q) {
      const T v = c[q * stride];
      mad2(a, b, P.me[rr][q], P.ke[rr][q], v, v);
    }
  }
  m = a;
  k = b;
}

}  // namespace dev

// B x B x B cells per CTA
template <typename T, int K, int B, int EPI>
__global__ void __launch_bounds__(128 * B) op3d_cell_kernel(const typename Storage<T>::type* __restrict__ u,
                                                            const OpParams<T> P,
                                                            const EpiParams<typename Storage<T>::type> E) {
  dev::pdl_enter();
  using S = typename Storage<T>::type;
  constexpr int NO = B * K;          // owned nodes per axis
  constexpr int NB = NO + K + 1;     // block nodes per axis
  constexpr int NX = NB * NB * NO, NY = NB * NO * NO, NZ = NO * NO * NO;
  __shared__ T ub[NB * NB * NB];
  __shared__ T mx[NX], kx[NX];
  __shared__ T g1[NY], g2[NY], g3[NY];
  const int N = P.N, n1 = P.n1, NC = (N + B - 1) / B;
  const int blk = blockIdx.x, s = blockIdx.z;
  const int cx = B * (blk % NC), cy = B * ((blk / NC) % NC), cz = B * (blk / (NC * NC));
  const int bx = K * cx - K, by = K * cy - K, bz = K * cz - K;  // block origin (may be negative)
  const S* __restrict__ us = u + (long long)s * P.ld;
  for (int i = threadIdx.x; i < NB * NB * NB; i += blockDim.x) {
    const int lx = i % NB, ly = (i / NB) % NB, lz = i / (NB * NB);
    const int gx = bx + lx, gy = by + ly, gz = bz + lz;
    T v = dev::zero<T>();
    if (gx >= 0 && gx < n1 && gy >= 0 && gy < n1 && gz >= 0 && gz < n1)
      v = dev::load<T>(us + gx + (long long)n1 * (gy + (long long)n1 * gz));
    ub[i] = v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NX; i += blockDim.x) {  // x: [lz][ly][rx]
    const int rx = i % NO, yz = i / NO;
    T m, k;
    dev::cell_row<T, K>(ub + yz * NB, 1, rx, P, m, k);
    mx[i] = m;
    kx[i] = k;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NY; i += blockDim.x) {  // y: [lz][ry][rx]
    const int rx = i % NO, ry = (i / NO) % NO, lz = i / (NO * NO);
    const int base = (lz * NB) * NO + rx;  // (lz, ly = 0, rx) in mx / kx
    T a, b, c, d;
    dev::cell_row<T, K>(mx + base, NO, ry, P, a, b);  // My Mx u, Ky Mx u
    dev::cell_row<T, K>(kx + base, NO, ry, P, c, d);  // My Kx u
    g1[i] = a;
    g2[i] = b;
    g3[i] = c;
  }
  __syncthreads();
  const T cm = P.cm[s], ck = P.ck[s];
  for (int i = threadIdx.x; i < NZ; i += blockDim.x) {  // z, then the epilogue of owned node i
    const int rx = i % NO, ry = (i / NO) % NO, rz = i / (NO * NO);
    const int gx = K * cx + rx, gy = K * cy + ry, gz = K * cz + rz;
    if (gx < 1 || gy < 1 || gz < 1 || gx > n1 - 2 || gy > n1 - 2 || gz > n1 - 2) continue;  // boundary
    // Mz (cm G1 + ck (G2 + G3)) + ck Kz G1 along z through (rx, ry)
    T az = dev::zero<T>(), kz = dev::zero<T>();
    const int col = ry * NO + rx, rr = rz % K;
    if (rr == 0) {
#pragma unroll
      for (int o = 0; o <= 2 * K; ++o) {
        const int j = (rz + o) * NO * NO + col;
        const T f = dev::mad(dev::mul(cm, g1[j]), ck, dev::add(g2[j], g3[j]));
        dev::mad2(az, kz, P.yvm[o], P.yvk[o], f, g1[j]);
      }
    } else {
#pragma unroll
      for (int q = 0; q <= K; ++q) {
        const int j = (K + rz - rr + q) * NO * NO + col;
        const T f = dev::mad(dev::mul(cm, g1[j]), ck, dev::add(g2[j], g3[j]));
        dev::mad2(az, kz, P.me[rr][q], P.ke[rr][q], f, g1[j]);
      }
    }
    const T va = dev::mad(az, ck, kz);
    S invD{};
    if constexpr (EPI == EPI_CHEB) invD = dev::inv_diag<S, 3>(E, (S)cm, (S)ck, rx % K, ry % K, rr);
    const long long o = (long long)s * P.ld + gx + (long long)n1 * (gy + (long long)n1 * gz);
    dev::epilogue<T, EPI>(E, o, s, va, dev::zero<T>(), invD);
  }
}

template <typename T, int B, int EPI>
cudaError_t launch_cell_op_b(int k, int nstage, const typename Storage<T>::type* u, const OpParams<T>& P,
                             const EpiParams<typename Storage<T>::type>& E, cudaStream_t st) {
  const int nc = (P.N + B - 1) / B;
  const dim3 grid((unsigned)(nc * nc * nc), 1, nstage);
  switch (k) {
    case 1: return launch_pdl(op3d_cell_kernel<T, 1, B, EPI>, grid, 128 * B, 0, st, u, P, E);
    case 2: return launch_pdl(op3d_cell_kernel<T, 2, B, EPI>, grid, 128 * B, 0, st, u, P, E);
    case 3: return launch_pdl(op3d_cell_kernel<T, 3, B, EPI>, grid, 128 * B, 0, st, u, P, E);
    case 4: return launch_pdl(op3d_cell_kernel<T, 4, B, EPI>, grid, 128 * B, 0, st, u, P, E);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int EPI>
cudaError_t launch_cell_op(int k, int nstage, const typename Storage<T>::type* u, const OpParams<T>& P,
                           const EpiParams<typename Storage<T>::type>& E, cudaStream_t st) {
  if (EPI == EPI_DUAL || nstage < 1 || nstage > kMaxStages || P.N < 1 || P.N > kCellKernelMaxN)
    return cudaErrorInvalidValue;
  // one cell per CTA: blocks of 2^3 cells on 16-cell levels measured slower than the streaming
  // kernel there (19.3 against 17.6 ms per step at degree 4 on 32^3 cells)
  return launch_cell_op_b<T, 1, EPI>(k, nstage, u, P, E, st);
}

}  // namespace irk
