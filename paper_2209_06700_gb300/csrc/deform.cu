// Stage operator on the curved mesh (sm_103a): v_s = cm[s] M u_s + ck[s] K u_s, or M u_s and
// K u_s separately, with the mapping data of every Gauss point read from memory.
//
// arXiv 2209.06700, Sec. 3.4 (batching of operations): on deformed cells the matrix-free cell loop
// loads the Jacobian data at each quadrature point; one cell loop over all Q stages loads it once
// instead of once per stage.  deform_cell_kernel does exactly that: one CTA per cell loads the
// cell's mapping data (w det J and the metric w det J J^-1 J^-T per Gauss point) into registers
// once and then, for each of the ns stage vectors, interpolates the nodal values and their
// reference gradients to the (k+1)^d Gauss points by sum factorisation (one 1D (k+1) x (k+1)
// matrix per axis pass), applies the mass weight and the metric, and integrates back with the
// transposed passes.  The cell results go to a cell-wise buffer; deform_gather_kernel sums, for
// every node, the contributions of its (up to 2^d) cells in a fixed order (deterministic, no
// atomics) and applies the output combination.  Launched with ns = 1 per stage, the same kernels
// give the per-stage loop that reloads the mapping data Q times.
#include <type_traits>

#include "deform_kernels.h"
#include "ffmath.cuh"
#include "pdl.cuh"

namespace irk {
namespace {

constexpr int kCellThreads = 128;

// 1D tables in the arithmetic type A: basis i (B) and its derivative (D) at Gauss point q
template <typename A> struct Tab;
template <> struct Tab<double> {
  __device__ __forceinline__ static double b(const DeformParams& P, int q, int i) { return P.B[q][i]; }
  __device__ __forceinline__ static double d(const DeformParams& P, int q, int i) { return P.D[q][i]; }
  __device__ __forceinline__ static double c(double v, float, float) { return v; }
};
template <> struct Tab<float> {
  __device__ __forceinline__ static float b(const DeformParams& P, int q, int i) { return P.Bh[q][i]; }
  __device__ __forceinline__ static float d(const DeformParams& P, int q, int i) { return P.Dh[q][i]; }
  __device__ __forceinline__ static float c(double, float h, float) { return h; }
};
template <> struct Tab<ff> {
  __device__ __forceinline__ static ff b(const DeformParams& P, int q, int i) { return ff{P.Bh[q][i], P.Bl[q][i]}; }
  __device__ __forceinline__ static ff d(const DeformParams& P, int q, int i) { return ff{P.Dh[q][i], P.Dl[q][i]}; }
  __device__ __forceinline__ static ff c(double, float h, float l) { return ff{h, l}; }
};

// T: element type of the vectors and of the mapping data in memory; A: arithmetic (double, ff,
// or float), also the element type of the cell-wise buffers.
template <typename T, typename A, int K, int DIM>
__global__ void __launch_bounds__(kCellThreads) deform_cell_kernel(const T* __restrict__ u, long long ld, int ns,
                                                                   const T* __restrict__ geo, A* __restrict__ eM,
                                                                   A* __restrict__ eK, const DeformParams P) {
  dev::pdl_enter();
  using dev::mad;
  constexpr int p = K + 1;
  constexpr int NP = (DIM == 3) ? p * p * p : p * p;
  constexpr int NF = 1 + DIM * (DIM + 1) / 2;
  __shared__ A s[9][NP];
  const long long cell = blockIdx.x;
  const int N = P.N, n1 = P.n1;
  const int cx = (int)(cell % N), cy = (int)((cell / N) % N), cz = (DIM == 3) ? (int)(cell / ((long long)N * N)) : 0;
  const int t = threadIdx.x;
  const bool act = t < NP;
  const int tx = t % p, ty = (t / p) % p, tz = (DIM == 3) ? t / (p * p) : 0;
  // this thread's node of the cell and its mapping data (read once for all stages)
  long long node = 0;
  A g[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) g[f] = dev::zero<A>();
  if (act) {
    node = (long long)(K * cx + tx) + (long long)n1 * ((K * cy + ty) + (long long)n1 * (K * cz + tz));
#pragma unroll
    for (int f = 0; f < NF; ++f) g[f] = dev::convert<A>(geo[(cell * NF + f) * NP + t]);
  }
  auto B = [&](int q, int i) { return Tab<A>::b(P, q, i); };
  auto D = [&](int q, int i) { return Tab<A>::d(P, q, i); };
  const A z = dev::zero<A>();
  for (int st = 0; st < ns; ++st) {
    if (act) s[0][t] = dev::convert<A>(u[st * ld + node]);
    __syncthreads();
    if constexpr (DIM == 3) {
      if (act) {  // x: (qx, j, l)
        A a = z, b = z;
#pragma unroll
        for (int i = 0; i < p; ++i) {
          const A v = s[0][i + p * ty + p * p * tz];
          a = mad(a, B(tx, i), v);
          b = mad(b, D(tx, i), v);
        }
        s[1][t] = a;
        s[2][t] = b;
      }
      __syncthreads();
      if (act) {  // y: (qx, qy, l)
        A a = z, b = z, c = z;
#pragma unroll
        for (int j = 0; j < p; ++j) {
          const A v1 = s[1][tx + p * j + p * p * tz], v2 = s[2][tx + p * j + p * p * tz];
          a = mad(a, B(ty, j), v1);
          b = mad(b, D(ty, j), v1);
          c = mad(c, B(ty, j), v2);
        }
        s[3][t] = a;  // B B u
        s[4][t] = b;  // B D_y u
        s[5][t] = c;  // B_y D_x u
      }
      __syncthreads();
      if (act) {  // z: values and reference gradients at Gauss point t, then mass weight and metric
        A U = z, Ux = z, Uy = z, Uz = z;
#pragma unroll
        for (int l = 0; l < p; ++l) {
          const int o = tx + p * ty + p * p * l;
          U = mad(U, B(tz, l), s[3][o]);
          Uz = mad(Uz, D(tz, l), s[3][o]);
          Uy = mad(Uy, B(tz, l), s[4][o]);
          Ux = mad(Ux, B(tz, l), s[5][o]);
        }
        // g: w det J, then (xx, yy, zz, xy, xz, yz) of w det J J^-1 J^-T
        s[6][t] = dev::mul(g[0], U);
        s[7][t] = mad(mad(dev::mul(g[1], Ux), g[4], Uy), g[5], Uz);
        s[8][t] = mad(mad(dev::mul(g[4], Ux), g[2], Uy), g[6], Uz);
        s[0][t] = mad(mad(dev::mul(g[5], Ux), g[6], Uy), g[3], Uz);
      }
      __syncthreads();
      if (act) {  // z^T: (qx, qy, l)
        A a = z, b = z, c = z, e = z;
#pragma unroll
        for (int q = 0; q < p; ++q) {
          const int o = tx + p * ty + p * p * q;
          a = mad(a, B(q, tz), s[6][o]);
          b = mad(b, B(q, tz), s[7][o]);
          c = mad(c, B(q, tz), s[8][o]);
          e = mad(e, D(q, tz), s[0][o]);
        }
        s[1][t] = a;
        s[2][t] = b;
        s[3][t] = c;
        s[4][t] = e;
      }
      __syncthreads();
      if (act) {  // y^T: (qx, j, l)
        A a = z, b = z, c = z;
#pragma unroll
        for (int q = 0; q < p; ++q) {
          const int o = tx + p * q + p * p * tz;
          a = mad(a, B(q, ty), s[1][o]);
          b = mad(b, B(q, ty), s[2][o]);
          c = mad(mad(c, D(q, ty), s[3][o]), B(q, ty), s[4][o]);
        }
        s[5][t] = a;
        s[6][t] = b;
        s[7][t] = c;
      }
      __syncthreads();
      if (act) {  // x^T: node (i, j, l)
        A m = z, k = z;
#pragma unroll
        for (int q = 0; q < p; ++q) {
          const int o = q + p * ty + p * p * tz;
          m = mad(m, B(q, tx), s[5][o]);
          k = mad(mad(k, D(q, tx), s[6][o]), B(q, tx), s[7][o]);
        }
        const long long e = (cell * ns + st) * NP + t;
        eM[e] = m;
        eK[e] = k;
      }
    } else {
      if (act) {  // x: (qx, j)
        A a = z, b = z;
#pragma unroll
        for (int i = 0; i < p; ++i) {
          const A v = s[0][i + p * ty];
          a = mad(a, B(tx, i), v);
          b = mad(b, D(tx, i), v);
        }
        s[1][t] = a;
        s[2][t] = b;
      }
      __syncthreads();
      if (act) {  // y: Gauss point (qx, qy); g: w det J, then (xx, yy, xy)
        A U = z, Ux = z, Uy = z;
#pragma unroll
        for (int j = 0; j < p; ++j) {
          const int o = tx + p * j;
          U = mad(U, B(ty, j), s[1][o]);
          Uy = mad(Uy, D(ty, j), s[1][o]);
          Ux = mad(Ux, B(ty, j), s[2][o]);
        }
        s[3][t] = dev::mul(g[0], U);
        s[4][t] = mad(dev::mul(g[1], Ux), g[3], Uy);
        s[5][t] = mad(dev::mul(g[3], Ux), g[2], Uy);
      }
      __syncthreads();
      if (act) {  // y^T: (qx, j)
        A a = z, b = z, c = z;
#pragma unroll
        for (int q = 0; q < p; ++q) {
          const int o = tx + p * q;
          a = mad(a, B(q, ty), s[3][o]);
          b = mad(b, B(q, ty), s[4][o]);
          c = mad(c, D(q, ty), s[5][o]);
        }
        s[6][t] = a;
        s[7][t] = b;
        s[8][t] = c;
      }
      __syncthreads();
      if (act) {  // x^T: node (i, j)
        A m = z, k = z;
#pragma unroll
        for (int q = 0; q < p; ++q) {
          const int o = q + p * ty;
          m = mad(m, B(q, tx), s[6][o]);
          k = mad(mad(k, D(q, tx), s[7][o]), B(q, tx), s[8][o]);
        }
        const long long e = (cell * ns + st) * NP + t;
        eM[e] = m;
        eK[e] = k;
      }
    }
    __syncthreads();  // s[0] is reloaded by the next stage
  }
}

// Node-wise sum of the cell contributions (fixed order: z, y, x candidates), then out.
template <typename T, typename A, int K, int DIM, int EPI>
__global__ void deform_gather_kernel(const A* __restrict__ eM, const A* __restrict__ eK, int ns, long long ld,
                                     T* __restrict__ out, T* __restrict__ out2, const DeformParams P) {
  dev::pdl_enter();
  constexpr int p = K + 1;
  constexpr int NP = (DIM == 3) ? p * p * p : p * p;
  const int st = blockIdx.y;
  const int N = P.N, n1 = P.n1;
  const long long n = (DIM == 3) ? (long long)n1 * n1 * n1 : (long long)n1 * n1;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(e % n1), iy = (int)((e / n1) % n1), iz = (DIM == 3) ? (int)(e / ((long long)n1 * n1)) : 1;
    const bool inner = ix > 0 && ix < n1 - 1 && iy > 0 && iy < n1 - 1 && (DIM == 2 || (iz > 0 && iz < n1 - 1));
    A sm = dev::zero<A>(), sk = dev::zero<A>();
    if (inner) {
      int c[3][2], r[3][2], nc[3];
      const int idx[3] = {ix, iy, iz};
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const int ch = idx[a] / K, rr = idx[a] - ch * K;
        if (rr == 0) {  // vertex: the cell below (local K) and the cell above (local 0)
          c[a][0] = ch - 1; r[a][0] = K;
          c[a][1] = ch;     r[a][1] = 0;
          nc[a] = 2;
        } else {
          c[a][0] = ch; r[a][0] = rr;
          nc[a] = 1;
        }
      }
      const int nz = (DIM == 3) ? nc[2] : 1;
      for (int bz = 0; bz < nz; ++bz)
        for (int by = 0; by < nc[1]; ++by)
          for (int bx = 0; bx < nc[0]; ++bx) {
            long long cell = c[0][bx] + (long long)N * c[1][by];
            int loc = r[0][bx] + p * r[1][by];
            if (DIM == 3) {
              cell += (long long)N * N * c[2][bz];
              loc += p * p * r[2][bz];
            }
            const long long o = (cell * ns + st) * NP + loc;
            sm = dev::add(sm, eM[o]);
            sk = dev::add(sk, eK[o]);
          }
    }
    if (EPI == EPI_DUAL) {
      out[st * ld + e] = dev::convert<T>(sm);
      out2[st * ld + e] = dev::convert<T>(sk);
    } else {
      const A cm = Tab<A>::c(P.cm[st], P.cmh[st], P.cml[st]), ck = Tab<A>::c(P.ck[st], P.ckh[st], P.ckl[st]);
      out[st * ld + e] = dev::convert<T>(dev::mad(dev::mul(cm, sm), ck, sk));
    }
  }
}

template <typename T, typename A, int K, int DIM>
cudaError_t launch_kd(const DeformDevice<T>& G, int ns, const T* u, long long ld, int epi, const DeformParams& P,
                      T* out, T* out2, cudaStream_t st) {
  A* eM = reinterpret_cast<A*>(G.eM);
  A* eK = reinterpret_cast<A*>(G.eK);
  launch_pdl(deform_cell_kernel<T, A, K, DIM>, (unsigned)G.ncell, kCellThreads, 0, st, u, ld, ns, G.geo, eM, eK, P);
  const long long n = (DIM == 3) ? (long long)P.n1 * P.n1 * P.n1 : (long long)P.n1 * P.n1;
  long long nb = (n + 255) / 256;
  if (nb > 152 * 16) nb = 152 * 16;
  dim3 grid((unsigned)nb, ns);
  if (epi == EPI_DUAL)
    launch_pdl(deform_gather_kernel<T, A, K, DIM, EPI_DUAL>, grid, 256, 0, st, eM, eK, ns, ld, out, out2, P);
  else
    launch_pdl(deform_gather_kernel<T, A, K, DIM, EPI_STORE>, grid, 256, 0, st, eM, eK, ns, ld, out, out2, P);
  return cudaGetLastError();
}

template <typename T, typename A>
cudaError_t launch_a(const DeformDevice<T>& G, int ns, const T* u, long long ld, int epi, const DeformParams& P,
                     T* out, T* out2, cudaStream_t st) {
#define IRK_DK(KK)                                                                                  \
  case KK:                                                                                          \
    return (G.dim == 3) ? launch_kd<T, A, KK, 3>(G, ns, u, ld, epi, P, out, out2, st)               \
                        : launch_kd<T, A, KK, 2>(G, ns, u, ld, epi, P, out, out2, st);
  switch (G.k) {
    IRK_DK(1) IRK_DK(2) IRK_DK(3) IRK_DK(4)
    default: return cudaErrorInvalidValue;
  }
#undef IRK_DK
}

void split(double v, float& h, float& l) {
  h = (float)v;
  l = (float)(v - (double)h);
}

}  // namespace

template <typename T>
cudaError_t launch_deformed(const DeformDevice<T>& G, int ns, const T* u, long long ld, int epi, const double* cm,
                            const double* ck, T* out, T* out2, cudaStream_t st) {
  if (ns < 1 || ns > G.max_ns || ns > kMaxStages || (epi != EPI_DUAL && epi != EPI_STORE) || !G.geo || !G.eM)
    return cudaErrorInvalidValue;
  if (epi == EPI_DUAL && !out2) return cudaErrorInvalidValue;
  DeformParams P;
  P.N = G.N;
  P.n1 = G.k * G.N + 1;
  const int p = G.k + 1;
  for (int q = 0; q < p; ++q)
    for (int i = 0; i < p; ++i) {
      P.B[q][i] = G.B[q * p + i];
      P.D[q][i] = G.D[q * p + i];
      split(P.B[q][i], P.Bh[q][i], P.Bl[q][i]);
      split(P.D[q][i], P.Dh[q][i], P.Dl[q][i]);
    }
  for (int s = 0; s < kMaxStages; ++s) {
    P.cm[s] = (epi == EPI_STORE && s < ns) ? cm[s] : 0.0;
    P.ck[s] = (epi == EPI_STORE && s < ns) ? ck[s] : 0.0;
    split(P.cm[s], P.cmh[s], P.cml[s]);
    split(P.ck[s], P.ckh[s], P.ckl[s]);
  }
  if constexpr (std::is_same<T, float>::value) {
    return launch_a<float, float>(G, ns, u, ld, epi, P, out, out2, st);
  } else {
    return G.ff ? launch_a<double, ff>(G, ns, u, ld, epi, P, out, out2, st)
                : launch_a<double, double>(G, ns, u, ld, epi, P, out, out2, st);
  }
}

template cudaError_t launch_deformed<double>(const DeformDevice<double>&, int, const double*, long long, int,
                                             const double*, const double*, double*, double*, cudaStream_t);
template cudaError_t launch_deformed<float>(const DeformDevice<float>&, int, const float*, long long, int,
                                            const double*, const double*, float*, float*, cudaStream_t);

}  // namespace irk
