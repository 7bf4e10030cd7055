// Stage-vector kernels of the outer solver of libirk (sm_103a).
//
// * Stage combination v_i = sum_j D_ij u_j: the "generalized matrix-vector
//   product" (D (x) I) u of arXiv 2209.06700, Sec. 2, used for A^{-1}, S~^{-1},
//   S~ (Eq. irk:A, irk:P) and T, T^{-1} (Eq. irk:Ainv, real form).  On one GPU
//   all stages of a node sit in the same memory, so the combination is an
//   elementwise kernel reading the Q stage values of each node.
// * Stage right-hand side and solution update (Sec. 1 and Sec. 2).
// * The vector work of FGMRES (Sec. 2, Sec. 5): fused classical Gram-Schmidt
//   passes with deterministic reductions (fixed block counts, fixed order),
//   norms, scalings, the final x += Z y.
//
// Every kernel is templated on the storage type S of the solver's vectors:
// double (the plain FP64 path) or ff (float-float pairs, computed on the FP32
// pipe).  Coefficients reach the ff kernels already split into hi + lo, on
// the host (CombineParams, scalars) or by the reduction that produced them
// (ReduceExtra), so that no FP64 instruction runs per element.
#include <algorithm>
#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include "ffmath.cuh"
#include "kernels.h"
#include "pdl.cuh"

namespace irk {

namespace {

constexpr int kThreads = 256;

// Accumulation for the Krylov reductions and updates.  mad_acc is a + c v without the final
// renormalisation of the ff result: the product c.hi v.hi is split exactly by an FMA, the cross
// terms are plain FP32, hi is the rounded sum of the leading parts and lo gathers the error terms
// (the compensated dot product of Ogita, Rump and Oishi, 2005, on ff operands).  Cancellation can
// leave |lo| >= |hi|, so such a value is only added to; fin() normalises it (two-sum, exact for
// any magnitudes) before it multiplies anything, is stored or enters a block reduction.
__device__ __forceinline__ double mad_acc(double a, double c, double v) { return fma(c, v, a); }
__device__ __forceinline__ ff mad_acc(ff a, ff c, ff v) {
  const float p = __fmul_rn(c.hi, v.hi);
  float pe = __fmaf_rn(c.hi, v.hi, -p);
  pe = __fmaf_rn(c.hi, v.lo, pe);
  pe = __fmaf_rn(c.lo, v.hi, pe);
  const float s = __fadd_rn(a.hi, p);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  return ff{s, __fadd_rn(e, __fadd_rn(a.lo, pe))};
}
__device__ __forceinline__ double fin(double a) { return a; }
__device__ __forceinline__ ff fin(ff a) {
  const float hi = __fadd_rn(a.hi, a.lo);
  const float bb = __fsub_rn(hi, a.hi);
  return ff{hi, __fadd_rn(__fsub_rn(a.hi, __fsub_rn(hi, bb)), __fsub_rn(a.lo, bb))};
}

inline int blocks_for(long long n, int per_thread = 1) {
  long long b = (n + (long long)kThreads * per_thread - 1) / ((long long)kThreads * per_thread);
  if (b < 1) b = 1;
  if (b > 152 * 32) b = 152 * 32;
  return (int)b;
}

// Blocks of one full wave of a grid-stride reduction kernel (its resident CTAs per SM x the SMs),
// at most cap: a grid of 4.1 waves leaves most SMs idle during the last one, a single wave none.
int wave_blocks(const void* kern, int cap) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> waves;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cap;
  std::lock_guard<std::mutex> lock(mu);
  auto it = waves.find({dev, kern});
  if (it == waves.end()) {
    int sms = 0, occ = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, 0) != cudaSuccess)
      return cap;
    it = waves.emplace(std::make_pair(dev, kern), std::max(1, sms * std::max(1, occ))).first;
  }
  return std::min(it->second, cap);
}

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

// arithmetic type of a combination: ff as soon as one operand is ff, else FP64
template <typename A, typename B, typename O>
struct ArithOf {
  static constexpr bool is_ff = std::is_same<A, ff>::value || std::is_same<B, ff>::value || std::is_same<O, ff>::value;
  using type = typename std::conditional<is_ff, ff, double>::type;
};

template <typename C> __device__ __forceinline__ C coef_a(const CombineParams& P, int i);
template <> __device__ __forceinline__ double coef_a<double>(const CombineParams& P, int i) { return P.Da[i]; }
template <> __device__ __forceinline__ ff coef_a<ff>(const CombineParams& P, int i) { return ff{P.Dah[i], P.Dal[i]}; }
template <typename C> __device__ __forceinline__ C coef_b(const CombineParams& P, int i);
template <> __device__ __forceinline__ double coef_b<double>(const CombineParams& P, int i) { return P.Db[i]; }
template <> __device__ __forceinline__ ff coef_b<ff>(const CombineParams& P, int i) { return ff{P.Dbh[i], P.Dbl[i]}; }


// block-wide sum of NR values per thread into partial rows (row r at partial[r * nb + blockIdx.x])
template <typename C, int NR>
__device__ __forceinline__ void block_partials(C (&acc)[NR], double* __restrict__ partial, int nb, int rows) {
  __shared__ C sred[NR][kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int g = 0; g < NR; ++g) {
    C x = fin(acc[g]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x = dev::add(x, dev::shfl_down(x, off));
    if (lane == 0) sred[g][warp] = x;
  }
  __syncthreads();
  if ((int)threadIdx.x < rows) {
    C x = sred[threadIdx.x][0];
    for (int q = 1; q < kThreads / 32; ++q) x = dev::add(x, sred[threadIdx.x][q]);
    partial[(long long)threadIdx.x * nb + blockIdx.x] = dev::to_double(x);
  }
}

// Final value of row i of a reduction, with the optional extras (thread-level).
__device__ __forceinline__ void finish_row(int i, double v, double* __restrict__ out, int take_sqrt,
                                           const ReduceExtra& X) {
  if (take_sqrt) v = sqrt(v);
  out[i] = v;
  if (X.out_ff) X.out_ff[i] = dev::from_double<ff>(v);
  if (i == 0 && (X.inv || X.inv_ff)) {
    const double r = (v > 0.0) ? 1.0 / v : 0.0;
    if (X.inv) X.inv[0] = r;
    if (X.inv_ff) X.inv_ff[0] = dev::from_double<ff>(r);
  }
  if (X.clear_flag && i == X.clear_row && __double_as_longlong(X.clear_flag[0]) == 0) {
    const double nrm = sqrt(v);
    const double r = (nrm > 0.0) ? 1.0 / nrm : 0.0;
    X.clear_norm[0] = nrm;
    if (X.clear_inv) X.clear_inv[0] = r;
    if (X.clear_inv_ff) X.clear_inv_ff[0] = dev::from_double<ff>(r);
  }
}

// Second Gram-Schmidt pass or not (thread 0 of the finishing block, rows final in out).  One
// classical pass leaves w' = w - V h with |V^T w'| / |w'| about (delta + rho) |w| / |w'|: the
// basis's own loss delta and the pass's rounding rho, both magnified by the cancellation |w| / |w'|
// (the loss of orthogonality of classical Gram-Schmidt grows this way step after step).  |w'|^2 is
// estimated before the second pass as |w|^2 - |h|^2 (exact for an orthonormal basis; with the basis
// orthogonal to sel_tol its error is far below the values that decide).  The pass is skipped while the
// estimated loss stays within sel_tol, and taken otherwise (or when the estimate is not positive),
// which brings the new vector's defect down to rounding level and leaves delta where it was.
__device__ void decide_second_pass(const double* out, const ReduceExtra& X) {
  const int nv = X.sel_nv;
  double hh = 0.0;
  for (int i = 0; i < nv; ++i) hh = fma(out[i], out[i], hh);
  const double ww = out[nv];
  const double d0 = (nv > 1) ? X.sel_delta[0] : 0.0;
  const double rest = ww - hh;
  bool redo = true;
  double d1 = fmax(d0, X.sel_round);
  if (rest > 0.0 && ww > 0.0) {  // false for NaN too: two passes, and the norm reports it
    const double dn = (d0 + X.sel_round) * sqrt(ww / rest);
    if (dn <= X.sel_tol) {
      redo = false;
      d1 = fmax(d0, dn);
    }
  }
  X.sel_flag[0] = redo ? 1.0 : 0.0;
  X.sel_delta[0] = d1;
}

// After the block's partials are written: the block that finishes last (of nblocks) sums every
// row over the nb blocks, one warp per row, each lane over blocks lane, lane + 32, ... then a
// shuffle tree (a fixed order, whichever block comes last), and resets the counter.
__device__ void finish_rows(const double* partial, int rows, int nb, unsigned nblocks, const RowSink& R) {
  __shared__ bool last;
  __threadfence();  // this block's partials are visible before its arrival is counted
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(R.count, 1u) == nblocks - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = warp; i < rows; i += blockDim.x >> 5) {
    double acc = 0.0;
    for (int b = lane; b < nb; b += 32) acc += __ldcg(partial + (long long)i * nb + b);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) finish_row(i, acc, R.out, R.take_sqrt, R.X);
  }
  if (R.X.sel_flag) {
    __syncthreads();  // every row's result is in R.out
    if (threadIdx.x == 0) decide_second_pass(R.out, R.X);
  }
  if (threadIdx.x == 0) *R.count = 0u;
}

// ------------------------------------------------------------ stage combination
// NMAX: compile-time bound on the number of input/output stage vectors (keeps the
// per-thread arrays in registers at a register count that allows full occupancy).
template <typename Ta, typename Tb, typename Tout, int NMAX>
__global__ void __launch_bounds__(kThreads) combine_kernel(const Ta* __restrict__ a, const Tb* __restrict__ b,
                                                           Tout* __restrict__ out, int n, long long ld,
                                                           const CombineParams C) {
  dev::pdl_enter();
  using A = typename ArithOf<Ta, Tb, Tout>::type;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    A av[NMAX], bv[NMAX];
#pragma unroll
    for (int j = 0; j < NMAX; ++j) {
      av[j] = (j < C.nina) ? dev::convert<A>(a[j * ld + e]) : dev::zero<A>();
      bv[j] = (j < C.ninb) ? dev::convert<A>(b[j * ld + e]) : dev::zero<A>();
    }
#pragma unroll
    for (int i = 0; i < NMAX; ++i) {
      if (i < C.nout) {
        A acc = dev::zero<A>();
        // zero coefficients (triangular S~, diagonal stiffness coupling) are skipped through
        // host-built integer masks
#pragma unroll
        for (int j = 0; j < NMAX; ++j) {
          if ((C.nza[i] >> j) & 1u) acc = dev::mad(acc, coef_a<A>(C, i * kMaxQ + j), av[j]);
          if ((C.nzb[i] >> j) & 1u) acc = dev::mad(acc, coef_b<A>(C, i * kMaxQ + j), bv[j]);
        }
        out[i * ld + e] = dev::convert<Tout>(acc);
      }
    }
  }
}

// Structured combinations with compile-time stage count Q (no dead instructions):
//  UNIT_LOWER: out_i = a_i + sum_{j<i} Da[i][j] a_j          (S~ and S~^{-1}, unit lower triangular)
//  FULL_DIAGB: out_i = sum_j Da[i][j] a_j + Db[i][i] b_i      (A^{-1} (x) M + tau I (x) K combination)
enum CombineStructure { CS_UNIT_LOWER = 1, CS_FULL_DIAGB = 2 };
template <typename Ta, typename Tb, typename Tout, int Q, int CS>
__global__ void __launch_bounds__(kThreads) combine_struct_kernel(const Ta* __restrict__ a, const Tb* __restrict__ b,
                                                                  Tout* __restrict__ out, int n, long long ld,
                                                                  const CombineParams C) {
  dev::pdl_enter();
  using A = typename ArithOf<Ta, Tb, Tout>::type;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    A av[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) av[j] = dev::convert<A>(dev::ldg<Ta>(a + j * ld + e));
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      A acc;
      if constexpr (CS == CS_UNIT_LOWER) {
        acc = av[i];
#pragma unroll
        for (int j = 0; j < i; ++j) acc = dev::mad(acc, coef_a<A>(C, i * kMaxQ + j), av[j]);
      } else {
        acc = dev::mul(coef_b<A>(C, i * kMaxQ + i), dev::convert<A>(dev::ldg<Tb>(b + i * ld + e)));
#pragma unroll
        for (int j = 0; j < Q; ++j) acc = dev::mad(acc, coef_a<A>(C, i * kMaxQ + j), av[j]);
      }
      out[i * ld + e] = dev::convert<Tout>(acc);
    }
  }
}

// ------------------------------------------------------------ RHS, update, conversions
// rhs_i = sum_j Ainv_ij (g_j - K y_n), g_j = phi_j G (built-in source) or the user stage loads
template <typename S>
__global__ void stage_rhs_kernel(GridInfo g, const RhsParams R, const S* __restrict__ Ky,
                                 const double* __restrict__ G1, const double* __restrict__ Gv,
                                 const double* __restrict__ loads, S* __restrict__ rhs) {
  dev::pdl_enter();
  using C = typename Coef<S>::type;
  const int n = (int)g.n;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    int ix, iy, iz;
    coords(e, g.dim, g.n1, ix, iy, iz);
    if (!interior(g.dim, g.n1, ix, iy, iz)) continue;
    const C mky = dev::neg(dev::ldg<S>(Ky + e));
    C f[kMaxQ];
    if (loads) {
#pragma unroll
      for (int j = 0; j < kMaxQ; ++j)
        if (j < R.Q) f[j] = dev::add(dev::from_double<C>(loads[j * g.ld + e]), mky);
    } else {
      // G = G1[x] G1[y] (G1[z]) in FP64 once per node (or the full load vector Gv of a curved
      // mesh), then phi_j G - K y_n per stage
      double G;
      if (Gv) {
        G = Gv[e];
      } else {
        G = G1[ix] * G1[iy];
        if (g.dim == 3) G *= G1[iz];
      }
      const C Gc = dev::from_double<C>(G);
#pragma unroll
      for (int j = 0; j < kMaxQ; ++j)
        if (j < R.Q) {
          if constexpr (std::is_same<C, ff>::value) f[j] = dev::mad(mky, ff{R.phih[j], R.phil[j]}, Gc);
          else f[j] = dev::mad(mky, R.phi[j], Gc);
        }
    }
#pragma unroll
    for (int i = 0; i < kMaxQ; ++i) {
      if (i >= R.Q) break;
      C acc = dev::zero<C>();
#pragma unroll
      for (int j = 0; j < kMaxQ; ++j)
        if (j < R.Q) {
          if constexpr (std::is_same<C, ff>::value)
            acc = dev::mad(acc, ff{R.Ainvh[i * kMaxQ + j], R.Ainvl[i * kMaxQ + j]}, f[j]);
          else
            acc = dev::mad(acc, R.Ainv[i * kMaxQ + j], f[j]);
        }
      rhs[i * g.ld + e] = acc;
    }
  }
}

struct UpdateParams {
  int Q;
  double tb[kMaxQ];          // tau b_i
  float tbh[kMaxQ], tbl[kMaxQ];
};

// y += tau sum_i b_i k_i: the stage sum in the vectors' arithmetic, the add to y in FP64
template <typename S>
__global__ void update_kernel(GridInfo g, const UpdateParams U, const S* __restrict__ kst, double* __restrict__ y) {
  dev::pdl_enter();
  using C = typename Coef<S>::type;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.n; e += (long long)gridDim.x * blockDim.x) {
    C acc = dev::zero<C>();
    for (int i = 0; i < U.Q; ++i) {
      if constexpr (std::is_same<C, ff>::value) acc = dev::mad(acc, ff{U.tbh[i], U.tbl[i]}, dev::ldg<S>(kst + i * g.ld + e));
      else acc = dev::mad(acc, U.tb[i], kst[i * g.ld + e]);
    }
    y[e] += dev::to_double(acc);
  }
}

__global__ void to_ff_kernel(const double* __restrict__ in, ff* __restrict__ out, long long n) {
  dev::pdl_enter();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    out[e] = dev::from_double<ff>(in[e]);
}
__global__ void from_ff_kernel(const ff* __restrict__ in, double* __restrict__ out, long long n) {
  dev::pdl_enter();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    out[e] = dev::to_double(dev::ldg<ff>(in + e));
}

// ------------------------------------------------------------ Gram-Schmidt
// Basis vectors in groups of 8 (blockIdx.y) beyond 16; the last group also reduces |w|^2 into row nv.
// MODE 1 without dots (*dots_flag == 0): group 0 alone computes w_out and its norm.
template <typename S, int MODE>  // 0: dots of w_in;  1: w_out = w_in - V h, then dots of w_out
__global__ void __launch_bounds__(kThreads) gs_kernel(const S* __restrict__ V, long long vstride, int nv,
                                                      const typename Coef<S>::type* __restrict__ h,
                                                      const double* __restrict__ dots_flag,
                                                      const S* __restrict__ w_in, S* __restrict__ w_out, int n,
                                                      double* __restrict__ partial, int nb, const RowSink R) {
  dev::pdl_enter();
  using C = typename Coef<S>::type;
  constexpr int G = 8;
  const int i0 = blockIdx.y * G;
  const bool dots = (MODE == 0) || dots_flag == nullptr || __double_as_longlong(dots_flag[0]) != 0;
  const bool last = dots ? (i0 + G >= nv) : (blockIdx.y == 0);  // the group that reduces |w|^2
  const bool active = dots || blockIdx.y == 0;
  __shared__ C hs[64];
  if (MODE == 1) {
    for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = dev::neg(h[i]);
    __syncthreads();
  }
  C acc[G + 1];
#pragma unroll
  for (int g = 0; g <= G; ++g) acc[g] = dev::zero<C>();
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; active && e < n; e += gridDim.x * blockDim.x) {
    C we = dev::ldg<S>(w_in + e);
    if (MODE == 1) {
      for (int i = 0; i < nv; ++i) we = mad_acc(we, hs[i], dev::ldg<S>(V + i * vstride + e));
      we = fin(we);
      if (blockIdx.y == 0) w_out[e] = we;
    }
    if (dots) {
#pragma unroll
      for (int g = 0; g < G; ++g)
        if (i0 + g < nv) acc[g] = mad_acc(acc[g], dev::ldg<S>(V + (i0 + g) * vstride + e), we);
    }
    acc[G] = mad_acc(acc[G], we, we);
  }
  const int cnt = min(G, nv - i0);
  // rows i0 .. i0 + cnt - 1, and row nv from the last group
  if (!last) acc[G] = dev::zero<C>();
  __shared__ C sred[G + 1][kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int g = 0; g <= G; ++g) {
    C x = fin(acc[g]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x = dev::add(x, dev::shfl_down(x, off));
    if (lane == 0) sred[g][warp] = x;
  }
  __syncthreads();
  if ((int)threadIdx.x <= G) {
    const int g = threadIdx.x;
    C x = sred[g][0];
    for (int q = 1; q < kThreads / 32; ++q) x = dev::add(x, sred[g][q]);
    if (g < cnt) partial[(long long)(i0 + g) * nb + blockIdx.x] = dev::to_double(x);
    if (g == G && last) partial[(long long)nv * nb + blockIdx.x] = dev::to_double(x);
  }
  finish_rows(partial, nv + 1, nb, gridDim.x * gridDim.y, R);
}

// Basis sizes up to 16: fully unrolled, one pass over the basis per kernel; in MODE 1 the
// basis values loaded for the update are reused for the dot products (skipped when *dots_flag ==
// 0), and w_out may be w_in (each element is read, then written, by the same thread).
template <typename S, int MODE, int NV>
__global__ void __launch_bounds__(kThreads) gs_small_kernel(const S* __restrict__ V, long long vstride,
                                                            const typename Coef<S>::type* __restrict__ h,
                                                            const double* __restrict__ dots_flag, const S* w_in,
                                                            S* w_out, int n, double* __restrict__ partial, int nb,
                                                            const RowSink R) {
  dev::pdl_enter();
  using C = typename Coef<S>::type;
  const bool dots = (MODE == 0) || dots_flag == nullptr || __double_as_longlong(dots_flag[0]) != 0;
  C hr[NV];
  if (MODE == 1) {
#pragma unroll
    for (int i = 0; i < NV; ++i) hr[i] = dev::neg(h[i]);
  }
  C acc[NV + 1];
#pragma unroll
  for (int i = 0; i <= NV; ++i) acc[i] = dev::zero<C>();
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    C vv[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) vv[i] = dev::ldg<S>(V + i * vstride + e);
    C we;
    if constexpr (MODE == 1) {
      we = w_in[e];  // a plain load: w_in may be w_out
#pragma unroll
      for (int i = 0; i < NV; ++i) we = mad_acc(we, hr[i], vv[i]);
      we = fin(we);
      w_out[e] = we;
    } else {
      we = dev::ldg<S>(w_in + e);
    }
    if (dots) {
#pragma unroll
      for (int i = 0; i < NV; ++i) acc[i] = mad_acc(acc[i], vv[i], we);
    }
    acc[NV] = mad_acc(acc[NV], we, we);
  }
  block_partials<C, NV + 1>(acc, partial, nb, NV + 1);
  finish_rows(partial, NV + 1, nb, gridDim.x, R);
}

// w_out = w_in - V h when the device flag asks for the second pass, else w_out = w_in; partial =
// |w_out|^2 per block.  In place (w_out == w_in) without the second pass there is nothing to do:
// the whole grid returns at once and the first pass's kernel has written the norm.
template <typename S, int NV>  // NV = 0: any basis size up to 64 (coefficients staged in shared memory)
__global__ void __launch_bounds__(kThreads) gs_reorth_kernel(const S* __restrict__ V, long long vstride, int nv,
                                                             const typename Coef<S>::type* __restrict__ h,
                                                             const double* __restrict__ redo_flag,
                                                             const S* w_in, S* w_out, int n,
                                                             double* __restrict__ partial, const RowSink R) {
  dev::pdl_enter();
  using C = typename Coef<S>::type;
  // the flag is 1.0 or 0.0: its bit pattern decides (no FP64 compare)
  const bool redo = __double_as_longlong(redo_flag[0]) != 0;
  if (!redo && w_in == w_out) return;
  C acc[1] = {dev::zero<C>()};
  if constexpr (NV > 0) {
    C hr[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) hr[i] = redo ? dev::neg(h[i]) : dev::zero<C>();
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
      C we = w_in[e];  // a plain load: w_in may be w_out
      if (redo) {
#pragma unroll
        for (int i = 0; i < NV; ++i) we = mad_acc(we, hr[i], dev::ldg<S>(V + i * vstride + e));
        we = fin(we);
      }
      w_out[e] = we;
      acc[0] = mad_acc(acc[0], we, we);
    }
  } else {
    __shared__ C hs[64];
    for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = redo ? dev::neg(h[i]) : dev::zero<C>();
    __syncthreads();
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
      C we = w_in[e];
      if (redo)
        for (int i = 0; i < nv; ++i) we = mad_acc(we, hs[i], dev::ldg<S>(V + i * vstride + e));
      we = fin(we);
      w_out[e] = we;
      acc[0] = mad_acc(acc[0], we, we);
    }
  }
  block_partials<C, 1>(acc, partial, gridDim.x, 1);
  finish_rows(partial, 1, gridDim.x, gridDim.x, R);
}

template <typename S>
__global__ void norm2_kernel(const S* __restrict__ w, long long n, double* __restrict__ partial, const RowSink R) {
  dev::pdl_enter();
  using C = typename Coef<S>::type;
  C acc[1] = {dev::zero<C>()};
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const C v = dev::ldg<S>(w + e);
    acc[0] = mad_acc(acc[0], v, v);
  }
  block_partials<C, 1>(acc, partial, gridDim.x, 1);
  finish_rows(partial, 1, gridDim.x, gridDim.x, R);
}

__global__ void reduce_partials_kernel(const double* __restrict__ partial, int nb, double* __restrict__ out,
                                       int take_sqrt, const ReduceExtra X) {
  dev::pdl_enter();
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
    finish_row(i, v, out, take_sqrt, X);
  }
}

// w += sign sum_i h_i V_i
template <typename S>
__global__ void multi_axpy_kernel(const S* __restrict__ V, long long vstride, int nv,
                                  const typename Coef<S>::type* __restrict__ h, int negate, S* w, long long n) {
  dev::pdl_enter();
  using C = typename Coef<S>::type;
  __shared__ C hs[64];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = negate ? dev::neg(h[i]) : h[i];
  __syncthreads();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    C acc = w[e];
    for (int i = 0; i < nv; ++i) acc = mad_acc(acc, hs[i], dev::ldg<S>(V + i * vstride + e));
    w[e] = fin(acc);
  }
}

// out = inv[0] w (inv on the device, written by the norm's reduction); out may alias w
template <typename S>
__global__ void scale_dev_kernel(const S* w, const typename Coef<S>::type* __restrict__ inv, S* out, long long n) {
  dev::pdl_enter();
  const typename Coef<S>::type f = inv[0];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    out[e] = dev::mul(f, w[e]);
}

template <typename S>
__global__ void scale_kernel(const S* x, typename Coef<S>::type a, S* out, long long n) {
  dev::pdl_enter();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    out[e] = dev::mul(a, x[e]);
}

template <typename S> typename Coef<S>::type host_coef(double a);
template <> double host_coef<double>(double a) { return a; }
template <> ff host_coef<ff>(double a) {
  const float hi = (float)a;
  return ff{hi, (float)(a - (double)hi)};
}

}  // namespace

void split_double(double d, float* hi, float* lo) {
  *hi = (float)d;
  *lo = (float)(d - (double)*hi);
}

// ------------------------------------------------------------ launchers
template <typename Ta, typename Tb, typename Tout>
cudaError_t launch_combine(const Ta* a, const Tb* b, Tout* out, long long n, long long ld, const CombineParams& C,
                           cudaStream_t st) {
  const int nmax = std::max(C.nout, std::max(C.nina, C.ninb));
  const int grid = blocks_for(n, 2);
  CombineParams Cz = C;
  for (int i = 0; i < kMaxQ * kMaxQ; ++i) {
    split_double(C.Da[i], &Cz.Dah[i], &Cz.Dal[i]);
    split_double(C.Db[i], &Cz.Dbh[i], &Cz.Dbl[i]);
  }
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
#define IRK_CS(QQ, CSV) \
  launch_pdl(combine_struct_kernel<Ta, Tb, Tout, QQ, CSV>, grid, kThreads, 0, st, a, b, out, (int)n, ld, Cz)
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
  if (nmax <= 2) launch_pdl(combine_kernel<Ta, Tb, Tout, 2>, grid, kThreads, 0, st, a, b, out, (int)n, ld, Cz);
  else if (nmax <= 4) launch_pdl(combine_kernel<Ta, Tb, Tout, 4>, grid, kThreads, 0, st, a, b, out, (int)n, ld, Cz);
  else launch_pdl(combine_kernel<Ta, Tb, Tout, kMaxQ>, grid, kThreads, 0, st, a, b, out, (int)n, ld, Cz);
  return cudaGetLastError();
}
#define IRK_COMBINE_INST(TA, TB, TO)                                                                        \
  template cudaError_t launch_combine<TA, TB, TO>(const TA*, const TB*, TO*, long long, long long,          \
                                                  const CombineParams&, cudaStream_t);
IRK_COMBINE_INST(double, double, double)
IRK_COMBINE_INST(double, double, float)
IRK_COMBINE_INST(float, double, double)
IRK_COMBINE_INST(ff, ff, ff)
IRK_COMBINE_INST(ff, ff, float)
IRK_COMBINE_INST(ff, ff, double)
IRK_COMBINE_INST(float, ff, ff)
IRK_COMBINE_INST(double, ff, ff)
#undef IRK_COMBINE_INST

template <typename S>
cudaError_t launch_stage_rhs(const GridInfo& g, const RhsParams& R, const S* Ky, const double* G1, const double* Gv,
                             const double* loads, S* rhs, cudaStream_t st) {
  RhsParams Rs = R;
  for (int i = 0; i < kMaxQ * kMaxQ; ++i) split_double(R.Ainv[i], &Rs.Ainvh[i], &Rs.Ainvl[i]);
  for (int j = 0; j < kMaxQ; ++j) split_double(R.phi[j], &Rs.phih[j], &Rs.phil[j]);
  launch_pdl(stage_rhs_kernel<S>, blocks_for(g.n, 2), kThreads, 0, st, g, Rs, Ky, G1, Gv, loads, rhs);
  return cudaGetLastError();
}
template cudaError_t launch_stage_rhs<double>(const GridInfo&, const RhsParams&, const double*, const double*,
                                              const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_stage_rhs<ff>(const GridInfo&, const RhsParams&, const ff*, const double*, const double*,
                                          const double*, ff*, cudaStream_t);

template <typename S>
cudaError_t launch_update(const GridInfo& g, int Q, const S* kst, const double* bw, double tau, double* y,
                          cudaStream_t st) {
  UpdateParams U;
  U.Q = Q;
  for (int i = 0; i < kMaxQ; ++i) {
    U.tb[i] = (i < Q) ? tau * bw[i] : 0.0;
    split_double(U.tb[i], &U.tbh[i], &U.tbl[i]);
  }
  launch_pdl(update_kernel<S>, blocks_for(g.n, 2), kThreads, 0, st, g, U, kst, y);
  return cudaGetLastError();
}
template cudaError_t launch_update<double>(const GridInfo&, int, const double*, const double*, double, double*,
                                           cudaStream_t);
template cudaError_t launch_update<ff>(const GridInfo&, int, const ff*, const double*, double, double*, cudaStream_t);

cudaError_t launch_to_ff(const double* in, ff* out, long long n, cudaStream_t st) {
  launch_pdl(to_ff_kernel, blocks_for(n, 2), kThreads, 0, st, in, out, n);
  return cudaGetLastError();
}
cudaError_t launch_from_ff(const ff* in, double* out, long long n, cudaStream_t st) {
  launch_pdl(from_ff_kernel, blocks_for(n, 2), kThreads, 0, st, in, out, n);
  return cudaGetLastError();
}

int reduction_blocks(long long n) { return blocks_for(n, 8); }

cudaError_t launch_reduce_partials(const double* partial, int nv, int nb, double* out, cudaStream_t st, int take_sqrt,
                                   const ReduceExtra* extra) {
  ReduceExtra X;
  if (extra) X = *extra;
  launch_pdl(reduce_partials_kernel, nv, kThreads, 0, st, partial, nb, out, take_sqrt, X);
  return cudaGetLastError();
}

#define IRK_GSC(MODE, NVV, ...)                                                         \
  case NVV:                                                                             \
    nb = wave_blocks((const void*)gs_small_kernel<S, MODE, NVV>, nb);                   \
    launch_pdl(gs_small_kernel<S, MODE, NVV>, nb, kThreads, 0, st, __VA_ARGS__);                \
    break;
#define IRK_GS_SMALL(MODE, ...)                                                                            \
  switch (nv) {                                                                                           \
    IRK_GSC(MODE, 1, __VA_ARGS__) IRK_GSC(MODE, 2, __VA_ARGS__) IRK_GSC(MODE, 3, __VA_ARGS__)            \
    IRK_GSC(MODE, 4, __VA_ARGS__) IRK_GSC(MODE, 5, __VA_ARGS__) IRK_GSC(MODE, 6, __VA_ARGS__)            \
    IRK_GSC(MODE, 7, __VA_ARGS__) IRK_GSC(MODE, 8, __VA_ARGS__) IRK_GSC(MODE, 9, __VA_ARGS__)            \
    IRK_GSC(MODE, 10, __VA_ARGS__) IRK_GSC(MODE, 11, __VA_ARGS__) IRK_GSC(MODE, 12, __VA_ARGS__)         \
    IRK_GSC(MODE, 13, __VA_ARGS__) IRK_GSC(MODE, 14, __VA_ARGS__) IRK_GSC(MODE, 15, __VA_ARGS__)         \
    default:                                                                                              \
      nb = wave_blocks((const void*)gs_small_kernel<S, MODE, 16>, nb);                                    \
      launch_pdl(gs_small_kernel<S, MODE, 16>, nb, kThreads, 0, st, __VA_ARGS__);                                 \
      break;                                                                                              \
  }

template <typename S>
cudaError_t launch_gs_dot(const S* V, long long vstride, int nv, const S* w, long long n, double* partial, int& nb,
                          const RowSink& R, cudaStream_t st) {
  if (nv < 1 || nv > 64 || !R.out || !R.count) return cudaErrorInvalidValue;
  using C = typename Coef<S>::type;
  if (nv <= 16) {
    IRK_GS_SMALL(0, V, vstride, (const C*)nullptr, (const double*)nullptr, w, (S*)nullptr, (int)n, partial, nb, R);
    return cudaGetLastError();
  }
  nb = wave_blocks((const void*)gs_kernel<S, 0>, nb);
  dim3 grid(nb, (nv + 7) / 8);
  launch_pdl(gs_kernel<S, 0>, grid, kThreads, 0, st, V, vstride, nv, nullptr, (const double*)nullptr, w, nullptr,
             (int)n, partial, nb, R);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_gs_axpy_dot(const S* V, long long vstride, int nv, const typename Coef<S>::type* h, const S* w_in,
                               S* w_out, long long n, double* partial, int& nb, const RowSink& R,
                               const double* dots_flag, cudaStream_t st) {
  if (nv < 1 || nv > 64 || !R.out || !R.count) return cudaErrorInvalidValue;
  if (nv <= 16) {
    IRK_GS_SMALL(1, V, vstride, h, dots_flag, w_in, w_out, (int)n, partial, nb, R);
    return cudaGetLastError();
  }
  // group 0 writes w_out; the other groups recompute it for their dots (so not in place)
  if (w_in == w_out) return cudaErrorInvalidValue;
  nb = wave_blocks((const void*)gs_kernel<S, 1>, nb);
  dim3 grid(nb, (nv + 7) / 8);
  launch_pdl(gs_kernel<S, 1>, grid, kThreads, 0, st, V, vstride, nv, h, dots_flag, w_in, w_out, (int)n, partial, nb,
             R);
  return cudaGetLastError();
}
#undef IRK_GS_SMALL
#undef IRK_GSC

template <typename S>
cudaError_t launch_gs_reorth(const S* V, long long vstride, int nv, const typename Coef<S>::type* h,
                             const double* redo_flag, const S* w_in, S* w_out, long long n, double* partial, int& nb,
                             const RowSink& R, cudaStream_t st) {
  if (nv < 1 || nv > 64 || !R.out || !R.count) return cudaErrorInvalidValue;
  switch (nv) {
#define IRK_GSR(NVV)                                                                                            \
  case NVV:                                                                                                     \
    nb = wave_blocks((const void*)gs_reorth_kernel<S, NVV>, nb);                                                 \
    launch_pdl(gs_reorth_kernel<S, NVV>, nb, kThreads, 0, st, V, vstride, nv, h, redo_flag, w_in, w_out, (int)n, partial, R); \
    return cudaGetLastError();
    IRK_GSR(1) IRK_GSR(2) IRK_GSR(3) IRK_GSR(4) IRK_GSR(5) IRK_GSR(6) IRK_GSR(7) IRK_GSR(8)
    IRK_GSR(9) IRK_GSR(10) IRK_GSR(11) IRK_GSR(12) IRK_GSR(13) IRK_GSR(14) IRK_GSR(15) IRK_GSR(16)
#undef IRK_GSR
    default: break;
  }
  nb = wave_blocks((const void*)gs_reorth_kernel<S, 0>, nb);
  launch_pdl(gs_reorth_kernel<S, 0>, nb, kThreads, 0, st, V, vstride, nv, h, redo_flag, w_in, w_out, (int)n, partial, R);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_norm2_partial(const S* w, long long n, double* partial, int& nb, const RowSink& R,
                                 cudaStream_t st) {
  if (!R.out || !R.count) return cudaErrorInvalidValue;
  nb = wave_blocks((const void*)norm2_kernel<S>, nb);
  launch_pdl(norm2_kernel<S>, nb, kThreads, 0, st, w, n, partial, R);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_multi_axpy(const S* V, long long vstride, int nv, const typename Coef<S>::type* h, double sign,
                              S* w, long long n, cudaStream_t st) {
  if (nv < 0 || nv > 64) return cudaErrorInvalidValue;
  if (nv == 0) return cudaSuccess;
  launch_pdl(multi_axpy_kernel<S>, blocks_for(n, 2), kThreads, 0, st, V, vstride, nv, h, sign < 0 ? 1 : 0, w, n);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_scale_dev(const S* w, const typename Coef<S>::type* inv, S* out, long long n, cudaStream_t st) {
  launch_pdl(scale_dev_kernel<S>, blocks_for(n, 2), kThreads, 0, st, w, inv, out, n);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_scale(const S* x, double a, S* out, long long n, cudaStream_t st) {
  launch_pdl(scale_kernel<S>, blocks_for(n, 2), kThreads, 0, st, x, host_coef<S>(a), out, n);
  return cudaGetLastError();
}

#define IRK_KRYLOV_INST(S)                                                                                        \
  template cudaError_t launch_gs_dot<S>(const S*, long long, int, const S*, long long, double*, int&,              \
                                        const RowSink&, cudaStream_t);                                             \
  template cudaError_t launch_gs_axpy_dot<S>(const S*, long long, int, const Coef<S>::type*, const S*, S*,          \
                                             long long, double*, int&, const RowSink&, const double*,             \
                                             cudaStream_t);                                                       \
  template cudaError_t launch_gs_reorth<S>(const S*, long long, int, const Coef<S>::type*, const double*,         \
                                           const S*, S*, long long, double*, int&, const RowSink&, cudaStream_t); \
  template cudaError_t launch_norm2_partial<S>(const S*, long long, double*, int&, const RowSink&, cudaStream_t);  \
  template cudaError_t launch_multi_axpy<S>(const S*, long long, int, const Coef<S>::type*, double, S*,           \
                                            long long, cudaStream_t);                                             \
  template cudaError_t launch_scale_dev<S>(const S*, const Coef<S>::type*, S*, long long, cudaStream_t);          \
  template cudaError_t launch_scale<S>(const S*, double, S*, long long, cudaStream_t);
IRK_KRYLOV_INST(double)
IRK_KRYLOV_INST(ff)
#undef IRK_KRYLOV_INST

}  // namespace irk
