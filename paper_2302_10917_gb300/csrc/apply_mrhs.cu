// Multi-RHS trace-operator apply (Sec. 3.3.2, steps 1-4, for nrhs vectors at
// once): Y_r = S X_r (or D^-1 S X_r) for r = 0 .. nrhs-1, every Schur block
// streamed from HBM once for all columns.
//
// One CTA per interior edge f. Its two element sides' trace values of all
// columns are gathered into shared memory (rows of the columns padded to a
// multiple of RPT, plus one against bank conflicts); thread (t, g) owns edge
// dof t and the RPT columns
// g RPT .. g RPT + RPT - 1, and accumulates
//     y_r(t) = sum_side sum_j S_side(t_side, j) x_side,r(j)
// over both sides in a fixed order (bitwise reproducible). Block types BT:
// 0 FP64, 1 split-FP32 pairs, 2 FP32; vector types VT: 0 FP64, 1 split-FP32
// pairs, 2 FP32. FP64 blocks with FP64 vectors use FP64 arithmetic, FP32
// blocks with FP32 vectors FP32 arithmetic, every other pairing split-FP32
// arithmetic.
#include "internal.h"
#include "df64.h"

namespace mehdg {

constexpr int RPT = 8;   // columns per thread

// shared-memory row length for nrhs columns
__host__ __device__ __forceinline__ int mrhs_row(int nrhs) { return (nrhs + RPT - 1) / RPT * RPT + 1; }

template <int BT, int VT>
struct MrhsTypes {
  static constexpr bool f64 = (BT == 0 && VT == 0);
  static constexpr bool f32 = (BT == 2 && VT == 2);
  using Acc = typename std::conditional<f64, double, typename std::conditional<f32, float, float2>::type>::type;
};

template <int VT>
__device__ __forceinline__ float2 load_split(const void* x, size_t i) {
  if constexpr (VT == 0) return df_from(static_cast<const double*>(x)[i]);
  else if constexpr (VT == 1) return static_cast<const float2*>(x)[i];
  else return make_float2(static_cast<const float*>(x)[i], 0.f);
}

template <int BT>
__device__ __forceinline__ float2 block_split(const void* S, size_t i) {
  if constexpr (BT == 0) return df_from(static_cast<const double*>(S)[i]);
  else if constexpr (BT == 1) return static_cast<const float2*>(S)[i];
  else return make_float2(static_cast<const float*>(S)[i], 0.f);
}

template <int BT, int VT>
__global__ void __launch_bounds__(544) apply_mrhs_kernel(Params P, const void* __restrict__ Sv,
                                                         const void* __restrict__ xv, void* __restrict__ yv,
                                                         int nrhs, int64_t vstride,
                                                         const double* __restrict__ escale) {
  using T = MrhsTypes<BT, VT>;
  using Acc = typename T::Acc;
  extern __shared__ unsigned char sraw[];
  // [2 n_t][NR1]: columns padded to a multiple of RPT (zeros), plus one against
  // bank conflicts, so that a thread's RPT reads stay inside its row
  Acc* xs = reinterpret_cast<Acc*>(sraw);
  const int nt = P.n_t, P1 = P.P1, PP = P.P, NR1 = mrhs_row(nrhs);
  const int f = blockIdx.x;
  const int tid = threadIdx.x;
  int e[2], k[2], fl[2];
  double len;
  edge_sides(f, P.n, e, k, fl, &len);
  // gather: consecutive threads take consecutive local dofs of one column
  for (int idx = tid; idx < 2 * nt * (NR1 - 1); idx += blockDim.x) {
    const int r = idx / (2 * nt), q = idx - r * 2 * nt;
    const int sd = q / nt, c = q - sd * nt;
    int code[3], flip[3];
    elem_edges(e[sd], P.n, code, flip);
    const int kk = c / P1, t = c - kk * P1;
    Acc v;
    if (r < nrhs && code[kk] >= 0) {
      const size_t gi = (size_t)r * vstride + (size_t)code[kk] * P1 + (flip[kk] ? PP - t : t);
      if constexpr (T::f64) v = static_cast<const double*>(xv)[gi];
      else if constexpr (T::f32) v = static_cast<const float*>(xv)[gi];
      else v = load_split<VT>(xv, gi);
    } else {
      if constexpr (T::f64 || T::f32) v = 0;
      else v = make_float2(0.f, 0.f);
    }
    xs[q * NR1 + r] = v;
  }
  __syncthreads();
  const int s = tid % P1, grp = tid / P1;
  const int r0 = grp * RPT;
  if (r0 >= nrhs) return;
  const int t0 = fl[0] ? PP - s : s, t1 = fl[1] ? PP - s : s;
  const size_t base0 = ((size_t)e[0] * 3 + k[0]) * (size_t)nt * P1 + t0;
  const size_t base1 = ((size_t)e[1] * 3 + k[1]) * (size_t)nt * P1 + t1;
  Acc acc[RPT];
#pragma unroll
  for (int u = 0; u < RPT; ++u) {
    if constexpr (T::f64 || T::f32) acc[u] = 0;
    else acc[u] = make_float2(0.f, 0.f);
  }
  for (int q = 0; q < 2 * nt; ++q) {
    const size_t bi = (q < nt ? base0 + (size_t)q * P1 : base1 + (size_t)(q - nt) * P1);
    const Acc* xr = xs + q * NR1 + r0;
    if constexpr (T::f64) {
      const double b = static_cast<const double*>(Sv)[bi];
#pragma unroll
      for (int u = 0; u < RPT; ++u) acc[u] = fma(b, xr[u], acc[u]);
    } else if constexpr (T::f32) {
      const float b = static_cast<const float*>(Sv)[bi];
#pragma unroll
      for (int u = 0; u < RPT; ++u) acc[u] = fmaf(b, xr[u], acc[u]);
    } else {
      const float2 b = block_split<BT>(Sv, bi);
#pragma unroll
      for (int u = 0; u < RPT; ++u) df_fma(acc[u].x, acc[u].y, b, xr[u]);
    }
  }
  const size_t oi = (size_t)f * P1 + s;
#pragma unroll
  for (int u = 0; u < RPT; ++u) {
    const int r = r0 + u;
    if (r >= nrhs) break;
    const size_t yo = (size_t)r * vstride + oi;
    if constexpr (T::f64) {
      double v = acc[u];
      if (escale) v *= escale[f];
      static_cast<double*>(yv)[yo] = v;
    } else if constexpr (T::f32) {
      float v = acc[u];
      if (escale) v = (float)((double)v * escale[f]);
      static_cast<float*>(yv)[yo] = v;
    } else {
      float h = acc[u].x, l = acc[u].y;
      if (escale) {
        float ph = 0.f, pl = 0.f;
        df_fma(ph, pl, df_norm(h, l), df_from(escale[f]));
        h = ph;
        l = pl;
      }
      const float2 o = df_norm(h, l);
      if constexpr (VT == 0) static_cast<double*>(yv)[yo] = df_to(o);
      else if constexpr (VT == 1) static_cast<float2*>(yv)[yo] = o;
      else static_cast<float*>(yv)[yo] = o.x + o.y;
    }
  }
}

template <int BT, int VT>
static cudaError_t launch_mrhs_t(const Params& P, const void* S, const void* x, void* y, int nrhs, int64_t vstride,
                                 const double* escale, cudaStream_t st) {
  using Acc = typename MrhsTypes<BT, VT>::Acc;
  const int groups = (nrhs + RPT - 1) / RPT;
  const int threads = (P.P1 * groups + 31) / 32 * 32;
  const size_t sm = (size_t)2 * P.n_t * mrhs_row(nrhs) * sizeof(Acc);
  if (sm > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t err = cudaFuncSetAttribute(apply_mrhs_kernel<BT, VT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
  if (err != cudaSuccess) return err;
  apply_mrhs_kernel<BT, VT><<<P.n_int, threads, sm, st>>>(P, S, x, y, nrhs, vstride, escale);
  return cudaGetLastError();
}

// bt: 0 FP64 blocks, 1 split-FP32 blocks, 2 FP32 blocks; vt: 0 FP64, 1 split, 2 FP32 vectors.
cudaError_t launch_apply_mrhs(int bt, int vt, const Params& P, const void* S, const void* x, void* y, int nrhs,
                              int64_t vstride, const double* escale, cudaStream_t st) {
  if (nrhs < 1 || nrhs > HDG_MAX_RHS || P.P1 * ((nrhs + RPT - 1) / RPT) > 544) return cudaErrorInvalidValue;
  if (bt == 0 && vt == 0) return launch_mrhs_t<0, 0>(P, S, x, y, nrhs, vstride, escale, st);
  if (bt == 1 && vt == 0) return launch_mrhs_t<1, 0>(P, S, x, y, nrhs, vstride, escale, st);
  if (bt == 2 && vt == 2) return launch_mrhs_t<2, 2>(P, S, x, y, nrhs, vstride, escale, st);
  if (bt == 0 && vt == 1) return launch_mrhs_t<0, 1>(P, S, x, y, nrhs, vstride, escale, st);
  if (bt == 1 && vt == 1) return launch_mrhs_t<1, 1>(P, S, x, y, nrhs, vstride, escale, st);
  if (bt == 2 && vt == 1) return launch_mrhs_t<2, 1>(P, S, x, y, nrhs, vstride, escale, st);
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Element-centric variant for split-FP32 vectors (the batched GMRES operator):
// (A) one CTA per element: Z_e,r = S_e X_e,r for all columns r, X_e gathered
//     once per element ([n_t][nrhs] in shared memory), Z written per element
//     ([N][nrhs][n_t] split pairs);
// (B) one thread per (column, edge dof): y_r(f, s) = scale_f (Z_e+,r(t+) +
//     Z_e-,r(t-)) in a fixed order. Each element's trace values are read once
//     (the edge-centric kernel reads them once per edge of the element).
// cmap (optional): the nrhs columns computed are cmap[0 .. nrhs-1] of x and y
// (the columns still iterating in the batched solver); Z holds them compactly.
template <int BT>
__global__ void __launch_bounds__(256) mrhs_element_kernel(Params P, const void* __restrict__ Sv,
                                                           const float2* __restrict__ x, int nrhs, int64_t vstride,
                                                           float2* __restrict__ Z, const int* __restrict__ cmap) {
  extern __shared__ float2 xs2[];            // [n_t][NR1]
  const int nt = P.n_t, P1 = P.P1, PP = P.P, NR1 = mrhs_row(nrhs);
  const int e = blockIdx.x;
  const int tid = threadIdx.x;
  int code[3], flip[3];
  elem_edges(e, P.n, code, flip);
  for (int idx = tid; idx < nt * (NR1 - 1); idx += blockDim.x) {
    const int r = idx / nt, c = idx - r * nt;
    const int kk = c / P1, t = c - kk * P1;
    float2 v = make_float2(0.f, 0.f);
    if (r < nrhs && code[kk] >= 0 && HDG_INB((size_t)code[kk] * P1 + (flip[kk] ? PP - t : t), P.N_tr, P.oob, 5))
      v = x[(size_t)(cmap ? cmap[r] : r) * vstride + (size_t)code[kk] * P1 + (flip[kk] ? PP - t : t)];
    xs2[c * NR1 + r] = v;
  }
  __syncthreads();
  const int groups = (nrhs + RPT - 1) / RPT;
  const size_t sb = (size_t)e * 3 * nt * P1;
  for (int item = tid; item < nt * groups; item += blockDim.x) {
    const int row = item % nt, grp = item / nt;
    const int k = row / P1, t = row - k * P1;
    const int r0 = grp * RPT;
    float h[RPT], l[RPT];
#pragma unroll
    for (int u = 0; u < RPT; ++u) { h[u] = 0.f; l[u] = 0.f; }
    const size_t rb = sb + (size_t)k * nt * P1 + t;     // S_e(row, c) = S[e][k][c][t]
    for (int c = 0; c < nt; ++c) {
      const float2 b = block_split<BT>(Sv, rb + (size_t)c * P1);
      const float2* xr = xs2 + c * NR1 + r0;
#pragma unroll
      for (int u = 0; u < RPT; ++u) df_fma(h[u], l[u], b, xr[u]);
    }
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      const int r = r0 + u;
      if (r < nrhs) Z[((size_t)e * nrhs + r) * nt + row] = df_norm(h[u], l[u]);
    }
  }
}

__global__ void mrhs_edge_sum_kernel(Params P, const float2* __restrict__ Z, int nrhs, int64_t vstride,
                                     const double* __restrict__ escale, float2* __restrict__ y,
                                     const int* __restrict__ cmap) {
  const int nt = P.n_t, P1 = P.P1, PP = P.P;
  const int64_t per = (int64_t)P.n_int * P1;
  const int64_t total = per * nrhs;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / per);
    const int64_t fs = idx - (int64_t)r * per;
    const int f = (int)(fs / P1), s = (int)(fs - (int64_t)f * P1);
    int e[2], k[2], fl[2];
    double len;
    edge_sides(f, P.n, e, k, fl, &len);
    float h = 0.f, l = 0.f;
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      const int t = fl[sd] ? PP - s : s;
      if (!HDG_INB((int64_t)e[sd] * 3 + k[sd], 3LL * P.N, P.oob, 6) || !HDG_INB(t, P1, P.oob, 6)) continue;
      const float2 z = Z[((size_t)e[sd] * nrhs + r) * nt + k[sd] * P1 + t];
      df_add(h, l, z.x, z.y);
    }
    if (escale) {
      float ph = 0.f, pl = 0.f;
      df_fma(ph, pl, df_norm(h, l), df_from(escale[f]));
      h = ph;
      l = pl;
    }
    y[(size_t)(cmap ? cmap[r] : r) * vstride + fs] = df_norm(h, l);
  }
}

// The same two kernels on FP64 vectors (the batched solve with the FP64
// Krylov basis): products in the block type's arithmetic (BT = 0: FP64
// fused multiply-adds, 1: split-FP32, 2: FP32), Z and the two-side sum in FP64.
template <int BT>
struct MrhsAccD;
template <>
struct MrhsAccD<0> { using T = double; };
template <>
struct MrhsAccD<1> { using T = float2; };
template <>
struct MrhsAccD<2> { using T = float; };

template <int BT>
__global__ void __launch_bounds__(256) mrhs_element_d_kernel(Params P, const void* __restrict__ Sv,
                                                             const double* __restrict__ x, int nrhs, int64_t vstride,
                                                             double* __restrict__ Z, const int* __restrict__ cmap) {
  using A = typename MrhsAccD<BT>::T;
  extern __shared__ unsigned char xraw[];
  A* xs = reinterpret_cast<A*>(xraw);          // [n_t][NR1]
  const int nt = P.n_t, P1 = P.P1, PP = P.P, NR1 = mrhs_row(nrhs);
  const int e = blockIdx.x;
  const int tid = threadIdx.x;
  int code[3], flip[3];
  elem_edges(e, P.n, code, flip);
  for (int idx = tid; idx < nt * (NR1 - 1); idx += blockDim.x) {
    const int r = idx / nt, c = idx - r * nt;
    const int kk = c / P1, t = c - kk * P1;
    double v = 0.0;
    if (r < nrhs && code[kk] >= 0 && HDG_INB((size_t)code[kk] * P1 + (flip[kk] ? PP - t : t), P.N_tr, P.oob, 5))
      v = x[(size_t)(cmap ? cmap[r] : r) * vstride + (size_t)code[kk] * P1 + (flip[kk] ? PP - t : t)];
    if constexpr (BT == 0) xs[c * NR1 + r] = v;
    else if constexpr (BT == 1) xs[c * NR1 + r] = df_from(v);
    else xs[c * NR1 + r] = (float)v;
  }
  __syncthreads();
  const int groups = (nrhs + RPT - 1) / RPT;
  const size_t sb = (size_t)e * 3 * nt * P1;
  for (int item = tid; item < nt * groups; item += blockDim.x) {
    const int row = item % nt, grp = item / nt;
    const int k = row / P1, t = row - k * P1;
    const int r0 = grp * RPT;
    const size_t rb = sb + (size_t)k * nt * P1 + t;     // S_e(row, c) = S[e][k][c][t]
    double out[RPT];
    if constexpr (BT == 0) {
      const double* S = static_cast<const double*>(Sv);
      double acc[RPT];
#pragma unroll
      for (int u = 0; u < RPT; ++u) acc[u] = 0.0;
      for (int c = 0; c < nt; ++c) {
        const double bv = S[rb + (size_t)c * P1];
        const double* xr = xs + c * NR1 + r0;
#pragma unroll
        for (int u = 0; u < RPT; ++u) acc[u] = fma(bv, xr[u], acc[u]);
      }
#pragma unroll
      for (int u = 0; u < RPT; ++u) out[u] = acc[u];
    } else if constexpr (BT == 1) {
      const float2* S = static_cast<const float2*>(Sv);
      float h[RPT], l[RPT];
#pragma unroll
      for (int u = 0; u < RPT; ++u) { h[u] = 0.f; l[u] = 0.f; }
      for (int c = 0; c < nt; ++c) {
        const float2 bv = S[rb + (size_t)c * P1];
        const float2* xr = xs + c * NR1 + r0;
#pragma unroll
        for (int u = 0; u < RPT; ++u) df_fma(h[u], l[u], bv, xr[u]);
      }
#pragma unroll
      for (int u = 0; u < RPT; ++u) out[u] = df_to(df_norm(h[u], l[u]));
    } else {
      const float* S = static_cast<const float*>(Sv);
      float acc[RPT];
#pragma unroll
      for (int u = 0; u < RPT; ++u) acc[u] = 0.f;
      for (int c = 0; c < nt; ++c) {
        const float bv = S[rb + (size_t)c * P1];
        const float* xr = xs + c * NR1 + r0;
#pragma unroll
        for (int u = 0; u < RPT; ++u) acc[u] = fmaf(bv, xr[u], acc[u]);
      }
#pragma unroll
      for (int u = 0; u < RPT; ++u) out[u] = (double)acc[u];
    }
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      const int r = r0 + u;
      if (r < nrhs) Z[((size_t)e * nrhs + r) * nt + row] = out[u];
    }
  }
}

__global__ void mrhs_edge_sum_d_kernel(Params P, const double* __restrict__ Z, int nrhs, int64_t vstride,
                                       const double* __restrict__ escale, double* __restrict__ y,
                                       const int* __restrict__ cmap) {
  const int nt = P.n_t, P1 = P.P1, PP = P.P;
  const int64_t per = (int64_t)P.n_int * P1;
  const int64_t total = per * nrhs;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / per);
    const int64_t fs = idx - (int64_t)r * per;
    const int f = (int)(fs / P1), s = (int)(fs - (int64_t)f * P1);
    int e[2], k[2], fl[2];
    double len;
    edge_sides(f, P.n, e, k, fl, &len);
    double v = 0.0;
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      const int t = fl[sd] ? PP - s : s;
      if (!HDG_INB((int64_t)e[sd] * 3 + k[sd], 3LL * P.N, P.oob, 6) || !HDG_INB(t, P1, P.oob, 6)) continue;
      v += Z[((size_t)e[sd] * nrhs + r) * nt + k[sd] * P1 + t];
    }
    if (escale) v *= escale[f];
    y[(size_t)(cmap ? cmap[r] : r) * vstride + fs] = v;
  }
}

// Element-centric multi-RHS apply; Z: [N][nrhs][n_t] (split pairs for split
// vectors, FP64 for FP64 vectors). vt: 0 FP64 / 1 split-FP32 vectors.
cudaError_t launch_apply_mrhs_el(int bt, const Params& P, const void* S, const void* x, void* y, int nrhs,
                                 int64_t vstride, const double* escale, void* Z, cudaStream_t st, const int* cmap,
                                 int vt) {
  if (nrhs < 1 || nrhs > HDG_MAX_RHS || bt < 0 || bt > 2) return cudaErrorInvalidValue;
  const size_t el = (vt == 0 && bt == 2) ? sizeof(float) : 8;
  const size_t sm = (size_t)P.n_t * mrhs_row(nrhs) * el;
  if (sm > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t err = cudaSuccess;
  auto run = [&](auto kern, auto xp, auto zp) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err == cudaSuccess) kern<<<P.N, 256, sm, st>>>(P, S, xp, nrhs, vstride, zp, cmap);
  };
  const float2* xf = static_cast<const float2*>(x);
  float2* zf = static_cast<float2*>(Z);
  const double* xd = static_cast<const double*>(x);
  double* zd = static_cast<double*>(Z);
  if (vt == 1) {
    if (bt == 0) run(mrhs_element_kernel<0>, xf, zf);
    else if (bt == 1) run(mrhs_element_kernel<1>, xf, zf);
    else run(mrhs_element_kernel<2>, xf, zf);
  } else {
    if (bt == 0) run(mrhs_element_d_kernel<0>, xd, zd);
    else if (bt == 1) run(mrhs_element_d_kernel<1>, xd, zd);
    else run(mrhs_element_d_kernel<2>, xd, zd);
  }
  if (err != cudaSuccess) return err;
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (vt == 1)
    mrhs_edge_sum_kernel<<<4 * 152 * 8, 256, 0, st>>>(P, zf, nrhs, vstride, escale, static_cast<float2*>(y), cmap);
  else
    mrhs_edge_sum_d_kernel<<<4 * 152 * 8, 256, 0, st>>>(P, zd, nrhs, vstride, escale, static_cast<double*>(y), cmap);
  return cudaGetLastError();
}

}  // namespace mehdg
