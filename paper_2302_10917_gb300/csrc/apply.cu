// Matrix-free trace-operator apply (Sec. 3.3.2, steps 1-4) over stored Schur
// blocks, edge-centric so that step 4 (the face reduction) needs no second
// pass and no atomics.
//
// Steps 1-3 of the paper, v^_e = C_e A_e^-1 B_e u^_e, are folded into the
// stored S_e = D_e - C_e A_e^-1 B_e (Eq. global_problem); step 4 sums the two
// element sides of every interior face in a fixed order (deterministic):
//   y_f = (S_{e+} x_{e+})|_f + (S_{e-} x_{e-})|_f .
// With the D^-1 preconditioner of Sec. 6.1, D_f = -(tau+ + tau-) L_f Gh (the
// advective parts cancel across a face), so D_f^-1 = scale_f Gh^-1; Gh^-1 is
// folded into the stored row-blocks at condensation and step 4 reduces to a
// per-face scale.
//
// One thread per (interior edge, trace position); a CTA covers EPB whole
// edges, stages the two element trace vectors of each edge in shared memory
// (gathered with orientation flips, Dirichlet edges contribute 0) and streams
// the matching row-blocks S[e][k][j][t] (contiguous in t) from HBM.
#include "internal.h"
#include "df64.h"
#include <type_traits>

namespace mehdg {

int apply_edges_per_block(const Params& P) {
  int epb = 256 / P.P1;
  return epb < 1 ? 1 : epb;
}

template <typename T, typename TX, typename Acc>
__global__ void __launch_bounds__(256) apply_kernel(Params P, const T* __restrict__ S, const TX* __restrict__ x,
                                                    TX* __restrict__ y, const double* __restrict__ escale,
                                                    int epb, const int* __restrict__ stop) {
  if (stop && *stop) return;
  extern __shared__ unsigned char sraw[];
  Acc* xs = reinterpret_cast<Acc*>(sraw);   // [epb][2][n_t]
  const int nt = P.n_t, P1 = P.P1, PP = P.P;
  const int f0 = blockIdx.x * epb;
  const int tid = threadIdx.x;

  // gather the element trace vectors of both sides of every edge of the CTA
  for (int idx = tid; idx < epb * 2 * nt; idx += blockDim.x) {
    const int le = idx / (2 * nt);
    const int rem = idx - le * 2 * nt;
    const int sd = rem / nt, c = rem - sd * nt;
    const int f = f0 + le;
    Acc v = Acc(0);
    if (f < P.n_int) {
      int e[2], k[2], fl[2];
      double len;
      edge_sides(f, P.n, e, k, fl, &len);
      int code[3], flip[3];
      elem_edges(e[sd], P.n, code, flip);
      const int kk = c / P1, t = c - kk * P1;
      if (code[kk] >= 0) v = Acc(x[(size_t)code[kk] * P1 + (flip[kk] ? PP - t : t)]);
    }
    xs[idx] = v;
  }
  __syncthreads();

  const int le = tid / P1, s = tid - le * P1;
  const int f = f0 + le;
  if (le >= epb || f >= P.n_int) return;
  int e[2], k[2], fl[2];
  double len;
  edge_sides(f, P.n, e, k, fl, &len);
  Acc acc0 = Acc(0), acc1 = Acc(0);
#pragma unroll
  for (int sd = 0; sd < 2; ++sd) {
    const int t = fl[sd] ? PP - s : s;
    const T* base = S + ((size_t)e[sd] * 3 + k[sd]) * (size_t)nt * P1 + t;
    const Acc* xv = xs + (le * 2 + sd) * nt;
    int j = 0;
    for (; j + 8 <= nt; j += 8) {
      T sv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) sv[u] = base[(size_t)(j + u) * P1];
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        acc0 += Acc(sv[u]) * xv[j + u];
        acc1 += Acc(sv[u + 1]) * xv[j + u + 1];
      }
    }
    for (; j < nt; ++j) acc0 += Acc(base[(size_t)j * P1]) * xv[j];
  }
  Acc r = acc0 + acc1;
  if (escale) r *= Acc(escale[f]);
  y[(size_t)f * P1 + s] = TX(r);
}

// ---------------------------------------------------------------------------
// Split-FP32 ("double-float") variant. GB300 issues FP64 FMAs at 1/63 of the
// FP32 rate, so the FP64 apply above is bound by the FP64 pipe, not by HBM.
// Here each block entry is stored as an unevaluated sum hi + lo of two FP32
// numbers (hi = fl32(s), lo = fl32(s - hi); 48 significant bits, same 8 bytes
// per entry), x is split the same way on the fly, and every product is
// accumulated with error-free transformations (Dekker's product via FMA,
// Knuth's two-sum) on the FP32 pipe; the two FP32 words are combined in FP64
// once per output.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) apply_df_kernel(Params P, const float2* __restrict__ S,
                                                       const double* __restrict__ x, double* __restrict__ y,
                                                       const double* __restrict__ escale, int epb,
                                                       const int* __restrict__ stop) {
  if (stop && *stop) return;
  extern __shared__ unsigned char sraw[];
  float2* xs = reinterpret_cast<float2*>(sraw);   // [epb][2][n_t] (hi, lo)
  const int nt = P.n_t, P1 = P.P1, PP = P.P;
  const int f0 = blockIdx.x * epb;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < epb * 2 * nt; idx += blockDim.x) {
    const int le = idx / (2 * nt);
    const int rem = idx - le * 2 * nt;
    const int sd = rem / nt, c = rem - sd * nt;
    const int f = f0 + le;
    double v = 0.0;
    if (f < P.n_int) {
      int e[2], k[2], fl[2];
      double len;
      edge_sides(f, P.n, e, k, fl, &len);
      int code[3], flip[3];
      elem_edges(e[sd], P.n, code, flip);
      const int kk = c / P1, t = c - kk * P1;
      if (code[kk] >= 0) v = x[(size_t)code[kk] * P1 + (flip[kk] ? PP - t : t)];
    }
    const float hi = (float)v;
    xs[idx] = make_float2(hi, (float)(v - (double)hi));
  }
  __syncthreads();
  const int le = tid / P1, s = tid - le * P1;
  const int f = f0 + le;
  if (le >= epb || f >= P.n_int) return;
  int e[2], k[2], fl[2];
  double len;
  edge_sides(f, P.n, e, k, fl, &len);
  float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
#pragma unroll
  for (int sd = 0; sd < 2; ++sd) {
    const int t = fl[sd] ? PP - s : s;
    const float2* base = S + ((size_t)e[sd] * 3 + k[sd]) * (size_t)nt * P1 + t;
    const float2* xv = xs + (le * 2 + sd) * nt;
    int j = 0;
    for (; j + 8 <= nt; j += 8) {
      float2 sv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) sv[u] = base[(size_t)(j + u) * P1];
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        df_fma(h0, l0, sv[u], xv[j + u]);
        df_fma(h1, l1, sv[u + 1], xv[j + u + 1]);
      }
    }
    for (; j < nt; ++j) {
      df_fma(h0, l0, base[(size_t)j * P1], xv[j]);
    }
  }
  double r = ((double)h0 + (double)h1) + ((double)l0 + (double)l1);
  if (escale) r *= escale[f];
  y[(size_t)f * P1 + s] = r;
}

// The same edge-centric apply on split-FP32 vectors (Krylov basis storage):
// BT = 0: FP64 blocks, FP64 accumulation; BT = 1: split-FP32 blocks and
// accumulation on the FP32 pipe; BT = 2: FP32 blocks, FP32 accumulation.
template <int BT>
__global__ void __launch_bounds__(512) apply_vdf_kernel(Params P, const void* __restrict__ Sv,
                                                        const float2* __restrict__ x, float2* __restrict__ y,
                                                        const double* __restrict__ escale, int epb,
                                                        const int* __restrict__ stop) {
  if (stop && *stop) return;
  using XT = typename std::conditional<BT == 0, double, typename std::conditional<BT == 1, float2, float>::type>::type;
  extern __shared__ unsigned char sraw[];
  XT* xs = reinterpret_cast<XT*>(sraw);   // [epb][2][n_t]
  const int nt = P.n_t, P1 = P.P1, PP = P.P;
  const int f0 = blockIdx.x * epb;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < epb * 2 * nt; idx += blockDim.x) {
    const int le = idx / (2 * nt);
    const int rem = idx - le * 2 * nt;
    const int sd = rem / nt, c = rem - sd * nt;
    const int f = f0 + le;
    float2 v = make_float2(0.f, 0.f);
    if (f < P.n_int) {
      int e[2], k[2], fl[2];
      double len;
      edge_sides(f, P.n, e, k, fl, &len);
      int code[3], flip[3];
      elem_edges(e[sd], P.n, code, flip);
      const int kk = c / P1, t = c - kk * P1;
      if (code[kk] >= 0) v = x[(size_t)code[kk] * P1 + (flip[kk] ? PP - t : t)];
    }
    if constexpr (BT == 0) xs[idx] = df_to(v);
    else if constexpr (BT == 1) xs[idx] = v;
    else xs[idx] = v.x;
  }
  __syncthreads();
  const int le = tid / P1, s = tid - le * P1;
  const int f = f0 + le;
  if (le >= epb || f >= P.n_int) return;
  int e[2], k[2], fl[2];
  double len;
  edge_sides(f, P.n, e, k, fl, &len);
  float2 out;
  // row t_side of each side's row-block (the edge dof s in the element's orientation)
  const int t0 = fl[0] ? PP - s : s, t1 = fl[1] ? PP - s : s;
  if constexpr (BT == 1) {
    const float2* S = static_cast<const float2*>(Sv);
    float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
    // side by side: the row of this trace position is a stride-P1 walk through the
    // element's row-block; groups of 8 loads, the next group issued before the
    // products of the current one, two independent accumulators
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      const float2* bp = S + ((size_t)e[sd] * 3 + k[sd]) * (size_t)nt * P1 + (sd ? t1 : t0);
      const float2* xv = xs + (le * 2 + sd) * nt;
      const int ng = nt / 8;                 // full groups of 8
      float2 cur[8], nxt[8];
      if (ng > 0) {
#pragma unroll
        for (int u = 0; u < 8; ++u) cur[u] = bp[u * P1];
      }
      for (int g = 0; g < ng; ++g) {
        const int j = g * 8;
        if (g + 1 < ng) {
#pragma unroll
          for (int u = 0; u < 8; ++u) nxt[u] = bp[(j + 8 + u) * P1];
        }
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
          df_fma(h0, l0, cur[u], xv[j + u]);
          df_fma(h1, l1, cur[u + 1], xv[j + u + 1]);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) cur[u] = nxt[u];
      }
      for (int j = ng * 8; j < nt; ++j) df_fma(h0, l0, bp[j * P1], xv[j]);
    }
    df_add(h0, l0, h1, l1);
    if (escale) {
      const float2 sc = df_from(escale[f]);
      float ph = 0.f, pl = 0.f;
      df_fma(ph, pl, make_float2(h0, l0), sc);
      h0 = ph;
      l0 = pl;
    }
    out = df_norm(h0, l0);
  } else if constexpr (BT == 2) {
    // both sides' terms as one sequence q = 0 .. 2 n_t - 1; loads of the next
    // batch of G2 are issued before the arithmetic of the current one (4-byte
    // entries: twice the split variant's loads in flight for the same bytes)
    constexpr int G2 = 16;
    const int nq = 2 * nt;
    const float* S = static_cast<const float*>(Sv);
    const float* b0 = S + ((size_t)e[0] * 3 + k[0]) * (size_t)nt * P1 + t0;
    const float* b1 = S + ((size_t)e[1] * 3 + k[1]) * (size_t)nt * P1 + t1 - (size_t)nt * P1;
    const float* xv = xs + le * 2 * nt;
    float acc0 = 0.f, acc1 = 0.f;
    float cur[G2], nxt[G2];
#pragma unroll
    for (int u = 0; u < G2; ++u) cur[u] = u < nq ? (u < nt ? b0 : b1)[(size_t)u * P1] : 0.f;
    for (int q0 = 0; q0 < nq; q0 += G2) {
#pragma unroll
      for (int u = 0; u < G2; ++u) {
        const int q = q0 + G2 + u;
        nxt[u] = q < nq ? (q < nt ? b0 : b1)[(size_t)q * P1] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < G2; u += 2) {
        const int q = q0 + u;
        if (q < nq) acc0 = fmaf(cur[u], xv[q], acc0);
        if (q + 1 < nq) acc1 = fmaf(cur[u + 1], xv[q + 1], acc1);
      }
#pragma unroll
      for (int u = 0; u < G2; ++u) cur[u] = nxt[u];
    }
    float r = acc0 + acc1;
    if (escale) r *= (float)escale[f];
    out = make_float2(r, 0.f);
  } else {
    const double* S = static_cast<const double*>(Sv);
    double acc0 = 0.0, acc1 = 0.0;
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      const double* base = S + ((size_t)e[sd] * 3 + k[sd]) * (size_t)nt * P1 + (sd ? t1 : t0);
      const XT* xv = xs + (le * 2 + sd) * nt;
      int j = 0;
      for (; j + 8 <= nt; j += 8) {
        double sv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) sv[u] = base[(size_t)(j + u) * P1];
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
          acc0 += sv[u] * xv[j + u];
          acc1 += sv[u + 1] * xv[j + u + 1];
        }
      }
      for (; j < nt; ++j) acc0 += base[(size_t)j * P1] * xv[j];
    }
    double r = acc0 + acc1;
    if (escale) r *= escale[f];
    out = df_from(r);
  }
  y[(size_t)f * P1 + s] = out;
}

cudaError_t launch_apply_vdf(int bt, const Params& P, const void* S, const float2* x, float2* y,
                             const double* escale, const int* stop, cudaStream_t st, int epb) {
  // epb edges per block, one thread per (edge, trace position): at most 512 threads
  if (epb <= 0 || epb * P.P1 > 512) epb = apply_edges_per_block(P);
  const int threads = (epb * P.P1 + 31) / 32 * 32;
  const int grid = (P.n_int + epb - 1) / epb;
  const size_t el = bt == 0 ? sizeof(double) : (bt == 1 ? sizeof(float2) : sizeof(float));
  const size_t sm = (size_t)epb * 2 * P.n_t * el;
  if (bt == 0) apply_vdf_kernel<0><<<grid, threads, sm, st>>>(P, S, x, y, escale, epb, stop);
  else if (bt == 1) apply_vdf_kernel<1><<<grid, threads, sm, st>>>(P, S, x, y, escale, epb, stop);
  else apply_vdf_kernel<2><<<grid, threads, sm, st>>>(P, S, x, y, escale, epb, stop);
  return cudaGetLastError();
}

// Split an FP64 array into hi/lo FP32 pairs.
__global__ void split_df_kernel(const double* __restrict__ a, float2* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = a[i];
    const float hi = (float)v;
    out[i] = make_float2(hi, (float)(v - (double)hi));
  }
}


cudaError_t launch_apply64(const Params& P, const double* S, const double* x, double* y, const double* escale,
                           const int* stop, cudaStream_t st) {
  const int epb = apply_edges_per_block(P);
  const int grid = (P.n_int + epb - 1) / epb;
  const size_t sm = (size_t)epb * 2 * P.n_t * sizeof(double);
  apply_kernel<double, double, double><<<grid, 256, sm, st>>>(P, S, x, y, escale, epb, stop);
  return cudaGetLastError();
}

cudaError_t launch_apply_df(const Params& P, const float2* S, const double* x, double* y, const double* escale,
                            const int* stop, cudaStream_t st) {
  const int epb = apply_edges_per_block(P);
  const int grid = (P.n_int + epb - 1) / epb;
  const size_t sm = (size_t)epb * 2 * P.n_t * sizeof(float2);
  apply_df_kernel<<<grid, 256, sm, st>>>(P, S, x, y, escale, epb, stop);
  return cudaGetLastError();
}

cudaError_t launch_split_df(const double* a, float2* out, int64_t n, cudaStream_t st) {
  split_df_kernel<<<2048, 256, 0, st>>>(a, out, n);
  return cudaGetLastError();
}

cudaError_t launch_apply32(const Params& P, const float* S, const float* x, float* y, const double* escale,
                           const int* stop, cudaStream_t st) {
  const int epb = apply_edges_per_block(P);
  const int grid = (P.n_int + epb - 1) / epb;
  const size_t sm = (size_t)epb * 2 * P.n_t * sizeof(float);
  apply_kernel<float, float, float><<<grid, 256, sm, st>>>(P, S, x, y, escale, epb, stop);
  return cudaGetLastError();
}


// Assembled right-hand side: g_f = gel_{e+}|_f + gel_{e-}|_f (fixed order).
__global__ void assemble_rhs_kernel(Params P, const double* gel, double* g) {
  const int64_t total = (int64_t)P.n_int * P.P1;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int f = (int)(idx / P.P1), s = (int)(idx - (int64_t)f * P.P1);
    int e[2], k[2], fl[2];
    double len;
    edge_sides(f, P.n, e, k, fl, &len);
    double acc = 0.0;
    for (int sd = 0; sd < 2; ++sd) {
      const int t = fl[sd] ? P.P - s : s;
      acc += gel[(size_t)e[sd] * P.n_t + k[sd] * P.P1 + t];
    }
    g[idx] = acc;
  }
}

// Face preconditioner on a vector: z_f = scale_f Gh^-1 y_f (Sec. 6.1).
__global__ void face_dinv_kernel(Params P, const double* Ghinv, const double* escale, const double* y, double* z) {
  const int64_t total = (int64_t)P.n_int * P.P1;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int f = (int)(idx / P.P1), s = (int)(idx - (int64_t)f * P.P1);
    const double* yf = y + (size_t)f * P.P1;
    double acc = 0.0;
    for (int t = 0; t < P.P1; ++t) acc += Ghinv[s * P.P1 + t] * yf[t];
    z[idx] = escale[f] * acc;
  }
}

// Per-face scale -1 / ((tau+ + tau-) L_f) of D_f^-1.
__global__ void face_scale_kernel(Params P, const double* kappa, double* escale) {
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < P.n_int; f += gridDim.x * blockDim.x) {
    int e[2], k[2], fl[2];
    double len;
    edge_sides(f, P.n, e, k, fl, &len);
    const double tsum = kappa[e[0]] / P.tau_len + kappa[e[1]] / P.tau_len + 2.0 * P.babs;
    escale[f] = -1.0 / (tsum * len);
  }
}

cudaError_t launch_assemble_rhs(const Params& P, const double* gel, double* g, cudaStream_t st) {
  assemble_rhs_kernel<<<1024, 256, 0, st>>>(P, gel, g);
  return cudaGetLastError();
}

cudaError_t launch_face_dinv(const Params& P, const double* Ghinv, const double* escale, const double* y, double* z,
                             cudaStream_t st) {
  face_dinv_kernel<<<1024, 256, 0, st>>>(P, Ghinv, escale, y, z);
  return cudaGetLastError();
}

cudaError_t launch_face_scale(const Params& P, const double* kappa, double* escale, cudaStream_t st) {
  face_scale_kernel<<<256, 256, 0, st>>>(P, kappa, escale);
  return cudaGetLastError();
}

}  // namespace mehdg
