// Restarted GMRES for the condensed trace system S x = g (Eq. global_problem),
// left-preconditioned by D^-1 (Sec. 6.1): the Krylov space is built for
// D^-1 S with right-hand side D^-1 g.
//
// The paper uses PETSc GMRES and fixes neither restart length,
// orthogonalisation nor stopping rule. Here: classical Gram-Schmidt applied
// twice (CGS2), Givens rotations on the device, and a device stop flag so a
// whole restart cycle is enqueued without host round trips; every kernel of
// the cycle returns at once when the flag is set. Convergence is decided on
// the TRUE relative residual ||g - S x|| / ||g|| (FP64 S), evaluated at each
// restart; the Arnoldi estimate of the preconditioned residual only decides
// when a cycle ends early. All reductions have a fixed order, so results are
// bitwise reproducible run to run.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>
#include "launch.h"

namespace mehdg {

constexpr int KG = 608;       // blocks of the vector kernels (4 per SM)
constexpr int KT = 256;       // threads per block
constexpr int VG = 8;         // vectors per pass of the multi-dot

// small-array layout (doubles) for restart length K
struct SmallLayout {
  int K;
  int H, cs, sn, gv, y, htmp, sc;
  int total;
  explicit SmallLayout(int k) : K(k) {
    H = 0;
    cs = H + (K + 1) * K;
    sn = cs + K;
    gv = sn + K;
    y = gv + K + 1;
    htmp = y + K;
    sc = htmp + K + 1;   // scalars: 0 beta, 1 est, 2 target, 3 hn, 4 inv, 5 norm
    total = sc + 8;
  }
};
enum { F_STOP = 0, F_JUSED = 1 };

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;   // valid in thread 0
}

// part[b * nv + i] = sum_{idx in chunk b} V_i[idx] w[idx]
__global__ void __launch_bounds__(KT) mdot_kernel(const double* __restrict__ V, int64_t n, int nv,
                                                  const double* __restrict__ w, double* part, const int* stop) {
  if (stop && stop[F_STOP]) return;
  __shared__ double red[KT / 32];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  for (int g0 = 0; g0 < nv; g0 += VG) {
    double acc[VG];
#pragma unroll
    for (int g = 0; g < VG; ++g) acc[g] = 0.0;
    for (int64_t idx = lo + threadIdx.x; idx < hi; idx += blockDim.x) {
      const double wv = w[idx];
#pragma unroll
      for (int g = 0; g < VG; ++g)
        if (g0 + g < nv) acc[g] += V[(size_t)(g0 + g) * n + idx] * wv;
    }
#pragma unroll
    for (int g = 0; g < VG; ++g) {
      if (g0 + g >= nv) break;
      const double s = block_sum(acc[g], red);
      if (threadIdx.x == 0) part[(size_t)blockIdx.x * nv + g0 + g] = s;
    }
  }
}

// out[i] = sum_b part[b * nv + i] in block order; mode 0: H column := s,
// mode 1: H column += s. htmp receives s (the coefficients of the update).
__global__ void mdot_reduce_kernel(const double* part, int G, int nv, double* Hcol, double* htmp, int mode,
                                   const int* stop) {
  if (stop && stop[F_STOP]) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = wid; i < nv; i += nw) {
    double s = 0.0;
    for (int b = lane; b < G; b += 32) s += part[(size_t)b * nv + i];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) {
      htmp[i] = s;
      Hcol[i] = mode ? Hcol[i] + s : s;
    }
  }
}

// w += sign * sum_i coef[i] V_i; optionally part[b] = sum over the block of w^2.
__global__ void __launch_bounds__(KT) update_kernel(const double* __restrict__ V, int64_t n, int nv,
                                                    const double* __restrict__ coef, double sign, double* w,
                                                    double* part, const int* stop) {
  if (stop && stop[F_STOP]) return;
  __shared__ double red[KT / 32];
  __shared__ double cf[130];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) cf[i] = sign * coef[i];
  __syncthreads();
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  double ss = 0.0;
  for (int64_t idx = lo + threadIdx.x; idx < hi; idx += blockDim.x) {
    double v = w[idx];
    int i = 0;
    for (; i + 4 <= nv; i += 4) {
      const double a0 = V[(size_t)(i + 0) * n + idx], a1 = V[(size_t)(i + 1) * n + idx];
      const double a2 = V[(size_t)(i + 2) * n + idx], a3 = V[(size_t)(i + 3) * n + idx];
      v += cf[i] * a0;
      v += cf[i + 1] * a1;
      v += cf[i + 2] * a2;
      v += cf[i + 3] * a3;
    }
    for (; i < nv; ++i) v += cf[i] * V[(size_t)i * n + idx];
    w[idx] = v;
    ss += v * v;
  }
  if (part) {
    const double s = block_sum(ss, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------
// Fused CGS2 passes for nv <= NVMAX basis vectors. Each thread keeps the nv
// basis entries of its index in registers; per-vector partial dot products
// are reduced across the warp with shuffles and accumulated by lane (i % 32).
// part[b * stride + i] receives the block's partial sum of vector i.
// ---------------------------------------------------------------------------
template <int NVMAX>
__device__ __forceinline__ void warp_dots_accum(const double (&v)[NVMAX], int nv, double wv,
                                                double (&acc)[(NVMAX + 31) / 32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < NVMAX; ++i) {
    if (i >= nv) break;
    double p = v[i] * wv;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) p += __shfl_xor_sync(0xffffffffu, p, off);
    if (lane == (i & 31)) acc[i >> 5] += p;
  }
}

template <int NVMAX>
__device__ __forceinline__ void block_store_dots(const double (&acc)[(NVMAX + 31) / 32], int nv, double* red,
                                                 double* out) {
  // red: [nwarps][NVMAX]
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int a = 0; a < (NVMAX + 31) / 32; ++a)
    if (a * 32 + lane < nv) red[wid * NVMAX + a * 32 + lane] = acc[a];
  __syncthreads();
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    double s = 0.0;
    for (int w2 = 0; w2 < nw; ++w2) s += red[w2 * NVMAX + i];
    out[i] = s;
  }
}

// part[b * (nv + 1) + i] = sum_chunk V_i w  (i < nv)
template <int NVMAX>
__global__ void __launch_bounds__(KT) cgs_dot_kernel(const double* __restrict__ V, int64_t n, int nv,
                                                     const double* __restrict__ w, double* part, const int* stop) {
  if (stop && stop[F_STOP]) return;
  __shared__ double red[(KT / 32) * NVMAX];
  const int64_t chunk = ((n + gridDim.x - 1) / gridDim.x + 31) / 32 * 32;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  double acc[(NVMAX + 31) / 32];
#pragma unroll
  for (int a = 0; a < (NVMAX + 31) / 32; ++a) acc[a] = 0.0;
  for (int64_t base = lo; base < hi; base += blockDim.x) {
    const int64_t idx = base + threadIdx.x;
    const bool in = idx < hi;
    double v[NVMAX];
#pragma unroll
    for (int i = 0; i < NVMAX; ++i) v[i] = (i < nv && in) ? V[(size_t)i * n + idx] : 0.0;
    const double wv = in ? w[idx] : 0.0;
    warp_dots_accum<NVMAX>(v, nv, wv, acc);
  }
  block_store_dots<NVMAX>(acc, nv, red, part + (size_t)blockIdx.x * (nv + 1));
}

// w' = w - sum_i h_i V_i (stored in place); part[b * (nv + 1) + i] = sum_chunk V_i w',
// part[b * (nv + 1) + nv] = sum_chunk w'^2
template <int NVMAX>
__global__ void __launch_bounds__(KT) cgs_update_dot_kernel(const double* __restrict__ V, int64_t n, int nv,
                                                            const double* __restrict__ h, double* w, double* part,
                                                            const int* stop) {
  if (stop && stop[F_STOP]) return;
  __shared__ double red[(KT / 32) * NVMAX];
  __shared__ double hs[NVMAX];
  __shared__ double ssum[KT / 32];
  for (int i = threadIdx.x; i < NVMAX; i += blockDim.x) hs[i] = i < nv ? h[i] : 0.0;
  __syncthreads();
  const int64_t chunk = ((n + gridDim.x - 1) / gridDim.x + 31) / 32 * 32;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  double acc[(NVMAX + 31) / 32];
#pragma unroll
  for (int a = 0; a < (NVMAX + 31) / 32; ++a) acc[a] = 0.0;
  double ss = 0.0;
  for (int64_t base = lo; base < hi; base += blockDim.x) {
    const int64_t idx = base + threadIdx.x;
    const bool in = idx < hi;
    double v[NVMAX];
#pragma unroll
    for (int i = 0; i < NVMAX; ++i) v[i] = (i < nv && in) ? V[(size_t)i * n + idx] : 0.0;
    double wv = in ? w[idx] : 0.0;
#pragma unroll
    for (int i = 0; i < NVMAX; ++i)
      if (i < nv) wv -= hs[i] * v[i];
    if (in) w[idx] = wv;
    ss += wv * wv;
    warp_dots_accum<NVMAX>(v, nv, wv, acc);
  }
  block_store_dots<NVMAX>(acc, nv, red, part + (size_t)blockIdx.x * (nv + 1));
  for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
  if ((threadIdx.x & 31) == 0) ssum[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) s += ssum[w2];
    part[(size_t)blockIdx.x * (nv + 1) + nv] = s;
  }
}

// V_{j+1} = (w' - sum_i h_i V_i) * sm[inv_off]
template <int NVMAX>
__global__ void __launch_bounds__(KT) cgs_update_scale_kernel(const double* __restrict__ V, int64_t n, int nv,
                                                              const double* __restrict__ h,
                                                              const double* __restrict__ w, const double* sm,
                                                              int inv_off, double* out, const int* stop) {
  if (stop && stop[F_STOP]) return;
  __shared__ double hs[NVMAX];
  for (int i = threadIdx.x; i < NVMAX; i += blockDim.x) hs[i] = i < nv ? h[i] : 0.0;
  __syncthreads();
  const double inv = sm[inv_off];
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    double v[NVMAX];
#pragma unroll
    for (int i = 0; i < NVMAX; ++i) v[i] = i < nv ? V[(size_t)i * n + idx] : 0.0;
    double wv = w[idx];
#pragma unroll
    for (int i = 0; i < NVMAX; ++i)
      if (i < nv) wv -= hs[i] * v[i];
    out[idx] = wv * inv;
  }
}

// Sum the per-block partials of nv dot products (stride nv + 1) in block order.
// mode 0: H column := s; mode 1: H column += s and the squared norm of the new
// vector is ||w'||^2 - ||s||^2 (the second projection removes s from w').
__global__ void cgs_reduce_kernel(const double* part, int G, int nv, double* Hcol, double* htmp, int mode,
                                  double* sm, int norm_off, const int* stop) {
  if (stop && stop[F_STOP]) return;
  __shared__ double sq[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int stride = nv + 1;
  const int cnt = mode ? nv + 1 : nv;
  double local_sq = 0.0;
  for (int i = wid; i < cnt; i += nw) {
    double s = 0.0;
    for (int b = lane; b < G; b += 32) s += part[(size_t)b * stride + i];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) {
      if (i < nv) {
        htmp[i] = s;
        Hcol[i] = mode ? Hcol[i] + s : s;
        local_sq += s * s;
      } else {
        sq[31] = s;   // ||w'||^2
      }
    }
  }
  if (!mode) return;
  if (lane == 0) sq[wid] = local_sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double hh = 0.0;
    for (int w2 = 0; w2 < nw; ++w2) hh += sq[w2];
    const double ww = sq[31];
    const double d = ww - hh;
    sm[norm_off] = d > 0.0 ? d : 0.0;
  }
}

// out = a * x + b * y; part[b] = block sum of out^2
__global__ void __launch_bounds__(KT) axpby_norm_kernel(double a, const double* x, double b, const double* y,
                                                        double* out, int64_t n, double* part) {
  __shared__ double red[KT / 32];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  double ss = 0.0;
  for (int64_t idx = lo + threadIdx.x; idx < hi; idx += blockDim.x) {
    const double v = a * x[idx] + (b != 0.0 ? b * y[idx] : 0.0);
    out[idx] = v;
    ss += v * v;
  }
  const double s = block_sum(ss, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__device__ double warp_sum_partials(const double* part, int G) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int b = lane; b < G; b += 32) s += part[b];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  return __shfl_sync(0xffffffffu, s, 0);
}

// start of a cycle: beta = ||r0||, g = beta e1
__global__ void cycle_init_kernel(double* sm, SmallLayout L, int* flags, const double* part, int G) {
  const double beta = sqrt(warp_sum_partials(part, G));
  if (threadIdx.x == 0) {
    sm[L.sc + 0] = beta;
    sm[L.sc + 4] = beta > 0.0 ? 1.0 / beta : 0.0;
    for (int i = 0; i <= L.K; ++i) sm[L.gv + i] = 0.0;
    sm[L.gv] = beta;
    flags[F_STOP] = beta > 0.0 ? 0 : 1;
    flags[F_JUSED] = 0;
  }
}

// norm of the new basis vector, Givens rotations, residual estimate
__global__ void givens_kernel(double* sm, SmallLayout L, int* flags, const double* part, int G, int j) {
  if (flags[F_STOP]) return;
  // squared norm of the new vector: from block partials, or precomputed in sm (part == nullptr)
  const double hn = sqrt(part ? warp_sum_partials(part, G) : sm[L.sc + 5]);
  if (threadIdx.x != 0) return;
  const int K1 = L.K + 1;
  double* h = sm + L.H + (size_t)j * K1;
  h[j + 1] = hn;
  for (int i = 0; i < j; ++i) {
    const double c = sm[L.cs + i], s = sm[L.sn + i];
    const double t = c * h[i] + s * h[i + 1];
    h[i + 1] = -s * h[i] + c * h[i + 1];
    h[i] = t;
  }
  const double a = h[j], b = h[j + 1];
  const double r = hypot(a, b);
  const double c = r > 0.0 ? a / r : 1.0, s = r > 0.0 ? b / r : 0.0;
  sm[L.cs + j] = c;
  sm[L.sn + j] = s;
  h[j] = r;
  h[j + 1] = 0.0;
  const double gj = sm[L.gv + j];
  sm[L.gv + j] = c * gj;
  sm[L.gv + j + 1] = -s * gj;
  const double est = fabs(sm[L.gv + j + 1]);
  sm[L.sc + 1] = est;
  sm[L.sc + 3] = hn;
  sm[L.sc + 4] = hn > 0.0 ? 1.0 / hn : 0.0;
  flags[F_JUSED] = j + 1;
  if (est <= sm[L.sc + 2] || hn == 0.0) flags[F_STOP] = 1;
}

// out = x * sm[sc + 4]
__global__ void __launch_bounds__(KT) scale_kernel(const double* x, const double* sm, int off, double* out,
                                                   int64_t n, const int* stop) {
  if (stop && stop[F_STOP]) return;
  const double f = sm[off];
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x)
    out[idx] = x[idx] * f;
}

// y = R^-1 g for the rotated Hessenberg matrix (jused columns)
__global__ void lsq_kernel(double* sm, SmallLayout L, const int* flags) {
  if (threadIdx.x != 0) return;
  const int k = flags[F_JUSED];
  const int K1 = L.K + 1;
  for (int i = k - 1; i >= 0; --i) {
    double s = sm[L.gv + i];
    for (int c = i + 1; c < k; ++c) s -= sm[L.H + (size_t)c * K1 + i] * sm[L.y + c];
    sm[L.y + i] = s / sm[L.H + (size_t)i * K1 + i];
  }
}

__global__ void sum_partials_kernel(const double* part, int G, double* out) {
  const double s = warp_sum_partials(part, G);
  if (threadIdx.x == 0) *out = s;
}

// pass 0: dots of w; pass 1: update w in place + dots + norm; pass 2: update + scale into out
template <int NV>
static void cgs_pass(int pass, const double* V, int64_t n, int nv, double* w, double* part, double* sm,
                     const SmallLayout& L, const int* fl, double* out, cudaStream_t st) {
  if (pass == 0) cgs_dot_kernel<NV><<<KG, KT, 0, st>>>(V, n, nv, w, part, fl);
  else if (pass == 1) cgs_update_dot_kernel<NV><<<KG, KT, 0, st>>>(V, n, nv, sm + L.htmp, w, part, fl);
  else cgs_update_scale_kernel<NV><<<KG, KT, 0, st>>>(V, n, nv, sm + L.htmp, w, sm, L.sc + 4, out, fl);
}

static cudaError_t launch_cgs(int nv, int pass, const double* V, int64_t n, double* w, double* part, double* sm,
                              const SmallLayout& L, double* Hcol, const int* fl, double* out, cudaStream_t st) {
  (void)Hcol;
  if (nv <= 8) cgs_pass<8>(pass, V, n, nv, w, part, sm, L, fl, out, st);
  else if (nv <= 16) cgs_pass<16>(pass, V, n, nv, w, part, sm, L, fl, out, st);
  else if (nv <= 32) cgs_pass<32>(pass, V, n, nv, w, part, sm, L, fl, out, st);
  else cgs_pass<64>(pass, V, n, nv, w, part, sm, L, fl, out, st);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ driver
namespace {
struct Cu {
  hdg_ctx* c;
  cudaError_t err = cudaSuccess;
  bool ok(cudaError_t e) {
    if (e != cudaSuccess && err == cudaSuccess) err = e;
    return e == cudaSuccess;
  }
};
}  // namespace

static hdg_status fail(hdg_ctx* c, hdg_status s, const std::string& msg) {
  c->err = msg;
  return s;
}

static cudaError_t ensure_krylov(hdg_ctx* c, int K) {
  if (c->krylov_restart == K && c->d_V) return cudaSuccess;
  cudaFree(c->d_V);
  cudaFree(c->d_part);
  cudaFree(c->d_small);
  cudaFree(c->d_flag);
  cudaFree(c->d_w);
  cudaFree(c->d_r);
  c->d_V = nullptr; c->d_part = nullptr; c->d_small = nullptr; c->d_flag = nullptr; c->d_w = nullptr; c->d_r = nullptr;
  c->krylov_restart = 0;
  const size_t n = (size_t)c->prm.N_tr;
  cudaError_t e;
  if ((e = cudaMalloc(&c->d_V, (size_t)(K + 1) * n * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->d_w, n * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->d_r, 3 * n * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->d_part, (size_t)KG * (K + 2) * sizeof(double))) != cudaSuccess) return e;
  SmallLayout L(K);
  if ((e = cudaMalloc(&c->d_small, (size_t)L.total * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->d_flag, 4 * sizeof(int))) != cudaSuccess) return e;
  c->krylov_restart = K;
  return cudaSuccess;
}

static double read_scalar(hdg_ctx* c, const double* p, Cu& cu) {
  double v = 0.0;
  cu.ok(cudaMemcpyAsync(&v, p, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  cu.ok(cudaStreamSynchronize(c->stream));
  return v;
}

#define LAUNCHED(k) (c->launches += (k))

namespace {

__global__ void __launch_bounds__(KT) axpy_kernel(double a, const double* __restrict__ xv, double* y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += a * xv[i];
}

// Restart cycles of left-preconditioned GMRES on one context.
struct Solver {
  hdg_ctx* c;
  const Params& P;
  int K;
  int64_t n;
  cudaStream_t st;
  Cu cu;
  SmallLayout L;
  double *sm, *V, *w, *part, *rr;
  int* fl;

  Solver(hdg_ctx* ctx, int k)
      : c(ctx), P(ctx->prm), K(k), n(ctx->prm.N_tr), st(ctx->stream), cu{ctx}, L(k), sm(ctx->d_small),
        V(ctx->d_V), w(ctx->d_w), part(ctx->d_part), rr(ctx->d_r + 2 * ctx->prm.N_tr), fl(ctx->d_flag) {}

  // ||v||^2 (synchronises)
  double norm2(const double* v) {
    axpby_norm_kernel<<<KG, KT, 0, st>>>(1.0, v, 0.0, v, rr, n, part);
    sum_partials_kernel<<<1, 32, 0, st>>>(part, KG, sm + L.sc + 5);
    LAUNCHED(2);
    return read_scalar(c, sm + L.sc + 5, cu);
  }

  // ||g - S x|| / gnorm with the FP64 S; leaves g - S x in rr
  double true_rel(const double* g, const double* x, double gnorm) {
    {
      ProfScope ps(c, HDG_PROF_APPLY);
      cu.ok(launch_apply64(P, c->d_S, x, w, nullptr, nullptr, st));
    }
    axpby_norm_kernel<<<KG, KT, 0, st>>>(1.0, g, -1.0, w, rr, n, part);
    sum_partials_kernel<<<1, 32, 0, st>>>(part, KG, sm + L.sc + 5);
    LAUNCHED(3);
    return std::sqrt(read_scalar(c, sm + L.sc + 5, cu)) / gnorm;
  }

  // One restart cycle for op(x) = bt (op = preconditioned operator, phase = its
  // profiling phase): at most jmax Arnoldi steps, early stop when the residual
  // estimate falls to target; x is updated. Returns the steps taken.
  template <class Op>
  int cycle(Op op, int phase, const double* bt, double* x, double target, int jmax, double& est) {
    double* r0 = w;   // op(x) lands in w, r0 in rr
    cu.ok(cudaMemcpyAsync(sm + L.sc + 2, &target, sizeof(double), cudaMemcpyHostToDevice, st));
    {
      ProfScope ps(c, phase);
      cu.ok(op(x, r0, nullptr));
    }
    axpby_norm_kernel<<<KG, KT, 0, st>>>(1.0, bt, -1.0, r0, rr, n, part);
    cycle_init_kernel<<<1, 32, 0, st>>>(sm, L, fl, part, KG);
    scale_kernel<<<KG, KT, 0, st>>>(rr, sm, L.sc + 4, V, n, fl);
    LAUNCHED(4);
    std::vector<size_t> mark(jmax + 1, 0);   // profiling entries recorded before Arnoldi step j
    for (int j = 0; j < jmax; ++j) {
      mark[j] = c->prof_ev.size();
      double* Vj = V + (size_t)j * n;
      double* Hcol = sm + L.H + (size_t)j * (K + 1);
      {
        ProfScope ps(c, phase);
        cu.ok(op(Vj, w, fl));
      }
      ProfScope po(c, HDG_PROF_ORTHO);
      const int nv = j + 1;
      if (nv <= 64) {
        // CGS2 in three passes over the basis: dots, update + second dots + norm, update + scale
        cu.ok(launch_cgs(nv, 0, V, n, w, part, sm, L, Hcol, fl, V + (size_t)(j + 1) * n, st));
        cgs_reduce_kernel<<<1, 256, 0, st>>>(part, KG, nv, Hcol, sm + L.htmp, 0, sm, L.sc + 5, fl);
        cu.ok(launch_cgs(nv, 1, V, n, w, part, sm, L, Hcol, fl, V + (size_t)(j + 1) * n, st));
        cgs_reduce_kernel<<<1, 256, 0, st>>>(part, KG, nv, Hcol, sm + L.htmp, 1, sm, L.sc + 5, fl);
        givens_kernel<<<1, 32, 0, st>>>(sm, L, fl, nullptr, 0, j);
        cu.ok(launch_cgs(nv, 2, V, n, w, part, sm, L, Hcol, fl, V + (size_t)(j + 1) * n, st));
        LAUNCHED(6);
      } else {
        mdot_kernel<<<KG, KT, 0, st>>>(V, n, nv, w, part, fl);
        mdot_reduce_kernel<<<1, 256, 0, st>>>(part, KG, nv, Hcol, sm + L.htmp, 0, fl);
        update_kernel<<<KG, KT, 0, st>>>(V, n, nv, sm + L.htmp, -1.0, w, nullptr, fl);
        mdot_kernel<<<KG, KT, 0, st>>>(V, n, nv, w, part, fl);
        mdot_reduce_kernel<<<1, 256, 0, st>>>(part, KG, nv, Hcol, sm + L.htmp, 1, fl);
        update_kernel<<<KG, KT, 0, st>>>(V, n, nv, sm + L.htmp, -1.0, w, part, fl);
        givens_kernel<<<1, 32, 0, st>>>(sm, L, fl, part, KG, j);
        scale_kernel<<<KG, KT, 0, st>>>(w, sm, L.sc + 4, V + (size_t)(j + 1) * n, n, fl);
        LAUNCHED(9);
      }
    }
    cu.ok(cudaGetLastError());
    int hflags[2] = {0, 0};
    cu.ok(cudaMemcpyAsync(hflags, fl, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    cu.ok(cudaStreamSynchronize(st));
    const int jused = hflags[F_JUSED];
    if (c->prof_on && jused < jmax) {
      // steps after the stop flag was raised were enqueued but returned at once: not timed work
      for (size_t i = mark[jused]; i < c->prof_ev.size(); ++i) c->prof_pool.push_back(c->prof_ev[i].second);
      c->prof_ev.resize(mark[jused]);
    }
    est = read_scalar(c, sm + L.sc + 1, cu);
    if (jused > 0) {
      lsq_kernel<<<1, 32, 0, st>>>(sm, L, fl);
      update_kernel<<<KG, KT, 0, st>>>(V, n, jused, sm + L.y, 1.0, x, nullptr, nullptr);
      LAUNCHED(2);
    }
    return jused;
  }
};

}  // namespace

// FP32 + iterative refinement: inner GMRES on the FP32 blocks reduces the
// preconditioned correction residual by this factor per outer sweep.
constexpr double IR_INNER_REDUCTION = 1e-4;

hdg_status gmres_solve(hdg_ctx* c, const double* g, double* x, const hdg_solve_opts& o, hdg_solve_report& rep) {
  const Params& P = c->prm;
  const int K = o.restart;
  const int64_t n = P.N_tr;
  cudaStream_t st = c->stream;
  Cu cu{c};
  if (!cu.ok(ensure_krylov(c, K))) return fail(c, HDG_ERR_OOM, std::string("Krylov workspace: ") + cudaGetErrorString(cu.err));
  Solver S(c, K);
  double* bt = c->d_r;          // preconditioned right-hand side
  double* d = c->d_r + n;       // IR correction
  rep = hdg_solve_report{};
  auto op64 = [&](const double* xin, double* yout, const int* stop) -> cudaError_t {
    return launch_apply64(P, c->d_St, xin, yout, c->d_escale, stop, st);
  };
  auto opdf = [&](const double* xin, double* yout, const int* stop) -> cudaError_t {
    return launch_apply_df(P, c->d_Stdf, xin, yout, c->d_escale, stop, st);
  };
  auto op32 = [&](const double* xin, double* yout, const int* stop) -> cudaError_t {
    return launch_apply32x64(P, c->d_St32, xin, yout, c->d_escale, stop, st);
  };

  const double gnorm = std::sqrt(S.norm2(g));
  if (S.cu.err != cudaSuccess) return fail(c, HDG_ERR_CUDA, cudaGetErrorString(S.cu.err));
  if (gnorm == 0.0) {
    cu.ok(cudaMemsetAsync(x, 0, n * sizeof(double), st));
    cu.ok(cudaStreamSynchronize(st));
    rep.converged = 1;
    return cu.err == cudaSuccess ? HDG_OK : fail(c, HDG_ERR_CUDA, cudaGetErrorString(cu.err));
  }
  int its = 0;
  double rel = 1.0;
  if (o.mode == 0 || o.mode == 2) {
    cu.ok(launch_face_dinv(P, c->dt.Ghinv, c->d_escale, g, bt, st));
    LAUNCHED(1);
    const double btnorm = std::sqrt(S.norm2(bt));
    double target = o.tol * btnorm;
    while (true) {
      double est = 0.0;
      const int jmax = std::min(K, o.maxit - its);
      const int jused = o.mode == 2 ? S.cycle(opdf, HDG_PROF_APPLY, bt, x, target, jmax, est)
                                    : S.cycle(op64, HDG_PROF_APPLY, bt, x, target, jmax, est);
      its += jused;
      rep.restarts += 1;
      rel = S.true_rel(g, x, gnorm);
      if (S.cu.err != cudaSuccess || cu.err != cudaSuccess)
        return fail(c, HDG_ERR_CUDA, cudaGetErrorString(S.cu.err != cudaSuccess ? S.cu.err : cu.err));
      rep.iterations = its;
      rep.rel_residual = rel;
      if (rel <= o.tol) {
        rep.converged = 1;
        return HDG_OK;
      }
      if (its >= o.maxit || jused == 0) break;
      if (est <= target) target *= 0.5 * o.tol / rel;
    }
  } else {
    // FP32 + iterative refinement: r = g - S x in FP64; D^-1 S32 d = D^-1 r
    // by GMRES on the FP32 blocks; x += d.
    while (true) {
      rel = S.true_rel(g, x, gnorm);           // leaves r in S.rr
      if (S.cu.err != cudaSuccess) return fail(c, HDG_ERR_CUDA, cudaGetErrorString(S.cu.err));
      rep.rel_residual = rel;
      rep.iterations = its;
      if (rel <= o.tol) {
        rep.converged = 1;
        return HDG_OK;
      }
      if (its >= o.maxit) break;
      rep.outer += 1;
      cu.ok(launch_face_dinv(P, c->dt.Ghinv, c->d_escale, S.rr, bt, st));
      cu.ok(cudaMemsetAsync(d, 0, n * sizeof(double), st));
      LAUNCHED(1);
      const double btnorm = std::sqrt(S.norm2(bt));
      const double target = IR_INNER_REDUCTION * btnorm;
      double est = btnorm;
      while (est > target && its < o.maxit) {
        const int jused = S.cycle(op32, HDG_PROF_APPLY32, bt, d, target, std::min(K, o.maxit - its), est);
        its += jused;
        rep.restarts += 1;
        if (jused == 0) break;
      }
      axpy_kernel<<<KG, KT, 0, st>>>(1.0, d, x, n);
      LAUNCHED(1);
    }
  }
  rep.converged = 0;
  return fail(c, HDG_ERR_NOCONV, "GMRES reached maxit with relative residual " + std::to_string(rel));
}

}  // namespace mehdg
