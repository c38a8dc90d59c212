// Restarted GMRES for the condensed trace system S x = g (Eq. global_problem),
// left-preconditioned by D^-1 (Sec. 6.1): the Krylov space is built for
// D^-1 S with right-hand side D^-1 g.
//
// The paper uses PETSc GMRES and fixes neither restart length,
// orthogonalisation nor stopping rule. Here:
//  * every restart cycle starts from the TRUE residual t = g - S x computed
//    with the FP64 Schur blocks; ||t|| / ||g|| <= tol is the stopping test, and
//    r0 = D^-1 t starts the Arnoldi process (residual replacement: with a
//    lower-precision Arnoldi operator this is iterative refinement in FP64);
//  * the Arnoldi operator D^-1 S is applied from FP64 blocks (mode 0, FP64
//    arithmetic), FP32 blocks (mode 1) or split-FP32 blocks (mode 2);
//  * the Krylov basis is stored and orthogonalised in split-FP32 arithmetic
//    on the FP32 pipe, because FP64 vector arithmetic runs at 2 lanes/clock/SM
//    on GB300: classical Gram-Schmidt applied twice (CGS2, four passes over
//    the basis), once with the norm from Pythagoras (two passes), or once with
//    a second projection only in the steps where more than half of the new
//    vector lay in the basis (Kahan-Parlett; decided on the device);
//  * Givens rotations run on the device and a device stop flag lets a whole
//    cycle be enqueued without host round trips (every kernel of the cycle
//    returns at once when the flag is set);
//  * all reductions have a fixed order: results are bitwise reproducible.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>
#include <type_traits>
#include "df64.h"
#include "launch.h"

namespace mehdg {

constexpr int KG = 304;       // blocks (partial sums) of the vector kernels, 2 per SM
constexpr int KT = 256;       // threads per block
constexpr int VG = 8;         // basis vectors per pass of the multi-dot

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
    sc = htmp + K + 1;   // scalars: 0 beta, 1 est, 2 target, 3 hn, 4 inv, 5 scratch
    total = sc + 8;
  }
};
// F_P2 = 1: the Arnoldi step needs no second Gram-Schmidt pass, or the instance has stopped (kept
// 1 whenever F_STOP is set, so that the second-pass kernels can use it as their stop flag)
enum { F_STOP = 0, F_JUSED = 1, F_CNT = 2, F_P2 = 3 };   // F_CNT: arrivals in reduce2_givens_kernel

// Strides of a batch of independent GMRES instances (several right-hand
// sides, blockIdx.z / .y / .x selecting the instance r): offsets per r of the
// basis, the work vector, the partial sums, the small arrays and the flags;
// vstr separates consecutive basis vectors of one instance. One instance:
// vstr = pairs per vector, every offset 0.
struct Batch {
  int64_t vstr, rv, rw, rpart, rsm;
  int rflag;
};
constexpr int KGU = 1216;     // blocks of the streaming update kernel, 8 per SM
constexpr int KGD = 1216;     // blocks (over all vector groups) of the multi-dot, 8 per SM
constexpr int KGD_MAX = 2432; // largest multi-dot block count the autotuner tries

// ------------------------------------------------------------ FP64 helpers
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

// out = a * x + b * y (FP64); part[b] = block sum of out^2
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

__global__ void sum_partials_kernel(const double* part, int G, double* out) {
  const double s = warp_sum_partials(part, G);
  if (threadIdx.x == 0) *out = s;
}

// ------------------------------------------------- split-FP32 vector kernels
// Block reduction of per-thread (h, l) partials of NV values, to FP64 out[0..nv).
template <int NV>
__device__ __forceinline__ void df_block_reduce(float (&h)[NV], float (&l)[NV], int nv, float2* red, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int g = 0; g < NV; ++g) {
    df_warp_sum(h[g], l[g]);
    if (lane == 0) red[wid * NV + g] = make_float2(h[g], l[g]);
  }
  __syncthreads();
  if ((int)threadIdx.x < NV && (int)threadIdx.x < nv) {
    double s = 0.0;
    for (int w2 = 0; w2 < nw; ++w2) s += df_to(red[w2 * NV + threadIdx.x]);
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// Basis rows have an even leading dimension ldv (zero padding), so the
// vector kernels below move element PAIRS with 16-byte loads: (x, y) is the
// first split-FP32 entry of a float4, (z, w) the second.
__device__ __forceinline__ void df_fma4(float& h, float& l, float4 a, float4 b) {
  df_fma(h, l, make_float2(a.x, a.y), make_float2(b.x, b.y));
  df_fma(h, l, make_float2(a.z, a.w), make_float2(b.z, b.w));
}

// part[b * ncol + i] = sum over pair chunk b of V_i . w, for gridDim.x chunks
// and gridDim.y groups of VG basis vectors. ncol = nv, or nv + 1 to append the
// squared norm w . w as column nv. One pair per thread per iteration; four
// blocks per SM. Blocks are numbered group-fastest (block k: chunk k / gy,
// group k % gy), so blocks dispatched together read all vectors of the same
// rows and the last rows of the basis are what the L2 holds when the update
// (which walks the rows backwards) starts. The sums do not depend on this.
__global__ void __launch_bounds__(KT, 4) df_mdot_kernel(const float4* __restrict__ V, int64_t np, int nv, int ncol,
                                                        const float4* __restrict__ w, double* part, const int* stop,
                                                        Batch bt) {
  const int rb = blockIdx.z;
  if (stop && stop[rb * bt.rflag + F_STOP]) return;
  V += rb * bt.rv;
  w += rb * bt.rw;
  part += rb * bt.rpart;
  __shared__ float2 red[(KT / 32) * VG];
  const unsigned k = blockIdx.y * gridDim.x + blockIdx.x;
  const int64_t cb = k / gridDim.y;
  const int g0 = (int)(k % gridDim.y) * VG;
  const int64_t chunk = (np + gridDim.x - 1) / gridDim.x;
  const int64_t lo = cb * chunk;
  const int64_t hi = lo + chunk < np ? lo + chunk : np;
  float h[VG], l[VG];
#pragma unroll
  for (int g = 0; g < VG; ++g) { h[g] = 0.f; l[g] = 0.f; }
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t p = lo + threadIdx.x; p < hi; p += blockDim.x) {
    float4 a[VG];
    const float4 wa = w[p];
#pragma unroll
    for (int g = 0; g < VG; ++g) a[g] = g0 + g < nv ? V[(size_t)(g0 + g) * bt.vstr + p] : (g0 + g < ncol ? wa : z4);
#pragma unroll
    for (int g = 0; g < VG; ++g) df_fma4(h[g], l[g], a[g], wa);
  }
  df_block_reduce<VG>(h, l, ncol - g0, red, part + (size_t)cb * ncol + g0);
}

// Sums the partials of one Arnoldi step (stride nv + 1: columns 0..nv-1 the
// projections, column nv the squared norm of the vector they were taken of)
// in block order; add = 1 adds them to the Hessenberg column (second
// projection of CGS2), add = 0 sets it (single projection). The new vector's
// norm follows from ||x - V s||^2 = ||x||^2 - ||s||^2 (orthonormal V). Then
// the Givens rotations. One block.
// add: 0 first (only) pass, 1 second pass (H += h), 2 first pass that decides
// whether a second pass is needed (Kahan-Parlett: ||w - V h||^2 < ||w||^2 / 2,
// i.e. more than half of w lay in the basis and the Pythagorean norm has lost
// digits): then it stores h, clears F_P2 and leaves the rotations to the second
// pass; 3 as 2 with the threshold 1e-6 ||w||^2. stopslot: the flag that makes
// the launch return at once.
// Grid (column groups, instances), 1024 threads: block k sums columns
// 32 k .. 32 k + 31 of the partial rows (warp w the rows w, w + 32, ..., then
// the 32 warps' sums in order) into sm[htmp + col]; the last block of an
// instance to arrive (arrival counter F_CNT, no waiting) reads all sums and
// applies the rotations. The order of every sum does not depend on the grid.
__global__ void __launch_bounds__(1024) reduce2_givens_kernel(const double* part, int G, int nv, double* sm,
                                                               SmallLayout L, int* flags, int j, int add, Batch bt,
                                                               int stopslot) {
  const int rb = blockIdx.y;
  part += rb * bt.rpart;
  sm += rb * bt.rsm;
  flags += rb * bt.rflag;
  if (flags[stopslot]) return;
  __shared__ double vals[136];
  __shared__ double red[32];
  __shared__ double wsum[32][33];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ncol = nv + 1;
  {
    const int col = blockIdx.x * 32 + lane;
    double acc = 0.0;
    if (col < ncol)
      for (int b = wid; b < G; b += nw) acc += part[(size_t)b * ncol + col];
    wsum[wid][lane] = acc;
    __syncthreads();
    if (threadIdx.x < 32 && blockIdx.x * 32 + threadIdx.x < ncol) {
      double t = 0.0;
      for (int w2 = 0; w2 < nw; ++w2) t += wsum[w2][threadIdx.x];
      sm[L.htmp + blockIdx.x * 32 + threadIdx.x] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&flags[F_CNT], 1) == (int)gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int i = threadIdx.x; i < ncol; i += blockDim.x) vals[i] = __ldcg(&sm[L.htmp + i]);
    if (threadIdx.x == 0) flags[F_CNT] = 0;
  }
  __syncthreads();
  const int K1 = L.K + 1;
  double* h = sm + L.H + (size_t)j * K1;
  double q2 = 0.0;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    const double s = vals[i];
    sm[L.htmp + i] = s;
    h[i] = add == 1 ? h[i] + s : s;
    q2 += s * s;
  }
  for (int off = 16; off > 0; off >>= 1) q2 += __shfl_down_sync(0xffffffffu, q2, off);
  if (lane == 0) red[wid] = q2;
  __syncthreads();
  // stage the column and the previous rotations: the rotations are a serial chain
  __shared__ double hs[136], cs_s[136], sn_s[136];
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    hs[i] = h[i];
    cs_s[i] = i < j ? sm[L.cs + i] : 0.0;
    sn_s[i] = i < j ? sm[L.sn + i] : 0.0;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double hh = 0.0;
  for (int i = 0; i < nw; ++i) hh += red[i];
  const double d = vals[nv] - hh;
  if (add >= 2) {
    // add = 2: Kahan-Parlett threshold 1/2; add = 3: only where the single projection cancelled
    // more than six decimal digits of ||w||^2 (the new vector then loses orthogonality to
    // about eps / 1e-3 = 1e-13 in FP64, harmless for GMRES, whose restarts use the true residual)
    const double eta = add == 2 ? 0.5 : 1e-6;
    if (!(d >= eta * vals[nv])) {   // second pass needed (also for a non-finite estimate)
      flags[F_P2] = 0;
      return;
    }
    flags[F_P2] = 1;
  }
  const double hn = d > 0.0 ? sqrt(d) : 0.0;
  hs[j + 1] = hn;
  // previous rotations: the running entry stays in a register
  double x = hs[0];
  for (int i = 0; i < j; ++i) {
    const double c = cs_s[i], s = sn_s[i], y = hs[i + 1];
    h[i] = c * x + s * y;
    x = -s * x + c * y;
  }
  const double a = x, b = hn;
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
  flags[F_P2] = 1;
  if (est <= sm[L.sc + 2] || hn == 0.0) flags[F_STOP] = 1;
}

// out = (w - sum_i coef_i V_i) * scale over element pairs, scale = sm[scale_off]
// (or 1 when scale_off < 0); out may be w itself. The loads of the next group
// of 8 basis vectors are issued before the products of the current group.
// Instances and pairs are walked last to first: the multi-dot before it read
// them first to last, so its most recent lines are still in L2.
__global__ void __launch_bounds__(KT) df_update_kernel(const float4* __restrict__ V, int64_t np, int nv,
                                                       const double* __restrict__ coef, const float4* w,
                                                       const double* sm, int scale_off, float4* out,
                                                       const int* stop, Batch bt, int64_t rout) {
  const int rb = gridDim.y - 1 - blockIdx.y;
  if (stop && stop[rb * bt.rflag + F_STOP]) return;
  V += rb * bt.rv;
  coef += rb * bt.rsm;
  w += rb * bt.rw;
  if (sm) sm += rb * bt.rsm;
  out += rb * rout;
  __shared__ float2 cf[144];
  for (int i = threadIdx.x; i < 144; i += blockDim.x) cf[i] = i < nv ? df_from(-coef[i]) : make_float2(0.f, 0.f);
  __syncthreads();
  const bool scaled = scale_off >= 0;
  const float2 inv = scaled ? df_from(sm[scale_off]) : make_float2(1.f, 0.f);
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t pf = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pf < np; pf += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = np - 1 - pf;
    const float4 wv = w[p];
    float ah = wv.x, al = wv.y, bh = wv.z, bl = wv.w;
    float4 v[8], nx[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = u < nv ? V[(size_t)u * bt.vstr + p] : z4;
    for (int i0 = 0; i0 < nv; i0 += 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u) nx[u] = i0 + 8 + u < nv ? V[(size_t)(i0 + 8 + u) * bt.vstr + p] : z4;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        df_fma(ah, al, cf[i0 + u], make_float2(v[u].x, v[u].y));
        df_fma(bh, bl, cf[i0 + u], make_float2(v[u].z, v[u].w));
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = nx[u];
    }
    float2 ra = df_norm(ah, al), rb = df_norm(bh, bl);
    if (scaled) {
      float sah = 0.f, sal = 0.f, sbh = 0.f, sbl = 0.f;
      df_fma(sah, sal, ra, inv);
      df_fma(sbh, sbl, rb, inv);
      ra = df_norm(sah, sal);
      rb = df_norm(sbh, sbl);
    }
    out[p] = make_float4(ra.x, ra.y, rb.x, rb.y);
  }
}

// out = split(a * sm[off]) for an FP64 vector a
__global__ void __launch_bounds__(KT) to_df_kernel(const double* a, const double* sm, int off, float2* out,
                                                   int64_t n, const int* stop) {
  if (stop && stop[F_STOP]) return;
  const double f = sm[off];
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x)
    out[idx] = df_from(a[idx] * f);
}

// x += sum_i y_i V_i (x in FP64; the sum in split FP32; basis row length ldv)
__global__ void __launch_bounds__(KT) df_xupdate_kernel(const float2* __restrict__ V, int64_t n, int64_t ldv, int nv,
                                                        const double* __restrict__ y, double* x) {
  __shared__ float2 cf[130];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) cf[i] = df_from(y[i]);
  __syncthreads();
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    float ah = 0.f, al = 0.f;
    for (int i = 0; i < nv; ++i) df_fma(ah, al, cf[i], V[(size_t)i * ldv + idx]);
    x[idx] += df_to(make_float2(ah, al));
  }
}

// ------------------------------------------------------ FP64 vector kernels
// The FP64 Krylov basis (HDG_BASIS_FP64): the same passes as the split-FP32
// kernels above, on FP64 entries with FP64 fused multiply-adds; rows have the
// same even length, so a thread moves an element pair with one 16-byte load.
// On GB300 these are bound by the FP64 pipe (one FMA per 8-byte basis entry
// against 2 FMA/clock/SM), not by HBM.
template <int NV>
__device__ __forceinline__ void d_block_reduce(double (&h)[NV], int nv, double* red, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int g = 0; g < NV; ++g) {
    double v = h[g];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[wid * NV + g] = v;
  }
  __syncthreads();
  if ((int)threadIdx.x < NV && (int)threadIdx.x < nv) {
    double s = 0.0;
    for (int w2 = 0; w2 < nw; ++w2) s += red[w2 * NV + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// Products of NG basis vectors with w over the pairs [lo, hi) (FP64 FMAs; NG is
// the number of columns the block really has, so a partial last group costs
// only its own FMAs: these passes are bound by the FP64 pipe).
template <int NG>
__device__ __forceinline__ void d_mdot_body(const double2* __restrict__ V, int64_t vstr, int g0, int nv,
                                            const double2* __restrict__ w, int64_t lo, int64_t hi, double (&h)[VG]) {
  for (int64_t p = lo + threadIdx.x; p < hi; p += blockDim.x) {
    double2 a[NG];
    const double2 wa = w[p];
#pragma unroll
    for (int g = 0; g < NG; ++g) a[g] = g0 + g < nv ? V[(size_t)(g0 + g) * vstr + p] : wa;
#pragma unroll
    for (int g = 0; g < NG; ++g) h[g] = fma(a[g].y, wa.y, fma(a[g].x, wa.x, h[g]));
  }
}

// part[b * ncol + i] = sum over pair chunk b of V_i . w (FP64); block
// numbering, columns and stop flags as in df_mdot_kernel.
__global__ void __launch_bounds__(KT, 4) d_mdot_kernel(const double2* __restrict__ V, int64_t np, int nv, int ncol,
                                                       const double2* __restrict__ w, double* part, const int* stop,
                                                       Batch bt) {
  const int rb = blockIdx.z;
  if (stop && stop[rb * bt.rflag + F_STOP]) return;
  V += rb * bt.rv;
  w += rb * bt.rw;
  part += rb * bt.rpart;
  __shared__ double red[(KT / 32) * VG];
  const unsigned k = blockIdx.y * gridDim.x + blockIdx.x;
  const int64_t cb = k / gridDim.y;
  const int g0 = (int)(k % gridDim.y) * VG;
  const int64_t chunk = (np + gridDim.x - 1) / gridDim.x;
  const int64_t lo = cb * chunk;
  const int64_t hi = lo + chunk < np ? lo + chunk : np;
  double h[VG];
#pragma unroll
  for (int g = 0; g < VG; ++g) h[g] = 0.0;
  switch (ncol - g0 < VG ? ncol - g0 : VG) {   // uniform over the block
    case 1: d_mdot_body<1>(V, bt.vstr, g0, nv, w, lo, hi, h); break;
    case 2: d_mdot_body<2>(V, bt.vstr, g0, nv, w, lo, hi, h); break;
    case 3: d_mdot_body<3>(V, bt.vstr, g0, nv, w, lo, hi, h); break;
    case 4: d_mdot_body<4>(V, bt.vstr, g0, nv, w, lo, hi, h); break;
    case 5: d_mdot_body<5>(V, bt.vstr, g0, nv, w, lo, hi, h); break;
    case 6: d_mdot_body<6>(V, bt.vstr, g0, nv, w, lo, hi, h); break;
    case 7: d_mdot_body<7>(V, bt.vstr, g0, nv, w, lo, hi, h); break;
    default: d_mdot_body<VG>(V, bt.vstr, g0, nv, w, lo, hi, h); break;
  }
  d_block_reduce<VG>(h, ncol - g0, red, part + (size_t)cb * ncol + g0);
}

// the last R (< 4) columns of an update: a -= sum cf_u v_u.x, b likewise
template <int R>
__device__ __forceinline__ void d_update_tail(double& a, double& b, const double* cf, const double2 (&v)[4]) {
#pragma unroll
  for (int u = 0; u < R; ++u) {
    a = fma(cf[u], v[u].x, a);
    b = fma(cf[u], v[u].y, b);
  }
}

// out = (w - sum_i coef_i V_i) * scale in FP64 (scale = sm[scale_off], or 1
// when scale_off < 0); out may be w. Loads of the next group of 8 basis
// vectors go out before the FMAs of the current one; rows walked last to
// first (the multi-dot's most recent rows are still in L2).
__global__ void __launch_bounds__(KT) d_update_kernel(const double2* __restrict__ V, int64_t np, int nv,
                                                      const double* __restrict__ coef, const double2* w,
                                                      const double* sm, int scale_off, double2* out,
                                                      const int* stop, Batch bt, int64_t rout) {
  const int rb = gridDim.y - 1 - blockIdx.y;
  if (stop && stop[rb * bt.rflag + F_STOP]) return;
  V += rb * bt.rv;
  coef += rb * bt.rsm;
  w += rb * bt.rw;
  if (sm) sm += rb * bt.rsm;
  out += rb * rout;
  __shared__ double cf[144];
  for (int i = threadIdx.x; i < 144; i += blockDim.x) cf[i] = i < nv ? -coef[i] : 0.0;
  __syncthreads();
  const bool scaled = scale_off >= 0;
  const double inv = scaled ? sm[scale_off] : 1.0;
  const double2 z2 = make_double2(0.0, 0.0);
  for (int64_t pf = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pf < np; pf += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = np - 1 - pf;
    const double2 wv = w[p];
    // two chains per entry (even and odd basis vectors): four DFMA chains per thread;
    // groups of 4 basis vectors, the next group's loads issued before this group's FMAs
    double a = wv.x, b = wv.y, a1 = 0.0, b1 = 0.0;
    double2 v[4], nx[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = u < nv ? V[(size_t)u * bt.vstr + p] : z2;
    int i0 = 0;
    for (; i0 + 4 <= nv; i0 += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) nx[u] = i0 + 4 + u < nv ? V[(size_t)(i0 + 4 + u) * bt.vstr + p] : z2;
#pragma unroll
      for (int u = 0; u < 4; u += 2) {
        a = fma(cf[i0 + u], v[u].x, a);
        b = fma(cf[i0 + u], v[u].y, b);
        a1 = fma(cf[i0 + u + 1], v[u + 1].x, a1);
        b1 = fma(cf[i0 + u + 1], v[u + 1].y, b1);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = nx[u];
    }
    switch (nv - i0) {   // the partial last group: only its own FMAs
      case 1: d_update_tail<1>(a, b, cf + i0, v); break;
      case 2: d_update_tail<2>(a, b, cf + i0, v); break;
      case 3: d_update_tail<3>(a, b, cf + i0, v); break;
      default: break;
    }
    a += a1;
    b += b1;
    if (scaled) {
      a *= inv;
      b *= inv;
    }
    out[p] = make_double2(a, b);
  }
}

// out = a * sm[off] (FP64 basis: the first vector of a cycle)
__global__ void __launch_bounds__(KT) to_d_kernel(const double* a, const double* sm, int off, double* out, int64_t n,
                                                  const int* stop) {
  if (stop && stop[F_STOP]) return;
  const double f = sm[off];
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x)
    out[idx] = a[idx] * f;
}

// x += sum_i y_i V_i (FP64 basis, row length ldv)
__global__ void __launch_bounds__(KT) d_xupdate_kernel(const double* __restrict__ V, int64_t n, int64_t ldv, int nv,
                                                       const double* __restrict__ y, double* x) {
  __shared__ double cf[130];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) cf[i] = y[i];
  __syncthreads();
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int i = 0; i < nv; ++i) a = fma(cf[i], V[(size_t)i * ldv + idx], a);
    x[idx] += a;
  }
}

// Fixed-order block sum (all threads get the result).
__device__ __forceinline__ double block_sum_all(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];
  __syncthreads();
  return s;
}

// ------------------------------------------------------- augmented restarts
// LGMRES (Baker, Jessup and Manteuffel, 2005): the last steps of a restart
// cycle take the normalised corrections of the previous cycles, z_i, as their
// operator inputs instead of new Krylov vectors (flexible Arnoldi: the images
// A z_i are orthogonalised into the same basis V), so the cycle's search space
// is span(V_0..V_{m-1}) + span(z_0..z_{nz-1}) and the correction is
// c = sum_{i<nv} y_i V_i + sum_{i<nzu} y_{m+i} z_i. x += c; c is kept in r0 and
// its squared norm's block partials in part, for the next z.
template <typename T>
__device__ __forceinline__ double basis_entry(const T* V, size_t i);
template <>
__device__ __forceinline__ double basis_entry<double>(const double* V, size_t i) { return V[i]; }
template <>
__device__ __forceinline__ double basis_entry<float2>(const float2* V, size_t i) { return df_to(V[i]); }

template <typename T>
__global__ void __launch_bounds__(KT) aug_correction_kernel(const T* __restrict__ V, const T* __restrict__ Z,
                                                            int64_t n, int64_t vstr, int nv, int nzu, int m,
                                                            const double* __restrict__ y, double* x, double* c,
                                                            double* part) {
  __shared__ double cf[136];
  __shared__ double red[KT / 32];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) cf[i] = y[i];
  for (int i = threadIdx.x; i < nzu; i += blockDim.x) cf[nv + i] = y[m + i];
  __syncthreads();
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  double ss = 0.0;
  for (int64_t idx = lo + threadIdx.x; idx < hi; idx += blockDim.x) {
    double a = 0.0;
    for (int i = 0; i < nv; ++i) a = fma(cf[i], basis_entry(V, (size_t)i * vstr + idx), a);
    for (int i = 0; i < nzu; ++i) a = fma(cf[nv + i], basis_entry(Z, (size_t)i * vstr + idx), a);
    c[idx] = a;
    x[idx] += a;
    ss = fma(a, a, ss);
  }
  const double s = block_sum(ss, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// z = c / ||c|| in the basis format (||c||^2 summed from G partials in block order);
// a zero correction leaves z = 0
template <typename T>
__global__ void __launch_bounds__(KT) aug_store_kernel(const double* __restrict__ c, const double* __restrict__ part,
                                                       int G, T* z, int64_t n) {
  __shared__ double red[KT / 32];
  __shared__ double s_inv;
  double s0 = 0.0;
  for (int b = threadIdx.x; b < G; b += blockDim.x) s0 += part[b];
  const double nrm2 = block_sum_all(s0, red);
  if (threadIdx.x == 0) s_inv = nrm2 > 0.0 ? 1.0 / sqrt(nrm2) : 0.0;
  __syncthreads();
  const double inv = s_inv;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const double v = c[idx] * inv;
    if constexpr (std::is_same<T, double>::value) z[idx] = v;
    else z[idx] = df_from(v);
  }
}


// out[i] = sum_b part[b * nv + i] in block order (block i sums vector i);
// mode 0: H column := s, mode 1: H column += s; htmp receives s.
// Column i = nv of a ncol = nv + 1 layout is ||w||^2 and goes to *wnorm2.
__global__ void mdot_reduce_kernel(const double* part, int G, int nv, int ncol, double* Hcol, double* htmp, int mode,
                                   const int* stop, double* wnorm2) {
  if (stop && stop[F_STOP]) return;
  __shared__ double red[32];
  const int i = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < G; b += blockDim.x) s += part[(size_t)b * ncol + i];
  s = block_sum_all(s, red);
  if (threadIdx.x == 0) {
    if (i == nv) {
      *wnorm2 = s;
    } else {
      htmp[i] = s;
      Hcol[i] = mode ? Hcol[i] + s : s;
    }
  }
}

// start of a cycle: beta = ||r0||, g = beta e1, inv = 1/beta; the target held
// in sm[sc + 2] as a reduction factor becomes an absolute target factor * beta
__global__ void cycle_init_kernel(double* sm, SmallLayout L, int* flags, const double* part, int G) {
  __shared__ double red[32];
  double s0 = 0.0;
  for (int b = threadIdx.x; b < G; b += blockDim.x) s0 += part[b];
  const double beta = sqrt(block_sum_all(s0, red));
  if (threadIdx.x == 0) {
    sm[L.sc + 0] = beta;
    sm[L.sc + 1] = beta;
    sm[L.sc + 4] = beta > 0.0 ? 1.0 / beta : 0.0;
    sm[L.sc + 2] *= beta;
    for (int i = 0; i <= L.K; ++i) sm[L.gv + i] = 0.0;
    sm[L.gv] = beta;
    flags[F_STOP] = beta > 0.0 ? 0 : 1;
    flags[F_JUSED] = 0;
    flags[F_CNT] = 0;
    flags[F_P2] = 1;
  }
}

// y = R^-1 g for the rotated Hessenberg matrix (jused columns), one warp:
// rows from the bottom, each row's sum over the solved entries across lanes
__global__ void lsq_kernel(double* sm, SmallLayout L, const int* flags) {
  const int lane = threadIdx.x & 31;
  if (threadIdx.x >= 32) return;
  const int k = flags[F_JUSED];
  const int K1 = L.K + 1;
  for (int i = k - 1; i >= 0; --i) {
    double s = 0.0;
    for (int c = i + 1 + lane; c < k; c += 32) s += sm[L.H + (size_t)c * K1 + i] * sm[L.y + c];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) sm[L.y + i] = (sm[L.gv + i] - s) / sm[L.H + (size_t)i * K1 + i];
    __syncwarp();
  }
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
  cudaFree(c->d_aug);
  cudaFree(c->d_Vs);
  cudaFree(c->d_vin);
  c->d_V = nullptr; c->d_part = nullptr; c->d_small = nullptr; c->d_flag = nullptr; c->d_w = nullptr; c->d_r = nullptr;
  c->d_aug = nullptr; c->d_Vs = nullptr; c->d_vin = nullptr;
  c->krylov_restart = 0;
  const size_t n = (size_t)c->prm.N_tr;
  const size_t ldv = n + (n & 1);   // even row length: 16-byte element pairs, zero padding
  cudaError_t e;
  // basis and work vector in split-FP32 pairs (8 bytes per entry)
  if ((e = cudaMalloc(&c->d_V, (size_t)(K + 1) * ldv * sizeof(float2))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->d_w, ldv * sizeof(float2))) != cudaSuccess) return e;
  if ((e = cudaMemset(c->d_V, 0, (size_t)(K + 1) * ldv * sizeof(float2))) != cudaSuccess) return e;
  if ((e = cudaMemset(c->d_w, 0, ldv * sizeof(float2))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->d_r, 2 * n * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->d_aug, (size_t)HDG_MAX_AUGMENT * ldv * 8)) != cudaSuccess) return e;
  if ((e = cudaMemset(c->d_aug, 0, (size_t)HDG_MAX_AUGMENT * ldv * 8)) != cudaSuccess) return e;
  // partial rows of a multi-dot: kgd / gy per group (at most KGD_MAX over all
  // groups) or 152 per group, each row (K + 2) columns at most
  if ((e = cudaMalloc(&c->d_part, (size_t)(KG > KGD_MAX ? KG : KGD_MAX) * (K + 2) * sizeof(double))) != cudaSuccess)
    return e;
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

// Multi-dot over nv basis vectors (ncol = nv + 1 appends ||w||^2): about kgd
// blocks over all groups of VG vectors (at least one per SM along x), fewer
// for short vectors. Returns the number of partial rows (blocks along x).
// f64: FP64 basis (double pairs), else split-FP32 pairs.
static int launch_mdot(const void* V4, int64_t np, int nv, int ncol, const void* w4, double* part,
                       const int* fl, cudaStream_t st, int kgd, const Batch& bt, int nb = 1, bool f64 = false) {
  const int gy = (ncol + VG - 1) / VG;
  // about kgd blocks over all groups: whole waves of the resident blocks (4 per SM), not a
  // partly filled last wave
  int64_t gx = kgd / gy > 0 ? kgd / gy : 1;
  const int64_t need = (np + KT - 1) / KT;
  if (gx > need) gx = need > 1 ? need : 1;
  const dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)nb);
  if (f64)
    d_mdot_kernel<<<grid, KT, 0, st>>>(static_cast<const double2*>(V4), np, nv, ncol, static_cast<const double2*>(w4),
                                       part, fl, bt);
  else
    df_mdot_kernel<<<grid, KT, 0, st>>>(static_cast<const float4*>(V4), np, nv, ncol, static_cast<const float4*>(w4),
                                        part, fl, bt);
  return (int)gx;
}

// out = (w - sum_i coef_i V_i) * scale over the basis of either type
static void launch_update(bool f64, dim3 grid, cudaStream_t st, const void* V4, int64_t np, int nv, const double* coef,
                          const void* w4, const double* sm, int scale_off, void* out, const int* stop, const Batch& bt,
                          int64_t rout) {
  if (f64)
    d_update_kernel<<<grid, KT, 0, st>>>(static_cast<const double2*>(V4), np, nv, coef, static_cast<const double2*>(w4),
                                         sm, scale_off, static_cast<double2*>(out), stop, bt, rout);
  else
    df_update_kernel<<<grid, KT, 0, st>>>(static_cast<const float4*>(V4), np, nv, coef, static_cast<const float4*>(w4),
                                          sm, scale_off, static_cast<float4*>(out), stop, bt, rout);
}

// first basis vector of a cycle: V0 = a * sm[off]
static void launch_first(bool f64, cudaStream_t st, const double* a, const double* sm, int off, void* V0, int64_t n,
                         const int* stop) {
  if (f64) to_d_kernel<<<KG, KT, 0, st>>>(a, sm, off, static_cast<double*>(V0), n, stop);
  else to_df_kernel<<<KG, KT, 0, st>>>(a, sm, off, static_cast<float2*>(V0), n, stop);
}

// x += sum_i y_i V_i
static void launch_xupdate(bool f64, cudaStream_t st, const void* V, int64_t n, int64_t ldv, int nv, const double* y,
                           double* x) {
  if (f64) d_xupdate_kernel<<<KG, KT, 0, st>>>(static_cast<const double*>(V), n, ldv, nv, y, x);
  else df_xupdate_kernel<<<KG, KT, 0, st>>>(static_cast<const float2*>(V), n, ldv, nv, y, x);
}

// The operator of the condensed system: the uniform-level kernels, or the
// level-mesh kernels (element-side products and a per-face sum).
static const void* op_blocks(hdg_ctx* c, int mode) {
  if (c->lv)
    return mode == 0 ? (const void*)c->lv->d_St : (mode == 2 ? (const void*)c->lv->d_Stdf : (const void*)c->lv->d_St32);
  if (mode == 3) return c->d_Sfix;
  return mode == 0 ? (const void*)c->d_St : (mode == 2 ? (const void*)c->d_Stdf : (const void*)c->d_St32);
}

// y = S x with the unpreconditioned FP64 blocks, nb columns of stride n
static cudaError_t op_resid(hdg_ctx* c, const double* x, double* y, int nb, int64_t n, cudaStream_t st) {
  if (c->lv) return launch_level_apply(c, 0, 0, c->lv->d_S, x, y, nb, n, nullptr, nullptr, st);
  if (nb == 1) return launch_apply64(c->prm, c->d_S, x, y, nullptr, nullptr, st);
  return launch_apply_mrhs(0, 0, c->prm, c->d_S, x, y, nb, n, nullptr, st);
}

// z = D^-1 y (or S_ff^-1 y face by face) on one FP64 vector
static cudaError_t op_dinv(hdg_ctx* c, const double* y, double* z, cudaStream_t st) {
  if (c->pc_face) {
    if (c->lv) return launch_level_face_pinv(c->lv->dv, c->lv->d_Pinv, y, z, 1, c->prm.N_tr, st);
    return launch_face_pinv(c->prm, c->d_Pinv, c->transposed, y, z, st);
  }
  if (c->lv) return launch_level_dinv(c, y, z, 1, c->prm.N_tr, st);
  return launch_face_dinv(c->prm, c->dt.Ghinv, c->d_escale, y, z, st);
}

// Cycle length of restarted GMRES. GMRES(K) can stagnate on a non-normal
// operator: the cycle's minimal-residual polynomial stops reducing the true
// residual and every later cycle repeats it (on the banded-level workload one
// column of 64 stays at 0.21, and which column is trapped changes with
// rounding alone). When a cycle cuts the true residual by less than 1 %, the
// next cycles get a different length: K - d, K - 2d, ... (d = K/8), back to K
// below K/2 (varying the restart length, after Baker, Jessup and Kolev 2009).
// A cycle shorter than K runs step by step instead of as the captured graph.
static int next_cycle_length(int cur, int K, bool stalled) {
  if (!stalled) return cur;
  const int d = std::max(1, K / 8), lo = std::max(1, (K + 1) / 2);
  return cur - d >= lo ? cur - d : K;
}

hdg_status gmres_solve(hdg_ctx* c, const double* g, double* x, const hdg_solve_opts& o, hdg_solve_report& rep) {
  const Params& P = c->prm;
  const int K = o.restart;
  const int64_t n = P.N_tr;
  cudaStream_t st = c->stream;
  Cu cu{c};
  if (!cu.ok(ensure_krylov(c, K))) return fail(c, HDG_ERR_OOM, std::string("Krylov workspace: ") + cudaGetErrorString(cu.err));
  SmallLayout L(K);
  double* sm = c->d_small;
  int* fl = c->d_flag;
  // basis entries: FP64, split-FP32 pairs or fixed-point limbs (8 bytes each); the operator
  // reads FP64 vectors except with the split-FP32 basis
  const bool f64b = o.basis == HDG_BASIS_FP64;
  const bool fixb = o.basis == HDG_BASIS_FIX;
  const int vt = o.basis == HDG_BASIS_DF64 ? 1 : 0;
  const size_t esz = 8;
  char* V = reinterpret_cast<char*>(c->d_V);
  void* w = c->d_w;
  const int64_t ldv = n + (n & 1), np = ldv / 2;   // basis row length (even) and element pairs
  // fixed-point basis: chunk scales and the FP64 copy of the newest vector
  const int64_t nch = fx_chunks(n);
  if (fixb && !c->d_Vs) {
    if (!cu.ok(cudaMalloc(&c->d_Vs, (size_t)(K + 1) * nch * sizeof(int))) ||
        !cu.ok(cudaMalloc(&c->d_vin, (size_t)ldv * sizeof(double))))
      return fail(c, HDG_ERR_OOM, std::string("fixed-point basis: ") + cudaGetErrorString(cu.err));
  }
  const Batch one{np, 0, 0, 0, 0, 0};
  const void* V4 = V;
  void* w4 = w;
  double* t = c->d_r;           // true residual g - S x (FP64)
  double* r0 = c->d_r + n;      // S x, then D^-1 t
  double* part = c->d_part;
  rep = hdg_solve_report{};
  // Arnoldi operator D^-1 S on split-FP32 vectors
  const int bt = o.mode == 0 ? 0 : (o.mode == 2 ? 1 : (o.mode == 3 ? 3 : 2));
  const void* Sop = op_blocks(c, o.mode);
  const int phase = o.mode == 1 ? HDG_PROF_APPLY32 : HDG_PROF_APPLY;
  // launch shapes: the autotuner's choices, else the defaults; the streaming
  // update needs no more than one pass of KT pairs per block
  const int kgd = c->tune_kgd > 0 ? c->tune_kgd : KGD;
  const int kgu = c->tune_kgu > 0 ? c->tune_kgu : KGU;
  // the pipelined shape runs on split-FP32 vectors only
  const int epb = (vt == 0 && c->tune_epb[bt] < 0) ? 0 : c->tune_epb[bt];
  const int gu = (int)std::min<int64_t>(kgu, std::max<int64_t>(1, (np + KT - 1) / KT));
  // the pipelined apply's timeout flag, read once the solve has synchronised
  auto bulk_wait_gave_up = [&]() -> bool {
    if (!(epb < 0 && bt == 1 && vt == 1)) return false;
    int err = 0;
    return !cu.ok(apply_bulk_take_error(st, &err)) || err != 0;
  };

  // ||g||
  axpby_norm_kernel<<<KG, KT, 0, st>>>(1.0, g, 0.0, g, t, n, part);
  sum_partials_kernel<<<1, 32, 0, st>>>(part, KG, sm + L.sc + 5);
  LAUNCHED(2);
  const double gnorm = std::sqrt(read_scalar(c, sm + L.sc + 5, cu));
  if (cu.err != cudaSuccess) return fail(c, HDG_ERR_CUDA, cudaGetErrorString(cu.err));
  if (gnorm == 0.0) {
    cu.ok(cudaMemsetAsync(x, 0, n * sizeof(double), st));
    cu.ok(cudaStreamSynchronize(st));
    rep.converged = 1;
    return cu.err == cudaSuccess ? HDG_OK : fail(c, HDG_ERR_CUDA, cudaGetErrorString(cu.err));
  }
  int its = 0, klen = K;
  // augmented restarts: nz stored corrections (ring of o.augment slots, zslot the oldest once full)
  char* Zr = reinterpret_cast<char*>(c->d_aug);
  int nz = 0, zslot = 0;
  double rel = 1.0, prev_rel = 0.0;
  while (true) {
    // true residual with the unpreconditioned FP64 operator (the stopping test)
    {
      ProfScope ps(c, HDG_PROF_RESID);
      cu.ok(op_resid(c, x, r0, 1, n, st));
    }
    axpby_norm_kernel<<<KG, KT, 0, st>>>(1.0, g, -1.0, r0, t, n, part);
    sum_partials_kernel<<<1, 32, 0, st>>>(part, KG, sm + L.sc + 5);
    LAUNCHED(3);
    rel = std::sqrt(read_scalar(c, sm + L.sc + 5, cu)) / gnorm;
    if (cu.err != cudaSuccess) return fail(c, HDG_ERR_CUDA, cudaGetErrorString(cu.err));
    rep.iterations = its;
    rep.rel_residual = rel;
    rep.outer += 1;
    if (rel <= o.tol) {
      rep.converged = 1;
      return bulk_wait_gave_up() ? fail(c, HDG_ERR_TIMEOUT, "pipelined apply: a bounded copy wait gave up") : HDG_OK;
    }
    if (its >= o.maxit) break;
    klen = next_cycle_length(klen, K, prev_rel > 0.0 && rel > 0.99 * prev_rel);
    prev_rel = rel;
    // r0 = D^-1 t; V0 = r0 / beta; the cycle aims at the reduction the true residual still needs
    cu.ok(op_dinv(c, t, r0, st));
    const double factor = 0.5 * o.tol / rel;
    cu.ok(cudaMemcpyAsync(sm + L.sc + 2, &factor, sizeof(double), cudaMemcpyHostToDevice, st));
    axpby_norm_kernel<<<KG, KT, 0, st>>>(1.0, r0, 0.0, r0, r0, n, part);
    cycle_init_kernel<<<1, 256, 0, st>>>(sm, L, fl, part, KG);
    if (fixb) launch_fx_combine(V, c->d_Vs, ldv, n, 0, nullptr, 0.0, r0, 1.0, sm, L.sc + 4, c->d_vin, V, c->d_Vs, fl, st);
    else launch_first(f64b, st, r0, sm, L.sc + 4, V, n, fl);
    LAUNCHED(4);
    const int jmax = std::min(klen, o.maxit - its);
    // steps m .. jmax-1 take the stored corrections as operator inputs (at least one Krylov step)
    const int nzc = std::min(nz, std::max(0, jmax - 1));
    const int m = jmax - nzc;
    std::vector<size_t> mark(jmax + 1, 0);   // profiling entries recorded before Arnoldi step j
    // one Arnoldi step j on stream s (timed phases only when profiling, i.e. not captured)
    // (ev: event quadruple of a captured, timed step: apply begin/end, vector work begin/end)
    auto enqueue_step = [&](int j, cudaStream_t s, bool timed, cudaEvent_t* ev) {
      const int nv = j + 1;
      double* Hcol = sm + L.H + (size_t)j * (K + 1);
      if (ev) cu.ok(cudaEventRecordWithFlags(ev[0], s, cudaEventRecordExternal));
      {
        ProfScope ps(c, timed ? phase : -1);
        const void* in = fixb ? (const void*)c->d_vin
                              : (j < m ? (const void*)(V + (size_t)j * ldv * esz)
                                       : (const void*)(Zr + (size_t)(j - m) * ldv * esz));
        if (c->lv) cu.ok(launch_level_apply(c, bt, vt, Sop, in, w, 1, ldv, precond_scale(c), fl, s));
        else cu.ok(launch_apply_vdf(bt, P, Sop, in, w, precond_scale(c), fl, s, epb, vt, &c->bulk_hooks));
      }
      if (ev) {
        cu.ok(cudaEventRecordWithFlags(ev[1], s, cudaEventRecordExternal));
        cu.ok(cudaEventRecordWithFlags(ev[2], s, cudaEventRecordExternal));
      }
      ProfScope po(c, timed ? HDG_PROF_ORTHO : -1);
      void* Vn = V + (size_t)(j + 1) * ldv * esz;
      // the basis passes of either representation: multi-dot (ncol = nv, or nv + 1 with
      // ||w||^2), w -= V htmp, and V_{j+1} = (w - V htmp) * sm[sc + 4]
      auto mdot = [&](int ncol, const int* flag) -> int {
        if (fixb) return launch_fx_mdot(V, c->d_Vs, ldv, n, nv, ncol, static_cast<const double*>(w), part, flag, s);
        return launch_mdot(V4, np, nv, ncol, w4, part, flag, s, kgd, one, 1, f64b);
      };
      auto update_w = [&](const int* flag) {
        if (fixb)
          launch_fx_combine(V, c->d_Vs, ldv, n, nv, sm + L.htmp, -1.0, static_cast<const double*>(w), 1.0, sm, -1,
                            static_cast<double*>(w), nullptr, nullptr, flag, s);
        else launch_update(f64b, dim3(gu), s, V4, np, nv, sm + L.htmp, w4, sm, -1, w4, flag, one, 0);
      };
      auto update_v = [&]() {
        if (fixb)
          launch_fx_combine(V, c->d_Vs, ldv, n, nv, sm + L.htmp, -1.0, static_cast<const double*>(w), 1.0, sm,
                            L.sc + 4, c->d_vin, Vn, c->d_Vs + (size_t)(j + 1) * nch, fl, s);
        else launch_update(f64b, dim3(gu), s, V4, np, nv, sm + L.htmp, w4, sm, L.sc + 4, Vn, fl, one, 0);
      };
      if (o.orth == 0) {
        // CGS2 in four passes over the basis: (1) h1 = V^T w; (2) w' = w - V h1;
        // (3) h2 = V^T w' and ||w'||^2; (4) V_{j+1} = (w' - V h2) / ||w' - V h2||,
        // the norm from ||w'||^2 - ||h2||^2
        int G = mdot(nv, fl);
        mdot_reduce_kernel<<<nv, 128, 0, s>>>(part, G, nv, nv, Hcol, sm + L.htmp, 0, fl, nullptr);
        update_w(fl);
        G = mdot(nv + 1, fl);
        reduce2_givens_kernel<<<dim3((nv + 32) / 32, 1), 1024, 0, s>>>(part, G, nv, sm, L, fl, j, 1, one, F_STOP);
      } else if (o.orth == 1) {
        // classical Gram-Schmidt, one projection in two passes: (1) h = V^T w and
        // ||w||^2; (2) V_{j+1} = (w - V h) / ||w - V h||, the norm from ||w||^2 - ||h||^2
        const int G = mdot(nv + 1, fl);
        reduce2_givens_kernel<<<dim3((nv + 32) / 32, 1), 1024, 0, s>>>(part, G, nv, sm, L, fl, j, 0, one, F_STOP);
      } else {
        // as orth = 1, plus a second projection (w' = w - V h; h2 = V^T w', ||w'||^2) only
        // when the first pass finds ||w - V h||^2 < ||w||^2 / 2; the second-pass kernels
        // are always launched and return at once when flag F_P2 says it is not needed
        int G = mdot(nv + 1, fl);
        reduce2_givens_kernel<<<dim3((nv + 32) / 32, 1), 1024, 0, s>>>(part, G, nv, sm, L, fl, j, o.orth, one, F_STOP);
        update_w(fl + F_P2);
        G = mdot(nv + 1, fl + F_P2);
        reduce2_givens_kernel<<<dim3((nv + 32) / 32, 1), 1024, 0, s>>>(part, G, nv, sm, L, fl, j, 1, one, F_P2);
      }
      update_v();
      if (ev) cu.ok(cudaEventRecordWithFlags(ev[3], s, cudaEventRecordExternal));
    };
    const int per_step = o.orth == 1 ? 4 : 6;
    const bool graph_cycle = jmax == K;
    if (graph_cycle) {
      // the whole cycle as one CUDA graph, captured once per configuration on a
      // private stream and replayed on the context stream; the device stop flag
      // turns the steps after convergence into immediate returns. With
      // profiling on, the capture carries an event quadruple per step.
      const int timed = c->prof_on ? 1 : 0;
      const std::vector<intptr_t> key = {K, bt, vt, o.basis, o.orth, timed, m, (intptr_t)Zr, (intptr_t)c->bulk_hooks.wait_cycles,
                                         c->bulk_hooks.skip_edge, (intptr_t)Sop, (intptr_t)V, (intptr_t)w,
                                         (intptr_t)part, (intptr_t)sm, (intptr_t)fl, (intptr_t)precond_scale(c),
                                         (intptr_t)np, kgd, kgu, epb, c->lv ? c->lv->rb : 0};
      if (timed && (int)c->gm_ev.size() < 4 * K) {
        while ((int)c->gm_ev.size() < 4 * K) {
          cudaEvent_t ev;
          if (!cu.ok(cudaEventCreate(&ev))) break;
          c->gm_ev.push_back(ev);
        }
        for (auto& gc : c->gm_cache) cudaGraphExecDestroy(gc.second);   // event handles are part of a timed capture
        c->gm_cache.clear();
      }
      // (augmented restarts use up to HDG_MAX_AUGMENT + 1 cycle shapes per solve: a small cache)
      constexpr size_t kGraphCache = 6;
      size_t hit = c->gm_cache.size();
      for (size_t i = 0; i < c->gm_cache.size(); ++i)
        if (c->gm_cache[i].first == key) hit = i;
      if (hit == c->gm_cache.size()) {
        if (c->gm_cache.size() >= kGraphCache) {
          cudaGraphExecDestroy(c->gm_cache.back().second);
          c->gm_cache.pop_back();
        }
        if (!c->cap_stream) cu.ok(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        if (cu.ok(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal))) {
          for (int j = 0; j < K; ++j) enqueue_step(j, c->cap_stream, false, timed ? &c->gm_ev[4 * j] : nullptr);
          cu.ok(cudaStreamEndCapture(c->cap_stream, &graph));
        }
        if (graph) {
          cu.ok(cudaGraphInstantiate(&exec, graph, 0));
          cudaGraphDestroy(graph);
        }
        if (cu.err != cudaSuccess) {
          if (exec) cudaGraphExecDestroy(exec);
          return fail(c, HDG_ERR_CUDA, std::string("GMRES cycle capture: ") + cudaGetErrorString(cu.err));
        }
        c->gm_cache.insert(c->gm_cache.begin(), {key, exec});
      } else if (hit > 0) {
        std::rotate(c->gm_cache.begin(), c->gm_cache.begin() + hit, c->gm_cache.begin() + hit + 1);
      }
      cu.ok(cudaGraphLaunch(c->gm_cache.front().second, st));
      LAUNCHED(per_step * K);
    } else {
      for (int j = 0; j < jmax; ++j) {
        mark[j] = c->prof_ev.size();
        enqueue_step(j, st, true, nullptr);
        LAUNCHED(per_step);
      }
    }
    cu.ok(cudaGetLastError());
    int hflags[2] = {0, 0};
    cu.ok(cudaMemcpyAsync(hflags, fl, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    cu.ok(cudaStreamSynchronize(st));
    if (cu.err != cudaSuccess) return fail(c, HDG_ERR_CUDA, cudaGetErrorString(cu.err));
    const int jused = hflags[F_JUSED];
    if (c->prof_on && graph_cycle) {
      // timed capture: fold the per-step events of the steps that did work
      for (int j = 0; j < jused; ++j) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->gm_ev[4 * j], c->gm_ev[4 * j + 1]) == cudaSuccess) {
          c->prof_ms[phase] += ms;
          c->prof_count[phase] += 1;
        }
        if (cudaEventElapsedTime(&ms, c->gm_ev[4 * j + 2], c->gm_ev[4 * j + 3]) == cudaSuccess) {
          c->prof_ms[HDG_PROF_ORTHO] += ms;
          c->prof_count[HDG_PROF_ORTHO] += 1;
        }
      }
    } else if (c->prof_on && jused < jmax) {
      // steps after the stop flag was raised were enqueued but returned at once: not timed work
      for (size_t i = mark[jused]; i < c->prof_ev.size(); ++i) c->prof_pool.push_back(c->prof_ev[i].second);
      c->prof_ev.resize(mark[jused]);
    }
    its += jused;
    rep.restarts += 1;
    if (jused == 0) break;
    lsq_kernel<<<1, 32, 0, st>>>(sm, L, fl);
    if (o.augment > 0) {
      // x += c = V y + Z y (the cycle's correction), then c / ||c|| becomes a stored correction
      const int nvv = std::min(jused, m), nzu = std::max(0, jused - m);
      const int slot = nz < o.augment ? nz : zslot;
      void* zdst = Zr + (size_t)slot * ldv * esz;
      if (f64b) {
        aug_correction_kernel<double><<<KG, KT, 0, st>>>(reinterpret_cast<const double*>(V),
                                                         reinterpret_cast<const double*>(Zr), n, ldv, nvv, nzu, m,
                                                         sm + L.y, x, r0, part);
        aug_store_kernel<double><<<KG, KT, 0, st>>>(r0, part, KG, static_cast<double*>(zdst), n);
      } else {
        aug_correction_kernel<float2><<<KG, KT, 0, st>>>(reinterpret_cast<const float2*>(V),
                                                         reinterpret_cast<const float2*>(Zr), n, ldv, nvv, nzu, m,
                                                         sm + L.y, x, r0, part);
        aug_store_kernel<float2><<<KG, KT, 0, st>>>(r0, part, KG, static_cast<float2*>(zdst), n);
      }
      if (nz < o.augment) ++nz;
      else zslot = (zslot + 1) % o.augment;
      LAUNCHED(3);
    } else {
      if (fixb) launch_fx_combine(V, c->d_Vs, ldv, n, jused, sm + L.y, 1.0, x, 1.0, sm, -1, x, nullptr, nullptr, nullptr, st);
      else launch_xupdate(f64b, st, V, n, ldv, jused, sm + L.y, x);
      LAUNCHED(2);
    }
  }
  rep.converged = 0;
  if (bulk_wait_gave_up()) return fail(c, HDG_ERR_TIMEOUT, "pipelined apply: a bounded copy wait gave up");
  return fail(c, HDG_ERR_NOCONV, "GMRES reached maxit with relative residual " + std::to_string(rel));
}

// ------------------------------------------------------------- autotuner
hdg_status autotune(hdg_ctx* c, const hdg_solve_opts& o, hdg_tune_report& rep) {
  const Params& P = c->prm;
  const int K = o.restart;
  Cu cu{c};
  if (!cu.ok(ensure_krylov(c, K))) return fail(c, HDG_ERR_OOM, std::string("Krylov workspace: ") + cudaGetErrorString(cu.err));
  cudaStream_t st = c->stream;
  const int64_t n = P.N_tr, ldv = n + (n & 1), np = ldv / 2;
  const Batch one{np, 0, 0, 0, 0, 0};
  const int bt = o.mode == 0 ? 0 : (o.mode == 2 ? 1 : (o.mode == 3 ? 3 : 2));
  const void* Sop = op_blocks(c, o.mode);
  // (the fixed-point basis runs its operator on FP64 vectors: tuned as the FP64 basis)
  const bool f64b = o.basis != HDG_BASIS_DF64;
  const int vt = f64b ? 0 : 1;
  char* V = reinterpret_cast<char*>(c->d_V);
  const void* V4 = V;
  void* w4 = c->d_w;
  // scratch: the update writes basis vector nv (contents of the basis are not
  // kept across solves); no stop flag, so every candidate does its full work
  const int nv = K / 2 > 1 ? K / 2 : 1;
  double* coef = c->d_small;   // coefficients read by the update (any values)
  cudaEvent_t e0, e1;
  cu.ok(cudaEventCreate(&e0));
  cu.ok(cudaEventCreate(&e1));
  auto time_it = [&](auto&& launch) -> double {
    launch();
    float best = 1e30f;
    for (int r = 0; r < 5; ++r) {
      cu.ok(cudaEventRecord(e0, st));
      launch();
      cu.ok(cudaEventRecord(e1, st));
      cu.ok(cudaEventSynchronize(e1));
      float ms = 0.f;
      cu.ok(cudaEventElapsedTime(&ms, e0, e1));
      best = ms < best ? ms : best;
    }
    return best;
  };
  // apply: edges per block for 128 .. 512 threads (level meshes: element-side rows per CTA)
  const int def_epb = c->lv ? 0 : apply_edges_per_block(P);
  int best_epb = def_epb, best_rb = 256;
  double best_apply = 1e30, def_apply = 0.0;
  if (c->lv) {
    if (!cu.ok(level_ensure_z(c, 1))) return fail(c, HDG_ERR_OOM, "element-side buffer");
    for (int rb : {128, 256, 512}) {
      c->lv->rb = rb;
      const double t = time_it([&] { cu.ok(launch_level_apply(c, bt, vt, Sop, V, c->d_w, 1, ldv, precond_scale(c),
                                                              nullptr, st)); });
      if (rb == 256) def_apply = t;
      if (t < best_apply) { best_apply = t; best_rb = rb; }
    }
    c->lv->rb = best_rb;
  }
  for (int threads : {128, 256, 384, 512}) {
    if (c->lv) break;
    const int epb = threads / P.P1 > 0 ? threads / P.P1 : 1;
    if (epb * P.P1 > 512) continue;
    const double t = time_it([&] { cu.ok(launch_apply_vdf(bt, P, Sop, V, c->d_w, precond_scale(c), nullptr, st, epb, vt)); });
    if (epb == def_epb) def_apply = t;
    if (t < best_apply) { best_apply = t; best_epb = epb; }
  }
  if (def_apply == 0.0 && !c->lv)
    def_apply = time_it([&] { cu.ok(launch_apply_vdf(bt, P, Sop, V, c->d_w, precond_scale(c), nullptr, st, def_epb, vt)); });
  // split-FP32 blocks: the pipelined bulk-copy apply with 1 .. 3 consumer warps per edge
  double best_bulk = 0.0;
  for (int q = 1; q <= 3 && bt == 1 && !c->lv && !f64b; ++q) {
    if (!apply_bulk_available(P, q)) continue;
    const double t = time_it([&] {
      cu.ok(launch_apply_vdf(bt, P, Sop, V, c->d_w, precond_scale(c), nullptr, st, -q, 1, &c->bulk_hooks));
    });
    int err = 0;
    if (!cu.ok(apply_bulk_take_error(st, &err)) || err)
      return fail(c, HDG_ERR_TIMEOUT, "autotune: pipelined apply: a bounded copy wait gave up");
    c->launches += 6;
    if (best_bulk == 0.0 || t < best_bulk) best_bulk = t;
    if (t < best_apply) { best_apply = t; best_epb = -q; }
  }
  // multi-dot blocks
  int best_kgd = KGD;
  double best_mdot = 1e30, def_mdot = 0.0;
  for (int kgd : {608, 1216, 2432}) {
    const double t = time_it([&] { launch_mdot(V4, np, nv, nv + 1, w4, c->d_part, nullptr, st, kgd, one, 1, f64b); });
    if (kgd == KGD) def_mdot = t;
    if (t < best_mdot) { best_mdot = t; best_kgd = kgd; }
  }
  // streaming-update blocks
  int best_kgu = KGU;
  double best_upd = 1e30, def_upd = 0.0;
  void* out = V + (size_t)nv * ldv * 8;
  for (int kgu : {608, 1216, 2432, 4864}) {   // (the streaming update's candidate block counts)
    const int gu = (int)std::min<int64_t>(kgu, std::max<int64_t>(1, (np + KT - 1) / KT));
    const double t = time_it([&] {
      launch_update(f64b, dim3(gu), st, V4, np, nv, coef, w4, nullptr, -1, out, nullptr, one, 0);
      cu.ok(cudaGetLastError());
    });
    if (kgu == KGU) def_upd = t;
    if (t < best_upd) { best_upd = t; best_kgu = kgu; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->launches += 6 * (4 + 3 + 4) + 1;
  if (cu.err != cudaSuccess) return fail(c, HDG_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(cu.err));
  if (!c->lv) c->tune_epb[bt] = best_epb;
  c->tune_kgd = best_kgd;
  c->tune_kgu = best_kgu;
  rep.apply_edges_per_block = best_epb > 0 ? best_epb : 0;
  rep.apply_threads = c->lv ? best_rb : (best_epb < 0 ? apply_bulk_threads(P, -best_epb) : (best_epb * P.P1 + 31) / 32 * 32);
  rep.apply_bulk = best_epb < 0 ? -best_epb : 0;
  rep.apply_bulk_ms = best_bulk;
  rep.mdot_blocks = best_kgd;
  rep.update_blocks = best_kgu;
  rep.apply_ms = best_apply;
  rep.mdot_ms = best_mdot;
  rep.update_ms = best_upd;
  rep.default_ms = def_apply + def_mdot + def_upd;
  return HDG_OK;
}

// ------------------------------------------------- batched (several RHS)
// out[r] = sm[r * rsm + off]
__global__ void gather_scalar_kernel(const double* sm, int64_t rsm, int off, double* out, int nb) {
  for (int r = threadIdx.x; r < nb; r += blockDim.x) out[r] = sm[(size_t)r * rsm + off];
}

// per instance r: stop flag = done[r] (an instance that has converged sits out
// the cycle), used-steps = 0; sm[r][off] = vals[r] when vals is not null
__global__ void set_cycle_kernel(int* flags, int rflag, const int* done, double* sm, int64_t rsm, int off,
                                 const double* vals, int nb) {
  for (int r = threadIdx.x; r < nb; r += blockDim.x) {
    flags[r * rflag + F_STOP] = done[r];
    flags[r * rflag + F_JUSED] = 0;
    flags[r * rflag + F_CNT] = 0;
    flags[r * rflag + F_P2] = 1;
    if (vals) sm[(size_t)r * rsm + off] = vals[r];
  }
}

static cudaError_t ensure_krylov_batched(hdg_ctx* c, int K, int nb) {
  if (c->kb_restart == K && c->kb_nrhs == nb && c->d_Vb) return cudaSuccess;
  cudaFree(c->d_Vb); cudaFree(c->d_wb); cudaFree(c->d_rb); cudaFree(c->d_partb); cudaFree(c->d_smallb);
  cudaFree(c->d_flagb); cudaFree(c->d_scalb); cudaFree(c->d_Zb); cudaFree(c->d_cmapb); cudaFree(c->d_augb);
  c->d_Vb = nullptr; c->d_wb = nullptr; c->d_rb = nullptr; c->d_partb = nullptr; c->d_smallb = nullptr;
  c->d_flagb = nullptr; c->d_scalb = nullptr; c->d_Zb = nullptr; c->d_cmapb = nullptr; c->d_augb = nullptr;
  c->kb_restart = c->kb_nrhs = 0;
  const size_t n = (size_t)c->prm.N_tr, ldv = n + (n & 1);
  SmallLayout L(K);
  const size_t rows = (size_t)(KG > KGD_MAX ? KG : KGD_MAX) * (K + 2);
  cudaError_t e;
  if ((e = cudaMalloc(&c->d_Vb, (size_t)(K + 1) * nb * ldv * sizeof(float2))) != cudaSuccess) return e;
  if ((e = cudaMemset(c->d_Vb, 0, (size_t)(K + 1) * nb * ldv * sizeof(float2))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->d_wb, (size_t)nb * ldv * sizeof(float2))) != cudaSuccess) return e;
  if ((e = cudaMemset(c->d_wb, 0, (size_t)nb * ldv * sizeof(float2))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->d_rb, 2 * (size_t)nb * n * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->d_partb, (size_t)nb * rows * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->d_smallb, (size_t)nb * L.total * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->d_flagb, (size_t)nb * 4 * sizeof(int))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->d_scalb, (size_t)nb * 2 * sizeof(double))) != cudaSuccess) return e;
  const size_t nzb = c->lv ? 1 : (size_t)c->prm.N * nb * c->prm.n_t;   // level meshes use their own buffer
  if ((e = cudaMalloc(&c->d_Zb, nzb * sizeof(float2))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->d_cmapb, (size_t)nb * sizeof(int))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->d_augb, (size_t)HDG_MAX_AUGMENT * nb * ldv * 8)) != cudaSuccess) return e;
  if ((e = cudaMemset(c->d_augb, 0, (size_t)HDG_MAX_AUGMENT * nb * ldv * 8)) != cudaSuccess) return e;
  c->kb_restart = K;
  c->kb_nrhs = nb;
  return cudaSuccess;
}

hdg_status gmres_solve_batched(hdg_ctx* c, const double* g, double* x, int nb, const hdg_solve_opts& o,
                               hdg_solve_report& rep) {
  const Params& P = c->prm;
  const int K = o.restart;
  const int64_t n = P.N_tr;
  cudaStream_t st = c->stream;
  Cu cu{c};
  if (!cu.ok(ensure_krylov_batched(c, K, nb)))
    return fail(c, HDG_ERR_OOM, std::string("batched Krylov workspace: ") + cudaGetErrorString(cu.err));
  SmallLayout L(K);
  const int64_t ldv = n + (n & 1), np = ldv / 2;
  const int64_t rpart = (int64_t)(KG > KGD_MAX ? KG : KGD_MAX) * (K + 2);
  const Batch bt{(int64_t)nb * np, np, np, rpart, L.total, 4};
  const bool f64b = o.basis == HDG_BASIS_FP64;
  const int vt = f64b ? 0 : 1;
  const size_t esz = 8;   // basis entries: FP64 or split-FP32 pairs
  char* V = reinterpret_cast<char*>(c->d_Vb);
  const void* V4 = V;
  void* w4 = c->d_wb;
  double* t = c->d_rb;                 // [nb][n] true residuals
  double* r0 = c->d_rb + (size_t)nb * n;   // [nb][n] S x, then D^-1 t
  double* part = c->d_partb;
  double* sm = c->d_smallb;
  int* fl = c->d_flagb;
  double* scal = c->d_scalb;
  const int btype = o.mode == 0 ? 0 : (o.mode == 2 ? 1 : 2);
  const void* Sop = op_blocks(c, o.mode);
  const int phase = o.mode == 1 ? HDG_PROF_APPLY32 : HDG_PROF_APPLY;
  const int kgd = c->tune_kgd > 0 ? c->tune_kgd : KGD;
  const int kgu = c->tune_kgu > 0 ? c->tune_kgu : KGU;
  const int gu = (int)std::min<int64_t>(kgu, std::max<int64_t>(1, (np + KT - 1) / KT));
  rep = hdg_solve_report{};
  std::vector<double> host(nb), gnorm(nb), rel(nb, 1.0), prev_rel(nb, 0.0);
  int klen = K;
  // augmented restarts: per column nz stored corrections ([slot][column][ldv]), as in gmres_solve
  char* Zr = reinterpret_cast<char*>(c->d_augb);
  int nz = 0, zslot = 0;
  std::vector<int> done(nb, 0), its(nb, 0), hfl(4 * nb);
  int* d_done = reinterpret_cast<int*>(scal + nb);   // [nb] converged flags (device copy)
  auto norms = [&](const double* vec, int64_t stride, double a, const double* y2, double bcoef, double* outv) {
    for (int r = 0; r < nb; ++r) {
      axpby_norm_kernel<<<KG, KT, 0, st>>>(a, vec + (size_t)r * stride, bcoef, y2 ? y2 + (size_t)r * stride : vec,
                                           outv + (size_t)r * stride, n, part + (size_t)r * rpart);
      sum_partials_kernel<<<1, 32, 0, st>>>(part + (size_t)r * rpart, KG, sm + (size_t)r * L.total + L.sc + 5);
    }
    gather_scalar_kernel<<<1, 64, 0, st>>>(sm, L.total, L.sc + 5, scal, nb);
    cu.ok(cudaMemcpyAsync(host.data(), scal, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    cu.ok(cudaStreamSynchronize(st));
    c->launches += 2 * nb + 1;
  };
  norms(g, n, 1.0, nullptr, 0.0, t);
  for (int r = 0; r < nb; ++r) gnorm[r] = std::sqrt(host[r]);
  if (cu.err != cudaSuccess) return fail(c, HDG_ERR_CUDA, cudaGetErrorString(cu.err));
  for (int r = 0; r < nb; ++r)
    if (gnorm[r] == 0.0) {
      cu.ok(cudaMemsetAsync(x + (size_t)r * n, 0, n * sizeof(double), st));
      done[r] = 1;
      rel[r] = 0.0;
    }
  while (true) {
    // true residuals t_r = g_r - S x_r with the FP64 blocks (multi-RHS apply)
    {
      ProfScope ps(c, HDG_PROF_RESID);
      cu.ok(op_resid(c, x, r0, nb, n, st));
      c->launches += 1;
    }
    norms(g, n, 1.0, r0, -1.0, t);
    if (cu.err != cudaSuccess) return fail(c, HDG_ERR_CUDA, cudaGetErrorString(cu.err));
    rep.outer += 1;
    int left = 0, maxits = 0;
    for (int r = 0; r < nb; ++r) {
      if (gnorm[r] > 0.0) rel[r] = std::sqrt(host[r]) / gnorm[r];
      if (rel[r] <= o.tol) done[r] = 1;
      if (!done[r]) ++left;
      maxits = std::max(maxits, its[r]);
    }
    rep.iterations = maxits;
    rep.rel_residual = *std::max_element(rel.begin(), rel.end());
    if (left == 0) {
      rep.converged = 1;
      return HDG_OK;
    }
    if (maxits >= o.maxit) break;
    bool stalled = false;
    for (int r = 0; r < nb; ++r) {
      if (!done[r] && prev_rel[r] > 0.0 && rel[r] > 0.99 * prev_rel[r]) stalled = true;
      prev_rel[r] = rel[r];
    }
    klen = next_cycle_length(klen, K, stalled);
    // cycle start for the instances still running: r0 = D^-1 t, V_0 = r0 / ||r0||
    std::vector<double> factor(nb, 0.0);
    for (int r = 0; r < nb; ++r) factor[r] = done[r] ? 1.0 : 0.5 * o.tol / rel[r];
    cu.ok(cudaMemcpyAsync(scal, factor.data(), nb * sizeof(double), cudaMemcpyHostToDevice, st));
    cu.ok(cudaMemcpyAsync(d_done, done.data(), nb * sizeof(int), cudaMemcpyHostToDevice, st));
    set_cycle_kernel<<<1, 64, 0, st>>>(fl, 4, d_done, sm, L.total, L.sc + 2, scal, nb);
    c->launches += 1;
    // the Arnoldi operator of this cycle computes only the columns still iterating
    std::vector<int> act;
    for (int r = 0; r < nb; ++r)
      if (!done[r]) act.push_back(r);
    const int na = (int)act.size();
    const int* cmap = nullptr;
    if (na < nb) {
      cu.ok(cudaMemcpyAsync(c->d_cmapb, act.data(), na * sizeof(int), cudaMemcpyHostToDevice, st));
      cmap = c->d_cmapb;
    }
    for (int r = 0; r < nb; ++r) {
      if (done[r]) continue;
      double* tr = t + (size_t)r * n;
      double* rr = r0 + (size_t)r * n;
      double* smr = sm + (size_t)r * L.total;
      int* flr = fl + 4 * r;
      double* pr = part + (size_t)r * rpart;
      cu.ok(op_dinv(c, tr, rr, st));
      axpby_norm_kernel<<<KG, KT, 0, st>>>(1.0, rr, 0.0, rr, rr, n, pr);
      cycle_init_kernel<<<1, 256, 0, st>>>(smr, L, flr, pr, KG);
      launch_first(f64b, st, rr, smr, L.sc + 4, V + (size_t)r * ldv * esz, n, flr);
      c->launches += 4;
    }
    const int jmax = std::min(klen, o.maxit - maxits);
    const int nzc = std::min(nz, std::max(0, jmax - 1));
    const int m = jmax - nzc;
    for (int j = 0; j < jmax; ++j) {
      const int nv = j + 1;
      {
        ProfScope ps(c, phase);
        const void* in = j < m ? (const void*)(V + (size_t)j * nb * ldv * esz)
                               : (const void*)(Zr + (size_t)(j - m) * nb * ldv * esz);
        if (c->lv)
          cu.ok(launch_level_apply(c, btype, vt, Sop, in, c->d_wb, na, ldv, precond_scale(c), nullptr, st, cmap));
        else
          cu.ok(launch_apply_mrhs_el(btype, P, Sop, in, c->d_wb, na, ldv, precond_scale(c), c->d_Zb, st, cmap, vt));
        c->launches += 1;
      }
      ProfScope po(c, HDG_PROF_ORTHO);
      void* Vn = V + (size_t)(j + 1) * nb * ldv * esz;
      if (o.orth == 0) {
        int G = launch_mdot(V4, np, nv, nv, w4, part, fl, st, kgd, bt, nb, f64b);
        for (int r = 0; r < nb; ++r)
          mdot_reduce_kernel<<<nv, 128, 0, st>>>(part + (size_t)r * rpart, G, nv, nv,
                                                 sm + (size_t)r * L.total + L.H + (size_t)j * (K + 1),
                                                 sm + (size_t)r * L.total + L.htmp, 0, fl + 4 * r, nullptr);
        launch_update(f64b, dim3(gu, nb), st, V4, np, nv, sm + L.htmp, w4, sm, -1, w4, fl, bt, np);
        G = launch_mdot(V4, np, nv, nv + 1, w4, part, fl, st, kgd, bt, nb, f64b);
        reduce2_givens_kernel<<<dim3((nv + 32) / 32, nb), 1024, 0, st>>>(part, G, nv, sm, L, fl, j, 1, bt, F_STOP);
        c->launches += 4 + nb;
      } else if (o.orth == 1) {
        const int G = launch_mdot(V4, np, nv, nv + 1, w4, part, fl, st, kgd, bt, nb, f64b);
        reduce2_givens_kernel<<<dim3((nv + 32) / 32, nb), 1024, 0, st>>>(part, G, nv, sm, L, fl, j, 0, bt, F_STOP);
        c->launches += 2;
      } else {
        int G = launch_mdot(V4, np, nv, nv + 1, w4, part, fl, st, kgd, bt, nb, f64b);
        reduce2_givens_kernel<<<dim3((nv + 32) / 32, nb), 1024, 0, st>>>(part, G, nv, sm, L, fl, j, o.orth, bt, F_STOP);
        launch_update(f64b, dim3(gu, nb), st, V4, np, nv, sm + L.htmp, w4, sm, -1, w4, fl + F_P2, bt, np);
        G = launch_mdot(V4, np, nv, nv + 1, w4, part, fl + F_P2, st, kgd, bt, nb, f64b);
        reduce2_givens_kernel<<<dim3((nv + 32) / 32, nb), 1024, 0, st>>>(part, G, nv, sm, L, fl, j, 1, bt, F_P2);
        c->launches += 5;
      }
      launch_update(f64b, dim3(gu, nb), st, V4, np, nv, sm + L.htmp, w4, sm, L.sc + 4, Vn, fl, bt, np);
      c->launches += 2;
    }
    cu.ok(cudaGetLastError());
    cu.ok(cudaMemcpyAsync(hfl.data(), fl, 4 * nb * sizeof(int), cudaMemcpyDeviceToHost, st));
    cu.ok(cudaStreamSynchronize(st));
    if (cu.err != cudaSuccess) return fail(c, HDG_ERR_CUDA, cudaGetErrorString(cu.err));
    rep.restarts += 1;
    int any = 0;
    for (int r = 0; r < nb; ++r) {
      if (done[r]) continue;
      const int jused = hfl[4 * r + F_JUSED];
      its[r] += jused;
      if (jused == 0) continue;
      any = 1;
      double* smr = sm + (size_t)r * L.total;
      lsq_kernel<<<1, 32, 0, st>>>(smr, L, fl + 4 * r);
      if (o.augment > 0) {
        const int nvv = std::min(jused, m), nzu = std::max(0, jused - m);
        const int slot = nz < o.augment ? nz : zslot;
        const int64_t vs = (int64_t)nb * ldv;
        char* vcol = V + (size_t)r * ldv * esz;
        char* zcol = Zr + (size_t)r * ldv * esz;
        void* zdst = zcol + (size_t)slot * vs * esz;
        double* cr = r0 + (size_t)r * n;
        double* pr = part + (size_t)r * rpart;
        if (f64b) {
          aug_correction_kernel<double><<<KG, KT, 0, st>>>(reinterpret_cast<const double*>(vcol),
                                                           reinterpret_cast<const double*>(zcol), n, vs, nvv, nzu, m,
                                                           smr + L.y, x + (size_t)r * n, cr, pr);
          aug_store_kernel<double><<<KG, KT, 0, st>>>(cr, pr, KG, static_cast<double*>(zdst), n);
        } else {
          aug_correction_kernel<float2><<<KG, KT, 0, st>>>(reinterpret_cast<const float2*>(vcol),
                                                           reinterpret_cast<const float2*>(zcol), n, vs, nvv, nzu, m,
                                                           smr + L.y, x + (size_t)r * n, cr, pr);
          aug_store_kernel<float2><<<KG, KT, 0, st>>>(cr, pr, KG, static_cast<float2*>(zdst), n);
        }
        c->launches += 3;
      } else {
        launch_xupdate(f64b, st, V + (size_t)r * ldv * esz, n, (int64_t)nb * ldv, jused, smr + L.y, x + (size_t)r * n);
        c->launches += 2;
      }
    }
    if (o.augment > 0 && any) {
      if (nz < o.augment) ++nz;
      else zslot = (zslot + 1) % o.augment;
    }
    if (!any) break;
  }
  rep.converged = 0;
  return fail(c, HDG_ERR_NOCONV, "batched GMRES reached maxit with largest relative residual " +
                                     std::to_string(rep.rel_residual));
}

}  // namespace mehdg
