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
// the matching row-blocks S[e][k][j][t] (contiguous in t) from HBM. The
// split-FP32 operator also has a pipelined form further down
// (apply_bulk_kernel: bulk asynchronous copies of the row-blocks into shared
// memory, consumed by warps), which the launch-shape autotuner times beside
// this one.
#include "internal.h"
#include "launch.h"
#include "df64.h"
#include <type_traits>
#include <algorithm>

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

// Split-FP32 ("double-float") arithmetic: GB300 issues FP64 FMAs at 1/63 of
// the FP32 rate, so the FP64 apply is bound by the FP64 pipe, not by HBM.
// With split-FP32 blocks each entry is stored as an unevaluated sum hi + lo
// of two FP32 numbers (hi = fl32(s), lo = fl32(s - hi); 48 significant bits,
// same 8 bytes per entry), x is split the same way, and every product is
// accumulated with error-free transformations (Dekker's product via FMA,
// Knuth's two-sum) on the FP32 pipe.
// Vector element types of the edge-centric apply below: VT = 0 FP64 vectors
// (the FP64 Krylov basis), VT = 1 split-FP32 pairs (the split-FP32 basis).
// A gathered entry is converted once to the block type's accumulation type
// (BT = 0: double, 1: split pair, 2: float).
template <int BT>
struct VAcc;
template <>
struct VAcc<0> { using T = double; };
template <>
struct VAcc<1> { using T = float2; };
template <>
struct VAcc<2> { using T = float; };

template <int BT, int VT>
__device__ __forceinline__ typename VAcc<BT>::T vgather(const void* x, size_t i) {
  if constexpr (VT == 0) {
    const double v = static_cast<const double*>(x)[i];
    if constexpr (BT == 0) return v;
    else if constexpr (BT == 1) return df_from(v);
    else return (float)v;
  } else {
    const float2 v = static_cast<const float2*>(x)[i];
    if constexpr (BT == 0) return df_to(v);
    else if constexpr (BT == 1) return v;
    else return v.x;
  }
}

template <int BT>
__device__ __forceinline__ typename VAcc<BT>::T vzero() {
  if constexpr (BT == 1) return make_float2(0.f, 0.f);
  else return typename VAcc<BT>::T(0);
}

// byte offset of the per-vector edge table behind the gathered traces (16-byte aligned)
__host__ __device__ inline size_t vdf_tab_offset(int epb, int nt, size_t el) {
  return ((size_t)epb * 2 * nt * el + 15) / 16 * 16;
}

// The same edge-centric apply on Krylov-basis vectors: BT = 0: FP64 blocks,
// FP64 accumulation; BT = 1: split-FP32 blocks and accumulation on the FP32
// pipe; BT = 2: FP32 blocks, FP32 accumulation. VT: vector type (above).
template <int BT, int VT>
__global__ void __launch_bounds__(512) apply_vdf_kernel(Params P, const void* __restrict__ Sv,
                                                        const void* __restrict__ x, void* __restrict__ y,
                                                        const double* __restrict__ escale, int epb,
                                                        const int* __restrict__ stop) {
  if (stop && *stop) return;
  using XT = typename VAcc<BT>::T;
  extern __shared__ unsigned char sraw[];
  const int nt = P.n_t, P1 = P.P1, PP = P.P;
  XT* xs = reinterpret_cast<XT*>(sraw);                                        // [epb][2][n_t]
  int4* tab = reinterpret_cast<int4*>(sraw + vdf_tab_offset(epb, nt, sizeof(XT)));   // [epb][2]
  const int f0 = blockIdx.x * epb;
  const int tid = threadIdx.x;
  // the three edges (code, orientation) of each side's element, once per vector; then
  // one warp per vector gathers its n_t trace values
  for (int i = tid; i < 2 * epb; i += blockDim.x) {
    const int f = f0 + (i >> 1);
    int4 te = make_int4(-1, -1, -1, 0);
    if (f < P.n_int) {
      int e[2], k[2], fl[2];
      double len;
      edge_sides(f, P.n, e, k, fl, &len);
      int code[3], flip[3];
      elem_edges(e[i & 1], P.n, code, flip);
      te = make_int4(code[0], code[1], code[2], flip[0] | (flip[1] << 1) | (flip[2] << 2));
    }
    tab[i] = te;
  }
  __syncthreads();
  {
    const int lane = tid & 31, nw = blockDim.x >> 5;
    for (int vi = tid >> 5; vi < 2 * epb; vi += nw) {
      const int4 te = tab[vi];
      for (int c = lane; c < nt; c += 32) {
        const int kk = c < P1 ? 0 : (c < 2 * P1 ? 1 : 2);
        const int t = c - kk * P1;
        const int code = kk == 0 ? te.x : (kk == 1 ? te.y : te.z);
        const size_t xi = (size_t)code * P1 + (((te.w >> kk) & 1) ? PP - t : t);
        XT v = vzero<BT>();
        if (code >= 0 && HDG_INB(xi, P.N_tr, P.oob, 1)) v = vgather<BT, VT>(x, xi);
        xs[vi * nt + c] = v;
      }
    }
  }
  __syncthreads();
  const int le = tid / P1, s = tid - le * P1;
  const int f = f0 + le;
  if (le >= epb || f >= P.n_int) return;
  int e[2], k[2], fl[2];
  double len;
  edge_sides(f, P.n, e, k, fl, &len);
  // row t_side of each side's row-block (the edge dof s in the element's orientation)
  const int t0 = fl[0] ? PP - s : s, t1 = fl[1] ? PP - s : s;
  if (!HDG_INB((int64_t)e[0] * 3 + k[0], 3LL * P.N, P.oob, 2) || !HDG_INB((int64_t)e[1] * 3 + k[1], 3LL * P.N, P.oob, 2) ||
      !HDG_INB(t0, P1, P.oob, 2) || !HDG_INB(t1, P1, P.oob, 2) || !HDG_INB((int64_t)f * P1 + s, P.N_tr, P.oob, 3))
    return;
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
    const float2 out = df_norm(h0, l0);
    if constexpr (VT == 1) static_cast<float2*>(y)[(size_t)f * P1 + s] = out;
    else static_cast<double*>(y)[(size_t)f * P1 + s] = df_to(out);
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
    if constexpr (VT == 1) static_cast<float2*>(y)[(size_t)f * P1 + s] = make_float2(r, 0.f);
    else static_cast<double*>(y)[(size_t)f * P1 + s] = (double)r;
  } else {
    // FP64: both sides' terms as one sequence q = 0 .. 2 n_t - 1 with the
    // next batch of G0 loads issued before the FMAs of the current one and
    // two accumulator chains; the only FP64 work besides the 2 n_t FMAs is
    // one add and the face scale. (The FP64 pipe, 2 FMA/clock/SM on GB300,
    // is the bound: one FMA per 8-byte block entry.)
    constexpr int G0 = 8;
    const int nq = 2 * nt;
    const double* S = static_cast<const double*>(Sv);
    const double* b0 = S + ((size_t)e[0] * 3 + k[0]) * (size_t)nt * P1 + t0;
    const double* b1 = S + ((size_t)e[1] * 3 + k[1]) * (size_t)nt * P1 + t1 - (size_t)nt * P1;
    const double* xv = xs + le * 2 * nt;
    // four accumulator chains: a DFMA's result returns through the short scoreboard
    // after a long latency, and two chains per thread left the FP64 pipe idle ~20 %
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    double cur[G0], nxt[G0];
#pragma unroll
    for (int u = 0; u < G0; ++u) cur[u] = u < nq ? (u < nt ? b0 : b1)[(size_t)u * P1] : 0.0;
    for (int q0 = 0; q0 < nq; q0 += G0) {
#pragma unroll
      for (int u = 0; u < G0; ++u) {
        const int q = q0 + G0 + u;
        nxt[u] = q < nq ? (q < nt ? b0 : b1)[(size_t)q * P1] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < G0; ++u) {
        const int q = q0 + u;
        if (q < nq) acc[u & 3] = fma(cur[u], xv[q], acc[u & 3]);
      }
#pragma unroll
      for (int u = 0; u < G0; ++u) cur[u] = nxt[u];
    }
    double r = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    if (escale) r *= escale[f];
    if constexpr (VT == 1) static_cast<float2*>(y)[(size_t)f * P1 + s] = df_from(r);
    else static_cast<double*>(y)[(size_t)f * P1 + s] = r;
  }
}

// ---------------------------------------------------------------------------
// Pipelined variant of the split-FP32 apply (the GMRES operator). The two
// element-side row-blocks of each edge are moved HBM -> shared memory by the
// bulk-copy (TMA) engine, so the bytes in flight no longer depend on how many
// loads the threads keep outstanding. Warp-specialised persistent CTAs (one
// per SM) take the edges f = blockIdx.x + i gridDim.x: warp 0 (one lane)
// issues the copies of edge i into slot i % NC once the slot's consumers have
// released it; the slot's Q consumer warps split the edge's 2 n_t columns
// (side 0, then side 1) into Q contiguous parts. Per slot an mbarrier counts
// the copy's transaction bytes (full) and one counts the Q consumers' releases
// (empty), so warps wait only on their own slot. A consumer lane walks one row
// (trace position s) through its part with the one-thread-per-row apply's
// accumulator pattern; parts 1 .. Q-1 hand their sums to part 0 through
// shared memory and a per-slot mbarrier, part 0 adds them in part order, so
// Q = 1 gives that apply's bits and every Q its own fixed order. Each consumer gathers its part of the next edge's
// trace values into registers while it computes the current one. A row-block
// starts on an 8-byte boundary: the copy starts at the 16-byte boundary below
// it and covers the block rounded up to 16 bytes (the split-FP32 array
// carries 16 bytes of slack at its end). Every wait is bounded: on timeout the
// CTA sets apply_bulk_wait_error, lets the copies it issued land (bounded
// again) and returns.
// ---------------------------------------------------------------------------
constexpr int ABK_MAX_WARPS = 16;                      // producer + consumers
constexpr int ABK_MAX_SLOTS = 14;
constexpr int ABK_BARRIER_BYTES = 3 * ABK_MAX_SLOTS * 8 + 48;   // full, empty, parts (multiple of 16)
constexpr int ABK_XR = 5;                              // trace values per lane: part width <= 32 ABK_XR
constexpr long long ABK_WAIT_CYCLES = 2000000000LL;   // about one second at 2 GHz

__device__ int apply_bulk_wait_error;

struct BulkShape {
  int nc;      // slots
  int q;       // consumer warps per slot
  int cpw;     // columns per consumer warp
  int seg;     // bytes of one side's segment in a slot (multiple of 16)
  long long wait_cycles;   // limit of every mbarrier wait (clock64 cycles)
  int skip_edge;           // test hook: the interior edge whose copy is not issued (-1: none)
};

namespace {
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0u;
}
// true once the phase of this parity has completed; false after the cycle limit
// or once another warp of the CTA has given up (abort flag)
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, const volatile int* abort_flag,
                                                  long long limit) {
  const long long t0 = clock64();
  while (!mbar_test(bar, parity)) {
    if (abort_flag && *abort_flag) return false;
    if (clock64() - t0 > limit) return false;
  }
  return true;
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
}  // namespace

__global__ void __launch_bounds__(32 * ABK_MAX_WARPS) apply_bulk_kernel(
    Params P, const float2* __restrict__ S, const float2* __restrict__ x, float2* __restrict__ y,
    const double* __restrict__ escale, const int* __restrict__ stop, BulkShape B) {
  if (stop && *stop) return;
  extern __shared__ __align__(128) unsigned char sraw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(sraw);                  // [nc] copy landed
  uint64_t* empty = full + ABK_MAX_SLOTS;                               // [nc] slot released by its Q warps
  uint64_t* parts = empty + ABK_MAX_SLOTS;                              // [nc] parts 1 .. Q-1 written
  unsigned char* slots = sraw + ABK_BARRIER_BYTES;                       // [nc][2][seg]
  const int nt = P.n_t, P1 = P.P1, PP = P.P, NC = B.nc, Q = B.q, CPW = B.cpw;
  float2* xsall = reinterpret_cast<float2*>(slots + (size_t)NC * 2 * B.seg);   // [nc q][cpw]
  float2* redall = xsall + (size_t)NC * Q * CPW;                               // [nc][q][32]
  __shared__ int s_abort;
  __shared__ int s_issued[ABK_MAX_SLOTS], s_done[ABK_MAX_SLOTS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int G = gridDim.x;
  const int nE = (int)blockIdx.x < P.n_int ? (P.n_int - 1 - (int)blockIdx.x) / G + 1 : 0;
  const size_t blk_bytes = (size_t)nt * P1 * sizeof(float2);
  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int c = 0; c < NC; ++c) {
      mbar_init(smem_addr(&full[c]), 1);
      mbar_init(smem_addr(&empty[c]), (uint32_t)Q);
      if (Q > 1) mbar_init(smem_addr(&parts[c]), (uint32_t)(Q - 1));
      s_issued[c] = 0;
      s_done[c] = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  volatile int* abort_flag = &s_abort;

  if (warp == 0) {
    // producer: edge i into slot i % NC once its Q consumers have released the slot's previous edge
    if (lane == 0) {
      for (int i = 0; i < nE; ++i) {
        const int c = i % NC, u = i / NC;
        if (u > 0 && !mbar_wait_bounded(smem_addr(&empty[c]), (uint32_t)((u - 1) & 1), abort_flag, B.wait_cycles)) {
          *abort_flag = 1;
          break;
        }
        const int f = (int)blockIdx.x + i * G;
        // test hook: this edge's copy is never issued, so its consumers' bounded wait runs out
        if (f == B.skip_edge) continue;
        int e[2], k[2], fl[2];
        double len;
        edge_sides(f, P.n, e, k, fl, &len);
        const uint32_t bar = smem_addr(&full[c]);
        const char* src[2];
        uint32_t sz[2];
        bool in_range = true;
        for (int sd = 0; sd < 2; ++sd) {
          const size_t off = ((size_t)e[sd] * 3 + k[sd]) * blk_bytes;
          const size_t a0 = off & ~(size_t)15;
          src[sd] = reinterpret_cast<const char*>(S) + a0;
          sz[sd] = (uint32_t)(((off - a0) + blk_bytes + 15) & ~(size_t)15);
          // the array carries 16 bytes of slack past its 3 N row-blocks
          in_range = in_range && HDG_INB(a0 + sz[sd] - 1, 3 * (size_t)P.N * blk_bytes + 16, P.oob, 4);
        }
        if (!in_range) continue;   // (bounds-checked build) its consumers' bounded wait gives up
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_tx(bar, sz[0] + sz[1]);
        for (int sd = 0; sd < 2; ++sd)
          bulk_load(smem_addr(slots + ((size_t)c * 2 + sd) * B.seg), src[sd], sz[sd], bar);
        s_issued[c] = u + 1;
      }
    }
  } else if (warp <= NC * Q) {
    // consumer part pq of slot c: edges i = c, c + NC, ...; columns [q0, q1) of the edge's 2 n_t
    const int cw = warp - 1, c = cw / Q, pq = cw - c * Q;
    const int q0 = pq * CPW, q1 = min(2 * nt, q0 + CPW);
    float2* xs = xsall + (size_t)cw * CPW;
    float2* red = redall + (size_t)c * Q * 32;
    const unsigned char* seg0 = slots + (size_t)c * 2 * B.seg;
    const int nk = nE > c ? (nE - 1 - c) / NC + 1 : 0;
    const int e8 = (nt / 8) * 8;   // the one-thread-per-row apply pairs columns below e8 (per side)
    float2 xr[ABK_XR];
    auto gather = [&](int i) {
      const int f = (int)blockIdx.x + i * G;
      int e[2], k[2], fl[2];
      double len;
      edge_sides(f, P.n, e, k, fl, &len);
      int code[2][3], flip[2][3];
      elem_edges(e[0], P.n, code[0], flip[0]);
      elem_edges(e[1], P.n, code[1], flip[1]);
#pragma unroll
      for (int r = 0; r < ABK_XR; ++r) {
        const int c2 = q0 + lane + 32 * r;
        float2 v = make_float2(0.f, 0.f);
        if (c2 < q1) {
          const int sd = c2 >= nt ? 1 : 0, cc = c2 - sd * nt;
          const int kq = cc / P1, t = cc - kq * P1;
          if (code[sd][kq] >= 0) v = x[(size_t)code[sd][kq] * P1 + (flip[sd][kq] ? PP - t : t)];
        }
        xr[r] = v;
      }
    };
    auto stash = [&]() {
#pragma unroll
      for (int r = 0; r < ABK_XR; ++r)
        if (q0 + lane + 32 * r < q1) xs[lane + 32 * r] = xr[r];
      __syncwarp();
    };
    if (nk > 0) {
      gather(c);
      stash();
    }
    for (int kq = 0; kq < nk; ++kq) {
      const int i = c + kq * NC;
      if (kq + 1 < nk) gather(i + NC);   // loads in flight during the products below
      // every lane polls; the warp goes on only if all lanes saw the copy land (a uniform decision)
      if (!__all_sync(0xffffffffu,
                      mbar_wait_bounded(smem_addr(&full[c]), (uint32_t)(kq & 1), abort_flag, B.wait_cycles))) {
        if (lane == 0) *abort_flag = 1;
        break;
      }
      const int f = (int)blockIdx.x + i * G;
      int e[2], k[2], fl[2];
      double len;
      edge_sides(f, P.n, e, k, fl, &len);
      float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
      if (lane < P1) {
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
          const int jlo = max(q0, sd * nt) - sd * nt, jhi = min(q1, (sd + 1) * nt) - sd * nt;
          if (jlo >= jhi) continue;
          const size_t off = ((size_t)e[sd] * 3 + k[sd]) * blk_bytes;
          const float2* row = reinterpret_cast<const float2*>(seg0 + (size_t)sd * B.seg + (off & 15)) +
                              (fl[sd] ? PP - lane : lane);
          const int xb = sd * nt - q0;   // xs[xb + j]: trace value of column j of side sd
          // columns below e8 alternate between the two sums (odd j to the second), the rest go to the first
          const int jp = min(jhi, e8);
          int j = jlo;
          if ((j & 1) && j < jp) {
            df_fma(h1, l1, row[j * P1], xs[xb + j]);
            ++j;
          }
          for (; j + 1 < jp; j += 2) {
            df_fma(h0, l0, row[j * P1], xs[xb + j]);
            df_fma(h1, l1, row[(j + 1) * P1], xs[xb + j + 1]);
          }
          for (; j < jhi; ++j) {
            if (j < e8 && (j & 1)) df_fma(h1, l1, row[j * P1], xs[xb + j]);
            else df_fma(h0, l0, row[j * P1], xs[xb + j]);
          }
        }
      }
      df_add(h0, l0, h1, l1);   // this part's sum
      if (Q > 1) {
        if (pq > 0) {
          red[pq * 32 + lane] = make_float2(h0, l0);
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_addr(&parts[c]));
        } else if (!__all_sync(0xffffffffu, mbar_wait_bounded(smem_addr(&parts[c]), (uint32_t)(kq & 1), abort_flag,
                                                              B.wait_cycles))) {
          if (lane == 0) *abort_flag = 1;
          break;
        } else {
          for (int pp = 1; pp < Q; ++pp) {   // the parts' sums in part order
            const float2 v = red[pp * 32 + lane];
            df_add(h0, l0, v.x, v.y);
          }
        }
      }
      if (pq == 0 && lane < P1) {
        if (escale) {
          const float2 sc = df_from(escale[f]);
          float ph = 0.f, pl = 0.f;
          df_fma(ph, pl, make_float2(h0, l0), sc);
          h0 = ph;
          l0 = pl;
        }
        y[(size_t)f * P1 + lane] = df_norm(h0, l0);
      }
      __syncwarp();
      // the slot (and, for part 0, the other parts' sums) has been read: release it
      if (lane == 0) {
        if (pq == 0) s_done[c] = kq + 1;
        mbar_arrive(smem_addr(&empty[c]));
      }
      if (kq + 1 < nk) stash();
    }
  }
  __syncthreads();
  if (s_abort) {   // a wait gave up: record it and let every copy still in flight land
    if (threadIdx.x == 0) {
      atomicExch(&apply_bulk_wait_error, 1);
      for (int c = 0; c < NC; ++c)
        if (s_issued[c] > s_done[c])
          mbar_wait_bounded(smem_addr(&full[c]), (uint32_t)((s_issued[c] - 1) & 1), nullptr, B.wait_cycles);
    }
    __syncthreads();
  }
}

// Device limits of the pipelined apply, queried once: SM count and the
// dynamic shared memory a CTA may take (the opt-in maximum less the kernel's
// static shared memory), which the kernel's attribute is raised to.
static cudaError_t bulk_limits(int* sms, size_t* max_dyn) {
  static bool done = false;
  static int s_sms = 0;
  static size_t s_max = 0;
  if (!done) {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, apply_bulk_kernel);
    if (e != cudaSuccess) return e;
    if ((size_t)optin <= fa.sharedSizeBytes) return cudaErrorInvalidValue;
    s_max = (size_t)optin - fa.sharedSizeBytes;
    if ((e = cudaFuncSetAttribute(apply_bulk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_max)) !=
        cudaSuccess)
      return e;
    done = true;
  }
  *sms = s_sms;
  *max_dyn = s_max;
  return cudaSuccess;
}

// Shape of the pipelined apply with q = 1 .. 3 consumer warps per edge: one
// CTA per SM with as many slots as fit in max_dyn bytes of dynamic shared
// memory and in ABK_MAX_WARPS warps; false where it does not apply (an edge
// row wider than a warp, a part wider than the lanes' registers, or no slot
// fits).
static bool bulk_shape(const Params& P, int q, size_t max_dyn, BulkShape& B, size_t& smem) {
  if (q < 1 || q > 3 || P.P1 > 32) return false;
  B.q = q;
  B.cpw = (2 * P.n_t + q - 1) / q;
  if (B.cpw > 32 * ABK_XR) return false;
  const size_t blk_bytes = (size_t)P.n_t * P.P1 * sizeof(float2);
  B.seg = (int)((blk_bytes + 8 + 15) & ~(size_t)15);
  const size_t per_slot = (size_t)2 * B.seg + (size_t)q * B.cpw * sizeof(float2) + (size_t)q * 32 * sizeof(float2);
  // 228 KB of shared memory per SM, 1 KB reserved per CTA, 1 KB left for static shared memory
  const size_t per_cta = (size_t)228 * 1024 - 2048;
  const size_t cap = per_cta < max_dyn ? per_cta : max_dyn;
  if (cap < ABK_BARRIER_BYTES + per_slot) return false;
  int nc = (int)((cap - ABK_BARRIER_BYTES) / per_slot);
  nc = std::min(nc, std::min(ABK_MAX_SLOTS, (ABK_MAX_WARPS - 1) / q));
  B.nc = nc;
  smem = ABK_BARRIER_BYTES + (size_t)nc * per_slot;
  return true;
}

int apply_bulk_threads(const Params& P, int q) {
  BulkShape B;
  size_t smem, max_dyn;
  int sms;
  if (bulk_limits(&sms, &max_dyn) != cudaSuccess || !bulk_shape(P, q, max_dyn, B, smem)) return 0;
  return 32 * (1 + B.nc * B.q);
}

bool apply_bulk_available(const Params& P, int q) {
  BulkShape B;
  size_t smem, max_dyn;
  int sms;
  if (bulk_limits(&sms, &max_dyn) != cudaSuccess) return false;
  return bulk_shape(P, q, max_dyn, B, smem);
}

cudaError_t launch_apply_bulk(const Params& P, const float2* S, const float2* x, float2* y, const double* escale,
                              const int* stop, cudaStream_t st, int q, long long wait_cycles, int skip_edge) {
  BulkShape B;
  B.wait_cycles = wait_cycles > 0 ? wait_cycles : ABK_WAIT_CYCLES;
  B.skip_edge = skip_edge;
  size_t smem, max_dyn;
  int sms;
  cudaError_t e = bulk_limits(&sms, &max_dyn);
  if (e != cudaSuccess) return e;
  if (!bulk_shape(P, q, max_dyn, B, smem)) return cudaErrorInvalidValue;
  const int grid = std::max(1, std::min(sms, P.n_int));
  apply_bulk_kernel<<<grid, 32 * (1 + B.nc * B.q), smem, st>>>(P, S, x, y, escale, stop, B);
  return cudaGetLastError();
}

// Reads (and clears) the timeout flag of the pipelined apply.
cudaError_t apply_bulk_take_error(cudaStream_t st, int* err) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(err, apply_bulk_wait_error, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && *err) e = cudaMemcpyToSymbolAsync(apply_bulk_wait_error, &zero, sizeof(int), 0,
                                                             cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

cudaError_t launch_apply_vdf(int bt, const Params& P, const void* S, const void* x, void* y,
                             const double* escale, const int* stop, cudaStream_t st, int epb, int vt,
                             const BulkHooks* hk) {
  // epb < 0: the pipelined bulk-copy apply with -epb consumer warps per edge (split-FP32 blocks and vectors)
  if (epb < 0 && bt == 1 && vt == 1)
    return launch_apply_bulk(P, static_cast<const float2*>(S), static_cast<const float2*>(x), static_cast<float2*>(y),
                             escale, stop, st, -epb, hk ? hk->wait_cycles : 0, hk ? hk->skip_edge : -1);
  // bt = 3: fixed-point blocks (exact integer products) on FP64 vectors
  if (bt == 3) {
    if (vt != 0) return cudaErrorInvalidValue;
    return launch_apply_fix(P, S, static_cast<const double*>(x), static_cast<double*>(y), escale, stop, st, epb);
  }
  // epb edges per block, one thread per (edge, trace position): at most 512 threads
  if (epb <= 0 || epb * P.P1 > 512) epb = apply_edges_per_block(P);
  const int threads = (epb * P.P1 + 31) / 32 * 32;
  const int grid = (P.n_int + epb - 1) / epb;
  const size_t el = bt == 0 ? sizeof(double) : (bt == 1 ? sizeof(float2) : sizeof(float));
  const size_t sm = vdf_tab_offset(epb, P.n_t, el) + (size_t)epb * 2 * sizeof(int4);
#define VDF_CASE(B, V) \
  if (bt == B && vt == V) apply_vdf_kernel<B, V><<<grid, threads, sm, st>>>(P, S, x, y, escale, epb, stop);
  VDF_CASE(0, 0) VDF_CASE(1, 0) VDF_CASE(2, 0) VDF_CASE(0, 1) VDF_CASE(1, 1) VDF_CASE(2, 1)
#undef VDF_CASE
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


// FP64 vectors: the Arnoldi operators of the FP64-basis solve (and the true
// residual), with the default edges per block
cudaError_t launch_apply64(const Params& P, const double* S, const double* x, double* y, const double* escale,
                           const int* stop, cudaStream_t st, int epb) {
  return launch_apply_vdf(0, P, S, x, y, escale, stop, st, epb, 0, nullptr);
}

cudaError_t launch_apply_df(const Params& P, const float2* S, const double* x, double* y, const double* escale,
                            const int* stop, cudaStream_t st) {
  return launch_apply_vdf(1, P, S, x, y, escale, stop, st, 0, 0, nullptr);
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
