// Trace-operator apply (Sec. 3.3.2, steps 1-4) with FP64 products carried out
// exactly in integer arithmetic.
//
// The FP64 apply does one FP64 FMA per 8-byte block entry, and GB300's FP64
// pipe (2 FMA per clock per SM) caps that at about 74 % of the HBM bandwidth.
// Here every row of the preconditioned blocks and every element trace vector
// is held as signed 56-bit fixed-point numbers sharing one power-of-two scale
// (the row's, or the vector's, largest binary exponent), split into a signed
// high limb and a 28-bit low limb. The dot product of a row with a trace
// vector is then a sum of exact limb products (64-bit integer multiply-adds,
// which run on the integer pipe) with no rounding at all; the exact 128-bit
// sum is rounded once to FP64 per element side. The two sides and the face
// scale are then added and multiplied in FP64 as in the FP64 apply.
//
// Accuracy: the only errors besides the final roundings are the fixed-point
// roundings of the inputs, at most 2^-55 of the row's (vector's) largest
// magnitude per entry, so |y - y_exact| <= 2^-55 (max|s| sum|x| + max|x| sum|s|)
// per side plus one FP64 rounding of the result, against the FP64 FMA chain's
// bound of about n_t 2^-53 sum |s||x|.
//
// Layout: limbs [N][3][n_t][P1] int2 {lo, hi} (the FP64 blocks' layout),
// followed by the row scales [N][3][P1] int32 (the biased FP64 exponent of the
// row's largest entry). Bounds of the integer accumulators, with |hi| <= 2^27
// and 0 <= lo < 2^28, over the n_t <= 240 terms of one side's row: sum hi*hi,
// sum hi*lo and sum lo*hi each below 2^63 in magnitude, sum lo*lo unsigned
// below 2^64; n_t is limited to FIX_MAX_NT accordingly.
#include "internal.h"
#include "launch.h"
#include "fixpoint.h"
#include <algorithm>

namespace mehdg {

constexpr int FIX_MAX_NT = 240;
constexpr int FIX_GATHER = (FIX_MAX_NT + 31) / 32;   // trace values per lane in the gather
constexpr int FIX_G = 8;    // row entries per load group

// Shared memory of the apply, per CTA: limbs of the gathered trace vectors
// [epb][2][ntp] (n_t padded to a multiple of FIX_G with zero limbs), their
// scales [epb][2] and the edge table [epb][2].
__host__ __device__ inline int fix_ntp(int nt) { return (nt + FIX_G - 1) / FIX_G * FIX_G; }
__host__ __device__ inline size_t fix_tab_offset(int epb, int nt) {
  return ((size_t)epb * 2 * fix_ntp(nt) * 8 + (size_t)epb * 2 * 4 + 15) / 16 * 16;
}

// Rows (e, k, t) of the FP64 blocks -> limbs and row scales; one thread per row.
__global__ void fix_convert_kernel(const double* __restrict__ S, int2* __restrict__ L, int* __restrict__ ex,
                                   int64_t rows, int nt, int P1) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t blk = r / P1;
    const int t = (int)(r - blk * P1);
    const double* row = S + (size_t)blk * nt * P1 + t;
    int Eb = 1;
    for (int j = 0; j < nt; ++j) Eb = max(Eb, fix_exp_field((unsigned long long)__double_as_longlong(row[(size_t)j * P1])));
    int2* out = L + (size_t)blk * nt * P1 + t;
    for (int j = 0; j < nt; ++j)
      out[(size_t)j * P1] = fix_limbs((unsigned long long)__double_as_longlong(row[(size_t)j * P1]), Eb);
    ex[r] = Eb;
  }
}

size_t fix_blocks_bytes(const Params& P) {
  return (size_t)P.N * 3 * P.n_t * P.P1 * sizeof(int2) + (size_t)P.N * 3 * P.P1 * sizeof(int);
}

bool fix_supported(const Params& P) { return P.n_t <= FIX_MAX_NT; }


// One thread per (interior edge, trace position), EPB edges per CTA, as the
// FP64 apply: the CTA gathers both sides' trace vectors of its edges, finds
// each vector's largest exponent (shared-memory max), converts the vector to
// limbs, then every thread walks its row of each side's row-block.
__global__ void __launch_bounds__(512) apply_fix_kernel(Params P, const int2* __restrict__ L,
                                                        const int* __restrict__ rex, const double* __restrict__ x,
                                                        double* __restrict__ y, const double* __restrict__ escale,
                                                        int epb, const int* __restrict__ stop) {
  if (stop && *stop) return;
  extern __shared__ unsigned char sraw[];
  const int nt = P.n_t, P1 = P.P1, PP = P.P;
  const int ntp = fix_ntp(nt);
  int2* xs = reinterpret_cast<int2*>(sraw);                                // [epb][2][ntp] limbs
  int* xe = reinterpret_cast<int*>(sraw + (size_t)epb * 2 * ntp * 8);      // [epb][2] vector scales
  int4* tab = reinterpret_cast<int4*>(sraw + fix_tab_offset(epb, nt));     // [epb][2] edge codes, flips
  const int f0 = blockIdx.x * epb;
  const int tid = threadIdx.x;
  // the three edges (code, orientation) of each side's element, once per vector
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
  // one warp per vector: gather (all of a lane's loads issued together), the
  // largest exponent by a warp reduction, then the limbs
  {
    const int lane = tid & 31, nw = blockDim.x >> 5;
    for (int v = tid >> 5; v < 2 * epb; v += nw) {
      const int4 te = tab[v];
      unsigned long long b[FIX_GATHER];
      int Eb = 1;
#pragma unroll
      for (int it = 0; it < FIX_GATHER; ++it) {
        const int c = lane + 32 * it;
        b[it] = 0ull;
        if (c < nt) {
          const int kk = c < P1 ? 0 : (c < 2 * P1 ? 1 : 2);
          const int t = c - kk * P1;
          const int code = kk == 0 ? te.x : (kk == 1 ? te.y : te.z);
          const size_t xi = (size_t)code * P1 + (((te.w >> kk) & 1) ? PP - t : t);
          if (code >= 0 && HDG_INB(xi, P.N_tr, P.oob, 15)) b[it] = (unsigned long long)__double_as_longlong(x[xi]);
          Eb = max(Eb, fix_exp_field(b[it]));
        }
      }
      Eb = __reduce_max_sync(0xffffffffu, Eb);
#pragma unroll
      for (int it = 0; it < FIX_GATHER; ++it) {
        const int c = lane + 32 * it;
        if (c < ntp) xs[v * ntp + c] = c < nt ? fix_limbs(b[it], Eb) : make_int2(0, 0);
      }
      if (lane == 0) xe[v] = Eb;
    }
  }
  __syncthreads();
  const int le = tid / P1, s = tid - le * P1;
  const int f = f0 + le;
  if (le >= epb || f >= P.n_int) return;
  int e[2], k[2], fl[2];
  double len;
  edge_sides(f, P.n, e, k, fl, &len);
  const int t0 = fl[0] ? PP - s : s, t1 = fl[1] ? PP - s : s;
  if (!HDG_INB((int64_t)e[0] * 3 + k[0], 3LL * P.N, P.oob, 16) || !HDG_INB((int64_t)e[1] * 3 + k[1], 3LL * P.N, P.oob, 16) ||
      !HDG_INB(t0, P1, P.oob, 16) || !HDG_INB(t1, P1, P.oob, 16) || !HDG_INB((int64_t)f * P1 + s, P.N_tr, P.oob, 16))
    return;
  double r = 0.0;
#pragma unroll
  for (int sd = 0; sd < 2; ++sd) {
    const size_t blk = (size_t)e[sd] * 3 + k[sd];
    const int t = sd ? t1 : t0;
    const int2* bp = L + blk * nt * P1 + t;
    const int2* xv = xs + (le * 2 + sd) * ntp;
    long long hh = 0, m0 = 0, m1 = 0;
    unsigned long long ll = 0;
    // groups of FIX_G entries, the next group's loads issued before the
    // current group's products (the integer multiply-adds are short next to
    // a load)
    int2 cur[FIX_G], nxt[FIX_G];
#pragma unroll
    for (int u = 0; u < FIX_G; ++u) cur[u] = u < nt ? bp[(size_t)u * P1] : make_int2(0, 0);
    for (int j0 = 0; j0 < nt; j0 += FIX_G) {
#pragma unroll
      for (int u = 0; u < FIX_G; ++u) {
        const int j = j0 + FIX_G + u;
        nxt[u] = j < nt ? bp[(size_t)j * P1] : make_int2(0, 0);
      }
#pragma unroll
      for (int u = 0; u < FIX_G; ++u) {
        const int j = j0 + u;
        if (j < nt) {
          const int2 a = cur[u], b = xv[j];
          hh += (long long)a.y * b.y;
          m0 += (long long)a.y * b.x;
          m1 += (long long)a.x * b.y;
          ll += (unsigned long long)(unsigned)a.x * (unsigned)b.x;
        }
      }
#pragma unroll
      for (int u = 0; u < FIX_G; ++u) cur[u] = nxt[u];
    }
    r += fix_result(hh, m0, m1, ll, rex[blk * P1 + t], xe[le * 2 + sd]);
  }
  if (escale) r *= escale[f];
  y[(size_t)f * P1 + s] = r;
}

size_t apply_fix_smem(const Params& P, int epb) { return fix_tab_offset(epb, P.n_t) + (size_t)epb * 2 * sizeof(int4); }

cudaError_t launch_apply_fix(const Params& P, const void* fix, const double* x, double* y, const double* escale,
                             const int* stop, cudaStream_t st, int epb) {
  if (!fix_supported(P)) return cudaErrorInvalidValue;
  if (epb <= 0 || epb * P.P1 > 512) epb = apply_edges_per_block(P);
  const int2* L = static_cast<const int2*>(fix);
  const int* ex = reinterpret_cast<const int*>(L + (size_t)P.N * 3 * P.n_t * P.P1);
  const int threads = (epb * P.P1 + 31) / 32 * 32;
  const int grid = (P.n_int + epb - 1) / epb;
  apply_fix_kernel<<<grid, threads, apply_fix_smem(P, epb), st>>>(P, L, ex, x, y, escale, epb, stop);
  return cudaGetLastError();
}

cudaError_t launch_fix_convert(const Params& P, const double* S, void* fix, cudaStream_t st) {
  if (!fix_supported(P)) return cudaErrorInvalidValue;
  int2* L = static_cast<int2*>(fix);
  int* ex = reinterpret_cast<int*>(L + (size_t)P.N * 3 * P.n_t * P.P1);
  const int64_t rows = (int64_t)P.N * 3 * P.P1;
  const int grid = (int)std::min<int64_t>(4096, (rows + 255) / 256);
  fix_convert_kernel<<<grid, 256, 0, st>>>(S, L, ex, rows, P.n_t, P.P1);
  return cudaGetLastError();
}

}  // namespace mehdg
