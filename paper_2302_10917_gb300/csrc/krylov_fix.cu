// Fixed-point Krylov basis (HDG_BASIS_FIX): the vector passes of the Arnoldi
// step of Sec. 6.1's GMRES (multi-dot V^T w with ||w||^2, update w - V h and
// the new basis vector, the first vector of a cycle, the solution update
// x + V y) with every product exact in 64-bit integers.
//
// An FP64 basis does one FP64 FMA per 8-byte basis entry in each pass, and
// GB300's FP64 pipe caps that at about 74 % of the HBM bandwidth. Here each
// basis vector is stored in chunks of FXC entries, every chunk as 56-bit
// fixed-point numbers at the scale of its largest entry (int2 limbs, 8 bytes
// per entry, plus one int32 scale per chunk). The multi-dot scales each chunk
// of w the same way inside the kernel and sums the limb products of one
// chunk exactly, rounding once per thread, chunk and vector; the updates scale
// the coefficients h_i 2^(chunk scale of V_i) of one chunk to a common
// fixed-point scale and sum sum_i h_i V_i exactly per entry, rounding once.
// The FP64 work left is per chunk or per entry, not per entry and vector.
// Besides the limbs, the update that writes a new basis vector also writes it
// in FP64 (the operator's input).
//
// Accuracy: storage rounds each entry to 2^-55 of its chunk's largest
// magnitude; sums are exact until one final FP64 rounding; the coefficient
// scaling rounds each h_i 2^s_i to 2^-55 of the largest of them. Accumulator
// bounds: per dot product sum at most 16 terms per thread (a warp's 512 summed
// exactly in 128 bits), per update sum at most 128 terms, inside 2^63
// (|hi| <= 2^27, 0 <= lo < 2^28).
#include "internal.h"
#include "fixpoint.h"
#include <algorithm>

namespace mehdg {

constexpr int FXC = 1024;          // entries per scale chunk of a basis vector
constexpr int FXT = 256;           // threads per block
constexpr int FXE = FXC / FXT;     // entries per thread and chunk
constexpr int FX_VG = 8;           // basis vectors per multi-dot block
constexpr int FX_MAXCOL = 130;     // basis vectors + 1 (restart <= 128)
constexpr int FX_ROWS = 2048;      // most partial rows of a multi-dot (chunks per row beyond that)
constexpr int FX_GRID = 2432;      // most blocks of one combine launch (16 per SM)

int64_t fx_chunks(int64_t n) { return (n + FXC - 1) / FXC; }

// block maximum of one int per thread (all threads call; red holds FXT / 32 ints)
__device__ __forceinline__ int block_max_i(int v, int* red) {
  v = __reduce_max_sync(0xffffffffu, v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  int m = red[0];
  for (int q = 1; q < FXT / 32; ++q) m = max(m, red[q]);
  return m;
}

// part[r * ncol + i] = sum over the chunks c = r, r + gridDim.x, ... of V_i . w for the
// FX_VG columns i = FX_VG blockIdx.y + ... (i < nv; column nv, when ncol = nv + 1, is
// w . w). A block of FXM_T threads covers one chunk, FXM_E entries per thread: the
// block scales the chunk of w to limbs, then per vector every thread sums its
// products exactly, the warp adds its 32 partial sums exactly (128 bits) and its
// lane 0 rounds once; the rounding and the warp sum are spread over FXM_E entries.
constexpr int FXM_T = 64;                 // threads per multi-dot block (one chunk)
constexpr int FXM_E = FXC / FXM_T;        // entries per thread
__global__ void __launch_bounds__(FXM_T, 16) fx_mdot_kernel(const int2* __restrict__ V, const int* __restrict__ Vs,
                                                            int nch, int64_t ldv, int64_t n, int nv, int ncol,
                                                            const double* __restrict__ w, double* part,
                                                            const int* stop) {
  if (stop && stop[0]) return;   // the flag word the caller points at (stop, or second pass not needed)
  constexpr int NW = FXM_T / 32;
  __shared__ double acc[FX_VG][NW];
  __shared__ int red[NW];
  __shared__ int2 wls[FXC];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int g0 = blockIdx.y * FX_VG, g1 = min(ncol, g0 + FX_VG);
  for (int i = threadIdx.x; i < FX_VG * NW; i += FXM_T) (&acc[0][0])[i] = 0.0;
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    const int64_t e0 = (int64_t)c * FXC + threadIdx.x;
    // this thread's limbs of w for the chunk, kept in shared memory (entry-major,
    // thread-minor: conflict-free) to leave the registers to the loads in flight
    int eb = 1;
#pragma unroll
    for (int k = 0; k < FXM_E; ++k) {
      const int64_t e = e0 + k * FXM_T;
      const unsigned long long b = e < n ? (unsigned long long)__double_as_longlong(w[e]) : 0ull;
      wls[k * FXM_T + threadIdx.x] = make_int2((int)(unsigned)b, (int)(unsigned)(b >> 32));   // the bits, for now
      eb = max(eb, fix_exp_field(b));
    }
    eb = __reduce_max_sync(0xffffffffu, eb);
    __syncthreads();
    if (lane == 0) red[wid] = eb;
    __syncthreads();
    int Ew = red[0];
#pragma unroll
    for (int q = 1; q < NW; ++q) Ew = max(Ew, red[q]);
#pragma unroll
    for (int k = 0; k < FXM_E; ++k) {
      const int2 b = wls[k * FXM_T + threadIdx.x];
      wls[k * FXM_T + threadIdx.x] = fix_limbs(((unsigned long long)(unsigned)b.y << 32) | (unsigned)b.x, Ew);
    }
    // (16 loads of a vector in flight per thread; column nv is w itself)
    for (int i = g0; i < g1; ++i) {
      long long hh = 0, m0 = 0, m1 = 0;
      unsigned long long ll = 0;
      if (i < nv) {
        const int2* vp = V + (size_t)i * ldv;
        int2 v[FXM_E];
#pragma unroll
        for (int k = 0; k < FXM_E; ++k) {
          const int64_t e = e0 + k * FXM_T;
          v[k] = e < n ? vp[e] : make_int2(0, 0);
        }
#pragma unroll
        for (int k = 0; k < FXM_E; ++k) fix_mac(hh, m0, m1, ll, v[k], wls[k * FXM_T + threadIdx.x]);
      } else {
#pragma unroll
        for (int k = 0; k < FXM_E; ++k) {
          const int2 b = wls[k * FXM_T + threadIdx.x];
          fix_mac(hh, m0, m1, ll, b, b);
        }
      }
      // the warp's products share one scale: summed exactly across the warp (|sum| < 2^120),
      // rounded once by lane 0
      __int128 t = fix_sum128(hh, m0, m1, ll);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const long long th = __shfl_down_sync(0xffffffffu, (long long)(t >> 64), off);
        const unsigned long long tl = __shfl_down_sync(0xffffffffu, (unsigned long long)t, off);
        t += ((__int128)th << 64) | (__int128)tl;
      }
      if (lane == 0) {
        const int Ev = i < nv ? Vs[(size_t)i * nch + c] : Ew;
        acc[i - g0][wid] += (Ev == 2047 || Ew == 2047) ? __longlong_as_double(0x7FF8000000000000ll)
                                                       : fix_round(t, Ev + Ew - 2154);
      }
    }
  }
  __syncthreads();
  for (int i = g0 + (int)threadIdx.x; i < g1; i += FXM_T) {
    double s = 0.0;
    for (int q = 0; q < NW; ++q) s += acc[i - g0][q];
    part[(size_t)blockIdx.x * ncol + i] = s;
  }
}

// val = (bcoef base + csign sum_{i < nv} coef_i V_i) * scale per entry (scale =
// sm[scale_off], or 1 when scale_off < 0), written in FP64 to out_d (may be
// base) and, when out_l is given, as a new basis vector: limbs out_l, chunk
// scales out_s.
__global__ void __launch_bounds__(FXT, 4) fx_combine_kernel(const int2* __restrict__ V, const int* __restrict__ Vs,
                                                         int nch, int64_t ldv, int64_t n, int nv,
                                                         const double* __restrict__ coef, double csign,
                                                         const double* base, double bcoef, const double* sm,
                                                         int scale_off, double* out_d, int2* out_l, int* out_s,
                                                         const int* stop) {
  if (stop && stop[0]) return;
  __shared__ int2 af[FX_MAXCOL];
  __shared__ int red[FXT / 32];
  const double scale = scale_off >= 0 ? sm[scale_off] : 1.0;
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    const int64_t e0 = (int64_t)c * FXC + threadIdx.x;
    // this chunk's coefficients a_i = coef_i 2^(s_i - 1077) at one fixed-point scale Ea
    unsigned long long ab = 0ull;
    int ea = 1;
    if ((int)threadIdx.x < nv) {
      const double a = fix_ldexp(coef[threadIdx.x], Vs[(size_t)threadIdx.x * nch + c] - 1077);
      ab = (unsigned long long)__double_as_longlong(a);
      ea = fix_exp_field(ab);
    }
    const int Ea = block_max_i(ea, red);
    if ((int)threadIdx.x < nv) af[threadIdx.x] = fix_limbs(ab, Ea);
    __syncthreads();
    double val[FXE];
    {
      long long hh[FXE], m0[FXE], m1[FXE];
      unsigned long long ll[FXE];
#pragma unroll
      for (int q = 0; q < FXE; ++q) hh[q] = m0[q] = m1[q] = 0, ll[q] = 0ull;
      // limbs of vectors i + 1 and i + 2 in flight while vector i's products run
      int2 v0[FXE], v1[FXE], v2[FXE];
      auto load = [&](int2 (&v)[FXE], int i) {
        const int2* vp = V + (size_t)i * ldv;
#pragma unroll
        for (int q = 0; q < FXE; ++q) {
          const int64_t e = e0 + q * FXT;
          v[q] = (i < nv && e < n) ? vp[e] : make_int2(0, 0);
        }
      };
      load(v0, 0);
      load(v1, 1);
      for (int i = 0; i < nv; ++i) {
        load(v2, i + 2);
        const int2 a = af[i];
#pragma unroll
        for (int q = 0; q < FXE; ++q) fix_mac(hh[q], m0[q], m1[q], ll[q], v0[q], a);
#pragma unroll
        for (int q = 0; q < FXE; ++q) {
          v0[q] = v1[q];
          v1[q] = v2[q];
        }
      }
#pragma unroll
      for (int q = 0; q < FXE; ++q) {
        const int64_t e = e0 + q * FXT;
        const double s = nv > 0 ? fix_result(hh[q], m0[q], m1[q], ll[q], Ea, 1077) : 0.0;
        const double b = (e < n && bcoef != 0.0) ? bcoef * base[e] : 0.0;
        val[q] = e < n ? (b + csign * s) * scale : 0.0;
      }
    }
    if (out_l) {
      int eo = 1;
#pragma unroll
      for (int k = 0; k < FXE; ++k) eo = max(eo, fix_exp_field((unsigned long long)__double_as_longlong(val[k])));
      const int Eo = block_max_i(eo, red);
#pragma unroll
      for (int k = 0; k < FXE; ++k) {
        const int64_t e = e0 + k * FXT;
        if (e < n) out_l[e] = fix_limbs((unsigned long long)__double_as_longlong(val[k]), Eo);
      }
      if (threadIdx.x == 0) out_s[c] = Eo;
    }
    if (out_d) {
#pragma unroll
      for (int k = 0; k < FXE; ++k) {
        const int64_t e = e0 + k * FXT;
        if (e < n) out_d[e] = val[k];
      }
    }
    __syncthreads();   // af and red are rewritten for the next chunk
  }
}

int launch_fx_mdot(const void* V, const int* Vs, int64_t ldv, int64_t n, int nv, int ncol, const double* w,
                   double* part, const int* stop, cudaStream_t st) {
  const int nch = (int)fx_chunks(n);
  const int gx = std::max(1, std::min(nch, FX_ROWS));
  const dim3 grid((unsigned)gx, (unsigned)((ncol + FX_VG - 1) / FX_VG));
  fx_mdot_kernel<<<grid, FXM_T, 0, st>>>(static_cast<const int2*>(V), Vs, nch, ldv, n, nv, ncol, w, part, stop);
  return gx;
}

void launch_fx_combine(const void* V, const int* Vs, int64_t ldv, int64_t n, int nv, const double* coef, double csign,
                       const double* base, double bcoef, const double* sm, int scale_off, double* out_d, void* out_l,
                       int* out_s, const int* stop, cudaStream_t st) {
  const int nch = (int)fx_chunks(n);
  const int gx = std::max(1, std::min(nch, FX_GRID));
  fx_combine_kernel<<<gx, FXT, 0, st>>>(static_cast<const int2*>(V), Vs, nch, ldv, n, nv, coef, csign, base, bcoef, sm,
                                        scale_off, out_d, static_cast<int2*>(out_l), out_s, stop);
}

}  // namespace mehdg
