// Batched static condensation of every macro-element (Eqs. global_problem and
// local_problem; block system Eq. D; element formation Sec. 6.1; LU remark of
// Sec. 3.3.2). One CTA per macro-element.
//
// Each CTA forms its element's bordered system in FP64
//
//          [ A_u  B_u  F ]     rows 0 .. Q-1      : u-equations after eliminating q
//      W = [ C_u  D_u  0 ]     rows Q .. Q+n_t-1  : trace equations
//
// where (q eliminated exactly through q_x = M^-1 (Dx u - Fx u^), q_y alike)
//   A_u = kappa (Dx^T M^-1 Dx + Dy^T M^-1 Dy) - (beta_x Dx + beta_y Dy) + tau E
//   B_u = Fa - tau F - kappa (Dx^T M^-1 Fx + Dy^T M^-1 Fy)
//   C_u = kappa (Fx^T M^-1 Dx + Fy^T M^-1 Dy) + tau F^T
//   D_u = Ga - tau G - kappa (Fx^T M^-1 Fx + Fy^T M^-1 Fy)
// and eliminates the first Q columns with partial pivoting restricted to the
// u-rows (blocked right-looking LU, panel width NB). The trailing block then
// holds [S_e | -C A^-1 R] with S_e = D_e - C_e A_e^-1 B_e, and rows 0..Q-1
// hold U, L^-1 P B_u and L^-1 P F for the back-solve.
//
// condense_df_kernel (split_update) does the same elimination with the system
// in split-FP32 form (hi, lo FP32 pairs, 48-bit significand, the same 8 bytes
// per entry) from its formation to the end of the elimination: formation from
// split copies of the tables, pivot search on the high words, panel
// factorisation, triangular solves and trailing updates with error-free
// transformations, all on the FP32 pipe. A last pass converts the system to
// FP64 in place, so that every reader sees FP64 entries.
#include "internal.h"
#include "df64.h"

namespace mehdg {

constexpr int NB = 16;        // panel width
constexpr int LDP = NB + 1;   // padded panel row stride (bank spread for column scans)
constexpr int RT = 8;         // rows per trailing-update work item

struct CondArgs {
  Params prm;
  DevTables dt;
  const double* kappa;
  const double* f_qp;
  const double* ghat;
  double* ws;
  int64_t e0;
  int slot_is_element;    // 1: workspace slot = element id; 0: slot = blockIdx.x
  int write_outputs;
  double* S;
  double* St;
  float* St32;
  double* gel;
  int* info;
  int split_update;       // 1: condense_df_kernel (split-FP32 elimination on the FP32 pipe),
                          // 2: condense_tc_kernel (FP64 panels, trailing updates on the tensor cores)
  int* piv;               // [N][Q] pivot row of every column (factors kept), or null
  // one refinement level of a level mesh: the launch covers slots e0.. of the
  // element list elist (outputs, workspace, info and pivots by slot; geometry,
  // kappa, sources and Dirichlet data by element id), nslots slots in all
  const int* elist;       // null: slot = element id
  int64_t nslots;         // slots of the outputs (N without a list)
  const int64_t* qoff;    // first source point of every element, or null (e n_qp)
  int64_t fstride;        // source values per right-hand side (N n_qp without qoff)
};

__device__ void condense_outputs(const CondArgs& a, const double* W, int e, int eb);
static cudaError_t launch_condense_args(CondArgs& a, int64_t count, cudaStream_t st);

// The load columns of element e, one source at a time: per sub-triangle
// projections of f_r (FP64, in proj: nsub * nloc doubles of shared memory)
// summed over the sub-triangles that share a lattice node, times
// detJ / m^2; put(i, r, value) stores row i of column r. Block-wide; ends
// with a barrier.
template <typename Put>
__device__ void load_columns(const CondArgs& a, int e, double detJ, double* proj, Put put, double ts = 0.0,
                             double bxi = 0.0, double beta_ = 0.0) {
  const Params& P = a.prm;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const double scale = detJ / (double)(P.m * P.m);
  for (int r = 0; r < P.nrhs; ++r) {
    const double* fe = a.f_qp + (size_t)r * a.fstride + (a.qoff ? a.qoff[e] : (int64_t)e * P.n_qp);
    for (int idx = tid; idx < P.nsub * P.nloc; idx += nthr) {
      const int s = idx / P.nloc, b = idx - s * P.nloc;
      double acc = 0.0;
      if (P.supg) {
        // SUPG load: (f, phi_b + tau_s a . grad phi_b) on the sub-triangle
        for (int q = 0; q < P.nqs; ++q) {
          const double* dg = a.dt.dphq + (((size_t)s * P.nqs + q) * P.nloc + b) * 2;
          acc += a.dt.wq[q] * fe[s * P.nqs + q] * (a.dt.phiq[q * P.nloc + b] + ts * (bxi * dg[0] + beta_ * dg[1]));
        }
      } else {
        for (int q = 0; q < P.nqs; ++q) acc += a.dt.wq[q] * fe[s * P.nqs + q] * a.dt.phiq[q * P.nloc + b];
      }
      proj[idx] = acc;
    }
    __syncthreads();
    for (int i = tid; i < P.Q; i += nthr) {
      double acc = 0.0;
      for (int q = a.dt.ns_ptr[i]; q < a.dt.ns_ptr[i + 1]; ++q) acc += proj[a.dt.ns_idx[q]];
      put(i, r, acc * scale);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void warp_argmax(double& v, int& i) {
  for (int off = 16; off > 0; off >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, v, off);
    const int oi = __shfl_down_sync(0xffffffffu, i, off);
    if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
  }
}

// Forms element e's bordered system in W (rows R, leading dimension ld; FP64):
// [A_u B_u F; C_u D_u 0] from the reference tables and the element's geometry,
// kappa, tau and source (the load columns use proj as shared scratch). Block-wide;
// ends with a barrier.
__device__ void form_system(const CondArgs& a, int e, double* W, double* proj) {
  const Params& P = a.prm;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int Q = P.Q, nt = P.n_t, P1 = P.P1, R = P.R, ld = P.ld;
  // ---------------------------------------------------------- element data
  ElemGeom g;
  elem_geom(e, P.n, g);
  const double kap = a.kappa[e];
  const double tau = kap / P.tau_len + P.babs;
  const double gxx = g.gxi[0] * g.gxi[0] + g.gxi[1] * g.gxi[1];
  const double gxy = g.gxi[0] * g.geta[0] + g.gxi[1] * g.geta[1];
  const double gyy = g.geta[0] * g.geta[0] + g.geta[1] * g.geta[1];
  const double bxi = P.bx * g.gxi[0] + P.by * g.gxi[1];
  const double beta_ = P.bx * g.geta[0] + P.by * g.geta[1];
  double nxi[3], neta[3], bn[3];
  for (int k = 0; k < 3; ++k) {
    nxi[k] = g.nrm[k][0] * g.gxi[0] + g.nrm[k][1] * g.gxi[1];
    neta[k] = g.nrm[k][0] * g.geta[0] + g.nrm[k][1] * g.geta[1];
    bn[k] = P.bx * g.nrm[k][0] + P.by * g.nrm[k][1];
  }
  const double cK = kap * g.detJ;
  // SUPG (Sec. 3.4): tau_s detJ [(a.grad)^2 products - kappa (a.grad)(Lap) products]
  const double ts = P.supg ? supg_tau(fmax(g.L[0], fmax(g.L[1], g.L[2])) / P.m, P.babs, kap) : 0.0;
  double cs[9];
  {
    const double bs = ts * g.detJ;
    cs[0] = bs * bxi * bxi; cs[1] = bs * bxi * beta_; cs[2] = bs * beta_ * beta_;
    cs[3] = -bs * kap * bxi * gxx; cs[4] = -bs * kap * bxi * 2.0 * gxy; cs[5] = -bs * kap * bxi * gyy;
    cs[6] = -bs * kap * beta_ * gxx; cs[7] = -bs * kap * beta_ * 2.0 * gxy; cs[8] = -bs * kap * beta_ * gyy;
  }


  // --------------------------------------------------- form the bordered system
  for (int i = 0; i < R; ++i) {
    double* row = W + (size_t)i * ld;
    if (i < Q) {
      const size_t qi = (size_t)i * Q;
      for (int j = tid; j < ld; j += nthr) {
        double v;
        if (j < Q) {
          v = cK * (gxx * a.dt.Kxx[qi + j] + gxy * a.dt.Ksym[qi + j] + gyy * a.dt.Kyy[qi + j])
              - g.detJ * (bxi * a.dt.Dxi[qi + j] + beta_ * a.dt.Deta[qi + j]);
          if (P.supg) {
            const size_t ij = qi + j;
            v += cs[0] * a.dt.Sxx[ij] + cs[1] * a.dt.Ssym[ij] + cs[2] * a.dt.Syy[ij] + cs[3] * a.dt.Lx_xx[ij] +
                 cs[4] * a.dt.Lx_xy[ij] + cs[5] * a.dt.Lx_yy[ij] + cs[6] * a.dt.Ly_xx[ij] + cs[7] * a.dt.Ly_xy[ij] +
                 cs[8] * a.dt.Ly_yy[ij];
          }
        } else if (j < Q + nt) {
          const int c = j - Q, k = c / P1;
          const size_t ic = (size_t)i * nt + c;
          v = g.L[k] * ((bn[k] - tau) * a.dt.Fh[ic] - kap * (nxi[k] * a.dt.Pxi[ic] + neta[k] * a.dt.Peta[ic]));
        } else {
          v = 0.0;   // load columns: formed below
        }
        row[j] = v;
      }
    } else {
      const int r = i - Q, k = r / P1, t = r - k * P1;
      for (int j = tid; j < ld; j += nthr) {
        double v;
        if (j < Q) {
          const size_t jr = (size_t)j * nt + r;
          v = g.L[k] * (kap * (nxi[k] * a.dt.Pxi[jr] + neta[k] * a.dt.Peta[jr]) + tau * a.dt.Fh[jr]);
        } else if (j < Q + nt) {
          const int c = j - Q, l = c / P1, t2 = c - l * P1;
          const double nn = g.nrm[k][0] * g.nrm[l][0] + g.nrm[k][1] * g.nrm[l][1];
          v = -kap * g.L[k] * g.L[l] * nn / g.detJ * a.dt.Hh[(size_t)r * nt + c];
          if (l == k) v += g.L[k] * (bn[k] - tau) * a.dt.Gh[t * P1 + t2];
        } else {
          v = 0.0;
        }
        row[j] = v;
      }
    }
  }
  __syncthreads();
  // load columns Q + n_t + r: per sub-triangle projections of source r (in
  // the panel area, free before the LU starts), summed per lattice node
  load_columns(a, e, g.detJ, proj, [&](int i, int r, double v) { W[(size_t)i * ld + Q + nt + r] = v; }, ts, bxi,
               beta_);
  // tau E: E = sum_k L_k Pi_k^T Gh Pi_k (edge by edge: corner nodes are shared)
  for (int k = 0; k < 3; ++k) {
    for (int idx = tid; idx < P1 * P1; idx += nthr) {
      const int t = idx / P1, t2 = idx - t * P1;
      const int ni = a.dt.enode[k * P1 + t], nj = a.dt.enode[k * P1 + t2];
      W[(size_t)ni * ld + nj] += tau * g.L[k] * a.dt.Gh[idx];
    }
    __syncthreads();
  }

}

// One panel of the bordered LU (columns j0 .. j0 + nb - 1, nb = min(NBW, Q - j0)):
// the panel rows j0 .. R - 1 in shared memory (Ls, row stride NBW + 1), partial
// pivoting over the u-rows, the factored panel written back to W, then the row
// interchanges and U12 = L11^-1 A12 on the columns right of the panel (one column
// per thread; also kept in Us, row stride ld, when KEEP_U). Returns nb; ends with a
// barrier when columns remain right of the panel.
template <int NBW, bool KEEP_U>
__device__ int factor_panel(const CondArgs& a, double* W, double* Ls, double* Us, int j0, int eb, int* piv_s,
                            double* red_v, int* red_i, int& singular_col) {
  const Params& P = a.prm;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int Q = P.Q, R = P.R, Cc = P.Cc, ld = P.ld;
  constexpr int LDPW = NBW + 1;
  const int nb = min(NBW, Q - j0);
  const int rows = R - j0;
  for (int idx = tid; idx < rows * NBW; idx += nthr) {
    const int r = idx / NBW, c = idx - r * NBW;
    Ls[r * LDPW + c] = (c < nb) ? W[(size_t)(j0 + r) * ld + j0 + c] : 0.0;
  }
  __syncthreads();
  for (int c = 0; c < nb; ++c) {
    // pivot: largest |a| among u-rows j0+c .. Q-1 (first one on ties)
    double best = -1.0;
    int bi = c;
    for (int r = c + tid; r < Q - j0; r += nthr) {
      const double v = fabs(Ls[r * LDPW + c]);
      if (v > best) { best = v; bi = r; }
    }
    warp_argmax(best, bi);
    if ((tid & 31) == 0) { red_v[tid >> 5] = best; red_i[tid >> 5] = bi; }
    __syncthreads();
    if (tid < 32) {
      const int nw = nthr >> 5;
      double v = tid < nw ? red_v[tid] : -1.0;
      int ii = tid < nw ? red_i[tid] : 0x7fffffff;
      warp_argmax(v, ii);
      if (tid == 0) piv_s[c] = ii;
    }
    __syncthreads();
    const int pr = piv_s[c];
    if (a.piv) {
      // kept factors: record the interchange and apply it to the columns of
      // the earlier panels too, so that rows 0..Q-1 hold P A_u = L U
      if (tid == 0) a.piv[(size_t)eb * Q + j0 + c] = j0 + pr;
      if (pr != c)
        for (int cc = tid; cc < j0; cc += nthr) {
          double* x0 = W + (size_t)(j0 + c) * ld + cc;
          double* x1 = W + (size_t)(j0 + pr) * ld + cc;
          const double t0 = *x0;
          *x0 = *x1;
          *x1 = t0;
        }
    }
    if (pr != c) {
      for (int cc = tid; cc < nb; cc += nthr) {
        const double t0 = Ls[c * LDPW + cc];
        Ls[c * LDPW + cc] = Ls[pr * LDPW + cc];
        Ls[pr * LDPW + cc] = t0;
      }
      __syncthreads();
    }
    const double d = Ls[c * LDPW + c];
    if (d == 0.0 && singular_col < 0) singular_col = j0 + c;
    const double inv = (d != 0.0) ? 1.0 / d : 0.0;
    for (int r = c + 1 + tid; r < rows; r += nthr) Ls[r * LDPW + c] *= inv;
    __syncthreads();
    const int nrem = nb - c - 1;
    if (nrem > 0) {
      const int nr = rows - c - 1;
      for (int idx = tid; idx < nr * nrem; idx += nthr) {
        const int r = c + 1 + idx / nrem, cc = c + 1 + idx % nrem;
        Ls[r * LDPW + cc] -= Ls[r * LDPW + c] * Ls[c * LDPW + cc];
      }
      __syncthreads();
    }
  }
  for (int idx = tid; idx < rows * nb; idx += nthr) {
    const int r = idx / nb, c = idx - r * nb;
    W[(size_t)(j0 + r) * ld + j0 + c] = Ls[r * LDPW + c];
  }
  const int jb = j0 + nb, ncol = Cc - jb;
  if (ncol > 0) {
    // row interchanges and U12 = L11^-1 A12, one column per thread
    for (int j = jb + tid; j < Cc; j += nthr) {
      double u[NBW];
      for (int c = 0; c < nb; ++c) {
        const int pr = piv_s[c];
        if (pr != c) {
          double* x0 = W + (size_t)(j0 + c) * ld + j;
          double* x1 = W + (size_t)(j0 + pr) * ld + j;
          const double t0 = *x0;
          *x0 = *x1;
          *x1 = t0;
        }
      }
#pragma unroll
      for (int c = 0; c < NBW; ++c) u[c] = (c < nb) ? W[(size_t)(j0 + c) * ld + j] : 0.0;
#pragma unroll
      for (int c = 1; c < NBW; ++c) {
        if (c < nb) {
          double s = u[c];
#pragma unroll
          for (int t = 0; t < c; ++t) s -= Ls[c * LDPW + t] * u[t];
          u[c] = s;
        }
      }
      for (int c = 0; c < nb; ++c) {
        W[(size_t)(j0 + c) * ld + j] = u[c];
        if (KEEP_U) Us[c * ld + j] = u[c];
      }
    }
    __syncthreads();
  }
  return nb;
}

__global__ void __launch_bounds__(256) condense_kernel(CondArgs a) {
  const Params& P = a.prm;
  const int eb = (int)(a.e0 + blockIdx.x);
  if (eb >= a.nslots) return;
  const int e = a.elist ? a.elist[eb] : eb;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int Q = P.Q, R = P.R, Cc = P.Cc, ld = P.ld;
  double* W = a.ws + (size_t)(a.slot_is_element ? eb : blockIdx.x) * (size_t)R * ld;

  extern __shared__ double smem[];
  double* Ls = smem;                       // [R][LDP]
  double* Us = smem + (size_t)R * LDP;     // [NB][ld]
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ int piv_s[NB];

  form_system(a, e, W, Ls);

  // ------------------------------------------------------- blocked LU, Q pivots
  int singular_col = -1;
  for (int j0 = 0; j0 < Q; j0 += NB) {
    const int nb = factor_panel<NB, true>(a, W, Ls, Us, j0, eb, piv_s, red_v, red_i, singular_col);
    const int jb = j0 + nb, ncol = Cc - jb;
    if (ncol > 0) {
      // trailing update A22 -= L21 U12 (rows jb..R-1, columns jb..Cc-1)
      const int nrow = R - jb;
      const int ntile = (nrow + RT - 1) / RT;
      for (int item = tid; item < ntile * ncol; item += nthr) {
        const int rt = item / ncol, j = jb + (item - rt * ncol);
        double u[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c) u[c] = (c < nb) ? Us[c * ld + j] : 0.0;
        const int r0 = jb + rt * RT;
        const int nr = min(RT, R - r0);
        // the tile's rows as RT independent FMA chains (each row keeps its order c = 0 .. NB-1):
        // one chain per thread left the FP64 pipe waiting on DFMA results
        double acc[RT];
#pragma unroll
        for (int rr = 0; rr < RT; ++rr) acc[rr] = rr < nr ? W[(size_t)(r0 + rr) * ld + j] : 0.0;
        const double* l = Ls + (r0 - j0) * LDP;
#pragma unroll
        for (int c = 0; c < NB; ++c)
#pragma unroll
          for (int rr = 0; rr < RT; ++rr) acc[rr] -= l[(rr < nr ? rr : 0) * LDP + c] * u[c];
#pragma unroll
        for (int rr = 0; rr < RT; ++rr)
          if (rr < nr) W[(size_t)(r0 + rr) * ld + j] = acc[rr];
      }
    }
    __syncthreads();
  }
  if (tid == 0 && a.info) a.info[eb] = singular_col >= 0 ? singular_col + 1 : 0;
  if (a.write_outputs) condense_outputs(a, W, e, eb);
}

// S_e, its preconditioned copies and the element right-hand side from the
// factored bordered system (FP64 entries).
// ------------------------------------------------ tensor-core trailing updates
// condense_tc_kernel eliminates with 32-column panels: pivot search, panel LU
// and U12 = L11^-1 A12 in FP64 as above, and the trailing update
// A22 -= L21 U12 on the tensor cores, FP64-accurate through exact slices
// (Ozaki's splitting of floating-point matrix products into error-free partial
// products, carried out here with integer bit operations):
//  * every row r of L21 is scaled by 2^-e_r (2^e_r above the row's largest
//    magnitude), every column c of U12 by 2^-f_c, and each scaled entry, a
//    fixed-point number below 1, is cut into 7 slices of 8 bits,
//    x = sum_i s_i 2^-8(i+1) + (less than 2^-56), |s_i| <= 255 (bf16-exact);
//  * the slice products with i + j = t are summed into one FP32 accumulator per
//    level t = 0..6 in tensor memory (tcgen05.mma kind::f16, M = 128, N = 32,
//    K = 16): products below 2^16, K = 32 of them per pair, at most 7 pairs,
//    so every level sum is an integer below 2^24 and exact;
//  * the levels are combined as 2^(e_r + f_c - 16) (A_0 + 2^-8 A_1 + 2^-16 A_2
//    + 2^-24 A_3 + 2^-32 (A_4 + 2^-8 A_5 + 2^-16 A_6)), the first four terms
//    exactly in FP64, the last three in FP32, and subtracted from A22 in FP64.
// The dropped parts (slice truncation, levels above 6, the FP32 tail) are below
// 2^-50 of 2^(e_r + f_c) per entry, under the FP64 rounding bound of a 32-term
// dot product. FP64 work per trailing entry and panel: 5 FMAs instead of 32.
constexpr int TCB = 32;                   // panel width = K of the slice products
constexpr int TC_SLICES = 7;
constexpr int TC_LEVELS = 7;              // t = i + j <= 6
constexpr int TC_M = 128, TC_N = 32;      // row tile (MMA M) and column tile (MMA N)
constexpr int TC_TMEM_COLS = 256;         // 7 levels x 32 columns, rounded to a power of two
constexpr int TC_EXP_NONE = -4000;        // a row or column without a normal entry
constexpr long long TC_WAIT_CYCLES = 2000000000LL;
constexpr size_t TC_A_BYTES = (size_t)TC_SLICES * TC_M * TCB * 2;
constexpr size_t TC_B_BYTES = (size_t)TC_SLICES * TC_N * TCB * 2;

size_t condense_tc_smem_bytes(const Params& P) {
  const size_t panel = (size_t)P.R * (TCB + 1) * sizeof(double);
  const size_t slices = TC_A_BYTES + TC_B_BYTES;
  return panel > slices ? panel : slices;
}

namespace {
__device__ __forceinline__ uint32_t tc_smem(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// element offset of (row, k) in a K-major slice plane without swizzle: 8-row x
// 16-byte core matrices, K-adjacent core matrices 128 bytes apart, 8-row groups
// 4 x 128 bytes apart (K = 32)
__device__ __forceinline__ int tc_kmaj(int row, int k) {
  return (((row >> 3) * (TCB / 8) + (k >> 3)) << 6) + ((row & 7) << 3) + (k & 7);
}

// shared-memory matrix descriptor (no swizzle): start, leading (K) and stride (8-row) byte offsets
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | ((uint64_t)1 << 46);
}

// 2^e above |x|max for a row or column (TC_EXP_NONE without a normal entry)
__device__ __forceinline__ int tc_exp_above(double mx) {
  const int E = (int)((__double_as_longlong(mx) >> 52) & 0x7FF);
  return E == 0 ? TC_EXP_NONE : E - 1023 + 1;
}

// bf16 bits of sign * n for an integer 0 <= n <= 255 (exact)
__device__ __forceinline__ uint16_t tc_bf16_int(uint32_t n, uint32_t sgn) {
  if (n == 0) return 0;
  const int p = 31 - __clz(n);
  return (uint16_t)((sgn << 15) | ((uint32_t)(127 + p) << 7) | ((n << (7 - p)) & 0x7Fu));
}

// the 7 slices of v 2^-e (|v| < 2^e) into planes dst[i * plane]
__device__ __forceinline__ void tc_slice(double v, int e, uint16_t* dst, int plane) {
  uint64_t F = 0;
  uint32_t sgn = 0;
  if (e != TC_EXP_NONE) {
    const uint64_t b = (uint64_t)__double_as_longlong(v);
    const int E = (int)((b >> 52) & 0x7FF);
    sgn = (uint32_t)(b >> 63);
    if (E != 0) {
      const uint64_t M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
      const int sh = (E - 1023) + 4 - e;   // F = |v| 2^(56 - e) = M 2^sh, sh <= 3
      F = sh >= 0 ? (M << sh) : (-sh < 64 ? (M >> -sh) : 0ull);
    }
  }
#pragma unroll
  for (int i = 0; i < TC_SLICES; ++i) dst[i * plane] = tc_bf16_int((uint32_t)(F >> (48 - 8 * i)) & 0xFFu, sgn);
}

// exact FP64 value of an FP32 integer below 2^24 (bit conversion on the integer pipe)
__device__ __forceinline__ double tc_f2d(float x) {
  const uint32_t b = __float_as_uint(x);
  if ((b & 0x7FFFFFFFu) == 0) return 0.0;
  const uint64_t r = ((uint64_t)(b >> 31) << 63) | ((uint64_t)(((b >> 23) & 0xFFu) + 896u) << 52) |
                     ((uint64_t)(b & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)r);
}

// FP64 value of any FP32 number by bit conversion (normal numbers exactly; zero and FP32
// subnormals, below 2^-126, give 0)
__device__ __forceinline__ double tc_f2d_any(float x) {
  const uint32_t b = __float_as_uint(x);
  if ((b & 0x7F800000u) == 0) return 0.0;
  const uint64_t r = ((uint64_t)(b >> 31) << 63) | ((uint64_t)(((b >> 23) & 0xFFu) + 896u) << 52) |
                     ((uint64_t)(b & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)r);
}

// 2^E as a double
__device__ __forceinline__ double tc_pow2(int E) {
  if (E >= -1022 && E <= 1023) return __longlong_as_double((long long)((uint64_t)(E + 1023) << 52));
  return scalbn(1.0, E);
}

__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > TC_WAIT_CYCLES) return false;
  }
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
}  // namespace

// A22 -= L21 U12 for the panel j0 .. j0 + nb - 1 on the tensor cores: 128-row
// tiles (A slices made once per tile) times 32-column tiles (B slices per
// tile), 28 slice products of K = 32 (56 MMAs of K = 16) into 7 level
// accumulators, then the FP64 epilogue (8 warps: TMEM lane quarter w % 4,
// column half w / 4). Returns false if the MMAs did not complete within the
// bounded wait (the caller then stops).
__device__ bool tc_trailing_update(const CondArgs& a, double* W, int j0, int nb, uint16_t* As, uint16_t* Bs,
                                   int* er_s, int* ec_s, uint32_t tmem, uint64_t* mbar, uint32_t& phase,
                                   int* s_fail) {
  const Params& P = a.prm;
  const int R = P.R, Cc = P.Cc, ld = P.ld, jb = j0 + nb;
  const int tid = threadIdx.x, nthr = blockDim.x, warp = tid >> 5, lane = tid & 31;
  // kind::f16 instruction descriptor: D FP32, A and B bf16, both K-major, N = 32, M = 128
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                         ((uint32_t)(TC_M >> 4) << 24);
  constexpr int APL = TC_M * TCB, BPL = TC_N * TCB;   // elements per slice plane
  for (int r0 = jb; r0 < R; r0 += TC_M) {
    const int mr = min(TC_M, R - r0);
    if (tid < TC_M) {
      double mx = 0.0;
      if (tid < mr)
        for (int c = 0; c < nb; ++c) mx = fmax(mx, fabs(W[(size_t)(r0 + tid) * ld + j0 + c]));
      er_s[tid] = tid < mr ? tc_exp_above(mx) : TC_EXP_NONE;
    }
    __syncthreads();
    for (int idx = tid; idx < TC_M * TCB; idx += nthr) {
      const int i = idx / TCB, k = idx - i * TCB;
      const double v = (i < mr && k < nb) ? W[(size_t)(r0 + i) * ld + j0 + k] : 0.0;
      tc_slice(v, er_s[i], As + tc_kmaj(i, k), APL);
    }
    for (int c0 = jb; c0 < Cc; c0 += TC_N) {
      const int nc = min(TC_N, Cc - c0);
      if (tid < TC_N) {
        double mx = 0.0;
        if (tid < nc)
          for (int k = 0; k < nb; ++k) mx = fmax(mx, fabs(W[(size_t)(j0 + k) * ld + c0 + tid]));
        ec_s[tid] = tid < nc ? tc_exp_above(mx) : TC_EXP_NONE;
      }
      __syncthreads();
      for (int idx = tid; idx < TC_N * TCB; idx += nthr) {
        const int j = idx / TCB, k = idx - j * TCB;
        const double v = (j < nc && k < nb) ? W[(size_t)(j0 + k) * ld + c0 + j] : 0.0;
        tc_slice(v, ec_s[j], Bs + tc_kmaj(j, k), BPL);
      }
      // the slices (generic-proxy stores) become visible to the tensor cores' async proxy
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (tid == 0) {
        const uint32_t a0 = tc_smem(As), b0 = tc_smem(Bs);
#pragma unroll 1
        for (int t = 0; t < TC_LEVELS; ++t)
#pragma unroll 1
          for (int i = 0; i <= t; ++i) {
            const int j = t - i;
#pragma unroll
            for (int h = 0; h < 2; ++h) {   // K = 32 as two K = 16 halves (two core matrices each)
              const uint64_t ad = tc_desc(a0 + (uint32_t)(i * APL * 2 + h * 256), 128, 4 * 128);
              const uint64_t bd = tc_desc(b0 + (uint32_t)(j * BPL * 2 + h * 256), 128, 4 * 128);
              tc_mma(tmem + (uint32_t)(t * TC_N), ad, bd, idesc, (i > 0 || h > 0) ? 1u : 0u);
            }
          }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         tc_smem(mbar))
                     : "memory");
      }
      // this thread's 16 entries of A22 (row i of the tile, column half hh), loaded while the MMAs run
      const int g = warp & 3, hh = warp >> 2;
      const int i = g * 32 + lane;
      const bool row_live = i < mr && er_s[i] != TC_EXP_NONE;
      double* row = W + (size_t)(r0 + (i < mr ? i : 0)) * ld + c0 + hh * 16;
      const int ncq = max(0, min(16, nc - hh * 16));   // live columns of this half
      double wv[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) wv[q] = (row_live && q < ncq) ? row[q] : 0.0;
      const bool ok = tc_wait(tc_smem(mbar), phase);
      phase ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (!ok) atomicExch(s_fail, 1);
      __syncthreads();
      if (*s_fail) return false;
      // epilogue: levels 6..4 in FP32, 3..0 exactly in FP64 (every lane loads: tcgen05.ld is warp-wide)
      const uint32_t tl = tmem + ((uint32_t)(g * 32) << 16) + (uint32_t)(hh * 16);
      float lv[16], tail[16];
      tc_ld16(tl + 6 * TC_N, tail);
      tc_ld16(tl + 5 * TC_N, lv);
#pragma unroll
      for (int q = 0; q < 16; ++q) tail[q] = fmaf(tail[q], 0.00390625f, lv[q]);
      tc_ld16(tl + 4 * TC_N, lv);
#pragma unroll
      for (int q = 0; q < 16; ++q) tail[q] = fmaf(tail[q], 0.00390625f, lv[q]);
      // FP64 work only in warps with a live row and only on live columns (both warp-uniform
      // tests: the FP64 pipe spends a warp instruction's time whatever its active lanes)
      const bool warp_live = __any_sync(0xffffffffu, row_live);
      double sum[16];
      tc_ld16(tl + 0 * TC_N, lv);
#pragma unroll
      for (int q = 0; q < 16; ++q) sum[q] = tc_f2d(lv[q]);
#pragma unroll
      for (int t = 1; t < 4; ++t) {
        tc_ld16(tl + t * TC_N, lv);
        const double w8 = t == 1 ? 0.00390625 : (t == 2 ? 1.52587890625e-05 : 5.9604644775390625e-08);
        if (warp_live) {
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (q < ncq) sum[q] = fma(tc_f2d(lv[q]), w8, sum[q]);
        }
      }
      if (warp_live) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          if (q < ncq) {
            const int jc = hh * 16 + q;
            const double s = fma(tc_f2d_any(tail[q]), 2.3283064365386963e-10, sum[q]);   // 2^-32
            const double upd = fma(-tc_pow2(er_s[i] + ec_s[jc] - 16), s, wv[q]);
            if (row_live && ec_s[jc] != TC_EXP_NONE) row[q] = upd;
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
    }
  }
  return true;
}

// The bordered LU of condense_kernel with 32-column panels and the trailing
// updates on the tensor cores (tc_trailing_update); same inputs, outputs and
// workspace layout. One CTA of 256 threads per element, two per SM (the panel
// and the slice planes share the dynamic shared memory; 256 TMEM columns each).
__global__ void __launch_bounds__(256, 2) condense_tc_kernel(CondArgs a) {
  const Params& P = a.prm;
  const int eb = (int)(a.e0 + blockIdx.x);
  if (eb >= a.nslots) return;
  const int e = a.elist ? a.elist[eb] : eb;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int Q = P.Q, R = P.R, Cc = P.Cc, ld = P.ld;
  double* W = a.ws + (size_t)(a.slot_is_element ? eb : blockIdx.x) * (size_t)R * ld;

  extern __shared__ __align__(1024) unsigned char tsm[];
  double* Ls = reinterpret_cast<double*>(tsm);                               // [R][TCB + 1] (panel phase)
  uint16_t* As = reinterpret_cast<uint16_t*>(tsm);                           // [7][128 x 32] (update phase)
  uint16_t* Bs = reinterpret_cast<uint16_t*>(tsm + TC_A_BYTES);              // [7][32 x 32]
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ int piv_s[TCB];
  __shared__ int er_s[TC_M], ec_s[TC_N];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_s;
  __shared__ int s_fail;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(&tmem_s)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_s;

  form_system(a, e, W, Ls);

  int singular_col = -1;
  uint32_t phase = 0;
  for (int j0 = 0; j0 < Q; j0 += TCB) {
    const int nb = factor_panel<TCB, false>(a, W, Ls, nullptr, j0, eb, piv_s, red_v, red_i, singular_col);
    if (Cc - (j0 + nb) > 0 && !tc_trailing_update(a, W, j0, nb, As, Bs, er_s, ec_s, tmem, &mbar, phase, &s_fail))
      break;
    __syncthreads();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  // info: 0 fine, c + 1 zero pivot in column c, -1 the tensor cores did not finish within the bounded wait
  if (tid == 0 && a.info) a.info[eb] = s_fail ? -1 : (singular_col >= 0 ? singular_col + 1 : 0);
  if (a.write_outputs && !s_fail) condense_outputs(a, W, e, eb);
}

__device__ void condense_outputs(const CondArgs& a, const double* W, int e, int eb) {
  const Params& P = a.prm;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int Q = P.Q, nt = P.n_t, P1 = P.P1, ld = P.ld;
  // S_e row-blocks per local edge: S[eb][k][j][t] = S_e(k P1 + t, j)
  const size_t sb = (size_t)eb * 3 * nt * P1;
  for (int idx = tid; idx < nt * nt; idx += nthr) {
    const int j = idx / nt, r = idx - j * nt;
    const int k = r / P1, t = r - k * P1;
    a.S[sb + ((size_t)k * nt + j) * P1 + t] = W[(size_t)(Q + r) * ld + Q + j];
  }
  // preconditioned rows: Gh^-1 applied to each edge block of rows
  for (int idx = tid; a.St && idx < nt * nt; idx += nthr) {
    const int j = idx / nt, r = idx - j * nt;
    const int k = r / P1, t = r - k * P1;
    double acc = 0.0;
    for (int t2 = 0; t2 < P1; ++t2) acc += a.dt.Ghinv[t * P1 + t2] * W[(size_t)(Q + k * P1 + t2) * ld + Q + j];
    const size_t o = sb + ((size_t)k * nt + j) * P1 + t;
    a.St[o] = acc;
    if (a.St32) a.St32[o] = (float)acc;
  }
  // element right-hand sides -C A^-1 R_r - S_e g^_e,r of every source r
  int code[3], flip[3];
  elem_edges(e, P.n, code, flip);
  for (int idx = tid; idx < P.nrhs * nt; idx += nthr) {
    const int rr = idx / nt, r = idx - rr * nt;
    double acc = W[(size_t)(Q + r) * ld + Q + nt + rr];
    if (a.ghat) {
      const double* ghr = a.ghat + (size_t)rr * P.n_bnd * P1;
      for (int k = 0; k < 3; ++k) {
        if (code[k] >= 0) continue;
        const double* gb = ghr + (size_t)(-1 - code[k]) * P1;
        for (int t = 0; t < P1; ++t)
          acc -= W[(size_t)(Q + r) * ld + Q + k * P1 + t] * gb[flip[k] ? P.P - t : t];
      }
    }
    a.gel[((size_t)rr * a.nslots + eb) * nt + r] = acc;
  }
}

// ------------------------------------------------------ split-FP32 kernel
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }

// a * b for split-FP32 values (Dekker product through FMA)
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  return df_norm(p, e);
}

// 1 / d: FP32 quotient refined by one Newton step in split arithmetic
__device__ __forceinline__ float2 df_recip(float2 d) {
  const float q = 1.0f / d.x;
  float r = fmaf(-d.x, q, 1.0f);
  r = fmaf(-d.y, q, r);
  return df_norm(q, q * r);
}

__device__ __forceinline__ void warp_argmax_f(float& v, int& i) {
  for (int off = 16; off > 0; off >>= 1) {
    const float ov = __shfl_down_sync(0xffffffffu, v, off);
    const int oi = __shfl_down_sync(0xffffffffu, i, off);
    if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
  }
}

__global__ void __launch_bounds__(256) condense_df_kernel(CondArgs a) {
  const Params& P = a.prm;
  const int eb = (int)(a.e0 + blockIdx.x);
  if (eb >= a.nslots) return;
  const int e = a.elist ? a.elist[eb] : eb;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int Q = P.Q, nt = P.n_t, P1 = P.P1, R = P.R, Cc = P.Cc, ld = P.ld;
  double* Wd = a.ws + (size_t)(a.slot_is_element ? eb : blockIdx.x) * (size_t)R * ld;
  float2* W = reinterpret_cast<float2*>(Wd);

  extern __shared__ double smem[];
  float2* Ls = reinterpret_cast<float2*>(smem);             // [R][LDP]
  float2* Us = reinterpret_cast<float2*>(smem + (size_t)R * LDP);   // [NB][ld]
  __shared__ int piv_s[NB];
  __shared__ float red_v[8];
  __shared__ int red_i[8];
  __shared__ float2 sc[32];     // element and edge scalars of the formation (23 .. 31: SUPG)

  // ---------------------------------------------------------- element data
  ElemGeom g;
  elem_geom(e, P.n, g);
  const double kap = a.kappa[e];
  const double tau = kap / P.tau_len + P.babs;
  const double bxi_e = P.bx * g.gxi[0] + P.by * g.gxi[1];
  const double beta_e = P.bx * g.geta[0] + P.by * g.geta[1];
  const double ts = P.supg ? supg_tau(fmax(g.L[0], fmax(g.L[1], g.L[2])) / P.m, P.babs, kap) : 0.0;
  if (tid == 0) {
    const double gxx = g.gxi[0] * g.gxi[0] + g.gxi[1] * g.gxi[1];
    const double gxy = g.gxi[0] * g.geta[0] + g.gxi[1] * g.geta[1];
    const double gyy = g.geta[0] * g.geta[0] + g.geta[1] * g.geta[1];
    const double cK = kap * g.detJ;
    sc[0] = df_from(cK * gxx);
    sc[1] = df_from(cK * gxy);
    sc[2] = df_from(cK * gyy);
    sc[3] = df_from(-g.detJ * (P.bx * g.gxi[0] + P.by * g.gxi[1]));
    sc[4] = df_from(-g.detJ * (P.bx * g.geta[0] + P.by * g.geta[1]));
    for (int k = 0; k < 3; ++k) {
      const double nxi = g.nrm[k][0] * g.gxi[0] + g.nrm[k][1] * g.gxi[1];
      const double neta = g.nrm[k][0] * g.geta[0] + g.nrm[k][1] * g.geta[1];
      const double bn = P.bx * g.nrm[k][0] + P.by * g.nrm[k][1];
      sc[5 + k] = df_from(g.L[k] * (bn - tau));          // Fh and Gh terms of B_u and D_u
      sc[8 + k] = df_from(g.L[k] * kap * nxi);           // Pxi terms
      sc[11 + k] = df_from(g.L[k] * kap * neta);         // Peta terms
      sc[14 + k] = df_from(g.L[k] * tau);                // Fh term of C_u, E
      for (int l = 0; l < 3; ++l) {
        const double nn = g.nrm[k][0] * g.nrm[l][0] + g.nrm[k][1] * g.nrm[l][1];
        if (l >= k) sc[17 + (k == 0 ? l : (k == 1 ? 2 + l : 5))] = df_from(-kap * g.L[k] * g.L[l] * nn / g.detJ);
      }
    }
    // SUPG scalars (Sec. 3.4), in the order of the split SUPG tables
    const double bs = ts * g.detJ;
    sc[23] = df_from(bs * bxi_e * bxi_e);
    sc[24] = df_from(bs * bxi_e * beta_e);
    sc[25] = df_from(bs * beta_e * beta_e);
    sc[26] = df_from(-bs * kap * bxi_e * gxx);
    sc[27] = df_from(-bs * kap * bxi_e * 2.0 * gxy);
    sc[28] = df_from(-bs * kap * bxi_e * gyy);
    sc[29] = df_from(-bs * kap * beta_e * gxx);
    sc[30] = df_from(-bs * kap * beta_e * 2.0 * gxy);
    sc[31] = df_from(-bs * kap * beta_e * gyy);
  }
  __syncthreads();

  // --------------------------------------------------- form the bordered system
  // one flat loop over all entries: independent table loads per thread
  const float2 z2 = make_float2(0.f, 0.f);
  for (int idx = tid; idx < R * ld; idx += nthr) {
    const int i = idx / ld, j = idx - i * ld;
    float h = 0.f, l = 0.f;
    if (i < Q) {
      if (j < Q) {
        const size_t qi = (size_t)i * Q + j;
        df_fma(h, l, sc[0], a.dt.Kxx2[qi]);
        df_fma(h, l, sc[1], a.dt.Ksym2[qi]);
        df_fma(h, l, sc[2], a.dt.Kyy2[qi]);
        df_fma(h, l, sc[3], a.dt.Dxi2[qi]);
        df_fma(h, l, sc[4], a.dt.Deta2[qi]);
        if (P.supg)
#pragma unroll
          for (int k9 = 0; k9 < 9; ++k9) df_fma(h, l, sc[23 + k9], a.dt.Sup2[k9][qi]);
      } else if (j < Q + nt) {
        const int c = j - Q, k = c / P1;
        const size_t ic = (size_t)i * nt + c;
        df_fma(h, l, sc[5 + k], a.dt.Fh2[ic]);
        df_fma(h, l, df_neg(sc[8 + k]), a.dt.Pxi2[ic]);
        df_fma(h, l, df_neg(sc[11 + k]), a.dt.Peta2[ic]);
      }
    } else {
      const int r = i - Q, k = r / P1, t = r - k * P1;
      if (j < Q) {
        const size_t jr = (size_t)j * nt + r;
        df_fma(h, l, sc[8 + k], a.dt.Pxi2[jr]);
        df_fma(h, l, sc[11 + k], a.dt.Peta2[jr]);
        df_fma(h, l, sc[14 + k], a.dt.Fh2[jr]);
      } else if (j < Q + nt) {
        const int c = j - Q, l2 = c / P1, t2 = c - l2 * P1;
        const int kk = k < l2 ? k : l2, ll = k < l2 ? l2 : k;
        df_fma(h, l, sc[17 + (kk == 0 ? ll : (kk == 1 ? 2 + ll : 5))], a.dt.Hh2[(size_t)r * nt + c]);
        if (l2 == k) df_fma(h, l, sc[5 + k], a.dt.Gh2[t * P1 + t2]);
      }
    }
    W[idx] = df_norm(h, l);
  }
  __syncthreads();
  // load columns (FP64 projections in the panel area, stored split)
  load_columns(a, e, g.detJ, smem, [&](int i, int r, double v) { W[(size_t)i * ld + Q + nt + r] = df_from(v); },
               ts, bxi_e, beta_e);
  // tau E: E = sum_k L_k Pi_k^T Gh Pi_k (edge by edge: corner nodes are shared)
  for (int k = 0; k < 3; ++k) {
    for (int idx = tid; idx < P1 * P1; idx += nthr) {
      const int ni = a.dt.enode[k * P1 + idx / P1], nj = a.dt.enode[k * P1 + idx % P1];
      float2* wp = W + (size_t)ni * ld + nj;
      const float2 w0 = *wp;
      float h = w0.x, l = w0.y;
      df_fma(h, l, sc[14 + k], a.dt.Gh2[idx]);
      *wp = df_norm(h, l);
    }
    __syncthreads();
  }

  // ------------------------------------------------------- blocked LU, Q pivots
  int singular_col = -1;
  for (int j0 = 0; j0 < Q; j0 += NB) {
    const int nb = min(NB, Q - j0);
    const int rows = R - j0;
    for (int idx = tid; idx < rows * NB; idx += nthr) {
      const int r = idx / NB, c = idx - r * NB;
      Ls[r * LDP + c] = (c < nb) ? W[(size_t)(j0 + r) * ld + j0 + c] : z2;
    }
    __syncthreads();
    // panel factorisation: each thread owns rows tid, tid + 256, ... of the
    // panel; the pivot candidates of column c + 1 come out of the update of
    // column c, so one column costs one block argmax and one barrier more
    // when rows are interchanged
    float cv = -1.0f;
    int ci = 0x7fffffff;
    for (int r = tid; r < Q - j0; r += nthr) {
      const float v = fabsf(Ls[r * LDP].x);
      if (v > cv) { cv = v; ci = r; }
    }
    for (int c = 0; c < nb; ++c) {
      // pivot: largest |hi| among u-rows j0+c .. Q-1 (first one on ties)
      warp_argmax_f(cv, ci);
      if ((tid & 31) == 0) { red_v[tid >> 5] = cv; red_i[tid >> 5] = ci; }
      __syncthreads();
      if (tid < 32) {
        float v = tid < (nthr >> 5) ? red_v[tid] : -1.0f;
        int ii = tid < (nthr >> 5) ? red_i[tid] : 0x7fffffff;
        warp_argmax_f(v, ii);
        if (tid == 0) piv_s[c] = (v >= 0.0f && ii < Q - j0) ? ii : c;
      }
      __syncthreads();
      const int pr = piv_s[c];
      if (a.piv) {
        if (tid == 0) a.piv[(size_t)eb * Q + j0 + c] = j0 + pr;
        if (pr != c)
          for (int cc = tid; cc < j0; cc += nthr) {
            float2* x0 = W + (size_t)(j0 + c) * ld + cc;
            float2* x1 = W + (size_t)(j0 + pr) * ld + cc;
            const float2 t0 = *x0;
            *x0 = *x1;
            *x1 = t0;
          }
      }
      if (pr != c) {
        if (tid < nb) {
          const float2 t0 = Ls[c * LDP + tid];
          Ls[c * LDP + tid] = Ls[pr * LDP + tid];
          Ls[pr * LDP + tid] = t0;
        }
        __syncthreads();
      }
      const float2 d = Ls[c * LDP + c];
      if (d.x == 0.0f && singular_col < 0) singular_col = j0 + c;
      const float2 inv = (d.x != 0.0f) ? df_recip(d) : z2;
      cv = -1.0f;
      ci = 0x7fffffff;
      for (int r = c + 1 + tid; r < rows; r += nthr) {
        const float2 m = df_mul(Ls[r * LDP + c], inv);
        Ls[r * LDP + c] = m;
        const float2 nm = df_neg(m);
        for (int cc = c + 1; cc < nb; ++cc) {
          const float2 w0 = Ls[r * LDP + cc];
          float h = w0.x, l = w0.y;
          df_fma(h, l, nm, Ls[c * LDP + cc]);
          Ls[r * LDP + cc] = df_norm(h, l);
        }
        if (c + 1 < nb && r < Q - j0) {
          const float v = fabsf(Ls[r * LDP + c + 1].x);
          if (v > cv) { cv = v; ci = r; }
        }
      }
    }
    __syncthreads();
    for (int idx = tid; idx < rows * nb; idx += nthr) {
      const int r = idx / nb, c = idx - r * nb;
      W[(size_t)(j0 + r) * ld + j0 + c] = Ls[r * LDP + c];
    }
    const int jb = j0 + nb, ncol = Cc - jb;
    if (ncol > 0) {
      // row interchanges and U12 = L11^-1 A12, one column per thread
      for (int j = jb + tid; j < Cc; j += nthr) {
        float2 u[NB];
        for (int c = 0; c < nb; ++c) {
          const int pr = piv_s[c];
          if (pr != c) {
            float2* x0 = W + (size_t)(j0 + c) * ld + j;
            float2* x1 = W + (size_t)(j0 + pr) * ld + j;
            const float2 t0 = *x0;
            *x0 = *x1;
            *x1 = t0;
          }
        }
#pragma unroll
        for (int c = 0; c < NB; ++c) u[c] = (c < nb) ? W[(size_t)(j0 + c) * ld + j] : z2;
#pragma unroll
        for (int c = 1; c < NB; ++c) {
          if (c < nb) {
            float h = u[c].x, l = u[c].y;
#pragma unroll
            for (int t = 0; t < c; ++t) df_fma(h, l, df_neg(Ls[c * LDP + t]), u[t]);
            u[c] = df_norm(h, l);
          }
        }
        for (int c = 0; c < nb; ++c) {
          W[(size_t)(j0 + c) * ld + j] = u[c];
          Us[c * ld + j] = u[c];
        }
      }
      __syncthreads();
      // -L21 in place, then A22 -= L21 U12 (rows jb..R-1, columns jb..Cc-1)
      const int nrow = R - jb;
      for (int idx = tid; idx < nrow * NB; idx += nthr) {
        float2* p = Ls + (nb + idx / NB) * LDP + idx % NB;
        *p = df_neg(*p);
      }
      __syncthreads();
      const int ntile = (nrow + RT - 1) / RT;
      for (int item = tid; item < ntile * ncol; item += nthr) {
        const int rt = item / ncol, j = jb + (item - rt * ncol);
        const int r0 = jb + rt * RT;
        // the RT entries are loaded first (in flight during the products)
        float2 w0[RT];
#pragma unroll
        for (int rr = 0; rr < RT; ++rr) w0[rr] = r0 + rr < R ? W[(size_t)(r0 + rr) * ld + j] : z2;
        float h[RT], lo[RT];
#pragma unroll
        for (int rr = 0; rr < RT; ++rr) { h[rr] = 0.f; lo[rr] = 0.f; }
        // RT independent product chains (rows past R repeat row R-1 and are not stored)
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          const float2 uc = (c < nb) ? Us[c * ld + j] : z2;
#pragma unroll
          for (int rr = 0; rr < RT; ++rr) {
            const int r = min(r0 + rr, R - 1);
            df_fma(h[rr], lo[rr], Ls[(r - j0) * LDP + c], uc);
          }
        }
#pragma unroll
        for (int rr = 0; rr < RT; ++rr) {
          if (r0 + rr < R) {
            float wh = w0[rr].x, wl = w0[rr].y;
            df_add(wh, wl, h[rr], lo[rr]);
            W[(size_t)(r0 + rr) * ld + j] = df_norm(wh, wl);
          }
        }
      }
    }
    __syncthreads();
  }
  // back to FP64 in place for every reader of the factored system
  for (int idx = tid; idx < R * Cc; idx += nthr) {
    const int r = idx / Cc, c = idx - r * Cc;
    const size_t o = (size_t)r * ld + c;
    Wd[o] = df_to(W[o]);
  }
  __syncthreads();
  if (tid == 0 && a.info) a.info[eb] = singular_col >= 0 ? singular_col + 1 : 0;
  if (a.write_outputs) condense_outputs(a, Wd, e, eb);
}

// Back-solve Eq. (local_matrix_problem) on the factored bordered system:
// U u = L^-1 P (F - B_u u^_e), then q = M^-1 (D u - F u^) per component.
struct RecArgs {
  Params prm;
  DevTables dt;
  int rcol;               // which source's load column (0 .. nrhs-1)
  const double* ws;
  int64_t e0;
  int slot_is_element;
  const double* x;
  const double* ghat;
  double* u;
  double* q;
  // one refinement level of a level mesh (see CondArgs): slots of elist, the
  // element traces already gathered (xel [nslots][n_t]) and u, q at uoff[e]
  const int* elist;
  int64_t nslots;
  const double* xel;
  const int64_t* uoff;
  // several sources (recover_mrhs_kernel): per-source strides of x, g^, xel, u (q: 2 ustride)
  int nrhs;
  int64_t xstride, ghstride, xelstride, ustride;
};

__global__ void __launch_bounds__(128) recover_kernel(RecArgs a) {
  const Params& P = a.prm;
  const int eb = (int)(a.e0 + blockIdx.x);
  if (eb >= a.nslots) return;
  const int e = a.elist ? a.elist[eb] : eb;
  const int Q = P.Q, nt = P.n_t, P1 = P.P1, ld = P.ld;
  const double* W = a.ws + (size_t)(a.slot_is_element ? eb : blockIdx.x) * (size_t)P.R * ld;
  extern __shared__ double sm[];
  double* xe = sm;             // n_t
  double* rhs = xe + nt;       // Q
  double* uu = rhs + Q;        // Q
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;

  int code[3], flip[3];
  elem_edges(e, P.n, code, flip);
  for (int c = tid; c < nt; c += blockDim.x) {
    const int k = c / P1, t = c - k * P1;
    const int s = flip[k] ? P.P - t : t;
    double v = 0.0;
    if (a.xel) v = a.xel[(size_t)eb * nt + c];
    else if (code[k] >= 0) {
      if (HDG_INB((size_t)code[k] * P1 + s, P.N_tr, P.oob, 9)) v = a.x[(size_t)code[k] * P1 + s];
    } else if (a.ghat) {
      v = a.ghat[(size_t)(-1 - code[k]) * P1 + s];
    }
    xe[c] = v;
  }
  __syncthreads();
  // rhs = c - W x_e, one warp per row
  for (int i = warp; i < Q; i += nw) {
    const double* row = W + (size_t)i * ld + Q;
    double acc = 0.0;
    for (int c = lane; c < nt; c += 32) acc += row[c] * xe[c];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) rhs[i] = row[nt + a.rcol] - acc;
  }
  __syncthreads();
  // back substitution by warp 0
  if (warp == 0) {
    for (int i = Q - 1; i >= 0; --i) {
      const double* row = W + (size_t)i * ld;
      double acc = 0.0;
      for (int j = i + 1 + lane; j < Q; j += 32) acc += row[j] * uu[j];
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
      if (lane == 0) uu[i] = (rhs[i] - acc) / row[i];
      __syncwarp();
    }
  }
  __syncthreads();
  ElemGeom g;
  elem_geom(e, P.n, g);
  double* ue = a.u + (a.uoff ? a.uoff[e] : (int64_t)e * Q);
  double* qe = a.q + 2 * (a.uoff ? a.uoff[e] : (int64_t)e * Q);
  // one thread per row i, the tables read column-major (coalesced over i)
  for (int i = tid; i < Q; i += blockDim.x) {
    double sx = 0.0, sy = 0.0;
    for (int j = 0; j < Q; ++j) {
      const double b = uu[j];
      sx += a.dt.XxiT[(size_t)j * Q + i] * b;
      sy += a.dt.XetaT[(size_t)j * Q + i] * b;
    }
    double cx = 0.0, cy = 0.0;
    for (int c = 0; c < nt; ++c) {
      const int k = c / P1;
      const double v = a.dt.YhT[(size_t)c * Q + i] * xe[c] * g.L[k];
      cx += g.nrm[k][0] * v;
      cy += g.nrm[k][1] * v;
    }
    // grad_x = gxi_x d_xi + geta_x d_eta, and M^-1 = Mh^-1 / detJ
    qe[i] = g.gxi[0] * sx + g.geta[0] * sy - cx / g.detJ;
    qe[Q + i] = g.gxi[1] * sx + g.geta[1] * sy - cy / g.detJ;
    ue[i] = uu[i];
  }
}

// The same back-solve for RCM sources at a time (blockIdx.y = group of
// sources): the element's traces and right-hand sides for the group staged
// once ([n_t][RCM], [Q][RCM] in shared memory), the right-hand sides
// F_r - B_u x_e,r with one thread per (row, source), the back substitution
// with two sources per warp (16 lanes each, no block barriers), u and q with
// one thread per (row, source). FP64 arithmetic, as recover_kernel.
constexpr int RCM = 16;
__global__ void __launch_bounds__(256) recover_mrhs_kernel(RecArgs a) {
  const Params& P = a.prm;
  const int eb = (int)(a.e0 + blockIdx.x);
  if (eb >= a.nslots) return;
  const int e = a.elist ? a.elist[eb] : eb;
  const int Q = P.Q, nt = P.n_t, P1 = P.P1, ld = P.ld;
  const int c0 = blockIdx.y * RCM;
  const int nc = min(RCM, a.nrhs - c0);
  const double* W = a.ws + (size_t)(a.slot_is_element ? eb : blockIdx.x) * (size_t)P.R * ld;
  extern __shared__ double sm[];
  double* xe = sm;                 // [nt][RCM]
  double* B = sm + nt * RCM;       // [Q][RCM]: right-hand sides, then the solution
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
  int code[3], flip[3];
  elem_edges(e, P.n, code, flip);
  for (int idx = tid; idx < nt * RCM; idx += nthr) {
    const int c = idx / RCM, r = idx - c * RCM;
    double v = 0.0;
    if (r < nc) {
      const int col = c0 + r, k = c / P1, t = c - k * P1, s = flip[k] ? P.P - t : t;
      if (a.xel) v = a.xel[(size_t)col * a.xelstride + (size_t)eb * nt + c];
      else if (code[k] >= 0) v = a.x[(size_t)col * a.xstride + (size_t)code[k] * P1 + s];
      else if (a.ghat) v = a.ghat[(size_t)col * a.ghstride + (size_t)(-1 - code[k]) * P1 + s];
    }
    xe[idx] = v;
  }
  __syncthreads();
  for (int idx = tid; idx < Q * RCM; idx += nthr) {
    const int i = idx / RCM, r = idx - i * RCM;
    const double* row = W + (size_t)i * ld + Q;
    double acc = r < nc ? row[nt + c0 + r] : 0.0;
    for (int c = 0; c < nt; ++c) acc -= row[c] * xe[c * RCM + r];
    B[idx] = acc;
  }
  __syncthreads();
  {
    const int hl = lane & 15, r = 2 * warp + (lane >> 4);     // 8 warps x 2 sources
    for (int i = Q - 1; i >= 0; --i) {
      const double* row = W + (size_t)i * ld;
      double acc = 0.0;
      for (int j = i + 1 + hl; j < Q; j += 16) acc += row[j] * B[j * RCM + r];
#pragma unroll
      for (int off = 8; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if (hl == 0) B[i * RCM + r] = (B[i * RCM + r] - acc) / row[i];
      __syncwarp();
    }
  }
  __syncthreads();
  ElemGeom g;
  elem_geom(e, P.n, g);
  const int64_t ub = a.uoff ? a.uoff[e] : (int64_t)e * Q;
  for (int idx = tid; idx < Q * RCM; idx += nthr) {
    const int i = idx / RCM, r = idx - i * RCM;
    if (r >= nc) continue;
    const int col = c0 + r;
    const double* xr = a.dt.Xxi + (size_t)i * Q;
    const double* yr = a.dt.Xeta + (size_t)i * Q;
    double sx = 0.0, sy = 0.0;
    for (int j = 0; j < Q; ++j) {
      const double b = B[j * RCM + r];
      sx += xr[j] * b;
      sy += yr[j] * b;
    }
    const double* fr = a.dt.Yh + (size_t)i * nt;
    double cx = 0.0, cy = 0.0;
    for (int c = 0; c < nt; ++c) {
      const int k = c / P1;
      const double v = fr[c] * xe[c * RCM + r] * g.L[k];
      cx += g.nrm[k][0] * v;
      cy += g.nrm[k][1] * v;
    }
    double* ue = a.u + (size_t)col * a.ustride + ub;
    double* qe = a.q + (size_t)col * 2 * a.ustride + 2 * ub;
    qe[i] = g.gxi[0] * sx + g.geta[0] * sy - cx / g.detJ;
    qe[Q + i] = g.gxi[1] * sx + g.geta[1] * sy - cy / g.detJ;
    ue[i] = B[i * RCM + r];
  }
}

// Dirichlet data: g^ = L2 projection of g_D on every boundary edge (Sec. 2.3).
// blist / boff (a level mesh): the listed boundary edges only, edge b's points at boff[b].
__global__ void project_dirichlet_kernel(Params P, DevTables dt, const double* gD, double* ghat, const int* blist,
                                         const int64_t* boff) {
  const int b = blist ? blist[blockIdx.x] : (int)blockIdx.x;
  if (b >= P.n_bnd) return;
  extern __shared__ double rhs[];
  for (int t = threadIdx.x; t < P.P1; t += blockDim.x) rhs[t] = 0.0;
  __syncthreads();
  if (threadIdx.x == 0) {
    const double* gb = gD + (boff ? boff[b] : (int64_t)b * P.n_bqp);
    for (int s = 0; s < P.m; ++s)
      for (int q = 0; q < P.ngb; ++q) {
        const double w = dt.bw[q] / P.m * gb[s * P.ngb + q];
        for (int r = 0; r <= P.p; ++r) rhs[s * P.p + r] += w * dt.bpsi[q * (P.p + 1) + r];
      }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < P.P1; t += blockDim.x) {
    double acc = 0.0;
    for (int t2 = 0; t2 < P.P1; ++t2) acc += dt.Ghinv[t * P.P1 + t2] * rhs[t2];
    ghat[(size_t)b * P.P1 + t] = acc;
  }
}

// Gather S_e from the row-block layout into row-major [count][n_t][n_t].
__global__ void get_schur_kernel(Params P, const double* S, int64_t e0, int64_t count, double* out) {
  const int64_t total = count * P.n_t * P.n_t;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t el = idx / (P.n_t * P.n_t);
    const int rc = (int)(idx - el * P.n_t * P.n_t);
    const int r = rc / P.n_t, c = rc - r * P.n_t;
    const int k = r / P.P1, t = r - k * P.P1;
    out[idx] = S[(size_t)(e0 + el) * 3 * P.n_t * P.P1 + ((size_t)k * P.n_t + c) * P.P1 + t];
  }
}

// ------------------------------------------------------------------ launchers
size_t condense_smem_bytes(const Params& P) {
  return ((size_t)P.R * LDP + (size_t)NB * P.ld) * sizeof(double);
}

cudaError_t launch_condense(const Params& P, const DevTables& dt, const double* kappa, const double* f_qp,
                            const double* ghat, double* ws, int64_t e0, int64_t count, int slot_is_element,
                            int write_outputs, double* S, double* St, float* St32, double* gel, int* info,
                            cudaStream_t st, int split_update, int* piv) {
  CondArgs a;
  a.split_update = split_update;
  a.piv = piv;
  a.prm = P; a.dt = dt; a.kappa = kappa; a.f_qp = f_qp; a.ghat = ghat; a.ws = ws; a.e0 = e0;
  a.slot_is_element = slot_is_element; a.write_outputs = write_outputs;
  a.S = S; a.St = St; a.St32 = St32; a.gel = gel; a.info = info;
  a.elist = nullptr; a.nslots = P.N; a.qoff = nullptr; a.fstride = (int64_t)P.N * P.n_qp;
  return launch_condense_args(a, count, st);
}

static cudaError_t launch_condense_args(CondArgs& a, int64_t count, cudaStream_t st) {
  const Params& P = a.prm;
  const int split_update = a.split_update;
  const size_t sm = condense_smem_bytes(P);
  if (split_update == 2) {
    const size_t smt = condense_tc_smem_bytes(P);
    if (smt > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t err = cudaFuncSetAttribute(condense_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smt);
    if (err != cudaSuccess) return err;
    condense_tc_kernel<<<(unsigned)count, 256, smt, st>>>(a);
  } else if (split_update) {
    cudaError_t err = cudaFuncSetAttribute(condense_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    condense_df_kernel<<<(unsigned)count, 256, sm, st>>>(a);
  } else {
    cudaError_t err = cudaFuncSetAttribute(condense_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    condense_kernel<<<(unsigned)count, 256, sm, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_recover(const Params& P, const DevTables& dt, const double* ws, int64_t e0, int64_t count,
                           int slot_is_element, const double* x, const double* ghat, double* u, double* q,
                           cudaStream_t st, int rcol) {
  RecArgs a;
  a.prm = P; a.dt = dt; a.ws = ws; a.e0 = e0; a.slot_is_element = slot_is_element; a.rcol = rcol;
  a.x = x; a.ghat = ghat; a.u = u; a.q = q;
  a.elist = nullptr; a.nslots = P.N; a.xel = nullptr; a.uoff = nullptr;
  const size_t sm = (size_t)(P.n_t + 2 * P.Q) * sizeof(double);
  recover_kernel<<<(unsigned)count, 128, sm, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_project_dirichlet(const Params& P, const DevTables& dt, const double* gD, double* ghat,
                                     cudaStream_t st) {
  project_dirichlet_kernel<<<P.n_bnd, 64, P.P1 * sizeof(double), st>>>(P, dt, gD, ghat, nullptr, nullptr);
  return cudaGetLastError();
}

// ------------------------------------------- one refinement level of a level mesh
cudaError_t launch_condense_bin(const Params& P, const DevTables& dt, const double* kappa, const double* f_qp,
                                const int64_t* qoff, int64_t fstride, const double* ghat, double* ws,
                                const int* elist, int64_t nslots, int64_t e0, int64_t count, int slot_is_element,
                                int write_outputs, double* S, double* gel, int* info, cudaStream_t st,
                                int split_update) {
  CondArgs a;
  a.prm = P; a.dt = dt; a.kappa = kappa; a.f_qp = f_qp; a.ghat = ghat; a.ws = ws; a.e0 = e0;
  a.slot_is_element = slot_is_element; a.write_outputs = write_outputs;
  a.S = S; a.St = nullptr; a.St32 = nullptr; a.gel = gel; a.info = info;
  a.split_update = split_update; a.piv = nullptr;
  a.elist = elist; a.nslots = nslots; a.qoff = qoff; a.fstride = fstride;
  return launch_condense_args(a, count, st);
}

cudaError_t launch_recover_bin(const Params& P, const DevTables& dt, const double* ws, const int* elist,
                               int64_t nslots, int64_t e0, int64_t count, int slot_is_element, const double* xel,
                               const int64_t* uoff, double* u, double* q, cudaStream_t st, int rcol) {
  RecArgs a;
  a.prm = P; a.dt = dt; a.ws = ws; a.e0 = e0; a.slot_is_element = slot_is_element; a.rcol = rcol;
  a.x = nullptr; a.ghat = nullptr; a.u = u; a.q = q;
  a.elist = elist; a.nslots = nslots; a.xel = xel; a.uoff = uoff;
  const size_t sm = (size_t)(P.n_t + 2 * P.Q) * sizeof(double);
  recover_kernel<<<(unsigned)count, 128, sm, st>>>(a);
  return cudaGetLastError();
}

// Back-solve of nrhs sources at once (elements e0 .. e0+count-1 of the launch's
// slots): per-source strides xstride (x), ghstride (g^), xelstride (xel, or
// null), ustride (u; q has twice that).
cudaError_t launch_recover_mrhs(const Params& P, const DevTables& dt, const double* ws, const int* elist,
                                int64_t nslots, int64_t e0, int64_t count, int slot_is_element, const double* x,
                                int64_t xstride, const double* ghat, int64_t ghstride, const double* xel,
                                int64_t xelstride, const int64_t* uoff, double* u, double* q, int64_t ustride,
                                int nrhs, cudaStream_t st) {
  RecArgs a;
  a.prm = P; a.dt = dt; a.ws = ws; a.e0 = e0; a.slot_is_element = slot_is_element; a.rcol = 0;
  a.x = x; a.ghat = ghat; a.u = u; a.q = q;
  a.elist = elist; a.nslots = nslots; a.xel = xel; a.uoff = uoff;
  a.nrhs = nrhs; a.xstride = xstride; a.ghstride = ghstride; a.xelstride = xelstride; a.ustride = ustride;
  const size_t sm = (size_t)(P.n_t + P.Q) * RCM * sizeof(double);
  if (sm > 48 * 1024) {
    const cudaError_t err = cudaFuncSetAttribute(recover_mrhs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)sm);
    if (err != cudaSuccess) return err;
  }
  recover_mrhs_kernel<<<dim3((unsigned)count, (unsigned)((nrhs + RCM - 1) / RCM)), 256, sm, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_project_dirichlet_bin(const Params& P, const DevTables& dt, const int* blist, int nbnd,
                                         const int64_t* boff, const double* gD, double* ghat, cudaStream_t st) {
  if (nbnd <= 0) return cudaSuccess;
  project_dirichlet_kernel<<<nbnd, 64, P.P1 * sizeof(double), st>>>(P, dt, gD, ghat, blist, boff);
  return cudaGetLastError();
}

cudaError_t launch_get_schur(const Params& P, const double* S, int64_t e0, int64_t count, double* out,
                             cudaStream_t st) {
  get_schur_kernel<<<1024, 256, 0, st>>>(P, S, e0, count, out);
  return cudaGetLastError();
}

}  // namespace mehdg
