// Internal declarations of the macro-element HDG library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>
#include "../../include/mehdg.h"

// Kind of elimination requested by hdg_condense's flags: 0 FP64 (DFMA), 1 split-FP32,
// 2 FP64 panels with the trailing updates on the tensor cores.
inline int update_kind(unsigned flags) {
  return (flags & HDG_SPLIT_UPDATE) ? 1 : ((flags & HDG_TC_UPDATE) ? 2 : 0);
}

namespace mehdg {

// ---------------------------------------------------------------------------
// Reference tables of one refinement level (m, p), computed once on the host
// (reference.cpp) and copied to the device. All matrices are row-major FP64.
//   Mh          Q x Q     int phi_j phi_i              (reference triangle)
//   Dxi, Deta   Q x Q     int phi_j d_xi phi_i, ...    (row = differentiated test fn)
//   Kxx, Kyy    Q x Q     Dxi^T Mh^-1 Dxi, Deta^T Mh^-1 Deta
//   Ksym        Q x Q     Dxi^T Mh^-1 Deta + Deta^T Mh^-1 Dxi
//   Xxi, Xeta   Q x Q     Mh^-1 Dxi, Mh^-1 Deta        (recovery of q)
//   Fh          Q x 3P1   int_0^1 psi_t phi_i ds on reference edge k (block k)
//   Pxi, Peta   Q x 3P1   Dxi^T Mh^-1 Fh, Deta^T Mh^-1 Fh
//   Yh          Q x 3P1   Mh^-1 Fh
//   Hh          3P1 x 3P1 Fh^T Mh^-1 Fh
//   Gh, Ghinv   P1 x P1   1D C0 trace mass on [0,1] (m sub-intervals) and inverse
//   enode       3 x P1    lattice node of position t along reference edge k
//   phiq        nqs x nloc  P_p basis of a sub-triangle at its source points
//   wq          nqs        source weights on the unit triangle (sum 1/2)
//   subnode     nsub x nloc lattice node of each local basis function
//   node_sub    CSR over lattice nodes -> (sub-triangle, local index)
//   bpsi        ngb x (p+1) 1D basis at the boundary Gauss points, bw weights
// ---------------------------------------------------------------------------
struct RefTables {
  int m = 0, p = 0, P = 0, P1 = 0, Q = 0, n_t = 0;
  int ng = 0, nqs = 0, nloc = 0, nsub = 0, ngb = 0;
  std::vector<double> Mh, Dxi, Deta, Kxx, Kyy, Ksym, Xxi, Xeta;
  std::vector<double> Fh, Pxi, Peta, Yh, Hh, Gh, Ghinv;
  std::vector<double> XxiT, XetaT, YhT;  // transposes of Xxi, Xeta (Q x Q) and Yh (n_t x Q)
  std::vector<int> enode;
  std::vector<double> phiq, wq, uq;     // uq: Gauss nodes on [0,1] (ng)
  std::vector<int> subtri;              // nsub x 6 corners (a,b) in units of 1/m
  std::vector<int> subnode;
  std::vector<int> ns_ptr, ns_idx;      // CSR: node -> entries s * nloc + a
  std::vector<double> bpsi, bw, bu;     // boundary rule: nodes bu, weights bw (ngb)
  // SUPG (Sec. 3.4): Sxx = int d_xi phi_i d_xi phi_j, Syy, Ssym (mixed, symmetrised);
  // Lx_ab = int d_xi phi_i d_ab phi_j, Ly_ab = int d_eta phi_i d_ab phi_j (sub-triangle-wise
  // second derivatives); dphq [nsub][nqs][nloc][2] macro-reference gradients at source points
  std::vector<double> Sxx, Syy, Ssym, Lx_xx, Lx_xy, Lx_yy, Ly_xx, Ly_xy, Ly_yy, dphq;
};

// Builds the tables of level (m, p). Throws std::runtime_error on failure.
void build_reference_tables(int m, int p, RefTables& T);

// Trace tables of the face levels of a level mesh (Sec. 4.2), one host array:
// Gh_R (trace mass on [0,1] with 2^R sub-intervals) at G_off[R], its inverse at
// Gi_off[R], and for r < R the transfer T_rR ((2^r p + 1) x (2^R p + 1),
// row-major) at T_off[r][R] (-1 where not defined).
constexpr int kMaxLevel = 4;
struct LevelTables {
  int p = 0;
  int64_t G_off[kMaxLevel + 1], Gi_off[kMaxLevel + 1], T_off[kMaxLevel + 1][kMaxLevel + 1];
  std::vector<double> data;
};
void build_level_tables(int p, LevelTables& L);

// Device copies of the reference tables (pointers into one allocation).
struct DevTables {
  double *Dxi, *Deta, *Kxx, *Kyy, *Ksym, *Xxi, *Xeta;
  double *Fh, *Pxi, *Peta, *Yh, *Hh, *Gh, *Ghinv;
  double *XxiT, *XetaT, *YhT;
  int* enode;
  double *phiq, *wq, *uq;
  int *subtri, *subnode, *ns_ptr, *ns_idx;
  double *bpsi, *bw, *bu;
  // split-FP32 (hi, lo) copies of the element-formation tables
  float2 *Kxx2, *Kyy2, *Ksym2, *Dxi2, *Deta2, *Fh2, *Pxi2, *Peta2, *Hh2, *Gh2;
  // SUPG tables (FP64 and split copies of the nine Q x Q products)
  double *Sxx, *Syy, *Ssym, *Lx_xx, *Lx_xy, *Lx_yy, *Ly_xx, *Ly_xy, *Ly_yy, *dphq;
  float2 *Sup2[9];
};

// Scalar problem parameters passed by value to kernels.
struct Params {
  int n, m, p, P, P1, Q, n_t;
  int N, n_int, n_bnd, N_tr;
  int ng, nqs, nloc, nsub, n_qp, ngb, n_bqp;
  double bx, by, babs, kappa0, tau_len;
  int supg;              // 1: SUPG terms in the u-equations (Sec. 3.4)
  int R, Cc, ld;         // bordered local system: rows, used columns, leading dimension
  int nrhs;              // right-hand sides (source columns of the bordered system)
  int* oob;              // bounds-checked build: first failing index check (site code), else unused
};

// Index checks of the bounds-checked build (-DHDG_BOUNDS_CHECK): an index
// outside [0, n) records its site code in *oob (the first one wins), and the
// access it guards is skipped; no trap, so the context stays usable and the
// host reads the code (hdg_info bounds_error). In the regular build every
// check is the constant true and costs nothing.
#if defined(HDG_BOUNDS_CHECK) && defined(__CUDACC__)
__device__ __forceinline__ bool hdg_in_bounds(long long i, long long n, int* oob, int site) {
  if (i >= 0 && i < n) return true;
  if (oob) atomicCAS(oob, 0, site);
  return false;
}
#define HDG_INB(i, n, oob, site) hdg_in_bounds((long long)(i), (long long)(n), (oob), (site))
#else
#define HDG_INB(i, n, oob, site) true
#endif

// By-value view of a level mesh for kernels (device pointers).
// Element-side rows: the n_t,e trace dofs of every element, elements in
// "apply order" (decreasing n_t,e, then id); element e's rows start at zoff[e]
// and its blocks (n_t,e x n_t,e, column-major) at soff[e].
struct LevelDev {
  int N, n, n_int, p;
  int64_t N_tr, nz;
  int64_t ns;                 // lifted Schur-block entries
  int* oob;                   // bounds-checked build: see HDG_INB
  const int64_t* eoff;        // [n_int + 1] first trace dof of every interior edge
  const int* dof_edge;        // [N_tr] interior edge of every trace dof
  const int* ez;              // [n_int][2] element-side row of dof 0 of the face block on each side
  const int* eflip;           // [n_int] bit s: side s runs against the edge's orientation
  const signed char* flev;    // [n_int] face level
  const signed char* elev;    // [N] element level
  const int* row_ap;          // [nz] apply-order position of the element of every row
  const int64_t* ap_soff;     // [N] first block entry, by apply-order position
  const int* ap_zoff;         // [N] first row, by apply-order position
  const int* ap_nt;           // [N] n_t,e, by apply-order position
  const int64_t* soff;        // [N] first block entry, by element id
  const int* zoff;            // [N] first row, by element id
  const int* xmap;            // [nz] trace dof of every row, -1 on Dirichlet faces
  const double* tab;          // level tables (LevelTables::data)
  int64_t G_off[kMaxLevel + 1], Gi_off[kMaxLevel + 1], T_off[kMaxLevel + 1][kMaxLevel + 1];
  const double* escale;       // [n_int] -1 / ((tau+ + tau-) L_f)
  const int* eside;           // [n_int][2] element of each side
  const int* nte;             // [N] n_t,e by element id
  const int64_t* poff;        // [n_int + 1] first entry of every face's n_f x n_f block (face preconditioner)
};

// Face levels of element e from the per-edge and per-element levels.
__host__ __device__ inline int face_level(const signed char* flev, const signed char* elev, int e, int code) {
  return code >= 0 ? (int)flev[code] : (int)elev[e];
}

// ---------------------------------------------------------------------------
// Structured-mesh geometry (closed form, host and device).
// ---------------------------------------------------------------------------
// SUPG parameter of Sec. 3.4: tau_s = h / (2 |a|) (coth Pe - 1 / Pe), Pe = |a| h / (2 kappa)
// (the Laurent series below Pe = 0.1, the limit h / (2 |a|) for kappa = 0, 0 without advection).
__host__ __device__ inline double supg_tau(double h, double babs, double kappa) {
  if (!(babs > 0.0)) return 0.0;
  if (!(kappa > 0.0)) return h / (2.0 * babs);
  const double pe = babs * h / (2.0 * kappa);
  double xi;
  if (pe < 0.1) {
    // coth x - 1/x = x/3 - x^3/45 + 2 x^5/945 - x^7/4725 + 2 x^9/93555 - ... (Bernoulli numbers)
    const double x2 = pe * pe;
    xi = pe * (1.0 / 3.0 + x2 * (-1.0 / 45.0 + x2 * (2.0 / 945.0 + x2 * (-1.0 / 4725.0 + x2 * (2.0 / 93555.0)))));
  } else {
    xi = 1.0 / tanh(pe) - 1.0 / pe;
  }
  return h / (2.0 * babs) * xi;
}

__host__ __device__ inline void elem_vertices(int e, int n, double v[3][2]) {
  const int sq = e >> 1, t = e & 1;
  const int j = sq / n, i = sq - j * n;
  const double h = 1.0 / n;
  const double x0 = i * h, x1 = (i + 1) * h, y0 = j * h, y1 = (j + 1) * h;
  if (t == 0) {
    v[0][0] = x1; v[0][1] = y0; v[1][0] = x1; v[1][1] = y1; v[2][0] = x0; v[2][1] = y0;
  } else {
    v[0][0] = x0; v[0][1] = y1; v[1][0] = x0; v[1][1] = y0; v[2][0] = x1; v[2][1] = y1;
  }
}

// Local edge k of element e -> code (>= 0: interior edge id; < 0: -1 - boundary id), flip.
__host__ __device__ inline void elem_edges(int e, int n, int code[3], int flip[3]) {
  const int sq = e >> 1, t = e & 1;
  const int j = sq / n, i = sq - j * n;
  const int nn = n * n;
  auto horiz = [&](int ii, int jj) -> int {
    if (jj == 0) return -1 - ii;
    if (jj == n) return -1 - (n + ii);
    return nn + (jj - 1) * n + ii;
  };
  auto vert = [&](int ii, int jj) -> int {
    if (ii == 0) return -1 - (2 * n + jj);
    if (ii == n) return -1 - (3 * n + jj);
    return nn + n * (n - 1) + jj * (n - 1) + (ii - 1);
  };
  code[0] = j * n + i;
  if (t == 0) {
    flip[0] = 1; code[1] = horiz(i, j); flip[1] = 0; code[2] = vert(i + 1, j); flip[2] = 0;
  } else {
    flip[0] = 0; code[1] = horiz(i, j + 1); flip[1] = 1; code[2] = vert(i, j); flip[2] = 1;
  }
}

// The two sides (element, local edge, flip) of interior edge f; also its length.
__host__ __device__ inline void edge_sides(int f, int n, int e[2], int k[2], int fl[2], double* len) {
  const int nn = n * n;
  const double h = 1.0 / n;
  if (f < nn) {
    const int j = f / n, i = f - j * n;
    e[0] = 2 * (j * n + i); k[0] = 0; fl[0] = 1;
    e[1] = 2 * (j * n + i) + 1; k[1] = 0; fl[1] = 0;
    *len = h * 1.4142135623730951;
  } else if (f < nn + n * (n - 1)) {
    const int r = f - nn, j = 1 + r / n, i = r % n;
    e[0] = 2 * ((j - 1) * n + i) + 1; k[0] = 1; fl[0] = 1;   // square below, upper-left
    e[1] = 2 * (j * n + i); k[1] = 1; fl[1] = 0;             // square above, lower-right
    *len = h;
  } else {
    const int r = f - nn - n * (n - 1), j = r / (n - 1), i = 1 + r % (n - 1);
    e[0] = 2 * (j * n + (i - 1)); k[0] = 2; fl[0] = 0;       // square left, lower-right
    e[1] = 2 * (j * n + i) + 1; k[1] = 2; fl[1] = 1;         // square right, upper-left
    *len = h;
  }
}

// Affine map data of element e: det J, reference gradients, edge lengths and
// outward normals (edge k from v_{k+1} to v_{k+2}).
struct ElemGeom {
  double detJ;
  double gxi[2], geta[2];   // grad xi, grad eta (rows of J^-1)
  double L[3], nrm[3][2];
};

__host__ __device__ inline void elem_geom(int e, int n, ElemGeom& g) {
  double v[3][2];
  elem_vertices(e, n, v);
  const double J00 = v[1][0] - v[0][0], J10 = v[1][1] - v[0][1];
  const double J01 = v[2][0] - v[0][0], J11 = v[2][1] - v[0][1];
  g.detJ = J00 * J11 - J01 * J10;
  const double id = 1.0 / g.detJ;
  g.gxi[0] = J11 * id;  g.gxi[1] = -J01 * id;
  g.geta[0] = -J10 * id; g.geta[1] = J00 * id;
  for (int k = 0; k < 3; ++k) {
    const int a = (k + 1) % 3, b = (k + 2) % 3;
    const double tx = v[b][0] - v[a][0], ty = v[b][1] - v[a][1];
    const double L = sqrt(tx * tx + ty * ty);
    g.L[k] = L;
    g.nrm[k][0] = ty / L;
    g.nrm[k][1] = -tx / L;
  }
}


// One refinement level of a level mesh: the uniform-level tables and the
// condensation state of the elements of that level.
struct LevelBin {
  int r = 0, count = 0, nbnd = 0, max_nt = 0;   // level, elements, boundary edges, largest lifted n_t
  Params prm;                   // uniform-level parameters (N, n, N_tr as the whole mesh)
  RefTables ref;
  DevTables dt;
  void* d_tables = nullptr;
  int* d_elist = nullptr;       // [count] element ids, ascending
  int* d_blist = nullptr;       // [nbnd] boundary edges whose element is in the bin
  double* d_Sb = nullptr;       // [count][3][n_t][P1] own-level Schur blocks
  double* d_gelb = nullptr;     // [nrhs][count][n_t] own-level element right-hand sides
  double* d_ghat = nullptr;     // [nrhs][n_bnd][P1] projected Dirichlet data (the bin's edges)
  double* d_ws = nullptr;       // factored local systems
  int64_t ws_slots = 0;
  int ws_ld = 0;
  int* d_info = nullptr;
  double* d_xel = nullptr;      // [count][n_t] own-level traces for the back-solve
  size_t bytes_S = 0, bytes_gel = 0, bytes_ghat = 0, bytes_ws = 0, bytes_tables = 0, bytes_xel = 0;
};

struct LevelMesh {
  std::vector<signed char> elev, flev;
  std::vector<int64_t> eoff, goff, qoff, boff, uoff, soff_e;   // host prefix sums (element / edge order)
  std::vector<int> zoff_e, nt_e;
  int64_t nz = 0, ns = 0;
  int max_nt = 0;
  LevelTables lt;
  std::vector<LevelBin> bins;
  void* d_mem = nullptr;        // one allocation for the index arrays and tables
  size_t mem_bytes = 0;
  LevelDev dv;
  int64_t* d_qoff = nullptr;
  int64_t* d_boff = nullptr;
  int64_t* d_uoff = nullptr;
  int64_t* d_seoff = nullptr;   // [N + 1] n_t,e^2 prefix sums in element order
  double* d_S = nullptr;        // [ns] lifted Schur blocks
  double* d_St = nullptr;       // [ns] preconditioned lifted blocks
  float* d_St32 = nullptr;
  float2* d_Stdf = nullptr;
  double* d_gel = nullptr;      // [nrhs][nz] lifted element right-hand sides
  double* d_z = nullptr;        // [HDG_MAX_RHS][nz] element-side products
  int z_rhs = 0;
  int max_nf = 0;               // largest face block (2^R p + 1)
  int rb = 256;                 // element-side rows per CTA of the apply (hdg_autotune: 128, 256 or 512)
  double* d_Pinv = nullptr;     // [poff[n_int]] inverted face blocks (HDG_PRECOND_FACE_SCHUR)
  int64_t pinv_count = 0;
};
}  // namespace mehdg

// ---------------------------------------------------------------------------
// Context (opaque to callers).
// ---------------------------------------------------------------------------
namespace mehdg {
// Wait limit of the pipelined apply's mbarrier waits (clock64 cycles; 0: the built-in
// limit of about one second) and a test hook: the interior edge whose bulk copy is not
// issued (-1: none), which makes the waiting consumers give up (HDG_ERR_TIMEOUT).
struct BulkHooks {
  long long wait_cycles = 0;
  int skip_edge = -1;
};
}  // namespace mehdg

struct hdg_ctx {
  mehdg::Params prm;
  mehdg::RefTables ref;
  mehdg::DevTables dt;
  cudaStream_t stream = nullptr;
  std::string err;
  int state = 0;            // 0 created, 1 source set, 2 condensed
  unsigned flags = 0;
  void* d_tables = nullptr;
  double* d_kappa = nullptr;      // [N]
  int* d_oob = nullptr;           // bounds-checked build: first failing index check (site code)
  const double* f_qp = nullptr;   // caller-owned
  const double* gD_qp = nullptr;  // caller-owned or null
  double* d_ghat = nullptr;       // [n_bnd][P1]
  double* d_S = nullptr;          // [N][3][n_t][P1]  S_e, row-blocks per edge
  double* d_St = nullptr;         // [N][3][n_t][P1]  Gh^-1 S_e (preconditioned rows)
  float* d_St32 = nullptr;        // FP32 copy of d_St
  float2* d_Stdf = nullptr;       // d_St as FP32 (hi, lo) pairs
  char* d_Sfix = nullptr;         // d_St as fixed-point limbs and row scales (HDG_STORE_FIX64)
  int* d_Vs = nullptr;            // chunk scales of the fixed-point Krylov basis [restart + 1][chunks]
  double* d_vin = nullptr;        // the newest fixed-point basis vector in FP64 (the operator's input)
  double* d_gel = nullptr;        // [N][n_t] element right-hand sides
  double* d_g = nullptr;          // [N_tr] assembled right-hand side
  double* d_ws = nullptr;         // factored bordered systems [slots][R][ld]
  int64_t ws_slots = 0;
  int* d_info = nullptr;          // [N] zero-pivot column + 1, or 0
  int* d_piv = nullptr;           // [N][Q] pivot rows of the kept factors
  double* d_gadj = nullptr;       // [N][n_t] element parts of the adjoint right-hand side
  int* d_bad = nullptr;           // invalid-kappa counter of hdg_set_kappa
  int transposed = 0;             // 1 while the stored blocks hold S_e^T (hdg_transpose)
  int alloc_nrhs = 0;             // right-hand sides the per-RHS buffers (ghat, gel, g) are sized for
  int ws_ld = 0;                  // leading dimension the local workspace was allocated with
  double* d_escale = nullptr;     // [n_int] -1 / ((tau+ + tau-) L_f)
  int pc_face = 0;                // 1: the stored preconditioned rows hold S_ff^-1 (HDG_PRECOND_FACE_SCHUR)
  double* d_Pinv = nullptr;       // [n_int][P1][P1] inverted diagonal face blocks of S
  // Krylov workspace
  float2* d_V = nullptr;          // Krylov basis, split-FP32 pairs [restart + 1][N_tr]
  float2* d_w = nullptr;          // Arnoldi work vector, split-FP32 pairs [N_tr]
  double* d_r = nullptr;          // [N_tr]
  double* d_part = nullptr;       // reduction partials
  double* d_small = nullptr;      // Hessenberg, Givens, scalars
  int* d_flag = nullptr;
  void* d_aug = nullptr;          // [3][ldv] augmentation vectors of the restarted GMRES (basis format)
  int krylov_restart = 0;
  // batched (several right-hand sides) Krylov workspace, sized for (restart, nrhs)
  float2* d_Vb = nullptr;         // [restart + 1][nrhs][ldv] split-FP32 pairs
  float2* d_wb = nullptr;         // [nrhs][ldv]
  double* d_rb = nullptr;         // [2][nrhs][N_tr]: true residuals, then S x / D^-1 t
  double* d_partb = nullptr;      // [nrhs][partial rows x (restart + 2)]
  double* d_smallb = nullptr;     // [nrhs][small-array layout]
  int* d_flagb = nullptr;         // [nrhs][4]
  double* d_scalb = nullptr;      // [nrhs] gathered scalars
  int* d_cmapb = nullptr;         // [nrhs] columns still iterating in the current restart cycle
  float2* d_Zb = nullptr;         // [N][nrhs][n_t] element products of the multi-RHS apply
  void* d_augb = nullptr;         // [3][nrhs][ldv] augmentation vectors of the batched GMRES
  int kb_restart = 0, kb_nrhs = 0;
  // launch shapes chosen by hdg_autotune (0: built-in defaults)
  int tune_epb[4] = {0, 0, 0, 0}; // apply edges per block, per block type (FP64, split, FP32, fixed-point)
  mehdg::BulkHooks bulk_hooks;    // pipelined apply: wait limit and the copy-skip test hook
  int tune_kgd = 0;               // multi-dot blocks over all vector groups
  int tune_kgu = 0;               // streaming-update blocks
  // captured GMRES cycles (one restart cycle of Arnoldi steps each), with the configuration each
  // capture is valid for; the most recently used first, at most kGraphCache of them
  std::vector<std::pair<std::vector<intptr_t>, cudaGraphExec_t>> gm_cache;
  cudaStream_t cap_stream = nullptr;   // private stream used only for the capture
  std::vector<cudaEvent_t> gm_ev;      // per-step event quadruples of a timed capture
  mehdg::LevelMesh* lv = nullptr;     // per-element refinement levels (null: one level m)
  size_t bytes = 0;
  int64_t launches = 0;     // kernels enqueued (reported by hdg_info)
  // per-phase event timing
  bool prof_on = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_ev;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_pool;
  int64_t prof_count[HDG_PROF_NPHASES] = {0};
  double prof_ms[HDG_PROF_NPHASES] = {0};
};

namespace mehdg {
// Face scale of the preconditioned apply: -1 / ((tau+ + tau-) L_f) with the
// D^-1 preconditioner of Sec. 6.1 (Gh^-1 folded into the rows), none when the
// rows hold the inverted diagonal face blocks of S.
inline const double* precond_scale(const hdg_ctx* c) { return c->pc_face ? nullptr : c->d_escale; }

// Event pair around a launch when profiling is on (no-op otherwise).
struct ProfScope {
  hdg_ctx* c;
  int phase;
  cudaEvent_t b = nullptr, e = nullptr;
  ProfScope(hdg_ctx* ctx, int ph) : c(ctx), phase(ph) {
    if (!c->prof_on || ph < 0) return;
    if (!c->prof_pool.empty()) {
      b = c->prof_pool.back().first;
      e = c->prof_pool.back().second;
      c->prof_pool.pop_back();
    } else {
      cudaEventCreate(&b);
      cudaEventCreate(&e);
    }
    cudaEventRecord(b, c->stream);
  }
  ~ProfScope() {
    if (!b) return;
    cudaEventRecord(e, c->stream);
    c->prof_ev.push_back({phase, {b, e}});
  }
};
void profile_collect(hdg_ctx* c);
}  // namespace mehdg
