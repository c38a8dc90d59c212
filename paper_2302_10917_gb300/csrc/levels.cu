// Macro-elements of uneven refinement level (Sec. 4.2, local adaptive
// refinement): element e carries its own level r_e (m_e = 2^r_e sub-edges per
// macro-edge, the level-r_e C0 lattice inside), and the trace space of a face
// is refined to its finer side, R_F = max(r+, r-) (a boundary face has its
// element's level), so that it holds the trace of either side exactly.
//
// Condensation runs per refinement level ("bin") with the uniform-level
// kernels, giving every element's own-level blocks S_e^r, g_e^r. A face of
// level R > r only changes the coarse side's face couplings: the level-r basis
// restricted to the edge lies in the level-r trace space, so with
// T = Gh_r^-1 Pi^T Gh_R (Pi the level-r nodal basis at the level-R nodes)
//     B_e^R = B_e^r T,   C_e^R = T^T C_e^r,   D_e^R = (beta.n - tau) L Gh_R,
// and the condensed blocks follow exactly (Eq. global_problem) as
//     S_e = T^T (S_e^r - D_e^r) T + D_e^R,    g_e = T^T g_e^r
// (T block-diagonal over the three faces, the identity on faces of level
// r). The back-solve (Eq. local_matrix_problem) needs B_e^R u^ = B_e^r (T u^):
// the element sees the L2 projection of the face trace onto its own level.
//
// The trace operator (Sec. 3.3.2) is applied element-side: one thread per
// element-side row computes (S_e x_e)_a from the element's column-major block
// (rows of all elements concatenated in "apply order", decreasing n_t,e), and
// a per-face kernel adds the two sides (fixed order) and applies the face
// scale of D_f^-1 (Sec. 6.1; the Gh_R^-1 part is folded into the stored rows).
#include <algorithm>
#include <climits>
#include <cstring>
#include <new>
#include <numeric>
#include <type_traits>
#include "launch.h"
#include "df64.h"

namespace mehdg {

namespace {

constexpr int LV_RB_MAX = 512;              // element-side rows per CTA of the apply: at most (default 256)
constexpr size_t kLvMaxSmem = 227 * 1024;

template <typename T>
cudaError_t lv_alloc(hdg_ctx* c, T** p, size_t count) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e == cudaSuccess) c->bytes += count * sizeof(T);
  return e;
}

template <typename T>
void lv_free(hdg_ctx* c, T*& p, size_t count) {
  if (p) {
    cudaFree((void*)p);
    c->bytes -= std::min(c->bytes, (count ? count : 1) * sizeof(T));
  }
  p = nullptr;
}

hdg_status lv_err(hdg_ctx* c, hdg_status s, const std::string& m) {
  c->err = m;
  return s;
}

hdg_status lv_cuda(hdg_ctx* c, cudaError_t e, const char* where) {
  return lv_err(c, e == cudaErrorMemoryAllocation ? HDG_ERR_OOM : HDG_ERR_CUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

// ------------------------------------------------------------------ kernels
// Lifted blocks of the elements of one level r (one CTA per element).
__global__ void __launch_bounds__(256) lv_lift_kernel(LevelDev L, Params P, int r, const int* __restrict__ elist,
                                                      int count, const double* __restrict__ Sb,
                                                      const double* __restrict__ gelb, int nrhs,
                                                      const double* __restrict__ kappa, double* __restrict__ S,
                                                      double* __restrict__ St, double* __restrict__ gel) {
  const int eb = blockIdx.x;
  if (eb >= count) return;
  const int e = elist[eb];
  const int nc = P.n_t, P1c = P.P1, tid = threadIdx.x, nthr = blockDim.x;
  int code[3], flip[3], R[3], nfk[3], off[4];
  elem_edges(e, L.n, code, flip);
  off[0] = 0;
  for (int k = 0; k < 3; ++k) {
    R[k] = face_level(L.flev, L.elev, e, code[k]);
    nfk[k] = (1 << R[k]) * L.p + 1;
    off[k + 1] = off[k] + nfk[k];
  }
  const int nf = off[3];
  ElemGeom g;
  elem_geom(e, L.n, g);
  const double tau = kappa[e] / P.tau_len + P.babs;
  double dk[3];
  for (int k = 0; k < 3; ++k) dk[k] = (P.bx * g.nrm[k][0] + P.by * g.nrm[k][1] - tau) * g.L[k];
  auto face_of = [&](int a) { return a < off[1] ? 0 : (a < off[2] ? 1 : 2); };
  extern __shared__ double sm[];
  const int na = max(nc * nc, nf * nf);
  double* A = sm;        // X = S^r - D^r [nc][nc], then the lifted block [nf][nf] (row-major)
  double* W = sm + na;   // X T [nc][nf]
  const double* Gr = L.tab + L.G_off[r];
  for (int idx = tid; idx < nc * nc; idx += nthr) {
    const int i = idx / nc, j = idx - i * nc;
    const int k = i / P1c, t = i - k * P1c, l = j / P1c, t2 = j - l * P1c;
    double v = Sb[(((size_t)eb * 3 + k) * nc + j) * P1c + t];
    if (l == k) v -= dk[k] * Gr[t * P1c + t2];
    A[idx] = v;
  }
  __syncthreads();
  for (int idx = tid; idx < nc * nf; idx += nthr) {
    const int i = idx / nf, b = idx - i * nf;
    const int l = face_of(b), bl = b - off[l];
    double v;
    if (R[l] == r) {
      v = A[i * nc + l * P1c + bl];
    } else {
      const double* T = L.tab + L.T_off[r][R[l]];
      v = 0.0;
      for (int t = 0; t < P1c; ++t) v += A[i * nc + l * P1c + t] * T[t * nfk[l] + bl];
    }
    W[idx] = v;
  }
  __syncthreads();
  for (int idx = tid; idx < nf * nf; idx += nthr) {
    const int a = idx / nf, b = idx - a * nf;
    const int k = face_of(a), al = a - off[k];
    double v;
    if (R[k] == r) {
      v = W[(k * P1c + al) * nf + b];
    } else {
      const double* T = L.tab + L.T_off[r][R[k]];
      v = 0.0;
      for (int t = 0; t < P1c; ++t) v += T[t * nfk[k] + al] * W[(k * P1c + t) * nf + b];
    }
    if (face_of(b) == k) v += dk[k] * L.tab[L.G_off[R[k]] + (size_t)al * nfk[k] + (b - off[k])];
    A[idx] = v;
  }
  __syncthreads();
  const int64_t so = L.soff[e];
  for (int idx = tid; idx < nf * nf; idx += nthr) {
    const int b = idx / nf, a = idx - b * nf;       // column-major: consecutive a
    const int k = face_of(a), al = a - off[k];
    const double* Gi = L.tab + L.Gi_off[R[k]] + (size_t)al * nfk[k];
    double acc = 0.0;
    for (int t = 0; t < nfk[k]; ++t) acc += Gi[t] * A[(off[k] + t) * nf + b];
    S[so + idx] = A[a * nf + b];
    St[so + idx] = acc;
  }
  for (int idx = tid; idx < nrhs * nf; idx += nthr) {
    const int rr = idx / nf, a = idx - rr * nf;
    const int k = face_of(a), al = a - off[k];
    const double* gs = gelb + ((size_t)rr * count + eb) * nc + k * P1c;
    double v;
    if (R[k] == r) {
      v = gs[al];
    } else {
      const double* T = L.tab + L.T_off[r][R[k]];
      v = 0.0;
      for (int t = 0; t < P1c; ++t) v += T[t * nfk[k] + al] * gs[t];
    }
    gel[(size_t)rr * L.nz + L.zoff[e] + a] = v;
  }
}

// Own-level element traces of the back-solve: T u^ on faces finer than the
// element, u^ on the others, the projected Dirichlet data on boundary faces.
__global__ void lv_own_trace_kernel(LevelDev L, Params P, int r, const int* __restrict__ elist, int count,
                                    const double* __restrict__ x, const double* __restrict__ ghat,
                                    double* __restrict__ xel) {
  const int nc = P.n_t, P1 = P.P1, Pc = P.P;
  const int64_t total = (int64_t)count * nc;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int eb = (int)(idx / nc), ci = (int)(idx - (int64_t)eb * nc);
    const int e = elist[eb], k = ci / P1, t = ci - k * P1;
    int code[3], flip[3];
    elem_edges(e, L.n, code, flip);
    double v = 0.0;
    if (code[k] < 0) {
      if (ghat) v = ghat[(size_t)(-1 - code[k]) * P1 + (flip[k] ? Pc - t : t)];
    } else {
      const int f = code[k], R = L.flev[f];
      const int64_t b0 = L.eoff[f];
      if (R == r) {
        v = x[b0 + (flip[k] ? Pc - t : t)];
      } else {
        const int nf = (int)(L.eoff[f + 1] - b0), Pf = nf - 1;
        const double* T = L.tab + L.T_off[r][R] + (size_t)t * nf;
        for (int j = 0; j < nf; ++j) v += T[j] * x[b0 + (flip[k] ? Pf - j : j)];
      }
    }
    xel[idx] = v;
  }
}

// ----------------------------------------------------------- trace apply
// Block types BT: 0 FP64 (FP64 arithmetic), 1 split-FP32 pairs (split
// arithmetic), 2 FP32 (FP32 arithmetic). Vector types VT: 0 FP64, 1 split
// pairs, 2 FP32.
template <int BT>
struct LvAcc;
template <>
struct LvAcc<0> { using T = double; using S = double; };
template <>
struct LvAcc<1> { using T = float2; using S = float2; };
template <>
struct LvAcc<2> { using T = float; using S = float; };

template <int BT, int VT>
__device__ __forceinline__ typename LvAcc<BT>::T lv_load(const void* x, size_t i) {
  if constexpr (VT == 0) {
    const double v = static_cast<const double*>(x)[i];
    if constexpr (BT == 0) return v;
    else if constexpr (BT == 1) return df_from(v);
    else return (float)v;
  } else if constexpr (VT == 1) {
    const float2 v = static_cast<const float2*>(x)[i];
    if constexpr (BT == 0) return df_to(v);
    else if constexpr (BT == 1) return v;
    else return v.x;
  } else {
    const float v = static_cast<const float*>(x)[i];
    if constexpr (BT == 0) return (double)v;
    else if constexpr (BT == 1) return make_float2(v, 0.f);
    else return v;
  }
}

template <int BT>
__device__ __forceinline__ typename LvAcc<BT>::T lv_zero() {
  if constexpr (BT == 1) return make_float2(0.f, 0.f);
  else return typename LvAcc<BT>::T(0);
}

// z_r[row] = (S_e x_e,r)_a for the element-side rows of the CTA and RPT columns.
// cols_fast: blockIdx.x = column group, blockIdx.y = row block, so that the CTAs
// sharing a row block (and its blocks of S) run together and read S once from HBM.
template <int BT, int VT, int RPT>
__global__ void __launch_bounds__(LV_RB_MAX) lv_elem_kernel(LevelDev L, const void* __restrict__ Sv,
                                                        const void* __restrict__ xv, int nrhs, int64_t vstride,
                                                        void* __restrict__ zv, const int* __restrict__ stop,
                                                        int cols_fast, const int* __restrict__ cmap) {
  if (stop && *stop) return;
  using Acc = typename LvAcc<BT>::T;
  using ST = typename LvAcc<BT>::S;
  const ST* S = static_cast<const ST*>(Sv);
  Acc* zb = static_cast<Acc*>(zv);
  extern __shared__ unsigned char sraw[];
  Acc* xs = reinterpret_cast<Acc*>(sraw);   // rows of the CTA's elements x RPT columns
  const int rb = cols_fast ? blockIdx.y : blockIdx.x, cg = cols_fast ? blockIdx.x : blockIdx.y;
  const int64_t z0 = (int64_t)rb * blockDim.x;    // one thread per element-side row
  const int64_t zl = min(z0 + (int64_t)blockDim.x, L.nz) - 1;
  const int apf = L.row_ap[z0], apl = L.row_ap[zl];
  const int64_t xb = L.ap_zoff[apf];
  const int64_t xn = (int64_t)L.ap_zoff[apl] + L.ap_nt[apl] - xb;
  const int c0 = cg * RPT;
  for (int64_t i = threadIdx.x; i < xn * RPT; i += blockDim.x) {
    const int64_t row = xb + i / RPT;
    const int rr = (int)(i % RPT);
    const int d = L.xmap[row];
    Acc v = lv_zero<BT>();
    if (d >= 0 && c0 + rr < nrhs && HDG_INB(d, L.N_tr, L.oob, 11))
      v = lv_load<BT, VT>(xv, (size_t)(cmap ? cmap[c0 + rr] : c0 + rr) * vstride + d);
    xs[i] = v;
  }
  __syncthreads();
  const int64_t z = z0 + threadIdx.x;
  if (z > zl) return;
  const int ap = L.row_ap[z];
  const int nt = L.ap_nt[ap];
  const int a = (int)(z - L.ap_zoff[ap]);
  // the row's entries S[soff + a + c nt], c < nt, inside the blocks and its output inside z
  if (!HDG_INB(L.ap_soff[ap] + a + (int64_t)(nt - 1) * nt, L.ns, L.oob, 12) || !HDG_INB(a, nt, L.oob, 12) ||
      !HDG_INB((int64_t)(L.ap_zoff[ap] - xb + nt - 1) * RPT, (int64_t)(xn) * RPT, L.oob, 13))
    return;
  const ST* sp = S + L.ap_soff[ap] + a;
  const Acc* xe = xs + (L.ap_zoff[ap] - xb) * RPT;
  if constexpr (BT == 1) {
    float h[RPT], l[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) { h[q] = 0.f; l[q] = 0.f; }
    int c = 0;
    for (; c + 4 <= nt; c += 4) {
      float2 s[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) s[u] = sp[(size_t)(c + u) * nt];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < RPT; ++q) df_fma(h[q], l[q], s[u], xe[(c + u) * RPT + q]);
    }
    for (; c < nt; ++c) {
      const float2 s = sp[(size_t)c * nt];
#pragma unroll
      for (int q = 0; q < RPT; ++q) df_fma(h[q], l[q], s, xe[c * RPT + q]);
    }
#pragma unroll
    for (int q = 0; q < RPT; ++q)
      if (c0 + q < nrhs) zb[(size_t)(c0 + q) * L.nz + z] = df_norm(h[q], l[q]);
  } else {
    Acc acc[RPT], acc2[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) { acc[q] = Acc(0); acc2[q] = Acc(0); }
    int c = 0;
    for (; c + 4 <= nt; c += 4) {
      ST s[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) s[u] = sp[(size_t)(c + u) * nt];
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        acc[q] += s[0] * xe[c * RPT + q];
        acc2[q] += s[1] * xe[(c + 1) * RPT + q];
        acc[q] += s[2] * xe[(c + 2) * RPT + q];
        acc2[q] += s[3] * xe[(c + 3) * RPT + q];
      }
    }
    for (; c < nt; ++c) {
      const ST s = sp[(size_t)c * nt];
#pragma unroll
      for (int q = 0; q < RPT; ++q) acc[q] += s * xe[c * RPT + q];
    }
#pragma unroll
    for (int q = 0; q < RPT; ++q)
      if (c0 + q < nrhs) zb[(size_t)(c0 + q) * L.nz + z] = acc[q] + acc2[q];
  }
}

// y_r(i) = scale_f ((S x)_{side 0} + (S x)_{side 1}) at trace dof i of face f
template <int BT, int VT>
__global__ void lv_face_kernel(LevelDev L, const void* __restrict__ zv, void* __restrict__ yv, int nrhs,
                               int64_t vstride, const double* __restrict__ escale, const int* __restrict__ stop,
                               const int* __restrict__ cmap) {
  if (stop && *stop) return;
  using Acc = typename LvAcc<BT>::T;
  const Acc* zb = static_cast<const Acc*>(zv);
  const int64_t total = L.N_tr * nrhs;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / L.N_tr);
    const int64_t i = idx - (int64_t)r * L.N_tr;
    const int f = L.dof_edge[i];
    const int64_t b0 = L.eoff[f];
    const int s = (int)(i - b0), Pf = (int)(L.eoff[f + 1] - b0) - 1;
    const int fl = L.eflip[f];
    const int t0 = (fl & 1) ? Pf - s : s, t1 = (fl & 2) ? Pf - s : s;
    if (!HDG_INB((int64_t)L.ez[2 * f] + t0, L.nz, L.oob, 14) || !HDG_INB((int64_t)L.ez[2 * f + 1] + t1, L.nz, L.oob, 14))
      continue;
    const Acc a0 = zb[(size_t)r * L.nz + L.ez[2 * f] + t0];
    const Acc a1 = zb[(size_t)r * L.nz + L.ez[2 * f + 1] + t1];
    const size_t o = (size_t)(cmap ? cmap[r] : r) * vstride + i;
    if constexpr (BT == 1) {
      float h = a0.x, l = a0.y;
      df_add(h, l, a1.x, a1.y);
      if (escale) {
        float ph = 0.f, pl = 0.f;
        df_fma(ph, pl, make_float2(h, l), df_from(escale[f]));
        h = ph;
        l = pl;
      }
      const float2 out = df_norm(h, l);
      if constexpr (VT == 0) static_cast<double*>(yv)[o] = df_to(out);
      else if constexpr (VT == 1) static_cast<float2*>(yv)[o] = out;
      else static_cast<float*>(yv)[o] = out.x;
    } else {
      Acc v = a0 + a1;
      if (escale) v *= (Acc)escale[f];
      if constexpr (VT == 0) static_cast<double*>(yv)[o] = (double)v;
      else if constexpr (VT == 1) static_cast<float2*>(yv)[o] = BT == 0 ? df_from((double)v) : make_float2((float)v, 0.f);
      else static_cast<float*>(yv)[o] = (float)v;
    }
  }
}

// z_f = scale_f Gh_{R_f}^-1 y_f (the face preconditioner of Sec. 6.1) on FP64 vectors
__global__ void lv_dinv_kernel(LevelDev L, const double* __restrict__ y, double* __restrict__ z, int nrhs,
                               int64_t vstride) {
  const int64_t total = L.N_tr * nrhs;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / L.N_tr);
    const int64_t i = idx - (int64_t)r * L.N_tr;
    const int f = L.dof_edge[i];
    const int64_t b0 = L.eoff[f];
    const int s = (int)(i - b0), n1 = (int)(L.eoff[f + 1] - b0);
    const double* Gi = L.tab + L.Gi_off[L.flev[f]] + (size_t)s * n1;
    const double* yf = y + (size_t)r * vstride + b0;
    double acc = 0.0;
    for (int t = 0; t < n1; ++t) acc += Gi[t] * yf[t];
    z[(size_t)r * vstride + i] = L.escale[f] * acc;
  }
}

// Elements e0 .. e0 + count - 1, each block row-major, consecutive in element order.
__global__ void lv_get_schur_kernel(LevelDev L, const double* __restrict__ S, const int64_t* __restrict__ seoff,
                                    int64_t e0, int64_t count, double* __restrict__ out) {
  for (int64_t el = blockIdx.x; el < count; el += gridDim.x) {
    const int e = (int)(e0 + el);
    const int64_t n2 = seoff[e + 1] - seoff[e];
    const int nt = (int)llround(sqrt((double)n2));
    const int64_t ob = seoff[e] - seoff[e0];
    const int64_t so = L.soff[e];
    for (int idx = threadIdx.x; idx < nt * nt; idx += blockDim.x) {
      const int a = idx / nt, b = idx - a * nt;
      out[ob + idx] = S[so + (int64_t)b * nt + a];
    }
  }
}

__global__ void lv_to_fp32_kernel(const double* __restrict__ a, float* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)a[i];
}

// Physical source points of the elements of one level (elist), element e's at qoff[e].
__global__ void lv_quad_points_kernel(Params P, DevTables dt, const int* __restrict__ elist, int count,
                                      const int64_t* __restrict__ qoff, double* __restrict__ xy) {
  const int64_t total = (int64_t)count * P.n_qp;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int eb = (int)(idx / P.n_qp);
    const int r = (int)(idx - (int64_t)eb * P.n_qp);
    const int e = elist[eb];
    const int s = r / P.nqs, q = r - s * P.nqs;
    const int qj = q / P.ng, qi = q - qj * P.ng;
    const double xh = dt.uq[qi] * (1.0 - dt.uq[qj]), eh = dt.uq[qj];
    const int* c = dt.subtri + 6 * s;
    const double xi = (c[0] + xh * (c[2] - c[0]) + eh * (c[4] - c[0])) / P.m;
    const double eta = (c[1] + xh * (c[3] - c[1]) + eh * (c[5] - c[1])) / P.m;
    double v[3][2];
    elem_vertices(e, P.n, v);
    const int64_t o = qoff[e] + r;
    xy[2 * o + 0] = v[0][0] + xi * (v[1][0] - v[0][0]) + eta * (v[2][0] - v[0][0]);
    xy[2 * o + 1] = v[0][1] + xi * (v[1][1] - v[0][1]) + eta * (v[2][1] - v[0][1]);
  }
}

// Dirichlet-data points of the boundary edges of one level (blist), edge b's at boff[b].
__global__ void lv_bnd_points_kernel(Params P, DevTables dt, const int* __restrict__ blist, int nb,
                                     const int64_t* __restrict__ boff, double* __restrict__ xy) {
  const int64_t total = (int64_t)nb * P.n_bqp;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int bi = (int)(idx / P.n_bqp);
    const int r = (int)(idx - (int64_t)bi * P.n_bqp);
    const int b = blist[bi];
    const int s = r / P.ngb, q = r - s * P.ngb;
    const int side = b / P.n, k = b - side * P.n;
    const double h = 1.0 / P.n;
    double a0[2], a1[2];
    if (side == 0) { a0[0] = k * h; a0[1] = 0.0; a1[0] = (k + 1) * h; a1[1] = 0.0; }
    else if (side == 1) { a0[0] = k * h; a0[1] = 1.0; a1[0] = (k + 1) * h; a1[1] = 1.0; }
    else if (side == 2) { a0[0] = 0.0; a0[1] = k * h; a1[0] = 0.0; a1[1] = (k + 1) * h; }
    else { a0[0] = 1.0; a0[1] = k * h; a1[0] = 1.0; a1[1] = (k + 1) * h; }
    const double th = (s + dt.bu[q]) / P.m;
    const int64_t o = boff[b] + r;
    xy[2 * o + 0] = a0[0] + th * (a1[0] - a0[0]);
    xy[2 * o + 1] = a0[1] + th * (a1[1] - a0[1]);
  }
}

template <int BT, int VT, int RPT>
cudaError_t lv_apply_t(const LevelMesh& L, const void* S, const void* x, void* y, int nrhs, int64_t vstride,
                       const double* escale, const int* stop, void* z, cudaStream_t st, const int* cmap) {
  using Acc = typename LvAcc<BT>::T;
  const int RB = L.rb;
  const unsigned rblocks = (unsigned)((L.nz + RB - 1) / RB), cgroups = (unsigned)((nrhs + RPT - 1) / RPT);
  const int cols_fast = (cgroups > 1 && rblocks <= 65535u) ? 1 : 0;
  const dim3 grid = cols_fast ? dim3(cgroups, rblocks) : dim3(rblocks, cgroups);
  const size_t sm = (size_t)(RB + 2 * L.max_nt) * RPT * sizeof(Acc);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(lv_elem_kernel<BT, VT, RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
  }
  lv_elem_kernel<BT, VT, RPT><<<grid, RB, sm, st>>>(L.dv, S, x, nrhs, vstride, z, stop, cols_fast, cmap);
  const int64_t total = L.dv.N_tr * nrhs;
  const int fg = (int)std::min<int64_t>(152 * 8, (total + 255) / 256);
  lv_face_kernel<BT, VT><<<fg, 256, 0, st>>>(L.dv, z, y, nrhs, vstride, escale, stop, cmap);
  return cudaGetLastError();
}

template <int BT, int VT>
cudaError_t lv_apply_r(const LevelMesh& L, const void* S, const void* x, void* y, int nrhs, int64_t vstride,
                       const double* escale, const int* stop, void* z, cudaStream_t st, const int* cmap) {
  return nrhs > 1 ? lv_apply_t<BT, VT, 8>(L, S, x, y, nrhs, vstride, escale, stop, z, st, cmap)
                  : lv_apply_t<BT, VT, 1>(L, S, x, y, nrhs, vstride, escale, stop, z, st, cmap);
}

Params level_params(const hdg_mesh_desc* d, const RefTables& T, int N, int n_int) {
  Params P{};
  P.n = d->n; P.m = T.m; P.p = d->p; P.P = T.P; P.P1 = T.P1; P.Q = T.Q; P.n_t = T.n_t;
  P.N = N; P.n_int = n_int; P.n_bnd = 4 * d->n; P.N_tr = 0;
  P.ng = T.ng; P.nqs = T.nqs; P.nloc = T.nloc; P.nsub = T.nsub; P.n_qp = T.nsub * T.nqs;
  P.ngb = T.ngb; P.n_bqp = T.m * T.ngb;
  P.bx = d->beta[0]; P.by = d->beta[1]; P.babs = std::hypot(d->beta[0], d->beta[1]);
  P.kappa0 = d->kappa0; P.tau_len = d->tau_len; P.supg = d->supg;
  P.R = T.Q + T.n_t; P.nrhs = 1; P.Cc = T.Q + T.n_t + 1; P.ld = (P.Cc + 3) / 4 * 4;
  return P;
}

void set_nrhs(Params& P, int nrhs) {
  P.nrhs = nrhs;
  P.Cc = P.Q + P.n_t + nrhs;
  P.ld = (P.Cc + 3) / 4 * 4;
}

}  // namespace

// --------------------------------------------------------------- ABI parts
hdg_status level_create(hdg_ctx* c, const hdg_mesh_desc* d) {
  LevelMesh* Lp = new (std::nothrow) LevelMesh();
  if (!Lp) return lv_err(c, HDG_ERR_OOM, "level mesh");
  c->lv = Lp;
  LevelMesh& L = *Lp;
  const int n = d->n, p = d->p;
  const int N = 2 * n * n, n_int = n * n + 2 * n * (n - 1), n_bnd = 4 * n;
  L.elev.assign(d->level, d->level + N);
  L.flev.assign(n_int, 0);
  std::vector<signed char> blev(n_bnd, 0);
  for (int e = 0; e < N; ++e) {
    int code[3], flip[3];
    elem_edges(e, n, code, flip);
    for (int k = 0; k < 3; ++k) {
      if (code[k] >= 0) L.flev[code[k]] = std::max(L.flev[code[k]], L.elev[e]);
      else blev[-1 - code[k]] = L.elev[e];
    }
  }
  const int ng = p + 2;
  L.eoff.assign(n_int + 1, 0);
  for (int f = 0; f < n_int; ++f) L.eoff[f + 1] = L.eoff[f] + (1 << L.flev[f]) * p + 1;
  L.goff.assign(n_bnd + 1, 0);
  L.boff.assign(n_bnd + 1, 0);
  for (int b = 0; b < n_bnd; ++b) {
    L.goff[b + 1] = L.goff[b] + (1 << blev[b]) * p + 1;
    L.boff[b + 1] = L.boff[b] + (int64_t)(1 << blev[b]) * ng;
  }
  L.qoff.assign(N + 1, 0);
  L.uoff.assign(N + 1, 0);
  L.nt_e.assign(N, 0);
  std::vector<int64_t> seoff(N + 1, 0);
  int rmax = 0;
  for (int e = 0; e < N; ++e) {
    const int m = 1 << L.elev[e], P_ = m * p;
    rmax = std::max(rmax, (int)L.elev[e]);
    L.qoff[e + 1] = L.qoff[e] + (int64_t)m * m * ng * ng;
    L.uoff[e + 1] = L.uoff[e] + (int64_t)(P_ + 1) * (P_ + 2) / 2;
    int code[3], flip[3], nt = 0;
    elem_edges(e, n, code, flip);
    for (int k = 0; k < 3; ++k) nt += (1 << face_level(L.flev.data(), L.elev.data(), e, code[k])) * p + 1;
    L.nt_e[e] = nt;
    L.max_nt = std::max(L.max_nt, nt);
    seoff[e + 1] = seoff[e] + (int64_t)nt * nt;
  }
  const int64_t N_tr = L.eoff[n_int];
  if (N_tr > INT_MAX) return lv_err(c, HDG_ERR_ARG, "too many trace unknowns");
  // apply order: decreasing n_t, then element id
  std::vector<int> ap(N);
  std::iota(ap.begin(), ap.end(), 0);
  std::stable_sort(ap.begin(), ap.end(), [&](int a, int b) { return L.nt_e[a] > L.nt_e[b]; });
  L.zoff_e.assign(N, 0);
  L.soff_e.assign(N, 0);
  std::vector<int64_t> ap_soff(N);
  std::vector<int> ap_zoff(N), ap_nt(N);
  int64_t z = 0, s = 0;
  for (int i = 0; i < N; ++i) {
    const int e = ap[i];
    L.zoff_e[e] = (int)z;
    L.soff_e[e] = s;
    ap_zoff[i] = (int)z;
    ap_soff[i] = s;
    ap_nt[i] = L.nt_e[e];
    z += L.nt_e[e];
    s += (int64_t)L.nt_e[e] * L.nt_e[e];
  }
  if (z > INT_MAX) return lv_err(c, HDG_ERR_ARG, "too many element-side trace dofs");
  L.nz = z;
  L.ns = s;
  std::vector<int> row_ap(z), xmap(z);
  for (int i = 0; i < N; ++i) {
    const int e = ap[i];
    int code[3], flip[3];
    elem_edges(e, n, code, flip);
    int a = ap_zoff[i];
    for (int k = 0; k < 3; ++k) {
      const int R = face_level(L.flev.data(), L.elev.data(), e, code[k]);
      const int PR = (1 << R) * p;
      for (int t = 0; t <= PR; ++t, ++a) {
        row_ap[a] = i;
        xmap[a] = code[k] >= 0 ? (int)(L.eoff[code[k]] + (flip[k] ? PR - t : t)) : -1;
      }
    }
  }
  std::vector<int> dof_edge(N_tr), ez(2 * (size_t)n_int), eflip(n_int), eside(2 * (size_t)n_int);
  std::vector<double> escale(n_int);
  std::vector<int64_t> poff(n_int + 1, 0);
  for (int f = 0; f < n_int; ++f) {
    for (int64_t i = L.eoff[f]; i < L.eoff[f + 1]; ++i) dof_edge[i] = f;
    const int64_t nf = L.eoff[f + 1] - L.eoff[f];
    poff[f + 1] = poff[f] + nf * nf;
    L.max_nf = std::max(L.max_nf, (int)nf);
    int es[2], ks[2], fl[2];
    double len;
    edge_sides(f, n, es, ks, fl, &len);
    eside[2 * f] = es[0];
    eside[2 * f + 1] = es[1];
    double tsum = 0.0;
    for (int sd = 0; sd < 2; ++sd) {
      int code[3], flip[3], o = 0;
      elem_edges(es[sd], n, code, flip);
      for (int k = 0; k < ks[sd]; ++k) o += (1 << face_level(L.flev.data(), L.elev.data(), es[sd], code[k])) * p + 1;
      ez[2 * f + sd] = L.zoff_e[es[sd]] + o;
      const double ke = d->kappa ? d->kappa[es[sd]] : d->kappa0;
      tsum += ke / d->tau_len + std::hypot(d->beta[0], d->beta[1]);
    }
    eflip[f] = (fl[0] ? 1 : 0) | (fl[1] ? 2 : 0);
    escale[f] = -1.0 / (tsum * len);
  }
  build_level_tables(p, L.lt);
  // one device allocation for the index arrays and tables
  struct Item { const void* src; size_t bytes; void** dst; };
  LevelDev& dv = L.dv;
  std::vector<Item> items = {
      {L.eoff.data(), L.eoff.size() * 8, (void**)&dv.eoff},       {dof_edge.data(), dof_edge.size() * 4, (void**)&dv.dof_edge},
      {ez.data(), ez.size() * 4, (void**)&dv.ez},                 {eflip.data(), eflip.size() * 4, (void**)&dv.eflip},
      {L.flev.data(), L.flev.size(), (void**)&dv.flev},          {L.elev.data(), L.elev.size(), (void**)&dv.elev},
      {row_ap.data(), row_ap.size() * 4, (void**)&dv.row_ap},     {ap_soff.data(), ap_soff.size() * 8, (void**)&dv.ap_soff},
      {ap_zoff.data(), ap_zoff.size() * 4, (void**)&dv.ap_zoff},  {ap_nt.data(), ap_nt.size() * 4, (void**)&dv.ap_nt},
      {L.soff_e.data(), L.soff_e.size() * 8, (void**)&dv.soff},   {L.zoff_e.data(), L.zoff_e.size() * 4, (void**)&dv.zoff},
      {xmap.data(), xmap.size() * 4, (void**)&dv.xmap},           {L.lt.data.data(), L.lt.data.size() * 8, (void**)&dv.tab},
      {escale.data(), escale.size() * 8, (void**)&dv.escale},     {L.qoff.data(), L.qoff.size() * 8, (void**)&L.d_qoff},
      {L.boff.data(), L.boff.size() * 8, (void**)&L.d_boff},      {L.uoff.data(), L.uoff.size() * 8, (void**)&L.d_uoff},
      {seoff.data(), seoff.size() * 8, (void**)&L.d_seoff},
      {eside.data(), eside.size() * 4, (void**)&dv.eside},        {L.nt_e.data(), L.nt_e.size() * 4, (void**)&dv.nte},
      {poff.data(), poff.size() * 8, (void**)&dv.poff},
  };
  L.pinv_count = poff[n_int];
  size_t total = 0;
  for (auto& it : items) total += (it.bytes + 255) / 256 * 256;
  cudaError_t e;
  if ((e = cudaMalloc(&L.d_mem, total)) != cudaSuccess) return lv_cuda(c, e, "level mesh arrays");
  c->bytes += total;
  L.mem_bytes = total;
  std::vector<unsigned char> host(total, 0);
  size_t off = 0;
  for (auto& it : items) {
    if (it.bytes) std::memcpy(host.data() + off, it.src, it.bytes);
    *it.dst = (unsigned char*)L.d_mem + off;
    off += (it.bytes + 255) / 256 * 256;
  }
  if ((e = cudaMemcpyAsync(L.d_mem, host.data(), total, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return lv_cuda(c, e, "level mesh upload");
  dv.N = N; dv.n = n; dv.n_int = n_int; dv.p = p; dv.N_tr = N_tr; dv.nz = z; dv.ns = L.ns; dv.oob = c->d_oob;
  for (int R = 0; R <= kMaxLevel; ++R) {
    dv.G_off[R] = L.lt.G_off[R];
    dv.Gi_off[R] = L.lt.Gi_off[R];
    for (int q = 0; q <= kMaxLevel; ++q) dv.T_off[R][q] = L.lt.T_off[R][q];
  }
  c->d_escale = const_cast<double*>(dv.escale);   // owned by d_mem
  // one bin per level present
  for (int r = 0; r <= kMaxLevel; ++r) {
    std::vector<int> el, bl;
    for (int e2 = 0; e2 < N; ++e2)
      if (L.elev[e2] == r) el.push_back(e2);
    if (el.empty()) continue;
    for (int b = 0; b < n_bnd; ++b)
      if (blev[b] == r) bl.push_back(b);
    L.bins.emplace_back();
    LevelBin& B = L.bins.back();
    B.r = r;
    B.count = (int)el.size();
    B.nbnd = (int)bl.size();
    for (int e2 : el) B.max_nt = std::max(B.max_nt, L.nt_e[e2]);
    {
      // the panel bound first (from the sizes alone), then the tables
      RefTables sz;
      sz.m = 1 << r; sz.P = sz.m * p; sz.P1 = sz.P + 1; sz.Q = sz.P1 * (sz.P + 2) / 2; sz.n_t = 3 * sz.P1;
      const Params t = level_params(d, sz, N, n_int);
      if (condense_smem_bytes(t) > kLvMaxSmem)
        return lv_err(c, HDG_ERR_ARG, "level " + std::to_string(r) + " (m = " + std::to_string(1 << r) + "), p = " +
                                          std::to_string(p) + ": one element's panel needs " +
                                          std::to_string(condense_smem_bytes(t) / 1024) +
                                          " KB of shared memory (at most 227 KB)");
    }
    try {
      build_reference_tables(1 << r, p, B.ref);
    } catch (const std::exception& ex) {
      return lv_err(c, HDG_ERR_ARG, ex.what());
    }
    B.prm = level_params(d, B.ref, N, n_int);
    B.prm.oob = c->d_oob;
    const size_t lift = ((size_t)std::max(B.prm.n_t * B.prm.n_t, B.max_nt * B.max_nt) + (size_t)B.prm.n_t * B.max_nt) * 8;
    if (lift > kLvMaxSmem) return lv_err(c, HDG_ERR_ARG, "level " + std::to_string(r) + ": lifted blocks exceed shared memory");
    size_t tb = 0;
    if ((e = upload_ref_tables(B.ref, B.dt, &B.d_tables, &tb, c->stream)) != cudaSuccess) return lv_cuda(c, e, "level tables");
    c->bytes += tb;
    B.bytes_tables = tb;
    if ((e = lv_alloc(c, &B.d_elist, el.size())) != cudaSuccess ||
        (e = cudaMemcpyAsync(B.d_elist, el.data(), el.size() * 4, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
      return lv_cuda(c, e, "level element list");
    if ((e = lv_alloc(c, &B.d_blist, bl.size())) != cudaSuccess ||
        (bl.size() && (e = cudaMemcpyAsync(B.d_blist, bl.data(), bl.size() * 4, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess))
      return lv_cuda(c, e, "level boundary list");
  }
  // the mesh-wide parameters (largest level's sizes where a single value is asked for)
  const RefTables& Tm = L.bins.back().ref;
  Params& P = c->prm;
  P = level_params(d, Tm, N, n_int);
  P.oob = c->d_oob;
  P.N_tr = (int)N_tr;
  P.n_t = L.max_nt;
  P.n_qp = 0;
  P.n_bqp = 0;
  (void)rmax;
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return lv_cuda(c, e, "level mesh set-up");
  return HDG_OK;
}

void level_destroy(hdg_ctx* c) {
  if (!c->lv) return;
  LevelMesh& L = *c->lv;
  for (LevelBin& B : L.bins) {
    cudaFree(B.d_tables); cudaFree(B.d_elist); cudaFree(B.d_blist); cudaFree(B.d_Sb); cudaFree(B.d_gelb);
    cudaFree(B.d_ghat); cudaFree(B.d_ws); cudaFree(B.d_info); cudaFree(B.d_xel);
  }
  cudaFree(L.d_mem); cudaFree(L.d_S); cudaFree(L.d_St); cudaFree(L.d_St32); cudaFree(L.d_Stdf);
  cudaFree(L.d_gel); cudaFree(L.d_z); cudaFree(L.d_Pinv);
  c->d_escale = nullptr;   // part of d_mem
  delete c->lv;
  c->lv = nullptr;
}

hdg_status level_quad_points(hdg_ctx* c, double* xy) {
  for (const LevelBin& B : c->lv->bins) {
    lv_quad_points_kernel<<<1024, 256, 0, c->stream>>>(B.prm, B.dt, B.d_elist, B.count, c->lv->d_qoff, xy);
    c->launches += 1;
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HDG_OK : lv_cuda(c, e, "hdg_quad_points");
}

hdg_status level_bnd_quad_points(hdg_ctx* c, double* xy) {
  for (const LevelBin& B : c->lv->bins) {
    if (!B.nbnd) continue;
    lv_bnd_points_kernel<<<64, 256, 0, c->stream>>>(B.prm, B.dt, B.d_blist, B.nbnd, c->lv->d_boff, xy);
    c->launches += 1;
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HDG_OK : lv_cuda(c, e, "hdg_bnd_quad_points");
}

hdg_status level_set_source(hdg_ctx* c, const double* f_qp, const double* gD_qp, int nrhs) {
  LevelMesh& L = *c->lv;
  cudaError_t e;
  for (LevelBin& B : L.bins) {
    Params t = B.prm;
    set_nrhs(t, nrhs);
    if (condense_smem_bytes(t) > kLvMaxSmem)
      return lv_err(c, HDG_ERR_ARG, std::to_string(nrhs) + " sources need " + std::to_string(condense_smem_bytes(t) / 1024) +
                                        " KB of shared memory per element of level " + std::to_string(B.r) +
                                        " (at most 227 KB)");
  }
  if (nrhs != c->alloc_nrhs || !L.d_gel) {
    lv_free(c, L.d_gel, (size_t)c->alloc_nrhs * L.nz);
    lv_free(c, c->d_g, (size_t)c->alloc_nrhs * c->prm.N_tr);
    for (LevelBin& B : L.bins) {
      lv_free(c, B.d_ghat, B.bytes_ghat / 8);
      lv_free(c, B.d_gelb, B.bytes_gel / 8);
      B.bytes_ghat = B.bytes_gel = 0;
    }
    c->alloc_nrhs = 0;
    if ((e = lv_alloc(c, &L.d_gel, (size_t)nrhs * L.nz)) != cudaSuccess) return lv_cuda(c, e, "element right-hand sides");
    if ((e = lv_alloc(c, &c->d_g, (size_t)nrhs * c->prm.N_tr)) != cudaSuccess) return lv_cuda(c, e, "right-hand side");
    for (LevelBin& B : L.bins) {
      const size_t ng = (size_t)nrhs * B.prm.n_bnd * B.prm.P1, ngel = (size_t)nrhs * B.count * B.prm.n_t;
      if ((e = lv_alloc(c, &B.d_ghat, ng)) != cudaSuccess) return lv_cuda(c, e, "Dirichlet traces");
      if ((e = lv_alloc(c, &B.d_gelb, ngel)) != cudaSuccess) return lv_cuda(c, e, "element right-hand sides");
      B.bytes_ghat = ng * 8;
      B.bytes_gel = ngel * 8;
    }
    c->alloc_nrhs = nrhs;
  }
  for (LevelBin& B : L.bins) set_nrhs(B.prm, nrhs);
  set_nrhs(c->prm, nrhs);
  c->f_qp = f_qp;
  c->gD_qp = gD_qp;
  for (LevelBin& B : L.bins) {
    if ((e = cudaMemsetAsync(B.d_ghat, 0, B.bytes_ghat, c->stream)) != cudaSuccess) return lv_cuda(c, e, "Dirichlet traces");
    if (!gD_qp) continue;
    for (int r = 0; r < nrhs; ++r) {
      e = launch_project_dirichlet_bin(B.prm, B.dt, B.d_blist, B.nbnd, L.d_boff, gD_qp + (size_t)r * L.boff.back(),
                                       B.d_ghat + (size_t)r * B.prm.n_bnd * B.prm.P1, c->stream);
      c->launches += 1;
      if (e != cudaSuccess) return lv_cuda(c, e, "Dirichlet projection");
    }
  }
  c->state = 1;
  return HDG_OK;
}

hdg_status level_condense(hdg_ctx* c, unsigned flags) {
  LevelMesh& L = *c->lv;
  const int split = update_kind(flags);
  const int keep = (flags & HDG_KEEP_FACTORS) ? 1 : 0;
  const int nrhs = c->prm.nrhs;
  cudaError_t e;
  if (!L.d_S && (e = lv_alloc(c, &L.d_S, L.ns)) != cudaSuccess) return lv_cuda(c, e, "S blocks");
  if (!L.d_St && (e = lv_alloc(c, &L.d_St, L.ns)) != cudaSuccess) return lv_cuda(c, e, "preconditioned S blocks");
  if ((flags & HDG_STORE_FP32) && !L.d_St32 && (e = lv_alloc(c, &L.d_St32, L.ns)) != cudaSuccess)
    return lv_cuda(c, e, "FP32 S blocks");
  if (!(flags & HDG_STORE_FP32)) lv_free(c, L.d_St32, L.ns);
  if ((flags & HDG_STORE_DF64) && !L.d_Stdf && (e = lv_alloc(c, &L.d_Stdf, L.ns)) != cudaSuccess)
    return lv_cuda(c, e, "split-FP32 S blocks");
  if (!(flags & HDG_STORE_DF64)) lv_free(c, L.d_Stdf, L.ns);
  for (LevelBin& B : L.bins) {
    const Params& P = B.prm;
    const size_t sblk = (size_t)B.count * 3 * P.n_t * P.P1;
    if (!B.d_Sb) {
      if ((e = lv_alloc(c, &B.d_Sb, sblk)) != cudaSuccess) return lv_cuda(c, e, "own-level S blocks");
      B.bytes_S = sblk * 8;
    }
    if (!B.d_info && (e = lv_alloc(c, &B.d_info, (size_t)B.count)) != cudaSuccess) return lv_cuda(c, e, "info");
    const size_t slot = (size_t)P.R * P.ld;
    const int64_t budget = std::max<int64_t>(1, (int64_t)((size_t(1) << 30) / (slot * sizeof(double))));
    const int64_t want = keep ? B.count : std::min<int64_t>(B.count, budget);
    if (B.ws_slots != want || B.ws_ld != P.ld) {
      lv_free(c, B.d_ws, B.bytes_ws / 8);
      B.ws_slots = 0;
      B.bytes_ws = 0;
      if ((e = lv_alloc(c, &B.d_ws, (size_t)want * slot)) != cudaSuccess) return lv_cuda(c, e, "local workspace");
      B.ws_slots = want;
      B.ws_ld = P.ld;
      B.bytes_ws = (size_t)want * slot * 8;
    }
    const double* gh = c->gD_qp ? B.d_ghat : nullptr;
    for (int64_t e0 = 0; e0 < B.count; e0 += B.ws_slots) {
      const int64_t cnt = std::min<int64_t>(B.ws_slots, B.count - e0);
      ProfScope ps(c, HDG_PROF_CONDENSE);
      e = launch_condense_bin(P, B.dt, c->d_kappa, c->f_qp, L.d_qoff, L.qoff.back(), gh, B.d_ws, B.d_elist, B.count,
                              e0, cnt, keep, 1, B.d_Sb, B.d_gelb, B.d_info, c->stream, split);
      c->launches += 1;
      if (e != cudaSuccess) return lv_cuda(c, e, "condense kernel");
    }
    const size_t sm = ((size_t)std::max(P.n_t * P.n_t, B.max_nt * B.max_nt) + (size_t)P.n_t * B.max_nt) * 8;
    if ((e = cudaFuncSetAttribute(lv_lift_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
      return lv_cuda(c, e, "lift kernel");
    {
      ProfScope ps(c, HDG_PROF_CONDENSE);
      lv_lift_kernel<<<B.count, 256, sm, c->stream>>>(L.dv, P, B.r, B.d_elist, B.count, B.d_Sb, B.d_gelb, nrhs,
                                                      c->d_kappa, L.d_S, L.d_St, L.d_gel);
    }
    c->launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return lv_cuda(c, e, "lift kernel");
  }
  c->pc_face = 0;
  if (flags & HDG_PRECOND_FACE_SCHUR) {
    if (!L.d_Pinv && (e = lv_alloc(c, &L.d_Pinv, (size_t)L.pinv_count)) != cudaSuccess)
      return lv_cuda(c, e, "face blocks");
    if (!c->d_bad && (e = lv_alloc(c, &c->d_bad, 1)) != cudaSuccess) return lv_cuda(c, e, "face block check");
    int bad = 0;
    if ((e = cudaMemsetAsync(c->d_bad, 0, sizeof(int), c->stream)) != cudaSuccess ||
        (e = launch_level_face_schur(L.dv, L.max_nf, L.d_S, L.d_Pinv, L.d_St, c->d_bad, c->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&bad, c->d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
      return lv_cuda(c, e, "face blocks");
    c->launches += 2;
    if (bad) {
      c->state = 1;
      return lv_err(c, HDG_ERR_SINGULAR, std::to_string(bad) + " diagonal face blocks of S have a zero pivot");
    }
    c->pc_face = 1;
  }
  if (flags & HDG_STORE_FP32) {
    lv_to_fp32_kernel<<<2048, 256, 0, c->stream>>>(L.d_St, L.d_St32, L.ns);
    c->launches += 1;
  }
  if (flags & HDG_STORE_DF64) {
    c->launches += 1;
    if ((e = launch_split_df(L.d_St, L.d_Stdf, L.ns, c->stream)) != cudaSuccess) return lv_cuda(c, e, "split");
  }
  // g = sum over the two sides of every face (no scale)
  {
    const int64_t total = L.dv.N_tr * nrhs;
    const int fg = (int)std::min<int64_t>(152 * 8, (total + 255) / 256);
    lv_face_kernel<0, 0><<<fg, 256, 0, c->stream>>>(L.dv, L.d_gel, c->d_g, nrhs, L.dv.N_tr, nullptr, nullptr,
                                                    nullptr);
    c->launches += 1;
  }
  for (LevelBin& B : L.bins) {
    std::vector<int> info(B.count), el(B.count);
    if ((e = cudaMemcpyAsync(info.data(), B.d_info, (size_t)B.count * 4, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(el.data(), B.d_elist, (size_t)B.count * 4, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
      return lv_cuda(c, e, "condense");
    for (int i = 0; i < B.count; ++i)
      if (info[i] < 0) {
        c->state = 1;
        return lv_err(c, HDG_ERR_TIMEOUT, "condensation: the tensor-core update of element " + std::to_string(el[i]) +
                                              " did not complete within the bounded wait");
      } else if (info[i]) {
        c->state = 1;
        return lv_err(c, HDG_ERR_SINGULAR, "zero pivot in column " + std::to_string(info[i] - 1) + " of element " +
                                               std::to_string(el[i]));
      }
  }
  c->flags = flags;
  c->state = 2;
  return HDG_OK;
}

hdg_status level_recover(hdg_ctx* c, const double* x, double* u, double* q, int nrhs) {
  LevelMesh& L = *c->lv;
  cudaError_t e;
  const int64_t nu = L.uoff.back();
  for (LevelBin& B : L.bins) {
    const Params& P = B.prm;
    const size_t nxel = (size_t)B.count * P.n_t * nrhs;
    if (B.bytes_xel < nxel * 8) {
      lv_free(c, B.d_xel, B.bytes_xel / 8);
      B.bytes_xel = 0;
      if ((e = lv_alloc(c, &B.d_xel, nxel)) != cudaSuccess) return lv_cuda(c, e, "element traces");
      B.bytes_xel = nxel * 8;
    }
    const int keep = (c->flags & HDG_KEEP_FACTORS) ? 1 : 0;
    const double* gh = c->gD_qp ? B.d_ghat : nullptr;
    if (nrhs > 1) {
      // own-level traces of every source, then one back-solve launch per element range
      for (int r = 0; r < nrhs; ++r) {
        lv_own_trace_kernel<<<256, 256, 0, c->stream>>>(L.dv, P, B.r, B.d_elist, B.count,
                                                        x + (size_t)r * c->prm.N_tr,
                                                        gh ? gh + (size_t)r * P.n_bnd * P.P1 : nullptr,
                                                        B.d_xel + (size_t)r * B.count * P.n_t);
        c->launches += 1;
      }
      for (int64_t e0 = 0; e0 < B.count; e0 += (keep ? B.count : B.ws_slots)) {
        const int64_t cnt = keep ? B.count : std::min<int64_t>(B.ws_slots, B.count - e0);
        if (!keep) {
          e = launch_condense_bin(P, B.dt, c->d_kappa, c->f_qp, L.d_qoff, L.qoff.back(), gh, B.d_ws, B.d_elist,
                                  B.count, e0, cnt, 0, 0, nullptr, nullptr, nullptr, c->stream,
                                  update_kind(c->flags));
          c->launches += 1;
          if (e != cudaSuccess) return lv_cuda(c, e, "refactor");
        }
        ProfScope ps(c, HDG_PROF_RECOVER);
        e = launch_recover_mrhs(P, B.dt, B.d_ws, B.d_elist, B.count, e0, cnt, keep, nullptr, 0, nullptr, 0, B.d_xel,
                                (int64_t)B.count * P.n_t, L.d_uoff, u, q, nu, nrhs, c->stream);
        c->launches += 1;
        if (e != cudaSuccess) return lv_cuda(c, e, "recover");
      }
      continue;
    }
    for (int64_t e0 = 0; e0 < B.count; e0 += (keep ? B.count : B.ws_slots)) {
      const int64_t cnt = keep ? B.count : std::min<int64_t>(B.ws_slots, B.count - e0);
      if (!keep) {
        e = launch_condense_bin(P, B.dt, c->d_kappa, c->f_qp, L.d_qoff, L.qoff.back(), gh, B.d_ws, B.d_elist, B.count,
                                e0, cnt, 0, 0, nullptr, nullptr, nullptr, c->stream, update_kind(c->flags));
        c->launches += 1;
        if (e != cudaSuccess) return lv_cuda(c, e, "refactor");
      }
      for (int r = 0; r < nrhs; ++r) {
        ProfScope ps(c, HDG_PROF_RECOVER);
        lv_own_trace_kernel<<<256, 256, 0, c->stream>>>(L.dv, P, B.r, B.d_elist, B.count, x + (size_t)r * c->prm.N_tr,
                                                        gh ? gh + (size_t)r * P.n_bnd * P.P1 : nullptr, B.d_xel);
        e = launch_recover_bin(P, B.dt, B.d_ws, B.d_elist, B.count, e0, cnt, keep, B.d_xel, L.d_uoff,
                               u + (size_t)r * nu, q + (size_t)r * 2 * nu, c->stream, r);
        c->launches += 2;
        if (e != cudaSuccess) return lv_cuda(c, e, "recover");
      }
    }
  }
  return HDG_OK;
}

hdg_status level_get_schur(hdg_ctx* c, int64_t e0, int64_t count, double* S) {
  lv_get_schur_kernel<<<(unsigned)std::min<int64_t>(count, 4096), 256, 0, c->stream>>>(c->lv->dv, c->lv->d_S,
                                                                                         c->lv->d_seoff, e0, count, S);
  c->launches += 1;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HDG_OK : lv_cuda(c, e, "hdg_get_schur");
}

cudaError_t level_ensure_z(hdg_ctx* c, int nrhs) {
  LevelMesh& L = *c->lv;
  if (L.z_rhs >= nrhs && L.d_z) return cudaSuccess;
  lv_free(c, L.d_z, (size_t)L.z_rhs * L.nz);
  L.z_rhs = 0;
  cudaError_t e = lv_alloc(c, &L.d_z, (size_t)nrhs * L.nz);
  if (e == cudaSuccess) L.z_rhs = nrhs;
  return e;
}

cudaError_t launch_level_apply(hdg_ctx* c, int bt, int vt, const void* S, const void* x, void* y, int nrhs,
                               int64_t vstride, const double* escale, const int* stop, cudaStream_t st,
                               const int* cmap) {
  const LevelMesh& L = *c->lv;
  if (!L.d_z || L.z_rhs < nrhs) return cudaErrorInvalidValue;
  void* z = L.d_z;
#define LV_CASE(B, V) \
  if (bt == B && vt == V) return lv_apply_r<B, V>(L, S, x, y, nrhs, vstride, escale, stop, z, st, cmap);
  LV_CASE(0, 0) LV_CASE(0, 1) LV_CASE(1, 0) LV_CASE(1, 1) LV_CASE(2, 0) LV_CASE(2, 1) LV_CASE(2, 2)
#undef LV_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_level_dinv(hdg_ctx* c, const double* y, double* z, int nrhs, int64_t vstride, cudaStream_t st) {
  const int64_t total = c->lv->dv.N_tr * nrhs;
  const int g = (int)std::min<int64_t>(152 * 8, (total + 255) / 256);
  lv_dinv_kernel<<<g, 256, 0, st>>>(c->lv->dv, y, z, nrhs, vstride);
  return cudaGetLastError();
}

}  // namespace mehdg
