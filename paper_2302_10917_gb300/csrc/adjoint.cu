// Discrete adjoint of the condensed problem (no counterpart in the paper).
//
// The reduced element system of the forward path (q eliminated, see
// condense.cu) is
//     A_u u_e + B_u x_e = F_e            (u-rows)
//     sum_e (C_u u_e + D_u x_e) = 0      (trace rows, interior trace dofs)
// For J(u) with r_e = dJ/du_e, the adjoint state (mu, nu) solves the
// transposed system
//     A_u^T mu_e + C_u^T nu_e = r_e,     sum_e (B_u^T mu_e + D_u^T nu_e) = 0,
// i.e. S^T nu = -sum_e B_u^T A_u^-T r_e and mu_e = A_u^-T (r_e - C_u^T nu_e),
// and the gradient follows from the derivative of the element blocks:
//     dJ/dkappa_e = -[mu_e; nu_e]^T (dK_e/dkappa_e) [u_e; x_e],
//     dJ/df_e     = mu_e^T dF_e/df_e.
// The kept factors supply everything: rows 0..Q-1 of the bordered system hold
// P A_u = L U and L^-1 P B_u, rows Q.. hold M21 = C_u U^-1, so
//     B_u^T A_u^-T r = (L^-1 P B_u)^T U^-T r,
//     mu = P^T L^-T (U^-T r - M21^T nu).
// The blocks are affine in kappa_e (tau_e = kappa_e / tau_len + |beta|), so
// dK_e/dkappa_e is the block system formed with kappa = 1, tau = 1/tau_len
// and beta = 0.
#include "internal.h"
#include "df64.h"

namespace mehdg {

// kappa <- src (device), counting entries that are negative or not finite.
__global__ void copy_kappa_kernel(int N, const double* src, double* kappa, int* bad) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x) {
    const double v = src[e];
    if (!(v >= 0.0) || !isfinite(v)) atomicAdd(bad, 1);
    kappa[e] = v;
  }
}

// S_e <- S_e^T in place (row-block layout S[e][k][j][t] = S_e(k P1 + t, j)),
// then the derived preconditioned copies are formed again from it.
__global__ void __launch_bounds__(256) transpose_kernel(Params P, DevTables dt, double* S, double* St, float* St32,
                                                       float2* Stdf) {
  const int e = blockIdx.x;
  if (e >= P.N) return;
  const int nt = P.n_t, P1 = P.P1;
  double* Se = S + (size_t)e * 3 * nt * P1;
  for (int idx = threadIdx.x; idx < nt * nt; idx += blockDim.x) {
    const int r = idx / nt, c = idx - r * nt;
    if (r >= c) continue;
    double* a = Se + ((size_t)(r / P1) * nt + c) * P1 + r % P1;
    double* b = Se + ((size_t)(c / P1) * nt + r) * P1 + c % P1;
    const double t0 = *a;
    *a = *b;
    *b = t0;
  }
  __syncthreads();
  // the same arithmetic as the condensation's preconditioned rows
  for (int idx = threadIdx.x; idx < nt * nt; idx += blockDim.x) {
    const int j = idx / nt, r = idx - j * nt;
    const int k = r / P1, t = r - k * P1;
    double acc = 0.0;
    for (int t2 = 0; t2 < P1; ++t2) acc += dt.Ghinv[t * P1 + t2] * Se[((size_t)k * nt + j) * P1 + t2];
    const size_t o = (size_t)e * 3 * nt * P1 + ((size_t)k * nt + j) * P1 + t;
    St[o] = acc;
    if (St32) St32[o] = (float)acc;
    if (Stdf) Stdf[o] = df_from(acc);
  }
}

// z <- U^-T z by one warp (U: upper triangle of rows 0..Q-1 of W, row stride ld).
__device__ void solve_ut_warp(const double* W, int Q, int ld, double* z, int lane) {
  for (int i = 0; i < Q; ++i) {
    const double* row = W + (size_t)i * ld;
    const double zi = z[i] / row[i];
    __syncwarp();
    if (lane == 0) z[i] = zi;
    for (int j = i + 1 + lane; j < Q; j += 32) z[j] -= row[j] * zi;
    __syncwarp();
  }
}

// Element part of the adjoint right-hand side: gadj_e = -(L^-1 P B_u)^T U^-T r_e.
__global__ void __launch_bounds__(128) adjoint_rhs_kernel(Params P, const double* ws, const double* r, double* gel) {
  const int e = blockIdx.x;
  if (e >= P.N) return;
  const int Q = P.Q, nt = P.n_t, ld = P.ld;
  const double* W = ws + (size_t)e * P.R * ld;
  extern __shared__ double z[];   // Q
  for (int i = threadIdx.x; i < Q; i += blockDim.x) z[i] = r[(size_t)e * Q + i];
  __syncthreads();
  if (threadIdx.x < 32) solve_ut_warp(W, Q, ld, z, threadIdx.x);
  __syncthreads();
  for (int j = threadIdx.x; j < nt; j += blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < Q; ++i) acc += W[(size_t)i * ld + Q + j] * z[i];
    gel[(size_t)e * nt + j] = -acc;
  }
}

// Element-local trace vector from a global one (zero on boundary edges).
__device__ __forceinline__ void gather_trace(const Params& P, int e, const double* x, const double* ghat, double* xe) {
  int code[3], flip[3];
  elem_edges(e, P.n, code, flip);
  for (int c = threadIdx.x; c < P.n_t; c += blockDim.x) {
    const int k = c / P.P1, t = c - k * P.P1;
    const int s = flip[k] ? P.P - t : t;
    double v = 0.0;
    if (code[k] >= 0) v = x[(size_t)code[k] * P.P1 + s];
    else if (ghat) v = ghat[(size_t)(-1 - code[k]) * P.P1 + s];
    xe[c] = v;
  }
}

// mu_e = P^T L^-T (U^-T r_e - M21^T nu_e).
__global__ void __launch_bounds__(128) adjoint_recover_kernel(Params P, const double* ws, const int* piv,
                                                             const double* r, const double* nu, double* mu) {
  const int e = blockIdx.x;
  if (e >= P.N) return;
  const int Q = P.Q, nt = P.n_t, ld = P.ld;
  const double* W = ws + (size_t)e * P.R * ld;
  extern __shared__ double sm[];
  double* z = sm;          // Q
  double* nue = z + Q;     // n_t
  const int tid = threadIdx.x, lane = tid & 31;
  for (int i = tid; i < Q; i += blockDim.x) z[i] = r[(size_t)e * Q + i];
  gather_trace(P, e, nu, nullptr, nue);
  __syncthreads();
  if (tid < 32) solve_ut_warp(W, Q, ld, z, lane);
  __syncthreads();
  for (int i = tid; i < Q; i += blockDim.x) {
    double acc = 0.0;
    for (int c = 0; c < nt; ++c) acc += W[(size_t)(Q + c) * ld + i] * nue[c];
    z[i] -= acc;
  }
  __syncthreads();
  // L^T (unit upper) back substitution, one warp, row k of L is contiguous
  if (tid < 32) {
    for (int k = Q - 1; k > 0; --k) {
      const double* row = W + (size_t)k * ld;
      const double zk = z[k];
      for (int i = lane; i < k; i += 32) z[i] -= row[i] * zk;
      __syncwarp();
    }
  }
  __syncthreads();
  // P^T: the interchanges in reverse order
  if (tid == 0) {
    const int* pv = piv + (size_t)e * Q;
    for (int c = Q - 1; c >= 0; --c) {
      const int p = pv[c];
      if (p != c) {
        const double t0 = z[c];
        z[c] = z[p];
        z[p] = t0;
      }
    }
  }
  __syncthreads();
  for (int i = tid; i < Q; i += blockDim.x) mu[(size_t)e * Q + i] = z[i];
}

// dJ/dkappa_e = -(T1 + T2 + T3) with the kappa-derivative of the blocks
//   dA_u = detJ (gxx Kxx + gxy Ksym + gyy Kyy) + E / tau_len
//   dB_u[i][c] = -L_k (nxi_k Pxi + neta_k Peta + Fh / tau_len)[i][c] = -dC_u[c][i]
//   dD_u[r][c] = -L_k L_l (n_k . n_l) / detJ Hh[r][c] - [k = l] L_k Gh[t][t2] / tau_len
// T1 = mu^T dA_u u, T2 = mu^T dB_u x + nu^T dC_u u, T3 = nu^T dD_u x,
// and dJ/df_e at every source point (sub-triangle s, point q):
//   (detJ / m^2) wq[q] sum_b mu[subnode(s, b)] phiq[q][b].
__global__ void __launch_bounds__(128) gradient_kernel(Params P, DevTables dt, const double* x, const double* ghat,
                                                      const double* u, const double* mu, const double* nu,
                                                      double* dkappa, double* df) {
  const int e = blockIdx.x;
  if (e >= P.N) return;
  const int Q = P.Q, nt = P.n_t, P1 = P.P1;
  extern __shared__ double sm[];
  double* ue = sm;           // Q
  double* me = ue + Q;       // Q
  double* xe = me + Q;       // n_t
  double* ne = xe + nt;      // n_t
  __shared__ double red[4];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int i = tid; i < Q; i += blockDim.x) {
    ue[i] = u[(size_t)e * Q + i];
    me[i] = mu[(size_t)e * Q + i];
  }
  gather_trace(P, e, x, ghat, xe);
  gather_trace(P, e, nu, nullptr, ne);
  __syncthreads();

  ElemGeom g;
  elem_geom(e, P.n, g);
  const double il = 1.0 / P.tau_len;
  const double gxx = g.gxi[0] * g.gxi[0] + g.gxi[1] * g.gxi[1];
  const double gxy = g.gxi[0] * g.geta[0] + g.gxi[1] * g.geta[1];
  const double gyy = g.geta[0] * g.geta[0] + g.geta[1] * g.geta[1];
  double nxi[3], neta[3];
  for (int k = 0; k < 3; ++k) {
    nxi[k] = g.nrm[k][0] * g.gxi[0] + g.nrm[k][1] * g.gxi[1];
    neta[k] = g.nrm[k][0] * g.geta[0] + g.nrm[k][1] * g.geta[1];
  }
  double acc = 0.0;
  // T1 (Q x Q part), one warp per row
  for (int i = warp; i < Q; i += nw) {
    const size_t qi = (size_t)i * Q;
    double s = 0.0;
    for (int j = lane; j < Q; j += 32)
      s += (gxx * dt.Kxx[qi + j] + gxy * dt.Ksym[qi + j] + gyy * dt.Kyy[qi + j]) * ue[j];
    acc += g.detJ * me[i] * s;
  }
  // T1 (E / tau_len part), edge by edge
  for (int idx = tid; idx < 3 * P1 * P1; idx += blockDim.x) {
    const int k = idx / (P1 * P1), tt = idx - k * P1 * P1;
    const int t = tt / P1, t2 = tt - t * P1;
    acc += il * g.L[k] * me[dt.enode[k * P1 + t]] * dt.Gh[tt] * ue[dt.enode[k * P1 + t2]];
  }
  // T2, one warp per row of the Q x n_t tables
  for (int i = warp; i < Q; i += nw) {
    double s = 0.0;
    for (int c = lane; c < nt; c += 32) {
      const int k = c / P1;
      const size_t ic = (size_t)i * nt + c;
      const double w = g.L[k] * (nxi[k] * dt.Pxi[ic] + neta[k] * dt.Peta[ic] + il * dt.Fh[ic]);
      s += w * (ue[i] * ne[c] - me[i] * xe[c]);
    }
    acc += s;
  }
  // T3
  for (int idx = tid; idx < nt * nt; idx += blockDim.x) {
    const int r = idx / nt, c = idx - r * nt;
    const int k = r / P1, t = r - k * P1, l = c / P1, t2 = c - l * P1;
    const double nn = g.nrm[k][0] * g.nrm[l][0] + g.nrm[k][1] * g.nrm[l][1];
    double d = -g.L[k] * g.L[l] * nn / g.detJ * dt.Hh[idx];
    if (k == l) d -= il * g.L[k] * dt.Gh[t * P1 + t2];
    acc += ne[r] * d * xe[c];
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w];
    dkappa[e] = -s;
  }
  if (df) {
    const double sc = g.detJ / (double)(P.m * P.m);
    for (int idx = tid; idx < P.n_qp; idx += blockDim.x) {
      const int s = idx / P.nqs, q = idx - s * P.nqs;
      double v = 0.0;
      for (int b = 0; b < P.nloc; ++b) v += me[dt.subnode[s * P.nloc + b]] * dt.phiq[q * P.nloc + b];
      df[(size_t)e * P.n_qp + idx] = sc * dt.wq[q] * v;
    }
  }
}

// ------------------------------------------------------------------ launchers
cudaError_t launch_copy_kappa(const Params& P, const double* src, double* kappa, int* bad, cudaStream_t st) {
  copy_kappa_kernel<<<(P.N + 255) / 256, 256, 0, st>>>(P.N, src, kappa, bad);
  return cudaGetLastError();
}

cudaError_t launch_transpose(const Params& P, const DevTables& dt, double* S, double* St, float* St32, float2* Stdf,
                             cudaStream_t st) {
  transpose_kernel<<<P.N, 256, 0, st>>>(P, dt, S, St, St32, Stdf);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_rhs(const Params& P, const double* ws, const double* r, double* gel, cudaStream_t st) {
  adjoint_rhs_kernel<<<P.N, 128, (size_t)P.Q * sizeof(double), st>>>(P, ws, r, gel);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_recover(const Params& P, const double* ws, const int* piv, const double* r,
                                   const double* nu, double* mu, cudaStream_t st) {
  adjoint_recover_kernel<<<P.N, 128, (size_t)(P.Q + P.n_t) * sizeof(double), st>>>(P, ws, piv, r, nu, mu);
  return cudaGetLastError();
}

cudaError_t launch_gradient(const Params& P, const DevTables& dt, const double* x, const double* ghat,
                            const double* u, const double* mu, const double* nu, double* dkappa, double* df,
                            cudaStream_t st) {
  gradient_kernel<<<P.N, 128, (size_t)(2 * P.Q + 2 * P.n_t) * sizeof(double), st>>>(P, dt, x, ghat, u, mu, nu,
                                                                                     dkappa, df);
  return cudaGetLastError();
}

}  // namespace mehdg
