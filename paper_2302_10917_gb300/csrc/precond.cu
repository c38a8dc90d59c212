// Face-block preconditioner with the exact diagonal blocks of the trace
// operator (HDG_PRECOND_FACE_SCHUR).
//
// The preconditioner of Sec. 6.1 inverts, face by face, the trace-trace block
// of the unreduced system, D_f = -(tau+ + tau-) L_f Gh. The condensed operator
// S = sum_e L_e^T S_e L_e has the diagonal face blocks
//     S_ff = sum over the two sides of S_e restricted to the face's rows and columns
//          = D_f - (the face's part of sum_e C_e A_e^-1 B_e),
// of which D_f is the part without the local solves. This option inverts S_ff
// itself (block Jacobi on the trace system): the same block-diagonal
// structure and the same cost per apply, since S_ff^-1 is folded into the
// stored preconditioned row-blocks of both adjacent elements exactly as
// D_f^-1 is (z_f = S_ff^-1 (y_f,side0 + y_f,side1) = sum_side S_ff^-1 y_f,side),
// and the face scale of the apply becomes 1.
//
// Per face: S_ff (global edge orientation) from the two sides' blocks, its
// inverse by Gauss-Jordan elimination with partial pivoting (one CTA per
// face, the augmented matrix in shared memory); per element face: the stored
// rows S_e[face rows, :] replaced by S_ff^-1 (element orientation) times them.
#include <algorithm>
#include "launch.h"

namespace mehdg {

namespace {

// In-place inverse of the n x n block M[:, 0:n] of the augmented matrix
// M = [A | I] (row stride 2n, shared memory) by Gauss-Jordan elimination with
// partial pivoting; fac: n doubles of shared scratch. Block-wide; returns
// false (on every thread) for a zero pivot.
__device__ bool gj_inverse(double* M, double* fac, int n) {
  const int tid = threadIdx.x, nthr = blockDim.x, w = 2 * n;
  __shared__ int s_pr;
  __shared__ double s_pv;
  for (int c = 0; c < n; ++c) {
    if (tid == 0) {
      int best = c;
      double bv = fabs(M[c * w + c]);
      for (int r = c + 1; r < n; ++r) {
        const double v = fabs(M[r * w + c]);
        if (v > bv) { bv = v; best = r; }
      }
      s_pr = best;
      s_pv = M[best * w + c];
    }
    __syncthreads();
    const int pr = s_pr;
    const double pv = s_pv;
    if (pv == 0.0) return false;
    if (pr != c)
      for (int j = tid; j < w; j += nthr) {
        const double t = M[c * w + j];
        M[c * w + j] = M[pr * w + j];
        M[pr * w + j] = t;
      }
    __syncthreads();
    const double inv = 1.0 / pv;
    for (int j = tid; j < w; j += nthr) M[c * w + j] *= inv;
    for (int r = tid; r < n; r += nthr) fac[r] = (r == c) ? 0.0 : M[r * w + c];
    __syncthreads();
    for (int idx = tid; idx < n * w; idx += nthr) {
      const int r = idx / w, j = idx - r * w;
      if (r != c) M[idx] -= fac[r] * M[c * w + j];
    }
    __syncthreads();
  }
  return true;
}

// ------------------------------------------------------------ uniform level
__global__ void face_schur_kernel(Params P, const double* __restrict__ S, double* __restrict__ Pinv,
                                  int* __restrict__ bad) {
  const int f = blockIdx.x;
  if (f >= P.n_int) return;
  const int n = P.P1, w = 2 * n, nt = P.n_t, PP = P.P;
  extern __shared__ double sm[];
  double* M = sm;            // [n][2n]
  double* fac = sm + n * w;  // [n]
  int e[2], k[2], fl[2];
  double len;
  edge_sides(f, P.n, e, k, fl, &len);
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int s1 = idx / n, s2 = idx - s1 * n;
    double v = 0.0;
    for (int sd = 0; sd < 2; ++sd) {
      const int t1 = fl[sd] ? PP - s1 : s1, t2 = fl[sd] ? PP - s2 : s2;
      // S[e][k][j][t] = S_e(k P1 + t, j): row t1 of face k, column k P1 + t2
      v += S[(((size_t)e[sd] * 3 + k[sd]) * nt + (size_t)k[sd] * n + t2) * n + t1];
    }
    M[s1 * w + s2] = v;
    M[s1 * w + n + s2] = (s1 == s2) ? 1.0 : 0.0;
  }
  __syncthreads();
  const bool ok = gj_inverse(M, fac, n);
  if (!ok && threadIdx.x == 0) atomicAdd(bad, 1);
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int s1 = idx / n, s2 = idx - s1 * n;
    Pinv[(size_t)f * n * n + idx] = ok ? M[s1 * w + n + s2] : 0.0;
  }
}

// St[e][k][j][t] = sum_t2 S_ff^-1(t, t2) S[e][k][j][t2] on interior faces (element orientation);
// trans: the blocks hold S_e^T (hdg_transpose), whose face blocks are S_ff^T, inverse (S_ff^-1)^T
__global__ void fold_kernel(Params P, const double* __restrict__ S, const double* __restrict__ Pinv, int trans,
                            double* __restrict__ St, float* __restrict__ St32) {
  const int e = blockIdx.x / 3, k = blockIdx.x - 3 * (blockIdx.x / 3);
  if (e >= P.N) return;
  int code[3], flip[3];
  elem_edges(e, P.n, code, flip);
  if (code[k] < 0) return;
  const int n = P.P1, nt = P.n_t, PP = P.P;
  extern __shared__ double Li[];    // [n][n]
  const double* Pf = Pinv + (size_t)code[k] * n * n;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int t = idx / n, t2 = idx - t * n;
    const int s = flip[k] ? PP - t : t, s2 = flip[k] ? PP - t2 : t2;
    Li[idx] = trans ? Pf[s2 * n + s] : Pf[s * n + s2];
  }
  __syncthreads();
  const size_t base = ((size_t)e * 3 + k) * nt * n;
  for (int idx = threadIdx.x; idx < nt * n; idx += blockDim.x) {
    const int j = idx / n, t = idx - j * n;
    const double* col = S + base + (size_t)j * n;
    double acc = 0.0;
    for (int t2 = 0; t2 < n; ++t2) acc += Li[t * n + t2] * col[t2];
    St[base + idx] = acc;
    if (St32) St32[base + idx] = (float)acc;
  }
}

// z_f = S_ff^-1 y_f (trans: (S_ff^-1)^T y_f) on one FP64 vector (global orientation)
__global__ void face_pinv_kernel(Params P, const double* __restrict__ Pinv, int trans, const double* __restrict__ y,
                                 double* __restrict__ z) {
  const int64_t total = (int64_t)P.n_int * P.P1;
  const int n = P.P1;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int f = (int)(idx / n), s = (int)(idx - (int64_t)f * n);
    const double* Pf = Pinv + (size_t)f * n * n;
    const double* yf = y + (size_t)f * n;
    double acc = 0.0;
    for (int t = 0; t < n; ++t) acc += (trans ? Pf[t * n + s] : Pf[s * n + t]) * yf[t];
    z[idx] = acc;
  }
}

// --------------------------------------------------------------- level mesh
// Lifted blocks: element e's n_t,e x n_t,e block column-major at soff[e];
// its face block on side sd of face f starts at local row ez[2f+sd] - zoff[e].
__global__ void lv_face_schur_kernel(LevelDev L, const double* __restrict__ S, double* __restrict__ Pinv,
                                     int* __restrict__ bad) {
  const int f = blockIdx.x;
  if (f >= L.n_int) return;
  const int n = (int)(L.eoff[f + 1] - L.eoff[f]), w = 2 * n;
  extern __shared__ double sm[];
  double* M = sm;
  double* fac = sm + n * w;
  const int fl = L.eflip[f];
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int s1 = idx / n, s2 = idx - s1 * n;
    double v = 0.0;
    for (int sd = 0; sd < 2; ++sd) {
      const int e = L.eside[2 * f + sd], nt = L.nte[e];
      const int a0 = L.ez[2 * f + sd] - L.zoff[e];
      const bool flp = (fl >> sd) & 1;
      const int t1 = flp ? n - 1 - s1 : s1, t2 = flp ? n - 1 - s2 : s2;
      v += S[L.soff[e] + (int64_t)(a0 + t2) * nt + (a0 + t1)];
    }
    M[s1 * w + s2] = v;
    M[s1 * w + n + s2] = (s1 == s2) ? 1.0 : 0.0;
  }
  __syncthreads();
  const bool ok = gj_inverse(M, fac, n);
  if (!ok && threadIdx.x == 0) atomicAdd(bad, 1);
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int s1 = idx / n, s2 = idx - s1 * n;
    Pinv[L.poff[f] + idx] = ok ? M[s1 * w + n + s2] : 0.0;
  }
}

// interior face rows of element e's preconditioned block: S_ff^-1 (element orientation) S_e[face rows, :]
__global__ void lv_fold_kernel(LevelDev L, const double* __restrict__ S, const double* __restrict__ Pinv,
                               double* __restrict__ St) {
  const int e = blockIdx.x;
  if (e >= L.N) return;
  const int nt = L.nte[e];
  const int64_t so = L.soff[e];
  int code[3], flip[3];
  elem_edges(e, L.n, code, flip);
  extern __shared__ double Li[];   // [n][n] of one face at a time
  int a0 = 0;
  for (int k = 0; k < 3; ++k) {
    const int n = (1 << face_level(L.flev, L.elev, e, code[k])) * L.p + 1;
    if (code[k] >= 0) {
      const double* Pf = Pinv + L.poff[code[k]];
      for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int t = idx / n, t2 = idx - t * n;
        const int s = flip[k] ? n - 1 - t : t, s2 = flip[k] ? n - 1 - t2 : t2;
        Li[idx] = Pf[s * n + s2];
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < nt * n; idx += blockDim.x) {
        const int b = idx / n, t = idx - b * n;
        const double* col = S + so + (int64_t)b * nt + a0;
        double acc = 0.0;
        for (int t2 = 0; t2 < n; ++t2) acc += Li[t * n + t2] * col[t2];
        St[so + (int64_t)b * nt + a0 + t] = acc;
      }
      __syncthreads();
    }
    a0 += n;
  }
}

__global__ void lv_face_pinv_kernel(LevelDev L, const double* __restrict__ Pinv, const double* __restrict__ y,
                                    double* __restrict__ z, int nrhs, int64_t vstride) {
  const int64_t total = L.N_tr * nrhs;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / L.N_tr);
    const int64_t i = idx - (int64_t)r * L.N_tr;
    const int f = L.dof_edge[i];
    const int64_t b0 = L.eoff[f];
    const int s = (int)(i - b0), n = (int)(L.eoff[f + 1] - b0);
    const double* row = Pinv + L.poff[f] + (int64_t)s * n;
    const double* yf = y + (size_t)r * vstride + b0;
    double acc = 0.0;
    for (int t = 0; t < n; ++t) acc += row[t] * yf[t];
    z[(size_t)r * vstride + i] = acc;
  }
}

cudaError_t set_smem(const void* fn, size_t sm) {
  if (sm <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

}  // namespace

cudaError_t launch_face_schur(const Params& P, const double* S, double* Pinv, double* St, float* St32, int* bad,
                              cudaStream_t st) {
  const size_t sm = (size_t)(2 * P.P1 * P.P1 + P.P1) * sizeof(double);
  cudaError_t e = set_smem((const void*)face_schur_kernel, sm);
  if (e != cudaSuccess) return e;
  face_schur_kernel<<<P.n_int, 128, sm, st>>>(P, S, Pinv, bad);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_face_fold(P, S, Pinv, 0, St, St32, st);
}

cudaError_t launch_face_fold(const Params& P, const double* S, const double* Pinv, int trans, double* St, float* St32,
                             cudaStream_t st) {
  const size_t sm2 = (size_t)P.P1 * P.P1 * sizeof(double);
  cudaError_t e = set_smem((const void*)fold_kernel, sm2);
  if (e != cudaSuccess) return e;
  fold_kernel<<<3 * P.N, 128, sm2, st>>>(P, S, Pinv, trans, St, St32);
  return cudaGetLastError();
}

cudaError_t launch_face_pinv(const Params& P, const double* Pinv, int trans, const double* y, double* z,
                             cudaStream_t st) {
  face_pinv_kernel<<<1024, 256, 0, st>>>(P, Pinv, trans, y, z);
  return cudaGetLastError();
}

cudaError_t launch_level_face_schur(const LevelDev& L, int max_nf, const double* S, double* Pinv, double* St,
                                    int* bad, cudaStream_t st) {
  const size_t sm = (size_t)(2 * max_nf * max_nf + max_nf) * sizeof(double);
  cudaError_t e = set_smem((const void*)lv_face_schur_kernel, sm);
  if (e != cudaSuccess) return e;
  lv_face_schur_kernel<<<L.n_int, 128, sm, st>>>(L, S, Pinv, bad);
  const size_t sm2 = (size_t)max_nf * max_nf * sizeof(double);
  if ((e = set_smem((const void*)lv_fold_kernel, sm2)) != cudaSuccess) return e;
  lv_fold_kernel<<<L.N, 128, sm2, st>>>(L, S, Pinv, St);
  return cudaGetLastError();
}

cudaError_t launch_level_face_pinv(const LevelDev& L, const double* Pinv, const double* y, double* z, int nrhs,
                                   int64_t vstride, cudaStream_t st) {
  const int64_t total = L.N_tr * nrhs;
  const int g = (int)std::min<int64_t>(152 * 8, (total + 255) / 256);
  lv_face_pinv_kernel<<<g, 256, 0, st>>>(L, Pinv, y, z, nrhs, vstride);
  return cudaGetLastError();
}

}  // namespace mehdg
