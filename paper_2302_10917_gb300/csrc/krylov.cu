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
  const double hn = sqrt(warp_sum_partials(part, G));
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
  if ((e = cudaMalloc(&c->d_r, 2 * n * sizeof(double))) != cudaSuccess) return e;
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
  double* V = c->d_V;
  double* w = c->d_w;
  double* bt = c->d_r;          // D^-1 g
  double* rr = c->d_r + n;      // scratch residual
  double* part = c->d_part;
  rep = hdg_solve_report{};

  // ||g||, D^-1 g, ||D^-1 g||
  axpby_norm_kernel<<<KG, KT, 0, st>>>(1.0, g, 0.0, g, rr, n, part);
  sum_partials_kernel<<<1, 32, 0, st>>>(part, KG, sm + L.sc + 5);
  LAUNCHED(2);
  const double gnorm = std::sqrt(read_scalar(c, sm + L.sc + 5, cu));
  cu.ok(launch_face_dinv(P, c->dt.Ghinv, c->d_escale, g, bt, st));
  axpby_norm_kernel<<<KG, KT, 0, st>>>(1.0, bt, 0.0, bt, rr, n, part);
  sum_partials_kernel<<<1, 32, 0, st>>>(part, KG, sm + L.sc + 5);
  LAUNCHED(3);
  const double btnorm = std::sqrt(read_scalar(c, sm + L.sc + 5, cu));
  if (cu.err != cudaSuccess) return fail(c, HDG_ERR_CUDA, cudaGetErrorString(cu.err));
  if (gnorm == 0.0) {
    cu.ok(cudaMemsetAsync(x, 0, n * sizeof(double), st));
    cu.ok(cudaStreamSynchronize(st));
    rep.converged = 1;
    return cu.err == cudaSuccess ? HDG_OK : fail(c, HDG_ERR_CUDA, cudaGetErrorString(cu.err));
  }
  double target = o.tol * btnorm;
  int its = 0;
  double rel = 1.0;
  while (true) {
    // r0 = D^-1 g - D^-1 S x ; V0 = r0 / beta
    double tgt = target;
    cu.ok(cudaMemcpyAsync(sm + L.sc + 2, &tgt, sizeof(double), cudaMemcpyHostToDevice, st));
    {
      ProfScope ps(c, HDG_PROF_APPLY);
      cu.ok(launch_apply64(P, c->d_St, x, w, c->d_escale, nullptr, st));
    }
    axpby_norm_kernel<<<KG, KT, 0, st>>>(1.0, bt, -1.0, w, rr, n, part);
    cycle_init_kernel<<<1, 32, 0, st>>>(sm, L, fl, part, KG);
    scale_kernel<<<KG, KT, 0, st>>>(rr, sm, L.sc + 4, V, n, fl);
    LAUNCHED(4);
    const int jmax = std::min(K, o.maxit - its);
    std::vector<size_t> mark(jmax + 1, 0);   // profiling entries recorded before Arnoldi step j
    for (int j = 0; j < jmax; ++j) {
      mark[j] = c->prof_ev.size();
      double* Vj = V + (size_t)j * n;
      double* Hcol = sm + L.H + (size_t)j * (K + 1);
      {
        ProfScope ps(c, HDG_PROF_APPLY);
        cu.ok(launch_apply64(P, c->d_St, Vj, w, c->d_escale, fl, st));
      }
      ProfScope po(c, HDG_PROF_ORTHO);
      mdot_kernel<<<KG, KT, 0, st>>>(V, n, j + 1, w, part, fl);
      mdot_reduce_kernel<<<1, 256, 0, st>>>(part, KG, j + 1, Hcol, sm + L.htmp, 0, fl);
      update_kernel<<<KG, KT, 0, st>>>(V, n, j + 1, sm + L.htmp, -1.0, w, nullptr, fl);
      mdot_kernel<<<KG, KT, 0, st>>>(V, n, j + 1, w, part, fl);
      mdot_reduce_kernel<<<1, 256, 0, st>>>(part, KG, j + 1, Hcol, sm + L.htmp, 1, fl);
      update_kernel<<<KG, KT, 0, st>>>(V, n, j + 1, sm + L.htmp, -1.0, w, part, fl);
      givens_kernel<<<1, 32, 0, st>>>(sm, L, fl, part, KG, j);
      scale_kernel<<<KG, KT, 0, st>>>(w, sm, L.sc + 4, V + (size_t)(j + 1) * n, n, fl);
      LAUNCHED(9);
    }
    cu.ok(cudaGetLastError());
    int hflags[2] = {0, 0};
    cu.ok(cudaMemcpyAsync(hflags, fl, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    cu.ok(cudaStreamSynchronize(st));
    if (cu.err != cudaSuccess) return fail(c, HDG_ERR_CUDA, cudaGetErrorString(cu.err));
    const int jused = hflags[F_JUSED];
    if (c->prof_on && jused < jmax) {
      // steps after the stop flag was raised were enqueued but returned at once: not timed work
      for (size_t i = mark[jused]; i < c->prof_ev.size(); ++i) c->prof_pool.push_back(c->prof_ev[i].second);
      c->prof_ev.resize(mark[jused]);
    }
    const double est = read_scalar(c, sm + L.sc + 1, cu);
    its += jused;
    rep.restarts += 1;
    if (jused > 0) {
      lsq_kernel<<<1, 32, 0, st>>>(sm, L, fl);
      update_kernel<<<KG, KT, 0, st>>>(V, n, jused, sm + L.y, 1.0, x, nullptr, nullptr);
      LAUNCHED(2);
    }
    // true residual with the unpreconditioned FP64 operator
    {
      ProfScope ps(c, HDG_PROF_APPLY);
      cu.ok(launch_apply64(P, c->d_S, x, w, nullptr, nullptr, st));
    }
    axpby_norm_kernel<<<KG, KT, 0, st>>>(1.0, g, -1.0, w, rr, n, part);
    sum_partials_kernel<<<1, 32, 0, st>>>(part, KG, sm + L.sc + 5);
    LAUNCHED(3);
    rel = std::sqrt(read_scalar(c, sm + L.sc + 5, cu)) / gnorm;
    if (cu.err != cudaSuccess) return fail(c, HDG_ERR_CUDA, cudaGetErrorString(cu.err));
    rep.iterations = its;
    rep.rel_residual = rel;
    if (rel <= o.tol) {
      rep.converged = 1;
      return HDG_OK;
    }
    if (its >= o.maxit || jused == 0) break;
    if (est <= target) target *= 0.5 * o.tol / rel;
  }
  rep.converged = 0;
  return fail(c, HDG_ERR_NOCONV, "GMRES reached maxit with relative residual " + std::to_string(rel));
}

}  // namespace mehdg
