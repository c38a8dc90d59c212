// C ABI of the macro-element HDG library (declarations and the paper passages
// each entry point follows are in include/mehdg.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <stdexcept>
#include <string>
#include <nvtx3/nvToolsExt.h>
#include "launch.h"

// Tracing: every phase entry point is an NVTX range (header-only NVTX; the
// calls do nothing unless a profiler or tracing tool is attached).
namespace {
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace

using namespace mehdg;

namespace {

hdg_status set_err(hdg_ctx* c, hdg_status s, const std::string& m) {
  if (c) c->err = m;
  return s;
}

hdg_status cuda_err(hdg_ctx* c, cudaError_t e, const char* where) {
  return set_err(c, e == cudaErrorMemoryAllocation ? HDG_ERR_OOM : HDG_ERR_CUDA,
                 std::string(where) + ": " + cudaGetErrorString(e));
}

template <typename T>
cudaError_t dev_alloc(hdg_ctx* c, T** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e == cudaSuccess) c->bytes += count * sizeof(T);
  return e;
}

template <typename T>
void dev_free(hdg_ctx* c, T*& p, size_t count) {
  if (p) {
    cudaFree((void*)p);
    c->bytes -= std::min(c->bytes, count * sizeof(T));
  }
  p = nullptr;
}

// Physical source points, [N][n_qp][2].
__global__ void quad_points_kernel(Params P, DevTables dt, double* xy) {
  const int64_t total = (int64_t)P.N * P.n_qp;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(idx / P.n_qp);
    const int r = (int)(idx - (int64_t)e * P.n_qp);
    const int s = r / P.nqs, q = r - s * P.nqs;
    const int qj = q / P.ng, qi = q - qj * P.ng;
    const double xh = dt.uq[qi] * (1.0 - dt.uq[qj]), eh = dt.uq[qj];
    const int* c = dt.subtri + 6 * s;
    const double xi = (c[0] + xh * (c[2] - c[0]) + eh * (c[4] - c[0])) / P.m;
    const double eta = (c[1] + xh * (c[3] - c[1]) + eh * (c[5] - c[1])) / P.m;
    double v[3][2];
    elem_vertices(e, P.n, v);
    xy[2 * idx + 0] = v[0][0] + xi * (v[1][0] - v[0][0]) + eta * (v[2][0] - v[0][0]);
    xy[2 * idx + 1] = v[0][1] + xi * (v[1][1] - v[0][1]) + eta * (v[2][1] - v[0][1]);
  }
}

// Dirichlet-data points, [4n][m * ngb][2].
__global__ void bnd_points_kernel(Params P, DevTables dt, double* xy) {
  const int64_t total = (int64_t)P.n_bnd * P.n_bqp;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(idx / P.n_bqp);
    const int r = (int)(idx - (int64_t)b * P.n_bqp);
    const int s = r / P.ngb, q = r - s * P.ngb;
    const int side = b / P.n, k = b - side * P.n;
    const double h = 1.0 / P.n;
    double a0[2], a1[2];
    if (side == 0) { a0[0] = k * h; a0[1] = 0.0; a1[0] = (k + 1) * h; a1[1] = 0.0; }
    else if (side == 1) { a0[0] = k * h; a0[1] = 1.0; a1[0] = (k + 1) * h; a1[1] = 1.0; }
    else if (side == 2) { a0[0] = 0.0; a0[1] = k * h; a1[0] = 0.0; a1[1] = (k + 1) * h; }
    else { a0[0] = 1.0; a0[1] = k * h; a1[0] = 1.0; a1[1] = (k + 1) * h; }
    const double th = (s + dt.bu[q]) / P.m;
    xy[2 * idx + 0] = a0[0] + th * (a1[0] - a0[0]);
    xy[2 * idx + 1] = a0[1] + th * (a1[1] - a0[1]);
  }
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

constexpr size_t kMaxSmem = 227 * 1024;   // dynamic shared memory one CTA may use on sm_103a

}  // namespace

namespace mehdg {
// Copy the host tables into one device allocation.
cudaError_t upload_ref_tables(const RefTables& T, DevTables& d, void** dmem, size_t* bytes, cudaStream_t st) {
  struct Item { const void* src; size_t bytes; void** dst; };
  std::vector<Item> items = {
      {T.Dxi.data(), T.Dxi.size() * 8, (void**)&d.Dxi},   {T.Deta.data(), T.Deta.size() * 8, (void**)&d.Deta},
      {T.Kxx.data(), T.Kxx.size() * 8, (void**)&d.Kxx},   {T.Kyy.data(), T.Kyy.size() * 8, (void**)&d.Kyy},
      {T.Ksym.data(), T.Ksym.size() * 8, (void**)&d.Ksym}, {T.Xxi.data(), T.Xxi.size() * 8, (void**)&d.Xxi},
      {T.Xeta.data(), T.Xeta.size() * 8, (void**)&d.Xeta}, {T.Fh.data(), T.Fh.size() * 8, (void**)&d.Fh},
      {T.Pxi.data(), T.Pxi.size() * 8, (void**)&d.Pxi},   {T.Peta.data(), T.Peta.size() * 8, (void**)&d.Peta},
      {T.Yh.data(), T.Yh.size() * 8, (void**)&d.Yh},      {T.Hh.data(), T.Hh.size() * 8, (void**)&d.Hh},
      {T.XxiT.data(), T.XxiT.size() * 8, (void**)&d.XxiT}, {T.XetaT.data(), T.XetaT.size() * 8, (void**)&d.XetaT},
      {T.YhT.data(), T.YhT.size() * 8, (void**)&d.YhT},
      {T.Gh.data(), T.Gh.size() * 8, (void**)&d.Gh},      {T.Ghinv.data(), T.Ghinv.size() * 8, (void**)&d.Ghinv},
      {T.phiq.data(), T.phiq.size() * 8, (void**)&d.phiq}, {T.wq.data(), T.wq.size() * 8, (void**)&d.wq},
      {T.uq.data(), T.uq.size() * 8, (void**)&d.uq},      {T.bpsi.data(), T.bpsi.size() * 8, (void**)&d.bpsi},
      {T.bw.data(), T.bw.size() * 8, (void**)&d.bw},      {T.bu.data(), T.bu.size() * 8, (void**)&d.bu},
      {T.enode.data(), T.enode.size() * 4, (void**)&d.enode}, {T.subtri.data(), T.subtri.size() * 4, (void**)&d.subtri},
      {T.subnode.data(), T.subnode.size() * 4, (void**)&d.subnode},
      {T.ns_ptr.data(), T.ns_ptr.size() * 4, (void**)&d.ns_ptr}, {T.ns_idx.data(), T.ns_idx.size() * 4, (void**)&d.ns_idx},
      {T.Sxx.data(), T.Sxx.size() * 8, (void**)&d.Sxx},   {T.Syy.data(), T.Syy.size() * 8, (void**)&d.Syy},
      {T.Ssym.data(), T.Ssym.size() * 8, (void**)&d.Ssym}, {T.Lx_xx.data(), T.Lx_xx.size() * 8, (void**)&d.Lx_xx},
      {T.Lx_xy.data(), T.Lx_xy.size() * 8, (void**)&d.Lx_xy}, {T.Lx_yy.data(), T.Lx_yy.size() * 8, (void**)&d.Lx_yy},
      {T.Ly_xx.data(), T.Ly_xx.size() * 8, (void**)&d.Ly_xx}, {T.Ly_xy.data(), T.Ly_xy.size() * 8, (void**)&d.Ly_xy},
      {T.Ly_yy.data(), T.Ly_yy.size() * 8, (void**)&d.Ly_yy}, {T.dphq.data(), T.dphq.size() * 8, (void**)&d.dphq},
  };
  // split-FP32 copies: hi = (float) v, lo = (float) (v - hi)
  std::vector<std::vector<float>> split;
  auto add_split = [&](const std::vector<double>& v, float2** dst) {
    std::vector<float> h(2 * v.size());
    for (size_t i = 0; i < v.size(); ++i) {
      const float hi = (float)v[i];
      h[2 * i] = hi;
      h[2 * i + 1] = (float)(v[i] - (double)hi);
    }
    split.push_back(std::move(h));
    items.push_back({split.back().data(), split.back().size() * 4, (void**)dst});
  };
  split.reserve(19);
  add_split(T.Kxx, &d.Kxx2); add_split(T.Kyy, &d.Kyy2); add_split(T.Ksym, &d.Ksym2);
  add_split(T.Dxi, &d.Dxi2); add_split(T.Deta, &d.Deta2); add_split(T.Fh, &d.Fh2);
  add_split(T.Pxi, &d.Pxi2); add_split(T.Peta, &d.Peta2); add_split(T.Hh, &d.Hh2); add_split(T.Gh, &d.Gh2);
  {
    const std::vector<double>* sup[9] = {&T.Sxx, &T.Ssym, &T.Syy, &T.Lx_xx, &T.Lx_xy, &T.Lx_yy,
                                         &T.Ly_xx, &T.Ly_xy, &T.Ly_yy};
    for (int k = 0; k < 9; ++k) add_split(*sup[k], &d.Sup2[k]);
  }
  size_t total = 0;
  for (auto& it : items) total += round_up(it.bytes, 256);
  cudaError_t e = cudaMalloc(dmem, total);
  if (e != cudaSuccess) return e;
  *bytes = total;
  std::vector<unsigned char> host(total, 0);
  size_t off = 0;
  for (auto& it : items) {
    if (it.bytes) std::memcpy(host.data() + off, it.src, it.bytes);
    *it.dst = (unsigned char*)*dmem + off;
    off += round_up(it.bytes, 256);
  }
  e = cudaMemcpyAsync(*dmem, host.data(), total, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}
}  // namespace mehdg

namespace {
cudaError_t upload_tables(hdg_ctx* c) {
  size_t b = 0;
  cudaError_t e = upload_ref_tables(c->ref, c->dt, &c->d_tables, &b, c->stream);
  c->bytes += b;
  return e;
}
}  // namespace

namespace mehdg {
// Fold the recorded event pairs into the per-phase totals and recycle them.
void profile_collect(hdg_ctx* c) {
  if (c->prof_ev.empty()) return;
  cudaStreamSynchronize(c->stream);
  for (auto& it : c->prof_ev) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, it.second.first, it.second.second) == cudaSuccess) {
      c->prof_ms[it.first] += ms;
      c->prof_count[it.first] += 1;
    }
    c->prof_pool.push_back(it.second);
  }
  c->prof_ev.clear();
}
}  // namespace mehdg

extern "C" {

hdg_status hdg_create(const hdg_mesh_desc* d, void* stream, hdg_ctx** out) {
  if (!out) return HDG_ERR_ARG;
  *out = nullptr;
  if (!d) return HDG_ERR_ARG;
  const int64_t N = 2LL * d->n * d->n;
  if (d->n < 1 || d->n > 1448 || d->p < 1 || d->p > 4) return HDG_ERR_ARG;
  if (d->level) {
    for (int64_t e = 0; e < N; ++e)
      if (d->level[e] < 0 || d->level[e] > kMaxLevel) return HDG_ERR_ARG;
  } else if (d->m < 1 || d->m > 16) {
    return HDG_ERR_ARG;
  }
  if (!(d->tau_len > 0.0) || !std::isfinite(d->beta[0]) || !std::isfinite(d->beta[1])) return HDG_ERR_ARG;
  for (int s = 0; s < 4; ++s)
    if (d->bc[s] != 0) return HDG_ERR_ARG;
  if (d->supg != 0 && d->supg != 1) return HDG_ERR_ARG;
  if (!d->kappa && !(d->kappa0 >= 0.0 && std::isfinite(d->kappa0))) return HDG_ERR_ARG;
  if (d->kappa)
    for (int64_t e = 0; e < N; ++e)
      if (!(d->kappa[e] >= 0.0) || !std::isfinite(d->kappa[e])) return HDG_ERR_ARG;
  const int P_ = (d->level ? (1 << kMaxLevel) : d->m) * d->p;
  const int64_t n_int = (int64_t)d->n * d->n + 2LL * d->n * (d->n - 1);
  if (n_int * (P_ + 1) > 0x7fffffffLL) return HDG_ERR_ARG;

  hdg_ctx* c = new (std::nothrow) hdg_ctx();
  if (!c) return HDG_ERR_OOM;
  c->stream = (cudaStream_t)stream;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    *out = c;
    return set_err(c, HDG_ERR_CUDA, std::string("no usable CUDA device: ") + cudaGetErrorString(e));
  }
  // the bounds-checked build's error word (one int; zero in the regular build)
  if ((e = dev_alloc(c, &c->d_oob, 1)) != cudaSuccess || (e = cudaMemset(c->d_oob, 0, sizeof(int))) != cudaSuccess) {
    *out = c;
    return cuda_err(c, e, "bounds word");
  }
  if (d->level) {
    // per-element refinement levels: kappa here, everything else in the level mesh
    *out = c;
    std::vector<double> kap(N, d->kappa0);
    if (d->kappa) std::copy(d->kappa, d->kappa + N, kap.begin());
    if ((e = dev_alloc(c, &c->d_kappa, N)) != cudaSuccess) return cuda_err(c, e, "kappa");
    if ((e = cudaMemcpyAsync(c->d_kappa, kap.data(), N * 8, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
      return cuda_err(c, e, "kappa upload");
    const hdg_status s = level_create(c, d);
    if (s != HDG_OK) return s;
    c->alloc_nrhs = 0;
    c->d_tables = c->lv->d_mem;   // marks the context initialised (owned by the level mesh)
    return HDG_OK;
  }
  try {
    build_reference_tables(d->m, d->p, c->ref);
  } catch (const std::exception& ex) {
    *out = c;
    return set_err(c, HDG_ERR_ARG, ex.what());
  }
  const RefTables& T = c->ref;
  Params& P = c->prm;
  P.oob = c->d_oob;
  P.n = d->n; P.m = d->m; P.p = d->p; P.P = T.P; P.P1 = T.P1; P.Q = T.Q; P.n_t = T.n_t;
  P.N = (int)N;
  P.n_int = (int)n_int;
  P.n_bnd = 4 * d->n;
  P.N_tr = (int)(n_int * T.P1);
  P.ng = T.ng; P.nqs = T.nqs; P.nloc = T.nloc; P.nsub = T.nsub; P.n_qp = T.nsub * T.nqs;
  P.ngb = T.ngb; P.n_bqp = d->m * T.ngb;
  P.bx = d->beta[0]; P.by = d->beta[1]; P.babs = std::hypot(d->beta[0], d->beta[1]);
  P.kappa0 = d->kappa0; P.tau_len = d->tau_len;
  P.supg = d->supg;
  P.R = T.Q + T.n_t;
  P.nrhs = 1;
  P.Cc = T.Q + T.n_t + 1;
  P.ld = (int)round_up(P.Cc, 4);
  *out = c;
  if (condense_smem_bytes(P) > kMaxSmem)
    return set_err(c, HDG_ERR_ARG, "level m = " + std::to_string(d->m) + ", p = " + std::to_string(d->p) +
                                       ": one element's panel needs " + std::to_string(condense_smem_bytes(P) / 1024) +
                                       " KB of shared memory (at most 227 KB)");
  if ((e = upload_tables(c)) != cudaSuccess) return cuda_err(c, e, "uploading reference tables");
  std::vector<double> kap(N, d->kappa0);
  if (d->kappa) std::copy(d->kappa, d->kappa + N, kap.begin());
  if ((e = dev_alloc(c, &c->d_kappa, N)) != cudaSuccess) return cuda_err(c, e, "kappa");
  if ((e = cudaMemcpyAsync(c->d_kappa, kap.data(), N * 8, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
    return cuda_err(c, e, "kappa upload");
  if ((e = dev_alloc(c, &c->d_escale, P.n_int)) != cudaSuccess) return cuda_err(c, e, "face scales");
  c->launches += 1;
  if ((e = launch_face_scale(P, c->d_kappa, c->d_escale, c->stream)) != cudaSuccess) return cuda_err(c, e, "face scales");
  if ((e = dev_alloc(c, &c->d_ghat, (size_t)P.n_bnd * P.P1)) != cudaSuccess) return cuda_err(c, e, "ghat");
  if ((e = cudaMemsetAsync(c->d_ghat, 0, (size_t)P.n_bnd * P.P1 * 8, c->stream)) != cudaSuccess)
    return cuda_err(c, e, "ghat");
  c->alloc_nrhs = 1;
  // hdg_condense_static's scratch array exists from here on (its module is loaded now, not at its first call)
  if ((e = static_scratch_prepare()) != cudaSuccess) return cuda_err(c, e, "static scratch array");
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_err(c, e, "create");
  return HDG_OK;
}

hdg_status hdg_info(const hdg_ctx* c, hdg_info_t* out) {
  if (!c || !out) return HDG_ERR_ARG;
  const Params& P = c->prm;
  out->N = P.N; out->Q = P.Q; out->n_t = P.n_t; out->N_tr = P.N_tr;
  out->n_int_edges = P.n_int; out->n_bnd_edges = P.n_bnd; out->n_qp = P.n_qp; out->n_bqp = P.n_bqp;
  out->device_bytes = c->bytes;
  out->launches = c->launches;
  if (c->lv) {
    const LevelMesh& L = *c->lv;
    int64_t qmax = 0;
    for (int64_t e = 0; e < P.N; ++e) qmax = std::max(qmax, L.uoff[e + 1] - L.uoff[e]);
    out->Q = qmax;
    out->n_qp = 0;
    out->n_bqp = 0;
    out->levels = 1;
    out->n_qp_total = L.qoff.back();
    out->n_bqp_total = L.boff.back();
    out->n_u_total = L.uoff.back();
    out->n_s_total = L.ns;
  } else {
    out->levels = 0;
    out->n_qp_total = (int64_t)P.N * P.n_qp;
    out->n_bqp_total = (int64_t)P.n_bnd * P.n_bqp;
    out->n_u_total = (int64_t)P.N * P.Q;
    out->n_s_total = (int64_t)P.N * P.n_t * P.n_t;
  }
  out->bounds_error = 0;
  if (c->d_oob) {
    // the first failing index check of the bounds-checked build (synchronises the stream)
    int code = 0;
    if (cudaMemcpyAsync(&code, c->d_oob, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      return HDG_ERR_CUDA;
    out->bounds_error = code;
  }
  return HDG_OK;
}

hdg_status hdg_offsets(const hdg_ctx* cc, int which, int64_t* out) {
  hdg_ctx* c = const_cast<hdg_ctx*>(cc);
  if (!c || !out) return HDG_ERR_ARG;
  if (!c->d_tables) return set_err(c, HDG_ERR_STATE, "context not initialised");
  const Params& P = c->prm;
  const LevelMesh* L = c->lv;
  auto fill = [&](int64_t count, auto size_of) {
    out[0] = 0;
    for (int64_t i = 0; i < count; ++i) out[i + 1] = out[i] + size_of(i);
  };
  switch (which) {
    case HDG_OFF_SOURCE:
      if (L) std::copy(L->qoff.begin(), L->qoff.end(), out);
      else fill(P.N, [&](int64_t) { return (int64_t)P.n_qp; });
      return HDG_OK;
    case HDG_OFF_DIRICHLET_POINTS:
      if (L) std::copy(L->boff.begin(), L->boff.end(), out);
      else fill(P.n_bnd, [&](int64_t) { return (int64_t)P.n_bqp; });
      return HDG_OK;
    case HDG_OFF_LATTICE:
      if (L) std::copy(L->uoff.begin(), L->uoff.end(), out);
      else fill(P.N, [&](int64_t) { return (int64_t)P.Q; });
      return HDG_OK;
    case HDG_OFF_TRACE:
      if (L) std::copy(L->eoff.begin(), L->eoff.end(), out);
      else fill(P.n_int, [&](int64_t) { return (int64_t)P.P1; });
      return HDG_OK;
    case HDG_OFF_SCHUR:
      if (L) fill(P.N, [&](int64_t e) { return (int64_t)L->nt_e[e] * L->nt_e[e]; });
      else fill(P.N, [&](int64_t) { return (int64_t)P.n_t * P.n_t; });
      return HDG_OK;
    case HDG_OFF_DIRICHLET_TRACE:
      if (L) std::copy(L->goff.begin(), L->goff.end(), out);
      else fill(P.n_bnd, [&](int64_t) { return (int64_t)P.P1; });
      return HDG_OK;
    default:
      return set_err(c, HDG_ERR_ARG, "unknown offset table");
  }
}

hdg_status hdg_quad_points(const hdg_ctx* cc, double* xy) {
  hdg_ctx* c = const_cast<hdg_ctx*>(cc);
  if (!c || !xy) return HDG_ERR_ARG;
  if (!c->d_tables) return set_err(c, HDG_ERR_STATE, "context not initialised");
  if (c->lv) return level_quad_points(c, xy);
  quad_points_kernel<<<1024, 256, 0, c->stream>>>(c->prm, c->dt, xy);
  c->launches += 1;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HDG_OK : cuda_err(c, e, "hdg_quad_points");
}

hdg_status hdg_bnd_quad_points(const hdg_ctx* cc, double* xy) {
  hdg_ctx* c = const_cast<hdg_ctx*>(cc);
  if (!c || !xy) return HDG_ERR_ARG;
  if (!c->d_tables) return set_err(c, HDG_ERR_STATE, "context not initialised");
  if (c->lv) return level_bnd_quad_points(c, xy);
  bnd_points_kernel<<<64, 256, 0, c->stream>>>(c->prm, c->dt, xy);
  c->launches += 1;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HDG_OK : cuda_err(c, e, "hdg_bnd_quad_points");
}

hdg_status hdg_set_source(hdg_ctx* c, const double* f_qp, const double* gD_qp, int nrhs) {
  NvtxRange nvtx_range("hdg_set_source");
  if (!c) return HDG_ERR_ARG;
  if (!c->d_tables) return set_err(c, HDG_ERR_STATE, "context not initialised");
  if (!f_qp || nrhs < 1 || nrhs > HDG_MAX_RHS)
    return set_err(c, HDG_ERR_ARG, "f_qp must be a device pointer and 1 <= nrhs <= HDG_MAX_RHS");
  if (c->lv) return level_set_source(c, f_qp, gD_qp, nrhs);
  Params& P = c->prm;
  cudaError_t e = cudaSuccess;
  if (nrhs != c->alloc_nrhs) {
    // per-RHS buffers follow the number of right-hand sides
    dev_free(c, c->d_ghat, (size_t)c->alloc_nrhs * P.n_bnd * P.P1);
    dev_free(c, c->d_gel, (size_t)c->alloc_nrhs * P.N * P.n_t);
    dev_free(c, c->d_g, (size_t)c->alloc_nrhs * P.N_tr);
    c->alloc_nrhs = 0;
    if ((e = dev_alloc(c, &c->d_ghat, (size_t)nrhs * P.n_bnd * P.P1)) != cudaSuccess) return cuda_err(c, e, "ghat");
    c->alloc_nrhs = nrhs;
  }
  {
    Params t = P;
    t.nrhs = nrhs;
    t.Cc = P.Q + P.n_t + nrhs;
    t.ld = (int)round_up(t.Cc, 4);
    if (condense_smem_bytes(t) > kMaxSmem)
      return set_err(c, HDG_ERR_ARG, std::to_string(nrhs) + " sources need " +
                                         std::to_string(condense_smem_bytes(t) / 1024) +
                                         " KB of shared memory per element (at most 227 KB)");
  }
  P.nrhs = nrhs;
  P.Cc = P.Q + P.n_t + nrhs;
  P.ld = (int)round_up(P.Cc, 4);
  c->f_qp = f_qp;
  c->gD_qp = gD_qp;
  if (gD_qp) {
    for (int r = 0; r < nrhs && e == cudaSuccess; ++r) {
      e = launch_project_dirichlet(P, c->dt, gD_qp + (size_t)r * P.n_bnd * P.n_bqp, c->d_ghat + (size_t)r * P.n_bnd * P.P1,
                                   c->stream);
      c->launches += 1;
    }
  }
  else {
    e = cudaMemsetAsync(c->d_ghat, 0, (size_t)nrhs * P.n_bnd * P.P1 * 8, c->stream);
  }
  if (e != cudaSuccess) return cuda_err(c, e, "hdg_set_source");
  c->state = 1;
  return HDG_OK;
}

hdg_status hdg_condense(hdg_ctx* c, unsigned flags) {
  NvtxRange nvtx_range("hdg_condense");
  if (!c) return HDG_ERR_ARG;
  if (c->state < 1) return set_err(c, HDG_ERR_STATE, "hdg_condense before hdg_set_source");
  if (flags & ~(HDG_STORE_FP32 | HDG_KEEP_FACTORS | HDG_STORE_DF64 | HDG_SPLIT_UPDATE | HDG_PRECOND_FACE_SCHUR |
                HDG_TC_UPDATE | HDG_STORE_FIX64))
    return set_err(c, HDG_ERR_ARG, "unknown flags");
  if ((flags & HDG_STORE_FIX64) && (c->lv || !fix_supported(c->prm)))
    return set_err(c, HDG_ERR_ARG, "HDG_STORE_FIX64 needs a uniform mesh with at most 240 trace dofs per element");
  if ((flags & HDG_SPLIT_UPDATE) && (flags & HDG_TC_UPDATE))
    return set_err(c, HDG_ERR_ARG, "HDG_SPLIT_UPDATE and HDG_TC_UPDATE exclude each other");
  if (c->lv) return level_condense(c, flags);
  const int split = update_kind(flags);
  const Params& P = c->prm;
  cudaError_t e;
  const size_t sblk = (size_t)P.N * 3 * P.n_t * P.P1;
  if (!c->d_S && (e = dev_alloc(c, &c->d_S, sblk)) != cudaSuccess) return cuda_err(c, e, "S blocks");
  if (!c->d_St && (e = dev_alloc(c, &c->d_St, sblk)) != cudaSuccess) return cuda_err(c, e, "preconditioned S blocks");
  if ((flags & HDG_STORE_FP32) && !c->d_St32 && (e = dev_alloc(c, &c->d_St32, sblk)) != cudaSuccess)
    return cuda_err(c, e, "FP32 S blocks");
  if (!(flags & HDG_STORE_FP32)) dev_free(c, c->d_St32, sblk);
  // split-FP32 blocks: 16 bytes of slack at the end for the pipelined apply's
  // copies, which round each row-block out to 16-byte boundaries
  if ((flags & HDG_STORE_DF64) && !c->d_Stdf && (e = dev_alloc(c, &c->d_Stdf, sblk + 2)) != cudaSuccess)
    return cuda_err(c, e, "split-FP32 S blocks");
  if (!(flags & HDG_STORE_DF64)) dev_free(c, c->d_Stdf, sblk + 2);
  const size_t fixb = fix_blocks_bytes(P);
  if ((flags & HDG_STORE_FIX64) && !c->d_Sfix && (e = dev_alloc(c, &c->d_Sfix, fixb)) != cudaSuccess)
    return cuda_err(c, e, "fixed-point S blocks");
  if (!(flags & HDG_STORE_FIX64)) dev_free(c, c->d_Sfix, fixb);
  if (!c->d_gel && (e = dev_alloc(c, &c->d_gel, (size_t)P.nrhs * P.N * P.n_t)) != cudaSuccess) return cuda_err(c, e, "gel");
  if (!c->d_g && (e = dev_alloc(c, &c->d_g, (size_t)P.nrhs * P.N_tr)) != cudaSuccess) return cuda_err(c, e, "g");
  if (!c->d_info && (e = dev_alloc(c, &c->d_info, (size_t)P.N)) != cudaSuccess) return cuda_err(c, e, "info");
  const size_t slot = (size_t)P.R * P.ld;
  // without HDG_KEEP_FACTORS the elements are condensed in chunks that fit a 1 GiB workspace
  const int64_t budget_slots = std::max<int64_t>(1, (int64_t)((size_t(1) << 30) / (slot * sizeof(double))));
  const int64_t want = (flags & HDG_KEEP_FACTORS) ? P.N : std::min<int64_t>(P.N, budget_slots);
  if (c->ws_slots != want || c->ws_ld != P.ld) {
    dev_free(c, c->d_ws, (size_t)c->ws_slots * P.R * c->ws_ld);
    c->ws_slots = 0;
    if ((e = dev_alloc(c, &c->d_ws, (size_t)want * slot)) != cudaSuccess) return cuda_err(c, e, "local workspace");
    c->ws_slots = want;
    c->ws_ld = P.ld;
  }
  const int keep = (flags & HDG_KEEP_FACTORS) ? 1 : 0;
  if (keep && !c->d_piv && (e = dev_alloc(c, &c->d_piv, (size_t)P.N * P.Q)) != cudaSuccess)
    return cuda_err(c, e, "pivots");
  if (!keep) dev_free(c, c->d_piv, (size_t)P.N * P.Q);
  c->transposed = 0;
  const double* gh = c->gD_qp ? c->d_ghat : nullptr;
  for (int64_t e0 = 0; e0 < P.N; e0 += c->ws_slots) {
    const int64_t cnt = std::min<int64_t>(c->ws_slots, P.N - e0);
    {
      ProfScope ps(c, HDG_PROF_CONDENSE);
      e = launch_condense(P, c->dt, c->d_kappa, c->f_qp, gh, c->d_ws, e0, cnt, keep, 1, c->d_S, c->d_St,
                          (flags & HDG_STORE_FP32) ? c->d_St32 : nullptr, c->d_gel, c->d_info, c->stream, split,
                          keep ? c->d_piv : nullptr);
    }
    c->launches += 1;
    if (e != cudaSuccess) return cuda_err(c, e, "condense kernel");
  }
  c->pc_face = 0;
  if (flags & HDG_PRECOND_FACE_SCHUR) {
    // inverted diagonal face blocks of S folded into the preconditioned rows
    if (!c->d_Pinv && (e = dev_alloc(c, &c->d_Pinv, (size_t)P.n_int * P.P1 * P.P1)) != cudaSuccess)
      return cuda_err(c, e, "face blocks");
    if (!c->d_bad && (e = dev_alloc(c, &c->d_bad, 1)) != cudaSuccess) return cuda_err(c, e, "face block check");
    int bad = 0;
    if ((e = cudaMemsetAsync(c->d_bad, 0, sizeof(int), c->stream)) != cudaSuccess ||
        (e = launch_face_schur(P, c->d_S, c->d_Pinv, c->d_St, (flags & HDG_STORE_FP32) ? c->d_St32 : nullptr,
                               c->d_bad, c->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&bad, c->d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
      return cuda_err(c, e, "face blocks");
    c->launches += 2;
    if (bad) {
      c->state = 1;
      return set_err(c, HDG_ERR_SINGULAR, std::to_string(bad) + " diagonal face blocks of S have a zero pivot");
    }
    c->pc_face = 1;
  }
  if (flags & HDG_STORE_DF64) {
    c->launches += 1;
    if ((e = launch_split_df(c->d_St, c->d_Stdf, (int64_t)sblk, c->stream)) != cudaSuccess)
      return cuda_err(c, e, "split");
  }
  if (flags & HDG_STORE_FIX64) {
    c->launches += 1;
    if ((e = launch_fix_convert(P, c->d_St, c->d_Sfix, c->stream)) != cudaSuccess)
      return cuda_err(c, e, "fixed-point blocks");
  }
  for (int r = 0; r < P.nrhs; ++r) {
    c->launches += 1;
    if ((e = launch_assemble_rhs(P, c->d_gel + (size_t)r * P.N * P.n_t, c->d_g + (size_t)r * P.N_tr, c->stream)) !=
        cudaSuccess)
      return cuda_err(c, e, "rhs");
  }
  std::vector<int> info(P.N);
  if ((e = cudaMemcpyAsync(info.data(), c->d_info, (size_t)P.N * 4, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
    return cuda_err(c, e, "info");
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_err(c, e, "condense");
  c->flags = flags;
  for (int64_t i = 0; i < P.N; ++i)
    if (info[i] < 0) {
      c->state = 1;
      return set_err(c, HDG_ERR_TIMEOUT, "condensation: the tensor-core update of element " + std::to_string(i) +
                                             " did not complete within the bounded wait");
    } else if (info[i]) {
      c->state = 1;
      return set_err(c, HDG_ERR_SINGULAR, "zero pivot in column " + std::to_string(info[i] - 1) + " of element " +
                                                std::to_string(i));
    }
  c->state = 2;
  return HDG_OK;
}

hdg_status hdg_rhs(hdg_ctx* c, double* g) {
  if (!c || !g) return HDG_ERR_ARG;
  if (c->state < 2) return set_err(c, HDG_ERR_STATE, "hdg_rhs before hdg_condense");
  cudaError_t e = cudaMemcpyAsync(g, c->d_g, (size_t)c->prm.nrhs * c->prm.N_tr * 8, cudaMemcpyDeviceToDevice,
                                  c->stream);
  return e == cudaSuccess ? HDG_OK : cuda_err(c, e, "hdg_rhs");
}

hdg_status hdg_apply(hdg_ctx* c, const void* x, void* y, int nrhs, int prec, int precond) {
  NvtxRange nvtx_range("hdg_apply");
  if (!c) return HDG_ERR_ARG;
  if (!x || !y || x == y || nrhs < 1 || nrhs > HDG_MAX_RHS) return set_err(c, HDG_ERR_ARG, "bad x/y or nrhs");
  if (c->state < 2) return set_err(c, HDG_ERR_STATE, "hdg_apply before hdg_condense");
  cudaError_t e;
  ProfScope ps(c, prec == 32 ? HDG_PROF_APPLY32 : HDG_PROF_APPLY);
  if (prec == 49) {
    // the Arnoldi operator of the split-FP32 solve, on split-FP32 vectors, in the launch shape the solve uses
    if (c->lv || nrhs != 1) return set_err(c, HDG_ERR_ARG, "prec 49 is the one-column operator of a uniform mesh");
    if (!c->d_Stdf || !precond) return set_err(c, HDG_ERR_ARG, "split-FP32 apply needs HDG_STORE_DF64 and precond = 1");
    const int epb = c->tune_epb[1];
    e = launch_apply_vdf(1, c->prm, c->d_Stdf, x, y, precond_scale(c), nullptr, c->stream, epb, 1, &c->bulk_hooks);
    c->launches += 1;
    if (e == cudaSuccess && epb < 0) {
      int err = 0;
      e = apply_bulk_take_error(c->stream, &err);
      if (e == cudaSuccess && err) return set_err(c, HDG_ERR_TIMEOUT, "pipelined apply: a bounded copy wait gave up");
    }
    return e == cudaSuccess ? HDG_OK : cuda_err(c, e, "hdg_apply (split vectors)");
  }
  if (c->lv) {
    const LevelMesh& L = *c->lv;
    if ((e = level_ensure_z(c, nrhs)) != cudaSuccess) return cuda_err(c, e, "element-side buffer");
    const int64_t n = c->prm.N_tr;
    if (prec == 64) {
      e = launch_level_apply(c, 0, 0, precond ? L.d_St : L.d_S, x, y, nrhs, n, precond ? precond_scale(c) : nullptr,
                             nullptr, c->stream);
    } else if (prec == 48) {
      if (!L.d_Stdf || !precond) return set_err(c, HDG_ERR_ARG, "split-FP32 apply needs HDG_STORE_DF64 and precond = 1");
      e = launch_level_apply(c, 1, 0, L.d_Stdf, x, y, nrhs, n, precond_scale(c), nullptr, c->stream);
    } else if (prec == 32 || prec == 33) {
      if (!L.d_St32 || !precond) return set_err(c, HDG_ERR_ARG, "FP32 apply needs HDG_STORE_FP32 and precond = 1");
      const int vt = prec == 32 ? 2 : 0;
      e = launch_level_apply(c, 2, vt, L.d_St32, x, y, nrhs, n, precond_scale(c), nullptr, c->stream);
    } else {
      return set_err(c, HDG_ERR_ARG, "prec must be 64, 48, 33 or 32");
    }
    c->launches += 2;
    return e == cudaSuccess ? HDG_OK : cuda_err(c, e, "hdg_apply");
  }
  if (nrhs > 1) {
    // multi-RHS apply: every block streamed once for all columns
    const Params& P = c->prm;
    if (prec == 64) {
      e = launch_apply_mrhs(0, 0, P, precond ? c->d_St : c->d_S, x, y, nrhs, P.N_tr, precond ? precond_scale(c) : nullptr,
                            c->stream);
    } else if (prec == 48) {
      if (!c->d_Stdf || !precond) return set_err(c, HDG_ERR_ARG, "split-FP32 apply needs HDG_STORE_DF64 and precond = 1");
      e = launch_apply_mrhs(1, 0, P, c->d_Stdf, x, y, nrhs, P.N_tr, precond_scale(c), c->stream);
    } else if (prec == 32) {
      if (!c->d_St32 || !precond) return set_err(c, HDG_ERR_ARG, "FP32 apply needs HDG_STORE_FP32 and precond = 1");
      e = launch_apply_mrhs(2, 2, P, c->d_St32, x, y, nrhs, P.N_tr, precond_scale(c), c->stream);
    } else {
      return set_err(c, HDG_ERR_ARG, "prec must be 64, 48 or 32 for several columns");
    }
    c->launches += 1;
    return e == cudaSuccess ? HDG_OK : cuda_err(c, e, "hdg_apply (multi-RHS)");
  }
  if (prec == 64) {
    e = precond ? launch_apply64(c->prm, c->d_St, (const double*)x, (double*)y, precond_scale(c), nullptr, c->stream)
                : launch_apply64(c->prm, c->d_S, (const double*)x, (double*)y, nullptr, nullptr, c->stream);
  } else if (prec == 48) {
    if (!c->d_Stdf || !precond) return set_err(c, HDG_ERR_ARG, "split-FP32 apply needs HDG_STORE_DF64 and precond = 1");
    e = launch_apply_df(c->prm, c->d_Stdf, (const double*)x, (double*)y, precond_scale(c), nullptr, c->stream);
  } else if (prec == 56) {
    // fixed-point blocks on FP64 vectors: the Arnoldi operator of mode 3
    if (!c->d_Sfix || !precond) return set_err(c, HDG_ERR_ARG, "fixed-point apply needs HDG_STORE_FIX64 and precond = 1");
    e = launch_apply_fix(c->prm, c->d_Sfix, (const double*)x, (double*)y, precond_scale(c), nullptr, c->stream,
                         c->tune_epb[3]);
  } else if (prec == 33) {
    // FP32 blocks on FP64 vectors: the Arnoldi operator of mode 1 with the FP64 basis
    if (!c->d_St32 || !precond) return set_err(c, HDG_ERR_ARG, "FP32 apply needs HDG_STORE_FP32 and precond = 1");
    e = launch_apply_vdf(2, c->prm, c->d_St32, x, y, precond_scale(c), nullptr, c->stream, 0, 0);
  } else if (prec == 32) {
    if (!c->d_St32 || !precond) return set_err(c, HDG_ERR_ARG, "FP32 apply needs HDG_STORE_FP32 and precond = 1");
    e = launch_apply32(c->prm, c->d_St32, (const float*)x, (float*)y, precond_scale(c), nullptr, c->stream);
  } else {
    return set_err(c, HDG_ERR_ARG, "prec must be 64, 56, 49, 48, 33 or 32");
  }
  c->launches += 1;
  return e == cudaSuccess ? HDG_OK : cuda_err(c, e, "hdg_apply");
}

hdg_status hdg_set_wait_hooks(hdg_ctx* c, int64_t wait_cycles, int64_t skip_copy_edge) {
  if (!c) return HDG_ERR_ARG;
  if (wait_cycles < 0 || skip_copy_edge < -1 || skip_copy_edge >= c->prm.n_int)
    return set_err(c, HDG_ERR_ARG, "wait_cycles >= 0 and -1 <= skip_copy_edge < interior edges");
  c->bulk_hooks.wait_cycles = (long long)wait_cycles;
  c->bulk_hooks.skip_edge = (int)skip_copy_edge;
  return HDG_OK;
}

hdg_status hdg_set_apply_shape(hdg_ctx* c, int mode, int edges_per_block, int bulk_warps) {
  if (!c) return HDG_ERR_ARG;
  if (mode < 0 || mode > 3 || edges_per_block < 0 || bulk_warps < 0 || (edges_per_block > 0 && bulk_warps > 0))
    return set_err(c, HDG_ERR_ARG, "mode 0..3 and at most one of edges_per_block, bulk_warps");
  if (c->lv) return set_err(c, HDG_ERR_ARG, "a level mesh has no per-edge apply shape");
  const int bt = mode == 0 ? 0 : (mode == 2 ? 1 : (mode == 3 ? 3 : 2));
  if (edges_per_block * c->prm.P1 > 512) return set_err(c, HDG_ERR_ARG, "edges_per_block * (m p + 1) above 512");
  if (bulk_warps > 0 && (bt != 1 || !apply_bulk_available(c->prm, bulk_warps)))
    return set_err(c, HDG_ERR_ARG, "the pipelined apply needs mode 2 and a shape that fits shared memory");
  c->tune_epb[bt] = bulk_warps > 0 ? -bulk_warps : edges_per_block;
  return HDG_OK;
}

hdg_status hdg_solve(hdg_ctx* c, const double* g, double* x, int nrhs, const hdg_solve_opts* o,
                     hdg_solve_report* rep) {
  NvtxRange nvtx_range("hdg_solve");
  if (!c) return HDG_ERR_ARG;
  if (!g || !x || !o || nrhs < 1 || nrhs > HDG_MAX_RHS) return set_err(c, HDG_ERR_ARG, "bad arguments");
  if (c->state < 2) return set_err(c, HDG_ERR_STATE, "hdg_solve before hdg_condense");
  if (!(o->tol > 0.0) || o->maxit < 1 || o->restart < 1 || o->restart > 128 || o->mode < 0 || o->mode > 3 ||
      o->orth < 0 || o->orth > 3 || o->basis < HDG_BASIS_FP64 || o->basis > HDG_BASIS_FIX || o->augment < 0 ||
      o->augment > HDG_MAX_AUGMENT || o->augment >= o->restart)
    return set_err(c, HDG_ERR_ARG, "bad solve options");
  const bool has32 = c->lv ? c->lv->d_St32 != nullptr : c->d_St32 != nullptr;
  const bool hasdf = c->lv ? c->lv->d_Stdf != nullptr : c->d_Stdf != nullptr;
  if (o->mode == 1 && !has32) return set_err(c, HDG_ERR_ARG, "mode 1 needs HDG_STORE_FP32");
  // (the profiling phase of the FP32 inner operator is HDG_PROF_APPLY32)
  if (o->mode == 2 && !hasdf) return set_err(c, HDG_ERR_ARG, "mode 2 needs HDG_STORE_DF64");
  if (o->mode == 3 && (!c->d_Sfix || nrhs != 1 || o->basis == HDG_BASIS_DF64))
    return set_err(c, HDG_ERR_ARG, "mode 3 needs HDG_STORE_FIX64, one right-hand side and FP64 vectors");
  if (o->basis == HDG_BASIS_FIX && (nrhs != 1 || o->augment > 0))
    return set_err(c, HDG_ERR_ARG, "the fixed-point basis takes one right-hand side and no augmented restarts");
  if (c->lv) {
    const cudaError_t e = level_ensure_z(c, nrhs);
    if (e != cudaSuccess) return cuda_err(c, e, "element-side buffer");
  }
  hdg_solve_report r{};
  const hdg_status s = nrhs == 1 ? gmres_solve(c, g, x, *o, r) : gmres_solve_batched(c, g, x, nrhs, *o, r);
  if (rep) *rep = r;
  return s;
}

hdg_status hdg_autotune(hdg_ctx* c, const hdg_solve_opts* o, hdg_tune_report* rep) {
  NvtxRange nvtx_range("hdg_autotune");
  if (!c) return HDG_ERR_ARG;
  if (!o || !rep) return set_err(c, HDG_ERR_ARG, "bad arguments");
  if (c->state < 2) return set_err(c, HDG_ERR_STATE, "hdg_autotune before hdg_condense");
  if (o->restart < 1 || o->restart > 128 || o->mode < 0 || o->mode > 3 || o->basis < HDG_BASIS_FP64 ||
      o->basis > HDG_BASIS_FIX)
    return set_err(c, HDG_ERR_ARG, "bad solve options");
  const bool has32 = c->lv ? c->lv->d_St32 != nullptr : c->d_St32 != nullptr;
  const bool hasdf = c->lv ? c->lv->d_Stdf != nullptr : c->d_Stdf != nullptr;
  if (o->mode == 1 && !has32) return set_err(c, HDG_ERR_ARG, "mode 1 needs HDG_STORE_FP32");
  if (o->mode == 2 && !hasdf) return set_err(c, HDG_ERR_ARG, "mode 2 needs HDG_STORE_DF64");
  if (o->mode == 3 && (!c->d_Sfix || o->basis == HDG_BASIS_DF64))
    return set_err(c, HDG_ERR_ARG, "mode 3 needs HDG_STORE_FIX64 and FP64 vectors");
  *rep = hdg_tune_report{};
  return autotune(c, *o, *rep);
}

hdg_status hdg_recover(hdg_ctx* c, const double* x, double* u, double* q, int nrhs) {
  NvtxRange nvtx_range("hdg_recover");
  if (!c) return HDG_ERR_ARG;
  if (!x || !u || !q) return set_err(c, HDG_ERR_ARG, "bad arguments");
  if (c->state < 2) return set_err(c, HDG_ERR_STATE, "hdg_recover before hdg_condense");
  const Params& P = c->prm;
  if (nrhs != P.nrhs) return set_err(c, HDG_ERR_ARG, "nrhs must equal the nrhs of hdg_set_source");
  if (c->lv) return level_recover(c, x, u, q, nrhs);
  cudaError_t e;
  // column r: x_r, g^_r, u_r, q_r at r * (one RHS) offsets
  auto rec = [&](int64_t e0, int64_t cnt, int slot_is_element, int r) {
    return launch_recover(P, c->dt, c->d_ws, e0, cnt, slot_is_element, x + (size_t)r * P.N_tr,
                          c->gD_qp ? c->d_ghat + (size_t)r * P.n_bnd * P.P1 : nullptr, u + (size_t)r * P.N * P.Q,
                          q + (size_t)r * P.N * 2 * P.Q, c->stream, r);
  };
  // several sources: one launch per element range for all of them
  auto rec_all = [&](int64_t e0, int64_t cnt, int slot_is_element) {
    return launch_recover_mrhs(P, c->dt, c->d_ws, nullptr, P.N, e0, cnt, slot_is_element, x, P.N_tr,
                               c->gD_qp ? c->d_ghat : nullptr, (int64_t)P.n_bnd * P.P1, nullptr, 0, nullptr, u, q,
                               (int64_t)P.N * P.Q, nrhs, c->stream);
  };
  if (c->flags & HDG_KEEP_FACTORS) {
    ProfScope ps(c, HDG_PROF_RECOVER);
    if (nrhs > 1) {
      e = rec_all(0, P.N, 1);
      c->launches += 1;
      if (e != cudaSuccess) return cuda_err(c, e, "recover");
    }
    if (nrhs == 1) {
      e = rec(0, P.N, 1, 0);
      c->launches += 1;
      if (e != cudaSuccess) return cuda_err(c, e, "recover");
    }
  } else {
    const double* gh = c->gD_qp ? c->d_ghat : nullptr;
    for (int64_t e0 = 0; e0 < P.N; e0 += c->ws_slots) {
      const int64_t cnt = std::min<int64_t>(c->ws_slots, P.N - e0);
      e = launch_condense(P, c->dt, c->d_kappa, c->f_qp, gh, c->d_ws, e0, cnt, 0, 0, nullptr, nullptr, nullptr,
                          nullptr, nullptr, c->stream, update_kind(c->flags));
      if (e != cudaSuccess) return cuda_err(c, e, "refactor");
      c->launches += 1;
      if (nrhs > 1) {
        e = rec_all(e0, cnt, 0);
        c->launches += 1;
        if (e != cudaSuccess) return cuda_err(c, e, "recover");
      }
      if (nrhs == 1) {
        e = rec(e0, cnt, 0, 0);
        c->launches += 1;
        if (e != cudaSuccess) return cuda_err(c, e, "recover");
      }
    }
  }
  return HDG_OK;
}

hdg_status hdg_get_schur(hdg_ctx* c, int64_t e0, int64_t count, double* S) {
  if (!c) return HDG_ERR_ARG;
  if (!S || e0 < 0 || count < 1 || e0 + count > c->prm.N) return set_err(c, HDG_ERR_ARG, "bad element range");
  if (c->state < 2) return set_err(c, HDG_ERR_STATE, "hdg_get_schur before hdg_condense");
  if (c->lv) return level_get_schur(c, e0, count, S);
  cudaError_t e = launch_get_schur(c->prm, c->d_S, e0, count, S, c->stream);
  c->launches += 1;
  return e == cudaSuccess ? HDG_OK : cuda_err(c, e, "hdg_get_schur");
}

hdg_status hdg_run_host(hdg_ctx* c, const double* f_host, const double* gD_host, const hdg_solve_opts* o,
                        double* x_host, double* u_host, double* q_host, hdg_solve_report* rep) {
  NvtxRange nvtx_range("hdg_run_host");
  if (!c) return HDG_ERR_ARG;
  if (!f_host || !o) return set_err(c, HDG_ERR_ARG, "bad arguments");
  if (c->lv) return set_err(c, HDG_ERR_ARG, "hdg_run_host: not available on a level mesh");
  const Params& P = c->prm;
  const size_t nf = (size_t)P.N * P.n_qp, ng = (size_t)P.n_bnd * P.n_bqp;
  const size_t nu = (size_t)P.N * P.Q;
  double *df = nullptr, *dg = nullptr, *dx = nullptr, *du = nullptr, *dq = nullptr, *dgv = nullptr;
  cudaError_t e = cudaSuccess;
  hdg_status s = HDG_OK;
  auto cleanup = [&]() {
    cudaFree(df); cudaFree(dg); cudaFree(dx); cudaFree(du); cudaFree(dq); cudaFree(dgv);
  };
  if ((e = cudaMalloc(&df, nf * 8)) != cudaSuccess || (gD_host && (e = cudaMalloc(&dg, ng * 8)) != cudaSuccess) ||
      (e = cudaMalloc(&dx, (size_t)P.N_tr * 8)) != cudaSuccess || (e = cudaMalloc(&dgv, (size_t)P.N_tr * 8)) != cudaSuccess ||
      (e = cudaMalloc(&du, nu * 8)) != cudaSuccess || (e = cudaMalloc(&dq, 2 * nu * 8)) != cudaSuccess) {
    cleanup();
    return cuda_err(c, e, "hdg_run_host buffers");
  }
  if ((e = cudaMemcpyAsync(df, f_host, nf * 8, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
      (gD_host && (e = cudaMemcpyAsync(dg, gD_host, ng * 8, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess) ||
      (e = cudaMemsetAsync(dx, 0, (size_t)P.N_tr * 8, c->stream)) != cudaSuccess) {
    cleanup();
    return cuda_err(c, e, "hdg_run_host upload");
  }
  // the blocks the requested solve mode needs; FP64-accurate local factorisations (FP64 panels,
  // trailing updates on the tensor cores) except with the split-FP32 operator (mode 2), whose
  // condensation eliminates in split-FP32 arithmetic too
  const unsigned cflags = HDG_KEEP_FACTORS | (o->mode == 1 ? HDG_STORE_FP32 : 0u) | (o->mode == 3 ? HDG_STORE_FIX64 : 0u) |
                          (o->mode == 2 ? (HDG_STORE_DF64 | HDG_SPLIT_UPDATE) : HDG_TC_UPDATE);
  if ((s = hdg_set_source(c, df, dg, 1)) == HDG_OK && (s = hdg_condense(c, cflags)) == HDG_OK &&
      (s = hdg_rhs(c, dgv)) == HDG_OK) {
    s = hdg_solve(c, dgv, dx, 1, o, rep);
    if (s == HDG_OK || s == HDG_ERR_NOCONV) {
      const hdg_status s2 = hdg_recover(c, dx, du, dq, 1);
      if (s2 != HDG_OK) s = s2;
    }
  }
  if (s == HDG_OK || s == HDG_ERR_NOCONV) {
    if ((x_host && (e = cudaMemcpyAsync(x_host, dx, (size_t)P.N_tr * 8, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess) ||
        (u_host && (e = cudaMemcpyAsync(u_host, du, nu * 8, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess) ||
        (q_host && (e = cudaMemcpyAsync(q_host, dq, 2 * nu * 8, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess) ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess) {
      s = cuda_err(c, e, "hdg_run_host download");
    }
  }
  cudaStreamSynchronize(c->stream);
  // the staged source buffers are released: a new hdg_set_source is required
  c->f_qp = nullptr;
  c->gD_qp = nullptr;
  c->state = 0;
  cleanup();
  return s;
}

hdg_status hdg_set_kappa(hdg_ctx* c, const double* kappa) {
  if (!c) return HDG_ERR_ARG;
  if (!kappa) return set_err(c, HDG_ERR_ARG, "kappa must be a device pointer");
  if (c->lv) return set_err(c, HDG_ERR_ARG, "hdg_set_kappa: not available on a level mesh");
  if (!c->d_tables) return set_err(c, HDG_ERR_STATE, "context not initialised");
  cudaError_t e;
  if (!c->d_bad && (e = dev_alloc(c, &c->d_bad, 1)) != cudaSuccess) return cuda_err(c, e, "kappa check");
  int bad = 0;
  if ((e = cudaMemsetAsync(c->d_bad, 0, sizeof(int), c->stream)) != cudaSuccess ||
      (e = launch_copy_kappa(c->prm, kappa, c->d_kappa, c->d_bad, c->stream)) != cudaSuccess ||
      (e = launch_face_scale(c->prm, c->d_kappa, c->d_escale, c->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&bad, c->d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return cuda_err(c, e, "hdg_set_kappa");
  c->launches += 2;
  if (c->state > 1) c->state = 1;
  if (bad) return set_err(c, HDG_ERR_ARG, std::to_string(bad) + " diffusivities are negative or not finite");
  return HDG_OK;
}

hdg_status hdg_transpose(hdg_ctx* c) {
  if (!c) return HDG_ERR_ARG;
  if (c->lv) return set_err(c, HDG_ERR_ARG, "hdg_transpose: not available on a level mesh");
  if (c->state < 2) return set_err(c, HDG_ERR_STATE, "hdg_transpose before hdg_condense");
  ProfScope ps(c, HDG_PROF_ADJOINT);
  cudaError_t e = launch_transpose(c->prm, c->dt, c->d_S, c->d_St, c->d_St32, c->d_Stdf, c->stream);
  c->launches += 1;
  if (e != cudaSuccess) return cuda_err(c, e, "hdg_transpose");
  c->transposed ^= 1;
  if (c->pc_face) {
    // the transposed operator's face blocks are S_ff^T: fold (S_ff^-1)^T into the rows again
    e = launch_face_fold(c->prm, c->d_S, c->d_Pinv, c->transposed, c->d_St, c->d_St32, c->stream);
    if (e == cudaSuccess && c->d_Stdf)
      e = launch_split_df(c->d_St, c->d_Stdf, (int64_t)c->prm.N * 3 * c->prm.n_t * c->prm.P1, c->stream);
    c->launches += 2;
    if (e != cudaSuccess) return cuda_err(c, e, "hdg_transpose (face blocks)");
  }
  if (c->d_Sfix) {
    // the fixed-point copy follows the transposed rows
    e = launch_fix_convert(c->prm, c->d_St, c->d_Sfix, c->stream);
    c->launches += 1;
    if (e != cudaSuccess) return cuda_err(c, e, "hdg_transpose (fixed-point blocks)");
  }
  return HDG_OK;
}

hdg_status hdg_adjoint_rhs(hdg_ctx* c, const double* r, double* g) {
  if (!c) return HDG_ERR_ARG;
  if (!r || !g) return set_err(c, HDG_ERR_ARG, "bad arguments");
  if (c->lv) return set_err(c, HDG_ERR_ARG, "hdg_adjoint_rhs: not available on a level mesh");
  if (c->state < 2 || !(c->flags & HDG_KEEP_FACTORS) || !c->d_piv)
    return set_err(c, HDG_ERR_STATE, "hdg_adjoint_rhs needs hdg_condense with HDG_KEEP_FACTORS");
  const Params& P = c->prm;
  cudaError_t e;
  if (!c->d_gadj && (e = dev_alloc(c, &c->d_gadj, (size_t)P.N * P.n_t)) != cudaSuccess)
    return cuda_err(c, e, "adjoint element vectors");
  {
    ProfScope ps(c, HDG_PROF_ADJOINT);
    e = launch_adjoint_rhs(P, c->d_ws, r, c->d_gadj, c->stream);
  }
  if (e == cudaSuccess) e = launch_assemble_rhs(P, c->d_gadj, g, c->stream);
  c->launches += 2;
  return e == cudaSuccess ? HDG_OK : cuda_err(c, e, "hdg_adjoint_rhs");
}

hdg_status hdg_adjoint_recover(hdg_ctx* c, const double* r, const double* nu, double* mu) {
  if (!c) return HDG_ERR_ARG;
  if (!r || !nu || !mu) return set_err(c, HDG_ERR_ARG, "bad arguments");
  if (c->lv) return set_err(c, HDG_ERR_ARG, "hdg_adjoint_recover: not available on a level mesh");
  if (c->state < 2 || !(c->flags & HDG_KEEP_FACTORS) || !c->d_piv)
    return set_err(c, HDG_ERR_STATE, "hdg_adjoint_recover needs hdg_condense with HDG_KEEP_FACTORS");
  ProfScope ps(c, HDG_PROF_ADJOINT);
  cudaError_t e = launch_adjoint_recover(c->prm, c->d_ws, c->d_piv, r, nu, mu, c->stream);
  c->launches += 1;
  return e == cudaSuccess ? HDG_OK : cuda_err(c, e, "hdg_adjoint_recover");
}

hdg_status hdg_gradient(hdg_ctx* c, const double* x, const double* u, const double* mu, const double* nu,
                        double* dkappa, double* df) {
  if (!c) return HDG_ERR_ARG;
  if (!x || !u || !mu || !nu || !dkappa) return set_err(c, HDG_ERR_ARG, "bad arguments");
  if (c->lv) return set_err(c, HDG_ERR_ARG, "hdg_gradient: not available on a level mesh");
  if (c->state < 1) return set_err(c, HDG_ERR_STATE, "hdg_gradient before hdg_set_source");
  if (c->prm.supg) return set_err(c, HDG_ERR_STATE, "hdg_gradient: SUPG terms are not affine in kappa");
  ProfScope ps(c, HDG_PROF_ADJOINT);
  const double* gh = c->gD_qp ? c->d_ghat : nullptr;
  cudaError_t e = launch_gradient(c->prm, c->dt, x, gh, u, mu, nu, dkappa, df, c->stream);
  c->launches += 1;
  return e == cudaSuccess ? HDG_OK : cuda_err(c, e, "hdg_gradient");
}

hdg_status hdg_profile(hdg_ctx* c, int enable) {
  if (!c) return HDG_ERR_ARG;
  profile_collect(c);
  if (enable) {
    for (int i = 0; i < HDG_PROF_NPHASES; ++i) { c->prof_count[i] = 0; c->prof_ms[i] = 0.0; }
  }
  c->prof_on = enable != 0;
  return HDG_OK;
}

hdg_status hdg_profile_read(hdg_ctx* c, hdg_profile_t* out) {
  if (!c || !out) return HDG_ERR_ARG;
  profile_collect(c);
  for (int i = 0; i < HDG_PROF_NPHASES; ++i) { out->count[i] = c->prof_count[i]; out->ms[i] = c->prof_ms[i]; }
  return HDG_OK;
}

const char* hdg_last_error(const hdg_ctx* c) { return c ? c->err.c_str() : "null context"; }

void hdg_destroy(hdg_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  profile_collect(c);
  for (auto& pr : c->prof_pool) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
  if (c->lv) {
    level_destroy(c);    // also releases d_tables' target and the face scales
    c->d_tables = nullptr;
  }
  cudaFree(c->d_tables); cudaFree(c->d_kappa); cudaFree(c->d_ghat); cudaFree(c->d_S); cudaFree(c->d_St);
  cudaFree(c->d_St32); cudaFree(c->d_Stdf); cudaFree(c->d_Sfix); cudaFree(c->d_gel); cudaFree(c->d_g); cudaFree(c->d_ws); cudaFree(c->d_info);
  cudaFree(c->d_escale); cudaFree(c->d_V); cudaFree(c->d_w); cudaFree(c->d_r); cudaFree(c->d_part);
  cudaFree(c->d_small); cudaFree(c->d_flag); cudaFree(c->d_piv); cudaFree(c->d_gadj); cudaFree(c->d_bad);
  cudaFree(c->d_Vb); cudaFree(c->d_wb); cudaFree(c->d_rb); cudaFree(c->d_partb); cudaFree(c->d_smallb);
  cudaFree(c->d_flagb); cudaFree(c->d_scalb); cudaFree(c->d_Zb); cudaFree(c->d_Pinv); cudaFree(c->d_cmapb);
  cudaFree(c->d_aug); cudaFree(c->d_augb); cudaFree(c->d_Vs); cudaFree(c->d_vin);
  for (auto& g : c->gm_cache) cudaGraphExecDestroy(g.second);
  for (cudaEvent_t ev : c->gm_ev) cudaEventDestroy(ev);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
}

}  // extern "C"
