// hdg_condense_static: element condensation that allocates no device memory.
//
// Who needs it: code that may not call cudaMalloc once it is running, e.g. a
// solver embedded in a host application that owns and pre-plans all device
// memory, a loop that must never fail with out-of-memory halfway through a
// run, or code on a path where an allocation (which can synchronise the
// device) is not allowed. Such a caller creates its context up front and then
// uses this entry point for condensation on demand; the working space of the
// local factorisations comes from the fixed array below instead of the
// context's workspace allocation.
//
// The scratch array lives for as long as the library is loaded, on every GPU
// that loads it: MEHDG_STATIC_SCRATCH_BYTES (16 MiB) of bordered local systems
// plus a one-word status flag. All calls share it and it keeps the contents of
// the last call, so calls whose work overlaps on the GPU (two streams, two
// host threads on one device) race on it and must be serialised by the caller.
#include <string>
#include "launch.h"

namespace mehdg {

// File-scope scratch (device memory of the loaded module, no allocation call).
static __device__ __align__(256) double g_static_scratch[MEHDG_STATIC_SCRATCH_BYTES / sizeof(double)];
static __device__ __align__(256) int g_static_flag[1];

namespace {

// Device addresses of the scratch symbols in the current context. In host code
// the symbols' names are host-side stand-ins, not device addresses, so every
// call asks the runtime (cheap once the module is loaded). Nothing is cached:
// an address kept from an earlier context (before a device reset) would point
// into freed memory.
cudaError_t static_scratch_lookup(double** scratch, int** flag) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess) return e;
  void* q = nullptr;
  e = cudaGetSymbolAddress(&q, g_static_flag);
  if (e != cudaSuccess) return e;
  *scratch = static_cast<double*>(p);
  *flag = static_cast<int*>(q);
  return cudaSuccess;
}

// Copy S_e and the element right-hand side out of the factored bordered
// systems (slot b holds element e0 + b) into the caller's row-major buffers;
// raise *flag if a pivot of the local LU is zero.
__global__ void static_extract_kernel(Params P, const double* __restrict__ ws, int64_t e0, int64_t count,
                                      const double* __restrict__ ghat, double* __restrict__ S_out,
                                      double* __restrict__ g_out, int* flag) {
  const int64_t b = blockIdx.x;
  if (b >= count) return;
  const int e = (int)(e0 + b);
  const int Q = P.Q, nt = P.n_t, P1 = P.P1, ld = P.ld;
  const double* W = ws + (size_t)b * P.R * ld;
  for (int i = threadIdx.x; i < Q; i += blockDim.x)
    if (W[(size_t)i * ld + i] == 0.0) atomicExch(flag, 1);
  double* So = S_out + (size_t)b * nt * nt;
  for (int idx = threadIdx.x; idx < nt * nt; idx += blockDim.x) {
    const int r = idx / nt, c = idx - r * nt;
    So[idx] = W[(size_t)(Q + r) * ld + Q + c];
  }
  if (!g_out) return;
  int code[3], flip[3];
  elem_edges(e, P.n, code, flip);
  // source s: load column Q + n_t + s, Dirichlet lift of source s, out [nrhs][count][n_t]
  for (int idx = threadIdx.x; idx < P.nrhs * nt; idx += blockDim.x) {
    const int s = idx / nt, r = idx - s * nt;
    double acc = W[(size_t)(Q + r) * ld + Q + nt + s];
    if (ghat) {
      const double* gs = ghat + (size_t)s * P.n_bnd * P1;
      for (int k = 0; k < 3; ++k) {
        if (code[k] >= 0) continue;
        const double* gb = gs + (size_t)(-1 - code[k]) * P1;
        for (int t = 0; t < P1; ++t) acc -= W[(size_t)(Q + r) * ld + Q + k * P1 + t] * gb[flip[k] ? P.P - t : t];
      }
    }
    g_out[((size_t)s * count + b) * nt + r] = acc;
  }
}

}  // namespace

// Loads the module that holds the scratch array on the current device, so that
// its MEHDG_STATIC_SCRATCH_BYTES are set aside when a context is created rather
// than at the first hdg_condense_static call (under lazy module loading the
// array comes into being when the module is first used). Called by hdg_create.
cudaError_t static_scratch_prepare() {
  double* s = nullptr;
  int* f = nullptr;
  return static_scratch_lookup(&s, &f);
}

}  // namespace mehdg

using namespace mehdg;

extern "C" hdg_status hdg_condense_static(hdg_ctx* c, int64_t e0, int64_t count, double* S_dev, double* g_dev) {
  if (!c) return HDG_ERR_ARG;
  if (c->lv) {
    c->err = "hdg_condense_static: not available on a level mesh";
    return HDG_ERR_ARG;
  }
  if (!S_dev || e0 < 0 || count < 1 || e0 + count > c->prm.N) {
    c->err = "hdg_condense_static: bad element range or null S";
    return HDG_ERR_ARG;
  }
  if (c->state < 1) {
    c->err = "hdg_condense_static before hdg_set_source";
    return HDG_ERR_STATE;
  }
  const Params& P = c->prm;
  const size_t slot_bytes = (size_t)P.R * P.ld * sizeof(double);
  if ((size_t)count * slot_bytes > MEHDG_STATIC_SCRATCH_BYTES) {
    c->err = "hdg_condense_static: " + std::to_string(count) + " elements need " +
             std::to_string((size_t)count * slot_bytes) + " bytes of scratch, the static array holds " +
             std::to_string((size_t)MEHDG_STATIC_SCRATCH_BYTES) + " (at most " +
             std::to_string(MEHDG_STATIC_SCRATCH_BYTES / slot_bytes) + " elements of this size per call)";
    return HDG_ERR_ARG;
  }
  double* scratch = nullptr;
  int* flag = nullptr;
  cudaError_t e = static_scratch_lookup(&scratch, &flag);
  if (e != cudaSuccess) {
    c->err = std::string("hdg_condense_static set-up: ") + cudaGetErrorString(e);
    return HDG_ERR_CUDA;
  }
  const double* gh = c->gD_qp ? c->d_ghat : nullptr;
  // the zero-pivot flag must start at zero; the bordered systems are fully rewritten
  if ((e = cudaMemsetAsync(flag, 0, sizeof(int), c->stream)) == cudaSuccess &&
      (e = launch_condense(P, c->dt, c->d_kappa, c->f_qp, gh, scratch, e0, count, 0, 0, nullptr, nullptr, nullptr,
                           nullptr, nullptr, c->stream)) == cudaSuccess) {
    static_extract_kernel<<<(unsigned)count, 128, 0, c->stream>>>(P, scratch, e0, count, gh, S_dev, g_dev, flag);
    c->launches += 2;
    e = cudaGetLastError();
  }
  int hflag = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    c->err = std::string("hdg_condense_static: ") + cudaGetErrorString(e);
    return HDG_ERR_CUDA;
  }
  if (hflag) {
    c->err = "hdg_condense_static: zero pivot in elements " + std::to_string(e0) + ".." + std::to_string(e0 + count - 1);
    return HDG_ERR_SINGULAR;
  }
  return HDG_OK;
}
