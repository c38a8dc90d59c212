// Kernel launchers shared between the translation units of the library.
#pragma once
#include "internal.h"

namespace mehdg {

size_t condense_smem_bytes(const Params& P);
cudaError_t launch_condense(const Params& P, const DevTables& dt, const double* kappa, const double* f_qp,
                            const double* ghat, double* ws, int64_t e0, int64_t count, int slot_is_element,
                            int write_outputs, double* S, double* St, float* St32, double* gel, int* info,
                            cudaStream_t st, int split_update = 0, int* piv = nullptr);
cudaError_t launch_recover(const Params& P, const DevTables& dt, const double* ws, int64_t e0, int64_t count,
                           int slot_is_element, const double* x, const double* ghat, double* u, double* q,
                           cudaStream_t st, int rcol = 0);
cudaError_t launch_project_dirichlet(const Params& P, const DevTables& dt, const double* gD, double* ghat,
                                     cudaStream_t st);
// one refinement level of a level mesh (condense.cu)
cudaError_t launch_condense_bin(const Params& P, const DevTables& dt, const double* kappa, const double* f_qp,
                                const int64_t* qoff, int64_t fstride, const double* ghat, double* ws,
                                const int* elist, int64_t nslots, int64_t e0, int64_t count, int slot_is_element,
                                int write_outputs, double* S, double* gel, int* info, cudaStream_t st,
                                int split_update);
cudaError_t launch_recover_bin(const Params& P, const DevTables& dt, const double* ws, const int* elist,
                               int64_t nslots, int64_t e0, int64_t count, int slot_is_element, const double* xel,
                               const int64_t* uoff, double* u, double* q, cudaStream_t st, int rcol);
cudaError_t launch_recover_mrhs(const Params& P, const DevTables& dt, const double* ws, const int* elist,
                                int64_t nslots, int64_t e0, int64_t count, int slot_is_element, const double* x,
                                int64_t xstride, const double* ghat, int64_t ghstride, const double* xel,
                                int64_t xelstride, const int64_t* uoff, double* u, double* q, int64_t ustride,
                                int nrhs, cudaStream_t st);
cudaError_t launch_project_dirichlet_bin(const Params& P, const DevTables& dt, const int* blist, int nbnd,
                                         const int64_t* boff, const double* gD, double* ghat, cudaStream_t st);
cudaError_t launch_get_schur(const Params& P, const double* S, int64_t e0, int64_t count, double* out,
                             cudaStream_t st);

cudaError_t launch_apply64(const Params& P, const double* S, const double* x, double* y, const double* escale,
                           const int* stop, cudaStream_t st, int epb = 0);
cudaError_t launch_apply32(const Params& P, const float* S, const float* x, float* y, const double* escale,
                           const int* stop, cudaStream_t st);
cudaError_t launch_apply_df(const Params& P, const float2* S, const double* x, double* y, const double* escale,
                            const int* stop, cudaStream_t st);
// bt: 0 FP64 / 1 split-FP32 / 2 FP32 blocks; vt: 0 FP64 / 1 split-FP32 vectors; hk: the pipelined
// apply's wait limit and test hook (null: defaults)
// Fixed-point Krylov basis: limbs [vectors][ldv] int2, chunk scales [vectors][fx_chunks(n)] int32.
int64_t fx_chunks(int64_t n);
int launch_fx_mdot(const void* V, const int* Vs, int64_t ldv, int64_t n, int nv, int ncol, const double* w,
                   double* part, const int* stop, cudaStream_t st);
void launch_fx_combine(const void* V, const int* Vs, int64_t ldv, int64_t n, int nv, const double* coef, double csign,
                       const double* base, double bcoef, const double* sm, int scale_off, double* out_d, void* out_l,
                       int* out_s, const int* stop, cudaStream_t st);
// Fixed-point apply (FP64 products exact in integer arithmetic): block conversion and apply.
// fix points to limbs [N][3][n_t][P1] int2 followed by row scales [N][3][P1] int32.
size_t fix_blocks_bytes(const Params& P);
bool fix_supported(const Params& P);
cudaError_t launch_fix_convert(const Params& P, const double* S, void* fix, cudaStream_t st);
cudaError_t launch_apply_fix(const Params& P, const void* fix, const double* x, double* y, const double* escale,
                             const int* stop, cudaStream_t st, int epb);
cudaError_t launch_apply_vdf(int bt, const Params& P, const void* S, const void* x, void* y,
                             const double* escale, const int* stop, cudaStream_t st, int epb = 0, int vt = 1,
                             const BulkHooks* hk = nullptr);
int apply_edges_per_block(const Params& P);
// Pipelined bulk-copy apply of split-FP32 blocks (q = 1 .. 3 consumer warps
// per edge); whether it applies to this problem shape; its timeout flag (read
// and cleared, synchronous).
bool apply_bulk_available(const Params& P, int q);
int apply_bulk_threads(const Params& P, int q);   // threads per CTA of that shape (0: not available)
cudaError_t launch_apply_bulk(const Params& P, const float2* S, const float2* x, float2* y, const double* escale,
                              const int* stop, cudaStream_t st, int q, long long wait_cycles = 0,
                              int skip_edge = -1);
cudaError_t apply_bulk_take_error(cudaStream_t st, int* err);
cudaError_t launch_apply_mrhs(int bt, int vt, const Params& P, const void* S, const void* x, void* y, int nrhs,
                              int64_t vstride, const double* escale, cudaStream_t st);
// cmap (optional): compute only the nrhs columns cmap[0 .. nrhs-1] of x and y
// vt: 0 FP64 / 1 split-FP32 vectors (Z of the same entry type)
cudaError_t launch_apply_mrhs_el(int bt, const Params& P, const void* S, const void* x, void* y, int nrhs,
                                 int64_t vstride, const double* escale, void* Z, cudaStream_t st,
                                 const int* cmap = nullptr, int vt = 1);
cudaError_t launch_split_df(const double* a, float2* out, int64_t n, cudaStream_t st);
cudaError_t launch_assemble_rhs(const Params& P, const double* gel, double* g, cudaStream_t st);
cudaError_t launch_face_dinv(const Params& P, const double* Ghinv, const double* escale, const double* y, double* z,
                             cudaStream_t st);
cudaError_t launch_face_scale(const Params& P, const double* kappa, double* escale, cudaStream_t st);

// Reference tables to the device (api.cu): one allocation, its size in *bytes.
cudaError_t upload_ref_tables(const RefTables& T, DevTables& d, void** dmem, size_t* bytes, cudaStream_t st);

// Level meshes (levels.cu): per-element refinement levels, faces at the finer side's level.
hdg_status level_create(hdg_ctx* c, const hdg_mesh_desc* d);
void level_destroy(hdg_ctx* c);
hdg_status level_quad_points(hdg_ctx* c, double* xy);
hdg_status level_bnd_quad_points(hdg_ctx* c, double* xy);
hdg_status level_set_source(hdg_ctx* c, const double* f_qp, const double* gD_qp, int nrhs);
hdg_status level_condense(hdg_ctx* c, unsigned flags);
hdg_status level_recover(hdg_ctx* c, const double* x, double* u, double* q, int nrhs);
hdg_status level_get_schur(hdg_ctx* c, int64_t e0, int64_t count, double* S);
// element-side product buffer for nrhs columns (allocated outside any stream capture)
cudaError_t level_ensure_z(hdg_ctx* c, int nrhs);
// y = S x (escale null) or D^-1 S x (preconditioned blocks, escale) for nrhs columns of stride vstride;
// bt: 0 FP64 / 1 split-FP32 / 2 FP32 blocks, vt: 0 FP64 / 1 split-FP32 / 2 FP32 vectors
cudaError_t launch_level_apply(hdg_ctx* c, int bt, int vt, const void* S, const void* x, void* y, int nrhs,
                               int64_t vstride, const double* escale, const int* stop, cudaStream_t st,
                               const int* cmap = nullptr);
cudaError_t launch_level_dinv(hdg_ctx* c, const double* y, double* z, int nrhs, int64_t vstride, cudaStream_t st);

// Face-block preconditioner with the diagonal blocks of S (precond.cu).
cudaError_t launch_face_schur(const Params& P, const double* S, double* Pinv, double* St, float* St32, int* bad,
                              cudaStream_t st);
// refold the preconditioned rows from S (trans: S holds S_e^T, the inverse blocks are transposed)
cudaError_t launch_face_fold(const Params& P, const double* S, const double* Pinv, int trans, double* St, float* St32,
                             cudaStream_t st);
cudaError_t launch_face_pinv(const Params& P, const double* Pinv, int trans, const double* y, double* z,
                             cudaStream_t st);
cudaError_t launch_level_face_schur(const LevelDev& L, int max_nf, const double* S, double* Pinv, double* St,
                                    int* bad, cudaStream_t st);
cudaError_t launch_level_face_pinv(const LevelDev& L, const double* Pinv, const double* y, double* z, int nrhs,
                                   int64_t vstride, cudaStream_t st);

// Adjoint path (adjoint.cu).
cudaError_t launch_copy_kappa(const Params& P, const double* src, double* kappa, int* bad, cudaStream_t st);
cudaError_t launch_transpose(const Params& P, const DevTables& dt, double* S, double* St, float* St32, float2* Stdf,
                             cudaStream_t st);
cudaError_t launch_adjoint_rhs(const Params& P, const double* ws, const double* r, double* gel, cudaStream_t st);
cudaError_t launch_adjoint_recover(const Params& P, const double* ws, const int* piv, const double* r,
                                   const double* nu, double* mu, cudaStream_t st);
cudaError_t launch_gradient(const Params& P, const DevTables& dt, const double* x, const double* ghat,
                            const double* u, const double* mu, const double* nu, double* dkappa, double* df,
                            cudaStream_t st);

// Loads the no-allocation entry point's scratch array on the current device (static_scratch.cu).
cudaError_t static_scratch_prepare();
// Restarted GMRES on the condensed system (krylov.cu).
hdg_status gmres_solve(hdg_ctx* c, const double* g, double* x, const hdg_solve_opts& o, hdg_solve_report& rep);
// nrhs independent instances in lockstep: one multi-RHS apply and batched
// vector kernels per Arnoldi step (krylov.cu).
hdg_status gmres_solve_batched(hdg_ctx* c, const double* g, double* x, int nrhs, const hdg_solve_opts& o,
                               hdg_solve_report& rep);
// Launch-shape autotuner of the GMRES kernels (krylov.cu).
hdg_status autotune(hdg_ctx* c, const hdg_solve_opts& o, hdg_tune_report& rep);

}  // namespace mehdg
