/*
 * mehdg.h - C ABI of the GB300 (sm_103a) macro-element HDG trace solver.
 *
 * Implements the data-parallel hot path of the macro-element hybridized DG
 * method of Badrkhani, Hiemstra, Mika and Schillinger, "A matrix-free
 * macro-element variant of the hybridized discontinuous Galerkin method"
 * (arXiv 2302.10917), for the 2D steady advection-diffusion problem
 *     -kappa Lap u + beta . grad u = f  on (0,1)^2,   u = g_D on the boundary
 * (Eq. C21 with a constant velocity a = beta, first-order form Eq. C22).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * Mesh (Sec. 5.1, d = 2): n x n squares, each split by its "/" diagonal into
 *   t = 0 (lower-right): v0 = (x_{i+1}, y_j), v1 = (x_{i+1}, y_{j+1}), v2 = (x_i, y_j)
 *   t = 1 (upper-left) : v0 = (x_i, y_{j+1}), v1 = (x_i, y_j),         v2 = (x_{i+1}, y_{j+1})
 *   element id e = 2 (j n + i) + t, N = 2 n^2. Local edge k is opposite v_k
 *   and runs from v_{k+1} to v_{k+2}.
 * Macro-element spaces (Sec. 3.2): C0 piecewise P_p on the uniform m-fold
 *   subdivision of each macro-triangle; P = m p; Q = (P+1)(P+2)/2 lattice
 *   nodes (a/P, b/P), a + b <= P, in reference coordinates of the affine map
 *   x = v0 + xi (v1 - v0) + eta (v2 - v0), numbered b-major, a fastest:
 *   node(a, b) = b (P+1) - b (b-1)/2 + a.
 * Trace (Sec. 3.2): C0 piecewise P_p on each macro-edge, P + 1 dofs per edge
 *   at equispaced points, oriented from the lower to the higher global vertex
 *   id (vertex (i, j) has id j (n+1) + i). Trace unknowns live on the
 *   n^2 + 2 n (n-1) interior edges (all four sides are Dirichlet):
 *     diagonal   D(i,j)        -> j n + i
 *     horizontal H(i,j), 1<=j<n -> n^2 + (j-1) n + i
 *     vertical   V(i,j), 1<=i<n -> n^2 + n (n-1) + j (n-1) + (i-1)
 *   global trace dof = edge (P + 1) + s; N_tr = (#interior edges)(P + 1).
 *   Boundary edges: bottom H(i,0) -> i, top H(i,n) -> n + i,
 *   left V(0,j) -> 2n + j, right V(n,j) -> 3n + j.
 * Source quadrature (element formation, Sec. 6.1): on every sub-triangle
 *   (upright ones (si,sj), si+sj<=m-1, with corners (si,sj),(si+1,sj),(si,sj+1)
 *   in units of 1/m, then inverted ones (si,sj), si+sj<=m-2, with corners
 *   (si+1,sj+1),(si,sj+1),(si+1,sj); sj outer, si inner) the collapsed
 *   Gauss rule with ng = p + 2 points per direction: local point
 *   (u_i (1 - u_j), u_j), index j ng + i, u_* the Gauss-Legendre nodes on
 *   [0,1]. n_qp = m^2 ng^2 points per element.
 * Dirichlet data: on each boundary edge, m sub-edges x (p + 2) Gauss points
 *   along its orientation; g_D is L2-projected onto the trace space (Sec. 2.3).
 * Stabilisation (Sec. 3.1, value not given in the paper):
 *   tau_e = kappa_e / tau_len + |beta| on all edges of element e.
 *
 * Memory, streams and errors
 * --------------------------
 * Pointers named *_dev are CUDA device pointers owned by the caller; *_host
 * pointers are host memory owned by the caller. The context owns every
 * internal buffer (Schur blocks, factors, Krylov basis). All device work is
 * enqueued on the stream given to hdg_create; entry points that return data
 * to the host (hdg_info, hdg_solve's report, hdg_run_host) synchronise that
 * stream. A failing call returns a status other than HDG_OK and records a
 * message that hdg_last_error returns; the context stays usable unless the
 * status is HDG_ERR_CUDA. Call order: hdg_create -> hdg_set_source ->
 * hdg_condense -> {hdg_rhs, hdg_apply, hdg_solve} -> hdg_recover; a call out
 * of order returns HDG_ERR_STATE.
 * Several right-hand sides (1 <= nrhs <= HDG_MAX_RHS, fixed by
 * hdg_set_source) share one condensation: every per-RHS array is RHS-major,
 * i.e. nrhs consecutive copies of the single-RHS layout ([nrhs][...]).
 * Nothing here falls back to the CPU: without a usable sm_103a device every
 * entry point that launches work returns HDG_ERR_CUDA.
 *
 * Level meshes (Sec. 4.2, local adaptive refinement; hdg_mesh_desc.level)
 * ------------------------------------------------------------------------
 * Element e carries its own level r_e (0 <= r_e <= 4, m_e = 2^r_e and the
 * level-m_e lattice inside); interior edge f carries the level R_f =
 * max(r+, r-) of its finer side and 2^R_f p + 1 trace dofs (C0 P_p on 2^R_f
 * sub-edges, along its orientation); a boundary edge has its element's
 * level. Every per-element or per-edge array is ragged, concatenated in
 * element (edge) order with the prefix sums hdg_offsets returns:
 *   trace vectors:   edge f's dofs at HDG_OFF_TRACE[f];  N_tr = last entry;
 *   source points:   element e's m_e^2 (p + 2)^2 points (the uniform-level
 *                    order of that level) at HDG_OFF_SOURCE[e];
 *   Dirichlet data:  boundary edge b's 2^r_b (p + 2) points at HDG_OFF_DIRICHLET_POINTS[b];
 *   u:               element e's Q_e lattice values at HDG_OFF_LATTICE[e];
 *   q:               element e's [2][Q_e] at 2 HDG_OFF_LATTICE[e];
 *   Schur blocks:    element e's n_t,e x n_t,e block (row-major, local trace
 *                    dofs face by face in the element's own edge orientation)
 *                    at HDG_OFF_SCHUR[e].
 * Several right-hand sides stack those arrays (RHS-major). On a level mesh
 * hdg_run_host, hdg_condense_static, hdg_set_kappa and the adjoint entry
 * points return HDG_ERR_ARG; hdg_autotune tunes the element-side rows per
 * CTA of the apply (128, 256 or 512) and the Krylov kernels.
 */
#ifndef MEHDG_H
#define MEHDG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hdg_ctx hdg_ctx;

typedef enum {
  HDG_OK = 0,
  HDG_ERR_ARG = 1,       /* invalid argument (null pointer, bad size, unsupported option) */
  HDG_ERR_STATE = 2,     /* call made out of the documented order */
  HDG_ERR_CUDA = 3,      /* CUDA runtime error (message holds the CUDA error string) */
  HDG_ERR_OOM = 4,       /* device allocation failed */
  HDG_ERR_SINGULAR = 5,  /* a local matrix had a zero pivot (element index in the message) */
  HDG_ERR_NOCONV = 6,    /* GMRES stopped at maxit; x holds the last iterate */
  HDG_ERR_TIMEOUT = 7    /* a bounded device wait gave up */
} hdg_status;

typedef struct {
  int n;                 /* macro squares per side (N = 2 n^2 macro-triangles), n >= 1 */
  int m;                 /* sub-edges per macro-edge (m^2 sub-triangles), 1 <= m <= 16; one element's
                            condensation panel must fit 227 KB of shared memory, which excludes
                            m >= 13 at p = 3 and m >= 10 at p = 4 (HDG_ERR_ARG with the size) */
  int p;                 /* polynomial degree, 1 <= p <= 4 */
  double beta[2];        /* constant advection velocity a */
  double kappa0;         /* diffusivity used when kappa == NULL; >= 0 (0 = pure advection) */
  const double* kappa;   /* host pointer, N per-element diffusivities >= 0, or NULL */
  double tau_len;        /* length scale of tau_e = kappa_e / tau_len + |beta|; > 0 */
  int bc[4];             /* boundary type per side (bottom, top, left, right); 0 = Dirichlet (only value accepted) */
  int supg;              /* 1: SUPG stabilisation inside every macro-element (Sec. 3.4), 0: none.
                            Adds tau_s (a . grad w, a . grad u - kappa Lap u - f) over the sub-triangles,
                            tau_s = h / (2 |a|) (coth Pe - 1 / Pe), Pe = |a| h / (2 kappa), h the
                            sub-triangle diameter (the printed formula's "+ 1/Pe" read as "- 1/Pe").
                            hdg_gradient refuses SUPG (its terms are not affine in kappa). */
  const int8_t* level;   /* host pointer, N refinement levels r_e in 0 .. 4 (m_e = 2^r_e), or NULL for the
                            uniform level m; with levels, m is ignored and every level present must fit the
                            same shared-memory bound as m (see the level-mesh conventions above) */
} hdg_mesh_desc;

typedef struct {
  int64_t N;             /* macro-elements */
  int64_t Q;             /* lattice nodes per element */
  int64_t n_t;           /* trace dofs per element, 3 (P + 1) */
  int64_t N_tr;          /* global trace unknowns */
  int64_t n_int_edges;   /* interior edges */
  int64_t n_bnd_edges;   /* boundary edges, 4 n */
  int64_t n_qp;          /* source points per element */
  int64_t n_bqp;         /* Dirichlet-data points per boundary edge */
  size_t device_bytes;   /* device memory currently held by the context */
  int64_t launches;      /* CUDA kernels this context has enqueued since hdg_create */
  int64_t levels;        /* 1 on a level mesh (Q, n_t: the largest element's; n_qp = n_bqp = 0), else 0 */
  int64_t n_qp_total;    /* source points per right-hand side */
  int64_t n_bqp_total;   /* Dirichlet-data points per right-hand side */
  int64_t n_u_total;     /* lattice values of u per right-hand side */
  int64_t n_s_total;     /* Schur-block entries */
  int64_t bounds_error;  /* library built with -DHDG_BOUNDS_CHECK: site code of the first device index check
                            that failed since hdg_create (the access it guarded was skipped), 0 if none;
                            always 0 in the regular build */
} hdg_info_t;

/* Solve options. Every restart cycle starts from the true FP64 residual
 * g - S x (the stopping test). mode selects the preconditioned Arnoldi
 * operator: 0 = FP64 blocks, FP64 arithmetic; 1 = FP32 blocks (requires
 * HDG_STORE_FP32), i.e. FP32 inside FP64 iterative refinement; 2 = split-FP32
 * blocks on the FP32 pipe (requires HDG_STORE_DF64); 3 = fixed-point blocks
 * (requires HDG_STORE_FIX64, one right-hand side, a uniform mesh and
 * HDG_BASIS_FP64): the FP64 products carried out exactly in integer
 * arithmetic, one FP64 rounding per element side. basis selects the
 * storage and arithmetic of the Krylov basis and its orthogonalisation:
 * HDG_BASIS_FP64 (0, the default) = FP64 vectors, FP64 dot products and
 * updates; HDG_BASIS_DF64 (1) = split-FP32 ("double-float", two FP32 words,
 * 48-bit significand, FP32 exponent range) on the FP32 pipe; HDG_BASIS_FIX
 * (2; one right-hand side, no augmented restarts) = FP64-accurate fixed-point
 * vectors: each chunk of 2048 entries of a basis vector held as 56-bit
 * integers at the scale of its largest entry (8 bytes per entry plus one int32
 * per chunk), the products of the multi-dot and the updates summed exactly in
 * 64-bit integers and rounded once per chunk and vector (multi-dot) or per
 * entry (updates), the operator applied to an FP64 copy of the newest vector;
 * no FP64 FMA per entry and vector. The pipelined
 * apply shape (hdg_set_apply_shape bulk_warps) runs with HDG_BASIS_DF64 only;
 * with FP64 vectors mode 2 uses the one-thread-per-row apply. */
#define HDG_BASIS_FP64 0
#define HDG_BASIS_DF64 1
#define HDG_BASIS_FIX 2
#define HDG_MAX_AUGMENT 3
typedef struct {
  double tol;            /* true relative residual ||g - S x|| / ||g|| to reach, > 0 */
  int maxit;             /* maximum number of operator applications inside GMRES */
  int restart;           /* GMRES restart length, 1 <= restart <= 128 */
  int mode;
  int orth;              /* Arnoldi orthogonalisation: 0 = classical Gram-Schmidt applied twice
                            (CGS2, four passes over the basis); 1 = classical Gram-Schmidt once,
                            the new vector's norm from ||w||^2 - ||V^T w||^2 (two passes; loses
                            orthogonality faster, which the restart from the true residual bounds);
                            2 = as 1, with a second projection in the steps where ||w - V V^T w||^2 <
                            ||w||^2 / 2 (Kahan-Parlett "twice is enough"; decided on the device, two
                            passes in the other steps); 3 = as 2 with the second projection only where
                            ||w - V V^T w||^2 < 1e-6 ||w||^2 (more than six digits cancelled) */
  int basis;             /* HDG_BASIS_FP64, HDG_BASIS_DF64 or HDG_BASIS_FIX (see above) */
  int augment;           /* 0 .. HDG_MAX_AUGMENT, below restart: augmented restarts (LGMRES, Baker, Jessup
                            and Manteuffel 2005): the last `augment` steps of every restart cycle take the
                            normalised corrections x_new - x_old of the previous cycles as their operator
                            inputs instead of new Krylov vectors (flexible Arnoldi, the images orthogonalised
                            into the same basis), which counters the stagnation of restarted GMRES; 0 = plain
                            GMRES(restart) */
} hdg_solve_opts;

typedef struct {
  int iterations;        /* Arnoldi steps (preconditioned operator applications) */
  int restarts;          /* GMRES cycles */
  int outer;             /* FP64 true-residual evaluations (one per restart cycle, plus the last) */
  int converged;         /* 1 if rel_residual <= tol */
  double rel_residual;   /* true relative residual at exit, computed with FP64 S */
} hdg_solve_report;

/* hdg_condense flags */
#define HDG_STORE_FP32 1u      /* also keep an FP32 copy of the preconditioned blocks */
#define HDG_KEEP_FACTORS 2u    /* keep the factored local systems and their pivots for hdg_recover and the
                                  adjoint (else hdg_recover refactors) */
#define HDG_STORE_DF64 4u      /* also keep the preconditioned blocks as FP32 hi/lo pairs (8 bytes per entry) */
#define HDG_SPLIT_UPDATE 8u    /* eliminate in split-FP32 arithmetic on the FP32 pipe (formation, pivot search,
                                  panel, triangular solves and trailing updates); the stored entries are FP64 */
#define HDG_TC_UPDATE 32u     /* FP64-accurate elimination with the trailing updates on the tensor cores: 32-column
                                  panels (pivot search, panel LU, U12 = L11^-1 A12) in FP64, and A22 -= L21 U12
                                  as exact products of 8-bit slices of the power-of-two-scaled rows of L21 and
                                  columns of U12 (seven slices each, 28 bf16 tcgen05 products per panel and tile,
                                  FP32 level sums exact below 2^24) combined in FP64; the dropped parts are below
                                  2^-50 of the row and column scales, under the FP64 rounding of the same dot
                                  product. Excludes HDG_SPLIT_UPDATE. HDG_ERR_TIMEOUT if a tensor-core wait
                                  gives up. No counterpart in the paper (its local solver is LAPACK LU). */
#define HDG_STORE_FIX64 64u   /* also keep the preconditioned blocks as fixed-point numbers (uniform mesh, n_t <= 240):
                                  every row (element, edge, trace position) scaled by the power of two of its largest
                                  entry's exponent and rounded to 56 bits (|v| <= 2^55, error <= 2^-55 of the row's
                                  largest magnitude), stored as a signed high and a 28-bit low 32-bit limb (8 bytes
                                  per entry, the FP64 layout) plus one int32 scale per row. The apply (prec = 56,
                                  mode 3) scales each gathered element trace vector the same way and sums the limb
                                  products exactly in 64-bit integers (no FP64 FMAs), rounding once to FP64 per
                                  element side. Kept through hdg_transpose. No counterpart in the paper. */
#define HDG_PRECOND_FACE_SCHUR 16u  /* precondition with the inverted diagonal face blocks of the condensed
                                       operator, S_ff = sum over both sides of S_e's face rows and columns,
                                       instead of D_f of Sec. 6.1 (folded into the stored preconditioned rows
                                       the same way; the apply costs the same). hdg_transpose keeps it (the
                                       transposed operator's face blocks are S_ff^T); HDG_ERR_SINGULAR if a
                                       face block has a zero pivot. */

/* Build the structured macro mesh, the reference-lattice tables of level m
 * (mass, derivative, boundary and trace matrices, quadrature) and the device
 * copies of those tables. Sec. 5.1 (mesh), Sec. 3.2 (spaces), Sec. 6.1
 * (element formation). stream: a cudaStream_t (NULL = legacy default
 * stream). *out receives a new context; free it with hdg_destroy.
 * Errors: HDG_ERR_ARG for an invalid descriptor, HDG_ERR_CUDA/OOM. */
hdg_status hdg_create(const hdg_mesh_desc* desc, void* stream, hdg_ctx** out);

/* Sizes of the problem and the context's device memory (host struct).
 * Synchronises the context's stream (it reads the bounds-check word). */
hdg_status hdg_info(const hdg_ctx* ctx, hdg_info_t* out);

/* Prefix sums of a ragged layout (host array, count + 1 entries): which =
 * HDG_OFF_SOURCE (per element: source points, N + 1), HDG_OFF_DIRICHLET_POINTS
 * (per boundary edge: Dirichlet-data points, 4 n + 1), HDG_OFF_LATTICE (per
 * element: lattice nodes, N + 1), HDG_OFF_TRACE (per interior edge: trace
 * dofs, n_int_edges + 1), HDG_OFF_SCHUR (per element: Schur-block entries,
 * N + 1), HDG_OFF_DIRICHLET_TRACE (per boundary edge: projected Dirichlet
 * trace values, 4 n + 1). Uniform meshes give the regular sums.
 * Errors: HDG_ERR_ARG for an unknown table. */
#define HDG_OFF_SOURCE 0
#define HDG_OFF_DIRICHLET_POINTS 1
#define HDG_OFF_LATTICE 2
#define HDG_OFF_TRACE 3
#define HDG_OFF_SCHUR 4
#define HDG_OFF_DIRICHLET_TRACE 5
hdg_status hdg_offsets(const hdg_ctx* ctx, int which, int64_t* out_host);

/* Physical coordinates of the source quadrature points, [N][n_qp][2] FP64
 * device array (layout in the header comment; ragged on a level mesh). The
 * caller evaluates f there. */
hdg_status hdg_quad_points(const hdg_ctx* ctx, double* xy_dev);

/* Physical coordinates of the Dirichlet-data points, [4 n][n_bqp][2] FP64. */
hdg_status hdg_bnd_quad_points(const hdg_ctx* ctx, double* xy_dev);

/* Record nrhs sources f at the quadrature points ([nrhs][N][n_qp] FP64,
 * device) and Dirichlet data g_D at the boundary points ([nrhs][4 n][n_bqp]
 * FP64, device, or NULL for g_D = 0). The arrays are read by hdg_condense and
 * hdg_recover and must stay valid until then. Eq. (weak_form): l(V), with
 * u^ = v^ + g^ (Sec. 3.1) and g^ the L2 projection of g_D (Sec. 2.3).
 * nrhs > 1 adds nrhs load columns to every element's bordered system. */
#define HDG_MAX_RHS 64
hdg_status hdg_set_source(hdg_ctx* ctx, const double* f_qp_dev, const double* gD_qp_dev, int nrhs);

/* Static condensation of every macro-element, Eqs. (global_problem) and
 * (local_problem) with the block system Eq. (D) and the forms of Eq.
 * (weak_form): forms A_e, B_e, C_e, D_e and the load of each element,
 * eliminates q and u with partial-pivoting LU in FP64, and stores the Schur
 * block S_e = D_e - C_e A_e^-1 B_e, its face-preconditioned form
 * (Sec. 6.1, D_f^-1 applied row-block-wise) and the element right-hand
 * side -C_e A_e^-1 R_e - S_e g^_e. flags: HDG_STORE_FP32, HDG_KEEP_FACTORS.
 * Errors: HDG_ERR_SINGULAR if a pivot is exactly zero (first such element
 * in the message), HDG_ERR_OOM, HDG_ERR_STATE before hdg_set_source. */
hdg_status hdg_condense(hdg_ctx* ctx, unsigned flags);

/* Assembled condensed right-hand sides g = R_u^ - C A^-1 R_u (Eq.
 * global_problem) including the Dirichlet lift; [nrhs][N_tr] FP64 device. */
hdg_status hdg_rhs(hdg_ctx* ctx, double* g_dev);

/* Matrix-free trace-operator apply (Sec. 3.3.2, steps 1-4):
 *   precond = 0: y = S x, S = sum_e L_e^T (D_e - C_e A_e^-1 B_e) L_e;
 *   precond = 1: y = D^-1 S x, the left-preconditioned operator of Sec. 6.1.
 * x, y: [nrhs][N_tr] device arrays (1 <= nrhs <= HDG_MAX_RHS, independent of
 * hdg_set_source's nrhs), FP64 (prec = 64), FP64 with the split-FP32 blocks
 * (prec = 48, precond = 1, HDG_STORE_DF64) or FP32 (prec = 32, the FP32
 * blocks, precond = 1). nrhs > 1 streams every block once for all columns
 * (multi-RHS apply). x and y must not overlap.
 * prec = 49 (uniform mesh, nrhs = 1, precond = 1, HDG_STORE_DF64): the
 * Arnoldi operator of the split-FP32 solve (mode 2) itself, on split-FP32
 * vectors (x and y [N_tr][2] FP32: entry i is x[i][0] + x[i][1]), with the
 * launch shape that solve uses (hdg_autotune's choice or hdg_set_apply_shape's);
 * with the pipelined shape it synchronises the stream to read that kernel's
 * timeout flag (HDG_ERR_TIMEOUT if a bounded wait gave up).
 * prec = 56 (uniform mesh, nrhs = 1, precond = 1, HDG_STORE_FIX64): the
 * fixed-point blocks on FP64 vectors, the Arnoldi operator of mode 3: each
 * side's dot product exact in integers from the 56-bit fixed-point row and
 * trace vector, rounded once to FP64; the two sides added and the face scale
 * applied in FP64.
 * prec = 33 (nrhs = 1, or a level mesh; precond = 1, HDG_STORE_FP32): the
 * FP32 blocks on FP64 vectors (x, y FP64; products and sums in FP32), the
 * Arnoldi operator of mode 1 with HDG_BASIS_FP64.
 * With FP64 vectors, prec = 64 and prec = 48 are the Arnoldi operators of
 * modes 0 and 2 with HDG_BASIS_FP64 (same kernels, same bits). */
hdg_status hdg_apply(hdg_ctx* ctx, const void* x_dev, void* y_dev, int nrhs, int prec, int precond);

/* Launch-shape override (no counterpart in the paper; project-written).
 * Sets the launch shape of the trace-operator apply inside hdg_solve for one
 * mode (0 FP64, 1 FP32 + refinement, 2 split-FP32, 3 fixed-point), as hdg_autotune would:
 * edges_per_block > 0 (with edges_per_block (m p + 1) <= 512) for the
 * one-thread-per-row apply, or bulk_warps = 1 .. 3 (mode 2 only) for the
 * pipelined apply with that many consumer warps per edge; both 0 restores
 * the default. The shape stays in the context until set again or replaced by
 * hdg_autotune; it applies from the next hdg_solve (and hdg_apply prec = 49).
 * Any state after hdg_create; no launch or copy (a pipelined shape queries
 * the device limits once). Uniform meshes only;
 * HDG_ERR_ARG for a shape that does not apply (the context is unchanged). */
hdg_status hdg_set_apply_shape(hdg_ctx* ctx, int mode, int edges_per_block, int bulk_warps);

/* Bounded device waits (no counterpart in the paper; project-written). The
 * pipelined apply (hdg_set_apply_shape bulk_warps) waits on shared-memory
 * barriers for its bulk copies; every such wait gives up after wait_cycles
 * SM clock cycles (0 restores the built-in limit of 2e9 cycles, about one
 * second), records the failure, lets the copies it issued land (bounded again)
 * and returns, and the entry point that launched it reports HDG_ERR_TIMEOUT;
 * the context stays usable. skip_copy_edge >= 0 is a test hook for exactly
 * that path: the row-block copies of that interior edge are not issued, so
 * the waits for them run out; -1 (the state after hdg_create) issues every
 * copy. Applies from the next launch; no device work. HDG_ERR_ARG for
 * wait_cycles < 0 or skip_copy_edge outside -1 .. interior edges - 1. */
hdg_status hdg_set_wait_hooks(hdg_ctx* ctx, int64_t wait_cycles, int64_t skip_copy_edge);

/* Solve S x = g (Eq. global_problem) with restarted GMRES, left-
 * preconditioned by D^-1 (Sec. 6.1). x_dev holds the initial guess on entry
 * and the solution on exit ([N_tr] FP64). report may be NULL.
 * Returns HDG_ERR_NOCONV (with x = last iterate and the report filled) if
 * maxit is reached first. */
hdg_status hdg_solve(hdg_ctx* ctx, const double* g_dev, double* x_dev, int nrhs,
                     const hdg_solve_opts* opts, hdg_solve_report* report);

/* Local back-solve Eq. (local_matrix_problem): A_e U_e = R_e - B_e u^_e for
 * every element, u^_e gathered from x (interior edges) and g^ (boundary).
 * u_dev: [N][Q] FP64, q_dev: [N][2][Q] FP64 (q = -grad u), lattice order. */
hdg_status hdg_recover(hdg_ctx* ctx, const double* x_dev, double* u_dev, double* q_dev, int nrhs);

/* Copy the FP64 Schur blocks S_e of elements e0 .. e0+count-1 into S_dev as
 * row-major [count][n_t][n_t] (element-local trace order: local edge k,
 * then position along the edge from v_{k+1} to v_{k+2}). On a level mesh the
 * blocks are ragged: element e's at HDG_OFF_SCHUR[e] - HDG_OFF_SCHUR[e0]. */
hdg_status hdg_get_schur(hdg_ctx* ctx, int64_t e0, int64_t count, double* S_dev);

/* End-to-end pipeline on HOST buffers: copies f (and g_D, may be NULL) to
 * the device, condenses (factors kept; modes 0, 1 and 3 with HDG_TC_UPDATE, mode 1
 * also keeping the FP32 blocks, mode 3 the fixed-point blocks; mode 2 the
 * split-FP32 blocks after split-FP32 elimination), assembles g, solves
 * from x = 0, recovers u and q and copies x, u, q back (each output may be
 * NULL to skip its copy). Synchronous. Same layouts as above. */
hdg_status hdg_run_host(hdg_ctx* ctx, const double* f_qp_host, const double* gD_qp_host,
                        const hdg_solve_opts* opts, double* x_host, double* u_host,
                        double* q_host, hdg_solve_report* report);

/* Condensation without any device allocation. This entry point has no
 * counterpart in the paper: it exists for callers that must not allocate
 * device memory after start-up (an application that owns and pre-plans all
 * device memory, a run that must not hit out-of-memory midway, code on a path
 * where an allocation and its implicit synchronisation are not allowed).
 * It condenses elements e0 .. e0+count-1 exactly like hdg_condense, but the
 * local factorisations use a fixed scratch array compiled into the library
 * (MEHDG_STATIC_SCRATCH_BYTES, held on every GPU that loads the library until
 * the process exits; hdg_create loads it on its device, so it is set aside
 * when a context is created, not at the first call) and the results go to
 * caller buffers: S_dev receives S_e row-major [count][n_t][n_t] (same layout
 * as hdg_get_schur) and g_dev, if not NULL, the element right-hand sides
 * -C_e A_e^-1 R_e - S_e g^_e of every source of hdg_set_source,
 * [nrhs][count][n_t]. Requires hdg_set_source; needs no hdg_condense and does
 * not change the context's stored blocks. count is limited to
 * MEHDG_STATIC_SCRATCH_BYTES / ((Q + n_t) * ld * 8) elements (ld = Q + n_t +
 * nrhs rounded up to a multiple of 4); a larger count returns HDG_ERR_ARG
 * with the limit in the message. Each call looks up the array's device
 * address in the current context (no allocation); do not call it inside a
 * stream capture. Every call shares the array and leaves its contents behind;
 * calls that overlap on the GPU race on it. Synchronous (it reads a
 * zero-pivot flag back): HDG_ERR_SINGULAR if a local pivot is zero. */
#define MEHDG_STATIC_SCRATCH_BYTES (16u * 1024u * 1024u)
hdg_status hdg_condense_static(hdg_ctx* ctx, int64_t e0, int64_t count, double* S_dev, double* g_dev);

/* ------------------------------------------------------------------------
 * Discrete adjoint and gradient. The paper has no counterpart: these entry
 * points differentiate a functional J(u) of the recovered element values u
 * with respect to the per-element diffusivities kappa_e and the source values
 * f at the quadrature points, through the reduced element system that
 * hdg_condense eliminates (q eliminated exactly):
 *     A_u u_e + B_u x_e = F_e,   sum_e (C_u u_e + D_u x_e) = 0 on interior
 * trace dofs (x_e includes g^ on Dirichlet edges). With r = dJ/du the adjoint
 * state solves S^T nu = g_adj = -sum_e L_e^T B_u^T A_u^-T r_e and
 * mu_e = A_u^-T (r_e - C_u^T nu_e); then
 *     dJ/dkappa_e = -[mu_e; nu_e]^T (dK_e/dkappa_e) [u_e; x_e],
 *     dJ/df_{e,i} = mu_e^T dF_e/df_{e,i}.
 * Sequence: forward solve and hdg_recover; hdg_adjoint_rhs; hdg_transpose;
 * hdg_solve(g_adj) -> nu; hdg_transpose (back); hdg_adjoint_recover -> mu;
 * hdg_gradient. hdg_adjoint_rhs and hdg_adjoint_recover need the factors
 * kept by hdg_condense (HDG_KEEP_FACTORS); otherwise HDG_ERR_STATE.
 * ------------------------------------------------------------------------ */

/* Replace the per-element diffusivities by kappa_dev ([N] FP64, device,
 * each >= 0 and finite; read before the call returns) and recompute the
 * face preconditioner's scales. The condensed blocks become stale: the
 * context returns to the "source set" state (hdg_condense required before
 * hdg_apply/hdg_solve/hdg_recover). Synchronous (it reads a validity count
 * back): HDG_ERR_ARG if an entry is negative or not finite (the stored
 * diffusivities are then undefined until a valid call). */
hdg_status hdg_set_kappa(hdg_ctx* ctx, const double* kappa_dev);

/* Transpose the stored trace operator in place, element by element
 * (S_e <- S_e^T and its preconditioned, FP32 and split-FP32 copies), so that
 * hdg_apply and hdg_solve act on S^T; D^-1 is symmetric and unchanged.
 * Calling it again restores S. hdg_condense resets the state to S. */
hdg_status hdg_transpose(hdg_ctx* ctx);

/* Adjoint right-hand side: g_dev ([N_tr] FP64) = -sum_e L_e^T B_u^T A_u^-T r_e
 * with r_dev = dJ/du as [N][Q] FP64 (the layout of hdg_recover's u). */
hdg_status hdg_adjoint_rhs(hdg_ctx* ctx, const double* r_dev, double* g_dev);

/* Adjoint element values: mu_dev ([N][Q] FP64) = A_u^-T (r_e - C_u^T nu_e)
 * for every element, nu_dev the solution of S^T nu = g_adj ([N_tr]). */
hdg_status hdg_adjoint_recover(hdg_ctx* ctx, const double* r_dev, const double* nu_dev, double* mu_dev);

/* Gradient of J: dkappa_dev[e] = dJ/dkappa_e ([N]) and, if df_dev is not
 * NULL, df_dev = dJ/df at the source points ([N][n_qp], layout of
 * hdg_set_source). x_dev: forward trace solution, u_dev: forward element
 * values (hdg_recover), mu_dev/nu_dev: adjoint state. Uses the current
 * diffusivities and Dirichlet data. Requires hdg_set_source. */
hdg_status hdg_gradient(hdg_ctx* ctx, const double* x_dev, const double* u_dev, const double* mu_dev,
                        const double* nu_dev, double* dkappa_dev, double* df_dev);

/* Launch-shape autotuner (no counterpart in the paper; project-written).
 * Times, with CUDA events on the context stream, the candidate launch shapes
 * of the GMRES kernels for opts->mode at this problem size: edges per block
 * of the trace-operator apply (one thread per edge and trace position, up to
 * 512 threads) and, for split-FP32 blocks on a uniform mesh, the pipelined
 * apply with 1 to 3 consumer warps per edge (bulk asynchronous copies of the
 * row-blocks into shared memory, consumed row by row; with one warp per edge
 * in the same summation order, with more in a fixed order of their own),
 * blocks of the multi-dot and of the streaming update (at
 * opts->restart / 2 basis vectors). Keeps the fastest of each in the context
 * for every later hdg_solve / hdg_apply and reports them. Arithmetic and
 * results are unchanged by the apply's edges per block; the multi-dot's partial sums
 * follow its block count (fixed per context, so solves stay reproducible).
 * Needs hdg_condense (with the blocks the mode uses). Synchronous. */
typedef struct {
  int apply_edges_per_block; /* chosen edges per block of the apply (0 on a level mesh) */
  int apply_threads;         /* threads per block that implies (level mesh: element-side rows per CTA) */
  int mdot_blocks;           /* multi-dot blocks over all vector groups */
  int update_blocks;         /* streaming-update blocks */
  double apply_ms;           /* best times of the three kernels */
  double mdot_ms;
  double update_ms;
  double default_ms;         /* the three kernels with the built-in shapes */
  int apply_bulk;            /* > 0: the pipelined apply was chosen, with this many consumer warps per edge
                                (split-FP32 blocks on a uniform mesh: the element-side row-blocks are brought
                                into shared memory by bulk asynchronous copies ahead of the products;
                                apply_edges_per_block is then 0 and apply_threads the CTA's threads) */
  double apply_bulk_ms;      /* best time of the pipelined apply (0 where it was not a candidate) */
} hdg_tune_report;
hdg_status hdg_autotune(hdg_ctx* ctx, const hdg_solve_opts* opts, hdg_tune_report* report);

/* Per-phase device timing (tracing). Phases: */
#define HDG_PROF_CONDENSE 0   /* condensation kernel launches (element build + LU + Schur) */
#define HDG_PROF_APPLY 1      /* preconditioned FP64 / split-FP32 apply launches (hdg_apply, GMRES's Arnoldi steps) */
#define HDG_PROF_ORTHO 2      /* GMRES vector work of one Arnoldi step (CGS2, norm, Givens, scaling) */
#define HDG_PROF_RECOVER 3    /* back-solve kernel launches */
#define HDG_PROF_APPLY32 4    /* FP32 trace-operator apply launches */
#define HDG_PROF_RESID 5      /* FP64 unpreconditioned applies for GMRES's true residual */
#define HDG_PROF_ADJOINT 6    /* adjoint kernels: transposition, adjoint right-hand side and back-solve, gradient */
#define HDG_PROF_NPHASES 7
typedef struct {
  int64_t count[HDG_PROF_NPHASES];   /* timed launches (or Arnoldi steps for ORTHO) */
  double ms[HDG_PROF_NPHASES];       /* summed CUDA-event time on the context stream */
} hdg_profile_t;

/* Start (enable != 0) or stop per-phase timing; starting clears the totals.
 * While enabled, every timed launch is bracketed by a CUDA event pair on the
 * context stream. */
hdg_status hdg_profile(hdg_ctx* ctx, int enable);

/* Synchronise the stream and return the totals since the last start. */
hdg_status hdg_profile_read(hdg_ctx* ctx, hdg_profile_t* out);

/* Last error message of the context (never NULL; "" if none). */
const char* hdg_last_error(const hdg_ctx* ctx);

/* Release every resource of the context (NULL is allowed). */
void hdg_destroy(hdg_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* MEHDG_H */
