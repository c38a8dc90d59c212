"""GB300 (sm_103a) macro-element HDG trace solver: thin Python binding.

Argument marshalling only: every step of the hot path (element formation,
batched static condensation, trace-operator apply, GMRES, back-solve) runs in
the CUDA library ``libmehdg.so`` behind the C ABI of ``include/mehdg.h``.
PyTorch supplies device memory and the CUDA stream. There is no CPU fallback:
if the library or a GPU is missing, every call raises.
"""
import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmehdg.so")

HDG_OK, HDG_ERR_ARG, HDG_ERR_STATE, HDG_ERR_CUDA, HDG_ERR_OOM = 0, 1, 2, 3, 4
HDG_ERR_SINGULAR, HDG_ERR_NOCONV, HDG_ERR_TIMEOUT = 5, 6, 7
HDG_STORE_FP32, HDG_KEEP_FACTORS, HDG_STORE_DF64, HDG_SPLIT_UPDATE, HDG_PRECOND_FACE_SCHUR = 1, 2, 4, 8, 16
HDG_TC_UPDATE = 32
HDG_STORE_FIX64 = 64
BASIS_FP64, BASIS_DF64, BASIS_FIX = 0, 1, 2   # hdg_solve_opts.basis: FP64, split-FP32 or fixed-point Krylov basis
STATUS_NAMES = {0: "HDG_OK", 1: "HDG_ERR_ARG", 2: "HDG_ERR_STATE", 3: "HDG_ERR_CUDA", 4: "HDG_ERR_OOM",
                5: "HDG_ERR_SINGULAR", 6: "HDG_ERR_NOCONV", 7: "HDG_ERR_TIMEOUT"}

EXPORTED = ["hdg_create", "hdg_info", "hdg_quad_points", "hdg_bnd_quad_points", "hdg_set_source",
            "hdg_condense", "hdg_rhs", "hdg_apply", "hdg_solve", "hdg_recover", "hdg_get_schur",
            "hdg_run_host", "hdg_profile", "hdg_profile_read", "hdg_condense_static", "hdg_set_kappa",
            "hdg_transpose", "hdg_adjoint_rhs", "hdg_adjoint_recover", "hdg_gradient", "hdg_autotune",
            "hdg_set_apply_shape", "hdg_set_wait_hooks",
            "hdg_offsets", "hdg_last_error",
            "hdg_destroy"]
STATIC_SCRATCH_BYTES = 16 * 1024 * 1024
PROF_PHASES = ["condense", "apply", "ortho", "recover", "apply32", "resid", "adjoint"]


class MeshDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("m", ctypes.c_int), ("p", ctypes.c_int),
                ("beta", ctypes.c_double * 2), ("kappa0", ctypes.c_double),
                ("kappa", ctypes.POINTER(ctypes.c_double)), ("tau_len", ctypes.c_double),
                ("bc", ctypes.c_int * 4), ("supg", ctypes.c_int), ("level", ctypes.c_void_p)]


class Info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("Q", ctypes.c_int64), ("n_t", ctypes.c_int64),
                ("N_tr", ctypes.c_int64), ("n_int_edges", ctypes.c_int64),
                ("n_bnd_edges", ctypes.c_int64), ("n_qp", ctypes.c_int64), ("n_bqp", ctypes.c_int64),
                ("device_bytes", ctypes.c_size_t), ("launches", ctypes.c_int64), ("levels", ctypes.c_int64),
                ("n_qp_total", ctypes.c_int64), ("n_bqp_total", ctypes.c_int64), ("n_u_total", ctypes.c_int64),
                ("n_s_total", ctypes.c_int64), ("bounds_error", ctypes.c_int64)]


# ragged-layout tables of hdg_offsets
OFF_SOURCE, OFF_DIRICHLET_POINTS, OFF_LATTICE, OFF_TRACE, OFF_SCHUR, OFF_DIRICHLET_TRACE = range(6)


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int), ("restart", ctypes.c_int),
                ("mode", ctypes.c_int), ("orth", ctypes.c_int), ("basis", ctypes.c_int), ("augment", ctypes.c_int)]


class SolveReport(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int), ("outer", ctypes.c_int),
                ("converged", ctypes.c_int), ("rel_residual", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TuneReport(ctypes.Structure):
    _fields_ = [("apply_edges_per_block", ctypes.c_int), ("apply_threads", ctypes.c_int),
                ("mdot_blocks", ctypes.c_int), ("update_blocks", ctypes.c_int), ("apply_ms", ctypes.c_double),
                ("mdot_ms", ctypes.c_double), ("update_ms", ctypes.c_double), ("default_ms", ctypes.c_double),
                ("apply_bulk", ctypes.c_int), ("apply_bulk_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Profile(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int64 * 7), ("ms", ctypes.c_double * 7)]


class HDGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path=LIB_PATH):
    """Load libmehdg.so and declare the C signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run __graft_entry__.build() (nvcc, sm_103a) first")
    lib = ctypes.CDLL(path)
    vp, dp, i64 = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64
    lib.hdg_create.argtypes = [ctypes.POINTER(MeshDesc), vp, ctypes.POINTER(vp)]
    lib.hdg_info.argtypes = [vp, ctypes.POINTER(Info)]
    lib.hdg_offsets.argtypes = [vp, ctypes.c_int, dp]
    lib.hdg_quad_points.argtypes = [vp, dp]
    lib.hdg_bnd_quad_points.argtypes = [vp, dp]
    lib.hdg_set_source.argtypes = [vp, dp, dp, ctypes.c_int]
    lib.hdg_condense.argtypes = [vp, ctypes.c_uint]
    lib.hdg_rhs.argtypes = [vp, dp]
    lib.hdg_apply.argtypes = [vp, dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.hdg_solve.argtypes = [vp, dp, dp, ctypes.c_int, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveReport)]
    lib.hdg_recover.argtypes = [vp, dp, dp, dp, ctypes.c_int]
    lib.hdg_get_schur.argtypes = [vp, i64, i64, dp]
    lib.hdg_run_host.argtypes = [vp, dp, dp, ctypes.POINTER(SolveOpts), dp, dp, dp, ctypes.POINTER(SolveReport)]
    lib.hdg_condense_static.argtypes = [vp, i64, i64, dp, dp]
    lib.hdg_set_kappa.argtypes = [vp, dp]
    lib.hdg_transpose.argtypes = [vp]
    lib.hdg_adjoint_rhs.argtypes = [vp, dp, dp]
    lib.hdg_adjoint_recover.argtypes = [vp, dp, dp, dp]
    lib.hdg_gradient.argtypes = [vp, dp, dp, dp, dp, dp, dp]
    lib.hdg_autotune.argtypes = [vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(TuneReport)]
    lib.hdg_set_apply_shape.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.hdg_set_wait_hooks.argtypes = [vp, i64, i64]
    lib.hdg_profile.argtypes = [vp, ctypes.c_int]
    lib.hdg_profile_read.argtypes = [vp, ctypes.POINTER(Profile)]
    lib.hdg_last_error.argtypes = [vp]
    lib.hdg_last_error.restype = ctypes.c_char_p
    lib.hdg_destroy.argtypes = [vp]
    lib.hdg_destroy.restype = None
    for name in EXPORTED:
        if name not in ("hdg_last_error", "hdg_destroy"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


class Problem:
    """One macro-element HDG problem on the structured unit-square mesh (one GPU).

    levels: None (every element of level m), or N per-element refinement levels r_e in 0..4
    (m_e = 2^r_e; faces at the finer side's level, Sec. 4.2). On such a level mesh every
    per-element array is ragged (flat, element-ordered; offsets())."""

    def __init__(self, n, m, p, beta=(0.0, 0.0), kappa=1.0, tau_len=1.0, device="cuda:0", stream=None,
                 supg=False, levels=None):
        self.lib = load_library()
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        d = MeshDesc()
        d.n, d.m, d.p = n, m, p
        d.beta[0], d.beta[1] = float(beta[0]), float(beta[1])
        d.tau_len = float(tau_len)
        self._kappa_host = None
        if isinstance(kappa, (int, float)):
            d.kappa0 = float(kappa)
            d.kappa = ctypes.POINTER(ctypes.c_double)()
        else:
            k = torch.as_tensor(kappa, dtype=torch.float64).contiguous().cpu()
            self._kappa_host = k
            d.kappa0 = 1.0
            d.kappa = ctypes.cast(ctypes.c_void_p(k.data_ptr()), ctypes.POINTER(ctypes.c_double))
        for s in range(4):
            d.bc[s] = 0
        d.supg = 1 if supg else 0
        self._level_host = None
        if levels is not None:
            lv = torch.as_tensor(levels).to(torch.int8).contiguous().cpu()
            if lv.numel() != 2 * n * n:
                raise ValueError("levels: one entry per macro-element (2 n^2)")
            self._level_host = lv
            d.level = ctypes.c_void_p(lv.data_ptr())
        else:
            d.level = ctypes.c_void_p(0)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = self.lib.hdg_create(ctypes.byref(d), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        self.h = h
        if st != HDG_OK:
            msg = self.lib.hdg_last_error(h).decode() if h.value else ""
            if h.value:
                self.lib.hdg_destroy(h)
            self.h = ctypes.c_void_p()
            raise HDGError(st, msg or "hdg_create failed")
        info = Info()
        self._check(self.lib.hdg_info(self.h, ctypes.byref(info)))
        self.info = {k: getattr(info, k) for k, _ in Info._fields_}
        self.n, self.m, self.p = n, m, p
        self.levels = self.info["levels"] == 1
        self._src = None
        self.nrhs = 1
        self.version = 0        # bumped by every condensation (the factors the adjoint reuses)

    def launches(self):
        """Kernels this context has enqueued so far (counted by the library)."""
        info = Info()
        self._check(self.lib.hdg_info(self.h, ctypes.byref(info)))
        return info.launches

    def bounds_error(self):
        """Site code of the first failed device index check since hdg_create (a library built
        with -DHDG_BOUNDS_CHECK), 0 if none; always 0 with the regular build."""
        info = Info()
        self._check(self.lib.hdg_info(self.h, ctypes.byref(info)))
        return info.bounds_error

    def profile(self, enable=True):
        """Start (clears totals) or stop per-phase CUDA-event timing in the library."""
        self._check(self.lib.hdg_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        """{phase: (timed launches, total ms)} since the last start."""
        pr = Profile()
        self._check(self.lib.hdg_profile_read(self.h, ctypes.byref(pr)))
        return {name: (pr.count[i], pr.ms[i]) for i, name in enumerate(PROF_PHASES)}

    # ------------------------------------------------------------------ utils
    def _check(self, st):
        if st != HDG_OK:
            raise HDGError(st, self.lib.hdg_last_error(self.h).decode())

    def _f64(self, *shape):
        return torch.empty(*shape, dtype=torch.float64, device=self.device)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.hdg_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------- API
    def offsets(self, which):
        """Prefix sums of a ragged layout (OFF_* table), host int64 tensor."""
        count = {OFF_SOURCE: self.info["N"], OFF_LATTICE: self.info["N"], OFF_SCHUR: self.info["N"],
                 OFF_TRACE: self.info["n_int_edges"], OFF_DIRICHLET_POINTS: self.info["n_bnd_edges"],
                 OFF_DIRICHLET_TRACE: self.info["n_bnd_edges"]}[which]
        out = torch.empty(count + 1, dtype=torch.int64)
        self._check(self.lib.hdg_offsets(self.h, which, _ptr(out)))
        return out

    def quad_points(self):
        """[N, n_qp, 2]; on a level mesh [n_qp_total, 2] (element e's at offsets(OFF_SOURCE)[e])."""
        if self.levels:
            xy = self._f64(self.info["n_qp_total"], 2)
        else:
            xy = self._f64(self.info["N"], self.info["n_qp"], 2)
        self._check(self.lib.hdg_quad_points(self.h, _ptr(xy)))
        return xy

    def bnd_quad_points(self):
        if self.levels:
            xy = self._f64(self.info["n_bqp_total"], 2)
        else:
            xy = self._f64(self.info["n_bnd_edges"], self.info["n_bqp"], 2)
        self._check(self.lib.hdg_bnd_quad_points(self.h, _ptr(xy)))
        return xy

    def set_source(self, f_qp, gD_qp=None):
        """f_qp: [N, n_qp] (one source) or [nrhs, N, n_qp]; gD_qp likewise ([4n, n_bqp] or
        [nrhs, 4n, n_bqp]) or None."""
        f_qp = f_qp.to(self.device, torch.float64).contiguous()
        one = 1 if self.levels else 2          # dimensions of one source
        nrhs = 1 if f_qp.dim() == one else f_qp.shape[0]
        gD_qp = None if gD_qp is None else gD_qp.to(self.device, torch.float64).contiguous()
        self._src = (f_qp, gD_qp)       # keep alive until condense / recover
        self.nrhs = nrhs
        self._check(self.lib.hdg_set_source(self.h, _ptr(f_qp), _ptr(gD_qp), nrhs))

    def condense(self, store_fp32=False, keep_factors=True, store_df64=False, split_update=False, precond="d",
                 tc_update=False, store_fix=False):
        """precond: "d" (D_f^-1 of Sec. 6.1) or "face_schur" (the inverted diagonal face blocks of S).
        split_update: split-FP32 elimination; tc_update: FP64 elimination with the trailing
        updates on the tensor cores (exact 8-bit slices); store_fix: also keep the
        preconditioned blocks as 56-bit fixed-point rows (mode 3, apply prec 56)."""
        if precond not in ("d", "face_schur"):
            raise ValueError("precond must be 'd' or 'face_schur'")
        flags = ((HDG_STORE_FP32 if store_fp32 else 0) | (HDG_KEEP_FACTORS if keep_factors else 0)
                 | (HDG_STORE_DF64 if store_df64 else 0) | (HDG_SPLIT_UPDATE if split_update else 0)
                 | (HDG_PRECOND_FACE_SCHUR if precond == "face_schur" else 0) | (HDG_TC_UPDATE if tc_update else 0)
                 | (HDG_STORE_FIX64 if store_fix else 0))
        self._check(self.lib.hdg_condense(self.h, flags))
        self.version += 1

    def rhs(self):
        """[N_tr], or [nrhs, N_tr] for several sources."""
        nrhs = getattr(self, "nrhs", 1)
        g = self._f64(self.info["N_tr"]) if nrhs == 1 else self._f64(nrhs, self.info["N_tr"])
        self._check(self.lib.hdg_rhs(self.h, _ptr(g)))
        return g

    def apply(self, x, precond=False, prec=64, out=None):
        """x: [N_tr] or [nrhs, N_tr] (multi-RHS apply); prec = 49: x [N_tr, 2] FP32 split pairs
        (the split-FP32 solve's own operator and launch shape), y likewise."""
        dt = torch.float32 if prec in (32, 49) else torch.float64   # 64, 56, 48, 33: FP64 vectors
        x = x.to(self.device, dt).contiguous()
        nrhs = 1 if x.dim() == 1 or prec == 49 else x.shape[0]
        y = out if out is not None else torch.empty_like(x)
        self._check(self.lib.hdg_apply(self.h, _ptr(x), _ptr(y), nrhs, prec, 1 if precond else 0))
        return y

    def solve(self, g, x0=None, tol=1e-10, maxit=20000, restart=50, mode=0, check=True, orth=0, basis=BASIS_FP64,
              augment=0):
        """g: [N_tr], or [nrhs, N_tr] (independent systems solved in lockstep: one multi-RHS
        apply and batched vector kernels per Arnoldi step; the report is the worst column's).
        mode: Arnoldi operator, 0 FP64 blocks, 1 FP32 blocks (FP64 refinement), 2 split-FP32 blocks,
        3 fixed-point rows with exact integer products (condense(store_fix=True)).
        basis: BASIS_FP64 (FP64 Krylov basis and orthogonalisation), BASIS_DF64 (split-FP32) or
        BASIS_FIX (fixed-point chunks, products exact in integers; one right-hand side).
        augment: 0..3 corrections of earlier restart cycles added to each cycle's search space
        (augmented restarts, LGMRES)."""
        g = g.to(self.device, torch.float64).contiguous()
        nrhs = 1 if g.dim() == 1 else g.shape[0]
        x = torch.zeros_like(g) if x0 is None else x0.to(self.device, torch.float64).clone()
        o = SolveOpts(tol=tol, maxit=maxit, restart=restart, mode=mode, orth=orth, basis=basis, augment=augment)
        r = SolveReport()
        st = self.lib.hdg_solve(self.h, _ptr(g), _ptr(x), nrhs, ctypes.byref(o), ctypes.byref(r))
        if check and st not in (HDG_OK, HDG_ERR_NOCONV):
            self._check(st)
        return x, r.as_dict(), st

    def set_wait_hooks(self, wait_cycles=0, skip_copy_edge=-1):
        """hdg_set_wait_hooks: the limit of the pipelined apply's bounded waits and its
        copy-skip test hook."""
        self._check(self.lib.hdg_set_wait_hooks(self.h, int(wait_cycles), int(skip_copy_edge)))

    def set_apply_shape(self, mode, edges_per_block=0, bulk_warps=0):
        """hdg_set_apply_shape: the apply's launch shape inside solves of this mode."""
        self._check(self.lib.hdg_set_apply_shape(self.h, mode, edges_per_block, bulk_warps))

    def autotune(self, mode=0, restart=80, basis=BASIS_FP64):
        """hdg_autotune: time candidate launch shapes of the GMRES kernels for this mode and
        problem size, keep the fastest; returns the report as a dict."""
        o = SolveOpts(tol=1e-10, maxit=1, restart=restart, mode=mode, orth=0, basis=basis)
        r = TuneReport()
        self._check(self.lib.hdg_autotune(self.h, ctypes.byref(o), ctypes.byref(r)))
        return r.as_dict()

    def recover(self, x):
        """x: [N_tr] -> u [N, Q], q [N, 2, Q]; or [nrhs, N_tr] -> [nrhs, ...]."""
        x = x.to(self.device, torch.float64).contiguous()
        N, Q = self.info["N"], self.info["Q"]
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        lead = () if x.dim() == 1 else (nrhs,)
        if self.levels:
            # ragged: u [n_u_total], q [2 n_u_total] (element e's [2][Q_e] at 2 offsets(OFF_LATTICE)[e])
            u = self._f64(*lead, self.info["n_u_total"])
            q = self._f64(*lead, 2 * self.info["n_u_total"])
        else:
            u = self._f64(*lead, N, Q)
            q = self._f64(*lead, N, 2, Q)
        self._check(self.lib.hdg_recover(self.h, _ptr(x), _ptr(u), _ptr(q), nrhs))
        return u, q

    def schur(self, e0=0, count=None):
        """[count, n_t, n_t]; on a level mesh the ragged blocks flat (offsets(OFF_SCHUR))."""
        count = self.info["N"] - e0 if count is None else count
        if self.levels:
            off = self.offsets(OFF_SCHUR)
            S = self._f64(int(off[e0 + count] - off[e0]))
        else:
            S = self._f64(count, self.info["n_t"], self.info["n_t"])
        self._check(self.lib.hdg_get_schur(self.h, e0, count, _ptr(S)))
        return S

    def condense_static(self, e0, count, S_out, g_out=None):
        """hdg_condense_static: condense elements e0..e0+count-1 into caller buffers using the
        library's fixed scratch array (no device allocation inside the call)."""
        self._check(self.lib.hdg_condense_static(self.h, e0, count, _ptr(S_out), _ptr(g_out)))

    def run_host(self, f_host, gD_host=None, tol=1e-10, maxit=20000, restart=50, outputs=True, mode=0, orth=0,
                 basis=BASIS_FP64):
        """End-to-end call on host (ideally pinned) tensors; returns (x, u, q, report)."""
        N, Q, N_tr = self.info["N"], self.info["Q"], self.info["N_tr"]
        x = torch.empty(N_tr, dtype=torch.float64, pin_memory=True) if outputs else None
        u = torch.empty(N, Q, dtype=torch.float64, pin_memory=True) if outputs else None
        q = torch.empty(N, 2, Q, dtype=torch.float64, pin_memory=True) if outputs else None
        o = SolveOpts(tol=tol, maxit=maxit, restart=restart, mode=mode, orth=orth, basis=basis)
        r = SolveReport()
        st = self.lib.hdg_run_host(self.h, _ptr(f_host), _ptr(gD_host), ctypes.byref(o), _ptr(x), _ptr(u),
                                   _ptr(q), ctypes.byref(r))
        if st not in (HDG_OK, HDG_ERR_NOCONV):
            self._check(st)
        return x, u, q, r.as_dict()

    # ------------------------------------------------------- adjoint / gradient
    def set_kappa(self, kappa):
        """hdg_set_kappa: new per-element diffusivities ([N], >= 0); condense again afterwards."""
        k = torch.as_tensor(kappa, dtype=torch.float64).to(self.device).contiguous()
        self._check(self.lib.hdg_set_kappa(self.h, _ptr(k)))
        self.version += 1

    def transpose(self):
        """hdg_transpose: the stored operator becomes S^T (again: S)."""
        self._check(self.lib.hdg_transpose(self.h))

    def adjoint_rhs(self, r):
        r = r.to(self.device, torch.float64).contiguous()
        g = self._f64(self.info["N_tr"])
        self._check(self.lib.hdg_adjoint_rhs(self.h, _ptr(r), _ptr(g)))
        return g

    def adjoint_recover(self, r, nu):
        r = r.to(self.device, torch.float64).contiguous()
        nu = nu.to(self.device, torch.float64).contiguous()
        mu = self._f64(self.info["N"], self.info["Q"])
        self._check(self.lib.hdg_adjoint_recover(self.h, _ptr(r), _ptr(nu), _ptr(mu)))
        return mu

    def gradient(self, x, u, mu, nu, want_df=True):
        dk = self._f64(self.info["N"])
        df = self._f64(self.info["N"], self.info["n_qp"]) if want_df else None
        args = [t.to(self.device, torch.float64).contiguous() for t in (x, u, mu, nu)]
        self._check(self.lib.hdg_gradient(self.h, *[_ptr(t) for t in args], _ptr(dk), _ptr(df)))
        return dk, df

    def adjoint(self, r, x, u, tol=1e-10, maxit=20000, restart=80, mode=0, want_df=True, orth=0, basis=BASIS_FP64):
        """dJ/dkappa [N] and dJ/df [N, n_qp] for dJ/du = r [N, Q], at the forward solution
        (x, u) of the current condensation (factors kept). Returns (dkappa, df, report)."""
        g = self.adjoint_rhs(r)
        self.transpose()
        try:
            nu, rep, st = self.solve(g, tol=tol, maxit=maxit, restart=restart, mode=mode, orth=orth, basis=basis)
        finally:
            self.transpose()
        if st != HDG_OK:
            raise HDGError(st, f"adjoint solve did not converge: {rep}")
        mu = self.adjoint_recover(r, nu)
        dk, df = self.gradient(x, u, mu, nu, want_df)
        return dk, df, rep


class HDGSolve(torch.autograd.Function):
    """u = solve(kappa, f): element values of the macro-element HDG solution as a
    differentiable function of the per-element diffusivities and the source values
    at the quadrature points; the backward pass is the discrete adjoint
    (hdg_adjoint_rhs, a transposed GMRES solve, hdg_adjoint_recover, hdg_gradient).
    If the problem was condensed again between forward and backward, the
    backward pass first condenses it again at the saved kappa and f."""

    @staticmethod
    def _prepare(problem, kappa, f, gD, mode, split, precond="d"):
        problem.set_kappa(kappa)
        problem.set_source(f, gD)
        problem.condense(keep_factors=True, store_fp32=(mode == 1), store_df64=(mode == 2), split_update=split,
                         precond=precond, store_fix=(mode == 3))

    @staticmethod
    def forward(ctx, kappa, f, problem, gD, opts):
        opts = dict(opts or {})
        tol, restart, mode = opts.get("tol", 1e-10), opts.get("restart", 80), opts.get("mode", 0)
        split, orth = opts.get("split_update", False), opts.get("orth", 0)
        precond, basis = opts.get("precond", "d"), opts.get("basis", BASIS_FP64)
        kappa_d, f_d = kappa.detach(), f.detach()
        HDGSolve._prepare(problem, kappa_d, f_d, gD, mode, split, precond)
        x, rep, st = problem.solve(problem.rhs(), tol=tol, restart=restart, mode=mode,
                                   maxit=opts.get("maxit", 20000), orth=orth, basis=basis)
        if st != HDG_OK:
            raise HDGError(st, f"forward solve did not converge: {rep}")
        u, _ = problem.recover(x)
        ctx.problem, ctx.version = problem, problem.version
        ctx.opts = (tol, restart, mode, split, orth, precond, basis)
        ctx.gD = gD
        ctx.save_for_backward(x, u, kappa_d, f_d)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        pr = ctx.problem
        x, u, kappa, f = ctx.saved_tensors
        tol, restart, mode, split, orth, precond, basis = ctx.opts
        if pr.version != ctx.version:
            HDGSolve._prepare(pr, kappa, f, ctx.gD, mode, split, precond)
        dk, df, _ = pr.adjoint(grad_u, x, u, tol=tol, restart=restart, mode=mode,
                               want_df=ctx.needs_input_grad[1], orth=orth, basis=basis)
        return (dk if ctx.needs_input_grad[0] else None), df, None, None, None


def solve_u(problem, kappa, f, gD=None, **opts):
    """Differentiable u = solve(kappa, f) on `problem` (see HDGSolve)."""
    return HDGSolve.apply(kappa, f, problem, gD, opts)
