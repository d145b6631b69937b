"""GB300-native even-odd staggered multi-shift CG (Gupta & Majumdar, arXiv:1710.09178, Sections 3-4).

Thin ctypes binding over liblqcd.so (include/lqcd.h).  Every step of the path
runs in the library's CUDA kernels; this module only marshals arguments
(torch tensors -> device pointers, stream handles, the stats struct).  There is
no CPU fallback: if the library is missing, every call raises.

    from paper_1710_09178_gb300 import Context, mshift_cg, dslash_eo
    ctx = Context((32, 32, 32, 8), mass=0.02)
    ctx.set_gauge(U)                      # complex128 cuda tensor (V, 4, 3, 3)
    st = mshift_cg(ctx, shifts, residues, c0, b, xs, y, tol=1e-10, prec=FP32)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblqcd.so")
LIB_DEBUG_PATH = os.path.join(HERE, "liblqcd_debug.so")

LQCD_OK = 0
LQCD_ERR_ARG = 1
LQCD_ERR_DIMS = 2
LQCD_ERR_CUDA = 3
LQCD_ERR_NOT_CONVERGED = 4
LQCD_ERR_NONFINITE = 5
LQCD_ERR_STATE = 6

FP64 = 0
FP32 = 1
FP32_R12 = 2
FP16FIX = 3
FP32_R8 = 4
FP32_L16 = 5
DF64 = 6
PRECISIONS = {"fp64": FP64, "fp32": FP32, "fp32_r12": FP32_R12, "fp16fix": FP16FIX, "fp32_r8": FP32_R8,
              "fp32_l16": FP32_L16, "df64": DF64}

OPT_RELIABLE_INTERVAL = 1
OPT_REFINE = 2
OPT_BATCH = 3
OPT_USE_GRAPH = 4
OPT_DSLASH_TPS = 5
OPT_RELIABLE_DELTA = 6
OPT_PDL = 7
OPT_DF_RESID = 8
OPT_DF_SWITCH = 9
OPT_DSLASH_BS = 10
OPT_DSLASH_ORDER = 11

MAX_SHIFTS = 32
MAX_BATCH = 128
MAX_RHS = 4

EXPORTED = [
    "lqcd_create", "lqcd_destroy", "lqcd_last_error", "lqcd_set_stream", "lqcd_set_gauge", "lqcd_vector_bytes",
    "lqcd_pack_vector", "lqcd_unpack_vector", "dslash_eo", "lqcd_apply_A", "lqcd_neighbour_table",
    "lqcd_set_option", "mshift_cg", "lqcd_rational_coeffs", "lqcd_launch_count", "lqcd_apply_A_noalloc",
    "fermion_force", "rhmc_trajectory", "mshift_cg_batch", "lqcd_autotune",
    "lqcd_share_gauge", "dslash_eo_batch", "lqcd_bounds_word", "mshift_cg_multi", "lqcd_autotune_shape",
]


class SolveStats(ctypes.Structure):
    """lqcd_solve_stats: iterations, reliable updates, refinement work, the FP64-class true
    residual of every shift, kernel launches and time of one mshift_cg call."""

    _fields_ = [
        ("iterations", ctypes.c_int),
        ("reliable_updates", ctypes.c_int),
        ("refine_iterations", ctypes.c_int),
        ("refined_shifts", ctypes.c_int),
        ("refine_rounds", ctypes.c_int),
        ("kernel_launches", ctypes.c_int),
        ("n_shifts", ctypes.c_int),
        ("true_residual", ctypes.c_double * MAX_SHIFTS),
        ("ms", ctypes.c_double),
        ("shift_iterations", ctypes.c_int),
        ("df_iterations", ctypes.c_int),
    ]

    def as_dict(self):
        """The fields as a dict (true_residual cut to the solve's shifts)."""
        n = self.n_shifts
        return dict(iterations=self.iterations, reliable_updates=self.reliable_updates,
                    refine_iterations=self.refine_iterations, refined_shifts=self.refined_shifts,
                    refine_rounds=self.refine_rounds,
                    kernel_launches=self.kernel_launches, true_residual=list(self.true_residual[:n]), ms=self.ms,
                    shift_iterations=self.shift_iterations, df_iterations=self.df_iterations)


class BatchProblem(ctypes.Structure):
    """lqcd_batch_problem: one independent shifted-CG problem of mshift_cg_batch."""

    _fields_ = [
        ("ctx", ctypes.c_void_p), ("shifts", ctypes.POINTER(ctypes.c_double)),
        ("residues", ctypes.POINTER(ctypes.c_double)), ("n", ctypes.c_int), ("c0", ctypes.c_double),
        ("b_dev", ctypes.c_void_p), ("x_dev", ctypes.POINTER(ctypes.c_void_p)), ("y_dev", ctypes.c_void_p),
        ("tol", ctypes.c_double), ("maxiter", ctypes.c_int), ("prec", ctypes.c_int),
        ("stats", ctypes.POINTER(SolveStats)), ("status", ctypes.c_int),
        ("nrhs", ctypes.c_int), ("b_devs", ctypes.POINTER(ctypes.c_void_p)),
        ("x_devs", ctypes.POINTER(ctypes.c_void_p)), ("y_devs", ctypes.POINTER(ctypes.c_void_p)),
    ]


class RhmcParams(ctypes.Structure):
    """lqcd_rhmc_params: gauge coupling, trajectory length and steps, the rational
    approximations of the action and the heatbath, solver tolerances and precisions."""

    _fields_ = [
        ("beta", ctypes.c_double), ("tau", ctypes.c_double), ("nsteps", ctypes.c_int), ("lambda_", ctypes.c_double),
        ("n_act", ctypes.c_int), ("act_shifts", ctypes.POINTER(ctypes.c_double)),
        ("act_residues", ctypes.POINTER(ctypes.c_double)), ("act_c0", ctypes.c_double),
        ("n_heat", ctypes.c_int), ("heat_shifts", ctypes.POINTER(ctypes.c_double)),
        ("heat_residues", ctypes.POINTER(ctypes.c_double)), ("heat_c0", ctypes.c_double),
        ("tol", ctypes.c_double), ("md_tol", ctypes.c_double), ("maxiter", ctypes.c_int), ("prec", ctypes.c_int),
        ("prec_action", ctypes.c_int), ("phi_given", ctypes.c_int), ("mom_out", ctypes.c_void_p),
        ("links_out", ctypes.c_void_p),
    ]


class TrajResult(ctypes.Structure):
    """lqcd_traj_result: the FP64 Hamiltonian pieces before and after, dH, acceptance, solver work."""

    _fields_ = [
        ("dH", ctypes.c_double), ("H0", ctypes.c_double), ("H1", ctypes.c_double),
        ("kinetic0", ctypes.c_double), ("kinetic1", ctypes.c_double), ("gauge0", ctypes.c_double),
        ("gauge1", ctypes.c_double), ("fermion0", ctypes.c_double), ("fermion1", ctypes.c_double),
        ("accepted", ctypes.c_int), ("solves", ctypes.c_int), ("iterations", ctypes.c_int), ("ms", ctypes.c_double),
    ]

    def as_dict(self):
        """The fields as a dict."""
        return {name: getattr(self, name) for name, _ in self._fields_}


class LqcdError(RuntimeError):
    """A non-zero status of a library call; .code is the LQCD_* status."""

    def __init__(self, code, msg):
        super().__init__(f"lqcd error {code}: {msg}")
        self.code = code


_lib = None
_lib_debug = None


def load_library(path: str = LIB_PATH):
    """Load liblqcd.so (built by build.build()); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    _lib = _bind(path)
    return _lib


def load_debug_library():
    """liblqcd_debug.so, the build with device-side neighbour-index checks (build.build(debug=True)),
    loaded beside the release library; pass it to Context(..., lib=...) to run contexts on it."""
    global _lib_debug
    if _lib_debug is None:
        _lib_debug = _bind(LIB_DEBUG_PATH)
    return _lib_debug


def _bind(path):
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run `python -c 'import __graft_entry__ as g; g.build()'` first")
    lib = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "lqcd_create": (i, [ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int), d, vp]),
        "lqcd_destroy": (i, [vp]),
        "lqcd_last_error": (ctypes.c_char_p, [vp]),
        "lqcd_set_stream": (i, [vp, vp]),
        "lqcd_set_gauge": (i, [vp, vp]),
        "lqcd_vector_bytes": (ctypes.c_size_t, [vp, i]),
        "lqcd_pack_vector": (i, [vp, vp, i, vp]),
        "lqcd_unpack_vector": (i, [vp, vp, vp, i]),
        "dslash_eo": (i, [vp, vp, vp, i, i]),
        "lqcd_apply_A": (i, [vp, vp, vp, d, i, ctypes.POINTER(d)]),
        "lqcd_neighbour_table": (i, [vp, vp, vp, vp]),
        "lqcd_set_option": (i, [vp, i, d]),
        "mshift_cg": (i, [vp, ctypes.POINTER(d), ctypes.POINTER(d), i, d, vp, ctypes.POINTER(vp), vp, d, i, i,
                          ctypes.POINTER(SolveStats)]),
        "lqcd_rational_coeffs": (i, [d, d, d, i, ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(d),
                                     ctypes.POINTER(d)]),
        "lqcd_launch_count": (ctypes.c_longlong, [vp]),
        "lqcd_apply_A_noalloc": (i, [vp, vp, vp, d, i, ctypes.POINTER(d)]),
        "fermion_force": (i, [vp, ctypes.POINTER(d), ctypes.POINTER(d), i, d, vp, vp, vp, ctypes.POINTER(d), d, i, i,
                              ctypes.POINTER(SolveStats)]),
        "rhmc_trajectory": (i, [vp, ctypes.POINTER(RhmcParams), vp, vp, vp, d, ctypes.POINTER(TrajResult)]),
        "mshift_cg_batch": (i, [ctypes.POINTER(BatchProblem), i, i]),
        "lqcd_autotune": (i, [vp, i, ctypes.POINTER(ctypes.c_int)]),
        "lqcd_autotune_shape": (i, [vp, i, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int)]),
        "lqcd_share_gauge": (i, [vp, vp]),
        "dslash_eo_batch": (i, [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i), i, i]),
        "lqcd_bounds_word": (i, [vp, ctypes.POINTER(ctypes.c_uint)]),
        "mshift_cg_multi": (i, [vp, i, ctypes.POINTER(d), ctypes.POINTER(d), i, d, ctypes.POINTER(vp),
                                ctypes.POINTER(vp), ctypes.POINTER(vp), d, i, i, ctypes.POINTER(SolveStats)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _current_stream():
    import torch

    return torch.cuda.current_stream().cuda_stream


class Context:
    """Owns one lqcd_ctx (device workspace and internal gauge copies) for a lattice."""

    def __init__(self, dims, mass, stream=None, lib=None):
        lib = lib if lib is not None else load_library()
        self.lib = lib
        self.dims = tuple(int(d) for d in dims)
        self.mass = float(mass)
        self.V = int(np.prod(self.dims))
        self.Vh = self.V // 2
        arr = (ctypes.c_int * 4)(*self.dims)
        h = ctypes.c_void_p()
        rc = lib.lqcd_create(ctypes.byref(h), arr, self.mass, stream if stream is not None else _current_stream())
        if rc != LQCD_OK:
            raise LqcdError(rc, f"lqcd_create failed for dims {self.dims}")
        self.handle = h

    def close(self):
        """Free the context (lqcd_destroy); further calls on it are invalid."""
        if getattr(self, "handle", None):
            self.lib.lqcd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc):
        """Raise LqcdError with the context's last message unless rc is LQCD_OK."""
        if rc != LQCD_OK:
            msg = self.lib.lqcd_last_error(self.handle)
            raise LqcdError(rc, msg.decode() if msg else "")
        return rc

    def set_stream(self, stream=None):
        """Enqueue the context's work on `stream` (a cudaStream_t; default torch's current stream)."""
        return self.check(self.lib.lqcd_set_stream(self.handle, stream if stream is not None
                                                         else _current_stream()))

    def set_gauge(self, U):
        """U: complex128 cuda tensor of shape (V, 4, 3, 3), canonical layout."""
        assert tuple(U.shape) == (self.V, 4, 3, 3) and U.is_contiguous()
        return self.check(self.lib.lqcd_set_gauge(self.handle, _ptr(U)))

    def share_gauge(self, src):
        """Use src's gauge copies (lqcd_share_gauge); src must outlive this context."""
        self._gauge_src = src  # keep the owner alive
        return self.check(self.lib.lqcd_share_gauge(self.handle, src.handle))

    def vector_bytes(self, prec):
        """Bytes of one internal half-lattice vector of precision prec (lqcd_vector_bytes)."""
        return int(self.lib.lqcd_vector_bytes(self.handle, prec))

    def new_vector(self, prec):
        """Uninitialised internal vector of precision prec (uint8 cuda tensor)."""
        import torch

        return torch.empty(self.vector_bytes(prec), dtype=torch.uint8, device="cuda")

    def pack(self, dst, prec, src):
        """Canonical complex128 [V/2][3] cuda tensor src -> internal vector dst of precision prec."""
        return self.check(self.lib.lqcd_pack_vector(self.handle, _ptr(dst), prec, _ptr(src)))

    def unpack(self, dst, src, prec):
        """Internal vector src of precision prec -> canonical complex128 [V/2][3] cuda tensor dst."""
        return self.check(self.lib.lqcd_unpack_vector(self.handle, _ptr(dst), _ptr(src), prec))

    def apply_A(self, q, p, sigma, prec, want_dot=False):
        """q = (A + sigma) p on internal vectors (lqcd_apply_A); returns Re<p, q> if want_dot."""
        pq = ctypes.c_double(0.0)
        self.check(self.lib.lqcd_apply_A(self.handle, _ptr(q), _ptr(p), float(sigma), prec,
                                               ctypes.byref(pq) if want_dot else None))
        return pq.value if want_dot else None

    def apply_A_noalloc(self, q, p, sigma, prec, want_dot=False):
        """apply_A with the library's static scratch instead of allocated scratch (see include/lqcd.h)."""
        pq = ctypes.c_double(0.0)
        self.check(self.lib.lqcd_apply_A_noalloc(self.handle, _ptr(q), _ptr(p), float(sigma), prec,
                                                       ctypes.byref(pq) if want_dot else None))
        return pq.value if want_dot else None

    def neighbour_table(self, fwd, bwd, sign):
        """Fill int32 [2][4][V/2] tensors with the forward and backward neighbours and hop signs."""
        return self.check(self.lib.lqcd_neighbour_table(self.handle, _ptr(fwd), _ptr(bwd), _ptr(sign)))

    def set_option(self, key, value):
        """lqcd_set_option(key, value) with an OPT_* key."""
        return self.check(self.lib.lqcd_set_option(self.handle, int(key), float(value)))

    def autotune(self, prec=FP32):
        """Pick the fastest Dslash launch shape on this lattice (lqcd_autotune); returns the threads
        per site (the block size and order chosen are set too: autotune_shape reports them)."""
        best = ctypes.c_int(0)
        self.check(self.lib.lqcd_autotune(self.handle, int(prec), ctypes.byref(best)))
        return best.value

    def autotune_shape(self, prec=FP32):
        """Pick the fastest Dslash launch shape on this lattice (lqcd_autotune_shape); returns
        (threads per site, threads per block, block-to-site order)."""
        t, b, o = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        self.check(self.lib.lqcd_autotune_shape(self.handle, int(prec), ctypes.byref(t), ctypes.byref(b),
                                                ctypes.byref(o)))
        return t.value, b.value, o.value

    def launch_count(self):
        """Kernels the library has launched on this context (graph nodes counted)."""
        return int(self.lib.lqcd_launch_count(self.handle))


def dslash_eo(ctx: Context, out, in_, out_parity: int, prec: int):
    """out = D_oe in (out_parity=1) or D_eo in (out_parity=0); internal vectors of precision prec."""
    return ctx.check(ctx.lib.dslash_eo(ctx.handle, _ptr(out), _ptr(in_), int(out_parity), int(prec)))


def dslash_eo_batch(ctxs, outs, ins, out_parities, prec: int):
    """dslash_eo on several lattices in one persistent launch (dslash_eo_batch); the lists are
    indexed alike; launched on ctxs[0]'s stream."""
    n = len(ctxs)
    if not (len(outs) == len(ins) == len(out_parities) == n):
        raise ValueError("dslash_eo_batch: lists of different lengths")
    H = ctypes.c_void_p * n
    rc = ctxs[0].lib.dslash_eo_batch(H(*[c.handle.value for c in ctxs]), H(*[_ptr(o) for o in outs]),
                                        H(*[_ptr(x) for x in ins]),
                                        (ctypes.c_int * n)(*[int(p) for p in out_parities]), n, int(prec))
    return ctxs[0].check(rc)


def mshift_cg(ctx: Context, shifts, residues, c0, b, xs=None, y=None, tol=1e-10, maxiter=20000, prec=FP32,
              raise_on_error=True):
    """Shifted CG (A + d_k) x_k = b for every shift and y = c0 b + sum_k c_k x_k.

    b, xs[k], y: complex128 cuda tensors of shape (Vh, 3) (canonical layout).
    Returns (status, stats dict).
    """
    lib = ctx.lib
    n = len(shifts)
    sh = (ctypes.c_double * n)(*[float(s) for s in shifts])
    rs = (ctypes.c_double * n)(*[float(c) for c in residues]) if residues is not None else None
    xp = (ctypes.c_void_p * n)(*[_ptr(x) for x in xs]) if xs is not None else None
    st = SolveStats()
    rc = lib.mshift_cg(ctx.handle, sh, rs, n, float(c0), _ptr(b), xp, _ptr(y), float(tol), int(maxiter),
                       int(prec), ctypes.byref(st))
    if raise_on_error and rc not in (LQCD_OK,):
        ctx.check(rc)
    return rc, st.as_dict()


def mshift_cg_multi(ctx: Context, shifts, residues, c0, bs, xs=None, ys=None, tol=1e-10, maxiter=20000, prec=FP32,
                    raise_on_error=True):
    """mshift_cg for several right-hand sides bs[s] of one lattice at once (mshift_cg_multi).

    bs[s], xs[s][k], ys[s]: complex128 cuda tensors of shape (Vh, 3); xs and ys may be None, and so
    may any xs[s] or ys[s].  Returns (status, [stats dict per right-hand side])."""
    lib = ctx.lib
    n, S = len(shifts), len(bs)
    vp = ctypes.c_void_p
    sh = (ctypes.c_double * n)(*[float(v) for v in shifts])
    rs = (ctypes.c_double * n)(*[float(c) for c in residues]) if residues is not None else None
    bp = (vp * S)(*[_ptr(b) for b in bs])
    keep = []
    xp = None
    if xs is not None:
        rows = []
        for s in range(S):
            if xs[s] is None:
                rows.append(None)
            else:
                row = (vp * n)(*[_ptr(x) for x in xs[s]])
                keep.append(row)
                rows.append(ctypes.cast(row, vp).value)
        xp = (vp * S)(*rows)
    yp = (vp * S)(*[_ptr(y) for y in ys]) if ys is not None else None
    st = (SolveStats * S)()
    rc = lib.mshift_cg_multi(ctx.handle, S, sh, rs, n, float(c0), bp, xp, yp, float(tol), int(maxiter), int(prec), st)
    if raise_on_error and rc not in (LQCD_OK,):
        ctx.check(rc)
    return rc, [st[s].as_dict() for s in range(S)]


def fermion_force(ctx: Context, shifts, residues, c0, phi, F=None, Falg=None, want_action=True, tol=1e-10,
                  maxiter=20000, prec=FP32, raise_on_error=True):
    """Force of S_f = phi^+ r(A) phi: F (V,4,3,3 complex128) and/or Falg (V,4,8 float64) device tensors.

    Returns (status, S_f or None, stats dict).  dS_f/dw^a = tr(lambda^a F) = Falg[..., a] for
    U -> exp(i w.lambda/2) U.
    """
    lib = ctx.lib
    n = len(shifts)
    sh = (ctypes.c_double * n)(*[float(s) for s in shifts])
    rs = (ctypes.c_double * n)(*[float(c) for c in residues])
    act = ctypes.c_double(0.0)
    st = SolveStats()
    rc = lib.fermion_force(ctx.handle, sh, rs, n, float(c0), _ptr(phi), _ptr(F), _ptr(Falg),
                           ctypes.byref(act) if want_action else None, float(tol), int(maxiter), int(prec),
                           ctypes.byref(st))
    if raise_on_error and rc != LQCD_OK:
        ctx.check(rc)
    return rc, (act.value if want_action else None), st.as_dict()


class FermionAction:
    """torch.autograd.Function for S_f(U) = phi^+ r(A[U]) phi in the algebra coordinates w of
    U -> exp(i w.lambda/2) U at w = 0: forward returns S_f, backward returns dS_f/dw from the
    library's adjoint kernel (fermion_force)."""

    _fn = None

    @classmethod
    def function(cls):
        """The torch.autograd.Function class (built on first use)."""
        if cls._fn is None:
            import torch

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(actx, w, ctx, shifts, residues, c0, phi, tol, prec):
                    """S_f and, saved for backward, the force in the algebra coordinates."""
                    if bool(torch.any(w != 0)):
                        raise ValueError("FermionAction is evaluated at w = 0 (update U itself, then reset w)")
                    Falg = torch.empty((ctx.V, 4, 8), dtype=torch.float64, device=phi.device)
                    rc, S, st = fermion_force(ctx, shifts, residues, c0, phi, Falg=Falg, tol=tol, prec=prec)
                    actx.save_for_backward(Falg)
                    return torch.tensor(S, dtype=torch.float64, device=phi.device)

                @staticmethod
                def backward(actx, grad):
                    """dS_f/dw times the incoming gradient."""
                    (Falg,) = actx.saved_tensors
                    return grad * Falg, None, None, None, None, None, None, None

            cls._fn = _F
        return cls._fn

    @classmethod
    def apply(cls, w, ctx, shifts, residues, c0, phi, tol=1e-10, prec=FP32):
        """S_f at w = 0 as a differentiable scalar; its gradient with respect to w is the force."""
        return cls.function().apply(w, ctx, shifts, residues, c0, phi, tol, prec)


def mshift_cg_batch(problems, nthreads=16, raise_on_error=True):
    """Run independent shifted-CG problems concurrently (mshift_cg_batch).

    problems: list of dicts with keys ctx, shifts, residues, c0, b, xs (list or None), y (or None),
    tol, maxiter, prec; a problem with several sources of its lattice has bs (list of sources), xss
    (list of lists or None), ys (list or None) instead of b, xs, y (mshift_cg_multi).  Returns
    (status, [status per problem], [stats dict per problem, or list of them per source]).
    """
    lib = problems[0]["ctx"].lib if problems else load_library()
    n = len(problems)
    arr = (BatchProblem * n)()
    keep = []
    stats = []
    vp = ctypes.c_void_p
    for i, pr in enumerate(problems):
        ns = len(pr["shifts"])
        sh = (ctypes.c_double * ns)(*[float(v) for v in pr["shifts"]])
        rs = (ctypes.c_double * ns)(*[float(v) for v in pr["residues"]])
        keep += [sh, rs]
        a = arr[i]
        a.ctx = pr["ctx"].handle
        a.shifts, a.residues, a.n, a.c0 = sh, rs, ns, float(pr.get("c0", 0.0))
        if "bs" in pr:
            S = len(pr["bs"])
            a.nrhs = S
            bp = (vp * S)(*[_ptr(b) for b in pr["bs"]])
            keep.append(bp)
            a.b_devs = ctypes.cast(bp, ctypes.POINTER(vp))
            xss = pr.get("xss")
            if xss is not None:
                rows = []
                for row in xss:
                    if row is None:
                        rows.append(None)
                    else:
                        r = (vp * ns)(*[_ptr(x) for x in row])
                        keep.append(r)
                        rows.append(ctypes.cast(r, vp).value)
                xp = (vp * S)(*rows)
                keep.append(xp)
                a.x_devs = ctypes.cast(xp, ctypes.POINTER(vp))
            ys = pr.get("ys")
            if ys is not None:
                yp = (vp * S)(*[_ptr(y) for y in ys])
                keep.append(yp)
                a.y_devs = ctypes.cast(yp, ctypes.POINTER(vp))
            st = (SolveStats * S)()
            a.stats = ctypes.cast(st, ctypes.POINTER(SolveStats))
        else:
            xs = pr.get("xs")
            xp = (vp * ns)(*[_ptr(x) for x in xs]) if xs is not None else None
            keep.append(xp)
            a.b_dev = _ptr(pr["b"])
            a.x_dev = xp
            a.y_dev = _ptr(pr.get("y"))
            st = SolveStats()
            a.stats = ctypes.pointer(st)
        stats.append(st)
        a.tol, a.maxiter, a.prec = float(pr.get("tol", 1e-10)), int(pr.get("maxiter", 20000)), int(pr.get("prec", FP32))
    rc = lib.mshift_cg_batch(arr, n, int(nthreads))
    st = [arr[i].status for i in range(n)]
    if raise_on_error and rc != LQCD_OK:
        bad = st.index(rc) if rc in st else 0
        problems[bad]["ctx"].check(rc)
    out = [[x.as_dict() for x in s] if isinstance(s, ctypes.Array) else s.as_dict() for s in stats]
    return rc, st, out


def rhmc_trajectory(ctx: Context, U, mom, xi, uniform, beta, tau, nsteps, act, heat=None, tol=1e-10, md_tol=0.0,
                    maxiter=20000, prec=FP32, prec_action=FP64, phi_given=False, mom_out=None, links_out=None,
                    lam=0.0, raise_on_error=True):
    """One RHMC trajectory (see include/lqcd.h).  act = (c0, residues, shifts) of x^{-1/2},
    heat = (c0, residues, shifts) of x^{1/4}; U (V,4,3,3) complex128 updated in place if accepted;
    mom (V,4,8) float64; xi (Vh,3) complex128.  Returns (status, result dict)."""
    lib = ctx.lib
    arr = lambda v: (ctypes.c_double * len(v))(*[float(x) for x in v])
    a_c0, a_res, a_sh = act
    keep = [arr(a_sh), arr(a_res)]
    prm = RhmcParams()
    prm.beta, prm.tau, prm.nsteps, prm.lambda_ = float(beta), float(tau), int(nsteps), float(lam)
    prm.n_act, prm.act_shifts, prm.act_residues, prm.act_c0 = len(a_sh), keep[0], keep[1], float(a_c0)
    if heat is not None:
        h_c0, h_res, h_sh = heat
        keep += [arr(h_sh), arr(h_res)]
        prm.n_heat, prm.heat_shifts, prm.heat_residues, prm.heat_c0 = len(h_sh), keep[2], keep[3], float(h_c0)
    prm.tol, prm.md_tol, prm.maxiter, prm.prec, prm.prec_action = float(tol), float(md_tol), int(maxiter), int(prec), int(
        prec_action)
    prm.phi_given = 1 if phi_given else 0
    prm.mom_out = _ptr(mom_out)
    prm.links_out = _ptr(links_out)
    res = TrajResult()
    rc = lib.rhmc_trajectory(ctx.handle, ctypes.byref(prm), _ptr(U), _ptr(mom), _ptr(xi), float(uniform),
                             ctypes.byref(res))
    if raise_on_error and rc != LQCD_OK:
        ctx.check(rc)
    return rc, res.as_dict()


def lqcd_rational_coeffs(power, lo, hi, n):
    """(c0, residues, poles, err) of the best relative (n, n) rational approximation of x^power on [lo, hi]."""
    lib = load_library()
    c0 = ctypes.c_double()
    err = ctypes.c_double()
    res = (ctypes.c_double * n)()
    pol = (ctypes.c_double * n)()
    rc = lib.lqcd_rational_coeffs(float(power), float(lo), float(hi), int(n), ctypes.byref(c0), res, pol,
                                  ctypes.byref(err))
    if rc != LQCD_OK:
        raise LqcdError(rc, f"lqcd_rational_coeffs({power}, {lo}, {hi}, {n}) failed")
    return c0.value, np.array(res[:]), np.array(pol[:]), err.value


def rational_coeffs(power, lo, hi, n):
    """(c0, residues, poles, max relative error) of the type-(n, n) approximation of x^power on
    [lo, hi] (lqcd_rational_coeffs)."""
    return lqcd_rational_coeffs(power, lo, hi, n)
