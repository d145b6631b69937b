"""ctypes binding of the C++ oracle (oracle/cpp/oracle.cpp).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The C++ oracle computes what oracle/lattice.py, oracle/staggered.py, oracle/solvers.py and
oracle/encode16.py compute (Section 2 geometry, the Section 3.2 hopping operator and
A = 4m^2 - D_eo D_oe, the Section 4 shifted CG with its true residuals and Eq. ratapprx's
rational application, the 16-bit storage), in plain FP64 C++ with one loop per formula.  It
exists to time the oracle on the host's cores (one core, and OpenMP on all of them) and to
run the oracle at the full 32^3 x 8 size in seconds.  It is pinned by tests/test_oracle_cpp.py
against the same closed forms and dense solves as the numpy oracle, and element by element
against the numpy oracle itself.

Usage:
    lib = load(threaded=True)          # or threaded=False for the one-core build
    lat = lib.lattice(dims, U, mass)   # U: complex128 (V, 4, 3, 3), kept alive by lat
    out = lat.dslash_eo(psi, 1)        # D_oe psi
    xs, info = lat.multishift_cg(b, shifts, tol=1e-10)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBS = {}


class CgInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("shift_iterations", ctypes.c_long), ("rr", ctypes.c_double),
                ("zeta", ctypes.c_double * 64), ("seconds", ctypes.c_double), ("seconds_dslash", ctypes.c_double),
                ("dslash_calls", ctypes.c_long)]


_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


def _ptr(a):
    return a.ctypes.data_as(_vp)


def load(threaded: bool = False) -> "CppOracle":
    """The one-core (threaded=False) or OpenMP (threaded=True) build, compiled on first use."""
    key = "omp" if threaded else "serial"
    if key not in _LIBS:
        import importlib.util

        spec = importlib.util.spec_from_file_location("_orc_build", os.path.join(_HERE, "cpp", "build.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        path = mod.build()[key]
        _LIBS[key] = CppOracle(ctypes.CDLL(path), threaded)
    return _LIBS[key]


class CppOracle:
    def __init__(self, lib, threaded):
        self.lib = lib
        self.threaded = threaded
        lib.orc_create.restype = _vp
        lib.orc_create.argtypes = [ctypes.POINTER(ctypes.c_int), _vp, ctypes.c_double]
        lib.orc_destroy.argtypes = [_vp]
        lib.orc_threads.restype = ctypes.c_int
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_neighbour_tables.argtypes = [_vp, _vp, _vp, _vp, _vp]
        lib.orc_dslash_eo.argtypes = [_vp, _vp, _vp, ctypes.c_int]
        lib.orc_A_apply.argtypes = [_vp, _vp, _vp, ctypes.c_double]
        lib.orc_cg.restype = ctypes.c_int
        lib.orc_cg.argtypes = [_vp, ctypes.c_double, _vp, _vp, ctypes.c_double, ctypes.c_int]
        lib.orc_mshift_cg.restype = ctypes.c_int
        lib.orc_mshift_cg.argtypes = [_vp, _vp, ctypes.c_int, _vp, ctypes.c_double, ctypes.c_int, ctypes.c_int, _vp,
                                      ctypes.POINTER(CgInfo)]
        lib.orc_true_residuals.argtypes = [_vp, _vp, ctypes.c_int, _vp, _vp, _vp]
        lib.orc_rational_apply.argtypes = [ctypes.c_long, _vp, ctypes.c_int, _vp, ctypes.c_double, _vp, _vp]
        lib.orc_encode16.argtypes = [ctypes.c_long, _vp, _vp, _vp]
        lib.orc_decode16.argtypes = [ctypes.c_long, _vp, _vp, _vp]

    def threads(self) -> int:
        return int(self.lib.orc_threads())

    def set_threads(self, n: int) -> None:
        self.lib.orc_set_threads(int(n))

    def lattice(self, dims, U, mass) -> "Lattice":
        return Lattice(self, dims, U, mass)

    def rational_apply(self, b, xs, c0, residues):
        b = np.ascontiguousarray(b, dtype=np.complex128)
        X = np.ascontiguousarray(np.stack(xs), dtype=np.complex128)
        res = np.ascontiguousarray(residues, dtype=np.float64)
        y = np.empty_like(b)
        self.lib.orc_rational_apply(b.shape[0], _ptr(b), len(res), _ptr(X), float(c0), _ptr(res), _ptr(y))
        return y

    def encode16(self, v):
        v = np.ascontiguousarray(v, dtype=np.float32)
        ns = v.size // 6
        q = np.empty(v.shape, dtype=np.int16)
        s = np.empty(v.shape[:-1], dtype=np.float32)
        self.lib.orc_encode16(ns, _ptr(v), _ptr(q), _ptr(s))
        return q, s

    def decode16(self, q, s):
        q = np.ascontiguousarray(q, dtype=np.int16)
        s = np.ascontiguousarray(s, dtype=np.float32)
        v = np.empty(q.shape, dtype=np.float32)
        self.lib.orc_decode16(q.size // 6, _ptr(q), _ptr(s), _ptr(v))
        return v


class Lattice:
    """One lattice of the C++ oracle: extents, mass and a (borrowed, kept alive) gauge field."""

    def __init__(self, orc, dims, U, mass):
        self.orc = orc
        self.dims = tuple(int(d) for d in dims)
        self.V = int(np.prod(self.dims))
        self.Vh = self.V // 2
        self.U = np.ascontiguousarray(U, dtype=np.complex128)
        assert self.U.shape == (self.V, 4, 3, 3)
        d = (ctypes.c_int * 4)(*self.dims)
        self.h = orc.lib.orc_create(d, _ptr(self.U), float(mass))
        if not self.h:
            raise ValueError(f"lattice extents must be positive and even: {dims}")
        self.mass = float(mass)

    def close(self):
        if self.h:
            self.orc.lib.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # interpreter shutdown
            pass

    def _vec(self, v):
        v = np.ascontiguousarray(v, dtype=np.complex128)
        assert v.shape == (self.Vh, 3)
        return v

    def neighbour_tables(self):
        shape = (2, 4, self.Vh)
        fwd, bwd, sf, sb = (np.empty(shape, dtype=np.int64) for _ in range(4))
        self.orc.lib.orc_neighbour_tables(self.h, _ptr(fwd), _ptr(bwd), _ptr(sf), _ptr(sb))
        return fwd, bwd, sf, sb

    def dslash_eo(self, psi, out_parity):
        psi = self._vec(psi)
        out = np.empty_like(psi)
        self.orc.lib.orc_dslash_eo(self.h, _ptr(out), _ptr(psi), int(out_parity))
        return out

    def D_oe(self, psi):
        return self.dslash_eo(psi, 1)

    def D_eo(self, psi):
        return self.dslash_eo(psi, 0)

    def A_apply(self, psi, sigma=0.0):
        psi = self._vec(psi)
        out = np.empty_like(psi)
        self.orc.lib.orc_A_apply(self.h, _ptr(out), _ptr(psi), float(sigma))
        return out

    def cg(self, b, sigma, tol=1e-10, maxiter=20000):
        b = self._vec(b)
        x = np.empty_like(b)
        it = self.orc.lib.orc_cg(self.h, float(sigma), _ptr(b), _ptr(x), float(tol), int(maxiter))
        return x, int(it)

    def multishift_cg(self, b, shifts, tol=1e-10, maxiter=20000, fixed_iters=None):
        """As oracle.solvers.multishift_cg; info also holds 'seconds', 'seconds_dslash', 'dslash_calls'."""
        b = self._vec(b)
        sh = np.ascontiguousarray(shifts, dtype=np.float64)
        X = np.empty((sh.size, self.Vh, 3), dtype=np.complex128)
        info = CgInfo()
        rc = self.orc.lib.orc_mshift_cg(self.h, _ptr(b), sh.size, _ptr(sh), float(tol), int(maxiter),
                                        int(fixed_iters or 0), _ptr(X), ctypes.byref(info))
        if rc != 0:
            raise ValueError("number of shifts must be 1..64")
        return list(X), dict(iterations=info.iterations, shift_iterations=info.shift_iterations, rr=info.rr,
                             zeta=np.array(info.zeta[:sh.size]), seconds=info.seconds,
                             seconds_dslash=info.seconds_dslash, dslash_calls=info.dslash_calls)

    def true_residuals(self, b, xs, shifts):
        b = self._vec(b)
        X = np.ascontiguousarray(np.stack(xs), dtype=np.complex128)
        sh = np.ascontiguousarray(shifts, dtype=np.float64)
        out = np.empty(sh.size)
        self.orc.lib.orc_true_residuals(self.h, _ptr(b), sh.size, _ptr(sh), _ptr(X), _ptr(out))
        return out
