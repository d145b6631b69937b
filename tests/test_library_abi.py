"""CPU checks of the C ABI: the library builds, loads, exports every symbol of include/lqcd.h,
rejects bad arguments without touching the GPU, and its host-side rational coefficients
(Eq. ratapprx, Appendix) agree with the oracle's Zolotarev solution."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1710_09178_gb300 import build as b

    b.build()
    import paper_1710_09178_gb300 as pkg

    return pkg.load_library()


def header_functions():
    src = open(os.path.join(ROOT, "include", "lqcd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    decl = r"^(?:int|size_t|long long|const char\s*\*)\s*\**\s*([a-z_][A-Za-z0-9_]*)\s*\("
    return sorted(set(re.findall(decl, src, flags=re.M)))


def test_header_symbols_exported(lib):
    import paper_1710_09178_gb300 as pkg

    names = header_functions()
    assert "dslash_eo" in names and "mshift_cg" in names and len(names) >= 14
    for nm in names:
        assert hasattr(lib, nm), nm
    assert sorted(names) == sorted(pkg.EXPORTED)


def test_create_rejects_bad_dims(lib):
    h = ctypes.c_void_p()
    # odd, zero and negative extents; half volumes one step above the 2^27 limit of 32-bit site indices
    for dims, code in [((4, 4, 4, 3), 2), ((0, 4, 4, 4), 2), ((4, 4, -2, 4), 2), ((512, 512, 512, 4), 2),
                       ((256, 256, 256, 18), 2)]:
        arr = (ctypes.c_int * 4)(*dims)
        assert lib.lqcd_create(ctypes.byref(h), arr, 0.1, None) == code
        assert not h.value
    assert lib.lqcd_create(None, (ctypes.c_int * 4)(4, 4, 4, 4), 0.1, None) == 1


def test_calls_without_gauge_or_with_bad_args_fail_cleanly(lib):
    h = ctypes.c_void_p()
    assert lib.lqcd_create(ctypes.byref(h), (ctypes.c_int * 4)(4, 4, 4, 4), 0.1, None) == 0
    try:
        buf = ctypes.create_string_buffer(64)
        # bad parity and unknown precision are argument errors; a valid call without a gauge field is a state error
        assert lib.dslash_eo(h, buf, ctypes.byref(ctypes.c_int(0)), 2, 1) == 1
        assert lib.dslash_eo(h, buf, ctypes.byref(ctypes.c_int(0)), 0, 7) == 1
        assert lib.dslash_eo(h, buf, ctypes.byref(ctypes.c_int(0)), 0, 1) == 6
        assert b"gauge" in lib.lqcd_last_error(h)
        sh = (ctypes.c_double * 2)(0.1, 0.2)
        assert lib.mshift_cg(h, sh, None, 0, 0.0, buf, None, None, 1e-10, 100, 1, None) == 1  # n = 0
        assert lib.mshift_cg(h, sh, None, 2, 0.0, buf, None, None, 0.0, 100, 1, None) == 1  # tol = 0
        bad = (ctypes.c_double * 2)(0.1, -1.0)
        assert lib.mshift_cg(h, bad, None, 2, 0.0, buf, None, None, 1e-10, 100, 1, None) == 1
        assert lib.mshift_cg(h, sh, None, 2, 0.0, buf, None, None, 1e-10, 100, 1, None) == 6  # no gauge
        assert lib.lqcd_set_option(h, 99, 1.0) == 1
        assert lib.lqcd_set_option(h, 5, 3.0) == 1
        assert lib.lqcd_vector_bytes(h, 0) == 48 * 128 and lib.lqcd_vector_bytes(h, 3) == 16 * 128
        assert lib.lqcd_vector_bytes(h, 9) == 0
    finally:
        assert lib.lqcd_destroy(h) == 0


@pytest.mark.parametrize("n,mass", [(12, 0.1), (14, 0.05), (16, 0.02)])
def test_rational_coeffs_match_oracle_zolotarev(lib, n, mass):
    from oracle import rational
    from paper_1710_09178_gb300 import rational_coeffs

    lo, hi = 4 * mass ** 2, 16 + 4 * mass ** 2
    c0, res, poles, err = rational_coeffs(-0.5, lo, hi, n)
    oc0, ores, opoles, oerr = rational.zolotarev_inv_sqrt(n, lo, hi)
    order = np.argsort(poles)
    oorder = np.argsort(opoles)
    assert np.allclose(poles[order], opoles[oorder], rtol=1e-9, atol=0)
    assert np.allclose(res[order], ores[oorder], rtol=1e-8, atol=0)
    assert abs(c0 - oc0) < 1e-9 * oc0
    assert abs(err - oerr) < 1e-2 * oerr
    # the library's coefficients are themselves minimax: the oracle's alternation scan confirms it
    assert rational.max_relative_error(c0, res, poles, -0.5, lo, hi) < 1.02 * oerr


def test_rational_coeffs_rejects_bad_interval(lib):
    from paper_1710_09178_gb300 import LqcdError, rational_coeffs

    for args in [(-0.5, 0.0, 1.0, 4), (-0.5, 2.0, 1.0, 4), (-0.5, 0.1, 1.0, 0), (-0.5, 0.1, 1.0, 40)]:
        with pytest.raises(LqcdError):
            rational_coeffs(*args)


@pytest.mark.parametrize("power,n,mass", [(0.25, 12, 0.1), (0.25, 16, 0.02), (-0.25, 14, 0.05)])
def test_rational_coeffs_remez_match_oracle(lib, power, n, mass):
    from oracle import rational
    from paper_1710_09178_gb300 import rational_coeffs

    lo, hi = 4 * mass ** 2, 16 + 4 * mass ** 2
    c0, res, poles, err = rational_coeffs(power, lo, hi, n)
    oc0, ores, opoles, oerr = rational.remez_power(power, lo, hi, n)
    assert np.allclose(np.sort(poles), np.sort(opoles), rtol=1e-4, atol=0)
    assert abs(c0 - oc0) < 1e-4 * abs(oc0)  # both level the error only to its ~1e-3 rounding noise
    # the library's result satisfies the alternation theorem under the oracle's own scan
    ext = rational.error_extrema(lambda x: rational.relative_error(c0, res, poles, power, x), lo, hi, floor=0.1)
    vals = np.array([v for _, v in ext])
    assert vals.size == 2 * n + 2 and np.all(np.sign(vals[1:]) == -np.sign(vals[:-1]))
    assert np.max(np.abs(vals)) <= 1.05 * oerr


def test_rational_coeffs_appendix_case(lib):
    # Appendix: 24/24 approximation of x^{1/4} on [5e-5, 34] with error below 1e-12
    from oracle import rational
    from paper_1710_09178_gb300 import rational_coeffs

    c0, res, poles, err = rational_coeffs(0.25, 5e-5, 34.0, 24)
    assert rational.max_relative_error(c0, res, poles, 0.25, 5e-5, 34.0) < 1e-12


def test_binding_constants_mirror_the_header():
    # every status code, precision mode, option key and limit of include/lqcd.h has the same value
    # in the Python binding (LQCD_X -> X, or LQCD_X for the status codes)
    import paper_1710_09178_gb300 as pkg

    src = open(os.path.join(ROOT, "include", "lqcd.h")).read()
    defs = dict(re.findall(r"^#define\s+(LQCD_[A-Z0-9_]+)\s+(-?\d+)\b", src, flags=re.M))
    assert len(defs) >= 20
    for name, value in defs.items():
        short = name[len("LQCD_"):]
        py = getattr(pkg, name, getattr(pkg, short, None))
        assert py is not None, name
        assert py == int(value), (name, py, value)
