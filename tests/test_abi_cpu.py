"""Host-side checks of the C ABI (no GPU needed): the library builds, loads
and exports every entry point declared in include/fock.h; the host-only
entry points agree with the oracle's reading of the quadrature rule."""
import os
import re
import subprocess

import numpy as np
import pytest

import lattice_inputs as li
from oracle import sinc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1702_00339_gb300 import build
    return build.build()


def _declared():
    src = open(os.path.join(ROOT, "include", "fock.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fock_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (fock_[a-z_]+)", out))
    declared = _declared()
    assert declared, "no declarations parsed"
    missing = [s for s in declared if s not in exported]
    assert not missing, missing


def test_binding_loads(libpath):
    from paper_1702_00339_gb300 import fock
    L = fock.lib()
    for s in _declared():
        assert hasattr(L, s)


@pytest.mark.parametrize("R,zmin,zmax", [(24, 1e-3, 1e2), (32, 1.3e-3, 420.0), (40, 6e-4, 1100.0)])
def test_default_rule_matches_oracle_reading(libpath, R, zmin, zmax):
    from paper_1702_00339_gb300 import fock
    t, c, e = fock.sinc_table(R, zmin, zmax)
    to, co, eo = sinc.sinc_table(R, zmin, zmax)
    assert np.allclose(t, to, rtol=1e-13, atol=0) and np.allclose(c, co, rtol=1e-13, atol=0)
    assert abs(e - eo) <= 1e-12


def test_default_range_matches(libpath):
    from paper_1702_00339_gb300 import fock
    for p in (li.config1(), li.config2(0), li.config3(0)):
        a, b = fock.default_range(p)
        ao, bo = sinc.default_range(p)
        assert a == pytest.approx(ao, rel=1e-15) and b == pytest.approx(bo, rel=1e-15)


def test_sinc_table_rejects_bad_arguments(libpath):
    from paper_1702_00339_gb300 import fock
    with pytest.raises(fock.FockError):
        fock.sinc_table(2, 1e-3, 1.0)
    with pytest.raises(fock.FockError):
        fock.sinc_table(16, 1.0, 0.5)


def test_serve_start_without_a_device_fails_cleanly(libpath):
    """Host-only: with no usable CUDA device the server refuses to start
    (FOCK_ECUDA) instead of crashing."""
    import ctypes as C
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1702_00339_gb300 import fock
    h = C.c_void_p()
    rc = fock.lib().fock_serve_start(0, None, C.byref(h))
    assert rc == fock.FOCK_ECUDA and not h.value


def _read(addr, n, ctype):
    import ctypes as C
    if not addr:
        return None
    return np.ctypeslib.as_array(C.cast(C.c_void_p(addr), C.POINTER(ctype)), shape=(n,)).copy()


def test_problem_marshalling_round_trip():
    """The struct handed to the C ABI carries every parameter of the problem
    (the double and int parameters live in two packed arrays): read back
    through the struct's addresses, they equal the problem's own arrays."""
    import ctypes as C
    from paper_1702_00339_gb300 import fock
    ps = [li.config2(s) for s in range(3)] + li.serving_stream(16, seed=3000)
    t, c, _ = sinc.table_for(ps[0])
    ps.append(ps[0].with_table(t, c))
    for p in ps:
        m = fock._Marshal(p)
        s = m.s
        assert list(s.L) == list(p.L) and list(s.periodic) == list(p.periodic) and list(s.N) == list(p.N)
        assert s.M0 == len(p.Z) and s.m0 == len(p.exps) and s.R == p.R and s.k_eig == p.k_eig
        assert np.array_equal(_read(s.Z, s.M0, C.c_double), np.asarray(p.Z, float))
        assert np.array_equal(_read(s.frac, 3 * s.M0, C.c_double), np.asarray(p.frac, float).ravel())
        assert np.array_equal(_read(s.exps, s.m0, C.c_double), np.asarray(p.exps, float))
        assert np.array_equal(_read(s.ang, s.m0, C.c_int), np.asarray(p.ang, np.int32))
        assert np.array_equal(_read(s.centre, s.m0, C.c_int), np.asarray(p.centre, np.int32))
        if p.sinc_t is None:
            assert not s.sinc_t and not s.sinc_c
        else:
            assert np.array_equal(_read(s.sinc_t, p.R, C.c_double), np.asarray(p.sinc_t, float))
            assert np.array_equal(_read(s.sinc_c, p.R, C.c_double), np.asarray(p.sinc_c, float))
        assert s.ndef == len(p.defects)
        if p.defects:
            d = C.cast(C.c_void_p(s.defects), C.POINTER(fock.c_defect))
            for i, x in enumerate(p.defects):
                assert list(d[i].cell) == list(x.cell) and d[i].nucleus == x.nucleus and d[i].newZ == x.newZ
