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


def test_problem_check_accepts_the_workloads(libpath):
    """The library's own host check (the one every solve runs first) accepts
    every workload recipe and agrees with the binding on the solve kind and
    the number of eigenvalues returned."""
    from paper_1702_00339_gb300 import fock
    ps = [li.config1(), li.config2(0), li.config3(0), li.config5_box(0), li.config5_periodic(0)]
    ps += li.serving_stream(128, seed=3000)
    for p in ps:
        r = fock.check_problem(p)
        assert r["kind"] == int(fock._structured(p))
        assert r["n_evals"] == fock.n_evals(p)


def _bad_problems():
    """(mutation, expected reason fragment) pairs on a small box chain."""
    import dataclasses
    base = li.config2(0, L=8, n0=5, pad=4, n_perp=16, R=16)
    base.k_eig = 4
    r = dataclasses.replace
    per = r(base, periodic=(1, 0, 0), N=(8 * 5, 16, 16), k_eig=0)
    yield r(base, n0=0), "n0 > 0"
    yield r(base, b0=0.0), "b0 > 0"
    yield r(base, Z=np.zeros(0), frac=np.zeros((0, 3))), "M0"
    yield r(base, exps=np.ones(33), ang=np.zeros(33, int), centre=np.zeros(33, int)), "m0"
    yield r(base, R=2), "R <= 64"
    yield r(base, R=65), "R <= 64"
    yield r(base, precision=3), "precision"
    yield r(base, L=(0, 1, 1)), "L >= 1"
    yield r(per, N=(41, 16, 16)), "N = L*n0"
    yield r(base, N=(39, 16, 16)), "N >= L*n0"
    yield r(base, L=(2, 2, 1), N=(14, 14, 16)), "chains"
    yield r(base, L=(1, 1, 1), N=(9, 16, 16), defects=[li.Defect((0, 0, 0), 0, 0.0)]), "chains"
    yield r(per, periodic=(1, 1, 0), N=(40, 5, 16), defects=[li.Defect((1, 0, 0), 0, 0.0)]), "transverse"
    yield r(base, defects=[li.Defect((8, 0, 0), 0, 0.0)]), "defect cell"
    yield r(base, defects=[li.Defect((1, 0, 0), 1, 0.0)]), "defect cell"
    yield r(base, defects=[li.Defect((1, 0, 0), 0, float("nan"))]), "newZ"
    e = base.exps.copy()
    e[3] = -1.0
    yield r(base, exps=e), "exponents"
    a = base.ang.copy()
    a[0] = 4
    yield r(base, ang=a), "ang"
    c = base.centre.copy()
    c[0] = 1
    yield r(base, centre=c), "centre"
    t, cq, _ = sinc.table_for(base)
    t = t.copy()
    t[0] = 0.0
    yield base.with_table(t, cq), "sinc_t"
    yield r(base, k_eig=65), "k_eig"
    long = li.config2(0, L=64, n0=5, pad=4, n_perp=16, R=16)
    yield r(long, k_eig=80), "k_eig"


@pytest.mark.parametrize("case", list(range(22)))
def test_problem_check_rejects_malformed_problems(libpath, case):
    """Every malformed field is refused with FOCK_EINVAL and a reason, by the
    host check alone (no device)."""
    from paper_1702_00339_gb300 import fock
    bad = list(_bad_problems())
    assert len(bad) == 22
    p, frag = bad[case]
    with pytest.raises(fock.FockError) as ei:
        fock.check_problem(p)
    assert ei.value.code == fock.FOCK_EINVAL
    assert frag in str(ei.value)


def test_problem_check_truncates_the_reason(libpath):
    import ctypes as C
    import dataclasses
    from paper_1702_00339_gb300 import fock
    p = dataclasses.replace(li.config2(0), n0=0)
    m = fock._Marshal(p)
    why = C.create_string_buffer(b"x" * 8, 8)
    rc = fock.lib().fock_problem_check(C.byref(m.s), None, None, why, 5)
    assert rc == fock.FOCK_EINVAL
    assert why.raw[:5] == b"n0 > "[:4] + b"\0"
    assert fock.lib().fock_problem_check(None, None, None, None, 0) == fock.FOCK_EINVAL
