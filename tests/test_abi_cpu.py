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
