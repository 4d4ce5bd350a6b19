"""Mixed forms.  FOCK_MIXED: the assembly's quadrature contractions and the
block iteration's Gram and basis products as exact split products on the
tensor cores.  FOCK_MIXED_F32: in addition, FP32 preconditioner solves and
FP32 embedded-FFT matvecs until a problem's residual falls below 1e-5, FP64
afterwards.  The stated bar: eigenvalues within 1e-8 relative of the oracle
(and of the FP64 form); problems in FP64 form are unaffected by mixed
problems in their batch (bitwise)."""
import dataclasses

import numpy as np
import pytest

import lattice_inputs as li
from oracle import dense
from tests import _cases
from tests.test_gpu_defects import CASES as DEFECT_CASES

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-8


@pytest.fixture(scope="module")
def ctx():
    from paper_1702_00339_gb300 import build, fock
    build.build()
    c = fock.Context(0)
    yield c
    c.close()


def _mixed(p, precision=1):
    q = dataclasses.replace(p, precision=precision)
    q.k_eig = p.k_eig
    return q


CASES = {
    "box_L12": lambda: _cases.box_chain_small(L=12, n0=5, pad=6, n_perp=20, R=16, k=6),
    "box_L40": lambda: _cases.box_chain_small(L=40, n0=4, pad=6, n_perp=14, seed=3, R=12, k=8),
    "box_defects": DEFECT_CASES["box_L10_two_defects"],
    "periodic_defects": DEFECT_CASES["periodic_long_L30_subst"],
}


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("name", sorted(CASES))
def test_mixed_within_stated_bar(ctx, name, precision):
    p = CASES[name]()
    H, S = dense.build(p)
    ref = _cases.reference(p, H, S, base=MIXED_TOL)
    mixed = ctx.solve([_mixed(p, precision)])[0]
    fp64 = ctx.solve([p])[0]
    assert mixed["status"] == 0
    _cases.report(f"{name}_mixed{precision}", _cases.check(ref, mixed["evals"]))
    assert np.max(np.abs(mixed["evals"] - fp64["evals"])) <= MIXED_TOL * ref.scale


def test_fp64_problems_unaffected_by_mixed_batch_mates(ctx):
    ps = [CASES[n]() for n in sorted(CASES)]
    batch = ps + [_mixed(p) for p in ps] + [_mixed(p, 2) for p in ps]
    together = ctx.solve(batch)
    for p, t in zip(ps, together[:len(ps)]):
        assert np.array_equal(ctx.solve([p])[0]["evals"], t["evals"])
