"""The box potential read as the plain lattice sum over the box's cells
(reading R2, Sec. 2.3 case (B): each nucleus once with its full charge),
box_potential = 1: the library adds the difference to the replicated
central-cell potential (reading R1) as blocks on every pair of cells whose
functions meet.  Against the oracle's dense matrices with the R2 potential
(grid.potential_slabs(p, "lattice_sum"), pinned by brute force and the
Boys-function attraction): the operator entries within 1e-12, the lowest
eigenvalues within the bar of tests/_cases.py, alone and with defects."""
import dataclasses

import numpy as np
import pytest

import lattice_inputs as li
from oracle import dense
from tests import _cases
from tests.test_gpu_parity import _dense_from_blocks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1702_00339_gb300 import build, fock
    build.build()
    c = fock.Context(0)
    yield c
    c.close()


def _r2(p):
    q = dataclasses.replace(p, box_potential=1)
    q.k_eig = p.k_eig
    return q


CASES = {
    "box_L12": lambda: _r2(_cases.box_chain_small(L=12, n0=5, pad=6, n_perp=20, R=16, k=6)),
    "box_L9_m0_8_seed3": lambda: _r2(_cases.box_chain_small(L=9, n0=4, pad=5, n_perp=16, seed=3, R=12, k=5)),
    "box_L10_defects": lambda: _r2(dataclasses.replace(
        _cases.box_chain_small(L=10, n0=4, pad=4, n_perp=14, seed=1, R=12, k=5),
        defects=[li.Defect((2, 0, 0), 0, 0.0), li.Defect((7, 0, 0), 0, 2.0)])),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_lattice_sum_box_operator_and_spectrum(ctx, name):
    p = CASES[name]()
    if name == "box_L10_defects":
        p.k_eig = 5
    H, S = dense.build(p)                      # the R2 potential (the problem's field)
    H1, _ = dense.build(p, box_potential="replicated")
    assert np.max(np.abs(H - H1)) > 1e-6 * np.max(np.abs(H))   # the readings differ
    b = ctx.assemble(p)
    TH, TS, EH, ES, rc = b.generators()
    assert np.max(np.abs(_dense_from_blocks(p, TH, EH, rc) - H)) <= 1e-12 * np.max(np.abs(H))
    assert np.max(np.abs(_dense_from_blocks(p, TS, ES, rc) - S)) <= 1e-12 * np.max(np.abs(S))
    b.close()
    out = ctx.solve([p])[0]
    assert out["status"] == 0
    _cases.report(name + "_R2", _cases.check(_cases.reference(p, H, S), out["evals"]))
