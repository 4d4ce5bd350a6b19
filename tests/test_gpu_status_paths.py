"""GPU checks of the solver's reported states: an iteration cap reached
before convergence returns FOCK_ENOCONV with its best estimates, and those
estimates are Rayleigh-Ritz values, so each lies above the eigenvalue it
approximates (Courant-Fischer); the context stays usable afterwards."""
import numpy as np
import pytest

from oracle import dense
from tests import _cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1702_00339_gb300 import build, fock
    build.build()
    c = fock.Context(0)
    yield c
    c.close()


def test_iteration_cap_reports_no_convergence_with_upper_estimates(ctx):
    from paper_1702_00339_gb300 import fock
    p = _cases.box_chain_small(L=12, n0=5, pad=6, n_perp=20, R=16, k=6)
    H, S = dense.build(p)
    ref = _cases.reference(p, H, S)
    b = ctx.assemble(p)
    ev, _, iters, rc = b.box_eig(p.k_eig, tol=1e-10, maxit=2)
    b.close()
    assert rc == fock.FOCK_ENOCONV and iters == 2
    assert np.all(np.isfinite(ev)) and np.all(np.diff(ev) >= 0)
    assert np.all(ev >= ref.ev - ref.cands[0][1])
    # the same problem then converges through the batched path
    out = ctx.solve([p])[0]
    assert out["status"] == 0
    _cases.check(ref, out["evals"])
