"""Known limitation, tracked: three periodic chains with defects of the
serving mix (requests 298, 377 and 478 of the seeded stream) ended
unconverged (FOCK_ENOCONV) when solved inside serving batches.  Each is
solved here alone; the outcome is recorded as an expected failure until the
cause is fixed (a pass shows up as XPASS).  Request 478's two
substitutions keep Z = 1, so its operator is exactly the periodic chain's:
when it converges, its 16 lowest eigenvalues are checked against the
oracle's Fourier-block spectrum of that chain."""
import dataclasses

import numpy as np
import pytest

import lattice_inputs as li
from oracle import blocks, dense
from tests import _cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1702_00339_gb300 import build, fock
    build.build()
    c = fock.Context(0)
    yield c
    c.close()


@pytest.mark.xfail(reason="unconverged in the serving run; cause under investigation", strict=False)
@pytest.mark.parametrize("rid", [478, 377, 298])
def test_unconverged_serving_chain_alone(ctx, rid):
    p = li.serving_stream(rid + 1, seed=3000)[rid]
    out = ctx.solve([p], check=False)[0]
    assert out["status"] == 0, (f"request {rid}: status {out['status']} after {out['iters']} "
                                f"iterations, residual {out['resid']:.3e}")
    if rid == 478:
        assert all(d.newZ == p.Z[d.nucleus] for d in p.defects)
        q = _cases.with_table(dataclasses.replace(p, defects=[]))
        H, S = dense.build(q)
        ev, _, kap = blocks.periodic_eigs(q, H, S)
        ref = ev[:p.k_eig]
        tol = max(1e-10, 16 * _cases.U64 * float(np.max(kap))) * float(np.max(np.abs(ref)))
        assert np.max(np.abs(out["evals"] - ref)) <= tol
