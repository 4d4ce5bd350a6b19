"""GPU parity for chains with vacancy / substitution defects (reading R-DEF):
the structured operator the library builds (Toeplitz generators plus wall,
wrap-around and defect blocks) reproduces the oracle's dense H and S with
the defect kernels, and the lowest eigenvalues match the oracle's
cell-reduced dense solve."""
import dataclasses

import numpy as np
import pytest

import lattice_inputs as li
from oracle import blocks, dense
from tests import _cases

pytestmark = pytest.mark.gpu

ENTRY_TOL = 1e-12


@pytest.fixture(scope="module")
def ctx():
    from paper_1702_00339_gb300 import build, fock
    build.build()
    c = fock.Context(0)
    yield c
    c.close()


def _with(p, defs, k):
    q = dataclasses.replace(p, defects=[li.Defect(cell=(c, 0, 0), nucleus=0, newZ=z) for c, z in defs])
    q.k_eig = k
    return q


CASES = {
    "box_L10_two_defects": lambda: _with(_cases.box_chain_small(L=10, n0=5, pad=5, n_perp=14, R=12, k=4),
                                         [(2, 0.0), (7, 2.0)], 4),
    "periodic_short_L6_vacancy": lambda: _with(_cases.periodic_chain_small(L=6, n0=6, n_perp=14, m0=4, R=12),
                                               [(1, 0.0)], 4),
    "periodic_long_L30_subst": lambda: _with(_cases.periodic_chain_small(L=30, n0=4, n_perp=12, m0=4, R=10),
                                             [(3, 3.0), (17, 0.0), (18, 2.0)], 6),
    "periodic_m0_8_L9": lambda: _with(_cases.periodic_chain_small(L=9, n0=5, n_perp=12, m0=8, seed=1, R=10),
                                      [(4, 0.5)], 5),
}


def _dense_from_blocks(p, T, E, rc):
    m0, L = p.m0, p.L[0]
    D = (T.shape[0] - 1) // 2
    M = np.zeros((L * m0, L * m0))
    for k in range(L):
        for m in range(L):
            if abs(k - m) <= D:
                M[k * m0:(k + 1) * m0, m * m0:(m + 1) * m0] = T[k - m + D]
    for e, (k, m) in enumerate(rc):
        M[k * m0:(k + 1) * m0, m * m0:(m + 1) * m0] += E[e]
    return M


@pytest.mark.parametrize("name", sorted(CASES))
def test_structured_operator_equals_dense_with_defects(ctx, name):
    p = CASES[name]()
    H, S = dense.build(p)
    b = ctx.assemble(p)
    TH, TS, EH, ES, rc = b.generators()
    b.close()
    assert np.max(np.abs(_dense_from_blocks(p, TH, EH, rc) - H)) <= ENTRY_TOL * np.max(np.abs(H))
    assert np.max(np.abs(_dense_from_blocks(p, TS, ES, rc) - S)) <= ENTRY_TOL * np.max(np.abs(S))


@pytest.mark.parametrize("name", sorted(CASES))
def test_lowest_eigenvalues_with_defects(ctx, name):
    p = CASES[name]()
    H, S = dense.build(p)
    ref = _cases.reference(p, H, S)
    out = ctx.solve([p])[0]
    assert out["status"] == 0
    _cases.report(name, _cases.check(ref, out["evals"]))


def test_defect_problems_batch_invariant(ctx):
    ps = [CASES[n]() for n in sorted(CASES)] + [_cases.box_chain_small(L=12, n0=5, pad=6, n_perp=20, R=16, k=6)]
    together = ctx.solve(ps)
    for p, t in zip(ps, together):
        assert np.array_equal(ctx.solve([p])[0]["evals"], t["evals"])


@pytest.mark.parametrize("name", sorted(CASES))
def test_structured_matvec_with_defects(ctx, name):
    """y = H x and S x through the embedded FFT plus the E blocks, against the
    dense oracle matrices (odd and even column counts)."""
    from paper_1702_00339_gb300 import fock
    p = CASES[name]()
    H, S = dense.build(p)
    b = ctx.assemble(p)
    for nvec in (1, 4, 7):
        x = np.random.default_rng(nvec).standard_normal((p.Nb, nvec))
        for which, M in ((fock.FOCK_OP_H, H), (fock.FOCK_OP_S, S)):
            y = b.matvec(x, which)
            assert np.max(np.abs(y - M @ x)) <= 1e-12 * np.max(np.abs(M)) * np.max(np.abs(x)) * p.m0 * 4
    b.close()


def test_whole_space_defect_chains_of_the_serving_mix(ctx):
    """Periodic defect chains small enough for the whole-space block (3 N_b
    <= 255): the start's Rayleigh-Ritz step over all directions is exact, and
    the solve ends there (iterating on such a block once broke these two
    requests of the serving mix down).  Against the oracle's dense solve."""
    ps = [li.serving_stream(128, seed=3100)[102], li.serving_stream(512, seed=3000)[262]]
    for p in ps:
        assert 3 * p.Nb <= 255 and p.defects
        q = _cases.with_table(p)
        q.k_eig = p.k_eig
        H, S = dense.build(q)
        ref = _cases.reference(q, H, S)
        out = ctx.solve([p])[0]
        assert out["status"] == 0 and out["iters"] == 0
        _cases.check(ref, out["evals"])
