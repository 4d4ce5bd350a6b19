"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on
the same seeded inputs.

Bars: matrix entries within 1e-12 of the largest entry; eigenvalues within
max(1e-10 max|lambda|, 256 u (||H|| + |lambda| ||S||) ||x||^2), the
eigenvalue's own condition number under rounding of the data (tests/_cases.py),
against the oracle's solve of the pencil (H, S) itself (only numerically
singular overlap directions removed); index maps (block_of, boundary block
positions) exact; removed directions (+inf) in the same places.  Each test
prints its measured largest relative error (pytest -s).
"""
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


def _ref(p):
    H, S = dense.build(p)
    return H, S, _cases.reference(p, H, S)


PERIODIC = {
    "chain_m0_4_L6": lambda: _cases.periodic_chain_small(L=6, n0=8, n_perp=24, m0=4, R=16),
    "chain_m0_8_L7_odd": lambda: _cases.periodic_chain_small(L=7, n0=6, n_perp=20, m0=8, R=16),
    "chain_L1": lambda: _cases.periodic_chain_small(L=1, n0=10, n_perp=20, m0=4, R=16),
    "chain_L2": lambda: _cases.periodic_chain_small(L=2, n0=8, n_perp=20, m0=8, seed=3, R=16),
    "single_s_L11_prime": lambda: _cases.single_gaussian(alpha=0.4, n0=6, R=16, L=11, periodic=True),
    "lattice_3d_3x2x4": lambda: _cases.periodic_3d_small(L=(3, 2, 4), n0=5, R=12),
}


@pytest.mark.parametrize("name", sorted(PERIODIC))
def test_periodic_eigenvalues_and_block_map(ctx, name):
    p = PERIODIC[name]()
    if name == "single_s_L11_prime":
        p = li.Problem(L=(11, 1, 1), periodic=(1, 0, 0), N=(66, 18, 18), n0=6, b0=2.0, Z=p.Z,
                       frac=p.frac, exps=p.exps, ang=p.ang, centre=p.centre, R=p.R,
                       sinc_t=p.sinc_t, sinc_c=p.sinc_c)
    H, S, ref = _ref(p)
    out = ctx.solve([p])[0]
    assert out["status"] == 0
    # block_of: each block's eigenvalues are that oracle block's spectrum
    _cases.report(name, _cases.check(ref, out["evals"], out["block_of"]))


@pytest.mark.parametrize("name", ["chain_m0_4_L6", "chain_m0_8_L7_odd", "lattice_3d_3x2x4"])
def test_periodic_generators(ctx, name):
    p = PERIODIC[name]()
    H, S = dense.build(p)
    b = ctx.assemble(p)
    gh, gs, _, _, _ = b.generators()
    rh = blocks.generators_from_dense(p, H)
    rs = blocks.generators_from_dense(p, S)
    assert np.max(np.abs(gh - rh)) <= ENTRY_TOL * np.max(np.abs(H))
    assert np.max(np.abs(gs - rs)) <= ENTRY_TOL * np.max(np.abs(S))
    ev, blk = b.circulant_eig()
    _cases.check(_cases.reference(p, H, S), ev, blk)
    b.close()


BOX = {
    "box_L12": lambda: _cases.box_chain_small(L=12, n0=5, pad=6, n_perp=20, R=16, k=6),
    "box_L24_seed2": lambda: _cases.box_chain_small(L=24, n0=5, pad=10, n_perp=18, seed=2, R=16, k=8),
    "box_L5_short": lambda: _cases.box_chain_small(L=5, n0=6, pad=4, n_perp=16, seed=4, R=12, k=4),
}


def _dense_from_blocks(p, T, E, rc):
    m0, L = p.m0, p.L[0]
    D = (T.shape[0] - 1) // 2
    M = np.zeros((L * m0, L * m0))
    for k in range(L):
        for m in range(L):
            d = k - m
            if abs(d) <= D:
                M[k * m0:(k + 1) * m0, m * m0:(m + 1) * m0] = T[d + D]
    for e, (k, m) in enumerate(rc):
        M[k * m0:(k + 1) * m0, m * m0:(m + 1) * m0] += E[e]
    return M


@pytest.mark.parametrize("name", sorted(BOX))
def test_box_toeplitz_plus_boundary_equals_dense(ctx, name):
    p = BOX[name]()
    H, S = dense.build(p)
    b = ctx.assemble(p)
    TH, TS, EH, ES, rc = b.generators()
    assert np.max(np.abs(_dense_from_blocks(p, TH, EH, rc) - H)) <= ENTRY_TOL * np.max(np.abs(H))
    assert np.max(np.abs(_dense_from_blocks(p, TS, ES, rc) - S)) <= ENTRY_TOL * np.max(np.abs(S))
    b.close()


@pytest.mark.parametrize("name", sorted(BOX))
def test_box_embedded_fft_matvec(ctx, name):
    from paper_1702_00339_gb300 import fock
    p = BOX[name]()
    H, S = dense.build(p)
    b = ctx.assemble(p)
    x = np.random.default_rng(7).standard_normal((p.Nb, 5))
    for which, M in ((fock.FOCK_OP_H, H), (fock.FOCK_OP_S, S)):
        y = b.matvec(x, which)
        ref = M @ x
        assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(M)) * np.max(np.abs(x)) * p.m0 * 4
    b.close()


@pytest.mark.parametrize("name", sorted(BOX))
def test_box_lowest_eigenpairs(ctx, name):
    p = BOX[name]()
    H, S, ref = _ref(p)
    b = ctx.assemble(p)
    ev, V, iters, rc = b.box_eig(p.k_eig, tol=1e-10, maxit=500, vectors=True)
    assert rc == 0, f"no convergence in {iters} iterations"
    _cases.report(name, _cases.check(ref, ev))
    # residual on the kept space (every direction unless a cell direction is
    # numerically singular), S-orthonormality in the original basis
    s, Q, tau = blocks.cell_null_directions(p)
    Xb = np.kron(np.eye(p.L[0]), Q[:, s > tau])
    R = Xb.T @ (H @ V - (S @ V) * ev)
    assert np.max(np.linalg.norm(R, axis=0) / (np.abs(ev) * np.linalg.norm(Xb.T @ (S @ V), axis=0))) < 1e-9
    G = V.T @ S @ V
    assert np.max(np.abs(G - np.eye(p.k_eig))) < 1e-8
    b.close()


def test_batched_solve_equals_alone(ctx):
    """Batch invariance: a problem's result does not depend on what else is
    in the batch (fixed per-problem reduction orders)."""
    ps = [PERIODIC["chain_m0_4_L6"](), BOX["box_L12"](), PERIODIC["lattice_3d_3x2x4"](),
          BOX["box_L5_short"]()]
    together = ctx.solve(ps)
    for p, t in zip(ps, together):
        alone = ctx.solve([p])[0]
        assert np.array_equal(alone["evals"], t["evals"])


def test_full_size_config1(ctx):
    p = _cases.with_table(li.config1())
    H, S, ref = _ref(p)
    out = ctx.solve([p])[0]
    _cases.report("config1", _cases.check(ref, out["evals"], out["block_of"]))


def test_full_size_config2_box(ctx):
    p = _cases.with_table(li.config2(0))
    H, S, ref = _ref(p)
    out = ctx.solve([p])[0]
    assert out["status"] == 0
    _cases.report("config2_box", _cases.check(ref, out["evals"]))


def test_fourier_index_ranges_merge_to_the_full_solve(ctx):
    """Ranks that each solve a contiguous Fourier-index range and merge their
    sorted parts obtain the single-call spectrum bit for bit."""
    from paper_1702_00339_gb300 import shard
    p = PERIODIC["lattice_3d_3x2x4"]()
    b = ctx.assemble(p)
    ev, blk = b.circulant_eig()
    for world in (2, 3, 5):
        parts = [b.circulant_eig_range(*shard.j_range(p.ncell, r, world)) for r in range(world)]
        mev, mblk = shard.merge(parts)
        assert np.array_equal(mev, ev) and np.array_equal(mblk, blk)
    b.close()
