"""Periodic eigenvectors (Prop. A.1): the Fourier-block eigenvectors of
fock_circulant_eig and the lattice eigenvectors of fock_bloch_vectors (the
inverse DFT over the lattice index, U = (F^* (x) I) Ubar, on the device),
against the oracle's dense matrices: residuals H u - lambda S u, S-
orthonormality, and the oracle's own back-transformed eigenvectors
(blocks.periodic_eigvecs) spanning the same eigenspaces."""
import numpy as np
import pytest

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


CASES = {
    "chain_m0_8_L7": lambda: _cases.periodic_chain_small(L=7, n0=6, n_perp=20, m0=8, R=16),
    "lattice_3d_3x2x4": lambda: _cases.periodic_3d_small(L=(3, 2, 4), n0=5, R=12),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_block_eigenvectors_solve_the_block_pencils(ctx, name):
    p = CASES[name]()
    H, S = dense.build(p)
    Hb, Sb = blocks.periodic_fourier_blocks(p, H, S)
    b = ctx.assemble(p)
    ev, blk, Y = b.circulant_eig(vectors=True)
    ev0, blk0 = b.circulant_eig()
    b.close()
    assert np.array_equal(ev, ev0) and np.array_equal(blk, blk0)   # the same eigenvalues either way
    scale = np.max(np.abs(ev[np.isfinite(ev)]))
    for j in range(p.ncell):
        lam = np.sort(ev[blk == j])
        r = int(np.isfinite(lam).sum())
        y = Y[j].T[:, :r]                                   # columns = eigenvectors
        G = y.conj().T @ Sb[j] @ y
        w = np.linalg.eigvalsh(Sb[j])
        kappa = w.max() / w[w > 0][-r:].min()                # of the kept part of the block overlap
        assert np.max(np.abs(G - np.eye(r))) < 1e-12 + 16 * _cases.U64 * kappa
        R = Hb[j] @ y - (Sb[j] @ y) * lam[:r]
        assert np.max(np.linalg.norm(R, axis=0)) < 1e-9 * scale * np.max(np.linalg.norm(Hb[j], 2))
        assert np.all(Y[j][r:] == 0)


@pytest.mark.parametrize("name", sorted(CASES))
def test_lattice_eigenvectors_against_the_oracle(ctx, name):
    p = CASES[name]()
    H, S = dense.build(p)
    b = ctx.assemble(p)
    ev, blk = b.circulant_eig()
    sel = [0, 1, 5, p.Nb // 3]
    jb = [int(blk[s]) for s in sel]
    rank = [int(np.sum(blk[:s] == blk[s])) for s in sel]
    U = b.bloch_vectors(jb, rank)
    b.close()
    lam = ev[sel]
    w = np.linalg.eigvalsh(S)
    kappa = w.max() / w[w > blocks.null_threshold(p)].min()
    assert np.max(np.abs(U.conj().T @ S @ U - np.eye(len(sel)))) < 1e-12 + 16 * _cases.U64 * kappa
    R = H @ U - (S @ U) * lam
    assert np.max(np.linalg.norm(R, axis=0)) < 1e-8 * np.max(np.abs(lam)) * np.linalg.norm(H, 2)
    # each vector lies in the oracle's eigenspace of its eigenvalue
    evo, Uo, jo = blocks.periodic_eigvecs(p, H, S)
    for c, s in enumerate(sel):
        near = np.abs(evo - lam[c]) <= 1e-8 * np.max(np.abs(evo))
        Q = Uo[:, near]
        proj = Q @ np.linalg.solve(Q.conj().T @ S @ Q, Q.conj().T @ S @ U[:, c])
        assert np.linalg.norm(U[:, c] - proj) < 1e-6 * np.linalg.norm(U[:, c])
