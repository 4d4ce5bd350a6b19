"""GPU parity at the full sizes of the large workloads (16^3 and 32^3 periodic
lattices, the 512-cell box chain), where the dense oracle does not fit:

* generator blocks sampled by the oracle's one-block 3D contraction;
* Fourier blocks of the GPU's generators by the oracle's direct DFT
  (explicit sum over every lattice offset) and LAPACK, against the GPU's
  eigenvalues carrying that block index;
* box chain: lowest eigenpairs against shift-invert ARPACK (SciPy) on the
  sparse block-banded matrix built from the GPU's blocks (those blocks are
  themselves sampled against the oracle), plus residuals and S-orthonormality;
* box chains of the timed workload (64 cells, grid 1024x256x256), where the
  dense oracle does fit: a batch solved together, each against the oracle.
"""
import numpy as np
import pytest

import lattice_inputs as li
from oracle import blocks, dense, grid
from tests import _cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1702_00339_gb300 import build, fock
    build.build()
    c = fock.Context(0)
    yield c
    c.close()


def _kbar(p, kc):
    return (kc[0] * p.L[1] + kc[1]) * p.L[2] + kc[2]


def _periodic_checks(ctx, p, kcells, jcells):
    b = ctx.assemble(p)
    gh, gs, _, _, _ = b.generators()
    scale_h = np.max(np.abs(gh))
    forms = dense.axis_forms(p)
    slab = grid.potential_slabs(p)
    for kc in kcells:
        h, s = blocks.generator_block(p, kc, forms=forms, slab=slab)
        kb = _kbar(p, kc)
        assert np.max(np.abs(gh[kb] - h)) <= 1e-12 * scale_h
        assert np.max(np.abs(gs[kb] - s)) <= 1e-12 * np.max(np.abs(gs))
    ev, blk = b.circulant_eig()
    b.close()
    fin = np.isfinite(ev)
    assert np.all(np.diff(ev[fin]) >= 0) and np.all(fin[:fin.sum()])   # +inf (dropped) last
    counts = np.bincount(blk, minlength=p.ncell)
    assert np.all(counts == p.m0)
    for jc in jcells:
        Hb, Sb, _ = blocks.fourier_block_from_generators(p, gh, gs, jc)
        ref, _, kappa = blocks.canonical(Hb, Sb)
        got = np.sort(ev[blk == _kbar(p, jc)])
        _cases.assert_spectra_match(got, ref, _cases.canon_tol(ref, kappa))


def test_periodic_16cubed_m0_16(ctx):
    p = _cases.with_table(li.config3(0))
    _periodic_checks(ctx, p, [(0, 0, 0), (1, 0, 0), (3, 2, 15), (8, 8, 8)],
                     [(0, 0, 0), (1, 2, 3), (8, 8, 8), (15, 0, 7)])


def test_periodic_32cubed_m0_32(ctx):
    p = _cases.with_table(li.config5_periodic(0))
    _periodic_checks(ctx, p, [(0, 0, 0), (1, 31, 0), (16, 16, 16)],
                     [(0, 0, 0), (5, 17, 30), (16, 16, 16)])


def test_box_512_m0_32_lowest_64(ctx):
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    p = _cases.with_table(li.config5_box(0))
    b = ctx.assemble(p)
    TH, TS, EH, ES, rc = b.generators()
    D = (TH.shape[0] - 1) // 2
    m0, L = p.m0, p.L[0]
    forms = None   # one-block route: only the sampled cells are evaluated
    slab = grid.potential_slabs(p)
    kc = L // 2
    scale = np.max(np.abs(TH))
    for d in (0, 1, 5):
        h, s = blocks.generator_block(p, (kc + d, 0, 0), forms=forms, slab=slab, mcell=(kc, 0, 0))
        assert np.max(np.abs(TH[D + d] - h)) <= 1e-12 * scale
        assert np.max(np.abs(TS[D + d] - s)) <= 1e-12 * np.max(np.abs(TS))
    e0 = [e for e, (k, m) in enumerate(rc) if k == 0 and m == 0][0]
    h, s = blocks.generator_block(p, (0, 0, 0), forms=forms, slab=slab, mcell=(0, 0, 0))
    assert np.max(np.abs(TH[D] + EH[e0] - h)) <= 1e-12 * scale
    # sparse block-banded (H, S) from the GPU's blocks
    def assemble(T, E):
        rows, cols, vals = [], [], []
        for k in range(L):
            for d in range(-D, D + 1):
                m = k - d
                if 0 <= m < L:
                    rows.append(k); cols.append(m); vals.append(T[d + D])
        for e, (k, m) in enumerate(rc):
            rows.append(k); cols.append(m); vals.append(E[e])
        blk = {}
        for r_, c_, v_ in zip(rows, cols, vals):
            blk[(r_, c_)] = blk.get((r_, c_), 0) + v_
        coo_r, coo_c, coo_v = [], [], []
        ii, jj = np.meshgrid(np.arange(m0), np.arange(m0), indexing="ij")
        for (r_, c_), v_ in blk.items():
            coo_r.append((r_ * m0 + ii).ravel()); coo_c.append((c_ * m0 + jj).ravel())
            coo_v.append(v_.ravel())
        return sp.csc_matrix((np.concatenate(coo_v), (np.concatenate(coo_r), np.concatenate(coo_c))),
                             shape=(L * m0, L * m0))
    Hs, Ss = assemble(TH, EH), assemble(TS, ES)
    # the oracle's canonical cell basis (from its own cell overlap)
    Xc, _ = blocks.lowdin_basis(blocks.cell_overlap(p))
    Xb = sp.kron(sp.identity(L, format="csc"), sp.csc_matrix(Xc), format="csc")
    Hr = (Xb.T @ Hs @ Xb).tocsc()
    Sr = (Xb.T @ Ss @ Xb).tocsc()
    k = p.k_eig
    ev, V, iters, rcode = b.box_eig(k, tol=1e-10, maxit=600, vectors=True)
    b.close()
    assert rcode == 0, f"no convergence in {iters} iterations"
    # Rayleigh quotients and S-orthonormality in the original basis, residual in the reduced one
    SV = Ss @ V
    assert np.max(np.abs(V.T @ SV - np.eye(k))) < 1e-7
    rq = np.einsum("ij,ij->j", V, Hs @ V) / np.einsum("ij,ij->j", V, SV)
    assert np.max(np.abs(rq - ev)) <= 1e-9 * np.max(np.abs(ev))
    R = Xb.T @ (Hs @ V - SV * ev)
    res = np.linalg.norm(R, axis=0) / (np.abs(ev) * np.linalg.norm(Xb.T @ SV, axis=0))
    assert np.max(res) < 1e-8
    sigma = ev[0] - 0.05 * (1 + abs(ev[0]))
    ref = np.sort(spla.eigsh(Hr, k=k, M=Sr, sigma=sigma, which="LM", return_eigenvectors=False,
                             tol=1e-13))
    assert np.max(np.abs(ev - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_box_chains_of_the_timed_workload(ctx):
    """Box chains 64x1x1 (n0=15, pad 32, 256^2 cross-section, m0=8, R=32,
    lowest 16) solved as one batch, each against the oracle's dense solve.
    Seed 301 once ended with a spurious Ritz pair reported as converged: the
    cell-transformed zero-offset generator was symmetric only to rounding
    amplified by the canonical factors, the one-sided Gram products of the
    block iteration were then inconsistent, and the Rayleigh-Ritz step broke
    down after the residual had reached its floor."""
    seeds = [0, 1, 77, 300, 301, 302, 511]
    ps = []
    for s in seeds:
        p = li.config2(s, L=64, n0=15, pad=32, n_perp=256, R=32)
        p.k_eig = 16
        ps.append(p)
    outs = ctx.solve(ps)
    for s, p, o in zip(seeds, ps, outs):
        q = _cases.with_table(p)
        q.k_eig = p.k_eig
        H, S = dense.build(q)
        ref, tol, _ = _cases.reference(q, H, S)
        assert o["status"] == 0, s
        assert np.max(np.abs(o["evals"] - ref)) <= tol, s
