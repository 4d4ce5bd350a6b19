"""The planner's block maps (host only, fock_problem_layout) against the
oracle's dense matrices, on the CPU: a box chain is banded block Toeplitz
(Remark 3.2) plus the blocks E the planner lists (walls, Sec. 2.3; defects;
wrap-around corners of periodic chains), so every block the planner does
not list must equal the Toeplitz generator of its offset, or vanish
outside the band.  Integer maps, compared exactly; block values to the
oracle's rounding."""
import dataclasses

import numpy as np
import pytest

import lattice_inputs as li
from oracle import dense
from tests import _cases


@pytest.fixture(scope="module")
def fock():
    from paper_1702_00339_gb300 import build, fock as f
    build.build()
    return f


def _blk(M, m0, k, m):
    return M[k * m0:(k + 1) * m0, m * m0:(m + 1) * m0]


def _check_box(fock, p, base=None):
    """base: the same chain without defects, whose interior cells give the
    Toeplitz generators (with defects every row carries defect blocks)."""
    lay = fock.problem_layout(p)
    m0, L, D = p.m0, p.L[0], lay["D"]
    E = lay["E"]
    listed = {(int(k), int(m)) for k, m, _ in E}
    # sorted by (row, column), no duplicates of a (pair, kind)
    assert [tuple(x) for x in E[:, :2]] == sorted(tuple(x) for x in E[:, :2])
    # a wall block below the diagonal is the transpose of its listed mirror
    kinds = {(int(k), int(m), int(c)) for k, m, c in E}
    for k, m, c in E:
        if c == 3:
            assert k > m and (int(m), int(k), 0) in kinds
        if c == 0:
            assert k <= m
    # the embedding holds the band without wrap-around, with 2/3/5 factors only
    M = lay["mcirc"]
    assert M >= L + D
    r = M
    for f in (2, 3, 5):
        while r % f == 0:
            r //= f
    assert r == 1
    H, S = dense.build(p)
    Hg, Sg = (H, S) if base is None else dense.build(base)
    listed_g = listed if base is None else {(int(k), int(m)) for k, m, _ in fock.problem_layout(base)["E"]}
    # Toeplitz generators from a cell whose row carries no listed block
    free = [k for k in range(D, L - D) if not any(kk == k for kk, _ in listed_g)]
    assert free, "no interior cell"
    kc = free[len(free) // 2]
    for X, Xg in ((H, Hg), (S, Sg)):
        scale = np.max(np.abs(X))
        T = {d: _blk(Xg, m0, kc + d, kc) for d in range(-D, D + 1)}
        band = 0
        for k in range(L):
            for m in range(L):
                if (k, m) in listed:
                    continue
                ref = T[k - m] if abs(k - m) <= D else np.zeros((m0, m0))
                assert np.max(np.abs(_blk(X, m0, k, m) - ref)) <= 1e-12 * scale, (k, m)
                band += abs(k - m) <= D
        assert band > 0 or base is not None      # with defects every in-band pair is listed
    # the reach covers the band and exceeds it by at most one block: the
    # planner takes D = floor(span / n0) for a support of `span` nodes plus
    # the stencil, one more than needed when span is a multiple of n0 (the
    # extra generator is then exactly zero)
    assert np.max(np.abs(_blk(Hg, m0, kc + D - 1, kc))) > 0.0
    return lay


def test_box_chain_maps(fock):
    lay = _check_box(fock, _cases.box_chain_small(L=24, n0=5, pad=8, n_perp=14, R=12, k=6))
    assert set(lay["E"][:, 2]) <= {0, 3}


def test_box_chain_with_defects_maps(fock):
    base = _cases.box_chain_small(L=20, n0=5, pad=6, n_perp=12, R=10, k=4, seed=2)
    p = dataclasses.replace(base, defects=[li.Defect((6, 0, 0), 0, 0.0), li.Defect((13, 0, 0), 0, 2.0)])
    p.k_eig = 4
    lay = _check_box(fock, p, base)
    # every block the defects change carries a defect entry
    Dm = dense.defect_matrix(p)
    dblocks = {(int(k), int(m)) for k, m, c in lay["E"] if c == 2}
    m0, L = p.m0, p.L[0]
    changed = {(k, m) for k in range(L) for m in range(L) if np.any(_blk(Dm, m0, k, m) != 0.0)}
    assert changed and changed <= dblocks


def test_periodic_chain_with_defect_maps(fock):
    """A periodic chain with a defect: the Toeplitz band of the ring's
    generators, the wrap-around corners (kind 1) and the defect blocks
    (kind 2) reproduce the dense matrix."""
    base = _cases.periodic_chain_small(L=30, n0=4, n_perp=12, m0=4, R=10)
    p = dataclasses.replace(base, defects=[li.Defect((3, 0, 0), 0, 3.0)])
    p.k_eig = 6
    lay = fock.problem_layout(p)
    m0, L, D = p.m0, p.L[0], lay["D"]
    assert D < L - 1                                   # band plus corners, not the whole circulant
    listed = {(int(k), int(m)) for k, m, _ in lay["E"]}
    assert {1, 2} <= set(lay["E"][:, 2])
    H, S = dense.build(p)
    Hp, Sp = dense.build(base)
    for X, Xp in ((H, Hp), (S, Sp)):
        scale = np.max(np.abs(X))
        for k in range(L):
            for m in range(L):
                if (k, m) in listed:
                    continue
                ref = _blk(Xp, m0, (k - m) % L, 0) if abs(k - m) <= D else np.zeros((m0, m0))
                assert np.max(np.abs(_blk(X, m0, k, m) - ref)) <= 1e-12 * scale, (k, m)


def _check_ring(fock, p):
    """Periodic chain with defects: unlisted blocks are the ring generators
    inside the band or zero; defect-changed blocks carry defect entries."""
    base = dataclasses.replace(p, defects=[])
    lay = fock.problem_layout(p)
    m0, L, D = p.m0, p.L[0], lay["D"]
    listed = {(int(k), int(m)) for k, m, _ in lay["E"]}
    Hp, Sp = dense.build(base)
    Dm = dense.defect_matrix(p)
    for X, Xp in ((Hp - Dm, Hp), (Sp, Sp)):
        scale = np.max(np.abs(X))
        for k in range(L):
            for m in range(L):
                if (k, m) in listed:
                    continue
                ref = _blk(Xp, m0, (k - m) % L, 0) if abs(k - m) <= D else np.zeros((m0, m0))
                assert np.max(np.abs(_blk(X, m0, k, m) - ref)) <= 1e-12 * scale, (k, m)
    dblocks = {(int(k), int(m)) for k, m, c in lay["E"] if c == 2}
    changed = {(k, m) for k in range(L) for m in range(L) if np.any(_blk(Dm, m0, k, m) != 0.0)}
    assert changed <= dblocks


# chains of the serving mix (16 nodes per cell, box or periodic, 0-4 defects), with the
# cross-section reduced to 16 x 16 nodes (the block maps depend on the chain axis only);
# box chains long enough to have a cell that no wall reaches, which gives the generators
SERVING_CHAINS = [27, 34, 49, 151, 167, 174, 185, 192, 200, 222]


@pytest.mark.parametrize("rid", SERVING_CHAINS)
def test_serving_mix_chain_maps(fock, rid):
    p = li.serving_stream(rid + 1, seed=3000)[rid]
    q = _cases.with_table(dataclasses.replace(p, N=(p.N[0], 16, 16)))
    q.k_eig = p.k_eig
    if q.periodic[0]:
        _check_ring(fock, q)
    else:
        lay = _check_box(fock, q, dataclasses.replace(q, defects=[]) if q.defects else None)
        if q.defects:
            Dm = dense.defect_matrix(q)
            m0, L = q.m0, q.L[0]
            dblocks = {(int(k), int(m)) for k, m, c in lay["E"] if c == 2}
            changed = {(k, m) for k in range(L) for m in range(L) if np.any(_blk(Dm, m0, k, m) != 0.0)}
            assert changed <= dblocks


def test_short_periodic_chain_is_its_whole_circulant(fock):
    """A ring too short for the band and the corners to separate is planned
    as its whole circulant written as a Toeplitz matrix (D = L - 1): no
    wrap-around entries, only the defect blocks."""
    base = _cases.periodic_chain_small(L=6, n0=6, n_perp=14, m0=4, R=12)
    p = dataclasses.replace(base, defects=[li.Defect((1, 0, 0), 0, 0.0)])
    p.k_eig = 4
    lay = fock.problem_layout(p)
    assert lay["D"] == p.L[0] - 1 and set(lay["E"][:, 2]) == {2}
    _check_ring(fock, p)


def test_periodic_lattice_layout(fock):
    p = _cases.periodic_3d_small(L=(3, 2, 4), n0=4, R=8)
    lay = fock.problem_layout(p)
    assert lay == {"Nb": 24 * p.m0, "mcirc": 24, "D": 0, "E": lay["E"]} and len(lay["E"]) == 0


def test_layout_refuses_malformed(fock):
    p = dataclasses.replace(_cases.box_chain_small(L=8, n0=5, pad=4, n_perp=12, R=8, k=4), n0=0)
    with pytest.raises(fock.FockError):
        fock.problem_layout(p)
