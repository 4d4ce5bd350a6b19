"""Pins of the oracle's second reading of the box potential (R2): the plain
lattice sum over the box's cells of Sec. 2.3 case (B), each nucleus of the
box counted once with its full charge, evaluated at the nodes' own
positions.  The library computes reading R1 (the central-cell sum
replicated to every cell, Sec. 3.3); R2 is the oracle of the next step,
the box matrix whose correction to the Toeplitz part spans the whole chain.

Pins: brute force over every cell in 3D; equality with R1 where the two
readings coincide (the central cell of an odd chain, a single cell);
the sum of single-nucleus kernels (an independent route through the defect
kernel); the Boys-function nuclear attraction of the nuclei of a chain,
which R1 does not reproduce; the band structure of the correction R1 - R2."""
import dataclasses

import numpy as np
import pytest

import lattice_inputs as li
from oracle import closed_forms as cf, dense, grid
from tests import _cases


def _expand(slab):
    so, slabs = slab
    return slabs[so]


def _box(L=(3, 2, 2), n0=4, pad=2, M0=2, m0=2, R=8, seed=3):
    """Small all-Dirichlet box with M0 nuclei per cell."""
    rng = np.random.default_rng(seed)
    N = tuple(l * n0 + 2 * pad for l in L)
    frac = rng.uniform(0.2, 0.8, size=(M0, 3))
    Z = rng.choice([1.0, 2.0, 3.0], size=M0)
    exps = np.sort(rng.uniform(0.5, 4.0, size=m0))
    p = li.Problem(L=L, periodic=(0, 0, 0), N=N, n0=n0, b0=2.0, Z=Z, frac=frac, exps=exps,
                   ang=np.zeros(m0, int), centre=np.arange(m0) % M0, R=R)
    return _cases.with_table(p)


def test_lattice_sum_potential_equals_cell_by_cell_sum():
    """The separable form (a product of per-axis sums over cells) equals the
    explicit loop over every 3D cell of the box."""
    p = _box()
    got = _expand(grid.potential_slabs(p, "lattice_sum"))
    ref = grid.potential_lattice_sum_brute(p)
    assert got.shape == ref.shape == tuple(p.N)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_lattice_sum_equals_window_sum_in_the_central_cell():
    """On an odd chain the window of the central cell is the whole chain, so
    the two readings agree on that cell's nodes, and disagree elsewhere."""
    p = _cases.box_chain_small(L=5, n0=6, pad=4, n_perp=10, R=12)
    P1 = _expand(grid.potential_slabs(p, "replicated"))
    P2 = _expand(grid.potential_slabs(p, "lattice_sum"))
    x, X0, _ = grid.axis_nodes(p, 0)
    cell = np.floor((x - X0) / p.b0)
    mid = cell == (p.L[0] - 1) // 2
    assert mid.sum() == p.n0
    scale = np.max(np.abs(P2))
    assert np.max(np.abs(P1[mid] - P2[mid])) <= 1e-14 * scale
    assert np.max(np.abs(P1[~mid] - P2[~mid])) > 1e-3 * scale


def test_single_cell_readings_coincide():
    p = _cases.single_gaussian(alpha=1.3, n0=6, box=8.0, R=16)
    P1 = _expand(grid.potential_slabs(p, "replicated"))
    P2 = _expand(grid.potential_slabs(p, "lattice_sum"))
    assert np.max(np.abs(P1 - P2)) <= 1e-15 * np.max(np.abs(P1))


def test_lattice_sum_is_the_sum_of_single_nucleus_kernels():
    """V under R2 equals minus the defect matrix of the box with every nucleus
    of every cell vacated: the defect route evaluates each nucleus' own 3D
    kernel separately, with no sum over cells factorised per axis."""
    p = _box(L=(4, 1, 1), n0=4, pad=3, M0=2, m0=3, R=8, seed=7)
    p = dataclasses.replace(p, N=(p.N[0], 10, 10))
    V = dense.potential_matrix(p, box_potential="lattice_sum")
    cells = [(k1, k2, k3) for k1 in range(p.L[0]) for k2 in range(p.L[1]) for k3 in range(p.L[2])]
    q = dataclasses.replace(p, defects=[li.Defect(cell=c, nucleus=nu, newZ=0.0)
                                        for c in cells for nu in range(p.M0)])
    D = dense.defect_matrix(q)
    assert np.max(np.abs(V + D)) <= 1e-13 * np.max(np.abs(V))


def test_chain_attraction_vs_boys_closed_form():
    """Three-cell chain, one normalised s-Gaussian and one proton per cell:
    the R2 entries approach the sum over the three nuclei of the
    Boys-function attraction integrals as h shrinks; R1 (each cell sees the
    window centred on itself, so an end cell sees a proton one cell beyond
    the end and misses the one two cells away) stays far from it."""
    alpha = 1.0
    err2, err1 = [], []
    for n0 in (8, 16):
        p = _cases.single_gaussian(alpha=alpha, n0=n0, box=14.0, R=40, L=3)
        _, X0, _ = grid.axis_nodes(p, 0)
        yc = grid.axis_nodes(p, 1)[1] + 0.5 * p.b0
        A = [np.array([X0 + (k + 0.5) * p.b0, yc, yc]) for k in range(3)]
        ref = np.array([[sum(cf.nuclear_ss(alpha, A[a], alpha, A[b], C) for C in A)
                         for b in range(3)] for a in range(3)])
        V2 = dense.potential_matrix(p, box_potential="lattice_sum")
        V1 = dense.potential_matrix(p, box_potential="replicated")
        err2.append(np.max(np.abs(V2 - ref)) / np.max(np.abs(ref)))
        err1.append(np.max(np.abs(V1 - ref)) / np.max(np.abs(ref)))
    assert err2[1] < err2[0] / 2.5
    assert err2[1] < 1e-2
    assert err1[1] > 10 * err2[1]


def test_correction_is_block_banded_over_the_whole_chain():
    """E = V(R1) - V(R2), the term the box matrix under R2 adds to the
    Toeplitz part, is symmetric, vanishes exactly on block pairs whose
    supports do not meet, and is not confined to the walls: every diagonal
    block carries it (largest at the ends, where R1 adds a proton beyond
    the wall; in the middle of an even chain the half-weight end terms of
    the window nearly cancel)."""
    p = _box(L=(8, 1, 1), n0=4, pad=3, M0=1, m0=2, R=10)
    p = dataclasses.replace(p, N=(p.N[0], 10, 10), exps=np.array([3.0, 6.0]))
    V1 = dense.potential_matrix(p, box_potential="replicated")
    V2 = dense.potential_matrix(p, box_potential="lattice_sum")
    E = V1 - V2
    m0, L = p.m0, p.L[0]
    G = grid.basis_axis(p, 0)                              # (N, L, m0)
    sup = np.abs(G).sum(axis=2) > 0                        # node in the support of cell k
    scale = np.max(np.abs(V2))
    assert np.max(np.abs(E - E.T)) <= 1e-14 * scale
    apart = 0
    for k in range(L):
        Ekk = E[k * m0:(k + 1) * m0, k * m0:(k + 1) * m0]
        assert np.max(np.abs(Ekk)) > 1e-6 * scale
        if k in (0, L - 1):
            assert np.max(np.abs(Ekk)) > 1e-2 * scale
        for m in range(L):
            blk = E[k * m0:(k + 1) * m0, m * m0:(m + 1) * m0]
            if not np.any(sup[:, k] & sup[:, m]):
                apart += 1
                assert np.all(blk == 0.0)
    assert apart > 0


def test_unknown_reading_is_refused():
    p = _cases.single_gaussian(alpha=1.0, n0=4, box=6.0, R=8)
    with pytest.raises(ValueError):
        grid.potential_slabs(p, "exact")
