"""GPU parity at the full sizes of the large workloads (16^3 and 32^3 periodic
lattices, the 512-cell box chain) against oracle results stored by
tests/golden/make_golden.py (CPU oracle only; nothing in them comes from the
GPU):

* generator blocks at sampled lattice offsets (3D grid contraction);
* Fourier-block spectra (direct DFT over every offset, LAPACK on each block
  pencil): every block of the 16^3 lattice, a seeded sample of 64 blocks of
  the 32^3 one, each against its admissible variants under the dependency
  rule, within the per-eigenvalue bar of tests/_cases.py;
* box chain: Toeplitz generators at an interior cell, the corner block of
  the first cell, and the lowest 64 eigenvalues of the dense pencil
  (LAPACK on 16384 x 16384);
* box chains of the timed workload (64 cells, grid 1024x256x256), where the
  dense oracle runs in the test: a batch solved together, each against it;
* a ring of 202 cells with two identical, distant substitutions, whose
  levels are all exactly degenerate pairs: the lowest 16 against the dense
  pencil's.

The mixed form (tensor-core split products in the assembly and in the block
iteration) is checked against the same stored results with the mixed bar
(base 1e-8).
"""
import dataclasses
import os

import numpy as np
import pytest

import lattice_inputs as li
from oracle import dense
from tests import _cases

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def ctx():
    from paper_1702_00339_gb300 import build, fock
    build.build()
    c = fock.Context(0)
    yield c
    c.close()


MIXED_BASE = 1e-8


def _mixed(p):
    q = dataclasses.replace(p, precision=1)
    q.k_eig = p.k_eig
    return q


def _periodic_against_golden(ctx, p, name, base=1e-10):
    g = np.load(os.path.join(GOLD, name + ".npz"))
    b = ctx.assemble(p)
    gh, gs, _, _, _ = b.generators()
    k = g["k"]
    assert np.max(np.abs(gh[k] - g["gen_H"])) <= 1e-12 * np.max(np.abs(g["gen_H"]))
    assert np.max(np.abs(gs[k] - g["gen_S"])) <= 1e-12 * np.max(np.abs(g["gen_S"]))
    ev, blk = b.circulant_eig()
    b.close()
    fin = np.isfinite(ev)
    assert np.all(np.diff(ev[fin]) >= 0) and np.all(fin[:fin.sum()])   # +inf (removed) last
    assert np.all(np.bincount(blk, minlength=p.ncell) == p.m0)
    cands, scale = _cases.golden_candidates(g, base)
    _cases.report(name + ("_mixed" if base != 1e-10 else ""), _cases.check_blocks(cands, scale, ev, blk))


def test_periodic_16cubed_m0_16(ctx):
    _periodic_against_golden(ctx, _cases.with_table(li.config3(0)), "config3_periodic_16cubed_seed0")


def test_periodic_32cubed_m0_32(ctx):
    _periodic_against_golden(ctx, _cases.with_table(li.config5_periodic(0)),
                             "config5_periodic_32cubed_seed0")


def test_periodic_32cubed_m0_32_mixed(ctx):
    _periodic_against_golden(ctx, _mixed(_cases.with_table(li.config5_periodic(0))),
                             "config5_periodic_32cubed_seed0", base=MIXED_BASE)


def test_periodic_16cubed_m0_16_mixed(ctx):
    _periodic_against_golden(ctx, _mixed(_cases.with_table(li.config3(0))),
                             "config3_periodic_16cubed_seed0", base=MIXED_BASE)


@pytest.mark.parametrize("precision", [0, 1])
def test_box_512_m0_32_lowest_64(ctx, precision):
    from paper_1702_00339_gb300 import fock
    name = "config5_box_512_seed0"
    g = np.load(os.path.join(GOLD, name + ".npz"))
    p = _cases.with_table(li.config5_box(0))
    if precision:
        p = _mixed(p)
    base = MIXED_BASE if precision else 1e-10
    b = ctx.assemble(p)
    TH, TS, EH, ES, rc = b.generators()
    D = (TH.shape[0] - 1) // 2
    for i, d in enumerate(g["d"]):
        assert np.max(np.abs(TH[D + d] - g["T_H"][i])) <= 1e-12 * np.max(np.abs(g["T_H"]))
        assert np.max(np.abs(TS[D + d] - g["T_S"][i])) <= 1e-12 * np.max(np.abs(g["T_S"]))
    e0 = [e for e, (kk, m) in enumerate(rc) if kk == 0 and m == 0][0]
    assert np.max(np.abs(TH[D] + EH[e0] - g["C_H"])) <= 1e-12 * np.max(np.abs(g["T_H"]))
    assert np.max(np.abs(TS[D] + ES[e0] - g["C_S"])) <= 1e-12 * np.max(np.abs(g["T_S"]))
    k = int(g["k"])
    ev, V, iters, rcode = b.box_eig(k, tol=1e-10, maxit=600, vectors=True)
    SV = b.matvec(V, fock.FOCK_OP_S)
    b.close()
    assert rcode == 0, f"no convergence in {iters} iterations"
    assert np.max(np.abs(V.T @ SV - np.eye(k))) < 1e-7          # S-orthonormal (GPU's own S)
    scale = float(np.max(np.abs(g["ev"][0])))
    cands = []
    for evv, vn in zip(g["ev"], g["vn2"]):
        tol = np.maximum(base * scale, _cases.EPS_DATA * (float(g["Hn"]) + np.abs(evv) * float(g["Sn"])) * vn)
        cands.append((evv, tol))
    e = _cases._match(np.asarray(ev), cands)
    assert e is not None, f"lowest {k} off every variant: max |d| {np.max(np.abs(ev - g['ev'][0])):.3e}"
    _cases.report(name + ("_mixed" if precision else ""), e / scale)


def test_box_chains_of_the_timed_workload(ctx):
    """Box chains 64x1x1 (n0=15, pad 32, 256^2 cross-section, m0=8, R=32,
    lowest 16) solved as one batch, each against the oracle's dense solve.
    Seed 301 once ended with a spurious Ritz pair reported as converged: the
    cell-transformed zero-offset generator was symmetric only to rounding
    amplified by the canonical factors, the one-sided Gram products of the
    block iteration were then inconsistent, and the Rayleigh-Ritz step broke
    down after the residual had reached its floor."""
    seeds = [0, 1, 2, 6, 31, 77, 300, 301, 302, 511]
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
        ref = _cases.reference(q, H, S)
        assert o["status"] == 0, s
        _cases.report(f"timed_box_seed{s}", _cases.check(ref, o["evals"]))


@pytest.mark.parametrize("precision", [0, 1])
def test_ring_with_degenerate_pairs(ctx, precision):
    """Ring 202 x 1 x 1 (m0 = 4) with Z = 3 substitutions at cells 92 and 171:
    every level is a pair, exactly degenerate in double precision, and the
    Ritz values of each pair split by about lambda res^2 as the block
    iteration converges.  When such a split fell inside one FP32 multisection
    bracket of the Rayleigh-Ritz eigensolver, both inverse-iteration vectors
    converged to one eigenvector, the Ritz basis lost rank and the solve
    ended without convergence (FP64 form after 30 iterations, mixed after 50);
    the vectors of a cluster of shifts are now orthogonalised against each
    other."""
    g = np.load(os.path.join(GOLD, "ring_202_two_defects.npz"))
    p = li.serving_stream(512, seed=3000)[328]
    assert p.L == (202, 1, 1) and p.periodic == (1, 0, 0) and len(p.defects) == 2
    q = _cases.with_table(p)
    q.k_eig = p.k_eig
    if precision:
        q = _mixed(q)
    o = ctx.solve([q], check=False)[0]
    assert o["status"] == 0, f"status {o['status']} after {o['iters']} iterations"
    k = int(g["k"])
    ev = np.asarray(o["evals"][:k])
    base = MIXED_BASE if precision else 1e-10
    scale = float(np.max(np.abs(g["ev"][0])))
    cands = []
    for evv, vn in zip(g["ev"], g["vn2"]):
        tol = np.maximum(base * scale, _cases.EPS_DATA * (float(g["Hn"]) + np.abs(evv) * float(g["Sn"])) * vn)
        cands.append((evv, tol))
    e = _cases._match(ev, cands)
    assert e is not None, f"lowest {k} off the oracle: max |d| {np.max(np.abs(ev - g['ev'][0])):.3e}"
    _cases.report("ring_202_two_defects" + ("_mixed" if precision else ""), e / scale)
