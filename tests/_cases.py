"""Small seeded problems for the CPU pins and the GPU parity tests.

Each is a scaled-down variant of one of the workloads (same recipe, fewer
nodes per cell and fewer transverse nodes) so that the oracle's dense
route finishes in seconds while the kernels still see several tiles and a
ragged tail.  The quadrature table always comes from the oracle's rule.
"""
import numpy as np

import lattice_inputs as li
from oracle import blocks, sinc


def with_table(p):
    t, c, _ = sinc.table_for(p)
    return p.with_table(t, c)


def single_gaussian(alpha=1.0, n0=16, box=12.0, R=32, ang=0, L=1, periodic=False):
    h = 2.0 / n0
    N = int(round(box / h))
    if periodic:
        N = L * n0
    p = li.Problem(L=(L, 1, 1), periodic=(int(periodic), 0, 0), N=(N, N, N), n0=n0, b0=2.0,
                   Z=np.array([1.0]), frac=np.array([[0.5, 0.5, 0.5]]),
                   exps=np.array([alpha]), ang=np.array([ang]), centre=np.array([0]), R=R)
    return with_table(p)


def periodic_chain_small(L=6, n0=8, n_perp=24, m0=4, seed=0, R=24):
    if m0 == 4:
        p = li.config1()
        p = li.Problem(L=(L, 1, 1), periodic=(1, 0, 0), N=(L * n0, n_perp, n_perp), n0=n0,
                       b0=2.0, Z=p.Z, frac=p.frac, exps=p.exps, ang=p.ang, centre=p.centre, R=R)
    else:
        q = li.config2(seed, L=L, n0=n0, pad=0, n_perp=n_perp, R=R)
        p = li.Problem(L=(L, 1, 1), periodic=(1, 0, 0), N=(L * n0, n_perp, n_perp), n0=n0,
                       b0=2.0, Z=q.Z, frac=q.frac, exps=q.exps, ang=q.ang, centre=q.centre, R=R)
    return with_table(p)


def box_chain_small(L=12, n0=5, pad=6, n_perp=20, seed=0, R=24, k=6):
    p = li.config2(seed, L=L, n0=n0, pad=pad, n_perp=n_perp, R=R)
    p.k_eig = k
    return with_table(p)


def periodic_3d_small(L=(3, 2, 4), n0=6, seed=0, R=16):
    q = li.config3(seed, L=2, n0=n0, R=R)
    p = li.Problem(L=tuple(L), periodic=(1, 1, 1), N=tuple(l * n0 for l in L), n0=n0, b0=2.0,
                   Z=q.Z, frac=q.frac, exps=q.exps, ang=q.ang, centre=q.centre, R=R)
    return with_table(p)


U64 = 2.0 ** -53


def eig_tol(S, ev_ref, base=1e-10):
    """Absolute eigenvalue tolerance: max(base, 4 u kappa_2(S)) * max|lambda|.
    A backward-stable FP64 solve of the pencil (H, S) perturbs eigenvalues by
    about u * kappa_2(S) * |lambda|, so no FP64 method can promise better than
    that when the GTO basis is nearly dependent."""
    w = np.linalg.eigvalsh(S)
    kappa = float(w.max() / w.min())
    return max(base, 4.0 * U64 * kappa) * float(np.max(np.abs(ev_ref)))


def canon_tol(ev_ref, kappa, base=1e-10):
    """Eigenvalue tolerance after canonical orthogonalisation:
    max(base, 16 u kappa_K) * max|lambda| with kappa_K the condition number of
    the kept part of the overlap (at most 1/CANON_TAU): a backward-stable
    solve of the reduced pencil perturbs eigenvalues by about
    u kappa_K |lambda|; the factor 16 covers the rounding of the Fourier sums
    that form the blocks (sums over up to 32768 lattice terms whose Bloch
    combinations cancel)."""
    fin = np.isfinite(ev_ref)
    return max(base, 16.0 * U64 * float(np.max(kappa))) * float(np.max(np.abs(ev_ref[fin])))


def reference(p, H, S):
    """The oracle's answer under the canonical-orthogonalisation reading and
    its tolerance: periodic -> (sorted spectrum with +inf, tol, per-block
    spectra); box -> (lowest k_eig, tol, (eigenvectors, reduced overlap,
    block-diagonal cell basis))."""
    if blocks.structured(p):
        ev, V, Sr = blocks.box_eigs(p, H, S, vectors=True)
        Xb, _ = blocks.box_basis(p)
        return ev, eig_tol(Sr, ev), (V, Sr, Xb)
    ev, per, kap = blocks.periodic_eigs(p, H, S)
    return ev, canon_tol(ev, kap), per


def assert_spectra_match(got, ref, tol):
    """Same removed directions (+inf in the same places) and finite
    eigenvalues within tol."""
    got = np.asarray(got)
    assert np.array_equal(np.isfinite(got), np.isfinite(ref))
    f = np.isfinite(ref)
    if f.any():
        assert np.max(np.abs(got[f] - ref[f])) <= tol
