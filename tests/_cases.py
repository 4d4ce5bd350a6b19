"""Small seeded problems for the CPU pins and the GPU parity tests, and the
comparison of a computed spectrum with the oracle's.

Each problem is a scaled-down variant of one of the workloads (same recipe,
fewer nodes per cell and fewer transverse nodes) so that the oracle's dense
route finishes in seconds while the kernels still see several tiles and a
ragged tail.  The quadrature table always comes from the oracle's rule.

Eigenvalue bar (reading G15).  An eigenvalue lambda_i of the pencil (H, S)
with S-normalised eigenvector x_i moves, to first order, by
x_i^T (dH - lambda_i dS) x_i under perturbations dH, dS of the data, so
perturbations of size eps ||H||, eps ||S|| move it by at most
eps (||H|| + |lambda_i| ||S||) ||x_i||^2 (the eigenvalue's condition number
for definite pencils).  Two FP64 computations of the same matrices differ by
rounding at about that eps, so the bar is

    |lambda_i - lambda_i^ref| <= max(base * max_j |lambda_j^ref|,
                                     EPS_DATA (||H||_inf + |lambda_i| ||S||_inf) ||x_i||^2)

with base = 1e-10 (FP64 form; 1e-8 mixed form), EPS_DATA = 256 u
(u = 2^-53, a few units of rounding per entry over sums of up to ~100
terms), x_i the oracle's eigenvector and ||.||_inf the largest row sum of
|H| and |S|.  On a well-conditioned basis the first term is the bar; the
second only widens it for eigenvalues whose eigenvectors lean on directions
of small overlap.  Directions whose overlap eigenvalue lies within a factor 4
of the dependency cut tau (reading G16) are decided by rounding: both
decisions are correct readings, the oracle computes each variant, and the
result must match one of them.
"""
import itertools

import numpy as np

import lattice_inputs as li
from oracle import blocks, sinc

U64 = 2.0 ** -53
EPS_DATA = 256 * U64


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


def _flips(amb, cap=3):
    """Subsets of the ambiguous indices (all of them when there are at most
    `cap`; else only the `cap` nearest the cut vary)."""
    amb = list(amb)[:cap]
    out = []
    for r in range(len(amb) + 1):
        out += [tuple(c) for c in itertools.combinations(amb, r)]
    return out


def _tols(ev, V, Hn, Sn, scale, base):
    """Per-eigenvalue bar of the module docstring for the finite ev (V:
    their S-normalised eigenvectors, columns)."""
    fin = np.isfinite(ev)
    t = np.full(ev.shape, np.inf)
    xn2 = np.sum(np.abs(V) ** 2, axis=0)
    t[fin] = np.maximum(base * scale, EPS_DATA * (Hn + np.abs(ev[fin]) * Sn) * xn2[:fin.sum()])
    return t


class Reference:
    """The oracle's answer to one problem with its bar.  kind 'periodic':
    `ev` = sorted spectrum (+inf for removed directions), `cands[j]` = the
    admissible (eigenvalues, bar) of Fourier block j; kind 'structured':
    `ev` = lowest k_eig, `cands` = admissible (eigenvalues, bar, vectors)."""

    def __init__(self, kind, ev, cands, scale, V=None, tau=None):
        self.kind, self.ev, self.cands, self.scale, self.V, self.tau = kind, ev, cands, scale, V, tau


def reference(p, H, S, base=1e-10):
    Hn = float(np.max(np.sum(np.abs(H), axis=1)))
    Sn = float(np.max(np.sum(np.abs(S), axis=1)))
    tau = blocks.null_threshold(p)
    if blocks.structured(p):
        s, _, _ = blocks.cell_null_directions(p, tau)
        variants = [blocks.box_eigs(p, H, S, tau=tau, vectors=True, flip=f)
                    for f in _flips(blocks.ambiguous(s, tau))]
        scale = float(np.max(np.abs(variants[0][0])))
        cands = [(ev, _tols(ev, V, Hn, Sn, scale, base), V) for ev, V, _ in variants]
        return Reference("structured", variants[0][0], cands, scale, V=variants[0][1], tau=tau)
    Hb, Sb = blocks.periodic_fourier_blocks(p, H, S)
    per = []
    for j in range(p.ncell):
        w = np.linalg.eigvalsh(Sb[j])
        per.append([blocks.block_pencil(Hb[j], Sb[j], tau, flip=f)
                    for f in _flips(blocks.ambiguous(w, tau))])
    allev = np.concatenate([c[0][0] for c in per])
    fin = np.isfinite(allev)
    scale = float(np.max(np.abs(allev[fin]))) if fin.any() else 1.0
    cands = [[(ev, _tols(ev, V, Hn, Sn, scale, base)) for ev, V, _ in c] for c in per]
    return Reference("periodic", np.sort(allev), cands, scale, tau=tau)


def _match(got, cands):
    """Largest |got - ref| / scale over the best-matching candidate, or None
    when none matches within its bar."""
    best = None
    for c in cands:
        ev, tol = c[0], c[1]
        if got.shape != ev.shape or not np.array_equal(np.isfinite(got), np.isfinite(ev)):
            continue
        f = np.isfinite(ev)
        d = np.abs(got[f] - ev[f])
        if np.all(d <= tol[f]):
            e = float(np.max(d)) if f.any() else 0.0
            best = e if best is None else min(best, e)
    return best


def check(ref, evals, block_of=None):
    """Asserts that a computed result matches the oracle within the bar and
    returns its largest error relative to max|lambda|.  Periodic problems are
    compared Fourier block by Fourier block (block_of), each block against
    its admissible variants; structured ones as the lowest k_eig."""
    evals = np.asarray(evals, float)
    if ref.kind == "structured":
        e = _match(evals, ref.cands)
        if e is None:
            c = ref.cands[0]
            d = np.abs(evals - c[0])
            raise AssertionError(f"lowest eigenvalues off the bar: max |d| {d.max():.3e}, "
                                 f"max |d|/tol {np.max(d / c[1]):.3e}, k {len(d)}")
        return e / ref.scale
    assert block_of is not None
    block_of = np.asarray(block_of)
    assert np.array_equal(np.bincount(block_of, minlength=len(ref.cands)),
                          np.full(len(ref.cands), len(ref.cands[0][0][0])))
    fin = np.isfinite(evals)
    assert np.all(np.diff(evals[fin]) >= 0) and np.all(fin[:fin.sum()])   # +inf last
    worst = 0.0
    for j, cands in enumerate(ref.cands):
        got = np.sort(evals[block_of == j])
        e = _match(got, cands)
        if e is None:
            ev, tol = cands[0]
            f = np.isfinite(ev) & np.isfinite(got)
            raise AssertionError(f"Fourier block {j}: finite {np.isfinite(got).sum()} vs "
                                 f"{np.isfinite(ev).sum()}, max |d|/tol "
                                 f"{np.max(np.abs(got[f] - ev[f]) / tol[f]) if f.any() else 0:.3e}")
        worst = max(worst, e)
    return worst / ref.scale


def report(label, err):
    """Prints the measured parity error of a test (visible with pytest -s)."""
    print(f"PARITY {label} max_rel_err={err:.3e}")


def golden_candidates(g, base=1e-10):
    """Admissible block spectra from a stored oracle file (tests/golden):
    {Fourier index: [(eigenvalues, bar), ...]} with the bar of the module
    docstring from the stored eigenvector norms."""
    scale = float(g["scale"])
    Hn, Sn = float(g["Hn"]), float(g["Sn"])

    def bar(ev, vn2):
        t = np.full(ev.shape, np.inf)
        f = np.isfinite(ev)
        t[f] = np.maximum(base * scale, EPS_DATA * (Hn + np.abs(ev[f]) * Sn) * vn2[f])
        return t
    out = {}
    for j, ev, vn in zip(g["j"], g["ev"], g["vn2"]):
        out[int(j)] = [(ev, bar(ev, vn))]
    for j, ev, vn in zip(g["alt_j"], g["alt_ev"], g["alt_vn2"]):
        out[int(j)].append((ev, bar(ev, vn)))
    return out, scale


def check_blocks(cands, scale, evals, block_of):
    """Every listed Fourier block of a computed spectrum against its
    admissible oracle spectra; returns the largest error relative to scale."""
    evals = np.asarray(evals, float)
    block_of = np.asarray(block_of)
    worst = 0.0
    for j, cs in cands.items():
        got = np.sort(evals[block_of == j])
        e = _match(got, cs)
        if e is None:
            ev, tol = cs[0]
            f = np.isfinite(ev) & np.isfinite(got)
            raise AssertionError(f"Fourier block {j}: finite {np.isfinite(got).sum()} vs "
                                 f"{np.isfinite(ev).sum()}, max |d|/tol "
                                 f"{np.max(np.abs(got[f] - ev[f]) / tol[f]) if f.any() else 0:.3e}")
        worst = max(worst, e)
    return worst / scale
