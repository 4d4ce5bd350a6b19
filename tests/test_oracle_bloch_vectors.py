"""Pins of the oracle's eigenvector back-transform for periodic lattices
(Prop. A.1: the lattice pencil's eigenvectors are the Fourier blocks'
eigenvectors times the columns of the inverse DFT over the lattice index)
and of the real-space orbitals evaluated from them on the grid.

Pins: residuals and S-orthonormality against the dense matrices (the
problems are chosen so that the Fourier blocks are genuinely complex, where
a wrong sign of the phase fails); plane waves for one function per cell
against numpy's inverse FFT; Bloch's theorem for the grid orbitals (a
translation by one cell multiplies them by the phase); the grid orbital's
P1 norm equals the Galerkin norm."""
import numpy as np
import pytest

from oracle import blocks, dense
from tests import _cases


def _kept_kappa(p, S):
    """Largest condition number of the kept part of a Fourier block's
    overlap (the rounding scale of an FP64 solve on it)."""
    Sb = blocks.fourier_blocks(p, blocks.generators_from_dense(p, S))
    tau = blocks.null_threshold(p)
    k = 1.0
    for j in range(p.ncell):
        w = np.linalg.eigvalsh(Sb[j])
        w = w[w > tau]
        if len(w):
            k = max(k, w.max() / w.min())
    return k

def _problems():
    yield _cases.periodic_chain_small(L=5, n0=6, n_perp=14, m0=8, R=12)
    yield _cases.periodic_3d_small(L=(3, 2, 2), n0=4, R=8)


@pytest.mark.parametrize("case", [0, 1])
def test_block_eigenvectors_solve_the_lattice_pencil(case):
    p = list(_problems())[case]
    H, S = dense.build(p)
    Hb = blocks.fourier_blocks(p, blocks.generators_from_dense(p, H))
    assert np.max(np.abs(Hb.imag)) > 1e-3 * np.max(np.abs(Hb))      # complex blocks
    ev, U, jj = blocks.periodic_eigvecs(p, H, S)
    assert U.shape == (p.Nb, len(ev))
    R = H @ U - (S @ U) * ev[None, :]
    scale = np.linalg.norm(H, 2) * np.max(np.linalg.norm(U, axis=0))
    # Galerkin condition on the kept space (the span over j of the lattice
    # phases times the block's kept overlap directions, orthonormal columns);
    # with nothing removed that space is everything and R itself vanishes
    Sb = blocks.fourier_blocks(p, blocks.generators_from_dense(p, S))
    tau = blocks.null_threshold(p)
    W = []
    for j in range(p.ncell):
        w, Q = np.linalg.eigh(Sb[j])
        Q = Q[:, w > tau]                 # the kept overlap directions (orthonormal)
        W.append(np.kron(blocks.bloch_phases(p, j)[:, None], Q) * np.sqrt(p.ncell))
    W = np.concatenate(W, axis=1)
    assert W.shape[1] == len(ev)
    assert np.max(np.abs(W.conj().T @ R)) <= 1e-11 * scale
    if len(ev) == p.Nb:
        assert np.max(np.linalg.norm(R, axis=0)) <= 1e-11 * scale
    else:
        assert p.L[1] > 1                 # only the 3D case removes directions here
    # orthonormality to the rounding of an FP64 solve with the kept overlap:
    # about u kappa_K (the m0 = 8 recipe draws close exponents)
    G = U.conj().T @ S @ U
    assert np.max(np.abs(G - np.eye(len(ev)))) <= 1e-12 + 16 * _cases.U64 * _kept_kappa(p, S)
    # nothing removed and S well conditioned: the dense LAPACK spectrum
    w = np.linalg.eigvalsh(S)
    if len(ev) == p.Nb and w.min() > 1e-6 * w.max():
        ref = dense.eigvals(H, S)
        assert np.max(np.abs(ev - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_wrong_phase_sign_is_caught():
    """The conjugate phase (a plausible slip) does not solve the pencil on
    complex blocks: the residual check above has teeth."""
    p = next(_problems())
    H, S = dense.build(p)
    ev, U, jj = blocks.periodic_eigvecs(p, H, S)
    m0 = p.m0
    bad = []
    for c in range(len(ev)):
        f = blocks.bloch_phases(p, int(jj[c]))
        y = U[:m0, c] / f[0]
        u = np.kron(f.conj()[:, None], y[:, None])[:, 0]
        bad.append(np.linalg.norm(H @ u - ev[c] * (S @ u)))
    assert max(bad) > 1e-3 * np.linalg.norm(H, 2)


def test_m0_1_eigenvectors_are_plane_waves():
    """One function per cell: the matrices are circulant and each eigenvector
    is a column of the inverse DFT matrix (numpy.fft.ifft), up to a scalar."""
    p = _cases.single_gaussian(alpha=0.7, n0=6, R=12, L=7, periodic=True)
    H, S = dense.build(p)
    ev, U, jj = blocks.periodic_eigvecs(p, H, S)
    F = np.fft.ifft(np.eye(p.L[0]), axis=0)                    # column j: exp(+2 pi i j k / L) / L
    for c in range(len(ev)):
        col = F[:, jj[c]]
        s = np.vdot(col, U[:, c]) / np.vdot(col, col)
        assert np.max(np.abs(U[:, c] - s * col)) <= 1e-12 * np.max(np.abs(U[:, c]))


def test_orbitals_obey_blochs_theorem():
    """psi_j(x + b0 e_1) = exp(2 pi i j_1 / L_1) psi_j(x): on the grid a
    translation by one cell is a cyclic shift by n0 nodes of the periodic
    axis."""
    p = _cases.periodic_chain_small(L=5, n0=6, n_perp=14, m0=8, R=12)
    H, S = dense.build(p)
    ev, U, jj = blocks.periodic_eigvecs(p, H, S)
    L = p.L[0]
    for c in (0, 3, 11, len(ev) - 1):
        psi = blocks.orbital_on_grid(p, U[:, c])
        shifted = np.roll(psi, p.n0, axis=0)                     # shifted[i] = psi[i - n0]
        ph = np.exp(2j * np.pi * int(jj[c]) / L)
        assert np.max(np.abs(psi - ph * shifted)) <= 1e-12 * np.max(np.abs(psi))


def test_orbital_p1_norm_is_the_galerkin_norm():
    """The P1 interpolant of the grid orbital has squared L2 norm
    psi^H (S1 x S1 x S1) psi, applied here as a 3D stencil on the grid
    function; for an S-normalised eigenvector it is 1 (to the rounding of
    the kept overlap's condition number)."""
    p = _cases.periodic_3d_small(L=(3, 2, 2), n0=4, R=8)
    H, S = dense.build(p)
    ev, U, jj = blocks.periodic_eigvecs(p, H, S)
    tol = 1e-12 + 16 * _cases.U64 * _kept_kappa(p, S)
    S1 = [dense.fem_1d(p.N[a], p.h, bool(p.periodic[a]))[0] for a in range(3)]
    for c in (0, 5, len(ev) // 2):
        psi = blocks.orbital_on_grid(p, U[:, c])
        t = np.einsum("ia,ajk->ijk", S1[0], psi)
        t = np.einsum("jb,ibk->ijk", S1[1], t)
        t = np.einsum("kc,ijc->ijk", S1[2], t)
        assert abs(np.vdot(psi, t) - 1.0) <= tol
