"""Block structure of the dense matrices, and the direct Fourier-block route.

Conventions (Appendix A.1, Prop. A.1; Sec. 3.1, Lemma 3.1):
  * generator A_k = block (row cell k, column cell 0) of H, so that the
    periodic matrix is sum_k pi^k (x) A_k with pi the downward cyclic shift;
  * Fourier block  Abar_j = sum_k prod_l omega_{L_l}^{j_l k_l} A_k,
    omega_L = exp(-2 pi i / L), no 1/sqrt(L) factor (Eq. A.3, Eq. 3.1);
  * the spectrum of the periodic problem is the union over j of the
    spectra of the m0 x m0 pencils (Hbar_j, Sbar_j) (Prop. A.1, Eq. 3.12).
Box chains (Remark 3.2, Sec. 2.3 defect split): T_d = block (k + d, k) of
an interior cell; the dense box matrix is the reference for the embedded
FFT matvec.
"""
import numpy as np
import scipy.linalg

from . import dense


def generators_from_dense(p, M):
    """A_k (k = 0..|L|-1 in kbar order) = M[(k, .), (0, .)], shape (|L|, m0, m0)."""
    m0 = p.m0
    return M[:, :m0].reshape(p.ncell, m0, m0).copy()


def fourier_blocks(p, Ak):
    """Direct DFT over the three lattice indices (explicit sums, no FFT)."""
    L1, L2, L3 = p.L
    m0 = p.m0
    A = Ak.reshape(L1, L2, L3, m0, m0)
    out = np.zeros((L1, L2, L3, m0, m0), complex)
    k1 = np.arange(L1)
    k2 = np.arange(L2)
    k3 = np.arange(L3)
    for j1 in range(L1):
        w1 = np.exp(-2j * np.pi * j1 * k1 / L1)
        for j2 in range(L2):
            w2 = np.exp(-2j * np.pi * j2 * k2 / L2)
            for j3 in range(L3):
                w3 = np.exp(-2j * np.pi * j3 * k3 / L3)
                w = w1[:, None, None] * w2[None, :, None] * w3[None, None, :]
                out[j1, j2, j3] = np.tensordot(w, A, axes=([0, 1, 2], [0, 1, 2]))
    return out.reshape(p.ncell, m0, m0)


def block_eigs(Hb, Sb):
    """Per-block generalized Hermitian eigenvalues (|L|, m0), ascending."""
    return np.stack([scipy.linalg.eigh(Hb[j], Sb[j], eigvals_only=True)
                     for j in range(Hb.shape[0])])


def circulant_route(p, H=None, S=None):
    """Fourier-block route of the periodic problem from the oracle's own
    generators; returns (sorted eigenvalues, per-block eigenvalues)."""
    if H is None:
        H, S = dense.build(p)
    Hk = generators_from_dense(p, H)
    Sk = generators_from_dense(p, S)
    ev = block_eigs(fourier_blocks(p, Hk), fourier_blocks(p, Sk))
    return np.sort(ev.ravel()), ev


def matvec(M, x):
    """Reference y = M x for the structured matvec (dense product)."""
    return M @ x
