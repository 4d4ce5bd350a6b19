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


def generator_block(p, kcell, forms=None, slab=None, mcell=(0, 0, 0)):
    """One block H[(k, .), (m, .)] (and S) by the plain 3D contraction,
    without building the dense matrix: V[mu,nu] = sum_i G1[i1,k1,mu]
    G1[i1,m1,nu] G2.. G3.. P(i), S and A from the 1D quadratic forms.  With
    m = 0 it is the generator A_k of a periodic problem.  For problems too
    large for the dense route."""
    from . import grid
    slab_of, slabs = slab if slab is not None else grid.potential_slabs(p)
    k1, k2, k3 = kcell
    m1, m2, m3 = mcell
    if forms is None:
        # only the two cells of each axis: 1D factors and 1D quadratic forms
        # with the P1 stencils applied directly (Sec. 2.4)
        one = []
        for ax, (ka, ma) in enumerate(((k1, m1), (k2, m2), (k3, m3))):
            G = grid.basis_axis(p, ax, cells=[ka, ma])
            gk, gm = G[:, 0, :], G[:, 1, :]
            h, per = p.h, bool(p.periodic[ax])
            def nb(u, s):
                if per:
                    return np.roll(u, s, axis=0)
                w = np.zeros_like(u)
                if s == 1:
                    w[1:] = u[:-1]
                else:
                    w[:-1] = u[1:]
                return w
            S1g = (h / 6.0) * (4 * gm + nb(gm, 1) + nb(gm, -1))
            A1g = (1.0 / h) * (2 * gm - nb(gm, 1) - nb(gm, -1))
            one.append((gk, gm, gk.T @ S1g, gk.T @ A1g))
        (gk1, gm1, sv1, av1), (gk2, gm2, sv2, av2), (gk3, gm3, sv3, av3) = one
        g3 = gk3[:, :, None] * gm3[:, None, :]
        g2 = gk2[:, :, None] * gm2[:, None, :]
        g1 = gk1[:, :, None] * gm1[:, None, :]
    else:
        (G1, s1, a1), (G2, s2, a2), (G3, s3, a3) = forms
        g3 = G3[:, k3, :][:, :, None] * G3[:, m3, :][:, None, :]         # (N3, mu, nu)
        g2 = G2[:, k2, :][:, :, None] * G2[:, m2, :][:, None, :]
        g1 = G1[:, k1, :][:, :, None] * G1[:, m1, :][:, None, :]
        sv1, av1 = s1[k1, :, m1, :], a1[k1, :, m1, :]
        sv2, av2 = s2[k2, :, m2, :], a2[k2, :, m2, :]
        sv3, av3 = s3[k3, :, m3, :], a3[k3, :, m3, :]
    W3 = np.tensordot(slabs, g3, axes=(2, 0))                         # (s, N2, mu, nu)
    W2 = np.einsum("iab,siab->sab", g2, W3)                           # (s, mu, nu)
    V = np.zeros((p.m0, p.m0))
    for s in range(slabs.shape[0]):
        rows = np.nonzero(slab_of == s)[0]
        V += np.einsum("iab->ab", g1[rows]) * W2[s]
    S = sv1 * sv2 * sv3
    A = av1 * sv2 * sv3 + sv1 * av2 * sv3 + sv1 * sv2 * av3
    return 0.5 * A - V, S


def fourier_block_from_generators(p, Hk, Sk, jcell):
    """Direct DFT (explicit sum over all lattice offsets) of given generators
    at one Fourier index, and the block's eigenvalues after canonical
    orthogonalisation (canonical_eigs)."""
    L1, L2, L3 = p.L
    j1, j2, j3 = jcell
    k = np.arange(p.ncell)
    k3 = k % L3
    k2 = (k // L3) % L2
    k1 = k // (L2 * L3)
    w = np.exp(-2j * np.pi * (j1 * k1 / L1 + j2 * k2 / L2 + j3 * k3 / L3))
    Hb = np.tensordot(w, Hk, axes=(0, 0))
    Sb = np.tensordot(w, Sk, axes=(0, 0))
    return Hb, Sb, canonical_eigs(Hb, Sb)


# Canonical (Loewdin) orthogonalisation.  A Galerkin basis of Gaussians can
# be numerically dependent (diffuse functions on a dense lattice; several
# close exponents on one centre): the overlap then has eigenvalues at the
# rounding level of its own assembly, and the pencil's eigenvalues in those
# directions are not determined by the data.  The reading used here removes
# from the variational space every eigen-direction of the overlap whose
# eigenvalue is at most CANON_TAU times the largest eigenvalue of the same
# matrix; on a full-rank, well-conditioned basis it is an exact change of
# basis and changes nothing.
CANON_TAU = 1e-8


def lowdin_basis(S, tau=CANON_TAU):
    """X = Q_K diag(s_K)^-1/2 for the eigen-directions of the Hermitian S with
    s > tau * max(s) (eigendecomposition by LAPACK); returns (X, s)."""
    s, Q = np.linalg.eigh(S)
    keep = s > tau * s.max()
    return Q[:, keep] / np.sqrt(s[keep]), s


def canonical(Hb, Sb, tau=CANON_TAU):
    """Eigenpairs of a Hermitian pencil block on the kept directions:
    C = X^H H X (X from lowdin_basis), C y = lambda y, eigenvectors X y in
    the original coordinates.  Returns (eigenvalues ascending followed by one
    +inf per removed direction, eigenvectors (m, r), condition number of the
    kept part of S)."""
    X, s = lowdin_basis(Sb, tau)
    C = X.conj().T @ Hb @ X
    ev, Y = np.linalg.eigh(0.5 * (C + C.conj().T))
    r = X.shape[1]
    kept = s[s > tau * s.max()]
    kappa = float(kept.max() / kept.min()) if r else 1.0
    return np.concatenate([ev, np.full(Sb.shape[0] - r, np.inf)]), X @ Y, kappa


def canonical_eigs(Hb, Sb, tau=CANON_TAU):
    """Eigenvalues of canonical(): the kept spectrum ascending, then +inf."""
    return canonical(Hb, Sb, tau)[0]


def periodic_eigs(p, H=None, S=None, tau=CANON_TAU):
    """The periodic problem's spectrum under canonical orthogonalisation per
    Fourier block (Prop. A.1): (all eigenvalues sorted, +inf last; per-block
    eigenvalues (|L|, m0); per-block kept-overlap condition numbers)."""
    if H is None:
        H, S = dense.build(p)
    Hb = fourier_blocks(p, generators_from_dense(p, H))
    Sb = fourier_blocks(p, generators_from_dense(p, S))
    per, kap = [], []
    for j in range(p.ncell):
        ev, _, kappa = canonical(Hb[j], Sb[j], tau)
        per.append(ev)
        kap.append(kappa)
    per = np.stack(per)
    return np.sort(per.ravel()), per, np.array(kap)


def bloch_phases(p, jbar):
    """Lattice factor of the back-transform at linear Fourier index jbar:
    f[kbar] = prod_l exp(+2 pi i j_l k_l / L_l) / sqrt(|L|).  With
    H = sum_k pi^k (x) A_k and Abar_j = sum_k omega^{jk} A_k,
    omega = exp(-2 pi i / L) (Eq. A.3), the vector u[k] = f[k] y gives
    (H u)[k] = f[k] Abar_j y block by block, so an eigenpair of the block
    pencil is one of the lattice pencil (Prop. A.1; the columns of the
    inverse DFT, U = (F^* (x) I) Ubar)."""
    L1, L2, L3 = p.L
    j3 = jbar % L3
    j2 = (jbar // L3) % L2
    j1 = jbar // (L2 * L3)
    k = np.arange(p.ncell)
    k3 = k % L3
    k2 = (k // L3) % L2
    k1 = k // (L2 * L3)
    ph = np.exp(2j * np.pi * (j1 * k1 / L1 + j2 * k2 / L2 + j3 * k3 / L3))
    return ph / np.sqrt(p.ncell)


def periodic_eigvecs(p, H=None, S=None, tau=CANON_TAU):
    """Eigenpairs of a periodic problem through its Fourier blocks: each
    block's canonical eigenpairs (kept directions only), back-transformed to
    the lattice by bloch_phases.  Returns (eigenvalues ascending, complex
    eigenvectors (N_b, n) in the basis order a = kbar*m0 + mu, Fourier index
    of each); the vectors are S-orthonormal."""
    if H is None:
        H, S = dense.build(p)
    Hb = fourier_blocks(p, generators_from_dense(p, H))
    Sb = fourier_blocks(p, generators_from_dense(p, S))
    evs, vecs, js = [], [], []
    for j in range(p.ncell):
        ev, Y, _ = canonical(Hb[j], Sb[j], tau)
        r = Y.shape[1]
        f = bloch_phases(p, j)
        evs.append(ev[:r])
        vecs.append(np.kron(f[:, None], Y))          # u[(k, mu), c] = f[k] Y[mu, c]
        js.append(np.full(r, j))
    ev = np.concatenate(evs)
    U = np.concatenate(vecs, axis=1)
    jj = np.concatenate(js)
    order = np.lexsort((jj, ev))
    return ev[order], U[:, order], jj[order]


def orbital_on_grid(p, u):
    """Real-space orbital psi(i1, i2, i3) = sum_{k, mu} u[(k, mu)]
    prod_l g_l(k_l, mu)(x_{i_l}) at the grid nodes (the separable GTO factors
    of Sec. 2.4; the P1 interpolant of psi is the Galerkin function)."""
    from . import grid
    m0 = p.m0
    L1, L2, L3 = p.L
    Gs = [grid.basis_axis(p, a) for a in range(3)]
    C = np.asarray(u).reshape(L1, L2, L3, m0)
    # contract one axis at a time: the cell index of each axis and mu
    T = np.einsum("iam,abcm->ibcm", Gs[0], C)                # (N1, L2, L3, m0)
    T = np.einsum("jbm,ibcm->ijcm", Gs[1], T)                # (N1, N2, L3, m0)
    return np.einsum("kcm,ijcm->ijk", Gs[2], T)              # (N1, N2, N3)


def cell_overlap(p):
    """Overlap of one cell's basis with itself as the structured (chain)
    solve sees it: for a box chain the interior cell of the Toeplitz
    generator T_S[0] (Remark 3.2) -- axis 0 on a node line long enough that no
    wall reaches the cell's functions; for a periodic chain the periodic
    diagonal block A_0 of S on its own ring.  The single-cell transverse axes
    as they are.  Product of the 1D mass forms."""
    if p.periodic[0]:
        q = p
    else:
        rmax = np.sqrt(np.log(1.0 / p.eps_support) / np.min(p.exps))
        pe = int(np.ceil(rmax / p.h)) + 2
        q = type(p)(L=(1, p.L[1], p.L[2]), periodic=(0, p.periodic[1], p.periodic[2]),
                    N=(p.n0 + 2 * pe, p.N[1], p.N[2]), n0=p.n0, b0=p.b0, Z=p.Z, frac=p.frac,
                    exps=p.exps, ang=p.ang, centre=p.centre, R=p.R, eps_support=p.eps_support)
    (_, s0, _), (_, s1, _), (_, s2, _) = dense.axis_forms(q)
    return s0[0, :, 0, :] * s1[0, :, 0, :] * s2[0, :, 0, :]


def box_basis(p, tau=CANON_TAU):
    """Block-diagonal change of basis of a chain on the structured path: the
    canonical cell basis Xc = lowdin_basis(cell_overlap) on every cell,
    I_L (x) Xc."""
    Xc, _ = lowdin_basis(cell_overlap(p), tau)
    return np.kron(np.eye(p.L[0]), Xc), Xc


def box_eigs(p, H=None, S=None, k=None, tau=CANON_TAU, vectors=False):
    """Lowest k eigenpairs of a chain on the structured path (box, or with
    defects) in the canonical cell basis:
    (Xb^T H Xb) y = lambda (Xb^T S Xb) y by LAPACK, eigenvectors Xb y in the
    original coordinates.  Returns (eigenvalues, vectors or None, reduced S)."""
    if H is None:
        H, S = dense.build(p)
    k = k or p.k_eig
    Xb, _ = box_basis(p, tau)
    Hr = Xb.T @ H @ Xb
    Sr = Xb.T @ S @ Xb
    ev, Y = scipy.linalg.eigh(Hr, Sr, subset_by_index=[0, k - 1])
    return ev, (Xb @ Y if vectors else None), Sr


def structured(p):
    """Box chains and problems with defects take the lowest-k structured
    solve; defect-free periodic lattices the Fourier-block route."""
    return bool(p.is_box or p.defects)


def solve(p, box_potential="replicated"):
    """The problem's answer under the canonical-orthogonalisation reading:
    a periodic problem's whole spectrum (+inf for removed directions), a box
    chain's or a defect problem's lowest k_eig eigenvalues.  box_potential
    selects reading R1 or R2 of a box's potential (grid.potential_slabs)."""
    H, S = dense.build(p, box_potential=box_potential)
    if structured(p):
        return box_eigs(p, H, S)[0]
    return periodic_eigs(p, H, S)[0]
