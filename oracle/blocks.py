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

from . import dense, grid


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


def generators_direct(p):
    """Generators A_k of H and S for every lattice offset k of a defect-free
    periodic problem (the first block column), without the dense matrix: V
    by the 3D grid contraction restricted to column cell 0, S and A from the
    1D quadratic forms (Sec. 2.4).  Shapes (|L|, m0, m0) in kbar order."""
    assert not p.defects and all(p.periodic[a] or p.L[a] == 1 for a in range(3))
    forms = dense.axis_forms(p)
    slab_of, slabs = grid.potential_slabs(p)
    V = dense._contract(p, [f[0] for f in forms], slab_of, slabs, col_cells=0)
    V = V.reshape(p.ncell, p.m0, p.m0)
    ks, _ = dense._index(p)
    kb = np.arange(p.ncell)
    k1 = kb // (p.L[1] * p.L[2])
    k2 = (kb // p.L[2]) % p.L[1]
    k3 = kb % p.L[2]
    sl = [forms[a][1][kk][:, :, 0, :] for a, kk in enumerate((k1, k2, k3))]
    al = [forms[a][2][kk][:, :, 0, :] for a, kk in enumerate((k1, k2, k3))]
    S = sl[0] * sl[1] * sl[2]
    A = al[0] * sl[1] * sl[2] + sl[0] * al[1] * sl[2] + sl[0] * sl[1] * al[2]
    return 0.5 * A - V, S


def fourier_block_from_generators(p, Hk, Sk, jcell, tau=None):
    """Direct DFT (explicit sum over all lattice offsets) of given generators
    at one Fourier index, and the block's eigenvalues under the dependency
    rule (block_pencil; tau defaults to null_threshold(p))."""
    L1, L2, L3 = p.L
    j1, j2, j3 = jcell
    k = np.arange(p.ncell)
    k3 = k % L3
    k2 = (k // L3) % L2
    k1 = k // (L2 * L3)
    w = np.exp(-2j * np.pi * (j1 * k1 / L1 + j2 * k2 / L2 + j3 * k3 / L3))
    Hb = np.tensordot(w, Hk, axes=(0, 0))
    Sb = np.tensordot(w, Sk, axes=(0, 0))
    if tau is None:
        tau = null_threshold(p)
    return Hb, Sb, block_pencil(Hb, Sb, tau)[0]


# ---- numerically singular overlap directions (reading G16) ----
#
# The problem is the Galerkin pencil H C = S C Lambda (Eqs. 2.4-2.5,
# Eqs. 3.11-3.12, Prop. A.1).  A Gaussian basis can be dependent to the
# rounding level of the overlap (several close exponents on one centre;
# diffuse functions on a dense lattice): along such a direction the computed
# overlap is zero or negative within its rounding, and the pencil's value
# there is not determined by the data.  Only those directions are removed.
# B[mu, nu] = sum over lattice offsets d of |S_d[mu, nu]| bounds every entry
# of every Fourier block and every block row of the lattice overlap
# (||S||_2 <= ||B||_F).  The lattice overlap is of order N_b = |L| m0, and the
# usual numerical-rank tolerance of a matrix of that order,
#     tau = N_b * eps * ||B||_F        (eps = 2^-52),
# is the cut: a direction whose overlap eigenvalue is at most tau is removed
# (per Fourier block, whose eigen-directions are the lattice overlap's; per
# cell on chains).  Where nothing lies at or below tau the pencil is solved
# exactly as stated (LAPACK).
U64 = 2.0 ** -53
EPS64 = 2.0 ** -52


def _wall_free_chain_forms(p):
    """1D mass forms s[d] (block row cell d, column cell 0) of axis 0 on a node
    line with no wall within reach of the functions (what a cell far from the
    ends of a box chain sees), for every offset d with a non-zero form."""
    rmax = np.sqrt(np.log(1.0 / p.eps_support) / np.min(p.exps))
    pe = int(np.ceil(rmax / p.h)) + 2
    reach = int(np.ceil((2 * pe) / p.n0)) + 1
    Lq = 2 * reach + 1
    q = type(p)(L=(Lq, 1, 1), periodic=(0, 0, 0), N=(Lq * p.n0 + 2 * pe, 3, 3), n0=p.n0,
                b0=p.b0, Z=p.Z, frac=p.frac, exps=p.exps, ang=p.ang, centre=p.centre, R=p.R,
                eps_support=p.eps_support)
    G = grid.basis_axis(q, 0)
    N, L, m0 = G.shape
    S1, _ = dense.fem_1d(N, q.h, False)
    Gf = G.reshape(N, L * m0)
    s = (Gf.T @ S1 @ Gf).reshape(L, m0, L, m0)
    return [s[c, :, reach, :] for c in range(L)]


def overlap_scale(p):
    """B = sum over lattice offsets of |S_offset| (m0 x m0, entrywise), from
    the 1D mass forms of the three axes (the overlap blocks are Hadamard
    products of per-axis forms, Lemma 3.4, so the sum factorises): periodic
    axis: the ring forms of the L offsets; Dirichlet axis of one cell: its
    form with itself; Dirichlet chain axis: the wall-free forms of every
    offset (the Toeplitz generators of Remark 3.2)."""
    forms = dense.axis_forms(p)
    B = np.ones((p.m0, p.m0))
    for ax in range(3):
        _, s, _ = forms[ax]
        if p.periodic[ax] or p.L[ax] == 1:
            acc = np.sum(np.abs(s[:, :, 0, :]), axis=0)
        else:
            acc = np.sum(np.abs(np.stack(_wall_free_chain_forms(p))), axis=0)
        B = B * acc
    return B


def null_threshold(p):
    """tau = N_b eps ||B||_F (see above)."""
    return p.Nb * EPS64 * float(np.linalg.norm(overlap_scale(p)))


def block_pencil(Hb, Sb, tau, flip=()):
    """Eigenpairs of one Hermitian pencil (Hb, Sb): eigenvalues ascending,
    then one +inf per removed direction; eigenvectors (m, r), Sb-orthonormal;
    r = number kept.  Directions of Sb with eigenvalue <= tau are removed:
    with none, LAPACK's generalized Hermitian eigensolver on the pencil as it
    stands; else the same on its restriction to the kept eigenvectors Q_K of
    Sb (Hr = Q_K^H Hb Q_K, Sr = Q_K^H Sb Q_K), vectors Q_K y.  `flip` lists
    indices (into the ascending eigenvalues of Sb) whose kept / removed
    decision is reversed (the variants of a direction near the cut)."""
    w, Q = np.linalg.eigh(Sb)
    keep = w > tau
    for i in flip:
        keep[i] = not keep[i]
    m = Sb.shape[0]
    if keep.all():
        ev, V = scipy.linalg.eigh(Hb, Sb)
        return ev, V, m
    Qk = Q[:, keep]
    Hr = Qk.conj().T @ Hb @ Qk
    Sr = Qk.conj().T @ Sb @ Qk
    r = Qk.shape[1]
    if r == 0:
        return np.full(m, np.inf), np.zeros((m, 0), Hb.dtype), 0
    ev, Y = scipy.linalg.eigh(0.5 * (Hr + Hr.conj().T), 0.5 * (Sr + Sr.conj().T))
    return np.concatenate([ev, np.full(m - r, np.inf)]), Qk @ Y, r


def block_eigs_rule(Hb, Sb, tau):
    """Eigenvalues of block_pencil (kept spectrum ascending, then +inf)."""
    return block_pencil(Hb, Sb, tau)[0]


def ambiguous(w, tau, band=4.0):
    """Indices of overlap eigenvalues w in (tau / band, band tau]: directions
    near the cut whose kept / removed decision rounding can flip; their
    pencil values are undetermined, and either decision is a correct reading."""
    idx = np.nonzero((w > tau / band) & (w <= tau * band))[0]
    return idx[np.argsort(np.abs(np.log(w[idx] / tau)))]   # nearest the cut first


def periodic_fourier_blocks(p, H=None, S=None):
    """(Hbar_j, Sbar_j) for every Fourier index by the direct DFT of the dense
    matrices' generators (Lemma 3.1, Eq. A.3)."""
    if H is None:
        H, S = dense.build(p)
    return (fourier_blocks(p, generators_from_dense(p, H)),
            fourier_blocks(p, generators_from_dense(p, S)))


def periodic_eigs(p, H=None, S=None, tau=None):
    """The periodic problem's spectrum through its Fourier blocks (Prop. A.1)
    under the dependency rule: (all eigenvalues sorted, +inf last; per-block
    eigenvalues (|L|, m0))."""
    Hb, Sb = periodic_fourier_blocks(p, H, S)
    if tau is None:
        tau = null_threshold(p)
    per = np.stack([block_pencil(Hb[j], Sb[j], tau)[0] for j in range(p.ncell)])
    return np.sort(per.ravel()), per


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


def periodic_eigvecs(p, H=None, S=None, tau=None):
    """Eigenpairs of a periodic problem through its Fourier blocks: each
    block's eigenpairs under the dependency rule (kept directions only),
    back-transformed to the lattice by bloch_phases.  Returns (eigenvalues
    ascending, complex eigenvectors (N_b, n) in the basis order
    a = kbar*m0 + mu, Fourier index of each); the vectors are S-orthonormal."""
    Hb, Sb = periodic_fourier_blocks(p, H, S)
    if tau is None:
        tau = null_threshold(p)
    evs, vecs, js = [], [], []
    for j in range(p.ncell):
        ev, Y, r = block_pencil(Hb[j], Sb[j], tau)
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


def cell_null_directions(p, tau=None):
    """Eigen-decomposition of the cell overlap: (eigenvalues ascending,
    eigenvectors, tau).  A cell direction v with eigenvalue <= tau spans, on
    every cell k, vectors e_k (x) v on which the chain's overlap form is at
    most tau: numerically singular directions of the lattice overlap."""
    if tau is None:
        tau = null_threshold(p)
    s, Q = np.linalg.eigh(cell_overlap(p))
    return s, Q, tau


def box_eigs(p, H=None, S=None, k=None, tau=None, vectors=False, flip=()):
    """Lowest k eigenpairs of a chain on the structured path (box, or with
    defects).  With no cell direction at or below tau: LAPACK's generalized
    symmetric eigensolver on (H, S) as they stand.  Else the cell directions
    at or below tau are removed from every cell: with Q_K the kept cell
    eigenvectors and Qb = I_L (x) Q_K, the pencil (Qb^T H Qb, Qb^T S Qb) by
    LAPACK, eigenvectors Qb y.  `flip` lists indices (into the ascending cell
    eigenvalues) whose kept / removed decision is reversed (the ambiguous
    variants of a direction near the cut).  Returns (eigenvalues, vectors or
    None, number of kept cell directions)."""
    if H is None:
        H, S = dense.build(p)
    k = k or p.k_eig
    s, Q, tau = cell_null_directions(p, tau)
    keep = s > tau
    for i in flip:
        keep[i] = not keep[i]
    if keep.all():
        ev, V = scipy.linalg.eigh(H, S, subset_by_index=[0, k - 1])
        return ev, (V if vectors else None), p.m0
    Qb = np.kron(np.eye(p.L[0]), Q[:, keep])
    Hr = Qb.T @ H @ Qb
    Sr = Qb.T @ S @ Qb
    ev, Y = scipy.linalg.eigh(0.5 * (Hr + Hr.T), 0.5 * (Sr + Sr.T), subset_by_index=[0, k - 1])
    return ev, (Qb @ Y if vectors else None), int(keep.sum())


def structured(p):
    """Box chains and problems with defects take the lowest-k structured
    solve; defect-free periodic lattices the Fourier-block route."""
    return bool(p.is_box or p.defects)


def solve(p, box_potential=None):
    """The problem's answer under the dependency rule: a periodic problem's
    whole spectrum (+inf for removed directions), a box chain's or a defect
    problem's lowest k_eig eigenvalues.  box_potential selects reading R1 or
    R2 of a box's potential (grid.potential_slabs)."""
    H, S = dense.build(p, box_potential=box_potential)
    if structured(p):
        return box_eigs(p, H, S)[0]
    return periodic_eigs(p, H, S)[0]
