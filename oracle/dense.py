"""Dense N_b x N_b core Hamiltonian and mass matrices, and their eigensolve.

Basis functions are indexed a = kbar*m0 + mu with kbar = (k1*L2 + k2)*L3 + k3
(k3 fastest).  Entries (Sec. 2.1, Eqs. 2.4-2.5; Sec. 2.3 Lemma 2.1;
Sec. 2.4 Eqs. 2.15-2.17):

  S_ab = <g_a, (S1 x S1 x S1) g_b>,
  A_ab = <g_a, (A1 x S1 x S1 + S1 x A1 x S1 + S1 x S1 x A1) g_b>,
  V_ab = sum_i g_a(i) g_b(i) P(i),
  H    = A/2 - V,     H C = S C Lambda.

S1 = (h/6) tridiag(1,4,1) and A1 = (1/h) tridiag(-1,2,-1) are the 1D P1
mass and stiffness matrices (cyclic on a periodic axis).  For a separable
g_a the Kronecker quadratic forms are products of 1D quadratic forms (the
definition of the Kronecker product), which is how S and A are formed.
V is formed by contracting the materialised 3D potential tensor against
the 3D products of basis functions, summing over i3, then i2, then i1.
"""
import numpy as np
import scipy.linalg

from . import grid


def fem_1d(N, h, periodic):
    """Dense 1D P1 mass and stiffness matrices (Sec. 2.4)."""
    S1 = np.zeros((N, N))
    A1 = np.zeros((N, N))
    idx = np.arange(N)
    S1[idx, idx] = 4.0 * h / 6.0
    A1[idx, idx] = 2.0 / h
    for s in (-1, 1):
        j = idx + s
        ok = (j >= 0) & (j < N)
        if periodic:
            j = j % N
            ok = np.ones(N, bool)
        S1[idx[ok], j[ok]] += h / 6.0
        A1[idx[ok], j[ok]] += -1.0 / h
    return S1, A1


def _index(p):
    """Per-axis (cell, mu) pair for every basis function."""
    L1, L2, L3 = p.L
    m0 = p.m0
    a = np.arange(p.Nb)
    mu = a % m0
    kb = a // m0
    k3 = kb % L3
    k2 = (kb // L3) % L2
    k1 = kb // (L2 * L3)
    return (k1, k2, k3), mu


def axis_forms(p):
    """Per axis: G, and the 1D quadratic forms s_l[(k,mu),(m,nu)], a_l."""
    out = []
    for ax in range(3):
        G = grid.basis_axis(p, ax)
        N, L, m0 = G.shape
        S1, A1 = fem_1d(N, p.h, bool(p.periodic[ax]))
        Gf = G.reshape(N, L * m0)
        s = Gf.T @ S1 @ Gf
        a = Gf.T @ A1 @ Gf
        out.append((G, s.reshape(L, m0, L, m0), a.reshape(L, m0, L, m0)))
    return out


def mass_kinetic(p, forms=None):
    """Dense S and A (products of 1D forms over the three axes)."""
    forms = forms or axis_forms(p)
    ks, mu = _index(p)
    sl, al = [], []
    for ax in range(3):
        _, s, a = forms[ax]
        kk = ks[ax]
        sl.append(s[kk[:, None], mu[:, None], kk[None, :], mu[None, :]])
        al.append(a[kk[:, None], mu[:, None], kk[None, :], mu[None, :]])
    S = sl[0] * sl[1] * sl[2]
    A = al[0] * sl[1] * sl[2] + sl[0] * al[1] * sl[2] + sl[0] * sl[1] * al[2]
    return S, A


def _contract(p, Gs, slab_of, slabs, col_cells=None):
    """V[(k,mu),(m,nu)] = sum_{i1,i2,i3} G1 G1 G2 G2 G3 G3 P.  With
    col_cells = 0 only the column cell (0,0,0) is formed (first block
    column)."""
    G1, G2, G3 = Gs
    L1, L2, L3 = p.L
    m0 = p.m0
    c1 = G1 if col_cells is None else G1[:, :1]
    c2 = G2 if col_cells is None else G2[:, :1]
    c3 = G3 if col_cells is None else G3[:, :1]
    nslab = slabs.shape[0]
    # W3[s, i2, k3, m3, mu, nu] = sum_i3 P_s[i2,i3] G3[i3,k3,mu] G3[i3,m3,nu]
    GG3 = np.einsum("ikm,ijn->ikjmn", G3, c3)                    # (N3,L3,M3,m0,m0)
    W3 = np.tensordot(slabs, GG3, axes=(2, 0))                    # (s,N2,L3,M3,m0,m0)
    GG2 = np.einsum("ikm,ijn->ikjmn", G2, c2)                    # (N2,L2,M2,m0,m0)
    # W2[s, k2, m2, k3, m3, mu, nu]
    W2 = np.einsum("iabmn,siczmn->sabczmn", GG2, W3, optimize=True)
    # GG1[s, k1, mu, m1, nu] = sum over the axis-0 nodes i1 of slab s of G1 G1
    GG1 = np.zeros((nslab, L1, m0, c1.shape[1], m0))
    for s in range(nslab):
        rows = np.nonzero(slab_of == s)[0]
        GG1[s] = np.einsum("ikm,ijn->kmjn", G1[rows], c1[rows])
    V = np.einsum("skmjn,sabczmn->kacmjbzn", GG1, W2, optimize=True)
    return V


def box_reading(p, box_potential=None):
    """The box-potential reading of problem p: the argument when given, else
    the problem's own field (box_potential 1 = "lattice_sum", reading R2;
    0 = "replicated", reading R1)."""
    if box_potential is not None:
        return box_potential
    return "lattice_sum" if getattr(p, "box_potential", 0) == 1 else "replicated"


def potential_matrix(p, forms=None, slab=None, box_potential=None):
    """Dense V; box_potential selects reading R1 ("replicated") or R2
    ("lattice_sum") of the box potential (grid.potential_slabs)."""
    box_potential = box_reading(p, box_potential)
    forms = forms or axis_forms(p)
    slab_of, slabs = slab if slab is not None else grid.potential_slabs(p, box_potential)
    V = _contract(p, [f[0] for f in forms], slab_of, slabs)
    return V.reshape(p.Nb, p.Nb)


def defect_matrix(p, forms=None):
    """Sum over defects of (newZ - Z_nu) <g_a g_b, P_single>, with P_single
    the rank-R kernel of the one substituted nucleus (no window, no
    replication, minimum image on periodic axes).  The paper only motivates
    defects (Sec. 1, Sec. 2.3 (B)); this model of a vacancy or substitution
    as a change of one nucleus' charge is the reading taken here.
    Pins: the single-molecule charge change, every cell of an odd periodic
    chain substituted (= a charge change of the window sum), every nucleus
    of a box vacated (= minus the box's lattice-sum potential)."""
    forms = forms or axis_forms(p)
    D = np.zeros((p.Nb, p.Nb))
    if not p.defects:
        return D
    c = np.asarray(p.sinc_c, float)
    Gs = [f[0] for f in forms]
    for d in p.defects:
        nu = d.nucleus
        dz = d.newZ - p.Z[nu]
        e = []
        for ax in range(3):
            _, X0, _ = grid.axis_nodes(p, ax)
            pos = X0 + (d.cell[ax] + p.frac[nu, ax]) * p.b0
            e.append(grid.single_nucleus_axis(p, ax, pos))
        # slabs: one per i1 (no replication) -> contract axis by axis on the fly
        coef = dz * c[None, :] * e[0].T                              # (N1, R)
        B = e[1][:, :, None] * e[2][:, None, :]                      # (R, N2, N3)
        slabs = np.tensordot(coef, B, axes=(1, 0))                   # (N1, N2, N3)
        V = _contract(p, Gs, np.arange(p.N[0]), slabs)
        D += V.reshape(p.Nb, p.Nb)
    return D


def chain_matrices(p, box_potential=None):
    """Dense H and S of a chain (L2 = L3 = 1, no defects) with the same
    entries as build(), for chains too long for build()'s cell-pair tensors:
    the sum over the 3D grid of V_ab = sum_i g_a(i) g_b(i) P(i) is grouped
    by basis-function pair (mu, nu) -- w_{mu nu}(i1) = sum_{i2, i3} P(i)
    g2_mu g2_nu g3_mu g3_nu (the transverse axes carry one cell), then
    V[(k, mu), (m, nu)] = sum_{i1} G1[i1, k, mu] G1[i1, m, nu] w_{mu nu}(i1) --
    and the 1D quadratic forms of axis 0 apply the P1 stencils to the nodal
    vectors directly (Sec. 2.4; Lemma 2.1)."""
    assert p.L[1] == 1 and p.L[2] == 1 and not p.defects
    L, m0, h = p.L[0], p.m0, p.h
    G1 = grid.basis_axis(p, 0)                                     # (N1, L, m0)
    N1 = G1.shape[0]
    Gf = G1.reshape(N1, L * m0)
    per = bool(p.periodic[0])

    def shift(u, s):                                              # u[i - s] (zero / wrap)
        if per:
            return np.roll(u, s, axis=0)
        w = np.zeros_like(u)
        if s == 1:
            w[1:] = u[:-1]
        else:
            w[:-1] = u[1:]
        return w
    s0 = (Gf.T @ ((h / 6.0) * (4.0 * Gf + shift(Gf, 1) + shift(Gf, -1)))).reshape(L, m0, L, m0)
    a0 = (Gf.T @ ((1.0 / h) * (2.0 * Gf - shift(Gf, 1) - shift(Gf, -1)))).reshape(L, m0, L, m0)
    tr = []
    for ax in (1, 2):
        G = grid.basis_axis(p, ax)[:, 0, :]
        S1, A1 = fem_1d(p.N[ax], h, bool(p.periodic[ax]))
        tr.append((G, G.T @ S1 @ G, G.T @ A1 @ G))
    (G2, s1, a1), (G3, s2, a2) = tr
    S = s0 * (s1 * s2)[None, :, None, :]
    A = a0 * (s1 * s2)[None, :, None, :] + s0 * (a1 * s2 + s1 * a2)[None, :, None, :]
    slab_of, slabs = grid.potential_slabs(p, box_reading(p, box_potential))
    GG3 = G3[:, :, None] * G3[:, None, :]                         # (N3, mu, nu)
    GG2 = G2[:, :, None] * G2[:, None, :]
    W2 = np.zeros((slabs.shape[0], m0, m0))
    for s in range(slabs.shape[0]):
        W3 = np.tensordot(slabs[s], GG3, axes=(1, 0))             # (N2, mu, nu)
        W2[s] = np.einsum("iab,iab->ab", GG2, W3)
    w = W2[slab_of]                                               # (N1, mu, nu)
    V = np.zeros((L, m0, L, m0))
    for mu in range(m0):
        for nu in range(m0):
            V[:, mu, :, nu] = G1[:, :, mu].T @ (w[:, mu, nu, None] * G1[:, :, nu])
    n = L * m0
    H = (0.5 * A - V).reshape(n, n)
    return H, S.reshape(n, n)


def build(p, with_parts=False, box_potential=None):
    """Dense (H, S) of problem p (and optionally A, V)."""
    forms = axis_forms(p)
    S, A = mass_kinetic(p, forms)
    V = potential_matrix(p, forms, box_potential=box_potential)
    if p.defects:
        V = V + defect_matrix(p, forms)
    H = 0.5 * A - V
    if with_parts:
        return H, S, A, V
    return H, S


def eigvals(H, S, k=None):
    """Generalized symmetric-definite eigenvalues, ascending (LAPACK)."""
    if k is None:
        return scipy.linalg.eigh(H, S, eigvals_only=True)
    return scipy.linalg.eigh(H, S, eigvals_only=True, subset_by_index=[0, k - 1])


def solve(p, box_potential="replicated"):
    H, S = build(p, box_potential=box_potential)
    return eigvals(H, S, p.k_eig if (p.k_eig and p.is_box) else None)
