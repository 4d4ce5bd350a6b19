"""Pins of the CPU oracle against closed forms, brute force, library
routines and invariants (none of them re-type the oracle's formulas)."""
import math

import numpy as np
import pytest
import scipy.integrate

import lattice_inputs as li
from oracle import blocks, closed_forms as cf, dense, grid, sinc
from tests import _cases


# ---------------- Eq. 2.7: the R-term rule for 1/z ----------------

def test_sinc_rule_converges_in_R():
    errs = [sinc.sinc_table(R, 1e-3, 1e2)[2] for R in (12, 20, 28, 36)]
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < errs[0] / 100
    # independent check of the reported error at off-grid points
    t, c, e = sinc.sinc_table(32, 1e-3, 1e2)
    z = np.exp(np.random.default_rng(1).uniform(np.log(1e-3), np.log(1e2), 500))
    approx = np.exp(-(z[:, None] * t[None, :]) ** 2) @ c
    assert np.max(np.abs(approx * z - 1)) < 2 * e + 1e-12


# ---------------- closed-form cell integral of a Gaussian ----------------

@pytest.mark.parametrize("t,lo,hi", [(0.3, -1.0, 0.5), (5.0, 2.0, 2.1), (5.0, -2.1, -2.0),
                                     (40.0, -0.01, 0.02), (0.01, 100.0, 100.5), (3.0, 4.0, 4.2)])
def test_gauss_cell_integral_vs_quad(t, lo, hi):
    ref, _ = scipy.integrate.quad(lambda s: math.exp(-(t * s) ** 2), lo, hi, epsabs=0,
                                  epsrel=1e-13)
    got = float(grid.gauss_cell_integral(np.float64(t), np.float64(lo), np.float64(hi)))
    assert abs(got - ref) <= 1e-13 * abs(ref) + 1e-300


def test_prism_formula_vs_quadrature():
    # a cell away from the origin: plain adaptive cubature
    lo, hi = (0.3, -0.2, 0.5), (0.7, 0.4, 0.9)
    ref, _ = scipy.integrate.tplquad(lambda z, y, x: 1 / math.sqrt(x * x + y * y + z * z),
                                     lo[0], hi[0], lo[1], hi[1], lo[2], hi[2], epsabs=1e-12)
    assert abs(cf.cell_integral_inv_r(lo, hi) - ref) < 1e-9
    # a cube centred on the singularity: 8 corner cubes by symmetry, and
    # int_{[0,1]^3} 1/r in spherical shells of the cube (1D quadrature)
    full = cf.cell_integral_inv_r((-0.5,) * 3, (0.5,) * 3)
    unit = cf.cell_integral_inv_r((0.0,) * 3, (1.0,) * 3)
    assert abs(full - 8 * unit / 4.0) < 1e-12          # scaling: int over [0,a]^3 ~ a^2
    ref, _ = scipy.integrate.tplquad(lambda z, y, x: 1 / math.sqrt(x * x + y * y + z * z + 1e-300),
                                     0, 1, 0, 1, 0, 1, epsabs=1e-9)
    assert abs(unit - ref) < 1e-6


def test_projected_kernel_vs_exact_prism():
    """Eqs. 2.6-2.7: the rank-R P0 tensor of one nucleus approaches the exact
    cell integrals of 1/|x|, faster for larger R."""
    errs = []
    for R in (16, 32):
        p = _cases.single_gaussian(alpha=1.0, n0=8, box=6.0, R=R)
        so, slabs = grid.potential_slabs(p)
        P = slabs[so]
        x, X0, _ = grid.axis_nodes(p, 0)
        a = X0 + 0.5 * p.b0
        h = p.h
        rng = np.random.default_rng(2)
        idx = [tuple(rng.integers(0, p.N[0], 3)) for _ in range(40)]
        idx += [tuple([int(np.argmin(abs(x - a)))] * 3)]   # the singular cell
        e = 0.0
        for i in idx:
            lo = [x[i[d]] - h / 2 - a for d in range(3)]
            hi = [x[i[d]] + h / 2 - a for d in range(3)]
            ex = cf.cell_integral_inv_r(lo, hi)
            e = max(e, abs(P[i] - ex) / ex)
        errs.append(e)
    assert errs[1] < errs[0] / 5
    assert errs[1] < 5e-3


def test_potential_product_of_window_sums_equals_3d_window():
    """Eq. 2.13 (window sums inside each axis factor) equals the explicit sum
    over the 3D window of lattice cells (brute force, tiny 3D lattice)."""
    p = _cases.periodic_3d_small(L=(3, 2, 4), n0=4, R=8)
    so, slabs = grid.potential_slabs(p)
    P = grid.potential_full_window(p)
    assert np.max(np.abs(slabs[so] - P)) <= 1e-13 * np.max(np.abs(P))


# ---------------- Galerkin matrices vs brute force on the 3D grid ----------------

def _phi3d(p):
    Gs = [grid.basis_axis(p, a) for a in range(3)]
    ks, mu = dense._index(p)
    return np.stack([Gs[0][:, ks[0][a], mu[a]][:, None, None] *
                     Gs[1][:, ks[1][a], mu[a]][None, :, None] *
                     Gs[2][:, ks[2][a], mu[a]][None, None, :] for a in range(p.Nb)])


def _stencil(u, ax, per, w_c, w_n):
    """Apply w_c*u_i + w_n*(u_{i-1} + u_{i+1}) along ax (zero outside for Dirichlet)."""
    out = w_c * u
    for s in (-1, 1):
        if per:
            out = out + w_n * np.roll(u, s, axis=ax)
        else:
            sh = np.zeros_like(u)
            src = [slice(None)] * 3
            dst = [slice(None)] * 3
            if s == 1:
                src[ax], dst[ax] = slice(0, -1), slice(1, None)
            else:
                src[ax], dst[ax] = slice(1, None), slice(0, -1)
            sh[tuple(dst)] = u[tuple(src)]
            out = out + w_n * sh
    return out


@pytest.mark.parametrize("case", ["periodic", "box"])
def test_mass_kinetic_potential_vs_3d_brute_force(case):
    if case == "periodic":
        p = _cases.periodic_3d_small(L=(2, 1, 2), n0=6, R=8)
    else:
        p = _cases.box_chain_small(L=3, n0=4, pad=3, n_perp=10, R=8)
    H, S, A, V = dense.build(p, with_parts=True)
    phi = _phi3d(p)
    h = p.h
    per = [bool(x) for x in p.periodic]
    S3 = phi.copy()
    for ax in range(3):
        S3 = np.stack([_stencil(f, ax, per[ax], 4 * h / 6, h / 6) for f in S3])
    Sb = np.einsum("aijk,bijk->ab", phi, S3)
    Ab = 0
    for pax in range(3):
        T = phi.copy()
        for ax in range(3):
            if ax == pax:
                T = np.stack([_stencil(f, ax, per[ax], 2 / h, -1 / h) for f in T])
            else:
                T = np.stack([_stencil(f, ax, per[ax], 4 * h / 6, h / 6) for f in T])
        Ab = Ab + np.einsum("aijk,bijk->ab", phi, T)
    so, slabs = grid.potential_slabs(p)
    P = grid.potential_full_window(p)
    Vb = np.einsum("aijk,bijk,ijk->ab", phi, phi, P)
    for M, B in ((S, Sb), (A, Ab), (V, Vb)):
        assert np.max(np.abs(M - B)) <= 1e-12 * np.max(np.abs(B))


# ---------------- grid quantities approach the continuum closed forms ----------------

def test_overlap_kinetic_converge_to_closed_forms():
    """s and p GTOs pairs, two centres on a periodic-free axis: the 1D P1
    mass/stiffness forms approach the analytic integrals as O(h^2)."""
    errs = []
    for n0 in (8, 16, 32):
        p = li.Problem(L=(2, 1, 1), periodic=(0, 0, 0), N=(2 * n0 + 2 * int(8 * n0 / 2), n0, n0),
                       n0=n0, b0=2.0, Z=np.array([1.0]), frac=np.array([[0.3, 0.5, 0.5]]),
                       exps=np.array([0.7, 1.3]), ang=np.array([0, 1]), centre=np.array([0, 0]),
                       R=8)
        forms = dense.axis_forms(p)
        _, s, a = forms[0]
        x, X0, _ = grid.axis_nodes(p, 0)
        e = 0.0
        for (k, mu), (m, nu) in [((0, 0), (1, 0)), ((0, 1), (1, 0)), ((0, 1), (1, 1)),
                                 ((0, 0), (0, 0))]:
            A = X0 + (k + 0.3) * p.b0
            B = X0 + (m + 0.3) * p.b0
            sref, tref = cf.overlap_and_stiffness_1d(p.exps[mu], A, p.ang[mu] == 1,
                                                     p.exps[nu], B, p.ang[nu] == 1)
            e = max(e, abs(s[k, mu, m, nu] - sref), abs(a[k, mu, m, nu] - tref) / 10)
        errs.append(e)
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3
    assert errs[2] < 2e-3


def test_nuclear_attraction_converges():
    """V entry of an s-Gaussian pair against the Boys-function closed form."""
    errs = []
    for n0 in (8, 16):
        p = _cases.single_gaussian(alpha=0.8, n0=n0, box=10.0, R=40)
        V = dense.potential_matrix(p)
        x, X0, _ = grid.axis_nodes(p, 0)
        C = [X0 + 0.5 * p.b0] * 3
        ref = cf.nuclear_ss(0.8, C, 0.8, C, C)
        errs.append(abs(V[0, 0] - ref) / ref)
    assert errs[1] < errs[0] / 2.5
    assert errs[1] < 1e-2


def test_hydrogen_single_gaussian_energy():
    """Textbook variational energy of one normalised s-Gaussian on a Z=1
    nucleus: E(a) = 3a/2 - 2 sqrt(2a/pi), minimum -4/(3 pi)."""
    alpha = 8 / (9 * math.pi)
    exact = cf.hydrogen_single_gaussian(alpha)
    assert abs(exact + 4 / (3 * math.pi)) < 1e-14
    errs = []
    for n0 in (8, 16):
        p = _cases.single_gaussian(alpha=alpha, n0=n0, box=20.0, R=40)
        ev = dense.solve(p)
        errs.append(abs(ev[0] - exact))
    assert errs[1] < errs[0] and errs[1] < 5e-3


# ---------------- block-circulant structure (Lemma 3.1, Prop. A.1) ----------------

@pytest.mark.parametrize("maker", ["chain_m0_4", "chain_m0_8", "lattice_3d"])
def test_union_of_block_spectra_equals_dense_spectrum(maker):
    if maker == "chain_m0_4":
        p = _cases.periodic_chain_small(L=5, n0=8, n_perp=16, m0=4, R=16)
    elif maker == "chain_m0_8":
        p = _cases.periodic_chain_small(L=6, n0=6, n_perp=16, m0=8, R=16)
    else:
        p = _cases.periodic_3d_small(L=(3, 2, 2), n0=5, R=8)
    H, S = dense.build(p)
    ev = dense.eigvals(H, S)
    evb, per_block = blocks.circulant_route(p, H, S)
    w = np.linalg.eigvalsh(S)
    tol = max(1e-11, 4 * _cases.U64 * w.max() / w.min()) * np.max(np.abs(ev))   # u kappa_2(S)
    assert np.max(np.abs(ev - evb)) <= tol
    # circulant structure: block (r, c) depends on r - c only, and A_{L-k} = A_k^T
    m0 = p.m0
    if p.L[1] == p.L[2] == 1:
        L = p.L[0]
        for r in range(L):
            for c in range(L):
                blk = H[r * m0:(r + 1) * m0, c * m0:(c + 1) * m0]
                ref = H[((r - c) % L) * m0:((r - c) % L + 1) * m0, :m0]
                assert np.max(np.abs(blk - ref)) <= 1e-13 * np.max(np.abs(H))


def test_m0_1_circulant_is_fft_of_first_column():
    """m0 = 1: the pencil is diagonalised by the DFT, eigenvalues are
    fft(H[:,0]) / fft(S[:,0]) (numpy.fft, Appendix A.1)."""
    p = _cases.single_gaussian(alpha=0.4, n0=6, R=16, L=7, periodic=True)
    p = li.Problem(L=(7, 1, 1), periodic=(1, 0, 0), N=(42, 18, 18), n0=6, b0=2.0,
                   Z=p.Z, frac=p.frac, exps=p.exps, ang=p.ang, centre=p.centre, R=16,
                   sinc_t=p.sinc_t, sinc_c=p.sinc_c)
    H, S = dense.build(p)
    lam = np.fft.fft(H[:, 0]) / np.fft.fft(S[:, 0])
    assert np.max(np.abs(lam.imag)) < 1e-13
    ev = dense.eigvals(H, S)
    assert np.max(np.abs(np.sort(lam.real) - ev)) < 1e-12
    # block j of the direct DFT is the j-th FFT coefficient (same sign convention)
    Hb = blocks.fourier_blocks(p, blocks.generators_from_dense(p, H))[:, 0, 0]
    Sb = blocks.fourier_blocks(p, blocks.generators_from_dense(p, S))[:, 0, 0]
    assert np.max(np.abs(Hb - np.fft.fft(H[:, 0]))) < 1e-13 * np.max(np.abs(H))
    assert np.max(np.abs(Sb - np.fft.fft(S[:, 0]))) < 1e-13 * np.max(np.abs(S))


def test_fourier_blocks_hermitian_and_conjugate_pairs():
    """Cor. A.2: symmetric generators give Hermitian blocks and
    Abar_{L-j} = conj(Abar_j)."""
    p = _cases.periodic_3d_small(L=(3, 2, 4), n0=4, R=8)
    H, S = dense.build(p)
    Hb = blocks.fourier_blocks(p, blocks.generators_from_dense(p, H))
    L1, L2, L3 = p.L
    Hb = Hb.reshape(L1, L2, L3, p.m0, p.m0)
    assert np.max(np.abs(Hb - np.conj(np.swapaxes(Hb, -1, -2)))) < 1e-12
    for j in np.ndindex(L1, L2, L3):
        jm = tuple((-np.array(j)) % np.array(p.L))
        assert np.max(np.abs(Hb[jm] - np.conj(Hb[j]))) < 1e-12


def test_periodic_matrix_is_multilevel_block_circulant():
    """Lemma 3.4: on a periodic lattice H and S are symmetric three-level
    block circulant -- the block of cells (k + d, m + d) (componentwise mod
    L) equals that of (k, m) for every shift d -- so A_{L-k} = A_k^T."""
    p = _cases.periodic_3d_small(L=(3, 2, 4), n0=4, R=8)
    H, S = dense.build(p)
    m0 = p.m0
    cells = list(np.ndindex(*p.L))
    kb = lambda c: (c[0] * p.L[1] + c[1]) * p.L[2] + c[2]
    for M in (H, S):
        scale = np.max(np.abs(M))
        assert np.max(np.abs(M - M.T)) <= 1e-14 * scale
        blk = lambda a, b: M[kb(a) * m0:(kb(a) + 1) * m0, kb(b) * m0:(kb(b) + 1) * m0]
        for k in cells:
            for d in [(1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 1, 3)]:
                k2 = tuple((np.array(k) + d) % p.L)
                m2 = tuple(np.array(d) % p.L)
                assert np.max(np.abs(blk(k2, m2) - blk(k, (0, 0, 0)))) <= 1e-13 * scale
        gen = blocks.generators_from_dense(p, M)
        for k in cells:
            km = tuple((-np.array(k)) % p.L)
            assert np.max(np.abs(gen[kb(km)] - gen[kb(k)].T)) <= 1e-13 * scale


def test_block_band_follows_the_support_overlap():
    """Sec. 2.3 (the overlap constant L0): a block is nonzero exactly when the
    two cells' basis supports (plus the one-node reach of the P1 stencils)
    meet; with support half-width r_cut the band has 2 L0 + 1 blocks per
    interior row, L0 = floor((2 r_cut + h) / b0)."""
    n0, L = 5, 16
    exps = np.array([2.0, 3.0])
    p = _cases.with_table(li.Problem(L=(L, 1, 1), periodic=(0, 0, 0), N=(L * n0 + 20, 12, 12), n0=n0,
                                     b0=2.0, Z=np.array([1.0]), frac=np.array([[0.5, 0.5, 0.5]]),
                                     exps=exps, ang=np.zeros(2, int), centre=np.zeros(2, int), R=8))
    rcut = math.sqrt(math.log(1.0 / p.eps_support) / exps.min())
    L0 = int((2 * rcut + p.h) // p.b0)
    assert 0.1 < (2 * rcut + p.h) / p.b0 - L0 < 0.9        # not at a rounding edge
    H, S = dense.build(p)
    m0 = p.m0
    for M in (H, S):
        for k in range(L):
            for m in range(L):
                nz = np.any(M[k * m0:(k + 1) * m0, m * m0:(m + 1) * m0] != 0.0)
                assert nz == (abs(k - m) <= L0), (k, m)


# ---------------- box chains: Toeplitz interior, boundary defect ----------------

def test_box_chain_toeplitz_interior_and_wall_defect():
    """Sec. 2.3 (A)/(B): with the replicated potential the box matrix is block
    Toeplitz away from the walls; the defect is confined to the blocks whose
    supports reach the padding / walls."""
    p = _cases.box_chain_small(L=24, n0=5, pad=8, n_perp=14, R=12)
    H, S = dense.build(p)
    m0, L = p.m0, p.L[0]
    blk = lambda M, r, c: M[r * m0:(r + 1) * m0, c * m0:(c + 1) * m0]
    kc = L // 2
    scale = np.max(np.abs(H))
    G = grid.basis_axis(p, 0)
    nz = np.nonzero(np.any(G[:, kc, :] != 0, axis=1))[0]
    x, X0, _ = grid.axis_nodes(p, 0)
    reach = int(np.ceil(max(abs(x[nz[0]] - X0 - kc * p.b0), abs(x[nz[-1]] - X0 - (kc + 1) * p.b0))
                        / p.b0)) + 1
    for d in range(-3, 4):
        T = blk(H, kc + d, kc)
        for k in range(L):
            if not (0 <= k + d < L):
                continue
            far = min(k, k + d) >= reach and max(k, k + d) <= L - 1 - reach
            diff = np.max(np.abs(blk(H, k + d, k) - T))
            if far:
                assert diff <= 1e-13 * scale
    # the end blocks differ from the interior ones (the defect exists)
    assert np.max(np.abs(blk(H, 0, 0) - blk(H, kc, kc))) > 1e-8 * scale


def test_defect_reduces_to_charge_change_single_molecule():
    """A substitution Z -> Z' of the only nucleus of a single molecule equals
    solving with charge Z' (the defect kernel is the molecule's kernel)."""
    p = _cases.single_gaussian(alpha=0.9, n0=6, box=8.0, R=16)
    import dataclasses
    q = dataclasses.replace(p, defects=[li.Defect(cell=(0, 0, 0), nucleus=0, newZ=2.5)])
    r = dataclasses.replace(p, Z=np.array([2.5]))
    Hq, _ = dense.build(q)
    Hr, _ = dense.build(r)
    assert np.max(np.abs(Hq - Hr)) <= 1e-13 * np.max(np.abs(Hr))


def test_single_block_contraction_equals_dense_route():
    """The one-block 3D contraction used for large problems reproduces the
    dense matrices' blocks (periodic generators and a box chain's blocks)."""
    p = _cases.periodic_3d_small(L=(3, 2, 4), n0=4, R=8)
    H, S = dense.build(p)
    m0 = p.m0
    for kc in [(0, 0, 0), (1, 1, 3), (2, 0, 1)]:
        kb = (kc[0] * p.L[1] + kc[1]) * p.L[2] + kc[2]
        h, s = blocks.generator_block(p, kc)
        assert np.max(np.abs(h - H[kb * m0:(kb + 1) * m0, :m0])) <= 1e-14 * np.max(np.abs(H))
        assert np.max(np.abs(s - S[kb * m0:(kb + 1) * m0, :m0])) <= 1e-14 * np.max(np.abs(S))
    q = _cases.box_chain_small(L=9, n0=4, pad=5, n_perp=12, R=8)
    H, S = dense.build(q)
    m0 = q.m0
    for k, m in [(0, 0), (3, 1), (8, 6), (4, 4)]:
        h, s = blocks.generator_block(q, (k, 0, 0), mcell=(m, 0, 0))
        h2, _ = blocks.generator_block(q, (k, 0, 0), forms=dense.axis_forms(q), mcell=(m, 0, 0))
        assert np.max(np.abs(h - h2)) <= 1e-14 * np.max(np.abs(H))
        assert np.max(np.abs(h - H[k * m0:(k + 1) * m0, m * m0:(m + 1) * m0])) <= 1e-14 * np.max(np.abs(H))
        assert np.max(np.abs(s - S[k * m0:(k + 1) * m0, m * m0:(m + 1) * m0])) <= 1e-14 * np.max(np.abs(S))


def test_block_pencil_reduces_to_range_of_S():
    """Dependent basis functions: with m functions spanning an r-dimensional
    space (S = F^H F, H = F^H H0 F, F of rank r), the finite eigenvalues are
    those of H0 on that space, the other m - r are dropped (+inf); full rank:
    LAPACK's generalized eigenvalues of the pencil as it stands."""
    rng = np.random.default_rng(5)
    m, r = 7, 4
    Hh = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    Hh = Hh + Hh.conj().T
    A = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    S = A @ A.conj().T + 0.1 * np.eye(m)
    tau = S.shape[0] * blocks.EPS64 * np.linalg.norm(np.abs(S))
    got = blocks.block_eigs_rule(Hh, S, tau)
    ref = scipy.linalg.eigh(Hh, S, eigvals_only=True)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    F = rng.standard_normal((r, m)) + 1j * rng.standard_normal((r, m))
    H0 = rng.standard_normal((r, r)) + 1j * rng.standard_normal((r, r))
    H0 = H0 + H0.conj().T
    S2 = F.conj().T @ F
    tau2 = S2.shape[0] * blocks.EPS64 * np.linalg.norm(np.abs(S2))
    got = blocks.block_eigs_rule(F.conj().T @ H0 @ F, S2, tau2)
    assert np.sum(np.isinf(got)) == m - r
    ref = np.linalg.eigvalsh(H0)
    assert np.max(np.abs(got[:r] - ref)) < 1e-9 * np.max(np.abs(ref))


def _with_duplicate(p, mu):
    """The same problem with basis function mu listed twice (an exactly
    dependent basis: the overlap gets an exact null vector e_mu - e_m0)."""
    q = li.Problem(L=p.L, periodic=p.periodic, N=p.N, n0=p.n0, b0=p.b0, Z=p.Z, frac=p.frac,
                   exps=np.append(p.exps, p.exps[mu]), ang=np.append(p.ang, p.ang[mu]),
                   centre=np.append(p.centre, p.centre[mu]), R=p.R, sinc_t=p.sinc_t,
                   sinc_c=p.sinc_c)
    q.k_eig = p.k_eig
    return q


def test_block_pencil_vectors_are_S_orthonormal_on_the_kept_directions():
    """V^H S V = I for the kept eigenvectors; exactly the overlap
    eigenvalues at or below tau are removed (a rank-6 overlap of order 9
    with a ridge at the rounding level)."""
    rng = np.random.default_rng(11)
    A = rng.standard_normal((9, 6)) + 1j * rng.standard_normal((9, 6))
    S = A @ A.conj().T + 1e-15 * np.eye(9)
    Hh = rng.standard_normal((9, 9)) + 1j * rng.standard_normal((9, 9))
    Hh = Hh + Hh.conj().T
    tau = S.shape[0] * blocks.EPS64 * np.linalg.norm(np.abs(S))
    ev, V, r = blocks.block_pencil(Hh, S, tau)
    assert r == 6 and V.shape == (9, 6) and np.sum(np.isinf(ev)) == 3
    assert np.max(np.abs(V.conj().T @ S @ V - np.eye(6))) < 1e-10
    R = Hh @ V - (S @ V) * ev[:6]
    w, Q = np.linalg.eigh(S)
    assert np.max(np.abs(Q[:, w > tau].conj().T @ R)) < 1e-10 * np.max(np.abs(ev[:6]))


def test_overlap_scale_is_the_sum_of_the_overlap_blocks():
    """B = sum over offsets |S_offset| (factorised over the axes) equals the
    sum of |S_k| over the dense periodic overlap's generators, and for a box
    chain the sum of |S| over a block row of a cell that no wall reaches."""
    p = _cases.periodic_3d_small(L=(3, 2, 4), n0=5, R=8)
    S = dense.mass_kinetic(p)[0]
    ref = np.sum(np.abs(blocks.generators_from_dense(p, S)), axis=0)
    assert np.max(np.abs(blocks.overlap_scale(p) - ref)) <= 1e-14 * np.max(ref)
    q = _cases.box_chain_small(L=45, n0=4, pad=90, n_perp=12, R=8, k=4, seed=1)
    S = dense.mass_kinetic(q)[0]
    m0, kc = q.m0, q.L[0] // 2
    row = sum(np.abs(S[kc * m0:(kc + 1) * m0, m * m0:(m + 1) * m0]) for m in range(q.L[0]))
    assert np.max(np.abs(blocks.overlap_scale(q) - row)) <= 1e-14 * np.max(row)
    assert np.abs(S[kc * m0:(kc + 1) * m0, :m0]).max() == 0.0   # the row reaches no chain end


@pytest.mark.parametrize("seed", [2, 6, 31])
def test_rule_removes_nothing_on_the_timed_box_chains(seed):
    """Box chains of the timed workload (64 cells, grid 1024x256x256, m0 = 8)
    whose overlaps are ill-conditioned (kappa_2(S) 3e8 - 2e9) but far from
    singular: no direction reaches the cut (the smallest cell eigenvalue is
    more than 1e3 tau), so the answer is LAPACK's on (H, S) as they stand."""
    p = _cases.with_table(li.config2(seed))
    s, _, tau = blocks.cell_null_directions(p)
    assert s.min() > 1e3 * tau
    H, S = dense.build(p)
    ev, _, kept = blocks.box_eigs(p, H, S)
    assert kept == p.m0
    ref = scipy.linalg.eigh(H, S, eigvals_only=True, subset_by_index=[0, 15])
    assert np.max(np.abs(ev - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_dependent_function_is_removed_periodic():
    """Periodic chain whose basis lists one GTO twice: every Fourier block
    loses exactly one direction (+inf) and the kept spectrum equals the
    original problem's, which itself has nothing removed and equals the
    dense LAPACK spectrum (Prop. A.1)."""
    p = _cases.periodic_chain_small(L=5, n0=6, n_perp=16, m0=4, R=12)
    H, S = dense.build(p)
    ref = _cases.reference(p, H, S)
    ev0, per0 = blocks.periodic_eigs(p, H, S)
    assert np.all(np.isfinite(ev0))
    assert np.max(np.abs(ev0 - dense.eigvals(H, S))) <= 1e-10 * np.max(np.abs(ev0))
    q = _with_duplicate(p, 1)
    ev1, per1 = blocks.periodic_eigs(q)
    assert np.all(np.sum(np.isinf(per1), axis=1) == 1)
    got = np.concatenate([per1[j][:-1] for j in range(p.ncell)])
    blk = np.repeat(np.arange(p.ncell), p.m0)
    order = np.lexsort((blk, got))
    _cases.check(ref, got[order], blk[order])


def test_dependent_function_is_removed_box():
    """Box chain whose basis lists one GTO twice: the cell loses one
    direction and the lowest eigenvalues equal the original problem's
    (nothing removed there, so the dense LAPACK ones)."""
    p = _cases.box_chain_small(L=6, n0=4, pad=4, n_perp=12, R=8, k=4, seed=3)
    H, S = dense.build(p)
    ev0, _, kept0 = blocks.box_eigs(p, H, S)
    assert kept0 == p.m0
    assert np.max(np.abs(ev0 - dense.eigvals(H, S, p.k_eig))) <= 1e-13 * np.max(np.abs(ev0))
    q = _with_duplicate(p, 2)
    ev1, _, kept1 = blocks.box_eigs(q)
    assert kept1 == p.m0
    _cases.check(_cases.reference(p, H, S), ev1)


def test_cell_overlap_is_the_interior_diagonal_block():
    """The cell overlap (Toeplitz generator T_S[0]) equals the dense overlap's
    diagonal block of a cell whose functions reach neither wall."""
    p = _cases.box_chain_small(L=5, n0=4, pad=80, n_perp=12, R=8, k=4, seed=1)
    m0 = p.m0
    S = dense.mass_kinetic(p)[0]
    T0 = blocks.cell_overlap(p)
    for k in range(p.L[0]):
        assert np.max(np.abs(S[k * m0:(k + 1) * m0, k * m0:(k + 1) * m0] - T0)) <= 1e-14 * np.max(np.abs(S))


def test_removing_cell_directions_is_variational():
    """Removing cell directions restricts the trial space, so every reduced
    eigenvalue lies at or above the full problem's (Courant-Fischer); the
    smallest cell direction is removed here by reversing its decision."""
    p = _cases.box_chain_small(L=8, n0=5, pad=6, n_perp=14, seed=2, R=12, k=6)
    H, S = dense.build(p)
    full, _, kept = blocks.box_eigs(p, H, S)
    assert kept == p.m0
    red, _, kept1 = blocks.box_eigs(p, H, S, flip=(0,))
    assert kept1 == p.m0 - 1
    assert np.all(red >= full - 1e-10 * np.max(np.abs(full)))
    assert np.max(red - full) > 1e-8      # the removed direction mattered


def _chain_with_defects(p, defects):
    import dataclasses
    return dataclasses.replace(p, defects=list(defects))


def test_defects_on_every_cell_equal_a_charge_change_periodic_odd_chain():
    """On a periodic chain with an odd number of cells and the nucleus at the
    cell centre, the minimum-image kernels of all L nuclei are exactly the
    symmetric lattice window (Eq. 3.6), so substituting Z -> Z + dZ on every
    cell gives H = A/2 - (1 + dZ/Z) V."""
    p = _cases.periodic_chain_small(L=5, n0=6, n_perp=14, m0=4, R=12)
    dz = 0.7
    q = _chain_with_defects(p, [li.Defect(cell=(c, 0, 0), nucleus=0, newZ=1.0 + dz) for c in range(5)])
    H, S, A, V = dense.build(p, with_parts=True)
    Hq, Sq = dense.build(q)
    ref = 0.5 * A - (1.0 + dz) * V
    assert np.max(np.abs(Hq - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.array_equal(Sq, S)


@pytest.mark.parametrize("maker", [
    lambda: _cases.periodic_chain_small(L=9, n0=6, n_perp=14, m0=4, R=12),
    lambda: _cases.box_chain_small(L=10, n0=5, pad=5, n_perp=14, seed=1, R=12, k=4),
])
def test_defect_contributions_add_and_scale_with_the_charge_change(maker):
    """The nuclear potential is linear in the charges, so substitutions enter
    H as independent terms proportional to their charge change: two defects
    give the sum of their separate changes of H, halving the charge change
    halves the term, a substitution Z -> Z changes nothing, and S is never
    touched.  (A charge change is not local: the second defect's Coulomb tail
    shifts the first one's bound levels, so the pin is on H, not on the
    spectrum.)"""
    p = maker()
    H0, S0 = dense.build(p)

    def build(defects):
        return dense.build(_chain_with_defects(p, defects))

    Ha, Sa = build([li.Defect((2, 0, 0), 0, 3.0)])
    Hb, _ = build([li.Defect((6, 0, 0), 0, 3.0)])
    Hab, Sab = build([li.Defect((2, 0, 0), 0, 3.0), li.Defect((6, 0, 0), 0, 3.0)])
    Hh, _ = build([li.Defect((2, 0, 0), 0, 2.0)])
    Hn, _ = build([li.Defect((2, 0, 0), 0, float(p.Z[0]))])
    scale = np.max(np.abs(Ha - H0))
    assert scale > 0.1
    assert np.max(np.abs((Hab - H0) - (Ha - H0) - (Hb - H0))) <= 1e-12 * scale
    assert np.max(np.abs(2.0 * (Hh - H0) - (Ha - H0))) <= 1e-12 * scale
    assert np.max(np.abs(Hn - H0)) <= 1e-12 * scale
    assert np.array_equal(Sa, S0) and np.array_equal(Sab, S0)


def test_defect_matrix_translation_covariance():
    """A defect moved by one cell moves its matrix by one cell: cyclically on
    a periodic chain (exact symmetry of the ring), and in the interior of a
    box chain whose walls no function reaches."""
    p = _cases.periodic_chain_small(L=6, n0=6, n_perp=14, m0=4, R=12)
    m0 = p.m0
    D0 = dense.defect_matrix(_chain_with_defects(p, [li.Defect((0, 0, 0), 0, 0.0)]))
    D2 = dense.defect_matrix(_chain_with_defects(p, [li.Defect((2, 0, 0), 0, 0.0)]))
    sh = np.roll(np.roll(D0, 2 * m0, axis=0), 2 * m0, axis=1)
    assert np.max(np.abs(D2 - sh)) <= 1e-13 * np.max(np.abs(D0))
    b = _cases.box_chain_small(L=7, n0=4, pad=90, n_perp=12, R=8, k=4, seed=3)
    m0 = b.m0
    E3 = dense.defect_matrix(_chain_with_defects(b, [li.Defect((3, 0, 0), 0, 2.0)]))
    E4 = dense.defect_matrix(_chain_with_defects(b, [li.Defect((4, 0, 0), 0, 2.0)]))
    assert np.max(np.abs(E4[m0:, m0:] - E3[:-m0, :-m0])) <= 1e-13 * np.max(np.abs(E3))


# ---------------- box vs periodic chains as L grows (Sec. 4, the average energy per cell) ----------------

def test_box_and_periodic_chains_relax_to_each_other():
    """A box chain and its periodic supercell (same basis, grid and rank):
    the lowest eigenvalues differ by a confinement term that falls like
    1/L^2, and the average of the lowest L eigenvalues (the energy per cell
    of the lowest band) differs by an end term that falls like 1/L -- the
    relaxation of the average energy per cell for both boundary conditions
    that the paper's chain experiments show.  (Higher in the spectrum the
    two keep a systematic difference, which the paper also reports.)"""
    base = li.config1()
    d_low, d_avg = [], []
    for L in (4, 8, 16):
        n0, nperp, pad = 8, 16, 40
        box = _cases.with_table(li.Problem(
            L=(L, 1, 1), periodic=(0, 0, 0), N=(L * n0 + 2 * pad, nperp, nperp), n0=n0, b0=2.0,
            Z=base.Z, frac=base.frac, exps=base.exps, ang=base.ang, centre=base.centre, R=16))
        per = box.as_periodic_chain().with_table(box.sinc_t, box.sinc_c)
        eb = dense.eigvals(*dense.build(box))
        ep = dense.eigvals(*dense.build(per))
        d_low.append(eb[0] - ep[0])
        d_avg.append(abs(eb[:L].mean() - ep[:L].mean()))
    assert all(d > 0 for d in d_low)                     # confinement raises the band bottom
    assert d_low[1] < d_low[0] / 2.5 and d_low[2] < d_low[1] / 2.5
    assert d_avg[1] < d_avg[0] / 1.6 and d_avg[2] < d_avg[1] / 1.6


def test_chain_lattice_sum_diverges_like_the_harmonic_series():
    """The lattice sum of a charged chain converges only conditionally (Sec.
    2.3, Eq. 2.13): on a periodic chain of protons the window of the central
    cell grows with L, and doubling L adds the charges between L/2 and L
    cells away on both sides, which lowers the band bottom by
    (2 Z / b0) ln 2 (the harmonic series) up to the discretisation error of
    the P0 potential against the P1 mass, O(h^2)."""
    base = li.config1()
    target = 2.0 * math.log(2.0) / 2.0
    excess = []
    for n0 in (8, 16, 32):
        low = []
        for L in (32, 64):
            p = _cases.with_table(li.Problem(
                L=(L, 1, 1), periodic=(1, 0, 0), N=(L * n0, 2 * n0, 2 * n0), n0=n0, b0=2.0, Z=base.Z,
                frac=base.frac, exps=base.exps, ang=base.ang, centre=base.centre, R=24))
            H, S = dense.build(p)
            low.append(blocks.periodic_eigs(p, H, S)[0][0])
        excess.append((low[0] - low[1]) - target)
    assert all(e > 0 for e in excess)
    assert excess[1] < excess[0] / 3.5 and excess[2] < excess[1] / 3.5      # O(h^2)
    assert excess[2] < 1e-3 * target * 2


# ---------------- routes for the large workloads (no dense 3D tensors) ----------------

@pytest.mark.parametrize("maker", ["box", "periodic"])
def test_chain_matrices_equal_the_dense_build(maker):
    """The pair-grouped chain route (long chains) gives the dense build's
    H and S: the same grid sums in another grouping."""
    if maker == "box":
        p = _cases.box_chain_small(L=12, n0=5, pad=6, n_perp=20, R=16, k=6)
    else:
        p = _cases.periodic_chain_small(L=6, n0=6, n_perp=16, m0=8, R=16)
    H, S = dense.build(p)
    H2, S2 = dense.chain_matrices(p)
    assert np.max(np.abs(H2 - H)) <= 1e-14 * np.max(np.abs(H))
    assert np.max(np.abs(S2 - S)) <= 1e-14 * np.max(np.abs(S))


def test_generators_direct_equal_the_dense_first_block_column_and_single_blocks():
    """Every generator of a 3D periodic lattice without the dense matrix:
    equal to the dense matrices' first block column and to the one-block
    contraction (generator_block, an independent grouping of the sum)."""
    p = _cases.periodic_3d_small(L=(3, 2, 4), n0=5, R=8)
    H, S = dense.build(p)
    gh, gs = blocks.generators_direct(p)
    assert np.max(np.abs(gh - blocks.generators_from_dense(p, H))) <= 1e-14 * np.max(np.abs(H))
    assert np.max(np.abs(gs - blocks.generators_from_dense(p, S))) <= 1e-14 * np.max(np.abs(S))
    for kc in [(0, 0, 0), (1, 1, 3), (2, 0, 1)]:
        h, s = blocks.generator_block(p, kc)
        kb = (kc[0] * p.L[1] + kc[1]) * p.L[2] + kc[2]
        assert np.max(np.abs(gh[kb] - h)) <= 1e-14 * np.max(np.abs(H))
        assert np.max(np.abs(gs[kb] - s)) <= 1e-14 * np.max(np.abs(S))
