"""Grid, nodal GTO vectors and the lattice-summed potential tensor.

Readings of the paper used throughout (where the paper leaves a choice
open, the choice made here):

* One uniform node set per axis with step h = b0/n0 (Sec. 2.3, the same h on
  all axes).  Periodic axis: N = L*n0 nodes at x_i = (i + 1/2) h, period
  N h.  Dirichlet axis: N interior nodes x_i = (i + 1) h, walls at 0 and
  (N + 1) h (Sec. 2.4), the lattice starting at X0 = (pad + 1/2) h with
  pad = (N - L n0) div 2.  Cell k of an axis spans [X0 + k b0, X0 + (k+1) b0).
* GTOs are separable products of 1D factors (Sec. 2.4): s-type
  exp(-a d^2), p-type d exp(-a d^2) on its own axis, L2-normalised in the
  continuum, set to zero where |d| > sqrt(ln(1/eps_s)/a) ("zero extension",
  Sec. 2.3); on a periodic axis d is the minimum-image displacement.
  Each basis function is sampled at the nodes (P1 interpolant for the
  Laplacian and mass, nodal values for the potential: Sec. 2.2, 2.4).
* The potential is the central-cell lattice sum (Eq. 3.6) over a symmetric
  window k in {-floor(L/2) .. floor(L/2)} per axis (weight 1/2 on +-L/2 when
  L is even), evaluated in the reference cell and replicated to every cell
  (Sec. 3.3).  On a Dirichlet axis the replication keeps the end cells'
  values over the padding (cell index clamped to 0..L-1), so an axis with a
  single cell is evaluated directly.  The same potential serves periodic
  and box problems (reading R1).  Reading R2, the plain lattice sum over
  the box's cells of Sec. 2.3 case (B), is available for box problems
  through potential_slabs(p, "lattice_sum"); the library computes R1.
* The Newton kernel is projected on piecewise-constant cells centred at the
  nodes (Eq. 2.6) and approximated by the R-term Gaussian sum (Eq. 2.7), so
  one axis factor is the cell integral of exp(-t_q^2 (x - a)^2), which has
  the closed form sqrt(pi)/(2 t) [erf(t (x_hi - a)) - erf(t (x_lo - a))]
  (evaluated through erfc in the tails to avoid cancellation).
"""
import numpy as np
from scipy.special import erf, erfc


def axis_nodes(p, ax):
    """Node coordinates x_i, lattice origin X0 and period (None if Dirichlet)."""
    N, L, n0, h = p.N[ax], p.L[ax], p.n0, p.h
    if p.periodic[ax]:
        if N != L * n0:
            raise ValueError("periodic axis needs N = L*n0")
        return (np.arange(N) + 0.5) * h, 0.0, N * h
    pad = (N - L * n0) // 2
    if pad < 0:
        raise ValueError("Dirichlet axis needs N >= L*n0")
    return (np.arange(N) + 1.0) * h, (pad + 0.5) * h, None


def min_image(d, period):
    if period is None:
        return d
    return d - period * np.floor(d / period + 0.5)


def gto_norm_1d(alpha, is_p):
    """Continuum L2 normalisation of exp(-a x^2) or x exp(-a x^2)."""
    n = (2.0 * alpha / np.pi) ** 0.25
    return n * 2.0 * np.sqrt(alpha) if is_p else n


def basis_axis(p, ax, cells=None):
    """G[i, c, mu] = 1D factor along `ax` of GTO mu of cell k at node i, for
    all cells k (c = k) or for the listed cells (c = position in `cells`)."""
    x, X0, period = axis_nodes(p, ax)
    N, L, m0 = p.N[ax], p.L[ax], p.m0
    cells = list(range(L)) if cells is None else list(cells)
    G = np.zeros((N, len(cells), m0))
    for mu in range(m0):
        alpha = float(p.exps[mu])
        is_p = int(p.ang[mu]) == ax + 1
        rcut = np.sqrt(np.log(1.0 / p.eps_support) / alpha)
        nrm = gto_norm_1d(alpha, is_p)
        f = float(p.frac[int(p.centre[mu]), ax])
        for c, k in enumerate(cells):
            A = X0 + (k + f) * p.b0
            d = min_image(x - A, period)
            v = nrm * np.exp(-alpha * d * d)
            if is_p:
                v = v * d
            v[np.abs(d) > rcut] = 0.0
            G[:, c, mu] = v
    return G


def gauss_cell_integral(t, lo, hi):
    """int_lo^hi exp(-t^2 s^2) ds (broadcasting), via erf / erfc."""
    a = t * lo
    b = t * hi
    with np.errstate(invalid="ignore"):
        val = np.where(a >= 0, erfc(a) - erfc(b),
                       np.where(b <= 0, erfc(-b) - erfc(-a), erf(b) - erf(a)))
    return val * (np.sqrt(np.pi) / (2.0 * t))


def window(L):
    """Lattice-sum window along one axis: offsets and weights."""
    if L == 1:
        return np.array([0]), np.array([1.0])
    hw = L // 2
    ks = np.arange(-hw, hw + 1)
    w = np.ones(len(ks))
    if L % 2 == 0:
        w[0] = w[-1] = 0.5
    return ks, w


def reduced_nodes(p, ax):
    """Node coordinate replicated into the reference cell (cell index taken
    modulo L on a periodic axis, clamped to 0..L-1 on a Dirichlet axis)."""
    x, X0, period = axis_nodes(p, ax)
    k = np.floor((x - X0) / p.b0)
    if period is not None:
        pass  # every node lies in some cell 0..L-1; shift it to cell 0
    else:
        k = np.clip(k, 0, p.L[ax] - 1)
    return x - k * p.b0


def potential_axis(p, ax):
    """Window-summed 1D factors pt[nu, q, i] (Eq. 2.13 per axis):
    sum_k w_k int_{cell(i)} exp(-t_q^2 (s - a_nu - k b0)^2) ds, where the
    cell is that of the node replicated into the reference cell."""
    y = reduced_nodes(p, ax)
    _, X0, _ = axis_nodes(p, ax)
    h = p.h
    ks, ws = window(p.L[ax])
    t = np.asarray(p.sinc_t, float)
    out = np.zeros((p.M0, len(t), len(y)))
    for nu in range(p.M0):
        a0 = X0 + p.frac[nu, ax] * p.b0
        for k, w in zip(ks, ws):
            a = a0 + k * p.b0
            lo = (y - h / 2 - a)[None, :]
            hi = (y + h / 2 - a)[None, :]
            out[nu] += w * gauss_cell_integral(t[:, None], lo, hi)
    return out


def potential_axis_lattice_sum(p, ax):
    """Box potential read as the plain lattice sum of Sec. 2.3 case (B)
    (reading R2): on a Dirichlet axis pB[nu, q, i] is the sum over the
    axis' cells k = 0..L-1 of int_{cell(x_i)} exp(-t_q^2 (s - a_nu - k b0)^2)
    ds at the node's own position: no window, no replication, so each
    nucleus of the box is counted once with its full charge.  A periodic
    axis keeps the window-summed, replicated factor of potential_axis
    (case (A)).  The 3D kernel of the box, a sum over all cells of products
    of these axis terms, is the product of the per-axis sums because the
    cell set is a product of per-axis ranges (Eq. 2.13 summed over k)."""
    if p.periodic[ax]:
        return potential_axis(p, ax)
    x, X0, _ = axis_nodes(p, ax)
    h = p.h
    t = np.asarray(p.sinc_t, float)
    out = np.zeros((p.M0, len(t), len(x)))
    for nu in range(p.M0):
        for k in range(p.L[ax]):
            a = X0 + (p.frac[nu, ax] + k) * p.b0
            out[nu] += gauss_cell_integral(t[:, None], (x - h / 2 - a)[None, :],
                                           (x + h / 2 - a)[None, :])
    return out


BOX_POTENTIALS = ("replicated", "lattice_sum")


def potential_slabs(p, box_potential="replicated"):
    """The 3D potential tensor P(i1,i2,i3) = sum_nu Z_nu sum_q c_q
    prod_l pt_l[nu,q,i_l], returned as the distinct axis-0 slabs: (slab
    index per i1, array (nslab, N2, N3)).  box_potential "replicated"
    (reading R1): Eq. 2.13 restricted to the reference cell and replicated
    (Eq. 3.6); two nodes of axis 0 share a slab exactly when they replicate
    to the same reference-cell node.  "lattice_sum" (reading R2): the plain
    sum over the box's cells on Dirichlet axes (potential_axis_lattice_sum);
    every node of a Dirichlet axis 0 has its own slab."""
    if box_potential not in BOX_POTENTIALS:
        raise ValueError(f"box_potential must be one of {BOX_POTENTIALS}")
    c = np.asarray(p.sinc_c, float)
    if box_potential == "replicated":
        pt = [potential_axis(p, a) for a in range(3)]
        y0 = reduced_nodes(p, 0)
    else:
        pt = [potential_axis_lattice_sum(p, a) for a in range(3)]
        y0 = reduced_nodes(p, 0) if p.periodic[0] else axis_nodes(p, 0)[0]
    uniq, slab_of = np.unique(np.round(y0 / p.h * 2).astype(np.int64), return_inverse=True)
    first = np.array([np.nonzero(slab_of == s)[0][0] for s in range(len(uniq))])
    N2, N3 = p.N[1], p.N[2]
    slabs = np.zeros((len(uniq), N2, N3))
    for nu in range(p.M0):
        coef = p.Z[nu] * c[None, :] * pt[0][nu][:, first].T      # (nslab, R)
        B = pt[1][nu][:, :, None] * pt[2][nu][:, None, :]         # (R, N2, N3)
        slabs += np.tensordot(coef, B, axes=(1, 0))
    return slab_of, slabs


def potential_full_window(p):
    """Brute-force 3D tensor with the explicit 3D window sum
    sum_{k1,k2,k3} w1 w2 w3 prod_l int exp(..)  (tiny grids only)."""
    c = np.asarray(p.sinc_c, float)
    t = np.asarray(p.sinc_t, float)
    h = p.h
    ys = [reduced_nodes(p, a) for a in range(3)]
    X0s = [axis_nodes(p, a)[1] for a in range(3)]
    wins = [window(p.L[a]) for a in range(3)]
    P = np.zeros(tuple(p.N))
    for nu in range(p.M0):
        for k1, w1 in zip(*wins[0]):
            for k2, w2 in zip(*wins[1]):
                for k3, w3 in zip(*wins[2]):
                    e = []
                    for a, k in enumerate((k1, k2, k3)):
                        aa = X0s[a] + (p.frac[nu, a] + k) * p.b0
                        e.append(gauss_cell_integral(t[:, None], (ys[a] - h / 2 - aa)[None, :],
                                                     (ys[a] + h / 2 - aa)[None, :]))
                    P += p.Z[nu] * w1 * w2 * w3 * np.einsum("q,qi,qj,qk->ijk", c, *e)
    return P


def potential_lattice_sum_brute(p):
    """Brute-force 3D tensor of the box potential under reading R2: an
    explicit loop over every cell (k1, k2, k3) of a box whose axes are all
    Dirichlet and every nucleus, each term the full 3D product of cell
    integrals at the nodes' own positions (tiny grids only)."""
    if any(p.periodic):
        raise ValueError("the lattice-sum brute force takes Dirichlet axes only")
    c = np.asarray(p.sinc_c, float)
    t = np.asarray(p.sinc_t, float)
    h = p.h
    xs = [axis_nodes(p, a)[0] for a in range(3)]
    X0s = [axis_nodes(p, a)[1] for a in range(3)]
    P = np.zeros(tuple(p.N))
    for nu in range(p.M0):
        for k1 in range(p.L[0]):
            for k2 in range(p.L[1]):
                for k3 in range(p.L[2]):
                    e = []
                    for a, k in enumerate((k1, k2, k3)):
                        aa = X0s[a] + (p.frac[nu, a] + k) * p.b0
                        e.append(gauss_cell_integral(t[:, None], (xs[a] - h / 2 - aa)[None, :],
                                                     (xs[a] + h / 2 - aa)[None, :]))
                    P += p.Z[nu] * np.einsum("q,qi,qj,qk->ijk", c, *e)
    return P


def single_nucleus_axis(p, ax, pos):
    """1D factors of one nucleus' kernel at coordinate `pos` (no window, no
    replication; minimum image on a periodic axis): e[q, i]."""
    x, _, period = axis_nodes(p, ax)
    t = np.asarray(p.sinc_t, float)
    d = min_image(x - pos, period)
    h = p.h
    return gauss_cell_integral(t[:, None], (d - h / 2)[None, :], (d + h / 2)[None, :])
