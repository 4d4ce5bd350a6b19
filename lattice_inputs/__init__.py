"""Seeded synthetic lattice problems (inputs only).

This module describes a lattice problem by the parameters the paper's
problem statement uses (Sec. 2.1-2.3, Sec. 3.3): lattice dimensions
L1 x L2 x L3, boundary conditions, the uniform grid (cell size b0 = n0*h,
nodes per axis), the nuclei of the unit cell (charges Z and positions),
the Gaussian (GTO) basis of the unit cell (exponents, angular type,
centre) and the rank R of the Newton-kernel quadrature.  It also draws the
seeded synthetic workloads shaped like the paper's hydrogen chains and 3D
lattices.

It holds none of the method's arithmetic: both the CPU oracle and the
CUDA path read these parameters and compute everything else themselves.
The quadrature table (t_q, c_q) is an input of the problem; callers fill
it from whichever rule they use.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np

ANG_S, ANG_PX, ANG_PY, ANG_PZ = 0, 1, 2, 3


@dataclass
class Defect:
    """Substitution of nucleus `nucleus` of lattice cell `cell` by charge
    `newZ` (newZ = 0 is a vacancy; the basis functions stay)."""
    cell: tuple
    nucleus: int
    newZ: float


@dataclass
class Problem:
    L: tuple                    # lattice cells per axis (L1, L2, L3)
    periodic: tuple             # 1 = periodic axis, 0 = Dirichlet (box) axis
    N: tuple                    # grid nodes per axis
    n0: int                     # grid nodes per cell, h = b0 / n0
    b0: float                   # cell size (bohr), same on all axes
    Z: np.ndarray               # (M0,) nuclear charges of the unit cell
    frac: np.ndarray            # (M0, 3) nucleus positions as cell fractions
    exps: np.ndarray            # (m0,) GTO exponents
    ang: np.ndarray             # (m0,) 0 = s, 1 = p_x, 2 = p_y, 3 = p_z
    centre: np.ndarray          # (m0,) index of the nucleus carrying the GTO
    R: int                      # Newton-kernel quadrature rank
    sinc_t: np.ndarray | None = None   # (R,) Gaussian parameters t_q
    sinc_c: np.ndarray | None = None   # (R,) weights c_q
    eps_support: float = 1e-14
    defects: list = field(default_factory=list)
    k_eig: int = 0              # eigenpairs wanted by a box solve (0 = all)
    precision: int = 0          # 0 FP64, 1 mixed (tensor-core split products), 2 mixed + FP32 phase
    box_potential: int = 0      # box chains: 0 replicated central cell, 1 plain lattice sum over the cells

    # ---- plain derived sizes (no method arithmetic) ----
    @property
    def h(self) -> float:
        return self.b0 / self.n0

    @property
    def M0(self) -> int:
        return int(len(self.Z))

    @property
    def m0(self) -> int:
        return int(len(self.exps))

    @property
    def ncell(self) -> int:
        return int(self.L[0] * self.L[1] * self.L[2])

    @property
    def Nb(self) -> int:
        return self.ncell * self.m0

    @property
    def is_box(self) -> bool:
        """A box problem has a Dirichlet axis that carries more than one cell."""
        return any((not self.periodic[a]) and self.L[a] > 1 for a in range(3))

    def with_table(self, t, c) -> "Problem":
        return dataclasses.replace(self, sinc_t=np.asarray(t, float).copy(),
                                   sinc_c=np.asarray(c, float).copy(), R=len(t))

    def as_periodic_chain(self) -> "Problem":
        """Same lattice, basis and grid along the chain axis made periodic
        (the paper's Table 1 pairs a box chain with its periodic supercell)."""
        per = list(self.periodic)
        N = list(self.N)
        for a in range(3):
            if self.L[a] > 1:
                per[a] = 1
                N[a] = self.L[a] * self.n0
        return dataclasses.replace(self, periodic=tuple(per), N=tuple(N),
                                   defects=list(self.defects))


def _basis8(rng):
    """One draw of the 8-function recipe: six exponents log-uniform in
    [0.1, 30], sorted; the four middle ones are s, the largest is shared by
    p_x, p_y, p_z, the smallest is a diffuse s."""
    a = np.sort(np.exp(rng.uniform(np.log(0.1), np.log(30.0), size=6)))
    exps = [a[1], a[2], a[3], a[4], a[5], a[5], a[5], a[0]]
    ang = [ANG_S] * 4 + [ANG_PX, ANG_PY, ANG_PZ] + [ANG_S]
    return exps, ang


def config1(seed_id: int = 0) -> Problem:
    """Periodic chain 8x1x1, cell 2.0 bohr, one Z=1 nucleus per cell,
    4 s-GTOs (0.25, 1, 4, 16), n0 = 32 (h = 1/16), 256 nodes per axis, R = 24."""
    return Problem(L=(8, 1, 1), periodic=(1, 0, 0), N=(256, 256, 256), n0=32, b0=2.0,
                   Z=np.array([1.0]), frac=np.array([[0.5, 0.5, 0.5]]),
                   exps=np.array([0.25, 1.0, 4.0, 16.0]), ang=np.zeros(4, int),
                   centre=np.zeros(4, int), R=24)


def config2(request_id: int = 0, L: int = 64, n0: int = 15, pad: int = 32,
            n_perp: int = 256, R: int = 32, config_index: int = 1) -> Problem:
    """Dirichlet box chain Lx1x1, Z=1 at the cell centre, m0 = 8 (one draw of
    the 8-function recipe), N_x = L*n0 + 2*pad, N_perp transverse, R = 32,
    lowest 16 eigenpairs."""
    rng = np.random.default_rng(1000 * config_index + request_id)
    exps, ang = _basis8(rng)
    return Problem(L=(L, 1, 1), periodic=(0, 0, 0), N=(L * n0 + 2 * pad, n_perp, n_perp),
                   n0=n0, b0=2.0, Z=np.array([1.0]), frac=np.array([[0.5, 0.5, 0.5]]),
                   exps=np.array(exps), ang=np.array(ang), centre=np.zeros(8, int), R=R,
                   k_eig=16)


def config3(request_id: int = 0, L: int = 16, n0: int = 32, R: int = 32,
            config_index: int = 2, draws_per_atom: int = 1) -> Problem:
    """Periodic LxLxL lattice, two sublattices at (1/4,1/4,1/4) and
    (3/4,3/4,3/4), each Z drawn from {1,2,3}, per atom the 8-function recipe
    (m0 = 16), n0 = 32 nodes per cell, R = 32 (rank M0*R = 64)."""
    rng = np.random.default_rng(1000 * config_index + request_id)
    Z = rng.integers(1, 4, size=2).astype(float)
    exps, ang, cen = [], [], []
    for atom in range(2):
        for _ in range(draws_per_atom):
            e, a = _basis8(rng)
            exps += e
            ang += a
            cen += [atom] * 8
    return Problem(L=(L, L, L), periodic=(1, 1, 1), N=(L * n0,) * 3, n0=n0, b0=2.0,
                   Z=Z, frac=np.array([[0.25] * 3, [0.75] * 3]), exps=np.array(exps),
                   ang=np.array(ang), centre=np.array(cen), R=R)


def config5_box(request_id: int = 0) -> Problem:
    """Dirichlet chain 512x1x1, n0 = 15, pad 256 (N_x = 8192), N_perp = 256,
    m0 = 32 on one Z=1 nucleus (four draws of the 8-function recipe), R = 40,
    lowest 64 eigenpairs."""
    rng = np.random.default_rng(1000 * 4 + request_id)
    exps, ang = [], []
    for _ in range(4):
        e, a = _basis8(rng)
        exps += e
        ang += a
    return Problem(L=(512, 1, 1), periodic=(0, 0, 0), N=(8192, 256, 256), n0=15, b0=2.0,
                   Z=np.array([1.0]), frac=np.array([[0.5, 0.5, 0.5]]), exps=np.array(exps),
                   ang=np.array(ang), centre=np.zeros(32, int), R=40, k_eig=64)


def config5_periodic(request_id: int = 0) -> Problem:
    """Periodic 32x32x32, n0 = 16 (N = 512 per axis), M0 = 2, m0 = 32 (two
    draws of the 8-function recipe per atom), R = 40 (rank 80)."""
    p = config3(request_id, L=32, n0=16, R=40, config_index=4, draws_per_atom=2)
    return p


def random_defects(rng, L, M0, count) -> list:
    """`count` defects in uniformly drawn cells: vacancy or substitution
    (new charge from {1,2,3}) with probability 1/2 each."""
    out = []
    cells = set()
    while len(out) < count:
        c = tuple(int(rng.integers(0, L[a])) for a in range(3))
        nu = int(rng.integers(0, M0))
        if (c, nu) in cells:
            continue
        cells.add((c, nu))
        newZ = 0.0 if rng.random() < 0.5 else float(rng.integers(1, 4))
        out.append(Defect(cell=c, nucleus=nu, newZ=newZ))
    return out


def serving_stream(n_requests: int = 512, seed: int = 3000, n0: int = 16, n_perp: int = 256,
                   R: int = 32):
    """Requests shaped like the serving mix: chains L in {4..256} x1x1 or
    cubes {8,12,16,24}^3 (half each), m0 in {4, 8, 16} with the recipes of the
    other workloads, periodic or box half each (cubes are periodic), 0-4
    defects on chains.  Returns a list of Problems (arrival times are drawn by
    the caller)."""
    rng = np.random.default_rng(seed)
    out = []
    for rid in range(n_requests):
        chain = rng.random() < 0.5
        m0 = int(rng.choice([4, 8, 16]))
        box = chain and (rng.random() < 0.5)
        if m0 == 4:
            exps, ang = [0.25, 1.0, 4.0, 16.0], [ANG_S] * 4
            cen = [0] * 4
        elif m0 == 8:
            exps, ang = _basis8(rng)
            cen = [0] * 8
        else:
            e1, a1 = _basis8(rng)
            e2, a2 = _basis8(rng)
            exps, ang = e1 + e2, a1 + a2
            cen = [0] * 16
        if chain:
            L = int(rng.integers(4, 257))
            Lv = (L, 1, 1)
            per = (0, 0, 0) if box else (1, 0, 0)
            N = (L * n0 + (2 * 32 if box else 0), n_perp, n_perp)
        else:
            L = int(rng.choice([8, 12, 16, 24]))
            Lv = (L, L, L)
            per = (1, 1, 1)
            N = (L * n0,) * 3
        # lowest 16 eigenpairs, fewer on chains too short for 16 (the block
        # iteration needs 3 (k + guard) <= L m0)
        nb = Lv[0] * m0
        k = 16 if nb >= 60 else max(1, nb // 5)
        p = Problem(L=Lv, periodic=per, N=N, n0=n0, b0=2.0, Z=np.array([1.0]),
                    frac=np.array([[0.5, 0.5, 0.5]]), exps=np.array(exps), ang=np.array(ang),
                    centre=np.array(cen), R=R, k_eig=k if box else 0)
        if chain:
            nd = int(rng.integers(0, 5))
            p.defects = random_defects(rng, Lv, 1, nd)
            if nd:
                p.k_eig = k
        out.append(p)
    return out
