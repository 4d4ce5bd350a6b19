"""The seeded synthetic workloads have the shapes stated for them (the
paper's hydrogen chains and 3D lattices: cells of 2.0 bohr, the grids,
bases, ranks and eigenpair counts of each configuration) and are
reproducible from their seeds."""
import numpy as np

import lattice_inputs as li

S, PX, PY, PZ = li.ANG_S, li.ANG_PX, li.ANG_PY, li.ANG_PZ


def _recipe8(exps, ang):
    """The 8-function recipe: six exponents log-uniform in [0.1, 30]; the four
    middle ones s, the largest shared by p_x, p_y, p_z, the smallest a
    diffuse s."""
    e = np.asarray(exps)
    assert list(ang) == [S, S, S, S, PX, PY, PZ, S]
    assert np.all((e >= 0.1) & (e <= 30.0))
    assert e[4] == e[5] == e[6] and e[7] < e[0] <= e[1] <= e[2] <= e[3] <= e[4]


def test_periodic_chain_8_cells():
    p = li.config1()
    assert p.L == (8, 1, 1) and p.periodic == (1, 0, 0) and p.N == (256, 256, 256)
    assert p.n0 == 32 and p.b0 == 2.0 and p.h == 1 / 16 and p.R == 24
    assert list(p.Z) == [1.0] and list(p.exps) == [0.25, 1.0, 4.0, 16.0] and list(p.ang) == [S] * 4
    assert p.Nb == 32 and not p.is_box


def test_box_chain_64_cells():
    for rid in (0, 1, 511):
        p = li.config2(rid)
        assert p.L == (64, 1, 1) and p.periodic == (0, 0, 0) and p.N == (1024, 256, 256)
        assert p.n0 == 15 and p.R == 32 and p.k_eig == 16 and p.Nb == 512 and p.is_box
        _recipe8(p.exps, p.ang)
    per = li.config2(0).as_periodic_chain()
    assert per.periodic == (1, 0, 0) and per.N == (960, 256, 256) and not per.is_box


def test_periodic_16_cubed():
    p = li.config3(0)
    assert p.L == (16, 16, 16) and p.periodic == (1, 1, 1) and p.N == (512, 512, 512)
    assert p.M0 == 2 and p.m0 == 16 and p.R * p.M0 == 64
    assert set(p.Z) <= {1.0, 2.0, 3.0}
    assert np.allclose(p.frac, [[0.25] * 3, [0.75] * 3])
    _recipe8(p.exps[:8], p.ang[:8])
    _recipe8(p.exps[8:], p.ang[8:])
    assert list(p.centre) == [0] * 8 + [1] * 8


def test_large_workloads():
    b = li.config5_box(0)
    assert b.L == (512, 1, 1) and b.N == (8192, 256, 256) and b.n0 == 15
    assert b.m0 == 32 and b.R == 40 and b.k_eig == 64 and b.Nb == 16384
    for q in range(4):
        _recipe8(b.exps[8 * q:8 * q + 8], b.ang[8 * q:8 * q + 8])
    p = li.config5_periodic(0)
    assert p.L == (32, 32, 32) and p.N == (512, 512, 512) and p.m0 == 32 and p.M0 * p.R == 80
    assert p.ncell == 32768


def test_serving_mix_shapes():
    ps = li.serving_stream(512, seed=3000)
    chains = [p for p in ps if p.L[1] == 1]
    cubes = [p for p in ps if p.L[1] > 1]
    assert 0.4 < len(chains) / len(ps) < 0.6
    for p in chains:
        assert 4 <= p.L[0] <= 256 and p.N[1:] == (256, 256) and p.n0 == 16 and p.R == 32
        assert len(p.defects) <= 4
        assert p.N[0] == p.L[0] * 16 + (64 if p.is_box else 0)
    for p in cubes:
        assert p.L[0] in (8, 12, 16, 24) and p.L[0] == p.L[1] == p.L[2]
        assert p.periodic == (1, 1, 1) and not p.defects
    assert {p.m0 for p in ps} == {4, 8, 16}
    box = sum(p.is_box for p in chains)
    assert 0.35 < box / len(chains) < 0.65
    kinds = {(d.newZ == 0.0) for p in chains for d in p.defects}
    assert kinds == {True, False}                         # vacancies and substitutions


def test_seeded_and_reproducible():
    a, b = li.config2(7), li.config2(7)
    assert np.array_equal(a.exps, b.exps)
    assert not np.array_equal(li.config2(7).exps, li.config2(8).exps)
    s1 = li.serving_stream(32, seed=3000)
    s2 = li.serving_stream(64, seed=3000)[:32]
    for p, q in zip(s1, s2):
        assert p.L == q.L and np.array_equal(p.exps, q.exps) and len(p.defects) == len(q.defects)
