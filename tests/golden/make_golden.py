"""Writes the stored oracle results of the large workloads (tests/golden/*.npz).

Calls only the CPU oracle (`oracle/`) and the seeded input module; nothing
here comes from the CUDA path.  Each file holds, for one seeded problem:

* periodic 16^3 (m0 = 16) and 32^3 (m0 = 32): the generator blocks A_k of H
  and S at sampled lattice offsets (3D grid contraction of the first block
  column, oracle.blocks.generators_direct); the spectra of Fourier blocks
  (direct DFT over every lattice offset, Eq. A.3; LAPACK on each block
  pencil under the dependency rule, Prop. A.1) -- every block of the 16^3
  lattice, a seeded sample of the 32^3 one -- with the squared norms of
  their S-normalised eigenvectors (the per-eigenvalue bar) and the variants
  of blocks with an overlap direction near the dependency cut;
* box chain 512 x 1 x 1 (m0 = 32, lowest 64): the dense H and S (oracle
  .dense.chain_matrices), the lowest 64 eigenpairs by LAPACK under the
  dependency rule (each variant of a cell direction near the cut), and
  sampled blocks: Toeplitz generators at an interior cell and the corner
  block of the first cell;
* ring 202 x 1 x 1 (m0 = 4, periodic, substitutions Z = 1 -> 3 at cells 92
  and 171; lowest 16): every level is a pair, exactly degenerate in double
  precision (two identical, distant defects on a ring).  The dense H and S
  (oracle.dense.build), the lowest 16 by LAPACK under the dependency rule.

Run: python tests/golden/make_golden.py [c3] [c5p] [c5box] [ring]   (minutes each;
the box chain needs ~20 GB of host memory).
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import lattice_inputs as li                      # noqa: E402
from oracle import blocks, dense, sinc          # noqa: E402


def _tab(p):
    t, c, _ = sinc.table_for(p)
    return p.with_table(t, c)


def _flips(amb, cap=3):
    import itertools
    amb = list(amb)[:cap]
    out = []
    for r in range(len(amb) + 1):
        out += [tuple(c) for c in itertools.combinations(amb, r)]
    return out


def periodic(p, name, jsample, ksample):
    t0 = time.time()
    gh, gs = blocks.generators_direct(p)
    print(f"{name}: generators {time.time() - t0:.0f} s", flush=True)
    tau = blocks.null_threshold(p)
    Hn = float(np.max(np.sum(np.abs(gh), axis=0).sum(axis=1)))   # largest row sum of |H|
    Sn = float(np.max(np.sum(np.abs(gs), axis=0).sum(axis=1)))
    L1, L2, L3 = p.L
    js, evs, vns, alt_j, alt_ev, alt_vn = [], [], [], [], [], []
    for jb in jsample:
        jc = (jb // (L2 * L3), (jb // L3) % L2, jb % L3)
        Hb, Sb, _ = blocks.fourier_block_from_generators(p, gh, gs, jc, tau=tau)
        w = np.linalg.eigvalsh(Sb)
        for n, f in enumerate(_flips(blocks.ambiguous(w, tau))):
            ev, V, r = blocks.block_pencil(Hb, Sb, tau, flip=f)
            vn = np.full(p.m0, np.inf)
            vn[:r] = np.sum(np.abs(V) ** 2, axis=0)
            if n == 0:
                js.append(jb); evs.append(ev); vns.append(vn)
            else:
                alt_j.append(jb); alt_ev.append(ev); alt_vn.append(vn)
    print(f"{name}: {len(js)} blocks, {len(alt_j)} variants, {time.time() - t0:.0f} s", flush=True)
    ev = np.array(evs)
    np.savez_compressed(os.path.join(HERE, name + ".npz"),
                        L=np.array(p.L), m0=p.m0, tau=tau, Hn=Hn, Sn=Sn,
                        k=np.array(ksample), gen_H=gh[ksample], gen_S=gs[ksample],
                        j=np.array(js), ev=ev, vn2=np.array(vns),
                        alt_j=np.array(alt_j, dtype=int), alt_ev=np.array(alt_ev).reshape(-1, p.m0),
                        alt_vn2=np.array(alt_vn).reshape(-1, p.m0),
                        scale=float(np.max(np.abs(ev[np.isfinite(ev)]))))


def box(p, name):
    t0 = time.time()
    H, S = dense.chain_matrices(p)
    print(f"{name}: matrices {time.time() - t0:.0f} s", flush=True)
    Hn = float(np.max(np.sum(np.abs(H), axis=1)))
    Sn = float(np.max(np.sum(np.abs(S), axis=1)))
    m0, L = p.m0, p.L[0]
    kc = L // 2
    ds = np.array([0, 1, 5])
    TH = np.array([H[(kc + d) * m0:(kc + d + 1) * m0, kc * m0:(kc + 1) * m0] for d in ds])
    TS = np.array([S[(kc + d) * m0:(kc + d + 1) * m0, kc * m0:(kc + 1) * m0] for d in ds])
    s, _, tau = blocks.cell_null_directions(p)
    evs, vns, kept = [], [], []
    for f in _flips(blocks.ambiguous(s, tau)):
        ev, V, r = blocks.box_eigs(p, H, S, tau=tau, vectors=True, flip=f)
        evs.append(ev); vns.append(np.sum(V * V, axis=0)); kept.append(r)
        print(f"{name}: variant {f} kept {r} {time.time() - t0:.0f} s", flush=True)
    np.savez_compressed(os.path.join(HERE, name + ".npz"),
                        L=np.array(p.L), m0=m0, k=p.k_eig, tau=tau, Hn=Hn, Sn=Sn, cell_eigs=s,
                        kc=kc, d=ds, T_H=TH, T_S=TS, C_H=H[:m0, :m0], C_S=S[:m0, :m0],
                        ev=np.array(evs), vn2=np.array(vns), kept=np.array(kept))


def ring(p, name):
    t0 = time.time()
    H, S = dense.build(p)
    print(f"{name}: matrices {time.time() - t0:.0f} s", flush=True)
    Hn = float(np.max(np.sum(np.abs(H), axis=1)))
    Sn = float(np.max(np.sum(np.abs(S), axis=1)))
    tau = blocks.null_threshold(p)
    s, _, _ = blocks.cell_null_directions(p, tau)
    evs, vns = [], []
    for f in _flips(blocks.ambiguous(s, tau)):
        ev, V, _ = blocks.box_eigs(p, H, S, tau=tau, vectors=True, flip=f)
        evs.append(ev); vns.append(np.sum(V * V, axis=0))
    np.savez_compressed(os.path.join(HERE, name + ".npz"), k=p.k_eig, Hn=Hn, Sn=Sn,
                        ev=np.array(evs), vn2=np.array(vns))


def ring_two_defects():
    """The ring 202 x 1 x 1 of the serving mix (request 328 of its stream
    with seed 3000: m0 = 4, two Z = 3 substitutions 79 cells apart)."""
    p = li.serving_stream(512, seed=3000)[328]
    assert p.L == (202, 1, 1) and p.periodic == (1, 0, 0) and len(p.defects) == 2
    q = _tab(p)
    q.k_eig = p.k_eig
    return q


if __name__ == "__main__":
    which = set(sys.argv[1:]) or {"c3", "c5p", "c5box", "ring"}
    rng = np.random.default_rng(20170201)
    if "c3" in which:
        p = _tab(li.config3(0))
        periodic(p, "config3_periodic_16cubed_seed0", list(range(p.ncell)),
                 sorted(set([0, 1, 17, 273, 4095] + list(rng.choice(p.ncell, 59, replace=False)))))
    if "c5p" in which:
        p = _tab(li.config5_periodic(0))
        corner = (16 * 32 + 16) * 32 + 16
        js = sorted(set([0, 1, 31, corner, p.ncell - 1] + list(rng.choice(p.ncell, 59, replace=False))))
        periodic(p, "config5_periodic_32cubed_seed0", js,
                 sorted(set([0, 1, 1057, corner] + list(rng.choice(p.ncell, 28, replace=False)))))
    if "c5box" in which:
        box(_tab(li.config5_box(0)), "config5_box_512_seed0")
    if "ring" in which:
        ring(ring_two_defects(), "ring_202_two_defects")
