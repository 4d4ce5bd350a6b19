#!/usr/bin/env python3
"""Throughput benchmark of the GB300 lattice Fock eigensolver.

Headline workload (the largest single-GPU configuration): one step solves,
per request, a Dirichlet box chain of 512 x 1 x 1 cells (n0 = 15, grid
8192 x 256 x 256, m0 = 32 GTOs per cell on one Z = 1 nucleus, rank R = 40,
lowest 64 eigenpairs: assembly + circulant embedding + preconditioned block
iteration) and a periodic 32 x 32 x 32 lattice (two sublattices, m0 = 32,
R = 40, all 1,048,576 eigenvalues: assembly + per-axis DFT + 32768 Fourier
block eigensolves).  value = solves per second (2 B solves per step) in the
FP64 form, all inputs resident in HBM when the timed region starts; mixed =
the same batch in the mixed form (tensor-core split-product assembly, FP32
phase of the box iteration); e2e = the FP64 batch through fock_solve with
host inputs and outputs.  The other workloads (the 64-cell chain pair in a
batch of 512, the 16^3 lattice) are timed the same way with fewer steps and
reported under other_configs; the serving stream (continuous batching) and
the CPU oracle are side legs at N = 1.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import dataclasses
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import lattice_inputs as li  # noqa: E402

METRIC = "lattice Fock solves/s"
UNIT = "solves/s"
L_CHAIN, N0, PAD, NPERP, R_RANK, K_EIG = 64, 15, 32, 256, 32, 16
FALLBACK_HBM_GBS, FALLBACK_BF16_TFLOPS = 6800.0, 1900.0


def workload(batch, rank):
    """The 64-cell chain pair: B box chains, then their periodic counterparts."""
    box = [li.config2(rank * batch + r, L=L_CHAIN, n0=N0, pad=PAD, n_perp=NPERP, R=R_RANK)
           for r in range(batch)]
    for p in box:
        p.k_eig = K_EIG
    per = [p.as_periodic_chain() for p in box]
    for p in per:
        p.k_eig = 0
    return box + per


def workload_large(batch, rank):
    """The headline: B box chains of 512 cells (m0 = 32, lowest 64) and B
    periodic 32^3 lattices (m0 = 32), one of each per request."""
    box = [li.config5_box(rank * batch + r) for r in range(batch)]
    per = [li.config5_periodic(rank * batch + r) for r in range(batch)]
    return box + per


def workload_cubes(batch, rank):
    """B periodic 16^3 lattices (two sublattices, m0 = 16, R = 32)."""
    return [li.config3(rank * batch + r) for r in range(batch)]


def config_dict(batch, world):
    return {"workload": "box chain 512x1x1 (n0=15, grid 8192x256x256, m0=32, R=40, lowest 64) + periodic "
                        "32x32x32 lattice (n0=16, grid 512^3, two sublattices, m0=32, R=40, all eigenvalues); "
                        f"{batch} of each per GPU",
            "requests_per_gpu": batch, "solves_per_step_per_gpu": 2 * batch,
            "parallelism": f"replicas x{world}", "l2": "flushed between timed steps (512 MB write)"}


def config_dict_chain64(batch):
    return {"workload": f"box chain {L_CHAIN}x1x1 (n0={N0}, grid {L_CHAIN * N0 + 2 * PAD}x{NPERP}x{NPERP}, "
                        f"m0=8, R={R_RANK}, lowest {K_EIG}) + periodic counterpart (all eigenvalues); "
                        f"batch {batch} requests/GPU", "solves_per_step_per_gpu": 2 * batch}


# --------------------------------------------------------------- serving
def serving_requests(n, seed):
    """Requests shaped like the serving mix (chains 4..256 cells with 0-4
    vacancy / substitution defects, cubes 8..24^3, m0 in {4, 8, 16}, periodic
    or box); the library's default quadrature rule."""
    return li.serving_stream(n, seed=seed)


def latency_summary(lat_ms, structured):
    """p50 / p99 of request latencies overall and per kind (periodic: one
    pass; structured: box chains and defects, iterated)."""
    lat = np.asarray(lat_ms, float)
    st = np.asarray(structured, bool)
    out = {}
    for name, sel in (("", np.ones(len(lat), bool)), ("_periodic", ~st), ("_structured", st)):
        if sel.any():
            out["p50_ms" + name] = float(np.percentile(lat[sel], 50))
            out["p99_ms" + name] = float(np.percentile(lat[sel], 99))
    out["n_periodic"] = int((~st).sum())
    out["n_structured"] = int(st.sum())
    return out


def _poll_all(srv, tickets, deadline):
    """Every ticket's result, or TimeoutError once `deadline` (perf_counter
    seconds) has passed with results outstanding."""
    out = []
    for t in tickets:
        left_ms = int(1000 * (deadline - time.perf_counter()))
        r = srv.poll(t, timeout_ms=max(left_ms, 1))
        if r is None:
            raise TimeoutError(f"{len(tickets) - len(out)} of {len(tickets)} serving results "
                               "outstanding at the deadline")
        out.append(r)
    return out


def _poisson_stream(fock, dev, reqs, rate, seed, slots, max_batch, limit_s):
    """Submit `reqs` with exponential gaps at `rate` per second to a fresh
    server; (results, wall seconds from the first submit, server stats)."""
    gaps = np.random.default_rng(seed).exponential(1.0 / rate, size=len(reqs))
    srv = fock.Server(dev, slots=slots, max_batch=max_batch)
    tickets = []
    t0 = time.perf_counter()
    nxt = t0
    for p, g in zip(reqs, gaps):
        nxt += g
        d = nxt - time.perf_counter()
        if d > 0:
            time.sleep(d)
        tickets.append(srv.submit(p))
    res = _poll_all(srv, tickets, time.perf_counter() + limit_s)
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.stop()
    return res, wall, st


def serving_run(fock, dev, n_stream=512, n_burst=128, n_sweep=128, slots=2, max_batch=64, limit_s=300.0):
    """Continuous batching (fock_serve_*) against the plain per-lattice FP64
    path (one fock_solve per request, one after the other), both on the same
    burst of n_burst requests of the serving mix: solves/s of each.  The
    server solves the burst in the FP64 form and in the mixed form; the
    mixed results are compared with the plain FP64 ones request by request
    (largest |difference| / max |lambda| over each request's eigenvalues), and
    the batched FP64 results must equal the plain ones bit for bit (a result
    does not depend on its batch).  Then n_stream requests with Poisson
    arrivals at 80 % of the mixed burst capacity, in the mixed form: p50 / p99
    latency (done - submit, server clock) and the stream's throughput."""
    burst = serving_requests(n_burst, seed=3100)
    mburst = mixed_of(burst)

    def batched(ps):
        srv = fock.Server(dev, slots=slots, max_batch=max_batch)
        _poll_all(srv, [srv.submit(p) for p in ps[:8]], time.perf_counter() + limit_s)   # warm-up
        t0 = time.perf_counter()
        res = _poll_all(srv, [srv.submit(p) for p in ps], t0 + limit_s)
        rate = len(ps) / (time.perf_counter() - t0)
        srv.stop()
        return rate, res

    cap64, r64 = batched(burst)
    capm, rm = batched(mburst)
    ctx = fock.Context(dev)
    ctx.solve([burst[0]], check=False)
    t1 = time.perf_counter()
    rp = [ctx.solve([p], check=False)[0] for p in burst]
    plain = len(burst) / (time.perf_counter() - t1)
    ctx.close()
    same = all(np.array_equal(a["evals"], b["evals"]) for a, b in zip(r64, rp))
    diff, diff_all = max_rel_diff(rp, rm, 64), max_rel_diff(rp, rm)

    stream = mixed_of(serving_requests(n_stream, seed=3000))
    rate = 0.8 * capm
    res, wall, st = _poisson_stream(fock, dev, stream, rate, 7, slots, max_batch, limit_s)
    lat = np.array([(r["t_done_ns"] - r["t_submit_ns"]) / 1e6 for r in res])
    # arrival-rate sweep: n_sweep requests at 0.5, 1 and 1.5 times the mixed capacity
    sweep = []
    sweep_runs = []
    for f in (0.5, 1.0, 1.5):
        reqs = mixed_of(serving_requests(n_sweep, seed=3300 + int(10 * f)))
        sr, sw, _ = _poisson_stream(fock, dev, reqs, f * capm, 11, slots, max_batch, limit_s)
        sl = np.array([(r["t_done_ns"] - r["t_submit_ns"]) / 1e6 for r in sr])
        sweep.append({"rate_over_capacity": f, "arrival_per_s": f * capm, "throughput": len(reqs) / sw,
                      "p50_ms": float(np.percentile(sl, 50)), "p99_ms": float(np.percentile(sl, 99)),
                      "status_ok": int(sum(r["status"] == 0 for r in sr))})
        sweep_runs.append((f"sweep_{f}", reqs, sr))
    runs = (("burst_fp64", burst, r64), ("burst_mixed", mburst, rm), ("plain_fp64", burst, rp),
            ("stream_mixed", stream, res)) + tuple(sweep_runs)
    ok = sum(r["status"] == 0 for _, _, rs_ in runs for r in rs_)
    total = sum(len(rs_) for _, _, rs_ in runs)
    fails = [{"run": nm, "i": i, "status": r["status"], "L": list(p.L), "periodic": list(p.periodic),
              "m0": len(p.exps), "k": p.k_eig, "iters": r["iters"], "resid": r["resid"]}
             for nm, ps_, rs_ in runs for i, (p, r) in enumerate(zip(ps_, rs_)) if r["status"] != 0][:8]
    out = {"burst_requests": n_burst, "batched_fp64": cap64, "batched_mixed": capm,
           "plain_per_lattice_fp64": plain, "unit": UNIT,
           "mixed_vs_plain": capm / plain, "fp64_batched_vs_plain": cap64 / plain,
           "batched_fp64_equals_plain_bitwise": bool(same),
           "max_rel_eig_diff_mixed_vs_plain_fp64": diff,
           "max_rel_eig_diff_mixed_vs_plain_fp64_all": diff_all,
           "diff_note": "lowest 64 eigenvalues of each request; _all: every eigenvalue.  The periodic cubes "
                        "of the mix have overlap blocks near the dependency cut: their eigenvalues are fixed "
                        "by the data only to about u / (overlap eigenvalue) x ||x||^2 in either form, the "
                        "per-eigenvalue bar within which tests/test_gpu_large.py checks both forms against "
                        "the oracle's stored 16^3 and 32^3 spectra",
           "requests": n_stream, "arrival": f"Poisson at 80% of the mixed burst capacity ({rate:.1f}/s)",
           "throughput": n_stream / wall, "arrival_sweep": sweep}
    out.update(latency_summary(lat, [bool(p.is_box or p.defects) for p in stream]))
    out.update({"slots": slots, "max_batch": max_batch, "batches": int(st["batches"]),
                "max_inflight": int(st["max_inflight"]),
                "peak_reserved_bytes": int(st["peak_reserved_bytes"]), "status_ok": int(ok),
                "status_total": int(total), "failures": fails,
                "mix": "chains 4..256 cells x1x1 (box or periodic) and periodic cubes 8,12,16,24^3; "
                       "m0 4/8/16; n0 16, N_perp 256, R 32; 0-4 defects per chain",
                "admission": "head of the queue, then later requests of the same kind "
                             "(periodic / structured)"})
    return out


# --------------------------------------------------------------- CPU oracle
def oracle_sample(npairs, seed0=0):
    """Time the CPU oracle on npairs (box, periodic) 64-cell chain requests."""
    from oracle import blocks, sinc
    ps = []
    for r in range(npairs):
        b = li.config2(seed0 + r, L=L_CHAIN, n0=N0, pad=PAD, n_perp=NPERP, R=R_RANK)
        b.k_eig = K_EIG
        ps += [b, b.as_periodic_chain()]
    t0 = time.perf_counter()
    for p in ps:
        t, c, _ = sinc.table_for(p)
        q = p.with_table(t, c)
        q.k_eig = p.k_eig
        blocks.solve(q)
    dt = time.perf_counter() - t0
    return len(ps), dt


def oracle_large_sample(seed=0, k3_cells=2, nblocks=32, pairs=16, cols=256, eig_order=2048):
    """Bounded sample of the CPU oracle on one headline request (one 512-cell
    box chain and one 32^3 lattice), each part timed and scaled to the whole
    solve by the fraction of the oracle's work it covers:

    periodic 32^3: the 3D contraction of the first block column (the oracle's
    generator route) for the lattice offsets k3 < k3_cells (x 32 / k3_cells),
    then for `nblocks` Fourier blocks the direct DFT over those offsets
    (x 32 / k3_cells per block) and the block pencil by LAPACK, x 32768 /
    nblocks;  box chain: the transverse contraction of the potential (whole),
    the axis-0 quadratic forms for `cols` of the 16384 basis columns and the
    per-pair potential contraction for `pairs` of the 1024 (mu, nu) pairs
    (each scaled by its fraction), and LAPACK's generalized eigensolver (64
    lowest) on the leading principal pencil of order eig_order, scaled by
    (N_b / eig_order)^3 (the dense route's cubic cost).  Returns (seconds per
    request estimated, description)."""
    import scipy.linalg
    from oracle import blocks, dense, grid, sinc

    def tab(p):
        t, c, _ = sinc.table_for(p)
        return p.with_table(t, c)
    # ---- periodic 32^3 ----
    p = tab(li.config5_periodic(seed))
    t0 = time.perf_counter()
    forms = dense.axis_forms(p)
    slab_of, slabs = grid.potential_slabs(p)
    Gs = [forms[0][0], forms[1][0], forms[2][0][:, :k3_cells]]
    V = dense._contract(p, Gs, slab_of, slabs, col_cells=0)
    L1, L2, L3 = p.L
    sl = [forms[a][1][:, :, 0, :] for a in range(3)]
    al = [forms[a][2][:, :, 0, :] for a in range(3)]
    k1, k2, k3 = np.meshgrid(np.arange(L1), np.arange(L2), np.arange(k3_cells), indexing="ij")
    Sk = sl[0][k1] * sl[1][k2] * sl[2][k3]
    Hk = 0.5 * (al[0][k1] * sl[1][k2] * sl[2][k3] + sl[0][k1] * al[1][k2] * sl[2][k3]
                + sl[0][k1] * sl[1][k2] * al[2][k3]) - V.reshape(L1, L2, k3_cells, p.m0, p.m0)
    t_gen = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    t1 = time.perf_counter()
    tau = blocks.null_threshold(p)
    for _ in range(nblocks):
        j = rng.integers(0, [L1, L2, L3])
        w = np.exp(-2j * np.pi * (j[0] * k1 / L1 + j[1] * k2 / L2 + j[2] * k3 / L3))
        Hb = np.tensordot(w, Hk, axes=([0, 1, 2], [0, 1, 2]))
        Sb = np.tensordot(w, Sk, axes=([0, 1, 2], [0, 1, 2]))
        blocks.block_pencil(Hb, Sb, tau)
    t_blk = time.perf_counter() - t1
    t_per = t_gen * L3 / k3_cells + t_blk * (L3 / k3_cells) * p.ncell / nblocks
    # ---- box chain 512 ----
    q = tab(li.config5_box(seed))
    t2 = time.perf_counter()
    G1 = grid.basis_axis(q, 0)
    N1 = G1.shape[0]
    Gf = G1.reshape(N1, -1)
    tf = time.perf_counter()
    Gf.T @ (4.0 * Gf[:, :cols])                       # one axis-0 form product, `cols` columns
    t_form = time.perf_counter() - tf
    s_of, sl = grid.potential_slabs(q)
    G2 = grid.basis_axis(q, 1)[:, 0, :]
    G3 = grid.basis_axis(q, 2)[:, 0, :]
    GG3 = G3[:, :, None] * G3[:, None, :]
    GG2 = G2[:, :, None] * G2[:, None, :]
    W2 = np.stack([np.einsum("iab,iab->ab", GG2, np.tensordot(sl[s], GG3, axes=(1, 0)))
                   for s in range(sl.shape[0])])
    w = W2[s_of]
    t_tr = time.perf_counter()
    for pr in range(pairs):
        mu, nu = divmod(pr * 37 % (q.m0 * q.m0), q.m0)
        G1[:, :, mu].T @ (w[:, mu, nu, None] * G1[:, :, nu])
    t_pairs = time.perf_counter() - t_tr
    H = np.random.default_rng(seed).standard_normal((eig_order, eig_order))   # a definite pencil of
    A = H @ H.T / eig_order + np.eye(eig_order)                               # that order (timing only)
    t3 = time.perf_counter()
    scipy.linalg.eigh(0.5 * (H + H.T), A, subset_by_index=[0, 63])
    t_eig = time.perf_counter() - t3
    t_box = ((t_tr - t2 - t_form) + t_form * 2 * q.Nb / cols + t_pairs * (q.m0 * q.m0) / pairs
             + t_eig * (q.Nb / eig_order) ** 3)
    desc = (f"periodic 32^3: generator contraction for {k3_cells} of 32 offsets along axis 3 "
            f"({t_gen:.1f} s, x{L3 // k3_cells}), {nblocks} Fourier blocks by direct DFT + LAPACK "
            f"({t_blk:.1f} s, scaled to 32768 blocks); box 512: transverse potential contraction "
            f"({t_tr - t2 - t_form:.1f} s), a {cols}-column axis-0 form product ({t_form:.2f} s, scaled to "
            f"the two forms' 2 x 16384 columns), {pairs} of 1024 pair contractions "
            f"({t_pairs:.1f} s, scaled), LAPACK generalized eigensolver on order {eig_order} "
            f"({t_eig:.2f} s, scaled by (N_b/{eig_order})^3)")
    return t_per + t_box, desc, {"periodic_s": t_per, "box_s": t_box}


def oracle_sample_one_thread(npairs):
    """The oracle sample in a fresh interpreter whose BLAS / OpenMP pools are
    limited to one thread (the limit must be set before numpy loads)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", str(npairs)],
                       env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return None
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["n"], d["dt"]


def cpu_baseline(npairs, one_thread_pairs=2):
    """The oracle on the host cores: the headline request by a bounded,
    scaled sample (oracle_large_sample), and the 64-cell chain pair timed
    whole."""
    t_req, desc, parts = oracle_large_sample()
    out = {"value": 2.0 / t_req, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
           "sample": desc, "seconds_per_request_estimated": t_req, **parts}
    n, dt = oracle_sample(npairs)
    out["chain64_pair"] = {"value": n / dt, "unit": UNIT,
                           "sample": f"{npairs} box + {npairs} periodic 64-cell chain requests (dense FP64 "
                                     f"Galerkin matrices by 3D grid contraction + LAPACK eigh), {dt:.1f} s"}
    if one_thread_pairs > 0:
        one = oracle_sample_one_thread(one_thread_pairs)
        if one is not None:
            out["chain64_pair"]["value_1thread"] = one[0] / one[1]
    return out


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle as it stands, on bounded samples of
    the headline workload (oracle_large_sample), one request per step."""
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_large_sample(seed=0, nblocks=8, pairs=2, cols=32, eig_order=512)
    tot, desc = 0.0, ""
    for s in range(args.steps):
        t_req, desc, _ = oracle_large_sample(seed=s)
        tot += t_req
    val = 2.0 * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(1, world),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": "per step one request, estimated from a bounded sample: " + desc},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- work models
def _conjugate_classes(L):
    """Fourier indices solved once: a block and its conjugate at -j share one
    eigensolve (the conjugate of the block at j, same spectrum)."""
    L1, L2, L3 = L
    seen = 0
    for j1 in range(L1):
        for j2 in range(L2):
            for j3 in range(L3):
                m = (((L1 - j1) % L1) * L2 + (L2 - j2) % L2) * L3 + (L3 - j3) % L3
                if m >= (j1 * L2 + j2) * L3 + j3:
                    seen += 1
    return seen


def fp64_flops_per_step(problems, outs):
    """Algorithmic FP64 operation counts of the kernels of one step (the
    models written out below), keyed by kernel timer name."""
    w = {}
    for p, o in zip(problems, outs):
        m0 = len(p.exps)
        if p.is_box or p.defects:
            k = p.k_eig
            n = p.L[0] * m0
            it = max(o["iters"], 1)
            # block size kb (k wanted + guards, or the whole space) and basis 3 kb
            kb = n if 3 * n <= 255 else k + max(4, k // 8)
            nb = 3 * kb
            # Rayleigh-Ritz per launch: pivoted LDL^T nb^3/3, the two triangular
            # solves 4 nb^3/3, Householder tridiagonal 4 nb^3/3, back-transformation
            # and coefficients 3 nb^2 kb, Cholesky-QR and Ritz projection 6 nb kb^2;
            # `it` launches on 3 kb columns plus the start on kb
            rr = lambda b: 3 * b ** 3 + 3 * b * b * kb + 6 * b * kb * kb
            w["k_rr"] = w.get("k_rr", 0) + it * rr(nb) + rr(kb)
            # Gram products: the two symmetric nb x nb products of the basis
            # (n nb (nb + 1) flops each), the kb x kb projection of W onto X and the
            # coefficient projection's z_X^T (G_S z_P) (nb rows); the start: the two
            # symmetric kb x kb products
            w["k_gemm_tn"] = (w.get("k_gemm_tn", 0) + it * (2 * n * nb * (nb + 1) + 2 * n * kb * kb
                                                            + 2 * nb * kb * kb)
                              + 2 * n * kb * (kb + 1))
            # basis update [X|P] = Y Cc, W -= X C, and the coefficient projection
            # G_S z_P (nb x nb x kb) and z_P -= z_X M (nb x kb x kb)
            w["k_gemm_nn"] = (w.get("k_gemm_nn", 0)
                              + it * (2 * n * nb * 2 * kb + 2 * n * kb * kb + 2 * nb * nb * kb + 2 * nb * kb * kb))
            # banded preconditioner: forward and backward block substitution over
            # L cells with D + 1 blocks of m0 x m0 per block row, kb columns
            D = o.get("D")
            # the library's rule: the banded factor when 2 L D^2 m0^3 <= 4e9
            band = D is not None and 2.0 * p.L[0] * D * D * m0 ** 3 <= 4e9
            if band:
                w["k_band_solve"] = w.get("k_band_solve", 0) + it * 4 * p.L[0] * (D + 1) * m0 * m0 * kb
            # circulant-embedding FFTs: per iteration 9 kb m0 column transforms (forward of W
            # and [X|P], inverse of their H and S images), 12 kb m0 at start; conventional
            # 5 M log2 M flops per complex transform of length M
            M = o.get("M")
            if M:
                w["k_fft"] = w.get("k_fft", 0) + (it * 9 + 12) * kb * m0 * 5 * M * math.log2(M)
                # block products at every frequency: a complex m0 x m0 block times
                # ncol / 2 packed columns (8 m0^2 flops per packed column), H and S on
                # W (kb columns) and on [X | P] (2 kb) per iteration, twice on [X | P]
                # at start; the circulant preconditioner (one operator on kb) when
                # the chain has no band factor
                bm = lambda ncol, nop: nop * 8 * M * m0 * m0 * (ncol / 2)
                pre = 0 if band else bm(kb, 1)
                w["k_blockmul"] = (w.get("k_blockmul", 0) + it * (bm(kb, 2) + bm(2 * kb, 2) + pre)
                                   + 2 * bm(2 * kb, 2))
        else:
            T = len(p.Z) * p.R
            # per Fourier block solved (conjugate pairs once): Hadamard combine over
            # T+3 factor terms on the upper triangle (complex, ~20 flops per entry
            # and term), then by the route the block took.  Cholesky route:
            # reduction C = L^-1 Hbar L^-H (~m0^3 complex multiply-adds = 8 m0^3).
            # Eigendecomposition route (a direction at the dependency cut): complex
            # Householder tridiagonal of Sbar (16/3 m0^3), QL with its rotations
            # accumulated (~6 m0^3), back-transformation (8 m0^3), C = X^H Hbar X
            # (16 m0^3).  Both: Householder tridiagonal of C (16/3 m0^3), Sturm
            # bisection (m0 eigenvalues x 55 steps x 3 m0)
            form = (T + 3) * m0 * (m0 + 1) // 2 * 20 + 16 / 3 * m0 ** 3 + 55 * 3 * m0 * m0
            chol = form + 8 * m0 ** 3
            eig = form + (16 / 3 + 6 + 8 + 16) * m0 ** 3
            ncls = _conjugate_classes(p.L)
            neig = min(int(o.get("n_eig", 0)), ncls)
            w["k_fblocks_eig"] = w.get("k_fblocks_eig", 0) + neig * eig + (ncls - neig) * chol
    return w


def matvec_bytes_per_step(problems, outs):
    """Algorithmic HBM bytes of the embedded matvec (k_fft + k_blockmul +
    k_eapply) of one step: per application to ncol columns, the Fourier blocks
    of H and S (M m0^2 complex each), the boundary / defect blocks, the
    columns in and their two images out; the FFT intermediates counted as
    on-chip.  Per iteration [X | P] (2 kb columns) and W (kb), at start 2 x
    [X | P]."""
    tot = 0
    for p, o in zip(problems, outs):
        if not (p.is_box or p.defects) or not o.get("M"):
            continue
        m0 = len(p.exps)
        n = p.L[0] * m0
        kb = n if 3 * n <= 255 else p.k_eig + max(4, p.k_eig // 8)
        M, nE = o["M"], o.get("nE", 0)
        per_app = lambda ncol: 2 * M * m0 * m0 * 16 + 2 * nE * m0 * m0 * 8 + 3 * n * ncol * 8
        it = max(o["iters"], 1)
        tot += it * (per_app(2 * kb) + per_app(kb)) + 2 * per_app(2 * kb)
    return tot


def load_peaks():
    """HBM GB/s and dense BF16 TFLOP/s measured on this machine
    (MEASURED_PEAKS.json, written by the driver), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, FALLBACK_BF16_TFLOPS, "fallback"


# --------------------------------------------------------------- timing
def timed_plan(ctx, stream, problems, steps, warmup, flush, maxit=1000, profile=False):
    """W untimed executions, then K executions timed with CUDA events on the
    context's stream, L2 flushed before each.  With `profile`, K more
    executions with the library's kernel timers on (the periodic and the
    structured pipelines then run one after the other instead of
    concurrently, so each timer holds its kernel alone).  Returns (ms total,
    outputs, per-kernel timers, plan, ms total of the timer pass)."""
    import torch
    plan = ctx.plan(problems)
    for _ in range(warmup):
        plan.execute(maxit=maxit)
    outs = plan.outputs(check=False)
    for i, o in enumerate(outs):
        _, o["M"], o["D"], o["nE"] = plan.sizes(i)
        o["n_eig"] = plan.block_routes(i)

    def run():
        torch.cuda.synchronize()
        tot = 0.0
        for s in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(s))
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plan.execute(maxit=maxit)
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b)
        return tot

    ms = run()
    prof, prof_ms = {}, None
    if profile:
        ctx.profile(True)
        ctx.profile_reset()
        prof_ms = run()
        prof = ctx.profile_read()
        ctx.profile(False)
    return ms, outs, prof, plan, prof_ms


def mixed_of(problems):
    out = []
    for q in problems:
        r = dataclasses.replace(q, precision=1)
        r.k_eig = q.k_eig
        out.append(r)
    return out


def max_rel_diff(outs, mouts, lowest=None):
    """Largest |mixed - FP64| / max|lambda| over the problems' eigenvalues
    (the `lowest` of each problem only when given: a periodic lattice's whole
    spectrum includes eigenvalues whose eigenvectors lean on overlap
    directions near the dependency cut, determined by the data only to
    ~u / (their overlap eigenvalue), in either form)."""
    rel = 0.0
    for o, mo in zip(outs, mouts):
        a, b = np.asarray(o["evals"]), np.asarray(mo["evals"])
        if lowest is not None:
            a, b = a[:lowest], b[:lowest]
        f = np.isfinite(a) & np.isfinite(b)
        if f.any():
            rel = max(rel, float(np.max(np.abs(b[f] - a[f])) / np.max(np.abs(a[f]))))
    return rel


def roof(name, bound, work, prof, steps, peak, unit, peak_source, step_ms, scale=1e12):
    """Achieved rate of one kernel (algorithmic work per launch / its mean
    launch time from the live CUDA-event timers) against a peak."""
    if name not in prof or not work:
        return None
    nl, dms = prof[name]
    per_launch = work * steps / nl
    achieved = per_launch / (dms / nl / 1e3) / scale
    return {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": None, "peak_source": peak_source,
            "share_of_step": dms / step_ms, "launches_per_step": nl / steps,
            "timers": "kernel-timer pass (pipelines serial; share of that pass's step)"}


# --------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=8, help="requests (box + periodic) per GPU and step")
    ap.add_argument("--chain-batch", type=int, default=512)
    ap.add_argument("--cube-batch", type=int, default=8)
    ap.add_argument("--cpu-pairs", type=int, default=8)
    ap.add_argument("--ref-pairs", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other", action="store_true")
    ap.add_argument("--profile-json", default="")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=512)
    ap.add_argument("--maxit", type=int, default=1000)
    ap.add_argument("--oracle-sample", type=int, default=0, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_sample:   # child of cpu_baseline: time the oracle only, print one JSON line
        n, dt = oracle_sample(args.oracle_sample)
        print(json.dumps({"n": n, "dt": dt}), flush=True)
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    from paper_1702_00339_gb300 import build, fock
    build.build()
    torch.cuda.set_device(local)
    dev = local
    stream = torch.cuda.Stream(device=dev)
    ctx = fock.Context(dev, stream=stream.cuda_stream)
    fp64_peak, fp32_peak = fock.measure_peaks(dev)
    hbm_peak, bf16_peak, peak_kind = load_peaks()
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=dev)   # 512 MB > L2
    problems = workload_large(args.batch, rank)
    nsolve = len(problems)

    # ---- device-resident timing, FP64 form ----
    clocks = ClockSampler(dev)
    clocks.start()
    if world > 1:
        dist.barrier()
    ms, outs, prof, plan, pms = timed_plan(ctx, stream, problems, args.steps, args.warmup, flush, args.maxit,
                                      profile=True)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = nsolve * world * args.steps / (ms_max / 1e3)
    bad = [o["status"] for o in outs if o["status"] != 0]

    # ---- mixed form of the same batch ----
    mms, mouts, mprof, mplan, mpms = timed_plan(ctx, stream, mixed_of(problems), args.steps, args.warmup, flush,
                                          args.maxit, profile=True)
    split_units = mplan.split_work()
    mplan.close()
    mt = torch.tensor([mms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(mt, op=dist.ReduceOp.MAX)
    mixed_val = nsolve * world * args.steps / (float(mt.item()) / 1e3)
    mixed = {"value": mixed_val, "unit": UNIT, "ms_per_step": float(mt.item()) / args.steps,
             "serial_ms_per_step": mpms / args.steps,
             "vs_fp64": mixed_val / value, "max_rel_eig_diff_vs_fp64": max_rel_diff(outs, mouts, 64),
             "max_rel_eig_diff_vs_fp64_all": max_rel_diff(outs, mouts),
             "max_rel_eig_diff_vs_fp64_box": max_rel_diff(outs[:args.batch], mouts[:args.batch], 64),
             "max_rel_eig_diff_vs_fp64_periodic": max_rel_diff(outs[args.batch:], mouts[args.batch:], 64),
             "stated_bar": 1e-8,
             "bar_note": "per eigenvalue max(1e-8 max|lambda|, 256 u (||H||inf + |lambda_i| ||S||inf) ||x_i||^2): "
                         "the second term is the rounding floor of the data, which both forms share; on the "
                         "periodic lattices (overlap blocks with condition numbers near 1e9) it exceeds the "
                         "first. Both forms are checked against stored oracle results at these sizes by "
                         "tests/test_gpu_large.py",
             "statuses_nonzero": sum(1 for o in mouts if o["status"] != 0),
             "box_iters": [int(o["iters"]) for o in mouts[:args.batch]],
             "form": "FOCK_MIXED: the assembly's quadrature contractions and the block iteration's Gram "
                     "and basis products as exact split products on tcgen05 tensor cores (BF16 digits, "
                     "FP32 TMEM sums, FP64 combination); Rayleigh-Ritz, matvecs, preconditioner and "
                     "Fourier-block eigensolves FP64"}

    # ---- end to end through fock_solve (host inputs and outputs) ----
    e2e_steps = max(1, min(args.steps, 2))
    ctx.solve(problems, check=False)   # grows the context arena once, outside the timed loop
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        res = ctx.solve(problems, check=False)
    torch.cuda.synchronize()
    te = time.perf_counter() - t0
    te_t = torch.tensor([te], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(te_t, op=dist.ReduceOp.MAX)
    e2e_val = nsolve * world * e2e_steps / float(te_t.item())
    d2h = sum(8 * r["n_evals"] + (4 * r["n_evals"] if r["block_of"] is not None else 0) for r in res)

    # ---- rooflines: dominant kernel of the step, and one per stage ----
    step_ms = ms / args.steps
    launches = sum(v[0] for v in prof.values())
    flops = fp64_flops_per_step(problems, outs)
    f64src = f"FP64 FMA throughput measured live by fock_measure_peaks ({fp64_peak:.3f} TFLOP/s)"
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0]
    main_roof = roof(dom, "alu", flops.get(dom), prof, args.steps, fp64_peak, "TFLOP/s", f64src, pms)
    if main_roof is None:
        main_roof = {"kernel": dom, "bound": "alu", "achieved": None, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": None, "traffic": None, "share_of_step": prof[dom][1] / pms}
    stages = {}
    stages["b3_block_eigensolves"] = roof("k_fblocks_eig", "alu", flops.get("k_fblocks_eig"), prof, args.steps,
                                          fp64_peak, "TFLOP/s", f64src, pms)
    stages["c4_rayleigh_ritz"] = roof("k_rr", "alu", flops.get("k_rr"), prof, args.steps, fp64_peak,
                                      "TFLOP/s", f64src, pms)
    stages["c4_gram_products"] = roof("k_gemm_tn", "alu", flops.get("k_gemm_tn"), prof, args.steps, fp64_peak,
                                      "TFLOP/s", f64src, pms)
    stages["c3_block_products"] = roof("k_blockmul", "alu", flops.get("k_blockmul"), prof, args.steps, fp64_peak,
                                       "TFLOP/s", f64src, pms)
    mv_ms = sum(prof[k][1] for k in ("k_fft", "k_blockmul", "k_eapply") if k in prof)
    mvb = matvec_bytes_per_step(problems, outs)
    if mv_ms > 0 and mvb:
        gbs = mvb * args.steps / (mv_ms / 1e3) / 1e9
        stages["c3_embedded_matvec"] = {"kernels": "k_fft + k_blockmul + k_eapply", "bound": "hbm",
                                        "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                                        "frac": gbs / hbm_peak, "peak_source": f"{peak_kind} HBM copy",
                                        "algorithmic_bytes_per_step": mvb, "share_of_step": mv_ms / pms,
                                        "working_set": "Fourier blocks of H and S + E blocks + [X|P|W] and "
                                                       "their images of the step's box chains"}
    if "k_split_gemm" in mprof and split_units:
        nl, sms = mprof["k_split_gemm"]
        tens = split_units["tensor_flops"] * args.steps / (sms / 1e3) / 1e12
        stages["a3_split_product_assembly"] = {
            "kernel": "k_split_gemm", "bound": "tensor", "achieved": tens, "peak": bf16_peak,
            "unit": "TFLOP/s", "frac": tens / bf16_peak, "peak_source": f"{peak_kind} dense BF16 (cuBLAS)",
            "fp64_equivalent_tflops": split_units["fp64_flops"] * args.steps / (sms / 1e3) / 1e12,
            "ms_per_step": sms / args.steps, "launches_per_step": nl / args.steps}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args.batch, world),
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(plan.upload_bytes),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches), "roofline": main_roof, "stage_rooflines": stages,
            "serial_ms_per_step": pms / args.steps, "tuning": plan.tuning(),
            "measured_peaks": {"fp64_tflops": fp64_peak, "fp32_tflops": fp32_peak, "hbm_gbs": hbm_peak,
                               "bf16_tflops": bf16_peak, "hbm_bf16_source": peak_kind},
            "clocks": clk, "mixed": mixed,
            "box_iters": [int(o["iters"]) for o in outs[:args.batch]],
            "statuses_nonzero": len(bad), "maxit": args.maxit}
    plan.close()
    if args.profile_json and rank == 0:
        with open(args.profile_json, "w") as f:
            json.dump({"fp64": {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items()},
                       "mixed": {k: {"launches": v[0], "ms": v[1]} for k, v in mprof.items()}}, f, indent=1)

    # ---- the other workloads (N = 1 only; fewer steps) ----
    if not args.no_other and world == 1:
        other = {}
        try:
            ps = workload(args.chain_batch, rank)
            o_ms, o_outs, o_prof, o_plan, o_pms = timed_plan(ctx, stream, ps, 2, 1, flush, profile=True)
            o_plan.close()
            m_ms, m_outs, _, m_plan, _ = timed_plan(ctx, stream, mixed_of(ps), 2, 1, flush)
            m_plan.close()
            o_fl = fp64_flops_per_step(ps, o_outs)
            o_dom = max(o_prof.items(), key=lambda kv: kv[1][1])[0]
            other["chain64_pair"] = {"config": config_dict_chain64(args.chain_batch),
                                     "value": len(ps) * 2 / (o_ms / 1e3), "unit": UNIT,
                                     "ms_per_step": o_ms / 2,
                                     "mixed_value": len(ps) * 2 / (m_ms / 1e3),
                                     "max_rel_eig_diff_mixed_vs_fp64": max_rel_diff(o_outs, m_outs, 16),
                                     "statuses_nonzero": sum(1 for o in o_outs if o["status"] != 0),
                                     "roofline": roof(o_dom, "alu", o_fl.get(o_dom), o_prof, 2, fp64_peak,
                                                      "TFLOP/s", f64src, o_pms)}
        except Exception as e:   # noqa: BLE001
            other["chain64_pair"] = {"error": f"{type(e).__name__}: {e}"}
        try:
            ps = workload_cubes(args.cube_batch, rank)
            c_ms, c_outs, c_prof, c_plan, c_pms = timed_plan(ctx, stream, ps, 2, 1, flush, profile=True)
            c_plan.close()
            cm_ms, cm_outs, _, cm_plan, _ = timed_plan(ctx, stream, mixed_of(ps), 2, 1, flush)
            cm_plan.close()
            c_fl = fp64_flops_per_step(ps, c_outs)
            other["cube16"] = {"config": {"workload": "periodic 16x16x16 lattice (n0=32, grid 512^3, two "
                                                      "sublattices Z in {1,2,3}, m0=16, R=32, all 65536 "
                                                      f"eigenvalues); batch {args.cube_batch}"},
                               "value": len(ps) * 2 / (c_ms / 1e3), "unit": UNIT, "ms_per_step": c_ms / 2,
                               "mixed_value": len(ps) * 2 / (cm_ms / 1e3),
                               "max_rel_eig_diff_mixed_vs_fp64": max_rel_diff(c_outs, cm_outs, 64),
                               "max_rel_eig_diff_mixed_vs_fp64_all": max_rel_diff(c_outs, cm_outs),
                               "roofline": roof("k_fblocks_eig", "alu", c_fl.get("k_fblocks_eig"), c_prof, 2,
                                                fp64_peak, "TFLOP/s", f64src, c_pms)}
        except Exception as e:   # noqa: BLE001
            other["cube16"] = {"error": f"{type(e).__name__}: {e}"}
        try:
            ps = [li.config5_box(rank * args.batch + r) for r in range(args.batch)]
            b_ms, b_outs, b_prof, b_plan, b_pms = timed_plan(ctx, stream, ps, 2, 1, flush, args.maxit, profile=True)
            b_plan.close()
            bm_ms, bm_outs, _, bm_plan, _ = timed_plan(ctx, stream, mixed_of(ps), 2, 1, flush, args.maxit)
            bm_plan.close()
            b_fl = fp64_flops_per_step(ps, b_outs)
            other["box512_only"] = {
                "config": {"workload": "box chain 512x1x1 (n0=15, grid 8192x256x256, m0=32, R=40, lowest 64) "
                                      f"without periodic problems; batch {args.batch}",
                           "rayleigh_ritz": "one thread-block cluster of 8 CTAs per chain (no periodic work "
                                            "to share the GPU with)"},
                "value": len(ps) * 2 / (b_ms / 1e3), "unit": UNIT, "ms_per_step": b_ms / 2,
                "mixed_value": len(ps) * 2 / (bm_ms / 1e3),
                "max_rel_eig_diff_mixed_vs_fp64": max_rel_diff(b_outs, bm_outs, 64),
                "statuses_nonzero": sum(1 for o in b_outs + bm_outs if o["status"] != 0),
                "roofline_rayleigh_ritz": roof("k_rr", "alu", b_fl.get("k_rr"), b_prof, 2, fp64_peak, "TFLOP/s",
                                               f64src, b_pms)}
        except Exception as e:   # noqa: BLE001
            other["box512_only"] = {"error": f"{type(e).__name__}: {e}"}
        line["other_configs"] = other

    if rank == 0:
        # the side legs (one GPU, N = 1 only) never cost the step's line: a failure
        # is reported in place
        if not args.no_serve and world == 1:
            try:
                line["serving"] = serving_run(fock, dev, n_stream=args.serve_requests)
            except Exception as e:   # noqa: BLE001
                line["serving"] = {"error": f"{type(e).__name__}: {e}"}
        if not args.no_cpu_baseline and world == 1:
            try:
                line["cpu_baseline"] = cpu_baseline(args.cpu_pairs)
            except Exception as e:   # noqa: BLE001
                line["cpu_baseline"] = {"error": f"{type(e).__name__}: {e}"}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
