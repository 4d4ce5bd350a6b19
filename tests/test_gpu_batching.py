"""Launch machinery of a plan: the FFT tuner, the CUDA graph of the block
iteration and the two-stream execution of periodic and structured problems.
None of them may change a result.  The graph replays the kernels of one
iteration with the arguments they were captured with, the FFT's column width
does not enter any column's arithmetic, and the two pipelines share no buffer
after the assembly.  With the kernel timers on, a plan runs eagerly on one
stream, so the two executions below take different launch paths over the same
arithmetic.
"""
import numpy as np
import pytest

import lattice_inputs as li
from tests import _cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1702_00339_gb300 import build, fock
    build.build()
    c = fock.Context(0)
    yield c
    c.close()


def _problems():
    ps = [_cases.box_chain_small(L=12, n0=5, pad=6, n_perp=20, R=16, k=6, seed=s) for s in (0, 1)]
    d = _cases.box_chain_small(L=14, n0=5, pad=6, n_perp=20, R=16, k=6, seed=2)
    d.defects = [li.Defect((5, 0, 0), 0, 2.0)]
    ps.append(d)
    ps.append(_cases.periodic_chain_small(L=6, seed=3))
    ps.append(_cases.periodic_3d_small(seed=4))
    for p in ps:
        if not p.is_box and not p.defects:
            p.k_eig = 0
    return ps


def test_graph_overlap_and_tuner_leave_results_bitwise_unchanged(ctx):
    ps = _problems()
    plan = ctx.plan(ps)
    try:
        plan.execute(maxit=400)
        a = plan.outputs()
        t = plan.tuning()
        assert t["fft_cc"] >= 1 and (t["fft_cc"] & (t["fft_cc"] - 1)) == 0
        assert t["graph_nodes"] > 0, "the block iteration was not captured"
        plan.execute(maxit=400)   # replay of the cached graph
        b = plan.outputs()
        ctx.profile(True)
        try:
            plan.execute(maxit=400)   # eager, one stream
            c = plan.outputs()
        finally:
            ctx.profile(False)
        for x, y, z in zip(a, b, c):
            assert x["status"] == 0
            assert np.array_equal(x["evals"], y["evals"]) and np.array_equal(x["evals"], z["evals"])
            assert x["iters"] == y["iters"] == z["iters"]
            if x["block_of"] is not None:
                assert np.array_equal(x["block_of"], z["block_of"])
    finally:
        plan.close()


def test_tuner_result_is_cached_per_context(ctx):
    ps = [li.config2(s) for s in range(4)]
    for p in ps:
        p.k_eig = 16
    p1 = ctx.plan(ps)
    p2 = ctx.plan(ps)
    try:
        p1.execute()
        p2.execute()
        assert p1.tuning()["fft_cc"] == p2.tuning()["fft_cc"] >= 1
        o1, o2 = p1.outputs(), p2.outputs()
        for x, y in zip(o1, o2):
            assert np.array_equal(x["evals"], y["evals"])
    finally:
        p1.close()
        p2.close()


def test_large_rayleigh_ritz_same_bits_on_a_cluster_and_on_one_cta(ctx):
    """A basis too large for one CTA's shared memory (k = 32 on a 64-cell
    chain: 3 x 36 columns) takes its Rayleigh-Ritz steps on a thread-block
    cluster in a batch without periodic problems and on one CTA beside a
    periodic problem.  Both give the same bits, and the oracle's eigenvalues."""
    from oracle import dense
    p = li.config2(5, L=64, n0=15, pad=32, n_perp=256, R=32)
    p.k_eig = 32
    per = li.config2(6, L=64, n0=15, pad=32, n_perp=256, R=32).as_periodic_chain()
    per.k_eig = 0
    alone = ctx.solve([p])[0]
    beside = ctx.solve([p, per])[0]
    assert alone["status"] == 0 and beside["status"] == 0
    assert np.array_equal(alone["evals"], beside["evals"]) and alone["iters"] == beside["iters"]
    q = _cases.with_table(p)
    q.k_eig = p.k_eig
    H, S = dense.build(q)
    ref = _cases.reference(q, H, S)
    _cases.report("box_k32_cluster", _cases.check(ref, alone["evals"]))


def test_block_route_count(ctx):
    """fock_plan_block_routes counts the Fourier blocks solved through the
    overlap's eigendecomposition: every block when a Gaussian is listed twice
    (each overlap block is then singular), conjugate pairs once."""
    import dataclasses
    p = _cases.periodic_chain_small(L=6, seed=3)
    p.k_eig = 0
    dup = dataclasses.replace(p, exps=np.concatenate([p.exps, p.exps[:1]]),
                              ang=np.concatenate([p.ang, p.ang[:1]]),
                              centre=np.concatenate([p.centre, p.centre[:1]]))
    dup.k_eig = 0
    plan = ctx.plan([dup])
    try:
        plan.execute()
        o = plan.outputs()[0]
        assert o["status"] == 0
        assert plan.block_routes(0) == 4          # j = 0, 3 and the pairs (1, 5), (2, 4)
        assert int(np.sum(~np.isfinite(o["evals"]))) == 6   # one direction removed per block
    finally:
        plan.close()
