"""The tensor-core FP64 product (fock_split_dgemm: exact split products on
tcgen05, the mixed form's quadrature contraction) against the plain matrix
product in FP64 on the host, on shapes that span several tiles, ragged
edges, K chunks and both operand layouts, and on the quadrature contraction
of a real problem (potential table times folded pair products)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1702_00339_gb300 import build, fock
    build.build()
    c = fock.Context(0)
    yield c
    c.close()


def _run(ctx, A, B, a_kcontig, b_kcontig, alpha=1.0, beta=0.0, C0=None, ksplit=1, sym=False):
    torch = pytest.importorskip("torch")
    M, K = A.shape
    N = B.shape[1]
    # device layouts: A row-major (k contiguous) or column-major; B likewise
    tA = torch.tensor(A if a_kcontig else np.asfortranarray(A).T.copy(), dtype=torch.float64, device="cuda")
    tB = torch.tensor(B.T.copy() if b_kcontig else B, dtype=torch.float64, device="cuda")
    a_m, a_k = (K, 1) if a_kcontig else (1, M)
    b_k, b_n = (1, K) if b_kcontig else (N, 1)
    tC = torch.tensor(C0 if C0 is not None else np.zeros((M, N)), dtype=torch.float64, device="cuda")
    ctx.split_dgemm(M, N, K, tA.data_ptr(), a_m, a_k, tB.data_ptr(), b_k, b_n, tC.data_ptr(), N, 1,
                    alpha, beta, ksplit, sym)
    torch.cuda.synchronize()
    return tC.cpu().numpy()


def _bound(A, B):
    """Per-entry bar: 2^-44 |row max of A| |column max of B| K (the digits keep
    49 of 53 bits, levels above 8 are dropped; a factor 4 of headroom)."""
    K = A.shape[1]
    return 2.0 ** -44 * np.max(np.abs(A), axis=1)[:, None] * np.max(np.abs(B), axis=0)[None, :] * K


@pytest.mark.parametrize("M,N,K,ak,bk", [(128, 64, 64, True, True), (200, 150, 37, True, False),
                                         (80, 1024, 15, True, False), (33, 70, 300, False, True),
                                         (257, 65, 129, False, False), (1, 1, 1, True, True)])
def test_split_product_matches_fp64_matmul(ctx, M, N, K, ak, bk):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-20, 20, size=(M, 1)))
    B = rng.standard_normal((K, N)) * np.exp(rng.uniform(-20, 20, size=(1, N)))
    A[rng.random((M, K)) < 0.2] = 0.0            # exact zeros and mixed magnitudes
    C = _run(ctx, A, B, ak, bk)
    ref = A @ B
    assert np.all(np.abs(C - ref) <= _bound(A, B) + 1e-300)


def test_split_product_alpha_beta(ctx):
    rng = np.random.default_rng(3)
    A, B, C0 = rng.standard_normal((70, 40)), rng.standard_normal((40, 90)), rng.standard_normal((70, 90))
    C = _run(ctx, A, B, True, False, alpha=-0.5, beta=2.0, C0=C0)
    ref = -0.5 * A @ B + 2.0 * C0
    assert np.all(np.abs(C - ref) <= 0.5 * _bound(A, B) + 4 * 2.0 ** -53 * np.abs(ref))


def _mixed(p):
    import dataclasses
    q = dataclasses.replace(p, precision=1)
    q.k_eig = p.k_eig
    return q


@pytest.mark.parametrize("maker", ["box", "periodic_3d", "periodic_chain_defect"])
def test_mixed_assembly_entries_within_1e12(ctx, maker):
    """Mixed form: the quadrature contractions of the assembly on the tensor
    cores; the generator blocks (and boundary / defect blocks) against the
    oracle's dense matrices within 1e-12 of the largest entry."""
    from oracle import blocks, dense
    from tests import _cases
    from tests.test_gpu_defects import CASES as DEFECTS
    from tests.test_gpu_parity import _dense_from_blocks
    if maker == "box":
        p = _cases.box_chain_small(L=12, n0=5, pad=6, n_perp=20, R=16, k=6)
    elif maker == "periodic_3d":
        p = _cases.periodic_3d_small(L=(3, 2, 4), n0=5, R=12)
    else:
        p = DEFECTS["periodic_long_L30_subst"]()
    H, S = dense.build(p)
    b = ctx.assemble(_mixed(p))
    gh, gs, EH, ES, rc = b.generators()
    b.close()
    if blocks.structured(p):
        gotH, gotS = _dense_from_blocks(p, gh, EH, rc), _dense_from_blocks(p, gs, ES, rc)
        assert np.max(np.abs(gotH - H)) <= 1e-12 * np.max(np.abs(H))
        assert np.max(np.abs(gotS - S)) <= 1e-12 * np.max(np.abs(S))
    else:
        assert np.max(np.abs(gh - blocks.generators_from_dense(p, H))) <= 1e-12 * np.max(np.abs(H))
        assert np.max(np.abs(gs - blocks.generators_from_dense(p, S))) <= 1e-12 * np.max(np.abs(S))


def test_mixed_periodic_solve_matches_the_oracle(ctx):
    """A periodic lattice in the mixed form (tensor-core assembly, FP64 block
    eigensolves) against the oracle within the FP64 bar."""
    from oracle import dense
    from tests import _cases
    p = _cases.periodic_3d_small(L=(3, 2, 4), n0=5, R=12)
    H, S = dense.build(p)
    out = ctx.solve([_mixed(p)])[0]
    assert out["status"] == 0
    _cases.report("mixed_periodic_3d", _cases.check(_cases.reference(p, H, S), out["evals"], out["block_of"]))


@pytest.mark.parametrize("ksplit", [1, 3, 32])
def test_split_product_k_ranges_and_symmetric_gram(ctx, ksplit):
    """The Gram form of the block iteration: Y^T (H Y) over a long sum split
    into K ranges added in a fixed order, the upper triangle mirrored."""
    rng = np.random.default_rng(ksplit)
    n, nb = 5000, 150
    Y = rng.standard_normal((n, nb))
    HY = Y @ np.diag(rng.uniform(1, 3, nb)) + 1e-3 * rng.standard_normal((n, nb))
    G = _run(ctx, Y.T.copy(), HY, True, True, ksplit=ksplit, sym=True)
    ref = Y.T @ HY
    up = np.triu_indices(nb)
    assert np.all(np.abs(G[up] - ref[up]) <= _bound(Y.T, HY)[up])
    assert np.array_equal(G, G.T)
