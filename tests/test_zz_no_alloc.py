"""The no-allocation matvec entry point against the allocating one.

fock_toeplitz_matvec_noalloc serves callers that cannot allocate device
memory (real-time loops that forbid allocator calls once running, hosts
whose own allocator owns the device): its FFT work arrays live in a fixed
per-device array inside the library.  It must return the same product
as fock_toeplitz_matvec, call after call (the shared array keeps the
previous call's contents).  This file is collected last on purpose.
"""
import numpy as np
import pytest

from tests import _cases

pytestmark = pytest.mark.gpu


def test_noalloc_matvec_matches_allocating_entry_point():
    torch = pytest.importorskip("torch")
    from paper_1702_00339_gb300 import build, fock
    build.build()
    ctx = fock.Context(0)
    try:
        p = _cases.box_chain_small(L=12, n0=5, pad=6, n_perp=20, R=16, k=6)
        b = ctx.assemble(p)
        nvec = 7
        g = torch.Generator().manual_seed(11)
        # column-major N_b x nvec: a (nvec, N_b) row-major tensor
        x = torch.randn(nvec, b.Nb, dtype=torch.float64, generator=g).cuda()
        for which in (fock.FOCK_OP_H, fock.FOCK_OP_S):
            y_ref = torch.zeros_like(x)
            b.matvec_device(x.data_ptr(), y_ref.data_ptr(), nvec, which)
            scale = float(y_ref.abs().max())
            for _ in range(2):   # two calls in a row share the scratch array
                y = torch.full_like(x, float("nan"))
                b.matvec_noalloc(x.data_ptr(), y.data_ptr(), nvec, which)
                torch.cuda.synchronize()
                err = float((y - y_ref).abs().max())
                assert np.isfinite(err) and err <= 1e-12 * scale
        # sizes beyond the fixed scratch are rejected with FOCK_EINVAL
        big = (fock_scratch_bytes() // (2 * 16 * b.mcirc * p.m0)) + 1
        xb = torch.zeros(big, b.Nb, dtype=torch.float64, device="cuda")
        with pytest.raises(fock.FockError) as ei:
            b.matvec_noalloc(xb.data_ptr(), xb.data_ptr(), big, fock.FOCK_OP_H)
        assert ei.value.code == fock.FOCK_EINVAL
        # x and y may not overlap (y is written before the boundary blocks read x)
        with pytest.raises(fock.FockError) as ei:
            b.matvec_noalloc(x.data_ptr(), x.data_ptr(), nvec, fock.FOCK_OP_H)
        assert ei.value.code == fock.FOCK_EINVAL
        # the caller's current device is unchanged
        assert torch.cuda.current_device() == 0
        b.close()
    finally:
        ctx.close()


def fock_scratch_bytes():
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "include", "fock.h")).read()
    m = re.search(r"#define FOCK_NOALLOC_SCRATCH_BYTES \((\d+)u << (\d+)\)", hdr)
    return int(m.group(1)) << int(m.group(2))
