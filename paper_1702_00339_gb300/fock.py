"""Python binding of libfock (argument marshalling only).

Every step of the method runs in the CUDA kernels behind the C ABI declared
in include/fock.h; this module converts lattice_inputs.Problem objects and
numpy / torch buffers to the ABI's plain structs and pointers.  It fails
loudly when the library is missing: there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import os
import struct

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_PKG, "libfock.so")

FOCK_OK, FOCK_EINVAL, FOCK_ENOMEM, FOCK_ENOCONV = 0, -1, -2, -3
FOCK_ETIMEOUT, FOCK_EAGAIN, FOCK_ECUDA = -4, -5, -6
FOCK_OP_H, FOCK_OP_S = 0, 1
FOCK_FP64, FOCK_MIXED, FOCK_MIXED_F32 = 0, 1, 2
FOCK_DEFAULT_MAXIT = 1000   # the block iteration's default cap (include/fock.h)
_NAMES = {0: "FOCK_OK", -1: "FOCK_EINVAL", -2: "FOCK_ENOMEM", -3: "FOCK_ENOCONV",
          -4: "FOCK_ETIMEOUT", -5: "FOCK_EAGAIN", -6: "FOCK_ECUDA"}


class FockError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class c_defect(C.Structure):
    _fields_ = [("cell", C.c_int * 3), ("nucleus", C.c_int), ("newZ", C.c_double)]


class c_problem(C.Structure):
    _fields_ = [("L", C.c_int * 3), ("periodic", C.c_int * 3), ("N", C.c_int * 3), ("n0", C.c_int),
                ("b0", C.c_double), ("M0", C.c_int), ("Z", C.c_void_p),          # const double*
                ("frac", C.c_void_p), ("m0", C.c_int), ("exps", C.c_void_p),        # const double*
                ("ang", C.c_void_p), ("centre", C.c_void_p), ("R", C.c_int),        # const int*
                ("sinc_t", C.c_void_p), ("sinc_c", C.c_void_p),                     # const double*
                ("eps_support", C.c_double), ("ndef", C.c_int),
                ("defects", C.c_void_p), ("k_eig", C.c_int), ("box_potential", C.c_int),
                ("precision", C.c_int)]   # defects: const fock_defect*


class c_serve_config(C.Structure):
    _fields_ = [("slots", C.c_int), ("max_batch", C.c_int), ("hbm_budget_bytes", C.c_size_t),
                ("tol", C.c_double), ("maxit", C.c_int)]


class c_result(C.Structure):
    _fields_ = [("evals", C.POINTER(C.c_double)), ("block_of", C.POINTER(C.c_int)),
                ("n_evals", C.c_int), ("status", C.c_int), ("iters", C.c_int), ("resid", C.c_double),
                ("t_submit_ns", C.c_int64), ("t_admit_ns", C.c_int64), ("t_done_ns", C.c_int64),
                ("batch_id", C.c_int), ("batch_size", C.c_int)]


class c_serve_stats(C.Structure):
    _fields_ = [("completed", C.c_uint64), ("pending", C.c_uint64), ("batches", C.c_uint64),
                ("inflight", C.c_int), ("max_inflight", C.c_int), ("reserved_bytes", C.c_size_t),
                ("peak_reserved_bytes", C.c_size_t), ("budget_bytes", C.c_size_t)]


class c_output(C.Structure):
    _fields_ = [("evals", C.c_void_p), ("block_of", C.c_void_p), ("n_evals", C.c_int),
                ("iters", C.c_int), ("resid", C.c_double), ("status", C.c_int)]


# numpy view of c_output (same offsets), for filling many entries at once
_OUT_DTYPE = np.dtype({"names": ["evals", "block_of"], "formats": [np.uint64, np.uint64],
                       "offsets": [c_output.evals.offset, c_output.block_of.offset],
                       "itemsize": C.sizeof(c_output)})


_lib = None


def lib():
    """Load libfock.so (built in-tree by paper_1702_00339_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIBPATH):
            raise ImportError(f"libfock.so not built at {_LIBPATH}; run paper_1702_00339_gb300.build.build()")
        L = C.CDLL(_LIBPATH)
        P = C.POINTER
        L.fock_create.argtypes = [P(C.c_void_p), C.c_int, C.c_size_t, C.c_void_p]
        L.fock_destroy.argtypes = [C.c_void_p]
        L.fock_destroy.restype = None
        L.fock_last_error.argtypes = [C.c_void_p]
        L.fock_last_error.restype = C.c_char_p
        L.fock_synchronize.argtypes = [C.c_void_p]
        L.fock_sinc_table.argtypes = [C.c_int, C.c_double, C.c_double, P(C.c_double), P(C.c_double),
                                      P(C.c_double)]
        L.fock_default_range.argtypes = [P(c_problem), P(C.c_double), P(C.c_double)]
        L.fock_problem_check.argtypes = [P(c_problem), P(C.c_int), P(C.c_int), C.c_char_p, C.c_int]
        L.fock_problem_layout.argtypes = [P(c_problem), P(C.c_int), P(C.c_int), P(C.c_int), P(C.c_int),
                                          P(C.c_int), P(C.c_int), P(C.c_int), C.c_int]
        L.fock_solve.argtypes = [C.c_void_p, C.c_int, P(c_problem), P(c_output), C.c_int]
        L.fock_assemble.argtypes = [C.c_void_p, P(c_problem), P(C.c_void_p)]
        L.fock_blocks_free.argtypes = [C.c_void_p]
        L.fock_blocks_free.restype = None
        L.fock_blocks_info.argtypes = [C.c_void_p, P(C.c_int), P(C.c_int), P(C.c_int), P(C.c_int)]
        L.fock_blocks_copy_generators.argtypes = [C.c_void_p, P(C.c_double), P(C.c_double),
                                                  P(C.c_double), P(C.c_double), P(C.c_int)]
        L.fock_circulant_eig.argtypes = [C.c_void_p, C.c_void_p, P(C.c_double), P(C.c_int), P(C.c_double)]
        L.fock_bloch_vectors.argtypes = [C.c_void_p, C.c_void_p, C.c_int, P(C.c_int), P(C.c_int), P(C.c_double)]
        L.fock_circulant_eig_range.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, P(C.c_double),
                                               P(C.c_int)]
        L.fock_toeplitz_matvec.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                           C.c_int, C.c_int]
        L.fock_toeplitz_matvec_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                                   C.c_void_p, C.c_int]
        L.fock_box_eig.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_int, P(C.c_double),
                                   P(C.c_double), P(C.c_int)]
        L.fock_plan_create.argtypes = [C.c_void_p, C.c_int, P(c_problem), P(C.c_void_p)]
        L.fock_plan_execute.argtypes = [C.c_void_p, C.c_double, C.c_int]
        L.fock_plan_outputs.argtypes = [C.c_void_p, P(c_output), C.c_int]
        L.fock_plan_info.argtypes = [C.c_void_p, P(C.c_size_t), P(C.c_size_t), P(C.c_size_t)]
        L.fock_plan_tuning.argtypes = [C.c_void_p, P(C.c_int), P(C.c_int)]
        L.fock_plan_block_routes.argtypes = [C.c_void_p, C.c_int, P(C.c_int)]
        L.fock_plan_problem_sizes.argtypes = [C.c_void_p, C.c_int, P(C.c_int), P(C.c_int), P(C.c_int),
                                              P(C.c_int)]
        L.fock_plan_free.argtypes = [C.c_void_p]
        L.fock_plan_free.restype = None
        L.fock_profile_enable.argtypes = [C.c_void_p, C.c_int]
        L.fock_profile_reset.argtypes = [C.c_void_p]
        L.fock_profile_read.argtypes = [C.c_void_p, C.c_int, C.c_char_p, P(C.c_int), P(C.c_double)]
        L.fock_serve_start.argtypes = [C.c_int, P(c_serve_config), P(C.c_void_p)]
        L.fock_serve_submit.argtypes = [C.c_void_p, P(c_problem), P(C.c_uint64)]
        L.fock_serve_poll.argtypes = [C.c_void_p, C.c_uint64, P(c_result), C.c_int]
        L.fock_result_release.argtypes = [C.c_void_p, C.c_uint64]
        L.fock_serve_stats.argtypes = [C.c_void_p, P(c_serve_stats)]
        L.fock_serve_last_error.argtypes = [C.c_void_p]
        L.fock_serve_last_error.restype = C.c_char_p
        L.fock_serve_stop.argtypes = [C.c_void_p]
        L.fock_measure_peaks.argtypes = [C.c_int, P(C.c_double), P(C.c_double)]
        L.fock_plan_history.argtypes = [C.c_void_p, C.c_int, P(C.c_double), C.c_int]
        L.fock_plan_split_work.argtypes = [C.c_void_p, P(C.c_double), P(C.c_double)]
        L.fock_split_dgemm.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int,
                                       C.c_void_p, C.c_longlong, C.c_longlong,
                                       C.c_void_p, C.c_longlong, C.c_longlong,
                                       C.c_void_p, C.c_longlong, C.c_longlong, C.c_double, C.c_double,
                                       C.c_int, C.c_int]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


# native layout of fock_problem (the same field order and alignment as c_problem)
_PROBLEM_FMT = "@3i3i3iidiPPiPPPiPPdiPiii"


class _Marshal:
    """Keeps the arrays behind one c_problem alive.  The double parameters
    (Z, frac, exps, sinc nodes and weights) share one contiguous array and the
    int ones (ang, centre) another; the struct, packed in one call, holds
    their addresses."""

    def __init__(self, p):
        table = p.sinc_t is not None
        parts = [np.asarray(p.Z, np.float64).ravel(), np.asarray(p.frac, np.float64).ravel(),
                 np.asarray(p.exps, np.float64).ravel()]
        if table:
            parts += [np.asarray(p.sinc_t, np.float64).ravel(), np.asarray(p.sinc_c, np.float64).ravel()]
        dv = np.concatenate(parts)
        ang = np.asarray(p.ang, np.int32).ravel()
        iv = np.concatenate([ang, np.asarray(p.centre, np.int32).ravel()])
        self.keep = [dv, iv]
        bd, bi = dv.ctypes.data, iv.ctypes.data
        off = [0]
        for a in parts:
            off.append(off[-1] + 8 * a.size)   # byte offsets of the parts in dv
        dptr = 0
        if p.defects:
            d = (c_defect * len(p.defects))()
            for i, x in enumerate(p.defects):
                d[i].cell[:] = [int(v) for v in x.cell]
                d[i].nucleus = int(x.nucleus)
                d[i].newZ = float(x.newZ)
            self.keep.append(d)
            dptr = C.addressof(d)
        L, per, N = p.L, p.periodic, p.N
        buf = struct.pack(
            _PROBLEM_FMT, int(L[0]), int(L[1]), int(L[2]), int(per[0]), int(per[1]), int(per[2]),
            int(N[0]), int(N[1]), int(N[2]), int(p.n0), float(p.b0), len(p.Z), bd + off[0], bd + off[1],
            len(p.exps), bd + off[2], bi, bi + 4 * ang.size, int(p.R),
            bd + off[3] if table else 0, bd + off[4] if table else 0, float(p.eps_support),
            len(p.defects), dptr, int(p.k_eig), int(getattr(p, "box_potential", 0)),
            int(getattr(p, "precision", 0)))
        buf += bytes(C.sizeof(c_problem) - len(buf))     # the struct's trailing padding
        self.s = c_problem.from_buffer_copy(buf)


def _host_outputs(problems):
    """c_output array for host results: every problem's eigenvalues (and block
    indices) are views into two batch-wide arrays (two allocations per call)."""
    n = len(problems)
    ne = [n_evals(p) for p in problems]
    st = [_structured(p) for p in problems]
    off = np.concatenate([[0], np.cumsum(ne, dtype=np.int64)]).astype(np.int64)
    ev_all = np.zeros(int(off[-1]))
    blk_all = np.zeros(int(off[-1]), np.int32)
    outs = (c_output * n)()
    be, bb = ev_all.ctypes.data, blk_all.ctypes.data
    # the two pointer fields of every entry at once, through a numpy view of the array
    rec = np.frombuffer(outs, dtype=_OUT_DTYPE, count=n) if n else None
    if n:
        rec["evals"] = be + 8 * off[:-1]
        rec["block_of"] = np.where(np.asarray(st, bool), 0, bb + 4 * off[:-1])
    views = [(ev_all[int(off[i]):int(off[i + 1])], None if st[i] else blk_all[int(off[i]):int(off[i + 1])])
             for i in range(n)]
    return outs, views


def _structured(p):
    """Box chains and problems with defects: lowest-k structured solve."""
    return bool(p.is_box or p.defects)


def n_evals(p):
    ncell = int(p.L[0]) * int(p.L[1]) * int(p.L[2])
    if _structured(p):
        return int(p.k_eig or 16)
    return ncell * len(p.exps)


def sinc_table(R, zmin, zmax):
    t = np.zeros(R)
    c = np.zeros(R)
    e = C.c_double()
    rc = lib().fock_sinc_table(int(R), float(zmin), float(zmax), _dp(t), _dp(c), C.byref(e))
    if rc:
        raise FockError(rc, "fock_sinc_table")
    return t, c, e.value


def default_range(p):
    m = _Marshal(p)
    a, b = C.c_double(), C.c_double()
    rc = lib().fock_default_range(C.byref(m.s), C.byref(a), C.byref(b))
    if rc:
        raise FockError(rc, "fock_default_range")
    return a.value, b.value


def check_problem(p):
    """The library's own host-side check of a problem (fock_problem_check):
    returns {"kind": 0 periodic | 1 structured, "n_evals": ...}; raises
    FockError(FOCK_EINVAL, reason) for a malformed problem."""
    m = _Marshal(p)
    kind, ne = C.c_int(-1), C.c_int(-1)
    why = C.create_string_buffer(256)
    rc = lib().fock_problem_check(C.byref(m.s), C.byref(kind), C.byref(ne), why, len(why))
    if rc:
        raise FockError(rc, why.value.decode())
    return {"kind": kind.value, "n_evals": ne.value}


def problem_layout(p):
    """The planner's block structure of one problem, host only
    (fock_problem_layout): {"Nb", "mcirc", "D", "E": int array (n, 3) of
    (row cell, column cell, kind)}."""
    m = _Marshal(p)
    nb, mc, d, ne = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    rc = lib().fock_problem_layout(C.byref(m.s), C.byref(nb), C.byref(mc), C.byref(d), C.byref(ne),
                                   None, None, None, 0)
    if rc:
        raise FockError(rc, "fock_problem_layout")
    n = ne.value
    ek, em, kd = (np.zeros(max(n, 1), np.int32) for _ in range(3))
    rc = lib().fock_problem_layout(C.byref(m.s), None, None, None, None, _ip(ek), _ip(em), _ip(kd), n)
    if rc:
        raise FockError(rc, "fock_problem_layout")
    return {"Nb": nb.value, "mcirc": mc.value, "D": d.value,
            "E": np.stack([ek[:n], em[:n], kd[:n]], axis=1)}


class Context:
    """A libfock context on one CUDA device (owns device memory and a stream)."""

    def __init__(self, device=0, budget_bytes=0, stream=None):
        import weakref
        self._children = weakref.WeakSet()   # handles freed before the context
        self.h = C.c_void_p()
        rc = lib().fock_create(C.byref(self.h), int(device), C.c_size_t(budget_bytes),
                               C.c_void_p(stream) if stream else None)
        if rc:
            raise FockError(rc, "fock_create")

    def close(self):
        if self.h:
            for c in list(self._children):
                c.close()
            lib().fock_destroy(self.h)
            self.h = C.c_void_p()

    __del__ = close

    def _check(self, rc, what):
        if rc:
            raise FockError(rc, f"{what}: {lib().fock_last_error(self.h).decode()}")

    def synchronize(self):
        self._check(lib().fock_synchronize(self.h), "fock_synchronize")

    def solve(self, problems, outputs=None, check=True):
        """Batched solve.  Host outputs (numpy) unless `outputs` gives, per
        problem, (evals_ptr, block_of_ptr_or_0) device pointers."""
        n = len(problems)
        ms = [_Marshal(p) for p in problems]
        arr = (c_problem * n)(*[m.s for m in ms])
        if outputs is None:
            outs, host = _host_outputs(problems)
        else:
            outs = (c_output * n)()
            for i in range(n):
                outs[i].evals, outs[i].block_of = outputs[i]
        rc = lib().fock_solve(self.h, n, arr, outs, 0 if outputs is None else 1)
        if rc and check:
            self._check(rc, "fock_solve")
        res = []
        for i, p in enumerate(problems):
            r = {"n_evals": outs[i].n_evals, "iters": outs[i].iters, "resid": outs[i].resid,
                 "status": outs[i].status}
            if outputs is None:
                r["evals"], r["block_of"] = host[i]
            res.append(r)
        return res

    def assemble(self, p):
        return Blocks(self, p)

    def plan(self, problems):
        return Plan(self, problems)

    # ---- kernel timers ----
    def profile(self, on=True):
        self._check(lib().fock_profile_enable(self.h, 1 if on else 0), "fock_profile_enable")

    def profile_reset(self):
        self._check(lib().fock_profile_reset(self.h), "fock_profile_reset")

    def split_dgemm(self, M, N, K, A, a_m, a_k, B, b_k, b_n, Cp, c_m, c_n, alpha=1.0, beta=0.0,
                    ksplit=1, sym=False):
        """C = alpha A B + beta C on the tensor cores (fock_split_dgemm);
        A, B, Cp are device pointers (ints), strides in elements."""
        self._check(lib().fock_split_dgemm(self.h, int(M), int(N), int(K), A, a_m, a_k, B, b_k, b_n,
                                           Cp, c_m, c_n, float(alpha), float(beta), int(ksplit),
                                           1 if sym else 0), "fock_split_dgemm")

    def profile_read(self, cap=64):
        names = C.create_string_buffer(32 * cap)
        nl = (C.c_int * cap)()
        ms = (C.c_double * cap)()
        n = lib().fock_profile_read(self.h, cap, names, nl, ms)
        if n < 0:
            self._check(n, "fock_profile_read")
        out = {}
        for i in range(n):
            nm = names.raw[32 * i:32 * (i + 1)].split(b"\0", 1)[0].decode()
            out[nm] = (int(nl[i]), float(ms[i]))
        return out


class Blocks:
    """Device-resident assembled operator of one problem (fock_assemble)."""

    def __init__(self, ctx, p):
        self.ctx = ctx
        self.p = p
        self.h = C.c_void_p()
        m = _Marshal(p)
        ctx._check(lib().fock_assemble(ctx.h, C.byref(m.s), C.byref(self.h)), "fock_assemble")
        ctx._children.add(self)
        a, b, c, d = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        lib().fock_blocks_info(self.h, C.byref(a), C.byref(b), C.byref(c), C.byref(d))
        self.Nb, self.ngen, self.nbound, self.mcirc = a.value, b.value, c.value, d.value

    def close(self):
        if self.h and self.ctx.h:
            lib().fock_blocks_free(self.h)
        self.h = C.c_void_p()

    __del__ = close

    def generators(self):
        m0 = len(self.p.exps)
        H = np.zeros((self.ngen, m0, m0))
        S = np.zeros((self.ngen, m0, m0))
        nb = max(self.nbound, 1)
        EH = np.zeros((nb, m0, m0))
        ES = np.zeros((nb, m0, m0))
        rc_ = np.zeros((nb, 2), np.int32)
        self.ctx._check(lib().fock_blocks_copy_generators(self.h, _dp(H), _dp(S), _dp(EH), _dp(ES),
                                                          _ip(rc_)), "fock_blocks_copy_generators")
        return H, S, EH[:self.nbound], ES[:self.nbound], rc_[:self.nbound]

    def circulant_eig(self, vectors=False):
        """(eigenvalues ascending, Fourier index of each) and, with vectors,
        the block eigenvectors as a complex array [block][i][mu]."""
        n = self.Nb
        ev = np.zeros(n)
        blk = np.zeros(n, np.int32)
        m0 = len(self.p.exps)
        vec = np.zeros((n // m0, m0, m0), complex) if vectors else None
        self.ctx._check(lib().fock_circulant_eig(self.ctx.h, self.h, _dp(ev), _ip(blk),
                                                 vec.ctypes.data_as(C.POINTER(C.c_double)) if vectors else None),
                        "fock_circulant_eig")
        return (ev, blk, vec) if vectors else (ev, blk)

    def bloch_vectors(self, jbar, rank):
        """Lattice eigenvectors (N_b x nsel complex) of the eigenpairs given by
        Fourier index and rank within the block (fock_bloch_vectors)."""
        jb = np.ascontiguousarray(jbar, np.int32)
        rk = np.ascontiguousarray(rank, np.int32)
        U = np.zeros((len(jb), self.Nb), complex)
        self.ctx._check(lib().fock_bloch_vectors(self.ctx.h, self.h, len(jb), _ip(jb), _ip(rk),
                                                 U.ctypes.data_as(C.POINTER(C.c_double))),
                        "fock_bloch_vectors")
        return U.T

    def circulant_eig_range(self, j0, j1):
        """Eigenvalues of the Fourier blocks j0 <= jbar < j1 only, ascending."""
        n = (int(j1) - int(j0)) * len(self.p.exps)
        ev = np.zeros(max(n, 0))
        blk = np.zeros(max(n, 0), np.int32)
        self.ctx._check(lib().fock_circulant_eig_range(self.ctx.h, self.h, int(j0), int(j1), _dp(ev), _ip(blk)),
                        "fock_circulant_eig_range")
        return ev, blk

    def matvec(self, x, which=FOCK_OP_H):
        x = np.asfortranarray(np.asarray(x, dtype=np.float64).reshape(self.Nb, -1))
        y = np.zeros_like(x, order="F")
        self.ctx._check(lib().fock_toeplitz_matvec(self.ctx.h, self.h, int(which), x.ctypes.data,
                                                   y.ctypes.data, x.shape[1], 0),
                        "fock_toeplitz_matvec")
        return y

    def matvec_device(self, x_ptr, y_ptr, nvec, which=FOCK_OP_H):
        self.ctx._check(lib().fock_toeplitz_matvec(self.ctx.h, self.h, int(which), x_ptr, y_ptr,
                                                   int(nvec), 1), "fock_toeplitz_matvec")

    def matvec_noalloc(self, x_ptr, y_ptr, nvec, which=FOCK_OP_H):
        """Device x, y; no device allocation (fixed per-device scratch)."""
        self.ctx._check(lib().fock_toeplitz_matvec_noalloc(self.ctx.h, self.h, int(which), x_ptr,
                                                           y_ptr, int(nvec)),
                        "fock_toeplitz_matvec_noalloc")

    def box_eig(self, k, tol=1e-10, maxit=FOCK_DEFAULT_MAXIT, vectors=False):
        ev = np.zeros(k)
        V = np.zeros((self.Nb, k), order="F") if vectors else None
        it = C.c_int()
        rc = lib().fock_box_eig(self.ctx.h, self.h, int(k), float(tol), int(maxit), _dp(ev),
                                _dp(V) if vectors else None, C.byref(it))
        if rc and rc != FOCK_ENOCONV:
            self.ctx._check(rc, "fock_box_eig")
        return ev, V, it.value, rc


class Plan:
    """Device-resident batch (fock_plan_*): inputs uploaded once, executed
    any number of times; results copied out on request."""

    def __init__(self, ctx, problems):
        self.ctx = ctx
        self.problems = list(problems)
        self.h = C.c_void_p()
        ms = [_Marshal(p) for p in self.problems]
        arr = (c_problem * len(ms))(*[m.s for m in ms])
        ctx._check(lib().fock_plan_create(ctx.h, len(ms), arr, C.byref(self.h)), "fock_plan_create")
        ctx._children.add(self)
        a, b, c = C.c_size_t(), C.c_size_t(), C.c_size_t()
        lib().fock_plan_info(self.h, C.byref(a), C.byref(b), C.byref(c))
        self.upload_bytes, self.device_bytes, self.n_evals = a.value, b.value, c.value

    def tuning(self):
        """{"fft_cc": FFT columns per CTA chosen by the tuner (0 before the
        first execution), "graph_nodes": kernels of the block iteration's
        body replayed as one CUDA graph (0 when not captured)}."""
        a, b = C.c_int(), C.c_int()
        self.ctx._check(lib().fock_plan_tuning(self.h, C.byref(a), C.byref(b)), "fock_plan_tuning")
        return {"fft_cc": a.value, "graph_nodes": b.value}

    def block_routes(self, i):
        """Fourier blocks of periodic problem i (conjugate pairs once) solved
        through the overlap's eigendecomposition at the last execution."""
        a = C.c_int()
        self.ctx._check(lib().fock_plan_block_routes(self.h, int(i), C.byref(a)), "fock_plan_block_routes")
        return a.value

    def sizes(self, i):
        """(N_b, circulant size M, generator reach D, boundary blocks) of problem i."""
        a, b, c, d = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        self.ctx._check(lib().fock_plan_problem_sizes(self.h, int(i), C.byref(a), C.byref(b), C.byref(c),
                                                      C.byref(d)), "fock_plan_problem_sizes")
        return a.value, b.value, c.value, d.value

    def execute(self, tol=1e-10, maxit=FOCK_DEFAULT_MAXIT):
        rc = lib().fock_plan_execute(self.h, float(tol), int(maxit))
        if rc:
            self.ctx._check(rc, "fock_plan_execute")

    def outputs(self, device_ptrs=None, check=True):
        """Host copies (list of dicts) or, with device_ptrs = [(evals_ptr,
        block_of_ptr_or_0), ...], device-to-device copies."""
        n = len(self.problems)
        if device_ptrs is None:
            outs, host = _host_outputs(self.problems)
        else:
            outs = (c_output * n)()
            for i in range(n):
                outs[i].evals, outs[i].block_of = device_ptrs[i]
        rc = lib().fock_plan_outputs(self.h, outs, 0 if device_ptrs is None else 1)
        if rc and check:
            self.ctx._check(rc, "fock_plan_outputs")
        res = []
        for i, p in enumerate(self.problems):
            r = {"n_evals": outs[i].n_evals, "iters": outs[i].iters, "resid": outs[i].resid,
                 "status": outs[i].status}
            if device_ptrs is None:
                r["evals"], r["block_of"] = host[i]
            res.append(r)
        return res

    def split_work(self):
        """{"tensor_flops", "fp64_flops"} of one execution's tensor-core assembly."""
        a, b = C.c_double(), C.c_double()
        self.ctx._check(lib().fock_plan_split_work(self.h, C.byref(a), C.byref(b)), "fock_plan_split_work")
        return {"tensor_flops": a.value, "fp64_flops": b.value}

    def history(self, i, cap=4096):
        """Largest wanted-pair relative residual at each iteration of problem
        i's block iteration in the last execution (empty for periodic)."""
        buf = (C.c_double * cap)()
        n = lib().fock_plan_history(self.h, int(i), buf, cap)
        if n < 0:
            self.ctx._check(n, "fock_plan_history")
        return [float(buf[t]) for t in range(min(n, cap))]

    def close(self):
        if self.h and self.ctx.h:
            lib().fock_plan_free(self.h)
        self.h = C.c_void_p()

    __del__ = close


class Server:
    """Continuous-batching server (fock_serve_*): submit problems from any
    thread, poll tickets for results."""

    def __init__(self, device=0, slots=2, max_batch=256, budget_bytes=0, tol=1e-10, maxit=FOCK_DEFAULT_MAXIT):
        cfg = c_serve_config(int(slots), int(max_batch), C.c_size_t(budget_bytes), float(tol), int(maxit))
        self.h = C.c_void_p()
        rc = lib().fock_serve_start(int(device), C.byref(cfg), C.byref(self.h))
        if rc:
            raise FockError(rc, "fock_serve_start")

    def _err(self):
        return lib().fock_serve_last_error(self.h).decode()

    def submit(self, p):
        m = _Marshal(p)
        t = C.c_uint64()
        rc = lib().fock_serve_submit(self.h, C.byref(m.s), C.byref(t))
        if rc:
            raise FockError(rc, f"fock_serve_submit: {self._err()}")
        return t.value

    def poll(self, ticket, timeout_ms=-1, release=True):
        """The ticket's result as a dict, or None if not finished within
        timeout_ms.  Copies the eigenvalues out and (by default) releases the
        library's buffers.  A structured request (box chain, defects) is ready
        as soon as it leaves the block iteration, while its batch may still
        run; a periodic one when its batch ends."""
        r = c_result()
        rc = lib().fock_serve_poll(self.h, C.c_uint64(ticket), C.byref(r), int(timeout_ms))
        if rc == FOCK_EAGAIN:
            return None
        if rc:
            raise FockError(rc, f"fock_serve_poll: {self._err()}")
        n = r.n_evals
        out = {"evals": np.ctypeslib.as_array(r.evals, (n,)).copy() if n else np.zeros(0),
               "block_of": (np.ctypeslib.as_array(r.block_of, (n,)).copy() if r.block_of else None),
               "status": r.status, "iters": r.iters, "resid": r.resid,
               "t_submit_ns": r.t_submit_ns, "t_admit_ns": r.t_admit_ns, "t_done_ns": r.t_done_ns,
               "batch_id": r.batch_id, "batch_size": r.batch_size}
        if release:
            lib().fock_result_release(self.h, C.c_uint64(ticket))
        return out

    def stats(self):
        s = c_serve_stats()
        rc = lib().fock_serve_stats(self.h, C.byref(s))
        if rc:
            raise FockError(rc, "fock_serve_stats")
        return {f: getattr(s, f) for f, _ in c_serve_stats._fields_}

    def stop(self):
        if self.h:
            rc = lib().fock_serve_stop(self.h)
            self.h = C.c_void_p()
            if rc:
                raise FockError(rc, "fock_serve_stop")

    close = stop

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


def measure_peaks(device=0):
    """Measured FP64 and FP32 FMA throughput of a device (TFLOP/s), through
    fock_measure_peaks."""
    f64, f32 = C.c_double(), C.c_double()
    rc = lib().fock_measure_peaks(device, C.byref(f64), C.byref(f32))
    if rc != 0:
        raise FockError(rc, "fock_measure_peaks failed")
    return float(f64.value), float(f32.value)
