"""ctypes binding of libace_gb300.so (include/ace.h), same entry-point names, marshalling only.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays; the library decides from the pointer
whether memory is on the device or the host.  There is no CPU implementation here: if the shared
library is missing, loading fails with an error that says how to build it.
"""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libace_gb300.so")

ACE_OK = 0
ACE_ERR_ARG = 1
ACE_ERR_CUDA = 2
ACE_ERR_OOM = 3
ACE_ERR_NOT_POSDEF = 4
ACE_ERR_NONFINITE = 5
ACE_ERR_UNSUPPORTED_GRID = 6
ACE_ERR_TIMEOUT = 7
STATUS_NAMES = {
    0: "ACE_OK", 1: "ACE_ERR_ARG", 2: "ACE_ERR_CUDA", 3: "ACE_ERR_OOM", 4: "ACE_ERR_NOT_POSDEF",
    5: "ACE_ERR_NONFINITE", 6: "ACE_ERR_UNSUPPORTED_GRID", 7: "ACE_ERR_TIMEOUT",
}

ACE_FP64 = 0
ACE_MIXED = 1
ACE_F32 = 0
ACE_F64 = 1
ACE_COULOMB_PERIODIC = 0
ACE_COULOMB_TRUNCATED = 1

ACE_GET_XI = 0
ACE_GET_W = 1
ACE_GET_M = 2
ACE_GET_M_RAW = 3
ACE_GET_L = 4
ACE_GET_PAIRS = 5
ACE_GET_OVERLAP = 6

EXPORTED = [
    "ace_build", "ace_build_batched", "ace_apply", "exchange_energy", "ace_get", "ace_pair_count",
    "ace_get_size", "ace_stage_times", "ace_kernel_launches", "ace_grid_supported", "ace_destroy",
    "ace_last_error", "ace_exchange_w_noalloc", "ace_autotune", "ace_build_pairs", "ace_scdm",
    "ace_exchange_w", "ace_m_partial", "ace_build_from_m", "ace_apply_coeffs", "ace_apply_finish",
    "ace_graph_create", "ace_graph_launch", "ace_graph_sync", "ace_graph_size", "ace_graph_op",
    "ace_graph_destroy",
]


class AceError(RuntimeError):
    def __init__(self, status: int, message: str, op=None):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.op = op


class AceDesc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3),
        ("lattice", (ctypes.c_double * 3) * 3),
        ("norb", ctypes.c_int),
        ("rho_cut", ctypes.c_double),
        ("spin_factor", ctypes.c_double),
        ("prec", ctypes.c_int),
        ("coulomb", ctypes.c_int),
        ("r_cut", ctypes.c_double),
    ]


def make_desc(grid, lattice, norb, rho_cut=0.0, spin_factor=2.0, prec=ACE_MIXED, coulomb=0, r_cut=0.0) -> AceDesc:
    """Descriptor of one build; coulomb = ACE_COULOMB_PERIODIC (4 pi/|G|^2) or ACE_COULOMB_TRUNCATED
    (isolated cell, 1/r cut off at r_cut; r_cut <= 0 selects the inscribed-sphere radius)."""
    d = AceDesc()
    for k in range(3):
        d.n[k] = int(grid[k])
    lat = np.asarray(lattice, dtype=np.float64).reshape(3, 3)
    for i in range(3):
        for j in range(3):
            d.lattice[i][j] = float(lat[i, j])
    d.norb = int(norb)
    d.rho_cut = float(rho_cut)
    d.spin_factor = float(spin_factor)
    d.prec = int(prec)
    d.coulomb = int(coulomb)
    d.r_cut = float(r_cut)
    return d


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library; raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(
                f"{path} is missing: build it with `python -m paper_2101_03155_gb300.build` "
                "(nvcc, sm_103a); there is no CPU implementation"
            )
        lib = ctypes.CDLL(path)
        vp, c_int, c_long, c_size = ctypes.c_void_p, ctypes.c_int, ctypes.c_long, ctypes.c_size_t
        lib.ace_build.argtypes = [ctypes.POINTER(AceDesc), vp, c_int, vp, ctypes.POINTER(vp)]
        lib.ace_build_pairs.argtypes = [ctypes.POINTER(AceDesc), vp, c_int, vp, ctypes.c_long, vp, ctypes.POINTER(vp)]
        lib.ace_build_batched.argtypes = [c_int, ctypes.POINTER(AceDesc), ctypes.POINTER(vp), c_int, vp,
                                          ctypes.POINTER(vp)]
        lib.ace_apply.argtypes = [vp, vp, c_int, c_int, vp, vp]
        lib.exchange_energy.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        lib.ace_get.argtypes = [vp, c_int, vp, c_size, vp]
        lib.ace_get_size.argtypes = [vp, c_int, ctypes.POINTER(c_size)]
        lib.ace_pair_count.argtypes = [vp, ctypes.POINTER(c_long)]
        lib.ace_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
        lib.ace_kernel_launches.argtypes = [vp, ctypes.POINTER(c_long)]
        lib.ace_autotune.argtypes = [ctypes.POINTER(AceDesc), vp, c_int, vp, ctypes.POINTER(c_int)]
        lib.ace_exchange_w_noalloc.argtypes = [ctypes.POINTER(AceDesc), vp, c_int, ctypes.POINTER(c_int), c_long,
                                               vp, vp]
        lib.ace_scdm.argtypes = [c_int, ctypes.c_longlong, c_int, vp, c_int, vp, ctypes.POINTER(c_int),
                                 ctypes.POINTER(ctypes.c_double), vp, ctypes.POINTER(c_long)]
        lib.ace_exchange_w.argtypes = [ctypes.POINTER(AceDesc), vp, c_int, vp, c_long, vp, vp]
        lib.ace_m_partial.argtypes = [ctypes.POINTER(AceDesc), vp, vp, c_int, ctypes.c_longlong, vp, vp]
        lib.ace_build_from_m.argtypes = [ctypes.POINTER(AceDesc), vp, vp, c_int, ctypes.c_longlong, vp,
                                         ctypes.POINTER(vp)]
        lib.ace_apply_coeffs.argtypes = [vp, vp, c_int, c_int, vp, vp]
        lib.ace_apply_finish.argtypes = [vp, vp, c_int, c_int, vp, vp]
        lib.ace_graph_create.argtypes = [c_int, ctypes.POINTER(AceDesc), ctypes.POINTER(vp), c_int,
                                         ctypes.POINTER(vp), ctypes.POINTER(c_long), vp, ctypes.POINTER(vp)]
        lib.ace_graph_launch.argtypes = [vp, vp]
        lib.ace_graph_sync.argtypes = [vp]
        lib.ace_graph_size.argtypes = [vp]
        lib.ace_graph_size.restype = c_int
        lib.ace_graph_op.argtypes = [vp, c_int, ctypes.POINTER(vp)]
        lib.ace_graph_destroy.argtypes = [vp]
        lib.ace_graph_destroy.restype = None
        lib.ace_grid_supported.argtypes = [c_int, c_int]
        lib.ace_grid_supported.restype = c_int
        lib.ace_destroy.argtypes = [vp]
        lib.ace_destroy.restype = None
        lib.ace_last_error.restype = ctypes.c_char_p
        for name in ("ace_build", "ace_build_batched", "ace_apply", "exchange_energy", "ace_get", "ace_get_size",
                     "ace_pair_count", "ace_stage_times", "ace_kernel_launches", "ace_exchange_w_noalloc",
                     "ace_autotune", "ace_build_pairs", "ace_scdm", "ace_exchange_w", "ace_m_partial",
                     "ace_build_from_m", "ace_apply_coeffs", "ace_apply_finish", "ace_graph_create",
                     "ace_graph_launch", "ace_graph_sync", "ace_graph_op"):
            getattr(lib, name).restype = c_int
        _lib = lib
        return lib


def ace_last_error() -> str:
    return load().ace_last_error().decode()


def _check(status: int, op=None):
    if status != ACE_OK:
        raise AceError(status, ace_last_error(), op)


def _array_info(a):
    """(pointer, dtype code, number of elements) of a contiguous torch tensor or numpy array."""
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        code = {np.dtype(np.float32): ACE_F32, np.dtype(np.float64): ACE_F64}.get(a.dtype)
        if code is None:
            raise TypeError(f"unsupported dtype {a.dtype}")
        return a.ctypes.data, code, a.size
    import torch

    if not isinstance(a, torch.Tensor):
        raise TypeError("expected a torch tensor or numpy array")
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    code = {torch.float32: ACE_F32, torch.float64: ACE_F64}.get(a.dtype)
    if code is None:
        raise TypeError(f"unsupported dtype {a.dtype}")
    return a.data_ptr(), code, a.numel()


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None  # torch.cuda.Stream


class AceOp:
    """Owner of an ace_op handle; ace_destroy runs on close() or garbage collection.  A borrowed
    handle (one build of an AceGraph) is released by its graph, never here."""

    def __init__(self, handle: int, desc: AceDesc, owned: bool = True):
        self.handle = handle
        self.desc = desc
        self.owned = owned

    @property
    def grid(self):
        return tuple(self.desc.n)

    @property
    def norb(self):
        return self.desc.norb

    def close(self):
        if self.handle and self.owned:
            load().ace_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def ace_build(desc: AceDesc, phi, stream=None, check: bool = True) -> AceOp:
    """ace_build: phi [norb][N1][N2][N3] (torch CUDA/CPU tensor or numpy array)."""
    ptr, code, numel = _array_info(phi)
    expect = desc.norb * desc.n[0] * desc.n[1] * desc.n[2]
    if numel != expect:
        raise ValueError(f"phi has {numel} elements, descriptor needs {expect}")
    h = ctypes.c_void_p()
    st = load().ace_build(ctypes.byref(desc), ptr, code, _stream_handle(stream), ctypes.byref(h))
    op = AceOp(h.value, desc) if h.value else None
    if check:
        _check(st, op)
    return op if check else (st, op)


def ace_build_pairs(desc: AceDesc, phi, pairs, stream=None, check: bool = True) -> AceOp:
    """ace_build_pairs: the build on a given pair list (int [npairs][2]) instead of the screen."""
    ptr, code, numel = _array_info(phi)
    if numel != desc.norb * desc.n[0] * desc.n[1] * desc.n[2]:
        raise ValueError("phi does not match the descriptor")
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    h = ctypes.c_void_p()
    st = load().ace_build_pairs(ctypes.byref(desc), ptr, code, pr.ctypes.data if len(pr) else None, len(pr),
                                _stream_handle(stream), ctypes.byref(h))
    op = AceOp(h.value, desc) if h.value else None
    if check:
        _check(st, op)
    return op if check else (st, op)


def ace_build_batched(descs, phis, stream=None):
    k = len(descs)
    arr = (AceDesc * k)(*descs)
    ptrs = []
    code = None
    for d, p in zip(descs, phis):
        ptr, c, numel = _array_info(p)
        if code is not None and c != code:
            raise TypeError("all inputs of a batch must have one dtype")
        code = c
        if numel != d.norb * d.n[0] * d.n[1] * d.n[2]:
            raise ValueError("input size does not match its descriptor")
        ptrs.append(ptr)
    pa = (ctypes.c_void_p * k)(*ptrs)
    outs = (ctypes.c_void_p * k)()
    _check(load().ace_build_batched(k, arr, pa, code if code is not None else ACE_F32, _stream_handle(stream), outs))
    return [AceOp(outs[i], descs[i]) for i in range(k)]


class AceGraph:
    """k builds on given pair lists recorded as one CUDA graph (ace_graph_create).  Holds the input
    tensors so that they outlive the graph; overwrite their contents, then launch() again."""

    def __init__(self, handle: int, descs, phis):
        self.handle = handle
        self.descs = list(descs)
        self._phis = list(phis)
        lib = load()
        self.ops = []
        for i in range(lib.ace_graph_size(handle)):
            h = ctypes.c_void_p()
            _check(lib.ace_graph_op(handle, i, ctypes.byref(h)))
            self.ops.append(AceOp(h.value, self.descs[i], owned=False))

    def launch(self, stream=None):
        _check(load().ace_graph_launch(self.handle, _stream_handle(stream)))

    def sync(self):
        _check(load().ace_graph_sync(self.handle))

    def close(self):
        if self.handle:
            for op in self.ops:
                op.handle = None
            load().ace_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def ace_graph_create(descs, phis, pairs=None, stream=None) -> AceGraph:
    """ace_graph_create: phis are device tensors of the working dtype; pairs is one int [npairs][2]
    list per build, or None for builds that screen on the device at every launch."""
    k = len(descs)
    if len(phis) != k or (pairs is not None and len(pairs) != k):
        raise ValueError("descs, phis and pairs must have one entry per build")
    arr = (AceDesc * k)(*descs)
    ptrs, lists = [], []
    code = None
    for d, p in zip(descs, phis):
        ptr, c, numel = _array_info(p)
        if code is not None and c != code:
            raise TypeError("all inputs of a graph must have one dtype")
        code = c
        if numel != d.norb * d.n[0] * d.n[1] * d.n[2]:
            raise ValueError("input size does not match its descriptor")
        ptrs.append(ptr)
    for pr in pairs or []:
        lists.append(np.ascontiguousarray(np.asarray(pr, dtype=np.int32).reshape(-1, 2)))
    pa = (ctypes.c_void_p * k)(*ptrs)
    la = (ctypes.c_void_p * k)(*[x.ctypes.data if len(x) else None for x in lists]) if pairs is not None else None
    na = (ctypes.c_long * k)(*[len(x) for x in lists]) if pairs is not None else None
    h = ctypes.c_void_p()
    _check(load().ace_graph_create(k, arr, pa, code if code is not None else ACE_F32, la, na,
                                   _stream_handle(stream), ctypes.byref(h)))
    return AceGraph(h.value, descs, phis)


def ace_graph_launch(graph: AceGraph, stream=None) -> None:
    graph.launch(stream)


def ace_graph_sync(graph: AceGraph) -> None:
    graph.sync()


def ace_graph_size(graph: AceGraph) -> int:
    return load().ace_graph_size(graph.handle)


def ace_graph_op(graph: AceGraph, i: int) -> AceOp:
    return graph.ops[i]


def ace_graph_destroy(graph: AceGraph) -> None:
    graph.close()


def ace_apply(op: AceOp, psi, out, stream=None):
    """ace_apply: out = V_X^ACE psi; psi and out [m][N] of one dtype, both on the host or both on the device."""
    p_ptr, p_code, p_numel = _array_info(psi)
    o_ptr, o_code, o_numel = _array_info(out)
    N = op.desc.n[0] * op.desc.n[1] * op.desc.n[2]
    if p_code != o_code or p_numel != o_numel or p_numel % N:
        raise ValueError("psi and out must have the same dtype and [m][N] shape")
    _check(load().ace_apply(op.handle, p_ptr, p_code, p_numel // N, o_ptr, _stream_handle(stream)))
    return out


def ace_scdm(psi, phi, prec: int = ACE_MIXED, stream=None, check: bool = True):
    """ace_scdm: SCDM-localised orbitals of psi [norb][...] written into phi (same shape and dtype,
    same side).  Returns (status, pivots int32 [norb], U float64 [norb][norb], kernel launches)."""
    p_ptr, p_code, p_numel = _array_info(psi)
    o_ptr, o_code, o_numel = _array_info(phi)
    n = int(psi.shape[0])
    if p_code != o_code or p_numel != o_numel or p_numel % n:
        raise ValueError("psi and phi must have the same dtype and shape")
    piv = np.zeros(n, dtype=np.int32)
    U = np.zeros((n, n), dtype=np.float64)
    nl = ctypes.c_long()
    st = load().ace_scdm(n, p_numel // n, prec, p_ptr, o_code, o_ptr, piv.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                         U.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream_handle(stream), ctypes.byref(nl))
    if check:
        _check(st)
    return st, piv, U, nl.value


def exchange_energy(op: AceOp) -> float:
    e = ctypes.c_double()
    _check(load().exchange_energy(op.handle, ctypes.byref(e)))
    return e.value


def ace_get_size(op: AceOp, what: int) -> int:
    b = ctypes.c_size_t()
    _check(load().ace_get_size(op.handle, what, ctypes.byref(b)))
    return b.value


def ace_get(op: AceOp, what: int, dst, stream=None):
    """Copy an internal array into dst (torch tensor or numpy array of exactly the item's size)."""
    if isinstance(dst, np.ndarray):
        ptr, nbytes = dst.ctypes.data, dst.nbytes
    else:
        ptr, nbytes = dst.data_ptr(), dst.numel() * dst.element_size()
    _check(load().ace_get(op.handle, what, ptr, nbytes, _stream_handle(stream)))
    return dst


def ace_pair_count(op: AceOp) -> int:
    n = ctypes.c_long()
    _check(load().ace_pair_count(op.handle, ctypes.byref(n)))
    return n.value


def ace_stage_times(op: AceOp):
    ms = (ctypes.c_float * 6)()
    _check(load().ace_stage_times(op.handle, ms))
    return {k: float(v) for k, v in zip(("screen", "pair_chain", "M", "cholesky", "xi", "total"), ms)}


def ace_autotune(desc: AceDesc, phi, stream=None) -> dict:
    """ace_autotune: pick the pair-chain batch / stream / L2 / pack-order / pencil-tile settings for this
    grid and precision."""
    ptr, code, numel = _array_info(phi)
    if numel != desc.norb * desc.n[0] * desc.n[1] * desc.n[2]:
        raise ValueError("phi does not match the descriptor")
    out = (ctypes.c_int * 7)()
    _check(load().ace_autotune(ctypes.byref(desc), ptr, code, _stream_handle(stream), out))
    return {"group": out[0], "batch": out[1], "streams": out[2], "l2_mb": out[3], "row_block": out[4],
            "persistent_lag": out[5], "pencil_tile": out[6]}


def ace_kernel_launches(op: AceOp) -> int:
    n = ctypes.c_long()
    _check(load().ace_kernel_launches(op.handle, ctypes.byref(n)))
    return n.value


def ace_grid_supported(n_axis: int, prec: int = ACE_MIXED) -> bool:
    return bool(load().ace_grid_supported(int(n_axis), int(prec)))


def ace_destroy(op: AceOp) -> None:
    op.close()


def ace_exchange_w_noalloc(desc: AceDesc, phi, pairs, W, stream=None):
    """W for an explicit pair list without any device allocation (fixed in-library workspace).

    phi and W: device tensors [norb][N] of the precision's working dtype; pairs: host int32 [npairs][2].
    """
    p_ptr, p_code, p_numel = _array_info(phi)
    w_ptr, w_code, w_numel = _array_info(W)
    if p_code != w_code or p_numel != w_numel:
        raise ValueError("phi and W must have the same dtype and shape")
    pr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    _check(load().ace_exchange_w_noalloc(ctypes.byref(desc), p_ptr, p_code,
                                         pr.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), len(pr), w_ptr,
                                         _stream_handle(stream)))
    return W


# ---- one build over several GPUs: the per-rank steps (the caller runs the collectives) ----

def ace_exchange_w(desc: AceDesc, phi, pairs, W, stream=None):
    """Partial W of Eq. (vx) over the listed pairs only, written into W ([norb][N], working dtype)."""
    p_ptr, p_code, p_numel = _array_info(phi)
    w_ptr, w_code, w_numel = _array_info(W)
    N = desc.n[0] * desc.n[1] * desc.n[2]
    if p_numel != desc.norb * N or w_numel != desc.norb * N:
        raise ValueError("phi and W must hold norb x N values")
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    _check(load().ace_exchange_w(ctypes.byref(desc), p_ptr, p_code, pr.ctypes.data if len(pr) else None, len(pr),
                                 w_ptr, _stream_handle(stream)))
    return W


def ace_m_partial(desc: AceDesc, phi_slab, W_slab, M, stream=None):
    """M_partial = -dV Phi_slab^T W_slab (FP64 [norb][norb] device tensor M) over a slab of points."""
    p_ptr, p_code, p_numel = _array_info(phi_slab)
    w_ptr, w_code, w_numel = _array_info(W_slab)
    m_ptr, m_code, m_numel = _array_info(M)
    if p_code != w_code or p_numel != w_numel or p_numel % desc.norb or m_code != ACE_F64 or m_numel != desc.norb ** 2:
        raise ValueError("phi_slab and W_slab: [norb][npts] of one dtype; M: FP64 [norb][norb]")
    _check(load().ace_m_partial(ctypes.byref(desc), p_ptr, w_ptr, p_code, p_numel // desc.norb, m_ptr,
                                _stream_handle(stream)))
    return M


def ace_build_from_m(desc: AceDesc, M, W_slab, stream=None, check: bool = True):
    """Operator on a slab of points from the summed M (App. A); the handle holds xi_slab."""
    m_ptr, m_code, m_numel = _array_info(M)
    w_ptr, w_code, w_numel = _array_info(W_slab)
    if m_code != ACE_F64 or m_numel != desc.norb ** 2 or w_numel % desc.norb:
        raise ValueError("M: FP64 [norb][norb]; W_slab: [norb][npts]")
    npts = w_numel // desc.norb
    h = ctypes.c_void_p()
    st = load().ace_build_from_m(ctypes.byref(desc), m_ptr, w_ptr, w_code, npts, _stream_handle(stream),
                                 ctypes.byref(h))
    d = AceDesc.from_buffer_copy(desc)
    op = AceOp(h.value, d) if h.value else None
    if op is not None:
        op.npts = npts
    if check:
        _check(st, op)
    return op if check else (st, op)


def ace_apply_coeffs(op: AceOp, psi, C, stream=None):
    """C = dV xi^T psi (FP64 [norb][m] device tensor) for psi of m rows of the handle's points."""
    p_ptr, p_code, p_numel = _array_info(psi)
    c_ptr, c_code, c_numel = _array_info(C)
    m = c_numel // op.norb
    if c_code != ACE_F64 or c_numel != op.norb * m or m < 1 or p_numel % m:
        raise ValueError("C must be FP64 [norb][m] with psi of m rows")
    _check(load().ace_apply_coeffs(op.handle, p_ptr, p_code, m, c_ptr, _stream_handle(stream)))
    return C


def ace_apply_finish(op: AceOp, C, out, stream=None):
    """out = -xi C for the summed C (FP64 [norb][m] device tensor); out of m rows of the handle's points."""
    c_ptr, c_code, c_numel = _array_info(C)
    o_ptr, o_code, o_numel = _array_info(out)
    m = c_numel // op.norb
    if c_code != ACE_F64 or c_numel != op.norb * m or m < 1 or o_numel % m:
        raise ValueError("C must be FP64 [norb][m] with out of m rows")
    _check(load().ace_apply_finish(op.handle, c_ptr, o_code, m, o_ptr, _stream_handle(stream)))
    return out


# ---- convenience readers (host numpy copies) ----

def get_numpy(op: AceOp, what: int) -> np.ndarray:
    n = op.norb
    N = getattr(op, "npts", None) or op.desc.n[0] * op.desc.n[1] * op.desc.n[2]
    work = np.float64 if op.desc.prec == ACE_FP64 else np.float32
    if what in (ACE_GET_XI, ACE_GET_W):
        out = np.empty((n, N), dtype=work)
    elif what == ACE_GET_PAIRS:
        out = np.empty((ace_pair_count(op), 2), dtype=np.int32)
    else:
        out = np.empty((n, n), dtype=np.float64)
    return ace_get(op, what, out)
