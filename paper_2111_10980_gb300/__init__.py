"""Python binding of libnd.so, the GB300 (sm_103a) (r,s) nucleus decomposition library.

Argument marshalling only: every function below calls the C entry point of the same name in
``include/nd.h`` through ctypes; all computation happens in the library's CUDA kernels. If
the library cannot be loaded, every call raises -- there is no CPU fallback.

Arrays may be numpy arrays (host memory) or torch CUDA tensors (device memory; the
ND_PTR_DEVICE flag is set automatically). Typical use::

    import paper_2111_10980_gb300 as nd
    ctx = nd.nd_ctx_create(0)
    g = nd.nd_load_csr(ctx, rowptr, col)          # int64[n+1], int32[2m]
    core, rnd, st = nd.nd_decompose(g, 2, 3)      # k-truss numbers (trussness - 2)
    nd.nd_graph_free(g); nd.nd_ctx_destroy(ctx)
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_PKG, "libnd.so")

ND_OK, ND_EINVAL, ND_ENOMEM, ND_EOVERFLOW, ND_ETIMEOUT, ND_EBUSY, ND_PENDING, ND_EINTERNAL, ND_ECUDA = range(9)
ND_PTR_DEVICE = 0x1
ND_VALIDATE = 0x2
ND_NO_GRAPH = 0x4
ND_PEEL_LOOP_GRAPH = 0x8
ND_PEEL_PERSISTENT = 0x10
ND_CONTRACT_OFF = 0x20
ND_CONTRACT_ALWAYS = 0x40
ND_DENSE_BUCKETS = 0x80
ND_ORIENT_DEGREE = 0
ND_ORIENT_DEGENERACY = 1
ND_LIMIT_DROP_BLOCK = 0x1
STATUS_NAMES = {0: "ND_OK", 1: "ND_EINVAL", 2: "ND_ENOMEM", 3: "ND_EOVERFLOW", 4: "ND_ETIMEOUT", 5: "ND_EBUSY",
                6: "ND_PENDING", 7: "ND_EINTERNAL", 8: "ND_ECUDA"}

# every entry point declared in include/nd.h
API = ["nd_ctx_create", "nd_ctx_set_allocator", "nd_ctx_set_limits", "nd_ctx_set_tuning", "nd_ctx_destroy", "nd_ctx_bytes_in_use", "nd_kernel_launches", "nd_last_error",
       "nd_load_csr", "nd_graph_free", "nd_graph_size", "nd_orient", "nd_graph_reset", "nd_count", "nd_decompose",
       "nd_rounds", "nd_round_times", "nd_rcliques", "nd_nuclei", "nd_hierarchy", "nd_batch_run", "nd_server_create", "nd_submit", "nd_poll", "nd_server_drain",
       "nd_server_destroy", "nd_kcore_noalloc"]
ND_NOALLOC_MAX_VERTICES = 262144


class NdError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {message}")
        self.code = code


class nd_stats(ctypes.Structure):
    _fields_ = [("n_r", ctypes.c_int64), ("n_s", ctypes.c_int64), ("rho", ctypes.c_int64),
                ("max_core", ctypes.c_int64), ("listed", ctypes.c_int64), ("advances", ctypes.c_int64),
                ("refills", ctypes.c_int64), ("count_width", ctypes.c_int32), ("orient_mode", ctypes.c_int32),
                ("t_orient_ms", ctypes.c_double), ("t_index_ms", ctypes.c_double), ("t_count_ms", ctypes.c_double),
                ("t_peel_ms", ctypes.c_double), ("t_total_ms", ctypes.c_double), ("decrements", ctypes.c_int64),
                ("t_phase_ms", ctypes.c_double * 6), ("t_contract_ms", ctypes.c_double),
                ("contractions", ctypes.c_int64), ("t_hash_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["t_phase_ms"] = list(self.t_phase_ms)
        return d


class nd_request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("r", ctypes.c_int32), ("s", ctypes.c_int32),
                ("rowptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("core_out", ctypes.c_void_p),
                ("core_cap", ctypes.c_int64), ("n_r", ctypes.c_int64), ("status", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class nd_batch_stats(ctypes.Structure):
    _fields_ = [("groups", ctypes.c_int32), ("requests", ctypes.c_int32), ("n_r_total", ctypes.c_int64),
                ("n_s_total", ctypes.c_int64), ("rho_max", ctypes.c_int64), ("t_total_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class nd_server_cfg(ctypes.Structure):
    _fields_ = [("mem_budget", ctypes.c_size_t), ("workers", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("queue_cap", ctypes.c_int32), ("flags", ctypes.c_int32)]


class nd_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("batch_size", ctypes.c_int32), ("n_r", ctypes.c_int64),
                ("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double), ("latency_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """Load libnd.so (building it first with nvcc if it is missing). Raises if it cannot be
    built or loaded: the binding never substitutes another implementation."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIBPATH):
            from . import build as _b
            _b.build()
        L = ctypes.CDLL(LIBPATH)
        vp, i32, i64, i32p, i64p = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(
            ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
        L.nd_ctx_create.argtypes = [ctypes.c_int, vp, ctypes.c_size_t, ctypes.POINTER(vp)]
        L.nd_ctx_set_allocator.argtypes = [vp, ALLOC_FN, FREE_FN, vp]
        L.nd_ctx_set_limits.argtypes = [vp, i64, i64, i64, i32]
        L.nd_ctx_set_tuning.argtypes = [vp, ctypes.c_int, ctypes.c_int, i64, i32]
        L.nd_ctx_destroy.argtypes = [vp]
        L.nd_ctx_bytes_in_use.argtypes = [vp]
        L.nd_ctx_bytes_in_use.restype = ctypes.c_size_t
        L.nd_kernel_launches.argtypes = []
        L.nd_kernel_launches.restype = ctypes.c_int64
        L.nd_last_error.argtypes = []
        L.nd_last_error.restype = ctypes.c_char_p
        L.nd_load_csr.argtypes = [vp, i32, vp, vp, ctypes.c_int, ctypes.POINTER(vp)]
        L.nd_graph_free.argtypes = [vp]
        L.nd_graph_size.argtypes = [vp, i32p, i64p]
        L.nd_orient.argtypes = [vp, ctypes.c_int]
        L.nd_graph_reset.argtypes = [vp]
        L.nd_count.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, i64p, i64p]
        L.nd_decompose.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_int,
                                   ctypes.POINTER(nd_stats)]
        L.nd_rounds.argtypes = [vp, vp, vp, i64, i64p]
        L.nd_round_times.argtypes = [vp, vp, i64]
        L.nd_rcliques.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, i64p]
        L.nd_nuclei.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, i32, vp, ctypes.c_int, i64p]
        L.nd_hierarchy.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, ctypes.c_int, i64p]
        L.nd_kcore_noalloc.argtypes = [i32, vp, vp, vp, vp]
        L.nd_batch_run.argtypes = [vp, ctypes.POINTER(nd_request), i32, ctypes.POINTER(nd_batch_stats)]
        L.nd_server_create.argtypes = [vp, ctypes.POINTER(nd_server_cfg), ctypes.POINTER(vp)]
        L.nd_submit.argtypes = [vp, ctypes.POINTER(nd_request), ctypes.POINTER(ctypes.c_uint64)]
        L.nd_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(nd_result)]
        L.nd_server_drain.argtypes = [vp]
        L.nd_server_destroy.argtypes = [vp]
        for name in API:
            if name not in ("nd_ctx_bytes_in_use", "nd_last_error", "nd_kernel_launches"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def _check(rc: int):
    if rc != ND_OK:
        msg = lib().nd_last_error()
        raise NdError(rc, msg.decode() if msg else "")


def _is_torch_cuda(a) -> bool:
    return hasattr(a, "is_cuda") and hasattr(a, "data_ptr") and bool(a.is_cuda)


def _ptr(a):
    """(address, is_device) of a numpy array or torch tensor (None -> (None, False))."""
    if a is None:
        return None, False
    if _is_torch_cuda(a):
        if not a.is_contiguous():
            raise ValueError("device tensors must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), True
    if hasattr(a, "data_ptr"):  # torch CPU tensor
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), False
    if not isinstance(a, np.ndarray) or not a.flags.c_contiguous:
        raise ValueError("host arrays must be C-contiguous numpy arrays")
    return ctypes.c_void_p(a.ctypes.data), False


class Handle:
    """An opaque library handle (context or graph)."""

    def __init__(self, ptr: ctypes.c_void_p, kind: str, owner=None):
        self.ptr = ptr
        self.kind = kind
        self.owner = owner
        self.hooks = None

    @property
    def value(self):
        return self.ptr


def nd_ctx_create(device: int = 0, stream=None, mem_budget: int = 0) -> Handle:
    """Create a context (nd.h: nd_ctx_create). ``stream`` is a torch.cuda.Stream, a raw
    cudaStream_t integer, or None (the library makes its own)."""
    raw = None
    if stream is not None:
        raw = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    out = ctypes.c_void_p()
    _check(lib().nd_ctx_create(int(device), raw, ctypes.c_size_t(int(mem_budget)), ctypes.byref(out)))
    return Handle(out, "ctx")


def nd_ctx_set_allocator(ctx: Handle, alloc, free):
    """Route device allocations through Python callables alloc(bytes, stream) -> int address
    and free(address, bytes, stream) (nd.h: nd_ctx_set_allocator). None restores the default."""
    if alloc is None:
        _check(lib().nd_ctx_set_allocator(ctx.ptr, ALLOC_FN(), FREE_FN(), None))
        ctx.hooks = None
        return
    a = ALLOC_FN(lambda nbytes, stream, user: int(alloc(int(nbytes), stream)) or None)
    f = FREE_FN(lambda p, nbytes, stream, user: free(int(p), int(nbytes), stream))
    _check(lib().nd_ctx_set_allocator(ctx.ptr, a, f, None))
    ctx.hooks = (a, f)  # keep the trampolines alive


def nd_ctx_set_limits(ctx: Handle, max_rounds: int = 0, barrier_timeout_ns: int = 0, count_limit: int = 0,
                      flags: int = 0):
    """Round cap, grid-barrier wait bound, width-4 count limit and test flags of a context
    (nd.h: nd_ctx_set_limits); 0 keeps each default."""
    _check(lib().nd_ctx_set_limits(ctx.ptr, int(max_rounds), int(barrier_timeout_ns), int(count_limit), int(flags)))


def nd_ctx_set_tuning(ctx: Handle, r: int, s: int, heavy_work: int = 0, flags: int = 0):
    """Heavy-phase threshold and extra flags (ND_DENSE_BUCKETS, ND_CONTRACT_OFF) for every
    decomposition of (r,s) on ctx (nd.h: nd_ctx_set_tuning); 0 / 0 restores the defaults."""
    _check(lib().nd_ctx_set_tuning(ctx.ptr, int(r), int(s), int(heavy_work), int(flags)))


def torch_allocator_hooks(device: int = 0):
    """(alloc, free) callables that take device memory from PyTorch's caching allocator."""
    import torch

    def alloc(nbytes, stream):
        return torch.cuda.caching_allocator_alloc(nbytes, device, stream)

    def free(p, nbytes, stream):
        torch.cuda.caching_allocator_delete(p)

    return alloc, free


def nd_ctx_destroy(ctx: Handle):
    _check(lib().nd_ctx_destroy(ctx.ptr))
    ctx.ptr = None


def nd_ctx_bytes_in_use(ctx: Handle) -> int:
    return int(lib().nd_ctx_bytes_in_use(ctx.ptr))


def nd_kernel_launches() -> int:
    """Kernels launched by the library in this process so far (nd.h: nd_kernel_launches)."""
    return int(lib().nd_kernel_launches())


def nd_last_error() -> str:
    m = lib().nd_last_error()
    return m.decode() if m else ""


def nd_load_csr(ctx: Handle, rowptr, col, flags: int = 0) -> Handle:
    """Copy a symmetric CSR graph to the device (nd.h: nd_load_csr)."""
    p_rp, d_rp = _ptr(rowptr)
    p_col, d_col = _ptr(col)
    if d_rp != d_col:
        raise ValueError("rowptr and col must both be host or both be device arrays")
    n = int(rowptr.shape[0]) - 1
    if str(rowptr.dtype).split(".")[-1] != "int64" or str(col.dtype).split(".")[-1] != "int32":
        raise ValueError("rowptr must be int64 and col int32")
    out = ctypes.c_void_p()
    _check(lib().nd_load_csr(ctx.ptr, n, p_rp, p_col, int(flags) | (ND_PTR_DEVICE if d_rp else 0),
                             ctypes.byref(out)))
    return Handle(out, "graph", ctx)


def nd_graph_free(g: Handle):
    if g is not None and g.ptr is not None:
        _check(lib().nd_graph_free(g.ptr))
        g.ptr = None


def nd_graph_size(g: Handle):
    n = ctypes.c_int32()
    m = ctypes.c_int64()
    _check(lib().nd_graph_size(g.ptr, ctypes.byref(n), ctypes.byref(m)))
    return n.value, m.value


def nd_orient(g: Handle, mode: int = ND_ORIENT_DEGREE):
    _check(lib().nd_orient(g.ptr, int(mode)))


def nd_graph_reset(g: Handle):
    _check(lib().nd_graph_reset(g.ptr))


def nd_count(g: Handle, r: int, s: int, count_width: int = 0, out=None):
    """s-clique counts per r-clique (nd.h: nd_count). Returns (counts, n_r, n_s); counts is
    ``out`` if given (host numpy or device tensor of the right width), else a new numpy array."""
    n_r = ctypes.c_int64()
    n_s = ctypes.c_int64()
    _check(lib().nd_count(g.ptr, r, s, count_width, None, 0, ctypes.byref(n_r), None))
    width = count_width
    if out is None:
        if width == 0:
            width = 8  # a host int64 array holds every width; ask the library for 8 bytes
        out = np.zeros(n_r.value, dtype=np.int64 if width == 8 else np.int32)
    else:
        width = out.element_size() if hasattr(out, "element_size") else out.itemsize
    p, dev = _ptr(out)
    _check(lib().nd_count(g.ptr, r, s, width, p, ND_PTR_DEVICE if dev else 0, ctypes.byref(n_r),
                          ctypes.byref(n_s)))
    return out, n_r.value, n_s.value


def nd_decompose(g: Handle, r: int, s: int, count_width: int = 0, core_out=None, round_out=None,
                 flags: int = 0, want_round: bool = True):
    """(r,s) nucleus decomposition (nd.h: nd_decompose). Returns (core, round, stats dict).
    With device tensors for core_out/round_out the results stay on the device."""
    if core_out is None:
        n_r = ctypes.c_int64()
        _check(lib().nd_count(g.ptr, r, s, count_width, None, 0, ctypes.byref(n_r), None))
        core_out = np.zeros(n_r.value, np.int32)
        if want_round and round_out is None:
            round_out = np.zeros(n_r.value, np.int32)
    pc, dc = _ptr(core_out)
    pr, dr = _ptr(round_out)
    if round_out is not None and dc != dr:
        raise ValueError("core_out and round_out must live in the same memory")
    st = nd_stats()
    _check(lib().nd_decompose(g.ptr, r, s, count_width, pc, pr, int(flags) | (ND_PTR_DEVICE if dc else 0),
                              ctypes.byref(st)))
    return core_out, round_out, st.as_dict()


def nd_rounds(g: Handle, cap: int | None = None):
    """(sizes, levels, rho) of the last decomposition on g (nd.h: nd_rounds)."""
    rho = ctypes.c_int64()
    _check(lib().nd_rounds(g.ptr, None, None, 0, ctypes.byref(rho)))
    k = rho.value if cap is None else min(cap, rho.value)
    sizes = np.zeros(max(k, 1), np.int64)
    levels = np.zeros(max(k, 1), np.int64)
    _check(lib().nd_rounds(g.ptr, ctypes.c_void_p(sizes.ctypes.data), ctypes.c_void_p(levels.ctypes.data), k,
                           ctypes.byref(rho)))
    return sizes[:k], levels[:k], rho.value


def nd_round_times(g: Handle, cap: int | None = None) -> np.ndarray:
    """Update wall time per round (ns) of the last decomposition on g (nd.h: nd_round_times)."""
    rho = ctypes.c_int64()
    _check(lib().nd_rounds(g.ptr, None, None, 0, ctypes.byref(rho)))
    k = rho.value if cap is None else min(cap, rho.value)
    out = np.zeros(max(k, 1), np.int64)
    _check(lib().nd_round_times(g.ptr, ctypes.c_void_p(out.ctypes.data), k))
    return out[:k]


def nd_rcliques(g: Handle, r: int, out=None):
    """The r-cliques as ascending tuples in canonical order (nd.h: nd_rcliques)."""
    n_r = ctypes.c_int64()
    _check(lib().nd_rcliques(g.ptr, r, None, 0, ctypes.byref(n_r)))
    if out is None:
        out = np.zeros((n_r.value, r), np.int32)
    p, dev = _ptr(out)
    _check(lib().nd_rcliques(g.ptr, r, p, ND_PTR_DEVICE if dev else 0, ctypes.byref(n_r)))
    return out


def nd_nuclei(g: Handle, r: int, s: int, core, level: int, out=None):
    """Connected nuclei at `level` (nd.h: nd_nuclei): (comp, n_components), comp[i] = smallest
    r-clique id of i's component among the r-cliques with core >= level, -1 elsewhere. core is
    the core array of nd_decompose(g, r, s) (numpy or CUDA tensor); comp follows its kind."""
    n = int(core.shape[0])
    if out is None:
        if _is_torch_cuda(core):
            import torch
            out = torch.empty(n, dtype=torch.int32, device=core.device)
        else:
            out = np.empty(n, np.int32)
    pc, dev = _ptr(core)
    po, dev_o = _ptr(out)
    if dev != dev_o:
        raise ValueError("core and out must both be host arrays or both CUDA tensors")
    nc = ctypes.c_int64()
    _check(lib().nd_nuclei(g.ptr, r, s, pc, int(level), po, ND_PTR_DEVICE if dev else 0, ctypes.byref(nc)))
    return out, nc.value


def nd_hierarchy(g: Handle, r: int, s: int, core):
    """The nucleus hierarchy (nd.h: nd_hierarchy): (comp, parent_level, parent_comp, n_nodes), int32
    arrays of n_r following core's kind (numpy or CUDA tensor). R's node is (core[R], comp[R]); its
    parent node is (parent_level[R], parent_comp[R]), (-1, -1) for a root."""
    n = int(core.shape[0])
    if _is_torch_cuda(core):
        import torch
        outs = [torch.empty(n, dtype=torch.int32, device=core.device) for _ in range(3)]
    else:
        outs = [np.empty(n, np.int32) for _ in range(3)]
    pc, dev = _ptr(core)
    ptrs = [_ptr(o)[0] for o in outs]
    nn = ctypes.c_int64()
    _check(lib().nd_hierarchy(g.ptr, r, s, pc, *ptrs, ND_PTR_DEVICE if dev else 0, ctypes.byref(nn)))
    return outs[0], outs[1], outs[2], nn.value


def nd_kcore_noalloc(rowptr, col, core_out, stream=None):
    """k-core coreness without any allocation by the library (nd.h: nd_kcore_noalloc).

    For callers that cannot let a library allocate device memory (a framework that has reserved
    the GPU's memory in its own pool, or a latency-critical loop where cudaMalloc may
    synchronise). rowptr (int64[n+1]), col (int32) and core_out (int32[n]) must be contiguous
    CUDA tensors on the current device; n <= ND_NOALLOC_MAX_VERTICES. Calls share one static
    scratch array, so calls that overlap on the GPU race: serialise them."""
    for a in (rowptr, col, core_out):
        if not _is_torch_cuda(a):
            raise ValueError("nd_kcore_noalloc takes CUDA tensors (device memory)")
    n = int(rowptr.shape[0]) - 1
    raw = None
    if stream is not None:
        raw = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib().nd_kcore_noalloc(n, _ptr(rowptr)[0], _ptr(col)[0], _ptr(core_out)[0], raw))
    return core_out


def _request(rowptr, col, r, s, core_out):
    for a, dt in ((rowptr, np.int64), (col, np.int32)):
        if not isinstance(a, np.ndarray) or a.dtype != dt or not a.flags.c_contiguous:
            raise ValueError("batch/server requests take contiguous host arrays: rowptr int64, col int32")
    q = nd_request()
    q.n = int(rowptr.shape[0]) - 1
    q.r, q.s = int(r), int(s)
    q.rowptr = rowptr.ctypes.data
    q.col = col.ctypes.data if col.size else None
    if core_out is not None:
        if core_out.dtype != np.int32 or not core_out.flags.c_contiguous:
            raise ValueError("core_out must be a contiguous int32 numpy array")
        q.core_out = core_out.ctypes.data
        q.core_cap = int(core_out.shape[0])
    return q


def nd_batch_run(ctx: Handle, graphs, outs=None):
    """Decompose a batch (nd.h: nd_batch_run). ``graphs`` is a list of (rowptr, col, r, s) with
    host numpy arrays; ``outs`` an optional list of int32 arrays (one per graph, large enough).
    Returns (outs, n_r list, status list, stats dict); allocates outputs when outs is None by
    asking the library for each n_r first."""
    k = len(graphs)
    if outs is None:
        reqs = (nd_request * k)(*[_request(rp, col, r, s, None) for rp, col, r, s in graphs])
        st = nd_batch_stats()
        lib().nd_batch_run(ctx.ptr, reqs, k, ctypes.byref(st))
        outs = [np.zeros(max(int(reqs[i].n_r), 1), np.int32) for i in range(k)]
    reqs = (nd_request * k)(*[_request(rp, col, r, s, o) for (rp, col, r, s), o in zip(graphs, outs)])
    st = nd_batch_stats()
    rc = lib().nd_batch_run(ctx.ptr, reqs, k, ctypes.byref(st))
    n_r = [int(reqs[i].n_r) for i in range(k)]
    status = [int(reqs[i].status) for i in range(k)]
    if rc != ND_OK and all(x != ND_OK for x in status):
        _check(rc)
    return [o[:n] for o, n in zip(outs, n_r)], n_r, status, st.as_dict()


class Server:
    """A continuous-batching server (nd.h: nd_server_create / nd_submit / nd_poll)."""

    def __init__(self, ctx: Handle, mem_budget: int = 0, workers: int = 2, max_batch: int = 64,
                 queue_cap: int = 1 << 20, flags: int = 0):
        cfg = nd_server_cfg(mem_budget, workers, max_batch, queue_cap, flags)
        out = ctypes.c_void_p()
        _check(lib().nd_server_create(ctx.ptr, ctypes.byref(cfg), ctypes.byref(out)))
        self.ptr = out
        self.keep = {}

    def submit(self, rowptr, col, r, s, core_out):
        q = _request(rowptr, col, r, s, core_out)
        t = ctypes.c_uint64()
        _check(lib().nd_submit(self.ptr, ctypes.byref(q), ctypes.byref(t)))
        self.keep[t.value] = (rowptr, col, core_out)  # the library reads them until the final poll
        return t.value

    def poll(self, ticket):
        res = nd_result()
        rc = lib().nd_poll(self.ptr, ctypes.c_uint64(ticket), ctypes.byref(res))
        if rc == ND_EINVAL and ticket not in self.keep:
            _check(rc)
        if rc != ND_PENDING:
            self.keep.pop(ticket, None)
        return rc, res.as_dict()

    def drain(self):
        _check(lib().nd_server_drain(self.ptr))

    def close(self):
        if self.ptr is not None:
            _check(lib().nd_server_destroy(self.ptr))
            self.ptr = None
            self.keep.clear()


def nd_server_create(ctx: Handle, mem_budget: int = 0, workers: int = 2, max_batch: int = 64,
                     queue_cap: int = 1 << 20, flags: int = 0) -> Server:
    return Server(ctx, mem_budget, workers, max_batch, queue_cap, flags)


def nd_submit(sv: Server, rowptr, col, r, s, core_out) -> int:
    return sv.submit(rowptr, col, r, s, core_out)


def nd_poll(sv: Server, ticket: int):
    return sv.poll(ticket)


def nd_server_drain(sv: Server):
    sv.drain()


def nd_server_destroy(sv: Server):
    sv.close()
