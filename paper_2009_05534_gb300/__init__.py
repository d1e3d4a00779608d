"""GB300-native layered min-sum LDPC decoder (Ling & Cautereels, "Fast LDPC GPU Decoder for
Cloud RAN").

Thin Python binding over the C ABI declared in ``include/ldpc.h`` (``libldpc.so`` next to
this file).  It only marshals arguments: torch supplies device buffers and the current
CUDA stream, and every step of decoding runs in the library's CUDA kernels.  There is no
CPU fallback: if the library is missing or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libldpc.so")

LLR_INT8, LLR_FP16, LLR_FP32 = 0, 1, 2
NORMALISED, OFFSET, LEARNED, SUM_PRODUCT = 0, 1, 2, 3

_STATUS = {0: "LDPC_OK", 1: "LDPC_ERR_INVALID_ARG", 2: "LDPC_ERR_UNSUPPORTED",
           3: "LDPC_ERR_OUT_OF_MEMORY", 4: "LDPC_ERR_CUDA", 5: "LDPC_ERR_TIMEOUT"}


class LdpcError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {_STATUS.get(status, status)}")
        self.status = status


class WorkItem(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_void_p), ("llr", ctypes.c_void_p),
                ("hard_bits", ctypes.c_void_p), ("iters", ctypes.c_void_p),
                ("n_rows", ctypes.c_int), ("n_tx", ctypes.c_int), ("max_iter", ctypes.c_int)]


class DecodeOpts(ctypes.Structure):
    _fields_ = [("llr_type", ctypes.c_int), ("algo", ctypes.c_int), ("alpha", ctypes.c_float),
                ("offset", ctypes.c_float), ("offset_q", ctypes.c_int), ("n_rows", ctypes.c_int),
                ("n_tx", ctypes.c_int), ("punct_cols", ctypes.c_int),
                ("early_stop", ctypes.c_int), ("cluster_size", ctypes.c_int),
                ("learned_params", ctypes.c_void_p), ("threads_per_row", ctypes.c_int)]


_lib = None
_lock = threading.Lock()

# exported symbols of the C ABI (checked by the CPU test-suite against include/ldpc.h)
ABI_SYMBOLS = ("ldpc_decode_opts_default", "ldpc_graph_create", "ldpc_graph_destroy",
               "ldpc_graph_edges", "ldpc_graph_vars", "ldpc_decode", "ldpc_decode_debug",
               "ldpc_graph_sync_status", "ldpc_status_string", "ldpc_launch_count",
               "ldpc_decode_host", "ldpc_decode_list", "ldpc_decode_list_noalloc",
               "ldpc_learned_workspace_floats", "ldpc_learned_forward", "ldpc_learned_backward",
               "ldpc_learned_forward_iter", "ldpc_learned_backward_iter",
               "ldpc_flooding_workspace_floats", "ldpc_decode_flooding", "ldpc_decode_rows",
               "ldpc_decode_rows_host_maps", "ldpc_selftest_wait_timeout", "ldpc_alloc_count",
               "ldpc_pair_jit", "ldpc_pair_jit_prepare", "ldpc_list_jit_prepare")


def lib():
    """Load libldpc.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(LIB_PATH)
            P, i = ctypes.c_void_p, ctypes.c_int
            L.ldpc_decode_opts_default.argtypes = [ctypes.POINTER(DecodeOpts)]
            L.ldpc_decode_opts_default.restype = None
            L.ldpc_graph_create.argtypes = [P, i, i, i, i, ctypes.POINTER(ctypes.c_void_p)]
            L.ldpc_graph_create.restype = i
            L.ldpc_graph_destroy.argtypes = [P]
            L.ldpc_graph_destroy.restype = i
            L.ldpc_graph_edges.argtypes = [P, i]
            L.ldpc_graph_edges.restype = i
            L.ldpc_graph_vars.argtypes = [P, i]
            L.ldpc_graph_vars.restype = i
            L.ldpc_decode.argtypes = [P, P, i, i, P, ctypes.POINTER(DecodeOpts), P, P]
            L.ldpc_decode.restype = i
            L.ldpc_decode_debug.argtypes = [P, P, i, i, P, ctypes.POINTER(DecodeOpts), P, P,
                                            P, P]
            L.ldpc_decode_debug.restype = i
            L.ldpc_decode_host.argtypes = [P, P, i, i, P, ctypes.POINTER(DecodeOpts), P, P]
            L.ldpc_decode_host.restype = i
            L.ldpc_decode_list.argtypes = [ctypes.POINTER(WorkItem), i, P,
                                           ctypes.POINTER(DecodeOpts)]
            L.ldpc_decode_list.restype = i
            # the same entry point taking the item table as a plain address (raw words)
            L.decode_list_words = L["ldpc_decode_list"]
            L.decode_list_words.argtypes = [P, i, P, ctypes.POINTER(DecodeOpts)]
            L.decode_list_words.restype = i
            L.ldpc_decode_list_noalloc.argtypes = [ctypes.POINTER(WorkItem), i, P,
                                                   ctypes.POINTER(DecodeOpts)]
            L.ldpc_decode_list_noalloc.restype = i
            L.ldpc_graph_sync_status.argtypes = [P, P]
            L.ldpc_graph_sync_status.restype = i
            L.ldpc_status_string.argtypes = [i]
            L.ldpc_status_string.restype = ctypes.c_char_p
            L.ldpc_launch_count.argtypes = []
            L.ldpc_launch_count.restype = ctypes.c_uint64
            L.ldpc_alloc_count.argtypes = []
            L.ldpc_alloc_count.restype = ctypes.c_uint64
            L.ldpc_pair_jit.argtypes = [i]
            L.ldpc_pair_jit.restype = i
            # background compilations must end before the process exits
            import atexit
            atexit.register(L.ldpc_pair_jit, 3)
            L.ldpc_pair_jit_prepare.argtypes = [P, i]
            L.ldpc_pair_jit_prepare.restype = i
            L.ldpc_list_jit_prepare.argtypes = [P, P, i]
            L.ldpc_list_jit_prepare.restype = i
            L.ldpc_decode_rows.argtypes = [P, P, P, P, i, i, P, ctypes.POINTER(DecodeOpts),
                                           P, P]
            L.ldpc_decode_rows.restype = i
            L.ldpc_decode_rows_host_maps.argtypes = L.ldpc_decode_rows.argtypes
            L.ldpc_decode_rows_host_maps.restype = i
            L.ldpc_selftest_wait_timeout.argtypes = [ctypes.c_uint, P,
                                                     ctypes.POINTER(ctypes.c_ulonglong)]
            L.ldpc_selftest_wait_timeout.restype = i
            L.ldpc_flooding_workspace_floats.argtypes = [P, i, i]
            L.ldpc_flooding_workspace_floats.restype = ctypes.c_size_t
            L.ldpc_decode_flooding.argtypes = [P, P, i, i, P, ctypes.POINTER(DecodeOpts), P, P,
                                               P, P]
            L.ldpc_decode_flooding.restype = i
            _lib = L
    return _lib


def _check(st: int, what: str):
    if st != 0:
        raise LdpcError(st, what)


def launch_count() -> int:
    """Kernels launched by libldpc.so since it was loaded."""
    return int(lib().ldpc_launch_count())


def alloc_count() -> int:
    """Device and pinned-host allocations libldpc.so has made since it was loaded."""
    return int(lib().ldpc_alloc_count())


def pair_jit(mode: int = -1) -> int:
    """The per-graph compiled batch kernels: 0 off, 1 compile in the background (default),
    2 compile at first use and wait, 3 wait for background compilations, -1 only query.  Returns the previous mode (bits 0-1),
    plus 4 once a kernel has been compiled and 8 once a compilation has failed
    (ldpc_pair_jit)."""
    return int(lib().ldpc_pair_jit(int(mode)))


def pair_jit_prepare(base, n_rows: int = 0) -> None:
    """Compile the 8-bit kernels (batch, and low-latency at alpha 2 and 4) for the first
    n_rows rows (0: all) of a base table (int array [M][N], -1 = no circulant) and wait
    (ldpc_pair_jit_prepare); raises when the sequence is invalid or a compilation failed."""
    import numpy as np
    b = np.asarray(base)
    n = int(n_rows) or b.shape[0]
    deg = np.ascontiguousarray((b[:n] >= 0).sum(axis=1), dtype=np.int32)
    _check(lib().ldpc_pair_jit_prepare(deg.ctypes.data_as(ctypes.c_void_p), n),
           "ldpc_pair_jit_prepare")


def list_jit_prepare(tables) -> None:
    """Compile the work-list kernel for the row sequences of (base table, n_rows) pairs
    (n_rows 0: every row) and wait (ldpc_list_jit_prepare); an empty list stops using
    compiled list kernels.  Raises when a sequence is invalid or the compilation failed."""
    import numpy as np
    degs, rows = [], []
    for base, n_rows in tables:
        b = np.asarray(base)
        n = int(n_rows) or b.shape[0]
        degs.append((b[:n] >= 0).sum(axis=1))
        rows.append(n)
    d = np.ascontiguousarray(np.concatenate(degs) if degs else np.zeros(1), dtype=np.int32)
    r = np.ascontiguousarray(rows if rows else [0], dtype=np.int32)
    _check(lib().ldpc_list_jit_prepare(d.ctypes.data_as(ctypes.c_void_p),
                                       r.ctypes.data_as(ctypes.c_void_p), len(rows)),
           "ldpc_list_jit_prepare")


class Graph:
    """Device-resident QC base graph lifted by Z (ldpc_graph_create)."""

    def __init__(self, base: np.ndarray, K_b: int, Z: int):
        b = np.ascontiguousarray(base, dtype=np.int16)
        if b.ndim != 2:
            raise ValueError("base table must be 2-D [M_bg][N_bg]")
        h = ctypes.c_void_p()
        _check(lib().ldpc_graph_create(b.ctypes.data_as(ctypes.c_void_p), b.shape[0],
                                       b.shape[1], int(K_b), int(Z), ctypes.byref(h)),
               "ldpc_graph_create")
        self._h = h
        self.M_bg, self.N_bg = b.shape
        self.K_b, self.Z = int(K_b), int(Z)
        self.base = b.copy()

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("graph is closed")
        return self._h

    @property
    def K(self) -> int:
        return self.K_b * self.Z

    def edges(self, n_rows: int = 0) -> int:
        return int(lib().ldpc_graph_edges(self.handle, int(n_rows)))

    def vars(self, n_rows: int = 0) -> int:
        return int(lib().ldpc_graph_vars(self.handle, int(n_rows)))

    def sync_status(self, stream=None):
        _check(lib().ldpc_graph_sync_status(self.handle, _stream_ptr(stream)), "device status")

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().ldpc_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stream_ptr(stream):
    """A torch stream (None: the current one) or a raw stream handle as ctypes.c_void_p."""
    if isinstance(stream, ctypes.c_void_p):
        return stream
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def make_opts(llr_type: int, *, algo=None, alpha=0.75, offset=0.0, offset_q=1, n_rows=0,
              n_tx=0, punct_cols=2, early_stop=True, learned=None,
              threads_per_row=0, cluster_size=1) -> DecodeOpts:
    o = DecodeOpts()
    lib().ldpc_decode_opts_default(ctypes.byref(o))
    o.llr_type = llr_type
    o.algo = (OFFSET if llr_type == LLR_INT8 else NORMALISED) if algo is None else algo
    o.alpha = alpha
    o.offset = offset
    o.offset_q = offset_q
    o.n_rows = n_rows
    o.n_tx = n_tx
    o.punct_cols = punct_cols
    o.early_stop = int(bool(early_stop))
    o.learned_params = None if learned is None else learned.data_ptr()
    o.threads_per_row = int(threads_per_row)
    o.cluster_size = int(cluster_size)
    return o


def _llr_type(t) -> int:
    import torch
    m = {torch.int8: LLR_INT8, torch.float16: LLR_FP16, torch.float32: LLR_FP32}
    if t.dtype not in m:
        raise TypeError(f"unsupported LLR dtype {t.dtype}")
    return m[t.dtype]


def decode(graph: Graph, llr, max_iter: int, *, bits=None, iters=None, stream=None,
           debug: bool = False, **kw):
    """Decode llr [batch][n_tx] (a CUDA tensor of int8 / float16 / float32).

    Returns (bits uint8 [batch][ceil(K/8)], iters int32 [batch]) and, with debug=True,
    also (posteriors [batch][vars], c2v [batch][E*Z]) in the LLR dtype.
    """
    import torch
    if not llr.is_cuda:
        raise ValueError("llr must be a CUDA tensor")
    llr = llr.contiguous()
    B = llr.shape[0]
    lt = _llr_type(llr)
    kw.setdefault("n_tx", llr.shape[1])          # one LLR row per codeword
    o = make_opts(lt, **kw)
    nb = (graph.K + 7) // 8
    dev = llr.device
    if bits is None:
        bits = torch.empty((B, nb), dtype=torch.uint8, device=dev)
    if iters is None:
        iters = torch.empty((B,), dtype=torch.int32, device=dev)
    sp = _stream_ptr(stream)
    if not debug:
        _check(lib().ldpc_decode(graph.handle, ctypes.c_void_p(llr.data_ptr()), B, int(max_iter),
                                 sp, ctypes.byref(o), ctypes.c_void_p(bits.data_ptr()),
                                 ctypes.c_void_p(iters.data_ptr())), "ldpc_decode")
        return bits, iters
    n_rows = kw.get("n_rows", 0)
    post = torch.empty((B, graph.vars(n_rows)), dtype=llr.dtype, device=dev)
    c2v = torch.empty((B, graph.edges(n_rows) * graph.Z), dtype=llr.dtype, device=dev)
    _check(lib().ldpc_decode_debug(graph.handle, ctypes.c_void_p(llr.data_ptr()), B,
                                   int(max_iter), sp, ctypes.byref(o),
                                   ctypes.c_void_p(bits.data_ptr()),
                                   ctypes.c_void_p(iters.data_ptr()),
                                   ctypes.c_void_p(post.data_ptr()),
                                   ctypes.c_void_p(c2v.data_ptr())), "ldpc_decode_debug")
    return bits, iters, post, c2v


def selftest_wait_timeout(spin_limit: int = 1 << 16, stream=None):
    """Run the bounded-wait self-test; returns (status code, SM cycles the wait took)."""
    cyc = ctypes.c_ulonglong(0)
    st = lib().ldpc_selftest_wait_timeout(int(spin_limit), _stream_ptr(stream), ctypes.byref(cyc))
    return st, int(cyc.value)


def decode_rows(graph: Graph, llr, in_rows, out_rows, max_iter: int, *, bits, iters,
                stream=None, check_rows: bool = True, **kw):
    """Decode codewords llr[in_rows[b]] (a CUDA pool [rows][n_tx]) into bits[out_rows[b]] and
    iters[out_rows[b]]; in_rows / out_rows are int32 CUDA tensors of the batch length.
    check_rows reads the maps back to validate them (a device sync); a caller that built
    them from validated indices passes False."""
    import torch
    if not (llr.is_cuda and in_rows.is_cuda and out_rows.is_cuda):
        raise ValueError("llr and the row maps must be CUDA tensors")
    if in_rows.dtype != torch.int32 or out_rows.dtype != torch.int32:
        raise TypeError("row maps must be int32")
    n = in_rows.numel()
    if out_rows.numel() != n:
        raise ValueError("row maps differ in length")
    if check_rows and n and (int(in_rows.max()) >= llr.shape[0] or
                             int(out_rows.max()) >= bits.shape[0] or
                             int(in_rows.min()) < 0 or int(out_rows.min()) < 0):
        raise ValueError("row map outside the buffers")
    llr = llr.contiguous()
    kw.setdefault("n_tx", llr.shape[1])
    o = make_opts(_llr_type(llr), **kw)
    _check(lib().ldpc_decode_rows(graph.handle, ctypes.c_void_p(llr.data_ptr()),
                                  ctypes.c_void_p(in_rows.data_ptr()),
                                  ctypes.c_void_p(out_rows.data_ptr()), n, int(max_iter),
                                  _stream_ptr(stream), ctypes.byref(o),
                                  ctypes.c_void_p(bits.data_ptr()),
                                  ctypes.c_void_p(iters.data_ptr())), "ldpc_decode_rows")
    return bits, iters


def decode_rows_host_maps(graph: Graph, llr, in_rows, out_rows, max_iter: int, *, bits, iters,
                          stream=None, opts: DecodeOpts | None = None, **kw):
    """decode_rows with the row maps given in host memory (int32 numpy arrays of the batch
    length; ldpc_decode_rows_host_maps stages and uploads them on the stream).  opts: a
    DecodeOpts from make_opts, reused across calls instead of building one from kw."""
    i = np.ascontiguousarray(in_rows, dtype=np.int32)
    o_ = np.ascontiguousarray(out_rows, dtype=np.int32)
    if i.shape != o_.shape or i.ndim != 1:
        raise ValueError("row maps must be 1-D and of one length")
    if opts is None:
        if not llr.is_cuda:
            raise ValueError("llr must be a CUDA tensor")
        kw.setdefault("n_tx", llr.shape[1])
        opts = make_opts(_llr_type(llr), **kw)
    _check(lib().ldpc_decode_rows_host_maps(graph.handle, ctypes.c_void_p(llr.data_ptr()),
                                            i.ctypes.data, o_.ctypes.data, len(i),
                                            int(max_iter), _stream_ptr(stream),
                                            ctypes.byref(opts),
                                            ctypes.c_void_p(bits.data_ptr()),
                                            ctypes.c_void_p(iters.data_ptr())),
           "ldpc_decode_rows_host_maps")
    return bits, iters


def decode_flooding(graph: Graph, llr, max_iter: int, *, want_post: bool = False,
                    stream=None, workspace=None, **kw):
    """Flooding-schedule decode of fp32 llr [batch][n_tx] (CUDA): min-sum (algo NORMALISED /
    OFFSET) or sum-product (algo SUM_PRODUCT).  Returns (bits, iters[, posteriors])."""
    import torch
    if not llr.is_cuda or llr.dtype != torch.float32:
        raise ValueError("llr must be a float32 CUDA tensor")
    llr = llr.contiguous()
    B = llr.shape[0]
    kw.setdefault("n_tx", llr.shape[1])
    o = make_opts(LLR_FP32, **kw)
    nb = (graph.K + 7) // 8
    bits = torch.empty((B, nb), dtype=torch.uint8, device=llr.device)
    iters = torch.empty((B,), dtype=torch.int32, device=llr.device)
    post = (torch.empty((B, graph.vars(o.n_rows)), dtype=torch.float32, device=llr.device)
            if want_post else None)
    n = int(lib().ldpc_flooding_workspace_floats(graph.handle, B, o.n_rows))
    if workspace is None or workspace.numel() < n:
        workspace = torch.empty((max(n, 1),), dtype=torch.float32, device=llr.device)
    _check(lib().ldpc_decode_flooding(graph.handle, ctypes.c_void_p(llr.data_ptr()), B,
                                      int(max_iter), _stream_ptr(stream), ctypes.byref(o),
                                      ctypes.c_void_p(bits.data_ptr()),
                                      ctypes.c_void_p(iters.data_ptr()),
                                      None if post is None else ctypes.c_void_p(post.data_ptr()),
                                      ctypes.c_void_p(workspace.data_ptr())),
           "ldpc_decode_flooding")
    return (bits, iters, post) if want_post else (bits, iters)


def decode_host(graph: Graph, llr, max_iter: int, *, bits=None, iters=None, stream=None,
                **kw):
    """Decode host LLRs (a CPU tensor or numpy array, pinned memory preferred) through
    ldpc_decode_host; returns host (bits uint8 [batch][ceil(K/8)], iters int32 [batch])."""
    import torch
    if isinstance(llr, np.ndarray):
        llr = torch.from_numpy(np.ascontiguousarray(llr))
    if llr.is_cuda:
        raise ValueError("decode_host takes host memory")
    llr = llr.contiguous()
    B = llr.shape[0]
    kw.setdefault("n_tx", llr.shape[1])
    o = make_opts(_llr_type(llr), **kw)
    nb = (graph.K + 7) // 8
    if bits is None:
        bits = torch.empty((B, nb), dtype=torch.uint8)
    if iters is None:
        iters = torch.empty((B,), dtype=torch.int32)
    _check(lib().ldpc_decode_host(graph.handle, ctypes.c_void_p(llr.data_ptr()), B,
                                  int(max_iter), _stream_ptr(stream), ctypes.byref(o),
                                  ctypes.c_void_p(bits.data_ptr()),
                                  ctypes.c_void_p(iters.data_ptr())), "ldpc_decode_host")
    return bits, iters


# numpy record layout of ldpc_work_item (pointers as uint64), for building work lists
# without per-item Python objects
work_item_dtype = np.dtype({
    "names": ["graph", "llr", "hard_bits", "iters", "n_rows", "n_tx", "max_iter"],
    "formats": [np.uint64, np.uint64, np.uint64, np.uint64, np.int32, np.int32, np.int32],
    "offsets": [WorkItem.graph.offset, WorkItem.llr.offset, WorkItem.hard_bits.offset,
                WorkItem.iters.offset, WorkItem.n_rows.offset, WorkItem.n_tx.offset,
                WorkItem.max_iter.offset],
    "itemsize": ctypes.sizeof(WorkItem)})


def decode_list_array(items: np.ndarray, *, stream=None, early_stop=True,
                      opts: DecodeOpts | None = None, threads_per_row=0):
    """ldpc_decode_list on a numpy record array of ``work_item_dtype`` (asynchronous).
    opts: a DecodeOpts from make_opts(LLR_INT8, ...) reused across calls (early_stop is then
    taken from it)."""
    arr = np.ascontiguousarray(items, dtype=work_item_dtype)
    o = (make_opts(LLR_INT8, early_stop=early_stop, threads_per_row=threads_per_row)
         if opts is None else opts)
    _check(lib().ldpc_decode_list(arr.ctypes.data_as(ctypes.POINTER(WorkItem)), len(arr),
                                  _stream_ptr(stream), ctypes.byref(o)), "ldpc_decode_list")


WORK_ITEM_WORDS = ctypes.sizeof(WorkItem) // 8


def decode_list_words(words: np.ndarray, *, stream=None, early_stop=True,
                      opts: DecodeOpts | None = None, threads_per_row=0):
    """ldpc_decode_list on work items held as raw 64-bit words: a C-contiguous uint64 array
    [n][WORK_ITEM_WORDS] laid out byte for byte as ``ldpc_work_item`` (e.g.
    ``items.view(np.uint64).reshape(n, -1)`` of a ``work_item_dtype`` array).  Gathering
    and patching rows of such an array is much cheaper than on a record array, which
    matters on a per-slot serving path."""
    if (words.dtype != np.uint64 or words.ndim != 2 or words.shape[1] != WORK_ITEM_WORDS
            or not words.flags.c_contiguous):
        raise ValueError("work items must be a C-contiguous uint64 [n][WORK_ITEM_WORDS] array")
    o = (make_opts(LLR_INT8, early_stop=early_stop, threads_per_row=threads_per_row)
         if opts is None else opts)
    _check(lib().decode_list_words(words.ctypes.data, words.shape[0], _stream_ptr(stream),
                                   ctypes.byref(o)), "ldpc_decode_list")


def decode_list(items, *, stream=None, early_stop=True, threads_per_row=0):
    """Decode a heterogeneous list in one launch (ldpc_decode_list).

    items: sequence of (graph, llr int8 CUDA tensor [n_tx], bits uint8 CUDA tensor
    [ceil(K/8)], iters int32 CUDA tensor [1], n_rows, n_tx, max_iter).  Outputs are written
    in place; the call is asynchronous on the stream.  threads_per_row: 0 picks the
    kernel (2 threads per row pair, messages in Tensor Memory, when every item allows it),
    1 forces the one-thread-per-row-pair list kernel, 2 the low-latency one.
    """
    arr = np.zeros(len(items), dtype=work_item_dtype)
    for k, (g, llr, bits, it, n_rows, n_tx, max_iter) in enumerate(items):
        arr[k] = (g.handle.value, llr.data_ptr(), bits.data_ptr(), it.data_ptr(), int(n_rows),
                  int(n_tx), int(max_iter))
    decode_list_array(arr, stream=stream, early_stop=early_stop,
                      threads_per_row=threads_per_row)


def decode_list_noalloc(items: np.ndarray, *, stream=None, early_stop=True,
                        threads_per_row=0):
    """ldpc_decode_list_noalloc on a numpy record array of ``work_item_dtype``.

    For callers that cannot allocate device memory: the library allocates nothing on this
    path; the work table (at most 2048 items) and the work counter sit in one static device
    array shared by every call, so calls must not overlap on the GPU.  The first call on a
    device looks the array up and should come before any stream capture."""
    arr = np.ascontiguousarray(items, dtype=work_item_dtype)
    o = make_opts(LLR_INT8, early_stop=early_stop, threads_per_row=threads_per_row)
    _check(lib().ldpc_decode_list_noalloc(arr.ctypes.data_as(ctypes.POINTER(WorkItem)), len(arr),
                                          _stream_ptr(stream), ctypes.byref(o)),
           "ldpc_decode_list_noalloc")


def state_bytes(n_vars: int, n_edges: int, Z: int, eps: int) -> tuple[int, int]:
    """Per-codeword decoder state in the storage model of Sec. IV: posteriors
    S_v = eps * N_c and check-to-variable messages S_c->v = eps * Z * sum_r w_r bytes, for
    N_c = n_vars posteriors, sum_r w_r = n_edges circulants and eps bytes per value.

    The batch kernels keep both on chip: the int8 decoder holds posteriors as binary16
    (eps = 2) in shared memory and messages as bytes (eps = 1) in Tensor Memory, the
    binary16 decoder both at eps = 2."""
    if min(n_vars, n_edges, Z, eps) < 0:
        raise ValueError("sizes must be non-negative")
    return eps * n_vars, eps * Z * n_edges


def unpack_bits(packed: np.ndarray, K: int) -> np.ndarray:
    """LSB-first packed hard bits [B][ceil(K/8)] -> uint8 [B][K]."""
    return np.unpackbits(np.asarray(packed, dtype=np.uint8), axis=1, bitorder="little")[:, :K]
