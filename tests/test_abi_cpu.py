"""CPU-only checks of the C-ABI library: it loads, exports every symbol the header declares,
and host-side argument validation answers without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2009_05534_gb300 import build
    build.build()
    import paper_2009_05534_gb300 as pkg
    return pkg.lib()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ldpc_[a-z0-9_]+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(L):
    import paper_2009_05534_gb300 as pkg
    decl = _declared()
    assert decl, "no declarations found"
    for name in decl:
        assert hasattr(L, name), name
    assert set(pkg.ABI_SYMBOLS) <= decl


def test_status_strings(L):
    for k, v in {0: b"LDPC_OK", 1: b"LDPC_ERR_INVALID_ARG", 5: b"LDPC_ERR_TIMEOUT"}.items():
        assert L.ldpc_status_string(k) == v


def test_default_opts(L):
    import paper_2009_05534_gb300 as pkg
    o = pkg.DecodeOpts()
    L.ldpc_decode_opts_default(ctypes.byref(o))
    assert (o.llr_type, o.algo, o.offset_q, o.punct_cols, o.early_stop, o.cluster_size) == \
        (pkg.LLR_INT8, pkg.OFFSET, 1, 2, 1, 1)
    assert abs(o.alpha - 0.75) < 1e-7
    assert o.threads_per_row == 0
    # the binding's structure has the header's size (the last field is threads_per_row)
    assert ctypes.sizeof(pkg.DecodeOpts) == 56


def test_invalid_args_rejected_on_host(L):
    import numpy as np
    h = ctypes.c_void_p()
    base = np.zeros((4, 8), np.int16)
    p = base.ctypes.data_as(ctypes.c_void_p)
    assert L.ldpc_graph_create(None, 4, 8, 2, 16, ctypes.byref(h)) == 1
    assert L.ldpc_graph_create(p, 0, 8, 2, 16, ctypes.byref(h)) == 1
    assert L.ldpc_graph_create(p, 4, 8, 8, 16, ctypes.byref(h)) == 1       # K_b >= N_bg
    assert L.ldpc_graph_create(p, 4, 8, 2, 0, ctypes.byref(h)) == 1
    assert L.ldpc_graph_create(p, 4, 8, 2, 2048, ctypes.byref(h)) == 1
    bad = base.copy()
    bad[0, 0] = -5
    assert L.ldpc_graph_create(bad.ctypes.data_as(ctypes.c_void_p), 4, 8, 2, 16,
                               ctypes.byref(h)) == 1
    assert L.ldpc_graph_create(p, 4, 8, 2, 16, None) == 1
    assert L.ldpc_decode(None, None, 1, 10, None, None, None, None) == 1
    assert L.ldpc_graph_edges(None, 0) == -1
    assert L.ldpc_graph_destroy(None) == 1


def test_flooding_and_learned_entry_points_reject_null_graph(L):
    L.ldpc_flooding_workspace_floats.restype = ctypes.c_size_t
    L.ldpc_flooding_workspace_floats.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
    assert L.ldpc_flooding_workspace_floats(None, 4, 0) == 0
    assert L.ldpc_decode_flooding(None, None, 1, 10, None, None, None, None, None, None) == 1
    L.ldpc_learned_workspace_floats.restype = ctypes.c_size_t
    L.ldpc_learned_workspace_floats.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int]
    assert L.ldpc_learned_workspace_floats(None, 4, 10, 0) == 0
    assert L.ldpc_learned_forward_iter(None, None, 1, 10, 0, 0, None, None, None, None) == 1
    assert L.ldpc_learned_backward_iter(None, None, 1, 10, 0, 0, None, None, None, None, None,
                                        0) == 1


def test_selftest_rejects_bad_limits_on_host(L):
    L.ldpc_selftest_wait_timeout.argtypes = [ctypes.c_uint, ctypes.c_void_p, ctypes.c_void_p]
    assert L.ldpc_selftest_wait_timeout(0, None, None) == 1
    assert L.ldpc_selftest_wait_timeout((1 << 22) + 1, None, None) == 1


def test_work_item_word_layout(L):
    """The raw-word view of a work-item table (the serving path's) puts each field where
    the C struct has it: four pointers in words 0..3, then the three ints packed in words 4
    and 5; the word offsets the serving backend patches are those of hard_bits and iters."""
    import numpy as np

    import paper_2009_05534_gb300 as pkg
    assert pkg.WORK_ITEM_WORDS * 8 == ctypes.sizeof(pkg.WorkItem) == pkg.work_item_dtype.itemsize
    t = np.zeros(3, dtype=pkg.work_item_dtype)
    t["graph"], t["llr"], t["hard_bits"], t["iters"] = 11, 22, 33, 44
    t["n_rows"], t["n_tx"], t["max_iter"] = 5, 6, 7
    w = t.view(np.uint64).reshape(3, pkg.WORK_ITEM_WORDS)
    assert (w[:, 0] == 11).all() and (w[:, 1] == 22).all()
    assert (w[:, pkg.WorkItem.hard_bits.offset // 8] == 33).all()
    assert (w[:, pkg.WorkItem.iters.offset // 8] == 44).all()
    c = pkg.WorkItem.from_buffer_copy(t[1].tobytes())
    assert (c.graph, c.llr, c.hard_bits, c.iters) == (11, 22, 33, 44)
    assert (c.n_rows, c.n_tx, c.max_iter) == (5, 6, 7)


def test_host_side_rejections_of_the_serving_entries(L):
    """Malformed work-item word arrays and row maps are refused on the host, before any
    library or device call."""
    import numpy as np

    import paper_2009_05534_gb300 as pkg
    good = np.zeros((4, pkg.WORK_ITEM_WORDS), np.uint64)
    for bad in (good.astype(np.int64), good[:, :5].copy(), good[::2], good.reshape(-1)):
        with pytest.raises(ValueError):
            pkg.decode_list_words(bad)
    with pytest.raises(ValueError):
        pkg.decode_rows_host_maps(None, None, np.zeros(3, np.int32), np.zeros(4, np.int32), 5,
                                  bits=None, iters=None)
    with pytest.raises(ValueError):
        pkg.decode_rows_host_maps(None, None, np.zeros((2, 2), np.int32),
                                  np.zeros((2, 2), np.int32), 5, bits=None, iters=None)


def test_storage_model_matches_the_paper():
    """Sec. IV storage model: the paper's printed S_v and S_c->v for BG1 at Z = 384 (8-bit
    and 16-bit values) from the per-codeword state the decoders keep on chip."""
    import json

    import paper_2009_05534_gb300 as pkg
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_storage.json")))
    Z, n_vars, E = g["Z"], g["N_bg"] * g["Z"], g["E_bg1"]
    for eps in (1, 2):
        s_v, s_c = pkg.state_bytes(n_vars, E, Z, eps)
        # the paper prints whole kB (1000 B), truncated: 121 344 B -> 121, 242 688 B -> 242
        assert s_v // 1000 == g["S_v_kB"][str(eps)]
        assert s_c // 1000 == g["S_c2v_kB"][str(eps)]
    # the int8 batch kernel's layout at the headline graph (E = 323): two codewords'
    # binary16 posteriors fill 104 448 B of shared memory and their byte messages 248 064 B
    # of the 256 kB of Tensor Memory
    s_v, _ = pkg.state_bytes(68 * 384, 323, 384, 2)
    _, s_c = pkg.state_bytes(68 * 384, 323, 384, 1)
    assert 2 * s_v == 104448 and 2 * s_c == 248064 <= 256 * 1024
