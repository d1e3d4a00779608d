"""CPU-only checks of the per-graph batch kernels (ldpc_pair_jit_prepare): the runtime
compiler turns the embedded kernel headers into a module for a degree sequence without a
GPU, rejects bad sequences on the host, and compiles each sequence once."""
import os
import re
import time

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    from paper_2009_05534_gb300 import build
    build.build()
    import paper_2009_05534_gb300 as p
    return p


def test_embedded_sources_are_the_kernel_headers(pkg):
    """The build embeds the current text of every header the compiled module includes."""
    from paper_2009_05534_gb300 import build
    gen = open(build.JIT_HEADER).read()
    files = dict(re.findall(r'\{"([^"]+)", R"LDPCSRC\((.*?)\)LDPCSRC"\}', gen, re.S))
    assert set(files) == {name for name, _ in build.JIT_FILES}
    for name, path in build.JIT_FILES:
        assert files[name] == open(path).read(), name
    # the module includes nothing outside the embedded set
    for name, text in files.items():
        for inc in re.findall(r'^\s*#include\s+"([^"]+)"', text, re.M):
            assert inc in files, (name, inc)


def test_prepare_compiles_the_headline_sequence_once(pkg):
    from synth import make_workload
    wl = make_workload("BG1", 384, 2, 1.5, seed=0)
    pkg.pair_jit_prepare(wl.base, wl.n_rows)          # compiles (seconds of host time)
    t = time.perf_counter()
    pkg.pair_jit_prepare(wl.base, wl.n_rows)          # cached
    assert time.perf_counter() - t < 0.5
    # a rate-8/9 prefix of the same table is another sequence and compiles on its own
    pkg.pair_jit_prepare(wl.base, 5)


@pytest.mark.parametrize("deg", [[1, 3], [3, 21], [], [3] * 65])
def test_prepare_rejects_bad_sequences(pkg, deg):
    """Degrees outside 2..20 and row counts outside 1..64: LDPC_ERR_INVALID_ARG, at once."""
    import ctypes
    arr = (ctypes.c_int * max(len(deg), 1))(*deg)
    assert pkg.lib().ldpc_pair_jit_prepare(arr, len(deg)) == 1
    assert pkg.lib().ldpc_pair_jit_prepare(None, 3) == 1


def test_list_prepare_compiles_a_set_of_sequences(pkg):
    """The work-list kernel for the BG1- and BG2-shaped tables at two rates each compiles
    on the host; an empty set switches compiled list kernels off."""
    from fractions import Fraction
    from synth import make_workload
    tabs = []
    for kind, rates in (("BG1", ("1/3", "8/9")), ("BG2", ("1/3", "5/6"))):
        for rate in rates:
            wl = make_workload(kind, 64, 1, 2.0, rate=Fraction(rate), seed=0, graph_seed=0)
            tabs.append((wl.base, wl.n_rows))
    pkg.list_jit_prepare(tabs)
    pkg.list_jit_prepare([])


def test_list_prepare_rejects_bad_sets(pkg):
    import ctypes
    L = pkg.lib()
    deg = (ctypes.c_int * 3)(3, 1, 4)
    rows = (ctypes.c_int * 1)(3)
    assert L.ldpc_list_jit_prepare(deg, rows, 1) == 1          # a degree below 2
    assert L.ldpc_list_jit_prepare(None, rows, 1) == 1
    rows0 = (ctypes.c_int * 1)(0)
    assert L.ldpc_list_jit_prepare(deg, rows0, 1) == 1         # no rows
    assert L.ldpc_list_jit_prepare(deg, rows, 65) == 1         # too many sequences
