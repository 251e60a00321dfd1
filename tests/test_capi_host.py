"""Host-side checks of the C ABI (no GPU needed): the library builds for sm_103a, loads, exports
every function declared in include/*.h, and its workspace queries and argument checks behave."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

from conftest import ROOT


def _declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?(?:size_t|int64_t|int|char|void)\s*\*?\s*(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = _declared_functions()
    for required in ("cpp_closest_pair", "tsmm_motif", "twolocus_scan", "frnn_query", "cpp_batch",
                     "cpp_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in _declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, flags=re.M))
    assert set(_declared_functions()) <= exported


def test_binding_covers_the_header(libpath):
    from paper_1407_5609_gb300 import capi
    assert set(capi.SIGNATURES) == set(_declared_functions())
    capi.load_library(libpath)


def test_workspace_queries(libpath):
    from paper_1407_5609_gb300 import capi
    a = capi.cpp_closest_pair_workspace_size(4096, 32, "plain_fp32")
    b = capi.cpp_closest_pair_workspace_size(8192, 32, "plain_fp32")
    assert 0 < a < b and a % 256 == 0
    assert capi.cpp_closest_pair_workspace_size(-1, 32, 0) == 0
    assert capi.cpp_closest_pair_workspace_size(10, 0, 0) == 0
    assert capi.tsmm_motif_workspace_size(262144, 512, "filter_fp16") > 261633 * 512 * 2
    assert capi.tsmm_motif_workspace_size(10, 20, 0) == 0
    assert capi.twolocus_scan_workspace_size(4096, 64) > 0
    assert capi.twolocus_scan_workspace_size(4096, 0) == 0
    # reference pruning: only with a tensor-core filter mode, and it needs its own buffers
    assert capi.tsmm_motif_workspace_size(262144, 512, "filter_bf16_prune") > \
        capi.tsmm_motif_workspace_size(262144, 512, "filter_bf16")
    assert capi.cpp_closest_pair_workspace_size(4096, 32, capi.MODE_PRUNE) == 0
    assert capi.cpp_closest_pair_workspace_size(4096, 32, 3 | capi.MODE_PRUNE) == 0


def test_argument_errors_need_no_gpu(libpath):
    """Bad arguments are rejected on the host before any CUDA call."""
    from paper_1407_5609_gb300 import capi
    lib = capi.lib()
    out = capi.cpp_pair_result()
    assert lib.cpp_closest_pair(None, 0, 10, 3, 3, 0, None, None, 0, None) == capi.ERR_ARG
    assert lib.cpp_closest_pair(None, 7, 10, 3, 3, 0, ctypes.byref(out), None, 0, None) == capi.ERR_ARG
    assert b"dtype" in lib.cpp_last_error()
    assert lib.tsmm_motif(None, 100, 10, 5, 0, ctypes.byref(out), None, 0, None) == capi.ERR_ARG
    assert lib.tsmm_motif(ctypes.c_void_p(256), 100, 10, 0, 0, ctypes.byref(out), None, 0, None) == capi.ERR_ARG
    tl = capi.twolocus_result()
    assert lib.twolocus_scan(ctypes.c_void_p(256), 10, 1, 100, 100, ctypes.byref(tl), None, 0, None) == capi.ERR_ARG
    assert b"words" in lib.cpp_last_error()
