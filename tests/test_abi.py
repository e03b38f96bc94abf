"""CPU checks of the C-ABI boundary: the library builds, loads and exports
every function declared in include/dawn.h; the Python binding carries the
same names.  No compute call is made (no GPU here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dawn.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?(?:int|void|char\s*\*|const char\s*\*)\s*\*?\s*(dawn_\w+)\s*\(",
                                 text, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2306_07872_gb300 import build
    try:
        subprocess.run(["nvcc", "--version"], check=True, capture_output=True)
    except (OSError, subprocess.CalledProcessError):
        pytest.skip("nvcc not available")
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dawn_create_graph", "dawn_sssp", "dawn_msssp", "dawn_destroy", "dawn_sssp_roots",
                     "dawn_sssp_backward", "dawn_status"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    import torch  # noqa: F401  (puts the CUDA runtime on the loader path like the tests do)
    lib = ctypes.CDLL(lib_path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (dawn_\w+)", out))
    assert set(declared_functions()) <= exported


def test_binding_has_the_same_names(lib_path):
    import paper_2306_07872_gb300 as pkg
    for name in declared_functions():
        assert hasattr(pkg.dawn, name), name
    assert set(pkg.EXPORTS) == set(declared_functions())
    assert pkg.dawn_status_string(5).startswith("DAWN_ERR_TIMEOUT")


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2306_07872_gb300 import dawn
    saved = dawn._lib
    dawn._lib = None
    try:
        with pytest.raises(ImportError):
            dawn.load_library(str(tmp_path / "missing.so"))
    finally:
        dawn._lib = saved


def test_oracle_is_not_imported_by_the_package():
    pkg_dir = os.path.join(ROOT, "paper_2306_07872_gb300")
    for dirpath, _, files in os.walk(pkg_dir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "graphgen" not in text, f


def test_tune_cache_keys_and_store(tmp_path):
    from paper_2306_07872_gb300 import dawn as d
    k1 = d.tune_cache_key(4194304, 65243778, 0, "sssp", 8, "GB300/152")
    assert k1 == d.tune_cache_key(4000000, 66000000, 0, "sssp", 8, "GB300/152")  # same shape class
    assert k1 != d.tune_cache_key(4194304, 65243778, 1, "sssp", 8, "GB300/152")  # weight type
    assert k1 != d.tune_cache_key(4194304, 16769024, 0, "sssp", 8, "GB300/152")  # degree
    assert k1 != d.tune_cache_key(4194304, 65243778, 0, "msssp", 8, "GB300/152")  # mode
    assert k1 != d.tune_cache_key(4194304, 65243778, 0, "sssp", 8, "B200/148")  # GPU model
    path = str(tmp_path / "tune.json")
    assert d.tune_cache_load(path) == {}
    res = {"ctas_per_sm": 4, "grid_blocks": 608, "batch": 0, "best_ms": 1.0, "default_ms": 1.1, "candidates": 11,
           "frontier": 2}
    d.tune_cache_store(path, k1, res)
    d.tune_cache_store(path, "other", dict(res, grid_blocks=0))
    got = d.tune_cache_load(path)
    assert got[k1]["grid_blocks"] == 608 and got["other"]["grid_blocks"] == 0 and "candidates" not in got[k1]
    assert got[k1]["frontier"] == 2
    (tmp_path / "bad.json").write_text("not json")
    assert d.tune_cache_load(str(tmp_path / "bad.json")) == {}


def test_host_argument_checks_reject_before_any_device_call(lib_path):
    """Malformed sizes, a bad weight type, missing arrays and a NULL handle are
    refused by the host-side checks of every entry point with
    DAWN_ERR_INVALID; none of these paths reaches the CUDA runtime, so the
    calls are safe without a GPU."""
    import ctypes as C
    import numpy as np
    from paper_2306_07872_gb300 import dawn as d
    lib = d.load_library(lib_path)
    rp = np.array([0, 1, 1], dtype=np.int32)
    col = np.array([1], dtype=np.int32)
    w = np.array([3], dtype=np.uint32)
    ptr = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    out = C.c_void_p(12345)

    def create(n, m, r=ptr(rp), c=ptr(col), wt=ptr(w), wtype=d.DAWN_W_U32):
        out.value = 12345
        rc = lib.dawn_create_graph(n, m, r, c, wt, wtype, 0, None, C.byref(out))
        assert out.value is None, "a refused call must clear *out"
        return rc

    assert create(0, 1) == d.DAWN_ERR_INVALID                        # no vertices
    assert create(-5, 1) == d.DAWN_ERR_INVALID
    assert create(2, -1) == d.DAWN_ERR_INVALID                       # negative edge count
    assert create(2, 1 << 31) == d.DAWN_ERR_INVALID                  # edge ids must fit int32
    assert create(2, 1, r=None) == d.DAWN_ERR_INVALID                # missing row pointers
    assert create(2, 1, c=None) == d.DAWN_ERR_INVALID                # missing columns with m > 0
    assert create(2, 1, wt=None) == d.DAWN_ERR_INVALID               # missing weights with m > 0
    assert create(2, 1, wtype=7) == d.DAWN_ERR_INVALID               # unknown weight type
    assert lib.dawn_create_graph(2, 1, ptr(rp), ptr(col), ptr(w), 0, 0, None, None) == d.DAWN_ERR_INVALID

    src = np.zeros(1, dtype=np.int32)
    buf = np.zeros(4, dtype=np.float32)
    INV = d.DAWN_ERR_INVALID
    assert lib.dawn_set_weights(None, ptr(w), 0, None) == INV
    assert lib.dawn_reserve(None, 1) == INV
    assert lib.dawn_sssp(None, 0, ptr(buf), None, None, None) == INV
    assert lib.dawn_msssp(None, ptr(src), 1, ptr(buf), None, None) == INV
    assert lib.dawn_sssp_roots(None, ptr(src), 1, ptr(buf), None, None, None) == INV
    assert lib.dawn_sssp_backward(None, ptr(src), ptr(buf), ptr(buf), None) == INV
    assert lib.dawn_sssp_noalloc(None, 0, ptr(buf), None, None, None, None) == INV
    assert lib.dawn_status(None, 0) == INV
    assert lib.dawn_get_stats(None, None) == INV
    assert lib.dawn_set_option(None, d.DAWN_OPT_BATCH, 1) == INV
    assert lib.dawn_get_trace(None, None, 0) == -INV
    assert lib.dawn_graph_info(None, None, None, None) == INV
    assert lib.dawn_autotune(None, d.DAWN_TUNE_SSSP, ptr(src), 1, 1, None, None) == INV
    lib.dawn_destroy(None)  # a NULL handle is a no-op


def test_stream_marshalling():
    # the binding passes streams as cudaStream_t values: an already marshalled
    # handle (the legacy default stream is NULL) and integer handles pass through
    import ctypes
    from paper_2306_07872_gb300 import dawn
    assert dawn._stream(ctypes.c_void_p(None)).value is None
    h = ctypes.c_void_p(0x1234)
    assert dawn._stream(h) is h
    assert dawn._stream(0x5678).value == 0x5678
    assert dawn._stream(0).value is None
