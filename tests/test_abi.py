"""The C-ABI library builds, loads and exports every function its header declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes

import pytest

from paper_2010_05371_gb300 import api, build


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_header_declares_entry_points():
    names = api.header_functions()
    for required in ("eap_dtw", "subseq_search", "subseq_search_ex", "subseq_search_host",
                     "eap_dtw_host", "eapdtw_strerror", "eapdtw_version", "eapdtw_release_scratch"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in api.header_functions() if not hasattr(L, n)]
    assert missing == []


def test_error_strings(libpath):
    assert api.strerror(0) == "ok"
    assert "invalid" in api.strerror(-1)
    assert api.strerror(-99) == "unknown error code"
    assert "sm_103a" in api.version()


def test_argument_errors_need_no_gpu(libpath):
    """Invalid arguments are rejected on the host before any CUDA call."""
    L = api.lib()
    out = ctypes.c_double(0)
    assert L.eap_dtw(None, 3, None, 3, 1, 1.0, None, None) == -1
    assert L.eap_dtw_host(None, 3, None, 3, 1, 1.0, ctypes.byref(out)) == -1
    assert L.subseq_search(None, 4, None, 10, 1, 1, None, None, None) == -1
    buf = (ctypes.c_float * 8)()
    i64 = (ctypes.c_int64 * 2)()
    f64 = (ctypes.c_double * 2)()
    # lQ > lR, w < 0, k < 1, NaN ub
    assert L.subseq_search(buf, 8, buf, 4, 1, 1, i64, f64, None) == -1
    assert L.subseq_search(buf, 4, buf, 8, -1, 1, i64, f64, None) == -1
    assert L.subseq_search(buf, 4, buf, 8, 1, 0, i64, f64, None) == -1
    assert L.eap_dtw(buf, 4, buf, 4, 1, float("nan"), f64, None) == -1
    # beyond this build's limits
    assert L.subseq_search(buf, 5000, buf, 6000, 1, 1, i64, f64, None) == -6
    assert L.subseq_search(buf, 4, buf, 8, 1, 65, i64, f64, None) == -6


def test_context_argument_errors_need_no_gpu(libpath):
    """The context and batch entry points reject invalid arguments before any CUDA call."""
    L = api.lib()
    assert L.eapdtw_ctx_create(0, 0, None) == -1
    assert L.eapdtw_ctx_create(0, -5, ctypes.byref(ctypes.c_void_p())) == -1
    assert L.eapdtw_ctx_destroy(None) == -1
    assert L.eapdtw_ref_register(None, None, 10, None, None) == -1
    assert L.eapdtw_ref_unregister(None, 0) == -1
    assert L.eapdtw_search_batch(None, None, 1, 1, None, None, None, None) == -1
    assert L.eapdtw_autotune(None, None, 1, 1000, None, None) == -1
    assert L.eapdtw_set_first_tile(None, 5, 1, 1, 8) == -1
    assert L.eapdtw_ctx_info(None, None, 1) == -1
    # the item struct of the binding has the header's layout
    assert ctypes.sizeof(api.Item) == 40


def test_serving_argument_errors_need_no_gpu(libpath):
    L = api.lib()
    rid = ctypes.c_int64(0)
    assert L.eapdtw_serve_start(None, 4, 1 << 16) == -1
    assert L.eapdtw_serve_stop(None) == -1
    assert L.eapdtw_serve_submit(None, None, 10, 0, 1, 1, 0, ctypes.byref(rid)) == -1
    assert L.eapdtw_serve_poll(None, 1, None, None, None, 0) == -1
    assert L.eapdtw_serve_cancel(None, 1) == -1
    assert L.eapdtw_serve_stats(None, None, 1) == -1
    assert api.strerror(-9) == "request cancelled"
    assert api.strerror(1) == "pending"


def test_whole_series_argument_errors_need_no_gpu(libpath):
    L = api.lib()
    assert L.eapdtw_pairwise(None, 1, None, 1, 10, 1, 1, None, None) == -1
    assert L.eapdtw_nn(None, 1, None, 1, 10, 1, 1, 1, None, None, None) == -1
