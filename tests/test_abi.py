"""The C ABI library (no GPU needed): it loads, exports every function include/tkf.h declares,
rejects invalid configurations before touching the device, and the product path never
refers to the test oracle."""
import ctypes as C
import os
import re

import pytest

from paper_1702_06359_gb300 import tkf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1702_06359_gb300 import build
    build.build()
    return tkf.lib()


def test_exports_every_declared_function(lib):
    names = tkf.declared_functions()
    assert {"tkf_create", "tkf_build_hit_index", "tkf_fit", "tkf_build_tracks", "tkf_seed_state"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n
    out = os.popen("nm -D --defined-only %s" % tkf.LIB_PATH).read()
    exported = set(re.findall(r"\bT (tkf_\w+)", out))
    assert set(names) <= exported


def test_default_config_is_the_plain_workload(lib):
    c = tkf.default_config()
    assert c.n_layers == 10 and list(c.radius)[:10] == [4.0 * (l + 1) for l in range(10)]
    assert c.bz == 3.8 and c.chi2_cut == 30.0 and c.n_cand == 6 and c.first_build_layer == 3
    assert c.n_eta_bins == 40 and c.n_phi_bins == 63 and c.eta_min == -2.0 and c.eta_bin_w == 0.1
    assert c.precision == tkf.FP32 and list(c.x_over_x0)[:10] == [0.03] * 10


@pytest.mark.parametrize("field,value", [("n_layers", 2), ("n_layers", 17), ("n_cand", 0), ("n_cand", 17),
                                         ("first_build_layer", 1), ("chi2_cut", 0.0), ("precision", 3),
                                         ("eta_bin_w", 0.0), ("seeds_per_block", -1), ("bz", 0.0)])
def test_invalid_config_is_rejected(lib, field, value):
    c = tkf.default_config(**{field: value})
    h = C.c_void_p()
    assert lib.tkf_create(C.byref(c), C.byref(h)) == tkf.ERR_INVALID
    assert not h.value


def test_radii_must_increase(lib):
    c = tkf.default_config()
    c.radius[3] = c.radius[2]
    h = C.c_void_p()
    assert lib.tkf_create(C.byref(c), C.byref(h)) == tkf.ERR_INVALID


def test_status_strings(lib):
    for code in range(8):
        assert lib.tkf_status_string(code)
    assert lib.tkf_status_string(tkf.ERR_KERNEL) == b"kernel reported an error"


def test_null_arguments(lib):
    assert lib.tkf_create(None, None) == tkf.ERR_INVALID
    assert lib.tkf_destroy(None) == tkf.ERR_INVALID
    assert lib.tkf_hit_index_free(None) == tkf.ERR_INVALID
    assert lib.tkf_build_tracks(None, None, None, None, None, None, None) == tkf.ERR_INVALID


def test_product_path_never_uses_the_oracle():
    pkg = os.path.join(ROOT, "paper_1702_06359_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\boracle\b|tkf_oracle|orc_", text), os.path.join(dirpath, f)


def test_server_options_are_checked_before_any_device_work(lib):
    c = tkf.default_config()
    h = C.c_void_p()
    o = tkf.server_options(result_bytes=1000)  # below one full batch of results
    assert lib.tkf_server_create(C.byref(c), C.byref(o), C.byref(h)) == tkf.ERR_INVALID
    o = tkf.server_options(n_slots=0)
    assert lib.tkf_server_create(C.byref(c), C.byref(o), C.byref(h)) == tkf.ERR_INVALID
    o = tkf.server_options()
    assert o.result_bytes >= o.max_batch_tracks * (29 + c.n_layers) * 4
    c64 = tkf.default_config(precision=tkf.FP64)
    assert lib.tkf_server_create(C.byref(c64), C.byref(o), C.byref(h)) == tkf.ERR_INVALID
    assert not h.value
