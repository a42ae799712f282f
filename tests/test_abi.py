"""The C-ABI library builds, loads and exports every entry point that
include/pp.h declares; host-side argument handling needs no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "pp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pp_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2405_05700_b300 import build
    build.build()
    from paper_2405_05700_b300 import pp
    return pp


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("pp_create", "pp_destroy", "pp_load_geometry", "pp_load_ice", "pp_propagate",
                 "pp_propagate_batch", "pp_propagate_batch_async", "pp_debug_trace"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(so, n)]
    assert not missing, missing
    # and the binding wraps each of them under the same name
    assert sorted(lib.EXPORTS) == _declared()
    for n in _declared():
        assert hasattr(lib, n)


def test_defaults_and_error_strings(lib):
    cfg = lib.pp_config_default()
    assert cfg.max_steps == 100000 and cfg.world_margin_m == 100.0
    assert cfg.depth_of_z0_m == 1950.0 and cfg.scatter_coeff_is_effective == 1
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8):
        assert lib.pp_strerror(code)
    assert lib.pp_strerror(-99) == "unknown error"
    assert lib._lib.pp_config_default(None) == lib.PP_EINVAL
    assert lib._lib.pp_destroy(None) == lib.PP_OK


def test_bad_arguments_are_refused_without_a_device(lib):
    # NULL context / bad config never reach CUDA
    assert lib._lib.pp_load_ice(None, None, None, 0, 0.0, 10.0, 0.9) == lib.PP_EINVAL
    assert lib._lib.pp_propagate(None, 0, None, 0, None, None) == lib.PP_EINVAL
    cfg = lib.pp_config_default()
    cfg.max_steps = 0
    h = ctypes.c_void_p()
    assert lib._lib.pp_create(ctypes.byref(cfg), ctypes.byref(h)) == lib.PP_EINVAL


def test_source_struct_layout_matches_workloads(lib):
    from paper_2405_05700_b300 import workloads as W
    assert ctypes.sizeof(lib.pp_source) == W.SOURCE_DTYPE.itemsize
    for name, _ in lib.pp_source._fields_:
        assert getattr(lib.pp_source, name).offset == W.SOURCE_DTYPE.fields[name][1]


def test_oracle_library_loads(orc):
    assert orc.lib() is not None


def test_issue_rate_probe_checks_its_arguments(lib):
    rate = ctypes.c_double()
    assert lib._lib.pp_measure_issue_rate(0, 7, ctypes.byref(rate), None) == lib.PP_EINVAL
    assert lib._lib.pp_measure_issue_rate(0, lib.PP_ISSUE_FP32_FMA, None, None) == lib.PP_EINVAL


def test_surrogate_entry_points_refuse_null_handles(lib):
    """Argument checks that happen before any device work."""
    L = lib._lib
    assert L.pp_mlp_set_activation(None, lib.PP_MLP_ACT_SILU) == lib.PP_EINVAL
    assert L.pp_mlp_set_exact_silu(None, 0) == lib.PP_EINVAL
    assert L.pp_mlp_train_step_rows(None, None, None, None, 10, None, 64, ctypes.c_float(1e-3),
                                    None) == lib.PP_EINVAL
    assert L.pp_mlp_near_pairs(None, None, 0, ctypes.c_float(1.0), 0, None, None, None) == lib.PP_EINVAL
    assert lib.PP_MLP_ACT_SILU == 0 and lib.PP_MLP_ACT_HARD_SWISH == 1


def test_hit_acceptance_is_checked_on_the_host(lib):
    L = lib._lib
    assert L.pp_set_hit_acceptance(None, None, 0) == lib.PP_EINVAL


def test_wait_probe_checks_its_arguments(lib):
    flag, ns = ctypes.c_int32(), ctypes.c_uint64()
    assert lib._lib.pp_debug_wait_timeout(0, 10, ctypes.byref(flag), ctypes.byref(ns)) == lib.PP_EINVAL
    assert lib._lib.pp_debug_wait_timeout(0, 10 ** 10, ctypes.byref(flag),
                                          ctypes.byref(ns)) == lib.PP_EINVAL
    assert lib._lib.pp_debug_wait_timeout(0, 10 ** 6, None, None) == lib.PP_EINVAL
