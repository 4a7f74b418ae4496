"""The C ABI library builds, loads and exports every symbol include/*.h declares (no GPU needed)."""

import glob
import os
import re

from paper_1603_06442_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(qw_[A-Za-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declares_entry_points():
    names = declared_symbols()
    assert {"qw_plan_create", "qw_plan_destroy", "qw_step", "qw_observables", "qw_last_error"} <= names


def test_library_exports_every_declared_symbol(qwlib):
    for name in sorted(declared_symbols()):
        assert hasattr(qwlib, name), name


def test_binding_covers_header():
    assert declared_symbols() <= set(binding.exported_names())


def test_argument_errors_without_gpu(qwlib):
    import ctypes
    h = ctypes.c_void_p()
    assert qwlib.qw_plan_create(4, 8, 0.1, 0, ctypes.byref(h)) == binding.QW_EINVAL
    assert b"dim" in qwlib.qw_last_error()
    assert qwlib.qw_plan_create(3, 7, 0.1, 0, ctypes.byref(h)) == binding.QW_EINVAL
    assert qwlib.qw_plan_create(1, 8, 1.5, 0, ctypes.byref(h)) == binding.QW_EINVAL
    assert qwlib.qw_plan_create(1, 8, 0.5, 9, ctypes.byref(h)) == binding.QW_EINVAL
    assert qwlib.qw_step(None, None, 1, None) == binding.QW_EINVAL
    assert qwlib.qw_plan_field_elems(None) == -1


def test_new_entry_points_reject_null_plans_without_gpu(qwlib):
    import ctypes
    obs = (binding.qw_obs * 1)()
    out10 = (ctypes.c_double * 10)()
    assert qwlib.qw_run_host(None, None, None, 0, 1, obs, None) == binding.QW_EINVAL
    assert qwlib.qw_projection(None, None, 1, None, None) == binding.QW_EINVAL
    assert qwlib.qw_projection_elems(None, 1) == -1
    assert qwlib.qw_position_moments(None, None, out10, None) == binding.QW_EINVAL
    assert qwlib.qw_fw_transform(None, None, None, None) == binding.QW_EINVAL
    assert b"null" in qwlib.qw_last_error()


def test_keep_masks():
    assert binding.keep_mask({0}) == 1
    assert binding.keep_mask([0, 2]) == 5
    assert binding.keep_mask((1, 2, 0)) == 7
    assert binding.keep_mask(6) == 6
