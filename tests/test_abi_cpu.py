"""C-ABI checks that need no GPU: the library loads, exports every function
declared in include/cmrt.h, agrees with the binding on the parameter struct,
and rejects bad parameters before touching a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    src = open(os.path.join(ROOT, "include", "cmrt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(cmrt_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def cm():
    from paper_2005_04642_gb300 import cmrt as cm
    if not os.path.exists(cm.LIB_PATH):
        from paper_2005_04642_gb300 import build
        build.build()
    cm.load()
    return cm


def test_exports_every_declared_symbol(cm):
    lib = ctypes.CDLL(cm.LIB_PATH)
    names = _header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    bound = {s[0] for s in cm._SIGNATURES}
    assert set(names) <= bound, set(names) - bound


def test_abi_version_and_struct_size(cm):
    assert cm.cmrt_abi_version() == 10
    assert cm.load().cmrt_params_size() == ctypes.sizeof(cm.cmrt_params)


def test_defaults_are_valid(cm):
    p = cm.cmrt_params()
    assert cm.load().cmrt_params_default(ctypes.byref(p), 64, 32) == cm.CMRT_OK
    assert (p.nx, p.ny, p.stencil_order) == (64, 32, 2)
    assert cm.cmrt_validate(p) == cm.CMRT_OK


@pytest.mark.parametrize("field,value,needle", [
    ("nx", 0, "nx, ny"),
    ("alpha_r", 0.9, "density ratio"),
    ("lambda3_r", 2.0, "lambda3"),
    ("lambda7", 0.0, "lambda6, lambda7"),
    ("sigma", -1.0, "sigma"),
    ("stencil_order", 4, "stencil_order"),
    ("precision", 3, "precision"),
    ("precision_reference", 3, "precision_reference"),
    ("adjoint_fused", 3, "adjoint_fused"),
    ("visc_mode", 3, "visc_mode"),
    ("wall_y", 2, "wall_y"),
    ("rho0_b", 0.0, "rho0"),
])
def test_validation_rejects(cm, field, value, needle):
    p = cm.make_params({"nx": 16, "ny": 16})
    setattr(p, field, value)
    assert cm.cmrt_validate(p) == cm.CMRT_EINVAL
    assert needle in cm.cmrt_last_error(None)
    # cmrt_init validates before it touches a device
    with pytest.raises(cm.CmrtError) as ei:
        cm.cmrt_init(p, 0, 0, 0)
    assert ei.value.status == cm.CMRT_EINVAL


def test_null_context_calls(cm):
    lib = cm.load()
    assert lib.cmrt_step(None, 1) == cm.CMRT_ESTATE
    assert lib.cmrt_set_graph_steps(None, 2) == cm.CMRT_ESTATE
    assert lib.cmrt_get_graph_steps(None) == -1
    assert lib.cmrt_save_bytes(None) == 0
    assert lib.cmrt_save(None, None, 0) == cm.CMRT_ESTATE
    assert lib.cmrt_load(None, None, 0) == cm.CMRT_ESTATE
    assert lib.cmrt_time(None) == -1
    assert lib.cmrt_launch_count(None) == -1
    lib.cmrt_destroy(None)  # no-op
    assert lib.cmrt_init(None, None, None, None, None) == cm.CMRT_EINVAL


def test_make_params_from_workload_dict(cm):
    from paper_2005_04642_gb300 import inputs as I
    d, _, _ = I.layered_channel(nx=32, ny=16)
    p = cm.make_params(d)
    assert p.wall_y == 1 and abs(p.g_acc[0] - 1e-6) < 1e-18
    assert abs(p.alpha_r - 0.995) < 1e-12 and abs(p.rho0_b - 0.01) < 1e-15
    assert cm.cmrt_validate(p) == cm.CMRT_OK


def test_batch_init_validates_before_touching_a_device(cm):
    good = cm.make_params({"nx": 16, "ny": 16})
    bad = cm.make_params({"nx": 16, "ny": 16})
    bad.sigma = -1.0
    with pytest.raises(cm.CmrtError) as ei:
        cm.cmrt_batch_init([good, bad], None, None, 0)
    assert ei.value.status == cm.CMRT_EINVAL and "member 1" in str(ei.value)
    mixed = cm.make_params({"nx": 32, "ny": 8, "precision": 2})
    with pytest.raises(cm.CmrtError) as ei:
        cm.cmrt_batch_init([good, mixed], None, None, 0)
    assert ei.value.status == cm.CMRT_EINVAL and "one storage precision" in str(ei.value)
    with pytest.raises(cm.CmrtError) as ei:
        cm.cmrt_batch_init([], None, None, 0)
    assert ei.value.status == cm.CMRT_EINVAL


def test_null_batch_calls(cm):
    lib = cm.load()
    assert lib.cmrt_batch_step(None, 1) == cm.CMRT_ESTATE
    assert lib.cmrt_batch_tune(None, None, 0, None) == cm.CMRT_ESTATE
    assert lib.cmrt_batch_set_rows(None, 8, 8, 0, 8) == cm.CMRT_ESTATE
    assert lib.cmrt_batch_get_rows(None, 8, 8, 0) == -1
    assert lib.cmrt_batch_size(None) == -1
    assert lib.cmrt_batch_time(None) == -1
    assert lib.cmrt_batch_launch_count(None) == -1
    assert lib.cmrt_batch_work_items(None) == -1
    assert lib.cmrt_batch_device_bytes(None) == 0
    lib.cmrt_batch_destroy(None)  # no-op


def test_order6_constraints(cm):
    p = cm.make_params({"nx": 16, "ny": 16, "stencil_order": 6})
    assert cm.cmrt_validate(p) == cm.CMRT_OK
    p.precision = 2
    assert cm.cmrt_validate(p) == cm.CMRT_EINVAL and "FP32" in cm.cmrt_last_error(None)
    q = cm.make_params({"nx": 16, "ny": 2, "stencil_order": 6, "wall_y": True})
    assert cm.cmrt_validate(q) == cm.CMRT_EINVAL and "ny >= 3" in cm.cmrt_last_error(None)
    q.wall_y = 0
    assert cm.cmrt_validate(q) == cm.CMRT_OK  # periodic: the stencil wraps
    with pytest.raises(cm.CmrtError) as ei:
        cm.cmrt_batch_init([cm.make_params({"nx": 16, "ny": 16, "stencil_order": 6})], None, None, 0)
    assert ei.value.status == cm.CMRT_EINVAL
