"""Host-side contract of the C ABI: the library loads without a GPU, exports every entry
point declared in include/fdm.h, and rejects bad arguments before touching the device."""
import ctypes as C
import os
import re
import subprocess

import pytest

import __graft_entry__
from paper_1911_03225_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return binding.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fdm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fdm_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(binding.EXPORTS) == names


def test_default_params(lib):
    p = binding.default_params(64, 32)
    assert (p.n1, p.n2, p.nz, p.nh, p.dx, p.E, p.nu) == (64, 32, 0, 4, 1.0, 1.0, 0.3)
    assert p.theta == 1.0 and p.cfl == 0.5 and p.precision == binding.FP64 and p.autotune == 1
    assert binding.device_bytes(p) > 5 * 64 * 32 * 8


def test_struct_layouts_match_header(lib, tmp_path):
    """The ctypes mirrors of the header's structs have the C compiler's layout."""
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "fdm.h"\n'
                   'int main(void) { printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(fdm_params),'
                   ' offsetof(fdm_params, autotune), sizeof(fdm_launch_config),'
                   ' offsetof(fdm_launch_config, kernel_us), sizeof(fdm_step_info),'
                   ' offsetof(fdm_step_info, status)); return 0; }\n')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert got == [C.sizeof(binding.CParams), binding.CParams.autotune.offset,
                   C.sizeof(binding.CLaunchConfig), binding.CLaunchConfig.kernel_us.offset,
                   C.sizeof(binding.CStepInfo), binding.CStepInfo.status.offset]


def test_launch_config_rejects_null(lib):
    cfg = binding.CLaunchConfig()
    assert lib.fdm_get_launch_config(None, C.byref(cfg)) == binding.FDM_ERR_INVALID_ARG
    assert lib.fdm_batch_get_launch_config(None, 0, C.byref(cfg)) == binding.FDM_ERR_INVALID_ARG


@pytest.mark.parametrize("field,value", [
    ("n1", 48), ("n1", 8), ("n2", 8192), ("nh", 0), ("nh", 300), ("dx", 0.0), ("nu", 0.5),
    ("theta", 0.5), ("theta", 2.5), ("cfl", 0.0), ("cfl", 1.5), ("velocity_mode", 7),
    ("loading_mode", 4), ("time_level", 2), ("precision", 3), ("E", -1.0), ("autotune", 2)])
def test_invalid_params_rejected_without_device(lib, field, value):
    p = binding.default_params(64, 64)
    setattr(p, field, value)
    assert binding.device_bytes(p) == 0
    h = C.c_void_p(123)
    st = lib.fdm_create(C.byref(p.to_c()), None, C.byref(h))
    assert st == binding.FDM_ERR_INVALID_ARG
    assert h.value is None


def test_null_arguments(lib):
    assert lib.fdm_create(None, None, None) == binding.FDM_ERR_INVALID_ARG
    assert lib.fdm_step(None, 1, None) == binding.FDM_ERR_INVALID_ARG
    assert lib.fdm_static_solve(None) == binding.FDM_ERR_INVALID_ARG
    assert lib.fdm_set_plastic_distortion(None, None) == binding.FDM_ERR_INVALID_ARG
    assert lib.fdm_read_fields(None, 1, None, None, None, None, None, None) == binding.FDM_ERR_INVALID_ARG
    assert lib.fdm_set_mobility_field(None, None) == binding.FDM_ERR_INVALID_ARG
    assert lib.fdm_set_loading(None, 0, 0.0, 0.0, 0.0) == binding.FDM_ERR_INVALID_ARG
    assert lib.fdm_read_stress_planes(None, binding.STRESS_COMPONENTS.index("11"), 0, None, None) == \
        binding.FDM_ERR_INVALID_ARG
    assert lib.fdm_read_stress13_planes(None, 0, None, None) == binding.FDM_ERR_INVALID_ARG
    assert lib.fdm_batch_sync_status(None, None, None) == binding.FDM_ERR_INVALID_ARG
    assert lib.fdm_static_solve_heterogeneous(None, None, 0.0, 1, None, None, None, None) == \
        binding.FDM_ERR_INVALID_ARG
    assert lib.fdm_set_shear_modulus_field(None, None, 0.0, 1) == binding.FDM_ERR_INVALID_ARG
    lib.fdm_destroy(None)   # NULL-safe


def test_status_strings(lib):
    for s in range(10):
        assert binding.status_str(s) not in ("", "unknown status")
    assert binding.status_str(99) == "unknown status"


def test_create_without_gpu_reports_device_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = binding.default_params(64, 64)
    h = C.c_void_p()
    st = lib.fdm_create(C.byref(p.to_c()), None, C.byref(h))
    assert st == binding.FDM_ERR_DEVICE and h.value is None
