"""Host-side checks of the C ABI (no GPU needed): the library builds and
loads, exports every function include/fhgs.h declares, the ctypes structs
match the C layout, and the host-only helpers behave."""
import ctypes
import os
import re
import subprocess

import pytest
import torch

from paper_2505_19154_gb300 import _build, api

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fhgs.h")


@pytest.fixture(scope="module")
def L():
    _build.build()
    return api.lib()


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fhgs_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(L, n), n
    assert set(api.EXPORTS) <= set(names)
    nm = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(r"\sT\s" + n + r"$", nm, re.M), n


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "fhgs.h"\nint main(void){\n'
                   'printf("%zu %zu %zu %zu\\n", sizeof(fhgs_camera), sizeof(fhgs_params), sizeof(fhgs_gaussians), sizeof(fhgs_bins));\n'
                   'printf("%zu %zu %zu\\n", offsetof(fhgs_params, znear), offsetof(fhgs_params, bg), offsetof(fhgs_bins, capacity));\n'
                   'return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()
    want = [ctypes.sizeof(api.Camera), ctypes.sizeof(api.Params), ctypes.sizeof(api.Gaussians),
            ctypes.sizeof(api.Bins), api.Params.znear.offset, api.Params.bg.offset, api.Bins.capacity.offset]
    assert [int(x) for x in out] == want


def test_host_helpers(L):
    p = api.make_params(sh_degree=3)
    assert (p.tile_w, p.tile_h, p.sh_degree) == (16, 16, 3)
    assert abs(p.alpha_min - 1 / 255) < 1e-9 and abs(p.alpha_max - 0.99) < 1e-7
    assert abs(p.t_eps - 1e-4) < 1e-10 and p.cutoff_sq == 9.0 and abs(p.dilation - 0.3) < 1e-7
    cams = api.make_cameras([dict(width=1920, height=1080, fx=1.0, fy=1.0, cx=0, cy=0, w2c=[[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]]),
                             dict(width=17, height=16, fx=1.0, fy=1.0, cx=0, cy=0, w2c=[[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]])])
    assert L.fhgs_total_tiles(cams, 2) == 120 * 68 + 2 * 1
    assert L.fhgs_total_tiles(cams, 0) == -1
    assert L.fhgs_proj_bytes(1000, 2) >= 2000 * (48 + 16 + 8)
    assert L.fhgs_proj_bytes(-1, 1) == -1
    assert L.fhgs_abi_version() == 2
    assert L.fhgs_status_string(api.ERR_CAPACITY) == b"instance buffer overflow"


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-device error on a CPU-only host")
def test_create_without_device_fails_cleanly(L):
    h = ctypes.c_void_p()
    assert L.fhgs_create(ctypes.byref(h), 0) == api.ERR_NO_DEVICE
    assert not h.value


def test_null_context_is_rejected(L):
    p = api.make_params()
    assert L.fhgs_sync_status(None, None) == api.ERR_INVALID_ARG
    assert L.fhgs_reserve(None, 1, None, 1) == api.ERR_INVALID_ARG
    assert L.fhgs_project(None, None, None, 0, ctypes.byref(p), None, None) == api.ERR_INVALID_ARG
    assert L.fhgs_ndfd_fwd(None, 0, None, None, None, None, 0, 64, None, 1, ctypes.byref(p), 20.0, 0.5, None, None,
                           None, None, None) == api.ERR_INVALID_ARG
    assert L.fhgs_ndfd_bwd(None, None, None, None, None, None, 0, 64, None, 1, ctypes.byref(p), 20.0, 0.5, None, None,
                           None, None, None, None, None, None, None) == api.ERR_INVALID_ARG


def test_new_calls_reject_a_null_context_and_size_the_adam_state(L):
    p = api.make_params()
    assert L.fhgs_point_features(None, 0, None, None, 1, None, 8, None, ctypes.byref(p), None, None, None,
                                 None) == api.ERR_INVALID_ARG
    assert L.fhgs_l1_loss(None, 0, None, None, 1.0, None, None, None) == api.ERR_INVALID_ARG
    opt = api.Adam()
    assert L.fhgs_adam_gaussians(None, 0, 0, *([None] * 5), None, 1, None, ctypes.byref(opt), None, None,
                                 None) == api.ERR_INVALID_ARG
    assert L.fhgs_activate_gaussians(None, 0, None, None, None, None, None) == api.ERR_INVALID_ARG
    assert L.fhgs_sum(None, 0, None, None, None) == api.ERR_INVALID_ARG
    for deg in range(4):
        K = (deg + 1) ** 2
        assert L.fhgs_adam_state_floats(1000, deg) == 2 * 1000 * (11 + 3 * K)
    assert L.fhgs_adam_state_floats(-1, 0) == -1 and L.fhgs_adam_state_floats(10, 4) == -1


def test_wait_probe_knob_is_host_side(L):
    """fhgs_debug_wait_probe only stores a limit: 0 and up to 10 s are taken,
    longer limits are rejected; nothing is launched."""
    assert L.fhgs_debug_wait_probe(10_000_000_001) == api.ERR_INVALID_ARG
    assert L.fhgs_debug_wait_probe(1000) == api.OK
    assert L.fhgs_debug_wait_probe(0) == api.OK


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-device error on a CPU-only host")
def test_noalloc_status_without_device_fails_cleanly(L):
    assert L.fhgs_noalloc_sync_status(None) == api.ERR_NO_DEVICE
