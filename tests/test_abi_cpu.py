"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every entry point include/wiresim.h declares, and the
host-only planner answers workspace sizes and rejects bad descriptions."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2203_02479_gb300 import build, wiresim
    build.build()
    return wiresim.load_library()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:ws_status|const char\*)\s+(ws_\w+)\s*\(", txt, re.M))
    return names


def test_every_declared_symbol_is_exported(lib):
    from paper_2203_02479_gb300 import wiresim
    declared = _declared()
    assert declared, "no declarations parsed"
    assert declared == set(wiresim.EXPORTED)
    for name in declared:
        assert hasattr(lib, name), name


def _desc(**kw):
    from paper_2203_02479_gb300 import wiresim
    d = dict(nwires=960, nticks=6000, pitch_mm=5.0, tick_us=0.5, resp_nwires=21, resp_nticks=200,
             resp_wire_center=10, conv_mode=0, fft_len_tick=0, nsigma=3.0, plane_id=0)
    d.update(kw)
    return wiresim.WsPlaneDesc(**d)


def test_workspace_bytes_and_planner(lib):
    from paper_2203_02479_gb300 import wiresim
    n = wiresim.ws_plane_workspace_bytes(_desc())
    # two nwires x round32(6250/2+1) complex64 spectra and one float grid dominate
    big = 2 * 960 * 3136 * 8 + 960 * 6000 * 4
    assert big <= n < big + 4 * 1024 * 1024
    assert n % 256 == 0
    # circular mode: transform at the grid length itself
    assert wiresim.ws_plane_workspace_bytes(_desc(conv_mode=1)) < n


@pytest.mark.parametrize("kw,code", [
    (dict(nwires=0), 1), (dict(resp_wire_center=21), 1), (dict(pitch_mm=0.0), 1),
    (dict(conv_mode=3), 1), (dict(plane_id=16), 1), (dict(resp_nwires=23, resp_wire_center=11), 2),
    (dict(conv_mode=1, nticks=6007), 2), (dict(fft_len_tick=7000), 2),
    (dict(fft_len_tick=6000), 1), (dict(nticks=20000), 2)])
def test_planner_rejects(lib, kw, code):
    from paper_2203_02479_gb300 import wiresim
    with pytest.raises(wiresim.WiresimError) as ei:
        wiresim.ws_plane_workspace_bytes(_desc(**kw))
    assert ei.value.status == code


def test_null_arguments_rejected_without_device_work(lib):
    from paper_2203_02479_gb300 import wiresim
    assert lib.ws_simulate(None, None, None, None, None) == 1
    assert lib.ws_convolve(None, None, None, None) == 1
    assert lib.ws_plane_sync(None, None, None) == 1
    assert lib.ws_plane_destroy(None) == 0
    d = _desc()
    h = ctypes.c_void_p(0)
    # workspace missing -> WS_ERR_WORKSPACE before any CUDA call
    assert lib.ws_plane_create(ctypes.byref(d), ctypes.c_void_p(256), None, 0, None, ctypes.byref(h)) == 6
    assert lib.ws_status_string(2) == b"unsupported size"
    assert lib.ws_status_string(99) == b"unknown status"
    from paper_2203_02479_gb300 import wiresim
    info = wiresim.WsPlaneInfo()
    assert lib.ws_plane_get_info(None, ctypes.byref(info)) == 1


def test_impact_planes_in_the_planner(lib):
    """Impact planes: the fine grid (nwires*I x nticks floats), I times the
    compensated path's low-part grid, and I times the first spectra, the
    response spectra, the adjoint's taps and the response gradient's
    spectra; with FP64 buffers also I times their double grid, first
    spectra and response spectra; more than 32 positions are refused before
    any device work."""
    from paper_2203_02479_gb300 import wiresim
    plain = wiresim.ws_plane_workspace_bytes(_desc())
    imp = wiresim.ws_plane_workspace_bytes(_desc(impacts=10))
    extra = 2 * 960 * 10 * 6000 * 4 - 960 * 6000 * 4 + 9 * 960 * 3136 * 8 + 3 * 9 * 21 * 3136 * 8
    assert extra <= imp - plain < extra + 1024 * 1024
    assert wiresim.ws_plane_workspace_bytes(_desc(impacts=1)) == plain
    plain64 = wiresim.ws_plane_workspace_bytes(_desc(fp64=1))
    imp64 = wiresim.ws_plane_workspace_bytes(_desc(impacts=10, fp64=1))
    extra64 = 9 * 960 * 6000 * 8 + 9 * 960 * 3136 * 16 + 9 * 21 * 3136 * 16
    assert extra + extra64 <= imp64 - plain64 < extra + extra64 + 2 * 1024 * 1024
    for kw, code in ((dict(impacts=33), 1), (dict(impacts=-1), 1)):
        with pytest.raises(wiresim.WiresimError) as ei:
            wiresim.ws_plane_workspace_bytes(_desc(**kw))
        assert ei.value.status == code


def test_new_entry_points_reject_null_planes(lib):
    """ws_plane_set_noise, like every entry point, answers a null plane with
    WS_ERR_INVALID_ARG and touches no device."""
    assert lib.ws_plane_set_noise(None, None, None, 0, None) == 1
    assert lib.ws_convolve_noalloc(None, None, None, None, None) == 1
