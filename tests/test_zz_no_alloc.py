"""ws_convolve_noalloc: the convolution for callers that cannot allocate.

Some callers (code running under another framework's allocator, plug-ins in
a process whose device memory is reserved up front) cannot call cudaMalloc or
hand over a workspace.  ws_convolve_noalloc takes only the response, the
input grid and the output grid and keeps its scratch in a fixed 16 MiB array
inside the library.  These checks call it through the C ABI twice in a row
(the array keeps the previous call's contents) and compare each result with
the workspace-based ws_convolve on the same inputs and with the FP64
oracle's convolution (Eq. 2), within the relative-L2 tolerance the other GPU
tests use; a third call writes its output over its input (the header allows
grid_dev == out_dev).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

REL_L2 = 1e-5


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2203_02479_gb300 import build, wiresim
    build.build()
    h = wiresim.load_library()
    torch.cuda.set_device(0)
    return h


def _desc(nw, nt, kw, kt, c, circular=False):
    from paper_2203_02479_gb300 import wiresim
    return wiresim.WsPlaneDesc(nw, nt, 5.0, 0.5, kw, kt, c, 1 if circular else 0, 0, 3.0, 0)


def test_noalloc_matches_workspace_convolution_twice(lib):
    import torch
    from paper_2203_02479_gb300 import inputs, wiresim
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(64, 2000, inputs.response("bipolar"), 10, False, 1),
             (37, 960, inputs.response("unipolar"), 10, True, 2)]
    for nw, nt, R, c, circ, seed in cases:
        rng = np.random.Generator(np.random.PCG64(seed))
        S = torch.from_numpy(rng.standard_normal((nw, nt)).astype(np.float32)).cuda()
        Rd = torch.from_numpy(np.ascontiguousarray(R)).cuda()
        out = torch.full((nw, nt), float("nan"), dtype=torch.float32, device="cuda")
        d = _desc(nw, nt, R.shape[0], R.shape[1], c, circ)
        st = lib.ws_convolve_noalloc(ctypes.byref(d), ctypes.c_void_p(Rd.data_ptr()),
                                     ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(stream))
        assert st == 0, lib.ws_last_error()
        plane = wiresim.Plane(nw, nt, R, wire_center=c, circular=circ)
        ref = plane.convolve(S)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        assert np.isfinite(got).all()
        assert _rel_l2(got, ref.cpu().numpy().astype(np.float64)) <= REL_L2
        exact = oracle.convolve_fft(S.cpu().numpy().astype(np.float64), R, c, circ)
        assert _rel_l2(got, exact) <= REL_L2
        # in place: the output buffer is the input grid
        st = lib.ws_convolve_noalloc(ctypes.byref(d), ctypes.c_void_p(Rd.data_ptr()),
                                     ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(S.data_ptr()),
                                     ctypes.c_void_p(stream))
        assert st == 0, lib.ws_last_error()
        torch.cuda.synchronize()
        assert _rel_l2(S.cpu().numpy().astype(np.float64), exact) <= REL_L2


def test_noalloc_rejects_planes_beyond_its_scratch(lib):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    d = _desc(960, 6000, 21, 200, 10)   # two 960 x 3136 complex64 spectra: 48 MB > 16 MiB
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    assert lib.ws_convolve_noalloc(ctypes.byref(d), p, p, p, ctypes.c_void_p(stream)) == 6
