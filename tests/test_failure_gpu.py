"""Failure detection on the GPU without a fault: a bounded wait that nothing
satisfies gives up, records WS_DEV_TIMEOUT in a status word the host reads,
and the context keeps working."""
import numpy as np
import pytest

import oracle
from paper_2203_02479_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ws():
    import torch
    from paper_2203_02479_gb300 import build, wiresim
    build.build()
    wiresim.load_library()
    torch.cuda.set_device(0)
    return wiresim


def test_bounded_wait_gives_up_and_context_survives(ws):
    import torch
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    cycles = torch.zeros(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    iters = 1000
    ws.ws_selftest_bounded_wait(status.data_ptr(), iters, cycles.data_ptr(), stream)
    torch.cuda.synchronize()
    assert int(status.item()) & ws.WS_DEV_TIMEOUT
    per_try = int(cycles.item()) / iters
    # the kernels' own bound (2^18 attempts) ends in about a second
    full_s = per_try * (1 << 18) / 2.07e9
    print(f"\nbounded wait: {per_try:.0f} cycles per attempt, full bound ~{full_s:.3f} s")
    assert 0 < full_s < 2.0
    # the context is still usable: a small simulation matches the oracle
    d = inputs.uniform_depos(100, 16, seed=5, nticks=500)
    R = inputs.response()
    plane = ws.Plane(16, 500, R)
    out = plane.simulate(ws.DeviceDepos.from_plane_depos(d), ws.Params())
    torch.cuda.synchronize()
    ref = oracle.simulate(d.q, d.x_mm, d.t_us, 16, 500, R, 10)
    assert np.linalg.norm(out.cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-5
    assert plane.status() == 0


def test_bounded_wait_rejects_bad_arguments(ws):
    import torch
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(ws.WiresimError):
        ws.ws_selftest_bounded_wait(status.data_ptr(), 0, 0, 0)
    with pytest.raises(ws.WiresimError):
        ws.ws_selftest_bounded_wait(0, 10, 0, 0)
