"""Argument checks of the Python binding that need no GPU: every tensor
whose raw pointer goes to the library is checked for shape, dtype,
contiguity and device before the call, and the depo arrays for length, so
that a wrong argument raises on the host instead of sending a kernel out of
bounds."""
import numpy as np
import pytest
import torch

from paper_2203_02479_gb300 import wiresim


def test_require_accepts_the_exact_tensor():
    t = torch.zeros((4, 7), dtype=torch.float32)
    assert wiresim._require(t, "grid", (4, 7), "cpu") is t
    g = torch.zeros(3, dtype=torch.float64)
    assert wiresim._require(g, "gD", (3,), "cpu", dtype=torch.float64) is g


@pytest.mark.parametrize("make,what", [
    (lambda: torch.zeros((4, 8)), "shape"),
    (lambda: torch.zeros((7, 4)), "shape"),
    (lambda: torch.zeros(28), "shape"),
    (lambda: torch.zeros((4, 7), dtype=torch.float64), "dtype"),
    (lambda: torch.zeros((4, 7), dtype=torch.float16), "dtype"),
    (lambda: torch.zeros((7, 4)).t(), "contiguous"),
    (lambda: torch.zeros((4, 14))[:, ::2], "contiguous"),
    (lambda: np.zeros((4, 7), np.float32), "tensor"),
])
def test_require_rejects(make, what):
    with pytest.raises(ValueError, match=what):
        wiresim._require(make(), "grid", (4, 7), "cpu")


def test_require_checks_the_device():
    t = torch.zeros((2, 3))
    with pytest.raises(ValueError, match="cuda"):
        wiresim._require(t, "out", (2, 3), "cuda")
    with pytest.raises(ValueError, match="cuda:1"):
        wiresim._require(t, "out", (2, 3), "cuda:1")


def test_device_depos_lengths():
    q, x, t = [1.0, 2.0, 3.0], [5.0, 6.0, 7.0], [10.0, 11.0, 12.0]
    d = wiresim.DeviceDepos(q, x, t, [0.5, 0.5, 0.5], [1.0, 1.0, 1.0], device="cpu")
    assert d.n == 3 and d.q.dtype == torch.float32
    c = d.c()
    assert c.n == 3 and c.q and c.sigma_t_us and c.sigma_x_mm
    assert not wiresim.DeviceDepos(q, x, t, device="cpu").c().sigma_t_us   # widths from diffusion
    for bad in (dict(x_mm=x[:2]), dict(t_us=t + [1.0]), dict(sigma_t_us=[0.5, 0.5]),
                dict(sigma_x_mm=[1.0] * 4)):
        kw = dict(q=q, x_mm=x, t_us=t)
        kw.update(bad)
        with pytest.raises(ValueError, match="length"):
            wiresim.DeviceDepos(device="cpu", **kw)
    with pytest.raises(ValueError, match="one-dimensional"):
        wiresim.DeviceDepos(np.ones((2, 2)), np.ones((2, 2)), np.ones((2, 2)), device="cpu")


def test_response_key_tracks_identity_and_in_place_changes():
    """Plane.use_response recomputes the spectrum only when the response's
    key changes: another tensor, another view, or an in-place change (the
    version counter); a detached alias of the same tensor keeps the key."""
    R = torch.ones((21, 200), dtype=torch.float32)
    k = wiresim.Plane._resp_key(R)
    assert k == wiresim.Plane._resp_key(R)
    assert k == wiresim.Plane._resp_key(R.detach())        # same storage, shared version counter
    assert k != wiresim.Plane._resp_key(R.clone())
    assert k != wiresim.Plane._resp_key(R[:, 1:])
    R.mul_(2.0)
    assert k != wiresim.Plane._resp_key(R)
    assert wiresim.Plane._resp_key(np.ones((21, 200), np.float32)) is None
