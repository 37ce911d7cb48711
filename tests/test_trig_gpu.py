"""Accuracy of the FP32 joint sine/cosine of the common-normal-frame kernels
(rd_joint_trig), against float64 sin/cos of the same float32 angles."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _eval(rd, x, fast=False):
    import torch

    xt = torch.from_numpy(x).cuda()
    s, c = rd.joint_trig(xt, fast=fast)
    torch.cuda.synchronize()
    return s.cpu().numpy().astype(np.float64), c.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("span", [np.pi, 50.0, 1e4, 1e5])
def test_polynomial_sincos_under_one_ulp(cuda_lib, span):
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.uniform(-span, span, 1 << 20),
                        np.linspace(-span, span, 1 << 18)]).astype(np.float32)
    # quadrant boundaries and exact multiples of pi/2 inside the span
    k = np.arange(-8, 9)
    x = np.concatenate([x, (k * np.pi / 2).astype(np.float32)])
    s, c = _eval(cuda_lib, x)
    xd = x.astype(np.float64)
    assert np.max(np.abs(s - np.sin(xd))) < 1.2e-7
    assert np.max(np.abs(c - np.cos(xd))) < 1.2e-7


def test_polynomial_sincos_special_values(cuda_lib):
    x = np.array([0.0, -0.0, 1e-30, -1e-30, 1e-7], dtype=np.float32)
    s, c = _eval(cuda_lib, x)
    assert np.all(c == 1.0)
    assert np.array_equal(s, x.astype(np.float64))


def test_sfu_sincos_within_its_bound(cuda_lib):
    x = np.random.default_rng(4).uniform(-np.pi, np.pi, 1 << 18).astype(np.float32)
    s, c = _eval(cuda_lib, x, fast=True)
    xd = x.astype(np.float64)
    assert np.max(np.abs(s - np.sin(xd))) < 1e-6
    assert np.max(np.abs(c - np.cos(xd))) < 1e-6


def test_joint_trig_rejects_bad_arguments(cuda_lib):
    import torch

    with pytest.raises(ValueError):
        cuda_lib.joint_trig(torch.zeros(4, dtype=torch.float64, device="cuda"))
