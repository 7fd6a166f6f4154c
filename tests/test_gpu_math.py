"""Error bounds of the rollout's FP32 function approximations (tanh of the
network layers, tan of the steering angle, sin/cos of the heading) against
correctly rounded values of the same FP32 arguments."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _eval(fn, x):
    import torch
    from paper_1904_06680_gb300 import npp
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    y = torch.empty_like(xd)
    y2 = torch.empty_like(xd) if fn == 2 else None
    npp.npp_math_eval(fn, xd, y, y2)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.float64), None if y2 is None else y2.cpu().numpy().astype(np.float64)


def test_tanh_bound():
    x = np.concatenate([np.linspace(-20, 20, 2_000_001), np.linspace(-1e-3, 1e-3, 20001),
                        [0.0, 1e-30, -1e-30, 88.0, -88.0, 1e4, -1e4]]).astype(np.float32)
    y, _ = _eval(0, x)
    err = np.abs(y - np.tanh(x.astype(np.float64)))
    assert err.max() < 5e-7, (err.max(), x[np.argmax(err)])
    assert np.all(np.abs(y) <= 1.0)
    yi, _ = _eval(0, np.array([np.inf, -np.inf], np.float32))
    assert yi.tolist() == [1.0, -1.0]


def test_tan_bound():
    z = np.linspace(-1, 1, 1_000_001).astype(np.float32)
    y, _ = _eval(1, z)
    err = np.abs(y - np.tan(z.astype(np.float64)))
    assert err.max() < 2e-6, (err.max(), z[np.argmax(err)])


def test_heading_sincos_bound():
    phi = np.concatenate([np.linspace(-1e3, 1e3, 2_000_001),
                          np.linspace(-7, 7, 1_000_001)]).astype(np.float32)
    s, c = _eval(2, phi)
    p64 = phi.astype(np.float64)
    es = np.abs(s - np.sin(p64))
    ec = np.abs(c - np.cos(p64))
    assert es.max() < 1e-6, (es.max(), phi[np.argmax(es)])
    assert ec.max() < 1e-6, (ec.max(), phi[np.argmax(ec)])


def test_fma_peak_microbenchmark():
    """The FMA-stream microbenchmark (roofline denominator) against the
    device's FP32 lanes at its maximum clock: between half and all of it
    (a few per cent above only from clock-reading noise)."""
    import subprocess
    import torch
    from paper_1904_06680_gb300 import npp
    props = torch.cuda.get_device_properties(0)
    try:
        mhz = float(subprocess.run(["nvidia-smi", "-i", "0", "--query-gpu=clocks.max.sm",
                                    "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                   timeout=10).stdout.split()[0])
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        pytest.skip("no SM clock reading")
    derived = props.multi_processor_count * 128 * mhz * 1e6
    for packed in (False, True):
        r = npp.npp_measure_fma_peak(0, packed) / derived
        assert 0.5 < r < 1.05, (packed, r)
    assert npp.lib().npp_measure_fma_peak(0, 2, None) == npp.NPP_INVALID_ARG
