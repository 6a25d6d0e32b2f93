"""The integer FP64 -> FP32 rounding the FP32 kernels apply to centred
offsets equals IEEE round-to-nearest-even (numpy's cast) in the normal float
range, on the CPU; and equals the GPU's own conversion there (gpu test)."""
import numpy as np
import pytest

from paper_1812_07313_gb300 import qgrav


def _cases(seed=0, n=400000):
    rng = np.random.default_rng(seed)
    # random magnitudes over the whole normal float range, both signs
    e = rng.uniform(-125.0, 127.0, n)
    x = np.sign(rng.standard_normal(n)) * np.exp2(e) * rng.uniform(1.0, 2.0, n)
    # exact halfway points between adjacent floats (ties), and one ulp of double either side
    f = rng.uniform(-1e4, 1e4, 20000).astype(np.float32)
    nxt = np.nextafter(f, np.float32(np.inf))
    half = (f.astype(np.float64) + nxt.astype(np.float64)) / 2.0
    ties = np.concatenate([half, np.nextafter(half, np.inf), np.nextafter(half, -np.inf)])
    # values that round up across a power of two, exact floats, zeros
    edge = np.concatenate([np.nextafter(np.exp2(np.arange(-120, 120.0)), 0.0), f.astype(np.float64),
                           [0.0, -0.0, 1.0, -1.0, float(np.finfo(np.float32).max)]])
    return np.concatenate([x, ties, edge])


def test_host_rounding_is_ieee_nearest_even():
    x = _cases()
    ref = x.astype(np.float32)
    got = qgrav.qg_round_f32_host(x)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_below_normal_range_is_signed_zero():
    x = np.array([1e-39, -1e-39, 1e-300, -1e-300, 5e-324])
    got = qgrav.qg_round_f32_host(x)
    assert np.all(got == 0.0)
    assert np.array_equal(np.signbit(got), np.signbit(x))


@pytest.mark.gpu
def test_device_rounding_matches_hardware_conversion():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    x = _cases(seed=1)
    xd = torch.as_tensor(x).cuda()
    out = torch.empty(len(x), dtype=torch.float32, device="cuda")
    hw = torch.empty_like(out)
    qgrav.qg_round_f32_dev(xd, out, hw)
    o, h = out.cpu().numpy(), hw.cpu().numpy()
    assert np.array_equal(o.view(np.uint32), h.view(np.uint32))
    assert np.array_equal(o.view(np.uint32), x.astype(np.float32).view(np.uint32))
