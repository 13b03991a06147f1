"""The pivot reciprocal of the factor kernels (an FP32 seed and two FP64
Newton-Raphson steps, csrc/pivot.cuh) against CUDA's FP64 division, over a
sweep of pivots: magnitudes from 1e-36 to 1e36 (the range the Newton path
takes) on both signs, values near powers of two and random significands, and
the division path outside that range.  Newton's method squares the FP32 seed's
relative error (2^-23) twice, so the result is within one ulp of the correctly
rounded 1/d; outside the range the kernel divides, so the two agree exactly."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _ulps(a, b):
    ia = a.view(np.int64)
    ib = b.view(np.int64)
    return np.abs(ia - ib)


def test_pivot_reciprocal_within_one_ulp_of_division():
    torch = _torch()
    from paper_1907_05420_gb300 import binding as B

    rng = np.random.default_rng(1907)
    mags = 10.0 ** rng.uniform(-36, 36, 200_000)
    sig = rng.choice([-1.0, 1.0], mags.size)
    pw = np.ldexp(1.0, np.arange(-119, 120))
    near = np.concatenate([pw, np.nextafter(pw, 0), np.nextafter(pw, np.inf), 3.0 * pw[:-2]])
    inside = np.concatenate([mags * sig, near, -near])
    outside = np.array([1e-300, -1e-300, 5e-324, 1e-37, 1e37, -1e300, 1.7e308, 1e-40])
    d = np.concatenate([inside, outside])
    dev = torch.device("cuda:0")
    dt = torch.from_numpy(d).to(dev)
    r, q = torch.empty_like(dt), torch.empty_like(dt)
    B.kkt_probe_pivot_reciprocal(dt, r, q)
    torch.cuda.synchronize()
    r, q = r.cpu().numpy(), q.cpu().numpy()
    n_in = inside.size
    # CUDA's division is correctly rounded: it equals numpy's on the host
    with np.errstate(over="ignore"):  # 1 / 5e-324 overflows to inf on both
        assert np.array_equal(q, 1.0 / d)
    assert np.all(np.sign(r[:n_in]) == np.sign(d[:n_in]))
    assert _ulps(r[:n_in], q[:n_in]).max() <= 1
    assert np.array_equal(r[n_in:], q[n_in:])
