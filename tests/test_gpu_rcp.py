"""The reciprocal the kernels use in place of IEEE division (Newton-Raphson
iteration for 1/x started from the hardware approximation, two steps)
against CUDA's correctly rounded 1.0 / x: within one unit in the last place
over the normal range, both signs, and exact on powers of two."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ulps(a, b):
    ia, ib = a.view(np.int64), b.view(np.int64)
    return np.abs(ia - ib)


def test_reciprocal_within_one_ulp_of_division():
    import torch
    from paper_2403_05910_b300 import build
    build.build()
    from paper_2403_05910_b300.xf import probe_rcp
    rng = np.random.default_rng(0)
    n = 1 << 21
    mant = rng.uniform(1.0, 2.0, size=n)
    expo = rng.integers(-500, 501, size=n)
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    x = np.concatenate([sign * np.ldexp(mant, expo),
                        np.ldexp(1.0, np.arange(-500, 501)),          # powers of two
                        1.0 + rng.uniform(-1e-12, 1e-12, size=4096)])  # near 1
    xd = torch.from_numpy(x).cuda()
    y, ref = torch.empty_like(xd), torch.empty_like(xd)
    probe_rcp(xd, y, ref)
    torch.cuda.synchronize()
    y, ref = y.cpu().numpy(), ref.cpu().numpy()
    assert np.all(np.isfinite(y))
    u = _ulps(y, ref)
    assert u.max() <= 1, (u.max(), x[np.argmax(u)])
    pow2 = slice(n, n + 1001)
    assert np.array_equal(y[pow2], ref[pow2])
