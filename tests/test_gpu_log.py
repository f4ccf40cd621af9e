"""The logarithm the primitive recovery uses for the transport fits' ln T
(Tang's table-driven method): within one unit in the last place of the
correctly rounded logarithm (300-bit references on a sample that includes
x near 1 and the table's nodes), within two of CUDA's log and the host's
over the temperatures the solver meets and the whole positive normal range,
and CUDA's log itself outside the positive normal doubles."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ulps(a, b):
    return np.abs(a.view(np.int64) - b.view(np.int64))


def test_table_driven_log_within_one_ulp():
    import mpmath as mp
    import torch
    from paper_2403_05910_b300 import build
    build.build()
    from paper_2403_05910_b300.xf import probe_log
    rng = np.random.default_rng(11)
    n = 1 << 21
    nodes = np.ldexp(1.0 + np.arange(129) / 128.0, rng.integers(-20, 20, 129))
    near1 = np.concatenate([1.0 - rng.uniform(0.0, 0.02, 4000), 1.0 + rng.uniform(0.0, 0.02, 4000)])
    x = np.concatenate([
        rng.uniform(100.0, 6000.0, n),                       # temperatures (K)
        np.exp(rng.uniform(-700.0, 700.0, n // 4)),          # the positive normal range
        near1, nodes, np.nextafter(nodes, 0.0), np.nextafter(nodes, 2.0 * nodes),
        np.array([1.0, 2.0, 0.5, 1e-300, 2.2250738585072014e-308, 1.7976931348623157e308]),
        np.array([0.0, -1.0, 5e-324, np.inf, np.nan]),       # outside: CUDA's log
    ])
    xd = torch.from_numpy(x).cuda()
    y, ref = torch.empty_like(xd), torch.empty_like(xd)
    probe_log(xd, y, ref)
    torch.cuda.synchronize()
    y, ref = y.cpu().numpy(), ref.cpu().numpy()
    normal = (x >= 2.2250738585072014e-308) & np.isfinite(x)
    u = _ulps(y[normal], ref[normal])
    assert u.max() <= 2, (u.max(), x[normal][np.argmax(u)])
    with np.errstate(divide="ignore", invalid="ignore"):
        host = np.log(x)
    uh = _ulps(y[normal], host[normal])
    assert uh.max() <= 2, (uh.max(), x[normal][np.argmax(uh)])
    # the correctly rounded logarithm on a sample: every temperature-range
    # point would be slow in 300-bit arithmetic
    mp.mp.prec = 300
    idx = np.concatenate([rng.integers(0, n, 1500), np.arange(n + n // 4, normal.size - 11)])
    idx = idx[normal[idx]]
    exact = np.array([float(mp.log(mp.mpf(float(v)))) for v in x[idx]])
    ue = _ulps(y[idx], exact)
    assert ue.max() <= 1, (ue.max(), x[idx][np.argmax(ue)])
    assert np.all(y[x == 1.0] == 0.0)
    out = ~normal
    assert np.array_equal(y[out], ref[out], equal_nan=True)
