"""The exponential the primitive recovery uses for the Eq. 29 transport fits
and the binary diffusion fits (Tang's table-driven method) against CUDA's exp
and the host's: within one unit in the last place over the fits' range and
beyond it to |x| = 700, exact at the table's nodes x = k ln2/64 up to the
rounding of x, and CUDA's exp itself outside |x| <= 700."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ulps(a, b):
    return np.abs(a.view(np.int64) - b.view(np.int64))


def test_table_driven_exp_within_one_ulp():
    import torch
    from paper_2403_05910_b300 import build
    build.build()
    from paper_2403_05910_b300.xf import probe_exp
    rng = np.random.default_rng(7)
    n = 1 << 21
    x = np.concatenate([
        rng.uniform(-12.0, 2.0, n),                  # 0.5 ln(mu), 0.5 ln(kappa), -ln(p D)
        rng.uniform(-700.0, 700.0, n // 4),
        np.arange(-64 * 40, 64 * 40) * (np.log(2.0) / 64.0),   # table nodes
        np.array([0.0, -0.0, 1e-300, -1e-300, 709.0, -720.0, 750.0]),
    ])
    xd = torch.from_numpy(x).cuda()
    y, ref = torch.empty_like(xd), torch.empty_like(xd)
    probe_exp(xd, y, ref)
    torch.cuda.synchronize()
    y, ref = y.cpu().numpy(), ref.cpu().numpy()
    finite = np.isfinite(ref)
    assert np.array_equal(np.isfinite(y), finite)
    u = _ulps(y[finite], ref[finite])
    assert u.max() <= 1, (u.max(), x[finite][np.argmax(u)])
    uh = _ulps(y[finite], np.exp(x[finite]))
    assert uh.max() <= 1, (uh.max(), x[finite][np.argmax(uh)])
    far = np.abs(x) > 700.0
    assert np.array_equal(y[far], ref[far])
    assert np.all(y[x == 0.0] == 1.0)
