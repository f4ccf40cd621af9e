"""Batched form (many uneven 2D instances in one persistent kernel per stage):
bitwise identical to stepping each instance alone, for every launch shape the
autotuner may pick; the bounded grid barrier reports a timeout instead of
hanging."""
import numpy as np
import pytest

from paper_2403_05910_b300 import cases
from oracle.xfo import Oracle

from gpu_util import dev, field_err, gpu_solver

pytestmark = pytest.mark.gpu


def _instances(count=6, scale=4, seed=3):
    return cases.batch(seed, count=count, scale=scale)


def _inputs(cs):
    out = []
    for c in cs:
        U, T = Oracle(c).prim_to_cons()
        out.append((U, T))
    return out


def _batch(cs, ins):
    from paper_2403_05910_b300 import build
    build.build()
    from paper_2403_05910_b300.xf import Batch
    b = Batch(cs)
    for i, (U, T) in enumerate(ins):
        b.set_state(i, dev(U), dev(T))
    return b


def _read(b, cs):
    import torch
    out = []
    for i, c in enumerate(cs):
        U = torch.empty((c.n_v, c.cells), dtype=torch.float64, device="cuda")
        T = torch.empty(c.cells, dtype=torch.float64, device="cuda")
        b.get_state(i, U, T)
        out.append((U, T))
    torch.cuda.synchronize()
    return [(U.cpu().numpy(), T.cpu().numpy()) for U, T in out]


def _plain(c, U, T, steps, dt):
    import torch
    s = gpu_solver(c)
    s.set_state(dev(U), dev(T))
    for _ in range(steps):
        s.step(dt)
    Uo = torch.empty((c.n_v, c.cells), dtype=torch.float64, device="cuda")
    To = torch.empty(c.cells, dtype=torch.float64, device="cuda")
    s.get_state(Uo, To)
    torch.cuda.synchronize()
    st = s.status()
    s.close()
    return Uo.cpu().numpy(), To.cpu().numpy(), st


@pytest.mark.parametrize("dt", [0.0, 1.5e-4])
def test_batch_is_bitwise_identical_to_single_grid_steps(dt):
    cs = _instances()
    assert len({c.n_species for c in cs}) > 1 and len({c.n for c in cs}) > 1
    ins = _inputs(cs)
    b = _batch(cs, ins)
    for _ in range(3):           # odd and even steps: both graph parities
        b.step(dt)
    got = _read(b, cs)
    assert b.status() == 0
    assert b.uses_graph()
    for c, (U, T), (Ug, Tg) in zip(cs, ins, got):
        Up, Tp, st = _plain(c, U, T, 3, dt)
        assert st == 0
        assert np.array_equal(Ug, Up), c.name
        assert np.array_equal(Tg, Tp), c.name
    b.close()


def test_batch_matches_oracle():
    cs = _instances(count=3, scale=4, seed=5)
    ins = _inputs(cs)
    b = _batch(cs, ins)
    b.step(0.0)
    got = _read(b, cs)
    for c, (U, T), (Ug, Tg) in zip(cs, ins, got):
        U1, T1 = U.copy(), T.copy()
        Oracle(c).step(U1, T1, 0.0)
        assert np.max(field_err(Ug, U1, c.dim)) <= 1e-11
    b.close()


def test_every_launch_shape_gives_the_same_bits():
    cs = _instances(count=4, scale=4, seed=7)
    ins = _inputs(cs)
    ref = None
    from paper_2403_05910_b300.xf import lib
    for choice in range(lib.xf_batch_num_candidates()):
        b = _batch(cs, ins)
        b.config(choice)
        b.step(0.0)
        got = _read(b, cs)
        if ref is None:
            ref = got
        else:
            for (Ua, Ta), (Ub, Tb) in zip(ref, got):
                assert np.array_equal(Ua, Ub) and np.array_equal(Ta, Tb), choice
        b.close()


def test_autotune_leaves_state_and_results_unchanged():
    cs = _instances(count=4, scale=4, seed=9)
    ins = _inputs(cs)
    b = _batch(cs, ins)
    before = _read(b, cs)
    choice = b.autotune(steps=1)
    assert 0 <= choice < 12
    after = _read(b, cs)
    for (Ua, Ta), (Ub, Tb) in zip(before, after):
        assert np.array_equal(Ua, Ub) and np.array_equal(Ta, Tb)
    b.step(0.0)
    got = _read(b, cs)
    for c, (U, T), (Ug, Tg) in zip(cs, ins, got):
        Up, Tp, st = _plain(c, U, T, 1, 0.0)
        assert np.array_equal(Ug, Up)
    assert b.status() == 0
    b.close()


def test_bounded_barrier_reports_timeout():
    from paper_2403_05910_b300 import build
    build.build()
    from paper_2403_05910_b300.xf import barrier_probe, FLAG_TIMEOUT
    assert barrier_probe(2_000_000_000, 0) == 0
    # one arrival too many is expected: every block waits ~0.05 s, then reports
    assert barrier_probe(100_000_000, 1) & FLAG_TIMEOUT
    assert barrier_probe(2_000_000_000, 0) == 0   # the device is still usable


def test_full_ensemble_is_bitwise_identical_to_single_grid_steps():
    """The bench's ensemble itself (64 instances, 128x64 .. 768x384, seed 0):
    one CFL step of the autotuned, graph-captured persistent form equals
    stepping each instance alone, bit for bit."""
    cs = cases.batch(0)
    assert len(cs) == 64
    ins = _inputs(cs)
    b = _batch(cs, ins)
    b.autotune(steps=1)
    b.step(0.0)
    got = _read(b, cs)
    assert b.status() == 0
    b.close()
    for c, (U, T), (Ug, Tg) in zip(cs, ins, got):
        Up, Tp, st = _plain(c, U, T, 1, 0.0)
        assert st == 0
        assert np.array_equal(Ug, Up), c.name
        assert np.array_equal(Tg, Tp), c.name


def test_batch_with_periodic_instances_is_bitwise_single_grid():
    """Periodic instances beside a shock-bubble one: the batched kernel
    recomputes every ghost cell, the single-grid step copies the ghost layers
    from their periodic, transmissive and symmetric images; the two agree bit
    for bit."""
    cs = [cases.smooth_periodic(2, (64, 32), 3, seed=4, amp=0.3),
          cases.smooth_periodic(2, (48, 40), 4, seed=5, amp=0.3),
          cases.smooth_periodic(2, (32, 32), 5, seed=6, amp=0.3)] + _instances(count=1, seed=9)
    ins = _inputs(cs)
    b = _batch(cs, ins)
    for _ in range(3):
        b.step(0.0)
    got = _read(b, cs)
    assert b.status() == 0
    b.close()
    for c, (U, T), (Ug, Tg) in zip(cs, ins, got):
        Up, Tp, st = _plain(c, U, T, 3, 0.0)
        assert st == 0
        assert np.array_equal(Ug, Up), c.name
        assert np.array_equal(Tg, Tp), c.name
