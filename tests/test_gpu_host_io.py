"""The state transfers that take host or device pointers (xf_set_state,
xf_set_primitive, xf_get_state): pinned and pageable host buffers give
bitwise the same state, steps and read-back as device buffers. This is the
path the end-to-end benchmark times (pinned host U and T every step)."""
import numpy as np
import pytest

from paper_2403_05910_b300 import cases
from oracle.xfo import Oracle

from gpu_util import dev, field_err, gpu_solver

pytestmark = pytest.mark.gpu


def _case():
    return cases.config(2, n=(24, 12, 10))


def _run(case, U, T, steps=2):
    """Set the state from (U, T) of whatever kind, step, read back to device."""
    import torch
    s = gpu_solver(case)
    s.set_state(U, T)
    for _ in range(steps):
        s.step(0.0)
    Uo = torch.empty((case.n_v, case.cells), dtype=torch.float64, device="cuda")
    To = torch.empty(case.cells, dtype=torch.float64, device="cuda")
    s.get_state(Uo, To)
    torch.cuda.synchronize()
    assert s.status() == 0
    s.close()
    return Uo.cpu().numpy(), To.cpu().numpy()


def test_set_state_from_host_buffers_is_bitwise_the_device_path():
    import torch
    case = _case()
    U, T = Oracle(case).prim_to_cons()
    ref = _run(case, dev(U), dev(T))
    pinned = (torch.from_numpy(U).pin_memory(), torch.from_numpy(T).pin_memory())
    for Ux, Tx in (pinned, (np.ascontiguousarray(U), np.ascontiguousarray(T))):
        got = _run(case, Ux, Tx)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_get_state_into_host_buffers_is_bitwise_the_device_copy():
    import torch
    case = _case()
    U, T = Oracle(case).prim_to_cons()
    s = gpu_solver(case)
    s.set_state(dev(U), dev(T))
    s.step(0.0)
    Ud = torch.empty((case.n_v, case.cells), dtype=torch.float64, device="cuda")
    Td = torch.empty(case.cells, dtype=torch.float64, device="cuda")
    s.get_state(Ud, Td)
    Up = torch.empty((case.n_v, case.cells), dtype=torch.float64).pin_memory()
    Tp = torch.empty(case.cells, dtype=torch.float64).pin_memory()
    s.get_state(Up, Tp)
    Un = np.empty((case.n_v, case.cells))
    s.get_state(Un, None)          # U alone, into pageable memory
    Tn = np.empty(case.cells)
    s.get_state(None, Tn)          # T alone
    torch.cuda.synchronize()
    s.close()
    Ud, Td = Ud.cpu().numpy(), Td.cpu().numpy()
    assert np.array_equal(Up.numpy(), Ud) and np.array_equal(Tp.numpy(), Td)
    assert np.array_equal(Un, Ud) and np.array_equal(Tn, Td)


def test_set_primitive_from_host_is_bitwise_the_device_path():
    import torch
    case = _case()
    out = []
    for P in (dev(case.prim), np.ascontiguousarray(case.prim),
              torch.from_numpy(np.ascontiguousarray(case.prim)).pin_memory()):
        s = gpu_solver(case)
        s.set_primitive(P)
        U = torch.empty((case.n_v, case.cells), dtype=torch.float64, device="cuda")
        T = torch.empty(case.cells, dtype=torch.float64, device="cuda")
        s.get_state(U, T)
        torch.cuda.synchronize()
        s.close()
        out.append((U.cpu().numpy(), T.cpu().numpy()))
    for U, T in out[1:]:
        assert np.array_equal(U, out[0][0]) and np.array_equal(T, out[0][1])
    # and the EOS conversion is the oracle's to round-off
    Uo, To = Oracle(case).prim_to_cons()
    assert np.max(field_err(out[0][0], Uo, case.dim)) <= 1e-13


def test_default_warm_start_converges_to_the_same_state():
    """T_guess = NULL seeds the Newton solve at 300 K: the temperatures it
    recovers equal those from the exact warm start to the Newton tolerance,
    and a step from either agrees to round-off."""
    case = _case()
    U, T = Oracle(case).prim_to_cons()
    a = _run(case, dev(U), dev(T), steps=1)
    b = _run(case, dev(U), None, steps=1)
    assert np.max(np.abs(a[1] - b[1]) / a[1]) <= 1e-12
    assert np.max(field_err(b[0], a[0], case.dim)) <= 1e-12


# (case, options, dt): grid sizes give 1, 2 and 8 slabs of the slowest axis
HOST_STEP = {
    "sbi3d_n5_8slabs": (lambda: cases.config(2, n=(128, 128, 128)), {}, 0.0),
    "sbi2d_n3_8slabs_weno7_blend": (lambda: cases.config(1, n=(2048, 1024)),
                                    {"weno": 7, "positivity": True}, 0.0),
    "sbi2d_n3_2slabs_dsm": (lambda: cases.with_binary_diffusion(cases.config(1, n=(1024, 512)), seed=1),
                            {"diffusion": 1}, 0.0),
    "smooth3d_n3_periodic_2slabs": (lambda: cases.smooth_periodic(3, (64, 64, 128), 3, seed=1, amp=0.3),
                                    {"weno": 6}, 2e-4),
    "tube1d_n2_2slabs": (lambda: cases.shock_tube(0, n=1 << 19), {}, 0.0),
    "sbi2d_n4_1slab": (lambda: cases.config(4, n=(64, 32)), {}, 1e-4),
}


@pytest.mark.parametrize("name", list(HOST_STEP))
def test_host_step_is_bitwise_set_step_get(name):
    """xf_step_rk3_host (slabbed uploads and downloads overlapped with the
    compute) against xf_set_state + xf_step_rk3 + xf_get_state: bitwise equal
    state, warm start and step size, over two steps with U_out = U_in, and
    with a NULL warm start."""
    import torch
    make, kw, dt = HOST_STEP[name]
    case = make()
    s = gpu_solver(case, **kw)
    s.set_primitive(dev(case.prim))
    U0 = torch.empty((case.n_v, case.cells), dtype=torch.float64, device="cuda")
    T0 = torch.empty(case.cells, dtype=torch.float64, device="cuda")
    s.get_state(U0, T0)
    dref = torch.zeros(2, dtype=torch.float64, device="cuda")
    dgot = torch.zeros(2, dtype=torch.float64, device="cuda")
    for warm in (True, False):
        # reference: the three calls
        s.set_state(U0, T0 if warm else None)
        for k in range(2):
            s.step(dt, dref[k:k + 1])
        Ur, Tr = torch.empty_like(U0), torch.empty_like(T0)
        s.get_state(Ur, Tr)
        # host step, in place on pinned buffers
        Uh = U0.cpu().pin_memory()
        Th = T0.cpu().pin_memory() if warm else None
        To = torch.empty(case.cells, dtype=torch.float64).pin_memory()
        s.step_host(Uh, Th, Uh, To, dt, dgot[0:1])
        s.step_host(Uh, To, Uh, To, dt, dgot[1:2])
        torch.cuda.synchronize()
        assert s.status() == 0
        assert torch.equal(Uh, Ur.cpu()), name
        assert torch.equal(To, Tr.cpu()), name
        assert torch.equal(dgot, dref), name
    s.close()


def test_host_step_leaves_the_handle_as_the_three_calls_do():
    """After xf_step_rk3_host the handle holds U^{n+1} and its warm start, so
    a plain step can follow it: bitwise the same as three plain steps."""
    import torch
    case = cases.config(2, n=(128, 128, 128))
    s = gpu_solver(case)
    s.set_primitive(dev(case.prim))
    U0 = torch.empty((case.n_v, case.cells), dtype=torch.float64, device="cuda")
    T0 = torch.empty(case.cells, dtype=torch.float64, device="cuda")
    s.get_state(U0, T0)
    for _ in range(3):
        s.step(0.0)
    Ur = torch.empty_like(U0)
    s.get_state(Ur)
    Uh, Th = U0.cpu().pin_memory(), T0.cpu().pin_memory()
    s.step_host(Uh, Th, Uh, None)
    s.step(0.0)
    s.step(0.0)
    Ug = torch.empty_like(U0)
    s.get_state(Ug)
    torch.cuda.synchronize()
    assert s.status() == 0
    s.close()
    assert torch.equal(Ug, Ur)
