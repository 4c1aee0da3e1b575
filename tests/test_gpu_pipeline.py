"""af_step_host: pipelined steps of host-resident states.  Each result must equal
af_set_state + af_step + af_get_state on the same input bit for bit, chained
calls (an output fed back as the next input) must equal consecutive af_step
calls, and the resident state must be left alone."""
import numpy as np
import pytest

import af_inputs as ai

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2506_04857_gb300 as af  # noqa: E402


def solver(pb):
    return af.Solver(pb.nx, pb.ny, pb.gamma, pb.bc, domain=(pb.x0, pb.x1, pb.y0, pb.y1), cfl=pb.cfl,
                     kappa=pb.kappa)


def pinned(U):
    return [torch.from_numpy(np.ascontiguousarray(u)).pin_memory() for u in U]


def reference_step(s, U):
    """One af_step through the resident state; returns the result and the counters."""
    s.status(reset=True)
    s.set_state(U)
    s.step()
    out = s.get_state(device=False)
    rc, cnt = s.status(reset=True)
    assert rc == af.AF_OK
    return out, np.array([cnt[k] for k in af.STAT_NAMES], dtype=np.int64)


def inputs(pb, count):
    """count distinct admissible states: the initial data and the states after 1, 2, ... steps."""
    s = solver(pb)
    U = ai.dofs(pb)
    s.set_state(U)
    out = [U]
    for _ in range(count - 1):
        s.step()
        out.append(s.get_state(device=False))
    s.close()
    return out


@pytest.mark.parametrize("make", [lambda: ai.blast(48), lambda: ai.orszag_tang(40), lambda: ai.vortex(32)])
def test_independent_inputs_bitwise(make):
    pb = make()
    states = inputs(pb, 4)
    s = solver(pb)
    resident = ai.dofs(pb)
    s.set_state(resident)
    h_in = [pinned(U) for U in states]
    h_out = [[torch.empty_like(t).pin_memory() for t in U] for U in h_in]
    s.status(reset=True)
    for a, b in zip(h_in, h_out):
        s.step_host(a, b)
    s.sync()
    rc, cnt = s.status(reset=True)
    assert rc == af.AF_OK
    # the resident state is untouched
    for r, g in zip(resident, s.get_state(device=False)):
        assert np.array_equal(r, g)
    total = np.zeros(af.AF_NSTAT, dtype=np.int64)
    ref = solver(pb)
    for U, b in zip(states, h_out):
        want, c = reference_step(ref, U)
        total += c
        for w, g in zip(want, b):
            assert np.array_equal(w, g.numpy())
    assert np.array_equal(np.array([cnt[k] for k in af.STAT_NAMES], dtype=np.int64), total)


def test_chained_outputs_equal_consecutive_steps():
    pb = ai.blast(40)
    U0 = ai.dofs(pb)
    A, B = pinned(U0), [torch.empty_like(t).pin_memory() for t in pinned(U0)]
    s = solver(pb)
    bufs = [A, B]
    for k in range(5):   # A -> B -> A -> ... : every input is the previous call's output
        s.step_host(bufs[k % 2], bufs[(k + 1) % 2])
    s.sync()
    ref = solver(pb)
    ref.set_state(U0)
    for _ in range(5):
        ref.step()
    for w, g in zip(ref.get_state(device=False), bufs[1]):
        assert np.array_equal(w, g.numpy())


def test_pageable_arrays_and_argument_checks():
    pb = ai.orszag_tang(24)
    U0 = [np.ascontiguousarray(u) for u in ai.dofs(pb)]
    out = [np.empty_like(u) for u in U0]
    s = solver(pb)
    s.step_host(U0, out)
    s.sync()
    want, _ = reference_step(solver(pb), U0)
    for w, g in zip(want, out):
        assert np.array_equal(w, g)
    with pytest.raises(ValueError):   # a strided view would need a temporary copy
        s.step_host([u[:, :, ::1].T for u in U0], out)
    with pytest.raises(ValueError):
        s.step_host([u.astype(np.float32) for u in U0], out)
    s.set_state(U0)
    s.stage(0)
    with pytest.raises(af.AFError):   # in the middle of a step
        s.step_host(U0, out)
