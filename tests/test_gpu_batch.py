"""Batched ensembles (af_batch_*): many independent runs of uneven sizes in one
persistent launch per pass.  Each run must equal -- bitwise -- the same run
stepped alone through an af_ctx, with and without the CUDA graph and after
autotuning, and one member is checked against the oracle."""
import numpy as np
import pytest

import af_inputs as ai
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2506_04857_gb300 as af  # noqa: E402


def members():
    pbs = [ai.orszag_tang(16, 24), ai.orszag_tang(33, 17, amp_v=1.1, phase_x=0.7), ai.blast(20),
           ai.vortex(24), ai.random_smooth(18, 12, seed=3, amp=0.2, bc=ai.OUTFLOW), ai.sine_wave(16),
           ai.rotor(20)]
    pbs[3].kappa = 0.0
    pbs[4].kappa = 1.0
    return pbs


def make_batch(pbs, stream, upwind=()):
    b = af.af_batch_create([p.nx for p in pbs], [p.ny for p in pbs], [p.gamma for p in pbs], [p.bc for p in pbs])
    af.af_batch_set_stream(b, stream)
    for r, p in enumerate(pbs):
        af.af_batch_set_domain(b, r, p.x0, p.x1, p.y0, p.y1)
        af.af_batch_set_params(b, r, cfl=p.cfl, kappa=p.kappa, pp_on=(r != 5), src_point_upwind=(r in upwind))
        af.af_batch_set_state(b, r, [torch.from_numpy(u).cuda() for u in ai.dofs(p)])
    return b


def singles(pbs, nsteps, stream, upwind=()):
    out = []
    for r, p in enumerate(pbs):
        s = af.Solver(p.nx, p.ny, p.gamma, p.bc, domain=(p.x0, p.x1, p.y0, p.y1), cfl=p.cfl, kappa=p.kappa,
                      pp_on=(r != 5), stream=stream, src_point_upwind=(r in upwind))
        s.set_state(ai.dofs(p))
        for _ in range(nsteps):
            s.step(dt_out=False)
        out.append(s.get_state())
        s.close()
    return out


def batch_state(b, r, p):
    shapes = [(8, e[1], e[0]) for e in ai.class_extents(p.nx, p.ny, p.bc)]
    return af.af_batch_get_state(b, r, [torch.empty(s, dtype=torch.float64, device="cuda") for s in shapes])


@pytest.mark.parametrize("graph", [False, True])
def test_batch_equals_single_runs(graph):
    stream = torch.cuda.Stream()
    pbs = members()
    with torch.cuda.stream(stream):
        b = make_batch(pbs, stream)
        if graph:
            af.af_batch_graph(b, True)
        af.af_batch_step(b, 7)          # with the graph: two 3-step cycles + one direct step
        ref = singles(pbs, 7, stream)
        torch.cuda.synchronize()
        for r, p in enumerate(pbs):
            got = batch_state(b, r, p)
            for x, y in zip(got, ref[r]):
                assert torch.equal(x, y), (r, p.name)
        rc, cnt = af.af_batch_status(b)
        assert rc == af.AF_OK, af.af_batch_last_error(b)
        af.af_batch_destroy(b)


def test_batch_with_upwind_runs():
    """Runs with the velocity-upwind point source (Example 4.2 variant) next to
    central ones: the batch selects the point kernel that evaluates the flag per run."""
    stream = torch.cuda.Stream()
    pbs = members()
    up = (1, 3, 4)
    with torch.cuda.stream(stream):
        b = make_batch(pbs, stream, upwind=up)
        af.af_batch_step(b, 4)
        ref = singles(pbs, 4, stream, upwind=up)
        plain = singles(pbs, 4, stream)
        torch.cuda.synchronize()
        for r, p in enumerate(pbs):
            got = batch_state(b, r, p)
            for x, y in zip(got, ref[r]):
                assert torch.equal(x, y), (r, p.name)
        assert not all(torch.equal(x, y) for x, y in zip(ref[4], plain[4]))
        rc, cnt = af.af_batch_status(b)
        assert rc == af.AF_OK, af.af_batch_last_error(b)
        af.af_batch_destroy(b)


def test_autotune_keeps_results_and_state():
    stream = torch.cuda.Stream()
    pbs = members()
    with torch.cuda.stream(stream):
        b = make_batch(pbs, stream)
        before = [batch_state(b, r, p) for r, p in enumerate(pbs)]
        choice = af.af_batch_autotune(b, reps=1)
        assert choice["tile"][0] * choice["tile"][1] in (128, 256)
        after = [batch_state(b, r, p) for r, p in enumerate(pbs)]
        for x, y in zip(before, after):   # the autotuner does not advance the state
            for u, v in zip(x, y):
                assert torch.equal(u, v)
        af.af_batch_graph(b, True)
        af.af_batch_step(b, 3)
        ref = singles(pbs, 3, stream)
        torch.cuda.synchronize()
        for r, p in enumerate(pbs):
            for x, y in zip(batch_state(b, r, p), ref[r]):
                assert torch.equal(x, y), (r, p.name, choice)
        af.af_batch_destroy(b)


def test_batch_member_matches_oracle():
    stream = torch.cuda.Stream()
    pbs = members()
    with torch.cuda.stream(stream):
        b = make_batch(pbs, stream)
        af.af_batch_step(b, 2)
        torch.cuda.synchronize()
        for r in (3, 5):    # smooth members (vortex with kappa 0; sine with PP off)
            p = pbs[r]
            V = ai.dofs(p)
            for _ in range(2):
                V, _ = oracle.step(p, V, pp_on=(r != 5))
            G = batch_state(b, r, p)
            for a, bb in zip(G, V):
                a = a.cpu().numpy()
                for k in range(8):
                    den = np.abs(bb[k]).max()
                    if den > 0:
                        assert np.abs(a[k] - bb[k]).max() / den <= 1e-12
        af.af_batch_destroy(b)
