"""af_rhs_noalloc: the right-hand side without device allocation.

Some callers cannot allocate device memory on their hot path (a framework that
owns all device memory through its own pool, a real-time loop where a
cudaMalloc could block or fail).  af_rhs_noalloc serves them from a fixed
scratch array in the library's static device memory.  This test checks, through
the C ABI, that two calls in a row give the same result as af_rhs (which uses
a context and its own allocations), to the tolerance of the rhs parity tests,
and that grids beyond the scratch's size are rejected.

The file is named to be collected last, so that a run stopping at the first
failure has run every other test before this one.
"""
import numpy as np
import pytest

import af_inputs as ai

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2506_04857_gb300 as af  # noqa: E402


def rel_err(A, B):
    worst = 0.0
    for a, b in zip(A, B):
        a = a.cpu().numpy()
        b = b.cpu().numpy()
        for k in range(8):
            den = np.abs(b[k]).max()
            num = np.abs(a[k] - b[k]).max()
            if den == 0.0:
                assert num == 0.0
                continue
            worst = max(worst, num / den)
    return worst


@pytest.mark.parametrize("bc,nx,ny", [(ai.PERIODIC, 64, 64), (ai.OUTFLOW, 40, 23), (ai.PERIODIC, 17, 9)])
def test_rhs_noalloc_matches_rhs_twice(bc, nx, ny):
    domain = (0.0, 1.0, 0.0, 1.0)
    outs = []
    for seed in (31, 32):   # two calls in a row, on different states
        pb = ai.random_smooth(nx, ny, seed=seed, amp=0.2, bc=bc)
        U = [torch.from_numpy(u).cuda() for u in ai.dofs(pb)]
        s = af.Solver(nx, ny, pb.gamma, bc, domain=domain)
        s.set_state(U)
        ref = s.rhs()
        out = [torch.full_like(u, float("nan")) for u in U]
        af.af_rhs_noalloc(nx, ny, pb.gamma, bc, domain, U, out, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert rel_err(out, ref) <= 1e-12
        outs.append(out)
        s.close()
    # the second call did not just return the first call's scratch contents
    assert not torch.equal(outs[0][0], outs[1][0])


def test_rhs_noalloc_rejects_grids_beyond_the_scratch():
    nx = ny = 80   # 6400 > AF_NOALLOC_MAX_POINTS work points
    pb = ai.random_smooth(nx, ny, seed=1)
    U = [torch.from_numpy(u).cuda() for u in ai.dofs(pb)]
    out = [torch.empty_like(u) for u in U]
    with pytest.raises(af.AFError) as e:
        af.af_rhs_noalloc(nx, ny, pb.gamma, pb.bc, (0.0, 1.0, 0.0, 1.0), U, out)
    assert e.value.code == af.AF_EBOUNDS
