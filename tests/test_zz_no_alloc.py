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


# (OUTFLOW, 64, 64) and (PERIODIC, 65, 65) use exactly AF_NOALLOC_MAX_POINTS = 65 x 65 work points
@pytest.mark.parametrize("bc,nx,ny", [(ai.PERIODIC, 64, 64), (ai.OUTFLOW, 64, 64), (ai.PERIODIC, 65, 65),
                                      (ai.OUTFLOW, 40, 23), (ai.PERIODIC, 17, 9)])
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


@pytest.mark.parametrize("bc,nx,ny", [(ai.PERIODIC, 80, 80), (ai.OUTFLOW, 65, 64), (ai.PERIODIC, 66, 65)])
def test_rhs_noalloc_rejects_grids_beyond_the_scratch(bc, nx, ny):
    # 6400, and one row or column past the limit: 66 x 65 = 4290 > AF_NOALLOC_MAX_POINTS work points
    pb = ai.random_smooth(nx, ny, seed=1, bc=bc)
    U = [torch.from_numpy(u).cuda() for u in ai.dofs(pb)]
    out = [torch.empty_like(u) for u in U]
    with pytest.raises(af.AFError) as e:
        af.af_rhs_noalloc(nx, ny, pb.gamma, pb.bc, (0.0, 1.0, 0.0, 1.0), U, out)
    assert e.value.code == af.AF_EBOUNDS


def test_rhs_noalloc_rejects_bad_buffers():
    nx, ny = 12, 10
    pb = ai.random_smooth(nx, ny, seed=2, bc=ai.OUTFLOW)
    U = [torch.from_numpy(u).cuda() for u in ai.dofs(pb)]
    dom = (0.0, 1.0, 0.0, 1.0)
    good = [torch.empty_like(u) for u in U]
    strided = torch.empty(8, nx + 1, ny, device="cuda", dtype=torch.float64).transpose(1, 2)
    bad_cases = [
        [good[0], good[1], good[2], good[3][:, :-1]],    # wrong extent
        [good[0].float(), good[1], good[2], good[3]],    # float32
        [good[0], strided, good[2], good[3]],            # right shape, not contiguous
        [good[0].cpu(), good[1], good[2], good[3]],      # host tensor
        [U[0], good[1], good[2], good[3]],               # output aliases an input
    ]
    for out in bad_cases:
        with pytest.raises(ValueError):
            af.af_rhs_noalloc(nx, ny, pb.gamma, pb.bc, dom, U, out)
    # the C entry point itself refuses an output that overlaps an input
    lib = af._lib()
    ins = af._ptr_array([u.data_ptr() for u in U])
    outs = af._ptr_array([good[0].data_ptr(), good[1].data_ptr(), U[2].data_ptr(), good[3].data_ptr()])
    rc = lib.af_rhs_noalloc(nx, ny, pb.gamma, pb.bc, *dom, ins, outs, None)
    assert rc == af.AF_EINVAL
