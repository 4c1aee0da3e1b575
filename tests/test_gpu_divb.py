"""The discrete divergence measures of Example 4.4 (af_divb) against the oracle
and against closed forms, on seeded states and after steps of the scheme."""
import numpy as np
import pytest

import af_inputs as ai
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2506_04857_gb300 as af  # noqa: E402


def solver(pb, **kw):
    return af.Solver(pb.nx, pb.ny, pb.gamma, pb.bc, domain=(pb.x0, pb.x1, pb.y0, pb.y1), cfl=pb.cfl,
                     kappa=pb.kappa, **kw)


def tol(pb, U):
    """Absolute tolerance of a measure: the node divergences are differences of
    B values over h, so rounding enters at about eps |B| / h per node."""
    bmax = max(float(np.abs(u[4:6]).max()) for u in U)
    return 1e-14 * (pb.x1 - pb.x0) * (pb.y1 - pb.y0) * bmax / min(pb.dx, pb.dy)


def b_field(B1, B2, nx=12, ny=10, box=(1.0, 2.0, 0.0, 1.0)):
    def prim(x, y):
        z = np.zeros(np.shape(x))
        return (z + 1.0, z, z, z, B1(x, y) + z, B2(x, y) + z, z, z + 1.0)
    return ai.Problem("bfield", nx, ny, box[0], box[1], box[2], box[3], ai.OUTFLOW, 5.0 / 3.0, prim)


@pytest.mark.parametrize("case,expect", [
    ((lambda x, y: x * x, lambda x, y: 0 * x, 12, 10, (1.0, 2.0, 0.0, 1.0)), (3.0, 3.0)),
    ((lambda x, y: 0 * x, lambda x, y: y * y, 9, 14, (0.0, 1.0, 1.0, 3.0)), (8.0, 8.0)),
    ((lambda x, y: (x - 1.5) ** 2, lambda x, y: 0 * x, 12, 10, (1.0, 2.0, 0.0, 1.0)), (0.5, 0.5)),
])
def test_closed_forms(case, expect):
    B1, B2, nx, ny, box = case
    pb = b_field(B1, B2, nx, ny, box)
    s = solver(pb)
    s.set_state(ai.dofs(pb))
    d1, d2 = s.divb()
    assert d1 == pytest.approx(expect[0], rel=1e-12)
    assert d2 == pytest.approx(expect[1], rel=1e-12)


def test_divergence_free_q2_field():
    pb = b_field(lambda x, y: 2 * x * x * y, lambda x, y: -2 * x * y * y)
    s = solver(pb)
    s.set_state(ai.dofs(pb))
    d1, d2 = s.divb()
    assert d1 <= 1e-12 and d2 <= 1e-12


@pytest.mark.parametrize("pb", [ai.random_smooth(16, 12, seed=3), ai.random_smooth(37, 29, seed=4, bc=ai.OUTFLOW),
                                ai.random_smooth(40, 33, seed=5, divfree=True), ai.orszag_tang(48)],
                         ids=["periodic", "outflow-ragged", "divfree", "orszag-tang"])
def test_matches_oracle(pb):
    s = solver(pb)
    U = ai.dofs(pb)
    s.set_state(U)
    got = s.divb()
    ref = oracle.divb(pb, U)
    for a, b in zip(got, ref):
        assert a == pytest.approx(b, rel=1e-12, abs=tol(pb, U))
    # fixed summation order: bitwise repeatable; device output path
    assert s.divb() == got
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    s.divb(out)
    torch.cuda.synchronize()
    assert tuple(out.tolist()) == got


def test_after_steps_on_common_states():
    """Orszag-Tang 128x128 and the blast 96x96 after 5 steps of the oracle: the
    measures of that state, by the GPU and by the oracle."""
    for pb in (ai.orszag_tang(128), ai.blast(96)):
        V = ai.dofs(pb)
        for _ in range(5):
            V, _ = oracle.step(pb, V)
        s = solver(pb)
        s.set_state(V)
        got = s.divb()
        ref = oracle.divb(pb, V)
        for a, b in zip(got, ref):
            assert a == pytest.approx(b, rel=1e-12, abs=tol(pb, V))


def test_full_size_orszag_tang_512():
    pb = ai.orszag_tang(512)
    V, _ = oracle.step(pb, ai.dofs(pb))
    s = solver(pb)
    s.set_state(V)
    got = s.divb()
    ref = oracle.divb(pb, V)
    for a, b in zip(got, ref):
        assert a == pytest.approx(b, rel=1e-12, abs=tol(pb, V))


def test_full_size_2048_outflow():
    """The size and launch configuration of the divergence benchmark (2048x2048,
    outflow): a smooth field with div B != 0, GPU against the oracle over the
    whole grid."""
    tp = 2.0 * np.pi
    pb = b_field(lambda x, y: 0.3 * np.sin(tp * x) * np.cos(tp * y) + x * x,
                 lambda x, y: 0.2 * np.cos(3 * tp * x) - y * x, 2048, 2048, (0.0, 1.0, 0.0, 1.0))
    U = ai.dofs(pb)
    s = solver(pb)
    s.set_state(U)
    got = s.divb()
    ref = oracle.divb(pb, U)
    assert ref[0] > 0.5 and ref[1] > 0.5
    for a, b in zip(got, ref):
        assert a == pytest.approx(b, rel=1e-12, abs=tol(pb, U))
