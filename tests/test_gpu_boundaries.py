"""Reflective and inflow sides (af_set_boundary; Example 4.8) against the
oracle: limited stages on the oracle's stage inputs for the jets, chained
steps with the sensor off, the reflective half domain of a symmetric blast,
a uniform inflow state, and the jets at the paper's size."""
import numpy as np
import pytest

import af_inputs as ai
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2506_04857_gb300 as af  # noqa: E402

GROUPS = [(0,), (1, 2, 3), (1, 2, 3), (1, 2, 3), (4, 5, 6), (4, 5, 6), (4, 5, 6), (7,)]


def rel_err(A, B, pb=None):
    """max |a - b| / scale per class and variable.  The scale of a variable is
    the largest value of its group (rho, momentum, B, E) over all classes of b
    and, with inflow, of the inflow state: in the first stages of the jets the
    averages' momentum is rounding noise next to the jet's (the inflow enters
    the averages through strongly limited fluxes), so a per-class scale would
    compare noise with noise.  Zero fields of a zero group must match exactly."""
    scale = [0.0] * 8
    for k in range(8):
        for b in B:
            scale[k] = max([scale[k]] + [float(np.abs(b[q]).max()) for q in GROUPS[k]])
        if pb is not None and pb.inflow_U is not None:
            scale[k] = max([scale[k]] + [abs(pb.inflow_U[q]) for q in GROUPS[k]])
    worst = 0.0
    for a, b in zip(A, B):
        a = a.cpu().numpy() if hasattr(a, "cpu") else np.asarray(a)
        for k in range(8):
            num = np.abs(a[k] - b[k]).max()
            if scale[k] == 0.0:
                assert num <= 1e-300, (k, num)
                continue
            worst = max(worst, num / scale[k])
    return worst


def solver(pb, **kw):
    p = dict(cfl=pb.cfl, kappa=pb.kappa)
    p.update(kw)
    return af.Solver(pb.nx, pb.ny, pb.gamma, pb.bc, domain=(pb.x0, pb.x1, pb.y0, pb.y1),
                     sides=pb.sides, inflow=(pb.inflow_lo, pb.inflow_hi, pb.inflow_U), **p)


def blast_b2(nx, ny, x1):
    def prim(x, y):
        z = 0.0 * np.asarray(x, dtype=np.float64)
        r2 = x * x + y * y
        return (z + 1.0, z, z, z, z, z + 1.0, z, np.where(r2 < 0.13 ** 2, 10.0, 0.1) + z)
    sides = (0, ai.REFLECT, 0, 0) if x1 == 0.0 else (0, 0, 0, 0)
    return ai.Problem("blast_b2", nx, ny, -0.5, x1, -0.5, 0.5, ai.OUTFLOW, 5.0 / 3.0, prim, sides=sides)


@pytest.mark.parametrize("case", ["jets", "blast_reflect"])
def test_fe_stage_parity(case):
    pb = ai.jets(16) if case == "jets" else blast_b2(12, 20, 0.0)
    if case == "blast_reflect":
        pb.kappa = 1.0
    coef = [(0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0)]
    Un = ai.dofs(pb)
    inputs = []
    for _ in range(2):
        dt = oracle.dt(pb, Un)
        Us = Un
        for a, b in coef:
            inputs.append((Us, dt))
            Us = oracle.stage(pb, Un, Us, dt, a, b)
        Un = Us
    for Us, dt in inputs:
        st = np.zeros(oracle.NSTATS, dtype=np.int64)
        R = oracle.stage(pb, Us, Us, dt, 0.0, 1.0, stats=st)
        s = solver(pb)
        s.set_state(Us)
        s.stage(0, dt)
        G = s.get_stage(device=False)
        rc, cnt = s.status()
        assert rc == af.AF_OK, af.af_last_error(s.ctx)
        assert rel_err(G, R, pb) <= 1e-12, case
        for q, name in enumerate(oracle.STAT_NAMES):
            if name in ("center_limited", "point_limited", "sensor_lt099", "lambda_lt1", "src_limited",
                        "face_theta_lt1", "shrink", "nonadmissible", "newton_solves", "cell_shrink"):
                assert cnt[name] == st[q], (case, name, cnt[name], st[q])
        s.close()


@pytest.mark.parametrize("case", ["jets", "blast_reflect"])
def test_fe_stage_parity_with_interior_blocks(case):
    """Grids wide enough (>= 68 indices) that the thread blocks of the interior run
    the plain kernels and only the boundary frame resolves ghosts: limited stages
    on the oracle's stage inputs of one step, <= 1e-12 with equal counters."""
    pb = ai.jets(80) if case == "jets" else blast_b2(72, 80, 0.0)
    if case == "blast_reflect":
        pb.kappa = 1.0
    assert pb.nx >= 68 and pb.ny >= 12
    Un = ai.dofs(pb)
    dt = oracle.dt(pb, Un)
    Us = Un
    for a, b in [(0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0)]:
        st = np.zeros(oracle.NSTATS, dtype=np.int64)
        R = oracle.stage(pb, Us, Us, dt, 0.0, 1.0, stats=st)
        s = solver(pb)
        s.set_state(Us)
        s.stage(0, dt)
        G = s.get_stage(device=False)
        rc, cnt = s.status()
        assert rc == af.AF_OK, af.af_last_error(s.ctx)
        assert rel_err(G, R, pb) <= 1e-12, case
        for q, name in enumerate(oracle.STAT_NAMES):
            if name in ("center_limited", "point_limited", "sensor_lt099", "lambda_lt1", "src_limited",
                        "face_theta_lt1", "shrink", "nonadmissible", "newton_solves", "cell_shrink"):
                assert cnt[name] == st[q], (case, name, cnt[name], st[q])
        s.close()
        Us = oracle.stage(pb, Un, Us, dt, a, b)


@pytest.mark.parametrize("case", ["jets", "blast_reflect"])
def test_chained_steps_sensor_off(case):
    pb = ai.jets(16) if case == "jets" else blast_b2(12, 20, 0.0)
    pb.kappa = 0.0
    s = solver(pb)
    U = ai.dofs(pb)
    s.set_state(U)
    V = U
    for _ in range(3):
        s.step(dt_out=False)
        V, _ = oracle.step(pb, V)
    assert rel_err(s.get_state(), V, pb) <= 1e-12


def test_reflective_half_domain_matches_full_domain_on_gpu():
    m, ny = 12, 20
    full, half = blast_b2(2 * m, ny, 0.5), blast_b2(m, ny, 0.0)
    sf, sh = solver(full, kappa=0.0), solver(half, kappa=0.0)
    sf.set_state(ai.dofs(full))
    sh.set_state(ai.dofs(half))
    for _ in range(4):
        df, dh = sf.step(), sh.step()
        assert dh == pytest.approx(df, rel=1e-14)
    F, H = sf.get_state(device=False), sh.get_state(device=False)
    for c in range(4):
        cols = H[c].shape[2]
        a, b = H[c], F[c][:, :, :cols]
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), c


def test_uniform_inflow_state_and_adjoint_refusal():
    pb = ai.jets(8)
    jet_prim = (1.4, 0.0, 800.0, 0.0, 0.0, pb.prim(0.0, 0.0)[5], 0.0, 1.0)
    uni = ai.Problem("jet_state", 8, 24, pb.x0, pb.x1, pb.y0, pb.y1, ai.OUTFLOW, pb.gamma,
                     lambda x, y: tuple(0.0 * np.asarray(x) + v for v in jet_prim),
                     sides=pb.sides, inflow_lo=pb.inflow_lo, inflow_hi=pb.inflow_hi, inflow_U=pb.inflow_U)
    s = solver(uni)
    U0 = ai.dofs(uni)
    s.set_state(U0)
    for _ in range(5):
        s.step(dt_out=False)
    for a, b in zip(s.get_state(device=False), U0):
        for k in range(8):
            assert np.abs(a[k] - b[k]).max() <= 1e-12 * max(np.abs(b[k]).max(), 1.0)
    lam = [torch.ones(u.shape, dtype=torch.float64, device="cuda") for u in U0]
    with pytest.raises(af.AFError):
        af.af_rhs_vjp(s.ctx, lam)
    with pytest.raises(af.AFError):   # periodic grids have no sides
        p = af.Solver(8, 8, 1.4, af.AF_BC_PERIODIC)
        af.af_set_boundary(p.ctx, (0, 1, 0, 0))


def test_jets_paper_size():
    """Example 4.8 at the paper's resolution (200 x 600 cells, B_a = sqrt(20000),
    kappa = 2): runs to T = 0.002 admissible; the step count and the number of
    round-off shrinks are recorded (the paper reports 6607 steps and 8 shrinks
    for its run with 401 x 1201 DoFs; measured here: 7098 steps and about 1.4e4
    cell-average shrinks, the absolute 1e-13 pressure floor lying far below the
    rounding of the pressure at E ~ 4.5e5)."""
    pb = ai.jets(200)
    s = solver(pb)
    s.set_state(ai.dofs(pb))
    t, n = 0.0, 0
    dtt = torch.zeros(1, dtype=torch.float64, device="cuda")
    while t < pb.t_end and n < 20000:
        s.step(dtt)
        n += 1
        t += float(dtt.item())
    rc, cnt = s.status()
    assert rc == af.AF_OK, af.af_last_error(s.ctx)
    print("jets: steps %d, t %.6g, shrink %d (cell averages %d), point_limited %d, lambda_lt1 %d, nonadmissible %d"
          % (n, t, cnt["shrink"], cnt["cell_shrink"], cnt["point_limited"], cnt["lambda_lt1"], cnt["nonadmissible"]))
    assert cnt["nonadmissible"] == 0
    assert 3000 < n < 15000


def test_full_size_jets_sampled():
    """The benchmark's size and launch configuration (jets, 1024x3072, reflective
    at x = 0, inflow at the bottom): one limited stage of the whole grid on the
    GPU, checked on sampled 48x48 windows run by the oracle as sub-problems that
    keep the true sides they touch (cells within 4 of an artificial window edge
    are not compared)."""
    import dataclasses
    pb = ai.jets(1024)
    nx, ny, w, pad = pb.nx, pb.ny, 48, 4
    U = ai.dofs(pb)
    dt = oracle.dt(pb, U)
    s = solver(pb)
    s.set_state(U)
    s.stage(0, dt)
    G = s.get_stage(device=False)
    rc, cnt = s.status()
    assert rc == af.AF_OK, af.af_last_error(s.ctx)
    edge = int(round((pb.inflow_lo - pb.x0) / pb.dx))   # column of the jet's edge x = inflow_lo
    starts = [(nx - w, 0), (edge - w // 2, 0), (0, 0), (nx - w, ny - w), (500, 1500), (nx - w, 1500)]
    ext = [(w, w), (w + 1, w), (w, w + 1), (w + 1, w + 1)]
    for i0, j0 in starts:
        sides = (pb.sides[0] if i0 == 0 else 0, pb.sides[1] if i0 + w == nx else 0,
                 pb.sides[2] if j0 == 0 else 0, pb.sides[3] if j0 + w == ny else 0)
        sub = dataclasses.replace(pb, nx=w, ny=w, x0=pb.x0 + i0 * pb.dx, x1=pb.x0 + (i0 + w) * pb.dx,
                                  y0=pb.y0 + j0 * pb.dy, y1=pb.y0 + (j0 + w) * pb.dy, sides=sides)
        V = [np.ascontiguousarray(U[c][:, j0:j0 + e[1], i0:i0 + e[0]]) for c, e in enumerate(ext)]
        R = oracle.stage(sub, V, V, dt, 0.0, 1.0)
        lo_i, hi_i = (0 if i0 == 0 else pad), (w if i0 + w == nx else w - pad)
        lo_j, hi_j = (0 if j0 == 0 else pad), (w if j0 + w == ny else w - pad)
        A, B = [], []
        for c in range(4):
            ex, ey = (1 if c in (1, 3) else 0), (1 if c in (2, 3) else 0)
            hic, hjc = hi_i + (ex if hi_i == w else 0), hi_j + (ey if hi_j == w else 0)
            A.append(G[c][:, j0 + lo_j:j0 + hjc, i0 + lo_i:i0 + hic])
            B.append(R[c][:, lo_j:hjc, lo_i:hic])
        assert rel_err(A, B, pb) <= 1e-12, (i0, j0)


def test_upwind_source_with_reflective_and_inflow_sides():
    """The velocity-upwind point source (Example 4.2 variant) on a grid with
    reflective and inflow sides (the ghost-aware point kernel with the upwind
    option), wide enough for interior blocks too: limited stages on the
    oracle's stage inputs of one step, <= 1e-12 with equal counters."""
    pb = ai.jets(80)
    Un = ai.dofs(pb)
    dt = oracle.dt(pb, Un, src_point_upwind=True)
    Us = Un
    for a, b in [(0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0)]:
        st = np.zeros(oracle.NSTATS, dtype=np.int64)
        R = oracle.stage(pb, Us, Us, dt, 0.0, 1.0, stats=st, src_point_upwind=True)
        s = solver(pb, src_point_upwind=True)
        s.set_state(Us)
        s.stage(0, dt)
        G = s.get_stage(device=False)
        rc, cnt = s.status()
        assert rc == af.AF_OK, af.af_last_error(s.ctx)
        assert rel_err(G, R, pb) <= 1e-12
        for q, name in enumerate(oracle.STAT_NAMES):
            if name in ("center_limited", "point_limited", "sensor_lt099", "lambda_lt1", "shrink", "nonadmissible"):
                assert cnt[name] == st[q], (name, cnt[name], st[q])
        s.close()
        Us = oracle.stage(pb, Un, Us, dt, a, b, src_point_upwind=True)
