"""Parity of the 1D scheme (af1d_*) with the 1D oracle: smooth chained steps,
limited forward-Euler stages on the oracle's stage inputs (Riemann problems of
Example 4.1 with their sensor strengths, a strong blast), chained steps with
the sensor off, the paper's grid sizes, and the stage-order contract."""
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


def rel_err(A, B):
    """max |a - b| / max |b| per class and variable, a momentum or B component
    against the largest component of its vector; zero fields must match exactly."""
    worst = 0.0
    for a, b in zip(A, B):
        a = a.cpu().numpy() if hasattr(a, "cpu") else np.asarray(a)
        for k in range(8):
            num = np.abs(a[k] - b[k]).max()
            if np.abs(b[k]).max() == 0.0:
                assert num <= 1e-300, (k, num)
                continue
            worst = max(worst, num / max(np.abs(b[q]).max() for q in GROUPS[k]))
    return worst


def solver(pb, **kw):
    p = dict(cfl=pb.cfl, kappa=pb.kappa)
    p.update(kw)
    return af.Solver1D(pb.n, pb.gamma, pb.bc, domain=(pb.x0, pb.x1), **p)


def okw(kw):
    return {k: v for k, v in kw.items() if k in ("kappa", "pp_on", "cfl")}


@pytest.mark.parametrize("kappa,pp_on", [(0.0, True), (1.0, True), (0.0, False)])
def test_smooth_chained_steps(kappa, pp_on):
    pb = ai.entropy_wave1d(48, amp=0.3)
    pb.kappa = kappa
    s = solver(pb, pp_on=pp_on)
    U = ai.dofs1(pb)
    s.set_state([torch.from_numpy(u).cuda() for u in U])
    V = U
    for n in range(5):
        dg = s.step()
        V, dr = oracle.step1(pb, V, pp_on=pp_on)
        assert dg == pytest.approx(dr, rel=1e-14)
    assert rel_err(s.get_state(), V) <= 1e-12
    rc, _ = s.status()
    assert rc == af.AF_OK


def test_hundred_smooth_steps_outflow():
    pb = ai.entropy_wave1d(40)
    pb.bc = ai.OUTFLOW
    U = ai.dofs1(pb)
    s = solver(pb)
    s.set_state(U)
    V = U
    for _ in range(100):
        s.step(dt_out=False)
        V, _ = oracle.step1(pb, V)
    assert rel_err(s.get_state(), V) <= 1e-10


CASES = {"riemann_rj": lambda: ai.riemann_rj(120), "riemann_2": lambda: ai.riemann_2(120),
         "blast1d": lambda: ai.blast1d(96), "blast1d_periodic": lambda: ai.blast1d(64)}


@pytest.mark.parametrize("case", sorted(CASES))
def test_fe_stage_parity_limited(case):
    """Every stage input of three oracle steps fed to both sides; one limited
    forward-Euler stage compared, with equal limiter counters."""
    pb = CASES[case]()
    if case == "blast1d_periodic":
        pb.bc = ai.PERIODIC
    coef = [(0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0)]
    Un = ai.dofs1(pb)
    inputs = []
    for _ in range(3):
        dt = oracle.dt1(pb, Un)
        Us = Un
        for a, b in coef:
            inputs.append((Us, dt))
            Us = oracle.stage1(pb, Un, Us, dt, a, b)
        Un = Us
    active = 0
    for Us, dt in inputs:
        st = np.zeros(oracle.NSTATS, dtype=np.int64)
        R = oracle.stage1(pb, Us, Us, dt, 0.0, 1.0, stats=st)
        s = solver(pb)
        s.set_state(Us)
        s.stage(0, dt)
        G = s.get_stage()
        rc, cnt = s.status()
        assert rc == af.AF_OK, af.af1d_last_error(s.ctx)
        assert rel_err(G, R) <= 1e-12, case
        for q, name in enumerate(oracle.STAT_NAMES):
            if name in ("center_limited", "point_limited", "sensor_lt099", "lambda_lt1", "face_theta_lt1", "shrink",
                        "nonadmissible", "newton_solves"):
                assert cnt[name] == st[q], (case, name, cnt[name], st[q])
        active += int(st[oracle.STAT_NAMES.index("point_limited")] + st[oracle.STAT_NAMES.index("sensor_lt099")])
        s.close()
    assert active > 0


@pytest.mark.parametrize("case", ["riemann_rj", "riemann_2", "blast1d"])
def test_chained_steps_sensor_off(case):
    """With kappa = 0 only the PP limiters branch; chained steps agree."""
    pb = CASES[case]()
    pb.kappa = 0.0
    s = solver(pb)
    U = ai.dofs1(pb)
    s.set_state(U)
    V = U
    st = np.zeros(oracle.NSTATS, dtype=np.int64)
    for _ in range(4):
        s.step(dt_out=False)
        V, _ = oracle.step1(pb, V, stats=st)
    assert rel_err(s.get_state(), V) <= 1e-12
    rc, cnt = s.status()
    assert rc == af.AF_OK
    for name in ("point_limited", "center_limited", "lambda_lt1", "shrink", "nonadmissible"):
        assert cnt[name] == st[oracle.STAT_NAMES.index(name)], name


@pytest.mark.parametrize("pb", [ai.riemann_rj(800), ai.riemann_2(800), ai.blast1d(2000)],
                         ids=["riemann_rj_800", "riemann_2_800", "blast1d_2000"])
def test_paper_sizes(pb):
    """The grid sizes of Examples 4.1-4.2 (800 cells; 2000 for the strong
    problem): one limited stage from the oracle's state after two steps, and
    50 GPU steps stay admissible."""
    U = ai.dofs1(pb)
    for _ in range(2):
        U, _ = oracle.step1(pb, U)
    dt = oracle.dt1(pb, U)
    st = np.zeros(oracle.NSTATS, dtype=np.int64)
    R = oracle.stage1(pb, U, U, dt, 0.0, 1.0, stats=st)
    s = solver(pb)
    s.set_state(U)
    s.stage(0, dt)
    assert rel_err(s.get_stage(), R) <= 1e-12
    s.set_state(U)
    for _ in range(50):
        s.step(dt_out=False)
    rc, cnt = s.status()
    assert rc == af.AF_OK, af.af1d_last_error(s.ctx)
    A, P = s.get_state(device=False)
    for a in (A, P):
        rho = a[0]
        p = (pb.gamma - 1.0) * (a[7] - 0.5 * (a[1] ** 2 + a[2] ** 2 + a[3] ** 2) / rho - 0.5 * (a[4] ** 2 + a[5] ** 2 + a[6] ** 2))
        assert rho.min() > 0 and p.min() > 0


def test_stage_order_and_host_buffers():
    pb = ai.entropy_wave1d(16)
    s = solver(pb)
    U = ai.dofs1(pb)
    s.set_state(U)
    with pytest.raises(af.AFError):
        s.stage(1, 1e-3)
    dt = oracle.dt1(pb, U)
    assert s.dt() == pytest.approx(dt, rel=1e-14)
    for k in range(3):
        s.stage(k, dt)
    A, P = s.get_state(device=False)
    V, _ = oracle.step1(pb, U, dt_in=dt)
    assert rel_err([A, P], V) <= 1e-12


def test_1d_reduction_of_the_2d_path():
    """On the GPU: one stage of the 2D path on y-invariant data whose y-face
    values are the 1D parabola centres equals one stage of the 1D path (the
    x-faces and averages; smooth data, sensor on)."""
    n, ny = 24, 4
    p1 = ai.entropy_wave1d(n, amp=0.3)
    p1.kappa = 1.0
    A1, P1 = ai.dofs1(p1)
    A = np.repeat(A1[:, None, :], ny, axis=1)
    X = np.repeat(P1[:, None, :], ny, axis=1)
    Y = np.repeat(((6.0 * A1 - P1 - np.roll(P1, -1, axis=1)) / 4.0)[:, None, :], ny, axis=1)
    U2 = [np.ascontiguousarray(a) for a in (A, X, Y, X.copy())]
    s1 = solver(p1)
    s1.set_state([A1, P1])
    dt = s1.dt()
    s1.set_state([A1, P1])
    s1.stage(0, dt)
    G1 = s1.get_stage(device=False)
    s2 = af.Solver(n, ny, p1.gamma, af.AF_BC_PERIODIC, domain=(0.0, 1.0, 0.0, 0.25), kappa=1.0)
    s2.set_state(U2)
    s2.stage(0, dt)
    G2 = s2.get_stage(device=False)
    for j in range(ny):
        for c in (0, 1):
            for k in range(8):
                ref = G1[c][k]
                assert np.abs(G2[c][k, j] - ref).max() <= 1e-13 * max(np.abs(ref).max(), 1.0), (c, j, k)


def test_kernel_timing_counts_every_launch():
    """af1d_timing brackets every launch of the 1D stages: over two steps with the
    positivity limiters on, each pass runs 6 times, the dt pass twice, and the
    timed steps give the same state as untimed ones."""
    pb = ai.blast1d(400)
    U = ai.dofs1(pb)
    s, r = solver(pb), solver(pb)
    s.set_state(U)
    r.set_state(U)
    s.timing(True)
    for _ in range(2):
        s.step(dt_out=False)
        r.step(dt_out=False)
    t = s.timing(False)
    for k in ("k1_pointdata", "k1_points", "k1_faces", "k1_cells", "k1_final", "k1_repair"):
        assert t[k][1] == 6 and t[k][0] > 0.0, (k, t[k])
    assert t["k_dt"][1] == 2
    for a, b in zip(s.get_state(), r.get_state()):
        assert torch.equal(a, b)
    assert s.timing(False)["k1_points"][1] == 0   # the record is cleared


def test_full_size_blast1d_sampled():
    """The benchmark's size and launch configuration (strong blast, 4,194,304
    cells, outflow): one limited stage of the whole grid on the GPU, checked on
    sampled 1024-cell windows that the oracle runs as outflow sub-problems
    (cells and points within 4 of an artificial window edge are not compared;
    the stage's dependence radius is 3)."""
    import dataclasses
    pb = ai.blast1d(1 << 22)
    n, w, pad = pb.n, 1024, 4
    U = ai.dofs1(pb)
    dt = oracle.dt1(pb, U)
    s = solver(pb)
    s.set_state(U)
    s.stage(0, dt)
    A, P = s.get_stage(device=False)
    rc, cnt = s.status()
    assert rc == af.AF_OK and cnt["nonadmissible"] == 0
    front = int(0.4 * n)   # x = -0.1
    starts = [0, n - w, front - w // 2, n - front - w // 2, n // 2 - w // 2, n // 5]
    windows = []
    for i0 in starts:
        sub = dataclasses.replace(pb, n=w, x0=pb.x0 + i0 * pb.dx, x1=pb.x0 + (i0 + w) * pb.dx)
        V = [np.ascontiguousarray(U[0][:, i0:i0 + w]), np.ascontiguousarray(U[1][:, i0:i0 + w + 1])]
        windows.append((i0, oracle.stage1(sub, V, V, dt, 0.0, 1.0)))
    scale = [[max(np.abs(R[c][k]).max() for _, R in windows) for k in range(8)] for c in range(2)]
    for i0, R in windows:
        lo = 0 if i0 == 0 else pad
        hi = w if i0 + w == n else w - pad
        for c, G in enumerate((A, P)):
            hc = hi + (1 if (c == 1 and hi == w) else 0)
            a, b = G[:, i0 + lo:i0 + hc], R[c][:, lo:hc]
            for k in range(8):
                if scale[c][k] == 0:
                    assert np.abs(a[k]).max() == 0
                    continue
                assert np.abs(a[k] - b[k]).max() / scale[c][k] <= 1e-12, (i0, c, k)
