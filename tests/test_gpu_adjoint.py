"""Discrete adjoint (af_rhs_vjp, af_adjoint_step, AFSteps).

- dot-product test of the transposed semi-discrete operator against central
  differences of af_rhs, class by class, periodic and outflow;
- one adjoint step against central differences of one step (dt fixed);
- the gradient of the magnetic energy after several steps against a
  complex-step derivative of the CPU oracle (smooth perturbed vortex,
  kappa = 0, limiters inactive);
- the adjoint workload at full size: 256x256 perturbed vortex, 200 steps,
  checkpoints every 20 steps, 32 seeded directions, central differences.
"""
import math

import numpy as np
import pytest

import af_inputs as ai
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2506_04857_gb300 as af  # noqa: E402
from paper_2506_04857_gb300.adjoint import af_steps, magnetic_energy  # noqa: E402


def solver_for(pb, **kw):
    p = dict(cfl=pb.cfl, kappa=0.0)
    p.update(kw)
    return af.Solver(pb.nx, pb.ny, pb.gamma, pb.bc, domain=(pb.x0, pb.x1, pb.y0, pb.y1), **p)


def cuda_state(U):
    return [torch.from_numpy(np.ascontiguousarray(u)).cuda() for u in U]


def dot(a, b):
    return sum(float((x * y).sum()) for x, y in zip(a, b))


def rand_like(U, gen, scale=1.0, only=None):
    out = []
    for c, u in enumerate(U):
        r = torch.randn(u.shape, generator=gen, dtype=torch.float64).cuda() * scale
        if only is not None and c != only:
            r.zero_()
        out.append(r)
    return out


def flat(U):
    return torch.cat([u.reshape(-1) for u in U])


def unflat(x, shapes):
    out, o = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append(x[o:o + n].reshape(s).contiguous())
        o += n
    return out


def step_fixed_dt(s, U, dt):
    s.set_state(U)
    for k in range(3):
        s.stage(k, dt)
    return s.get_state()


def full_jacobians(s, U, forward, transpose_row, eps=1e-6):
    """(J by central differences column by column, J by the transpose row by row)."""
    shapes = [tuple(u.shape) for u in U]
    x0 = flat(U)
    n = x0.numel()
    Jfd = torch.zeros(n, n, dtype=torch.float64, device="cuda")
    for k in range(n):
        xp, xm = x0.clone(), x0.clone()
        xp[k] += eps
        xm[k] -= eps
        Jfd[:, k] = (flat(forward(unflat(xp, shapes))) - flat(forward(unflat(xm, shapes)))) / (2 * eps)
    Jad = torch.zeros(n, n, dtype=torch.float64, device="cuda")
    for k in range(n):
        e = torch.zeros(n, dtype=torch.float64, device="cuda")
        e[k] = 1.0
        Jad[k, :] = flat(transpose_row(unflat(e, shapes)))
    return Jfd, Jad


# Tiny grids: the 5-point stencils wrap onto themselves (periodic 4x5) or reach
# the mirrored boundary from both sides (outflow); every entry of the Jacobian
# is compared.  Central differences with eps = 1e-6 carry O(eps^2) truncation
# and O(1e-16/eps) rounding error: about 1e-10 of the largest entry.
TINY = [(ai.PERIODIC, 4, 5), (ai.OUTFLOW, 5, 4), (ai.OUTFLOW, 7, 6)]


@pytest.mark.parametrize("bc,nx,ny", TINY)
def test_vjp_full_jacobian(bc, nx, ny):
    pb = ai.random_smooth(nx, ny, seed=41, amp=0.2, bc=bc)
    U = cuda_state(ai.dofs(pb))
    s = solver_for(pb)

    def fwd(V):
        s.set_state(V)
        return s.rhs()

    def row(e):
        s.set_state(U)
        return af.af_rhs_vjp(s.ctx, e)

    Jfd, Jad = full_jacobians(s, U, fwd, row)
    scale = Jfd.abs().max().item()
    assert (Jad - Jfd).abs().max().item() <= 1e-8 * scale


@pytest.mark.parametrize("bc,nx,ny", TINY[:2])
def test_adjoint_step_full_jacobian(bc, nx, ny):
    pb = ai.random_smooth(nx, ny, seed=41, amp=0.2, bc=bc)
    U = cuda_state(ai.dofs(pb))
    s = solver_for(pb)
    s.set_state(U)
    dt = s.dt()

    def row(e):
        s.set_state(U)
        return af.af_adjoint_step(s.ctx, dt, e)

    Jfd, Jad = full_jacobians(s, U, lambda V: step_fixed_dt(s, V, dt), row)
    scale = Jfd.abs().max().item()
    assert (Jad - Jfd).abs().max().item() <= 1e-8 * scale


@pytest.mark.parametrize("bc,nx,ny", [(ai.PERIODIC, 12, 10), (ai.OUTFLOW, 11, 9), (ai.PERIODIC, 33, 17)])
def test_vjp_dot_product(bc, nx, ny):
    """<J^T v, d> = <v, J d> along smooth directions d, with J d by central differences."""
    pb = ai.random_smooth(nx, ny, seed=41, amp=0.2, bc=bc)
    U = cuda_state(ai.dofs(pb))
    s = solver_for(pb)
    gen = torch.Generator().manual_seed(7)
    unorm = math.sqrt(dot(U, U))
    for trial in range(4):
        v = rand_like(U, gen)
        d = cuda_state(ai.smooth_direction(pb, seed=trial))
        eps = 1e-6 * unorm
        s.set_state(U)
        jtv = af.af_rhs_vjp(s.ctx, v)
        s.set_state([u + eps * x for u, x in zip(U, d)])
        Lp = s.rhs()
        s.set_state([u - eps * x for u, x in zip(U, d)])
        Lm = s.rhs()
        fd = dot(v, [(p - m) / (2 * eps) for p, m in zip(Lp, Lm)])
        ad = dot(jtv, d)
        assert abs(fd - ad) <= 1e-8 * abs(fd), (trial, fd, ad)


def test_adjoint_step_against_central_differences():
    pb = ai.perturbed_vortex(24, seed=1)
    U = cuda_state(ai.dofs(pb))
    s = solver_for(pb)
    s.set_state(U)
    dt = s.dt()
    gen = torch.Generator().manual_seed(3)
    lam = rand_like(U, gen)
    s.set_state(U)
    lam_n = af.af_adjoint_step(s.ctx, dt, lam)
    # the state is not advanced by the adjoint
    for a, b in zip(s.get_state(), U):
        assert torch.equal(a, b)
    # the same numbers with a device dt, without the last-stage recomputation,
    # through host buffers, and in place
    dtt = torch.tensor([dt], dtype=torch.float64, device="cuda")
    for got in (af.af_adjoint_step(s.ctx, dtt, lam, recorded=True),
                af.af_adjoint_step(s.ctx, dt, [x.cpu().numpy() for x in lam], device=False),
                af.af_adjoint_step(s.ctx, dt, lam, recorded=True)):
        for a, b in zip(got, lam_n):
            assert torch.equal(torch.as_tensor(a).cuda(), b)
    inplace = [x.clone() for x in lam]
    af.af_adjoint_step(s.ctx, dtt, inplace, out=inplace)
    for a, b in zip(inplace, lam_n):
        assert torch.equal(a, b)
    # central differences along smooth directions, step 1e-6 |U|: the branch
    # points of the max in the LLF coefficient and rounding leave about 2e-8
    unorm = math.sqrt(dot(U, U))
    for trial in range(4):
        d = cuda_state(ai.smooth_direction(pb, seed=10 + trial))
        eps = 1e-6 * unorm
        Up = step_fixed_dt(s, [u + eps * x for u, x in zip(U, d)], dt)
        Um = step_fixed_dt(s, [u - eps * x for u, x in zip(U, d)], dt)
        fd = dot(lam, [(p - m) / (2 * eps) for p, m in zip(Up, Um)])
        ad = dot(lam_n, d)
        assert abs(fd - ad) <= 1e-7 * abs(fd), (trial, fd, ad)


def test_adjoint_refuses_sensor_and_active_limiters():
    pb = ai.blast(16)
    U = cuda_state(ai.dofs(pb))
    s = solver_for(pb, kappa=1.0)
    s.set_state(U)
    lam = [torch.ones_like(u) for u in U]
    with pytest.raises(af.AFError):
        af.af_adjoint_step(s.ctx, 1e-5, lam)
    s2 = solver_for(pb, kappa=0.0)
    s2.set_state(U)
    dt = s2.dt()
    s2.set_state(U)
    with pytest.raises(af.AFError):       # the blast limits its point values at once
        af.af_adjoint_step(s2.ctx, dt, lam)
    # the differentiable solve records the limiter activity of its forward pass and takes
    # the limited branch in backward (tests/test_gpu_adjoint_limited.py checks its values)
    X0 = [t.clone().requires_grad_(True) for t in U]
    out = af_steps(s2, X0, 2, checkpoint_every=1)
    J = magnetic_energy(out, pb.dx, pb.dy, pb.bc)
    J.backward()
    assert all(torch.isfinite(x.grad).all() for x in X0)


def magnetic_energy_np(U, pb):
    """The same objective on (complex) numpy states, periodic grids."""
    A, X, Y, Cn = U
    r = lambda t: np.roll(t, -1, axis=2)
    u = lambda t: np.roll(t, -1, axis=1)
    XL, XR, YD, YU = X, r(X), Y, u(Y)
    C00, C10, C01, C11 = Cn, r(Cn), u(Cn), u(r(Cn))
    Uc = 2.25 * A - 0.25 * ((XL + XR) + (YD + YU)) - 0.0625 * ((C00 + C10) + (C01 + C11))
    w = (1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0)
    nodes = [[C00, YD, C10], [XL, Uc, XR], [C01, YU, C11]]
    J = 0.0
    for m in range(3):
        for l in range(3):
            B = nodes[m][l][4:7]
            J = J + w[l] * w[m] * 0.5 * (B * B).sum()
    return J * pb.dx * pb.dy


def test_gradient_matches_oracle_complex_step():
    pb = ai.perturbed_vortex(16, seed=2)
    U0 = ai.dofs(pb)
    nsteps = 5
    s = solver_for(pb)
    X0 = [t.clone().requires_grad_(True) for t in cuda_state(U0)]
    out = af_steps(s, X0, nsteps, checkpoint_every=2)
    J = magnetic_energy(out, pb.dx, pb.dy, pb.bc)
    J.backward()
    grad = [x.grad for x in X0]
    # oracle: its own dt sequence, then complex-step derivatives along seeded directions
    dts, V = [], U0
    for _ in range(nsteps):
        V, d_ = oracle.step(pb, V)
        dts.append(d_)
    rng = np.random.default_rng(5)
    h = 1e-30
    for trial in range(3):
        d = [rng.normal(size=u.shape) for u in U0]
        re, im = [u.copy() for u in U0], [h * x for x in d]
        for n in range(nsteps):
            re, im, act = oracle.step_complex(pb, re, im, dts[n])
            assert act == 0
        Jc = magnetic_energy_np([a + 1j * b for a, b in zip(re, im)], pb)
        cs = Jc.imag / h
        ad = dot(grad, [torch.from_numpy(x).cuda() for x in d])
        assert abs(ad - cs) <= 1e-8 * abs(cs), (trial, ad, cs)
        assert abs(Jc.real - J.item()) <= 1e-12 * abs(Jc.real)


@pytest.mark.slow
def test_adjoint_workload_full_size():
    """256x256 perturbed vortex, 200 steps, checkpoints every 20 steps; the
    gradient of the magnetic energy against central differences (step
    1e-6 |U|, dt sequence recorded) along 32 seeded smooth directions."""
    pb = ai.perturbed_vortex(256, seed=0)
    U0 = cuda_state(ai.dofs(pb))
    nsteps = 200
    s = solver_for(pb)
    X0 = [t.clone().requires_grad_(True) for t in U0]
    out = af_steps(s, X0, nsteps, checkpoint_every=20)
    J = magnetic_energy(out, pb.dx, pb.dy, pb.bc)
    J.backward()
    grad = [x.grad for x in X0]
    s.set_state(U0)
    dts = [s.step() for _ in range(nsteps)]
    rc, cnt = s.status()
    assert rc == af.AF_OK and cnt["point_limited"] == 0 and cnt["lambda_lt1"] == 0

    def run(U):
        s.set_state(U)
        for n in range(nsteps):
            for k in range(3):
                s.stage(k, dts[n])
        return magnetic_energy(s.get_state(), pb.dx, pb.dy, pb.bc).item()

    assert abs(run(U0) - J.item()) <= 1e-14 * abs(J.item())
    eps = 1e-6 * math.sqrt(dot(U0, U0))
    worst = 0.0
    for seed in range(32):
        d = cuda_state(ai.smooth_direction(pb, seed=seed))
        fd = (run([u + eps * x for u, x in zip(U0, d)]) - run([u - eps * x for u, x in zip(U0, d)])) / (2 * eps)
        ad = dot(grad, d)
        worst = max(worst, abs(ad - fd) / abs(fd))
    assert worst <= 1e-6, worst


def test_dt_sensitivity_matches_oracle_complex_step():
    """With dt differentiated through its formula, the gradient of the magnetic
    energy after 5 steps equals the complex-step derivative of the oracle with
    the steps' own dt (dt of the complex state), and differs from the
    frozen-dt gradient."""
    pb = ai.perturbed_vortex(16, seed=2)
    U0 = ai.dofs(pb)
    nsteps = 5
    grads = {}
    for sens in (False, True):
        s = solver_for(pb)
        X0 = [t.clone().requires_grad_(True) for t in cuda_state(U0)]
        out = af_steps(s, X0, nsteps, checkpoint_every=2, dt_sensitivity=sens)
        magnetic_energy(out, pb.dx, pb.dy, pb.bc).backward()
        grads[sens] = [x.grad for x in X0]
    h = 1e-30
    for seed in range(3):
        d = ai.smooth_direction(pb, seed=20 + seed)
        re, im = [u.copy() for u in U0], [h * x for x in d]
        for _ in range(nsteps):
            re, im, act = oracle.step_complex(pb, re, im, 0.0)
            assert act == 0
        cs = magnetic_energy_np([a + 1j * b for a, b in zip(re, im)], pb).imag / h
        dd = cuda_state(d)
        ad = dot(grads[True], dd)
        frozen = dot(grads[False], dd)
        assert abs(ad - cs) <= 1e-8 * abs(cs), (seed, ad, cs)
        assert abs(frozen - cs) > 100 * abs(ad - cs), (seed, frozen, ad, cs)


def test_dt_sensitivity_step_against_central_differences():
    """One adjoint step with AF_ADJ_DT against central differences of af_step
    (dt recomputed from the perturbed state), host and device buffers."""
    pb = ai.perturbed_vortex(24, seed=1)
    U = cuda_state(ai.dofs(pb))
    s = solver_for(pb)
    s.set_state(U)
    dt = s.dt()
    gen = torch.Generator().manual_seed(5)
    lam = rand_like(U, gen)
    s.set_state(U)
    lam_n = af.af_adjoint_step(s.ctx, dt, lam, dt_sensitivity=True)
    host = af.af_adjoint_step(s.ctx, dt, [x.cpu().numpy() for x in lam], device=False, dt_sensitivity=True)
    for a, b in zip(host, lam_n):
        assert torch.equal(torch.as_tensor(a).cuda(), b)

    def natural_step(V):
        s.set_state(V)
        s.step(dt_out=False)
        return s.get_state()

    unorm = math.sqrt(dot(U, U))
    for seed in range(3):
        d = cuda_state(ai.smooth_direction(pb, seed=30 + seed))
        eps = 1e-7 * unorm
        Up = natural_step([u + eps * x for u, x in zip(U, d)])
        Um = natural_step([u - eps * x for u, x in zip(U, d)])
        fd = dot(lam, [(p - m) / (2 * eps) for p, m in zip(Up, Um)])
        ad = dot(lam_n, d)
        assert abs(fd - ad) <= 1e-6 * abs(fd), (seed, fd, ad)


@pytest.mark.parametrize("sens", [False, True])
@pytest.mark.parametrize("device", [True, False])
def test_adjoint_step_with_recorded_stages_is_bitwise(sens, device):
    """af_adjoint_step_stages on the forward step's stage states equals
    af_adjoint_step (which recomputes them) bit for bit, with and without the
    dt sensitivity, device and host buffers; and it refuses a stage state on
    which the cell-centre limiter acts."""
    pb = ai.perturbed_vortex(24, seed=3)
    U = cuda_state(ai.dofs(pb))
    s = solver_for(pb)
    s.set_state(U)
    dt = s.dt()
    gen = torch.Generator(device="cpu").manual_seed(7)
    lam = rand_like(U, gen)
    s.set_state(U)
    want = af.af_adjoint_step(s.ctx, dt, lam, recorded=True, dt_sensitivity=sens)
    s.set_state(U)
    stages = []
    for k in range(3):
        s.stage(k, dt)
        stages.append(s.get_stage())
    s.set_state(U)
    host = (lambda X: [x.cpu().numpy() for x in X]) if not device else (lambda X: X)
    got = af.af_adjoint_step_stages(s.ctx, dt, host(stages[0]), host(stages[1]), host(lam),
                                    U3=host(stages[2]) if sens else None, device=device, dt_sensitivity=sens)
    for w, g in zip(want, got):
        g = torch.as_tensor(g).cuda() if not device else g
        assert torch.equal(w, g)
    # the state is not advanced, and a repeated call gives the same result
    for a, b in zip(s.get_state(), U):
        assert torch.equal(a, b)
    if not sens:
        with pytest.raises(af.AFError):   # the dt sensitivity needs U3
            af.af_adjoint_step_stages(s.ctx, dt, stages[0], stages[1], lam, dt_sensitivity=True)
    # ten times denser corners: the centre value (36 avg - 4 faces - corners)/16
    # has negative density, so the Remark 3.2 limiter acts on every cell
    Ub = [u.clone() for u in U]
    Ub[3][0] *= 10.0
    s.set_state(Ub)
    with pytest.raises(af.AFError):
        af.af_adjoint_step_stages(s.ctx, dt, Ub, Ub, lam)
