"""The discrete adjoint along a limited branch (af_record_coeffs, af_freeze_coeffs,
af_stage_vjp, af_adjoint_step_frozen).

With the limiter coefficients of Sec. 3.2-3.4 (theta^s, theta_ij, the face theta,
the scaling-limiter theta*, theta** of points and cell centres) held at the values a
forward stage took, the stage is a smooth function of its input.  Checked here:
- recording and freezing reproduce the limited step (GPU), and the recorded
  coefficients equal the oracle's on the same stage input;
- the frozen GPU stage equals the oracle's frozen stage, with the recorded
  coefficients and with arbitrary ones;
- every entry of the transposed Jacobian of a frozen stage against central
  differences of the frozen GPU stage, on tiny grids with the sensor on (kappa = 1)
  and the limiters active;
- the transpose against the complex-step derivative of the oracle's frozen stage;
- a limited blast stage and a limited step against central differences.

States carry seeded grid-scale noise (1e-2 of each variable's size where central
differences are taken), so that no two values compared by a maximum -- the spectral
radii on an FVS line, |v_l| and c_f of the two states of an LLF flux -- lie within the
finite-difference perturbation of each other: the maxima are then differentiable at
the state and the perturbation stays on one branch, as the transpose assumes (it
differentiates along the branch the maxima take).  With 1e-3 noise on the lattice,
whose |v| = 6 everywhere, a few FVS lines had their two largest radii within the
perturbation, and central differences there averaged two branches.  The
finite-difference directions are smooth fields.  The magnetic field of the limited
problems is made generic (all three components non-zero): with B along one axis,
c_f along that axis equals max(c, |B|/sqrt(rho)) (the root of eq. cf has the
discriminant (c^2 - b^2)^2), which is not differentiable where the two speeds cross,
and the rarefactions sweep through that point.
"""
import dataclasses

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

GROUPS = [(0,), (1, 2, 3), (1, 2, 3), (1, 2, 3), (4, 5, 6), (4, 5, 6), (4, 5, 6), (7,)]


def rel_err(A, B):
    worst = 0.0
    for a, b in zip(A, B):
        a = a.cpu().numpy() if hasattr(a, "cpu") else np.asarray(a)
        for k in range(8):
            den = max(np.abs(b[q]).max() for q in GROUPS[k])
            if den == 0.0:
                assert np.abs(a[k] - b[k]).max() <= 1e-300
                continue
            worst = max(worst, np.abs(a[k] - b[k]).max() / den)
    return worst


def solver_for(pb, **kw):
    p = dict(cfl=pb.cfl, kappa=pb.kappa)
    p.update(kw)
    return af.Solver(pb.nx, pb.ny, pb.gamma, pb.bc, domain=(pb.x0, pb.x1, pb.y0, pb.y1), **p)


def cuda_state(U):
    return [torch.from_numpy(np.ascontiguousarray(u)).cuda() for u in U]


def noisy(pb, U, rel, seed):
    """U with seeded relative noise on every conserved variable (momenta and B scaled by
    the size of their vectors), the energy raised so that the pressure keeps its value."""
    rng = np.random.default_rng(seed)
    out = []
    for u in U:
        v = u.copy()
        scale = [np.abs(u[0]).max()] + [np.abs(u[1:4]).max() + 1e-3] * 3 + [np.abs(u[4:7]).max() + 1e-3] * 3
        p = (pb.gamma - 1) * (u[7] - 0.5 * (u[1:4] ** 2).sum(0) / u[0] - 0.5 * (u[4:7] ** 2).sum(0))
        for k in range(7):
            v[k] = u[k] + rel * scale[k] * rng.uniform(-1, 1, size=u[k].shape)
        v[0] = np.maximum(v[0], 0.5 * u[0])
        v[7] = p / (pb.gamma - 1) + 0.5 * (v[1:4] ** 2).sum(0) / v[0] + 0.5 * (v[4:7] ** 2).sum(0)
        out.append(v)
    return out


def generic_field(pb, B=(0.3, 0.5, 0.2)):
    """pb with its magnetic field replaced by the constant field B (all components non-zero)."""
    base = pb.prim

    def prim(x, y):
        w = list(base(x, y))
        z = 0.0 * np.asarray(w[0], dtype=np.float64)
        w[4], w[5], w[6] = z + B[0], z + B[1], z + B[2]
        return tuple(w)
    return dataclasses.replace(pb, prim=prim)


def smooth_dir(pb, U, seed):
    """A smooth seeded direction (af_inputs.smooth_direction), each variable of each class
    scaled to the largest magnitude that variable has in U."""
    d = ai.smooth_direction(pb, seed=seed)
    out = []
    for x, u in zip(d, U):
        u = u.cpu().numpy() if hasattr(u, "cpu") else u
        sc = np.abs(u).max(axis=(1, 2), keepdims=True) + 1e-3
        out.append(x * sc / np.abs(x).max(axis=(1, 2), keepdims=True))
    return out


def run_oracle(pb, U, nsteps):
    for _ in range(nsteps):
        U, _ = oracle.step(pb, U)
    return U


def record_stage(s, U, dt):
    """Stage 0 of the current state U with time step dt, recording its coefficients:
    (result, coefficient buffer of three blocks with block 0 filled)."""
    L = af.af_coeff_len(s.ctx)
    co = torch.full((3 * L,), float("nan"), dtype=torch.float64, device="cuda")
    s.set_state(U)
    af.af_record_coeffs(s.ctx, co)
    s.stage(0, dt)
    af.af_record_coeffs(s.ctx, None)
    G = s.get_stage()
    rc, _ = s.status(reset=True)
    assert rc == af.AF_OK
    return G, co


def frozen_stage(s, U, dt, co3):
    af.af_freeze_coeffs(s.ctx, co3)
    s.set_state(U)
    s.stage(0, dt)
    af.af_freeze_coeffs(s.ctx, None)
    return s.get_stage()


def block_shape(pb):
    nxa = pb.nx + (pb.bc == ai.OUTFLOW)
    nya = pb.ny + (pb.bc == ai.OUTFLOW)
    return nya, nxa


def oracle_to_block(pb, rec):
    """The oracle's coefficient dict as one stage block [AF_NCOEF][nya][nxa] (af.h order)."""
    nya, nxa = block_shape(pb)
    Bk = np.ones((af.AF_NCOEF, nya, nxa))
    put = lambda q, a: Bk[q, :a.shape[0], :a.shape[1]].__setitem__(Ellipsis, a)
    put(0, rec["ths_x"]); put(1, rec["ths_y"]); put(2, rec["th_x"]); put(3, rec["th_y"]); put(4, rec["th_src"])
    for c in range(4):
        put(5 + 2 * c, rec["th_pt%d" % c][0])
        put(6 + 2 * c, rec["th_pt%d" % c][1])
    return Bk


def block_to_dict(pb, blk):
    """A GPU stage block cut to the oracle's shapes."""
    shapes = oracle.coeff_shapes(pb.nx, pb.ny, pb.bc)
    nya, nxa = block_shape(pb)
    Bk = blk.reshape(af.AF_NCOEF, nya, nxa)
    cut = lambda q, sh: Bk[q, :sh[-2], :sh[-1]]
    d = {"ths_x": cut(0, shapes["ths_x"]), "ths_y": cut(1, shapes["ths_y"]), "th_x": cut(2, shapes["th_x"]),
         "th_y": cut(3, shapes["th_y"]), "th_src": cut(4, shapes["th_src"])}
    for c in range(4):
        sh = shapes["th_pt%d" % c]
        d["th_pt%d" % c] = np.stack([cut(5 + 2 * c, sh), cut(6 + 2 * c, sh)])
    return d


def three_blocks(blk0, L):
    co = torch.ones(3 * L, dtype=torch.float64, device="cuda")
    co[:L] = torch.as_tensor(np.ascontiguousarray(blk0).reshape(-1), device="cuda")
    return co


def n_limited(rec):
    return sum(int((np.asarray(v) < 1.0).sum()) for k, v in rec.items() if k not in ("ths_x", "ths_y", "ths_c"))


# limited problems and how far the oracle runs them first
CASES = {
    "double_rarefaction": (lambda: generic_field(ai.double_rarefaction(40, speed=6.0)), 20),
    "blast": (lambda: ai.blast(40), 2),
    "lattice": (lambda: generic_field(ai.rarefaction_lattice(48, periods=2)), 4),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_record_and_freeze_reproduce_the_limited_step(case):
    make, nsteps = CASES[case]
    pb = make()
    U = cuda_state(run_oracle(pb, ai.dofs(pb), nsteps))
    s = solver_for(pb)
    L = af.af_coeff_len(s.ctx)
    co = torch.full((3 * L,), float("nan"), dtype=torch.float64, device="cuda")
    s.set_state(U)
    af.af_record_coeffs(s.ctx, co)
    dt = s.step()
    af.af_record_coeffs(s.ctx, None)
    G1 = s.get_state()
    rc, cnt = s.status(reset=True)
    assert rc == af.AF_OK and cnt["point_limited"] + cnt["center_limited"] + cnt["lambda_lt1"] > 0
    for b in range(3):   # every entry the stage forms was written (outflow blocks have unused entries)
        rec = block_to_dict(pb, co[b * L:(b + 1) * L].cpu().numpy())
        assert not any(np.isnan(v).any() for v in rec.values())
    s.set_state(U)
    af.af_freeze_coeffs(s.ctx, co)
    assert s.step() == dt
    af.af_freeze_coeffs(s.ctx, None)
    G2 = s.get_state()
    rc, cnt2 = s.status(reset=True)
    assert rc == af.AF_OK and cnt2["newton_solves"] == 0
    # the frozen Lim1 is always U^LLF + theta_ij (U^src - U^LLF); the certified fast path forms
    # U^src directly, which rounds differently
    assert rel_err(G2, [g.cpu().numpy() for g in G1]) <= 1e-13
    s.close()


@pytest.mark.parametrize("case", sorted(CASES))
def test_recorded_coefficients_match_the_oracle(case):
    """On the oracle's stage inputs, the coefficients the GPU stage records equal the ones
    the oracle's stage takes (theta in [0, 1]: absolute difference)."""
    make, nsteps = CASES[case]
    pb = make()
    Un = run_oracle(pb, ai.dofs(pb), nsteps)
    dt = oracle.dt(pb, Un)
    s = solver_for(pb)
    active = 0
    Us = Un
    for a, b in [(0.0, 1.0), (0.75, 0.25)]:
        R, rec = oracle.stage_record(pb, Us, Us, dt, 0.0, 1.0)
        _, co = record_stage(s, cuda_state(Us), dt)
        got = block_to_dict(pb, co[:af.af_coeff_len(s.ctx)].cpu().numpy())
        for k in got:
            assert np.abs(got[k] - rec[k]).max() <= 1e-10, (k, np.abs(got[k] - rec[k]).max())
        active += n_limited(rec)
        Us = oracle.stage(pb, Un, Us, dt, a, b)
    assert active > 0
    s.close()


@pytest.mark.parametrize("case", sorted(CASES))
def test_frozen_stage_matches_the_oracle(case):
    """Both paths frozen at the same coefficients: the oracle's recorded ones, and seeded
    arbitrary ones in [0.85, 1] on every face, cell and point."""
    make, nsteps = CASES[case]
    pb = make()
    Us = run_oracle(pb, ai.dofs(pb), nsteps)
    dt = oracle.dt(pb, Us)
    _, rec = oracle.stage_record(pb, Us, Us, dt, 0.0, 1.0)
    rng = np.random.default_rng(7)
    arbitrary = {k: rng.uniform(0.85, 1.0, size=v.shape) for k, v in rec.items()}
    s = solver_for(pb)
    L = af.af_coeff_len(s.ctx)
    for coeffs in (rec, arbitrary):
        R, _ = oracle.stage_record(pb, Us, Us, dt, 0.0, 1.0, frozen=coeffs)
        G = frozen_stage(s, cuda_state(Us), dt, three_blocks(oracle_to_block(pb, coeffs), L))
        assert rel_err(G, R) <= 1e-12
    s.close()


def _jacobian_check(pb, U, dt, blk=None):
    """Every entry of (dFE/dU)^T (af_stage_vjp, unit cotangents) against central
    differences of the frozen stage, frozen at the coefficients the stage records (or at
    the block blk); returns (max error / max entry, number of limited coefficients)."""
    s = solver_for(pb)
    L = af.af_coeff_len(s.ctx)
    if blk is None:
        _, co = record_stage(s, U, dt)
        blk = co[:L].clone()
    else:
        co = three_blocks(blk, L)
        blk = co[:L].clone()
    rec = block_to_dict(pb, blk.cpu().numpy())
    shapes = [tuple(u.shape) for u in U]
    sizes = [int(np.prod(sh)) for sh in shapes]
    n = sum(sizes)
    flat = torch.cat([u.reshape(-1) for u in U])

    def unflat(x):
        out, o = [], 0
        for sh, m in zip(shapes, sizes):
            out.append(x[o:o + m].reshape(sh).contiguous())
            o += m
        return out

    JT = torch.empty((n, n), dtype=torch.float64)
    s.set_state(U)
    for m in range(n):
        e = torch.zeros(n, dtype=torch.float64, device="cuda")
        e[m] = 1.0
        out = af.af_stage_vjp(s.ctx, dt, blk, unflat(e))
        JT[:, m] = torch.cat([o.reshape(-1) for o in out]).cpu()   # row of J = column of J^T
    # central differences: column m of J from perturbing input m
    JF = torch.empty((n, n), dtype=torch.float64)
    # step: 1e-6 times the size of the input's variable over its class (rounding of the
    # stage output then stays near 1e-10 of the entries)
    hs = torch.cat([(u.abs().amax(dim=(1, 2), keepdim=True).clamp_min(1e-3) * 1e-6).expand(u.shape).reshape(-1)
                    for u in U]).cpu()
    for m in range(n):
        h = float(hs[m])
        x = flat.clone()
        x[m] += h
        Gp = frozen_stage(s, unflat(x), dt, co)
        x[m] -= 2 * h
        Gm = frozen_stage(s, unflat(x), dt, co)
        col = (torch.cat([g.reshape(-1) for g in Gp]) - torch.cat([g.reshape(-1) for g in Gm])) / (2 * h)
        JF[:, m] = col.cpu()
    s.close()
    # JT[i, m] = d FE_m / d U_i ; JF[m, i] = d FE_m / d U_i
    err = (JT - JF.T).abs().max().item() / JF.abs().max().item()
    return err, n_limited(rec)


FAMILIES = {"points": [7, 8, 9, 10, 11, 12], "face_theta": [2, 3], "theta_s": [0, 1], "theta_src": [4],
            "centre": [5, 6]}


@pytest.mark.parametrize("family", sorted(FAMILIES))
@pytest.mark.parametrize("bc", [ai.PERIODIC, ai.OUTFLOW])
def test_stage_vjp_each_coefficient_family(family, bc):
    """One family of limiter coefficients at seeded values in [0.3, 0.9], every other one
    at 1, on a smooth seeded state with grid-scale noise: every entry of the transposed
    Jacobian against central differences of the frozen stage (<= 1e-8 of the largest)."""
    nx, ny = (6, 6) if bc == ai.PERIODIC else (6, 5)
    pb = ai.random_smooth(nx, ny, seed=61, amp=0.3, bc=bc)
    pb.kappa = 1.0
    U = noisy(pb, ai.dofs(pb), 1e-3, 62)
    dt = oracle.dt(pb, U)
    nya, nxa = block_shape(pb)
    blk = np.ones((af.AF_NCOEF, nya, nxa))
    rng = np.random.default_rng(63)
    for q in FAMILIES[family]:
        blk[q] = rng.uniform(0.3, 0.9, size=(nya, nxa))
    err, _ = _jacobian_check(pb, cuda_state(U), dt, blk)
    assert err <= 1e-8, err


@pytest.mark.parametrize("case", ["lattice_periodic", "rarefaction_outflow"])
def test_stage_vjp_jacobian_against_central_differences(case):
    if case == "lattice_periodic":
        pb = generic_field(ai.rarefaction_lattice(8, periods=1))
        U = noisy(pb, ai.dofs(pb), 2e-2, 11)
    else:
        pb = generic_field(ai.double_rarefaction(6, speed=6.0))
        pb.ny = 5
        U = noisy(pb, run_oracle(pb, ai.dofs(pb), 3), 2e-2, 12)
    assert pb.kappa == 1.0
    dt = oracle.dt(pb, U)
    err, nlim = _jacobian_check(pb, cuda_state(U), dt)
    assert nlim > 0
    assert err <= 1e-8, err


@pytest.mark.parametrize("case", ["blast", "double_rarefaction"])
def test_stage_vjp_against_the_oracle_complex_step(case):
    """lam . (J d) from the complex step of the oracle's frozen stage (step 1e-30) against
    (J^T lam) . d of af_stage_vjp, both frozen at the oracle's coefficients: <= 1e-8 relative."""
    if case == "blast":
        pb = ai.blast(24)
        U = noisy(pb, run_oracle(pb, ai.dofs(pb), 2), 1e-4, 21)
    else:
        pb = generic_field(ai.double_rarefaction(20, speed=6.0))
        U = noisy(pb, run_oracle(pb, ai.dofs(pb), 8), 1e-4, 22)
    dt = oracle.dt(pb, U)
    _, rec = oracle.stage_record(pb, U, U, dt, 0.0, 1.0)
    assert n_limited(rec) > 0
    s = solver_for(pb)
    s.set_state(cuda_state(U))
    blk = torch.as_tensor(oracle_to_block(pb, rec).reshape(-1), device="cuda")
    rng = np.random.default_rng(5)
    for trial in range(3):
        d = [rng.standard_normal(u.shape) * (np.abs(u).max(axis=(1, 2), keepdims=True) + 1e-3) for u in U]
        lam = [rng.standard_normal(u.shape) for u in U]
        h = 1e-30
        re, im = oracle.stage_complex(pb, U, [h * x for x in d], U, [h * x for x in d], dt, 0.0, 1.0, frozen=rec)
        lhs = sum(float((l * (i / h)).sum()) for l, i in zip(lam, im))
        mu = af.af_stage_vjp(s.ctx, dt, blk, cuda_state(lam))
        rhs = sum(float((m.cpu().numpy() * x).sum()) for m, x in zip(mu, d))
        assert abs(lhs - rhs) <= 1e-8 * max(abs(lhs), abs(rhs)), (trial, lhs, rhs)
    s.close()


def test_limited_blast_stage_adjoint_against_central_differences():
    """The low-beta blast on 64x64 (kappa = 1) after three oracle steps, noise 1e-2: the
    adjoint of one limited forward-Euler stage along 8 seeded smooth directions (each
    variable scaled to its size), central differences of the frozen GPU stage with step
    1e-7 (|v| sits at the noise level in the quiet region; a larger step flips its sign
    at some DoFs, a kink of alpha)."""
    pb = ai.blast(64)
    U = cuda_state(noisy(pb, run_oracle(pb, ai.dofs(pb), 3), 1e-2, 31))
    dt = oracle.dt(pb, [u.cpu().numpy() for u in U])
    s = solver_for(pb)
    _, co = record_stage(s, U, dt)
    rec = block_to_dict(pb, co[:af.af_coeff_len(s.ctx)].cpu().numpy())
    assert n_limited(rec) > 0
    gen = torch.Generator().manual_seed(3)
    worst = 0.0
    for trial in range(8):
        d = cuda_state(smooth_dir(pb, U, 100 + trial))
        lam = [torch.randn(u.shape, generator=gen, dtype=torch.float64).cuda() for u in U]
        eps = 1e-7
        Gp = frozen_stage(s, [u + eps * x for u, x in zip(U, d)], dt, co)
        Gm = frozen_stage(s, [u - eps * x for u, x in zip(U, d)], dt, co)
        fd = sum(float((l * (p - m)).sum()) for l, p, m in zip(lam, Gp, Gm)) / (2 * eps)
        s.set_state(U)
        mu = af.af_stage_vjp(s.ctx, dt, co[:af.af_coeff_len(s.ctx)], lam)
        ad = sum(float((m * x).sum()) for m, x in zip(mu, d))
        worst = max(worst, abs(fd - ad) / max(abs(fd), abs(ad)))
    s.close()
    assert worst <= 1e-6, worst


@pytest.mark.parametrize("dt_sensitivity", [False, True])
def test_limited_step_adjoint_against_central_differences(dt_sensitivity):
    """One SSP-RK3 step of the double rarefaction near vacuum (every limiter and the Newton
    branch active in the recorded forward step), noise 1e-2: af_adjoint_step_frozen along 6
    seeded smooth directions against central differences of the frozen step -- dt held at
    the recorded value, or (dt_sensitivity) recomputed from the perturbed state."""
    pb = generic_field(ai.double_rarefaction(32, speed=6.0))
    U = cuda_state(noisy(pb, run_oracle(pb, ai.dofs(pb), 12), 1e-2, 41))
    s = solver_for(pb)
    L = af.af_coeff_len(s.ctx)
    co = torch.full((3 * L,), float("nan"), dtype=torch.float64, device="cuda")
    s.set_state(U)
    af.af_record_coeffs(s.ctx, co)
    dt = s.dt()
    stages = []
    for k in range(3):
        s.stage(k, dt)
        stages.append(s.get_stage())
    af.af_record_coeffs(s.ctx, None)
    rc, cnt = s.status(reset=True)
    assert rc == af.AF_OK and cnt["newton_solves"] > 0 and cnt["point_limited"] > 0

    def frozen_step(V):
        af.af_freeze_coeffs(s.ctx, co)
        s.set_state(V)
        if dt_sensitivity:
            s.step(dt_out=False)
        else:
            for k in range(3):
                s.stage(k, dt)
        af.af_freeze_coeffs(s.ctx, None)
        return s.get_state()

    gen = torch.Generator().manual_seed(4)
    worst = 0.0
    for trial in range(6):
        d = cuda_state(smooth_dir(pb, U, 200 + trial))
        lam = [torch.randn(u.shape, generator=gen, dtype=torch.float64).cuda() for u in U]
        eps = 1e-7
        Gp = frozen_step([u + eps * x for u, x in zip(U, d)])
        Gm = frozen_step([u - eps * x for u, x in zip(U, d)])
        fd = sum(float((l * (p - m)).sum()) for l, p, m in zip(lam, Gp, Gm)) / (2 * eps)
        s.set_state(U)
        mu = af.af_adjoint_step_frozen(s.ctx, dt, stages[0], stages[1], co, lam, U3=stages[2],
                                       dt_sensitivity=dt_sensitivity)
        ad = sum(float((m * x).sum()) for m, x in zip(mu, d))
        worst = max(worst, abs(fd - ad) / max(abs(fd), abs(ad)))
    s.close()
    assert worst <= 1e-6, worst


def test_checkpointed_solve_gradient_on_a_limited_run():
    """af_steps on a limited run (the double rarefaction near vacuum, kappa = 1, every
    limiter active; 6 steps, checkpoints every 4): the gradient of the magnetic energy
    against central differences of the same six steps, each frozen at the coefficients its
    forward step recorded and with its recorded dt, along 4 smooth directions (<= 1e-6)."""
    pb = generic_field(ai.double_rarefaction(32, speed=6.0))
    U = cuda_state(noisy(pb, run_oracle(pb, ai.dofs(pb), 10), 1e-2, 51))
    s = solver_for(pb)
    L = af.af_coeff_len(s.ctx)
    nsteps = 6
    X0 = [t.clone().requires_grad_(True) for t in U]
    out = af_steps(s, X0, nsteps, checkpoint_every=4)
    J = magnetic_energy(out, pb.dx, pb.dy, pb.bc)
    J.backward()
    grad = [x.grad for x in X0]
    # the forward steps again, recording each step's coefficients and dt
    s.set_state(U)
    cos, dts = [], []
    for _ in range(nsteps):
        co = torch.empty(3 * L, dtype=torch.float64, device="cuda")
        af.af_record_coeffs(s.ctx, co)
        dts.append(s.step())
        af.af_record_coeffs(s.ctx, None)
        cos.append(co)
    rc, cnt = s.status(reset=True)
    assert rc == af.AF_OK and cnt["point_limited"] > 0 and cnt["newton_solves"] > 0

    def frozen_run(V):
        s.set_state(V)
        for co, dt in zip(cos, dts):
            af.af_freeze_coeffs(s.ctx, co)
            for k in range(3):
                s.stage(k, dt)
            af.af_freeze_coeffs(s.ctx, None)
        return float(magnetic_energy(s.get_state(), pb.dx, pb.dy, pb.bc))

    worst = 0.0
    for trial in range(4):
        d = cuda_state(smooth_dir(pb, U, 300 + trial))
        eps = 1e-7
        fd = (frozen_run([u + eps * x for u, x in zip(U, d)]) - frozen_run([u - eps * x for u, x in zip(U, d)])) / (2 * eps)
        ad = sum(float((g_ * x).sum()) for g_, x in zip(grad, d))
        worst = max(worst, abs(fd - ad) / max(abs(fd), abs(ad)))
    s.close()
    assert worst <= 1e-6, worst
