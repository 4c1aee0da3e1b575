"""Seeded synthetic inputs for the Active Flux MHD hot path.

This module is shared by the CUDA path's tests/bench and by the CPU oracle's
tests.  It holds no arithmetic of the scheme: only the initial conditions of
the paper's test problems (and of the benchmark workloads built on them),
evaluated into the four DoF classes, plus seeded random draws.

DoF layout (one class): numpy float64 array [8, nyp, nxp], conserved variables
U = (rho, rho v1, rho v2, rho v3, B1, B2, B3, E), x fastest.  Classes: 0 cell
averages, 1 x-face point values at (x0 + f dx, y_j), 2 y-face point values at
(x_i, y0 + g dy), 3 corner point values at (x0 + f dx, y0 + g dy).
Periodic grids store nx x ny of every class; outflow grids store
(nx+1) x ny x-faces, nx x (ny+1) y-faces and (nx+1) x (ny+1) corners.

Point values are exact pointwise evaluations of the initial condition; cell
averages use 5x5 Gauss-Legendre tensor quadrature of the conserved variables
(the paper does not say how its initial DoFs are formed).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Sequence

import numpy as np

PERIODIC = 0
OUTFLOW = 1


@dataclasses.dataclass
class Problem:
    """A test problem: domain, boundary condition, gamma and the primitive IC.

    prim(x, y) returns (rho, v1, v2, v3, B1, B2, B3, p) arrays broadcast to x's shape.
    """
    name: str
    nx: int
    ny: int
    x0: float
    x1: float
    y0: float
    y1: float
    bc: int
    gamma: float
    prim: Callable
    kappa: float = 0.0
    cfl: float = 0.2
    t_end: float = 0.0
    # outflow problems only: boundary kind of each side (left, right, bottom,
    # top): 0 outflow, 1 reflective, 2 inflow (bottom/top) with the conserved
    # inflow state inflow_U where inflow_lo < x < inflow_hi
    sides: tuple = (0, 0, 0, 0)
    inflow_lo: float = 0.0
    inflow_hi: float = 0.0
    inflow_U: tuple = None

    @property
    def dx(self) -> float:
        return (self.x1 - self.x0) / self.nx

    @property
    def dy(self) -> float:
        return (self.y1 - self.y0) / self.ny


def class_extents(nx: int, ny: int, bc: int) -> List[tuple]:
    """(nxp, nyp) of classes 0..3."""
    fx = nx if bc == PERIODIC else nx + 1
    fy = ny if bc == PERIODIC else ny + 1
    return [(nx, ny), (fx, ny), (nx, fy), (fx, fy)]


def prim_to_cons(w: Sequence[np.ndarray], gamma: float) -> np.ndarray:
    """Conserved variables from (rho, v, B, p): E = p/(gamma-1) + rho|v|^2/2 + |B|^2/2."""
    rho, v1, v2, v3, b1, b2, b3, p = [np.asarray(a, dtype=np.float64) for a in w]
    shape = np.broadcast(rho, v1, v2, v3, b1, b2, b3, p).shape
    out = np.empty((8,) + shape)
    out[0] = rho
    out[1] = rho * v1
    out[2] = rho * v2
    out[3] = rho * v3
    out[4] = b1
    out[5] = b2
    out[6] = b3
    out[7] = p / (gamma - 1.0) + 0.5 * rho * (v1 * v1 + v2 * v2 + v3 * v3) + 0.5 * (b1 * b1 + b2 * b2 + b3 * b3)
    return out


def _gauss_legendre(n: int):
    xg, wg = np.polynomial.legendre.leggauss(n)
    return 0.5 * xg, 0.5 * wg  # nodes/weights on [-1/2, 1/2]


def dofs(pb: Problem, quad: int = 5) -> List[np.ndarray]:
    """The four DoF classes of pb's initial condition."""
    return class_values(pb, lambda X, Y: prim_to_cons(pb.prim(X, Y), pb.gamma), quad)


def class_values(pb: Problem, fn, quad: int = 5) -> List[np.ndarray]:
    """The four DoF classes of a field fn(X, Y) -> (8, ...) on pb's grid: cell
    averages by tensor Gauss-Legendre quadrature, point values exactly."""
    nx, ny = pb.nx, pb.ny
    dx, dy = pb.dx, pb.dy
    ext = class_extents(nx, ny, pb.bc)
    xc = pb.x0 + (np.arange(nx) + 0.5) * dx
    yc = pb.y0 + (np.arange(ny) + 0.5) * dy
    xf = pb.x0 + np.arange(ext[1][0]) * dx
    yf = pb.y0 + np.arange(ext[2][1]) * dy
    out = []
    xg, wg = _gauss_legendre(quad)
    acc = None
    for a in range(quad):
        for b in range(quad):
            X, Y = np.meshgrid(xc + xg[a] * dx, yc + xg[b] * dy, indexing="xy")
            v = wg[a] * wg[b] * np.asarray(fn(X, Y))
            acc = v if acc is None else acc + v
    out.append(np.ascontiguousarray(acc))
    for xs, ys in ((xf, yc), (xc, yf), (xf, yf)):
        X, Y = np.meshgrid(xs, ys, indexing="xy")
        out.append(np.ascontiguousarray(np.asarray(fn(X, Y))))
    return out


def smooth_direction(pb: Problem, seed: int, kmax: int = 4) -> List[np.ndarray]:
    """A seeded smooth direction in state space: every conserved variable is a
    random Fourier series with wave numbers |k| <= kmax, periodic on pb's
    domain, taken as DoFs like a state; scaled to unit 2-norm over all DoFs.
    Used for directional-derivative (finite-difference) checks."""
    rng = np.random.default_rng(seed)
    Lx, Ly = pb.x1 - pb.x0, pb.y1 - pb.y0
    ks = [(a, b) for a in range(-kmax, kmax + 1) for b in range(-kmax, kmax + 1) if a * a + b * b <= kmax * kmax]
    coef = rng.normal(size=(8, len(ks)))
    phase = rng.uniform(0.0, 2.0 * math.pi, size=(8, len(ks)))
    # sum_k c cos(2 pi (a x' + b y') + ph) = Re(Ey^T M Ex) on a tensor grid,
    # M[b, a] = sum of c e^{i ph} over the modes (a, b)
    M = np.zeros((8, 2 * kmax + 1, 2 * kmax + 1), dtype=complex)
    for t, (a, b) in enumerate(ks):
        M[:, b + kmax, a + kmax] += coef[:, t] * np.exp(1j * phase[:, t])
    kk = np.arange(-kmax, kmax + 1)

    def fn(X, Y):
        xs, ys = X[0, :], Y[:, 0]     # class_values evaluates on meshgrids (indexing "xy")
        Ex = np.exp(2j * math.pi * np.outer(kk, (xs - pb.x0) / Lx))
        Ey = np.exp(2j * math.pi * np.outer(kk, (ys - pb.y0) / Ly))
        return np.real(np.matmul(Ey.T, np.matmul(M, Ex)))

    d = class_values(pb, fn)
    nrm = math.sqrt(sum(float((x * x).sum()) for x in d))
    return [x / nrm for x in d]


def _b(x, v):
    return np.broadcast_to(np.asarray(v, dtype=np.float64), np.shape(x)).copy()


# ---------------------------------------------------------------------------
# The paper's problems (Sec. 4) and the benchmark workloads built on them.
# ---------------------------------------------------------------------------

def vortex(n: int = 64, mu: float = 1.0, xi: float = 1.0, half_width: float = 5.0, t: float = 0.0,
           gamma: float = 5.0 / 3.0) -> Problem:
    """MHD vortex (Example 4.3, second case) advected by v = (1, 1).

    Perturbations, with the 1/(2 pi) amplitude factors of the source problem:
      dv = xi/(2 pi) e^{(1-r^2)/2} (-y, x), dB = mu/(2 pi) e^{(1-r^2)/2} (-y, x),
      dp = (mu^2 (1 - r^2) - xi^2) e^{1-r^2} / (8 pi^2).
    With mu = 5.389489439, xi = sqrt(2) mu this gives p_min = 1 - mu^2 e/(8 pi^2)
    ~ 5.3e-12 as the paper states (without the 1/(2 pi) factors it would be
    negative).  The exact solution at time t is the initial state shifted by
    (t, t) in the periodic box.
    """
    L = 2.0 * half_width

    def prim(x, y):
        xs = np.mod(x - t + half_width, L) - half_width
        ys = np.mod(y - t + half_width, L) - half_width
        r2 = xs * xs + ys * ys
        e = np.exp(0.5 * (1.0 - r2))
        a = 1.0 / (2.0 * math.pi)
        v1 = 1.0 + xi * a * e * (-ys)
        v2 = 1.0 + xi * a * e * xs
        b1 = mu * a * e * (-ys)
        b2 = mu * a * e * xs
        p = 1.0 + (mu * mu * (1.0 - r2) - xi * xi) * np.exp(1.0 - r2) / (8.0 * math.pi ** 2)
        return (_b(x, 1.0), v1, v2, _b(x, 0.0), b1, b2, _b(x, 0.0), p)

    return Problem("vortex", n, n, -half_width, half_width, -half_width, half_width, PERIODIC, gamma, prim)


def sine_wave(n: int = 32, t: float = 0.0) -> Problem:
    """Smooth sine wave (Example 4.3, first case), exact at any time t:
    (rho, v, B, p) = (1 + 0.99 sin(2 pi (x + y - 2 t)), 1, 1, 0, 0.1, 0.1, 0, 1)."""

    def prim(x, y):
        rho = 1.0 + 0.99 * np.sin(2.0 * math.pi * (x + y - 2.0 * t))
        return (rho, _b(x, 1.0), _b(x, 1.0), _b(x, 0.0), _b(x, 0.1), _b(x, 0.1), _b(x, 0.0), _b(x, 1.0))

    return Problem("sine_wave", n, n, 0.0, 1.0, 0.0, 1.0, PERIODIC, 5.0 / 3.0, prim)


def orszag_tang(n: int = 512, ny: int | None = None, amp_v: float = 1.0, amp_b: float = 1.0,
                phase_x: float = 0.0, phase_y: float = 0.0, kappa: float = 1.0) -> Problem:
    """Orszag-Tang vortex on [0, 2 pi]^2 (benchmark normalisation, gamma = 5/3):
    rho = gamma^2, p = gamma, v = a_v (-sin y', sin x', 0), B = a_B (-sin y', sin 2x', 0)
    with x' = x + phase_x, y' = y + phase_y."""
    gamma = 5.0 / 3.0

    def prim(x, y):
        xp, yp = x + phase_x, y + phase_y
        return (_b(x, gamma * gamma), -amp_v * np.sin(yp), amp_v * np.sin(xp), _b(x, 0.0),
                -amp_b * np.sin(yp), amp_b * np.sin(2.0 * xp), _b(x, 0.0), _b(x, gamma))

    return Problem("orszag_tang", n, ny or n, 0.0, 2.0 * math.pi, 0.0, 2.0 * math.pi, PERIODIC, gamma, prim,
                   kappa=kappa)


def orszag_tang_paper(n: int = 400, kappa: float = 1.0) -> Problem:
    """Orszag-Tang in the paper's normalisation (Example 4.4), [0,1]^2:
    (rho, v, B, p) = (25/(36 pi), -sin 2 pi y, sin 2 pi x, 0, -sin(2 pi y)/sqrt(4 pi),
    sin(4 pi x)/sqrt(4 pi), 0, 5/(12 pi))."""
    s4 = math.sqrt(4.0 * math.pi)

    def prim(x, y):
        return (_b(x, 25.0 / (36.0 * math.pi)), -np.sin(2 * math.pi * y), np.sin(2 * math.pi * x), _b(x, 0.0),
                -np.sin(2 * math.pi * y) / s4, np.sin(4 * math.pi * x) / s4, _b(x, 0.0), _b(x, 5.0 / (12.0 * math.pi)))

    return Problem("orszag_tang_paper", n, n, 0.0, 1.0, 0.0, 1.0, PERIODIC, 5.0 / 3.0, prim, kappa=kappa)


def blast(n: int = 2048, low_beta: bool = True, kappa: float = 1.0) -> Problem:
    """Blast wave on [-0.5, 0.5]^2 with outflow boundaries.

    low_beta=True (benchmark workload): gamma = 1.4, rho = 1, v = 0,
    p = 1000 for r < 0.1 else 0.1, B = (100/sqrt(4 pi)) (1/sqrt 2, 1/sqrt 2, 0).
    low_beta=False (Example 4.6): gamma = 5/3, p = 10 / 0.1, B = (1/sqrt 2, 1/sqrt 2, 0).
    """
    if low_beta:
        gamma, pin, pout, bmag = 1.4, 1000.0, 0.1, 100.0 / math.sqrt(4.0 * math.pi)
    else:
        gamma, pin, pout, bmag = 5.0 / 3.0, 10.0, 0.1, 1.0
    b = bmag / math.sqrt(2.0)

    def prim(x, y):
        r2 = x * x + y * y
        p = np.where(r2 < 0.01, pin, pout)
        return (_b(x, 1.0), _b(x, 0.0), _b(x, 0.0), _b(x, 0.0), _b(x, b), _b(x, b), _b(x, 0.0), p)

    return Problem("blast_low_beta" if low_beta else "blast", n, n, -0.5, 0.5, -0.5, 0.5, OUTFLOW, gamma, prim,
                   kappa=kappa)


def rotor(n: int = 400, kappa: float = 2.0) -> Problem:
    """Second rotor problem (Example 4.5), periodic [0,1]^2, gamma = 5/3.

    The taper is read as f = (r1 - r)/(r1 - r0), which makes the state continuous
    at r0 and r1; the printed (r1 - r)/(r - r0) is singular at r = r0."""
    r0, r1 = 0.1, 0.115
    b1 = 2.5 / math.sqrt(4.0 * math.pi)

    def prim(x, y):
        dx_, dy_ = x - 0.5, y - 0.5
        r = np.sqrt(dx_ * dx_ + dy_ * dy_)
        f = (r1 - r) / (r1 - r0)
        inside = r < r0
        mid = (r >= r0) & (r < r1)
        rho = np.where(inside, 10.0, np.where(mid, 1.0 + 9.0 * f, 1.0))
        rs = np.maximum(r, 1e-300)
        v1 = np.where(inside, -dy_ / r0, np.where(mid, -f * dy_ / rs, 0.0))
        v2 = np.where(inside, dx_ / r0, np.where(mid, f * dx_ / rs, 0.0))
        return (rho, v1, v2, _b(x, 0.0), _b(x, b1), _b(x, 0.0), _b(x, 0.0), _b(x, 0.5))

    return Problem("rotor", n, n, 0.0, 1.0, 0.0, 1.0, PERIODIC, 5.0 / 3.0, prim, kappa=kappa)


def quadrants_hydro(n: int = 48, kappa: float = 1.0) -> Problem:
    """A degenerate case: pure hydrodynamics (B = 0) on [0,1]^2, outflow, gamma
    = 1.4, at rest, with four constant quadrants around (0.5, 0.5):
    (rho, p) = (1, 1) top right, (0.25, 0.1) top left, (0.5, 0.4) bottom left,
    (2, 2) bottom right.  With B = 0 the fast speed is the sound speed, the
    sensor's phi_3 is 0 / 1e-40 and the Powell source vanishes; B must stay
    exactly zero."""
    def prim(x, y):
        x = np.asarray(x, dtype=np.float64)
        z = 0.0 * x
        right, top = x > 0.5, y > 0.5
        rho = np.where(top, np.where(right, 1.0, 0.25), np.where(right, 2.0, 0.5))
        p = np.where(top, np.where(right, 1.0, 0.1), np.where(right, 2.0, 0.4))
        return (rho + z, z, z, z, z, z, z, p + z)
    return Problem("quadrants_hydro", n, n, 0.0, 1.0, 0.0, 1.0, OUTFLOW, 1.4, prim, kappa=kappa)


def double_rarefaction(n: int = 48, speed: float = 2.5, kappa: float = 1.0) -> Problem:
    """A degenerate case: two rarefactions moving apart (v1 = -speed for x <
    0.5, +speed beyond) in rho = 1, p = 0.4, B = (0, 0.5, 0), gamma = 1.4,
    outflow on [0,1]^2.  The centre is driven towards vacuum, where the
    positivity limiters and the 1e-13 floors act."""
    def prim(x, y):
        x = np.asarray(x, dtype=np.float64)
        z = 0.0 * x
        v1 = np.where(x < 0.5, -speed, speed) + z
        return (z + 1.0, v1, z, z, z, z + 0.5, z, z + 0.4)
    return Problem("double_rarefaction", n, n, 0.0, 1.0, 0.0, 1.0, OUTFLOW, 1.4, prim, kappa=kappa)


def rarefaction_lattice(n: int = 2048, periods: int = 64, speed: float = 6.0, kappa: float = 1.0) -> Problem:
    """The double rarefaction's gas (rho = 1, p = 0.4, B = (0, 0.5, 0), gamma = 1.4) on the
    periodic unit square with v = speed (sgn sin 2 pi m x, sgn sin 2 pi m y, 0), m = periods:
    where both components diverge the flow opens towards vacuum (every limiter of Sec. 3.2-3.3
    and the Newton solve act), where they collide it drives shocks.  A workload that keeps
    the positivity limiters busy on a large grid."""
    def prim(x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64) + 0.0 * x
        z = 0.0 * x
        v1 = np.where(np.sin(2.0 * math.pi * periods * x) < 0.0, -speed, speed) + z
        v2 = np.where(np.sin(2.0 * math.pi * periods * y) < 0.0, -speed, speed) + z
        return (z + 1.0, v1, v2, z, z, z + 0.5, z, z + 0.4)
    return Problem("rarefaction_lattice", n, n, 0.0, 1.0, 0.0, 1.0, PERIODIC, 1.4, prim, kappa=kappa)


def shock_cloud(n: int = 400, kappa: float = 1.0) -> Problem:
    """Shock-cloud interaction (Example 4.7) on [0,1]^2, gamma = 5/3, outflow
    boundaries.  Reading: the printed state vectors list (rho, v1, v2, v3, p, B1,
    B2, B3) (as printed in the order (rho, v, B, p) the left pressure would be
    negative); left of x = 0.6: rho = 3.86859, v = 0, p = 167.345,
    B = (0, 2.1826182, -2.1826182); right: rho = 1, v = (-11.2536, 0, 0), p = 1,
    B = (0, 0.56418958, 0.56418958); a cloud rho = 10 of radius 0.15 centred at
    (0.8, 0.5), in pressure balance with the right state."""
    def prim(x, y):
        left = x < 0.6
        cloud = (x - 0.8) ** 2 + (y - 0.5) ** 2 < 0.15 ** 2
        rho = np.where(left, 3.86859, np.where(cloud, 10.0, 1.0))
        v1 = np.where(left, 0.0, -11.2536)
        p = np.where(left, 167.345, 1.0)
        b2 = np.where(left, 2.1826182, 0.56418958)
        b3 = np.where(left, -2.1826182, 0.56418958)
        return (rho, v1, _b(x, 0.0), _b(x, 0.0), _b(x, 0.0), b2, b3, p)

    return Problem("shock_cloud", n, n, 0.0, 1.0, 0.0, 1.0, OUTFLOW, 5.0 / 3.0, prim, kappa=kappa)


REFLECT, INFLOW = 1, 2


def jets(n: int = 200, ba: float = math.sqrt(20000.0), kappa: float = 2.0) -> Problem:
    """MHD jets (Example 4.8): the left half [-0.5, 0] x [0, 1.5] on n x 3n
    cells, gamma = 1.4; ambient rho = 0.1 gamma, p = 1, v = 0, B = (0, ba, 0);
    the jet (rho, v1, v2, p) = (gamma, 0, 800, 1) enters through the bottom for
    |x| < 0.05; reflective at x = 0, outflow on the other sides; T = 0.002.
    Reading: the jet carries the ambient field B = (0, ba, 0)."""
    g = 1.4
    jet = prim_to_cons((g, 0.0, 800.0, 0.0, 0.0, ba, 0.0, 1.0), g)

    def prim(x, y):
        z = 0.0 * np.asarray(x, dtype=np.float64) + 0.0 * np.asarray(y, dtype=np.float64)
        return (z + 0.1 * g, z, z, z, z, z + ba, z, z + 1.0)

    return Problem("jets", n, 3 * n, -0.5, 0.0, 0.0, 1.5, OUTFLOW, g, prim, kappa=kappa, t_end=0.002,
                   sides=(0, REFLECT, INFLOW, 0), inflow_lo=-0.05, inflow_hi=0.05,
                   inflow_U=tuple(float(v) for v in jet))


def constant(n: int = 16, ny: int | None = None, bc: int = PERIODIC, gamma: float = 5.0 / 3.0,
             w=(1.3, 0.4, -0.7, 0.2, 0.6, -0.3, 0.25, 2.1)) -> Problem:
    """A uniform state (free-stream preservation)."""

    def prim(x, y):
        return tuple(_b(x, c) for c in w)

    return Problem("constant", n, ny or n, 0.0, 1.0, 0.0, 1.0, bc, gamma, prim)


def random_smooth(n: int = 16, ny: int | None = None, seed: int = 0, modes: int = 3, amp: float = 0.2,
                  gamma: float = 5.0 / 3.0, bc: int = PERIODIC, divfree: bool = False) -> Problem:
    """A seeded smooth periodic state on [0,1]^2: each primitive is a mean plus
    a few random Fourier modes.  With divfree=True, B = curl(A_z e_z) + const."""
    rng = np.random.default_rng(seed)
    means = np.array([1.0, 0.3, -0.2, 0.1, 0.5, -0.4, 0.2, 1.0])
    coef = rng.uniform(-1.0, 1.0, size=(8, modes, modes, 2))
    phase = rng.uniform(0.0, 2.0 * math.pi, size=(8, modes, modes, 2))

    def field(q, x, y, dxo=0, dyo=0):
        # value (or first derivative) of the Fourier series of variable q
        out = np.zeros(np.shape(x), dtype=np.result_type(x, y, 1.0))
        for a in range(modes):
            for b in range(modes):
                k1, k2 = 2.0 * math.pi * a, 2.0 * math.pi * (b + (1 if a == 0 else 0))
                for s in range(2):
                    kk2 = k2 if s == 0 else -k2
                    arg = k1 * x + kk2 * y + phase[q, a, b, s]
                    c = coef[q, a, b, s] / (1.0 + a * a + b * b)
                    if dxo == 0 and dyo == 0:
                        out += c * np.cos(arg)
                    elif dxo == 1:
                        out += -c * k1 * np.sin(arg)
                    else:
                        out += -c * kk2 * np.sin(arg)
        return out

    def prim(x, y):
        w = [means[q] + amp * field(q, x, y) for q in range(8)]
        if divfree:
            # A_z from the B1 series: B = (dA/dy, -dA/dx)
            w[4] = means[4] + amp * field(4, x, y, dyo=1) / (2.0 * math.pi)
            w[5] = means[5] - amp * field(4, x, y, dxo=1) / (2.0 * math.pi)
        return tuple(w)

    return Problem("random_smooth", n, ny or n, 0.0, 1.0, 0.0, 1.0, bc, gamma, prim)


def ot_ensemble(count: int = 256, seed: int = 0, sizes=(64, 128, 256, 512), kappa: float = 1.0) -> List[Problem]:
    """Seeded ensemble of Orszag-Tang runs: nx and ny drawn independently from
    sizes, amplitude factors a_v, a_B ~ U(0.8, 1.2), phases ~ U(0, 2 pi)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nx = int(rng.choice(sizes))
        ny = int(rng.choice(sizes))
        av, ab = rng.uniform(0.8, 1.2, size=2)
        px, py = rng.uniform(0.0, 2.0 * math.pi, size=2)
        pb = orszag_tang(nx, ny, float(av), float(ab), float(px), float(py), kappa=kappa)
        out.append(pb)
    return out


def transpose_state(U: List[np.ndarray]) -> List[np.ndarray]:
    """The x<->y mirror image of a state: (x, y, v1, v2, B1, B2) -> (y, x, v2, v1, B2, B1).
    x-faces and y-faces swap roles."""
    perm = [0, 2, 1, 3, 5, 4, 6, 7]

    def tr(a):
        return np.ascontiguousarray(a[perm].transpose(0, 2, 1))

    return [tr(U[0]), tr(U[2]), tr(U[1]), tr(U[3])]


def perturbed_vortex(n: int = 256, seed: int = 0, amp: float = 1e-3, kmax: int = 4,
                     half_width: float = 5.0) -> Problem:
    """Smooth vortex (mu = xi = 1) with a seeded random Fourier perturbation of
    rho and of B (modes |k| <= kmax).  B is perturbed through A_z so that the
    perturbation is divergence free; both perturbations are scaled to max amp."""
    base = vortex(n, 1.0, 1.0, half_width)
    rng = np.random.default_rng(seed)
    L = 2.0 * half_width
    ks = [(a, b) for a in range(-kmax, kmax + 1) for b in range(-kmax, kmax + 1)
          if (a, b) != (0, 0) and a * a + b * b <= kmax * kmax]
    cr = rng.normal(size=len(ks))
    pr = rng.uniform(0, 2 * math.pi, size=len(ks))
    ca = rng.normal(size=len(ks))
    pa = rng.uniform(0, 2 * math.pi, size=len(ks))
    # normalisation on a fine sample grid
    xs = np.linspace(-half_width, half_width, 257)
    X, Y = np.meshgrid(xs, xs, indexing="xy")

    def series(X, Y, c, ph, deriv=None):
        out = np.zeros(np.shape(X), dtype=np.result_type(X, Y, 1.0))
        for (a, b), cc, pp in zip(ks, c, ph):
            k1, k2 = 2 * math.pi * a / L, 2 * math.pi * b / L
            arg = k1 * (X + half_width) + k2 * (Y + half_width) + pp
            if deriv is None:
                out += cc * np.cos(arg)
            elif deriv == "x":
                out += -cc * k1 * np.sin(arg)
            else:
                out += -cc * k2 * np.sin(arg)
        return out

    sr = amp / np.abs(series(X, Y, cr, pr)).max()
    bmax = np.sqrt(series(X, Y, ca, pa, "y") ** 2 + series(X, Y, ca, pa, "x") ** 2).max()
    sa = amp / bmax

    def prim(x, y):
        w = list(base.prim(x, y))
        w[0] = w[0] + sr * series(x, y, cr, pr)
        w[4] = w[4] + sa * series(x, y, ca, pa, "y")
        w[5] = w[5] - sa * series(x, y, ca, pa, "x")
        return tuple(w)

    return Problem("perturbed_vortex", n, n, -half_width, half_width, -half_width, half_width, PERIODIC,
                   base.gamma, prim)


# ---------------------------------------------------------------------------
# 1D problems (Sec. 4, Examples 4.1-4.2): states [averages [8, n], point values [8, nf]]
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Problem1D:
    """A 1D test problem on [x0, x1]; prim(x) returns (rho, v1, v2, v3, B1, B2, B3, p)."""
    name: str
    n: int
    x0: float
    x1: float
    bc: int
    gamma: float
    prim: Callable
    kappa: float = 0.0
    cfl: float = 0.2
    t_end: float = 0.0
    y0: float = 0.0     # unused; lets the 2D parameter helpers serve 1D problems
    y1: float = 1.0

    @property
    def dx(self) -> float:
        return (self.x1 - self.x0) / self.n

    @property
    def nf(self) -> int:
        return self.n if self.bc == PERIODIC else self.n + 1


def dofs1(pb: Problem1D, quad: int = 5) -> List[np.ndarray]:
    """Cell averages (Gauss-Legendre quadrature of the conserved variables) and
    exact interface point values of pb's initial condition."""
    xg, wg = _gauss_legendre(quad)
    xc = pb.x0 + (np.arange(pb.n) + 0.5) * pb.dx
    acc = None
    for a in range(quad):
        v = wg[a] * prim_to_cons(pb.prim(xc + xg[a] * pb.dx), pb.gamma)
        acc = v if acc is None else acc + v
    xf = pb.x0 + np.arange(pb.nf) * pb.dx
    return [np.ascontiguousarray(acc), np.ascontiguousarray(prim_to_cons(pb.prim(xf), pb.gamma))]


def _piecewise(left, right, x_split=0.5):
    def prim(x):
        x = np.asarray(x, dtype=np.float64)
        return tuple(np.where(x < x_split, l, r) + 0.0 * x for l, r in zip(left, right))
    return prim


def riemann_rj(n: int = 800, kappa: float = 10.0) -> Problem1D:
    """Example 4.1, first case: gamma = 2, [0,1], split at 0.5, T = 0.2."""
    return Problem1D("riemann_rj", n, 0.0, 1.0, OUTFLOW, 2.0,
                     _piecewise((1.0, 0.0, 0.0, 0.0, 0.75, 1.0, 0.0, 1.0),
                                (0.125, 0.0, 0.0, 0.0, 0.75, -1.0, 0.0, 0.1)), kappa=kappa, t_end=0.2)


def riemann_2(n: int = 800, kappa: float = 50.0) -> Problem1D:
    """Example 4.1, second case: gamma = 5/3, [0,1], split at 0.5, T = 0.2."""
    s = math.sqrt(4.0 * math.pi)
    return Problem1D("riemann_2", n, 0.0, 1.0, OUTFLOW, 5.0 / 3.0,
                     _piecewise((1.08, 1.2, 0.01, 0.5, 2.0 / s, 3.6 / s, 2.0 / s, 0.95),
                                (1.0, 0.0, 0.0, 0.0, 2.0 / s, 4.0 / s, 2.0 / s, 1.0)), kappa=kappa, t_end=0.2)


def blast1d(n: int = 400, kappa: float = 1.0) -> Problem1D:
    """A strong 1D blast: the low-beta blast's pressure jump (1000 / 0.1) and field
    B = (100/sqrt(4 pi)) (1/sqrt 2, 1/sqrt 2, 0), gamma = 1.4, on [-0.5, 0.5] with
    p = 1000 for |x| < 0.1; outflow.  Positivity test for the 1D limiters."""
    b = 100.0 / math.sqrt(4.0 * math.pi) / math.sqrt(2.0)

    def prim(x):
        x = np.asarray(x, dtype=np.float64)
        z = 0.0 * x
        return (z + 1.0, z, z, z, z + b, z + b, z, np.where(np.abs(x) < 0.1, 1000.0, 0.1) + z)
    return Problem1D("blast1d", n, -0.5, 0.5, OUTFLOW, 1.4, prim, kappa=kappa)


def entropy_wave1d(n: int = 64, t: float = 0.0, amp: float = 0.2, gamma: float = 5.0 / 3.0) -> Problem1D:
    """A density wave rho = 1 + amp sin(2 pi (x - t)) carried by uniform v = (1, 0.2, -0.1),
    B = (0.6, 0.3, 0.1), p = 1 on the periodic [0,1]: an exact solution (shifted by t)."""
    def prim(x):
        x = np.asarray(x, dtype=np.float64)
        z = 0.0 * x
        return (1.0 + amp * np.sin(2.0 * math.pi * (x - t)), z + 1.0, z + 0.2, z - 0.1, z + 0.6, z + 0.3, z + 0.1,
                z + 1.0)
    return Problem1D("entropy_wave1d", n, 0.0, 1.0, PERIODIC, gamma, prim)


def mirror1d(U: List[np.ndarray]) -> List[np.ndarray]:
    """The mirror image x -> -x of a 1D state: reversed order, v1 and B1 negated
    (the averages reverse; the point values reverse onto the same face set)."""
    out = []
    for a in U:
        b = a[:, ::-1].copy()
        b[1] = -b[1]
        b[4] = -b[4]
        out.append(b)
    return out
