"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle (``oracle/mg_oracle.c``) against something other than
itself: a closed form, an exact discrete solution, a library routine (FFT,
dense linear algebra), an invariant, or a value the paper prints.  The discrete
operator is recomputed here in a different algebraic form (the unsplit equation
with a full discrete Hessian, no operator splitting and no root formula), so a
dropped term, a wrong sign or a transposed index in the oracle's Sigma_ijk, its
branch choice or its root fails at least one test.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1303_0008_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
W = 1.0 / 3.0


# ---------------------------------------------------------------------------
# independent discrete forms (numpy), a[k, j, i] with x = i fastest
# ---------------------------------------------------------------------------
def sh(a, dx=0, dy=0, dz=0):
    """a shifted so that out[k, j, i] = a[k+dz, j+dy, i+dx] (periodic)."""
    return np.roll(a, shift=(-dz, -dy, -dx), axis=(0, 1, 2))


def hessian(phi, h):
    """Discrete Hessian: second differences on the diagonal, the four-point cross
    differences with their 1/4 off the diagonal (Sec. III.B)."""
    H = np.empty((3, 3) + phi.shape)
    unit = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    for a in range(3):
        ea = unit[a]
        H[a, a] = (sh(phi, *ea) + sh(phi, *[-e for e in ea]) - 2 * phi) / h ** 2
        for b in range(a + 1, 3):
            eb = unit[b]
            pp = sh(phi, *[x + y for x, y in zip(ea, eb)])
            mm = sh(phi, *[-x - y for x, y in zip(ea, eb)])
            pm = sh(phi, *[x - y for x, y in zip(ea, eb)])
            mp = sh(phi, *[-x + y for x, y in zip(ea, eb)])
            H[a, b] = H[b, a] = (pp + mm - pm - mp) / (4 * h ** 2)
    return H


def unsplit_lhs(phi, h, alpha):
    """lap(phi) + alpha [ (lap phi)^2 - (grad_i grad_j phi)^2 ] with the discrete Hessian."""
    H = hessian(phi, h)
    lap = H[0, 0] + H[1, 1] + H[2, 2]
    trh2 = np.einsum("ab...,ba...->...", H, H)
    return lap + alpha * (lap * lap - trh2), lap, trh2


def max_rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# ---------------------------------------------------------------------------
# linear limit: FFT Poisson solve with the exact discrete eigenvalues
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [12, 16, 24])
def test_fft_poisson_pin(n):
    rng = np.random.default_rng(7 + n)
    delta = rng.standard_normal((n, n, n))
    delta -= delta.mean()
    kappa = 1.7
    phi, st = O.fas_solve(delta, 0.0, kappa, tol=1e-12)
    assert st["status"] == O.OK
    h = 1.0 / n
    k = np.arange(n)
    s2 = np.sin(np.pi * k / n) ** 2
    eig = -(4 / h ** 2) * (s2[:, None, None] + s2[None, :, None] + s2[None, None, :])
    eig[0, 0, 0] = 1.0
    ph = np.fft.fftn(kappa * delta) / eig
    ph[0, 0, 0] = 0.0
    ref = np.fft.ifftn(ph).real
    assert max_rel(phi, ref) < 1e-11
    assert abs(st["lambda"]) < 1e-12


# ---------------------------------------------------------------------------
# 1D tests of Sec. IV.B: the nonlinear term vanishes in 1D
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("alpha", [0.3, -0.3, 0.05, 0.0])
def test_sine_1d_exact(alpha):
    g = GOLD["sine_1d"]
    K = g["K_over_pi2"] * math.pi ** 2
    n = 32
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    kd = -K * np.sin(2 * np.pi * x)            # kappa * delta, Eq. delta_sine
    kappa = 1.0 if alpha >= 0 else -1.0        # flip beta: alpha and kappa together
    delta = np.broadcast_to(kd / kappa, (n, n, n)).copy()
    # in the split form the 1D root equals kappa*delta while |2(1-w) alpha kappa delta| < 1
    assert abs(2 * (1 - W) * alpha * K) < 1
    phi, st = O.fas_solve(delta, alpha, kappa, tol=1e-12)
    assert st["status"] == O.OK
    A_h = K * h * h / (4 * math.sin(math.pi * h) ** 2)
    exact = np.broadcast_to(A_h * np.sin(2 * np.pi * x), (n, n, n))
    assert max_rel(phi, exact) < 1e-10
    # the discrete amplitude tends to the paper's 0.032 at O(h^2)
    assert abs(A_h / g["amplitude"] - 1 - (math.pi * h) ** 2 / 3) < 1e-4
    assert abs(A_h - g["amplitude"]) / g["amplitude"] < 4e-3


def test_gaussian_1d_manufactured():
    """The paper's Gaussian profile with its printed constants; delta is rebuilt from
    phi with the discrete second difference (the printed delta is not the second
    derivative of the printed phi: its bracket should read 1 - 2(x-0.5)^2/w^2)."""
    g = GOLD["gaussian_1d"]
    J, a, w = g["J"], g["alpha"], g["w"]
    n = 32
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    phi1 = J * (1 - a * np.exp(-((x - 0.5) ** 2) / w ** 2))
    lap1 = (np.roll(phi1, -1) + np.roll(phi1, 1) - 2 * phi1) / h ** 2
    # continuum check of the reading: the second derivative of phi
    u = x - 0.5
    d2 = 2 * J * a / w ** 2 * (1 - 2 * u * u / w ** 2) * np.exp(-u * u / w ** 2)
    inner = slice(1, -1)   # the profile is periodic only approximately (Sec. IV.B)
    assert np.abs(lap1 - d2)[inner].max() < 0.03 * np.abs(d2).max()
    printed = 2 * J * a / w ** 2 * (1 - u * u / w ** 2) * np.exp(-u * u / w ** 2)
    assert np.abs(printed - d2).max() > 0.1 * np.abs(d2).max()
    delta = np.broadcast_to(lap1, (n, n, n)).copy()
    for alpha in (0.3, -0.3):
        kappa = 1.0 if alpha > 0 else -1.0
        phi, st = O.fas_solve(delta / kappa, alpha, kappa, tol=1e-11)
        assert st["status"] == O.OK
        ref = np.broadcast_to(phi1 - phi1.mean(), (n, n, n))
        assert max_rel(phi, ref) < 1e-10


# ---------------------------------------------------------------------------
# 3D manufactured solution against the unsplit equation
# ---------------------------------------------------------------------------
def manufactured_phi(n, amp):
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    t = 2 * np.pi
    return amp * (np.sin(t * X) * np.cos(2 * t * Y) + 0.5 * np.cos(t * (Y + Z))
                  + 0.3 * np.sin(t * (X + 2 * Z)) + 0.2 * np.cos(t * (X - Y + Z)))


@pytest.mark.parametrize("alpha,kappa", [(0.3, 1.0), (-0.3, 1.0), (-0.3, -1.0), (2.4, 1.0)])
def test_manufactured_3d(alpha, kappa):
    n = 16
    h = 1.0 / n
    phis = manufactured_phi(n, 0.0012 / abs(alpha))  # keeps alpha * lap(phi*) of order 0.4
    lhs, lap, trh2 = unsplit_lhs(phis, h, alpha)
    # phi* must sit on the physical root of the split quadratic: 1 + 2(1-w) alpha lap > 0
    assert (1 + 2 * (1 - W) * alpha * lap).min() > 0.2
    delta = lhs / kappa
    phi, st = O.fas_solve(delta, alpha, kappa, tol=1e-12)
    assert st["status"] == O.OK and st["guard_hits"] == 0
    assert max_rel(phi, phis - phis.mean()) < 1e-10
    assert abs(st["lambda"]) < 1e-10
    # the oracle's residual of phi* itself is zero to rounding
    d, _ = O.residual(phis, delta, alpha, kappa)
    assert np.abs(d).max() < 1e-9 * np.abs(lhs).max()


def test_manufactured_detects_planted_sign_error():
    """The unsplit form is sensitive to the cross terms: flipping the sign of the
    mixed-derivative contribution changes the manufactured source."""
    n = 16
    h = 1.0 / n
    phis = manufactured_phi(n, 0.004)
    H = hessian(phis, h)
    lap = H[0, 0] + H[1, 1] + H[2, 2]
    good = np.einsum("ab...,ba...->...", H, H)
    bad = H[0, 0] ** 2 + H[1, 1] ** 2 + H[2, 2] ** 2 - 2 * (H[0, 1] ** 2 + H[0, 2] ** 2 + H[1, 2] ** 2)
    d_good, _ = O.residual(phis, lap + 0.3 * (lap * lap - good), 0.3, 1.0)
    d_bad, _ = O.residual(phis, lap + 0.3 * (lap * lap - bad), 0.3, 1.0)
    assert np.abs(d_good).max() < 1e-9 * np.abs(lap).max()
    assert np.abs(d_bad).max() > 1e-3 * np.abs(lap).max()


# ---------------------------------------------------------------------------
# brute-force Newton on the bordered system (8^3 + lambda)
# ---------------------------------------------------------------------------
def bordered_residual(x, delta, alpha, kappa, h, n):
    """G(phi, lambda): per cell the split quadratic in D = lap - lambda (or, where the
    discriminant is negative, D equal to the real part of the root), plus mean(phi)."""
    phi = x[:-1].reshape(n, n, n)
    lam = x[-1]
    H = hessian(phi, h)
    lap = H[0, 0] + H[1, 1] + H[2, 2]
    trh2 = np.einsum("ab...,ba...->...", H, H)
    D = lap - lam
    u = kappa * delta + alpha * (trh2 - W * lap * lap)
    q = 1 + 4 * (1 - W) * alpha * u
    G = np.where(q >= 0, alpha * (1 - W) * D * D + D - u, D + 1 / (2 * (1 - W) * alpha))
    return np.concatenate([G.ravel(), [phi.mean() * 1e3]]), q, D


def bordered_jacobian(x, delta, alpha, kappa, h, n, eps=1e-4):
    """Central-difference Jacobian of the bordered residual.  G is at most quadratic in
    x away from the guard switch, so central differences are exact up to rounding.
    Columns of cells 4 apart in every axis share no equation, so they are perturbed
    together (64 colours + lambda)."""
    N = n ** 3
    J = np.zeros((N + 1, N + 1))
    idx = np.arange(N).reshape(n, n, n)
    kk, jj, ii = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    for cz in range(4):
        for cy in range(4):
            for cx in range(4):
                cols = idx[(kk % 4 == cz) & (jj % 4 == cy) & (ii % 4 == cx)]
                e = np.zeros_like(x)
                e[cols] = eps
                dG = (bordered_residual(x + e, delta, alpha, kappa, h, n)[0]
                      - bordered_residual(x - e, delta, alpha, kappa, h, n)[0]) / (2 * eps)
                # row c belongs to the column whose stencil holds it
                for col in cols:
                    k0, j0, i0 = np.unravel_index(col, (n, n, n))
                    for dz in (-1, 0, 1):
                        for dy in (-1, 0, 1):
                            for dx in (-1, 0, 1):
                                r = idx[(k0 + dz) % n, (j0 + dy) % n, (i0 + dx) % n]
                                J[r, col] = dG[r]
                    J[N, col] = dG[N]
    e = np.zeros_like(x)
    e[N] = eps
    J[:, N] = (bordered_residual(x + e, delta, alpha, kappa, h, n)[0]
               - bordered_residual(x - e, delta, alpha, kappa, h, n)[0]) / (2 * eps)
    return J


def newton_bordered(delta, alpha, kappa, n, steps):
    """Newton with backtracking on ||G||_inf, by continuation in alpha."""
    h = 1.0 / n
    x = np.zeros(n ** 3 + 1)
    for t in np.linspace(1.0 / steps, 1.0, steps):
        a = alpha * t
        for it in range(60 if t == 1.0 else 15):
            G = bordered_residual(x, delta, a, kappa, h, n)[0]
            g0 = np.abs(G).max()
            if g0 < 1e-11:
                break
            dx = np.linalg.solve(bordered_jacobian(x, delta, a, kappa, h, n), G)
            s = 1.0
            while s > 1e-4 and np.abs(bordered_residual(x - s * dx, delta, a, kappa, h, n)[0]).max() >= g0:
                s *= 0.5
            x = x - s * dx
    return x


@pytest.mark.parametrize("ak,amp,steps", [(0.05, 1.0, 1), (0.3, 1.0, 1), (2.4, 0.3, 10)])
def test_bordered_newton_8cube(ak, amp, steps):
    """Brute-force Newton on the 513 x 513 bordered system (phi on 8^3, lambda), with
    the guard active in about a fifth of the cells for alpha*kappa = 2.4."""
    n = 8
    h = 1.0 / n
    rng = np.random.default_rng(81)
    delta = rng.uniform(-amp, amp, size=(n, n, n))
    delta -= delta.mean()
    alpha, kappa = ak, 1.0
    x = newton_bordered(delta, alpha, kappa, n, steps)
    G, q, D = bordered_residual(x, delta, alpha, kappa, h, n)
    assert np.abs(G).max() < 1e-10
    ok = q >= 0
    assert (1 + 2 * (1 - W) * alpha * D[ok]).min() >= 0  # physical root
    phi_ref, lam_ref = x[:-1].reshape(n, n, n), x[-1]
    phi, st = O.fas_solve(delta, alpha, kappa, tol=1e-12, max_cycles=200)
    assert st["status"] == O.OK
    assert max_rel(phi, phi_ref) < 1e-9
    assert abs(st["lambda"] - lam_ref) < 1e-9 * max(1.0, abs(lam_ref))
    assert st["guard_hits"] == int((~ok).sum())
    if ak == 2.4:
        assert st["guard_hits"] > 50


# ---------------------------------------------------------------------------
# Sec. IV.A uniform density, the wrong branch, the sign of alpha
# ---------------------------------------------------------------------------
def test_uniform_density_relaxes_to_constant():
    g = GOLD["uniform_density"]
    n = 16
    rng = np.random.default_rng(338)
    phi0 = rng.uniform(g["phi0_low"], g["phi0_high"], size=(n, n, n))
    phi, st = O.fas_solve(np.zeros((n, n, n)), 0.3, 1.0, tol=g["residual_eps"], phi0=phi0)
    assert st["status"] == O.OK and st["res"] < g["residual_eps"]
    assert phi.max() - phi.min() < 1e-11
    assert abs(st["lambda"]) < 1e-12


def test_wrong_branch_offsets_by_three_over_two_alpha():
    """Taking the other root at uniform density leaves lap(phi) != 0 unless the
    compatibility constant absorbs it: lambda = 3/(2 alpha) (Sec. III.A, after
    Eq. one_branch)."""
    n = 8
    rng = np.random.default_rng(217)
    phi0 = rng.uniform(-0.05, 0.05, size=(n, n, n))
    for alpha in (0.3, -0.7):
        wrong = -1 if alpha > 0 else 1
        phi, st = O.fas_solve(np.zeros((n, n, n)), alpha, 1.0, branch=wrong, tol=1e-11,
                              phi0=phi0)
        assert st["status"] == O.OK
        assert abs(st["lambda"] - 3 / (2 * alpha)) < 1e-10 * abs(3 / (2 * alpha))
        assert phi.max() - phi.min() < 1e-11
        _, st_ok = O.fas_solve(np.zeros((n, n, n)), alpha, 1.0, tol=1e-11, phi0=phi0)
        assert abs(st_ok["lambda"]) < 1e-12


def test_branch_flip_is_odd():
    n = 16
    delta = I.lognormal_delta(n, 1.5, 1302)
    a = I.alpha_kappa_for_rv(8.0)
    p1, s1 = O.fas_solve(delta, a, 1.0, tol=1e-11)
    p2, s2 = O.fas_solve(delta, -a, -1.0, tol=1e-11)
    assert s1["status"] == O.OK and s2["status"] == O.OK
    assert np.array_equal(p1, -p2)
    assert s1["cycles"] == s2["cycles"]


def test_guard_counts_and_is_sign_symmetric():
    n = 16
    delta = I.lognormal_delta(n, 1.5, 1302)
    a = I.alpha_kappa_for_rv(32.0)  # strong screening, voids fall below -3/(8 alpha kappa)
    p1, s1 = O.fas_solve(delta, a, 1.0, tol=1e-10, max_cycles=300)
    p2, s2 = O.fas_solve(delta, -a, -1.0, tol=1e-10, max_cycles=300)
    assert s1["guard_hits"] > 0 and s1["guard_hits"] == s2["guard_hits"]
    assert np.array_equal(p1, -p2)
    # cells that are guarded at u = kappa*delta alone (Sigma >= 0 can only lift u)
    assert s1["guard_hits"] <= int((1 + 8.0 / 3.0 * a * delta < 0).sum())


# ---------------------------------------------------------------------------
# transfers and force
# ---------------------------------------------------------------------------
def test_restriction_preserves_mean_and_linear_fields():
    n = 16
    rng = np.random.default_rng(5)
    f = rng.standard_normal((n, n, n))
    c = O.restrict(f)
    assert abs(c.mean() - f.mean()) < 1e-15
    x = np.arange(n) + 0.5
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    lin = 0.3 * X - 1.1 * Y + 0.7 * Z + 2.0
    xc = 2 * np.arange(n // 2) + 1.0
    Zc, Yc, Xc = np.meshgrid(xc, xc, xc, indexing="ij")
    assert np.abs(O.restrict(lin) - (0.3 * Xc - 1.1 * Yc + 0.7 * Zc + 2.0)).max() < 1e-13


def test_prolongation_exact_on_linear_fields_and_constants():
    nc = 8
    xc = 2 * np.arange(nc) + 1.0        # coarse centres in fine-cell units
    Zc, Yc, Xc = np.meshgrid(xc, xc, xc, indexing="ij")
    lin_c = 0.3 * Xc - 1.1 * Yc + 0.7 * Zc + 2.0
    out = O.prolong_add(lin_c, np.zeros((2 * nc,) * 3))
    x = np.arange(2 * nc) + 0.5
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    lin_f = 0.3 * X - 1.1 * Y + 0.7 * Z + 2.0
    inner = (slice(1, -1),) * 3        # away from the periodic wrap
    assert np.abs(out[inner] - lin_f[inner]).max() < 1e-12
    const = O.prolong_add(np.full((nc,) * 3, 1.25), np.full((2 * nc,) * 3, 0.5))
    assert np.abs(const - 1.75).max() < 1e-15


def test_force_is_minus_half_central_gradient():
    n = 16
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    phi = np.sin(2 * np.pi * X) + 0.5 * np.cos(2 * np.pi * Y) * np.sin(4 * np.pi * Z)
    g = O.force(phi)
    s = math.sin(2 * np.pi * h) / h
    s2 = math.sin(4 * np.pi * h) / h
    assert np.abs(g[0] - (-0.5 * np.cos(2 * np.pi * X) * s)).max() < 1e-12
    assert np.abs(g[1] - (0.5 * 0.5 * np.sin(2 * np.pi * Y) * s * np.sin(4 * np.pi * Z))).max() < 1e-12
    assert np.abs(g[2] - (-0.5 * 0.5 * np.cos(2 * np.pi * Y) * np.cos(4 * np.pi * Z) * s2)).max() < 1e-12


def test_num_levels():
    assert O.num_levels(32) == 4       # 32 16 8 4
    assert O.num_levels(128) == 6
    assert O.num_levels(96) == 5       # 96 48 24 12 6
    assert O.num_levels(6) == 1


# ---------------------------------------------------------------------------
# spherical top-hat: the closed-form Vainshtein profile (Sec. II.B, Sec. IV.C)
# ---------------------------------------------------------------------------
def _tophat_errors(n, R):
    delta = I.tophat(n, 10.0, R)
    nin = int((delta == 10.0).sum())
    Reff = (3 * nin / (4 * np.pi)) ** (1 / 3) / n
    dout = float(delta[delta != 10.0][0])
    alpha = I.alpha_kappa_for_rv(8.0)
    phi, st = O.fas_solve(delta, alpha, 1.0, tol=1e-10)
    phil, stl = O.fas_solve(delta, 0.0, 1.0, tol=1e-10)
    assert st["status"] == O.OK and stl["status"] == O.OK
    g, gl = -2 * O.force(phi), -2 * O.force(phil)
    x = (np.arange(n) + 0.5 - n / 2) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z)
    gr = (g[0] * X + g[1] * Y + g[2] * Z) / r
    glr = (gl[0] * X + gl[1] * Y + gl[2] * Z) / r
    m = np.where(r < Reff, 10.0 * r ** 3 / 3, (10.0 - dout) * Reff ** 3 / 3 + dout * r ** 3 / 3)
    ratio_cf = (r ** 3 / (4 * alpha * m)) * (np.sqrt(1 + 8 * alpha * m / r ** 3) - 1)
    sel = (r > Reff + 1.0 / n) & (r < 0.25)
    return np.abs(gr[sel] / glr[sel] - ratio_cf[sel]).max(), ratio_cf[sel]


def test_spherical_tophat_force_ratio_converges():
    """Fifth force over its unscreened value against the closed form
    (r/r_V)^3-type profile, with the compensating background in m(r).  Periodic
    images make it approximate (Sec. IV.C); the error must fall with h."""
    e32, ratio = _tophat_errors(32, 4.0)
    e64, _ = _tophat_errors(64, 8.0)
    assert ratio.min() < 0.7               # screening is visible inside r_V = 8 cells
    assert e32 < 0.06 and e64 < 0.03
    assert e64 < 0.7 * e32


def test_spherical_cases_read_with_radii_swapped():
    """Sec. IV.C says the two top-hats hold the same mass; that holds only with the
    radii exchanged (23.77 with R = 0.1, 190.9 with R = 0.05)."""
    (d1, r1), (d2, r2) = GOLD["spherical"]["cases"]
    literal = (d1 * r1 ** 3) / (d2 * r2 ** 3)
    swapped = (d1 * r2 ** 3) / (d2 * r1 ** 3)
    assert literal < 0.05                  # 64 times apart as printed
    assert abs(swapped - 1) < 0.01


# ---------------------------------------------------------------------------
# refinement levels (Sec. III.C first paragraph, Sec. IV.D)
# ---------------------------------------------------------------------------
def _quadratic(A, b, x, y, z):
    X = np.stack([x, y, z])
    return np.einsum("a...,ab,b...->...", X, A, X) + np.einsum("a,a...->...", b, X)


A_Q = np.array([[0.8, 0.3, -0.2], [0.3, -0.5, 0.25], [-0.2, 0.25, 0.4]])
B_Q = np.array([0.1, -0.2, 0.05])


def _level_centres(n):
    x = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return X, Y, Z


def _patch_cells(org, n):
    """Cell-centre coordinates of each 8^3 patch (count, 8, 8, 8)."""
    o = np.asarray(org)
    i = np.arange(8)
    xs = (o[:, 0, None] + i + 0.5) / n
    ys = (o[:, 1, None] + i + 0.5) / n
    zs = (o[:, 2, None] + i + 0.5) / n
    X = np.broadcast_to(xs[:, None, None, :], (len(o), 8, 8, 8))
    Y = np.broadcast_to(ys[:, None, :, None], (len(o), 8, 8, 8))
    Z = np.broadcast_to(zs[:, :, None, None], (len(o), 8, 8, 8))
    return X, Y, Z


def test_patch_ghosts_exact_on_linear_fields():
    n0 = 16
    X, Y, Z = _level_centres(n0)
    lin0 = 0.3 * X - 1.1 * Y + 0.7 * Z + 2.0
    org = np.array([[8, 8, 8], [16, 8, 8]], dtype=np.int32)
    gh = O.patch_ghosts(n0, 1, org, lin0)
    i = np.arange(-1, 9)
    for q, o in enumerate(org):
        xs, ys, zs = (o[0] + i + 0.5) / 32, (o[1] + i + 0.5) / 32, (o[2] + i + 0.5) / 32
        Zg, Yg, Xg = np.meshgrid(zs, ys, xs, indexing="ij")
        ref = 0.3 * Xg - 1.1 * Yg + 0.7 * Zg + 2.0
        m = ~np.isnan(gh[q])
        assert m.sum() > 0
        assert np.abs(gh[q][m] - ref[m]).max() < 1e-13
    # faces shared by the two patches are unknowns, not ghosts
    assert np.isnan(gh[0][1:9, 1:9, 9]).all() and np.isnan(gh[1][1:9, 1:9, 0]).all()
    # corners are not part of the 19-point stencil
    assert np.isnan(gh[0][0, 0, 0])


def test_patch_manufactured_quadratic_two_levels():
    """A quadratic phi* is reproduced exactly by the coarse-to-fine fill once the
    parent holds phi* - (3 H^2/16) tr(A) (the cell-centred trilinear offset), and its
    discrete Hessian is exact, so the refinement solve must return phi* to rounding."""
    n0, alpha, kappa = 16, 0.3, 1.0
    lap = 2 * np.trace(A_Q)
    H2 = 2 * A_Q
    lhs = lap + alpha * (lap * lap - np.sum(H2 * H2))
    assert 1 + 2 * (1 - W) * alpha * lap > 0
    # level 1: a 2x2x2 block of patches over [8, 24)^3
    org1 = np.array([[x, y, z] for z in (8, 16) for y in (8, 16) for x in (8, 16)], dtype=np.int32)
    X0, Y0, Z0 = _level_centres(n0)
    parent0 = _quadratic(A_Q, B_Q, X0, Y0, Z0) - 3 * (1.0 / n0) ** 2 / 16 * np.trace(A_Q)
    delta1 = np.full((len(org1), 8, 8, 8), lhs / kappa)
    phi1, st1 = O.patch_solve(n0, 1, org1, delta1, parent0, alpha, kappa, tol=1e-11)
    assert st1["status"] == O.OK
    ref1 = _quadratic(A_Q, B_Q, *_patch_cells(org1, 2 * n0))
    assert max_rel(phi1, ref1) < 1e-11
    # level 2: two patches whose parents (dilated by one cell) sit inside level 1
    org2 = np.array([[24, 24, 24], [32, 24, 24]], dtype=np.int32)
    parent1 = ref1 - 3 * (1.0 / (2 * n0)) ** 2 / 16 * np.trace(A_Q)
    delta2 = np.full((len(org2), 8, 8, 8), lhs / kappa)
    phi2, st2 = O.patch_solve(n0, 2, org2, delta2, parent1, alpha, kappa, parent_org=org1,
                              tol=1e-11)
    assert st2["status"] == O.OK
    ref2 = _quadratic(A_Q, B_Q, *_patch_cells(org2, 4 * n0))
    assert max_rel(phi2, ref2) < 1e-11
    d2, _ = O.patch_residual(n0, 2, org2, ref2, delta2, parent1, alpha, kappa, parent_org=org1)
    assert np.abs(d2).max() < 1e-8


def test_patch_nesting_violation_is_reported():
    org1 = np.array([[8, 8, 8]], dtype=np.int32)
    org2 = np.array([[24, 24, 24]], dtype=np.int32)   # parents 12..15, dilated 11..16: 16 missing
    with pytest.raises(ValueError):
        O.patch_ghosts(16, 2, org2, np.zeros((1, 8, 8, 8)), parent_org=org1)


def test_multilevel_tophat_refinement_improves_accuracy():
    """Sec. IV.D: a refinement over the sphere with the same density and boundary
    values interpolated from the domain grid.  The refined solution must sit much
    closer to a solve on a domain grid of the refined resolution than the domain
    solution interpolated onto the refined cells does."""
    n0 = 16
    alpha = I.alpha_kappa_for_rv(8.0)
    delta0 = I.tophat(n0, 10.0, 2.0)
    phi0, st0 = O.fas_solve(delta0, alpha, 1.0, tol=1e-11)
    org1 = np.array([[x, y, z] for z in (8, 16) for y in (8, 16) for x in (8, 16)], dtype=np.int32)
    fine = I.tophat(2 * n0, 10.0, 4.0)
    same = fine.copy()
    same[same != 10.0] = delta0[delta0 != 10.0][0]
    cut = lambda a: np.stack([a[o[2]:o[2] + 8, o[1]:o[1] + 8, o[0]:o[0] + 8] for o in org1])
    phi1, st1 = O.patch_solve(n0, 1, org1, cut(same), phi0, alpha, 1.0, tol=1e-11)
    assert st1["status"] == O.OK
    phif, stf = O.fas_solve(fine, alpha, 1.0, tol=1e-11)
    interp = O.prolong_add(phi0, np.zeros((2 * n0,) * 3))
    e_ref = np.abs(phi1 - cut(phif)).max()
    e_int = np.abs(cut(interp) - cut(phif)).max()
    assert e_ref < 0.3 * e_int
    assert e_ref < 0.03 * (phif.max() - phif.min())


# ---------------------------------------------------------------------------
# source floor (the reading used where alpha*kappa*delta < -3/8)
# ---------------------------------------------------------------------------
def test_density_floor_bound_and_symmetry():
    delta = I.lognormal_delta(16, 1.5, 1302)
    a = I.alpha_kappa_for_rv(32.0)
    fl, hits = O.density_floor(delta, a, 1.0)
    assert hits == int((1 + 4 * (1 - W) * a * delta < 0).sum()) > 0
    assert (1 + 4 * (1 - W) * a * fl >= -1e-12).all()
    assert np.array_equal(fl[fl != delta], np.full(hits, -1 / (4 * (1 - W) * a)))
    fl2, hits2 = O.density_floor(delta, -a, -1.0)        # flipping beta: same cells
    assert hits2 == hits and np.array_equal(fl, fl2)
    same, none = O.density_floor(delta, I.alpha_kappa_for_rv(8.0), 1.0)   # alpha*kappa < 3/8
    assert none == 0 and np.array_equal(same, delta)


def test_floored_system_has_no_imaginary_root_and_matches_brute_force():
    """With the floor, the discriminant is non-negative for any field: the solve sees no
    guarded cell, and brute-force Newton on the unsplit bordered 8^3 system agrees."""
    n = 8
    rng = np.random.default_rng(82)
    delta = rng.uniform(-1.0, 2.0, size=(n, n, n))
    delta -= delta.mean()
    alpha = 2.4
    fl, hits = O.density_floor(delta, alpha, 1.0)
    assert hits > 20
    phi, st = O.fas_solve(fl, alpha, 1.0, tol=1e-12, max_cycles=200)
    assert st["status"] == O.OK and st["guard_hits"] == 0
    x = newton_bordered(fl, alpha, 1.0, n, 8)
    G, q, D = bordered_residual(x, fl, alpha, 1.0, 1.0 / n, n)
    assert np.abs(G).max() < 1e-10 and (q >= 0).all()
    assert max_rel(phi, x[:-1].reshape(n, n, n)) < 1e-9


def test_floor_makes_the_strong_screening_case_converge():
    """r_V = 32 cells (alpha*kappa = 19.2) on the 32^3 lognormal field: with the
    real-part reading alone the Newton-Gauss-Seidel iteration cycles; with the floor
    it converges."""
    delta = I.lognormal_delta(32, 1.5, 1302)
    a = I.alpha_kappa_for_rv(32.0)
    _, st_root = O.fas_solve(delta, a, 1.0, tol=1e-10, max_cycles=40)
    assert st_root["status"] != O.OK and st_root["res"] > 1e-4
    fl, hits = O.density_floor(delta, a, 1.0)
    _, st = O.fas_solve(fl, a, 1.0, tol=1e-10, max_cycles=60)
    assert st["status"] == O.OK and st["guard_hits"] == 0


# ---------------------------------------------------------------------------
# Mass assignment (Sec. VI) and the refinement criterion (Sec. III.B)
# ---------------------------------------------------------------------------
def _rand_particles(count, seed):
    return np.random.default_rng(seed).random((3, count))


@pytest.mark.parametrize("scheme", [1, 2])
def test_assignment_conserves_mass_and_maps_a_lattice_to_uniform_density(scheme):
    n = 12
    pos = _rand_particles(500, 3)
    mass = np.random.default_rng(4).random(500)
    mass /= mass.sum()
    d = O.assign_density(n, pos, mass, scheme)
    assert abs((d + 1.0).sum() / n ** 3 - 1.0) < 1e-14
    # particles on the cell centres: the weights sum to one on every cell
    g = (np.arange(n) + 0.5) / n
    lat = np.stack([a.ravel() for a in np.meshgrid(g, g, g, indexing="ij")])
    assert np.abs(O.assign_density(n, lat, None, scheme)).max() < 1e-13


def test_tsc_is_cic_averaged_over_one_cell():
    """TSC is the cloud-in-cell kernel convolved with a one-cell box: the TSC
    density of a particle equals the mean of CIC densities of copies spread
    uniformly over a cell around it (midpoint rule, error O(1/m^2))."""
    n, m = 8, 24
    x0 = np.array([3.3, 4.71, 2.05]) / n
    t = ((np.arange(m) + 0.5) / m - 0.5) / n
    sx, sy, sz = np.meshgrid(t, t, t, indexing="ij")
    pos = np.stack([x0[0] + sx.ravel(), x0[1] + sy.ravel(), x0[2] + sz.ravel()])
    cic = O.assign_density(n, pos, None, 1)
    tsc = O.assign_density(n, x0.reshape(3, 1), None, 2)
    assert np.abs((cic + 1) - (tsc + 1)).max() < 3.0 / m ** 2 * np.abs(tsc + 1).max()


@pytest.mark.parametrize("scheme", [1, 2])
def test_assignment_is_periodic_and_translation_equivariant(scheme):
    n = 10
    pos = _rand_particles(200, 9)
    d = O.assign_density(n, pos, None, scheme)
    shifted = np.mod(pos + np.array([[3.0], [-1.0], [7.0]]) / n, 1.0)
    d2 = O.assign_density(n, shifted, None, scheme)
    assert np.abs(np.roll(d, (7, -1, 3), axis=(0, 1, 2)) - d2).max() < 1e-12


@pytest.mark.parametrize("scheme", [1, 2])
def test_assignment_keeps_the_centre_of_mass(scheme):
    n = 16
    x = np.array([[0.41], [0.52], [0.37]])
    rho = O.assign_density(n, x, None, scheme) + 1.0
    c = (np.arange(n) + 0.5) / n
    w = rho / rho.sum()
    com = [(w * c[None, None, :]).sum(), (w * c[None, :, None]).sum(),
           (w * c[:, None, None]).sum()]
    assert np.allclose(com, x.ravel(), atol=1e-14)


def test_refinement_blocks_hand_built():
    n = 16
    delta = np.zeros((n, n, n))
    mp = 1.0 / n ** 3                       # one particle per cell on average
    delta[9, 2, 13] = 9.5                   # 10.5 effective particles: refine
    delta[0, 0, 0] = 7.9                    # 8.9 effective particles: not with npc = 9
    org = O.refine_blocks(delta, 9.0, mp)
    assert org.tolist() == [[24, 0, 16]]    # block (3, 0, 2) -> level-1 origin x2 x4
    assert O.refine_blocks(delta, 8.0, mp).tolist() == [[0, 0, 0], [24, 0, 16]]


@pytest.mark.parametrize("w", [0.2, 1.0 / 3.0, 0.5])
def test_general_w_solution_satisfies_the_unsplit_equation(w):
    """For any splitting constant w the split root of Eq. two_branch, with the
    periodic compatibility constant lambda (D = lap - lambda), is equivalent to
    the unsplit discrete equation with a known lambda term:
      lap + a [lap^2 - tr H^2] = kappa delta + lambda + a (1 - w) lambda (2 lap - lambda),
    H the discrete Hessian of Sec. III.B (computed here independently)."""
    n = 16
    h = 1.0 / n
    rng = np.random.default_rng(90)
    delta = rng.uniform(-0.8, 0.8, size=(n, n, n))
    delta -= delta.mean()
    alpha, kappa = 0.3, 1.0
    phi, st = O.fas_solve(delta, alpha, kappa, tol=1e-13, max_cycles=200, w=w)
    assert st["status"] == O.OK and st["guard_hits"] == 0
    lhs, lap, _ = unsplit_lhs(phi, h, alpha)
    lam = st["lambda"]
    rhs = kappa * delta + lam + alpha * (1 - w) * lam * (2 * lap - lam)
    assert np.abs(lhs - rhs).max() < 1e-9 * np.abs(kappa * delta).max()
