"""Pins of the four-colour OpenMP build of the oracle (the CPU baseline).

It is checked against an exact discrete solution built from the unsplit
equation (as the lexicographic oracle is), against the lexicographic oracle's
fixed point on lognormal fields of both branches and with the source floor, and
for independence of the thread count.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1303_0008_gb300 import inputs as I

from test_oracle_pins import manufactured_phi, max_rel, unsplit_lhs

W = 1.0 / 3.0


@pytest.mark.parametrize("alpha,kappa", [(0.3, 1.0), (-0.3, -1.0), (2.4, 1.0)])
def test_colour_solve_recovers_manufactured_solution(alpha, kappa):
    n = 16
    phis = manufactured_phi(n, 0.0012 / abs(alpha))
    lhs, lap, _ = unsplit_lhs(phis, 1.0 / n, alpha)
    assert (1 + 2 * (1 - W) * alpha * lap).min() > 0.2
    phi, st = O.fas_solve_colour(lhs / kappa, alpha, kappa, tol=1e-12, threads=2)
    assert st["status"] == O.OK and st["guard_hits"] == 0
    assert max_rel(phi, phis - phis.mean()) < 1e-10
    assert abs(st["lambda"]) < 1e-10


@pytest.mark.parametrize("n,rv,sign", [(16, 8.0, 1.0), (24, 8.0, -1.0), (16, 16.0, 1.0),
                                       (32, 2.0, 1.0)])
def test_colour_solve_reaches_the_lexicographic_fixed_point(n, rv, sign):
    delta = I.lognormal_delta(n, 1.5, 4000 + n)
    a = sign * I.alpha_kappa_for_rv(rv)
    fl, _ = O.density_floor(delta, a, sign)
    p_lex, s_lex = O.fas_solve(fl, a, sign, tol=1e-11)
    p_col, s_col = O.fas_solve_colour(fl, a, sign, tol=1e-11)
    assert s_lex["status"] == O.OK and s_col["status"] == O.OK
    assert max_rel(p_col, p_lex) < 1e-10
    assert abs(s_col["lambda"] - s_lex["lambda"]) < 1e-9 * max(1.0, abs(s_lex["lambda"]))
    # and the colour result is a solution by the lexicographic oracle's residual
    d, _ = O.residual(p_col, fl, a, sign)
    assert np.abs(d - d.mean()).max() < 2e-11


def test_colour_sweep_is_a_sweep_of_the_same_update():
    """One colour sweep from phi = 0 touches every cell once: cells of colour 0 see
    only zeros, so their update equals the oracle's pointwise solve there."""
    n = 12
    delta = I.lognormal_delta(n, 1.0, 77)
    a = I.alpha_kappa_for_rv(8.0)
    phi, threads = O.colour_sweeps(np.zeros_like(delta), delta, a, 1.0, sweeps=1, threads=2)
    assert threads == 2
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    col0 = (((i + k) & 1) + 2 * ((j + k) & 1)) == 0
    # a cell of colour 0 with all neighbours at zero: Sigma_d = 0, so 6 phi = -h^2 D(kappa delta)
    one = O.gs_sweeps(np.zeros_like(delta), delta, a, 1.0, sweeps=1)
    # the lexicographic sweep's first cell (0, 0, 0) also sees only zeros
    assert phi[0, 0, 0] == one[0, 0, 0]
    assert np.all(phi[col0] != 0.0)


def test_colour_solve_does_not_depend_on_the_thread_count():
    delta = I.lognormal_delta(16, 1.5, 91)
    a = I.alpha_kappa_for_rv(8.0)
    p1, s1 = O.fas_solve_colour(delta, a, 1.0, tol=1e-11, threads=1)
    p3, s3 = O.fas_solve_colour(delta, a, 1.0, tol=1e-11, threads=3)
    assert s1["threads"] == 1 and s3["threads"] == 3
    assert s1["cycles"] == s3["cycles"]
    assert max_rel(p3, p1) < 1e-12
