"""The seeded synthetic inputs: each generator has the properties its docstring
states, so the workloads the tests and the benchmark name are the ones they get."""
import math

import numpy as np
import pytest

from paper_1303_0008_gb300 import inputs as I


def test_gaussian_field_is_zero_mean_unit_variance_and_seeded():
    a = I.gaussian_field(32, 7)
    assert abs(a.mean()) < 1e-12 and abs(a.std() - 1.0) < 1e-12
    assert np.array_equal(a, I.gaussian_field(32, 7))
    assert not np.array_equal(a, I.gaussian_field(32, 8))


def test_gaussian_field_has_the_power_law_spectrum():
    """Shell-averaged |g_k|^2 of the field falls as k^-2 (the index the lognormal
    workload uses), fitted over the shells 2..n/4 of a few seeds."""
    n = 64
    f = np.fft.fftfreq(n) * n
    kz, ky, kx = np.meshgrid(f, f, f, indexing="ij")
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    shells = np.arange(2, n // 4)
    power = np.zeros(len(shells))
    for seed in range(4):
        gk = np.abs(np.fft.fftn(I.gaussian_field(n, 100 + seed))) ** 2
        power += np.array([gk[(kk >= s - 0.5) & (kk < s + 0.5)].mean() for s in shells])
    slope = np.polyfit(np.log(shells), np.log(power), 1)[0]
    assert abs(slope - (-2.0)) < 0.1


@pytest.mark.parametrize("sigma", [0.5, 1.5, 2.0])
def test_lognormal_delta_has_mean_zero_and_log_density_spread_sigma(sigma):
    d = I.lognormal_delta(32, sigma, 1302)
    assert abs(d.mean()) < 1e-12
    assert d.min() > -1.0
    # log rho = sigma g + constant with g of unit variance
    assert abs(np.log1p(d).std() - sigma) < 1e-10
    assert np.array_equal(d, I.lognormal_delta(32, sigma, 1302))


def test_vainshtein_radius_parameter_closed_form():
    """r_V^3 = 8 alpha kappa m with m = delta0 R^3 / 3 for the reference top-hat
    (delta0 = 10, R = 4 cells): r_V = 8 cells gives alpha kappa = 0.3."""
    assert I.alpha_kappa_for_rv(8.0) == pytest.approx(0.3, rel=1e-15)
    for rv in (2.0, 16.0, 32.0):
        ak = I.alpha_kappa_for_rv(rv)
        m = I.TOPHAT_DELTA0 * I.TOPHAT_RADIUS ** 3 / 3.0
        assert (8.0 * ak * m) ** (1.0 / 3.0) == pytest.approx(rv, rel=1e-12)


def test_tophat_mass_and_zero_mean():
    n = 32
    d = I.tophat(n)
    inside = d == I.TOPHAT_DELTA0
    x = np.arange(n) + 0.5 - n / 2
    zz, yy, xx = np.meshgrid(x, x, x, indexing="ij")
    assert np.array_equal(inside, xx ** 2 + yy ** 2 + zz ** 2 < I.TOPHAT_RADIUS ** 2)
    assert abs(d.mean()) < 1e-14
    # a ball of radius 4 cells holds about (4/3) pi 4^3 cell centres
    assert abs(inside.sum() - 4.0 / 3.0 * math.pi * 64) < 0.1 * 4.0 / 3.0 * math.pi * 64


def test_benchmark_workload_is_three_radii_times_two_signs():
    w = I.workload_lognormal_sweep(16, 1.5, 1302)
    pairs = [(s["r_v"], s["alpha"], s["kappa"]) for s in w["solves"]]
    assert [p[0] for p in pairs] == [2.0, 2.0, 8.0, 8.0, 32.0, 32.0]
    for k in range(0, 6, 2):
        (rv, a, kp), (_, a2, kp2) = pairs[k], pairs[k + 1]
        assert a == I.alpha_kappa_for_rv(rv) and kp == 1.0 and (a2, kp2) == (-a, -1.0)


def test_batch_workload_ranges():
    b = I.workload_batch()
    assert len(b) == 64 and {s["n"] for s in b} <= {32, 64, 96, 128}
    for s in b:
        assert 0.5 <= s["sigma"] <= 2.5 and 2.0 <= s["r_v"] <= 16.0
        assert s["alpha"] == pytest.approx(math.copysign(I.alpha_kappa_for_rv(s["r_v"]), s["kappa"]))


@pytest.mark.parametrize("n0,sigma,thr", [(16, 2.0, (15.0, 40.0)), (32, 2.0, (20.0, 80.0))])
def test_refined_hierarchy_patches_are_aligned_unique_and_properly_nested(n0, sigma, thr):
    """Patch origins are multiples of 8 inside their level's periodic index space,
    each appears once, and every level-2 patch's parent block, dilated by one
    level-1 cell (the trilinear ghost stencil of Sec. III.C), lies inside level-1
    patches.  The densities are contrasts of a positive density."""
    h = I.refined_hierarchy(n0, sigma, 5, thresholds=thr)
    assert all(L["origins"].shape[0] > 0 for L in h["levels"])   # both levels exercised
    n = n0
    covered = None
    for lvl, L in enumerate(h["levels"], start=1):
        n *= 2
        org = L["origins"]
        if org.shape[0] == 0:
            continue
        assert org.dtype == np.int32 and (org % I.PATCH == 0).all()
        assert (org >= 0).all() and (org < n).all()
        assert len({tuple(o) for o in org}) == org.shape[0]
        assert L["delta"].shape == (org.shape[0], 8, 8, 8) and L["delta"].min() > -1.0
        if lvl == 2:
            n1 = n // 2
            for o in org:
                par = o // 2
                for dz in range(-1, 5):
                    for dy in range(-1, 5):
                        for dx in range(-1, 5):
                            c = ((par[0] + dx) % n1, (par[1] + dy) % n1, (par[2] + dz) % n1)
                            assert (c[0] // 8, c[1] // 8, c[2] // 8) in covered
        covered = {tuple(o // I.PATCH) for o in org}
    h2 = I.refined_hierarchy(n0, sigma, 5, thresholds=thr)
    assert np.array_equal(h["delta0"], h2["delta0"])
    for a, b in zip(h["levels"], h2["levels"]):
        assert np.array_equal(a["origins"], b["origins"]) and np.array_equal(a["delta"], b["delta"])
