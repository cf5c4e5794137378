"""Newtonian potential (Eq. newton) and the total force -grad(phi_N + phi/2)
through the C-ABI, against the CPU oracle's linear (alpha = 0) solve and its
force stencil, on the domain and on refinement levels."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1303_0008_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1303_0008_gb300 import mg  # noqa: E402

COEF = 1.5 * 0.27  # (3/2) Omega_m a at a = 1


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_newton_potential_and_total_force_domain():
    n = 48
    delta = I.lognormal_delta(n, 1.5, 4242)
    alpha = I.alpha_kappa_for_rv(8.0)
    g = mg.mg_create_grid(n)
    try:
        mg.mg_set_density(g, 0, -1, delta)
        with pytest.raises(mg.MGError):
            mg.mg_get_total_force(g, 0, -1, np.empty((3, n, n, n)))
        mg.mg_solve(g, 0, alpha, 1.0, 1e-11)
        phi = np.empty((n,) * 3)
        mg.mg_get_field(g, 0, -1, phi)
        st = mg.mg_solve_newton(g, COEF, 1e-11)
        assert st["rc"] == mg.MG_OK
        phi_after = np.empty((n,) * 3)
        mg.mg_get_field(g, 0, -1, phi_after)
        phin = np.empty((n,) * 3)
        mg.mg_get_newton_field(g, 0, -1, phin)
        total = np.empty((3, n, n, n))
        mg.mg_get_total_force(g, 0, -1, total)
        fifth = np.empty((3, n, n, n))
        mg.mg_get_force(g, 0, -1, fifth)
    finally:
        mg.mg_destroy_grid(g)
    assert np.array_equal(phi, phi_after)          # the scalar field is untouched
    ref, _ = O.fas_solve(delta, 0.0, COEF, tol=1e-12, max_cycles=200)
    assert rel(phin - phin.mean(), ref - ref.mean()) < 1e-10
    # total force = -1/2 grad (phi + 2 phi_N) = fifth force - grad phi_N
    want = O.force(phi + 2.0 * phin)
    assert np.abs(total - want).max() <= 1e-12 * np.abs(want).max()
    assert np.abs(total - (fifth + 2.0 * O.force(phin))).max() <= 1e-12 * np.abs(want).max()


def test_newton_potential_on_refinements():
    h = I.refined_hierarchy(16, 2.0, 5, thresholds=(15.0, 40.0))
    levels = [L for L in h["levels"] if len(L["origins"])]
    g = mg.mg_create_grid(16)
    gb = mg.mg_create_grid(16)
    try:
        for hh in (g, gb):
            mg.mg_set_density(hh, 0, -1, h["delta0"])
            for lvl, L in enumerate(levels, start=1):
                mg.mg_add_patches(hh, lvl, L["origins"])
                mg.mg_set_density(hh, lvl, -1, np.ascontiguousarray(L["delta"]))
        mg.mg_solve(g, 0, 0.3, 1.0, 1e-11)
        mg.mg_solve_newton(g, COEF, 1e-11)
        phin0 = np.empty((16,) * 3)
        mg.mg_get_newton_field(g, 0, -1, phin0)
        parent, parent_org = phin0, None
        for lvl, L in enumerate(levels, start=1):
            p = np.empty((len(L["origins"]), 8, 8, 8))
            mg.mg_get_newton_field(g, lvl, -1, p)
            d, _ = O.patch_residual(16, lvl, L["origins"], p, L["delta"], parent, 0.0, COEF,
                                    parent_org=parent_org)
            assert np.abs(d).max() < 1e-11, lvl
            parent, parent_org = p, L["origins"]
        # total force on level 1 = fifth force + 2 x (force of phi_N): grid gb solves
        # phi_N as its scalar field (alpha = 0, same coefficient)
        mg.mg_solve(gb, 0, 0.0, COEF, 1e-11)
        c1 = len(levels[0]["origins"])
        tot = np.empty((3, c1 * 512))
        mg.mg_get_total_force(g, 1, -1, tot)
        fifth = np.empty((3, c1 * 512))
        mg.mg_get_force(g, 1, -1, fifth)
        fn = np.empty((3, c1 * 512))
        mg.mg_get_force(gb, 1, -1, fn)
        scale = np.abs(tot).max()
        assert np.abs(tot - (fifth + 2.0 * fn)).max() <= 1e-9 * scale
    finally:
        mg.mg_destroy_grid(g)
        mg.mg_destroy_grid(gb)


def test_newton_rejects_batch_and_bad_input():
    g = mg.mg_create_grid(16)
    try:
        with pytest.raises(mg.MGError):
            mg.mg_solve_newton(g, COEF, 1e-8)          # density not set
        mg.mg_set_density(g, 0, -1, I.lognormal_delta(16, 1.0, 3))
        with pytest.raises(mg.MGError):
            mg.mg_solve_newton(g, float("nan"), 1e-8)
    finally:
        mg.mg_destroy_grid(g)
    b = mg.mg_create_batch([16, 16])
    try:
        with pytest.raises(mg.MGError):
            mg.mg_solve_newton(b, COEF, 1e-8)
    finally:
        mg.mg_destroy_grid(b)
