"""Full-size workloads against the CPU oracle by properties that hold at any size:
the oracle's own residual of the GPU fields (C3: 256^3 domain with two levels of
8^3 patches; C4: 512^3, mixed and FP64), and mixed against FP64."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1303_0008_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1303_0008_gb300 import mg  # noqa: E402

TOL = 1e-8


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_c3_refined_levels_full_size():
    """256^3 domain (sigma 2.0) with 72,167 level-1 and 4,449 level-2 patches and
    alpha*kappa = 1e-3.  The level-1 density reaches delta = 3382 with 10% noise at
    the cell scale; from alpha*kappa ~ 5e-3 up, alpha*kappa*delta ~ 16 there makes the
    linearised operator strongly anisotropic cell by cell and the FAS correction of
    the 8^3 -> 4^3 -> 2^3 union hierarchy diverges."""
    h = I.refined_hierarchy(256, 2.0, 1303)
    alpha = 1e-3
    l1, l2 = h["levels"]
    assert len(l1["origins"]) > 1000 and len(l2["origins"]) > 100
    g = mg.mg_create_grid(256)
    try:
        mg.mg_set_density(g, 0, -1, h["delta0"])
        for lvl, L in enumerate(h["levels"], start=1):
            mg.mg_add_patches(g, lvl, L["origins"])
            mg.mg_set_density(g, lvl, -1, np.ascontiguousarray(L["delta"]))
        st = mg.mg_solve(g, 0, alpha, 1.0, TOL)
        phi0 = np.empty_like(h["delta0"])
        mg.mg_get_field(g, 0, -1, phi0)
        p1 = np.empty((len(l1["origins"]), 8, 8, 8))
        p2 = np.empty((len(l2["origins"]), 8, 8, 8))
        mg.mg_get_field(g, 1, -1, p1)
        mg.mg_get_field(g, 2, -1, p2)
    finally:
        mg.mg_destroy_grid(g)
    d0, _ = O.residual(phi0, h["delta0"], alpha, 1.0)
    assert np.abs(d0 - d0.mean()).max() < TOL
    d1, _ = O.patch_residual(256, 1, l1["origins"], p1, l1["delta"], phi0, alpha, 1.0)
    assert np.abs(d1).max() < TOL
    d2, _ = O.patch_residual(256, 2, l2["origins"], p2, l2["delta"], p1, alpha, 1.0,
                             parent_org=l1["origins"])
    assert np.abs(d2).max() < TOL


def test_c4_512_mixed_and_fp64():
    n = 512
    delta = I.lognormal_delta(n, 2.0, 1304)
    alpha = I.alpha_kappa_for_rv(16.0)
    out = {}
    for prec in (1, 0):
        g = mg.mg_create_grid(n, mg.options(prec=prec))
        try:
            d = torch.from_numpy(delta).cuda()
            mg.mg_set_density(g, 0, -1, d)
            st = mg.mg_solve(g, 0, alpha, 1.0, TOL if prec else 1e-10)
            phi = np.empty_like(delta)
            mg.mg_get_field(g, 0, -1, phi)
            out[prec] = (st, phi)
        finally:
            mg.mg_destroy_grid(g)
    fl, hits = O.density_floor(delta, alpha, 1.0)
    assert out[1][0]["guard_hits"] == hits == out[0][0]["guard_hits"]
    for prec, tol in ((1, TOL), (0, 1e-10)):
        d, g = O.residual(out[prec][1], fl, alpha, 1.0)
        assert np.abs(d - d.mean()).max() < 1.5 * tol and g == 0
    # the mixed answer is the FP64 system's solution to the bound of the target
    assert rel(out[1][1], out[0][1]) < 1e-7
    assert rel(O.force(out[1][1]), O.force(out[0][1])) < 1e-7
