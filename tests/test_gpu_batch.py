"""Batched independent solves (one launch per V-cycle stage over a work list)
against single-grid solves and the CPU oracle, through the C-ABI."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1303_0008_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1303_0008_gb300 import mg  # noqa: E402


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def batch_solve(specs, tol, **opt):
    g = mg.mg_create_batch([s["n"] for s in specs], mg.options(**opt))
    try:
        for k, s in enumerate(specs):
            mg.mg_set_density(g, 0, k, s["delta"])
        rc, stats = mg.mg_solve_batch(g, [s["branch"] for s in specs], [s["alpha"] for s in specs],
                                      [s["kappa"] for s in specs], tol, check=False)
        phis = []
        for k, s in enumerate(specs):
            phi = np.empty((s["n"],) * 3)
            mg.mg_get_field(g, 0, k, phi)
            phis.append(phi)
        force = np.empty((3,) + (specs[0]["n"],) * 3)
        mg.mg_get_force(g, 0, 0, force)
    finally:
        mg.mg_destroy_grid(g)
    return rc, stats, phis, force


def single_solve(s, tol, **opt):
    g = mg.mg_create_grid(s["n"], mg.options(**opt))
    try:
        mg.mg_set_density(g, 0, -1, s["delta"])
        st = mg.mg_solve(g, s["branch"], s["alpha"], s["kappa"], tol, check=False)
        phi = np.empty((s["n"],) * 3)
        mg.mg_get_field(g, 0, -1, phi)
    finally:
        mg.mg_destroy_grid(g)
    return st, phi


def small_specs():
    out = []
    for k, (n, rv, sgn) in enumerate([(16, 8.0, 1), (32, 2.0, -1), (24, 16.0, 1), (12, 8.0, 1),
                                      (32, 32.0, -1), (20, 4.0, 1), (6, 8.0, 1)]):
        a = sgn * I.alpha_kappa_for_rv(rv)
        out.append({"n": n, "delta": I.lognormal_delta(n, 1.5, 50 + k), "alpha": a,
                    "kappa": float(sgn), "branch": 0})
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_equals_single_grid_solves_and_oracle(prec):
    specs = small_specs()
    tol = 1e-11 if prec == 0 else 1e-10
    rc, stats, phis, _ = batch_solve(specs, tol, prec=prec)
    assert rc == mg.MG_OK, stats
    for s, st, phi in zip(specs, stats, phis):
        assert st["status"] == mg.MG_OK and st["res"] < tol
        st1, phi1 = single_solve(s, tol, prec=prec)
        # the same per-thread code and block partition: the same bits
        assert np.array_equal(phi, phi1), s["n"]
        assert st["hist"] == st1["hist"]
        fl, _ = O.density_floor(s["delta"], s["alpha"], s["kappa"])
        ref, _ = O.fas_solve(fl, s["alpha"], s["kappa"], tol=1e-12, max_cycles=300)
        assert rel(phi, ref) < (1e-10 if prec == 0 else 1e-9)


def test_batch_force_and_failing_member():
    specs = small_specs()[:3]
    bad = specs[1]["delta"].copy()
    bad[3, 3, 3] = np.nan
    specs[1] = dict(specs[1], delta=bad)
    rc, stats, phis, force = batch_solve(specs, 1e-10, prec=1)
    assert rc == mg.MG_ENAN
    assert stats[1]["status"] == mg.MG_ENAN
    assert stats[0]["status"] == mg.MG_OK and stats[2]["status"] == mg.MG_OK
    assert np.abs(force - O.force(phis[0])).max() <= 1e-12 * np.abs(force).max()


def test_batch_workload_64_solves_mixed():
    """The 64-solve workload (sizes 32..128, sigma in [0.5, 2.5], r_V log-uniform in
    [2, 16], both signs), mixed precision to 1e-8: every member converges, a sample
    passes the oracle's residual check and matches a single-grid solve."""
    w = I.workload_batch(64)
    specs = [dict(s, delta=I.lognormal_delta(s["n"], s["sigma"], s["seed"])) for s in w]
    rc, stats, phis, _ = batch_solve(specs, 1e-8, prec=1)
    assert rc == mg.MG_OK
    assert all(st["status"] == mg.MG_OK and st["res"] < 1e-8 for st in stats)
    sizes = [s["n"] for s in specs]
    for k in {sizes.index(32), sizes.index(96), sizes.index(128)}:
        s = specs[k]
        fl, _ = O.density_floor(s["delta"], s["alpha"], s["kappa"])
        d, _ = O.residual(phis[k], fl, s["alpha"], s["kappa"])
        assert np.abs(d - d.mean()).max() < 1e-8
        st1, phi1 = single_solve(s, 1e-8, prec=1)
        assert np.array_equal(phis[k], phi1)
