"""GPU parity of the mixed-precision solve (FP32 correction V-cycles in an FP64
defect-correction loop) against the FP64 CPU oracle, through the C-ABI.

The outer residual is FP64, so the converged field is the FP64 system's solution;
the stated bound is 1e-7 relative for phi and its gradient, and at tight
tolerances it reaches the FP64 bound of 1e-10.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1303_0008_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1303_0008_gb300 import mg  # noqa: E402


def solve(delta, alpha, kappa, branch=0, tol=1e-11, **opt):
    n = delta.shape[0]
    o = dict(prec=mg.MG_MIXED)
    o.update(opt)
    g = mg.mg_create_grid(n, mg.options(**o))
    try:
        mg.mg_set_stream(g, torch.cuda.current_stream())
        mg.mg_set_density(g, 0, -1, torch.from_numpy(delta).cuda())
        st = mg.mg_solve(g, branch, alpha, kappa, tol, check=False)
        phi = np.empty_like(delta)
        mg.mg_get_field(g, 0, -1, phi)
        force = np.empty((3,) + delta.shape)
        mg.mg_get_force(g, 0, -1, force)
    finally:
        mg.mg_destroy_grid(g)
    return phi, force, st


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_tophat_mixed_matches_oracle():
    w = I.workload_tophat(32)
    phi, force, st = solve(w["delta"], w["alpha"], w["kappa"], tol=1e-8)
    assert st["rc"] == mg.MG_OK and st["res"] < 1e-8
    ref, _ = O.fas_solve(w["delta"], w["alpha"], w["kappa"], tol=1e-12)
    assert rel(phi, ref) < 1e-7
    assert rel(force, O.force(ref)) < 1e-7
    phi, force, st = solve(w["delta"], w["alpha"], w["kappa"], tol=1e-11)
    assert st["rc"] == mg.MG_OK
    assert rel(phi, ref) < 1e-10 and rel(force, O.force(ref)) < 1e-10


@pytest.mark.parametrize("rv", [2.0, 8.0, 32.0])
@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_lognormal_mixed_matches_oracle(rv, sign):
    delta = I.lognormal_delta(32, 1.5, 1302)
    a = sign * I.alpha_kappa_for_rv(rv)
    phi, force, st = solve(delta, a, sign, tol=1e-10, max_cycles=60)
    assert st["rc"] == mg.MG_OK, st
    fl, hits = O.density_floor(delta, a, sign)
    ref, rst = O.fas_solve(fl, a, sign, tol=1e-12, max_cycles=300)
    assert rst["status"] == O.OK
    assert rel(phi, ref) < 1e-9
    assert rel(force, O.force(ref)) < 1e-9
    assert st["guard_hits"] == hits


@pytest.mark.parametrize("inner", [1, 2, 4])
def test_inner_cycle_counts_all_converge(inner):
    delta = I.lognormal_delta(32, 2.0, 1304)
    a = I.alpha_kappa_for_rv(16.0)
    phi, _, st = solve(delta, a, 1.0, tol=1e-9, inner_cycles=inner)
    assert st["rc"] == mg.MG_OK, st
    fl, _ = O.density_floor(delta, a, 1.0)
    ref, _ = O.fas_solve(fl, a, 1.0, tol=1e-12, max_cycles=300)
    assert rel(phi, ref) < 1e-8


def test_mixed_poisson_and_wrong_branch():
    n = 16
    delta = I.lognormal_delta(n, 1.0, 9)
    phi, _, st = solve(delta, 0.0, 1.0, tol=1e-11)
    ref, _ = O.fas_solve(delta, 0.0, 1.0, tol=1e-12)
    assert st["rc"] == mg.MG_OK and rel(phi, ref) < 1e-10
    phi, _, st = solve(np.zeros((n, n, n)), 0.3, 1.0, branch=-1, tol=1e-11)
    assert st["rc"] == mg.MG_OK
    assert st["lambda"] == pytest.approx(3 / (2 * 0.3), rel=1e-10)


def test_mixed_full_size_128_against_fp64_and_oracle_residual():
    w = I.workload_lognormal_sweep(128)
    delta = w["delta"]
    s = w["solves"][2]  # r_V = 8 cells, physical branch
    phi_m, force_m, st_m = solve(delta, s["alpha"], s["kappa"], tol=1e-8)
    assert st_m["rc"] == mg.MG_OK
    d, _ = O.residual(phi_m, delta, s["alpha"], s["kappa"])
    assert np.abs(d - d.mean()).max() < 1e-8
    g = mg.mg_create_grid(128)
    try:
        mg.mg_set_density(g, 0, -1, delta)
        st = mg.mg_solve(g, 0, s["alpha"], s["kappa"], 1e-10)
        phi_64 = np.empty_like(delta)
        mg.mg_get_field(g, 0, -1, phi_64)
    finally:
        mg.mg_destroy_grid(g)
    assert rel(phi_m, phi_64) < 1e-7
    assert rel(force_m, O.force(phi_64)) < 1e-7


def test_mixed_fused_coarse_subcycle_is_bit_identical():
    delta = I.lognormal_delta(64, 1.5, 8)
    a, _, s1 = solve(delta, 0.3, 1.0, tol=1e-10, fuse_coarse=1)
    b, _, s2 = solve(delta, 0.3, 1.0, tol=1e-10, fuse_coarse=0)
    assert s1["rc"] == s2["rc"] == mg.MG_OK
    assert np.array_equal(a, b) and s1["hist"] == s2["hist"]
