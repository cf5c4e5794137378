"""Truncation-error stopping rule of Sec. III.C: with tau_stop > 0 a domain
solve also stops once max|d - lambda| <= tau_stop * max|tau - mean tau|, where
tau = L^H(R phi) - R L^h(phi) at the iterate of the check; checked against the
same estimate built from the oracle's operators."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1303_0008_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1303_0008_gb300 import mg  # noqa: E402


def solve(delta, alpha, tol, **opt):
    n = delta.shape[0]
    g = mg.mg_create_grid(n, mg.options(**opt))
    try:
        mg.mg_set_density(g, 0, -1, delta)
        st = mg.mg_solve(g, 0, alpha, 1.0, tol)
        phi = np.empty((n,) * 3)
        mg.mg_get_field(g, 0, -1, phi)
    finally:
        mg.mg_destroy_grid(g)
    return st, phi


@pytest.mark.parametrize("rv", [0.0, 8.0])
def test_tau_stop_stops_at_the_truncation_error(rv):
    n = 64
    delta = I.lognormal_delta(n, 1.5, 77)
    alpha = I.alpha_kappa_for_rv(rv) if rv else 0.0
    st, phi = solve(delta, alpha, 1e-14, tau_stop=1.0 / 3.0, max_cycles=60)
    tight, _ = solve(delta, alpha, 1e-12)
    assert st["rc"] == mg.MG_OK and st["tau"] > 0.0
    assert st["res"] <= st["tau"] / 3.0
    assert st["cycles"] < tight["cycles"]
    # the same estimate from the oracle at the returned iterate (the solve stopped
    # at the check, so phi is the iterate the estimate was taken at)
    fl, _ = O.density_floor(delta, alpha, 1.0)
    dh, _ = O.residual(phi, fl, alpha, 1.0)
    dH, _ = O.residual(O.restrict(phi), O.restrict(fl), alpha, 1.0)
    tau = dH - O.restrict(dh)
    want = np.abs(tau - tau.mean()).max()
    assert abs(st["tau"] - want) <= 1e-6 * want


def test_tau_stop_off_changes_nothing():
    delta = I.lognormal_delta(32, 1.5, 78)
    a, pa = solve(delta, 0.3, 1e-10)
    b, pb = solve(delta, 0.3, 1e-10, tau_stop=0.0)
    assert a["hist"] == b["hist"] and b["tau"] == 0.0
    assert np.array_equal(pa, pb)
