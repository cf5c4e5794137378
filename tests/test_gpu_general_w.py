"""General operator-splitting constant w (Sec. III.A-B): Sigma_ijk then involves
the cell's own value and each smoothing update is a full Newton step with the
Jacobian diagonal of Sec. III.B.  The discrete system itself does not depend on
w except through the periodic compatibility constant lambda: the solution at
any w satisfies the unsplit equation with a known lambda term, and matches the
oracle's at the same w."""
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


def solve(delta, alpha, kappa, tol, **opt):
    n = delta.shape[0]
    g = mg.mg_create_grid(n, mg.options(**opt))
    try:
        mg.mg_set_density(g, 0, -1, delta)
        st = mg.mg_solve(g, 0, alpha, kappa, tol, check=False)
        phi = np.empty((n,) * 3)
        mg.mg_get_field(g, 0, -1, phi)
    finally:
        mg.mg_destroy_grid(g)
    return st, phi


@pytest.mark.parametrize("n,w,rv,sign", [(32, 0.2, 8.0, 1.0), (32, 0.5, 8.0, -1.0),
                                         (48, 0.25, 4.0, 1.0), (24, 0.6, 2.0, 1.0)])
def test_general_w_matches_oracle_and_the_unsplit_equation(n, w, rv, sign):
    delta = I.lognormal_delta(n, 1.0, 500 + n)
    alpha = sign * I.alpha_kappa_for_rv(rv)
    st, phi = solve(delta, alpha, sign, 1e-11, w=w)
    assert st["rc"] == mg.MG_OK, st
    fl, _ = O.density_floor(delta, alpha, sign, w)
    ref, rs = O.fas_solve(fl, alpha, sign, tol=1e-12, max_cycles=200, w=w)
    assert rs["status"] == 0
    assert rel(phi, ref) < 1e-9
    d, g = O.residual(phi, fl, alpha, sign, w=w)
    assert np.abs(d - d.mean()).max() < 1e-10 and g == 0
    # the unsplit discrete equation with the known lambda term (the same identity
    # pins the oracle's general-w path)
    from test_oracle_pins import unsplit_lhs
    lhs, lap, _ = unsplit_lhs(phi, 1.0 / n, alpha)
    lam = st["lambda"]
    rhs = sign * fl + lam + alpha * (1 - w) * lam * (2 * lap - lam)
    assert np.abs(lhs - rhs).max() < 1e-8 * np.abs(sign * fl).max()


def test_general_w_rejected_where_not_built():
    delta = I.lognormal_delta(16, 1.0, 3)
    g = mg.mg_create_grid(16, mg.options(w=0.25, prec=mg.MG_MIXED))
    try:
        mg.mg_set_density(g, 0, -1, delta)
        with pytest.raises(mg.MGError):
            mg.mg_solve(g, 0, 0.3, 1.0, 1e-8)
        # the linear problem does not involve w
        assert mg.mg_solve(g, 0, 0.0, 1.0, 1e-8)["rc"] == mg.MG_OK
    finally:
        mg.mg_destroy_grid(g)
    with pytest.raises(mg.MGError):
        mg.mg_create_grid(16, mg.options(w=1.0))
    b = mg.mg_create_batch([16], mg.options(w=0.25))
    try:
        mg.mg_set_density(b, 0, 0, delta)
        with pytest.raises(mg.MGError):
            mg.mg_solve_batch(b, [0], [0.3], [1.0], 1e-8)
    finally:
        mg.mg_destroy_grid(b)
