"""The one-launch four-colour FP32 sweep and the two-cells-per-thread colour stage (z-marching wavefront, packed FP32x2
arithmetic) against the per-colour launches: the same cell updates in the same
order with the same roundings, so mixed-precision solves must agree bit for
bit, histories included.  Sizes cover ragged 64 x 16 tiles (n = 40, 96), grids
narrower than one tile window (n = 32, 40), and plane runs of every length."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1303_0008_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1303_0008_gb300 import mg  # noqa: E402


def mixed_solve(delta, alpha, kappa, tol, **opt):
    n = delta.shape[0]
    g = mg.mg_create_grid(n, mg.options(prec=mg.MG_MIXED, **opt))
    try:
        mg.mg_set_density(g, 0, -1, delta)
        st = mg.mg_solve(g, 0, alpha, kappa, tol, check=False)
        phi = np.empty((n,) * 3)
        mg.mg_get_field(g, 0, -1, phi)
    finally:
        mg.mg_destroy_grid(g)
    return st, phi


CASES = [(32, 8.0, 1.0), (40, 4.0, -1.0), (64, 16.0, 1.0), (96, 8.0, -1.0), (128, 2.0, 1.0),
         (64, 0.0, 1.0)]


@pytest.mark.parametrize("n,rv,sign", CASES)
def test_sweep32_matches_per_colour_launches_bitwise(n, rv, sign):
    delta = I.lognormal_delta(n, 1.5, 900 + n)
    alpha = sign * I.alpha_kappa_for_rv(rv) if rv > 0 else 0.0
    st1, phi1 = mixed_solve(delta, alpha, sign, 1e-10, sweep32=1)
    st0, phi0 = mixed_solve(delta, alpha, sign, 1e-10, sweep32=0)
    assert st0["rc"] == mg.MG_OK and st1["rc"] == mg.MG_OK
    assert st1["hist"] == st0["hist"]
    assert np.array_equal(phi1, phi0)


@pytest.mark.parametrize("pre,post", [(1, 1), (3, 2), (2, 3)])
def test_sweep32_odd_sweep_counts(pre, post):
    n = 64
    delta = I.lognormal_delta(n, 2.0, 77)
    alpha = I.alpha_kappa_for_rv(8.0)
    st1, phi1 = mixed_solve(delta, alpha, 1.0, 1e-9, sweep32=1, nu_pre=pre, nu_post=post)
    st0, phi0 = mixed_solve(delta, alpha, 1.0, 1e-9, sweep32=0, nu_pre=pre, nu_post=post)
    assert st1["rc"] == mg.MG_OK
    assert st1["hist"] == st0["hist"]
    assert np.array_equal(phi1, phi0)


def test_sweep32_solution_against_oracle():
    n = 96
    delta = I.lognormal_delta(n, 1.5, 31)
    alpha = I.alpha_kappa_for_rv(8.0)
    st, phi = mixed_solve(delta, alpha, 1.0, 1e-10, sweep32=1)
    assert st["rc"] == mg.MG_OK
    fl, _ = O.density_floor(delta, alpha, 1.0)
    d, _ = O.residual(phi, fl, alpha, 1.0)
    assert np.abs(d - d.mean()).max() < 1e-10


def test_sweep32_option_is_validated():
    with pytest.raises(mg.MGError):
        mg.mg_create_grid(32, mg.options(sweep32=2))


@pytest.mark.parametrize("n,rv,sign", [(32, 8.0, 1.0), (40, 4.0, -1.0), (96, 8.0, -1.0),
                                       (128, 32.0, 1.0), (64, 0.0, 1.0)])
def test_pair32_matches_one_cell_per_thread_bitwise(n, rv, sign):
    """Two cells of a row per thread (packed FP32x2) against one cell per thread."""
    delta = I.lognormal_delta(n, 1.5, 700 + n)
    alpha = sign * I.alpha_kappa_for_rv(rv) if rv > 0 else 0.0
    st1, phi1 = mixed_solve(delta, alpha, sign, 1e-10, pair32=1)
    st0, phi0 = mixed_solve(delta, alpha, sign, 1e-10, pair32=0)
    assert st0["rc"] == mg.MG_OK and st1["rc"] == mg.MG_OK
    assert st1["hist"] == st0["hist"]
    assert np.array_equal(phi1, phi0)
