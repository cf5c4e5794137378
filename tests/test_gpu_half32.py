"""The FP32 correction sweep as two half sweeps (option half32, n = 256 and 512):
the same bits as the four per-colour launches, and a bounded wait for its
asynchronous copies that reports MG_ETIMEOUT and leaves the handle usable."""
import numpy as np
import pytest

from paper_1303_0008_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1303_0008_gb300 import mg  # noqa: E402


def mixed_solve(delta, alpha, kappa, tol=1e-8, **opt):
    n = delta.shape[0]
    g = mg.mg_create_grid(n, mg.options(prec=mg.MG_MIXED, **opt))
    try:
        mg.mg_set_density(g, 0, -1, delta)
        st = mg.mg_solve(g, 0, alpha, kappa, tol)
        phi = torch.empty_like(delta)
        mg.mg_get_field(g, 0, -1, phi)
    finally:
        mg.mg_destroy_grid(g)
    return st, phi


@pytest.mark.parametrize("n,sigma,rv,sign", [(256, 2.0, 16.0, 1.0), (256, 1.5, 8.0, -1.0),
                                             (512, 2.0, 16.0, 1.0)])
def test_half_sweeps_give_the_bits_of_the_per_colour_launches(n, sigma, rv, sign):
    delta = torch.from_numpy(I.lognormal_delta(n, sigma, 1304 + n)).cuda()
    alpha = sign * I.alpha_kappa_for_rv(rv)
    st0, phi0 = mixed_solve(delta, alpha, sign, half32=0)
    st1, phi1 = mixed_solve(delta, alpha, sign, half32=1)
    assert st0["rc"] == st1["rc"] == mg.MG_OK
    assert (st0["cycles"], st0["outer"]) == (st1["cycles"], st1["outer"])
    assert st0["hist"] == st1["hist"]
    assert torch.equal(phi0, phi1)


def test_a_wait_that_runs_out_reports_etimeout_and_the_handle_stays_usable():
    """barrier_timeout_s = 0 accepts only copies that have already landed: the
    first waits of the half sweeps run out, the kernels record it and return, and
    the solve returns MG_ETIMEOUT.  A solve on the same handle with the default
    limit then converges to the answer of a fresh handle."""
    n = 256
    delta = torch.from_numpy(I.lognormal_delta(n, 1.5, 77)).cuda()
    alpha = I.alpha_kappa_for_rv(8.0)
    g = mg.mg_create_grid(n, mg.options(prec=mg.MG_MIXED, half32=1, barrier_timeout_s=0.0))
    try:
        mg.mg_set_density(g, 0, -1, delta)
        st = mg.mg_solve(g, 0, alpha, 1.0, 1e-8, check=False)
        assert st["rc"] == mg.MG_ETIMEOUT
        assert "barrier_timeout_s" in mg.mg_last_error()
        opt = mg.mg_get_options(g)
        opt.barrier_timeout_s = 1.0
        mg.mg_set_options(g, opt)
        mg.mg_set_field(g, 0, -1, torch.zeros_like(delta))   # the field is undefined now
        st = mg.mg_solve(g, 0, alpha, 1.0, 1e-8)
        phi = torch.empty_like(delta)
        mg.mg_get_field(g, 0, -1, phi)
    finally:
        mg.mg_destroy_grid(g)
    ref_st, ref = mixed_solve(delta, alpha, 1.0, half32=1)
    assert st["rc"] == mg.MG_OK and st["hist"] == ref_st["hist"]
    assert torch.equal(phi, ref)
