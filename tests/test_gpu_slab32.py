"""The FP32 correction sweep in staggered slabs of z planes (option slab32,
n >= 256): the same bits as four whole colour stages, for every slab thickness,
both branches, with and without CUDA graphs, and with the finest-level timing on."""
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


@pytest.mark.parametrize("n,sigma,rv,sign,slabs", [
    (256, 2.0, 16.0, 1.0, (8, 16, 32, 128)),
    (256, 1.5, 8.0, -1.0, (16,)),
    (512, 2.0, 16.0, 1.0, (16, 64)),
])
def test_slab_sweeps_give_the_bits_of_whole_colour_stages(n, sigma, rv, sign, slabs):
    delta = torch.from_numpy(I.lognormal_delta(n, sigma, 1304 + n)).cuda()
    alpha = sign * I.alpha_kappa_for_rv(rv)
    st0, phi0 = mixed_solve(delta, alpha, sign, slab32=0)
    assert st0["rc"] == mg.MG_OK
    for S in slabs:
        st1, phi1 = mixed_solve(delta, alpha, sign, slab32=S)
        assert st1["rc"] == mg.MG_OK
        assert (st0["cycles"], st0["outer"]) == (st1["cycles"], st1["outer"]), S
        assert st0["hist"] == st1["hist"], S
        assert torch.equal(phi0, phi1), S


def test_slab_sweeps_without_graphs_and_timed():
    n = 256
    delta = torch.from_numpy(I.lognormal_delta(n, 2.0, 1305)).cuda()
    alpha = I.alpha_kappa_for_rv(16.0)
    st0, phi0 = mixed_solve(delta, alpha, 1.0, slab32=0)
    st1, phi1 = mixed_solve(delta, alpha, 1.0, slab32=16, use_graphs=0, time_kernels=2)
    assert st1["rc"] == mg.MG_OK
    assert torch.equal(phi0, phi1)
    # one timed unit per finest smoothing call, each a whole sweep of n^3 cell updates
    assert st1["kernel_launches"] > 0
    assert st1["kernel_cells"] == st1["kernel_launches"] * n ** 3
    assert st1["kernel_ms"] > 0


def test_levels_without_a_slab_order_keep_whole_stages():
    """slab32 on a 128^3 grid (no level with n >= 256) changes nothing."""
    n = 128
    delta = torch.from_numpy(I.lognormal_delta(n, 1.5, 1306)).cuda()
    alpha = I.alpha_kappa_for_rv(8.0)
    st0, phi0 = mixed_solve(delta, alpha, 1.0, slab32=0)
    st1, phi1 = mixed_solve(delta, alpha, 1.0, slab32=16)
    assert st0["launches"] == st1["launches"]
    assert torch.equal(phi0, phi1)
