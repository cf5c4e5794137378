"""CTA tiles of the FP32 colour stages (option tile32: 32 cells in x by 8/T rows
of the colour by T planes per 256-thread CTA, or 256 consecutive cells): every
shape updates every cell of the colour once with the same arithmetic, so the
solve gives the same bits."""
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


@pytest.mark.parametrize("n,sigma,rv,sign,tiles", [
    (64, 1.5, 8.0, 1.0, (1, 2, 4, 8)),
    (128, 2.0, 16.0, -1.0, (1, 4, 8)),
    (256, 2.0, 16.0, 1.0, (2, 4)),
    (512, 2.0, 16.0, 1.0, (4,)),
])
def test_every_tile_shape_gives_the_same_bits(n, sigma, rv, sign, tiles):
    delta = torch.from_numpy(I.lognormal_delta(n, sigma, 1330 + n)).cuda()
    alpha = sign * I.alpha_kappa_for_rv(rv)
    st0, phi0 = mixed_solve(delta, alpha, sign, tile32=0)
    for T in tiles:
        st1, phi1 = mixed_solve(delta, alpha, sign, tile32=T)
        assert (st0["cycles"], st0["outer"]) == (st1["cycles"], st1["outer"]), T
        assert st0["hist"] == st1["hist"], T
        assert torch.equal(phi0, phi1), T
