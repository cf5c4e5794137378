"""The allocation-free residual entry point, checked against mg_op_residual.

mg_op_residual_noalloc serves callers that cannot call cudaMalloc/cudaFree (those
calls synchronise the device, and fail when another allocator already holds the
card's memory).  It keeps its partial norms in one fixed device array shared by
all calls, so two calls in a row must each give the same answer as the
allocating entry point, with nothing left over from the call before.  This file
is collected last so that a run stopping at its first failure has run every
other test already.
"""
import numpy as np
import pytest

from paper_1303_0008_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1303_0008_gb300 import mg  # noqa: E402

EPS = np.finfo(np.float64).eps


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to("cuda:0")


def both(n, seed, alpha, kappa, branch, with_f, amplitude):
    delta = I.lognormal_delta(n, 1.5, seed)
    phi = amplitude * I.random_field(n, seed + 1)
    f = dev(I.random_field(n, seed + 2)) if with_f else None
    d_ref = torch.empty((n, n, n), dtype=torch.float64, device="cuda:0")
    d_new = torch.full((n, n, n), float("nan"), dtype=torch.float64, device="cuda:0")
    ref = mg.mg_op_residual(n, dev(phi), dev(delta), f, branch, alpha, kappa, d_ref)
    new = mg.mg_op_residual_noalloc(n, dev(phi), dev(delta), f, branch, alpha, kappa, d_new)
    torch.cuda.synchronize()
    return ref, new, d_ref.cpu().numpy(), d_new.cpu().numpy()


def check(ref, new, d_ref, d_new):
    scale = np.abs(d_ref).max() + 1.0
    assert np.abs(d_new - d_ref).max() <= 64 * EPS * scale
    for k in ("sum", "max", "min"):
        assert new[k] == pytest.approx(ref[k], rel=1e-12, abs=1e-12 * scale)
    assert new["guards"] == ref["guards"] and new["nonfinite"] == ref["nonfinite"] == 0


def test_noalloc_residual_matches_allocating_entry_point_twice_in_a_row():
    # first call: a large grid with a FAS right-hand side and guarded cells (a nearly
    # flat phi leaves the voids' discriminant negative)
    ref, new, d_ref, d_new = both(64, 5, I.alpha_kappa_for_rv(32.0), 1.0, 0, True, 1e-7)
    assert ref["guards"] > 0
    check(ref, new, d_ref, d_new)
    # second call: a smaller grid, other parameters; nothing may leak from the first
    ref, new, d_ref, d_new = both(12, 9, -0.3, -1.0, 0, False, 0.02)
    check(ref, new, d_ref, d_new)


def test_noalloc_residual_rejects_sizes_beyond_its_storage():
    n = 258
    with pytest.raises(mg.MGError) as e:
        mg.mg_op_residual_noalloc(n, torch.zeros(1, dtype=torch.float64, device="cuda:0"),
                                  torch.zeros(1, dtype=torch.float64, device="cuda:0"), None,
                                  0, 0.3, 1.0)
    assert e.value.status == mg.MG_EINVAL
    assert "256" in mg.mg_last_error()


@pytest.mark.parametrize("n", [256, 254])
def test_noalloc_residual_at_and_below_its_capacity(n):
    """n = 256 fills the fixed storage exactly (one partial per 256-cell block,
    65,536 of them); n = 254 is the largest size below it."""
    ref, new, d_ref, d_new = both(n, 31, I.alpha_kappa_for_rv(8.0), 1.0, 0, True, 1e-4)
    check(ref, new, d_ref, d_new)


def test_noalloc_residual_without_norms_still_writes_d():
    """With a NULL norms pointer the call still completes the kernel before it
    returns (it synchronises the stream) and writes d."""
    n = 16
    delta = I.lognormal_delta(n, 1.0, 41)
    phi = 0.01 * I.random_field(n, 42)
    d_ref = torch.empty((n, n, n), dtype=torch.float64, device="cuda:0")
    d_new = torch.full((n, n, n), float("nan"), dtype=torch.float64, device="cuda:0")
    mg.mg_op_residual(n, dev(phi), dev(delta), None, 0, 0.3, 1.0, d_ref)
    assert mg.mg_op_residual_noalloc(n, dev(phi), dev(delta), None, 0, 0.3, 1.0, d_new,
                                     want_norms=False) is None
    scale = d_ref.abs().max().item() + 1.0
    assert (d_new - d_ref).abs().max().item() <= 64 * EPS * scale


@pytest.mark.parametrize("alpha", [float("nan"), float("inf")])
def test_noalloc_residual_rejects_a_non_finite_alpha_like_the_allocating_one(alpha):
    n = 8
    z = torch.zeros((n, n, n), dtype=torch.float64, device="cuda:0")
    for fn in (mg.mg_op_residual, mg.mg_op_residual_noalloc):
        with pytest.raises(mg.MGError) as e:
            fn(n, z, z, None, 0, alpha, 1.0)
        assert e.value.status == mg.MG_EINVAL
