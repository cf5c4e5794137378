"""The native autotuner: picks converging sweep counts, caches them by grid size,
precision and device, and leaves the caller's field untouched."""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1303_0008_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1303_0008_gb300 import mg  # noqa: E402


@pytest.mark.parametrize("prec", [0, 1])
def test_autotune_picks_caches_and_restores(tmp_path, prec):
    n = 32
    delta = I.lognormal_delta(n, 1.5, 1302)
    a = I.alpha_kappa_for_rv(8.0)
    cache = str(tmp_path / "tune.json")
    g = mg.mg_create_grid(n, mg.options(prec=prec))
    try:
        mg.mg_set_density(g, 0, -1, delta)
        phi0 = 1e-3 * I.random_field(n, 3)
        mg.mg_set_field(g, 0, -1, phi0)
        best, t = mg.mg_autotune(g, 0, a, 1.0, 1e-10, cache, use_cache=False)
        assert t > 0 and 1 <= best.nu_pre <= 5 and 1 <= best.nu_post <= 5
        assert abs(best.nu_pre - best.nu_post) <= 1
        back = np.empty((n, n, n))
        mg.mg_get_field(g, 0, -1, back)
        assert np.array_equal(back, phi0)                       # the caller's field
        data = json.load(open(cache))
        key = [k for k in data if k.startswith(f"n={n},prec={'mixed' if prec else 'fp64'}")]
        assert len(key) == 1 and data[key[0]]["nu_pre"] == best.nu_pre
        # a cached choice is applied without trials
        again, t2 = mg.mg_autotune(g, 0, a, 1.0, 1e-10, cache, use_cache=True)
        assert mg.options_dict(again) == mg.options_dict(best)
        assert mg.options_dict(mg.mg_get_options(g))["nu_post"] == best.nu_post
        st = mg.mg_solve(g, 0, a, 1.0, 1e-11)
        phi = np.empty((n, n, n))
        mg.mg_get_field(g, 0, -1, phi)
    finally:
        mg.mg_destroy_grid(g)
    ref, _ = O.fas_solve(delta, a, 1.0, tol=1e-12)
    assert np.abs(phi - ref).max() / np.abs(ref).max() < 1e-10


def test_autotune_tries_the_fp32_sweep_shapes_at_256(tmp_path):
    """From n = 256 the mixed tuner's second stage times the FP32 sweep shapes (CTA
    tiles, slabs, half sweeps) at the first stage's counts; the choice is a valid
    shape, is cached with the counts, and the solve it gives meets the tolerance."""
    n = 256
    delta = torch.from_numpy(I.lognormal_delta(n, 1.5, 1340)).cuda()
    a = I.alpha_kappa_for_rv(8.0)
    cache = str(tmp_path / "tune256.json")
    g = mg.mg_create_grid(n, mg.options(prec=mg.MG_MIXED))
    try:
        mg.mg_set_density(g, 0, -1, delta)
        best, t = mg.mg_autotune(g, 0, a, 1.0, 1e-8, cache, use_cache=False)
        assert t > 0
        assert best.tile32 in (0, 1, 2, 4, 8)
        assert best.slab32 in (0, 8, 16, 32, 64)
        assert best.half32 in (0, 1)
        assert not (best.half32 and best.slab32)
        entry = list(json.load(open(cache)).values())[0]
        for k in ("nu_pre", "nu_post", "inner_cycles", "half32", "slab32", "tile32"):
            assert entry[k] == getattr(best, k), k
        again, _ = mg.mg_autotune(g, 0, a, 1.0, 1e-8, cache, use_cache=True)
        assert mg.options_dict(again) == mg.options_dict(best)
        mg.mg_set_field(g, 0, -1, torch.zeros_like(delta))
        st = mg.mg_solve(g, 0, a, 1.0, 1e-8)
        assert st["rc"] == mg.MG_OK and st["res"] < 1e-8
    finally:
        mg.mg_destroy_grid(g)
