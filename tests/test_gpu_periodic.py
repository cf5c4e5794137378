"""GPU parity of the periodic FP64 path against the CPU oracle, through the C-ABI.

Kernel-level checks compare each CUDA step with the oracle element by element on
the same seeded inputs; solve-level checks compare converged fields (relative
max-norm 1e-10, the FP64 target) and, at the full 128^3 size, evaluate the
oracle's own residual on the GPU solution.
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

DEV = "cuda:0"
EPS = np.finfo(np.float64).eps


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def colours(n):
    i = np.arange(n)
    K, J, Ii = np.meshgrid(i, i, i, indexing="ij")
    return ((Ii + K) & 1) + 2 * ((J + K) & 1)


def op_scale(phi, n):
    """Magnitude of the terms that enter the residual of each cell."""
    s = np.zeros_like(phi)
    for ax in range(3):
        s += np.abs(np.roll(phi, 1, ax)) + np.abs(np.roll(phi, -1, ax))
    return (s + 6 * np.abs(phi)) * n * n


CASES = [  # (alpha, kappa, branch)
    (0.3, 1.0, 0), (-0.3, -1.0, 0), (0.3, 1.0, -1), (0.0, 1.0, 0),
    (I.alpha_kappa_for_rv(2.0), 1.0, 0), (I.alpha_kappa_for_rv(32.0), 1.0, 0), (5e-5, 1.0, 0),
]


# ---------------------------------------------------------------------------
# kernel level
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [8, 24, 32])
@pytest.mark.parametrize("alpha,kappa,branch", CASES)
def test_residual_kernel_matches_oracle(n, alpha, kappa, branch):
    delta = I.lognormal_delta(n, 1.5, 100 + n)
    phi = 0.02 * I.random_field(n, 7 + n) + 0.05 * np.sin(2 * np.pi * (np.arange(n) + 0.5) / n)
    ref, g_ref = O.residual(phi, delta, alpha, kappa, branch)
    d = torch.empty((n, n, n), dtype=torch.float64, device=DEV)
    norms = mg.mg_op_residual(n, dev(phi), dev(delta), None, branch, alpha, kappa, d)
    got = host(d)
    tol = 64 * EPS * (op_scale(phi, n) + np.abs(ref) + np.abs(kappa * delta) + 1.0)
    # the oracle evaluates the root in the paper's form, which cancels to about
    # eps * |alpha_paper| = eps / |alpha| in absolute terms
    tol += 8 * EPS / abs(alpha) if alpha else 0.0
    assert (np.abs(got - ref) <= tol).all(), np.abs(got - ref).max()
    assert norms["guards"] == g_ref
    assert norms["nonfinite"] == 0
    assert abs(norms["sum"] - ref.sum()) <= 1e-12 * np.abs(ref).sum()
    assert norms["max"] == pytest.approx(ref.max(), rel=1e-12, abs=1e-9)
    assert norms["min"] == pytest.approx(ref.min(), rel=1e-12, abs=1e-9)


def test_residual_kernel_with_fas_rhs_and_ragged_sizes():
    for n in (6, 10, 12, 20):
        delta = I.lognormal_delta(n, 1.0, n)
        phi = 0.01 * I.random_field(n, 3 * n)
        f = I.random_field(n, 5 * n)
        ref, _ = O.residual(phi, delta, 0.3, 1.0, 0, f=f)
        d = torch.empty((n, n, n), dtype=torch.float64, device=DEV)
        mg.mg_op_residual(n, dev(phi), dev(delta), dev(f), 0, 0.3, 1.0, d)
        tol = 64 * EPS * (op_scale(phi, n) + np.abs(ref) + np.abs(f) + 1.0)
        assert (np.abs(host(d) - ref) <= tol).all()


def test_residual_flags_non_finite():
    n = 8
    delta = np.zeros((n, n, n))
    delta[3, 4, 5] = np.nan
    norms = mg.mg_op_residual(n, dev(np.zeros((n, n, n))), dev(delta), None, 0, 0.3, 1.0)
    assert norms["nonfinite"] == 1


@pytest.mark.parametrize("alpha,kappa,branch", CASES[:4])
def test_colour_sweep_solves_each_colour_exactly(alpha, kappa, branch):
    """After one four-colour sweep the cells of the last colour satisfy their own
    equation L^h phi = f + lambda (their 18 neighbours are of other colours and
    did not move afterwards): the oracle's residual there equals lambda."""
    n = 16
    delta = I.lognormal_delta(n, 1.5, 11)
    phi0 = 0.01 * I.random_field(n, 12)
    f = 0.5 * I.random_field(n, 13)
    lam = 0.37
    t = dev(phi0)
    mg.mg_op_smooth(n, t, dev(delta), dev(f), branch, alpha, kappa, lam, 1)
    got = host(t)
    d, _ = O.residual(got, delta, alpha, kappa, branch, f=f)
    last = colours(n) == 3
    tol = 64 * EPS * (op_scale(got, n) + np.abs(f) + np.abs(kappa * delta) + 1.0)
    assert (np.abs(d - lam)[last] <= tol[last]).all()
    assert (np.abs(d - lam)[~last] > 1e-6).mean() > 0.5   # the other colours moved since


def test_four_colour_sweeps_reach_the_bordered_fixed_point():
    """With lambda fixed at the oracle's compatibility constant, plain four-colour
    sweeps converge to the oracle's solution (up to the constant mode, which the
    sweeps leave free)."""
    n = 8
    delta = I.lognormal_delta(n, 1.0, 21)
    ref, rst = O.fas_solve(delta, 0.3, 1.0, tol=1e-13)
    phi_gpu = dev(np.zeros((n, n, n)))
    mg.mg_op_smooth(n, phi_gpu, dev(delta), None, 0, 0.3, 1.0, rst["lambda"], 300)
    got = host(phi_gpu)
    assert np.abs((got - got.mean()) - ref).max() < 1e-9 * np.abs(ref).max()
    lex = O.gs_sweeps(np.zeros((n, n, n)), delta, 0.3, 1.0, lam=rst["lambda"], sweeps=300)
    assert np.abs((lex - lex.mean()) - ref).max() < 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("n", [8, 12, 34])
def test_restriction_is_bit_exact(n):
    x = I.random_field(n, n)
    c = torch.empty((n // 2,) * 3, dtype=torch.float64, device=DEV)
    mg.mg_op_restrict(n, dev(x), c)
    assert np.array_equal(host(c), O.restrict(x))


@pytest.mark.parametrize("n", [8, 12, 34])
def test_prolongation_matches_oracle(n):
    nc = n // 2
    a, b = I.random_field(nc, 1), I.random_field(nc, 2)
    fine = I.random_field(n, 3)
    t = dev(fine)
    mg.mg_op_prolong_correct(n, dev(a), dev(b), t)
    ref = O.prolong_add(a - b, fine)
    assert np.abs(host(t) - ref).max() <= 8 * EPS * (np.abs(fine).max() + 2)


@pytest.mark.parametrize("n", [8, 20, 32])
def test_force_matches_oracle(n):
    phi = I.random_field(n, 4 * n)
    out = torch.empty((3, n, n, n), dtype=torch.float64, device=DEV)
    mg.mg_op_force(n, dev(phi), out)
    ref = O.force(phi)
    assert np.abs(host(out) - ref).max() <= 4 * EPS * n * np.abs(phi).max()


# ---------------------------------------------------------------------------
# full solves
# ---------------------------------------------------------------------------
def gpu_solve(delta, alpha, kappa, branch=0, tol=1e-11, phi0=None, on_device=True, **opt):
    n = delta.shape[0]
    g = mg.mg_create_grid(n, mg.options(**opt))
    try:
        mg.mg_set_stream(g, torch.cuda.current_stream())
        mg.mg_set_density(g, 0, -1, dev(delta) if on_device else np.ascontiguousarray(delta))
        if phi0 is not None:
            mg.mg_set_field(g, 0, -1, dev(phi0))
        st = mg.mg_solve(g, branch, alpha, kappa, tol, check=False)
        phi = np.empty((n, n, n))
        mg.mg_get_field(g, 0, -1, phi)
        force = np.empty((3, n, n, n))
        mg.mg_get_force(g, 0, -1, force)
    finally:
        mg.mg_destroy_grid(g)
    return phi, force, st


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def floored(delta, alpha, kappa):
    """The density the default guard (MG_GUARD_FLOOR) solves with, from the oracle."""
    return O.density_floor(delta, alpha, kappa)


def test_tophat_32_matches_oracle():
    w = I.workload_tophat(32)
    phi, force, st = gpu_solve(w["delta"], w["alpha"], w["kappa"])
    assert st["rc"] == mg.MG_OK and st["res"] < 1e-11
    ref, rst = O.fas_solve(w["delta"], w["alpha"], w["kappa"], tol=1e-11)
    assert rel(phi, ref) < 1e-10
    assert rel(force, O.force(ref)) < 1e-10
    assert st["lambda"] == pytest.approx(rst["lambda"], rel=1e-8)
    assert 5 <= st["cycles"] <= 25


@pytest.mark.parametrize("alpha,kappa", [(a * s, s) for a in (I.alpha_kappa_for_rv(2.0),
                                                                I.alpha_kappa_for_rv(8.0),
                                                                I.alpha_kappa_for_rv(32.0))
                                          for s in (1.0, -1.0)])
def test_lognormal_32_both_branches_match_oracle(alpha, kappa):
    delta = I.lognormal_delta(32, 1.5, 1302)
    phi, force, st = gpu_solve(delta, alpha, kappa, max_cycles=300)
    assert st["rc"] == mg.MG_OK, st
    fl, hits = floored(delta, alpha, kappa)
    ref, rst = O.fas_solve(fl, alpha, kappa, tol=1e-11, max_cycles=300)
    assert rst["status"] == O.OK
    assert rel(phi, ref) < 1e-10
    assert rel(force, O.force(ref)) < 1e-10
    assert st["guard_hits"] == hits
    assert rst["guard_hits"] == 0


@pytest.mark.parametrize("n,sigma,rv", [(16, 1.5, 16.0), (16, 1.5, 32.0), (32, 1.5, 12.0),
                                         (32, 1.0, 16.0)])
def test_root_guard_reading_matches_oracle(n, sigma, rv):
    """The real-part reading of a negative discriminant (MG_GUARD_ROOT) on grids
    where its iteration still converges (found with the oracle; at r_V >= 12 cells
    about half of the cells have a negative discriminant there).  The guarded
    system is not smooth where q = 0 and need not have one solution: at 32^3,
    sigma 1.5, r_V = 20 cells the GPU and the oracle both converge, to fields 8e-4
    apart, and at 64^3, sigma 1.0, r_V = 16 the oracle converges where the GPU's
    iteration stalls, so neither is a parity case."""
    delta = I.lognormal_delta(n, sigma, 1302)
    a = I.alpha_kappa_for_rv(rv)
    phi, _, st = gpu_solve(delta, a, 1.0, max_cycles=300, guard=mg.MG_GUARD_ROOT)
    assert st["rc"] == mg.MG_OK, st
    ref, rst = O.fas_solve(delta, a, 1.0, tol=1e-11, max_cycles=300)
    assert rst["status"] == O.OK
    assert rel(phi, ref) < 1e-10
    assert st["guard_hits"] == rst["guard_hits"] > 0


def test_lognormal_128_full_size_oracle_residual_and_symmetry():
    """The full 128^3 workload: the oracle's residual of each GPU solution is below
    tol, the sign flip of (alpha, kappa) is odd, and one pair is compared with a full
    oracle solve."""
    w = I.workload_lognormal_sweep(128)
    delta = w["delta"]
    sols = {}
    for s in w["solves"]:
        phi, _, st = gpu_solve(delta, s["alpha"], s["kappa"], tol=1e-10, max_cycles=300)
        assert st["rc"] == mg.MG_OK, (s, st)
        fl, hits = floored(delta, s["alpha"], s["kappa"])
        assert st["guard_hits"] == hits
        d, g = O.residual(phi, fl, s["alpha"], s["kappa"])
        assert np.abs(d - d.mean()).max() < 1.5e-10 and g == 0
        sols[(s["r_v"], s["kappa"])] = phi
    for rv in (2.0, 8.0, 32.0):
        a, b = sols[(rv, 1.0)], sols[(rv, -1.0)]
        assert np.abs(a + b).max() < 1e-9 * np.abs(a).max()
    s = w["solves"][2]
    ref, _ = O.fas_solve(delta, s["alpha"], s["kappa"], tol=1e-10)
    assert rel(sols[(s["r_v"], s["kappa"])], ref) < 1e-9


@pytest.mark.parametrize("n", [4, 6, 12, 20, 48])
def test_ragged_and_degenerate_sizes(n):
    delta = I.lognormal_delta(n, 1.0, 40 + n)
    phi, _, st = gpu_solve(delta, 0.3, 1.0, max_cycles=400)
    assert st["rc"] == mg.MG_OK, st
    ref, _ = O.fas_solve(delta, 0.3, 1.0, tol=1e-11, max_cycles=400)
    assert rel(phi, ref) < 1e-10


def test_poisson_limit_matches_fft():
    n = 32
    delta = I.lognormal_delta(n, 1.0, 77)
    phi, _, st = gpu_solve(delta, 0.0, 1.3)
    h = 1.0 / n
    k = np.arange(n)
    s2 = np.sin(np.pi * k / n) ** 2
    eig = -(4 / h ** 2) * (s2[:, None, None] + s2[None, :, None] + s2[None, None, :])
    eig[0, 0, 0] = 1.0
    ph = np.fft.fftn(1.3 * delta) / eig
    ph[0, 0, 0] = 0
    assert rel(phi, np.fft.ifftn(ph).real) < 1e-10


def test_uniform_density_and_wrong_branch():
    n = 16
    phi0 = np.random.default_rng(5).uniform(-0.05, 0.05, (n, n, n))
    phi, _, st = gpu_solve(np.zeros((n, n, n)), 0.3, 1.0, phi0=phi0, tol=1e-10)
    assert st["rc"] == mg.MG_OK and phi.max() - phi.min() < 1e-11
    phi, _, st = gpu_solve(np.zeros((n, n, n)), 0.3, 1.0, branch=-1, phi0=phi0, tol=1e-10)
    assert st["rc"] == mg.MG_OK
    assert st["lambda"] == pytest.approx(3 / (2 * 0.3), rel=1e-10)


def test_host_buffers_and_determinism():
    w = I.workload_tophat(32)
    a, _, s1 = gpu_solve(w["delta"], w["alpha"], w["kappa"], on_device=False)
    b, _, s2 = gpu_solve(w["delta"], w["alpha"], w["kappa"])
    c, _, s3 = gpu_solve(w["delta"], w["alpha"], w["kappa"], use_graphs=0)
    assert np.array_equal(a, b) and np.array_equal(a, c)
    assert s1["hist"] == s2["hist"] == s3["hist"]


@pytest.mark.parametrize("n", [32, 48, 64])
def test_fused_coarse_subcycle_is_bit_identical(n):
    """The levels with <= 16 cells per side run as one cluster launch that calls the
    per-level kernels' bodies with the same block partition: the same bits."""
    delta = I.lognormal_delta(n, 1.5, 7)
    a, _, s1 = gpu_solve(delta, 0.3, 1.0, tol=1e-10, fuse_coarse=1)
    b, _, s2 = gpu_solve(delta, 0.3, 1.0, tol=1e-10, fuse_coarse=0)
    assert s1["rc"] == s2["rc"] == mg.MG_OK
    assert np.array_equal(a, b) and s1["hist"] == s2["hist"]
    assert s1["launches"] < s2["launches"]


@pytest.mark.gpu
def test_kernel_timing_modes_leave_the_solve_unchanged():
    """time_kernels = 1 brackets every finest-level colour stage with events, 2 only
    the first of each smoothing call (2 sweeps x 4 colours -> 1); the solve is the
    same bits in every mode."""
    n = 32
    delta = I.lognormal_delta(n, 1.5, 7)
    a, _, s0 = gpu_solve(delta, 0.3, 1.0, tol=1e-10, time_kernels=0)
    b, _, s1 = gpu_solve(delta, 0.3, 1.0, tol=1e-10, time_kernels=1)
    c, _, s2 = gpu_solve(delta, 0.3, 1.0, tol=1e-10, time_kernels=2)
    assert s0["rc"] == s1["rc"] == s2["rc"] == mg.MG_OK
    assert np.array_equal(a, b) and np.array_equal(a, c)
    assert s0["kernel_launches"] == 0
    assert s1["kernel_launches"] == 8 * s2["kernel_launches"] > 0
    assert s1["kernel_ms"] > 0 and s2["kernel_ms"] > 0
    with pytest.raises(mg.MGError):
        mg.mg_create_grid(n, mg.options(time_kernels=3))


def test_errors_are_reported():
    n = 16
    with pytest.raises(mg.MGError) as e:
        mg.mg_create_grid(18)           # coarsest 9 is odd -> coarsest 18 > 16
    assert e.value.status == mg.MG_EINVAL
    g = mg.mg_create_grid(n)
    try:
        with pytest.raises(mg.MGError) as e:
            mg.mg_solve(g, 0, 0.3, 1.0, 1e-8)
        assert e.value.status == mg.MG_ESTATE
        delta = np.zeros((n, n, n))
        delta[1, 2, 3] = np.nan
        mg.mg_set_density(g, 0, -1, delta)
        st = mg.mg_solve(g, 0, 0.3, 1.0, 1e-8, check=False)
        assert st["rc"] == mg.MG_ENAN
        mg.mg_set_density(g, 0, -1, I.lognormal_delta(n, 1.0, 3))
        mg.mg_set_field(g, 0, -1, np.zeros((n, n, n)))
        st = mg.mg_solve(g, 0, 0.3, 1.0, 1e-18, check=False)   # below the rounding floor
        assert st["rc"] == mg.MG_ENOCONV
        assert "stalled" in mg.mg_last_error() or "max_cycles" in mg.mg_last_error()
        with pytest.raises(mg.MGError) as e:
            mg.mg_solve(g, 1, 0.0, 1.0, 1e-8)
        assert e.value.status == mg.MG_EINVAL
        with pytest.raises(mg.MGError):
            mg.mg_solve(g, 2, 0.3, 1.0, 1e-8)
    finally:
        mg.mg_destroy_grid(g)
