"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds no arithmetic of the solver: it only draws density contrasts,
parameters and patch lists.  The paper's own inputs are particle density fields
of cosmological N-body runs (Sec. V.A); these generators stand in for them with
fields of the same kind (a top-hat overdensity as in Sec. IV.C, lognormal
Gaussian random fields with a power-law spectrum, refined patches over the
densest regions, as the refinement criterion of Sec. III.C would place them).

Arrays are float64, indexed ``a[k, j, i]`` (x fastest), box length 1, and
``delta = rho - 1`` with mean rho = 1 (the code units of Eq. code_unit).
"""
from __future__ import annotations

import math

import numpy as np

#: reference top-hat used to express the Vainshtein radius in cells
TOPHAT_DELTA0 = 10.0
TOPHAT_RADIUS = 4.0


def tophat(n: int, delta0: float = TOPHAT_DELTA0, radius: float = TOPHAT_RADIUS) -> np.ndarray:
    """delta0 in the cells whose centre lies strictly within `radius` cells of the box
    centre, and the constant that makes the mean zero everywhere else."""
    x = np.arange(n, dtype=np.float64) + 0.5 - n / 2.0
    zz, yy, xx = np.meshgrid(x, x, x, indexing="ij")
    inside = (xx * xx + yy * yy + zz * zz) < radius * radius
    nin = int(inside.sum())
    out = np.full((n, n, n), -delta0 * nin / (n ** 3 - nin))
    out[inside] = delta0
    return out


def alpha_kappa_for_rv(r_v_cells: float) -> float:
    """alpha*kappa that puts the Vainshtein radius of the reference top-hat
    (delta0 = 10, radius 4 cells) at `r_v_cells` cells: r_V^3 = 8 alpha kappa m,
    m = delta0 R^3 / 3 (the spherical solution of Sec. II.B in these units)."""
    m_ref = TOPHAT_DELTA0 * TOPHAT_RADIUS ** 3 / 3.0
    return r_v_cells ** 3 / (8.0 * m_ref)


def gaussian_field(n: int, seed: int, spectral_index: float = -2.0) -> np.ndarray:
    """Zero-mean, unit-variance Gaussian random field with P(k) ~ |k|^index, P(0) = 0."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((n, n, n))
    wk = np.fft.rfftn(white)
    f = np.fft.fftfreq(n) * n
    fr = np.fft.rfftfreq(n) * n
    kz, ky, kx = np.meshgrid(f, f, fr, indexing="ij")
    k2 = (2.0 * math.pi) ** 2 * (kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(k2)
    nz = k2 > 0
    amp[nz] = k2[nz] ** (spectral_index / 4.0)  # sqrt(P), P ~ k^index
    g = np.fft.irfftn(wk * amp, s=(n, n, n), axes=(0, 1, 2))
    g -= g.mean()
    g /= g.std()
    return g


def lognormal_delta_device(n: int, sigma: float, seed: int, device="cuda"):
    """The lognormal recipe of lognormal_delta drawn with torch on `device` (for
    grids whose host FFT would be slow); its own random stream, float64."""
    import torch
    gen = torch.Generator(device=device).manual_seed(seed)
    white = torch.randn((n, n, n), generator=gen, dtype=torch.float64, device=device)
    wk = torch.fft.rfftn(white)
    del white
    f = torch.fft.fftfreq(n, device=device, dtype=torch.float64) * n
    fr = torch.fft.rfftfreq(n, device=device, dtype=torch.float64) * n
    k2 = (2.0 * math.pi) ** 2 * (f[:, None, None] ** 2 + f[None, :, None] ** 2 +
                                 fr[None, None, :] ** 2)
    amp = torch.where(k2 > 0, k2.clamp_min(1e-300) ** (-0.5), torch.zeros_like(k2))
    del k2
    wk *= amp
    del amp
    g = torch.fft.irfftn(wk, s=(n, n, n))
    del wk
    g -= g.mean()
    g /= g.std()
    rho = torch.exp(sigma * g - 0.5 * sigma * sigma)
    del g
    rho /= rho.mean()
    return rho - 1.0


def lognormal_delta(n: int, sigma: float, seed: int) -> np.ndarray:
    """delta = rho - 1 with rho = exp(sigma g - sigma^2/2) renormalised to mean 1."""
    g = sigma * gaussian_field(n, seed)
    rho = np.exp(g - 0.5 * sigma * sigma)
    rho /= rho.mean()
    return rho - 1.0


# ---------------------------------------------------------------------------
# Refined patches (8^3 level-l cells, origin a multiple of 8)
# ---------------------------------------------------------------------------
PATCH = 8


def _upsample_trilinear(coarse: np.ndarray, origin_coarse, size_coarse: int) -> np.ndarray:
    """Cell-centred trilinear interpolation of a periodic coarse array onto the
    2*size_coarse fine cells of the block starting at origin_coarse."""
    n = coarse.shape[0]
    fine = 2 * size_coarse
    out = np.zeros((fine, fine, fine))
    idx = np.arange(fine)
    par = idx // 2
    side = np.where(idx % 2 == 1, 1, -1)
    ox, oy, oz = origin_coarse
    for a in (0, 1):
        wx = 0.75 if a == 0 else 0.25
        ix = (ox + par + a * side) % n
        for b in (0, 1):
            wy = 0.75 if b == 0 else 0.25
            iy = (oy + par + b * side) % n
            for c in (0, 1):
                wz = 0.75 if c == 0 else 0.25
                iz = (oz + par + c * side) % n
                out += wx * wy * wz * coarse[np.ix_(iz, iy, ix)]
    return out


def flag_blocks(delta: np.ndarray, threshold: float, block: int = 4):
    """Origins (x, y, z) of the block-aligned blocks of `delta` holding any cell above
    `threshold`."""
    n = delta.shape[0]
    nb = n // block
    m = delta.reshape(nb, block, nb, block, nb, block).max(axis=(1, 3, 5))
    kz, jy, ix = np.nonzero(m > threshold)
    return np.stack([ix * block, jy * block, kz * block], axis=1).astype(np.int32)


def refine_density(rho_parent_lookup, origins_fine: np.ndarray, seed: int, noise: float = 0.1):
    """Density contrast on fine 8^3 patches: trilinear of the parent rho times
    (1 + noise u), u ~ U[-1, 1].  `rho_parent_lookup(origin_parent)` returns the
    parent rho on the 6^3 block (4^3 parents plus one cell each side) around it."""
    rng = np.random.default_rng(seed)
    out = np.empty((origins_fine.shape[0], PATCH, PATCH, PATCH))
    for q, o in enumerate(origins_fine):
        block = rho_parent_lookup(o // 2)
        fine = _upsample_trilinear(block, (1, 1, 1), PATCH // 2)
        u = rng.uniform(-1.0, 1.0, size=fine.shape)
        out[q] = fine * (1.0 + noise * u) - 1.0
    return out


def refined_hierarchy(n0: int, sigma: float, seed: int, thresholds=(20.0, 80.0)):
    """Domain delta plus two levels of 8^3 patches over the blocks whose delta
    exceeds the thresholds.  Level-2 parents are made properly nested by adding
    every level-1 patch touched by the level-2 parents dilated by one level-1 cell.
    Returns dict(delta0, levels=[dict(origins, delta), ...])."""
    delta0 = lognormal_delta(n0, sigma, seed)
    rho0 = delta0 + 1.0
    n1 = 2 * n0
    # level 1: 4^3-aligned domain blocks -> 8^3 level-1 patches
    org1 = flag_blocks(delta0, thresholds[0], block=4) * 2

    def lookup0(o):
        idx = [(o[d] - 1 + np.arange(6)) % n0 for d in range(3)]
        return rho0[np.ix_(idx[2], idx[1], idx[0])]

    delta1 = refine_density(lookup0, org1, seed * 10 + 1)
    # level 2: 4^3-aligned level-1 blocks with delta1 > threshold
    cand = []
    for q, o in enumerate(org1):
        sub = flag_blocks(delta1[q], thresholds[1], block=4)
        for s in sub:
            cand.append((o + s) * 2)
    org2 = np.array(cand, dtype=np.int32).reshape(-1, 3)
    if org2.shape[0]:
        org2 = np.unique(org2, axis=0)
    # nesting: level-1 cells within one cell of the level-2 parents must be refined
    have = {tuple(o // PATCH) for o in org1}
    extra = set()
    for o in org2:
        par = o // 2
        for dz in (-1, 0, 4):
            for dy in (-1, 0, 4):
                for dx in (-1, 0, 4):
                    c = ((par[0] + dx) % n1, (par[1] + dy) % n1, (par[2] + dz) % n1)
                    b = (c[0] // PATCH, c[1] // PATCH, c[2] // PATCH)
                    if b not in have:
                        extra.add(b)
    if extra:
        add = np.array(sorted(extra), dtype=np.int32) * PATCH
        delta_add = refine_density(lookup0, add, seed * 10 + 3)
        org1 = np.concatenate([org1, add])
        delta1 = np.concatenate([delta1, delta_add])
        have |= extra
    order = np.lexsort((org1[:, 0], org1[:, 1], org1[:, 2]))
    org1, delta1 = org1[order], delta1[order]
    table1 = {tuple(o // PATCH): q for q, o in enumerate(org1)}
    rho1 = delta1 + 1.0

    def lookup1(o):
        # parent block of a level-2 patch: 4^3 level-1 cells plus a one-cell shell
        block = np.empty((6, 6, 6))
        for kk in range(6):
            for jj in range(6):
                for ii in range(6):
                    c = ((o[0] - 1 + ii) % n1, (o[1] - 1 + jj) % n1, (o[2] - 1 + kk) % n1)
                    q = table1[(c[0] // PATCH, c[1] // PATCH, c[2] // PATCH)]
                    block[kk, jj, ii] = rho1[q, c[2] % PATCH, c[1] % PATCH, c[0] % PATCH]
        return block

    delta2 = refine_density(lookup1, org2, seed * 10 + 2) if org2.shape[0] else \
        np.zeros((0, PATCH, PATCH, PATCH))
    if org2.shape[0]:
        order = np.lexsort((org2[:, 0], org2[:, 1], org2[:, 2]))
        org2, delta2 = org2[order], delta2[order]
    return {"delta0": delta0,
            "levels": [{"origins": org1, "delta": delta1}, {"origins": org2, "delta": delta2}]}


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------
def workload_tophat(n: int = 32):
    """32^3 top-hat, alpha = 0.3 (Vainshtein radius 8 cells), kappa = 1."""
    return {"delta": tophat(n), "alpha": alpha_kappa_for_rv(8.0), "kappa": 1.0, "branch": 0}


def workload_lognormal_sweep(n: int = 128, sigma: float = 1.5, seed: int = 1302,
                             r_v=(2.0, 8.0, 32.0)):
    """One lognormal field and six (alpha, kappa) pairs: three Vainshtein radii,
    each with the sign of alpha flipped (alpha and kappa flip together)."""
    delta = lognormal_delta(n, sigma, seed)
    solves = []
    for rv in r_v:
        ak = alpha_kappa_for_rv(rv)
        for sgn in (1.0, -1.0):
            solves.append({"alpha": sgn * ak, "kappa": sgn * 1.0, "branch": 0, "r_v": rv})
    return {"delta": delta, "solves": solves}


def workload_batch(count: int = 64, seed: int = 1305, sizes=(32, 64, 96, 128)):
    """`count` independent periodic solves of mixed sizes, sigma ~ U[0.5, 2.5],
    r_V log-uniform in [2, 16] cells, branch sign +-1 with probability 1/2."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(count):
        n = int(rng.choice(sizes))
        sigma = float(rng.uniform(0.5, 2.5))
        rv = float(math.exp(rng.uniform(math.log(2.0), math.log(16.0))))
        sgn = 1.0 if rng.uniform() < 0.5 else -1.0
        out.append({"n": n, "sigma": sigma, "r_v": rv, "alpha": sgn * alpha_kappa_for_rv(rv),
                    "kappa": sgn, "branch": 0, "seed": seed * 1000 + s})
    return out


def random_field(n: int, seed: int, amplitude: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return amplitude * rng.uniform(-1.0, 1.0, size=(n, n, n))
