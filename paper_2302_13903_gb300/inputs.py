"""Seeded synthetic inputs shaped like the paper's test problems.

This module holds only input generation: densities, grid lists and request
streams.  It contains none of the solver's arithmetic, so both the CUDA path and
its CPU oracle can take their inputs from here.

Recipes (the paper has no public dataset; these stand in for its tests):

* ``sinusoid`` -- the periodic sinusoidal density of Sec. 4.1 with rho_0 = 0
  and A = 1 on the unit cube, point-sampled at cell centres (i + 1/2) h.
* ``gaussian_blobs`` -- a periodic superposition of Gaussian blobs: centres
  uniform in the unit cube, sigma uniform in [0.02, 0.08], amplitudes
  lognormal (sigma = 1), minimum-image distance per axis, mean removed.
  Contributions are separable, so each blob is an outer product of three 1-D
  profiles; the accumulation order is fixed (blob by blob, one rounding for
  the product and one for the sum), so numpy and torch on any device give the
  same bits.
* ``uniform_sphere`` -- the uniform sphere (rho = 1, radius R) on
  [-0.5, 0.5]^3, each cell averaged over sub^3 sub-cell centres, as the paper
  does for its binary test (Sec. 4.2.1).
* ``batch_specs`` -- many independent grids: sizes from {16, 32, 64, 128}^3
  with Zipf weights 1/rank, boundary kinds uniform over periodic / fixed 0 /
  zero gradient, 1-8 blobs per grid.
* ``serving_stream`` -- Poisson arrivals of requests with sizes in
  {32, 64, 128, 256}^3, mixed boundary kinds including open (lmax uniform in
  0..4) and tolerances log-uniform in [1e-10, 1e-6].
"""
from __future__ import annotations

import math

import numpy as np

PERIODIC, FIXED, ZEROGRAD, OPEN = 0, 1, 2, 3


def cell_centres(n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    h = (hi - lo) / n
    return lo + (np.arange(n, dtype=np.float64) + 0.5) * h


def sinusoid(n: int) -> np.ndarray:
    """rho = sin(2 pi x) sin(2 pi y) sin(2 pi z) on the unit cube, shape (n, n, n)."""
    s = np.sin(2.0 * np.pi * cell_centres(n))
    return (s[:, None, None] * s[None, :, None]) * s[None, None, :]


def _blob_params(rng, n_blobs, sigma_range):
    centres = rng.random((n_blobs, 3))
    sigma = rng.uniform(sigma_range[0], sigma_range[1], n_blobs)
    amp = np.exp(rng.normal(0.0, 1.0, n_blobs))
    return centres, sigma, amp


def _profile(x, c, sigma, periodic):
    d = x - c
    if periodic:
        d = d - np.round(d)
    return np.exp(-(d * d) / (2.0 * sigma * sigma))


def blob_factors(n, n_blobs=64, seed=20230227, sigma_range=(0.02, 0.08), periodic=True):
    """Per-blob 1-D factors (amplitude folded into the z factor) and the mean."""
    rng = np.random.default_rng(seed)
    centres, sigma, amp = _blob_params(rng, n_blobs, sigma_range)
    x = cell_centres(n)
    facs = []
    mean = 0.0
    for b in range(n_blobs):
        gx = _profile(x, centres[b, 0], sigma[b], periodic)
        gy = _profile(x, centres[b, 1], sigma[b], periodic)
        gz = amp[b] * _profile(x, centres[b, 2], sigma[b], periodic)
        facs.append((gz, gy, gx))
        mean += float(gz.mean() * gy.mean() * gx.mean())
    return facs, mean


def gaussian_blobs(n, n_blobs=64, seed=20230227, sigma_range=(0.02, 0.08), periodic=True,
                   remove_mean=True, device=None):
    """Sum of Gaussian blobs on the unit cube, shape (n, n, n), float64.

    With ``device=None`` a numpy array is returned; otherwise a torch tensor on
    that device (same bits: each step is one correctly rounded IEEE operation).
    """
    facs, mean = blob_factors(n, n_blobs, seed, sigma_range, periodic)
    if device is None:
        rho = np.zeros((n, n, n))
        for gz, gy, gx in facs:
            t = gz[:, None, None] * gy[None, :, None]
            rho += t * gx[None, None, :]
        if remove_mean:
            rho -= mean
        return rho
    import torch
    rho = torch.zeros((n, n, n), dtype=torch.float64, device=device)
    for gz, gy, gx in facs:
        t = torch.from_numpy(gz[:, None, None] * gy[None, :, None]).to(device)
        rho += t * torch.from_numpy(gx[None, None, :]).to(device)
    if remove_mean:
        rho -= mean
    return rho


def uniform_sphere(n: int, R: float = 0.25, sub: int = 10) -> np.ndarray:
    """Cell-averaged uniform sphere (rho = 1, radius R) on [-0.5, 0.5]^3."""
    h = 1.0 / n
    x = cell_centres(n, -0.5, 0.5)
    ax = np.abs(x)
    near = np.maximum(ax - 0.5 * h, 0.0)  # nearest distance per axis
    far = ax + 0.5 * h                    # farthest distance per axis
    dmin2 = near[:, None, None] ** 2 + near[None, :, None] ** 2 + near[None, None, :] ** 2
    dmax2 = far[:, None, None] ** 2 + far[None, :, None] ** 2 + far[None, None, :] ** 2
    rho = np.where(dmax2 <= R * R, 1.0, 0.0)
    cut = np.argwhere((dmin2 <= R * R) & (dmax2 > R * R))
    s = (np.arange(sub) + 0.5) / sub - 0.5
    sx, sy, sz = np.meshgrid(s, s, s, indexing="ij")
    for chunk in np.array_split(cut, max(1, len(cut) // 4096 + 1)):
        if len(chunk) == 0:
            continue
        k, j, i = chunk[:, 0], chunk[:, 1], chunk[:, 2]
        px = x[i][:, None] + h * sz.reshape(1, -1)
        py = x[j][:, None] + h * sy.reshape(1, -1)
        pz = x[k][:, None] + h * sx.reshape(1, -1)
        inside = (px * px + py * py + pz * pz) <= R * R
        rho[k, j, i] = inside.sum(axis=1) / float(sub ** 3)
    return rho


def sphere_potential(n: int, R: float = 0.25, G: float = 1.0) -> np.ndarray:
    """Analytic potential of the uniform sphere (rho = 1) at cell centres."""
    x = cell_centres(n, -0.5, 0.5)
    r = np.sqrt(x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2)
    M = 4.0 / 3.0 * math.pi * R ** 3
    inside = -2.0 * math.pi * G * (3.0 * R * R - r * r) / 3.0
    outside = -G * M / np.maximum(r, 1e-300)
    return np.where(r < R, inside, outside)


BATCH_SIZES = (16, 32, 64, 128)
BATCH_BCS = (PERIODIC, FIXED, ZEROGRAD)


def batch_specs(n_grids: int = 512, seed: int = 20230227):
    """Grid list for a batched solve: (n, bc, blob_seed, n_blobs) per grid."""
    rng = np.random.default_rng(seed)
    w = np.array([1.0 / (r + 1) for r in range(len(BATCH_SIZES))])
    w /= w.sum()
    sizes = rng.choice(BATCH_SIZES, size=n_grids, p=w)
    bcs = rng.choice(BATCH_BCS, size=n_grids)
    nblobs = rng.integers(1, 9, size=n_grids)
    return [dict(n=int(sizes[g]), bc=int(bcs[g]), seed=seed * 1000 + g, n_blobs=int(nblobs[g]))
            for g in range(n_grids)]


def batch_source(spec, device=None):
    """Density for one grid of ``batch_specs``; mean removed for periodic and
    zero-gradient grids (their solutions need a mean-free source)."""
    periodic = spec["bc"] == PERIODIC
    remove = spec["bc"] in (PERIODIC, ZEROGRAD)
    return gaussian_blobs(spec["n"], spec["n_blobs"], spec["seed"], periodic=periodic,
                          remove_mean=remove, device=device)


SERVE_SIZES = (32, 64, 128, 256)
SERVE_BCS = (PERIODIC, FIXED, ZEROGRAD, OPEN)


def serving_stream(rate: float, duration: float, seed: int = 20230227):
    """Poisson arrivals: list of dicts (t, n, bc, lmax, tol, seed, n_blobs)."""
    rng = np.random.default_rng(seed + int(rate))
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        bc = int(rng.choice(SERVE_BCS))
        out.append(dict(t=t, n=int(rng.choice(SERVE_SIZES)), bc=bc,
                        lmax=int(rng.integers(0, 5)) if bc == OPEN else 0,
                        tol=float(10.0 ** rng.uniform(-10.0, -6.0)),
                        seed=int(rng.integers(0, 2 ** 31)), n_blobs=int(rng.integers(1, 9))))
    return out


def serving_source(req, device=None):
    """Density for one request: blobs for periodic / fixed / zero gradient,
    a compact blob cluster around the centre for open boundaries."""
    if req["bc"] == OPEN:
        return _central_blobs(req, device)
    periodic = req["bc"] == PERIODIC
    remove = req["bc"] in (PERIODIC, ZEROGRAD)
    return gaussian_blobs(req["n"], req["n_blobs"], req["seed"], periodic=periodic,
                          remove_mean=remove, device=device)


def _central_blobs(req, device=None):
    n = req["n"]
    rng = np.random.default_rng(req["seed"])
    centres = 0.5 + 0.15 * (rng.random((req["n_blobs"], 3)) - 0.5)
    sigma = rng.uniform(0.02, 0.05, req["n_blobs"])
    amp = np.exp(rng.normal(0.0, 1.0, req["n_blobs"]))
    x = cell_centres(n)
    rho = np.zeros((n, n, n))
    for b in range(req["n_blobs"]):
        gx = _profile(x, centres[b, 0], sigma[b], False)
        gy = _profile(x, centres[b, 1], sigma[b], False)
        gz = amp[b] * _profile(x, centres[b, 2], sigma[b], False)
        rho += (gz[:, None, None] * gy[None, :, None]) * gx[None, None, :]
    if device is None:
        return rho
    import torch
    return torch.from_numpy(rho).to(device)
