"""Seeded synthetic point sets shared by the tests, the benchmark and the oracle.

This module only draws and places points; it holds none of the kNN / FoF
arithmetic.  Every coordinate it returns is float32, lies in [0, 1) and is a
multiple of 2**-24, so that coordinate differences are exact in float32 and
squared distances are exact in float64 (the two sides of every comparison then
see the same ties).

Workloads (shapes follow the paper's benchmark setups, Sec. III-E/III-G and
Sec. IV-C; the paper's cosmological simulation outputs are not available, so
a Zel'dovich-displaced lattice stands in for them):

* ``uniform``      -- uniform random in the unit cube (Sec. III-F, Fig. knnlib).
* ``clustered``    -- 70 % of points in isotropic Gaussian blobs with log-uniform
                      widths, 30 % uniform background, periodic unit box.
* ``zeldovich``    -- n^3 lattice displaced by the Zel'dovich approximation of a
                      Gaussian random field with P(k) ~ k^-2 (Sec. III-G: the
                      cosmological setup, box side proportional to N^(1/3)).
* ``lattice``      -- a regular grid (Sec. III-G, "uniform grid").
* ``batched_sets`` / ``serving_stream`` -- many independent sets / requests.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SNAP_BITS = 24
SNAP = float(1 << SNAP_BITS)


def snap_unit(u: np.ndarray) -> np.ndarray:
    """Map values in R to [0,1) on the 2**-24 grid (periodic wrap), as float32."""
    q = np.floor(np.asarray(u, dtype=np.float64) * SNAP).astype(np.int64)
    q %= (1 << SNAP_BITS)
    return (q.astype(np.float64) / SNAP).astype(np.float32)


def clip_unit(u: np.ndarray) -> np.ndarray:
    """Map values to [0,1) on the 2**-24 grid by clamping (open boundaries)."""
    q = np.floor(np.asarray(u, dtype=np.float64) * SNAP).astype(np.int64)
    q = np.clip(q, 0, (1 << SNAP_BITS) - 1)
    return (q.astype(np.float64) / SNAP).astype(np.float32)


def uniform(n: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return snap_unit(rng.random((n, 3)))


def clustered(n: int, seed: int, n_blobs: int = 4096, frac_blob: float = 0.7,
              sigma_lo: float = 1e-4, sigma_hi: float = 1e-2) -> np.ndarray:
    """70 % Gaussian blobs (uniform centres, log-uniform sigma), 30 % uniform; wrapped mod 1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_blobs = max(1, int(n_blobs))
    centres = rng.random((n_blobs, 3))
    sigmas = np.exp(rng.uniform(math.log(sigma_lo), math.log(sigma_hi), n_blobs))
    n_in = int(round(frac_blob * n))
    out = np.empty((n, 3), dtype=np.float64)
    blob = rng.integers(0, n_blobs, n_in)
    out[:n_in] = centres[blob] + rng.standard_normal((n_in, 3)) * sigmas[blob, None]
    out[n_in:] = rng.random((n - n_in, 3))
    perm = rng.permutation(n)
    return snap_unit(out[perm])


def zeldovich(n_side: int, seed: int, rms_cells: float = 0.5, spectral_index: float = -2.0,
              workers: int = -1) -> np.ndarray:
    """n_side^3 lattice in the periodic unit box displaced by the Zel'dovich field.

    White noise -> real FFT -> multiply by sqrt(P(k)), P ~ k^spectral_index for
    0 < |k| <= k_Nyquist (spherical cut, k = 0 removed) -> psi(k) = i k delta(k) / k^2
    -> three inverse FFTs; psi is scaled so that the 3-D rms |psi| equals
    ``rms_cells`` lattice spacings.  Points are returned in lattice order
    (index = (i*n + j)*n + l).
    """
    import scipy.fft as sfft

    n = int(n_side)
    rng = np.random.Generator(np.random.PCG64(seed))
    noise = rng.standard_normal((n, n, n), dtype=np.float32)
    dk = sfft.rfftn(noise, workers=workers)
    del noise
    m_full = np.fft.fftfreq(n, d=1.0 / n).astype(np.float32)   # integer wave numbers
    m_half = np.fft.rfftfreq(n, d=1.0 / n).astype(np.float32)
    kx = (2 * np.pi * m_full)[:, None, None]
    ky = (2 * np.pi * m_full)[None, :, None]
    kz = (2 * np.pi * m_half)[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    k_nyq = np.float32(np.pi * n)
    keep = (k2 > 0) & (k2 <= k_nyq * k_nyq)
    with np.errstate(divide="ignore", invalid="ignore"):
        amp = np.where(keep, k2 ** (spectral_index / 4.0), 0.0).astype(np.float32)  # sqrt(P)
        inv_k2 = np.where(keep, 1.0 / k2, 0.0).astype(np.float32)
    dk *= amp
    del amp
    dk *= inv_k2
    del inv_k2, keep
    psi = []
    for kc in (kx, ky, kz):
        comp = sfft.irfftn(1j * kc * dk, s=(n, n, n), workers=workers).astype(np.float32)
        psi.append(comp)
    del dk
    rms = math.sqrt(sum(float(np.mean(c.astype(np.float64) ** 2)) for c in psi))
    scale = (rms_cells / n) / rms if rms > 0 else 0.0
    q = (np.arange(n, dtype=np.float64) / n)
    out = np.empty((n, n, n, 3), dtype=np.float32)
    for d, comp in enumerate(psi):
        shape = [1, 1, 1]
        shape[d] = n
        base = q.reshape(shape)
        out[..., d] = snap_unit(base + comp.astype(np.float64) * scale)
    return out.reshape(-1, 3)


def lattice(n_side, spacing_bits: int = 9, offset_units: int = 0, dims=None) -> np.ndarray:
    """Regular grid with spacing 2**-spacing_bits (exact in float32), C order."""
    if dims is None:
        dims = (n_side, n_side, n_side)
    h = 1.0 / (1 << spacing_bits)
    ii = np.indices(dims).reshape(3, -1).T.astype(np.float64)
    x = (ii * h + offset_units / SNAP) % 1.0
    return snap_unit(x)


def mean_spacing(n: int, volume: float = 1.0) -> float:
    """(V/N)^(1/3): FoF linking lengths are quoted in these units (Sec. IV, R_link)."""
    return (volume / n) ** (1.0 / 3.0)


# --------------------------------------------------------------------------- named configurations

@dataclass(frozen=True)
class Workload:
    name: str
    n: int
    periodic_L: float  # 0 = open
    k: int
    b: float


def config_small_uniform() -> tuple[Workload, np.ndarray]:
    """N = 32768 uniform in the unit cube, open; k = 16, b = 0.2 N^(-1/3)."""
    n = 32768
    w = Workload("uniform-32768-open", n, 0.0, 16, 0.2 * mean_spacing(n))
    return w, uniform(n, 1)


def config_clustered_16m(n: int = 1 << 24) -> tuple[Workload, np.ndarray]:
    """N = 2^24 clustered (4096 blobs), periodic unit box; k = 32, b = 0.2 spacing."""
    w = Workload(f"clustered-{n}-periodic", n, 1.0, 32, 0.2 * mean_spacing(n))
    return w, clustered(n, 2)


def config_zeldovich(n_side: int = 512) -> tuple[Workload, np.ndarray]:
    """n_side^3 Zel'dovich lattice, periodic unit box; k = 16, b = 0.2 spacing."""
    n = n_side ** 3
    w = Workload(f"zeldovich-{n_side}^3-periodic", n, 1.0, 16, 0.2 / n_side)
    return w, zeldovich(n_side, 3)


def batched_specs(n_sets: int = 512, seed: int = 4, n_lo: float = 1e3, n_hi: float = 2e6,
                  total_cap: int | None = None):
    """The per-set draws of ``batched_sets`` without the points: a list of dicts
    {n, seed, n_blobs, op ('knn'|'fof'), k, b, periodic_L}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.floor(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), n_sets))).astype(np.int64)
    if total_cap is not None:
        while sizes.sum() > total_cap:
            sizes = np.maximum(sizes // 2, 1)
    specs = []
    for n in sizes:
        spec = dict(n=int(n), seed=int(rng.integers(0, 2**62)), n_blobs=max(1, int(n) // 4096), periodic_L=1.0)
        if rng.random() < 0.5:
            spec.update(op="knn", k=int(rng.choice([8, 16, 32])), b=0.0)
        else:
            fac = float(rng.choice([0.15, 0.2, 0.25]))
            spec.update(op="fof", k=0, b=fac * mean_spacing(int(n)))
        specs.append(spec)
    return specs


def _clustered_spec(spec):
    return clustered(spec["n"], spec["seed"], n_blobs=spec["n_blobs"])


def batched_sets(n_sets: int = 512, seed: int = 4, n_lo: float = 1e3, n_hi: float = 2e6,
                 total_cap: int | None = None, workers: int = 1):
    """Independent clustered sets with log-uniform sizes, each with its own op.

    Returns a list of dicts {points, op ('knn'|'fof'), k, b, periodic_L}.
    Blob count scales with the set size so blob occupancy matches the 2^24 case.
    ``workers`` > 1 draws the sets in that many spawned processes (same points).
    """
    specs = batched_specs(n_sets, seed, n_lo, n_hi, total_cap)
    if workers > 1:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            pts = list(ex.map(_clustered_spec, specs, chunksize=4))
    else:
        pts = [_clustered_spec(sp) for sp in specs]
    return [dict(points=x, op=sp["op"], k=sp["k"], b=sp["b"], periodic_L=sp["periodic_L"])
            for sp, x in zip(specs, pts)]


def clustered_device(n: int, seed: int, device, n_blobs: int | None = None, frac_blob: float = 0.7,
                     sigma_lo: float = 1e-4, sigma_hi: float = 1e-2):
    """Device-side draw of a ``clustered``-shaped set (same recipe, torch's Philox
    generator instead of PCG64, so the points differ from ``clustered``'s): for
    sets too large or too many to draw on the host.  Deterministic for a given
    (n, seed, device type); coordinates on the 2**-24 grid in [0, 1), float32."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) % (2**63))
    nb = max(1, int(n_blobs if n_blobs is not None else n // 4096))
    centres = torch.rand((nb, 3), generator=g, device=device, dtype=torch.float64)
    sig = torch.exp(torch.empty(nb, device=device, dtype=torch.float64).uniform_(
        math.log(sigma_lo), math.log(sigma_hi), generator=g))
    n_in = int(round(frac_blob * n))
    u = torch.empty((n, 3), device=device, dtype=torch.float64)
    blob = torch.randint(0, nb, (n_in,), generator=g, device=device)
    u[:n_in] = centres[blob] + torch.randn((n_in, 3), generator=g, device=device,
                                           dtype=torch.float64) * sig[blob, None]
    u[n_in:] = torch.rand((n - n_in, 3), generator=g, device=device, dtype=torch.float64)
    perm = torch.randperm(n, generator=g, device=device)
    q = torch.remainder(torch.floor(u[perm] * SNAP).to(torch.int64), 1 << SNAP_BITS)
    return (q.to(torch.float64) / SNAP).to(torch.float32).contiguous()


def serving_stream(n_req: int = 20000, seed: int = 5, n_lo: float = 1e4, n_hi: float = float(1 << 24),
                   repeat_frac: float = 0.3, rate_hz: float = 100.0):
    """Poisson arrivals of kNN/FoF requests; a fraction repeats an earlier set id.

    Returns a list of dicts {t_arrival, set_id, n, op, k, b, seed}; point sets are
    drawn lazily from (seed) with ``clustered``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n_req))
    reqs = []
    known = []
    for r in range(n_req):
        if known and rng.random() < repeat_frac:
            sid, n, pseed = known[int(rng.integers(0, len(known)))]
        else:
            n = int(np.floor(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
            sid, pseed = len(known), int(rng.integers(0, 2**62))
            known.append((sid, n, pseed))
        if rng.random() < 0.5:
            op, k, b = "knn", int(rng.choice([8, 16, 32])), 0.0
        else:
            op, k, b = "fof", 0, float(rng.choice([0.15, 0.2, 0.25])) * mean_spacing(n)
        reqs.append(dict(t_arrival=float(t[r]), set_id=sid, n=n, op=op, k=k, b=b, seed=pseed))
    return reqs
