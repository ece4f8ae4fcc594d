"""The synthetic inputs follow their stated recipes (no GPU): every generator
returns float32 points on the 2^-24 grid of [0, 1), reproducibly by seed; the
clustered set puts 70 % of its points in blobs; the Zel'dovich set is a potential
flow (its displacement is parallel to k in Fourier space) with no mean, no power
beyond the spherical Nyquist cut, a 3-D rms displacement of half a cell and a
displacement spectrum P_psi ~ k^-4 (= P_delta / k^2 for P_delta ~ k^-2)."""
import numpy as np
import pytest

import workloads


def _on_grid(x):
    assert x.dtype == np.float32 and np.all(x >= 0) and np.all(x < 1)
    s = x.astype(np.float64) * 2.0 ** 24
    assert np.array_equal(s, np.floor(s))


@pytest.mark.parametrize("gen", ["uniform", "clustered"])
def test_grid_and_seed(gen):
    f = getattr(workloads, gen)
    a, b, c = f(5000, 1), f(5000, 1), f(5000, 2)
    _on_grid(a)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_clustered_blob_fraction():
    spatial = pytest.importorskip("scipy.spatial")
    x = workloads.clustered(20000, 3, n_blobs=10, sigma_lo=1e-4, sigma_hi=1e-4)
    _on_grid(x)
    near = spatial.cKDTree(x, boxsize=1.0).query_ball_point(x, 2e-3, return_length=True)
    # a blob point has ~1400 others within 20 sigma; a background point almost none
    assert abs(np.mean(near > 50) - 0.7) < 0.01


def test_zeldovich_recipe():
    n = 32
    x = workloads.zeldovich(n, 3)
    _on_grid(x)
    assert np.array_equal(x, workloads.zeldovich(n, 3))
    g = np.arange(n) / n
    q = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)  # lattice order (i n + j) n + l
    psi = x.astype(np.float64) - q
    psi -= np.round(psi)                                                  # minimum image
    assert abs(np.sqrt(np.mean(np.sum(psi ** 2, 1))) * n - 0.5) < 1e-3   # rms |psi| = 0.5 cells
    assert np.all(np.abs(psi.mean(0)) * n < 1e-5)                         # k = 0 removed
    f = np.fft.fftn(psi.reshape(n, n, n, 3), axes=(0, 1, 2))
    m = np.fft.fftfreq(n, 1.0 / n)
    k = np.stack(np.meshgrid(m, m, m, indexing="ij"), -1)
    k2 = np.sum(k ** 2, -1)
    power = np.sum(np.abs(f) ** 2, -1)
    total = power.sum()
    nz = k2 > 0
    par = (np.sum(k * f, -1)[..., None] * k)[nz] / k2[nz][:, None]      # component along k
    assert np.sum(np.abs(f[nz] - par) ** 2) < 1e-8 * total               # curl-free
    assert power[k2 > (n / 2) ** 2].sum() < 1e-8 * total                 # spherical cut at k_Nyquist
    shells = np.arange(2, 13)
    kk = np.sqrt(k2)
    mean_p = [power[(kk >= s - 0.5) & (kk < s + 0.5)].mean() for s in shells]
    slope = np.polyfit(np.log(shells), np.log(mean_p), 1)[0]
    assert abs(slope + 4.0) < 0.4


def test_clustered_device_recipe_on_the_host_generator():
    """The device-side draw (torch's generator; run here on the CPU) keeps the
    clustered recipe: grid, reproducibility by seed, 70 % of points in blobs."""
    torch = pytest.importorskip("torch")
    spatial = pytest.importorskip("scipy.spatial")
    a = workloads.clustered_device(20000, 3, "cpu", n_blobs=10, sigma_lo=1e-4, sigma_hi=1e-4)
    b = workloads.clustered_device(20000, 3, "cpu", n_blobs=10, sigma_lo=1e-4, sigma_hi=1e-4)
    c = workloads.clustered_device(20000, 4, "cpu", n_blobs=10, sigma_lo=1e-4, sigma_hi=1e-4)
    assert torch.equal(a, b) and not torch.equal(a, c)
    x = a.numpy()
    _on_grid(x)
    near = spatial.cKDTree(x, boxsize=1.0).query_ball_point(x, 2e-3, return_length=True)
    assert abs(np.mean(near > 50) - 0.7) < 0.01
