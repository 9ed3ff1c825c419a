"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method itself: it only draws random fields
and builds grids, so that the CUDA path and the CPU oracle can be fed identical
inputs.  Every generator takes an explicit seed (numpy PCG64).

Workloads (sizes and parameters as in the paper's Hertz and rough-surface cases,
Sec. 6.2 and Sec. 8 / App. C):
* ``plastic_strain_field``: i.i.d. N(0, std^2) per voxel and component, times the
  depth envelope exp(-z / z_decay) (operator-apply workload).
* ``hertz_profile``: paraboloid h(x) = -r^2 / (2R) about the cell centre.
* ``self_affine_surface``: isotropic self-affine surface by Fourier filtering of
  white noise with the PSD of Sec. 8 (flat from k_l to k_r, power law
  |k|^(-2(1+H)) up to k_s, zero elsewhere), scaled to a given rms slope.
"""
import numpy as np


def uniform_depth(nz, depth):
    """Depth nodes [0, depth]_nz, both ends included (App. C notation)."""
    return np.linspace(0.0, float(depth), int(nz))


def plastic_strain_field(n1, n2, z, seed, std=1.0e-3, z_decay=0.1, dtype=np.float64):
    """Random symmetric plastic strain [Nz, 6, N2, N1] (x1 fastest)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z = np.asarray(z, dtype=np.float64)
    f = rng.standard_normal((z.size, 6, n2, n1)) * std
    f *= np.exp(-z / z_decay)[:, None, None, None]
    return f.astype(dtype)


def random_field(shape, seed, std=1.0, dtype=np.float64):
    """Plain i.i.d. normal field of the given shape."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.standard_normal(shape) * std).astype(dtype)


def hertz_profile(n1, n2, L1, L2, R):
    """Paraboloid h = -r^2/(2R) on the grid x_n = -L/2 + n L/N (cell centre at a node)."""
    x1 = -0.5 * L1 + np.arange(n1) * L1 / n1
    x2 = -0.5 * L2 + np.arange(n2) * L2 / n2
    X2, X1 = np.meshgrid(x2, x1, indexing="ij")
    return -(X1 ** 2 + X2 ** 2) / (2.0 * R)


def self_affine_surface(n, L, hurst, k_l, k_r, k_s, rms_slope, seed):
    """Isotropic self-affine surface [n, n] with zero mean and the given rms slope."""
    rng = np.random.Generator(np.random.PCG64(seed))
    noise = rng.standard_normal((n, n))
    k = np.fft.fftfreq(n, 1.0 / n)
    K2, K1 = np.meshgrid(k, k, indexing="ij")
    kk = np.hypot(K1, K2)
    psd = np.zeros_like(kk)
    flat = (kk >= k_l) & (kk < k_r)
    tail = (kk >= k_r) & (kk <= k_s)
    psd[flat] = 1.0
    psd[tail] = (kk[tail] / k_r) ** (-2.0 * (1.0 + hurst))
    h_hat = np.fft.fft2(noise) * np.sqrt(psd)
    h_hat[0, 0] = 0.0
    h = np.fft.ifft2(h_hat).real
    # spectral rms slope sqrt(mean |grad h|^2)
    qx = 2.0 * np.pi * K1 / L
    qy = 2.0 * np.pi * K2 / L
    gh = np.fft.fft2(h)
    slope = np.sqrt(np.sum((qx ** 2 + qy ** 2) * np.abs(gh) ** 2)) / (n * n)
    return h * (rms_slope / slope)
