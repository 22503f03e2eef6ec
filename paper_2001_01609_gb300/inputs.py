"""Seeded synthetic inputs for the Rayleigh-Benard workloads.

This module holds no arithmetic of the method: it only draws the initial
temperature field that the paper describes (Sec. 2.1: a linear temperature
profile with small perturbations, u = 0) on the native collocation grid, so that
the CUDA library and the CPU checker start from the same numbers.

Native grid: x_i = Lx i / Nx (i < Nx), z_j = -cos(pi j / (Nz - 1)) / 2 (j < Nz,
ascending from the bottom wall z = -1/2 to the top wall z = 1/2).  Arrays are
(Nz, Nx), z-major.
"""
import numpy as np


def native_grid(Nx, Nz, Lx=2.0):
    x = Lx * np.arange(Nx) / Nx
    z = -0.5 * np.cos(np.pi * np.arange(Nz) / (Nz - 1))
    return x, z


def noise(Nx, Nz, seed):
    """xi_ij ~ N(0, 1), PCG64 seeded, shape (Nz, Nx)."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal((Nz, Nx))


def initial_temperature(Nx, Nz, seed, amplitude=1e-3, Lx=2.0):
    """T = (1/2 - z) + amplitude * xi * (z + 1/2)(1/2 - z) on the native grid.

    The perturbation envelope vanishes on both walls, so the wall temperatures
    T(-1/2) = 1, T(1/2) = 0 of Eq. 6 hold exactly on the grid.
    """
    _, z = native_grid(Nx, Nz, Lx)
    zz = z[:, None]
    return (0.5 - zz) + amplitude * noise(Nx, Nz, seed) * (zz + 0.5) * (0.5 - zz)
