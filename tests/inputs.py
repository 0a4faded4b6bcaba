"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

This module holds no arithmetic of the method: only the configured instance's
constants (the physics of the Gardner-closure workloads) and seeded random
arrays that stand in for soil fields in unit tests.
"""
import numpy as np

# Physics of every configured workload (Gardner closure, infiltration into a
# dry column): theta_r, theta_s, initial head, Dirichlet top / bottom heads.
PHYSICS = dict(theta_r=0.1, theta_s=0.5, p_init=-5.0, p_top=-0.5, p_bottom=-5.0)
SOLVER = dict(picard_tol=1e-8, picard_maxit=50, mg_tol=1e-10, mg_maxit=100, nu1=2, nu2=2)

# Workloads: (grid side, samples, steps, dt).
WORKLOADS = {
    "mc32": (32, 64, 10, 0.01),        # plain MC, 32^2 x 64, T = 0.1
    "mc128": (128, 4096, 20, 0.005),   # batched MC, 128^2 x 4096, T = 0.1
}


def smooth_random_fields(nx, nz, nsamples, seed, lnks_amp=1.0, alpha_lo=0.5, alpha_hi=2.0):
    """Cheap seeded fields (sum of a few random Fourier modes) for unit tests."""
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) / nz
    z = (np.arange(nz) + 0.5) / nz
    X, Z = np.meshgrid(x, z)
    lnks = np.zeros((nsamples, nz, nx))
    g = np.zeros((nsamples, nz, nx))
    for s in range(nsamples):
        for _ in range(6):
            kx, kz = rng.integers(0, 4, size=2)
            ph = rng.uniform(0, 2 * np.pi, size=2)
            lnks[s] += rng.normal() * np.cos(np.pi * kx * X + ph[0]) * np.cos(np.pi * kz * Z + ph[1])
            g[s] += rng.normal() * np.cos(np.pi * kx * X + ph[1]) * np.cos(np.pi * kz * Z + ph[0])
    lnks *= lnks_amp / max(1e-12, np.abs(lnks).max())
    u = 0.5 + 0.5 * np.tanh(g)
    alpha = alpha_lo + (alpha_hi - alpha_lo) * u
    return lnks, alpha
