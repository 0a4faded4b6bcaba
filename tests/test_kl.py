"""KL basis: exact covariance mat-vec, eigenpairs vs a dense eigensolve,
orthonormality, and the truncated covariance."""
import numpy as np

from paper_1903_08741_gb300.kl import covariance_matvec, kl_basis


def dense_cov(nx, nz, sigma2, lam):
    h = 1.0 / nz
    x = (np.arange(nx) + 0.5) * h
    z = (np.arange(nz) + 0.5) * h
    X, Z = np.meshgrid(x, z)
    P = np.stack([X.ravel(), Z.ravel()], 1)
    d = np.sqrt(((P[:, None, :] - P[None, :, :]) ** 2).sum(-1))
    return sigma2 * np.exp(-d / lam)


def test_matvec_is_exact():
    C = dense_cov(12, 8, 1.0, 0.2)
    mv = covariance_matvec(12, 8, 1.0, 0.2)
    v = np.random.default_rng(0).normal(size=96)
    assert np.abs(mv(v) - C @ v).max() < 1e-12


def test_lanczos_matches_dense_eigensolve():
    nx = nz = 48                      # n = 2304 > 2048: Lanczos branch
    B, lam = kl_basis(nx, nz, 16, 1.0, 0.2)
    C = dense_cov(nx, nz, 1.0, 0.2)
    ref = np.linalg.eigvalsh(C)[::-1][:16]
    assert np.abs(lam - ref).max() < 1e-9 * ref[0]
    psi = B.reshape(16, -1) / np.sqrt(lam)[:, None]
    assert np.abs(psi @ psi.T - np.eye(16)).max() < 1e-9
    # C psi_j = lambda_j psi_j
    assert np.abs(C @ psi[3] - lam[3] * psi[3]).max() < 1e-8 * lam[0]


def test_dense_branch_and_truncated_covariance():
    B, lam = kl_basis(16, 16, 256, 1.0, 0.2)       # complete basis: sum B B^T = C
    C = dense_cov(16, 16, 1.0, 0.2)
    Bm = B.reshape(256, -1)
    assert np.abs(Bm.T @ Bm - C).max() < 1e-10
