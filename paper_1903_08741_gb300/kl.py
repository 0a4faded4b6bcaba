"""Karhunen-Loeve basis of the discrete ln Ks covariance (Sec. 3, Eqs.
KLexp_ch6, eq:Fred): the n_kl leading eigenpairs of the covariance matrix
C_ij = sigma2 exp(-|x_i - x_j| / corr_len) between cell centres, found once on
the host by Lanczos (scipy eigsh) with an exact matrix-vector product: C is
block Toeplitz with Toeplitz blocks, so C v is a circular convolution on a
(2 nx) x (2 nz) torus whose periodic distances equal the true ones for every
offset that occurs.  The basis is returned with sqrt(lambda_j) folded in, so
ln Ks = sum_j xi_j basis_j with xi_j ~ N(0, 1) (the input of rich_kl_fields and
rich_solve_batch_adjoint).  This is an offline set-up step, like building a
preconditioner; the per-sample work runs in the CUDA library.
"""
from __future__ import annotations

import numpy as np


def covariance_matvec(nx, nz, sigma2=1.0, corr_len=0.2):
    """v [nz*nx] -> C v, exact, by FFT convolution on the doubled torus."""
    h = 1.0 / nz
    px, pz = 2 * nx, 2 * nz
    a = np.minimum(np.arange(px), px - np.arange(px)) * h
    b = np.minimum(np.arange(pz), pz - np.arange(pz)) * h
    c = sigma2 * np.exp(-np.hypot(a[None, :], b[:, None]) / corr_len)
    fc = np.fft.rfft2(c)

    def mv(v):
        pad = np.zeros((pz, px))
        pad[:nz, :nx] = np.asarray(v).reshape(nz, nx)
        return np.fft.irfft2(fc * np.fft.rfft2(pad), s=(pz, px))[:nz, :nx].ravel()
    return mv


def kl_basis(nx, nz, n_kl, sigma2=1.0, corr_len=0.2, tol=1e-12):
    """(basis [n_kl, nz, nx] with sqrt(lambda) folded, lambda [n_kl]), eigenvalues
    descending; each eigenvector's sign makes its largest component positive."""
    import scipy.sparse.linalg as spla
    n = nx * nz
    mv = covariance_matvec(nx, nz, sigma2, corr_len)
    if n <= 2048:
        C = np.stack([mv(e) for e in np.eye(n)], axis=1)
        lam, vec = np.linalg.eigh(0.5 * (C + C.T))
        lam, vec = lam[::-1][:n_kl], vec[:, ::-1][:, :n_kl]
    else:
        op = spla.LinearOperator((n, n), matvec=mv, dtype=np.float64)
        v0 = np.ones(n) / np.sqrt(n)
        lam, vec = spla.eigsh(op, k=n_kl, which="LA", tol=tol, v0=v0, ncv=min(n, max(2 * n_kl + 1, n_kl + 64)))
        order = np.argsort(lam)[::-1]
        lam, vec = lam[order], vec[:, order]
    sgn = np.sign(vec[np.argmax(np.abs(vec), axis=0), np.arange(vec.shape[1])])
    vec = vec * sgn
    basis = (vec * np.sqrt(np.maximum(lam, 0.0))).T.reshape(n_kl, nz, nx)
    return np.ascontiguousarray(basis), lam
