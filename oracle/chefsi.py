"""Chebyshev-filtered subspace iteration (Sec. 2.1: "partial diagonalization ... using the
CheFSI method"; Y. Zhou, Y. Saad, M. L. Tiago, J. R. Chelikowsky, J. Comput. Phys. 219 (2006)
172, and the scaled filter of Y. Zhou and Y. Saad, SIAM J. Matrix Anal. Appl. 29 (2007) 954).

Each pass: filter the block with a degree-m Chebyshev polynomial of H mapped so that the
unwanted interval [a, b] goes to [-1, 1] (scaled so that the value at a0 is 1), then a
Rayleigh-Ritz step on the filtered block.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def lanczos_bounds(apply_h, v0, steps=20):
    """Plain Lanczos on one vector (no reorthogonalisation).  Returns (lower, upper):
    the smallest Ritz value and the largest Ritz value plus the norm of the last residual."""
    v = v0 / np.linalg.norm(v0)
    v_prev = np.zeros_like(v)
    beta = 0.0
    alphas, betas = [], []
    for _ in range(steps):
        w = apply_h(v[None, :])[0]
        alpha = float(np.real(np.vdot(v, w)))
        w = w - alpha * v - beta * v_prev
        beta_next = float(np.linalg.norm(w))
        alphas.append(alpha)
        betas.append(beta_next)
        v_prev, v, beta = v, w / beta_next, beta_next
    theta = sla.eigh_tridiagonal(np.array(alphas), np.array(betas[:-1]), eigvals_only=True)
    return float(theta[0]), float(theta[-1] + betas[-1])


def chebyshev_filter(apply_h, X, m, a, b, a0):
    """Degree-m scaled Chebyshev filter applied to the block X (rows are vectors):
        e = (b-a)/2, c = (b+a)/2, sigma_1 = e/(a0 - c)
        Y_1 = sigma_1/e (H - c) X
        sigma_{k+1} = 1/(2/sigma_1 - sigma_k)
        Y_{k+1} = 2 sigma_{k+1}/e (H - c) Y_k - sigma_k sigma_{k+1} Y_{k-1}
    returns Y_m."""
    e = 0.5 * (b - a)
    c = 0.5 * (b + a)
    sigma1 = e / (a0 - c)
    sigma = sigma1
    Y_prev = X
    Y = (sigma1 / e) * (apply_h(X) - c * X)
    for _ in range(2, m + 1):
        sigma_next = 1.0 / (2.0 / sigma1 - sigma)
        Y_next = (2.0 * sigma_next / e) * (apply_h(Y) - c * Y) - (sigma * sigma_next) * Y_prev
        Y_prev, Y, sigma = Y, Y_next, sigma_next
    return Y


def rayleigh_ritz(apply_h, Y):
    """Rayleigh-Ritz on span(Y): M_s = Y^H Y, H_s = Y^H (H Y), solve H_s q = lambda M_s q
    (LAPACK generalized symmetric eigensolver), X = Y Q (rows orthonormal).  Returns (lam, X)."""
    HY = apply_h(Y)
    Ms = Y.conj() @ Y.T
    Hs = Y.conj() @ HY.T
    Ms = 0.5 * (Ms + Ms.conj().T)
    Hs = 0.5 * (Hs + Hs.conj().T)
    lam, Q = sla.eigh(Hs, Ms)
    X = (Y.T @ Q).T
    return lam, X


def chefsi_pass(apply_h, X, m, a, b, a0):
    """One CheFSI pass: filter then Rayleigh-Ritz."""
    return rayleigh_ritz(apply_h, chebyshev_filter(apply_h, X, m, a, b, a0))


def residual_norms(apply_h, X, lam):
    """max-abs of H x_n - lambda_n x_n for each row."""
    R = apply_h(X) - lam[:, None] * X
    return np.max(np.abs(R), axis=1)
