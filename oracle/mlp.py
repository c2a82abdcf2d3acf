"""FP64 reference of the learned initial-density model (test infrastructure).

The paper's SCF starts from a superposition of atomic densities and lists machine learning as
future work (Sec. 2.1, Sec. 4).  The learned guess adds a small network that predicts the
correction rho* - rho_SAD at every grid point from atom-centred radial descriptors
(Behler-Parrinello-type radial symmetry functions):

  G_j(x) = sum_a sum_T exp(-(r - mu_j)^2 / (2 eta^2)) f_c(r),  r = |x - R_a - T| <= R_c,
  f_c(r) = (cos(pi r / R_c) + 1) / 2,  mu_j = 6 j / 31 (j = 0..31),  eta = 6/31,  R_c = 6.5 bohr,

  MLP: h1 = silu(W1 G + b1) (64), h2 = silu(W2 h1 + b2) (64), y = w3 . h2 + b3,
  loss = mean over points of (y - t)^2, Adam (beta1 0.9, beta2 0.999, eps 1e-8).

Parameters are one flat vector: W1 [64 x 32] row-major, b1 [64], W2 [64 x 64], b2 [64], w3 [64], b3 [1].
Pinned by tests/test_oracle_mlp.py (finite differences of the loss; brute-force descriptors).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

NFEAT, HIDDEN = 32, 64
R_CUT = 6.5
ETA = 6.0 / 31.0
MU = 6.0 * np.arange(NFEAT) / 31.0
NPARAM = HIDDEN * NFEAT + HIDDEN + HIDDEN * HIDDEN + HIDDEN + HIDDEN + 1


def unpack(p):
    p = np.asarray(p, float)
    o = 0
    W1 = p[o:o + HIDDEN * NFEAT].reshape(HIDDEN, NFEAT); o += HIDDEN * NFEAT
    b1 = p[o:o + HIDDEN]; o += HIDDEN
    W2 = p[o:o + HIDDEN * HIDDEN].reshape(HIDDEN, HIDDEN); o += HIDDEN * HIDDEN
    b2 = p[o:o + HIDDEN]; o += HIDDEN
    w3 = p[o:o + HIDDEN]; o += HIDDEN
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, w3, [b3]])


def descriptors(cell) -> np.ndarray:
    """G [ngrid, 32] for every grid point of the cell (images summed within R_c)."""
    n = cell.n
    x = [np.arange(n[d]) * cell.h[d] for d in range(3)]
    Z, Y, X = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    G = np.zeros((P.shape[0], NFEAT))
    L = np.array(cell.L)
    for a in range(cell.natom):
        nimg = [int(math.ceil(R_CUT / L[d])) + 1 for d in range(3)]
        for t in itertools.product(*[range(-k, k + 1) for k in nimg]):
            d = P - (cell.pos[a] + np.array(t) * L)
            r = np.sqrt(np.sum(d * d, axis=1))
            m = r <= R_CUT
            if not np.any(m):
                continue
            rr = r[m]
            fc = 0.5 * (np.cos(np.pi * rr / R_CUT) + 1.0)
            G[m] += np.exp(-((rr[:, None] - MU[None, :]) ** 2) / (2 * ETA * ETA)) * fc[:, None]
    return G


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(G, p):
    W1, b1, W2, b2, w3, b3 = unpack(p)
    z1 = G @ W1.T + b1
    h1 = silu(z1)
    z2 = h1 @ W2.T + b2
    h2 = silu(z2)
    return h2 @ w3 + b3


def loss_grad(G, t, p):
    """Mean-squared loss and its gradient with respect to the flat parameter vector."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    npt = G.shape[0]
    z1 = G @ W1.T + b1
    h1 = silu(z1)
    z2 = h1 @ W2.T + b2
    h2 = silu(z2)
    y = h2 @ w3 + b3
    e = y - t
    loss = float(np.mean(e * e))
    dy = 2.0 * e / npt
    gw3 = h2.T @ dy
    gb3 = float(np.sum(dy))
    dz2 = (dy[:, None] * w3[None, :]) * dsilu(z2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * dsilu(z1)
    gW1 = dz1.T @ G
    gb1 = dz1.sum(axis=0)
    return loss, pack(gW1, gb1, gW2, gb2, gw3, gb3)


def adam(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (bias-corrected), step counted from 1; returns (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
