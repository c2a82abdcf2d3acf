"""Pins of the learned-guess oracle (oracle/mlp.py) against facts outside it:
finite differences of its own loss (gradient), a brute-force per-point descriptor loop written with
scalar math, the single-atom closed form of a descriptor, permutation under a lattice translation,
and Adam's closed form for a constant gradient.
"""
import math

import numpy as np
import pytest

import workloads
from oracle import mlp



def _rand_params(seed, scale=0.4):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, mlp.NPARAM)


def test_parameter_count_and_layout():
    assert mlp.NPARAM == 6337 == workloads.MLP_NPARAM
    p = np.arange(mlp.NPARAM, dtype=float)
    W1, b1, W2, b2, w3, b3 = mlp.unpack(p)
    assert W1.shape == (64, 32) and W1[1, 0] == 32 and b1[0] == 2048
    assert W2.shape == (64, 64) and W2[0, 1] == 2048 + 64 + 1
    assert b3 == mlp.NPARAM - 1
    np.testing.assert_array_equal(mlp.pack(W1, b1, W2, b2, w3, b3), p)


def test_silu_derivative_and_special_values():
    z = np.linspace(-6, 6, 41)
    h = 1e-5
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.dsilu(z), fd, atol=1e-9)
    assert mlp.silu(np.array(0.0)) == 0.0 and mlp.dsilu(np.array(0.0)) == 0.5


def test_forward_with_zero_weights_is_the_bias_chain():
    p = np.zeros(mlp.NPARAM)
    W1, b1, W2, b2, w3, b3 = mlp.unpack(p)
    b2[:] = 0.7
    w3[:] = 0.25
    G = np.random.default_rng(1).normal(size=(5, 32))
    y = mlp.forward(G, mlp.pack(W1, b1, W2, b2, w3, 0.3))
    np.testing.assert_allclose(y, 0.3 + 64 * 0.25 * 0.7 / (1 + math.exp(-0.7)), rtol=1e-14)


def test_loss_gradient_matches_central_differences():
    rng = np.random.default_rng(7)
    G = rng.uniform(0.0, 1.5, size=(9, 32))
    t = rng.normal(0.0, 0.3, size=9)
    p = _rand_params(3)
    loss, g = mlp.loss_grad(G, t, p)
    np.testing.assert_allclose(loss, np.mean((mlp.forward(G, p) - t) ** 2), rtol=1e-14)
    h = 1e-6
    fd = np.empty(mlp.NPARAM)
    for i in range(mlp.NPARAM):
        e = np.zeros(mlp.NPARAM)
        e[i] = h
        fd[i] = (mlp.loss_grad(G, t, p + e)[0] - mlp.loss_grad(G, t, p - e)[0]) / (2 * h)
    scale = np.max(np.abs(fd))
    assert np.max(np.abs(g - fd)) < 1e-7 * scale
    # every block is exercised (no block of the gradient is identically zero)
    W1, b1, W2, b2, w3, b3 = mlp.unpack(g)
    for blk in (W1, b1, W2, b2, w3, np.array([b3])):
        assert np.max(np.abs(blk)) > 1e-6 * scale


def _descriptor_brute(cell, idx):
    """Scalar loops over points, atoms and every image within range, with math.exp/math.cos."""
    n, h, L = cell.n, cell.h, cell.L
    out = np.zeros((len(idx), 32))
    for row, g in enumerate(idx):
        i, j, k = g % n[0], (g // n[0]) % n[1], g // (n[0] * n[1])
        x = (i * h[0], j * h[1], k * h[2])
        for a in range(cell.natom):
            for t0 in range(-4, 5):
                for t1 in range(-4, 5):
                    for t2 in range(-4, 5):
                        d = [x[0] - cell.pos[a][0] - t0 * L[0], x[1] - cell.pos[a][1] - t1 * L[1],
                             x[2] - cell.pos[a][2] - t2 * L[2]]
                        r = math.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
                        if r > 6.5:
                            continue
                        fc = 0.5 * (math.cos(math.pi * r / 6.5) + 1.0)
                        for q in range(32):
                            mu = 6.0 * q / 31.0
                            eta = 6.0 / 31.0
                            out[row, q] += math.exp(-(r - mu) ** 2 / (2 * eta * eta)) * fc
    return out


def test_descriptors_match_brute_force_on_a_small_cell():
    cell = workloads.small_cell(npts=7, L=3.1, natom=2, seed=4)
    cell.n = (5, 6, 7)
    G = mlp.descriptors(cell)
    idx = np.random.default_rng(0).choice(cell.ngrid, 25, replace=False)
    np.testing.assert_allclose(G[idx], _descriptor_brute(cell, idx), rtol=1e-12, atol=1e-14)


def test_descriptor_single_atom_closed_form():
    """One atom in a box wider than 2 R_c: only the nearest image contributes."""
    cell = workloads.small_cell(npts=8, L=16.0, natom=1, seed=1)
    cell.pos = np.array([[4.0, 2.0, 6.0]])
    G = mlp.descriptors(cell)
    n, h = cell.n, cell.h
    g = 3 + n[0] * (1 + n[1] * 5)
    x = np.array([3 * h[0], 1 * h[1], 5 * h[2]])
    r = np.linalg.norm(x - cell.pos[0])
    fc = 0.5 * (np.cos(np.pi * r / 6.5) + 1)
    expect = np.exp(-(r - 6.0 * np.arange(32) / 31) ** 2 / (2 * (6 / 31) ** 2)) * fc
    np.testing.assert_allclose(G[g], expect, rtol=1e-13)
    # far from the atom (beyond R_c in every image) all features vanish
    far = 7 + n[0] * (7 + n[1] * 1)      # point (14, 14, 2): distance to the atom > 6.5
    assert np.linalg.norm(np.array([14.0, 14.0, 2.0]) - cell.pos[0]) > 6.5
    assert np.all(G[far] == 0.0)


def test_descriptors_permute_under_a_grid_translation():
    cell = workloads.small_cell(npts=6, L=4.2, natom=2, seed=9)
    G = mlp.descriptors(cell)
    shifted = workloads.small_cell(npts=6, L=4.2, natom=2, seed=9)
    shifted.pos = cell.pos + np.array([cell.h[0], 0.0, 0.0])
    G2 = mlp.descriptors(shifted)
    n = cell.n
    G_grid = G.reshape(n[2], n[1], n[0], 32)
    G2_grid = G2.reshape(n[2], n[1], n[0], 32)
    np.testing.assert_allclose(np.roll(G_grid, 1, axis=2), G2_grid, rtol=1e-10, atol=1e-13)


def test_adam_constant_gradient_closed_form():
    p0 = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -1e-3, 2.0])
    m = np.zeros(3)
    v = np.zeros(3)
    p = p0.copy()
    for step in range(1, 6):
        p, m, v = mlp.adam(p, g, m, v, step, lr=0.01)
    # bias-corrected moments equal g and g^2 for a constant gradient
    np.testing.assert_allclose(p, p0 - 5 * 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_adam_training_reduces_the_loss_on_a_smooth_target():
    rng = np.random.default_rng(2)
    G = rng.uniform(0, 1, size=(64, 32))
    t = np.sin(G[:, 0] * 3) * 0.2 + 0.1 * G[:, 5]
    p = workloads.mlp_init_params(11).astype(float)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    l0 = mlp.loss_grad(G, t, p)[0]
    for step in range(1, 301):
        loss, g = mlp.loss_grad(G, t, p)
        p, m, v = mlp.adam(p, g, m, v, step, lr=3e-3)
    assert mlp.loss_grad(G, t, p)[0] < 0.05 * l0
