"""Pins of the Kerker-preconditioned Pulay oracle (oracle/kerker.py) against facts that do not
come from its FFT path: eigenvalues of plane waves measured with the real-space FD stencil, the
uniform mode, the screened-Poisson identity checked with the real-space Laplacian, and the plain
Pulay mixer it must reduce to when k0 = 0."""
import numpy as np
import pytest

import workloads
from oracle import fd, kerker, scf


def _cell():
    c = workloads.small_cell(npts=12, L=4.0, natom=1, seed=3, nstates=4)
    c.n = (12, 10, 8)
    c.L = (4.0, 3.5, 3.0)
    return c


def _grid(c):
    z, y, x = np.meshgrid(*[np.arange(c.n[d]) * c.h[d] for d in (2, 1, 0)], indexing="ij")
    return x, y, z


@pytest.mark.parametrize("m", [(1, 0, 0), (0, 2, 1), (3, 1, 2), (6, 0, 0)])
@pytest.mark.parametrize("k0", [0.5, 1.3])
def test_plane_wave_factor_matches_real_space_eigenvalue(m, k0):
    c = _cell()
    x, y, z = _grid(c)
    f = np.cos(2 * np.pi * (m[0] * x / c.L[0] + m[1] * y / c.L[1] + m[2] * z / c.L[2]))
    Lf = fd.laplacian(f, c.h)
    lam = -float(np.sum(Lf * f) / np.sum(f * f))     # f is an eigenvector of the periodic stencil
    assert np.max(np.abs(Lf + lam * f)) < 1e-9 * max(lam, 1.0)
    Pf = kerker.kerker(c, f.reshape(-1), k0).reshape(f.shape)
    assert np.max(np.abs(Pf - lam / (lam + k0 * k0) * f)) < 1e-12


def test_uniform_mode_removed_and_identity_at_zero_screening():
    c = _cell()
    one = np.ones(c.ngrid)
    assert np.max(np.abs(kerker.kerker(c, one, 0.8))) < 1e-13
    f = np.random.default_rng(1).normal(size=c.ngrid)
    assert np.max(np.abs(kerker.kerker(c, f, 0.0) - f)) < 1e-13


@pytest.mark.parametrize("k0", [0.3, 1.0, 2.5])
def test_screened_poisson_identity(k0):
    """y = (f - P f) / k0^2 solves (-L_h + k0^2) y = f, checked with the real-space stencil."""
    c = _cell()
    f = np.random.default_rng(2).normal(size=c.ngrid)
    y = (f - kerker.kerker(c, f, k0)) / (k0 * k0)
    lhs = -fd.laplacian(y.reshape(c.n[::-1]), c.h).reshape(-1) + k0 * k0 * y
    assert np.max(np.abs(lhs - f)) < 1e-10 * np.max(np.abs(f))


def test_channels_are_preconditioned_independently():
    c = _cell()
    f = np.random.default_rng(3).normal(size=(2, c.ngrid))
    both = kerker.kerker(c, f, 0.7)
    assert np.array_equal(both[0], kerker.kerker(c, f[0], 0.7))
    assert np.array_equal(both[1], kerker.kerker(c, f[1], 0.7))


@pytest.mark.parametrize("period,restart", [(1, False), (2, True)])
def test_mixer_reduces_to_plain_pulay_without_screening(period, restart):
    c = _cell()
    rng = np.random.default_rng(4)
    a = kerker.KerkerPulayMixer(c, k0=0.0, beta=0.3, hist=4, period=period, restart=restart)
    b = scf.PulayMixer(beta=0.3, hist=4, period=period, restart=restart)
    x = rng.normal(size=c.ngrid)
    for _ in range(8):
        x_out = 0.6 * x + rng.normal(size=c.ngrid) * 0.1
        xa, xb = a.update(x, x_out), b.update(x, x_out)
        assert np.max(np.abs(xa - xb)) < 1e-11 * np.max(np.abs(xb))
        x = xb


def test_linear_step_damps_long_waves_more_than_short_waves():
    """The first (linear) step moves a long-wave residual by beta * lam/(lam + k0^2) of itself and a
    short-wave one by nearly beta: the long wave is damped."""
    c = _cell()
    x, y, z = _grid(c)
    for m, expect_small in ((1, True), (5, False)):
        f = np.cos(2 * np.pi * m * x / c.L[0]).reshape(-1)
        mix = kerker.KerkerPulayMixer(c, k0=3.0, beta=0.5)
        step = mix.update(np.zeros(c.ngrid), f)
        ratio = float(np.dot(step, f) / np.dot(f, f)) / 0.5
        assert (ratio < 0.5) == expect_small


def test_pulay_step_matches_columnwise_preconditioned_form():
    """With screening, a Pulay step equals x + P(beta f) - (X + P(beta F)) gamma evaluated column by
    column (the mixer uses the equivalent optimal-residual form x - X gamma + P(beta (f - F gamma)))."""
    c = _cell()
    rng = np.random.default_rng(6)
    k0, beta = 0.9, 0.4
    mix = kerker.KerkerPulayMixer(c, k0=k0, beta=beta, hist=3)
    xs, fs = [], []
    x = rng.normal(size=c.ngrid)
    for it in range(5):
        x_out = 0.5 * x + 0.2 * rng.normal(size=c.ngrid)
        f = x_out - x
        xs.append(x.copy())
        fs.append(f)
        x_new = mix.update(x, x_out)
        if it > 0:
            X = np.array([xs[j] - xs[j - 1] for j in range(max(1, it - 2), it + 1)]).T
            F = np.array([fs[j] - fs[j - 1] for j in range(max(1, it - 2), it + 1)]).T
            gamma = np.linalg.lstsq(F, f, rcond=None)[0]
            PF = np.stack([kerker.kerker(c, beta * F[:, j], k0) for j in range(F.shape[1])], axis=1)
            ref = x + kerker.kerker(c, beta * f, k0) - (X + PF) @ gamma
            assert np.max(np.abs(x_new - ref)) < 1e-10 * np.max(np.abs(ref))
        x = x_new
