"""Pins of the MD density extrapolation oracle (oracle/extrapolation.py)."""
import numpy as np

from oracle import extrapolation as ex


def _traj(kind, rng, n=6):
    R0 = rng.uniform(0, 10, (n, 3))
    v = rng.normal(0, 0.1, (n, 3))
    a = rng.normal(0, 0.05, (n, 3))
    if kind == "velocity":
        return [R0 + v * t for t in range(4)]
    return [R0 + v * t + 0.5 * a * t * t for t in range(4)]


def test_constant_velocity_gives_linear_extrapolation():
    rng = np.random.default_rng(0)
    R = _traj("velocity", rng)
    # collinear displacements: one-term fit alpha = 1
    assert np.allclose(ex.alfe_coefficients(R[3], [R[2], R[1], R[0]], (10, 10, 10)), (1.0, 0.0), atol=1e-12)
    assert np.allclose(ex.alfe_coefficients(R[3], [R[2], R[1]], (10, 10, 10)), (1.0, 0.0), atol=1e-12)


def test_uniform_acceleration_is_fitted_exactly():
    # R(t+1) - R(t) = 2 (R(t) - R(t-1)) - (R(t-1) - R(t-2)) for every atom
    rng = np.random.default_rng(1)
    R = _traj("accel", rng)
    a, b = ex.alfe_coefficients(R[3], [R[2], R[1], R[0]], (10, 10, 10))
    assert abs(a - 2.0) < 1e-10 and abs(b + 1.0) < 1e-10


def test_periodic_images_do_not_change_the_fit():
    rng = np.random.default_rng(2)
    L = np.array([7.0, 8.0, 9.0])
    R = _traj("accel", rng)
    shifted = [r + L * rng.integers(-2, 3, r.shape) for r in R]
    assert np.allclose(ex.alfe_coefficients(R[3], [R[2], R[1], R[0]], L),
                       ex.alfe_coefficients(shifted[3], [shifted[2], shifted[1], shifted[0]], L), atol=1e-10)


def test_static_correction_passes_through_and_electrons_are_conserved():
    rng = np.random.default_rng(3)
    sad = rng.uniform(0.5, 1.5, (1, 64))
    D = rng.normal(0, 0.05, (1, 64))
    D -= D.mean()
    g = ex.extrapolated_density(sad, [D, D, D], 0.7, -0.2, nelec=sad.sum() * 0.1, dV=0.1)
    assert np.allclose(g, sad + D, atol=1e-13)
    g = ex.extrapolated_density(sad, [D, 0.5 * D, 0.2 * D], 1.3, -0.4, nelec=12.0, dV=0.1)
    assert abs(0.1 * g.sum() - 12.0) < 1e-12 and g.min() >= 0.0
