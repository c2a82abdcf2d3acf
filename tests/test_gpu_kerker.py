"""GPU parity of the Kerker-preconditioned mixing (paper Sec. 2.1: periodic Pulay mixing with a
real-space preconditioner of Kerker type) against the FP64 oracle (oracle/kerker.py, which applies
P = (-L_h)(-L_h + k0^2)^-1 through the FD symbol and FFTs, while the GPU solves the screened Poisson
equation by AAR in real space).

Tolerances: the GPU solve stops at a relative residual of 1e-11 (preconditioner test) or 1e-10 (the
solve inside the mixer); the error of P f is then a few 1e-10 of max|f|, which the 1e-8 / 1e-7 bounds
below cover with room.  The SCF test compares converged free energies, which do not depend on the
mixer, at the FP64 bound of 1e-9 Ha/atom.
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import workloads  # noqa: E402
from oracle import kerker  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def sd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_10431_gb300 import build
    build.build()
    import paper_2005_10431_gb300 as m
    return m


def _cell():
    c = workloads.small_cell(npts=12, L=4.0, natom=1, seed=3, nstates=4)
    c.n = (12, 10, 8)
    c.L = (4.0, 3.5, 3.0)
    return c


def _ctx(sd, cell, nspin=1, **opts):
    return sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species,
                          dict(nstates=cell.nstates, precision=sd.SDFT_FP64, nspin=nspin, **opts))


@pytest.mark.parametrize("k0", [0.5, 1.3])
def test_kerker_preconditioner_matches_oracle(sd, k0):
    cell = _cell()
    ctx = _ctx(sd, cell)
    f = np.random.default_rng(7).normal(size=(2, cell.ngrid))
    fd_ = torch.from_numpy(f.copy()).cuda()
    out = torch.empty_like(fd_)
    sd.sdft_kerker(ctx, fd_, out, nchan=2, k0=k0, tol=1e-11)
    ref = kerker.kerker(cell, f, k0)
    err = np.max(np.abs(out.cpu().numpy() - ref)) / np.max(np.abs(f))
    assert err < 1e-8
    # the uniform mode is removed: each channel of P f has zero mean
    assert np.max(np.abs(out.cpu().numpy().mean(axis=1))) < 1e-10 * np.max(np.abs(f))


@pytest.mark.parametrize("nspin", [1, 2])
@pytest.mark.parametrize("period,restart", [(1, False), (2, True)])
def test_kerker_pulay_steps_match_oracle(sd, nspin, period, restart):
    # a sequence of (x_in, x_out) pairs through the GPU mixer and the oracle mixer, step by step
    cell = _cell()
    k0, beta, hist = 0.9, 0.4, 3
    ctx = _ctx(sd, cell, nspin=nspin, kerker_k0=k0, mix_beta=beta, mix_hist=hist, pulay_period=period,
               pulay_restart=1 if restart else 0)
    mix = kerker.KerkerPulayMixer(cell, k0=k0, beta=beta, hist=hist, period=period, restart=restart, nchan=nspin)
    rng = np.random.default_rng(11)
    nv = nspin * cell.ngrid
    x = 1.0 + 0.1 * rng.normal(size=nv)
    for _ in range(7):
        x_out = 0.5 * x + 0.5 + 0.05 * rng.normal(size=nv)
        ref = mix.update(x.copy(), x_out.copy())
        xi, xo = torch.from_numpy(x.copy()).cuda(), torch.from_numpy(x_out.copy()).cuda()
        xn = torch.empty_like(xi)
        sd.sdft_mix_step(ctx, xi, xo, xn)
        got = xn.cpu().numpy()
        assert np.max(np.abs(got - ref)) < 1e-7 * np.max(np.abs(ref))
        x = ref


def test_kerker_mixed_scf_reaches_the_oracle_fixed_point(sd):
    # the converged energy does not depend on the mixer: Kerker-preconditioned FP64 SCF of the two-atom
    # cell against the oracle reference (tests/golden/two_atom_24.json, plain Pulay)
    cell = workloads.two_atom_cell()
    g = json.load(open(os.path.join(HERE, "golden", "two_atom_24.json")))
    ctx = sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species,
                         dict(nstates=cell.nstates, cheb_degree=cell.cheb_degree, precision=sd.SDFT_FP64,
                              scf_tol=1e-10, max_scf=300, kT=cell.kT, seed=cell.seed, kerker_k0=0.8))
    r = sd.sdft_scf(ctx)
    assert r["converged"]
    assert abs(r["energy"] - g["energy"]) / cell.natom < 1e-9
    assert np.max(np.abs(sd.sdft_get_forces(ctx) - np.array(g["forces"]))) < 1e-6
