"""GPU parity of the PBE GGA exchange-correlation (paper Sec. 2.2 functionalities) against the FP64
oracle (oracle/gga.py): the pointwise functional and the discrete gradient/divergence elementwise, and
the PBE SCF of the two-atom cell against the oracle's converged reference
(tests/golden/two_atom_24_pbe.json).  FP64 bounds: 1e-11 relative for one evaluation (the analytic
derivatives of the GPU against the oracle's complex-step ones), 1e-9 Ha/atom and 1e-8 Ha for the SCF;
mixed precision: 1e-5 Ha/atom and 1e-5 Ha."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import workloads  # noqa: E402
from oracle import gga  # noqa: E402

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
    c.n = (14, 12, 10)
    c.L = (4.2, 3.9, 3.3)
    c.xc = "gga_pbe"
    return c


def test_pbe_xc_matches_oracle(sd):
    cell = _cell()
    ctx = sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species,
                         dict(nstates=4, precision=sd.SDFT_FP64, xc=sd.SDFT_XC_GGA_PBE))
    z, y, x = np.meshgrid(*[np.arange(cell.n[d]) * cell.h[d] for d in (2, 1, 0)], indexing="ij")
    rng = np.random.default_rng(9)
    rho = (0.04 + 0.03 * np.cos(2 * np.pi * x / cell.L[0]) * np.cos(4 * np.pi * z / cell.L[2]) ** 2
           + 0.005 * rng.uniform(size=x.shape)).reshape(-1)
    exc_ref, vxc_ref = gga.pbe_unpolarized(cell, rho)
    r = torch.from_numpy(rho.copy()).cuda()
    exc = torch.empty_like(r)
    vxc = torch.empty_like(r)
    sd.sdft_lda(ctx, 1, r, exc, vxc, cell.ngrid)
    e, v = exc.cpu().numpy(), vxc.cpu().numpy()
    assert np.max(np.abs(e - exc_ref)) < 1e-11 * np.max(np.abs(exc_ref))
    assert np.max(np.abs(v - vxc_ref)) < 1e-11 * np.max(np.abs(vxc_ref))
    # the gradient term matters here: the PBE potential differs from the LDA one by far more than the bound
    from oracle import xc
    _, v_lda = xc.lda_pz_unpolarized(rho)
    assert np.max(np.abs(v - v_lda)) > 1e-3


def test_pbe_rejects_spin_polarised_contexts(sd):
    cell = _cell()
    with pytest.raises(sd.SdftError):
        sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species,
                       dict(nstates=4, precision=sd.SDFT_FP64, xc=sd.SDFT_XC_GGA_PBE, nspin=2))


@pytest.mark.parametrize("precision", [0, 1])
def test_pbe_scf_two_atom_matches_oracle(sd, precision):
    g = json.load(open(os.path.join(HERE, "golden", "two_atom_24_pbe.json")))
    cell = workloads.two_atom_cell()
    fp64 = precision == sd.SDFT_FP64
    ctx = sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species,
                         dict(nstates=cell.nstates, cheb_degree=cell.cheb_degree, precision=precision,
                              scf_tol=1e-10 if fp64 else 1e-6, max_scf=300, kT=cell.kT, seed=cell.seed,
                              xc=sd.SDFT_XC_GGA_PBE, final_fp64_pass=0 if fp64 else 1))
    r = sd.sdft_scf(ctx)
    assert r["converged"]
    tol_e, tol_eig, tol_f = (1e-9, 1e-8, 1e-6) if fp64 else (1e-5, 1e-5, 1e-4)
    assert abs(r["energy"] - g["energy"]) / cell.natom < tol_e
    eig = sd.sdft_get_eigenvalues(ctx)[0, 0]
    occ = np.array(g["occ"])[0, 0]
    nocc = int(np.sum(occ > 1e-10))
    assert np.max(np.abs(eig[:nocc] - np.array(g["eigs"])[0, 0, :nocc])) < tol_eig
    assert np.max(np.abs(sd.sdft_get_forces(ctx) - np.array(g["forces"]))) < tol_f
