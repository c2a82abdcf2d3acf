"""Failure handling on the GPU without faulting it: bounded device-side waits and host-side
input validation.  The barrier test makes a grid barrier unsatisfiable from the host (it waits
for one CTA more than the launch has), so every CTA's bounded spin runs out and the library must
return SDFT_ERR_DEVICE_TIMEOUT and keep the device usable."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import workloads  # noqa: E402
from oracle import ham, model  # noqa: E402


@pytest.fixture(scope="module")
def sd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_10431_gb300 import build
    build.build()
    import paper_2005_10431_gb300 as m
    return m


def _poisson(sd, ctx, cell):
    f = torch.from_numpy(model.sad_density(cell) + model.pseudocharge(cell)).cuda()
    phi = torch.zeros_like(f)
    sd.sdft_poisson(ctx, f, phi, 1e-10, 4000)
    return phi


def test_persistent_barrier_timeout_is_reported_not_hung(sd, monkeypatch):
    cell = workloads.two_atom_cell()
    monkeypatch.setenv("SDFT_AAR_MG", "0")   # the persistent (Jacobi) AAR kernel holds the grid barrier
    monkeypatch.setenv("SDFT_TEST_BARRIER_EXTRA", "1")
    bad = sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species, dict(nstates=8, precision=1))
    with pytest.raises(sd.SdftError) as e:
        _poisson(sd, bad, cell)
    assert e.value.code == -6
    monkeypatch.delenv("SDFT_TEST_BARRIER_EXTRA")
    # the device and a fresh context still work, and give the right answer
    good = sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species, dict(nstates=8, precision=1))
    phi = _poisson(sd, good, cell).cpu().numpy()
    ref = ham.poisson_exact(cell, model.sad_density(cell) + model.pseudocharge(cell))
    assert np.max(np.abs(phi - ref)) < 1e-8 * np.max(np.abs(ref))


def test_non_finite_density_guess_is_rejected(sd):
    cell = workloads.two_atom_cell()
    ctx = sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species, dict(nstates=8))
    rho = np.ones(cell.ngrid)
    rho[5] = np.nan
    with pytest.raises(sd.SdftError) as e:
        sd.sdft_set_density(ctx, rho)
    assert e.value.code == -7
    with pytest.raises(sd.SdftError) as e:
        sd.sdft_set_density(ctx, np.ones(cell.ngrid - 1))
    assert e.value.code == -1


def test_misaligned_allocation_callback_is_rejected(sd, monkeypatch):
    # an allocator whose blocks start 64 bytes past a 256-byte boundary: the context must refuse them
    # (the TMA copies need 16-byte aligned bases) and hand every block back, not run on them
    from paper_2005_10431_gb300 import _lib
    handed = []

    def fake(device):
        def alloc(nbytes, user):
            p = torch.cuda.caching_allocator_alloc(int(nbytes) + 256, device=device)
            handed.append(p)
            return p + 64

        def free(ptr, user):
            handed.remove(ptr - 64)
            torch.cuda.caching_allocator_delete(ptr - 64)

        return _lib.ALLOC_FN(alloc), _lib.FREE_FN(free)

    monkeypatch.setattr(sd, "_torch_allocator", fake)
    cell = workloads.two_atom_cell()
    with pytest.raises(sd.SdftError) as e:
        sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species, dict(nstates=8, precision=1))
    assert e.value.code == -1 and "256-byte aligned" in str(e.value)
    assert handed == []
