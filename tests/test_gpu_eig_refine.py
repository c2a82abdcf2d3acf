"""The refined subspace eigensolver (real, 64 < n <= 1024): an FP32 Cholesky + Jacobi solve in one
CTA (n <= 160; cuSOLVER's FP32 sygvd above), two FP64 Ogita-Aishima refinement steps and an FP64
Rayleigh-Ritz inside clusters of (near-)degenerate eigenvalues.  SDFT_EIGEN=2 forces it and turns a rejected result into an error
instead of the cuSOLVER fallback, so these tests see the refined path itself."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_10431_gb300 as m
    return m


def _problem(n, seed, clusters=((2, 0.0), (3, 1e-7), (6, 0.0), (4, 1e-5))):
    """H, M with generalized eigenvalues that include exactly and nearly degenerate groups; M has
    the column scales of a filtered block (condition ~1e4 before equilibration)."""
    rng = np.random.default_rng(seed)
    lam = np.sort(rng.normal(size=n))
    p = 3
    for k, spread in clusters:
        if p + k > n:
            break
        lam[p:p + k] = lam[p] + spread * rng.normal(size=k)
        p += k + 17
    lam = np.sort(lam)
    B = rng.normal(size=(3 * n, n)) * np.logspace(0, -2, n)
    M = B.T @ B
    L = np.linalg.cholesky(M)
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    H = L @ Q @ np.diag(lam) @ Q.T @ L.T
    return 0.5 * (H + H.T), M


def _indefinite(n):
    # positive diagonal, indefinite (a 2 x 2 minor with |M_56| > sqrt(M_55 M_66))
    H, M = _problem(n, 3)
    M[5, 6] = M[6, 5] = 2.0 * np.sqrt(M[5, 5] * M[6, 6])
    return H, M


def _solve(sd, n, H, M):
    cell = workloads.small_cell(npts=6, L=3.0, natom=1, seed=1, nstates=n + 1)
    ctx = sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species,
                         dict(nstates=n + 1, precision=sd.SDFT_FP64))
    m = torch.from_numpy(np.ascontiguousarray(M.T)).cuda()
    h = torch.from_numpy(np.ascontiguousarray(H.T)).cuda()
    eig = torch.zeros(n, dtype=torch.float64, device="cuda")
    sd.sdft_subspace_eig(ctx, False, m, h, eig, n)
    out = eig.cpu().numpy(), h.cpu().numpy().T
    sd.sdft_destroy(ctx)
    return out


@pytest.mark.parametrize("n", [65, 100, 154, 160, 180, 300])
def test_refined_eig_matches_lapack(sd, n, monkeypatch):
    import scipy.linalg as sla
    monkeypatch.setenv("SDFT_EIGEN", "2")
    H, M = _problem(n, 11 + n)
    lam_ref, _ = sla.eigh(H, M)
    lam, Q = _solve(sd, n, H, M)
    scale = np.max(np.abs(lam_ref))
    assert np.all(np.diff(lam) >= -1e-12 * scale)
    assert np.max(np.abs(lam - lam_ref)) < 1e-11 * scale
    assert np.max(np.abs(Q.T @ M @ Q - np.eye(n))) < 1e-10
    assert np.max(np.abs(H @ Q - M @ Q * lam[None, :])) < 1e-9 * scale * np.max(np.abs(M))


def test_refined_eig_degenerate_spectrum(sd, monkeypatch):
    """A 12-fold exactly degenerate eigenvalue and a 24-fold one (the cluster solve is exact in
    FP64 inside each group): eigenvalues and the M-orthonormality still hold to FP64 accuracy."""
    import scipy.linalg as sla
    monkeypatch.setenv("SDFT_EIGEN", "2")
    n = 120
    H, M = _problem(n, 5, clusters=((12, 0.0), (24, 0.0)))
    lam_ref, _ = sla.eigh(H, M)
    lam, Q = _solve(sd, n, H, M)
    scale = np.max(np.abs(lam_ref))
    assert np.max(np.abs(lam - lam_ref)) < 1e-11 * scale
    assert np.max(np.abs(Q.T @ M @ Q - np.eye(n))) < 1e-10
    assert np.max(np.abs(H @ Q - M @ Q * lam[None, :])) < 1e-9 * scale * np.max(np.abs(M))


def test_refined_eig_rejects_indefinite_overlap(sd, monkeypatch):
    monkeypatch.setenv("SDFT_EIGEN", "2")
    n = 70
    H, M = _indefinite(n)
    with pytest.raises(sd.SdftError) as e:
        _solve(sd, n, H, M)
    assert e.value.code == -5


def test_default_falls_back_on_indefinite_overlap(sd):
    """Default method on a mixed-precision context: the refined solver rejects the indefinite M and
    cuSOLVER, which the caller falls back to, reports it."""
    n = 70
    H, M = _indefinite(n)
    cell = workloads.small_cell(npts=6, L=3.0, natom=1, seed=1, nstates=n + 2)
    ctx = sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species,
                         dict(nstates=n + 2, precision=sd.SDFT_MIXED))
    m = torch.from_numpy(np.ascontiguousarray(M.T)).cuda()
    h = torch.from_numpy(np.ascontiguousarray(H.T)).cuda()
    eig = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(sd.SdftError) as e:
        sd.sdft_subspace_eig(ctx, False, m, h, eig, n)
    assert e.value.code == -5
    sd.sdft_destroy(ctx)


def test_mixed_scf_refined_vs_cusolver(sd, monkeypatch):
    """Mixed-precision SCF of the displaced 8-atom lattice with 72 states (Rayleigh-Ritz n = 72):
    the refined eigensolver (never rejected: SDFT_EIGEN=2 would raise) and cuSOLVER's sygvd reach
    the same free energy and eigenvalues."""
    cell = workloads.qmd_lattice8_cell(5)
    cell.nstates = 72
    res = {}
    for method in ("2", "0"):
        monkeypatch.setenv("SDFT_EIGEN", method)
        ctx = sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species,
                             dict(nstates=cell.nstates, cheb_degree=cell.cheb_degree, precision=sd.SDFT_MIXED,
                                  scf_tol=1e-5, max_scf=80, seed=cell.seed))
        r = sd.sdft_scf(ctx)
        res[method] = (r["energy"], r["converged"], sd.sdft_get_eigenvalues(ctx))
        sd.sdft_destroy(ctx)
    assert res["2"][1] and res["0"][1]
    assert abs(res["2"][0] - res["0"][0]) / cell.natom < 1e-6
    assert np.max(np.abs(res["2"][2] - res["0"][2])[:40]) < 1e-5
