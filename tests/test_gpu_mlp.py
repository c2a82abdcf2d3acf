"""Learned initial density on the GPU against the FP64 oracle (oracle/mlp.py).

Descriptors: BF16 features within one BF16 rounding of the FP64 descriptors.  Network kernels:
the GPU rounds parameters to BF16 and computes in FP32; the oracle is evaluated in FP64 on the
same BF16-rounded parameters and BF16 features, so the remaining difference is FP32 rounding.
Gradients: every parameter block within 1e-3 of its largest entry, cosine >= 0.99999.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import workloads  # noqa: E402
from oracle import mlp as omlp  # noqa: E402

P_MULT = 1000003


@pytest.fixture(scope="module")
def sd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_10431_gb300 import build
    build.build()
    import paper_2005_10431_gb300 as m
    return m


def bf16_round(x):
    """Round FP32 values to BF16 (nearest, ties to even) and return them as float64."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def bf16_bits(x):
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    return ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint16)


def bits_to_float(bits):
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def _features(npts, seed):
    rng = np.random.default_rng(seed)
    # magnitudes like the descriptors: sums of a few Gaussians, zero beyond the cutoff
    G = rng.gamma(0.6, 0.7, size=(npts, 32)) * (rng.uniform(size=(npts, 32)) < 0.7)
    return bf16_bits(G)


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dtype, device="cuda")


def _dev_bits(bits):
    return torch.from_numpy(np.ascontiguousarray(bits.view(np.int16))).cuda()


def _check_grad(g, gref):
    for k, (a, b) in enumerate(zip(omlp.unpack(g), omlp.unpack(gref))):
        a, b = np.atleast_1d(a).ravel(), np.atleast_1d(b).ravel()
        assert np.max(np.abs(a - b)) <= 1e-3 * np.max(np.abs(b)) + 1e-12, f"block {k}"
    cos = g @ gref / (np.linalg.norm(g) * np.linalg.norm(gref))
    assert cos >= 0.99999


def test_descriptors_and_target_match_oracle(sd):
    cell = workloads.small_cell(npts=12, L=5.0, natom=3, seed=21, nstates=8)
    cell.n = (18, 19, 20)
    ctx = sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species,
                         dict(nstates=8, precision=sd.SDFT_FP64, scf_tol=1e-6))
    ng = cell.ngrid
    feat = torch.zeros((ng, 32), dtype=torch.int16, device="cuda")
    sd.sdft_mlp_dataset(ctx, feat)
    G = bits_to_float(feat.cpu().numpy().view(np.uint16))
    Gref = omlp.descriptors(cell)
    # one BF16 rounding of an FP32 evaluation: relative 2^-8, plus FP32 underflow of tails
    assert np.all(np.abs(G - Gref) <= 2.0 ** -8 * np.abs(Gref) + 1e-30)
    # target after an SCF: rho_out - rho_SAD (FP32)
    r = sd.sdft_scf(ctx)
    assert r["converged"]
    target = torch.zeros(ng, dtype=torch.float32, device="cuda")
    sd.sdft_mlp_dataset(ctx, feat, target)
    want = sd.sdft_get_density(ctx).reshape(-1, ng).sum(axis=0) - sd.sdft_get_sad_density(ctx)
    np.testing.assert_allclose(target.cpu().numpy(), want, rtol=1e-6, atol=1e-7 * np.max(np.abs(want)))


@pytest.mark.parametrize("npts", [1, 63, 1000, 4097])
def test_forward_matches_oracle(sd, npts):
    bits = _features(npts, seed=npts)
    p = workloads.mlp_init_params(5) * 2.0
    p[2048:2112] = 0.1
    y = torch.full((npts,), float("nan"), dtype=torch.float32, device="cuda")
    sd.sdft_mlp_forward(_dev_bits(bits), npts, _dev(p, torch.float32), y)
    yref = omlp.forward(bits_to_float(bits), bf16_round(p))
    np.testing.assert_allclose(y.cpu().numpy(), yref, rtol=0, atol=2e-5 * max(1.0, np.max(np.abs(yref))))


@pytest.mark.parametrize("npts,batch,start", [(1000, 1000, 0), (4097, 777, 3500), (130, 64, 129)])
def test_loss_grad_matches_oracle(sd, npts, batch, start):
    bits = _features(npts, seed=11)
    t = np.random.default_rng(3).normal(0, 0.05, npts).astype(np.float32)
    p = workloads.mlp_init_params(9) * 1.5
    p[2048:2112] = np.linspace(-0.2, 0.2, 64)
    grad = torch.full((omlp.NPARAM,), float("nan"), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    sd.sdft_mlp_loss_grad(_dev_bits(bits), _dev(t, torch.float32), npts, batch, start, _dev(p, torch.float32),
                          grad, loss)
    idx = (((start + np.arange(batch)) % npts) * P_MULT) % npts
    assert len(np.unique(idx)) == batch
    lref, gref = omlp.loss_grad(bits_to_float(bits)[idx], t[idx].astype(np.float64), bf16_round(p))
    assert abs(loss.item() - lref) <= 1e-5 * lref
    _check_grad(grad.cpu().numpy().astype(np.float64), gref)


def test_adam_and_train_loop_match_oracle(sd):
    npts, batch = 3000, 1024
    bits = _features(npts, seed=4)
    G = bits_to_float(bits)
    t = (0.05 * np.tanh(G[:, 3] - G[:, 10])).astype(np.float32)
    p0 = workloads.mlp_init_params(2)
    params = _dev(p0, torch.float32)
    grad = torch.zeros(omlp.NPARAM, dtype=torch.float32, device="cuda")
    m = torch.zeros_like(grad)
    v = torch.zeros_like(grad)
    nsteps, lr = 4, 1e-3
    loss = torch.zeros(nsteps, dtype=torch.float64, device="cuda")
    sd.sdft_mlp_train(_dev_bits(bits), _dev(t, torch.float32), npts, batch, params, grad, m, v, 1, nsteps, lr, loss)
    # oracle: the same batches, FP64 Adam on the FP32 master weights
    pr, mr, vr = p0.astype(np.float64), np.zeros(omlp.NPARAM), np.zeros(omlp.NPARAM)
    losses = []
    for step in range(1, nsteps + 1):
        s = (step - 1) * batch % npts
        idx = (((s + np.arange(batch)) % npts) * P_MULT) % npts
        lr_, g = omlp.loss_grad(G[idx], t[idx].astype(np.float64), bf16_round(pr.astype(np.float32)))
        losses.append(lr_)
        pr, mr, vr = omlp.adam(pr, g, mr, vr, step, lr)
    np.testing.assert_allclose(loss.cpu().numpy(), losses, rtol=1e-4)
    # Adam moves each weight by about lr per step; FP32 gradients near zero may flip a step's sign
    d = np.abs(params.cpu().numpy() - pr)
    assert np.median(d) < 1e-3 * lr and np.max(d) <= 2 * nsteps * lr
    np.testing.assert_allclose(m.cpu().numpy(), mr, rtol=1e-3, atol=1e-3 * np.max(np.abs(mr)))


def test_single_adam_step_matches_oracle(sd):
    rng = np.random.default_rng(8)
    p = rng.normal(size=omlp.NPARAM).astype(np.float32)
    g = rng.normal(size=omlp.NPARAM).astype(np.float32)
    m = rng.normal(size=omlp.NPARAM).astype(np.float32) * 0.1
    v = rng.uniform(0.1, 1, size=omlp.NPARAM).astype(np.float32)
    P, M, V = _dev(p, torch.float32), _dev(m, torch.float32), _dev(v, torch.float32)
    sd.sdft_mlp_adam(P, _dev(g, torch.float32), M, V, 7, 1e-2)
    pr, mr, vr = omlp.adam(p.astype(float), g.astype(float), m.astype(float), v.astype(float), 7, 1e-2)
    np.testing.assert_allclose(P.cpu().numpy(), pr, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(M.cpu().numpy(), mr, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(V.cpu().numpy(), vr, rtol=1e-6, atol=1e-7)


def test_full_size_loss_grad_and_sampled_inference(sd):
    """512000 points (one 80^3 configuration): gradient of the whole batch against the oracle,
    inference checked on sampled points."""
    npts = 80 ** 3
    bits = _features(npts, seed=99)
    t = np.random.default_rng(5).normal(0, 0.02, npts).astype(np.float32)
    p = workloads.mlp_init_params(13)
    fd, td, pd = _dev_bits(bits), _dev(t, torch.float32), _dev(p, torch.float32)
    grad = torch.zeros(omlp.NPARAM, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    sd.sdft_mlp_loss_grad(fd, td, npts, npts, 0, pd, grad, loss)
    lref, gref = omlp.loss_grad(bits_to_float(bits), t.astype(np.float64), bf16_round(p))
    assert abs(loss.item() - lref) <= 1e-4 * lref
    _check_grad(grad.cpu().numpy().astype(np.float64), gref)
    y = torch.empty(npts, dtype=torch.float32, device="cuda")
    sd.sdft_mlp_forward(fd, npts, pd, y)
    idx = np.random.default_rng(0).choice(npts, 500, replace=False)
    yref = omlp.forward(bits_to_float(bits[idx]), bf16_round(p))
    np.testing.assert_allclose(y.cpu().numpy()[idx], yref, atol=2e-5 * max(1.0, np.max(np.abs(yref))))


def test_argument_errors(sd):
    z = torch.zeros(8, dtype=torch.float32, device="cuda")
    with pytest.raises(sd.SdftError):
        sd.sdft_mlp_loss_grad(z, z, 4, 5, 0, z, z, z)      # batch > npts
    with pytest.raises(sd.SdftError):
        sd.sdft_mlp_adam(z, z, z, z, 0, 1e-3)             # step 0
