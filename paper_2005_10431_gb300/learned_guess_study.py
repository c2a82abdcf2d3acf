"""Learned initial density on the 64-atom QMD-like sequence: train on the GPU, evaluate held out.

    python -m paper_2005_10431_gb300.learned_guess_study [--train 200] [--test 50] [--out weights.npy]

Training data: the converged output densities of `--train` displaced 4x4x4-lattice cells (seeds
1000.., sigma 0.15 bohr, 80^3 grid, 154 states, mixed precision) solved by the plain SCF from the
superposition of atomic densities (SAD); targets rho* - rho_SAD per grid point, features the 32
radial descriptors.  The network is trained by the library's own kernels (sdft_mlp_train:
mini-batch Adam).  Evaluation on `--test` held-out cells (seeds 2000..): SCF from SAD and from the
learned guess, both with 12 filter passes in the first SCF iteration, reporting the iterations and
device seconds until the free energy stays within 1e-5 Ha/atom of the SAD run's final energy, the
SCF-tolerance iteration counts, and the L1 distance of each start density to the converged one.
Prints one JSON object; --out saves the trained FP32 parameters.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def hit(log, e_ref, natom, tol=1e-5):
    """(iterations, device seconds) after which |F - e_ref|/natom <= tol for every later iteration."""
    it = t = None
    for k, rec in enumerate(log):
        ok = abs(rec["energy"] - e_ref) / natom <= tol
        if ok and it is None:
            it, t = k + 1, rec["seconds"]
        elif not ok:
            it = t = None
    return it, t


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--train", type=int, default=200)
    p.add_argument("--test", type=int, default=50)
    p.add_argument("--max-scf", type=int, default=60)
    p.add_argument("--epochs", type=float, default=3.0)
    p.add_argument("--batch", type=int, default=65536)
    p.add_argument("--out", default=None)
    a = p.parse_args()
    import numpy as np
    import torch
    import workloads
    import paper_2005_10431_gb300 as sd

    def ctx_for(cell, passes, max_scf):
        return sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species,
                              dict(nstates=cell.nstates, cheb_degree=cell.cheb_degree, precision=sd.SDFT_MIXED,
                                   scf_tol=1e-6, max_scf=max_scf, seed=cell.seed, first_scf_filter_passes=passes))

    t0 = time.time()
    ng = 80 ** 3
    F = torch.empty((a.train * ng, 32), dtype=torch.int16, device="cuda")
    T = torch.empty(a.train * ng, dtype=torch.float32, device="cuda")
    train_iters = []
    for i in range(a.train):
        cell = workloads.qmd_lattice64_cell(1000 + i)
        ctx = ctx_for(cell, 4, a.max_scf)
        r = sd.sdft_scf(ctx)
        train_iters.append(r["niter"])
        sd.sdft_mlp_dataset(ctx, F[i * ng:(i + 1) * ng], T[i * ng:(i + 1) * ng])
        sd.sdft_destroy(ctx)
    t_data = time.time() - t0
    npts = a.train * ng
    params = torch.from_numpy(workloads.mlp_init_params(1)).cuda()
    g, m, v = torch.zeros_like(params), torch.zeros_like(params), torch.zeros_like(params)
    steps = int(a.epochs * npts / a.batch)
    sched = [(steps // 2, 3e-3), (steps // 3, 1e-3), (steps - steps // 2 - steps // 3, 3e-4)]
    step = 1
    losses = []
    torch.cuda.synchronize()
    t1 = time.time()
    for nst, lr in sched:
        if nst <= 0:
            continue
        loss = torch.zeros(nst, dtype=torch.float64, device="cuda")
        sd.sdft_mlp_train(F, T, npts, a.batch, params, g, m, v, step, nst, lr, loss)
        step += nst
        losses.append(float(loss[-min(100, nst):].mean()))
    torch.cuda.synchronize()
    t_train = time.time() - t1
    var_t = float(T.var())
    del F, T
    rows = []
    for i in range(a.test):
        cell = workloads.qmd_lattice64_cell(2000 + i)
        c0 = ctx_for(cell, 12, a.max_scf + 20)
        r0 = sd.sdft_scf(c0)
        log0 = sd.sdft_get_scf_log(c0)
        rho_star = sd.sdft_get_density(c0).sum(axis=0)
        sad = sd.sdft_get_sad_density(c0)
        sd.sdft_destroy(c0)
        c1 = ctx_for(cell, 12, a.max_scf + 20)
        sd.sdft_mlp_predict(c1, params)
        feat = torch.empty((ng, 32), dtype=torch.int16, device="cuda")
        y = torch.empty(ng, dtype=torch.float32, device="cuda")
        sd.sdft_mlp_dataset(c1, feat)
        sd.sdft_mlp_forward(feat, ng, params, y)
        r1 = sd.sdft_scf(c1)
        log1 = sd.sdft_get_scf_log(c1)
        sd.sdft_destroy(c1)
        dV = float(np.prod(cell.h))
        guess = np.maximum(sad + y.cpu().numpy(), 0.0)
        guess *= cell.nelec / (guess.sum() * dV)
        e_ref = r0["energy"]
        n0, s0 = hit(log0, e_ref, cell.natom)
        n1, s1 = hit(log1, e_ref, cell.natom)
        rows.append(dict(seed=2000 + i, sad_iters_to_1e5=n0, mlp_iters_to_1e5=n1, sad_s_to_1e5=s0, mlp_s_to_1e5=s1,
                         sad_niter=r0["niter"], mlp_niter=r1["niter"],
                         dE_per_atom=abs(r1["energy"] - r0["energy"]) / cell.natom,
                         drho1_sad=float(np.abs(sad - rho_star).sum() * dV),
                         drho1_mlp=float(np.abs(guess - rho_star).sum() * dV)))
    ok = [r for r in rows if r["sad_iters_to_1e5"] and r["mlp_iters_to_1e5"]]

    def mean(k, src):
        return float(np.mean([r[k] for r in src])) if src else None

    out = dict(train_configs=a.train, test_configs=a.test, points=npts, train_steps=step - 1, batch=a.batch,
               data_seconds=t_data, train_seconds=t_train, target_variance=var_t, final_losses=losses,
               mean_train_niter=float(np.mean(train_iters)),
               mean_iters_to_1e5={"sad": mean("sad_iters_to_1e5", ok), "mlp": mean("mlp_iters_to_1e5", ok)},
               mean_s_to_1e5={"sad": mean("sad_s_to_1e5", ok), "mlp": mean("mlp_s_to_1e5", ok)},
               mean_drho1={"sad": mean("drho1_sad", rows), "mlp": mean("drho1_mlp", rows)},
               max_dE_per_atom=max(r["dE_per_atom"] for r in rows) if rows else None, rows=rows)
    print(json.dumps(out), flush=True)
    if a.out:
        np.save(a.out, params.cpu().numpy())


if __name__ == "__main__":
    main()
