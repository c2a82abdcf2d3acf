"""Write the oracle's converged reference values for the parity tests and the benchmark.

Every number in the JSON files next to this script comes from this script, which calls only
the FP64 CPU oracle (oracle/) on the seeded synthetic cells of `workloads`.

usage: python tests/golden/make_golden.py two_atom_24 [lattice64_80 ...]
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import workloads  # noqa: E402
from oracle import scf  # noqa: E402

CELLS = {
    "two_atom_24": (workloads.two_atom_cell, dict(tol=1e-10, max_iter=300, final_tol=1e-10)),
    "lattice64_80": (workloads.lattice64_cell, dict(tol=1e-8, max_iter=150, final_tol=None)),
    "kspin_20": (workloads.kspin_small_cell, dict(tol=1e-8, max_iter=300, final_tol=None)),
}


def main(names):
    for name in names:
        make, kw = CELLS[name]
        cell = make()
        t0 = time.time()
        r = scf.scf(cell, with_forces=True, verbose=True, **kw)
        out = dict(
            cell=name,
            generator="tests/golden/make_golden.py (oracle.scf.scf, FP64 CPU)",
            scf_options=dict(kw, mix_beta=0.3, mix_hist=7, pulay_period=1, first_passes=4,
                             lanczos_steps=20),
            natom=cell.natom, nelec=cell.nelec, nstates=cell.nstates, n=list(cell.n), L=list(cell.L),
            energy=r.energy, energy_ks=r.energy_ks, mu=r.mu, converged=r.converged, niter=r.niter,
            eigs=r.eigs.tolist(), occ=r.occ.tolist(), forces=r.forces.tolist(),
            history=[{k: float(v) for k, v in h.items()} for h in r.history],
            seconds=time.time() - t0,
        )
        with open(os.path.join(HERE, f"{name}.json"), "w") as f:
            json.dump(out, f, indent=1)
        np.save(os.path.join(HERE, f"{name}_rho.npy"), r.rho.astype(np.float64)) if cell.ngrid <= 20000 else None
        print(f"wrote {name}: F = {r.energy:.12f} (KS {r.energy_ks:.12f}) in {time.time() - t0:.0f}s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["two_atom_24"])
