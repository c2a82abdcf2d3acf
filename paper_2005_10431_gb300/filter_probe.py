"""Run one short Chebyshev filter on a benchmark cell, for profiling the fused stencil kernel.

    python -m paper_2005_10431_gb300.filter_probe [--workload lattice64_80] [--variant K] [--degree 4]
                                                   [--precision mixed|fp64] [--kpoint]

One sdft_chebyshev_filter call of the given degree on the cell's full orbital block (seeded
orbitals, constant V_eff = -0.3 Ha, the cell's KB projectors), i.e. `degree` launches of the stencil
kernel and as many KB projections.  --variant forces a stencil tile (SDFT_STENCIL_VARIANT), so that
an ncu capture (-k regex:cheb_) sees the kernel of interest on a known launch index.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default="lattice64_80")
    p.add_argument("--variant", type=int, default=None)
    p.add_argument("--degree", type=int, default=4)
    p.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    p.add_argument("--kpoint", action="store_true", help="complex Bloch block at k = (0.25, 0.125, -0.5)")
    a = p.parse_args()
    if a.variant is not None:
        os.environ["SDFT_STENCIL_VARIANT"] = str(a.variant)
    import numpy as np
    import torch
    import workloads
    import paper_2005_10431_gb300 as sd
    cell = {"lattice64_80": workloads.lattice64_cell, "lattice216_120": workloads.lattice216_cell,
            "two_atom_24": workloads.two_atom_cell, "kpoint8_40": lambda: workloads.kpoint_cell(4, 40)}[a.workload]()
    prec = sd.SDFT_MIXED if a.precision == "mixed" else sd.SDFT_FP64
    kpts = [(0.25, 0.125, -0.5)] if a.kpoint else None
    ctx = sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species,
                         dict(nstates=cell.nstates, cheb_degree=a.degree, precision=prec), kpts=kpts)
    sd.sdft_set_veff(ctx, 0, np.full(cell.ngrid, -0.3))
    X = workloads.initial_orbitals(0, cell.ngrid, cell.nstates, complex_valued=a.kpoint)
    x = sd.pack_block(X, prec)
    y = torch.empty_like(x)
    sd.sdft_chebyshev_filter(ctx, 0, 0, prec, x, y, cell.nstates, a.degree, 5.0, 160.0, -1.0)
    torch.cuda.synchronize()
    print("filter done; stencil variant", sd.sdft_get_stencil_variant(ctx, a.kpoint), flush=True)


if __name__ == "__main__":
    main()
