"""Writes the stored expected values under tests/golden/ from the oracle alone.

Run from the repository root:  python tests/golden/make_golden.py
Each file is the dense LAPACK spectrum (numpy.linalg.eigh of the oracle's sector
matrix) of one seeded workload: the 8 eigenvalues nearest the spectrum midpoint
sigma = (E_min + E_max) / 2 and ||H|| = max(|E_min|, |E_max|).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as wl  # noqa: E402
from oracle import hamiltonian as ham  # noqa: E402


def nearest_file(cfg, path):
    ch = ham.Chain(cfg["L"], wl.fields(cfg["L"], cfg["W"], cfg["seed"]), delta=cfg["delta"],
                   periodic=cfg["periodic"])
    ev = np.linalg.eigvalsh(ham.dense_sector(ch))
    emin, emax = float(ev[0]), float(ev[-1])
    sigma = 0.5 * (emin + emax)
    norm_h = max(abs(emin), abs(emax))
    mu = ev - sigma
    sel = np.sort(ev[np.lexsort((ev, np.abs(mu)))[: cfg["nev"]]])
    with open(path, "w") as f:
        f.write("# %s: L=%d %s delta=%g h~U[-%g,%g] seed %d; dense eigh of the oracle sector matrix\n"
                % (cfg["name"], cfg["L"], "periodic" if cfg["periodic"] else "open", cfg["delta"],
                   cfg["W"], cfg["W"], cfg["seed"]))
        f.write("emin %.17g\nemax %.17g\nsigma %.17g\nnorm_h %.17g\n" % (emin, emax, sigma, norm_h))
        for v in sel:
            f.write("eval %.17g\n" % v)


if __name__ == "__main__":
    nearest_file(wl.SOLVE_L12, os.path.join(HERE, "l12_open_w5_seed0_nearest8.txt"))
    print("written")
