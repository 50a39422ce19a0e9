"""Writes tests/golden/dmrg_oracle.json: per-sweep DMRG energies from the CPU oracle.

Calls only ``oracle`` and ``synth``.  Run from the repository root:
    python tests/golden/make_golden.py
Cases:
  abinitio_n8_M64   ab initio n = 8, N = 8, Sz = 0 (integral seed 0), MPS seed 100,
                    M = 64, 6 sweeps
  hubbard_L12_M48   Hubbard open chain L = 12, t = 1, U = 4, half filling, MPS seed 112,
                    M = 48, 4 sweeps
Davidson: |r|^2 <= 1e-12 with up to 200 products and a 40-vector subspace, so that every
solve converges (a solve stopped early depends on rounding, which differs between any two
implementations).
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import dmrg, fci, mpo  # noqa: E402
from synth import (config_integrals, hubbard_integrals, occupancies, random_mps,  # noqa: E402
                   sector_sizes)

CASES = {
    "abinitio_n8_M64": dict(ints="abinitio_n8", M=64, sweeps=6, mps_seed=100, max_iter=200, tol=1e-12,
                            max_sub=40),
    "hubbard_L12_M48": dict(ints=("hubbard", 12, 1.0, 4.0), M=48, sweeps=4, mps_seed=112, tol=1e-12,
                            max_iter=200, max_sub=40),
}


def case_inputs(name):
    c = CASES[name]
    if isinstance(c["ints"], str):
        h, eri, N, tsz, kind = config_integrals(c["ints"])
    else:
        _, L, t, U = c["ints"]
        h, eri = hubbard_integrals(L, t, U)
        N, tsz, kind = L, 0, "hubbard"
    n = h.shape[0]
    bonds = sector_sizes(n, N, tsz, c["M"], occupancies(n, N, kind))
    sites = random_mps(bonds, seed=c["mps_seed"])
    return h, eri, N, tsz, bonds, sites, c


def main():
    out = {"generator": "tests/golden/make_golden.py (oracle only)", "cases": {}}
    for name in CASES:
        h, eri, N, tsz, bonds, sites, c = case_inputs(name)
        t0 = time.time()
        d = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites)
        es = d.run([c["M"]] * c["sweeps"], tol=c["tol"], max_iter=c["max_iter"], max_sub=c["max_sub"])
        rec = {"sweep_energies": es, "n_matvec": sum(s["n_matvec"] for s in d.stats),
               "seconds": time.time() - t0}
        if h.shape[0] <= 12:
            rec["fci"] = fci.fci_ground_state(h, eri, N, tsz)[0]
        out["cases"][name] = rec
        print(name, rec, flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "dmrg_oracle.json"),
              "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
