"""Writes the stored expected values of tests/golden/ from the FP64 oracle
alone (no CUDA code is imported or run).

    python tests/golden/make_golden.py

line40_farfield.json: the 40-atom line workload (40 s-type atoms at 1.5 bohr,
exponents 3.0 and 0.5, coefficients 0.4 and 0.7, 20 Loewdin-orthonormalised
seeded orbitals, octree depth 3): the far-field exchange energy
E^ff = -1/2 sum_ri C_ri K^ff_ri with K^ff_ri = 2 sum_j (rj|ji)^ff (Sec. II,
Eq. kri with the factor 2 of Eq. occex) from the hierarchical method at ranks
0..6, the same energy from exact four-centre integrals over the far boxes
(the limit the ranks converge to), and the first row of K^ff at rank 2.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import brute, fmm  # noqa: E402
from oracle import tree as otree  # noqa: E402
from paper_1708_05353_gb300 import inputs  # noqa: E402  (seeded input generator only)


def main():
    s = inputs.tiny_line()
    tr = otree.build_tree(s.basis, s.depth, s.target_atoms_per_leaf)
    out = {"workload": "line40: 40 s atoms at 1.5 bohr, nocc 20, depth 3",
           "source": "oracle/ (FP64 NumPy), written by tests/golden/make_golden.py",
           "energy_by_rank": {}}
    for L in range(0, 7):
        K, E = fmm.farfield(s, L=L, tree=tr)
        out["energy_by_rank"][str(L)] = E
        if L == 2:
            out["K_row0_rank2"] = [float(x) for x in K[0]]
    _, Ex = brute.farfield_exact(s.basis, tr, s.C)
    out["energy_exact"] = Ex
    with open(os.path.join(HERE, "line40_farfield.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: v for k, v in out.items() if k != "K_row0_rank2"}, indent=1))


if __name__ == "__main__":
    main()
