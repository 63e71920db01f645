"""Writes tests/golden/oracle_columns.npz: exact columns of the far-field
exchange matrix from the FP64 oracle alone (no CUDA code is imported or run).

    python tests/golden/make_columns.py [name ...]

K^ff_{r,i} = 2 sum_j sum_lm O^{rj,X}_lm Mcal^{ij}_lm(X) (Sec. II, Eq. kri with
the factor 2 of Eq. occex) for a few occupied columns i of workloads whose
full oracle run takes minutes.  A column needs only the occupied pairs (i, j)
for all j, so each stored column is exactly the one a full run would give.
The columns are chosen across the 64- and 128-wide orbital tiles of the CUDA
kernels and at the ragged last tile.  Each entry also stores the input
fingerprint (AO and orbital counts, tree depth, box and M2L edge counts, the
sum of C over the stored columns) so that a test can tell that the seeded
inputs it regenerates are the ones the columns were computed from.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import fmm  # noqa: E402
from oracle import tree as otree  # noqa: E402
from paper_1708_05353_gb300 import inputs  # noqa: E402  (seeded input generator only)

OUT = os.path.join(HERE, "oracle_columns.npz")

# name -> (system factory, ranks, columns)
CASES = {
    # 60-carbon chain, 241 occupied: two full 128-wide tiles and a ragged one
    "chain60": (lambda: inputs.alkane(60, lmax=2), (2, 6), [0, 63, 64, 127, 128, 200, 240]),
    # the 150-carbon chain at the benchmark's size (601 occupied, 5 tiles)
    "chain150": (lambda: inputs.alkane(150, lmax=2), (2,), [0, 127, 300, 600]),
    # the 20-carbon chain of the tensor-core translation tests (81 occupied)
    "chain20": (lambda: inputs.alkane(20, lmax=10, seed_k=4), (2, 4, 6, 10), [0, 40, 80]),
    # the 150-carbon chain with localised orbitals (the pair-screening workload)
    "chain150loc": (lambda: inputs.alkane_localised(150, lmax=2), (2,), [0, 300, 600]),
    # the protein-sized cluster (3577 AOs, 660 occupied), the benchmark's workload
    "protein": (lambda: inputs.protein_like(lmax=2), (2,), [0, 329, 659]),
}


def run(name, data):
    make, ranks, cols = CASES[name]
    s = make()
    tr = otree.build_tree(s.basis, s.depth, s.target_atoms_per_leaf)
    data[f"{name}/cols"] = np.asarray(cols, dtype=np.int64)
    data[f"{name}/fingerprint"] = np.array([s.basis.nao, s.nocc, tr["depth"], tr["nbox"], len(tr["m2l_tgt"]),
                                            float(np.sum(s.C[:, cols]))])
    for L in ranks:
        t0 = time.time()
        K, E = fmm.farfield(s, L=L, tree=tr, i_subset=cols)
        data[f"{name}/L{L}/K"] = K
        data[f"{name}/L{L}/E_cols"] = np.array(E)
        print(f"{name} L={L}: nao {s.basis.nao} nocc {s.nocc}, {time.time() - t0:.1f} s", flush=True)


def tau_near(norm2, target, gap):
    """A screening threshold in a gap of the pair-norm distribution (ratio of
    consecutive distinct norms above 1 + gap) as close as possible, in log
    scale, to `target`: no pair sits near it, so a decision taken in reduced
    precision is the same as the oracle's."""
    n = np.unique(np.sqrt(norm2[np.triu_indices(norm2.shape[0])]))
    k = np.nonzero(n[1:] > n[:-1] * (1 + gap))[0]
    mid = np.sqrt(n[k] * n[k + 1])
    return float(mid[np.argmin(np.abs(np.log(mid / target)))])


def run_screen(data, name="chain150loc_screen", cols=(0, 300, 600)):
    """Occupied-pair screening (the extension proposed in Sec. IV) on the
    150-carbon chain with localised orbitals: the pair norms of every occupied
    pair, a threshold near 1e-4 in a gap 1e-3 wide, the number of kept pairs
    i <= j, and screened K columns."""
    s = inputs.alkane_localised(150, lmax=2)
    tr = otree.build_tree(s.basis, s.depth, s.target_atoms_per_leaf)
    t0 = time.time()
    _, _, parts = fmm.farfield(s, L=2, tree=tr, pair_tau=1.0, return_parts=True)
    norm2 = parts["norm2"]
    tau = tau_near(norm2, 1e-4, 1e-3)
    kept = int(np.count_nonzero(norm2[np.triu_indices(s.nocc)] >= tau * tau))
    K, E = fmm.farfield(s, L=2, tree=tr, pair_tau=tau, i_subset=list(cols))
    data[f"{name}/cols"] = np.asarray(cols, dtype=np.int64)
    data[f"{name}/fingerprint"] = np.array([s.basis.nao, s.nocc, tr["depth"], tr["nbox"], len(tr["m2l_tgt"]),
                                            float(np.sum(s.C[:, list(cols)]))])
    data[f"{name}/tau"] = np.array(tau)
    data[f"{name}/kept"] = np.array(kept)
    data[f"{name}/L2/K"] = K
    data[f"{name}/L2/E_cols"] = np.array(E)
    print(f"{name}: tau {tau:.6e}, kept {kept} of {s.nocc * (s.nocc + 1) // 2}, {time.time() - t0:.1f} s",
          flush=True)


def main():
    names = sys.argv[1:] or list(CASES) + ["chain150loc_screen"]
    data = dict(np.load(OUT)) if os.path.exists(OUT) else {}
    for n in names:
        if n == "chain150loc_screen":
            run_screen(data)
        else:
            run(n, data)
        np.savez_compressed(OUT, **data)


if __name__ == "__main__":
    main()
