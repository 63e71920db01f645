"""FP64 CPU oracle for the far-field occupied-orbital FMM exchange (occ-FMM-K).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, direct restatement
of the method of Le & Shiozaki (arXiv:1708.05353) in complex double-precision
arithmetic, written from the paper's equations.  It exists to check the CUDA
path.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it; the library under
``paper_1708_05353_gb300`` never does, and the two share no code.  The only
shared module is ``paper_1708_05353_gb300.inputs`` (seeded synthetic inputs),
which holds none of the method's arithmetic.

Modules
  solid   scaled regular/irregular solid harmonics O_lm, M_lm (Sec. I, Eq. mmexp
          and the definitions that follow it)
  gauss   s/p Cartesian Gaussians, AO-pair multipole integrals (Sec. II, the
          multipole-integral definition), Boys function, McMurchie-Davidson
          ERIs (Eq. erib) for the brute-force far-field reference
  tree    box hierarchy, neighbours and interaction lists (Sec. II)
  fmm     occ-FMM-K: MO transforms (Eq. motrans), occupied M2M/M2L/L2L, K^ff_ri
          (Eq. kri) and the exchange energy
  brute   brute-force far-field exchange from exact ERIs
  fmm_j   far-field Coulomb matrix J^ff_rs by the FMM (Sec. II, Eq. fmmc and
          the J^ff formula) and its exact far-box counterpart
  mlp     reference forward/backward/Adam of the lmax-selector MLP
"""
