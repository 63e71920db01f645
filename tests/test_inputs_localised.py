"""The localised-orbital input recipe used by the occupied-pair screening
workloads: the orbitals are orthonormal in the AO overlap metric and each
stays within a few bohr of its centre along the chain."""
import numpy as np

from paper_1708_05353_gb300 import inputs


def test_localised_orbitals_orthonormal_and_local():
    s = inputs.alkane_localised(20)
    S = inputs.overlap_matrix(s.basis)
    assert np.abs(s.C.T @ S @ s.C - np.eye(s.nocc)).max() < 1e-10
    ao_atom = np.repeat(s.basis.shell_atom, np.diff(s.basis.shell_ao_offset))
    x = s.basis.xyz[:, 0]
    w = np.zeros((s.basis.natom, s.nocc))
    np.add.at(w, ao_atom, s.C ** 2)
    cen = (w * x[:, None]).sum(0) / w.sum(0)
    spread = np.sqrt((w * (x[:, None] - cen) ** 2).sum(0) / w.sum(0))
    assert spread.max() < 4.0                     # bohr, on a ~60-bohr chain
    # centres follow the orbital order along the chain
    assert np.corrcoef(np.arange(s.nocc), cen)[0, 1] > 0.99


def test_localised_same_geometry_and_basis():
    a = inputs.alkane(20)
    b = inputs.alkane_localised(20)
    assert np.array_equal(a.basis.xyz, b.basis.xyz)
    assert np.array_equal(a.basis.exps, b.basis.exps) and a.nocc == b.nocc
