"""CPU checks of the C ABI: the library loads, exports every function that
include/occk.h declares, rejects bad arguments, and its host-built tree equals
the oracle's tree exactly (integers bit-exact; centres to the last bit)."""
import ctypes

import numpy as np
import pytest

from oracle import tree as otree
from paper_1708_05353_gb300 import inputs
from paper_1708_05353_gb300 import occk


def test_library_exports_header():
    L = occk.lib()
    names = occk.header_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n


def test_host_only_context_rejects_device_work():
    ctx = occk.Context(-1)
    s = inputs.tiny_line()
    t = occk.Tree(ctx, s.basis, depth=3)
    with pytest.raises(occk.OcckError) as e:
        t.pair_multipoles(2, stream=0)
    assert e.value.code == -6


def test_bad_arguments():
    ctx = occk.Context(-1)
    s = inputs.tiny_line()
    b = s.basis
    bad = inputs.Basis(xyz=b.xyz, elements=b.elements, shell_atom=b.shell_atom,
                       shell_l=np.full_like(b.shell_l, 2), shell_nprim=b.shell_nprim,
                       exps=b.exps, coefs=b.coefs)
    with pytest.raises(occk.OcckError) as e:
        occk.Tree(ctx, bad, depth=3)
    assert e.value.code == -6
    neg = inputs.Basis(xyz=b.xyz, elements=b.elements, shell_atom=b.shell_atom,
                       shell_l=b.shell_l, shell_nprim=b.shell_nprim,
                       exps=-b.exps, coefs=b.coefs)
    with pytest.raises(occk.OcckError) as e:
        occk.Tree(ctx, neg, depth=3)
    assert e.value.code == -1
    t = occk.Tree(ctx, b, depth=3)
    out = np.zeros(3, dtype=np.int32)
    assert occk.lib().occk_tree_export(t._h, 0, out.ctypes.data_as(ctypes.c_void_p), out.nbytes) == -2
    with pytest.raises(occk.OcckError):
        t.set_edge_lmax([0, 1])


def _compare(sysm, depth=None):
    ctx = occk.Context(-1)
    d = sysm.depth if depth is None else depth
    t = occk.Tree(ctx, sysm.basis, depth=d, target_atoms_per_leaf=sysm.target_atoms_per_leaf)
    o = otree.build_tree(sysm.basis, d, sysm.target_atoms_per_leaf)
    inf = t.info()
    assert inf["depth"] == o["depth"]
    assert inf["nao"] == sysm.basis.nao
    np.testing.assert_array_equal(t.export("level_off"), o["level_off"])
    np.testing.assert_array_equal(t.export("box_key"), o["box_key"])
    np.testing.assert_array_equal(t.export("parent"), o["parent"])
    np.testing.assert_array_equal(t.export("m2l"), np.stack([o["m2l_tgt"], o["m2l_src"]], axis=1)
                                  if len(o["m2l_tgt"]) else np.zeros((0, 2)))
    pairs = t.export("pairs")
    np.testing.assert_array_equal(pairs[:, 0], o["pair_a"])
    np.testing.assert_array_equal(pairs[:, 1], o["pair_b"])
    np.testing.assert_array_equal(pairs[:, 2], o["leaf_of_pair"])
    np.testing.assert_array_equal(t.export("centre"), o["centre"])
    np.testing.assert_allclose(t.export("pair_centre"), o["pair_centre"], rtol=0, atol=1e-13)
    rowoff = t.export("leaf_rowoff")
    aos = t.export("leaf_aos")
    for k, S in enumerate(o["ao_sets"]):
        np.testing.assert_array_equal(aos[rowoff[k]:rowoff[k + 1]], S)
    return inf


def test_tree_matches_oracle_line():
    inf = _compare(inputs.tiny_line())
    assert inf["nm2l"] == 24


def test_tree_matches_oracle_sp():
    _compare(inputs.small_sp(natom=6, nocc=4, spacing=3.0, depth=3))


def test_tree_matches_oracle_water_auto_depth():
    inf = _compare(inputs.water(nmol=20, lmax=2), depth=0)
    assert inf["depth"] >= 1


def test_tree_matches_oracle_chain_auto_depth():
    s = inputs.alkane(30, lmax=2)
    inf = _compare(s, depth=0)
    assert inf["nm2l"] > 0


@pytest.mark.slow
def test_tree_matches_oracle_full_chain():
    """The 150-carbon chain at full size: same boxes, lists and pair owners."""
    _compare(inputs.alkane(150, lmax=2), depth=0)


def test_pair_screen_arguments():
    """occk_set_pair_screen takes a finite tau >= 0; the kept count is -1 when
    no screened build has run."""
    ctx = occk.Context(-1)
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(occk.OcckError) as e:
            ctx.set_pair_screen(bad)
        assert e.value.code == -1
    ctx.set_pair_screen(1e-4)
    ctx.set_pair_screen(0.0)
    assert ctx.pair_screen_count(stream=0) == -1
