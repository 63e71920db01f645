"""The learned per-edge rank selector on the GPU.

* MLP kernels vs the FP64 NumPy reference (oracle/mlp.py): loss and every
  parameter gradient, and one Adam step.
* Labels: per-edge far-field energies at every truncation rank vs the oracle's
  edge split, and their sum vs the far-field energy of the full run (exact
  splitting, because M2M and L2L re-expand exactly).
* Features vs a NumPy recomputation from the oracle's box multipoles.
* Gain: a network trained on small chain/water systems, applied to held-out
  systems, reaches the energy error of a fixed rank with a cheaper M2L.
"""
import numpy as np
import pytest

from oracle import fmm, mlp
from oracle import tree as otree
from paper_1708_05353_gb300 import inputs
from tests.helpers import complex_to_real, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_1708_05353_gb300 import occk
    return occk.Context(0)


def _rand_model(seed):
    from paper_1708_05353_gb300 import occk
    rng = np.random.default_rng(seed)
    theta = mlp.init(occk.MLP_NIN, occk.MLP_HIDDEN, occk.MLP_NOUT, seed)
    theta[:] += 0.05 * rng.normal(size=theta.size)      # non-zero biases too
    mx = rng.normal(size=occk.MLP_NIN)
    sx = rng.uniform(0.5, 2.0, size=occk.MLP_NIN)
    norm = np.concatenate([mx, sx, np.zeros(occk.MLP_NOUT), np.ones(occk.MLP_NOUT)])
    X = rng.normal(size=(300, occk.MLP_NIN)) * sx + mx
    T = rng.normal(size=(300, occk.MLP_NOUT))
    return theta, norm, X, T


def test_mlp_gradient_matches_oracle(ctx):
    from paper_1708_05353_gb300 import occk
    theta, norm, X, T = _rand_model(5)
    occk.mlp_set(ctx, theta, norm)
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda:0")
    Td = torch.tensor(T, dtype=torch.float32, device="cuda:0")
    loss, g = occk.mlp_grad(ctx, Xd, Td)
    Xn = (X - norm[:occk.MLP_NIN]) / norm[occk.MLP_NIN:2 * occk.MLP_NIN]
    lref, gref = mlp.loss_and_grad(theta.astype(np.float32).astype(np.float64), Xn, T,
                                   occk.MLP_NIN, occk.MLP_HIDDEN, occk.MLP_NOUT)
    assert loss == pytest.approx(lref, rel=1e-5)
    assert rel_err(g.cpu().double().numpy(), gref) < 1e-4


def test_mlp_adam_step_matches_oracle(ctx):
    from paper_1708_05353_gb300 import occk
    theta, norm, X, T = _rand_model(6)
    theta32 = theta.astype(np.float32)
    occk.mlp_set(ctx, theta32, norm)
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda:0")
    Td = torch.tensor(T, dtype=torch.float32, device="cuda:0")
    occk.mlp_train(ctx, Xd, Td, 1, 1e-3)
    p, _ = occk.mlp_get(ctx)
    Xn = (X - norm[:occk.MLP_NIN]) / norm[occk.MLP_NIN:2 * occk.MLP_NIN]
    _, g = mlp.loss_and_grad(theta32.astype(np.float64), Xn, T, occk.MLP_NIN, occk.MLP_HIDDEN, occk.MLP_NOUT)
    ref, _, _ = mlp.adam_step(theta32.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1, 1e-3)
    # first Adam step moves each weight by ~lr * sign(g); entries with |g| near
    # zero may differ in sign between FP32 and FP64 gradients
    ok = np.abs(g) > 1e-6 * np.abs(g).max()
    np.testing.assert_allclose(p[ok], ref[ok], atol=2e-6)


def test_edge_energies_match_oracle(ctx):
    from paper_1708_05353_gb300 import learn, occk
    s = inputs.small_sp(natom=6, nocc=4, spacing=3.0, depth=3)
    L = 4
    tree, K, E = learn.run_far_field(ctx, s, L)
    Eg = occk.edge_energies(ctx, tree).cpu().numpy()
    tr = otree.build_tree(s.basis, 3, 8.0)
    _, Er, parts = fmm.farfield(s, L=L, tree=tr, return_parts=True)
    ref = fmm.edge_energies(tr, parts["Obox"], L, list(range(L + 1)))
    assert rel_err(Eg, ref) < 1e-10
    assert np.sum(Eg[:, L]) == pytest.approx(E, rel=1e-10)
    assert E == pytest.approx(Er, rel=1e-10)


def test_edge_features_match_oracle(ctx):
    from paper_1708_05353_gb300 import learn, occk
    s = inputs.small_sp(natom=6, nocc=4, spacing=3.0, depth=3)
    L = 4
    tree, K, E = learn.run_far_field(ctx, s, L)
    F = occk.edge_features(ctx, tree).cpu().numpy()
    tr = otree.build_tree(s.basis, 3, 8.0)
    _, _, parts = fmm.farfield(s, L=L, tree=tr, return_parts=True)
    Ob = complex_to_real(np.moveaxis(parts["Obox"], 1, -1), L)     # [box, i, j, nc]
    ref = np.zeros_like(F)
    for e, (t, src) in enumerate(zip(tr["m2l_tgt"], tr["m2l_src"])):
        lev = tr["box_level"][t]
        h = tr["h"][lev]
        d = np.abs(tr["box_key"][t] - tr["box_key"][src]).astype(float)
        r = np.linalg.norm(d)
        ds = np.sort(d)[::-1]
        ref[e, :6] = [lev / tr["depth"], r, ds[0] / r, ds[1] / r, ds[2] / r, np.log10(h)]
        for q in range(5):
            l = min(2 * q, L)
            sl = slice(l * l, (l + 1) * (l + 1))
            ref[e, 6 + q] = np.log10(np.sqrt(np.sum(Ob[t][..., sl] ** 2)) / h ** l)
            ref[e, 11 + q] = np.log10(np.sqrt(np.sum(Ob[src][..., sl] ** 2)) / h ** l)
    np.testing.assert_allclose(F, ref, rtol=1e-5, atol=1e-5)


def test_learned_selector_gain(ctx):
    from paper_1708_05353_gb300 import learn
    Xs, Ys = [], []
    for sysm in learn.training_systems("small"):
        X, Y, _ = learn.edge_dataset(ctx, sysm)
        Xs.append(X)
        Ys.append(Y)
    loss, margin = learn.train(ctx, np.concatenate(Xs), np.concatenate(Ys), steps=3000, lr=2e-3)
    print("train loss", loss, "margin", margin)
    assert loss < 0.3, loss
    held = [inputs.alkane(40, lmax=10, seed_k=6)]
    w = inputs.water(25, lmax=10, seed_k=5)
    w.depth = 2
    held.append(w)
    for sysm in held:
        res = learn.compare(ctx, sysm, tau=1e-6)
        print(sysm.name, {k: res[k] for k in ("learned", "optimal", "matched_fixed_rank", "gain_vs_matched",
                                               "gain_vs_lref")})
        # within the budget (slack for a calibration on a few hundred edges) ...
        assert res["learned"]["err"] <= 10 * res["tau"]
        # ... cheaper than the method without the selector (every edge at rank
        # 10) and than the cheapest fixed rank that is at least as accurate ...
        assert res["gain_vs_lref"] > 1.0
        assert res["gain_vs_matched"] >= 1.0
        # ... and close to the best choice the true errors allow
        assert res["learned"]["cost"] <= 2.0 * res["optimal"]["cost"]
