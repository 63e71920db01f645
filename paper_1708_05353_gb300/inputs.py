"""Seeded synthetic inputs: geometries, s/p Gaussian basis sets and occupied
MO coefficients.

This module serves both the CUDA path and the CPU oracle and holds none of the
far-field exchange arithmetic (no multipoles, no translations, no tree).  It
builds the workloads that stand in for the paper's def2-SVP benchmark systems
(alkane chains, a graphene flake, water clusters, a protein-sized cluster;
Sec. III, Table II), whose geometries, basis data and converged orbitals are
not available.  Every random draw uses ``numpy.random.default_rng(1000*k+s)``
with k the workload number (1-5) and s = 0 geometry, 1 basis, 2 coefficients.

The occupied coefficients are C = C0 (C0^T S C0)^(-1/2) (Loewdin
orthonormalisation in the AO overlap metric) with C0 ~ N(0,1).  The overlap S
used for that step is computed here from the closed-form product-Gaussian
overlap of s/p Cartesian primitives; it is input preparation only.

Units are bohr.  AO order is shell order; a p shell contributes (x, y, z).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# Data containers
# ---------------------------------------------------------------------------


@dataclass
class Basis:
    """Contracted s/p basis on a set of atoms.

    ``coefs`` multiply *normalised* primitives; consumers renormalise each
    contracted function to unit self-overlap.
    """
    xyz: np.ndarray                 # [natom, 3] float64, bohr
    elements: list                  # [natom] element symbols
    shell_atom: np.ndarray          # [nshell] int32
    shell_l: np.ndarray             # [nshell] int32, 0 or 1
    shell_nprim: np.ndarray         # [nshell] int32
    exps: np.ndarray                # [sum nprim] float64
    coefs: np.ndarray               # [sum nprim] float64

    @property
    def natom(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def nshell(self) -> int:
        return int(self.shell_l.shape[0])

    @property
    def nao(self) -> int:
        return int(np.sum(np.where(self.shell_l == 0, 1, 3)))

    @property
    def shell_prim_offset(self) -> np.ndarray:
        off = np.zeros(self.nshell + 1, dtype=np.int64)
        off[1:] = np.cumsum(self.shell_nprim)
        return off

    @property
    def shell_ao_offset(self) -> np.ndarray:
        off = np.zeros(self.nshell + 1, dtype=np.int64)
        off[1:] = np.cumsum(np.where(self.shell_l == 0, 1, 3))
        return off


@dataclass
class System:
    name: str
    basis: Basis
    nocc: int
    C: np.ndarray                   # [nao, nocc] float64, column-major semantics
    depth: int                      # 0 => choose from target_atoms_per_leaf
    target_atoms_per_leaf: float
    lmax: int
    meta: dict = field(default_factory=dict)


# ---------------------------------------------------------------------------
# Geometries
# ---------------------------------------------------------------------------

ANG_CCC = math.radians(111.5)
ANG_TET = math.radians(109.4712206)
R_CC_CHAIN = 2.91
R_CH = 2.06
R_OH = 1.81
ANG_HOH = math.radians(104.5)
R_CC_GRAPHENE = 2.68

ELECTRONS = {"H": 1, "C": 6, "N": 7, "O": 8, "S": 16}


def line_atoms(n: int, spacing: float) -> np.ndarray:
    xyz = np.zeros((n, 3))
    xyz[:, 0] = spacing * np.arange(n)
    return xyz


def alkane_chain(ncarbon: int):
    """Zig-zag C_n H_(2n+2): C-C 2.91 bohr at 111.5 deg, tetrahedral C-H 2.06."""
    half = ANG_CCC / 2.0
    dx = R_CC_CHAIN * math.sin(half)
    dy = R_CC_CHAIN * math.cos(half)
    cpos = np.zeros((ncarbon, 3))
    cpos[:, 0] = dx * np.arange(ncarbon)
    cpos[:, 1] = dy * (np.arange(ncarbon) % 2)
    zhat = np.array([0.0, 0.0, 1.0])
    hs = []
    for k in range(ncarbon):
        nb = []
        for q in (k - 1, k + 1):
            if 0 <= q < ncarbon:
                nb.append(cpos[q])
            else:  # virtual continuation of the zig-zag
                nb.append(np.array([dx * q, dy * (q % 2), 0.0]))
        u = [(p - cpos[k]) / np.linalg.norm(p - cpos[k]) for p in nb]
        b = -(u[0] + u[1])
        b /= np.linalg.norm(b)
        ch = math.cos(ANG_TET / 2.0)
        sh = math.sin(ANG_TET / 2.0)
        hs.append(cpos[k] + R_CH * (ch * b + sh * zhat))
        hs.append(cpos[k] + R_CH * (ch * b - sh * zhat))
        # terminal carbons take a third H where the chain would continue
        if k == 0:
            hs.append(cpos[k] + R_CH * u[0])
        if k == ncarbon - 1:
            hs.append(cpos[k] + R_CH * u[1])
    hpos = np.array(hs)
    xyz = np.vstack([cpos, hpos])
    elements = ["C"] * ncarbon + ["H"] * len(hs)
    return xyz, elements


def _rotation(rng) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([
        [a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
        [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
        [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d],
    ])


def water_cluster(nmol: int, rng, spacing: float = 5.7, jitter: float = 0.3):
    """n H2O at random orientations on a jittered cubic lattice."""
    side = int(math.ceil(nmol ** (1.0 / 3.0) - 1e-9))
    sites = []
    for ix in range(side):
        for iy in range(side):
            for iz in range(side):
                sites.append((ix, iy, iz))
    sites = np.array(sites[:nmol], dtype=float) * spacing
    sites += rng.uniform(-jitter, jitter, size=sites.shape)
    local = np.array([
        [0.0, 0.0, 0.0],
        [R_OH * math.sin(ANG_HOH / 2), 0.0, R_OH * math.cos(ANG_HOH / 2)],
        [-R_OH * math.sin(ANG_HOH / 2), 0.0, R_OH * math.cos(ANG_HOH / 2)],
    ])
    xyz, el = [], []
    for s in sites:
        R = _rotation(rng)
        for a, e in zip(local @ R.T + s, ("O", "H", "H")):
            xyz.append(a)
            el.append(e)
    return np.array(xyz), el


def graphene_flake(ncarbon: int = 150, nh: int = 30):
    """Round honeycomb flake of ``ncarbon`` C (2.68 bohr) with ``nh`` edge H."""
    a = R_CC_GRAPHENE
    a1 = np.array([1.5 * a, math.sqrt(3) / 2 * a, 0.0])
    a2 = np.array([1.5 * a, -math.sqrt(3) / 2 * a, 0.0])
    basis_pts = [np.zeros(3), np.array([a, 0.0, 0.0])]
    pts = []
    for i in range(-12, 13):
        for j in range(-12, 13):
            for b in basis_pts:
                pts.append(i * a1 + j * a2 + b)
    pts = np.array(pts)
    centre = np.array([0.5 * a, 0.0, 0.0])
    d = np.linalg.norm(pts - centre, axis=1)
    order = np.lexsort((pts[:, 1], pts[:, 0], np.round(d, 9)))
    cpos = pts[order[:ncarbon]]
    dist = np.linalg.norm(cpos[:, None, :] - cpos[None, :, :], axis=2)
    nbr = (dist < 1.1 * a) & (dist > 0.1)
    ncount = nbr.sum(axis=1)
    dc = np.linalg.norm(cpos - centre, axis=1)
    cand = np.lexsort((-dc, ncount))
    hs = []
    for k in cand[:nh]:
        nb = cpos[nbr[k]]
        if len(nb) == 0:
            v = cpos[k] - centre
        else:
            v = -np.sum(nb - cpos[k], axis=0)
            if np.linalg.norm(v) < 1e-8:
                v = cpos[k] - centre
        v /= np.linalg.norm(v)
        hs.append(cpos[k] + R_CH * v)
    xyz = np.vstack([cpos, np.array(hs)])
    return xyz, ["C"] * ncarbon + ["H"] * nh


def protein_like_cluster(rng, counts=None, semi_axes=(22.5, 15.0, 12.0),
                         dmin: float = 2.0):
    """Random sequential addition of atoms inside an ellipsoid, min spacing dmin."""
    if counts is None:
        counts = {"C": 202, "H": 317, "O": 64, "N": 55, "S": 6}
    n = sum(counts.values())
    ax = np.array(semi_axes)
    pts = np.zeros((0, 3))
    tries = 0
    while pts.shape[0] < n:
        cand = rng.uniform(-1.0, 1.0, size=(4096, 3))
        cand = cand[np.sum(cand * cand, axis=1) <= 1.0] * ax
        for c in cand:
            if pts.shape[0] >= n:
                break
            if pts.shape[0] == 0 or np.min(np.sum((pts - c) ** 2, axis=1)) >= dmin * dmin:
                pts = np.vstack([pts, c])
        tries += 1
        if tries > 10000:
            raise RuntimeError("random sequential addition did not converge")
    el = []
    for e, c in counts.items():
        el += [e] * c
    perm = rng.permutation(n)
    el = [el[p] for p in perm]
    return pts, el


# ---------------------------------------------------------------------------
# Basis sets
# ---------------------------------------------------------------------------

def draw_element_basis(rng, shells: dict, nprim: int = 3,
                       lo: float = 0.1, hi: float = 50.0):
    """For each element, shells[el] = list of l; exponents log-uniform [lo, hi]
    (sorted descending), contraction coefficients uniform(0.2, 1.0)."""
    out = {}
    for el in sorted(shells):
        lst = []
        for l in shells[el]:
            e = np.sort(np.exp(rng.uniform(math.log(lo), math.log(hi), size=nprim)))[::-1]
            c = rng.uniform(0.2, 1.0, size=nprim)
            lst.append((int(l), e.copy(), c.copy()))
        out[el] = lst
    return out


def make_basis(xyz, elements, element_basis) -> Basis:
    sa, sl, sn, ex, co = [], [], [], [], []
    for a, el in enumerate(elements):
        for (l, e, c) in element_basis[el]:
            sa.append(a)
            sl.append(l)
            sn.append(len(e))
            ex.extend(e.tolist())
            co.extend(c.tolist())
    return Basis(xyz=np.ascontiguousarray(xyz, dtype=np.float64), elements=list(elements),
                 shell_atom=np.array(sa, dtype=np.int32), shell_l=np.array(sl, dtype=np.int32),
                 shell_nprim=np.array(sn, dtype=np.int32), exps=np.array(ex, dtype=np.float64),
                 coefs=np.array(co, dtype=np.float64))


# ---------------------------------------------------------------------------
# Overlap (input preparation for the Loewdin step only)
# ---------------------------------------------------------------------------

def _ao_primitives(basis: Basis):
    """Expand to per-AO primitive lists: (centre, cart index k or -1, exps, normalised coefs)."""
    poff = basis.shell_prim_offset
    aos = []
    for s in range(basis.nshell):
        A = basis.xyz[basis.shell_atom[s]]
        e = basis.exps[poff[s]:poff[s + 1]]
        c = basis.coefs[poff[s]:poff[s + 1]]
        ns = (2.0 * e / math.pi) ** 0.75
        if basis.shell_l[s] == 0:
            aos.append((A, -1, e, c * ns))
        else:
            for k in range(3):
                aos.append((A, k, e, c * ns * 2.0 * np.sqrt(e)))
    return aos


def overlap_matrix(basis: Basis) -> np.ndarray:
    """AO overlap of the renormalised contracted s/p functions.

    Product of two Gaussians: exp(-a|r-A|^2) exp(-b|r-B|^2) = K exp(-p|r-P|^2),
    p = a+b, P = (aA+bB)/p, K = exp(-ab/p |A-B|^2).  Then
      <s|s>     = (pi/p)^1.5 K
      <s|p_k>   = (P-B)_k (pi/p)^1.5 K
      <p_k|p_q> = ((P-A)_k (P-B)_q + delta_kq / (2p)) (pi/p)^1.5 K
    """
    aos = _ao_primitives(basis)
    n = len(aos)
    A = np.array([a[0] for a in aos])
    kk = np.array([a[1] for a in aos])
    npmax = max(len(a[2]) for a in aos)
    E = np.zeros((n, npmax))
    Cc = np.zeros((n, npmax))
    for i, a in enumerate(aos):
        E[i, :len(a[2])] = a[2]
        Cc[i, :len(a[2])] = a[3]
        if len(a[2]) < npmax:
            E[i, len(a[2]):] = 1.0
    S = np.zeros((n, n))
    for p in range(npmax):
        for q in range(npmax):
            a = E[:, p][:, None]
            b = E[:, q][None, :]
            pp = a + b
            AB = A[:, None, :] - A[None, :, :]
            K = np.exp(-a * b / pp * np.sum(AB * AB, axis=2))
            P = (a[..., None] * A[:, None, :] + b[..., None] * A[None, :, :]) / pp[..., None]
            PA = P - A[:, None, :]
            PB = P - A[None, :, :]
            base = (math.pi / pp) ** 1.5 * K
            fa = np.ones((n, n))
            fb = np.ones((n, n))
            ia = kk[:, None] * np.ones((1, n), dtype=int)
            ib = np.ones((n, 1), dtype=int) * kk[None, :]
            pa_k = np.take_along_axis(PA, np.clip(ia, 0, 2)[..., None], axis=2)[..., 0]
            pb_k = np.take_along_axis(PB, np.clip(ib, 0, 2)[..., None], axis=2)[..., 0]
            both = (ia >= 0) & (ib >= 0)
            val = np.where(ia >= 0, pa_k, fa) * np.where(ib >= 0, pb_k, fb)
            val = val + np.where(both & (ia == ib), 1.0 / (2.0 * pp), 0.0)
            S += Cc[:, p][:, None] * Cc[:, q][None, :] * base * val
    d = 1.0 / np.sqrt(np.diag(S))
    return S * d[:, None] * d[None, :]


def loewdin_occupied(basis: Basis, nocc: int, rng) -> np.ndarray:
    S = overlap_matrix(basis)
    C0 = rng.normal(size=(basis.nao, nocc))
    M = C0.T @ S @ C0
    w, V = np.linalg.eigh(M)
    return np.ascontiguousarray(C0 @ (V * (1.0 / np.sqrt(w))) @ V.T)


def localised_occupied(basis: Basis, nocc: int, rng, sigma: float = 3.0) -> np.ndarray:
    """Localised occupied orbitals: orbital j starts as N(0,1) coefficients
    under a Gaussian envelope exp(-|A - X_j|^2 / sigma^2) of the distance from
    its AO's atom A to a centre atom X_j (centres evenly spaced along the
    atoms sorted by their first principal coordinate), then the same Loewdin
    orthonormalisation in the AO overlap metric as ``loewdin_occupied``.  The
    orthonormalised orbitals keep exponentially decaying tails, so orbital
    pairs far apart have negligible pair densities."""
    S = overlap_matrix(basis)
    xyz = basis.xyz
    x0 = xyz - xyz.mean(axis=0)
    axis = np.linalg.svd(x0, full_matrices=False)[2][0]
    order = np.argsort(x0 @ axis, kind="stable")
    centres = xyz[order[(np.arange(nocc) * len(order)) // nocc]]          # [nocc, 3]
    ao_atom = np.repeat(basis.shell_atom, np.diff(basis.shell_ao_offset))
    d2 = ((xyz[ao_atom][:, None, :] - centres[None, :, :]) ** 2).sum(axis=2)   # [nao, nocc]
    C0 = rng.normal(size=(basis.nao, nocc)) * np.exp(-d2 / sigma ** 2)
    M = C0.T @ S @ C0
    w, V = np.linalg.eigh(M)
    return np.ascontiguousarray(C0 @ (V * (1.0 / np.sqrt(w))) @ V.T)


def electrons(elements) -> int:
    return sum(ELECTRONS[e] for e in elements)


# ---------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------

SHELLS_CHAIN = {"C": [0, 0, 1], "H": [0, 0]}
SHELLS_HEAVY = {"C": [0, 0, 0, 1, 1], "N": [0, 0, 0, 1, 1], "O": [0, 0, 0, 1, 1],
                "S": [0, 0, 0, 1, 1], "H": [0, 0]}


def tiny_line(natom: int = 40, nocc: int = 20, lmax: int = 2) -> System:
    """40 s-type atoms at 1.5 bohr on a line, exponents (3.0, 0.5), coefficients
    (0.4, 0.7), nocc = 20, octree depth 3, lmax = 2."""
    xyz = line_atoms(natom, 1.5)
    eb = {"H": [(0, np.array([3.0, 0.5]), np.array([0.4, 0.7]))]}
    basis = make_basis(xyz, ["H"] * natom, eb)
    C = loewdin_occupied(basis, nocc, np.random.default_rng(1000 * 1 + 2))
    return System("line40", basis, nocc, C, depth=3, target_atoms_per_leaf=8.0, lmax=lmax)


def alkane(ncarbon: int = 150, lmax: int = 2, seed_k: int = 2, nocc: int | None = None) -> System:
    xyz, el = alkane_chain(ncarbon)
    eb = draw_element_basis(np.random.default_rng(1000 * seed_k + 1), SHELLS_CHAIN)
    basis = make_basis(xyz, el, eb)
    if nocc is None:
        nocc = electrons(el) // 2
    C = loewdin_occupied(basis, nocc, np.random.default_rng(1000 * seed_k + 2 + ncarbon * 0))
    return System(f"C{ncarbon}H{2 * ncarbon + 2}", basis, nocc, C, depth=0,
                  target_atoms_per_leaf=8.0, lmax=lmax)


def alkane_localised(ncarbon: int = 150, lmax: int = 2, seed_k: int = 2, sigma: float = 3.0) -> System:
    """The alkane chain with localised occupied orbitals (the occupied-pair
    screening workload): same geometry and basis as ``alkane``."""
    s = alkane(ncarbon, lmax=lmax, seed_k=seed_k)
    C = localised_occupied(s.basis, s.nocc, np.random.default_rng(1000 * seed_k + 7), sigma)
    return System(f"C{ncarbon}H{2 * ncarbon + 2}-loc", s.basis, s.nocc, C, depth=0,
                  target_atoms_per_leaf=8.0, lmax=lmax)


def small_sp_localised(natom: int = 10, nocc: int = 8, spacing: float = 2.6, seed: int = 11,
                       lmax: int = 2, depth: int = 3, sigma: float = 2.5) -> System:
    """A small s/p line with localised occupied orbitals."""
    s = small_sp(natom=natom, nocc=nocc, spacing=spacing, seed=seed, lmax=lmax, depth=depth)
    C = localised_occupied(s.basis, nocc, np.random.default_rng(seed + 3), sigma)
    return System(f"sp{natom}-loc", s.basis, nocc, C, depth=depth, target_atoms_per_leaf=8.0, lmax=lmax)


def water(nmol: int = 100, lmax: int = 4, seed_k: int = 3, nocc: int | None = None,
          geom_seed: int | None = None) -> System:
    g = np.random.default_rng(1000 * seed_k + 0 if geom_seed is None else geom_seed)
    xyz, el = water_cluster(nmol, g)
    eb = draw_element_basis(np.random.default_rng(1000 * seed_k + 1), SHELLS_HEAVY)
    basis = make_basis(xyz, el, eb)
    if nocc is None:
        nocc = electrons(el) // 2
    C = loewdin_occupied(basis, nocc, np.random.default_rng(1000 * seed_k + 2))
    return System(f"(H2O){nmol}", basis, nocc, C, depth=0, target_atoms_per_leaf=8.0, lmax=lmax)


def flake(lmax: int = 4, seed_k: int = 4) -> System:
    xyz, el = graphene_flake(150, 30)
    eb = draw_element_basis(np.random.default_rng(1000 * seed_k + 1), SHELLS_CHAIN)
    basis = make_basis(xyz, el, eb)
    nocc = electrons(el) // 2
    C = loewdin_occupied(basis, nocc, np.random.default_rng(1000 * seed_k + 2))
    return System("C150H30", basis, nocc, C, depth=0, target_atoms_per_leaf=8.0, lmax=lmax)


def batch_workload(lmax: int = 4, waters=None, chains=(50, 100, 200)) -> list:
    """The uneven batch: one flake, three chains, sixteen water clusters of
    10 + round(50 k / 15) molecules, k = 0..15."""
    systems = [flake(lmax)]
    for n in chains:
        s = alkane(n, lmax=lmax, seed_k=4)
        systems.append(s)
    if waters is None:
        waters = [10 + int(round(50 * k / 15)) for k in range(16)]
    for k, n in enumerate(waters):
        systems.append(water(n, lmax=lmax, seed_k=4, geom_seed=4000 + 10 * k))
    return systems


def protein_like(lmax: int = 10, nocc: int = 660, seed_k: int = 5) -> System:
    xyz, el = protein_like_cluster(np.random.default_rng(1000 * seed_k + 0))
    eb = draw_element_basis(np.random.default_rng(1000 * seed_k + 1), SHELLS_HEAVY)
    basis = make_basis(xyz, el, eb)
    C = loewdin_occupied(basis, nocc, np.random.default_rng(1000 * seed_k + 2))
    return System("C202H317O64N55S6-like", basis, nocc, C, depth=0,
                  target_atoms_per_leaf=8.0, lmax=lmax)


def small_sp(natom: int = 6, nocc: int = 4, spacing: float = 3.2, seed: int = 7,
             lmax: int = 2, depth: int = 2) -> System:
    """Tiny s/p test system on a bent line (used for brute-force (sp|sp) checks)."""
    rng = np.random.default_rng(seed)
    xyz = line_atoms(natom, spacing)
    xyz[:, 1] = rng.uniform(-0.4, 0.4, size=natom)
    xyz[:, 2] = rng.uniform(-0.4, 0.4, size=natom)
    eb = {"X": [(0, np.array([4.0, 0.9]), np.array([0.5, 0.6])),
                (1, np.array([1.3]), np.array([1.0]))]}
    basis = make_basis(xyz, ["X"] * natom, eb)
    C = loewdin_occupied(basis, nocc, np.random.default_rng(seed + 1))
    return System(f"sp{natom}", basis, nocc, C, depth=depth, target_atoms_per_leaf=8.0, lmax=lmax)


def reduced(system_fn, **kw) -> System:
    return system_fn(**kw)
