// Host side of the occ-FMM-K library: contexts, the box hierarchy, the ABI.
//
// Compiled with -ffp-contract=off: every floating-point decision that feeds
// the integer tree (pair screening, pair centres, box indices) is a plain IEEE
// double expression evaluated in a fixed order, so the tree is reproducible.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <set>
#include <tuple>
#include <vector>

#include "occk_internal.h"

using occk::OpDesc;
using occk::PairDesc;

namespace {

occk_status fail(occk_ctx* ctx, occk_status code, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return code;
}

occk_status cuda_fail(occk_ctx* ctx, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(ctx, OCCK_ERR_CUDA, m);
}

template <typename T>
cudaError_t upload(T** dst, const std::vector<T>& v) {
    *dst = nullptr;
    if (v.empty()) return cudaSuccess;
    cudaError_t e = cudaMalloc((void**)dst, v.size() * sizeof(T));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

template <typename T>
void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

cudaError_t ensure(occk::DevBuf& b, size_t bytes) {
    if (b.bytes >= bytes && b.p) return cudaSuccess;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    if (bytes == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e == cudaSuccess) b.bytes = bytes;
    return e;
}

void free_tree_device(occk_tree* t) {
    auto& d = t->dev;
    dfree(d.row_ptr); dfree(d.ent_col); dfree(d.ent_val);
    dfree(d.leaf_rowoff); dfree(d.leaf_aos); dfree(d.ao_row_ptr); dfree(d.ao_rows);
    dfree(d.child_ptr); dfree(d.child_list); dfree(d.m2m_op);
    dfree(d.m2l_ptr); dfree(d.m2l_src); dfree(d.m2l_op);
    dfree(d.m2l_lmax_full); dfree(d.m2l_lmax_edge); dfree(d.parent);
    dfree(d.pairs); dfree(d.prim_exp); dfree(d.prim_coef);
    dfree(d.pair_vals); dfree(d.pair_vals_f); dfree(d.ops); dfree(d.ops_f); dfree(d.opdesc);
    dfree(d.l2l_op); dfree(d.lscale); dfree(d.box_scale);
    dfree(d.box_key); dfree(d.box_level); dfree(d.hlev); dfree(d.m2l_tgt);
    dfree(d.grp_child); dfree(d.grp_parent); dfree(d.grp_ptr); dfree(d.grp_src); dfree(d.grp_op);
}

inline long long ifloor_clamp(double v, long long n) {
    double f = std::floor(v);
    long long k = (long long)f;
    if (k < 0) k = 0;
    if (k > n - 1) k = n - 1;
    return k;
}

}  // namespace

// ===========================================================================
// Context
// ===========================================================================

extern "C" occk_status occk_create(occk_ctx** out, int device) {
    if (!out) return OCCK_ERR_ARG;
    *out = nullptr;
    occk_ctx* c = new (std::nothrow) occk_ctx();
    if (!c) return OCCK_ERR_OOM;
    c->device = device;
    if (device >= 0) {
        int n = 0;
        cudaError_t e = cudaGetDeviceCount(&n);
        if (e != cudaSuccess || device >= n) {
            delete c;
            return OCCK_ERR_UNSUPPORTED;
        }
        e = cudaSetDevice(device);
        if (e != cudaSuccess) {
            delete c;
            return OCCK_ERR_CUDA;
        }
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    }
    *out = c;
    return OCCK_OK;
}

extern "C" void occk_destroy(occk_ctx* c) {
    if (!c) return;
    if (c->device >= 0) {
        cudaSetDevice(c->device);
        for (int k = 0; k <= OCCK_NSTAGE; ++k)
            if (c->ev[k]) cudaEventDestroy(c->ev[k]);
        for (occk::DevBuf* b : {&c->ct, &c->w, &c->obox, &c->mbox, &c->kb, &c->part, &c->edev,
                                &c->scratch, &c->mlp_prm, &c->mlp_norm, &c->mlp_m, &c->mlp_v, &c->mlp_h,
                                &c->mlp_grad, &c->mlp_ws, &c->feat, &c->pred, &c->ranks, &c->nrm, &c->gram, &c->rank_err,
                                &c->pplan, &c->panels, &c->tpan, &c->tscale, &c->tops, &c->sob, &c->smb,
                                &c->jbox, &c->scr_o, &c->scr_m, &c->scr_aux, &c->splan, &c->spanels}) {
            if (b->p) cudaFree(b->p);
            b->p = nullptr;
        }
    }
    delete c;
}

extern "C" const char* occk_last_error(const occk_ctx* c) {
    if (!c) return "null context";
    return c->err.c_str();
}

// ===========================================================================
// Tree
// ===========================================================================

namespace {

struct Key3 {
    long long x, y, z;
    bool operator<(const Key3& o) const {
        return std::tie(x, y, z) < std::tie(o.x, o.y, o.z);
    }
    bool operator==(const Key3& o) const { return x == o.x && y == o.y && z == o.z; }
};

inline long long cheb(const Key3& a, const Key3& b) {
    long long dx = std::llabs(a.x - b.x), dy = std::llabs(a.y - b.y), dz = std::llabs(a.z - b.z);
    return std::max(dx, std::max(dy, dz));
}

}  // namespace

extern "C" occk_status occk_build_tree(occk_ctx* ctx, const occk_basis* bs,
                                       const occk_tree_params* prm, occk_tree** out) {
    if (!ctx || !bs || !prm || !out) return fail(ctx, OCCK_ERR_ARG, "null argument");
    *out = nullptr;
    if (bs->natom <= 0 || bs->nshell <= 0 || !bs->xyz || !bs->shell_atom || !bs->shell_l ||
        !bs->shell_nprim || !bs->exps || !bs->coefs)
        return fail(ctx, OCCK_ERR_ARG, "basis: empty or null arrays");
    if (prm->ws_boxes != 1)
        return fail(ctx, OCCK_ERR_UNSUPPORTED, "only ws_boxes = 1 (nearest neighbours excluded)");
    if (prm->depth < 0 || prm->depth > 20)
        return fail(ctx, OCCK_ERR_ARG, "depth out of range");
    if (prm->depth == 0 && !(prm->target_atoms_per_leaf > 0))
        return fail(ctx, OCCK_ERR_ARG, "target_atoms_per_leaf must be > 0 when depth = 0");

    occk_tree* t = new (std::nothrow) occk_tree();
    if (!t) return fail(ctx, OCCK_ERR_OOM, "host allocation");
    t->device = ctx->device;
    const int ns = bs->nshell;
    t->natom = bs->natom;
    t->nshell = ns;
    t->shell_l.resize(ns);
    t->shell_nprim.resize(ns);
    t->shell_prim_off.resize(ns + 1);
    t->shell_ao_off.resize(ns + 1);
    t->shell_xyz.resize(3 * ns);
    t->shell_prim_off[0] = 0;
    t->shell_ao_off[0] = 0;
    for (int s = 0; s < ns; ++s) {
        int a = bs->shell_atom[s];
        int l = bs->shell_l[s];
        int np = bs->shell_nprim[s];
        if (a < 0 || a >= bs->natom || np < 1) {
            delete t;
            return fail(ctx, OCCK_ERR_ARG, "basis: bad shell_atom or shell_nprim");
        }
        if (l != 0 && l != 1) {
            delete t;
            return fail(ctx, OCCK_ERR_UNSUPPORTED, "only s and p shells are supported");
        }
        t->shell_l[s] = l;
        t->shell_nprim[s] = np;
        t->shell_prim_off[s + 1] = t->shell_prim_off[s] + np;
        t->shell_ao_off[s + 1] = t->shell_ao_off[s] + (l == 0 ? 1 : 3);
        for (int k = 0; k < 3; ++k) t->shell_xyz[3 * s + k] = bs->xyz[3 * a + k];
    }
    t->nao = t->shell_ao_off[ns];
    const int nprim = t->shell_prim_off[ns];
    for (int p = 0; p < nprim; ++p) {
        if (!(bs->exps[p] > 0)) {
            delete t;
            return fail(ctx, OCCK_ERR_ARG, "basis: exponents must be positive");
        }
    }

    // ---- primitive coefficients with primitive and contracted normalisation
    t->prim_exp.assign(bs->exps, bs->exps + nprim);
    t->prim_coef.resize(nprim);
    for (int s = 0; s < ns; ++s) {
        int o = t->shell_prim_off[s], np = t->shell_nprim[s], l = t->shell_l[s];
        std::vector<double> d(np);
        for (int p = 0; p < np; ++p) {
            double a = bs->exps[o + p];
            double n = std::pow(2.0 * a / M_PI, 0.75);
            if (l == 1) n = n * 2.0 * std::sqrt(a);
            d[p] = bs->coefs[o + p] * n;
        }
        double self = 0.0;
        for (int p = 0; p < np; ++p)
            for (int q = 0; q < np; ++q) {
                double pq = bs->exps[o + p] + bs->exps[o + q];
                double v = std::pow(M_PI / pq, 1.5);
                if (l == 1) v = v / (2.0 * pq);
                self += d[p] * d[q] * v;
            }
        double inv = 1.0 / std::sqrt(self);
        for (int p = 0; p < np; ++p) t->prim_coef[o + p] = d[p] * inv;
    }

    // ---- screened shell pairs (a <= b) and their centres
    const double thresh = prm->pair_thresh;
    std::vector<double> cen;
    for (int a = 0; a < ns; ++a) {
        const double* A = &t->shell_xyz[3 * a];
        for (int b = a; b < ns; ++b) {
            const double* B = &t->shell_xyz[3 * b];
            double dx = A[0] - B[0], dy = A[1] - B[1], dz = A[2] - B[2];
            double R2 = dx * dx + dy * dy + dz * dz;
            double est = 0.0, sw = 0.0, swx[3] = {0.0, 0.0, 0.0};
            int oa = t->shell_prim_off[a], ob = t->shell_prim_off[b];
            for (int p = 0; p < t->shell_nprim[a]; ++p) {
                for (int q = 0; q < t->shell_nprim[b]; ++q) {
                    double ea = bs->exps[oa + p], eb = bs->exps[ob + q];
                    double ca = bs->coefs[oa + p], cb = bs->coefs[ob + q];
                    double pp = ea + eb;
                    double mu = ea * eb / pp;
                    double w = std::exp(-mu * R2);
                    double tt = 2.0 * std::sqrt(ea * eb) / pp;
                    double e = std::fabs(ca * cb) * (tt * std::sqrt(tt)) * w;
                    est = std::max(est, e);
                    sw = sw + w;
                    for (int k = 0; k < 3; ++k) {
                        double P = (ea * A[k] + eb * B[k]) / pp;
                        swx[k] = swx[k] + w * P;
                    }
                }
            }
            if (est > thresh) {
                t->pair_a.push_back(a);
                t->pair_b.push_back(b);
                for (int k = 0; k < 3; ++k) cen.push_back(swx[k] / sw);
            }
        }
    }
    const int npair = (int)t->pair_a.size();
    if (npair == 0) {
        delete t;
        return fail(ctx, OCCK_ERR_ARG, "no shell pair passes the screen");
    }
    t->pair_centre = cen;

    // ---- root cube
    double lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = cen[k];
        hi[k] = cen[k];
    }
    for (int i = 1; i < npair; ++i)
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], cen[3 * i + k]);
            hi[k] = std::max(hi[k], cen[3 * i + k]);
        }
    double extent = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
    double delta = extent > 0 ? 1e-6 * extent : 1e-6;
    for (int k = 0; k < 3; ++k) t->x0[k] = lo[k] - delta;
    t->side = extent + 2.0 * delta;

    // ---- depth
    int D = prm->depth;
    if (D <= 0) {
        double best_err = -1.0;
        int best_D = 1;
        for (int d = 1; d <= 12; ++d) {
            long long n = 1LL << d;
            double h = t->side / (double)n;
            std::set<Key3> occ;
            for (int i = 0; i < bs->natom; ++i) {
                Key3 kk;
                kk.x = ifloor_clamp((bs->xyz[3 * i + 0] - t->x0[0]) / h, n);
                kk.y = ifloor_clamp((bs->xyz[3 * i + 1] - t->x0[1]) / h, n);
                kk.z = ifloor_clamp((bs->xyz[3 * i + 2] - t->x0[2]) / h, n);
                occ.insert(kk);
            }
            double mean = (double)bs->natom / (double)occ.size();
            double err = std::fabs(mean - prm->target_atoms_per_leaf);
            if (best_err < 0 || err < best_err) {
                best_err = err;
                best_D = d;
            }
        }
        D = best_D;
    }
    t->depth = D;
    const long long nD = 1LL << D;
    const double hD = t->side / (double)nD;
    std::vector<Key3> leafkey(npair);
    for (int i = 0; i < npair; ++i) {
        leafkey[i].x = ifloor_clamp((cen[3 * i + 0] - t->x0[0]) / hD, nD);
        leafkey[i].y = ifloor_clamp((cen[3 * i + 1] - t->x0[1]) / hD, nD);
        leafkey[i].z = ifloor_clamp((cen[3 * i + 2] - t->x0[2]) / hD, nD);
    }

    // ---- boxes per level, ordered (level, ix, iy, iz)
    t->level_off.assign(1, 0);
    std::vector<std::map<Key3, int>> index(D + 1);
    std::vector<Key3> keys;
    std::vector<int> level;
    for (int lev = 0; lev <= D; ++lev) {
        std::set<Key3> u;
        int sh = D - lev;
        for (auto& k : leafkey) u.insert(Key3{k.x >> sh, k.y >> sh, k.z >> sh});
        for (auto& k : u) {
            index[lev][k] = (int)keys.size();
            keys.push_back(k);
            level.push_back(lev);
        }
        t->level_off.push_back((int)keys.size());
    }
    const int nbox = (int)keys.size();
    t->h.resize(D + 1);
    for (int lev = 0; lev <= D; ++lev) t->h[lev] = t->side / (double)(1LL << lev);
    t->box_key.resize(3 * nbox);
    t->parent.assign(nbox, -1);
    t->centre.resize(3 * nbox);
    for (int b = 0; b < nbox; ++b) {
        t->box_key[3 * b + 0] = (int)keys[b].x;
        t->box_key[3 * b + 1] = (int)keys[b].y;
        t->box_key[3 * b + 2] = (int)keys[b].z;
        int lev = level[b];
        if (lev > 0) t->parent[b] = index[lev - 1][Key3{keys[b].x >> 1, keys[b].y >> 1, keys[b].z >> 1}];
        const long long kk[3] = {keys[b].x, keys[b].y, keys[b].z};
        for (int k = 0; k < 3; ++k)
            t->centre[3 * b + k] = t->x0[k] + ((double)kk[k] + 0.5) * t->h[lev];
    }

    // ---- interaction lists, levels 2..D
    for (int lev = 2; lev <= D; ++lev) {
        int lo_ = t->level_off[lev], hi_ = t->level_off[lev + 1];
        for (int a = lo_; a < hi_; ++a) {
            Key3 pa{keys[a].x >> 1, keys[a].y >> 1, keys[a].z >> 1};
            for (int c = lo_; c < hi_; ++c) {
                Key3 pc{keys[c].x >> 1, keys[c].y >> 1, keys[c].z >> 1};
                if (cheb(pa, pc) <= 1 && cheb(keys[a], keys[c]) > 1) {
                    t->m2l_tgt.push_back(a);
                    t->m2l_src.push_back(c);
                }
            }
        }
    }

    // ---- pair -> leaf, leaf AO sets
    const int leaf0 = t->level_off[D];
    const int nleaf = t->level_off[D + 1] - leaf0;
    t->pair_leaf.resize(npair);
    std::vector<std::set<int>> aoset(nleaf);
    for (int i = 0; i < npair; ++i) {
        int leaf = index[D][leafkey[i]];
        t->pair_leaf[i] = leaf;
        int a = t->pair_a[i], b = t->pair_b[i];
        for (int r = t->shell_ao_off[a]; r < t->shell_ao_off[a + 1]; ++r) aoset[leaf - leaf0].insert(r);
        for (int r = t->shell_ao_off[b]; r < t->shell_ao_off[b + 1]; ++r) aoset[leaf - leaf0].insert(r);
    }
    t->leaf_rowoff.assign(1, 0);
    std::vector<std::map<int, int>> localrow(nleaf);
    for (int B = 0; B < nleaf; ++B) {
        for (int r : aoset[B]) {
            localrow[B][r] = (int)t->leaf_aos.size() - t->leaf_rowoff[B];
            t->leaf_aos.push_back(r);
        }
        t->leaf_rowoff.push_back((int)t->leaf_aos.size());
    }
    const int nrow = (int)t->leaf_aos.size();

    // ---- ordered AO-pair entries (row r, column s, value row)
    std::vector<std::vector<std::pair<int, int>>> rows(nrow);
    int vo = 0;
    for (int i = 0; i < npair; ++i) {
        int a = t->pair_a[i], b = t->pair_b[i];
        int B = t->pair_leaf[i] - leaf0;
        int na = t->shell_ao_off[a + 1] - t->shell_ao_off[a];
        int nb = t->shell_ao_off[b + 1] - t->shell_ao_off[b];
        for (int ia = 0; ia < na; ++ia)
            for (int ib = 0; ib < nb; ++ib) {
                int r = t->shell_ao_off[a] + ia, s = t->shell_ao_off[b] + ib;
                int v = vo + ia * nb + ib;
                rows[t->leaf_rowoff[B] + localrow[B][r]].push_back({s, v});
                if (a != b) rows[t->leaf_rowoff[B] + localrow[B][s]].push_back({r, v});
            }
        vo += na * nb;
    }
    t->nvals = vo;
    t->row_ptr.assign(1, 0);
    for (int r = 0; r < nrow; ++r) {
        for (auto& e : rows[r]) {
            t->ent_col.push_back(e.first);
            t->ent_val.push_back(e.second);
        }
        t->row_ptr.push_back((int)t->ent_col.size());
    }
    // AO -> rows
    std::vector<std::vector<int>> aorows(t->nao);
    for (int r = 0; r < nrow; ++r) aorows[t->leaf_aos[r]].push_back(r);
    t->ao_row_ptr.assign(1, 0);
    for (int r = 0; r < t->nao; ++r) {
        for (int x : aorows[r]) t->ao_rows.push_back(x);
        t->ao_row_ptr.push_back((int)t->ao_rows.size());
    }

    // ---- translation schedule: distinct operators per (kind, level, offset)
    std::map<std::tuple<int, int, int, int, int>, int> opid;
    auto get_op = [&](int kind, int lev, int ox, int oy, int oz) {
        auto key = std::make_tuple(kind, lev, ox, oy, oz);
        auto it = opid.find(key);
        if (it != opid.end()) return it->second;
        OpDesc d{};
        d.kind = kind;
        if (kind == 2) {
            d.d[0] = (double)ox * t->h[lev];
            d.d[1] = (double)oy * t->h[lev];
            d.d[2] = (double)oz * t->h[lev];
        } else {
            d.d[0] = ((double)ox - 0.5) * t->h[lev];
            d.d[1] = ((double)oy - 0.5) * t->h[lev];
            d.d[2] = ((double)oz - 0.5) * t->h[lev];
        }
        int id = (int)t->ops.size();
        t->ops.push_back(d);
        opid[key] = id;
        return id;
    };
    t->m2m_op.assign(nbox, -1);
    t->l2l_op.assign(nbox, -1);
    std::vector<std::vector<int>> ch(nbox);
    for (int lev = 3; lev <= D; ++lev)
        for (int c = t->level_off[lev]; c < t->level_off[lev + 1]; ++c) {
            int ox = (int)(keys[c].x & 1), oy = (int)(keys[c].y & 1), oz = (int)(keys[c].z & 1);
            t->m2m_op[c] = get_op(0, lev, ox, oy, oz);
            t->l2l_op[c] = get_op(1, lev, ox, oy, oz);
            ch[t->parent[c]].push_back(c);
        }
    t->child_ptr.assign(1, 0);
    for (int b = 0; b < nbox; ++b) {
        for (int c : ch[b]) t->child_list.push_back(c);
        t->child_ptr.push_back((int)t->child_list.size());
    }
    const int ne = (int)t->m2l_tgt.size();
    t->m2l_op.resize(ne);
    t->m2l_ptr.assign(nbox + 1, 0);
    for (int e = 0; e < ne; ++e) {
        int a = t->m2l_tgt[e], c = t->m2l_src[e];
        int lev = level[a];
        t->m2l_op[e] = get_op(2, lev, (int)(keys[a].x - keys[c].x), (int)(keys[a].y - keys[c].y),
                              (int)(keys[a].z - keys[c].z));
        t->m2l_ptr[a + 1]++;
    }
    for (int b = 0; b < nbox; ++b) t->m2l_ptr[b + 1] += t->m2l_ptr[b];
    // sibling groups of the M2L pass (levels 2..D): one group per parent
    t->grp_level_off.assign(D + 2, 0);
    t->grp_gain.assign(D + 1, 0.0);
    t->grp_ptr.assign(1, 0);
    {
        int ng = 0;
        for (int lev = 0; lev <= D; ++lev) {
            if (lev >= 2) t->grp_level_off[lev] = ng;
            if (lev < 2) continue;
            std::map<int, std::vector<int>> kids;      // parent -> children, both ascending
            for (int c = t->level_off[lev]; c < t->level_off[lev + 1]; ++c) kids[t->parent[c]].push_back(c);
            long long nedge = 0, nunion = 0;
            for (auto& pk : kids) {
                std::vector<int> slots(8, -1);
                std::map<int, std::vector<int>> srcop;   // source -> op per slot
                const int nk = std::min<int>(8, (int)pk.second.size());
                for (int k = 0; k < nk; ++k) {
                    const int c = pk.second[k];
                    slots[k] = c;
                    for (int e = t->m2l_ptr[c]; e < t->m2l_ptr[c + 1]; ++e) {
                        auto& v = srcop[t->m2l_src[e]];
                        if (v.empty()) v.assign(8, -1);
                        v[k] = t->m2l_op[e];
                        ++nedge;
                    }
                }
                for (int k = 0; k < 8; ++k) t->grp_child.push_back(slots[k]);
                t->grp_parent.push_back(pk.first);
                for (auto& so : srcop) {
                    t->grp_src.push_back(so.first);
                    for (int k = 0; k < 8; ++k) t->grp_op.push_back(so.second[k]);
                }
                nunion += (long long)srcop.size();
                t->grp_ptr.push_back((int)t->grp_src.size());
                ++ng;
            }
            t->grp_gain[lev] = nunion > 0 ? (double)nedge / (double)nunion : 0.0;
        }
        t->grp_level_off[D + 1] = ng;
        if (D < 2) t->grp_level_off.assign(D + 2, 0);
    }

    // ---- device upload
    if (ctx->device >= 0) {
        cudaError_t e = cudaSetDevice(ctx->device);
        auto& d = t->dev;
        std::vector<PairDesc> pd(npair);
        int voff = 0;
        for (int i = 0; i < npair; ++i) {
            int a = t->pair_a[i], b = t->pair_b[i];
            PairDesc& p = pd[i];
            for (int k = 0; k < 3; ++k) {
                p.A[k] = t->shell_xyz[3 * a + k];
                p.B[k] = t->shell_xyz[3 * b + k];
                p.X[k] = t->centre[3 * t->pair_leaf[i] + k];
            }
            p.prim_a = t->shell_prim_off[a];
            p.nprim_a = t->shell_nprim[a];
            p.prim_b = t->shell_prim_off[b];
            p.nprim_b = t->shell_nprim[b];
            p.la = t->shell_l[a];
            p.lb = t->shell_l[b];
            p.val_off = voff;
            voff += (p.la ? 3 : 1) * (p.lb ? 3 : 1);
        }
        std::vector<int> m2l_src_dev(t->m2l_src), lmfull(ne, 0);
        if (e == cudaSuccess) e = upload(&d.row_ptr, t->row_ptr);
        if (e == cudaSuccess) e = upload(&d.ent_col, t->ent_col);
        if (e == cudaSuccess) e = upload(&d.ent_val, t->ent_val);
        if (e == cudaSuccess) e = upload(&d.leaf_rowoff, t->leaf_rowoff);
        if (e == cudaSuccess) e = upload(&d.leaf_aos, t->leaf_aos);
        if (e == cudaSuccess) e = upload(&d.ao_row_ptr, t->ao_row_ptr);
        if (e == cudaSuccess) e = upload(&d.ao_rows, t->ao_rows);
        if (e == cudaSuccess) e = upload(&d.child_ptr, t->child_ptr);
        if (e == cudaSuccess) e = upload(&d.child_list, t->child_list);
        if (e == cudaSuccess) e = upload(&d.m2m_op, t->m2m_op);
        if (e == cudaSuccess) e = upload(&d.l2l_op, t->l2l_op);
        if (e == cudaSuccess) e = upload(&d.m2l_ptr, t->m2l_ptr);
        if (e == cudaSuccess) e = upload(&d.m2l_src, m2l_src_dev);
        if (e == cudaSuccess) e = upload(&d.m2l_op, t->m2l_op);
        if (e == cudaSuccess) e = upload(&d.parent, t->parent);
        if (e == cudaSuccess) e = upload(&d.pairs, pd);
        if (e == cudaSuccess) e = upload(&d.prim_exp, t->prim_exp);
        if (e == cudaSuccess) e = upload(&d.prim_coef, t->prim_coef);
        if (e == cudaSuccess) e = upload(&d.opdesc, t->ops);
        if (e == cudaSuccess) e = upload(&d.m2l_lmax_full, lmfull);
        if (e == cudaSuccess) e = upload(&d.box_key, t->box_key);
        if (e == cudaSuccess) e = upload(&d.box_level, level);
        if (e == cudaSuccess) e = upload(&d.hlev, t->h);
        if (e == cudaSuccess) e = upload(&d.m2l_tgt, t->m2l_tgt);
        if (!t->grp_parent.empty()) {
            if (e == cudaSuccess) e = upload(&d.grp_child, t->grp_child);
            if (e == cudaSuccess) e = upload(&d.grp_parent, t->grp_parent);
            if (e == cudaSuccess) e = upload(&d.grp_ptr, t->grp_ptr);
            if (e == cudaSuccess && !t->grp_src.empty()) e = upload(&d.grp_src, t->grp_src);
            if (e == cudaSuccess && !t->grp_op.empty()) e = upload(&d.grp_op, t->grp_op);
        }
        if (e != cudaSuccess) {
            free_tree_device(t);
            delete t;
            return cuda_fail(ctx, e, "occk_build_tree upload");
        }
    }
    *out = t;
    return OCCK_OK;
}

extern "C" void occk_tree_destroy(occk_tree* t) {
    if (!t) return;
    if (t->device >= 0) {
        cudaSetDevice(t->device);
        free_tree_device(t);
    }
    delete t;
}

extern "C" occk_status occk_query(const occk_tree* t, occk_tree_info* info) {
    if (!t || !info) return OCCK_ERR_ARG;
    info->nao = t->nao;
    info->natom = t->natom;
    info->nshell = t->nshell;
    info->depth = t->depth;
    info->nbox = (int)t->parent.size();
    info->nleaf = (int)t->leaf_rowoff.size() - 1;
    info->npair = (int)t->pair_a.size();
    info->nentry = (int)t->ent_col.size();
    info->nrow = (int)t->leaf_aos.size();
    info->nm2l = (int)t->m2l_tgt.size();
    info->lmax = t->lmax;
    for (int k = 0; k < 3; ++k) info->x0[k] = t->x0[k];
    info->side = t->side;
    return OCCK_OK;
}

extern "C" occk_status occk_tree_export(const occk_tree* t, int what, void* out, size_t bytes) {
    if (!t || !out) return OCCK_ERR_ARG;
    std::vector<int> iv;
    const void* src = nullptr;
    size_t n = 0;
    switch (what) {
        case OCCK_TREE_LEVEL_OFF: src = t->level_off.data(); n = t->level_off.size() * 4; break;
        case OCCK_TREE_BOX_KEY: src = t->box_key.data(); n = t->box_key.size() * 4; break;
        case OCCK_TREE_PARENT: src = t->parent.data(); n = t->parent.size() * 4; break;
        case OCCK_TREE_CENTRE: src = t->centre.data(); n = t->centre.size() * 8; break;
        case OCCK_TREE_M2L:
            for (size_t e = 0; e < t->m2l_tgt.size(); ++e) {
                iv.push_back(t->m2l_tgt[e]);
                iv.push_back(t->m2l_src[e]);
            }
            src = iv.data(); n = iv.size() * 4; break;
        case OCCK_TREE_PAIRS:
            for (size_t e = 0; e < t->pair_a.size(); ++e) {
                iv.push_back(t->pair_a[e]);
                iv.push_back(t->pair_b[e]);
                iv.push_back(t->pair_leaf[e]);
            }
            src = iv.data(); n = iv.size() * 4; break;
        case OCCK_TREE_PAIR_CENTRE: src = t->pair_centre.data(); n = t->pair_centre.size() * 8; break;
        case OCCK_TREE_LEAF_AOS: src = t->leaf_aos.data(); n = t->leaf_aos.size() * 4; break;
        case OCCK_TREE_LEAF_ROWOFF: src = t->leaf_rowoff.data(); n = t->leaf_rowoff.size() * 4; break;
        default: return OCCK_ERR_ARG;
    }
    if (n != bytes) return OCCK_ERR_SHAPE;
    if (n) std::memcpy(out, src, n);
    return OCCK_OK;
}

// ===========================================================================
// Pair multipoles and operators (step a0)
// ===========================================================================

extern "C" occk_status occk_pair_multipoles(occk_ctx* ctx, occk_tree* t, int lmax, void* stream) {
    if (!ctx || !t) return fail(ctx, OCCK_ERR_ARG, "null argument");
    if (ctx->device < 0 || t->device != ctx->device)
        return fail(ctx, OCCK_ERR_UNSUPPORTED, "no device bound to this context or tree");
    if (lmax < 0 || lmax > 12) return fail(ctx, OCCK_ERR_UNSUPPORTED, "lmax must be in 0..12");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(ctx->device);
    auto& d = t->dev;
    const int nc = occk::ncomp(lmax);
    const int nops = (int)t->ops.size();
    dfree(d.pair_vals); dfree(d.pair_vals_f); dfree(d.ops); dfree(d.ops_f);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d.pair_vals, sizeof(double) * (size_t)t->nvals * nc);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d.pair_vals_f, sizeof(float) * (size_t)t->nvals * nc);
    if (nops > 0) {
        if (e == cudaSuccess) e = cudaMalloc((void**)&d.ops, sizeof(double) * (size_t)nops * nc * nc);
        if (e == cudaSuccess) e = cudaMalloc((void**)&d.ops_f, sizeof(float) * (size_t)nops * nc * nc);
    }
    if (e != cudaSuccess) {
        dfree(d.pair_vals); dfree(d.pair_vals_f); dfree(d.ops); dfree(d.ops_f);
        return e == cudaErrorMemoryAllocation ? fail(ctx, OCCK_ERR_OOM, "pair multipole storage")
                                              : cuda_fail(ctx, e, "occk_pair_multipoles alloc");
    }
    {
        // per-component scale factors of the low-precision forms at the leaf
        // level, sqrt((l+m)!(l-m)!) / h^l: they bring every component of the
        // leaf multipoles to O(1), so no FP16 operand of steps (a) and (e)
        // overflows or flushes to zero at high l
        std::vector<float> ls(nc), bsc(t->parent.size());
        const double sl = t->h[t->depth];
        for (int l = 0; l <= lmax; ++l)
            for (int c = l * l; c < (l + 1) * (l + 1); ++c) {
                const int m = c == l * l ? 0 : (c - l * l + 1) / 2;
                ls[c] = (float)(std::sqrt(std::tgamma(l + m + 1.0) * std::tgamma(l - m + 1.0)) / std::pow(sl, l));
            }
        for (size_t b = 0; b < bsc.size(); ++b) {
            int lev = 0;
            while (lev + 1 < (int)t->level_off.size() && t->level_off[lev + 1] <= (int)b) ++lev;
            bsc[b] = (float)t->h[lev];
        }
        dfree(d.lscale);
        dfree(d.box_scale);
        if (e == cudaSuccess) e = upload(&d.lscale, ls);
        if (e == cudaSuccess) e = upload(&d.box_scale, bsc);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "scale upload");
    }
    e = occk::launch_pair_multipoles(d.pairs, (int)t->pair_a.size(), d.prim_exp, d.prim_coef, lmax,
                                     d.pair_vals, d.pair_vals_f, t->nvals, s);
    if (e == cudaSuccess && nops > 0) e = occk::launch_gen_ops(d.opdesc, nops, lmax, d.ops, d.ops_f, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "occk_pair_multipoles launch");
    t->lmax = lmax;
    static std::atomic<long long> gen_counter{0};
    t->gen = ++gen_counter;
    return OCCK_OK;
}

extern "C" occk_status occk_set_edge_lmax(occk_ctx* ctx, occk_tree* t, const int* ranks, int n) {
    if (!ctx || !t || !ranks) return fail(ctx, OCCK_ERR_ARG, "null argument");
    if (n != (int)t->m2l_tgt.size()) return fail(ctx, OCCK_ERR_SHAPE, "ranks length != nm2l");
    if (t->lmax < 0) return fail(ctx, OCCK_ERR_STATE, "call occk_pair_multipoles first");
    for (int i = 0; i < n; ++i)
        if (ranks[i] < 0 || ranks[i] > t->lmax) return fail(ctx, OCCK_ERR_ARG, "rank out of [0, lmax]");
    t->edge_lmax.assign(ranks, ranks + n);
    if (ctx->device >= 0 && n > 0) {
        cudaSetDevice(ctx->device);
        dfree(t->dev.m2l_lmax_edge);
        cudaError_t e = upload(&t->dev.m2l_lmax_edge, t->edge_lmax);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "occk_set_edge_lmax");
    }
    return OCCK_OK;
}

// ===========================================================================
// Far-field K (steps a-e)
// ===========================================================================

namespace occk {
FmmArgs simt_args(const occk_ctx* ctx, const occk_tree* t, int nocc, int prec, const double* C, int ldc, double* K,
                  int ldk, double* Ex, void* ct, void* w, void* obox, void* mbox, double* kb, double* part,
                  int* err_word) {
    FmmArgs a{};
    const int L = t->lmax, D = t->depth;
    const int nbox = (int)t->parent.size();
    const int nleaf = (int)t->leaf_rowoff.size() - 1;
    int max_rows = 0;
    for (int B = 0; B < nleaf; ++B) max_rows = std::max(max_rows, t->leaf_rowoff[B + 1] - t->leaf_rowoff[B]);
    auto& d = t->dev;
    a.nao = t->nao; a.nocc = nocc; a.ldc = ldc; a.ldk = ldk; a.nc = ncomp(L); a.L = L; a.depth = D;
    a.nbox = nbox; a.first_box = D >= 2 ? t->level_off[2] : nbox; a.nleaf = nleaf; a.leaf0 = t->level_off[D];
    a.nrow = (int)t->leaf_aos.size();
    a.level_off = t->level_off.data();
    a.prec = prec; a.C = C; a.K = K; a.Ex_dev = Ex;
    a.row_ptr = d.row_ptr; a.ent_col = d.ent_col; a.ent_val = d.ent_val;
    a.leaf_rowoff = d.leaf_rowoff; a.leaf_aos = d.leaf_aos;
    a.ao_row_ptr = d.ao_row_ptr; a.ao_rows = d.ao_rows;
    a.child_ptr = d.child_ptr; a.child_list = d.child_list; a.m2m_op = d.m2m_op; a.l2l_op = d.l2l_op;
    a.parent = d.parent;
    a.m2l_ptr = d.m2l_ptr; a.m2l_src = d.m2l_src; a.m2l_op = d.m2l_op; a.m2l_lmax = nullptr;
    a.pair_vals = prec == OCCK_FP64 ? (const void*)d.pair_vals : (const void*)d.pair_vals_f;
    a.ops = prec == OCCK_FP64 ? (const void*)d.ops : (const void*)d.ops_f;
    a.ct = ct; a.w = w; a.obox = obox; a.mbox = mbox; a.kb = kb; a.part = part;
    a.leaf_rowoff_host = t->leaf_rowoff.data();
    a.max_rows = max_rows;
    a.l2p_nsplit = 1;
    a.ev = nullptr;
    a.lscale = d.lscale; a.box_scale = d.box_scale;
    a.err_word = err_word;
    a.tr_pan = nullptr; a.ops_scaled = nullptr; a.tr_nlev = D + 1; a.tr_on = 0; a.tr_mask = 0;
    a.sm_count = ctx->sm_count;
    a.inv_h_leaf = (float)(1.0 / t->h[D]);
    a.box_level = d.box_level;
    a.learned = 0;
    return a;
}
}  // namespace occk

extern "C" occk_status occk_farfield_K(occk_ctx* ctx, const occk_tree* tc, int nocc,
                                       const double* C_dev, int ldc, int prec, int lmax_policy,
                                       double* K_dev, int ldk, double* Ex_dev, double* Ex_host,
                                       void* stream) {
    if (!ctx || !tc) return fail(ctx, OCCK_ERR_ARG, "null argument");
    occk_tree* t = const_cast<occk_tree*>(tc);
    if (ctx->device < 0 || t->device != ctx->device)
        return fail(ctx, OCCK_ERR_UNSUPPORTED, "no device bound to this context or tree");
    if (t->lmax < 0) return fail(ctx, OCCK_ERR_STATE, "call occk_pair_multipoles first");
    if (nocc <= 0 || !C_dev || !K_dev) return fail(ctx, OCCK_ERR_ARG, "nocc <= 0 or null C/K");
    if (nocc > 65535) return fail(ctx, OCCK_ERR_SHAPE, "nocc above 65535 (pair indices are 32-bit)");
    if (ldc < t->nao || ldk < t->nao) return fail(ctx, OCCK_ERR_SHAPE, "ldc/ldk < nao");
    if (prec < OCCK_FP64 || prec > OCCK_FP16X3) return fail(ctx, OCCK_ERR_ARG, "unknown precision");
    if (lmax_policy < 0 || lmax_policy > 2) return fail(ctx, OCCK_ERR_ARG, "lmax_policy must be 0, 1 or 2");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");

    const int L = t->lmax, nc = occk::ncomp(L), D = t->depth;
    const int nbox = (int)t->parent.size();
    const int first = D >= 2 ? t->level_off[2] : nbox;
    const int nleaf = (int)t->leaf_rowoff.size() - 1;
    const int nrow = (int)t->leaf_aos.size();
    const size_t P = (size_t)nocc * (nocc + 1) / 2;   // stored occupied pairs i <= j
    const size_t es = prec == OCCK_FP64 ? 8 : 4;
    int max_rows = 0;
    for (int B = 0; B < nleaf; ++B) max_rows = std::max(max_rows, t->leaf_rowoff[B + 1] - t->leaf_rowoff[B]);

    size_t nstore = (size_t)(nbox - first);
    size_t bytes_ct = es * (size_t)t->nao * nocc;
    size_t bytes_w = es * (size_t)nc * nrow * nocc;
    size_t bytes_box = es * nstore * nc * P;
    // Step (e): split the (lm, j) range until the grid covers the GPU about
    // eight times; each split writes its own copy of KB, summed by the K
    // reduction.  Tiles and resident blocks per SM: FP64 32 rows x 128 (four
    // 256-thread blocks), FP32 96 x 128 (two), tensor core 128 x 128 (one
    // CTA).  Measured on GB300 (C150H302 L 2 and 6, (H2O)100 L 4): FP32
    // 1.3-1.6x faster than one split, including the longer reduction.
    int l2p_nsplit = 1;
    {
        const bool tcl = occk::tc_mode(prec) >= 0;
        const int rows = tcl ? 128 : (prec == OCCK_FP64 ? 32 : 96);
        const int bps = tcl ? 1 : (prec == OCCK_FP64 ? 4 : 2);
        const int bk = tcl ? 128 / occk::panel_elem_bytes(prec) : (prec == OCCK_FP64 ? 8 : 32);
        long long tiles = 0;
        for (int B = 0; B < nleaf; ++B) tiles += (t->leaf_rowoff[B + 1] - t->leaf_rowoff[B] + rows - 1) / rows;
        tiles *= (nocc + 127) / 128;
        const long long want = 8LL * std::max(ctx->sm_count, 1) * bps;
        const int nkt = nc * ((nocc + bk - 1) / bk);
        l2p_nsplit = (int)std::min<long long>((want + tiles - 1) / std::max<long long>(tiles, 1), 8);
        l2p_nsplit = std::max(1, std::min(l2p_nsplit, nkt / 8));
        if (ctx->l2p_split > 0) l2p_nsplit = std::min(ctx->l2p_split, std::max(1, nkt));
    }
    // FP64 steps (a) and (e) from integer slices on the tensor core: every
    // pair, all columns (the DFMA kernels serve screening and column blocks)
    const int nslices = prec == OCCK_FP64 ? ctx->f64_slices : prec == OCCK_FP32 ? ctx->f32_slices : 0;
    const bool sliced = nslices > 0 && ctx->col_i1 == 0 && ctx->screen_tau <= 0;
    occk::SliceArgs sa{};
    // host plan of the sliced steps, alive until the launches below
    std::vector<long long> offA(nleaf + 1), item0(nleaf + 1), offAa(nleaf + 1), offBa(nleaf + 1);
    std::vector<int> batch_e, batch_a;
    occk::SM2LArgs sm{};
    std::vector<int> m_lt0(D + 2, 0), m_lnt(D + 2, 0), m_lopl0(D + 2, 0), m_lnopl(D + 2, 0), m_ltb(D + 2, 1);
    std::vector<long long> m_lst0(D + 2, 0);
    if (sliced) {
        const int SK = occk::slice_stage_k(), SN = occk::slice_tile_n();
        const int jc = (nocc + SK - 1) / SK, KC = nc * jc, nct = (nocc + SN - 1) / SN;
        std::vector<int> rtA(nleaf);
        long long cA = 0, items1 = 0;
        int max_rt = 0;
        for (int B = 0; B < nleaf; ++B) {
            rtA[B] = (t->leaf_rowoff[B + 1] - t->leaf_rowoff[B] + 127) / 128;
            offA[B] = cA;
            cA += (long long)rtA[B] * KC;
            items1 += (long long)rtA[B] * nct;
            max_rt = std::max(max_rt, rtA[B]);
        }
        offA[nleaf] = cA;
        // K splits: as many as the exact int32 group sums need, more while
        // the tiles cover the GPU less than twice (each split writes a KB copy)
        const int need = (KC + occk::slice_max_stages() - 1) / occk::slice_max_stages();
        const long long fill = (2LL * std::max(ctx->sm_count, 1) + items1 - 1) / std::max<long long>(items1, 1);
        const int nsplit = std::max<int>(need, (int)std::min<long long>(fill, std::max(1, KC / 16)));
        item0[0] = 0;
        for (int B = 0; B < nleaf; ++B) item0[B + 1] = item0[B] + (long long)rtA[B] * nct * nsplit;
        auto al16 = [](size_t x) { return (x + 15) / 16 * 16; };
        const size_t o_off = al16(4 * (size_t)nleaf), o_item = o_off + al16(8 * (size_t)nleaf);
        const size_t o_erow = o_item + al16(8 * (size_t)(nleaf + 1)), o_fcol = o_erow + al16(4 * (size_t)nrow);
        // step (a): panels of C (128 orbitals x 32 AO rows) and of W (32
        // orbitals x 32 AO rows) per leaf; output tiles: triangular pairs of
        // a 128-orbital row tile and a 32-orbital column tile
        const int nti = (nocc + 127) / 128;
        std::vector<int> tpair, kca(nleaf);
        for (int ti = 0; ti < nti; ++ti)
            for (int tj = ti * 128 / SN; tj < nct; ++tj) tpair.push_back(ti | (tj << 16));
        long long cAa = 0, cBa = 0;
        int max_kca = 0;
        for (int B = 0; B < nleaf; ++B) {
            kca[B] = (t->leaf_rowoff[B + 1] - t->leaf_rowoff[B] + SK - 1) / SK;
            offAa[B] = cAa;
            cAa += (long long)nti * kca[B];
            offBa[B] = cBa;
            cBa += (long long)nc * nct * kca[B];
            max_kca = std::max(max_kca, kca[B]);
        }
        offAa[nleaf] = cAa;
        offBa[nleaf] = cBa;
        const size_t o_kca = o_fcol + al16(4 * (size_t)nleaf * nocc), o_offAa = o_kca + al16(4 * (size_t)nleaf);
        const size_t o_offBa = o_offAa + al16(8 * (size_t)nleaf), o_tp = o_offBa + al16(8 * (size_t)nleaf);
        const size_t o_eC = o_tp + al16(4 * tpair.size()), o_eW = o_eC + al16(4 * (size_t)nleaf * nocc);
        const size_t nops = t->ops.size();
        const size_t o_ff = o_eW + al16(4 * (size_t)nleaf * nc * nocc);
        const size_t o_vff = o_ff + al16(8 * nops * nc * nc);
        const size_t o_cff = o_vff + al16(8 * (size_t)t->nvals * nc);
        size_t plan_bytes = o_cff + al16(8 * (size_t)t->nao * nocc);
        // leaf batches whose panels fit a workspace of at most 32 GB (one
        // batch for the protein-sized cluster at L = 2; several at high rank)
        const size_t pa = occk::slice_panel_bytes(nslices, true);
        const size_t pbb = occk::slice_panel_bytes(nslices, false);
        const size_t budget = ctx->slice_budget > 0 ? ctx->slice_budget : size_t(32) << 30;
        auto e_bytes = [&](int B0, int B1) {
            return pa * (size_t)(offA[B1] - offA[B0]) + pbb * (size_t)(B1 - B0) * nct * KC;
        };
        auto a_bytes = [&](int B0, int B1) {
            return pa * (size_t)(offAa[B1] - offAa[B0]) + pbb * (size_t)(offBa[B1] - offBa[B0]);
        };
        size_t need_bytes = 0;
        auto cut = [&](std::vector<int>& bt, auto bytes) {
            bt.assign(1, 0);
            int b0 = 0;
            for (int B = 1; B <= nleaf; ++B)
                if (bytes(b0, B) > budget && B - 1 > b0) {
                    bt.push_back(B - 1);
                    b0 = B - 1;
                }
            bt.push_back(nleaf);
            for (size_t k = 0; k + 1 < bt.size(); ++k) need_bytes = std::max(need_bytes, bytes(bt[k], bt[k + 1]));
        };
        cut(batch_e, e_bytes);
        cut(batch_a, a_bytes);
        // M2L of the FP64-accurate form from slices as well, from 25
        // components on (below that the 32-wide tiles are mostly padding):
        // per level the distinct operators, each edge's operator within them,
        // and room for every (target, output chunk)'s stage list
        const int nq = (nc + SN - 1) / SN, ncs = (nc + SK - 1) / SK;
        const int nvar = lmax_policy != 0 ? L + 1 : 1;
        const int ntile = (int)((P + 127) / 128);
        const size_t nm2l = t->m2l_tgt.size();
        bool use_m2l = prec == OCCK_FP64 && ctx->slice_m2l != 0 && nc >= 25 && D >= 2 && nm2l > 0;
        std::vector<int> m_bop(nm2l, 0), m_opl, opmap(t->ops.size(), -1);
        std::vector<long long> m_sto;
        size_t max_opl = 0, max_st = 0, max_tq = 0, max_nb = 0;
        for (int lev = 2; use_m2l && lev <= D; ++lev) {
            const int t0 = t->level_off[lev], nt = t->level_off[lev + 1] - t0;
            m_lt0[lev] = t0;
            m_lnt[lev] = nt;
            m_lopl0[lev] = (int)m_opl.size();
            m_lst0[lev] = (long long)m_sto.size();
            long long st = 0;
            for (int tl = 0; tl < nt; ++tl) {
                const int ne = t->m2l_ptr[t0 + tl + 1] - t->m2l_ptr[t0 + tl];
                if ((long long)ne * ncs > occk::slice_max_stages()) use_m2l = false;   // exact int32 sums
                for (int qc = 0; qc < nq; ++qc) {
                    m_sto.push_back(st);
                    st += (long long)ne * ncs;
                }
                for (int e2 = t->m2l_ptr[t0 + tl]; e2 < t->m2l_ptr[t0 + tl + 1]; ++e2) {
                    const int op = t->m2l_op[e2];
                    if (opmap[op] < 0) {
                        opmap[op] = (int)m_opl.size() - m_lopl0[lev];
                        m_opl.push_back(op);
                    }
                    m_bop[e2] = opmap[op];
                }
            }
            m_lnopl[lev] = (int)m_opl.size() - m_lopl0[lev];
            for (int k = m_lopl0[lev]; k < (int)m_opl.size(); ++k) opmap[m_opl[k]] = -1;
            max_opl = std::max(max_opl, (size_t)m_lnopl[lev]);
            max_st = std::max(max_st, (size_t)st);
            max_tq = std::max(max_tq, (size_t)nt * nq);
            max_nb = std::max(max_nb, (size_t)nt);
        }
        size_t o_bop = plan_bytes, o_opl = o_bop, o_sto = o_bop;
        if (use_m2l) {
            o_opl = o_bop + al16(4 * nm2l);
            o_sto = o_opl + al16(4 * m_opl.size());
            plan_bytes = o_sto + al16(8 * m_sto.size());
            // workspace: operator panels, stage lists, exponents, then the
            // expansions' panels of as many pair tiles as the budget allows
            auto al1k = [](size_t x) { return (x + 1023) / 1024 * 1024; };
            const size_t w_b = al1k(pbb * max_opl * nvar * nq * ncs);
            const size_t w_st = al1k(8 * max_st), w_nk = al1k(4 * max_tq), w_ex = al1k(8 * (size_t)nc);
            const size_t w_gp = al1k(4 * P);
            const size_t fixed = w_b + w_st + w_nk + w_ex + w_gp;
            size_t wa = 0;
            for (int lev = 2; lev <= D; ++lev) {
                const size_t per_tile = pa * (size_t)m_lnt[lev] * ncs;
                const size_t room = budget > fixed + per_tile ? budget - fixed : per_tile;
                m_ltb[lev] = (int)std::max<size_t>(1, std::min<size_t>(ntile, room / std::max<size_t>(per_tile, 1)));
                wa = std::max(wa, per_tile * m_ltb[lev]);
            }
            need_bytes = std::max(need_bytes, fixed + wa);
            sm.S = nslices; sm.nq = nq; sm.ncs = ncs; sm.nvar = nvar; sm.ntile = ntile;
            sm.lt0 = m_lt0.data(); sm.lnt = m_lnt.data(); sm.lopl0 = m_lopl0.data(); sm.lnopl = m_lnopl.data();
            sm.lst0 = m_lst0.data(); sm.ltb = m_ltb.data();
            // device pointers are set once both buffers exist (below)
            sm.capB = (long long)(max_opl * nvar * nq * ncs);
            sm.capA = (long long)(wa / pa);
            sm.panB = nullptr;
            sm.stab = reinterpret_cast<int2*>(w_b);                  // offsets for now
            sm.nk = reinterpret_cast<int*>(w_b + w_st);
            sm.ec = reinterpret_cast<int*>(w_b + w_st + w_nk);
            sm.fq = reinterpret_cast<int*>(w_b + w_st + w_nk + 4 * (size_t)nc);
            sm.gp = reinterpret_cast<int*>(w_b + w_st + w_nk + w_ex);
            sm.panA = reinterpret_cast<uint8_t*>(fixed);
        }
        if ((e = ensure(ctx->splan, plan_bytes)) != cudaSuccess ||
            (e = ensure(ctx->spanels, need_bytes)) != cudaSuccess)
            return e == cudaErrorMemoryAllocation ? fail(ctx, OCCK_ERR_OOM, "slice panels of steps (a) and (e)")
                                                  : cuda_fail(ctx, e, "slice panels of steps (a) and (e)");
        std::vector<char> hp(plan_bytes, 0);
        std::memcpy(hp.data(), rtA.data(), 4 * (size_t)nleaf);
        std::memcpy(hp.data() + o_off, offA.data(), 8 * (size_t)nleaf);
        std::memcpy(hp.data() + o_item, item0.data(), 8 * (size_t)(nleaf + 1));
        std::memcpy(hp.data() + o_kca, kca.data(), 4 * (size_t)nleaf);
        std::memcpy(hp.data() + o_offAa, offAa.data(), 8 * (size_t)nleaf);
        std::memcpy(hp.data() + o_offBa, offBa.data(), 8 * (size_t)nleaf);
        std::memcpy(hp.data() + o_tp, tpair.data(), 4 * tpair.size());
        if ((e = cudaMemcpy(ctx->splan.p, hp.data(), o_eC, cudaMemcpyHostToDevice)) != cudaSuccess)
            return cuda_fail(ctx, e, "slice plan upload");
        char* x = (char*)ctx->splan.p;
        if (use_m2l) {
            if ((e = cudaMemcpy(x + o_bop, m_bop.data(), 4 * nm2l, cudaMemcpyHostToDevice)) != cudaSuccess ||
                (e = cudaMemcpy(x + o_opl, m_opl.data(), 4 * m_opl.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
                (e = cudaMemcpy(x + o_sto, m_sto.data(), 8 * m_sto.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
                return cuda_fail(ctx, e, "slice plan upload (M2L)");
            char* w0 = (char*)ctx->spanels.p;
            sm.edge_bop = (const int*)(x + o_bop);
            sm.oplist = (const int*)(x + o_opl);
            sm.stoff = (const long long*)(x + o_sto);
            sm.panB = (uint8_t*)w0;
            sm.stab = (int2*)(w0 + (size_t)sm.stab);
            sm.nk = (int*)(w0 + (size_t)sm.nk);
            sm.ec = (int*)(w0 + (size_t)sm.ec);
            sm.fq = (int*)(w0 + (size_t)sm.fq);
            sm.gp = (int*)(w0 + (size_t)sm.gp);
            sm.panA = (uint8_t*)(w0 + (size_t)sm.panA);
            sa.m2l = &sm;
        }
        // step (a) from slices while a leaf's K range fits the exact int32
        // group sums (about 4000 AO rows); the DFMA kernel otherwise
        sa.full = max_kca <= occk::slice_max_stages() ? 1 : 0;
        sa.max_kca = max_kca;
        sa.ntp = (int)tpair.size();
        sa.leaf_aos = t->dev.leaf_aos;
        sa.kca = (const int*)(x + o_kca);
        sa.offAa = (const long long*)(x + o_offAa);
        sa.offBa = (const long long*)(x + o_offBa);
        sa.tpair = (const int*)(x + o_tp);
        sa.eC = (int*)(x + o_eC);
        sa.eW = (int*)(x + o_eW);
        sa.ff = prec == OCCK_FP64 ? 1 : 0;   // the FP32 form keeps its FP32 SIMT passes
        sa.f32 = prec == OCCK_FP32 ? 1 : 0;
        sa.nops = (int)nops;
        sa.ops_ff = (float2*)(x + o_ff);
        sa.nvals = t->nvals;
        sa.vals_ff = (float2*)(x + o_vff);
        sa.C_ff = (float2*)(x + o_cff);
        sa.panAa = (uint8_t*)ctx->spanels.p;
        sa.nbatch_e = (int)batch_e.size() - 1;
        sa.nbatch_a = (int)batch_a.size() - 1;
        sa.batch_e = batch_e.data();
        sa.batch_a = batch_a.data();
        sa.offA_h = offA.data();
        sa.item0_h = item0.data();
        sa.offAa_h = offAa.data();
        sa.offBa_h = offBa.data();
        sa.S = nslices;
        sa.nocc = nocc; sa.nc = nc; sa.nrow = nrow; sa.nleaf = nleaf;
        sa.leaf_store0 = t->level_off[D] - first;
        sa.max_rt = max_rt; sa.nsplit = nsplit; sa.sm_count = std::max(ctx->sm_count, 1);
        sa.nitems = item0[nleaf];
        sa.leaf_rowoff = t->dev.leaf_rowoff;
        sa.lscale = t->dev.lscale;
        sa.rtA = (const int*)x;
        sa.offA = (const long long*)(x + o_off);
        sa.item0 = (const long long*)(x + o_item);
        sa.erow = (int*)(x + o_erow);
        sa.fcol = (int*)(x + o_fcol);
        sa.panA = (uint8_t*)ctx->spanels.p;
        l2p_nsplit = nsplit;
    }
    size_t bytes_kb = 8 * (size_t)nrow * nocc * l2p_nsplit;
    size_t bytes_part = 8 * (size_t)(4096 + 2);
    if ((e = ensure(ctx->ct, bytes_ct)) != cudaSuccess ||
        (e = ensure(ctx->w, bytes_w)) != cudaSuccess ||
        (e = ensure(ctx->obox, std::max<size_t>(bytes_box, 8))) != cudaSuccess ||
        (e = ensure(ctx->mbox, std::max<size_t>(bytes_box, 8))) != cudaSuccess ||
        (e = ensure(ctx->kb, bytes_kb)) != cudaSuccess ||
        (e = ensure(ctx->part, bytes_part)) != cudaSuccess ||
        (e = ensure(ctx->edev, 8)) != cudaSuccess ||
        (e = ensure(ctx->scratch, 256)) != cudaSuccess) {
        return e == cudaErrorMemoryAllocation ? fail(ctx, OCCK_ERR_OOM, "far-field workspaces")
                                              : cuda_fail(ctx, e, "workspace allocation");
    }
    occk::FmmArgs a{};
    a.nao = t->nao; a.nocc = nocc; a.ldc = ldc; a.ldk = ldk; a.nc = nc; a.L = L; a.depth = D;
    a.nbox = nbox; a.first_box = first; a.nleaf = nleaf; a.leaf0 = t->level_off[D]; a.nrow = nrow;
    a.level_off = t->level_off.data();
    a.prec = prec; a.C = C_dev; a.K = K_dev;
    a.Ex_dev = Ex_dev ? Ex_dev : (double*)ctx->edev.p;
    auto& d = t->dev;
    a.row_ptr = d.row_ptr; a.ent_col = d.ent_col; a.ent_val = d.ent_val;
    a.leaf_rowoff = d.leaf_rowoff; a.leaf_aos = d.leaf_aos;
    a.ao_row_ptr = d.ao_row_ptr; a.ao_rows = d.ao_rows;
    a.child_ptr = d.child_ptr; a.child_list = d.child_list; a.m2m_op = d.m2m_op; a.l2l_op = d.l2l_op;
    a.parent = d.parent;
    a.m2l_ptr = d.m2l_ptr; a.m2l_src = d.m2l_src; a.m2l_op = d.m2l_op;
    a.m2l_lmax = (lmax_policy == 1 && d.m2l_lmax_edge) ? d.m2l_lmax_edge : nullptr;
    a.pair_vals = prec == OCCK_FP64 ? (const void*)d.pair_vals : (const void*)d.pair_vals_f;
    a.ops = prec == OCCK_FP64 ? (const void*)d.ops : (const void*)d.ops_f;
    a.ct = ctx->ct.p; a.w = ctx->w.p; a.obox = ctx->obox.p; a.mbox = ctx->mbox.p;
    a.kb = (double*)ctx->kb.p; a.part = (double*)ctx->part.p;
    a.leaf_rowoff_host = t->leaf_rowoff.data();
    a.max_rows = max_rows;
    a.l2p_nsplit = l2p_nsplit;
    if (sliced) {
        sa.W = ctx->w.p;
        sa.Mbox = ctx->mbox.p;
        sa.KB = (double*)ctx->kb.p;
        a.slices = &sa;
    }
    ctx->last_sliced = sliced ? 1 : 0;
    a.learned = 0;
    ctx->ranks_valid = 0;
    const int nm2l = (int)t->m2l_tgt.size();
    if (lmax_policy == 2 && ctx->mlp_ready && L >= 2 && nm2l > 0) {
        if ((e = ensure(ctx->feat, sizeof(float) * (size_t)nm2l * OCCK_MLP_NIN)) != cudaSuccess ||
            (e = ensure(ctx->pred, sizeof(float) * (size_t)nm2l * OCCK_MLP_NOUT)) != cudaSuccess ||
            (e = ensure(ctx->ranks, sizeof(int) * (size_t)nm2l)) != cudaSuccess ||
            (e = ensure(ctx->nrm, sizeof(double) * (size_t)nbox * (L + 1))) != cudaSuccess ||
            (e = ensure(ctx->rank_err, sizeof(double) * (size_t)nm2l * (L + 1))) != cudaSuccess)
            return cuda_fail(ctx, e, "selector workspace");
        a.learned = 1;
        a.mlp_prm = (const float*)ctx->mlp_prm.p;
        a.mlp_h = ctx->mlp_h.p;
        a.mlp_norm = (const float*)ctx->mlp_norm.p;
        a.feat = (float*)ctx->feat.p;
        a.pred = (float*)ctx->pred.p;
        a.ranks = (int*)ctx->ranks.p;
        a.nrm = (double*)ctx->nrm.p;
        a.rank_err = (double*)ctx->rank_err.p;
        a.tau = ctx->tau;
        a.nm2l = nm2l;
        a.m2l_tgt = d.m2l_tgt;
        a.box_key = d.box_key;
        a.box_level = d.box_level;
        a.hlev = d.hlev;
        ctx->ranks_valid = 1;
    }
    // occupied-pair screening: every precision, with the tree passes on the
    // SIMT kernel over unscaled storage (the tensor-core translations are
    // turned off below); not with the learned selector, whose features read
    // every box
    a.screen = 0;
    a.col0 = a.col1 = 0;
    ctx->last_screen = 0;
    const bool colblk = ctx->col_i1 > 0;
    if (colblk) {
        if (ctx->col_i1 > nocc)
            return fail(ctx, OCCK_ERR_SHAPE, "column block [" + std::to_string(ctx->col_i0) + ", " +
                                                 std::to_string(ctx->col_i1) + ") beyond nocc " +
                                                 std::to_string(nocc));
        a.col0 = ctx->col_i0;
        a.col1 = ctx->col_i1;
    }
    if (ctx->screen_tau > 0 || colblk) {
        if (a.learned)
            return fail(ctx, OCCK_ERR_UNSUPPORTED,
                        "occupied-pair screening or a column block with the learned selector");
        // layout of scr_aux: norms (8P), keep (4P), inverse (4P), count (16),
        // block counts, step (e) tile flags, bound factors a2 and b2, step (a)
        // tile flags (64-pair tiles, the finer of the two SIMT tilings)
        const size_t o_bc = 16 * P + 16, n_bc = 4 * ((P + 255) / 256);
        const size_t o_tf = o_bc + n_bc + 16, n_tf = (size_t)((nocc + 127) / 128) * ((nocc + 7) / 8);
        const size_t o_ab = (o_tf + n_tf + 15) / 16 * 16, n_ab = 4 * (size_t)nleaf * nocc;
        const size_t nt64 = (size_t)(nocc + 63) / 64;
        const size_t o_ts = o_ab + (1 + (size_t)nc) * n_ab, n_ts = nt64 * (nt64 + 1) / 2;
        const size_t scr_bytes = o_ts + n_ts + 16;
        if ((e = ensure(ctx->scr_o, std::max<size_t>(bytes_box, 8))) != cudaSuccess ||
            (e = ensure(ctx->scr_m, std::max<size_t>(bytes_box, 8))) != cudaSuccess ||
            (e = ensure(ctx->scr_aux, scr_bytes)) != cudaSuccess)
            return e == cudaErrorMemoryAllocation ? fail(ctx, OCCK_ERR_OOM, "pair screening workspaces")
                                                  : cuda_fail(ctx, e, "pair screening workspaces");
        char* x = (char*)ctx->scr_aux.p;
        a.screen = 1;
        a.screen_tau2 = ctx->screen_tau > 0 ? ctx->screen_tau * ctx->screen_tau : 0.0;
        a.scr_o = ctx->scr_o.p;
        a.scr_m = ctx->scr_m.p;
        a.scr_norm = (double*)x;
        a.scr_keep = (int*)(x + 8 * P);
        a.scr_inv = (int*)(x + 12 * P);
        a.scr_count = (int*)(x + 16 * P);
        a.scr_bcount = (int*)(x + o_bc);
        a.scr_tiles = (unsigned char*)(x + o_tf);
        a.scr_a2 = (float*)(x + o_ab);
        a.scr_b2 = (float*)(x + o_ab + n_ab);
        a.scr_tskip = (unsigned char*)(x + o_ts);
        ctx->last_screen = 1;
        ctx->last_screen_P = P;
        // step (a) tiles of the SIMT forms (FP64: 64 x 64, FP32: 128 x 128)
        // that the bound may skip; the tensor-core forms form every tile
        ctx->last_tskip_n = 0;
        ctx->last_tskip = a.scr_tskip;
        if (prec == OCCK_FP64 || prec == OCCK_FP32) {
            const size_t bm = prec == OCCK_FP64 ? occk::kFullTileFP64 : occk::full_tile_fp32(nocc);
            const size_t nt = (nocc + bm - 1) / bm;
            ctx->last_tskip_n = nt * (nt + 1) / 2;
        }
    }
    // panel plan of the tensor-core steps (a) and (e): panel counts per leaf
    if (occk::tc_mode(prec) >= 0) {
        const int esz = occk::panel_elem_bytes(prec), pbytes = occk::panel_bytes(prec);
        if (ctx->pp_tree != t || ctx->pp_nocc != nocc || ctx->pp_nc != nc || ctx->pp_esz != esz ||
            ctx->pp_pbytes != pbytes) {
            const int BK = 128 / esz;
            const int jc = (nocc + BK - 1) / BK, it = (nocc + 127) / 128, KC = nc * jc;
            std::vector<int> rtA(nleaf), kca(nleaf);
            std::vector<long long> offA(nleaf), offAa(nleaf), offBa(nleaf);
            long long cA = 0, cAa = 0, cBa = 0;
            int max_rt = 0, max_kca = 0;
            for (int B = 0; B < nleaf; ++B) {
                const int nr = t->leaf_rowoff[B + 1] - t->leaf_rowoff[B];
                rtA[B] = (nr + 127) / 128;
                kca[B] = (nr + BK - 1) / BK;
                offA[B] = cA;
                cA += (long long)rtA[B] * KC;
                offAa[B] = cAa;
                cAa += (long long)it * kca[B];
                offBa[B] = cBa;
                cBa += (long long)nc * it * kca[B];
                max_rt = std::max(max_rt, rtA[B]);
                max_kca = std::max(max_kca, kca[B]);
            }
            const size_t bytes = 8 * (size_t)nleaf * 5 + 256;
            if ((e = ensure(ctx->pplan, bytes)) != cudaSuccess) return cuda_fail(ctx, e, "panel plan");
            std::vector<char> hbuf(bytes);
            char* hp = hbuf.data();
            std::memcpy(hp, offA.data(), 8 * nleaf);
            std::memcpy(hp + 8 * nleaf, offAa.data(), 8 * nleaf);
            std::memcpy(hp + 16 * nleaf, offBa.data(), 8 * nleaf);
            std::memcpy(hp + 24 * nleaf, rtA.data(), 4 * nleaf);
            std::memcpy(hp + 28 * nleaf, kca.data(), 4 * nleaf);
            if ((e = cudaMemcpy(ctx->pplan.p, hp, bytes, cudaMemcpyHostToDevice)) != cudaSuccess)
                return cuda_fail(ctx, e, "panel plan upload");
            const size_t l2p = (size_t)(cA + (long long)nleaf * it * KC), a2 = (size_t)(cAa + cBa);
            if ((e = ensure(ctx->panels, (size_t)pbytes * std::max(l2p, a2) + 1024)) != cudaSuccess)
                return e == cudaErrorMemoryAllocation ? fail(ctx, OCCK_ERR_OOM, "tensor-core panels")
                                                      : cuda_fail(ctx, e, "panels");
            ctx->pp_tree = t;
            ctx->pp_nocc = nocc;
            ctx->pp_nc = nc;
            ctx->pp_esz = esz;
            ctx->pp_pbytes = pbytes;
            ctx->pp_KC = KC;
            ctx->pp_jc = jc;
            ctx->pp_it = it;
            ctx->pp_max_rt = max_rt;
            ctx->pp_max_kca = max_kca;
            ctx->pp_l2pA = (size_t)cA;
            ctx->pp_a2A = (size_t)cAa;
        }
        char* pb = (char*)ctx->pplan.p;
        a.pp_offA = (const long long*)pb;
        a.pp_offAa = (const long long*)(pb + 8 * (size_t)nleaf);
        a.pp_offBa = (const long long*)(pb + 16 * (size_t)nleaf);
        a.pp_rtA = (const int*)(pb + 24 * (size_t)nleaf);
        a.pp_kca = (const int*)(pb + 28 * (size_t)nleaf);
        a.pp_KC = ctx->pp_KC;
        a.pp_jc = ctx->pp_jc;
        a.pp_it = ctx->pp_it;
        a.pp_max_rt = ctx->pp_max_rt;
        a.pp_max_kca = ctx->pp_max_kca;
        uint8_t* base = (uint8_t*)ctx->panels.p;
        a.pan_l2pA = base;
        a.pan_l2pB = base + (size_t)ctx->pp_pbytes * ctx->pp_l2pA;
        a.pan_a2A = base;
        a.pan_a2B = base + (size_t)ctx->pp_pbytes * ctx->pp_a2A;
    }
    // operator panels of the tensor-core translations (b)-(d), once per
    // operator set and precision
    a.tr_pan = nullptr;
    a.tr_on = 0;
    a.tr_nlev = D + 1;
    a.inv_h_leaf = (float)(1.0 / t->h[D]);
    a.sm_count = ctx->sm_count;
    a.box_level = d.box_level;
    if (occk::tc_mode(prec) >= 0 && occk::tr_np(nc) > 0 && D >= 2 && !t->ops.empty()) {
        if (ctx->tp_gen != t->gen || ctx->tp_prec != prec) {
            ctx->tp_ok = 0;
            const int nops = (int)t->ops.size(), nlev = D + 1;
            std::vector<int> lev(nbox), opinfo(4 * (size_t)nops, 0), seen(nops, 0);
            for (int l = 0; l <= D; ++l)
                for (int b = t->level_off[l]; b < t->level_off[l + 1]; ++b) lev[b] = l;
            bool consistent = true;
            auto setop = [&](int o, int kin, int lin, int kout, int lout) {
                if (o < 0 || o >= nops) return;
                int* r = &opinfo[4 * (size_t)o];
                if (!seen[o]) {
                    seen[o] = 1;
                    r[0] = kin; r[1] = lin; r[2] = kout; r[3] = lout;
                } else if (r[0] != kin || r[1] != lin || r[2] != kout || r[3] != lout) {
                    consistent = false;
                }
            };
            for (int b = 0; b < nbox; ++b) {
                if (lev[b] < 1) continue;
                setop(t->m2m_op[b], 0, lev[b], 0, lev[b] - 1);
                setop(t->l2l_op[b], 1, lev[b] - 1, 1, lev[b]);
            }
            for (size_t q = 0; q < t->m2l_tgt.size(); ++q) {
                const int l = lev[t->m2l_tgt[q]];
                setop(t->m2l_op[q], 0, l, 1, l);
            }
            // component scales: multipoles sqrt((l+m)!(l-m)!) / h^l, local
            // expansions h^(l+1) / sqrt((l+m)!(l-m)!)
            std::vector<double> scd(2 * (size_t)nlev * nc);
            for (int l = 0; l <= L; ++l) {
                for (int c = l * l; c < (l + 1) * (l + 1); ++c) {
                    const int m = c == l * l ? 0 : (c - l * l + 1) / 2;
                    const double g = std::sqrt(std::tgamma(l + m + 1.0) * std::tgamma(l - m + 1.0));
                    for (int k = 0; k < nlev; ++k) {
                        const double h = t->h[k];
                        scd[(size_t)k * nc + c] = g / std::pow(h, l);
                        scd[((size_t)nlev + k) * nc + c] = std::pow(h, l + 1) / g;
                    }
                }
            }
            const size_t nsc = scd.size();
            const size_t bytes_tab = 8 * nsc + 4 * opinfo.size() + 64;
            if ((e = ensure(ctx->tscale, bytes_tab)) != cudaSuccess ||
                (e = ensure(ctx->tpan, (size_t)nops * occk::tr_panel_bytes(prec, nc))) != cudaSuccess ||
                (e = ensure(ctx->tops, sizeof(float) * (size_t)nops * nc * nc)) != cudaSuccess)
                return e == cudaErrorMemoryAllocation ? fail(ctx, OCCK_ERR_OOM, "translation panels")
                                                      : cuda_fail(ctx, e, "translation panels");
            char* tb = (char*)ctx->tscale.p;
            if ((e = cudaMemcpy(tb, scd.data(), 8 * nsc, cudaMemcpyHostToDevice)) != cudaSuccess ||
                (e = cudaMemcpy(tb + 8 * nsc, opinfo.data(), 4 * opinfo.size(), cudaMemcpyHostToDevice)) !=
                    cudaSuccess)
                return cuda_fail(ctx, e, "translation scales upload");
            ctx->tp_scd = scd;
            e = occk::tr_build_panels(prec, d.ops, nops, nc, (const int*)(tb + 8 * nsc), (const double*)tb, nlev,
                                      (uint8_t*)ctx->tpan.p, (float*)ctx->tops.p, s);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "translation panels launch");
            ctx->tp_ok = consistent ? 1 : 0;
            ctx->tp_gen = t->gen;
            ctx->tp_prec = prec;
        }
        if (ctx->tp_ok) a.tr_pan = (const uint8_t*)ctx->tpan.p;
    }
    // the tensor-core translations keep a target's edge table in shared
    // memory (at most 256 edges; an interaction list has at most 189); they
    // run when every M2L edge has the full rank (per-edge ranks keep all
    // three translations on SIMT, with unscaled storage)
    int max_m2l_edges = 0;
    for (int b = 0; b + 1 < (int)t->m2l_ptr.size(); ++b)
        max_m2l_edges = std::max(max_m2l_edges, t->m2l_ptr[b + 1] - t->m2l_ptr[b]);
    a.tr_on = (a.tr_pan && a.m2l_lmax == nullptr && !a.learned && !a.screen && max_m2l_edges <= 256) ? 1 : 0;
    // which translations go to the tensor core, measured on GB300 (C150H302 at
    // ranks 2, 6, 8 and (H2O)100 at rank 4): from rank 4 on the slot pipeline
    // (all three translations on the tensor core, operands kept in its layout)
    // is fastest -- whole FP16X3 build 1.5x (rank 4), 2.0x (6), 3.1x (8)
    // faster than SIMT; at rank 2 the SIMT forms win.  The split forms are
    // chosen for accuracy: their tensor-core M2L carries every operand in 22
    // bits, which on (H2O)100 at rank 4 gives 1.6e-6 Eh against 7.2e-7 Eh with
    // the FP32 SIMT translations, so they take the slot pipeline from rank 6 on
    // (8.3e-7 Eh on C150H302 at rank 6).  SIMT keeps the storage unscaled.
    const bool split_form = prec == OCCK_BF16X3 || prec == OCCK_FP16X3;
    a.tr_mask = ctx->tr_engine >= 0 ? ctx->tr_engine : (L >= (split_form ? 6 : 4) ? 15 : 0);
    if (!a.tr_mask) a.tr_on = 0;
    a.ops_scaled = (const float*)ctx->tops.p;
    // sibling-grouped M2L for the FP32 SIMT translations: a level is grouped
    // when its children share enough of their interaction lists (M2L edges
    // per distinct source >= 2, e.g. 3-D clusters; chains share few), or
    // always / never as occk_set_m2l_group asks
    a.grp_use = 0;
    a.grp_level_off = t->grp_level_off.data();
    a.grp_child = d.grp_child; a.grp_parent = d.grp_parent; a.grp_ptr = d.grp_ptr;
    a.grp_src = d.grp_src; a.grp_op = d.grp_op;
    // measured on GB300 (protein-sized cluster, (H2O)100): grouped M2L at
    // rank 2 1.36-1.42x faster than per target; at rank 3 (16 components,
    // half the pairs per block) slower, so the default groups rank <= 2 only
    if (prec != OCCK_FP64 && (nc == 4 || nc == 9 || nc == 16) && d.grp_parent && ctx->m2l_group != 0) {
        for (int lev = 2; lev <= D && lev < 32; ++lev)
            if (ctx->m2l_group == 1 || (nc <= 9 && t->grp_gain[lev] >= 2.0)) a.grp_use |= 1u << lev;
    }
    // slot pipeline (mask 15): O~ and Mcal~ of every stored box in the tensor
    // core's operand layout between the steps
    a.slot_o = a.slot_m = nullptr;
    if (a.tr_on && a.tr_mask == 15) {
        const int ntile = (int)((P + 127) / 128);
        const size_t sbytes = (size_t)(nbox - first) * occk::tr_slot_box_bytes(prec, nc, ntile);
        if ((e = ensure(ctx->sob, sbytes)) != cudaSuccess || (e = ensure(ctx->smb, sbytes)) != cudaSuccess)
            return e == cudaErrorMemoryAllocation ? fail(ctx, OCCK_ERR_OOM, "slot storage")
                                                  : cuda_fail(ctx, e, "slot storage");
        a.slot_o = (uint8_t*)ctx->sob.p;
        a.slot_m = (uint8_t*)ctx->smb.p;
    }
    a.lscale = d.lscale;
    a.box_scale = d.box_scale;
    a.err_word = (int*)ctx->scratch.p;
    sa.err = a.err_word;
    e = cudaMemsetAsync(a.err_word, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "error word");
    a.ev = nullptr;
    if (ctx->timing) {
        for (int k = 0; k <= OCCK_NSTAGE; ++k)
            if (!ctx->ev[k]) cudaEventCreate(&ctx->ev[k]);
        a.ev = ctx->ev;
    }
    e = occk::run_farfield(a, s);
    ctx->ev_recorded = ctx->timing ? 1 : 0;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "occk_farfield_K launch");
    ctx->last_prec = prec;
    ctx->last_scaled = a.tr_on;
    ctx->last_slot = a.slot_o != nullptr;
    ctx->last_nocc = nocc;
    ctx->last_lmax = L;
    ctx->last_first_box = first;
    ctx->last_tree = t;
    if (Ex_host) {
        int werr = 0;
        e = cudaMemcpyAsync(Ex_host, a.Ex_dev, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&werr, a.err_word, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "energy copy");
        if (werr) return fail(ctx, OCCK_ERR_TIMEOUT, "a tensor-core wait gave up; results are invalid");
    }
    return OCCK_OK;
}

extern "C" occk_status occk_set_pair_screen(occk_ctx* ctx, double tau) {
    if (!ctx) return OCCK_ERR_ARG;
    if (!(tau >= 0.0) || std::isinf(tau)) return fail(ctx, OCCK_ERR_ARG, "tau must be finite and >= 0");
    ctx->screen_tau = tau;
    return OCCK_OK;
}

extern "C" occk_status occk_set_column_block(occk_ctx* ctx, int i0, int i1) {
    if (!ctx) return OCCK_ERR_ARG;
    if (i0 == 0 && i1 == 0) {
        ctx->col_i0 = ctx->col_i1 = 0;
        return OCCK_OK;
    }
    if (i0 < 0 || i1 <= i0) return fail(ctx, OCCK_ERR_ARG, "column block needs 0 <= i0 < i1 (or 0, 0 for off)");
    ctx->col_i0 = i0;
    ctx->col_i1 = i1;
    return OCCK_OK;
}

extern "C" occk_status occk_exchange_energy(occk_ctx* ctx, int nao, int nocc, const double* C_dev, int ldc,
                                            const double* K_dev, int ldk, double* E_dev, void* stream) {
    if (!ctx) return OCCK_ERR_ARG;
    if (ctx->device < 0) return fail(ctx, OCCK_ERR_UNSUPPORTED, "no device bound to this context");
    if (!C_dev || !K_dev || !E_dev || nao <= 0 || nocc <= 0)
        return fail(ctx, OCCK_ERR_ARG, "null buffer or non-positive size");
    if (ldc < nao || ldk < nao) return fail(ctx, OCCK_ERR_SHAPE, "ldc/ldk < nao");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = ensure(ctx->part, 8 * (size_t)(4096 + 2));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "occk_exchange_energy workspace");
    e = occk::energy_from_K(nao, nocc, C_dev, ldc, K_dev, ldk, (double*)ctx->part.p, E_dev, (cudaStream_t)stream);
    return e == cudaSuccess ? OCCK_OK : cuda_fail(ctx, e, "occk_exchange_energy launch");
}

extern "C" occk_status occk_pair_screen_count(occk_ctx* ctx, long long* kept, void* stream) {
    if (!ctx || !kept) return fail(ctx, OCCK_ERR_ARG, "null argument");
    *kept = -1;
    if (!ctx->last_screen || !ctx->scr_aux.p) return OCCK_OK;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    // the count sits after the norms and the two maps (16 bytes per pair)
    const size_t P = ctx->last_screen_P;
    int n = 0;
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemcpyAsync(&n, (const char*)ctx->scr_aux.p + 16 * P, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pair screening count");
    *kept = n;
    return OCCK_OK;
}

extern "C" occk_status occk_farfield_J(occk_ctx* ctx, const occk_tree* tc, const double* D_dev, int ldd,
                                       double* J_dev, int ldj, double* Ej_dev, double* Ej_host, void* stream) {
    if (!ctx || !tc) return fail(ctx, OCCK_ERR_ARG, "null argument");
    occk_tree* t = const_cast<occk_tree*>(tc);
    if (ctx->device < 0 || t->device != ctx->device)
        return fail(ctx, OCCK_ERR_UNSUPPORTED, "no device bound to this context or tree");
    if (t->lmax < 0) return fail(ctx, OCCK_ERR_STATE, "call occk_pair_multipoles first");
    if (!D_dev || !J_dev) return fail(ctx, OCCK_ERR_ARG, "null D or J");
    if (ldd < t->nao || ldj < t->nao) return fail(ctx, OCCK_ERR_SHAPE, "ldd/ldj < nao");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    const int L = t->lmax, nc = occk::ncomp(L), D = t->depth;
    const int nbox = (int)t->parent.size();
    const int first = D >= 2 ? t->level_off[2] : nbox;
    const int nleaf = (int)t->leaf_rowoff.size() - 1;
    const size_t nstore = (size_t)(nbox - first);
    if ((e = ensure(ctx->jbox, 8 * (2 * nstore * nc + nleaf + 1) + 64)) != cudaSuccess ||
        (e = ensure(ctx->edev, 8)) != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? fail(ctx, OCCK_ERR_OOM, "far-field J workspaces")
                                              : cuda_fail(ctx, e, "far-field J workspaces");
    auto& d = t->dev;
    occk::JArgs a{};
    a.nao = t->nao; a.nc = nc; a.L = L; a.depth = D; a.nbox = nbox; a.first_box = first; a.nleaf = nleaf;
    a.leaf0 = t->level_off[D];
    a.level_off = t->level_off.data();
    a.leaf_rowoff = d.leaf_rowoff; a.leaf_aos = d.leaf_aos; a.row_ptr = d.row_ptr; a.ent_col = d.ent_col;
    a.ent_val = d.ent_val;
    a.child_ptr = d.child_ptr; a.child_list = d.child_list; a.m2m_op = d.m2m_op; a.l2l_op = d.l2l_op;
    a.parent = d.parent; a.m2l_ptr = d.m2l_ptr; a.m2l_src = d.m2l_src; a.m2l_op = d.m2l_op;
    a.vals = d.pair_vals; a.ops = d.ops;
    a.D = D_dev; a.ldd = ldd; a.J = J_dev; a.ldj = ldj;
    a.Ej_dev = Ej_dev ? Ej_dev : (double*)ctx->edev.p;
    double* jb = (double*)ctx->jbox.p;
    a.ob = jb;
    a.mb = jb + nstore * nc;
    a.part = jb + 2 * nstore * nc;
    e = occk::run_farfield_J(a, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "occk_farfield_J launch");
    if (Ej_host) {
        e = cudaMemcpyAsync(Ej_host, a.Ej_dev, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "energy copy");
    }
    return OCCK_OK;
}

extern "C" occk_status occk_debug_fetch(occk_ctx* ctx, const occk_tree* t, int what, void* out,
                                        size_t bytes, void* stream) {
    if (!ctx || !t || !out) return fail(ctx, OCCK_ERR_ARG, "null argument");
    if (ctx->device < 0) return fail(ctx, OCCK_ERR_UNSUPPORTED, "no device");
    cudaStream_t s = (cudaStream_t)stream;
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sync");
    if (what == OCCK_DBG_PAIR_MULT) {
        if (t->lmax < 0) return fail(ctx, OCCK_ERR_STATE, "no multipoles");
        size_t n = (size_t)t->nvals * occk::ncomp(t->lmax);
        if (bytes != n * 8) return fail(ctx, OCCK_ERR_SHAPE, "size mismatch");
        e = cudaMemcpy(out, t->dev.pair_vals, bytes, cudaMemcpyDeviceToHost);
        return e == cudaSuccess ? OCCK_OK : cuda_fail(ctx, e, "copy");
    }
    if (what == OCCK_DBG_SCREEN_TILES) {
        if (bytes != 2 * sizeof(int)) return fail(ctx, OCCK_ERR_SHAPE, "size mismatch (2 ints)");
        if (!ctx->last_screen) return fail(ctx, OCCK_ERR_STATE, "the last occk_farfield_K did not screen");
        std::vector<unsigned char> f(ctx->last_tskip_n);
        if (!f.empty()) {
            e = cudaMemcpy(f.data(), ctx->last_tskip, f.size(), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "copy");
        }
        int* o = (int*)out;
        o[0] = (int)std::count_if(f.begin(), f.end(), [](unsigned char v) { return v != 0; });
        o[1] = (int)f.size();
        return OCCK_OK;
    }
    if (what != OCCK_DBG_OBOX && what != OCCK_DBG_MBOX) return fail(ctx, OCCK_ERR_ARG, "bad what");
    if (ctx->last_tree != t) return fail(ctx, OCCK_ERR_STATE, "last run used another tree");
    const int nbox = (int)t->parent.size();
    const int nc = occk::ncomp(ctx->last_lmax);
    const int no = ctx->last_nocc;
    const size_t P = (size_t)no * no;
    const size_t Ps = (size_t)no * (no + 1) / 2;
    const size_t n = (size_t)nbox * nc * P;
    if (bytes != n * 8) return fail(ctx, OCCK_ERR_SHAPE, "size mismatch");
    std::memset(out, 0, bytes);
    const size_t nst = (size_t)(nbox - ctx->last_first_box) * nc * Ps;
    const void* src = what == OCCK_DBG_OBOX ? ctx->obox.p : ctx->mbox.p;
    std::vector<double> tmp(nst);
    if (ctx->last_slot) {
        // slot pipeline: every stored box lives in the tensor core's layout;
        // decode it on the device into a temporary FP32 array
        float* dbuf = nullptr;
        e = cudaMalloc((void**)&dbuf, std::max<size_t>(nst, 1) * 4);
        const int ntile = (int)((Ps + 127) / 128);
        if (e == cudaSuccess)
            e = occk::tr_slots_unpack(ctx->last_prec, nc, (const uint8_t*)(what == OCCK_DBG_OBOX ? ctx->sob.p : ctx->smb.p),
                                      (int)Ps, ntile, 0, nbox - ctx->last_first_box, dbuf, s);
        std::vector<float> tf(nst);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaMemcpy(tf.data(), dbuf, nst * 4, cudaMemcpyDeviceToHost);
        if (dbuf) cudaFree(dbuf);
        for (size_t i = 0; i < nst; ++i) tmp[i] = tf[i];
    } else if (ctx->last_prec == OCCK_FP64) {
        e = cudaMemcpy(tmp.data(), src, nst * 8, cudaMemcpyDeviceToHost);
    } else {
        std::vector<float> tf(nst);
        e = cudaMemcpy(tf.data(), src, nst * 4, cudaMemcpyDeviceToHost);
        for (size_t i = 0; i < nst; ++i) tmp[i] = tf[i];
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy");
    // stored upper triangle -> full i,j square (scaled storage: back to O, Mcal)
    double* dst = (double*)out;
    const int nlev = t->depth + 1;
    const bool unscale = ctx->last_scaled && ctx->tp_scd.size() == 2 * (size_t)nlev * nc;
    for (int b = ctx->last_first_box; b < nbox; ++b)
        for (int c = 0; c < nc; ++c) {
            double* sp = tmp.data() + ((size_t)(b - ctx->last_first_box) * nc + c) * Ps;
            if (unscale) {
                int lev = 0;
                while (lev + 1 < nlev && t->level_off[lev + 1] <= b) ++lev;
                const int kind = what == OCCK_DBG_OBOX ? 0 : 1;
                const double f = 1.0 / ctx->tp_scd[((size_t)kind * nlev + lev) * nc + c];
                for (size_t q = 0; q < Ps; ++q) sp[q] *= f;
            }
            double* dp = dst + ((size_t)b * nc + c) * P;
            size_t q = 0;
            for (int i = 0; i < no; ++i)
                for (int j = i; j < no; ++j, ++q) {
                    dp[(size_t)i * no + j] = sp[q];
                    dp[(size_t)j * no + i] = sp[q];
                }
        }
    return OCCK_OK;
}

extern "C" occk_status occk_probe_fma_peak(occk_ctx* ctx, int prec, double* flops, void* stream) {
    if (!ctx || !flops) return fail(ctx, OCCK_ERR_ARG, "null argument");
    if (ctx->device < 0) return fail(ctx, OCCK_ERR_UNSUPPORTED, "no device");
    if (prec != OCCK_FP64 && prec != OCCK_FP32) return fail(ctx, OCCK_ERR_ARG, "prec");
    cudaSetDevice(ctx->device);
    cudaError_t e = occk::probe_fma(prec, ctx->sm_count, flops, (cudaStream_t)stream);
    return e == cudaSuccess ? OCCK_OK : cuda_fail(ctx, e, "probe");
}

extern "C" occk_status occk_set_timing(occk_ctx* ctx, int on) {
    if (!ctx) return OCCK_ERR_ARG;
    if (ctx->device < 0) return fail(ctx, OCCK_ERR_UNSUPPORTED, "no device");
    ctx->timing = on ? 1 : 0;
    return OCCK_OK;
}

extern "C" occk_status occk_get_timings(occk_ctx* ctx, float* ms, int n) {
    if (!ctx || !ms) return fail(ctx, OCCK_ERR_ARG, "null argument");
    if (n < OCCK_NSTAGE) return fail(ctx, OCCK_ERR_SHAPE, "n < OCCK_NSTAGE");
    if (!ctx->ev_recorded) return fail(ctx, OCCK_ERR_STATE, "no timed call recorded");
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaEventSynchronize(ctx->ev[OCCK_NSTAGE]);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "event sync");
    for (int k = 0; k < OCCK_NSTAGE; ++k) {
        e = cudaEventElapsedTime(&ms[k], ctx->ev[k], ctx->ev[k + 1]);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "elapsed");
    }
    return OCCK_OK;
}

extern "C" occk_status occk_device_status(occk_ctx* ctx, void* stream) {
    if (!ctx) return OCCK_ERR_ARG;
    if (ctx->device < 0 || !ctx->scratch.p) return OCCK_OK;
    cudaSetDevice(ctx->device);
    int werr = 0;
    cudaError_t e = cudaMemcpyAsync(&werr, ctx->scratch.p, sizeof(int), cudaMemcpyDeviceToHost,
                                    (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "occk_device_status");
    if (werr) return fail(ctx, OCCK_ERR_TIMEOUT, "a tensor-core wait gave up in the last call");
    return OCCK_OK;
}

extern "C" occk_status occk_debug_set_wait_limit(occk_ctx* ctx, long long polls) {
    if (!ctx) return OCCK_ERR_ARG;
    if (ctx->device < 0) return fail(ctx, OCCK_ERR_UNSUPPORTED, "no device bound to this context");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = occk::set_mma_wait_limit(polls);
    if (e == cudaSuccess) e = occk::set_slice_wait_limit(polls);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "occk_debug_set_wait_limit");
    return OCCK_OK;
}

extern "C" occk_status occk_set_m2l_group(occk_ctx* ctx, int mode) {
    if (!ctx) return OCCK_ERR_ARG;
    if (mode < -1 || mode > 1) return fail(ctx, OCCK_ERR_ARG, "m2l group mode must be -1, 0 or 1");
    ctx->m2l_group = mode;
    return OCCK_OK;
}

extern "C" occk_status occk_set_l2p_split(occk_ctx* ctx, int nsplit) {
    if (!ctx) return OCCK_ERR_ARG;
    if (nsplit < 0 || nsplit > 64) return fail(ctx, OCCK_ERR_ARG, "nsplit must be 0..64");
    ctx->l2p_split = nsplit;
    return OCCK_OK;
}

extern "C" occk_status occk_set_fp32_slices(occk_ctx* ctx, int slices) {
    if (!ctx) return OCCK_ERR_ARG;
    if (slices != 0 && slices != 4) return fail(ctx, OCCK_ERR_ARG, "slices must be 0 or 4");
    ctx->f32_slices = slices;
    if (slices == 0 && ctx->f64_slices == 0 && (ctx->spanels.p || ctx->splan.p)) {
        if (ctx->device >= 0) cudaSetDevice(ctx->device);
        cudaDeviceSynchronize();
        for (occk::DevBuf* b : {&ctx->spanels, &ctx->splan}) {
            if (b->p) cudaFree(b->p);
            b->p = nullptr;
            b->bytes = 0;
        }
    }
    return OCCK_OK;
}

extern "C" occk_status occk_set_fp64_slice_m2l(occk_ctx* ctx, int on) {
    if (!ctx) return OCCK_ERR_ARG;
    if (on != 0 && on != 1) return fail(ctx, OCCK_ERR_ARG, "on must be 0 or 1");
    ctx->slice_m2l = on;
    return OCCK_OK;
}

extern "C" occk_status occk_set_slice_workspace(occk_ctx* ctx, long long bytes) {
    if (!ctx) return OCCK_ERR_ARG;
    if (bytes < 0) return fail(ctx, OCCK_ERR_ARG, "bytes must be >= 0");
    ctx->slice_budget = (size_t)bytes;
    return OCCK_OK;
}

extern "C" occk_status occk_set_fp64_slices(occk_ctx* ctx, int slices) {
    if (!ctx) return OCCK_ERR_ARG;
    if (slices != 0 && slices != 6 && slices != 7) return fail(ctx, OCCK_ERR_ARG, "slices must be 0, 6 or 7");
    ctx->f64_slices = slices;
    if (slices == 0 && ctx->f32_slices == 0 && (ctx->spanels.p || ctx->splan.p)) {
        // the form is off: give its panels and plan back (a later call
        // allocates them again); wait for work in flight that may use them
        if (ctx->device >= 0) cudaSetDevice(ctx->device);
        cudaDeviceSynchronize();
        for (occk::DevBuf* b : {&ctx->spanels, &ctx->splan}) {
            if (b->p) cudaFree(b->p);
            b->p = nullptr;
            b->bytes = 0;
        }
    }
    return OCCK_OK;
}

extern "C" occk_status occk_set_translate_engine(occk_ctx* ctx, int mask) {
    if (!ctx) return OCCK_ERR_ARG;
    if (mask < -1 || (mask > 7 && mask != 15)) return fail(ctx, OCCK_ERR_ARG, "mask must be -1..7 or 15");
    ctx->tr_engine = mask;
    return OCCK_OK;
}

extern "C" occk_status occk_debug_tc_gemm(occk_ctx* ctx, int prec, int M, int N, int K, const float* A,
                                          const float* B, float* D, void* stream) {
    if (!ctx || !A || !B || !D) return fail(ctx, OCCK_ERR_ARG, "null argument");
    if (ctx->device < 0) return fail(ctx, OCCK_ERR_UNSUPPORTED, "no device");
    if (occk::tc_mode(prec) < 0) return fail(ctx, OCCK_ERR_ARG, "not a tensor-core precision");
    if (M <= 0 || N <= 0 || K <= 0) return fail(ctx, OCCK_ERR_ARG, "sizes must be positive");
    cudaSetDevice(ctx->device);
    cudaError_t e = ensure(ctx->scratch, 256);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "scratch");
    e = ensure(ctx->panels, occk::tc_gemm_panel_bytes(prec, M, N, K) + 1024);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "panels");
    ctx->pp_tree = nullptr;   // the panel buffer no longer holds a far-field plan's panels
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemsetAsync(ctx->scratch.p, 0, sizeof(int), s);
    if (e == cudaSuccess)
        e = occk::tc_gemm(prec, M, N, K, A, B, D, (uint8_t*)ctx->panels.p, (int*)ctx->scratch.p, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "occk_debug_tc_gemm");
    return occk_device_status(ctx, stream);
}

// ===========================================================================
// Learned rank selector
// ===========================================================================

namespace {

occk_status mlp_alloc(occk_ctx* ctx) {
    const size_t np = (size_t)OCCK_MLP_NPARAM;
    cudaError_t e;
    if ((e = ensure(ctx->mlp_prm, 4 * np)) != cudaSuccess || (e = ensure(ctx->mlp_m, 4 * np)) != cudaSuccess ||
        (e = ensure(ctx->mlp_v, 4 * np)) != cudaSuccess || (e = ensure(ctx->mlp_h, 2 * np)) != cudaSuccess ||
        (e = ensure(ctx->mlp_grad, 4 * np)) != cudaSuccess ||
        (e = ensure(ctx->mlp_norm, 4 * (size_t)OCCK_MLP_NNORM)) != cudaSuccess)
        return cuda_fail(ctx, e, "MLP storage");
    return OCCK_OK;
}

struct MlpWs {
    float *Xn, *Z1, *Z2, *Y, *dY, *dZ1, *dZ2;
    double* part;
};

occk_status mlp_workspace(occk_ctx* ctx, int n, MlpWs* w) {
    const size_t N = (size_t)n;
    const size_t nfl = N * (OCCK_MLP_NIN + 4 * OCCK_MLP_HIDDEN + 2 * OCCK_MLP_NOUT);
    cudaError_t e = ensure(ctx->mlp_ws, nfl * 4 + 8 * 256 + 256);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "MLP workspace");
    float* f = (float*)ctx->mlp_ws.p;
    w->Xn = f; f += N * OCCK_MLP_NIN;
    w->Z1 = f; f += N * OCCK_MLP_HIDDEN;
    w->Z2 = f; f += N * OCCK_MLP_HIDDEN;
    w->dZ1 = f; f += N * OCCK_MLP_HIDDEN;
    w->dZ2 = f; f += N * OCCK_MLP_HIDDEN;
    w->Y = f; f += N * OCCK_MLP_NOUT;
    w->dY = f; f += N * OCCK_MLP_NOUT;
    uintptr_t u = ((uintptr_t)f + 255) & ~(uintptr_t)255;
    w->part = (double*)u;
    return OCCK_OK;
}

double host_loss(const double* part, int n) {
    double s = 0;
    for (int i = 0; i < n; ++i) s += part[i];
    return s;
}

}  // namespace

extern "C" occk_status occk_mlp_init(occk_ctx* ctx, uint64_t seed) {
    if (!ctx) return OCCK_ERR_ARG;
    if (ctx->device < 0) return fail(ctx, OCCK_ERR_UNSUPPORTED, "no device");
    if (occk::mlp_nparams() != OCCK_MLP_NPARAM) return fail(ctx, OCCK_ERR_STATE, "MLP size mismatch");
    cudaSetDevice(ctx->device);
    occk_status st = mlp_alloc(ctx);
    if (st) return st;
    std::vector<float> p(OCCK_MLP_NPARAM, 0.f), nrm(OCCK_MLP_NNORM, 0.f);
    uint64_t x = seed ? seed : 0x9E3779B97F4A7C15ull;
    auto next = [&]() {   // splitmix64
        x += 0x9E3779B97F4A7C15ull;
        uint64_t z = x;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto fill = [&](int off, int fan_in, int count) {
        const double lim = std::sqrt(6.0 / fan_in);
        for (int k = 0; k < count; ++k) {
            double u = (double)(next() >> 11) / 9007199254740992.0;
            p[off + k] = (float)((2.0 * u - 1.0) * lim);
        }
    };
    const int NIN = OCCK_MLP_NIN, H = OCCK_MLP_HIDDEN, NO = OCCK_MLP_NOUT;
    fill(0, NIN, NIN * H);
    fill(NIN * H + H, H, H * H);
    fill(NIN * H + H + H * H + H, H, H * NO);
    for (int i = 0; i < NIN; ++i) nrm[NIN + i] = 1.f;
    for (int k = 0; k < NO; ++k) nrm[2 * NIN + NO + k] = 1.f;
    cudaError_t e = cudaMemcpy(ctx->mlp_prm.p, p.data(), 4 * p.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ctx->mlp_norm.p, nrm.data(), 4 * nrm.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(ctx->mlp_m.p, 0, 4 * (size_t)OCCK_MLP_NPARAM);
    if (e == cudaSuccess) e = cudaMemset(ctx->mlp_v.p, 0, 4 * (size_t)OCCK_MLP_NPARAM);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "occk_mlp_init");
    ctx->mlp_t = 0;
    ctx->mlp_ready = 0;
    return OCCK_OK;
}

extern "C" occk_status occk_mlp_set(occk_ctx* ctx, const float* params, const float* norm) {
    if (!ctx || !params || !norm) return fail(ctx, OCCK_ERR_ARG, "null argument");
    if (ctx->device < 0) return fail(ctx, OCCK_ERR_UNSUPPORTED, "no device");
    cudaSetDevice(ctx->device);
    occk_status st = mlp_alloc(ctx);
    if (st) return st;
    for (int k = 0; k < OCCK_MLP_NIN + OCCK_MLP_NOUT; ++k) {
        const float sd = k < OCCK_MLP_NIN ? norm[OCCK_MLP_NIN + k] : norm[2 * OCCK_MLP_NIN + OCCK_MLP_NOUT + k - OCCK_MLP_NIN];
        if (!(sd > 0.f)) return fail(ctx, OCCK_ERR_ARG, "normalisation standard deviations must be > 0");
    }
    cudaError_t e = cudaMemcpy(ctx->mlp_prm.p, params, 4 * (size_t)OCCK_MLP_NPARAM, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ctx->mlp_norm.p, norm, 4 * (size_t)OCCK_MLP_NNORM, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(ctx->mlp_m.p, 0, 4 * (size_t)OCCK_MLP_NPARAM);
    if (e == cudaSuccess) e = cudaMemset(ctx->mlp_v.p, 0, 4 * (size_t)OCCK_MLP_NPARAM);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "occk_mlp_set");
    ctx->mlp_t = 0;
    ctx->mlp_ready = 1;
    return OCCK_OK;
}

extern "C" occk_status occk_mlp_get(occk_ctx* ctx, float* params, float* norm) {
    if (!ctx || !params || !norm) return fail(ctx, OCCK_ERR_ARG, "null argument");
    if (!ctx->mlp_prm.p) return fail(ctx, OCCK_ERR_STATE, "no MLP on this context");
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaMemcpy(params, ctx->mlp_prm.p, 4 * (size_t)OCCK_MLP_NPARAM, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(norm, ctx->mlp_norm.p, 4 * (size_t)OCCK_MLP_NNORM, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? OCCK_OK : cuda_fail(ctx, e, "occk_mlp_get");
}

extern "C" occk_status occk_mlp_grad(occk_ctx* ctx, const float* X, const float* T, int n, float* grad,
                                     float* loss_host, void* stream) {
    if (!ctx || !X || !T || !grad || n <= 0) return fail(ctx, OCCK_ERR_ARG, "bad argument");
    if (!ctx->mlp_prm.p) return fail(ctx, OCCK_ERR_STATE, "call occk_mlp_init or occk_mlp_set first");
    cudaSetDevice(ctx->device);
    MlpWs w;
    occk_status st = mlp_workspace(ctx, n, &w);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const float* prm = (const float*)ctx->mlp_prm.p;
    cudaError_t e = occk::mlp_forward_train(prm, (const float*)ctx->mlp_norm.p, X, n, w.Xn, w.Z1, w.Z2, w.Y, s);
    if (e == cudaSuccess)
        e = occk::mlp_backward(prm, w.Xn, w.Z1, w.Z2, w.Y, T, n, w.dY, w.dZ1, w.dZ2, grad, w.part, 256, s);
    double part[256];
    if (e == cudaSuccess) e = cudaMemcpyAsync(part, w.part, sizeof(part), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "occk_mlp_grad");
    if (loss_host) *loss_host = (float)(host_loss(part, 256) / ((double)n * OCCK_MLP_NOUT));
    return OCCK_OK;
}

extern "C" occk_status occk_mlp_train(occk_ctx* ctx, const float* X, const float* T, int n, int steps, float lr,
                                      float* loss_host, void* stream) {
    if (!ctx || !X || !T || n <= 0 || steps < 0) return fail(ctx, OCCK_ERR_ARG, "bad argument");
    if (!ctx->mlp_prm.p) return fail(ctx, OCCK_ERR_STATE, "call occk_mlp_init or occk_mlp_set first");
    cudaSetDevice(ctx->device);
    MlpWs w;
    occk_status st = mlp_workspace(ctx, n, &w);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    float* prm = (float*)ctx->mlp_prm.p;
    float* g = (float*)ctx->mlp_grad.p;
    cudaError_t e = cudaSuccess;
    for (int it = 0; it < steps && e == cudaSuccess; ++it) {
        e = occk::mlp_forward_train(prm, (const float*)ctx->mlp_norm.p, X, n, w.Xn, w.Z1, w.Z2, w.Y, s);
        if (e == cudaSuccess)
            e = occk::mlp_backward(prm, w.Xn, w.Z1, w.Z2, w.Y, T, n, w.dY, w.dZ1, w.dZ2, g, w.part, 256, s);
        if (e == cudaSuccess)
            e = occk::mlp_adam(prm, g, (float*)ctx->mlp_m.p, (float*)ctx->mlp_v.p, ++ctx->mlp_t, lr, s);
    }
    double part[256];
    if (e == cudaSuccess) e = cudaMemcpyAsync(part, w.part, sizeof(part), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "occk_mlp_train");
    if (loss_host) *loss_host = (float)(host_loss(part, 256) / ((double)n * OCCK_MLP_NOUT));
    ctx->mlp_ready = 1;
    return OCCK_OK;
}

extern "C" occk_status occk_mlp_predict(occk_ctx* ctx, const float* X, int n, float* Y, void* stream) {
    if (!ctx || !X || !Y || n < 0) return fail(ctx, OCCK_ERR_ARG, "bad argument");
    if (!ctx->mlp_prm.p) return fail(ctx, OCCK_ERR_STATE, "no MLP on this context");
    cudaSetDevice(ctx->device);
    cudaError_t e = occk::mlp_predict_fp16((const float*)ctx->mlp_prm.p, (__half*)ctx->mlp_h.p,
                                           (const float*)ctx->mlp_norm.p, X, n, Y, (cudaStream_t)stream);
    return e == cudaSuccess ? OCCK_OK : cuda_fail(ctx, e, "occk_mlp_predict");
}

static occk_status last_run_check(occk_ctx* ctx, const occk_tree* t) {
    if (ctx->last_tree != t || ctx->last_lmax != t->lmax || !ctx->obox.p)
        return fail(ctx, OCCK_ERR_STATE, "needs a previous occk_farfield_K on this tree and rank");
    if (ctx->last_prec != OCCK_FP64 && ctx->last_prec != OCCK_FP32 && occk::tc_mode(ctx->last_prec) < 0)
        return fail(ctx, OCCK_ERR_STATE, "unknown precision of the last run");
    return OCCK_OK;
}

extern "C" occk_status occk_edge_features(occk_ctx* ctx, const occk_tree* t, float* F, void* stream) {
    if (!ctx || !t || !F) return fail(ctx, OCCK_ERR_ARG, "null argument");
    occk_status st = last_run_check(ctx, t);
    if (st) return st;
    cudaSetDevice(ctx->device);
    const int nbox = (int)t->parent.size(), L = t->lmax;
    cudaError_t e = ensure(ctx->nrm, sizeof(double) * (size_t)nbox * (L + 1));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "norm workspace");
    const long long P = (long long)ctx->last_nocc * (ctx->last_nocc + 1) / 2;
    e = occk::edge_features(ctx->last_prec == OCCK_FP64, ctx->obox.p, ctx->last_first_box, nbox,
                            occk::ncomp(L), L, P, ctx->last_nocc, (int)t->m2l_tgt.size(), t->dev.m2l_tgt, t->dev.m2l_src,
                            t->dev.box_key, t->dev.box_level, t->dev.hlev, t->depth, (double*)ctx->nrm.p, F,
                            (cudaStream_t)stream);
    return e == cudaSuccess ? OCCK_OK : cuda_fail(ctx, e, "occk_edge_features");
}

extern "C" occk_status occk_edge_energies(occk_ctx* ctx, const occk_tree* t, double* E, void* stream) {
    if (!ctx || !t || !E) return fail(ctx, OCCK_ERR_ARG, "null argument");
    occk_status st = last_run_check(ctx, t);
    if (st) return st;
    cudaSetDevice(ctx->device);
    const int L = t->lmax, nc = occk::ncomp(L), ne = (int)t->m2l_tgt.size();
    cudaError_t e = ensure(ctx->gram, sizeof(double) * (size_t)std::max(ne, 1) * nc * nc);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "Gram workspace");
    const long long P = (long long)ctx->last_nocc * (ctx->last_nocc + 1) / 2;
    e = occk::edge_energies(ctx->last_prec == OCCK_FP64, ctx->obox.p, ctx->last_first_box, nc, L, P,
                            ctx->last_nocc, ne,
                            t->dev.m2l_tgt, t->dev.m2l_src, t->dev.ops, t->dev.m2l_op, (double*)ctx->gram.p, E,
                            (cudaStream_t)stream);
    return e == cudaSuccess ? OCCK_OK : cuda_fail(ctx, e, "occk_edge_energies");
}

extern "C" occk_status occk_set_learned_tau(occk_ctx* ctx, double tau) {
    if (!ctx || !(tau > 0)) return fail(ctx, OCCK_ERR_ARG, "tau must be > 0");
    ctx->tau = tau;
    return OCCK_OK;
}

extern "C" occk_status occk_get_edge_ranks(occk_ctx* ctx, const occk_tree* t, int* ranks, int n) {
    if (!ctx || !t || !ranks) return fail(ctx, OCCK_ERR_ARG, "null argument");
    if (n != (int)t->m2l_tgt.size()) return fail(ctx, OCCK_ERR_SHAPE, "n != nm2l");
    if (!ctx->ranks_valid || ctx->last_tree != t) return fail(ctx, OCCK_ERR_STATE, "no learned run on this tree");
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaMemcpy(ranks, ctx->ranks.p, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? OCCK_OK : cuda_fail(ctx, e, "occk_get_edge_ranks");
}
