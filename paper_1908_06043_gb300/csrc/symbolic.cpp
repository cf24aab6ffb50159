// Symbolic analysis of the sparse LDL^T of A - sigma B (done once per pattern).
//
// The paper factors A - sigma B with a sparse direct solver whose ordering is nested
// dissection (Section 2.1 names the sparse LDL^T as the major cost; Section 5 runs it
// with a nested-dissection ordering).  This file computes, from the CSR pattern only:
//   1. a nested-dissection ordering from BFS level-structure vertex separators;
//   2. supernodes = the dissection blocks (leaves and separators), each a dense
//      diagonal block, with its off-diagonal row structure from the supernodal
//      symbolic factorisation (union of its columns' structure and its children's);
//   3. the assembly tree, its levels, the front arena layout (level-ordered), the
//      assembly map of every stored entry, child->parent extend-add maps;
//   4. the panel schedule of the blocked front factorisation and the level schedule
//      of the panel triangular solves; exact flop and storage counts.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
#include <numeric>

#include "internal.h"

namespace {

struct Graph {
    int64_t n;
    const int64_t *xadj;
    const int32_t *adj;
};

class Dissector {
  public:
    Dissector(const Graph &g, int leaf)
        : g_(g), leaf_(leaf), stamp_(g.n, 0), level_(g.n, -1) {}

    void run(std::vector<int32_t> &order, std::vector<int32_t> &first) {
        order_ = &order;
        first_ = &first;
        std::vector<int32_t> all(g_.n);
        std::iota(all.begin(), all.end(), 0);
        dissect(all);
        first.push_back((int32_t)order.size());
    }

  private:
    // BFS over vertices stamped `st`; fills q (visit order) and lstart (level starts).
    int bfs(int32_t root, int32_t st, std::vector<int32_t> &q, std::vector<int64_t> &lstart) {
        q.clear();
        lstart.clear();
        q.push_back(root);
        level_[root] = 0;
        size_t head = 0;
        int cur = -1;
        while (head < q.size()) {
            int32_t v = q[head];
            if (level_[v] != cur) {
                cur = level_[v];
                lstart.push_back((int64_t)head);
            }
            ++head;
            for (int64_t p = g_.xadj[v]; p < g_.xadj[v + 1]; ++p) {
                int32_t u = g_.adj[p];
                if (stamp_[u] == st && level_[u] < 0) {
                    level_[u] = cur + 1;
                    q.push_back(u);
                }
            }
        }
        lstart.push_back((int64_t)q.size());
        return cur + 1;
    }

    void reset_levels(const std::vector<int32_t> &v) {
        for (int32_t x : v) level_[x] = -1;
    }

    void emit(std::vector<int32_t> &verts) {
        std::sort(verts.begin(), verts.end());
        first_->push_back((int32_t)order_->size());
        order_->insert(order_->end(), verts.begin(), verts.end());
    }

    void dissect(std::vector<int32_t> &verts) {
        if ((int64_t)verts.size() <= leaf_) {
            emit(verts);
            return;
        }
        const int32_t st = ++cur_;
        for (int32_t v : verts) stamp_[v] = st;
        reset_levels(verts);
        std::vector<int32_t> q;
        std::vector<int64_t> ls;
        bfs(verts[0], st, q, ls);
        if (q.size() < verts.size()) {
            // several connected components: each is an independent subtree
            std::vector<std::vector<int32_t>> comps;
            comps.push_back(q);
            for (int32_t v : verts) {
                if (level_[v] < 0) {
                    bfs(v, st, q, ls);
                    comps.push_back(q);
                }
            }
            reset_levels(verts);
            for (auto &c : comps) dissect(c);
            return;
        }
        // pseudo-peripheral root: repeat BFS from a min-degree vertex of the last level
        int32_t root = verts[0];
        int h = (int)ls.size() - 1;
        for (int it = 0; it < 6; ++it) {
            int32_t best = -1;
            int64_t bdeg = INT64_MAX;
            for (int64_t p = ls[h - 1]; p < ls[h]; ++p) {
                int32_t v = q[p];
                int64_t d = g_.xadj[v + 1] - g_.xadj[v];
                if (d < bdeg) { bdeg = d; best = v; }
            }
            reset_levels(verts);
            std::vector<int32_t> q2;
            std::vector<int64_t> ls2;
            int h2 = bfs(best, st, q2, ls2);
            if (h2 > h) {
                root = best; h = h2; q.swap(q2); ls.swap(ls2);
            } else {
                reset_levels(verts);
                h = bfs(root, st, q, ls);
                break;
            }
        }
        const int64_t nv = (int64_t)verts.size();
        if (h < 3) {
            reset_levels(verts);
            emit(verts);
            return;
        }
        // choose the level l whose boundary part (vertices adjacent to level l+1) is the
        // smallest separator among balanced splits
        int best_l = -1;
        int64_t best_s = INT64_MAX, best_imb = INT64_MAX;
        int fallback_l = -1;
        int64_t fallback_imb = INT64_MAX;
        for (int l = 1; l <= h - 2; ++l) {
            int64_t s = 0;
            for (int64_t p = ls[l]; p < ls[l + 1]; ++p) {
                int32_t v = q[p];
                for (int64_t e = g_.xadj[v]; e < g_.xadj[v + 1]; ++e) {
                    int32_t u = g_.adj[e];
                    if (stamp_[u] == st && level_[u] == l + 1) { ++s; break; }
                }
            }
            int64_t p1 = ls[l + 1] - s;
            int64_t p2 = nv - ls[l + 1];
            int64_t imb = std::llabs(p1 - p2);
            if (imb < fallback_imb) { fallback_imb = imb; fallback_l = l; }
            if (std::min(p1, p2) * 4 >= (nv - s) && (s < best_s || (s == best_s && imb < best_imb))) {
                best_s = s; best_imb = imb; best_l = l;
            }
        }
        int l = best_l >= 0 ? best_l : fallback_l;
        std::vector<int32_t> P1, P2, S;
        for (int64_t p = 0; p < ls[l]; ++p) P1.push_back(q[p]);
        for (int64_t p = ls[l]; p < ls[l + 1]; ++p) {
            int32_t v = q[p];
            bool adj_next = false;
            for (int64_t e = g_.xadj[v]; e < g_.xadj[v + 1]; ++e) {
                int32_t u = g_.adj[e];
                if (stamp_[u] == st && level_[u] == l + 1) { adj_next = true; break; }
            }
            (adj_next ? S : P1).push_back(v);
        }
        for (int64_t p = ls[l + 1]; p < nv; ++p) P2.push_back(q[p]);
        reset_levels(verts);
        if (P1.empty() || P2.empty() || (int64_t)S.size() * 10 > nv * 6) {
            emit(verts);
            return;
        }
        std::vector<int32_t>().swap(verts);
        dissect(P1);
        dissect(P2);
        emit(S);
    }

    const Graph &g_;
    int leaf_;
    std::vector<int32_t> stamp_;
    int32_t cur_ = 0;
    std::vector<int32_t> level_;
    std::vector<int32_t> *order_ = nullptr;
    std::vector<int32_t> *first_ = nullptr;
};

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

static int analyze_impl(ss_ctx *ctx, int64_t n, const int64_t *rowptr, const int32_t *colind,
                        const ss_options *opt, ss_symbolic *s) {
    auto t0 = std::chrono::steady_clock::now();
    s->ctx = ctx;
    s->n = n;
    s->nnz = rowptr[n];
    int leaf = (opt && opt->nd_leaf > 0) ? opt->nd_leaf : 64;
    int nb = (opt && opt->panel > 0) ? opt->panel : 64;
    if (nb != 64) return ctx->set_error(SS_ERR_ARG, "panel width must be 64");
    s->nb = nb;
    // ---- validate the pattern: sorted in-range columns, diagonal present, symmetric
    if (rowptr[0] != 0) return ctx->set_error(SS_ERR_ARG, "rowptr[0] != 0");
    for (int64_t i = 0; i < n; ++i)
        if (rowptr[i + 1] < rowptr[i]) return ctx->set_error(SS_ERR_ARG, "rowptr not monotone");
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(| : bad)
    for (int64_t i = 0; i < n; ++i) {
        bool diag = false;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int32_t j = colind[p];
            if (j < 0 || j >= n) { bad |= 1; break; }
            if (p > rowptr[i] && colind[p - 1] >= j) { bad |= 2; break; }
            if (j == i) diag = true;
            const int32_t *b = colind + rowptr[j], *e = colind + rowptr[j + 1];
            const int32_t *f = std::lower_bound(b, e, (int32_t)i);
            if (f == e || *f != i) { bad |= 4; break; }
        }
        if (!diag) bad |= 8;
    }
    if (bad & 1) return ctx->set_error(SS_ERR_ARG, "column index out of range");
    if (bad & 2) return ctx->set_error(SS_ERR_ARG, "column indices not strictly increasing in a row");
    if (bad & 4) return ctx->set_error(SS_ERR_ARG, "pattern is not symmetric");
    if (bad & 8) return ctx->set_error(SS_ERR_ARG, "a diagonal entry is missing from the pattern");
    s->rowptr.assign(rowptr, rowptr + n + 1);
    s->colind.assign(colind, colind + s->nnz);

    // ---- 1. nested dissection
    Graph g{n, s->rowptr.data(), s->colind.data()};
    std::vector<int32_t> order, first;
    order.reserve(n);
    Dissector(g, leaf).run(order, first);
    s->perm = order;
    s->iperm.assign(n, 0);
    for (int64_t i = 0; i < n; ++i) s->iperm[order[i]] = (int32_t)i;
    const int32_t nsn = (int32_t)first.size() - 1;
    s->nsn = nsn;
    s->sn_first = first;
    std::vector<int32_t> blockof(n);
    for (int32_t b = 0; b < nsn; ++b)
        for (int32_t j = first[b]; j < first[b + 1]; ++j) blockof[j] = b;

    // ---- 2. supernodal row structures, parents and levels
    s->sn_parent.assign(nsn, -1);
    s->sn_nrow.assign(nsn, 0);
    s->sn_level.assign(nsn, 0);
    s->sn_idx_off.assign(nsn + 1, 0);
    std::vector<std::vector<int32_t>> children(nsn);
    std::vector<int32_t> mark(n, -1);
    std::vector<int32_t> &idx = s->idx;
    idx.clear();
    std::vector<int32_t> rows;
    for (int32_t b = 0; b < nsn; ++b) {
        const int32_t f0 = first[b], last = first[b + 1] - 1;
        rows.clear();
        for (int32_t j = f0; j <= last; ++j) {
            int32_t old = s->perm[j];
            for (int64_t p = s->rowptr[old]; p < s->rowptr[old + 1]; ++p) {
                int32_t i = s->iperm[s->colind[p]];
                if (i > last && mark[i] != b) { mark[i] = b; rows.push_back(i); }
            }
        }
        int lev = 0;
        for (int32_t c : children[b]) {
            lev = std::max(lev, s->sn_level[c] + 1);
            const int64_t o = s->sn_idx_off[c] + (first[c + 1] - first[c]);
            for (int32_t r = 0; r < s->sn_nrow[c]; ++r) {
                int32_t i = idx[o + r];
                if (i > last && mark[i] != b) { mark[i] = b; rows.push_back(i); }
            }
        }
        std::sort(rows.begin(), rows.end());
        s->sn_level[b] = lev;
        s->sn_nrow[b] = (int32_t)rows.size();
        s->sn_idx_off[b] = (int64_t)idx.size();
        for (int32_t j = f0; j <= last; ++j) idx.push_back(j);
        idx.insert(idx.end(), rows.begin(), rows.end());
        if (!rows.empty()) {
            int32_t p = blockof[rows[0]];
            s->sn_parent[b] = p;
            children[p].push_back(b);
        }
    }
    s->sn_idx_off[nsn] = (int64_t)idx.size();
    int32_t nlev = 0;
    for (int32_t b = 0; b < nsn; ++b) nlev = std::max(nlev, s->sn_level[b] + 1);
    s->nlev = nlev;

    auto ncol = [&](int32_t b) { return first[b + 1] - first[b]; };
    auto msz = [&](int32_t b) { return (int64_t)ncol(b) + s->sn_nrow[b]; };

    // ---- 3. memory plan of the numeric factorisation (per shift)
    // L storage: supernode b keeps the first ncol columns of its m x m front (column-major,
    // leading dimension m) -- the factor the solves read.  Level workspace: while level l
    // is factored, its fronts are packed from offset 0 of one workspace reused by every
    // level.  Contribution-block pool: after level l is factored, the trailing nr x nr
    // block (nr = m - ncol) of each of its fronts is stored in the pool until the parent's
    // extend-add reads it; the pool addresses are planned here by first fit over the
    // blocks' lifetimes (stored at the end of the child's level, dead once the parent's
    // level has started).  Blocks are stored as packed lower triangles.
    std::vector<std::vector<int32_t>> lev_sn(nlev);
    for (int32_t b = 0; b < nsn; ++b) lev_sn[s->sn_level[b]].push_back(b);
    auto al32 = [](int64_t x) { return (x + 31) / 32 * 32; };      // 256-byte aligned blocks
    auto tri = [](int64_t r) { return r * (r + 1) / 2; };          // packed lower triangle
    s->front_off.assign(nsn, 0);
    s->l_off.assign(nsn, 0);
    s->cb_off.assign(nsn, -1);
    s->lev_ws.assign(nlev, 0);
    s->ws_total = 0;
    int64_t loff = 0;
    for (int32_t l = 0; l < nlev; ++l) {
        int64_t off = 0;
        for (int32_t b : lev_sn[l]) {
            s->front_off[b] = off;
            off += al32(msz(b) * msz(b));
            s->l_off[b] = loff;
            loff += al32(msz(b) * ncol(b));
        }
        s->lev_ws[l] = off;
        s->ws_total = std::max(s->ws_total, off);
    }
    s->l_total = loff;
    {
        std::map<int64_t, int64_t> hole;         // free intervals of the pool: start -> length
        int64_t top = 0;
        auto release = [&](int64_t st, int64_t len) {
            auto it = hole.emplace(st, len).first;
            if (it != hole.begin()) {
                auto pv = std::prev(it);
                if (pv->first + pv->second == it->first) { pv->second += it->second; hole.erase(it); it = pv; }
            }
            auto nx = std::next(it);
            if (nx != hole.end() && it->first + it->second == nx->first) { it->second += nx->second; hole.erase(nx); }
            if (it->first + it->second == top) { top = it->first; hole.erase(it); }
        };
        for (int32_t l = 0; l < nlev; ++l) {
            for (int32_t p : lev_sn[l])
                for (int32_t c : children[p])
                    if (s->cb_off[c] >= 0) release(s->cb_off[c], al32(tri((int64_t)s->sn_nrow[c])));
            for (int32_t b : lev_sn[l]) {
                const int64_t nr = s->sn_nrow[b];
                if (nr == 0) continue;
                const int64_t need = al32(tri(nr));
                auto it = hole.begin();
                while (it != hole.end() && it->second < need) ++it;
                if (it != hole.end()) {
                    s->cb_off[b] = it->first;
                    const int64_t st = it->first + need, len = it->second - need;
                    hole.erase(it);
                    if (len > 0) hole.emplace(st, len);
                } else {
                    s->cb_off[b] = top;
                    top += need;
                    s->cb_total = std::max(s->cb_total, top);
                }
            }
        }
    }
    // per-level store tasks: copy each front's L columns to L storage and its
    // contribution block to the pool (one unit per front column)
    s->store_tasks.clear();
    s->lev_store_off.assign(nlev + 1, 0);
    s->lev_store_cols.assign(nlev, 0);
    for (int32_t l = 0; l < nlev; ++l) {
        s->lev_store_off[l] = (int32_t)s->store_tasks.size();
        int32_t cols = 0;
        for (int32_t b : lev_sn[l]) {
            StoreTask t{};
            t.ws_off = s->front_off[b];
            t.l_off = s->l_off[b];
            t.cb_off = s->cb_off[b];
            t.m = (int32_t)msz(b);
            t.ncol = ncol(b);
            t.col_pre = cols;
            cols += t.m;
            s->store_tasks.push_back(t);
        }
        s->lev_store_cols[l] = cols;
    }
    s->lev_store_off[nlev] = (int32_t)s->store_tasks.size();

    // assembly map of the stored entries whose permuted position is in the lower triangle
    {
        std::vector<int32_t> elev(s->nnz);
        std::vector<int64_t> edest(s->nnz);
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t i_old = 0; i_old < n; ++i_old) {
            int32_t r = s->iperm[i_old];
            for (int64_t p = s->rowptr[i_old]; p < s->rowptr[i_old + 1]; ++p) {
                int32_t c = s->iperm[s->colind[p]];
                if (r < c) { elev[p] = -1; continue; }
                int32_t b = blockof[c];
                int32_t lc = c - first[b];
                int64_t lr;
                if (r < first[b + 1]) {
                    lr = r - first[b];
                } else {
                    const int32_t *rb = idx.data() + s->sn_idx_off[b] + ncol(b);
                    const int32_t *re = rb + s->sn_nrow[b];
                    lr = ncol(b) + (std::lower_bound(rb, re, r) - rb);
                }
                elev[p] = s->sn_level[b];
                edest[p] = s->front_off[b] + (int64_t)lc * msz(b) + lr;   // workspace offset
            }
        }
        s->asm_lev_off.assign(nlev + 1, 0);
        for (int64_t p = 0; p < s->nnz; ++p)
            if (elev[p] >= 0) s->asm_lev_off[elev[p] + 1]++;
        for (int32_t l = 0; l < nlev; ++l) s->asm_lev_off[l + 1] += s->asm_lev_off[l];
        std::vector<int64_t> fill(s->asm_lev_off.begin(), s->asm_lev_off.end() - 1);
        s->asm_e.assign(s->asm_lev_off[nlev], 0);
        s->asm_dest.assign(s->asm_lev_off[nlev], 0);
        for (int64_t p = 0; p < s->nnz; ++p) {
            if (elev[p] < 0) continue;
            int64_t q = fill[elev[p]]++;
            s->asm_e[q] = (int32_t)p;
            s->asm_dest[q] = edest[p];
        }
    }

    // child -> parent relative maps and extend-add passes per parent level
    std::vector<int64_t> rel_off(nsn, -1);
    s->relmap.clear();
    for (int32_t b = 0; b < nsn; ++b) {
        int32_t p = s->sn_parent[b];
        if (p < 0) continue;
        rel_off[b] = (int64_t)s->relmap.size();
        const int32_t *prow = idx.data() + s->sn_idx_off[p] + ncol(p);
        const int32_t *prow_end = prow + s->sn_nrow[p];
        const int64_t o = s->sn_idx_off[b] + ncol(b);
        for (int32_t r = 0; r < s->sn_nrow[b]; ++r) {
            int32_t i = idx[o + r];
            int32_t pos;
            if (i < first[p + 1]) pos = i - first[p];
            else pos = ncol(p) + (int32_t)(std::lower_bound(prow, prow_end, i) - prow);
            s->relmap.push_back(pos);
        }
    }
    s->ext_tasks.clear();
    s->ext_pass.clear();
    s->lev_ext_pass_off.assign(nlev + 1, 0);
    for (int32_t l = 0; l < nlev; ++l) {
        s->lev_ext_pass_off[l] = (int32_t)s->ext_pass.size();
        size_t maxc = 0;
        for (int32_t p : lev_sn[l]) maxc = std::max(maxc, children[p].size());
        for (size_t qn = 0; qn < maxc; ++qn) {
            ExtendPass ps{(int64_t)s->ext_tasks.size(), 0, 0};
            for (int32_t p : lev_sn[l]) {
                if (qn >= children[p].size()) continue;
                int32_t c = children[p][qn];
                if (s->sn_nrow[c] == 0) continue;
                ExtendTask t{};
                t.child_off = s->cb_off[c];              // the child's block in the pool
                t.parent_off = s->front_off[p];          // the parent's front in the workspace
                t.rel_off = rel_off[c];
                t.child_m = s->sn_nrow[c];               // leading dimension of the block
                t.child_ncol = 0;
                t.parent_m = (int32_t)msz(p);
                t.col_pre = ps.cols;
                ps.cols += s->sn_nrow[c];
                ps.count++;
                s->ext_tasks.push_back(t);
            }
            if (ps.count) s->ext_pass.push_back(ps);
        }
    }
    s->lev_ext_pass_off[nlev] = (int32_t)s->ext_pass.size();

    // ---- 4. panels, factor steps and solve levels
    s->panels.clear();
    std::vector<int32_t> sn_panel0(nsn);
    for (int32_t b = 0; b < nsn; ++b) {
        sn_panel0[b] = (int32_t)s->panels.size();
        for (int32_t k0 = 0; k0 < ncol(b); k0 += nb) {
            PanelDesc pd{};
            pd.front_off = s->l_off[b];                  // the solves read L storage
            pd.idx_off = s->sn_idx_off[b];
            pd.m = (int32_t)msz(b);
            pd.k0 = k0;
            pd.w = std::min(nb, ncol(b) - k0);
            pd.g0 = first[b] + k0;
            pd.sn = b;
            s->panels.push_back(pd);
        }
    }
    s->tasks.clear();
    s->steps.clear();
    s->lev_step_off.assign(nlev + 1, 0);
    s->wbuf_max = 0;
    s->mt_max = 0;
    s->sl_max = 0;
    s->ex_max = 0;
    for (int32_t l = 0; l < nlev; ++l) {
        s->lev_step_off[l] = (int32_t)s->steps.size();
        int32_t T = 0;
        for (int32_t b : lev_sn[l]) T = std::max<int32_t>(T, (int32_t)cdiv(ncol(b), nb));
        for (int32_t t = 0; t < T; ++t) {
            StepDesc sd{(int64_t)s->tasks.size(), 0, 0, 0, l, 0.0, 0.0, 0, 0, 0, 0};
            int64_t wb = 0;
            for (int32_t b : lev_sn[l]) {
                if ((int64_t)t * nb >= ncol(b)) continue;
                StepTask tk{};
                tk.front_off = s->front_off[b];
                tk.m = (int32_t)msz(b);
                tk.k0 = t * nb;
                tk.w = std::min(nb, ncol(b) - t * nb);
                tk.r = tk.m - tk.k0 - tk.w;
                tk.panel = sn_panel0[b] + t;
                tk.mt_slot = sd.count;
                tk.wbuf_off = wb;
                wb += (int64_t)tk.r * tk.w;
                tk.tiles4_pre = sd.tiles4;
                tk.tiles3_pre = sd.tiles3;
                int32_t nt = (int32_t)cdiv(tk.r, 64);
                sd.tiles4 += nt;
                sd.tiles3 += nt * (nt + 1) / 2;
                // tensor-core Schur update: 128-row slice tiles of L21 and W, and the
                // 128 x 64 output tiles (bi, bj <= 2 bi + 1) of the lower triangle
                const int32_t nrt = (int32_t)cdiv(tk.r, 128), nct = nt;
                tk.sl_pre = sd.sl_tiles;
                tk.tc_pre = sd.tc_tiles;
                tk.sl_off = sd.sl_bytes;
                tk.ex_off = sd.ex_count;
                sd.sl_tiles += 2 * nrt;
                sd.tc_tiles += nrt > 0 ? (nrt - 1) * nrt + nct : 0;
                sd.sl_bytes += (int64_t)2 * nrt * kTcSlices * kTcSliceBytes;
                sd.ex_count += 2 * (int64_t)tk.r;
                sd.flops4 += 2.0 * tk.r * (double)tk.w * tk.w;
                sd.flops3 += (double)tk.w * tk.r * (tk.r + 1.0);
                sd.count++;
                s->tasks.push_back(tk);
            }
            s->wbuf_max = std::max(s->wbuf_max, wb);
            s->mt_max = std::max(s->mt_max, sd.count);
            s->sl_max = std::max(s->sl_max, sd.sl_bytes);
            s->ex_max = std::max(s->ex_max, sd.ex_count);
            s->steps.push_back(sd);
        }
    }
    s->lev_step_off[nlev] = (int32_t)s->steps.size();
    s->step_mode.assign(s->steps.size(), -1);

    // solve levels: panel (b, t) waits for panel (b, t-1), or for the last panel of
    // every child when t = 0
    std::vector<int32_t> plev(s->panels.size(), 0);
    int32_t nplev = 0;
    for (int32_t b = 0; b < nsn; ++b) {
        int32_t np = (int32_t)cdiv(ncol(b), nb);
        int32_t base = 0;
        for (int32_t c : children[b]) {
            int32_t cl = sn_panel0[c] + (int32_t)cdiv(ncol(c), nb) - 1;
            base = std::max(base, plev[cl] + 1);
        }
        for (int32_t t = 0; t < np; ++t) {
            plev[sn_panel0[b] + t] = base + t;
            nplev = std::max(nplev, base + t + 1);
        }
    }
    std::vector<std::vector<int32_t>> by_lev(nplev);
    for (int32_t p = 0; p < (int32_t)s->panels.size(); ++p) by_lev[plev[p]].push_back(p);
    s->solve_panels.clear();
    s->solve_levels.clear();
    s->solve_tile_pre.clear();
    for (int32_t l = 0; l < nplev; ++l) {
        SolveLevel sl{(int64_t)s->solve_panels.size(), 0, 0, 0.0};
        for (int32_t p : by_lev[l]) {
            const PanelDesc &pd = s->panels[p];
            s->solve_panels.push_back(p);
            s->solve_tile_pre.push_back(sl.row_tiles);
            sl.row_tiles += (int32_t)cdiv(pd.m - pd.k0 - pd.w, 64);
            sl.offdiag += (double)(pd.m - pd.k0 - pd.w) * pd.w;
            sl.count++;
        }
        s->solve_levels.push_back(sl);
    }

    // ---- counts
    ss_symbolic_info &inf = s->info;
    inf = ss_symbolic_info{};
    inf.n = n;
    inf.nnz = s->nnz;
    inf.n_supernodes = nsn;
    inf.n_levels = nlev;
    inf.n_panels = (int64_t)s->panels.size();
    inf.n_panel_levels = nplev;
    for (int32_t b = 0; b < nsn; ++b) {
        double sc = ncol(b), bb = s->sn_nrow[b];
        inf.max_front = std::max<int64_t>(inf.max_front, msz(b));
        inf.factor_entries += msz(b) * ncol(b);
        inf.front_entries += msz(b) * msz(b);
        inf.factor_flops += sc * sc * sc / 3.0 + sc * sc * bb + sc * bb * bb;
    }
    for (const StepTask &tk : s->tasks) {
        const double r = tk.r, w = tk.w;
        inf.schur_flops += w * r * (r + 1.0);
        inf.panel_flops += 2.0 * r * w * w;
        inf.l_offdiag_entries += (int64_t)tk.r * tk.w;
        inf.l_diag_entries += (int64_t)tk.w * tk.w;
    }
    inf.l_storage_entries = s->l_total;
    inf.workspace_entries = s->ws_total;
    inf.cb_pool_entries = s->cb_total;
    inf.analyze_seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return SS_OK;
}

extern "C" ss_status ss_analyze(ss_ctx *ctx, int64_t n, const int64_t *rowptr,
                                const int32_t *colind, const ss_options *opt, ss_symbolic **out) {
    if (!ctx) return SS_ERR_ARG;
    if (!out || !rowptr || !colind || n <= 0 || n > INT32_MAX - 1)
        return ctx->set_error(SS_ERR_ARG, "ss_analyze: null pointer or bad n");
    *out = nullptr;
    ss_symbolic *s = new (std::nothrow) ss_symbolic();
    if (!s) return ctx->set_error(SS_ERR_OOM, "ss_analyze: host allocation failed");
    int rc;
    try {
        rc = analyze_impl(ctx, n, rowptr, colind, opt, s);
        if (rc == SS_OK) rc = ss_symbolic_upload(s);
    } catch (const std::bad_alloc &) {
        rc = ctx->set_error(SS_ERR_OOM, "ss_analyze: host allocation failed");
    }
    if (rc != SS_OK) {
        ss_symbolic_free_device(s);
        delete s;
        return rc;
    }
    *out = s;
    return SS_OK;
}

extern "C" ss_status ss_symbolic_info_get(const ss_symbolic *sym, ss_symbolic_info *info) {
    if (!sym || !info) return SS_ERR_ARG;
    *info = sym->info;
    return SS_OK;
}

extern "C" ss_status ss_symbolic_perm(const ss_symbolic *sym, int32_t *perm) {
    if (!sym || !perm) return SS_ERR_ARG;
    std::memcpy(perm, sym->perm.data(), sizeof(int32_t) * sym->n);
    return SS_OK;
}

extern "C" ss_status ss_symbolic_destroy(ss_symbolic *sym) {
    if (!sym) return SS_OK;
    ss_free_plans(sym);
    oz_free_symbolic(sym);
    ss_symbolic_free_device(sym);
    delete sym;
    return SS_OK;
}

// ---------------------------------------------------------------- validation
static int validate_impl(const ss_symbolic *s, std::string &why) {
    auto fail = [&](const std::string &m) { why = m; return SS_ERR_INTERNAL; };
    const int64_t n = s->n;
    std::vector<char> seen(n, 0);
    for (int64_t i = 0; i < n; ++i) {
        int32_t p = s->perm[i];
        if (p < 0 || p >= n || seen[p]) return fail("perm is not a permutation");
        seen[p] = 1;
        if (s->iperm[p] != i) return fail("iperm is not the inverse of perm");
    }
    const int32_t nsn = s->nsn;
    if ((int64_t)s->sn_first[nsn] != n || s->sn_first[0] != 0) return fail("supernodes do not cover 0..n");
    for (int32_t b = 0; b < nsn; ++b) {
        const int32_t ncol = s->sn_first[b + 1] - s->sn_first[b];
        if (ncol <= 0) return fail("empty supernode");
        const int64_t m = (int64_t)ncol + s->sn_nrow[b];
        if (s->sn_idx_off[b + 1] - s->sn_idx_off[b] != m) return fail("index list length != m");
        const int32_t *ix = s->idx.data() + s->sn_idx_off[b];
        for (int32_t i = 0; i < ncol; ++i)
            if (ix[i] != s->sn_first[b] + i) return fail("supernode columns not contiguous");
        for (int64_t i = ncol; i < m; ++i) {
            if (ix[i] <= s->sn_first[b + 1] - 1 || ix[i] >= n) return fail("row index out of range");
            if (i > ncol && ix[i] <= ix[i - 1]) return fail("row indices not increasing");
        }
        const int32_t lev = s->sn_level[b];
        if (lev < 0 || lev >= s->nlev) return fail("bad level");
        if (s->front_off[b] < 0 || s->front_off[b] + m * m > s->lev_ws[lev] || s->lev_ws[lev] > s->ws_total)
            return fail("front outside its level's workspace");
        if (s->front_off[b] % 32 || s->l_off[b] % 32) return fail("front or L block not 256-byte aligned");
        if (s->l_off[b] < 0 || s->l_off[b] + m * ncol > s->l_total) return fail("L block outside L storage");
        const int64_t nr = s->sn_nrow[b];
        if ((nr > 0) != (s->cb_off[b] >= 0)) return fail("contribution block without a pool slot (or vice versa)");
        if (nr > 0 && (s->cb_off[b] % 32 || s->cb_off[b] + nr * (nr + 1) / 2 > s->cb_total))
            return fail("contribution block outside the pool");
        const int32_t p = s->sn_parent[b];
        if (p >= 0 && (p <= b || s->sn_level[p] <= lev)) return fail("parent not after child");
        if ((p >= 0) != (nr > 0)) return fail("a root with rows below its block, or a child without");
    }
    // fronts of one level do not overlap in the workspace; L blocks never overlap
    for (int32_t l = 0; l < s->nlev; ++l) {
        std::vector<std::pair<int64_t, int64_t>> iv;
        for (int32_t b = 0; b < nsn; ++b)
            if (s->sn_level[b] == l) {
                const int64_t m = (int64_t)(s->sn_first[b + 1] - s->sn_first[b]) + s->sn_nrow[b];
                iv.push_back({s->front_off[b], s->front_off[b] + m * m});
            }
        std::sort(iv.begin(), iv.end());
        for (size_t i = 1; i < iv.size(); ++i)
            if (iv[i].first < iv[i - 1].second) return fail("two fronts of one level overlap");
    }
    {
        std::vector<std::pair<int64_t, int64_t>> iv;
        for (int32_t b = 0; b < nsn; ++b) {
            const int64_t nc = s->sn_first[b + 1] - s->sn_first[b];
            iv.push_back({s->l_off[b], s->l_off[b] + (nc + s->sn_nrow[b]) * nc});
        }
        std::sort(iv.begin(), iv.end());
        for (size_t i = 1; i < iv.size(); ++i)
            if (iv[i].first < iv[i - 1].second) return fail("two L blocks overlap");
    }
    // two contribution blocks alive at the same time never share pool entries: block b
    // lives from the end of level(b) until level(parent(b)) has started
    {
        struct Live { int64_t a, e; int32_t born, dies; };
        std::vector<Live> lv;
        for (int32_t b = 0; b < nsn; ++b)
            if (s->cb_off[b] >= 0)
                lv.push_back({s->cb_off[b], s->cb_off[b] + (int64_t)s->sn_nrow[b] * (s->sn_nrow[b] + 1) / 2, s->sn_level[b],
                              s->sn_level[s->sn_parent[b]]});
        std::sort(lv.begin(), lv.end(), [](const Live &x, const Live &y) { return x.a < y.a; });
        for (size_t i = 0; i < lv.size(); ++i)
            for (size_t j = i + 1; j < lv.size() && lv[j].a < lv[i].e; ++j) {
                // overlapping addresses: one must die (its parent's level starts) no later
                // than the level whose end stores the other
                const bool ok = lv[i].dies <= lv[j].born || lv[j].dies <= lv[i].born;
                if (!ok) return fail("two live contribution blocks share pool entries");
            }
    }
    // store tasks: every front of a level, column prefixes, offsets matching the plan
    for (int32_t l = 0; l < s->nlev; ++l) {
        int32_t cols = 0;
        for (int32_t q = s->lev_store_off[l]; q < s->lev_store_off[l + 1]; ++q) {
            const StoreTask &t = s->store_tasks[q];
            if (t.col_pre != cols) return fail("store column prefix");
            cols += t.m;
            if (t.ws_off + (int64_t)t.m * t.m > s->lev_ws[l]) return fail("store source outside the workspace");
            if (t.l_off + (int64_t)t.m * t.ncol > s->l_total) return fail("store L destination out of range");
            const int64_t nr = t.m - t.ncol;
            if (nr > 0 && (t.cb_off < 0 || t.cb_off + nr * (nr + 1) / 2 > s->cb_total)) return fail("store pool destination");
        }
        if (cols != s->lev_store_cols[l]) return fail("store column total");
    }
    for (int32_t l = 0; l < s->nlev; ++l) {
        for (int64_t q = s->asm_lev_off[l]; q < s->asm_lev_off[l + 1]; ++q) {
            if (s->asm_e[q] < 0 || s->asm_e[q] >= s->nnz) return fail("assembly entry out of range");
            if (s->asm_dest[q] < 0 || s->asm_dest[q] >= s->lev_ws[l])
                return fail("assembly destination outside the level's workspace");
        }
    }
    // every stored lower entry is assembled exactly once, into the right front
    std::vector<int32_t> blockof(n);
    for (int32_t b = 0; b < nsn; ++b)
        for (int32_t j = s->sn_first[b]; j < s->sn_first[b + 1]; ++j) blockof[j] = b;
    std::vector<char> hit(s->nnz, 0);
    for (int64_t q = 0; q < (int64_t)s->asm_e.size(); ++q) {
        if (hit[s->asm_e[q]]) return fail("entry assembled twice");
        hit[s->asm_e[q]] = 1;
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = s->rowptr[i]; p < s->rowptr[i + 1]; ++p) {
            int32_t r = s->iperm[i], c = s->iperm[s->colind[p]];
            if ((r >= c) != (bool)hit[p]) return fail("lower entry not assembled (or upper assembled)");
            if (r < c) continue;
            int32_t b = blockof[c];
            const int64_t m = (int64_t)(s->sn_first[b + 1] - s->sn_first[b]) + s->sn_nrow[b];
            const int32_t *ix = s->idx.data() + s->sn_idx_off[b];
            if (!std::binary_search(ix, ix + m, r)) return fail("stored entry outside its front");
        }
    for (const ExtendPass &ps : s->ext_pass) {
        std::vector<int64_t> parents;
        int32_t cols = 0;
        for (int32_t t = 0; t < ps.count; ++t) {
            const ExtendTask &et = s->ext_tasks[ps.task_off + t];
            if (et.col_pre != cols) return fail("extend-add column prefix mismatch");
            const int32_t nr = et.child_m - et.child_ncol;
            cols += nr;
            parents.push_back(et.parent_off);
            if (et.rel_off < 0 || et.rel_off + nr > (int64_t)s->relmap.size()) return fail("relmap range");
            for (int32_t r = 0; r < nr; ++r) {
                int32_t v = s->relmap[et.rel_off + r];
                if (v < 0 || v >= et.parent_m) return fail("relmap entry outside the parent front");
                if (r > 0 && v <= s->relmap[et.rel_off + r - 1]) return fail("relmap not increasing");
            }
            if (et.child_ncol != 0 || et.child_off < 0 || et.child_off + (int64_t)et.child_m * (et.child_m + 1) / 2 > s->cb_total)
                return fail("extend-add source outside the contribution-block pool");
            if (et.parent_off < 0 || et.parent_off + (int64_t)et.parent_m * et.parent_m > s->ws_total)
                return fail("extend-add destination outside the workspace");
        }
        if (cols != ps.cols) return fail("extend-add pass column count");
        std::sort(parents.begin(), parents.end());
        if (std::adjacent_find(parents.begin(), parents.end()) != parents.end())
            return fail("two children of one parent in the same extend-add pass");
    }
    const int64_t npan = (int64_t)s->panels.size();
    for (const PanelDesc &pd : s->panels) {
        const int32_t b = pd.sn;
        const int32_t ncol = s->sn_first[b + 1] - s->sn_first[b];
        if (pd.w <= 0 || pd.w > s->nb || pd.k0 < 0 || pd.k0 + pd.w > ncol) return fail("panel columns");
        if (pd.g0 != s->sn_first[b] + pd.k0 || pd.front_off != s->l_off[b] ||
            pd.idx_off != s->sn_idx_off[b] || pd.m != ncol + s->sn_nrow[b])
            return fail("panel descriptor mismatch");
    }
    for (const StepDesc &sd : s->steps) {
        int32_t t4 = 0, t3 = 0, tsl = 0, ttc = 0;
        int64_t slb = 0, exc = 0;
        for (int32_t t = 0; t < sd.count; ++t) {
            const StepTask &tk = s->tasks[sd.task_off + t];
            if (tk.panel < 0 || tk.panel >= npan) return fail("step panel id");
            const PanelDesc &pd = s->panels[tk.panel];
            if (tk.k0 != pd.k0 || tk.w != pd.w || tk.m != pd.m || tk.front_off != s->front_off[pd.sn])
                return fail("step task / panel mismatch");
            if (tk.r != tk.m - tk.k0 - tk.w || tk.r < 0) return fail("step trailing size");
            if (tk.wbuf_off < 0 || tk.wbuf_off + (int64_t)tk.r * tk.w > s->wbuf_max) return fail("W scratch range");
            if (tk.mt_slot != t || tk.mt_slot >= s->mt_max) return fail("Mt scratch slot");
            if (tk.tiles4_pre != t4 || tk.tiles3_pre != t3) return fail("tile prefixes");
            int32_t nt = (tk.r + 63) / 64;
            t4 += nt;
            t3 += nt * (nt + 1) / 2;
            // tensor-core path: slice tiles, output tiles, scratch ranges of this task
            const int32_t nrt = (tk.r + 127) / 128;
            if (tk.sl_pre != tsl || tk.tc_pre != ttc || tk.sl_off != slb || tk.ex_off != exc)
                return fail("tensor-core prefixes");
            tsl += 2 * nrt;
            ttc += nrt > 0 ? (nrt - 1) * nrt + nt : 0;
            slb += (int64_t)2 * nrt * kTcSlices * kTcSliceBytes;
            exc += 2 * (int64_t)tk.r;
            if (slb > s->sl_max || exc > s->ex_max) return fail("tensor-core scratch range");
            if (tk.sl_off % 16) return fail("slice block not 16-byte aligned");
        }
        if (t4 != sd.tiles4 || t3 != sd.tiles3) return fail("step tile totals");
        if (tsl != sd.sl_tiles || ttc != sd.tc_tiles || slb != sd.sl_bytes || exc != sd.ex_count)
            return fail("tensor-core step totals");
    }
    std::vector<char> pseen(npan, 0);
    for (const SolveLevel &sl : s->solve_levels) {
        int32_t tiles = 0;
        for (int32_t t = 0; t < sl.count; ++t) {
            int32_t p = s->solve_panels[sl.panel_off + t];
            if (p < 0 || p >= npan || pseen[p]) return fail("solve level panel id");
            pseen[p] = 1;
            if (s->solve_tile_pre[sl.panel_off + t] != tiles) return fail("solve tile prefix");
            const PanelDesc &pd = s->panels[p];
            tiles += (pd.m - pd.k0 - pd.w + 63) / 64;
        }
        if (tiles != sl.row_tiles) return fail("solve level tile total");
    }
    for (int64_t p = 0; p < npan; ++p)
        if (!pseen[p]) return fail("panel missing from the solve schedule");
    return SS_OK;
}

extern "C" ss_status ss_symbolic_validate(const ss_symbolic *sym) {
    if (!sym) return SS_ERR_ARG;
    std::string why;
    int rc = validate_impl(sym, why);
    if (rc != SS_OK) sym->ctx->set_error(rc, "ss_symbolic_validate: " + why);
    return rc;
}
