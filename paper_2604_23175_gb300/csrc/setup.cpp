// Host-side symbolic setup (see setup.h).
#include "setup.h"

#include <algorithm>
#include <queue>
#include <cmath>
#include <numeric>
#include <stdexcept>

namespace mase {

namespace {

[[noreturn]] void fail(const std::string &m) { throw std::runtime_error(m); }

inline int packed_col_start(int cb, int nb) { return cb * nb - cb * (cb - 1) / 2; }

}  // namespace

SmemLayout area_smem_layout(int nv, int nb_loc, int n_ends, int n_own, size_t rg, size_t rs) {
    auto a16 = [](size_t x) { return (x + 15) & ~size_t(15); };
    SmemLayout L;
    const size_t endstride = std::max<size_t>(16, 4 * rg);
    size_t o = 0;
    L.off_g = o;
    o = a16(o + (size_t)nv * sizeof(double));
    L.off_y = o;
    o = a16(o + (size_t)nv * rs);
    L.off_bus = o;
    o = a16(o + 3 * (size_t)nb_loc * sizeof(double));
    L.off_end = o;
    o = a16(o + (size_t)n_ends * endstride);
    L.off_inj = o;
    o = a16(o + (size_t)n_own * 16);
    L.off_self = o;
    o = a16(o + 4 * (size_t)n_own * rg);
    L.off_st = o;
    L.vector_bytes = o;
    return L;
}

int SymFactor::pos(int r, int c) const {
    if (r < c) std::swap(r, c);
    if (c >= n_int) {
        int rb = r - n_int, cb = c - n_int;
        return off_B + packed_col_start(cb, n_bnd) + (rb - cb);
    }
    int t = var_sn[c];
    int c0 = sn_c0[t], w = sn_w[t], nr = sn_nr[t];
    int ld = w + nr;
    int rp;
    if (r < c0 + w) {
        rp = r - c0;
    } else {
        const int *b = rows.data() + sn_rows[t];
        const int *e = b + nr;
        const int *it = std::lower_bound(b, e, r);
        if (it == e || *it != r) return -1;
        rp = w + (int)(it - b);
    }
    return sn_off[t] + (c - c0) * ld + rp;
}

// Dataflow task list of the numeric factorisation (Sec. 4.3 Schur mode).
// Tasks: D(s) factors the diagonal block of supernode s and forward-solves its
// rhs; C(s, r0) solves 32 rows of the panel below it; U(s, j0) applies up to
// kUnitCols target columns of s's update to an ancestor (or to the trailing
// Schur block) and, when j0 starts a target segment, that segment's rhs rows.
// Counters: ctr[t] counts finished updates into supernode t, ctr[nsn + s]
// counts finished D(s) and C(s, .) tasks.  The order is a list schedule of
// nwarps workers with estimated cycle costs, highest bottom level first among
// the ready tasks, so it is a topological order in which warps that take the
// next task rarely wait.
void build_tasks(SymFactor &F, int nwarps, bool level_sched) {
    const int nsn = F.nsn();
    F.tasks.clear();
    F.n_tasks = 0;
    F.level_sched = level_sched ? 1 : 0;
    F.lev_tasks.assign(3 * (size_t)F.nlev() + 1, 0);
    if (nsn == 0) return;
    struct Task {
        int type, s, idx;   // idx: r0 (chunk) or unit number
        double cost;
    };
    std::vector<Task> tk;
    std::vector<int> d_of(nsn), nchunk(nsn, 0), nin(nsn, 0);
    std::vector<std::vector<int>> c_of(nsn), u_of(nsn), u_into(nsn);
    for (int s = 0; s < nsn; ++s) {
        const int w = F.sn_w[s], ld = w + F.sn_nr[s];
        d_of[s] = (int)tk.size();
        // estimated cycles (fitted to per-task timings of the area kernel on GB300)
        tk.push_back({0, s, 0, 300.0 + 550.0 * w});
        for (int r0 = w; r0 < ld; r0 += 32) {
            c_of[s].push_back((int)tk.size());
            tk.push_back({1, s, r0, 300.0 + 300.0 * w});
            ++nchunk[s];
        }
    }
    std::vector<int> u_tgt(F.unit_sn.size()), u_rhs(F.unit_sn.size(), 0);
    for (size_t u = 0; u < F.unit_sn.size(); ++u) {
        const int s = F.unit_sn[u], j = F.unit_j[u], nj = F.unit_nj[u], w = F.sn_w[s];
        const int R = F.sn_nr[s], rb = F.sn_rows[s];
        auto tgt = [&](int jj) {
            const int c = F.rows[rb + jj];
            return c < F.n_int ? F.var_sn[c] : -1;
        };
        const int t = tgt(j);
        u_tgt[u] = t;
        if (j == 0 || tgt(j - 1) != t) {
            int e = j + 1;
            while (e < R && tgt(e) == t) ++e;
            u_rhs[u] = e;
        }
        const int tid = (int)tk.size();
        const double passes = std::ceil((R - j) / 96.0);
        const double mc = std::min(3.0, std::ceil((R - j) / 32.0));
        tk.push_back({2, s, (int)u, 2500.0 + passes * w * std::max(50.0, 60.0 * nj + 110.0 * mc - 250.0)});
        u_of[s].push_back(tid);
        if (t >= 0) {
            u_into[t].push_back(tid);
            ++nin[t];
        }
    }
    const int nt = (int)tk.size();
    // successors and predecessor counts
    std::vector<std::vector<int>> succ(nt);
    std::vector<int> npred(nt, 0);
    auto edge = [&](int a, int b) {
        succ[a].push_back(b);
        ++npred[b];
    };
    for (int s = 0; s < nsn; ++s) {
        for (int c : c_of[s]) edge(d_of[s], c);
        for (int u : u_of[s]) {
            edge(d_of[s], u);
            for (int c : c_of[s]) edge(c, u);
        }
        for (int u : u_into[s]) edge(u, d_of[s]);
    }
    // bottom levels (longest cost path to a sink); tasks were created with
    // every edge pointing to a later D, or from D/C to U of the same s
    std::vector<double> bl(nt, 0.0);
    {
        // reverse topological order by Kahn on the reversed graph
        std::vector<int> nsucc(nt), order;
        order.reserve(nt);
        for (int i = 0; i < nt; ++i) {
            nsucc[i] = (int)succ[i].size();
            if (!nsucc[i]) order.push_back(i);
        }
        std::vector<std::vector<int>> pred(nt);
        for (int i = 0; i < nt; ++i)
            for (int j : succ[i]) pred[j].push_back(i);
        for (size_t q = 0; q < order.size(); ++q) {
            const int i = order[q];
            double m = 0.0;
            for (int j : succ[i]) m = std::max(m, bl[j]);
            bl[i] = tk[i].cost + m;
            for (int p : pred[i])
                if (--nsucc[p] == 0) order.push_back(p);
        }
        if ((int)order.size() != nt) fail("symbolic: task graph has a cycle");
    }
    // list schedule: the earliest free warp takes the ready task of highest
    // bottom level, else the task that becomes ready first
    std::vector<double> ready(nt, 0.0), fin(nt, 0.0);
    std::vector<int> left = npred;
    using PQ = std::pair<double, int>;
    std::priority_queue<PQ, std::vector<PQ>, std::greater<PQ>> pending;   // by ready time
    std::priority_queue<PQ> avail;                                         // by bottom level
    for (int i = 0; i < nt; ++i)
        if (!left[i]) pending.push({0.0, i});
    std::priority_queue<double, std::vector<double>, std::greater<double>> wfree;
    for (int w = 0; w < std::max(1, nwarps); ++w) wfree.push(0.0);
    std::vector<int> order;
    order.reserve(nt);
    while ((int)order.size() < nt) {
        const double tau = wfree.top();
        wfree.pop();
        while (!pending.empty() && pending.top().first <= tau) {
            avail.push({bl[pending.top().second], pending.top().second});
            pending.pop();
        }
        int i;
        if (!avail.empty()) {
            i = avail.top().second;
            avail.pop();
        } else {
            if (pending.empty()) fail("symbolic: task schedule stalled");
            i = pending.top().second;
            pending.pop();
        }
        const double start = std::max(tau, ready[i]);
        fin[i] = start + tk[i].cost;
        wfree.push(fin[i]);
        order.push_back(i);
        for (int j : succ[i]) {
            ready[j] = std::max(ready[j], fin[i]);
            if (--left[j] == 0) pending.push({ready[j], j});
        }
    }
    if (level_sched) {
        std::vector<int> lev(nsn, 0);
        for (int l = 0; l < F.nlev(); ++l)
            for (int i = F.lev_off[l]; i < F.lev_off[l + 1]; ++i) lev[F.sn_order[i]] = l;
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            if (lev[tk[a].s] != lev[tk[b].s]) return lev[tk[a].s] < lev[tk[b].s];
            return tk[a].type < tk[b].type;
        });
        int q = 0;
        for (int l = 0; l < F.nlev(); ++l)
            for (int ty = 0; ty < 3; ++ty) {
                F.lev_tasks[3 * l + ty] = q;
                while (q < nt && lev[tk[order[q]].s] == l && tk[order[q]].type == ty) ++q;
            }
        F.lev_tasks[3 * F.nlev()] = q;
        if (q != nt) fail("symbolic: level task groups incomplete");
    }
    // records
    F.tasks.assign((size_t)nt * 16, 0);
    for (int q = 0; q < nt; ++q) {
        const Task &T = tk[order[q]];
        int *r = F.tasks.data() + (size_t)q * 16;
        const int s = T.s, w = F.sn_w[s], ld = w + F.sn_nr[s];
        if (T.type == 0) {
            r[0] = (0 << 24) | s;
            r[1] = s;
            r[2] = nin[s];
            r[3] = nsn + s;
            r[4] = F.sn_off[s]; r[5] = w; r[6] = ld; r[7] = F.sn_c0[s];
        } else if (T.type == 1) {
            r[0] = (1 << 24) | s;
            r[1] = nsn + s;
            r[2] = 1;
            r[3] = nsn + s;
            r[4] = F.sn_off[s]; r[5] = w; r[6] = ld; r[7] = T.idx;
        } else {
            const int u = T.idx, j = F.unit_j[u], nj = F.unit_nj[u], rb = F.sn_rows[s];
            r[0] = (2 << 24) | s;
            r[1] = nsn + s;
            r[2] = 1 + nchunk[s];
            r[3] = u_tgt[u] >= 0 ? u_tgt[u] : -1;
            r[4] = F.sn_off[s] + w; r[5] = F.relbase[rb + j]; r[6] = rb; r[7] = F.sn_c0[s];
            r[8] = w | (nj << 8); r[9] = ld | (j << 16); r[10] = u_rhs[u];
            for (int k = 0; k < nj; ++k) r[11 + k] = F.colbase[rb + j + k];
        }
    }
    F.n_tasks = nt;
    // estimated makespan of the schedule (cycles)
    double mk = 0.0;
    for (int i = 0; i < nt; ++i) mk = std::max(mk, fin[i]);
    F.sched_cycles = mk;
}

SymResult build_symbolic(const BusSystem &sys, double relax_alpha, int relax_wmax, int max_panel,
                         bool level_sched) {
    if (max_panel < 1 || max_panel > kMaxPanel) fail("symbolic: panel width out of range");
    const int ni = sys.nb_int, nbn = sys.nb_bnd, n = ni + nbn;
    SymResult out;
    // --- exact minimum degree on the elimination graph (dense bitmap) ---
    std::vector<uint8_t> A((size_t)n * n, 0);
    std::vector<int> deg(n, 0);
    for (int v = 0; v < n; ++v)
        for (int u : sys.adj[v])
            if (u != v && !A[(size_t)v * n + u]) {
                A[(size_t)v * n + u] = A[(size_t)u * n + v] = 1;
                ++deg[v];
                ++deg[u];
            }
    std::vector<char> elim(n, 0);
    std::vector<std::vector<int>> snodes(n);
    std::vector<int> nb;
    out.order.reserve(n);
    for (int step = 0; step < ni; ++step) {
        int best = -1;
        for (int v = 0; v < ni; ++v)
            if (!elim[v] && (best < 0 || deg[v] < deg[best])) best = v;
        nb.clear();
        const uint8_t *row = A.data() + (size_t)best * n;
        for (int u = 0; u < n; ++u)
            if (!elim[u] && row[u]) nb.push_back(u);
        snodes[best] = nb;
        for (int a : nb) {
            A[(size_t)a * n + best] = A[(size_t)best * n + a] = 0;
            --deg[a];
        }
        for (size_t i = 0; i < nb.size(); ++i)
            for (size_t j = i + 1; j < nb.size(); ++j) {
                int a = nb[i], b = nb[j];
                if (!A[(size_t)a * n + b]) {
                    A[(size_t)a * n + b] = A[(size_t)b * n + a] = 1;
                    ++deg[a];
                    ++deg[b];
                }
            }
        elim[best] = 1;
        out.order.push_back(best);
    }
    for (int v = ni; v < n; ++v) out.order.push_back(v);
    out.pos_of.assign(n, -1);
    for (int p = 0; p < n; ++p) out.pos_of[out.order[p]] = p;
    out.var0.assign(n + 1, 0);
    for (int p = 0; p < n; ++p) out.var0[p + 1] = out.var0[p] + sys.nvar[out.order[p]];

    // --- structure in positions, elimination tree ---
    std::vector<std::vector<int>> S(ni);
    std::vector<int> parent(ni, -1), nchild(ni, 0);
    for (int p = 0; p < ni; ++p) {
        for (int u : snodes[out.order[p]]) S[p].push_back(out.pos_of[u]);
        std::sort(S[p].begin(), S[p].end());
        if (!S[p].empty() && S[p][0] <= p) fail("symbolic: structure not above diagonal");
        if (!S[p].empty() && S[p][0] < ni) {
            parent[p] = S[p][0];
            ++nchild[S[p][0]];
        }
    }
    // --- relaxed supernodes ---
    // Fundamental supernodes first; then, bottom-up, a supernode absorbs the
    // child group that adds the fewest explicit zeros if the zeros stay below
    // a fraction of the merged panel and the group stays narrow.  An
    // elimination-tree postorder that visits the absorbed child last keeps
    // every group contiguous; any topological order of the tree gives the
    // same factor structure, so the fill does not change.
    std::vector<int> sn_first;
    {
        std::vector<int> f_first;
        for (int p = 0; p < ni; ++p) {
            bool merge = p > 0 && parent[p - 1] == p && nchild[p] == 1 &&
                         S[p - 1].size() == S[p].size() + 1 &&
                         std::equal(S[p].begin(), S[p].end(), S[p - 1].begin() + 1);
            if (!merge) f_first.push_back(p);
        }
        f_first.push_back(ni);
        const int nf = (int)f_first.size() - 1;
        std::vector<int> f_of(ni);
        for (int f = 0; f < nf; ++f)
            for (int p = f_first[f]; p < f_first[f + 1]; ++p) f_of[p] = f;
        std::vector<int> f_par(nf, -1);
        std::vector<std::vector<int>> f_kids(nf);
        for (int f = 0; f < nf; ++f) {
            int top = f_first[f + 1] - 1;
            if (parent[top] >= 0) {
                f_par[f] = f_of[parent[top]];
                f_kids[f_par[f]].push_back(f);
            }
        }
        // group state per fundamental supernode (as the top of its group)
        std::vector<long long> gw(nf), gzero(nf, 0);   // width (buses), explicit zeros so far
        std::vector<int> absorbed(nf, -1);
        const double alpha = relax_alpha;
        const int wmax = relax_alpha > 0 ? relax_wmax : 0;   // buses per merged supernode
        for (int t = 0; t < nf; ++t) {
            const long long wt = f_first[t + 1] - f_first[t];
            const long long Rt = (long long)S[f_first[t + 1] - 1].size();
            gw[t] = wt;
            int best = -1;
            long long best_z = 0;
            for (int c : f_kids[t]) {
                const long long Rc = (long long)S[f_first[c + 1] - 1].size();
                const long long W = gw[c] + wt;
                if (W > wmax) continue;
                const long long z = gzero[c] + gw[c] * (wt + Rt - Rc);
                const long long nz = W * (W - 1) / 2 + W * Rt;
                if (z > alpha * (double)nz) continue;
                if (best < 0 || gw[c] > gw[best] || (gw[c] == gw[best] && z < best_z)) {
                    best = c;
                    best_z = z;
                }
            }
            if (best >= 0) {
                absorbed[t] = best;
                gw[t] = gw[best] + wt;
                gzero[t] = best_z;
            }
        }
        // postorder of the fundamental-supernode forest, absorbed child last
        std::vector<int> new_of_old(ni, -1), group_start;
        std::vector<char> is_absorbed(nf, 0);
        for (int t = 0; t < nf; ++t)
            if (absorbed[t] >= 0) is_absorbed[absorbed[t]] = 1;
        int next = 0;
        std::vector<std::pair<int, int>> stack;   // (supernode, next child index)
        std::vector<std::vector<int>> kids_ord(nf);
        for (int t = 0; t < nf; ++t) {
            for (int c : f_kids[t])
                if (c != absorbed[t]) kids_ord[t].push_back(c);
            if (absorbed[t] >= 0) kids_ord[t].push_back(absorbed[t]);
        }
        for (int root = 0; root < nf; ++root) {
            if (f_par[root] != -1) continue;
            stack.push_back({root, 0});
            while (!stack.empty()) {
                auto &top = stack.back();
                const int t = top.first;
                if (top.second < (int)kids_ord[t].size()) {
                    const int c = kids_ord[t][top.second++];
                    stack.push_back({c, 0});
                    continue;
                }
                if (!is_absorbed[t]) group_start.push_back(next);
                else if (absorbed[f_par[t]] != t) group_start.push_back(next);
                for (int p = f_first[t]; p < f_first[t + 1]; ++p) new_of_old[p] = next++;
                stack.pop_back();
            }
        }
        if (next != ni) fail("symbolic: postorder incomplete");
        // a group starts at the bottom of its chain: recompute starts from the chains
        std::vector<char> starts(ni + 1, 0);
        for (int t = 0; t < nf; ++t) {
            if (is_absorbed[t]) continue;            // t is the top of a group
            int b = t;
            while (absorbed[b] >= 0) b = absorbed[b];
            starts[new_of_old[f_first[b]]] = 1;
        }
        // relabel positions, structures and the tree
        std::vector<int> order_new(n), old_of_new(ni);
        for (int p = 0; p < ni; ++p) old_of_new[new_of_old[p]] = p;
        for (int q = 0; q < ni; ++q) order_new[q] = out.order[old_of_new[q]];
        for (int q = ni; q < n; ++q) order_new[q] = out.order[q];
        out.order = order_new;
        for (int q = 0; q < n; ++q) out.pos_of[out.order[q]] = q;
        for (int q = 0; q < n; ++q) out.var0[q + 1] = out.var0[q] + sys.nvar[out.order[q]];
        std::vector<std::vector<int>> S2(ni);
        for (int p = 0; p < ni; ++p) {
            for (int q : S[p]) S2[new_of_old[p]].push_back(q < ni ? new_of_old[q] : q);
            std::sort(S2[new_of_old[p]].begin(), S2[new_of_old[p]].end());
        }
        S.swap(S2);
        for (int p = 0; p < ni; ++p) {
            if (!S[p].empty() && S[p][0] <= p) fail("symbolic: postorder broke the structure");
            parent[p] = (!S[p].empty() && S[p][0] < ni) ? S[p][0] : -1;
        }
        for (int p = 0; p < ni; ++p)
            if (starts[p]) sn_first.push_back(p);
        (void)group_start;
    }
    // Supernodes wider than max_panel scalars are cut into consecutive pieces:
    // a piece's structure is the later columns of the supernode plus its rows,
    // so each piece is a valid supernode and the pieces form a chain.
    {
        std::vector<int> cut;
        sn_first.push_back(ni);
        for (size_t g = 0; g + 1 < sn_first.size(); ++g) {
            int p = sn_first[g];
            const int p1 = sn_first[g + 1];
            while (p < p1) {
                cut.push_back(p);
                int wsc = 0, q = p;
                while (q < p1 && wsc + sys.nvar[out.order[q]] <= max_panel) wsc += sys.nvar[out.order[q++]];
                if (q == p) ++q;
                p = q;
            }
        }
        sn_first.swap(cut);
    }
    sn_first.push_back(ni);
    const int nsn = (int)sn_first.size() - 1;
    std::vector<int> bus_sn(ni, -1);
    SymFactor &F = out.F;
    F.n_int = out.var0[ni];
    F.n_bnd = out.var0[n] - out.var0[ni];
    F.var_sn.assign(F.n_int, -1);
    int off = 0;
    for (int s = 0; s < nsn; ++s) {
        int p0 = sn_first[s], p1 = sn_first[s + 1];
        for (int p = p0; p < p1; ++p) bus_sn[p] = s;
        int c0 = out.var0[p0], w = out.var0[p1] - c0;
        F.sn_c0.push_back(c0);
        F.sn_w.push_back(w);
        F.sn_rows.push_back((int)F.rows.size());
        for (int q : S[p1 - 1])
            for (int v = out.var0[q]; v < out.var0[q + 1]; ++v) F.rows.push_back(v);
        int nr = (int)F.rows.size() - F.sn_rows.back();
        F.sn_nr.push_back(nr);
        F.sn_off.push_back(off);
        off += w * (w + nr);
        for (int c = c0; c < c0 + w; ++c) F.var_sn[c] = s;
        F.max_w = std::max(F.max_w, w);
    }
    F.store_int = off;
    F.off_B = off;
    F.store_total = off + F.n_bnd * (F.n_bnd + 1) / 2;

    // --- level schedule of the supernodal elimination tree ---
    std::vector<int> level(nsn, 0);
    for (int s = 0; s < nsn; ++s) {
        int plast = sn_first[s + 1] - 1;
        if (!S[plast].empty() && S[plast][0] < ni) {
            int t = bus_sn[S[plast][0]];
            if (t <= s) fail("symbolic: supernode parent not later");
            level[t] = std::max(level[t], level[s] + 1);
        }
    }
    int nlev = nsn ? *std::max_element(level.begin(), level.end()) + 1 : 0;
    F.sn_order.resize(nsn);
    std::iota(F.sn_order.begin(), F.sn_order.end(), 0);
    std::stable_sort(F.sn_order.begin(), F.sn_order.end(),
                     [&](int a, int b) { return level[a] < level[b]; });
    F.lev_off.assign(nlev + 1, 0);
    for (int s = 0; s < nsn; ++s) ++F.lev_off[level[s] + 1];
    for (int l = 0; l < nlev; ++l) F.lev_off[l + 1] += F.lev_off[l];
    F.lev_items.assign(nlev, 0);
    for (int l = 0; l < nlev; ++l) {
        int acc = 0;
        for (int i = F.lev_off[l]; i < F.lev_off[l + 1]; ++i) {
            long long R = F.sn_nr[F.sn_order[i]];
            acc += (int)(R * (R + 1) / 2 + R);
        }
        F.lev_items[l] = acc;
    }

    // --- update maps: target column base + relative row positions ---
    F.colbase.assign(F.rows.size(), 0);
    F.relbase.assign(F.rows.size(), 0);
    for (int s = 0; s < nsn; ++s) {
        const int R = F.sn_nr[s], rb = F.sn_rows[s], w = F.sn_w[s];
        int cur_t = -2, relstart = 0, seg_j0 = 0;
        for (int j = 0; j < R; ++j) {
            int c = F.rows[rb + j];
            int t = c < F.n_int ? F.var_sn[c] : -1;
            if (t != cur_t) {
                cur_t = t;
                seg_j0 = j;
                relstart = (int)F.rel.size();
                for (int i = j; i < R; ++i) {
                    int r = F.rows[rb + i];
                    if (t >= 0) {
                        int c0t = F.sn_c0[t], wt = F.sn_w[t];
                        int rp;
                        if (r < c0t + wt) {
                            rp = r - c0t;
                        } else {
                            const int *b = F.rows.data() + F.sn_rows[t];
                            const int *e = b + F.sn_nr[t];
                            const int *it = std::lower_bound(b, e, r);
                            if (it == e || *it != r) fail("symbolic: row not in target supernode");
                            rp = wt + (int)(it - b);
                        }
                        F.rel.push_back(rp);
                    } else {
                        F.rel.push_back(r - F.n_int);
                    }
                }
            }
            if (t >= 0) {
                int ld = F.sn_w[t] + F.sn_nr[t];
                F.colbase[rb + j] = F.sn_off[t] + (c - F.sn_c0[t]) * ld;
            } else {
                int cb = c - F.n_int;
                F.colbase[rb + j] = F.off_B + packed_col_start(cb, F.n_bnd) - cb;
            }
            F.relbase[rb + j] = relstart - seg_j0;
        }
        // cost of the supernode: panel factorisation + update of ancestors
        const int ld = w + R;
        for (int c = 0; c < w; ++c)
            for (int c2 = c + 1; c2 < w; ++c2) F.flops += ld - c2;
        F.flops += (long long)w * R * (R + 1) / 2;
        F.pairs += (long long)R * (R + 1) / 2;
    }
    F.lev_chunks.assign(nlev + 1, 0);
    for (int l = 0; l < nlev; ++l) {
        for (int i = F.lev_off[l]; i < F.lev_off[l + 1]; ++i) {
            const int s = F.sn_order[i], w = F.sn_w[s], ld = w + F.sn_nr[s];
            for (int r0 = w; r0 < ld; r0 += 32) {
                const int rec[8] = {F.sn_off[s], w, ld, r0, F.sn_c0[s], F.sn_rows[s], 0, 0};
                F.chunk_rec.insert(F.chunk_rec.end(), rec, rec + 8);
            }
        }
        F.lev_chunks[l + 1] = (int)F.chunk_rec.size() / 8;
    }
    // update units: consecutive target columns of one segment, kUnitCols at most
    F.lev_units.assign(nlev + 1, 0);
    for (int l = 0; l < nlev; ++l) {
        for (int i = F.lev_off[l]; i < F.lev_off[l + 1]; ++i) {
            const int s = F.sn_order[i], R = F.sn_nr[s], rb = F.sn_rows[s];
            for (int j = 0; j < R;) {
                int nj = 1;
                while (nj < kUnitCols && j + nj < R && F.relbase[rb + j + nj] == F.relbase[rb + j]) ++nj;
                F.unit_sn.push_back(s);
                F.unit_j.push_back(j);
                F.unit_nj.push_back(nj);
                j += nj;
            }
        }
        F.lev_units[l + 1] = (int)F.unit_sn.size();
    }
    build_tasks(F, kTaskWarps, level_sched);
    return out;
}

// ---------------------------------------------------------------------------

bool build_setup(const NetIn &net, int K, const int32_t *area_of_bus, Setup &st,
                 int smem_limit) {
    try {
        const int N = net.n_bus, L = net.n_branch;
        if (N < 2 || L < 1) fail("need at least 2 buses and 1 branch");
        if (K < 1 || K > N) fail("n_area out of range");
        if (net.slack < 0 || net.slack >= N) fail("slack bus out of range");
        if (!net.from || !net.to || !net.r || !net.x || !net.bc || !area_of_bus)
            fail("null network or partition array");
        st.N = N;
        st.L = L;
        st.K = K;
        st.slack = net.slack;
        st.m = 3 * N + 4 * L;
        std::vector<std::vector<int>> inc(N);   // incident branches
        for (int l = 0; l < L; ++l) {
            int f = net.from[l], t = net.to[l];
            if (f < 0 || f >= N || t < 0 || t >= N) fail("branch bus index out of range");
            if (f == t) fail("branch with from == to");
            if (!std::isfinite(net.r[l]) || !std::isfinite(net.x[l]) || !std::isfinite(net.bc[l]))
                fail("non-finite branch parameter");
            if (net.r[l] * net.r[l] + net.x[l] * net.x[l] <= 0.0) fail("zero series impedance");
            inc[f].push_back(l);
            inc[t].push_back(l);
        }
        std::vector<int> area(N);
        std::vector<int> count(K, 0);
        for (int b = 0; b < N; ++b) {
            int a = area_of_bus[b];
            if (a < 0 || a >= K) fail("area index out of range");
            area[b] = a;
            ++count[a];
        }
        for (int k = 0; k < K; ++k)
            if (!count[k]) fail("empty area");
        for (int b = 0; b < N; ++b)
            if (inc[b].empty()) fail("isolated bus");
        std::vector<char> bnd(N, 0);
        for (int l = 0; l < L; ++l)
            if (area[net.from[l]] != area[net.to[l]]) bnd[net.from[l]] = bnd[net.to[l]] = 1;
        auto other = [&](int l, int b) { return net.from[l] == b ? net.to[l] : net.from[l]; };
        auto nvar_of = [&](int b) { return b == net.slack ? 1 : 2; };

        // ---------------- pass 1: per-area symbolic factor + internal numbering
        std::vector<std::vector<int>> own(K), lbuses(K), nodes(K);
        for (int b = 0; b < N; ++b) own[area[b]].push_back(b);
        std::vector<SymResult> sym(K);
        std::vector<int> node_of(N, -1);
        st.areas.resize(K);
        st.ibus_of_bus.assign(N, -1);
        int next_ibus = 0;
        for (int k = 0; k < K; ++k) {
            std::vector<int> intern, lb;
            for (int b : own[k]) {
                if (!bnd[b]) intern.push_back(b);
                else lb.push_back(b);
                for (int l : inc[b]) {
                    int o = other(l, b);
                    if (area[o] != k) lb.push_back(o);
                }
            }
            std::sort(lb.begin(), lb.end());
            lb.erase(std::unique(lb.begin(), lb.end()), lb.end());
            std::vector<int> &nd = nodes[k];
            nd = intern;
            nd.insert(nd.end(), lb.begin(), lb.end());
            lbuses[k] = lb;
            for (int i = 0; i < (int)nd.size(); ++i) node_of[nd[i]] = i;
            BusSystem sys;
            sys.nb_int = (int)intern.size();
            sys.nb_bnd = (int)lb.size();
            sys.adj.assign(nd.size(), {});
            sys.nvar.resize(nd.size());
            for (int i = 0; i < (int)nd.size(); ++i) sys.nvar[i] = nvar_of(nd[i]);
            for (int b : own[k]) {
                std::vector<int> cl{node_of[b]};
                for (int l : inc[b]) cl.push_back(node_of[other(l, b)]);
                for (int a : cl)
                    for (int c : cl)
                        if (a != c) sys.adj[a].push_back(c);
            }
            for (auto &v : sys.adj) {
                std::sort(v.begin(), v.end());
                v.erase(std::unique(v.begin(), v.end()), v.end());
            }
            sym[k] = build_symbolic(sys);
            if (smem_limit > 0) {
                int nv = 0, n_ends = 0;
                for (int i = 0; i < (int)nd.size(); ++i) nv += sys.nvar[i];
                for (int b : own[k]) n_ends += (int)inc[b].size();
                const SmemLayout lay = area_smem_layout(nv, (int)nd.size(), n_ends,
                                                        (int)own[k].size(), 4, 4);
                const long long budget =
                    ((long long)smem_limit - (long long)lay.vector_bytes) / 4;
                // less relaxation only when it brings the factor on chip; a factor
                // that stays in global memory keeps the wider panels (fewer tasks)
                if (budget > 0 && sym[k].F.store_total > budget) {
                    SymResult alt = build_symbolic(sys, 0.10, 8);
                    if (alt.F.store_total > budget) alt = build_symbolic(sys, 0.0, 0);
                    if (alt.F.store_total <= budget) sym[k] = std::move(alt);
                }
            }
            for (int i = 0; i < (int)nd.size(); ++i) node_of[nd[i]] = -1;
            // internal numbering: internal buses in elimination order, then own boundary buses
            const int ni = sys.nb_int;
            for (int p = 0; p < ni; ++p) st.ibus_of_bus[nd[sym[k].order[p]]] = next_ibus++;
            for (int p = ni; p < (int)nd.size(); ++p) {
                int b = nd[sym[k].order[p]];
                if (area[b] == k) st.ibus_of_bus[b] = next_ibus++;
            }
        }
        if (next_ibus != N) fail("internal numbering incomplete");
        st.bus_of_ibus.assign(N, -1);
        st.area_of_ibus.assign(N, -1);
        for (int b = 0; b < N; ++b) {
            st.bus_of_ibus[st.ibus_of_bus[b]] = b;
            st.area_of_ibus[st.ibus_of_bus[b]] = area[b];
        }

        // ---------------- boundary system (Sec. 3.2, 4.4)
        std::vector<int> bbus;
        for (int b = 0; b < N; ++b)
            if (bnd[b]) bbus.push_back(b);
        st.n_boundary_bus = (int)bbus.size();
        BoundarySetup &B = st.B;
        B.n_bbus = (int)bbus.size();
        std::vector<int> bnode(N, -1);
        for (int i = 0; i < (int)bbus.size(); ++i) bnode[bbus[i]] = i;
        SymResult bsym;
        if (!bbus.empty()) {
            BusSystem bs;
            bs.nb_int = (int)bbus.size();
            bs.nb_bnd = 0;
            bs.adj.assign(bbus.size(), {});
            bs.nvar.resize(bbus.size());
            for (int i = 0; i < (int)bbus.size(); ++i) bs.nvar[i] = nvar_of(bbus[i]);
            for (int k = 0; k < K; ++k)
                for (int a : lbuses[k])
                    for (int c : lbuses[k])
                        if (a != c) bs.adj[bnode[a]].push_back(bnode[c]);
            for (auto &v : bs.adj) {
                std::sort(v.begin(), v.end());
                v.erase(std::unique(v.begin(), v.end()), v.end());
            }
            bsym = build_symbolic(bs, 0.30, 16, kBoundaryPanel, true);
            B.F = bsym.F;
        }
        B.n_gamma = B.F.n_int;
        // x_Gamma in oracle order: ascending boundary bus, magnitude then angle
        std::vector<int> xg0(bbus.size() + 1, 0);
        for (size_t i = 0; i < bbus.size(); ++i) xg0[i + 1] = xg0[i] + nvar_of(bbus[i]);
        B.bvar_ibus.assign(B.n_gamma, -1);
        B.bvar_isT.assign(B.n_gamma, 0);
        B.xg_of_b.assign(B.n_gamma, -1);
        for (int p = 0; p < (int)bbus.size(); ++p) {
            int node = bsym.order[p];
            int b = bbus[node];
            int v0 = bsym.var0[p];
            B.bvar_ibus[v0] = st.ibus_of_bus[b];
            B.xg_of_b[v0] = xg0[node];
            if (nvar_of(b) == 2) {
                B.bvar_ibus[v0 + 1] = st.ibus_of_bus[b];
                B.bvar_isT[v0 + 1] = 1;
                B.xg_of_b[v0 + 1] = xg0[node] + 1;
            }
        }
        auto bscalar = [&](int b, int isT) {
            int p = bsym.pos_of[bnode[b]];
            return bsym.var0[p] + isT;
        };

        // ---------------- pass 2: templates and slot maps per area
        std::vector<int> locpos(N, -1);
        std::vector<std::vector<int>> asm_lists(B.F.store_total);
        std::vector<std::vector<std::pair<int, int>>> rhs_lists(B.n_gamma);
        int zrow = 0;
        st.zrow_base.assign(K, 0);
        st.zperm.clear();
        st.zperm.reserve(st.m);
        for (int k = 0; k < K; ++k) {
            AreaSetup &A = st.areas[k];
            SymResult &sr = sym[k];
            const std::vector<int> &nd = nodes[k];
            A.k = k;
            A.F = sr.F;
            A.nb_int = (int)nd.size() - (int)lbuses[k].size();
            A.nb_loc = (int)nd.size();
            A.n_int = A.F.n_int;
            A.n_bnd = A.F.n_bnd;
            A.locbus.resize(A.nb_loc);
            A.qvarV.resize(A.nb_loc);
            A.qvarT.resize(A.nb_loc);
            std::vector<int> bus_at(A.nb_loc);
            for (int q = 0; q < A.nb_loc; ++q) {
                int b = nd[sr.order[q]];
                bus_at[q] = b;
                locpos[b] = q;
                A.locbus[q] = st.ibus_of_bus[b];
                A.qvarV[q] = sr.var0[q];
                A.qvarT[q] = (sr.var0[q + 1] - sr.var0[q] == 2) ? sr.var0[q] + 1 : -1;
            }
            // own buses in internal-numbering order
            for (int q = 0; q < A.nb_loc; ++q)
                if (area[bus_at[q]] == k) A.own_q.push_back(q);
            std::sort(A.own_q.begin(), A.own_q.end(),
                      [&](int a, int b) { return A.locbus[a] < A.locbus[b]; });
            A.n_own = (int)A.own_q.size();
            auto gp = [&](int va, int vb) { return (va < 0 || vb < 0) ? -1 : A.F.pos(va, vb); };
            const int G = 0;
            (void)G;
            for (int o = 0; o < A.n_own; ++o) {
                int q = A.own_q[o], b = bus_at[q];
                A.own_ebeg.push_back((int)A.end_qi.size());
                A.own_sbeg.push_back((int)A.slot_q.size());
                int pvv = gp(A.qvarV[q], A.qvarV[q]);
                if (pvv < 0) fail("diagonal slot missing");
                A.own_gvv.push_back(pvv);
                std::vector<int> ls = inc[b];
                std::sort(ls.begin(), ls.end(), [&](int l1, int l2) {
                    int q1 = locpos[other(l1, b)], q2 = locpos[other(l2, b)];
                    return q1 != q2 ? q1 < q2 : l1 < l2;
                });
                int last_q = -1;
                for (int l : ls) {
                    int o2 = other(l, b);
                    int qj = locpos[o2];
                    if (qj < 0) fail("neighbour not local");
                    if (qj != last_q) {
                        A.slot_q.push_back(qj);
                        A.slot_ebeg.push_back((int)A.end_qi.size());
                        A.slot_ecnt.push_back(0);
                        last_q = qj;
                    }
                    ++A.slot_ecnt.back();
                    A.end_qi.push_back(q);
                    A.end_qj.push_back(qj);
                    A.end_own.push_back(o);
                    int v4[4] = {A.qvarV[q], A.qvarT[q], A.qvarV[qj], A.qvarT[qj]};
                    for (int a = 0; a < 4; ++a) A.end_var.push_back(v4[a]);
                    for (int a = 0; a < 4; ++a)
                        for (int c = a; c < 4; ++c) {
                            int p = gp(v4[a], v4[c]);
                            if (v4[a] >= 0 && v4[c] >= 0 && p < 0) fail("flow slot missing");
                            A.end_gpos.push_back(p);
                        }
                    bool is_from = net.from[l] == b;
                    A.end_canon.push_back(is_from ? 3 * N + l : 3 * N + 2 * L + l);
                    double den = net.r[l] * net.r[l] + net.x[l] * net.x[l];
                    A.end_g.push_back(net.r[l] / den);
                    A.end_b.push_back(-net.x[l] / den);
                    A.end_bh.push_back(0.5 * net.bc[l]);
                }
            }
            A.n_ends = (int)A.end_qi.size();
            A.n_slots = (int)A.slot_q.size();
            A.own_ebeg.push_back(A.n_ends);
            A.own_sbeg.push_back(A.n_slots);
            // injection-row gain items over {bus itself, neighbour slots}
            long long gup = A.n_own;
            for (int o = 0; o < A.n_own; ++o) {
                int s0 = A.own_sbeg[o], d = A.own_sbeg[o + 1] - s0;
                auto slot_bus = [&](int u) { return u == 0 ? A.own_q[o] : A.slot_q[s0 + u - 1]; };
                for (int u = 0; u <= d; ++u)
                    for (int v = u; v <= d; ++v) {
                        int qa = slot_bus(u), qb = slot_bus(v);
                        int Va = A.qvarV[qa], Ta = A.qvarT[qa], Vb = A.qvarV[qb], Tb = A.qvarT[qb];
                        int p4[4];
                        if (u == v) {
                            p4[0] = gp(Va, Va);
                            p4[1] = gp(Ta, Va);
                            p4[2] = gp(Ta, Ta);
                            p4[3] = -1;
                        } else {
                            p4[0] = gp(Va, Vb);
                            p4[1] = gp(Va, Tb);
                            p4[2] = gp(Ta, Vb);
                            p4[3] = gp(Ta, Tb);
                        }
                        if (p4[0] < 0) fail("injection slot missing");
                        auto first_end = [&](int u_) { return u_ == 0 ? -1 : A.slot_ebeg[s0 + u_ - 1]; };
                        auto n_end = [&](int u_) { return u_ == 0 ? 0 : A.slot_ecnt[s0 + u_ - 1]; };
                        A.item_rec.push_back(o);
                        A.item_rec.push_back(first_end(u));
                        A.item_rec.push_back(first_end(v));
                        A.item_rec.push_back(n_end(u) | (n_end(v) << 16));
                        A.item_own.push_back(o);
                        A.item_uv.push_back(u | (v << 16));
                        for (int a = 0; a < 4; ++a) {
                            A.item_pos.push_back(p4[a]);
                            if (p4[a] >= 0) ++gup;
                        }
                    }
            }
            for (int p : A.end_gpos)
                if (p >= 0) ++gup;
            A.n_items = (int)A.item_own.size();
            // A warp adds the gain terms of 32 consecutive items with one atomic
            // instruction per slot, and lanes on one address serialise.  Items of
            // different rows that share a gain entry (a bus pair in the
            // injection rows of both buses) are spread over different windows
            // of 32: each window takes, in order, the earliest remaining items
            // whose entries are new to it.
            {
                const int n = A.n_items;
                std::vector<int> order;
                order.reserve(n);
                std::vector<char> placed(n, 0);
                std::vector<int> seen;   // entries of the current window
                int first = 0;
                while ((int)order.size() < n) {
                    seen.clear();
                    int cnt = 0;
                    for (int i = first; i < n && cnt < 32; ++i) {
                        if (placed[i]) continue;
                        const int *p4 = &A.item_pos[4 * (size_t)i];
                        bool clash = false;
                        for (int a = 0; a < 4 && !clash; ++a)
                            if (p4[a] >= 0 && std::find(seen.begin(), seen.end(), p4[a]) != seen.end())
                                clash = true;
                        if (clash) continue;
                        for (int a = 0; a < 4; ++a)
                            if (p4[a] >= 0) seen.push_back(p4[a]);
                        placed[i] = 1;
                        order.push_back(i);
                        ++cnt;
                    }
                    while (first < n && placed[first]) ++first;
                }
                std::vector<int> rec(A.item_rec.size()), own(n), uv(n), pos(A.item_pos.size());
                for (int j = 0; j < n; ++j) {
                    const int i = order[j];
                    for (int a = 0; a < 4; ++a) {
                        rec[4 * (size_t)j + a] = A.item_rec[4 * (size_t)i + a];
                        pos[4 * (size_t)j + a] = A.item_pos[4 * (size_t)i + a];
                    }
                    own[j] = A.item_own[i];
                    uv[j] = A.item_uv[i];
                }
                A.item_rec.swap(rec);
                A.item_own.swap(own);
                A.item_uv.swap(uv);
                A.item_pos.swap(pos);
            }
            A.g_updates = gup;
            // boundary selector E_k (Eq. Ek_select)
            A.ebnd.assign(A.n_bnd, -1);
            A.bnd_xg.assign(A.n_bnd, -1);
            for (int q = A.nb_int; q < A.nb_loc; ++q) {
                int b = bus_at[q];
                int lvV = A.qvarV[q] - A.n_int;
                A.ebnd[lvV] = bscalar(b, 0);
                if (A.qvarT[q] >= 0) A.ebnd[lvV + 1] = bscalar(b, 1);
            }
            for (int lv = 0; lv < A.n_bnd; ++lv) {
                if (A.ebnd[lv] < 0) fail("boundary selector incomplete");
                A.bnd_xg[lv] = B.xg_of_b[A.ebnd[lv]];
            }
            // coordinator gather lists (Eq. global_assembly)
            for (int cb = 0; cb < A.n_bnd; ++cb)
                for (int rb = cb; rb < A.n_bnd; ++rb) {
                    int P = B.F.pos(A.ebnd[rb], A.ebnd[cb]);
                    if (P < 0) fail("boundary slot missing");
                    asm_lists[P].push_back(k);
                    asm_lists[P].push_back(A.F.off_B + packed_col_start(cb, A.n_bnd) + (rb - cb));
                }
            for (int lv = 0; lv < A.n_bnd; ++lv) rhs_lists[A.ebnd[lv]].push_back({k, lv});
            // measurement rows of the area (Sec. 4.1 SoA templates)
            st.zrow_base[k] = zrow;
            for (int o = 0; o < A.n_own; ++o) st.zperm.push_back(bus_at[A.own_q[o]]);
            for (int o = 0; o < A.n_own; ++o) st.zperm.push_back(N + bus_at[A.own_q[o]]);
            for (int o = 0; o < A.n_own; ++o) st.zperm.push_back(2 * N + bus_at[A.own_q[o]]);
            for (int e = 0; e < A.n_ends; ++e) st.zperm.push_back(A.end_canon[e]);
            for (int e = 0; e < A.n_ends; ++e) st.zperm.push_back(A.end_canon[e] + L);
            zrow += 3 * A.n_own + 2 * A.n_ends;
            A.work = A.F.flops + 40LL * A.n_ends + A.g_updates;
            for (int q = 0; q < A.nb_loc; ++q) locpos[bus_at[q]] = -1;
        }
        if (zrow != st.m || (int)st.zperm.size() != st.m) fail("measurement rows incomplete");
        {
            std::vector<char> seen(st.m, 0);
            for (int r : st.zperm) {
                if (r < 0 || r >= st.m || seen[r]) fail("measurement row permutation invalid");
                seen[r] = 1;
            }
        }
        B.asm_beg.assign(B.F.store_total + 1, 0);
        for (int P = 0; P < B.F.store_total; ++P) {
            B.asm_beg[P + 1] = B.asm_beg[P] + (int)asm_lists[P].size() / 2;
            for (size_t i = 0; i < asm_lists[P].size(); i += 2) {
                B.asm_area.push_back(asm_lists[P][i]);
                B.asm_off.push_back(asm_lists[P][i + 1]);
            }
        }
        B.rhs_beg.assign(B.n_gamma + 1, 0);
        for (int g = 0; g < B.n_gamma; ++g) {
            B.rhs_beg[g + 1] = B.rhs_beg[g] + (int)rhs_lists[g].size();
            if (rhs_lists[g].empty()) fail("boundary unknown without an area");
            for (auto &pr : rhs_lists[g]) {
                B.rhs_area.push_back(pr.first);
                B.rhs_lv.push_back(pr.second);
            }
        }
    } catch (const std::exception &e) {
        st.error = e.what();
        return false;
    }
    return true;
}

}  // namespace mase

// ---------------------------------------------------------------------------
// Host self-check of the symbolic setup (no GPU): scatter random gain terms
// through the slot maps exactly as the device accumulation does, check them
// against a dense assembly, run the supernodal schedule serially and compare
// the Schur block and the solves with dense Cholesky results.
// ---------------------------------------------------------------------------
namespace mase {
namespace {

struct Rng {
    unsigned long long s;
    double next() {   // splitmix64 -> [0, 1)
        unsigned long long z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    }
    double sym() { return 2.0 * next() - 1.0; }
};

// one task of the dataflow factorisation, as the device runs it
void host_task(const SymFactor &F, const int *r, std::vector<double> &st, std::vector<double> &y) {
    const int type = r[0] >> 24;
    if (type == 0) {
        const int w = r[5], ld = r[6];
        double *P = st.data() + r[4];
        double *yc = y.data() + r[7];
        for (int c = 0; c < w; ++c) {
            double *col = P + (size_t)c * ld;
            double d = col[c];
            if (!(d > 0)) throw std::runtime_error("selfcheck: non-positive pivot");
            d = std::sqrt(d);
            for (int r2 = c + 1; r2 < w; ++r2) col[r2] /= d;
            col[c] = 1.0 / d;   // diagonal kept as its reciprocal, as on the device
            for (int c2 = c + 1; c2 < w; ++c2)
                for (int r2 = c2; r2 < w; ++r2) P[(size_t)c2 * ld + r2] -= col[r2] * col[c2];
        }
        for (int c = 0; c < w; ++c) {
            yc[c] *= P[(size_t)c * ld + c];
            for (int r2 = c + 1; r2 < w; ++r2) yc[r2] -= P[(size_t)c * ld + r2] * yc[c];
        }
    } else if (type == 1) {
        const int w = r[5], ld = r[6], r0 = r[7];
        double *P = st.data() + r[4];
        for (int row = r0; row < std::min(ld, r0 + 32); ++row)
            for (int c = 0; c < w; ++c) {
                double v = P[(size_t)c * ld + row];
                for (int k = 0; k < c; ++k) v -= P[(size_t)k * ld + row] * P[(size_t)k * ld + c];
                P[(size_t)c * ld + row] = v * P[(size_t)c * ld + c];
            }
    } else {
        const double *Ps = st.data() + r[4];
        const int *relp = F.rel.data() + r[5];
        const int rb = r[6], c0 = r[7], w = r[8] & 0xff, nj = r[8] >> 8, ld = r[9] & 0xffff,
                  j0 = r[9] >> 16, rhs_end = r[10];
        const int R = ld - w;
        for (int ir = j0; ir < R; ++ir) {
            for (int k = 0; k < nj; ++k) {
                const int jr = j0 + k;
                if (ir < jr) continue;
                double v = 0;
                for (int c = 0; c < w; ++c) v += Ps[(size_t)c * ld + ir] * Ps[(size_t)c * ld + jr];
                st[r[11 + k] + relp[ir]] -= v;
            }
            if (ir < rhs_end) {
                double vr = 0;
                for (int c = 0; c < w; ++c) vr += Ps[(size_t)c * ld + ir] * y[c0 + c];
                y[F.rows[rb + ir]] -= vr;
            }
        }
    }
}

// Emulation of the device schedules.  Factorisation: warps take tasks in list
// order and run one whose wait condition holds; the emulation keeps a window
// of kTaskWarps taken tasks and completes a pseudo-random ready one at a time,
// so a missing dependency shows up as a wrong result or as a stall.
void host_factor(const SymFactor &F, std::vector<double> &st, std::vector<double> &y, bool factor,
                 unsigned long long seed = 1) {
    if (factor && F.level_sched) {
        // each group (level, task kind) in a pseudo-random order
        unsigned long long rs = seed;
        for (size_t g = 0; g + 1 < F.lev_tasks.size(); ++g) {
            std::vector<int> grp;
            for (int t = F.lev_tasks[g]; t < F.lev_tasks[g + 1]; ++t) grp.push_back(t);
            for (size_t i = grp.size(); i > 1; --i) {
                rs = rs * 6364136223846793005ull + 1442695040888963407ull;
                std::swap(grp[i - 1], grp[(rs >> 33) % i]);
            }
            for (int t : grp) host_task(F, F.tasks.data() + (size_t)t * 16, st, y);
        }
        return;
    }
    if (factor) {
        const int nsn = F.nsn();
        std::vector<int> ctr(2 * (size_t)nsn, 0);
        std::vector<int> window;
        int next = 0;
        unsigned long long rs = seed;
        auto rnd = [&rs]() {
            rs = rs * 6364136223846793005ull + 1442695040888963407ull;
            return (unsigned)(rs >> 33);
        };
        while (next < F.n_tasks || !window.empty()) {
            while ((int)window.size() < kTaskWarps && next < F.n_tasks) window.push_back(next++);
            std::vector<int> ok;
            for (size_t i = 0; i < window.size(); ++i) {
                const int *r = F.tasks.data() + (size_t)window[i] * 16;
                if (ctr[r[1]] >= r[2]) ok.push_back((int)i);
            }
            if (ok.empty()) throw std::runtime_error("selfcheck: task schedule deadlocks");
            const int pick = ok[rnd() % ok.size()];
            const int *r = F.tasks.data() + (size_t)window[pick] * 16;
            host_task(F, r, st, y);
            if (r[3] >= 0) ++ctr[r[3]];
            window.erase(window.begin() + pick);
        }
        return;
    }
    for (int lev = 0; lev < F.nlev(); ++lev) {
        for (int i = F.lev_off[lev]; i < F.lev_off[lev + 1]; ++i) {
            const int s = F.sn_order[i], w = F.sn_w[s], R = F.sn_nr[s], ld = w + R;
            const double *P = st.data() + F.sn_off[s];
            double *yc = y.data() + F.sn_c0[s];
            for (int c = 0; c < w; ++c) {
                yc[c] *= P[(size_t)c * ld + c];
                for (int r = c + 1; r < w; ++r) yc[r] -= P[(size_t)c * ld + r] * yc[c];
            }
        }
        for (int i = F.lev_off[lev]; i < F.lev_off[lev + 1]; ++i) {
            const int s = F.sn_order[i], w = F.sn_w[s], R = F.sn_nr[s], ld = w + R;
            const double *Ps = st.data() + F.sn_off[s] + w;
            const int rb = F.sn_rows[s];
            for (int ir = 0; ir < R; ++ir) {
                double v = 0;
                for (int c = 0; c < w; ++c) v += Ps[(size_t)c * ld + ir] * y[F.sn_c0[s] + c];
                y[F.rows[rb + ir]] -= v;
            }
        }
    }
}

void host_back(const SymFactor &F, const std::vector<double> &st, std::vector<double> &y) {
    for (int lev = F.nlev() - 1; lev >= 0; --lev)
        for (int i = F.lev_off[lev]; i < F.lev_off[lev + 1]; ++i) {
            const int s = F.sn_order[i], w = F.sn_w[s], R = F.sn_nr[s], ld = w + R, c0 = F.sn_c0[s];
            const double *P = st.data() + F.sn_off[s];
            for (int c = 0; c < w; ++c)
                for (int ir = 0; ir < R; ++ir) y[c0 + c] -= P[(size_t)c * ld + w + ir] * y[F.rows[F.sn_rows[s] + ir]];
            for (int c = w - 1; c >= 0; --c) {
                for (int r = c + 1; r < w; ++r) y[c0 + c] -= P[(size_t)c * ld + r] * y[c0 + r];
                y[c0 + c] *= P[(size_t)c * ld + c];
            }
        }
}

// dense Cholesky in place (lower, row-major n x n); returns false if not SPD
bool dense_chol(std::vector<double> &A, int n) {
    for (int j = 0; j < n; ++j) {
        double d = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
        if (!(d > 0)) return false;
        d = std::sqrt(d);
        A[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double v = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) v -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
            A[(size_t)i * n + j] = v / d;
        }
    }
    return true;
}
void dense_solve(const std::vector<double> &Lc, int n, std::vector<double> &b) {
    for (int i = 0; i < n; ++i) {
        for (int k = 0; k < i; ++k) b[i] -= Lc[(size_t)i * n + k] * b[k];
        b[i] /= Lc[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        for (int k = i + 1; k < n; ++k) b[i] -= Lc[(size_t)k * n + i] * b[k];
        b[i] /= Lc[(size_t)i * n + i];
    }
}

double rel_err(const std::vector<double> &a, const std::vector<double> &b) {
    double num = 0, den = 0;
    for (size_t i = 0; i < a.size(); ++i) {
        num = std::max(num, std::fabs(a[i] - b[i]));
        den = std::max(den, std::fabs(b[i]));
    }
    return den > 0 ? num / den : num;
}

// factor a dense SPD matrix given in full (nv x nv) through symbolic factor F;
// returns max relative errors of (Schur block, full solve)
void check_system(const SymFactor &F, const std::vector<double> &Gd, const std::vector<double> &st0,
                  Rng &rng, double &e_schur, double &e_solve) {
    const int ni = F.n_int, nb = F.n_bnd, nv = ni + nb;
    std::vector<double> st = st0, y(nv, 0.0);
    host_factor(F, st, y, true);
    // dense Schur: S = G_bb - G_bi G_ii^{-1} G_ib
    std::vector<double> Gii((size_t)ni * ni);
    for (int i = 0; i < ni; ++i)
        for (int j = 0; j < ni; ++j) Gii[(size_t)i * ni + j] = Gd[(size_t)i * nv + j];
    if (!dense_chol(Gii, ni)) throw std::runtime_error("selfcheck: dense G_ii not SPD");
    if (nb) {
        std::vector<double> Sd((size_t)nb * nb), Sg((size_t)nb * nb);
        for (int c = 0; c < nb; ++c) {
            std::vector<double> col(ni);
            for (int i = 0; i < ni; ++i) col[i] = Gd[(size_t)i * nv + ni + c];
            if (ni) dense_solve(Gii, ni, col);
            for (int r = 0; r < nb; ++r) {
                double v = Gd[(size_t)(ni + r) * nv + ni + c];
                for (int i = 0; i < ni; ++i) v -= Gd[(size_t)(ni + r) * nv + i] * col[i];
                Sd[(size_t)r * nb + c] = v;
            }
        }
        for (int c = 0; c < nb; ++c)
            for (int r = 0; r < nb; ++r) {
                int rr = std::max(r, c), cc = std::min(r, c);
                Sg[(size_t)r * nb + c] = st[F.pos(ni + rr, ni + cc)];
            }
        e_schur = std::max(e_schur, rel_err(Sg, Sd));
    }
    // full solve with a random rhs: internal elimination, then the boundary part densely
    std::vector<double> b(nv);
    for (auto &v : b) v = rng.sym();
    std::vector<double> yy = b;
    std::vector<double> st2 = st0;
    host_factor(F, st2, yy, true);
    if (nb) {
        std::vector<double> Sb((size_t)nb * nb);
        for (int r = 0; r < nb; ++r)
            for (int c = 0; c < nb; ++c) Sb[(size_t)r * nb + c] = st2[F.pos(ni + std::max(r, c), ni + std::min(r, c))];
        if (!dense_chol(Sb, nb)) throw std::runtime_error("selfcheck: Schur block not SPD");
        std::vector<double> xb(yy.begin() + ni, yy.end());
        dense_solve(Sb, nb, xb);
        for (int r = 0; r < nb; ++r) yy[ni + r] = xb[r];
    }
    host_back(F, st2, yy);
    std::vector<double> Gfull = Gd;
    if (!dense_chol(Gfull, nv)) throw std::runtime_error("selfcheck: dense G not SPD");
    std::vector<double> xd = b;
    dense_solve(Gfull, nv, xd);
    e_solve = std::max(e_solve, rel_err(yy, xd));
}

}  // namespace

bool selfcheck(const Setup &S, unsigned long long seed, double out[4], std::string &err) {
    try {
        Rng rng{seed};
        double e_slot = 0, e_schur = 0, e_solve = 0, e_bnd = 0;
        for (const AreaSetup &A : S.areas) {
            const SymFactor &F = A.F;
            const int nv = F.n_int + F.n_bnd;
            std::vector<double> Gd((size_t)nv * nv, 0.0), st(F.store_total, 0.0);
            auto addd = [&](int a, int b, double v) {
                if (a < 0 || b < 0) return;
                Gd[(size_t)a * nv + b] += v;
                if (a != b) Gd[(size_t)b * nv + a] += v;
            };
            // voltage rows
            for (int o = 0; o < A.n_own; ++o) {
                double w = 0.5 + rng.next();
                st[A.own_gvv[o]] += w;
                addd(A.qvarV[A.own_q[o]], A.qvarV[A.own_q[o]], w);
            }
            std::vector<double> dPe(4 * A.n_ends), dQe(4 * A.n_ends);
            for (int e = 0; e < A.n_ends; ++e) {
                double dP[4], dQ[4];
                for (int a = 0; a < 4; ++a) {
                    dP[a] = rng.sym();
                    dQ[a] = rng.sym();
                    dPe[4 * e + a] = dP[a];
                    dQe[4 * e + a] = dQ[a];
                }
                double wp = 0.5 + rng.next(), wq = 0.5 + rng.next();
                const int *v = &A.end_var[4 * e];
                int idx = 0;
                for (int a = 0; a < 4; ++a)
                    for (int c = a; c < 4; ++c, ++idx) {
                        double val = wp * dP[a] * dP[c] + wq * dQ[a] * dQ[c];
                        int p = A.end_gpos[10 * e + idx];
                        if (p >= 0) st[p] += val;
                        if (v[a] >= 0 && v[c] >= 0) addd(std::max(v[a], v[c]), std::min(v[a], v[c]), val);
                    }
            }
            // injection rows: h = self part + neighbour parts of the bus's ends
            std::vector<double> wP(A.n_own), wQ(A.n_own);
            for (int o = 0; o < A.n_own; ++o) {
                wP[o] = 0.5 + rng.next();
                wQ[o] = 0.5 + rng.next();
                std::vector<double> hP(nv, 0.0), hQ(nv, 0.0);
                for (int e = A.own_ebeg[o]; e < A.own_ebeg[o + 1]; ++e) {
                    const int *v = &A.end_var[4 * e];
                    for (int a = 0; a < 4; ++a)
                        if (v[a] >= 0) {
                            hP[v[a]] += dPe[4 * e + a];
                            hQ[v[a]] += dQe[4 * e + a];
                        }
                }
                for (int a = 0; a < nv; ++a)
                    if (hP[a] != 0 || hQ[a] != 0)
                        for (int b = 0; b <= a; ++b) {
                            double val = wP[o] * hP[a] * hP[b] + wQ[o] * hQ[a] * hQ[b];
                            if (val != 0) addd(a, b, val);
                        }
            }
            for (int it = 0; it < A.n_items; ++it) {
                const int o = A.item_own[it], u = A.item_uv[it] & 0xffff, v = A.item_uv[it] >> 16;
                const int sb = A.own_sbeg[o];
                double pu[4], pv[4];
                for (int t = 0; t < 2; ++t) {
                    int sl = t == 0 ? u : v;
                    double *dst = t == 0 ? pu : pv;
                    for (int a = 0; a < 4; ++a) dst[a] = 0;
                    if (sl == 0) {
                        for (int e = A.own_ebeg[o]; e < A.own_ebeg[o + 1]; ++e) {
                            dst[0] += dPe[4 * e + 0];
                            dst[1] += dPe[4 * e + 1];
                            dst[2] += dQe[4 * e + 0];
                            dst[3] += dQe[4 * e + 1];
                        }
                    } else {
                        int ss = sb + sl - 1;
                        for (int e = A.slot_ebeg[ss]; e < A.slot_ebeg[ss] + A.slot_ecnt[ss]; ++e) {
                            dst[0] += dPe[4 * e + 2];
                            dst[1] += dPe[4 * e + 3];
                            dst[2] += dQe[4 * e + 2];
                            dst[3] += dQe[4 * e + 3];
                        }
                    }
                }
                const int *p4 = &A.item_pos[4 * it];
                double wp = wP[o], wq = wQ[o];
                if (u == v) {
                    st[p4[0]] += wp * pu[0] * pu[0] + wq * pu[2] * pu[2];
                    if (p4[1] >= 0) st[p4[1]] += wp * pu[1] * pu[0] + wq * pu[3] * pu[2];
                    if (p4[2] >= 0) st[p4[2]] += wp * pu[1] * pu[1] + wq * pu[3] * pu[3];
                } else {
                    st[p4[0]] += wp * pu[0] * pv[0] + wq * pu[2] * pv[2];
                    if (p4[1] >= 0) st[p4[1]] += wp * pu[0] * pv[1] + wq * pu[2] * pv[3];
                    if (p4[2] >= 0) st[p4[2]] += wp * pu[1] * pv[0] + wq * pu[3] * pv[2];
                    if (p4[3] >= 0) st[p4[3]] += wp * pu[1] * pv[1] + wq * pu[3] * pv[3];
                }
            }
            // every dense entry must sit at its storage slot with the same value
            double scale = 0;
            for (double v : Gd) scale = std::max(scale, std::fabs(v));
            for (int c = 0; c < nv; ++c)
                for (int r = c; r < nv; ++r) {
                    double d = Gd[(size_t)r * nv + c];
                    int p = F.pos(r, c);
                    if (p < 0) {
                        if (d != 0) throw std::runtime_error("selfcheck: gain entry outside the pattern");
                        continue;
                    }
                    e_slot = std::max(e_slot, std::fabs(st[p] - d) / scale);
                }
            // make it comfortably SPD (diagonal shift) in both copies
            for (int i = 0; i < nv; ++i) {
                Gd[(size_t)i * nv + i] += 4.0 * scale;
                st[F.pos(i, i)] += 4.0 * scale;
            }
            check_system(F, Gd, st, rng, e_schur, e_solve);
        }
        // boundary system: random SPD blocks per area scattered through the gather lists
        const BoundarySetup &B = S.B;
        if (B.n_gamma > 0) {
            const int nG = B.n_gamma;
            std::vector<std::vector<double>> Sk(S.areas.size());
            for (size_t k = 0; k < S.areas.size(); ++k) {
                const AreaSetup &A = S.areas[k];
                Sk[k].assign(A.F.store_total, 0.0);
                for (int c = 0; c < A.n_bnd; ++c)
                    for (int r = c; r < A.n_bnd; ++r)
                        Sk[k][A.F.pos(A.n_int + r, A.n_int + c)] = rng.sym() + (r == c ? 2.0 * A.n_bnd : 0.0);
            }
            std::vector<double> st(B.F.store_total, 0.0), Sd((size_t)nG * nG, 0.0);
            for (int P = 0; P < B.F.store_total; ++P)
                for (int i = B.asm_beg[P]; i < B.asm_beg[P + 1]; ++i) st[P] += Sk[B.asm_area[i]][B.asm_off[i]];
            for (size_t k = 0; k < S.areas.size(); ++k) {
                const AreaSetup &A = S.areas[k];
                for (int c = 0; c < A.n_bnd; ++c)
                    for (int r = c; r < A.n_bnd; ++r) {
                        double v = Sk[k][A.F.pos(A.n_int + r, A.n_int + c)];
                        int gr = A.ebnd[r], gc = A.ebnd[c];
                        Sd[(size_t)gr * nG + gc] += v;
                        if (gr != gc) Sd[(size_t)gc * nG + gr] += v;
                    }
            }
            double sb = 0, dummy = 0;
            check_system(B.F, Sd, st, rng, dummy, sb);
            e_bnd = sb;
        }
        out[0] = e_slot;
        out[1] = e_schur;
        out[2] = e_solve;
        out[3] = e_bnd;
    } catch (const std::exception &e) {
        err = e.what();
        return false;
    }
    return true;
}

}  // namespace mase
