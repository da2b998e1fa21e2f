// symbolic.cpp -- host symbolic analysis: ordering, assembly tree, fronts, maps, schedule.
//
// Ordering.  The Hilbert-space graph of Eq. 1 (vertices = basis states, edges = the spin
// exchanges of antiparallel neighbours) is expander-like, with coordination ~ L (the
// Hilbert-space-graph paragraph of arXiv:1411.0660).  Generic minimum degree leaves a root front
// of about a third of the sector.  This build instead uses nested dissection with separators
// taken from the physics: the weighted magnetization
//     f_k(s) = sum_i w_k(i) n_i(s),   w_k(i) = cos(2 pi k i / L) or sin(2 pi k i / L)
// changes by at most D_k = 2 sin(pi k / L) under one exchange across a bond, so the states with
// f_k in a band [m, m + D_k) separate {f_k < m} from {f_k >= m + D_k}.  (On this graph the f_k are
// exact eigenvectors of the graph Laplacian, with eigenvalue 2 - 2 cos(2 pi k / L): k = 1 is the
// spectral-bisection direction of the whole sector.)  Two separator rules:
//   MBL_ORDER_BAND: the band itself, with the mode chosen from the two numbered depth and
//     depth + 1.
//   MBL_ORDER_MODES: every mode k <= L/2 is tried, and the band of least cost near the median
//     (cost |S| + 0.3 ||V1| - |V2||) over all of them is taken.  A subgraph already split along one
//     mode can then be split along an orthogonal one (the band rule re-splits a depth-1 subgraph
//     along the sine mode that depth 0 used).  At L = 18: 27% less fill, 43% fewer flops.
//   MBL_ORDER_AUTO (default): MODES for sectors of dimension >= 40000, BAND below (at L = 16 the
//     saving is small and the factorization is bound by its per-level launch chain).
//   MBL_ORDER_HYBRID: COVER on subgraphs of at least HYBRID_COVER_MIN vertices, where the
//     separators set the fill, MODES below, where the covers would leave single-column leaves.
//   MBL_ORDER_COVER: every mode k <= L/2 is ranked by its best band near the median
//     (cost |S| + 0.3 ||V1| - |V2||); for the three best, the separator is the minimum vertex
//     cover of the edges crossing the band's midpoint (Koenig's theorem on a maximum bipartite
//     matching), and the cheapest cover is kept.  A cover is never larger than the band, and
//     searching all modes lets a subgraph already split along one mode be split along an
//     orthogonal one.  At L = 18 this needs 40% less fill and 58% fewer flops, but the covers
//     leave about twice as many single-column supernodes, whose pivots in-panel pivoting cannot
//     choose, and its unrefined factor has a heavier tail of element growth.
// The separator is then thinned (a separator vertex with no neighbour on one side moves to the
// other side), and the two halves are dissected recursively.  Subgraphs of at most LEAF vertices
// are ordered by minimum degree.
//
// Symbolic factorization.  Elimination tree (Liu), postorder, column counts (Gilbert, Ng and Peyton),
// fundamental supernodes, relaxed amalgamation, and supernodal row structures by merging the
// children's update rows.
#include <algorithm>
#include <map>
#include <chrono>
#include <cmath>
#include <numeric>
#include <exception>
#include <system_error>
#include <thread>

#include "plan.h"

namespace mbl {

namespace {

constexpr int LEAF = 64;
constexpr int HYBRID_COVER_MIN = 2000;  // MBL_ORDER_HYBRID: cover separators on subgraphs this large

struct Graph {
    int64_t n;
    const std::vector<int64_t> *rowptr;
    const std::vector<int32_t> *col;
};

// Minimum degree on a small induced subgraph (<= 64 vertices, bitset elimination graph).
void md_leaf(const Graph &g, const std::vector<int32_t> &V, std::vector<int32_t> &pos_in, std::vector<int32_t> &out) {
    int k = (int)V.size();
    for (int a = 0; a < k; ++a) pos_in[V[a]] = a;
    std::vector<uint64_t> adj(k, 0);
    for (int a = 0; a < k; ++a) {
        int32_t v = V[a];
        for (int64_t e = (*g.rowptr)[v]; e < (*g.rowptr)[v + 1]; ++e) {
            int32_t u = (*g.col)[e];
            int b = pos_in[u];
            if (b >= 0 && b != a) adj[a] |= 1ull << b;
        }
    }
    uint64_t alive = (k == 64) ? ~0ull : ((1ull << k) - 1);
    for (int t = 0; t < k; ++t) {
        int best = -1, bd = 1 << 30;
        for (int a = 0; a < k; ++a)
            if ((alive >> a) & 1) {
                int d = __builtin_popcountll(adj[a] & alive);
                if (d < bd) { bd = d; best = a; }
            }
        uint64_t N = adj[best] & alive & ~(1ull << best);
        for (int a = 0; a < k; ++a)
            if ((N >> a) & 1) adj[a] |= N & ~(1ull << a);
        alive &= ~(1ull << best);
        out.push_back(V[best]);
    }
    for (int a = 0; a < k; ++a) pos_in[V[a]] = -1;
}

struct ND {
    const Graph &g;
    int L;
    const std::vector<uint32_t> &states;
    int ordering;
    std::vector<std::vector<double>> w;  // modes: k = 1..L, cosine then sine
    std::vector<double> D;
    std::vector<int8_t> part;            // scratch membership: 0 none, 1 V1, 2 V2, 3 S
    std::vector<int32_t> pos_in;
    std::vector<int32_t> order;

    ND(const Graph &g_, int L_, const std::vector<uint32_t> &st, int ordering_)
        : g(g_), L(L_), states(st), ordering(ordering_) {
        for (int k = 1; k <= L; ++k) {
            std::vector<double> c(L), s(L);
            for (int i = 0; i < L; ++i) {
                c[i] = std::cos(2.0 * M_PI * k * i / L);
                s[i] = std::sin(2.0 * M_PI * k * i / L);
            }
            double d = 2.0 * std::sin(M_PI * k / L);
            w.push_back(c); D.push_back(d);
            w.push_back(s); D.push_back(d);
        }
        part.assign(g.n, 0);
        pos_in.assign(g.n, -1);
    }

    double fval(int mode, uint32_t s) const {
        double f = 0.0;
        const std::vector<double> &wm = w[mode];
        for (int i = 0; i < L; ++i)
            if ((s >> i) & 1u) f += wm[i];
        return f;
    }

    // Band of least cost |S| + 0.3 ||V1| - |V2|| for one mode, over bands starting near the 30% to
    // 70% quantiles of f on V.  Returns the cost (1e300: no band splits V) and the band start m.
    double best_band(const std::vector<int32_t> &V, int mode, double &m_out) const {
        const int N = (int)V.size();
        std::vector<double> fs(N);
        for (int a = 0; a < N; ++a) fs[a] = fval(mode, states[V[a]]);
        std::sort(fs.begin(), fs.end());
        const double Dm = D[mode];
        double best = 1e300;
        for (int qi = 0; qi <= 40; ++qi) {
            double q = 0.3 + 0.01 * qi;
            double m = fs[(size_t)(q * (N - 1))] - 0.5 * Dm;
            int64_t n1 = std::lower_bound(fs.begin(), fs.end(), m - 1e-12) - fs.begin();
            int64_t nS = (std::lower_bound(fs.begin(), fs.end(), m + Dm - 1e-12) - fs.begin()) - n1;
            int64_t n2 = N - n1 - nS;
            double cost = (double)nS + 0.3 * (double)std::llabs(n1 - n2);
            if (n1 == 0 || n2 == 0) cost = 1e300;
            if (cost < best) { best = cost; m_out = m; }
        }
        return best;
    }

    // Minimum vertex separator drawn from the edges that cross a threshold: with V split into
    // A = {f < t} and B = {f >= t}, the crossing edges form a bipartite graph, and a minimum vertex
    // cover of it (Koenig's theorem: from a maximum matching, Hopcroft-Karp) removes every edge
    // between A and B.  Sets cov[a] = 1 for the cover and returns its size.  pos_in must hold the
    // local index of each vertex of V.
    int64_t min_cover(const std::vector<int32_t> &V, const std::vector<double> &fv, double t, std::vector<char> &cov) const {
        const int N = (int)V.size();
        std::vector<int32_t> rid(N, -1), Lv, Rv;
        std::vector<int64_t> ap{0};
        std::vector<int32_t> adj;
        for (int a = 0; a < N; ++a) {
            if (!(fv[a] < t)) continue;
            const int32_t v = V[a];
            const size_t before = adj.size();
            for (int64_t e = (*g.rowptr)[v]; e < (*g.rowptr)[v + 1]; ++e) {
                const int32_t b = pos_in[(*g.col)[e]];
                if (b < 0 || fv[b] < t) continue;
                if (rid[b] < 0) { rid[b] = (int32_t)Rv.size(); Rv.push_back(b); }
                adj.push_back(rid[b]);
            }
            if (adj.size() > before) { Lv.push_back(a); ap.push_back((int64_t)adj.size()); }
        }
        const int nl = (int)Lv.size(), nr = (int)Rv.size();
        std::vector<int32_t> mL(nl, -1), mR(nr, -1), dist(nl), q, stk;
        std::vector<int64_t> it(nl);
        for (;;) {
            // breadth-first layers from the free left vertices along alternating paths
            q.clear();
            bool found = false;
            for (int u = 0; u < nl; ++u) {
                dist[u] = mL[u] < 0 ? 0 : -1;
                if (mL[u] < 0) q.push_back(u);
            }
            for (size_t h = 0; h < q.size(); ++h) {
                const int u = q[h];
                for (int64_t e = ap[u]; e < ap[u + 1]; ++e) {
                    const int w2 = mR[adj[e]];
                    if (w2 < 0) found = true;
                    else if (dist[w2] < 0) { dist[w2] = dist[u] + 1; q.push_back(w2); }
                }
            }
            if (!found) break;
            // layered depth-first augmentation, iterative; dist strictly increases along the stack
            for (int u = 0; u < nl; ++u) it[u] = ap[u];
            for (int s0 = 0; s0 < nl; ++s0) {
                if (mL[s0] >= 0) continue;
                stk.assign(1, s0);
                while (!stk.empty()) {
                    const int u = stk.back();
                    if (it[u] == ap[u + 1]) { dist[u] = -1; stk.pop_back(); continue; }
                    const int w2 = mR[adj[it[u]]];
                    if (w2 < 0) {
                        for (int k = (int)stk.size() - 1; k >= 0; --k) {
                            const int uu = stk[k], rr = adj[it[uu]];
                            mL[uu] = rr;
                            mR[rr] = uu;
                        }
                        break;
                    }
                    if (dist[w2] == dist[u] + 1) stk.push_back(w2);
                    else ++it[u];
                }
            }
        }
        // Koenig: Z = vertices reached from free left vertices by alternating paths; the cover is
        // the left vertices outside Z and the right vertices inside it
        std::vector<char> zL(nl, 0), zR(nr, 0);
        q.clear();
        for (int u = 0; u < nl; ++u)
            if (mL[u] < 0) { zL[u] = 1; q.push_back(u); }
        for (size_t h = 0; h < q.size(); ++h) {
            const int u = q[h];
            for (int64_t e = ap[u]; e < ap[u + 1]; ++e) {
                const int r = adj[e];
                if (zR[r]) continue;
                zR[r] = 1;
                const int w2 = mR[r];
                if (w2 >= 0 && !zL[w2]) { zL[w2] = 1; q.push_back(w2); }
            }
        }
        cov.assign(N, 0);
        int64_t c = 0;
        for (int u = 0; u < nl; ++u)
            if (!zL[u]) { cov[Lv[u]] = 1; ++c; }
        for (int r = 0; r < nr; ++r)
            if (zR[r]) { cov[Rv[r]] = 1; ++c; }
        return c;
    }

    // part[] of the band [m, m + D) of one mode: 1 below it (V1), 3 inside (S), 2 above (V2).
    void assign_band(const std::vector<int32_t> &V, int mode, double m) {
        const double Dm = D[mode];
        for (int32_t v : V) {
            const double f = fval(mode, states[v]);
            part[v] = f < m - 1e-12 ? 1 : (f < m + Dm - 1e-12 ? 3 : 2);
        }
    }

    // Split V into part[] = 1 (V1), 2 (V2), 3 (S).  Returns false if no mode splits V.
    bool split_band(const std::vector<int32_t> &V, int depth) {
        double best_cost = 1e300, best_m = 0.0;
        int best_mode = -1;
        for (int cand = 0; cand < 2; ++cand) {
            const int mode = std::min<int>(depth + cand, (int)w.size() - 1);
            double m = 0.0;
            const double cost = best_band(V, mode, m);
            if (cost < best_cost) { best_cost = cost; best_m = m; best_mode = mode; }
        }
        if (best_mode < 0) return false;
        assign_band(V, best_mode, best_m);
        return true;
    }

    bool split_modes(const std::vector<int32_t> &V, bool cover) {
        // modes k = 1..L/2 (k and L - k give the same functions up to sign): rank them by their
        // best band; then either take the best band, or refine the three best by a minimum cover at
        // the band's midpoint
        const int N = (int)V.size();
        const int nmodes = 2 * (L / 2);
        std::vector<std::pair<double, int>> rank;
        std::vector<double> mstart(nmodes, 0.0), cost(nmodes, 1e300);
        // the modes are independent (best_band only reads): large subgraphs spread them over threads.
        // A thread that cannot be started leaves its stride to the calling thread; an exception in
        // a worker (host memory) is carried back and rethrown after every worker has joined.
        const int nt = N >= 1024 ? std::min<int>(nmodes, std::max(1, (int)std::thread::hardware_concurrency())) : 1;
        std::vector<std::exception_ptr> err(nt);
        auto some_modes = [&](int m0) {
            try {
                for (int mode = m0; mode < nmodes; mode += nt) cost[mode] = best_band(V, mode, mstart[mode]);
            } catch (...) {
                err[m0] = std::current_exception();
            }
        };
        std::vector<std::thread> pool;
        int started = 1;
        try {
            for (; started < nt; ++started) pool.emplace_back(some_modes, started);
        } catch (const std::system_error &) {
        }
        some_modes(0);
        for (int t = started; t < nt; ++t) some_modes(t);
        for (std::thread &th : pool) th.join();
        for (const std::exception_ptr &e : err)
            if (e) std::rethrow_exception(e);
        for (int mode = 0; mode < nmodes; ++mode)
            if (cost[mode] < 1e300) rank.push_back({cost[mode], mode});
        if (rank.empty()) return false;
        std::sort(rank.begin(), rank.end());
        if (!cover) {
            assign_band(V, rank[0].second, mstart[rank[0].second]);
            return true;
        }
        for (int a = 0; a < N; ++a) pos_in[V[a]] = a;
        double best = 1e300, best_t = 0.0;
        std::vector<char> cov, best_cov;
        std::vector<double> fv(N), best_fv;
        for (int c = 0; c < std::min<int>(3, (int)rank.size()); ++c) {
            const int mode = rank[c].second;
            for (int a = 0; a < N; ++a) fv[a] = fval(mode, states[V[a]]);
            const double t = mstart[mode] + 0.5 * D[mode];
            const int64_t nc = min_cover(V, fv, t, cov);
            int64_t n1 = 0, n2 = 0;
            for (int a = 0; a < N; ++a)
                if (!cov[a]) ++(fv[a] < t ? n1 : n2);
            if (n1 == 0 || n2 == 0) continue;
            const double cost = (double)nc + 0.3 * (double)std::llabs(n1 - n2);
            if (cost < best) { best = cost; best_t = t; best_cov.swap(cov); best_fv.swap(fv); fv.resize(N); }
        }
        for (int a = 0; a < N; ++a) pos_in[V[a]] = -1;
        if (best >= 1e300) {  // every cover emptied a side: the band of the best mode
            assign_band(V, rank[0].second, mstart[rank[0].second]);
            return true;
        }
        for (int a = 0; a < N; ++a) part[V[a]] = best_cov[a] ? 3 : (best_fv[a] < best_t ? 1 : 2);
        return true;
    }

    void run(std::vector<int32_t> V, int depth) {
        if ((int)V.size() <= LEAF) {
            md_leaf(g, V, pos_in, order);
            return;
        }
        const int N = (int)V.size();
        const bool cover = ordering == MBL_ORDER_COVER || (ordering == MBL_ORDER_HYBRID && N >= HYBRID_COVER_MIN);
        const bool ok = ordering == MBL_ORDER_BAND ? split_band(V, depth) : split_modes(V, cover);
        if (!ok) {  // cannot split (degenerate values): minimum degree in chunks
            std::vector<int32_t> chunk;
            for (int a = 0; a < N; ++a) {
                chunk.push_back(V[a]);
                if ((int)chunk.size() == LEAF) { md_leaf(g, chunk, pos_in, order); chunk.clear(); }
            }
            if (!chunk.empty()) md_leaf(g, chunk, pos_in, order);
            return;
        }
        // thin the separator: a separator vertex with no neighbour on one side joins the other
        for (int a = 0; a < N; ++a) {
            int32_t v = V[a];
            if (part[v] != 3) continue;
            bool n1 = false, n2 = false;
            for (int64_t e = (*g.rowptr)[v]; e < (*g.rowptr)[v + 1]; ++e) {
                int8_t pu = part[(*g.col)[e]];
                n1 |= pu == 1;
                n2 |= pu == 2;
            }
            if (!n1) part[v] = 2;
            else if (!n2) part[v] = 1;
        }
        std::vector<int32_t> V1, V2, S;
        for (int a = 0; a < N; ++a) {
            int8_t pv = part[V[a]];
            (pv == 1 ? V1 : pv == 2 ? V2 : S).push_back(V[a]);
        }
        for (int a = 0; a < N; ++a) part[V[a]] = 0;
        std::vector<int32_t>().swap(V);
        run(std::move(V1), depth + 1);
        run(std::move(V2), depth + 1);
        for (int32_t v : S) order.push_back(v);
    }
};

}  // namespace

std::shared_ptr<Plan> build_plan(int L, const std::vector<uint32_t> &states, const std::vector<int64_t> &rowptr,
                                 const std::vector<int32_t> &col, int ordering) {
    if (ordering < MBL_ORDER_BAND || ordering > MBL_ORDER_HYBRID) fail(MBL_ERR_INVALID, "unknown ordering");
    ordering = resolve_ordering(ordering, (int64_t)states.size());
    auto t0 = std::chrono::steady_clock::now();
    auto P = std::make_shared<Plan>();
    Plan &p = *P;
    int64_t n = (int64_t)states.size();
    p.ordering = ordering;
    p.L = L;
    p.n = n;
    p.nnzA = rowptr[n];
    Graph g{n, &rowptr, &col};

    // ---- 1. nested-dissection order ----
    {
        ND nd(g, L, states, ordering);
        std::vector<int32_t> all(n);
        std::iota(all.begin(), all.end(), 0);
        nd.run(std::move(all), 0);
        p.perm = std::move(nd.order);
    }
    if ((int64_t)p.perm.size() != n) fail(MBL_ERR_INVALID, "ordering lost vertices");

    auto lower_lists = [&](const std::vector<int32_t> &perm, std::vector<int32_t> &iperm, std::vector<int64_t> &lp,
                           std::vector<int32_t> &li) {
        // li[lp[i]..lp[i+1]) = new neighbours k < i of new vertex i (ascending)
        iperm.assign(n, -1);
        for (int64_t k = 0; k < n; ++k) iperm[perm[k]] = (int32_t)k;
        lp.assign(n + 1, 0);
        for (int64_t r = 0; r < n; ++r) {
            int32_t a = iperm[r];
            for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
                int32_t b = iperm[col[e]];
                if (b < a) lp[a + 1]++;
            }
        }
        for (int64_t i = 0; i < n; ++i) lp[i + 1] += lp[i];
        li.assign(lp[n], 0);
        std::vector<int64_t> fill(lp.begin(), lp.end() - 1);
        for (int64_t r = 0; r < n; ++r) {
            int32_t a = iperm[r];
            for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
                int32_t b = iperm[col[e]];
                if (b < a) li[fill[a]++] = b;
            }
        }
        for (int64_t i = 0; i < n; ++i) std::sort(li.begin() + lp[i], li.begin() + lp[i + 1]);
    };
    auto etree = [&](const std::vector<int64_t> &lp, const std::vector<int32_t> &li, std::vector<int32_t> &parent) {
        parent.assign(n, -1);
        std::vector<int32_t> anc(n, -1);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t e = lp[i]; e < lp[i + 1]; ++e) {
                int32_t r = li[e];
                while (anc[r] != -1 && anc[r] != i) {
                    int32_t t = anc[r];
                    anc[r] = (int32_t)i;
                    r = t;
                }
                if (anc[r] == -1) {
                    anc[r] = (int32_t)i;
                    parent[r] = (int32_t)i;
                }
            }
    };

    std::vector<int64_t> lp;
    std::vector<int32_t> li, parent;
    lower_lists(p.perm, p.iperm, lp, li);
    etree(lp, li, parent);

    // ---- 2. postorder (children visited in ascending order), compose with the ND order ----
    {
        std::vector<int32_t> head(n, -1), next(n, -1);
        for (int64_t j = n - 1; j >= 0; --j)
            if (parent[j] >= 0) {
                next[j] = head[parent[j]];
                head[parent[j]] = (int32_t)j;
            }
        std::vector<int32_t> post;
        post.reserve(n);
        std::vector<int32_t> stack;
        for (int64_t r = 0; r < n; ++r) {
            if (parent[r] != -1) continue;
            stack.push_back((int32_t)r);
            while (!stack.empty()) {
                int32_t v = stack.back();
                if (head[v] != -1) {
                    int32_t c = head[v];
                    head[v] = next[c];
                    stack.push_back(c);
                } else {
                    stack.pop_back();
                    post.push_back(v);
                }
            }
        }
        std::vector<int32_t> perm2(n);
        for (int64_t k = 0; k < n; ++k) perm2[k] = p.perm[post[k]];
        p.perm = std::move(perm2);
    }
    lower_lists(p.perm, p.iperm, lp, li);
    etree(lp, li, parent);

    // ---- 3. column counts (strictly lower), Gilbert, Ng and Peyton (1994) ----
    // Column j of L holds row i > j exactly when j lies in the row subtree T_i (the union of the
    // tree paths from each k < i with A(i, k) != 0 up to i).  With the columns in postorder,
    // colcount(j) = 1 + #{i > j : j in T_i} is the sum over the subtree of j of
    //   delta(d) = [d a leaf of the tree] - #children(d)
    //            + #{i : d a leaf of T_i} - #{i : d the lowest common ancestor of two leaves of
    //              T_i adjacent in postorder},
    // which takes O(nnz(A)) work plus near-constant-time ancestor queries, instead of one step per
    // entry of L.  d is a leaf of T_i iff no earlier neighbour k of row i lies in d's subtree,
    // i.e. the last neighbour seen is before first(d), the first descendant of d; the common
    // ancestor of the previous leaf and d is the root of the previous leaf's set in a union-find
    // whose completed nodes point at their parents (Tarjan's offline ancestors).
    std::vector<int64_t> cc(n, 0);
    {
        std::vector<int64_t> up(n + 1, 0);  // upper pattern: rows i > j of column j, ascending
        for (int64_t i = 0; i < n; ++i)
            for (int64_t e = lp[i]; e < lp[i + 1]; ++e) up[li[e] + 1]++;
        for (int64_t j = 0; j < n; ++j) up[j + 1] += up[j];
        std::vector<int32_t> ui(up[n]);
        {
            std::vector<int64_t> fill(up.begin(), up.end() - 1);
            for (int64_t i = 0; i < n; ++i)
                for (int64_t e = lp[i]; e < lp[i + 1]; ++e) ui[fill[li[e]]++] = (int32_t)i;
        }
        std::vector<int32_t> first(n, -1), last(n, -1), prevleaf(n, -1), anc(n);
        std::vector<int64_t> delta(n, 0);
        for (int64_t k = 0; k < n; ++k)
            for (int64_t j = k; j != -1 && first[j] == -1; j = parent[j]) first[j] = (int32_t)k;
        std::iota(anc.begin(), anc.end(), 0);
        auto find = [&](int32_t x) {  // root of x's set, with path halving
            while (anc[x] != x) {
                anc[x] = anc[anc[x]];
                x = anc[x];
            }
            return x;
        };
        for (int64_t j = 0; j < n; ++j) {
            if (first[j] == j) delta[j] += 1;      // a leaf of the elimination tree
            if (parent[j] >= 0) delta[parent[j]] -= 1;
            for (int64_t e = up[j]; e < up[j + 1]; ++e) {
                const int32_t i = ui[e];
                if (last[i] < first[j]) {           // j is a leaf of T_i
                    delta[j] += 1;
                    if (prevleaf[i] >= 0) delta[find(prevleaf[i])] -= 1;
                    prevleaf[i] = (int32_t)j;
                }
                last[i] = (int32_t)j;
            }
            if (parent[j] >= 0) anc[j] = parent[j];
        }
        for (int64_t j = 0; j < n; ++j) {
            if (parent[j] >= 0) delta[parent[j]] += delta[j];
            cc[j] = delta[j] - 1;
        }
    }
    std::vector<int32_t> nchild(n, 0);
    for (int64_t j = 0; j < n; ++j)
        if (parent[j] >= 0) nchild[parent[j]]++;

    // ---- 4. fundamental supernodes ----
    std::vector<int32_t> fs_start;
    for (int64_t j = 0; j < n; ++j) {
        bool cont = j > 0 && parent[j - 1] == j && cc[j - 1] == cc[j] + 1 && nchild[j] == 1;
        if (!cont) fs_start.push_back((int32_t)j);
    }
    fs_start.push_back((int32_t)n);
    int32_t nfs = (int32_t)fs_start.size() - 1;
    std::vector<int32_t> col2fs(n);
    for (int32_t s = 0; s < nfs; ++s)
        for (int32_t j = fs_start[s]; j < fs_start[s + 1]; ++j) col2fs[j] = s;

    // ---- 5. relaxed amalgamation on the supernode tree (postorder = column order) ----
    // A supernode is [first, last] with front size f = nc + |update rows|; merging the child that
    // ends at first-1 into its parent keeps columns contiguous.
    struct SN {
        int32_t first, last, parent;
        int64_t f, true_nnz, stored;
        bool alive;
    };
    std::vector<SN> sn(nfs);
    for (int32_t s = 0; s < nfs; ++s) {
        int32_t a = fs_start[s], b = fs_start[s + 1] - 1;
        int64_t nc = b - a + 1;
        int64_t f = nc + cc[b];
        int64_t tn = 0;
        for (int32_t j = a; j <= b; ++j) tn += cc[j] + 1;
        sn[s] = SN{a, b, parent[b] >= 0 ? col2fs[parent[b]] : -1, f, tn, nc * f - nc * (nc - 1) / 2, true};
    }
    std::vector<int32_t> into(nfs);
    std::iota(into.begin(), into.end(), 0);
    auto find = [&](int32_t x) {
        while (into[x] != x) {
            into[x] = into[into[x]];
            x = into[x];
        }
        return x;
    };
    for (int32_t s = 0; s < nfs; ++s) {
        // repeatedly absorb the child ending right before our first column
        while (sn[s].first > 0) {
            int32_t c = col2fs[sn[s].first - 1];
            if (!sn[c].alive || sn[c].parent < 0 || find(sn[c].parent) != s) break;
            int64_t ncc = sn[c].last - sn[c].first + 1, ncp = sn[s].last - sn[s].first + 1;
            int64_t nc = ncc + ncp;
            int64_t f = ncc + sn[s].f;
            int64_t stored = nc * f - nc * (nc - 1) / 2;
            int64_t tn = sn[c].true_nnz + sn[s].true_nnz;
            bool ok = (nc <= 16) || ((double)(stored - tn) <= 0.15 * (double)stored);
            if (!ok) break;
            sn[c].alive = false;
            into[c] = s;
            for (int32_t j = sn[c].first; j <= sn[c].last; ++j) col2fs[j] = s;
            sn[s].first = sn[c].first;
            sn[s].f = f;
            sn[s].true_nnz = tn;
            sn[s].stored = stored;
        }
    }
    // renumber alive supernodes in column order
    std::vector<int32_t> newid(nfs, -1);
    int32_t ns = 0;
    for (int32_t s = 0; s < nfs; ++s)
        if (sn[s].alive) newid[s] = ns++;
    p.ns = ns;
    p.sn_start.assign(ns + 1, 0);
    p.sn_nc.assign(ns, 0);
    for (int32_t s = 0; s < nfs; ++s)
        if (sn[s].alive) {
            p.sn_start[newid[s]] = sn[s].first;
            p.sn_nc[newid[s]] = sn[s].last - sn[s].first + 1;
        }
    p.sn_start[ns] = (int32_t)n;
    p.col_snode.assign(n, 0);
    for (int32_t s = 0; s < ns; ++s)
        for (int32_t j = p.sn_start[s]; j < p.sn_start[s + 1]; ++j) p.col_snode[j] = s;

    // ---- 6. row structures (own columns, then update rows ascending) and tree ----
    p.sn_f.assign(ns, 0);
    p.sn_parent.assign(ns, -1);
    p.sn_rows_off.assign(ns + 1, 0);
    std::vector<std::vector<int32_t>> upd(ns);
    std::vector<std::vector<int32_t>> children(ns);
    {
        std::vector<int32_t> mark(n, -1);
        for (int32_t s = 0; s < ns; ++s) {
            int32_t a = p.sn_start[s], b = p.sn_start[s + 1] - 1;
            std::vector<int32_t> &u = upd[s];
            // columns of s appear as rows of later vertices: scan their lower lists is expensive;
            // use the symmetric pattern: rows i > b adjacent to a column j in [a, b]
            for (int32_t j = a; j <= b; ++j) {
                int32_t r = p.perm[j];
                for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
                    int32_t i = p.iperm[col[e]];
                    if (i > b && mark[i] != s) {
                        mark[i] = s;
                        u.push_back(i);
                    }
                }
            }
            for (int32_t c : children[s])
                for (int32_t i : upd[c])
                    if (i > b && mark[i] != s) {
                        mark[i] = s;
                        u.push_back(i);
                    }
            std::sort(u.begin(), u.end());
            if (!u.empty()) {
                int32_t ps = p.col_snode[u[0]];
                p.sn_parent[s] = ps;
                children[ps].push_back(s);
            }
            p.sn_f[s] = p.sn_nc[s] + (int32_t)u.size();
        }
    }
    for (int32_t s = 0; s < ns; ++s) p.sn_rows_off[s + 1] = p.sn_rows_off[s] + p.sn_f[s];
    p.rows.resize(p.sn_rows_off[ns]);
    for (int32_t s = 0; s < ns; ++s) {
        int64_t o = p.sn_rows_off[s];
        for (int32_t t = 0; t < p.sn_nc[s]; ++t) p.rows[o + t] = p.sn_start[s] + t;
        std::copy(upd[s].begin(), upd[s].end(), p.rows.begin() + o + p.sn_nc[s]);
    }
    p.ch_ptr.assign(ns + 1, 0);
    for (int32_t s = 0; s < ns; ++s) p.ch_ptr[s + 1] = p.ch_ptr[s] + (int32_t)children[s].size();
    p.ch_list.resize(p.ch_ptr[ns]);
    for (int32_t s = 0; s < ns; ++s) std::copy(children[s].begin(), children[s].end(), p.ch_list.begin() + p.ch_ptr[s]);

    // relative indices of each child's update rows in its parent's row list
    p.sn_rel_off.assign(ns + 1, 0);
    for (int32_t s = 0; s < ns; ++s) p.sn_rel_off[s + 1] = p.sn_rel_off[s] + (p.sn_f[s] - p.sn_nc[s]);
    p.relind.resize(p.sn_rel_off[ns]);
    for (int32_t s = 0; s < ns; ++s) {
        int32_t ps = p.sn_parent[s];
        if (ps < 0) continue;
        const int32_t *pr = p.rows.data() + p.sn_rows_off[ps];
        int32_t pf = p.sn_f[ps];
        int32_t q = 0;
        for (int32_t t = 0; t < p.sn_f[s] - p.sn_nc[s]; ++t) {
            int32_t i = upd[s][t];
            while (q < pf && pr[q] < i) ++q;
            if (q >= pf || pr[q] != i) fail(MBL_ERR_INVALID, "symbolic: child row missing from parent front");
            p.relind[p.sn_rel_off[s] + t] = q;
        }
    }

    // ---- 7. levels, offsets, assembly map, statistics ----
    p.sn_level.assign(ns, 0);
    for (int32_t s = 0; s < ns; ++s)
        for (int32_t c : children[s]) p.sn_level[s] = std::max(p.sn_level[s], p.sn_level[c] + 1);
    p.nlevels = 0;
    for (int32_t s = 0; s < ns; ++s) p.nlevels = std::max(p.nlevels, p.sn_level[s] + 1);
    p.lvl_ptr.assign(p.nlevels + 1, 0);
    for (int32_t s = 0; s < ns; ++s) p.lvl_ptr[p.sn_level[s] + 1]++;
    for (int l = 0; l < p.nlevels; ++l) p.lvl_ptr[l + 1] += p.lvl_ptr[l];
    p.lvl_fronts.resize(ns);
    {
        std::vector<int32_t> fill(p.lvl_ptr.begin(), p.lvl_ptr.end() - 1);
        for (int32_t s = 0; s < ns; ++s) p.lvl_fronts[fill[p.sn_level[s]]++] = s;
    }
    // Fronts are grouped by (level, release level), the release level of a front being its parent's
    // level -- the assembly that reads its contribution block last -- or its own for a root.  Each
    // group is one region of the arena starting on an ARENA_ALIGN boundary, so that the memory-lean
    // factorization can back each region with its own physical memory: mapped before its level
    // assembles, released right after its release level's assembly (a root's after its own level's
    // solve-factor build).  Regions are ordered by level, then release level.
    p.sn_fo.assign(ns + 1, 0);
    p.sn_zo.assign(ns + 1, 0);
    for (int32_t s = 0; s < ns; ++s) p.sn_zo[s + 1] = p.sn_zo[s] + p.sn_f[s];
    p.regions.clear();
    {
        int64_t cur = 0;
        for (int l = 0; l < p.nlevels; ++l) {
            std::vector<std::pair<int32_t, int32_t>> fr;  // (release level, front)
            for (int32_t q = p.lvl_ptr[l]; q < p.lvl_ptr[l + 1]; ++q) {
                const int32_t s = p.lvl_fronts[q];
                fr.push_back({p.sn_parent[s] < 0 ? l : p.sn_level[p.sn_parent[s]], s});
            }
            std::stable_sort(fr.begin(), fr.end(),
                             [](const std::pair<int32_t, int32_t> &x, const std::pair<int32_t, int32_t> &y) {
                                 return x.first < y.first;
                             });
            for (size_t i = 0; i < fr.size(); ++i) {
                if (i == 0 || fr[i].first != fr[i - 1].first) {
                    cur = (cur + ARENA_ALIGN - 1) / ARENA_ALIGN * ARENA_ALIGN;
                    p.regions.push_back(ArenaRegion{l, fr[i].first, cur, cur});
                }
                const int32_t s = fr[i].second;
                p.sn_fo[s] = cur;
                cur += (int64_t)p.sn_f[s] * p.sn_f[s];
                p.regions.back().fo1 = cur;
            }
        }
        p.arena_elems = (cur + ARENA_ALIGN - 1) / ARENA_ALIGN * ARENA_ALIGN;
        p.sn_fo[ns] = p.arena_elems;
    }
    // Peak of the memory-lean arena.  Each region is mapped as chunks of LEAN_CHUNK elements (the last
    // one rounded up to ARENA_ALIGN) when its level assembles; a region whose release level is later is
    // released right after that level's assembly; once a level's panels and solve-factor build are done,
    // the chunks lying wholly inside one of its fronts' fully summed columns [fo, fo + nc f) (the
    // factor, now copied to the solve factor) and its root regions are released too.  The peak is
    // taken after each assembly and after each level's panels, the two points where nothing has been
    // released yet since the last mapping.
    {
        auto chunk_sz = [](int64_t a0, int64_t a1) {
            return (std::min(a1, a0 + LEAN_CHUNK) - a0 + ARENA_ALIGN - 1) / ARENA_ALIGN * ARENA_ALIGN;
        };
        std::vector<std::vector<char>> gone(p.regions.size());
        for (size_t r = 0; r < p.regions.size(); ++r)
            gone[r].assign((size_t)((p.regions[r].fo1 - p.regions[r].fo0 + LEAN_CHUNK - 1) / LEAN_CHUNK), 0);
        auto release_region = [&](size_t r, int64_t &mapped) {
            const ArenaRegion &g = p.regions[r];
            for (size_t c = 0; c < gone[r].size(); ++c)
                if (!gone[r][c]) {
                    gone[r][c] = 1;
                    mapped -= chunk_sz(g.fo0 + (int64_t)c * LEAN_CHUNK, g.fo1);
                }
        };
        // chunks wholly inside a front's fully summed columns, by level: released after its build
        p.lean_prefix_ptr.assign(p.nlevels + 1, 0);
        p.lean_prefix.clear();
        for (int l = 0; l < p.nlevels; ++l) {
            for (size_t r = 0; r < p.regions.size(); ++r) {
                const ArenaRegion &g = p.regions[r];
                if (g.level != l || g.release == l) continue;
                for (size_t c = 0; c < gone[r].size(); ++c) {
                    const int64_t a0 = g.fo0 + (int64_t)c * LEAN_CHUNK, a1 = std::min(g.fo1, a0 + LEAN_CHUNK);
                    for (int32_t q = p.lvl_ptr[l]; q < p.lvl_ptr[l + 1]; ++q) {
                        const int32_t s = p.lvl_fronts[q];
                        if (p.sn_fo[s] <= a0 && a1 <= p.sn_fo[s] + (int64_t)p.sn_nc[s] * p.sn_f[s]) {
                            p.lean_prefix.push_back({(int32_t)r, (int32_t)c});
                            break;
                        }
                    }
                }
            }
            p.lean_prefix_ptr[l + 1] = (int64_t)p.lean_prefix.size();
        }
        int64_t mapped = 0, peak = 0;
        for (int l = 0; l < p.nlevels; ++l) {
            for (const ArenaRegion &g : p.regions)
                if (g.level == l)
                    for (int64_t a0 = g.fo0; a0 < g.fo1; a0 += LEAN_CHUNK) mapped += chunk_sz(a0, g.fo1);
            peak = std::max(peak, mapped);  // the assembly of level l
            for (size_t r = 0; r < p.regions.size(); ++r)
                if (p.regions[r].level < l && p.regions[r].release == l) release_region(r, mapped);
            peak = std::max(peak, mapped);  // its panels and solve-factor build
            for (int64_t i = p.lean_prefix_ptr[l]; i < p.lean_prefix_ptr[l + 1]; ++i) {
                const int32_t r = p.lean_prefix[i].first, c = p.lean_prefix[i].second;
                if (!gone[r][c]) {
                    gone[r][c] = 1;
                    mapped -= chunk_sz(p.regions[r].fo0 + (int64_t)c * LEAN_CHUNK, p.regions[r].fo1);
                }
            }
            for (size_t r = 0; r < p.regions.size(); ++r)
                if (p.regions[r].level == l && p.regions[r].release == l) release_region(r, mapped);
        }
        p.lean_peak_elems = peak;
    }
    p.zwork_elems = p.sn_zo[ns];
    p.max_front = 0;
    p.nnz_l = 0;
    p.flops = 0.0;
    for (int32_t s = 0; s < ns; ++s) {
        int64_t f = p.sn_f[s], nc = p.sn_nc[s];
        p.max_front = std::max<int32_t>(p.max_front, (int32_t)f);
        p.nnz_l += nc * (nc - 1) / 2 + nc * (f - nc);
        for (int64_t k = 0; k < nc; ++k) p.flops += (double)(f - k - 1) * (double)(f - k - 1);
    }
    // assembly map: CSR entry (r, c) with new indices a >= b goes to column b's front at local row of a
    p.amap_ptr.assign(n + 1, 0);
    for (int64_t r = 0; r < n; ++r)
        for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
            int32_t a = p.iperm[r], b = p.iperm[col[e]];
            if (a >= b) p.amap_ptr[b + 1]++;
        }
    for (int64_t j = 0; j < n; ++j) p.amap_ptr[j + 1] += p.amap_ptr[j];
    p.amap_src.resize(p.amap_ptr[n]);
    p.amap_row.resize(p.amap_ptr[n]);
    {
        std::vector<int64_t> fill(p.amap_ptr.begin(), p.amap_ptr.end() - 1);
        for (int64_t r = 0; r < n; ++r)
            for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
                int32_t a = p.iperm[r], b = p.iperm[col[e]];
                if (a < b) continue;
                int32_t s = p.col_snode[b];
                const int32_t *pr = p.rows.data() + p.sn_rows_off[s];
                int32_t lr = (int32_t)(std::lower_bound(pr, pr + p.sn_f[s], a) - pr);
                if (lr >= p.sn_f[s] || pr[lr] != a) fail(MBL_ERR_INVALID, "symbolic: entry outside front");
                int64_t q = fill[b]++;
                p.amap_src[q] = e;
                p.amap_row[q] = lr;
            }
    }
    // assembly items and panel schedule per level
    p.asm_ptr.assign(p.nlevels + 1, 0);
    p.lvl_step_ptr.assign(p.nlevels + 1, 0);
    p.lvl_sstep_ptr.assign(p.nlevels + 1, 0);
    p.bu_ptr.assign(1, 0);
    std::vector<int64_t> fd_off(ns + 1, 0);  // factor descriptor of (front, panel) at fd_of[fd_off[s] + kk]
    for (int32_t s = 0; s < ns; ++s) fd_off[s + 1] = fd_off[s] + (p.sn_nc[s] + NB - 1) / NB;
    std::vector<int32_t> fd_of(fd_off[ns], -1);
    for (int l = 0; l < p.nlevels; ++l) {
        int32_t maxnc = 0;
        for (int32_t q = p.lvl_ptr[l]; q < p.lvl_ptr[l + 1]; ++q) {
            int32_t s = p.lvl_fronts[q];
            for (int32_t c0 = 0; c0 < p.sn_f[s]; c0 += ACOLS) p.asm_items.push_back(AsmItem{s, c0});
            maxnc = std::max(maxnc, p.sn_nc[s]);
        }
        p.asm_ptr[l + 1] = (int32_t)p.asm_items.size();
        for (int32_t kk = 0; kk * NB < maxnc; ++kk) {
            PanelStep stp{l, kk, (int32_t)p.descs.size(), 0, 0, 0, 0, 0};
            for (int32_t q = p.lvl_ptr[l]; q < p.lvl_ptr[l + 1]; ++q) {
                int32_t s = p.lvl_fronts[q];
                int32_t k0 = kk * NB;
                if (p.sn_nc[s] <= k0) continue;
                int32_t w = std::min(NB, p.sn_nc[s] - k0);
                int32_t m2 = p.sn_f[s] - k0 - w;
                PanelDesc d{s, k0, w, m2, stp.n2, stp.n3, stp.wsize, stp.n3t};
                fd_of[fd_off[s] + kk] = (int32_t)p.descs.size();
                int64_t nb2 = (m2 + RB - 1) / RB;
                int64_t T = (m2 + TB - 1) / TB;
                stp.n2 += nb2;
                stp.n3 += T * (T + 1) / 2;
                int64_t Tt = (m2 + 127) / 128;
                stp.n3t += Tt * (Tt + 1) / 2;
                stp.wsize += (int64_t)m2 * NB;
                p.descs.push_back(d);
            }
            stp.nd = (int32_t)p.descs.size() - stp.d0;
            {
                int64_t mx = 0;
                for (int32_t q = stp.d0; q < stp.d0 + stp.nd; ++q) mx = std::max<int64_t>(mx, p.descs[q].m2);
                p.step_class.push_back(tune_class(mx));
            }
            p.max_desc_per_step = std::max<int64_t>(p.max_desc_per_step, stp.nd);
            p.max_step_n2 = std::max<int64_t>(p.max_step_n2, stp.n2);
            p.wscratch_elems = std::max(p.wscratch_elems, stp.wsize);
            p.steps.push_back(stp);
        }
        p.lvl_step_ptr[l + 1] = (int32_t)p.steps.size();
        // solve schedule: SPW-wide panels
        for (int32_t ks = 0; ks * SPW < maxnc; ++ks) {
            SolveStep ss{l, (int32_t)p.sdescs.size(), 0, 0, 0, 0, 0, (int64_t)p.fblk_desc.size(),
                         (int64_t)p.bblk_desc.size()};
            for (int32_t q = p.lvl_ptr[l]; q < p.lvl_ptr[l + 1]; ++q) {
                int32_t s = p.lvl_fronts[q];
                int32_t k0 = ks * SPW;
                if (p.sn_nc[s] <= k0) continue;
                int32_t w = std::min(SPW, p.sn_nc[s] - k0);
                SolveDesc sd;
                sd.front = s;
                sd.k0 = k0;
                sd.w = w;
                sd.m2 = p.sn_f[s] - k0 - w;
                sd.off = ss.nrb;
                sd.offb = ss.nrbb;
                sd.offk = ss.nrbk;
                sd.moff = p.m_elems;
                sd.goff = p.sg_elems;
                for (int u = 0; u < SUBS; ++u) {
                    int32_t kk = (k0 + u * NB) / NB;
                    sd.fdesc[u] = (u * NB < w) ? fd_of[fd_off[s] + kk] : -1;
                }
                ss.nrb += (w + sd.m2 + RBF - 1) / RBF;
                ss.nrbb += (w + sd.m2 + RBB - 1) / RBB;
                ss.nrbk += (w + sd.m2 + RBK - 1) / RBK;
                ss.maxw = std::max(ss.maxw, w);
                const int32_t local = (int32_t)p.sdescs.size() - ss.d0;
                for (int32_t b = 0; b < (w + sd.m2 + RBF - 1) / RBF; ++b) p.fblk_desc.push_back(local);
                for (int32_t b = 0; b < (w + sd.m2 + RBK - 1) / RBK; ++b) p.bblk_desc.push_back(local);
                p.m_elems += (int64_t)w * w;
                p.sg_elems += sg_ld(w + sd.m2) * w;
                p.sdescs.push_back(sd);
            }
            ss.nd = (int32_t)p.sdescs.size() - ss.d0;
            p.max_sstep_nrbb = std::max(p.max_sstep_nrbb, ss.nrbb);
            p.max_sstep_nrbk = std::max(p.max_sstep_nrbk, ss.nrbk);
            p.ssteps.push_back(ss);
        }
        p.lvl_sstep_ptr[l + 1] = (int32_t)p.ssteps.size();
        // backward: level-wide start over the level's descriptors (contiguous), then the updates
        {
            const int32_t d0 = p.ssteps[p.lvl_sstep_ptr[l]].d0;
            const int32_t d1 = (int32_t)p.sdescs.size();
            int64_t nrbk = 0;
            int32_t maxw = 0, maxr = 0;
            p.lvl_d0.push_back(d0);
            p.lvl_nd.push_back(d1 - d0);
            p.lvl_bblk0.push_back((int64_t)p.lvl_bblk_desc.size());
            std::vector<std::vector<int32_t>> panels_of;  // per front of the level: its descriptors in panel order
            std::map<int32_t, int32_t> slot;
            for (int32_t q = d0; q < d1; ++q) {
                SolveDesc &sd = p.sdescs[q];
                sd.offk_l = nrbk;
                const int32_t nb = bwd_start_blocks(sd.w + sd.m2, p.sn_nc[sd.front] - sd.k0);
                for (int32_t b = 0; b < nb; ++b) p.lvl_bblk_desc.push_back(q - d0);
                nrbk += nb;
                maxw = std::max(maxw, sd.w);
                maxr = std::max(maxr, sd.w + sd.m2);
                auto it = slot.find(sd.front);
                if (it == slot.end()) {
                    it = slot.emplace(sd.front, (int32_t)panels_of.size()).first;
                    panels_of.emplace_back();
                }
                panels_of[it->second].push_back(q);
            }
            p.lvl_nrbk.push_back(nrbk);
            p.lvl_maxw.push_back(maxw);
            p.lvl_maxr.push_back(maxr);
            p.max_lvl_nrbk = std::max(p.max_lvl_nrbk, nrbk);
            size_t kmax = 0;
            for (auto &v : panels_of) kmax = std::max(kmax, v.size());
            for (int32_t j = (int32_t)kmax - 1; j >= 1; --j) {
                BwdUpd u{l, j, (int64_t)p.bu_items.size() / 2, 0};
                for (auto &v : panels_of) {
                    if ((int32_t)v.size() <= j) continue;
                    for (int32_t i = 0; i < j; ++i) {
                        p.bu_items.push_back(v[i]);
                        p.bu_items.push_back(v[j]);
                        ++u.nit;
                    }
                }
                p.bupd.push_back(u);
            }
            p.bu_ptr.push_back((int32_t)p.bupd.size());
        }
    }
    // forward-solve gather lists
    p.lvl_fg_ptr.assign(p.nlevels + 1, 0);
    p.fg_cptr.push_back(0);
    for (int l = 0; l < p.nlevels; ++l) {
        for (int32_t q = p.lvl_ptr[l]; q < p.lvl_ptr[l + 1]; ++q) {
            const int32_t s = p.lvl_fronts[q];
            const int32_t f = p.sn_f[s], ncs = p.sn_nc[s];
            std::vector<std::vector<int64_t>> in(f);
            for (int32_t c = p.ch_ptr[s]; c < p.ch_ptr[s + 1]; ++c) {
                const int32_t ch = p.ch_list[c];
                const int32_t uc = p.sn_f[ch] - p.sn_nc[ch];
                for (int32_t a = 0; a < uc; ++a)
                    in[p.relind[p.sn_rel_off[ch] + a]].push_back(p.sn_zo[ch] + p.sn_nc[ch] + a);
            }
            for (int32_t r = 0; r < f; ++r) {
                p.fg_dst.push_back(p.sn_zo[s] + r);
                p.fg_own.push_back(r < ncs ? (int64_t)p.sn_start[s] + r : -1);
                p.fg_src.insert(p.fg_src.end(), in[r].begin(), in[r].end());
                p.fg_cptr.push_back((int64_t)p.fg_src.size());
            }
        }
        p.lvl_fg_ptr[l + 1] = (int64_t)p.fg_dst.size();
    }
    // dataflow solve tables.  Forward order: level by level, gathers of the level's fronts, then
    // its panel steps in order; backward: levels in reverse, gathers, then panel steps last to first.
    {
        const int32_t ns_ = p.ns;
        p.df_gchunks.assign(ns_, 0);
        p.df_ftotal.assign(ns_, 0);
        p.df_btotal.assign(ns_, 0);
        p.df_fg_off.assign(ns_, 0);
        p.df_fprefix.assign(p.sdescs.size(), 0);
        p.df_bprefix.assign(p.sdescs.size(), 0);
        p.df_poff.assign(p.sdescs.size(), 0);
        {
            int64_t row = 0;
            for (int l = 0; l < p.nlevels; ++l)
                for (int32_t q = p.lvl_ptr[l]; q < p.lvl_ptr[l + 1]; ++q) {
                    const int32_t s = p.lvl_fronts[q];
                    p.df_fg_off[s] = row;
                    row += p.sn_f[s];
                }
        }
        std::vector<std::vector<int32_t>> panels(ns_);  // solve descriptors of each front, in panel order
        for (size_t q = 0; q < p.sdescs.size(); ++q) panels[p.sdescs[q].front].push_back((int32_t)q);
        for (int32_t s = 0; s < ns_; ++s) {
            p.df_gchunks[s] = (p.sn_f[s] + GR - 1) / GR;
            int32_t acc = 0;
            for (int32_t q : panels[s]) {
                const SolveDesc &d = p.sdescs[q];
                p.df_fprefix[q] = acc;
                acc += (d.w + d.m2 + RBF - 1) / RBF;
            }
            p.df_ftotal[s] = acc;
            acc = 0;
            for (auto it = panels[s].rbegin(); it != panels[s].rend(); ++it) {
                const SolveDesc &d = p.sdescs[*it];
                p.df_bprefix[*it] = acc;
                acc += (d.w + RBB - 1) / RBB;
            }
            p.df_btotal[s] = acc;
        }
        int64_t slots = 0;
        for (size_t q = 0; q < p.sdescs.size(); ++q) {
            p.df_poff[q] = slots;
            slots += (int64_t)((p.sdescs[q].w + p.sdescs[q].m2 + RBK - 1) / RBK) * SUBS;
        }
        p.df_pslots = slots;
        for (int l = 0; l < p.nlevels; ++l) {
            for (int32_t q = p.lvl_ptr[l]; q < p.lvl_ptr[l + 1]; ++q) {
                const int32_t s = p.lvl_fronts[q];
                for (int32_t c = 0; c < p.df_gchunks[s]; ++c) p.df_fwd.push_back(SolveItem{0, 0, s, c, 0});
            }
            for (int si = p.lvl_sstep_ptr[l]; si < p.lvl_sstep_ptr[l + 1]; ++si) {
                const SolveStep &ss = p.ssteps[si];
                for (int32_t q = ss.d0; q < ss.d0 + ss.nd; ++q) {
                    const SolveDesc &d = p.sdescs[q];
                    const int32_t nb = (d.w + d.m2 + RBF - 1) / RBF;
                    for (int32_t b = 0; b < nb; ++b) p.df_fwd.push_back(SolveItem{1, 0, d.front, q, b});
                }
            }
        }
        for (int l = p.nlevels - 1; l >= 0; --l) {
            for (int32_t q = p.lvl_ptr[l]; q < p.lvl_ptr[l + 1]; ++q) {
                const int32_t s = p.lvl_fronts[q];
                for (int32_t c = 0; c < p.df_gchunks[s]; ++c) p.df_bwd.push_back(SolveItem{0, 0, s, c, 0});
            }
            for (int si = p.lvl_sstep_ptr[l + 1] - 1; si >= p.lvl_sstep_ptr[l]; --si) {
                const SolveStep &ss = p.ssteps[si];
                for (int32_t q = ss.d0; q < ss.d0 + ss.nd; ++q) {
                    const SolveDesc &d = p.sdescs[q];
                    const int32_t nb = (d.w + d.m2 + RBK - 1) / RBK;
                    for (int32_t b = 0; b < nb; ++b)
                        for (int16_t cc = 0; cc * RBB < d.w; ++cc) p.df_bwd.push_back(SolveItem{1, cc, d.front, q, b});
                }
            }
        }
    }
    p.ms_analyse = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return P;
}

template <class T>
static void up(Ctx *ctx, DVec<T> &d, const std::vector<T> &h) {
    d.alloc(ctx, std::max<size_t>(h.size(), 1));
    if (!h.empty()) MBL_CUDA(cudaMemcpy(d.data(), h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
}

void upload_plan(Ctx *ctx, Plan &p) {
    if (p.on_device) return;
    up(ctx, p.d_perm, p.perm);
    up(ctx, p.d_iperm, p.iperm);
    up(ctx, p.d_sn_start, p.sn_start);
    up(ctx, p.d_sn_nc, p.sn_nc);
    up(ctx, p.d_sn_f, p.sn_f);
    up(ctx, p.d_rows, p.rows);
    up(ctx, p.d_relind, p.relind);
    up(ctx, p.d_ch_ptr, p.ch_ptr);
    up(ctx, p.d_ch_list, p.ch_list);
    up(ctx, p.d_amap_row, p.amap_row);
    up(ctx, p.d_sn_rows_off, p.sn_rows_off);
    up(ctx, p.d_sn_fo, p.sn_fo);
    up(ctx, p.d_sn_zo, p.sn_zo);
    up(ctx, p.d_sn_rel_off, p.sn_rel_off);
    up(ctx, p.d_amap_ptr, p.amap_ptr);
    up(ctx, p.d_amap_src, p.amap_src);
    up(ctx, p.d_asm_items, p.asm_items);
    up(ctx, p.d_descs, p.descs);
    up(ctx, p.d_sdescs, p.sdescs);
    up(ctx, p.d_fblk_desc, p.fblk_desc);
    up(ctx, p.d_bblk_desc, p.bblk_desc);
    up(ctx, p.d_lvl_bblk_desc, p.lvl_bblk_desc);
    up(ctx, p.d_bu_items, p.bu_items);
    up(ctx, p.d_fg_dst, p.fg_dst);
    up(ctx, p.d_fg_own, p.fg_own);
    up(ctx, p.d_fg_cptr, p.fg_cptr);
    up(ctx, p.d_fg_src, p.fg_src);
    up(ctx, p.d_sn_parent, p.sn_parent);
    up(ctx, p.d_df_fwd, p.df_fwd);
    up(ctx, p.d_df_bwd, p.df_bwd);
    up(ctx, p.d_df_gchunks, p.df_gchunks);
    up(ctx, p.d_df_ftotal, p.df_ftotal);
    up(ctx, p.d_df_btotal, p.df_btotal);
    up(ctx, p.d_df_fprefix, p.df_fprefix);
    up(ctx, p.d_df_bprefix, p.df_bprefix);
    up(ctx, p.d_df_fg_off, p.df_fg_off);
    up(ctx, p.d_df_poff, p.df_poff);
    p.on_device = true;
}

}  // namespace mbl
