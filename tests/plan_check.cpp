// plan_check.cpp -- host-only checks of the symbolic analysis (test helper, no GPU).
//
// Builds the pattern of the sector with nup up spins of an L-site ring (Eq. 1: one off-diagonal per
// antiparallel bond, the diagonal always present), runs the library's build_plan on it and checks
// structural invariants that the numeric factorization and the solves rely on.  Prints "ok ..." and
// exits 0, or prints the first violated invariant and exits 1.
//
// Usage: plan_check L nup [ordering]   (MBL_ORDER_BAND = 0, MBL_ORDER_COVER = 1, MBL_ORDER_MODES = 2,
//                                      MBL_ORDER_AUTO = 3 (default), MBL_ORDER_HYBRID = 4)
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <set>
#include <vector>

#include "plan.h"

using namespace mbl;

// The checks only use host data: the device mirror's memory management is not exercised.
namespace mbl {
DevMem &DevMem::operator=(DevMem &&o) noexcept {
    p = o.p;
    bytes = o.bytes;
    ctx = o.ctx;
    o.p = nullptr;
    return *this;
}
void DevMem::alloc(Ctx *, size_t) {}
void DevMem::release() {}
}  // namespace mbl

static int bad(const char *what, long a = 0, long b = 0) {
    std::printf("FAIL: %s (%ld, %ld)\n", what, a, b);
    return 1;
}

static int popcount32(uint32_t s) {
    int c = 0;
    for (; s; s &= s - 1) ++c;
    return c;
}

int main(int argc, char **argv) {
    if (argc != 3 && argc != 4) return bad("usage: plan_check L nup [ordering]");
    const int L = std::atoi(argv[1]), nup = std::atoi(argv[2]);
    const int ordering = argc == 4 ? std::atoi(argv[3]) : MBL_ORDER_AUTO;
    std::vector<uint32_t> st;
    for (uint32_t s = 0; s < (1u << L); ++s)
        if (popcount32(s) == nup) st.push_back(s);
    const int64_t n = (int64_t)st.size();
    std::vector<int64_t> rp(n + 1, 0);
    std::vector<int32_t> col;
    for (int64_t k = 0; k < n; ++k) {
        std::vector<int32_t> c{(int32_t)k};
        for (int i = 0; i < L; ++i) {
            const int j = (i + 1) % L;
            if (((st[k] >> i) & 1u) != ((st[k] >> j) & 1u)) {
                const uint32_t t = st[k] ^ (1u << i) ^ (1u << j);
                c.push_back((int32_t)(std::lower_bound(st.begin(), st.end(), t) - st.begin()));
            }
        }
        std::sort(c.begin(), c.end());
        c.erase(std::unique(c.begin(), c.end()), c.end());
        col.insert(col.end(), c.begin(), c.end());
        rp[k + 1] = (int64_t)col.size();
    }
    std::shared_ptr<Plan> P;
    try {
        P = build_plan(L, st, rp, col, ordering);
    } catch (const Error &e) {
        return bad(e.msg.c_str(), e.code);
    }
    const Plan &p = *P;

    // 1. the ordering is a permutation with its inverse
    if (p.n != n || (int64_t)p.perm.size() != n || (int64_t)p.iperm.size() != n) return bad("sizes", p.n, n);
    for (int64_t i = 0; i < n; ++i)
        if (p.perm[i] < 0 || p.perm[i] >= n || p.iperm[p.perm[i]] != i) return bad("perm/iperm", i, p.perm[i]);

    // 2. supernodes partition the columns in order; col_snode agrees
    int64_t next = 0;
    for (int s = 0; s < p.ns; ++s) {
        if (p.sn_start[s] != next || p.sn_nc[s] < 1 || p.sn_f[s] < p.sn_nc[s]) return bad("supernode columns", s, next);
        for (int c = 0; c < p.sn_nc[s]; ++c)
            if (p.col_snode[p.sn_start[s] + c] != s) return bad("col_snode", s, c);
        next += p.sn_nc[s];
    }
    if (next != n) return bad("columns covered", next, n);

    // 3. front rows: the own columns first, then ancestors' columns in ascending order; the parent
    // comes later in the order and sits on a higher level
    std::vector<std::set<int32_t>> rowset(p.ns);
    for (int s = 0; s < p.ns; ++s) {
        const int32_t *r = p.rows.data() + p.sn_rows_off[s];
        const int f = p.sn_f[s], nc = p.sn_nc[s];
        for (int i = 0; i < nc; ++i)
            if (r[i] != p.sn_start[s] + i) return bad("own rows", s, i);
        for (int i = nc; i < f; ++i) {
            if (r[i] < p.sn_start[s] + nc || (i > nc && r[i] <= r[i - 1])) return bad("contribution rows order", s, i);
            // the row's supernode is an ancestor of s
            int a = p.sn_parent[s];
            const int target = p.col_snode[r[i]];
            while (a >= 0 && a != target) a = p.sn_parent[a];
            if (a != target) return bad("contribution row not in an ancestor", s, r[i]);
        }
        rowset[s].insert(r, r + f);
        const int pa = p.sn_parent[s];
        if (pa >= 0 && (pa <= s || p.sn_level[pa] <= p.sn_level[s])) return bad("parent order / level", s, pa);
        if (pa < 0 && f != nc) return bad("root with a contribution block", s, f - nc);
    }
    // 4. multifrontal nesting: a child's contribution rows are rows of its parent
    for (int s = 0; s < p.ns; ++s) {
        const int pa = p.sn_parent[s];
        if (pa < 0) continue;
        const int32_t *r = p.rows.data() + p.sn_rows_off[s];
        for (int i = p.sn_nc[s]; i < p.sn_f[s]; ++i)
            if (!rowset[pa].count(r[i])) return bad("contribution row missing in parent", s, r[i]);
    }
    // 5. L's structure holds the pattern of P A P^T: entry (i, j), i > j (new), is a row of j's front
    for (int64_t jo = 0; jo < n; ++jo) {
        const int32_t j = p.iperm[jo];
        for (int64_t e = rp[jo]; e < rp[jo + 1]; ++e) {
            const int32_t i = p.iperm[col[e]];
            if (i > j && !rowset[p.col_snode[j]].count(i)) return bad("pattern entry outside L", i, j);
        }
    }
    // 6. nnz(L), strictly below the diagonal (unit diagonal implied)
    int64_t nnz = 0;
    for (int s = 0; s < p.ns; ++s)
        for (int k = 0; k < p.sn_nc[s]; ++k) nnz += p.sn_f[s] - k - 1;
    if (nnz != p.nnz_l) return bad("nnz_l", nnz, p.nnz_l);

    // 7. solve panels tile every front's fully summed block; solve steps cover each panel once;
    // packed factor offsets: consecutive, 16-byte aligned, columns of sg_ld(rows)
    for (size_t d = 0; d < p.sdescs.size(); ++d) {
        const SolveDesc &sd = p.sdescs[d];
        const int s = sd.front;
        if (sd.w < 1 || sd.w > SPW || sd.m2 != p.sn_f[s] - sd.k0 - sd.w) return bad("solve panel shape", (long)d, sd.w);
        if (sd.goff % 4 != 0 || sd.goff + sg_ld(sd.w + sd.m2) * sd.w > p.sg_elems)
            return bad("G offset alignment or range", (long)d, sd.goff);
    }
    std::vector<std::vector<const SolveDesc *>> by_front(p.ns);
    for (const SolveDesc &sd : p.sdescs) by_front[sd.front].push_back(&sd);
    int64_t sg = 0;
    for (int s = 0; s < p.ns; ++s) {
        auto v = by_front[s];
        std::sort(v.begin(), v.end(), [](const SolveDesc *a, const SolveDesc *b) { return a->k0 < b->k0; });
        int k = 0;
        for (const SolveDesc *sd : v) {
            if (sd->k0 != k) return bad("solve panels not contiguous", s, sd->k0);
            k += sd->w;
            sg += sg_ld(sd->w + sd->m2) * sd->w;
        }
        if (k != p.sn_nc[s]) return bad("solve panels do not cover the front", s, k);
    }
    if (sg != p.sg_elems) return bad("packed factor size", sg, p.sg_elems);
    std::vector<int> seen(p.sdescs.size(), 0);
    for (const SolveStep &ss : p.ssteps)
        for (int d = ss.d0; d < ss.d0 + ss.nd; ++d) {
            if (d < 0 || d >= (int)p.sdescs.size()) return bad("solve step range", ss.d0, ss.nd);
            ++seen[d];
        }
    for (size_t d = 0; d < seen.size(); ++d)
        if (seen[d] != 1) return bad("solve panel in steps", (long)d, seen[d]);

    // 8. the forward gather writes every row of every front exactly once
    {
        std::set<int64_t> dst;
        for (int64_t r = 0; r < (int64_t)p.fg_dst.size(); ++r)
            if (!dst.insert(p.fg_dst[r]).second) return bad("gather row written twice", r, p.fg_dst[r]);
        int64_t rows_total = 0;
        for (int s = 0; s < p.ns; ++s) {
            rows_total += p.sn_f[s];
            for (int i = 0; i < p.sn_f[s]; ++i)
                if (!dst.count(p.sn_zo[s] + i)) return bad("front row not gathered", s, i);
        }
        if ((int64_t)dst.size() != rows_total) return bad("gather rows", (long)dst.size(), rows_total);
    }

    // 9. dataflow item lists: every dependency is met by items earlier in the list
    {
        std::vector<int> gc(p.ns, 0), fc(p.ns, 0), bgc(p.ns, 0), bc(p.ns, 0);
        std::map<std::pair<int, int>, int> arrived;
        for (const SolveItem &it : p.df_fwd) {
            if (it.kind == 0) {
                for (int c = p.ch_ptr[it.front]; c < p.ch_ptr[it.front + 1]; ++c)
                    if (fc[p.ch_list[c]] != p.df_ftotal[p.ch_list[c]]) return bad("forward gather before a child", it.front, c);
                ++gc[it.front];
            } else {
                if (gc[it.front] != p.df_gchunks[it.front] || fc[it.front] < p.df_fprefix[it.a])
                    return bad("forward block before its inputs", it.front, it.a);
                ++fc[it.front];
            }
        }
        for (int s = 0; s < p.ns; ++s)
            if (fc[s] != p.df_ftotal[s] || gc[s] != p.df_gchunks[s]) return bad("forward totals", s, fc[s]);
        for (const SolveItem &it : p.df_bwd) {
            if (it.kind == 0) {
                const int pa = p.sn_parent[it.front];
                if (pa >= 0 && bc[pa] != p.df_btotal[pa]) return bad("backward gather before the parent", it.front, pa);
                ++bgc[it.front];
            } else {
                if (bgc[it.front] != p.df_gchunks[it.front] || bc[it.front] < p.df_bprefix[it.a])
                    return bad("backward block before its inputs", it.front, it.a);
                const SolveDesc &sd = p.sdescs[it.a];
                const int nb = (sd.w + sd.m2 + RBK - 1) / RBK;
                if (++arrived[{it.a, it.cc}] == nb) ++bc[it.front];
            }
        }
        for (int s = 0; s < p.ns; ++s)
            if (bc[s] != p.df_btotal[s] || bgc[s] != p.df_gchunks[s]) return bad("backward totals", s, bc[s]);
    }
    // fronts arena: aligned, disjoint regions ordered by (level, release); every front inside the
    // region of its level and its parent's level; the lean peak does not exceed the whole arena
    {
        std::map<std::pair<int, int>, int> reg;
        for (size_t i = 0; i < p.regions.size(); ++i) {
            const ArenaRegion &r = p.regions[i];
            if (r.fo0 % ARENA_ALIGN) return bad("region alignment", (long)i);
            if (r.fo1 < r.fo0 || r.fo1 > p.arena_elems) return bad("region bounds", (long)i);
            if (i && (p.regions[i - 1].fo1 > r.fo0)) return bad("regions overlap", (long)i);
            if (i && std::make_pair(p.regions[i - 1].level, p.regions[i - 1].release) >= std::make_pair(r.level, r.release))
                return bad("region order", (long)i);
            if (r.release < r.level || r.release >= p.nlevels) return bad("release level", (long)i);
            reg[{r.level, r.release}] = (int)i;
        }
        std::vector<std::pair<int64_t, int64_t>> iv;
        for (int32_t s = 0; s < p.ns; ++s) {
            const int l = p.sn_level[s], rl = p.sn_parent[s] < 0 ? l : p.sn_level[p.sn_parent[s]];
            auto it = reg.find({l, rl});
            if (it == reg.end()) return bad("front without region", s);
            const ArenaRegion &r = p.regions[it->second];
            const int64_t f = p.sn_f[s];
            if (p.sn_fo[s] < r.fo0 || p.sn_fo[s] + f * f > r.fo1) return bad("front outside its region", s);
            iv.push_back({p.sn_fo[s], p.sn_fo[s] + f * f});
        }
        std::sort(iv.begin(), iv.end());
        for (size_t i = 1; i < iv.size(); ++i)
            if (iv[i].first < iv[i - 1].second) return bad("fronts overlap", (long)i);
    }
    if (p.lean_peak_elems <= 0 || p.lean_peak_elems > p.arena_elems) return bad("lean peak", p.lean_peak_elems);
    std::printf("ok L=%d nup=%d n=%ld supernodes=%d levels=%d nnz_l=%ld solve_panels=%zu arena=%ld lean_peak=%ld "
                "flops=%.6e max_front=%d ordering=%d\n",
                L, nup, (long)n, p.ns, p.nlevels, (long)p.nnz_l, p.sdescs.size(), (long)p.arena_elems,
                (long)p.lean_peak_elems, p.flops, (int)p.max_front, p.ordering);
    return 0;
}
