// CPU oracle for the maximum common induced subgraph (MCIS) problem.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
// calls this file; only the tests, the package's smoke() check and the CPU
// baseline leg of the benchmark do.  It shares no code, header, table or
// helper with the CUDA path.
//
// Contents (each function cites the passage it follows):
//   oracle_verify      definition of a common induced subgraph (Section II-A)
//   oracle_mcs         sequential recursive McSplit (Section II-B, Algorithm 1,
//                      Eq. 1), plain vertex-list domains, one vertex pair per
//                      recursion level
//   oracle_bruteforce  enumeration of injective partial mappings (definition)
//   oracle_clique      maximum clique of the modular product graph (textbook
//                      reduction; independent of McSplit)
//   oracle_branch_log  oracle_mcs instrumented to record, per branching
//                      decision, which candidate pairs (v,u) lay on an optimal
//                      extension (training signal for the ordering network)
//   oracle_mcs_goal    one goal-directed search (Section IV-A, top-down
//                      strategy): the incumbent starts at a floor with no
//                      mapping, and the search stops once it reaches a cap
//   oracle_mcs_topdown the top-down strategy of Section IV-A: one goal-directed
//                      search per goal size min(|V_G|,|V_H|), one less, ...,
//                      until a goal is reached
//   oracle_hr_order    the static vertex order of the portfolio section
//                      (connected components, then a Hellerman-Rarick-style
//                      column order inside each); oracle_mcs_hr runs McSplit
//                      with it in place of the degree order
//   oracle_mcs_restart randomized restarts (Section IV-A): McSplit on an
//                      explicit stack of pending branches (the record of what
//                      is left to visit); when the node count has doubled
//                      since the last new incumbent, the pending branches are
//                      put in a random order and the search goes on from the
//                      first of them
//   oracle_mcs_deadend dead-end forecasting with a bound increase and a binary
//                      search (Section IV-A): the plain search raises its
//                      incumbent size by 1 (or doubles it) after a number of
//                      nodes without improvement; an unreachable raised value
//                      is an upper bound, closed by goal-directed searches
//
// Readings where the paper is silent (the McSplit publication it cites fixes
// them; none of them changes the optimum, only the traversal):
//   * vertices of each graph are renumbered by descending degree (total
//     in+out degree when directed; Section IV-A), ties by lower original index;
//   * the branching class minimises max(|L|,|R|), ties to the class holding
//     the lowest-numbered left vertex; v is the lowest-numbered left vertex of
//     that class; candidates u are tried in ascending number;
//   * directed graphs split each class four ways by the pair of bits
//     (x->v is an arc, v->x is an arc), matched against (y->u, u->y);
//   * a self-loop is part of a vertex's label;
//   * the prune test is bound <= |incumbent| (Algorithm 1), not the looser
//     "smaller than" of the prose around Eq. 1.
#include <algorithm>
#include <chrono>
#include <cstdint>
#include <cstring>
#include <utility>
#include <vector>

namespace {

struct OGraph {
    int n = 0;
    std::vector<uint8_t> a;     // a[i*n+j] = 1 iff arc i->j
    std::vector<int> lab;       // vertex label (0 if unlabelled)
    bool edge(int i, int j) const { return a[(size_t)i * n + j] != 0; }
};

OGraph make_graph(int n, const uint8_t* adj, const int32_t* labels) {
    OGraph g;
    g.n = n;
    g.a.assign(adj, adj + (size_t)n * n);
    g.lab.assign(n, 0);
    if (labels)
        for (int i = 0; i < n; ++i) g.lab[i] = labels[i];
    return g;
}

// Descending (total) degree order, stable by original index (Section IV-A).
std::vector<int> degree_order(const OGraph& g, bool directed) {
    std::vector<int> deg(g.n, 0);
    for (int i = 0; i < g.n; ++i)
        for (int j = 0; j < g.n; ++j) {
            if (i == j) continue;
            if (g.edge(i, j)) deg[i]++;
            if (directed && g.edge(j, i)) deg[i]++;
        }
    std::vector<int> ord(g.n);
    for (int i = 0; i < g.n; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(),
                     [&](int x, int y) { return deg[x] > deg[y]; });
    return ord;
}

// Static order of the portfolio modifications (Section IV-A: block structure
// of the adjacency matrix).  Readings where the text is rough:
//   * components are weakly connected (arcs in either direction), self-loops
//     ignored; a component's "rows" are its vertices with an out-arc, its
//     "columns" those with an in-arc; components go in decreasing
//     rows/columns ratio (0/0 counts as 0, r/0 with r > 0 as infinite), then
//     decreasing size, then increasing lowest vertex;
//   * inside a component the active submatrix starts as its nonzero rows and
//     columns; each step takes the shortest nonempty active rows (fewest
//     nonzeros in active columns), picks the active column with a nonzero in
//     the most of them (ties: lowest vertex), gives it the next position and
//     removes it from the active columns; rows leave once empty.  When no
//     active row is left, the remaining active columns follow in increasing
//     order, then the component's vertices without an in-arc.
// Returns ord with ord[position] = original vertex.
std::vector<int> hr_order(const OGraph& g, bool directed) {
    const int n = g.n;
    auto arc = [&](int i, int j) { return i != j && (g.edge(i, j) || (!directed && g.edge(j, i))); };
    std::vector<int> comp(n, -1);
    std::vector<std::vector<int>> comps;
    for (int s = 0; s < n; ++s) {
        if (comp[s] >= 0) continue;
        std::vector<int> c{s}, stack{s};
        comp[s] = (int)comps.size();
        while (!stack.empty()) {
            int x = stack.back();
            stack.pop_back();
            for (int y = 0; y < n; ++y)
                if (comp[y] < 0 && (arc(x, y) || arc(y, x))) { comp[y] = comp[s]; c.push_back(y); stack.push_back(y); }
        }
        std::sort(c.begin(), c.end());
        comps.push_back(c);
    }
    struct Key { long long rows, cols; int size, low; int idx; };
    std::vector<Key> keys;
    for (int i = 0; i < (int)comps.size(); ++i) {
        Key k{0, 0, (int)comps[i].size(), comps[i][0], i};
        for (int x : comps[i]) {
            bool r = false, c = false;
            for (int y = 0; y < n; ++y) { r |= arc(x, y); c |= arc(y, x); }
            k.rows += r; k.cols += c;
        }
        keys.push_back(k);
    }
    auto ratio_gt = [](const Key& a, const Key& b) {        // a.rows/a.cols > b.rows/b.cols
        auto inf = [](const Key& k) { return k.cols == 0 && k.rows > 0; };
        if (inf(a) || inf(b)) return inf(a) && !inf(b);
        const long long an = a.cols ? a.rows : 0, ad = a.cols ? a.cols : 1;
        const long long bn = b.cols ? b.rows : 0, bd = b.cols ? b.cols : 1;
        return an * bd > bn * ad;
    };
    std::sort(keys.begin(), keys.end(), [&](const Key& a, const Key& b) {
        if (ratio_gt(a, b)) return true;
        if (ratio_gt(b, a)) return false;
        if (a.size != b.size) return a.size > b.size;
        return a.low < b.low;
    });
    std::vector<int> ord;
    for (const Key& k : keys) {
        const std::vector<int>& c = comps[k.idx];
        std::vector<char> colact(n, 0), placed(n, 0);
        for (int x : c)
            for (int y : c) if (arc(y, x)) colact[x] = 1;
        for (;;) {
            int minlen = 1 << 30;
            std::vector<int> len(n, 0);
            for (int r : c) {
                for (int x : c) if (colact[x] && arc(r, x)) ++len[r];
                if (len[r] > 0) minlen = std::min(minlen, len[r]);
            }
            bool any_col = false;
            for (int x : c) any_col |= colact[x] != 0;
            if (!any_col) break;
            if (minlen == (1 << 30)) {                       // no active row: the rest in order
                for (int x : c) if (colact[x]) { ord.push_back(x); placed[x] = 1; colact[x] = 0; }
                break;
            }
            int best = -1, bestc = -1;
            for (int x : c) {
                if (!colact[x]) continue;
                int cnt = 0;
                for (int r : c) if (len[r] == minlen && arc(r, x)) ++cnt;
                if (cnt > bestc) { bestc = cnt; best = x; }
            }
            ord.push_back(best);
            placed[best] = 1;
            colact[best] = 0;
        }
        for (int x : c) if (!placed[x]) ord.push_back(x);
    }
    return ord;
}

OGraph relabel(const OGraph& g, const std::vector<int>& ord) {
    OGraph r;
    r.n = g.n;
    r.a.assign((size_t)g.n * g.n, 0);
    r.lab.assign(g.n, 0);
    for (int i = 0; i < g.n; ++i) {
        r.lab[i] = g.lab[ord[i]];
        for (int j = 0; j < g.n; ++j) r.a[(size_t)i * g.n + j] = g.a[(size_t)ord[i] * g.n + ord[j]];
    }
    return r;
}

// ---------------------------------------------------------------------------
// McSplit (Section II-B; Algorithm 1 without the thread pool)
// ---------------------------------------------------------------------------
struct LabelClass {            // one "bidomain": vertices of G and of H sharing a label
    std::vector<int> L, R;
};

struct BranchRecord {          // filled only by the instrumented run
    int depth;
    int v;                     // renumbered G vertex chosen at this node
    std::vector<int> cands;    // renumbered H vertices tried, in order
    std::vector<int64_t> sub_nodes;   // nodes in each candidate's subtree
    std::vector<int> sub_best;        // best mapping size found inside each subtree
};

struct McSplit {
    const OGraph& G;
    const OGraph& H;
    bool directed;
    int64_t node_limit;
    double time_limit;
    std::chrono::steady_clock::time_point t0;
    int64_t nodes = 0;
    bool aborted = false;
    std::vector<std::pair<int, int>> M, best;
    std::vector<BranchRecord>* log = nullptr;
    int log_max_depth = 0;
    // Goal-directed search (Section IV-A): the incumbent size starts at `floor`
    // without a mapping (a solution must beat it to be recorded), and the
    // search stops as soon as the incumbent reaches `cap` (a solution of the
    // goal size was found).  The plain search has floor 0 and no cap.
    int floor = 0;
    int cap = 1 << 30;
    bool reached = false;
    // Dead-end forecast (Section IV-A): after `dead_threshold` nodes without a
    // new incumbent the incumbent size is raised -- by one, or doubled -- as
    // if a mapping of that size were known (0: off).
    int64_t dead_threshold = 0;
    bool dead_double = false;
    int64_t since = 0;

    int incumbent() const { return std::max((int)best.size(), floor); }

    McSplit(const OGraph& g, const OGraph& h, bool d, int64_t nl, double tl)
        : G(g), H(h), directed(d), node_limit(nl), time_limit(tl),
          t0(std::chrono::steady_clock::now()) {}

    // The part of the "label string" a newly mapped vertex adds to x (Table 1):
    // one bit (adjacent or not) for undirected graphs, two bits when directed.
    int rel(const OGraph& g, int x, int v) const {
        int k = g.edge(x, v) ? 1 : 0;
        if (directed && g.edge(v, x)) k |= 2;
        return k;
    }

    bool out_of_budget() {
        if (node_limit > 0 && nodes > node_limit) return true;
        if (time_limit > 0 && (nodes & 1023) == 0) {
            double s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (s > time_limit) return true;
        }
        return false;
    }

    // Eq. 1: |M| + sum over label classes of min(|L|, |R|).
    int bound(const std::vector<LabelClass>& cl) const {
        int b = (int)M.size();
        for (const auto& c : cl) b += (int)std::min(c.L.size(), c.R.size());
        return b;
    }

    // filterDomain on both graphs (Algorithm 1): drop v and u,
    // then split every class by each vertex's relation to v (in G) / u (in H).
    std::vector<LabelClass> filter(const std::vector<LabelClass>& cl, int v, int u) const {
        std::vector<LabelClass> out;
        const int parts = directed ? 4 : 2;
        for (const auto& c : cl) {
            std::vector<LabelClass> sub(parts);
            for (int x : c.L)
                if (x != v) sub[rel(G, x, v)].L.push_back(x);
            for (int y : c.R)
                if (y != u) sub[rel(H, y, u)].R.push_back(y);
            for (auto& s : sub)
                if (!s.L.empty() && !s.R.empty()) out.push_back(std::move(s));
        }
        return out;
    }

    // One call = one search node (Algorithm 1, procedure Solve).
    void solve(std::vector<LabelClass> cl, int depth) {
        ++nodes;
        if (aborted || out_of_budget()) { aborted = true; return; }
        ++since;
        if ((int)M.size() > incumbent()) {                    // incumbent (Algorithm 1)
            best = M;
            since = 0;
            if ((int)best.size() >= cap) { reached = true; return; }   // goal reached (Section IV-A)
        }
        if (dead_threshold > 0 && since >= dead_threshold) {  // dead end forecast (Section IV-A)
            const int inc = incumbent();
            floor = dead_double ? std::max(inc + 1, 2 * inc) : inc + 1;
            since = 0;
        }
        if (bound(cl) <= incumbent()) return;                 // prune (Algorithm 1, Eq. 1)
        // selectLabelClass (Algorithm 1): smallest max(|L|,|R|), ties to the
        // class with the lowest-numbered left vertex.
        int c = -1, ckey = 0, cmin = 0;
        for (int i = 0; i < (int)cl.size(); ++i) {
            int key = (int)std::max(cl[i].L.size(), cl[i].R.size());
            int mn = *std::min_element(cl[i].L.begin(), cl[i].L.end());
            if (c < 0 || key < ckey || (key == ckey && mn < cmin)) { c = i; ckey = key; cmin = mn; }
        }
        const int v = cmin;                                   // selectVertex (Algorithm 1)
        std::vector<int> cand = cl[c].R;
        std::sort(cand.begin(), cand.end());
        BranchRecord* rec = nullptr;
        size_t rec_idx = 0;
        if (log && depth < log_max_depth) {
            rec_idx = log->size();
            log->push_back(BranchRecord{depth, v, {}, {}, {}});
        }
        for (int u : cand) {                                  // try every u of the class
            std::vector<LabelClass> child = filter(cl, v, u);
            M.emplace_back(v, u);
            int64_t before = nodes;
            int best_before = (int)best.size();
            solve(std::move(child), depth + 1);
            M.pop_back();
            if (log && depth < log_max_depth) {
                rec = &(*log)[rec_idx];
                rec->cands.push_back(u);
                rec->sub_nodes.push_back(nodes - before);
                rec->sub_best.push_back((int)best.size() > best_before ? (int)best.size() : -1);
            }
            if (aborted || reached) return;
        }
        // "G = G \ v" (Algorithm 1): v stays unmatched; only this class loses it.
        auto& L = cl[c].L;
        L.erase(std::find(L.begin(), L.end(), v));
        if (L.empty()) cl.erase(cl.begin() + c);
        solve(std::move(cl), depth);                          // the unmatched-v branch
    }
};

std::vector<LabelClass> initial_classes(const OGraph& G, const OGraph& H) {
    // One class per (label, self-loop) value present in both graphs.
    std::vector<std::pair<int, int>> keys;
    auto key = [](const OGraph& g, int i) { return std::make_pair(g.lab[i], g.edge(i, i) ? 1 : 0); };
    for (int i = 0; i < G.n; ++i) keys.push_back(key(G, i));
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    std::vector<LabelClass> cl;
    for (auto& k : keys) {
        LabelClass c;
        for (int i = 0; i < G.n; ++i) if (key(G, i) == k) c.L.push_back(i);
        for (int j = 0; j < H.n; ++j) if (key(H, j) == k) c.R.push_back(j);
        if (!c.L.empty() && !c.R.empty()) cl.push_back(std::move(c));
    }
    return cl;
}

// ---------------------------------------------------------------------------
// Brute force over injective partial mappings (definition, Section II-A)
// ---------------------------------------------------------------------------
struct Brute {
    const OGraph& G;
    const OGraph& H;
    std::vector<int> mapg;     // mapg[x] = y or -1
    std::vector<char> used;
    std::vector<int> dom;      // mapped G vertices in order
    int best = 0;
    std::vector<int> best_map;
    int64_t leaves = 0;
    Brute(const OGraph& g, const OGraph& h) : G(g), H(h), mapg(g.n, -1), used(h.n, 0) {}

    bool ok(int x, int y) const {
        if (G.lab[x] != H.lab[y]) return false;
        if (G.edge(x, x) != H.edge(y, y)) return false;
        for (int x2 : dom) {
            int y2 = mapg[x2];
            if (G.edge(x, x2) != H.edge(y, y2)) return false;
            if (G.edge(x2, x) != H.edge(y2, y)) return false;
        }
        return true;
    }
    void dfs(int x) {
        if (x == G.n) {
            ++leaves;
            if ((int)dom.size() > best) { best = (int)dom.size(); best_map = mapg; }
            return;
        }
        // counting bound: even mapping every remaining G vertex cannot beat best
        if ((int)dom.size() + (G.n - x) <= best) return;
        for (int y = 0; y < H.n; ++y) {
            if (used[y] || !ok(x, y)) continue;
            used[y] = 1; mapg[x] = y; dom.push_back(x);
            dfs(x + 1);
            dom.pop_back(); mapg[x] = -1; used[y] = 0;
        }
        dfs(x + 1);
    }
};

// ---------------------------------------------------------------------------
// Maximum clique of the modular product graph (Bron-Kerbosch with pivoting)
// ---------------------------------------------------------------------------
struct Bits {
    std::vector<uint64_t> w;
    explicit Bits(int n = 0) : w((n + 63) / 64, 0) {}
    void set(int i) { w[i >> 6] |= 1ull << (i & 63); }
    bool get(int i) const { return (w[i >> 6] >> (i & 63)) & 1; }
    int count() const { int c = 0; for (auto x : w) c += __builtin_popcountll(x); return c; }
    bool any() const { for (auto x : w) if (x) return true; return false; }
};

struct Clique {
    int N;
    std::vector<Bits> adj;
    int best = 0;
    std::vector<int> cur, best_set;

    void bk(Bits P, Bits X) {
        int pc = P.count();
        if (!P.any() && !X.any()) {
            if ((int)cur.size() > best) { best = (int)cur.size(); best_set = cur; }
            return;
        }
        if ((int)cur.size() + pc <= best) return;
        // pivot: vertex of P u X with most neighbours in P
        int piv = -1, pbest = -1;
        for (size_t k = 0; k < P.w.size(); ++k) {
            uint64_t m = P.w[k] | X.w[k];
            while (m) {
                int i = (int)(k * 64 + __builtin_ctzll(m));
                m &= m - 1;
                int c = 0;
                for (size_t q = 0; q < P.w.size(); ++q) c += __builtin_popcountll(P.w[q] & adj[i].w[q]);
                if (c > pbest) { pbest = c; piv = i; }
            }
        }
        for (size_t k = 0; k < P.w.size(); ++k) {
            uint64_t m = P.w[k] & ~adj[piv].w[k];
            while (m) {
                int i = (int)(k * 64 + __builtin_ctzll(m));
                m &= m - 1;
                if (!P.get(i)) continue;
                Bits P2(N), X2(N);
                for (size_t q = 0; q < P.w.size(); ++q) {
                    P2.w[q] = P.w[q] & adj[i].w[q];
                    X2.w[q] = X.w[q] & adj[i].w[q];
                }
                cur.push_back(i);
                bk(P2, X2);
                cur.pop_back();
                P.w[i >> 6] &= ~(1ull << (i & 63));
                X.set(i);
                if ((int)cur.size() + P.count() <= best) return;
            }
        }
    }
};

}  // namespace

extern "C" {

// Checks that (g_idx[i], h_idx[i]), i < k, is an injective partial map whose
// image is a common induced subgraph: equal labels, and for every ordered pair
// (i, j) including i == j, arc g_i->g_j exists iff arc h_i->h_j exists.
// Returns 1 if valid, otherwise a negative reason code.
int oracle_verify(int nG, const uint8_t* adjG, const int32_t* labG,
                  int nH, const uint8_t* adjH, const int32_t* labH,
                  int k, const int32_t* g_idx, const int32_t* h_idx) {
    if (k < 0 || k > nG || k > nH) return -1;
    std::vector<char> ug(nG, 0), uh(nH, 0);
    for (int i = 0; i < k; ++i) {
        int x = g_idx[i], y = h_idx[i];
        if (x < 0 || x >= nG || y < 0 || y >= nH) return -2;    // out of range
        if (ug[x] || uh[y]) return -3;                          // not injective
        ug[x] = uh[y] = 1;
        int lx = labG ? labG[x] : 0, ly = labH ? labH[y] : 0;
        if (lx != ly) return -4;                                // label mismatch
    }
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            uint8_t eg = adjG[(size_t)g_idx[i] * nG + g_idx[j]] != 0;
            uint8_t eh = adjH[(size_t)h_idx[i] * nH + h_idx[j]] != 0;
            if (eg != eh) return i == j ? -6 : -5;              // loop / edge mismatch
        }
    return 1;
}

// Sequential McSplit.  Returns the size of the best mapping found and writes
// it (original vertex numbers) to out_g/out_h (capacity min(nG,nH)).
// *status = 0 when the search completed (optimum proven), 1 when the node or
// time limit stopped it (then the size is a lower bound).  *nodes = number of
// calls of the recursive procedure (one per search node, Algorithm 1).
int oracle_mcs(int nG, const uint8_t* adjG, const int32_t* labG,
               int nH, const uint8_t* adjH, const int32_t* labH,
               int directed, int64_t node_limit, double time_limit_s,
               int32_t* out_g, int32_t* out_h, int64_t* nodes, int* status) {
    OGraph g0 = make_graph(nG, adjG, labG), h0 = make_graph(nH, adjH, labH);
    std::vector<int> og = degree_order(g0, directed != 0), oh = degree_order(h0, directed != 0);
    OGraph G = relabel(g0, og), H = relabel(h0, oh);
    McSplit s(G, H, directed != 0, node_limit, time_limit_s);
    s.solve(initial_classes(G, H), 0);
    int k = (int)s.best.size();
    for (int i = 0; i < k; ++i) {
        if (out_g) out_g[i] = og[s.best[i].first];
        if (out_h) out_h[i] = oh[s.best[i].second];
    }
    if (nodes) *nodes = s.nodes;
    if (status) *status = s.aborted ? 1 : 0;
    return k;
}

// One goal-directed McSplit search (Section IV-A, top-down strategy): the
// incumbent size starts at `floor` with no mapping, so only a mapping larger
// than `floor` is recorded, and the search stops once the incumbent reaches
// `cap`.  Returns the size of the best mapping recorded (0 when none beat the
// floor) and writes it like oracle_mcs; *status = 0 when the search ended by
// itself (completed, or stopped at the cap), 1 when a limit stopped it.
int oracle_mcs_goal(int nG, const uint8_t* adjG, const int32_t* labG,
                    int nH, const uint8_t* adjH, const int32_t* labH,
                    int directed, int floor, int cap, int64_t node_limit, double time_limit_s,
                    int32_t* out_g, int32_t* out_h, int64_t* nodes, int* status) {
    OGraph g0 = make_graph(nG, adjG, labG), h0 = make_graph(nH, adjH, labH);
    std::vector<int> og = degree_order(g0, directed != 0), oh = degree_order(h0, directed != 0);
    OGraph G = relabel(g0, og), H = relabel(h0, oh);
    McSplit s(G, H, directed != 0, node_limit, time_limit_s);
    s.floor = floor;
    s.cap = cap;
    s.solve(initial_classes(G, H), 0);
    int k = (int)s.best.size();
    for (int i = 0; i < k; ++i) {
        if (out_g) out_g[i] = og[s.best[i].first];
        if (out_h) out_h[i] = oh[s.best[i].second];
    }
    if (nodes) *nodes = s.nodes;
    if (status) *status = s.aborted ? 1 : 0;
    return k;
}

// The top-down strategy (Section IV-A): goal-directed searches for the goal
// sizes k = min(|V_G|, |V_H|), k - 1, ..., 1, each with floor k - 1 and cap k,
// from the root; the first goal reached is the maximum (every larger goal was
// proven unreachable).  With an empty graph it is the plain search.  Returns
// the size (0 when no goal is reached), the mapping as oracle_mcs, *nodes
// summed over the goal searches, *status as oracle_mcs (1: a limit stopped it;
// then the size is that of a recorded mapping, 0 when none).
int oracle_mcs_topdown(int nG, const uint8_t* adjG, const int32_t* labG,
                       int nH, const uint8_t* adjH, const int32_t* labH,
                       int directed, int64_t node_limit, double time_limit_s,
                       int32_t* out_g, int32_t* out_h, int64_t* nodes, int* status) {
    OGraph g0 = make_graph(nG, adjG, labG), h0 = make_graph(nH, adjH, labH);
    std::vector<int> og = degree_order(g0, directed != 0), oh = degree_order(h0, directed != 0);
    OGraph G = relabel(g0, og), H = relabel(h0, oh);
    const int kmax = std::min(nG, nH);
    const auto t0 = std::chrono::steady_clock::now();
    int64_t total = 0;
    int k = 0, st = 0;
    std::vector<std::pair<int, int>> best;
    for (int goal = kmax; goal >= (kmax > 0 ? 1 : 0); --goal) {
        double left = 0.0;
        if (time_limit_s > 0) {
            left = time_limit_s - std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (left <= 0) { st = 1; break; }
        }
        int64_t nl = 0;
        if (node_limit > 0) {
            nl = node_limit - total;
            if (nl <= 0) { st = 1; break; }
        }
        McSplit s(G, H, directed != 0, nl, left);
        if (kmax > 0) { s.floor = goal - 1; s.cap = goal; }
        s.solve(initial_classes(G, H), 0);
        total += s.nodes;
        if (!s.best.empty() || kmax == 0) { best = s.best; k = (int)best.size(); }
        if (s.aborted) { st = 1; break; }
        if (k > 0 || kmax == 0) break;          // the goal was reached
    }
    for (int i = 0; i < k; ++i) {
        if (out_g) out_g[i] = og[best[i].first];
        if (out_h) out_h[i] = oh[best[i].second];
    }
    if (nodes) *nodes = total;
    if (status) *status = st;
    return k;
}

// Dead-end forecasting with a bound increase (Section IV-A).  The plain search
// runs with the forecast on (raise by one, or double when `doubling`, after
// `threshold` nodes without a new incumbent).  When it ends, a recorded
// mapping larger than the last raised value is optimal.  Otherwise the raised
// value U is an upper bound and the best recorded mapping size L a lower
// bound, and a binary search closes [L, U]: a goal-directed search (floor
// m - 1, cap m) for m = ceil((L + U) / 2) sets L = m when it reaches m, else
// U = m - 1.  Returns the optimum with its mapping as oracle_mcs; *nodes sums
// all searches; *status 1 when a limit stopped it (then the size is the best
// recorded mapping's).
int oracle_mcs_deadend(int nG, const uint8_t* adjG, const int32_t* labG,
                       int nH, const uint8_t* adjH, const int32_t* labH,
                       int directed, int64_t threshold, int doubling,
                       int64_t node_limit, double time_limit_s,
                       int32_t* out_g, int32_t* out_h, int64_t* nodes, int* status) {
    OGraph g0 = make_graph(nG, adjG, labG), h0 = make_graph(nH, adjH, labH);
    std::vector<int> og = degree_order(g0, directed != 0), oh = degree_order(h0, directed != 0);
    OGraph G = relabel(g0, og), H = relabel(h0, oh);
    const auto t0 = std::chrono::steady_clock::now();
    auto left = [&](double lim) {
        return lim > 0 ? lim - std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() : 0.0;
    };
    McSplit s(G, H, directed != 0, node_limit, time_limit_s);
    s.dead_threshold = threshold;
    s.dead_double = doubling != 0;
    s.solve(initial_classes(G, H), 0);
    int64_t total = s.nodes;
    int st = s.aborted ? 1 : 0;
    std::vector<std::pair<int, int>> best = s.best;
    int lo = (int)best.size();
    int hi = std::max(lo, s.floor);
    while (!st && lo < hi) {
        const int m = (lo + hi + 1) / 2;
        const double tl = left(time_limit_s);
        const int64_t nl = node_limit > 0 ? node_limit - total : 0;
        if ((time_limit_s > 0 && tl <= 0) || (node_limit > 0 && nl <= 0)) { st = 1; break; }
        McSplit q(G, H, directed != 0, nl, tl);
        q.floor = m - 1;
        q.cap = m;
        q.solve(initial_classes(G, H), 0);
        total += q.nodes;
        if ((int)q.best.size() >= m) { lo = m; best = q.best; }
        else if (q.aborted) st = 1;
        else hi = m - 1;
    }
    const int k = (int)best.size();
    for (int i = 0; i < k; ++i) {
        if (out_g) out_g[i] = og[best[i].first];
        if (out_h) out_h[i] = oh[best[i].second];
    }
    if (nodes) *nodes = total;
    if (status) *status = st;
    return k;
}

// The static order of hr_order for one graph: out_perm[position] = vertex.
void oracle_hr_order(int n, const uint8_t* adj, int directed, int32_t* out_perm) {
    OGraph g = make_graph(n, adj, nullptr);
    std::vector<int> ord = hr_order(g, directed != 0);
    for (int i = 0; i < n; ++i) out_perm[i] = ord[i];
}

// oracle_mcs with the hr_order renumbering of both graphs in place of the
// degree order (everything else identical).
int oracle_mcs_hr(int nG, const uint8_t* adjG, const int32_t* labG,
                  int nH, const uint8_t* adjH, const int32_t* labH,
                  int directed, int64_t node_limit, double time_limit_s,
                  int32_t* out_g, int32_t* out_h, int64_t* nodes, int* status) {
    OGraph g0 = make_graph(nG, adjG, labG), h0 = make_graph(nH, adjH, labH);
    std::vector<int> og = hr_order(g0, directed != 0), oh = hr_order(h0, directed != 0);
    OGraph G = relabel(g0, og), H = relabel(h0, oh);
    McSplit s(G, H, directed != 0, node_limit, time_limit_s);
    s.solve(initial_classes(G, H), 0);
    int k = (int)s.best.size();
    for (int i = 0; i < k; ++i) {
        if (out_g) out_g[i] = og[s.best[i].first];
        if (out_h) out_h[i] = oh[s.best[i].second];
    }
    if (nodes) *nodes = s.nodes;
    if (status) *status = s.aborted ? 1 : 0;
    return k;
}

// SplitMix64 (Steele, Lea, Flood 2014), one output per counter value.
static uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Randomized restarts (Section IV-A).  The recursion of oracle_mcs written as
// an explicit stack of pending branches: a branch is a node already entered
// (incumbent test, Eq. 1 bound, class and v chosen) with the candidates u
// still to try and whether its "v unmatched" branch is still to do.  The
// stack is the record of every part of the tree not yet visited, so the order
// in which branches are taken does not change the optimum.  A restart fires
// when the node count reaches twice the count at the last new incumbent (and
// at least min_nodes): the pending branches are reordered by the keys
// splitmix64(seed + restart index * 2^32 + position) and the search goes on.
// Returns the optimum and mapping as oracle_mcs; *restarts counts restarts.
int oracle_mcs_restart(int nG, const uint8_t* adjG, const int32_t* labG,
                       int nH, const uint8_t* adjH, const int32_t* labH,
                       int directed, int64_t min_nodes, uint64_t seed,
                       int64_t node_limit, double time_limit_s,
                       int32_t* out_g, int32_t* out_h, int64_t* nodes, int* status, int64_t* restarts) {
    OGraph g0 = make_graph(nG, adjG, labG), h0 = make_graph(nH, adjH, labH);
    std::vector<int> og = degree_order(g0, directed != 0), oh = degree_order(h0, directed != 0);
    OGraph G = relabel(g0, og), H = relabel(h0, oh);
    McSplit s(G, H, directed != 0, node_limit, time_limit_s);   // filter, bound and limits
    struct Branch {
        std::vector<LabelClass> cl;
        std::vector<std::pair<int, int>> M;
        int c, v;
        std::vector<int> cand;          // candidates u still to try, next at the back
        bool unmatched;                 // the "v unmatched" branch is still to do
    };
    std::vector<Branch> stack;
    int64_t mark = 0, nrestart = 0;
    // node entry (Algorithm 1): incumbent, Eq. 1 bound, selection; a branch when not pruned
    auto enter = [&](std::vector<LabelClass> cl, std::vector<std::pair<int, int>> M) {
        ++s.nodes;
        if (s.aborted || s.out_of_budget()) { s.aborted = true; return; }
        s.M = M;
        if (M.size() > s.best.size()) { s.best = M; mark = s.nodes; }
        if (s.bound(cl) <= (int)s.best.size()) return;
        int c = -1, ckey = 0, cmin = 0;
        for (int i = 0; i < (int)cl.size(); ++i) {
            int key = (int)std::max(cl[i].L.size(), cl[i].R.size());
            int mn = *std::min_element(cl[i].L.begin(), cl[i].L.end());
            if (c < 0 || key < ckey || (key == ckey && mn < cmin)) { c = i; ckey = key; cmin = mn; }
        }
        std::vector<int> cand = cl[c].R;
        std::sort(cand.rbegin(), cand.rend());            // ascending order, taken from the back
        stack.push_back(Branch{std::move(cl), std::move(M), c, cmin, std::move(cand), true});
    };
    enter(initial_classes(G, H), {});
    while (!stack.empty() && !s.aborted) {
        if (s.nodes >= std::max(min_nodes, 2 * mark) && stack.size() > 1) {
            // restart: a random order of the pending branches (every one is kept)
            std::vector<std::pair<uint64_t, size_t>> key(stack.size());
            for (size_t i = 0; i < stack.size(); ++i)
                key[i] = {splitmix64(seed + ((uint64_t)nrestart << 32) + i), i};
            std::sort(key.begin(), key.end());
            std::vector<Branch> shuffled;
            for (auto& k : key) shuffled.push_back(std::move(stack[k.second]));
            stack = std::move(shuffled);
            ++nrestart;
            mark = s.nodes;
        }
        Branch& b = stack.back();
        if (!b.cand.empty()) {
            const int u = b.cand.back();
            b.cand.pop_back();
            std::vector<LabelClass> child = s.filter(b.cl, b.v, u);
            std::vector<std::pair<int, int>> M = b.M;
            M.emplace_back(b.v, u);
            enter(std::move(child), std::move(M));
        } else if (b.unmatched) {
            b.unmatched = false;
            std::vector<LabelClass> cl = b.cl;
            auto& L = cl[b.c].L;
            L.erase(std::find(L.begin(), L.end(), b.v));
            if (L.empty()) cl.erase(cl.begin() + b.c);
            std::vector<std::pair<int, int>> M = b.M;
            stack.pop_back();
            enter(std::move(cl), std::move(M));
        } else {
            stack.pop_back();
        }
    }
    const int k = (int)s.best.size();
    for (int i = 0; i < k; ++i) {
        if (out_g) out_g[i] = og[s.best[i].first];
        if (out_h) out_h[i] = oh[s.best[i].second];
    }
    if (nodes) *nodes = s.nodes;
    if (status) *status = s.aborted ? 1 : 0;
    if (restarts) *restarts = nrestart;
    return k;
}

// Exhaustive enumeration of injective partial maps (with only the trivial
// counting cut).  For tiny graphs (n <= 9 or so).  Returns the maximum size.
int oracle_bruteforce(int nG, const uint8_t* adjG, const int32_t* labG,
                      int nH, const uint8_t* adjH, const int32_t* labH,
                      int32_t* out_g, int32_t* out_h) {
    OGraph G = make_graph(nG, adjG, labG), H = make_graph(nH, adjH, labH);
    Brute b(G, H);
    b.dfs(0);
    int k = 0;
    for (int x = 0; x < nG && !b.best_map.empty(); ++x)
        if (b.best_map[x] >= 0) {
            if (out_g) out_g[k] = x;
            if (out_h) out_h[k] = b.best_map[x];
            ++k;
        }
    return b.best;
}

// Maximum common induced subgraph size as the maximum clique of the modular
// product: vertices (x, y) with equal label and equal self-loop bit; (x, y)
// and (x', y') adjacent iff x != x', y != y' and both arc directions agree.
int oracle_clique(int nG, const uint8_t* adjG, const int32_t* labG,
                  int nH, const uint8_t* adjH, const int32_t* labH,
                  int32_t* out_g, int32_t* out_h) {
    OGraph G = make_graph(nG, adjG, labG), H = make_graph(nH, adjH, labH);
    std::vector<std::pair<int, int>> V;
    for (int x = 0; x < nG; ++x)
        for (int y = 0; y < nH; ++y)
            if (G.lab[x] == H.lab[y] && G.edge(x, x) == H.edge(y, y)) V.emplace_back(x, y);
    Clique c;
    c.N = (int)V.size();
    c.adj.assign(c.N, Bits(c.N));
    for (int p = 0; p < c.N; ++p)
        for (int q = 0; q < c.N; ++q) {
            int x = V[p].first, y = V[p].second, x2 = V[q].first, y2 = V[q].second;
            if (x == x2 || y == y2) continue;
            if (G.edge(x, x2) == H.edge(y, y2) && G.edge(x2, x) == H.edge(y2, y)) c.adj[p].set(q);
        }
    Bits P(c.N), X(c.N);
    for (int p = 0; p < c.N; ++p) P.set(p);
    if (c.N) c.bk(P, X);
    for (int i = 0; i < (int)c.best_set.size(); ++i) {
        if (out_g) out_g[i] = V[c.best_set[i]].first;
        if (out_h) out_h[i] = V[c.best_set[i]].second;
    }
    return c.best;
}

// Instrumented McSplit for the ordering network's training signal.  For each
// branching node at depth < max_depth it records the chosen v and, for every
// candidate u tried, the nodes spent in (v,u)'s subtree and whether a new
// incumbent was found inside it.  Records are written as flat int64 rows:
//   [depth, v, u, sub_nodes, improved_to (or -1), cand_rank]
// in renumbered (degree-order) vertex ids, plus the two renumberings in
// perm_g/perm_h (perm[i] = original id of renumbered vertex i).  Returns the
// number of rows written (at most max_rows); *size gets the optimum.
int64_t oracle_branch_log(int nG, const uint8_t* adjG, const int32_t* labG,
                          int nH, const uint8_t* adjH, const int32_t* labH,
                          int directed, int max_depth, int64_t node_limit,
                          int64_t* rows, int64_t max_rows,
                          int32_t* perm_g, int32_t* perm_h, int* size, int* status) {
    OGraph g0 = make_graph(nG, adjG, labG), h0 = make_graph(nH, adjH, labH);
    std::vector<int> og = degree_order(g0, directed != 0), oh = degree_order(h0, directed != 0);
    OGraph G = relabel(g0, og), H = relabel(h0, oh);
    McSplit s(G, H, directed != 0, node_limit, 0.0);
    std::vector<BranchRecord> log;
    s.log = &log;
    s.log_max_depth = max_depth;
    s.solve(initial_classes(G, H), 0);
    int64_t r = 0;
    for (const auto& rec : log)
        for (size_t i = 0; i < rec.cands.size() && r < max_rows; ++i, ++r) {
            int64_t* row = rows + r * 6;
            row[0] = rec.depth; row[1] = rec.v; row[2] = rec.cands[i];
            row[3] = rec.sub_nodes[i]; row[4] = rec.sub_best[i]; row[5] = (int64_t)i;
        }
    for (int i = 0; i < nG; ++i) if (perm_g) perm_g[i] = og[i];
    for (int i = 0; i < nH; ++i) if (perm_h) perm_h[i] = oh[i];
    if (size) *size = (int)s.best.size();
    if (status) *status = s.aborted ? 1 : 0;
    return r;
}

// Applies filterDomain for the pairs (g_seq[t], h_seq[t]), t < k, one after
// the other, starting from the initial label classes, without renumbering.
// After each step t it writes Eq. 1's bound to bounds[t] and, for every
// unmatched vertex, the index of the class holding it (or -1 when its class
// was dropped) to cls_g[t*nG + x] / cls_h[t*nH + y].  Class indices are
// positions in the class list, so only the partition is meaningful.  Used to
// pin the split and the bound against the worked example of Table 1.
int oracle_split_trace(int nG, const uint8_t* adjG, const int32_t* labG,
                       int nH, const uint8_t* adjH, const int32_t* labH,
                       int directed, int k, const int32_t* g_seq, const int32_t* h_seq,
                       int32_t* bounds, int32_t* cls_g, int32_t* cls_h) {
    OGraph G = make_graph(nG, adjG, labG), H = make_graph(nH, adjH, labH);
    McSplit s(G, H, directed != 0, 0, 0.0);
    std::vector<LabelClass> cl = initial_classes(G, H);
    for (int t = 0; t < k; ++t) {
        cl = s.filter(cl, g_seq[t], h_seq[t]);
        s.M.emplace_back(g_seq[t], h_seq[t]);
        bounds[t] = s.bound(cl);
        for (int x = 0; x < nG; ++x) cls_g[(size_t)t * nG + x] = -1;
        for (int y = 0; y < nH; ++y) cls_h[(size_t)t * nH + y] = -1;
        for (int c = 0; c < (int)cl.size(); ++c) {
            for (int x : cl[c].L) cls_g[(size_t)t * nG + x] = c;
            for (int y : cl[c].R) cls_h[(size_t)t * nH + y] = c;
        }
    }
    return (int)cl.size();
}

}  // extern "C"
