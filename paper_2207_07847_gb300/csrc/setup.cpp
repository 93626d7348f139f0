// Host setup of the solver: input validation, the aggregation hierarchy
// (Section 2.2), the tree-ordered storage layout, the elimination data of the
// multilevel sparsifier T (Section 3.3), the top-level pseudo-inverse and, for
// PEGP, the Laplacian of the positively weighted expanded graph H (Section 3.2).
#include <algorithm>
#include <memory>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <thread>
#include <utility>

#include "lap_internal.h"

namespace lap {
namespace {

// Host worker threads for the setup loops whose results do not depend on how
// the work is split (each output is computed by one thread, in the same
// order as the sequential loop would): at most 16 (or LAP_SETUP_THREADS from
// the environment), one for small inputs.
int setup_threads(int64_t work)
{
    if (work < (int64_t(1) << 16)) return 1;
    unsigned cap = 16;
    if (const char *e = std::getenv("LAP_SETUP_THREADS")) {
        const long v = std::strtol(e, nullptr, 10);
        if (v >= 1 && v <= 256) cap = static_cast<unsigned>(v);
    }
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    return static_cast<int>(std::min(hw, cap));
}

// fn(t, begin, end) on T contiguous chunks of [0, n); a failed allocation in
// any worker is rethrown on the calling thread.
template <typename Fn>
void parallel_chunks(int64_t n, int T, Fn fn)
{
    if (T <= 1) {
        fn(0, int64_t(0), n);
        return;
    }
    std::atomic<bool> oom{false};
    std::vector<std::thread> th;
    th.reserve(static_cast<size_t>(T));
    for (int t = 0; t < T; ++t)
        th.emplace_back([&, t] {
            try {
                fn(t, n * t / T, n * (t + 1) / T);
            } catch (const std::bad_alloc &) {
                oom = true;
            }
        });
    for (auto &x : th) x.join();
    if (oom) throw std::bad_alloc();
}

}  // namespace

uint64_t splitmix64(uint64_t seed, uint64_t i)
{
    // Steele, Lea & Flood (2014): state advances by the golden gamma, output
    // is the variant-13 finaliser of the state.
    uint64_t z = seed + i * 0x9E3779B97F4A7C15ull;
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z;
}

// ---------------------------------------------------------------------------
// validation
// ---------------------------------------------------------------------------
lap_status validate_csr(int64_t n, const int64_t *rp, const int32_t *ci, const double *w,
                        std::string *why)
{
    auto fail = [&](lap_status s, const char *msg) {
        if (why) *why = msg;
        return s;
    };
    if (n < 2 || !rp || !ci || !w) return fail(LAP_ERR_INVALID_ARG, "n < 2 or null array");
    if (n >= (int64_t(1) << 31) - 1) return fail(LAP_ERR_UNSUPPORTED, "n >= 2^31");
    if (rp[0] != 0) return fail(LAP_ERR_INVALID_ARG, "row_ptr[0] != 0");
    for (int64_t u = 0; u < n; ++u)
        if (rp[u + 1] < rp[u]) return fail(LAP_ERR_INVALID_ARG, "row_ptr decreasing");
    const int64_t nnz = rp[n];
    if (nnz >= (int64_t(1) << 31)) return fail(LAP_ERR_UNSUPPORTED, "nnz >= 2^31");
    // three passes over the rows, each split over the host threads; a pass
    // reports the failure of its smallest failing row (as one sequential scan
    // would), and the passes run in order
    const int T = setup_threads(nnz);
    std::vector<int64_t> bad_row(static_cast<size_t>(T));
    std::vector<int> bad_kind(static_cast<size_t>(T));
    auto first_failure = [&](auto row_check) {
        std::fill(bad_row.begin(), bad_row.end(), n);
        parallel_chunks(n, T, [&](int t, int64_t u0, int64_t u1) {
            for (int64_t u = u0; u < u1; ++u) {
                const int k = row_check(u);
                if (k) {
                    bad_row[t] = u;
                    bad_kind[t] = k;
                    return;
                }
            }
        });
        int64_t r = n;
        int k = 0;
        for (int t = 0; t < T; ++t)
            if (bad_row[t] < r) {
                r = bad_row[t];
                k = bad_kind[t];
            }
        return k;
    };
    // entries: columns in range, no self-loops, positive finite weights
    switch (first_failure([&](int64_t u) {
        for (int64_t p = rp[u]; p < rp[u + 1]; ++p) {
            const int64_t v = ci[p];
            if (v < 0 || v >= n) return 1;
            if (v == u) return 2;
            if (!(w[p] > 0.0) || !std::isfinite(w[p])) return 3;
        }
        return 0;
    })) {
    case 1: return fail(LAP_ERR_INVALID_ARG, "column out of range");
    case 2: return fail(LAP_ERR_INVALID_ARG, "self-loop");
    case 3: return fail(LAP_ERR_BAD_WEIGHT, "weight not positive and finite");
    default: break;
    }
    // sorted copy of every row: duplicates and symmetry
    std::vector<std::pair<int32_t, double>> s(static_cast<size_t>(nnz));
    if (first_failure([&](int64_t u) {
            for (int64_t p = rp[u]; p < rp[u + 1]; ++p) s[p] = {ci[p], w[p]};
            auto b = s.begin() + rp[u], e = s.begin() + rp[u + 1];
            std::sort(b, e, [](const auto &x, const auto &y) { return x.first < y.first; });
            for (auto it = b; it + 1 < e; ++it)
                if (it->first == (it + 1)->first) return 1;
            return 0;
        }))
        return fail(LAP_ERR_INVALID_ARG, "duplicate entry");
    if (first_failure([&](int64_t u) {
            for (int64_t p = rp[u]; p < rp[u + 1]; ++p) {
                const int32_t v = s[p].first;
                auto b = s.begin() + rp[v], e = s.begin() + rp[v + 1];
                auto it = std::lower_bound(b, e, static_cast<int32_t>(u),
                                           [](const auto &x, int32_t key) { return x.first < key; });
                if (it == e || it->first != u || it->second != s[p].second) return 1;
            }
            return 0;
        }))
        return fail(LAP_ERR_NOT_SYMMETRIC, "matrix not symmetric");
    // connectivity by breadth-first search
    std::vector<char> seen(static_cast<size_t>(n), 0);
    std::vector<int32_t> queue;
    queue.reserve(static_cast<size_t>(n));
    queue.push_back(0);
    seen[0] = 1;
    for (size_t h = 0; h < queue.size(); ++h) {
        const int32_t u = queue[h];
        for (int64_t p = rp[u]; p < rp[u + 1]; ++p)
            if (!seen[ci[p]]) {
                seen[ci[p]] = 1;
                queue.push_back(ci[p]);
            }
    }
    if (static_cast<int64_t>(queue.size()) != n)
        return fail(LAP_ERR_NOT_CONNECTED, "graph not connected");
    return LAP_OK;
}

// ---------------------------------------------------------------------------
// aggregation hierarchy (Section 2.2)
// ---------------------------------------------------------------------------
namespace {

// Heaviest neighbour of u among those accepted by `eligible`; ties go to the
// smaller id.  Returns -1 when no neighbour is eligible.
template <class Pred>
int32_t heaviest_neighbour(const HostLevel &L, int64_t u, Pred eligible)
{
    int32_t best = -1;
    double best_w = 0.0;
    for (int64_t p = L.rp[u]; p < L.rp[u + 1]; ++p) {
        const int32_t v = L.ci[p];
        if (!eligible(v)) continue;
        const double wv = L.w[p];
        if (best < 0 || wv > best_w || (wv == best_w && v < best)) {
            best = v;
            best_w = wv;
        }
    }
    return best;
}

// Random-order maximal-weight matching of one level; level is 1-based.
int64_t aggregate_level(HostLevel &L, uint64_t seed, int level, bool randomise)
{
    const int64_t n = L.n;
    std::vector<int32_t> visit(static_cast<size_t>(n));
    if (randomise) {
        std::vector<std::pair<uint64_t, int32_t>> key(static_cast<size_t>(n));
        const uint64_t hi = static_cast<uint64_t>(static_cast<uint32_t>(level)) << 32;
        for (int64_t u = 0; u < n; ++u)
            key[u] = {splitmix64(seed, (hi | static_cast<uint64_t>(u)) + 1), static_cast<int32_t>(u)};
        std::sort(key.begin(), key.end());
        for (int64_t i = 0; i < n; ++i) visit[i] = key[i].second;
    } else {
        std::iota(visit.begin(), visit.end(), 0);
    }
    L.agg.assign(static_cast<size_t>(n), -1);
    L.pa.clear();
    L.pb.clear();
    for (int64_t i = 0; i < n; ++i) {
        const int32_t u = visit[i];
        if (L.agg[u] >= 0) continue;
        const int32_t v = heaviest_neighbour(L, u, [&](int32_t x) { return L.agg[x] < 0; });
        if (v < 0) continue;                         // leftover, handled below
        const int32_t id = static_cast<int32_t>(L.pa.size());
        L.agg[u] = L.agg[v] = id;
        L.pa.push_back(u);
        L.pb.push_back(v);
    }
    const int64_t nagg = static_cast<int64_t>(L.pa.size());
    // A leftover saw only aggregated neighbours when it was visited and no later
    // pair can have used it, so its heaviest neighbour is always a matched vertex.
    for (int64_t u = 0; u < n; ++u) {
        if (L.agg[u] >= 0) continue;
        const int32_t v = heaviest_neighbour(L, u, [](int32_t) { return true; });
        L.agg[u] = L.agg[v];
    }
    return nagg;
}

// Deterministic parallel matching (a method change against the paper's
// random-order greedy pass, chosen with LAP_MATCH_HANDSHAKE): in rounds, every
// unmatched vertex points at its heaviest unmatched neighbour (ties to the
// smaller id) and two vertices pointing at each other are matched, until no
// unmatched vertex has an unmatched neighbour.  Each round matches at least
// the pair at the heaviest remaining edge: the smallest vertex on an edge of
// that weight points along it, and so does its partner.  Pairs are numbered by
// their smaller end (pa), ascending; leftovers join the aggregate of their
// heaviest neighbour, which is matched.  The rounds' two phases run on the
// host threads; every decision reads only the previous phase's state.
int64_t aggregate_level_handshake(HostLevel &L)
{
    const int64_t n = L.n;
    std::vector<int32_t> mate(static_cast<size_t>(n), -1), cand(static_cast<size_t>(n), -1);
    std::vector<int32_t> active(static_cast<size_t>(n));
    std::iota(active.begin(), active.end(), 0);
    const int T = setup_threads(L.rp[n]);
    while (!active.empty()) {
        const int64_t na = static_cast<int64_t>(active.size());
        parallel_chunks(na, T, [&](int, int64_t a0, int64_t a1) {
            for (int64_t a = a0; a < a1; ++a) {
                const int32_t u = active[a];
                cand[u] = heaviest_neighbour(L, u, [&](int32_t x) { return mate[x] < 0; });
            }
        });
        std::atomic<int64_t> matched{0};
        parallel_chunks(na, T, [&](int, int64_t a0, int64_t a1) {
            int64_t m = 0;
            for (int64_t a = a0; a < a1; ++a) {
                const int32_t u = active[a];
                const int32_t c = cand[u];
                if (c >= 0 && cand[c] == u) {
                    mate[u] = c;
                    ++m;
                }
            }
            matched += m;
        });
        if (matched.load() == 0) break;
        // still unmatched with an unmatched neighbour: the next round's vertices
        std::vector<int32_t> next;
        next.reserve(active.size());
        for (int32_t u : active)
            if (mate[u] < 0 && cand[u] >= 0) next.push_back(u);
        active.swap(next);
    }
    L.agg.assign(static_cast<size_t>(n), -1);
    L.pa.clear();
    L.pb.clear();
    for (int64_t u = 0; u < n; ++u) {
        if (mate[u] > u) {
            const int32_t id = static_cast<int32_t>(L.pa.size());
            L.agg[u] = L.agg[mate[u]] = id;
            L.pa.push_back(static_cast<int32_t>(u));
            L.pb.push_back(mate[u]);
        }
    }
    const int64_t nagg = static_cast<int64_t>(L.pa.size());
    for (int64_t u = 0; u < n; ++u) {
        if (L.agg[u] >= 0) continue;
        const int32_t v = heaviest_neighbour(L, u, [](int32_t) { return true; });
        L.agg[u] = L.agg[v];
    }
    return nagg;
}

// Galerkin coarse graph: weight(I, J) = sum of fine weights between the two
// aggregates, accumulated fine vertex by fine vertex in increasing id and CSR
// position; coarse rows have sorted columns.
void coarse_graph(const HostLevel &F, int64_t nc, HostLevel &C)
{
    const int64_t n = F.n;
    std::vector<int64_t> start(static_cast<size_t>(nc) + 1, 0);
    for (int64_t u = 0; u < n; ++u) ++start[F.agg[u] + 1];
    std::partial_sum(start.begin(), start.end(), start.begin());
    std::vector<int32_t> members(static_cast<size_t>(n));
    {
        std::vector<int64_t> cursor(start.begin(), start.end() - 1);
        for (int64_t u = 0; u < n; ++u) members[cursor[F.agg[u]]++] = static_cast<int32_t>(u);
    }
    C.n = nc;
    // coarse rows by ranges of aggregates; within an aggregate its members
    // are visited in increasing id and their CSR entries in order, so every
    // coarse weight is summed in the same order as one sequential pass
    const int T = setup_threads(F.rp[n]);
    std::vector<std::vector<int32_t>> pci(static_cast<size_t>(T));
    std::vector<std::vector<double>> pw(static_cast<size_t>(T));
    std::vector<int64_t> rowlen(static_cast<size_t>(nc), 0);
    parallel_chunks(nc, T, [&](int t, int64_t I0, int64_t I1) {
        std::vector<double> acc(static_cast<size_t>(nc), 0.0);
        std::vector<int32_t> stamp(static_cast<size_t>(nc), -1);
        std::vector<int32_t> cols;
        for (int64_t I = I0; I < I1; ++I) {
            cols.clear();
            for (int64_t q = start[I]; q < start[I + 1]; ++q) {
                const int32_t u = members[q];
                for (int64_t p = F.rp[u]; p < F.rp[u + 1]; ++p) {
                    const int32_t J = F.agg[F.ci[p]];
                    if (J == I) continue;
                    if (stamp[J] != I) {
                        stamp[J] = static_cast<int32_t>(I);
                        acc[J] = 0.0;
                        cols.push_back(J);
                    }
                    acc[J] += F.w[p];
                }
            }
            std::sort(cols.begin(), cols.end());
            for (int32_t J : cols) {
                pci[t].push_back(J);
                pw[t].push_back(acc[J]);
            }
            rowlen[I] = static_cast<int64_t>(cols.size());
        }
    });
    C.rp.assign(static_cast<size_t>(nc) + 1, 0);
    for (int64_t I = 0; I < nc; ++I) C.rp[I + 1] = C.rp[I] + rowlen[I];
    C.ci.clear();
    C.w.clear();
    C.ci.reserve(static_cast<size_t>(C.rp[nc]));
    C.w.reserve(static_cast<size_t>(C.rp[nc]));
    for (int t = 0; t < T; ++t) {
        C.ci.insert(C.ci.end(), pci[t].begin(), pci[t].end());
        C.w.insert(C.w.end(), pw[t].begin(), pw[t].end());
    }
}

void degrees(HostLevel &L)
{
    L.deg.assign(static_cast<size_t>(L.n), 0.0);
    for (int64_t u = 0; u < L.n; ++u) {
        double d = 0.0;
        for (int64_t p = L.rp[u]; p < L.rp[u + 1]; ++p) d += L.w[p];
        L.deg[u] = d;
    }
}

double edge_weight(const HostLevel &L, int64_t u, int64_t v)
{
    for (int64_t p = L.rp[u]; p < L.rp[u + 1]; ++p)
        if (L.ci[p] == v) return L.w[p];
    return 0.0;
}

// Dense inverse of an SPD matrix by Cholesky (row-major, in place -> out).
bool spd_inverse(std::vector<double> &A, int64_t m)
{
    // A = R^T R with R upper triangular stored in the upper triangle
    for (int64_t j = 0; j < m; ++j) {
        double d = A[j * m + j];
        for (int64_t k = 0; k < j; ++k) d -= A[k * m + j] * A[k * m + j];
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        A[j * m + j] = d;
        for (int64_t i = j + 1; i < m; ++i) {
            double s = A[j * m + i];
            for (int64_t k = 0; k < j; ++k) s -= A[k * m + j] * A[k * m + i];
            A[j * m + i] = s / d;
        }
    }
    // inverse of R (upper triangular) into Ri
    std::vector<double> Ri(static_cast<size_t>(m * m), 0.0);
    for (int64_t j = 0; j < m; ++j) {
        Ri[j * m + j] = 1.0 / A[j * m + j];
        for (int64_t i = j - 1; i >= 0; --i) {
            double s = 0.0;
            for (int64_t k = i + 1; k <= j; ++k) s += A[i * m + k] * Ri[k * m + j];
            Ri[i * m + j] = -s / A[i * m + i];
        }
    }
    // A^{-1} = Ri Ri^T
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < m; ++j) {
            double s = 0.0;
            for (int64_t k = std::max(i, j); k < m; ++k) s += Ri[i * m + k] * Ri[j * m + k];
            A[i * m + j] = s;
        }
    return true;
}

}  // namespace

// ---------------------------------------------------------------------------
// PEGP: Laplacian of H, the positive part of P(mu)^T L P(mu) (Section 3.2).
//
// For u on level k and J on level j >= k the entry of L_Gt is
// (-mu)^(k+j-2) (L_k Pi_{k->j})(u, J), Pi the 0/1 map to level-j ancestors.
// That entry is -W_k(u,J) for a non-ancestor J (W = weight from u into J's
// level-k descendants) and out_{k->j}(u) for u's own ancestor (weight leaving
// that ancestor's subtree).  The edge weight is minus the entry, so H keeps
// all same-level edges, the ancestor edges at odd level distance with
// out > 0, and the non-ancestor edges at even distance.  On two levels this
// is the rule stated for the worked example of Section 3.1.
// ---------------------------------------------------------------------------
namespace {

struct EdgeAcc {
    std::vector<int64_t> i, j;
    std::vector<double> w;
};

void build_pegp(HostModel &m)
{
    const int l = m.levels;
    const double mu = m.mu;
    std::vector<double> mpow(static_cast<size_t>(2 * l + 2), 1.0);
    for (size_t t = 1; t < mpow.size(); ++t) mpow[t] = mpow[t - 1] * mu;
    // expanded index in tree order
    auto xidx = [&](int k, int64_t u) { return m.offset[k] + m.lev[k].pos[u]; };

    // every kept edge is produced once, by the finer endpoint u (same-level
    // edges by their smaller end), with a weight computed from u's row alone;
    // the threads split the vertices of each level, so the edge set and every
    // weight are those of one sequential pass
    std::vector<EdgeAcc> parts;
    for (int k = 0; k < l; ++k) {
        const HostLevel &L = m.lev[k];
        const int T = setup_threads(L.rp[L.n] * (l - k));
        const size_t base = parts.size();
        parts.resize(base + static_cast<size_t>(T));
        parallel_chunks(L.n, T, [&](int t, int64_t u0, int64_t u1) {
            EdgeAcc &E = parts[base + static_cast<size_t>(t)];
            std::vector<int32_t> nbr_anc;   // current ancestor of each neighbour
            std::vector<double> nbr_w;
            std::vector<std::pair<int32_t, double>> grp;
            for (int64_t u = u0; u < u1; ++u) {
                const int64_t deg = L.rp[u + 1] - L.rp[u];
                nbr_anc.resize(static_cast<size_t>(deg));
                nbr_w.resize(static_cast<size_t>(deg));
                for (int64_t q = 0; q < deg; ++q) {
                    nbr_anc[q] = L.ci[L.rp[u] + q];
                    nbr_w[q] = L.w[L.rp[u] + q];
                    // same-level edge (k, k): weight mu^(2k) w; stored once (u < v)
                    if (nbr_anc[q] > u)
                        E.i.push_back(xidx(k, u)), E.j.push_back(xidx(k, nbr_anc[q])),
                            E.w.push_back(mpow[2 * k] * nbr_w[q]);
                }
                int32_t a = static_cast<int32_t>(u);
                for (int j = k + 1; j < l; ++j) {
                    const std::vector<int32_t> &up = m.lev[j - 1].agg;
                    a = up[a];
                    for (int64_t q = 0; q < deg; ++q) nbr_anc[q] = up[nbr_anc[q]];
                    const double scale = mpow[k + j];
                    if ((j - k) % 2 == 1) {
                        double out = 0.0;
                        for (int64_t q = 0; q < deg; ++q)
                            if (nbr_anc[q] != a) out += nbr_w[q];
                        if (out > 0.0)
                            E.i.push_back(xidx(k, u)), E.j.push_back(xidx(j, a)),
                                E.w.push_back(scale * out);
                    } else {
                        grp.clear();
                        for (int64_t q = 0; q < deg; ++q)
                            if (nbr_anc[q] != a) grp.push_back({nbr_anc[q], nbr_w[q]});
                        std::stable_sort(grp.begin(), grp.end(),
                                         [](const auto &x, const auto &y) { return x.first < y.first; });
                        for (size_t s = 0; s < grp.size();) {
                            size_t e = s;
                            double W = 0.0;
                            while (e < grp.size() && grp[e].first == grp[s].first) W += grp[e++].second;
                            E.i.push_back(xidx(k, u)), E.j.push_back(xidx(j, grp[s].first)),
                                E.w.push_back(scale * W);
                            s = e;
                        }
                    }
                }
            }
        });
    }
    // symmetric CSR over the expanded vertices (tree order); every row's
    // columns are distinct, so sorting them fixes the row whatever order the
    // edges arrived in
    const int64_t nt = m.offset[l];
    HostCsr &H = m.LH;
    H.n = nt;
    {
        // rows filled without shared counters: every directed entry first goes
        // to the bucket of the thread that owns its row (T ranges of equal
        // length), producer by producer; then each owner counts and fills its
        // own rows (slot order within a row is then arbitrary; the sort below
        // fixes it)
        const int T = setup_threads(nt);
        const int64_t span = (nt + T - 1) / T;
        auto owner = [&](int64_t row) { return static_cast<int>(row / span); };
        // thread t takes the t-th slice of every part's edges (balanced
        // whatever the parts' sizes)
        auto slice = [&](const EdgeAcc &E, int t) {
            const size_t m = E.i.size();
            return std::make_pair(m * t / T, m * (t + 1) / T);
        };
        std::vector<int64_t> cnt(static_cast<size_t>(T) * T, 0);
        parallel_chunks(T, T, [&](int t, int64_t, int64_t) {
            int64_t *c = cnt.data() + static_cast<size_t>(t) * T;
            for (const EdgeAcc &E : parts) {
                const auto r = slice(E, t);
                for (size_t e = r.first; e < r.second; ++e) {
                    ++c[owner(E.i[e])];
                    ++c[owner(E.j[e])];
                }
            }
        });
        std::vector<int64_t> off(static_cast<size_t>(T) * T, 0), bstart(static_cast<size_t>(T) + 1, 0);
        for (int b = 0; b < T; ++b) {
            int64_t s = 0;
            for (int t = 0; t < T; ++t) {
                off[static_cast<size_t>(t) * T + b] = s;
                s += cnt[static_cast<size_t>(t) * T + b];
            }
            bstart[b + 1] = bstart[b] + s;
        }
        struct Ent {
            int32_t row, col;
            double w;
        };
        // default-initialised storage: every slot is written by the scatter
        // below, whose threads then touch the pages first
        std::unique_ptr<Ent[]> ent(new Ent[static_cast<size_t>(std::max<int64_t>(bstart[T], 1))]);
        parallel_chunks(T, T, [&](int t, int64_t, int64_t) {
            std::vector<int64_t> pos(static_cast<size_t>(T));
            for (int b = 0; b < T; ++b) pos[b] = bstart[b] + off[static_cast<size_t>(t) * T + b];
            for (const EdgeAcc &E : parts) {
                const auto r = slice(E, t);
                for (size_t e = r.first; e < r.second; ++e) {
                    const int32_t i = static_cast<int32_t>(E.i[e]), j = static_cast<int32_t>(E.j[e]);
                    ent[static_cast<size_t>(pos[owner(i)]++)] = {i, j, E.w[e]};
                    ent[static_cast<size_t>(pos[owner(j)]++)] = {j, i, E.w[e]};
                }
            }
        });
        parts.clear();
        parts.shrink_to_fit();
        H.rp.assign(static_cast<size_t>(nt) + 1, 0);
        // owner b writes the lengths of its rows r0 .. r1 - 1 at rp[r + 1]
        parallel_chunks(T, T, [&](int b, int64_t, int64_t) {
            for (int64_t q = bstart[b]; q < bstart[b + 1]; ++q) ++H.rp[static_cast<size_t>(ent[q].row) + 1];
        });
        for (int64_t r = 0; r < nt; ++r) H.rp[r + 1] += H.rp[r];
        H.ci.assign(static_cast<size_t>(H.rp[nt]), 0);
        H.w.assign(static_cast<size_t>(H.rp[nt]), 0.0);
        parallel_chunks(T, T, [&](int b, int64_t, int64_t) {
            const int64_t r0 = std::min(nt, static_cast<int64_t>(b) * span), r1 = std::min(nt, r0 + span);
            std::vector<int64_t> cur(H.rp.begin() + r0, H.rp.begin() + r1);
            for (int64_t q = bstart[b]; q < bstart[b + 1]; ++q) {
                const Ent &x = ent[q];
                const int64_t a = cur[static_cast<size_t>(x.row - r0)]++;
                H.ci[a] = x.col;
                H.w[a] = x.w;
            }
        });
    }
    H.diag.assign(static_cast<size_t>(nt), 0.0);
    parallel_chunks(nt, setup_threads(H.rp[nt]), [&](int, int64_t r0, int64_t r1) {
        std::vector<std::pair<int32_t, double>> row;
        for (int64_t r = r0; r < r1; ++r) {
            row.clear();
            for (int64_t p = H.rp[r]; p < H.rp[r + 1]; ++p) row.push_back({H.ci[p], H.w[p]});
            std::sort(row.begin(), row.end());
            double d = 0.0;
            for (size_t q = 0; q < row.size(); ++q) {
                H.ci[H.rp[r] + q] = row[q].first;
                H.w[H.rp[r] + q] = row[q].second;
                d += row[q].second;
            }
            H.diag[r] = d;
        }
    });
    m.has_LH = true;
}

}  // namespace

// ---------------------------------------------------------------------------
lap_status build_model(int64_t n, const int64_t *rp, const int32_t *ci, const double *w,
                       const lap_options &opt, HostModel &m, void *stream)
{
    m.opt = opt;
    m.mu = opt.mu > 0.0 ? opt.mu : 1.0 / std::sqrt(static_cast<double>(n));
    if (!(m.mu > 0.0 && m.mu < 1.0)) return LAP_ERR_INVALID_ARG;
    if (opt.coarse_max < 1 || opt.max_levels < 0) return LAP_ERR_INVALID_ARG;
    if (opt.setup_device && !opt.host_only) {
        // hierarchy and L_H assembled by device kernels (handshake matching only)
        if (opt.matching != LAP_MATCH_HANDSHAKE) return LAP_ERR_INVALID_ARG;
        return device_build_model(n, rp, ci, w, m, stream);
    }
    build_hierarchy_host(n, rp, ci, w, m);
    const lap_status st = finish_model(m);
    if (st != LAP_OK) return st;
    if (opt.prec == LAP_PREC_PEGP_INNER || opt.prec == LAP_PREC_PEGP_EXACT) build_pegp(m);
    return LAP_OK;
}

// Aggregation hierarchy on the host: levels, aggregates, pairs, degrees and
// out-weights (the fields a device builder fills the same way).
void build_hierarchy_host(int64_t n, const int64_t *rp, const int32_t *ci, const double *w, HostModel &m)
{
    const lap_options &opt = m.opt;
    m.lev.clear();
    m.lev.emplace_back();
    {
        HostLevel &L = m.lev.back();
        L.n = n;
        L.rp.assign(rp, rp + n + 1);
        L.ci.assign(ci, ci + rp[n]);
        L.w.assign(w, w + rp[n]);
        degrees(L);
    }
    for (int k = 1;; ++k) {
        HostLevel &F = m.lev.back();
        if (F.n <= opt.coarse_max) break;
        if (opt.max_levels && k >= opt.max_levels) break;
        if (k >= LAP_MAX_LEVELS) break;
        const int64_t nc = opt.matching == LAP_MATCH_HANDSHAKE
                               ? aggregate_level_handshake(F)
                               : aggregate_level(F, opt.seed, k, opt.order_random != 0);
        if (nc < 2) {
            F.agg.clear();
            F.pa.clear();
            F.pb.clear();
            break;
        }
        HostLevel C;
        coarse_graph(F, nc, C);
        degrees(C);
        // weight from each vertex to other aggregates (no cancellation)
        F.out.assign(static_cast<size_t>(F.n), 0.0);
        for (int64_t u = 0; u < F.n; ++u) {
            double o = 0.0;
            for (int64_t p = F.rp[u]; p < F.rp[u + 1]; ++p)
                if (F.agg[F.ci[p]] != F.agg[u]) o += F.w[p];
            F.out[u] = o;
        }
        m.lev.push_back(std::move(C));
    }
}

// Everything after the hierarchy but L_H: tree order, the sparsifier's
// elimination data, the level-1 Laplacian in tree order, the dense top-level
// pseudo-inverse and T's edge count.
lap_status finish_model(HostModel &m)
{
    const int l = static_cast<int>(m.lev.size());
    m.levels = l;
    m.offset.assign(static_cast<size_t>(l) + 1, 0);
    for (int k = 0; k < l; ++k) m.offset[k + 1] = m.offset[k] + m.lev[k].n;
    m.c.assign(static_cast<size_t>(l), 1.0);
    for (int k = 1; k < l; ++k) m.c[k] = m.c[k - 1] + std::pow(-m.mu, k);

    // ---- tree order, top level down -------------------------------------
    {
        HostLevel &T = m.lev[l - 1];
        T.perm.resize(static_cast<size_t>(T.n));
        std::iota(T.perm.begin(), T.perm.end(), 0);
        T.pos = T.perm;
    }
    m.msp.assign(static_cast<size_t>(l > 1 ? l - 1 : 0), HostMspLevel{});
    for (int k = l - 2; k >= 0; --k) {
        HostLevel &F = m.lev[k];
        const HostLevel &C = m.lev[k + 1];
        const int64_t nagg = C.n;
        // leftovers of each aggregate in increasing id
        std::vector<int64_t> lstart(static_cast<size_t>(nagg) + 1, 0);
        std::vector<char> paired(static_cast<size_t>(F.n), 0);
        for (int64_t J = 0; J < nagg; ++J) paired[F.pa[J]] = paired[F.pb[J]] = 1;
        for (int64_t u = 0; u < F.n; ++u)
            if (!paired[u]) ++lstart[F.agg[u] + 1];
        std::partial_sum(lstart.begin(), lstart.end(), lstart.begin());
        std::vector<int32_t> left(static_cast<size_t>(lstart[nagg]));
        {
            std::vector<int64_t> cur(lstart.begin(), lstart.end() - 1);
            for (int64_t u = 0; u < F.n; ++u)
                if (!paired[u]) left[cur[F.agg[u]]++] = static_cast<int32_t>(u);
        }
        HostMspLevel &S = m.msp[k];
        S.n = F.n;
        S.nagg = nagg;
        S.seg.assign(static_cast<size_t>(nagg) + 1, 0);
        S.inv.assign(static_cast<size_t>(4 * nagg), 0.0);
        S.lcf.assign(static_cast<size_t>(3 * (F.n - 2 * nagg)), 0.0);
        F.perm.clear();
        F.perm.reserve(static_cast<size_t>(F.n));
        const double s = std::pow(m.mu, 2 * k);        // level scaling mu^(2(k-1)), 1-based
        const double pw = std::pow(m.mu, 2 * k + 1);   // parent-edge scaling mu^(2k-1)
        for (int64_t Jp = 0; Jp < nagg; ++Jp) {
            const int32_t J = C.perm[Jp];
            const int32_t a = F.pa[J], b = F.pb[J];
            S.seg[Jp] = static_cast<int32_t>(F.perm.size());
            F.perm.push_back(a);
            F.perm.push_back(b);
            // Elimination of T restricted to this aggregate (Section 3.3):
            // M = s L_intra + pw diag(out).  Leftovers touch only a and b, so
            // eliminating them leaves a 2x2 Schur complement
            // [[alpha + cpl, -cpl], [-cpl, beta + cpl]] with nonnegative parts.
            // It is solved through the difference and the weighted sum of the
            // pair (coefficients below), never through its inverse, whose
            // entries are all ~ 1/(alpha + beta) for weakly coupled pairs.
            const double wab = edge_weight(F, a, b);
            double alpha = pw * F.out[a], beta = pw * F.out[b], cpl = s * wab;
            for (int64_t t = lstart[J]; t < lstart[J + 1]; ++t) {
                const int32_t lu = left[t];
                const double wla = edge_weight(F, lu, a), wlb = edge_weight(F, lu, b);
                const double po = pw * F.out[lu];
                const double d = s * (wla + wlb) + po;
                const int64_t li = static_cast<int64_t>(F.perm.size()) - 2 * (Jp + 1);
                S.lcf[3 * li + 0] = s * wla / d;
                S.lcf[3 * li + 1] = s * wlb / d;
                S.lcf[3 * li + 2] = 1.0 / d;
                alpha += s * wla * po / d;
                beta += s * wlb * po / d;
                cpl += s * wla * s * wlb / d;
                F.perm.push_back(lu);
            }
            const double det = alpha * beta + cpl * (alpha + beta);
            S.inv[4 * Jp + 0] = beta / det;               // delta_a - delta_b =
            S.inv[4 * Jp + 1] = alpha / det;              //   (beta h_a - alpha h_b) / det
            S.inv[4 * Jp + 2] = 1.0 / (alpha + beta);     // delta_b = (h_a + h_b - alpha D)
            S.inv[4 * Jp + 3] = alpha / (alpha + beta);   //           / (alpha + beta)
        }
        S.seg[nagg] = static_cast<int32_t>(F.perm.size());
        F.pos.assign(static_cast<size_t>(F.n), 0);
        for (int64_t i = 0; i < F.n; ++i) F.pos[F.perm[i]] = static_cast<int32_t>(i);
    }

    // ---- level-1 Laplacian in tree order ---------------------------------
    {
        const HostLevel &F = m.lev[0];
        HostCsr &A = m.L1;
        A.n = F.n;
        A.rp.assign(static_cast<size_t>(F.n) + 1, 0);
        A.ci.resize(F.ci.size());
        A.w.resize(F.w.size());
        A.diag.resize(static_cast<size_t>(F.n));
        for (int64_t i = 0; i < F.n; ++i) {
            const int32_t u = F.perm[i];
            A.rp[i + 1] = A.rp[i] + (F.rp[u + 1] - F.rp[u]);
        }
        // rows on the host threads, each sorted by its (distinct) columns
        parallel_chunks(F.n, setup_threads(A.rp[F.n]), [&](int, int64_t i0, int64_t i1) {
            std::vector<std::pair<int32_t, double>> row;
            for (int64_t i = i0; i < i1; ++i) {
                const int32_t u = F.perm[i];
                row.clear();
                for (int64_t p = F.rp[u]; p < F.rp[u + 1]; ++p) row.push_back({F.pos[F.ci[p]], F.w[p]});
                std::sort(row.begin(), row.end(),
                          [](const auto &x, const auto &y) { return x.first < y.first; });
                for (size_t t = 0; t < row.size(); ++t) {
                    A.ci[A.rp[i] + t] = row[t].first;
                    A.w[A.rp[i] + t] = row[t].second;
                }
                A.diag[i] = F.deg[u];
            }
        });
    }

    // ---- top level: dense pseudo-inverse of mu^(2(l-1)) L_l ---------------
    {
        const HostLevel &T = m.lev[l - 1];
        const int64_t nt = T.n;
        if (nt > 4096) return LAP_ERR_UNSUPPORTED;
        std::vector<double> A(static_cast<size_t>(nt * nt), 1.0 / static_cast<double>(nt));
        for (int64_t u = 0; u < nt; ++u) {
            A[u * nt + u] += T.deg[u];
            for (int64_t p = T.rp[u]; p < T.rp[u + 1]; ++p) A[u * nt + T.ci[p]] -= T.w[p];
        }
        if (!spd_inverse(A, nt)) return LAP_ERR_BREAKDOWN;
        const double inv_s = 1.0 / std::pow(m.mu, 2 * (l - 1));
        for (auto &x : A) x = (x - 1.0 / static_cast<double>(nt)) * inv_s;
        m.coarse_pinv = std::move(A);
    }

    // ---- number of edges of T --------------------------------------------
    {
        int64_t e = 0;
        for (int k = 0; k + 1 < l; ++k) {
            const HostLevel &F = m.lev[k];
            const int T = setup_threads(F.rp[F.n]);
            std::vector<int64_t> part(static_cast<size_t>(T), 0);
            parallel_chunks(F.n, T, [&](int t, int64_t u0, int64_t u1) {
                int64_t c = 0;
                for (int64_t u = u0; u < u1; ++u) {
                    if (F.out[u] > 0.0) ++c;                           // parent edge
                    for (int64_t p = F.rp[u]; p < F.rp[u + 1]; ++p)
                        if (F.ci[p] > u && F.agg[F.ci[p]] == F.agg[u]) ++c;  // intra edge
                }
                part[t] = c;
            });
            for (int64_t c : part) e += c;
        }
        e += m.lev[l - 1].rp[m.lev[l - 1].n] / 2;                  // top level
        m.edges_T = e;
    }
    return LAP_OK;
}

// ---------------------------------------------------------------------------
// Long-row threshold of the SELL layout.  The default is eight times the mean
// row length (at least 64); another candidate is taken only if it stores at
// least a fifth fewer entries, counting each slice padded to its longest
// short row and each long row padded to whole 128-entry groups plus one group
// of overhead (power-law rows: hubs otherwise pad whole slices).
static int64_t choose_long_threshold(const HostCsr &A)
{
    const int64_t n = A.n, ns = (n + 31) / 32;
    auto cost = [&](int64_t T) {
        int64_t c = 0;
        for (int64_t s = 0; s < ns; ++s) {
            int64_t w = 0;
            for (int64_t r = 32 * s; r < std::min(n, 32 * s + 32); ++r) {
                const int64_t d = A.rp[r + 1] - A.rp[r];
                if (d > T) c += (d + 127) / 128 * 128 + 128;
                else w = std::max(w, d);
            }
            c += 32 * w;
        }
        return c;
    };
    const double avg = n > 0 ? static_cast<double>(A.rp[n]) / static_cast<double>(n) : 0.0;
    const int64_t t0 = std::max<int64_t>(64, static_cast<int64_t>(8 * avg));
    const int64_t c0 = cost(t0);
    int64_t best = t0, best_cost = c0;
    for (int64_t T : {32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 2048, 4096}) {
        const int64_t c = cost(T);
        if (c < best_cost) {
            best_cost = c;
            best = T;
        }
    }
    return best_cost * 5 < c0 * 4 ? best : t0;
}

void make_sell(const HostCsr &A, HostSell &S, int64_t long_threshold, int vec)
{
    const int64_t n = A.n;
    if (long_threshold <= 0) long_threshold = choose_long_threshold(A);
    S.n = n;
    S.nslices = (n + 31) / 32;
    S.sptr.assign(static_cast<size_t>(S.nslices) + 1, 0);
    S.longmask.assign(static_cast<size_t>(S.nslices), 0u);
    S.lrow.clear();
    S.lrp.assign(1, 0);
    S.lci.clear();
    S.lw.clear();
    // slot order: within windows of kSigma slices the rows are sorted by
    // decreasing length (stable), so that a slice pads to similar rows; long
    // rows count as empty (their slot is masked)
    const int64_t kWin = 32 * 8;
    auto len = [&](int64_t r) {
        const int64_t d = A.rp[r + 1] - A.rp[r];
        return d > long_threshold ? int64_t(0) : d;
    };
    S.rowperm.assign(static_cast<size_t>(S.nslices) * 32, -1);
    for (int64_t r = 0; r < n; ++r) S.rowperm[r] = static_cast<int32_t>(r);
    auto slices_size = [&]() {
        int64_t t = 0;
        for (int64_t s0 = 0; s0 < n; s0 += 32) {
            int64_t w = 0;
            for (int64_t k = s0; k < std::min(n, s0 + 32); ++k) w = std::max(w, len(S.rowperm[k]));
            t += 32 * w;
        }
        return t;
    };
    const int64_t unsorted = slices_size();
    const int64_t nwin = (n + kWin - 1) / kWin;
    parallel_chunks(nwin, setup_threads(n), [&](int, int64_t v0, int64_t v1) {
        for (int64_t v = v0; v < v1; ++v) {
            const int64_t w0 = v * kWin, w1 = std::min(n, w0 + kWin);
            std::stable_sort(S.rowperm.begin() + w0, S.rowperm.begin() + w1,
                             [&](int32_t a, int32_t b) { return len(a) > len(b); });
        }
    });
    // sorting pays only if it saves padding: else keep the rows in place (an
    // empty rowperm: slot = row)
    const bool sorted = slices_size() * 20 < unsorted * 19;
    if (!sorted)
        for (int64_t r = 0; r < n; ++r) S.rowperm[r] = static_cast<int32_t>(r);
    std::vector<int64_t> width(static_cast<size_t>(S.nslices), 0);
    for (int64_t s = 0; s < S.nslices; ++s) {
        for (int64_t lane = 0; lane < 32; ++lane) {
            const int64_t slot = 32 * s + lane;
            if (slot >= n) break;
            const int64_t r = S.rowperm[slot];
            const int64_t d = A.rp[r + 1] - A.rp[r];
            if (d > long_threshold) {
                S.longmask[s] |= 1u << lane;
                S.lrow.push_back(static_cast<int32_t>(r));
                for (int64_t p = A.rp[r]; p < A.rp[r + 1]; ++p) {
                    S.lci.push_back(A.ci[p]);
                    S.lw.push_back(A.w[p]);
                }
                S.lrp.push_back(static_cast<int64_t>(S.lci.size()));
            } else {
                width[s] = std::max(width[s], d);
            }
        }
    }
    if (vec <= 0) {
        auto size = [&](int v) {
            int64_t t = 0;
            for (int64_t w : width) t += 32 * ((w + v - 1) / v * v);
            return t;
        };
        const int64_t base = size(1);
        vec = 1;
        for (int v : {4, 2})
            if (size(v) * 100 <= base * 106) {
                vec = v;
                break;
            }
    }
    S.vec = vec;
    for (int64_t s = 0; s < S.nslices; ++s) {
        const int64_t w = (width[s] + vec - 1) / vec * vec;
        S.sptr[s + 1] = S.sptr[s] + 32 * w;
    }
    // chunks of the long rows: at most kChunk entries each, padded (column =
    // the row itself, weight 0) to a multiple of 128 entries, so that a warp
    // reads a chunk as groups of 4 consecutive entries per lane; lrp becomes
    // the padded range of each long row
    const int64_t kChunk = 4096;
    S.lchunk_ptr.assign(1, 0);
    S.chunk_row.clear();
    S.chunk_beg.assign(1, 0);
    {
        std::vector<int32_t> ci;
        std::vector<double> w;
        std::vector<int64_t> rp(1, 0);
        for (size_t r = 0; r < S.lrow.size(); ++r) {
            for (int64_t b = S.lrp[r]; b < S.lrp[r + 1]; b += kChunk) {
                const int64_t e = std::min(b + kChunk, S.lrp[r + 1]);
                ci.insert(ci.end(), S.lci.begin() + b, S.lci.begin() + e);
                w.insert(w.end(), S.lw.begin() + b, S.lw.begin() + e);
                while (ci.size() % 128) {
                    ci.push_back(S.lrow[r]);
                    w.push_back(0.0);
                }
                S.chunk_row.push_back(static_cast<int32_t>(r));
                S.chunk_beg.push_back(static_cast<int64_t>(ci.size()));
            }
            S.lchunk_ptr.push_back(static_cast<int32_t>(S.chunk_row.size()));
            rp.push_back(static_cast<int64_t>(ci.size()));
        }
        S.lci.swap(ci);
        S.lw.swap(w);
        S.lrp.swap(rp);
    }
    S.eci.assign(static_cast<size_t>(S.sptr[S.nslices]), 0);
    S.ew.assign(static_cast<size_t>(S.sptr[S.nslices]), 0.0);
    parallel_chunks(S.nslices, setup_threads(S.sptr[S.nslices]), [&](int, int64_t s0, int64_t s1) {
        for (int64_t s = s0; s < s1; ++s) {
            const int64_t w = (S.sptr[s + 1] - S.sptr[s]) / 32;
            for (int64_t lane = 0; lane < 32; ++lane) {
                const int64_t slot = 32 * s + lane;
                const int64_t r = slot < n ? S.rowperm[slot] : -1;
                const bool real = r >= 0 && !((S.longmask[s] >> lane) & 1u);
                const int64_t d = real ? A.rp[r + 1] - A.rp[r] : 0;
                for (int64_t j = 0; j < w; ++j) {
                    const int64_t q = S.sptr[s] + (j / vec) * 32 * vec + lane * vec + j % vec;
                    if (j < d) {
                        S.eci[q] = A.ci[A.rp[r] + j];
                        S.ew[q] = A.w[A.rp[r] + j];
                    } else {
                        S.eci[q] = static_cast<int32_t>(r >= 0 ? r : 0);   // weight 0: no contribution
                    }
                }
            }
        }
    });
    if (!sorted) S.rowperm.clear();
}

// ---------------------------------------------------------------------------
void expanded_edges(const HostModel &m, int which, std::vector<int64_t> &I,
                    std::vector<int64_t> &J, std::vector<double> &W)
{
    I.clear();
    J.clear();
    W.clear();
    const int l = m.levels;
    // tree-order expanded index -> hierarchy expanded index
    std::vector<int64_t> back(static_cast<size_t>(m.offset[l]));
    for (int k = 0; k < l; ++k)
        for (int64_t i = 0; i < m.lev[k].n; ++i) back[m.offset[k] + i] = m.offset[k] + m.lev[k].perm[i];
    std::vector<std::tuple<int64_t, int64_t, double>> e;
    if (which == 0) {
        const HostCsr &H = m.LH;
        for (int64_t r = 0; r < H.n; ++r)
            for (int64_t p = H.rp[r]; p < H.rp[r + 1]; ++p) {
                int64_t a = back[r], b = back[H.ci[p]];
                if (a < b) e.emplace_back(a, b, H.w[p]);
            }
    } else {
        for (int k = 0; k < l; ++k) {
            const HostLevel &F = m.lev[k];
            const double s = std::pow(m.mu, 2 * k);
            for (int64_t u = 0; u < F.n; ++u) {
                for (int64_t p = F.rp[u]; p < F.rp[u + 1]; ++p) {
                    const int32_t v = F.ci[p];
                    if (v <= u) continue;
                    if (k == l - 1 || F.agg[v] == F.agg[u])
                        e.emplace_back(m.offset[k] + u, m.offset[k] + v, s * F.w[p]);
                }
                if (k + 1 < l && F.out[u] > 0.0)
                    e.emplace_back(m.offset[k] + u, m.offset[k + 1] + F.agg[u],
                                   std::pow(m.mu, 2 * k + 1) * F.out[u]);
            }
        }
    }
    std::sort(e.begin(), e.end());
    for (auto &t : e) {
        I.push_back(std::get<0>(t));
        J.push_back(std::get<1>(t));
        W.push_back(std::get<2>(t));
    }
}

// ---------------------------------------------------------------------------
// Band planning (setup).  start[j][P] is the first level-(k0+j) descendant of
// level-k1 vertex P in tree order (start[j][N] = n_{k0+j}): seg of each level
// maps the first aggregate of a range to its first member.
static std::vector<std::vector<int64_t>> band_starts(const HostModel &m, int k0, int k1)
{
    const int L = k1 - k0;
    const int64_t N = m.lev[k1].n;
    std::vector<std::vector<int64_t>> start(static_cast<size_t>(L + 1));
    start[L].resize(static_cast<size_t>(N + 1));
    for (int64_t P = 0; P <= N; ++P) start[L][P] = P;
    for (int j = L - 1; j >= 0; --j) {
        const auto &seg = m.msp[k0 + j].seg;
        start[j].resize(static_cast<size_t>(N + 1));
        for (int64_t P = 0; P <= N; ++P) start[j][P] = seg[start[j + 1][P]];
    }
    return start;
}

// Shared-memory bytes of a tile holding the level-k1 vertices [a, b) with
// values of sv bytes: the largest of its upward layout (packed segments and
// coefficients, then the values of every level), its downward layout
// (segments, the deltas of levels k0..k1-1, the level-k1 values and r of the
// finest level) and the downward layout with deltas read level by level from
// an expanded array.
// Every range copied from global memory is rounded out to 16 bytes.
static int64_t band_need(const std::vector<std::vector<int64_t>> &start, int64_t a, int64_t b, int sv)
{
    const int L = static_cast<int>(start.size()) - 1;
    auto r16 = [](int64_t x) { return (x + 15) / 16 * 16; };
    std::vector<int64_t> c(static_cast<size_t>(L + 1));
    for (int j = 0; j <= L; ++j) c[j] = start[j][b] - start[j][a];
    int64_t segs = 0, coefs = 0, vals_up = 0, vals_dn = 0, dx = 0;
    for (int j = 0; j < L; ++j) {
        segs += c[j + 1] + 1;
        coefs += 4 * c[j + 1] + 3 * (c[j] - 2 * c[j + 1]);
        vals_dn += c[j];
        dx += r16(16 + c[j] * sv);
    }
    for (int j = 1; j <= L; ++j) vals_up += c[j];
    const int64_t seg_bytes = r16(4 * segs);
    const int64_t up = seg_bytes + r16(coefs * sv) + r16(16 + c[0] * sv) + r16(vals_up * sv);
    const int64_t par = r16(16 + c[L] * sv), rfin = r16(16 + c[0] * sv);
    const int64_t down = seg_bytes + r16(vals_dn * sv) + par + rfin;
    const int64_t downx = seg_bytes + dx + par + rfin;
    return std::max(up, std::max(down, downx));
}

// Band tops: from level 0 up, the highest k1 <= min(kmax, k0 + kBandMaxLevels)
// whose oversized subtrees (more than `cap` bytes, run in global memory)
// hold at most a tenth of the band's values; at least one level per band.
std::vector<int> plan_band_tops(const HostModel &m, int kmax, int cap, int sv)
{
    std::vector<int> tops;
    int k0 = 0;
    while (k0 < kmax) {
        int best = k0 + 1;
        for (int k1 = std::min(kmax, k0 + kBandMaxLevels); k1 > k0 + 1; --k1) {
            const auto start = band_starts(m, k0, k1);
            const int64_t N = m.lev[k1].n;
            int64_t big = 0, all = 0;
            for (int64_t P = 0; P < N; ++P) {
                int64_t v = 0;
                for (const auto &st : start) v += st[P + 1] - st[P];
                all += v;
                if (band_need(start, P, P + 1, sv) > cap) big += v;
            }
            if (10 * big <= all) {
                best = k1;
                break;
            }
        }
        tops.push_back(best);
        k0 = best;
    }
    return tops;
}

// Tiles of band [k0, k1): runs of consecutive level-k1 vertices needing at
// most `cap` bytes (one vertex at least).  tab: ntiles + 1 rows of the L + 1
// first indices; fits: per tile, whether it needs at most `cap_fit` bytes
// (else it runs in global memory).
void plan_band_tiles(const HostModel &m, int k0, int k1, int cap, int cap_fit, int sv, std::vector<int> &tab,
                     std::vector<char> &fits, int &ntiles)
{
    const int L = k1 - k0;
    const auto start = band_starts(m, k0, k1);
    const int64_t N = m.lev[k1].n;
    tab.clear();
    fits.clear();
    auto push = [&](int64_t P) {
        for (int j = 0; j <= L; ++j) tab.push_back(static_cast<int>(start[j][P]));
    };
    push(0);
    ntiles = 0;
    for (int64_t P0 = 0; P0 < N;) {
        int64_t P1 = P0 + 1;
        while (P1 < N && band_need(start, P0, P1 + 1, sv) <= cap) ++P1;
        fits.push_back(band_need(start, P0, P1, sv) <= cap_fit ? 1 : 0);
        push(P1);
        ++ntiles;
        P0 = P1;
    }
}


}  // namespace lap
