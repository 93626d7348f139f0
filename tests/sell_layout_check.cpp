// Host check of the SELL-32 layout (make_sell in setup.cpp) used by the
// library's matvecs: for the level-1 Laplacian of a graph and, when it has
// more than one level, the PEGP Laplacian L_H, every row's entries are stored
// exactly once and in CSR order -- in its slice lane or, for a long row, in its
// chunks -- and every padding slot has weight 0 on the row itself.  Built by
// tests/test_sell_layout.py against setup.cpp alone (the two device entry
// points that setup.cpp can call are stubbed: the check runs host-only).
//
// Input: a binary CSR file (int64 n, int64 nnz, int64 row_ptr[n+1],
// int32 col[nnz], double w[nnz]).  Prints one line per matrix, exits non-zero
// on the first violation.
#include <cstdio>
#include <cstring>
#include <vector>

#include "lap_internal.h"

namespace lap {
lap_status device_build_model(int64_t, const int64_t *, const int32_t *, const double *, HostModel &, void *)
{
    return LAP_ERR_UNSUPPORTED;
}
void *dev_alloc(size_t, void *) { return nullptr; }
void dev_free(void *, void *) {}
}  // namespace lap

using namespace lap;

static int fail(const char *what, long long a, long long b)
{
    std::printf("FAIL %s (%lld, %lld)\n", what, a, b);
    return 1;
}

static int check(const char *name, const HostCsr &A)
{
    HostSell S;
    make_sell(A, S, 0);
    const int64_t n = A.n;
    if (S.n != n || S.nslices != (n + 31) / 32) return fail("slice count", S.nslices, n);
    if (S.vec != 1 && S.vec != 2 && S.vec != 4) return fail("vec", S.vec, 0);
    const bool perm = !S.rowperm.empty();
    if (perm && static_cast<int64_t>(S.rowperm.size()) != 32 * S.nslices) return fail("rowperm size", 0, 0);
    std::vector<int> seen(static_cast<size_t>(n), 0);
    std::vector<char> is_long(static_cast<size_t>(n), 0);
    for (int32_t r : S.lrow) {
        if (r < 0 || r >= n) return fail("long row id", r, n);
        is_long[r] = 1;
    }
    for (int64_t s = 0; s < S.nslices; ++s) {
        const int64_t span = S.sptr[s + 1] - S.sptr[s];
        if (span < 0 || span % 32) return fail("slice span", s, span);
        const int64_t w = span / 32;
        if (w % S.vec) return fail("width not a multiple of vec", s, w);
        for (int lane = 0; lane < 32; ++lane) {
            const int64_t slot = 32 * s + lane;
            const int64_t r = perm ? S.rowperm[slot] : (slot < n ? slot : -1);
            if (slot >= n && r != -1) return fail("row beyond n", slot, r);
            const bool masked = (S.longmask[s] >> lane) & 1u;
            if (r >= 0 && masked != static_cast<bool>(is_long[r])) return fail("long mask", r, masked);
            const bool real = r >= 0 && !masked;
            const int64_t d = real ? A.rp[r + 1] - A.rp[r] : 0;
            if (d > w) return fail("row longer than its slice", r, d);
            if (real) ++seen[r];
            for (int64_t j = 0; j < w; ++j) {
                const int64_t q = S.sptr[s] + (j / S.vec) * 32 * S.vec + lane * S.vec + j % S.vec;
                if (j < d) {
                    if (S.eci[q] != A.ci[A.rp[r] + j] || S.ew[q] != A.w[A.rp[r] + j]) return fail("entry", r, j);
                } else if (S.ew[q] != 0.0 || S.eci[q] != (r >= 0 ? r : 0)) {
                    return fail("padding", r, j);
                }
            }
        }
    }
    if (S.lrp.size() != S.lrow.size() + 1 || S.lchunk_ptr.size() != S.lrow.size() + 1) return fail("long sizes", 0, 0);
    for (size_t li = 0; li < S.lrow.size(); ++li) {
        const int64_t r = S.lrow[li], d = A.rp[r + 1] - A.rp[r];
        ++seen[r];
        int64_t real = 0;
        for (int c = S.lchunk_ptr[li]; c < S.lchunk_ptr[li + 1]; ++c) {
            if (S.chunk_row[c] != static_cast<int32_t>(li)) return fail("chunk row", c, li);
            const int64_t b = S.chunk_beg[c], e = S.chunk_beg[c + 1];
            if (b % 128 || e % 128 || e <= b) return fail("chunk bounds", b, e);
            if (c == S.lchunk_ptr[li] && b != S.lrp[li]) return fail("first chunk start", b, S.lrp[li]);
            for (int64_t p = b; p < e; ++p) {
                if (real < d && p - b < 4096) {
                    if (S.lci[p] != A.ci[A.rp[r] + real] || S.lw[p] != A.w[A.rp[r] + real]) return fail("long entry", r, real);
                    ++real;
                } else if (S.lw[p] != 0.0 || S.lci[p] != r) {
                    return fail("long padding", r, p);
                }
            }
        }
        if (real != d) return fail("long row entries", r, real);
        if (S.lrp[li + 1] != S.chunk_beg[S.lchunk_ptr[li + 1]]) return fail("long row end", r, S.lrp[li + 1]);
    }
    for (int64_t r = 0; r < n; ++r)
        if (seen[r] != 1) return fail("row stored once", r, seen[r]);
    std::printf("%s n %lld nnz %lld vec %d slices %lld stored %lld long rows %zu chunks %zu %s\n", name,
                static_cast<long long>(n), static_cast<long long>(A.rp[n]), S.vec, static_cast<long long>(S.nslices),
                static_cast<long long>(S.sptr[S.nslices]), S.lrow.size(), S.chunk_row.size(),
                perm ? "sorted" : "in place");
    return 0;
}

int main(int argc, char **argv)
{
    if (argc < 2) return 9;
    FILE *f = std::fopen(argv[1], "rb");
    if (!f) return 9;
    int64_t n = 0, nnz = 0;
    if (std::fread(&n, 8, 1, f) != 1 || std::fread(&nnz, 8, 1, f) != 1) return 9;
    std::vector<int64_t> rp(static_cast<size_t>(n) + 1);
    std::vector<int32_t> ci(static_cast<size_t>(nnz));
    std::vector<double> w(static_cast<size_t>(nnz));
    if (std::fread(rp.data(), 8, rp.size(), f) != rp.size() || std::fread(ci.data(), 4, ci.size(), f) != ci.size() ||
        std::fread(w.data(), 8, w.size(), f) != w.size())
        return 9;
    std::fclose(f);
    lap_options o;
    std::memset(&o, 0, sizeof(o));
    o.prec = LAP_PREC_PEGP_INNER;
    o.mu = 0.8;
    o.coarse_max = 32;
    o.order_random = 1;
    o.seed = 7;
    o.host_only = 1;
    HostModel m;
    const lap_status st = build_model(n, rp.data(), ci.data(), w.data(), o, m);
    if (st != LAP_OK) {
        std::printf("FAIL build_model %d\n", static_cast<int>(st));
        return 1;
    }
    if (check("L1", m.L1)) return 1;
    if (m.has_LH && check("L_H", m.LH)) return 1;
    return 0;
}
