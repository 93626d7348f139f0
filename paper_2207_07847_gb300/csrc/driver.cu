// Device upload, kernel sequencing and the CG drivers of a solver handle.
//
// Per CG iteration on L (Section 4 recast on n unknowns, see lap.h):
//   k_sell            q = L p, p.q -> alpha
//   k_up_tiled<1>     x += alpha p, r -= alpha q, ||r|| test; level-1 restriction
//                     and elimination of T's finest aggregates (Section 3.3)
//   k_up_tiled<0>     middle levels: restriction + elimination
//   k_msp_tail        the deepest levels up, the top-level pseudo-inverse of
//                     mu^(2(l-1)) L_l, and back down, in one block
//   k_down_tiled      middle levels: back-substitution + prolongation
//   k_down_tiled<1>   z on level 1, sums for the projection and rho/beta
//   k_pupdate         p = Pi z + beta p
// captured as a CUDA graph of `check_every` iterations; every kernel returns at
// once when the device-side convergence flag is set.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <type_traits>

#include "dense.cuh"
#include "fgmres.cuh"
#include "stretch.cuh"
#include "kernels.cuh"
#include "merge.cuh"
#include "solver.cuh"

namespace lap {

#define LAP_CK(x)                                                                             \
    do {                                                                                      \
        cudaError_t e_ = (x);                                                                 \
        if (e_ != cudaSuccess) {                                                              \
            (void)cudaGetLastError();                                                         \
            return e_ == cudaErrorMemoryAllocation ? LAP_ERR_OOM : LAP_ERR_CUDA;              \
        }                                                                                     \
    } while (0)

namespace {

using Clock = std::chrono::steady_clock;

int grid_for(const lap_handle_s &h, int64_t work)
{
    const int64_t b = (work + kBlock - 1) / kBlock;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(b, h.grid_cap)));
}

template <typename T>
T *dalloc(lap_handle_s &h, size_t count)
{
    auto b = std::make_unique<DevBuf>();
    if (!b->alloc(count * sizeof(T))) return nullptr;
    T *p = b->as<T>();
    // every buffer starts as zeros, so no kernel can read stale bit patterns
    if (cudaMemset(p, 0, b->bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    h.device_bytes += static_cast<int64_t>(b->bytes);
    h.bufs.push_back(std::move(b));
    return p;
}

// Returns a buffer from dalloc to the allocator before the handle goes away
// (a buffer it does not own is ignored).
void release(lap_handle_s &h, const void *p)
{
    for (auto it = h.bufs.begin(); it != h.bufs.end(); ++it)
        if ((*it)->p == p) {
            h.device_bytes -= static_cast<int64_t>((*it)->bytes);
            h.bufs.erase(it);
            return;
        }
}

template <typename T, typename U>
lap_status upload(lap_handle_s &h, T **dst, const std::vector<U> &src)
{
    *dst = dalloc<T>(h, std::max<size_t>(src.size(), 1));
    if (!*dst) return LAP_ERR_OOM;
    if (src.empty()) return LAP_OK;
    if (std::is_same<T, U>::value) {
        LAP_CK(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    } else {
        std::vector<T> tmp(src.begin(), src.end());
        LAP_CK(cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice));
    }
    return LAP_OK;
}

#define LAP_TRY(x)                        \
    do {                                  \
        lap_status s_ = (x);              \
        if (s_ != LAP_OK) return s_;      \
    } while (0)

template <typename V>
lap_status upload_csr(lap_handle_s &h, const HostCsr &c, const HostSell &sl, DevCsr<V> &d,
                      const DevCsr<double> *share)
{
    d.n = static_cast<int>(c.n);
    d.nnz = c.rp[c.n];
    d.nslices = static_cast<int>(sl.nslices);
    d.nlong = static_cast<int>(sl.lrow.size());
    d.ell_entries = static_cast<int64_t>(sl.eci.size());
    d.vec = sl.vec;
    d.long_entries = static_cast<int64_t>(sl.lci.size());
    if (share) {
        d.rp = share->rp;
        d.ci = share->ci;
        d.sptr = share->sptr;
        d.lmask = share->lmask;
        d.rowperm = share->rowperm;
        d.eci = share->eci;
        d.lrow = share->lrow;
        d.lrp = share->lrp;
        d.lci = share->lci;
        d.lchunk_ptr = share->lchunk_ptr;
        d.chunk_row = share->chunk_row;
        d.chunk_beg = share->chunk_beg;
        d.is_long = share->is_long;
        d.lrow_of = share->lrow_of;
        d.kernel = share->kernel;
    } else {
        if (!sl.lrow.empty()) {
            std::vector<unsigned char> isl(static_cast<size_t>(c.n), 0);
            std::vector<int32_t> lof(static_cast<size_t>(c.n), -1);
            for (size_t r = 0; r < sl.lrow.size(); ++r) {
                isl[sl.lrow[r]] = 1;
                lof[sl.lrow[r]] = static_cast<int32_t>(r);
            }
            LAP_TRY(upload(h, &d.is_long, isl));
            LAP_TRY(upload(h, &d.lrow_of, lof));
        }
        LAP_TRY(upload(h, &d.lchunk_ptr, sl.lchunk_ptr));
        LAP_TRY(upload(h, &d.chunk_row, sl.chunk_row));
        LAP_TRY(upload(h, &d.chunk_beg, sl.chunk_beg));
        LAP_TRY(upload(h, &d.rp, c.rp));
        LAP_TRY(upload(h, &d.ci, c.ci));
        LAP_TRY(upload(h, &d.sptr, sl.sptr));
        if (!sl.rowperm.empty()) LAP_TRY(upload(h, &d.rowperm, sl.rowperm));
        LAP_TRY(upload(h, &d.lmask, sl.longmask));
        LAP_TRY(upload(h, &d.eci, sl.eci));
        LAP_TRY(upload(h, &d.lrow, sl.lrow));
        LAP_TRY(upload(h, &d.lrp, sl.lrp));
        LAP_TRY(upload(h, &d.lci, sl.lci));
    }
    LAP_TRY(upload(h, &d.w, c.w));
    LAP_TRY(upload(h, &d.ew, sl.ew));
    LAP_TRY(upload(h, &d.lw, sl.lw));
    d.nchunks = static_cast<int>(sl.chunk_row.size());
    d.chunk_part = dalloc<V>(h, std::max<size_t>(sl.chunk_row.size(), 1));
    if (!d.chunk_part) return LAP_ERR_OOM;
    d.merge_nb = static_cast<int>((c.n + d.nnz + kMergeTile - 1) / kMergeTile);
    const size_t nb = static_cast<size_t>(std::max(d.merge_nb, 1));
    d.mg_hrow = dalloc<int>(h, nb);
    d.mg_trow = dalloc<int>(h, nb);
    d.mg_hval = dalloc<V>(h, nb);
    d.mg_tval = dalloc<V>(h, nb);
    d.mg_hend = dalloc<unsigned char>(h, nb);
    if (!d.mg_hrow || !d.mg_trow || !d.mg_hval || !d.mg_tval || !d.mg_hend) return LAP_ERR_OOM;
    return LAP_OK;
}


template <typename V>
lap_status upload_msp(lap_handle_s &h, const HostModel &m, DevMsp<V> &d, const DevMsp<double> *share)
{
    const int l = m.levels;
    d.levels = l;
    d.off.assign(m.offset.begin(), m.offset.end());
    d.mu = static_cast<V>(m.mu);
    d.lev.resize(static_cast<size_t>(std::max(l - 1, 0)));
    d.gamma.resize(d.lev.size());
    for (int k = 0; k + 1 < l; ++k) {
        const HostMspLevel &S = m.msp[k];
        DevMspLevel<V> &L = d.lev[k];
        L.n = static_cast<int>(S.n);
        L.nagg = static_cast<int>(S.nagg);
        L.off = m.offset[k];
        if (share) L.seg = share->lev[k].seg;
        else LAP_TRY(upload(h, &L.seg, S.seg));
        LAP_TRY(upload(h, &L.inv, S.inv));
        LAP_TRY(upload(h, &L.lcf, S.lcf));
        d.gamma[k] = static_cast<V>(m.c[k + 1] / m.c[k]);
        {
            std::vector<int32_t> big;
            for (int64_t J = 0; J < S.nagg; ++J)
                if (S.seg[J + 1] - S.seg[J] > kBatchBigAgg) big.push_back(static_cast<int32_t>(J));
            L.nbig = static_cast<int>(big.size());
            if (!big.empty()) LAP_TRY(upload(h, &L.big, big));
        }
    }
    d.c.assign(m.c.begin(), m.c.end());
    d.ntop = static_cast<int>(m.lev[l - 1].n);
    if (share) d.G = share->G;
    else LAP_TRY(upload(h, &d.G, m.coarse_pinv));
    // fused tail: the deepest levels whose values (twice), segments and
    // coefficients fit the shared-memory budget, laid out as bulk copies
    // need them (16-byte aligned, sizes rounded up)
    const int budget = 200 * 1024;
    const int sv = static_cast<int>(sizeof(V));
    auto r16 = [](int64_t b) { return (b + 15) / 16 * 16; };
    auto tail_bytes = [&](int t) {
        const int64_t ntl = m.offset[l] - m.offset[t];
        int64_t b = r16(16 + ntl * sv) + r16(ntl * sv);
        for (int k = t; k + 1 < l; ++k) {
            const int64_t na = m.msp[k].nagg, nl = m.msp[k].n - 2 * na;
            b += r16(4 * (na + 1)) + r16(4 * na * sv) + r16(3 * nl * sv);
        }
        return b;
    };
    d.tail0 = -1;
    if (l >= 2) {
        for (int t = l - 1; t >= 1; --t) {
            if (tail_bytes(t) > budget || l - 1 - t > kTailMaxLevels) break;
            d.tail0 = t;
        }
    }
    if (d.tail0 >= 1) {
        const int t0 = d.tail0;
        const int64_t ntl = m.offset[l] - m.offset[t0];
        const int head0 = static_cast<int>((m.offset[t0] * sv) & 15);
        int cur = 0;
        const int sa_s = cur + head0;
        cur += static_cast<int>(r16(head0 + ntl * sv));
        const int sz_s = cur;
        cur += static_cast<int>(r16(ntl * sv));
        std::vector<std::array<int, 6>> lay(static_cast<size_t>(l - 1 - t0));
        for (int k = 0; k < l - 1 - t0; ++k) {
            const int64_t na = m.msp[t0 + k].nagg, nl = m.msp[t0 + k].n - 2 * na;
            const int sb = static_cast<int>(r16(4 * (na + 1))), ib = static_cast<int>(r16(4 * na * sv)),
                      lb = static_cast<int>(r16(3 * nl * sv));
            lay[k] = {cur, sb, cur + sb, ib, cur + sb + ib, lb};
            cur += sb + ib + lb;
        }
        for (TailParams<V> *P : {&d.tail_n, &d.tail_t}) {
            const bool nspace = P == &d.tail_n;
            P->nlev = l - 1 - t0;
            P->ntail = static_cast<int>(ntl);
            P->ntop = d.ntop;
            P->loc_top = static_cast<int>(m.offset[l - 1] - m.offset[t0]);
            P->off0 = m.offset[t0];
            P->n0 = static_cast<int>(m.lev[t0].n);
            P->sa_s = sa_s;
            P->sz_s = sz_s;
            P->a0_head = head0;
            P->smem = cur;
            P->G = d.G;
            P->top_scale = nspace ? m.c[l - 1] : 1.0;
            P->pc = V(1);
            P->write_all = nspace ? 0 : 1;
            for (int k = 0; k < P->nlev; ++k) {
                const DevMspLevel<V> &Lk = d.lev[t0 + k];
                TailLevel<V> &T = P->lev[k];
                T.nagg = Lk.nagg;
                T.loc = static_cast<int>(m.offset[t0 + k] - m.offset[t0]);
                T.seg = Lk.seg;
                T.inv = Lk.inv;
                T.lcf = Lk.lcf;
                T.seg_s = lay[k][0];
                T.seg_b = lay[k][1];
                T.inv_s = lay[k][2];
                T.inv_b = lay[k][3];
                T.lcf_s = lay[k][4];
                T.lcf_b = lay[k][5];
                T.gamma = nspace ? d.gamma[t0 + k] : V(1);
                T.dcoef = nspace ? static_cast<V>(m.c[t0 + k]) : V(1);
            }
        }
        d.tail_smem = static_cast<size_t>(cur);
        LAP_CK(cudaFuncSetAttribute(k_msp_tail<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, budget));
        // the levels below the tail in bands
        const int cap = kBandSmemBytes;
        const std::vector<int> tops = plan_band_tops(m, t0, cap, sv);
        // resident band blocks: the grid, and the unit the tile count is balanced to
        for (const void *f : {(const void *)k_band_up<V, 0>, (const void *)k_band_up<V, 1>,
                              (const void *)k_band_up<V, 2>, (const void *)k_band_up<V, 3>,
                              (const void *)k_band_down<V, true, false>,
                              (const void *)k_band_down<V, false, false>, (const void *)k_band_down<V, true, true>,
                              (const void *)k_band_down<V, false, true>,
                              (const void *)k_band_down<V, false, false, true>})
            LAP_CK(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kBandSmemBytes));
        int occ_up = 0, occ_dn = 0;
        LAP_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_up, k_band_up<V, 1>, kBandThreads, kBandSmemBytes));
        LAP_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_dn, k_band_down<V, true, false>, kBandThreads,
                                                             kBandSmemBytes));
        const int resident = std::max(1, std::min(occ_up, occ_dn)) * h.sms;
        int k0 = 0;
        for (int k1 : tops) {
            const int L = k1 - k0;
            int ntiles = 0;
            std::vector<int> tab;
            std::vector<char> fits;
            plan_band_tiles(m, k0, k1, cap, cap, sv, tab, fits, ntiles);
            if (ntiles > resident && resident < kMaxRedBlocks) {
                // every block loops over the same number of tiles: shrink the
                // tiles until the count reaches the next multiple of the
                // resident blocks, then grow them back just under it
                const int waves = (ntiles + resident - 1) / resident;
                const int want = waves * resident;
                int c = static_cast<int>(static_cast<int64_t>(cap) * ntiles / want);
                for (int it = 0; it < 40; ++it) {
                    int nt2 = 0;
                    std::vector<int> tab2;
                    std::vector<char> fits2;
                    plan_band_tiles(m, k0, k1, c, cap, sv, tab2, fits2, nt2);
                    if (nt2 <= want) {
                        tab.swap(tab2);
                        fits.swap(fits2);
                        ntiles = nt2;
                        break;
                    }
                    c += std::max(16, c / 50);
                    if (c >= cap) break;
                }
            }
            // per tile: segments of all its levels as tile-local member
            // offsets, then pair and leftover coefficients, one 16-byte
            // aligned block; deltas get a 16-byte aligned block of the scratch
            std::vector<unsigned char> coef;
            std::vector<BandRec> rec(static_cast<size_t>(ntiles));
            long long ds = 0;
            auto put = [&](const void *src, size_t bytes) {
                const auto *c = static_cast<const unsigned char *>(src);
                coef.insert(coef.end(), c, c + bytes);
            };
            auto pad16 = [&]() { coef.resize((coef.size() + 15) / 16 * 16, 0); };
            for (int t = 0; t < ntiles; ++t) {
                const int *s0 = &tab[static_cast<size_t>(t) * (L + 1)];
                const int *s1 = &tab[static_cast<size_t>(t + 1) * (L + 1)];
                BandRec &R = rec[t];
                R.cb = R.ds = 0;
                R.cbytes = R.sbytes = -1;
                if (!fits[t]) continue;
                R.cb = static_cast<long long>(coef.size());
                for (int j = 0; j < L; ++j) {
                    const auto &S = m.msp[k0 + j];
                    for (int J = s0[j + 1]; J <= s1[j + 1]; ++J) {
                        const int32_t loc = S.seg[J] - s0[j];
                        put(&loc, 4);
                    }
                }
                pad16();
                R.sbytes = static_cast<int>(coef.size() - R.cb);
                for (int j = 0; j < L; ++j) {
                    const auto &S = m.msp[k0 + j];
                    for (int64_t i = 4ll * s0[j + 1]; i < 4ll * s1[j + 1]; ++i) {
                        const V v = static_cast<V>(S.inv[i]);
                        put(&v, sizeof(V));
                    }
                }
                for (int j = 0; j < L; ++j) {
                    const auto &S = m.msp[k0 + j];
                    const int64_t l0 = 3ll * (s0[j] - 2ll * s0[j + 1]), l1 = 3ll * (s1[j] - 2ll * s1[j + 1]);
                    for (int64_t i = l0; i < l1; ++i) {
                        const V v = static_cast<V>(S.lcf[i]);
                        put(&v, sizeof(V));
                    }
                }
                pad16();
                R.cbytes = static_cast<int>(coef.size() - R.cb);
                R.ds = ds;
                int64_t vals = 0;
                for (int j = 0; j < L; ++j) vals += s1[j] - s0[j];
                ds += (vals * sv + 15) / 16 * 16;
            }
            int *dtab = nullptr;
            unsigned char *dcoef = nullptr;
            BandRec *drec = nullptr;
            LAP_TRY(upload(h, &dtab, tab));
            LAP_TRY(upload(h, &dcoef, coef));
            {
                std::vector<unsigned char> raw(rec.size() * sizeof(BandRec));
                std::memcpy(raw.data(), rec.data(), raw.size());
                unsigned char *p = nullptr;
                LAP_TRY(upload(h, &p, raw));
                drec = reinterpret_cast<BandRec *>(p);
            }
            V *scratch = dalloc<V>(h, static_cast<size_t>(ds / sv + 1));
            if (!scratch) return LAP_ERR_OOM;
            BandParams<V> P{};
            P.nlev = L;
            P.ntiles = ntiles;
            P.smem = kBandSmemBytes;
            // one block per tile, at most what stays resident (the blocks then
            // loop over the tiles)
            P.grid_up = P.grid_down = std::max(1, std::min({ntiles, resident, kMaxRedBlocks}));
            P.tstart = dtab;
            P.rec = drec;
            P.coef = dcoef;
            P.scratch = scratch;
            P.off_top = m.offset[k1];
            P.pc = V(1);
            for (int j = 0; j < P.nlev; ++j) {
                const DevMspLevel<V> &Lk = d.lev[k0 + j];
                P.lev[j] = BandLevel<V>{Lk.seg, Lk.inv, Lk.lcf, m.offset[k0 + j], d.gamma[k0 + j],
                                        static_cast<V>(m.c[k0 + j])};
            }
            d.band_n.push_back(P);
            for (int j = 0; j < P.nlev; ++j) {
                P.lev[j].gamma = V(1);
                P.lev[j].dcoef = V(1);
            }
            d.band_t.push_back(P);
            P.pc = -d.mu;
            d.band_p.push_back(P);
            k0 = k1;
        }
        // partial pairs of the expanded-space CG fused into the sweep: the
        // up pairs of every band, the tail's down pair, the upper bands'
        // down pairs, then the first band's own grid reduction
        if (!d.band_t.empty()) {
            int off = 0;
            for (size_t b = 0; b < d.band_t.size(); ++b) {
                d.band_t[b].first = b == 0;
                d.band_t[b].red_up = off;
                off += 2 * d.band_t[b].grid_up;
            }
            d.xfuse_fin_n = off / 2;
            d.xfuse_slot = off;
            off += 2;
            for (size_t b = 1; b < d.band_t.size(); ++b) {
                d.band_t[b].red_dn = off;
                off += 2 * d.band_t[b].grid_down;
            }
            d.band_t[0].xred_base = d.xfuse_slot;
            d.band_t[0].xred_n = (off - d.xfuse_slot) / 2;
            d.band_t[0].red_gs = off;
            off += 2 * d.band_t[0].grid_down;
            d.xfuse = off <= kMaxRedBlocks * kRedSlots;
        }
    }
    return LAP_OK;
}

template <typename V>
lap_status alloc_vectors(lap_handle_s &h, CgVectors<V> &w, int64_t n, int64_t nt, bool sweeps,
                         bool need_T)
{
    w.x = dalloc<V>(h, n);
    w.r = dalloc<V>(h, n);
    w.p = dalloc<V>(h, n);
    w.q = dalloc<V>(h, n);
    w.z = dalloc<V>(h, n);
    if (!w.x || !w.r || !w.p || !w.q || !w.z) return LAP_ERR_OOM;
    if (sweeps) {
        w.A = dalloc<V>(h, nt);
        w.Y = dalloc<V>(h, nt);
        if (!w.A || !w.Y) return LAP_ERR_OOM;
        if (need_T) {
            w.T = dalloc<V>(h, nt);
            if (!w.T) return LAP_ERR_OOM;
        }
    }
    return LAP_OK;
}

lap_status alloc_state(lap_handle_s &h, CgState &st)
{
    st.sc = dalloc<CgScalars>(h, 1);
    st.part = dalloc<double>(h, static_cast<size_t>(kMaxRedBlocks) * kRedSlots);
    st.ticket = dalloc<unsigned>(h, 1);
    if (!st.sc || !st.part || !st.ticket) return LAP_ERR_OOM;
    LAP_CK(cudaMemset(st.sc, 0, sizeof(CgScalars)));
    LAP_CK(cudaMemset(st.ticket, 0, sizeof(unsigned)));
    return LAP_OK;
}

// Matvec autotuner: time SELL-32 and CSR with 2..16 threads per row on the
// matrix itself (FP64, 5 launches each after a warm-up) and keep the fastest.
template <typename V, int MODE>
void spmv(const lap_handle_s &h, const DevCsr<V> &A, int tpr, const V *x, V *y, const double *bs,
          double *yres, const CgState &st, cudaStream_t s);

// Matvec kernel of one matrix copy, chosen by timing: SELL with one, two or
// three waves of resident blocks (more blocks than fit let the hardware
// balance slices of uneven cost), or CSR with 2..16 threads per row.  The
// reductions of SELL launches hold one partial pair per block, so a grid
// stays within the partials buffer.
template <typename V>
void autotune_spmv(lap_handle_s &h, DevCsr<V> &A, V *x, V *y)
{
    struct Cand { int kernel, grid, hint; };
    std::vector<Cand> cand;
    const int64_t need = (static_cast<int64_t>(A.nslices + A.nlong) * 32 + kBlock - 1) / kBlock;
    for (int waves = 1; waves <= 3; ++waves) {
        const int64_t g = std::min<int64_t>(need, int64_t(h.grid_cap) * waves);
        if (g > kMaxRedBlocks * kRedSlots / 2) break;
        if (waves > 1 && g <= int64_t(h.grid_cap) * (waves - 1)) break;   // no new launch shape
        for (int hint = 0; hint < 2; ++hint) cand.push_back({-1, static_cast<int>(std::max<int64_t>(g, 1)), hint});
    }
    // (the merge-path matvec is not a candidate: slower on every matrix
    // measured, and on tiny ones a timing tie would change the reduction order)
    for (int t : {2, 4, 8, 16}) cand.push_back({t, 0, 0});
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return;
    Cand best = cand[0];
    float best_ms = 1e30f;
    for (const Cand &c : cand) {
        A.sell_grid = c.grid;
        A.stream_hint = c.hint;
        spmv<V, 2>(h, A, c.kernel, x, y, nullptr, nullptr, h.stb, h.s);
        cudaEventRecord(e0, h.s);
        for (int i = 0; i < 5; ++i) spmv<V, 2>(h, A, c.kernel, x, y, nullptr, nullptr, h.stb, h.s);
        cudaEventRecord(e1, h.s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    (void)cudaGetLastError();
    A.kernel = best.kernel == kMergeKernel ? kMergeKernel : best.kernel < 0 ? 0 : best.kernel;
    A.sell_grid = best.grid;
    A.stream_hint = best.hint;
}

// --------------------------------------------------------------------------
// kernel sequences
// --------------------------------------------------------------------------
// The SELL matvec of A in the stored-diagonal form (y = dg x - W x, see
// k_sell), with A's tuned grid, lane groups and load policy; timed by
// lap_kernel_bench against the edge-difference form the solves use.
template <typename V>
void spmv_diag(const lap_handle_s &h, const DevCsr<V> &A, const V *dg, const V *x, V *y, const CgState &st,
               cudaStream_t s)
{
    const bool hint = A.stream_hint != 0;
    if (A.nchunks > 0) {
        const int gc = grid_for(h, static_cast<int64_t>(A.nchunks) * 32);
        if (hint)
            k_long_chunks<V, true, true><<<gc, kBlock, 0, s>>>(A.nchunks, A.chunk_row, A.chunk_beg, A.lrow, A.lci,
                                                               A.lw, x, A.chunk_part, st.sc, 0);
        else
            k_long_chunks<V, false, true><<<gc, kBlock, 0, s>>>(A.nchunks, A.chunk_row, A.chunk_beg, A.lrow, A.lci,
                                                                A.lw, x, A.chunk_part, st.sc, 0);
    }
    const int g = A.sell_grid > 0 ? A.sell_grid : grid_for(h, static_cast<int64_t>(A.nslices + A.nlong) * 32);
#define LAP_SELL_D(VEC, HINT)                                                                              \
    k_sell<V, 2, VEC, HINT, true><<<g, kBlock, 0, s>>>(A.n, A.nslices, A.sptr, A.lmask, A.rowperm, A.eci,  \
                                                       A.ew, A.nlong, A.lrow, A.lchunk_ptr, A.chunk_part, \
                                                       x, y, nullptr, nullptr, st.sc, st.part, st.ticket, dg)
    if (A.vec == 4) {
        if (hint) LAP_SELL_D(4, true);
        else LAP_SELL_D(4, false);
    } else if (A.vec == 2) {
        if (hint) LAP_SELL_D(2, true);
        else LAP_SELL_D(2, false);
    } else {
        if (hint) LAP_SELL_D(1, true);
        else LAP_SELL_D(1, false);
    }
#undef LAP_SELL_D
}

template <typename V, int MODE>
void spmv(const lap_handle_s &h, const DevCsr<V> &A, int tpr, const V *x, V *y, const double *bs,
          double *yres, const CgState &st, cudaStream_t s)
{
    if (tpr == 0) tpr = A.kernel;      // 0: the tuned choice, -1: SELL, -2: merge path, t > 0: CSR
    if (tpr == kMergeKernel) {
        CgScalars *sc = st.sc;
        h.launches += MODE == 2 ? 2 : 3;
        k_merge<V, MODE><<<A.merge_nb, kBlock, 0, s>>>(A.n, A.nnz, A.rp, A.ci, A.w, x, y, bs, yres, A.mg_hrow,
                                                        A.mg_hval, A.mg_hend, A.mg_trow, A.mg_tval, sc);
        k_merge_fix<V, MODE><<<(A.merge_nb + kBlock - 1) / kBlock, kBlock, 0, s>>>(
            A.merge_nb, y, bs, yres, A.mg_hrow, A.mg_hval, A.mg_hend, A.mg_trow, A.mg_tval, sc);
        if (MODE != 2) {
            const int g = static_cast<int>(std::min<int64_t>((A.n + kBlock - 1) / kBlock, 1024));
            k_merge_reduce<V, MODE><<<std::max(g, 1), kBlock, 0, s>>>(A.n, x, y, yres, sc, st.part, st.ticket);
        }
        return;
    }
    if (tpr <= 0) {
        const bool hint = A.stream_hint != 0;
        if (A.nchunks > 0) {
            h.launches += 1;
            const int gc = grid_for(h, static_cast<int64_t>(A.nchunks) * 32);
            if (hint)
                k_long_chunks<V, true><<<gc, kBlock, 0, s>>>(A.nchunks, A.chunk_row, A.chunk_beg, A.lrow, A.lci,
                                                             A.lw, x, A.chunk_part, st.sc, MODE != 2);
            else
                k_long_chunks<V, false><<<gc, kBlock, 0, s>>>(A.nchunks, A.chunk_row, A.chunk_beg, A.lrow, A.lci,
                                                              A.lw, x, A.chunk_part, st.sc, MODE != 2);
        }
        h.launches += 1;
        const int g = A.sell_grid > 0 ? A.sell_grid
                                      : grid_for(h, static_cast<int64_t>(A.nslices + A.nlong) * 32);
#define LAP_SELL(VEC, HINT)                                                                                      \
    k_sell<V, MODE, VEC, HINT><<<g, kBlock, 0, s>>>(A.n, A.nslices, A.sptr, A.lmask, A.rowperm, A.eci, A.ew,      \
                                                    A.nlong, A.lrow, A.lchunk_ptr, A.chunk_part, x, y, bs, yres, \
                                                    st.sc, st.part, st.ticket)
        if (A.vec == 4) {
            if (hint) LAP_SELL(4, true);
            else LAP_SELL(4, false);
        } else if (A.vec == 2) {
            if (hint) LAP_SELL(2, true);
            else LAP_SELL(2, false);
        } else {
            if (hint) LAP_SELL(1, true);
            else LAP_SELL(1, false);
        }
#undef LAP_SELL
        return;
    }
    const int g = grid_for(h, static_cast<int64_t>(A.n) * tpr);
    CgScalars *sc = st.sc;
    double *part = st.part;
    unsigned *tk = st.ticket;
#define LAP_SPMV_CASE(T)                                                                             \
    case T:                                                                                          \
        k_spmv<V, T, MODE><<<g, kBlock, 0, s>>>(A.n, A.rp, A.ci, A.w, x, y, bs, yres, sc, part, tk); \
        break;
    h.launches += 1;
    switch (tpr) {
        LAP_SPMV_CASE(1)
        LAP_SPMV_CASE(2)
        LAP_SPMV_CASE(4)
        LAP_SPMV_CASE(8)
        LAP_SPMV_CASE(16)
    default:
        k_spmv<V, 32, MODE><<<g, kBlock, 0, s>>>(A.n, A.rp, A.ci, A.w, x, y, bs, yres, sc, part, tk);
    }
#undef LAP_SPMV_CASE
}

// z = B r for the n-space CG (MSP sweeps, dense single level, or plain Pi).
// With update, the CG step x += alpha p, r -= alpha q is fused in front.
template <typename V>
void precond_msp(const lap_handle_s &h, const DevMsp<V> &M, const CgVectors<V> &w,
                 const CgState &st, bool update, bool plain, cudaStream_t s)
{
    const int n = static_cast<int>(M.off[1]);
    CgScalars *sc = st.sc;
    h.launches += plain ? 1
                  : M.levels == 1 ? 2
                  : !M.band_n.empty() ? static_cast<int64_t>(2 * M.band_n.size() + 1)
                                      : 2 * ((M.tail0 >= 1 ? M.tail0 : M.levels - 1) - 1) + 3;
    if (plain || M.levels == 1) {
        const int g = grid_for(h, n);
#define LAP_UPD(U, P) \
    k_update<V, U, P><<<g, kBlock, 0, s>>>(n, w.x, w.r, w.p, w.q, nullptr, sc, st.part, st.ticket)
        if (update && plain) LAP_UPD(true, true);
        else if (update) LAP_UPD(true, false);
        else if (plain) LAP_UPD(false, true);
        else LAP_UPD(false, false);
#undef LAP_UPD
        if (plain) return;
        k_dense_z<V><<<grid_for(h, int64_t(n) * 32), kBlock, 0, s>>>(n, M.G, w.r, w.q, w.z, sc, st.part,
                                                                      st.ticket);
        return;
    }
    const int l = M.levels;
    if (!M.band_n.empty()) {
        // levels below the tail in bands (one launch per band and direction),
        // the tail in one block
        const size_t nb = M.band_n.size();
        for (size_t b = 0; b < nb; ++b) {
            const BandParams<V> &P = M.band_n[b];
            const size_t sm = static_cast<size_t>(P.smem);
            if (b > 0)
                k_band_up<V, 0><<<P.grid_up, kBandThreads, sm, s>>>(P, nullptr, nullptr, nullptr, nullptr,
                                                                      w.A, nullptr, sc, nullptr, nullptr);
            else if (update)
                k_band_up<V, 1><<<P.grid_up, kBandThreads, sm, s>>>(P, w.x, w.r, w.p, w.q, w.A, nullptr, sc,
                                                                      st.part, st.ticket);
            else
                k_band_up<V, 2><<<P.grid_up, kBandThreads, sm, s>>>(P, w.x, w.r, w.p, w.q, w.A, nullptr, sc,
                                                                      st.part, st.ticket);
        }
        TailParams<V> T = M.tail_n;
        T.A = w.A;
        T.Y = w.Y;
        T.F = nullptr;
        T.fin = update ? 1 : 2;                  // the first band's reductions
        T.fin_n = M.band_n[0].grid_up;
        T.fin_part = st.part;
        k_msp_tail<V><<<1, 1024, M.tail_smem, s>>>(T, sc);
        for (size_t b = nb; b-- > 0;) {
            const BandParams<V> &P = M.band_n[b];
            const size_t sm = static_cast<size_t>(P.smem);
            if (b == 0)
                k_band_down<V, true, false><<<P.grid_down, kBandThreads, sm, s>>>(P, w.A, w.Y, w.Y, w.z, 0, n, w.r,
                                                                           w.q, sc, st.part, st.ticket);
            else
                k_band_down<V, false, false><<<P.grid_down, kBandThreads, sm, s>>>(
                    P, w.A, w.Y, w.Y, w.Y + P.lev[0].off, 0, n, nullptr, nullptr, sc, nullptr, nullptr);
        }
        return;
    }
    const auto &L0 = M.lev[0];
    if (update)
        k_up_tiled<V, 1><<<grid_for(h, L0.nagg), kTA, 0, s>>>(
            L0.nagg, L0.seg, L0.inv, L0.lcf, w.x, w.r, w.p, w.q, w.A, w.A + M.off[1], M.gamma[0],
            nullptr, sc, st.part, st.ticket);
    else
        k_up_tiled<V, 2><<<grid_for(h, L0.nagg), kTA, 0, s>>>(
            L0.nagg, L0.seg, L0.inv, L0.lcf, w.x, w.r, w.p, w.q, w.A, w.A + M.off[1], M.gamma[0],
            nullptr, sc, st.part, st.ticket);
    // levels below the fused tail one launch each, the tail in one block
    const int t0 = M.tail0 >= 1 ? M.tail0 : l - 1;
    for (int k = 1; k < t0; ++k) {
        const auto &Lk = M.lev[k];
        V *a = w.A + M.off[k];
        k_up_tiled<V, 0><<<grid_for(h, Lk.nagg), kTA, 0, s>>>(
            Lk.nagg, Lk.seg, Lk.inv, Lk.lcf, nullptr, a, nullptr, nullptr, a, w.A + M.off[k + 1],
            M.gamma[k], nullptr, sc, nullptr, nullptr);
    }
    if (M.tail0 >= 1) {
        TailParams<V> P = M.tail_n;
        P.A = w.A;
        P.Y = w.Y;
        P.F = nullptr;
        k_msp_tail<V><<<1, 1024, M.tail_smem, s>>>(P, sc);
    } else {
        const int64_t ot = M.off[l - 1];
        k_coarse<V><<<grid_for(h, int64_t(M.ntop) * 32), kBlock, 0, s>>>(M.ntop, M.G, w.A + ot,
                                                                          w.Y + ot, M.c[l - 1], sc);
    }
    for (int k = t0 - 1; k >= 1; --k) {
        const auto &Lk = M.lev[k];
        k_down_tiled<V, false><<<grid_for(h, Lk.nagg), kTA, 0, s>>>(
            Lk.n, Lk.nagg, Lk.seg, w.A + M.off[k], w.Y + M.off[k + 1], w.Y + M.off[k], V(1),
            static_cast<V>(M.c[k]), nullptr, nullptr, sc, nullptr, nullptr);
    }
    k_down_tiled<V, true><<<grid_for(h, L0.nagg), kTA, 0, s>>>(n, L0.nagg, L0.seg, w.A, w.Y + M.off[1],
                                                              w.z, V(1), V(1), w.r, w.q, sc, st.part,
                                                              st.ticket);
}

template <typename V>
void pupdate(const lap_handle_s &h, int64_t n, const V *z, V *p, const CgState &st, cudaStream_t s)
{
    h.launches += 1;
    k_pupdate<V><<<grid_for(h, n), kBlock, 0, s>>>(n, z, p, st.sc);
}

// Expanded-space MSP solve y~ = L_T^+ f (up to a constant): f in A (tree order,
// overwritten), result in Y.  Section 3.3: elimination without fill-in level by
// level, dense pseudo-inverse on the top level, back-substitution.
template <typename V>
void msp_tilde(const lap_handle_s &h, const DevMsp<V> &M, V *A, V *Y, const CgScalars *sc,
               cudaStream_t s)
{
    const int l = M.levels;
    if (!M.band_t.empty()) {
        // bands below the tail (f added on restriction), the tail, bands down;
        // every level of Y is written
        const size_t nb = M.band_t.size();
        h.launches += static_cast<int64_t>(2 * nb + 1);
        CgScalars *scm = const_cast<CgScalars *>(sc);
        for (size_t b = 0; b < nb; ++b) {
            const BandParams<V> &P = M.band_t[b];
            k_band_up<V, 0><<<P.grid_up, kBandThreads, static_cast<size_t>(P.smem), s>>>(
                P, nullptr, nullptr, nullptr, nullptr, A, A, scm, nullptr, nullptr);
        }
        TailParams<V> T = M.tail_t;
        T.A = A;
        T.Y = Y;
        T.F = A;
        k_msp_tail<V><<<1, 1024, M.tail_smem, s>>>(T, scm);
        for (size_t b = nb; b-- > 0;) {
            const BandParams<V> &P = M.band_t[b];
            k_band_down<V, false, false><<<P.grid_down, kBandThreads, static_cast<size_t>(P.smem), s>>>(
                P, A, Y, Y, Y + P.lev[0].off, 1, 0, nullptr, nullptr, scm, nullptr, nullptr);
        }
        return;
    }
    const int t0 = M.tail0 >= 0 ? std::max(M.tail0, 0) : l - 1;
    const int up_end = M.tail0 >= 1 ? t0 : l - 1;
    h.launches += 2 * up_end + 1;
    for (int k = 0; k < up_end; ++k) {
        const auto &Lk = M.lev[k];
        V *a = A + M.off[k];
        k_up_tiled<V, 0><<<grid_for(h, Lk.nagg), kTA, 0, s>>>(
            Lk.nagg, Lk.seg, Lk.inv, Lk.lcf, nullptr, a, nullptr, nullptr, a, A + M.off[k + 1], V(1),
            A + M.off[k + 1], const_cast<CgScalars *>(sc), nullptr, nullptr);
    }
    if (M.tail0 >= 1) {
        TailParams<V> P = M.tail_t;
        P.A = A;
        P.Y = Y;
        P.F = A;
        k_msp_tail<V><<<1, 1024, M.tail_smem, s>>>(P, const_cast<CgScalars *>(sc));
    } else {
        const int64_t ot = M.off[l - 1];
        k_coarse<V><<<grid_for(h, int64_t(M.ntop) * 32), kBlock, 0, s>>>(M.ntop, M.G, A + ot, Y + ot,
                                                                          1.0, sc);
    }
    for (int k = up_end - 1; k >= 0; --k) {
        const auto &Lk = M.lev[k];
        k_down_tiled<V, false><<<grid_for(h, Lk.nagg), kTA, 0, s>>>(
            Lk.n, Lk.nagg, Lk.seg, A + M.off[k], Y + M.off[k + 1], Y + M.off[k], V(1), V(1), nullptr,
            nullptr, const_cast<CgScalars *>(sc), nullptr, nullptr);
    }
}

// r~ = P(mu)^T r into rt and A (tree order); S is scratch for the level sums.
template <typename V>
void restrict_tilde(const lap_handle_s &h, const DevMsp<V> &M, const V *r, V *rt, V *A, V *S,
                    const CgScalars *sc, cudaStream_t s)
{
    const int64_t n = M.off[1];
    h.launches += M.levels;
    k_copy2<V><<<grid_for(h, n), kBlock, 0, s>>>(n, r, rt, A, sc);
    const V *sin = r;
    double coef = 1.0;
    for (int k = 0; k + 1 < M.levels; ++k) {
        const auto &Lk = M.lev[k];
        coef *= -static_cast<double>(M.mu);
        V *sout = S + M.off[k + 1];
        k_restrict_level<V><<<grid_for(h, Lk.nagg), kBlock, 0, s>>>(
            Lk.nagg, Lk.seg, sin, sout, rt + M.off[k + 1], A ? A + M.off[k + 1] : nullptr,
            static_cast<V>(coef), sc);
        sin = sout;
    }
}

// t = P(mu) y~ by Horner from the top (tree order): T holds t_k on levels >= 2;
// the finest level goes through the finest down pass with the outer CG's
// reductions.
template <typename V>
void prolong_tilde_to_z(const lap_handle_s &h, const DevMsp<V> &M, const V *yt, V *T,
                        const CgVectors<V> &w, const CgState &st, cudaStream_t s)
{
    const int l = M.levels;
    const int64_t ot = M.off[l - 1];
    if (!M.band_p.empty()) {
        // per level from the top down to the tail's first level, then the bands
        const int t0 = M.tail0;
        const size_t nb = M.band_p.size();
        h.launches += 1 + (l - 1 - t0) + static_cast<int64_t>(nb);
        k_copy2<V><<<grid_for(h, M.ntop), kBlock, 0, s>>>(M.ntop, yt + ot, T + ot, nullptr, st.sc);
        for (int k = l - 2; k >= t0; --k) {
            const auto &Lk = M.lev[k];
            k_down_tiled<V, false><<<grid_for(h, Lk.nagg), kTA, 0, s>>>(
                Lk.n, Lk.nagg, Lk.seg, yt + M.off[k], T + M.off[k + 1], T + M.off[k], -M.mu, V(1), nullptr,
                nullptr, st.sc, nullptr, nullptr);
        }
        const int n = static_cast<int>(M.off[1]);
        for (size_t b = nb; b-- > 0;) {
            const BandParams<V> &P = M.band_p[b];
            const size_t sm = static_cast<size_t>(P.smem);
            if (b == 0)
                k_band_down<V, true, true><<<P.grid_down, kBandThreads, sm, s>>>(P, yt, T, T, w.z, 0, n, w.r,
                                                                                 w.q, st.sc, st.part, st.ticket);
            else
                k_band_down<V, false, true><<<P.grid_down, kBandThreads, sm, s>>>(
                    P, yt, T, T, T + P.lev[0].off, 0, n, nullptr, nullptr, st.sc, nullptr, nullptr);
        }
        return;
    }
    h.launches += l;
    k_copy2<V><<<grid_for(h, M.ntop), kBlock, 0, s>>>(M.ntop, yt + ot, T + ot, nullptr, st.sc);
    for (int k = l - 2; k >= 1; --k) {
        const auto &Lk = M.lev[k];
        k_down_tiled<V, false><<<grid_for(h, Lk.nagg), kTA, 0, s>>>(
            Lk.n, Lk.nagg, Lk.seg, yt + M.off[k], T + M.off[k + 1], T + M.off[k], -M.mu, V(1), nullptr,
            nullptr, st.sc, nullptr, nullptr);
    }
    const auto &L0 = M.lev[0];
    k_down_tiled<V, true><<<grid_for(h, L0.nagg), kTA, 0, s>>>(
        static_cast<int>(M.off[1]), L0.nagg, L0.seg, yt, T + M.off[1], w.z, -M.mu, V(1), w.r, w.q,
        st.sc, st.part, st.ticket);
}

// One expanded-space CG iteration of the PEGP inner solve L_H y~ = r~ with the
// MSP preconditioner (vectors e: x = y~, r = r~, p, q, z unused, A/Y sweeps).
// With the bands and the tail in place the step x += alpha p, r -= alpha q
// and the reductions of z = M r run inside the sweep (q = L_H p, bands up
// with the step, tail with the convergence test, bands down with sum z and
// r.z, p = Pi z + beta p); otherwise step, sweep and reductions are
// separate launches.
template <typename V>
void inner_iteration(const lap_handle_s &h, const DevCsr<V> &H, const DevMsp<V> &M,
                     const CgVectors<V> &e, const CgState &st, cudaStream_t s)
{
    const int64_t nt = M.off[M.levels];
    if (M.xfuse) {
        // the matvec without reductions, p.q by a streaming pass (cheaper
        // than the matvec's own epilogue for L_H)
        spmv<V, 2>(h, H, h.tprH, e.p, e.q, nullptr, nullptr, st, s);
        h.launches += 1;
        k_pq<V><<<grid_for(h, nt / 4 + 1), kBlock, 0, s>>>(nt, e.p, e.q, st.sc, st.part, st.ticket);
        const size_t nb = M.band_t.size();
        h.launches += static_cast<int64_t>(2 * nb + 1);
        for (size_t b = 0; b < nb; ++b) {
            const BandParams<V> &P = M.band_t[b];
            k_band_up<V, 3><<<P.grid_up, kBandThreads, static_cast<size_t>(P.smem), s>>>(
                P, e.x, e.r, e.p, e.q, e.A, nullptr, st.sc, st.part, st.ticket);
        }
        TailParams<V> T = M.tail_t;
        T.A = e.A;
        T.Y = e.Y;
        T.F = e.r;
        T.fin = 3;
        T.fin_n = M.xfuse_fin_n;
        T.fin_part = st.part;
        T.cx = e.x;
        T.cr = e.r;
        T.cp = e.p;
        T.cq = e.q;
        T.xred_slot = M.xfuse_slot;
        T.xred_part = st.part;
        k_msp_tail<V><<<1, 1024, M.tail_smem, s>>>(T, st.sc);
        for (size_t b = nb; b-- > 0;) {
            const BandParams<V> &P = M.band_t[b];
            k_band_down<V, false, false, true><<<P.grid_down, kBandThreads, static_cast<size_t>(P.smem), s>>>(
                P, e.A, e.Y, e.Y, e.Y + P.lev[0].off, 1, static_cast<int>(nt), e.r, nullptr, st.sc, st.part,
                st.ticket);
        }
        pupdate<V>(h, nt, e.Y, e.p, st, s);
        return;
    }
    spmv<V, 0>(h, H, h.tprH, e.p, e.q, nullptr, nullptr, st, s);
    h.launches += 2;
    k_update<V, true, false><<<grid_for(h, nt), kBlock, 0, s>>>(static_cast<int>(nt), e.x, e.r, e.p,
                                                                e.q, e.A, st.sc, st.part, st.ticket);
    msp_tilde<V>(h, M, e.A, e.Y, st.sc, s);
    k_zred<V><<<grid_for(h, nt), kBlock, 0, s>>>(nt, e.Y, e.r, st.sc, st.part, st.ticket);
    pupdate<V>(h, nt, e.Y, e.p, st, s);
}

// Start of the inner solve: y~ = 0, z~ = MSP(r~), p~ = Pi z~ (A holds r~).
template <typename V>
void inner_start(const lap_handle_s &h, const DevMsp<V> &M, const CgVectors<V> &e, const CgState &st,
                 double tol, int maxit, cudaStream_t s)
{
    const int64_t nt = M.off[M.levels];
    k_cg_reset<<<1, 1, 0, s>>>(st.sc, tol, maxit, 0, nullptr, 0);
    h.launches += 1;
    k_vec_init<V><<<grid_for(h, nt), kBlock, 0, s>>>(nt, e.r, e.x, st.sc, st.part, st.ticket);
    h.launches += 2;
    msp_tilde<V>(h, M, e.A, e.Y, st.sc, s);
    k_zred<V><<<grid_for(h, nt), kBlock, 0, s>>>(nt, e.Y, e.r, st.sc, st.part, st.ticket);
    pupdate<V>(h, nt, e.Y, e.p, st, s);
}

template <typename V> struct Sel;
template <> struct Sel<double> {
    static const DevCsr<double> &L(const lap_handle_s &h) { return h.L64; }
    static const DevCsr<double> &H(const lap_handle_s &h) { return h.H64; }
    static const DevMsp<double> &M(const lap_handle_s &h) { return h.M64; }
    static const CgVectors<double> &w(const lap_handle_s &h) { return h.w64; }
    static const CgVectors<double> &e(const lap_handle_s &h) { return h.e64; }
    static const double *G(const lap_handle_s &h) { return h.G64; }
    static const CgState &st(const lap_handle_s &h) { return h.st64; }
    static const CgState &ste(const lap_handle_s &h) { return h.ste64; }
    static cudaGraphExec_t &gi(lap_handle_s &h) { return h.g_iter64; }
    static cudaGraphExec_t &gin(lap_handle_s &h) { return h.g_in64; }
    static int64_t &ni(lap_handle_s &h) { return h.nodes_iter64; }
    static int64_t &nin(lap_handle_s &h) { return h.nodes_in64; }
};
template <> struct Sel<float> {
    static const DevCsr<float> &L(const lap_handle_s &h) { return h.L32; }
    static const DevCsr<float> &H(const lap_handle_s &h) { return h.H32; }
    static const DevMsp<float> &M(const lap_handle_s &h) { return h.M32; }
    static const CgVectors<float> &w(const lap_handle_s &h) { return h.w32; }
    static const CgVectors<float> &e(const lap_handle_s &h) { return h.e32; }
    static const float *G(const lap_handle_s &h) { return h.G32; }
    static const CgState &st(const lap_handle_s &h) { return h.st32; }
    static const CgState &ste(const lap_handle_s &h) { return h.ste32; }
    static cudaGraphExec_t &gi(lap_handle_s &h) { return h.g_iter32; }
    static cudaGraphExec_t &gin(lap_handle_s &h) { return h.g_in32; }
    static int64_t &ni(lap_handle_s &h) { return h.nodes_iter32; }
    static int64_t &nin(lap_handle_s &h) { return h.nodes_in32; }
};

bool is_plain(const lap_handle_s &h) { return h.m.opt.prec == LAP_PREC_NONE; }
bool is_pegp(const lap_handle_s &h) { return h.m.opt.prec == LAP_PREC_PEGP_INNER; }
// exact PEGP with at least two levels (one level: H = T = G, the MSP path)
bool is_exact(const lap_handle_s &h) { return h.m.opt.prec == LAP_PREC_PEGP_EXACT && h.G64; }

// Exact PEGP (Section 3.2, M = L_H^+): z = Pi P(mu) G P(mu)^T r with the dense
// G applied between the restriction and the prolongation; UPDATE first takes
// the CG step x += alpha p, r -= alpha q.  Every kernel checks the device
// flag, so the sequence can be captured in a graph.
template <typename V>
void precond_exact(const lap_handle_s &h, bool update, cudaStream_t s)
{
    const auto &w = Sel<V>::w(h);
    const auto &st = Sel<V>::st(h);
    const auto &M = Sel<V>::M(h);
    const auto &e = Sel<V>::e(h);
    const int64_t n = M.off[1], nt = M.off[M.levels];
    if (update) {
        h.launches += 1;
        k_update<V, true, false><<<grid_for(h, n), kBlock, 0, s>>>(static_cast<int>(n), w.x, w.r, w.p,
                                                                   w.q, nullptr, st.sc, st.part,
                                                                   st.ticket);
    }
    restrict_tilde<V>(h, M, w.r, e.r, nullptr, e.T, st.sc, s);
    h.launches += 1;
    k_dense_gemv<V><<<grid_for(h, nt * 32), kBlock, 0, s>>>(static_cast<int>(nt), h.g_ld, Sel<V>::G(h),
                                                          e.r, e.x, st.sc);
    prolong_tilde_to_z<V>(h, M, e.x, e.T, w, st, s);
}

// one outer CG iteration for the graph-captured preconditioners (MSP, none)
template <typename V>
void outer_iteration(const lap_handle_s &h, cudaStream_t s)
{
    const auto &w = Sel<V>::w(h);
    const auto &st = Sel<V>::st(h);
    spmv<V, 0>(h, Sel<V>::L(h), h.tpr, w.p, w.q, nullptr, nullptr, st, s);
    if (is_exact(h)) precond_exact<V>(h, true, s);
    else precond_msp<V>(h, Sel<V>::M(h), w, st, true, is_plain(h), s);
    pupdate<V>(h, Sel<V>::M(h).off[1], is_plain(h) ? w.r : w.z, w.p, st, s);
}

// PEGP inner solves with at most this many iterations are sequenced on the
// device: the outer iteration needs no host poll and is captured in a graph.
constexpr int kDevInnerMax = 32;

bool device_sequenced_pegp(const lap_handle_s &h)
{
    return is_pegp(h) && h.m.opt.inner_maxit <= kDevInnerMax && h.M64.levels > 1;
}

// One outer PEGP_inner iteration sequenced entirely on the device: the outer
// step and its convergence test, r~ = P(mu)^T r, the inner CG on L_H run to
// its cap (iterations after its own convergence return at once, and the
// whole inner solve is stopped before it starts when the outer CG is not
// running), its iteration count tallied, z = Pi P(mu) y~ with the outer
// reductions, and the new direction.  Every kernel after the outer step
// checks a flag, so check_every iterations are captured as one graph.
template <typename V>
void outer_pegp_iteration(const lap_handle_s &h, cudaStream_t s)
{
    const auto &w = Sel<V>::w(h);
    const auto &st = Sel<V>::st(h);
    const auto &M = Sel<V>::M(h);
    const auto &e = Sel<V>::e(h);
    const auto &ste = Sel<V>::ste(h);
    const int64_t n = M.off[1], nt = M.off[M.levels];
    spmv<V, 0>(h, Sel<V>::L(h), h.tpr, w.p, w.q, nullptr, nullptr, st, s);
    h.launches += 3;
    k_update<V, true, false><<<grid_for(h, n), kBlock, 0, s>>>(static_cast<int>(n), w.x, w.r, w.p, w.q, nullptr,
                                                               st.sc, st.part, st.ticket);
    restrict_tilde<V>(h, M, w.r, e.r, e.A, e.T, st.sc, s);
    k_inner_reset<<<1, 1, 0, s>>>(ste.sc, st.sc, h.m.opt.inner_tol, h.m.opt.inner_maxit);
    k_vec_init<V><<<grid_for(h, nt), kBlock, 0, s>>>(nt, e.r, e.x, ste.sc, ste.part, ste.ticket);
    msp_tilde<V>(h, M, e.A, e.Y, ste.sc, s);
    h.launches += 1;
    k_zred<V><<<grid_for(h, nt), kBlock, 0, s>>>(nt, e.Y, e.r, ste.sc, ste.part, ste.ticket);
    pupdate<V>(h, nt, e.Y, e.p, ste, s);
    for (int i = 0; i < h.m.opt.inner_maxit; ++i) inner_iteration<V>(h, Sel<V>::H(h), M, e, ste, s);
    h.launches += 1;
    k_inner_tally<<<1, 1, 0, s>>>(ste.sc, st.sc);
    prolong_tilde_to_z<V>(h, M, e.x, e.T, w, st, s);
    pupdate<V>(h, n, w.z, w.p, st, s);
}

template <typename Fn>
lap_status capture(lap_handle_s &h, cudaGraphExec_t &g, int64_t &nodes, Fn body)
{
    cudaGraph_t graph = nullptr;
    const int64_t l0 = h.launches;
    LAP_CK(cudaStreamBeginCapture(h.s, cudaStreamCaptureModeThreadLocal));
    body();
    cudaError_t e = cudaStreamEndCapture(h.s, &graph);
    h.launches = l0;
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return LAP_ERR_CUDA;
    }
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    nodes = static_cast<int64_t>(nn);
    e = cudaGraphInstantiate(&g, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        g = nullptr;
        return LAP_ERR_CUDA;
    }
    return LAP_OK;
}

lap_status poll(lap_handle_s &h, const CgState &st, CgScalars &out)
{
    LAP_CK(cudaMemcpyAsync(h.hsc, st.sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, h.s));
    LAP_CK(cudaStreamSynchronize(h.s));
    out = *h.hsc;
    return LAP_OK;
}

bool timed_out(const lap_handle_s &h, Clock::time_point t0)
{
    return h.m.opt.timeout_s > 0.0 &&
           std::chrono::duration<double>(Clock::now() - t0).count() > h.m.opt.timeout_s;
}

// Preconditioner application B r for the outer CG (fresh start or after an
// update).  For PEGP_INNER this runs the inner CG with host polling.
template <typename V>
lap_status apply_precond(lap_handle_s &h, bool update, Clock::time_point t0, int &inner_total)
{
    const cudaStream_t s = h.s;
    const auto &w = Sel<V>::w(h);
    const auto &st = Sel<V>::st(h);
    const auto &M = Sel<V>::M(h);
    const int64_t n = M.off[1];
    if (is_exact(h)) {
        precond_exact<V>(h, update, s);
        return LAP_OK;
    }
    if (!is_pegp(h) || M.levels == 1) {
        // one level: H = T = G, so the dense top-level solve is PEGP exactly
        precond_msp<V>(h, M, w, st, update, is_plain(h), s);
        return LAP_OK;
    }
    if (update) {
        h.launches += 1;
        k_update<V, true, false><<<grid_for(h, n), kBlock, 0, s>>>(static_cast<int>(n), w.x, w.r, w.p,
                                                                   w.q, nullptr, st.sc, st.part,
                                                                   st.ticket);
    }
    CgScalars sc;
    LAP_TRY(poll(h, st, sc));
    if (sc.flag != kRun) return LAP_OK;          // converged / stopped: nothing to apply
    const auto &e = Sel<V>::e(h);
    const auto &ste = Sel<V>::ste(h);
    restrict_tilde<V>(h, M, w.r, e.r, e.A, e.T, nullptr, s);
    inner_start<V>(h, M, e, ste, h.m.opt.inner_tol, h.m.opt.inner_maxit, s);
    cudaGraphExec_t &g = Sel<V>::gin(h);
    const int K = std::max(1, std::min(h.m.opt.check_every, 16));
    if (!g) {
        LAP_TRY(capture(h, g, Sel<V>::nin(h), [&] {
            for (int i = 0; i < K; ++i) inner_iteration<V>(h, Sel<V>::H(h), M, e, ste, s);
        }));
    }
    // the device stops at inner_maxit; the launch cap only guards the host loop
    const int cap_in = h.m.opt.inner_maxit / K + 4;
    for (int launches = 0;; ++launches) {
        LAP_CK(cudaGraphLaunch(g, s));
        h.launches += Sel<V>::nin(h);
        CgScalars si;
        LAP_TRY(poll(h, ste, si));
        if (si.flag != kRun) {
            inner_total += si.iter;
            break;
        }
        if (launches >= cap_in) return LAP_ERR_BREAKDOWN;
        if (timed_out(h, t0)) return LAP_ERR_TIMEOUT;
    }
    prolong_tilde_to_z<V>(h, M, e.x, e.T, w, st, s);
    return LAP_OK;
}

// CG iterations on the current system until the device flag stops them.
template <typename V>
lap_status iterate(lap_handle_s &h, Clock::time_point t0, int &inner_total, CgScalars &sc)
{
    const cudaStream_t s = h.s;
    const auto &w = Sel<V>::w(h);
    const auto &st = Sel<V>::st(h);
    const int64_t n = Sel<V>::M(h).off[1];
    const bool dev_pegp = device_sequenced_pegp(h);
    if (is_pegp(h) && !dev_pegp) {
        for (int guard = 0; guard <= h.m.opt.maxit + 4; ++guard) {
            spmv<V, 0>(h, Sel<V>::L(h), h.tpr, w.p, w.q, nullptr, nullptr, st, s);
            LAP_TRY(apply_precond<V>(h, true, t0, inner_total));
            pupdate<V>(h, n, w.z, w.p, st, s);
            LAP_TRY(poll(h, st, sc));
            if (sc.flag != kRun) return LAP_OK;
            if (timed_out(h, t0)) return LAP_ERR_TIMEOUT;
        }
        return LAP_ERR_BREAKDOWN;
    }
    cudaGraphExec_t &g = Sel<V>::gi(h);
    if (!g) LAP_TRY(capture(h, g, Sel<V>::ni(h), [&] {
            for (int i = 0; i < h.m.opt.check_every; ++i) {
                if (dev_pegp) outer_pegp_iteration<V>(h, s);
                else outer_iteration<V>(h, s);
            }
        }));
    int tally0 = 0;
    if (dev_pegp) {
        CgScalars s0;
        LAP_TRY(poll(h, st, s0));
        tally0 = s0.inner_total;
    }
    struct Tally {
        bool on;
        int base;
        int &total;
        const CgScalars &sc;
        ~Tally()
        {
            if (on) total += sc.inner_total - base;
        }
    } tally{dev_pegp, tally0, inner_total, sc};
    // the device stops at maxit; the launch cap only guards the host loop
    const int cap = h.m.opt.maxit / h.m.opt.check_every + 4;
    // stall detection (mixed precision inner solves only): stop once the
    // recurrence residual has set no new minimum for `window` iterations
    const bool watch = std::is_same<V, float>::value && h.m.opt.stall_window > 0;
    const int window = std::max(h.m.opt.stall_window, h.m.opt.check_every);
    double best = 1e300;
    int best_iter = 0;
    for (int launches = 0;; ++launches) {
        LAP_CK(cudaGraphLaunch(g, s));
        h.launches += Sel<V>::ni(h);
        LAP_TRY(poll(h, st, sc));
        if (sc.flag != kRun) return LAP_OK;
        if (launches >= cap) return LAP_ERR_BREAKDOWN;
        if (timed_out(h, t0)) return LAP_ERR_TIMEOUT;
        if (watch) {
            if (sc.relres < best) {
                best = sc.relres;
                best_iter = sc.iter;
            } else if (sc.iter - best_iter >= window) {
                sc.flag = kConverged;                // stalled: hand back to refinement
                return LAP_OK;
            }
        }
    }
}

// FP64 preconditioned CG on the centred right-hand side h.bs (tree order).
lap_status cg_fp64(lap_handle_s &h, Clock::time_point t0, lap_solve_info &info)
{
    const cudaStream_t s = h.s;
    const auto &w = h.w64;
    const auto &st = h.st64;
    const int64_t n = h.M64.off[1];
    const lap_options &o = h.m.opt;
    k_cg_reset<<<1, 1, 0, s>>>(st.sc, o.tol, o.maxit, is_pegp(h) ? 1 : 0, h.hist, o.maxit, h.lz);
    h.launches += 2;
    k_center_init<double><<<grid_for(h, n), kBlock, 0, s>>>(static_cast<int>(n), h.bs, w.r, w.x, st.sc,
                                                            st.part, st.ticket);
    CgScalars sc;
    LAP_TRY(poll(h, st, sc));
    if (!(sc.bnorm > 0.0)) {
        info.relres = 0.0;
        return LAP_OK;
    }
    int inner = 0;
    LAP_TRY(apply_precond<double>(h, false, t0, inner));
    pupdate<double>(h, n, is_plain(h) ? w.r : w.z, w.p, st, s);
    lap_status result = LAP_ERR_NO_CONVERGENCE;
    for (;;) {
        lap_status it = iterate<double>(h, t0, inner, sc);
        if (h.lz_run < 0) h.lz_run = sc.iter;     // the first run ends here
        if (it != LAP_OK) {
            result = it;
            break;
        }
        info.relres_recurrence = sc.relres;
        if (sc.flag == kConverged) {
            // confirm with the true residual r = Pi b - L x
            spmv<double, 1>(h, h.L64, h.tpr, w.x, nullptr, h.bs, w.r, st, s);
            LAP_TRY(poll(h, st, sc));
            if (sc.relres <= o.tol) {
                result = LAP_OK;
                break;
            }
            if (sc.iter >= o.maxit || info.restarts >= 8) break;
            info.restarts += 1;
            h.launches += 1;
            k_cg_restart<<<1, 1, 0, s>>>(st.sc);
            LAP_TRY(apply_precond<double>(h, false, t0, inner));
            pupdate<double>(h, n, is_plain(h) ? w.r : w.z, w.p, st, s);
            continue;
        }
        result = sc.flag == kBreakdown ? LAP_ERR_BREAKDOWN : LAP_ERR_NO_CONVERGENCE;
        break;
    }
    if (result != LAP_OK) {
        spmv<double, 1>(h, h.L64, h.tpr, w.x, nullptr, h.bs, w.r, st, s);
        CgScalars tmp;
        LAP_TRY(poll(h, st, tmp));
        sc.relres = tmp.relres;
    }
    info.iterations = sc.iter;
    info.inner_iterations = inner;
    info.relres = sc.relres;
    return result;
}

// Mixed precision: FP64 residual refresh + FP32 inner CG per refinement step.
lap_status cg_mixed(lap_handle_s &h, Clock::time_point t0, lap_solve_info &info)
{
    const cudaStream_t s = h.s;
    const int64_t n = h.M64.off[1];
    const int ni = static_cast<int>(n);
    const lap_options &o = h.m.opt;
    const CgState &so = h.st64;
    const CgState &si = h.st32;
    k_cg_reset<<<1, 1, 0, s>>>(so.sc, o.tol, o.maxit, 0, nullptr, 0);
    h.launches += 2;
    k_center_init<double><<<grid_for(h, n), kBlock, 0, s>>>(ni, h.bs, h.w64.r, h.w64.x, so.sc, so.part,
                                                            so.ticket);
    CgScalars sc;
    LAP_TRY(poll(h, so, sc));
    if (!(sc.bnorm > 0.0)) {
        info.relres = 0.0;
        return LAP_OK;
    }
    double relres = 1.0;
    int total = 0, inner = 0;
    lap_status result = LAP_ERR_NO_CONVERGENCE;
    for (int ref = 0;; ++ref) {
        if (ref > 0) {
            spmv<double, 1>(h, h.L64, h.tpr, h.w64.x, nullptr, h.bs, h.w64.r, so, s);
            LAP_TRY(poll(h, so, sc));
            relres = sc.relres;
            info.refinements = ref;
            if (relres <= o.tol) {
                result = LAP_OK;
                break;
            }
            if (!std::isfinite(relres)) {
                result = LAP_ERR_BREAKDOWN;
                break;
            }
        }
        if (ref >= o.max_refine || total >= o.maxit) break;
        if (timed_out(h, t0)) {
            result = LAP_ERR_TIMEOUT;
            break;
        }
        const double tol_in = std::min(0.5, std::max(o.refine_tol, 0.3 * o.tol / relres));
        k_cg_reset<<<1, 1, 0, s>>>(si.sc, tol_in, o.maxit - total, is_pegp(h) ? 1 : 0, h.hist + total,
                                   o.maxit - total, h.lz + 2 * total);
        h.launches += 5;
        k_gather_sum<float><<<grid_for(h, n), kBlock, 0, s>>>(ni, nullptr, h.w64.r, h.w32.r, si.sc,
                                                             si.part, si.ticket);
        k_center_init<float><<<grid_for(h, n), kBlock, 0, s>>>(ni, h.w64.r, h.w32.r, h.w32.x, si.sc,
                                                              si.part, si.ticket);
        LAP_TRY(apply_precond<float>(h, false, t0, inner));
        pupdate<float>(h, n, is_plain(h) ? h.w32.r : h.w32.z, h.w32.p, si, s);
        CgScalars sci;
        lap_status it = iterate<float>(h, t0, inner, sci);
        if (h.lz_run < 0) h.lz_run = sci.iter;    // the first inner solve
        if (it != LAP_OK) {
            result = it;
            break;
        }
        total += sci.iter;
        h.launches += 1;
        k_add_correction<float><<<grid_for(h, n), kBlock, 0, s>>>(ni, h.w64.x, h.w32.x);
        info.relres_recurrence = sci.relres;
        if (sci.flag == kBreakdown && sci.iter == 0) {
            result = LAP_ERR_BREAKDOWN;
            break;
        }
    }
    if (result != LAP_OK && result != LAP_ERR_BREAKDOWN) {
        spmv<double, 1>(h, h.L64, h.tpr, h.w64.x, nullptr, h.bs, h.w64.r, so, s);
        LAP_TRY(poll(h, so, sc));
        relres = sc.relres;
    }
    info.iterations = total;
    info.inner_iterations = inner;
    info.relres = relres;
    return result;
}

// ---------------------------------------------------------------------------
// Flexible GMRES(m) in FP64 (fgmres.cuh): the cycle's kernels check the device
// flag, so for the preconditioners without host polling (MSP, exact PEGP,
// none) a whole cycle is captured once as a CUDA graph and replayed; the
// PEGP inner solve polls the host and runs the cycle's launches directly.
template <typename T>
T *member(GmState *gm, size_t off)
{
    return reinterpret_cast<T *>(reinterpret_cast<char *>(gm) + off);
}

lap_status gm_alloc(lap_handle_s &h, int m)
{
    if (h.gm_V && h.gm_m == m) return LAP_OK;
    if (h.g_gm) {
        cudaGraphExecDestroy(h.g_gm);
        h.g_gm = nullptr;
    }
    for (const void *p : {static_cast<const void *>(h.gm_V), static_cast<const void *>(h.gm_Z),
                          static_cast<const void *>(h.gm_part), static_cast<const void *>(h.gm)})
        release(h, p);
    const size_t n = static_cast<size_t>(h.M64.off[1]);
    h.gm_V = dalloc<double>(h, n * (m + 1));
    h.gm_Z = dalloc<double>(h, n * m);
    h.gm_part = dalloc<double>(h, static_cast<size_t>(m + 1) * kGmDotBlocks);
    h.gm = dalloc<GmState>(h, 1);
    if (!h.gm_V || !h.gm_Z || !h.gm_part || !h.gm) return LAP_ERR_OOM;
    h.gm_m = m;
    return LAP_OK;
}

// step j of the cycle: z_j = B v_j, w = L z_j, two Gram-Schmidt passes,
// v_(j+1), the Givens update
lap_status gm_step(lap_handle_s &h, int j, Clock::time_point t0, int &inner)
{
    const cudaStream_t s = h.s;
    const auto &w = h.w64;
    const auto &st = h.st64;
    const int n = static_cast<int>(h.M64.off[1]);
    double *Vj = h.gm_V + static_cast<int64_t>(j) * n;
    double *Zj = h.gm_Z + static_cast<int64_t>(j) * n;
    double *Vn = Vj + n;
    const int gn = grid_for(h, n);
    if (is_plain(h)) {
        h.launches += 1;
        k_gm_store_z<<<gn, kBlock, 0, s>>>(n, Vj, nullptr, Zj, st.sc);
    } else {
        h.launches += 2;
        k_copy2<double><<<gn, kBlock, 0, s>>>(n, Vj, w.r, nullptr, st.sc);
        LAP_TRY(apply_precond<double>(h, false, t0, inner));
        k_gm_store_z<<<gn, kBlock, 0, s>>>(n, w.z, &st.sc->zmean, Zj, st.sc);
    }
    // MODE 0 stops with the flag (its CG scalars are not used here)
    spmv<double, 0>(h, h.L64, h.tpr, Zj, w.q, nullptr, nullptr, st, s);
    const int nc = j + 1;
    const int nbx = std::max(1, std::min(kGmDotBlocks, (n + kBlock - 1) / kBlock));
    double *h1 = member<double>(h.gm, offsetof(GmState, h1));
    double *h2 = member<double>(h.gm, offsetof(GmState, h2));
    for (double *hc : {h1, h2}) {
        k_gm_dots<<<dim3(nbx, nc), kBlock, 0, s>>>(n, h.gm_V, w.q, h.gm_part, st.sc);
        k_gm_dots_sum<<<nc, kBlock, 0, s>>>(nbx, h.gm_part, hc, st.sc);
        k_gm_orth<<<gn, kBlock, 0, s>>>(n, nc, h.gm_V, hc, w.q, h.gm, st.sc, st.part, st.ticket);
    }
    k_gm_scale<<<gn, kBlock, 0, s>>>(n, w.q, Vn, h.gm, st.sc);
    k_gm_givens<<<1, 1, 0, s>>>(j, h.gm, st.sc);
    h.launches += 8;
    return LAP_OK;
}

// one cycle from the residual in w.r: start, m steps, y and x += Z y, then
// the true residual r = Pi b - L x (into w.r, ||r|| into the scalars)
lap_status gm_cycle(lap_handle_s &h, Clock::time_point t0, int &inner)
{
    const cudaStream_t s = h.s;
    const auto &w = h.w64;
    const auto &st = h.st64;
    const int n = static_cast<int>(h.M64.off[1]);
    const int gn = grid_for(h, n);
    h.launches += 3;
    k_gm_start<<<gn, kBlock, 0, s>>>(n, w.r, h.gm_V, st.sc, h.gm);
    for (int j = 0; j < h.gm_m; ++j) LAP_TRY(gm_step(h, j, t0, inner));
    k_gm_solve<<<1, 1, 0, s>>>(h.gm, st.sc);
    k_gm_xupdate<<<gn, kBlock, 0, s>>>(n, h.gm_Z, h.gm, w.x);
    spmv<double, 1>(h, h.L64, h.tpr, w.x, nullptr, h.bs, w.r, st, s);
    return LAP_OK;
}

lap_status fgmres_fp64(lap_handle_s &h, Clock::time_point t0, lap_solve_info &info)
{
    const cudaStream_t s = h.s;
    const auto &w = h.w64;
    const auto &st = h.st64;
    const int64_t n = h.M64.off[1];
    const lap_options &o = h.m.opt;
    LAP_TRY(gm_alloc(h, o.restart));
    k_cg_reset<<<1, 1, 0, s>>>(st.sc, o.tol, o.maxit, 0, h.hist, o.maxit, nullptr);
    h.launches += 2;
    k_center_init<double><<<grid_for(h, n), kBlock, 0, s>>>(static_cast<int>(n), h.bs, w.r, w.x, st.sc,
                                                            st.part, st.ticket);
    CgScalars sc;
    LAP_TRY(poll(h, st, sc));
    if (!(sc.bnorm > 0.0)) {
        info.relres = 0.0;
        return LAP_OK;
    }
    const bool graph = !is_pegp(h);
    int inner = 0, cycles = 0;
    lap_status result = LAP_ERR_NO_CONVERGENCE;
    for (;;) {
        if (graph) {
            if (!h.g_gm) LAP_TRY(capture(h, h.g_gm, h.nodes_gm, [&] { (void)gm_cycle(h, t0, inner); }));
            LAP_CK(cudaGraphLaunch(h.g_gm, s));
            h.launches += h.nodes_gm;
        } else {
            LAP_TRY(gm_cycle(h, t0, inner));
        }
        LAP_TRY(poll(h, st, sc));
        ++cycles;
        if (sc.relres <= o.tol) {
            result = LAP_OK;
            break;
        }
        if (sc.stop == kBreakdown) {
            result = LAP_ERR_BREAKDOWN;
            break;
        }
        if (sc.iter >= o.maxit) break;
        if (timed_out(h, t0)) {
            result = LAP_ERR_TIMEOUT;
            break;
        }
    }
    info.iterations = sc.iter;
    info.restarts = cycles - 1;
    info.inner_iterations = inner;
    info.relres = sc.relres;
    info.relres_recurrence = sc.relres;
    return result;
}

// caller stream -> private stream ordering
lap_status enter(lap_handle_s &h, cudaStream_t user)
{
    LAP_CK(cudaSetDevice(h.device));
    LAP_CK(cudaEventRecord(h.ev_in, user));
    LAP_CK(cudaStreamWaitEvent(h.s, h.ev_in, 0));
    return LAP_OK;
}

lap_status leave(lap_handle_s &h, cudaStream_t user)
{
    LAP_CK(cudaEventRecord(h.ev_out, h.s));
    LAP_CK(cudaStreamWaitEvent(user, h.ev_out, 0));
    LAP_CK(cudaGetLastError());
    return LAP_OK;
}

lap_status solve_core(lap_handle_s &h, const double *b, double *x, lap_solve_info &info)
{
    const auto t0 = Clock::now();
    const cudaStream_t s = h.s;
    const int n = static_cast<int>(h.M64.off[1]);
    k_gather_sum<double><<<grid_for(h, n), kBlock, 0, s>>>(n, h.perm1, b, h.bs, h.st64.sc, h.st64.part,
                                                          h.st64.ticket);
    h.launches += 3;   // gather, mean, scatter
    h.lz_run = -1;
    lap_status st;
    if (h.m.opt.krylov == LAP_KRYLOV_FGMRES)
        st = h.m.opt.precision == LAP_MIXED ? LAP_ERR_UNSUPPORTED : fgmres_fp64(h, t0, info);
    else
        st = h.m.opt.precision == LAP_MIXED ? cg_mixed(h, t0, info) : cg_fp64(h, t0, info);
    h.hist_count = std::min(info.iterations, h.m.opt.maxit);
    h.lz_run = std::min(std::max(h.lz_run, 0), h.hist_count);
    // x = Pi x back in the caller's numbering (also for a non-converged result)
    k_mean<double><<<grid_for(h, n), kBlock, 0, s>>>(n, h.w64.x, h.stb.sc, h.stb.part, h.stb.ticket);
    k_scatter_shift<double><<<grid_for(h, n), kBlock, 0, s>>>(n, h.perm1, h.w64.x, x,
                                                             &h.stb.sc->tmp);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return LAP_ERR_CUDA;
    return st;
}

// Exact PEGP: G = S (S L_H S + v v^T / v^T v)^-1 S (see dense.cuh), inverted
// on the device by blocked Gauss-Jordan, with an FP32 copy for mixed
// precision.  Expanded sizes above kDenseMaxN are not inverted densely.
lap_status upload_dense_pegp(lap_handle_s &h, bool mixed)
{
    const HostCsr &H = h.m.LH;
    if (H.n > kDenseMaxN) return LAP_ERR_UNSUPPORTED;
    const int nt = static_cast<int>(H.n);
    const int np = (nt + kGjB - 1) / kGjB * kGjB;
    std::vector<double> sv(static_cast<size_t>(nt)), vv(static_cast<size_t>(nt));
    double vtv = 0.0;
    for (int i = 0; i < nt; ++i) {
        const double d = H.diag[i];
        if (!(d > 0.0) || !std::isfinite(d)) return LAP_ERR_BREAKDOWN;
        vv[i] = std::sqrt(d);
        sv[i] = 1.0 / vv[i];
        vtv += d;
    }
    const size_t nn = static_cast<size_t>(np) * np;
    h.G64 = dalloc<double>(h, nn);
    if (!h.G64) return LAP_ERR_OOM;
    if (mixed) {
        h.G32 = dalloc<float>(h, nn);
        if (!h.G32) return LAP_ERR_OOM;
    }
    h.g_ld = np;
    // set-up scratch, released on return
    DevBuf brp, bci, bw, bs, bv, bB, bC, bR, bbad;
    if (!brp.alloc(sizeof(int64_t) * (nt + 1)) || !bci.alloc(sizeof(int) * std::max<size_t>(H.ci.size(), 1)) ||
        !bw.alloc(sizeof(double) * std::max<size_t>(H.w.size(), 1)) || !bs.alloc(sizeof(double) * nt) ||
        !bv.alloc(sizeof(double) * nt) || !bB.alloc(sizeof(double) * kGjB * kGjB) ||
        !bC.alloc(sizeof(double) * static_cast<size_t>(np) * kGjB) ||
        !bR.alloc(sizeof(double) * static_cast<size_t>(np) * kGjB) || !bbad.alloc(sizeof(int)))
        return LAP_ERR_OOM;
    const cudaStream_t s = h.s;
    LAP_CK(cudaMemcpyAsync(brp.p, H.rp.data(), sizeof(int64_t) * (nt + 1), cudaMemcpyHostToDevice, s));
    if (!H.ci.empty()) {
        LAP_CK(cudaMemcpyAsync(bci.p, H.ci.data(), sizeof(int) * H.ci.size(), cudaMemcpyHostToDevice, s));
        LAP_CK(cudaMemcpyAsync(bw.p, H.w.data(), sizeof(double) * H.w.size(), cudaMemcpyHostToDevice, s));
    }
    LAP_CK(cudaMemcpyAsync(bs.p, sv.data(), sizeof(double) * nt, cudaMemcpyHostToDevice, s));
    LAP_CK(cudaMemcpyAsync(bv.p, vv.data(), sizeof(double) * nt, cudaMemcpyHostToDevice, s));
    LAP_CK(cudaMemsetAsync(bbad.p, 0, sizeof(int), s));
    const int gfill = static_cast<int>(std::min<int64_t>((static_cast<int64_t>(nn) + kBlock - 1) / kBlock,
                                                         int64_t(h.sms) * 16));
    k_dense_fill<<<gfill, kBlock, 0, s>>>(np, nt, bv.as<double>(), 1.0 / vtv, h.G64);
    k_dense_scatter<<<grid_for(h, nt), kBlock, 0, s>>>(nt, np, brp.as<int64_t>(), bci.as<int>(),
                                                       bw.as<double>(), bs.as<double>(), h.G64);
    const int tiles = np / kGjB;
    for (int t = 0; t < tiles; ++t) {
        const int k0 = t * kGjB;
        k_gj_pivot<<<1, kGjThreads, 0, s>>>(np, k0, h.G64, bB.as<double>(), bbad.as<int>());
        k_gj_panels<<<tiles, kGjThreads, 0, s>>>(np, k0, h.G64, bB.as<double>(), bC.as<double>(),
                                                  bR.as<double>());
        k_gj_update<<<dim3(tiles, tiles), kGjThreads, 0, s>>>(np, k0, h.G64, bB.as<double>(),
                                                             bC.as<double>(), bR.as<double>());
    }
    k_dense_finish<<<gfill, kBlock, 0, s>>>(np, nt, bs.as<double>(), h.G64, h.G32);
    int bad = 0;
    LAP_CK(cudaMemcpyAsync(&bad, bbad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    LAP_CK(cudaStreamSynchronize(s));
    return bad ? LAP_ERR_BREAKDOWN : LAP_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
lap_status upload_model(lap_handle_s &h, cudaStream_t user)
{
    (void)user;
    const HostModel &m = h.m;
    LAP_CK(cudaGetDevice(&h.device));
    LAP_CK(cudaDeviceGetAttribute(&h.sms, cudaDevAttrMultiProcessorCount, h.device));
    h.grid_cap = std::min(h.sms * 8, kMaxRedBlocks);
    LAP_CK(cudaStreamCreateWithFlags(&h.s, cudaStreamNonBlocking));
    LAP_CK(cudaEventCreateWithFlags(&h.ev_in, cudaEventDisableTiming));
    LAP_CK(cudaEventCreateWithFlags(&h.ev_out, cudaEventDisableTiming));
    LAP_CK(cudaMallocHost(&h.hsc, sizeof(CgScalars)));

    const bool mixed = m.opt.precision == LAP_MIXED;
    const int64_t n = m.lev[0].n, nt = m.offset[m.levels];
    {
        HostSell sl;
        make_sell(m.L1, sl, 0);
        LAP_TRY(upload_csr<double>(h, m.L1, sl, h.L64, nullptr));
        if (mixed) LAP_TRY(upload_csr<float>(h, m.L1, sl, h.L32, &h.L64));
    }
    LAP_TRY(upload_msp<double>(h, m, h.M64, nullptr));
    if (mixed) LAP_TRY(upload_msp<float>(h, m, h.M32, &h.M64));
    if (m.has_LH) {
        HostSell sl;
        make_sell(m.LH, sl, 0);
        LAP_TRY(upload_csr<double>(h, m.LH, sl, h.H64, nullptr));
        if (mixed) LAP_TRY(upload_csr<float>(h, m.LH, sl, h.H32, &h.H64));
        if (m.opt.prec == LAP_PREC_PEGP_EXACT && m.levels > 1) LAP_TRY(upload_dense_pegp(h, mixed));
    }
    LAP_TRY(upload(h, &h.perm1, m.lev[0].perm));
    {
        std::vector<int64_t> xm(static_cast<size_t>(nt));
        for (int k = 0; k < m.levels; ++k)
            for (int64_t i = 0; i < m.lev[k].n; ++i) xm[m.offset[k] + i] = m.offset[k] + m.lev[k].perm[i];
        LAP_TRY(upload(h, &h.xmap, xm));
    }
    h.bs = dalloc<double>(h, n);
    if (!h.bs) return LAP_ERR_OOM;
    LAP_TRY(alloc_vectors<double>(h, h.w64, n, nt, true, true));
    if (mixed) LAP_TRY(alloc_vectors<float>(h, h.w32, n, nt, true, true));
    if (m.has_LH) {
        LAP_TRY(alloc_vectors<double>(h, h.e64, nt, nt, true, true));
        if (mixed) LAP_TRY(alloc_vectors<float>(h, h.e32, nt, nt, true, true));
    }
    LAP_TRY(alloc_state(h, h.st64));
    LAP_TRY(alloc_state(h, h.st32));
    LAP_TRY(alloc_state(h, h.ste64));
    LAP_TRY(alloc_state(h, h.ste32));
    LAP_TRY(alloc_state(h, h.stb));
    h.hist_capacity = std::max(m.opt.maxit, 1000);
    h.hist = dalloc<double>(h, static_cast<size_t>(h.hist_capacity));
    h.lz = dalloc<double>(h, 2 * static_cast<size_t>(h.hist_capacity));
    if (!h.hist || !h.lz) return LAP_ERR_OOM;
    // matvec kernel choice: the option forces one, 0 times the candidates
    h.tpr = 0;
    h.tprH = 0;
    if (m.opt.spmv_tpr != 0) {
        h.L64.kernel = h.L32.kernel = h.H64.kernel = h.H32.kernel =
            m.opt.spmv_tpr == kMergeKernel ? kMergeKernel : std::max(m.opt.spmv_tpr, 0);
    } else {
        // each copy on its own: the FP64 and FP32 matvecs prefer different shapes
        autotune_spmv<double>(h, h.L64, h.w64.p, h.w64.q);
        if (mixed) autotune_spmv<float>(h, h.L32, h.w32.p, h.w32.q);
        if (m.has_LH) {
            autotune_spmv<double>(h, h.H64, h.e64.p, h.e64.q);
            if (mixed) autotune_spmv<float>(h, h.H32, h.e32.p, h.e32.q);
        }
    }
    LAP_CK(cudaDeviceSynchronize());
    return LAP_OK;
}

void destroy_handle(lap_handle_s &h)
{
    if (h.s) cudaStreamSynchronize(h.s);
    h.batch.reset();
    for (cudaGraphExec_t *g : {&h.g_iter64, &h.g_iter32, &h.g_in64, &h.g_in32, &h.g_gm})
        if (*g) {
            cudaGraphExecDestroy(*g);
            *g = nullptr;
        }
    h.bufs.clear();
    if (h.hsc) cudaFreeHost(h.hsc);
    if (h.ev_in) cudaEventDestroy(h.ev_in);
    if (h.ev_out) cudaEventDestroy(h.ev_out);
    if (h.s) cudaStreamDestroy(h.s);
    h.hsc = nullptr;
    h.s = nullptr;
}

lap_status solve_device(lap_handle_s &h, const double *b, double *x, cudaStream_t user,
                        lap_solve_info &info)
{
    LAP_TRY(enter(h, user));
    const lap_status st = solve_core(h, b, x, info);
    const lap_status st2 = leave(h, user);
    LAP_CK(cudaStreamSynchronize(h.s));
    return st != LAP_OK ? st : st2;
}

lap_status solve_host(lap_handle_s &h, const double *b, double *x, cudaStream_t user,
                      lap_solve_info &info)
{
    const int64_t n = h.M64.off[1];
    if (!h.bin) {
        h.bin = dalloc<double>(h, n);
        h.xout = dalloc<double>(h, n);
        if (!h.bin || !h.xout) return LAP_ERR_OOM;
    }
    LAP_TRY(enter(h, user));
    LAP_CK(cudaMemcpyAsync(h.bin, b, n * sizeof(double), cudaMemcpyHostToDevice, h.s));
    const lap_status st = solve_core(h, h.bin, h.xout, info);
    LAP_CK(cudaMemcpyAsync(x, h.xout, n * sizeof(double), cudaMemcpyDeviceToHost, h.s));
    const lap_status st2 = leave(h, user);
    LAP_CK(cudaStreamSynchronize(h.s));
    return st != LAP_OK ? st : st2;
}

// ---------------------------------------------------------------------------
// building blocks (FP64, device-resident)
// ---------------------------------------------------------------------------
lap_status block_laplacian(lap_handle_s &h, const double *x, double *y, cudaStream_t user)
{
    LAP_TRY(enter(h, user));
    const int n = h.L64.n;
    k_gather<double><<<grid_for(h, n), kBlock, 0, h.s>>>(n, h.perm1, x, h.w64.p);
    spmv<double, 2>(h, h.L64, h.tpr, h.w64.p, h.w64.q, nullptr, nullptr, h.stb, h.s);
    k_scatter_shift<double><<<grid_for(h, n), kBlock, 0, h.s>>>(n, h.perm1, h.w64.q, y, nullptr);
    return leave(h, user);
}

lap_status block_precond(lap_handle_s &h, const double *r, double *z, cudaStream_t user)
{
    LAP_TRY(enter(h, user));
    const int n = h.L64.n;
    const CgState &st = h.st64;
    k_gather_sum<double><<<grid_for(h, n), kBlock, 0, h.s>>>(n, h.perm1, r, h.bs, st.sc, st.part,
                                                            st.ticket);
    k_center_init<double><<<grid_for(h, n), kBlock, 0, h.s>>>(n, h.bs, h.w64.r, h.w64.x, st.sc, st.part,
                                                             st.ticket);
    k_cg_reset<<<1, 1, 0, h.s>>>(st.sc, 0.0, 1, is_pegp(h) ? 1 : 0, nullptr, 0);
    int inner = 0;
    LAP_TRY(apply_precond<double>(h, false, Clock::now(), inner));
    k_scatter_shift<double><<<grid_for(h, n), kBlock, 0, h.s>>>(n, h.perm1, is_plain(h) ? h.w64.r : h.w64.z,
                                                               z, &st.sc->zmean);
    return leave(h, user);
}

lap_status block_restrict(lap_handle_s &h, const double *r, double *rt, cudaStream_t user)
{
    LAP_TRY(enter(h, user));
    const int n = h.L64.n;
    const int64_t nt = h.M64.off[h.M64.levels];
    k_gather<double><<<grid_for(h, n), kBlock, 0, h.s>>>(n, h.perm1, r, h.w64.r);
    restrict_tilde<double>(h, h.M64, h.w64.r, h.w64.Y, nullptr, h.w64.T, nullptr, h.s);
    k_permute<double><<<grid_for(h, nt), kBlock, 0, h.s>>>(nt, h.xmap, h.w64.Y, rt, 1);
    return leave(h, user);
}

lap_status block_prolong(lap_handle_s &h, const double *yt, double *z, cudaStream_t user)
{
    LAP_TRY(enter(h, user));
    const int n = h.L64.n;
    const int64_t nt = h.M64.off[h.M64.levels];
    const auto &M = h.M64;
    k_permute<double><<<grid_for(h, nt), kBlock, 0, h.s>>>(nt, h.xmap, yt, h.w64.Y, 0);
    // Horner from the top: t_l = y_l, t_k = y_k - mu t_{k+1}(parent)
    const int l = M.levels;
    const int64_t ot = M.off[l - 1];
    k_copy2<double><<<grid_for(h, M.ntop), kBlock, 0, h.s>>>(M.ntop, h.w64.Y + ot, h.w64.T + ot, nullptr,
                                                            nullptr);
    for (int k = l - 2; k >= 0; --k) {
        const auto &Lk = M.lev[k];
        k_down_tiled<double, false><<<grid_for(h, Lk.nagg), kTA, 0, h.s>>>(
            Lk.n, Lk.nagg, Lk.seg, h.w64.Y + M.off[k], h.w64.T + M.off[k + 1], h.w64.T + M.off[k],
            -M.mu, 1.0, nullptr, nullptr, nullptr, nullptr, nullptr);
    }
    k_scatter_shift<double><<<grid_for(h, n), kBlock, 0, h.s>>>(n, h.perm1, h.w64.T, z, nullptr);
    return leave(h, user);
}

lap_status block_msp_solve(lap_handle_s &h, const double *rt, double *yt, cudaStream_t user)
{
    LAP_TRY(enter(h, user));
    const int64_t nt = h.M64.off[h.M64.levels];
    k_permute<double><<<grid_for(h, nt), kBlock, 0, h.s>>>(nt, h.xmap, rt, h.w64.A, 0);
    msp_tilde<double>(h, h.M64, h.w64.A, h.w64.Y, nullptr, h.s);
    k_permute<double><<<grid_for(h, nt), kBlock, 0, h.s>>>(nt, h.xmap, h.w64.Y, yt, 1);
    return leave(h, user);
}

lap_status block_pegp(lap_handle_s &h, const double *xt, double *yt, cudaStream_t user)
{
    LAP_TRY(enter(h, user));
    const int64_t nt = h.H64.n;
    k_permute<double><<<grid_for(h, nt), kBlock, 0, h.s>>>(nt, h.xmap, xt, h.e64.p, 0);
    spmv<double, 2>(h, h.H64, h.tprH, h.e64.p, h.e64.q, nullptr, nullptr, h.stb, h.s);
    k_permute<double><<<grid_for(h, nt), kBlock, 0, h.s>>>(nt, h.xmap, h.e64.q, yt, 1);
    return leave(h, user);
}

// ---------------------------------------------------------------------------
lap_status get_history(lap_handle_s &h, double *out, int cap, int *count)
{
    const int c = std::min(h.hist_count, h.hist_capacity);
    *count = c;
    if (cap <= 0 || c == 0) return LAP_OK;
    LAP_CK(cudaMemcpy(out, h.hist, sizeof(double) * std::min(c, cap), cudaMemcpyDeviceToHost));
    return LAP_OK;
}

// Hutchinson samples of tr(L_T^+ L_H) (stretch.cuh): per sample, z, y = L_H z,
// u = L_T^+ y by the expanded-space MSP solve, z^T (u - mean u); FP64.
lap_status estimate_stretch(lap_handle_s &h, int samples, uint64_t seed, double *vals)
{
    if (!h.H64.w || h.M64.levels < 2) return LAP_ERR_UNSUPPORTED;
    const cudaStream_t s = h.s;
    const int64_t nt = h.M64.off[h.M64.levels];
    const auto &e = h.e64;
    double *dv = dalloc<double>(h, static_cast<size_t>(samples));
    if (!dv) return LAP_ERR_OOM;
    const int g = grid_for(h, nt);
    for (int k = 0; k < samples; ++k) {
        k_rademacher<<<g, kBlock, 0, s>>>(nt, seed, static_cast<uint32_t>(k), h.xmap, e.p);
        spmv<double, 2>(h, h.H64, h.tprH, e.p, e.q, nullptr, nullptr, h.stb, s);
        k_copy2<double><<<g, kBlock, 0, s>>>(nt, e.q, e.A, nullptr, nullptr);
        msp_tilde<double>(h, h.M64, e.A, e.Y, nullptr, s);
        k_stretch_dot<<<g, kBlock, 0, s>>>(nt, e.p, e.Y, dv + k, h.stb.part, h.stb.ticket);
        h.launches += 4;
    }
    LAP_CK(cudaMemcpyAsync(vals, dv, sizeof(double) * samples, cudaMemcpyDeviceToHost, s));
    LAP_CK(cudaStreamSynchronize(s));
    release(h, dv);
    return LAP_OK;
}

lap_status get_lanczos(lap_handle_s &h, double *alpha, double *beta, int cap, int *count)
{
    const int c = std::min(h.lz_run, h.hist_capacity);
    *count = c;
    if (cap <= 0 || c == 0) return LAP_OK;
    const int m = std::min(c, cap);
    std::vector<double> ab(2 * static_cast<size_t>(m));
    LAP_CK(cudaMemcpy(ab.data(), h.lz, sizeof(double) * ab.size(), cudaMemcpyDeviceToHost));
    for (int j = 0; j < m; ++j) {
        if (alpha) alpha[j] = ab[2 * j];
        if (beta) beta[j] = j + 1 < c ? ab[2 * j + 1] : 0.0;   // the last step has no successor
    }
    return LAP_OK;
}

lap_status update_options(lap_handle_s &h, const lap_options &o)
{
    if (!(o.tol > 0.0) || o.maxit < 1 || o.check_every < 1 || o.inner_maxit < 1 ||
        o.max_refine < 0 || !(o.refine_tol > 0.0) || !(o.inner_tol > 0.0))
        return LAP_ERR_INVALID_ARG;
    if (o.precision != LAP_FP64 && o.precision != LAP_MIXED) return LAP_ERR_INVALID_ARG;
    if (o.precision == LAP_MIXED && !h.L32.w) return LAP_ERR_INVALID_ARG;
    if (o.krylov != LAP_KRYLOV_CG && o.krylov != LAP_KRYLOV_FGMRES) return LAP_ERR_INVALID_ARG;
    if (o.restart < 1 || o.restart > kGmMax) return LAP_ERR_INVALID_ARG;
    if (h.host_only) return LAP_ERR_INVALID_ARG;
    lap_options &cur = h.m.opt;
    if (o.maxit > h.hist_capacity) {
        double *p = dalloc<double>(h, static_cast<size_t>(o.maxit));
        double *q = dalloc<double>(h, 2 * static_cast<size_t>(o.maxit));
        if (!p || !q) return LAP_ERR_OOM;
        release(h, h.hist);
        release(h, h.lz);
        h.hist = p;
        h.lz = q;
        h.hist_capacity = o.maxit;
        h.hist_count = h.lz_run = 0;
    }
    // the graphs hold the iteration counts (and the device-sequenced PEGP
    // outer iterations the inner solve's tolerance and cap)
    if (o.check_every != cur.check_every || o.inner_tol != cur.inner_tol || o.inner_maxit != cur.inner_maxit) {
        for (cudaGraphExec_t *g : {&h.g_iter64, &h.g_iter32, &h.g_in64, &h.g_in32})
            if (*g) {
                cudaGraphExecDestroy(*g);
                *g = nullptr;
            }
    }
    cur.tol = o.tol;
    cur.maxit = o.maxit;
    cur.inner_tol = o.inner_tol;
    cur.inner_maxit = o.inner_maxit;
    cur.refine_tol = o.refine_tol;
    cur.max_refine = o.max_refine;
    cur.check_every = o.check_every;
    cur.timeout_s = o.timeout_s;
    cur.precision = o.precision;
    cur.stall_window = o.stall_window;
    cur.krylov = o.krylov;
    cur.restart = o.restart;
    return LAP_OK;
}

namespace {
template <typename V>
double sweep_bytes(const DevMsp<V> &M)
{
    // MSP sweep z = B r, every array moved once: r read and z written (n
    // values each), each level's segments and elimination coefficients read
    // once, every level's deltas stored on the way up and read on the way
    // down, and the top level's dense pseudo-inverse read.  Intermediate
    // restrictions and prolongations need no memory traffic of their own.
    const double s = sizeof(V);
    const int l = M.levels;
    double b = 2.0 * s * static_cast<double>(M.off[1]);
    for (int k = 0; k + 1 < l; ++k) {
        const double n = M.lev[k].n, na = M.lev[k].nagg, nl = n - 2 * na;
        b += 4.0 * (na + 1) + s * (4 * na + 3 * nl) + 2.0 * s * n;
    }
    b += 8.0 * M.ntop * M.ntop;
    return b;
}

// Algorithmic bytes of the first upward band with the CG step fused: x, p, q,
// r read and x, r written, the band's coefficients read, its deltas and the
// next level's right-hand side written.
template <typename V>
double band_up_bytes(const DevMsp<V> &M)
{
    const double s = sizeof(V);
    const BandParams<V> &P = M.band_n[0];
    const int k1 = P.nlev;
    double b = 6.0 * s * static_cast<double>(M.off[1]);
    for (int k = 0; k < k1; ++k) {
        const double n = M.lev[k].n, na = M.lev[k].nagg, nl = n - 2 * na;
        b += 4.0 * (na + 1) + s * (4 * na + 3 * nl) + (k > 0 ? s * n : 0.0);
    }
    b += s * static_cast<double>(M.off[k1 + 1] - M.off[k1]);
    return b;
}
}  // namespace

// Algorithmic bytes of the expanded-space MSP solve y~ = L_T^+ f: f read,
// every level's segments and elimination coefficients read once, the deltas
// of every level below the top stored on the way up and read on the way down,
// y~ written, the top pseudo-inverse read.
template <typename V>
double sweep_tilde_bytes(const DevMsp<V> &M)
{
    const double s = sizeof(V);
    const int l = M.levels;
    const double nt = static_cast<double>(M.off[l]);
    double b = 2.0 * s * nt + 2.0 * s * (nt - M.ntop) + 8.0 * M.ntop * M.ntop;
    for (int k = 0; k + 1 < l; ++k) {
        const double na = M.lev[k].nagg, nl = M.lev[k].n - 2 * na;
        b += 4.0 * (na + 1) + s * (4 * na + 3 * nl);
    }
    return b;
}

// One inner CG iteration: the L_H matvec (entries, row pointers, p read once,
// q written), the step (x, p, q, r read; x, r written), the sweep without its
// right-hand side read (the updated r is used where it is produced), r read
// again for r.z, and p = Pi z + beta p (z, p read, p written).
template <typename V>
double inner_iteration_bytes(const DevCsr<V> &H, const DevMsp<V> &M)
{
    const double s = sizeof(V);
    const double nt = static_cast<double>(M.off[M.levels]);
    const double mv = H.nnz * (4.0 + s) + 4.0 * (H.n + 1) + 2.0 * s * H.n;
    return mv + 6.0 * s * nt + (sweep_tilde_bytes(M) - s * nt) + s * nt + 3.0 * s * nt;
}

lap_status kernel_bench(lap_handle_s &h, int kernel, int precision, int reps, double *ms, double *bytes)
{
    if (precision == 1 && !h.L32.w) return LAP_ERR_INVALID_ARG;
    if ((kernel == 1 || kernel == 7 || kernel == 8 || kernel == 9) && !h.H64.w) return LAP_ERR_INVALID_ARG;
    if ((kernel == 7 || kernel == 8) && (h.M64.levels < 2 || !is_pegp(h))) return LAP_ERR_INVALID_ARG;
    if (kernel == 6 && !h.G64) return LAP_ERR_INVALID_ARG;
    if (kernel == 9 && static_cast<int64_t>(h.m.LH.diag.size()) != h.H64.n) return LAP_ERR_INVALID_ARG;
    if (kernel < 0 || kernel > 9) return LAP_ERR_INVALID_ARG;
    const cudaStream_t s = h.s;
    // kernel 9: L_H's diagonal on the device in the timed precision
    DevBuf dgbuf;
    if (kernel == 9) {
        const int64_t nt = h.H64.n;
        if (!dgbuf.alloc(static_cast<size_t>(nt) * (precision == 1 ? 4 : 8))) return LAP_ERR_OOM;
        if (precision == 1) {
            std::vector<float> d32(h.m.LH.diag.begin(), h.m.LH.diag.end());
            LAP_CK(cudaMemcpyAsync(dgbuf.p, d32.data(), 4 * nt, cudaMemcpyHostToDevice, s));
            LAP_CK(cudaStreamSynchronize(s));
        } else {
            LAP_CK(cudaMemcpyAsync(dgbuf.p, h.m.LH.diag.data(), 8 * nt, cudaMemcpyHostToDevice, s));
            LAP_CK(cudaStreamSynchronize(s));
        }
    }
    cudaEvent_t e0, e1;
    LAP_CK(cudaEventCreate(&e0));
    LAP_CK(cudaEventCreate(&e1));
    k_bench_scalars<<<1, 1, 0, s>>>(h.stb.sc);
    auto run = [&](auto tag) {
        using V = decltype(tag);
        const auto &w = Sel<V>::w(h);
        const auto &M = Sel<V>::M(h);
        const int64_t n = M.off[1];
        double by = 0.0;
        auto launch = [&]() {
            switch (kernel) {
            case 0: spmv<V, 2>(h, Sel<V>::L(h), h.tpr, w.p, w.q, nullptr, nullptr, h.stb, s); break;
            case 1: spmv<V, 2>(h, Sel<V>::H(h), h.tprH, Sel<V>::e(h).p, Sel<V>::e(h).q, nullptr,
                               nullptr, h.stb, s); break;
            case 2: precond_msp<V>(h, M, w, h.stb, false, false, s); break;
            case 3: {
                const BandParams<V> &P = M.band_n[0];
                k_band_up<V, 1><<<P.grid_up, kBandThreads, static_cast<size_t>(P.smem), s>>>(
                    P, w.x, w.r, w.p, w.q, w.A, nullptr, h.stb.sc, h.stb.part, h.stb.ticket);
                break;
            }
            case 4: {
                TailParams<V> T = M.tail_n;
                T.A = w.A;
                T.Y = w.Y;
                T.F = nullptr;
                k_msp_tail<V><<<1, 1024, M.tail_smem, s>>>(T, h.stb.sc);
                break;
            }
            case 6: {
                const int64_t nt = M.off[M.levels];
                k_dense_gemv<V><<<grid_for(h, nt * 32), kBlock, 0, s>>>(
                    static_cast<int>(nt), h.g_ld, Sel<V>::G(h), Sel<V>::e(h).r, Sel<V>::e(h).x, h.stb.sc);
                break;
            }
            case 7: inner_iteration<V>(h, Sel<V>::H(h), M, Sel<V>::e(h), h.stb, s); break;
            case 8: msp_tilde<V>(h, M, Sel<V>::e(h).A, Sel<V>::e(h).Y, h.stb.sc, s); break;
            case 9: spmv_diag<V>(h, Sel<V>::H(h), dgbuf.as<V>(), Sel<V>::e(h).p, Sel<V>::e(h).q, h.stb, s); break;
            default: {
                const BandParams<V> &P = M.band_n[0];
                k_band_down<V, true, false><<<P.grid_down, kBandThreads, static_cast<size_t>(P.smem), s>>>(
                    P, w.A, w.Y, w.Y, w.z, 0, static_cast<int>(n), w.r, w.q, h.stb.sc, h.stb.part,
                    h.stb.ticket);
            }
            }
        };
        const double sv = sizeof(V);
        if (kernel == 0 || kernel == 1) {
            const auto &A = kernel == 0 ? Sel<V>::L(h) : Sel<V>::H(h);
            by = A.nnz * (4.0 + sv) + 4.0 * (A.n + 1) + 2.0 * sv * A.n;
        } else if (kernel == 9) {
            const auto &A = Sel<V>::H(h);
            by = A.nnz * (4.0 + sv) + 4.0 * (A.n + 1) + 3.0 * sv * A.n;   // the diagonal read too
        } else if (kernel == 2) {
            by = sweep_bytes(M);
        } else if (kernel == 3) {
            if (M.band_n.empty()) return -1.0;
            by = band_up_bytes(M);
        } else if (kernel == 4) {
            if (M.tail0 < 1) return -1.0;
            // the tail's levels: values read and written, coefficients and the
            // top pseudo-inverse read once
            const int l = M.levels;
            by = 2.0 * sv * static_cast<double>(M.off[l] - M.off[M.tail0]) + 8.0 * M.ntop * M.ntop;
            for (int k = M.tail0; k + 1 < l; ++k) {
                const double nk = M.lev[k].n, na = M.lev[k].nagg;
                by += 4.0 * (na + 1) + sv * (4 * na + 3 * (nk - 2 * na));
            }
        } else if (kernel == 6) {
            // exact PEGP matvec: G (ntilde^2) and r~ read, y~ written
            const double nt = static_cast<double>(M.off[M.levels]);
            by = sv * nt * nt + 2.0 * sv * nt;
        } else if (kernel == 7) {
            by = inner_iteration_bytes(Sel<V>::H(h), M);
            // a direction, a residual and an iterate to start from
            const auto &e = Sel<V>::e(h);
            const int64_t nt = M.off[M.levels];
            k_bench_fill<V><<<grid_for(h, nt), kBlock, 0, s>>>(nt, e.p, 0x1234567u);
            k_bench_fill<V><<<grid_for(h, nt), kBlock, 0, s>>>(nt, e.r, 0x7654321u);
            k_bench_fill<V><<<grid_for(h, nt), kBlock, 0, s>>>(nt, e.x, 0x0badf00du);
        } else if (kernel == 8) {
            by = sweep_tilde_bytes(M);
            const auto &e = Sel<V>::e(h);
            const int64_t nt = M.off[M.levels];
            k_bench_fill<V><<<grid_for(h, nt), kBlock, 0, s>>>(nt, e.A, 0x2468aceu);
        } else {
            if (M.band_n.empty()) return -1.0;
            // first band down: deltas and segments of its levels read, the
            // parents read, z written, r read for the reductions
            const BandParams<V> &P = M.band_n[0];
            by = 2.0 * sv * static_cast<double>(n);
            for (int k = 0; k < P.nlev; ++k) by += sv * M.lev[k].n + 4.0 * (M.lev[k].nagg + 1);
            by += sv * static_cast<double>(M.off[P.nlev + 1] - M.off[P.nlev]);
        }
        // (kernel 8 overwrites its right-hand side in A with deltas; the values
        // it leaves are as valid a right-hand side for the next launch)
        launch();                                   // warm-up
        cudaEventRecord(e0, s);
        for (int i = 0; i < reps; ++i) launch();
        cudaEventRecord(e1, s);
        return by;
    };
    const double by = precision == 1 ? run(float{}) : run(double{});
    if (by < 0) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return LAP_ERR_INVALID_ARG;
    }
    LAP_CK(cudaEventSynchronize(e1));
    float t = 0.f;
    LAP_CK(cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = static_cast<double>(t) / reps;
    *bytes = by;
    if (kernel == 7) {
        // every timed iteration must have run to its end
        CgScalars sc;
        LAP_TRY(poll(h, h.stb, sc));
        if (sc.flag != kRun) return LAP_ERR_BREAKDOWN;
    }
    return LAP_OK;
}

}  // namespace lap
