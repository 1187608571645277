// Host side of msat_create: check the caller's CNF, make its clauses
// canonical and build the transposed CSR, spread over the host's cores.
//
// The result is the one a single thread produces, bit for bit: clauses keep
// their order and their literals the order of their first occurrence; the
// occurrence list of each variable is in (clause, position) order.  Each
// thread takes a contiguous range of clauses (or literals), and the
// per-thread pieces are joined in range order; every reported error is the
// first one in input order, as a sequential scan would find it.

#include <stdint.h>

#include <algorithm>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "msat_internal.cuh"
#include "host_cnf.cuh"

namespace msat {

namespace {

// Runs f(t, begin, end) on T threads over [0, N) in T contiguous ranges.
template <class F>
void parallel_ranges(int64_t N, int T, F f) {
    if (T <= 1 || N < 2) {
        f(0, (int64_t)0, N);
        return;
    }
    std::vector<std::thread> th;
    th.reserve((size_t)T);
    for (int t = 0; t < T; ++t) {
        const int64_t b = N * t / T, e = N * (t + 1) / T;
        th.emplace_back([=, &f] { f(t, b, e); });
    }
    for (auto &x : th) x.join();
}

int threads_for(int64_t work) {
    unsigned hc = std::thread::hardware_concurrency();
    if (hc == 0) hc = 1;
    int64_t t = std::min<int64_t>((int64_t)hc, 32);
    t = std::min<int64_t>(t, std::max<int64_t>(1, work / (1 << 16)));
    return (int)t;
}

}  // namespace

int build_host_cnf(int32_t n, int64_t m, const int64_t *off, const int32_t *lits, const int64_t *w,
                   HostCnf &out) {
    if (off[0] != 0) return fail(MSAT_EINVAL, "msat_create: clause_off[0] must be 0");
    const int Tm = threads_for(m);
    {
        std::vector<int64_t> bad((size_t)Tm, -1);
        parallel_ranges(m, Tm, [&](int t, int64_t b, int64_t e) {
            for (int64_t j = b; j < e; ++j)
                if (off[j + 1] < off[j]) {
                    bad[(size_t)t] = j;
                    return;
                }
        });
        for (int64_t j : bad)
            if (j >= 0)
                return fail(MSAT_EINVAL, "msat_create: clause_off is not non-decreasing at clause " +
                                             std::to_string(j));
    }
    const int64_t raw = off[m];
    if (raw > 0 && !lits) return fail(MSAT_EINVAL, "msat_create: lits is NULL");
    if (raw >= (1LL << 31)) return fail(MSAT_EINVAL, "msat_create: more than 2^31-1 literals");
    {
        const int Tq = threads_for(raw);
        std::vector<int64_t> bad((size_t)Tq, -1);
        parallel_ranges(raw, Tq, [&](int t, int64_t b, int64_t e) {
            for (int64_t q = b; q < e; ++q) {
                const int32_t l = lits[q];
                if (l == 0 || l > n || l < -n) {
                    bad[(size_t)t] = q;
                    return;
                }
            }
        });
        for (int64_t q : bad)
            if (q >= 0)
                return fail(MSAT_EINVAL, "msat_create: literal " + std::to_string(lits[q]) + " at position " +
                                             std::to_string(q) + " is 0 or names no variable");
    }
    if (w) {
        std::vector<int64_t> bad((size_t)Tm, -1);
        parallel_ranges(m, Tm, [&](int t, int64_t b, int64_t e) {
            for (int64_t j = b; j < e; ++j)
                if (w[j] < 1) {
                    bad[(size_t)t] = j;
                    return;
                }
        });
        for (int64_t j : bad)
            if (j >= 0)
                return fail(MSAT_EINVAL, "msat_create: weight of clause " + std::to_string(j) + " is below 1");
    }

    // canonical clauses: drop a literal equal to an earlier one of its clause
    // (the first occurrence keeps its place); after that a variable seen
    // twice in a clause appears as x and not x, and the clause can never be
    // unsat.  Short clauses compare pairwise; a long one marks literals and
    // variables in the thread's own arrays (marked with the clause index).
    struct Part {
        std::vector<int32_t> lit;
        int64_t wsum = 0;
        int32_t max_len = 0;
        int32_t first_len = -1;  // length of the part's first clause
        bool same_len = true;    // every clause of the part has first_len literals
        int64_t too_long = -1;
        std::vector<int32_t> seen, vseen;
    };
    std::vector<Part> parts((size_t)Tm);
    out.clen.assign((size_t)m, 0);
    out.taut.assign((size_t)m, 0);
    parallel_ranges(m, Tm, [&](int t, int64_t b, int64_t e) {
        Part &P = parts[(size_t)t];
        P.lit.reserve((size_t)(off[e] - off[b]));
        for (int64_t j = b; j < e; ++j) {
            const size_t start = P.lit.size();
            const int64_t len_in = off[j + 1] - off[j];
            bool taut = false;
            if (len_in <= 32) {
                for (int64_t p = off[j]; p < off[j + 1]; ++p) {
                    const int32_t l = lits[p];
                    const int32_t packed = ((std::abs(l) - 1) << 1) | (l < 0 ? 1 : 0);
                    bool dup = false;
                    for (size_t r = start; r < P.lit.size(); ++r) {
                        if (P.lit[r] == packed) dup = true;
                        else if ((P.lit[r] >> 1) == (packed >> 1)) taut = true;
                    }
                    if (!dup) P.lit.push_back(packed);
                }
            } else {
                if (P.seen.empty()) {
                    P.seen.assign((size_t)n * 2, -1);
                    P.vseen.assign((size_t)n, -1);
                }
                for (int64_t p = off[j]; p < off[j + 1]; ++p) {
                    const int32_t l = lits[p];
                    const int32_t packed = ((std::abs(l) - 1) << 1) | (l < 0 ? 1 : 0);
                    if (P.seen[(size_t)packed] == (int32_t)j) continue;
                    P.seen[(size_t)packed] = (int32_t)j;
                    P.lit.push_back(packed);
                    if (P.vseen[(size_t)(packed >> 1)] == (int32_t)j) taut = true;
                    P.vseen[(size_t)(packed >> 1)] = (int32_t)j;
                }
            }
            const int32_t len = (int32_t)(P.lit.size() - start);
            if (P.first_len < 0) P.first_len = len;
            P.same_len = P.same_len && len == P.first_len;
            if (len > kMaxClauseLen && P.too_long < 0) P.too_long = j;
            P.max_len = std::max(P.max_len, len);
            out.clen[(size_t)j] = len;
            out.taut[(size_t)j] = taut ? 1 : 0;
            P.wsum += w ? w[j] : 1;
        }
    });
    for (const Part &P : parts)
        if (P.too_long >= 0)
            return fail(MSAT_EINVAL, "msat_create: clause " + std::to_string(P.too_long) + " has " +
                                         std::to_string(out.clen[(size_t)P.too_long]) +
                                         " literals (limit " + std::to_string(kMaxClauseLen) + ")");
    // join the parts in clause order
    std::vector<int64_t> lbase((size_t)Tm + 1, 0);
    out.wsum = 0;
    out.max_len = 0;
    for (int t = 0; t < Tm; ++t) {
        lbase[(size_t)t + 1] = lbase[(size_t)t] + (int64_t)parts[(size_t)t].lit.size();
        out.wsum += parts[(size_t)t].wsum;
        out.max_len = std::max(out.max_len, parts[(size_t)t].max_len);
    }
    out.nnz = lbase[(size_t)Tm];
    out.lit.alloc((size_t)out.nnz);
    out.coff.alloc((size_t)m + 1);
    out.coff[0] = 0;
    parallel_ranges(m, Tm, [&](int t, int64_t b, int64_t e) {
        const Part &P = parts[(size_t)t];
        std::copy(P.lit.begin(), P.lit.end(), out.lit.data() + lbase[(size_t)t]);
        int64_t at = lbase[(size_t)t];
        for (int64_t j = b; j < e; ++j) {
            at += out.clen[(size_t)j];
            out.coff[(size_t)j + 1] = (int32_t)at;
        }
    });
    // the common clause length (0 if the lengths differ), from the parts'
    out.kfix = 0;
    if (m > 0) {
        out.kfix = out.clen[0];
        for (const Part &P : parts)
            if (P.first_len >= 0 && (!P.same_len || P.first_len != out.kfix)) out.kfix = 0;
    }
    parts.clear();

    // transposed CSR, stable: per-thread counts of each variable's
    // occurrences in the thread's clause range, turned into per-thread
    // write positions (earlier ranges first), then one scatter pass
    int Tt = threads_for(out.nnz);
    while (Tt > 1 && (int64_t)Tt * n > (int64_t)64 << 20) --Tt;  // counts within 256 MB
    std::unique_ptr<int32_t[]> cnt(new int32_t[(size_t)Tt * n]);
    parallel_ranges(m, Tt, [&](int t, int64_t b, int64_t e) {
        int32_t *c = cnt.get() + (size_t)t * n;
        std::fill(c, c + n, 0);
        for (int64_t p = out.coff[(size_t)b]; p < out.coff[(size_t)e]; ++p) ++c[out.lit[(size_t)p] >> 1];
    });
    // occurrence offsets: the variables split into Tt ranges; each range's
    // degrees and total, the ranges' starts in order, then each range's
    // offsets and every thread's first slot per variable
    out.voff.alloc((size_t)n + 1);
    std::vector<int64_t> rtot((size_t)Tt + 1, 0);
    std::vector<int32_t> rmax((size_t)Tt, 0);
    parallel_ranges(n, Tt, [&](int r, int64_t b, int64_t e) {
        int64_t tot = 0;
        int32_t mx = 0;
        for (int64_t i = b; i < e; ++i) {
            int32_t d = 0;
            for (int t = 0; t < Tt; ++t) d += cnt[(size_t)t * n + (size_t)i];
            tot += d;
            mx = std::max(mx, d);
        }
        rtot[(size_t)r + 1] = tot;
        rmax[(size_t)r] = mx;
    });
    out.max_deg = 0;
    for (int r = 0; r < Tt; ++r) {
        rtot[(size_t)r + 1] += rtot[(size_t)r];
        out.max_deg = std::max(out.max_deg, rmax[(size_t)r]);
    }
    parallel_ranges(n, Tt, [&](int r, int64_t b, int64_t e) {
        int64_t acc = rtot[(size_t)r];
        for (int64_t i = b; i < e; ++i) {
            out.voff[(size_t)i] = (int32_t)acc;
            for (int t = 0; t < Tt; ++t) {
                int32_t &c = cnt[(size_t)t * n + (size_t)i];
                const int32_t k = c;
                c = (int32_t)acc;  // thread t's first slot for variable i
                acc += k;
            }
        }
    });
    out.voff[(size_t)n] = (int32_t)rtot[(size_t)Tt];
    // every thread's first slot per variable, for scatter_occurrences
    out.slots = std::move(cnt);
    out.slot_threads = Tt;
    return MSAT_OK;
}

void scatter_occurrences(int32_t n, int64_t m, HostCnf &hc, const I32Buf *row) {
    const int Tt = hc.slot_threads;
    hc.occ.alloc((size_t)hc.nnz);
    parallel_ranges(m, Tt, [&](int t, int64_t b, int64_t e) {
        int32_t *c = hc.slots.get() + (size_t)t * n;
        for (int64_t j = b; j < e; ++j) {
            const int32_t r = row ? (*row)[(size_t)j] : (int32_t)j;
            for (int32_t p = hc.coff[(size_t)j]; p < hc.coff[(size_t)j + 1]; ++p) {
                const int32_t L = hc.lit[(size_t)p];
                hc.occ[(size_t)c[L >> 1]++] = (r << 1) | (L & 1);
            }
        }
    });
    hc.slots.reset();
}

}  // namespace msat

namespace msat {

int build_block_rows(int32_t n, int64_t m, int32_t kfix, const I32Buf &coff, const I32Buf &lit,
                     const int64_t *w, const std::vector<int2> &lblk, RowOrder &ro) {
    // light block of every light variable (-1: heavy)
    std::vector<int32_t> vblk((size_t)n, -1);
    for (size_t b = 0; b < lblk.size(); ++b)
        for (int32_t v = lblk[b].x; v < lblk[b].y; ++v) vblk[(size_t)v] = (int32_t)b;
    const int32_t nb = (int32_t)lblk.size();
    // home block of each clause: that of its first light variable (nb: none)
    ro.row.alloc((size_t)m);
    I32Buf home;
    home.alloc((size_t)m);
    const int T = threads_for(m);
    std::vector<std::vector<int64_t>> cnt((size_t)T, std::vector<int64_t>((size_t)nb + 1, 0));
    parallel_ranges(m, T, [&](int t, int64_t b, int64_t e) {
        for (int64_t j = b; j < e; ++j) {
            int32_t h = nb;
            for (int32_t p = coff[(size_t)j]; p < coff[(size_t)j + 1]; ++p) {
                const int32_t vb = vblk[(size_t)(lit[(size_t)p] >> 1)];
                if (vb >= 0) {
                    h = vb;
                    break;
                }
            }
            home[(size_t)j] = h;
            ++cnt[(size_t)t][(size_t)h];
        }
    });
    // rows grouped by home block, clause order inside a group (stable):
    // thread t's clauses of home h start after every earlier thread's.
    // The groups run from the last light block down to the first, then the
    // clauses with no light variable: the clause pass writes the rows of
    // the variable pass's first blocks last, so more of them are still in
    // L2 when that pass starts.
    int64_t at = 0;
    for (int32_t g = 0; g <= nb; ++g)
        for (int t = 0; t < T; ++t) {
            const int32_t h = g < nb ? nb - 1 - g : nb;
            const int64_t k = cnt[(size_t)t][(size_t)h];
            cnt[(size_t)t][(size_t)h] = at;
            at += k;
        }
    // each clause's row; with a common length the literals go to their row
    // in the same pass, and the clause pass's arrays follow in row order
    const int64_t nnz = (int64_t)lit.size();
    ro.plit.alloc((size_t)nnz);
    parallel_ranges(m, T, [&](int t, int64_t b, int64_t e) {
        std::vector<int64_t> &c = cnt[(size_t)t];
        for (int64_t j = b; j < e; ++j) {
            const int32_t r = (int32_t)c[(size_t)home[(size_t)j]]++;
            ro.row[(size_t)j] = r;
            if (kfix > 0)
                for (int32_t p = 0; p < kfix; ++p)
                    ro.plit[(size_t)r * kfix + p] = lit[(size_t)j * kfix + p];
        }
    });
    if (kfix == 0) {
        I32Buf len;
        len.alloc((size_t)m);
        parallel_ranges(m, T, [&](int, int64_t b, int64_t e) {
            for (int64_t j = b; j < e; ++j)
                len[(size_t)ro.row[(size_t)j]] = coff[(size_t)j + 1] - coff[(size_t)j];
        });
        ro.pcoff.alloc((size_t)m + 1);
        ro.pcoff[0] = 0;
        for (int64_t r = 0; r < m; ++r) ro.pcoff[(size_t)r + 1] = ro.pcoff[(size_t)r] + len[(size_t)r];
        parallel_ranges(m, T, [&](int, int64_t b, int64_t e) {
            for (int64_t j = b; j < e; ++j) {
                int32_t q = ro.pcoff[(size_t)ro.row[(size_t)j]];
                for (int32_t p = coff[(size_t)j]; p < coff[(size_t)j + 1]; ++p) ro.plit[(size_t)q++] = lit[(size_t)p];
            }
        });
    }
    if (w) {
        ro.pw.resize((size_t)m);
        parallel_ranges(m, T, [&](int, int64_t b, int64_t e) {
            for (int64_t j = b; j < e; ++j) ro.pw[(size_t)ro.row[(size_t)j]] = w[j];
        });
    }
    return MSAT_OK;
}

}  // namespace msat
