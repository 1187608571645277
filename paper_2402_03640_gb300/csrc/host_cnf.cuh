// Host-side CNF preparation of msat_create (host_cnf.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <vector>

namespace msat {

// An int32 array that is not zero-filled when sized (its filler threads
// write every element).
struct I32Buf {
    std::unique_ptr<int32_t[]> p;
    size_t len = 0;
    void alloc(size_t k) {
        p.reset(new int32_t[k > 0 ? k : 1]);
        len = k;
    }
    int32_t *data() { return p.get(); }
    const int32_t *data() const { return p.get(); }
    size_t size() const { return len; }
    int32_t &operator[](size_t i) { return p[i]; }
    const int32_t &operator[](size_t i) const { return p[i]; }
    int32_t *begin() { return p.get(); }
    int32_t *end() { return p.get() + len; }
};

// A checked CNF in canonical form (repeated literals dropped, first
// occurrence kept) with its transpose.  lit = var << 1 | neg; occ =
// clause << 1 | neg in (clause, position) order per variable.
struct HostCnf {
    I32Buf coff;  // [m+1]
    I32Buf lit;   // [nnz]
    I32Buf voff;  // [n+1]
    I32Buf occ;   // [nnz]
    std::vector<int32_t> clen;  // [m] canonical clause lengths
    std::vector<uint8_t> taut;  // [m] clause holds some x and not x
    int64_t nnz = 0;
    int64_t wsum = 0;           // total clause weight
    int32_t max_len = 0, max_deg = 0;
    int32_t kfix = 0;           // common clause length, or 0
    // between build_host_cnf and scatter_occurrences: thread t's first
    // occurrence slot of variable i at [t * n + i]
    std::unique_ptr<int32_t[]> slots;
    int slot_threads = 0;
};

// Checks the caller's arrays (offsets non-decreasing from 0, literals in
// range, weights >= 1, canonical clauses of at most kMaxClauseLen literals)
// and fills `out` up to the occurrence offsets (voff); MSAT_EINVAL with the
// message of the first violation in input order.  The work is spread over
// the host's hardware threads.
int build_host_cnf(int32_t n, int64_t m, const int64_t *off, const int32_t *lits, const int64_t *w,
                   HostCnf &out);

// Rows of the clause pass's store of w*f grouped by the variable pass's
// light blocks: a clause's home is the block of its first light variable
// (clauses with none come last), the groups run from the last block down to
// the first and keep clause order inside.  row[j] is clause j's row; plit (and pcoff
// for clauses of different lengths, pw for weights) are the clause arrays
// in row order, which the clause pass reads.
struct RowOrder {
    I32Buf row;               // [m]
    I32Buf plit;              // [nnz]
    I32Buf pcoff;             // [m+1], empty when every clause has kfix literals
    std::vector<int64_t> pw;  // [m] or empty
};

int build_block_rows(int32_t n, int64_t m, int32_t kfix, const I32Buf &coff, const I32Buf &lit,
                     const int64_t *w, const std::vector<int2> &lblk, RowOrder &ro);

// The occurrence list (transposed CSR, each variable's occurrences in
// (clause, position) order): words row << 1 | neg, with row = row[j] of
// clause j when `row` is given (the grouped store), else j.
void scatter_occurrences(int32_t n, int64_t m, HostCnf &hc, const I32Buf *row);

}  // namespace msat
