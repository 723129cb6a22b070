// Host build of the SpMV layout builder (the same header the solver uses),
// for CPU tests of the invariants its kernel relies on.
#include <cstring>

#include "../paper_1312_3039_gb300/csrc/spmv.cuh"

// threads: host threads of the copy (0: the solver's choice); the values of
// the layout are the source positions of the entries (out_val, may be null)
extern "C" int host_spmv_layout_t(int rows, const int32_t *rowptr, const int32_t *col, int ctas, int threads,
                                  int32_t *out_rowptr, int32_t *out_col, int32_t *out_rowid, int32_t *info,
                                  double *out_val) {
    std::vector<int32_t> rp(rowptr, rowptr + rows + 1), cl(col, col + rowptr[rows]);
    std::vector<double> vl(cl.size());
    for (size_t t = 0; t < vl.size(); ++t) vl[t] = (double)t;
    scs::SpmvLayout<double> L = scs::spmv_layout(rp, cl, vl, ctas, threads);
    if (out_val) std::memcpy(out_val, L.val.data(), sizeof(double) * L.val.size());
    std::memcpy(out_rowptr, L.rowptr.data(), sizeof(int32_t) * L.rowptr.size());
    std::memcpy(out_col, L.col.data(), sizeof(int32_t) * L.col.size());
    std::memcpy(out_rowid, L.rowid.data(), sizeof(int32_t) * L.rowid.size());
    info[0] = L.reg.n;
    for (int k = 0; k < L.reg.n; ++k) {
        info[1 + 4 * k] = L.reg.row0[k];
        info[2 + 4 * k] = L.reg.row1[k];
        info[3 + 4 * k] = L.reg.lanes[k];
        info[4 + 4 * k] = L.reg.cta0[k + 1] - L.reg.cta0[k];
    }
    return 0;
}

extern "C" int host_spmv_layout(int rows, const int32_t *rowptr, const int32_t *col, int ctas, int32_t *out_rowptr,
                                int32_t *out_col, int32_t *out_rowid, int32_t *info) {
    return host_spmv_layout_t(rows, rowptr, col, ctas, 0, out_rowptr, out_col, out_rowid, info, nullptr);
}

// tile table of the layout above (first stored row of each tile, ntiles + 1
// entries; 0 entries when no row length calls for tiles); returns the count
extern "C" int host_spmv_tiles(int rows, const int32_t *rowptr, const int32_t *col, int ctas, int32_t *out,
                               int cap) {
    std::vector<int32_t> rp(rowptr, rowptr + rows + 1), cl(col, col + rowptr[rows]);
    std::vector<double> vl(cl.size(), 1.0);
    scs::SpmvLayout<double> L = scs::spmv_layout(rp, cl, vl, ctas);
    const int n = static_cast<int>(L.tile_row.size());
    if (n > cap) return -1;
    if (n) std::memcpy(out, L.tile_row.data(), sizeof(int32_t) * n);
    return n;
}

// 1 when the plan-only layout (copy = false, empty column and value arrays,
// as the solver builds it before gathering rows on the device) has the same
// row order, row starts, regions and tiles as the copying layout
extern "C" int host_spmv_plan_matches(int rows, const int32_t *rowptr, const int32_t *col, int ctas) {
    std::vector<int32_t> rp(rowptr, rowptr + rows + 1), cl(col, col + rowptr[rows]), none;
    std::vector<double> vl(cl.size(), 1.0), nonev;
    scs::SpmvLayout<double> A = scs::spmv_layout(rp, cl, vl, ctas);
    scs::SpmvLayout<double> B = scs::spmv_layout(rp, none, nonev, ctas, 0, false);
    if (!B.col.empty() || !B.val.empty()) return 0;
    if (A.rowid != B.rowid || A.rowptr != B.rowptr || A.tile_row != B.tile_row) return 0;
    if (A.reg.n != B.reg.n) return 0;
    for (int k = 0; k < A.reg.n; ++k)
        if (A.reg.row0[k] != B.reg.row0[k] || A.reg.row1[k] != B.reg.row1[k] || A.reg.lanes[k] != B.reg.lanes[k] ||
            A.reg.cta0[k + 1] != B.reg.cta0[k + 1])
            return 0;
    return 1;
}
