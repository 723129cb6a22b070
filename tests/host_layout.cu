// Host build of the SpMV layout builder (the same header the solver uses),
// for CPU tests of the invariants its kernel relies on.
#include <cstring>

#include "../paper_1312_3039_gb300/csrc/spmv.cuh"

extern "C" int host_spmv_layout(int rows, const int32_t *rowptr, const int32_t *col, int grid, int32_t *out_rowptr,
                                int32_t *out_col, int32_t *out_rowid, int32_t *out_chunk, int32_t *out_kind,
                                int32_t *out_cta, int32_t *counts, int max_chunks) {
    std::vector<int32_t> rp(rowptr, rowptr + rows + 1), cl(col, col + rowptr[rows]);
    std::vector<double> vl(cl.size(), 1.0);
    scs::SpmvLayout<double> L = scs::spmv_layout(rp, cl, vl, grid);
    if (L.nchunk > max_chunks) return -1;
    std::memcpy(out_rowptr, L.rowptr.data(), sizeof(int32_t) * L.rowptr.size());
    std::memcpy(out_col, L.col.data(), sizeof(int32_t) * L.col.size());
    std::memcpy(out_rowid, L.rowid.data(), sizeof(int32_t) * L.rowid.size());
    std::memcpy(out_chunk, L.chunk.data(), sizeof(int32_t) * L.chunk.size());
    std::memcpy(out_kind, L.kind.data(), sizeof(int32_t) * L.kind.size());
    std::memcpy(out_cta, L.cta_item.data(), sizeof(int32_t) * L.cta_item.size());
    counts[0] = L.nchunk;
    counts[1] = 0;
    counts[2] = L.grid;
    counts[3] = scs::kChunkNnz;
    counts[4] = scs::kChunkRows;
    counts[5] = scs::kPad;
    counts[6] = (int)scs::SpmvSmem<float, float>::kColWords;
    counts[7] = (int)scs::SpmvSmem<float, float>::kRowWords;
    return 0;
}
