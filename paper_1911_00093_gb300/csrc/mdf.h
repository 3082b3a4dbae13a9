// The double-float H-matrix product of several columns at once (multi_df.cu).
#pragma once

#include "kernels.h"

namespace hmat_internal {

constexpr int kMdfCols = 16;  // columns per pass: the work buffers hold one pass

// Work buffers of the many-column double-float product: the operand copies,
// the projections T and the phase-2 operands of kMdfCols columns, each column
// a whole copy of its one-column buffer (double-float pairs, float2).
struct MdfBufs {
    int cap = 0;                                          // columns held (0: not allocated)
    void *xs = nullptr, *part = nullptr, *g = nullptr;    // [cap][ldxs], [cap][ldt], [cap][ldg]
    int64_t ldxs = 0, ldt = 0, ldg = 0;                   // entries per column
};

// y(:, k) = A x(:, k) for the columns k = cols[j], j < ncols (k = j when cols
// is null; cols is a device array) with the double-float panels of (ix, P), x
// and y in cluster order, columns ldx and ldy apart.  Every column's result is
// bit for bit the one-column product's (enqueue of prep, phase 1, reduce and
// phase 2 with Store::DF).
// sys != nullptr (many-system solver; sys[k * nprob + p] is system (p, k)):
//   sysmode 1 skips the work of a system whose run has stopped (state or flag
//   set); sysmode 2 keeps only that of a system awaiting its true residual
//   (its run stopped: flag set, state not); the skipped rows of y are left as
//   they were.
void launch_mdf_product(const DevIndex &ix, const DevPanels &P, const MdfBufs &b, const double *x, int64_t ldx,
                        double *y, int64_t ldy, int ncols, const int32_t *cols, const SysScalars *sys, int sysmode,
                        int nprob, cudaStream_t st);
// kernel launches of one such product of ncols columns
int mdf_launches(const DevIndex &ix, int ncols);

}  // namespace hmat_internal
