// Instantiations of the product kernels for the paper's precision variants
// (Section 3, Table 1): stores PM, PS, PM1 and PS2 (FP32 panels, FP64 operands).
// Their FP64 segments (Method 2-Double, the FP64 part of Method 3) use the F64
// kernels of kernels.cu.
#include "product.cuh"

namespace hmat_internal {

#define HMAT_T1_DISPATCH(S, CALL)                                   \
    switch (S) {                                                    \
    case Store::PM: { constexpr Store SS = Store::PM; CALL; } break;   \
    case Store::PS: { constexpr Store SS = Store::PS; CALL; } break;   \
    case Store::PM1: { constexpr Store SS = Store::PM1; CALL; } break; \
    case Store::PS2: { constexpr Store SS = Store::PS2; CALL; } break; \
    default: break;                                                 \
    }

void launch_phase1_table1(Store s, const DevIndex &ix, const DevPanels &P, const SolverScalars *skipS, int mode,
                          cudaStream_t st, const SysScalars *sys) {
    HMAT_T1_DISPATCH(s, phase1_launch<SS>(ix, P, skipS, mode, st, sys));
}

void launch_reduce_table1(Store s, const DevIndex &ix, const DevPanels &P, const SolverScalars *skipS, int mode,
                          cudaStream_t st, const SysScalars *sys) {
    HMAT_T1_DISPATCH(s, reduce_launch<SS>(ix, P, skipS, mode, st, sys));
}

void launch_phase2_table1(Store s, const DevIndex &ix, const DevPanels &P, double *y, const int32_t *out_perm,
                          int accum, const SolverScalars *skipS, int mode, cudaStream_t st, const double *w,
                          int dotmode, double *dpart, const SysScalars *sys) {
    HMAT_T1_DISPATCH(s, phase2_launch<SS>(ix, P, y, out_perm, accum, skipS, mode, st, w, dotmode, dpart, sys));
}

}  // namespace hmat_internal
