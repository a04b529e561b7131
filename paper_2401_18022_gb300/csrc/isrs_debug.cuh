// Bounds checks of the debug build (nvcc -DISRS_DEBUG).  A failed check
// records its code in the launch's flag (the first failure wins) and clamps
// the index into range, so no access leaves its array and every thread still
// reaches every barrier; the host reads the flag after the call and returns
// ISRS_ERR_CHECK.  The release build compiles the checks away.
#pragma once
#include <cuda_runtime.h>

namespace isrs {

enum DbgCode : unsigned {
    kDbgPiece = 1,      // piece index of a work tile outside the piece list
    kDbgRow = 2,        // grid row outside [0, G)
    kDbgCand = 3,       // F_c candidate outside the piece's candidates
    kDbgList = 4,       // per-warp point list overflow
    kDbgVrow = 5,       // PSD bucket channel outside the plan
    kDbgCell = 6,       // MCI cell decoded outside the plan
};

__device__ __forceinline__ int dbg_clamp(int i, int n, unsigned code, unsigned *flag)
{
#ifdef ISRS_DEBUG
    if (i < 0 || i >= n) {
        if (flag) atomicCAS(flag, 0u, code);
        return i < 0 || n <= 0 ? 0 : n - 1;
    }
#else
    (void)n;
    (void)code;
    (void)flag;
#endif
    return i;
}

}  // namespace isrs
