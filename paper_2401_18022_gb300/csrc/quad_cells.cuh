// Cell decoding of the multi-channel-interference (MCI) grid, shared by the
// MCI quadrature and its adjoint: a work item is a range of cells (a, b),
// a <= b, a, b != CUT, in triangular order over the other N - 1 channels.
#pragma once
#include <cuda_runtime.h>

namespace isrs {

// (a', b') of triangular index t over n2 channels: rows a' hold n2 - a'
// pairs starting at S(a') = a' (2 n2 - a' + 1) / 2.
__device__ __forceinline__ void tri_decode(int t, int n2, int &ap, int &bp)
{
    const float q = 2.0f * n2 + 1.0f;
    int a = (int)floorf(0.5f * (q - sqrtf(fmaxf(q * q - 8.0f * (float)t, 0.0f))));
    a = max(0, min(a, n2 - 1));
    while (a > 0 && a * (2 * n2 - a + 1) / 2 > t) --a;
    while (a + 1 < n2 && (a + 1) * (2 * n2 - a) / 2 <= t) ++a;
    ap = a;
    bp = a + (t - a * (2 * n2 - a + 1) / 2);
}

// index of the channel containing offset u from the CUT, or -1
// (lo[c] = rel[c] - hb[c] ascending, channels disjoint)
template <typename T>
__device__ __forceinline__ int channel_of(const T *rel, const T *hb, int n, T u)
{
    int lo = 0, hi = n - 1, c = -1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        if (rel[mid] - hb[mid] <= u) {
            c = mid;
            lo = mid + 1;
        } else {
            hi = mid - 1;
        }
    }
    return (c >= 0 && u < rel[c] + hb[c]) ? c : -1;
}

}  // namespace isrs
