// Device helpers shared by the quadrature kernels (forward and adjoint).
#pragma once
#include <cuda_runtime.h>

#include "isrs_internal.cuh"

namespace isrs {

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// nearest integer of |t| < 2^22 on the FMA pipe (round-to-nearest-even add)
__device__ __forceinline__ float round_magic(float t)
{
    return __fadd_rn(__fadd_rn(t, 12582912.0f), -12582912.0f);
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum of one double per thread (blockDim multiple of 32).
__device__ __forceinline__ double block_sum_d(double v, double *scratch)
{
    v = warp_sum_d(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += scratch[w];
        scratch[0] = r;
    }
    __syncthreads();
    r = scratch[0];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// Piece set-up shared by the quadrature kernels (FP64, once per piece).
// Row r (uniform in s = ln upsilon1): upsilon1 = exp(s_r); the |f2| range
// [ymin, ymax] of that row; upsilon2 spans ln(ymax/ymin) in G columns.
// Stored relative to the row centre so FP32 points keep full precision:
//   x_j = xc e^{d_j}, y_j = yc e^{-d_j}, d_j = (j + 1/2 - G/2) du2,
//   weight = upsilon1 ds du2 (the Jacobian of (f1, f2) -> (u1, u2) is 1).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void piece_rows(const DevPiece &pc, int G, double eps, T *rows)
{
    const double u1hi = pc.xhi * pc.yhi;
    const double u1lo = fmax(pc.xlo * pc.ylo, eps * u1hi);
    const double llo = log(u1lo);
    const double ds = (log(u1hi) - llo) / G;
    for (int r = threadIdx.x; r < G; r += blockDim.x) {
        const double u1 = exp(llo + (r + 0.5) * ds);
        const double ymin = fmax(pc.ylo, u1 / pc.xhi);
        const double ymax = pc.xlo > 0.0 ? fmin(pc.yhi, u1 / pc.xlo) : pc.yhi;
        T rw;
        if (ymax > ymin) {
            const double du2 = log1p((ymax - ymin) / ymin) / G;
            const double yc = sqrt(ymin * ymax);
            rw.xc = u1 / yc;
            rw.yc = yc;
            rw.du2 = du2;
            rw.w = u1 * ds * du2;
        } else {
            rw.xc = 0; rw.yc = 0; rw.du2 = 0; rw.w = 0;
        }
        rows[r] = rw;
    }
}

struct RowF { float xc, yc, du2, w; };
struct RowD { double xc, yc, du2, w; };

// Per-piece constants: CUT offset, signs, the PSD factors of F_a and F_b, the
// attenuation part of ln p and the candidate channels of F_c (edges relative
// to the CUT so that F_c - f_i = f1 + f2 is compared without cancellation).
template <typename T>
struct PieceConst {
    T fi, s1, s2, wab, at_ab, mult;
    int nc;
    T lo[kMaxCand], hi[kMaxCand], pd[kMaxCand], hat[kMaxCand];
};

template <typename T>
__device__ __forceinline__ void piece_consts(const QuadParams &qp, const DevPiece &pc, int prof, T at_scale,
                             const T *pdv, PieceConst<T> &k)
{
    if (threadIdx.x == 0) {
        const int coff = qp.plan_ch_off[pc.plan];
        const int poff = qp.prof_ch_off[prof];
        const double fi = qp.ch_frel[coff + pc.cut];
        k.fi = (T)fi;
        k.s1 = (pc.flags & 1) ? T(-1) : T(1);
        k.s2 = (pc.flags & 2) ? T(-1) : T(1);
        k.wab = pdv[poff + pc.a] * pdv[poff + pc.b];
        k.at_ab = (T)(0.5 * (qp.ch_alpha[coff + pc.a] + qp.ch_alpha[coff + pc.b] -
                             qp.ch_alpha[coff + pc.cut])) * at_scale;
        k.mult = (T)pc.mult;
        int nc = 0;
        for (int c = pc.c_lo; c <= pc.c_hi && nc < kMaxCand; ++c, ++nc) {
            const double fc = qp.ch_frel[coff + c], hb = 0.5 * qp.ch_B[coff + c];
            k.lo[nc] = (T)((fc - hb) - fi);
            k.hi[nc] = (T)((fc + hb) - fi);
            k.pd[nc] = pdv[poff + c];
            k.hat[nc] = (T)(0.5 * qp.ch_alpha[coff + c]) * at_scale;
        }
        k.nc = nc;
    }
}

__device__ __forceinline__ void sincos_rev(float t, float &sn, float &cs)
{
    const float fr = __fadd_rn(t, -round_magic(t));
    __sincosf(fr * 6.283185307179586f, &sn, &cs);
}

__device__ __forceinline__ void phasor_rev_ff(float phi, float hi, float lo, float &sn, float &cs)
{
    const float th = phi * hi;
    float tl = fmaf(phi, hi, -th);
    tl = fmaf(phi, lo, tl);
    const float fr = __fadd_rn(th, -round_magic(th)) + tl;
    __sincosf(fr * 6.283185307179586f, &sn, &cs);
}


}  // namespace isrs
