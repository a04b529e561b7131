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


__device__ __forceinline__ double sinc_d(double x)
{
    return fabs(x) < 1e-4 ? 1.0 - x * x / 6.0 : sin(x) / x;
}

// Phased-array factor of n identical spans (Eq. new_gn_model with
// L-tilde_k = (k-1) L): |sum_{k<n} e^{j k phi L}|^2, by rotation from the
// float-float phase phi L / 2pi.
__device__ __forceinline__ float array_factor_f(float phi, const QuadParams &qp)
{
    if (qp.n_spans <= 1) return 1.0f;
    float sn, cs;
    phasor_rev_ff(phi, qp.Lrev_hi, qp.Lrev_lo, sn, cs);
    float sr = 0.0f, si = 0.0f, zr = 1.0f, zi = 0.0f;
    for (int k = 0; k < qp.n_spans; ++k) {
        sr += zr;
        si += zi;
        const float t = fmaf(zr, cs, -zi * sn);
        zi = fmaf(zr, sn, zi * cs);
        zr = t;
    }
    return fmaf(sr, sr, si * si);
}

__device__ __forceinline__ double array_factor_d(double phi, const QuadParams &qp)
{
    if (qp.n_spans <= 1) return 1.0;
    double sn, cs;
    sincos(phi * qp.Ld, &sn, &cs);
    double sr = 0.0, si = 0.0, zr = 1.0, zi = 0.0;
    for (int k = 0; k < qp.n_spans; ++k) {
        sr += zr;
        si += zi;
        const double t = zr * cs - zi * sn;
        zi = zr * sn + zi * cs;
        zr = t;
    }
    return sr * sr + si * si;
}

// ---------------------------------------------------------------------------
// Chebyshev contraction of the small-phase moments (App. A, Eq. slow_vary to
// second order in phi).  Inside candidate channel c, F_c - f_ref = F0 + h x
// with x in [-1, 1], and the per-step weight factorises:
//   w_m = 2^{A2d_m + K2_m F_c - at z_m} = 2^{A2d_m - at z_m + K2_m F0} e^{a_m x},
//   a_m = K2_m h ln 2,  e^{a x} = I0(a) + 2 sum_{n>=1} In(a) Tn(x)
// so M_k(x) = sum_n C_kn Tn(x), n <= 3, with C_kn summed over the steps once
// per piece and candidate.  Truncation ~ (a/2)^4/12 < 4e-8 for |a| <= 0.05,
// which holds when kappa(L) h <= 0.05; otherwise the per-step sum is used.
// ---------------------------------------------------------------------------
constexpr float kChebMaxA = 0.05f;

struct ChebTab {
    float c[kMaxCand][12];      // [candidate][k * 4 + n], k: g = 1, z, z^2 + dz^2/12
    float mid[kMaxCand];        // channel centre relative to the CUT
    float invh[kMaxCand];       // 1 / (B_c / 2)
    int ok;
};

// Called by every thread of the block after piece_consts; the caller syncs.
__device__ __forceinline__ void cheb_setup(const QuadParams &qp, const DevPiece &pc, int prof,
                                           const float4 *sT, int M, const PieceConst<float> &k, ChebTab &ct)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int coff = qp.plan_ch_off[pc.plan];
    const double kapL = qp.kap_L ? qp.kap_L[prof] : 1e30;
    double hmax = 0.0;
    for (int c = 0; c < k.nc; ++c) hmax = fmax(hmax, 0.5 * qp.ch_B[coff + pc.c_lo + c]);
    const bool ok = kapL * hmax <= (double)kChebMaxA;
    if (threadIdx.x == 0) ct.ok = ok ? 1 : 0;
    if (!ok) return;
    for (int c = warp; c < k.nc; c += nw) {
        const double F0 = qp.ch_frel[coff + pc.c_lo + c];
        const double h = 0.5 * qp.ch_B[coff + pc.c_lo + c];
        const double at = (double)(k.at_ab + k.hat[c]);
        for (int kk = 0; kk < 3; ++kk) {          // one moment at a time keeps registers low
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
            for (int m = lane; m < M; m += 32) {
                const float4 a = sT[m];
                const double g = kk == 0 ? 1.0 : (kk == 1 ? (double)a.z : (double)a.w);
                const double base = g * exp2((double)a.x - at * (double)a.z + (double)a.y * F0);
                const double t = 0.5 * (double)a.y * h * 0.69314718055994530942, t2 = t * t;
                s0 += base * (1.0 + t2 * (1.0 + t2 * (0.25 + t2 / 36.0)));                   // I0
                s1 += base * (2.0 * t * (1.0 + t2 * (0.5 + t2 / 12.0)));                     // 2 I1
                s2 += base * (2.0 * t2 * (0.5 + t2 * (1.0 / 6.0 + t2 / 48.0)));              // 2 I2
                s3 += base * (2.0 * t2 * t * (1.0 / 6.0 + t2 * (1.0 / 24.0 + t2 / 240.0)));  // 2 I3
            }
            s0 = warp_sum_d(s0);
            s1 = warp_sum_d(s1);
            s2 = warp_sum_d(s2);
            s3 = warp_sum_d(s3);
            if (lane == 0) {
                ct.c[c][kk * 4 + 0] = (float)s0;
                ct.c[c][kk * 4 + 1] = (float)s1;
                ct.c[c][kk * 4 + 2] = (float)s2;
                ct.c[c][kk * 4 + 3] = (float)s3;
            }
        }
        if (lane == 0) {
            ct.mid[c] = 0.5f * (k.lo[c] + k.hi[c]);
            ct.invh[c] = (float)(1.0 / h);
        }
    }
}

// Small-phase |S|^2 of a point in candidate ci from the contracted moments.
__device__ __forceinline__ void cheb_moments(const ChebTab &ct, int ci, float u, float &M0, float &M1, float &M2)
{
    const float x = (u - ct.mid[ci]) * ct.invh[ci];
    const float T2 = fmaf(2.0f * x, x, -1.0f);
    const float T3 = fmaf(2.0f * x, T2, -x);
    const float *c = ct.c[ci];
    M0 = fmaf(c[3], T3, fmaf(c[2], T2, fmaf(c[1], x, c[0])));
    M1 = fmaf(c[7], T3, fmaf(c[6], T2, fmaf(c[5], x, c[4])));
    M2 = fmaf(c[11], T3, fmaf(c[10], T2, fmaf(c[9], x, c[8])));
}

}  // namespace isrs
