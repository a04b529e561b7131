// FP32 z-sums of the closed-form profile, shared by the quadrature kernels.
#pragma once
#include <cuda_runtime.h>

#include "quad_common.cuh"

namespace isrs {

// ---------------------------------------------------------------------------
// FP32 z-sums.  Per-step tables staged in shared memory:
//   sT[m] = {A2_m + log2 dz_m, K2_m, z_m, c_m = z_m^2 + dz_m^2/12}
//   sR[m] = {A2_m + log2 dz_m, K2_m, z_m, dz_m}
//   sE[m] = {z_{m+1}/2pi hi, lo (float-float), A2_m, K2_m}
// with log2 p_m = A2_m + K2_m Fc - at z_m (Eq. pk for the closed-form
// profile).  The phase is carried in revolutions (z / 2pi).
//
// Exact-to-FP32 evaluations of S = sum_m p_m dz_m sinc(phi dz_m/2)
// e^{j phi z_m} (Eq. slow_vary), chosen per grid point by |phi|:
//  * contracted small phase (|phi| L <= 6, when the piece's Chebyshev
//    contraction applies): the centred series about the span centre with
//    6, 11 or 19 moments by phase (quad_common.cuh), no per-step work;
//  * small (|phi| L <= 0.02, otherwise): second-order expansion in phi,
//      |S|^2 = M0^2 - phi^2 (M0 M2 - M1^2) + O((phi L)^4),
//    M0 = sum p dz, M1 = sum p dz z, M2 = sum p dz (z^2 + dz^2/12); the
//    truncation is below 1e-9 relative (one exp per step, no phasor).
//  * direct (|phi| dz_max <= pi): the formula as written, sinc by its even
//    Taylor polynomial in x = phi dz/2 (|x| <= pi/2, truncation < 4e-8),
//    phase phi z/2pi < L/(2 dz_max) revolutions formed in FP32.
//  * telescoped (otherwise): dz sinc(phi dz/2) e^{j phi z_m} equals
//    (E_{m+1} - E_m)/(j phi) with E_e = e^{j phi z_e}, so one complex
//    exponential per edge suffices; the phase phi z_e / 2pi (up to ~1e5
//    revolutions) is an error-free float-float product reduced to [-1/2, 1/2].
// The final division by phi^2 takes the MUFU reciprocal (2 ulp; phi^2 lies
// far inside the range where it is accurate): an IEEE division there costs
// a branch to its slow path at every point.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float zsum_small_f(float phi, float Fc, float at, const float4 *sT, int M)
{
    float M0 = 0.0f, M1 = 0.0f, M2 = 0.0f;
#pragma unroll 4
    for (int m = 0; m < M; ++m) {
        const float4 a = sT[m];
        float lp = fmaf(a.y, Fc, a.x);
        lp = fmaf(-at, a.z, lp);
        const float w = ex2_approx(lp);          // p_m dz_m
        M0 += w;
        M1 = fmaf(w, a.z, M1);
        M2 = fmaf(w, a.w, M2);
    }
    return fmaf(-phi * phi, fmaf(M0, M2, -M1 * M1), M0 * M0);
}

__device__ __forceinline__ float zsum_direct_f(float phi, float Fc, float at, const float4 *sR, int M)
{
    // sR[m] = {A2_m + log2 dz_m, K2_m, z_m, dz_m}; phase in revolutions phi/2pi * z_m
    float Sr = 0.0f, Si = 0.0f;
    const float hphi = 0.5f * phi;
    const float phir = phi * 0.15915494309189535f;
#pragma unroll 4
    for (int m = 0; m < M; ++m) {
        const float4 a = sR[m];
        float sn, cs;
        sincos_rev(phir * a.z, sn, cs);
        const float x = hphi * a.w;
        const float x2 = x * x;
        float sc = fmaf(x2, -2.5052108e-8f, 2.7557319e-6f);   // -1/11!, 1/9!
        sc = fmaf(x2, sc, -1.9841270e-4f);                     // -1/7!
        sc = fmaf(x2, sc, 8.3333333e-3f);                      // 1/5!
        sc = fmaf(x2, sc, -1.6666667e-1f);                     // -1/3!
        sc = fmaf(x2, sc, 1.0f);
        float lp = fmaf(a.y, Fc, a.x);
        lp = fmaf(-at, a.z, lp);
        const float amp = ex2_approx(lp) * sc;   // p_m dz_m sinc
        Sr = fmaf(amp, cs, Sr);
        Si = fmaf(amp, sn, Si);
    }
    return Sr * Sr + Si * Si;
}

__device__ __forceinline__ float zsum_tele_f(float phi, float Fc, float at, const float4 *sT,
                                             const float4 *sE, int M)
{
    float Er = 1.0f, Ei = 0.0f, Sr = 0.0f, Si = 0.0f;
#pragma unroll 4
    for (int m = 0; m < M; ++m) {
        const float4 e = sE[m];
        const float zm = sT[m].z;
        float sn, cs;
        phasor_rev_ff(phi, e.x, e.y, sn, cs);
        float lp = fmaf(e.w, Fc, e.z);
        lp = fmaf(-at, zm, lp);
        const float p = ex2_approx(lp);
        Sr = fmaf(p, cs - Er, Sr);
        Si = fmaf(p, sn - Ei, Si);
        Er = cs;
        Ei = sn;
    }
    return __fdividef(Sr * Sr + Si * Si, phi * phi);
}

// The same two forms with the candidate's attenuation folded into the step
// tables (rows of a per-candidate copy):
//   sRc[m] = {A2_m + log2 dz_m - at z_m, K2_m, z_m, dz_m},
//   sEc[m] = {z_{m+1}/2pi hi, lo, A2_m - at z_m, K2_m},
// so log2 p_m = row + K2_m Fc in one FMA and the telescoped form needs no z.
__device__ __forceinline__ float zsum_direct_fc(float phi, float Fc, const float4 *sRc, int M)
{
    float Sr = 0.0f, Si = 0.0f;
    const float hphi = 0.5f * phi;
    const float phir = phi * 0.15915494309189535f;
#pragma unroll 4
    for (int m = 0; m < M; ++m) {
        const float4 a = sRc[m];
        float sn, cs;
        sincos_rev(phir * a.z, sn, cs);
        const float x = hphi * a.w;
        const float x2 = x * x;
        float sc = fmaf(x2, -2.5052108e-8f, 2.7557319e-6f);   // -1/11!, 1/9!
        sc = fmaf(x2, sc, -1.9841270e-4f);                     // -1/7!
        sc = fmaf(x2, sc, 8.3333333e-3f);                      // 1/5!
        sc = fmaf(x2, sc, -1.6666667e-1f);                     // -1/3!
        sc = fmaf(x2, sc, 1.0f);
        const float amp = ex2_approx(fmaf(a.y, Fc, a.x)) * sc;
        Sr = fmaf(amp, cs, Sr);
        Si = fmaf(amp, sn, Si);
    }
    return Sr * Sr + Si * Si;
}

__device__ __forceinline__ float zsum_tele_fc(float phi, float Fc, const float4 *sEc, int M)
{
    float Er = 1.0f, Ei = 0.0f, Sr = 0.0f, Si = 0.0f;
#pragma unroll 4
    for (int m = 0; m < M; ++m) {
        const float4 e = sEc[m];
        float sn, cs;
        phasor_rev_ff(phi, e.x, e.y, sn, cs);
        const float p = ex2_approx(fmaf(e.w, Fc, e.z));
        Sr = fmaf(p, cs - Er, Sr);
        Si = fmaf(p, sn - Ei, Si);
        Er = cs;
        Ei = sn;
    }
    return __fdividef(Sr * Sr + Si * Si, phi * phi);
}

// As phasor_rev_ff, for phases far beyond 2^22 revolutions (the MCI cells):
// once |phi z / 2pi| >= 2^22 the first magic-number rounding leaves an
// integer (or half-integer) on top of the fraction, and FRND's exact
// th - rint(th) can leave tl beyond one revolution; a second rounding of the
// sum removes either.
template <bool Xu = false>
__device__ __forceinline__ void phasor_rev_ff_wide(float phi, float hi, float lo, float &sn, float &cs)
{
    const float th = phi * hi;
    float tl = fmaf(phi, hi, -th);
    tl = fmaf(phi, lo, tl);
    float fr = __fadd_rn(th, -(Xu ? round_nearest(th) : round_magic(th))) + tl;
    fr = __fadd_rn(fr, -(Xu ? round_nearest(fr) : round_magic(fr)));
    __sincosf(fr * 6.283185307179586f, &sn, &cs);
}

__device__ __forceinline__ float zsum_tele_wide_f(float phi, float Fc, float at, const float4 *sT,
                                                  const float4 *sE, int M)
{
    float Er = 1.0f, Ei = 0.0f, Sr = 0.0f, Si = 0.0f;
#pragma unroll 4
    for (int m = 0; m < M; ++m) {
        const float4 e = sE[m];
        const float zm = sT[m].z;
        float sn, cs;
        phasor_rev_ff_wide(phi, e.x, e.y, sn, cs);
        float lp = fmaf(e.w, Fc, e.z);
        lp = fmaf(-at, zm, lp);
        const float p = ex2_approx(lp);
        Sr = fmaf(p, cs - Er, Sr);
        Si = fmaf(p, sn - Ei, Si);
        Er = cs;
        Ei = sn;
    }
    return __fdividef(Sr * Sr + Si * Si, phi * phi);
}

}  // namespace isrs
