// Half-warp walks of the FP32 adjoint kernels (closed-form profile): the
// z-sum of one grid point (App. A, Eq. slow_vary) spread over the 16 lanes of
// a half-warp, each lane owning K consecutive steps, with the terms kept in
// registers for the bucket terms d|S|^2/d ln p_m = 2 Re(conj(S) t_m).
#pragma once
#include <cuda_runtime.h>

#include "quad_common.cuh"
#include "quad_zsum.cuh"

namespace isrs {

constexpr unsigned kWarpAll = 0xffffffffu;

__device__ __forceinline__ float sinc_poly(float x)
{
    const float x2 = x * x;
    float sc = fmaf(x2, -2.5052108e-8f, 2.7557319e-6f);   // -1/11!, 1/9!
    sc = fmaf(x2, sc, -1.9841270e-4f);                     // -1/7!
    sc = fmaf(x2, sc, 8.3333333e-3f);                      // 1/5!
    sc = fmaf(x2, sc, -1.6666667e-1f);                     // -1/3!
    return fmaf(x2, sc, 1.0f);
}

// sum over the 16 lanes of each half-warp (both halves in step)
__device__ __forceinline__ float half_sum(float v)
{
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(kWarpAll, v, o, 16);
    return v;
}

// ---------------------------------------------------------------------------
// Half-warp walks of one grid point (state: weight w W af, phi, F_c - f_ref,
// at).  Lane l16 owns steps [K l16, K l16 + K) with tables
//   o0[k] = {A2 + log2 dz, K2, z, dz},  o1[k] = {edge/2pi hi, lo, A2, c}
// (padding steps carry log2 weight -1000, so their terms vanish), and for
// the first F_c candidates of the piece oc[k] = {edge/2pi hi, lo,
// A2 - at_c z, K2}.  Each walk
// adds the lane's bucket terms and returns the point's w W af |S|^2.
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ float walk_direct(const float4 *o0s, float wq, float ph, float fc, float at, float mult,
                                             float (&R)[K], float (&Rp)[K])
{
    // S = sum_m p_m dz_m sinc(phi dz_m/2) e^{j phi z_m}; d|S|^2/d ln p_m = 2 Re(conj(S) t_m)
    const float hph = 0.5f * ph;
    const float phr = ph * 0.15915494309189535f;
    float tr[K], ti[K];
    float sr = 0.0f, si = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float4 o = o0s[k * 16];
        float sn, cs;
        sincos_rev<true>(phr * o.z, sn, cs);
        float lp = fmaf(o.y, fc, o.x);
        lp = fmaf(-at, o.z, lp);
        const float amp = ex2_approx(lp) * sinc_poly(hph * o.w);
        tr[k] = amp * cs;
        ti[k] = amp * sn;
        sr += tr[k];
        si += ti[k];
    }
    sr = half_sum(sr);
    si = half_sum(si);
    const float c2 = 2.0f * mult * wq, c2F = c2 * fc;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float rr = fmaf(sr, tr[k], si * ti[k]);
        R[k] = fmaf(c2, rr, R[k]);
        Rp[k] = fmaf(c2F, rr, Rp[k]);
    }
    return wq * fmaf(sr, sr, si * si);
}

// Folded: o1s holds the point's candidate rows {edge/2pi hi, lo, A2 - at z, K2}
// (attenuation folded in), so a step takes one table load and one FMA for
// ln p; o0s and at are then unused.
template <int K, bool Wide = false, bool Folded = false>
__device__ __forceinline__ float walk_tele(const float4 *o0s, const float4 *o1s, int l16, float wq, float ph,
                                           float fc, float at, float mult, float (&R)[K], float (&Rp)[K])
{
    // U = sum_m p_m (E_{m+1} - E_m), E_e = e^{j phi z_e}, |S|^2 = |U|^2/phi^2;
    // d|S|^2/d ln p_m = 2 Re(conj(U) p_m (E_{m+1} - E_m)) / phi^2
    float tr[K], ti[K];
    float Er = 1.0f, Ei = 0.0f, p0 = 0.0f, e1r = 1.0f, e1i = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float4 b = o1s[k * 16];
        float sn, cs;
        if (Wide) phasor_rev_ff_wide<true>(ph, b.x, b.y, sn, cs);
        else phasor_rev_ff<true>(ph, b.x, b.y, sn, cs);
        float lp;
        if constexpr (Folded) {
            lp = fmaf(b.w, fc, b.z);
        } else {
            const float4 a = o0s[k * 16];
            lp = fmaf(a.y, fc, b.z);
            lp = fmaf(-at, a.z, lp);
        }
        const float pm = ex2_approx(lp);
        if (k == 0) {
            p0 = pm;
            e1r = cs;
            e1i = sn;
            tr[0] = 0.0f;
            ti[0] = 0.0f;
        } else {
            tr[k] = pm * (cs - Er);
            ti[k] = pm * (sn - Ei);
        }
        Er = cs;
        Ei = sn;
    }
    // the lower edge of this lane's first step is the previous lane's last edge
    float elr = __shfl_up_sync(kWarpAll, Er, 1, 16);
    float eli = __shfl_up_sync(kWarpAll, Ei, 1, 16);
    elr = l16 == 0 ? 1.0f : elr;
    eli = l16 == 0 ? 0.0f : eli;
    tr[0] = p0 * (e1r - elr);
    ti[0] = p0 * (e1i - eli);
    float ur = 0.0f, ui = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        ur += tr[k];
        ui += ti[k];
    }
    ur = half_sum(ur);
    ui = half_sum(ui);
    const float iph2 = __fdividef(1.0f, ph * ph);   // MUFU reciprocal (2 ulp): phi^2 is far from the range limits
    const float c2 = 2.0f * mult * wq * iph2, c2F = c2 * fc;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float rr = fmaf(ur, tr[k], ui * ti[k]);
        R[k] = fmaf(c2, rr, R[k]);
        Rp[k] = fmaf(c2F, rr, Rp[k]);
    }
    return wq * fmaf(ur, ur, ui * ui) * iph2;
}

template <int K>
__device__ __forceinline__ float walk_small(const float4 *o0s, const float4 *o1s, float wq, float ph, float fc,
                                            float at, float mult, float (&R)[K], float (&Rp)[K])
{
    // |S|^2 = M0^2 - phi^2 (M0 M2 - M1^2);
    // d|S|^2/d ln p_m = w_m (2 M0 - phi^2 (M2 + M0 c_m - 2 M1 z_m))
    float wk[K];
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float4 a = o0s[k * 16];
        const float cm = o1s[k * 16].w;
        float lp = fmaf(a.y, fc, a.x);
        lp = fmaf(-at, a.z, lp);
        wk[k] = ex2_approx(lp);
        s0 += wk[k];
        s1 = fmaf(wk[k], a.z, s1);
        s2 = fmaf(wk[k], cm, s2);
    }
    s0 = half_sum(s0);
    s1 = half_sum(s1);
    s2 = half_sum(s2);
    const float ph2 = ph * ph;
    const float al0 = 2.0f * s0 - ph2 * s2, al1 = -ph2 * s0, al2 = 2.0f * ph2 * s1;
    const float cp = mult * wq, cF = cp * fc;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float zm = o0s[k * 16].z;
        const float cm = o1s[k * 16].w;
        const float rr = wk[k] * fmaf(al2, zm, fmaf(al1, cm, al0));
        R[k] = fmaf(cp, rr, R[k]);
        Rp[k] = fmaf(cF, rr, Rp[k]);
    }
    return wq * fmaf(-ph2, fmaf(s0, s2, -s1 * s1), s0 * s0);
}

}  // namespace isrs
