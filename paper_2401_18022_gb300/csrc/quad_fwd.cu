// Forward kernels of the ISRS GN integral model (arXiv 2401.18022, App. A).
//
//  k_prep        per profile and z-step (FP64): P_tot, the ISRS
//                normalisation ln N(z_m) by log-sum-exp over channels, and the
//                per-step power tables of Eq. pk for the linear-slope
//                closed-form profile.
//  k_quad_f32    persistent quadrature: one block per work tile (a range of
//                pieces of one CUT); G x G hyperbolic grid per piece
//                (Eqs. q1..q4), z-sum of Eq. slow_vary per grid point in FP32:
//                the moment series about the span centre (|phi| L <= 6) or
//                about the centres of 2, 4 or 8 segments (|phi| L up to ~42),
//                else the direct or telescoped step sums with a float-float
//                phase and mod-2pi reduction; compensated accumulation; one
//                FP64 partial per tile.
//  k_quad_f64    the same quadrature in plain FP64 (direct form of
//                Eq. slow_vary with sinc), used as the reference GPU path.
//  k_finish      per profile: deterministic FP64 sum of tile partials per CUT,
//                eta (Eq. gain_fin), P_NLI, SNR and throughput (Eq. loss).
#include <cuda_runtime.h>

#include "isrs_internal.cuh"
#include "isrs_kernels.h"
#include "quad_common.cuh"
#include "quad_zsum.cuh"

namespace isrs {

// ---------------------------------------------------------------------------
// k_prep: ISRS profile tables (FP64).  One block per (profile, z-step), the
// last step index standing for z = L:
//   rho(z,F) = e^{-alpha_c z} P_tot e^{-kappa(z)(F - f_ref)} / N(z)
//   kappa(z) = P_tot C_r L_eff(z),  N(z) = sum_k P_k e^{-kappa f_k'} sinhc(kappa B_k/2)
// so ln p_m (Eq. pk) = lnPtot - lnN_m - kappa_m (F_c - f_ref) - at z_m with
// at = (alpha_a + alpha_b + alpha_c - alpha_i)/2, because F_a + F_b + F_c - f
// = 2 F_c.  Writes, per step, {A2, K2} = log2(e) {lnPtot - lnN, -kappa} and
// {lnPtot - lnN, kappa}; per channel P/B (step 0's block) and ln rho(L, f_c)
// (the z = L block).  ln N is a log-sum-exp over the channels with a block
// maximum and a block sum in fixed order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double sinhc_d(double x)
{
    return fabs(x) < 1e-4 ? 1.0 + x * x / 6.0 : sinh(x) / x;
}

__global__ void __launch_bounds__(256) k_prep(PrepParams pp)
{
    __shared__ double scratch[32];
    const int p = blockIdx.x, m = blockIdx.y;
    const int plan = pp.prof_plan[p];
    const int n = pp.plan_n[plan];
    const int coff = pp.plan_ch_off[plan];
    const int poff = pp.prof_ch_off[p];
    const double *P = pp.P + poff;
    const double *fr = pp.ch_frel + coff;
    const double *B = pp.ch_B + coff;
    const int M = pp.n_steps;

    double part = 0.0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) part += P[c];
    const double Ptot = block_sum_d(part, scratch);
    const double lnPtot = log(Ptot);
    if (m == 0) {
        for (int c = threadIdx.x; c < n; c += blockDim.x) {
            double pd = P[c] / B[c];
            pp.pd_d[poff + c] = pd;
            pp.pd_f[poff + c] = (float)pd;
        }
    }
    const double z = (m < M) ? pp.zs_d[m].x : pp.L;
    const double leff = pp.alpha_R > 0.0 ? -expm1(-pp.alpha_R * z) / pp.alpha_R : z;
    const double kap = Ptot * pp.Cr * leff;
    double mx = -1e300;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        if (P[c] > 0.0) mx = fmax(mx, log(P[c]) - kap * fr[c] + log(sinhc_d(0.5 * kap * B[c])));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = -1e300;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, scratch[w]);
    double sum = 0.0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        if (P[c] > 0.0) sum += exp(log(P[c]) - kap * fr[c] + log(sinhc_d(0.5 * kap * B[c])) - mx);
    }
    sum = block_sum_d(sum, scratch);
    const double lnN = mx + log(sum);
    if (m < M) {
        if (threadIdx.x == 0) {
            pp.step_d[(size_t)p * M + m] = make_double2(lnPtot - lnN, kap);
            pp.step_f[(size_t)p * M + m] = make_float2((float)((lnPtot - lnN) * kLog2e), (float)(-kap * kLog2e));
        }
        return;
    }
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        pp.lnrho_L[poff + c] = -pp.ch_alpha[coff + c] * pp.L + lnPtot - lnN - kap * fr[c];
    }
    if (threadIdx.x == 0) {
        pp.ptot[p] = Ptot;
        if (pp.kap_L) pp.kap_L[p] = kap;
    }
}

// ---------------------------------------------------------------------------
// k_quad_f32: persistent FP32 quadrature.
// ---------------------------------------------------------------------------
constexpr int kFwdCand = 4;          // F_c candidates with their own step rows (attenuation folded in) ...
constexpr int kFwdCandSteps = 256;   // ... when the z-grid has at most this many steps (shared memory)

__host__ __device__ constexpr int fwd_cand_rows(int n_steps)
{
    return n_steps <= kFwdCandSteps ? kFwdCand : 0;
}

// Dynamic shared memory of k_quad_f32 in float4 units: the step tables, the
// per-candidate rows, the G row descriptors, then (G >= kSegMinG) the
// segment tables.
__host__ __device__ constexpr size_t fwd_seg_offset_f4(int n_steps, int G)
{
    return (size_t)n_steps * (3 + 2 * fwd_cand_rows(n_steps)) +
           ((size_t)G * sizeof(RowF) + sizeof(float4) - 1) / sizeof(float4);
}
#ifndef ISRS_FWD_MIN_BLOCKS
#define ISRS_FWD_MIN_BLOCKS 4   // resident blocks per SM the register budget is sized for
#endif

__global__ void __launch_bounds__(256, ISRS_FWD_MIN_BLOCKS) k_quad_f32(QuadParams qp)
{
    extern __shared__ float4 smem_f4[];
    const int M = qp.n_steps, G = qp.G;
    float4 *sT = smem_f4;                              // [M] {A2 + log2 dz, K2, z, z^2 + dz^2/12}
    float4 *sE = sT + M;                               // [M] {edge/2pi hi, lo, A2, K2}
    float4 *sR = sE + M;                               // [M] {A2 + log2 dz, K2, z, dz}
    const int ncr = fwd_cand_rows(M);
    float4 *sRc = sR + M;                              // [ncr][M] sR rows with - at_c z folded in
    float4 *sEc = sRc + ncr * M;                       // [ncr][M] sE rows with - at_c z folded in
    RowF *rows = reinterpret_cast<RowF *>(sEc + ncr * M);   // [G]
    // segment tables (G >= kSegMinG only; the launch sizes the space for them)
    SegTab *sg = reinterpret_cast<SegTab *>(smem_f4 + fwd_seg_offset_f4(M, G));
    __shared__ PieceConst<float> kc;
    __shared__ ChebTab ct;
    __shared__ double scratch[32];
    __shared__ int s_item;

    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const float4 za = qp.zs_a[m];   // {z_m, c_m, log2 dz_m, dz_m}
        const float4 zb = qp.zs_b[m];   // {edge(m+1)/2pi hi, lo, z_m/2pi, 0}
        sT[m] = make_float4(0.0f, 0.0f, za.x, za.y);
        sE[m] = make_float4(zb.x, zb.y, 0.0f, 0.0f);
        sR[m] = make_float4(0.0f, 0.0f, za.x, za.w);
    }
    const float c3 = (float)(kPi * qp.beta3);
    const float c4 = (float)(2.0 * kPi * kPi / 3.0 * qp.beta4);
    const float b2 = (float)qp.beta2;
    const float m4pi2 = (float)(-4.0 * kPi * kPi);
    const float phi_direct = 3.14159265f / qp.dz_max;
    const float phi_small = 0.02f / qp.L;
    const float phi_cheb = kChebPhiL / qp.L;
    const float phi_c6 = kChebPhiL6 / qp.L, phi_c11 = kChebPhiL11 / qp.L;
    const float phi_s0 = qp.phi_seg[0], phi_s1 = qp.phi_seg[1], phi_s2 = qp.phi_seg[2];
    const float log2e = (float)kLog2e;
    const float invG = 1.0f / (float)G;
    unsigned n_small = 0, n_direct = 0, n_tele = 0;
    int cur_prof = -1;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(qp.counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= qp.n_items) break;
        const DevItem item = qp.items[it];
        if (item.prof != cur_prof) {
            const float2 *st = qp.step_f + (size_t)item.prof * M;
            for (int m = threadIdx.x; m < M; m += blockDim.x) {
                const float2 v = st[m];
                const float a2d = v.x + qp.zs_a[m].z;
                sT[m].x = a2d;
                sT[m].y = v.y;
                sE[m].z = v.x;
                sE[m].w = v.y;
                sR[m].x = a2d;
                sR[m].y = v.y;
            }
            cur_prof = item.prof;
        }
        double acc = 0.0;
        for (int k = item.piece0; k < item.piece1; ++k) {
            const DevPiece pc = qp.pieces[dbg_clamp(k, qp.n_pieces, kDbgPiece, qp.dbg)];
            piece_rows<RowF>(pc, G, qp.eps_v1, rows);
            piece_consts<float>(qp, pc, item.prof, log2e, qp.pd_f, kc);
            __syncthreads();
            // step weights of the contracted candidates, once per piece, in the
            // space of the per-candidate rows (filled after the tables)
            int nW = 0;
            if (ncr > 0 && cheb_applies(qp, pc, item.prof, kc)) {
                nW = min(kc.nc, 2 * ncr);
                cheb_weights(qp, pc, sT, M, kc, nW, sRc);
                __syncthreads();
            }
            const bool segs = cheb_setup<kChebMom>(qp, pc, item.prof, sT, M, kc, ct, sRc, nW) &&
                              qp.zs_gseg != nullptr && G >= kSegMinG;
            if (segs) seg_setup(qp, pc, sT, M, kc, *sg, sRc, nW);
            if (nW > 0) __syncthreads();
            // per-candidate step rows with the candidate's attenuation folded in
            const int ncf = min(kc.nc, ncr);
            for (int t = threadIdx.x; t < ncf * M; t += blockDim.x) {
                const int c = t / M, m = t - c * M;
                const float at = kc.at_ab + kc.hat[c];
                const float4 r = sR[m], e = sE[m];
                sRc[t] = make_float4(fmaf(-at, r.z, r.x), r.y, r.z, r.w);
                sEc[t] = make_float4(e.x, e.y, fmaf(-at, r.z, e.z), e.w);
            }
            __syncthreads();
            const float fi = kc.fi, s1g = kc.s1, s2g = kc.s2;
            const float three_fi2 = 3.0f * fi * fi;
            const bool cheb = ct.ok != 0;
            const float phi_lim = cheb ? phi_cheb : phi_small;   // upper |phi| of the small-phase forms
            float sum = 0.0f, comp = 0.0f;
            const int npts = G * G;
            for (int q = threadIdx.x; q < npts; q += blockDim.x) {
                // row r = floor(q / G): (q + 1/2)/G is at least 1/(2G) from an integer
                const int r = (int)(((float)q + 0.5f) * invG);
                const int j = q - r * G;
                const RowF rw = rows[dbg_clamp(r, G, kDbgRow, qp.dbg)];
                if (rw.w == 0.0f) continue;
                const float d = ((float)j + 0.5f - 0.5f * (float)G) * rw.du2;
                const float e = expf(d);
                const float f1 = s1g * (rw.xc * e);
                const float f2 = s2g * (rw.yc * __frcp_rn(e));
                const float u = f1 + f2;                    // F_c - f_i
                int ci = -1;
                for (int c = 0; c < kc.nc; ++c) {
                    if (u >= kc.lo[c] && u < kc.hi[c]) { ci = c; break; }
                }
                if (ci < 0) continue;                       // F_c in a gap
                ci = dbg_clamp(ci, kc.nc, kDbgCand, qp.dbg);
                const float W = kc.wab * kc.pd[ci];
                const float at = kc.at_ab + kc.hat[ci];
                const float Fc = fi + u;                    // F_c - f_ref
                // Eq. phi
                const float br = b2 + c3 * (u + 2.0f * fi) +
                                 c4 * (f1 * f1 + 1.5f * f1 * f2 + 3.0f * fi * u + f2 * f2 + three_fi2);
                const float phi = m4pi2 * f1 * f2 * br;
                const float aphi = fabsf(phi);
                float S2;
                if (aphi <= phi_lim) {
                    if (cheb) {
                        float x, A, B;
                        cheb_point(ct, ci, u, phi, aphi, phi_c6, phi_c11, x, A, B);
                        S2 = fmaf(A, A, B * B);
                    } else {
                        S2 = zsum_small_f(phi, Fc, at, sT, M);
                    }
                    ++n_small;
                } else if (segs && ci < kSegCand && aphi <= phi_s2) {
                    // the series per segment: 2, 4 or 8 segments by |phi|
                    const int s0 = aphi <= phi_s0 ? 0 : (aphi <= phi_s1 ? 2 : 6);
                    const int s1 = aphi <= phi_s0 ? 2 : (aphi <= phi_s1 ? 6 : kSegSlots);
                    const float x = (u - ct.mid[ci]) * ct.invh[ci];
                    const float T2 = fmaf(2.0f * x, x, -1.0f);
                    const float T3 = fmaf(2.0f * x, T2, -x);
                    S2 = seg_s2(*sg, ci, s0, s1, x, T2, T3, phi);
                    ++n_small;
                } else if (aphi <= phi_direct) {
                    S2 = ci < ncr ? zsum_direct_fc(phi, Fc, sRc + ci * M, M) : zsum_direct_f(phi, Fc, at, sR, M);
                    ++n_direct;
                } else {
                    S2 = ci < ncr ? zsum_tele_fc(phi, Fc, sEc + ci * M, M) : zsum_tele_f(phi, Fc, at, sT, sE, M);
                    ++n_tele;
                }
                // compensated accumulation over this thread's points
                const float y = rw.w * W * S2 * array_factor_f(phi, qp) - comp;
                const float t = sum + y;
                comp = (t - sum) - y;
                sum = t;
            }
            acc += (double)kc.mult * ((double)sum - (double)comp);
            __syncthreads();
        }
        const double tot = block_sum_d(acc, scratch);
        if (threadIdx.x == 0) qp.partial[it] = tot;
    }
    if (qp.path_count) {
        unsigned long long c0 = n_small, c1 = n_direct, c2 = n_tele;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c0 += __shfl_xor_sync(0xffffffffu, c0, o);
            c1 += __shfl_xor_sync(0xffffffffu, c1, o);
            c2 += __shfl_xor_sync(0xffffffffu, c2, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&qp.path_count[0], c0);
            atomicAdd(&qp.path_count[1], c1);
            atomicAdd(&qp.path_count[2], c2);
        }
    }
}

// ---------------------------------------------------------------------------
// k_quad_f64: the same quadrature in plain FP64 (direct form, libm functions).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_quad_f64(QuadParams qp)
{
    extern __shared__ double2 smem_d2[];
    const int M = qp.n_steps, G = qp.G;
    double2 *sz = smem_d2;                 // [M] {z_m, dz_m}
    double2 *st = sz + M;                  // [M] {lnPtot - lnN, kappa}
    RowD *rows = reinterpret_cast<RowD *>(st + M);
    __shared__ PieceConst<double> kc;
    __shared__ double scratch[32];
    __shared__ int s_item;

    for (int m = threadIdx.x; m < M; m += blockDim.x) sz[m] = qp.zs_d[m];
    const double c3 = kPi * qp.beta3;
    const double c4 = 2.0 * kPi * kPi / 3.0 * qp.beta4;
    int cur_prof = -1;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(qp.counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= qp.n_items) break;
        const DevItem item = qp.items[it];
        if (item.prof != cur_prof) {
            for (int m = threadIdx.x; m < M; m += blockDim.x) st[m] = qp.step_d[(size_t)item.prof * M + m];
            cur_prof = item.prof;
        }
        double acc = 0.0;
        for (int k = item.piece0; k < item.piece1; ++k) {
            const DevPiece pc = qp.pieces[dbg_clamp(k, qp.n_pieces, kDbgPiece, qp.dbg)];
            piece_rows<RowD>(pc, G, qp.eps_v1, rows);
            piece_consts<double>(qp, pc, item.prof, 1.0, qp.pd_d, kc);
            __syncthreads();
            const double fi = kc.fi;
            double sum = 0.0;
            const int npts = G * G;
            for (int q = threadIdx.x; q < npts; q += blockDim.x) {
                const int r = q / G;
                const int j = q - r * G;
                const RowD rw = rows[dbg_clamp(r, G, kDbgRow, qp.dbg)];
                if (rw.w == 0.0) continue;
                const double d = ((double)j + 0.5 - 0.5 * (double)G) * rw.du2;
                const double f1 = kc.s1 * (rw.xc * exp(d));
                const double f2 = kc.s2 * (rw.yc * exp(-d));
                const double u = f1 + f2;
                int ci = -1;
                for (int c = 0; c < kc.nc; ++c) {
                    if (u >= kc.lo[c] && u < kc.hi[c]) { ci = c; break; }
                }
                if (ci < 0) continue;
                const double W = kc.wab * kc.pd[ci];
                const double at = kc.at_ab + kc.hat[ci];
                const double Fc = fi + u;
                const double br = qp.beta2 + c3 * (u + 2.0 * fi) +
                                  c4 * (f1 * f1 + 1.5 * f1 * f2 + 3.0 * fi * u + f2 * f2 + 3.0 * fi * fi);
                const double phi = -4.0 * kPi * kPi * f1 * f2 * br;
                double Sr = 0.0, Si = 0.0;
                for (int m = 0; m < M; ++m) {
                    const double2 zz = sz[m];
                    const double2 tt = st[m];
                    const double p = exp(tt.x - tt.y * Fc - at * zz.x);
                    const double amp = p * zz.y * sinc_d(0.5 * phi * zz.y);
                    double sn, cs;
                    sincos(phi * zz.x, &sn, &cs);
                    Sr += amp * cs;
                    Si += amp * sn;
                }
                sum += rw.w * W * (Sr * Sr + Si * Si) * array_factor_d(phi, qp);
            }
            acc += kc.mult * sum;
            __syncthreads();
        }
        const double tot = block_sum_d(acc, scratch);
        if (threadIdx.x == 0) qp.partial[it] = tot;
    }
}

// ---------------------------------------------------------------------------
// k_finish: per profile, Sigma_i = ordered sum of the CUT's tile partials;
// eta_i = (16/27) gamma_i^2 B_i Sigma_i / P_i^3 (Eq. gain_fin, P_NLI = G B);
// SNR_i = P_i / (P_NLI,i + P_ASE,i) with P_ASE,i = NF h f (1/rho(L,f) - 1) B
// and optional transceiver noise; T = 2 sum B log2(1 + SNR) (Eq. loss).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_finish(FinishParams fp)
{
    __shared__ double scratch[32];
    const int p = blockIdx.x;
    const int plan = fp.prof_plan[p];
    const int coff = fp.plan_ch_off[plan];
    const int poff = fp.prof_ch_off[p];
    const int s0 = fp.prof_slot_off[p], s1 = fp.prof_slot_off[p + 1];
    double tpart = 0.0;
    for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
        const int2 rg = fp.slot_items[s];
        const int i = fp.slot_cut[s];
        double sig = 0.0;
        for (int it = rg.x; it < rg.y; ++it) sig += fp.partial[it];
        if (fp.slot_items2) {
            const int2 r2 = fp.slot_items2[s];
            for (int it = r2.x; it < r2.y; ++it) sig += fp.partial2[it];
        }
        const double g = fp.ch_gamma[coff + i];
        const double B = fp.ch_B[coff + i];
        const double P = fp.P[poff + i];
        const double pnli = 16.0 / 27.0 * g * g * B * sig;
        const double eta = P > 0.0 ? pnli / (P * P * P) : __longlong_as_double(0x7ff8000000000000LL);
        if (fp.sigma) fp.sigma[s] = sig;
        if (fp.pnli) fp.pnli[s] = pnli;
        if (fp.eta) fp.eta[s] = eta;
        if (fp.snr) {
            const double nf = fp.ch_nf ? pow(10.0, fp.ch_nf[coff + i] / 10.0) : 1.0;
            const double f_abs = fp.ch_frel[coff + i] + fp.f_ref;
            const double gain = exp(-fp.lnrho_L[poff + i]);
            const double pase = fp.n_spans * nf * 6.62607015e-34 * (f_abs * 1e12) * (gain - 1.0) * (B * 1e12);
            const bool off = !(P > 0.0) || (fp.guard && fp.guard[coff + i]);
            double snr = 0.0;
            if (!off) {
                snr = P / (pnli + pase);
                if (fp.snr_trx_lin_inv > 0.0) snr = 1.0 / (1.0 / snr + fp.snr_trx_lin_inv);
                tpart += 2.0 * B * log2(1.0 + snr);
            }
            fp.snr[s] = snr;
            if (fp.pase) fp.pase[s] = pase;
        }
    }
    const double T = block_sum_d(tpart, scratch);
    if (threadIdx.x == 0 && fp.T) fp.T[p] = T;
}

// ---------------------------------------------------------------------------
// k_snr_from_eta: the Eq. loss part of k_finish for every channel, from a
// given eta (gathered from the shards of a split gradient): P_NLI = eta P^3,
// P_ASE, SNR and T.  One block.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_snr_from_eta(SnrFromEtaParams sp)
{
    __shared__ double scratch[32];
    double tpart = 0.0;
    for (int i = threadIdx.x; i < sp.n; i += blockDim.x) {
        const double B = sp.ch_B[i], P = sp.P[i];
        const double pnli = sp.eta[i] * P * P * P;
        const double nf = sp.ch_nf ? pow(10.0, sp.ch_nf[i] / 10.0) : 1.0;
        const double f_abs = sp.ch_frel[i] + sp.f_ref;
        const double gain = exp(-sp.lnrho_L[i]);
        const double pase = sp.n_spans * nf * 6.62607015e-34 * (f_abs * 1e12) * (gain - 1.0) * (B * 1e12);
        const bool off = !(P > 0.0) || (sp.guard && sp.guard[i]);
        double snr = 0.0;
        if (!off) {
            snr = P / (pnli + pase);
            if (sp.snr_trx_lin_inv > 0.0) snr = 1.0 / (1.0 / snr + sp.snr_trx_lin_inv);
            tpart += 2.0 * B * log2(1.0 + snr);
        }
        sp.snr[i] = snr;
        sp.pnli[i] = pnli;
        sp.pase[i] = pase;
    }
    const double T = block_sum_d(tpart, scratch);
    if (threadIdx.x == 0 && sp.T) sp.T[0] = T;
}

cudaError_t launch_snr_from_eta(const SnrFromEtaParams &sp, cudaStream_t st)
{
    k_snr_from_eta<<<1, 256, 0, st>>>(sp);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
size_t quad_smem_bytes(int precision, int n_steps, int G)
{
    if (precision == 0)
        return fwd_seg_offset_f4(n_steps, G) * sizeof(float4) + (G >= kSegMinG ? sizeof(SegTab) : 0);
    return (size_t)n_steps * 2 * sizeof(double2) + (size_t)G * sizeof(RowD);
}

cudaError_t launch_prep(const PrepParams &pp, int n_prof, cudaStream_t st)
{
    k_prep<<<dim3(n_prof, pp.n_steps + 1), 256, 0, st>>>(pp);
    return cudaGetLastError();
}

cudaError_t launch_quad(const QuadParams &qp, int precision, int grid, int block, cudaStream_t st)
{
    const size_t smem = quad_smem_bytes(precision, qp.n_steps, qp.G);
    if (precision == 0) {
        cudaFuncSetAttribute(k_quad_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_quad_f32<<<grid, block, smem, st>>>(qp);
    } else {
        cudaFuncSetAttribute(k_quad_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_quad_f64<<<grid, block, smem, st>>>(qp);
    }
    return cudaGetLastError();
}

cudaError_t launch_finish(const FinishParams &fp, int n_prof, cudaStream_t st)
{
    k_finish<<<n_prof, 256, 0, st>>>(fp);
    return cudaGetLastError();
}

int quad_blocks_per_sm(int precision, int n_steps, int G, int block)
{
    int nb = 0;
    const size_t smem = quad_smem_bytes(precision, n_steps, G);
    if (precision == 0) {
        cudaFuncSetAttribute(k_quad_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_quad_f32, block, smem);
    } else {
        cudaFuncSetAttribute(k_quad_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_quad_f64, block, smem);
    }
    return nb > 0 ? nb : 1;
}

}  // namespace isrs
