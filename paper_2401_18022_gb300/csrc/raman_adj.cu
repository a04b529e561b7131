// Adjoint of the FP32 quadrature with the tabulated (Raman-ODE) profile: the
// sensitivities of the throughput T (Sec. IV, Eq. loss) to the profile tables
// {a_c(m), b_c(m)} and to the PSD products, given dT/dSigma_i of every CUT.
//
// For a grid point of piece (a, b) of CUT i with F_c in candidate channel c,
//   ln p_m = A(m) + Sa(m) da + Sb(m) db,
//   A = (a_a + a_b + a_c - a_i + b_c D) / 2,  Sa = (b_a + b_c)/2,  Sb = (b_b + b_c)/2,
// with da = F_a - f_a, db = F_b - f_b, D = f_a + f_b - f_i - f_c.  With the
// per-(piece, candidate) buckets
//   R(m)  = sum_points ybar_i w W d|S|^2/d ln p_m,   Ra(m) = same * da,   Rb(m) = same * db,
// the chain rule gives
//   dT/da_a, dT/da_b, dT/da_c += R/2,   dT/da_i -= R/2,
//   dT/db_a += Ra/2,  dT/db_b += Rb/2,  dT/db_c += (D R + Ra + Rb)/2,
// and the PSD products W = P_a P_b P_c / (B_a B_b B_c) add
//   dT/d ln P_x += ybar_i w W |S|^2 for x = a, b, c.
//
// k_quad_adj_tab walks every piece once per candidate channel, so a warp's
// buckets stay in registers, and evaluates every step term once: the warp
// classifies 32 grid points (one per lane; points of other candidates are
// skipped), appends them to one list per z-sum form, and walks the lists two
// points at a time on half-warps: each of the 16 lanes of a half owns
// K = ceil(M/16) consecutive steps, keeps their terms t_m in registers, the
// half sums them into S with shuffles, and the same registers give
// d|S|^2/d ln p_m = 2 Re(conj(S) t_m).  FP32 lane buckets are folded into
// FP64 shared buckets every 8 batches; at the end of a candidate the block
// reduces them and scatters to the channel tables with FP64 atomics.
#include <cuda_runtime.h>

#include "isrs_internal.cuh"
#include "isrs_kernels.h"
#include "quad_common.cuh"

namespace isrs {

namespace {

constexpr unsigned kFullT = 0xffffffffu;
constexpr int kClsSmallT = 0, kClsDirectT = 1, kClsTeleT = 2;
constexpr int kListCapT = 34;       // a form's list: one carried point + 32 new (+1 pad)
constexpr float kPadLog2T = -1000.0f;

__device__ __forceinline__ float sinc_poly_t(float x)
{
    const float x2 = x * x;
    float sc = fmaf(x2, -2.5052108e-8f, 2.7557319e-6f);   // -1/11!, 1/9!
    sc = fmaf(x2, sc, -1.9841270e-4f);                     // -1/7!
    sc = fmaf(x2, sc, 8.3333333e-3f);                      // 1/5!
    sc = fmaf(x2, sc, -1.6666667e-1f);                     // -1/3!
    return fmaf(x2, sc, 1.0f);
}

__device__ __forceinline__ float half_sum_t(float v)
{
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(kFullT, v, o, 16);
    return v;
}

// Per-piece table (the forward's layout): {A + log2 dz, Sa, Sb, A} in log2 units.
__device__ void tab_setup_adj(const QuadParams &qp, const DevPiece &pc, int nc, float4 *sQ)
{
    const int M = qp.n_steps;
    const int coff = qp.plan_ch_off[pc.plan];
    const double2 *T = qp.ab;
    const double fa = qp.ch_frel[coff + pc.a], fb = qp.ch_frel[coff + pc.b], fi = qp.ch_frel[coff + pc.cut];
    for (int t = threadIdx.x; t < nc * M; t += blockDim.x) {
        const int ci = t / M, m = t - ci * M;
        const int c = pc.c_lo + ci;
        const double2 ta = T[(size_t)pc.a * M + m], tb = T[(size_t)pc.b * M + m];
        const double2 ti = T[(size_t)pc.cut * M + m], tc = T[(size_t)c * M + m];
        const double D = (fa + fb) - (fi + qp.ch_frel[coff + c]);
        const double A = 0.5 * (ta.x + tb.x + tc.x - ti.x + tc.y * D) * kLog2e;
        sQ[t] = make_float4((float)A + qp.zs_a[m].z, (float)(0.5 * (ta.y + tc.y) * kLog2e),
                            (float)(0.5 * (tb.y + tc.y) * kLog2e), (float)A);
    }
}

// Half-warp walks of one grid point of the candidate (weight cp = mult w W af
// ybar, phase rate ph, in-channel offsets da, db).  Lane l16 owns steps
// [K l16, K l16 + K) with tables oq = {A + log2 dz, Sa, Sb, A},
// oz = {z, z^2 + dz^2/12, dz, .}, oe = {edge/2pi hi, lo, ., .}; padding steps
// carry log2 weight -1000.  Each walk adds the lane's bucket terms
// R += cp d|S|^2/d ln p_m, Ra += da (same), Rb += db (same) and returns |S|^2.
template <int K>
__device__ __forceinline__ float walk_direct_t(const float4 *oq, const float4 *oz, float cp, float ph, float da,
                                               float db, float (&R)[K], float (&Ra)[K], float (&Rb)[K])
{
    const float hph = 0.5f * ph;
    const float phr = ph * 0.15915494309189535f;
    float tr[K], ti[K];
    float sr = 0.0f, si = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float4 q = oq[k * 16];
        const float4 z = oz[k * 16];
        float sn, cs;
        sincos_rev(phr * z.x, sn, cs);
        float lp = fmaf(q.y, da, q.x);
        lp = fmaf(q.z, db, lp);
        const float amp = ex2_approx(lp) * sinc_poly_t(hph * z.z);
        tr[k] = amp * cs;
        ti[k] = amp * sn;
        sr += tr[k];
        si += ti[k];
    }
    sr = half_sum_t(sr);
    si = half_sum_t(si);
    const float c2 = 2.0f * cp, ca = c2 * da, cb = c2 * db;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float rr = fmaf(sr, tr[k], si * ti[k]);
        R[k] = fmaf(c2, rr, R[k]);
        Ra[k] = fmaf(ca, rr, Ra[k]);
        Rb[k] = fmaf(cb, rr, Rb[k]);
    }
    return fmaf(sr, sr, si * si);
}

template <int K>
__device__ __forceinline__ float walk_tele_t(const float4 *oq, const float4 *oe, int l16, float cp, float ph,
                                             float da, float db, float (&R)[K], float (&Ra)[K], float (&Rb)[K])
{
    float tr[K], ti[K];
    float Er = 1.0f, Ei = 0.0f, p0 = 0.0f, e1r = 1.0f, e1i = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float4 q = oq[k * 16];
        const float4 e = oe[k * 16];
        float sn, cs;
        phasor_rev_ff(ph, e.x, e.y, sn, cs);
        float lp = fmaf(q.y, da, q.w);
        lp = fmaf(q.z, db, lp);
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
    float elr = __shfl_up_sync(kFullT, Er, 1, 16);
    float eli = __shfl_up_sync(kFullT, Ei, 1, 16);
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
    ur = half_sum_t(ur);
    ui = half_sum_t(ui);
    const float iph2 = 1.0f / (ph * ph);
    const float c2 = 2.0f * cp * iph2, ca = c2 * da, cb = c2 * db;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float rr = fmaf(ur, tr[k], ui * ti[k]);
        R[k] = fmaf(c2, rr, R[k]);
        Ra[k] = fmaf(ca, rr, Ra[k]);
        Rb[k] = fmaf(cb, rr, Rb[k]);
    }
    return fmaf(ur, ur, ui * ui) * iph2;
}

template <int K>
__device__ __forceinline__ float walk_small_t(const float4 *oq, const float4 *oz, float cp, float ph, float da,
                                              float db, float (&R)[K], float (&Ra)[K], float (&Rb)[K])
{
    // |S|^2 = M0^2 - phi^2 (M0 M2 - M1^2); d|S|^2/d ln p_m = w_m (2 M0 - phi^2 (M2 + M0 c_m - 2 M1 z_m))
    float wk[K];
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float4 q = oq[k * 16];
        const float4 z = oz[k * 16];
        float lp = fmaf(q.y, da, q.x);
        lp = fmaf(q.z, db, lp);
        wk[k] = ex2_approx(lp);
        s0 += wk[k];
        s1 = fmaf(wk[k], z.x, s1);
        s2 = fmaf(wk[k], z.y, s2);
    }
    s0 = half_sum_t(s0);
    s1 = half_sum_t(s1);
    s2 = half_sum_t(s2);
    const float ph2 = ph * ph;
    const float al0 = 2.0f * s0 - ph2 * s2, al1 = -ph2 * s0, al2 = 2.0f * ph2 * s1;
    const float ca = cp * da, cb = cp * db;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float4 z = oz[k * 16];
        const float rr = wk[k] * fmaf(al2, z.x, fmaf(al1, z.y, al0));
        R[k] = fmaf(cp, rr, R[k]);
        Ra[k] = fmaf(ca, rr, Ra[k]);
        Rb[k] = fmaf(cb, rr, Rb[k]);
    }
    return fmaf(-ph2, fmaf(s0, s2, -s1 * s1), s0 * s0);
}

}  // namespace

#ifndef ISRS_ADJ_TAB_MIN_BLOCKS
#define ISRS_ADJ_TAB_MIN_BLOCKS 2   // resident blocks per SM the register budget is sized for
#endif

template <int K>
__global__ void __launch_bounds__(256, ISRS_ADJ_TAB_MIN_BLOCKS) k_quad_adj_tab(AdjTabParams ap)
{
    const QuadParams &qp = ap.q;
    extern __shared__ float4 smem_f4[];
    const int M = qp.n_steps, G = qp.G;
    const int nw = blockDim.x >> 5;
    float4 *sQ = smem_f4;                                           // [nc_max][M]
    float4 *sOQ = sQ + (size_t)qp.nc_max * M;                       // [K][16] owned {Ad, Sa, Sb, A} of the candidate
    float4 *sOZ = sOQ + K * 16;                                     // [K][16] owned {z, c, dz, 0}
    float4 *sOE = sOZ + K * 16;                                     // [K][16] owned {edge hi, lo, 0, 0}
    float4 *sL = sOE + K * 16;                                      // [nw][3][kListCapT] {cp, phi, da, db}
    double *sB = reinterpret_cast<double *>(sL + nw * 3 * kListCapT);   // [nw][3][K][16] FP64 buckets
    RowF *rows = reinterpret_cast<RowF *>(sB + (size_t)nw * 3 * K * 16);   // [G]
    __shared__ PieceConst<float> kc;
    __shared__ float s_d0[2];
    __shared__ double scratch[32];
    __shared__ int s_item;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int l16 = lane & 15, half = lane >> 4;
    // the owned z and edge tables never change; padding steps repeat the last edge
    {
        const float4 zl = qp.zs_b[M - 1];
        for (int t = threadIdx.x; t < K * 16; t += blockDim.x) {
            const int k = t >> 4, l = t & 15, m = l * K + k;
            float4 z = make_float4(0.f, 0.f, 0.f, 0.f), e = make_float4(zl.x, zl.y, 0.f, 0.f);
            if (m < M) {
                const float4 za = qp.zs_a[m];
                const float4 zb = qp.zs_b[m];
                z = make_float4(za.x, za.y, za.w, 0.f);
                e = make_float4(zb.x, zb.y, 0.f, 0.f);
            }
            sOZ[k * 16 + l] = z;
            sOE[k * 16 + l] = e;
        }
    }
    for (int t = threadIdx.x; t < nw * 3 * K * 16; t += blockDim.x) sB[t] = 0.0;

    const float c3 = (float)(kPi * qp.beta3);
    const float c4 = (float)(2.0 * kPi * kPi / 3.0 * qp.beta4);
    const float b2 = (float)qp.beta2;
    const float m4pi2 = (float)(-4.0 * kPi * kPi);
    const float phi_direct = 3.14159265f / qp.dz_max;
    const float phi_small = 0.02f / qp.L;
    const float invG = 1.0f / (float)G;
    const float4 *oq = sOQ + l16, *oz = sOZ + l16, *oe = sOE + l16;
    float4 *Ls = sL + warp * 3 * kListCapT;
    float4 *Ld = Ls + kListCapT;
    float4 *Lt = Ld + kListCapT;
    double *myB = sB + (size_t)warp * 3 * K * 16;
    const unsigned lt_mask = (1u << lane) - 1u;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(qp.counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= qp.n_items) break;
        const DevItem item = qp.items[it];
        const float ybar = (float)ap.ybar[ap.item_slot[it]];
        for (int kp = item.piece0; kp < item.piece1; ++kp) {
            const DevPiece pc = qp.pieces[kp];
            piece_rows<RowF>(pc, G, qp.eps_v1, rows);
            piece_consts<float>(qp, pc, item.prof, 0.0f, qp.pd_f, kc);
            const int coff = qp.plan_ch_off[pc.plan];
            const double fi_d = qp.ch_frel[coff + pc.cut];
            if (threadIdx.x == 0) {
                s_d0[0] = (float)(qp.ch_frel[coff + pc.a] - fi_d);
                s_d0[1] = (float)(qp.ch_frel[coff + pc.b] - fi_d);
            }
            __syncthreads();
            tab_setup_adj(qp, pc, kc.nc, sQ);
            __syncthreads();
            const float fi = kc.fi, s1g = kc.s1, s2g = kc.s2, mult = kc.mult;
            const float da0 = s_d0[0], db0 = s_d0[1];
            const float three_fi2 = 3.0f * fi * fi;
            const int npts = G * G;
            const int nc = kc.nc;
            for (int cc = 0; cc < nc; ++cc) {
                // lane-contiguous copy of the candidate's owned step tables
                for (int t = threadIdx.x; t < K * 16; t += blockDim.x) {
                    const int k = t >> 4, l = t & 15, m = l * K + k;
                    sOQ[k * 16 + l] = m < M ? sQ[cc * M + m] : make_float4(kPadLog2T, 0.f, 0.f, kPadLog2T);
                }
                __syncthreads();
                float R[K], Ra[K], Rb[K];
#pragma unroll
                for (int k = 0; k < K; ++k) R[k] = Ra[k] = Rb[k] = 0.0f;
                float vsum = 0.0f;
                int ns = 0, nd = 0, nt = 0;
                int batches = 0;
                for (int qb = warp * 32; qb < npts; qb += blockDim.x) {
                    // ---- 1. this lane's grid point, if its F_c is in candidate cc
                    const int q = qb + lane;
                    float cp = 0.0f, phi = 0.0f, da = 0.0f, db = 0.0f;
                    int cls = -1;
                    if (q < npts) {
                        const int r = (int)(((float)q + 0.5f) * invG);
                        const int j = q - r * G;
                        const RowF rw = rows[r];
                        if (rw.w != 0.0f) {
                            const float d = ((float)j + 0.5f - 0.5f * (float)G) * rw.du2;
                            const float e = expf(d);
                            const float f1 = s1g * (rw.xc * e);
                            const float f2 = s2g * (rw.yc * __frcp_rn(e));
                            const float u = f1 + f2;
                            if (u >= kc.lo[cc] && u < kc.hi[cc]) {
                                // the candidates are disjoint: the first match is cc itself
                                bool earlier = false;
                                for (int c = 0; c < cc; ++c) earlier |= (u >= kc.lo[c] && u < kc.hi[c]);
                                if (!earlier) {
                                    const float W = kc.wab * kc.pd[cc];
                                    da = f1 - da0;
                                    db = f2 - db0;
                                    const float br = b2 + c3 * (u + 2.0f * fi) +
                                                     c4 * (f1 * f1 + 1.5f * f1 * f2 + 3.0f * fi * u + f2 * f2 +
                                                           three_fi2);
                                    phi = m4pi2 * f1 * f2 * br;
                                    const float aphi = fabsf(phi);
                                    cls = aphi <= phi_small ? kClsSmallT : (aphi <= phi_direct ? kClsDirectT : kClsTeleT);
                                    cp = mult * rw.w * W * array_factor_f(phi, qp) * ybar;
                                }
                            }
                        }
                    }
                    // append to the form's list
                    const unsigned bs = __ballot_sync(kFullT, cls == kClsSmallT);
                    const unsigned bd = __ballot_sync(kFullT, cls == kClsDirectT);
                    const unsigned bt = __ballot_sync(kFullT, cls == kClsTeleT);
                    if (cls >= 0) {
                        const float4 v = make_float4(cp, phi, da, db);
                        if (cls == kClsSmallT) Ls[ns + __popc(bs & lt_mask)] = v;
                        else if (cls == kClsDirectT) Ld[nd + __popc(bd & lt_mask)] = v;
                        else Lt[nt + __popc(bt & lt_mask)] = v;
                    }
                    ns += __popc(bs);
                    nd += __popc(bd);
                    nt += __popc(bt);
                    __syncwarp();
                    // ---- 2. walk the lists in pairs, one point per half-warp
                    for (int p = half; p + 1 - half < nd; p += 2) {
                        const float4 st = Ld[p];
                        const float s2 = walk_direct_t<K>(oq, oz, st.x, st.y, st.z, st.w, R, Ra, Rb);
                        vsum += l16 == 0 ? st.x * s2 : 0.0f;
                    }
                    for (int p = half; p + 1 - half < nt; p += 2) {
                        const float4 st = Lt[p];
                        const float s2 = walk_tele_t<K>(oq, oe, l16, st.x, st.y, st.z, st.w, R, Ra, Rb);
                        vsum += l16 == 0 ? st.x * s2 : 0.0f;
                    }
                    for (int p = half; p + 1 - half < ns; p += 2) {
                        const float4 st = Ls[p];
                        const float s2 = walk_small_t<K>(oq, oz, st.x, st.y, st.z, st.w, R, Ra, Rb);
                        vsum += l16 == 0 ? st.x * s2 : 0.0f;
                    }
                    // an odd point waits at the head of its list for the next batch
                    __syncwarp();
                    if (lane == 0) {
                        if (nd & 1) Ld[0] = Ld[nd - 1];
                        if (nt & 1) Lt[0] = Lt[nt - 1];
                        if (ns & 1) Ls[0] = Ls[ns - 1];
                    }
                    nd &= 1;
                    nt &= 1;
                    ns &= 1;
                    if (++batches == 8) {
                        batches = 0;
#pragma unroll
                        for (int k = 0; k < K; ++k) {
                            const float r0 = R[k] + __shfl_xor_sync(kFullT, R[k], 16);
                            const float r1 = Ra[k] + __shfl_xor_sync(kFullT, Ra[k], 16);
                            const float r2 = Rb[k] + __shfl_xor_sync(kFullT, Rb[k], 16);
                            if (half == 0) {
                                myB[(0 * K + k) * 16 + l16] += (double)r0;
                                myB[(1 * K + k) * 16 + l16] += (double)r1;
                                myB[(2 * K + k) * 16 + l16] += (double)r2;
                            }
                            R[k] = Ra[k] = Rb[k] = 0.0f;
                        }
                    }
                    __syncwarp();          // the next batch appends to the lists
                }
                // the last odd point of each form, beside a zero-weight copy of itself
                if (nd) {
                    float4 st = Ld[0];
                    if (half) st.x = 0.0f;
                    const float s2 = walk_direct_t<K>(oq, oz, st.x, st.y, st.z, st.w, R, Ra, Rb);
                    vsum += l16 == 0 ? st.x * s2 : 0.0f;
                }
                if (nt) {
                    float4 st = Lt[0];
                    if (half) st.x = 0.0f;
                    const float s2 = walk_tele_t<K>(oq, oe, l16, st.x, st.y, st.z, st.w, R, Ra, Rb);
                    vsum += l16 == 0 ? st.x * s2 : 0.0f;
                }
                if (ns) {
                    float4 st = Ls[0];
                    if (half) st.x = 0.0f;
                    const float s2 = walk_small_t<K>(oq, oz, st.x, st.y, st.z, st.w, R, Ra, Rb);
                    vsum += l16 == 0 ? st.x * s2 : 0.0f;
                }
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const float r0 = R[k] + __shfl_xor_sync(kFullT, R[k], 16);
                    const float r1 = Ra[k] + __shfl_xor_sync(kFullT, Ra[k], 16);
                    const float r2 = Rb[k] + __shfl_xor_sync(kFullT, Rb[k], 16);
                    if (half == 0) {
                        myB[(0 * K + k) * 16 + l16] += (double)r0;
                        myB[(1 * K + k) * 16 + l16] += (double)r1;
                        myB[(2 * K + k) * 16 + l16] += (double)r2;
                    }
                }
                const double vtot = block_sum_d((double)vsum, scratch);   // syncs the block
                const int c = pc.c_lo + cc;
                const double D = (qp.ch_frel[coff + pc.a] + qp.ch_frel[coff + pc.b]) -
                                 (fi_d + qp.ch_frel[coff + c]);
                for (int m = threadIdx.x; m < M; m += blockDim.x) {
                    const int ln = m / K, kk = m - ln * K;
                    double r0 = 0.0, r1 = 0.0, r2 = 0.0;
                    for (int w = 0; w < nw; ++w) {
                        double *b = sB + (size_t)w * 3 * K * 16;
                        r0 += b[(0 * K + kk) * 16 + ln];
                        r1 += b[(1 * K + kk) * 16 + ln];
                        r2 += b[(2 * K + kk) * 16 + ln];
                        b[(0 * K + kk) * 16 + ln] = 0.0;
                        b[(1 * K + kk) * 16 + ln] = 0.0;
                        b[(2 * K + kk) * 16 + ln] = 0.0;
                    }
                    if (r0 == 0.0 && r1 == 0.0 && r2 == 0.0) continue;
                    double2 *g = ap.gAB;
                    atomicAdd(&g[(size_t)pc.a * M + m].x, 0.5 * r0);
                    atomicAdd(&g[(size_t)pc.b * M + m].x, 0.5 * r0);
                    atomicAdd(&g[(size_t)c * M + m].x, 0.5 * r0);
                    atomicAdd(&g[(size_t)pc.cut * M + m].x, -0.5 * r0);
                    atomicAdd(&g[(size_t)pc.a * M + m].y, 0.5 * r1);
                    atomicAdd(&g[(size_t)pc.b * M + m].y, 0.5 * r2);
                    atomicAdd(&g[(size_t)c * M + m].y, 0.5 * (D * r0 + r1 + r2));
                }
                if (threadIdx.x == 0 && vtot != 0.0) {
                    atomicAdd(&ap.gV[pc.a], vtot);
                    atomicAdd(&ap.gV[pc.b], vtot);
                    atomicAdd(&ap.gV[c], vtot);
                }
                __syncthreads();
            }
            __syncthreads();
        }
    }
}

namespace {

template <int K>
void *adj_tab_fn()
{
    return (void *)k_quad_adj_tab<K>;
}

void *adj_tab_kernel_for(int n_steps)
{
    switch ((n_steps + 15) / 16) {
    case 1: return adj_tab_fn<1>();
    case 2: return adj_tab_fn<2>();
    case 3: return adj_tab_fn<3>();
    case 4: return adj_tab_fn<4>();
    case 5: return adj_tab_fn<5>();
    case 6: return adj_tab_fn<6>();
    case 7: return adj_tab_fn<7>();
    case 8: return adj_tab_fn<8>();
    }
    return nullptr;
}

}  // namespace

size_t adjoint_tab_smem_bytes(int n_steps, int G, int nc_max, int block)
{
    const int K = (n_steps + 15) / 16, nw = block / 32;
    return ((size_t)n_steps * nc_max + 3 * K * 16 + (size_t)nw * 3 * kListCapT) * sizeof(float4) +
           (size_t)nw * 3 * K * 16 * sizeof(double) + (size_t)G * sizeof(RowF);
}

int adjoint_tab_blocks_per_sm(int n_steps, int G, int nc_max, int block)
{
    void *fn = adj_tab_kernel_for(n_steps);
    if (!fn) return 0;
    const size_t smem = adjoint_tab_smem_bytes(n_steps, G, nc_max, block);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, smem);
    return nb > 0 ? nb : 1;
}

cudaError_t launch_adjoint_tab(const AdjTabParams &ap, int grid, int block, cudaStream_t st)
{
    void *fn = adj_tab_kernel_for(ap.q.n_steps);
    if (!fn) return cudaErrorInvalidValue;
    const size_t smem = adjoint_tab_smem_bytes(ap.q.n_steps, ap.q.G, ap.q.nc_max, block);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    AdjTabParams a = ap;
    void *args[] = {&a};
    return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, st);
}

}  // namespace isrs
