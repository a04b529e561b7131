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
// buckets stay in registers: pass 1 (one grid point per lane, points of other
// candidates skipped) forms the z-sum as the forward kernel does; pass 2 turns
// the warp around (every lane owns K consecutive steps, their tables held in
// registers) and accumulates the buckets over the warp's 32 points.  FP32
// lane sums are folded into FP64 shared buckets every 8 batches; at the end of
// a candidate the block reduces them and scatters to the channel tables with
// FP64 atomics.
#include <cuda_runtime.h>

#include "isrs_internal.cuh"
#include "isrs_kernels.h"
#include "quad_common.cuh"

namespace isrs {

namespace {

constexpr int kPathSmall = 0, kPathDirect = 1, kPathTele = 2;

__device__ __forceinline__ float sinc_poly_t(float x)
{
    const float x2 = x * x;
    float sc = fmaf(x2, -2.5052108e-8f, 2.7557319e-6f);   // -1/11!, 1/9!
    sc = fmaf(x2, sc, -1.9841270e-4f);                     // -1/7!
    sc = fmaf(x2, sc, 8.3333333e-3f);                      // 1/5!
    sc = fmaf(x2, sc, -1.6666667e-1f);                     // -1/3!
    return fmaf(x2, sc, 1.0f);
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

}  // namespace

template <int K>
__global__ void __launch_bounds__(256, 2) k_quad_adj_tab(AdjTabParams ap)
{
    const QuadParams &qp = ap.q;
    extern __shared__ float4 smem_f4[];
    const int M = qp.n_steps, G = qp.G;
    const int nw = blockDim.x >> 5;
    float4 *sZ = smem_f4;                                           // [M] {z, z^2 + dz^2/12, dz, 0}
    float4 *sE = sZ + M;                                            // [M] {edge/2pi hi, lo, 0, 0}
    float4 *sQ = sE + M;                                            // [nc_max][M]
    RowF *rows = reinterpret_cast<RowF *>(sQ + (size_t)qp.nc_max * M);   // [G]
    float4 *sPs = reinterpret_cast<float4 *>(rows + G);             // [nw][32][2] staged point states
    double *sB = reinterpret_cast<double *>(sPs + nw * 64);         // [nw][3][K][32] FP64 buckets
    __shared__ PieceConst<float> kc;
    __shared__ float s_d0[2];
    __shared__ double scratch[32];
    __shared__ int s_item;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const float4 za = qp.zs_a[m];
        const float4 zb = qp.zs_b[m];
        sZ[m] = make_float4(za.x, za.y, za.w, 0.0f);
        sE[m] = make_float4(zb.x, zb.y, 0.0f, 0.0f);
    }
    for (int t = threadIdx.x; t < nw * 3 * K * 32; t += blockDim.x) sB[t] = 0.0;
    __syncthreads();

    const float c3 = (float)(kPi * qp.beta3);
    const float c4 = (float)(2.0 * kPi * kPi / 3.0 * qp.beta4);
    const float b2 = (float)qp.beta2;
    const float m4pi2 = (float)(-4.0 * kPi * kPi);
    const float phi_direct = 3.14159265f / qp.dz_max;
    const float phi_small = 0.02f / qp.L;
    const float invG = 1.0f / (float)G;
    const int m0 = lane * K;
    float4 *myPs = sPs + warp * 64;
    double *myB = sB + (size_t)warp * 3 * K * 32;

    // this lane's steps: the z tables never change
    float oz[K], oc[K], odz[K], oeh[K], oel[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const bool ok = m0 + k < M;
        const float4 z = ok ? sZ[m0 + k] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 e = ok ? sE[m0 + k] : make_float4(0.f, 0.f, 0.f, 0.f);
        oz[k] = z.x;
        oc[k] = z.y;
        odz[k] = z.z;
        oeh[k] = e.x;
        oel[k] = e.y;
    }
    const float e0h = (m0 > 0 && m0 < M) ? sE[m0 - 1].x : 0.0f;     // lower edge of the lane's block
    const float e0l = (m0 > 0 && m0 < M) ? sE[m0 - 1].y : 0.0f;

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
                const float4 *Q = sQ + cc * M;
                float oAd[K], oA[K], oSa[K], oSb[K];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const float4 q = (m0 + k < M) ? Q[m0 + k] : make_float4(0.f, 0.f, 0.f, 0.f);
                    oAd[k] = q.x;
                    oSa[k] = q.y;
                    oSb[k] = q.z;
                    oA[k] = q.w;
                }
                float R[K], Ra[K], Rb[K];
#pragma unroll
                for (int k = 0; k < K; ++k) R[k] = Ra[k] = Rb[k] = 0.0f;
                float vsum = 0.0f;
                int batches = 0;
                for (int qb = warp * 32; qb < npts; qb += blockDim.x) {
                    // ---- pass 1: this lane's grid point, if its F_c is in candidate cc
                    const int q = qb + lane;
                    float cp = 0.0f, phi = 0.0f, da = 0.0f, db = 0.0f, q0 = 0.0f, q1 = 0.0f, q2 = 0.0f;
                    int path = 0;
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
                                    float S2;
                                    if (aphi <= phi_small) {
                                        path = kPathSmall;
                                        for (int m = 0; m < M; ++m) {
                                            const float4 t = Q[m];
                                            const float4 z = sZ[m];
                                            float lp = fmaf(t.y, da, t.x);
                                            lp = fmaf(t.z, db, lp);
                                            const float w = ex2_approx(lp);
                                            q0 += w;
                                            q1 = fmaf(w, z.x, q1);
                                            q2 = fmaf(w, z.y, q2);
                                        }
                                        S2 = fmaf(-phi * phi, fmaf(q0, q2, -q1 * q1), q0 * q0);
                                    } else if (aphi <= phi_direct) {
                                        path = kPathDirect;
                                        const float hphi = 0.5f * phi;
                                        const float phir = phi * 0.15915494309189535f;
                                        for (int m = 0; m < M; ++m) {
                                            const float4 t = Q[m];
                                            const float4 z = sZ[m];
                                            float sn, cs;
                                            sincos_rev(phir * z.x, sn, cs);
                                            float lp = fmaf(t.y, da, t.x);
                                            lp = fmaf(t.z, db, lp);
                                            const float amp = ex2_approx(lp) * sinc_poly_t(hphi * z.z);
                                            q0 = fmaf(amp, cs, q0);
                                            q1 = fmaf(amp, sn, q1);
                                        }
                                        S2 = q0 * q0 + q1 * q1;
                                    } else {
                                        path = kPathTele;
                                        float Er = 1.0f, Ei = 0.0f;
                                        for (int m = 0; m < M; ++m) {
                                            const float4 t = Q[m];
                                            const float4 eg = sE[m];
                                            float sn, cs;
                                            phasor_rev_ff(phi, eg.x, eg.y, sn, cs);
                                            float lp = fmaf(t.y, da, t.w);
                                            lp = fmaf(t.z, db, lp);
                                            const float p = ex2_approx(lp);
                                            q0 = fmaf(p, cs - Er, q0);
                                            q1 = fmaf(p, sn - Ei, q1);
                                            Er = cs;
                                            Ei = sn;
                                        }
                                        S2 = (q0 * q0 + q1 * q1) / (phi * phi);
                                    }
                                    cp = mult * rw.w * W * array_factor_f(phi, qp) * ybar;
                                    vsum = fmaf(cp, S2, vsum);
                                }
                            }
                        }
                    }
                    myPs[2 * lane] = make_float4(cp, phi, da, db);
                    myPs[2 * lane + 1] = make_float4(q0, q1, q2, __int_as_float(path));
                    __syncwarp();
                    // ---- pass 2: the warp's 32 points, every lane on its own steps
                    for (int p = 0; p < 32; ++p) {
                        const float4 st0 = myPs[2 * p];
                        const float cpp = st0.x;
                        if (cpp == 0.0f) continue;
                        const float4 st1 = myPs[2 * p + 1];
                        const float ph = st0.y, pda = st0.z, pdb = st0.w;
                        const float p0 = st1.x, p1 = st1.y, p2 = st1.z;
                        const int pth = __float_as_int(st1.w);
                        const float ca = cpp * pda, cb = cpp * pdb;
                        if (pth == kPathSmall) {
                            // d|S|^2/d ln p_m = w_m (2 M0 - phi^2 (M2 + M0 c_m - 2 M1 z_m))
                            const float ph2 = ph * ph;
                            const float al0 = 2.0f * p0 - ph2 * p2, al1 = -ph2 * p0, al2 = 2.0f * ph2 * p1;
#pragma unroll
                            for (int k = 0; k < K; ++k) {
                                if (m0 + k < M) {
                                    float lp = fmaf(oSa[k], pda, oAd[k]);
                                    lp = fmaf(oSb[k], pdb, lp);
                                    const float rr = ex2_approx(lp) * fmaf(al2, oz[k], fmaf(al1, oc[k], al0));
                                    R[k] = fmaf(cpp, rr, R[k]);
                                    Ra[k] = fmaf(ca, rr, Ra[k]);
                                    Rb[k] = fmaf(cb, rr, Rb[k]);
                                }
                            }
                        } else if (pth == kPathDirect) {
                            // d|S|^2/d ln p_m = 2 Re(conj(S) p_m dz_m sinc e^{j phi z_m})
                            const float hph = 0.5f * ph;
                            const float phr = ph * 0.15915494309189535f;
#pragma unroll
                            for (int k = 0; k < K; ++k) {
                                if (m0 + k < M) {
                                    float sn, cs;
                                    sincos_rev(phr * oz[k], sn, cs);
                                    float lp = fmaf(oSa[k], pda, oAd[k]);
                                    lp = fmaf(oSb[k], pdb, lp);
                                    const float amp = ex2_approx(lp) * sinc_poly_t(hph * odz[k]);
                                    const float rr = 2.0f * amp * fmaf(p0, cs, p1 * sn);
                                    R[k] = fmaf(cpp, rr, R[k]);
                                    Ra[k] = fmaf(ca, rr, Ra[k]);
                                    Rb[k] = fmaf(cb, rr, Rb[k]);
                                }
                            }
                        } else {
                            // d|S|^2/d ln p_m = 2 Re(conj(U) p_m (E_{m+1} - E_m)) / phi^2
                            float Er = 1.0f, Ei = 0.0f;
                            if (m0 > 0) phasor_rev_ff(ph, e0h, e0l, Ei, Er);
                            const float g = 2.0f / (ph * ph);
#pragma unroll
                            for (int k = 0; k < K; ++k) {
                                if (m0 + k < M) {
                                    float sn, cs;
                                    phasor_rev_ff(ph, oeh[k], oel[k], sn, cs);
                                    float lp = fmaf(oSa[k], pda, oA[k]);
                                    lp = fmaf(oSb[k], pdb, lp);
                                    const float rr = g * ex2_approx(lp) * fmaf(p0, cs - Er, p1 * (sn - Ei));
                                    R[k] = fmaf(cpp, rr, R[k]);
                                    Ra[k] = fmaf(ca, rr, Ra[k]);
                                    Rb[k] = fmaf(cb, rr, Rb[k]);
                                    Er = cs;
                                    Ei = sn;
                                }
                            }
                        }
                    }
                    if (++batches == 8) {
                        batches = 0;
#pragma unroll
                        for (int k = 0; k < K; ++k) {
                            myB[(0 * K + k) * 32 + lane] += (double)R[k];
                            myB[(1 * K + k) * 32 + lane] += (double)Ra[k];
                            myB[(2 * K + k) * 32 + lane] += (double)Rb[k];
                            R[k] = Ra[k] = Rb[k] = 0.0f;
                        }
                    }
                    __syncwarp();          // the next batch overwrites the staged states
                }
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    myB[(0 * K + k) * 32 + lane] += (double)R[k];
                    myB[(1 * K + k) * 32 + lane] += (double)Ra[k];
                    myB[(2 * K + k) * 32 + lane] += (double)Rb[k];
                }
                const double vtot = block_sum_d((double)vsum, scratch);   // syncs the block
                const int c = pc.c_lo + cc;
                const double D = (qp.ch_frel[coff + pc.a] + qp.ch_frel[coff + pc.b]) -
                                 (fi_d + qp.ch_frel[coff + c]);
                for (int m = threadIdx.x; m < M; m += blockDim.x) {
                    const int ln = m / K, kk = m - ln * K;
                    double r0 = 0.0, r1 = 0.0, r2 = 0.0;
                    for (int w = 0; w < nw; ++w) {
                        double *b = sB + (size_t)w * 3 * K * 32;
                        r0 += b[(0 * K + kk) * 32 + ln];
                        r1 += b[(1 * K + kk) * 32 + ln];
                        r2 += b[(2 * K + kk) * 32 + ln];
                        b[(0 * K + kk) * 32 + ln] = 0.0;
                        b[(1 * K + kk) * 32 + ln] = 0.0;
                        b[(2 * K + kk) * 32 + ln] = 0.0;
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
    switch ((n_steps + 31) / 32) {
    case 1: return adj_tab_fn<1>();
    case 2: return adj_tab_fn<2>();
    case 3: return adj_tab_fn<3>();
    case 4: return adj_tab_fn<4>();
    }
    return nullptr;
}

}  // namespace

size_t adjoint_tab_smem_bytes(int n_steps, int G, int nc_max, int block)
{
    const int K = (n_steps + 31) / 32, nw = block / 32;
    return (size_t)n_steps * (2 + nc_max) * sizeof(float4) + (size_t)G * sizeof(RowF) +
           (size_t)nw * 64 * sizeof(float4) + (size_t)nw * 3 * K * 32 * sizeof(double);
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
