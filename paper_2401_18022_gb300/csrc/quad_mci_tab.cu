// Multi-channel-interference (MCI) cells on their own grid with the
// tabulated (Raman-ODE) power profile (Sec. III, App. A: the integral of
// Eq. gain_fin over the whole band, with rho(z, f) from the Raman
// power-evolution ODEs).
//
// The cells, their triangular enumeration and their G_mci x G_mci hyperbolic
// grids are those of quad_mci.cu.  Only the profile term of Eq. pk changes:
// inside channel c, ln rho(z_m, F) = a_c(m) + b_c(m) (F - f_c), so for a point
// of cell (a, b) with F_c in channel c and in-channel offsets
// da = F_a - f_a, db = F_b - f_b, dc = F_c - f_c,
//   ln p_m = 1/2 [a_a + a_b - a_i + a_c + b_a da + b_b db + b_c dc](m).
// The first three terms belong to the cell; per chunk of cells the FP32
// kernel tabulates, per cell and step, {A + log2 dz, S_a, S_b, A} (log2
// units) in shared memory, and reads {a_c, b_c}(m) of the point's F_c channel
// from an FP32 copy of the profile tables (one float2 per channel and step,
// L1/L2-resident), so a step costs two loads and four FMAs for ln p.  The
// z-sum forms are those of the closed-form MCI kernel (second-order small
// phase, direct, telescoped with the wide phase reduction).
#include <cuda_runtime.h>

#include <algorithm>

#include "isrs_internal.cuh"
#include "isrs_kernels.h"
#include "quad_cells.cuh"
#include "quad_common.cuh"
#include "quad_zsum.cuh"

namespace isrs {

namespace {

constexpr int kMciTabCells = 32;   // cells per chunk at most (their step rows share the block's memory)

// {1/2 log2(e) a_c(m), 1/2 log2(e) b_c(m)} in FP32, same index as qp.ab
__global__ void __launch_bounds__(256) k_tab_half_log2(const double2 *ab, float2 *abf, int n)
{
    for (int t = threadIdx.x + blockIdx.x * blockDim.x; t < n; t += blockDim.x * gridDim.x) {
        const double2 v = ab[t];
        abf[t] = make_float2((float)(0.5 * kLog2e * v.x), (float)(0.5 * kLog2e * v.y));
    }
}

// FP32 z-sums of Eq. slow_vary with
//   log2 p_m (dz_m) = Q.x + Q.y da + Q.z db + T.x + T.y dc   (Q.w for the
// telescoped form, without log2 dz); sA[m] = {z, z^2 + dz^2/12, log2 dz, dz},
// sB[m] = {z_{m+1}/2pi hi, lo, ., .}.
__device__ __forceinline__ float lp_tab(const float4 &q, float qx, const float2 &t, float da, float db, float dc)
{
    float lp = fmaf(q.y, da, qx);
    lp = fmaf(q.z, db, lp);
    lp = fmaf(t.y, dc, lp);
    return lp + t.x;
}

__device__ __forceinline__ float zsum_small_mt(float phi, float da, float db, float dc, const float4 *Q,
                                               const float2 *Tc, const float4 *sA, int M)
{
    float M0 = 0.0f, M1 = 0.0f, M2 = 0.0f;
#pragma unroll 4
    for (int m = 0; m < M; ++m) {
        const float4 q = Q[m];
        const float4 a = sA[m];
        const float w = ex2_approx(lp_tab(q, q.x, __ldg(Tc + m), da, db, dc));   // p_m dz_m
        M0 += w;
        M1 = fmaf(w, a.x, M1);
        M2 = fmaf(w, a.y, M2);
    }
    return fmaf(-phi * phi, fmaf(M0, M2, -M1 * M1), M0 * M0);
}

__device__ __forceinline__ float zsum_direct_mt(float phi, float da, float db, float dc, const float4 *Q,
                                                const float2 *Tc, const float4 *sA, int M)
{
    float Sr = 0.0f, Si = 0.0f;
    const float hphi = 0.5f * phi;
    const float phir = phi * 0.15915494309189535f;
#pragma unroll 4
    for (int m = 0; m < M; ++m) {
        const float4 q = Q[m];
        const float4 a = sA[m];
        float sn, cs;
        sincos_rev(phir * a.x, sn, cs);
        const float x = hphi * a.w;
        const float x2 = x * x;
        float sc = fmaf(x2, -2.5052108e-8f, 2.7557319e-6f);   // -1/11!, 1/9!
        sc = fmaf(x2, sc, -1.9841270e-4f);                     // -1/7!
        sc = fmaf(x2, sc, 8.3333333e-3f);                      // 1/5!
        sc = fmaf(x2, sc, -1.6666667e-1f);                     // -1/3!
        sc = fmaf(x2, sc, 1.0f);
        const float amp = ex2_approx(lp_tab(q, q.x, __ldg(Tc + m), da, db, dc)) * sc;   // p_m dz_m sinc
        Sr = fmaf(amp, cs, Sr);
        Si = fmaf(amp, sn, Si);
    }
    return Sr * Sr + Si * Si;
}

__device__ __forceinline__ float zsum_tele_mt(float phi, float da, float db, float dc, const float4 *Q,
                                              const float2 *Tc, const float4 *sB, int M)
{
    float Er = 1.0f, Ei = 0.0f, Sr = 0.0f, Si = 0.0f;
#pragma unroll 4
    for (int m = 0; m < M; ++m) {
        const float4 q = Q[m];
        const float4 e = sB[m];
        float sn, cs;
        phasor_rev_ff_wide(phi, e.x, e.y, sn, cs);
        const float p = ex2_approx(lp_tab(q, q.w, __ldg(Tc + m), da, db, dc));
        Sr = fmaf(p, cs - Er, Sr);
        Si = fmaf(p, sn - Ei, Si);
        Er = cs;
        Ei = sn;
    }
    return __fdividef(Sr * Sr + Si * Si, phi * phi);
}

}  // namespace

// ---------------------------------------------------------------------------
// k_quad_mci_f32_tab: persistent over MCI work items (cell ranges of one
// CUT).  The item's cells are taken in chunks of qp.mci_cpc: the chunk's
// cells are decoded once, their step rows built (FP32, from the FP32 profile
// tables), then one thread per (cell, grid row) walks the row's G_mci points.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 3) k_quad_mci_f32_tab(QuadParams qp)
{
    extern __shared__ float4 smem_f4[];
    const int M = qp.n_steps, G = qp.G, CPC = qp.mci_cpc;
    float4 *sA = smem_f4;                              // [M] {z, z^2 + dz^2/12, log2 dz, dz}
    float4 *sB = sA + M;                               // [M] {edge/2pi hi, lo, ., .}
    float4 *sQ = sB + M;                               // [CPC][M] {A + log2 dz, Sa, Sb, A}
    float *rel = reinterpret_cast<float *>(sQ + (size_t)CPC * M);   // [n] channel centre - f_i
    float *hb = rel + qp.mci_n_max;                    // [n] B/2
    float *pd = hb + qp.mci_n_max;                     // [n] P/B
    __shared__ int2 sCell[kMciTabCells];
    __shared__ double scratch[32];
    __shared__ int s_item;

    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        sA[m] = qp.zs_a[m];
        sB[m] = qp.zs_b[m];
    }
    const float c3 = (float)(kPi * qp.beta3);
    const float c4 = (float)(2.0 * kPi * kPi / 3.0 * qp.beta4);
    const float b2 = (float)qp.beta2;
    const float m4pi2 = (float)(-4.0 * kPi * kPi);
    const float phi_direct = 3.14159265f / qp.dz_max;
    const float phi_small = 0.02f / qp.L;
    const float eps = (float)qp.eps_v1;
    int cur_prof = -1, cur_cut = -1;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(qp.counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= qp.n_items) break;
        const DevItem item = qp.items[it];
        const int plan = qp.prof_plan[item.prof];
        const int coff = qp.plan_ch_off[plan];
        const int poff = qp.prof_ch_off[item.prof];
        const int n = qp.plan_n[plan];
        const int i = item.cut;
        if (item.prof != cur_prof || i != cur_cut) {
            const double fi = qp.ch_frel[coff + i];
            for (int c = threadIdx.x; c < n; c += blockDim.x) {
                rel[c] = (float)(qp.ch_frel[coff + c] - fi);
                hb[c] = (float)(0.5 * qp.ch_B[coff + c]);
                pd[c] = qp.pd_f[poff + c];
            }
            cur_prof = item.prof;
            cur_cut = i;
        }
        const float2 *T = qp.ab_f + (size_t)poff * M;   // this profile's channel rows
        const float fi = (float)qp.ch_frel[coff + i];
        const float three_fi2 = 3.0f * fi * fi;
        const int n2 = n - 1;
        float sum = 0.0f, comp = 0.0f;
        for (int t0 = item.piece0; t0 < item.piece1; t0 += CPC) {
            const int ncc = min(CPC, item.piece1 - t0);
            __syncthreads();                          // the previous chunk's rows are no longer read
            if (threadIdx.x < ncc) {
                int ap, bp;
                tri_decode(t0 + threadIdx.x, n2, ap, bp);
                sCell[threadIdx.x] = make_int2(dbg_clamp(ap + (ap >= i), n, kDbgCell, qp.dbg),
                                               dbg_clamp(bp + (bp >= i), n, kDbgCell, qp.dbg));
            }
            __syncthreads();
            for (int e = threadIdx.x; e < ncc * M; e += blockDim.x) {
                const int cc = e / M, m = e - cc * M;
                const int2 ab = sCell[cc];
                const float2 ta = T[(size_t)ab.x * M + m], tb = T[(size_t)ab.y * M + m];
                const float A = (ta.x + tb.x) - T[(size_t)i * M + m].x;
                sQ[e] = make_float4(A + sA[m].z, ta.y, tb.y, A);
            }
            __syncthreads();
            for (int q = threadIdx.x; q < ncc * G; q += blockDim.x) {
                const int cc = q / G, r = q - cc * G;
                const int2 ab = sCell[cc];
                const int a = ab.x, b = ab.y;
                const float mult = a == b ? 1.0f : 2.0f;
                const float ra = rel[a], rb = rel[b];
                const float s1 = ra > 0.0f ? 1.0f : -1.0f, s2 = rb > 0.0f ? 1.0f : -1.0f;
                const float xlo = fabsf(ra) - hb[a], xhi = fabsf(ra) + hb[a];
                const float ylo = fabsf(rb) - hb[b], yhi = fabsf(rb) + hb[b];
                // row r of the cell's hyperbolic grid
                const float u1hi = xhi * yhi;
                const float llo = logf(fmaxf(xlo * ylo, eps * u1hi));
                const float ds = (logf(u1hi) - llo) / (float)G;
                const float u1 = expf(fmaf((float)r + 0.5f, ds, llo));
                const float ymin = fmaxf(ylo, u1 / xhi), ymax = fminf(yhi, u1 / xlo);
                if (!(ymax > ymin)) continue;
                const float du2 = log1pf((ymax - ymin) / ymin) / (float)G;
                const float yc = sqrtf(ymin * ymax), xc = u1 / yc;
                const float w = u1 * ds * du2 * mult;
                const float Wab = pd[a] * pd[b];
                const float4 *Q = sQ + (size_t)cc * M;
                for (int j = 0; j < G; ++j) {
                    const float d = ((float)j + 0.5f - 0.5f * (float)G) * du2;
                    const float ex = expf(d);
                    const float f1 = s1 * (xc * ex), f2 = s2 * (yc * __frcp_rn(ex));
                    const float u = f1 + f2;
                    const int c = channel_of(rel, hb, n, u);
                    if (c < 0) continue;
                    const float W = Wab * pd[c];
                    if (W == 0.0f) continue;
                    const float da = f1 - ra, db = f2 - rb, dc = u - rel[c];
                    const float br = b2 + c3 * (u + 2.0f * fi) +
                                     c4 * (f1 * f1 + 1.5f * f1 * f2 + 3.0f * fi * u + f2 * f2 + three_fi2);
                    const float phi = m4pi2 * f1 * f2 * br;
                    const float aphi = fabsf(phi);
                    const float2 *Tc = T + (size_t)c * M;
                    float S2;
                    if (aphi <= phi_small) S2 = zsum_small_mt(phi, da, db, dc, Q, Tc, sA, M);
                    else if (aphi <= phi_direct) S2 = zsum_direct_mt(phi, da, db, dc, Q, Tc, sA, M);
                    else S2 = zsum_tele_mt(phi, da, db, dc, Q, Tc, sB, M);
                    const float y = w * W * S2 * array_factor_f(phi, qp) - comp;
                    const float t = sum + y;
                    comp = (t - sum) - y;
                    sum = t;
                }
            }
        }
        const double tot = block_sum_d((double)sum - (double)comp, scratch);
        if (threadIdx.x == 0) qp.partial[it] = tot;
    }
}

// Plain FP64 reference kernel: every step reads the profile rows of a, b, c
// and the CUT from the FP64 tables; the z-sum as written (Eq. slow_vary).
__global__ void __launch_bounds__(256) k_quad_mci_f64_tab(QuadParams qp)
{
    extern __shared__ double2 smem_d2[];
    const int M = qp.n_steps, G = qp.G;
    double2 *sz = smem_d2;                 // [M] {z_m, dz_m}
    double *sti = reinterpret_cast<double *>(sz + M);   // [M] a_i(m) of the item's CUT
    __shared__ double scratch[32];
    __shared__ int s_item;

    for (int m = threadIdx.x; m < M; m += blockDim.x) sz[m] = qp.zs_d[m];
    const double c3 = kPi * qp.beta3;
    const double c4 = 2.0 * kPi * kPi / 3.0 * qp.beta4;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(qp.counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= qp.n_items) break;
        const DevItem item = qp.items[it];
        const int plan = qp.prof_plan[item.prof];
        const int coff = qp.plan_ch_off[plan];
        const int poff = qp.prof_ch_off[item.prof];
        const int n = qp.plan_n[plan];
        const int i = item.cut;
        const double2 *T = qp.ab + (size_t)poff * M;
        for (int m = threadIdx.x; m < M; m += blockDim.x) sti[m] = T[(size_t)i * M + m].x;
        __syncthreads();
        const double *fr = qp.ch_frel + coff;
        const double *Bc = qp.ch_B + coff;
        const double *pdv = qp.pd_d + poff;
        const double fi = fr[i];
        const int n2 = n - 1;
        double sum = 0.0;
        const int nrows = (item.piece1 - item.piece0) * G;
        for (int q = threadIdx.x; q < nrows; q += blockDim.x) {
            const int tl = q / G, r = q - tl * G;
            int ap, bp;
            tri_decode(item.piece0 + tl, n2, ap, bp);
            const int a = dbg_clamp(ap + (ap >= i), n, kDbgCell, qp.dbg), b = dbg_clamp(bp + (bp >= i), n, kDbgCell, qp.dbg);
            const double mult = a == b ? 1.0 : 2.0;
            const double ra = fr[a] - fi, rb = fr[b] - fi;
            const double s1 = ra > 0.0 ? 1.0 : -1.0, s2 = rb > 0.0 ? 1.0 : -1.0;
            const double xlo = fabs(ra) - 0.5 * Bc[a], xhi = fabs(ra) + 0.5 * Bc[a];
            const double ylo = fabs(rb) - 0.5 * Bc[b], yhi = fabs(rb) + 0.5 * Bc[b];
            const double u1hi = xhi * yhi;
            const double llo = log(fmax(xlo * ylo, qp.eps_v1 * u1hi));
            const double ds = (log(u1hi) - llo) / G;
            const double u1 = exp(llo + (r + 0.5) * ds);
            const double ymin = fmax(ylo, u1 / xhi), ymax = fmin(yhi, u1 / xlo);
            if (!(ymax > ymin)) continue;
            const double du2 = log1p((ymax - ymin) / ymin) / G;
            const double yc = sqrt(ymin * ymax), xc = u1 / yc;
            const double w = u1 * ds * du2 * mult;
            const double2 *Ta = T + (size_t)a * M, *Tb = T + (size_t)b * M;
            for (int j = 0; j < G; ++j) {
                const double d = ((double)j + 0.5 - 0.5 * (double)G) * du2;
                const double f1 = s1 * (xc * exp(d)), f2 = s2 * (yc * exp(-d));
                const double u = f1 + f2;
                // channel of F_c = f_i + u
                int lo = 0, hi = n - 1, c = -1;
                while (lo <= hi) {
                    const int mid = (lo + hi) >> 1;
                    if (fr[mid] - fi - 0.5 * Bc[mid] <= u) {
                        c = mid;
                        lo = mid + 1;
                    } else {
                        hi = mid - 1;
                    }
                }
                if (c < 0 || !(u < fr[c] - fi + 0.5 * Bc[c])) continue;
                const double W = pdv[a] * pdv[b] * pdv[c];
                if (W == 0.0) continue;
                const double da = f1 - ra, db = f2 - rb, dc = u - (fr[c] - fi);
                const double br = qp.beta2 + c3 * (u + 2.0 * fi) +
                                  c4 * (f1 * f1 + 1.5 * f1 * f2 + 3.0 * fi * u + f2 * f2 + 3.0 * fi * fi);
                const double phi = -4.0 * kPi * kPi * f1 * f2 * br;
                const double2 *Tc = T + (size_t)c * M;
                double Sr = 0.0, Si = 0.0;
                for (int m = 0; m < M; ++m) {
                    const double2 zz = sz[m];
                    const double2 ta = Ta[m], tb = Tb[m], tc = Tc[m];
                    const double p = exp(0.5 * (ta.x + tb.x + tc.x - sti[m] + ta.y * da + tb.y * db + tc.y * dc));
                    const double amp = p * zz.y * sinc_d(0.5 * phi * zz.y);
                    double sn, cs;
                    sincos(phi * zz.x, &sn, &cs);
                    Sr += amp * cs;
                    Si += amp * sn;
                }
                sum += w * W * (Sr * Sr + Si * Si) * array_factor_d(phi, qp);
            }
        }
        const double tot = block_sum_d(sum, scratch);
        if (threadIdx.x == 0) qp.partial[it] = tot;
    }
}

size_t quad_mci_tab_smem_bytes(int precision, int n_steps, int n_max, int cpc)
{
    if (precision == 0)
        return (size_t)n_steps * (2 + cpc) * sizeof(float4) + (size_t)n_max * 3 * sizeof(float);
    return (size_t)n_steps * (sizeof(double2) + sizeof(double));
}

int quad_mci_tab_cells(int n_steps, int n_max, int G, int block)
{
    const size_t fixed = (size_t)n_steps * 2 * sizeof(float4) + (size_t)n_max * 3 * sizeof(float);
    const size_t budget = 200 * 1024;
    if (fixed >= budget) return 0;
    const int by_mem = (int)((budget - fixed) / ((size_t)n_steps * sizeof(float4)));
    return std::min(std::min(kMciTabCells, block / std::max(1, G)), by_mem);
}

static void *mci_tab_fn(int precision)
{
    return precision == 0 ? (void *)k_quad_mci_f32_tab : (void *)k_quad_mci_f64_tab;
}

int quad_mci_tab_blocks_per_sm(int precision, int n_steps, int n_max, int cpc, int block)
{
    int nb = 0;
    const size_t smem = quad_mci_tab_smem_bytes(precision, n_steps, n_max, cpc);
    void *fn = mci_tab_fn(precision);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, smem);
    return nb > 0 ? nb : 1;
}

cudaError_t launch_tab_half_log2(const double2 *ab, float2 *abf, int n, int n_sms, cudaStream_t st)
{
    const int grid = std::max(1, std::min((n + 255) / 256, 4 * n_sms));
    k_tab_half_log2<<<grid, 256, 0, st>>>(ab, abf, n);
    return cudaGetLastError();
}

cudaError_t launch_quad_mci_tab(const QuadParams &qp, int precision, int grid, int block, cudaStream_t st)
{
    const size_t smem = quad_mci_tab_smem_bytes(precision, qp.n_steps, qp.mci_n_max, qp.mci_cpc);
    void *fn = mci_tab_fn(precision);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    QuadParams q = qp;
    void *args[] = {&q};
    return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, st);
}

}  // namespace isrs
