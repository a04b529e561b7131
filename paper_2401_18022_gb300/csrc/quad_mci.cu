// Multi-channel-interference (MCI) cells of the ISRS GN integral (App. A:
// the frequency integral of Eq. gain_fin runs over the whole band, so besides
// the CUT's own row and column of channel-pair cells (SCI, XCI) it contains
// every cell (a, b) with neither F_a nor F_b in the CUT's channel).
//
// For N channels there are (N-1) N / 2 such cells per CUT after folding the
// mirror cell (b, a) onto (a, b) (the integrand is symmetric in f1, f2), so
// no piece list is built: a work item is a range of cells of one CUT in the
// triangular order of the pairs (a', b'), a' <= b', of the N - 1 channels
// other than the CUT (a = a' + [a' >= i], likewise b), and every thread
// decodes its cell and grid row from its index.  Each cell lies in one
// quadrant (channel a does not straddle f_i) and gets its own G_mci x G_mci
// hyperbolic grid: rows uniform in ln(upsilon1), columns uniform in upsilon2,
// exactly as the per-piece grids of the SCI/XCI cells.  The z-sum and the
// closed-form profile are those of k_quad_f32 / k_quad_f64; far cells reach
// phases of ~1e8 revolutions, so the FP32 kernel's telescoped form uses the
// wide phase reduction.
#include <cuda_runtime.h>

#include "isrs_internal.cuh"
#include "isrs_kernels.h"
#include "quad_common.cuh"
#include "quad_zsum.cuh"
#include "quad_cells.cuh"

namespace isrs {

__global__ void __launch_bounds__(256, 4) k_quad_mci_f32(QuadParams qp)
{
    extern __shared__ float4 smem_f4[];
    const int M = qp.n_steps, G = qp.G;
    float4 *sT = smem_f4;                              // [M] {A2 + log2 dz, K2, z, z^2 + dz^2/12}
    float4 *sE = sT + M;                               // [M] {edge/2pi hi, lo, A2, K2}
    float4 *sR = sE + M;                               // [M] {A2 + log2 dz, K2, z, dz}
    float *rel = reinterpret_cast<float *>(sR + M);    // [n] channel centre - f_i
    float *hb = rel + qp.mci_n_max;                    // [n] B/2
    float *pd = hb + qp.mci_n_max;                     // [n] P/B
    float *ha = pd + qp.mci_n_max;                     // [n] alpha/2 log2 e
    __shared__ double scratch[32];
    __shared__ int s_item;

    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const float4 za = qp.zs_a[m];
        const float4 zb = qp.zs_b[m];
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
        }
        if (item.prof != cur_prof || i != cur_cut) {
            const double fi = qp.ch_frel[coff + i];
            for (int c = threadIdx.x; c < n; c += blockDim.x) {
                rel[c] = (float)(qp.ch_frel[coff + c] - fi);
                hb[c] = (float)(0.5 * qp.ch_B[coff + c]);
                pd[c] = qp.pd_f[poff + c];
                ha[c] = (float)(0.5 * qp.ch_alpha[coff + c] * kLog2e);
            }
            cur_prof = item.prof;
            cur_cut = i;
        }
        __syncthreads();
        const float fi = (float)qp.ch_frel[coff + i];
        const float three_fi2 = 3.0f * fi * fi;
        const float ha_i = ha[i];
        const int n2 = n - 1;
        float sum = 0.0f, comp = 0.0f;
        const int nrows = (item.piece1 - item.piece0) * G;
        for (int q = threadIdx.x; q < nrows; q += blockDim.x) {
            const int tl = q / G, r = q - tl * G;
            int ap, bp;
            tri_decode(item.piece0 + tl, n2, ap, bp);
            const int a = dbg_clamp(ap + (ap >= i), n, kDbgCell, qp.dbg), b = dbg_clamp(bp + (bp >= i), n, kDbgCell, qp.dbg);
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
            const float at_ab = ha[a] + ha[b] - ha_i;
            for (int j = 0; j < G; ++j) {
                const float d = ((float)j + 0.5f - 0.5f * (float)G) * du2;
                const float e = expf(d);
                const float f1 = s1 * (xc * e), f2 = s2 * (yc * __frcp_rn(e));
                const float u = f1 + f2;
                const int c = channel_of(rel, hb, n, u);
                if (c < 0) continue;
                const float W = Wab * pd[c];
                if (W == 0.0f) continue;
                const float at = at_ab + ha[c];
                const float Fc = fi + u;
                const float br = b2 + c3 * (u + 2.0f * fi) +
                                 c4 * (f1 * f1 + 1.5f * f1 * f2 + 3.0f * fi * u + f2 * f2 + three_fi2);
                const float phi = m4pi2 * f1 * f2 * br;
                const float aphi = fabsf(phi);
                float S2;
                if (aphi <= phi_small) S2 = zsum_small_f(phi, Fc, at, sT, M);
                else if (aphi <= phi_direct) S2 = zsum_direct_f(phi, Fc, at, sR, M);
                else S2 = zsum_tele_wide_f(phi, Fc, at, sT, sE, M);
                const float y = w * W * S2 * array_factor_f(phi, qp) - comp;
                const float t = sum + y;
                comp = (t - sum) - y;
                sum = t;
            }
        }
        const double tot = block_sum_d((double)sum - (double)comp, scratch);
        if (threadIdx.x == 0) qp.partial[it] = tot;
    }
}

__global__ void __launch_bounds__(256) k_quad_mci_f64(QuadParams qp)
{
    extern __shared__ double2 smem_d2[];
    const int M = qp.n_steps, G = qp.G;
    double2 *sz = smem_d2;                 // [M] {z_m, dz_m}
    double2 *st = sz + M;                  // [M] {lnPtot - lnN, kappa}
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
        __syncthreads();
        const int plan = qp.prof_plan[item.prof];
        const int coff = qp.plan_ch_off[plan];
        const int poff = qp.prof_ch_off[item.prof];
        const int n = qp.plan_n[plan];
        const int i = item.cut;
        const double *fr = qp.ch_frel + coff;
        const double *Bc = qp.ch_B + coff;
        const double *al = qp.ch_alpha + coff;
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
                const double at = 0.5 * (al[a] + al[b] + al[c] - al[i]);
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
                sum += w * W * (Sr * Sr + Si * Si) * array_factor_d(phi, qp);
            }
        }
        const double tot = block_sum_d(sum, scratch);
        if (threadIdx.x == 0) qp.partial[it] = tot;
    }
}

size_t quad_mci_smem_bytes(int precision, int n_steps, int n_max)
{
    if (precision == 0) return (size_t)n_steps * 3 * sizeof(float4) + (size_t)n_max * 4 * sizeof(float);
    return (size_t)n_steps * 2 * sizeof(double2);
}

int quad_mci_blocks_per_sm(int precision, int n_steps, int n_max, int block)
{
    int nb = 0;
    const size_t smem = quad_mci_smem_bytes(precision, n_steps, n_max);
    void *fn = precision == 0 ? (void *)k_quad_mci_f32 : (void *)k_quad_mci_f64;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, smem);
    return nb > 0 ? nb : 1;
}

cudaError_t launch_quad_mci(const QuadParams &qp, int precision, int grid, int block, cudaStream_t st)
{
    const size_t smem = quad_mci_smem_bytes(precision, qp.n_steps, qp.mci_n_max);
    void *fn = precision == 0 ? (void *)k_quad_mci_f32 : (void *)k_quad_mci_f64;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    QuadParams q = qp;
    void *args[] = {&q};
    return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, st);
}

}  // namespace isrs
