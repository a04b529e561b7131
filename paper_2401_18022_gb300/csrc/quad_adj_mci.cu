// Adjoint over the multi-channel-interference (MCI) cells on their own grid
// (App. A: the frequency integral of Eq. gain_fin over the whole band; the
// cells (a, b) with neither F_a nor F_b in the CUT's channel, each on a
// G_mci x G_mci hyperbolic grid as in the MCI quadrature).  With the
// closed-form profile it fills, for its work items, the same quantities as
// the fused adjoint of the SCI/XCI pieces:
//   R_im  = sum_points w W d|S|^2/d ln p_m,   R'_im = same * (F_c - f_ref),
//   V_ij += w W |S|^2 for each of the point's channels a, b, c,
// and the forward partial of each item, so the chain rule (k_chain_*) takes the
// MCI items as further tiles of their CUTs.
//
// A warp takes 32 grid points of its item (cell, row, column decoded from the
// point index; the row set-up is per point), appends them to one list per
// z-sum form and walks the lists two at a time on half-warps (quad_walk.cuh):
// each of the 16 lanes owns K = ceil(M/16) steps, every step term is
// evaluated once and reused for the bucket terms.  Far cells reach phases of
// ~1e8 revolutions, so the telescoped walk uses the wide phase reduction.
// The PSD buckets of an item go to one shared row per warp over the plan's
// channels (the two halves' owner lanes add in turn, so the order is fixed),
// summed over the warps in order and added to V with one FP64 atomic per
// channel.
#include <cuda_runtime.h>

#include "isrs_internal.cuh"
#include "isrs_kernels.h"
#include "quad_cells.cuh"
#include "quad_common.cuh"
#include "quad_walk.cuh"

namespace isrs {

namespace {

constexpr int kClsSmallM = 0, kClsDirectM = 1, kClsTeleM = 2;
constexpr int kListCapM = 34;      // a form's list: one carried point + 32 new (+1 pad)
constexpr int kFoldBatchesM = 256;   // batches between FP64 folds of the register buckets
constexpr float kPadLog2M = -1000.0f;

// PSD buckets of a walked pair: lane 0 (the first half's point) adds to the
// warp's row, then lane 16 (the second half's); a point adds to each of its
// channels a, b, c (a channel counted as often as it occurs).
__device__ __forceinline__ void v_add(float *row, int4 abc, float val, int lane)
{
    if (lane == 0) {
        row[abc.x] += val;
        row[abc.y] += val;
        row[abc.z] += val;
    }
    __syncwarp();
    if (lane == 16) {
        row[abc.x] += val;
        row[abc.y] += val;
        row[abc.z] += val;
    }
    __syncwarp();
}

}  // namespace

#ifndef ISRS_ADJ_MCI_MIN_BLOCKS
#define ISRS_ADJ_MCI_MIN_BLOCKS 3   // resident blocks per SM the register budget is sized for
#endif

template <int K>
__global__ void __launch_bounds__(256, ISRS_ADJ_MCI_MIN_BLOCKS) k_quad_adj_mci(AdjParams ap)
{
    const QuadParams &qp = ap.q;
    extern __shared__ float4 smem_f4[];
    const int M = qp.n_steps, G = qp.G;
    const int G2 = G * G;
    const int nw = blockDim.x >> 5;
    const int nmax = qp.mci_n_max;
    float4 *sO0 = smem_f4;                                    // [K][16] owned {A2 + log2 dz, K2, z, dz}
    float4 *sO1 = sO0 + K * 16;                               // [K][16] owned {edge/2pi hi, lo, A2, c}
    float4 *sL = sO1 + K * 16;                                // [nw][3][kListCapM] {w W af, phi, F_c, at}
    int4 *sLi = reinterpret_cast<int4 *>(sL + nw * 3 * kListCapM);        // [nw][3][kListCapM] {a, b, c, -}
    double2 *sB = reinterpret_cast<double2 *>(sLi + nw * 3 * kListCapM);  // [nw][K][16] FP64 step buckets
    float *rel = reinterpret_cast<float *>(sB + nw * K * 16);             // [nmax] channel centre - f_i
    float *hb = rel + nmax;                                               // [nmax] B/2
    float *pd = hb + nmax;                                                // [nmax] P/B
    float *ha = pd + nmax;                                                // [nmax] alpha/2 log2 e
    float *sV = ha + nmax;                                                // [nw][nmax] PSD buckets of the item
    __shared__ double scratch[32];
    __shared__ int s_item;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int l16 = lane & 15, half = lane >> 4;
    for (int t = threadIdx.x; t < nw * K * 16; t += blockDim.x) sB[t] = make_double2(0.0, 0.0);

    const float c3 = (float)(kPi * qp.beta3);
    const float c4 = (float)(2.0 * kPi * kPi / 3.0 * qp.beta4);
    const float b2 = (float)qp.beta2;
    const float m4pi2 = (float)(-4.0 * kPi * kPi);
    const float phi_direct = 3.14159265f / qp.dz_max;
    const float phi_small = 0.02f / qp.L;
    const float eps = (float)qp.eps_v1;
    const float4 *o0s = sO0 + l16;
    const float4 *o1s = sO1 + l16;
    float4 *Ls = sL + warp * 3 * kListCapM;
    float4 *Ld = Ls + kListCapM;
    float4 *Lt = Ld + kListCapM;
    int4 *Is = sLi + warp * 3 * kListCapM;
    int4 *Id = Is + kListCapM;
    int4 *It = Id + kListCapM;
    double2 *myB = sB + warp * K * 16;
    const unsigned lt_mask = (1u << lane) - 1u;
    unsigned n_small = 0, n_direct = 0, n_tele = 0;
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
            // lane-contiguous owned step tables; padding steps repeat the last edge
            const float2 *st = qp.step_f + (size_t)item.prof * M;
            const float4 zl = qp.zs_b[M - 1];
            for (int t = threadIdx.x; t < K * 16; t += blockDim.x) {
                const int k = t >> 4, l = t & 15, m = l * K + k;
                float4 o0 = make_float4(kPadLog2M, 0.f, 0.f, 0.f);
                float4 o1 = make_float4(zl.x, zl.y, kPadLog2M, 0.f);
                if (m < M) {
                    const float2 v = st[m];
                    const float4 za = qp.zs_a[m];
                    const float4 zb = qp.zs_b[m];
                    o0 = make_float4(v.x + za.z, v.y, za.x, za.w);
                    o1 = make_float4(zb.x, zb.y, v.x, za.y);
                }
                sO0[k * 16 + l] = o0;
                sO1[k * 16 + l] = o1;
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
        for (int t = threadIdx.x; t < nw * nmax; t += blockDim.x) sV[t] = 0.0f;
        __syncthreads();
        float *myV = sV + warp * nmax;
        const float fi = (float)qp.ch_frel[coff + i];
        const float three_fi2 = 3.0f * fi * fi;
        const float ha_i = ha[i];
        const int n2 = n - 1;
        float sum = 0.0f, comp = 0.0f;
        float R[K], Rp[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            R[k] = 0.0f;
            Rp[k] = 0.0f;
        }
        int ns = 0, nd = 0, nt = 0;         // list lengths (warp-uniform)
        int batches = 0;
        const int npts = (item.piece1 - item.piece0) * G2;
        for (int qb = warp * 32; qb < npts; qb += blockDim.x) {
            // ---- 1. this lane's grid point: cell, row and column from its index
            const int q = qb + lane;
            float phi = 0.0f, Fc = 0.0f, at = 0.0f, wwa = 0.0f;
            int cls = -1, a = 0, b = 0, c = -1;
            if (q < npts) {
                const int tl = q / G2, rem = q - tl * G2;
                const int r = rem / G, j = rem - r * G;
                int ap_, bp_;
                tri_decode(item.piece0 + tl, n2, ap_, bp_);
                a = dbg_clamp(ap_ + (ap_ >= i), n, kDbgCell, qp.dbg);
                b = dbg_clamp(bp_ + (bp_ >= i), n, kDbgCell, qp.dbg);
                const float mult = a == b ? 1.0f : 2.0f;
                const float ra = rel[a], rb = rel[b];
                const float s1 = ra > 0.0f ? 1.0f : -1.0f, s2 = rb > 0.0f ? 1.0f : -1.0f;
                const float xlo = fabsf(ra) - hb[a], xhi = fabsf(ra) + hb[a];
                const float ylo = fabsf(rb) - hb[b], yhi = fabsf(rb) + hb[b];
                const float u1hi = xhi * yhi;
                const float llo = logf(fmaxf(xlo * ylo, eps * u1hi));
                const float ds = (logf(u1hi) - llo) / (float)G;
                const float u1 = expf(fmaf((float)r + 0.5f, ds, llo));
                const float ymin = fmaxf(ylo, u1 / xhi), ymax = fminf(yhi, u1 / xlo);
                if (ymax > ymin) {
                    const float du2 = log1pf((ymax - ymin) / ymin) / (float)G;
                    const float yc = sqrtf(ymin * ymax), xc = u1 / yc;
                    const float w = u1 * ds * du2 * mult;
                    const float d = ((float)j + 0.5f - 0.5f * (float)G) * du2;
                    const float e = expf(d);
                    const float f1 = s1 * (xc * e), f2 = s2 * (yc * __frcp_rn(e));
                    const float u = f1 + f2;
                    c = channel_of(rel, hb, n, u);
                    if (c >= 0) {
                        const float W = pd[a] * pd[b] * pd[c];
                        if (W != 0.0f) {
                            at = ha[a] + ha[b] - ha_i + ha[c];
                            Fc = fi + u;
                            const float br = b2 + c3 * (u + 2.0f * fi) +
                                             c4 * (f1 * f1 + 1.5f * f1 * f2 + 3.0f * fi * u + f2 * f2 + three_fi2);
                            phi = m4pi2 * f1 * f2 * br;
                            const float aphi = fabsf(phi);
                            wwa = w * W * array_factor_f(phi, qp);
                            cls = aphi <= phi_small ? kClsSmallM : (aphi <= phi_direct ? kClsDirectM : kClsTeleM);
                        }
                    }
                }
            }
            // append to the form's list
            const unsigned bs = __ballot_sync(kWarpAll, cls == kClsSmallM);
            const unsigned bd = __ballot_sync(kWarpAll, cls == kClsDirectM);
            const unsigned bt = __ballot_sync(kWarpAll, cls == kClsTeleM);
            if (cls >= 0) {
                const float4 v = make_float4(wwa, phi, Fc, at);
                const int4 abc = make_int4(a, b, c, 0);
                int pos;
                if (cls == kClsSmallM) {
                    pos = ns + __popc(bs & lt_mask);
                    Ls[pos] = v;
                    Is[pos] = abc;
                } else if (cls == kClsDirectM) {
                    pos = nd + __popc(bd & lt_mask);
                    Ld[pos] = v;
                    Id[pos] = abc;
                } else {
                    pos = nt + __popc(bt & lt_mask);
                    Lt[pos] = v;
                    It[pos] = abc;
                }
            }
            if (lane == 0) {
                n_small += __popc(bs);
                n_direct += __popc(bd);
                n_tele += __popc(bt);
            }
            ns += __popc(bs);
            nd += __popc(bd);
            nt += __popc(bt);
            __syncwarp();
            // ---- 2. walk the lists in pairs, one point per half-warp
            for (int p = half; p + 1 - half < nd; p += 2) {
                const float4 st = Ld[p];
                const float val = walk_direct<K>(o0s, st.x, st.y, st.z, st.w, 1.0f, R, Rp);
                const float vv = l16 == 0 ? val : 0.0f;
                const float y = vv - comp, t = sum + y;
                comp = (t - sum) - y;
                sum = t;
                const int4 abc = Id[p];
                v_add(myV, abc, val, lane);
            }
            for (int p = half; p + 1 - half < nt; p += 2) {
                const float4 st = Lt[p];
                const float val = walk_tele<K, true>(o0s, o1s, l16, st.x, st.y, st.z, st.w, 1.0f, R, Rp);
                const float vv = l16 == 0 ? val : 0.0f;
                const float y = vv - comp, t = sum + y;
                comp = (t - sum) - y;
                sum = t;
                const int4 abc = It[p];
                v_add(myV, abc, val, lane);
            }
            for (int p = half; p + 1 - half < ns; p += 2) {
                const float4 st = Ls[p];
                const float val = walk_small<K>(o0s, o1s, st.x, st.y, st.z, st.w, 1.0f, R, Rp);
                const float vv = l16 == 0 ? val : 0.0f;
                const float y = vv - comp, t = sum + y;
                comp = (t - sum) - y;
                sum = t;
                const int4 abc = Is[p];
                v_add(myV, abc, val, lane);
            }
            // an odd point waits at the head of its list for the next batch
            __syncwarp();
            if (lane == 0) {
                if (nd & 1) {
                    Ld[0] = Ld[nd - 1];
                    Id[0] = Id[nd - 1];
                }
                if (nt & 1) {
                    Lt[0] = Lt[nt - 1];
                    It[0] = It[nt - 1];
                }
                if (ns & 1) {
                    Ls[0] = Ls[ns - 1];
                    Is[0] = Is[ns - 1];
                }
            }
            nd &= 1;
            nt &= 1;
            ns &= 1;
            if (++batches == kFoldBatchesM) {
                batches = 0;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const float rx = R[k] + __shfl_xor_sync(kWarpAll, R[k], 16);
                    const float ry = Rp[k] + __shfl_xor_sync(kWarpAll, Rp[k], 16);
                    if (half == 0) {
                        double2 &dd = myB[k * 16 + l16];
                        dd.x += (double)rx;
                        dd.y += (double)ry;
                    }
                    R[k] = 0.0f;
                    Rp[k] = 0.0f;
                }
            }
            __syncwarp();          // the next batch appends to the lists
        }
        // the last odd point of each form, beside a zero-weight copy of itself
        if (nd) {
            float4 st = Ld[0];
            if (half) st.x = 0.0f;
            const float val = walk_direct<K>(o0s, st.x, st.y, st.z, st.w, 1.0f, R, Rp);
            const float vv = l16 == 0 ? val : 0.0f;
            const float y = vv - comp, t = sum + y;
            comp = (t - sum) - y;
            sum = t;
            v_add(myV, Id[0], val, lane);
        }
        if (nt) {
            float4 st = Lt[0];
            if (half) st.x = 0.0f;
            const float val = walk_tele<K, true>(o0s, o1s, l16, st.x, st.y, st.z, st.w, 1.0f, R, Rp);
            const float vv = l16 == 0 ? val : 0.0f;
            const float y = vv - comp, t = sum + y;
            comp = (t - sum) - y;
            sum = t;
            v_add(myV, It[0], val, lane);
        }
        if (ns) {
            float4 st = Ls[0];
            if (half) st.x = 0.0f;
            const float val = walk_small<K>(o0s, o1s, st.x, st.y, st.z, st.w, 1.0f, R, Rp);
            const float vv = l16 == 0 ? val : 0.0f;
            const float y = vv - comp, t = sum + y;
            comp = (t - sum) - y;
            sum = t;
            v_add(myV, Is[0], val, lane);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float rx = R[k] + __shfl_xor_sync(kWarpAll, R[k], 16);
            const float ry = Rp[k] + __shfl_xor_sync(kWarpAll, Rp[k], 16);
            if (half == 0) {
                double2 &dd = myB[k * 16 + l16];
                dd.x += (double)rx;
                dd.y += (double)ry;
            }
        }
        // item outputs: the forward partial, the PSD buckets and the step buckets
        const double tot = block_sum_d((double)sum - (double)comp, scratch);   // syncs the block
        if (threadIdx.x == 0) qp.partial[it] = tot;
        double *Vrow = ap.V + (size_t)it * ap.n_ch;     // this tile's own row (k_v_reduce sums them)
        for (int c = threadIdx.x; c < n; c += blockDim.x) {
            double v = 0.0;
            for (int w = 0; w < nw; ++w) v += (double)sV[w * nmax + c];
            Vrow[c] = v;
        }
        for (int m = threadIdx.x; m < M; m += blockDim.x) {
            const int ln = m / K, kk = m - ln * K;
            double rx = 0.0, ry = 0.0;
            for (int w = 0; w < nw; ++w) {
                double2 &bb = sB[(w * K + kk) * 16 + ln];
                rx += bb.x;
                ry += bb.y;
                bb = make_double2(0.0, 0.0);
            }
            ap.item_R[(size_t)it * M + m] = make_double2(rx, ry);
        }
    }
    if (qp.path_count && lane == 0) {
        atomicAdd(&qp.path_count[0], (unsigned long long)n_small);
        atomicAdd(&qp.path_count[1], (unsigned long long)n_direct);
        atomicAdd(&qp.path_count[2], (unsigned long long)n_tele);
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
size_t adjoint_mci_smem_bytes(int n_steps, int n_max, int block)
{
    const int K = (n_steps + 15) / 16, nw = block / 32;
    return (size_t)(2 * K * 16 + nw * 3 * kListCapM) * sizeof(float4) + (size_t)nw * 3 * kListCapM * sizeof(int4) +
           (size_t)nw * K * 16 * sizeof(double2) + (size_t)(4 + nw) * n_max * sizeof(float);
}

namespace {

template <int K>
void *adj_mci_fn()
{
    return (void *)k_quad_adj_mci<K>;
}

void *adj_mci_kernel_for(int n_steps)
{
    switch ((n_steps + 15) / 16) {
    case 1: return adj_mci_fn<1>();
    case 2: return adj_mci_fn<2>();
    case 3: return adj_mci_fn<3>();
    case 4: return adj_mci_fn<4>();
    case 5: return adj_mci_fn<5>();
    case 6: return adj_mci_fn<6>();
    case 7: return adj_mci_fn<7>();
    case 8: return adj_mci_fn<8>();
    }
    return nullptr;
}

}  // namespace

int adjoint_mci_blocks_per_sm(int n_steps, int n_max, int block)
{
    void *fn = adj_mci_kernel_for(n_steps);
    if (!fn) return 0;
    const size_t smem = adjoint_mci_smem_bytes(n_steps, n_max, block);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, smem);
    return nb > 0 ? nb : 1;
}

cudaError_t launch_adjoint_mci(const AdjParams &ap, int grid, int block, cudaStream_t st)
{
    void *fn = adj_mci_kernel_for(ap.q.n_steps);
    if (!fn) return cudaErrorInvalidValue;
    const size_t smem = adjoint_mci_smem_bytes(ap.q.n_steps, ap.q.mci_n_max, block);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    AdjParams a = ap;
    void *args[] = {&a};
    return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, st);
}

}  // namespace isrs
