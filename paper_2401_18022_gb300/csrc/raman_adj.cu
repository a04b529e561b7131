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
// FP64 shared buckets once per piece.  The same pass sums the forward value
// w W |S|^2 (the tile's partial of Sigma_i), so no separate forward runs.
// The buckets are not yet weighted by dT/dSigma_i (unknown until every tile
// of CUT i is done): at the end of a candidate the block adds them, in
// order, into the rows of its own tile (one row per plan channel the tile
// touches, owned by this block alone), and k_tab_gather applies
// dT/dSigma_i and sums each channel's rows in tile order.  No atomics: the
// gradient is reproducible bit for bit.
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
// Batches between folds of the FP32 lane buckets into the FP64 shared ones:
// one per piece at G = 256.  A lane bucket then sums at most ~512 terms in
// FP32 (relative rounding ~1e-6, at worst ~3e-5, against the gradient's 1e-3),
// and the FP64 pipe, ~1/64 of the FP32 rate on this GPU, stays nearly idle.
constexpr int kFoldBatchesT = 256;

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

// ---------------------------------------------------------------------------
// Contracted small phase (|phi| L <= 2) with the tabulated profile.  As in
// the forward (raman.cu), S of a point in candidate c follows from 11 moments
// about the span centre, nu_n(x, y) = sum_{k,l<=3} C_nkl T_k(x) T_l(y), with
// x = da / h_a, y = db / h_b the offsets inside channels a and b.  Its bucket
// terms d|S|^2/d ln p_m = w_m(x, y) sum_n fold_n g_n(m) al_n, al_n = 2 (A|B)
// phi^n (A even, B odd orders), need w_m(x, y) = base_m e^{alpha_m x + beta_m y}
// at the point; expanded to total degree 3 in (x, y) (|alpha|, |beta| <= 0.05:
// truncation below (0.1)^4/4! = 4e-6 of the term), the buckets of a batch are
// sums of cp al_n x^i y^j over its points, i + j <= 4 (the R_a, R_b buckets
// carry one more power of x or y): 15 monomials per order, n <= 5 for a batch
// whose phases are all |phi| L <= 0.2 (90 values, three warp butterflies),
// n <= 10 otherwise (165 values, six).  The buckets of every step follow once
// per candidate.
// ---------------------------------------------------------------------------
constexpr int kTabMom = 11;                       // nu_0 .. nu_10
constexpr int kTabMono = 15;                      // x^i y^j, i + j <= 4
constexpr int kTabShortN = 6 * kTabMono;          // n <= 5
constexpr int kTabCtrN = kTabMom * kTabMono;      // n <= 10
constexpr int kTabCtrS = 192;                     // slots (six butterflies)
constexpr float kTabShortPhiL = 0.2f;

// position of x^i y^j in the monomial list: by total degree, then by j
__host__ __device__ constexpr int mono_idx(int i, int j) { return (i + j) * (i + j + 1) / 2 + j; }

// The forward's contracted coefficients of one candidate (its table rows Q):
// C[n][k][l] = fold_n sum_m base_m b_k(alpha_m) b_l(beta_m) g_n(m), stored as
// sCc[n * 4 + k] = float4 over l.  sW: [M][4] float4 scratch.  Every thread
// calls; the block is synchronised on return.
__device__ void tab_adj_coeffs(const QuadParams &qp, const float4 *Q, float ha, float hb, float4 *sW, float4 *sCc)
{
    const int M = qp.n_steps;
    const float ln2 = 0.69314718f;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const float4 q = Q[m];
        const float base = ex2_approx(q.x);
        const float4 bk = bessel_b4(q.y * ha * ln2), bl = bessel_b4(q.z * hb * ln2);
        const float bkv[4] = {bk.x, bk.y, bk.z, bk.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float wk = base * bkv[k];
            sW[m * 4 + k] = make_float4(wk * bl.x, wk * bl.y, wk * bl.z, wk * bl.w);
        }
    }
    __syncthreads();
    const float *g = reinterpret_cast<const float *>(qp.zs_g);   // kZsG float4 = 20 floats per step
    for (int t = threadIdx.x; t < kTabMom * 16; t += blockDim.x) {
        const int n = t >> 4, k = (t >> 2) & 3, l = t & 3;
        float sum = 0.0f, comp = 0.0f;
        for (int m = 0; m < M; ++m) {
            const float4 w = sW[m * 4 + k];
            const float wl = l == 0 ? w.x : (l == 1 ? w.y : (l == 2 ? w.z : w.w));
            const float y = wl * g[m * 4 * kZsG + n] - comp;
            const float tt = sum + y;
            comp = (tt - sum) - y;
            sum = tt;
        }
        reinterpret_cast<float *>(sCc + n * 4 + k)[l] = sum * (float)cheb_fold(n);
    }
    __syncthreads();
}

// A and B (|S|^2 = A^2 + B^2) of a contracted point at offsets (x, y)
// (6 moments serve |phi| L <= 0.2, as in cheb_point).
__device__ __forceinline__ void tab_adj_AB(const float4 *sCc, float x, float y, float phi, float aphi, float phi6,
                                           float &A, float &B)
{
    if (aphi <= phi6) cheb2_AB<6>(sCc, x, y, phi, A, B);
    else cheb2_AB<kTabMom>(sCc, x, y, phi, A, B);
}

// Warp sums of the contracted bucket values of group G0 (values 32 G0 ..
// 32 G0 + 31 of the first nv): value v = al_n mono_t with n = v / 15,
// t = v mod 15, al_n = ae (phi^2)^{n/2} (n even) or ao (phi^2)^{(n-1)/2} (n
// odd; ao carries one phi).  A group spans at most three orders.
template <int G0>
__device__ __forceinline__ float tab_ctr_group(float ae, float ao, float p2, const float (&mono)[kTabMono], int nv,
                                               int lane)
{
    constexpr int N0 = (32 * G0) / kTabMono;
    float pw = 1.0f;
#pragma unroll
    for (int i = 0; i < N0 / 2; ++i) pw *= p2;
    float a[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int n = N0 + j;
        const int extra = ((N0 & 1) + j) >> 1;
        float v = ((n & 1) ? ao : ae) * pw;
        if (extra >= 1) v *= p2;
        if (extra >= 2) v *= p2;
        a[j] = v;
    }
    return butterfly32(
        [&](int v) {
            const int va = 32 * G0 + v;
            return va < nv ? a[va / kTabMono - N0] * mono[va % kTabMono] : 0.0f;
        },
        lane);
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
        sincos_rev<true>(phr * z.x, sn, cs);
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
        phasor_rev_ff<true>(ph, e.x, e.y, sn, cs);
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
    const float iph2 = __fdividef(1.0f, ph * ph);
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
    float4 *sW = reinterpret_cast<float4 *>(rows + G);                     // [M][4] contraction scratch
    __shared__ PieceConst<float> kc;
    __shared__ float s_d0[2];
    __shared__ double scratch[32];
    __shared__ int s_item;
    // contracted small phase: the candidate's forward coefficients, per-warp
    // bucket sums (FP32 between folds, FP64 after) and their block totals
    __shared__ float4 sCc[kTabMom * 4];
    __shared__ float sYt[8][kTabCtrS];
    __shared__ double sYd[8][kTabCtrN];
    __shared__ double sZ[kTabCtrN];
    __shared__ float s_amax;

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
    for (int t = threadIdx.x; t < 8 * kTabCtrS; t += blockDim.x) (&sYt[0][0])[t] = 0.0f;
    for (int t = threadIdx.x; t < 8 * kTabCtrN; t += blockDim.x) (&sYd[0][0])[t] = 0.0;

    const float c3 = (float)(kPi * qp.beta3);
    const float c4 = (float)(2.0 * kPi * kPi / 3.0 * qp.beta4);
    const float b2 = (float)qp.beta2;
    const float m4pi2 = (float)(-4.0 * kPi * kPi);
    const float phi_direct = 3.14159265f / qp.dz_max;
    const float phi_small = 0.02f / qp.L;
    const float phi_cheb = kChebPhiLA / qp.L;
    const float phi_c6 = kChebPhiL6 / qp.L;
    const float invG = 1.0f / (float)G;
    const float4 *oq = sOQ + l16, *oz = sOZ + l16, *oe = sOE + l16;
    float *Yw = sYt[warp];
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
        // this tile's rows start at zero
        const int row0 = ap.row_off[it];
        const int nrow = ap.row_off[it + 1] - row0;
        double2 *trows = ap.rows + (size_t)row0 * M;
        double *trowsV = ap.rowsV + row0;
        for (int t = threadIdx.x; t < nrow * M; t += blockDim.x) trows[t] = make_double2(0.0, 0.0);
        for (int t = threadIdx.x; t < nrow; t += blockDim.x) trowsV[t] = 0.0;
        double acc = 0.0;           // the tile's partial of Sigma_i
        for (int kp = item.piece0; kp < item.piece1; ++kp) {
            const DevPiece pc = qp.pieces[dbg_clamp(kp, qp.n_pieces, kDbgPiece, qp.dbg)];
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
            // the contraction applies when the in-channel exponents are small
            const float ha = (float)(0.5 * qp.ch_B[coff + pc.a]), hb = (float)(0.5 * qp.ch_B[coff + pc.b]);
            if (threadIdx.x == 0) s_amax = 0.0f;
            __syncthreads();
            {
                float amax = 0.0f;
                for (int t = threadIdx.x; t < kc.nc * M; t += blockDim.x) {
                    const float4 q = sQ[t];
                    amax = fmaxf(amax, fmaxf(fabsf(q.y * ha), fabsf(q.z * hb)) * 0.69314718f);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(kFullT, amax, o));
                if (lane == 0) atomicMax(reinterpret_cast<unsigned *>(&s_amax), __float_as_uint(amax));
            }
            __syncthreads();
            const bool cheb = qp.zs_g != nullptr && s_amax <= kChebMaxA;
            const float invha = 1.0f / ha, invhb = 1.0f / hb;
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
                if (cheb) tab_adj_coeffs(qp, sQ + cc * M, ha, hb, sW, sCc);   // syncs the block
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
                    bool ctr = false;            // contracted small-phase point
                    float cA = 0.0f, cB = 0.0f, cx = 0.0f, cy = 0.0f;
                    if (q < npts) {
                        const int r = (int)(((float)q + 0.5f) * invG);
                        const int j = q - r * G;
                        const RowF rw = rows[dbg_clamp(r, G, kDbgRow, qp.dbg)];
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
                                    cp = mult * rw.w * W * array_factor_f(phi, qp);
                                    if (cheb && aphi <= phi_cheb) {
                                        cx = da * invha;
                                        cy = db * invhb;
                                        tab_adj_AB(sCc, cx, cy, phi, aphi, phi_c6, cA, cB);
                                        vsum += cp * fmaf(cA, cA, cB * cB);
                                        ctr = true;
                                    } else {
                                        cls = aphi <= phi_small ? kClsSmallT
                                                                : (aphi <= phi_direct ? kClsDirectT : kClsTeleT);
                                    }
                                }
                            }
                        }
                    }
                    // contracted points: their bucket sums, as many orders as the batch needs
                    if (__ballot_sync(kFullT, ctr)) {
                        const unsigned phl =
                            __reduce_max_sync(kFullT, __float_as_uint(ctr ? fabsf(phi) * qp.L : 0.0f));
                        const int nv = __uint_as_float(phl) <= kTabShortPhiL ? kTabShortN : kTabCtrN;
                        const float xp[5] = {1.0f, cx, cx * cx, cx * cx * cx, (cx * cx) * (cx * cx)};
                        const float yp[5] = {1.0f, cy, cy * cy, cy * cy * cy, (cy * cy) * (cy * cy)};
                        float mono[kTabMono];
#pragma unroll
                        for (int d = 0; d <= 4; ++d)
#pragma unroll
                            for (int j = 0; j <= d; ++j) mono[mono_idx(d - j, j)] = xp[d - j] * yp[j];
                        const float ae = ctr ? 2.0f * cp * cA : 0.0f;
                        const float ao = ctr ? 2.0f * cp * cB * phi : 0.0f;
                        const float p2 = phi * phi;
                        Yw[lane] += tab_ctr_group<0>(ae, ao, p2, mono, nv, lane);
                        Yw[lane + 32] += tab_ctr_group<1>(ae, ao, p2, mono, nv, lane);
                        Yw[lane + 64] += tab_ctr_group<2>(ae, ao, p2, mono, nv, lane);
                        if (nv > kTabShortN) {
                            Yw[lane + 96] += tab_ctr_group<3>(ae, ao, p2, mono, nv, lane);
                            Yw[lane + 128] += tab_ctr_group<4>(ae, ao, p2, mono, nv, lane);
                            Yw[lane + 160] += tab_ctr_group<5>(ae, ao, p2, mono, nv, lane);
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
                    if (++batches == kFoldBatchesT) {
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
                        for (int t = lane; t < kTabCtrN; t += 32) {
                            sYd[warp][t] += (double)Yw[t];
                            Yw[t] = 0.0f;
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
                for (int t = lane; t < kTabCtrN; t += 32) {
                    sYd[warp][t] += (double)Yw[t];
                    Yw[t] = 0.0f;
                }
                const double vtot = block_sum_d((double)vsum, scratch);   // syncs the block
                acc += vtot;
                if (cheb) {
                    // the contracted points' bucket sums of the whole block, in warp order
                    for (int t = threadIdx.x; t < kTabCtrN; t += blockDim.x) {
                        double z = 0.0;
                        for (int w = 0; w < nw; ++w) {
                            z += sYd[w][t];
                            sYd[w][t] = 0.0;
                        }
                        sZ[t] = z;
                    }
                    __syncthreads();
                }
                const int c = pc.c_lo + cc;
                const double D = (qp.ch_frel[coff + pc.a] + qp.ch_frel[coff + pc.b]) -
                                 (fi_d + qp.ch_frel[coff + c]);
                // the tile's rows: each thread owns its steps m, so the adds are
                // ordered (rows may coincide, e.g. a == CUT: same thread, in turn)
                const int4 pr = ap.prow[kp];
                double2 *ra = trows + (size_t)pr.x * M, *rb = trows + (size_t)pr.y * M;
                double2 *ri = trows + (size_t)pr.z * M, *rc = trows + (size_t)(pr.w + cc) * M;
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
                    if (cheb) {
                        // d|S|^2/d ln p_m of the contracted points: w_m(x, y) =
                        // base e^{al x + be y} to total degree 3, so the three buckets are
                        // base sum_n fold_n g_n(m) sum_{i+j<=3} al^i be^j / (i! j!) Z_n(x^i y^j),
                        // with one more power of x (R_a, times h_a) or y (R_b, times h_b)
                        const float4 q = sQ[cc * M + m];
                        const float al = q.y * ha * 0.69314718f, be = q.z * hb * 0.69314718f;
                        float cij[10];
                        {
                            const float ap[4] = {1.0f, al, al * al * 0.5f, al * al * al * (1.0f / 6.0f)};
                            const float bp[4] = {1.0f, be, be * be * 0.5f, be * be * be * (1.0f / 6.0f)};
#pragma unroll
                            for (int d = 0; d <= 3; ++d)
#pragma unroll
                                for (int j = 0; j <= d; ++j) cij[mono_idx(d - j, j)] = ap[d - j] * bp[j];
                        }
                        const float *gm = reinterpret_cast<const float *>(qp.zs_g + kZsG * m);
                        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
#pragma unroll
                        for (int n = 0; n < kTabMom; ++n) {
                            const double *Z = sZ + n * kTabMono;
                            float t0 = 0.0f, t1 = 0.0f, t2 = 0.0f;
#pragma unroll
                            for (int d = 0; d <= 3; ++d)
#pragma unroll
                                for (int j = 0; j <= d; ++j) {
                                    const int i = d - j;
                                    const float c = cij[mono_idx(i, j)];
                                    t0 = fmaf(c, (float)Z[mono_idx(i, j)], t0);
                                    t1 = fmaf(c, (float)Z[mono_idx(i + 1, j)], t1);
                                    t2 = fmaf(c, (float)Z[mono_idx(i, j + 1)], t2);
                                }
                            const float gf = (float)cheb_fold(n) * gm[n];
                            s0 = fmaf(gf, t0, s0);
                            s1 = fmaf(gf, t1, s1);
                            s2 = fmaf(gf, t2, s2);
                        }
                        const double base = (double)ex2_approx(q.x);
                        r0 += base * (double)s0;
                        r1 += base * (double)ha * (double)s1;
                        r2 += base * (double)hb * (double)s2;
                    }
                    ra[m].x += 0.5 * r0;
                    rb[m].x += 0.5 * r0;
                    rc[m].x += 0.5 * r0;
                    ri[m].x -= 0.5 * r0;
                    ra[m].y += 0.5 * r1;
                    rb[m].y += 0.5 * r2;
                    rc[m].y += 0.5 * (D * r0 + r1 + r2);
                }
                if (threadIdx.x == 0) {
                    trowsV[pr.x] += vtot;
                    trowsV[pr.y] += vtot;
                    trowsV[pr.w + cc] += vtot;
                }
                __syncthreads();
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) qp.partial[it] = acc;
    }
}

// dT/d{a_c, b_c}(m) and dT/d ln P_c (PSD): the rows of channel c from every
// tile that touches it, weighted by dT/dSigma of the tile's CUT, in tile
// order.  One block per plan channel.
__global__ void __launch_bounds__(128) k_tab_gather(TabGatherParams gp)
{
    const int c = blockIdx.x, M = gp.n_steps;
    const int e0 = gp.gath_off[c], e1 = gp.gath_off[c + 1];
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        double ga = 0.0, gb = 0.0;
        for (int e = e0; e < e1; ++e) {
            const int2 rs = gp.gath[e];
            const double y = gp.ybar[gp.slot_cut[rs.y]];
            const double2 v = gp.rows[(size_t)rs.x * M + m];
            ga += y * v.x;
            gb += y * v.y;
        }
        gp.gAB[(size_t)c * M + m] = make_double2(ga, gb);
    }
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int e = e0; e < e1; ++e) {
            const int2 rs = gp.gath[e];
            v += gp.ybar[gp.slot_cut[rs.y]] * gp.rowsV[rs.x];
        }
        gp.gV[c] = v;
    }
}

cudaError_t launch_tab_gather(const TabGatherParams &gp, cudaStream_t st)
{
    k_tab_gather<<<gp.n_ch, 128, 0, st>>>(gp);
    return cudaGetLastError();
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
           (size_t)nw * 3 * K * 16 * sizeof(double) + (size_t)G * sizeof(RowF) +
           (size_t)n_steps * 4 * sizeof(float4);
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
