// Tabulated power profile from the Raman ODEs, and the quadratures that use it
// (arXiv 2401.18022, Sec. III and App. A: the profile term of Eq. pk comes
// from the Raman power-evolution ODEs, with the gain scaled by the effective
// area at the channel frequency).
//
// Model.  Channel k is a line of power P_k at f_k; with y_i = ln P_i
//   dy_i/dz = -alpha_i + s_i C_r sum_{k != i} h(f_k, f_i) P_k,
//   h = f_k - f_i               for 0 < f_k - f_i <= df_max  (k pumps i)
//   h = (f_k - f_i) f_i / f_k   for 0 < f_i - f_k <= df_max  (photon ratio;
//                                                              1 if disabled)
// so the partners of channel i form one index window [lo_i, hi_i] of the
// sorted plan, and the sum splits into prefix sums over the window:
//   above i:  sum (fr_k - fr_i) P_k = S(fr P) - fr_i S(P)
//   below i:  sum (fr_k - fr_i) (f_i / f_k) P_k = f_i (S(fr P / f) - fr_i S(P / f))
// (fr = f - f_ref), i.e. four block-wide scans per right-hand side instead of
// an n x n sum.  A slot with P = 0 pumps nothing and follows the gain of a
// zero-power probe (its y starts at 0).
//
// k_raman_ode   one block per profile: classical RK4 through the nodes
//               e_m -> z_m -> e_{m+1} of every z-step, each half in
//               half_steps[m] equal steps; tables
//                 a_c(m) = y_c(z_m) - y_c(0),  ln rho_c(L) = y_c(L) - y_c(0),
//                 b_c(m) = central difference over the neighbouring channels
//                          of the Raman part a + alpha z_m (one-sided at the
//                          plan's ends),
//               so that ln rho(z_m, F) = a_c(m) + b_c(m) (F - f_c) in channel c.
// k_quad_f32_tab, k_quad_f64_tab
//               the persistent quadratures of the closed-form kernels with
//               this profile.  For a grid point of piece (a, b) of CUT i with
//               F_c in candidate channel c,
//                 ln p_m = 1/2 [ln rho(F_a) + ln rho(F_b) + ln rho(F_c) - ln rho(f_i)]
//                        = A_c(m) + Sa_c(m) da + Sb_c(m) db,
//               da = F_a - f_a, db = F_b - f_b, A = (a_a + a_b + a_c - a_i +
//               b_c (f_a + f_b - f_i - f_c)) / 2, Sa = (b_a + b_c)/2,
//               Sb = (b_b + b_c)/2, tabulated per piece and candidate, so a
//               grid point costs the same two FMAs per step as the closed form.
#include <cuda_runtime.h>

#include "isrs_internal.cuh"
#include "isrs_kernels.h"
#include "quad_common.cuh"

namespace isrs {

namespace {

constexpr int kOdeThreads = 1024;

// Exclusive prefix sums of four arrays v0..v3 [0, n) into x0..x3 [0, n]
// (x[k] = sum_{j<k} v[j]), all in shared memory.  Each thread scans a run of
// ceil(n / blockDim) consecutive entries; run totals are scanned by warp
// shuffles.  Called by every thread of the block.
__device__ void scan4(const double *v0, const double *v1, const double *v2, const double *v3, double *x0,
                      double *x1, double *x2, double *x3, int n, double *wsum /* [4 * 32] */)
{
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int b = threadIdx.x * per, e = min(n, b + per);
    double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
    for (int k = b; k < e; ++k) {
        t0 += v0[k];
        t1 += v1[k];
        t2 += v2[k];
        t3 += v3[k];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double i0 = t0, i1 = t1, i2 = t2, i3 = t3;            // inclusive within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double u0 = __shfl_up_sync(0xffffffffu, i0, o), u1 = __shfl_up_sync(0xffffffffu, i1, o);
        const double u2 = __shfl_up_sync(0xffffffffu, i2, o), u3 = __shfl_up_sync(0xffffffffu, i3, o);
        if (lane >= o) {
            i0 += u0;
            i1 += u1;
            i2 += u2;
            i3 += u3;
        }
    }
    if (lane == 31) {
        wsum[wid] = i0;
        wsum[32 + wid] = i1;
        wsum[64 + wid] = i2;
        wsum[96 + wid] = i3;
    }
    __syncthreads();
    if (wid == 0) {
        double w0 = lane < nw ? wsum[lane] : 0.0, w1 = lane < nw ? wsum[32 + lane] : 0.0;
        double w2 = lane < nw ? wsum[64 + lane] : 0.0, w3 = lane < nw ? wsum[96 + lane] : 0.0;
        const double s0 = w0, s1 = w1, s2 = w2, s3 = w3;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double u0 = __shfl_up_sync(0xffffffffu, w0, o), u1 = __shfl_up_sync(0xffffffffu, w1, o);
            const double u2 = __shfl_up_sync(0xffffffffu, w2, o), u3 = __shfl_up_sync(0xffffffffu, w3, o);
            if (lane >= o) {
                w0 += u0;
                w1 += u1;
                w2 += u2;
                w3 += u3;
            }
        }
        if (lane < nw) {                                  // exclusive warp offsets
            wsum[lane] = w0 - s0;
            wsum[32 + lane] = w1 - s1;
            wsum[64 + lane] = w2 - s2;
            wsum[96 + lane] = w3 - s3;
        }
    }
    __syncthreads();
    double r0 = wsum[wid] + i0 - t0, r1 = wsum[32 + wid] + i1 - t1;
    double r2 = wsum[64 + wid] + i2 - t2, r3 = wsum[96 + wid] + i3 - t3;
    for (int k = b; k < e; ++k) {
        x0[k] = r0;
        x1[k] = r1;
        x2[k] = r2;
        x3[k] = r3;
        r0 += v0[k];
        r1 += v1[k];
        r2 += v2[k];
        r3 += v3[k];
    }
    if (threadIdx.x == blockDim.x - 1) {                  // its running sum is the total
        x0[n] = r0;
        x1[n] = r1;
        x2[n] = r2;
        x3[n] = r3;
    }
    __syncthreads();
}

struct OdeShared {
    double *y, *yt, *kacc, *ev0, *ev1, *ev2, *ev3, *x0, *x1, *x2, *x3;
};

// dy/dz at state Y into K (shared arrays; every thread calls).
__device__ void raman_rhs(const RamanParams &rp, int coff, int poff, int n, const double *Y, double *K,
                          const OdeShared &s, double *wsum)
{
    const double *fr = rp.ch_frel + coff;
    const double *P0 = rp.P + poff;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const double e = P0[k] > 0.0 ? exp(Y[k]) : 0.0;
        const double invf = 1.0 / (fr[k] + rp.f_ref);
        s.ev0[k] = e;
        s.ev1[k] = fr[k] * e;
        s.ev2[k] = e * invf;
        s.ev3[k] = fr[k] * e * invf;
    }
    __syncthreads();
    scan4(s.ev0, s.ev1, s.ev2, s.ev3, s.x0, s.x1, s.x2, s.x3, n, wsum);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int lo = rp.win_lo[coff + i], hi = rp.win_hi[coff + i];
        const double fri = fr[i];
        // partners above i: k in (i, hi]
        double g = 0.0;
        if (hi > i) g += (s.x1[hi + 1] - s.x1[i + 1]) - fri * (s.x0[hi + 1] - s.x0[i + 1]);
        // partners below i: k in [lo, i)
        if (lo < i) {
            if (rp.photon)
                g += (fri + rp.f_ref) * ((s.x3[i] - s.x3[lo]) - fri * (s.x2[i] - s.x2[lo]));
            else
                g += (s.x1[i] - s.x1[lo]) - fri * (s.x0[i] - s.x0[lo]);
        }
        K[i] = -rp.ch_alpha[coff + i] + rp.ch_scale[coff + i] * rp.Cr * g;
    }
    __syncthreads();
}

}  // namespace

__global__ void __launch_bounds__(kOdeThreads) k_raman_ode(RamanParams rp)
{
    extern __shared__ double smem_d[];
    __shared__ double wsum[128];
    const int p = blockIdx.x;
    const int plan = rp.prof_plan[p];
    const int n = rp.plan_n[plan];
    const int coff = rp.plan_ch_off[plan];
    const int poff = rp.prof_ch_off[p];
    const int M = rp.n_steps;
    OdeShared s;
    s.y = smem_d;
    s.yt = s.y + n;
    s.kacc = s.yt + n;
    s.ev0 = s.kacc + n;
    s.ev1 = s.ev0 + n;
    s.ev2 = s.ev1 + n;
    s.ev3 = s.ev2 + n;
    s.x0 = s.ev3 + n;
    s.x1 = s.x0 + n + 1;
    s.x2 = s.x1 + n + 1;
    s.x3 = s.x2 + n + 1;
    double *K = s.x3 + n + 1;                 // [n] stage slope
    double *y0 = K + n;                       // [n] initial state
    const double *P0 = rp.P + poff;
    double2 *ab = rp.ab + (size_t)poff * M;
    double *yn = (p == 0) ? rp.y_nodes : nullptr;

    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const double v = P0[c] > 0.0 ? log(P0[c]) : 0.0;
        s.y[c] = v;
        y0[c] = v;
    }
    __syncthreads();
    int node = 0;
    for (int m = 0; m < M; ++m) {
        const int ns = rp.half_steps[m];
        const double h = 0.5 * rp.zs_d[m].y / ns;
        for (int half = 0; half < 2; ++half) {
            for (int t = 0; t < ns; ++t) {
                if (yn)
                    for (int c = threadIdx.x; c < n; c += blockDim.x) yn[(size_t)node * n + c] = s.y[c];
                ++node;
                raman_rhs(rp, coff, poff, n, s.y, K, s, wsum);                   // k1
                for (int c = threadIdx.x; c < n; c += blockDim.x) {
                    s.kacc[c] = K[c];
                    s.yt[c] = s.y[c] + 0.5 * h * K[c];
                }
                __syncthreads();
                raman_rhs(rp, coff, poff, n, s.yt, K, s, wsum);                  // k2
                for (int c = threadIdx.x; c < n; c += blockDim.x) {
                    s.kacc[c] += 2.0 * K[c];
                    s.yt[c] = s.y[c] + 0.5 * h * K[c];
                }
                __syncthreads();
                raman_rhs(rp, coff, poff, n, s.yt, K, s, wsum);                  // k3
                for (int c = threadIdx.x; c < n; c += blockDim.x) {
                    s.kacc[c] += 2.0 * K[c];
                    s.yt[c] = s.y[c] + h * K[c];
                }
                __syncthreads();
                raman_rhs(rp, coff, poff, n, s.yt, K, s, wsum);                  // k4
                for (int c = threadIdx.x; c < n; c += blockDim.x) s.y[c] += h / 6.0 * (s.kacc[c] + K[c]);
                __syncthreads();
            }
            if (half == 0)
                for (int c = threadIdx.x; c < n; c += blockDim.x) ab[(size_t)c * M + m].x = s.y[c] - y0[c];
        }
    }
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        rp.lnrho_L[poff + c] = s.y[c] - y0[c];
        if (yn) yn[(size_t)node * n + c] = s.y[c];
    }
    __syncthreads();
    // in-channel slopes: central differences of a + alpha z_m
    const double *fr = rp.ch_frel + coff;
    const double *al = rp.ch_alpha + coff;
    for (int t = threadIdx.x; t < n * M; t += blockDim.x) {
        const int c = t / M, m = t - c * M;
        const int lo = c > 0 ? c - 1 : 0, hi = c < n - 1 ? c + 1 : n - 1;
        double b = 0.0;
        if (hi != lo) {
            const double zm = rp.zs_d[m].x;
            const double rlo = ab[(size_t)lo * M + m].x + al[lo] * zm;
            const double rhi = ab[(size_t)hi * M + m].x + al[hi] * zm;
            b = (rhi - rlo) / (fr[hi] - fr[lo]);
        }
        ab[(size_t)c * M + m].y = b;
    }
}

size_t raman_smem_bytes(int n_ch)
{
    return sizeof(double) * (size_t)(13 * n_ch + 4);
}

cudaError_t launch_raman(const RamanParams &rp, int n_prof, int max_n, cudaStream_t st)
{
    const size_t smem = raman_smem_bytes(max_n);
    cudaError_t e = cudaFuncSetAttribute(k_raman_ode, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_raman_ode<<<n_prof, kOdeThreads, smem, st>>>(rp);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Discrete adjoint of the profile (single profile, plan 0).
//
// T depends on the tables through a_c(m) = y_c(z_m) - y_c(0), b_c(m) (central
// differences of a + alpha z) and ln rho_c(L) = y_c(L) - y_c(0).  k_fold_slope
// moves dT/db onto dT/da (the stencil), k_raman_adj runs the RK4 steps
// backwards: with lambda = dT/dy after a step y' = y + h/6 (k1 + 2k2 + 2k3 + k4),
//   mu4 = J(Y4)^T (h/6 lambda),            mu3 = J(Y3)^T (h/3 lambda + h mu4),
//   mu2 = J(Y2)^T (h/3 lambda + h/2 mu3),  mu1 = J(Y1)^T (h/6 lambda + h/2 mu2),
//   dT/dy = lambda + mu1 + mu2 + mu3 + mu4,
// with the stage states Y recomputed from the stored step states, the table
// sensitivities injected at the nodes z_m and L, and
//   (J^T v)_k = C_r e^{Y_k} sum_i s_i v_i h(f_k, f_i)
// again by prefix sums over the partner window of k:
//   i below k:  sum u_i (fr_k - fr_i)              = fr_k S(u) - S(fr u)
//   i above k:  sum u_i (fr_k - fr_i) f_i / f_k    = (fr_k S(f u) - S(fr f u)) / f_k
// (u = s v; the ratio f_i/f_k is 1 without the photon term).  Finally
//   dT/dP_j = (dT/dy_j(0) + dT/d ln P_j|_PSD) / P_j + dT/dSNR_j dSNR_j/dP_j|_N.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_fold_slope(RamanAdjParams ap)
{
    const int n = ap.n, M = ap.r.n_steps;
    const double *fr = ap.r.ch_frel;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * M; t += gridDim.x * blockDim.x) {
        const int c = t / M, m = t - c * M;
        double g = ap.gAB[t].x;
        for (int q = max(0, c - 1); q <= min(n - 1, c + 1); ++q) {
            const int lo = q > 0 ? q - 1 : 0, hi = q < n - 1 ? q + 1 : n - 1;
            if (lo == hi) continue;
            const double gb = ap.gAB[(size_t)q * M + m].y / (fr[hi] - fr[lo]);
            if (hi == c) g += gb;
            if (lo == c) g -= gb;
        }
        ap.gAt[t] = g;
    }
}

namespace {

// out = J(Y)^T v (shared arrays; every thread calls)
__device__ void raman_jt(const RamanParams &rp, int n, const double *Y, const double *v, double *out,
                         const OdeShared &s, double *wsum)
{
    const double *fr = rp.ch_frel;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double u = rp.ch_scale[i] * v[i];
        const double f = fr[i] + rp.f_ref;
        s.ev0[i] = u;
        s.ev1[i] = fr[i] * u;
        s.ev2[i] = f * u;
        s.ev3[i] = fr[i] * f * u;
    }
    __syncthreads();
    scan4(s.ev0, s.ev1, s.ev2, s.ev3, s.x0, s.x1, s.x2, s.x3, n, wsum);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double r = 0.0;
        if (rp.P[k] > 0.0) {
            const int lo = rp.win_lo[k], hi = rp.win_hi[k];
            const double frk = fr[k];
            double g = 0.0;
            if (lo < k) g += frk * (s.x0[k] - s.x0[lo]) - (s.x1[k] - s.x1[lo]);
            if (hi > k) {
                if (rp.photon)
                    g += (frk * (s.x2[hi + 1] - s.x2[k + 1]) - (s.x3[hi + 1] - s.x3[k + 1])) / (frk + rp.f_ref);
                else
                    g += frk * (s.x0[hi + 1] - s.x0[k + 1]) - (s.x1[hi + 1] - s.x1[k + 1]);
            }
            r = rp.Cr * exp(Y[k]) * g;
        }
        out[k] = r;
    }
    __syncthreads();
}

}  // namespace

__global__ void __launch_bounds__(kOdeThreads) k_raman_adj(RamanAdjParams ap)
{
    extern __shared__ double smem_d[];
    __shared__ double wsum[128];
    const RamanParams &rp = ap.r;
    const int n = ap.n, M = rp.n_steps;
    double *lam = smem_d, *acc = lam + n, *w = acc + n, *mu = w + n, *Y2 = mu + n, *Y3 = Y2 + n, *Y4 = Y3 + n;
    OdeShared s;
    s.y = s.yt = s.kacc = nullptr;
    s.ev0 = Y4 + n;
    s.ev1 = s.ev0 + n;
    s.ev2 = s.ev1 + n;
    s.ev3 = s.ev2 + n;
    s.x0 = s.ev3 + n;
    s.x1 = s.x0 + n + 1;
    s.x2 = s.x1 + n + 1;
    s.x3 = s.x2 + n + 1;

    for (int c = threadIdx.x; c < n; c += blockDim.x)
        lam[c] = ap.with_direct ? -ap.aase[c] : 0.0;                               // dT/d ln rho(L)
    __syncthreads();
    int node = ap.n_rk;
    for (int m = M - 1; m >= 0; --m) {
        const int ns = rp.half_steps[m];
        const double h = 0.5 * rp.zs_d[m].y / ns;
        for (int half = 1; half >= 0; --half) {
            for (int t = 0; t < ns; ++t) {
                --node;
                const double *Y1 = ap.y_nodes + (size_t)node * n;
                // stage states of this step
                raman_rhs(rp, 0, 0, n, Y1, mu, s, wsum);
                for (int c = threadIdx.x; c < n; c += blockDim.x) Y2[c] = Y1[c] + 0.5 * h * mu[c];
                __syncthreads();
                raman_rhs(rp, 0, 0, n, Y2, mu, s, wsum);
                for (int c = threadIdx.x; c < n; c += blockDim.x) Y3[c] = Y1[c] + 0.5 * h * mu[c];
                __syncthreads();
                raman_rhs(rp, 0, 0, n, Y3, mu, s, wsum);
                for (int c = threadIdx.x; c < n; c += blockDim.x) {
                    Y4[c] = Y1[c] + h * mu[c];
                    acc[c] = lam[c];
                    w[c] = h / 6.0 * lam[c];
                }
                __syncthreads();
                raman_jt(rp, n, Y4, w, mu, s, wsum);                         // mu4
                for (int c = threadIdx.x; c < n; c += blockDim.x) {
                    acc[c] += mu[c];
                    w[c] = h / 3.0 * lam[c] + h * mu[c];
                }
                __syncthreads();
                raman_jt(rp, n, Y3, w, mu, s, wsum);                         // mu3
                for (int c = threadIdx.x; c < n; c += blockDim.x) {
                    acc[c] += mu[c];
                    w[c] = h / 3.0 * lam[c] + 0.5 * h * mu[c];
                }
                __syncthreads();
                raman_jt(rp, n, Y2, w, mu, s, wsum);                         // mu2
                for (int c = threadIdx.x; c < n; c += blockDim.x) {
                    acc[c] += mu[c];
                    w[c] = h / 6.0 * lam[c] + 0.5 * h * mu[c];
                }
                __syncthreads();
                raman_jt(rp, n, Y1, w, mu, s, wsum);                         // mu1
                for (int c = threadIdx.x; c < n; c += blockDim.x) lam[c] = acc[c] + mu[c];
                __syncthreads();
            }
            if (half == 1)
                for (int c = threadIdx.x; c < n; c += blockDim.x) lam[c] += ap.gAt[(size_t)c * M + m];
            __syncthreads();
        }
    }
    // a = y - y(0): every table entry also depends on y(0) directly
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double direct = ap.with_direct ? ap.aase[j] : 0.0;             // - dT/d ln rho(L)
        for (int m = 0; m < M; ++m) direct -= ap.gAt[(size_t)j * M + m];
        const double P = rp.P[j];
        double g = (lam[j] + direct + ap.gV[j]) / P;
        if (ap.with_direct) {                                          // the SNR numerator
            const double snr = ap.snr[j], B = ap.ch_B[j];
            const double N = ap.pnli[j] + ap.pase[j];
            const double dTds = 2.0 * B / (0.69314718055994530942 * (1.0 + snr));
            g += dTds * snr * snr * N / (P * P);
        }
        ap.dT_dP[j] = g;
    }
}

size_t raman_adj_smem_bytes(int n_ch)
{
    return sizeof(double) * (size_t)(15 * n_ch + 4);
}

cudaError_t launch_raman_adj(const RamanAdjParams &ap, cudaStream_t st)
{
    const int nm = ap.n * ap.r.n_steps;
    k_fold_slope<<<(nm + 255) / 256, 256, 0, st>>>(ap);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = raman_adj_smem_bytes(ap.n);
    e = cudaFuncSetAttribute(k_raman_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_raman_adj<<<1, kOdeThreads, smem, st>>>(ap);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Quadratures with the tabulated profile.
// ---------------------------------------------------------------------------
namespace {

// Per-piece table: for every candidate channel ci of F_c and step m (log2
// units, FP32) {A + log2 dz, Sa, Sb, A}, built in FP64 from the profile
// tables.  Every thread calls; the caller syncs before use.
__device__ void tab_setup_f(const QuadParams &qp, const DevPiece &pc, int prof, int nc, float4 *sQ)
{
    const int M = qp.n_steps;
    const int coff = qp.plan_ch_off[pc.plan];
    const double2 *T = qp.ab + (size_t)qp.prof_ch_off[prof] * M;
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

// FP32 z-sums of Eq. slow_vary with log2 p_m = Q.w + Q.y da + Q.z db (the
// three forms of the closed-form kernel: small-phase expansion, direct,
// telescoped).  sZ[m] = {z_m, z_m^2 + dz_m^2/12, dz_m, -}, sE[m] = {z_{m+1}/2pi
// hi, lo, -, -}.
__device__ __forceinline__ float zsum_small_t(float phi, float da, float db, const float4 *Q, const float4 *sZ,
                                              int M)
{
    float M0 = 0.0f, M1 = 0.0f, M2 = 0.0f;
#pragma unroll 4
    for (int m = 0; m < M; ++m) {
        const float4 q = Q[m];
        const float4 z = sZ[m];
        float lp = fmaf(q.y, da, q.x);
        lp = fmaf(q.z, db, lp);
        const float w = ex2_approx(lp);          // p_m dz_m
        M0 += w;
        M1 = fmaf(w, z.x, M1);
        M2 = fmaf(w, z.y, M2);
    }
    return fmaf(-phi * phi, fmaf(M0, M2, -M1 * M1), M0 * M0);
}

__device__ __forceinline__ float zsum_direct_t(float phi, float da, float db, const float4 *Q, const float4 *sZ,
                                               int M)
{
    float Sr = 0.0f, Si = 0.0f;
    const float hphi = 0.5f * phi;
    const float phir = phi * 0.15915494309189535f;
#pragma unroll 4
    for (int m = 0; m < M; ++m) {
        const float4 q = Q[m];
        const float4 z = sZ[m];
        float sn, cs;
        sincos_rev(phir * z.x, sn, cs);
        const float x = hphi * z.z;
        const float x2 = x * x;
        float sc = fmaf(x2, -2.5052108e-8f, 2.7557319e-6f);   // -1/11!, 1/9!
        sc = fmaf(x2, sc, -1.9841270e-4f);                     // -1/7!
        sc = fmaf(x2, sc, 8.3333333e-3f);                      // 1/5!
        sc = fmaf(x2, sc, -1.6666667e-1f);                     // -1/3!
        sc = fmaf(x2, sc, 1.0f);
        float lp = fmaf(q.y, da, q.x);
        lp = fmaf(q.z, db, lp);
        const float amp = ex2_approx(lp) * sc;
        Sr = fmaf(amp, cs, Sr);
        Si = fmaf(amp, sn, Si);
    }
    return Sr * Sr + Si * Si;
}

__device__ __forceinline__ float zsum_tele_t(float phi, float da, float db, const float4 *Q, const float4 *sE,
                                             int M)
{
    float Er = 1.0f, Ei = 0.0f, Sr = 0.0f, Si = 0.0f;
#pragma unroll 4
    for (int m = 0; m < M; ++m) {
        const float4 q = Q[m];
        const float4 e = sE[m];
        float sn, cs;
        phasor_rev_ff(phi, e.x, e.y, sn, cs);
        float lp = fmaf(q.y, da, q.w);
        lp = fmaf(q.z, db, lp);
        const float p = ex2_approx(lp);
        Sr = fmaf(p, cs - Er, Sr);
        Si = fmaf(p, sn - Ei, Si);
        Er = cs;
        Ei = sn;
    }
    return __fdividef(Sr * Sr + Si * Si, phi * phi);
}

// ---------------------------------------------------------------------------
// Contracted small-phase series for the tabulated profile (the moment series
// of the closed-form kernels, App. A Eq. slow_vary, at 11 moments for
// |phi| L <= 2: the 2-D expansion costs 16 coefficients per moment).  Inside
// the piece, log2 w_m = Ad_m + Sa_m da + Sb_m db with da = h_a x, db = h_b y the offsets
// of F_a and F_b inside their channels, so
//   w_m = 2^{Ad_m} e^{alpha_m x} e^{beta_m y},  alpha = Sa h_a ln 2, beta = Sb h_b ln 2,
// and with e^{a x} = I0(a) + 2 sum Ik(a) Tk(x) in each offset
//   nu_n(x, y) = sum_{k,l <= 3} C_nkl Tk(x) Tl(y),
//   C_nkl = sum_m 2^{Ad_m} b_k(alpha_m) b_l(beta_m) g_n(m)
// (truncation ~ (a/2)^4/12 per offset for |alpha|, |beta| <= 0.05).  The
// coefficients are stored times (-1)^{floor(n/2)}/n!, as row k = float4 over l.
// ---------------------------------------------------------------------------
constexpr int kTabMom = kChebMomA;

// Every thread calls after tab_setup_f (synced); returns whether the piece's
// small-phase points use the contraction.  sW: [M][4] float4 scratch,
// sG: [M][4 kZsG] moments, sC: [nc][kTabMom][4] float4, s_flag: shared int.
__device__ bool tab_cheb_setup(const QuadParams &qp, const DevPiece &pc, int nc, const float4 *sQ, float4 *sW,
                               float *sG, float4 *sC, float *s_amax)
{
    const int M = qp.n_steps;
    if (qp.zs_g == nullptr) return false;
    const int coff = qp.plan_ch_off[pc.plan];
    const float ha = (float)(0.5 * qp.ch_B[coff + pc.a]), hb = (float)(0.5 * qp.ch_B[coff + pc.b]);
    const float ln2 = 0.69314718f;
    if (threadIdx.x == 0) *s_amax = 0.0f;
    __syncthreads();
    float amax = 0.0f;
    for (int t = threadIdx.x; t < nc * M; t += blockDim.x) {
        const float4 q = sQ[t];
        amax = fmaxf(amax, fmaxf(fabsf(q.y * ha), fabsf(q.z * hb)) * ln2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned *>(s_amax), __float_as_uint(amax));
    for (int t = threadIdx.x; t < M * 4 * kZsG; t += blockDim.x) sG[t] = reinterpret_cast<const float *>(qp.zs_g)[t];
    __syncthreads();
    if (!(*s_amax <= kChebMaxA)) return false;
    for (int c = 0; c < nc; ++c) {
        const float4 *Q = sQ + c * M;
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
        // one coefficient (n, k, l) per thread: compensated sum over the steps
        for (int t = threadIdx.x; t < kTabMom * 16; t += blockDim.x) {
            const int n = t >> 4, k = (t >> 2) & 3, l = t & 3;
            float sum = 0.0f, comp = 0.0f;
            for (int m = 0; m < M; ++m) {
                const float4 w = sW[m * 4 + k];
                const float wl = l == 0 ? w.x : (l == 1 ? w.y : (l == 2 ? w.z : w.w));
                const float y = wl * sG[m * 4 * kZsG + n] - comp;
                const float tt = sum + y;
                comp = (tt - sum) - y;
                sum = tt;
            }
            reinterpret_cast<float *>(sC + (c * kTabMom + n) * 4 + k)[l] = sum * (float)cheb_fold(n);
        }
        __syncthreads();
    }
    return true;
}

// |S|^2 of a small-phase point of candidate ci from the contracted series
// (6 moments serve |phi| L <= 0.2, as in cheb_point).
__device__ __forceinline__ float tab_cheb_s2(const float4 *sC, int ci, float x, float y, float phi, float aphi,
                                             float phi6)
{
    const float4 *C = sC + ci * kTabMom * 4;
    float A, B;
    if (aphi <= phi6) cheb2_AB<6>(C, x, y, phi, A, B);
    else cheb2_AB<kTabMom>(C, x, y, phi, A, B);
    return fmaf(A, A, B * B);
}

}  // namespace

__global__ void __launch_bounds__(256, 4) k_quad_f32_tab(QuadParams qp)
{
    extern __shared__ float4 smem_f4[];
    const int M = qp.n_steps, G = qp.G;
    float4 *sZ = smem_f4;                              // [M] {z, z^2 + dz^2/12, dz, 0}
    float4 *sE = sZ + M;                               // [M] {edge/2pi hi, lo, 0, 0}
    float4 *sQ = sE + M;                               // [nc_max][M] {A + log2 dz, Sa, Sb, A}
    float4 *sW = sQ + (size_t)qp.nc_max * M;           // [M][4] contraction weights of one candidate
    float4 *sC = sW + (size_t)M * 4;                   // [nc_max][kTabMom][4] contracted coefficients
    float *sG = reinterpret_cast<float *>(sC + (size_t)qp.nc_max * kTabMom * 4);   // [M][4 kZsG] step moments
    RowF *rows = reinterpret_cast<RowF *>(sG + (size_t)M * 4 * kZsG);   // [G]
    __shared__ PieceConst<float> kc;
    __shared__ float s_d0[2];
    __shared__ float s_amax;
    __shared__ double scratch[32];
    __shared__ int s_item;

    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const float4 za = qp.zs_a[m];   // {z_m, c_m, log2 dz_m, dz_m}
        const float4 zb = qp.zs_b[m];   // {edge(m+1)/2pi hi, lo, z_m/2pi, 0}
        sZ[m] = make_float4(za.x, za.y, za.w, 0.0f);
        sE[m] = make_float4(zb.x, zb.y, 0.0f, 0.0f);
    }
    const float c3 = (float)(kPi * qp.beta3);
    const float c4 = (float)(2.0 * kPi * kPi / 3.0 * qp.beta4);
    const float b2 = (float)qp.beta2;
    const float m4pi2 = (float)(-4.0 * kPi * kPi);
    const float phi_direct = 3.14159265f / qp.dz_max;
    const float phi_small = 0.02f / qp.L;
    const float phi_cheb = kChebPhiLA / qp.L;
    const float phi_c6 = kChebPhiL6 / qp.L;
    const float invG = 1.0f / (float)G;
    unsigned n_small = 0, n_direct = 0, n_tele = 0;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(qp.counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= qp.n_items) break;
        const DevItem item = qp.items[it];
        double acc = 0.0;
        for (int k = item.piece0; k < item.piece1; ++k) {
            const DevPiece pc = qp.pieces[dbg_clamp(k, qp.n_pieces, kDbgPiece, qp.dbg)];
            piece_rows<RowF>(pc, G, qp.eps_v1, rows);
            piece_consts<float>(qp, pc, item.prof, 0.0f, qp.pd_f, kc);
            if (threadIdx.x == 0) {
                const int coff = qp.plan_ch_off[pc.plan];
                const double fi = qp.ch_frel[coff + pc.cut];
                s_d0[0] = (float)(qp.ch_frel[coff + pc.a] - fi);
                s_d0[1] = (float)(qp.ch_frel[coff + pc.b] - fi);
            }
            __syncthreads();
            tab_setup_f(qp, pc, item.prof, kc.nc, sQ);
            __syncthreads();
            const bool cheb = tab_cheb_setup(qp, pc, kc.nc, sQ, sW, sG, sC, &s_amax);
            const float phi_lim = cheb ? phi_cheb : phi_small;   // upper |phi| of the small-phase forms
            float inv_ha = 0.0f, inv_hb = 0.0f;
            {
                const int coff = qp.plan_ch_off[pc.plan];
                inv_ha = (float)(2.0 / qp.ch_B[coff + pc.a]);
                inv_hb = (float)(2.0 / qp.ch_B[coff + pc.b]);
            }
            const float fi = kc.fi, s1g = kc.s1, s2g = kc.s2;
            const float da0 = s_d0[0], db0 = s_d0[1];
            const float three_fi2 = 3.0f * fi * fi;
            float sum = 0.0f, comp = 0.0f;
            const int npts = G * G;
            for (int q = threadIdx.x; q < npts; q += blockDim.x) {
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
                const float W = kc.wab * kc.pd[ci];
                const float da = f1 - da0, db = f2 - db0;   // F_a - f_a, F_b - f_b
                const float4 *Q = sQ + ci * M;
                // Eq. phi
                const float br = b2 + c3 * (u + 2.0f * fi) +
                                 c4 * (f1 * f1 + 1.5f * f1 * f2 + 3.0f * fi * u + f2 * f2 + three_fi2);
                const float phi = m4pi2 * f1 * f2 * br;
                const float aphi = fabsf(phi);
                float S2;
                if (aphi <= phi_lim) {
                    S2 = cheb ? tab_cheb_s2(sC, ci, da * inv_ha, db * inv_hb, phi, aphi, phi_c6) : zsum_small_t(phi, da, db, Q, sZ, M);
                    ++n_small;
                } else if (aphi <= phi_direct) {
                    S2 = zsum_direct_t(phi, da, db, Q, sZ, M);
                    ++n_direct;
                } else {
                    S2 = zsum_tele_t(phi, da, db, Q, sE, M);
                    ++n_tele;
                }
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

// Plain FP64 quadrature with the tabulated profile (direct form, libm).
__global__ void __launch_bounds__(256) k_quad_f64_tab(QuadParams qp)
{
    extern __shared__ double2 smem_d2[];
    const int M = qp.n_steps, G = qp.G;
    double2 *sz = smem_d2;                              // [M] {z_m, dz_m}
    double2 *sQ = sz + M;                               // [nc_max][M][2] {A, Sa}, {Sb, 0}
    RowD *rows = reinterpret_cast<RowD *>(sQ + (size_t)2 * qp.nc_max * M);
    __shared__ PieceConst<double> kc;
    __shared__ double s_d0[2];
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
        double acc = 0.0;
        for (int k = item.piece0; k < item.piece1; ++k) {
            const DevPiece pc = qp.pieces[dbg_clamp(k, qp.n_pieces, kDbgPiece, qp.dbg)];
            piece_rows<RowD>(pc, G, qp.eps_v1, rows);
            piece_consts<double>(qp, pc, item.prof, 0.0, qp.pd_d, kc);
            const int coff = qp.plan_ch_off[pc.plan];
            const double fa = qp.ch_frel[coff + pc.a], fb = qp.ch_frel[coff + pc.b];
            const double fic = qp.ch_frel[coff + pc.cut];
            if (threadIdx.x == 0) {
                s_d0[0] = fa - fic;
                s_d0[1] = fb - fic;
            }
            {
                const double2 *T = qp.ab + (size_t)qp.prof_ch_off[item.prof] * M;
                const int nc = min(pc.c_hi - pc.c_lo + 1, kMaxCand);
                for (int t = threadIdx.x; t < nc * M; t += blockDim.x) {
                    const int ci = t / M, m = t - ci * M;
                    const int c = pc.c_lo + ci;
                    const double2 ta = T[(size_t)pc.a * M + m], tb = T[(size_t)pc.b * M + m];
                    const double2 ti = T[(size_t)pc.cut * M + m], tc = T[(size_t)c * M + m];
                    const double D = (fa + fb) - (fic + qp.ch_frel[coff + c]);
                    sQ[2 * t] = make_double2(0.5 * (ta.x + tb.x + tc.x - ti.x + tc.y * D), 0.5 * (ta.y + tc.y));
                    sQ[2 * t + 1] = make_double2(0.5 * (tb.y + tc.y), 0.0);
                }
            }
            __syncthreads();
            const double fi = kc.fi;
            const double da0 = s_d0[0], db0 = s_d0[1];
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
                const double da = f1 - da0, db = f2 - db0;
                const double br = qp.beta2 + c3 * (u + 2.0 * fi) +
                                  c4 * (f1 * f1 + 1.5 * f1 * f2 + 3.0 * fi * u + f2 * f2 + 3.0 * fi * fi);
                const double phi = -4.0 * kPi * kPi * f1 * f2 * br;
                const double2 *Q = sQ + (size_t)2 * ci * M;
                double Sr = 0.0, Si = 0.0;
                for (int m = 0; m < M; ++m) {
                    const double2 zz = sz[m];
                    const double2 q0 = Q[2 * m], q1 = Q[2 * m + 1];
                    const double p = exp(q0.x + q0.y * da + q1.x * db);
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

size_t quad_tab_smem_bytes(int precision, int n_steps, int G, int nc_max)
{
    if (precision == 0)
        return (size_t)n_steps * (2 + nc_max + 4) * sizeof(float4) + (size_t)nc_max * kTabMom * 4 * sizeof(float4) +
               (size_t)n_steps * 4 * kZsG * sizeof(float) + (size_t)G * sizeof(RowF);
    return (size_t)n_steps * (1 + 2 * nc_max) * sizeof(double2) + (size_t)G * sizeof(RowD);
}

int quad_tab_blocks_per_sm(int precision, int n_steps, int G, int nc_max, int block)
{
    int nb = 0;
    const size_t smem = quad_tab_smem_bytes(precision, n_steps, G, nc_max);
    void *fn = precision == 0 ? (void *)k_quad_f32_tab : (void *)k_quad_f64_tab;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, smem);
    return nb > 0 ? nb : 1;
}

cudaError_t launch_quad_tab(const QuadParams &qp, int precision, int grid, int block, cudaStream_t st)
{
    const size_t smem = quad_tab_smem_bytes(precision, qp.n_steps, qp.G, qp.nc_max);
    void *fn = precision == 0 ? (void *)k_quad_f32_tab : (void *)k_quad_f64_tab;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    QuadParams q = qp;
    void *args[] = {&q};
    return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, st);
}

}  // namespace isrs
