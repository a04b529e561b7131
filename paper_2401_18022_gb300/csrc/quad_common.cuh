// Device helpers shared by the quadrature kernels (forward and adjoint).
#pragma once
#include <cuda_runtime.h>

#include "isrs_internal.cuh"

namespace isrs {

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Nearest integer of t (round to nearest even), two ways:
//  * round_magic: two adds on the FMA pipe, exact for |t| < 2^22;
//  * round_nearest: one FRND, exact for every FP32 value, issued to the
//    XU pipe that also runs the MUFU (sin, cos, ex2) instructions.
// The forward kernels (3 MUFU per step, XU ~40 % busy) measured faster with
// round_magic (FRND raised XU to ~49 % and added mio_throttle stalls); the
// adjoint walks (XU ~25 % busy, issue-bound) with round_nearest.  Either way
// t - round(t) is exact (Sterbenz).
__device__ __forceinline__ float round_magic(float t)
{
    return __fadd_rn(__fadd_rn(t, 12582912.0f), -12582912.0f);
}

__device__ __forceinline__ float round_nearest(float t)
{
    return rintf(t);
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum of one double per thread (blockDim multiple of 32).
__device__ __forceinline__ double block_sum_d(double v, double *scratch)
{
    v = warp_sum_d(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += scratch[w];
        scratch[0] = r;
    }
    __syncthreads();
    r = scratch[0];
    __syncthreads();
    return r;
}

// Warp sum of 32 values per lane in one butterfly: each level halves the
// values a lane carries, and lane L ends with the sum of value L.  val(i)
// gives this lane's value i.
template <typename F>
__device__ __forceinline__ float butterfly32(const F &val, int lane)
{
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2, b0 = lane & 1;
    float x16[16];
#pragma unroll
    for (int i = 0; i < 16; ++i)
        x16[i] = (b4 ? val(i + 16) : val(i)) + __shfl_xor_sync(0xffffffffu, b4 ? val(i) : val(i + 16), 16);
    float x8[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
        x8[i] = (b3 ? x16[i + 8] : x16[i]) + __shfl_xor_sync(0xffffffffu, b3 ? x16[i] : x16[i + 8], 8);
    float x4[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        x4[i] = (b2 ? x8[i + 4] : x8[i]) + __shfl_xor_sync(0xffffffffu, b2 ? x8[i] : x8[i + 4], 4);
    float x2[2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
        x2[i] = (b1 ? x4[i + 2] : x4[i]) + __shfl_xor_sync(0xffffffffu, b1 ? x4[i] : x4[i + 2], 2);
    return (b0 ? x2[1] : x2[0]) + __shfl_xor_sync(0xffffffffu, b0 ? x2[0] : x2[1], 1);
}

// ---------------------------------------------------------------------------
// Piece set-up shared by the quadrature kernels (FP64, once per piece).
// Row r (uniform in s = ln upsilon1): upsilon1 = exp(s_r); the |f2| range
// [ymin, ymax] of that row; upsilon2 spans ln(ymax/ymin) in G columns.
// Stored relative to the row centre so FP32 points keep full precision:
//   x_j = xc e^{d_j}, y_j = yc e^{-d_j}, d_j = (j + 1/2 - G/2) du2,
//   weight = upsilon1 ds du2 (the Jacobian of (f1, f2) -> (u1, u2) is 1).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void piece_rows(const DevPiece &pc, int G, double eps, T *rows)
{
    const double u1hi = pc.xhi * pc.yhi;
    const double u1lo = fmax(pc.xlo * pc.ylo, eps * u1hi);
    const double llo = log(u1lo);
    const double ds = (log(u1hi) - llo) / G;
    for (int r = threadIdx.x; r < G; r += blockDim.x) {
        const double u1 = exp(llo + (r + 0.5) * ds);
        const double ymin = fmax(pc.ylo, u1 / pc.xhi);
        const double ymax = pc.xlo > 0.0 ? fmin(pc.yhi, u1 / pc.xlo) : pc.yhi;
        T rw;
        if (ymax > ymin) {
            const double du2 = log1p((ymax - ymin) / ymin) / G;
            const double yc = sqrt(ymin * ymax);
            rw.xc = u1 / yc;
            rw.yc = yc;
            rw.du2 = du2;
            rw.w = u1 * ds * du2;
        } else {
            rw.xc = 0; rw.yc = 0; rw.du2 = 0; rw.w = 0;
        }
        rows[r] = rw;
    }
}

struct RowF { float xc, yc, du2, w; };
struct RowD { double xc, yc, du2, w; };

// Per-piece constants: CUT offset, signs, the PSD factors of F_a and F_b, the
// attenuation part of ln p and the candidate channels of F_c (edges relative
// to the CUT so that F_c - f_i = f1 + f2 is compared without cancellation).
template <typename T>
struct PieceConst {
    T fi, s1, s2, wab, at_ab, mult;
    int nc;
    T lo[kMaxCand], hi[kMaxCand], pd[kMaxCand], hat[kMaxCand];
};

template <typename T>
__device__ __forceinline__ void piece_consts(const QuadParams &qp, const DevPiece &pc, int prof, T at_scale,
                             const T *pdv, PieceConst<T> &k)
{
    if (threadIdx.x == 0) {
        const int coff = qp.plan_ch_off[pc.plan];
        const int poff = qp.prof_ch_off[prof];
        const double fi = qp.ch_frel[coff + pc.cut];
        k.fi = (T)fi;
        k.s1 = (pc.flags & 1) ? T(-1) : T(1);
        k.s2 = (pc.flags & 2) ? T(-1) : T(1);
        k.wab = pdv[poff + pc.a] * pdv[poff + pc.b];
        k.at_ab = (T)(0.5 * (qp.ch_alpha[coff + pc.a] + qp.ch_alpha[coff + pc.b] -
                             qp.ch_alpha[coff + pc.cut])) * at_scale;
        k.mult = (T)pc.mult;
        int nc = 0;
        for (int c = pc.c_lo; c <= pc.c_hi && nc < kMaxCand; ++c, ++nc) {
            const double fc = qp.ch_frel[coff + c], hb = 0.5 * qp.ch_B[coff + c];
            k.lo[nc] = (T)((fc - hb) - fi);
            k.hi[nc] = (T)((fc + hb) - fi);
            k.pd[nc] = pdv[poff + c];
            k.hat[nc] = (T)(0.5 * qp.ch_alpha[coff + c]) * at_scale;
        }
        k.nc = nc;
    }
}

// sin and cos of 2 pi t for |t| < 2^22 revolutions (Xu: round with FRND)
template <bool Xu = false>
__device__ __forceinline__ void sincos_rev(float t, float &sn, float &cs)
{
    const float fr = __fadd_rn(t, -(Xu ? round_nearest(t) : round_magic(t)));
    __sincosf(fr * 6.283185307179586f, &sn, &cs);
}

// e^{j phi z}: the phase phi (hi + lo) in revolutions as an error-free
// float-float product, reduced to [-1/2, 1/2] (Xu: round with FRND)
template <bool Xu = false>
__device__ __forceinline__ void phasor_rev_ff(float phi, float hi, float lo, float &sn, float &cs)
{
    const float th = phi * hi;
    float tl = fmaf(phi, hi, -th);
    tl = fmaf(phi, lo, tl);
    const float fr = __fadd_rn(th, -(Xu ? round_nearest(th) : round_magic(th))) + tl;
    __sincosf(fr * 6.283185307179586f, &sn, &cs);
}


__device__ __forceinline__ double sinc_d(double x)
{
    return fabs(x) < 1e-4 ? 1.0 - x * x / 6.0 : sin(x) / x;
}

// Phased-array factor of n identical spans (Eq. new_gn_model with
// L-tilde_k = (k-1) L): |sum_{k<n} e^{j k phi L}|^2, by rotation from the
// float-float phase phi L / 2pi.
__device__ __forceinline__ float array_factor_f(float phi, const QuadParams &qp)
{
    if (qp.n_spans <= 1) return 1.0f;
    float sn, cs;
    phasor_rev_ff(phi, qp.Lrev_hi, qp.Lrev_lo, sn, cs);
    float sr = 0.0f, si = 0.0f, zr = 1.0f, zi = 0.0f;
    for (int k = 0; k < qp.n_spans; ++k) {
        sr += zr;
        si += zi;
        const float t = fmaf(zr, cs, -zi * sn);
        zi = fmaf(zr, sn, zi * cs);
        zr = t;
    }
    return fmaf(sr, sr, si * si);
}

__device__ __forceinline__ double array_factor_d(double phi, const QuadParams &qp)
{
    if (qp.n_spans <= 1) return 1.0;
    double sn, cs;
    sincos(phi * qp.Ld, &sn, &cs);
    double sr = 0.0, si = 0.0, zr = 1.0, zi = 0.0;
    for (int k = 0; k < qp.n_spans; ++k) {
        sr += zr;
        si += zi;
        const double t = zr * cs - zi * sn;
        zi = zr * sn + zi * cs;
        zr = t;
    }
    return sr * sr + si * si;
}

// ---------------------------------------------------------------------------
// Contracted small-phase z-sum (App. A, Eq. slow_vary).  With w_m = p_m dz_m,
// dz_m sinc(phi dz_m/2) e^{j phi z_m} is the mean of e^{j phi zeta} over step
// m, so about the span centre z0 = L/2
//   S e^{-j phi z0} = sum_n (j phi)^n / n! nu_n,   nu_n = sum_m w_m g_n(m),
//   g_n(m) = mean of (zeta - z0)^n over step m,
// exactly; |S|^2 = A^2 + B^2 with A (B) the even (odd) part, and truncating
// at n = N leaves a relative error below 2 (phi L/2)^{N+1}/(N+1)!: the
// closed-form kernels keep n <= 18 for |phi| L <= 6 (< 2e-8; the adjoint keeps
// fewer orders in its bucket sums when a batch's phases allow), the
// tabulated-profile forward n <= 10 for |phi| L <= 2 (< 5e-8).
// The moments depend on the point only through F_c (and the candidate
// channel's attenuation): inside channel c, F_c - f_ref = F0 + h x with
// x in [-1, 1], and
//   w_m = 2^{A2d_m - at z_m + K2_m F0} e^{a_m x},   a_m = K2_m h ln 2,
//   e^{a x} = I0(a) + 2 sum_{k>=1} Ik(a) Tk(x),
// so nu_n(x) = sum_{k<=3} C_nk Tk(x), with C_nk summed over the steps once
// per piece and candidate.  Truncation in x ~ (a/2)^4/12 < 4e-8 for
// |a| <= 0.05, which holds when kappa(L) h <= 0.05; otherwise the per-step
// sum is used.
// ---------------------------------------------------------------------------
constexpr float kChebMaxA = 0.05f;
constexpr int kChebMom = 19;        // nu_0 .. nu_18 (forward kernels)
constexpr float kChebPhiL = 6.0f;   // |phi| L limit of the 19-moment form: error < 2e-8
constexpr float kChebPhiL6 = 0.2f;  // ... of its first 6 moments: error < (0.1)^6/6! = 1.4e-9
constexpr float kChebPhiL11 = 2.0f; // ... of its first 11 moments: error < 1/11! = 2.5e-8
constexpr int kChebMomA = 11;       // nu_0 .. nu_10 (adjoint)
constexpr float kChebPhiLA = 2.0f;  // |phi| L limit of the 11-moment form: error < 5e-8
constexpr int kZsG = 5;             // float4 per step of the centred step moments g_0..g_19 (g_19 = 0)

template <int NC>
struct ChebTabN {
    float4 c[NC][kChebMom];         // [candidate][n] = C_n0..C_n3 times (-1)^{floor(n/2)} / n!
    float mid[NC];                  // channel centre relative to the CUT
    float invh[NC];                 // 1 / (B_c / 2)
    int ok;
};
using ChebTab = ChebTabN<kMaxCand>;

// (-1)^{floor(n/2)} / n!
__host__ __device__ constexpr double cheb_fold(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f /= (double)i;
    return ((n >> 1) & 1) ? -f : f;
}

// 2^x for an FP64 exponent: the integer part goes to the FP32 exponent field,
// the fraction (|f| <= 1/2, exact in FP32 to 1e-16 absolute) to ex2.approx.
__device__ __forceinline__ float exp2_split(double x)
{
    const double xr = rint(x);
    if (xr < -126.0) return 0.0f;
    const float sc = __int_as_float(((int)fmin(xr, 127.0) + 127) << 23);
    return ex2_approx((float)(x - xr)) * sc;
}

// The Chebyshev coefficients of e^{a x} on [-1, 1]: I0(a), 2 I1(a), 2 I2(a),
// 2 I3(a) from their power series (|a| <= 0.05: the terms kept are exact to
// FP32 rounding).
__device__ __forceinline__ float4 bessel_b4(float a)
{
    const float t = 0.5f * a, t2 = t * t;
    return make_float4(1.0f + t2 * (1.0f + t2 * (0.25f + t2 * (1.0f / 36.0f))),              // I0
                       2.0f * t * (1.0f + t2 * (0.5f + t2 * (1.0f / 12.0f))),                 // 2 I1
                       2.0f * t2 * (0.5f + t2 * (1.0f / 6.0f + t2 * (1.0f / 48.0f))),         // 2 I2
                       2.0f * t2 * t * (1.0f / 6.0f + t2 * (1.0f / 24.0f + t2 * (1.0f / 240.0f)))); // 2 I3
}

// The four weights of step m for a candidate (F0 its channel centre, h its
// half-width, at its attenuation term): W_k(m) = 2^{A2d_m + K2_m F0 - at z_m}
// times the k-th Chebyshev coefficient of e^{K2_m ln2 h x} on [-1, 1]
// (I0, 2 I1, 2 I2, 2 I3).  The exponent is formed in FP64, so the weight is
// exact to FP32 rounding.
__device__ __forceinline__ float4 cheb_w4(float4 a, double F0, float h, double at)
{
    const float base = exp2_split((double)a.x - at * (double)a.z + (double)a.y * F0);
    const float t = 0.5f * a.y * h * 0.69314718f, t2 = t * t;
    return make_float4(base * (1.0f + t2 * (1.0f + t2 * (0.25f + t2 * (1.0f / 36.0f)))),                  // I0
                       base * (2.0f * t * (1.0f + t2 * (0.5f + t2 * (1.0f / 12.0f)))),                     // 2 I1
                       base * (2.0f * t2 * (0.5f + t2 * (1.0f / 6.0f + t2 * (1.0f / 48.0f)))),             // 2 I2
                       base * (2.0f * t2 * t * (1.0f / 6.0f + t2 * (1.0f / 24.0f + t2 * (1.0f / 240.0f))))); // 2 I3
}

// Moment sums of one candidate for n in [N0, N0 + NN) over the steps
// [m0, m1): s[n][k] = sum_m W_k(m) g_n(m), with g_n(m) from gtab (kZsG float4
// per step).  The weights come from sWc (one float4 per step, cheb_w4) when
// it is given, else they are formed here from sT.
template <int N0, int NN>
__device__ __forceinline__ void cheb_sums(const float4 *gtab, const float4 *sT, const float4 *sWc, int m0, int m1,
                                          double F0, float h, double at, int lane, float4 *out)
{
    float s[NN][4];
#pragma unroll
    for (int n = 0; n < NN; ++n) s[n][0] = s[n][1] = s[n][2] = s[n][3] = 0.0f;
    auto add = [&](const float4 W, int m) {
        const float *g = reinterpret_cast<const float *>(gtab + kZsG * m) + N0;
#pragma unroll
        for (int n = 0; n < NN; ++n) {
            const float gn = g[n];
            s[n][0] = fmaf(W.x, gn, s[n][0]);
            s[n][1] = fmaf(W.y, gn, s[n][1]);
            s[n][2] = fmaf(W.z, gn, s[n][2]);
            s[n][3] = fmaf(W.w, gn, s[n][3]);
        }
    };
    if (sWc) {
        for (int m = m0 + lane; m < m1; m += 32) add(sWc[m], m);
    } else {
        for (int m = m0 + lane; m < m1; m += 32) add(cheb_w4(sT[m], F0, h, at), m);
    }
#pragma unroll
    for (int n = 0; n < NN; ++n) {
        const float f = (float)cheb_fold(N0 + n);
        float v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float x = s[n][j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            v[j] = x * f;
        }
        if (lane == 0) out[n] = make_float4(v[0], v[1], v[2], v[3]);
    }
}

// Whether the contracted small-phase tables apply to this piece (block
// uniform): the centred step moments exist and every candidate channel is
// narrow enough for the 4-term Chebyshev series of e^{kappa F_c}.
__device__ __forceinline__ bool cheb_applies(const QuadParams &qp, const DevPiece &pc, int prof,
                                             const PieceConst<float> &k)
{
    const int coff = qp.plan_ch_off[pc.plan];
    const double kapL = qp.kap_L ? qp.kap_L[prof] : 1e30;
    double hmax = 0.0;
    for (int c = 0; c < k.nc; ++c) hmax = fmax(hmax, 0.5 * qp.ch_B[coff + pc.c_lo + c]);
    return qp.zs_g != nullptr && kapL * hmax <= (double)kChebMaxA;
}

// The step weights of the first nW candidates of the piece into sW[c M + m]
// (all threads; the caller syncs before the tables are built from them).
__device__ __forceinline__ void cheb_weights(const QuadParams &qp, const DevPiece &pc, const float4 *sT, int M,
                                             const PieceConst<float> &k, int nW, float4 *sW)
{
    const int coff = qp.plan_ch_off[pc.plan];
    for (int t = threadIdx.x; t < nW * M; t += blockDim.x) {
        const int c = t / M, m = t - c * M;
        const double F0 = qp.ch_frel[coff + pc.c_lo + c];
        const double h = 0.5 * qp.ch_B[coff + pc.c_lo + c];
        sW[t] = cheb_w4(sT[m], F0, (float)h, (double)(k.at_ab + k.hat[c]));
    }
}

// Called by every thread of the block after piece_consts; the caller syncs.
// sT[m] = {A2d_m, K2_m, z_m, .}; qp.zs_g[kZsG m ...] = g_0..g_19 of step m.
// For the first NC candidates of the piece, one warp per (candidate, group of
// up to 6 moments) fills nu_0..nu_{NM-1}; the step weights are exact to FP32
// rounding (FP64 exponent), read from sW for the first nW candidates
// (cheb_weights) and formed per moment group for the rest; the sums run over
// the lane's steps and a warp tree.
template <int NM, int NC>
__device__ __forceinline__ bool cheb_setup(const QuadParams &qp, const DevPiece &pc, int prof,
                                           const float4 *sT, int M, const PieceConst<float> &k, ChebTabN<NC> &ct,
                                           const float4 *sW = nullptr, int nW = 0)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int coff = qp.plan_ch_off[pc.plan];
    const bool ok = cheb_applies(qp, pc, prof, k);
    if (threadIdx.x == 0) ct.ok = ok ? 1 : 0;
    if (!ok) return false;
    const int ncs = k.nc < NC ? k.nc : NC;
    static_assert(NM > 6 && NM <= kChebMom, "moment count");
    constexpr int ng = NM <= 12 ? 2 : 3;     // moment groups of at most 6
    // one warp per (candidate, moment group), so that small pieces do not
    // wait on one warp per candidate
    for (int t = warp; t < ncs * ng; t += nw) {
        const int c = t / ng, gr = t - c * ng;
        const double F0 = qp.ch_frel[coff + pc.c_lo + c];
        const double h = 0.5 * qp.ch_B[coff + pc.c_lo + c];
        const double at = (double)(k.at_ab + k.hat[c]);
        const float4 *sWc = c < nW ? sW + (size_t)c * M : nullptr;
        if (gr == 0) {
            cheb_sums<0, 6>(qp.zs_g, sT, sWc, 0, M, F0, (float)h, at, lane, ct.c[c]);
            if (lane == 0) {
                ct.mid[c] = 0.5f * (k.lo[c] + k.hi[c]);
                ct.invh[c] = (float)(1.0 / h);
            }
        } else if (gr == 1) {
            cheb_sums<6, (NM <= 12 ? NM - 6 : 6)>(qp.zs_g, sT, sWc, 0, M, F0, (float)h, at, lane, ct.c[c] + 6);
        } else if constexpr (NM > 12) {
            cheb_sums<12, NM - 12>(qp.zs_g, sT, sWc, 0, M, F0, (float)h, at, lane, ct.c[c] + 12);
        }
    }
    return true;
}

// Folded moments nu'_n (n < NM) of a point in candidate ci at u = F_c - f_i.
template <int NM, int NC>
__device__ __forceinline__ void cheb_moments(const ChebTabN<NC> &ct, int ci, float u, float (&nu)[NM], float &x)
{
    x = (u - ct.mid[ci]) * ct.invh[ci];
    const float T2 = fmaf(2.0f * x, x, -1.0f);
    const float T3 = fmaf(2.0f * x, T2, -x);
#pragma unroll
    for (int n = 0; n < NM; ++n) {
        const float4 c = ct.c[ci][n];
        nu[n] = fmaf(c.w, T3, fmaf(c.z, T2, fmaf(c.y, x, c.x)));
    }
}

// A = sum_{n even} phi^n nu'_n, B = sum_{n odd} phi^n nu'_n, |S|^2 = A^2 + B^2.
template <int NM>
__device__ __forceinline__ void cheb_AB(const float (&nu)[NM], float phi, float &A, float &B)
{
    const float p2 = phi * phi;
    constexpr int ne = (NM + 1) / 2, no = NM / 2;
    A = nu[2 * (ne - 1)];
#pragma unroll
    for (int i = ne - 2; i >= 0; --i) A = fmaf(A, p2, nu[2 * i]);
    float b = nu[2 * (no - 1) + 1];
#pragma unroll
    for (int i = no - 2; i >= 0; --i) b = fmaf(b, p2, nu[2 * i + 1]);
    B = phi * b;
}

// A and B of a contracted point of the 2-D series of the tabulated
// (Raman-ODE) profile: C[4 n + k] = {c_nk0..c_nk3}, nu_n = sum_{k,l} c_nkl
// T_k(x) T_l(y) for the point's in-channel offsets (x, y), n < NM.
template <int NM>
__device__ __forceinline__ void cheb2_AB(const float4 *C, float x, float y, float phi, float &A, float &B)
{
    const float Tx2 = fmaf(2.0f * x, x, -1.0f), Tx3 = fmaf(2.0f * x, Tx2, -x);
    const float Ty2 = fmaf(2.0f * y, y, -1.0f), Ty3 = fmaf(2.0f * y, Ty2, -y);
    float nu[NM];
#pragma unroll
    for (int n = 0; n < NM; ++n) {
        float r[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 c = C[n * 4 + k];
            r[k] = fmaf(c.w, Ty3, fmaf(c.z, Ty2, fmaf(c.y, y, c.x)));
        }
        nu[n] = fmaf(r[3], Tx3, fmaf(r[2], Tx2, fmaf(r[1], x, r[0])));
    }
    cheb_AB<NM>(nu, phi, A, B);
}

// A and B of a contracted point with as many moments as its phase needs:
// the omitted orders of the centred series are below (|phi| L / 2)^n / n!
// of the kept ones, so 6 moments serve |phi| L <= 0.2, 11 serve |phi| L <= 2
// and 19 the rest of the contracted range (rows of the grid have nearly
// constant phi, so a warp seldom splits between the forms).
template <int NC>
__device__ __forceinline__ void cheb_point(const ChebTabN<NC> &ct, int ci, float u, float phi, float aphi,
                                           float phi6, float phi11, float &x, float &A, float &B)
{
    if (aphi <= phi6) {
        float nu[6];
        cheb_moments<6>(ct, ci, u, nu, x);
        cheb_AB<6>(nu, phi, A, B);
    } else if (aphi <= phi11) {
        float nu[11];
        cheb_moments<11>(ct, ci, u, nu, x);
        cheb_AB<11>(nu, phi, A, B);
    } else {
        float nu[kChebMom];
        cheb_moments<kChebMom>(ct, ci, u, nu, x);
        cheb_AB<kChebMom>(nu, phi, A, B);
    }
}

// ---------------------------------------------------------------------------
// Segmented small-phase series (forward FP32).  Cut the span at step edges
// into segments s with centres c_s; each segment's part of Eq. slow_vary is,
// exactly as for the whole span,
//   S_s = e^{j phi c_s} sum_n (j phi)^n / n! nu_n^s,  nu_n^s = sum_{m in s} w_m g_n^s(m),
// g_n^s(m) the mean of (zeta - c_s)^n over step m, and S = sum_s S_s.  With
// |phi| (segment length) <= 6 the 19-moment truncation stays below 2e-8 of
// each part, so a point that is too fast for the whole-span series but slow
// enough for 2, 4 or 8 segments costs 2, 4 or 8 series evaluations (and as
// many phasors) instead of a walk over all steps.  The moments are contracted
// in F_c as in cheb_setup, per piece, candidate and segment.
// ---------------------------------------------------------------------------
constexpr int kSegCand = 3;          // F_c candidates with segment tables

struct SegTab {
    float4 c[kSegCand][kSegSlots][kChebMom];   // as ChebTab.c, per segment
    float hi[kSegSlots], lo[kSegSlots];        // segment centre / 2pi (float-float)
};

// Called by every thread after cheb_setup (ct.ok block-uniform); the caller
// syncs.  One warp per (candidate, segment); the step weights of the first nW
// candidates come from sW as in cheb_setup.
__device__ __forceinline__ void seg_setup(const QuadParams &qp, const DevPiece &pc, const float4 *sT, int M,
                                          const PieceConst<float> &k, SegTab &sg, const float4 *sW = nullptr,
                                          int nW = 0)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int coff = qp.plan_ch_off[pc.plan];
    const int ncs = k.nc < kSegCand ? k.nc : kSegCand;
    if (threadIdx.x < kSegSlots) {
        const int4 si = qp.seg[threadIdx.x];
        sg.hi[threadIdx.x] = __int_as_float(si.z);
        sg.lo[threadIdx.x] = __int_as_float(si.w);
    }
    for (int t = warp; t < ncs * kSegSlots; t += nw) {
        const int c = t / kSegSlots, sl = t - c * kSegSlots;
        const int lv = sl < 2 ? 0 : (sl < 6 ? 1 : 2);
        const int4 si = qp.seg[sl];
        const float4 *gtab = qp.zs_gseg + (size_t)lv * M * kZsG;
        const double F0 = qp.ch_frel[coff + pc.c_lo + c];
        const double h = 0.5 * qp.ch_B[coff + pc.c_lo + c];
        const double at = (double)(k.at_ab + k.hat[c]);
        float4 *out = sg.c[c][sl];
        const float4 *sWc = c < nW ? sW + (size_t)c * M : nullptr;
        cheb_sums<0, 6>(gtab, sT, sWc, si.x, si.y, F0, (float)h, at, lane, out);
        cheb_sums<6, 6>(gtab, sT, sWc, si.x, si.y, F0, (float)h, at, lane, out + 6);
        cheb_sums<12, kChebMom - 12>(gtab, sT, sWc, si.x, si.y, F0, (float)h, at, lane, out + 12);
    }
}

// |S|^2 of a point of candidate ci at in-channel coordinate x (T2, T3 its
// Chebyshev values) from the segments [s0, s1).
__device__ __forceinline__ float seg_s2(const SegTab &sg, int ci, int s0, int s1, float x, float T2, float T3,
                                        float phi)
{
    float Sr = 0.0f, Si = 0.0f;
    for (int s = s0; s < s1; ++s) {
        float nu[kChebMom];
        const float4 *C = sg.c[ci][s];
#pragma unroll
        for (int n = 0; n < kChebMom; ++n) {
            const float4 c = C[n];
            nu[n] = fmaf(c.w, T3, fmaf(c.z, T2, fmaf(c.y, x, c.x)));
        }
        float A, B;
        cheb_AB<kChebMom>(nu, phi, A, B);
        float sn, cs;
        phasor_rev_ff(phi, sg.hi[s], sg.lo[s], sn, cs);
        Sr = fmaf(cs, A, fmaf(-sn, B, Sr));
        Si = fmaf(sn, A, fmaf(cs, B, Si));
    }
    return fmaf(Sr, Sr, Si * Si);
}

}  // namespace isrs
