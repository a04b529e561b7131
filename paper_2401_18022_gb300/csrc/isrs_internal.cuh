// Internal device-side structures of the ISRS GN library (not part of the ABI).
//
// Layout in HBM (all buffers owned by the handle):
//   plan tables   per channel, plans concatenated:  f_rel (f - f_ref), B, alpha, gamma, nf
//   pieces        DevPiece[], plans concatenated; per CUT contiguous
//   items         DevItem[]: work queue of (profile, piece range) tiles, ordered by
//                 (profile, CUT) so that each CUT owns a contiguous item range
//   z tables      per step m: z_m, dz_m, log2 dz_m, the centred step moments and
//                 the edge phase z_{m+1}/2pi (float-float)
//   profile tabs  per profile and step: float2 {A2_m, K2_m}; per profile and
//                 channel: P/B (float, double), lnrho(L, f_c)
//   partials      one double per item
#pragma once
#include <cstdint>
#include "isrs_debug.cuh"

namespace isrs {

constexpr int kMaxCand = 16;        // max channels a piece's F_c range may touch
constexpr int kMaxSteps = 2048;     // max z-steps (n_edges - 1)
constexpr int kMaxG = 4096;         // max grid points per dimension
constexpr int kMaxRamanCh = 2048;   // max channels of a plan with the Raman-ODE profile
constexpr int kMaxRamanGradCh = 1536;   // ... and of its gradient (shared memory of the ODE adjoint)
constexpr int kSegLevels = 3;       // segmented small phase: 2, 4 and 8 segments ...
constexpr int kSegSlots = 14;       // ... 14 segments in all
constexpr int kSegMinG = 160;       // ... used from G = 160: their tables cost a fixed time per piece,
                                    // which the few points they serve repay only on large pieces
constexpr double kPi = 3.14159265358979323846;
constexpr double kLog2e = 1.44269504088896340736;

// One rectangular piece of a channel-pair cell clipped to a quadrant:
// |f1| in [xlo, xhi], |f2| in [ylo, yhi], f1 = s1 |f1|, f2 = s2 |f2|,
// F_a = f_i + f1 in channel a, F_b = f_i + f2 in channel b, and F_c = f_i +
// f1 + f2 can only fall in channels c_lo..c_hi.  mult = 2 when the mirror
// piece (f1 <-> f2) is folded in.  Channel indices are plan-local.
struct DevPiece {
    double xlo, xhi, ylo, yhi;
    int cut, a, b, c_lo;
    int c_hi, flags, plan, pad;   // flags bit0: s1 < 0, bit1: s2 < 0
    float mult, pad2, pad3, pad4;
};
static_assert(sizeof(DevPiece) == 80, "DevPiece layout");

// One work tile: pieces [piece0, piece1) of one CUT for one profile.
struct DevItem {
    int prof;
    int piece0;
    int piece1;
    int cut;        // plan-local CUT index (for bookkeeping)
};

// Per-launch constants of the quadrature kernels.
struct QuadParams {
    const DevPiece *pieces;
    const DevItem *items;
    int n_items;
    int n_pieces;
    unsigned *dbg;              // debug build: code of the first failed bounds check (else null)
    int G;
    int n_steps;
    double eps_v1;
    // fibre
    double beta2, beta3, beta4;
    // per plan channel tables (concatenated, index plan_ch_off[plan] + c)
    const double *ch_frel;      // f_c - f_ref
    const double *ch_B;
    const double *ch_alpha;     // 1/km
    const int *plan_ch_off;
    // per profile channel tables (index prof_ch_off[prof] + c)
    const float *pd_f;          // P/B
    const double *pd_d;
    const int *prof_ch_off;
    const int *prof_plan;
    // per profile step tables (index prof * n_steps + m)
    const float2 *step_f;       // {A2_m, K2_m}: log2 p = A2 + K2 (F_c - f_ref) - at2 z_m
    const double2 *step_d;      // {ln Ptot - ln N_m, kappa_m}
    // z tables (per step m)
    const float4 *zs_a;         // {z_m, z_m^2 + dz_m^2/12, log2 dz_m, dz_m}
    const float4 *zs_b;         // {z_{m+1}/2pi hi, lo (float-float), z_m/2pi, 0}
    const double2 *zs_d;        // {z_m, dz_m}
    const float4 *zs_g;         // [5 per step] g_0..g_19: mean of (zeta - L/2)^n over step m (g_19 = 0)
    // segmented small-phase series (forward FP32): the span cut at step edges
    // into 2, 4 and 8 segments (kSegLevels levels, kSegSlots segments in all);
    // per level and step the moments about the step's segment centre, and per
    // segment its steps and centre in revolutions (float-float).  Null: off.
    const float4 *zs_gseg;      // [kSegLevels][M][5]
    const int4 *seg;            // [kSegSlots] {m0, m1, bits of centre/2pi hi, lo}
    float phi_seg[3];           // per level: |phi| limit [rad/km] (6 / longest segment)
    const double *kap_L;        // per profile: kappa(L) [1/THz]
    float dz_max;
    float L;                    // span length [km]
    int n_spans;                // identical spans (array factor when > 1)
    float Lrev_hi, Lrev_lo;     // L / 2pi as a float-float pair
    double Ld;                  // L in double (FP64 path)
    // outputs / scheduling
    double *partial;            // one per item
    int *counter;               // persistent work counter (zeroed before launch)
    int *err_flag;
    unsigned long long *path_count;   // [3] grid points per z-sum form (small, direct, telescoped)
    // tabulated profile (Raman ODE): per profile, channel and step {a, b} with
    // ln rho(z_m, F) = a + b (F - f_c) inside channel c; index
    // (prof_ch_off[prof] + c) * n_steps + m.  Null for the closed-form profile.
    const double2 *ab;
    const float2 *ab_f;         // MCI cells (FP32): {a, b} / 2 * log2(e), same index (k_tab_half_log2)
    int nc_max;                 // largest F_c candidate count of any piece
    // multi-channel-interference cells (k_quad_mci_*): items are cell ranges
    // of one CUT (DevItem.piece0/piece1 = triangular cell indices), G = G_mci
    const int *plan_n;          // channels per plan
    int mci_n_max;              // largest plan
    int mci_cpc;                // tabulated profile (FP32): cells per chunk of k_quad_mci_f32_tab
};

}  // namespace isrs
