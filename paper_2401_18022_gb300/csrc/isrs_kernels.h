// Internal launcher interface between the host API and the CUDA kernels.
#pragma once
#include <cuda_runtime.h>

#include "isrs_internal.cuh"

namespace isrs {

struct PrepParams {
    const double *P;            // per profile channel powers (prof_ch_off)
    const double *ch_frel, *ch_B, *ch_alpha;
    const int *plan_ch_off, *plan_n, *prof_ch_off, *prof_plan;
    const double2 *zs_d;        // {z_m, dz_m}
    int n_steps;
    double L, Cr, alpha_R;
    // outputs
    double *pd_d;
    float *pd_f;
    double2 *step_d;
    float2 *step_f;
    double *lnrho_L;
    double *ptot;
    double *kap_L;              // kappa(L) per profile (the largest ISRS exponent slope)
};

struct FinishParams {
    const double *partial;
    const int2 *slot_items;     // per output slot: item range
    const double *partial2;     // MCI cell items (nullable)
    const int2 *slot_items2;    // per output slot: MCI item range (nullable)
    const int *slot_cut;        // per output slot: plan-local CUT index
    const int *prof_slot_off;   // [n_prof + 1]
    const int *prof_plan, *plan_ch_off, *prof_ch_off;
    const double *ch_gamma, *ch_B, *ch_frel, *ch_nf;
    const unsigned char *guard;
    const double *P;
    const double *lnrho_L;
    double f_ref;
    double snr_trx_lin_inv;     // 10^(-SNR_TRX/10) or 0
    double n_spans;             // ASE adds over the span amplifiers
    // outputs (indexed by slot; any may be null)
    double *sigma, *pnli, *eta, *snr, *pase;
    double *T;                  // per profile
};

// Adjoint of the FP32 quadrature (single profile): per work tile the step
// buckets {R_m, R'_m} and the PSD buckets V of every channel (the tile's own
// row, written only by its block; k_v_reduce sums a CUT's rows in tile order).
struct AdjParams {
    QuadParams q;
    double2 *item_R;            // [n_items x n_steps]
    double *V;                  // [n_items x n_ch]
    const int *item_slot;       // output slot of each item
    int n_ch;
    double *Yg;                 // per block and warp: FP64 contracted bucket sums (adjoint_scratch_bytes)
};

// Chain rule from the buckets to dT/dP_j (FP64, single profile).  The
// buckets may cover a shard of the CUTs (n_slots output slots, slot_cut maps
// a slot to its channel); SNR, P_NLI, P_ASE, ybar and aase are per channel.
struct ChainParams {
    const double *P, *ch_frel, *ch_B, *ch_gamma, *ch_nf;
    const double2 *zs_d;        // {z_m, dz_m}
    const double2 *step_d;      // {lnPtot - lnN_m, kappa_m}
    const double *snr, *pnli, *pase, *lnrho_L;   // [n_ch]
    const double2 *item_R;
    const double *V;            // [n_slots x n_ch] PSD buckets per output slot (from Vt)
    const double *Vt;           // [(n_items) x n_ch] PSD buckets per tile (regular, then MCI tiles)
    double *Vs;                 // = V, written by k_v_reduce
    const int2 *slot_items;     // per slot: regular tile range
    const int2 *slot_items2;    // per slot: MCI tile range (nullable), offset by n_items_reg
    int n_items_reg;
    const int *item_slot, *slot_cut;
    int n_items, n_slots, n_ch, n_steps;
    int with_direct;            // add the terms outside the buckets (ASE gain, SNR numerator)
    double L, Cr, alpha_R, f_ref, snr_trx_lin_inv, n_spans;
    double *ybar;               // [n_ch] dT/dSigma_i
    double *aase;               // [n_ch] dT/dASE_i * dASE_i/d ln G_i
    double2 *Rb;                // [n_steps] sum over the shard's tiles of ybar_i {R_im, R'_im}
    double *cs;                 // [4 (n_steps + 1) + 4] profile terms per step (ln N, kappa, L_eff, Fbar), then
                                // the channel-independent sums of the chain rule
    double *dT_dP;              // [n_ch]
};

// SNR, P_NLI, P_ASE and throughput of every channel from a given eta (the
// second phase of a gradient split by CUT shards).
struct SnrFromEtaParams {
    const double *eta, *P, *ch_B, *ch_frel, *ch_nf, *lnrho_L;
    const unsigned char *guard;
    double f_ref, snr_trx_lin_inv, n_spans;
    int n;
    double *snr, *pnli, *pase, *T;
};
cudaError_t launch_snr_from_eta(const SnrFromEtaParams &sp, cudaStream_t st);

// Raman-ODE profile (one block per profile): RK4 on y = ln P through the
// edge -> midpoint -> edge nodes of every z-step, then the tables {a, b}.
struct RamanParams {
    const double *P;            // per profile channel powers (prof_ch_off)
    const double *ch_frel, *ch_alpha, *ch_scale;   // plan-concatenated
    const int *win_lo, *win_hi; // per plan channel: first / last partner (plan-local)
    const int *plan_ch_off, *plan_n, *prof_ch_off, *prof_plan;
    const double2 *zs_d;        // {z_m, dz_m}
    const int *half_steps;      // per z-step: RK4 steps in each half
    int n_steps;
    double f_ref, Cr;
    int photon;
    double2 *ab;                // out: (prof_ch_off[p] + c) * n_steps + m -> {a, b}
    double *lnrho_L;            // out: prof_ch_off[p] + c
    double *y_nodes;            // out (nullable, profile 0 only): state before every RK4 step and at L
};

// Discrete adjoint of the Raman ODE and of the profile tables (single
// profile): from dT/d{a, b} (per channel and step) and dT/d ln rho(L) to
// dT/dP through the RK4 steps (states of k_raman_ode's y_nodes), then the
// total gradient with the PSD and SNR-numerator terms.
struct RamanAdjParams {
    RamanParams r;              // the forward's tables (profile 0)
    int n;                      // channels
    int n_rk;                   // RK4 steps
    const double *y_nodes;      // [(n_rk + 1) x n]
    const double2 *gAB;         // [n x n_steps] dT/da, dT/db
    double *gAt;                // [n x n_steps] scratch: dT/da with the slope stencil folded in
    const double *aase;         // [n] dT/d ln G_i (G = 1/rho(L))
    const double *gV;           // [n] dT/d ln P_j through the PSD products
    const double *snr, *pnli, *pase, *ch_B;
    int with_direct;            // add the terms outside every eta (ASE gain, SNR numerator); a CUT
                                // shard of a split gradient leaves them to one rank
    double *dT_dP;              // [n]
};

// Fused forward + adjoint of the FP32 quadrature with the tabulated profile
// (single profile): per work tile the forward partial of Sigma_i and, for
// every plan channel the tile's pieces touch, dSigma_i/d{a, b}(m) and
// dSigma_i/d ln P through the PSD products (unscaled: the gather applies
// dT/dSigma_i).
struct AdjTabParams {
    QuadParams q;
    const int *row_off;         // [n_items + 1] first row of each tile
    const int4 *prow;           // [n_pieces] local rows {a, b, CUT, first F_c candidate}
    double2 *rows;              // [n_rows x n_steps] {dSigma/da, dSigma/db}
    double *rowsV;              // [n_rows] dSigma/d ln P
};

// dT/d{a, b} and dT/d ln P (PSD) per plan channel: the tile rows of each
// channel times dT/dSigma of the tile's CUT, summed in tile order.
struct TabGatherParams {
    const int *gath_off;        // [n_ch + 1]
    const int2 *gath;           // (row, output slot)
    const double2 *rows;
    const double *rowsV;
    const double *ybar;         // [n_ch] dT/dSigma_i
    const int *slot_cut;
    int n_ch, n_steps;
    double2 *gAB;               // [n_ch x n_steps]
    double *gV;                 // [n_ch]
};
cudaError_t launch_tab_gather(const TabGatherParams &gp, cudaStream_t st);

size_t adjoint_tab_smem_bytes(int n_steps, int G, int nc_max, int block);
int adjoint_tab_blocks_per_sm(int n_steps, int G, int nc_max, int block);
cudaError_t launch_adjoint_tab(const AdjTabParams &ap, int grid, int block, cudaStream_t st);
cudaError_t launch_ybar(const ChainParams &cp, cudaStream_t st);

size_t raman_smem_bytes(int n_ch);
size_t raman_adj_smem_bytes(int n_ch);
cudaError_t launch_raman_adj(const RamanAdjParams &ap, cudaStream_t st);
cudaError_t launch_raman(const RamanParams &rp, int n_prof, int max_n, cudaStream_t st);
size_t quad_smem_bytes(int precision, int n_steps, int G);
int quad_blocks_per_sm(int precision, int n_steps, int G, int block);
cudaError_t launch_prep(const PrepParams &pp, int n_prof, cudaStream_t st);
cudaError_t launch_quad(const QuadParams &qp, int precision, int grid, int block, cudaStream_t st);
// the same quadratures with the tabulated profile (qp.ab set)
size_t quad_tab_smem_bytes(int precision, int n_steps, int G, int nc_max);
int quad_tab_blocks_per_sm(int precision, int n_steps, int G, int nc_max, int block);
cudaError_t launch_quad_tab(const QuadParams &qp, int precision, int grid, int block, cudaStream_t st);
cudaError_t launch_finish(const FinishParams &fp, int n_prof, cudaStream_t st);
// MCI cells with their own grid (closed-form profile)
size_t quad_mci_smem_bytes(int precision, int n_steps, int n_max);
int quad_mci_blocks_per_sm(int precision, int n_steps, int n_max, int block);
cudaError_t launch_quad_mci(const QuadParams &qp, int precision, int grid, int block, cudaStream_t st);
// ... with the tabulated (Raman-ODE) profile: qp.ab (FP64 kernel) or qp.ab_f
// (FP32 kernel, filled by launch_tab_half_log2) and qp.mci_cpc cells per chunk
// (quad_mci_tab_cells; 0: the step rows do not fit shared memory)
int quad_mci_tab_cells(int n_steps, int n_max, int G, int block);
size_t quad_mci_tab_smem_bytes(int precision, int n_steps, int n_max, int cpc);
int quad_mci_tab_blocks_per_sm(int precision, int n_steps, int n_max, int cpc, int block);
cudaError_t launch_tab_half_log2(const double2 *ab, float2 *abf, int n, int n_sms, cudaStream_t st);
cudaError_t launch_quad_mci_tab(const QuadParams &qp, int precision, int grid, int block, cudaStream_t st);
size_t adjoint_smem_bytes(int n_steps, int G, int block);
size_t adjoint_scratch_bytes(int grid);   // AdjParams.Yg of a launch of `grid` blocks
// adjoint over the MCI cells of a separate grid (closed-form profile)
size_t adjoint_mci_smem_bytes(int n_steps, int n_max, int block);
int adjoint_mci_blocks_per_sm(int n_steps, int n_max, int block);
cudaError_t launch_adjoint_mci(const AdjParams &ap, int grid, int block, cudaStream_t st);
int adjoint_blocks_per_sm(int n_steps, int G, int block);
cudaError_t launch_adjoint(const AdjParams &ap, int grid, int block, cudaStream_t st);
cudaError_t launch_chain(const ChainParams &cp, cudaStream_t st);

}  // namespace isrs
