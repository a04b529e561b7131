/*
 * isrs_gn.h -- C ABI of the GB300 (sm_103a) ISRS Gaussian-noise integral
 * model of arXiv 2401.18022 (Jarmolovicius et al., "Optimising O-to-U band
 * transmission using fast ISRS Gaussian noise numerical integral model").
 *
 * The library computes, for every channel under test (CUT) i of a WDM plan,
 * the nonlinear-interference (NLI) coefficient eta_i of App. A, Eqs.
 * gain_fin / psi_fin: the frequency double integral of the ISRS GN model,
 * split into quadrants (Eqs. q1a..q4d) and evaluated as a Riemann sum in
 * hyperbolic coordinates (Eqs. q1..q4), with the power profile term p of
 * Eq. pk, the phase mismatch of Eq. phi (beta2, beta3, beta4) and the
 * slowly-varying-power z-sum of Eq. slow_vary.  From eta it derives the SNR
 * and Shannon throughput of Sec. IV, Eq. loss, and the gradient of that
 * throughput with respect to the per-channel launch powers.
 *
 * Units: frequency THz, length km, power W, beta_k in ps^k/km,
 * alpha in 1/km (power), gamma in 1/(W km), C_r in 1/(W km THz).
 *
 * Conventions for every call:
 *  - No C++ exception crosses this boundary; every call returns an
 *    isrs_status.  On error nothing is written to the outputs and
 *    isrs_last_error() describes the cause.
 *  - Channel-plan arrays (isrs_channels) are HOST pointers, read during the
 *    call only.  Channels must be sorted by frequency and disjoint.
 *  - Launch powers and per-channel outputs may be host or device pointers;
 *    the library detects which (cudaPointerGetAttributes).  Device pointers
 *    must belong to the handle's device (device memory of another GPU is
 *    INVALID_ARG).  With device outputs the call is asynchronous on `stream`;
 *    with any host output it synchronises `stream` before returning.
 *  - The compute calls read the launch powers back for validation and may
 *    synchronise `stream`, so they cannot run on a stream that is being
 *    captured into a CUDA graph: there they return ISRS_ERR_UNSUPPORTED
 *    before issuing any work.  isrs_gn_eta_batched captures and replays its
 *    own graph internally.
 *  - The caller owns all input and output buffers.  The handle owns its
 *    device workspace and a cache of per-plan tables (pieces, z-grid).  A
 *    handle must not be used from two host threads at once.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).
 */
#ifndef ISRS_GN_H
#define ISRS_GN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ISRS_OK = 0,
    ISRS_ERR_INVALID_ARG = 1,   /* argument outside the documented domain */
    ISRS_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    ISRS_ERR_ALLOC = 3,         /* device or host allocation failed */
    ISRS_ERR_TIMEOUT = 4,       /* reserved: no kernel here waits on a flag, peer or grid barrier */
    ISRS_ERR_NUMERIC = 5,       /* non-finite intermediate (e.g. overflow) */
    ISRS_ERR_UNSUPPORTED = 6,   /* valid but not supported by this build */
    ISRS_ERR_CHECK = 7          /* a device bounds check of the debug build failed (see isrs_debug_build) */
} isrs_status;

typedef struct isrs_handle_s *isrs_handle;

/* Cell sets (which channel-pair cells (a,b) of the (f1,f2) plane of a CUT
 * are integrated; F_a = f_i + f1 in channel a, F_b = f_i + f2 in channel b). */
#define ISRS_CELLS_SCI_XCI 0   /* a == i or b == i: self- and cross-channel */
#define ISRS_CELLS_ALL     1   /* every cell: adds multi-channel interference */

/* Arithmetic of the quadrature kernel. */
#define ISRS_PREC_FP32 0       /* FP32 bulk, float-float phase, compensated sums */
#define ISRS_PREC_FP64 1       /* plain FP64 throughout (reference GPU path) */

/* Power-profile models (the rho(z, f) of Eq. pk). */
#define ISRS_PROFILE_CLOSED_FORM 0   /* linear Raman slope, closed form */
#define ISRS_PROFILE_RAMAN_ODE   1   /* Raman power-evolution ODEs (RK4) */

/* Fibre of one span (Sec. II; App. A).  beta_k are the Taylor coefficients of
 * the propagation constant at f_ref (Eqs. d, d_slope, d_curve).  alpha_R sets
 * the equal-power-drop z-grid.  Power profile:
 *  - ISRS_PROFILE_CLOSED_FORM: the ISRS solution for a linear Raman gain
 *    slope C_r over the whole band, L_eff(z) = (1 - exp(-alpha_R z))/alpha_R,
 *    normalised by the integral of the transmitted PSD;
 *  - ISRS_PROFILE_RAMAN_ODE: the Raman power-evolution ODEs of Sec. III /
 *    App. A for the channel powers (each channel a line at f_c):
 *      dy_i/dz = -alpha_i + s_i C_r sum_k h(f_k, f_i) P_k,  y = ln P,
 *      h = f_k - f_i for 0 < f_k - f_i <= raman_max_THz (k pumps i),
 *      h = (f_k - f_i) f_i / f_k for 0 < f_i - f_k <= raman_max_THz (i pumps
 *          k; the ratio f_i/f_k is 1 when raman_photon is 0),
 *      h = 0 beyond raman_max_THz (<= 0: no cut-off),
 *    s_i = isrs_channels.raman_scale[i] (the effective-area ratio
 *    Aeff(f_ref)/Aeff(f_i); 1 when NULL), solved by classical RK4 (step
 *    bound isrs_quad.ode_h_km) through the midpoint of every z-step; inside
 *    channel c, ln rho(z_m, F) = ln rho_c(z_m) + b_c(z_m) (F - f_c) with b_c
 *    the central difference of ln rho + alpha z over the neighbouring
 *    channels.  At most 2048 channels per plan. */
typedef struct {
    double L_km;
    double f_ref_THz;
    double beta2, beta3, beta4;
    double Cr;
    double alpha_R_per_km;
    int n_spans;                /* identical spans (0 or 1: one span); each amplifier
                                 * restores the launch profile (Sec. IV), so span k adds
                                 * the phase offset (k-1) L of Eq. new_gn_model and the
                                 * ASE of n amplifiers adds up; at most 100 */
    int profile;                /* ISRS_PROFILE_* (0 for a zero-initialised struct) */
    double raman_max_THz;       /* Raman ODE: gain cut-off [THz]; <= 0: none */
    int raman_photon;           /* Raman ODE: 1 = photon ratio in the pump depletion */
} isrs_fibre;

/* Channel plan (host pointers, n_ch entries each).  nf_dB and guard may be
 * NULL (noise figure then 0 dB; no guard channels).  gamma is that of each
 * channel; the model uses the CUT's gamma for the whole integral (App. A). */
typedef struct {
    int n_ch;
    const double *f_THz;
    const double *B_THz;
    const double *alpha_per_km;
    const double *gamma_per_W_km;
    const double *nf_dB;
    const unsigned char *guard;
    const double *raman_scale;  /* Raman ODE gain scale s_i > 0 (NULL: 1); unused otherwise */
} isrs_channels;

/* Quadrature settings.  G x G grid points per piece (a cell clipped to one
 * quadrant): G rows uniform in ln(upsilon1) from eps_v1 * upsilon1_max, G
 * columns uniform in upsilon2 per row (App. A, Eqs. q1..q4).  n_edges z-grid
 * edges (n_edges - 1 steps, Eq. slow_vary). */
typedef struct {
    int G;
    int n_edges;
    double eps_v1;
    int cell_set;
    int precision;
    double snr_trx_dB;          /* <= 0: no transceiver noise (Sec. IV) */
    double ode_h_km;            /* Raman ODE: largest RK4 step [km]; <= 0 selects 0.25 */
    int G_mci;                  /* with ISRS_CELLS_ALL and > 0: the multi-channel-interference
                                 * cells (neither F_a nor F_b in the CUT's channel) get their own
                                 * G_mci x G_mci grid (<= 32) and are enumerated on the device
                                 * (no piece list); eta and SNR with either profile, the
                                 * gradient with the closed-form profile.
                                 * 0: every cell uses G. */
} isrs_quad;

/* ------------------------------------------------------------------------ */
/* Handle                                                                    */
/* ------------------------------------------------------------------------ */

/* Creates a handle bound to CUDA device `device`.  Allocates no device
 * memory until the first compute call.  Errors: INVALID_ARG (NULL out or bad
 * device), CUDA. */
isrs_status isrs_create(isrs_handle *out, int device);

/* Frees the handle and all device memory it owns.  NULL is accepted. */
isrs_status isrs_destroy(isrs_handle h);

const char *isrs_status_string(isrs_status s);

/* Last error message of the handle (never NULL; "" if none).  Valid until
 * the next call on the handle. */
const char *isrs_last_error(isrs_handle h);

/* ------------------------------------------------------------------------ */
/* Host helpers (Sec. II)                                                    */
/* ------------------------------------------------------------------------ */

/* Eqs. d, d_slope, d_curve: beta2 [ps^2/km], beta3 [ps^3/km], beta4
 * [ps^4/km] from D [ps/nm/km], S [ps/nm^2/km] and Sdot [ps/nm^3/km] at
 * lambda_nm.  Writes beta[0..2].  Errors: INVALID_ARG (NULL or lambda <= 0). */
isrs_status isrs_beta_from_dispersion(double lambda_nm, double D, double S, double Sdot,
                                      double *beta);

/* Eq. gamma: gamma = 2 pi n2 / (lambda Aeff) [1/(W km)] with n2 [m^2/W] and
 * Aeff [um^2].  Returns NaN on a non-positive argument. */
double isrs_gamma_from_aeff(double lambda_nm, double n2_m2_per_W, double aeff_um2);

/* ------------------------------------------------------------------------ */
/* Forward                                                                   */
/* ------------------------------------------------------------------------ */

/* eta_i for the CUTs listed in `cuts` (n_cuts entries, any order, no
 * repeats; cuts == NULL means all channels 0..n_ch-1 and n_cuts is then
 * ignored).  Eq. gain_fin with P_NLI,i = G(f_i) B_i and eta_i = P_NLI,i/P_i^3.
 *   P_W[n_ch]       launch powers (>= 0; 0 marks an empty slot)
 *   eta[n_out]      eta_i [1/W^2]; NaN for an empty CUT          (nullable)
 *   pnli[n_out]     P_NLI,i [W]                                   (nullable)
 *   sigma[n_out]    the frequency integral without 16/27 gamma^2
 *                   [W^3 km^2/THz]                                (nullable)
 * n_out = n_cuts (or n_ch).  Errors: INVALID_ARG (plan not sorted/disjoint,
 * B <= 0, P < 0 or NaN, G < 1, n_edges < 2, L <= 0, bad cell_set/precision/
 * profile, raman_scale <= 0, bad cut index), UNSUPPORTED (a piece whose F_c
 * range covers more than 16 channels; the Raman ODE with more than 2048
 * channels or with per-piece tables beyond shared memory), ALLOC, CUDA,
 * NUMERIC. */
isrs_status isrs_gn_eta(isrs_handle h, const isrs_fibre *fibre, const isrs_channels *ch,
                        const double *P_W, const isrs_quad *quad, const int *cuts, int n_cuts,
                        double *eta, double *pnli, double *sigma, void *stream);

/* SNR and throughput for all channels (Sec. IV, Eq. loss):
 *   SNR_i = P_i / (eta_i P_i^3 + P_ASE,i), optional 1/SNR += 1/SNR_TRX,
 *   P_ASE,i = NF_i h f_i (G_i - 1) B_i with G_i = 1 / rho(L, f_i),
 *   T = 2 sum_{i not guard, P_i > 0} B_i log2(1 + SNR_i)  [Tb/s].
 *   snr[n_ch], eta[n_ch] (nullable), T_host (nullable, host double). */
isrs_status isrs_gn_snr(isrs_handle h, const isrs_fibre *fibre, const isrs_channels *ch,
                        const double *P_W, const isrs_quad *quad, double *snr, double *eta,
                        double *T_host, void *stream);

/* ------------------------------------------------------------------------ */
/* Gradient                                                                  */
/* ------------------------------------------------------------------------ */

/* dT/dP_j [Tb/s per W] of the throughput T of isrs_gn_snr with respect to
 * every launch power, through eta (the PSD product and the ISRS profile of
 * every grid point, including the MCI cells of a separate G_mci grid with the
 * closed-form profile), the ASE gain G_i and the SNR numerator.  Computed by a
 * hand-written adjoint of the FP32 forward (quad->precision must be
 * ISRS_PREC_FP32).  All P_j must be > 0 and no channel may be a guard.
 * Errors: UNSUPPORTED for G_mci > 0 with the Raman-ODE profile.
 *   dT_dP[n_ch], snr[n_ch] (nullable), eta[n_ch] (nullable),
 *   T_host (nullable, host double). */
isrs_status isrs_gn_grad(isrs_handle h, const isrs_fibre *fibre, const isrs_channels *ch,
                         const double *P_W, const isrs_quad *quad, double *dT_dP, double *snr,
                         double *eta, double *T_host, void *stream);

/* Gradient split by CUT shards, for one gradient spread over several GPUs
 * (one process and one handle per GPU; Sec. III: every GPU takes a group of
 * channels under test, Fig. gpu_nodes).  Every eta_i is a sum over CUT i's own
 * grid, so the adjoint buckets of a CUT depend only on that CUT; what couples
 * the shards is dT/deta_i, which needs the SNR of every channel.  Two phases:
 *
 * isrs_gn_grad_shard_fwd: the fused forward + adjoint quadrature of
 * isrs_gn_grad over the CUTs in `cuts` only (n_cuts entries, no repeats);
 * writes eta[n_cuts] of those CUTs (host or device) and keeps the shard's
 * buckets in the handle (with the Raman-ODE profile also the RK4 states of
 * the profile, whose discrete adjoint is linear in the shard's bucket
 * terms); requirements and errors are those of isrs_gn_grad.
 *
 * The caller gathers eta of every channel from all shards (eta_all[n_ch]).
 *
 * isrs_gn_grad_shard_bwd: from eta_all, the SNR of every channel, T and
 * dT/deta; then this shard's part of dT/dP_j (through its CUTs' PSD
 * products and ISRS profile terms).  with_direct = 1 also adds the terms that
 * do not pass through any eta (the ASE gain of every channel and the SNR
 * numerator): exactly one shard sets it.  The sum of dT_dP[n_ch] over the
 * shards is isrs_gn_grad's dT_dP.  snr[n_ch] (nullable) and T_host (nullable)
 * are those of the whole system.  No other compute call may use the handle
 * between the two phases (INVALID_ARG otherwise).
 * Errors: INVALID_ARG (no preceding shard forward, eta_all not finite >= 0,
 * NULL output), CUDA. */
isrs_status isrs_gn_grad_shard_fwd(isrs_handle h, const isrs_fibre *fibre, const isrs_channels *ch,
                                   const double *P_W, const isrs_quad *quad, const int *cuts, int n_cuts,
                                   double *eta, void *stream);
isrs_status isrs_gn_grad_shard_bwd(isrs_handle h, const double *eta_all, int with_direct, double *dT_dP,
                                   double *snr, double *T_host, void *stream);

/* ------------------------------------------------------------------------ */
/* Batched                                                                   */
/* ------------------------------------------------------------------------ */

/* eta for n_prof launch-power profiles over n_plans channel plans in one
 * persistent launch (one work queue over (profile, CUT, piece-chunk) tiles).
 *   plans[n_plans]           channel plans (host)
 *   plan_of_profile[n_prof]  host int, plan index of each profile
 *   P_W                      concatenated powers: profile p occupies
 *                            n_ch(plan_of_profile[p]) entries starting at
 *                            the sum of the previous profiles' sizes
 *   eta                      same layout as P_W (host or device)
 * Errors as isrs_gn_eta. */
isrs_status isrs_gn_eta_batched(isrs_handle h, const isrs_fibre *fibre, int n_plans,
                                const isrs_channels *plans, int n_prof,
                                const int *plan_of_profile, const double *P_W,
                                const isrs_quad *quad, double *eta, void *stream);

/* Work-tile shape used by the quadrature kernels: points per work item and
 * threads per block.  0 selects the built-in default / autotuned choice.
 * Errors: INVALID_ARG (negative or not a supported block size). */
isrs_status isrs_set_tile(isrs_handle h, int points_per_item, int threads_per_block);

/* Test hook for the failure paths (no counterpart in the paper): arms one
 * simulated failure on this handle.  kind 1: the after-th device allocation
 * the handle makes from now on fails as if cudaMalloc had returned
 * cudaErrorMemoryAllocation (the call returns ISRS_ERR_ALLOC); kind 2: the
 * after-th checked CUDA runtime call fails as if it had returned an error
 * (ISRS_ERR_CUDA).  The failure is made on the host: the simulated call is
 * not executed and the device is untouched.  It fires once; kind 0 disarms.
 * Errors: INVALID_ARG (NULL handle, kind outside 0..2, after < 1). */
isrs_status isrs_debug_inject_fault(isrs_handle h, int kind, int after);

/* 1 when this library is the bounds-checked debug build (compiled with
 * ISRS_DEBUG), else 0.  In the debug build the quadrature kernels check their
 * piece, row, candidate, list and bucket-row indices; a failed check records
 * its code on the device, clamps the index into range (no access leaves its
 * array and every thread still reaches every barrier), and the call then
 * returns ISRS_ERR_CHECK with the code in isrs_last_error.  The release build
 * compiles the checks away.  No arguments, no errors. */
int isrs_debug_build(void);

/* Number of quadrature-kernel launches and grid points of the last compute
 * call (for throughput accounting).  Any argument may be NULL. */
isrs_status isrs_last_launch_info(isrs_handle h, int64_t *n_points, int64_t *n_point_steps,
                                  int *n_kernel_launches);

/* Duration [ms] of the last quadrature (which = 0) or adjoint (which = 1)
 * kernel launch of this handle, from CUDA events recorded on the launch
 * stream immediately around it (not recorded while the stream is being
 * captured into a graph).  Waits for that launch to finish.
 * Errors: INVALID_ARG (bad which, or no such launch recorded yet), CUDA. */
isrs_status isrs_last_kernel_ms(isrs_handle h, int which, float *ms);

/* 1 if the last isrs_gn_eta_batched call replayed its captured CUDA graph
 * (prep, quadrature and finish captured once per launch signature), 0 if it
 * ran the kernels directly (first call of a signature, or capture not
 * possible).  Errors: INVALID_ARG (NULL). */
isrs_status isrs_last_graph_replay(isrs_handle h, int *replayed);

/* Grid points of the last FP32 quadrature launch (forward, or the fused
 * forward + adjoint of isrs_gn_grad) by the form its z-sum took (App. A,
 * Eq. slow_vary): counts[0] moment expansions (small phase: about the span
 * centre, contracted or per step; in the forward at G >= 160 also about the
 * centres of 2, 4 or 8 segments of the span), counts[1] direct form, counts[2]
 * telescoped form.  Synchronises the device.  Errors: INVALID_ARG (NULL, or
 * no launch yet), CUDA. */
isrs_status isrs_last_path_counts(isrs_handle h, int64_t *counts);

/* Measured throughput of the ALU pipes that bound the quadrature kernels
 * (a measurement utility; the paper has no counterpart).  which = 0: the SFU
 * (MUFU ex2.approx, the unit of the sin, cos and ex2 of every z-step of
 * Eq. slow_vary); which = 1: the FP32 FMA pipe (one FFMA counted as one
 * operation).  Runs one warm-up and one timed launch of independent
 * dependency chains on `device` (~15 ms each) and writes operations per
 * second (ops_per_s) and the timed launch's duration (ms, nullable).
 * Allocates and frees a small output buffer.  Errors: INVALID_ARG (bad
 * device or which, NULL ops_per_s), ALLOC, CUDA. */
isrs_status isrs_probe_alu_peaks(int device, int which, double *ops_per_s, float *ms);

/* ------------------------------------------------------------------------ */
/* Allocation-free forward                                                   */
/* ------------------------------------------------------------------------ */

/* eta_i and P_NLI,i for every channel, like isrs_gn_eta with cuts == NULL,
 * but without allocating device memory: for callers that cannot call
 * cudaMalloc (code inside a host framework that owns the device allocator,
 * a memory-budgeted real-time loop, a process whose allocator is locked).
 * The paper has no counterpart; this is a deployment variant.
 *
 * All scratch (plan tables, per-profile tables, the z-grid with its step
 * moments, tile partials) lives in one file-scope device array of 4 MiB that
 * every GPU loading this library holds until the process exits.  The first
 * call on a device looks up that array's address with the device current;
 * make that first call before any stream capture.  Every call shares the
 * array and leaves the last call's contents in it; calls whose GPU work
 * overlaps (two streams, two host threads, two devices' worth of work on one
 * device) race on it and must be serialised by the caller.
 *   P_W[n_ch], eta[n_ch]: device pointers of the current device (or managed
 *   memory); pnli[n_ch]: the same, or NULL.
 * No handle is used; the call reads the powers back to the host and
 * synchronises `stream` once after uploading the plan tables, then runs
 * asynchronously.  On a stream that is being captured it returns
 * UNSUPPORTED before issuing any work, leaving the capture intact.
 * Errors: INVALID_ARG (as isrs_gn_eta, a host pointer, or device memory of
 * another GPU), UNSUPPORTED (the tables need more than the 4 MiB scratch:
 * e.g. more than ~5e4 pieces, or the FP32 phase range; more than one span;
 * the Raman-ODE profile; a capturing stream), CUDA. */
isrs_status isrs_gn_eta_noalloc(const isrs_fibre *fibre, const isrs_channels *ch, const double *P_W,
                                const isrs_quad *quad, double *eta, double *pnli, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* ISRS_GN_H */
