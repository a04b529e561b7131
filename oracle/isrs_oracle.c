/*
 * isrs_oracle.c -- plain, slow FP64 CPU oracle of the ISRS Gaussian-noise
 * integral model of arXiv 2401.18022 (App. A, Eqs. gain/pk/phi/slow_vary/
 * q1..q4/gain_fin/psi_fin; Sec. II Eqs. d, d_slope, d_curve, gamma; Sec. IV
 * Eq. loss).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this library; the product path never
 * calls it, and it shares no code, header, table or constant generator with
 * the CUDA library.  Everything is double precision, loops are written in the
 * order of the paper's definitions, and no blocking, fusion or reordering is
 * applied beyond tabulating per-z quantities once per z.
 *
 * Readings of the paper that this oracle fixes (the paper is silent on them):
 *  - Riemann grid: G x G midpoints per rectangular "piece" (a channel-pair
 *    cell clipped to one quadrant), uniform in s = ln(upsilon1) and, per row,
 *    uniform in upsilon2 between the row's limits; upsilon1 is cut off below
 *    at eps * upsilon1_max.
 *  - z-grid: N_M edges with equal power drop per step, z-tilde_m = z_m.
 *  - Power profile R1: the closed-form ISRS profile for a linear Raman slope
 *    (the model the paper builds on, App. A), normalised by the integral of
 *    the transmitted PSD, with per-channel attenuation.
 *  - Power profile R2: RK4 solution of the Raman ODEs for line channels,
 *    triangular gain cut off at df_max, photon ratio, Aeff scale; inside a
 *    channel ln rho is linear with the central-difference slope.
 *  - P_NLI,i = G(f_i) B_i and eta_i = P_NLI,i / P_i^3.
 *
 * Units: THz, ps, km, W.  phi in rad/km.
 */
#define _GNU_SOURCE
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define ORC_C_NM_PER_PS 299792.458
#define ORC_H_PLANCK 6.62607015e-34

/* ---------------------------------------------------------------------- */
/* Sec. II, Eqs. d, d_slope, d_curve: beta2, beta3, beta4 from D, S, Sdot  */
/* at the reference wavelength.  lambda [nm], D [ps/nm/km], S [ps/nm^2/km],*/
/* Sdot [ps/nm^3/km]  ->  beta_k [ps^k/km].                                */
/* ---------------------------------------------------------------------- */
void orc_beta_from_dispersion(double lambda_nm, double D, double S, double Sdot,
                              double *beta /* [3] */)
{
    double w = 2.0 * ORC_PI * ORC_C_NM_PER_PS;          /* 2 pi c [nm/ps] */
    double l = lambda_nm;
    beta[0] = -D * l * l / w;
    beta[1] = l * l * l / (w * w) * (2.0 * D + S * l);
    beta[2] = -l * l * l * l / (w * w * w) * (6.0 * D + 6.0 * S * l + Sdot * l * l);
}

/* Sec. II, Eq. gamma: gamma = 2 pi n2 / (lambda Aeff)  [1/(W km)].        */
double orc_gamma(double lambda_nm, double n2_m2_per_W, double aeff_um2)
{
    double lam_m = lambda_nm * 1e-9, aeff_m2 = aeff_um2 * 1e-12;
    return 2.0 * ORC_PI / lam_m * n2_m2_per_W / aeff_m2 * 1e3;
}

/* ---------------------------------------------------------------------- */
/* Sec. III-A / App. A (slowly varying power): N_M edges, "log-scale      */
/* distance intervals" with equal power change per step:                  */
/*   exp(-a z_e(m)) = 1 - (m / (N_M - 1)) (1 - exp(-a L)).                 */
/* ---------------------------------------------------------------------- */
int orc_zgrid(double L, double a, int n_edges, double *z)
{
    if (n_edges < 2 || !(L > 0.0)) return -1;
    double drop = (a > 0.0) ? 1.0 - exp(-a * L) : 0.0;
    for (int m = 0; m < n_edges; ++m) {
        double t = (double)m / (double)(n_edges - 1);
        z[m] = (a > 0.0) ? -log(1.0 - t * drop) / a : t * L;
    }
    z[n_edges - 1] = L;
    return 0;
}

/* ---------------------------------------------------------------------- */
/* App. A, Eq. phi: phase mismatch per unit length [rad/km] for offsets    */
/* f1, f2 from the channel under test, fi = CUT offset from the reference. */
/* ---------------------------------------------------------------------- */
double orc_phi(double f1, double f2, double fi, double b2, double b3, double b4)
{
    double bracket = b2
        + ORC_PI * b3 * (f1 + f2 + 2.0 * fi)
        + (2.0 * ORC_PI * ORC_PI / 3.0) * b4
          * (f1 * f1 + 1.5 * f1 * f2 + 3.0 * f1 * fi + f2 * f2 + 3.0 * f2 * fi + 3.0 * fi * fi);
    return -4.0 * ORC_PI * ORC_PI * f1 * f2 * bracket;
}

/* ---------------------------------------------------------------------- */
/* Channel plan helpers.  G_Tx is rectangular per channel (Sec. III):      */
/* G_Tx(F) = P_c / B_c on [f_c - B_c/2, f_c + B_c/2), zero in the gaps.    */
/* ---------------------------------------------------------------------- */
typedef struct {
    int n;
    const double *f, *B, *P, *alpha;
} orc_plan;

/* index of the channel containing F, or -1 (channels sorted, disjoint) */
static int orc_channel_of(const orc_plan *pl, double F)
{
    int lo = 0, hi = pl->n - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        double a = pl->f[mid] - 0.5 * pl->B[mid], b = pl->f[mid] + 0.5 * pl->B[mid];
        if (F < a) hi = mid - 1;
        else if (F >= b) lo = mid + 1;
        else return mid;
    }
    return -1;
}

/* ---------------------------------------------------------------------- */
/* ISRS power profile, linear Raman slope (App. A; the closed form the     */
/* model builds on):                                                       */
/*  rho(z,F) = e^{-alpha_c z} P_tot e^{-kappa(z)(F - f_ref)} / N(z),       */
/*  kappa(z) = P_tot C_r L_eff(z),  L_eff(z) = (1 - e^{-alpha_R z})/alpha_R,*/
/*  N(z) = int G_Tx(nu) e^{-kappa(z)(nu - f_ref)} dnu                      */
/*       = sum_k P_k e^{-kappa (f_k - f_ref)} sinh(kappa B_k/2)/(kappa B_k/2)*/
/* ln N is accumulated with a max shift so that large tilts stay finite.   */
/* ---------------------------------------------------------------------- */
static double orc_sinhc(double x)
{
    if (fabs(x) < 1e-4) return 1.0 + x * x / 6.0;
    return sinh(x) / x;
}

double orc_leff(double z, double alpha_R)
{
    return (alpha_R > 0.0) ? (1.0 - exp(-alpha_R * z)) / alpha_R : z;
}

static double orc_ptot(const orc_plan *pl)
{
    double s = 0.0;
    for (int k = 0; k < pl->n; ++k) s += pl->P[k];
    return s;
}

static double orc_kappa(const orc_plan *pl, double z, double Cr, double alpha_R)
{
    return orc_ptot(pl) * Cr * orc_leff(z, alpha_R);
}

static double orc_lnN(const orc_plan *pl, double kappa, double f_ref)
{
    double mx = -INFINITY;
    for (int k = 0; k < pl->n; ++k) {
        if (pl->P[k] <= 0.0) continue;
        double e = log(pl->P[k]) - kappa * (pl->f[k] - f_ref) + log(orc_sinhc(0.5 * kappa * pl->B[k]));
        if (e > mx) mx = e;
    }
    double s = 0.0;
    for (int k = 0; k < pl->n; ++k) {
        if (pl->P[k] <= 0.0) continue;
        double e = log(pl->P[k]) - kappa * (pl->f[k] - f_ref) + log(orc_sinhc(0.5 * kappa * pl->B[k]));
        s += exp(e - mx);
    }
    return mx + log(s);
}

/* ln rho(z, F) for F inside channel c. */
static double orc_lnrho_c(const orc_plan *pl, int c, double z, double F, double lnPtot,
                          double lnN, double kappa, double f_ref)
{
    return -pl->alpha[c] * z + lnPtot - lnN - kappa * (F - f_ref);
}

/* Public: ln rho(z, F) at an arbitrary z (F must lie in a channel, else NaN). */
double orc_lnrho(int n, const double *f, const double *B, const double *P, const double *alpha,
                 double f_ref, double Cr, double alpha_R, double z, double F)
{
    orc_plan pl = {n, f, B, P, alpha};
    int c = orc_channel_of(&pl, F);
    if (c < 0) return NAN;
    double kappa = orc_kappa(&pl, z, Cr, alpha_R);
    return orc_lnrho_c(&pl, c, z, F, log(orc_ptot(&pl)), orc_lnN(&pl, kappa, f_ref), kappa, f_ref);
}

/* ---------------------------------------------------------------------- */
/* Profile model R2 (Sec. III and App. A: the profile is the solution of   */
/* the Raman power-evolution ODEs, with the Raman gain scaled by the       */
/* effective area at the channel frequency).  Channel k is a line of power */
/* P_k at f_k (THz, absolute); with y_i = ln P_i                           */
/*   dy_i/dz = -alpha_i + s_i C_r sum_{k != i} h(f_k, f_i) P_k,            */
/*   h = f_k - f_i                 if 0 < f_k - f_i <= df_max (k pumps i), */
/*   h = (f_k - f_i) f_i / f_k     if 0 < f_i - f_k <= df_max (i pumps k;  */
/*                                  the photon ratio, replaced by 1 when   */
/*                                  photon == 0),                          */
/*   h = 0 beyond df_max (df_max <= 0: no cut-off),                        */
/* i.e. a triangular gain C_r |df| cut off at df_max, and s_i =            */
/* Aeff(f_ref)/Aeff(f_i).  A slot with P_k = 0 pumps nothing; its y_k      */
/* starts at 0 and follows the gain a zero-power probe would see.          */
/* ---------------------------------------------------------------------- */
typedef struct {
    int n;
    const double *f, *P0, *alpha, *scale;
    double Cr, df_max;
    int photon;
} orc_raman;

static void orc_raman_rhs(const orc_raman *r, const double *y, double *dy)
{
    for (int i = 0; i < r->n; ++i) {
        double s = 0.0;
        for (int k = 0; k < r->n; ++k) {
            if (k == i || !(r->P0[k] > 0.0)) continue;
            double d = r->f[k] - r->f[i];
            if (r->df_max > 0.0 && fabs(d) > r->df_max) continue;
            double h = (d > 0.0 || !r->photon) ? d : d * r->f[i] / r->f[k];
            s += h * exp(y[k]);
        }
        double si = r->scale ? r->scale[i] : 1.0;
        dy[i] = -r->alpha[i] + si * r->Cr * s;
    }
}

/* one classical RK4 step of length h, in place */
static void orc_rk4_step(const orc_raman *r, double h, double *y, double *w /* 5 n */)
{
    int n = r->n;
    double *k1 = w, *k2 = w + n, *k3 = w + 2 * n, *k4 = w + 3 * n, *t = w + 4 * n;
    orc_raman_rhs(r, y, k1);
    for (int i = 0; i < n; ++i) t[i] = y[i] + 0.5 * h * k1[i];
    orc_raman_rhs(r, t, k2);
    for (int i = 0; i < n; ++i) t[i] = y[i] + 0.5 * h * k2[i];
    orc_raman_rhs(r, t, k3);
    for (int i = 0; i < n; ++i) t[i] = y[i] + h * k3[i];
    orc_raman_rhs(r, t, k4);
    for (int i = 0; i < n; ++i) y[i] += h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

/*
 * Integrates the ODE through nodes z_nodes[0..n_seg], segment s split into
 * n_sub[s] equal RK4 steps.  y_out[(s * n) + i] = y_i at node s (node 0: ln P
 * of loaded channels, 0 for empty ones).
 */
int orc_raman_solve(int n, const double *f, const double *P, const double *alpha, const double *scale,
                    double Cr, double df_max, int photon, int n_seg, const double *z_nodes,
                    const int *n_sub, double *y_out)
{
    if (n < 1 || n_seg < 0) return -1;
    orc_raman r = {n, f, P, alpha, scale, Cr, df_max, photon};
    double *y = (double *)malloc(sizeof(double) * (size_t)n);
    double *w = (double *)malloc(sizeof(double) * (size_t)(5 * n));
    for (int i = 0; i < n; ++i) y[i] = P[i] > 0.0 ? log(P[i]) : 0.0;
    memcpy(y_out, y, sizeof(double) * (size_t)n);
    for (int s = 0; s < n_seg; ++s) {
        int ns = n_sub[s] > 0 ? n_sub[s] : 1;
        double h = (z_nodes[s + 1] - z_nodes[s]) / ns;
        for (int k = 0; k < ns; ++k) orc_rk4_step(&r, h, y, w);
        memcpy(y_out + (size_t)(s + 1) * n, y, sizeof(double) * (size_t)n);
    }
    free(y);
    free(w);
    return 0;
}

/* RK4 steps in each half of a z-step of length dz: ceil((dz/2) / h_max). */
static int orc_half_steps(double dz, double h_max)
{
    int ns = (int)ceil(0.5 * dz / h_max - 1e-9);
    return ns < 1 ? 1 : ns;
}

/*
 * The R2 tables on the z-grid of n_edges equal-power-drop edges: the ODE is
 * integrated edge -> midpoint -> edge through every step, each half in
 * orc_half_steps equal RK4 steps.  Per channel c and step m:
 *   a[c M + m] = ln rho_c(z_m) = y_c(z_m) - y_c(0),
 *   b[c M + m] = d ln rho / dF inside channel c: the central difference, over
 *                the neighbouring channels, of the Raman part a + alpha z_m
 *                (one-sided at the ends of the plan, 0 for one channel),
 * and aL[c] = ln rho_c(L).  Inside channel c, ln rho(z_m, F) = a + b (F - f_c).
 * fibre[12]: {L, f_ref, b2, b3, b4, Cr, alpha_R, n_spans, profile,
 *             df_max, photon, h_max}.
 */
int orc_raman_profile(int n, const double *f, const double *P, const double *alpha, const double *scale,
                      const double *fibre, int n_edges, double *a, double *b, double *aL)
{
    if (n < 1 || n_edges < 2 || !(fibre[11] > 0.0)) return -1;
    int M = n_edges - 1;
    double *ze = (double *)malloc(sizeof(double) * (size_t)n_edges);
    orc_zgrid(fibre[0], fibre[6], n_edges, ze);
    double *zn = (double *)malloc(sizeof(double) * (size_t)(2 * M + 1));
    int *ns = (int *)malloc(sizeof(int) * (size_t)(2 * M));
    for (int m = 0; m < M; ++m) {
        zn[2 * m] = ze[m];
        zn[2 * m + 1] = 0.5 * (ze[m] + ze[m + 1]);
        ns[2 * m] = ns[2 * m + 1] = orc_half_steps(ze[m + 1] - ze[m], fibre[11]);
    }
    zn[2 * M] = ze[M];
    double *yo = (double *)malloc(sizeof(double) * (size_t)(2 * M + 1) * (size_t)n);
    orc_raman_solve(n, f, P, alpha, scale, fibre[5], fibre[9], fibre[10] != 0.0, 2 * M, zn, ns, yo);
    for (int c = 0; c < n; ++c) {
        for (int m = 0; m < M; ++m) a[c * M + m] = yo[(size_t)(2 * m + 1) * n + c] - yo[c];
        aL[c] = yo[(size_t)(2 * M) * n + c] - yo[c];
    }
    for (int m = 0; m < M; ++m) {
        double zm = zn[2 * m + 1];
        for (int c = 0; c < n; ++c) {
            int lo = c > 0 ? c - 1 : 0, hi = c < n - 1 ? c + 1 : n - 1;
            if (lo == hi) { b[c * M + m] = 0.0; continue; }
            double rlo = a[lo * M + m] + alpha[lo] * zm, rhi = a[hi * M + m] + alpha[hi] * zm;
            b[c * M + m] = (rhi - rlo) / (f[hi] - f[lo]);
        }
    }
    free(ze); free(zn); free(ns); free(yo);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* App. A, Eq. slow_vary: the z-sum                                        */
/*   S = sum_m p_m dz_m sinc(phi dz_m / 2) e^{j phi z_m}                   */
/* for given per-step powers p_m (single span, L-tilde = 0).               */
/* ---------------------------------------------------------------------- */
static double orc_sinc(double x)
{
    if (fabs(x) < 1e-4) return 1.0 - x * x / 6.0;
    return sin(x) / x;
}

void orc_zsum(int n_steps, const double *z_mid, const double *dz, const double *p, double phi,
              double *S /* [2] re, im */)
{
    double re = 0.0, im = 0.0;
    for (int m = 0; m < n_steps; ++m) {
        double a = p[m] * dz[m] * orc_sinc(0.5 * phi * dz[m]);
        re += a * cos(phi * z_mid[m]);
        im += a * sin(phi * z_mid[m]);
    }
    S[0] = re;
    S[1] = im;
}

/* Eq. new_gn_model: the link's z-sum over n identical spans, span k adding */
/* the phase offset L-tilde_k = (k - 1) L:                                 */
/*   S = sum_k sum_m p_m dz_m sinc(phi dz_m / 2) e^{j phi ((k-1) L + z_m)}  */
void orc_zsum_spans(int n_steps, const double *z_mid, const double *dz, const double *p, double phi,
                    double L, int n_spans, double *S /* [2] */)
{
    double re = 0.0, im = 0.0;
    for (int k = 0; k < n_spans; ++k)
        for (int m = 0; m < n_steps; ++m) {
            double a = p[m] * dz[m] * orc_sinc(0.5 * phi * dz[m]);
            re += a * cos(phi * (k * L + z_mid[m]));
            im += a * sin(phi * (k * L + z_mid[m]));
        }
    S[0] = re;
    S[1] = im;
}

/* ---------------------------------------------------------------------- */
/* Pieces.  The plane of offsets (f1, f2) of CUT i is split into channel-  */
/* pair cells (a,b): F_a = f_i + f1 in channel a, F_b = f_i + f2 in        */
/* channel b.  Each cell is cut at f1 = 0 and f2 = 0 into quadrant pieces  */
/* (App. A, Eqs. q1a..q4d): |f1| in [x_lo, x_hi], |f2| in [y_lo, y_hi],    */
/* signs (s1, s2).  cell_set 0: SCI + XCI cells (a == i or b == i);        */
/* cell_set 1: all cells.                                                  */
/* ---------------------------------------------------------------------- */
typedef struct {
    int a, b, s1, s2;
    double xlo, xhi, ylo, yhi;
} orc_piece;

static int orc_split(double lo, double hi, int *sg, double *plo, double *phi_)
{
    int k = 0;
    if (hi > 0.0) { sg[k] = +1; plo[k] = lo > 0.0 ? lo : 0.0; phi_[k] = hi; ++k; }
    if (lo < 0.0) { sg[k] = -1; plo[k] = hi < 0.0 ? -hi : 0.0; phi_[k] = -lo; ++k; }
    return k;
}

/* Writes the pieces of CUT i into out (if non-NULL); returns their count. */
int orc_pieces(int n, const double *f, const double *B, int i, int cell_set, orc_piece *out)
{
    int cnt = 0;
    for (int a = 0; a < n; ++a) {
        for (int b = 0; b < n; ++b) {
            if (cell_set == 0 && a != i && b != i) continue;
            int sa[2], sb[2];
            double xl[2], xh[2], yl[2], yh[2];
            int na = orc_split(f[a] - 0.5 * B[a] - f[i], f[a] + 0.5 * B[a] - f[i], sa, xl, xh);
            int nb = orc_split(f[b] - 0.5 * B[b] - f[i], f[b] + 0.5 * B[b] - f[i], sb, yl, yh);
            for (int u = 0; u < na; ++u)
                for (int v = 0; v < nb; ++v) {
                    if (!(xh[u] > xl[u]) || !(yh[v] > yl[v])) continue;
                    if (out) {
                        orc_piece *q = &out[cnt];
                        q->a = a; q->b = b; q->s1 = sa[u]; q->s2 = sb[v];
                        q->xlo = xl[u]; q->xhi = xh[u]; q->ylo = yl[v]; q->yhi = yh[v];
                    }
                    ++cnt;
                }
        }
    }
    return cnt;
}

/* Flat export of the piece list for tests: rows of
 * (a, b, s1, s2, xlo, xhi, ylo, yhi) as doubles. */
int orc_pieces_flat(int n, const double *f, const double *B, int i, int cell_set, double *out8)
{
    int cnt = orc_pieces(n, f, B, i, cell_set, NULL);
    if (!out8) return cnt;
    orc_piece *p = (orc_piece *)malloc(sizeof(orc_piece) * (size_t)(cnt > 0 ? cnt : 1));
    orc_pieces(n, f, B, i, cell_set, p);
    for (int k = 0; k < cnt; ++k) {
        double *r = out8 + 8 * k;
        r[0] = p[k].a; r[1] = p[k].b; r[2] = p[k].s1; r[3] = p[k].s2;
        r[4] = p[k].xlo; r[5] = p[k].xhi; r[6] = p[k].ylo; r[7] = p[k].yhi;
    }
    free(p);
    return cnt;
}

/* ---------------------------------------------------------------------- */
/* The problem: plan, fibre, z-grid tables.                                */
/* ---------------------------------------------------------------------- */
typedef struct {
    orc_plan pl;
    double L, f_ref, b2, b3, b4, Cr, alpha_R, eps;
    int n_spans;                        /* identical spans, launch profile restored per span */
    int G, n_steps, cell_set;
    int G_mci;                          /* grid of cells with a != i and b != i (0: G) */
    double lnPtot;
    double *z_mid, *dz, *kappa, *lnN;   /* per step */
    /* ones-mode: Psi's PSD product and link factor replaced by 1 (area). */
    int unit_integrand;
    /* profile model: 0 closed form (linear slope), 1 Raman ODE tables */
    int profile;
    const double *fibre, *scale;
    double *ra, *rb, *raL;              /* R2: [n x n_steps], [n x n_steps], [n] */
} orc_problem;

static void orc_problem_tables(orc_problem *pr, int n_edges)
{
    pr->n_steps = n_edges - 1;
    double *ze = (double *)malloc(sizeof(double) * (size_t)n_edges);
    orc_zgrid(pr->L, pr->alpha_R, n_edges, ze);
    pr->z_mid = (double *)malloc(sizeof(double) * (size_t)pr->n_steps);
    pr->dz = (double *)malloc(sizeof(double) * (size_t)pr->n_steps);
    pr->kappa = (double *)malloc(sizeof(double) * (size_t)pr->n_steps);
    pr->lnN = (double *)malloc(sizeof(double) * (size_t)pr->n_steps);
    pr->lnPtot = log(orc_ptot(&pr->pl));
    for (int m = 0; m < pr->n_steps; ++m) {
        pr->z_mid[m] = 0.5 * (ze[m] + ze[m + 1]);     /* z-tilde_m = z_m */
        pr->dz[m] = ze[m + 1] - ze[m];
        pr->kappa[m] = orc_kappa(&pr->pl, pr->z_mid[m], pr->Cr, pr->alpha_R);
        pr->lnN[m] = orc_lnN(&pr->pl, pr->kappa[m], pr->f_ref);
    }
    free(ze);
    if (pr->profile == 1) {
        size_t nm = (size_t)pr->pl.n * (size_t)pr->n_steps;
        pr->ra = (double *)malloc(sizeof(double) * nm);
        pr->rb = (double *)malloc(sizeof(double) * nm);
        pr->raL = (double *)malloc(sizeof(double) * (size_t)pr->pl.n);
        orc_raman_profile(pr->pl.n, pr->pl.f, pr->pl.P, pr->pl.alpha, pr->scale, pr->fibre, n_edges,
                          pr->ra, pr->rb, pr->raL);
    }
}

static void orc_problem_free(orc_problem *pr)
{
    free(pr->z_mid); free(pr->dz); free(pr->kappa); free(pr->lnN);
    free(pr->ra); free(pr->rb); free(pr->raL);
}

/* ln rho(z_m, F) for F inside channel c, under the problem's profile model */
static double orc_lnrho_m(const orc_problem *pr, int c, int m, double F)
{
    if (pr->profile == 1) {
        size_t k = (size_t)c * (size_t)pr->n_steps + (size_t)m;
        return pr->ra[k] + pr->rb[k] * (F - pr->pl.f[c]);
    }
    return orc_lnrho_c(&pr->pl, c, pr->z_mid[m], F, pr->lnPtot, pr->lnN[m], pr->kappa[m], pr->f_ref);
}

/* ---------------------------------------------------------------------- */
/* App. A, Eqs. q1..q4 and psi_fin: Riemann sum of one piece in hyperbolic */
/* coordinates upsilon1 = |f1||f2|, upsilon2 = ln sqrt(|f1|/|f2|), whose   */
/* Jacobian is 1; g1 = sqrt(u1) e^{u2}, g2 = sqrt(u1) e^{-u2}.             */
/* ---------------------------------------------------------------------- */
static double orc_piece_sum(const orc_problem *pr, int i, const orc_piece *q)
{
    const orc_plan *pl = &pr->pl;
    /* multi-channel-interference cells (neither F_a nor F_b in the CUT's
       channel) may use their own grid size */
    const int G = (pr->G_mci > 0 && q->a != i && q->b != i) ? pr->G_mci : pr->G;
    double fi = pl->f[i];
    double fi_off = fi - pr->f_ref;
    double u1_hi = q->xhi * q->yhi;
    double u1_lo = q->xlo * q->ylo;
    if (u1_lo < pr->eps * u1_hi) u1_lo = pr->eps * u1_hi;
    double ds = (log(u1_hi) - log(u1_lo)) / G;
    double total = 0.0, comp = 0.0;
    double *pv = (double *)malloc(sizeof(double) * (size_t)pr->n_steps);   /* p_m of a point */
    for (int r = 0; r < G; ++r) {
        double u1 = exp(log(u1_lo) + (r + 0.5) * ds);
        double ymin = q->ylo, ymax = q->yhi;
        if (u1 / q->xhi > ymin) ymin = u1 / q->xhi;
        if (q->xlo > 0.0 && u1 / q->xlo < ymax) ymax = u1 / q->xlo;
        if (!(ymax > ymin)) continue;
        double u2_lo = 0.5 * log(u1) - log(ymax);
        double u2_hi = 0.5 * log(u1) - log(ymin);
        double du2 = (u2_hi - u2_lo) / G;
        double w = u1 * ds * du2;                     /* d(u1) = u1 ds */
        for (int c = 0; c < G; ++c) {
            double u2 = u2_lo + (c + 0.5) * du2;
            double g1 = sqrt(u1) * exp(u2), g2 = sqrt(u1) * exp(-u2);
            double f1 = q->s1 * g1, f2 = q->s2 * g2;
            double val;
            if (pr->unit_integrand) {
                val = 1.0;
            } else {
                double Fa = fi + f1, Fb = fi + f2, Fc = fi + f1 + f2;
                int ca = orc_channel_of(pl, Fa), cb = orc_channel_of(pl, Fb), cc = orc_channel_of(pl, Fc);
                if (ca < 0 || cb < 0 || cc < 0) continue;
                /* G_Tx(f1) G_Tx(f2) G_Tx(f1 + f2 - f) */
                double W = (pl->P[ca] / pl->B[ca]) * (pl->P[cb] / pl->B[cb]) * (pl->P[cc] / pl->B[cc]);
                if (W == 0.0) continue;
                double phi = orc_phi(f1, f2, fi_off, pr->b2, pr->b3, pr->b4);
                for (int m = 0; m < pr->n_steps; ++m) {
                    /* Eq. pk: p = sqrt(rho(F_a) rho(F_b) rho(F_c) / rho(f)) */
                    double lra = orc_lnrho_m(pr, ca, m, Fa);
                    double lrb = orc_lnrho_m(pr, cb, m, Fb);
                    double lrc = orc_lnrho_m(pr, cc, m, Fc);
                    double lri = orc_lnrho_m(pr, i, m, fi);
                    pv[m] = exp(0.5 * (lra + lrb + lrc - lri));
                }
                /* Eqs. slow_vary / new_gn_model: the z-sum, over every span */
                double S[2];
                orc_zsum_spans(pr->n_steps, pr->z_mid, pr->dz, pv, phi, pr->L, pr->n_spans, S);
                double Sre = S[0], Sim = S[1];
                val = W * (Sre * Sre + Sim * Sim);
            }
            /* Neumaier-compensated accumulation in FP64 */
            double term = w * val, t = total + term;
            if (fabs(total) >= fabs(term)) comp += (total - t) + term;
            else comp += (term - t) + total;
            total = t;
        }
    }
    free(pv);
    return total + comp;
}

/* ---------------------------------------------------------------------- */
/* Parallel driver: work items are (CUT, piece); each thread takes the    */
/* next item from a shared counter; per-CUT sums run in piece order.      */
/* ---------------------------------------------------------------------- */
typedef struct {
    const orc_problem *pr;
    const int *item_cut;
    const orc_piece *item_piece;
    double *item_val;
    long n_items;
    long stride;
    long next;
    pthread_mutex_t mu;
} orc_work;

static void *orc_worker(void *arg)
{
    orc_work *wk = (orc_work *)arg;
    for (;;) {
        pthread_mutex_lock(&wk->mu);
        long k = wk->next;
        wk->next += wk->stride;
        pthread_mutex_unlock(&wk->mu);
        if (k >= wk->n_items) break;
        wk->item_val[k] = orc_piece_sum(wk->pr, wk->item_cut[k], &wk->item_piece[k]);
    }
    return NULL;
}

/*
 * Sigma_i = sum over the CUT's pieces of the Riemann sums, i.e. the frequency
 * integral of Eq. gain_fin at f = f_i without the 16/27 gamma^2 factor
 * [W^3 km^2 / THz].
 *
 * fibre[12] = {L_km, f_ref_THz, beta2, beta3, beta4, Cr, alpha_R, n_spans,
 *              profile (0 closed form, 1 Raman ODE), df_max_THz, photon, h_max_km};
 * scale: per-channel Raman gain scale s_i of the ODE (NULL: 1).
 * the last four entries and scale are read only when profile == 1.
 * quad[4]  = {G, n_edges, cell_set, G_mci}: G x G points per piece, except
 *            G_mci x G_mci in cells with a != i and b != i when G_mci > 0
 * piece_out (optional): per-piece sums, in the order of orc_pieces, for each
 * requested CUT one after another.
 * unit_integrand != 0 replaces the integrand by 1 (returns covered area).
 * item_stride > 1 evaluates only every item_stride-th piece (the others are
 * left at zero): a bounded sample used to time the oracle, not a result.
 */
int orc_sigma_sampled(int n, const double *f, const double *B, const double *P, const double *alpha,
                      const double *scale, const double *fibre, const int *quad, double eps,
                      const int *cuts, int n_cuts, int n_threads, int unit_integrand, int item_stride,
                      double *sigma_out, double *piece_out)
{
    if (n < 1 || n_cuts < 0 || quad[0] < 1 || quad[1] < 2) return -1;
    orc_problem pr;
    memset(&pr, 0, sizeof(pr));
    pr.pl.n = n; pr.pl.f = f; pr.pl.B = B; pr.pl.P = P; pr.pl.alpha = alpha;
    pr.L = fibre[0]; pr.f_ref = fibre[1]; pr.b2 = fibre[2]; pr.b3 = fibre[3]; pr.b4 = fibre[4];
    pr.Cr = fibre[5]; pr.alpha_R = fibre[6];
    pr.n_spans = fibre[7] >= 1.0 ? (int)fibre[7] : 1;
    pr.G = quad[0]; pr.cell_set = quad[2]; pr.eps = eps; pr.unit_integrand = unit_integrand;
    pr.G_mci = quad[3] > 0 ? quad[3] : 0;
    pr.profile = fibre[8] == 1.0 ? 1 : 0;
    pr.fibre = fibre; pr.scale = scale;
    if (pr.profile == 1 && !(fibre[11] > 0.0)) return -1;
    orc_problem_tables(&pr, quad[1]);

    long total = 0;
    int *cnt = (int *)malloc(sizeof(int) * (size_t)(n_cuts > 0 ? n_cuts : 1));
    for (int k = 0; k < n_cuts; ++k) {
        cnt[k] = orc_pieces(n, f, B, cuts[k], pr.cell_set, NULL);
        total += cnt[k];
    }
    orc_piece *pieces = (orc_piece *)malloc(sizeof(orc_piece) * (size_t)(total > 0 ? total : 1));
    int *item_cut = (int *)malloc(sizeof(int) * (size_t)(total > 0 ? total : 1));
    double *val = (double *)calloc((size_t)(total > 0 ? total : 1), sizeof(double));
    long off = 0;
    for (int k = 0; k < n_cuts; ++k) {
        orc_pieces(n, f, B, cuts[k], pr.cell_set, pieces + off);
        for (int j = 0; j < cnt[k]; ++j) item_cut[off + j] = cuts[k];
        off += cnt[k];
    }

    orc_work wk;
    wk.pr = &pr; wk.item_cut = item_cut; wk.item_piece = pieces; wk.item_val = val;
    wk.n_items = total; wk.next = 0; wk.stride = item_stride > 1 ? item_stride : 1;
    pthread_mutex_init(&wk.mu, NULL);
    if (n_threads < 1) n_threads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, orc_worker, &wk);
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&wk.mu);
    free(th);

    off = 0;
    for (int k = 0; k < n_cuts; ++k) {
        double s = 0.0, comp = 0.0;
        for (int j = 0; j < cnt[k]; ++j) {
            double term = val[off + j], t = s + term;
            if (fabs(s) >= fabs(term)) comp += (s - t) + term;
            else comp += (term - t) + s;
            s = t;
            if (piece_out) piece_out[off + j] = term;
        }
        sigma_out[k] = s + comp;
        off += cnt[k];
    }
    free(cnt); free(pieces); free(item_cut); free(val);
    orc_problem_free(&pr);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Eq. gain_fin with P_NLI,i = G(f_i) B_i:                                 */
/*   eta_i = (16/27) gamma_i^2 B_i Sigma_i / P_i^3   [1/W^2]               */
/* ---------------------------------------------------------------------- */
void orc_eta_from_sigma(int n_cuts, const double *sigma, const double *gamma, const double *B,
                        const double *P, double *eta, double *pnli)
{
    for (int k = 0; k < n_cuts; ++k) {
        double g = 16.0 / 27.0 * gamma[k] * gamma[k] * sigma[k] * B[k];
        if (pnli) pnli[k] = g;
        eta[k] = (P[k] > 0.0) ? g / (P[k] * P[k] * P[k]) : NAN;
    }
}

/* ---------------------------------------------------------------------- */
/* Sec. IV, Eq. loss: amplifiers restore the launch profile, so           */
/*   SNR_i = P_i / (eta_i P_i^3 + P_ASE,i),                               */
/*   P_ASE,i = NF_i h f_i (G_i - 1) B_i,  G_i = 1 / rho(L, f_i),          */
/* optional transceiver noise 1/SNR += 1/SNR_TRX, and the throughput      */
/*   T = 2 sum_{i not guard} B_i log2(1 + SNR_i)    [Tb/s with B in THz]. */
/* ---------------------------------------------------------------------- */
double orc_snr_throughput(int n, const double *f, const double *B, const double *P,
                          const double *alpha, const double *scale, const double *fibre, int n_edges,
                          const double *eta, const double *nf_dB, double snr_trx_dB,
                          const unsigned char *guard, double *snr, double *pase)
{
    orc_plan pl = {n, f, B, P, alpha};
    double f_ref = fibre[1], Cr = fibre[5], alpha_R = fibre[6], L = fibre[0];
    double n_spans = fibre[7] >= 1.0 ? fibre[7] : 1.0;
    double kappa = orc_kappa(&pl, L, Cr, alpha_R);
    double lnN = orc_lnN(&pl, kappa, f_ref), lnPtot = log(orc_ptot(&pl));
    double *aL = NULL;
    if (fibre[8] == 1.0) {          /* R2: ln rho(L, f_i) from the ODE on the same z-grid */
        size_t nm = (size_t)n * (size_t)(n_edges > 1 ? n_edges - 1 : 1);
        double *ta = (double *)malloc(sizeof(double) * nm), *tb = (double *)malloc(sizeof(double) * nm);
        aL = (double *)malloc(sizeof(double) * (size_t)n);
        if (orc_raman_profile(n, f, P, alpha, scale, fibre, n_edges, ta, tb, aL) != 0) {
            free(ta); free(tb); free(aL);
            return NAN;
        }
        free(ta); free(tb);
    }
    double T = 0.0;
    for (int i = 0; i < n; ++i) {
        double lr = aL ? aL[i] : orc_lnrho_c(&pl, i, L, f[i], lnPtot, lnN, kappa, f_ref);
        double gain = exp(-lr);
        double nf = pow(10.0, nf_dB[i] / 10.0);
        /* one amplifier per span, each restoring the launch power */
        double pa = n_spans * nf * ORC_H_PLANCK * (f[i] * 1e12) * (gain - 1.0) * (B[i] * 1e12);
        if (pase) pase[i] = pa;
        if (P[i] <= 0.0 || (guard && guard[i])) { snr[i] = 0.0; continue; }
        double s = P[i] / (eta[i] * P[i] * P[i] * P[i] + pa);
        if (snr_trx_dB > 0.0) s = 1.0 / (1.0 / s + pow(10.0, -snr_trx_dB / 10.0));
        snr[i] = s;
        T += 2.0 * B[i] * log2(1.0 + s);
    }
    free(aL);
    return T;
}

int orc_sigma(int n, const double *f, const double *B, const double *P, const double *alpha,
              const double *scale, const double *fibre, const int *quad, double eps, const int *cuts,
              int n_cuts, int n_threads, int unit_integrand, double *sigma_out, double *piece_out)
{
    return orc_sigma_sampled(n, f, B, P, alpha, scale, fibre, quad, eps, cuts, n_cuts, n_threads,
                             unit_integrand, 1, sigma_out, piece_out);
}
