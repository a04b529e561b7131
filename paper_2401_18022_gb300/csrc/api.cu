// Host side of the ISRS GN library: argument validation, the per-plan piece
// list (App. A, Eqs. q1a..q4d: channel-pair cells cut into quadrant pieces),
// the work-tile queue, the z-grid tables (Sec. III-A: equal power drop per
// step), workspace management and the C ABI entry points of isrs_gn.h.
//
// Everything that depends on the launch powers runs in the kernels; the
// plan-dependent tables built here are cached in HBM per plan signature.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "../../include/isrs_gn.h"
#include "isrs_kernels.h"
#include "ptr_class.h"

using namespace isrs;

namespace {

constexpr double kCnmPerPs = 299792.458;

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

// Geometry of one launch signature: plans, CUT lists, profiles -> plan,
// quadrature and tile.  Owned by the handle's cache.
struct Geom {
    uint64_t key = 0;
    int n_prof = 0, n_plans = 0, n_steps = 0, G = 0;
    double eps_v1 = 0.0;
    double phase_rev_max = 0.0;   // bound of |phi| L / 2pi over all pieces
    int n_items = 0, n_slots = 0;
    int64_t n_pieces = 0, n_points = 0, n_points_unfolded = 0;
    float dz_max = 0.f;
    std::vector<int> prof_ch_off, plan_ch_off, plan_n, prof_plan;
    int total_prof_ch = 0, total_plan_ch = 0;
    DevBuf pieces, items, slot_items, slot_cut, prof_slot_off, plan_ch_off_d, plan_n_d, prof_ch_off_d,
        prof_plan_d, ch_frel, ch_B, ch_alpha, ch_gamma, ch_nf, guard, zs_a, zs_b, zs_d, zs_g, item_slot, zs_gseg,
        seg;
    float phi_seg[3] = {0.f, 0.f, 0.f};
    bool has_nf = false, has_guard = false;
    // Raman-ODE profile: partner windows and gain scale per plan channel, RK4
    // steps per half z-step, largest candidate count of a piece
    int profile = 0, nc_max = 1, n_rk = 0, max_plan_n = 0;
    DevBuf win_lo, win_hi, ch_scale, half_steps;
    // Raman-ODE gradient: per work tile the rows of the plan channels its
    // pieces touch, per piece its local rows {a, b, CUT, first candidate},
    // and per plan channel the (row, slot) pairs the gather sums in tile order
    int64_t n_tab_rows = 0;
    DevBuf tab_row_off, tab_prow, tab_gath_off, tab_gath;
    // multi-channel-interference cells on their own grid: work items over
    // triangular cell ranges and, per output slot, their item range
    int G_mci = 0, n_mci_items = 0;
    double mci_phase_rev_max = 0.0;
    DevBuf mci_items, slot_items2, item_slot_all;   // item_slot_all: regular then MCI items
    // replayable graph of the batched launch (prep -> quadrature -> finish)
    cudaGraphExec_t gexec = nullptr;
    uint64_t gkey = 0;                 // fibre, precision and tile the graph was captured with
    std::vector<void *> gptrs;         // workspace pointers baked into the graph
    ~Geom();                           // frees whatever device tables it still holds
};

}  // namespace

struct isrs_handle_s {
    int device = 0;
    int num_sms = 1;
    std::string err;
    DevBuf paths, kapL;
    DevBuf P, pd_d, pd_f, step_d, step_f, lnrho_L, ptot, partial, counter, o_sigma, o_pnli, o_eta, o_snr,
        o_pase, o_T, gA, gK, gPd, gVs, gY, dbg, ybar, dTdP, ab, ab_f, ode_y, gAB, gV, gAt, partial_mci, tab_rows,
        tab_rowsV;
    std::vector<std::unique_ptr<Geom>> cache;   // most recent first
    int tile_points = 0, tile_threads = 0;
    int64_t last_points = 0, last_psteps = 0;
    int last_launches = 0;
    cudaStream_t cap_stream = nullptr;   // private stream used only to capture graphs
    bool last_graph = false;             // the last batched call replayed a graph
    cudaEvent_t ev[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // [quad, adjoint][start, end]
    bool ev_valid[2] = {false, false};
    // host-side fault injection (isrs_debug_inject_fault): kind 1 allocation, 2 CUDA call
    int inj_kind = 0, inj_countdown = 0;
    // split gradient: the shard whose buckets the last isrs_gn_grad_shard_fwd left
    DevBuf eta_all;                      // [4 n]: gathered eta, then SNR, P_NLI, P_ASE per channel
    bool shard_valid = false;
    uint64_t shard_key = 0;
    isrs_fibre shard_fibre;
    isrs_quad shard_quad;
    int shard_n = 0;
};

namespace {

// ----------------------------------------------------------------------------
// errors
// ----------------------------------------------------------------------------
isrs_status fail(isrs_handle h, isrs_status s, const char *fmt, ...)
{
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return s;
}

// NVTX range over a scope (host timeline of a profiler; no cost without one).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

// True once, when an armed injection of this kind reaches its count.
bool inject_hit(isrs_handle h, int kind)
{
    if (!h || h->inj_kind != kind) return false;
    if (--h->inj_countdown > 0) return false;
    h->inj_kind = 0;
    return true;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        if (inject_hit(h, 2))                                                                 \
            return fail(h, ISRS_ERR_CUDA, "%s: injected failure (not executed)", #call);      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(h, e_ == cudaErrorMemoryAllocation ? ISRS_ERR_ALLOC : ISRS_ERR_CUDA,  \
                        "%s: %s", #call, cudaGetErrorString(e_));                             \
    } while (0)

#ifdef ISRS_DEBUG
constexpr bool kDebugBuild = true;
#else
constexpr bool kDebugBuild = false;
#endif

// Debug build: the first failed device bounds check since the last call
// (its code, see isrs_debug.cuh) becomes ISRS_ERR_CHECK; the flag is cleared.
isrs_status dbg_check(isrs_handle h, cudaStream_t st)
{
    if (!kDebugBuild || !h->dbg.p) return ISRS_OK;
    unsigned code = 0;
    CK(cudaMemcpyAsync(&code, h->dbg.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (code == 0) return ISRS_OK;
    CK(cudaMemsetAsync(h->dbg.p, 0, sizeof(unsigned), st));
    return fail(h, ISRS_ERR_CHECK, "device bounds check %u failed", code);
}

isrs_status ensure(isrs_handle h, DevBuf &b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (b.cap >= bytes) return ISRS_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    if (inject_hit(h, 1)) return fail(h, ISRS_ERR_ALLOC, "cudaMalloc(%zu) failed: injected", bytes);
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        b.p = nullptr;
        return fail(h, ISRS_ERR_ALLOC, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    b.cap = bytes;
    return ISRS_OK;
}

void release(DevBuf &b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
}

template <typename T>
isrs_status upload(isrs_handle h, DevBuf &b, const std::vector<T> &v, cudaStream_t st)
{
    isrs_status s = ensure(h, b, v.size() * sizeof(T));
    if (s != ISRS_OK) return s;
    if (!v.empty()) CK(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    return ISRS_OK;
}

// Where a caller's pointer lives relative to the current device (ptr_class.h).
int where_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return kPtrHost;
    }
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        return kPtrOtherDevice;
    }
    return ptr_class((int)a.type, a.device, cur);
}

bool is_device_ptr(const void *p) { return where_ptr(p) == kPtrDevice; }

// Rejects a device pointer of another GPU (a kernel on this device would
// write into that GPU's memory, or fault without peer access).
isrs_status check_ptr(isrs_handle h, const void *p, const char *name)
{
    if (p && where_ptr(p) == kPtrOtherDevice)
        return fail(h, ISRS_ERR_INVALID_ARG, "%s is device memory of another GPU", name);
    return ISRS_OK;
}

// Every call copies results to the host or synchronises `stream`, which a
// stream capture forbids: reject a capturing stream before issuing any work,
// so that the caller's capture stays valid.
isrs_status reject_capture(isrs_handle h, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone)
        return fail(h, ISRS_ERR_UNSUPPORTED, "the stream is being captured; this call synchronises it");
    return ISRS_OK;
}

// Records event `pos` (0 start, 1 end) of kernel class `which` on the stream,
// unless the stream is being captured.
isrs_status mark(isrs_handle h, int which, int pos, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) {
        h->ev_valid[which] = false;
        return ISRS_OK;
    }
    if (!h->ev[which][pos]) CK(cudaEventCreate(&h->ev[which][pos]));
    CK(cudaEventRecord(h->ev[which][pos], st));
    if (pos == 1) h->ev_valid[which] = true;
    return ISRS_OK;
}

// ----------------------------------------------------------------------------
// validation
// ----------------------------------------------------------------------------
bool finite(double x) { return std::isfinite(x); }

isrs_status check_fibre(isrs_handle h, const isrs_fibre *fb)
{
    if (!fb) return fail(h, ISRS_ERR_INVALID_ARG, "fibre is NULL");
    if (!(fb->L_km > 0.0) || !finite(fb->L_km)) return fail(h, ISRS_ERR_INVALID_ARG, "L_km must be > 0");
    if (!finite(fb->f_ref_THz) || !finite(fb->beta2) || !finite(fb->beta3) || !finite(fb->beta4) ||
        !finite(fb->Cr))
        return fail(h, ISRS_ERR_INVALID_ARG, "non-finite fibre parameter");
    if (!(fb->alpha_R_per_km >= 0.0) || !finite(fb->alpha_R_per_km))
        return fail(h, ISRS_ERR_INVALID_ARG, "alpha_R must be >= 0");
    if (fb->n_spans < 0 || fb->n_spans > 100) return fail(h, ISRS_ERR_INVALID_ARG, "n_spans must be in [0, 100]");
    if (fb->profile != ISRS_PROFILE_CLOSED_FORM && fb->profile != ISRS_PROFILE_RAMAN_ODE)
        return fail(h, ISRS_ERR_INVALID_ARG, "bad profile %d", fb->profile);
    if (fb->profile == ISRS_PROFILE_RAMAN_ODE &&
        (!finite(fb->raman_max_THz) || (fb->raman_photon != 0 && fb->raman_photon != 1)))
        return fail(h, ISRS_ERR_INVALID_ARG, "bad Raman cut-off or photon flag");
    return ISRS_OK;
}

isrs_status check_plan(isrs_handle h, const isrs_channels *c)
{
    if (!c) return fail(h, ISRS_ERR_INVALID_ARG, "channels is NULL");
    if (c->n_ch < 1) return fail(h, ISRS_ERR_INVALID_ARG, "n_ch must be >= 1");
    if (!c->f_THz || !c->B_THz || !c->alpha_per_km || !c->gamma_per_W_km)
        return fail(h, ISRS_ERR_INVALID_ARG, "channel array is NULL");
    for (int k = 0; k < c->n_ch; ++k) {
        if (!finite(c->f_THz[k]) || !(c->B_THz[k] > 0.0) || !finite(c->B_THz[k]))
            return fail(h, ISRS_ERR_INVALID_ARG, "channel %d: bad frequency or bandwidth", k);
        if (!(c->alpha_per_km[k] >= 0.0) || !finite(c->alpha_per_km[k]) || !finite(c->gamma_per_W_km[k]))
            return fail(h, ISRS_ERR_INVALID_ARG, "channel %d: bad alpha or gamma", k);
        if (c->nf_dB && !finite(c->nf_dB[k])) return fail(h, ISRS_ERR_INVALID_ARG, "channel %d: bad NF", k);
        if (c->raman_scale && !(c->raman_scale[k] > 0.0 && finite(c->raman_scale[k])))
            return fail(h, ISRS_ERR_INVALID_ARG, "channel %d: raman_scale must be > 0", k);
        if (k > 0) {
            if (!(c->f_THz[k] > c->f_THz[k - 1]))
                return fail(h, ISRS_ERR_INVALID_ARG, "channels not sorted at %d", k);
            if (c->f_THz[k - 1] + 0.5 * c->B_THz[k - 1] > c->f_THz[k] - 0.5 * c->B_THz[k] + 1e-12)
                return fail(h, ISRS_ERR_INVALID_ARG, "channels %d and %d overlap", k - 1, k);
        }
    }
    return ISRS_OK;
}

isrs_status check_quad(isrs_handle h, const isrs_quad *q)
{
    if (!q) return fail(h, ISRS_ERR_INVALID_ARG, "quad is NULL");
    if (q->G < 1 || q->G > kMaxG) return fail(h, ISRS_ERR_INVALID_ARG, "G must be in [1, %d]", kMaxG);
    if (q->n_edges < 2 || q->n_edges > kMaxSteps + 1)
        return fail(h, ISRS_ERR_INVALID_ARG, "n_edges must be in [2, %d]", kMaxSteps + 1);
    if (!(q->eps_v1 > 0.0 && q->eps_v1 < 1.0)) return fail(h, ISRS_ERR_INVALID_ARG, "eps_v1 must be in (0,1)");
    if (q->cell_set != ISRS_CELLS_SCI_XCI && q->cell_set != ISRS_CELLS_ALL)
        return fail(h, ISRS_ERR_INVALID_ARG, "bad cell_set");
    if (q->precision != ISRS_PREC_FP32 && q->precision != ISRS_PREC_FP64)
        return fail(h, ISRS_ERR_INVALID_ARG, "bad precision");
    if (!finite(q->snr_trx_dB)) return fail(h, ISRS_ERR_INVALID_ARG, "bad snr_trx_dB");
    if (!finite(q->ode_h_km)) return fail(h, ISRS_ERR_INVALID_ARG, "bad ode_h_km");
    if (q->G_mci < 0 || q->G_mci > 32) return fail(h, ISRS_ERR_INVALID_ARG, "G_mci must be in [0, 32]");
    if (q->G_mci > 0 && q->cell_set != ISRS_CELLS_ALL)
        return fail(h, ISRS_ERR_INVALID_ARG, "G_mci needs cell_set ISRS_CELLS_ALL");
    return ISRS_OK;
}

isrs_status check_powers(isrs_handle h, const double *P, int n)
{
    double tot = 0.0;
    for (int k = 0; k < n; ++k) {
        if (!(P[k] >= 0.0) || !finite(P[k])) return fail(h, ISRS_ERR_INVALID_ARG, "P[%d] must be finite and >= 0", k);
        tot += P[k];
    }
    if (!(tot > 0.0)) return fail(h, ISRS_ERR_INVALID_ARG, "total launch power must be > 0");
    return ISRS_OK;
}

// ----------------------------------------------------------------------------
// signature hashing (FNV-1a)
// ----------------------------------------------------------------------------
struct Hasher {
    uint64_t v = 1469598103934665603ull;
    void bytes(const void *p, size_t n)
    {
        const unsigned char *c = static_cast<const unsigned char *>(p);
        for (size_t k = 0; k < n; ++k) {
            v ^= c[k];
            v *= 1099511628211ull;
        }
    }
    template <typename T> void val(const T &x) { bytes(&x, sizeof(T)); }
};

// ----------------------------------------------------------------------------
// pieces of one CUT (App. A, Eqs. q1a..q4d).  Cells (a,b) with F_a in channel
// a, F_b in channel b; the mirror cell (b,a) has the same Riemann sum because
// the integrand is symmetric in (f1, f2), so only a <= b (ALL) or a == i
// (SCI+XCI) is kept with multiplicity 2, and in the SCI cell the (-,+)
// quadrant is folded into (+,-).
// ----------------------------------------------------------------------------
int split_interval(double lo, double hi, int *sg, double *plo, double *phi)
{
    int k = 0;
    if (hi > 0.0) { sg[k] = +1; plo[k] = lo > 0.0 ? lo : 0.0; phi[k] = hi; ++k; }
    if (lo < 0.0) { sg[k] = -1; plo[k] = hi < 0.0 ? -hi : 0.0; phi[k] = -lo; ++k; }
    return k;
}

// first channel whose upper edge is > F (channels sorted, disjoint)
int first_above(const isrs_channels *c, double F)
{
    int lo = 0, hi = c->n_ch;
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (c->f_THz[mid] + 0.5 * c->B_THz[mid] > F) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// last channel whose lower edge is < F
int last_below(const isrs_channels *c, double F)
{
    int lo = -1, hi = c->n_ch - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (c->f_THz[mid] - 0.5 * c->B_THz[mid] < F) lo = mid; else hi = mid - 1;
    }
    return lo;
}

isrs_status cut_pieces(isrs_handle h, const isrs_channels *c, int plan, int i, int cell_set,
                       std::vector<DevPiece> &out)
{
    const int n = c->n_ch;
    const double fi = c->f_THz[i];
    for (int a = 0; a < n; ++a) {
        for (int b = 0; b < n; ++b) {
            if (cell_set == ISRS_CELLS_SCI_XCI) {
                if (a != i) continue;               // keep (i, b); (b, i) is its mirror
            } else if (b < a) {
                continue;                           // keep a <= b
            }
            const bool mirror_cell = (a != b);
            int sa[2], sb[2];
            double xl[2], xh[2], yl[2], yh[2];
            const int na = split_interval(c->f_THz[a] - 0.5 * c->B_THz[a] - fi,
                                          c->f_THz[a] + 0.5 * c->B_THz[a] - fi, sa, xl, xh);
            const int nb = split_interval(c->f_THz[b] - 0.5 * c->B_THz[b] - fi,
                                          c->f_THz[b] + 0.5 * c->B_THz[b] - fi, sb, yl, yh);
            for (int u = 0; u < na; ++u) {
                for (int v = 0; v < nb; ++v) {
                    if (!(xh[u] > xl[u]) || !(yh[v] > yl[v])) continue;
                    float mult = mirror_cell ? 2.0f : 1.0f;
                    if (!mirror_cell && sa[u] != sb[v]) {
                        // diagonal cell: quadrants (+,-) and (-,+) are mirrors
                        if (sa[u] < 0) continue;
                        mult = 2.0f;
                    }
                    DevPiece p;
                    std::memset(&p, 0, sizeof(p));
                    p.xlo = xl[u]; p.xhi = xh[u]; p.ylo = yl[v]; p.yhi = yh[v];
                    p.cut = i; p.a = a; p.b = b; p.plan = plan;
                    p.flags = (sa[u] < 0 ? 1 : 0) | (sb[v] < 0 ? 2 : 0);
                    p.mult = mult;
                    // range of F_c - f_i = s1 |f1| + s2 |f2| over the rectangle
                    const double ux0 = sa[u] > 0 ? xl[u] : -xh[u], ux1 = sa[u] > 0 ? xh[u] : -xl[u];
                    const double uy0 = sb[v] > 0 ? yl[v] : -yh[v], uy1 = sb[v] > 0 ? yh[v] : -yl[v];
                    const int c0 = first_above(c, fi + ux0 + uy0);
                    const int c1 = last_below(c, fi + ux1 + uy1);
                    if (c1 < c0) continue;                   // F_c always in a gap: zero
                    if (c1 - c0 + 1 > kMaxCand)
                        return fail(h, ISRS_ERR_UNSUPPORTED,
                                    "a piece's F_c range covers %d channels (max %d)", c1 - c0 + 1, kMaxCand);
                    p.c_lo = c0;
                    p.c_hi = c1;
                    out.push_back(p);
                }
            }
        }
    }
    return ISRS_OK;
}

// ----------------------------------------------------------------------------
// z-grid (Sec. III-A, App. A): equal power drop per step,
//   exp(-a z_e) = 1 - (e/(N_M - 1)) (1 - exp(-a L)),  z-tilde_m = z_m (midpoint)
// Stored per step as FP64 {z_m, dz_m}, FP32 {z_m, dz_m} and the phase
// positions in revolutions (z / 2 pi) as float-float pairs.
// ----------------------------------------------------------------------------
// Segments of the span for the segmented small-phase series: level v cuts
// [0, L] into 2^{v+1} segments at the step edges nearest to s L / 2^{v+1}
// (fewer where two targets share an edge).  Per segment {m0, m1, centre/2pi
// as float-float}; per level and step the moments g_n (n <= 18) of the step
// about its segment's centre; per level the |phi| limit 6 / (longest
// segment), below which 19 moments truncate the series by < 2e-8.
void segment_tables(const std::vector<double> &ze, std::vector<float4> &gseg, std::vector<int4> &seg,
                    float *phi_seg)
{
    const int M = (int)ze.size() - 1;
    const double L = ze[M];
    gseg.assign((size_t)kSegLevels * M * 5, make_float4(0.f, 0.f, 0.f, 0.f));
    seg.assign(kSegSlots, make_int4(0, 0, 0, 0));
    int slot = 0;
    for (int v = 0; v < kSegLevels; ++v) {
        const int J = 2 << v;
        std::vector<int> b{0};
        for (int s = 1; s < J; ++s) {
            int best = 0;
            for (int e = 0; e <= M; ++e)
                if (std::fabs(ze[e] - s * L / J) < std::fabs(ze[best] - s * L / J)) best = e;
            if (best > b.back() && best < M) b.push_back(best);
        }
        b.push_back(M);
        double lmax = 0.0;
        const int nseg = (int)b.size() - 1;
        for (int s = 0; s < (1 << (v + 1)); ++s, ++slot) {
            if (s >= nseg) {                    // fewer segments than slots: an empty one
                seg[slot] = make_int4(M, M, 0, 0);
                continue;
            }
            const int m0 = b[s], m1 = b[s + 1];
            const double c = 0.5 * (ze[m0] + ze[m1]);
            lmax = std::max(lmax, ze[m1] - ze[m0]);
            const double cr = c / (2.0 * 3.14159265358979323846);
            const float hi = (float)cr, lo = (float)(cr - (double)hi);
            int hib, lob;
            std::memcpy(&hib, &hi, 4);
            std::memcpy(&lob, &lo, 4);
            seg[slot] = make_int4(m0, m1, hib, lob);
            for (int m = m0; m < m1; ++m) {
                const double lo2 = ze[m] - c, hi2 = ze[m + 1] - c;
                float g[20] = {0.f};
                double pa = lo2, pb = hi2;
                for (int n = 0; n <= 18; ++n) {
                    g[n] = (float)((pb - pa) / ((n + 1) * (hi2 - lo2)));
                    pa *= lo2;
                    pb *= hi2;
                }
                for (int q = 0; q < 5; ++q)
                    gseg[((size_t)v * M + m) * 5 + q] = make_float4(g[4 * q], g[4 * q + 1], g[4 * q + 2], g[4 * q + 3]);
            }
        }
        phi_seg[v] = (float)(6.0 / lmax);
    }
}

void zgrid_tables(double L, double a, int n_edges, std::vector<float4> &za, std::vector<float4> &zb,
                  std::vector<double2> &zd, float &dz_max, std::vector<float4> *zg = nullptr,
                  std::vector<float4> *gseg = nullptr, std::vector<int4> *seg = nullptr, float *phi_seg = nullptr)
{
    std::vector<double> ze(n_edges);
    const double drop = a > 0.0 ? -std::expm1(-a * L) : 0.0;
    for (int e = 0; e < n_edges; ++e) {
        const double t = (double)e / (double)(n_edges - 1);
        ze[e] = a > 0.0 ? -std::log1p(-t * drop) / a : t * L;
    }
    ze[n_edges - 1] = L;
    const int M = n_edges - 1;
    za.resize(M); zb.resize(M); zd.resize(M);
    const double inv2pi = 1.0 / (2.0 * 3.14159265358979323846);
    double dmax = 0.0;
    for (int m = 0; m < M; ++m) {
        const double zm = 0.5 * (ze[m] + ze[m + 1]);
        const double dz = ze[m + 1] - ze[m];
        dmax = std::max(dmax, dz);
        zd[m] = make_double2(zm, dz);
        // {z_m, z_m^2 + dz_m^2/12 (second moment incl. the sinc term), log2 dz_m, dz_m}
        za[m] = make_float4((float)zm, (float)(zm * zm + dz * dz / 12.0), (float)std::log2(dz), (float)dz);
        const double re = ze[m + 1] * inv2pi, rm = zm * inv2pi;
        const float reh = (float)re;
        zb[m] = make_float4(reh, (float)(re - (double)reh), (float)rm, 0.f);
    }
    dz_max = (float)dmax;
    if (zg) {
        // centred step moments g_n(m) = mean of (zeta - L/2)^n over [ze_m, ze_{m+1}]
        // = (b^{n+1} - a^{n+1}) / ((n + 1)(b - a)), n = 0..18, and g_19 = 0
        zg->assign(5 * (size_t)M, make_float4(0.f, 0.f, 0.f, 0.f));
        for (int m = 0; m < M; ++m) {
            const double lo = ze[m] - 0.5 * L, hi = ze[m + 1] - 0.5 * L;
            float g[20] = {0.f};
            double pa = lo, pb = hi;
            for (int n = 0; n <= 18; ++n) {
                g[n] = (float)((pb - pa) / ((n + 1) * (hi - lo)));
                pa *= lo;
                pb *= hi;
            }
            for (int q = 0; q < 5; ++q)
                (*zg)[5 * m + q] = make_float4(g[4 * q], g[4 * q + 1], g[4 * q + 2], g[4 * q + 3]);
        }
    }
    if (gseg && seg && phi_seg) segment_tables(ze, *gseg, *seg, phi_seg);
}

// ----------------------------------------------------------------------------
// Build (or fetch from the cache) the geometry of a launch.
//   cuts_per_plan[q]: CUT list of plan q (all channels if empty)
//   prof_plan: plan of each profile; every profile evaluates its plan's CUT list
// ----------------------------------------------------------------------------
isrs_status get_geom(isrs_handle h, const isrs_fibre *fb, int n_plans, const isrs_channels *plans,
                     const std::vector<std::vector<int>> &cuts_per_plan, const std::vector<int> &prof_plan,
                     const isrs_quad *q, cudaStream_t st, Geom **out)
{
    Hasher hs;
    hs.val(n_plans);
    for (int k = 0; k < n_plans; ++k) {
        const isrs_channels &c = plans[k];
        hs.val(c.n_ch);
        hs.bytes(c.f_THz, sizeof(double) * c.n_ch);
        hs.bytes(c.B_THz, sizeof(double) * c.n_ch);
        hs.bytes(c.alpha_per_km, sizeof(double) * c.n_ch);
        hs.bytes(c.gamma_per_W_km, sizeof(double) * c.n_ch);
        hs.val((int)(c.nf_dB != nullptr));
        if (c.nf_dB) hs.bytes(c.nf_dB, sizeof(double) * c.n_ch);
        hs.val((int)(c.guard != nullptr));
        if (c.guard) hs.bytes(c.guard, c.n_ch);
        hs.val((int)cuts_per_plan[k].size());
        if (!cuts_per_plan[k].empty()) hs.bytes(cuts_per_plan[k].data(), sizeof(int) * cuts_per_plan[k].size());
    }
    hs.val((int)prof_plan.size());
    hs.bytes(prof_plan.data(), sizeof(int) * prof_plan.size());
    hs.val(q->G); hs.val(q->n_edges); hs.val(q->eps_v1); hs.val(q->cell_set);
    hs.val(fb->L_km); hs.val(fb->f_ref_THz); hs.val(fb->alpha_R_per_km);
    hs.val(h->tile_points);
    hs.val(q->G_mci);
    hs.val(fb->profile);
    const double ode_h = q->ode_h_km > 0.0 ? q->ode_h_km : 0.25;
    if (fb->profile == ISRS_PROFILE_RAMAN_ODE) {
        hs.val(fb->raman_max_THz);
        hs.val(ode_h);
        for (int k = 0; k < n_plans; ++k) {
            hs.val((int)(plans[k].raman_scale != nullptr));
            if (plans[k].raman_scale) hs.bytes(plans[k].raman_scale, sizeof(double) * plans[k].n_ch);
        }
    }
    const uint64_t key = hs.v;
    for (size_t k = 0; k < h->cache.size(); ++k) {
        if (h->cache[k]->key == key) {
            if (k != 0) std::rotate(h->cache.begin(), h->cache.begin() + k, h->cache.begin() + k + 1);
            *out = h->cache[0].get();
            return ISRS_OK;
        }
    }

    std::unique_ptr<Geom> g(new (std::nothrow) Geom());
    if (!g) return fail(h, ISRS_ERR_ALLOC, "host allocation failed");
    g->key = key;
    g->n_plans = n_plans;
    g->n_prof = (int)prof_plan.size();
    g->n_steps = q->n_edges - 1;
    g->G = q->G;
    g->eps_v1 = q->eps_v1;
    const int64_t G2 = (int64_t)q->G * q->G;

    // channel tables
    std::vector<double> frel, Bv, av, gv, nfv;
    std::vector<unsigned char> gd;
    g->has_nf = false;
    g->has_guard = false;
    for (int k = 0; k < n_plans; ++k) {
        g->has_nf |= plans[k].nf_dB != nullptr;
        g->has_guard |= plans[k].guard != nullptr;
    }
    for (int k = 0; k < n_plans; ++k) {
        const isrs_channels &c = plans[k];
        g->plan_ch_off.push_back((int)frel.size());
        g->plan_n.push_back(c.n_ch);
        for (int j = 0; j < c.n_ch; ++j) {
            frel.push_back(c.f_THz[j] - fb->f_ref_THz);
            Bv.push_back(c.B_THz[j]);
            av.push_back(c.alpha_per_km[j]);
            gv.push_back(c.gamma_per_W_km[j]);
            nfv.push_back(c.nf_dB ? c.nf_dB[j] : 0.0);
            gd.push_back(c.guard ? c.guard[j] : 0);
        }
    }
    g->total_plan_ch = (int)frel.size();

    // pieces per plan and CUT (with a separate MCI grid only the SCI and XCI
    // cells become pieces)
    const bool mci = q->cell_set == ISRS_CELLS_ALL && q->G_mci > 0;
    const int piece_cells = mci ? ISRS_CELLS_SCI_XCI : q->cell_set;
    g->G_mci = mci ? q->G_mci : 0;
    std::vector<DevPiece> pieces;
    std::vector<std::vector<std::pair<int, int>>> cut_range(n_plans);   // per plan, per listed CUT
    for (int k = 0; k < n_plans; ++k) {
        const std::vector<int> &cl = cuts_per_plan[k];
        const int ncut = cl.empty() ? plans[k].n_ch : (int)cl.size();
        for (int s = 0; s < ncut; ++s) {
            const int i = cl.empty() ? s : cl[s];
            const int p0 = (int)pieces.size();
            isrs_status st2 = cut_pieces(h, &plans[k], k, i, piece_cells, pieces);
            if (st2 != ISRS_OK) return st2;
            cut_range[k].push_back({p0, (int)pieces.size()});
        }
    }
    g->n_pieces = (int64_t)pieces.size();

    // Bound of the phase phi z over all pieces (Eq. phi): the FP32 path forms
    // phi z / 2pi in float-float and rounds it on the FMA pipe, valid below 2^22.
    {
        const double pi = 3.14159265358979323846;
        double tmax = 0.0;
        for (const DevPiece &pc : pieces) {
            const double fi = std::fabs(plans[pc.plan].f_THz[pc.cut] - fb->f_ref_THz);
            const double v1 = pc.xhi * pc.yhi, s12 = pc.xhi + pc.yhi;
            const double br = std::fabs(fb->beta2) + pi * std::fabs(fb->beta3) * (s12 + 2.0 * fi) +
                              2.0 * pi * pi / 3.0 * std::fabs(fb->beta4) *
                                  (s12 * s12 + 1.5 * v1 + 3.0 * fi * s12 + 3.0 * fi * fi);
            tmax = std::max(tmax, 4.0 * pi * pi * v1 * br * fb->L_km / (2.0 * pi));
        }
        g->phase_rev_max = tmax;
        // MCI cells: bound over the whole band of every plan
        double tm = 0.0;
        if (mci)
            for (int k = 0; k < n_plans; ++k) {
                const isrs_channels &c = plans[k];
                const double flo = c.f_THz[0] - 0.5 * c.B_THz[0];
                const double fhi = c.f_THz[c.n_ch - 1] + 0.5 * c.B_THz[c.n_ch - 1];
                for (int i = 0; i < c.n_ch; ++i) {
                    const double xm = std::max(fhi - c.f_THz[i], c.f_THz[i] - flo);
                    const double fi = std::fabs(c.f_THz[i] - fb->f_ref_THz);
                    const double v1 = xm * xm, s12 = 2.0 * xm;
                    const double br = std::fabs(fb->beta2) + pi * std::fabs(fb->beta3) * (s12 + 2.0 * fi) +
                                      2.0 * pi * pi / 3.0 * std::fabs(fb->beta4) *
                                          (s12 * s12 + 1.5 * v1 + 3.0 * fi * s12 + 3.0 * fi * fi);
                    tm = std::max(tm, 4.0 * pi * pi * v1 * br * fb->L_km / (2.0 * pi));
                }
            }
        g->mci_phase_rev_max = tm;
    }

    // work items, output slots
    const int tile_pts = h->tile_points > 0 ? h->tile_points : (1 << 20);
    const int chunk = (int)std::max<int64_t>(1, tile_pts / G2);
    std::vector<DevItem> items, mitems;
    std::vector<int2> slot_items, slot_items2;
    std::vector<int> slot_cut, prof_slot_off, item_slot, mitem_slot;
    const int mchunk = mci ? (int)std::max<int64_t>(1, tile_pts / ((int64_t)q->G_mci * q->G_mci)) : 1;
    g->n_points = 0;
    g->n_points_unfolded = 0;
    for (int p = 0; p < g->n_prof; ++p) {
        const int k = prof_plan[p];
        g->prof_plan.push_back(k);
        g->prof_ch_off.push_back(g->total_prof_ch);
        g->total_prof_ch += plans[k].n_ch;
        prof_slot_off.push_back((int)slot_items.size());
        const std::vector<int> &cl = cuts_per_plan[k];
        for (size_t s = 0; s < cut_range[k].size(); ++s) {
            const int i = cl.empty() ? (int)s : cl[s];
            const int it0 = (int)items.size();
            const int slot = (int)slot_items.size();
            for (int a = cut_range[k][s].first; a < cut_range[k][s].second; a += chunk) {
                const int b = std::min(a + chunk, cut_range[k][s].second);
                items.push_back(DevItem{p, a, b, i});
                item_slot.push_back(slot);
            }
            for (int a = cut_range[k][s].first; a < cut_range[k][s].second; ++a) {
                g->n_points += G2;
                g->n_points_unfolded += (int64_t)(pieces[a].mult) * G2;
            }
            slot_items.push_back(make_int2(it0, (int)items.size()));
            slot_cut.push_back(i);
            if (mci) {
                // cells (a, b), a <= b, a, b != i: triangular index over n - 1 channels
                const int n2 = plans[k].n_ch - 1;
                const int ncell = n2 * (n2 + 1) / 2;
                const int m0 = (int)mitems.size();
                for (int t = 0; t < ncell; t += mchunk) {
                    mitems.push_back(DevItem{p, t, std::min(t + mchunk, ncell), i});
                    mitem_slot.push_back(slot);
                }
                slot_items2.push_back(make_int2(m0, (int)mitems.size()));
                g->n_points += (int64_t)ncell * q->G_mci * q->G_mci;
                g->n_points_unfolded += (int64_t)n2 * n2 * q->G_mci * q->G_mci;
            }
        }
    }
    prof_slot_off.push_back((int)slot_items.size());
    g->n_items = (int)items.size();
    g->n_slots = (int)slot_items.size();
    g->n_mci_items = (int)mitems.size();

    std::vector<float4> za, zb, zg, zgs;
    std::vector<int4> segv;
    std::vector<double2> zd;
    zgrid_tables(fb->L_km, fb->alpha_R_per_km, q->n_edges, za, zb, zd, g->dz_max, &zg, &zgs, &segv, g->phi_seg);

    // Raman-ODE profile: the partners of channel i are the k != i with
    // |f_k - f_i| <= raman_max_THz, one index window of the sorted plan; the
    // RK4 steps in each half of z-step m are ceil((dz_m / 2) / h).
    g->profile = fb->profile;
    std::vector<int> wlo, whi, hsteps;
    std::vector<double> scl;
    if (fb->profile == ISRS_PROFILE_RAMAN_ODE) {
        const double dfm = fb->raman_max_THz;
        for (int k = 0; k < n_plans; ++k) {
            const isrs_channels &c = plans[k];
            if (c.n_ch > kMaxRamanCh)
                return fail(h, ISRS_ERR_UNSUPPORTED, "Raman-ODE profile supports at most %d channels", kMaxRamanCh);
            g->max_plan_n = std::max(g->max_plan_n, c.n_ch);
            int lo = 0, hi = 0;
            for (int i = 0; i < c.n_ch; ++i) {
                if (dfm > 0.0) {
                    while (std::fabs(c.f_THz[lo] - c.f_THz[i]) > dfm) ++lo;
                    if (hi < i) hi = i;
                    while (hi + 1 < c.n_ch && std::fabs(c.f_THz[hi + 1] - c.f_THz[i]) <= dfm) ++hi;
                } else {
                    lo = 0;
                    hi = c.n_ch - 1;
                }
                wlo.push_back(lo);
                whi.push_back(hi);
                scl.push_back(c.raman_scale ? c.raman_scale[i] : 1.0);
            }
        }
        g->n_rk = 0;
        for (int m = 0; m < g->n_steps; ++m) {
            const int ns = std::max(1, (int)std::ceil(0.5 * zd[m].y / ode_h - 1e-9));
            hsteps.push_back(ns);
            g->n_rk += 2 * ns;
        }
        int ncm = 1;
        for (const DevPiece &pc : pieces) ncm = std::max(ncm, std::min(pc.c_hi - pc.c_lo + 1, kMaxCand));
        g->nc_max = ncm;
        if (quad_tab_smem_bytes(0, g->n_steps, q->G, ncm) > 200 * 1024)
            return fail(h, ISRS_ERR_UNSUPPORTED, "Raman-ODE tables of %d candidates x %d steps exceed shared memory",
                        ncm, g->n_steps);
    }
    std::vector<int> trow_off, gath_off;
    std::vector<int4> prow;
    std::vector<int2> gath;
    if (fb->profile == ISRS_PROFILE_RAMAN_ODE) {
        // the channels of a tile: its CUT, every piece's a and b and F_c
        // candidates (consecutive channels, so consecutive rows)
        prow.resize(pieces.size());
        trow_off.push_back(0);
        std::vector<int> chs, row_ch;
        for (const DevItem &it : items) {
            chs.clear();
            for (int k = it.piece0; k < it.piece1; ++k) {
                const DevPiece &pc = pieces[k];
                chs.push_back(pc.cut);
                chs.push_back(pc.a);
                chs.push_back(pc.b);
                for (int c = pc.c_lo; c <= std::min(pc.c_hi, pc.c_lo + kMaxCand - 1); ++c) chs.push_back(c);
            }
            std::sort(chs.begin(), chs.end());
            chs.erase(std::unique(chs.begin(), chs.end()), chs.end());
            const auto local = [&](int c) { return (int)(std::lower_bound(chs.begin(), chs.end(), c) - chs.begin()); };
            for (int k = it.piece0; k < it.piece1; ++k) {
                const DevPiece &pc = pieces[k];
                prow[k] = make_int4(local(pc.a), local(pc.b), local(pc.cut), local(pc.c_lo));
            }
            const int coff = g->plan_ch_off[prof_plan[it.prof]];
            for (int c : chs) row_ch.push_back(coff + c);
            trow_off.push_back(trow_off.back() + (int)chs.size());
        }
        g->n_tab_rows = trow_off.back();
        // gather lists by plan-concatenated channel, rows in tile order
        gath_off.assign(g->total_plan_ch + 1, 0);
        for (int c : row_ch) ++gath_off[c + 1];
        for (int c = 0; c < g->total_plan_ch; ++c) gath_off[c + 1] += gath_off[c];
        gath.resize(row_ch.size());
        std::vector<int> fill(gath_off.begin(), gath_off.end() - 1);
        for (size_t t = 0; t < items.size(); ++t)
            for (int r = trow_off[t]; r < trow_off[t + 1]; ++r) gath[fill[row_ch[r]]++] = make_int2(r, item_slot[t]);
    }

    isrs_status s;
#define UP(buf, vec) if ((s = upload(h, g->buf, vec, st)) != ISRS_OK) return s
    UP(pieces, pieces);
    UP(items, items);
    UP(slot_items, slot_items);
    UP(slot_cut, slot_cut);
    UP(prof_slot_off, prof_slot_off);
    UP(plan_ch_off_d, g->plan_ch_off);
    UP(plan_n_d, g->plan_n);
    UP(prof_ch_off_d, g->prof_ch_off);
    UP(prof_plan_d, g->prof_plan);
    UP(ch_frel, frel);
    UP(ch_B, Bv);
    UP(ch_alpha, av);
    UP(ch_gamma, gv);
    UP(ch_nf, nfv);
    UP(guard, gd);
    UP(zs_a, za);
    UP(zs_b, zb);
    UP(zs_d, zd);
    UP(zs_g, zg);
    UP(zs_gseg, zgs);
    UP(seg, segv);
    UP(item_slot, item_slot);
    if (mci) {
        UP(mci_items, mitems);
        UP(slot_items2, slot_items2);
        std::vector<int> slot_all(item_slot);
        slot_all.insert(slot_all.end(), mitem_slot.begin(), mitem_slot.end());
        UP(item_slot_all, slot_all);
    }
    if (g->profile == ISRS_PROFILE_RAMAN_ODE) {
        UP(win_lo, wlo);
        UP(win_hi, whi);
        UP(ch_scale, scl);
        UP(half_steps, hsteps);
        UP(tab_row_off, trow_off);
        UP(tab_prow, prow);
        UP(tab_gath_off, gath_off);
        UP(tab_gath, gath);
    }
#undef UP
    CK(cudaStreamSynchronize(st));   // host vectors die at return

    h->cache.insert(h->cache.begin(), std::move(g));
    while (h->cache.size() > 4) h->cache.pop_back();   // ~Geom frees the evicted tables and graph
    *out = h->cache[0].get();
    return ISRS_OK;
}

void free_geom(Geom *g);
Geom::~Geom() { free_geom(this); }

void free_geom(Geom *g)
{
    if (g->gexec) cudaGraphExecDestroy(g->gexec);
    g->gexec = nullptr;
    DevBuf *bufs[] = {&g->pieces, &g->items, &g->slot_items, &g->slot_cut, &g->prof_slot_off,
                      &g->plan_ch_off_d, &g->plan_n_d, &g->prof_ch_off_d, &g->prof_plan_d,
                      &g->ch_frel, &g->ch_B, &g->ch_alpha, &g->ch_gamma, &g->ch_nf,
                      &g->guard, &g->zs_a, &g->zs_b, &g->zs_d, &g->zs_g, &g->item_slot,
                      &g->win_lo, &g->win_hi, &g->ch_scale, &g->half_steps, &g->mci_items, &g->slot_items2,
                      &g->item_slot_all, &g->tab_row_off, &g->tab_prow, &g->tab_gath_off, &g->tab_gath,
                      &g->zs_gseg, &g->seg};
    for (DevBuf *b : bufs) release(*b);
}

struct Launch {
    Geom *g = nullptr;
    int precision = 0;
    int block = 256;
};

RamanParams raman_params(isrs_handle h, const isrs_fibre *fb, Geom *g, bool keep_nodes)
{
    RamanParams rp;
    std::memset(&rp, 0, sizeof(rp));
    rp.P = (const double *)h->P.p;
    rp.ch_frel = (const double *)g->ch_frel.p;
    rp.ch_alpha = (const double *)g->ch_alpha.p;
    rp.ch_scale = (const double *)g->ch_scale.p;
    rp.win_lo = (const int *)g->win_lo.p;
    rp.win_hi = (const int *)g->win_hi.p;
    rp.plan_ch_off = (const int *)g->plan_ch_off_d.p;
    rp.plan_n = (const int *)g->plan_n_d.p;
    rp.prof_ch_off = (const int *)g->prof_ch_off_d.p;
    rp.prof_plan = (const int *)g->prof_plan_d.p;
    rp.zs_d = (const double2 *)g->zs_d.p;
    rp.half_steps = (const int *)g->half_steps.p;
    rp.n_steps = g->n_steps;
    rp.f_ref = fb->f_ref_THz;
    rp.Cr = fb->Cr;
    rp.photon = fb->raman_photon;
    rp.ab = (double2 *)h->ab.p;
    rp.lnrho_L = (double *)h->lnrho_L.p;
    rp.y_nodes = keep_nodes ? (double *)h->ode_y.p : nullptr;
    return rp;
}

// Launch constants of the quadrature kernels over the handle's workspace.
QuadParams quad_params(isrs_handle h, const isrs_fibre *fb, Geom *g)
{
    QuadParams qp;
    std::memset(&qp, 0, sizeof(qp));
    qp.pieces = (const DevPiece *)g->pieces.p;
    qp.items = (const DevItem *)g->items.p;
    qp.n_items = g->n_items;
    qp.n_pieces = (int)g->n_pieces;
    qp.dbg = kDebugBuild ? (unsigned *)h->dbg.p : nullptr;
    qp.G = g->G;
    qp.eps_v1 = g->eps_v1;
    qp.n_steps = g->n_steps;
    qp.beta2 = fb->beta2;
    qp.beta3 = fb->beta3;
    qp.beta4 = fb->beta4;
    qp.ch_frel = (const double *)g->ch_frel.p;
    qp.ch_B = (const double *)g->ch_B.p;
    qp.ch_alpha = (const double *)g->ch_alpha.p;
    qp.plan_ch_off = (const int *)g->plan_ch_off_d.p;
    qp.pd_f = (const float *)h->pd_f.p;
    qp.pd_d = (const double *)h->pd_d.p;
    qp.prof_ch_off = (const int *)g->prof_ch_off_d.p;
    qp.prof_plan = (const int *)g->prof_plan_d.p;
    qp.step_f = (const float2 *)h->step_f.p;
    qp.step_d = (const double2 *)h->step_d.p;
    qp.zs_a = (const float4 *)g->zs_a.p;
    qp.zs_b = (const float4 *)g->zs_b.p;
    qp.zs_d = (const double2 *)g->zs_d.p;
    qp.zs_g = (const float4 *)g->zs_g.p;
    qp.zs_gseg = (const float4 *)g->zs_gseg.p;
    qp.seg = (const int4 *)g->seg.p;
    for (int v = 0; v < 3; ++v) qp.phi_seg[v] = g->phi_seg[v];
    qp.dz_max = g->dz_max;
    qp.kap_L = (const double *)h->kapL.p;
    qp.L = (float)fb->L_km;
    qp.n_spans = fb->n_spans > 1 ? fb->n_spans : 1;
    {
        const double lr = fb->L_km / (2.0 * 3.14159265358979323846);
        qp.Lrev_hi = (float)lr;
        qp.Lrev_lo = (float)(lr - (double)qp.Lrev_hi);
        qp.Ld = fb->L_km;
    }
    qp.partial = (double *)h->partial.p;
    qp.counter = (int *)h->counter.p;
    qp.ab = g->profile == ISRS_PROFILE_RAMAN_ODE ? (const double2 *)h->ab.p : nullptr;
    qp.nc_max = g->nc_max;
    qp.path_count = (unsigned long long *)h->paths.p;
    qp.plan_n = (const int *)g->plan_n_d.p;
    qp.mci_n_max = 0;
    for (int k = 0; k < g->n_plans; ++k) qp.mci_n_max = std::max(qp.mci_n_max, g->plan_n[k]);
    return qp;
}

// Runs prep (+ Raman ODE) + quadrature on the powers already in h->P (device,
// concatenated).  With adjoint set, the fused forward + adjoint kernel of the
// closed-form profile also fills the step buckets and the PSD buckets (single
// profile, FP32).  keep_nodes keeps the Raman ODE's RK4 states (profile 0).
isrs_status run_forward(isrs_handle h, const isrs_fibre *fb, Geom *g, int precision, cudaStream_t st,
                        bool adjoint = false, bool keep_nodes = false, bool prep_only = false)
{
    isrs_status s;
    const int M = g->n_steps;
    if (precision == ISRS_PREC_FP32 && g->phase_rev_max > 2097152.0)
        return fail(h, ISRS_ERR_UNSUPPORTED, "phase range %.3g revolutions exceeds the FP32 reduction range",
                    g->phase_rev_max);
    if (precision == ISRS_PREC_FP32 && g->mci_phase_rev_max > 536870912.0)
        return fail(h, ISRS_ERR_UNSUPPORTED, "MCI phase range %.3g revolutions exceeds the FP32 reduction range",
                    g->mci_phase_rev_max);
    if (adjoint && g->n_mci_items > 0 && g->profile == ISRS_PROFILE_RAMAN_ODE)
        return fail(h, ISRS_ERR_UNSUPPORTED, "the Raman-ODE adjoint does not cover the separate MCI grid");
    if (g->n_mci_items > 0 && (s = ensure(h, h->partial_mci, sizeof(double) * g->n_mci_items)) != ISRS_OK)
        return s;
    if ((s = ensure(h, h->pd_d, sizeof(double) * g->total_prof_ch)) != ISRS_OK) return s;
    if ((s = ensure(h, h->pd_f, sizeof(float) * g->total_prof_ch)) != ISRS_OK) return s;
    if ((s = ensure(h, h->lnrho_L, sizeof(double) * g->total_prof_ch)) != ISRS_OK) return s;
    if ((s = ensure(h, h->step_d, sizeof(double2) * (size_t)g->n_prof * M)) != ISRS_OK) return s;
    if ((s = ensure(h, h->step_f, sizeof(float2) * (size_t)g->n_prof * M)) != ISRS_OK) return s;
    if ((s = ensure(h, h->ptot, sizeof(double) * g->n_prof)) != ISRS_OK) return s;
    if ((s = ensure(h, h->kapL, sizeof(double) * g->n_prof)) != ISRS_OK) return s;
    if ((s = ensure(h, h->partial, sizeof(double) * std::max(1, g->n_items))) != ISRS_OK) return s;
    if ((s = ensure(h, h->counter, sizeof(int) * 4)) != ISRS_OK) return s;

    {
        Range r_prep("isrs prep (ISRS profile tables)");
        PrepParams pp;
        pp.P = (const double *)h->P.p;
        pp.ch_frel = (const double *)g->ch_frel.p;
        pp.ch_B = (const double *)g->ch_B.p;
        pp.ch_alpha = (const double *)g->ch_alpha.p;
        pp.plan_ch_off = (const int *)g->plan_ch_off_d.p;
        pp.plan_n = (const int *)g->plan_n_d.p;
        pp.prof_ch_off = (const int *)g->prof_ch_off_d.p;
        pp.prof_plan = (const int *)g->prof_plan_d.p;
        pp.zs_d = (const double2 *)g->zs_d.p;
        pp.n_steps = M;
        pp.L = fb->L_km;
        pp.Cr = fb->Cr;
        pp.alpha_R = fb->alpha_R_per_km;
        pp.pd_d = (double *)h->pd_d.p;
        pp.pd_f = (float *)h->pd_f.p;
        pp.step_d = (double2 *)h->step_d.p;
        pp.step_f = (float2 *)h->step_f.p;
        pp.lnrho_L = (double *)h->lnrho_L.p;
        pp.ptot = (double *)h->ptot.p;
        pp.kap_L = (double *)h->kapL.p;
        CK(launch_prep(pp, g->n_prof, st));
        if (g->profile == ISRS_PROFILE_RAMAN_ODE) {
            // the Raman ODE overwrites ln rho(L) and fills the {a, b} tables
            if ((s = ensure(h, h->ab, sizeof(double2) * (size_t)g->total_prof_ch * M)) != ISRS_OK) return s;
            if (keep_nodes &&
                (s = ensure(h, h->ode_y, sizeof(double) * (size_t)(g->n_rk + 1) * g->plan_n[0])) != ISRS_OK)
                return s;
            CK(launch_raman(raman_params(h, fb, g, keep_nodes), g->n_prof, g->max_plan_n, st));
        }
    }
    if ((s = ensure(h, h->paths, sizeof(unsigned long long) * 4)) != ISRS_OK) return s;
    if (prep_only) {
        h->last_launches = g->profile == ISRS_PROFILE_RAMAN_ODE ? 2 : 1;
        return ISRS_OK;
    }
    Range r_quad(adjoint ? "isrs quadrature + adjoint" : "isrs quadrature");
    QuadParams qp = quad_params(h, fb, g);
    CK(cudaMemsetAsync(h->counter.p, 0, sizeof(int) * 4, st));
    CK(cudaMemsetAsync(h->paths.p, 0, sizeof(unsigned long long) * 4, st));
    const int block = h->tile_threads > 0 ? h->tile_threads : 256;
    if (adjoint) {
        const int n_ch = g->plan_n[0];
        if ((s = ensure(h, h->gA, sizeof(double2) * (size_t)std::max(1, g->n_items + g->n_mci_items) * M)) !=
            ISRS_OK)
            return s;
        // per-tile PSD buckets (regular tiles, then MCI tiles); every tile writes its whole row
        if ((s = ensure(h, h->gPd, sizeof(double) * (size_t)std::max(1, g->n_items + g->n_mci_items) * n_ch)) !=
            ISRS_OK)
            return s;
        AdjParams ap;
        ap.q = qp;
        ap.item_R = (double2 *)h->gA.p;
        ap.V = (double *)h->gPd.p;
        ap.item_slot = (const int *)g->item_slot.p;
        ap.n_ch = n_ch;
        const int per_sm = adjoint_blocks_per_sm(M, g->G, block);
        int grid = h->num_sms * per_sm;
        if (g->n_items < grid) grid = std::max(1, g->n_items);
        if ((s = ensure(h, h->gY, adjoint_scratch_bytes(grid))) != ISRS_OK) return s;
        ap.Yg = (double *)h->gY.p;
        if ((s = mark(h, 1, 0, st)) != ISRS_OK) return s;
        if (g->n_items > 0) CK(launch_adjoint(ap, grid, block, st));
        if (g->n_mci_items > 0) {
            // the MCI cells of the separate grid: further tiles of their CUTs
            AdjParams am = ap;
            am.q.items = (const DevItem *)g->mci_items.p;
            am.q.n_items = g->n_mci_items;
            am.q.G = g->G_mci;
            am.q.partial = (double *)h->partial_mci.p;
            am.q.counter = (int *)h->counter.p + 1;
            am.item_R = (double2 *)h->gA.p + (size_t)g->n_items * M;
            am.V = (double *)h->gPd.p + (size_t)g->n_items * n_ch;
            am.item_slot = (const int *)g->item_slot_all.p + g->n_items;
            int mgrid = h->num_sms * adjoint_mci_blocks_per_sm(M, am.q.mci_n_max, block);
            if (g->n_mci_items < mgrid) mgrid = g->n_mci_items;
            CK(launch_adjoint_mci(am, mgrid, block, st));
        }
        if ((s = mark(h, 1, 1, st)) != ISRS_OK) return s;
    } else {
        const bool tab = g->profile == ISRS_PROFILE_RAMAN_ODE;
        if (tab && quad_tab_smem_bytes(precision, M, g->G, g->nc_max) > 200 * 1024)
            return fail(h, ISRS_ERR_UNSUPPORTED, "profile tables exceed shared memory at this precision");
        const int per_sm = tab ? quad_tab_blocks_per_sm(precision, M, g->G, g->nc_max, block)
                               : quad_blocks_per_sm(precision, M, g->G, block);
        int grid = h->num_sms * per_sm;
        if (g->n_items < grid) grid = std::max(1, g->n_items);
        if ((s = mark(h, 0, 0, st)) != ISRS_OK) return s;
        if (g->n_items > 0) CK(tab ? launch_quad_tab(qp, precision, grid, block, st)
                                   : launch_quad(qp, precision, grid, block, st));
        if (g->n_mci_items > 0) {
            QuadParams qm = qp;
            qm.items = (const DevItem *)g->mci_items.p;
            qm.n_items = g->n_mci_items;
            qm.G = g->G_mci;
            qm.partial = (double *)h->partial_mci.p;
            qm.counter = (int *)h->counter.p + 1;
            if (tab) {
                // the MCI cells with the tabulated profile: FP32 rows of {a, b}, cells in chunks
                int cpc = 0;
                if (precision == ISRS_PREC_FP32) {
                    cpc = quad_mci_tab_cells(M, qm.mci_n_max, qm.G, block);
                    if (cpc < 1)
                        return fail(h, ISRS_ERR_UNSUPPORTED, "MCI step rows of %d steps exceed shared memory", M);
                    const size_t nab = (size_t)g->total_prof_ch * M;
                    if (nab > (size_t)INT32_MAX)
                        return fail(h, ISRS_ERR_UNSUPPORTED, "profile tables of %zu entries exceed the MCI conversion", nab);
                    if ((s = ensure(h, h->ab_f, sizeof(float2) * nab)) != ISRS_OK) return s;
                    qm.ab_f = (const float2 *)h->ab_f.p;
                    CK(launch_tab_half_log2((const double2 *)h->ab.p, (float2 *)h->ab_f.p, (int)nab, h->num_sms,
                                            st));
                }
                qm.mci_cpc = cpc;
                int mgrid = h->num_sms * quad_mci_tab_blocks_per_sm(precision, M, qm.mci_n_max, cpc, block);
                if (g->n_mci_items < mgrid) mgrid = g->n_mci_items;
                CK(launch_quad_mci_tab(qm, precision, mgrid, block, st));
            } else {
                int mgrid = h->num_sms * quad_mci_blocks_per_sm(precision, M, qm.mci_n_max, block);
                if (g->n_mci_items < mgrid) mgrid = g->n_mci_items;
                CK(launch_quad_mci(qm, precision, mgrid, block, st));
            }
        }
        if ((s = mark(h, 0, 1, st)) != ISRS_OK) return s;
    }
    h->last_points = g->n_points;
    h->last_psteps = g->n_points * (int64_t)M;
    h->last_launches = (g->profile == ISRS_PROFILE_RAMAN_ODE ? 3 : 2) +   // prep (+ Raman ODE) + quadrature
                       (g->n_mci_items > 0 ? 1 : 0) +                      // + MCI cells
                       (g->n_mci_items > 0 && g->profile == ISRS_PROFILE_RAMAN_ODE &&
                                precision == ISRS_PREC_FP32 ? 1 : 0);      // + their FP32 profile rows
    return ISRS_OK;
}

isrs_status run_finish(isrs_handle h, const isrs_fibre *fb, const isrs_quad *q, Geom *g, bool want_snr,
                       cudaStream_t st)
{
    Range r("isrs finish (eta, SNR, T)");
    isrs_status s;
    const size_t ns = (size_t)std::max(1, g->n_slots);
    if ((s = ensure(h, h->o_sigma, sizeof(double) * ns)) != ISRS_OK) return s;
    if ((s = ensure(h, h->o_pnli, sizeof(double) * ns)) != ISRS_OK) return s;
    if ((s = ensure(h, h->o_eta, sizeof(double) * ns)) != ISRS_OK) return s;
    if ((s = ensure(h, h->o_snr, sizeof(double) * ns)) != ISRS_OK) return s;
    if ((s = ensure(h, h->o_pase, sizeof(double) * ns)) != ISRS_OK) return s;
    if ((s = ensure(h, h->o_T, sizeof(double) * std::max(1, g->n_prof))) != ISRS_OK) return s;
    FinishParams fp;
    std::memset(&fp, 0, sizeof(fp));
    fp.partial = (const double *)h->partial.p;
    fp.slot_items = (const int2 *)g->slot_items.p;
    if (g->n_mci_items > 0) {
        fp.partial2 = (const double *)h->partial_mci.p;
        fp.slot_items2 = (const int2 *)g->slot_items2.p;
    }
    fp.slot_cut = (const int *)g->slot_cut.p;
    fp.prof_slot_off = (const int *)g->prof_slot_off.p;
    fp.prof_plan = (const int *)g->prof_plan_d.p;
    fp.plan_ch_off = (const int *)g->plan_ch_off_d.p;
    fp.prof_ch_off = (const int *)g->prof_ch_off_d.p;
    fp.ch_gamma = (const double *)g->ch_gamma.p;
    fp.ch_B = (const double *)g->ch_B.p;
    fp.ch_frel = (const double *)g->ch_frel.p;
    fp.ch_nf = g->has_nf ? (const double *)g->ch_nf.p : nullptr;
    fp.guard = g->has_guard ? (const unsigned char *)g->guard.p : nullptr;
    fp.P = (const double *)h->P.p;
    fp.lnrho_L = (const double *)h->lnrho_L.p;
    fp.f_ref = fb->f_ref_THz;
    fp.snr_trx_lin_inv = q->snr_trx_dB > 0.0 ? std::pow(10.0, -q->snr_trx_dB / 10.0) : 0.0;
    fp.n_spans = fb->n_spans > 1 ? fb->n_spans : 1;
    fp.sigma = (double *)h->o_sigma.p;
    fp.pnli = (double *)h->o_pnli.p;
    fp.eta = (double *)h->o_eta.p;
    if (want_snr) {
        fp.snr = (double *)h->o_snr.p;
        fp.pase = (double *)h->o_pase.p;
    }
    fp.T = (double *)h->o_T.p;
    CK(launch_finish(fp, g->n_prof, st));
    h->last_launches += 1;
    return ISRS_OK;
}

isrs_status copy_out(isrs_handle h, double *dst, const DevBuf &src, size_t n, cudaStream_t st, bool &host_out)
{
    if (!dst || n == 0) return ISRS_OK;
    const bool dev = is_device_ptr(dst);
    if (!dev) host_out = true;
    CK(cudaMemcpyAsync(dst, src.p, n * sizeof(double), dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    return ISRS_OK;
}

// Load launch powers (host or device) into h->P and validate them on the host.
isrs_status load_powers(isrs_handle h, const double *P, size_t n, cudaStream_t st)
{
    if (!P) return fail(h, ISRS_ERR_INVALID_ARG, "P_W is NULL");
    isrs_status s;
    if ((s = ensure(h, h->P, n * sizeof(double))) != ISRS_OK) return s;
    if (is_device_ptr(P)) {
        CK(cudaMemcpyAsync(h->P.p, P, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
        CK(cudaMemcpyAsync(h->P.p, P, n * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));   // pageable source: keep the copy complete before return
    }
    return ISRS_OK;
}

isrs_status check_powers_any(isrs_handle h, const double *P, size_t off, int n, cudaStream_t st)
{
    if (is_device_ptr(P)) {
        std::vector<double> tmp(n);
        CK(cudaMemcpyAsync(tmp.data(), P + off, n * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        return check_powers(h, tmp.data(), n);
    }
    return check_powers(h, P + off, n);
}

isrs_status set_device(isrs_handle h)
{
    CK(cudaSetDevice(h->device));
    return ISRS_OK;
}

// The batched launch as a replayable CUDA graph.  The first call for a launch
// signature runs directly (which also sizes every workspace buffer) and then
// captures the same sequence on a private stream; later calls replay it on
// the caller's stream.  The graph is re-captured whenever the fibre,
// precision, tile or any workspace pointer it baked in has changed.
std::vector<void *> workspace_ptrs(isrs_handle h)
{
    return {h->P.p, h->pd_d.p, h->pd_f.p, h->lnrho_L.p, h->step_d.p, h->step_f.p, h->ptot.p, h->partial.p,
            h->counter.p, h->paths.p, h->kapL.p, h->o_sigma.p, h->o_pnli.p, h->o_eta.p, h->o_snr.p, h->o_pase.p, h->o_T.p,
            h->ab.p, h->ab_f.p, h->partial_mci.p};
}

isrs_status run_batched_graph(isrs_handle h, const isrs_fibre *fb, const isrs_quad *q, Geom *g, cudaStream_t st)
{
    isrs_status s;
    Hasher hs;            // fields one by one: the struct has padding
    hs.val(fb->L_km); hs.val(fb->f_ref_THz); hs.val(fb->beta2); hs.val(fb->beta3); hs.val(fb->beta4);
    hs.val(fb->Cr); hs.val(fb->alpha_R_per_km); hs.val(fb->n_spans);
    hs.val(fb->profile); hs.val(fb->raman_max_THz); hs.val(fb->raman_photon);
    hs.val(q->precision);
    hs.val(h->tile_threads);
    const uint64_t key = hs.v;
    if (g->gexec && g->gkey == key && g->gptrs == workspace_ptrs(h)) {
        CK(cudaGraphLaunch(g->gexec, st));
        h->last_graph = true;
        h->last_points = g->n_points;
        h->last_psteps = g->n_points * (int64_t)g->n_steps;
        h->last_launches = 3;
        return ISRS_OK;
    }
    if ((s = run_forward(h, fb, g, q->precision, st)) != ISRS_OK) return s;
    if ((s = run_finish(h, fb, q, g, false, st)) != ISRS_OK) return s;
    h->last_graph = false;
    if (g->gexec) {
        cudaGraphExecDestroy(g->gexec);
        g->gexec = nullptr;
    }
    if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    const int saved = h->last_launches;
    const int64_t sp = h->last_points, ss = h->last_psteps;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        isrs_status s1 = run_forward(h, fb, g, q->precision, h->cap_stream);
        isrs_status s2 = s1 == ISRS_OK ? run_finish(h, fb, q, g, false, h->cap_stream) : s1;
        cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
        if (s2 == ISRS_OK && e == cudaSuccess && graph &&
            cudaGraphInstantiate(&g->gexec, graph, 0) == cudaSuccess) {
            g->gkey = key;
            g->gptrs = workspace_ptrs(h);
        } else {
            g->gexec = nullptr;          // capture not possible: keep running directly
        }
        if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();
    h->err.clear();
    h->last_launches = saved;
    h->last_points = sp;
    h->last_psteps = ss;
    return ISRS_OK;
}

ChainParams chain_params(isrs_handle h, const isrs_fibre *fb, const isrs_quad *q, Geom *g, int n)
{
    ChainParams cp;
    std::memset(&cp, 0, sizeof(cp));
    cp.P = (const double *)h->P.p;
    cp.ch_frel = (const double *)g->ch_frel.p;
    cp.ch_B = (const double *)g->ch_B.p;
    cp.ch_gamma = (const double *)g->ch_gamma.p;
    cp.ch_nf = g->has_nf ? (const double *)g->ch_nf.p : nullptr;
    cp.zs_d = (const double2 *)g->zs_d.p;
    cp.step_d = (const double2 *)h->step_d.p;
    cp.snr = (const double *)h->o_snr.p;
    cp.pnli = (const double *)h->o_pnli.p;
    cp.pase = (const double *)h->o_pase.p;
    cp.lnrho_L = (const double *)h->lnrho_L.p;
    // the MCI items of a separate grid follow the regular ones in the bucket rows
    cp.item_slot = (const int *)(g->n_mci_items > 0 ? g->item_slot_all.p : g->item_slot.p);
    cp.slot_cut = (const int *)g->slot_cut.p;
    cp.n_items = g->n_items + g->n_mci_items;
    cp.n_slots = g->n_slots;
    cp.n_ch = n;
    cp.n_steps = g->n_steps;
    cp.L = fb->L_km;
    cp.Cr = fb->Cr;
    cp.alpha_R = fb->alpha_R_per_km;
    cp.f_ref = fb->f_ref_THz;
    cp.snr_trx_lin_inv = q->snr_trx_dB > 0.0 ? std::pow(10.0, -q->snr_trx_dB / 10.0) : 0.0;
    cp.n_spans = fb->n_spans > 1 ? fb->n_spans : 1;
    cp.with_direct = 1;
    cp.ybar = (double *)h->ybar.p;
    cp.aase = (double *)h->ybar.p + n;
    cp.dT_dP = (double *)h->dTdP.p;
    return cp;
}

// Gradient with the Raman-ODE profile, first half: the profile tables with
// the RK4 states kept, then the fused forward + adjoint quadrature over the
// geometry's CUTs (Sigma into the partials, the unweighted buckets into the
// tile rows).
isrs_status run_grad_tab_fwd(isrs_handle h, const isrs_fibre *fb, Geom *g, cudaStream_t st)
{
    isrs_status s;
    const int n = g->plan_n[0], M = g->n_steps;
    // profile tables and the RK4 states; the fused quadrature below gives Sigma
    if ((s = run_forward(h, fb, g, ISRS_PREC_FP32, st, false, true, true)) != ISRS_OK) return s;
    if ((s = ensure(h, h->ybar, sizeof(double) * 2 * n)) != ISRS_OK) return s;
    if ((s = ensure(h, h->dTdP, sizeof(double) * n)) != ISRS_OK) return s;
    if ((s = ensure(h, h->gAB, sizeof(double2) * (size_t)n * M)) != ISRS_OK) return s;
    if ((s = ensure(h, h->gAt, sizeof(double) * (size_t)n * M)) != ISRS_OK) return s;
    if ((s = ensure(h, h->gV, sizeof(double) * n)) != ISRS_OK) return s;
    if ((s = ensure(h, h->tab_rows, sizeof(double2) * (size_t)std::max<int64_t>(1, g->n_tab_rows) * M)) != ISRS_OK)
        return s;
    if ((s = ensure(h, h->tab_rowsV, sizeof(double) * (size_t)std::max<int64_t>(1, g->n_tab_rows))) != ISRS_OK)
        return s;
    CK(cudaMemsetAsync(h->counter.p, 0, sizeof(int) * 4, st));
    AdjTabParams ap;
    ap.q = quad_params(h, fb, g);
    ap.row_off = (const int *)g->tab_row_off.p;
    ap.prow = (const int4 *)g->tab_prow.p;
    ap.rows = (double2 *)h->tab_rows.p;
    ap.rowsV = (double *)h->tab_rowsV.p;
    const int block = h->tile_threads > 0 ? h->tile_threads : 256;
    int grid = h->num_sms * adjoint_tab_blocks_per_sm(M, g->G, g->nc_max, block);
    if (g->n_items < grid) grid = std::max(1, g->n_items);
    {
        Range r_adj("isrs quadrature + adjoint (tabulated profile)");
        if ((s = mark(h, 1, 0, st)) != ISRS_OK) return s;
        if (g->n_items > 0) CK(launch_adjoint_tab(ap, grid, block, st));
        if ((s = mark(h, 1, 1, st)) != ISRS_OK) return s;
    }
    h->last_points = g->n_points;
    h->last_psteps = g->n_points * (int64_t)M;
    h->last_launches += 1;   // fused quadrature + adjoint (prep and Raman ODE counted)
    return ISRS_OK;
}

// Second half: dT/dSigma of every channel from cp.snr/pnli/pase (ybar), the
// gather of the tile rows of the geometry's CUTs, then the discrete adjoint
// of the profile tables and the RK4 steps.  with_direct adds the terms
// outside every eta (the ASE gain and the SNR numerator); the parts of
// disjoint CUT shards, one of them with_direct, sum to the full gradient,
// since the adjoint is linear in the bucket terms.
isrs_status run_grad_tab_bwd(isrs_handle h, const isrs_fibre *fb, Geom *g, const ChainParams &cp, bool with_direct,
                             cudaStream_t st)
{
    const int n = g->plan_n[0], M = g->n_steps;
    Range r_chain("isrs chain rule (tabulated profile, Raman ODE)");
    CK(launch_ybar(cp, st));
    TabGatherParams gp;
    gp.gath_off = (const int *)g->tab_gath_off.p;
    gp.gath = (const int2 *)g->tab_gath.p;
    gp.rows = (const double2 *)h->tab_rows.p;
    gp.rowsV = (const double *)h->tab_rowsV.p;
    gp.ybar = cp.ybar;
    gp.slot_cut = (const int *)g->slot_cut.p;
    gp.n_ch = n;
    gp.n_steps = M;
    gp.gAB = (double2 *)h->gAB.p;
    gp.gV = (double *)h->gV.p;
    CK(launch_tab_gather(gp, st));
    RamanAdjParams rap;
    std::memset(&rap, 0, sizeof(rap));
    rap.r = raman_params(h, fb, g, true);
    rap.n = n;
    rap.n_rk = g->n_rk;
    rap.y_nodes = (const double *)h->ode_y.p;
    rap.gAB = (const double2 *)h->gAB.p;
    rap.gAt = (double *)h->gAt.p;
    rap.aase = cp.aase;
    rap.gV = (const double *)h->gV.p;
    rap.snr = cp.snr;
    rap.pnli = cp.pnli;
    rap.pase = cp.pase;
    rap.ch_B = (const double *)g->ch_B.p;
    rap.with_direct = with_direct ? 1 : 0;
    rap.dT_dP = (double *)h->dTdP.p;
    CK(launch_raman_adj(rap, st));
    h->last_launches += 4;   // ybar, gather, slope fold, ODE adjoint
    return ISRS_OK;
}

// Gradient with the Raman-ODE profile: both halves around the finish (eta,
// SNR, T of every channel).
isrs_status run_grad_tab(isrs_handle h, const isrs_fibre *fb, const isrs_quad *q, Geom *g, cudaStream_t st)
{
    isrs_status s;
    if ((s = run_grad_tab_fwd(h, fb, g, st)) != ISRS_OK) return s;
    if ((s = run_finish(h, fb, q, g, true, st)) != ISRS_OK) return s;
    const ChainParams cp = chain_params(h, fb, q, g, g->plan_n[0]);
    return run_grad_tab_bwd(h, fb, g, cp, true, st);
}

// Argument checks shared by the gradient entry points; selects the device and
// rejects a capturing stream.  All powers must be > 0 and no channel a guard.
isrs_status grad_checks(isrs_handle h, const isrs_fibre *fibre, const isrs_channels *ch, const double *P_W,
                        const isrs_quad *quad, cudaStream_t st)
{
    isrs_status s;
    if ((s = check_fibre(h, fibre)) != ISRS_OK) return s;
    if ((s = check_plan(h, ch)) != ISRS_OK) return s;
    if ((s = check_quad(h, quad)) != ISRS_OK) return s;
    if (!P_W) return fail(h, ISRS_ERR_INVALID_ARG, "P_W is NULL");
    if (quad->precision != ISRS_PREC_FP32)
        return fail(h, ISRS_ERR_INVALID_ARG, "the gradient is the adjoint of the FP32 path");
    if (quad->n_edges - 1 > 128) return fail(h, ISRS_ERR_UNSUPPORTED, "gradient supports at most 128 z-steps");
    if (quad->G_mci > 0 && fibre->profile == ISRS_PROFILE_RAMAN_ODE)
        return fail(h, ISRS_ERR_UNSUPPORTED, "the Raman-ODE gradient does not cover the separate MCI grid");
    if (fibre->profile == ISRS_PROFILE_RAMAN_ODE && ch->n_ch > kMaxRamanGradCh)
        return fail(h, ISRS_ERR_UNSUPPORTED, "Raman-ODE gradient supports at most %d channels", kMaxRamanGradCh);
    if (ch->guard)
        for (int k = 0; k < ch->n_ch; ++k)
            if (ch->guard[k]) return fail(h, ISRS_ERR_INVALID_ARG, "gradient needs every channel lit (guard %d)", k);
    if ((s = set_device(h)) != ISRS_OK) return s;
    if ((s = reject_capture(h, st)) != ISRS_OK) return s;
    if ((s = check_ptr(h, P_W, "P_W")) != ISRS_OK) return s;
    std::vector<double> hp(ch->n_ch);
    if (is_device_ptr(P_W)) {
        CK(cudaMemcpyAsync(hp.data(), P_W, sizeof(double) * ch->n_ch, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    } else {
        std::memcpy(hp.data(), P_W, sizeof(double) * ch->n_ch);
    }
    if ((s = check_powers(h, hp.data(), ch->n_ch)) != ISRS_OK) return s;
    for (int k = 0; k < ch->n_ch; ++k)
        if (!(hp[k] > 0.0)) return fail(h, ISRS_ERR_INVALID_ARG, "gradient needs P[%d] > 0", k);
    return ISRS_OK;
}

// Chain-rule constants over the buckets of the last fused forward + adjoint.
isrs_status chain_buffers(isrs_handle h, const isrs_fibre *fb, const isrs_quad *q, Geom *g, int n,
                          ChainParams &cp)
{
    isrs_status s;
    if ((s = ensure(h, h->ybar, sizeof(double) * 2 * n)) != ISRS_OK) return s;
    if ((s = ensure(h, h->gK, sizeof(double2) * g->n_steps + sizeof(double) * (4 * (g->n_steps + 1) + 4))) !=
        ISRS_OK)
        return s;
    if ((s = ensure(h, h->dTdP, sizeof(double) * n)) != ISRS_OK) return s;
    if ((s = ensure(h, h->gVs, sizeof(double) * (size_t)std::max(1, g->n_slots) * n)) != ISRS_OK) return s;
    cp = chain_params(h, fb, q, g, n);
    cp.item_R = (const double2 *)h->gA.p;
    cp.Vt = (const double *)h->gPd.p;
    cp.Vs = (double *)h->gVs.p;
    cp.V = cp.Vs;
    cp.slot_items = (const int2 *)g->slot_items.p;
    cp.slot_items2 = g->n_mci_items > 0 ? (const int2 *)g->slot_items2.p : nullptr;
    cp.n_items_reg = g->n_items;
    cp.Rb = (double2 *)h->gK.p;
    cp.cs = (double *)((double2 *)h->gK.p + g->n_steps);
    return ISRS_OK;
}

isrs_status grad_outputs(isrs_handle h, int n, double *dT_dP, double *snr, double *eta, double *T_host,
                         cudaStream_t st)
{
    isrs_status s;
    bool host_out = false;
    if ((s = copy_out(h, dT_dP, h->dTdP, n, st, host_out)) != ISRS_OK) return s;
    if ((s = copy_out(h, snr, h->o_snr, n, st, host_out)) != ISRS_OK) return s;
    if ((s = copy_out(h, eta, h->o_eta, n, st, host_out)) != ISRS_OK) return s;
    if (T_host) {
        CK(cudaMemcpyAsync(T_host, h->o_T.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        host_out = true;
    }
    if (host_out) CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    return dbg_check(h, st);
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

const char *isrs_status_string(isrs_status s)
{
    switch (s) {
    case ISRS_OK: return "ok";
    case ISRS_ERR_INVALID_ARG: return "invalid argument";
    case ISRS_ERR_CUDA: return "CUDA error";
    case ISRS_ERR_ALLOC: return "allocation failed";
    case ISRS_ERR_TIMEOUT: return "timeout";
    case ISRS_ERR_NUMERIC: return "numeric error";
    case ISRS_ERR_UNSUPPORTED: return "unsupported";
    case ISRS_ERR_CHECK: return "debug bounds check failed";
    }
    return "unknown status";
}

isrs_status isrs_create(isrs_handle *out, int device)
{
    if (!out) return ISRS_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) {
        cudaGetLastError();
        return ISRS_ERR_CUDA;
    }
    if (device < 0 || device >= n) return ISRS_ERR_INVALID_ARG;
    isrs_handle h = new (std::nothrow) isrs_handle_s();
    if (!h) return ISRS_ERR_ALLOC;
    h->device = device;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete h;
        return ISRS_ERR_CUDA;
    }
    if (kDebugBuild) {
        if (cudaMalloc(&h->dbg.p, sizeof(unsigned)) != cudaSuccess ||
            cudaMemset(h->dbg.p, 0, sizeof(unsigned)) != cudaSuccess) {
            cudaGetLastError();
            if (h->dbg.p) cudaFree(h->dbg.p);
            delete h;
            return ISRS_ERR_ALLOC;
        }
        h->dbg.cap = sizeof(unsigned);
    }
    *out = h;
    return ISRS_OK;
}

isrs_status isrs_destroy(isrs_handle h)
{
    if (!h) return ISRS_OK;
    cudaSetDevice(h->device);
    for (auto &g : h->cache) free_geom(g.get());
    DevBuf *bufs[] = {&h->P, &h->pd_d, &h->pd_f, &h->step_d, &h->step_f, &h->lnrho_L, &h->ptot, &h->partial,
                      &h->counter, &h->o_sigma, &h->o_pnli, &h->o_eta, &h->o_snr, &h->o_pase, &h->o_T,
                      &h->gA, &h->gK, &h->gPd, &h->ybar, &h->dTdP, &h->ab, &h->ode_y, &h->gAB, &h->gV,
                      &h->gAt, &h->partial_mci, &h->eta_all, &h->tab_rows, &h->tab_rowsV, &h->gVs,
                      &h->gY, &h->dbg, &h->ab_f};
    for (DevBuf *b : bufs) release(*b);
    release(h->paths);
    release(h->kapL);
    for (int w = 0; w < 2; ++w)
        for (int k = 0; k < 2; ++k)
            if (h->ev[w][k]) cudaEventDestroy(h->ev[w][k]);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    delete h;
    return ISRS_OK;
}

const char *isrs_last_error(isrs_handle h) { return h ? h->err.c_str() : ""; }

int isrs_debug_build(void) { return kDebugBuild ? 1 : 0; }

isrs_status isrs_beta_from_dispersion(double lambda_nm, double D, double S, double Sdot, double *beta)
{
    if (!beta || !(lambda_nm > 0.0)) return ISRS_ERR_INVALID_ARG;
    const double w = 2.0 * 3.14159265358979323846 * kCnmPerPs;     // 2 pi c [nm/ps]
    const double l = lambda_nm;
    beta[0] = -D * l * l / w;                                        // Eq. d
    beta[1] = l * l * l / (w * w) * (2.0 * D + S * l);               // Eq. d_slope
    beta[2] = -l * l * l * l / (w * w * w) * (6.0 * D + 6.0 * S * l + Sdot * l * l);   // Eq. d_curve
    return ISRS_OK;
}

double isrs_gamma_from_aeff(double lambda_nm, double n2, double aeff_um2)
{
    if (!(lambda_nm > 0.0) || !(n2 > 0.0) || !(aeff_um2 > 0.0)) return NAN;
    return 2.0 * 3.14159265358979323846 * n2 / ((lambda_nm * 1e-9) * (aeff_um2 * 1e-12)) * 1e3;   // Eq. gamma
}

isrs_status isrs_set_tile(isrs_handle h, int points_per_item, int threads_per_block)
{
    if (!h) return ISRS_ERR_INVALID_ARG;
    if (points_per_item < 0 || threads_per_block < 0 ||
        (threads_per_block != 0 && (threads_per_block % 32 != 0 || threads_per_block > 256)))
        return fail(h, ISRS_ERR_INVALID_ARG, "bad tile (%d, %d)", points_per_item, threads_per_block);
    h->tile_points = points_per_item;
    h->tile_threads = threads_per_block;
    return ISRS_OK;
}

isrs_status isrs_debug_inject_fault(isrs_handle h, int kind, int after)
{
    if (!h || kind < 0 || kind > 2 || (kind != 0 && after < 1)) return ISRS_ERR_INVALID_ARG;
    h->inj_kind = kind;
    h->inj_countdown = kind ? after : 0;
    return ISRS_OK;
}

isrs_status isrs_last_launch_info(isrs_handle h, int64_t *n_points, int64_t *n_point_steps, int *n_launches)
{
    if (!h) return ISRS_ERR_INVALID_ARG;
    if (n_points) *n_points = h->last_points;
    if (n_point_steps) *n_point_steps = h->last_psteps;
    if (n_launches) *n_launches = h->last_launches;
    return ISRS_OK;
}

isrs_status isrs_last_graph_replay(isrs_handle h, int *replayed)
{
    if (!h || !replayed) return ISRS_ERR_INVALID_ARG;
    *replayed = h->last_graph ? 1 : 0;
    return ISRS_OK;
}

isrs_status isrs_last_kernel_ms(isrs_handle h, int which, float *ms)
{
    if (!h || !ms || which < 0 || which > 1) return ISRS_ERR_INVALID_ARG;
    if (!h->ev_valid[which]) return fail(h, ISRS_ERR_INVALID_ARG, "no launch recorded");
    CK(cudaSetDevice(h->device));
    CK(cudaEventSynchronize(h->ev[which][1]));
    CK(cudaEventElapsedTime(ms, h->ev[which][0], h->ev[which][1]));
    return ISRS_OK;
}

isrs_status isrs_last_path_counts(isrs_handle h, int64_t *counts)
{
    if (!h || !counts) return ISRS_ERR_INVALID_ARG;
    if (!h->paths.p) return fail(h, ISRS_ERR_INVALID_ARG, "no launch recorded");
    unsigned long long c[4] = {0, 0, 0, 0};
    CK(cudaSetDevice(h->device));
    CK(cudaMemcpy(c, h->paths.p, sizeof(c), cudaMemcpyDeviceToHost));
    for (int k = 0; k < 3; ++k) counts[k] = (int64_t)c[k];
    return ISRS_OK;
}

isrs_status isrs_gn_eta(isrs_handle h, const isrs_fibre *fibre, const isrs_channels *ch, const double *P_W,
                        const isrs_quad *quad, const int *cuts, int n_cuts, double *eta, double *pnli,
                        double *sigma, void *stream)
{
    Range r_call("isrs_gn_eta");
    if (!h) return ISRS_ERR_INVALID_ARG;
    h->err.clear();
    h->shard_valid = false;    // the workspace is about to be overwritten
    isrs_status s;
    if ((s = check_fibre(h, fibre)) != ISRS_OK) return s;
    if ((s = check_plan(h, ch)) != ISRS_OK) return s;
    if ((s = check_quad(h, quad)) != ISRS_OK) return s;
    if (!P_W) return fail(h, ISRS_ERR_INVALID_ARG, "P_W is NULL");
    std::vector<int> cl;
    if (cuts) {
        if (n_cuts < 1) return fail(h, ISRS_ERR_INVALID_ARG, "n_cuts must be >= 1");
        std::vector<char> seen(ch->n_ch, 0);
        for (int k = 0; k < n_cuts; ++k) {
            if (cuts[k] < 0 || cuts[k] >= ch->n_ch) return fail(h, ISRS_ERR_INVALID_ARG, "cut %d out of range", cuts[k]);
            if (seen[cuts[k]]) return fail(h, ISRS_ERR_INVALID_ARG, "cut %d repeated", cuts[k]);
            seen[cuts[k]] = 1;
            cl.push_back(cuts[k]);
        }
    }
    if ((s = set_device(h)) != ISRS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = reject_capture(h, st)) != ISRS_OK) return s;
    if ((s = check_ptr(h, P_W, "P_W")) != ISRS_OK || (s = check_ptr(h, eta, "eta")) != ISRS_OK ||
        (s = check_ptr(h, pnli, "pnli")) != ISRS_OK || (s = check_ptr(h, sigma, "sigma")) != ISRS_OK)
        return s;
    if ((s = check_powers_any(h, P_W, 0, ch->n_ch, st)) != ISRS_OK) return s;
    Geom *g = nullptr;
    std::vector<std::vector<int>> cpp{cl};
    std::vector<int> pp{0};
    if ((s = get_geom(h, fibre, 1, ch, cpp, pp, quad, st, &g)) != ISRS_OK) return s;
    if ((s = load_powers(h, P_W, ch->n_ch, st)) != ISRS_OK) return s;
    if ((s = run_forward(h, fibre, g, quad->precision, st)) != ISRS_OK) return s;
    if ((s = run_finish(h, fibre, quad, g, false, st)) != ISRS_OK) return s;
    bool host_out = false;
    const size_t n = g->n_slots;
    if ((s = copy_out(h, eta, h->o_eta, n, st, host_out)) != ISRS_OK) return s;
    if ((s = copy_out(h, pnli, h->o_pnli, n, st, host_out)) != ISRS_OK) return s;
    if ((s = copy_out(h, sigma, h->o_sigma, n, st, host_out)) != ISRS_OK) return s;
    if (host_out) CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    return dbg_check(h, st);
}

isrs_status isrs_gn_snr(isrs_handle h, const isrs_fibre *fibre, const isrs_channels *ch, const double *P_W,
                        const isrs_quad *quad, double *snr, double *eta, double *T_host, void *stream)
{
    Range r_call("isrs_gn_snr");
    if (!h) return ISRS_ERR_INVALID_ARG;
    h->err.clear();
    h->shard_valid = false;    // the workspace is about to be overwritten
    isrs_status s;
    if ((s = check_fibre(h, fibre)) != ISRS_OK) return s;
    if ((s = check_plan(h, ch)) != ISRS_OK) return s;
    if ((s = check_quad(h, quad)) != ISRS_OK) return s;
    if (!P_W || !snr) return fail(h, ISRS_ERR_INVALID_ARG, "P_W or snr is NULL");
    if ((s = set_device(h)) != ISRS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = reject_capture(h, st)) != ISRS_OK) return s;
    if ((s = check_ptr(h, P_W, "P_W")) != ISRS_OK || (s = check_ptr(h, snr, "snr")) != ISRS_OK ||
        (s = check_ptr(h, eta, "eta")) != ISRS_OK)
        return s;
    if ((s = check_powers_any(h, P_W, 0, ch->n_ch, st)) != ISRS_OK) return s;
    Geom *g = nullptr;
    std::vector<std::vector<int>> cpp{std::vector<int>()};
    std::vector<int> pp{0};
    if ((s = get_geom(h, fibre, 1, ch, cpp, pp, quad, st, &g)) != ISRS_OK) return s;
    if ((s = load_powers(h, P_W, ch->n_ch, st)) != ISRS_OK) return s;
    if ((s = run_forward(h, fibre, g, quad->precision, st)) != ISRS_OK) return s;
    if ((s = run_finish(h, fibre, quad, g, true, st)) != ISRS_OK) return s;
    bool host_out = false;
    const size_t n = g->n_slots;
    if ((s = copy_out(h, snr, h->o_snr, n, st, host_out)) != ISRS_OK) return s;
    if ((s = copy_out(h, eta, h->o_eta, n, st, host_out)) != ISRS_OK) return s;
    if (T_host) {
        CK(cudaMemcpyAsync(T_host, h->o_T.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        host_out = true;
    }
    if (host_out) CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    return dbg_check(h, st);
}

isrs_status isrs_gn_eta_batched(isrs_handle h, const isrs_fibre *fibre, int n_plans, const isrs_channels *plans,
                                int n_prof, const int *plan_of_profile, const double *P_W,
                                const isrs_quad *quad, double *eta, void *stream)
{
    Range r_call("isrs_gn_eta_batched");
    if (!h) return ISRS_ERR_INVALID_ARG;
    h->err.clear();
    h->shard_valid = false;    // the workspace is about to be overwritten
    isrs_status s;
    if ((s = check_fibre(h, fibre)) != ISRS_OK) return s;
    if ((s = check_quad(h, quad)) != ISRS_OK) return s;
    if (n_plans < 1 || !plans) return fail(h, ISRS_ERR_INVALID_ARG, "no plans");
    if (n_prof < 1 || !plan_of_profile || !P_W || !eta) return fail(h, ISRS_ERR_INVALID_ARG, "bad profiles");
    for (int k = 0; k < n_plans; ++k)
        if ((s = check_plan(h, &plans[k])) != ISRS_OK) return s;
    size_t total = 0;
    std::vector<int> pp(n_prof);
    for (int p = 0; p < n_prof; ++p) {
        if (plan_of_profile[p] < 0 || plan_of_profile[p] >= n_plans)
            return fail(h, ISRS_ERR_INVALID_ARG, "profile %d: bad plan index", p);
        pp[p] = plan_of_profile[p];
        total += plans[pp[p]].n_ch;
    }
    if ((s = set_device(h)) != ISRS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = reject_capture(h, st)) != ISRS_OK) return s;
    if ((s = check_ptr(h, P_W, "P_W")) != ISRS_OK || (s = check_ptr(h, eta, "eta")) != ISRS_OK) return s;
    size_t off = 0;
    for (int p = 0; p < n_prof; ++p) {
        if ((s = check_powers_any(h, P_W, off, plans[pp[p]].n_ch, st)) != ISRS_OK) return s;
        off += plans[pp[p]].n_ch;
    }
    Geom *g = nullptr;
    std::vector<std::vector<int>> cpp(n_plans);
    if ((s = get_geom(h, fibre, n_plans, plans, cpp, pp, quad, st, &g)) != ISRS_OK) return s;
    if ((s = load_powers(h, P_W, total, st)) != ISRS_OK) return s;
    if ((s = run_batched_graph(h, fibre, quad, g, st)) != ISRS_OK) return s;
    bool host_out = false;
    if ((s = copy_out(h, eta, h->o_eta, total, st, host_out)) != ISRS_OK) return s;
    if (host_out) CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    return dbg_check(h, st);
}

isrs_status isrs_gn_grad(isrs_handle h, const isrs_fibre *fibre, const isrs_channels *ch, const double *P_W,
                         const isrs_quad *quad, double *dT_dP, double *snr, double *eta, double *T_host,
                         void *stream)
{
    Range r_call("isrs_gn_grad");
    if (!h) return ISRS_ERR_INVALID_ARG;
    h->err.clear();
    isrs_status s;
    if (!dT_dP) return fail(h, ISRS_ERR_INVALID_ARG, "dT_dP is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = grad_checks(h, fibre, ch, P_W, quad, st)) != ISRS_OK) return s;
    if ((s = check_ptr(h, dT_dP, "dT_dP")) != ISRS_OK || (s = check_ptr(h, snr, "snr")) != ISRS_OK ||
        (s = check_ptr(h, eta, "eta")) != ISRS_OK)
        return s;
    Geom *g = nullptr;
    std::vector<std::vector<int>> cpp{std::vector<int>()};
    std::vector<int> pp{0};
    if ((s = get_geom(h, fibre, 1, ch, cpp, pp, quad, st, &g)) != ISRS_OK) return s;
    if ((s = load_powers(h, P_W, ch->n_ch, st)) != ISRS_OK) return s;
    h->shard_valid = false;
    const int n = ch->n_ch;
    if (fibre->profile == ISRS_PROFILE_RAMAN_ODE) {
        if ((s = run_grad_tab(h, fibre, quad, g, st)) != ISRS_OK) return s;
        return grad_outputs(h, n, dT_dP, snr, eta, T_host, st);
    }
    if ((s = run_forward(h, fibre, g, ISRS_PREC_FP32, st, true)) != ISRS_OK) return s;
    if ((s = run_finish(h, fibre, quad, g, true, st)) != ISRS_OK) return s;
    ChainParams cp;
    if ((s = chain_buffers(h, fibre, quad, g, n, cp)) != ISRS_OK) return s;
    {
        Range r_chain("isrs chain rule (dT/dP)");
        CK(launch_chain(cp, st));
    }
    h->last_launches += 6;   // ybar, PSD-bucket reduction, step-bucket reduction, chain rule (3)
    return grad_outputs(h, n, dT_dP, snr, eta, T_host, st);
}

isrs_status isrs_gn_grad_shard_fwd(isrs_handle h, const isrs_fibre *fibre, const isrs_channels *ch,
                                   const double *P_W, const isrs_quad *quad, const int *cuts, int n_cuts,
                                   double *eta, void *stream)
{
    Range r_call("isrs_gn_grad_shard_fwd");
    if (!h) return ISRS_ERR_INVALID_ARG;
    h->err.clear();
    h->shard_valid = false;
    isrs_status s;
    if (!eta || !cuts || n_cuts < 1) return fail(h, ISRS_ERR_INVALID_ARG, "eta, cuts or n_cuts missing");
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = grad_checks(h, fibre, ch, P_W, quad, st)) != ISRS_OK) return s;
    if ((s = check_ptr(h, eta, "eta")) != ISRS_OK) return s;
    std::vector<int> cl;
    {
        std::vector<char> seen(ch->n_ch, 0);
        for (int k = 0; k < n_cuts; ++k) {
            if (cuts[k] < 0 || cuts[k] >= ch->n_ch) return fail(h, ISRS_ERR_INVALID_ARG, "cut %d out of range", cuts[k]);
            if (seen[cuts[k]]) return fail(h, ISRS_ERR_INVALID_ARG, "cut %d repeated", cuts[k]);
            seen[cuts[k]] = 1;
            cl.push_back(cuts[k]);
        }
    }
    Geom *g = nullptr;
    std::vector<std::vector<int>> cpp{cl};
    std::vector<int> pp{0};
    if ((s = get_geom(h, fibre, 1, ch, cpp, pp, quad, st, &g)) != ISRS_OK) return s;
    if ((s = load_powers(h, P_W, ch->n_ch, st)) != ISRS_OK) return s;
    if (fibre->profile == ISRS_PROFILE_RAMAN_ODE) {
        if ((s = run_grad_tab_fwd(h, fibre, g, st)) != ISRS_OK) return s;
    } else if ((s = run_forward(h, fibre, g, ISRS_PREC_FP32, st, true)) != ISRS_OK) {
        return s;
    }
    if ((s = run_finish(h, fibre, quad, g, false, st)) != ISRS_OK) return s;
    bool host_out = false;
    if ((s = copy_out(h, eta, h->o_eta, g->n_slots, st, host_out)) != ISRS_OK) return s;
    if (host_out) CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    if ((s = dbg_check(h, st)) != ISRS_OK) return s;
    h->shard_key = g->key;
    h->shard_fibre = *fibre;
    h->shard_quad = *quad;
    h->shard_n = ch->n_ch;
    h->shard_valid = true;
    return ISRS_OK;
}

isrs_status isrs_gn_grad_shard_bwd(isrs_handle h, const double *eta_all, int with_direct, double *dT_dP,
                                   double *snr, double *T_host, void *stream)
{
    Range r_call("isrs_gn_grad_shard_bwd");
    if (!h) return ISRS_ERR_INVALID_ARG;
    h->err.clear();
    isrs_status s;
    if (!h->shard_valid)
        return fail(h, ISRS_ERR_INVALID_ARG, "no shard forward to continue (isrs_gn_grad_shard_fwd first)");
    if (!eta_all || !dT_dP) return fail(h, ISRS_ERR_INVALID_ARG, "eta_all or dT_dP is NULL");
    Geom *g = nullptr;
    for (auto &c : h->cache)
        if (c->key == h->shard_key) g = c.get();
    if (!g) return fail(h, ISRS_ERR_INVALID_ARG, "the shard's tables were evicted by later calls");
    if ((s = set_device(h)) != ISRS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = reject_capture(h, st)) != ISRS_OK) return s;
    if ((s = check_ptr(h, eta_all, "eta_all")) != ISRS_OK || (s = check_ptr(h, dT_dP, "dT_dP")) != ISRS_OK ||
        (s = check_ptr(h, snr, "snr")) != ISRS_OK)
        return s;
    const int n = h->shard_n;
    {
        std::vector<double> he(n);
        if (is_device_ptr(eta_all)) {
            CK(cudaMemcpyAsync(he.data(), eta_all, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
        } else {
            std::memcpy(he.data(), eta_all, sizeof(double) * n);
        }
        for (int k = 0; k < n; ++k)
            if (!(std::isfinite(he[k]) && he[k] >= 0.0))
                return fail(h, ISRS_ERR_INVALID_ARG, "eta_all[%d] = %g is not a finite eta >= 0", k, he[k]);
    }
    if ((s = ensure(h, h->eta_all, sizeof(double) * 4 * n)) != ISRS_OK) return s;
    double *e_all = (double *)h->eta_all.p;
    CK(cudaMemcpyAsync(e_all, eta_all, sizeof(double) * n,
                       is_device_ptr(eta_all) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    if ((s = ensure(h, h->o_T, sizeof(double))) != ISRS_OK) return s;
    SnrFromEtaParams sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.eta = e_all;
    sp.P = (const double *)h->P.p;
    sp.ch_B = (const double *)g->ch_B.p;
    sp.ch_frel = (const double *)g->ch_frel.p;
    sp.ch_nf = g->has_nf ? (const double *)g->ch_nf.p : nullptr;
    sp.lnrho_L = (const double *)h->lnrho_L.p;
    sp.f_ref = h->shard_fibre.f_ref_THz;
    sp.snr_trx_lin_inv = h->shard_quad.snr_trx_dB > 0.0 ? std::pow(10.0, -h->shard_quad.snr_trx_dB / 10.0) : 0.0;
    sp.n_spans = h->shard_fibre.n_spans > 1 ? h->shard_fibre.n_spans : 1;
    sp.n = n;
    sp.snr = e_all + n;
    sp.pnli = e_all + 2 * n;
    sp.pase = e_all + 3 * n;
    sp.T = (double *)h->o_T.p;
    CK(launch_snr_from_eta(sp, st));
    ChainParams cp;
    if ((s = chain_buffers(h, &h->shard_fibre, &h->shard_quad, g, n, cp)) != ISRS_OK) return s;
    cp.snr = sp.snr;
    cp.pnli = sp.pnli;
    cp.pase = sp.pase;
    cp.with_direct = with_direct ? 1 : 0;
    if (h->shard_fibre.profile == ISRS_PROFILE_RAMAN_ODE) {
        // the tile rows and the RK4 states of the shard's forward
        h->last_launches = 1;   // SNR from eta
        if ((s = run_grad_tab_bwd(h, &h->shard_fibre, g, cp, with_direct != 0, st)) != ISRS_OK) return s;
    } else {
        Range r_chain("isrs chain rule (dT/dP)");
        CK(launch_chain(cp, st));
        h->last_launches = 7;    // SNR from eta, ybar, PSD-bucket reduction, step-bucket reduction, chain rule (3)
    }
    bool host_out = false;
    if ((s = copy_out(h, dT_dP, h->dTdP, n, st, host_out)) != ISRS_OK) return s;
    if (snr) {
        const bool dev = is_device_ptr(snr);
        if (!dev) host_out = true;
        CK(cudaMemcpyAsync(snr, sp.snr, sizeof(double) * n, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    }
    if (T_host) {
        CK(cudaMemcpyAsync(T_host, h->o_T.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        host_out = true;
    }
    if (host_out) CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    return dbg_check(h, st);
}

}  // extern "C"

// ============================================================================
// Allocation-free forward entry point (isrs_gn_eta_noalloc).
//
// For callers that cannot allocate device memory themselves: code running
// inside a host framework that owns the device allocator, or a real-time loop
// in which a cudaMalloc would block or break the memory budget.  All scratch
// lives in one file-scope device array of fixed size that every GPU loading
// this library holds until the process exits.
// ============================================================================
#include <mutex>

namespace {

constexpr size_t kNoAllocBytes = (size_t)4 << 20;     // 4 MiB of scratch per device
constexpr int kNoAllocMaxDevices = 64;

}  // namespace

static __device__ __align__(256) unsigned char g_isrs_noalloc_scratch[kNoAllocBytes];

namespace {

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
isrs_status noalloc_scratch(int dev, void **out)
{
    if (dev < 0 || dev >= kNoAllocMaxDevices) return ISRS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_isrs_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return ISRS_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return ISRS_OK;
}

// Bump layout of the tables inside the scratch array (256-byte aligned slots).
struct NoAllocLayout {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        const size_t at = off;
        off += (bytes + 255) & ~(size_t)255;
        return at;
    }
};

}  // namespace

extern "C" isrs_status isrs_gn_eta_noalloc(const isrs_fibre *fibre, const isrs_channels *ch, const double *P_W,
                                           const isrs_quad *quad, double *eta, double *pnli, void *stream)
{
    isrs_status s;
    if ((s = check_fibre(nullptr, fibre)) != ISRS_OK) return s;
    if ((s = check_plan(nullptr, ch)) != ISRS_OK) return s;
    if ((s = check_quad(nullptr, quad)) != ISRS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    {
        // a capturing stream would be invalidated by the synchronisations below
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
            cudaGetLastError();
            return ISRS_ERR_CUDA;
        }
        if (cs != cudaStreamCaptureStatusNone) return ISRS_ERR_UNSUPPORTED;
    }
    // inputs and outputs: device memory of the current device (or managed)
    if (!P_W || !eta || !is_device_ptr(P_W) || !is_device_ptr(eta) || (pnli && !is_device_ptr(pnli)))
        return ISRS_ERR_INVALID_ARG;
    if (fibre->n_spans > 1) return ISRS_ERR_UNSUPPORTED;         // single span only
    if (fibre->profile != ISRS_PROFILE_CLOSED_FORM) return ISRS_ERR_UNSUPPORTED;   // closed-form profile only
    if (quad->G_mci > 0) return ISRS_ERR_UNSUPPORTED;                             // one grid for every cell
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ISRS_ERR_CUDA;
    const int n = ch->n_ch;

    // launch powers: validated on the host
    std::vector<double> hp(n);
    if (cudaMemcpyAsync(hp.data(), P_W, sizeof(double) * n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return ISRS_ERR_CUDA;
    if ((s = check_powers(nullptr, hp.data(), n)) != ISRS_OK) return s;

    // host tables: pieces of every CUT, work tiles, output slots, z-grid
    std::vector<DevPiece> pieces;
    std::vector<DevItem> items;
    std::vector<int2> slot_items;
    std::vector<int> slot_cut, item_slot;
    const int64_t G2 = (int64_t)quad->G * quad->G;
    const int chunk = (int)std::max<int64_t>(1, (int64_t)(1 << 20) / G2);
    for (int i = 0; i < n; ++i) {
        const int p0 = (int)pieces.size();
        if ((s = cut_pieces(nullptr, ch, 0, i, quad->cell_set, pieces)) != ISRS_OK) return s;
        const int p1 = (int)pieces.size();
        const int it0 = (int)items.size();
        for (int a = p0; a < p1; a += chunk) {
            items.push_back(DevItem{0, a, std::min(a + chunk, p1), i});
            item_slot.push_back(i);
        }
        slot_items.push_back(make_int2(it0, (int)items.size()));
        slot_cut.push_back(i);
    }
    std::vector<double> frel(n), Bv(n), av(n), gv(n);
    for (int k = 0; k < n; ++k) {
        frel[k] = ch->f_THz[k] - fibre->f_ref_THz;
        Bv[k] = ch->B_THz[k];
        av[k] = ch->alpha_per_km[k];
        gv[k] = ch->gamma_per_W_km[k];
    }
    std::vector<float4> za, zb, zg, zgs;
    std::vector<int4> segv;
    std::vector<double2> zd;
    float dz_max = 0.f, phi_seg[3] = {0.f, 0.f, 0.f};
    zgrid_tables(fibre->L_km, fibre->alpha_R_per_km, quad->n_edges, za, zb, zd, dz_max, &zg, &zgs, &segv, phi_seg);
    const int M = quad->n_edges - 1;
    if (quad->precision == ISRS_PREC_FP32) {
        const double pi = 3.14159265358979323846;
        for (const DevPiece &pc : pieces) {
            const double fi = std::fabs(frel[pc.cut]);
            const double v1 = pc.xhi * pc.yhi, s12 = pc.xhi + pc.yhi;
            const double br = std::fabs(fibre->beta2) + pi * std::fabs(fibre->beta3) * (s12 + 2.0 * fi) +
                              2.0 * pi * pi / 3.0 * std::fabs(fibre->beta4) *
                                  (s12 * s12 + 1.5 * v1 + 3.0 * fi * s12 + 3.0 * fi * fi);
            if (4.0 * pi * pi * v1 * br * fibre->L_km / (2.0 * pi) > 2097152.0) return ISRS_ERR_UNSUPPORTED;
        }
    }
    const std::vector<int> zero1{0}, plan_n{n}, slot_off{0, n};

    // layout in the scratch array; anything beyond its size is rejected
    NoAllocLayout L;
    const size_t o_pieces = L.take(sizeof(DevPiece) * pieces.size());
    const size_t o_items = L.take(sizeof(DevItem) * items.size());
    const size_t o_slot_items = L.take(sizeof(int2) * n);
    const size_t o_slot_cut = L.take(sizeof(int) * n);
    const size_t o_slot_off = L.take(sizeof(int) * 2);
    const size_t o_zero = L.take(sizeof(int));
    const size_t o_plan_n = L.take(sizeof(int));
    const size_t o_frel = L.take(sizeof(double) * n), o_B = L.take(sizeof(double) * n);
    const size_t o_alpha = L.take(sizeof(double) * n), o_gamma = L.take(sizeof(double) * n);
    const size_t o_za = L.take(sizeof(float4) * M), o_zb = L.take(sizeof(float4) * M);
    const size_t o_zd = L.take(sizeof(double2) * M);
    const size_t o_zg = L.take(sizeof(float4) * zg.size());   // centred step moments (contracted small phase)
    const size_t o_zgs = L.take(sizeof(float4) * zgs.size());  // the same about segment centres
    const size_t o_seg = L.take(sizeof(int4) * segv.size());
    const size_t o_kapL = L.take(sizeof(double));
    const size_t o_P = L.take(sizeof(double) * n);
    const size_t o_pdd = L.take(sizeof(double) * n), o_pdf = L.take(sizeof(float) * n);
    const size_t o_lnL = L.take(sizeof(double) * n), o_ptot = L.take(sizeof(double));
    const size_t o_stepd = L.take(sizeof(double2) * M), o_stepf = L.take(sizeof(float2) * M);
    const size_t o_partial = L.take(sizeof(double) * std::max<size_t>(1, items.size()));
    const size_t o_counter = L.take(sizeof(int) * 4), o_T = L.take(sizeof(double));
    const size_t o_paths = L.take(sizeof(unsigned long long) * 4);
    if (L.off > kNoAllocBytes) return ISRS_ERR_UNSUPPORTED;

    unsigned char *base = nullptr;
    if ((s = noalloc_scratch(dev, (void **)&base)) != ISRS_OK) return s;
    struct Up { size_t off; const void *src; size_t bytes; } ups[] = {
        {o_pieces, pieces.data(), sizeof(DevPiece) * pieces.size()},
        {o_items, items.data(), sizeof(DevItem) * items.size()},
        {o_slot_items, slot_items.data(), sizeof(int2) * n}, {o_slot_cut, slot_cut.data(), sizeof(int) * n},
        {o_slot_off, slot_off.data(), sizeof(int) * 2}, {o_zero, zero1.data(), sizeof(int)},
        {o_plan_n, plan_n.data(), sizeof(int)}, {o_frel, frel.data(), sizeof(double) * n},
        {o_B, Bv.data(), sizeof(double) * n}, {o_alpha, av.data(), sizeof(double) * n},
        {o_gamma, gv.data(), sizeof(double) * n}, {o_za, za.data(), sizeof(float4) * M},
        {o_zb, zb.data(), sizeof(float4) * M}, {o_zd, zd.data(), sizeof(double2) * M},
        {o_zg, zg.data(), sizeof(float4) * zg.size()}, {o_zgs, zgs.data(), sizeof(float4) * zgs.size()},
        {o_seg, segv.data(), sizeof(int4) * segv.size()}};
    for (const Up &u : ups)
        if (u.bytes && cudaMemcpyAsync(base + u.off, u.src, u.bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return ISRS_ERR_CUDA;
    if (cudaMemcpyAsync(base + o_P, P_W, sizeof(double) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(base + o_counter, 0, sizeof(int) * 4, st) != cudaSuccess ||
        cudaMemsetAsync(base + o_paths, 0, sizeof(unsigned long long) * 4, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)      // the host tables are freed at return
        return ISRS_ERR_CUDA;

    PrepParams pp;
    std::memset(&pp, 0, sizeof(pp));
    pp.P = (const double *)(base + o_P);
    pp.ch_frel = (const double *)(base + o_frel);
    pp.ch_B = (const double *)(base + o_B);
    pp.ch_alpha = (const double *)(base + o_alpha);
    pp.plan_ch_off = pp.prof_ch_off = pp.prof_plan = (const int *)(base + o_zero);
    pp.plan_n = (const int *)(base + o_plan_n);
    pp.zs_d = (const double2 *)(base + o_zd);
    pp.n_steps = M;
    pp.L = fibre->L_km;
    pp.Cr = fibre->Cr;
    pp.alpha_R = fibre->alpha_R_per_km;
    pp.pd_d = (double *)(base + o_pdd);
    pp.pd_f = (float *)(base + o_pdf);
    pp.step_d = (double2 *)(base + o_stepd);
    pp.step_f = (float2 *)(base + o_stepf);
    pp.lnrho_L = (double *)(base + o_lnL);
    pp.ptot = (double *)(base + o_ptot);
    pp.kap_L = (double *)(base + o_kapL);
    if (launch_prep(pp, 1, st) != cudaSuccess) return ISRS_ERR_CUDA;

    QuadParams qp;
    std::memset(&qp, 0, sizeof(qp));
    qp.pieces = (const DevPiece *)(base + o_pieces);
    qp.items = (const DevItem *)(base + o_items);
    qp.n_items = (int)items.size();
    qp.n_pieces = (int)pieces.size();
    qp.G = quad->G;
    qp.n_steps = M;
    qp.eps_v1 = quad->eps_v1;
    qp.beta2 = fibre->beta2;
    qp.beta3 = fibre->beta3;
    qp.beta4 = fibre->beta4;
    qp.ch_frel = pp.ch_frel;
    qp.ch_B = pp.ch_B;
    qp.ch_alpha = pp.ch_alpha;
    qp.plan_ch_off = qp.prof_ch_off = qp.prof_plan = (const int *)(base + o_zero);
    qp.pd_f = pp.pd_f;
    qp.pd_d = pp.pd_d;
    qp.step_f = pp.step_f;
    qp.step_d = pp.step_d;
    qp.zs_a = (const float4 *)(base + o_za);
    qp.zs_b = (const float4 *)(base + o_zb);
    qp.zs_d = pp.zs_d;
    qp.zs_g = (const float4 *)(base + o_zg);
    qp.zs_gseg = (const float4 *)(base + o_zgs);
    qp.seg = (const int4 *)(base + o_seg);
    for (int v = 0; v < 3; ++v) qp.phi_seg[v] = phi_seg[v];
    qp.kap_L = pp.kap_L;
    qp.n_spans = 1;
    qp.dz_max = dz_max;
    qp.L = (float)fibre->L_km;
    qp.partial = (double *)(base + o_partial);
    qp.counter = (int *)(base + o_counter);
    qp.path_count = (unsigned long long *)(base + o_paths);
    int n_sms = 1;
    cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev);
    int grid = n_sms * quad_blocks_per_sm(quad->precision, M, quad->G, 256);
    if ((int)items.size() < grid) grid = std::max(1, (int)items.size());
    if (!items.empty() && launch_quad(qp, quad->precision, grid, 256, st) != cudaSuccess) return ISRS_ERR_CUDA;

    FinishParams fp;
    std::memset(&fp, 0, sizeof(fp));
    fp.partial = qp.partial;
    fp.slot_items = (const int2 *)(base + o_slot_items);
    fp.slot_cut = (const int *)(base + o_slot_cut);
    fp.prof_slot_off = (const int *)(base + o_slot_off);
    fp.prof_plan = fp.plan_ch_off = fp.prof_ch_off = (const int *)(base + o_zero);
    fp.ch_gamma = (const double *)(base + o_gamma);
    fp.ch_B = pp.ch_B;
    fp.ch_frel = pp.ch_frel;
    fp.P = pp.P;
    fp.lnrho_L = pp.lnrho_L;
    fp.f_ref = fibre->f_ref_THz;
    fp.eta = eta;
    fp.pnli = pnli;
    fp.T = (double *)(base + o_T);
    if (launch_finish(fp, 1, st) != cudaSuccess) return ISRS_ERR_CUDA;
    return ISRS_OK;
}
