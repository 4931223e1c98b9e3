// Internal declarations of the GB300 messenger-field Wiener filter library.
//
// Data layout in HBM (HEALPix):
//   a_lm      FP64 complex, m-major (index(l,m) = m(2 lmax+3-m)/2 + l-m)
//   G, F      ring-Fourier coefficients, [pair][m][hemisphere] complex in the
//             working precision T; pair p couples north ring p with south
//             ring 4 nside - 2 - p (the equator ring, p = 2 nside - 1, is
//             alone).  G is written by the Legendre synthesis and read by the
//             ring pass; F the other way round.
//   r, nu, t  pixel maps in T (source, inverse noise variance, messenger t)
//   tables    per alm: recurrence multiplier A and scale c (mu-form, below);
//             per (m, pair): first active l and two seeds;
//             per ring length: roots e^{i pi p / n} and Bluestein filters.
//
// Legendre recurrence in "mu form": lambda_lm = c_lm mu_lm with
//   mu_l = A_l x mu_{l-1} - mu_{l-2},
// which is the textbook three-term recurrence for the normalised associated
// Legendre functions rescaled so that the l-2 coefficient is one (one
// multiply and one FMA per step).  c is folded into a_lm on synthesis and
// applied after the ring sum on analysis.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/wf.h"

namespace wf {

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
template <typename T> struct V2;
template <> struct V2<double> { using type = double2; };
template <> struct V2<float> { using type = float2; };
template <typename T> using cx = typename V2<T>::type;

template <typename T> __host__ __device__ __forceinline__ cx<T> mk(T a, T b) { cx<T> r; r.x = a; r.y = b; return r; }
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C, typename S> __host__ __device__ __forceinline__ C cscale(C a, S s) { a.x *= s; a.y *= s; return a; }

// ---------------------------------------------------------------------------
// ring table (one entry per north/south ring pair)
// ---------------------------------------------------------------------------
enum RingKind : int { RING_NAIVE = 0, RING_POW2 = 1, RING_BLUESTEIN = 2 };

struct RingTab {
    int n;             // pixels in each ring of the pair
    int q;             // first-pixel longitude is q pi / n (q = 0 or 1)
    int kind;          // RingKind
    int logF;          // log2 of the smem FFT length (pow2: n; Bluestein: M/2)
    long long offN;    // first pixel of the north ring
    long long offS;    // first pixel of the south ring, -1 for the equator
    long long rootOff; // offset of e^{i pi p / n}, p < 2n, in the roots table
    long long vOff;    // offset of the Bluestein filter (M entries: even half, odd half)
    long long cOff;    // offset of the Bluestein chirp e^{-i pi j^2 / n}, j < n, in the chirp table
};

constexpr int NAIVE_MAX = 32;   // rings this short use a direct DFT
constexpr int LEG_THREADS = 256;
constexpr int RING_THREADS = 512;

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------
struct FlatPlan;  // flat-grid state (wf_flat.cu)
// Polarisation (ncomp = 3): spin-2 tables and the (I, Q, U) / (T, E, B) workspace
struct PolState {
    double *al = nullptr, *be = nullptr, *ga = nullptr;  // per alm: spin -+2 recurrence coefficients
    int *ls = nullptr;                                   // per (m, pair): first kept l
    double *p0 = nullptr, *p1 = nullptr, *m0 = nullptr, *m1 = nullptr;  // 2lambda/2, -2lambda/2 at ls and ls + 1
    double2 *a = nullptr, *a_new = nullptr, *b = nullptr;  // 3 x n_alm each: T, E, B
    void *GQ = nullptr, *GU = nullptr, *FQ = nullptr, *FU = nullptr;  // ring coefficients of Q, U (working precision)
    double *r = nullptr;  // 3 x npix: source nu d
    void *t = nullptr;    // 3 x npix: the messenger field (working precision)
    double *nu = nullptr;               // 6 x npix: inverse noise blocks (II, QQ, UU, IQ, IU, QU)
    float *r32 = nullptr, *nu32 = nullptr;  // mixed plans: FP32 copies of r and nu for the blend
    double4 *hbt = nullptr;  // 3 x (lmax + 1): per-l factors of the harmonic blend
    double *part = nullptr, *part2 = nullptr;  // pixel and harmonic partial sums
    // mixed precision: FP32 spin-2 kernels in mu form (lambda = c mu), FP64 block l < lcm(lc, m)
    float4 *tab = nullptr;     // per alm: (A, A be, A (1 + be) - 2, A (1 - be) - 2)
    double *c = nullptr;       // per alm
    int *ls_mx = nullptr;      // per (m, pair): first l of the FP32 recurrence
    float4 *seed = nullptr;    // per (m, pair): mu+ at ls_mx, ls_mx + 1; mu- at ls_mx, ls_mx + 1
    float4 *ac32 = nullptr;    // tensor-core plans: c (Re A, Im A, Re C, Im C) in FP32, the spin-2 B operand's source
    float2 *GQlow = nullptr, *GUlow = nullptr;  // FP64 block's ring coefficients [pair][m < lc][hemisphere]
    double2 *Elow = nullptr, *Blow = nullptr;   // FP64 block's (E, B)
    int lc = -1, low_cap = 0;
};

struct Workspace {
    // HEALPix working buffers; T-typed ones are void* and cast per precision
    double2 *a = nullptr, *a_new = nullptr, *b = nullptr;
    void *G = nullptr, *F = nullptr;
    void *r = nullptr, *nu = nullptr, *t = nullptr;
    void *scr = nullptr;          // per-CTA Bluestein scratch (2 * max Bluestein n complex per CTA)
    float2 *Glow = nullptr;       // mixed: FP64-block synthesis coefficients, rounded to FP32 [pair][glow_cap][hemisphere]
    double2 *b_low = nullptr;     // mixed: FP64-block analysis output (alm layout, m < lc)
    float2 *ca32 = nullptr;       // tensor-core plans: c a_lm in FP32, the synthesis B operand's source
    double *part_pix = nullptr;   // per ring-pair partial sums
    double *part_harm = nullptr;  // per m: [chi2_h, resid^2, x^T S^-1 x, x^T S^-2 x]
    double4 *epi = nullptr;       // per l: factors of the harmonic blend (Eq. 4) for the current lambda
    double *scal = nullptr;       // reduced scalars (device)
    double *h_scal = nullptr;     // pinned host mirror
    double *d_in = nullptr, *nv_in = nullptr, *out_map = nullptr, *cl_in = nullptr, *alm_io = nullptr;  // host-API staging
    uint8_t *mask_in = nullptr;
    double *g1_in = nullptr, *g2_in = nullptr;
    int *flag = nullptr;          // device flags (invalid input)
    int *tc_err = nullptr;        // tensor-core kernels: set when a bounded wait gave up
    double *redu = nullptr;       // reduction scratch
    // mixed plans in correction form (wf_options.mixed_correction), allocated on first use:
    // the iterate x0 at the switch, d0 = G(x0) - x0, delta - d0, and a zero FP32 source map
    double2 *cx0 = nullptr, *cd0 = nullptr, *caold = nullptr;
    void *r0 = nullptr;
};

struct HpTables {
    RingTab *rings = nullptr;
    void *roots = nullptr, *V = nullptr, *tw = nullptr;  // T-typed complex
    void *chirp = nullptr;                               // T-typed complex, per Bluestein length
    // FP64 recurrence (always present): per alm A, c; per (m, pair) first l and seeds; per pair x
    double *A64 = nullptr, *c64 = nullptr;
    int *ls = nullptr;
    double *s0_64 = nullptr, *s1_64 = nullptr;
    double *x64 = nullptr;
    double *st64 = nullptr;  // sin(theta) per pair
    // mixed precision: FP32 A and B = A - 2 per alm, x and w = 1 - x per pair,
    // and the FP32 seeds that start the recurrence at max(l_s, l_c) (m < l_c)
    float *A32 = nullptr, *B32 = nullptr, *x32 = nullptr, *w32 = nullptr;
    int *ls_mx = nullptr;
    float *s0_mx = nullptr, *s1_mx = nullptr;
    int lc_mx = 0;         // FP64 block l < lc_mx of the mixed path
    // the block's Legendre table (double-float pairs, rows of np_pad columns) when it fits the
    // plan's table budget; low_df = 0 runs the FP64 recurrence kernels instead
    float2 *lowtab = nullptr;
    long long lowtab_cap = 0;     // float2 entries allocated
    long long *lowrow = nullptr;  // first row of each m (lmax + 2 entries)
    int low_df = 0, np_pad = 0;
    int glow_cap = 0;      // row length of the FP64-block ring coefficients
    int logNmax = 0;       // twiddle table is e^{-2 pi i t / 2^logNmax}, t < 2^logNmax
    int bmax = 0;          // smem FFT buffer length (complex entries)
    int maxBlue = 0;       // longest Bluestein ring
    int ringGrid = 0;      // persistent grid of the ring kernels
    int *order = nullptr;  // ring pairs by decreasing transform cost
    int *ticket = nullptr; // work counter of the ring kernels (zeroed before each launch)
};

}  // namespace wf

struct wf_plan_s {
    wf_geometry g{};
    int lmax = 0;
    wf_precision prec = WF_PREC_FP64;
    cudaStream_t stream = nullptr;
    int device = 0;
    int nsm = 0;
    long long npix = 0, nalm = 0;
    int nside = 0, nrings = 0, npairs = 0;
    double omega = 0;
    wf::HpTables tab;
    wf::Workspace ws;
    wf::FlatPlan *flat = nullptr;
    wf::PolState *pol = nullptr;  // polarised plans (ncomp = 3)
    wf_options opt{};
    const double2 *start = nullptr;  // starting iterate of the next solves (wf_set_start), or zero
    std::vector<double> replay_lambda;
    std::vector<int> replay_L;
    long long device_bytes = 0;
    std::vector<void *> allocations;
    cudaEvent_t ev[34] = {};  // profiling events: [0..31] kernel pairs, [32..33] iteration
    wf_plan sub = nullptr;    // mixed precision: FP64 plan of the same geometry for the correction sweeps
    bool df_legendre = false; // FP64 plan whose Legendre transforms run in double-float (the sweeps' sub-plan)
    double bnorm_given = 0;   // > 0: the next solve's residual norm |Y^T r| (the sweeps take their parent's)
    bool events_ready = false;
    int tile_syn = 4, tile_ana = 8;  // mixed Legendre tiles: ring pairs per thread / per lane
    bool tc_deferred = false;        // tensor-core plan in a batch step: its synthesis ran in the group launch
    cudaStream_t aux = nullptr;      // mixed precision: stream of the FP64 low-l block
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    long long kcnt[WF_NK] = {};  // kernels launched on this plan, by family (WF_K_*)
    int kfam = WF_K_OTHER;       // family the next launches are counted under
};

namespace wf {

// error reporting (wf_api.cu)
wf_status set_error(wf_status s, const char *fmt, ...);
wf_status cuda_check(cudaError_t e, const char *what);
#define WF_CUDA(call)                                                          \
    do {                                                                       \
        cudaError_t _e = (call);                                               \
        if (_e != cudaSuccess) return ::wf::cuda_check(_e, #call);             \
    } while (0)

// every kernel launch of the HEALPix path is counted on its plan, under the
// family of the stage that is open (Prof::begin) or WF_K_OTHER
#define WF_COUNT_LAUNCH(p) (++(p)->kcnt[(p)->kfam])
// device allocation owned by the plan
wf_status plan_alloc(wf_plan p, void **ptr, size_t bytes);
wf_status host_staging(wf_plan p);
long long hp_estimate_bytes(int nside, int lmax, wf_precision prec, bool staging, int ncomp);
// copies ordered on the plan's stream (no legacy-default-stream copies: the
// plan may run on a non-blocking stream beside other plans); to_host waits
wf_status to_device(wf_plan p, void *dst, const void *src, size_t bytes);
wf_status to_host(wf_plan p, void *dst, const void *src, size_t bytes);
// raise a kernel's dynamic shared-memory limit to at least `bytes` (never lowers it;
// serialised, so plans used from several host threads cannot undo each other)
wf_status raise_smem_limit(const void *func, size_t bytes);

// Per-call kernel accounting: launch counts always; device time per kernel
// family with CUDA events on the plan's stream when profiling is on.
struct Prof {
    wf_plan p = nullptr;
    wf_info *info = nullptr;
    bool on = false;
    int nopen = 0;
    int fam[16];
    long long launches = 0;
    double ms[WF_NK] = {};
    long long cnt[WF_NK] = {};
    long long k0[WF_NK] = {};  // plan launch counters when this accounting started
    Prof() = default;
    Prof(wf_plan p_, wf_info *i, bool profile) { init(p_, i, profile); }
    void init(wf_plan p_, wf_info *i, bool profile);
    void begin(int family);  // call before the launches of a stage of `family`
    void end();              // call after them
    void collect();          // after a stream synchronisation: harvest event times
    void iter_begin();
    double iter_end();       // after a synchronisation: ms since iter_begin (NaN when off)
    void finish();           // copy into info
};

// Legendre transforms (wf_legendre.cu)
wf_status hp_build_legendre_tables(wf_plan p, const std::vector<double> &xpair, const std::vector<double> &stpair);
enum LegMode { LEG_ADJOINT = 0, LEG_BLEND = 1 };
struct BlendArgs {
    double lam_tauh = 0;   // lambda tau Omega
    double tauh = 0;       // tau Omega
    const double *S = nullptr;  // C_ell (device)
    const double4 *epi = nullptr;  // per l: (Omega S/(S + lambda tau_h), 1/S, 1/S + 1/tau_h, S > 0); filled per launch
    int want_resid = 0;
};
wf_status hp_set_low_block(wf_plan p, int lc);
long long hp_low_table_bytes(int lmax, int npairs, int lc);
wf_status hp_autotune(wf_plan p, int reps);
wf_status hp_legendre_synthesis(wf_plan p, const double2 *alm, int L);
wf_status hp_legendre_analysis(wf_plan p, int L, LegMode mode, const BlendArgs &ba, const double2 *a_old,
                               double2 *out);
// tensor-core transforms (wf_tc.cu): ncols columns sharing p's geometry, tables and FP64 block
constexpr int TC_MAX_COLUMNS = 16;
// precisions whose Legendre synthesis runs on the tensor cores
inline bool tc_prec(wf_precision p) { return p == WF_PREC_MIXED_TF32 || p == WF_PREC_MIXED_SPLITBF16; }
wf_status hp_tc_synthesis(wf_plan p, int ncols, const double2 *const *a, float2 *const *ca, float2 *const *G,
                          const int *L, int Lmax, cudaStream_t stream);
size_t tc_syn_smem(int nc, int L);
wf_status tc_prepare(int lmax);
// polarised plans: the spin-2 synthesis of up to TCP_MAX_COLUMNS columns (four B rows per column)
constexpr int TCP_MAX_COLUMNS = 8;
wf_status hp_pol_tc_synthesis(wf_plan p, int ncols, const double2 *const *E, const double2 *const *B,
                              float4 *const *ac, float2 *const *GQ, float2 *const *GU, const int *L, int Lmax,
                              cudaStream_t stream);

// ring transforms (wf_ring.cu)
wf_status hp_build_ring_tables(wf_plan p);
// RS_BLEND_ANA: the blended ring goes straight into the forward DFT and the unfold to F
enum RingSynMode { RS_BLEND = 0, RS_MAP = 1, RS_SYN = 2, RS_BLEND_ANA = 3 };
wf_status hp_ring_synthesis(wf_plan p, int L, RingSynMode mode, double lam, double tau, double *out_map);
wf_status hp_ring_analysis(wf_plan p, int L, const void *map_T);
// the same passes on explicit buffers (G / F in the working precision, maps T-typed or FP64 out)
wf_status hp_ring_synthesis_buf(wf_plan p, int L, RingSynMode mode, double lam, double tau, const void *G,
                                void *tmap, double *out_map);
wf_status hp_ring_analysis_buf(wf_plan p, int L, const void *map_T, void *F);
// mixed plans: the FP32 synthesis pass with an explicit FP64-block buffer (m < lc)
wf_status hp_ring_synthesis_analysis(wf_plan p, int L, double lam, double tau);
wf_status hp_ring_synthesis_buf_low(wf_plan p, int L, RingSynMode mode, double lam, double tau, const void *G,
                                    const float2 *glow, int lc, int glow_stride, void *tmap, double *out_map);
// FP64 temperature Legendre transforms on explicit buffers (FP64 plans)
wf_status hp_legendre_synthesis_buf(wf_plan p, const double2 *alm, int L, double2 *G);
wf_status hp_legendre_adjoint_buf(wf_plan p, int L, const double2 *F, double2 *out);
// polarisation (wf_spin.cu)
wf_status hp_pol_create(wf_plan p, const double *xpair_dev, const double *stpair_dev);
void hp_pol_destroy(wf_plan p);
wf_status hp_pol_legendre_synthesis(wf_plan p, const double2 *E, const double2 *B, int L);
wf_status hp_pol_legendre_analysis(wf_plan p, int L, double2 *E, double2 *B);
wf_status hp_pol_setup(wf_plan p, const double *d, const double *N6, const uint8_t *mask, double *tau, long long *ndof);
wf_status hp_pol_blend(wf_plan p, double lam, double tau, int *nblocks);
wf_status hp_pol_hblend(wf_plan p, int L, const double *C, double lam_tauh, double tauh, int want_resid);
wf_status hp_pol_alm_norm(wf_plan p, const double *C, const double2 *a, int mode);
wf_status hp_pol_pix_chi2(wf_plan p, const double *d, const double *s_map, int *nblocks);
wf_status hp_pol_isqrt_prior(wf_plan p, const double *C, const double2 *g2, double2 *out);  // S^+1/2 g2
// the FP64 block of the mixed spin-2 transforms (m < lc, l < lcm(lc, m)): synthesis into FP32 ring
// coefficients with stride lc, analysis from the FP32 ring coefficients
wf_status hp_pol_legendre_synthesis_low(wf_plan p, const double2 *E, const double2 *B, int L, int lc, float2 *GQ,
                                        float2 *GU);
wf_status hp_pol_legendre_analysis_low(wf_plan p, int L, int lc, const float2 *FQ, const float2 *FU, double2 *E,
                                       double2 *B);
// mixed precision (wf_spin_mx.cu)
wf_status hp_pol_create_mx(wf_plan p);
wf_status hp_pol_set_low_block(wf_plan p, int lc);
wf_status hp_pol_legendre_synthesis_mx(wf_plan p, const double2 *E, const double2 *B, int L);
wf_status hp_pol_legendre_analysis_mx(wf_plan p, int L, double2 *E, double2 *B);
wf_status hp_pol_fluct_source(wf_plan p, const double *g1, const double *z);  // r = nu^1/2 g1 + Omega z
wf_status hp_pol_round_pixels(wf_plan p);  // mixed plans: FP32 copies of r and nu

// flat grid (wf_flat.cu)
wf_status flat_create(wf_plan p);
void flat_destroy(wf_plan p);
wf_status flat_solve(wf_plan p, const double *r_or_d, const double *noise_var, const uint8_t *mask,
                     const double *S, double tol, bool fluct, const double *g1, const double *g2, double *s_out,
                     double *alm_out, wf_info *info);
wf_status flat_alm2map(wf_plan p, const double *alm, double *map);
wf_status flat_map2alm(wf_plan p, const double *map, double *alm);

}  // namespace wf
