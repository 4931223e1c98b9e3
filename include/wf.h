/*
 * wf.h -- C ABI of the GB300 messenger-field Wiener filter.
 *
 * Solves the Wiener-filter equation (Elsner & Wandelt 2013, Eq. 2)
 *     (S^-1 + N^-1) s_WF = N^-1 d
 * for a signal covariance S that is diagonal in harmonic space and a noise
 * covariance N that is diagonal in pixel space, by the messenger iteration of
 * Sect. 2.1 (Eqs. 3-4): a pixel-space blend of the data with the current
 * signal through an auxiliary field of covariance T = tau 1 (tau = min N),
 * then a harmonic-space blend with the prior, with the cooling parameter
 * lambda >= 1 of Sect. 2.2 and Sect. 3.  wf_fluct runs the same iteration on
 * the source of Eq. (9) to draw fluctuation maps for constrained
 * realisations (Sect. 2.3).
 *
 * Geometries: a periodic flat ny x nx grid with the unitary 2-D DFT, and the
 * HEALPix RING sphere with spherical harmonics up to lmax (Sect. 3).
 *
 * Conventions
 *   - Pixel maps: FP64, row-major ny x nx (flat) or HEALPix RING order
 *     (sphere).  mask: uint8 per pixel, 1 = observed, 0 = masked (N^-1 = 0).
 *   - Harmonic vectors ("alm"), complex FP64 interleaved (re, im):
 *       flat:    the rfft half plane, ny rows of nx/2+1, row-major, unitary;
 *       HEALPix: a_lm for m >= 0, m-major: index(l, m) = m(2 lmax+3-m)/2 + l-m,
 *                Y_lm with the Condon-Shortley phase, orthonormal; a real map
 *                is f = sum_l [a_l0 Y_l0 + 2 Re sum_{m>0} a_lm Y_lm].
 *   - Prior: HEALPix C_ell[l], l = 0..lmax (beam included; C_0 = C_1 = 0
 *     holds those modes at zero).  Flat: S per half-plane mode (ny x nx/2+1).
 *   - Unless a function says otherwise, every array pointer is a DEVICE
 *     pointer, owned by the caller, read or written on the plan's stream.
 *
 * Errors: functions return a wf_status; nothing throws or aborts across the
 * ABI.  wf_last_error() gives a human-readable detail for the calling thread.
 * Calls on one plan must not overlap (a plan holds one solve's workspace);
 * different plans may be used from different threads.
 */
#ifndef WF_H
#define WF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wf_plan_s *wf_plan; /* opaque; created and owned by the library */

typedef enum {
    WF_OK = 0,
    WF_EINVAL = 1,    /* bad argument or input (NaN / negative noise, all pixels masked, ...) */
    WF_ENOMEM = 2,    /* device or host allocation failed */
    WF_ECUDA = 3,     /* a CUDA call failed; see wf_last_error() */
    WF_ENOCONV = 4,   /* iteration cap reached; the last iterate is still written */
    WF_EDIVERGE = 5,  /* residual grew without bound (e.g. lmax far above 2 nside, where the HEALPix
                         analysis Omega Y^T is too far from the inverse of the synthesis to contract) */
    WF_ETIMEOUT = 6,  /* a bounded device wait gave up */
    WF_EUNSUPPORTED = 7
} wf_status;

typedef enum { WF_GEOM_FLAT = 0, WF_GEOM_HEALPIX = 1 } wf_geom_kind;

typedef enum {
    WF_PREC_FP64 = 0,       /* every step in FP64 */
    WF_PREC_MIXED_FP32 = 1, /* FP32 Legendre recurrence/contraction and ring FFTs from FP64 seeds;
                               FP64 a_lm, reductions and residual refinement */
    WF_PREC_MIXED_TF32 = 2, /* as MIXED_FP32, with the Legendre synthesis contraction on the tensor cores
                               (tcgen05): the FP32 recurrence values and c a_lm split into TF32 head + tail,
                               hi*hi + hi*lo + lo*hi accumulated in FP32 ("3xTF32", FP32-grade accuracy).
                               Maps of one geometry in one wf_solve_batch share the recurrence (one launch).
                               HEALPix plans; polarised ones (ncomp = 3) run the spin-2 synthesis on the
                               tensor cores too (the (Re, Im) of E + iB and E - iB against the spin +-2
                               recurrences) */
    WF_PREC_MIXED_SPLITBF16 = 3 /* as MIXED_TF32 with BF16 operands: each value split into three BF16 pieces
                                   (successive round-to-nearest of the exact remainders, ~24 significant bits)
                                   and the six products of total order <= 2 accumulated in FP32 */
} wf_precision;

typedef struct {
    wf_geom_kind kind;
    int nx, ny;  /* flat only: nx = ny, a power of two, 16 <= n <= 128 */
    int nside;   /* HEALPix only */
    int ncomp;   /* 1 (temperature) or 3 (polarised I, Q, U: HEALPix, any precision) */
} wf_geometry;

/* Options of the cooling schedule and stopping rule (Sect. 3).  Zero-filled
 * fields take the defaults shown. */
typedef struct {
    int maxiter;        /* total iteration cap (default 20000) */
    int level_cap;      /* iterations at one lambda level before it is left anyway (HEALPix 300, flat 200) */
    double eta;         /* plateau: |chi2_k - chi2_{k-1}| < eta sqrt(2 n_dof) (HEALPix 3e-5, flat 1e-2) */
    int ell0;           /* HEALPix: first l_iter (20) */
    int ell_step_max;   /* HEALPix: largest increase of l_iter per level (500) */
    int band_margin;    /* HEALPix: transform band limit L = l_iter + margin (100) */
    double lambda_max;  /* flat: first lambda level (100) */
    int refine_sweeps;  /* mixed precision: FP64 lambda = 1 sweeps from the mixed result, stopping at tol (0);
                           with sweeps, wf_info.converged and the status report the FP64 operator's verdict */
    int profile;        /* nonzero: time every kernel family with CUDA events (fills wf_info.kernel_ms) */
    double mixed_kappa; /* mixed precision: modes with S_l / (tau Omega) >= kappa run in FP64 (3e4); polarised
                           plans use the largest eigenvalue of each l's prior block for S_l */
    int mixed_lc;       /* mixed precision: > 0 forces the FP64 block l < mixed_lc, < 0 disables it, 0 = auto */
    int schedule;       /* 0: heuristic cooling of Sect. 3 (default); 1: chi^2-bound cooling of Sect. 2.2
                           (HEALPix Wiener filter only: lambda such that chi^2(lambda, x) = b every iteration,
                           b = n_dof - m_sigma sqrt(2 n_dof), raised when lambda stalls; full band) */
    double m_sigma;     /* chi^2-bound cooling: initial b = n_dof - m_sigma sigma_chi2 (5) */
    double stall_tol;   /* chi^2-bound cooling: lambda - 1 changing by less than this fraction in one
                           iteration counts as converged at lambda > 1 and raises b (1e-7) */
    long long mixed_table_bytes; /* mixed precision: device-memory cap of the FP64 block's Legendre table
                                    (lambda_lm for l < l_c, every ring pair, as double-float pairs; 0 = 2 GiB,
                                    < 0 = no table).  A block whose table fits is contracted from it on the FP32
                                    pipe in double-float arithmetic; otherwise the FP64 recurrence kernels run.
                                    A nonzero mixed_lc in these options, or a changed cap, applies at once, so
                                    the basis-change calls below use that block too. */
    int fp64_emulation; /* FP64 temperature plans: nonzero runs the Legendre transforms in double-float
                           arithmetic on the FP32 pipe (pairs of FP32 numbers, about 48 significant bits;
                           error-free products and sums), several times faster than the FP64 pipe on GPUs
                           whose FP64 rate is a small fraction of FP32.  Mixed temperature plans: the
                           correction sweeps' transforms run this way unless it is negative, which runs
                           them on the FP64 pipe. */
    double mixed_tol_factor; /* mixed plans with refine_sweeps > 0: the FP32 iteration stops at tol x factor
                                (0 < factor < 1; 0 = 1) before the FP64 sweeps check the result against tol
                                under the FP64 operator.  The FP32 operator's fixed point differs from the
                                FP64 one in the slowest modes, so the FP64-operator residual of an FP32
                                iterate at tol can lie above tol (by ~20 % on the nside 2048 map) */
    int tile_syn;       /* mixed plans: > 0 sets the FP32 Legendre synthesis tile (2, 4 or 8 ring pairs per
                           thread) in place of the default or autotuned one; 0 keeps it */
    int tile_ana;       /* mixed plans: > 0 sets the FP32 Legendre analysis tile (2, 4 or 8 ring pairs per
                           lane); 0 keeps it */
    double mixed_correction; /* mixed temperature plans, single solves (wf_solve, wf_fluct, their host forms
                                and requests of the request loop; not wf_solve_batch): > 0 switches the FP32 iteration to correction form once, at lambda = 1
                                on the full band, when its residual is below tol x mixed_correction.  The
                                messenger iteration is affine, a_{k+1} = B a_k + c (Eqs. 3-4).  One FP64
                                iteration from the current iterate x0 (double-float Legendre transforms, as
                                in the correction sweeps) gives d0 = B x0 + c - x0; the FP32 kernels then
                                iterate on delta = a - x0, delta <- d0 + B delta (the same kernels with the
                                source set to zero), so their rounding scales with |delta| instead of |a|,
                                and the residual they report is the FP64 operator's to that rounding.  The
                                FP64 iteration counts as one iteration of the trace (chi^2 NaN from there on:
                                the kernels no longer see the iterate itself).  Allocates three a_lm arrays
                                and one FP32 map on first use.  0 (default): off */
} wf_options;

/* Kernel families reported in wf_info (HEALPix path; the flat path is one
 * fused kernel, reported under WF_K_FLAT). */
enum {
    WF_K_LEG_SYN = 0,   /* Legendre synthesis a_lm -> G_m(theta) */
    WF_K_RING_SYN = 1,  /* ring fold + inverse ring DFT + pixel blend (Eq. 3) */
    WF_K_RING_ANA = 2,  /* forward ring DFT + unfold */
    WF_K_LEG_ANA = 3,   /* Legendre analysis + harmonic blend (Eq. 4) */
    WF_K_OTHER = 4,     /* setup, reductions, conversions */
    WF_K_FLAT = 5,      /* fused flat-grid solve */
    WF_NK = 6
};

/* Per-solve report.  The trace arrays are optional and caller-owned HOST
 * memory of trace_cap entries; entry k describes iteration k. */
typedef struct {
    int iters;              /* messenger iterations run */
    int converged;          /* 1 if the residual fell below tol at lambda = 1, full band */
    double final_residual;  /* relative residual of the last full-band lambda = 1 iteration */
    double chi2_over_ndof;  /* chi^2(s, 1) / n_dof of the result (Wiener filter only) */
    long long n_dof;        /* observed pixels */
    double tau;             /* min noise variance over observed pixels */
    int n_levels;           /* lambda levels visited (chi^2-bound schedule: values the bound b took) */
    int refine_sweeps;      /* FP64 correction sweeps run (mixed precision) */
    int mixed_lc;           /* FP64 block l < mixed_lc used by the mixed-precision transforms */
    double *lambda_trace;   /* optional, lambda_k */
    int *L_trace;           /* optional, band limit L_k (HEALPix; -1 on the flat grid) */
    double *chi2_trace;     /* optional, chi^2 of the iterate entering iteration k (Eq. 6, x-independent part
                               dropped); under the chi^2-bound schedule the full chi^2(lambda_k, x_k), which
                               equals the bound b while lambda_k > 1 */
    double *resid_trace;    /* optional, relative residual (NaN where lambda > 1 or L < lmax) */
    double *iter_ms_trace;  /* optional, device time of iteration k in ms (CUDA events; HEALPix) */
    int trace_cap;
    long long launches;                 /* kernels this call launched */
    double kernel_ms[WF_NK];            /* device time per kernel family (wf_options.profile) */
    long long kernel_launches[WF_NK];   /* launches per kernel family */
} wf_info;

/* Build a plan for one geometry and band limit (HEALPix lmax <= 2 nside is
 * the supported range; flat: lmax ignored).  Precomputes the ring geometry,
 * the Legendre seeds and recurrence tables, the ring-FFT tables and the
 * workspace.  cuda_stream: a cudaStream_t (NULL = the legacy default stream)
 * that every later call on this plan uses.  *out receives the plan. */
wf_status wf_plan_create(const wf_geometry *g, int lmax, wf_precision p, void *cuda_stream, wf_plan *out);
void wf_plan_destroy(wf_plan p);
wf_status wf_set_options(wf_plan p, const wf_options *opt);

/* Replay mode: the next solves run exactly n iterations with lambda[k] and
 * band limit L[k] (ignored on the flat grid) instead of the cooling schedule,
 * so that two implementations can be compared iteration for iteration.
 * Host arrays, copied; n = 0 returns to the schedule. */
wf_status wf_set_schedule(wf_plan p, const double *lambda, const int *L, int n);

/* Checkpoint / resume.  The messenger iteration keeps no state but its
 * iterate a_k and the schedule's (lambda, L): the next solves on this plan
 * start from alm0 (device, n_alm complex per component, the layout of
 * alm_out) instead of zero; NULL restores the zero start.  The pointer is kept,
 * not copied: the array must stay valid while the plan solves.  A run stopped
 * after k iterations (alm_out and the (lambda, L) trace of its report) and
 * resumed with wf_set_start(alm_out) and wf_set_schedule(the rest of the
 * trace) repeats the uninterrupted run (to the atomics' reduction order).
 * HEALPix plans; not with the chi^2-bound schedule (WF_EUNSUPPORTED at the
 * solve); in a replay the run stops at the first full-band lambda = 1
 * iteration whose residual is below tol. */
wf_status wf_set_start(wf_plan p, const double *alm0);

/* Wiener filter (Eq. 2) by the messenger iteration.  d, noise_var: n_pix
 * FP64; mask: n_pix uint8 (may be NULL: all observed); C_ell: prior (see
 * conventions).  tol: relative residual |(S^-1 + N^-1) s - N^-1 d| / |N^-1 d|
 * in harmonic coordinates at which to stop.  s_wf: n_pix FP64 output.
 * alm_out: optional harmonic output.  info: optional report.
 * Noise variance must be finite and > 0 on observed pixels, and the prior
 * (C_ell, or S on the flat grid) finite and >= 0 everywhere (WF_EINVAL).
 * Polarised plans (ncomp = 3; Eqs. 10-11, heuristic cooling or replay): d and
 * s_wf are 3 x n_pix (I, Q, U, component-major); noise_var is the 3x3 noise
 * covariance per pixel as 6 x n_pix (II, QQ, UU, IQ, IU, QU); the mask byte of a
 * pixel is a code: 0 nothing observed, 1 I, Q and U, 2 I only (polarisation
 * masked), 3 Q and U only (temperature masked), others WF_EINVAL (NULL: all
 * observed).  Masking is infinite noise component by component: N^-1 is the
 * inverse of the observed sub-block, which must be positive definite, tau
 * the smallest eigenvalue of any observed sub-block and n_dof the number of
 * observed components; d may hold anything in unobserved components.  C_ell is 4 x (lmax + 1)
 * (TT, EE, BB, TE), each block [[TT, TE, 0], [TE, EE, 0], [0, 0, BB]] positive
 * semi-definite with TE^2 < TT EE wherever TE != 0 (WF_EINVAL otherwise); zero
 * entries act through the pseudo-inverse (e.g. BB = 0, or l < 2); alm_out is
 * 3 x n_alm (T, E, B).  Spin-2 convention: (Q + iU) = sum_{l >= 2, |m| <= l}
 * 2a_lm 2Y_lm, 2a = -(E + iB), sY_lm = sqrt((2l+1)/(4 pi)) d^l_{m,-s}(theta)
 * e^{i m phi}.  tau is the smallest eigenvalue of any observed noise block. */
wf_status wf_solve(wf_plan p, const double *d, const double *noise_var, const uint8_t *mask,
                   const double *C_ell, double tol, double *s_wf, double *alm_out, wf_info *info);

/* Same as wf_solve with every array in HOST memory: the library copies the
 * inputs to the device and the outputs back, inside the call. */
wf_status wf_solve_host(wf_plan p, const double *d, const double *noise_var, const uint8_t *mask,
                        const double *C_ell, double tol, double *s_wf, double *alm_out, wf_info *info);

/* Fluctuation map (Sect. 2.3, Eqs. 8-9): the messenger iteration with the
 * source N^-1/2 g1 + S^-1/2 g2 (g1: n_pix FP64 unit normal draws; g2: unit
 * complex normal harmonic draws in the harmonic layout, m = 0 / kx-Hermitian
 * entries real).  f_out: n_pix FP64 with covariance (S^-1 + N^-1)^-1.
 * A constrained realisation is s_WF + f_out.
 * Polarised plans (ncomp = 3): g1 3 x n_pix (I, Q, U), g2 3 x n_alm (T, E,
 * B), f_out 3 x n_pix, noise and C_ell as for wf_solve; N^-1/2 is the
 * symmetric square root of each pixel's inverse noise block and S^-1/2 the
 * pseudo-inverse square root of each l's prior block.  chi2_over_ndof of the
 * report is NaN (it needs data). */
wf_status wf_fluct(wf_plan p, const double *noise_var, const uint8_t *mask, const double *C_ell,
                   const double *g1, const double *g2, double tol, double *f_out, double *alm_out,
                   wf_info *info);

/* Basis change used by the iteration (Sect. 2.1), exposed for users and for
 * checking: map = Y a restricted to l <= L (HEALPix) or the unitary inverse
 * real DFT (flat, L ignored); and its adjoint alm = Y^T map (the analysis
 * without the pixel area, Omega Y^T being the HEALPix analysis). */
wf_status wf_alm2map(wf_plan p, const double *alm, int L, double *map);
wf_status wf_map2alm_adjoint(wf_plan p, const double *map, int L, double *alm);

/* Template marginalisation before the solve (Sect. 3, Eq. 12): the sigma ->
 * infinity limit of (1 + sigma V V^T)^-1 d_raw by the Woodbury identity,
 *     d_out = d_raw - V (V^T V)^-1 V^T d_raw,
 * with V the monopole and the three dipole templates (1, sin th cos ph,
 * sin th sin ph, cos th) on the observed pixels (mask != 0; NULL = all).
 * Masked pixels are copied unchanged.  HEALPix plans only.  d_raw, mask,
 * d_out: device; d_out may equal d_raw.  coef: optional HOST array of 4,
 * receives the removed template amplitudes.  Synchronises the stream. */
wf_status wf_remove_templates(wf_plan p, const double *d_raw, const uint8_t *mask, double *d_out, double *coef);

/* Several data sets of one signal with the same beam and pixelisation (the
 * generalisation the paper's outlook names, Sect. 4).  For data d_k = s + n_k
 * with noise variance N_k the stacked Wiener-filter equation
 *     (S^-1 + sum_k N_k^-1) s = sum_k N_k^-1 d_k
 * is Eq. (2) of one data set with, per pixel over the data sets observing it,
 *     N^-1 = sum_k N_k^-1,   N^-1 d = sum_k N_k^-1 d_k.
 * This call forms that data set: d_out = (sum N_k^-1 d_k) / (sum N_k^-1),
 * noise_var_out = 1 / sum N_k^-1, mask_out = 1 where any data set observes
 * the pixel (unobserved pixels: d_out = 0, noise_var_out = 1, mask_out = 0);
 * wf_solve / wf_fluct on the outputs then give the stacked solution.
 * Data sets with different beams are not reducible this way.
 * k: 1..16 data sets.  d, noise_var, mask: HOST arrays of k DEVICE pointers
 * (n_pix FP64 maps; mask may be NULL, or hold NULL entries: all observed).
 * d_out, noise_var_out (n_pix FP64) and mask_out (n_pix uint8): device.
 * Temperature plans (ncomp = 1; WF_EUNSUPPORTED otherwise), flat or HEALPix.
 * Non-finite or non-positive noise, or non-finite data, on an observed
 * pixel: WF_EINVAL.  Synchronises the plan's stream. */
wf_status wf_combine_datasets(wf_plan p, int k, const double *const *d, const double *const *noise_var,
                              const uint8_t *const *mask, double *d_out, double *noise_var_out, uint8_t *mask_out);

/* Sizes of the plan's arrays. */
long long wf_npix(wf_plan p);
long long wf_nalm(wf_plan p); /* complex entries */
/* Device bytes the plan holds (tables + workspace, including the FP64
 * sub-plan of the correction sweeps once created). */
long long wf_plan_device_bytes(wf_plan p);
/* Device bytes a plan of this geometry will hold, computed without creating
 * it (upper estimate; with_host_staging adds the buffers of the *_host entry
 * points).  -1 for an invalid geometry. */
long long wf_plan_estimate_bytes(const wf_geometry *g, int lmax, wf_precision prec, int with_host_staging);
/* Autotuner of the mixed-precision Legendre tiles: times each variant (2, 4
 * or 8 ring pairs per thread in the synthesis, per lane in the analysis) on
 * this plan's own buffers at the full band and keeps the fastest; reps timed
 * launches per variant (<= 0: 3).  FP64 and flat plans: no effect.  Overwrites
 * the plan's iterate buffers (call it between solves).  wf_plan_tiles reports
 * the current choice (defaults 4 and 8). */
wf_status wf_plan_autotune(wf_plan p, int reps);
wf_status wf_plan_tiles(wf_plan p, int *syn_pairs, int *ana_pairs);
/* Move the plan to another CUDA stream (waits for work queued on the old one). */
wf_status wf_plan_set_stream(wf_plan p, void *cuda_stream);
/* wf_fluct with HOST buffers (copies in, solves, copies the map out). */
wf_status wf_fluct_host(wf_plan p, const double *noise_var, const uint8_t *mask, const double *C_ell,
                        const double *g1, const double *g2, double tol, double *f_out, double *alm_out,
                        wf_info *info);

const char *wf_strerror(wf_status s);
const char *wf_last_error(void);
/* Size in bytes of one of this header's structs as the library was built, by its name
 * ("wf_geometry", "wf_options", "wf_info", "wf_batch_item", "wf_request", "wf_result",
 * "wf_server_stats"); 0 for any other name or a null pointer.  A binding that mirrors the
 * structs compares the sizes with its own layouts before it passes one.  Host only. */
long long wf_abi_sizeof(const char *name);

/* Measurement utility; the paper has no counterpart.  Times an FP32 FMA loop
 * (independent chains, two 512-thread CTAs per SM; packed != 0 issues packed
 * f32x2 FMAs as the mixed Legendre kernels do) on cuda_stream and writes the
 * best of three timed launches, in TFLOP/s (2 flops per FMA), to *tflops: the
 * measured peak of the FP32 pipe that bounds the mixed Legendre transforms.
 * Synchronises the stream; allocates nothing. */
wf_status wf_probe_fp32_fma(void *cuda_stream, int packed, double *tflops);

/* Flat-grid Wiener filter that allocates no device memory: the paper has no
 * counterpart; it exists for callers that cannot allocate at solve time (a
 * solve inside another framework's memory pool, or where cudaMalloc is not
 * allowed).  Same arithmetic and results as wf_solve on a flat plan of the
 * same n, with the solver's scratch in one static device array (0.71 MiB,
 * resident on every device that loads the library) instead of plan memory.
 * n: power of two in [16, 128]; opt: may be NULL (defaults), opt->maxiter <=
 * 20000; anything larger is rejected with WF_EINVAL.  d, noise_var, mask, S,
 * s_wf, alm_out: device pointers as for wf_solve; cuda_stream: the stream to
 * use.  S must be finite and >= 0 (WF_EINVAL otherwise).  Each call looks up
 * the array's device address on the current device (cudaGetSymbolAddress);
 * nothing is cached between calls.  All calls share
 * the array, so calls that overlap on the GPU race; each call writes what it
 * reads first.  Every copy of the call (status, traces) is ordered on
 * cuda_stream, and the call returns after that stream has synchronised. */
wf_status wf_flat_solve_noalloc(int n, const double *d, const double *noise_var, const uint8_t *mask,
                                const double *S, double tol, const wf_options *opt, void *cuda_stream,
                                double *s_wf, double *alm_out, wf_info *info);

/* Kinds of solve (batch items and serving requests). */
typedef enum { WF_REQ_WF = 0, WF_REQ_FLUCT = 1, WF_REQ_CR = 2 } wf_request_kind;

/* Batched solves: n HEALPix solves (Wiener filter of Sect. 2.1 or fluctuation
 * map of Eq. 9; plans of any nside / lmax / precision, one distinct plan per
 * item) advanced together.  Each step captures one messenger iteration of
 * every unfinished solve, each on its own stream, in one CUDA graph and
 * launches it with one call; the host then runs each solve's own cooling
 * schedule (heuristic of Sect. 3 or a replay).  The graph is replayed while no
 * solve changes (lambda, L) and updated when one does.  Results equal those
 * of wf_solve / wf_fluct on the same plan (to rounding).  Items use device
 * pointers as in wf_solve; info may be NULL.  Polarised plans (ncomp = 3)
 * may be mixed with temperature plans; their items take the three-component
 * layouts of wf_solve / wf_fluct (per-item sizes below are for ncomp = 1).
 * The chi^2-bound schedule is not batchable (WF_EUNSUPPORTED).  cuda_stream:
 * stream the graph is launched on;
 * statuses[i]: the status of item i (WF_OK / WF_ENOCONV / error).  The return
 * value reports argument and CUDA errors of the batch as a whole. */
typedef struct {
    int kind;                 /* WF_REQ_WF or WF_REQ_FLUCT */
    const double *d;          /* WF: npix */
    const double *noise_var;  /* npix */
    const uint8_t *mask;      /* npix or NULL */
    const double *C_ell;      /* lmax + 1 */
    const double *g1, *g2;    /* FLUCT: npix real and n_alm complex draws */
    double tol;
    double *s_out;            /* npix */
    double *alm_out;          /* n_alm complex, optional */
    wf_info *info;            /* optional */
} wf_batch_item;
wf_status wf_solve_batch(int n, wf_plan *plans, const wf_batch_item *items, void *cuda_stream, wf_status *statuses);

/* ------------------------------------------------------------------------
 * Serving: a request loop over many HEALPix solves of mixed size.
 *
 * The paper solves one map at a time; this engine runs many Wiener-filter
 * (Sect. 2.1), fluctuation (Eq. 9) and constrained-realization (Sect. 2.3:
 * s_WF + f) requests concurrently on one GPU.  Requests carry HOST buffers
 * and wait in a FIFO queue.  Each of `slots` worker threads owns a CUDA
 * stream and takes the next request that can be admitted:
 *   - a plan (tables + workspace) of the request's (nside, lmax, precision, ncomp) is
 *     taken from the pool of idle plans, or created if the plans' device bytes
 *     stay within `mem_budget` after it (estimate from wf_plan_estimate_bytes),
 *     evicting least recently used idle plans for the queue head if needed;
 *   - the head of the queue has priority; a request behind it is admitted
 *     before it only into memory that is free without evicting anything.
 * Plans stay resident between requests, so a geometry's Legendre tables are
 * built once; the solves of different slots run on different streams and
 * overlap on the device.  Every result is that of the corresponding direct
 * call (wf_solve_host / wf_fluct_host) on a plan of the same geometry. */
typedef struct wf_server_s *wf_server;

typedef struct {
    unsigned long long tag;   /* caller's identifier, returned in the result */
    int kind;                 /* wf_request_kind */
    int nside, lmax;          /* HEALPix geometry, 2 <= lmax <= 2 nside */
    wf_precision precision;
    double tol;
    wf_options opt;           /* per-request options (zero-filled: defaults) */
    /* host buffers, owned by the caller, valid until the result is returned */
    const double *d;          /* WF, CR: npix */
    const double *noise_var;  /* npix */
    const uint8_t *mask;      /* npix or NULL */
    const double *C_ell;      /* lmax + 1 */
    const double *g1, *g2;    /* FLUCT, CR: npix real and n_alm complex draws of Eq. (9) */
    double *s_out;            /* npix: s_WF (WF), f (FLUCT), s_WF + f (CR) */
    double *f_out;            /* CR only, optional: npix, the fluctuation map f */
    int ncomp;                /* 0 or 1: temperature; 3: polarised (I, Q, U), every array in the
                                 three-component layouts of wf_solve / wf_fluct */
} wf_request;

typedef struct {
    unsigned long long tag;
    wf_status status;         /* of the solve (WF_ENOCONV: the last iterate is written) */
    int iters;                /* messenger iterations (CR: both solves) */
    int converged;
    double final_residual;
    double chi2_over_ndof;    /* WF and CR */
    double t_submit, t_start, t_done;  /* seconds since wf_server_create */
    int slot;                 /* worker that ran it */
    int plan_reused;          /* 1 if an existing plan served it */
} wf_result;

typedef struct {
    long long pending, active, completed, rejected;
    long long bytes_in_use;   /* device bytes of all pooled plans (busy and idle) */
    long long peak_bytes;     /* maximum of bytes_in_use */
    long long budget;
    int plans, max_active;    /* pooled plans; most solves in flight at once */
    long long plans_created, plans_evicted;
} wf_server_stats;

/* device: CUDA device index; mem_budget: bytes of device memory for plans;
 * slots: concurrent solves (1..64). */
wf_status wf_server_create(int device, long long mem_budget, int slots, wf_server *out);
/* Queue a request (the struct is copied; the arrays are not).  A request that
 * can never fit the budget, or is invalid, completes at once with an error
 * status in its result. */
wf_status wf_server_submit(wf_server s, const wf_request *req);
/* Completed results, oldest first: up to cap are moved to out.  poll returns
 * at once; wait blocks until at least one is available or timeout_s passes.
 * Return value: the number written. */
int wf_server_poll(wf_server s, wf_result *out, int cap);
int wf_server_wait(wf_server s, wf_result *out, int cap, double timeout_s);
wf_status wf_server_get_stats(wf_server s, wf_server_stats *st);
/* Stops the workers after the solves in flight; queued requests are dropped
 * (their buffers are no longer touched).  Destroys the pooled plans. */
void wf_server_destroy(wf_server s);

#ifdef __cplusplus
}
#endif

#endif /* WF_H */
