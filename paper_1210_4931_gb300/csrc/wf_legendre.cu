// Associated-Legendre part of the spherical-harmonic basis change (the
// expensive half of "change the basis" in Sect. 2.1; O(nside lmax^2) per
// transform, Sect. 3) and the harmonic-space blend of Eq. (4), fused into
// the analysis epilogue.
//
//   synthesis  G_m(theta_r) = sum_{l=m..L} a_lm lambda_lm(cos theta_r)
//   analysis   b_lm = sum_r lambda_lm(cos theta_r) F_m(theta_r)
//              a_new = S_l / (S_l + lambda tau Omega) * Omega b_lm   (Eq. 4)
//
// North/south ring pairs share lambda up to (-1)^(l-m): synthesis keeps an
// even and an odd partial sum per pair, analysis folds F_N +- F_S before the
// sum.  The recurrence runs in "mu form" (wf_internal.cuh) from per-(m, pair)
// seeds at the first l where |lambda_lm| exceeds 2^-80 (computed in FP64 with
// an explicit binary exponent, since sin^m(theta) underflows FP64 near the
// poles at large m); below that l every term is < 2^-80 and is dropped.
//
// Two precisions:
//   FP64     k_legsyn<double>, k_legana<double,...>: one ring pair per thread.
//   mixed    k_legsyn_mx<NP>, k_legana_mx<NP, CH>: FP32 recurrence and
//            contraction, NP ring pairs per thread (synthesis) or per lane
//            (analysis) in packed f32x2 lanes (__ffma2_rn); NP is the plan's
//            tile choice (4 and 8 by default, or what wf_plan_autotune timed).
//            Near the poles the plain recurrence mu_l = A x mu_{l-1} - mu_{l-2}
//            loses ~1/sin(theta) digits (its two characteristic roots merge
//            at x = 1), so rings with x > 0.4 run the same recurrence in
//            difference form (Reinsch's modification):
//                D_l = D_{l-1} + (B_l - A_l w) mu_{l-1},  mu_l = mu_{l-1} + D_l,
//            w = 1 - x exact from the grid, B_l = A_l - 2 tabulated in FP64.
//            The block l < l_c, where the messenger iteration's contraction
//            margin tau_h / S_l is below the FP32 error, runs through the FP64
//            kernels instead (the FP32 recurrence restarts at l_c from FP64
//            seeds), so the mixed iteration keeps the FP64 iteration's
//            stability on the modes that converge slowest.
#include <climits>
#include <cmath>
#include <cstdio>

#include "wf_internal.cuh"

namespace wf {

namespace {

constexpr double SEED_LOG2_THRESHOLD = -80.0;
// ring pairs per thread (mixed synthesis) and per lane (mixed analysis): the
// plan's tile choice, 4 and 8 unless wf_plan_autotune measured better
constexpr float X_DIFFERENCE_FORM = 0.4f;
constexpr int BIG = INT_MAX / 2;

__host__ __device__ inline long long mbase(int lmax, int m) { return (long long)m * (2 * lmax + 3 - m) / 2; }

// first l of the FP32 range for m < lc: l_c rounded up to the parity of m
__host__ __device__ inline int lcm_of(int lc, int m) { return m + 2 * ((lc - m + 1) / 2); }

// ---------------------------------------------------------------------------
// seeds: one thread per (m, pair), FP64 with a carried binary exponent
// ---------------------------------------------------------------------------
__global__ void k_seeds(int lmax, int npairs, const double *__restrict__ xp, const double *__restrict__ stp,
                        const double *__restrict__ log2c, const double *__restrict__ A,
                        const double *__restrict__ c, int *__restrict__ ls_out, double *__restrict__ s0_out,
                        double *__restrict__ s1_out)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)(lmax + 1) * npairs) return;
    const int m = (int)(idx / npairs);
    const int p = (int)(idx % npairs);
    const double x = xp[p], st = stp[p];
    const long long base = mbase(lmax, m);
    const double lg2 = log2c[m] + (m > 0 ? m * log2(st) : 0.0);
    int E = (int)floor(lg2);
    double u = exp2(lg2 - E);  // mu_m * 2^-E (c_m = 1)
    if (m & 1) u = -u;
    double up = 0.0;           // mu_{l-1} * 2^-E
    double thr = ldexp(1.0, (int)(SEED_LOG2_THRESHOLD) - E);
    int l = m;
    for (;;) {
        if (fabs(c[base + (l - m)] * u) >= thr) break;
        if (l >= lmax) { l = lmax + 1; break; }
        const double un = A[base + (l + 1 - m)] * x * u - up;
        up = u;
        u = un;
        ++l;
        if (fabs(u) > 0x1p+500) {
            u *= 0x1p-500;
            up *= 0x1p-500;
            E += 500;
            thr = ldexp(1.0, (int)(SEED_LOG2_THRESHOLD) - E);
        }
    }
    int ls;
    double s0 = 0.0, s1 = 0.0;
    if (l > lmax) {
        ls = lmax + 1;
    } else if (((l - m) & 1) == 0) {
        ls = l;
        s0 = ldexp(u, E);
        s1 = (l < lmax) ? ldexp(A[base + (l + 1 - m)] * x * u - up, E) : 0.0;
    } else {
        ls = l - 1;
        s0 = ldexp(up, E);
        s1 = ldexp(u, E);
    }
    ls_out[idx] = ls;
    s0_out[idx] = s0;
    s1_out[idx] = s1;
}

// FP32 seeds of the mixed kernels for a given FP64 block l < lc: for m < lc
// the FP32 recurrence starts at max(l_s, lcm) from FP64-accurate values
__global__ void k_restart_seeds(int lmax, int npairs, int lc, const double *__restrict__ xp,
                                const double *__restrict__ A, const int *__restrict__ ls_in,
                                const double *__restrict__ s0_in, const double *__restrict__ s1_in,
                                int *__restrict__ ls_out, float *__restrict__ s0_out, float *__restrict__ s1_out)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)(lmax + 1) * npairs) return;
    const int m = (int)(idx / npairs);
    const int p = (int)(idx % npairs);
    int ls = ls_in[idx];
    double s0 = s0_in[idx], s1 = s1_in[idx];
    if (m < lc && ls <= lmax) {
        const int l1 = lcm_of(lc, m);
        if (ls < l1) {
            if (l1 > lmax) {
                ls = lmax + 1;
                s0 = s1 = 0.0;
            } else {
                const long long base = mbase(lmax, m);
                const double x = xp[p];
                double a = s0, b = s1;  // mu_l, mu_{l+1} at l = ls
                for (int l = ls + 2; l <= l1 + 1 && l <= lmax; ++l) {
                    const double c2 = A[base + (l - m)] * x * b - a;
                    a = b;
                    b = c2;
                }
                // now (a, b) = (mu_{l1}, mu_{l1+1}), or (mu_{lmax-1}, mu_{lmax}) if l1 = lmax
                if (l1 == lmax && ls + 1 < lmax) {
                    s0 = b;
                    s1 = 0.0;
                } else {
                    s0 = a;
                    s1 = b;
                }
                ls = l1;
            }
        }
    }
    ls_out[idx] = ls;
    s0_out[idx] = (float)s0;
    s1_out[idx] = (float)s1;
}

template <typename T>
__global__ void k_to_T(const double *__restrict__ in, T *__restrict__ out, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (T)in[i];
}

// ---------------------------------------------------------------------------
// FP64 synthesis: CTA per (m, block of pairs); thread per pair.
// lcut > 0: the FP64 block of the mixed path, l < lcm_of(lcut, m), output
// into Gout with row stride gstride.
// ---------------------------------------------------------------------------
// TG: element type of the output (FP32 for the FP64 block of the mixed path,
// whose ring pass adds it to the FP32 coefficients in FP32 anyway: converting
// here keeps the 1/64-rate conversions off the ring kernel).
template <typename T, typename TG>
__global__ void __launch_bounds__(LEG_THREADS) k_legsyn(int lmax, int L, int npairs, int lcut,
                                                        const double2 *__restrict__ alm, const T *__restrict__ A,
                                                        const double *__restrict__ c64,
                                                        const int *__restrict__ ls_tab, const T *__restrict__ s0_tab,
                                                        const T *__restrict__ s1_tab, const T *__restrict__ xp,
                                                        cx<TG> *__restrict__ G, int gstride)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m = blockIdx.y;
    const int Lm = lcut > 0 ? min(L, lcm_of(lcut, m) - 1) : L;
    const int nl = Lm - m + 1;
    const long long base = mbase(lmax, m);
    cx<T> *sac = reinterpret_cast<cx<T> *>(smem_raw);
    T *sA = reinterpret_cast<T *>(sac + (nl + 2));
    for (int i = threadIdx.x; i < nl + 2; i += blockDim.x) {
        if (i < nl) {
            const double2 a = alm[base + i];
            const double cc = c64[base + i];
            sac[i] = mk<T>((T)(a.x * cc), (T)(a.y * cc));
            sA[i] = A[base + i];
        } else {
            sac[i] = mk<T>(0, 0);
            sA[i] = 0;
        }
    }
    __syncthreads();
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += gridDim.x * blockDim.x) {
        const size_t sidx = (size_t)m * npairs + p;
        const int ls = ls_tab[sidx];
        T er = 0, ei = 0, orr = 0, oi = 0;
        if (ls <= Lm) {
            const T x = xp[p];
            T mu0 = s0_tab[sidx], mu1 = s1_tab[sidx];
            int i = ls - m;
            cx<T> a0 = sac[i], a1 = sac[i + 1];
            er = a0.x * mu0;
            ei = a0.y * mu0;
            orr = a1.x * mu1;
            oi = a1.y * mu1;
            for (i += 2; i < nl; i += 2) {
                mu0 = fma(sA[i] * x, mu1, -mu0);
                a0 = sac[i];
                er = fma(a0.x, mu0, er);
                ei = fma(a0.y, mu0, ei);
                mu1 = fma(sA[i + 1] * x, mu0, -mu1);
                a1 = sac[i + 1];
                orr = fma(a1.x, mu1, orr);
                oi = fma(a1.y, mu1, oi);
            }
        }
        cx<TG> *g = G + ((size_t)p * gstride + m) * 2;
        g[0] = mk<TG>((TG)(er + orr), (TG)(ei + oi));
        g[1] = mk<TG>((TG)(er - orr), (TG)(ei - oi));
    }
}

// ---------------------------------------------------------------------------
// warp reduce-scatter of CH complex values: lane i ends with the sum over the
// warp of value (i >> (5 - log2 CH)).
// ---------------------------------------------------------------------------
template <typename T, int CH>
__device__ __forceinline__ void warp_reduce_scatter(T (&vr)[CH], T (&vi)[CH], int lane)
{
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        const int off = 16 >> r;
        const int n = CH >> r;
        if (n >= 2) {
            const int half = n / 2;
            const bool up = (lane & off) != 0;
#pragma unroll
            for (int i = 0; i < half; ++i) {
                const T sr = up ? vr[i] : vr[i + half];
                const T kr = up ? vr[i + half] : vr[i];
                const T si = up ? vi[i] : vi[i + half];
                const T ki = up ? vi[i + half] : vi[i];
                vr[i] = kr + __shfl_xor_sync(0xffffffffu, sr, off);
                vi[i] = ki + __shfl_xor_sync(0xffffffffu, si, off);
            }
        } else {
            vr[0] += __shfl_xor_sync(0xffffffffu, vr[0], off);
            vi[0] += __shfl_xor_sync(0xffffffffu, vi[0], off);
        }
    }
}

template <int CH> struct Log2;
template <> struct Log2<8> { static constexpr int v = 3; };
template <> struct Log2<16> { static constexpr int v = 4; };
template <> struct Log2<32> { static constexpr int v = 5; };

__device__ __forceinline__ void block_reduce4(double (&v)[4], double (*red)[LEG_THREADS / 32])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        if (lane == 0) red[k][warp] = v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double x = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x += red[k][w];
            v[k] = x;
        }
    }
}

// Eq. (4) epilogue shared by both precisions: t_hat = Omega (c acc + low),
// a_new = S/(S + lam tau_h) t_hat, chi^2 of a_old, lambda = 1 residual.
// per-l factors of the harmonic blend (Eq. 4) and of the chi^2 / residual sums
__global__ void k_epi_table(int lmax, const double *__restrict__ S, double omega, double lam_tauh, double tauh,
                            double4 *__restrict__ epi)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l > lmax) return;
    const double s = S[l];
    double4 e = make_double4(0.0, 0.0, 0.0, 0.0);
    if (s > 0.0) {
        e.x = omega * s / (s + lam_tauh);
        e.y = 1.0 / s;
        e.z = 1.0 / s + 1.0 / tauh;
        e.w = 1.0;
    }
    epi[l] = e;
}

template <typename ACC>
__device__ __forceinline__ void blend_epilogue(int lmax, int L, int m, long long base, int mode, double omega,
                                               const BlendArgs &ba, const double *__restrict__ c64,
                                               const ACC *acc, const double2 *__restrict__ low, int low_lim,
                                               const double2 *__restrict__ a_old, double2 *__restrict__ out,
                                               double *__restrict__ part, double (*red)[LEG_THREADS / 32])
{
    double chi2 = 0.0, res2 = 0.0, hnew = 0.0, qnew = 0.0;
    const double wm = (m == 0) ? 1.0 : 2.0;
    for (int j = threadIdx.x; j <= lmax - m; j += blockDim.x) {
        const int l = m + j;
        const long long idx = base + j;
        double2 b = make_double2(0.0, 0.0);
        if (l <= L) {
            b.x = c64[idx] * (double)acc[j].x;
            b.y = c64[idx] * (double)acc[j].y;
            if (low && l < low_lim) {
                const double2 q = low[idx];
                b.x += q.x;
                b.y += q.y;
            }
        }
        if (mode == LEG_ADJOINT) {
            out[idx] = b;
        } else {
            // per-l factors tabulated once per launch (no FP64 division per a_lm)
            const double4 e = ba.epi[l];
            const double2 ao = a_old[idx];
            double2 an = make_double2(0.0, 0.0);
            if (l <= L && e.w > 0.0) {
                an.x = e.x * b.x;
                an.y = e.x * b.y;
            }
            if (e.w > 0.0) {
                chi2 += wm * (ao.x * ao.x + ao.y * ao.y) * e.y;
                const double an2 = wm * (an.x * an.x + an.y * an.y) * e.y;
                hnew += an2;
                qnew += an2 * e.y;
                if (ba.want_resid) {
                    const double dx = e.z * (ao.x - an.x), dy = e.z * (ao.y - an.y);
                    res2 += wm * (dx * dx + dy * dy);
                }
            }
            out[idx] = an;
        }
    }
    if (mode == LEG_BLEND) {
        double v[4] = {chi2, res2, hnew, qnew};
        block_reduce4(v, red);
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < 4; ++k) part[4 * m + k] = v[k];
    }
}

// ---------------------------------------------------------------------------
// FP64 analysis: CTA per m; warp per 32 pairs; register chunks of CH values
// of l reduced across the warp, added into FP64 shared accumulators.
// TF is the storage type of F (FP64 plans: double; FP64 block of the mixed
// path: float).
// ---------------------------------------------------------------------------
template <typename T, typename TF, int CH, bool SPLIT>
__global__ void __launch_bounds__(LEG_THREADS) k_legana(int lmax, int L, int npairs, int lcut,
                                                        const cx<TF> *__restrict__ F, const T *__restrict__ A,
                                                        const int *__restrict__ ls_tab, const T *__restrict__ s0_tab,
                                                        const T *__restrict__ s1_tab, const T *__restrict__ xp,
                                                        const double *__restrict__ c64, int mode, double omega,
                                                        BlendArgs ba, const double2 *__restrict__ a_old,
                                                        double2 *__restrict__ out, double *__restrict__ part)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[4][LEG_THREADS / 32];
    const int m = blockIdx.x;
    const int Lm = lcut > 0 ? min(L, lcm_of(lcut, m) - 1) : L;
    const int nl = Lm - m + 1;
    const int nlp = nl + CH + 2;
    const long long base = mbase(lmax, m);
    double2 *acc = reinterpret_cast<double2 *>(smem_raw);
    T *sA = reinterpret_cast<T *>(acc + nlp);
    for (int i = threadIdx.x; i < nlp; i += blockDim.x) {
        acc[i] = make_double2(0.0, 0.0);
        sA[i] = (i < nl) ? A[base + i] : (T)0;
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int ngroups = (npairs + 31) / 32;
    // SPLIT: the ring pairs of one m are shared by gridDim.y CTAs
    const int gpc = SPLIT ? (ngroups + gridDim.y - 1) / gridDim.y : ngroups;
    const int g0 = SPLIT ? blockIdx.y * gpc : 0;
    const int g1 = min(ngroups, g0 + gpc);
    for (int grp = g0 + warp; grp < g1; grp += nwarps) {
        const int p = grp * 32 + lane;
        const size_t sidx = (size_t)m * npairs + p;
        int ls = (p < npairs) ? ls_tab[sidx] : BIG;
        if (ls > Lm) ls = BIG;
        const int lmin = __reduce_min_sync(0xffffffffu, ls);
        if (lmin > Lm) continue;
        cx<T> FE = mk<T>(0, 0), FO = mk<T>(0, 0);
        T x = 0, s0 = 0, s1 = 0;
        if (ls <= Lm) {
            const cx<TF> *f = F + ((size_t)p * (lmax + 1) + m) * 2;
            const cx<TF> fn = f[0], fs = f[1];
            FE = mk<T>((T)fn.x + (T)fs.x, (T)fn.y + (T)fs.y);
            FO = mk<T>((T)fn.x - (T)fs.x, (T)fn.y - (T)fs.y);
            x = xp[p];
            s0 = s0_tab[sidx];
            s1 = s1_tab[sidx];
        }
        T mua = 0, mub = 0;
        for (int l0 = lmin; l0 <= Lm; l0 += CH) {
            T vr[CH], vi[CH];
#pragma unroll
            for (int i = 0; i < CH; i += 2) {
                const int j = l0 - m + i;
                T v0 = fma(sA[j] * x, mub, -mua);
                T v1 = fma(sA[j + 1] * x, v0, -mub);
                if (l0 + i == ls) { v0 = s0; v1 = s1; }
                vr[i] = v0 * FE.x;
                vi[i] = v0 * FE.y;
                vr[i + 1] = v1 * FO.x;
                vi[i + 1] = v1 * FO.y;
                mua = v0;
                mub = v1;
            }
            warp_reduce_scatter<T, CH>(vr, vi, lane);
            constexpr int sh = 5 - Log2<CH>::v;
            if ((lane & ((1 << sh) - 1)) == 0) {
                const int l = l0 + (lane >> sh);
                if (l <= Lm) {
                    atomicAdd(&acc[l - m].x, (double)vr[0]);
                    atomicAdd(&acc[l - m].y, (double)vi[0]);
                }
            }
        }
    }
    __syncthreads();
    if (SPLIT) {  // adjoint only: add this CTA's share into the (zeroed) output
        for (int j = threadIdx.x; j < nl; j += blockDim.x) {
            const double cc = c64[base + j];
            atomicAdd(&out[base + j].x, cc * acc[j].x);
            atomicAdd(&out[base + j].y, cc * acc[j].y);
        }
        return;
    }
    blend_epilogue(lmax, Lm, m, base, mode, omega, ba, c64, acc, nullptr, 0, a_old, out, part, red);
}

// ---------------------------------------------------------------------------
// FP64 block of the mixed path from a table.  The block (m < l_c,
// m <= l < lcm(l_c, m)) holds few (l, m) but every ring pair, and GB300 runs
// FP64 at 1/64 of the FP32 rate, so the FP64 recurrence kernels above spend
// more time on it than the FP32 kernels spend on a far larger share of the
// band.  Here lambda_lm(x_p) is computed once per l_c by the FP64 recurrence
// and stored as a pair of FP32 numbers (hi, lo) with hi + lo = lambda to 48
// significant bits; both directions then stream the table and accumulate in
// double-float arithmetic on the FP32 pipe: products split exactly with an
// FMA (Dekker's product) and sums with Knuth's two-sum, so each term carries
// about 2^-46 relative error against 2^-53 in FP64, far below the FP32
// operator error the block exists to avoid.
// Layout: row r = rowoff[m] + (l - m), column p (ring pair), row stride
// np_pad (npairs rounded up to 32; padding columns hold zeros).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (shi, slo) += (xh + xl)(yh + yl), dropping only the xl yl term (2^-48 relative)
__device__ __forceinline__ void df_fma(float &shi, float &slo, float xh, float xl, float yh, float yl)
{
    const float p = __fmul_rn(xh, yh);
    float e = __fmaf_rn(xh, yh, -p);  // xh yh - p exactly
    e = __fmaf_rn(xh, yl, e);
    e = __fmaf_rn(xl, yh, e);
    float s, t;
    two_sum(shi, p, s, t);
    shi = s;
    slo = __fadd_rn(slo, __fadd_rn(t, e));
}

// (ahi, alo) += (bhi, blo)
__device__ __forceinline__ void df_add(float &ahi, float &alo, float bhi, float blo)
{
    float s, e;
    two_sum(ahi, bhi, s, e);
    ahi = s;
    alo = __fadd_rn(alo, __fadd_rn(e, blo));
}

// FP64 value split into (hi, lo) floats
__device__ __forceinline__ float2 df_split(double v)
{
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

__host__ __device__ inline int low_rows(int lmax, int lc, int m) { return min(lcm_of(lc, m), lmax + 1) - m; }

// one thread per (m, column): the FP64 recurrence from the plan's FP64 seeds
__global__ void k_lowtab_build(int lmax, int npairs, int np_pad, int lc, const long long *__restrict__ rowoff,
                               const double *__restrict__ A, const double *__restrict__ c,
                               const int *__restrict__ ls_tab, const double *__restrict__ s0_tab,
                               const double *__restrict__ s1_tab, const double *__restrict__ xp,
                               float2 *__restrict__ tab)
{
    const int m = blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np_pad) return;
    const int nr = low_rows(lmax, lc, m);
    const long long base = mbase(lmax, m);
    const size_t sidx = (size_t)m * npairs + p;
    const int ls = (p < npairs) ? ls_tab[sidx] : BIG;
    const double x = (p < npairs) ? xp[p] : 0.0;
    float2 *col = tab + (size_t)rowoff[m] * np_pad + p;
    double mu2 = 0.0, mu1 = 0.0;  // mu_{l-2}, mu_{l-1}
    for (int i = 0; i < nr; ++i) {
        const int l = m + i;
        double mu = 0.0;
        if (l == ls) mu = s0_tab[sidx];
        else if (l == ls + 1) mu = s1_tab[sidx];
        else if (l > ls + 1) mu = A[base + i] * x * mu1 - mu2;
        mu2 = mu1;
        mu1 = mu;
        col[(size_t)i * np_pad] = df_split(c[base + i] * mu);
    }
}

// synthesis: G_m(theta_p) = sum over the block's l <= L of a_lm lambda_lm, as even and
// odd partial sums (north = E + O, south = E - O), rounded to FP32 into the block's
// [pair][m][hemisphere] layout (row stride gstride)
__global__ void __launch_bounds__(LEG_THREADS) k_lowsyn_df(int lmax, int L, int npairs, int np_pad, int lc,
                                                           const long long *__restrict__ rowoff,
                                                           const float2 *__restrict__ tab,
                                                           const double2 *__restrict__ alm, float2 *__restrict__ G,
                                                           int gstride)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *sa = reinterpret_cast<float4 *>(smem_raw);  // a_lm as (re hi, re lo, im hi, im lo)
    const int m = blockIdx.y;
    const int nr = min(low_rows(lmax, lc, m), L - m + 1);
    const long long base = mbase(lmax, m);
    for (int i = threadIdx.x; i < nr + 1; i += blockDim.x) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < nr) {
            const double2 a = alm[base + i];
            const float2 re = df_split(a.x), im = df_split(a.y);
            v = make_float4(re.x, re.y, im.x, im.y);
        }
        sa[i] = v;
    }
    __syncthreads();
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += gridDim.x * blockDim.x) {
        const float2 *col = tab + (size_t)rowoff[m] * np_pad + p;
        float erh = 0.f, erl = 0.f, eih = 0.f, eil = 0.f, orh = 0.f, orl = 0.f, oih = 0.f, oil = 0.f;
        for (int i = 0; i < nr; i += 2) {  // sa[nr] is zero, so an odd nr needs no tail
            const float2 t0 = col[(size_t)i * np_pad];
            const float2 t1 = (i + 1 < nr) ? col[(size_t)(i + 1) * np_pad] : make_float2(0.f, 0.f);
            const float4 a0 = sa[i], a1 = sa[i + 1];
            df_fma(erh, erl, t0.x, t0.y, a0.x, a0.y);
            df_fma(eih, eil, t0.x, t0.y, a0.z, a0.w);
            df_fma(orh, orl, t1.x, t1.y, a1.x, a1.y);
            df_fma(oih, oil, t1.x, t1.y, a1.z, a1.w);
        }
        float nrh = erh, nrl = erl, nih = eih, nil = eil;  // E + O
        df_add(nrh, nrl, orh, orl);
        df_add(nih, nil, oih, oil);
        float srh = erh, srl = erl, sih = eih, sil = eil;  // E - O
        df_add(srh, srl, -orh, -orl);
        df_add(sih, sil, -oih, -oil);
        float2 *g = G + ((size_t)p * gstride + m) * 2;
        g[0] = make_float2(nrh + nrl, nih + nil);
        g[1] = make_float2(srh + srl, sih + sil);
    }
}

// analysis: b_lm = sum_p lambda_lm(x_p) (F_N +- F_S)(p) for the block's l <= L (sign
// + for even l - m).  CTA = (rows of one parity of one m, LOWANA_ROWS at most): it
// stages F_N +- F_S exactly as double-float for every pair in shared memory, each
// warp then takes LOWANA_RW rows at a time, lanes over pairs, and reduces across
// the warp.
constexpr int LOWANA_ROWS = 32, LOWANA_RW = 4;

__global__ void __launch_bounds__(LEG_THREADS) k_lowana_df(int lmax, int L, int npairs, int np_pad, int lc,
                                                           const long long *__restrict__ rowoff,
                                                           const float2 *__restrict__ tab,
                                                           const float2 *__restrict__ F, double2 *__restrict__ out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *sf = reinterpret_cast<float4 *>(smem_raw);  // F_N +- F_S as (re hi, re lo, im hi, im lo)
    const int m = blockIdx.z, parity = blockIdx.y;
    const int nr = min(low_rows(lmax, lc, m), L - m + 1);
    const int npar = (nr - parity + 1) / 2;  // rows i = parity + 2 k, k < npar
    const int k0 = blockIdx.x * LOWANA_ROWS;
    if (k0 >= npar) return;
    const int k1 = min(npar, k0 + LOWANA_ROWS);
    const size_t pstride = (size_t)(lmax + 1) * 2;
    const float sg = parity ? -1.f : 1.f;
#pragma unroll 4
    for (int p = threadIdx.x; p < np_pad; p += blockDim.x) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (p < npairs) {
            const float2 *f = F + (size_t)p * pstride + 2 * (size_t)m;
            const float2 fn = f[0], fs = f[1];
            float rh, rl, ih, il;
            two_sum(fn.x, sg * fs.x, rh, rl);
            two_sum(fn.y, sg * fs.y, ih, il);
            v = make_float4(rh, rl, ih, il);
        }
        sf[p] = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const long long base = mbase(lmax, m);
    const float2 *rows = tab + (size_t)rowoff[m] * np_pad;
    // LOWANA_RW rows of this parity per warp and pass: one shared F value feeds all of
    // them, and the unrolled pair loop keeps several table loads in flight per lane
    for (int k = k0 + LOWANA_RW * warp; k < k1; k += LOWANA_RW * nwarps) {
        const float2 *r[LOWANA_RW];
        float acc[LOWANA_RW][4];
#pragma unroll
        for (int q = 0; q < LOWANA_RW; ++q) {
            const int kq = min(k + q, k1 - 1);  // rows past k1 repeat the last one, unwritten
            r[q] = rows + (size_t)(parity + 2 * kq) * np_pad;
            acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
        }
#pragma unroll 4
        for (int p = lane; p < np_pad; p += 32) {
            const float4 f = sf[p];
#pragma unroll
            for (int q = 0; q < LOWANA_RW; ++q) {
                const float2 t = r[q][p];
                df_fma(acc[q][0], acc[q][1], t.x, t.y, f.x, f.y);
                df_fma(acc[q][2], acc[q][3], t.x, t.y, f.z, f.w);
            }
        }
#pragma unroll
        for (int q = 0; q < LOWANA_RW; ++q) {
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                const float a = __shfl_xor_sync(0xffffffffu, acc[q][0], o), b = __shfl_xor_sync(0xffffffffu, acc[q][1], o);
                const float c = __shfl_xor_sync(0xffffffffu, acc[q][2], o), d = __shfl_xor_sync(0xffffffffu, acc[q][3], o);
                df_add(acc[q][0], acc[q][1], a, b);
                df_add(acc[q][2], acc[q][3], c, d);
            }
            if (lane == 0 && k + q < k1)
                out[base + parity + 2 * (k + q)] =
                    make_double2((double)acc[q][0] + (double)acc[q][1], (double)acc[q][2] + (double)acc[q][3]);
        }
    }
}

// ---------------------------------------------------------------------------
// Double-float transforms for the FP64 correction sweeps of mixed plans.  The
// sweeps' FP64 plan ran these transforms at the FP64 rate (1/64 of FP32 on
// GB300): three FP64 synthesis/analysis pairs per solve cost about a tenth of
// a 1000-iteration benchmark solve.  Here the recurrence, the seeds, x, A and
// c a_lm are (hi, lo) float pairs and every product and sum is an error-free
// FP32 transformation (Dekker's product via FMA, Knuth's two-sum): about 48
// significant bits, against the 24 of the mixed kernels that the sweeps
// correct.  Near the poles the plain recurrence loses ~log2(1/sin theta) bits
// in any precision (12 at nside 2048), so the sweeps stay ~10 digits accurate.
// ---------------------------------------------------------------------------
// Cross-lane sum of one chunk (CH = 8) through shared memory: lane w stores its
// (AR.x, AR.y, AI.x, AI.y) for each row i of the chunk; lane (i, q) = (lane / 4,
// lane % 4) then adds the eight stores of lanes 8q..8q+7 for row i, and two shuffles
// combine the four quarters.  Per chunk that is 8 stores, 8 loads, 16 packed adds
// and 4 shuffles per lane against 16 adds, 18 shuffles, 18 adds and 28 selects for
// the shuffle reduce-scatter.  Slots are XOR-swizzled so that both the stores (8
// lanes of one q) and the loads (8 lanes over two rows and four q) of each
// 128-byte phase hit distinct bank groups.
__device__ __forceinline__ int stage_slot(int i, int w)
{
    const int q = w >> 3, j = w & 7;
    return 32 * i + 8 * q + (j ^ (q + 4 * (i & 1)));
}

// (ph, pl) ~ (ah + al)(bh + bl), unnormalised (|pl| ~ 2^-23 |ph|)
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float &ph, float &pl)
{
    ph = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -ph);
    e = __fmaf_rn(ah, bl, e);
    pl = __fmaf_rn(al, bh, e);
}

// (sh, sl) = (ah + al) - (bh + bl), normalised
__device__ __forceinline__ void df_sub(float ah, float al, float bh, float bl, float &sh, float &sl)
{
    float s, e;
    two_sum(ah, -bh, s, e);
    e = __fadd_rn(e, __fsub_rn(al, bl));
    sh = __fadd_rn(s, e);
    sl = __fsub_rn(e, __fsub_rn(sh, s));
}

// one recurrence step mu_l = A_l x mu_{l-1} - mu_{l-2} in double-float
__device__ __forceinline__ void df_step(float2 Al, float xh, float xl, float m1h, float m1l, float &m0h, float &m0l)
{
    float th, tl, uh, ul;
    df_mul(Al.x, Al.y, xh, xl, th, tl);
    df_mul(th, tl, m1h, m1l, uh, ul);
    df_sub(uh, ul, m0h, m0l, m0h, m0l);
}

__device__ __forceinline__ double df_val(float h, float l) { return (double)h + (double)l; }

// synthesis: CTA per (m, block of pairs), thread per pair, as the FP64 kernel
__global__ void __launch_bounds__(LEG_THREADS) k_legsyn_df(int lmax, int L, int npairs,
                                                           const double2 *__restrict__ alm, const double *__restrict__ A,
                                                           const double *__restrict__ c64,
                                                           const int *__restrict__ ls_tab,
                                                           const double *__restrict__ s0_tab,
                                                           const double *__restrict__ s1_tab,
                                                           const double *__restrict__ xp, double2 *__restrict__ G)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m = blockIdx.y;
    const int nl = L - m + 1;
    const long long base = mbase(lmax, m);
    float4 *sac = reinterpret_cast<float4 *>(smem_raw);  // c a_lm as (re hi, re lo, im hi, im lo)
    float2 *sA = reinterpret_cast<float2 *>(sac + (nl + 2));
    for (int i = threadIdx.x; i < nl + 2; i += blockDim.x) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 a = make_float2(0.f, 0.f);
        if (i < nl) {
            const double2 q = alm[base + i];
            const double cc = c64[base + i];
            const float2 re = df_split(q.x * cc), im = df_split(q.y * cc);
            v = make_float4(re.x, re.y, im.x, im.y);
            a = df_split(A[base + i]);
        }
        sac[i] = v;
        sA[i] = a;
    }
    __syncthreads();
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += gridDim.x * blockDim.x) {
        const size_t sidx = (size_t)m * npairs + p;
        const int ls = ls_tab[sidx];
        float erh = 0.f, erl = 0.f, eih = 0.f, eil = 0.f, orh = 0.f, orl = 0.f, oih = 0.f, oil = 0.f;
        if (ls <= L) {
            const float2 x = df_split(xp[p]), s0 = df_split(s0_tab[sidx]), s1 = df_split(s1_tab[sidx]);
            float m0h = s0.x, m0l = s0.y, m1h = s1.x, m1l = s1.y;
            int i = ls - m;
            float4 a0 = sac[i], a1 = sac[i + 1];
            df_fma(erh, erl, a0.x, a0.y, m0h, m0l);
            df_fma(eih, eil, a0.z, a0.w, m0h, m0l);
            df_fma(orh, orl, a1.x, a1.y, m1h, m1l);
            df_fma(oih, oil, a1.z, a1.w, m1h, m1l);
            for (i += 2; i < nl; i += 2) {
                df_step(sA[i], x.x, x.y, m1h, m1l, m0h, m0l);
                a0 = sac[i];
                df_fma(erh, erl, a0.x, a0.y, m0h, m0l);
                df_fma(eih, eil, a0.z, a0.w, m0h, m0l);
                df_step(sA[i + 1], x.x, x.y, m0h, m0l, m1h, m1l);
                a1 = sac[i + 1];
                df_fma(orh, orl, a1.x, a1.y, m1h, m1l);
                df_fma(oih, oil, a1.z, a1.w, m1h, m1l);
            }
        }
        const double er = df_val(erh, erl), ei = df_val(eih, eil), orr = df_val(orh, orl), oi = df_val(oih, oil);
        double2 *g = G + ((size_t)p * (lmax + 1) + m) * 2;
        g[0] = make_double2(er + orr, ei + oi);
        g[1] = make_double2(er - orr, ei - oi);
    }
}

// analysis: CTA per m; a warp covers 32 lanes x DFP ring pairs taken dynamically,
// equator first; chunks of 8 values of l are summed over the lane's pairs in
// double-float, across the warp through a swizzled shared stage (as in the mixed
// analysis, with (hi, lo) of the real and imaginary parts per slot and double-float
// additions), and added into FP64 shared accumulators.
constexpr int DFP = 4;

template <bool INJ>
__device__ __forceinline__ void df_ana_pair_step(int l, const int (&ls)[DFP], const float2 (&s0)[DFP],
                                                 const float2 (&s1)[DFP], const float2 (&x)[DFP], float2 A0, float2 A1,
                                                 float2 (&m0)[DFP], float2 (&m1)[DFP])
{
#pragma unroll
    for (int k = 0; k < DFP; ++k) {
        df_step(A0, x[k].x, x[k].y, m1[k].x, m1[k].y, m0[k].x, m0[k].y);
        df_step(A1, x[k].x, x[k].y, m0[k].x, m0[k].y, m1[k].x, m1[k].y);
        if (INJ && l == ls[k]) {
            m0[k] = s0[k];
            m1[k] = s1[k];
        }
    }
}

__global__ void __launch_bounds__(LEG_THREADS, 2) k_legana_df(int lmax, int L, int npairs,
                                                           const double2 *__restrict__ F, const double *__restrict__ A,
                                                           const int *__restrict__ ls_tab,
                                                           const double *__restrict__ s0_tab,
                                                           const double *__restrict__ s1_tab,
                                                           const double *__restrict__ xp,
                                                           const double *__restrict__ c64, int mode, double omega,
                                                           BlendArgs ba, const double2 *__restrict__ a_old,
                                                           double2 *__restrict__ out, double *__restrict__ part)
{
    constexpr int CH = 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[4][LEG_THREADS / 32];
    __shared__ int next_group;
    const int m = blockIdx.x;
    const int nl = L - m + 1;
    const int nlp = nl + CH + 2;
    const long long base = mbase(lmax, m);
    double2 *acc = reinterpret_cast<double2 *>(smem_raw);
    float4 *sAA = reinterpret_cast<float4 *>(acc + nlp);   // (A_l hi, lo, A_l+1 hi, lo) from l - m = 0, even
    float4 *stage = sAA + (nlp + 1) / 2;                      // per warp: 8 rows x 32 lanes of (re hi, lo, im hi, lo)
    for (int i = threadIdx.x; i < nlp; i += blockDim.x) acc[i] = make_double2(0.0, 0.0);
    for (int i = threadIdx.x; i < (nlp + 1) / 2; i += blockDim.x) {
        const int j = 2 * i;
        const float2 a0 = j < nl ? df_split(A[base + j]) : make_float2(0.f, 0.f);
        const float2 a1 = j + 1 < nl ? df_split(A[base + j + 1]) : make_float2(0.f, 0.f);
        sAA[i] = make_float4(a0.x, a0.y, a1.x, a1.y);
    }
    if (threadIdx.x == 0) next_group = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    float4 *wst = stage + (threadIdx.x >> 5) * 256;
    const int per_group = 32 * DFP;
    const int ngroups = (npairs + per_group - 1) / per_group;
    const size_t pstride = (size_t)(lmax + 1) * 2;
    for (;;) {
        int grp = 0;
        if (lane == 0) grp = atomicAdd(&next_group, 1);
        grp = __shfl_sync(0xffffffffu, grp, 0);
        if (grp >= ngroups) break;
        const int p0 = (ngroups - 1 - grp) * per_group + lane * DFP;
        int ls[DFP];
        float2 s0[DFP], s1[DFP], x[DFP], m0[DFP], m1[DFP], fer[DFP], fei[DFP], forr[DFP], foi[DFP];
        int lmin = BIG, lmaxs = -1;
#pragma unroll
        for (int k = 0; k < DFP; ++k) {
            const int p = p0 + k;
            ls[k] = BIG;
            s0[k] = s1[k] = x[k] = m0[k] = m1[k] = make_float2(0.f, 0.f);
            fer[k] = fei[k] = forr[k] = foi[k] = make_float2(0.f, 0.f);
            if (p < npairs) {
                const size_t sidx = (size_t)m * npairs + p;
                const int l0 = ls_tab[sidx];
                if (l0 <= L) {
                    ls[k] = l0;
                    s0[k] = df_split(s0_tab[sidx]);
                    s1[k] = df_split(s1_tab[sidx]);
                    x[k] = df_split(xp[p]);
                    const double2 *f = F + (size_t)p * pstride + 2 * (size_t)m;
                    const double2 fn = f[0], fs = f[1];
                    fer[k] = df_split(fn.x + fs.x);
                    fei[k] = df_split(fn.y + fs.y);
                    forr[k] = df_split(fn.x - fs.x);
                    foi[k] = df_split(fn.y - fs.y);
                    lmin = min(lmin, l0);
                    lmaxs = max(lmaxs, l0);
                }
            }
        }
        const int lmin_w = __reduce_min_sync(0xffffffffu, lmin);
        const int lmaxs_w = __reduce_max_sync(0xffffffffu, lmaxs);
        if (lmin_w > L) continue;
        for (int l0 = lmin_w; l0 <= L; l0 += CH) {
            const bool inj = l0 <= lmaxs_w;
#pragma unroll
            for (int i = 0; i < CH; i += 2) {
                const float4 aa = sAA[(l0 - m + i) >> 1];  // l0 - m is even
                if (inj) df_ana_pair_step<true>(l0 + i, ls, s0, s1, x, make_float2(aa.x, aa.y), make_float2(aa.z, aa.w), m0, m1);
                else df_ana_pair_step<false>(l0 + i, ls, s0, s1, x, make_float2(aa.x, aa.y), make_float2(aa.z, aa.w), m0, m1);
                float r0h = 0.f, r0l = 0.f, i0h = 0.f, i0l = 0.f, r1h = 0.f, r1l = 0.f, i1h = 0.f, i1l = 0.f;
#pragma unroll
                for (int k = 0; k < DFP; ++k) {
                    df_fma(r0h, r0l, fer[k].x, fer[k].y, m0[k].x, m0[k].y);
                    df_fma(i0h, i0l, fei[k].x, fei[k].y, m0[k].x, m0[k].y);
                    df_fma(r1h, r1l, forr[k].x, forr[k].y, m1[k].x, m1[k].y);
                    df_fma(i1h, i1l, foi[k].x, foi[k].y, m1[k].x, m1[k].y);
                }
                wst[stage_slot(i, lane)] = make_float4(r0h, r0l, i0h, i0l);
                wst[stage_slot(i + 1, lane)] = make_float4(r1h, r1l, i1h, i1l);
            }
            __syncwarp();
            {
                const int i = lane >> 2, q = lane & 3;
                const float4 *row = wst + 32 * i + 8 * q;
                const int c = q + 4 * (i & 1);
                float4 v = row[c];
                float rh = v.x, rl = v.y, ih = v.z, il = v.w;
#pragma unroll
                for (int j = 1; j < 8; ++j) {
                    v = row[j ^ c];
                    df_add(rh, rl, v.x, v.y);
                    df_add(ih, il, v.z, v.w);
                }
#pragma unroll
                for (int o = 1; o <= 2; o <<= 1) {
                    const float a = __shfl_xor_sync(0xffffffffu, rh, o), b = __shfl_xor_sync(0xffffffffu, rl, o);
                    const float cc = __shfl_xor_sync(0xffffffffu, ih, o), d = __shfl_xor_sync(0xffffffffu, il, o);
                    df_add(rh, rl, a, b);
                    df_add(ih, il, cc, d);
                }
                if (q == 0) {
                    const int l = l0 + i;
                    if (l <= L) {
                        atomicAdd(&acc[l - m].x, df_val(rh, rl));
                        atomicAdd(&acc[l - m].y, df_val(ih, il));
                    }
                }
            }
            __syncwarp();
        }
    }
    __syncthreads();
    blend_epilogue(lmax, L, m, base, mode, omega, ba, c64, acc, nullptr, 0, a_old, out, part, red);
}

// ---------------------------------------------------------------------------
// mixed precision: FP32 kernels, four ring pairs per thread in two f32x2
// packs, plain or difference-form recurrence by ring
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 dup(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float get(const float2 &v, int k) { return k ? v.y : v.x; }
__device__ __forceinline__ void put(float2 &v, int k, float a)
{
    if (k) v.y = a;
    else v.x = a;
}

template <int NP> struct MxPairs {
    static constexpr int NPK = NP / 2;
    int ls[NP];
    float s0[NP], s1[NP];
    float2 X[NP / 2], W[NP / 2];
    int lmin, lmaxs;
    bool diff;
};

template <int NP>
__device__ __forceinline__ void mx_load_pairs(MxPairs<NP> &P, int m, int L, int npairs, int p0,
                                              const int *__restrict__ ls_tab, const float *__restrict__ s0_tab,
                                              const float *__restrict__ s1_tab, const float *__restrict__ xp,
                                              const float *__restrict__ wp)
{
    P.lmin = BIG;
    P.lmaxs = -1;
    float xs[NP], ws[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int p = p0 + k;
        int ls = BIG;
        float s0 = 0.f, s1 = 0.f, x = 0.f, w = 1.f;
        if (p < npairs) {
            const size_t sidx = (size_t)m * npairs + p;
            ls = ls_tab[sidx];
            if (ls > L) ls = BIG;
            else {
                s0 = s0_tab[sidx];
                s1 = s1_tab[sidx];
            }
            x = xp[p];
            w = wp[p];
        }
        P.ls[k] = ls;
        P.s0[k] = s0;
        P.s1[k] = s1;
        xs[k] = x;
        ws[k] = w;
        if (ls < P.lmin) P.lmin = ls;
        if (ls != BIG && ls > P.lmaxs) P.lmaxs = ls;
    }
#pragma unroll
    for (int pk = 0; pk < NP / 2; ++pk) {
        P.X[pk] = make_float2(xs[2 * pk], xs[2 * pk + 1]);
        P.W[pk] = make_float2(ws[2 * pk], ws[2 * pk + 1]);
    }
    P.diff = xs[0] > X_DIFFERENCE_FORM;
}

// one double step (l, l+1) of the recurrence for both packs.
// plain state: (Sa, Sb) = (mu_{l-2}, mu_{l-1}); difference state: (Sa, Sb) =
// (D_{l-1}, mu_{l-1}).  Outputs mu_l (V0) and mu_{l+1} (V1).
template <bool DIFF, bool INJECT, int NP>
__device__ __forceinline__ void mx_step(const MxPairs<NP> &P, int l, float A0, float B0, float A1, float B1,
                                        float2 (&Sa)[NP / 2], float2 (&Sb)[NP / 2], float2 (&V0)[NP / 2],
                                        float2 (&V1)[NP / 2])
{
#pragma unroll
    for (int pk = 0; pk < NP / 2; ++pk) {
        if (DIFF) {
            float2 D = Sa[pk], mu = Sb[pk];
            D = __ffma2_rn(__ffma2_rn(dup(-A0), P.W[pk], dup(B0)), mu, D);
            const float2 v0 = __fadd2_rn(mu, D);
            D = __ffma2_rn(__ffma2_rn(dup(-A1), P.W[pk], dup(B1)), v0, D);
            const float2 v1 = __fadd2_rn(v0, D);
            V0[pk] = v0;
            V1[pk] = v1;
            Sa[pk] = D;
            Sb[pk] = v1;
        } else {
            const float2 v0 = __ffma2_rn(__fmul2_rn(dup(A0), P.X[pk]), Sb[pk], neg2(Sa[pk]));
            const float2 v1 = __ffma2_rn(__fmul2_rn(dup(A1), P.X[pk]), v0, neg2(Sb[pk]));
            V0[pk] = v0;
            V1[pk] = v1;
            Sa[pk] = v0;
            Sb[pk] = v1;
        }
        if (INJECT) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = 2 * pk + h;
                if (l == P.ls[k]) {
                    put(V0[pk], h, P.s0[k]);
                    put(V1[pk], h, P.s1[k]);
                    if (DIFF) {
                        put(Sa[pk], h, P.s1[k] - P.s0[k]);
                        put(Sb[pk], h, P.s1[k]);
                    } else {
                        put(Sa[pk], h, P.s0[k]);
                        put(Sb[pk], h, P.s1[k]);
                    }
                }
            }
        }
    }
}

// lmin, lmaxs: the warp's smallest first l and largest seeding l, so that the
// warp runs one loop with one trip count (lanes not yet started add zeros)
template <bool DIFF, int NP>
__device__ __forceinline__ void mx_syn_run(const MxPairs<NP> &P, int m, int L, const float4 *__restrict__ sAB,
                                           const float4 *__restrict__ sac, float2 (&ER)[NP / 2],
                                           float2 (&EI)[NP / 2], float2 (&OR)[NP / 2], float2 (&OI)[NP / 2],
                                           int lmin, int lmaxs)
{
    float2 Sa[NP / 2], Sb[NP / 2], V0[NP / 2], V1[NP / 2];
#pragma unroll
    for (int pk = 0; pk < NP / 2; ++pk) Sa[pk] = Sb[pk] = dup(0.f);
    int l = lmin;
    for (; l <= L && l <= lmaxs; l += 2) {
        const int j = (l - m) >> 1;
        const float4 ab = sAB[j], ac = sac[j];
        mx_step<DIFF, true, NP>(P, l, ab.x, ab.y, ab.z, ab.w, Sa, Sb, V0, V1);
#pragma unroll
        for (int pk = 0; pk < NP / 2; ++pk) {
            ER[pk] = __ffma2_rn(dup(ac.x), V0[pk], ER[pk]);
            EI[pk] = __ffma2_rn(dup(ac.y), V0[pk], EI[pk]);
            OR[pk] = __ffma2_rn(dup(ac.z), V1[pk], OR[pk]);
            OI[pk] = __ffma2_rn(dup(ac.w), V1[pk], OI[pk]);
        }
    }
    for (; l <= L; l += 2) {
        const int j = (l - m) >> 1;
        const float4 ab = sAB[j], ac = sac[j];
        mx_step<DIFF, false, NP>(P, l, ab.x, ab.y, ab.z, ab.w, Sa, Sb, V0, V1);
#pragma unroll
        for (int pk = 0; pk < NP / 2; ++pk) {
            ER[pk] = __ffma2_rn(dup(ac.x), V0[pk], ER[pk]);
            EI[pk] = __ffma2_rn(dup(ac.y), V0[pk], EI[pk]);
            OR[pk] = __ffma2_rn(dup(ac.z), V1[pk], OR[pk]);
            OI[pk] = __ffma2_rn(dup(ac.w), V1[pk], OI[pk]);
        }
    }
}

// shared-memory staging: per pair of l (l = m + 2j, l + 1):
//   sAB[j] = (A_l, B_l, A_{l+1}, B_{l+1}),  sac[j] = (Re a'_l, Im a'_l, Re a'_{l+1}, Im a'_{l+1})
template <int NP>
__global__ void __launch_bounds__(LEG_THREADS) k_legsyn_mx(int lmax, int L, int npairs,
                                                           const double2 *__restrict__ alm,
                                                           const float *__restrict__ A, const float *__restrict__ B,
                                                           const double *__restrict__ c64,
                                                           const int *__restrict__ ls_tab,
                                                           const float *__restrict__ s0_tab,
                                                           const float *__restrict__ s1_tab,
                                                           const float *__restrict__ xp, const float *__restrict__ wp,
                                                           float2 *__restrict__ G)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m = blockIdx.y;
    const int nl = L - m + 1;
    const int nj = (nl + 1) / 2 + 1;
    const long long base = mbase(lmax, m);
    float4 *sAB = reinterpret_cast<float4 *>(smem_raw);
    float4 *sac = sAB + nj;
    for (int j = threadIdx.x; j < nj; j += blockDim.x) {
        float4 ab = make_float4(0.f, 0.f, 0.f, 0.f), ac = make_float4(0.f, 0.f, 0.f, 0.f);
        const int i0 = 2 * j, i1 = 2 * j + 1;
        if (i0 < nl) {
            const double2 a = alm[base + i0];
            const double cc = c64[base + i0];
            ab.x = A[base + i0];
            ab.y = B[base + i0];
            ac.x = (float)(a.x * cc);
            ac.y = (float)(a.y * cc);
        }
        if (i1 < nl) {
            const double2 a = alm[base + i1];
            const double cc = c64[base + i1];
            ab.z = A[base + i1];
            ab.w = B[base + i1];
            ac.z = (float)(a.x * cc);
            ac.w = (float)(a.y * cc);
        }
        sAB[j] = ab;
        sac[j] = ac;
    }
    __syncthreads();
    const size_t pstride = (size_t)(lmax + 1) * 2;
    for (int p0 = (blockIdx.x * blockDim.x + threadIdx.x) * NP; p0 < npairs; p0 += gridDim.x * blockDim.x * NP) {
        MxPairs<NP> P;
        mx_load_pairs<NP>(P, m, L, npairs, p0, ls_tab, s0_tab, s1_tab, xp, wp);
        float2 ER[NP / 2], EI[NP / 2], OR[NP / 2], OI[NP / 2];
#pragma unroll
        for (int pk = 0; pk < NP / 2; ++pk) ER[pk] = EI[pk] = OR[pk] = OI[pk] = dup(0.f);
        // warp-uniform control flow: one first l, one seeding range and one recurrence
        // form (the first active lane's) per warp -- per-lane forms split the warp across
        // both loop bodies; measured 9 % faster at nside 2048
        const unsigned am = __activemask();
        const int lmin = __reduce_min_sync(am, P.lmin), lmaxs = __reduce_max_sync(am, P.lmaxs);
        const bool diff = __shfl_sync(am, P.diff ? 1 : 0, __ffs(am) - 1) != 0;
        if (lmin <= L) {
            if (diff) mx_syn_run<true, NP>(P, m, L, sAB, sac, ER, EI, OR, OI, lmin, lmaxs);
            else mx_syn_run<false, NP>(P, m, L, sAB, sac, ER, EI, OR, OI, lmin, lmaxs);
        }
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const int p = p0 + k;
            if (p >= npairs) break;
            const int pk = k >> 1, h = k & 1;
            const float er = get(ER[pk], h), ei = get(EI[pk], h), orr = get(OR[pk], h), oi = get(OI[pk], h);
            float2 *g = G + (size_t)p * pstride + 2 * (size_t)m;
            g[0] = make_float2(er + orr, ei + oi);
            g[1] = make_float2(er - orr, ei - oi);
        }
    }
}

// analysis: CTA per m; a warp covers 32 lanes x NP pairs; chunks of CH
// values of l accumulate the packs in f32x2 registers, then are summed across
// the warp (through the swizzled shared stage for CH = 8, by a shuffle
// reduce-scatter otherwise).  Eight pairs per lane halve the cross-lane sum
// per (l, m, pair) against four; two CTAs per SM (128 registers) measured
// faster than one CTA with no spills.


template <bool DIFF, int NP, int CH>
__device__ __forceinline__ void mx_ana_run(const MxPairs<NP> &P, int m, int L, int lmin_w, int lmaxs_w,
                                           const float4 *__restrict__ sAB,
                                           const float2 (&FEr)[NP / 2], const float2 (&FEi)[NP / 2],
                                           const float2 (&FOr)[NP / 2], const float2 (&FOi)[NP / 2],
                                           float2 *acc, float4 *stage, int lane)
{
    constexpr int NPK = NP / 2;
    float2 Sa[NPK], Sb[NPK], V0[NPK], V1[NPK];
#pragma unroll
    for (int pk = 0; pk < NPK; ++pk) Sa[pk] = Sb[pk] = dup(0.f);
    for (int l0 = lmin_w; l0 <= L; l0 += CH) {
        float2 AR[CH], AI[CH];
        const bool inj = l0 <= lmaxs_w;
#pragma unroll
        for (int i = 0; i < CH; i += 2) {
            const float4 ab = sAB[(l0 - m + i) >> 1];  // l0 - m is even
            if (inj) mx_step<DIFF, true, NP>(P, l0 + i, ab.x, ab.y, ab.z, ab.w, Sa, Sb, V0, V1);
            else mx_step<DIFF, false, NP>(P, l0 + i, ab.x, ab.y, ab.z, ab.w, Sa, Sb, V0, V1);
            AR[i] = __fmul2_rn(FEr[0], V0[0]);
            AI[i] = __fmul2_rn(FEi[0], V0[0]);
            AR[i + 1] = __fmul2_rn(FOr[0], V1[0]);
            AI[i + 1] = __fmul2_rn(FOi[0], V1[0]);
#pragma unroll
            for (int pk = 1; pk < NPK; ++pk) {
                AR[i] = __ffma2_rn(FEr[pk], V0[pk], AR[i]);
                AI[i] = __ffma2_rn(FEi[pk], V0[pk], AI[i]);
                AR[i + 1] = __ffma2_rn(FOr[pk], V1[pk], AR[i + 1]);
                AI[i + 1] = __ffma2_rn(FOi[pk], V1[pk], AI[i + 1]);
            }
            if constexpr (CH == 8) {
                stage[stage_slot(i, lane)] = make_float4(AR[i].x, AR[i].y, AI[i].x, AI[i].y);
                stage[stage_slot(i + 1, lane)] = make_float4(AR[i + 1].x, AR[i + 1].y, AI[i + 1].x, AI[i + 1].y);
            }
        }
        if constexpr (CH == 8) {
            __syncwarp();
            const int i = lane >> 2, q = lane & 3;
            const float4 *row = stage + 32 * i + 8 * q;
            const int c = q + 4 * (i & 1);
            // the eight stores summed as a tree of depth 3 (a chain of 7 dependent adds held
            // each lane on its loads' latency)
            float2 tr[8], ti[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float4 v = row[j ^ c];
                tr[j] = make_float2(v.x, v.y);
                ti[j] = make_float2(v.z, v.w);
            }
#pragma unroll
            for (int w = 4; w >= 1; w >>= 1)
#pragma unroll
                for (int j = 0; j < w; ++j) {
                    tr[j] = __fadd2_rn(tr[j], tr[j + w]);
                    ti[j] = __fadd2_rn(ti[j], ti[j + w]);
                }
            float vr = tr[0].x + tr[0].y, vi = ti[0].x + ti[0].y;
            vr += __shfl_xor_sync(0xffffffffu, vr, 1);
            vi += __shfl_xor_sync(0xffffffffu, vi, 1);
            vr += __shfl_xor_sync(0xffffffffu, vr, 2);
            vi += __shfl_xor_sync(0xffffffffu, vi, 2);
            if (q == 0) {
                const int l = l0 + i;
                if (l <= L) {
                    atomicAdd(&acc[l - m].x, vr);
                    atomicAdd(&acc[l - m].y, vi);
                }
            }
            __syncwarp();  // the next chunk rewrites the stage
        } else {
            float vr[CH], vi[CH];
#pragma unroll
            for (int i = 0; i < CH; ++i) {
                vr[i] = AR[i].x + AR[i].y;
                vi[i] = AI[i].x + AI[i].y;
            }
            warp_reduce_scatter<float, CH>(vr, vi, lane);
            constexpr int sh = 5 - Log2<CH>::v;  // each l ends in 2^sh lanes
            if ((lane & ((1 << sh) - 1)) == 0) {
                const int l = l0 + (lane >> sh);
                if (l <= L) {
                    atomicAdd(&acc[l - m].x, vr[0]);
                    atomicAdd(&acc[l - m].y, vi[0]);
                }
            }
        }
    }
}

template <int NP, int CH>
__global__ void __launch_bounds__(LEG_THREADS, 2) k_legana_mx(int lmax, int L, int npairs, int lc,
                                                           const float2 *__restrict__ F, const float *__restrict__ A,
                                                           const float *__restrict__ B,
                                                           const int *__restrict__ ls_tab,
                                                           const float *__restrict__ s0_tab,
                                                           const float *__restrict__ s1_tab,
                                                           const float *__restrict__ xp, const float *__restrict__ wp,
                                                           const double *__restrict__ c64, int mode, double omega,
                                                           BlendArgs ba, const double2 *__restrict__ low,
                                                           const double2 *__restrict__ a_old,
                                                           double2 *__restrict__ out, double *__restrict__ part)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[4][LEG_THREADS / 32];
    __shared__ int next_group;
    const int m = blockIdx.x;
    const int nl = L - m + 1;
    const int nlp = nl + CH + 2;
    const long long base = mbase(lmax, m);
    // (A_l, B_l, A_l+1, B_l+1) per pair of l from l - m = 0; for CH = 8 the per-warp
    // stages of the cross-lane sum; FP32 accumulators (each entry sums one cross-lane
    // result per group of ring pairs; the epilogue converts to FP64)
    const int nab = (nlp + 1) / 2;
    float4 *sAB = reinterpret_cast<float4 *>(smem_raw);
    float4 *stage = sAB + nab;
    float2 *acc = reinterpret_cast<float2 *>(stage + (CH == 8 ? LEG_THREADS * 8 : 0));
    for (int i = threadIdx.x; i < nab; i += blockDim.x) {
        const int j = 2 * i;
        sAB[i] = make_float4(j < nl ? A[base + j] : 0.f, j < nl ? B[base + j] : 0.f,
                             j + 1 < nl ? A[base + j + 1] : 0.f, j + 1 < nl ? B[base + j + 1] : 0.f);
    }
    for (int i = threadIdx.x; i < nlp; i += blockDim.x) acc[i] = make_float2(0.f, 0.f);
    if (threadIdx.x == 0) next_group = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int per_group = 32 * NP;
    const int ngroups = (npairs + per_group - 1) / per_group;
    const size_t pstride = (size_t)(lmax + 1) * 2;
    for (;;) {
        // warps take groups of ring pairs dynamically (their work differs with latitude)
        int grp = 0;
        if (lane == 0) grp = atomicAdd(&next_group, 1);
        grp = __shfl_sync(0xffffffffu, grp, 0);
        if (grp >= ngroups) break;
        // equator first: the work per pair grows towards the equator (more l above the
        // first kept one), so handing out the largest groups first shortens the tail at the
        // barrier before the epilogue
        const int p0 = (ngroups - 1 - grp) * per_group + lane * NP;
        MxPairs<NP> P;
        mx_load_pairs<NP>(P, m, L, npairs, p0, ls_tab, s0_tab, s1_tab, xp, wp);
        // one recurrence form per warp: the shuffles below need warp-uniform control flow
        P.diff = __shfl_sync(0xffffffffu, P.diff ? 1 : 0, 0) != 0;
        const int lmin_w = __reduce_min_sync(0xffffffffu, P.lmin);
        const int lmaxs_w = __reduce_max_sync(0xffffffffu, P.lmaxs);  // one seeding range per warp
        if (lmin_w > L) continue;
        float fer[NP], fei[NP], forr[NP], foi[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            fer[k] = fei[k] = forr[k] = foi[k] = 0.f;
            if (P.ls[k] != BIG) {
                const float2 *f = F + (size_t)(p0 + k) * pstride + 2 * (size_t)m;
                const float2 fn = f[0], fs = f[1];
                fer[k] = fn.x + fs.x;
                fei[k] = fn.y + fs.y;
                forr[k] = fn.x - fs.x;
                foi[k] = fn.y - fs.y;
            }
        }
        float2 FEr[NP / 2], FEi[NP / 2], FOr[NP / 2], FOi[NP / 2];
#pragma unroll
        for (int pk = 0; pk < NP / 2; ++pk) {
            FEr[pk] = make_float2(fer[2 * pk], fer[2 * pk + 1]);
            FEi[pk] = make_float2(fei[2 * pk], fei[2 * pk + 1]);
            FOr[pk] = make_float2(forr[2 * pk], forr[2 * pk + 1]);
            FOi[pk] = make_float2(foi[2 * pk], foi[2 * pk + 1]);
        }
        float4 *wstage = stage + (threadIdx.x >> 5) * 256;
        if (P.diff) mx_ana_run<true, NP, CH>(P, m, L, lmin_w, lmaxs_w, sAB, FEr, FEi, FOr, FOi, acc, wstage, lane);
        else mx_ana_run<false, NP, CH>(P, m, L, lmin_w, lmaxs_w, sAB, FEr, FEi, FOr, FOi, acc, wstage, lane);
    }
    __syncthreads();
    const int low_lim = (low && m < lc) ? lcm_of(lc, m) : 0;
    blend_epilogue(lmax, L, m, base, mode, omega, ba, c64, acc, low, low_lim, a_old, out, part, red);
}

// ---------------------------------------------------------------------------
// launches
// ---------------------------------------------------------------------------
template <typename T>
size_t syn_smem(int L) { return (size_t)(L + 3) * (sizeof(cx<T>) + sizeof(T)) + 16; }

template <typename T, int CH>
size_t ana_smem(int L) { return (size_t)(L + 1 + CH + 2) * (sizeof(double2) + sizeof(T)) + 16; }

size_t syn_mx_smem(int L) { return (size_t)((L + 2) / 2 + 2) * 2 * sizeof(float4) + 16; }
size_t ana_mx_smem(int L, int ch)
{
    return (size_t)(L + 1 + ch + 2) * (sizeof(float2) + 2 * sizeof(float)) + 32 +
           (ch == 8 ? (size_t)LEG_THREADS * 8 * sizeof(float4) : 0);
}

template <typename TG>
wf_status launch_syn64(wf_plan p, const double2 *alm, int L, int lcut, cx<TG> *G, int gstride, cudaStream_t s)
{
    const HpTables &t = p->tab;
    const int Lgrid = lcut > 0 ? std::min(L, lcut - 1) : L;
    if (Lgrid < 0) return WF_OK;
    const int gx = (p->npairs + 4 * LEG_THREADS - 1) / (4 * LEG_THREADS);
    dim3 grid(gx, Lgrid + 1);
    const size_t sm = syn_smem<double>(lcut > 0 ? std::min(L, lcut + 1) : L);
    if (wf_status st = raise_smem_limit((const void *)k_legsyn<double, TG>, sm)) return st;
    k_legsyn<double, TG><<<grid, LEG_THREADS, sm, s>>>(p->lmax, L, p->npairs, lcut, alm, t.A64, t.c64, t.ls,
                                                            t.s0_64, t.s1_64, t.x64, G, gstride);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    return WF_OK;
}

template <typename TF>
wf_status launch_ana64(wf_plan p, int L, int lcut, const void *F, LegMode mode, const BlendArgs &ba,
                       const double2 *a_old, double2 *out, cudaStream_t s)
{
    constexpr int CH = 16;
    const HpTables &t = p->tab;
    const int Lgrid = lcut > 0 ? std::min(L, lcut - 1) : L;
    if (Lgrid < 0) return WF_OK;
    const size_t sm = ana_smem<double, CH>(lcut > 0 ? std::min(L, lcut + 1) : L);
    if (wf_status st = raise_smem_limit((const void *)k_legana<double, TF, CH, false>, sm)) return st;
    k_legana<double, TF, CH, false><<<Lgrid + 1, LEG_THREADS, sm, s>>>(
        p->lmax, L, p->npairs, lcut, (const cx<TF> *)F, t.A64, t.ls, t.s0_64, t.s1_64, t.x64, t.c64, (int)mode,
        p->omega, ba, a_old, out, p->ws.part_harm);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    return WF_OK;
}

// FP64 block of the mixed analysis (adjoint, l < lcm(lcut, m)): the block is
// triangular in m, so one CTA per m would leave m = 0 as the critical path;
// each m is split over ring-pair chunks whose shares are added atomically.
wf_status launch_ana64_low(wf_plan p, int L, int lcut, const float2 *F, double2 *out, cudaStream_t s)
{
    constexpr int CH = 16;
    const HpTables &t = p->tab;
    const int nm = std::min(L, lcut - 1) + 1;
    if (nm <= 0) return WF_OK;
    WF_CUDA(cudaMemsetAsync(out, 0, (size_t)mbase(p->lmax, nm) * sizeof(double2), s));
    const size_t sm = ana_smem<double, CH>(std::min(L, lcut + 1));
    if (wf_status st = raise_smem_limit((const void *)k_legana<double, float, CH, true>, sm)) return st;
    const int nchunk = std::max(1, std::min(16, p->npairs / 512));
    BlendArgs none;
    k_legana<double, float, CH, true><<<dim3(nm, nchunk), LEG_THREADS, sm, s>>>(
        p->lmax, L, p->npairs, lcut, F, t.A64, t.ls, t.s0_64, t.s1_64, t.x64, t.c64, (int)LEG_ADJOINT, p->omega, none,
        nullptr, out, nullptr);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    return WF_OK;
}

// FP64 block from the double-float table: synthesis into the block's FP32 ring
// coefficients, analysis into the FP64 output that the FP32 analysis epilogue adds
wf_status launch_lowsyn_df(wf_plan p, const double2 *alm, int L, cudaStream_t s)
{
    const HpTables &t = p->tab;
    const int lc = t.lc_mx, nm = std::min(L, lc - 1) + 1;
    if (nm <= 0) return WF_OK;
    const int gx = (p->npairs + LEG_THREADS - 1) / LEG_THREADS;
    const size_t sm = (size_t)(std::min(low_rows(p->lmax, lc, 0), L + 1) + 1) * sizeof(float4);
    k_lowsyn_df<<<dim3(gx, nm), LEG_THREADS, sm, s>>>(p->lmax, L, p->npairs, t.np_pad, lc, t.lowrow, t.lowtab, alm,
                                                       p->ws.Glow, t.glow_cap);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    return WF_OK;
}

wf_status launch_lowana_df(wf_plan p, int L, const float2 *F, double2 *out, cudaStream_t s)
{
    const HpTables &t = p->tab;
    const int lc = t.lc_mx, nm = std::min(L, lc - 1) + 1;
    if (nm <= 0) return WF_OK;
    const int rows0 = std::min(low_rows(p->lmax, lc, 0), L + 1);
    const int gx = ((rows0 + 1) / 2 + LOWANA_ROWS - 1) / LOWANA_ROWS;
    const size_t sm = (size_t)t.np_pad * sizeof(float4);
    k_lowana_df<<<dim3(gx, 2, nm), LEG_THREADS, sm, s>>>(p->lmax, L, p->npairs, t.np_pad, lc, t.lowrow, t.lowtab, F,
                                                          out);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    return WF_OK;
}

// double-float transforms of a sweep sub-plan (FP64 plan, G and F in FP64)
size_t syn_df_smem(int L) { return (size_t)(L + 3) * (sizeof(float4) + sizeof(float2)) + 16; }
size_t ana_df_smem(int L)
{
    const size_t nlp = (size_t)L + 1 + 8 + 2;
    return nlp * sizeof(double2) + ((nlp + 1) / 2) * sizeof(float4) + (size_t)LEG_THREADS * 8 * sizeof(float4) + 32;
}

wf_status launch_syn_df(wf_plan p, const double2 *alm, int L)
{
    const HpTables &t = p->tab;
    const int gx = (p->npairs + 4 * LEG_THREADS - 1) / (4 * LEG_THREADS);
    const size_t sm = syn_df_smem(L);
    k_legsyn_df<<<dim3(gx, L + 1), LEG_THREADS, sm, p->stream>>>(p->lmax, L, p->npairs, alm, t.A64, t.c64, t.ls, t.s0_64,
                                                                 t.s1_64, t.x64, (double2 *)p->ws.G);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    return WF_OK;
}

wf_status launch_ana_df(wf_plan p, int L, LegMode mode, const BlendArgs &ba, const double2 *a_old, double2 *out)
{
    const HpTables &t = p->tab;
    const size_t sm = ana_df_smem(L);
    k_legana_df<<<L + 1, LEG_THREADS, sm, p->stream>>>(p->lmax, L, p->npairs, (const double2 *)p->ws.F, t.A64, t.ls,
                                                       t.s0_64, t.s1_64, t.x64, t.c64, (int)mode, p->omega, ba, a_old,
                                                       out, p->ws.part_harm);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    return WF_OK;
}

// Device bytes of the block's table for l_c on this plan
long long low_table_bytes(int lmax, int npairs, int lc)
{
    const long long np_pad = (npairs + 31) & ~31;
    long long rows = 0;
    for (int m = 0; m < std::min(lc, lmax + 1); ++m) rows += low_rows(lmax, lc, m);
    return rows * np_pad * (long long)sizeof(float2);
}

}  // namespace

long long hp_low_table_bytes(int lmax, int npairs, int lc) { return low_table_bytes(lmax, npairs, lc); }

// ---------------------------------------------------------------------------
// host: recurrence tables and seeds
// ---------------------------------------------------------------------------
wf_status hp_build_legendre_tables(wf_plan p, const std::vector<double> &xpair, const std::vector<double> &stpair)
{
    const int lmax = p->lmax, np = p->npairs;
    const long long nalm = p->nalm;
    std::vector<double> A(nalm), c(nalm), Bm2(nalm), log2c(lmax + 1);
    for (int m = 0; m <= lmax; ++m) {
        const long long b = mbase(lmax, m);
        auto coef = [m](int l) { return std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m)); };
        c[b] = 1.0;
        if (m + 1 <= lmax) c[b + 1] = 1.0;
        for (int l = m + 2; l <= lmax; ++l) c[b + (l - m)] = (coef(l) / coef(l - 1)) * c[b + (l - 2 - m)];
        // scale the l - m odd chain so that c_l / c_{l-1} -> 1 at lmax: the
        // multiplier A_l then tends to 2 x-independently, which the
        // difference form needs
        if (lmax - m >= 2) {
            const double r = c[b + (lmax - m)] / c[b + (lmax - 1 - m)];
            const double f = ((lmax - m) & 1) ? 1.0 / r : r;
            for (int l = m + 1; l <= lmax; l += 2) c[b + (l - m)] *= f;
        }
        A[b] = 0.0;
        if (m + 1 <= lmax) A[b + 1] = std::sqrt(2.0 * m + 3.0) * c[b] / c[b + 1];
        for (int l = m + 2; l <= lmax; ++l) A[b + (l - m)] = coef(l) * c[b + (l - 1 - m)] / c[b + (l - m)];
        for (int l = m; l <= lmax; ++l) Bm2[b + (l - m)] = A[b + (l - m)] - 2.0;
        // log2 of sqrt((2m+1)/(4 pi) (2m)! / (2^m m!)^2)
        log2c[m] = 0.5 * (std::log(2.0 * m + 1.0) - std::log(4.0 * M_PI) + std::lgamma(2.0 * m + 1.0) -
                          2.0 * std::lgamma(m + 1.0) - 2.0 * m * std::log(2.0)) / std::log(2.0);
    }
    std::vector<double> wpair(np);
    for (int i = 0; i < np; ++i) wpair[i] = 1.0 - xpair[i];
    // 1 - x exactly for the polar-cap rings (1 - z = k^2 / (3 nside^2))
    for (int i = 0; i + 1 < p->nside && i < np; ++i)
        wpair[i] = (double)(i + 1) * (i + 1) / (3.0 * p->nside * p->nside);
    const bool f32 = p->prec != WF_PREC_FP64;
    double *dx64 = nullptr, *dst64 = nullptr, *dlog2c = nullptr;
    wf_status st;
    HpTables &t = p->tab;
    if ((st = plan_alloc(p, (void **)&t.c64, nalm * sizeof(double))) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&t.A64, nalm * sizeof(double))) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&t.x64, np * sizeof(double))) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&dst64, np * sizeof(double))) != WF_OK) return st;
    t.st64 = dst64;
    if ((st = plan_alloc(p, (void **)&dlog2c, (lmax + 1) * sizeof(double))) != WF_OK) return st;
    const long long ns = (long long)(lmax + 1) * np;
    if ((st = plan_alloc(p, (void **)&t.ls, ns * sizeof(int))) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&t.s0_64, ns * sizeof(double))) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&t.s1_64, ns * sizeof(double))) != WF_OK) return st;
    if ((st = to_device(p, t.A64, A.data(), nalm * sizeof(double))) != WF_OK) return st;
    if ((st = to_device(p, t.c64, c.data(), nalm * sizeof(double))) != WF_OK) return st;
    if ((st = to_device(p, t.x64, xpair.data(), np * sizeof(double))) != WF_OK) return st;
    if ((st = to_device(p, dst64, stpair.data(), np * sizeof(double))) != WF_OK) return st;
    if ((st = to_device(p, dlog2c, log2c.data(), (lmax + 1) * sizeof(double))) != WF_OK) return st;
    {
        const int th = 256;
        const long long nb = (ns + th - 1) / th;
        k_seeds<<<(unsigned)nb, th, 0, p->stream>>>(lmax, np, t.x64, dst64, dlog2c, t.A64, t.c64, t.ls, t.s0_64,
                                                     t.s1_64);
        WF_COUNT_LAUNCH(p);
        WF_CUDA(cudaGetLastError());
    }
    if (f32) {
        if ((st = plan_alloc(p, (void **)&t.A32, nalm * sizeof(float))) != WF_OK) return st;
        if ((st = plan_alloc(p, (void **)&t.B32, nalm * sizeof(float))) != WF_OK) return st;
        if ((st = plan_alloc(p, (void **)&t.x32, np * sizeof(float))) != WF_OK) return st;
        if ((st = plan_alloc(p, (void **)&t.w32, np * sizeof(float))) != WF_OK) return st;
        if ((st = plan_alloc(p, (void **)&t.ls_mx, ns * sizeof(int))) != WF_OK) return st;
        if ((st = plan_alloc(p, (void **)&t.s0_mx, ns * sizeof(float))) != WF_OK) return st;
        if ((st = plan_alloc(p, (void **)&t.s1_mx, ns * sizeof(float))) != WF_OK) return st;
        std::vector<float> Af(nalm), Bf(nalm), xf(np), wf(np);
        for (long long i = 0; i < nalm; ++i) {
            Af[i] = (float)A[i];
            Bf[i] = (float)Bm2[i];
        }
        for (int i = 0; i < np; ++i) {
            xf[i] = (float)xpair[i];
            wf[i] = (float)wpair[i];
        }
        if ((st = to_device(p, t.A32, Af.data(), nalm * sizeof(float))) != WF_OK) return st;
        if ((st = to_device(p, t.B32, Bf.data(), nalm * sizeof(float))) != WF_OK) return st;
        if ((st = to_device(p, t.x32, xf.data(), np * sizeof(float))) != WF_OK) return st;
        if ((st = to_device(p, t.w32, wf.data(), np * sizeof(float))) != WF_OK) return st;
        t.lc_mx = -1;
        if ((st = hp_set_low_block(p, 0)) != WF_OK) return st;
    }
    // raise the shared-memory limits of every Legendre kernel this plan can launch to
    // their lmax sizes now, so that no launch (e.g. inside a graph capture) needs to
    if (f32) {
        const void *syn[] = {(const void *)k_legsyn_mx<2>, (const void *)k_legsyn_mx<4>, (const void *)k_legsyn_mx<8>};
        for (const void *f : syn)
            if ((st = raise_smem_limit(f, syn_mx_smem(lmax))) != WF_OK) return st;
        if ((st = raise_smem_limit((const void *)k_legana_mx<2, 16>, ana_mx_smem(lmax, 16))) != WF_OK) return st;
        if ((st = raise_smem_limit((const void *)k_legana_mx<4, 16>, ana_mx_smem(lmax, 16))) != WF_OK) return st;
        if ((st = raise_smem_limit((const void *)k_legana_mx<8, 8>, ana_mx_smem(lmax, 8))) != WF_OK) return st;
        if ((st = raise_smem_limit((const void *)k_legsyn<double, float>, syn_smem<double>(lmax))) != WF_OK)
            return st;
        if ((st = raise_smem_limit((const void *)k_legana<double, float, 16, true>, ana_smem<double, 16>(lmax))) !=
            WF_OK)
            return st;
        if ((st = raise_smem_limit((const void *)k_lowsyn_df, (size_t)(lmax + 2) * sizeof(float4))) != WF_OK)
            return st;
        if ((st = raise_smem_limit((const void *)k_lowana_df, (size_t)((np + 31) & ~31) * sizeof(float4))) != WF_OK)
            return st;
        if (tc_prec(p->prec)) {
            if ((st = tc_prepare(lmax)) != WF_OK) return st;
            if ((st = plan_alloc(p, (void **)&p->ws.ca32, nalm * sizeof(float2))) != WF_OK) return st;
        }
    } else {
        if ((st = raise_smem_limit((const void *)k_legsyn_df, syn_df_smem(lmax))) != WF_OK) return st;
        if ((st = raise_smem_limit((const void *)k_legana_df, ana_df_smem(lmax))) != WF_OK) return st;
        if ((st = raise_smem_limit((const void *)k_legsyn<double, double>, syn_smem<double>(lmax))) != WF_OK)
            return st;
        if ((st = raise_smem_limit((const void *)k_legana<double, double, 16, false>, ana_smem<double, 16>(lmax))) !=
            WF_OK)
            return st;
    }
    WF_CUDA(cudaStreamSynchronize(p->stream));
    return WF_OK;
}

// Select the FP64 block l < lc of the mixed path and build the FP32 seeds
// that restart the recurrence at lc (cached for the current lc).
wf_status hp_set_low_block(wf_plan p, int lc)
{
    HpTables &t = p->tab;
    if (p->prec == WF_PREC_FP64) return WF_OK;
    if (lc < 0) lc = 0;
    if (lc > p->lmax + 1) lc = p->lmax + 1;
    if (lc == t.lc_mx) return WF_OK;
    const long long ns = (long long)(p->lmax + 1) * p->npairs;
    const int th = 256;
    k_restart_seeds<<<(unsigned)((ns + th - 1) / th), th, 0, p->stream>>>(p->lmax, p->npairs, lc, t.x64, t.A64, t.ls,
                                                                        t.s0_64, t.s1_64, t.ls_mx, t.s0_mx, t.s1_mx);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    if (lc > 0 && lc > t.glow_cap) {
        wf_status st = plan_alloc(p, (void **)&p->ws.Glow, (size_t)p->npairs * lc * 2 * sizeof(float2));
        if (st != WF_OK) return st;
        t.glow_cap = lc;
    }
    // the block's Legendre table, when it fits the budget (wf_options.mixed_table_bytes)
    t.low_df = 0;
    const long long budget = p->opt.mixed_table_bytes == 0 ? (2LL << 30) : p->opt.mixed_table_bytes;
    const long long bytes = lc > 0 ? low_table_bytes(p->lmax, p->npairs, lc) : 0;
    if (lc > 0 && bytes <= budget) {
        wf_status st;
        const int np_pad = (p->npairs + 31) & ~31, nm = std::min(lc, p->lmax + 1);
        const long long entries = bytes / (long long)sizeof(float2);
        if (entries > t.lowtab_cap) {
            if ((st = plan_alloc(p, (void **)&t.lowtab, (size_t)bytes)) != WF_OK) return st;
            t.lowtab_cap = entries;
        }
        if (!t.lowrow && (st = plan_alloc(p, (void **)&t.lowrow, (size_t)(p->lmax + 2) * sizeof(long long))) != WF_OK)
            return st;
        std::vector<long long> off(nm + 1, 0);
        for (int m = 0; m < nm; ++m) off[m + 1] = off[m] + low_rows(p->lmax, lc, m);
        if ((st = to_device(p, t.lowrow, off.data(), off.size() * sizeof(long long))) != WF_OK) return st;
        k_lowtab_build<<<dim3((np_pad + 255) / 256, nm), 256, 0, p->stream>>>(
            p->lmax, p->npairs, np_pad, lc, t.lowrow, t.A64, t.c64, t.ls, t.s0_64, t.s1_64, t.x64, t.lowtab);
        WF_COUNT_LAUNCH(p);
        WF_CUDA(cudaGetLastError());
        t.np_pad = np_pad;
        t.low_df = 1;
    }
    t.lc_mx = lc;
    return WF_OK;
}

wf_status hp_legendre_synthesis_buf(wf_plan p, const double2 *alm, int L, double2 *G)
{
    if (p->prec != WF_PREC_FP64) return set_error(WF_EUNSUPPORTED, "explicit-buffer transforms need an FP64 plan");
    return launch_syn64<double>(p, alm, L, 0, G, p->lmax + 1, p->stream);
}

wf_status hp_legendre_adjoint_buf(wf_plan p, int L, const double2 *F, double2 *out)
{
    if (p->prec != WF_PREC_FP64) return set_error(WF_EUNSUPPORTED, "explicit-buffer transforms need an FP64 plan");
    WF_CUDA(cudaMemsetAsync(out, 0, p->nalm * sizeof(double2), p->stream));
    BlendArgs none;
    return launch_ana64<double>(p, L, 0, F, LEG_ADJOINT, none, nullptr, out, p->stream);
}

// Mixed precision: the FP64 low-l block (FP64 pipe, few CTAs) runs on the
// plan's auxiliary stream next to the FP32 kernels (FMA pipes); the two write
// disjoint buffers and are joined before their results are combined.
wf_status fork_aux(wf_plan p)
{
    WF_CUDA(cudaEventRecord(p->fork_ev, p->stream));
    WF_CUDA(cudaStreamWaitEvent(p->aux, p->fork_ev, 0));
    return WF_OK;
}

wf_status join_aux(wf_plan p)
{
    WF_CUDA(cudaEventRecord(p->join_ev, p->aux));
    WF_CUDA(cudaStreamWaitEvent(p->stream, p->join_ev, 0));
    return WF_OK;
}

template <int NP>
wf_status launch_syn_mx(wf_plan p, const double2 *alm, int L)
{
    const HpTables &t = p->tab;
    const int gx = (p->npairs + NP * LEG_THREADS - 1) / (NP * LEG_THREADS);
    dim3 grid(gx, L + 1);
    const size_t sm = syn_mx_smem(L);
    if (wf_status st = raise_smem_limit((const void *)k_legsyn_mx<NP>, sm)) return st;
    k_legsyn_mx<NP><<<grid, LEG_THREADS, sm, p->stream>>>(p->lmax, L, p->npairs, alm, t.A32, t.B32, t.c64, t.ls_mx,
                                                           t.s0_mx, t.s1_mx, t.x32, t.w32, (float2 *)p->ws.G);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    return WF_OK;
}

wf_status hp_legendre_synthesis(wf_plan p, const double2 *alm, int L)
{
    const HpTables &t = p->tab;
    if (p->prec == WF_PREC_FP64)
        return p->df_legendre ? launch_syn_df(p, alm, L)
                              : launch_syn64<double>(p, alm, L, 0, (double2 *)p->ws.G, p->lmax + 1, p->stream);
    wf_status st;
    const bool low = t.lc_mx > 0;
    if (low) {
        if ((st = fork_aux(p)) != WF_OK) return st;
        st = t.low_df ? launch_lowsyn_df(p, alm, L, p->aux)
                      : launch_syn64<float>(p, alm, L, t.lc_mx, p->ws.Glow, t.glow_cap, p->aux);
        if (st != WF_OK) return st;
    }
    if (tc_prec(p->prec)) {
        // in a batch step the group launch (wf_solve_batch) has written G already
        float2 *G = (float2 *)p->ws.G;
        st = p->tc_deferred ? WF_OK : hp_tc_synthesis(p, 1, &alm, &p->ws.ca32, &G, &L, L, p->stream);
    } else {
        switch (p->tile_syn) {
        case 2: st = launch_syn_mx<2>(p, alm, L); break;
        case 8: st = launch_syn_mx<8>(p, alm, L); break;
        default: st = launch_syn_mx<4>(p, alm, L); break;
        }
    }
    if (st != WF_OK) return st;
    if (low) return join_aux(p);
    return WF_OK;
}

namespace {
template <int NP, int CH>
wf_status launch_ana_mx_t(wf_plan p, int L, LegMode mode, const BlendArgs &ba, const double2 *low,
                          const double2 *a_old, double2 *out)
{
    const HpTables &t = p->tab;
    const size_t sm = ana_mx_smem(L, CH);
    if (wf_status st = raise_smem_limit((const void *)k_legana_mx<NP, CH>, sm)) return st;
    k_legana_mx<NP, CH><<<L + 1, LEG_THREADS, sm, p->stream>>>(
        p->lmax, L, p->npairs, t.lc_mx, (const float2 *)p->ws.F, t.A32, t.B32, t.ls_mx, t.s0_mx, t.s1_mx, t.x32,
        t.w32, t.c64, (int)mode, p->omega, ba, low, a_old, out, p->ws.part_harm);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    return WF_OK;
}

wf_status launch_ana_mx(wf_plan p, int L, LegMode mode, const BlendArgs &ba, const double2 *low, const double2 *a_old,
                        double2 *out)
{
    switch (p->tile_ana) {
    case 2: return launch_ana_mx_t<2, 16>(p, L, mode, ba, low, a_old, out);
    case 4: return launch_ana_mx_t<4, 16>(p, L, mode, ba, low, a_old, out);
    default: return launch_ana_mx_t<8, 8>(p, L, mode, ba, low, a_old, out);
    }
}
}  // namespace

// Autotuner of the mixed Legendre tiles: each variant of the synthesis (2, 4
// or 8 ring pairs per thread) and of the analysis (2, 4 or 8 pairs per lane)
// runs on this plan's own buffers at the full band; the fastest is kept.
wf_status hp_autotune(wf_plan p, int reps)
{
    if (p->prec == WF_PREC_FP64) return WF_OK;
    if (reps <= 0) reps = 3;
    const int L = p->lmax;
    WF_CUDA(cudaMemsetAsync(p->ws.a, 0, p->nalm * sizeof(double2), p->stream));
    WF_CUDA(cudaMemsetAsync(p->ws.F, 0, (size_t)p->npairs * (L + 1) * 2 * sizeof(float2), p->stream));
    cudaEvent_t e0, e1;
    WF_CUDA(cudaEventCreate(&e0));
    WF_CUDA(cudaEventCreate(&e1));
    const int saved_syn = p->tile_syn, saved_ana = p->tile_ana;
    const int np[3] = {2, 4, 8};
    float best_syn = 1e30f, best_ana = 1e30f;
    int pick_syn = saved_syn, pick_ana = saved_ana;
    wf_status st = WF_OK;
    BlendArgs none;
    for (int v = 0; v < 3 && st == WF_OK; ++v) {
        p->tile_syn = np[v];
        p->tile_ana = np[v];
        float ms[2] = {0.f, 0.f};
        for (int which = 0; which < 2 && st == WF_OK; ++which) {
            for (int r = -1; r < reps && st == WF_OK; ++r) {  // r = -1: untimed warm-up
                if (r == 0) cudaEventRecord(e0, p->stream);
                if (which == 0)
                    st = np[v] == 2 ? launch_syn_mx<2>(p, p->ws.a, L)
                                    : np[v] == 8 ? launch_syn_mx<8>(p, p->ws.a, L) : launch_syn_mx<4>(p, p->ws.a, L);
                else
                    st = launch_ana_mx(p, L, LEG_ADJOINT, none, nullptr, nullptr, p->ws.b);
            }
            cudaEventRecord(e1, p->stream);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms[which], e0, e1);
        }
        if (st != WF_OK) break;
        if (ms[0] < best_syn) { best_syn = ms[0]; pick_syn = np[v]; }
        if (ms[1] < best_ana) { best_ana = ms[1]; pick_ana = np[v]; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->tile_syn = st == WF_OK ? pick_syn : saved_syn;
    p->tile_ana = st == WF_OK ? pick_ana : saved_ana;
    return st;
}

wf_status hp_legendre_analysis(wf_plan p, int L, LegMode mode, const BlendArgs &ba_in, const double2 *a_old,
                               double2 *out)
{
    const HpTables &t = p->tab;
    BlendArgs ba = ba_in;
    if (mode == LEG_BLEND) {
        k_epi_table<<<(p->lmax + 256) / 256, 256, 0, p->stream>>>(p->lmax, ba.S, p->omega, ba.lam_tauh, ba.tauh,
                                                                  p->ws.epi);
        WF_COUNT_LAUNCH(p);
        WF_CUDA(cudaGetLastError());
        ba.epi = p->ws.epi;
    }
    if (p->prec == WF_PREC_FP64)
        return p->df_legendre ? launch_ana_df(p, L, mode, ba, a_old, out)
                              : launch_ana64<double>(p, L, 0, p->ws.F, mode, ba, a_old, out, p->stream);
    const int lc = t.lc_mx;
    if (lc <= 0) return launch_ana_mx(p, L, mode, ba, nullptr, a_old, out);
    // sequential: the FP32 epilogue of m < lc reads the block's result
    wf_status st = t.low_df ? launch_lowana_df(p, L, (const float2 *)p->ws.F, p->ws.b_low, p->stream)
                            : launch_ana64_low(p, L, lc, (const float2 *)p->ws.F, p->ws.b_low, p->stream);
    if (st != WF_OK) return st;
    return launch_ana_mx(p, L, mode, ba, p->ws.b_low, a_old, out);
}

}  // namespace wf
