// Mixed precision for polarised plans: the spin-2 Legendre synthesis and its
// adjoint (Eqs. 10-11 run them once each per iteration) in FP32, with the
// temperature path's safeguards.
//
// mu form.  The spin +2 and -2 columns P, M (halves, see wf_spin.cu) obey
//     P_l = al_l (x + be_l) P_{l-1} - ga_l P_{l-2},   M_l = al_l (x - be_l) M_{l-1} - ga_l M_{l-2},
// with the same al, ga for both signs.  With P = c mu, c_l = ga_l c_{l-2} (per
// parity chain from c = 1 at l0, l0 + 1) the subtraction loses its multiplier,
//     mu+-_l = A_l (x +- be_l) mu+-_{l-1} - mu+-_{l-2},   A_l = al_l c_{l-1} / c_l,
// and the chain of l0 + 1 is rescaled so that A_l -> 2 at large l.  Rings
// with x > 0.4 run the difference form (Reinsch's modification, as for T):
//     D_l = D_{l-1} + (B+-_l - A_l w) mu_{l-1},  mu_l = mu_{l-1} + D_l,
// w = 1 - x exact from the grid and B+-_l = A_l (1 +- be_l) - 2 tabulated in
// FP64, which keeps the digits that the plain form loses near the poles.
//
// Contraction.  With A = E + iB and C = E - iB (times c_l),
//     Q_m = -(sum A mu+ + sum C mu-),   U_m = i (sum A mu+ - sum C mu-),
// and on the mirror ring mu+ -> sigma mu-, mu- -> sigma mu+ (sigma = (-1)^(l+m)),
// so the north ring takes sum A mu+ + sum C mu-, the south ring
// sum sigma A mu- + sum sigma C mu+.  The adjoint collects
//     YP_l = sum_r mu+ G+,  YM_l = sum_r mu- G-,  G+- = FQ +- i FU,
//     E_l = -c_l (YP + YM),   B_l = i c_l (YP - YM).
//
// FP64 block.  Modes l < lcm(lc, m) (m < lc) go through the FP64 spin-2
// kernels, and the FP32 recurrence restarts there from FP64 values, as for
// the temperature path.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "wf_internal.cuh"

namespace wf {

namespace {

constexpr int PM_THREADS = 256;
constexpr int PM_CH = 8;  // values of l per analysis chunk
constexpr float PM_X_DIFF = 0.4f;
constexpr int PM_BIG = INT_MAX / 2;

__host__ __device__ inline long long pmb(int lmax, int m) { return (long long)m * (2 * lmax + 3 - m) / 2; }
__host__ __device__ inline int lcm_of(int lc, int m) { return m + 2 * ((lc - m + 1) / 2); }

__device__ __forceinline__ float2 dup(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float get(const float2 &v, int k) { return k ? v.y : v.x; }
__device__ __forceinline__ void put(float2 &v, int k, float a)
{
    if (k) v.y = a;
    else v.x = a;
}

// FP32 seeds in mu units: the FP32 recurrence starts at ls_mx, the first kept
// l (for m < lc: lcm(lc, m) when that is larger, computed in FP64 from the
// seeds) on the parity of m, since the FP32 kernels step through l in pairs
// m + 2j, m + 2j + 1.  A first kept l of the other parity moves down by one
// with mu = 0 there when it is l0 = max(m, 2) (the columns vanish below l0),
// and up by one otherwise: the dropped term is below the 2^-81 cut, while a
// zero below it would be an O(1) error in the starting pair that the growth
// through the evanescent region keeps.
__global__ void k_pol_seeds_mx(int lmax, int npairs, int lc, const double *__restrict__ xp,
                               const double *__restrict__ al, const double *__restrict__ be,
                               const double *__restrict__ ga, const double *__restrict__ c,
                               const int *__restrict__ ls_in, const double *__restrict__ p0,
                               const double *__restrict__ p1, const double *__restrict__ m0,
                               const double *__restrict__ m1, int *__restrict__ ls_out, float4 *__restrict__ seed)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)(lmax + 1) * npairs) return;
    const int m = (int)(idx / npairs), p = (int)(idx % npairs);
    const int ls = ls_in[idx];
    int l1 = lmax + 1;
    float4 sd = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ls <= lmax) {
        l1 = ls;
        if (m < lc) l1 = max(l1, lcm_of(lc, m));
        const int l0 = m > 2 ? m : 2;
        // only when l1 = ls (lcm has the parity of m)
        const bool shift = ((l1 - m) & 1) != 0 && l1 == l0;
        if (((l1 - m) & 1) != 0 && l1 != l0) ++l1;
        if (l1 <= lmax) {
            const long long base = pmb(lmax, m);
            const double x = xp[p];
            double Pa = p0[idx], Pb = p1[idx], Ma = m0[idx], Mb = m1[idx];  // at cur, cur + 1
            for (int cur = ls; cur < l1; ++cur) {
                double Pn = 0.0, Mn = 0.0;
                if (cur + 2 <= lmax) {
                    const long long k = base + (cur + 2 - m);
                    Pn = al[k] * (x + be[k]) * Pb - ga[k] * Pa;
                    Mn = al[k] * (x - be[k]) * Mb - ga[k] * Ma;
                }
                Pa = Pb;
                Pb = Pn;
                Ma = Mb;
                Mb = Mn;
            }
            if (shift) {
                --l1;
                Pb = Pa;
                Mb = Ma;
                Pa = Ma = 0.0;
            }
            const double c0 = c[base + (l1 - m)];
            const double c1 = l1 + 1 <= lmax ? c[base + (l1 + 1 - m)] : 1.0;
            sd = make_float4((float)(Pa / c0), (float)(Pb / c1), (float)(Ma / c0), (float)(Mb / c1));
        } else {
            l1 = lmax + 1;
        }
    }
    ls_out[idx] = l1;
    seed[idx] = sd;
}

// NP ring pairs in NP/2 f32x2 packs: first l, seeds, x and w per pair
template <int NP> struct PmPairs {
    int ls[NP];
    float4 s[NP];
    float2 X[NP / 2], W[NP / 2];
    int lmin, lmaxs;
    bool diff;
};

template <int NP>
__device__ __forceinline__ void pm_load_pairs(PmPairs<NP> &P, int m, int L, int npairs, int p0,
                                              const int *__restrict__ ls_tab, const float4 *__restrict__ seed,
                                              const float *__restrict__ xp, const float *__restrict__ wp)
{
    P.lmin = PM_BIG;
    P.lmaxs = -1;
    float xs[NP], ws[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int p = p0 + k;
        int ls = PM_BIG;
        float4 sd = make_float4(0.f, 0.f, 0.f, 0.f);
        float x = 0.f, w = 1.f;
        if (p < npairs) {
            const size_t sidx = (size_t)m * npairs + p;
            ls = ls_tab[sidx];
            if (ls > L) ls = PM_BIG;
            else sd = seed[sidx];
            x = xp[p];
            w = wp[p];
        }
        P.ls[k] = ls;
        P.s[k] = sd;
        xs[k] = x;
        ws[k] = w;
        if (ls < P.lmin) P.lmin = ls;
        if (ls != PM_BIG && ls > P.lmaxs) P.lmaxs = ls;
    }
#pragma unroll
    for (int pk = 0; pk < NP / 2; ++pk) {
        P.X[pk] = make_float2(xs[2 * pk], xs[2 * pk + 1]);
        P.W[pk] = make_float2(ws[2 * pk], ws[2 * pk + 1]);
    }
    P.diff = xs[0] > PM_X_DIFF;
}

// one double step (l, l + 1) of both recurrences for all packs.  Table entries
// t = (A, A be, B+, B-).  Plain state (Sa, Sb) = (mu_{l-2}, mu_{l-1}); difference
// state (Sa, Sb) = (D_{l-1}, mu_{l-1}).  Outputs mu_l (V0) and mu_{l+1} (V1) for
// the + (p) and - (q) columns.
template <bool DIFF, bool INJECT, int NP>
__device__ __forceinline__ void pm_step(const PmPairs<NP> &P, int l, float4 t0, float4 t1, float2 (&Spa)[NP / 2],
                                        float2 (&Spb)[NP / 2], float2 (&Sqa)[NP / 2], float2 (&Sqb)[NP / 2],
                                        float2 (&Vp0)[NP / 2], float2 (&Vp1)[NP / 2], float2 (&Vq0)[NP / 2],
                                        float2 (&Vq1)[NP / 2])
{
#pragma unroll
    for (int pk = 0; pk < NP / 2; ++pk) {
        if (DIFF) {
            float2 D = Spa[pk];
            D = __ffma2_rn(__ffma2_rn(dup(-t0.x), P.W[pk], dup(t0.z)), Spb[pk], D);
            const float2 p0 = __fadd2_rn(Spb[pk], D);
            D = __ffma2_rn(__ffma2_rn(dup(-t1.x), P.W[pk], dup(t1.z)), p0, D);
            const float2 p1 = __fadd2_rn(p0, D);
            Spa[pk] = D;
            Spb[pk] = p1;
            float2 Dq = Sqa[pk];
            Dq = __ffma2_rn(__ffma2_rn(dup(-t0.x), P.W[pk], dup(t0.w)), Sqb[pk], Dq);
            const float2 q0 = __fadd2_rn(Sqb[pk], Dq);
            Dq = __ffma2_rn(__ffma2_rn(dup(-t1.x), P.W[pk], dup(t1.w)), q0, Dq);
            const float2 q1 = __fadd2_rn(q0, Dq);
            Sqa[pk] = Dq;
            Sqb[pk] = q1;
            Vp0[pk] = p0;
            Vp1[pk] = p1;
            Vq0[pk] = q0;
            Vq1[pk] = q1;
        } else {
            const float2 p0 = __ffma2_rn(__ffma2_rn(dup(t0.x), P.X[pk], dup(t0.y)), Spb[pk], neg2(Spa[pk]));
            const float2 p1 = __ffma2_rn(__ffma2_rn(dup(t1.x), P.X[pk], dup(t1.y)), p0, neg2(Spb[pk]));
            const float2 q0 = __ffma2_rn(__ffma2_rn(dup(t0.x), P.X[pk], dup(-t0.y)), Sqb[pk], neg2(Sqa[pk]));
            const float2 q1 = __ffma2_rn(__ffma2_rn(dup(t1.x), P.X[pk], dup(-t1.y)), q0, neg2(Sqb[pk]));
            Spa[pk] = p0;
            Spb[pk] = p1;
            Sqa[pk] = q0;
            Sqb[pk] = q1;
            Vp0[pk] = p0;
            Vp1[pk] = p1;
            Vq0[pk] = q0;
            Vq1[pk] = q1;
        }
        if (INJECT) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = 2 * pk + h;
                if (l == P.ls[k]) {
                    const float4 s = P.s[k];
                    put(Vp0[pk], h, s.x);
                    put(Vp1[pk], h, s.y);
                    put(Vq0[pk], h, s.z);
                    put(Vq1[pk], h, s.w);
                    if (DIFF) {
                        put(Spa[pk], h, s.y - s.x);
                        put(Spb[pk], h, s.y);
                        put(Sqa[pk], h, s.w - s.z);
                        put(Sqb[pk], h, s.w);
                    } else {
                        put(Spa[pk], h, s.x);
                        put(Spb[pk], h, s.y);
                        put(Sqa[pk], h, s.z);
                        put(Sqb[pk], h, s.w);
                    }
                }
            }
        }
    }
}

// synthesis accumulators of one pack: sums of A mu+, A mu-, C mu+, C mu- for
// even (l - m even, sigma = +1) and odd l, real and imaginary parts
struct PmAcc {
    float2 ApR[2], ApI[2], AmR[2], AmI[2], CpR[2], CpI[2], CmR[2], CmI[2];  // [parity]
};

template <bool DIFF, bool INJECT, int NP>
__device__ __forceinline__ void pm_syn_pair(const PmPairs<NP> &P, int l, int m, const float4 *__restrict__ sT,
                                            const float4 *__restrict__ sAC, float2 (&Spa)[NP / 2],
                                            float2 (&Spb)[NP / 2], float2 (&Sqa)[NP / 2], float2 (&Sqb)[NP / 2],
                                            PmAcc (&acc)[NP / 2])
{
    const int j = l - m;
    const float4 t0 = sT[j], t1 = sT[j + 1], c0 = sAC[j], c1 = sAC[j + 1];
    float2 Vp0[NP / 2], Vp1[NP / 2], Vq0[NP / 2], Vq1[NP / 2];
    pm_step<DIFF, INJECT, NP>(P, l, t0, t1, Spa, Spb, Sqa, Sqb, Vp0, Vp1, Vq0, Vq1);
#pragma unroll
    for (int pk = 0; pk < NP / 2; ++pk) {
        PmAcc &a = acc[pk];
        a.ApR[0] = __ffma2_rn(dup(c0.x), Vp0[pk], a.ApR[0]);
        a.ApI[0] = __ffma2_rn(dup(c0.y), Vp0[pk], a.ApI[0]);
        a.AmR[0] = __ffma2_rn(dup(c0.x), Vq0[pk], a.AmR[0]);
        a.AmI[0] = __ffma2_rn(dup(c0.y), Vq0[pk], a.AmI[0]);
        a.CpR[0] = __ffma2_rn(dup(c0.z), Vp0[pk], a.CpR[0]);
        a.CpI[0] = __ffma2_rn(dup(c0.w), Vp0[pk], a.CpI[0]);
        a.CmR[0] = __ffma2_rn(dup(c0.z), Vq0[pk], a.CmR[0]);
        a.CmI[0] = __ffma2_rn(dup(c0.w), Vq0[pk], a.CmI[0]);
        a.ApR[1] = __ffma2_rn(dup(c1.x), Vp1[pk], a.ApR[1]);
        a.ApI[1] = __ffma2_rn(dup(c1.y), Vp1[pk], a.ApI[1]);
        a.AmR[1] = __ffma2_rn(dup(c1.x), Vq1[pk], a.AmR[1]);
        a.AmI[1] = __ffma2_rn(dup(c1.y), Vq1[pk], a.AmI[1]);
        a.CpR[1] = __ffma2_rn(dup(c1.z), Vp1[pk], a.CpR[1]);
        a.CpI[1] = __ffma2_rn(dup(c1.w), Vp1[pk], a.CpI[1]);
        a.CmR[1] = __ffma2_rn(dup(c1.z), Vq1[pk], a.CmR[1]);
        a.CmI[1] = __ffma2_rn(dup(c1.w), Vq1[pk], a.CmI[1]);
    }
}

// lmin, lmaxs: the warp's smallest first l and largest seeding l (one loop, one
// trip count per warp; lanes not yet started add zeros)
template <bool DIFF, int NP>
__device__ __forceinline__ void pm_syn_run(const PmPairs<NP> &P, int m, int L, const float4 *__restrict__ sT,
                                           const float4 *__restrict__ sAC, PmAcc (&acc)[NP / 2], int lmin, int lmaxs)
{
    float2 Spa[NP / 2], Spb[NP / 2], Sqa[NP / 2], Sqb[NP / 2];
#pragma unroll
    for (int pk = 0; pk < NP / 2; ++pk) Spa[pk] = Spb[pk] = Sqa[pk] = Sqb[pk] = dup(0.f);
    int l = lmin;
    for (; l <= L && l <= lmaxs; l += 2) pm_syn_pair<DIFF, true, NP>(P, l, m, sT, sAC, Spa, Spb, Sqa, Sqb, acc);
    for (; l <= L; l += 2) pm_syn_pair<DIFF, false, NP>(P, l, m, sT, sAC, Spa, Spb, Sqa, Sqb, acc);
}

// synthesis: CTA row per m, NP ring pairs per thread.  Shared staging per l
// (l = m + i, i < nl, zero-padded): sT[i] = (A, A be, B+, B-), sAC[i] =
// c_l (Re A, Im A, Re C, Im C) with A = E + iB, C = E - iB
template <int NP>
__global__ void __launch_bounds__(PM_THREADS) k_legsyn_pol_mx(int lmax, int L, int npairs,
                                                              const double2 *__restrict__ E,
                                                              const double2 *__restrict__ B,
                                                              const float4 *__restrict__ tab,
                                                              const double *__restrict__ c,
                                                              const int *__restrict__ ls_tab,
                                                              const float4 *__restrict__ seed,
                                                              const float *__restrict__ xp,
                                                              const float *__restrict__ wp, float2 *__restrict__ GQ,
                                                              float2 *__restrict__ GU)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m = blockIdx.y;
    const int nl = L - m + 1;
    const int ns = nl + 2;
    const long long base = pmb(lmax, m);
    float4 *sT = reinterpret_cast<float4 *>(smem_raw);
    float4 *sAC = sT + ns;
    for (int i = threadIdx.x; i < ns; i += blockDim.x) {
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f), ac = t;
        if (i < nl) {
            t = tab[base + i];
            const double2 e = E[base + i], b = B[base + i];
            const double cc = c[base + i];
            ac = make_float4((float)((e.x - b.y) * cc), (float)((e.y + b.x) * cc), (float)((e.x + b.y) * cc),
                             (float)((e.y - b.x) * cc));
        }
        sT[i] = t;
        sAC[i] = ac;
    }
    __syncthreads();
    const size_t pstride = (size_t)(lmax + 1) * 2;
    for (int p0 = (blockIdx.x * blockDim.x + threadIdx.x) * NP; p0 < npairs; p0 += gridDim.x * blockDim.x * NP) {
        PmPairs<NP> P;
        pm_load_pairs<NP>(P, m, L, npairs, p0, ls_tab, seed, xp, wp);
        PmAcc acc[NP / 2];
#pragma unroll
        for (int pk = 0; pk < NP / 2; ++pk)
#pragma unroll
            for (int h = 0; h < 2; ++h)
                acc[pk].ApR[h] = acc[pk].ApI[h] = acc[pk].AmR[h] = acc[pk].AmI[h] = acc[pk].CpR[h] =
                    acc[pk].CpI[h] = acc[pk].CmR[h] = acc[pk].CmI[h] = dup(0.f);
        // warp-uniform control flow, as in the temperature synthesis
        const unsigned am = __activemask();
        const int lmin = __reduce_min_sync(am, P.lmin), lmaxs = __reduce_max_sync(am, P.lmaxs);
        const bool diff = __shfl_sync(am, P.diff ? 1 : 0, __ffs(am) - 1) != 0;
        if (lmin <= L) {
            if (diff) pm_syn_run<true, NP>(P, m, L, sT, sAC, acc, lmin, lmaxs);
            else pm_syn_run<false, NP>(P, m, L, sT, sAC, acc, lmin, lmaxs);
        }
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const int p = p0 + k;
            if (p >= npairs) break;
            const int pk = k >> 1, h = k & 1;
            const PmAcc &a = acc[pk];
            // north: sum A mu+ + sum C mu-;  south: sum sigma A mu- + sum sigma C mu+
            const float sapNr = get(a.ApR[0], h) + get(a.ApR[1], h), sapNi = get(a.ApI[0], h) + get(a.ApI[1], h);
            const float scmNr = get(a.CmR[0], h) + get(a.CmR[1], h), scmNi = get(a.CmI[0], h) + get(a.CmI[1], h);
            const float sapSr = get(a.AmR[0], h) - get(a.AmR[1], h), sapSi = get(a.AmI[0], h) - get(a.AmI[1], h);
            const float scmSr = get(a.CpR[0], h) - get(a.CpR[1], h), scmSi = get(a.CpI[0], h) - get(a.CpI[1], h);
            float2 *gq = GQ + (size_t)p * pstride + 2 * (size_t)m;
            float2 *gu = GU + (size_t)p * pstride + 2 * (size_t)m;
            // Q = -(SAP + SCM),  U = i (SAP - SCM)
            gq[0] = make_float2(-(sapNr + scmNr), -(sapNi + scmNi));
            gq[1] = make_float2(-(sapSr + scmSr), -(sapSi + scmSi));
            gu[0] = make_float2(-(sapNi - scmNi), sapNr - scmNr);
            gu[1] = make_float2(-(sapSi - scmSi), sapSr - scmSr);
        }
    }
}

// warp reduce-scatter of CH values per lane: afterwards lane groups of
// 32 / CH lanes hold the sum over the warp of one value (the l of the chunk
// given by lane >> (5 - log2 CH))
template <int CH>
__device__ __forceinline__ void pm_rscatter(float (&vr)[CH], float (&vi)[CH], int lane)
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
                const float sr = up ? vr[i] : vr[i + half];
                const float kr = up ? vr[i + half] : vr[i];
                const float si = up ? vi[i] : vi[i + half];
                const float ki = up ? vi[i + half] : vi[i];
                vr[i] = kr + __shfl_xor_sync(0xffffffffu, sr, off);
                vi[i] = ki + __shfl_xor_sync(0xffffffffu, si, off);
            }
        } else {
            vr[0] += __shfl_xor_sync(0xffffffffu, vr[0], off);
            vi[0] += __shfl_xor_sync(0xffffffffu, vi[0], off);
        }
    }
}

// ring coefficients of one pack: G+ = FQ + i FU and G- = FQ - i FU of the
// north (N) and south (S) rings, real and imaginary parts
struct PmRing {
    float2 pNr, pNi, pSr, pSi, qNr, qNi, qSr, qSi;
};

template <bool DIFF, int NP>
__device__ __forceinline__ void pm_ana_run(const PmPairs<NP> &P, int m, int L, int lmin_w, int lmaxs_w,
                                           const float4 *__restrict__ sT, const PmRing (&G)[NP / 2], float2 *accP,
                                           float2 *accM, int lane)
{
    constexpr int NPK = NP / 2;
    float2 Spa[NPK], Spb[NPK], Sqa[NPK], Sqb[NPK], Vp0[NPK], Vp1[NPK], Vq0[NPK], Vq1[NPK];
#pragma unroll
    for (int pk = 0; pk < NPK; ++pk) Spa[pk] = Spb[pk] = Sqa[pk] = Sqb[pk] = dup(0.f);
    for (int l0 = lmin_w; l0 <= L; l0 += PM_CH) {
        float2 YPr[PM_CH], YPi[PM_CH], YMr[PM_CH], YMi[PM_CH];
        const bool inj = l0 <= lmaxs_w;
#pragma unroll
        for (int i = 0; i < PM_CH; i += 2) {
            const int j = l0 - m + i;
            const float4 t0 = sT[j], t1 = sT[j + 1];
            if (inj) pm_step<DIFF, true, NP>(P, l0 + i, t0, t1, Spa, Spb, Sqa, Sqb, Vp0, Vp1, Vq0, Vq1);
            else pm_step<DIFF, false, NP>(P, l0 + i, t0, t1, Spa, Spb, Sqa, Sqb, Vp0, Vp1, Vq0, Vq1);
            YPr[i] = YPi[i] = YMr[i] = YMi[i] = YPr[i + 1] = YPi[i + 1] = YMr[i + 1] = YMi[i + 1] = dup(0.f);
#pragma unroll
            for (int pk = 0; pk < NPK; ++pk) {
                const PmRing &g = G[pk];
                // even l (sigma = +1): YP += mu+ G+N + mu- G+S, YM += mu- G-N + mu+ G-S
                YPr[i] = __ffma2_rn(Vp0[pk], g.pNr, __ffma2_rn(Vq0[pk], g.pSr, YPr[i]));
                YPi[i] = __ffma2_rn(Vp0[pk], g.pNi, __ffma2_rn(Vq0[pk], g.pSi, YPi[i]));
                YMr[i] = __ffma2_rn(Vq0[pk], g.qNr, __ffma2_rn(Vp0[pk], g.qSr, YMr[i]));
                YMi[i] = __ffma2_rn(Vq0[pk], g.qNi, __ffma2_rn(Vp0[pk], g.qSi, YMi[i]));
                // odd l (sigma = -1)
                YPr[i + 1] = __ffma2_rn(Vp1[pk], g.pNr, __ffma2_rn(neg2(Vq1[pk]), g.pSr, YPr[i + 1]));
                YPi[i + 1] = __ffma2_rn(Vp1[pk], g.pNi, __ffma2_rn(neg2(Vq1[pk]), g.pSi, YPi[i + 1]));
                YMr[i + 1] = __ffma2_rn(Vq1[pk], g.qNr, __ffma2_rn(neg2(Vp1[pk]), g.qSr, YMr[i + 1]));
                YMi[i + 1] = __ffma2_rn(Vq1[pk], g.qNi, __ffma2_rn(neg2(Vp1[pk]), g.qSi, YMi[i + 1]));
            }
        }
        float pr[PM_CH], pi[PM_CH], mr[PM_CH], mi[PM_CH];
#pragma unroll
        for (int i = 0; i < PM_CH; ++i) {
            pr[i] = YPr[i].x + YPr[i].y;
            pi[i] = YPi[i].x + YPi[i].y;
            mr[i] = YMr[i].x + YMr[i].y;
            mi[i] = YMi[i].x + YMi[i].y;
        }
        pm_rscatter<PM_CH>(pr, pi, lane);
        pm_rscatter<PM_CH>(mr, mi, lane);
        constexpr int sh = 2;  // 32 lanes, 8 values: each l ends in 4 lanes
        if ((lane & ((1 << sh) - 1)) == 0) {
            const int l = l0 + (lane >> sh);
            if (l <= L) {
                atomicAdd(&accP[l - m].x, pr[0]);
                atomicAdd(&accP[l - m].y, pi[0]);
                atomicAdd(&accM[l - m].x, mr[0]);
                atomicAdd(&accM[l - m].y, mi[0]);
            }
        }
    }
}

// analysis: CTA per m; warps take groups of 32 x NP ring pairs from a shared
// counter; chunks of PM_CH values of l are summed over the packs in
// registers, reduced across the warp and added into FP32 shared
// accumulators; the epilogue scales by c_l, adds the FP64 block (l < lcm(lc, m))
// and writes E, B in FP64 (zero outside 2 <= l <= L).  Two CTAs per SM (128
// registers, a 96-byte spill) measured 17 % faster at nside 1024 than one CTA
// at 160 registers; chunks of 4 l (118 registers, no spill) and 2 or 8 pairs
// per lane were slower.
template <int NP>
__global__ void __launch_bounds__(PM_THREADS, 2) k_legana_pol_mx(int lmax, int L, int npairs, int lc,
                                                              const float2 *__restrict__ FQ,
                                                              const float2 *__restrict__ FU,
                                                              const float4 *__restrict__ tab,
                                                              const double *__restrict__ c,
                                                              const int *__restrict__ ls_tab,
                                                              const float4 *__restrict__ seed,
                                                              const float *__restrict__ xp,
                                                              const float *__restrict__ wp,
                                                              const double2 *__restrict__ Elow,
                                                              const double2 *__restrict__ Blow,
                                                              double2 *__restrict__ Eo, double2 *__restrict__ Bo)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int next_group;
    const int m = blockIdx.x;
    const int nl = L - m + 1;
    const int nlp = nl + PM_CH + 2;
    const long long base = pmb(lmax, m);
    float4 *sT = reinterpret_cast<float4 *>(smem_raw);
    float2 *accP = reinterpret_cast<float2 *>(sT + nlp);
    float2 *accM = accP + nlp;
    for (int i = threadIdx.x; i < nlp; i += blockDim.x) {
        sT[i] = (i < nl) ? tab[base + i] : make_float4(0.f, 0.f, 0.f, 0.f);
        accP[i] = accM[i] = make_float2(0.f, 0.f);
    }
    if (threadIdx.x == 0) next_group = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int per_group = 32 * NP;
    const int ngroups = (npairs + per_group - 1) / per_group;
    const size_t pstride = (size_t)(lmax + 1) * 2;
    for (;;) {
        int grp = 0;
        if (lane == 0) grp = atomicAdd(&next_group, 1);
        grp = __shfl_sync(0xffffffffu, grp, 0);
        if (grp >= ngroups) break;
        // equator first: the work per pair grows towards the equator (more l above the
        // first kept one), so handing out the largest groups first shortens the tail at the
        // barrier before the epilogue
        const int p0 = (ngroups - 1 - grp) * per_group + lane * NP;
        PmPairs<NP> P;
        pm_load_pairs<NP>(P, m, L, npairs, p0, ls_tab, seed, xp, wp);
        // one recurrence form per warp: the shuffles need warp-uniform control flow
        P.diff = __shfl_sync(0xffffffffu, P.diff ? 1 : 0, 0) != 0;
        const int lmin_w = __reduce_min_sync(0xffffffffu, P.lmin);
        const int lmaxs_w = __reduce_max_sync(0xffffffffu, P.lmaxs);  // one seeding range per warp
        if (lmin_w > L) continue;
        float g[8][NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
#pragma unroll
            for (int q = 0; q < 8; ++q) g[q][k] = 0.f;
            if (P.ls[k] != PM_BIG) {
                const size_t o = (size_t)(p0 + k) * pstride + 2 * (size_t)m;
                const float2 qn = FQ[o], qs = FQ[o + 1], un = FU[o], us = FU[o + 1];
                g[0][k] = qn.x - un.y;  // G+ north
                g[1][k] = qn.y + un.x;
                g[2][k] = qs.x - us.y;  // G+ south
                g[3][k] = qs.y + us.x;
                g[4][k] = qn.x + un.y;  // G- north
                g[5][k] = qn.y - un.x;
                g[6][k] = qs.x + us.y;  // G- south
                g[7][k] = qs.y - us.x;
            }
        }
        PmRing G[NP / 2];
#pragma unroll
        for (int pk = 0; pk < NP / 2; ++pk) {
            G[pk].pNr = make_float2(g[0][2 * pk], g[0][2 * pk + 1]);
            G[pk].pNi = make_float2(g[1][2 * pk], g[1][2 * pk + 1]);
            G[pk].pSr = make_float2(g[2][2 * pk], g[2][2 * pk + 1]);
            G[pk].pSi = make_float2(g[3][2 * pk], g[3][2 * pk + 1]);
            G[pk].qNr = make_float2(g[4][2 * pk], g[4][2 * pk + 1]);
            G[pk].qNi = make_float2(g[5][2 * pk], g[5][2 * pk + 1]);
            G[pk].qSr = make_float2(g[6][2 * pk], g[6][2 * pk + 1]);
            G[pk].qSi = make_float2(g[7][2 * pk], g[7][2 * pk + 1]);
        }
        if (P.diff) pm_ana_run<true, NP>(P, m, L, lmin_w, lmaxs_w, sT, G, accP, accM, lane);
        else pm_ana_run<false, NP>(P, m, L, lmin_w, lmaxs_w, sT, G, accP, accM, lane);
    }
    __syncthreads();
    const bool low = Elow && m < lc;
    const int llim = low ? lcm_of(lc, m) : 0;
    for (int j = threadIdx.x; j <= lmax - m; j += blockDim.x) {
        const int l = m + j;
        double2 e = make_double2(0.0, 0.0), b = e;
        if (l >= 2 && l <= L) {
            if (l < llim) {
                e = Elow[base + j];
                b = Blow[base + j];
            } else {
                const double cc = c[base + j];
                const double ypr = accP[j].x, ypi = accP[j].y, ymr = accM[j].x, ymi = accM[j].y;
                e = make_double2(-cc * (ypr + ymr), -cc * (ypi + ymi));
                b = make_double2(-cc * (ypi - ymi), cc * (ypr - ymr));
            }
        }
        Eo[base + j] = e;
        Bo[base + j] = b;
    }
}

template <int NP> size_t syn_pm_smem(int L, int m0) { return (size_t)2 * (L - m0 + 3) * sizeof(float4) + 16; }
size_t ana_pm_smem(int L) { return (size_t)(L + 1 + PM_CH + 2) * (sizeof(float4) + 2 * sizeof(float2)) + 16; }

constexpr int SYN_NP = 4;  // ring pairs per thread (synthesis)
constexpr int ANA_NP = 4;  // ring pairs per lane (analysis)

}  // namespace

// mu-form tables (FP64 on the host, FP32 on the device) and the x, w rings
wf_status hp_pol_create_mx(wf_plan p)
{
    PolState *s = p->pol;
    const int lmax = p->lmax, np = p->npairs;
    const long long nalm = p->nalm, ns = (long long)(lmax + 1) * np;
    std::vector<double> c(nalm, 1.0);
    std::vector<float4> tab(nalm, make_float4(0.f, 0.f, 0.f, 0.f));
    std::vector<double> al(lmax + 2), be(lmax + 2), ga(lmax + 2);
    for (int m = 0; m <= lmax; ++m) {
        const long long b = pmb(lmax, m);
        const int l0 = std::max(m, 2);
        if (l0 > lmax) continue;
        const double mm = m;
        for (int l = l0 + 1; l <= lmax; ++l) {
            const double L = l, L1 = L - 1.0;
            const double d = std::sqrt((L * L - mm * mm) * (L * L - 4.0));
            al[l] = std::sqrt((2.0 * L + 1.0) * (2.0 * L - 1.0)) * L / d;
            be[l] = 2.0 * mm / (L * (L - 1.0));
            ga[l] = L * std::sqrt((2.0 * L + 1.0) / (2.0 * L - 3.0)) *
                    std::sqrt(std::max(0.0, (L1 * L1 - mm * mm) * (L1 * L1 - 4.0))) / (L1 * d);
        }
        // c = 1 at l0 and l0 + 1, c_l = ga_l c_{l-2}
        for (int l = l0 + 2; l <= lmax; ++l) c[b + (l - m)] = ga[l] * c[b + (l - 2 - m)];
        // rescale the chain of l0 + 1 so that c_lmax = c_{lmax-1} (A -> 2)
        if (lmax - l0 >= 2) {
            const double r = c[b + (lmax - m)] / c[b + (lmax - 1 - m)];
            const double f = ((lmax - l0) & 1) ? 1.0 / r : r;
            for (int l = l0 + 1; l <= lmax; l += 2) c[b + (l - m)] *= f;
        }
        for (int l = l0 + 1; l <= lmax; ++l) {
            const double A = al[l] * c[b + (l - 1 - m)] / c[b + (l - m)];
            const double Ab = A * be[l];
            tab[b + (l - m)] = make_float4((float)A, (float)Ab, (float)((A - 2.0) + Ab), (float)((A - 2.0) - Ab));
        }
    }
    wf_status st;
    if ((st = plan_alloc(p, (void **)&s->c, nalm * sizeof(double))) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&s->tab, nalm * sizeof(float4))) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&s->ls_mx, ns * sizeof(int))) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&s->seed, ns * sizeof(float4))) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&s->Elow, nalm * sizeof(double2))) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&s->Blow, nalm * sizeof(double2))) != WF_OK) return st;
    if ((st = to_device(p, s->c, c.data(), nalm * sizeof(double))) != WF_OK) return st;
    if ((st = to_device(p, s->tab, tab.data(), nalm * sizeof(float4))) != WF_OK) return st;
    if (tc_prec(p->prec) && (st = plan_alloc(p, (void **)&s->ac32, nalm * sizeof(float4))) != WF_OK) return st;
    s->lc = -1;
    if ((st = hp_pol_set_low_block(p, 0)) != WF_OK) return st;
    const size_t syn_max = syn_pm_smem<SYN_NP>(lmax, 0), ana_max = ana_pm_smem(lmax);
    if ((st = raise_smem_limit((const void *)k_legsyn_pol_mx<SYN_NP>, syn_max)) != WF_OK) return st;
    if ((st = raise_smem_limit((const void *)k_legana_pol_mx<ANA_NP>, ana_max)) != WF_OK) return st;
    return WF_OK;
}

// select the FP64 block l < lcm(lc, m) and rebuild the FP32 seeds (cached per lc)
wf_status hp_pol_set_low_block(wf_plan p, int lc)
{
    PolState *s = p->pol;
    if (!s || p->prec == WF_PREC_FP64) return WF_OK;
    if (lc < 0) lc = 0;
    if (lc > p->lmax + 1) lc = p->lmax + 1;
    if (lc == s->lc) return WF_OK;
    const long long ns = (long long)(p->lmax + 1) * p->npairs;
    const int th = 256;
    k_pol_seeds_mx<<<(unsigned)((ns + th - 1) / th), th, 0, p->stream>>>(
        p->lmax, p->npairs, lc, p->tab.x64, s->al, s->be, s->ga, s->c, s->ls, s->p0, s->p1, s->m0, s->m1, s->ls_mx,
        s->seed);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    if (lc > 0 && lc > s->low_cap) {
        const size_t bytes = (size_t)p->npairs * lc * 2 * sizeof(float2);
        wf_status st;
        if ((st = plan_alloc(p, (void **)&s->GQlow, bytes)) != WF_OK) return st;
        if ((st = plan_alloc(p, (void **)&s->GUlow, bytes)) != WF_OK) return st;
        s->low_cap = lc;
    }
    s->lc = lc;
    return WF_OK;
}

// (E, B) -> FP32 ring coefficients of Q and U (GQ, GU), l <= L; the FP64 block
// (when lc > 0) into GQlow / GUlow, which the ring synthesis adds
wf_status hp_pol_legendre_synthesis_mx(wf_plan p, const double2 *E, const double2 *B, int L)
{
    PolState *s = p->pol;
    const HpTables &t = p->tab;
    wf_status st;
    if (s->lc > 0 && (st = hp_pol_legendre_synthesis_low(p, E, B, L, s->lc, s->GQlow, s->GUlow)) != WF_OK) return st;
    if (tc_prec(p->prec)) {
        // on the tensor cores; in a batch step the group launch (wf_solve_batch) has written GQ, GU already
        if (p->tc_deferred) return WF_OK;
        float2 *gq = (float2 *)s->GQ, *gu = (float2 *)s->GU;
        return hp_pol_tc_synthesis(p, 1, &E, &B, &s->ac32, &gq, &gu, &L, L, p->stream);
    }
    const int per_cta = PM_THREADS * SYN_NP;
    dim3 grid((p->npairs + per_cta - 1) / per_cta, L + 1);
    k_legsyn_pol_mx<SYN_NP><<<grid, PM_THREADS, syn_pm_smem<SYN_NP>(L, 0), p->stream>>>(
        p->lmax, L, p->npairs, E, B, s->tab, s->c, s->ls_mx, s->seed, t.x32, t.w32, (float2 *)s->GQ, (float2 *)s->GU);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    return WF_OK;
}

// FP32 ring coefficients (FQ, FU) -> (E, B) in FP64, l <= L (zero above; columns
// m > L zeroed)
wf_status hp_pol_legendre_analysis_mx(wf_plan p, int L, double2 *E, double2 *B)
{
    PolState *s = p->pol;
    const HpTables &t = p->tab;
    wf_status st;
    const bool low = s->lc > 0;
    if (low && (st = hp_pol_legendre_analysis_low(p, L, s->lc, (const float2 *)s->FQ, (const float2 *)s->FU,
                                                  s->Elow, s->Blow)) != WF_OK)
        return st;
    k_legana_pol_mx<ANA_NP><<<L + 1, PM_THREADS, ana_pm_smem(L), p->stream>>>(
        p->lmax, L, p->npairs, s->lc, (const float2 *)s->FQ, (const float2 *)s->FU, s->tab, s->c, s->ls_mx, s->seed,
        t.x32, t.w32, low ? s->Elow : nullptr, low ? s->Blow : nullptr, E, B);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    if (L < p->lmax) {
        const long long from = pmb(p->lmax, L + 1);
        WF_CUDA(cudaMemsetAsync(E + from, 0, (p->nalm - from) * sizeof(double2), p->stream));
        WF_CUDA(cudaMemsetAsync(B + from, 0, (p->nalm - from) * sizeof(double2), p->stream));
    }
    return WF_OK;
}

}  // namespace wf
