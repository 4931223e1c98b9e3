// Polarisation: the spin-2 half of the basis change for (I, Q, U) maps and the
// 3x3 blends of the polarised messenger iteration (Eqs. 10-11).  The spin-2
// Legendre kernels here are FP64: the whole transform of FP64 plans, and the
// low-l block of mixed plans (whose FP32 kernels are in wf_spin_mx.cu).
//
// Convention: sY_lm = slambda_lm(theta) e^{i m phi}, slambda_lm =
// sqrt((2l+1)/(4 pi)) d^l_{m,-s}(theta) (s = 0: the Condon-Shortley Y_lm of
// the temperature path); (Q + iU) = sum_{l>=2, |m|<=l} 2a_lm 2Y_lm with
// 2a = -(E + iB).  In terms of W = (2lambda + -2lambda)/2 and
// X = (2lambda - -2lambda)/2 (m >= 0), the ring coefficients are
//     Q_m = -sum_l (E_lm W_lm + i B_lm X_lm),   U_m = -sum_l (B_lm W_lm - i E_lm X_lm),
// and Q, U are real ring DFTs of them, like the temperature map.  Wigner's
// recurrence in l carries P = 2lambda/2 and M = -2lambda/2 separately
// (b = -s = -+2 flips the sign of its middle term):
//     P_l = al_l (x + be_l) P_{l-1} - ga_l P_{l-2},   M_l = al_l (x - be_l) M_{l-1} - ga_l M_{l-2},
//     al_l = sqrt((2l+1)(2l-1)) l / sqrt((l^2-m^2)(l^2-4)),  be_l = 2m / (l(l-1)),
//     ga_l = l sqrt((2l+1)/(2l-3)) sqrt(((l-1)^2-m^2)((l-1)^2-4)) / ((l-1) sqrt((l^2-m^2)(l^2-4))),
// and W = P + M, X = P - M at each l.  (Recurring W and X as a coupled pair
// is the same arithmetic on paper but not in rounding: near the poles
// -2lambda is orders of magnitude below 2lambda and grows faster in l, so
// the coupling feeds it rounding errors of 2lambda's size; at nside 64 that
// costs 1e-11 relative, against 1e-14 for the separate recurrences.)
// Mirror symmetry: W(pi - theta) = (-1)^(l+m) W, X(pi - theta) = -(-1)^(l+m) X,
// so a north/south ring pair keeps even and odd partial sums (as for T).
// Seeds at l0 = max(m, 2) from Wigner's explicit sum (one term there), carried
// in FP64 with a binary exponent up to the first l where |P| or |M| exceeds
// 2^-81 (terms below are dropped), as for the temperature seeds.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "wf_internal.cuh"

namespace wf {

namespace {

constexpr int POL_THREADS = 256;
constexpr int POL_CH = 8;
constexpr double POL_SEED_LOG2_MIN = -80.0;

__host__ __device__ inline long long pmbase(int lmax, int m) { return (long long)m * (2 * lmax + 3 - m) / 2; }

__device__ __forceinline__ double2 cmad(double2 acc, double2 a, double w)
{
    acc.x = fma(a.x, w, acc.x);
    acc.y = fma(a.y, w, acc.y);
    return acc;
}
__device__ __forceinline__ double2 times_i(double2 z) { return make_double2(-z.y, z.x); }
__device__ __forceinline__ double2 dadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 dsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 dneg(double2 a) { return make_double2(-a.x, -a.y); }

// recurrence coefficients per (l, m), zero at l <= max(m, 2)
__global__ void k_pol_coefs(int lmax, double *__restrict__ al, double *__restrict__ be, double *__restrict__ ga)
{
    const int m = blockIdx.x;
    const long long base = pmbase(lmax, m);
    const int l0 = m > 2 ? m : 2;
    for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
        double a = 0.0, b = 0.0, g = 0.0;
        if (l > l0) {
            const double L = l, mm = m;
            const double d = sqrt((L * L - mm * mm) * (L * L - 4.0));
            a = sqrt((2.0 * L + 1.0) * (2.0 * L - 1.0)) * L / d;
            b = 2.0 * mm / (L * (L - 1.0));
            const double L1 = L - 1.0;
            g = L * sqrt((2.0 * L + 1.0) / (2.0 * L - 3.0)) * sqrt(fmax(0.0, (L1 * L1 - mm * mm) * (L1 * L1 - 4.0))) /
                (L1 * d);
        }
        al[base + (l - m)] = a;
        be[base + (l - m)] = b;
        ga[base + (l - m)] = g;
    }
}

// log2 |slambda_{l0 m}| and its sign, l0 = max(m, 2), from the single term of
// Wigner's explicit sum (b = -s)
__device__ void spin_seed(int m, int s, double ch, double sh, double *lg2, int *sign)
{
    const int a = m, b = -s;
    const int j = (a > 2 ? a : 2);
    int kk;
    if (a == j) kk = 0;
    else if (b == j) kk = j - a;
    else kk = 0;  // b == -j
    const int ec = 2 * j + b - a - 2 * kk, es = a - b + 2 * kk;
    double lg = 0.5 * (lgamma(j + a + 1.0) + lgamma(j - a + 1.0) + lgamma(j + b + 1.0) + lgamma(j - b + 1.0)) -
                (lgamma(j + b - kk + 1.0) + lgamma(kk + 1.0) + lgamma(a - b + kk + 1.0) + lgamma(j - a - kk + 1.0));
    lg += 0.5 * log((2.0 * j + 1.0) / (4.0 * M_PI));
    if (ec > 0) lg += ec * log(ch);
    if (es > 0) lg += es * log(sh);
    *lg2 = lg / log(2.0);
    *sign = ((a - b + kk) & 1) ? -1 : 1;
}

// per (m, pair): first l whose P or M reaches 2^-81, and P, M at ls and ls + 1
__global__ void k_seeds_pol(int lmax, int npairs, const double *__restrict__ xp, const double *__restrict__ stp,
                            const double *__restrict__ al, const double *__restrict__ be,
                            const double *__restrict__ ga, int *__restrict__ ls_out, double *__restrict__ p0,
                            double *__restrict__ p1, double *__restrict__ m0, double *__restrict__ m1)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)(lmax + 1) * npairs) return;
    const int m = (int)(idx / npairs), p = (int)(idx % npairs);
    const double x = xp[p], st = stp[p];
    double ch, sh;
    if (x >= 0.0) {
        ch = sqrt(0.5 * (1.0 + x));
        sh = st / (2.0 * ch);
    } else {
        sh = sqrt(0.5 * (1.0 - x));
        ch = st / (2.0 * sh);
    }
    const int l0 = m > 2 ? m : 2;
    int ls = lmax + 1;
    double P0 = 0, P1 = 0, M0 = 0, M1 = 0;
    if (l0 <= lmax) {
        double lp, lm;
        int sp, sm;
        spin_seed(m, 2, ch, sh, &lp, &sp);
        spin_seed(m, -2, ch, sh, &lm, &sm);
        int E = (int)floor(fmax(lp, lm));
        double P = 0.5 * sp * exp2(lp - E), M = 0.5 * sm * exp2(lm - E), Pp = 0.0, Mp = 0.0;
        const long long base = pmbase(lmax, m);
        int l = l0;
        double thr = ldexp(1.0, (int)POL_SEED_LOG2_MIN - 1 - E);
        for (;;) {
            if (fmax(fabs(P), fabs(M)) >= thr) break;
            if (l >= lmax) { l = lmax + 1; break; }
            const long long k = base + (l + 1 - m);
            const double Pn = fma(al[k] * (x + be[k]), P, -ga[k] * Pp);
            const double Mn = fma(al[k] * (x - be[k]), M, -ga[k] * Mp);
            Pp = P;
            Mp = M;
            P = Pn;
            M = Mn;
            ++l;
            if (fmax(fabs(P), fabs(M)) > 0x1p+500) {
                P *= 0x1p-500;
                M *= 0x1p-500;
                Pp *= 0x1p-500;
                Mp *= 0x1p-500;
                E += 500;
                thr = ldexp(1.0, (int)POL_SEED_LOG2_MIN - 1 - E);
            }
        }
        if (l <= lmax) {
            ls = l;
            P0 = ldexp(P, E);
            M0 = ldexp(M, E);
            if (l < lmax) {
                const long long k = base + (l + 1 - m);
                P1 = ldexp(fma(al[k] * (x + be[k]), P, -ga[k] * Pp), E);
                M1 = ldexp(fma(al[k] * (x - be[k]), M, -ga[k] * Mp), E);
            }
        }
    }
    ls_out[idx] = ls;
    p0[idx] = P0;
    p1[idx] = P1;
    m0[idx] = M0;
    m1[idx] = M1;
}

// first l of the FP32 range for m < lc (mixed plans): lc rounded up to the
// parity of m, as for the temperature kernels; the FP64 kernels then cover
// l < lcm_of(lc, m) for those m
__host__ __device__ inline int lcm_of(int lc, int m) { return m + 2 * ((lc - m + 1) / 2); }

// synthesis: (E, B) -> ring coefficients (Q_m, U_m) of both rings of each pair,
// l <= L (and l < lcm_of(lcut, m) when lcut > 0: the FP64 block of a mixed
// plan); output [pair][m][hemisphere] with gstride columns per pair, in TG
template <typename TG>
__global__ void __launch_bounds__(POL_THREADS) k_legsyn_pol(int lmax, int L, int lcut, int gstride, int npairs,
                                                            const double2 *__restrict__ E,
                                                            const double2 *__restrict__ B,
                                                            const double *__restrict__ al,
                                                            const double *__restrict__ be,
                                                            const double *__restrict__ ga,
                                                            const int *__restrict__ ls_tab,
                                                            const double *__restrict__ p0t,
                                                            const double *__restrict__ p1t,
                                                            const double *__restrict__ m0t,
                                                            const double *__restrict__ m1t,
                                                            const double *__restrict__ xp, cx<TG> *__restrict__ GQ,
                                                            cx<TG> *__restrict__ GU)
{
    const int m = blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npairs) return;
    const long long base = pmbase(lmax, m);
    const size_t sidx = (size_t)m * npairs + p;
    const int ls = ls_tab[sidx];
    if (lcut > 0) L = min(L, lcm_of(lcut, m) - 1);
    const double2 z = make_double2(0.0, 0.0);
    double2 EWe = z, EWo = z, BXe = z, BXo = z, BWe = z, BWo = z, EXe = z, EXo = z;
    if (ls <= L) {
        const double x = xp[p];
        double P = p0t[sidx], M = m0t[sidx], Pn = p1t[sidx], Mn = m1t[sidx], Pp = 0.0, Mp = 0.0;
        for (int l = ls; l <= L; ++l) {
            if (l > ls + 1) {
                const long long k = base + (l - m);
                Pn = fma(al[k] * (x + be[k]), P, -ga[k] * Pp);
                Mn = fma(al[k] * (x - be[k]), M, -ga[k] * Mp);
            }
            if (l > ls) {
                Pp = P;
                Mp = M;
                P = Pn;
                M = Mn;
            }
            const double W = P + M, X = P - M;
            const double2 e = E[base + (l - m)], b = B[base + (l - m)];
            if (((l + m) & 1) == 0) {
                EWe = cmad(EWe, e, W);
                BXe = cmad(BXe, b, X);
                BWe = cmad(BWe, b, W);
                EXe = cmad(EXe, e, X);
            } else {
                EWo = cmad(EWo, e, W);
                BXo = cmad(BXo, b, X);
                BWo = cmad(BWo, b, W);
                EXo = cmad(EXo, e, X);
            }
        }
    }
    // north ring: sigma = +1 for both parities; south ring: W -> sigma W, X -> -sigma X
    const double2 QN = dneg(dadd(dadd(EWe, EWo), times_i(dadd(BXe, BXo))));
    const double2 QS = dneg(dsub(dsub(EWe, EWo), times_i(dsub(BXe, BXo))));
    const double2 UN = dneg(dsub(dadd(BWe, BWo), times_i(dadd(EXe, EXo))));
    const double2 US = dneg(dadd(dsub(BWe, BWo), times_i(dsub(EXe, EXo))));
    const size_t o = ((size_t)p * gstride + m) * 2;
    GQ[o] = mk<TG>((TG)QN.x, (TG)QN.y);
    GQ[o + 1] = mk<TG>((TG)QS.x, (TG)QS.y);
    GU[o] = mk<TG>((TG)UN.x, (TG)UN.y);
    GU[o + 1] = mk<TG>((TG)US.x, (TG)US.y);
}

// warp reduce-scatter (same pattern as the temperature analysis)
template <int CH>
__device__ __forceinline__ void rscatter(double (&vr)[CH], double (&vi)[CH], int lane)
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
                const double sr = up ? vr[i] : vr[i + half];
                const double kr = up ? vr[i + half] : vr[i];
                const double si = up ? vi[i] : vi[i + half];
                const double ki = up ? vi[i + half] : vi[i];
                vr[i] = kr + __shfl_xor_sync(0xffffffffu, sr, off);
                vi[i] = ki + __shfl_xor_sync(0xffffffffu, si, off);
            }
        } else {
            vr[0] += __shfl_xor_sync(0xffffffffu, vr[0], off);
            vi[0] += __shfl_xor_sync(0xffffffffu, vi[0], off);
        }
    }
}

// analysis (the adjoint of k_legsyn_pol): ring coefficients FQ, FU of both
// rings of each pair -> (E, B);  E = -sum_r (W FQ + i X FU), B = -sum_r (W FU - i X FQ);
// l <= L (and l < lcm_of(lcut, m) when lcut > 0); ring coefficients in TF
template <typename TF>
__global__ void __launch_bounds__(POL_THREADS) k_legana_pol(int lmax, int L, int lcut, int npairs,
                                                            const cx<TF> *__restrict__ FQ,
                                                            const cx<TF> *__restrict__ FU,
                                                            const double *__restrict__ al,
                                                            const double *__restrict__ be,
                                                            const double *__restrict__ ga,
                                                            const int *__restrict__ ls_tab,
                                                            const double *__restrict__ p0t,
                                                            const double *__restrict__ p1t,
                                                            const double *__restrict__ m0t,
                                                            const double *__restrict__ m1t,
                                                            const double *__restrict__ xp, double2 *__restrict__ Eo,
                                                            double2 *__restrict__ Bo)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m = blockIdx.x;
    if (lcut > 0) L = min(L, lcm_of(lcut, m) - 1);
    const int nl = max(L - m + 1, 0);
    const long long base = pmbase(lmax, m);
    double2 *accE = reinterpret_cast<double2 *>(smem_raw);
    double2 *accB = accE + (nl + POL_CH + 2);
    for (int i = threadIdx.x; i < nl + POL_CH + 2; i += blockDim.x) accE[i] = accB[i] = make_double2(0.0, 0.0);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int ngroups = (npairs + 31) / 32;
    // gridDim.y > 1 splits the ring pairs of each m over CTAs (the FP64 block of
    // mixed plans: its few m would otherwise leave most SMs idle); they add
    // their sums into pre-zeroed outputs
    for (int grp = warp + nwarps * blockIdx.y; grp < ngroups; grp += nwarps * gridDim.y) {
        const int p = grp * 32 + lane;
        const size_t sidx = (size_t)m * npairs + p;
        int ls = (p < npairs) ? ls_tab[sidx] : lmax + 1;
        if (ls > L) ls = 1 << 29;
        const int lmin = __reduce_min_sync(0xffffffffu, ls);
        if (lmin > L) continue;
        double2 Pq = make_double2(0, 0), Mq = Pq, Pu = Pq, Mu = Pq;
        double x = 0.0, P0 = 0.0, P1 = 0.0, M0 = 0.0, M1 = 0.0;
        if (ls <= L) {
            const size_t o = ((size_t)p * (lmax + 1) + m) * 2;
            const cx<TF> fq0 = FQ[o], fq1 = FQ[o + 1], fu0 = FU[o], fu1 = FU[o + 1];
            const double2 qn = make_double2(fq0.x, fq0.y), qs = make_double2(fq1.x, fq1.y);
            const double2 un = make_double2(fu0.x, fu0.y), us = make_double2(fu1.x, fu1.y);
            Pq = dadd(qn, qs);
            Mq = dsub(qn, qs);
            Pu = dadd(un, us);
            Mu = dsub(un, us);
            x = xp[p];
            P0 = p0t[sidx];
            P1 = p1t[sidx];
            M0 = m0t[sidx];
            M1 = m1t[sidx];
        }
        double P = 0.0, M = 0.0, Pp = 0.0, Mp = 0.0;
        for (int l0 = lmin; l0 <= L; l0 += POL_CH) {
            double er[POL_CH], ei[POL_CH], br[POL_CH], bi[POL_CH];
#pragma unroll
            for (int i = 0; i < POL_CH; ++i) {
                const int l = l0 + i;
                if (l == ls) {
                    P = P0;
                    M = M0;
                } else if (l == ls + 1) {
                    Pp = P;
                    Mp = M;
                    P = P1;
                    M = M1;
                } else if (l > ls + 1 && l <= L) {
                    const long long k = base + (l - m);
                    const double Pn = fma(al[k] * (x + be[k]), P, -ga[k] * Pp);
                    const double Mn = fma(al[k] * (x - be[k]), M, -ga[k] * Mp);
                    Pp = P;
                    Mp = M;
                    P = Pn;
                    M = Mn;
                }
                const double W = P + M, X = P - M;
                double2 e = make_double2(0, 0), b = e;
                if (l >= ls && l <= L) {
                    // sigma = +1: (Pq, Mu; Pu, Mq); sigma = -1: (Mq, Pu; Mu, Pq)
                    const bool even = ((l + m) & 1) == 0;
                    const double2 fqw = even ? Pq : Mq, fux = even ? Mu : Pu;
                    const double2 fuw = even ? Pu : Mu, fqx = even ? Mq : Pq;
                    e = dneg(dadd(make_double2(W * fqw.x, W * fqw.y), times_i(make_double2(X * fux.x, X * fux.y))));
                    b = dneg(dsub(make_double2(W * fuw.x, W * fuw.y), times_i(make_double2(X * fqx.x, X * fqx.y))));
                }
                er[i] = e.x;
                ei[i] = e.y;
                br[i] = b.x;
                bi[i] = b.y;
            }
            rscatter<POL_CH>(er, ei, lane);
            rscatter<POL_CH>(br, bi, lane);
            constexpr int sh = 2;  // 32 lanes, 8 values: each l ends in 4 lanes
            if ((lane & ((1 << sh) - 1)) == 0) {
                const int l = l0 + (lane >> sh);
                if (l <= L) {
                    atomicAdd(&accE[l - m].x, er[0]);
                    atomicAdd(&accE[l - m].y, ei[0]);
                    atomicAdd(&accB[l - m].x, br[0]);
                    atomicAdd(&accB[l - m].y, bi[0]);
                }
            }
        }
    }
    __syncthreads();
    if (gridDim.y > 1) {
        for (int j = threadIdx.x; j < nl; j += blockDim.x) {
            if (m + j < 2) continue;
            atomicAdd(&Eo[base + j].x, accE[j].x);
            atomicAdd(&Eo[base + j].y, accE[j].y);
            atomicAdd(&Bo[base + j].x, accB[j].x);
            atomicAdd(&Bo[base + j].y, accB[j].y);
        }
        return;
    }
    for (int j = threadIdx.x; j <= lmax - m; j += blockDim.x) {
        const int l = m + j;
        const bool in = l <= L && l >= 2;
        Eo[base + j] = in ? accE[j] : make_double2(0.0, 0.0);
        Bo[base + j] = in ? accB[j] : make_double2(0.0, 0.0);
    }
}

// ---------------------------------------------------------------------------
// pixel side: 3x3 symmetric blocks stored as 6 maps (II, QQ, UU, IQ, IU, QU)
// ---------------------------------------------------------------------------
struct Sym3 {
    double a, b, c, d, e, f;  // [[a d e] [d b f] [e f c]]
};

__device__ __forceinline__ Sym3 load6(const double *__restrict__ v, long long n, long long p)
{
    return Sym3{v[p], v[n + p], v[2 * n + p], v[3 * n + p], v[4 * n + p], v[5 * n + p]};
}
__device__ __forceinline__ void store6(double *__restrict__ v, long long n, long long p, const Sym3 &s)
{
    v[p] = s.a;
    v[n + p] = s.b;
    v[2 * n + p] = s.c;
    v[3 * n + p] = s.d;
    v[4 * n + p] = s.e;
    v[5 * n + p] = s.f;
}
__device__ __forceinline__ double det3(const Sym3 &s)
{
    return s.a * (s.b * s.c - s.f * s.f) - s.d * (s.d * s.c - s.f * s.e) + s.e * (s.d * s.f - s.b * s.e);
}
__device__ __forceinline__ Sym3 inv3(const Sym3 &s)
{
    const double id = 1.0 / det3(s);
    return Sym3{(s.b * s.c - s.f * s.f) * id, (s.a * s.c - s.e * s.e) * id, (s.a * s.b - s.d * s.d) * id,
                (s.e * s.f - s.d * s.c) * id, (s.d * s.f - s.b * s.e) * id, (s.d * s.e - s.a * s.f) * id};
}
__device__ __forceinline__ void mv3(const Sym3 &s, const double (&v)[3], double (&o)[3])
{
    o[0] = s.a * v[0] + s.d * v[1] + s.e * v[2];
    o[1] = s.d * v[0] + s.b * v[1] + s.f * v[2];
    o[2] = s.e * v[0] + s.f * v[1] + s.c * v[2];
}
// smallest eigenvalue of a symmetric 3x3 matrix (Smith 1961: trigonometric
// solution of the characteristic cubic)
__device__ double eigmin3(const Sym3 &s)
{
    const double p1 = s.d * s.d + s.e * s.e + s.f * s.f;
    if (p1 == 0.0) return fmin(s.a, fmin(s.b, s.c));
    const double q = (s.a + s.b + s.c) / 3.0;
    const double p2 = (s.a - q) * (s.a - q) + (s.b - q) * (s.b - q) + (s.c - q) * (s.c - q) + 2.0 * p1;
    const double pp = sqrt(p2 / 6.0);
    const Sym3 Bm{(s.a - q) / pp, (s.b - q) / pp, (s.c - q) / pp, s.d / pp, s.e / pp, s.f / pp};
    const double r = fmin(1.0, fmax(-1.0, det3(Bm) / 2.0));
    const double phi = acos(r) / 3.0;
    return q + 2.0 * pp * cos(phi + 2.0 * M_PI / 3.0);
}

// all three eigenvalues, descending (same trigonometric solution)
__device__ void eig3(const Sym3 &s, double (&l)[3])
{
    const double p1 = s.d * s.d + s.e * s.e + s.f * s.f;
    if (p1 == 0.0) {
        l[0] = s.a;
        l[1] = s.b;
        l[2] = s.c;
        return;
    }
    const double q = (s.a + s.b + s.c) / 3.0;
    const double p2 = (s.a - q) * (s.a - q) + (s.b - q) * (s.b - q) + (s.c - q) * (s.c - q) + 2.0 * p1;
    const double pp = sqrt(p2 / 6.0);
    const Sym3 Bm{(s.a - q) / pp, (s.b - q) / pp, (s.c - q) / pp, s.d / pp, s.e / pp, s.f / pp};
    const double r = fmin(1.0, fmax(-1.0, det3(Bm) / 2.0));
    const double phi = acos(r) / 3.0;
    l[0] = q + 2.0 * pp * cos(phi);
    l[2] = q + 2.0 * pp * cos(phi + 2.0 * M_PI / 3.0);
    l[1] = 3.0 * q - l[0] - l[2];
}

// X Y for symmetric X, Y that commute (so X Y is symmetric), symmetrised
__device__ __forceinline__ Sym3 symmul(const Sym3 &X, const Sym3 &Y)
{
    const double p00 = X.a * Y.a + X.d * Y.d + X.e * Y.e, p11 = X.d * Y.d + X.b * Y.b + X.f * Y.f;
    const double p22 = X.e * Y.e + X.f * Y.f + X.c * Y.c;
    const double p01 = X.a * Y.d + X.d * Y.b + X.e * Y.f, p10 = X.d * Y.a + X.b * Y.d + X.f * Y.e;
    const double p02 = X.a * Y.e + X.d * Y.f + X.e * Y.c, p20 = X.e * Y.a + X.f * Y.d + X.c * Y.e;
    const double p12 = X.d * Y.e + X.b * Y.f + X.f * Y.c, p21 = X.e * Y.d + X.f * Y.b + X.c * Y.f;
    return Sym3{p00, p11, p22, 0.5 * (p01 + p10), 0.5 * (p02 + p20), 0.5 * (p12 + p21)};
}

// symmetric square root of a symmetric positive definite 3x3 block.  With
// mu_i = sqrt(lambda_i) and I1, I2, I3 the invariants of U = A^1/2, the
// Cayley-Hamilton theorem for U (U^3 - I1 U^2 + I2 U - I3 = 0, U^2 = A) gives
// U = (A + I2)^-1 (I1 A + I3); the invariants are symmetric in the eigenvalues,
// so a close pair (where the trigonometric roots lose half their digits) costs
// only second order.  One Newton step U <- (U + A U^-1) / 2 then restores full
// accuracy for ill-conditioned blocks.
__device__ Sym3 sqrt3(const Sym3 &A)
{
    double l[3];
    eig3(A, l);
    const double m0 = sqrt(fmax(l[0], 0.0)), m1 = sqrt(fmax(l[1], 0.0)), m2 = sqrt(fmax(l[2], 0.0));
    const double I1 = m0 + m1 + m2, I2 = m0 * m1 + m0 * m2 + m1 * m2, I3 = m0 * m1 * m2;
    const Sym3 K{A.a + I2, A.b + I2, A.c + I2, A.d, A.e, A.f};
    const Sym3 R{I1 * A.a + I3, I1 * A.b + I3, I1 * A.c + I3, I1 * A.d, I1 * A.e, I1 * A.f};
    const Sym3 U = symmul(inv3(K), R);
    const Sym3 AUi = symmul(A, inv3(U));
    return Sym3{0.5 * (U.a + AUi.a), 0.5 * (U.b + AUi.b), 0.5 * (U.c + AUi.c),
                0.5 * (U.d + AUi.d), 0.5 * (U.e + AUi.e), 0.5 * (U.f + AUi.f)};
}

__device__ __forceinline__ void atomic_min_posd(double *addr, double v)
{
    atomicMin(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

// Per-pixel mask codes of polarised plans: 0 nothing observed, 1 I, Q, U,
// 2 I only (polarisation masked), 3 Q, U only (temperature masked).  Masking
// is infinite noise (N^-1 = 0, Sect. 2.1) component by component: nu is the
// inverse of the observed sub-block, zero in the other rows and columns (its
// limit as the unobserved variances grow), r = nu d, and tau is the smallest
// eigenvalue of any observed sub-block.  Counts observed components (n_dof)
// and flags invalid inputs: a code above 3, or an observed sub-block that is
// not finite and positive definite, or observed d not finite.
__global__ void k_setup_pol(long long npix, const double *__restrict__ d, const double *__restrict__ N6,
                            const uint8_t *__restrict__ mask, double *__restrict__ r, double *__restrict__ nu6,
                            double *__restrict__ scal, int *__restrict__ flag)
{
    double tmin = INFINITY;
    unsigned long long cnt = 0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
         p += (long long)gridDim.x * blockDim.x) {
        const int code = mask ? mask[p] : 1;
        const Sym3 zero{0, 0, 0, 0, 0, 0};
        if (code == 0 || code > 3) {
            if (code > 3) atomicOr(flag, 1);
            store6(nu6, npix, p, zero);
            r[p] = r[npix + p] = r[2 * npix + p] = 0.0;
            continue;
        }
        const bool oI = code != 3, oP = code != 2;
        const Sym3 N = load6(N6, npix, p);
        bool ok = true;
        double dv[3] = {0.0, 0.0, 0.0};
        if (d) {
            dv[0] = oI ? d[p] : 0.0;
            dv[1] = oP ? d[npix + p] : 0.0;
            dv[2] = oP ? d[2 * npix + p] : 0.0;
            ok = isfinite(dv[0]) && isfinite(dv[1]) && isfinite(dv[2]);
        }
        Sym3 nu = zero;
        double tl = INFINITY;
        if (code == 1) {
            const double m2 = N.a * N.b - N.d * N.d, m3 = det3(N);
            ok = ok && isfinite(N.a) && isfinite(N.b) && isfinite(N.c) && isfinite(N.d) && isfinite(N.e) &&
                 isfinite(N.f) && N.a > 0.0 && m2 > 0.0 && m3 > 0.0;
            if (ok) {
                nu = inv3(N);
                tl = eigmin3(N);
            }
        } else if (code == 2) {
            ok = ok && isfinite(N.a) && N.a > 0.0;
            if (ok) {
                nu.a = 1.0 / N.a;
                tl = N.a;
            }
        } else {
            const double det = N.b * N.c - N.f * N.f;
            ok = ok && isfinite(N.b) && isfinite(N.c) && isfinite(N.f) && N.b > 0.0 && det > 0.0;
            if (ok) {
                nu.b = N.c / det;
                nu.c = N.b / det;
                nu.f = -N.f / det;
                const double h = 0.5 * (N.b - N.c);
                tl = 0.5 * (N.b + N.c) - sqrt(h * h + N.f * N.f);
            }
        }
        if (!ok) {
            atomicOr(flag, 1);
            store6(nu6, npix, p, zero);
            r[p] = r[npix + p] = r[2 * npix + p] = 0.0;
            continue;
        }
        store6(nu6, npix, p, nu);
        double rv[3];
        mv3(nu, dv, rv);
        r[p] = rv[0];
        r[npix + p] = rv[1];
        r[2 * npix + p] = rv[2];
        tmin = fmin(tmin, tl);
        cnt += code == 1 ? 3 : (code == 2 ? 1 : 2);
    }
    for (int o = 16; o >= 1; o >>= 1) {
        tmin = fmin(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (tmin < INFINITY) atomic_min_posd(&scal[0], tmin);
        atomicAdd(reinterpret_cast<unsigned long long *>(&scal[1]), cnt);
    }
}

// Eq. (10): t = s + lam tau (1 + (lam - 1) tau nu)^-1 (r - nu s), in place on
// the synthesised maps, and the pixel term of chi^2,
// sum (nu s) . u - 2 r . u with u = (1 + (lam - 1) tau nu)^-1 s; per-block partials
__global__ void k_blend_pol(long long npix, const double *__restrict__ r, const double *__restrict__ nu6,
                            double *__restrict__ t, double lt, double lm1t, double *__restrict__ part)
{
    __shared__ double red[32];
    double chi = 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
         p += (long long)gridDim.x * blockDim.x) {
        const Sym3 nu = load6(nu6, npix, p);
        const double s[3] = {t[p], t[npix + p], t[2 * npix + p]};
        const double rv[3] = {r[p], r[npix + p], r[2 * npix + p]};
        double ns[3];
        mv3(nu, s, ns);
        const Sym3 M{1.0 + lm1t * nu.a, 1.0 + lm1t * nu.b, 1.0 + lm1t * nu.c, lm1t * nu.d, lm1t * nu.e, lm1t * nu.f};
        const Sym3 Mi = inv3(M);
        const double res[3] = {rv[0] - ns[0], rv[1] - ns[1], rv[2] - ns[2]};
        double y[3], u[3];
        mv3(Mi, res, y);
        mv3(Mi, s, u);
        t[p] = s[0] + lt * y[0];
        t[npix + p] = s[1] + lt * y[1];
        t[2 * npix + p] = s[2] + lt * y[2];
        chi += (ns[0] - 2.0 * rv[0]) * u[0] + (ns[1] - 2.0 * rv[1]) * u[1] + (ns[2] - 2.0 * rv[2]) * u[2];
    }
    for (int o = 16; o >= 1; o >>= 1) chi += __shfl_xor_sync(0xffffffffu, chi, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = chi;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

// Eq. (10) for mixed plans: the same step on FP32 copies of r and nu, in
// FP32 arithmetic (1 + (lam - 1) tau nu has eigenvalues in [1, lam], so its
// cofactor inverse is well conditioned), chi^2 partials accumulated in FP64
__global__ void k_blend_pol_f32(long long npix, const float *__restrict__ r, const float *__restrict__ nu6,
                                float *__restrict__ t, float lt, float lm1t, double *__restrict__ part)
{
    __shared__ double red[32];
    double chi = 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
         p += (long long)gridDim.x * blockDim.x) {
        const float na = nu6[p], nb = nu6[npix + p], nc = nu6[2 * npix + p];
        const float nd = nu6[3 * npix + p], ne = nu6[4 * npix + p], nf = nu6[5 * npix + p];
        const float s0 = t[p], s1 = t[npix + p], s2 = t[2 * npix + p];
        const float r0 = r[p], r1 = r[npix + p], r2 = r[2 * npix + p];
        const float ns0 = na * s0 + nd * s1 + ne * s2;
        const float ns1 = nd * s0 + nb * s1 + nf * s2;
        const float ns2 = ne * s0 + nf * s1 + nc * s2;
        // M = 1 + lm1t nu, inverse by cofactors
        const float a = 1.f + lm1t * na, b = 1.f + lm1t * nb, c = 1.f + lm1t * nc;
        const float d = lm1t * nd, e = lm1t * ne, f = lm1t * nf;
        const float c00 = b * c - f * f, c11 = a * c - e * e, c22 = a * b - d * d;
        const float c01 = e * f - d * c, c02 = d * f - b * e, c12 = d * e - a * f;
        const float id = 1.f / (a * c00 + d * c01 + e * c02);
        const float q0 = r0 - ns0, q1 = r1 - ns1, q2 = r2 - ns2;
        const float y0 = (c00 * q0 + c01 * q1 + c02 * q2) * id;
        const float y1 = (c01 * q0 + c11 * q1 + c12 * q2) * id;
        const float y2 = (c02 * q0 + c12 * q1 + c22 * q2) * id;
        const float u0 = (c00 * s0 + c01 * s1 + c02 * s2) * id;
        const float u1 = (c01 * s0 + c11 * s1 + c12 * s2) * id;
        const float u2 = (c02 * s0 + c12 * s1 + c22 * s2) * id;
        t[p] = s0 + lt * y0;
        t[npix + p] = s1 + lt * y1;
        t[2 * npix + p] = s2 + lt * y2;
        chi += (double)((ns0 - 2.f * r0) * u0 + (ns1 - 2.f * r1) * u1 + (ns2 - 2.f * r2) * u2);
    }
    for (int o = 16; o >= 1; o >>= 1) chi += __shfl_xor_sync(0xffffffffu, chi, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = chi;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
        part[blockIdx.x] = sum;
    }
}

__global__ void k_to_f32(long long n, const double *__restrict__ in, float *__restrict__ out)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

// prior block of one l: TE block [[TT, TE], [TE, EE]] and BB
struct Prior {
    double tt, ee, bb, te;
};
__device__ __forceinline__ Prior prior(const double *__restrict__ C, int lmax, int l)
{
    return Prior{C[l], C[(lmax + 1) + l], C[2 * (lmax + 1) + l], C[3 * (lmax + 1) + l]};
}
// pseudo-inverse of the 2x2 TE block (and of BB): entries (it, ie, ix) = [[it, ix], [ix, ie]]
__device__ __forceinline__ void pinv_te(const Prior &S, double &it, double &ie, double &ix, double &ib)
{
    const double det = S.tt * S.ee - S.te * S.te;
    if (S.tt > 0.0 && S.ee > 0.0 && det > 0.0) {
        it = S.ee / det;
        ie = S.tt / det;
        ix = -S.te / det;
    } else {
        it = S.tt > 0.0 ? 1.0 / S.tt : 0.0;
        ie = S.ee > 0.0 ? 1.0 / S.ee : 0.0;
        ix = 0.0;
    }
    ib = S.bb > 0.0 ? 1.0 / S.bb : 0.0;
}

// sum w a^H S^+ a (mode 0) or sum w |P b|^2 with P the projector on the range of S (mode 1), per m
__global__ void k_pol_alm_norm(int lmax, const double *__restrict__ C, const double2 *__restrict__ a, long long nalm,
                               int mode, double *__restrict__ part)
{
    __shared__ double red[32];
    const int m = blockIdx.x;
    const long long base = pmbase(lmax, m);
    const double wm = m == 0 ? 1.0 : 2.0;
    double acc = 0.0;
    for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
        const long long k = base + (l - m);
        const double2 aT = a[k], aE = a[nalm + k], aB = a[2 * nalm + k];
        const Prior S = prior(C, lmax, l);
        double it, ie, ix, ib;
        pinv_te(S, it, ie, ix, ib);
        if (mode == 0) {
            const double re = it * (aT.x * aT.x + aT.y * aT.y) + ie * (aE.x * aE.x + aE.y * aE.y) +
                              2.0 * ix * (aT.x * aE.x + aT.y * aE.y) + ib * (aB.x * aB.x + aB.y * aB.y);
            acc += wm * re;
        } else {
            // projector: identity on the active components (a singular TE block has one active axis)
            const bool t = S.tt > 0.0, e = S.ee > 0.0, b = S.bb > 0.0;
            acc += wm * ((t ? aT.x * aT.x + aT.y * aT.y : 0.0) + (e ? aE.x * aE.x + aE.y * aE.y : 0.0) +
                         (b ? aB.x * aB.x + aB.y * aB.y : 0.0));
        }
    }
    for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        part[m] = s;
    }
}

// per-l factors of Eq. (11) for one launch (the a_lm kernel then does no
// divisions): T0 = Omega S (S + lam tau_h)^-1 on the TE block (f00, f01, f10,
// f11); T1 = (Omega BB / (BB + lam tau_h), S^+ entries it, ie, ix); T2 = (ib,
// and the residual multipliers S^+ + P / tau_h on the TE block diagonal and BB)
__global__ void k_hblend_table(int lmax, const double *__restrict__ C, double omega, double lam_tauh, double tauh,
                               double4 *__restrict__ tab)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l > lmax) return;
    const Prior S = prior(C, lmax, l);
    const double c = lam_tauh;
    const double m00 = S.tt + c, m11 = S.ee + c, m01 = S.te;
    const double det = m00 * m11 - m01 * m01;
    const double i00 = m11 / det, i11 = m00 / det, i01 = -m01 / det;
    const double f00 = S.tt * i00 + S.te * i01, f01 = S.tt * i01 + S.te * i11;
    const double f10 = S.te * i00 + S.ee * i01, f11 = S.te * i01 + S.ee * i11;
    const double fb = S.bb > 0.0 ? S.bb / (S.bb + c) : 0.0;
    double it, ie, ix, ib;
    pinv_te(S, it, ie, ix, ib);
    const double ih = 1.0 / tauh;
    tab[3 * l] = make_double4(omega * f00, omega * f01, omega * f10, omega * f11);
    tab[3 * l + 1] = make_double4(omega * fb, it, ie, ix);
    tab[3 * l + 2] = make_double4(ib, it + (S.tt > 0.0 ? ih : 0.0), ie + (S.ee > 0.0 ? ih : 0.0),
                                  ib + (S.bb > 0.0 ? ih : 0.0));
}

// Eq. (11): a_new = S (S + lam tau_h)^-1 Omega b for l <= L (0 above), and per-m
// partial sums [chi2_h(a_old), |(S^+ + 1/tau_h)(a_old - a_new)|^2]
__global__ void k_hblend_pol(int lmax, int L, long long nalm, const double4 *__restrict__ tab, int want_resid,
                             const double2 *__restrict__ b, const double2 *__restrict__ a_old,
                             double2 *__restrict__ a_new, double *__restrict__ part)
{
    __shared__ double red[2][32];
    const int m = blockIdx.x;
    const long long base = pmbase(lmax, m);
    const double wm = m == 0 ? 1.0 : 2.0;
    double chi = 0.0, res = 0.0;
    for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
        const long long k = base + (l - m);
        const double4 T0 = tab[3 * l], T1 = tab[3 * l + 1], T2 = tab[3 * l + 2];
        double2 nT = make_double2(0, 0), nE = nT, nB = nT;
        if (l <= L) {
            const double2 tT = b[k], tE = b[nalm + k], tB = b[2 * nalm + k];
            nT = make_double2(T0.x * tT.x + T0.y * tE.x, T0.x * tT.y + T0.y * tE.y);
            nE = make_double2(T0.z * tT.x + T0.w * tE.x, T0.z * tT.y + T0.w * tE.y);
            nB = make_double2(T1.x * tB.x, T1.x * tB.y);
        }
        const double2 oT = a_old[k], oE = a_old[nalm + k], oB = a_old[2 * nalm + k];
        const double it = T1.y, ie = T1.z, ix = T1.w, ib = T2.x;
        chi += wm * (it * (oT.x * oT.x + oT.y * oT.y) + ie * (oE.x * oE.x + oE.y * oE.y) +
                     2.0 * ix * (oT.x * oE.x + oT.y * oE.y) + ib * (oB.x * oB.x + oB.y * oB.y));
        if (want_resid) {
            const double2 dT = dsub(oT, nT), dE = dsub(oE, nE), dB = dsub(oB, nB);
            const double2 rT = make_double2(T2.y * dT.x + ix * dE.x, T2.y * dT.y + ix * dE.y);
            const double2 rE = make_double2(ix * dT.x + T2.z * dE.x, ix * dT.y + T2.z * dE.y);
            const double2 rB = make_double2(T2.w * dB.x, T2.w * dB.y);
            res += wm * (rT.x * rT.x + rT.y * rT.y + rE.x * rE.x + rE.y * rE.y + rB.x * rB.x + rB.y * rB.y);
        }
        a_new[k] = nT;
        a_new[nalm + k] = nE;
        a_new[2 * nalm + k] = nB;
    }
    for (int o = 16; o >= 1; o >>= 1) {
        chi += __shfl_xor_sync(0xffffffffu, chi, o);
        res += __shfl_xor_sync(0xffffffffu, res, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = chi;
        red[1][threadIdx.x >> 5] = res;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            s0 += red[0][w];
            s1 += red[1][w];
        }
        part[2 * m] = s0;
        part[2 * m + 1] = s1;
    }
}

// fluctuation source of Eq. (9) for (I, Q, U) maps: r = nu^1/2 g1 + Omega z,
// z the synthesised S^+1/2 g2 (nu = 0 in masked pixels, where r = Omega z)
__global__ void k_fluct_source_pol(long long npix, const double *__restrict__ nu6, const double *__restrict__ g1,
                                   const double *__restrict__ z, double omega, double *__restrict__ r)
{
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
         p += (long long)gridDim.x * blockDim.x) {
        const Sym3 nu = load6(nu6, npix, p);
        double o[3] = {0.0, 0.0, 0.0};
        const double g[3] = {g1[p], g1[npix + p], g1[2 * npix + p]};
        const bool hasI = nu.a != 0.0, hasP = nu.b != 0.0 || nu.c != 0.0;
        if (hasI && hasP) {
            mv3(sqrt3(nu), g, o);
        } else if (hasI) {  // I only: the block is nu_II alone
            o[0] = sqrt(nu.a) * g[0];
        } else if (hasP) {  // Q, U only: sqrt of [[b, f], [f, c]] = ([[b, f], [f, c]] + s) / t, s = det^1/2, t = (b + c + 2 s)^1/2
            const double sd = sqrt(nu.b * nu.c - nu.f * nu.f), t = sqrt(nu.b + nu.c + 2.0 * sd);
            o[1] = ((nu.b + sd) * g[1] + nu.f * g[2]) / t;
            o[2] = (nu.f * g[1] + (nu.c + sd) * g[2]) / t;
        }
        r[p] = o[0] + omega * z[p];
        r[npix + p] = o[1] + omega * z[npix + p];
        r[2 * npix + p] = o[2] + omega * z[2 * npix + p];
    }
}

// S^+1/2 g2 per (l, m): the pseudo-inverse square root of the prior block.  A
// TE block with TE != 0 is positive definite (checked on the host) and its
// inverse square root is closed-form: with s = det^1/2 and t = (TT + EE + 2 s)^1/2,
// [[TT, TE], [TE, EE]]^-1/2 = [[EE + s, -TE], [-TE, TT + s]] / (s t).
__global__ void k_isqrt_S_pol(int lmax, long long nalm, const double *__restrict__ C, const double2 *__restrict__ g2,
                              double2 *__restrict__ out)
{
    const int m = blockIdx.x;
    const long long base = pmbase(lmax, m);
    for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
        const long long k = base + (l - m);
        const Prior S = prior(C, lmax, l);
        double jt, je, jx;
        if (S.te != 0.0) {
            const double sd = sqrt(S.tt * S.ee - S.te * S.te), t = sqrt(S.tt + S.ee + 2.0 * sd);
            const double q = 1.0 / (sd * t);
            jt = (S.ee + sd) * q;
            je = (S.tt + sd) * q;
            jx = -S.te * q;
        } else {
            jt = S.tt > 0.0 ? 1.0 / sqrt(S.tt) : 0.0;
            je = S.ee > 0.0 ? 1.0 / sqrt(S.ee) : 0.0;
            jx = 0.0;
        }
        const double jb = S.bb > 0.0 ? 1.0 / sqrt(S.bb) : 0.0;
        const double2 gT = g2[k], gE = g2[nalm + k], gB = g2[2 * nalm + k];
        out[k] = make_double2(jt * gT.x + jx * gE.x, jt * gT.y + jx * gE.y);
        out[nalm + k] = make_double2(jx * gT.x + je * gE.x, jx * gT.y + je * gE.y);
        out[2 * nalm + k] = make_double2(jb * gB.x, jb * gB.y);
    }
}

// sum over observed pixels of (d - s)^T nu (d - s) (chi^2 of the result), per-block partials
__global__ void k_pix_chi2_pol(long long npix, const double *__restrict__ d, const double *__restrict__ nu6,
                               const double *__restrict__ s, double *__restrict__ part)
{
    __shared__ double red[32];
    double acc = 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
         p += (long long)gridDim.x * blockDim.x) {
        const Sym3 nu = load6(nu6, npix, p);
        // unobserved components (zero rows of nu) may hold anything in d, NaN included
        const double e[3] = {nu.a != 0.0 ? d[p] - s[p] : 0.0, nu.b != 0.0 ? d[npix + p] - s[npix + p] : 0.0,
                             nu.c != 0.0 ? d[2 * npix + p] - s[2 * npix + p] : 0.0};
        double ne[3];
        mv3(nu, e, ne);
        acc += e[0] * ne[0] + e[1] * ne[1] + e[2] * ne[2];
    }
    for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
wf_status hp_pol_create(wf_plan p, const double *xpair_dev, const double *stpair_dev)
{
    PolState *s = new (std::nothrow) PolState();
    if (!s) return set_error(WF_ENOMEM, "host allocation");
    p->pol = s;
    const int lmax = p->lmax, np = p->npairs;
    const long long nalm = p->nalm, ns = (long long)(lmax + 1) * np, npix = p->npix;
    const bool f64 = p->prec == WF_PREC_FP64;
    const size_t gsz = (size_t)np * (lmax + 1) * 2 * (f64 ? sizeof(double2) : sizeof(float2));
    wf_status st;
    if ((st = plan_alloc(p, (void **)&s->al, nalm * 8)) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&s->be, nalm * 8)) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&s->ga, nalm * 8)) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&s->ls, ns * 4)) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&s->p0, ns * 8)) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&s->p1, ns * 8)) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&s->m0, ns * 8)) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&s->m1, ns * 8)) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&s->a, 3 * nalm * sizeof(double2))) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&s->a_new, 3 * nalm * sizeof(double2))) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&s->b, 3 * nalm * sizeof(double2))) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&s->GQ, gsz)) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&s->GU, gsz)) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&s->FQ, gsz)) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&s->FU, gsz)) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&s->r, 3 * npix * 8)) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&s->t, 3 * npix * (f64 ? 8 : 4))) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&s->nu, 6 * npix * 8)) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&s->hbt, (size_t)3 * (lmax + 1) * sizeof(double4))) != WF_OK) return st;
    if (!f64) {
        if ((st = plan_alloc(p, (void **)&s->r32, 3 * npix * 4)) != WF_OK) return st;
        if ((st = plan_alloc(p, (void **)&s->nu32, 6 * npix * 4)) != WF_OK) return st;
    }
    const int npart = std::max(2 * (lmax + 2), std::max(256, 4 * p->nsm));
    if ((st = plan_alloc(p, (void **)&s->part, (size_t)npart * 8)) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&s->part2, (size_t)npart * 8)) != WF_OK) return st;
    k_pol_coefs<<<lmax + 1, 256, 0, p->stream>>>(lmax, s->al, s->be, s->ga);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    const int th = 256;
    k_seeds_pol<<<(unsigned)((ns + th - 1) / th), th, 0, p->stream>>>(lmax, np, xpair_dev, stpair_dev, s->al, s->be,
                                                                     s->ga, s->ls, s->p0, s->p1, s->m0, s->m1);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    // shared-memory limits at their lmax sizes now, so no launch (e.g. inside a graph capture) needs to
    const size_t sm_ana = (size_t)2 * (lmax + 1 + POL_CH + 2) * sizeof(double2) + 16;
    if ((st = raise_smem_limit((const void *)(f64 ? (const void *)k_legana_pol<double>
                                                  : (const void *)k_legana_pol<float>), sm_ana)) != WF_OK)
        return st;
    if (!f64 && (st = hp_pol_create_mx(p)) != WF_OK) return st;
    WF_CUDA(cudaStreamSynchronize(p->stream));
    return WF_OK;
}

void hp_pol_destroy(wf_plan p)
{
    delete p->pol;
    p->pol = nullptr;
}

// (E, B) -> ring coefficients (GQ, GU), l <= L
wf_status hp_pol_legendre_synthesis(wf_plan p, const double2 *E, const double2 *B, int L)
{
    const PolState *s = p->pol;
    dim3 grid((p->npairs + POL_THREADS - 1) / POL_THREADS, L + 1);
    k_legsyn_pol<double><<<grid, POL_THREADS, 0, p->stream>>>(p->lmax, L, 0, p->lmax + 1, p->npairs, E, B, s->al,
                                                               s->be, s->ga, s->ls, s->p0, s->p1, s->m0, s->m1,
                                                               p->tab.x64, (double2 *)s->GQ, (double2 *)s->GU);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    return WF_OK;
}

// ring coefficients (FQ, FU) -> (E, B) (adjoint), l <= L
wf_status hp_pol_legendre_analysis(wf_plan p, int L, double2 *E, double2 *B)
{
    const PolState *s = p->pol;
    const size_t sm = (size_t)2 * (L + 1 + POL_CH + 2) * sizeof(double2) + 16;
    if (wf_status st = raise_smem_limit((const void *)k_legana_pol<double>, sm)) return st;
    k_legana_pol<double><<<L + 1, POL_THREADS, sm, p->stream>>>(p->lmax, L, 0, p->npairs, (const double2 *)s->FQ,
                                                                 (const double2 *)s->FU, s->al, s->be, s->ga, s->ls,
                                                                 s->p0, s->p1, s->m0, s->m1, p->tab.x64, E, B);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    if (L < p->lmax) {  // columns m > L are not visited: zero them
        const long long from = pmbase(p->lmax, L + 1);
        WF_CUDA(cudaMemsetAsync(E + from, 0, (p->nalm - from) * sizeof(double2), p->stream));
        WF_CUDA(cudaMemsetAsync(B + from, 0, (p->nalm - from) * sizeof(double2), p->stream));
    }
    return WF_OK;
}

wf_status hp_pol_legendre_synthesis_low(wf_plan p, const double2 *E, const double2 *B, int L, int lc, float2 *GQ,
                                        float2 *GU)
{
    const PolState *s = p->pol;
    const int nm = std::min(lc, L + 1);
    if (nm <= 0) return WF_OK;
    dim3 grid((p->npairs + POL_THREADS - 1) / POL_THREADS, nm);
    k_legsyn_pol<float><<<grid, POL_THREADS, 0, p->stream>>>(p->lmax, L, lc, s->low_cap, p->npairs, E, B, s->al, s->be,
                                                              s->ga, s->ls, s->p0, s->p1, s->m0, s->m1, p->tab.x64, GQ,
                                                              GU);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    return WF_OK;
}

wf_status hp_pol_legendre_analysis_low(wf_plan p, int L, int lc, const float2 *FQ, const float2 *FU, double2 *E,
                                       double2 *B)
{
    const PolState *s = p->pol;
    const int nm = std::min(lc, L + 1);
    if (nm <= 0) return WF_OK;
    const int Lb = std::min(L, lc + 1);
    const size_t sm = (size_t)2 * (Lb + 1 + POL_CH + 2) * sizeof(double2) + 16;
    if (wf_status st = raise_smem_limit((const void *)k_legana_pol<float>, sm)) return st;
    // about four CTAs per SM: each m's ring pairs split over CTAs that add into zeroed outputs
    const int ngroups = (p->npairs + 31) / 32, per_cta = POL_THREADS / 32;
    const int split = std::max(1, std::min((4 * p->nsm + nm - 1) / nm, (ngroups + per_cta - 1) / per_cta));
    const long long nz = pmbase(p->lmax, nm);
    WF_CUDA(cudaMemsetAsync(E, 0, nz * sizeof(double2), p->stream));
    WF_CUDA(cudaMemsetAsync(B, 0, nz * sizeof(double2), p->stream));
    k_legana_pol<float><<<dim3(nm, split), POL_THREADS, sm, p->stream>>>(p->lmax, L, lc, p->npairs, FQ, FU, s->al,
                                                                          s->be, s->ga, s->ls, s->p0, s->p1, s->m0,
                                                                          s->m1, p->tab.x64, E, B);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    return WF_OK;
}

wf_status hp_pol_setup(wf_plan p, const double *d, const double *N6, const uint8_t *mask, double *tau,
                       long long *ndof)
{
    PolState *s = p->pol;
    const double init[2] = {INFINITY, 0.0};
    WF_CUDA(cudaMemcpyAsync(p->ws.scal, init, sizeof init, cudaMemcpyHostToDevice, p->stream));
    WF_CUDA(cudaMemsetAsync(p->ws.flag, 0, sizeof(int), p->stream));
    const int grid = (int)std::min<long long>((p->npix + 255) / 256, 8LL * p->nsm);
    k_setup_pol<<<grid, 256, 0, p->stream>>>(p->npix, d, N6, mask, s->r, s->nu, p->ws.scal, p->ws.flag);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    double sc[2];
    int flag = 0;
    WF_CUDA(cudaMemcpyAsync(sc, p->ws.scal, sizeof sc, cudaMemcpyDeviceToHost, p->stream));
    WF_CUDA(cudaMemcpyAsync(&flag, p->ws.flag, sizeof flag, cudaMemcpyDeviceToHost, p->stream));
    WF_CUDA(cudaStreamSynchronize(p->stream));
    unsigned long long cnt;
    std::memcpy(&cnt, &sc[1], sizeof cnt);
    if (flag) return set_error(WF_EINVAL, "mask codes must be 0..3, and the noise covariance finite and positive "
                                          "definite (and d finite) on the observed components");
    if (cnt == 0) return set_error(WF_EINVAL, "every pixel is masked");
    *tau = sc[0];
    *ndof = (long long)cnt;  // observed components
    return WF_OK;
}

wf_status hp_pol_blend(wf_plan p, double lam, double tau, int *nblocks)
{
    PolState *s = p->pol;
    const int grid = (int)std::min<long long>((p->npix + 255) / 256, 2LL * p->nsm);
    if (p->prec == WF_PREC_FP64)
        k_blend_pol<<<grid, 256, 0, p->stream>>>(p->npix, s->r, s->nu, (double *)s->t, lam * tau, (lam - 1.0) * tau,
                                                 s->part);
    else
        k_blend_pol_f32<<<grid, 256, 0, p->stream>>>(p->npix, s->r32, s->nu32, (float *)s->t, (float)(lam * tau),
                                                     (float)((lam - 1.0) * tau), s->part);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    *nblocks = grid;
    return WF_OK;
}

wf_status hp_pol_hblend(wf_plan p, int L, const double *C, double lam_tauh, double tauh, int want_resid)
{
    PolState *s = p->pol;
    k_hblend_table<<<(p->lmax + 256) / 256, 256, 0, p->stream>>>(p->lmax, C, p->omega, lam_tauh, tauh, s->hbt);
    WF_COUNT_LAUNCH(p);
    k_hblend_pol<<<p->lmax + 1, 256, 0, p->stream>>>(p->lmax, L, p->nalm, s->hbt, want_resid, s->b, s->a, s->a_new,
                                                      s->part2);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    return WF_OK;
}

wf_status hp_pol_alm_norm(wf_plan p, const double *C, const double2 *a, int mode)
{
    k_pol_alm_norm<<<p->lmax + 1, 256, 0, p->stream>>>(p->lmax, C, a, p->nalm, mode, p->pol->part2);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    return WF_OK;
}

wf_status hp_pol_isqrt_prior(wf_plan p, const double *C, const double2 *g2, double2 *out)
{
    k_isqrt_S_pol<<<p->lmax + 1, 256, 0, p->stream>>>(p->lmax, p->nalm, C, g2, out);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    return WF_OK;
}

// mixed plans: FP32 copies of the source and the inverse-noise blocks for the blend
wf_status hp_pol_round_pixels(wf_plan p)
{
    PolState *s = p->pol;
    if (p->prec == WF_PREC_FP64) return WF_OK;
    const long long n3 = 3 * p->npix, n6 = 6 * p->npix;
    const int grid = (int)std::min<long long>((n6 + 255) / 256, 4LL * p->nsm);
    k_to_f32<<<grid, 256, 0, p->stream>>>(n3, s->r, s->r32);
    WF_COUNT_LAUNCH(p);
    k_to_f32<<<grid, 256, 0, p->stream>>>(n6, s->nu, s->nu32);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    return WF_OK;
}

wf_status hp_pol_fluct_source(wf_plan p, const double *g1, const double *z)
{
    const int grid = (int)std::min<long long>((p->npix + 255) / 256, 2LL * p->nsm);
    k_fluct_source_pol<<<grid, 256, 0, p->stream>>>(p->npix, p->pol->nu, g1, z, p->omega, p->pol->r);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    return WF_OK;
}

wf_status hp_pol_pix_chi2(wf_plan p, const double *d, const double *s_map, int *nblocks)
{
    const int grid = 256;
    k_pix_chi2_pol<<<grid, 256, 0, p->stream>>>(p->npix, d, p->pol->nu, s_map, p->pol->part);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    *nblocks = grid;
    return WF_OK;
}

}  // namespace wf
