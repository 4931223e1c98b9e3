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
// sum.  The recurrence runs in "mu form" (see wf_internal.cuh) from per-(m,
// pair) seeds at the first l where |lambda_lm| exceeds 2^-80 (computed in FP64
// with an explicit binary exponent, since sin^m(theta) underflows FP64 near
// the poles at large m); below that l every term is < 2^-80 and is dropped.
#include <climits>
#include <cmath>
#include <cstdio>

#include "wf_internal.cuh"

namespace wf {

namespace {

constexpr double SEED_LOG2_THRESHOLD = -80.0;

__host__ __device__ inline long long mbase(int lmax, int m) { return (long long)m * (2 * lmax + 3 - m) / 2; }

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

template <typename T>
__global__ void k_to_T(const double *__restrict__ in, T *__restrict__ out, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (T)in[i];
}

// ---------------------------------------------------------------------------
// synthesis: CTA per (m, block of pairs); thread per pair
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(LEG_THREADS) k_legsyn(int lmax, int L, int npairs, const double2 *__restrict__ alm,
                                                        const T *__restrict__ A, const T *__restrict__ c,
                                                        const int *__restrict__ ls_tab, const T *__restrict__ s0_tab,
                                                        const T *__restrict__ s1_tab, const T *__restrict__ xp,
                                                        cx<T> *__restrict__ G)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m = blockIdx.y;
    const int nl = L - m + 1;
    const long long base = mbase(lmax, m);
    cx<T> *sac = reinterpret_cast<cx<T> *>(smem_raw);
    T *sA = reinterpret_cast<T *>(sac + (nl + 2));
    for (int i = threadIdx.x; i < nl + 2; i += blockDim.x) {
        if (i < nl) {
            const double2 a = alm[base + i];
            const T cc = c[base + i];
            sac[i] = mk<T>((T)a.x * cc, (T)a.y * cc);
            sA[i] = A[base + i];
        } else {
            sac[i] = mk<T>(0, 0);
            sA[i] = 0;
        }
    }
    __syncthreads();
    const size_t pstride = (size_t)(lmax + 1) * 2;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += gridDim.x * blockDim.x) {
        const size_t sidx = (size_t)m * npairs + p;
        const int ls = ls_tab[sidx];
        T er = 0, ei = 0, orr = 0, oi = 0;
        if (ls <= L) {
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
        cx<T> *g = G + (size_t)p * pstride + 2 * (size_t)m;
        g[0] = mk<T>(er + orr, ei + oi);
        g[1] = mk<T>(er - orr, ei - oi);
    }
}

// ---------------------------------------------------------------------------
// analysis: CTA per m; warp per 32 pairs; register chunks of CH values of l
// reduced across the warp by a shuffle reduce-scatter, then added into FP64
// shared accumulators.
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
template <> struct Log2<16> { static constexpr int v = 4; };
template <> struct Log2<32> { static constexpr int v = 5; };

template <typename T, int CH>
__global__ void __launch_bounds__(LEG_THREADS) k_legana(int lmax, int L, int npairs, const cx<T> *__restrict__ F,
                                                        const T *__restrict__ A, const int *__restrict__ ls_tab,
                                                        const T *__restrict__ s0_tab, const T *__restrict__ s1_tab,
                                                        const T *__restrict__ xp, const double *__restrict__ c64,
                                                        int mode, double omega, BlendArgs ba,
                                                        const double2 *__restrict__ a_old, double2 *__restrict__ out,
                                                        double *__restrict__ part)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[2][LEG_THREADS / 32];
    const int m = blockIdx.x;
    const int nl = L - m + 1;
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
    constexpr int BIG = INT_MAX / 2;
    for (int grp = warp; grp < ngroups; grp += nwarps) {
        const int p = grp * 32 + lane;
        const size_t sidx = (size_t)m * npairs + p;
        int ls = (p < npairs) ? ls_tab[sidx] : BIG;
        if (ls > L) ls = BIG;
        const int lmin = __reduce_min_sync(0xffffffffu, ls);
        if (lmin > L) continue;
        cx<T> FE = mk<T>(0, 0), FO = mk<T>(0, 0);
        T x = 0, s0 = 0, s1 = 0;
        if (ls <= L) {
            const cx<T> *f = F + ((size_t)p * (lmax + 1) + m) * 2;
            const cx<T> fn = f[0], fs = f[1];
            FE = cadd(fn, fs);
            FO = csub(fn, fs);
            x = xp[p];
            s0 = s0_tab[sidx];
            s1 = s1_tab[sidx];
        }
        T mua = 0, mub = 0;
        for (int l0 = lmin; l0 <= L; l0 += CH) {
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
                if (l <= L) {
                    atomicAdd(&acc[l - m].x, (double)vr[0]);
                    atomicAdd(&acc[l - m].y, (double)vi[0]);
                }
            }
        }
    }
    __syncthreads();

    double chi2 = 0.0, res2 = 0.0;
    const double wm = (m == 0) ? 1.0 : 2.0;
    for (int j = threadIdx.x; j <= lmax - m; j += blockDim.x) {
        const int l = m + j;
        const long long idx = base + j;
        if (mode == LEG_ADJOINT) {
            double2 v = make_double2(0.0, 0.0);
            if (l <= L) { v.x = c64[idx] * acc[j].x; v.y = c64[idx] * acc[j].y; }
            out[idx] = v;
        } else {
            const double S = ba.S[l];
            const double2 ao = a_old[idx];
            double2 an = make_double2(0.0, 0.0);
            if (l <= L && S > 0.0) {
                const double f = omega * c64[idx] * S / (S + ba.lam_tauh);
                an.x = f * acc[j].x;
                an.y = f * acc[j].y;
            }
            if (S > 0.0) {
                chi2 += wm * (ao.x * ao.x + ao.y * ao.y) / S;
                if (ba.want_resid) {
                    const double k = 1.0 / S + 1.0 / ba.tauh;
                    const double dx = k * (ao.x - an.x), dy = k * (ao.y - an.y);
                    res2 += wm * (dx * dx + dy * dy);
                }
            }
            out[idx] = an;
        }
    }
    if (mode == LEG_BLEND) {
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            chi2 += __shfl_xor_sync(0xffffffffu, chi2, o);
            res2 += __shfl_xor_sync(0xffffffffu, res2, o);
        }
        if (lane == 0) { red[0][warp] = chi2; red[1][warp] = res2; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0, b = 0.0;
            for (int w = 0; w < nwarps; ++w) { a += red[0][w]; b += red[1][w]; }
            part[2 * m] = a;
            part[2 * m + 1] = b;
        }
    }
}

template <typename T>
size_t syn_smem(int L, int m0) { return (size_t)(L - m0 + 3) * (sizeof(cx<T>) + sizeof(T)) + 16; }

template <typename T, int CH>
size_t ana_smem(int L) { return (size_t)(L + 1 + CH + 2) * (sizeof(double2) + sizeof(T)) + 16; }

template <typename T>
wf_status launch_syn(wf_plan p, const double2 *alm, int L)
{
    const HpTables &t = p->tab;
    const int gx = (p->npairs + 4 * LEG_THREADS - 1) / (4 * LEG_THREADS);
    dim3 grid(gx, L + 1);
    const size_t sm = syn_smem<T>(L, 0);
    WF_CUDA(cudaFuncSetAttribute(k_legsyn<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_legsyn<T><<<grid, LEG_THREADS, sm, p->stream>>>(p->lmax, L, p->npairs, alm, (const T *)t.A, (const T *)t.c, t.ls,
                                                       (const T *)t.s0, (const T *)t.s1, (const T *)t.x,
                                                       (cx<T> *)p->ws.G);
    WF_CUDA(cudaGetLastError());
    return WF_OK;
}

template <typename T>
wf_status launch_ana(wf_plan p, int L, LegMode mode, const BlendArgs &ba, const double2 *a_old, double2 *out)
{
    constexpr int CH = sizeof(T) == 8 ? 16 : 32;
    const HpTables &t = p->tab;
    const size_t sm = ana_smem<T, CH>(L);
    WF_CUDA(cudaFuncSetAttribute(k_legana<T, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_legana<T, CH><<<L + 1, LEG_THREADS, sm, p->stream>>>(
        p->lmax, L, p->npairs, (const cx<T> *)p->ws.F, (const T *)t.A, t.ls, (const T *)t.s0, (const T *)t.s1,
        (const T *)t.x, t.c64, (int)mode, p->omega, ba, a_old, out, p->ws.part_harm);
    WF_CUDA(cudaGetLastError());
    return WF_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// host: recurrence tables and seeds
// ---------------------------------------------------------------------------
wf_status hp_build_legendre_tables(wf_plan p, const std::vector<double> &xpair, const std::vector<double> &stpair)
{
    const int lmax = p->lmax, np = p->npairs;
    const long long nalm = p->nalm;
    std::vector<double> A(nalm), c(nalm), log2c(lmax + 1);
    for (int m = 0; m <= lmax; ++m) {
        const long long b = mbase(lmax, m);
        auto coef = [m](int l) { return std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m)); };
        c[b] = 1.0;
        A[b] = 0.0;
        if (m + 1 <= lmax) {
            c[b + 1] = 1.0;
            A[b + 1] = std::sqrt(2.0 * m + 3.0);
        }
        for (int l = m + 2; l <= lmax; ++l) {
            const double al = coef(l), alm1 = coef(l - 1);
            c[b + (l - m)] = (al / alm1) * c[b + (l - 2 - m)];
            A[b + (l - m)] = al * c[b + (l - 1 - m)] / c[b + (l - m)];
        }
        // log2 of sqrt((2m+1)/(4 pi) (2m)! / (2^m m!)^2)
        log2c[m] = 0.5 * (std::log(2.0 * m + 1.0) - std::log(4.0 * M_PI) + std::lgamma(2.0 * m + 1.0) -
                          2.0 * std::lgamma(m + 1.0) - 2.0 * m * std::log(2.0)) / std::log(2.0);
    }
    const bool f32 = p->prec != WF_PREC_FP64;
    const size_t es = f32 ? sizeof(float) : sizeof(double);
    double *dA64 = nullptr, *dx64 = nullptr, *dst64 = nullptr, *dlog2c = nullptr, *ds0 = nullptr, *ds1 = nullptr;
    wf_status st;
    if ((st = plan_alloc(p, (void **)&p->tab.c64, nalm * sizeof(double))) != WF_OK) return st;
    WF_CUDA(cudaMalloc(&dA64, nalm * sizeof(double)));
    WF_CUDA(cudaMalloc(&dx64, np * sizeof(double)));
    WF_CUDA(cudaMalloc(&dst64, np * sizeof(double)));
    WF_CUDA(cudaMalloc(&dlog2c, (lmax + 1) * sizeof(double)));
    const long long ns = (long long)(lmax + 1) * np;
    if ((st = plan_alloc(p, (void **)&p->tab.ls, ns * sizeof(int))) != WF_OK) return st;
    WF_CUDA(cudaMalloc(&ds0, ns * sizeof(double)));
    WF_CUDA(cudaMalloc(&ds1, ns * sizeof(double)));
    WF_CUDA(cudaMemcpy(dA64, A.data(), nalm * sizeof(double), cudaMemcpyHostToDevice));
    WF_CUDA(cudaMemcpy(p->tab.c64, c.data(), nalm * sizeof(double), cudaMemcpyHostToDevice));
    WF_CUDA(cudaMemcpy(dx64, xpair.data(), np * sizeof(double), cudaMemcpyHostToDevice));
    WF_CUDA(cudaMemcpy(dst64, stpair.data(), np * sizeof(double), cudaMemcpyHostToDevice));
    WF_CUDA(cudaMemcpy(dlog2c, log2c.data(), (lmax + 1) * sizeof(double), cudaMemcpyHostToDevice));
    {
        const int th = 256;
        const long long nb = (ns + th - 1) / th;
        k_seeds<<<(unsigned)nb, th, 0, p->stream>>>(lmax, np, dx64, dst64, dlog2c, dA64, p->tab.c64, p->tab.ls, ds0, ds1);
        WF_CUDA(cudaGetLastError());
    }
    if ((st = plan_alloc(p, &p->tab.A, nalm * es)) != WF_OK) return st;
    if ((st = plan_alloc(p, &p->tab.c, nalm * es)) != WF_OK) return st;
    if ((st = plan_alloc(p, &p->tab.s0, ns * es)) != WF_OK) return st;
    if ((st = plan_alloc(p, &p->tab.s1, ns * es)) != WF_OK) return st;
    if ((st = plan_alloc(p, &p->tab.x, np * es)) != WF_OK) return st;
    const int cvb = 1024;
    if (f32) {
        k_to_T<float><<<cvb, 256, 0, p->stream>>>(dA64, (float *)p->tab.A, nalm);
        k_to_T<float><<<cvb, 256, 0, p->stream>>>(p->tab.c64, (float *)p->tab.c, nalm);
        k_to_T<float><<<cvb, 256, 0, p->stream>>>(ds0, (float *)p->tab.s0, ns);
        k_to_T<float><<<cvb, 256, 0, p->stream>>>(ds1, (float *)p->tab.s1, ns);
        k_to_T<float><<<cvb, 256, 0, p->stream>>>(dx64, (float *)p->tab.x, np);
    } else {
        WF_CUDA(cudaMemcpyAsync(p->tab.A, dA64, nalm * 8, cudaMemcpyDeviceToDevice, p->stream));
        WF_CUDA(cudaMemcpyAsync(p->tab.c, p->tab.c64, nalm * 8, cudaMemcpyDeviceToDevice, p->stream));
        WF_CUDA(cudaMemcpyAsync(p->tab.s0, ds0, ns * 8, cudaMemcpyDeviceToDevice, p->stream));
        WF_CUDA(cudaMemcpyAsync(p->tab.s1, ds1, ns * 8, cudaMemcpyDeviceToDevice, p->stream));
        WF_CUDA(cudaMemcpyAsync(p->tab.x, dx64, np * 8, cudaMemcpyDeviceToDevice, p->stream));
    }
    WF_CUDA(cudaGetLastError());
    WF_CUDA(cudaStreamSynchronize(p->stream));
    cudaFree(dA64);
    cudaFree(dx64);
    cudaFree(dst64);
    cudaFree(dlog2c);
    cudaFree(ds0);
    cudaFree(ds1);
    return WF_OK;
}

wf_status hp_legendre_synthesis(wf_plan p, const double2 *alm, int L)
{
    return p->prec == WF_PREC_FP64 ? launch_syn<double>(p, alm, L) : launch_syn<float>(p, alm, L);
}

wf_status hp_legendre_analysis(wf_plan p, int L, LegMode mode, const BlendArgs &ba, const double2 *a_old, double2 *out)
{
    return p->prec == WF_PREC_FP64 ? launch_ana<double>(p, L, mode, ba, a_old, out)
                                   : launch_ana<float>(p, L, mode, ba, a_old, out);
}

}  // namespace wf
