// Flat-sky messenger-field Wiener filter on a periodic n x n grid with the
// unitary 2-D DFT (the "e.g. Fourier space" basis of Sect. 2.1).
//
// The whole solve -- every iteration of Eqs. (3)-(4), the chi^2 of Eq. (6),
// the residual and the cooling schedule -- runs in ONE persistent launch of a
// single thread-block cluster of CS CTAs (CS = 16 where the device co-schedules
// that non-portable size, else 8; flat_cluster_size).  The grid never leaves the
// cluster's shared memory:
//   CTA c owns pixel rows [c n/CS, (c+1) n/CS) (source r, inverse noise nu)
//   and spectrum columns kx in [c P, (c+1) P), P = ceil((n/2+1)/CS) (a, S).
// One iteration:
//   1. column inverse FFTs (ky) of the owned a columns          (local)
//   2. cluster barrier; each CTA gathers its rows' spectra from every CTA's
//      column buffer through distributed shared memory, c2r FFTs the rows,
//      applies the pixel blend of Eq. (3) and r2c FFTs the result
//   3. cluster barrier; each CTA gathers its columns from every CTA's row
//      buffer, forward FFTs them (ky) and applies the harmonic blend of
//      Eq. (4), accumulating chi^2 and the lambda = 1 residual
//   4. cluster barrier; every CTA sums all CTAs' partials in the same order
//      and takes the same schedule decision (no broadcast needed).
// FFTs are radix-2, one warp per row/column, in shared memory.
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <vector>

#include "wf_internal.cuh"

namespace cg = cooperative_groups;

namespace wf {

constexpr int FLAT_CS = 8;      // portable cluster size; the smallest the solve runs on
constexpr int FLAT_CS_MAX = 16; // non-portable cluster size, used where the device co-schedules it
constexpr int FLAT_THREADS = 256;
constexpr int FLAT_WARPS = FLAT_THREADS / 32;
constexpr int FLAT_MAXN = 128;

struct FlatStatus {
    int iters, converged, levels, stop_reason;  // stop_reason: 0 schedule/replay end, 1 converged, 2 maxiter, 3 diverged
    double final_resid, chi2_final, bnorm;
};

struct FlatPlan {
    int n = 0, logn = 0, nh = 0, P = 0, RP = 0, cs = 8;
    size_t smem = 0;
    double *r = nullptr, *nu = nullptr;  // device pixel maps
    double *levels = nullptr;            // device lambda levels
    double *tr_lam = nullptr, *tr_chi2 = nullptr, *tr_res = nullptr;
    int tr_cap = 0;
    FlatStatus *status = nullptr;
    double *replay = nullptr;
    int replay_cap = 0;
};

namespace {

struct FlatArgs {
    int n, logn, nh, P, RP;
    const double *r, *nu, *S;
    const double *g1;      // fluct: unit draws in pixel space (or null)
    const double2 *g2;     // fluct: unit harmonic draws (or null)
    const double *levels;
    int nlevels;
    const double *replay;  // lambda per iteration (or null)
    int nreplay;
    double tau, sigma, eta, tol;
    int level_cap, maxiter;
    double *s_out;
    double2 *alm_out;
    double *tr_lam, *tr_chi2, *tr_res;
    int tr_cap;
    FlatStatus *status;
};

__device__ __forceinline__ double2 dmul(double2 a, double2 b) { return cmul(a, b); }

// radix-2 DIT FFT of length 2^logn on x (shared memory) by one warp
__device__ void warp_fft(double2 *x, int logn, int sign, const double2 *tw /* e^{-2 pi i t / n}, t < n/2 */)
{
    const int n = 1 << logn, lane = threadIdx.x & 31;
    for (int i = lane; i < n; i += 32) {
        const int j = (int)(__brev((unsigned)i) >> (32 - logn));
        if (i < j) {
            const double2 t = x[i];
            x[i] = x[j];
            x[j] = t;
        }
    }
    __syncwarp();
    for (int s = 1; s <= logn; ++s) {
        const int half = 1 << (s - 1);
        for (int b = lane; b < n / 2; b += 32) {
            const int pos = b & (half - 1);
            const int i0 = ((b >> (s - 1)) << s) + pos, i1 = i0 + half;
            double2 w = tw[pos << (logn - s)];
            if (sign > 0) w.y = -w.y;
            const double2 u = x[i0], v = dmul(x[i1], w);
            x[i0] = cadd(u, v);
            x[i1] = csub(u, v);
        }
        __syncwarp();
    }
}

enum FlatStep { FS_ITER = 0, FS_PROLOGUE = 1, FS_FLUCT_SRC = 2, FS_OUT = 3 };

// dynamic shared memory of k_flat_solve: twiddles; a, column and row buffers; per-warp FFT
// rows; S, 1/S and S / (S + lam tau) per owned mode; r, nu and 1 / (1 + (lam - 1) tau nu)
// per owned pixel
inline size_t flat_smem(int n, int P, int RP, int nh)
{
    return (size_t)(n / 2) * 16 + (size_t)P * n * 16 * 2 + (size_t)RP * nh * 16 + (size_t)FLAT_WARPS * n * 16 +
           (size_t)P * n * 8 * 3 + (size_t)RP * n * 8 * 3;
}

__global__ void __launch_bounds__(FLAT_THREADS) k_flat_solve(FlatArgs A)
{
    cg::cluster_group cluster = cg::this_cluster();
    const int c = (int)cluster.block_rank();
    const int n = A.n, nh = A.nh, P = A.P, RP = A.RP, logn = A.logn;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c0 = c * P;
    const double inv_tau = 1.0 / A.tau;
    const int ncol = max(0, min(nh, c0 + P) - c0);
    const int y0 = c * RP;
    const double sy = rsqrt((double)n), sx = rsqrt((double)n);

    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *tw = reinterpret_cast<double2 *>(smem_raw);            // n/2
    double2 *acol = tw + n / 2;                                      // P * n
    double2 *colbuf = acol + (size_t)P * n;                          // P * n
    double2 *rowbuf = colbuf + (size_t)P * n;                        // RP * nh
    double2 *wscr = rowbuf + (size_t)RP * nh;                        // FLAT_WARPS * n
    double *Scol = reinterpret_cast<double *>(wscr + (size_t)FLAT_WARPS * n);  // P * n
    double *rpix = Scol + (size_t)P * n;                             // RP * n
    double *nupix = rpix + (size_t)RP * n;                           // RP * n
    double *invden = nupix + (size_t)RP * n;                         // RP * n: 1 / (1 + (lam - 1) tau nu)
    double *Sinv = invden + (size_t)RP * n;                          // P * n: 1 / S (0 where S = 0)
    double *fcol = Sinv + (size_t)P * n;                             // P * n: S / (S + lam tau)
    __shared__ double part[4];   // pix chi2, harm chi2, resid^2, spare
    __shared__ double red[FLAT_WARPS][3];

    for (int t = tid; t < n / 2; t += blockDim.x) {
        double s, co;
        sincospi(-2.0 * t / n, &s, &co);
        tw[t] = make_double2(co, s);
    }
    for (int i = tid; i < P * n; i += blockDim.x) {
        const int kl = i / n, ky = i % n;
        const int kx = c0 + kl;
        acol[i] = make_double2(0.0, 0.0);
        const double S = (kl < ncol) ? A.S[(size_t)ky * nh + kx] : 0.0;
        Scol[i] = S;
        Sinv[i] = S > 0.0 ? 1.0 / S : 0.0;
    }
    for (int i = tid; i < RP * n; i += blockDim.x) {
        const size_t g = (size_t)y0 * n + i;
        rpix[i] = A.r[g];
        nupix[i] = A.nu[g];
    }
    __syncthreads();

    // the per-pixel and per-mode factors of Eqs. (3) and (4) for one lambda (FP64 divisions
    // once per cooling level, not once per iteration)
    double cur_lam = NAN;
    auto set_level = [&](double lam) {
        const double lm1t = (lam - 1.0) * A.tau, lt = lam * A.tau;
        for (int i = tid; i < RP * n; i += blockDim.x) invden[i] = 1.0 / (1.0 + lm1t * nupix[i]);
        for (int i = tid; i < P * n; i += blockDim.x) {
            const double S = Scol[i];
            fcol[i] = S > 0.0 ? S / (S + lt) : 0.0;
        }
        cur_lam = lam;
        __syncthreads();
    };

    auto block_reduce3 = [&](double a, double b, double d) {
        for (int o = 16; o >= 1; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
            d += __shfl_xor_sync(0xffffffffu, d, o);
        }
        if (lane == 0) { red[warp][0] = a; red[warp][1] = b; red[warp][2] = d; }
        __syncthreads();
        if (tid == 0) {
            double s0 = 0, s1 = 0, s2 = 0;
            for (int w = 0; w < FLAT_WARPS; ++w) { s0 += red[w][0]; s1 += red[w][1]; s2 += red[w][2]; }
            part[0] = s0; part[1] = s1; part[2] = s2;
        }
        __syncthreads();
    };

    // ---- step 1: inverse column FFTs of acol into colbuf ----
    auto step1 = [&]() {
        for (int kl = warp; kl < ncol; kl += FLAT_WARPS) {
            double2 *x = colbuf + (size_t)kl * n;
            for (int ky = lane; ky < n; ky += 32) x[ky] = acol[(size_t)kl * n + ky];
            __syncwarp();
            warp_fft(x, logn, +1, tw);
            for (int y = lane; y < n; y += 32) x[y] = cscale(x[y], sy);
            __syncwarp();
        }
    };

    // ---- step 2: rows: gather, c2r, blend (or other use), r2c into rowbuf ----
    // Two real rows per complex FFT: the inverse DFT of Xa + i Xb (both Hermitian) is
    // xa + i xb, and the forward DFT Z of ta + i tb gives Ta = (Z_k + conj Z_-k) / 2 and
    // Tb = (Z_k - conj Z_-k) / 2i.
    auto step2 = [&](int mode, double lam) -> double {
        for (int i = tid; i < RP * nh; i += blockDim.x) {
            const int yl = i / nh, kx = i % nh;
            const int o = kx / P, kl = kx - o * P;
            const double2 *rc = cluster.map_shared_rank(colbuf, o);
            rowbuf[(size_t)yl * nh + kx] = rc[(size_t)kl * n + (y0 + yl)];
        }
        __syncthreads();
        const double lt = lam * A.tau;
        double acc = 0.0;
        double2 *x = wscr + (size_t)warp * n;
        for (int yp = warp; 2 * yp < RP; yp += FLAT_WARPS) {
            const int ya = 2 * yp;
            double2 *ba = rowbuf + (size_t)ya * nh, *bb = ba + nh;
            for (int kx = lane; kx < n; kx += 32) {
                double2 va, vb;
                if (kx < nh) {
                    va = ba[kx];
                    vb = bb[kx];
                } else {
                    va = cconj(ba[n - kx]);
                    vb = cconj(bb[n - kx]);
                }
                x[kx] = make_double2(va.x - vb.y, va.y + vb.x);
            }
            __syncwarp();
            warp_fft(x, logn, +1, tw);  // real part: row ya, imaginary part: row ya + 1
            for (int xx = lane; xx < n; xx += 32) {
                double tt[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const double s = (h ? x[xx].y : x[xx].x) * sx;
                    const int pi = (ya + h) * n + xx;
                    double t = s;
                    if (mode == FS_ITER) {
                        const double nv = nupix[pi], rv = rpix[pi], id = invden[pi];
                        t = s + lt * (rv - nv * s) * id;
                        acc += (nv * s * s - 2.0 * rv * s) * id;
                    } else if (mode == FS_PROLOGUE) {
                        t = rpix[pi];
                    } else if (mode == FS_FLUCT_SRC) {
                        const double rv = sqrt(nupix[pi]) * A.g1[(size_t)y0 * n + pi] + s;
                        rpix[pi] = rv;
                        t = rv;
                    } else {  // FS_OUT
                        A.s_out[(size_t)y0 * n + pi] = s;
                        const double nv = nupix[pi];
                        if (nv > 0.0) {
                            const double e = rpix[pi] - nv * s;
                            acc += e * e / nv;  // nu (d - s)^2
                        }
                    }
                    tt[h] = t;
                }
                x[xx] = make_double2(tt[0], tt[1]);
            }
            __syncwarp();
            if (mode == FS_ITER || mode == FS_PROLOGUE) {
                warp_fft(x, logn, -1, tw);
                for (int kx = lane; kx < nh; kx += 32) {
                    const double2 z = x[kx], zc = cconj(x[(n - kx) & (n - 1)]);
                    const double2 d = make_double2(0.5 * (z.x - zc.x), 0.5 * (z.y - zc.y));
                    ba[kx] = cscale(make_double2(0.5 * (z.x + zc.x), 0.5 * (z.y + zc.y)), sx);
                    bb[kx] = cscale(make_double2(d.y, -d.x), sx);
                }
            }
            __syncwarp();
        }
        return acc;
    };

    // ---- step 3: columns: gather, forward FFT, harmonic blend ----
    // mode FS_ITER: a = S/(S + lam tau) t_hat; chi2 of a_old; residual if lam == 1
    // mode FS_PROLOGUE: accumulate |t_hat|^2 (the b norm), a untouched
    auto step3 = [&](int mode, double lam, double &chi2h, double &res2) {
        for (int i = tid; i < ncol * n; i += blockDim.x) {
            const int kl = i / n, y = i % n;
            const int o = y / RP, yl = y - o * RP;
            const double2 *rb = cluster.map_shared_rank(rowbuf, o);
            colbuf[i] = rb[(size_t)yl * nh + (c0 + kl)];
        }
        __syncthreads();
        const bool full = (lam == 1.0);
        for (int kl = warp; kl < ncol; kl += FLAT_WARPS) {
            double2 *x = colbuf + (size_t)kl * n;
            warp_fft(x, logn, -1, tw);
            const int kx = c0 + kl;
            const double w = (kx == 0 || 2 * kx == n) ? 1.0 : 2.0;
            for (int ky = lane; ky < n; ky += 32) {
                const double2 th = cscale(x[ky], sy);
                const double S = Scol[(size_t)kl * n + ky];
                if (mode == FS_PROLOGUE) {
                    if (S > 0.0) res2 += w * (th.x * th.x + th.y * th.y);
                    continue;
                }
                const double2 ao = acol[(size_t)kl * n + ky];
                double2 an = make_double2(0.0, 0.0);
                if (S > 0.0) {
                    const double si = Sinv[(size_t)kl * n + ky];
                    an = cscale(th, fcol[(size_t)kl * n + ky]);
                    chi2h += w * (ao.x * ao.x + ao.y * ao.y) * si;
                    if (full) {
                        const double k = si + inv_tau;
                        const double dx = k * (ao.x - an.x), dy = k * (ao.y - an.y);
                        res2 += w * (dx * dx + dy * dy);
                    }
                }
                acol[(size_t)kl * n + ky] = an;
            }
            __syncwarp();
        }
    };

    // sum partial triplets over the cluster (same order in every CTA)
    auto cluster_sum = [&](double out[3]) {
        out[0] = out[1] = out[2] = 0.0;
        for (int o = 0; o < (int)cluster.num_blocks(); ++o) {
            const double *pp = cluster.map_shared_rank(part, o);
            out[0] += pp[0];
            out[1] += pp[1];
            out[2] += pp[2];
        }
    };

    double tot[3];
    // ---- fluctuation source: r = nu^1/2 g1 + F^-1 (S^-1/2 g2) ----
    if (A.g1) {
        for (int i = tid; i < ncol * n; i += blockDim.x) {
            const int kl = i / n, ky = i % n;
            const double S = Scol[i];
            const double f = S > 0.0 ? rsqrt(S) : 0.0;
            acol[i] = cscale(A.g2[(size_t)ky * nh + c0 + kl], f);
        }
        __syncthreads();
        step1();
        cluster.sync();
        step2(FS_FLUCT_SRC, 1.0);
        __syncthreads();
        for (int i = tid; i < P * n; i += blockDim.x) acol[i] = make_double2(0.0, 0.0);
        cluster.sync();
    }
    // ---- prologue: |b| = |F r| ----
    {
        step2(FS_PROLOGUE, 1.0);
        cluster.sync();
        double ch = 0.0, rs = 0.0;
        step3(FS_PROLOGUE, 1.0, ch, rs);
        block_reduce3(0.0, 0.0, rs);
        cluster.sync();
        cluster_sum(tot);
    }
    const double bnorm = sqrt(tot[2]);
    cluster.sync();

    // ---- iterations ----
    int k = 0, lev = 0, level_iters = 0, have_prev = 0, converged = 0, stop_reason = 0;
    double prev = 0.0, last_res = NAN, best = INFINITY;
    for (;;) {
        double lam;
        if (A.replay) {
            if (k >= A.nreplay) break;
            lam = A.replay[k];
        } else {
            if (k >= A.maxiter) { stop_reason = 2; break; }
            lam = A.levels[lev];
        }
        if (!(lam == cur_lam)) set_level(lam);
        step1();
        cluster.sync();
        const double pc = step2(FS_ITER, lam);
        cluster.sync();
        double ch = 0.0, rs = 0.0;
        step3(FS_ITER, lam, ch, rs);
        block_reduce3(pc, ch, rs);
        cluster.sync();
        cluster_sum(tot);
        const double chi2 = tot[0] + tot[1];
        const bool full = lam == 1.0;
        const double resid = full ? sqrt(tot[2]) / bnorm : NAN;
        if (c == 0 && tid == 0 && k < A.tr_cap) {
            A.tr_lam[k] = lam;
            A.tr_chi2[k] = chi2;
            A.tr_res[k] = resid;
        }
        ++k;
        if (full) {
            last_res = resid;
            if (!isfinite(resid) || (k > 50 && resid > 1e3 * best)) { stop_reason = 3; break; }
            best = fmin(best, resid);
        }
        if (A.replay) continue;
        if (lam == 1.0) {
            if (resid < A.tol) { converged = 1; stop_reason = 1; break; }
        } else {
            ++level_iters;
            const bool plateau = have_prev && fabs(chi2 - prev) < A.eta * A.sigma;
            if (plateau || level_iters >= A.level_cap) {
                lev = min(lev + 1, A.nlevels - 1);
                level_iters = 0;
                have_prev = 0;
                continue;
            }
        }
        prev = chi2;
        have_prev = 1;
    }
    if (A.replay && isfinite(last_res) && last_res < A.tol) converged = 1;
    // ---- output: s = F^-1 a, chi^2(s, 1) ----
    cluster.sync();
    step1();
    cluster.sync();
    const double pc = step2(FS_OUT, 1.0);
    double chh = 0.0;
    for (int i = tid; i < ncol * n; i += blockDim.x) {
        const int kl = i / n, ky = i % n;
        const int kx = c0 + kl;
        const double2 a = acol[i];
        if (A.alm_out) A.alm_out[(size_t)ky * nh + kx] = a;
        const double S = Scol[i];
        const double w = (kx == 0 || 2 * kx == n) ? 1.0 : 2.0;
        if (S > 0.0) chh += w * (a.x * a.x + a.y * a.y) / S;
    }
    block_reduce3(pc, chh, 0.0);
    cluster.sync();
    cluster_sum(tot);
    if (c == 0 && tid == 0) {
        A.status->iters = k;
        A.status->converged = converged;
        A.status->levels = lev + 1;
        A.status->stop_reason = stop_reason;
        A.status->final_resid = last_res;
        A.status->chi2_final = tot[0] + tot[1];
        A.status->bnorm = bnorm;
    }
    cluster.sync();  // keep every CTA's shared memory alive until all remote reads are done
}

// nu = N^-1 (0 where masked), r = nu d; tau = min N and count over observed pixels
__global__ void k_flat_setup(long long npix, const double *__restrict__ d, const double *__restrict__ nv,
                             const uint8_t *__restrict__ mask, double *__restrict__ r, double *__restrict__ nu,
                             double *__restrict__ out /* [min, count, flag] */)
{
    __shared__ double smin[32], scnt[32], sfl[32];
    double mn = INFINITY, cnt = 0, fl = 0;
    for (long long i = threadIdx.x; i < npix; i += blockDim.x) {
        const bool obs = mask ? mask[i] != 0 : true;
        double rv = 0.0, nuv = 0.0;
        if (obs) {
            const double N = nv[i], dv = d ? d[i] : 0.0;
            if (!(N > 0.0) || !isfinite(N) || !isfinite(dv)) fl = 1;
            else {
                nuv = 1.0 / N;
                rv = dv / N;
                mn = fmin(mn, N);
                cnt += 1;
            }
        }
        r[i] = rv;
        nu[i] = nuv;
    }
    for (int o = 16; o >= 1; o >>= 1) {
        mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        fl = fmax(fl, __shfl_xor_sync(0xffffffffu, fl, o));
    }
    if ((threadIdx.x & 31) == 0) {
        smin[threadIdx.x >> 5] = mn;
        scnt[threadIdx.x >> 5] = cnt;
        sfl[threadIdx.x >> 5] = fl;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = INFINITY, b = 0, f = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a = fmin(a, smin[w]);
            b += scnt[w];
            f = fmax(f, sfl[w]);
        }
        out[0] = a;
        out[1] = b;
        out[2] = f;
    }
}

// Cluster size of one solve of an n x n grid: FLAT_CS_MAX CTAs (half the columns and rows of
// each CTA, on twice the SMs) where the device co-schedules such a cluster with this kernel's
// shared memory and n >= 32 (the packed row FFTs need two rows per CTA), FLAT_CS otherwise.
// Decided once per device, after the kernel's shared-memory limit is set.
int flat_cluster_size(int n)
{
    if (n < 2 * FLAT_CS_MAX) return FLAT_CS;
    static std::mutex mu;
    static int cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return FLAT_CS;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (cache[dev]) return cache[dev];
    int cs = FLAT_CS;
    if (cudaFuncSetAttribute(k_flat_solve, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
        const int nm = FLAT_MAXN, nhm = nm / 2 + 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(FLAT_CS_MAX);
        cfg.blockDim = dim3(FLAT_THREADS);
        cfg.dynamicSmemBytes = flat_smem(nm, (nhm + FLAT_CS_MAX - 1) / FLAT_CS_MAX, nm / FLAT_CS_MAX, nhm);
        cudaLaunchAttribute at;
        at.id = cudaLaunchAttributeClusterDimension;
        at.val.clusterDim.x = FLAT_CS_MAX;
        at.val.clusterDim.y = 1;
        at.val.clusterDim.z = 1;
        cfg.attrs = &at;
        cfg.numAttrs = 1;
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, k_flat_solve, &cfg) == cudaSuccess && ncl >= 1) cs = FLAT_CS_MAX;
    }
    cudaGetLastError();  // an unsupported size leaves the portable one
    cache[dev] = cs;
    return cs;
}

// one solve: a single cluster of cs CTAs
wf_status flat_launch(const FlatArgs &A, int cs, size_t smem, cudaStream_t stream)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(FLAT_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = cs;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    WF_CUDA(cudaLaunchKernelEx(&cfg, k_flat_solve, A));
    return WF_OK;
}

}  // namespace

wf_status flat_create(wf_plan p)
{
    const int n = p->g.nx;
    if (p->g.ny != n) return set_error(WF_EUNSUPPORTED, "flat grid must be square");
    if (n < 16 || n > FLAT_MAXN || (n & (n - 1))) return set_error(WF_EUNSUPPORTED, "flat n must be a power of two in [16, 128]");
    FlatPlan *f = new (std::nothrow) FlatPlan();
    if (!f) return set_error(WF_ENOMEM, "host allocation");
    p->flat = f;
    f->n = n;
    f->logn = 0;
    while ((1 << f->logn) < n) ++f->logn;
    f->nh = n / 2 + 1;
    p->npix = (long long)n * n;
    p->nalm = (long long)n * f->nh;
    p->omega = 1.0;
    wf_status st;
    if ((st = plan_alloc(p, (void **)&f->r, p->npix * 8)) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&f->nu, p->npix * 8)) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&f->levels, 64 * 8)) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&f->status, sizeof(FlatStatus))) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&p->ws.redu, 16 * 8)) != WF_OK) return st;
    // the attribute is per function, shared by every plan: set it for the largest grid
    // (n = FLAT_MAXN) so that a smaller plan never lowers it under a larger one
    {
        const int nm = FLAT_MAXN, nhm = nm / 2 + 1, Pm = (nhm + FLAT_CS - 1) / FLAT_CS, RPm = nm / FLAT_CS;
        const size_t smax = flat_smem(nm, Pm, RPm, nhm);
        WF_CUDA(cudaFuncSetAttribute(k_flat_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax));
    }
    f->cs = flat_cluster_size(n);
    f->P = (f->nh + f->cs - 1) / f->cs;
    f->RP = n / f->cs;
    f->smem = flat_smem(n, f->P, f->RP, f->nh);
    return WF_OK;
}

void flat_destroy(wf_plan p)
{
    delete p->flat;
    p->flat = nullptr;
}

static wf_status ensure_trace(wf_plan p, int cap)
{
    FlatPlan *f = p->flat;
    if (f->tr_cap >= cap) return WF_OK;
    wf_status st;
    if ((st = plan_alloc(p, (void **)&f->tr_lam, (size_t)cap * 8)) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&f->tr_chi2, (size_t)cap * 8)) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&f->tr_res, (size_t)cap * 8)) != WF_OK) return st;
    f->tr_cap = cap;
    return WF_OK;
}

wf_status flat_solve(wf_plan p, const double *d, const double *noise_var, const uint8_t *mask, const double *S,
                     double tol, bool fluct, const double *g1, const double *g2, double *s_out, double *alm_out,
                     wf_info *info)
{
    FlatPlan *f = p->flat;
    const wf_options o = [&] {
        wf_options q = p->opt;
        if (q.maxiter <= 0) q.maxiter = 20000;
        if (q.level_cap <= 0) q.level_cap = 200;
        if (!(q.eta > 0)) q.eta = 1e-2;
        if (!(q.lambda_max > 0)) q.lambda_max = 100.0;
        return q;
    }();
    const int n = f->n, nh = f->nh;
    Prof pr(p, info, p->opt.profile != 0);
    k_flat_setup<<<1, 1024, 0, p->stream>>>(p->npix, fluct ? nullptr : d, noise_var, mask, f->r, f->nu, p->ws.redu);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    double h[3];
    WF_CUDA(cudaMemcpyAsync(h, p->ws.redu, sizeof h, cudaMemcpyDeviceToHost, p->stream));
    WF_CUDA(cudaStreamSynchronize(p->stream));
    if (h[2] != 0.0) return set_error(WF_EINVAL, "noise variance must be finite and > 0 (and d finite) on observed pixels");
    if (h[1] == 0.0) return set_error(WF_EINVAL, "every pixel is masked");
    const double tau = h[0];
    const long long ndof = (long long)h[1];

    // lambda levels: k_iter = 1, 2, 4, ...; lambda = clip(max S on |k| = k_iter / tau, 1, lambda_max)
    std::vector<double> Sh((size_t)n * nh);
    wf_status st = to_host(p, Sh.data(), S, Sh.size() * 8);
    if (st != WF_OK) return st;
    for (size_t i = 0; i < Sh.size(); ++i)
        if (!(Sh[i] >= 0.0 && std::isfinite(Sh[i])))
            return set_error(WF_EINVAL, "the prior S must be finite and >= 0 (mode %zu: %g)", i, Sh[i]);
    std::vector<double> lev{o.lambda_max};
    int kmax = 0;
    std::vector<int> kr(Sh.size());
    for (int ky = 0; ky < n; ++ky)
        for (int kx = 0; kx < nh; ++kx) {
            const int sy = ky < (n + 1) / 2 ? ky : ky - n;
            const int r = (int)std::lrint(std::sqrt((double)sy * sy + (double)kx * kx));
            kr[(size_t)ky * nh + kx] = r;
            kmax = std::max(kmax, r);
        }
    for (int kit = 2; lev.back() != 1.0; kit *= 2) {
        double lam = 1.0;
        if (kit <= kmax) {
            double smax = -1.0;
            for (size_t i = 0; i < Sh.size(); ++i)
                if (kr[i] == kit) smax = std::max(smax, Sh[i]);
            if (smax >= 0.0) lam = std::min(o.lambda_max, std::max(1.0, smax / tau));
        }
        if (lam != lev.back()) lev.push_back(lam);
        if ((int)lev.size() >= 60) { lev.push_back(1.0); break; }
    }
    WF_CUDA(cudaMemcpyAsync(f->levels, lev.data(), lev.size() * 8, cudaMemcpyHostToDevice, p->stream));
    const bool replay = !p->replay_lambda.empty();
    const int nrep = (int)p->replay_lambda.size();
    if (replay && nrep > f->replay_cap) {
        wf_status st = plan_alloc(p, (void **)&f->replay, (size_t)nrep * 8);
        if (st != WF_OK) return st;
        f->replay_cap = nrep;
    }
    if (replay)
        WF_CUDA(cudaMemcpyAsync(f->replay, p->replay_lambda.data(), nrep * 8, cudaMemcpyHostToDevice, p->stream));
    const int cap = replay ? nrep : o.maxiter;
    st = ensure_trace(p, std::max(cap, 1));
    if (st != WF_OK) return st;

    FlatArgs A{};
    A.n = n;
    A.logn = f->logn;
    A.nh = nh;
    A.P = f->P;
    A.RP = f->RP;
    A.r = f->r;
    A.nu = f->nu;
    A.S = S;
    A.g1 = fluct ? g1 : nullptr;
    A.g2 = fluct ? (const double2 *)g2 : nullptr;
    A.levels = f->levels;
    A.nlevels = (int)lev.size();
    A.replay = replay ? f->replay : nullptr;
    A.nreplay = nrep;
    A.tau = tau;
    A.sigma = std::sqrt(2.0 * (double)ndof);
    A.eta = o.eta;
    A.tol = tol;
    A.level_cap = o.level_cap;
    A.maxiter = o.maxiter;
    A.s_out = s_out;
    A.alm_out = (double2 *)alm_out;
    A.tr_lam = f->tr_lam;
    A.tr_chi2 = f->tr_chi2;
    A.tr_res = f->tr_res;
    A.tr_cap = f->tr_cap;
    A.status = f->status;
    pr.begin(WF_K_FLAT);
    if (wf_status ls = flat_launch(A, f->cs, f->smem, p->stream)) return ls;
    WF_COUNT_LAUNCH(p);
    pr.end();
    FlatStatus fs;
    WF_CUDA(cudaMemcpyAsync(&fs, f->status, sizeof fs, cudaMemcpyDeviceToHost, p->stream));
    WF_CUDA(cudaStreamSynchronize(p->stream));
    pr.collect();
    pr.finish();
    if (info) {
        info->iters = fs.iters;
        info->converged = fs.converged;
        info->final_residual = fs.final_resid;
        info->chi2_over_ndof = fluct ? NAN : fs.chi2_final / (double)ndof;
        info->n_dof = ndof;
        info->tau = tau;
        info->n_levels = fs.levels;
        info->refine_sweeps = 0;
        const int nt = std::min(fs.iters, info->trace_cap);
        if (nt > 0) {
            std::vector<double> tl(nt), tc(nt), trs(nt);
            if ((st = to_host(p, tl.data(), f->tr_lam, nt * 8)) != WF_OK) return st;
            if ((st = to_host(p, tc.data(), f->tr_chi2, nt * 8)) != WF_OK) return st;
            if ((st = to_host(p, trs.data(), f->tr_res, nt * 8)) != WF_OK) return st;
            for (int i = 0; i < nt; ++i) {
                if (info->lambda_trace) info->lambda_trace[i] = tl[i];
                if (info->L_trace) info->L_trace[i] = -1;
                if (info->chi2_trace) info->chi2_trace[i] = tc[i];
                if (info->resid_trace) info->resid_trace[i] = trs[i];
            }
        }
    }
    if (fs.stop_reason == 3) return set_error(WF_EDIVERGE, "residual grew (%.3e)", fs.final_resid);
    if (fs.stop_reason == 2) return set_error(WF_ENOCONV, "iteration cap reached (residual %.3e)", fs.final_resid);
    return WF_OK;
}

wf_status flat_alm2map(wf_plan p, const double *alm, double *map)
{
    return set_error(WF_EUNSUPPORTED, "flat-grid basis change is internal to the fused solve");
}

wf_status flat_map2alm(wf_plan p, const double *map, double *alm)
{
    return set_error(WF_EUNSUPPORTED, "flat-grid basis change is internal to the fused solve");
}

// ---------------------------------------------------------------------------
// Flat-grid solve that allocates nothing (wf_flat_solve_noalloc).
//
// For callers that cannot allocate device memory at solve time -- code that
// runs inside another framework's memory pool (a cudaMalloc there would go
// around the pool's accounting), or on a context where allocation is locked
// down -- this entry point runs the same two kernels as wf_solve on the flat grid
// (k_flat_setup, k_flat_solve), with the solver's scratch (the source and
// inverse-noise maps, the lambda levels, the status block and the per-
// iteration traces) in one file-scope device array instead of plan memory.
// Limits: n <= 128 (a power of two >= 16) and at most 20000 iterations;
// the array is 0.71 MiB and stays resident on every device that loads the
// library.  In host code the array's symbol is not a device address: every
// call looks up its address on the current device with cudaGetSymbolAddress,
// so no address outlives the context it belongs to (a cudaDeviceReset between
// calls is safe).  All calls share the one array: calls that overlap on the
// GPU race; everything a call reads is written by that call first.  The prior
// S must be finite and >= 0 (the largest S per radius is taken as an integer
// maximum over the bit patterns, an order that holds for S >= 0 only).
// ---------------------------------------------------------------------------
namespace {
constexpr int NOALLOC_MAXN = 128;
constexpr int NOALLOC_MAXITER = 20000;
constexpr int NOALLOC_LEVELS = 64;
constexpr size_t NA_PIX = (size_t)NOALLOC_MAXN * NOALLOC_MAXN;
constexpr size_t NA_R = 0;
constexpr size_t NA_NU = NA_R + NA_PIX * sizeof(double);
constexpr size_t NA_LEV = NA_NU + NA_PIX * sizeof(double);
constexpr size_t NA_RAD = NA_LEV + NOALLOC_LEVELS * sizeof(double);
constexpr size_t NA_REDU = NA_RAD + 32 * sizeof(double);
constexpr size_t NA_STATUS = NA_REDU + 16 * sizeof(double);
constexpr size_t NA_TRACE = NA_STATUS + 256;
constexpr size_t NA_BYTES = NA_TRACE + 3 * (size_t)NOALLOC_MAXITER * sizeof(double);

// max S over the half-plane modes whose rounded |k| equals 2^j, j = 1..15
// (-1 where no mode has that radius): the priors the flat schedule needs.
// out[16] counts the modes whose S is not finite and >= 0 (rejected by the
// caller: the maximum below compares bit patterns, valid for S >= 0 only).
__global__ void k_flat_radial_max(int n, const double *__restrict__ S, double *__restrict__ out)
{
    __shared__ unsigned long long best[16];
    __shared__ unsigned int bad;
    if (threadIdx.x < 16) best[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) bad = 0u;
    __syncthreads();
    const int nh = n / 2 + 1;
    for (int i = threadIdx.x; i < n * nh; i += blockDim.x) {
        if (!(S[i] >= 0.0 && isfinite(S[i]))) {
            atomicAdd(&bad, 1u);
            continue;
        }
        const int ky = i / nh, kx = i % nh;
        const int sy = ky < (n + 1) / 2 ? ky : ky - n;
        const long r = lrint(sqrt((double)sy * sy + (double)kx * kx));
        if (r >= 2 && (r & (r - 1)) == 0) {
            int j = 0;
            while ((1L << j) < r) ++j;
            if (j < 16) atomicMax(&best[j], (unsigned long long)__double_as_longlong(S[i]) | 0ull);
        }
    }
    __syncthreads();
    if (threadIdx.x < 16) {
        const unsigned long long b = best[threadIdx.x];
        out[threadIdx.x] = b ? __longlong_as_double((long long)b) : -1.0;
    }
    if (threadIdx.x == 0) out[16] = (double)bad;
}
}  // namespace

static __device__ __align__(256) unsigned char g_flat_noalloc_scratch[NA_BYTES];

namespace {
wf_status noalloc_base(unsigned char **out)
{
    void *p = nullptr;
    WF_CUDA(cudaGetSymbolAddress(&p, g_flat_noalloc_scratch));
    *out = (unsigned char *)p;
    return WF_OK;
}
}  // namespace

}  // namespace wf

extern "C" wf_status wf_flat_solve_noalloc(int n, const double *d, const double *noise_var, const uint8_t *mask,
                                           const double *S, double tol, const wf_options *opt, void *cuda_stream,
                                           double *s_wf, double *alm_out, wf_info *info)
{
    using namespace wf;
    if (!d || !noise_var || !S || !s_wf) return set_error(WF_EINVAL, "null argument");
    if (n < 16 || n > NOALLOC_MAXN || (n & (n - 1)))
        return set_error(WF_EINVAL, "wf_flat_solve_noalloc: n must be a power of two in [16, %d] (got %d)",
                         NOALLOC_MAXN, n);
    if (!(tol > 0)) return set_error(WF_EINVAL, "tol must be > 0");
    wf_options o = opt ? *opt : wf_options{};
    if (o.maxiter <= 0) o.maxiter = NOALLOC_MAXITER;
    if (o.maxiter > NOALLOC_MAXITER)
        return set_error(WF_EINVAL, "wf_flat_solve_noalloc: maxiter %d exceeds the %d iterations its scratch holds",
                         o.maxiter, NOALLOC_MAXITER);
    if (o.level_cap <= 0) o.level_cap = 200;
    if (!(o.eta > 0)) o.eta = 1e-2;
    if (!(o.lambda_max > 0)) o.lambda_max = 100.0;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    unsigned char *base = nullptr;
    wf_status st = noalloc_base(&base);
    if (st != WF_OK) return st;
    double *r = (double *)(base + NA_R), *nu = (double *)(base + NA_NU), *lev_d = (double *)(base + NA_LEV);
    double *rad = (double *)(base + NA_RAD), *redu = (double *)(base + NA_REDU);
    FlatStatus *status = (FlatStatus *)(base + NA_STATUS);
    double *tr = (double *)(base + NA_TRACE);
    const long long npix = (long long)n * n;
    const int nh = n / 2 + 1;

    k_flat_setup<<<1, 1024, 0, stream>>>(npix, d, noise_var, mask, r, nu, redu);
    WF_CUDA(cudaGetLastError());
    k_flat_radial_max<<<1, 256, 0, stream>>>(n, S, rad);
    WF_CUDA(cudaGetLastError());
    double h[3], smax[17];
    WF_CUDA(cudaMemcpyAsync(h, redu, sizeof h, cudaMemcpyDeviceToHost, stream));
    WF_CUDA(cudaMemcpyAsync(smax, rad, sizeof smax, cudaMemcpyDeviceToHost, stream));
    WF_CUDA(cudaStreamSynchronize(stream));
    if (h[2] != 0.0) return set_error(WF_EINVAL, "noise variance must be finite and > 0 (and d finite) on observed pixels");
    if (h[1] == 0.0) return set_error(WF_EINVAL, "every pixel is masked");
    if (smax[16] != 0.0)
        return set_error(WF_EINVAL, "the prior S must be finite and >= 0 (%.0f modes are not)", smax[16]);
    const double tau = h[0];
    const long long ndof = (long long)h[1];

    // lambda levels of the flat schedule: k_iter = 1, 2, 4, ..., first level at lambda_max
    double lev[NOALLOC_LEVELS];
    int nlev = 0;
    lev[nlev++] = o.lambda_max;
    for (int j = 1; lev[nlev - 1] != 1.0 && nlev < NOALLOC_LEVELS - 1; ++j) {
        double lam = 1.0;
        if (j < 16 && smax[j] >= 0.0) lam = std::min(o.lambda_max, std::max(1.0, smax[j] / tau));
        if (j >= 16) lam = 1.0;
        if (lam != lev[nlev - 1]) lev[nlev++] = lam;
    }
    if (lev[nlev - 1] != 1.0) lev[nlev++] = 1.0;
    WF_CUDA(cudaMemcpyAsync(lev_d, lev, nlev * sizeof(double), cudaMemcpyHostToDevice, stream));

    FlatArgs A{};
    A.n = n;
    A.logn = 0;
    while ((1 << A.logn) < n) ++A.logn;
    A.nh = nh;
    // (the cluster size is chosen below, once the kernel's shared-memory limit is set)
    A.r = r;
    A.nu = nu;
    A.S = S;
    A.levels = lev_d;
    A.nlevels = nlev;
    A.tau = tau;
    A.sigma = std::sqrt(2.0 * (double)ndof);
    A.eta = o.eta;
    A.tol = tol;
    A.level_cap = o.level_cap;
    A.maxiter = o.maxiter;
    A.s_out = s_wf;
    A.alm_out = (double2 *)alm_out;
    A.tr_lam = tr;
    A.tr_chi2 = tr + NOALLOC_MAXITER;
    A.tr_res = tr + 2 * NOALLOC_MAXITER;
    A.tr_cap = NOALLOC_MAXITER;
    A.status = status;
    {
        // the dynamic shared-memory limit is per function: set it for the largest grid this
        // entry point takes (n = NOALLOC_MAXN), on every call (a plan may have changed it)
        const int nm = NOALLOC_MAXN, nhm = nm / 2 + 1, Pm = (nhm + FLAT_CS - 1) / FLAT_CS, RPm = nm / FLAT_CS;
        const size_t smax = flat_smem(nm, Pm, RPm, nhm);
        WF_CUDA(cudaFuncSetAttribute(k_flat_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax));
    }
    const int cs = flat_cluster_size(n);
    A.P = (nh + cs - 1) / cs;
    A.RP = n / cs;
    if (wf_status ls = flat_launch(A, cs, flat_smem(n, A.P, A.RP, nh), stream)) return ls;
    FlatStatus fs;
    WF_CUDA(cudaMemcpyAsync(&fs, status, sizeof fs, cudaMemcpyDeviceToHost, stream));
    WF_CUDA(cudaStreamSynchronize(stream));
    if (info) {
        info->iters = fs.iters;
        info->converged = fs.converged;
        info->final_residual = fs.final_resid;
        info->chi2_over_ndof = fs.chi2_final / (double)ndof;
        info->n_dof = ndof;
        info->tau = tau;
        info->n_levels = fs.levels;
        info->refine_sweeps = 0;
        info->mixed_lc = 0;
        info->launches = 3;
        const int nt = std::min(fs.iters, info->trace_cap);
        if (nt > 0) {
            // ordered on the caller's stream like every other copy of this call
            if (info->lambda_trace)
                WF_CUDA(cudaMemcpyAsync(info->lambda_trace, A.tr_lam, nt * 8, cudaMemcpyDeviceToHost, stream));
            if (info->chi2_trace)
                WF_CUDA(cudaMemcpyAsync(info->chi2_trace, A.tr_chi2, nt * 8, cudaMemcpyDeviceToHost, stream));
            if (info->resid_trace)
                WF_CUDA(cudaMemcpyAsync(info->resid_trace, A.tr_res, nt * 8, cudaMemcpyDeviceToHost, stream));
            WF_CUDA(cudaStreamSynchronize(stream));
            if (info->L_trace)
                for (int i = 0; i < nt; ++i) info->L_trace[i] = -1;
        }
    }
    if (fs.stop_reason == 3) return set_error(WF_EDIVERGE, "residual grew (%.3e)", fs.final_resid);
    if (fs.stop_reason == 2) return set_error(WF_ENOCONV, "iteration cap reached (residual %.3e)", fs.final_resid);
    return WF_OK;
}
