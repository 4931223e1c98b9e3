// C ABI, plan construction and the solve driver of the messenger-field
// Wiener filter (Elsner & Wandelt 2013).
//
// One iteration on HEALPix (Sect. 2.1, Eqs. 3-4):
//   legendre synthesis  a_k        -> G_m(theta)        (wf_legendre.cu)
//   ring synthesis      G          -> s -> t (Eq. 3)    (wf_ring.cu)
//   ring analysis       t          -> F_m(theta)        (wf_ring.cu)
//   legendre analysis   F          -> a_{k+1} (Eq. 4)   (wf_legendre.cu)
//   reduce              chi^2 (Eq. 6) and the lambda = 1 residual
// with the cooling schedule of Sect. 3 run on the host between iterations
// (three FP64 scalars cross the PCIe/C2C link per iteration).  Polarised
// plans (ncomp = 3, Eqs. 10-11) run the same phases with the spin-2
// transforms and 3x3 blends of wf_spin.cu (FP64) and wf_spin_mx.cu (mixed).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <map>
#include <array>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "wf_internal.cuh"

namespace wf {

static thread_local char g_err[512] = "";

wf_status set_error(wf_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return s;
}

wf_status cuda_check(cudaError_t e, const char *what)
{
    (void)cudaGetLastError();  // do not leave a non-sticky error behind for the caller's next CUDA call
    if (e == cudaErrorMemoryAllocation) return set_error(WF_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return set_error(WF_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

wf_status raise_smem_limit(const void *func, size_t bytes)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> limit;
    int dev = 0;
    WF_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    size_t &cur = limit[{dev, func}];
    if (bytes <= cur) return WF_OK;
    WF_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    cur = bytes;
    return WF_OK;
}

wf_status to_device(wf_plan p, void *dst, const void *src, size_t bytes)
{
    WF_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, p->stream));
    return WF_OK;
}

wf_status to_host(wf_plan p, void *dst, const void *src, size_t bytes)
{
    WF_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, p->stream));
    WF_CUDA(cudaStreamSynchronize(p->stream));
    return WF_OK;
}

wf_status plan_alloc(wf_plan p, void **ptr, size_t bytes)
{
    void *d = nullptr;
    cudaError_t e = cudaMalloc(&d, bytes ? bytes : 16);
    if (e != cudaSuccess) return cuda_check(e, "cudaMalloc (plan)");
    p->allocations.push_back(d);
    p->device_bytes += (long long)bytes;
    *ptr = d;
    return WF_OK;
}

void Prof::init(wf_plan p_, wf_info *i, bool profile)
{
    p = p_;
    info = i;
    on = profile;
    for (int k = 0; k < WF_NK; ++k) k0[k] = p->kcnt[k];
    p->kfam = WF_K_OTHER;
    if (on && !p->events_ready) {
        for (auto &e : p->ev) cudaEventCreate(&e);
        p->events_ready = true;
    }
}

void Prof::begin(int family)
{
    p->kfam = family;
    if (!on || nopen >= 16) return;
    fam[nopen] = family;
    cudaEventRecord(p->ev[2 * nopen], p->stream);
}

void Prof::end()
{
    p->kfam = WF_K_OTHER;
    if (!on || nopen >= 16) return;
    cudaEventRecord(p->ev[2 * nopen + 1], p->stream);
    ++nopen;
}

void Prof::collect()
{
    if (!on) return;
    for (int i = 0; i < nopen; ++i) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, p->ev[2 * i], p->ev[2 * i + 1]) == cudaSuccess) ms[fam[i]] += t;
    }
    nopen = 0;
}

void Prof::iter_begin()
{
    if (on) cudaEventRecord(p->ev[32], p->stream);
}

double Prof::iter_end()
{
    if (!on) return NAN;
    cudaEventRecord(p->ev[33], p->stream);
    cudaEventSynchronize(p->ev[33]);
    float t = 0.f;
    cudaEventElapsedTime(&t, p->ev[32], p->ev[33]);
    return t;
}

void Prof::finish()
{
    p->kfam = WF_K_OTHER;
    for (int k = 0; k < WF_NK; ++k) {
        cnt[k] += p->kcnt[k] - k0[k];
        launches += p->kcnt[k] - k0[k];
        k0[k] = p->kcnt[k];
    }
    if (!info) return;
    info->launches = launches;
    for (int k = 0; k < WF_NK; ++k) {
        info->kernel_ms[k] = ms[k];
        info->kernel_launches[k] = cnt[k];
    }
}

namespace {

__device__ __forceinline__ void atomic_min_pos(double *addr, double v)
{
    // positive doubles order like their bit patterns
    atomicMin(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

// validate inputs, build nu = N^-1 (0 where masked) and the source r = nu d;
// reduce tau = min N over observed pixels and the observed count
template <typename T>
__global__ void k_setup(long long npix, const double *__restrict__ d, const double *__restrict__ nv,
                        const uint8_t *__restrict__ mask, T *__restrict__ r, T *__restrict__ nu,
                        double *__restrict__ scal, int *__restrict__ flag)
{
    unsigned long long cnt = 0;
    double mn = INFINITY;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += (long long)gridDim.x * blockDim.x) {
        const bool obs = mask ? (mask[i] != 0) : true;
        T rv = 0, nuv = 0;
        if (obs) {
            const double N = nv[i];
            const double dv = d ? d[i] : 0.0;
            if (!(N > 0.0) || !isfinite(N) || !isfinite(dv)) {
                atomicOr(flag, 1);
            } else {
                nuv = (T)(1.0 / N);
                rv = (T)(dv / N);
                mn = fmin(mn, N);
                ++cnt;
            }
        }
        r[i] = rv;
        nu[i] = nuv;
    }
    for (int o = 16; o >= 1; o >>= 1) {
        mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (cnt) {
            atomic_min_pos(&scal[0], mn);
            atomicAdd(reinterpret_cast<unsigned long long *>(&scal[1]), cnt);
        }
    }
}

// fluctuation source, Eq. (9): r = nu^1/2 g1 + Omega z with z = Y (S^-1/2 g2)
template <typename T>
__global__ void k_fluct_source(long long npix, const T *__restrict__ nu, const double *__restrict__ g1,
                               const double *__restrict__ z, double omega, T *__restrict__ r)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += (long long)gridDim.x * blockDim.x)
        r[i] = (T)(sqrt((double)nu[i]) * g1[i] + omega * z[i]);
}

// h_lm = S_l^-1/2 g2_lm (0 where S_l = 0)
__global__ void k_isqrt_S(int lmax, const double *__restrict__ S, const double2 *__restrict__ g2, double2 *__restrict__ h)
{
    const int m = blockIdx.x;
    const long long base = (long long)m * (2 * lmax + 3 - m) / 2;
    for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
        const double s = S[l];
        const double f = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
        const double2 g = g2[base + (l - m)];
        h[base + (l - m)] = make_double2(f * g.x, f * g.y);
    }
}

// per-m partial sums over a_lm: kind 0: sum_{S>0} w |v|^2 ; kind 1: sum_{S>0} w |v|^2 / S
__global__ void k_alm_norm(int lmax, const double *__restrict__ S, const double2 *__restrict__ v, int kind,
                           double *__restrict__ part)
{
    __shared__ double red[32];
    const int m = blockIdx.x;
    const long long base = (long long)m * (2 * lmax + 3 - m) / 2;
    const double wm = m == 0 ? 1.0 : 2.0;
    double s = 0.0;
    for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
        const double Sl = S[l];
        if (Sl > 0.0) {
            const double2 a = v[base + (l - m)];
            const double q = wm * (a.x * a.x + a.y * a.y);
            s += kind == 0 ? q : q / Sl;
        }
    }
    for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[m] = t;
    }
}

// per-block partials of sum_obs nu (d - s)^2
__global__ void k_pix_chi2(long long npix, const double *__restrict__ d, const double *__restrict__ nv,
                           const uint8_t *__restrict__ mask, const double *__restrict__ s, double *__restrict__ part)
{
    __shared__ double red[32];
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += (long long)gridDim.x * blockDim.x) {
        if (mask && !mask[i]) continue;
        const double e = d[i] - s[i];
        acc += e * e / nv[i];
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

// deterministic fixed-order sums: out[k] = sum_i in[off_k + i * stride_k], i < n_k
struct SumSpec {
    const double *in[5];
    int n[5];
    int stride[5];
};
__global__ void k_sums(SumSpec sp, int nsum, double *__restrict__ out)
{
    __shared__ double red[32];
    for (int k = 0; k < nsum; ++k) {
        double s = 0.0;
        for (int i = threadIdx.x; i < sp.n[k]; i += blockDim.x) s += sp.in[k][(long long)i * sp.stride[k]];
        for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            out[k] = t;
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void k_map_to_T(long long n, const double *__restrict__ in, T *__restrict__ out)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (T)in[i];
}

// out = x + s y over n complex coefficients (the correction form of the mixed iteration);
// out may be x or y
__global__ void k_alm_axpy(long long n, const double2 *x, const double2 *y, double s, double2 *out)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double2 a = x[i], b = y[i];
        out[i] = make_double2(a.x + s * b.x, a.y + s * b.y);
    }
}


// Template marginalisation (Sect. 3, Eq. 12): d = d_raw - V (V^T V)^-1 V^T d_raw,
// V = masked monopole and dipole templates (1, sin th cos ph, sin th sin ph, cos th).
// Pass 1: per-CTA partial sums of V^T d (4) and the upper triangle of V^T V (10).
__device__ __forceinline__ void pixel_templates(double x, int n, int q, int j, bool south, double v[4])
{
    double s, c;
    sincospi((double)(2 * j + q) / (double)n, &s, &c);
    const double st = sqrt((1.0 - x) * (1.0 + x));
    v[0] = 1.0;
    v[1] = st * c;
    v[2] = st * s;
    v[3] = south ? -x : x;
}

__global__ void k_template_sums(int npairs, const RingTab *__restrict__ rings, const double *__restrict__ xp,
                                const double *__restrict__ d, const uint8_t *__restrict__ mask,
                                double *__restrict__ part /* [14][gridDim.x] */)
{
    __shared__ double red[14][32];
    double acc[14];
#pragma unroll
    for (int k = 0; k < 14; ++k) acc[k] = 0.0;
    for (int pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
        const RingTab R = rings[pr];
        const double x = xp[pr];
        for (int h = 0; h < 2; ++h) {
            const long long off = h ? R.offS : R.offN;
            if (off < 0) continue;
            for (int j = threadIdx.x; j < R.n; j += blockDim.x) {
                const long long i = off + j;
                if (mask && !mask[i]) continue;
                double v[4];
                pixel_templates(x, R.n, R.q, j, h == 1, v);
                const double dv = d[i];
                int t = 4;
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    acc[a] += v[a] * dv;
#pragma unroll
                    for (int b = a; b < 4; ++b) acc[t++] += v[a] * v[b];
                }
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 14; ++k) {
        double s = acc[k];
        for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[k][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x < 14) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
        part[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
    }
}

__global__ void k_template_apply(int npairs, const RingTab *__restrict__ rings, const double *__restrict__ xp,
                                 const double *__restrict__ d, const uint8_t *__restrict__ mask, double c0,
                                 double c1, double c2, double c3, double *__restrict__ out)
{
    for (int pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
        const RingTab R = rings[pr];
        const double x = xp[pr];
        for (int h = 0; h < 2; ++h) {
            const long long off = h ? R.offS : R.offN;
            if (off < 0) continue;
            for (int j = threadIdx.x; j < R.n; j += blockDim.x) {
                const long long i = off + j;
                double r = d[i];
                if (!mask || mask[i]) {
                    double v[4];
                    pixel_templates(x, R.n, R.q, j, h == 1, v);
                    r -= c0 * v[0] + c1 * v[1] + c2 * v[2] + c3 * v[3];
                }
                out[i] = r;
            }
        }
    }
}

// solve the symmetric 4x4 system G c = b by Gaussian elimination with partial pivoting
bool solve4(double G[4][4], double b[4], double c[4])
{
    double A[4][5];
    for (int i = 0; i < 4; ++i) {
        for (int j = 0; j < 4; ++j) A[i][j] = G[i][j];
        A[i][4] = b[i];
    }
    for (int k = 0; k < 4; ++k) {
        int piv = k;
        for (int i = k + 1; i < 4; ++i)
            if (std::fabs(A[i][k]) > std::fabs(A[piv][k])) piv = i;
        if (A[piv][k] == 0.0) return false;
        for (int j = 0; j < 5; ++j) std::swap(A[k][j], A[piv][j]);
        for (int i = k + 1; i < 4; ++i) {
            const double f = A[i][k] / A[k][k];
            for (int j = k; j < 5; ++j) A[i][j] -= f * A[k][j];
        }
    }
    for (int i = 3; i >= 0; --i) {
        double s = A[i][4];
        for (int j = i + 1; j < 4; ++j) s -= A[i][j] * c[j];
        c[i] = s / A[i][i];
    }
    return true;
}


// chi^2-bound cooling (Sect. 2.2): pixel sums at u = (lambda - 1) tau for the
// current synthesis s,  A(u) = sum (d - s)^2 / (N + u) = sum (r - nu s)^2 / (nu (1 + u nu)),
// D(u) = -dA/du = sum (r - nu s)^2 / (1 + u nu)^2, over observed pixels; per-block partials.
template <typename T>
__global__ void k_pixsums(long long npix, const T *__restrict__ r, const T *__restrict__ nu, const T *__restrict__ s,
                          double u, double *__restrict__ part /* [2][gridDim.x] */)
{
    __shared__ double red[2][32];
    double A = 0.0, D = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += (long long)gridDim.x * blockDim.x) {
        const double nv = (double)nu[i];
        if (nv > 0.0) {
            const double e = (double)r[i] - nv * (double)s[i];
            const double den = 1.0 + u * nv;
            A += e * e / (nv * den);
            D += e * e / (den * den);
        }
    }
    for (int o = 16; o >= 1; o >>= 1) {
        A += __shfl_xor_sync(0xffffffffu, A, o);
        D += __shfl_xor_sync(0xffffffffu, D, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = A;
        red[1][threadIdx.x >> 5] = D;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += red[0][w];
            b += red[1][w];
        }
        part[blockIdx.x] = a;
        part[gridDim.x + blockIdx.x] = b;
    }
}

// Eq. (3) blend in place on the synthesised map: t = s + lam tau (r - nu s) / (1 + (lam - 1) tau nu)
template <typename T>
__global__ void k_blend(long long npix, const T *__restrict__ r, const T *__restrict__ nu, T *__restrict__ st, T lt,
                        T lm1t)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += (long long)gridDim.x * blockDim.x) {
        const T s = st[i], nv = nu[i];
        st[i] = s + lt * (r[i] - nv * s) / ((T)1 + lm1t * nv);
    }
}

int grid_for(long long n, int nsm) { return (int)std::min<long long>((n + 255) / 256, (long long)nsm * 8); }

// reduce the partial sums in a fixed order into ws.scal and copy them to the
// pinned host mirror ws.h_scal (enqueued only: valid after the stream syncs)
wf_status sums_enqueue(wf_plan p, SumSpec sp, int nsum)
{
    k_sums<<<1, 256, 0, p->stream>>>(sp, nsum, p->ws.scal);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    WF_CUDA(cudaMemcpyAsync(p->ws.h_scal, p->ws.scal, nsum * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    return WF_OK;
}

wf_status sums(wf_plan p, SumSpec sp, int nsum, Prof *pr = nullptr)
{
    wf_status st = sums_enqueue(p, sp, nsum);
    if (st != WF_OK) return st;
    WF_CUDA(cudaStreamSynchronize(p->stream));
    return WF_OK;
}


// A(u), D(u) of the chi^2-bound schedule for the synthesis currently in ws.t
wf_status pix_sums(wf_plan p, double u, double *A, double *D, Prof *pr)
{
    const int grid = std::min((int)((p->npix + 255) / 256), 2 * p->nsm);
    if (p->prec == WF_PREC_FP64)
        k_pixsums<double><<<grid, 256, 0, p->stream>>>(p->npix, (const double *)p->ws.r, (const double *)p->ws.nu,
                                                       (const double *)p->ws.t, u, p->ws.part_pix);
    else
        k_pixsums<float><<<grid, 256, 0, p->stream>>>(p->npix, (const float *)p->ws.r, (const float *)p->ws.nu,
                                                      (const float *)p->ws.t, u, p->ws.part_pix);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    SumSpec sp{};
    sp.in[0] = p->ws.part_pix;
    sp.n[0] = grid;
    sp.stride[0] = 1;
    sp.in[1] = p->ws.part_pix + grid;
    sp.n[1] = grid;
    sp.stride[1] = 1;
    wf_status st = sums(p, sp, 2, pr);
    if (st != WF_OK) return st;
    *A = p->ws.h_scal[0];
    *D = p->ws.h_scal[1];
    return WF_OK;
}

// Root of g(u) = h + A(u) - b on [0, hi] (g decreasing and convex in u):
// safeguarded Newton inside a shrinking bracket.  Returns 0 when g(0) <= 0;
// when g(hi) > 0 it widens hi by factors of 4 if `expand` (the first lambda),
// else returns hi (lambda never rises).
wf_status bound_root(wf_plan p, double h, double b, double hi, bool expand, double *u_out, double *chi2_out, Prof *pr)
{
    double A, D;
    wf_status st = pix_sums(p, 0.0, &A, &D, pr);
    if (st != WF_OK) return st;
    if (h + A - b <= 0.0) {
        *u_out = 0.0;
        *chi2_out = h + A;
        return WF_OK;
    }
    double lo = 0.0, u = hi;
    if ((st = pix_sums(p, u, &A, &D, pr)) != WF_OK) return st;
    double g = h + A - b;
    while (expand && g > 0.0 && u < 1e300) {  // bracket from above (the first lambda only)
        lo = u;
        u *= 4.0;
        if ((st = pix_sums(p, u, &A, &D, pr)) != WF_OK) return st;
        g = h + A - b;
    }
    if (g >= 0.0) {
        *u_out = u;
        *chi2_out = h + A;
        return WF_OK;
    }
    hi = u;
    for (int it = 0; it < 100; ++it) {
        double un = u + g / D;  // Newton: g' = -D
        if (!(un > lo && un < hi)) un = 0.5 * (lo + hi);
        if ((st = pix_sums(p, un, &A, &D, pr)) != WF_OK) return st;
        const double gn = h + A - b;
        if (gn > 0.0) lo = un;
        else hi = un;
        const bool done = std::fabs(un - u) <= 1e-13 * std::max(un, 1e-300) || std::fabs(gn) <= 1e-13 * b;
        u = un;
        g = gn;
        if (done) break;
    }
    *u_out = u;
    *chi2_out = h + A;
    return WF_OK;
}

// Sect. 3 heuristic cooling on the sphere (same rules as the oracle's)
struct HpSchedule {
    std::vector<double> c;
    double tau_h = 0;
    int lmax = 0, ell_iter = 0, step_max = 500, margin = 100;
    double lam = 1;
    int L = 0;
    void level()
    {
        if (ell_iter >= lmax) { lam = 1.0; L = lmax; return; }
        lam = std::max(1.0, c[ell_iter] / tau_h);
        L = std::min(lmax, ell_iter + margin);
    }
    bool final_level() const { return lam == 1.0 && L == lmax; }
    void advance()
    {
        const double l0 = lam;
        const int L0 = L;
        for (;;) {
            ell_iter = std::min(2 * ell_iter, ell_iter + step_max);
            level();
            if (lam != l0 || L != L0 || final_level()) return;
        }
    }
};

// HEALPix defaults.  The plateau constant and level cap decide how long each
// lambda level of the Sect. 3 cooling runs (the paper gives no values): a
// strict plateau (eta = 3e-5 of sigma_chi2) removes more of the slow modes'
// error while lambda > 1, where they converge faster (Eq. 5), and reached 1e-4
// three times sooner than eta = 1e-2 on the nside 512 and 2048 workloads and on
// the serving problems.  Fluctuation solves (Eq. 9), whose source excites the
// masked high-prior modes, rarely meet that plateau: the cap of 300 iterations
// per level bounds their levels (a 3000 cap took them 2-4x more iterations)
// and leaves the Wiener-filter solves unchanged (they leave each level on the
// plateau).  The flat grid keeps its own schedule (flat_solve).
wf_options defaults(wf_options o)
{
    if (o.maxiter <= 0) o.maxiter = 20000;
    if (o.level_cap <= 0) o.level_cap = 300;
    if (!(o.eta > 0)) o.eta = 3e-5;
    if (o.ell0 <= 0) o.ell0 = 20;
    if (o.ell_step_max <= 0) o.ell_step_max = 500;
    if (o.band_margin <= 0) o.band_margin = 100;
    if (!(o.lambda_max > 0)) o.lambda_max = 100.0;
    if (o.refine_sweeps < 0) o.refine_sweeps = 0;
    if (!(o.mixed_kappa > 0)) o.mixed_kappa = 3e4;
    if (!(o.m_sigma > 0)) o.m_sigma = 5.0;
    if (!(o.stall_tol > 0)) o.stall_tol = 1e-7;
    return o;
}

void record(wf_info *info, int k, double lam, int L, double chi2, double resid, double ms)
{
    if (!info || k >= info->trace_cap) return;
    if (info->lambda_trace) info->lambda_trace[k] = lam;
    if (info->L_trace) info->L_trace[k] = L;
    if (info->chi2_trace) info->chi2_trace[k] = chi2;
    if (info->resid_trace) info->resid_trace[k] = resid;
    if (info->iter_ms_trace) info->iter_ms_trace[k] = ms;
}

template <typename T>
wf_status hp_setup_T(wf_plan p, const double *d, const double *nv, const uint8_t *mask, double *tau, long long *ndof)
{
    const double init[2] = {std::numeric_limits<double>::infinity(), 0.0};
    WF_CUDA(cudaMemcpyAsync(p->ws.scal, init, sizeof init, cudaMemcpyHostToDevice, p->stream));
    WF_CUDA(cudaMemsetAsync(p->ws.flag, 0, sizeof(int), p->stream));
    k_setup<T><<<grid_for(p->npix, p->nsm), 256, 0, p->stream>>>(p->npix, d, nv, mask, (T *)p->ws.r, (T *)p->ws.nu,
                                                                 p->ws.scal, p->ws.flag);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    int flag = 0;
    double sc[2];
    WF_CUDA(cudaMemcpyAsync(sc, p->ws.scal, sizeof sc, cudaMemcpyDeviceToHost, p->stream));
    WF_CUDA(cudaMemcpyAsync(&flag, p->ws.flag, sizeof flag, cudaMemcpyDeviceToHost, p->stream));
    WF_CUDA(cudaStreamSynchronize(p->stream));
    unsigned long long cnt;
    std::memcpy(&cnt, &sc[1], sizeof cnt);
    if (flag) return set_error(WF_EINVAL, "noise variance must be finite and > 0 (and d finite) on observed pixels");
    if (cnt == 0) return set_error(WF_EINVAL, "every pixel is masked");
    *tau = sc[0];
    *ndof = (long long)cnt;
    return WF_OK;
}

wf_status hp_setup(wf_plan p, const double *d, const double *nv, const uint8_t *mask, double *tau, long long *ndof)
{
    return p->prec == WF_PREC_FP64 ? hp_setup_T<double>(p, d, nv, mask, tau, ndof)
                                   : hp_setup_T<float>(p, d, nv, mask, tau, ndof);
}

// map (FP64) = Y a, restricted to l <= L
wf_status hp_alm2map(wf_plan p, const double2 *a, int L, double *map)
{
    wf_status st = hp_legendre_synthesis(p, a, L);
    if (st != WF_OK) return st;
    return hp_ring_synthesis(p, L, RS_MAP, 1.0, 0.0, map);
}

// out = Y^T map_T (map in the working precision), l <= L; entries above L zeroed
wf_status hp_adjoint_T(wf_plan p, const void *map_T, int L, double2 *out)
{
    WF_CUDA(cudaMemsetAsync(out, 0, p->nalm * sizeof(double2), p->stream));
    wf_status st = hp_ring_analysis(p, L, map_T);
    if (st != WF_OK) return st;
    BlendArgs ba;
    return hp_legendre_analysis(p, L, LEG_ADJOINT, ba, nullptr, out);
}

// Resumable state of one HEALPix solve.  hp_solve runs
//   begin -> { pick -> launch -> (stream sync) -> absorb } -> end
// on the plan's stream; the batch solver runs the same phases for several
// plans, with the launches of one step of all of them captured in one graph.
struct HpRun {
    wf_plan p = nullptr;
    const double *d = nullptr, *nv = nullptr, *C_ell = nullptr, *g1 = nullptr, *g2 = nullptr;
    const uint8_t *mask = nullptr;
    double tol = 0;
    double tol_stop = 0;  // the mixed phase stops below this (tol, or tol x mixed_tol_factor before FP64 sweeps)
    bool fluct = false;
    double *s_out = nullptr, *alm_out = nullptr;
    wf_info *info = nullptr;
    const double2 *a_init = nullptr;
    bool copy_back = false;  // a <- a_new by a device copy in the iteration (pointers fixed for graphs)
    bool graph = false;      // the launches are being captured: no profiling events
    wf_options o{};
    int lmax = 0;
    double tau = 0, tau_h = 0, bnorm = 0, sigma = 0;
    long long ndof = 0;
    int lc = 0;
    HpSchedule sch;
    bool replay = false, rigorous = false;
    int nrep = 0;
    double bound = 0, u_cur = 0, h_cur = 0, q_cur = 0;
    int bound_updates = 0;
    int k = 0, level_iters = 0, levels = 1;
    bool have_prev = false, converged = false, chi2_bad = false;
    double prev_chi2 = 0, last_resid = NAN, best_resid = INFINITY;
    wf_status result = WF_OK;
    double lam = 1.0, chi2_bound = NAN;  // the current iteration
    int L = 0;
    bool corr = false, corr_pending = false;  // correction form (mixed_correction): on / due at the next launch
    Prof pr;
};

wf_status hp_begin_pol(HpRun &R);
wf_status hp_launch_pol(HpRun &R);
// a bounded wait of a tensor-core kernel that gave up voids the result (WF_ETIMEOUT; the flag is cleared)
wf_status tc_check(wf_plan p)
{
    if (!tc_prec(p->prec)) return WF_OK;
    int tc_err = 0;
    WF_CUDA(cudaMemcpyAsync(&tc_err, p->ws.tc_err, sizeof tc_err, cudaMemcpyDeviceToHost, p->stream));
    WF_CUDA(cudaStreamSynchronize(p->stream));
    if (!tc_err) return WF_OK;
    WF_CUDA(cudaMemsetAsync(p->ws.tc_err, 0, sizeof(int), p->stream));
    return set_error(WF_ETIMEOUT, "a tensor-core kernel's bounded wait for its MMAs gave up");
}

wf_status hp_end_pol(HpRun &R);

wf_status hp_begin(HpRun &R)
{
    wf_plan p = R.p;
    R.o = defaults(p->opt);
    const wf_options &o = R.o;
    const int lmax = R.lmax = p->lmax;
    // mixed precision with FP64 correction sweeps: the FP32 phase may stop below a tighter
    // tolerance, so that the result's FP64-operator residual, which the sweeps check, is below tol
    R.tol_stop = R.tol;
    if (p->prec != WF_PREC_FP64 && o.refine_sweeps > 0 && o.mixed_tol_factor > 0.0 && o.mixed_tol_factor < 1.0)
        R.tol_stop = R.tol * o.mixed_tol_factor;
    if (p->pol) return hp_begin_pol(R);
    if (o.schedule == 1 && R.fluct && p->replay_lambda.empty())
        return set_error(WF_EUNSUPPORTED, "the chi^2-bound schedule needs data (Wiener filter, not wf_fluct)");
    if (o.schedule == 1 && R.a_init && p->replay_lambda.empty())
        return set_error(WF_EUNSUPPORTED, "chi^2-bound schedule with a starting iterate");
    R.pr.init(p, R.info, o.profile != 0 && !R.graph);
    wf_status st = hp_setup(p, R.fluct ? nullptr : R.d, R.nv, R.mask, &R.tau, &R.ndof);
    if (st != WF_OK) return st;
    const double tau_h = R.tau_h = R.tau * p->omega;
    HpSchedule &sch = R.sch;
    sch.c.resize(lmax + 1);
    if ((st = to_host(p, sch.c.data(), R.C_ell, (lmax + 1) * sizeof(double))) != WF_OK) return st;
    for (int l = 0; l <= lmax; ++l)
        if (!(sch.c[l] >= 0.0 && std::isfinite(sch.c[l])))
            return set_error(WF_EINVAL, "C_ell must be finite and >= 0 (l = %d: %g)", l, sch.c[l]);
    // Mixed precision: the messenger iteration contracts a mode by about
    // tau_h / S_l per iteration where the mask leaves it unconstrained, so a
    // systematic operator error larger than that margin makes the iteration
    // grow.  Modes with S_l / tau_h >= kappa take the FP64 block.
    R.lc = 0;
    if (p->prec != WF_PREC_FP64) {
        if (o.mixed_lc > 0) R.lc = std::min(o.mixed_lc, lmax + 1);
        else if (o.mixed_lc == 0)
            for (int l = lmax; l >= 0; --l)
                if (sch.c[l] / tau_h >= o.mixed_kappa) { R.lc = l + 1; break; }
        if ((st = hp_set_low_block(p, R.lc)) != WF_OK) return st;
    }
    if (R.fluct) {
        // r = nu^1/2 g1 + Omega Y (S^-1/2 g2), z synthesised into the output map as scratch
        k_isqrt_S<<<lmax + 1, 256, 0, p->stream>>>(lmax, R.C_ell, (const double2 *)R.g2, p->ws.a_new);
        WF_COUNT_LAUNCH(p);
        WF_CUDA(cudaGetLastError());
        if ((st = hp_alm2map(p, p->ws.a_new, lmax, R.s_out)) != WF_OK) return st;
        if (p->prec == WF_PREC_FP64)
            k_fluct_source<double><<<grid_for(p->npix, p->nsm), 256, 0, p->stream>>>(
                p->npix, (const double *)p->ws.nu, R.g1, R.s_out, p->omega, (double *)p->ws.r);
        else
            k_fluct_source<float><<<grid_for(p->npix, p->nsm), 256, 0, p->stream>>>(
                p->npix, (const float *)p->ws.nu, R.g1, R.s_out, p->omega, (float *)p->ws.r);
        WF_COUNT_LAUNCH(p);
        WF_CUDA(cudaGetLastError());
    }
    // |b| = |Y^T r| over modes with S > 0 (correction sweeps reuse their parent solve's,
    // which differs from this plan's only by the parent's transform rounding)
    if (p->bnorm_given > 0) {
        R.bnorm = p->bnorm_given;
    } else {
        if ((st = hp_adjoint_T(p, p->ws.r, lmax, p->ws.b)) != WF_OK) return st;
        k_alm_norm<<<lmax + 1, 256, 0, p->stream>>>(lmax, R.C_ell, p->ws.b, 0, p->ws.part_harm);
        WF_COUNT_LAUNCH(p);
        WF_CUDA(cudaGetLastError());
        SumSpec sp{};
        sp.in[0] = p->ws.part_harm;
        sp.n[0] = lmax + 1;
        sp.stride[0] = 1;
        if ((st = sums(p, sp, 1, &R.pr)) != WF_OK) return st;
        R.bnorm = std::sqrt(p->ws.h_scal[0]);
    }
    if (!(R.bnorm > 0)) return set_error(WF_EINVAL, "the source has no component on modes with S > 0");

    sch.tau_h = tau_h;
    sch.lmax = lmax;
    sch.step_max = o.ell_step_max;
    sch.margin = o.band_margin;
    sch.ell_iter = std::min(o.ell0, lmax);
    sch.level();

    if (R.a_init)
        WF_CUDA(cudaMemcpyAsync(p->ws.a, R.a_init, p->nalm * sizeof(double2), cudaMemcpyDeviceToDevice, p->stream));
    else
        WF_CUDA(cudaMemsetAsync(p->ws.a, 0, p->nalm * sizeof(double2), p->stream));
    WF_CUDA(cudaMemsetAsync(p->ws.a_new, 0, p->nalm * sizeof(double2), p->stream));
    R.replay = !p->replay_lambda.empty();
    R.nrep = (int)p->replay_lambda.size();
    R.rigorous = o.schedule == 1 && !R.replay;  // a replay overrides the schedule
    R.bound = (double)R.ndof - o.m_sigma * std::sqrt(2.0 * (double)R.ndof);
    if (R.rigorous && !(R.bound > 0.0))
        return set_error(WF_EINVAL, "chi^2 bound n_dof - m sigma = %.3g is not positive (too few observed pixels)",
                         R.bound);
    R.sigma = std::sqrt(2.0 * (double)R.ndof);
    return WF_OK;
}

// (lambda, L) of iteration R.k; false when the loop is over (R.result set)
bool hp_pick(HpRun &R)
{
    wf_plan p = R.p;
    if (R.replay) {
        if (R.k >= R.nrep) return false;
        R.lam = p->replay_lambda[R.k];
        R.L = std::min(std::max(p->replay_L[R.k], 0), R.lmax);
    } else {
        if (R.k >= R.o.maxiter) {
            R.result = WF_ENOCONV;
            return false;
        }
        R.lam = R.sch.lam;
        R.L = R.sch.L;
    }
    return true;
}

wf_status alm_axpy(wf_plan p, const double2 *x, const double2 *y, double s, double2 *out)
{
    k_alm_axpy<<<grid_for(p->nalm, p->nsm), 256, 0, p->stream>>>(p->nalm, x, y, s, out);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    return WF_OK;
}

wf_status hp_launch(HpRun &R);
bool hp_absorb(HpRun &R);

// The switch to the correction form of the mixed iteration (wf_options.mixed_correction).
// The messenger iteration (Eqs. 3-4) is affine, G(a) = B a + c.  One FP64 iteration from the
// current iterate x0, on the FP64 sub-plan of the correction sweeps, gives a1 = G(x0); the
// plan's a then holds delta = a - x0, starting at d0 = a1 - x0, and the FP32 kernels apply
// G(x0 + delta) - x0 = d0 + B delta (hp_launch).  The FP64 iteration is one iteration of the
// trace (synchronous; its residual is the FP64 operator's at x0).
wf_status hp_enter_correction(HpRun &R)
{
    wf_plan p = R.p;
    const wf_options &o = R.o;
    const int lmax = R.lmax;
    const size_t abytes = (size_t)p->nalm * sizeof(double2);
    wf_status st;
    // each buffer on its own, so that a failed allocation leaves no half-set state behind
    if (!p->ws.cx0 && (st = plan_alloc(p, (void **)&p->ws.cx0, abytes)) != WF_OK) return st;
    if (!p->ws.cd0 && (st = plan_alloc(p, (void **)&p->ws.cd0, abytes)) != WF_OK) return st;
    if (!p->ws.caold && (st = plan_alloc(p, (void **)&p->ws.caold, abytes)) != WF_OK) return st;
    if (!p->ws.r0) {
        void *z = nullptr;
        if ((st = plan_alloc(p, &z, (size_t)p->npix * sizeof(float))) != WF_OK) return st;
        WF_CUDA(cudaMemsetAsync(z, 0, (size_t)p->npix * sizeof(float), p->stream));
        p->ws.r0 = z;  // set once it is zero
    }
    if (!p->sub) {
        wf_plan sub = nullptr;
        if ((st = wf_plan_create(&p->g, lmax, WF_PREC_FP64, (void *)p->stream, &sub)) != WF_OK) return st;
        p->sub = sub;
    }
    wf_plan sub = p->sub;
    sub->df_legendre = o.fp64_emulation >= 0;
    sub->stream = p->stream;
    sub->opt = p->opt;
    sub->opt.profile = o.profile;
    sub->opt.refine_sweeps = 0;
    sub->opt.schedule = 0;
    sub->opt.mixed_correction = 0;
    sub->replay_lambda.assign(1, 1.0);
    sub->replay_L.assign(1, lmax);
    WF_CUDA(cudaMemcpyAsync(p->ws.cx0, p->ws.a, abytes, cudaMemcpyDeviceToDevice, p->stream));
    double t_lam = NAN, t_chi2 = NAN, t_res = NAN, t_ms = NAN;
    int t_L = 0;
    wf_info si{};
    si.lambda_trace = &t_lam;
    si.L_trace = &t_L;
    si.chi2_trace = &t_chi2;
    si.resid_trace = &t_res;
    si.iter_ms_trace = &t_ms;
    si.trace_cap = 1;
    HpRun S;
    S.p = sub;
    S.d = R.d;
    S.nv = R.nv;
    S.mask = R.mask;
    S.C_ell = R.C_ell;
    S.tol = R.tol;
    S.fluct = R.fluct;
    S.g1 = R.g1;
    S.g2 = R.g2;
    S.s_out = R.s_out;  // scratch of the fluctuation source; written again at the end
    S.info = &si;
    S.a_init = p->ws.cx0;
    sub->bnorm_given = R.bnorm;
    st = hp_begin(S);
    if (st == WF_OK) {
        if (!hp_pick(S)) {
            st = set_error(WF_ECUDA, "correction form: the FP64 step did not run");
        } else if ((st = hp_launch(S)) == WF_OK) {
            WF_CUDA(cudaStreamSynchronize(p->stream));
            hp_absorb(S);
        }
    }
    sub->bnorm_given = 0;
    S.pr.finish();
    if (st != WF_OK) return st;
    // delta_0 = d0 = a1 - x0 (a1 is the sub-plan's iterate after the absorb)
    if ((st = alm_axpy(p, sub->ws.a, p->ws.cx0, -1.0, p->ws.cd0)) != WF_OK) return st;
    WF_CUDA(cudaMemcpyAsync(p->ws.a, p->ws.cd0, abytes, cudaMemcpyDeviceToDevice, p->stream));
    for (int f = 0; f < WF_NK; ++f) {
        R.pr.ms[f] += si.kernel_ms[f];
        R.pr.cnt[f] += si.kernel_launches[f];
    }
    R.pr.launches += si.launches;
    record(R.info, R.k, 1.0, lmax, NAN, S.last_resid, t_ms);
    ++R.k;
    R.last_resid = S.last_resid;
    R.corr = true;
    return WF_OK;
}

// one messenger iteration (Eqs. 3-4) and its sums, enqueued on the plan's
// stream; the chi^2-bound schedule synchronises inside to find lambda
wf_status hp_launch(HpRun &R)
{
    wf_plan p = R.p;
    if (p->pol) return hp_launch_pol(R);
    Prof &pr = R.pr;
    const wf_options &o = R.o;
    const double tau = R.tau;
    wf_status st;
    if (R.corr_pending) {
        R.corr_pending = false;
        if ((st = hp_enter_correction(R)) != WF_OK) return st;
    }
    pr.iter_begin();
    R.chi2_bound = NAN;
    if (R.rigorous) {
        // x_k = Y a_k, then lambda_k from chi^2(lambda_k, x_k) = b (Sect. 2.2)
        R.L = R.lmax;
        pr.begin(WF_K_LEG_SYN);
        if ((st = hp_legendre_synthesis(p, p->ws.a, R.L)) != WF_OK) return st;
        pr.end();
        pr.begin(WF_K_RING_SYN);
        if ((st = hp_ring_synthesis(p, R.L, RS_SYN, 1.0, tau, nullptr)) != WF_OK) return st;
        pr.end();
        double u_new = 0.0;
        if (R.k == 0) {
            if ((st = bound_root(p, R.h_cur, R.bound, 1.0, true, &u_new, &R.chi2_bound, &pr)) != WF_OK) return st;
        } else if (R.u_cur > 0.0) {
            if ((st = bound_root(p, R.h_cur, R.bound, R.u_cur, false, &u_new, &R.chi2_bound, &pr)) != WF_OK) return st;
            if (u_new > 0.0 && (R.u_cur - u_new) <= o.stall_tol * u_new) {
                // converged at lambda > 1: raise b to chi2_min(lambda) + (lambda - 1) tau_h x^T S^-2 x
                R.bound = R.chi2_bound + u_new * p->omega * R.q_cur;
                ++R.bound_updates;
                if ((st = bound_root(p, R.h_cur, R.bound, R.u_cur, false, &u_new, &R.chi2_bound, &pr)) != WF_OK)
                    return st;
            }
        }
        if (u_new / tau < 1e-9) u_new = 0.0;
        if (u_new == 0.0) {
            // lambda = 1 (reached or floored): report chi^2(1, x_k)
            double A, D;
            if ((st = pix_sums(p, 0.0, &A, &D, &pr)) != WF_OK) return st;
            R.chi2_bound = R.h_cur + A;
        }
        R.u_cur = u_new;
        R.lam = 1.0 + R.u_cur / tau;
        const double lam = R.lam;
        if (p->prec == WF_PREC_FP64)
            k_blend<double><<<grid_for(p->npix, p->nsm), 256, 0, p->stream>>>(
                p->npix, (const double *)p->ws.r, (const double *)p->ws.nu, (double *)p->ws.t, lam * tau,
                (lam - 1.0) * tau);
        else
            k_blend<float><<<grid_for(p->npix, p->nsm), 256, 0, p->stream>>>(
                p->npix, (const float *)p->ws.r, (const float *)p->ws.nu, (float *)p->ws.t, (float)(lam * tau),
                (float)((lam - 1.0) * tau));
        WF_COUNT_LAUNCH(p);
        WF_CUDA(cudaGetLastError());
    } else {
        pr.begin(WF_K_LEG_SYN);
        if ((st = hp_legendre_synthesis(p, p->ws.a, R.L)) != WF_OK) return st;
        pr.end();
        // one ring kernel: fold, inverse DFT, Eq. 3 and the forward DFT of t, which never
        // leaves shared memory (its time is reported under the ring synthesis)
        pr.begin(WF_K_RING_SYN);
        void *r_src = p->ws.r;
        if (R.corr) p->ws.r = p->ws.r0;  // correction form: B delta, the iteration without its source
        st = hp_ring_synthesis_analysis(p, R.L, R.lam, tau);
        p->ws.r = r_src;
        if (st != WF_OK) return st;
        pr.end();
    }
    const int L = R.L;
    const bool full = (R.lam == 1.0 && L == R.lmax);
    if (R.rigorous) {
        pr.begin(WF_K_RING_ANA);
        if ((st = hp_ring_analysis(p, L, p->ws.t)) != WF_OK) return st;
        pr.end();
    }
    BlendArgs ba;
    ba.lam_tauh = R.lam * R.tau_h;
    ba.tauh = R.tau_h;
    ba.S = R.C_ell;
    ba.want_resid = full ? 1 : 0;
    const double2 *a_old = p->ws.a;
    if (R.corr) {
        // the epilogue's residual compares its output B delta_k with delta_k - d0, i.e.
        // delta_{k+1} = d0 + B delta_k with delta_k; d0 is added to the output below
        if ((st = alm_axpy(p, p->ws.a, p->ws.cd0, -1.0, p->ws.caold)) != WF_OK) return st;
        a_old = p->ws.caold;
    }
    pr.begin(WF_K_LEG_ANA);
    if ((st = hp_legendre_analysis(p, L, LEG_BLEND, ba, a_old, p->ws.a_new)) != WF_OK) return st;
    pr.end();
    if (R.corr && (st = alm_axpy(p, p->ws.a_new, p->ws.cd0, 1.0, p->ws.a_new)) != WF_OK) return st;
    SumSpec sp{};
    sp.in[0] = p->ws.part_pix;
    sp.n[0] = p->npairs;
    sp.stride[0] = 1;
    for (int q = 0; q < 4; ++q) {
        sp.in[1 + q] = p->ws.part_harm + q;
        sp.n[1 + q] = L + 1;
        sp.stride[1 + q] = 4;
    }
    if ((st = sums_enqueue(p, sp, 5)) != WF_OK) return st;
    if (R.copy_back)
        WF_CUDA(cudaMemcpyAsync(p->ws.a, p->ws.a_new, p->nalm * sizeof(double2), cudaMemcpyDeviceToDevice, p->stream));
    return WF_OK;
}

// after the iteration's sums reached the host: trace, residual, schedule;
// false when the loop is over
bool hp_absorb(HpRun &R)
{
    wf_plan p = R.p;
    const double ims = R.pr.iter_end();
    R.pr.collect();
    const bool full = (R.lam == 1.0 && R.L == R.lmax);
    // (in correction form the kernels see delta, not the iterate: no chi^2)
    const double chi2 = R.corr ? NAN : R.rigorous ? R.chi2_bound : p->ws.h_scal[0] + p->ws.h_scal[1];
    const double resid = full ? std::sqrt(p->ws.h_scal[2]) / R.bnorm : NAN;
    R.h_cur = p->ws.h_scal[3];  // x_{k+1}^T S^-1 x_{k+1} and x^T S^-2 x for the next lambda
    R.q_cur = p->ws.h_scal[4];
    record(R.info, R.k, R.lam, R.L, chi2, resid, ims);
    if (!R.copy_back) {
        if (p->pol) std::swap(p->pol->a, p->pol->a_new);
        else std::swap(p->ws.a, p->ws.a_new);
    }
    ++R.k;
    if (full) {
        R.last_resid = resid;
        if (!std::isfinite(resid) || (R.k > 50 && resid > 1e3 * R.best_resid)) {
            R.result = WF_EDIVERGE;
            return false;
        }
        R.best_resid = std::min(R.best_resid, resid);
    }
    if (!R.corr && !std::isfinite(chi2)) {
        R.result = WF_EDIVERGE;
        R.chi2_bad = true;
        return false;
    }
    if (R.rigorous) {
        if (full && resid < R.tol_stop) {
            R.converged = true;
            return false;
        }
        return true;
    }
    if (R.replay) {
        if (full && resid < R.tol_stop) {
            R.converged = true;
            if (R.a_init) return false;  // correction sweeps stop at the tolerance
        }
        return true;
    }
    HpSchedule &sch = R.sch;
    if (sch.final_level()) {
        if (resid < R.tol_stop) {
            R.converged = true;
            return false;
        }
        if (full && !R.corr && R.o.mixed_correction > 0.0 && p->prec != WF_PREC_FP64 && !p->pol && !R.copy_back &&
            resid < R.tol * R.o.mixed_correction)
            R.corr_pending = true;
    } else {
        ++R.level_iters;
        const bool plateau = R.have_prev && std::fabs(chi2 - R.prev_chi2) < R.o.eta * R.sigma;
        if (plateau || R.level_iters >= R.o.level_cap) {
            sch.advance();
            ++R.levels;
            R.have_prev = false;
            R.level_iters = 0;
            return true;
        }
    }
    R.prev_chi2 = chi2;
    R.have_prev = true;
    return true;
}

wf_status hp_solve(wf_plan p, const double *d, const double *nv, const uint8_t *mask, const double *C_ell, double tol,
                   bool fluct, const double *g1, const double *g2, double *s_out, double *alm_out, wf_info *info,
                   const double2 *a_init = nullptr);

// refinement sweeps (mixed precision), output map, chi^2 of the result, report
wf_status hp_end(HpRun &R)
{
    wf_plan p = R.p;
    if (p->pol) return hp_end_pol(R);
    const wf_options &o = R.o;
    const int lmax = R.lmax;
    Prof &pr = R.pr;
    wf_status st;
    if (R.corr) {
        // correction form: a = x0 + delta
        if ((st = alm_axpy(p, p->ws.cx0, p->ws.a, 1.0, p->ws.a)) != WF_OK) return st;
        R.corr = false;
    }
    // Mixed precision, row a9: FP64 correction sweeps.  Up to refine_sweeps
    // messenger iterations at lambda = 1 on the full band run in FP64 from the
    // mixed-precision iterate (an FP64 sub-plan of the same geometry); their
    // residual is the FP64 operator's, and the output map is synthesised in FP64.
    if (p->prec != WF_PREC_FP64 && o.refine_sweeps > 0 && R.result != WF_EDIVERGE) {
        if (!p->sub) {
            wf_plan sub = nullptr;
            if ((st = wf_plan_create(&p->g, lmax, WF_PREC_FP64, (void *)p->stream, &sub)) != WF_OK) return st;
            p->sub = sub;
        }
        wf_plan sub = p->sub;
        // its Legendre transforms run in double-float on the FP32 pipe (48-bit significands;
        // FP64 runs at 1/64 of the FP32 rate on this GPU) unless fp64_emulation < 0
        sub->df_legendre = o.fp64_emulation >= 0;
        sub->stream = p->stream;
        sub->opt = p->opt;
        sub->opt.profile = o.profile;
        sub->opt.refine_sweeps = 0;
        sub->opt.schedule = 0;
        sub->replay_lambda.assign(o.refine_sweeps, 1.0);
        sub->replay_L.assign(o.refine_sweeps, lmax);
        wf_info si{};
        std::vector<double> tl(o.refine_sweeps), tc(o.refine_sweeps), tr(o.refine_sweeps), tm(o.refine_sweeps);
        std::vector<int> tL(o.refine_sweeps);
        si.lambda_trace = tl.data();
        si.L_trace = tL.data();
        si.chi2_trace = tc.data();
        si.resid_trace = tr.data();
        si.iter_ms_trace = tm.data();
        si.trace_cap = o.refine_sweeps;
        sub->bnorm_given = R.bnorm;
        st = hp_solve(sub, R.d, R.nv, R.mask, R.C_ell, R.tol, R.fluct, R.g1, R.g2, R.s_out, R.alm_out, &si, p->ws.a);
        sub->bnorm_given = 0;
        if (st != WF_OK) return st;
        for (int i = 0; i < si.iters; ++i) record(R.info, R.k + i, tl[i], tL[i], tc[i], tr[i], tm[i]);
        for (int f = 0; f < WF_NK; ++f) {
            pr.ms[f] += si.kernel_ms[f];
            pr.cnt[f] += si.kernel_launches[f];
        }
        pr.launches += si.launches;
        pr.finish();
        if (R.info) {
            wf_info *info = R.info;
            info->iters = R.k + si.iters;
            info->converged = si.converged ? 1 : 0;  // the FP64 operator's verdict
            info->final_residual = si.final_residual;
            info->chi2_over_ndof = si.chi2_over_ndof;
            info->n_dof = R.ndof;
            info->tau = R.tau;
            info->n_levels = R.rigorous ? 1 + R.bound_updates : R.levels;
            info->refine_sweeps = si.iters;
            info->mixed_lc = R.lc;
        }
        if (si.converged) return WF_OK;
        set_error(WF_ENOCONV, "not converged after %d FP64 sweeps (residual %.3e)", si.iters, si.final_residual);
        return R.replay ? WF_OK : WF_ENOCONV;
    }
    if ((st = hp_alm2map(p, p->ws.a, lmax, R.s_out)) != WF_OK) return st;
    if (R.alm_out)
        WF_CUDA(cudaMemcpyAsync(R.alm_out, p->ws.a, p->nalm * sizeof(double2), cudaMemcpyDeviceToDevice, p->stream));
    double chi2n = NAN;
    if (!R.fluct) {
        k_alm_norm<<<lmax + 1, 256, 0, p->stream>>>(lmax, R.C_ell, p->ws.a, 1, p->ws.part_harm);
        WF_COUNT_LAUNCH(p);
        const int gb = 256;
        k_pix_chi2<<<gb, 256, 0, p->stream>>>(p->npix, R.d, R.nv, R.mask, R.s_out, p->ws.part_pix);
        WF_COUNT_LAUNCH(p);
        WF_CUDA(cudaGetLastError());
        SumSpec sp{};
        sp.in[0] = p->ws.part_harm;
        sp.n[0] = lmax + 1;
        sp.stride[0] = 1;
        sp.in[1] = p->ws.part_pix;
        sp.n[1] = gb;
        sp.stride[1] = 1;
        if ((st = sums(p, sp, 2, &pr)) != WF_OK) return st;
        chi2n = (p->ws.h_scal[0] + p->ws.h_scal[1]) / (double)R.ndof;
    } else {
        WF_CUDA(cudaStreamSynchronize(p->stream));
    }
    if (R.info) {
        wf_info *info = R.info;
        info->iters = R.k;
        info->converged = R.converged ? 1 : 0;
        info->final_residual = R.last_resid;
        info->chi2_over_ndof = chi2n;
        info->n_dof = R.ndof;
        info->tau = R.tau;
        info->n_levels = R.rigorous ? 1 + R.bound_updates : R.levels;
        info->refine_sweeps = 0;
        info->mixed_lc = R.lc;
    }
    pr.finish();
    wf_status result = R.result;
    if (wf_status te = tc_check(p)) return te;
    if (result == WF_OK && !R.replay && !R.converged) result = WF_ENOCONV;
    if (result == WF_ENOCONV) set_error(result, "iteration cap reached (residual %.3e)", R.last_resid);
    if (result == WF_EDIVERGE && R.chi2_bad) set_error(result, "chi^2 is not finite at iteration %d", R.k);
    else if (result == WF_EDIVERGE)
        set_error(result, "residual grew (%.3e); lmax too large for this nside?", R.last_resid);
    return result;
}

wf_status hp_solve(wf_plan p, const double *d, const double *nv, const uint8_t *mask, const double *C_ell, double tol,
                   bool fluct, const double *g1, const double *g2, double *s_out, double *alm_out, wf_info *info,
                   const double2 *a_init)
{
    HpRun R;
    R.p = p;
    R.d = d;
    R.nv = nv;
    R.mask = mask;
    R.C_ell = C_ell;
    R.tol = tol;
    R.fluct = fluct;
    R.g1 = g1;
    R.g2 = g2;
    R.s_out = s_out;
    R.alm_out = alm_out;
    R.info = info;
    R.a_init = a_init;
    wf_status st = hp_begin(R);
    if (st != WF_OK) return st;
    while (hp_pick(R)) {
        if ((st = hp_launch(R)) != WF_OK) return st;
        WF_CUDA(cudaStreamSynchronize(p->stream));
        if (!hp_absorb(R)) break;
    }
    return hp_end(R);
}

// (T, E, B) -> (I, Q, U) maps: FP64 map out (omap, 3 x npix) or the plan's
// working maps (tmap) when omap is null; l <= L
wf_status pol_synthesis(wf_plan p, const double2 *a3, int L, double *omap, void *tmap)
{
    PolState *P = p->pol;
    const long long nalm = p->nalm, npix = p->npix;
    const RingSynMode mode = omap ? RS_MAP : RS_SYN;
    const size_t es = p->prec == WF_PREC_FP64 ? sizeof(double) : sizeof(float);
    auto tm = [&](int c) -> void * { return tmap ? (void *)((char *)tmap + (size_t)c * npix * es) : nullptr; };
    auto om = [&](int c) -> double * { return omap ? omap + (size_t)c * npix : nullptr; };
    wf_status st;
    if (p->prec == WF_PREC_FP64) {
        if ((st = hp_legendre_synthesis_buf(p, a3, L, (double2 *)p->ws.G)) != WF_OK) return st;
        if ((st = hp_ring_synthesis_buf(p, L, mode, 1.0, 0.0, p->ws.G, tm(0), om(0))) != WF_OK) return st;
        if ((st = hp_pol_legendre_synthesis(p, a3 + nalm, a3 + 2 * nalm, L)) != WF_OK) return st;
        if ((st = hp_ring_synthesis_buf(p, L, mode, 1.0, 0.0, P->GQ, tm(1), om(1))) != WF_OK) return st;
        return hp_ring_synthesis_buf(p, L, mode, 1.0, 0.0, P->GU, tm(2), om(2));
    }
    // mixed: T through the temperature kernels (with their FP64 block), E, B
    // through the FP32 spin-2 kernels, whose FP64 block the ring pass adds
    if ((st = hp_legendre_synthesis(p, a3, L)) != WF_OK) return st;
    if ((st = hp_ring_synthesis_buf(p, L, mode, 1.0, 0.0, p->ws.G, tm(0), om(0))) != WF_OK) return st;
    if ((st = hp_pol_legendre_synthesis_mx(p, a3 + nalm, a3 + 2 * nalm, L)) != WF_OK) return st;
    const bool low = P->lc > 0;
    if ((st = hp_ring_synthesis_buf_low(p, L, mode, 1.0, 0.0, P->GQ, low ? P->GQlow : nullptr, P->lc, P->low_cap,
                                        tm(1), om(1))) != WF_OK)
        return st;
    return hp_ring_synthesis_buf_low(p, L, mode, 1.0, 0.0, P->GU, low ? P->GUlow : nullptr, P->lc, P->low_cap,
                                     tm(2), om(2));
}

// adjoint: (I, Q, U) maps in the working precision (3 x npix) -> (T, E, B) = Y^T map, l <= L
wf_status pol_adjoint(wf_plan p, const void *map3, int L, double2 *out3)
{
    PolState *P = p->pol;
    const long long nalm = p->nalm, npix = p->npix;
    wf_status st;
    if (p->prec == WF_PREC_FP64) {
        const double *m = (const double *)map3;
        if ((st = hp_ring_analysis_buf(p, L, m, p->ws.F)) != WF_OK) return st;
        if ((st = hp_legendre_adjoint_buf(p, L, (const double2 *)p->ws.F, out3)) != WF_OK) return st;
        if ((st = hp_ring_analysis_buf(p, L, m + npix, P->FQ)) != WF_OK) return st;
        if ((st = hp_ring_analysis_buf(p, L, m + 2 * npix, P->FU)) != WF_OK) return st;
        return hp_pol_legendre_analysis(p, L, out3 + nalm, out3 + 2 * nalm);
    }
    const float *m = (const float *)map3;
    if ((st = hp_adjoint_T(p, m, L, out3)) != WF_OK) return st;
    if ((st = hp_ring_analysis_buf(p, L, m + npix, P->FQ)) != WF_OK) return st;
    if ((st = hp_ring_analysis_buf(p, L, m + 2 * npix, P->FU)) != WF_OK) return st;
    return hp_pol_legendre_analysis_mx(p, L, out3 + nalm, out3 + 2 * nalm);
}

// Y^T of FP64 maps (3 x npix): mixed plans round them into the working maps first
wf_status pol_adjoint_f64(wf_plan p, const double *map3, int L, double2 *out3)
{
    if (p->prec == WF_PREC_FP64) return pol_adjoint(p, map3, L, out3);
    const long long n = 3 * p->npix;
    k_map_to_T<float><<<grid_for(n, p->nsm), 256, 0, p->stream>>>(n, map3, (float *)p->pol->t);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    return pol_adjoint(p, p->pol->t, L, out3);
}

// Polarised Wiener filter (Eqs. 10-11), FP64, with the heuristic cooling of
// Sect. 3 on the largest eigenvalue of each l's prior block (or a replay).
// d: 3 x npix (I, Q, U); N6: 6 x npix noise covariance (II, QQ, UU, IQ, IU, QU);
// C4: 4 x (lmax + 1) spectra (TT, EE, BB, TE); s_out 3 x npix; alm_out 3 x n_alm.
// R.fluct: the fluctuation solve of Eq. (9) instead, source r = nu^1/2 g1 +
// Omega Y (S^+1/2 g2) from g1 (3 x npix) and g2 (3 x n_alm), d unused.
// The phases mirror the temperature ones (hp_begin / hp_launch / hp_end), so
// the batched solver runs polarised items too.
wf_status hp_begin_pol(HpRun &R)
{
    wf_plan p = R.p;
    const wf_options &o = R.o;
    if (o.schedule == 1 && p->replay_lambda.empty())
        return set_error(WF_EUNSUPPORTED, "the chi^2-bound schedule is built for temperature maps only");
    PolState *P = p->pol;
    const int lmax = R.lmax;
    const long long nalm = p->nalm;
    R.pr.init(p, R.info, o.profile != 0 && !R.graph);
    wf_status st;
    std::vector<double> C((size_t)4 * (lmax + 1));
    if ((st = to_host(p, C.data(), R.C_ell, C.size() * sizeof(double))) != WF_OK) return st;
    HpSchedule &sch = R.sch;
    sch.c.resize(lmax + 1);
    for (int l = 0; l <= lmax; ++l) {
        const double tt = C[l], ee = C[lmax + 1 + l], bb = C[2 * (lmax + 1) + l], te = C[3 * (lmax + 1) + l];
        // a TE correlation must be below 1 in magnitude (the pseudo-inverse of a
        // singular TE block with TE != 0 is left undefined)
        if (!(std::isfinite(tt) && std::isfinite(ee) && std::isfinite(bb) && std::isfinite(te)) || tt < 0 ||
            ee < 0 || bb < 0 || (te != 0.0 && !(te * te < tt * ee)))
            return set_error(WF_EINVAL, "prior block of l = %d is not positive semi-definite with |TE| < "
                                        "sqrt(TT EE)", l);
        const double h = 0.5 * (tt - ee);
        sch.c[l] = std::max(0.5 * (tt + ee) + std::sqrt(h * h + te * te), bb);
    }
    if ((st = hp_pol_setup(p, R.fluct ? nullptr : R.d, R.nv, R.mask, &R.tau, &R.ndof)) != WF_OK) return st;
    R.tau_h = R.tau * p->omega;
    // mixed precision: modes whose prior block's largest eigenvalue reaches
    // kappa tau_h take the FP64 blocks of both the temperature and the spin-2
    // kernels (the same reading as for temperature plans)
    R.lc = 0;
    if (p->prec != WF_PREC_FP64) {
        if (o.mixed_lc > 0) R.lc = std::min(o.mixed_lc, lmax + 1);
        else if (o.mixed_lc == 0)
            for (int l = lmax; l >= 0; --l)
                if (sch.c[l] / R.tau_h >= o.mixed_kappa) { R.lc = l + 1; break; }
        if ((st = hp_set_low_block(p, R.lc)) != WF_OK) return st;
        if ((st = hp_pol_set_low_block(p, R.lc)) != WF_OK) return st;
    }
    if (R.fluct) {
        // z = Y (S^+1/2 g2) into the output maps as scratch, then r = nu^1/2 g1 + Omega z
        if ((st = hp_pol_isqrt_prior(p, R.C_ell, (const double2 *)R.g2, P->a_new)) != WF_OK) return st;
        if ((st = pol_synthesis(p, P->a_new, lmax, R.s_out, nullptr)) != WF_OK) return st;
        if ((st = hp_pol_fluct_source(p, R.g1, R.s_out)) != WF_OK) return st;
    }
    if ((st = hp_pol_round_pixels(p)) != WF_OK) return st;
    if ((st = pol_adjoint_f64(p, P->r, lmax, P->b)) != WF_OK) return st;
    if ((st = hp_pol_alm_norm(p, R.C_ell, P->b, 1)) != WF_OK) return st;
    {
        SumSpec sp{};
        sp.in[0] = P->part2;
        sp.n[0] = lmax + 1;
        sp.stride[0] = 1;
        if ((st = sums(p, sp, 1, &R.pr)) != WF_OK) return st;
    }
    R.bnorm = std::sqrt(p->ws.h_scal[0]);
    if (!(R.bnorm > 0)) return set_error(WF_EINVAL, "the source has no component on modes with S > 0");
    sch.tau_h = R.tau_h;
    sch.lmax = lmax;
    sch.step_max = o.ell_step_max;
    sch.margin = o.band_margin;
    sch.ell_iter = std::min(o.ell0, lmax);
    sch.level();
    if (R.a_init)
        WF_CUDA(cudaMemcpyAsync(P->a, R.a_init, 3 * nalm * sizeof(double2), cudaMemcpyDeviceToDevice, p->stream));
    else
        WF_CUDA(cudaMemsetAsync(P->a, 0, 3 * nalm * sizeof(double2), p->stream));
    WF_CUDA(cudaMemsetAsync(P->a_new, 0, 3 * nalm * sizeof(double2), p->stream));
    R.replay = !p->replay_lambda.empty();
    R.nrep = (int)p->replay_lambda.size();
    R.rigorous = false;
    R.sigma = std::sqrt(2.0 * (double)R.ndof);
    return WF_OK;
}

// one polarised messenger iteration (Eqs. 10-11) and its sums [chi^2 pixel
// term, chi^2 harmonic term, residual^2], enqueued on the plan's stream
wf_status hp_launch_pol(HpRun &R)
{
    wf_plan p = R.p;
    PolState *P = p->pol;
    Prof &pr = R.pr;
    const int L = R.L;
    const bool full = (R.lam == 1.0 && L == R.lmax);
    wf_status st;
    pr.iter_begin();
    R.chi2_bound = NAN;
    pr.begin(WF_K_LEG_SYN);
    if ((st = pol_synthesis(p, P->a, L, nullptr, P->t)) != WF_OK) return st;
    pr.end();
    int nb = 0;
    if ((st = hp_pol_blend(p, R.lam, R.tau, &nb)) != WF_OK) return st;
    pr.begin(WF_K_LEG_ANA);
    if ((st = pol_adjoint(p, P->t, L, P->b)) != WF_OK) return st;
    if ((st = hp_pol_hblend(p, L, R.C_ell, R.lam * R.tau_h, R.tau_h, full ? 1 : 0)) != WF_OK) return st;
    pr.end();
    SumSpec sp{};
    sp.in[0] = P->part;
    sp.n[0] = nb;
    sp.stride[0] = 1;
    sp.in[1] = P->part2;
    sp.n[1] = R.lmax + 1;
    sp.stride[1] = 2;
    sp.in[2] = P->part2 + 1;
    sp.n[2] = R.lmax + 1;
    sp.stride[2] = 2;
    if ((st = sums_enqueue(p, sp, 3)) != WF_OK) return st;
    if (R.copy_back)
        WF_CUDA(cudaMemcpyAsync(P->a, P->a_new, 3 * p->nalm * sizeof(double2), cudaMemcpyDeviceToDevice, p->stream));
    return WF_OK;
}

wf_status hp_solve_pol(wf_plan p, const double *d, const double *N6, const uint8_t *mask, const double *C4,
                       double tol, bool fluct, const double *g1, const double2 *g2, double *s_out, double *alm_out,
                       wf_info *info, const double2 *a_init = nullptr);

// FP64 correction sweeps of a mixed polarised solve (as for temperature plans:
// lambda = 1 iterations on an FP64 sub-plan from the mixed iterate, whose
// residual is the FP64 operator's), output maps, chi^2 of the result, report
wf_status hp_end_pol(HpRun &R)
{
    wf_plan p = R.p;
    PolState *P = p->pol;
    const int lmax = R.lmax;
    const wf_options &o = R.o;
    wf_status st;
    if (p->prec != WF_PREC_FP64 && o.refine_sweeps > 0 && R.result != WF_EDIVERGE) {
        if (!p->sub) {
            wf_plan sub = nullptr;
            if ((st = wf_plan_create(&p->g, lmax, WF_PREC_FP64, (void *)p->stream, &sub)) != WF_OK) return st;
            p->sub = sub;
        }
        wf_plan sub = p->sub;
        sub->stream = p->stream;
        sub->opt = p->opt;
        sub->opt.profile = o.profile;
        sub->opt.refine_sweeps = 0;
        sub->opt.schedule = 0;
        sub->replay_lambda.assign(o.refine_sweeps, 1.0);
        sub->replay_L.assign(o.refine_sweeps, lmax);
        wf_info si{};
        std::vector<double> tl(o.refine_sweeps), tc(o.refine_sweeps), tr(o.refine_sweeps), tm(o.refine_sweeps);
        std::vector<int> tL(o.refine_sweeps);
        si.lambda_trace = tl.data();
        si.L_trace = tL.data();
        si.chi2_trace = tc.data();
        si.resid_trace = tr.data();
        si.iter_ms_trace = tm.data();
        si.trace_cap = o.refine_sweeps;
        st = hp_solve_pol(sub, R.d, R.nv, R.mask, R.C_ell, R.tol, R.fluct, R.g1, (const double2 *)R.g2, R.s_out,
                          R.alm_out, &si, P->a);
        if (st != WF_OK) return st;
        for (int i = 0; i < si.iters; ++i) record(R.info, R.k + i, tl[i], tL[i], tc[i], tr[i], tm[i]);
        for (int f = 0; f < WF_NK; ++f) {
            R.pr.ms[f] += si.kernel_ms[f];
            R.pr.cnt[f] += si.kernel_launches[f];
        }
        R.pr.launches += si.launches;
        R.pr.finish();
        if (R.info) {
            wf_info *info = R.info;
            info->iters = R.k + si.iters;
            info->converged = si.converged ? 1 : 0;  // the FP64 operator's verdict
            info->final_residual = si.final_residual;
            info->chi2_over_ndof = si.chi2_over_ndof;
            info->n_dof = R.ndof;
            info->tau = R.tau;
            info->n_levels = R.levels;
            info->refine_sweeps = si.iters;
            info->mixed_lc = R.lc;
        }
        if ((st = tc_check(p)) != WF_OK) return st;
        if (si.converged) return WF_OK;
        set_error(WF_ENOCONV, "not converged after %d FP64 sweeps (residual %.3e)", si.iters, si.final_residual);
        return R.replay ? WF_OK : WF_ENOCONV;
    }
    if ((st = pol_synthesis(p, P->a, lmax, R.s_out, nullptr)) != WF_OK) return st;
    if (R.alm_out)
        WF_CUDA(cudaMemcpyAsync(R.alm_out, P->a, 3 * p->nalm * sizeof(double2), cudaMemcpyDeviceToDevice,
                                p->stream));
    double chi2n = NAN;  // chi^2 of the result needs data: not defined for the fluctuation solve
    if (!R.fluct) {
        int nb = 0;
        if ((st = hp_pol_alm_norm(p, R.C_ell, P->a, 0)) != WF_OK) return st;
        if ((st = hp_pol_pix_chi2(p, R.d, R.s_out, &nb)) != WF_OK) return st;
        SumSpec sp{};
        sp.in[0] = P->part2;
        sp.n[0] = lmax + 1;
        sp.stride[0] = 1;
        sp.in[1] = P->part;
        sp.n[1] = nb;
        sp.stride[1] = 1;
        if ((st = sums(p, sp, 2, &R.pr)) != WF_OK) return st;
        chi2n = (p->ws.h_scal[0] + p->ws.h_scal[1]) / (double)R.ndof;
    } else {
        WF_CUDA(cudaStreamSynchronize(p->stream));
    }
    if (R.info) {
        wf_info *info = R.info;
        info->iters = R.k;
        info->converged = R.converged ? 1 : 0;
        info->final_residual = R.last_resid;
        info->chi2_over_ndof = chi2n;
        info->n_dof = R.ndof;
        info->tau = R.tau;
        info->n_levels = R.levels;
        info->refine_sweeps = 0;
        info->mixed_lc = R.lc;
    }
    R.pr.finish();
    if ((st = tc_check(p)) != WF_OK) return st;
    wf_status result = R.result;
    if (result == WF_OK && !R.replay && !R.converged) result = WF_ENOCONV;
    if (result == WF_ENOCONV) set_error(result, "iteration cap reached (residual %.3e)", R.last_resid);
    if (result == WF_EDIVERGE && R.chi2_bad) set_error(result, "chi^2 is not finite at iteration %d", R.k);
    else if (result == WF_EDIVERGE) set_error(result, "residual grew (%.3e)", R.last_resid);
    return result;
}

wf_status hp_solve_pol(wf_plan p, const double *d, const double *N6, const uint8_t *mask, const double *C4,
                       double tol, bool fluct, const double *g1, const double2 *g2, double *s_out, double *alm_out,
                       wf_info *info, const double2 *a_init)
{
    HpRun R;
    R.a_init = a_init;
    R.p = p;
    R.d = d;
    R.nv = N6;
    R.mask = mask;
    R.C_ell = C4;
    R.tol = tol;
    R.fluct = fluct;
    R.g1 = g1;
    R.g2 = (const double *)g2;
    R.s_out = s_out;
    R.alm_out = alm_out;
    R.info = info;
    wf_status st = hp_begin(R);
    if (st != WF_OK) return st;
    while (hp_pick(R)) {
        if ((st = hp_launch(R)) != WF_OK) return st;
        WF_CUDA(cudaStreamSynchronize(p->stream));
        if (!hp_absorb(R)) break;
    }
    return hp_end(R);
}

// Several HEALPix solves advanced together: one step of every active solve
// (its iteration's kernels on its own branch stream) is captured in one CUDA
// graph and launched at once; the host then reads every solve's sums and runs
// its schedule.  The graph is replayed while every solve keeps its (lambda,
// L), and updated in place (or re-instantiated) when one changes or a solve
// leaves the batch.  The iterate is copied a <- a_new inside the step, so the
// captured pointers stay valid from one step to the next.
wf_status hp_solve_batch(int n, wf_plan *plans, const wf_batch_item *items, cudaStream_t user,
                         wf_status *statuses)
{
    for (int i = 0; i < n; ++i) {
        if (!plans[i] || plans[i]->g.kind != WF_GEOM_HEALPIX)
            return set_error(WF_EINVAL, "batch item %d: needs a HEALPix plan", i);
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return set_error(WF_EINVAL, "batch items %d and %d share a plan", j, i);
        const wf_batch_item &it = items[i];
        if (it.kind != WF_REQ_WF && it.kind != WF_REQ_FLUCT)
            return set_error(WF_EINVAL, "batch item %d: kind must be WF_REQ_WF or WF_REQ_FLUCT", i);
        if (!it.noise_var || !it.C_ell || !it.s_out || (it.kind == WF_REQ_WF && !it.d) ||
            (it.kind == WF_REQ_FLUCT && (!it.g1 || !it.g2)) || !(it.tol > 0))
            return set_error(WF_EINVAL, "batch item %d: missing buffer or bad tol", i);
        if (defaults(plans[i]->opt).schedule == 1 && plans[i]->replay_lambda.empty())
            return set_error(WF_EUNSUPPORTED, "batch item %d: the chi^2-bound schedule synchronises inside an "
                                              "iteration and cannot be batched", i);
    }
    auto ck = [](cudaError_t e, const char *what) { return e == cudaSuccess ? WF_OK : cuda_check(e, what); };
    std::vector<cudaStream_t> saved(n), branch(n, nullptr);
    std::vector<cudaEvent_t> join(n, nullptr);
    cudaEvent_t fork = nullptr;
    cudaStream_t origin = nullptr;  // capture stream (the caller's may be the legacy one, which cannot be captured)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<HpRun> R(n);
    std::vector<char> active(n, 0);
    std::vector<std::array<long long, WF_NK>> per_step(n);
    wf_status st = WF_OK;
    auto bind = [](wf_plan p, cudaStream_t s) {
        for (; p; p = p->sub) p->stream = s;
    };
    auto cleanup = [&]() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (int i = 0; i < n; ++i) {
            if (branch[i]) {
                cudaStreamSynchronize(branch[i]);
                bind(plans[i], saved[i]);
                cudaStreamDestroy(branch[i]);
            }
            if (join[i]) cudaEventDestroy(join[i]);
        }
        if (fork) cudaEventDestroy(fork);
        if (origin) {
            cudaStreamSynchronize(origin);
            cudaStreamDestroy(origin);
        }
    };
    // work queued on the plans' own streams finishes before their branch streams take over
    for (int i = 0; i < n; ++i) {
        saved[i] = plans[i]->stream;
        if (saved[i]) WF_CUDA(cudaStreamSynchronize(saved[i]));
    }
    WF_CUDA(cudaStreamSynchronize(user));
    if (cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess) {
        cleanup();
        return set_error(WF_ECUDA, "cudaEventCreate failed");
    }
    for (int i = 0; i < n; ++i) {
        if (cudaStreamCreateWithFlags(&branch[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming) != cudaSuccess) {
            cleanup();
            return set_error(WF_ECUDA, "batch stream or event creation failed");
        }
        bind(plans[i], branch[i]);
    }
    for (int i = 0; i < n; ++i) {
        const wf_batch_item &it = items[i];
        HpRun &r = R[i];
        r.p = plans[i];
        r.fluct = it.kind == WF_REQ_FLUCT;
        r.d = it.d;
        r.nv = it.noise_var;
        r.mask = it.mask;
        r.C_ell = it.C_ell;
        r.g1 = it.g1;
        r.g2 = it.g2;
        r.tol = it.tol;
        r.s_out = it.s_out;
        r.alm_out = it.alm_out;
        r.info = it.info;
        r.copy_back = true;
        r.graph = true;
        r.a_init = plans[i]->start;
        statuses[i] = hp_begin(r);
        active[i] = statuses[i] == WF_OK;
    }
    // tensor-core items of one geometry and FP64 block share one synthesis launch per step
    std::vector<cudaEvent_t> gev(n, nullptr);
    for (int i = 0; i < n; ++i)
        if (cudaEventCreateWithFlags(&gev[i], cudaEventDisableTiming) != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaEventDestroy(gev[j]);
            cleanup();
            return set_error(WF_ECUDA, "batch event creation failed");
        }
    std::vector<int> group_of(n, -1);
    std::vector<std::array<long long, WF_NK>> group_cnt(n);
    std::vector<std::pair<int, std::pair<double, int>>> cfg, cur;
    for (;;) {
        cfg.clear();
        for (int i = 0; i < n; ++i)
            if (active[i]) {
                if (!hp_pick(R[i])) active[i] = 0;
                else cfg.push_back({i, {R[i].lam, R[i].L}});
            }
        if (cfg.empty()) break;
        if (!exec || cfg != cur) {
            cudaGraph_t ng = nullptr;
            if ((st = ck(cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal), "capture"))) break;
            cudaEventRecord(fork, origin);
            // groups: (nside, lmax, FP64 block) of the tensor-core items, at most TC_MAX_COLUMNS each
            std::fill(group_of.begin(), group_of.end(), -1);
            for (auto &gc : group_cnt) gc.fill(0);
            int ngroups = 0;
            for (size_t u = 0; u < cfg.size() && st == WF_OK; ++u) {
                const int i0 = cfg[u].first;
                wf_plan p0 = plans[i0];
                if (!tc_prec(p0->prec) || R[i0].rigorous || group_of[i0] >= 0) continue;
                // polarised items group with polarised items of the same spin-2 FP64 block; their
                // T columns (the temperature kernel) and E, B columns (the spin-2 kernel) share a launch each
                const bool pol = p0->pol != nullptr;
                const int cap = pol ? std::min(TC_MAX_COLUMNS, TCP_MAX_COLUMNS) : TC_MAX_COLUMNS;
                std::vector<int> mem{i0};
                for (size_t v = u + 1; v < cfg.size() && (int)mem.size() < cap; ++v) {
                    const int j = cfg[v].first;
                    wf_plan pj = plans[j];
                    if (group_of[j] < 0 && pj->prec == p0->prec && !R[j].rigorous &&
                        pj->nside == p0->nside && pj->lmax == p0->lmax && pj->tab.lc_mx == p0->tab.lc_mx &&
                        (pj->pol != nullptr) == pol && (!pol || pj->pol->lc == p0->pol->lc))
                        mem.push_back(j);
                }
                std::vector<const double2 *> ga, gE, gB;
                std::vector<float2 *> gG, gca, gQ, gU;
                std::vector<float4 *> gac;
                std::vector<int> gL;
                int Lmax = 0;
                for (int j : mem) {
                    group_of[j] = ngroups;
                    wf_plan pj = plans[j];
                    const double2 *a = pol ? pj->pol->a : pj->ws.a;
                    ga.push_back(a);
                    gca.push_back(pj->ws.ca32);
                    gG.push_back((float2 *)pj->ws.G);
                    if (pol) {
                        gE.push_back(a + pj->nalm);
                        gB.push_back(a + 2 * pj->nalm);
                        gac.push_back(pj->pol->ac32);
                        gQ.push_back((float2 *)pj->pol->GQ);
                        gU.push_back((float2 *)pj->pol->GU);
                    }
                    gL.push_back(R[j].L);
                    Lmax = std::max(Lmax, R[j].L);
                }
                long long k0[WF_NK];
                for (int f = 0; f < WF_NK; ++f) k0[f] = p0->kcnt[f];
                const int fam = p0->kfam;
                p0->kfam = WF_K_LEG_SYN;
                st = hp_tc_synthesis(p0, (int)mem.size(), ga.data(), gca.data(), gG.data(), gL.data(), Lmax, origin);
                if (st == WF_OK && pol)
                    st = hp_pol_tc_synthesis(p0, (int)mem.size(), gE.data(), gB.data(), gac.data(), gQ.data(),
                                             gU.data(), gL.data(), Lmax, origin);
                p0->kfam = fam;
                for (int f = 0; f < WF_NK; ++f) {
                    group_cnt[i0][f] = p0->kcnt[f] - k0[f];
                    p0->kcnt[f] = k0[f];
                }
                cudaEventRecord(gev[ngroups], origin);
                ++ngroups;
            }
            for (auto &c : cfg) {
                if (st != WF_OK) break;
                const int i = c.first;
                wf_plan p = plans[i];
                cudaStreamWaitEvent(branch[i], fork, 0);
                if (group_of[i] >= 0) {
                    cudaStreamWaitEvent(branch[i], gev[group_of[i]], 0);
                    p->tc_deferred = true;
                }
                long long k0[WF_NK];
                for (int f = 0; f < WF_NK; ++f) k0[f] = p->kcnt[f];
                st = hp_launch(R[i]);
                p->tc_deferred = false;
                for (int f = 0; f < WF_NK; ++f) {
                    per_step[i][f] = p->kcnt[f] - k0[f];
                    p->kcnt[f] = k0[f];  // counted when the graph runs
                    per_step[i][f] += group_cnt[i][f];  // the group launch, counted on its first item
                }
                if (st != WF_OK) break;
                cudaEventRecord(join[i], branch[i]);
                cudaStreamWaitEvent(origin, join[i], 0);
            }
            cudaError_t ce = cudaStreamEndCapture(origin, &ng);
            if (st == WF_OK) st = ck(ce, "cudaStreamEndCapture");
            if (st != WF_OK) {
                if (ng) cudaGraphDestroy(ng);
                break;
            }
            if (exec) {
                cudaGraphExecUpdateResultInfo ui;
                if (cudaGraphExecUpdate(exec, ng, &ui) != cudaSuccess) {
                    cudaGetLastError();
                    cudaGraphExecDestroy(exec);
                    exec = nullptr;
                }
            }
            if (!exec && (st = ck(cudaGraphInstantiate(&exec, ng, 0), "cudaGraphInstantiate")) != WF_OK) {
                cudaGraphDestroy(ng);
                break;
            }
            if (graph) cudaGraphDestroy(graph);
            graph = ng;
            cur = cfg;
        }
        if ((st = ck(cudaGraphLaunch(exec, origin), "cudaGraphLaunch")) != WF_OK) break;
        if ((st = ck(cudaStreamSynchronize(origin), "batch step")) != WF_OK) break;
        for (auto &c : cfg) {
            const int i = c.first;
            for (int f = 0; f < WF_NK; ++f) plans[i]->kcnt[f] += per_step[i][f];
            if (!hp_absorb(R[i])) active[i] = 0;
        }
    }
    if (st == WF_OK)
        for (int i = 0; i < n; ++i)
            if (statuses[i] == WF_OK) statuses[i] = hp_end(R[i]);
    cleanup();
    for (int i = 0; i < n; ++i) cudaEventDestroy(gev[i]);
    return st;
}

wf_status hp_create(wf_plan p)
{
    const int nside = p->nside;
    p->nrings = 4 * nside - 1;
    p->npairs = 2 * nside;
    p->npix = 12LL * nside * nside;
    p->nalm = (long long)(p->lmax + 1) * (p->lmax + 2) / 2;
    p->omega = 4.0 * M_PI / (double)p->npix;
    std::vector<double> xp(p->npairs), stp(p->npairs);
    for (int pr = 0; pr < p->npairs; ++pr) {
        const int i = pr + 1;  // 1-based north ring
        if (i < nside) {
            const double omz = (double)i * i / (3.0 * nside * nside);
            xp[pr] = 1.0 - omz;
            stp[pr] = std::sqrt(omz * (2.0 - omz));
        } else {
            const double z = 4.0 / 3.0 - 2.0 * i / (3.0 * nside);
            xp[pr] = z;
            stp[pr] = std::sqrt((1.0 - z) * (1.0 + z));
        }
    }
    if (p->prec != WF_PREC_FP64) {
        WF_CUDA(cudaStreamCreateWithFlags(&p->aux, cudaStreamNonBlocking));
        WF_CUDA(cudaEventCreateWithFlags(&p->fork_ev, cudaEventDisableTiming));
        WF_CUDA(cudaEventCreateWithFlags(&p->join_ev, cudaEventDisableTiming));
    }
    wf_status st;
    if ((st = hp_build_legendre_tables(p, xp, stp)) != WF_OK) return st;
    if ((st = hp_build_ring_tables(p)) != WF_OK) return st;
    const size_t es = p->prec == WF_PREC_FP64 ? sizeof(double) : sizeof(float);
    const size_t gsz = (size_t)p->npairs * (p->lmax + 1) * 2 * 2 * es;
    if ((st = plan_alloc(p, (void **)&p->ws.a, p->nalm * sizeof(double2))) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&p->ws.a_new, p->nalm * sizeof(double2))) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&p->ws.b, p->nalm * sizeof(double2))) != WF_OK) return st;
    if (p->prec != WF_PREC_FP64 &&
        (st = plan_alloc(p, (void **)&p->ws.b_low, p->nalm * sizeof(double2))) != WF_OK)
        return st;
    if ((st = plan_alloc(p, &p->ws.G, gsz)) != WF_OK) return st;
    if ((st = plan_alloc(p, &p->ws.F, gsz)) != WF_OK) return st;
    if ((st = plan_alloc(p, &p->ws.r, p->npix * es)) != WF_OK) return st;
    if ((st = plan_alloc(p, &p->ws.nu, p->npix * es)) != WF_OK) return st;
    if ((st = plan_alloc(p, &p->ws.t, p->npix * es)) != WF_OK) return st;
    // per ring pair; also the 2 x (<= 2 nsm) chi^2-bound sums
    const int npart = std::max(p->npairs, std::max(256, 4 * p->nsm));
    if ((st = plan_alloc(p, (void **)&p->ws.part_pix, npart * sizeof(double))) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&p->ws.part_harm, 4 * (p->lmax + 2) * sizeof(double))) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&p->ws.epi, (p->lmax + 1) * sizeof(double4))) != WF_OK) return st;
    return WF_OK;
}

}  // namespace

// Device bytes a HEALPix plan allocates (tables, workspace, host-API staging),
// mirroring hp_create and the table builders; the mixed path's FP64-block
// buffer is counted for l_c = (lmax + 1) / 8 (it grows with l_c on demand).
long long hp_estimate_bytes(int nside, int lmax, wf_precision prec, bool staging, int ncomp)
{
    const bool f32 = prec != WF_PREC_FP64;
    const long long np = 2LL * nside, npix = 12LL * nside * nside;
    const long long nalm = (long long)(lmax + 1) * (lmax + 2) / 2, ns = (long long)(lmax + 1) * np;
    const long long es = f32 ? 4 : 8, ec = 2 * es;
    long long b = 0;
    b += nalm * 16 + np * 16 + (lmax + 1) * 8 + ns * (4 + 16);  // A64, c64, x, st, log2 c, seeds
    if (f32) b += nalm * 8 + np * 8 + ns * 12;                   // A32, B32, x32, w32, FP32 seeds
    // ring tables: roots per distinct length, Bluestein filters, twiddles, scratch
    long long roots = 0, V = 0, nmaxF = 2, maxBlue = 1;
    for (int k = 1; k <= nside; ++k) {
        const long long n = 4LL * k;
        roots += 2 * n;
        if (n <= 32) continue;
        if ((n & (n - 1)) == 0) {
            nmaxF = std::max(nmaxF, n);
        } else {
            long long M = 1;
            while (M < 2 * n - 1) M <<= 1;
            V += M + n;  // filter and chirp
            nmaxF = std::max(nmaxF, M);
            maxBlue = std::max(maxBlue, n);
        }
    }
    const long long zl = std::max(maxBlue, 32LL);
    b += (roots + V + nmaxF) * ec + np * (48 + 4) + 64;
    b += std::min<long long>(np, 8LL * 152) * 2 * zl * ec;
    // workspace
    b += nalm * 16 * (f32 ? 4 : 3);                              // a, a_new, b (+ b_low)
    b += 2 * np * (lmax + 1) * 2 * ec;                           // G, F
    b += 3 * npix * es;                                          // r, nu, t
    b += std::max(np, 1024LL) * 8 + 4LL * (lmax + 2) * 8 + (lmax + 1) * 32 + 256;
    if (f32) b += np * ((lmax + 1) / 8 + 1) * 2 * 8;             // FP64-block coefficients (stored FP32)
    if (f32) b += std::min(hp_low_table_bytes(lmax, (int)np, (lmax + 1) / 8 + 1), 2LL << 30) + (lmax + 2) * 8;  // its table
    if (staging) b += npix * (3 * 8 + 1) + (lmax + 1) * 8 + nalm * 16 * 2 + npix * 8;
    if (tc_prec(prec)) b += nalm * 8;                            // c a_lm in FP32 (tensor-core synthesis)
    if (ncomp == 3) {  // polarisation (PolState)
        const long long lcap = (lmax + 1) / 8 + 1;                  // FP64-block allowance, as above
        if (tc_prec(prec)) b += nalm * 16;                           // spin-2 B operand source (FP32 x 4)
        b += nalm * 8 * 3 + ns * (4 + 32);                           // al, be, ga; ls and the four seeds
        b += 3 * 3 * nalm * 16;                                      // a, a_new, b for T, E, B
        b += 4 * np * (lmax + 1) * 2 * ec;                           // GQ, GU, FQ, FU
        b += 3 * npix * 8 + 3 * npix * es + 6 * npix * 8;            // r, t, nu
        b += 3 * (lmax + 1) * 32 + 2 * std::max(2LL * (lmax + 2), 8LL * 152) * 8;  // blend table, partials
        if (f32) {
            b += 9 * npix * 4;                                       // FP32 r, nu
            b += nalm * (8 + 16 + 2 * 16);                           // c, mu-form table, FP64-block (E, B)
            b += ns * (4 + 16);                                      // FP32 seeds
            b += 2 * np * lcap * 2 * 8;                              // FP64-block ring coefficients
        }
        if (staging) b += npix * 8 * (2 + 5 + 2 + 2) + 3 * (lmax + 1) * 8 + 4 * nalm * 16;  // 3-component buffers
    }
    return b + (1LL << 20);
}

}  // namespace wf

using namespace wf;

extern "C" {

const char *wf_strerror(wf_status s)
{
    switch (s) {
    case WF_OK: return "ok";
    case WF_EINVAL: return "invalid argument";
    case WF_ENOMEM: return "out of memory";
    case WF_ECUDA: return "CUDA error";
    case WF_ENOCONV: return "not converged";
    case WF_EDIVERGE: return "diverged";
    case WF_ETIMEOUT: return "device wait timed out";
    case WF_EUNSUPPORTED: return "unsupported configuration";
    }
    return "unknown status";
}

const char *wf_last_error(void) { return wf::g_err; }

long long wf_abi_sizeof(const char *name)
{
    if (!name) return 0;
    const struct {
        const char *name;
        size_t size;
    } sizes[] = {{"wf_geometry", sizeof(wf_geometry)},     {"wf_options", sizeof(wf_options)},
                 {"wf_info", sizeof(wf_info)},             {"wf_batch_item", sizeof(wf_batch_item)},
                 {"wf_request", sizeof(wf_request)},       {"wf_result", sizeof(wf_result)},
                 {"wf_server_stats", sizeof(wf_server_stats)}};
    for (const auto &e : sizes)
        if (std::strcmp(name, e.name) == 0) return (long long)e.size;
    return 0;
}

wf_status wf_plan_create(const wf_geometry *g, int lmax, wf_precision prec, void *cuda_stream, wf_plan *out)
{
    if (!g || !out) return set_error(WF_EINVAL, "null argument");
    *out = nullptr;
    if (g->ncomp != 0 && g->ncomp != 1 && g->ncomp != 3)
        return set_error(WF_EUNSUPPORTED, "ncomp must be 1 (temperature) or 3 (I, Q, U)");
    if (g->ncomp == 3 && g->kind != WF_GEOM_HEALPIX)
        return set_error(WF_EUNSUPPORTED, "polarised plans (ncomp = 3) are HEALPix");
    if (prec != WF_PREC_FP64 && prec != WF_PREC_MIXED_FP32 && prec != WF_PREC_MIXED_TF32 &&
        prec != WF_PREC_MIXED_SPLITBF16)
        return set_error(WF_EINVAL, "unknown precision");
    if (tc_prec(prec) && g->kind != WF_GEOM_HEALPIX)
        return set_error(WF_EUNSUPPORTED, "tensor-core plans are HEALPix plans");
    wf_plan p = new (std::nothrow) wf_plan_s();
    if (!p) return set_error(WF_ENOMEM, "host allocation");
    p->g = *g;
    p->prec = prec;
    p->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_check(e, "device query");
    }
    wf_status st = WF_OK;
    if (g->kind == WF_GEOM_HEALPIX) {
        if (g->nside < 1 || g->nside > 8192) st = set_error(WF_EINVAL, "nside out of range");
        else if (lmax < 2 || lmax > 2 * g->nside) st = set_error(WF_EINVAL, "need 2 <= lmax <= 2 nside (got %d)", lmax);
        else {
            p->nside = g->nside;
            p->lmax = lmax;
            st = hp_create(p);
            if (st == WF_OK && g->ncomp == 3) st = hp_pol_create(p, p->tab.x64, p->tab.st64);
        }
    } else if (g->kind == WF_GEOM_FLAT) {
        p->lmax = 0;
        st = flat_create(p);
    } else {
        st = set_error(WF_EINVAL, "unknown geometry");
    }
    if (st == WF_OK) {
        if ((st = plan_alloc(p, (void **)&p->ws.scal, 16 * sizeof(double))) == WF_OK &&
            (st = plan_alloc(p, (void **)&p->ws.flag, 16)) == WF_OK &&
            (st = plan_alloc(p, (void **)&p->ws.tc_err, 16)) == WF_OK &&
            (st = (cudaMemsetAsync(p->ws.tc_err, 0, 16, p->stream) == cudaSuccess
                       ? WF_OK
                       : set_error(WF_ECUDA, "cudaMemsetAsync"))) == WF_OK) {
            if (cudaMallocHost(&p->ws.h_scal, 16 * sizeof(double)) != cudaSuccess)
                st = set_error(WF_ENOMEM, "pinned host allocation");
        }
    }
    if (st != WF_OK) {
        wf_plan_destroy(p);
        return st;
    }
    *out = p;
    return WF_OK;
}

void wf_plan_destroy(wf_plan p)
{
    if (!p) return;
    if (p->stream) cudaStreamSynchronize(p->stream);
    else cudaDeviceSynchronize();
    if (p->aux) cudaStreamSynchronize(p->aux);
    if (p->flat) flat_destroy(p);
    if (p->pol) hp_pol_destroy(p);
    if (p->sub) wf_plan_destroy(p->sub);
    if (p->aux) cudaStreamDestroy(p->aux);
    if (p->fork_ev) cudaEventDestroy(p->fork_ev);
    if (p->join_ev) cudaEventDestroy(p->join_ev);
    if (p->events_ready)
        for (auto &e : p->ev) cudaEventDestroy(e);
    for (void *a : p->allocations) cudaFree(a);
    if (p->ws.h_scal) cudaFreeHost(p->ws.h_scal);
    delete p;
}

wf_status wf_set_options(wf_plan p, const wf_options *opt)
{
    if (!p) return set_error(WF_EINVAL, "null plan");
    if (opt && (opt->schedule < 0 || opt->schedule > 1))
        return set_error(WF_EINVAL, "schedule must be 0 (heuristic) or 1 (chi^2 bound)");
    if (opt && ((opt->tile_syn != 0 && opt->tile_syn != 2 && opt->tile_syn != 4 && opt->tile_syn != 8) ||
                (opt->tile_ana != 0 && opt->tile_ana != 2 && opt->tile_ana != 4 && opt->tile_ana != 8)))
        return set_error(WF_EINVAL, "tile_syn and tile_ana must be 2, 4 or 8 (0: keep)");
    const long long old_cap = p->opt.mixed_table_bytes;
    p->opt = opt ? *opt : wf_options{};
    if (p->opt.tile_syn > 0) p->tile_syn = p->opt.tile_syn;
    if (p->opt.tile_ana > 0) p->tile_ana = p->opt.tile_ana;
    if (p->g.kind == WF_GEOM_HEALPIX && p->prec == WF_PREC_FP64 && p->g.ncomp == 1)
        p->df_legendre = p->opt.fp64_emulation != 0;
    // mixed temperature tables: a forced block (or a changed table cap) takes effect now
    if (p->g.kind == WF_GEOM_HEALPIX && p->prec != WF_PREC_FP64) {
        if (p->opt.mixed_table_bytes != old_cap) p->tab.lc_mx = -1;
        if (p->opt.mixed_lc != 0 || p->tab.lc_mx < 0) {
            const int lc = p->opt.mixed_lc > 0 ? std::min(p->opt.mixed_lc, p->lmax + 1) : 0;
            if (wf_status st = hp_set_low_block(p, lc)) return st;
            if (p->pol)  // the spin-2 block as a polarised solve sets it
                if (wf_status st = hp_pol_set_low_block(p, lc)) return st;
            WF_CUDA(cudaStreamSynchronize(p->stream));
        }
    }
    return WF_OK;
}

wf_status wf_set_start(wf_plan p, const double *alm0)
{
    if (!p) return set_error(WF_EINVAL, "null plan");
    if (p->g.kind != WF_GEOM_HEALPIX && alm0) return set_error(WF_EUNSUPPORTED, "a starting iterate needs a HEALPix plan");
    p->start = (const double2 *)alm0;
    return WF_OK;
}

wf_status wf_set_schedule(wf_plan p, const double *lambda, const int *L, int n)
{
    if (!p || n < 0 || (n > 0 && !lambda)) return set_error(WF_EINVAL, "bad schedule");
    p->replay_lambda.assign(lambda, lambda + n);
    p->replay_L.assign(n, p->lmax);
    if (L) for (int i = 0; i < n; ++i) p->replay_L[i] = L[i];
    for (double v : p->replay_lambda)
        if (!(v >= 1.0)) return set_error(WF_EINVAL, "lambda must be >= 1");
    return WF_OK;
}

long long wf_npix(wf_plan p) { return p ? p->npix : 0; }
long long wf_nalm(wf_plan p) { return p ? p->nalm : 0; }
long long wf_plan_device_bytes(wf_plan p)
{
    if (!p) return 0;
    return p->device_bytes + (p->sub ? wf_plan_device_bytes(p->sub) : 0);
}

long long wf_plan_estimate_bytes(const wf_geometry *g, int lmax, wf_precision prec, int with_host_staging)
{
    if (!g) return -1;
    if (g->kind == WF_GEOM_FLAT) return 8LL << 20;  // n <= 128: a few hundred KB of maps and traces
    if (g->kind != WF_GEOM_HEALPIX || g->nside < 1 || lmax < 2 || lmax > 2 * g->nside) return -1;
    if (g->ncomp != 0 && g->ncomp != 1 && g->ncomp != 3) return -1;
    return wf::hp_estimate_bytes(g->nside, lmax, prec, with_host_staging != 0, g->ncomp == 3 ? 3 : 1);
}

wf_status wf_plan_autotune(wf_plan p, int reps)
{
    if (!p) return set_error(WF_EINVAL, "null plan");
    if (p->g.kind != WF_GEOM_HEALPIX) return WF_OK;
    wf_status st = hp_autotune(p, reps);
    if (st != WF_OK) return st;
    WF_CUDA(cudaStreamSynchronize(p->stream));
    return WF_OK;
}

wf_status wf_plan_tiles(wf_plan p, int *syn_pairs, int *ana_pairs)
{
    if (!p) return set_error(WF_EINVAL, "null plan");
    if (syn_pairs) *syn_pairs = p->tile_syn;
    if (ana_pairs) *ana_pairs = p->tile_ana;
    return WF_OK;
}

wf_status wf_plan_set_stream(wf_plan p, void *cuda_stream)
{
    if (!p) return set_error(WF_EINVAL, "null plan");
    if (p->stream != (cudaStream_t)cuda_stream) {
        // work queued on the old stream finishes before the new one is used
        if (p->stream) WF_CUDA(cudaStreamSynchronize(p->stream));
        else WF_CUDA(cudaDeviceSynchronize());
    }
    p->stream = (cudaStream_t)cuda_stream;
    if (p->sub) return wf_plan_set_stream(p->sub, cuda_stream);
    return WF_OK;
}

wf_status wf_solve(wf_plan p, const double *d, const double *noise_var, const uint8_t *mask, const double *C_ell,
                   double tol, double *s_wf, double *alm_out, wf_info *info)
{
    if (!p || !d || !noise_var || !C_ell || !s_wf) return set_error(WF_EINVAL, "null argument");
    if (!(tol > 0)) return set_error(WF_EINVAL, "tol must be > 0");
    if (p->g.kind == WF_GEOM_FLAT) {
        if (p->opt.schedule == 1 && p->replay_lambda.empty())
            return set_error(WF_EUNSUPPORTED, "the chi^2-bound schedule is implemented on the HEALPix sphere only");
        return flat_solve(p, d, noise_var, mask, C_ell, tol, false, nullptr, nullptr, s_wf, alm_out, info);
    }
    if (p->pol)
        return hp_solve_pol(p, d, noise_var, mask, C_ell, tol, false, nullptr, nullptr, s_wf, alm_out, info, p->start);
    return hp_solve(p, d, noise_var, mask, C_ell, tol, false, nullptr, nullptr, s_wf, alm_out, info, p->start);
}

wf_status wf_solve_batch(int n, wf_plan *plans, const wf_batch_item *items, void *cuda_stream, wf_status *statuses)
{
    if (n < 0 || (n > 0 && (!plans || !items || !statuses))) return set_error(WF_EINVAL, "null argument");
    if (n == 0) return WF_OK;
    for (int i = 0; i < n; ++i) statuses[i] = WF_EINVAL;
    return hp_solve_batch(n, plans, items, (cudaStream_t)cuda_stream, statuses);
}

wf_status wf_fluct(wf_plan p, const double *noise_var, const uint8_t *mask, const double *C_ell, const double *g1,
                   const double *g2, double tol, double *f_out, double *alm_out, wf_info *info)
{
    if (!p || !noise_var || !C_ell || !g1 || !g2 || !f_out) return set_error(WF_EINVAL, "null argument");
    if (!(tol > 0)) return set_error(WF_EINVAL, "tol must be > 0");
    if (p->g.kind == WF_GEOM_FLAT) {
        if (p->opt.schedule == 1 && p->replay_lambda.empty())
            return set_error(WF_EUNSUPPORTED, "the chi^2-bound schedule needs data (Wiener filter, not wf_fluct)");
        return flat_solve(p, nullptr, noise_var, mask, C_ell, tol, true, g1, g2, f_out, alm_out, info);
    }
    if (p->pol)
        return hp_solve_pol(p, nullptr, noise_var, mask, C_ell, tol, true, g1, (const double2 *)g2, f_out, alm_out,
                            info, p->start);
    return hp_solve(p, nullptr, noise_var, mask, C_ell, tol, true, g1, g2, f_out, alm_out, info, p->start);
}

}  // extern "C"

namespace wf {
// device staging of the host-buffer entry points (allocated on first use)
wf_status host_staging(wf_plan p)
{
    if (p->ws.d_in) return WF_OK;
    const size_t npx = (size_t)p->npix;
    const size_t nS = p->g.kind == WF_GEOM_FLAT ? (size_t)p->g.ny * (p->g.nx / 2 + 1) : (size_t)p->lmax + 1;
    const size_t nh = p->g.kind == WF_GEOM_FLAT ? (size_t)p->g.ny * (p->g.nx / 2 + 1) * 2 : (size_t)p->nalm * 2;
    const size_t nc = p->pol ? 3 : 1;  // maps and harmonic vectors per solve
    wf_status st;
    if ((st = plan_alloc(p, (void **)&p->ws.d_in, nc * npx * 8)) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&p->ws.nv_in, (p->pol ? 6 : 1) * npx * 8)) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&p->ws.mask_in, npx)) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&p->ws.out_map, nc * npx * 8)) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&p->ws.cl_in, (p->pol ? 4 : 1) * nS * 8)) != WF_OK) return st;
    return plan_alloc(p, (void **)&p->ws.alm_io, nc * nh * 8);
}
}  // namespace wf

extern "C" {

wf_status wf_solve_host(wf_plan p, const double *d, const double *noise_var, const uint8_t *mask, const double *C_ell,
                        double tol, double *s_wf, double *alm_out, wf_info *info)
{
    if (!p || !d || !noise_var || !C_ell || !s_wf) return set_error(WF_EINVAL, "null argument");
    const size_t npx = (size_t)p->npix;
    const size_t nS = p->g.kind == WF_GEOM_FLAT ? (size_t)p->g.ny * (p->g.nx / 2 + 1) : (size_t)p->lmax + 1;
    const size_t nh = (size_t)p->nalm * 2;
    const size_t nc = p->pol ? 3 : 1, nn = p->pol ? 6 : 1, ncl = p->pol ? 4 : 1;  // components per array
    wf_status st;
    if ((st = host_staging(p)) != WF_OK) return st;
    cudaStream_t s = p->stream;
    WF_CUDA(cudaMemcpyAsync(p->ws.d_in, d, nc * npx * 8, cudaMemcpyHostToDevice, s));
    WF_CUDA(cudaMemcpyAsync(p->ws.nv_in, noise_var, nn * npx * 8, cudaMemcpyHostToDevice, s));
    if (mask) WF_CUDA(cudaMemcpyAsync(p->ws.mask_in, mask, npx, cudaMemcpyHostToDevice, s));
    WF_CUDA(cudaMemcpyAsync(p->ws.cl_in, C_ell, ncl * nS * 8, cudaMemcpyHostToDevice, s));
    st = wf_solve(p, p->ws.d_in, p->ws.nv_in, mask ? p->ws.mask_in : nullptr, p->ws.cl_in, tol, p->ws.out_map,
                  alm_out ? p->ws.alm_io : nullptr, info);
    if (st != WF_OK && st != WF_ENOCONV) return st;
    WF_CUDA(cudaMemcpyAsync(s_wf, p->ws.out_map, nc * npx * 8, cudaMemcpyDeviceToHost, s));
    if (alm_out) WF_CUDA(cudaMemcpyAsync(alm_out, p->ws.alm_io, nc * nh * 8, cudaMemcpyDeviceToHost, s));
    WF_CUDA(cudaStreamSynchronize(s));
    return st;
}

wf_status wf_fluct_host(wf_plan p, const double *noise_var, const uint8_t *mask, const double *C_ell, const double *g1,
                        const double *g2, double tol, double *f_out, double *alm_out, wf_info *info)
{
    if (!p || !noise_var || !C_ell || !g1 || !g2 || !f_out) return set_error(WF_EINVAL, "null argument");
    const size_t npx = (size_t)p->npix;
    const size_t nS = p->g.kind == WF_GEOM_FLAT ? (size_t)p->g.ny * (p->g.nx / 2 + 1) : (size_t)p->lmax + 1;
    const size_t nh = p->g.kind == WF_GEOM_FLAT ? (size_t)p->g.ny * (p->g.nx / 2 + 1) * 2 : (size_t)p->nalm * 2;
    const size_t nc = p->pol ? 3 : 1, nn = p->pol ? 6 : 1, ncl = p->pol ? 4 : 1;  // components per array
    wf_status st;
    if ((st = host_staging(p)) != WF_OK) return st;
    if (!p->ws.g1_in) {
        if ((st = plan_alloc(p, (void **)&p->ws.g1_in, nc * npx * 8)) != WF_OK) return st;
        if ((st = plan_alloc(p, (void **)&p->ws.g2_in, nc * nh * 8)) != WF_OK) return st;
    }
    cudaStream_t s = p->stream;
    WF_CUDA(cudaMemcpyAsync(p->ws.nv_in, noise_var, nn * npx * 8, cudaMemcpyHostToDevice, s));
    if (mask) WF_CUDA(cudaMemcpyAsync(p->ws.mask_in, mask, npx, cudaMemcpyHostToDevice, s));
    WF_CUDA(cudaMemcpyAsync(p->ws.cl_in, C_ell, ncl * nS * 8, cudaMemcpyHostToDevice, s));
    WF_CUDA(cudaMemcpyAsync(p->ws.g1_in, g1, nc * npx * 8, cudaMemcpyHostToDevice, s));
    WF_CUDA(cudaMemcpyAsync(p->ws.g2_in, g2, nc * nh * 8, cudaMemcpyHostToDevice, s));
    st = wf_fluct(p, p->ws.nv_in, mask ? p->ws.mask_in : nullptr, p->ws.cl_in, p->ws.g1_in, p->ws.g2_in, tol,
                  p->ws.out_map, alm_out ? p->ws.alm_io : nullptr, info);
    if (st != WF_OK && st != WF_ENOCONV) return st;
    WF_CUDA(cudaMemcpyAsync(f_out, p->ws.out_map, nc * npx * 8, cudaMemcpyDeviceToHost, s));
    if (alm_out) WF_CUDA(cudaMemcpyAsync(alm_out, p->ws.alm_io, nc * nh * 8, cudaMemcpyDeviceToHost, s));
    WF_CUDA(cudaStreamSynchronize(s));
    return st;
}

wf_status wf_remove_templates(wf_plan p, const double *d_raw, const uint8_t *mask, double *d_out, double *coef)
{
    if (!p || !d_raw || !d_out) return set_error(WF_EINVAL, "null argument");
    if (p->g.kind != WF_GEOM_HEALPIX) return set_error(WF_EUNSUPPORTED, "template marginalisation needs a HEALPix plan");
    // on a polarised plan the monopole / dipole of Eq. (12) are removed from the I map (the first npix values)
    const int grid = std::min(p->npairs, 4 * p->nsm);
    const size_t need = (size_t)14 * grid * sizeof(double);
    if (!p->ws.redu) {
        wf_status st = plan_alloc(p, (void **)&p->ws.redu, (size_t)14 * 4 * p->nsm * sizeof(double));
        if (st != WF_OK) return st;
    }
    k_template_sums<<<grid, 256, 0, p->stream>>>(p->npairs, p->tab.rings, p->tab.x64, d_raw, mask, p->ws.redu);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    std::vector<double> part((size_t)14 * grid);
    WF_CUDA(cudaMemcpyAsync(part.data(), p->ws.redu, need, cudaMemcpyDeviceToHost, p->stream));
    WF_CUDA(cudaStreamSynchronize(p->stream));
    double s[14] = {};
    for (int k = 0; k < 14; ++k)
        for (int b = 0; b < grid; ++b) s[k] += part[(size_t)k * grid + b];
    double G[4][4], b[4], c[4];
    int t = 4;
    for (int i = 0; i < 4; ++i) {
        b[i] = s[i];
        for (int j = i; j < 4; ++j) G[i][j] = G[j][i] = s[t++];
    }
    if (!solve4(G, b, c)) return set_error(WF_EINVAL, "templates are degenerate on the observed pixels");
    k_template_apply<<<grid, 256, 0, p->stream>>>(p->npairs, p->tab.rings, p->tab.x64, d_raw, mask, c[0], c[1], c[2],
                                                  c[3], d_out);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    WF_CUDA(cudaStreamSynchronize(p->stream));
    if (coef)
        for (int i = 0; i < 4; ++i) coef[i] = c[i];
    return WF_OK;
}

wf_status wf_alm2map(wf_plan p, const double *alm, int L, double *map)
{
    if (!p || !alm || !map) return set_error(WF_EINVAL, "null argument");
    if (p->g.kind == WF_GEOM_FLAT) return flat_alm2map(p, alm, map);
    if (L < 0 || L > p->lmax) L = p->lmax;
    wf_status st = p->pol ? pol_synthesis(p, (const double2 *)alm, L, map, nullptr)
                          : hp_alm2map(p, (const double2 *)alm, L, map);
    if (st != WF_OK) return st;
    WF_CUDA(cudaStreamSynchronize(p->stream));
    return WF_OK;
}

wf_status wf_map2alm_adjoint(wf_plan p, const double *map, int L, double *alm)
{
    if (!p || !alm || !map) return set_error(WF_EINVAL, "null argument");
    if (p->g.kind == WF_GEOM_FLAT) return flat_map2alm(p, map, alm);
    if (L < 0 || L > p->lmax) L = p->lmax;
    if (p->pol) {
        wf_status st = pol_adjoint_f64(p, map, L, (double2 *)alm);
        if (st != WF_OK) return st;
        WF_CUDA(cudaStreamSynchronize(p->stream));
        return WF_OK;
    }
    if (p->prec == WF_PREC_FP64) {
        WF_CUDA(cudaMemcpyAsync(p->ws.t, map, p->npix * 8, cudaMemcpyDeviceToDevice, p->stream));
    } else {
        k_map_to_T<float><<<grid_for(p->npix, p->nsm), 256, 0, p->stream>>>(p->npix, map, (float *)p->ws.t);
        WF_COUNT_LAUNCH(p);
        WF_CUDA(cudaGetLastError());
    }
    wf_status st = hp_adjoint_T(p, p->ws.t, L, (double2 *)alm);
    if (st != WF_OK) return st;
    WF_CUDA(cudaStreamSynchronize(p->stream));
    return WF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// FP32 FMA throughput probe (a measurement utility; the paper has no
// counterpart).  The Legendre kernels are bound by the FP32 FMA pipe, so
// their roofline fraction is taken against this measured rate instead of a
// figure built from unit counts and clocks.  Every thread runs independent
// FMA chains (16 scalar, or 8 packed f32x2 through __ffma2_rn) that stay
// bounded (x <- b x + c with b < 1); the result is written only under a
// condition that never holds, which keeps the chains live.
// ---------------------------------------------------------------------------
namespace wf {
namespace {
__device__ float g_fma_probe_sink;

template <bool PACKED>
__global__ void __launch_bounds__(512) k_fma_probe(int iters, float b, float c)
{
    float s = 0.0f;
    if (PACKED) {
        float2 x[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = make_float2(1e-7f * threadIdx.x + i, 1e-7f * blockIdx.x - i);
        const float2 bb = make_float2(b, b), cc = make_float2(c, c);
        for (int k = 0; k < iters; ++k) {
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = __ffma2_rn(x[i], bb, cc);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) s += x[i].x + x[i].y;
    } else {
        float x[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = 1e-7f * threadIdx.x + 1e-7f * blockIdx.x + i;
        for (int k = 0; k < iters; ++k) {
#pragma unroll
            for (int i = 0; i < 16; ++i) x[i] = fmaf(x[i], b, c);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) s += x[i];
    }
    if (s == -1.0f) g_fma_probe_sink = s;
}
}  // namespace
}  // namespace wf

extern "C" wf_status wf_probe_fp32_fma(void *cuda_stream, int packed, double *tflops)
{
    using namespace wf;
    if (!tflops) return set_error(WF_EINVAL, "null argument");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, nsm = 0;
    WF_CUDA(cudaGetDevice(&dev));
    WF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = 2 * nsm, threads = 512, iters = 1 << 16;
    const double flops = (double)blocks * threads * (double)iters * 16.0 * 2.0;
    cudaEvent_t e0, e1;
    WF_CUDA(cudaEventCreate(&e0));
    WF_CUDA(cudaEventCreate(&e1));
    double best = 0.0;
    wf_status status = WF_OK;
    for (int rep = 0; rep < 4 && status == WF_OK; ++rep) {
        cudaEventRecord(e0, st);
        if (packed) k_fma_probe<true><<<blocks, threads, 0, st>>>(iters, 0.9999999f, 1e-7f);
        else k_fma_probe<false><<<blocks, threads, 0, st>>>(iters, 0.9999999f, 1e-7f);
        cudaEventRecord(e1, st);
        cudaError_t ce = cudaGetLastError();
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
        if (ce != cudaSuccess) status = set_error(WF_ECUDA, "fma probe: %s", cudaGetErrorString(ce));
        else if (rep > 0 && ms > 0.0f) best = std::max(best, flops / (ms * 1e-3) / 1e12);  // rep 0 warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *tflops = best;
    return status;
}

// ---------------------------------------------------------------------------
// Several data sets of one signal with the same beam and pixelisation (the
// outlook of Sect. 4): the stacked Wiener-filter equation
//     (S^-1 + sum_k N_k^-1) s = sum_k N_k^-1 d_k
// is Eq. (2) of one data set with N^-1 = sum_k N_k^-1 and N^-1 d =
// sum_k N_k^-1 d_k per pixel, over the data sets that observe the pixel.
// ---------------------------------------------------------------------------
namespace wf {
namespace {
constexpr int MAX_DATASETS = 16;
struct DatasetPtrs {
    const double *d[MAX_DATASETS];
    const double *nv[MAX_DATASETS];
    const uint8_t *mask[MAX_DATASETS];
};

__global__ void k_combine_datasets(long long npix, int k, DatasetPtrs in, double *__restrict__ d_out,
                                   double *__restrict__ nv_out, uint8_t *__restrict__ mask_out,
                                   int *__restrict__ flag)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < npix;
         i += (long long)gridDim.x * blockDim.x) {
        double w = 0.0, wd = 0.0;
        bool bad = false;
        for (int j = 0; j < k; ++j) {
            if (in.mask[j] && in.mask[j][i] == 0) continue;
            const double n = in.nv[j][i], d = in.d[j][i];
            if (!(n > 0.0 && isfinite(n) && isfinite(d))) {
                bad = true;
                continue;
            }
            w += 1.0 / n;
            wd += d / n;
        }
        if (bad) atomicOr(flag, 1);
        const bool seen = w > 0.0;
        nv_out[i] = seen ? 1.0 / w : 1.0;
        d_out[i] = seen ? wd / w : 0.0;
        mask_out[i] = seen ? 1 : 0;
    }
}
}  // namespace
}  // namespace wf

extern "C" wf_status wf_combine_datasets(wf_plan p, int k, const double *const *d, const double *const *noise_var,
                                         const uint8_t *const *mask, double *d_out, double *noise_var_out,
                                         uint8_t *mask_out)
{
    using namespace wf;
    if (!p || !d || !noise_var || !d_out || !noise_var_out || !mask_out) return set_error(WF_EINVAL, "null argument");
    if (k < 1 || k > MAX_DATASETS) return set_error(WF_EINVAL, "need 1 <= k <= %d data sets (got %d)", MAX_DATASETS, k);
    if (p->g.ncomp == 3) return set_error(WF_EUNSUPPORTED, "wf_combine_datasets: temperature plans only");
    DatasetPtrs in{};
    for (int j = 0; j < k; ++j) {
        if (!d[j] || !noise_var[j]) return set_error(WF_EINVAL, "data set %d: null map", j);
        in.d[j] = d[j];
        in.nv[j] = noise_var[j];
        in.mask[j] = mask ? mask[j] : nullptr;
    }
    WF_CUDA(cudaMemsetAsync(p->ws.flag, 0, sizeof(int), p->stream));
    k_combine_datasets<<<grid_for(p->npix, p->nsm), 256, 0, p->stream>>>(p->npix, k, in, d_out, noise_var_out,
                                                                        mask_out, p->ws.flag);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    int flag = 0;
    WF_CUDA(cudaMemcpyAsync(&flag, p->ws.flag, sizeof flag, cudaMemcpyDeviceToHost, p->stream));
    WF_CUDA(cudaStreamSynchronize(p->stream));
    if (flag) return set_error(WF_EINVAL, "noise variance must be finite and > 0 (and d finite) where observed");
    return WF_OK;
}
