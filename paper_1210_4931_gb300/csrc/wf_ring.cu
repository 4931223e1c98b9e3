// Ring part of the HEALPix basis change (Sect. 2.1 / Sect. 3) and the
// pixel-space blend of Eq. (3), fused into the synthesis side.
//
// Each HEALPix ring r has n_r equally spaced pixels at longitudes
// phi_j = (2j + q) pi / n_r.  Synthesis on a ring is
//     f_j = sum_{m=-L..L} G_m e^{i m phi_j}      (G_{-m} = conj G_m)
//         = sum_{k<n} H_k e^{2 pi i k j / n},   H_k = sum_{m = k mod n} G_m e^{i pi m q / n},
// an inverse DFT of the folded coefficients H; analysis is the forward DFT
// F_m = e^{-i pi m q / n} DFT(f)[m mod n].  The north and south rings of a
// pair have the same n and q, so both are packed into one complex DFT
// (z = f_N + i f_S).
//
// DFT engines, chosen per ring length at plan time:
//   n <= 32            direct sum from shared memory;
//   n a power of two   in-place radix-2 FFT in shared memory;
//   otherwise          Bluestein: X_k = c_k sum_j (x_j c_j) conj(c_{k-j}),
//                      c_j = e^{-i pi j^2 / n}, a circular convolution of
//                      power-of-two length M >= 2n - 1.  Since the input is
//                      zero beyond n <= M/2, the length-M transforms split
//                      into two independent half-length ones (even and odd
//                      outputs), so the shared buffer holds M/2 values and
//                      the per-CTA global scratch holds the input and the
//                      even-half result.
//
// Pixel blend (Eq. 3 solved for t with nu = N^-1, r = nu d):
//     t = s + lambda tau (r - nu s) / (1 + (lambda - 1) tau nu)
// and the pixel term of chi^2 (Eq. 6, x-independent part dropped):
//     sum (nu s^2 - 2 r s) / (1 + (lambda - 1) tau nu).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>

#include "wf_internal.cuh"

namespace wf {

namespace {

int ilog2(long long v)
{
    int l = 0;
    while ((1LL << l) < v) ++l;
    return l;
}

bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }

// host radix-2 FFT (FP64), forward e^{-2 pi i jk / n}; used once per ring
// length to tabulate the Bluestein filters
void host_fft(std::vector<double2> &x)
{
    const size_t n = x.size();
    const int lg = ilog2((long long)n);
    for (size_t i = 0; i < n; ++i) {
        size_t j = 0;
        for (int b = 0; b < lg; ++b)
            if (i & (1ull << b)) j |= 1ull << (lg - 1 - b);
        if (i < j) std::swap(x[i], x[j]);
    }
    for (size_t half = 1; half < n; half <<= 1) {
        for (size_t pos = 0; pos < half; ++pos) {
            const double ang = -M_PI * (double)pos / (double)half;
            const double2 w = make_double2(std::cos(ang), std::sin(ang));
            for (size_t i0 = pos; i0 < n; i0 += 2 * half) {
                const size_t i1 = i0 + half;
                const double2 u = x[i0], v = cmul(x[i1], w);
                x[i0] = cadd(u, v);
                x[i1] = csub(u, v);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// device FFT helpers
// ---------------------------------------------------------------------------
// In-place power-of-two FFT in shared memory by all threads of the CTA:
// Stockham autosort passes with radix-8 butterflies held in registers (one
// radix-2 or radix-4 head pass when log2 N is not a multiple of 3).  Each
// pass reads every element once into registers, waits at a barrier, and
// writes every element once, so shared memory sees 2 log8(N) round trips
// instead of 2 log2(N) for radix-2.  sign -1: e^{-2 pi i jk/N}; +1:
// e^{+2 pi i jk/N} (unnormalised).  Twiddles come from a shared-memory table laid out
// by pass: stw[Ns + k] = e^{-2 pi i k / (8 Ns)}, k < Ns, for every power of two
// Ns <= 2^logB / 8 (2^logB / 4 entries: 16 KB in FP32 for the 8192-point rings).
// A warp of one pass reads consecutive entries (Ns >= 32) or a few broadcast ones;
// one table of the circle indexed k 2^logB / (8 Ns) put the lanes of the middle
// passes on one bank.
// Supports N <= 8192 with NT = 512 threads (two radix-8 butterflies per thread) or
// NT = 1024 (one).
template <typename T>
__device__ __forceinline__ cx<T> mul_i(cx<T> a, int sign)
{
    return sign > 0 ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);  // (sign i) a
}

// Radix-R DFT in registers, in place, decimation in frequency: on return
// v[k] holds output X[brev_R(k)] (bit-reversed index), which the caller
// undoes at compile time when it stores.
template <typename T>
__device__ __forceinline__ void bfly(cx<T> &a, cx<T> &b)
{
    const cx<T> t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <typename T, int R> struct SmallDft;
template <typename T> struct SmallDft<T, 2> {
    static __device__ __forceinline__ void run(cx<T> (&v)[2], int) { bfly<T>(v[0], v[1]); }
    static __device__ __forceinline__ constexpr int out(int k) { return k; }
};
template <typename T> struct SmallDft<T, 4> {
    static __device__ __forceinline__ void run(cx<T> (&v)[4], int sign)
    {
        bfly<T>(v[0], v[2]);
        bfly<T>(v[1], v[3]);
        v[3] = mul_i<T>(v[3], sign);
        bfly<T>(v[0], v[1]);
        bfly<T>(v[2], v[3]);
    }
    static __device__ __forceinline__ constexpr int out(int k) { return ((k & 1) << 1) | ((k >> 1) & 1); }
};
template <typename T> struct SmallDft<T, 8> {
    static __device__ __forceinline__ void run(cx<T> (&v)[8], int sign)
    {
        const T c = (T)0.70710678118654752440;
        const T s = sign > 0 ? c : -c;
        bfly<T>(v[0], v[4]);
        bfly<T>(v[1], v[5]);
        bfly<T>(v[2], v[6]);
        bfly<T>(v[3], v[7]);
        v[5] = cmul(v[5], mk<T>(c, s));
        v[6] = mul_i<T>(v[6], sign);
        v[7] = cmul(v[7], mk<T>(-c, s));
        bfly<T>(v[0], v[2]);
        bfly<T>(v[1], v[3]);
        bfly<T>(v[4], v[6]);
        bfly<T>(v[5], v[7]);
        v[3] = mul_i<T>(v[3], sign);
        v[7] = mul_i<T>(v[7], sign);
        bfly<T>(v[0], v[1]);
        bfly<T>(v[2], v[3]);
        bfly<T>(v[4], v[5]);
        bfly<T>(v[6], v[7]);
    }
    static __device__ __forceinline__ constexpr int out(int k)
    {
        return ((k & 1) << 2) | (k & 2) | ((k >> 2) & 1);
    }
};

// Shared-memory FFT buffers are padded by one entry per 16: the Stockham
// writes at small strides (8 Ns entries apart) would otherwise fall on one
// or two banks for the whole warp.
__device__ __forceinline__ int pidx(int i) { return i + (i >> 4); }
inline size_t padded_len(int n) { return (size_t)n + (size_t)n / 16 + 1; }

template <typename T, int R, int LOGR, int BPT>
__device__ __forceinline__ void stockham_pass(cx<T> *x, int logN, int logNs, int sign, const cx<T> *stw)
{
    static_assert(R == 2 || R == 4 || R == 8, "radix 2, 4 or 8");
    const int NR = (1 << logN) >> LOGR;
    const int Ns = 1 << logNs;
    // w1 = e^{-2 pi i k / (R Ns)} = stw[Ns + k]: radix 2 and 4 run only as the first pass
    // (Ns = 1, k = 0, w1 = 1), so the table of R = 8 serves every pass
    cx<T> v[BPT][R];
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int j = b * blockDim.x + threadIdx.x;
        if (j < NR) {
            const int k = j & (Ns - 1);
            // twiddles w^r, r < R, from one table entry w = e^{-+2 pi i k / (R Ns)} by products
            // in a tree of depth log2 R (w^2 = w w, w^3 = w^2 w, w^4 = w^2 w^2, ...), not a
            // chain of R - 2 dependent products
            cx<T> w[R];
            w[0] = mk<T>(1, 0);
            w[1] = stw[Ns + k];
            if (sign > 0) w[1].y = -w[1].y;
#pragma unroll
            for (int r = 2; r < R; ++r) {
                const int hb = r >= 4 ? 4 : 2;  // highest power of two <= r (R <= 8)
                w[r] = r == hb ? cmul(w[hb / 2], w[hb / 2]) : cmul(w[hb], w[r - hb]);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) v[b][r] = x[pidx(j + r * NR)];
#pragma unroll
            for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], w[r]);
            SmallDft<T, R>::run(v[b], sign);
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int j = b * blockDim.x + threadIdx.x;
        if (j < NR) {
            const int k = j & (Ns - 1);
            const int d = ((j >> logNs) << (logNs + LOGR)) + k;
#pragma unroll
            for (int r = 0; r < R; ++r) x[pidx(d + SmallDft<T, R>::out(r) * Ns)] = v[b][r];
        }
    }
    __syncthreads();
}

// Threads of the ring kernels: FP32 plans run 1024 (32 warps per SM, one radix-8
// butterfly per thread and pass at N = 8192: twice the warps of 512 threads to hide the
// shared-memory and L2 latencies of one pair's chain of passes), FP64 plans 512 (their
// butterflies need twice the registers).
template <typename T> __host__ __device__ constexpr int ring_threads() { return sizeof(T) == 4 ? 1024 : 512; }

template <typename T>
__device__ __noinline__ void fft_pow2(cx<T> *x, int logN, int sign, const cx<T> *stw)
{
    constexpr int NT = ring_threads<T>();
    int logNs = 0;
    const int head = logN % 3;
    if (head == 1) {
        stockham_pass<T, 2, 1, 4096 / NT>(x, logN, 0, sign, stw);
        logNs = 1;
    } else if (head == 2) {
        stockham_pass<T, 4, 2, 2048 / NT>(x, logN, 0, sign, stw);
        logNs = 2;
    }
    while (logNs < logN) {
        stockham_pass<T, 8, 3, 1024 / NT>(x, logN, logNs, sign, stw);
        logNs += 3;
    }
}

// The n outputs of a ring DFT: in the padded FFT buffer (power-of-two rings)
// or in the plain zout buffer (direct and Bluestein rings).
template <typename T> struct RingOut {
    const cx<T> *p;
    int padded;
    __device__ __forceinline__ cx<T> operator[](int j) const { return p[padded ? pidx(j) : j]; }
};

// DFT of one ring pair.  Input: padded buf (direct / pow2) or plain zin (Bluestein).
template <typename T>
__device__ RingOut<T> ring_dft(const RingTab &R, cx<T> *buf, cx<T> *zin, cx<T> *zout, int sign,
                               const cx<T> *__restrict__ roots, const cx<T> *__restrict__ V,
                               const cx<T> *__restrict__ chirp, const cx<T> *__restrict__ tw, int logNmax,
                               const cx<T> *stw)
{
    const int n = R.n;
    const unsigned twon = 2u * (unsigned)n;
    const cx<T> *root = roots + R.rootOff;
    if (R.kind == RING_NAIVE) {
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            cx<T> acc = mk<T>(0, 0);
            for (int k = 0; k < n; ++k) {
                cx<T> w = root[(2u * (unsigned)(j * k)) % twon];
                if (sign < 0) w.y = -w.y;
                acc = cadd(acc, cmul(buf[pidx(k)], w));
            }
            zout[j] = acc;
        }
        __syncthreads();
        return RingOut<T>{zout, 0};
    }
    if (R.kind == RING_POW2) {
        fft_pow2<T>(buf, R.logF, sign, stw);
        return RingOut<T>{buf, 1};
    }
    // Bluestein, two half-length passes; the chirp c_j = e^{-i pi j^2 / n} is read
    // from its own table in order (consecutive lanes, consecutive entries)
    const int H = 1 << R.logF;                 // M / 2
    const int mstep = logNmax - (R.logF + 1);  // index step of w_M in tw
    const cx<T> *Vh = V + R.vOff;
    const cx<T> *ch = chirp + R.cOff;
    for (int h = 0; h < 2; ++h) {
#pragma unroll 4
        for (int j = threadIdx.x; j < H; j += blockDim.x) {
            cx<T> v = mk<T>(0, 0);
            if (j < n) {
                cx<T> u = zin[j];
                if (sign > 0) u.y = -u.y;
                v = cmul(u, ch[j]);
                if (h) v = cmul(v, tw[j << mstep]);
            }
            buf[pidx(j)] = v;
        }
        __syncthreads();
        fft_pow2<T>(buf, R.logF, -1, stw);
        for (int k = threadIdx.x; k < H; k += blockDim.x) buf[pidx(k)] = cmul(buf[pidx(k)], Vh[h * H + k]);
        __syncthreads();
        fft_pow2<T>(buf, R.logF, +1, stw);
#pragma unroll 4
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            if (h == 0) {
                zout[k] = buf[pidx(k)];
            } else {
                cx<T> w = tw[k << mstep];
                w.y = -w.y;  // w_M^{-k}
                cx<T> y = cmul(cadd(zout[k], cmul(buf[pidx(k)], w)), ch[k]);
                if (sign > 0) y.y = -y.y;
                zout[k] = y;
            }
        }
        __syncthreads();
    }
    return RingOut<T>{zout, 0};
}

template <typename T>
__device__ __forceinline__ double block_sum(double v, double *red)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    __syncthreads();  // red is reused by the next call
    return s;
}

struct RingCommon {
    int npairs, lmax, L, logNmax;
    int logB;             // log2 of the longest FFT run (the shared twiddle table has 2^logB / 4 entries)
    const RingTab *rings;
    const int *order;     // ring pairs by decreasing cost
    int *ticket;          // work counter (zeroed before the launch)
    long long scr_stride;
    const float2 *Glow;   // mixed path: FP64-block coefficients for m < lc, rounded to FP32 (or null)
    int lc, glow_stride;
    int bpad;             // padded shared FFT buffer length
    int zsmem;            // 1: Bluestein / direct buffers follow the FFT buffer in shared memory
};

__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// prefetch a byte range into L2, one 128-byte line per thread and step
__device__ __forceinline__ void prefetch_range(const void *base, size_t bytes)
{
    const char *b = reinterpret_cast<const char *>(base);
    for (size_t off = (size_t)threadIdx.x * 128; off < bytes; off += (size_t)blockDim.x * 128) prefetch_l2(b + off);
}

__device__ __forceinline__ bool aligned16(const void *p) { return ((size_t)p & 15) == 0; }

// Eq. 3 blend of four pixels (float4 lanes), adding their chi^2 pixel terms to chi
__device__ __forceinline__ float4 blend4(float4 s, float4 r, float4 nu, float lt, float lm1t, float &chi)
{
    auto one = [&](float sv, float rv, float nv) {
        const float den = 1.f + lm1t * nv;
        chi += (nv * sv * sv - 2.f * rv * sv) / den;
        return sv + lt * (rv - nv * sv) / den;
    };
    return make_float4(one(s.x, r.x, nu.x), one(s.y, r.y, nu.y), one(s.z, r.z, nu.z), one(s.w, r.w, nu.w));
}

// Shared twiddle table by pass: stw[Ns + k] = e^{-2 pi i k / (8 Ns)} = tw[k 2^logNmax / (8 Ns)]
// for the powers of two Ns <= 2^logB / 8 (entry 0 unused).
template <typename T>
__device__ __forceinline__ void load_twiddles(cx<T> *stw, const cx<T> *__restrict__ tw, const RingCommon &rc)
{
    const int n = (1 << rc.logB) >> 2;
    for (int u = threadIdx.x; u < n; u += blockDim.x) {
        if (u == 0) continue;
        const int logNs = 31 - __clz(u), k = u - (1 << logNs);
        stw[u] = tw[(size_t)k << (rc.logNmax - 3 - logNs)];
    }
}

// The next pair's ring tables into L2: e^{i pi p / n} (fold phases and Bluestein chirps)
// and, for a Bluestein ring, its filter spectrum (M entries).
template <typename T>
__device__ __forceinline__ void prefetch_ring_tables(const RingTab &Rn, const cx<T> *roots, const cx<T> *V,
                                                     const cx<T> *chirp)
{
    if (Rn.kind == RING_BLUESTEIN) {
        prefetch_range(roots + Rn.rootOff, (size_t)2 * Rn.n * sizeof(cx<T>));
        prefetch_range(V + Rn.vOff, ((size_t)2 << Rn.logF) * sizeof(cx<T>));
        prefetch_range(chirp + Rn.cOff, (size_t)Rn.n * sizeof(cx<T>));
    } else if (Rn.q) {
        prefetch_range(roots + Rn.rootOff, (size_t)2 * Rn.n * sizeof(cx<T>));
    }
}

// Work distribution: CTAs take ring pairs from a global counter in order of
// decreasing cost (Bluestein rings first), one ticket ahead so that the next
// pair's rows can be prefetched while this one is transformed.
__device__ __forceinline__ int take_ticket(int *ticket, int *s_tick)
{
    if (threadIdx.x == 0) *s_tick = atomicAdd(ticket, 1);
    __syncthreads();
    const int t = *s_tick;
    __syncthreads();
    return t;
}

// Unfold a forward ring DFT of the packed pair (z = f_N + i f_S) to
// F_m = e^{-i pi m q / n} DFT(f)[m mod n] for both rings, m <= L; ends with a barrier.
template <typename T>
__device__ __forceinline__ void unfold_ring(const RingTab &R, const RingOut<T> &z, const cx<T> *__restrict__ root, int q,
                                            unsigned twon, bool south, cx<T> *__restrict__ f, int L)
{
    const int n = R.n;
#pragma unroll 4
    for (int m = threadIdx.x; m <= L; m += blockDim.x) {
        const int k = m % n;
        const int nk = (n - k) % n;
        const cx<T> zk = z[k], znk = z[nk];
        const cx<T> tn = mk<T>((T)0.5 * (zk.x + znk.x), (T)0.5 * (zk.y - znk.y));
        const cx<T> ts = mk<T>((T)0.5 * (zk.y + znk.y), (T)-0.5 * (zk.x - znk.x));
        cx<T> ph = root[q ? (unsigned)m % twon : 0u];
        ph.y = -ph.y;
        f[2 * m] = cmul(ph, tn);
        f[2 * m + 1] = south ? cmul(ph, ts) : mk<T>(0, 0);
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// synthesis side: fold -> inverse ring DFT -> blend (or write the map)
// ---------------------------------------------------------------------------
// Fold H_k = sum_{m = k mod n} G_m e^{i pi m q / n} + conj terms of -m, for
// the packed north/south pair.  Each bin is summed by S sub-lanes of one warp
// (S = n > 256 ? 1 : up to 32), each taking every S-th alias of the bin, and
// the S partial sums are combined by shuffles in a fixed order: small polar
// rings, whose bins collect up to 2L/n aliases, no longer serialise the CTA.
template <typename T>
__global__ void __launch_bounds__(ring_threads<T>(), 1) k_ringsyn(RingCommon rc, const cx<T> *__restrict__ roots,
                                                          const cx<T> *__restrict__ V,
                                                          const cx<T> *__restrict__ chirp, const cx<T> *__restrict__ tw,
                                                          cx<T> *__restrict__ scr, const cx<T> *__restrict__ G,
                                                          int mode, const T *__restrict__ r, const T *__restrict__ nu,
                                                          T lam, T tau, T *__restrict__ tmap,
                                                          double *__restrict__ omap, double *__restrict__ part,
                                                          cx<T> *__restrict__ F)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    __shared__ int s_tick;
    cx<T> *buf = reinterpret_cast<cx<T> *>(smem_raw);
    cx<T> *zin = rc.zsmem ? buf + rc.bpad : scr + (size_t)blockIdx.x * rc.scr_stride;
    cx<T> *zout = zin + rc.scr_stride / 2;
    cx<T> *stw = buf + rc.bpad + (rc.zsmem ? rc.scr_stride : 0);
    load_twiddles<T>(stw, tw, rc);
    const int L = rc.L;
    const T lt = lam * tau, lm1t = (lam - (T)1) * tau;
    int cur = take_ticket(rc.ticket, &s_tick);
    while (cur < rc.npairs) {
        if (threadIdx.x == 0) s_tick = atomicAdd(rc.ticket, 1);
        __syncthreads();
        const int nxt = s_tick;
        const int pair = rc.order[cur];
        const RingTab R = rc.rings[pair];
        const int n = R.n, q = R.q;
        const unsigned twon = 2u * (unsigned)n;
        const cx<T> *root = roots + R.rootOff;
        const cx<T> *g = G + (size_t)pair * (rc.lmax + 1) * 2;
        const bool blue = R.kind == RING_BLUESTEIN;
        const bool south = R.offS >= 0;
        if (nxt < rc.npairs) {  // next pair of this CTA: pull its rows into L2
            const int pn = rc.order[nxt];
            const RingTab Rn = rc.rings[pn];
            prefetch_range(G + (size_t)pn * (rc.lmax + 1) * 2, (size_t)(L + 1) * 2 * sizeof(cx<T>));
            prefetch_ring_tables<T>(Rn, roots, V, chirp);
            if (mode == RS_BLEND) {
                prefetch_range(r + Rn.offN, (size_t)Rn.n * sizeof(T));
                prefetch_range(nu + Rn.offN, (size_t)Rn.n * sizeof(T));
                if (Rn.offS >= 0) {
                    prefetch_range(r + Rn.offS, (size_t)Rn.n * sizeof(T));
                    prefetch_range(nu + Rn.offS, (size_t)Rn.n * sizeof(T));
                }
            }
        }
        const float2 *gl = rc.Glow ? rc.Glow + (size_t)pair * rc.glow_stride * 2 : nullptr;
        auto coef = [&](int m, int h) -> cx<T> {
            cx<T> v = g[2 * m + h];
            if (gl && m < rc.lc) {
                const float2 w = gl[2 * m + h];
                v.x += (T)w.x;
                v.y += (T)w.y;
            }
            return v;
        };
        int S = 1;
        while (S < 32 && 2 * S * n <= (int)blockDim.x) S *= 2;
        const int sub = threadIdx.x & (S - 1);
        const int nb = blockDim.x / S;
        // rings longer than L: each bin k has at most one alias of each sign (m = k and
        // m = n - k), so the bins are independent and four of them are loaded at once
        const bool single = n > L;
        if (single) {
#pragma unroll 4
            for (int k = threadIdx.x; k < n; k += blockDim.x) {
                cx<T> hn = mk<T>(0, 0), hs = mk<T>(0, 0);
                if (k <= L) {
                    const cx<T> ph = root[q ? k : 0];
                    hn = cmul(coef(k, 0), ph);
                    hs = cmul(coef(k, 1), ph);
                }
                const int mneg = n - k;
                if (k > 0 && mneg <= L) {
                    const cx<T> ph = root[q ? mneg : 0];
                    hn = cadd(hn, cconj(cmul(coef(mneg, 0), ph)));
                    hs = cadd(hs, cconj(cmul(coef(mneg, 1), ph)));
                }
                if (!south) hs = mk<T>(0, 0);
                const cx<T> z = mk<T>(hn.x - hs.y, hn.y + hs.x);
                if (blue) zin[k] = z;
                else buf[pidx(k)] = z;
            }
        }
        for (int base = 0; base < (single ? 0 : n); base += nb) {
            const int k = base + threadIdx.x / S;
            cx<T> hn = mk<T>(0, 0), hs = mk<T>(0, 0);
            if (k < n) {
                for (int m = k + sub * n; m <= L; m += S * n) {
                    const cx<T> ph = root[q ? (unsigned)m % twon : 0u];
                    hn = cadd(hn, cmul(coef(m, 0), ph));
                    hs = cadd(hs, cmul(coef(m, 1), ph));
                }
                for (int m = (k == 0 ? n : n - k) + sub * n; m <= L; m += S * n) {
                    const cx<T> ph = root[q ? (unsigned)m % twon : 0u];
                    hn = cadd(hn, cconj(cmul(coef(m, 0), ph)));
                    hs = cadd(hs, cconj(cmul(coef(m, 1), ph)));
                }
            }
            for (int o = S >> 1; o >= 1; o >>= 1) {
                hn.x += __shfl_xor_sync(0xffffffffu, hn.x, o);
                hn.y += __shfl_xor_sync(0xffffffffu, hn.y, o);
                hs.x += __shfl_xor_sync(0xffffffffu, hs.x, o);
                hs.y += __shfl_xor_sync(0xffffffffu, hs.y, o);
            }
            if (k < n && sub == 0) {
                if (!south) hs = mk<T>(0, 0);
                const cx<T> z = mk<T>(hn.x - hs.y, hn.y + hs.x);
                if (blue) zin[k] = z;
                else buf[pidx(k)] = z;
            }
        }
        __syncthreads();
        const RingOut<T> z = ring_dft<T>(R, buf, zin, zout, +1, roots, V, chirp, tw, rc.logNmax, stw);
        T chi_pair = 0;  // per-thread partial of this pair in the working precision
        int j0 = threadIdx.x, jstep = blockDim.x;
        if constexpr (sizeof(T) == 4) {
            // four consecutive pixels per thread with 16-byte loads and stores (ring
            // lengths and offsets are multiples of 4); the scalar loop below takes over
            // for unaligned map views
            const bool fused = mode == RS_BLEND_ANA, blend = mode == RS_BLEND || fused;
            if (mode != RS_MAP && (fused || (aligned16(tmap + R.offN) && (!south || aligned16(tmap + R.offS)))) &&
                (!blend ||
                 (aligned16(r + R.offN) && aligned16(nu + R.offN) &&
                  (!south || (aligned16(r + R.offS) && aligned16(nu + R.offS)))))) {
                for (int j = 4 * threadIdx.x; j < n; j += 4 * blockDim.x) {
                    const cx<T> z0 = z[j], z1 = z[j + 1], z2 = z[j + 2], z3 = z[j + 3];
                    float4 sN = make_float4(z0.x, z1.x, z2.x, z3.x), sS = make_float4(z0.y, z1.y, z2.y, z3.y);
                    if (blend) {
                        sN = blend4(sN, *reinterpret_cast<const float4 *>(r + R.offN + j),
                                    *reinterpret_cast<const float4 *>(nu + R.offN + j), lt, lm1t, chi_pair);
                        if (south)
                            sS = blend4(sS, *reinterpret_cast<const float4 *>(r + R.offS + j),
                                        *reinterpret_cast<const float4 *>(nu + R.offS + j), lt, lm1t, chi_pair);
                    }
                    if (fused) {  // packed north/south input of the forward DFT (same indices as z)
                        if (!south) sS = make_float4(0.f, 0.f, 0.f, 0.f);
                        cx<T> *d = blue ? zin + j : nullptr;
                        const cx<T> v0 = mk<T>(sN.x, sS.x), v1 = mk<T>(sN.y, sS.y), v2 = mk<T>(sN.z, sS.z),
                                    v3 = mk<T>(sN.w, sS.w);
                        if (d) {
                            d[0] = v0;
                            d[1] = v1;
                            d[2] = v2;
                            d[3] = v3;
                        } else {
                            buf[pidx(j)] = v0;
                            buf[pidx(j + 1)] = v1;
                            buf[pidx(j + 2)] = v2;
                            buf[pidx(j + 3)] = v3;
                        }
                    } else {
                        *reinterpret_cast<float4 *>(tmap + R.offN + j) = sN;
                        if (south) *reinterpret_cast<float4 *>(tmap + R.offS + j) = sS;
                    }
                }
                j0 = n;  // done
            }
        }
        for (int j = j0; j < n; j += jstep) {
            const cx<T> zz = z[j];
            const long long iN = R.offN + j;
            if (mode == RS_MAP) {
                omap[iN] = (double)zz.x;
                if (south) omap[R.offS + j] = (double)zz.y;
            } else if (mode == RS_SYN) {
                tmap[iN] = zz.x;
                if (south) tmap[R.offS + j] = zz.y;
            } else {
                T tN, tS = 0;
                {
                    const T s = zz.x, nv = nu[iN], rv = r[iN];
                    const T den = (T)1 + lm1t * nv;
                    tN = s + lt * (rv - nv * s) / den;
                    chi_pair += (nv * s * s - (T)2 * rv * s) / den;
                }
                if (south) {
                    const long long iS = R.offS + j;
                    const T s = zz.y, nv = nu[iS], rv = r[iS];
                    const T den = (T)1 + lm1t * nv;
                    tS = s + lt * (rv - nv * s) / den;
                    chi_pair += (nv * s * s - (T)2 * rv * s) / den;
                }
                if (mode == RS_BLEND_ANA) {  // same index as z: read and written by this thread only
                    if (blue) zin[j] = mk<T>(tN, tS);
                    else buf[pidx(j)] = mk<T>(tN, tS);
                } else {
                    tmap[iN] = tN;
                    if (south) tmap[R.offS + j] = tS;
                }
            }
        }
        if (mode == RS_BLEND || mode == RS_BLEND_ANA) {  // per-pair partial: the reduction order does not depend on the schedule
            const double s = block_sum<T>((double)chi_pair, red);
            if (threadIdx.x == 0) part[pair] = s;
        } else {
            __syncthreads();
        }
        if (mode == RS_BLEND_ANA) {  // forward DFT of the blended ring and unfold to F_m, m <= L
            const RingOut<T> zf = ring_dft<T>(R, buf, zin, zout, -1, roots, V, chirp, tw, rc.logNmax, stw);
            unfold_ring<T>(R, zf, root, q, twon, south, F + (size_t)pair * (rc.lmax + 1) * 2, L);
        }
        cur = nxt;
    }
}

// ---------------------------------------------------------------------------
// analysis side: pack -> forward ring DFT -> unfold to F_m, m <= L
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(ring_threads<T>(), 1) k_ringana(RingCommon rc, const cx<T> *__restrict__ roots,
                                                          const cx<T> *__restrict__ V,
                                                          const cx<T> *__restrict__ chirp, const cx<T> *__restrict__ tw,
                                                          cx<T> *__restrict__ scr, const T *__restrict__ map,
                                                          cx<T> *__restrict__ F)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_tick;
    cx<T> *buf = reinterpret_cast<cx<T> *>(smem_raw);
    cx<T> *zin = rc.zsmem ? buf + rc.bpad : scr + (size_t)blockIdx.x * rc.scr_stride;
    cx<T> *zout = zin + rc.scr_stride / 2;
    cx<T> *stw = buf + rc.bpad + (rc.zsmem ? rc.scr_stride : 0);
    load_twiddles<T>(stw, tw, rc);
    const int L = rc.L;
    int cur = take_ticket(rc.ticket, &s_tick);
    while (cur < rc.npairs) {
        if (threadIdx.x == 0) s_tick = atomicAdd(rc.ticket, 1);
        __syncthreads();
        const int nxt = s_tick;
        const int pair = rc.order[cur];
        const RingTab R = rc.rings[pair];
        const int n = R.n, q = R.q;
        const unsigned twon = 2u * (unsigned)n;
        const cx<T> *root = roots + R.rootOff;
        const bool blue = R.kind == RING_BLUESTEIN;
        const bool south = R.offS >= 0;
        if (nxt < rc.npairs) {
            const RingTab Rn = rc.rings[rc.order[nxt]];
            prefetch_ring_tables<T>(Rn, roots, V, chirp);
            prefetch_range(map + Rn.offN, (size_t)Rn.n * sizeof(T));
            if (Rn.offS >= 0) prefetch_range(map + Rn.offS, (size_t)Rn.n * sizeof(T));
        }
        int j0 = threadIdx.x;
        if constexpr (sizeof(T) == 4) {
            // four consecutive pixels per thread with 16-byte loads (aligned map views)
            if (aligned16(map + R.offN) && (!south || aligned16(map + R.offS))) {
                for (int j = 4 * threadIdx.x; j < n; j += 4 * blockDim.x) {
                    const float4 a = *reinterpret_cast<const float4 *>(map + R.offN + j);
                    const float4 b = south ? *reinterpret_cast<const float4 *>(map + R.offS + j) : make_float4(0, 0, 0, 0);
                    cx<T> *d = blue ? zin + j : nullptr;
                    const cx<T> v0 = mk<T>(a.x, b.x), v1 = mk<T>(a.y, b.y), v2 = mk<T>(a.z, b.z), v3 = mk<T>(a.w, b.w);
                    if (d) {
                        d[0] = v0;
                        d[1] = v1;
                        d[2] = v2;
                        d[3] = v3;
                    } else {
                        buf[pidx(j)] = v0;
                        buf[pidx(j + 1)] = v1;
                        buf[pidx(j + 2)] = v2;
                        buf[pidx(j + 3)] = v3;
                    }
                }
                j0 = n;
            }
        }
        for (int j = j0; j < n; j += blockDim.x) {
            const cx<T> v = mk<T>(map[R.offN + j], south ? map[R.offS + j] : (T)0);
            if (blue) zin[j] = v;
            else buf[pidx(j)] = v;
        }
        __syncthreads();
        const RingOut<T> z = ring_dft<T>(R, buf, zin, zout, -1, roots, V, chirp, tw, rc.logNmax, stw);
        unfold_ring<T>(R, z, root, q, twon, south, F + (size_t)pair * (rc.lmax + 1) * 2, L);
        cur = nxt;
    }
}

template <typename T> struct RingLaunch {
    static RingCommon common(wf_plan p, int L)
    {
        const HpTables &t = p->tab;
        RingCommon rc{};
        rc.npairs = p->npairs;
        rc.lmax = p->lmax;
        rc.L = L;
        rc.logNmax = t.logNmax;
        rc.rings = t.rings;
        rc.order = t.order;
        rc.ticket = t.ticket;
        rc.scr_stride = 2LL * zlen(t);
        rc.bpad = (int)padded_len(t.bmax);
        rc.logB = ilog2(t.bmax);
        rc.zsmem = zsmem();
        return rc;
    }
    static wf_status syn(wf_plan p, int L, RingSynMode mode, double lam, double tau, double *omap)
    {
        return syn_buf(p, L, mode, lam, tau, p->ws.G, p->ws.t, omap);
    }
    static wf_status syn_buf(wf_plan p, int L, RingSynMode mode, double lam, double tau, const void *G, void *tmap,
                             double *omap)
    {
        const HpTables &t = p->tab;
        if (p->prec != WF_PREC_FP64 && t.lc_mx > 0)
            return syn_buf_low(p, L, mode, lam, tau, G, p->ws.Glow, t.lc_mx, t.glow_cap, tmap, omap);
        return syn_buf_low(p, L, mode, lam, tau, G, nullptr, 0, 0, tmap, omap);
    }
    // with the FP64 block's coefficients (m < lc, [pair][m][hemisphere] with
    // glow_stride columns per pair) added to G, or none (glow null)
    static wf_status syn_buf_low(wf_plan p, int L, RingSynMode mode, double lam, double tau, const void *G,
                                 const float2 *glow, int lc, int glow_stride, void *tmap, double *omap,
                                 void *F = nullptr)
    {
        const HpTables &t = p->tab;
        RingCommon rc = common(p, L);
        if (glow && lc > 0) {
            rc.Glow = glow;
            rc.lc = lc;
            rc.glow_stride = glow_stride;
        }
        const size_t sm = smem_bytes(t);
        WF_CUDA(cudaMemsetAsync(t.ticket, 0, sizeof(int), p->stream));
        k_ringsyn<T><<<t.ringGrid, ring_threads<T>(), sm, p->stream>>>(
            rc, (const cx<T> *)t.roots, (const cx<T> *)t.V, (const cx<T> *)t.chirp, (const cx<T> *)t.tw,
            (cx<T> *)p->ws.scr,
            (const cx<T> *)G, (int)mode, (const T *)p->ws.r, (const T *)p->ws.nu, (T)lam, (T)tau,
            (T *)tmap, omap, p->ws.part_pix, (cx<T> *)F);
        WF_COUNT_LAUNCH(p);
        WF_CUDA(cudaGetLastError());
        return WF_OK;
    }
    // messenger step on the rings: fold, inverse DFT, Eq. 3, forward DFT, unfold into F
    static wf_status syn_ana(wf_plan p, int L, double lam, double tau)
    {
        const HpTables &t = p->tab;
        if (p->prec != WF_PREC_FP64 && t.lc_mx > 0)
            return syn_buf_low(p, L, RS_BLEND_ANA, lam, tau, p->ws.G, p->ws.Glow, t.lc_mx, t.glow_cap, nullptr,
                               nullptr, p->ws.F);
        return syn_buf_low(p, L, RS_BLEND_ANA, lam, tau, p->ws.G, nullptr, 0, 0, nullptr, nullptr, p->ws.F);
    }
    static wf_status ana(wf_plan p, int L, const void *map) { return ana_buf(p, L, map, p->ws.F); }
    static wf_status ana_buf(wf_plan p, int L, const void *map, void *F)
    {
        const HpTables &t = p->tab;
        RingCommon rc = common(p, L);
        const size_t sm = smem_bytes(t);
        WF_CUDA(cudaMemsetAsync(t.ticket, 0, sizeof(int), p->stream));
        k_ringana<T><<<t.ringGrid, ring_threads<T>(), sm, p->stream>>>(rc, (const cx<T> *)t.roots, (const cx<T> *)t.V,
                                                                  (const cx<T> *)t.chirp, (const cx<T> *)t.tw,
                                                                  (cx<T> *)p->ws.scr,
                                                                  (const T *)map, (cx<T> *)F);
        WF_COUNT_LAUNCH(p);
        WF_CUDA(cudaGetLastError());
        return WF_OK;
    }
    // FP32: the Bluestein / direct buffers fit next to the FFT buffer (the kernel
    // runs one CTA per SM anyway, bounded by registers); FP64 keeps them in
    // per-CTA global scratch
    static int zsmem() { return sizeof(T) == 4 ? 1 : 0; }
    static long long zlen(const HpTables &t) { return t.maxBlue > NAIVE_MAX ? t.maxBlue : NAIVE_MAX; }
    static size_t smem_bytes(const HpTables &t)
    {
        return (padded_len(t.bmax) + (zsmem() ? 2 * (size_t)zlen(t) : 0) + (size_t)t.bmax / 4) * sizeof(cx<T>);
    }
    // The dynamic shared-memory limit is raised once per kernel and size, before
    // any launch that needs it, and never lowered: plans of several sizes may
    // launch concurrently from different host threads.
    static wf_status grid(wf_plan p, int *out)
    {
        const size_t sm = smem_bytes(p->tab);
        wf_status st;
        if ((st = raise_smem_limit((const void *)k_ringsyn<T>, sm)) != WF_OK) return st;
        if ((st = raise_smem_limit((const void *)k_ringana<T>, sm)) != WF_OK) return st;
        int b1 = 0, b2 = 0;
        WF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_ringsyn<T>, ring_threads<T>(), sm));
        WF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_ringana<T>, ring_threads<T>(), sm));
        int b = b1 < b2 ? b1 : b2;
        if (b < 1) return set_error(WF_EUNSUPPORTED, "ring kernel does not fit on an SM (smem %zu bytes)", sm);
        long long g = (long long)b * p->nsm;
        if (g > p->npairs) g = p->npairs;
        *out = (int)g;
        return WF_OK;
    }
};

template <typename T>
wf_status upload_cx(wf_plan p, void **dst, const std::vector<double2> &src)
{
    wf_status st = plan_alloc(p, dst, src.size() * sizeof(cx<T>) + 16);
    if (st != WF_OK) return st;
    std::vector<cx<T>> tmp(src.size());
    for (size_t i = 0; i < src.size(); ++i) tmp[i] = mk<T>((T)src[i].x, (T)src[i].y);
    if ((st = to_device(p, *dst, tmp.data(), tmp.size() * sizeof(cx<T>))) != WF_OK) return st;
    return WF_OK;
}

}  // namespace

wf_status hp_build_ring_tables(wf_plan p)
{
    const int nside = p->nside, np = p->npairs;
    const int R = 4 * nside - 1;
    // ring offsets (RING order)
    std::vector<long long> off(R + 1, 0);
    std::vector<int> nr(R), qr(R);
    for (int i = 1; i <= R; ++i) {
        const int k = (i <= 2 * nside) ? i : 4 * nside - i;
        if (k < nside) {
            nr[i - 1] = 4 * k;
            qr[i - 1] = 1;
        } else {
            nr[i - 1] = 4 * nside;
            qr[i - 1] = ((i + nside) & 1) ? 0 : 1;
        }
        off[i] = off[i - 1] + nr[i - 1];
    }
    std::vector<RingTab> rt(np);
    std::map<int, long long> rootOff, vOff, cOff;
    std::vector<double2> roots, Vtab, chirp;
    long long nmaxF = 2;  // largest full FFT length (pow2 n or Bluestein M)
    int bmax = 2 * NAIVE_MAX, maxBlue = 1;
    for (int pr = 0; pr < np; ++pr) {
        RingTab &t = rt[pr];
        const int i0 = pr;  // north ring, 0-based
        t.n = nr[i0];
        t.q = qr[i0];
        t.offN = off[i0];
        t.offS = (pr < np - 1) ? off[R - 1 - pr] : -1;
        const int n = t.n;
        if (!rootOff.count(n)) {
            rootOff[n] = (long long)roots.size();
            for (int q = 0; q < 2 * n; ++q) {
                const double a = M_PI * (double)q / (double)n;
                roots.push_back(make_double2(std::cos(a), std::sin(a)));
            }
        }
        t.rootOff = rootOff[n];
        t.vOff = 0;
        t.cOff = 0;
        if (n <= NAIVE_MAX) {
            t.kind = RING_NAIVE;
            t.logF = 0;
        } else if (is_pow2(n)) {
            t.kind = RING_POW2;
            t.logF = ilog2(n);
            if (n > nmaxF) nmaxF = n;
            if (n > bmax) bmax = n;
        } else {
            t.kind = RING_BLUESTEIN;
            const int lgM = ilog2(2LL * n - 1);
            const long long M = 1LL << lgM;
            t.logF = lgM - 1;
            if (M > nmaxF) nmaxF = M;
            if (M / 2 > bmax) bmax = (int)(M / 2);
            if (n > maxBlue) maxBlue = n;
            if (!vOff.count(n)) {
                vOff[n] = (long long)Vtab.size();
                std::vector<double2> v(M, make_double2(0.0, 0.0));
                for (long long j = 0; j < n; ++j) {
                    const long long e = (j * j) % (2LL * n);
                    const double a = M_PI * (double)e / (double)n;  // conj(c_j) = e^{+i pi j^2 / n}
                    v[j] = make_double2(std::cos(a), std::sin(a));
                    if (j > 0) v[M - j] = v[j];
                }
                host_fft(v);
                for (long long k = 0; k < M / 2; ++k) Vtab.push_back(cscale(v[2 * k], 1.0 / (double)M));
                for (long long k = 0; k < M / 2; ++k) Vtab.push_back(cscale(v[2 * k + 1], 1.0 / (double)M));
            }
            t.vOff = vOff[n];
            if (!cOff.count(n)) {  // c_j = e^{-i pi j^2 / n}, j^2 reduced mod 2n exactly
                cOff[n] = (long long)chirp.size();
                for (long long j = 0; j < n; ++j) {
                    const double a = -M_PI * (double)((j * j) % (2LL * n)) / (double)n;
                    chirp.push_back(make_double2(std::cos(a), std::sin(a)));
                }
            }
            t.cOff = cOff[n];
        }
    }
    const int logNmax = ilog2(nmaxF);
    if (bmax > 8192) return set_error(WF_EUNSUPPORTED, "ring FFT longer than 8192 (nside > 2048)");
    std::vector<double2> tw((size_t)1 << logNmax);
    for (size_t t = 0; t < tw.size(); ++t) {
        const double a = -2.0 * M_PI * (double)t / (double)(1LL << logNmax);
        tw[t] = make_double2(std::cos(a), std::sin(a));
    }
    if (Vtab.empty()) Vtab.push_back(make_double2(0, 0));
    if (chirp.empty()) chirp.push_back(make_double2(0, 0));
    p->tab.logNmax = logNmax;
    p->tab.bmax = bmax;
    p->tab.maxBlue = maxBlue;
    wf_status st;
    if ((st = plan_alloc(p, (void **)&p->tab.rings, rt.size() * sizeof(RingTab))) != WF_OK) return st;
    if ((st = to_device(p, p->tab.rings, rt.data(), rt.size() * sizeof(RingTab))) != WF_OK) return st;
    const bool f32 = p->prec != WF_PREC_FP64;
    if (f32) {
        if ((st = upload_cx<float>(p, &p->tab.roots, roots)) != WF_OK) return st;
        if ((st = upload_cx<float>(p, &p->tab.V, Vtab)) != WF_OK) return st;
        if ((st = upload_cx<float>(p, &p->tab.chirp, chirp)) != WF_OK) return st;
        if ((st = upload_cx<float>(p, &p->tab.tw, tw)) != WF_OK) return st;
        if ((st = RingLaunch<float>::grid(p, &p->tab.ringGrid)) != WF_OK) return st;
    } else {
        if ((st = upload_cx<double>(p, &p->tab.roots, roots)) != WF_OK) return st;
        if ((st = upload_cx<double>(p, &p->tab.V, Vtab)) != WF_OK) return st;
        if ((st = upload_cx<double>(p, &p->tab.chirp, chirp)) != WF_OK) return st;
        if ((st = upload_cx<double>(p, &p->tab.tw, tw)) != WF_OK) return st;
        if ((st = RingLaunch<double>::grid(p, &p->tab.ringGrid)) != WF_OK) return st;
    }
    // pairs by decreasing cost: Bluestein (four half-length FFTs), then the rest by length
    std::vector<int> order(np);
    std::vector<double> cost(np);
    for (int i = 0; i < np; ++i) {
        order[i] = i;
        const RingTab &t = rt[i];
        const double F = (double)(1LL << t.logF);
        cost[i] = t.kind == RING_BLUESTEIN ? 4.0 * F * (t.logF + 2) : t.kind == RING_POW2 ? F * t.logF : (double)t.n * t.n / 8;
        cost[i] += 2.0 * p->lmax / 64.0;
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    if ((st = plan_alloc(p, (void **)&p->tab.order, np * sizeof(int))) != WF_OK) return st;
    if ((st = to_device(p, p->tab.order, order.data(), np * sizeof(int))) != WF_OK) return st;
    if ((st = plan_alloc(p, (void **)&p->tab.ticket, 16)) != WF_OK) return st;
    const size_t es = f32 ? sizeof(float2) : sizeof(double2);
    const long long zl = maxBlue > NAIVE_MAX ? maxBlue : NAIVE_MAX;
    return plan_alloc(p, &p->ws.scr, (size_t)p->tab.ringGrid * 2 * zl * es + 16);
}

wf_status hp_ring_synthesis(wf_plan p, int L, RingSynMode mode, double lam, double tau, double *out_map)
{
    return p->prec == WF_PREC_FP64 ? RingLaunch<double>::syn(p, L, mode, lam, tau, out_map)
                                   : RingLaunch<float>::syn(p, L, mode, lam, tau, out_map);
}

wf_status hp_ring_synthesis_analysis(wf_plan p, int L, double lam, double tau)
{
    return p->prec == WF_PREC_FP64 ? RingLaunch<double>::syn_ana(p, L, lam, tau)
                                   : RingLaunch<float>::syn_ana(p, L, lam, tau);
}

wf_status hp_ring_synthesis_buf(wf_plan p, int L, RingSynMode mode, double lam, double tau, const void *G,
                                void *tmap, double *out_map)
{
    return p->prec == WF_PREC_FP64 ? RingLaunch<double>::syn_buf(p, L, mode, lam, tau, G, tmap, out_map)
                                   : RingLaunch<float>::syn_buf(p, L, mode, lam, tau, G, tmap, out_map);
}

wf_status hp_ring_synthesis_buf_low(wf_plan p, int L, RingSynMode mode, double lam, double tau, const void *G,
                                    const float2 *glow, int lc, int glow_stride, void *tmap, double *out_map)
{
    if (p->prec == WF_PREC_FP64) return set_error(WF_EINVAL, "FP64 plans have no FP64 block");
    return RingLaunch<float>::syn_buf_low(p, L, mode, lam, tau, G, glow, lc, glow_stride, tmap, out_map);
}

wf_status hp_ring_analysis_buf(wf_plan p, int L, const void *map_T, void *F)
{
    return p->prec == WF_PREC_FP64 ? RingLaunch<double>::ana_buf(p, L, map_T, F)
                                   : RingLaunch<float>::ana_buf(p, L, map_T, F);
}

wf_status hp_ring_analysis(wf_plan p, int L, const void *map_T)
{
    return p->prec == WF_PREC_FP64 ? RingLaunch<double>::ana(p, L, map_T) : RingLaunch<float>::ana(p, L, map_T);
}

}  // namespace wf
