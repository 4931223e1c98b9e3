// Tensor-core Legendre transforms (tcgen05, sm_103a) for plans whose
// precision is WF_PREC_MIXED_TF32 or WF_PREC_MIXED_SPLITBF16: the per-m contraction of the basis change
// (Sect. 2.1; the O(nside lmax^2) cost of Sect. 3) as a dense matrix product
// on the 5th-generation tensor cores, for one or several columns (maps of one
// geometry: a solve alone, or the Wiener-filter and fluctuation solves of a
// batch that share nside, lmax and the FP64 block).
//
//   synthesis  G_c(p, m) = sum_l lambda_lm(x_p) a_c(l, m)
//              per m: D[p, n] = sum_k A[p, k] B[k, n], rows p = ring pairs,
//              k = l - m, columns n = (Re, Im) of every map c; the even and
//              odd l - m terms go to two accumulators (D_E, D_O) so that the
//              north and south rings of a pair come out as D_E +- D_O.
//
// Arithmetic ("3xTF32"): the FP32 recurrence value mu (mu form, lambda = c mu,
// c folded into B) and the FP32 value c a are each split into a TF32 head and
// an FP32 tail (x = hi + lo exactly, hi = x truncated to 10 explicit mantissa
// bits); the products hi*hi + hi*lo + lo*hi accumulate in FP32 in tensor
// memory.  The dropped lo*lo term and the tails' own truncation to TF32 are
// below 2^-20 of each product, so the contraction is as accurate as the FP32
// FMA kernels.
//
// Layout on chip (one CTA = one M = 128 tile of ring pairs, 128 threads, a
// thread per ring pair = per tensor-memory lane; 128 tensor-memory columns
// per CTA, so four CTAs share an SM and one CTA's MMA latency hides behind
// the others' recurrences):
//   tensor memory  D_E, D_O (N = NC columns each, NC = 2 ncols rounded up to
//                  16) and the A operand of the current chunk of 32 l (per
//                  parity and piece 16 TF32 or 8 packed BF16 columns); each
//                  thread writes its own lane (tcgen05.st), so the recurrence
//                  values never pass through shared memory;
//   shared memory  the B operand of the chunk (E hi, E lo, O hi, O lo; NC
//                  rows x 16 k, K-major core matrices of 8 rows x 16 bytes)
//                  and the chunk's recurrence coefficients.
// The MMAs of chunk q run while the threads compute chunk q + 1's recurrence
// in registers; the threads wait on the chunk's mbarrier (bounded) before
// they overwrite its operands.
#include <cuda_bf16.h>

#include <cstdint>
#include <cstdio>

#include "wf_internal.cuh"

namespace wf {

namespace {

constexpr int TC_THREADS = 128;   // one M = 128 tile: a thread per ring pair and tensor-memory lane
constexpr int TC_BITEMS = 4;      // B items per thread per chunk (16 columns x 32 l / 128 threads)
constexpr int TC_TMEM_COLS = 128; // D_E, D_O (nc each, nc <= 32) + the A operand (64 columns)
constexpr int TC_KC = 32;         // l values per chunk (16 even, 16 odd)
constexpr int TC_MAXC = TC_MAX_COLUMNS;  // columns (maps) per launch
constexpr float TC_X_DIFF = 0.4f; // rings with x > 0.4 run the difference form (as the FP32 kernels)
constexpr long long TC_SPIN = 1LL << 22;  // bound on every mbarrier wait (then the error flag is set)
// Chunks per tensor-memory accumulation run (temperature synthesis): the accumulators restart
// from zero every TC_FLUSH chunks and each run is added into FP32 sums in shared memory with
// round-to-nearest adds.  The tensor core adds its products into a running accumulator without that
// rounding, so a run of hundreds of chunks drifts with the size of the running sum (2.5e-5 of
// the largest value at lmax 4096, against 5e-6 for the FP32 FMA kernel).
constexpr int TC_FLUSH = 4;

__host__ __device__ inline long long tc_mbase(int lmax, int m) { return (long long)m * (2 * lmax + 3 - m) / 2; }

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor, K-major, no swizzle: 8-row x 16-byte core
// matrices; lbo = byte distance between core matrices adjacent along K,
// sbo = along M/N
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of the 5th-generation tensor cores
    return d;
}

__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_f16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                           uint32_t accumulate)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(smem_addr(mbar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// bounded wait; false (and the error flag set) if the phase did not complete
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, int *err)
{
    for (long long it = 0; it < TC_SPIN; ++it)
        if (mbar_try(mbar, parity)) return true;
    atomicOr(err, 1);
    return false;
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::
            "r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
        "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(v[0]),
                 "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

// x ~ hi + lo: hi keeps the sign, exponent and top 10 mantissa bits of x (the TF32
// head, by truncation: one logical operation); x - hi is exact in FP32 with
// |x - hi| < 2^-10 |x|, and lo is it rounded to the nearest TF32 value (an error
// below 2^-21 |x| of either sign, not a truncation towards zero), which the tensor
// core then takes exactly.
__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo)
{
    hi = __float_as_uint(x) & 0xFFFFE000u;
    lo = (__float_as_uint(x - __uint_as_float(hi)) + 0x1000u) & 0xFFFFE000u;
}

// x = b0 + b1 + b2 + (below 2^-24 |x|): three BF16 pieces by successive round-
// to-nearest of the exact FP32 remainders (8 significant bits each)
__device__ __forceinline__ void split_bf16(float x, uint16_t (&b)[3])
{
    const __nv_bfloat16 h0 = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h0);
    const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(h1);
    b[0] = __bfloat16_as_ushort(h0);
    b[1] = __bfloat16_as_ushort(h1);
    b[2] = __bfloat16_as_ushort(__float2bfloat16_rn(r2));
}

// The two arithmetic variants of the contraction.
//   KIND 0 (WF_PREC_MIXED_TF32): pieces (hi, lo) in TF32, products hi*hi + hi*lo + lo*hi.
//   KIND 1 (WF_PREC_MIXED_SPLITBF16): pieces (b0, b1, b2) in BF16, the six products of total
//     order <= 2 (b0 b0, b0 b1, b1 b0, b0 b2, b1 b1, b2 b0); the dropped terms are below
//     2^-24 of each product.
// Both take 32 bytes of K per instruction (8 TF32 or 16 BF16), i.e. 8 tensor-memory columns of
// the A operand; per chunk of 16 k per parity: 2 (TF32) or 1 (BF16) K steps.
template <int KIND> struct TcArith;
template <> struct TcArith<0> {
    static constexpr int PIECES = 2, EB = 4, KSTEPS = 2, ACOLS = 16, NPROD = 3;
    // product u: A piece pa(u) times B piece pb(u)
    __host__ __device__ static constexpr int pa(int u) { return u == 2 ? 1 : 0; }
    __host__ __device__ static constexpr int pb(int u) { return u == 1 ? 1 : 0; }
    static constexpr uint32_t FMT = 2u;  // TF32
};
template <> struct TcArith<1> {
    static constexpr int PIECES = 3, EB = 2, KSTEPS = 1, ACOLS = 8, NPROD = 6;
    __host__ __device__ static constexpr int pa(int u) { return u == 2 ? 1 : u == 4 ? 1 : u == 5 ? 2 : 0; }
    __host__ __device__ static constexpr int pb(int u) { return u == 1 ? 1 : u == 3 ? 2 : u == 4 ? 1 : 0; }
    static constexpr uint32_t FMT = 1u;  // BF16
};

// instruction descriptor: FP32 accumulator, A and B K-major, M x N, operand format fmt
__host__ __device__ constexpr uint32_t idesc_of(uint32_t fmt, int M, int N)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---------------------------------------------------------------------------
// B operand tile of a chunk: NC rows (n) x 16 k, K-major core matrices (8 rows
// x 16 bytes) with the K-direction core matrices NC/8 * 128 bytes apart
// (k-group major); eb = bytes per element
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t b_offset(int n, int k, int nc, int eb)
{
    const int t = 16 / eb;  // elements per 16 bytes
    return (uint32_t)((k / t) * (nc >> 3) * 128 + (n >> 3) * 128 + (n & 7) * 16 + (k % t) * eb);
}

struct TcSynArgs {
    int lmax, Lmax, npairs, ncols, nc;
    const float *A32, *B32;       // recurrence multipliers per a_lm (mu form), B = A - 2
    const double *c64;            // lambda = c mu
    const int *ls;                // per (m, pair): first l of the FP32 recurrence (> lmax: none)
    const float *s0, *s1;         // mu at ls and ls + 1
    const float *xp, *wp;         // per pair: x = cos theta and w = 1 - x
    const float2 *ca[TC_MAXC];    // per column: c a_lm rounded to FP32 (zero above the column's band limit)
    float2 *G[TC_MAXC];           // per column: ring coefficients [pair][m][hemisphere]
    int L[TC_MAXC];               // per column: band limit
    int *err;                     // set when a bounded wait gives up
};

// one double step (l, l + 1) of the recurrence for one ring pair (scalar form
// of the FP32 kernels' step); v0 = mu_l, v1 = mu_{l+1}
template <bool DIFF>
__device__ __forceinline__ void tc_step(float A0, float B0, float A1, float B1, float x, float w, float &Sa, float &Sb,
                                        float &v0, float &v1)
{
    if (DIFF) {
        float D = fmaf(fmaf(-A0, w, B0), Sb, Sa);
        v0 = Sb + D;
        D = fmaf(fmaf(-A1, w, B1), v0, D);
        v1 = v0 + D;
        Sa = D;
        Sb = v1;
    } else {
        v0 = fmaf(A0 * x, Sb, -Sa);
        v1 = fmaf(A1 * x, v0, -Sb);
        Sa = v0;
        Sb = v1;
    }
}

template <bool DIFF, bool INJ>
__device__ __forceinline__ void tc_chunk(int l0, int ls, float s0, float s1, float x, float w, const float4 *coef,
                                         float &Sa, float &Sb, float (&mu)[TC_KC])
{
#pragma unroll
    for (int j = 0; j < TC_KC / 2; ++j) {
        const float4 ab = coef[j];
        float v0, v1;
        tc_step<DIFF>(ab.x, ab.y, ab.z, ab.w, x, w, Sa, Sb, v0, v1);
        if (INJ && l0 + 2 * j == ls) {
            v0 = s0;
            v1 = s1;
            Sa = DIFF ? s1 - s0 : s0;
            Sb = s1;
        }
        mu[2 * j] = v0;
        mu[2 * j + 1] = v1;
    }
}

template <int KIND>
__global__ void __launch_bounds__(TC_THREADS) k_legsyn_tc(TcSynArgs P)
{
    using AR = TcArith<KIND>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int qmin_s;
    const int m = blockIdx.y;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    const int p = blockIdx.x * TC_THREADS + tid;
    const int nc = P.nc;
    const long long base = tc_mbase(P.lmax, m);
    const size_t pstride = (size_t)(P.lmax + 1) * 2;

    // this pair's seeds
    int ls = INT_MAX;
    float s0 = 0.f, s1 = 0.f, x = 0.f, w = 1.f;
    if (p < P.npairs) {
        const size_t si = (size_t)m * P.npairs + p;
        const int l = P.ls[si];
        if (l <= P.Lmax) {
            ls = l;
            s0 = P.s0[si];
            s1 = P.s1[si];
        }
        x = P.xp[p];
        w = P.wp[p];
    }
    // first chunk any pair of the CTA needs
    if (tid == 0) qmin_s = INT_MAX;
    __syncthreads();
    if (ls != INT_MAX) atomicMin(&qmin_s, (ls - m) / TC_KC);
    __syncthreads();
    const int q0 = qmin_s, q1 = (P.Lmax - m) / TC_KC;
    if (q0 > q1) {  // no pair of the CTA has a term: zero coefficients (block-uniform exit)
        if (p < P.npairs)
            for (int c = 0; c < P.ncols; ++c) {
                float2 *g = P.G[c] + (size_t)p * pstride + 2 * (size_t)m;
                *reinterpret_cast<float4 *>(g) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        return;
    }
    const bool diff = __shfl_sync(0xffffffffu, x > TC_X_DIFF ? 1 : 0, 0) != 0;  // one form per warp

    // shared B operand: 2 PIECES tiles ([parity][piece]) of nc x 16 elements, then the recurrence
    // coefficients (A_l, B_l, A_l+1, B_l+1) of every double step of the chunks this CTA runs,
    // indexed by (l - m) / 2 (zero past lmax: those terms have B = 0)
    const uint32_t btile = (uint32_t)nc * 16 * AR::EB;
    unsigned char *B = smem;
    // FP32 sums of the finished accumulation runs: entry j (D_E columns, then D_O) of thread t
    // at j * TC_THREADS + t
    float *fsum = reinterpret_cast<float *>(smem + 2 * AR::PIECES * btile);
    float4 *coef = reinterpret_cast<float4 *>(fsum + 2 * nc * TC_THREADS);
    for (int i = tid; i < (int)(2 * AR::PIECES * btile / 4); i += TC_THREADS)
        reinterpret_cast<uint32_t *>(B)[i] = 0u;  // padding rows stay zero
    for (int j = 0; j < 2 * nc; ++j) fsum[j * TC_THREADS + tid] = 0.f;
    for (int j = 16 * q0 + tid; j < 16 * (q1 + 1); j += TC_THREADS) {
        const int la = m + 2 * j, lb = la + 1;
        coef[j] = make_float4(la <= P.lmax ? P.A32[base + (la - m)] : 0.f, la <= P.lmax ? P.B32[base + (la - m)] : 0.f,
                              lb <= P.lmax ? P.A32[base + (lb - m)] : 0.f, lb <= P.lmax ? P.B32[base + (lb - m)] : 0.f);
    }
    // B values (c a of one column at one l) this thread stages: items tid and tid + 256 of a chunk
    // (ncols x 32 items), loaded one chunk ahead so that their latency hides behind the recurrence
    const int nitems = P.ncols * TC_KC;
    float2 pa[TC_BITEMS];
    auto prefetch = [&](int q) {
#pragma unroll
        for (int r = 0; r < TC_BITEMS; ++r) {
            const int it = tid + r * TC_THREADS;
            pa[r] = make_float2(0.f, 0.f);
            if (it < nitems && q <= q1) {
                const int c = it / TC_KC, l = m + TC_KC * q + it % TC_KC;
                if (l <= P.lmax) pa[r] = P.ca[c][base + (l - m)];
            }
        }
    };
    prefetch(q0);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "n"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    // columns: D_E [0, nc), D_O [nc, 2 nc); A at 2 nc, laid out [parity][piece] in blocks of
    // ACOLS columns (16 k each)
    const uint32_t dE = tmem, dO = dE + nc;
    const uint32_t aT = tmem + 2u * nc;
    const uint32_t idesc = idesc_of(AR::FMT, 128, nc);
    const uint32_t lbo = (uint32_t)(nc >> 3) * 128, sbo = 128;
    const uint32_t bsm = smem_addr(B);

    // B descriptors (loop-invariant: one operand buffer): [parity][piece][k step]
    uint64_t bdesc[2][AR::PIECES][AR::KSTEPS];
#pragma unroll
    for (int par = 0; par < 2; ++par)
#pragma unroll
        for (int h = 0; h < AR::PIECES; ++h)
#pragma unroll
            for (int s2 = 0; s2 < AR::KSTEPS; ++s2)
                bdesc[par][h][s2] =
                    smem_desc(bsm + (uint32_t)(AR::PIECES * par + h) * btile + 2 * s2 * lbo, lbo, sbo);
    // a finished run (this thread's lane of D_E and D_O) into the FP32 sums
    auto flush = [&]() {
        for (int b = 0; 16 * b < nc; ++b) {
            uint32_t e[16], o[16];
            tmem_ld16(dE + lane_base + 16 * b, e);
            tmem_ld16(dO + lane_base + 16 * b, o);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                fsum[(16 * b + j) * TC_THREADS + tid] += __uint_as_float(e[j]);
                fsum[(nc + 16 * b + j) * TC_THREADS + tid] += __uint_as_float(o[j]);
            }
        }
    };
    float Sa = 0.f, Sb = 0.f;
    bool ok = true;
    uint32_t phase = 0;
    for (int q = q0; q <= q1; ++q) {
        const int l0 = m + TC_KC * q;
        float mu[TC_KC];
        // seeds enter only in the chunk holding a lane's first l: one test per warp and chunk
        const bool inj = __any_sync(0xffffffffu, ls >= l0 && ls < l0 + TC_KC);
        if (diff) {
            if (inj) tc_chunk<true, true>(l0, ls, s0, s1, x, w, coef + 16 * q, Sa, Sb, mu);
            else tc_chunk<true, false>(l0, ls, s0, s1, x, w, coef + 16 * q, Sa, Sb, mu);
        } else {
            if (inj) tc_chunk<false, true>(l0, ls, s0, s1, x, w, coef + 16 * q, Sa, Sb, mu);
            else tc_chunk<false, false>(l0, ls, s0, s1, x, w, coef + 16 * q, Sa, Sb, mu);
        }
        // the previous chunk's MMAs have read A (tensor memory) and B (shared memory)
        if (q > q0) {
            ok = ok && mbar_wait(&mbar, phase, P.err);
            phase ^= 1u;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (q > q0 && (q - q0) % TC_FLUSH == 0) flush();  // this chunk's MMAs restart the run
#pragma unroll
        for (int par = 0; par < 2; ++par) {
            if constexpr (KIND == 0) {
                uint32_t hi[16], lo[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) split_tf32(mu[2 * j + par], hi[j], lo[j]);
                tmem_st16(aT + lane_base + 32 * par, hi);
                tmem_st16(aT + lane_base + 32 * par + 16, lo);
            } else {
                uint32_t pk[3][8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    uint16_t e0[3], e1[3];
                    split_bf16(mu[4 * j + par], e0);      // k = 2 j     (l - l0 = 4 j + par)
                    split_bf16(mu[4 * j + 2 + par], e1);  // k = 2 j + 1
#pragma unroll
                    for (int h = 0; h < 3; ++h) pk[h][j] = (uint32_t)e0[h] | ((uint32_t)e1[h] << 16);
                }
#pragma unroll
                for (int h = 0; h < 3; ++h) tmem_st8(aT + lane_base + 24 * par + 8 * h, pk[h]);
            }
        }
        // B: (c a) of every column for the chunk's 32 l, split the same way
#pragma unroll
        for (int r = 0; r < TC_BITEMS; ++r) {
            const int it = tid + r * TC_THREADS;
            if (it >= nitems) break;
            const int c = it / TC_KC, i = it % TC_KC;
            const int k = i >> 1, par = i & 1;
            const uint32_t offr = b_offset(2 * c, k, nc, AR::EB), offi = b_offset(2 * c + 1, k, nc, AR::EB);
            unsigned char *Bp = B + (size_t)(AR::PIECES * par) * btile;
            if constexpr (KIND == 0) {
                uint32_t rh, rl, ih, il;
                split_tf32(pa[r].x, rh, rl);
                split_tf32(pa[r].y, ih, il);
                *reinterpret_cast<uint32_t *>(Bp + offr) = rh;
                *reinterpret_cast<uint32_t *>(Bp + offi) = ih;
                *reinterpret_cast<uint32_t *>(Bp + btile + offr) = rl;
                *reinterpret_cast<uint32_t *>(Bp + btile + offi) = il;
            } else {
                uint16_t br[3], bi[3];
                split_bf16(pa[r].x, br);
                split_bf16(pa[r].y, bi);
#pragma unroll
                for (int h = 0; h < 3; ++h) {
                    *reinterpret_cast<uint16_t *>(Bp + h * btile + offr) = br[h];
                    *reinterpret_cast<uint16_t *>(Bp + h * btile + offi) = bi[h];
                }
            }
        }
        prefetch(q + 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t acc0 = (q > q0 && (q - q0) % TC_FLUSH != 0) ? 1u : 0u;
            {
#pragma unroll
                for (int par = 0; par < 2; ++par) {
                    const uint32_t d = dE + (par ? nc : 0);
                    const uint32_t a0 = aT + (uint32_t)(AR::PIECES * AR::ACOLS * par);
#pragma unroll
                    for (int s = 0; s < AR::KSTEPS; ++s)
#pragma unroll
                        for (int u = 0; u < AR::NPROD; ++u) {
                            const uint32_t a = a0 + AR::ACOLS * AR::pa(u) + 8 * s;
                            const uint32_t acc = (s == 0 && u == 0) ? acc0 : 1u;
                            if constexpr (KIND == 0) mma_tf32_ts(d, a, bdesc[par][AR::pb(u)][s], idesc, acc);
                            else mma_f16_ts(d, a, bdesc[par][AR::pb(u)][s], idesc, acc);
                        }
                }
            }
            mma_commit(&mbar);
        }
    }
    ok = ok && mbar_wait(&mbar, phase, P.err);
    ok = __syncthreads_and(ok) != 0;  // block-uniform: the loads below are warp-collective
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue: the last run into the sums, then G_N = E + O, G_S = E - O per column
    if (ok) {
        flush();
        if (p < P.npairs) {
            for (int c = 0; c < P.ncols; ++c) {
                {
                    const float er = fsum[(2 * c) * TC_THREADS + tid], ei = fsum[(2 * c + 1) * TC_THREADS + tid];
                    const float orr = fsum[(nc + 2 * c) * TC_THREADS + tid];
                    const float oi = fsum[(nc + 2 * c + 1) * TC_THREADS + tid];
                    float2 *g = P.G[c] + (size_t)p * pstride + 2 * (size_t)m;
                    *reinterpret_cast<float4 *>(g) = make_float4(er + orr, ei + oi, er - orr, ei - oi);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TC_TMEM_COLS)
                     : "memory");
    }
}

// c a_lm in FP32 for every column (rounded once from FP64; zero above the column's band
// limit): the B operand's source
struct TcPrepArgs {
    const double2 *a[TC_MAXC];
    float2 *ca[TC_MAXC];
    int L[TC_MAXC];
};

__global__ void k_tc_ca(int lmax, int ncols, const double *__restrict__ c64, TcPrepArgs A)
{
    const int m = blockIdx.y;
    const long long base = tc_mbase(lmax, m);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= lmax - m; j += gridDim.x * blockDim.x) {
        const double cc = c64[base + j];
        for (int c = 0; c < ncols; ++c) {
            float2 v = make_float2(0.f, 0.f);
            if (m + j <= A.L[c]) {
                const double2 a = A.a[c][base + j];
                v = make_float2((float)(a.x * cc), (float)(a.y * cc));
            }
            A.ca[c][base + j] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// Spin-2 synthesis of polarised plans on the tensor cores.  Per m the FP32
// kernels accumulate, for each ring pair and parity h of l - m,
//     Ap_h = sum A mu+,  Am_h = sum A mu-,  Cp_h = sum C mu+,  Cm_h = sum C mu-,
// A = c (E + iB), C = c (E - iB), and combine them into Q and U on the north
// and south rings.  Here those sums are two products per parity,
//     D+_h[p, n] = sum_k mu+[p, k] B_h[k, n],   D-_h[p, n] = sum_k mu-[p, k] B_h[k, n],
// with the columns n = (Re A, Im A, Re C, Im C) of every map, so four
// accumulators of nc = 4 ncols (rounded up to 16) columns, and an A operand of
// two functions x two parities per chunk.  Arithmetic, layouts, waits and
// staging as in k_legsyn_tc.
// ---------------------------------------------------------------------------
constexpr int TCP_BITEMS = 2;       // B items per thread per chunk (8 maps x 32 l / 128 threads)
constexpr int TCP_TMEM_COLS = 256;  // D+E, D+O, D-E, D-O (nc <= 32 each) + the A operand (<= 128 columns)

struct TcPolArgs {
    int lmax, Lmax, npairs, ncols, nc;
    const float4 *tab;             // per alm: (A, A be, A (1 + be) - 2, A (1 - be) - 2) of the mu+- recurrences
    const int *ls;                 // per (m, pair): first l of the FP32 recurrences (> lmax: none)
    const float4 *seed;            // per (m, pair): mu+ at ls, ls + 1; mu- at ls, ls + 1
    const float *xp, *wp;          // per pair: x = cos theta and w = 1 - x
    const float4 *ac[TCP_MAX_COLUMNS];  // per column: c (Re A, Im A, Re C, Im C) in FP32 (zero above its band limit)
    float2 *GQ[TCP_MAX_COLUMNS], *GU[TCP_MAX_COLUMNS];  // per column: ring coefficients [pair][m][hemisphere]
    int *err;                      // set when a bounded wait gives up
};

// one double step (l, l + 1) of both recurrences for one ring pair, the + and - functions in
// the two halves of packed f32x2 operations (each half is the FP32 spin-2 kernels' step, with
// the same roundings); t0, t1: the table entries of l and l + 1.  State S = (S+, S-).
template <bool DIFF>
__device__ __forceinline__ void tcp_step(float4 t0, float4 t1, float2 x2, float2 w2, float2 &Sa, float2 &Sb,
                                         float2 &V0, float2 &V1)
{
    if (DIFF) {
        float2 D = __ffma2_rn(__ffma2_rn(make_float2(-t0.x, -t0.x), w2, make_float2(t0.z, t0.w)), Sb, Sa);
        V0 = __fadd2_rn(Sb, D);
        D = __ffma2_rn(__ffma2_rn(make_float2(-t1.x, -t1.x), w2, make_float2(t1.z, t1.w)), V0, D);
        V1 = __fadd2_rn(V0, D);
        Sa = D;
        Sb = V1;
    } else {
        V0 = __ffma2_rn(__ffma2_rn(make_float2(t0.x, t0.x), x2, make_float2(t0.y, -t0.y)), Sb,
                        make_float2(-Sa.x, -Sa.y));
        V1 = __ffma2_rn(__ffma2_rn(make_float2(t1.x, t1.x), x2, make_float2(t1.y, -t1.y)), V0,
                        make_float2(-Sb.x, -Sb.y));
        Sa = V0;
        Sb = V1;
    }
}

template <bool DIFF, bool INJ>
__device__ __forceinline__ void tcp_chunk(int l0, int ls, float4 sd, float2 x2, float2 w2, const float4 *tb,
                                          float2 &Sa, float2 &Sb, float (&mup)[TC_KC], float (&mum)[TC_KC])
{
#pragma unroll
    for (int j = 0; j < TC_KC / 2; ++j) {
        float2 V0, V1;
        tcp_step<DIFF>(tb[2 * j], tb[2 * j + 1], x2, w2, Sa, Sb, V0, V1);
        if (INJ && l0 + 2 * j == ls) {
            V0 = make_float2(sd.x, sd.z);
            V1 = make_float2(sd.y, sd.w);
            Sa = DIFF ? make_float2(sd.y - sd.x, sd.w - sd.z) : V0;
            Sb = V1;
        }
        mup[2 * j] = V0.x;
        mup[2 * j + 1] = V1.x;
        mum[2 * j] = V0.y;
        mum[2 * j + 1] = V1.y;
    }
}

template <int KIND>
__global__ void __launch_bounds__(TC_THREADS) k_legsyn_pol_tc(TcPolArgs P)
{
    using AR = TcArith<KIND>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int qmin_s;
    const int m = blockIdx.y;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    const int p = blockIdx.x * TC_THREADS + tid;
    const int nc = P.nc;
    const long long base = tc_mbase(P.lmax, m);
    const size_t pstride = (size_t)(P.lmax + 1) * 2;

    int ls = INT_MAX;
    float4 sd = make_float4(0.f, 0.f, 0.f, 0.f);
    float x = 0.f, w = 1.f;
    if (p < P.npairs) {
        const size_t si = (size_t)m * P.npairs + p;
        const int l = P.ls[si];
        if (l <= P.Lmax) {
            ls = l;
            sd = P.seed[si];
        }
        x = P.xp[p];
        w = P.wp[p];
    }
    if (tid == 0) qmin_s = INT_MAX;
    __syncthreads();
    if (ls != INT_MAX) atomicMin(&qmin_s, (ls - m) / TC_KC);
    __syncthreads();
    const int q0 = qmin_s, q1 = (P.Lmax - m) / TC_KC;
    if (q0 > q1) {  // no pair of the CTA has a term (block-uniform exit)
        if (p < P.npairs)
            for (int c = 0; c < P.ncols; ++c) {
                const size_t o = (size_t)p * pstride + 2 * (size_t)m;
                *reinterpret_cast<float4 *>(P.GQ[c] + o) = make_float4(0.f, 0.f, 0.f, 0.f);
                *reinterpret_cast<float4 *>(P.GU[c] + o) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        return;
    }
    const bool diff = __shfl_sync(0xffffffffu, x > TC_X_DIFF ? 1 : 0, 0) != 0;

    // shared: the B tiles ([parity][piece], nc x 16 k each), then the recurrence table of every l
    // of the chunks this CTA runs, indexed by l - m (zero past lmax)
    const uint32_t btile = (uint32_t)nc * 16 * AR::EB;
    unsigned char *B = smem;
    float4 *tb = reinterpret_cast<float4 *>(smem + 2 * AR::PIECES * btile);
    for (int i = tid; i < (int)(2 * AR::PIECES * btile / 4); i += TC_THREADS) reinterpret_cast<uint32_t *>(B)[i] = 0u;
    for (int j = TC_KC * q0 + tid; j < TC_KC * (q1 + 1); j += TC_THREADS)
        tb[j] = m + j <= P.lmax ? P.tab[base + j] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int nitems = P.ncols * TC_KC;
    float4 pa[TCP_BITEMS];
    auto prefetch = [&](int q) {
#pragma unroll
        for (int r = 0; r < TCP_BITEMS; ++r) {
            const int it = tid + r * TC_THREADS;
            pa[r] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (it < nitems && q <= q1) {
                const int c = it / TC_KC, l = m + TC_KC * q + it % TC_KC;
                if (l <= P.lmax) pa[r] = P.ac[c][base + (l - m)];
            }
        }
    };
    prefetch(q0);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "n"(TCP_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    // columns: D+ E, D+ O, D- E, D- O (nc each); A at 4 nc, laid out [function][parity][piece] in
    // blocks of ACOLS columns
    const uint32_t dP = tmem, dM = tmem + 2u * nc;
    const uint32_t aT = tmem + 4u * nc;
    const uint32_t idesc = idesc_of(AR::FMT, 128, nc);
    const uint32_t lbo = (uint32_t)(nc >> 3) * 128, sbo = 128;
    const uint32_t bsm = smem_addr(B);
    uint64_t bdesc[2][AR::PIECES][AR::KSTEPS];
#pragma unroll
    for (int par = 0; par < 2; ++par)
#pragma unroll
        for (int h = 0; h < AR::PIECES; ++h)
#pragma unroll
            for (int s2 = 0; s2 < AR::KSTEPS; ++s2)
                bdesc[par][h][s2] =
                    smem_desc(bsm + (uint32_t)(AR::PIECES * par + h) * btile + 2 * s2 * lbo, lbo, sbo);
    float2 Sa = make_float2(0.f, 0.f), Sb = make_float2(0.f, 0.f);
    const float2 x2 = make_float2(x, x), w2 = make_float2(w, w);
    bool ok = true;
    uint32_t phase = 0;
    for (int q = q0; q <= q1; ++q) {
        const int l0 = m + TC_KC * q;
        float mup[TC_KC], mum[TC_KC];
        const bool inj = __any_sync(0xffffffffu, ls >= l0 && ls < l0 + TC_KC);
        const float4 *tq = tb + TC_KC * q;
        if (diff) {
            if (inj) tcp_chunk<true, true>(l0, ls, sd, x2, w2, tq, Sa, Sb, mup, mum);
            else tcp_chunk<true, false>(l0, ls, sd, x2, w2, tq, Sa, Sb, mup, mum);
        } else {
            if (inj) tcp_chunk<false, true>(l0, ls, sd, x2, w2, tq, Sa, Sb, mup, mum);
            else tcp_chunk<false, false>(l0, ls, sd, x2, w2, tq, Sa, Sb, mup, mum);
        }
        if (q > q0) {
            ok = ok && mbar_wait(&mbar, phase, P.err);
            phase ^= 1u;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int fn = 0; fn < 2; ++fn) {
            const float(&mu)[TC_KC] = fn ? mum : mup;
#pragma unroll
            for (int par = 0; par < 2; ++par) {
                const uint32_t blk = aT + lane_base + (uint32_t)((2 * fn + par) * AR::PIECES * AR::ACOLS);
                if constexpr (KIND == 0) {
                    uint32_t hi[16], lo[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) split_tf32(mu[2 * j + par], hi[j], lo[j]);
                    tmem_st16(blk, hi);
                    tmem_st16(blk + 16, lo);
                } else {
                    uint32_t pk[3][8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        uint16_t e0[3], e1[3];
                        split_bf16(mu[4 * j + par], e0);
                        split_bf16(mu[4 * j + 2 + par], e1);
#pragma unroll
                        for (int h = 0; h < 3; ++h) pk[h][j] = (uint32_t)e0[h] | ((uint32_t)e1[h] << 16);
                    }
#pragma unroll
                    for (int h = 0; h < 3; ++h) tmem_st8(blk + 8 * h, pk[h]);
                }
            }
        }
        // B: the four coefficient rows of every column for the chunk's 32 l, split the same way
#pragma unroll
        for (int r = 0; r < TCP_BITEMS; ++r) {
            const int it = tid + r * TC_THREADS;
            if (it >= nitems) break;
            const int c = it / TC_KC, i = it % TC_KC;
            const int k = i >> 1, par = i & 1;
            unsigned char *Bp = B + (size_t)(AR::PIECES * par) * btile;
            const float v[4] = {pa[r].x, pa[r].y, pa[r].z, pa[r].w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const uint32_t off = b_offset(4 * c + e, k, nc, AR::EB);
                if constexpr (KIND == 0) {
                    uint32_t h0, h1;
                    split_tf32(v[e], h0, h1);
                    *reinterpret_cast<uint32_t *>(Bp + off) = h0;
                    *reinterpret_cast<uint32_t *>(Bp + btile + off) = h1;
                } else {
                    uint16_t b3[3];
                    split_bf16(v[e], b3);
#pragma unroll
                    for (int h = 0; h < 3; ++h) *reinterpret_cast<uint16_t *>(Bp + h * btile + off) = b3[h];
                }
            }
        }
        prefetch(q + 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t acc0 = q > q0 ? 1u : 0u;
#pragma unroll
            for (int fn = 0; fn < 2; ++fn)
#pragma unroll
                for (int par = 0; par < 2; ++par) {
                    const uint32_t d = (fn ? dM : dP) + (par ? nc : 0);
                    const uint32_t a0 = aT + (uint32_t)((2 * fn + par) * AR::PIECES * AR::ACOLS);
#pragma unroll
                    for (int s2 = 0; s2 < AR::KSTEPS; ++s2)
#pragma unroll
                        for (int u = 0; u < AR::NPROD; ++u) {
                            const uint32_t a = a0 + AR::ACOLS * AR::pa(u) + 8 * s2;
                            const uint32_t acc = (s2 == 0 && u == 0) ? acc0 : 1u;
                            if constexpr (KIND == 0) mma_tf32_ts(d, a, bdesc[par][AR::pb(u)][s2], idesc, acc);
                            else mma_f16_ts(d, a, bdesc[par][AR::pb(u)][s2], idesc, acc);
                        }
                }
            mma_commit(&mbar);
        }
    }
    ok = ok && mbar_wait(&mbar, phase, P.err);
    ok = __syncthreads_and(ok) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue, four columns (16 tensor-memory columns) per pass:
    //   north: SAP = Ap_E + Ap_O, SCM = Cm_E + Cm_O;  south: SAP = Am_E - Am_O, SCM = Cp_E - Cp_O;
    //   Q = -(SAP + SCM),  U = i (SAP - SCM)
    if (ok) {
        for (int c0 = 0; c0 < P.ncols; c0 += 4) {
            uint32_t pe[16], po[16], me[16], mo[16];
            tmem_ld16(dP + lane_base + 4 * c0, pe);
            tmem_ld16(dP + nc + lane_base + 4 * c0, po);
            tmem_ld16(dM + lane_base + 4 * c0, me);
            tmem_ld16(dM + nc + lane_base + 4 * c0, mo);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (p < P.npairs) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int c = c0 + j;
                    if (c < P.ncols) {
                        auto f = [&](const uint32_t(&v)[16], int e) { return __uint_as_float(v[4 * j + e]); };
                        const float sapNr = f(pe, 0) + f(po, 0), sapNi = f(pe, 1) + f(po, 1);
                        const float scmNr = f(me, 2) + f(mo, 2), scmNi = f(me, 3) + f(mo, 3);
                        const float sapSr = f(me, 0) - f(mo, 0), sapSi = f(me, 1) - f(mo, 1);
                        const float scmSr = f(pe, 2) - f(po, 2), scmSi = f(pe, 3) - f(po, 3);
                        const size_t o = (size_t)p * pstride + 2 * (size_t)m;
                        *reinterpret_cast<float4 *>(P.GQ[c] + o) =
                            make_float4(-(sapNr + scmNr), -(sapNi + scmNi), -(sapSr + scmSr), -(sapSi + scmSi));
                        *reinterpret_cast<float4 *>(P.GU[c] + o) =
                            make_float4(-(sapNi - scmNi), sapNr - scmNr, -(sapSi - scmSi), sapSr - scmSr);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TCP_TMEM_COLS)
                     : "memory");
    }
}

// c (Re A, Im A, Re C, Im C) with A = E + iB, C = E - iB, in FP32 for every column (zero above the
// column's band limit): the polarised B operand's source
struct TcPolPrepArgs {
    const double2 *E[TCP_MAX_COLUMNS], *B[TCP_MAX_COLUMNS];
    float4 *ac[TCP_MAX_COLUMNS];
    int L[TCP_MAX_COLUMNS];
};

__global__ void k_tcp_ac(int lmax, int ncols, const double *__restrict__ c, TcPolPrepArgs A)
{
    const int m = blockIdx.y;
    const long long base = tc_mbase(lmax, m);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= lmax - m; j += gridDim.x * blockDim.x) {
        const double cc = c[base + j];
        for (int k = 0; k < ncols; ++k) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (m + j <= A.L[k]) {
                const double2 e = A.E[k][base + j], b = A.B[k][base + j];
                v = make_float4((float)((e.x - b.y) * cc), (float)((e.y + b.x) * cc), (float)((e.x + b.y) * cc),
                                (float)((e.y - b.x) * cc));
            }
            A.ac[k][base + j] = v;
        }
    }
}

}  // namespace

// B tiles (the larger of the two variants: 4 x 64 or 6 x 32 bytes per row), the run sums, and the
// coefficient table of up to L / 32 + 1 chunks
size_t tc_syn_smem(int nc, int L)
{
    return (size_t)4 * nc * 64 + (size_t)2 * nc * TC_THREADS * 4 + (size_t)16 * 16 * (L / TC_KC + 1) + 64;
}

// polarised: B tiles (nc <= 32) plus one table entry per l of up to L / 32 + 1 chunks
size_t tcp_syn_smem(int nc, int L) { return (size_t)4 * nc * 64 + (size_t)16 * TC_KC * (L / TC_KC + 1) + 64; }

// raise the synthesis kernels' shared-memory limits for plans up to lmax (at plan creation,
// outside any stream capture)
wf_status tc_prepare(int lmax)
{
    wf_status st = raise_smem_limit((const void *)k_legsyn_tc<0>, tc_syn_smem(32, lmax));
    if (st == WF_OK) st = raise_smem_limit((const void *)k_legsyn_tc<1>, tc_syn_smem(32, lmax));
    if (st == WF_OK) st = raise_smem_limit((const void *)k_legsyn_pol_tc<0>, tcp_syn_smem(32, lmax));
    if (st == WF_OK) st = raise_smem_limit((const void *)k_legsyn_pol_tc<1>, tcp_syn_smem(32, lmax));
    return st;
}

// Synthesis of ncols columns sharing p's geometry and FP32 seeds (every
// column's plan has p's nside, lmax and FP64 block): one launch on `stream`,
// counted on p.
wf_status hp_tc_synthesis(wf_plan p, int ncols, const double2 *const *a, float2 *const *ca, float2 *const *G,
                          const int *L, int Lmax, cudaStream_t stream)
{
    if (ncols < 1 || ncols > TC_MAXC) return set_error(WF_EINVAL, "tensor-core synthesis: 1..%d columns", TC_MAXC);
    const HpTables &t = p->tab;
    {
        TcPrepArgs pa{};
        for (int c = 0; c < ncols; ++c) {
            pa.a[c] = a[c];
            pa.ca[c] = ca[c];
            pa.L[c] = L[c];
        }
        dim3 g((Lmax + 256) / 256, Lmax + 1);
        k_tc_ca<<<g, 256, 0, stream>>>(p->lmax, ncols, t.c64, pa);
        WF_COUNT_LAUNCH(p);
        WF_CUDA(cudaGetLastError());
    }
    TcSynArgs A{};
    A.lmax = p->lmax;
    A.Lmax = Lmax;
    A.npairs = p->npairs;
    A.ncols = ncols;
    A.nc = ((2 * ncols + 15) / 16) * 16;
    A.A32 = t.A32;
    A.B32 = t.B32;
    A.c64 = t.c64;
    A.ls = t.ls_mx;
    A.s0 = t.s0_mx;
    A.s1 = t.s1_mx;
    A.xp = t.x32;
    A.wp = t.w32;
    for (int c = 0; c < ncols; ++c) {
        A.ca[c] = ca[c];
        A.G[c] = G[c];
        A.L[c] = L[c];
    }
    A.err = p->ws.tc_err;
    const size_t sm = tc_syn_smem(A.nc, Lmax);  // the limit is raised at plan creation (tc_prepare)
    dim3 grid((p->npairs + TC_THREADS - 1) / TC_THREADS, Lmax + 1);
    if (p->prec == WF_PREC_MIXED_SPLITBF16) k_legsyn_tc<1><<<grid, TC_THREADS, sm, stream>>>(A);
    else k_legsyn_tc<0><<<grid, TC_THREADS, sm, stream>>>(A);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    return WF_OK;
}

// Spin-2 synthesis of ncols polarised columns sharing p's geometry and FP32 seeds (every
// column's plan has p's nside, lmax and spin-2 FP64 block): one launch on `stream`, counted on p.
wf_status hp_pol_tc_synthesis(wf_plan p, int ncols, const double2 *const *E, const double2 *const *B,
                              float4 *const *ac, float2 *const *GQ, float2 *const *GU, const int *L, int Lmax,
                              cudaStream_t stream)
{
    if (ncols < 1 || ncols > TCP_MAX_COLUMNS)
        return set_error(WF_EINVAL, "polarised tensor-core synthesis: 1..%d columns", TCP_MAX_COLUMNS);
    const PolState *s = p->pol;
    const HpTables &t = p->tab;
    {
        TcPolPrepArgs pa{};
        for (int c = 0; c < ncols; ++c) {
            pa.E[c] = E[c];
            pa.B[c] = B[c];
            pa.ac[c] = ac[c];
            pa.L[c] = L[c];
        }
        dim3 g((Lmax + 256) / 256, Lmax + 1);
        k_tcp_ac<<<g, 256, 0, stream>>>(p->lmax, ncols, s->c, pa);
        WF_COUNT_LAUNCH(p);
        WF_CUDA(cudaGetLastError());
    }
    TcPolArgs A{};
    A.lmax = p->lmax;
    A.Lmax = Lmax;
    A.npairs = p->npairs;
    A.ncols = ncols;
    A.nc = ((4 * ncols + 15) / 16) * 16;
    A.tab = s->tab;
    A.ls = s->ls_mx;
    A.seed = s->seed;
    A.xp = t.x32;
    A.wp = t.w32;
    for (int c = 0; c < ncols; ++c) {
        A.ac[c] = ac[c];
        A.GQ[c] = GQ[c];
        A.GU[c] = GU[c];
    }
    A.err = p->ws.tc_err;
    const size_t sm = tcp_syn_smem(A.nc, Lmax);  // the limit is raised at plan creation (tc_prepare)
    dim3 grid((p->npairs + TC_THREADS - 1) / TC_THREADS, Lmax + 1);
    if (p->prec == WF_PREC_MIXED_SPLITBF16) k_legsyn_pol_tc<1><<<grid, TC_THREADS, sm, stream>>>(A);
    else k_legsyn_pol_tc<0><<<grid, TC_THREADS, sm, stream>>>(A);
    WF_COUNT_LAUNCH(p);
    WF_CUDA(cudaGetLastError());
    return WF_OK;
}

}  // namespace wf
