// Restart / output basis update of Alg. 2 (the restart and the final
// output of the svds-C paper): C (rows x k) = W (rows x t) Q (t x k), W tall and skinny, on the
// 5th-generation tensor cores (tcgen05.mma, accumulators in TMEM).
//
// Operands are cut into BF16 "slices" and the slice pairs that matter are
// multiplied on the tensor cores with FP32 accumulation:
//   * FP64 form (Ozaki-style error-free splitting, Ozaki et al. 2012): each row
//     of W and each column of Q is scaled by a power of two, its fixed-point
//     value (54 bits) is cut into S = 8 balanced base-128 digits in [-64, 63],
//     built directly as BF16 bit patterns, and the 36 digit products with
//     s + s' <= 7 are summed in 8 TMEM accumulators, one per digit weight
//     g = s + s'.  Every accumulator holds an integer below 8 * 448 * 64^2 <
//     2^24 (t <= 448), so the FP32 tensor-core sums are exact; the epilogue
//     recombines the 8 integers exactly in two int64 groups and rounds once to
//     FP64.  The dropped products (s + s' >= 8) and the truncation below
//     2^-54 of each row's or column's scale bound the error by about
//     2^-49 max|W(r,:)| max|Q(:,j)| per term of the K sum in the worst case
//     (random signs: far less; inside 8 eps sum |W||Q| + 2^-47 max max in the
//     parity tests).
//   * mixed form: W (FP32 shadow) and Q are cut into 3 floating BF16 pieces
//     (hi, mid, lo: 24 bits) and the 6 products with s + s' <= 4 accumulate in
//     one FP32 accumulator.
// A CTA owns 128 rows x NT columns of C; the K dimension (t) streams through a
// two-stage shared-memory pipeline of 32-wide chunks: the CTA's threads cut the
// next chunk into slices while the tensor cores multiply the current one.
// C must not alias W (the caller ping-pongs two bases).
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>
#include "internal.cuh"

namespace svdsc {

// ------------------------------------------------------------------ PTX

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(1000u)  // suspend at most ~1 us per try
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after 2^22 polls (each try_wait suspends for at most
// ~1 us, so ~4 s in all) and reports the timeout instead of hanging.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    for (uint32_t i = 0; i < (1u << 22); i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared on the TMA engine; completion counted in bytes
// on `bar` (dst, src 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor, K-major operand without swizzling: core
// matrices of 8 rows x 16 bytes stored contiguously (128 B); lbo = byte
// distance between core matrices adjacent along K, sbo = along M/N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor of kind::f16: BF16 A and B, FP32 D, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ------------------------------------------------------------- geometry
constexpr int kTM = 128;        // rows per CTA (MMA M)
constexpr int kKC = 32;         // K chunk per pipeline stage
constexpr int kCutThreads = 512;             // cutters: four threads per row of the tile
constexpr int kThreads = kCutThreads + 32;   // + one warp that issues the MMAs
constexpr int kTPR = kCutThreads / kTM;      // threads per row
constexpr int kGPT = (kKC / 8) / kTPR;       // groups of 8 K entries each thread cuts per chunk
static_assert(kGPT >= 1 && kGPT * kTPR * 8 == kKC, "chunk split");
constexpr int kMaxT = 448;      // exactness bound of the FP64 form

template <int S, int NT>
struct TileCfg {
    static constexpr int a_slice_bytes = kTM * kKC * 2;          // 8 KB
    static constexpr int b_slice_bytes = NT * kKC * 2;
    static constexpr int a_bytes = S * a_slice_bytes;
    static constexpr int b_bytes = S * b_slice_bytes;
    static constexpr int stage_bytes = a_bytes + b_bytes;
    static constexpr int smem_bytes = 2 * stage_bytes + 1024;    // + alignment slack
};

// byte offset of element (row, kk) inside one K-major no-swizzle slice of
// `rows` rows and kKC columns: [kgroup][rowgroup][8 rows][8 elements]
__host__ __device__ __forceinline__ int core_off(int row, int kk, int rows)
{
    return ((kk >> 3) * (rows >> 3) + (row >> 3)) * 128 + (row & 7) * 16 + (kk & 7) * 2;
}

// ------------------------------------------------------------ slicing
// FP64 form: x = sum_{s=0..7} d_s 2^(e - 5 - 7 s) up to a truncation below
// 2^(e - 54), with balanced base-128 digits d_s in [-64, 63] and e the row (or
// column) exponent with max |x| < 2^e.  (Eight balanced digits reach
// 63 (128^8 - 1) / 127 ~ 0.99 * 2^55; the fixed-point value stays below 2^54.)
__device__ __forceinline__ int dexp_of(double v)
{
    const uint64_t b = (uint64_t)__double_as_longlong(v);
    const int E = (int)((b >> 52) & 0x7FF);
    return E == 0 ? -100000 : E - 1022;  // |v| < 2^(E-1022); zero/denormal ignored
}

constexpr int kDigits = 8;
// 64 * sum_{s<8} 128^s: adding it makes every base-128 digit of F + bias equal
// d_s + 64 (in [0, 127]) for the balanced digits d_s of F, |F| < 2^54
constexpr int64_t kDigitBias = 64ll * (((1ll << 56) - 1) / 127);

// The FP32 bit patterns of d_s (their high halves are the exact BF16 values:
// |d_s| <= 64 has at most 7 significant bits).  Integer ops and one FP32 add
// per digit, no conversion instructions: float(2^23 + u) - (2^23 + 64) = u - 64.
__device__ __forceinline__ void ozaki_digits(double v, int e, uint32_t (&bits)[kDigits])
{
    const uint64_t b = (uint64_t)__double_as_longlong(v);
    const int E = (int)((b >> 52) & 0x7FF);
    int64_t F = 0;
    if (E != 0) {
        const uint64_t mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int sh = e - (E - 1022);   // >= 0 since |v| < 2^e
        F = sh >= 54 ? 0 : (int64_t)((mant << 1) >> sh);  // |v| 2^(54 - e), < 2^54
        if (b >> 63) F = -F;
    }
    const uint64_t G = (uint64_t)(F + kDigitBias);
#pragma unroll
    for (int s = 0; s < kDigits; s++) {
        const uint32_t u = (uint32_t)(G >> (7 * (kDigits - 1 - s))) & 127u;
        bits[s] = __float_as_uint(__uint_as_float(0x4B000000u | u) - 8388672.0f);
    }
}

// round(Z 2^(E - 59)) for the exact integer Z = zh 2^28 + zl (|zh|, |zl| < 2^46),
// to nearest even, assembled from integer ops (the FP64 pipe is GB300's
// scarcest); false when the result is not a normal FP64 number.
__device__ __forceinline__ bool compose_f64(long long zh, long long zl, int E, double &out)
{
    const __int128 Z = ((__int128)zh << 28) + (__int128)zl;
    if (Z == 0) { out = 0.0; return true; }
    const bool neg = Z < 0;
    const unsigned __int128 M = neg ? (unsigned __int128)(-Z) : (unsigned __int128)Z;
    const uint64_t hi = (uint64_t)(M >> 64), lo = (uint64_t)M;
    const int p = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);  // leading bit
    int ex = p + E - 59 + 1023;
    uint64_t mant;
    if (p <= 52) {
        mant = lo << (52 - p);
    } else {
        const int sh = p - 52;  // 1 .. 75
        mant = (uint64_t)(M >> sh);
        const unsigned __int128 rem = M & (((unsigned __int128)1 << sh) - 1);
        const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
        if (rem > half || (rem == half && (mant & 1ull))) {
            mant++;
            if (mant >> 53) { mant >>= 1; ex++; }
        }
    }
    if (ex <= 0 || ex >= 2047) return false;
    out = __longlong_as_double((long long)(((uint64_t)neg << 63) | ((uint64_t)ex << 52) |
                                           (mant & ((1ull << 52) - 1))));
    return true;
}

// mixed form: x = hi + mid + lo, each a BF16 number (24 significant bits)
__device__ __forceinline__ void float_pieces(float x, float (&p)[3])
{
    const float h = __bfloat162float(__float2bfloat16_rn(x));
    const float r1 = x - h;
    const float m = __bfloat162float(__float2bfloat16_rn(r1));
    const float r2 = r1 - m;
    p[0] = h;
    p[1] = m;
    p[2] = __bfloat162float(__float2bfloat16_rn(r2));
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    const uint32_t lo = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a));
    const uint32_t hi = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b));
    return lo | (hi << 16);
}

// ------------------------------------------------------------- B prep
// Q (t x k, FP64) -> slices in the exact shared-memory layout each CTA copies:
// Bs[(cb * nchunks + chunk) * S + s][NT x kKC core layout]; column exponents fexp[k].
template <int S, int NT, bool OZAKI>
__global__ void prep_b_kernel(const double *__restrict__ Q, int64_t ldq, int t, int k, int nchunks,
                              int ncb, uint16_t *__restrict__ Bs, int *__restrict__ fexp)
{
    // one thread per (column j of the padded column space, chunk)
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int chunk = blockIdx.y;
    if (j >= ncb * NT) return;
    const int cb = j / NT, jn = j % NT;
    int e = -100000;
    if (OZAKI && j < k)
        for (int c = 0; c < t; c++) e = max(e, dexp_of(Q[c + (int64_t)j * ldq]));
    if (OZAKI && chunk == 0 && j < k) fexp[j] = e;
    for (int kk = 0; kk < kKC; kk++) {
        const int c = chunk * kKC + kk;
        const double q = (j < k && c < t) ? Q[c + (int64_t)j * ldq] : 0.0;
        uint16_t pieces[S];
        if constexpr (OZAKI) {
            uint32_t d[kDigits];
            ozaki_digits(q, e, d);
#pragma unroll
            for (int s = 0; s < S; s++) pieces[s] = (uint16_t)(d[s] >> 16);
        } else {
            float p3[3];
            float_pieces((float)q, p3);
#pragma unroll
            for (int s = 0; s < S; s++) pieces[s] = __bfloat16_as_ushort(__float2bfloat16_rn(p3[s]));
        }
#pragma unroll
        for (int s = 0; s < S; s++) {
            uint16_t *dst = Bs + ((int64_t)(cb * nchunks + chunk) * S + s) * (NT * kKC);
            dst[core_off(jn, kk, NT) / 2] = pieces[s];
        }
    }
}

// ------------------------------------------------------------- main kernel
// G accumulators of NT columns: OZAKI -> one per digit weight g = s + s' <= 7
// (G = 8, 36 digit products), else a single one.  C = W Q for rows
// [128 tile, +128) and columns [NT cb, +NT).
template <int S, int NT, bool OZAKI, typename WT>
__global__ void __launch_bounds__(kThreads, 1)
tc_gemm_kernel(const WT *__restrict__ W, int64_t ldw, int64_t rows, int t, int k,
               const uint16_t *__restrict__ Bs, const int *__restrict__ fexp, int nchunks, int ncb,
               double *__restrict__ C, int64_t ldc, float *__restrict__ C32, int *err)
{
    constexpr int G = OZAKI ? 8 : 1;            // accumulators
    constexpr int kMaxSum = OZAKI ? 7 : S - 1;  // kept pairs: s + s2 <= kMaxSum (0-based)
    static_assert(!OZAKI || S == kDigits, "digit count");
    constexpr uint32_t kTmemCols = (G * NT <= 32) ? 32 : (G * NT <= 64) ? 64 : (G * NT <= 128) ? 128
                                   : (G * NT <= 256) ? 256 : 512;
    static_assert(G * NT <= 512, "TMEM capacity");
    using Cfg = TileCfg<S, NT>;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    // per stage: A slices written (one arrival per cutter warp), B slices
    // landed (bulk copy bytes), MMAs that read the stage done (tcgen05.commit)
    __shared__ uint64_t a_full[2], b_full[2], mma_done[2];
    __shared__ uint32_t tmem_base_slot;
    __shared__ int s_er[kTM];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool cutter = tid < kCutThreads;
    const int trow = tid & (kTM - 1), part = tid >> 7;  // cutters: part in [0, kTPR)
    // the column blocks of one row tile are adjacent in launch order, so the
    // tile's rows of W are re-read from L2 rather than DRAM
    const int64_t tile = (int64_t)blockIdx.x / ncb;
    const int cb = (int)(blockIdx.x % ncb);
    const int64_t row0 = tile * kTM;
    const int64_t r = row0 + trow;
    const bool row_ok = cutter && r < rows;

    if (tid == 0) {
        for (int i = 0; i < 2; i++) {
            mbar_init(&a_full[i], kCutThreads / 32);
            mbar_init(&b_full[i], 1);
            mbar_init(&mma_done[i], 1);
        }
        fence_barrier_init();
    }
    if (warp == 0) {
        tmem_alloc(&tmem_base_slot, kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_slot;

    // row exponent (FP64 form): each part scans every kTPR-th column
    int e_r = -100000;
    if (OZAKI) {
        int e_h = -100000;
        if (row_ok)
            for (int c = part; c < t; c += kTPR) e_h = max(e_h, dexp_of((double)W[r + (int64_t)c * ldw]));
        if (cutter && part == 0) s_er[trow] = -100000;
        __syncthreads();
        if (cutter) atomicMax(&s_er[trow], e_h);
        __syncthreads();
        e_r = cutter ? s_er[trow] : 0;
    }

    uint32_t parity[2] = {0u, 0u};
    bool used[2] = {false, false};
    bool ok = true;
    if (!cutter) {
        // MMA warp, one thread: stage free -> bulk copy of the B slices ->
        // A slices written and B landed -> 36 (FP64) or 6 (mixed) products per
        // 16-wide K step -> commit
        if (lane == 0) {
            uint32_t apar[2] = {0u, 0u}, bpar[2] = {0u, 0u};
            for (int chunk = 0; chunk < nchunks; chunk++) {
                const int st = chunk & 1;
                uint8_t *A = smem + st * Cfg::stage_bytes;
                uint8_t *B = A + Cfg::a_bytes;
                if (used[st]) {
                    if (!mbar_wait_bounded(&mma_done[st], parity[st])) ok = false;
                    parity[st] ^= 1u;
                }
                mbar_expect_tx(&b_full[st], (uint32_t)Cfg::b_bytes);
                bulk_g2s(B, Bs + (int64_t)(cb * nchunks + chunk) * S * (NT * kKC), (uint32_t)Cfg::b_bytes,
                         &b_full[st]);
                if (!mbar_wait_bounded(&a_full[st], apar[st])) ok = false;
                apar[st] ^= 1u;
                if (!mbar_wait_bounded(&b_full[st], bpar[st])) ok = false;
                bpar[st] ^= 1u;
                tc_fence_after();
                if (ok) {
                    constexpr uint32_t idesc = idesc_bf16(kTM, NT);
                    const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
                    constexpr uint32_t a_lbo = (kTM / 8) * 128, a_sbo = 128;
                    constexpr uint32_t b_lbo = (NT / 8) * 128, b_sbo = 128;
#pragma unroll
                    for (int ks = 0; ks < kKC / 16; ks++) {
#pragma unroll
                        for (int s = 0; s < S; s++) {
#pragma unroll
                            for (int s2 = 0; s2 < S; s2++) {
                                if (s + s2 > kMaxSum) continue;
                                const int g = OZAKI ? (s + s2) : 0;
                                const uint64_t ad =
                                    smem_desc(a0 + s * Cfg::a_slice_bytes + ks * 2 * a_lbo, a_lbo, a_sbo);
                                const uint64_t bd =
                                    smem_desc(b0 + s2 * Cfg::b_slice_bytes + ks * 2 * b_lbo, b_lbo, b_sbo);
                                // the first product into each accumulator overwrites it:
                                // group g = s + s2 is first reached at s = max(0, g - (S - 1))
                                const int s_first = (OZAKI && g > S - 1) ? g - (S - 1) : 0;
                                const bool first = chunk == 0 && ks == 0 && s == s_first && (OZAKI || s2 == 0);
                                umma_bf16(tmem + (uint32_t)(g * NT), ad, bd, idesc, first ? 0u : 1u);
                            }
                        }
                    }
                }
                // (after a failed wait the commit arrives with no MMAs: the
                // stage is released and the error surfaces through `ok`)
                umma_commit(&mma_done[st]);
                used[st] = true;
            }
        }
        __syncwarp();  // reconverge before the block-wide barrier
    } else {
        // cutters: this thread's W entries of a chunk are its row, K groups
        // kg = kGPT part + kh; the next chunk's load while this one is cut
        double cur[kGPT][8], nxt[kGPT][8];
        auto load_chunk = [&](int chunk, double (&dst)[kGPT][8]) {
#pragma unroll
            for (int kh = 0; kh < kGPT; kh++)
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const int c = chunk * kKC + (part * kGPT + kh) * 8 + q;
                    dst[kh][q] = (row_ok && c < t) ? (double)W[r + (int64_t)c * ldw] : 0.0;
                }
        };
        load_chunk(0, cur);
        for (int chunk = 0; chunk < nchunks; chunk++) {
            if (chunk + 1 < nchunks) load_chunk(chunk + 1, nxt);
            const int st = chunk & 1;
            uint8_t *A = smem + st * Cfg::stage_bytes;
            if (used[st]) {  // the MMAs that read this stage two chunks ago must be done
                if (!mbar_wait_bounded(&mma_done[st], parity[st])) ok = false;
                parity[st] ^= 1u;
            }
            tc_fence_after();
#pragma unroll
            for (int kh = 0; kh < kGPT; kh++) {
                const int kg = part * kGPT + kh;
                const double *vals = cur[kh];
                const int off = core_off(trow, kg * 8, kTM);
                if constexpr (OZAKI) {
                    uint32_t pc[8][kDigits];
#pragma unroll
                    for (int q = 0; q < 8; q++) ozaki_digits(vals[q], e_r, pc[q]);
#pragma unroll
                    for (int s = 0; s < S; s++) {
                        uint4 w4;  // BF16 = high half of each FP32 pattern; two per word
                        w4.x = __byte_perm(pc[0][s], pc[1][s], 0x7632);
                        w4.y = __byte_perm(pc[2][s], pc[3][s], 0x7632);
                        w4.z = __byte_perm(pc[4][s], pc[5][s], 0x7632);
                        w4.w = __byte_perm(pc[6][s], pc[7][s], 0x7632);
                        *(uint4 *)(A + s * Cfg::a_slice_bytes + off) = w4;
                    }
                } else {
                    float pc[S][8];
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        float p3[3];
                        float_pieces((float)vals[q], p3);
#pragma unroll
                        for (int s = 0; s < S; s++) pc[s][q] = p3[s];
                    }
#pragma unroll
                    for (int s = 0; s < S; s++) {
                        uint4 w4;
                        w4.x = pack_bf16(pc[s][0], pc[s][1]);
                        w4.y = pack_bf16(pc[s][2], pc[s][3]);
                        w4.z = pack_bf16(pc[s][4], pc[s][5]);
                        w4.w = pack_bf16(pc[s][6], pc[s][7]);
                        *(uint4 *)(A + s * Cfg::a_slice_bytes + off) = w4;
                    }
                }
            }
            // generic-proxy writes -> visible to the tensor cores, then one
            // arrival per warp
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&a_full[st]);
            used[st] = true;
#pragma unroll
            for (int kh = 0; kh < kGPT; kh++)
#pragma unroll
                for (int q = 0; q < 8; q++) cur[kh][q] = nxt[kh][q];
        }
        // wait for the last commits of both stages
        for (int st = 0; st < 2; st++)
            if (used[st]) {
                if (!mbar_wait_bounded(&mma_done[st], parity[st])) ok = false;
                parity[st] ^= 1u;
            }
    }
    tc_fence_after();
    ok = __syncthreads_and(ok) != 0;
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
    } else if (cutter) {
        // epilogue: warp w reads TMEM lanes 32(w mod 4).. = rows 32(w mod 4)..;
        // the kTPR parts of a row take interleaved groups of 8 columns
        const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
        const int j0 = cb * NT;
        for (int c8 = part * 8; c8 < NT; c8 += 8 * kTPR) {
            if (j0 + c8 >= k) break;
            double out[8];
            if constexpr (OZAKI) {
                // X_g = sum over K and s + s' = g of d_s d'_s' are exact integers
                // (|X_g| <= 8 * 448 * 64^2 < 2^24); the product is
                // sum_g X_g 2^(e_r + e_j - 10 - 7 g).  Horner in two exact int64
                // groups (|z| < 2^46): g = 0..3 and 4..7, then one FP64 rounding.
                long long zh[8], zl[8];
#pragma unroll
                for (int q = 0; q < 8; q++) { zh[q] = 0; zl[q] = 0; }
#pragma unroll
                for (int g = 0; g < G; g++) {
                    uint32_t x[8];
                    tmem_ld8(tmem + lane_base + (uint32_t)(g * NT + c8), x);
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        const long long xi = (long long)__float2int_rn(__uint_as_float(x[q]));
                        if (g < 4) zh[q] = zh[q] * 128 + xi;
                        else zl[q] = zl[q] * 128 + xi;
                    }
                }
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const int j = j0 + c8 + q;
                    const int ef = (j < k) ? fexp[j] : 0;
                    double o = 0.0;
                    if (e_r > -99999 && ef > -99999 && !compose_f64(zh[q], zl[q], e_r + ef, o))
                        o = ldexp(fma((double)zh[q], 0x1p-31, (double)zl[q] * 0x1p-59), e_r + ef);
                    out[q] = o;
                }
            } else {
                uint32_t x[8];
                tmem_ld8(tmem + lane_base + (uint32_t)c8, x);
#pragma unroll
                for (int q = 0; q < 8; q++) out[q] = (double)__uint_as_float(x[q]);
            }
            if (row_ok) {
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const int j = j0 + c8 + q;
                    if (j < k) {
                        C[r + (int64_t)j * ldc] = out[q];
                        if (C32) C32[r + (int64_t)j * ldc] = (float)out[q];
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------- row-tile form (FP64)
// For 64 < k <= 128 the kernel above cuts every row of W once per 64-column
// block of C, i.e. twice.  Here the roles of the operands are swapped so that
// each W entry is cut once: the MMA's M dimension (128) holds all k output
// columns (A operand = the digit slices of Q^T, prepared once and copied per
// chunk), its N dimension 64 rows of W (B operand = the CTA's own cut of W).
// The eight TMEM accumulators (one per digit weight g = s + s') of 64 columns
// each fill the 512 columns; TMEM lane j holds output column j, TMEM column
// n row n of the tile.  The arithmetic (digits, exact sums, recombination,
// one rounding) is the same as above.
constexpr int kRN = 64;                         // rows of W per CTA (MMA N)
constexpr int kRCut = 512;                      // cutter threads: eight per row
constexpr int kRThreads = kRCut + 32;           // + the MMA warp
constexpr int kRTPR = kRCut / kRN;              // threads per row (8)
constexpr int kREPT = kKC / kRTPR;              // W entries each cutter cuts per chunk (4)
static_assert(kREPT == 4, "row-tile chunk split");
constexpr int kRA_slice = 128 * kKC * 2;        // Q^T slice: 128 x 32 BF16 = 8 KB
constexpr int kRB_slice = kRN * kKC * 2;        // W slice: 64 x 32 BF16 = 4 KB
constexpr int kRStage = kDigits * (kRA_slice + kRB_slice);   // 96 KB
constexpr int kRSmem = 2 * kRStage + 1024;

__global__ void __launch_bounds__(kRThreads, 1)
tc_gemm_rows_kernel(const double *__restrict__ W, int64_t ldw, int64_t rows, int t, int k,
                    const uint16_t *__restrict__ Bs, const int *__restrict__ fexp, int nchunks,
                    double *__restrict__ C, int64_t ldc, int *err)
{
    constexpr int S = kDigits;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t a_full[2], b_full[2], mma_done[2];
    __shared__ uint32_t tmem_base_slot;
    __shared__ int s_er[kRN];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool cutter = tid < kRCut;
    const int trow = tid & (kRN - 1), part = tid >> 6;  // cutters: part in [0, 8)
    const int64_t row0 = (int64_t)blockIdx.x * kRN;
    const int64_t r = row0 + trow;
    const bool row_ok = cutter && r < rows;

    if (tid == 0) {
        for (int i = 0; i < 2; i++) {
            mbar_init(&a_full[i], kRCut / 32);
            mbar_init(&b_full[i], 1);
            mbar_init(&mma_done[i], 1);
        }
        fence_barrier_init();
    }
    if (warp == 0) {
        tmem_alloc(&tmem_base_slot, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_slot;

    // row exponents: each part scans every kRTPR-th column of its row
    {
        int e_h = -100000;
        if (row_ok)
            for (int c = part; c < t; c += kRTPR) e_h = max(e_h, dexp_of(W[r + (int64_t)c * ldw]));
        if (cutter && part == 0) s_er[trow] = -100000;
        __syncthreads();
        if (cutter) atomicMax(&s_er[trow], e_h);
        __syncthreads();
    }
    const int e_r = cutter ? s_er[trow] : 0;

    uint32_t parity[2] = {0u, 0u};
    bool used[2] = {false, false};
    bool ok = true;
    if (!cutter) {
        // MMA warp, one thread: stage free -> bulk copy of the Q^T slices ->
        // W slices cut and Q^T landed -> 36 products per 16-wide K step -> commit
        if (lane == 0) {
            uint32_t apar[2] = {0u, 0u}, bpar[2] = {0u, 0u};
            for (int chunk = 0; chunk < nchunks; chunk++) {
                const int st = chunk & 1;
                uint8_t *Aq = smem + st * kRStage;               // Q^T slices (A operand)
                uint8_t *Bw = Aq + S * kRA_slice;                // W slices (B operand)
                if (used[st]) {
                    if (!mbar_wait_bounded(&mma_done[st], parity[st])) ok = false;
                    parity[st] ^= 1u;
                }
                mbar_expect_tx(&b_full[st], (uint32_t)(S * kRA_slice));
                bulk_g2s(Aq, Bs + (int64_t)chunk * S * (128 * kKC), (uint32_t)(S * kRA_slice), &b_full[st]);
                if (!mbar_wait_bounded(&a_full[st], apar[st])) ok = false;
                apar[st] ^= 1u;
                if (!mbar_wait_bounded(&b_full[st], bpar[st])) ok = false;
                bpar[st] ^= 1u;
                tc_fence_after();
                if (ok) {
                    constexpr uint32_t idesc = idesc_bf16(128, kRN);
                    const uint32_t a0 = smem_u32(Aq), b0 = smem_u32(Bw);
                    constexpr uint32_t a_lbo = (128 / 8) * 128, a_sbo = 128;
                    constexpr uint32_t b_lbo = (kRN / 8) * 128, b_sbo = 128;
#pragma unroll
                    for (int ks = 0; ks < kKC / 16; ks++) {
#pragma unroll
                        for (int s = 0; s < S; s++) {
#pragma unroll
                            for (int s2 = 0; s2 < S; s2++) {
                                if (s + s2 > S - 1) continue;
                                const int g = s + s2;
                                const uint64_t ad = smem_desc(a0 + s * kRA_slice + ks * 2 * a_lbo, a_lbo, a_sbo);
                                const uint64_t bd = smem_desc(b0 + s2 * kRB_slice + ks * 2 * b_lbo, b_lbo, b_sbo);
                                // the first product into each accumulator overwrites it
                                const bool first = chunk == 0 && ks == 0 && s == 0;
                                umma_bf16(tmem + (uint32_t)(g * kRN), ad, bd, idesc, first ? 0u : 1u);
                            }
                        }
                    }
                }
                umma_commit(&mma_done[st]);
                used[st] = true;
            }
        }
        __syncwarp();
    } else {
        // cutters: thread (row, part) cuts entries kk = 4 part .. 4 part + 3 of
        // each chunk of its row; the next chunk's entries load while this one is cut
        double cur[kREPT], nxt[kREPT];
        auto load_chunk = [&](int chunk, double (&dst)[kREPT]) {
#pragma unroll
            for (int q = 0; q < kREPT; q++) {
                const int c = chunk * kKC + part * kREPT + q;
                dst[q] = (row_ok && c < t) ? W[r + (int64_t)c * ldw] : 0.0;
            }
        };
        load_chunk(0, cur);
        for (int chunk = 0; chunk < nchunks; chunk++) {
            if (chunk + 1 < nchunks) load_chunk(chunk + 1, nxt);
            const int st = chunk & 1;
            uint8_t *Bw = smem + st * kRStage + S * kRA_slice;
            if (used[st]) {
                if (!mbar_wait_bounded(&mma_done[st], parity[st])) ok = false;
                parity[st] ^= 1u;
            }
            tc_fence_after();
            uint32_t pc[kREPT][kDigits];
#pragma unroll
            for (int q = 0; q < kREPT; q++) ozaki_digits(cur[q], e_r, pc[q]);
            // four BF16 values (high halves of the FP32 patterns) = 8 bytes per slice
            const int off = core_off(trow, part * kREPT, kRN);
#pragma unroll
            for (int s = 0; s < S; s++) {
                uint2 w2;
                w2.x = __byte_perm(pc[0][s], pc[1][s], 0x7632);
                w2.y = __byte_perm(pc[2][s], pc[3][s], 0x7632);
                *(uint2 *)(Bw + s * kRB_slice + off) = w2;
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&a_full[st]);
            used[st] = true;
#pragma unroll
            for (int q = 0; q < kREPT; q++) cur[q] = nxt[q];
        }
        for (int st = 0; st < 2; st++)
            if (used[st]) {
                if (!mbar_wait_bounded(&mma_done[st], parity[st])) ok = false;
                parity[st] ^= 1u;
            }
    }
    tc_fence_after();
    ok = __syncthreads_and(ok) != 0;
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
    } else if (cutter) {
        // epilogue: warp w reads TMEM lanes 32 (w mod 4) .. (output columns j);
        // the four warp groups w / 4 take interleaved groups of 8 TMEM columns
        // (rows of the tile).  Each thread then writes 8 consecutive rows of
        // its column j of C.
        const int jq = warp & 3, grp = warp >> 2;
        const uint32_t lane_base = (uint32_t)(jq * 32) << 16;
        const int j = jq * 32 + lane;
        const int ef = (j < k) ? fexp[j] : -100000;
        for (int c8 = grp * 8; c8 < kRN; c8 += 32) {
            if (row0 + c8 >= rows) break;  // uniform across the warp
            long long zh[8], zl[8];
#pragma unroll
            for (int q = 0; q < 8; q++) { zh[q] = 0; zl[q] = 0; }
#pragma unroll
            for (int g = 0; g < kDigits; g++) {
                uint32_t x[8];
                tmem_ld8(tmem + lane_base + (uint32_t)(g * kRN + c8), x);
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const long long xi = (long long)__float2int_rn(__uint_as_float(x[q]));
                    if (g < 4) zh[q] = zh[q] * 128 + xi;
                    else zl[q] = zl[q] * 128 + xi;
                }
            }
            if (j < k) {
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const int64_t rr = row0 + c8 + q;
                    if (rr >= rows) break;
                    const int er = s_er[c8 + q];
                    double o = 0.0;
                    if (er > -99999 && ef > -99999 && !compose_f64(zh[q], zl[q], er + ef, o))
                        o = ldexp(fma((double)zh[q], 0x1p-31, (double)zl[q] * 0x1p-59), er + ef);
                    C[rr + (int64_t)j * ldc] = o;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------- host side

template <int S, int NT, bool OZAKI>
static size_t bs_bytes(int t, int k)
{
    const int nchunks = (t + kKC - 1) / kKC;
    const int ncb = (k + NT - 1) / NT;
    return (size_t)ncb * nchunks * S * NT * kKC * 2;
}

static size_t slices_bytes(int t, int k)
{
    size_t a = bs_bytes<kDigits, 64, true>(t, k);  // 8 x 64 = 512 TMEM columns
    size_t b = bs_bytes<3, 128, false>(t, k);
    return ((a > b ? a : b) + 255) & ~(size_t)255;
}

// workspace: the B slices, then k column exponents
size_t tc_gemm_ws_bytes(int t, int k) { return slices_bytes(t, k) + sizeof(int) * (size_t)k + 256; }

template <int S, int NT, bool OZAKI, typename WT>
static cudaError_t launch_tc(const WT *W, int64_t ldw, int64_t rows, int t, const double *Q, int64_t ldq,
                             int k, double *C, int64_t ldc, float *C32, uint16_t *bs, int *fexp, int *err,
                             cudaStream_t s)
{
    using Cfg = TileCfg<S, NT>;
    static std::atomic<unsigned long long> attr_done{0};
    cudaError_t e = set_smem_limit_once((const void *)tc_gemm_kernel<S, NT, OZAKI, WT>, Cfg::smem_bytes,
                                        &attr_done);
    if (e != cudaSuccess) return e;
    const int nchunks = (t + kKC - 1) / kKC;
    const int ncb = (k + NT - 1) / NT;
    dim3 pg((unsigned)((ncb * NT + 127) / 128), (unsigned)nchunks);
    prep_b_kernel<S, NT, OZAKI><<<pg, 128, 0, s>>>(Q, ldq, t, k, nchunks, ncb, bs, fexp);
    // 1-D grid over (row tile, column block), column block fastest
    dim3 grid((unsigned)(((rows + kTM - 1) / kTM) * ncb));
    tc_gemm_kernel<S, NT, OZAKI, WT><<<grid, kThreads, Cfg::smem_bytes, s>>>(W, ldw, rows, t, k, bs, fexp,
                                                                          nchunks, ncb, C, ldc, C32, err);
    return cudaGetLastError();
}

// mode 0: FP64 (Ozaki digits), mode 1: three BF16 pieces with FP32 accumulation.
// Self-test of the bounded mbarrier wait: nothing arrives on the barrier, so
// mbar_wait_bounded must give up; the kernel records it in *err and returns.
__global__ void mbar_probe_kernel(int *err)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0)) atomicExch(err, 1);
}

cudaError_t probe_mbarrier(int *err, cudaStream_t s)
{
    mbar_probe_kernel<<<1, 32, 0, s>>>(err);
    return cudaGetLastError();
}

cudaError_t tc_gemm(int mode, const double *W, const float *W32, int64_t ldw, int64_t rows, int t,
                    const double *Q, int64_t ldq, int k, double *C, int64_t ldc, float *C32, void *ws,
                    int *err, cudaStream_t s, int *launches)
{
    if (t < 1 || k < 1 || rows < 1) return cudaErrorInvalidValue;
    if (mode == 0 && t > kMaxT) return cudaErrorInvalidValue;
    uint16_t *bs = (uint16_t *)ws;
    int *fx = (int *)((uint8_t *)ws + slices_bytes(t, k));
    if (launches) *launches += 2;
    if (mode == 0 && k > 64 && k <= 128 && !C32) {
        // every W entry cut once: the row-tile form (Q^T slices for 128 columns)
        static std::atomic<unsigned long long> attr_done{0};
        cudaError_t e = set_smem_limit_once((const void *)tc_gemm_rows_kernel, kRSmem, &attr_done);
        if (e != cudaSuccess) return e;
        const int nchunks = (t + kKC - 1) / kKC;
        dim3 pg((unsigned)((128 + 127) / 128), (unsigned)nchunks);
        prep_b_kernel<kDigits, 128, true><<<pg, 128, 0, s>>>(Q, ldq, t, k, nchunks, 1, bs, fx);
        tc_gemm_rows_kernel<<<(unsigned)((rows + kRN - 1) / kRN), kRThreads, kRSmem, s>>>(
            W, ldw, rows, t, k, bs, fx, nchunks, C, ldc, err);
        return cudaGetLastError();
    }
    if (mode == 0)
        return launch_tc<kDigits, 64, true, double>(W, ldw, rows, t, Q, ldq, k, C, ldc, C32, bs, fx, err, s);
    if (W32) return launch_tc<3, 128, false, float>(W32, ldw, rows, t, Q, ldq, k, C, ldc, C32, bs, fx, err, s);
    return launch_tc<3, 128, false, double>(W, ldw, rows, t, Q, ldq, k, C, ldc, C32, bs, fx, err, s);
}

}  // namespace svdsc
