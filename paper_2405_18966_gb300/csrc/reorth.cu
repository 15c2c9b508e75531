// Full re-orthogonalization (Sec. 2.1 of the svds-C paper) as CGS2 on the
// device: h = W^T w (GEMV-T, per-CTA partial sums over row chunks + an ordered
// reduction), w -= W h (GEMV-N, fused with the partial sums of ||w||^2 on the
// last pass), then the norm / breakdown test / scaling of Alg. 1; and the
// estimate-driven gate of the optional partial re-orthogonalization.
// Every reduction runs in a fixed order, so results are bitwise reproducible.
#include <cstdint>
#include <cstdio>
#include "internal.cuh"

namespace svdsc {

Chunk make_chunk(int64_t len, int target_blocks)
{
    Chunk c;
    c.len = len;
    int64_t R = (len + target_blocks - 1) / target_blocks;
    R = (R + 63) & ~int64_t(63);
    if (R < 256) R = 256;
    if (R > 4096) R = 4096;
    c.R = R;
    c.nb = (int)((len + R - 1) / R);
    if (c.nb < 1) c.nb = 1;
    // FP64 GEMV-N: one 512-row pass per 256-thread CTA from 684,032 rows on
    // (1.1 x 152 SMs x 8 CTAs x 512 rows); below that, the chunks above
    // (about two CTAs per SM) keep the SMs evenly loaded.  Measured on GB300
    // over 250,000 - 4,000,000 rows: small CTAs lose below ~one wave (500,000
    // rows: 77 % of the FP64 FMA peak against 80 %) and win from 750,000 rows
    // on (82-90 % against 58-84 %: the chunks' partial last pass and, past
    // the 4,096-row cap, SMs holding one CTA more than the others).  A
    // constant, not a query of the device, so the summation order of the
    // norm never depends on it.
    if (len >= kUpdSmallMinRows) {
        c.Ru = 2 * kUpdSmallThreads;
        c.thu = kUpdSmallThreads;
    } else {
        c.Ru = c.R;
        c.thu = kRowThreads;
    }
    c.nbu = (int)((len + c.Ru - 1) / c.Ru);
    if (c.nbu < 1) c.nbu = 1;
    return c;
}

__device__ __forceinline__ bool poisoned(const int *poison)
{
    return poison && *(volatile const int *)poison;
}

// ---------------------------------------------------------------- GEMV-T

constexpr int kProjWarps = 16;

// P[c * nb + b] = sum over the rows of chunk b of W(r, c) * w(r).
// FP64: each lane keeps one accumulator per column (the FP64 pipe, at 2 FMA
// per clock per SM on GB300, is the bound, not the FMA latency), the 32 lane
// partials of a column go to shared memory, and one thread per column adds
// them: 1 FP64 add per lane and column instead of a 5-step shuffle tree plus
// merging of several accumulators.
template <typename WT>
__global__ void __launch_bounds__(kProjWarps * 32)
proj_partial_kernel(const WT *__restrict__ W, int64_t ld, int ncols, const double *__restrict__ w,
                    int64_t len, int64_t R, int nb, double *__restrict__ P, const int *poison)
{
    if (poisoned(poison)) return;
    extern __shared__ double ws[];
    // FP32 pass: the chunk of w is converted once (double -> float conversions
    // run on the FP64 pipe, so none may sit in the inner loop)
    float *ws32 = (float *)ws;
    const int64_t r0 = (int64_t)blockIdx.x * R;
    const int rows = (int)min(R, len - r0);
    for (int j = threadIdx.x; j < rows; j += blockDim.x) {
        if constexpr (sizeof(WT) == 8) ws[j] = w[r0 + j];
        else ws32[j] = (float)w[r0 + j];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if constexpr (sizeof(WT) == 8) {
        double *lp = ws + ((R + 1) & ~int64_t(1));  // lane partials: [column][32]
        for (int c = warp; c < ncols; c += kProjWarps) {
            const double *col = W + (int64_t)c * ld + r0;
            double a = 0.0;
            int j = 2 * lane;
            for (; j + 65 < rows; j += 128) {
                const double2 v0 = __ldcs((const double2 *)(col + j));
                const double2 v1 = __ldcs((const double2 *)(col + j + 64));
                a = fma(v0.x, ws[j], a);
                a = fma(v0.y, ws[j + 1], a);
                a = fma(v1.x, ws[j + 64], a);
                a = fma(v1.y, ws[j + 65], a);
            }
            for (; j < rows; j += 64) {
                a = fma((double)col[j], ws[j], a);
                if (j + 1 < rows) a = fma((double)col[j + 1], ws[j + 1], a);
            }
            lp[c * 32 + lane] = a;
        }
        __syncthreads();
        for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
            double s = 0.0;
#pragma unroll 8
            for (int l = 0; l < 32; l++) s += lp[c * 32 + l];
            P[(int64_t)c * nb + blockIdx.x] = s;
        }
    } else {
        for (int c = warp; c < ncols; c += kProjWarps) {
            const WT *col = W + (int64_t)c * ld + r0;
            // FP32 shadow (first CGS pass of the mixed form): FP32 products and
            // sums, four 16-byte loads in flight per lane
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
            int j = 4 * lane;
            for (; j + 387 < rows; j += 512) {
                float4 v[4], x[4];
#pragma unroll
                for (int u = 0; u < 4; u++) v[u] = __ldcs((const float4 *)(col + j + 128 * u));
#pragma unroll
                for (int u = 0; u < 4; u++) x[u] = *(const float4 *)(ws32 + j + 128 * u);
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    a0 = fmaf(v[u].x, x[u].x, a0);
                    a1 = fmaf(v[u].y, x[u].y, a1);
                    a2 = fmaf(v[u].z, x[u].z, a2);
                    a3 = fmaf(v[u].w, x[u].w, a3);
                }
            }
            for (; j + 3 < rows; j += 128) {
                const float4 v = __ldcs((const float4 *)(col + j));
                const float4 x = *(const float4 *)(ws32 + j);
                a0 = fmaf(v.x, x.x, a0);
                a1 = fmaf(v.y, x.y, a1);
                a2 = fmaf(v.z, x.z, a2);
                a3 = fmaf(v.w, x.w, a3);
            }
            // this lane's last, partial group of four
#pragma unroll
            for (int q = 0; q < 4; q++)
                if (j + q < rows) a0 = fmaf((float)col[j + q], ws32[j + q], a0);
            double s = (double)((a0 + a1) + (a2 + a3));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) P[(int64_t)c * nb + blockIdx.x] = s;
        }
    }
}

void proj_partial(const double *W, int64_t ld, int ncols, const double *w, const Chunk &c,
                  double *P, const int *poison, cudaStream_t s)
{
    if (ncols <= 0) return;
    const size_t smem = sizeof(double) * (((c.R + 1) & ~int64_t(1)) + 32 * (size_t)ncols);
    static std::atomic<unsigned long long> attr_done{0};
    if (smem > 48 * 1024)  // up to 4,096 rows of w plus 32 partials for up to 513 columns: < 170 KB
        set_smem_limit_once((const void *)proj_partial_kernel<double>, 200 * 1024, &attr_done);
    proj_partial_kernel<double><<<c.nb, kProjWarps * 32, smem, s>>>(W, ld, ncols, w, c.len, c.R, c.nb, P, poison);
}

void proj_partial_f32(const float *W32, int64_t ld, int ncols, const double *w, const Chunk &c,
                      double *P, const int *poison, cudaStream_t s)
{
    if (ncols <= 0) return;
    proj_partial_kernel<float><<<c.nb, kProjWarps * 32, sizeof(double) * c.R, s>>>(
        W32, ld, ncols, w, c.len, c.R, c.nb, P, poison);
}

// h[c] = sum over b of P[c * nb + b], in a fixed order.
__global__ void __launch_bounds__(128)
proj_reduce_kernel(const double *__restrict__ P, int nb, double *__restrict__ h, const int *poison)
{
    if (poisoned(poison)) return;
    const double *p = P + (int64_t)blockIdx.x * nb;
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += 128) s += p[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double red[4];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) h[blockIdx.x] = (red[0] + red[1]) + (red[2] + red[3]);
}

void proj_reduce(const double *P, int nb, int ncols, double *h, const int *poison, cudaStream_t s)
{
    if (ncols <= 0) return;
    proj_reduce_kernel<<<ncols, 128, 0, s>>>(P, nb, h, poison);
}

// ---------------------------------------------------------------- GEMV-N

__device__ __forceinline__ double block_sum_256(double v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += red[i];
    }
    return t;
}

// w(r) -= sum_c W(r, c) h(c) over chunk rows; Pn[b] = sum of the new w(r)^2
template <typename WT, int TH>
__device__ __forceinline__ void update_body(const WT *__restrict__ W, int64_t ld, int ncols,
                                            const double *__restrict__ h, double *__restrict__ w,
                                            int64_t len, int64_t R, double *__restrict__ Pn)
{
    extern __shared__ double hs[];
    __shared__ double red[TH / 32];
    float *hs32 = (float *)(hs + ncols);  // FP32 copy for the FP32 pass (converted once)
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
        hs[c] = h[c];
        if constexpr (sizeof(WT) == 4) hs32[c] = (float)h[c];
    }
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * R;
    const int rows = (int)min(R, len - r0);
    double nrm = 0.0;
    for (int j = 2 * threadIdx.x; j < rows; j += 2 * TH) {
        const int64_t r = r0 + j;
        if (j + 1 < rows) {
            double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
            const WT *p = W + r;
            int c = 0;
            if constexpr (sizeof(WT) == 8) {
                for (; c + 1 < ncols; c += 2) {
                    const double2 v0 = __ldcs((const double2 *)(p + (int64_t)c * ld));
                    const double2 v1 = __ldcs((const double2 *)(p + (int64_t)(c + 1) * ld));
                    a0 = fma(v0.x, hs[c], a0);
                    a1 = fma(v0.y, hs[c], a1);
                    b0 = fma(v1.x, hs[c + 1], b0);
                    b1 = fma(v1.y, hs[c + 1], b1);
                }
                for (; c < ncols; c++) {
                    const double2 v0 = __ldcs((const double2 *)(p + (int64_t)c * ld));
                    a0 = fma(v0.x, hs[c], a0);
                    a1 = fma(v0.y, hs[c], a1);
                }
            } else {
                float f0 = 0.f, f1 = 0.f, g0 = 0.f, g1 = 0.f;
                // four 8-byte loads in flight per thread (the FP32 pass is HBM-bound);
                // same accumulation order as the two-column loop below
                for (; c + 3 < ncols; c += 4) {
                    const float2 v0 = __ldcs((const float2 *)(p + (int64_t)c * ld));
                    const float2 v1 = __ldcs((const float2 *)(p + (int64_t)(c + 1) * ld));
                    const float2 v2 = __ldcs((const float2 *)(p + (int64_t)(c + 2) * ld));
                    const float2 v3 = __ldcs((const float2 *)(p + (int64_t)(c + 3) * ld));
                    f0 = fmaf(v0.x, hs32[c], f0);
                    f1 = fmaf(v0.y, hs32[c], f1);
                    g0 = fmaf(v1.x, hs32[c + 1], g0);
                    g1 = fmaf(v1.y, hs32[c + 1], g1);
                    f0 = fmaf(v2.x, hs32[c + 2], f0);
                    f1 = fmaf(v2.y, hs32[c + 2], f1);
                    g0 = fmaf(v3.x, hs32[c + 3], g0);
                    g1 = fmaf(v3.y, hs32[c + 3], g1);
                }
                for (; c + 1 < ncols; c += 2) {
                    const float2 v0 = __ldcs((const float2 *)(p + (int64_t)c * ld));
                    const float2 v1 = __ldcs((const float2 *)(p + (int64_t)(c + 1) * ld));
                    f0 = fmaf(v0.x, hs32[c], f0);
                    f1 = fmaf(v0.y, hs32[c], f1);
                    g0 = fmaf(v1.x, hs32[c + 1], g0);
                    g1 = fmaf(v1.y, hs32[c + 1], g1);
                }
                for (; c < ncols; c++) {
                    const float2 v0 = __ldcs((const float2 *)(p + (int64_t)c * ld));
                    f0 = fmaf(v0.x, hs32[c], f0);
                    f1 = fmaf(v0.y, hs32[c], f1);
                }
                a0 = (double)f0; a1 = (double)f1; b0 = (double)g0; b1 = (double)g1;
            }
            const double n0 = w[r] - (a0 + b0);
            const double n1 = w[r + 1] - (a1 + b1);
            w[r] = n0;
            w[r + 1] = n1;
            nrm = fma(n0, n0, nrm);
            nrm = fma(n1, n1, nrm);
        } else {
            double a0 = 0.0;
            if constexpr (sizeof(WT) == 4) {
                float f = 0.f;
                for (int c = 0; c < ncols; c++) f = fmaf((float)W[r + (int64_t)c * ld], hs32[c], f);
                a0 = (double)f;
            } else {
                for (int c = 0; c < ncols; c++) a0 = fma((double)W[r + (int64_t)c * ld], hs[c], a0);
            }
            const double n0 = w[r] - a0;
            w[r] = n0;
            nrm = fma(n0, n0, nrm);
        }
    }
    if (Pn) {
        const double t = block_sum_256(nrm, red);
        if (threadIdx.x == 0) Pn[blockIdx.x] = t;
    }
}

template <typename WT>
__global__ void __launch_bounds__(kRowThreads)
update_kernel(const WT *__restrict__ W, int64_t ld, int ncols, const double *__restrict__ h,
              double *__restrict__ w, int64_t len, int64_t R, double *__restrict__ Pn,
              const int *poison)
{
    if (poisoned(poison)) return;
    update_body<WT, kRowThreads>(W, ld, ncols, h, w, len, R, Pn);
}

// The small-CTA layout of the FP64 GEMV-N, with the arithmetic of
// update_kernel<double> written out: this body compiles to 40 registers (six
// CTAs resident per SM), the shared template to 44 (five).  Asking for eight
// CTAs (32 registers) spills and measured slower.
__global__ void __launch_bounds__(kUpdSmallThreads)
update_small_kernel(const double *__restrict__ W, int64_t ld, int ncols, const double *__restrict__ h,
                    double *__restrict__ w, int64_t len, int64_t R, double *__restrict__ Pn,
                    const int *poison)
{
    if (poisoned(poison)) return;
    extern __shared__ double hs[];
    __shared__ double red[kUpdSmallThreads / 32];
    for (int c = threadIdx.x; c < ncols; c += kUpdSmallThreads) hs[c] = h[c];
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * R;
    const int rows = (int)min(R, len - r0);
    double nrm = 0.0;
    for (int j = 2 * threadIdx.x; j < rows; j += 2 * kUpdSmallThreads) {
        const int64_t r = r0 + j;
        if (j + 1 < rows) {
            double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
            const double *p = W + r;
            int c = 0;
            for (; c + 1 < ncols; c += 2) {
                const double2 v0 = __ldcs((const double2 *)(p + (int64_t)c * ld));
                const double2 v1 = __ldcs((const double2 *)(p + (int64_t)(c + 1) * ld));
                a0 = fma(v0.x, hs[c], a0);
                a1 = fma(v0.y, hs[c], a1);
                b0 = fma(v1.x, hs[c + 1], b0);
                b1 = fma(v1.y, hs[c + 1], b1);
            }
            for (; c < ncols; c++) {
                const double2 v0 = __ldcs((const double2 *)(p + (int64_t)c * ld));
                a0 = fma(v0.x, hs[c], a0);
                a1 = fma(v0.y, hs[c], a1);
            }
            const double n0 = w[r] - (a0 + b0);
            const double n1 = w[r + 1] - (a1 + b1);
            w[r] = n0;
            w[r + 1] = n1;
            nrm = fma(n0, n0, nrm);
            nrm = fma(n1, n1, nrm);
        } else {
            double a0 = 0.0;
            for (int c = 0; c < ncols; c++) a0 = fma(W[r + (int64_t)c * ld], hs[c], a0);
            const double n0 = w[r] - a0;
            w[r] = n0;
            nrm = fma(n0, n0, nrm);
        }
    }
    if (Pn) {
        const double t = block_sum_256(nrm, red);
        if (threadIdx.x == 0) Pn[blockIdx.x] = t;
    }
}

void update_sub(const double *W, int64_t ld, int ncols, const double *h, double *w, const Chunk &c,
                double *Pn, const int *poison, cudaStream_t s)
{
    if (ncols <= 0 && !Pn) return;
    const size_t smem = sizeof(double) * (ncols > 0 ? ncols : 1);
    if (c.thu == kUpdSmallThreads)
        update_small_kernel<<<c.nbu, kUpdSmallThreads, smem, s>>>(W, ld, ncols, h, w, c.len, c.Ru, Pn,
                                                                  poison);
    else
        update_kernel<double><<<c.nbu, kRowThreads, smem, s>>>(W, ld, ncols, h, w, c.len, c.Ru, Pn, poison);
}

void update_sub_f32(const float *W32, int64_t ld, int ncols, const double *h, double *w,
                    const Chunk &c, const int *poison, cudaStream_t s)
{
    if (ncols <= 0) return;
    update_kernel<float><<<c.nb, kRowThreads, sizeof(double) * ncols + sizeof(float) * ncols, s>>>(
        W32, ld, ncols, h, w, c.len, c.R, nullptr, poison);
}

__global__ void __launch_bounds__(kRowThreads)
norm_partial_kernel(const double *__restrict__ w, int64_t len, int64_t R, double *__restrict__ Pn,
                    const int *poison)
{
    if (poisoned(poison)) return;
    __shared__ double red[kRowThreads / 32];
    const int64_t r0 = (int64_t)blockIdx.x * R;
    const int rows = (int)min(R, len - r0);
    double nrm = 0.0;
    for (int j = threadIdx.x; j < rows; j += kRowThreads) nrm = fma(w[r0 + j], w[r0 + j], nrm);
    const double t = block_sum_256(nrm, red);
    if (threadIdx.x == 0) Pn[blockIdx.x] = t;
}

void norm_partial(const double *w, const Chunk &c, double *Pn, const int *poison, cudaStream_t s)
{
    norm_partial_kernel<<<c.nbu, kRowThreads, 0, s>>>(w, c.len, c.Ru, Pn, poison);
}

// *out = sqrt(sum of the nb partial sums of ||w||^2), in a fixed order (one CTA).
__global__ void __launch_bounds__(256)
norm_from_partials_kernel(const double *__restrict__ Pn, int nb, double *out)
{
    __shared__ double red[8];
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += Pn[b];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        *out = sqrt(t);
    }
}

void norm_from_partials(const double *Pn, int nb, double *out, cudaStream_t s)
{
    norm_from_partials_kernel<<<1, 256, 0, s>>>(Pn, nb, out);
}

// ---------------------------------------------------------------- finalize

__global__ void __launch_bounds__(kRowThreads)
finalize_kernel(double *__restrict__ w, int64_t len, int64_t R, const double *__restrict__ Pn, int nb,
                double *T_entry, DevStatus *st, int step, int parity, int mode, float *w32)
{
    if (*(volatile int *)&st->poison) return;
    __shared__ double red[kRowThreads / 32];
    __shared__ double s_nrm;
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += kRowThreads) v += Pn[b];
    const double tot = block_sum_256(v, red);
    if (threadIdx.x == 0) s_nrm = sqrt(tot);
    __syncthreads();
    const double nrm = s_nrm;
    const double anorm = st->anorm[parity];
    bool bad;
    if (mode == 0) bad = !(nrm > 1e-13 * anorm) || !isfinite(nrm);
    else if (mode == 2) bad = !(nrm > 1e-8) || !isfinite(nrm);
    else bad = !(nrm > 0.0) || !isfinite(nrm);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (bad) {
            atomicMin(&st->bd_step, step);
            if (!isfinite(nrm)) st->nonfinite = 1;
            st->poison = 1;
        }
        if (mode == 0 && T_entry) *T_entry = bad ? 0.0 : nrm;
        if (mode == 2 && T_entry) *T_entry = 0.0;
        st->anorm[parity ^ 1] = (mode == 0 && !bad && nrm > anorm) ? nrm : anorm;
        st->last_norm = nrm;
    }
    if (bad) return;
    const double inv = 1.0 / nrm;
    const int64_t r0 = (int64_t)blockIdx.x * R;
    const int rows = (int)min(R, len - r0);
    for (int j = threadIdx.x; j < rows; j += kRowThreads) {
        const double x = w[r0 + j] * inv;
        w[r0 + j] = x;
        if (w32) w32[r0 + j] = (float)x;
    }
}

void finalize(double *w, const Chunk &c, const double *Pn, double *T_entry, DevStatus *st, int step,
              int parity, int mode, float *w32, cudaStream_t s)
{
    finalize_kernel<<<c.nb, kRowThreads, 0, s>>>(w, c.len, c.R, Pn, c.nbu, T_entry, st, step, parity,
                                                 mode, w32);
}

// ------------------------------------------- partial re-orthogonalization
//
// Opt-in alternative to re-orthogonalizing every Lanczos vector (the scheme
// lansvd uses, Table 1).  With A v_l = sum_r T(r,l) u_r and
// A^T u_l = sum_r T(l,r) v_r (true also after an augmented restart, whose T
// has the spike column of Eq. 6-7), the inner products of a new vector with
// the earlier ones follow
//   ||w|| nu'_l = sum_{r<=l} T(r,l) mu_r - alpha_i nu_l         (v_{i+1}, l <= i)
//   ||w|| mu'_l = sum_{r>=l} T(l,r) nu_r - beta_i  mu_l         (u_{i+1}, l <= i)
// (w: the vector before normalization), each grown by a rounding term
// eps ||A|| / ||w|| of the estimate's sign.  When the largest estimate passes
// eps^(3/4), the vector gets the full CGS2 against all earlier ones (and so
// does the next vector of its kind), and its estimates drop to eps.  (At
// sqrt(eps) the singular values stay accurate, but the components CGS2 then
// removes, which T does not record, leave true residuals near sqrt(eps)||A||;
// eps^(3/4) keeps them near 1e-12 ||A|| for a few more CGS2 passes.)  One CTA;
// T is bidiagonal except for the spike column kk + 1 after a restart (kk = 0
// before the first), so only its non-zero entries are visited, in ascending
// order.  The decision goes to pr->gate (0: run the CGS2 kernels, 1: skip).

constexpr double kPrEps = 2.220446049250313e-16;      // DBL_EPSILON
constexpr double kPrDelta = 1.8189894035458565e-12;   // DBL_EPSILON^(3/4) = 2^-39

__global__ void __launch_bounds__(kRowThreads)
pr_omega_kernel(int side, int i, int kk, const double *__restrict__ T, int ldt, double *__restrict__ mu,
                double *__restrict__ nu, const double *__restrict__ Pn, int nb, const DevStatus *st,
                int parity, PrState *pr, double bt, double bn, double fl)
{
    __shared__ double red[kRowThreads / 32];
    __shared__ double s_w, s_mx;
    if (*(volatile const int *)&st->poison) {
        if (threadIdx.x == 0) pr->gate = 1;
        return;
    }
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += kRowThreads) v += Pn[b];
    const double tot = block_sum_256(v, red);
    if (threadIdx.x == 0) s_w = sqrt(tot);
    __syncthreads();
    const double wn = s_w;
    auto Tv = [&](int r, int c) { return T[(r - 1) + (int64_t)(c - 1) * ldt]; };  // 1-based
    const bool ok = wn > 0.0 && isfinite(wn);
    double mx = 0.0;
    if (ok) {
        const double tau = kPrEps * st->anorm[parity] / wn;
        if (side == 1) {
            const double alpha_i = Tv(i, i);
            for (int l = 1 + threadIdx.x; l <= i; l += blockDim.x) {
                double s = 0.0;
                if (kk > 0 && l == kk + 1) {
                    for (int r = 1; r <= l; r++) s += Tv(r, l) * mu[r - 1];
                } else {
                    if (l > 1 && l - 1 > kk) s += Tv(l - 1, l) * mu[l - 2];
                    s += Tv(l, l) * mu[l - 1];
                }
                double x = (s - alpha_i * nu[l - 1]) / wn;
                x += x >= 0.0 ? tau : -tau;
                nu[l - 1] = x;
                mx = fmax(mx, fabs(x));
            }
        } else {
            const double beta_i = Tv(i, i + 1);
            for (int l = 1 + threadIdx.x; l <= i; l += blockDim.x) {
                double s = Tv(l, l) * nu[l - 1];
                if (l <= kk) s += Tv(l, kk + 1) * nu[kk];
                else s += Tv(l, l + 1) * nu[l];
                double x = (s - beta_i * mu[l - 1]) / wn;
                x += x >= 0.0 ? tau : -tau;
                mu[l - 1] = x;
                mx = fmax(mx, fabs(x));
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) m2 = fmax(m2, red[w]);
        s_mx = m2;
    }
    __syncthreads();
    int *force = side ? &pr->force_v : &pr->force_u;
    const bool need = !ok || s_mx > kPrDelta || *force;
    double *est = side ? nu : mu;
    if (need)
        for (int l = threadIdx.x; l < i; l += blockDim.x) est[l] = kPrEps;
    if (threadIdx.x == 0) {
        est[i] = 1.0;
        pr->gate = need ? 0 : 1;
        if (need) {
            pr->n_reorth++;
            pr->bytes_t += bt;
            pr->bytes_n += bn;
            pr->flops += fl;
            *force = !*force;
        }
    }
}

void pr_omega(int side, int i, int kk, const double *T, int ldt, double *mu, double *nu, const Chunk &c,
              const double *Pn, const DevStatus *st, int parity, PrState *pr, double bt, double bn,
              double fl, cudaStream_t s)
{
    pr_omega_kernel<<<1, kRowThreads, 0, s>>>(side, i, kk, T, ldt, mu, nu, Pn, c.nbu, st, parity, pr, bt,
                                              bn, fl);
}

// After an augmented restart: v_{k+1} = v_{t+1} against V~_k = V(:,1:t) Vh(:,1:k)
// is bounded by sum_l |Vh(l,j)| |nu_l| (+ eps); u_{k+1} gets CGS2 (eps).
__global__ void __launch_bounds__(kRowThreads)
pr_restart_kernel(int t, int k, const double *__restrict__ Vh, double *__restrict__ mu,
                  double *__restrict__ nu, PrState *pr)
{
    __shared__ double anu[512];
    for (int l = threadIdx.x; l < t; l += blockDim.x) anu[l] = fabs(nu[l]);
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        double acc = 0.0;
        for (int l = 0; l < t; l++) acc += fabs(Vh[l + (int64_t)j * t]) * anu[l];
        nu[j] = acc + kPrEps;
        mu[j] = kPrEps;
    }
    if (threadIdx.x == 0) {
        nu[k] = 1.0;
        mu[k] = 1.0;
        pr->force_u = 0;
        pr->force_v = 0;
    }
}

void pr_restart(int t, int k, const double *Vh, double *mu, double *nu, PrState *pr, cudaStream_t s)
{
    pr_restart_kernel<<<1, kRowThreads, 0, s>>>(t, k, Vh, mu, nu, pr);
}

// est[0..col-1] = eps (a vector that was orthogonalized against all earlier ones);
// col < 0: start of a solve (nu_1 = mu_1 = 1, flags and counter cleared).
__global__ void pr_reset_kernel(int side, int col, double *mu, double *nu, PrState *pr)
{
    if (col < 0) {
        if (threadIdx.x == 0) {
            mu[0] = 1.0;
            nu[0] = 1.0;
            pr->gate = 1;
            pr->force_u = pr->force_v = 0;
            pr->n_reorth = 0;
            pr->bytes_t = pr->bytes_n = pr->flops = 0.0;
        }
        return;
    }
    double *est = side ? nu : mu;
    for (int l = threadIdx.x; l < col; l += blockDim.x) est[l] = kPrEps;
}

void pr_reset(int side, int col, double *mu, double *nu, PrState *pr, cudaStream_t s)
{
    pr_reset_kernel<<<1, 256, 0, s>>>(side, col, mu, nu, pr);
}

// ---------------------------------------------------------------- random draws

__global__ void rng_normal_kernel(uint64_t seed, uint64_t draw, int64_t len, double *x)
{
    const uint64_t key = splitmix_mix(seed);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < len;
         j += (int64_t)gridDim.x * blockDim.x)
        x[j] = normal_draw(key, draw, (uint64_t)j);
}

void rng_normal_vec(uint64_t seed, uint64_t draw, int64_t len, double *x, cudaStream_t s)
{
    const int64_t blocks = std::min<int64_t>((len + 255) / 256, 4 * 152);
    rng_normal_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(seed, draw, len, x);
}

__global__ void f64_to_f32_kernel(const double *__restrict__ x, float *__restrict__ y, int64_t len)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < len;
         j += (int64_t)gridDim.x * blockDim.x)
        y[j] = (float)x[j];
}

void copy_f64_to_f32(const double *x, float *y, int64_t len, cudaStream_t s)
{
    const int64_t blocks = std::min<int64_t>((len + 255) / 256, 8 * 152);
    f64_to_f32_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(x, y, len);
}

}  // namespace svdsc
