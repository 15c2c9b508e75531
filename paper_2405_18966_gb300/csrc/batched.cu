// Batched form: many independent truncated SVDs (uneven shapes and k) in ONE
// persistent launch.  A thread-block cluster of C CTAs (C = 1, 2, 4 or 8)
// takes matrices from an atomic work queue (largest estimated cost first) and
// runs Alg. 2 of the svds-C paper for each from start to finish; the rows of
// A, A^T and of the Lanczos bases are split across the cluster's CTAs, and
// every reduction (projection coefficients, norms, the sign rule's argmax) is
// combined through distributed shared memory in a fixed rank order, so every
// CTA takes the same decisions.  The steps are: Lanczos bidiagonalization with CGS2 full
// re-orthogonalization, the projected SVD (one-sided Jacobi in shared memory),
// the Eq. (4) residual test and the augmented restart, then the outputs.
// Precision is the mixed form: FP32 CSR values, FP32 SpMV with FP32
// accumulation, FP32 first CGS pass on FP32 basis shadows, FP64 second pass,
// norms, projected SVD and residuals, FP32 restart GEMM.  CTAs synchronize
// only inside their own cluster (hardware cluster barrier); clusters never
// wait on one another.  The launch (with the
// parameter upload and queue reset) is captured once in a CUDA graph and
// replayed by every solve.  SpMV lanes-per-row and the GEMV-T column tile are
// chosen per matrix-shape class by timing the candidates (autotuner below).
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>
#include "internal.cuh"

namespace svdsc {

constexpr int kBT = 512;          // threads per CTA
constexpr int kBW = kBT / 32;     // warps per CTA
constexpr int kBMaxT = 80;        // subspace limit of the batched form (shared-memory Jacobi)
constexpr int kBMaxK = 48;        // rank limit (register accumulators of the GEMM)

struct BMat {
    int64_t m, n, nnz;
    int k, t;
    const int64_t *rp, *rpT;
    const int32_t *col, *colT;
    const float *val, *valT;
    double *S, *U, *V, *res;   // outputs (device), U: m x k (ld m), V: n x k (ld n)
    int gA, gAT, tc, pad;      // tuned: lanes per row for A and A^T, GEMV-T columns per warp
    uint64_t seed;
    double *ckv;               // hand-off: v_{k+1} (n entries); U~_k and V~_k go to U and V
    struct BHand *hand;        // hand-off: the rest of the restart state
};

// The state of a matrix handed from the first launch to the second at a
// restart boundary, after the restart GEMM: U~_k (in the output U), V~_k (in
// the output V), v_{k+1} (ckv), and this.
struct BHand {
    double anorm;
    unsigned long long draws;
    int restarts, it;
    long long cycles_total, cycles_svd, cycles_lbp;
    long long work;  // cycles x CTAs of the first launch's share
    double S[kBMaxK], rho[kBMaxK];  // the k Ritz values and restart coefficients
};

// Queue state of one batch solve (device memory, reset by the graph).
struct BQueue {
    int next;      // next position in the first launch's queue
    int idle;      // clusters of the first launch that found the queue empty
    int ho_count;  // matrices handed to the second launch
    int next2;     // next position in the hand-off list
};

struct BStat {
    int converged, nconv, restarts, breakdowns;
    int64_t n_matvec, n_steps;
    double anorm, beta_t;
    int err, svd_sweeps;
    int64_t cycles_total, cycles_svd, cycles_lbp;  // SM clock cycles on the cluster leader
    int cluster, pad;
    int64_t cycles_phase[5];  // SpMV, FP32 CGS pass, FP64 CGS pass, norm/scale, restart/output GEMM
    int64_t work;             // SM cycles: cycles on the leader x CTAs of its cluster, summed over launches
};

struct BSlot {   // one per cluster (bases), T one per CTA
    double *U0, *U1, *V0, *V1;
    float *U32_0, *U32_1, *V32_0, *V32_1;
    float *wf;      // FP32 copy of the vector being orthogonalized (each CTA its rows)
    int64_t ldu, ldv;
};

struct BParams {
    double tol;
    int maxit;
    int handoff_idle;  // hand off once this many clusters are idle (0: never)
};

// ------------------------------------------------------------ cluster helpers
__device__ __forceinline__ uint32_t cl_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cl_size()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cl_id()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}

// all threads of every CTA of the cluster; orders shared and global memory
// at cluster scope
__device__ __forceinline__ void cl_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t cl_map(const void *p, uint32_t rank)
{
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
    return ra;
}

__device__ __forceinline__ double cl_ld(const double *p, uint32_t rank)
{
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(cl_map(p, rank)) : "memory");
    return v;
}

__device__ __forceinline__ long long cl_ld_i64(const long long *p, uint32_t rank)
{
    long long v;
    asm volatile("ld.shared::cluster.s64 %0, [%1];" : "=l"(v) : "r"(cl_map(p, rank)) : "memory");
    return v;
}

__device__ __forceinline__ int cl_ld_i32(const int *p, uint32_t rank)
{
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(cl_map(p, rank)) : "memory");
    return v;
}

// shared-memory layout (doubles)
constexpr int kSmB = 0;                               // B: t x t (Jacobi columns)
constexpr int kSmW = kSmB + kBMaxT * kBMaxT;          // W: t x t (rotations)
// The sparse products gather from a copy of the whole input vector (FP32) in
// shared memory when it fits in the region of B and W, which only the
// projected SVD uses (never during a product); the region is padded to hold
// 30,720 floats, every v-side vector of the batch workload (n <= 30,000).
// (A much larger dedicated region was measured slower: it shrinks the L1
// cache that the gathers of longer vectors rely on.)
constexpr int kXCap = 30720;                          // floats
constexpr int kSmBW = (kXCap / 2 > 2 * kBMaxT * kBMaxT) ? kXCap / 2 : 2 * kBMaxT * kBMaxT;
constexpr int kSmS = kSmB + kSmBW;                    // sorted sigma (t)
constexpr int kSmUt = kSmS + kBMaxT;                  // Uh(t, j) for j < k
constexpr int kSmRho = kSmUt + kBMaxT;                // rho (k)
constexpr int kSmH = kSmRho + kBMaxT;                 // projection coefficients (t + 2)
constexpr int kSmRed = kSmH + kBMaxT + 8;             // reductions (4 x warps)
constexpr int kSmSig = kSmRed + 4 * kBW;              // unsorted sigma (t)
constexpr int kSmPart = kSmSig + kBMaxT;               // cluster partials: 2 x (t + 8)
constexpr int kSmRowPart = kSmPart + 2 * (kBMaxT + 8);  // projection partials: 8 x (t + 8)
constexpr int kSmDoubles = kSmRowPart + 8 * (kBMaxT + 8);
// floats after the doubles: Q_U (t x k, row c at Q + c kBMaxK), Q_V (the same), h32 (t + 2)
constexpr int kSmQU = 0;
constexpr int kSmQV = kSmQU + kBMaxT * kBMaxK;
constexpr int kSmH32 = kSmQV + kBMaxT * kBMaxK;
constexpr int kSmFloats = kSmH32 + kBMaxT + 8;
constexpr size_t kSmBytes = sizeof(double) * kSmDoubles + sizeof(float) * kSmFloats + 64;

// ------------------------------------------------------------ CTA helpers

// Deterministic CTA sum: every thread adds the warp partials in the same order.
__device__ __forceinline__ double cta_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kBW; w++) t += red[w];
    return t;
}

template <int G>
__device__ void cta_spmv_g(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                           const float *__restrict__ val, const float *x, int64_t rows,
                           const double *__restrict__ z, double coef, double *__restrict__ y)
{
    const int grp = threadIdx.x / G, lg = threadIdx.x % G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
    constexpr int64_t kStep = kBT / G;
    // the next row's extent is loaded while this row is summed, so a row costs
    // one dependent memory latency (the matrix entries) instead of two
    int64_t e0n = 0, e1n = 0;
    if (grp < rows) { e0n = rp[grp]; e1n = rp[grp + 1]; }
    for (int64_t r = grp; r < rows; r += kStep) {
        const int64_t e0 = e0n, e1 = e1n;
        if (r + kStep < rows) { e0n = rp[r + kStep]; e1n = rp[r + kStep + 1]; }
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        int64_t e = e0 + lg;
        // the matrix streams with evict-first loads, four entries in flight per
        // lane; x was written earlier in this launch by the cluster's CTAs, so it
        // is read with ordinary (coherent) loads, never through the read-only path
        for (; e + 3 * G < e1; e += 4 * G) {
            const int32_t c0 = __ldcs(col + e), c1 = __ldcs(col + e + G);
            const int32_t c2 = __ldcs(col + e + 2 * G), c3 = __ldcs(col + e + 3 * G);
            const float v0 = __ldcs(val + e), v1 = __ldcs(val + e + G);
            const float v2 = __ldcs(val + e + 2 * G), v3 = __ldcs(val + e + 3 * G);
            a0 = fmaf(v0, x[c0], a0);
            a1 = fmaf(v1, x[c1], a1);
            a2 = fmaf(v2, x[c2], a2);
            a3 = fmaf(v3, x[c3], a3);
        }
        for (; e < e1; e += G) a0 = fmaf(__ldcs(val + e), x[__ldcs(col + e)], a0);
        float s = (a0 + a1) + (a2 + a3);
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o);
        if (lg == 0) y[r] = (double)s - (z ? coef * z[r] : 0.0);
    }
}

// y = A x - coef z with FP32 values, FP32 x and FP32 accumulation.  When the
// whole x (xlen entries, 16-byte aligned) fits in the staging region xs, the
// CTA first copies it there, so every gather is a shared-memory load; else
// the gathers go to L1 / L2.  (Splitting a longer x across the cluster's
// shared memory, gathered with ld.shared::cluster, measured slower than the
// L2 gathers: 16.1 s against 12.5 s for the 256-matrix batch.)
__device__ void cta_spmv(int G, const int64_t *rp, const int32_t *col, const float *val, const float *x,
                         int64_t xlen, float *xs, int64_t rows, const double *z, double coef, double *y)
{
    if (xs && xlen <= kXCap) {
        const int64_t n4 = xlen >> 2;
        for (int64_t j = threadIdx.x; j < n4; j += kBT) ((float4 *)xs)[j] = ((const float4 *)x)[j];
        for (int64_t j = 4 * n4 + threadIdx.x; j < xlen; j += kBT) xs[j] = x[j];
        __syncthreads();
        x = xs;
    }
    switch (G) {
    case 1: cta_spmv_g<1>(rp, col, val, x, rows, z, coef, y); break;
    case 2: cta_spmv_g<2>(rp, col, val, x, rows, z, coef, y); break;
    case 4: cta_spmv_g<4>(rp, col, val, x, rows, z, coef, y); break;
    case 8: cta_spmv_g<8>(rp, col, val, x, rows, z, coef, y); break;
    case 16: cta_spmv_g<16>(rp, col, val, x, rows, z, coef, y); break;
    default: cta_spmv_g<32>(rp, col, val, x, rows, z, coef, y); break;
    }
    __syncthreads();
}

// h[c] = W(:, c)^T w for c < ncols.  Work items are (TC columns) x (one of
// kRowParts row ranges), spread over the warps so that all of them stay busy
// even when ncols is a little above a multiple of the warp count; each lane
// keeps 4 rows x (TC + 1) independent loads in flight.  Partial sums per row
// range go to shared memory and are added in range order.
constexpr int kRowParts = 8;

template <typename WT, int TC>
__device__ void cta_proj_t(const WT *__restrict__ W, int64_t ld, int ncols, const WT *w,
                           int64_t len, double *h, double *part)
{
    using AT = WT;  // FP32 products and sums for the FP32 shadow, FP64 otherwise
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ngroups = (ncols + TC - 1) / TC;
    const int items = ngroups * kRowParts;
    for (int it = warp; it < items; it += kBW) {
        const int g = it / kRowParts, rp = it % kRowParts;
        const int c0 = g * TC;
        const int64_t rbeg = len * rp / kRowParts, rend = len * (rp + 1) / kRowParts;
        AT acc[TC];
#pragma unroll
        for (int q = 0; q < TC; q++) acc[q] = AT(0);
        const WT *col[TC];
#pragma unroll
        for (int q = 0; q < TC; q++) col[q] = W + (int64_t)min(c0 + q, ncols - 1) * ld;
        int64_t r = rbeg + lane;
        for (; r + 96 < rend; r += 128) {
            AT wr[4];
            WT v[TC][4];
#pragma unroll
            for (int u = 0; u < 4; u++) wr[u] = (AT)w[r + 32 * u];  // written in this launch: coherent loads
#pragma unroll
            for (int q = 0; q < TC; q++)
#pragma unroll
                for (int u = 0; u < 4; u++) v[q][u] = __ldcs(col[q] + r + 32 * u);
#pragma unroll
            for (int q = 0; q < TC; q++)
#pragma unroll
                for (int u = 0; u < 4; u++) acc[q] = fma((AT)v[q][u], wr[u], acc[q]);
        }
        for (; r < rend; r += 32) {
            const AT wr = (AT)w[r];
#pragma unroll
            for (int q = 0; q < TC; q++) acc[q] = fma((AT)col[q][r], wr, acc[q]);
        }
#pragma unroll
        for (int q = 0; q < TC; q++) {
            double sum = (double)acc[q];
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (lane == 0 && c0 + q < ncols) part[rp * (kBMaxT + 8) + c0 + q] = sum;
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < ncols; c += kBT) {
        double sum = 0.0;
#pragma unroll
        for (int rp = 0; rp < kRowParts; rp++) sum += part[rp * (kBMaxT + 8) + c];
        h[c] = sum;
    }
    __syncthreads();
}

// w has the type of W: the FP32 pass reads an FP32 copy of the vector
// (double -> float conversions run on the FP64 pipe)
template <typename WT>
__device__ void cta_proj(int tc, const WT *W, int64_t ld, int ncols, const WT *w, int64_t len, double *h,
                         double *part)
{
    if (tc >= 4) cta_proj_t<WT, 4>(W, ld, ncols, w, len, h, part);
    else if (tc == 2) cta_proj_t<WT, 2>(W, ld, ncols, w, len, h, part);
    else cta_proj_t<WT, 1>(W, ld, ncols, w, len, h, part);
}

// w -= W h; returns sum of the new w^2 (CTA-wide, deterministic) if asked.
// Each thread owns two adjacent rows and keeps 8 column loads in flight.
template <typename WT, typename HT>
__device__ double cta_update(const WT *__restrict__ W, int64_t ld, int ncols, const HT *__restrict__ h,
                             double *__restrict__ w, int64_t len, bool want_norm, double *red)
{
    double nrm = 0.0;
    for (int64_t r = 2 * threadIdx.x; r < len; r += 2 * kBT) {
        const bool two = r + 1 < len;
        WT a0 = WT(0), a1 = WT(0), b0 = WT(0), b1 = WT(0);
        int c = 0;
        if (two) {
            for (; c + 3 < ncols; c += 4) {
                WT x[4], y[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    x[u] = __ldcs(W + r + (int64_t)(c + u) * ld);
                    y[u] = __ldcs(W + r + 1 + (int64_t)(c + u) * ld);
                }
                a0 = fma(x[0], (WT)h[c], a0); a1 = fma(y[0], (WT)h[c], a1);
                b0 = fma(x[1], (WT)h[c + 1], b0); b1 = fma(y[1], (WT)h[c + 1], b1);
                a0 = fma(x[2], (WT)h[c + 2], a0); a1 = fma(y[2], (WT)h[c + 2], a1);
                b0 = fma(x[3], (WT)h[c + 3], b0); b1 = fma(y[3], (WT)h[c + 3], b1);
            }
            for (; c < ncols; c++) {
                a0 = fma(W[r + (int64_t)c * ld], (WT)h[c], a0);
                a1 = fma(W[r + 1 + (int64_t)c * ld], (WT)h[c], a1);
            }
            const double n0 = w[r] - (double)(a0 + b0);
            const double n1 = w[r + 1] - (double)(a1 + b1);
            w[r] = n0;
            w[r + 1] = n1;
            nrm = fma(n0, n0, nrm);
            nrm = fma(n1, n1, nrm);
        } else {
            for (; c < ncols; c++) a0 = fma(W[r + (int64_t)c * ld], (WT)h[c], a0);
            const double n0 = w[r] - (double)a0;
            w[r] = n0;
            nrm = fma(n0, n0, nrm);
        }
    }
    __syncthreads();
    return want_norm ? cta_sum(nrm, red) : 0.0;
}

__device__ double cta_norm2(const double *w, int64_t len, double *red)
{
    double nrm = 0.0;
    for (int64_t r = threadIdx.x; r < len; r += kBT) nrm = fma(w[r], w[r], nrm);
    return cta_sum(nrm, red);
}

__device__ void cta_scale(double *w, float *w32, int64_t len, double inv)
{
    for (int64_t r = threadIdx.x; r < len; r += kBT) {
        const double x = w[r] * inv;
        w[r] = x;
        w32[r] = (float)x;
    }
    __syncthreads();
}

struct BRun {
    float *wf;
    const BMat *M;
    BStat *st;
    double *U, *V, *Ua, *Va, *T;
    float *U32, *V32, *U32a, *V32a;
    int64_t ldu, ldv, m, n;
    int64_t m0, m1, n0, n1;   // this CTA's rows of the u-side and v-side vectors
    int t, k, tc;
    uint32_t rank, csize;
    int phase;                 // which partial buffer the next cluster reduction uses
    uint64_t key, draws;
    double anorm;
    double *sm;
    float *smf;
    float *xs;                 // staging region of the products' input vector
    bool failed;
    bool lead;                 // rank 0 of the cluster writes the per-matrix outputs
    long long cyc[5];          // SM cycles per phase (see BStat::cycles_phase)
};

__device__ __forceinline__ double *Tb(BRun &R, int r, int c) { return R.T + r + (int64_t)c * (R.t + 1); }

// The partial buffer the next reduction writes into.
__device__ __forceinline__ double *part_buf(BRun &R) { return R.sm + kSmPart + R.phase * (kBMaxT + 8); }

// Cluster reduction: every CTA wrote `cnt` partial values into part_buf(R);
// out[c] = sum over ranks (in rank order) of those values, identical in every
// CTA.  Double-buffered: one cluster barrier per reduction suffices, because a
// buffer is rewritten only after a later barrier that every CTA reached after
// reading it.
__device__ void cl_gather(BRun &R, int cnt, double *out)
{
    const double *buf = part_buf(R);
    __syncthreads();
    cl_sync();
    for (int c = threadIdx.x; c < cnt; c += kBT) {
        double s = 0.0;
        for (uint32_t q = 0; q < R.csize; q++) s += cl_ld(buf + c, q);
        out[c] = s;
    }
    R.phase ^= 1;
    __syncthreads();
}

__device__ double cl_sum_scalar(BRun &R, double v)
{
    double *buf = part_buf(R);
    if (threadIdx.x == 0) buf[0] = v;
    double *tmp = R.sm + kSmRed + 2 * kBW;
    cl_gather(R, 1, tmp);
    return tmp[0];
}

// CGS2 of the column w (this CTA's rows [r0, r1)) against ncols columns:
// pass 1 on the FP32 shadow, pass 2 in FP64.  Returns the cluster-wide ||w||^2.
__device__ double cl_cgs2(BRun &R, const double *W, const float *W32, int64_t ld, int ncols, double *w,
                          int64_t r0, int64_t r1)
{
    double *red = R.sm + kSmRed, *h = R.sm + kSmH;
    float *h32 = R.smf + kSmH32;
    const int64_t len = r1 - r0;
    if (ncols <= 0) return cl_sum_scalar(R, cta_norm2(w + r0, len, red));
    const long long c0 = clock64();
    for (int64_t j = threadIdx.x; j < len; j += kBT) R.wf[r0 + j] = (float)w[r0 + j];
    __syncthreads();
    cta_proj<float>(R.tc, W32 + r0, ld, ncols, R.wf + r0, len, part_buf(R), R.sm + kSmRowPart);
    cl_gather(R, ncols, h);
    for (int c = threadIdx.x; c < ncols; c += kBT) h32[c] = (float)h[c];
    __syncthreads();
    cta_update<float, float>(W32 + r0, ld, ncols, h32, w + r0, len, false, red);
    const long long c1 = clock64();
    cta_proj<double>(R.tc, W + r0, ld, ncols, w + r0, len, part_buf(R), R.sm + kSmRowPart);
    cl_gather(R, ncols, h);
    const double n2 = cl_sum_scalar(R, cta_update<double, double>(W + r0, ld, ncols, h, w + r0, len, true, red));
    R.cyc[1] += c1 - c0;
    R.cyc[2] += clock64() - c1;
    return n2;
}

// Normalises the freshly orthogonalized column `col` of side (0: U, 1: V);
// a breakdown (norm <= 1e-13 * largest alpha/beta/sigma so far) draws random
// replacement vectors.  Returns the T entry (0 after a breakdown).  Ends with
// a cluster barrier so every CTA sees the whole vector.
__device__ double finish_vector(BRun &R, int side, int col, double nrm2)
{
    const int64_t r0 = side ? R.n0 : R.m0, r1 = side ? R.n1 : R.m1;
    double *W = side ? R.V : R.U;
    float *W32 = side ? R.V32 : R.U32;
    const int64_t ld = side ? R.ldv : R.ldu;
    double *w = W + (int64_t)col * ld;
    float *w32 = W32 + (int64_t)col * ld;
    const double nrm = sqrt(nrm2);
    double out = 0.0;
    if (!isfinite(nrm)) {
        R.failed = true;
        if (threadIdx.x == 0 && R.lead) R.st->err = SVDSC_ERR_NONFINITE;
    } else if (nrm > 1e-13 * R.anorm) {
        if (nrm > R.anorm) R.anorm = nrm;
        cta_scale(w + r0, w32 + r0, r1 - r0, 1.0 / nrm);
        out = nrm;
    } else {
        if (threadIdx.x == 0 && R.lead) R.st->breakdowns++;
        bool done = false;
        for (int attempt = 0; attempt < 8 && !done; attempt++) {
            const uint64_t d = R.draws++;
            for (int64_t j = r0 + threadIdx.x; j < r1; j += kBT) w[j] = normal_draw(R.key, d, (uint64_t)j);
            __syncthreads();
            const double nr = sqrt(cl_cgs2(R, W, W32, ld, col, w, r0, r1));
            if (nr > 1e-8 && isfinite(nr)) {
                cta_scale(w + r0, w32 + r0, r1 - r0, 1.0 / nr);
                done = true;
            }
        }
        if (!done) {
            for (int64_t j = r0 + threadIdx.x; j < r1; j += kBT) { w[j] = 0.0; w32[j] = 0.f; }
            __syncthreads();
        }
    }
    cl_sync();
    return out;
}

// Alg. 1 for iterations i = s..t (u_{t+1} not formed)
__device__ void lbp_from(BRun &R, int s)
{
    const BMat &M = *R.M;
    double *red = R.sm + kSmRed;
    (void)red;
    for (int i = s; i <= R.t && !R.failed; i++) {
        // v_{i+1} = A^T u_i - alpha_i v_i, CGS2 against v_1..v_i
        double *vout = R.V + (int64_t)i * R.ldv;
        long long c0 = clock64();
        cta_spmv(M.gAT, M.rpT + R.n0, M.colT, M.valT, R.U32 + (int64_t)(i - 1) * R.ldu, R.m, R.xs, R.n1 - R.n0,
                 R.V + (int64_t)(i - 1) * R.ldv + R.n0, *Tb(R, i - 1, i - 1), vout + R.n0);
        R.cyc[0] += clock64() - c0;
        double n2 = cl_cgs2(R, R.V, R.V32, R.ldv, i, vout, R.n0, R.n1);
        c0 = clock64();
        const double beta = finish_vector(R, 1, i, n2);
        R.cyc[3] += clock64() - c0;
        if (threadIdx.x == 0) *Tb(R, i - 1, i) = beta;
        __syncthreads();
        if (threadIdx.x == 0 && R.lead) { R.st->n_matvec++; R.st->n_steps++; }
        if (i == R.t) break;
        // u_{i+1} = A v_{i+1} - beta_i u_i, CGS2 against u_1..u_i
        double *uout = R.U + (int64_t)i * R.ldu;
        c0 = clock64();
        cta_spmv(M.gA, M.rp + R.m0, M.col, M.val, R.V32 + (int64_t)i * R.ldv, R.n, R.xs, R.m1 - R.m0,
                 R.U + (int64_t)(i - 1) * R.ldu + R.m0, beta, uout + R.m0);
        R.cyc[0] += clock64() - c0;
        n2 = cl_cgs2(R, R.U, R.U32, R.ldu, i, uout, R.m0, R.m1);
        c0 = clock64();
        const double alpha = finish_vector(R, 0, i, n2);
        R.cyc[3] += clock64() - c0;
        if (threadIdx.x == 0) *Tb(R, i, i) = alpha;
        __syncthreads();
        if (threadIdx.x == 0 && R.lead) { R.st->n_matvec++; R.st->n_steps++; }
    }
}

// Projected SVD of T(1:t,1:t) by one-sided Jacobi in shared memory (FP64,
// round-robin pairs, eight lanes per pair), computed by every CTA of the cluster
// on identical input.  Leaves the descending sigma in sm[kSmS], Uh(t, j) in
// sm[kSmUt] and the leading k columns of Uh and Vh (as FP32) in the Q buffers.
__device__ void cta_small_svd(BRun &R)
{
    const int t = R.t, k = R.k;
    double *B = R.sm + kSmB, *Wm = R.sm + kSmW, *sig = R.sm + kSmSig, *S = R.sm + kSmS, *ut = R.sm + kSmUt;
    float *QU = R.smf + kSmQU, *QV = R.smf + kSmQV;
    __shared__ int rot_count;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kLP = 8;  // lanes per column pair (t <= 80: at most 40 pairs, 64 groups)
    const int grp = threadIdx.x / kLP, gl = threadIdx.x % kLP;
    const unsigned gmask = 0xFFu << (lane & ~(kLP - 1));
    const int n2 = t + (t & 1);
    // FP32 preconditioning: the same round-robin sweeps on an FP32 copy of T
    // (scaled by a power of two to max |T| < 1) and an FP32 W, both inside B's
    // region, until every pair is orthogonal to 1e-5 (at most 12 sweeps); the
    // FP32 pipe has ~64x the FP64 one's rate, and the FP64 sweeps below then
    // only remove what FP32 cannot resolve (two or three instead of eight or
    // more).  W is then orthonormalized in FP64 (CGS2) and B = T W is formed
    // in FP64, so the FP64 sweeps keep the invariant B = T W exactly.
    {
        float *B32 = (float *)B, *W32 = (float *)B + t * t;
        __shared__ unsigned s_exp, s_off;
        if (threadIdx.x == 0) s_exp = 0u;
        __syncthreads();
        unsigned emax = 0u;
        for (int i = threadIdx.x; i < t * t; i += kBT) {
            const double x = *Tb(R, i % t, i / t);
            const unsigned ex = (unsigned)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FFu;
            if (ex != 0x7FFu && ex > emax) emax = ex;
        }
        atomicMax(&s_exp, emax);
        __syncthreads();
        const int eb = s_exp == 0u ? 0 : (int)s_exp - 1022;
        const double scale = ldexp(1.0, -max(-1000, min(1000, eb)));
        for (int i = threadIdx.x; i < t * t; i += kBT) {
            const int r = i % t, c = i / t;
            B32[i] = (float)(*Tb(R, r, c) * scale);
            W32[i] = (r == c) ? 1.f : 0.f;
        }
        __syncthreads();
        const float tol32 = FLT_EPSILON * sqrtf((float)t);
        for (int sw = 0; sw < 12; sw++) {
            if (threadIdx.x == 0) s_off = 0u;
            __syncthreads();
            for (int round = 0; round < n2 - 1; round++) {
                for (int slot = grp; slot < n2 / 2; slot += kBT / kLP) {
                    auto player = [&](int pos) { return pos == 0 ? 0 : ((pos - 1 + round) % (n2 - 1)) + 1; };
                    int p = player(slot), q = player(n2 - 1 - slot);
                    if (p > q) { const int x = p; p = q; q = x; }
                    if (q >= t) continue;
                    float *bp = B32 + p * t, *bq = B32 + q * t;
                    float a = 0.f, b = 0.f, g = 0.f;
                    for (int r = gl; r < t; r += kLP) {
                        const float x = bp[r], y = bq[r];
                        a = fmaf(x, x, a);
                        b = fmaf(y, y, b);
                        g = fmaf(x, y, g);
                    }
#pragma unroll
                    for (int o = kLP / 2; o > 0; o >>= 1) {
                        a += __shfl_xor_sync(gmask, a, o);
                        b += __shfl_xor_sync(gmask, b, o);
                        g += __shfl_xor_sync(gmask, g, o);
                    }
                    const float den = sqrtf(a * b);
                    if (gl == 0 && den > 0.f) {
                        const float rel = fabsf(g) / den;
                        if (rel == rel) atomicMax(&s_off, __float_as_uint(rel));
                    }
                    if (g == 0.f || !(fabsf(g) > tol32 * den)) continue;
                    const float d = b - a, g2 = 2.f * g;
                    const float rr = sqrtf(fmaf(d, d, g2 * g2));
                    const bool neg = d != 0.f && ((d > 0.f) != (g > 0.f));
                    const float tn = (neg ? -fabsf(g2) : fabsf(g2)) / (fabsf(d) + rr);
                    if (!(fabsf(tn) <= 1.f)) continue;  // |tan| <= 1 by construction; drops NaN
                    const float c = rsqrtf(fmaf(tn, tn, 1.f)), sn = c * tn;
                    for (int r = gl; r < t; r += kLP) {
                        const float x = bp[r], y = bq[r];
                        bp[r] = c * x - sn * y;
                        bq[r] = sn * x + c * y;
                    }
                    float *wp = W32 + p * t, *wq = W32 + q * t;
                    for (int r = gl; r < t; r += kLP) {
                        const float x = wp[r], y = wq[r];
                        wp[r] = c * x - sn * y;
                        wq[r] = sn * x + c * y;
                    }
                }
                __syncthreads();
            }
            const bool stop = __uint_as_float(s_off) < 1e-5f;
            __syncthreads();  // every thread has read s_off before it is reset
            if (stop) break;
        }
        for (int i = threadIdx.x; i < t * t; i += kBT) Wm[i] = (double)W32[i];
        __syncthreads();
        // CGS2 in FP64, column by column: W orthonormal to FP64 precision
        double *hb = R.sm + kSmH;  // t + 2 doubles, idle during the projected SVD
        for (int j = 0; j < t; j++) {
            double *wj = Wm + j * t;
            for (int pass = 0; pass < 2 && j > 0; pass++) {
                for (int i = warp; i < j; i += kBW) {
                    const double *wi = Wm + i * t;
                    double d = 0.0;
                    for (int r = lane; r < t; r += 32) d = fma(wi[r], wj[r], d);
                    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
                    if (lane == 0) hb[i] = d;
                }
                __syncthreads();
                for (int r = threadIdx.x; r < t; r += kBT) {
                    double sacc = 0.0;
                    for (int i = 0; i < j; i++) sacc = fma(hb[i], Wm[r + i * t], sacc);
                    wj[r] -= sacc;
                }
                __syncthreads();
            }
            if (warp == 0) {
                double nn = 0.0;
                for (int r = lane; r < t; r += 32) nn = fma(wj[r], wj[r], nn);
                for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
                if (lane == 0) hb[t] = nn;
            }
            __syncthreads();
            const double inv = hb[t] > 0.0 ? 1.0 / sqrt(hb[t]) : 0.0;
            for (int r = threadIdx.x; r < t; r += kBT) wj[r] *= inv;
            __syncthreads();
        }
        // B = T W (FP64; B32 and W32 are no longer needed)
        for (int i = threadIdx.x; i < t * t; i += kBT) {
            const int r = i % t, jc = i / t;
            double sacc = 0.0;
            for (int c = 0; c < t; c++) sacc = fma(*Tb(R, r, c), Wm[c + jc * t], sacc);
            B[r + jc * t] = sacc;
        }
        __syncthreads();
    }
    const double tol = DBL_EPSILON * sqrt((double)t);
    int sweeps = 0;
    bool conv = false;
    while (sweeps < 100) {
        if (threadIdx.x == 0) rot_count = 0;
        __syncthreads();
        sweeps++;
        for (int round = 0; round < n2 - 1; round++) {
            // one group of kLP lanes per pair: every pair of the round is in flight at once
            for (int slot = grp; slot < n2 / 2; slot += kBT / kLP) {
                auto player = [&](int pos) { return pos == 0 ? 0 : ((pos - 1 + round) % (n2 - 1)) + 1; };
                int p = player(slot), q = player(n2 - 1 - slot);
                if (p > q) { const int x = p; p = q; q = x; }
                if (q >= t) continue;
                double *bp = B + p * t, *bq = B + q * t;
                double a = 0.0, b = 0.0, g = 0.0;
                for (int r = gl; r < t; r += kLP) {
                    a += bp[r] * bp[r];
                    b += bq[r] * bq[r];
                    g += bp[r] * bq[r];
                }
#pragma unroll
                for (int o = kLP / 2; o > 0; o >>= 1) {
                    a += __shfl_xor_sync(gmask, a, o);
                    b += __shfl_xor_sync(gmask, b, o);
                    g += __shfl_xor_sync(gmask, g, o);
                }
                if (g == 0.0 || fabs(g) <= tol * sqrt(a * b)) continue;
                const double zeta = (b - a) / (2.0 * g);
                const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / sqrt(1.0 + tt * tt), s = c * tt;
                if (gl == 0) atomicAdd(&rot_count, 1);
                for (int r = gl; r < t; r += kLP) {
                    const double x = bp[r], y = bq[r];
                    bp[r] = c * x - s * y;
                    bq[r] = s * x + c * y;
                }
                double *wp = Wm + p * t, *wq = Wm + q * t;
                for (int r = gl; r < t; r += kLP) {
                    const double x = wp[r], y = wq[r];
                    wp[r] = c * x - s * y;
                    wq[r] = s * x + c * y;
                }
            }
            __syncthreads();
        }
        if (rot_count == 0) { conv = true; break; }
        __syncthreads();
    }
    for (int j = warp; j < t; j += kBW) {
        double a = 0.0;
        for (int r = lane; r < t; r += 32) a += B[r + j * t] * B[r + j * t];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) sig[j] = sqrt(a);
    }
    __syncthreads();
    for (int j = warp; j < t; j += kBW) {
        const double sj = sig[j];
        int rank = 0;
        for (int i = 0; i < t; i++) rank += (sig[i] > sj) || (sig[i] == sj && i < j);
        if (lane == 0) {
            S[rank] = sj;
            if (rank < k) ut[rank] = sj > 0.0 ? B[(t - 1) + j * t] / sj : 0.0;
        }
        if (rank < k)
            for (int r = lane; r < t; r += 32) {
                QU[rank + r * kBMaxK] = sj > 0.0 ? (float)(B[r + j * t] / sj) : 0.f;
                QV[rank + r * kBMaxK] = (float)Wm[r + j * t];
            }
    }
    __syncthreads();
    if (threadIdx.x == 0 && R.lead) R.st->svd_sweeps = conv ? sweeps : -1;
}

// C (rows x k) = W32 (rows x t) Q (t x k, FP32 in shared memory, row c of Q
// at Q + c kBMaxK), FP32 FMA, each output summed over c in order; C in FP64
// (and its FP32 shadow when C32 != null).  KB (k rounded up to 16) accumulators
// per row; a row of Q is read as float4, and the next W entry is loaded while
// the current one is used.
template <int KB>
__device__ void cta_gemm32_k(const float *__restrict__ W32, int64_t ld, int64_t rows, int t, const float *Q,
                             int k, double *__restrict__ C, float *__restrict__ C32, int64_t ldc)
{
    for (int64_t r = threadIdx.x; r < rows; r += kBT) {
        float acc[KB];
#pragma unroll
        for (int j = 0; j < KB; j++) acc[j] = 0.f;
        float a_next = t > 0 ? W32[r] : 0.f;
        for (int c = 0; c < t; c++) {
            const float a = a_next;
            if (c + 1 < t) a_next = W32[r + (int64_t)(c + 1) * ld];
            const float4 *q = (const float4 *)(Q + c * kBMaxK);
#pragma unroll
            for (int jj = 0; jj < KB / 4; jj++) {
                const float4 qv = q[jj];
                acc[4 * jj] = fmaf(a, qv.x, acc[4 * jj]);
                acc[4 * jj + 1] = fmaf(a, qv.y, acc[4 * jj + 1]);
                acc[4 * jj + 2] = fmaf(a, qv.z, acc[4 * jj + 2]);
                acc[4 * jj + 3] = fmaf(a, qv.w, acc[4 * jj + 3]);
            }
        }
#pragma unroll
        for (int j = 0; j < KB; j++)
            if (j < k) {
                C[r + (int64_t)j * ldc] = (double)acc[j];
                if (C32) C32[r + (int64_t)j * ldc] = acc[j];
            }
    }
    __syncthreads();
}

__device__ void cta_gemm32(const float *__restrict__ W32, int64_t ld, int64_t rows, int t, const float *Q, int k,
                           double *__restrict__ C, float *__restrict__ C32, int64_t ldc)
{
    static_assert(kBMaxK == 48, "accumulator buckets");
    if (k <= 16) cta_gemm32_k<16>(W32, ld, rows, t, Q, k, C, C32, ldc);
    else if (k <= 32) cta_gemm32_k<32>(W32, ld, rows, t, Q, k, C, C32, ldc);
    else cta_gemm32_k<48>(W32, ld, rows, t, Q, k, C, C32, ldc);
}

// sign rule: v_j's largest-magnitude entry (lowest index on ties) positive;
// the argmax is combined over the cluster in rank order.
__device__ void cl_sign(BRun &R, double *U, int64_t ldU, double *V, int64_t ldV)
{
    __shared__ double sb[kBW];
    __shared__ int64_t si[kBW];
    for (int j = 0; j < R.k; j++) {
        double *v = V + (int64_t)j * ldV;
        double best = -1.0;
        int64_t bi = R.n0;
        for (int64_t r = R.n0 + threadIdx.x; r < R.n1; r += kBT) {
            const double a = fabs(v[r]);
            if (a > best) { best = a; bi = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double b2 = __shfl_xor_sync(0xffffffffu, best, o);
            const int64_t i2 = __shfl_xor_sync(0xffffffffu, bi, o);
            if (b2 > best || (b2 == best && i2 < bi)) { best = b2; bi = i2; }
        }
        __syncthreads();
        if ((threadIdx.x & 31) == 0) { sb[threadIdx.x >> 5] = best; si[threadIdx.x >> 5] = bi; }
        __syncthreads();
        double *buf = part_buf(R);
        if (threadIdx.x == 0) {
            double bb = sb[0];
            int64_t ii = si[0];
            for (int w = 1; w < kBW; w++)
                if (sb[w] > bb || (sb[w] == bb && si[w] < ii)) { bb = sb[w]; ii = si[w]; }
            buf[0] = bb;
            buf[1] = (double)ii;
            buf[2] = (ii >= R.n0 && ii < R.n1) ? v[ii] : 0.0;
        }
        __syncthreads();
        cl_sync();
        double bb = -2.0, val = 0.0;
        int64_t ii = 0;
        for (uint32_t q = 0; q < R.csize; q++) {
            const double b2 = cl_ld(buf, q);
            const int64_t i2 = (int64_t)cl_ld(buf + 1, q);
            if (b2 > bb || (b2 == bb && i2 < ii)) { bb = b2; ii = i2; val = cl_ld(buf + 2, q); }
        }
        R.phase ^= 1;
        if (val < 0.0) {
            for (int64_t r = R.n0 + threadIdx.x; r < R.n1; r += kBT) v[r] = -v[r];
            double *u = U + (int64_t)j * ldU;
            for (int64_t r = R.m0 + threadIdx.x; r < R.m1; r += kBT) u[r] = -u[r];
        }
        __syncthreads();
    }
}

// u_{k+1} = A v_{k+1} - U~ rho (Eq. 7), CGS2 against U~, alpha_{k+1}: the part
// of the augmented restart after the restart GEMM and the new T.
__device__ void restart_tail(BRun &R, const double *rho, double *red)
{
    const BMat &M = *R.M;
    const int k = R.k;
    double *uk = R.U + (int64_t)k * R.ldu;
    cta_spmv(M.gA, M.rp + R.m0, M.col, M.val, R.V32 + (int64_t)k * R.ldv, R.n, R.xs, R.m1 - R.m0, nullptr, 0.0,
             uk + R.m0);
    cta_update<double, double>(R.U + R.m0, R.ldu, k, rho, uk + R.m0, R.m1 - R.m0, false, red);
    const double n2 = cl_cgs2(R, R.U, R.U32, R.ldu, k, uk, R.m0, R.m1);
    const double ak = finish_vector(R, 0, k, n2);
    if (threadIdx.x == 0) *Tb(R, k, k) = ak;
    if (threadIdx.x == 0 && R.lead) { R.st->n_matvec++; R.st->n_steps++; }
    __syncthreads();
}

// Hand-off copies of this CTA's rows between the cluster's bases (ld ldu,
// ldv) and the matrix's global state (U~_k in MU, V~_k in MV, v_{k+1} in ckv;
// leading dimensions m, n).  to_global: save, else load (with the FP32
// shadows, the FP32 roundings of the FP64 values as the restart GEMM wrote
// them).  Out of line: both run once per hand-off, and keeping them out of
// the solver loop keeps its register allocation unchanged.
__device__ __noinline__ void handoff_rows(bool to_global, double *MU, double *MV, double *ckv, int64_t m,
                                          int64_t n, double *U, float *U32, int64_t ldu, double *V, float *V32,
                                          int64_t ldv, int64_t m0, int64_t m1, int64_t n0, int64_t n1, int k)
{
    for (int j = 0; j <= k; j++) {
        if (j < k)
            for (int64_t r = m0 + threadIdx.x; r < m1; r += kBT) {
                if (to_global) {
                    MU[r + (int64_t)j * m] = U[r + (int64_t)j * ldu];
                } else {
                    const double x = MU[r + (int64_t)j * m];
                    U[r + (int64_t)j * ldu] = x;
                    U32[r + (int64_t)j * ldu] = (float)x;
                }
            }
        double *src = j < k ? MV + (int64_t)j * n : ckv;  // column k: v_{k+1}
        for (int64_t r = n0 + threadIdx.x; r < n1; r += kBT) {
            if (to_global) {
                src[r] = V[r + (int64_t)j * ldv];
            } else {
                const double x = src[r];
                V[r + (int64_t)j * ldv] = x;
                V32[r + (int64_t)j * ldv] = (float)x;
            }
        }
    }
    __syncthreads();
}

// One matrix on this cluster.  mode 0: from the start; the matrix may be
// handed off at a restart boundary (once P.handoff_idle clusters of this
// launch found the queue empty), and is then finished by the second launch
// (mode 1), which resumes from the saved state.  Returns nothing; the
// outputs, or the hand-off state, are in global memory.
__device__ void solve_one(const BMat &M, int b, BStat *st, const BSlot &slot, double *Tpriv, const BParams &P,
                          double *sm, float *smf, int &phase, int mode, BQueue *q, int *ho_list)
{
    BRun R;
    R.M = &M;
    R.wf = slot.wf;
    R.st = st;
    R.U = slot.U0; R.Ua = slot.U1; R.V = slot.V0; R.Va = slot.V1; R.T = Tpriv;
    R.U32 = slot.U32_0; R.U32a = slot.U32_1; R.V32 = slot.V32_0; R.V32a = slot.V32_1;
    R.ldu = slot.ldu; R.ldv = slot.ldv; R.m = M.m; R.n = M.n; R.t = M.t; R.k = M.k; R.tc = M.tc;
    R.rank = cl_rank();
    R.csize = cl_size();
    R.lead = R.rank == 0;
    R.m0 = M.m * R.rank / R.csize; R.m1 = M.m * (R.rank + 1) / R.csize;
    R.n0 = M.n * R.rank / R.csize; R.n1 = M.n * (R.rank + 1) / R.csize;
    R.phase = phase;
    R.key = splitmix_mix(M.seed);
    R.draws = 0;
    R.anorm = 0.0;
    R.sm = sm;
    R.smf = smf;
    R.xs = (float *)(sm + kSmB);
    R.failed = false;
    for (int q2 = 0; q2 < 5; q2++) R.cyc[q2] = 0;
    double *red = sm + kSmRed;
    const int t = R.t, k = R.k;
    const long long c_start = clock64();
    long long c_svd = 0, c_lbp = 0;
    int restarts = 0, it0 = 1;
    if (mode != 1) {
        if (threadIdx.x == 0 && R.lead) {
            st->converged = 0; st->nconv = 0; st->restarts = 0; st->breakdowns = 0;
            st->n_matvec = 0; st->n_steps = 0; st->err = 0; st->svd_sweeps = 0;
            st->cluster = (mode == 2 ? 200000 : 0) + (int)cl_id();
            for (int q2 = 0; q2 < 5; q2++) st->cycles_phase[q2] = 0;
        }
        for (int64_t i = threadIdx.x; i < (int64_t)(t + 1) * (t + 1); i += kBT) R.T[i] = 0.0;
        // v_1: draw 0, normalised
        for (int64_t j = R.n0 + threadIdx.x; j < R.n1; j += kBT) R.V[j] = normal_draw(R.key, 0, (uint64_t)j);
        R.draws = 1;
        __syncthreads();
        {
            const double nv = sqrt(cl_sum_scalar(R, cta_norm2(R.V + R.n0, R.n1 - R.n0, red)));
            cta_scale(R.V + R.n0, R.V32 + R.n0, R.n1 - R.n0, 1.0 / nv);
            cl_sync();
        }
        // u_1 = A v_1, alpha_1
        cta_spmv(M.gA, M.rp + R.m0, M.col, M.val, R.V32, R.n, R.xs, R.m1 - R.m0, nullptr, 0.0, R.U + R.m0);
        {
            const double a1 = finish_vector(R, 0, 0, cl_sum_scalar(R, cta_norm2(R.U + R.m0, R.m1 - R.m0, red)));
            if (threadIdx.x == 0) *Tb(R, 0, 0) = a1;
            if (threadIdx.x == 0 && R.lead) { st->n_matvec++; st->n_steps++; }
            __syncthreads();
        }
        const long long c0 = clock64();
        lbp_from(R, 1);
        c_lbp += clock64() - c0;
    } else {
        // resume: this CTA's rows of U~_k, V~_k and v_{k+1} (FP32 shadows are
        // the FP32 roundings of the FP64 values, as the restart GEMM wrote
        // them), T = [diag(sigma) rho], the restart coefficients, the counters
        const BHand *H = M.hand;
        handoff_rows(false, M.U, M.V, M.ckv, M.m, M.n, R.U, R.U32, R.ldu, R.V, R.V32, R.ldv, R.m0, R.m1, R.n0,
                     R.n1, k);
        for (int64_t i = threadIdx.x; i < (int64_t)(t + 1) * (t + 1); i += kBT) R.T[i] = 0.0;
        __syncthreads();
        if (threadIdx.x < k) {
            const int j = threadIdx.x;
            *Tb(R, j, j) = H->S[j];
            *Tb(R, j, k) = H->rho[j];
            sm[kSmRho + j] = H->rho[j];
        }
        R.anorm = H->anorm;
        R.draws = H->draws;
        restarts = H->restarts;
        it0 = H->it;  // the first pass of the loop finishes that restart
        if (threadIdx.x == 0 && R.lead) st->cluster = 100000 + (int)cl_id();
        __syncthreads();
    }
    bool resume = mode == 1;
    for (int it = it0; it <= P.maxit && !R.failed; it++) {
        double *rho = sm + kSmRho;
        if (!resume) {
        {
            const long long c0 = clock64();
            cta_small_svd(R);
            c_svd += clock64() - c0;
        }
        const double *S = sm + kSmS, *ut = sm + kSmUt;
        const double beta_t = *Tb(R, t - 1, t);
        if (S[0] > R.anorm) R.anorm = S[0];
        int nconv = 0;
        for (int j = 0; j < k; j++) {
            const double den = S[j] > DBL_EPSILON * S[0] ? S[j] : DBL_EPSILON * S[0];
            const double r = den > 0.0 ? fabs(beta_t * ut[j]) / den : 0.0;
            nconv += (r < P.tol);
        }
        if (threadIdx.x < k) {
            const int j = threadIdx.x;
            const double den = S[j] > DBL_EPSILON * S[0] ? S[j] : DBL_EPSILON * S[0];
            if (R.lead) M.res[j] = den > 0.0 ? fabs(beta_t * ut[j]) / den : 0.0;
            rho[j] = beta_t * ut[j];
        }
        if (threadIdx.x == 0 && R.lead) { st->nconv = nconv; st->converged = (nconv == k); st->beta_t = beta_t; }
        __syncthreads();
        if (nconv == k || it == P.maxit) break;
        // augmented restart: this CTA's rows of U~ = U(:,1:t) Uh(:,1:k), V~ = V(:,1:t) Vh(:,1:k)
        const long long cg = clock64();
        cta_gemm32(R.U32 + R.m0, R.ldu, R.m1 - R.m0, t, R.smf + kSmQU, k, R.Ua + R.m0, R.U32a + R.m0, R.ldu);
        cta_gemm32(R.V32 + R.n0, R.ldv, R.n1 - R.n0, t, R.smf + kSmQV, k, R.Va + R.n0, R.V32a + R.n0, R.ldv);
        R.cyc[4] += clock64() - cg;
        for (int64_t j = R.n0 + threadIdx.x; j < R.n1; j += kBT) {  // v_{k+1} = v_{t+1}
            R.Va[j + (int64_t)k * R.ldv] = R.V[j + (int64_t)t * R.ldv];
            R.V32a[j + (int64_t)k * R.ldv] = R.V32[j + (int64_t)t * R.ldv];
        }
        {
            double *x = R.U; R.U = R.Ua; R.Ua = x;
            x = R.V; R.V = R.Va; R.Va = x;
            float *y = R.U32; R.U32 = R.U32a; R.U32a = y;
            y = R.V32; R.V32 = R.V32a; R.V32a = y;
        }
        // hand-off test (first launch only): the decision of the cluster's first
        // CTA, read by every CTA through the cluster reduction, so all agree
        if (mode == 0 && P.handoff_idle > 0) {
            double flag = 0.0;
            if (threadIdx.x == 0 && R.lead)
                flag = (*(volatile int *)&q->idle >= P.handoff_idle) ? 1.0 : 0.0;
            if (cl_sum_scalar(R, flag) > 0.5) {
                // save this CTA's rows of U~_k, V~_k, v_{k+1}; the first CTA the rest
                handoff_rows(true, M.U, M.V, M.ckv, M.m, M.n, R.U, R.U32, R.ldu, R.V, R.V32, R.ldv, R.m0, R.m1,
                             R.n0, R.n1, k);
                if (R.lead) {
                    BHand *H = M.hand;
                    for (int j = threadIdx.x; j < k; j += kBT) {
                        H->S[j] = S[j];
                        H->rho[j] = rho[j];
                    }
                    if (threadIdx.x == 0) {
                        H->anorm = R.anorm;
                        H->draws = R.draws;
                        H->restarts = restarts;
                        H->it = it;
                        H->cycles_total = clock64() - c_start;
                        H->work = H->cycles_total * (long long)R.csize;
                        H->cycles_svd = c_svd;
                        H->cycles_lbp = c_lbp;
                        for (int q2 = 0; q2 < 5; q2++) st->cycles_phase[q2] = R.cyc[q2];
                        ho_list[atomicAdd(&q->ho_count, 1)] = b;
                    }
                }
                __syncthreads();
                phase = R.phase;
                return;
            }
        }
        for (int64_t i = threadIdx.x; i < (int64_t)(t + 1) * (t + 1); i += kBT) R.T[i] = 0.0;
        __syncthreads();
        if (threadIdx.x < k) {
            const int j = threadIdx.x;
            *Tb(R, j, j) = S[j];
            *Tb(R, j, k) = rho[j];
        }
        __syncthreads();
        }  // !resume
        resume = false;
        cl_sync();  // v_{k+1} complete on every CTA before the product reads it
        restart_tail(R, rho, red);
        restarts++;
        if (threadIdx.x == 0 && R.lead) st->restarts = restarts;
        const long long c0 = clock64();
        lbp_from(R, k + 1);
        c_lbp += clock64() - c0;
    }
    if (!R.failed) {
        // outputs: S, this CTA's rows of U = U(:,1:t) Uh(:,1:k), V = V(:,1:t) Vh(:,1:k), sign rule
        const long long cg = clock64();
        if (R.lead)
            for (int j = threadIdx.x; j < k; j += kBT) M.S[j] = sm[kSmS + j];
        cta_gemm32(R.U32 + R.m0, R.ldu, R.m1 - R.m0, t, smf + kSmQU, k, M.U + R.m0, nullptr, R.m);
        cta_gemm32(R.V32 + R.n0, R.ldv, R.n1 - R.n0, t, smf + kSmQV, k, M.V + R.n0, nullptr, R.n);
        cl_sign(R, M.U, R.m, M.V, R.n);
        R.cyc[4] += clock64() - cg;
        if (threadIdx.x == 0 && R.lead) st->anorm = R.anorm;
    }
    if (threadIdx.x == 0 && R.lead) {
        long long c_tot = clock64() - c_start;
        long long work = c_tot * (long long)R.csize;
        if (mode == 1) {  // add the first launch's share
            work += M.hand->work;
            c_tot += M.hand->cycles_total;
            c_svd += M.hand->cycles_svd;
            c_lbp += M.hand->cycles_lbp;
        }
        st->cycles_total = c_tot;
        st->work = work;
        st->cycles_svd = c_svd;
        st->cycles_lbp = c_lbp;
        for (int q2 = 0; q2 < 5; q2++) st->cycles_phase[q2] += R.cyc[q2];
    }
    phase = R.phase;
}

// The persistent kernel.  mode 0 takes matrices from the queue order[0..n),
// largest cost first; a cluster that finds it empty counts itself idle and
// leaves.  mode 1 (the second launch, larger clusters) resumes the matrices
// the first launch handed off.  mode 2 (the lead launch: a few larger
// clusters running beside mode 0) takes queue position cl_id() first, the
// costliest matrices, then shares the queue with mode 0; it never hands off
// and is not counted as idle.  A lead launch lets the launch that follows it
// in the stream start as soon as every one of its CTAs is running.
__global__ void __launch_bounds__(kBT, 1)
batched_kernel(const BMat *__restrict__ mats, const int *__restrict__ order, int n, BQueue *q, int *ho_list,
               int mode, BStat *stats, const BSlot *__restrict__ slots, double *Tall, int64_t tstride,
               const BParams *prm)
{
    extern __shared__ __align__(16) double bsm[];
    double *sm = bsm;
    float *smf = (float *)(bsm + kSmDoubles);
    __shared__ int item;
    const BSlot slot = slots[cl_id()];
    double *Tpriv = Tall + (int64_t)blockIdx.x * tstride;
    const BParams P = *prm;
    if (mode == 2) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    int phase = 0;
    bool reserved = mode == 2;
    while (true) {
        __syncthreads();
        cl_sync();  // every CTA has read the previous item
        if (threadIdx.x == 0 && cl_rank() == 0) {
            int b = -1;
            if (mode != 1) {
                const int i = reserved ? (int)cl_id() : atomicAdd(&q->next, 1);
                if (i < n) b = order[i];
                else if (mode == 0) atomicAdd(&q->idle, 1);
            } else {
                const int i = atomicAdd(&q->next2, 1);
                if (i < *(volatile int *)&q->ho_count) b = ho_list[i];
            }
            item = b;
        }
        __syncthreads();
        cl_sync();
        const int b = cl_ld_i32(&item, 0);
        cl_sync();  // no CTA leaves while another still reads its shared memory
        if (b < 0) break;
        reserved = false;
        solve_one(mats[b], b, stats + b, slot, Tpriv, P, sm, smf, phase, mode, q, ho_list);
    }
}

// ------------------------------------------------------------ autotuner
// Times each candidate on one CTA per SM, all running the same product of the
// class representative (the per-SM throughput the persistent kernel sees).
__global__ void __launch_bounds__(kBT, 1)
tune_spmv_kernel(const int64_t *rp, const int32_t *col, const float *val, const float *x, int64_t xlen, int64_t rows,
                 double *y_slots, int64_t ldy, int G, int reps)
{
    extern __shared__ __align__(16) double bsm[];
    double *y = y_slots + (int64_t)blockIdx.x * ldy;
    for (int r = 0; r < reps; r++) cta_spmv(G, rp, col, val, x, xlen, (float *)bsm, rows, nullptr, 0.0, y);
}

__global__ void __launch_bounds__(kBT, 1)
tune_proj_kernel(const double *W_slots, int64_t ldw_slot, int64_t ld, int ncols, const double *w, int64_t len,
                 int tc, int reps)
{
    extern __shared__ __align__(16) double bsm[];
    const double *W = W_slots + (int64_t)blockIdx.x * ldw_slot;
    for (int r = 0; r < reps; r++) cta_proj<double>(tc, W, ld, ncols, w, len, bsm, bsm + (kBMaxT + 8));
}

}  // namespace svdsc

// ============================================================ host side
using namespace svdsc;

// One persistent launch: its cluster size, clusters (one workspace slot
// each, sized for the largest matrix) and a private projected matrix per CTA.
struct BLaunch {
    int csize = 0;
    int nslots = 0;
    void *slot_mem = nullptr;
    BSlot *d_slots = nullptr;
    double *d_T = nullptr;
    size_t slot_bytes = 0;       // bytes of slot_mem
    int64_t t_count = 0;         // doubles of d_T
    bool owns = true;            // false: slot_mem and d_T belong to another launch
};

struct svdsc_batch {
    int nb = 0;
    cudaStream_t stream = nullptr;
    std::vector<DevCSR> A, AT;
    std::vector<BMat> hm;        // host copy of the descriptors
    BMat *h_mats = nullptr;      // pinned staging copy (graph memcpy source)
    BParams *h_prm = nullptr;    // pinned
    BMat *d_mats = nullptr;
    BStat *d_stats = nullptr;
    BParams *d_prm = nullptr;
    int *d_order = nullptr;      // matrix ids, largest (estimated or measured) cost first
    std::vector<int> order;      // host copy of the queue order
    bool reorder = true;         // after a solve, order the queue by the measured cycles
    BQueue *d_q = nullptr;       // queue positions and hand-off counters
    int64_t tstride = 0;
    BLaunch L;                   // the first launch (all matrices)
    BLaunch L2;                  // the second launch (matrices handed off), csize 0 when off
    BLaunch LA;                  // the lead launch beside L (8-CTA clusters), nslots 0 when off
    int handoff_idle = 0;        // hand off once this many clusters of L are idle (0: never)
    BQueue *h_q0 = nullptr;      // pinned: the queue state each solve starts from
    int *d_ho = nullptr;         // hand-off list (nb entries)
    double *ckv_mem = nullptr;   // v_{k+1} of each matrix (sum of n)
    BHand *d_hand = nullptr;     // nb entries
    double *out_mem = nullptr;   // device outputs when the caller wants host outputs
    std::vector<size_t> out_off;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double tune_ms = 0.0;
};

namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, int> g_tune_spmv;    // (avg-len bucket, rows bucket, which) -> G
std::map<std::tuple<int, int>, int> g_tune_proj;         // (len bucket, ncols bucket) -> columns per warp

int bucket(double x) { return (int)std::lround(2.0 * std::log2(std::max(x, 1.0))); }

double time_ms(cudaStream_t s, const std::function<void()> &f)
{
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    f();  // warm
    cudaEventRecord(a, s);
    f();
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}
}  // namespace

static int tune_matrix(svdsc_batch *B, int b, int nsm, double *yscratch, int64_t ldy, float *x32, double *wsc)
{
    BMat &M = B->hm[b];
    const int cand[] = {1, 2, 4, 8, 16, 32};
    for (int which = 0; which < 2; which++) {
        const DevCSR &C = which ? B->AT[b] : B->A[b];
        const double avg = C.m > 0 ? (double)C.nnz / (double)C.m : 1.0;
        const auto key = std::make_tuple(bucket(avg), bucket((double)C.m), which);
        int best = -1;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto f = g_tune_spmv.find(key);
            if (f != g_tune_spmv.end()) best = f->second;
        }
        if (best < 0) {
            double bt = 1e30;
            for (int G : cand) {
                const double ms = time_ms(B->stream, [&] {
                    tune_spmv_kernel<<<nsm, kBT, sizeof(float) * kXCap, B->stream>>>(
                        C.row_ptr, C.col, C.val32, x32, C.n, C.m, yscratch, ldy, G, 2);
                });
                B->tune_ms += 2 * ms;
                if (ms < bt) { bt = ms; best = G; }
            }
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune_spmv[key] = best;
        }
        if (which) M.gAT = best; else M.gA = best;
    }
    {
        const int ncols = std::max(1, M.t / 2);
        const auto key = std::make_tuple(bucket((double)M.m), bucket((double)ncols));
        int best = -1;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto f = g_tune_proj.find(key);
            if (f != g_tune_proj.end()) best = f->second;
        }
        if (best < 0) {
            double bt = 1e30;
            for (int tc : {1, 2, 4}) {
                const double ms = time_ms(B->stream, [&] {
                    tune_proj_kernel<<<nsm, kBT, sizeof(double) * 9 * (kBMaxT + 8), B->stream>>>(
                        wsc, 0, M.m, ncols, wsc, M.m, tc, 2);
                });
                B->tune_ms += 2 * ms;
                if (ms < bt) { bt = ms; best = tc; }
            }
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune_proj[key] = best;
        }
        M.tc = best;
    }
    return cudaGetLastError() == cudaSuccess ? SVDSC_OK : SVDSC_ERR_CUDA;
}

extern "C" {

static void free_launch(BLaunch &L)
{
    if (L.owns) {
        cudaFree(L.slot_mem);
        cudaFree(L.d_T);
    }
    cudaFree(L.d_slots);
    L = BLaunch();
}

int svdsc_batch_destroy(svdsc_batch *B)
{
    if (!B) return SVDSC_OK;
    if (B->stream) cudaStreamSynchronize(B->stream);
    for (auto &a : B->A) csr_free(&a);
    for (auto &a : B->AT) csr_free(&a);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    cudaFreeHost(B->h_mats);
    cudaFreeHost(B->h_prm);
    cudaFreeHost(B->h_q0);
    cudaFree(B->d_mats);
    cudaFree(B->d_stats);
    cudaFree(B->d_prm);
    cudaFree(B->d_order);
    cudaFree(B->d_q);
    cudaFree(B->d_ho);
    cudaFree(B->ckv_mem);
    cudaFree(B->d_hand);
    free_launch(B->L2);  // may alias L's memory: freed first, without it
    free_launch(B->LA);
    free_launch(B->L);
    cudaFree(B->out_mem);
    if (B->stream) cudaStreamDestroy(B->stream);
    delete B;
    return SVDSC_OK;
}

static int max_clusters(int C)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(C * 64);
    cfg.blockDim = dim3(kBT);
    cfg.dynamicSmemBytes = kSmBytes;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, batched_kernel, &cfg) != cudaSuccess) return 0;
    return ncl;
}

// Workspace of one launch: a slot (two sets of bases, FP64 and FP32) per
// cluster, sized for the largest matrix, and a projected matrix per CTA.
// With `alias`, the memory of that launch is reused when it is large enough
// (the two launches run one after the other on one stream).
static int setup_launch(svdsc_batch *B, BLaunch &L, int64_t mmax, int64_t nmax, int tmax,
                        const BLaunch *alias = nullptr)
{
    const int64_t ldu = (mmax + 63) & ~int64_t(63), ldv = (nmax + 63) & ~int64_t(63);
    const int64_t cols = tmax + 2;
    const size_t per_slot = sizeof(double) * (size_t)(2 * ldu * cols + 2 * ldv * cols + 64) +
                            sizeof(float) * (size_t)(2 * ldu * cols + 2 * ldv * cols + std::max(ldu, ldv)) + 4096;
    std::vector<BSlot> slots(L.nslots);
    L.slot_bytes = per_slot * L.nslots;
    L.t_count = B->tstride * L.nslots * L.csize;
    if (alias && alias->slot_bytes >= L.slot_bytes && alias->t_count >= L.t_count) {
        L.slot_mem = alias->slot_mem;
        L.d_T = alias->d_T;
        L.owns = false;
    } else {
        if (cudaMalloc(&L.slot_mem, L.slot_bytes) != cudaSuccess) return SVDSC_ERR_NOMEM;
        cudaMemsetAsync(L.slot_mem, 0, L.slot_bytes, B->stream);
        if (cudaMalloc(&L.d_T, sizeof(double) * L.t_count) != cudaSuccess) return SVDSC_ERR_NOMEM;
    }
    for (int s = 0; s < L.nslots; s++) {
        uint8_t *base = (uint8_t *)L.slot_mem + per_slot * s;
        auto take = [&](size_t bytes) { uint8_t *p = base; base += (bytes + 255) & ~(size_t)255; return p; };
        BSlot &S = slots[s];
        S.ldu = ldu; S.ldv = ldv;
        S.U0 = (double *)take(sizeof(double) * ldu * cols);
        S.U1 = (double *)take(sizeof(double) * ldu * cols);
        S.V0 = (double *)take(sizeof(double) * ldv * cols);
        S.V1 = (double *)take(sizeof(double) * ldv * cols);
        S.U32_0 = (float *)take(sizeof(float) * ldu * cols);
        S.U32_1 = (float *)take(sizeof(float) * ldu * cols);
        S.V32_0 = (float *)take(sizeof(float) * ldv * cols);
        S.V32_1 = (float *)take(sizeof(float) * ldv * cols);
        S.wf = (float *)take(sizeof(float) * std::max(ldu, ldv));
    }
    if (cudaMalloc(&L.d_slots, sizeof(BSlot) * L.nslots) != cudaSuccess) return SVDSC_ERR_NOMEM;
    cudaMemcpyAsync(L.d_slots, slots.data(), sizeof(BSlot) * L.nslots, cudaMemcpyHostToDevice, B->stream);
    return cudaGetLastError() == cudaSuccess ? SVDSC_OK : SVDSC_ERR_CUDA;
}

int svdsc_batch_create(svdsc_batch **out, int nb, const svdsc_matrix *As, const int *k, const int *p,
                       const svdsc_options *opt, void *stream)
{
    (void)stream;
    if (!out || nb < 1 || !As || !k) return SVDSC_ERR_ARG;
    *out = nullptr;
    if (opt && opt->precision != SVDSC_MIXED) return SVDSC_ERR_ARG;  // the batched form is the mixed one
    if (opt && opt->which != SVDSC_LARGEST) return SVDSC_ERR_ARG;    // and keeps the largest triplets
    if (opt && opt->reorth != SVDSC_REORTH_FULL) return SVDSC_ERR_ARG;  // with full re-orthogonalization
    if (opt && opt->block > 1) return SVDSC_ERR_ARG;                  // one vector at a time
    for (int b = 0; b < nb; b++) {
        const svdsc_matrix &a = As[b];
        if (a.format != SVDSC_CSR || a.m < 1 || a.n < 1) return SVDSC_ERR_ARG;
        const int pb = p ? p[b] : -1;
        const int t = pb < 0 ? std::max(15, 3 * k[b]) : k[b] + pb;
        if (k[b] < 1 || k[b] > kBMaxK || t < k[b] || t > kBMaxT || t > a.m || t + 1 > a.n) return SVDSC_ERR_SIZE;
    }
    const int Cfix = opt ? opt->batch_cluster : 0;
    if (Cfix != 0 && Cfix != 1 && Cfix != 2 && Cfix != 4 && Cfix != 8) return SVDSC_ERR_ARG;
    const int Hopt = opt ? opt->batch_handoff : 0;
    if (Hopt < -1) return SVDSC_ERR_ARG;
    const int Oopt = opt ? opt->batch_order : 0;
    if (Oopt != 0 && Oopt != 1) return SVDSC_ERR_ARG;
    const int Aopt = opt ? opt->batch_lead : 0;
    if (Aopt < -1) return SVDSC_ERR_ARG;
    svdsc_batch *B = new (std::nothrow) svdsc_batch();
    if (!B) return SVDSC_ERR_NOMEM;
    B->nb = nb;
    int rc = SVDSC_OK;
    int dev = 0, nsm = 0, occ = 0;
    if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        svdsc_batch_destroy(B);
        return SVDSC_ERR_CUDA;
    }
    if (cudaFuncSetAttribute(tune_spmv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(float) * kXCap)) != cudaSuccess ||
        cudaFuncSetAttribute(batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmBytes) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batched_kernel, kBT, kSmBytes) != cudaSuccess || occ < 1) {
        svdsc_batch_destroy(B);
        return SVDSC_ERR_CUDA;
    }
    B->A.resize(nb);
    B->AT.resize(nb);
    B->hm.resize(nb);
    int64_t mmax = 0, nmax = 0;
    int tmax = 0;
    for (int b = 0; b < nb && rc == SVDSC_OK; b++) {
        rc = csr_prepare(&As[b], true, false, &B->A[b], &B->AT[b], B->stream);
        BMat &M = B->hm[b];
        memset(&M, 0, sizeof(M));
        M.m = As[b].m; M.n = As[b].n; M.nnz = B->A[b].nnz;
        M.k = k[b];
        const int pb = p ? p[b] : -1;
        M.t = pb < 0 ? std::max(15, 3 * k[b]) : k[b] + pb;
        M.rp = B->A[b].row_ptr; M.col = B->A[b].col; M.val = B->A[b].val32;
        M.rpT = B->AT[b].row_ptr; M.colT = B->AT[b].col; M.valT = B->AT[b].val32;
        M.seed = (opt ? opt->seed : 0) + (uint64_t)b;
        M.gA = 8; M.gAT = 8; M.tc = 1;
        mmax = std::max(mmax, M.m);
        nmax = std::max(nmax, M.n);
        tmax = std::max(tmax, M.t);
    }
    if (rc) { svdsc_batch_destroy(B); return rc; }
    B->tstride = ((int64_t)(tmax + 1) * (tmax + 1) + 31) & ~int64_t(31);
    // Estimated work of one Lanczos pass: CGS2 ~ (m + n) t^2, products ~ nnz t.
    auto est_cost = [&](int b) {
        const BMat &M = B->hm[b];
        return (double)(M.m + M.n) * M.t * M.t + 4.0 * (double)M.nnz * M.t;
    };
    // The first solve's queue (later solves use measured cycles): largest
    // first by the pass cost times a prior on the number of passes.  Restart
    // counts are not known in advance, but they fall roughly as 1/k when p
    // grows with k (the 256-matrix batch: median 187 restarts at k ~ 5, 40 at
    // k ~ 20, 18 at k ~ 40), so a pass is weighted by 1 + 200 / k; on that
    // batch this brings the slowest matrix from queue position 46 to 24,
    // inside the first wave of clusters.
    auto est_total = [&](int b) { return est_cost(b) * (1.0 + 200.0 / (double)B->hm[b].k); };
    std::vector<int> &order = B->order;
    order.resize(nb);
    for (int b = 0; b < nb; b++) order[b] = b;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return est_total(x) > est_total(y); });
    B->reorder = Oopt == 0;
    double total = 0.0, worst = 0.0;
    for (int b = 0; b < nb; b++) { total += est_cost(b); worst = std::max(worst, est_cost(b)); }
    // Cluster size: the smallest power of two <= 8 for which the costliest
    // matrix on its cluster stays within its share of the batch's estimated
    // work.  (Two concurrent launches on one queue, 8-CTA clusters taking the
    // largest matrices and 2-CTA clusters the smallest, measured slower: the
    // matrix that dominates the batch is not among the largest by this
    // estimate, because its cost is its restart count, unknown in advance.)
    int C = Cfix;
    if (C == 0) {
        C = 1;
        while (C < 8 && worst * nsm > total * C) C *= 2;
    }
    const int cap = max_clusters(C);
    if (cap < 1) { svdsc_batch_destroy(B); return SVDSC_ERR_CUDA; }
    B->L.csize = C;
    B->L.nslots = std::min(nb, cap);
    // Lead launch: a few 8-CTA clusters that start before the main launch
    // and take the first queue positions, the costliest matrices (by the
    // previous solve's cycles once there is one), which scale almost linearly
    // from 4 to 8 CTAs and would otherwise be the batch's critical path on
    // the main launch's smaller clusters.  Automatic: one (1, 2, 3 and 4
    // measured within 3 % of each other on the 256-matrix batch, one best),
    // when the batch is longer than one wave of the main launch's clusters.
    // The main launch gives up the SMs the lead clusters hold.
    if (C < 8 && Aopt >= 0) {
        const int cap8 = max_clusters(8);
        int nlead = Aopt > 0 ? std::min(Aopt, cap8) : ((nb > cap && cap8 >= 2) ? 1 : 0);
        nlead = std::min(nlead, nb);
        const int displaced = (nlead * 8 + C - 1) / C;
        if (nlead > 0 && cap - displaced >= 1) {
            B->L.nslots = std::min(B->L.nslots, cap - displaced);
            B->LA.csize = 8;
            B->LA.nslots = nlead;
            rc = setup_launch(B, B->LA, mmax, nmax, tmax);
            if (rc) { svdsc_batch_destroy(B); return rc; }
        }
    }
    rc = setup_launch(B, B->L, mmax, nmax, tmax);
    if (rc) { svdsc_batch_destroy(B); return rc; }
    // Hand-off: once the queue is empty and enough clusters are idle, the
    // matrices still running stop at their next restart boundary and a
    // second launch of 8-CTA clusters finishes them.  Automatic: when the
    // first launch has more clusters than the second can hold, from the
    // moment no more are busy than the second launch has clusters.
    if (C < 8 && Hopt >= 0) {
        const int cap8 = max_clusters(8);
        int thr = 0;
        if (Hopt > 0) thr = Hopt;
        else if (cap8 >= 1 && B->L.nslots > cap8) thr = B->L.nslots - cap8;
        if (thr > 0 && cap8 >= 1) {
            B->handoff_idle = thr;
            B->L2.csize = 8;
            B->L2.nslots = std::max(1, std::min(cap8, B->L.nslots - std::min(thr, B->L.nslots - 1)));
            rc = setup_launch(B, B->L2, mmax, nmax, tmax, &B->L);
            if (rc) { svdsc_batch_destroy(B); return rc; }
        }
    }
    int64_t ntot = 0;
    for (int b = 0; b < nb; b++) ntot += B->hm[b].n;
    bool ok = cudaMalloc(&B->d_mats, sizeof(BMat) * nb) == cudaSuccess &&
              cudaMalloc(&B->d_order, sizeof(int) * nb) == cudaSuccess &&
              cudaMalloc(&B->d_stats, sizeof(BStat) * nb) == cudaSuccess &&
              cudaMalloc(&B->d_prm, sizeof(BParams)) == cudaSuccess &&
              cudaMalloc(&B->d_q, sizeof(BQueue)) == cudaSuccess &&
              cudaMallocHost(&B->h_mats, sizeof(BMat) * nb) == cudaSuccess &&
              cudaMallocHost(&B->h_prm, sizeof(BParams)) == cudaSuccess &&
              cudaMallocHost(&B->h_q0, sizeof(BQueue)) == cudaSuccess;
    if (ok) {
        memset(B->h_q0, 0, sizeof(BQueue));
        B->h_q0->next = B->LA.nslots;  // the lead clusters hold positions [0, nslots)
    }
    if (ok && B->handoff_idle > 0)
        ok = cudaMalloc(&B->d_ho, sizeof(int) * nb) == cudaSuccess &&
             cudaMalloc(&B->ckv_mem, sizeof(double) * ntot) == cudaSuccess &&
             cudaMalloc(&B->d_hand, sizeof(BHand) * nb) == cudaSuccess;
    if (!ok) { svdsc_batch_destroy(B); return SVDSC_ERR_NOMEM; }
    if (B->handoff_idle > 0) {
        int64_t off = 0;
        for (int b = 0; b < nb; b++) {
            B->hm[b].ckv = B->ckv_mem + off;
            B->hm[b].hand = B->d_hand + b;
            off += B->hm[b].n;
        }
    }
    cudaMemsetAsync(B->d_q, 0, sizeof(BQueue), B->stream);
    cudaMemcpyAsync(B->d_order, order.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, B->stream);
    // device output staging (used when outputs go to the host)
    size_t tot = 0;
    B->out_off.resize(nb);
    for (int b = 0; b < nb; b++) {
        B->out_off[b] = tot;
        tot += (size_t)B->hm[b].k * (B->hm[b].m + B->hm[b].n + 2);
    }
    if (cudaMalloc(&B->out_mem, sizeof(double) * std::max<size_t>(tot, 1)) != cudaSuccess) {
        svdsc_batch_destroy(B);
        return SVDSC_ERR_NOMEM;
    }
    // autotune (per shape class, cached process-wide)
    {
        double *ysc = nullptr, *wsc = nullptr;
        float *x32 = nullptr;
        const int64_t ldy = std::max(mmax, nmax) + 64;
        if (cudaMalloc(&ysc, sizeof(double) * ldy * nsm) != cudaSuccess ||
            cudaMalloc(&x32, sizeof(float) * ldy) != cudaSuccess ||
            cudaMalloc(&wsc, sizeof(double) * (size_t)mmax * (tmax / 2 + 1) + 64) != cudaSuccess) {
            cudaFree(ysc); cudaFree(x32); cudaFree(wsc);
            svdsc_batch_destroy(B);
            return SVDSC_ERR_NOMEM;
        }
        cudaMemsetAsync(x32, 0, sizeof(float) * ldy, B->stream);
        cudaMemsetAsync(wsc, 0, sizeof(double) * (size_t)mmax * (tmax / 2 + 1) + 64, B->stream);
        for (int b = 0; b < nb && rc == SVDSC_OK; b++) rc = tune_matrix(B, b, nsm, ysc, ldy, x32, wsc);
        cudaStreamSynchronize(B->stream);
        cudaFree(ysc); cudaFree(x32); cudaFree(wsc);
    }
    if (rc == SVDSC_OK && cudaStreamSynchronize(B->stream) != cudaSuccess) rc = SVDSC_ERR_CUDA;
    if (rc) { svdsc_batch_destroy(B); return rc; }
    *out = B;
    return SVDSC_OK;
}

static cudaError_t launch_batched(svdsc_batch *B, const BLaunch &L, int mode, cudaStream_t s, bool after_lead = false)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[2];
    // after the lead launch: start once every lead CTA runs (they signal it
    // at their start), not when the lead launch ends
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = L.csize;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(L.nslots * L.csize);
    cfg.blockDim = dim3(kBT);
    cfg.dynamicSmemBytes = kSmBytes;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = after_lead ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, batched_kernel, (const BMat *)B->d_mats, (const int *)B->d_order, B->nb,
                              B->d_q, B->d_ho, mode, B->d_stats, (const BSlot *)L.d_slots, L.d_T, B->tstride,
                              (const BParams *)B->d_prm);
}

int svdsc_batch_solve(svdsc_batch *B, double tol, int maxit, double *const *S, double *const *U,
                      double *const *V, double *const *res, int out_on_device, svdsc_info *infos)
{
    if (!B || !(tol > 0.0) || maxit < 1 || !S || !U || !V) return SVDSC_ERR_ARG;
    const int nb = B->nb;
    for (int b = 0; b < nb; b++) {
        BMat &M = B->hm[b];
        if (!S[b] || !U[b] || !V[b]) return SVDSC_ERR_ARG;
        if (out_on_device) {
            M.S = S[b]; M.U = U[b]; M.V = V[b];
            M.res = res && res[b] ? res[b] : B->out_mem + B->out_off[b] + (size_t)M.k * (M.m + M.n + 1);
        } else {
            double *o = B->out_mem + B->out_off[b];
            M.U = o; M.V = o + (size_t)M.k * M.m; M.S = M.V + (size_t)M.k * M.n; M.res = M.S + M.k;
        }
    }
    memcpy(B->h_mats, B->hm.data(), sizeof(BMat) * nb);
    B->h_prm->tol = tol;
    B->h_prm->maxit = maxit;
    B->h_prm->handoff_idle = B->handoff_idle;
    if (!B->exec) {  // capture upload + reset + the persistent launch(es) once; replay afterwards
        if (cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SVDSC_ERR_CUDA;
        cudaMemcpyAsync(B->d_mats, B->h_mats, sizeof(BMat) * nb, cudaMemcpyHostToDevice, B->stream);
        cudaMemcpyAsync(B->d_prm, B->h_prm, sizeof(BParams), cudaMemcpyHostToDevice, B->stream);
        cudaMemcpyAsync(B->d_q, B->h_q0, sizeof(BQueue), cudaMemcpyHostToDevice, B->stream);
        cudaMemsetAsync(B->d_stats, 0, sizeof(BStat) * nb, B->stream);
        cudaError_t e = cudaSuccess;
        if (B->LA.nslots > 0) e = launch_batched(B, B->LA, 2, B->stream);
        if (e == cudaSuccess) e = launch_batched(B, B->L, 0, B->stream, B->LA.nslots > 0);
        if (e == cudaSuccess && B->handoff_idle > 0) e = launch_batched(B, B->L2, 1, B->stream);
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(B->stream, &g);
        if (e != cudaSuccess || ec != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return SVDSC_ERR_CUDA;
        }
        B->graph = g;
        if (cudaGraphInstantiate(&B->exec, B->graph, 0) != cudaSuccess) return SVDSC_ERR_CUDA;
    }
    if (cudaGraphLaunch(B->exec, B->stream) != cudaSuccess) return SVDSC_ERR_CUDA;
    std::vector<BStat> st(nb);
    if (cudaMemcpyAsync(st.data(), B->d_stats, sizeof(BStat) * nb, cudaMemcpyDeviceToHost, B->stream) != cudaSuccess)
        return SVDSC_ERR_CUDA;
    if (!out_on_device) {
        for (int b = 0; b < nb; b++) {
            const BMat &M = B->hm[b];
            cudaMemcpyAsync(U[b], M.U, sizeof(double) * M.m * M.k, cudaMemcpyDeviceToHost, B->stream);
            cudaMemcpyAsync(V[b], M.V, sizeof(double) * M.n * M.k, cudaMemcpyDeviceToHost, B->stream);
            cudaMemcpyAsync(S[b], M.S, sizeof(double) * M.k, cudaMemcpyDeviceToHost, B->stream);
            if (res && res[b]) cudaMemcpyAsync(res[b], M.res, sizeof(double) * M.k, cudaMemcpyDeviceToHost, B->stream);
        }
    }
    if (cudaStreamSynchronize(B->stream) != cudaSuccess) return SVDSC_ERR_CUDA;
    int worst = SVDSC_OK;
    for (int b = 0; b < nb; b++) {
        if (infos) {
            svdsc_info &I = infos[b];
            memset(&I, 0, sizeof(I));
            I.converged = st[b].converged; I.nconv = st[b].nconv; I.restarts = st[b].restarts;
            I.breakdowns = st[b].breakdowns; I.n_matvec = st[b].n_matvec; I.n_steps = st[b].n_steps;
            I.anorm_est = st[b].anorm; I.beta_t = st[b].beta_t; I.t = B->hm[b].t;
            I.reserved = st[b].err;
        }
        if (st[b].err) worst = st[b].err;
        else if (!st[b].converged && worst == SVDSC_OK) worst = SVDSC_NOT_CONVERGED;
    }
    if (B->reorder) {
        // The next solve of this batch takes the matrices in the order of the
        // SM cycles they took in this one (cycles times the CTAs of the
        // cluster, so that a matrix that ran on a larger cluster is not
        // ranked cheaper for it; largest first, ties by index): a matrix's
        // cost is mostly its restart count, which no estimate made before the
        // first solve predicts, so the costliest start first.
        std::vector<int> &order = B->order;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            return st[x].work != st[y].work ? st[x].work > st[y].work : x < y;
        });
        if (cudaMemcpyAsync(B->d_order, order.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, B->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(B->stream) != cudaSuccess)
            return SVDSC_ERR_CUDA;
    }
    return worst;
}

int svdsc_solve_batched(int nb, const svdsc_matrix *As, const int *k, const int *p, double tol, int maxit,
                        double *const *S, double *const *U, double *const *V, double *const *res,
                        int out_on_device, const svdsc_options *opt, svdsc_info *infos)
{
    svdsc_batch *B = nullptr;
    int rc = svdsc_batch_create(&B, nb, As, k, p, opt, nullptr);
    if (rc) return rc;
    rc = svdsc_batch_solve(B, tol, maxit, S, U, V, res, out_on_device, infos);
    svdsc_batch_destroy(B);
    return rc;
}

int svdsc_batch_tuning(const svdsc_batch *B, int b, int *lanes_A, int *lanes_AT, int *gemv_cols, double *tune_ms)
{
    if (!B || b < 0 || b >= B->nb) return SVDSC_ERR_ARG;
    if (lanes_A) *lanes_A = B->hm[b].gA;
    if (lanes_AT) *lanes_AT = B->hm[b].gAT;
    if (gemv_cols) *gemv_cols = B->hm[b].tc;
    if (tune_ms) *tune_ms = B->tune_ms;
    return SVDSC_OK;
}

int svdsc_batch_profile(const svdsc_batch *B, int64_t *cycles_total, int64_t *cycles_svd, int64_t *cycles_lbp,
                        int32_t *cluster)
{
    if (!B) return SVDSC_ERR_ARG;
    std::vector<BStat> st(B->nb);
    if (cudaMemcpy(st.data(), B->d_stats, sizeof(BStat) * B->nb, cudaMemcpyDeviceToHost) != cudaSuccess)
        return SVDSC_ERR_CUDA;
    for (int b = 0; b < B->nb; b++) {
        if (cycles_total) cycles_total[b] = st[b].cycles_total;
        if (cycles_svd) cycles_svd[b] = st[b].cycles_svd;
        if (cycles_lbp) cycles_lbp[b] = st[b].cycles_lbp;
        if (cluster) cluster[b] = st[b].cluster;
    }
    return SVDSC_OK;
}

int svdsc_batch_phase_cycles(const svdsc_batch *B, int64_t *cycles)
{
    if (!B || !cycles) return SVDSC_ERR_ARG;
    std::vector<BStat> st(B->nb);
    if (cudaMemcpy(st.data(), B->d_stats, sizeof(BStat) * B->nb, cudaMemcpyDeviceToHost) != cudaSuccess)
        return SVDSC_ERR_CUDA;
    for (int b = 0; b < B->nb; b++)
        for (int q = 0; q < 5; q++) cycles[(int64_t)b * 5 + q] = st[b].cycles_phase[q];
    return SVDSC_OK;
}

int svdsc_batch_layout(const svdsc_batch *B, int *cluster_size, int *clusters)
{
    if (!B) return SVDSC_ERR_ARG;
    if (cluster_size) *cluster_size = B->L.csize;
    if (clusters) *clusters = B->L.nslots;
    return SVDSC_OK;
}

int svdsc_batch_lead(const svdsc_batch *B, int *cluster_size, int *clusters)
{
    if (!B) return SVDSC_ERR_ARG;
    if (cluster_size) *cluster_size = B->LA.csize;
    if (clusters) *clusters = B->LA.nslots;
    return SVDSC_OK;
}

int svdsc_batch_handoff(const svdsc_batch *B, int *idle_threshold, int *cluster_size, int *clusters,
                        int *handed_off)
{
    if (!B) return SVDSC_ERR_ARG;
    if (idle_threshold) *idle_threshold = B->handoff_idle;
    if (cluster_size) *cluster_size = B->L2.csize;
    if (clusters) *clusters = B->L2.nslots;
    if (handed_off) {
        BQueue q = {};
        if (cudaMemcpy(&q, B->d_q, sizeof(BQueue), cudaMemcpyDeviceToHost) != cudaSuccess) return SVDSC_ERR_CUDA;
        *handed_off = q.ho_count;
    }
    return SVDSC_OK;
}

}  // extern "C"
