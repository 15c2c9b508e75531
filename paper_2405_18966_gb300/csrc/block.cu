// Block form of the method: block Lanczos bidiagonalization (Golub, Luk &
// Overton 1981) with the full re-orthogonalization of Sec. 2.1 and the
// augmented restart of Eq. (5)-(7) / Alg. 2 carried over from single vectors
// to blocks of b columns (b = 2, 4, 8 or 16).
//
// Per block of b Lanczos vectors (one side):
//   spmm:        Y = A X - Z C   (X: the previous block of the other side, kept
//                row-major so that each nonzero gathers b contiguous values;
//                Z C: the previous block of this side times a b x b block of T)
//   CGS2:        two passes of H = W^T Y (per-chunk partials, ordered reduce)
//                and Y -= W H against the earlier blocks W (coefficients
//                discarded); in the mixed form the first pass runs on the FP32
//                shadow of W with FP32 products; the second pass is FP64
//   CholQR2:     G = Y^T Y = R1^T R1, Y <- Y R1^-1, again (R2), R = R2 R1; a
//                numerically rank-deficient or ill-conditioned block (a
//                diagonal entry of R1 below 1e-13 times the largest norm seen,
//                or below 1e-6 times the block's largest) is flagged, and the
//                host redoes that block's QR column by column (each column
//                projected twice against the earlier columns, a broken-down
//                column replaced by a random vector), as the oracle does
//   T entries:   R -> T(c:c+b, c:c+b) for a U block, R^T -> T(c-b:c, c:c+b)
//                for a V block; the block is then copied row-major (and to the
//                FP32 shadow) for the next product.
// The projected matrix T is upper triangular with bandwidth b; its SVD is the
// same device Jacobi as the single-vector form; the residual of Eq. (4)
// becomes ||F^T Uh(t-b:t, j)|| with F = T(t-b:t, t:t+b), and the restart keeps
// the k Ritz vectors plus the residual block with rho = Uh(t-b:t, 0:k)^T F.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cstdint>
#include <cstring>
#include <vector>
#include "context.cuh"

namespace svdsc {

constexpr int kBlkThreads = 512;  // threads per CTA of the block kernels

// rows per chunk of the block kernels: the FP64 chunk of Y staged in shared
// memory is at most 64 KB
__host__ __device__ constexpr int blk_rows(int B) { return B <= 8 ? 1024 : 512; }

struct BlockWork {
    int b = 0;
    int64_t cap_m = 0, cap_n = 0;
    int tcap = 0;
    double *Xu = nullptr, *Xv = nullptr;      // row-major copies of the newest U / V block
    float *Xu32 = nullptr, *Xv32 = nullptr;   // FP32 copies (mixed form)
    double *P = nullptr;                      // GEMM-T / Gram partial sums
    double *H = nullptr;                      // projection coefficients (tcap x b, row-major)
    double *G = nullptr;                      // Gram matrix (b x b)
    double *R1 = nullptr, *Rinv = nullptr, *R2 = nullptr, *Rcc = nullptr;  // b x b each
    double *rho = nullptr;                    // restart coefficients (k x b, row-major)
    int *flag = nullptr;                      // repair: column broke down
    size_t P_doubles = 0;
    std::vector<std::pair<int64_t, int64_t>> counts;  // (products, vectors) after each recorded block
};

__device__ __forceinline__ bool blk_poisoned(const int *poison)
{
    return poison && *(volatile const int *)poison;
}

// ------------------------------------------------------------------- SpMM

// B accumulators of one row over the nonzeros handled by this lane.
template <int B, typename VT, typename XT, typename AT>
__device__ __forceinline__ void spmm_lane(const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                          const VT *__restrict__ val, const XT *__restrict__ X, int64_t r,
                                          int lg, int G, AT (&acc)[B])
{
    const int64_t e0 = row_ptr[r], e1 = row_ptr[r + 1];
    for (int64_t e = e0 + lg; e < e1; e += G) {
        const AT v = AT(__ldcs(val + e));
        const XT *x = X + (int64_t)__ldcs(col + e) * B;
#pragma unroll
        for (int l = 0; l < B; l++) acc[l] += v * AT(__ldg(x + l));
    }
}

// y(r, l) = acc(l) - sum_i Z(r, i) C(i, l); C(i, l) = Cb[i + l ldc] (or
// Cb[l + i ldc] when ctrans), written to column l of Y (leading dimension ldy).
template <int B, typename AT>
__device__ __forceinline__ void spmm_store(int64_t r, const AT (&acc)[B], const double *__restrict__ Z,
                                           int64_t ldz, const double *__restrict__ Cb, int64_t ldc, int ctrans,
                                           double *__restrict__ Y, int64_t ldy)
{
    double z[B];
    if (Z) {
#pragma unroll
        for (int i = 0; i < B; i++) z[i] = Z[r + (int64_t)i * ldz];
    }
#pragma unroll
    for (int l = 0; l < B; l++) {
        double y = double(acc[l]);
        if (Z) {
#pragma unroll
            for (int i = 0; i < B; i++) {
                const double cf = ctrans ? Cb[l + (int64_t)i * ldc] : Cb[i + (int64_t)l * ldc];
                y -= z[i] * cf;
            }
        }
        Y[r + (int64_t)l * ldy] = y;
    }
}

template <int B, typename VT, typename XT, typename AT>
__global__ void __launch_bounds__(kSpmvThreads)
spmm_kernel(const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col, const VT *__restrict__ val,
            const XT *__restrict__ X, const int32_t *__restrict__ perm, const __grid_constant__ Bins bins,
            int64_t sell_rows, int64_t sell_blocks, const int32_t *__restrict__ sell_perm,
            const int64_t *__restrict__ sell_off, const int32_t *__restrict__ sell_col,
            const VT *__restrict__ sell_val, const double *__restrict__ Z, int64_t ldz,
            const double *__restrict__ Cb, int64_t ldc, int ctrans, double *__restrict__ Y, int64_t ldy,
            const int *poison)
{
    if (blk_poisoned(poison)) return;
    AT acc[B];
#pragma unroll
    for (int l = 0; l < B; l++) acc[l] = AT(0);
    if ((int64_t)blockIdx.x < sell_blocks) {
        // SELL-32 rows: one thread per row, coalesced (column, value) streams
        const int64_t i = (int64_t)blockIdx.x * kSpmvThreads + threadIdx.x;
        if (i >= sell_rows) return;
        const int64_t sl = i >> 5;
        const int lane = (int)(i & 31);
        const int64_t off = sell_off[sl];
        const int w = (int)((sell_off[sl + 1] - off) >> 5);
        const int32_t *cp = sell_col + off + lane;
        const VT *vp = sell_val + off + lane;
        for (int j = 0; j < w; j++) {
            const AT v = AT(__ldcs(vp + 32 * j));
            const XT *x = X + (int64_t)__ldcs(cp + 32 * j) * B;
#pragma unroll
            for (int l = 0; l < B; l++) acc[l] += v * AT(__ldg(x + l));
        }
        spmm_store<B, AT>(sell_perm[i], acc, Z, ldz, Cb, ldc, ctrans, Y, ldy);
        return;
    }
    const int64_t bidx = blockIdx.x - sell_blocks;
    int bin = 0;
#pragma unroll
    for (int i = 1; i < kNumBins; i++)
        if (bidx >= bins.block_start[i]) bin = i;
    const int64_t lb = bidx - bins.block_start[bin];
    const int64_t rb = bins.row_start[bin], re = bins.row_start[bin + 1];
    if (bin < kNumBins - 1) {
        const int G = bin <= 3 ? 1 : 1 << (bin - 3);
        const int grp = threadIdx.x / G, lg = threadIdx.x % G;
        const int64_t idx = rb + lb * (kSpmvThreads / G) + grp;
        if (idx >= re) return;  // whole lane groups leave together
        const int64_t r = perm[idx];
        spmm_lane<B, VT, XT, AT>(row_ptr, col, val, X, r, lg, G, acc);
        const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
        for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
            for (int l = 0; l < B; l++) acc[l] += __shfl_xor_sync(gmask, acc[l], o);
        if (lg == 0) spmm_store<B, AT>(r, acc, Z, ldz, Cb, ldc, ctrans, Y, ldy);
        return;
    }
    // a whole CTA per (very long) row
    const int64_t r = perm[rb + lb];
    spmm_lane<B, VT, XT, AT>(row_ptr, col, val, X, r, threadIdx.x, kSpmvThreads, acc);
    __shared__ AT red[kSpmvThreads / 32][B];
#pragma unroll
    for (int l = 0; l < B; l++) {
        AT s = acc[l];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][l] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int l = 0; l < B; l++) {
            AT t = AT(0);
            for (int w = 0; w < kSpmvThreads / 32; w++) t += red[w][l];
            acc[l] = t;
        }
        spmm_store<B, AT>(r, acc, Z, ldz, Cb, ldc, ctrans, Y, ldy);
    }
}

template <int B>
static cudaError_t launch_spmm(const DevCSR &A, bool f32, const void *X, const double *Z, int64_t ldz,
                               const double *Cb, int64_t ldc, int ctrans, double *Y, int64_t ldy,
                               const int *poison, cudaStream_t s)
{
    const int64_t sb = (A.sell_rows + kSpmvThreads - 1) / kSpmvThreads;
    const int64_t nblk = sb + A.bins.block_start[kNumBins];
    if (nblk == 0) return cudaSuccess;
    if (f32)
        spmm_kernel<B, float, float, float><<<(unsigned)nblk, kSpmvThreads, 0, s>>>(
            A.row_ptr, A.col, A.val32, (const float *)X, A.perm, A.bins, A.sell_rows, sb, A.sell_perm, A.sell_off,
            A.sell_col, A.sell_val32, Z, ldz, Cb, ldc, ctrans, Y, ldy, poison);
    else
        spmm_kernel<B, double, double, double><<<(unsigned)nblk, kSpmvThreads, 0, s>>>(
            A.row_ptr, A.col, A.val, (const double *)X, A.perm, A.bins, A.sell_rows, sb, A.sell_perm, A.sell_off,
            A.sell_col, A.sell_val, Z, ldz, Cb, ldc, ctrans, Y, ldy, poison);
    return cudaGetLastError();
}

// --------------------------------------------------------- block GEMM-T

// P[(c B + l) nbk + chunk] = sum over the chunk's rows of W(r, c) Y(r, l).
// The chunk of Y (rows x B) is staged in shared memory (as AT: the FP32 pass
// converts it once); each warp takes CW columns of W at a time, each lane
// keeps CW x B accumulators over its rows, then the warp adds them up.
template <int B, int CW, typename WT>
__global__ void __launch_bounds__(kBlkThreads)
bgemm_t_kernel(const WT *__restrict__ W, int64_t ldw, int ncols, const double *__restrict__ Y, int64_t ldy,
               int64_t len, int nbk, double *__restrict__ P, const int *poison)
{
    if (blk_poisoned(poison)) return;
    using AT = WT;
    constexpr int RB = blk_rows(B);
    extern __shared__ __align__(16) unsigned char blk_smem[];
    AT *ys = (AT *)blk_smem;  // [row][B]
    const int64_t r0 = (int64_t)blockIdx.x * RB;
    const int rows = (int)min((int64_t)RB, len - r0);
    for (int i = threadIdx.x; i < rows * B; i += kBlkThreads) {
        const int j = i % rows, l = i / rows;  // coalesced over rows of column l
        ys[j * B + l] = (AT)Y[r0 + j + (int64_t)l * ldy];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ngroups = (ncols + CW - 1) / CW;
    for (int g = warp; g < ngroups; g += kBlkThreads / 32) {
        const int c0 = g * CW;
        AT acc[CW][B];
#pragma unroll
        for (int q = 0; q < CW; q++)
#pragma unroll
            for (int l = 0; l < B; l++) acc[q][l] = AT(0);
        const WT *wc[CW];
#pragma unroll
        for (int q = 0; q < CW; q++) wc[q] = W + (int64_t)min(c0 + q, ncols - 1) * ldw + r0;
        for (int j = lane; j < rows; j += 32) {
            AT w[CW];
#pragma unroll
            for (int q = 0; q < CW; q++) w[q] = __ldcs(wc[q] + j);
            const AT *yr = ys + j * B;
#pragma unroll
            for (int l = 0; l < B; l++) {
                const AT y = yr[l];
#pragma unroll
                for (int q = 0; q < CW; q++) acc[q][l] = fma(w[q], y, acc[q][l]);
            }
        }
#pragma unroll
        for (int q = 0; q < CW; q++)
#pragma unroll
            for (int l = 0; l < B; l++) {
                double sum = (double)acc[q][l];
                for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
                if (lane == 0 && c0 + q < ncols) P[((int64_t)(c0 + q) * B + l) * nbk + blockIdx.x] = sum;
            }
    }
}

// --------------------------------------------------------- block GEMM-N

// Y(r, l) -= sum_c W(r, c) H(c, l) (H row-major ncols x B, in shared memory).
template <int B, typename WT>
__global__ void __launch_bounds__(kBlkThreads)
bgemm_n_kernel(const WT *__restrict__ W, int64_t ldw, int ncols, const double *__restrict__ H,
               double *__restrict__ Y, int64_t ldy, int64_t len, const int *poison)
{
    if (blk_poisoned(poison)) return;
    constexpr int RB = blk_rows(B);
    extern __shared__ __align__(16) unsigned char blk_smem[];
    WT *hs = (WT *)blk_smem;  // ncols x B
    for (int i = threadIdx.x; i < ncols * B; i += kBlkThreads) hs[i] = (WT)H[i];
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * RB;
    const int rows = (int)min((int64_t)RB, len - r0);
    for (int j = threadIdx.x; j < rows; j += kBlkThreads) {
        const int64_t r = r0 + j;
        WT acc[B];
#pragma unroll
        for (int l = 0; l < B; l++) acc[l] = WT(0);
        for (int c = 0; c < ncols; c++) {
            const WT w = __ldcs(W + r + (int64_t)c * ldw);
            const WT *hc = hs + c * B;
#pragma unroll
            for (int l = 0; l < B; l++) acc[l] = fma(w, hc[l], acc[l]);
        }
#pragma unroll
        for (int l = 0; l < B; l++) Y[r + (int64_t)l * ldy] -= (double)acc[l];
    }
}

// Gram partial sums of the block Y: Pg[(l B + l') nbk + chunk] = sum over the
// chunk's rows of Y(r, l) Y(r, l').  The chunk is staged in shared memory; each
// thread takes one pair (l <= l') and every ng-th row, and the row groups are
// added in a fixed order.
template <int B>
__global__ void __launch_bounds__(kBlkThreads)
bgram_kernel(const double *__restrict__ Y, int64_t ldy, int64_t len, int nbk, double *__restrict__ Pg,
             const int *poison)
{
    if (blk_poisoned(poison)) return;
    constexpr int RB = blk_rows(B);
    constexpr int NP = B * (B + 1) / 2;
    constexpr int NG = kBlkThreads / NP;
    extern __shared__ __align__(16) unsigned char blk_smem[];
    double *ys = (double *)blk_smem;  // [row][B]
    __shared__ double part[NG * NP];
    const int64_t r0 = (int64_t)blockIdx.x * RB;
    const int rows = (int)min((int64_t)RB, len - r0);
    for (int i = threadIdx.x; i < rows * B; i += kBlkThreads) {
        const int j = i % rows, l = i / rows;
        ys[j * B + l] = Y[r0 + j + (int64_t)l * ldy];
    }
    __syncthreads();
    const int q = threadIdx.x % NP, g = threadIdx.x / NP;
    int l = 0, l2 = q;  // pair q -> (l, l2), l <= l2, in row order of the upper triangle
    while (l2 >= B - l) { l2 -= B - l; l++; }
    l2 += l;
    if (g < NG) {
        double a = 0.0;
        for (int j = g; j < rows; j += NG) a = fma(ys[j * B + l], ys[j * B + l2], a);
        part[g * NP + q] = a;
    }
    __syncthreads();
    if (threadIdx.x < NP) {
        double t = 0.0;
        for (int gg = 0; gg < NG; gg++) t += part[gg * NP + q];
        Pg[((int64_t)l * B + l2) * nbk + blockIdx.x] = t;
        Pg[((int64_t)l2 * B + l) * nbk + blockIdx.x] = t;
    }
}

// ------------------------------------------------------- CholQR steps

// One thread: G = R^T R (upper R, Cholesky), Rinv = R^-1.  stage 1 (first
// pass): the checks of the block (breakdown, conditioning) poison the
// segment on failure, recording `step`; stage 2: R2 must be close to the
// identity; the total R = R2 R1 goes to T (transposed for a V block: T gets
// R^T at T(tr, tc)), the running ||A|| estimate to the status block.
__global__ void bchol_kernel(int B, const double *__restrict__ Gm, double *__restrict__ Rout,
                             double *__restrict__ Rinv, const double *__restrict__ R1, int stage, double *T,
                             int64_t ldt, int trans, DevStatus *st, int parity, int step)
{
    if (*(volatile int *)&st->poison) return;
    if (threadIdx.x != 0) return;
    double R[16 * 16], Ri[16 * 16];
    for (int i = 0; i < B * B; i++) { R[i] = 0.0; Ri[i] = 0.0; }
    bool bad = false;
    for (int j = 0; j < B && !bad; j++) {
        double d = Gm[j * B + j];
        for (int i = 0; i < j; i++) d -= R[i + j * B] * R[i + j * B];
        if (!(d > 0.0) || !isfinite(d)) { bad = true; break; }
        const double rjj = sqrt(d);
        R[j + j * B] = rjj;
        for (int l = j + 1; l < B; l++) {
            double s = Gm[j * B + l];
            for (int i = 0; i < j; i++) s -= R[i + j * B] * R[i + l * B];
            R[j + l * B] = s / rjj;
        }
    }
    const double anorm = st->anorm[parity];
    double amax = anorm, dmax = 0.0, dmin = DBL_MAX;
    if (!bad) {
        for (int j = 0; j < B; j++) {
            dmax = fmax(dmax, R[j + j * B]);
            dmin = fmin(dmin, R[j + j * B]);
        }
        if (stage == 1) {
            // the oracle's column-by-column breakdown test, in column order
            double an = anorm;
            for (int j = 0; j < B && !bad; j++) {
                if (!(R[j + j * B] > 1e-13 * an)) bad = true;
                an = fmax(an, R[j + j * B]);
            }
            if (dmin < 1e-6 * dmax) bad = true;  // ill-conditioned: the column-by-column path instead
        } else if (dmin < 0.5 || dmax > 2.0) {
            bad = true;
        }
    }
    if (bad) {
        atomicMin(&st->bd_step, step);
        st->poison = 1;
        st->anorm[parity ^ 1] = anorm;
        if (stage == 1)  // the repair composes with R1 = I
            for (int i = 0; i < B * B; i++) Rout[i] = (i % (B + 1) == 0) ? 1.0 : 0.0;
        return;
    }
    // Rinv: upper triangular inverse, column by column
    for (int l = 0; l < B; l++) {
        Ri[l + l * B] = 1.0 / R[l + l * B];
        for (int i = l - 1; i >= 0; i--) {
            double s = 0.0;
            for (int q = i + 1; q <= l; q++) s += R[i + q * B] * Ri[q + l * B];
            Ri[i + l * B] = -s / R[i + i * B];
        }
    }
    for (int i = 0; i < B * B; i++) Rinv[i] = Ri[i];
    if (stage == 1) {
        for (int i = 0; i < B * B; i++) Rout[i] = R[i];
        st->anorm[parity ^ 1] = anorm;
        return;
    }
    // R = R2 R1 (both upper triangular) into T
    for (int l = 0; l < B; l++)
        for (int i = 0; i < B; i++) {
            double s = 0.0;
            for (int q = i; q <= l; q++) s += R[i + q * B] * R1[q + l * B];
            if (i <= l) amax = fmax(amax, i == l ? s : 0.0);
            const double v = i <= l ? s : 0.0;
            if (trans) T[l + (int64_t)i * ldt] = v;
            else T[i + (int64_t)l * ldt] = v;
        }
    st->anorm[parity ^ 1] = amax;
}

// Y(r, :) <- Y(r, :) Rinv; on the final pass also the FP32 shadow and the
// row-major copies for the next product.
template <int B>
__global__ void __launch_bounds__(kBlkThreads, 1)
btrsm_kernel(double *__restrict__ Y, int64_t ldy, int64_t len, const double *__restrict__ Rinv,
             float *__restrict__ Y32, double *__restrict__ X, float *__restrict__ X32, const int *poison)
{
    if (blk_poisoned(poison)) return;
    constexpr int RB = blk_rows(B);
    __shared__ double ri[B * B];
    for (int i = threadIdx.x; i < B * B; i += kBlkThreads) ri[i] = Rinv[i];
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * RB;
    const int rows = (int)min((int64_t)RB, len - r0);
    for (int j = threadIdx.x; j < rows; j += kBlkThreads) {
        const int64_t r = r0 + j;
        double y[B];
#pragma unroll
        for (int l = 0; l < B; l++) y[l] = Y[r + (int64_t)l * ldy];
        double o[B];
#pragma unroll
        for (int l = 0; l < B; l++) o[l] = 0.0;
#pragma unroll
        for (int i = 0; i < B; i++) {
#pragma unroll
            for (int l = i; l < B; l++) o[l] = fma(y[i], ri[i + l * B], o[l]);
        }
#pragma unroll
        for (int l = 0; l < B; l++) y[l] = o[l];
#pragma unroll
        for (int l = 0; l < B; l++) Y[r + (int64_t)l * ldy] = y[l];
        if (Y32) {
#pragma unroll
            for (int l = 0; l < B; l++) Y32[r + (int64_t)l * ldy] = (float)y[l];
        }
        if (X) {
#pragma unroll
            for (int l = 0; l < B; l++) X[r * B + l] = y[l];
        }
        if (X32) {
#pragma unroll
            for (int l = 0; l < B; l++) X32[r * B + l] = (float)y[l];
        }
    }
}

// Row-major (and FP32) copies of a block that is already in the basis.
template <int B>
__global__ void bcopy_rows_kernel(const double *__restrict__ Y, int64_t ldy, int64_t len, double *__restrict__ X,
                                  float *__restrict__ X32, float *__restrict__ Y32)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len * B;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / B;
        const int l = (int)(i % B);
        const double v = Y[r + (int64_t)l * ldy];
        if (X) X[i] = v;
        if (X32) X32[i] = (float)v;
        if (Y32) Y32[r + (int64_t)l * ldy] = (float)v;
    }
}

// ------------------------------------------------ residual test, restart

// Block Eq. (4): res_j = ||F^T Uh(t-b:t, j)|| / max(sigma_j, eps sigma_1) with
// F = T(t-b:t, t:t+b); rho(j, l) = sum_i Uh(t-b+i, j) F(i, l) (row-major k x b).
__global__ void bresidual_kernel(int t, int k, int B, double tol, const double *__restrict__ T, int64_t ldt,
                                 const double *__restrict__ Sh, const double *__restrict__ Uh,
                                 double *__restrict__ res, double *__restrict__ rho, DevStatus *st, int parity)
{
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const double s0 = Sh[0];
    int local = 0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        double r2 = 0.0;
        for (int l = 0; l < B; l++) {
            double s = 0.0;
            for (int i = 0; i < B; i++) s += T[(t - B + i) + (int64_t)(t + l) * ldt] * Uh[(t - B + i) + (int64_t)j * t];
            rho[j * B + l] = s;
            r2 += s * s;
        }
        const double den = Sh[j] > DBL_EPSILON * s0 ? Sh[j] : DBL_EPSILON * s0;
        const double r = den > 0.0 ? sqrt(r2) / den : 0.0;
        res[j] = r;
        local += (r < tol);
    }
    atomicAdd(&cnt, local);
    __syncthreads();
    if (threadIdx.x == 0) {
        double f = 0.0;
        for (int l = 0; l < B; l++)
            for (int i = 0; i < B; i++) {
                const double x = T[(t - B + i) + (int64_t)(t + l) * ldt];
                f += x * x;
            }
        st->nconv = cnt;
        st->converged = (cnt == k);
        st->beta_t = sqrt(f);
        if (s0 > st->anorm[parity]) st->anorm[parity] = s0;
    }
}

// T <- 0; T(j, j) = sigma_j; T(j, k + l) = rho(j, l)  (j < k, l < b)
__global__ void brestart_T_kernel(int ldt, int k, int B, double *__restrict__ T, const double *__restrict__ Sh,
                                  const double *__restrict__ rho)
{
    const int64_t tot = (int64_t)ldt * ldt;
    for (int64_t i = threadIdx.x; i < tot; i += blockDim.x) T[i] = 0.0;
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        T[j + (int64_t)j * ldt] = Sh[j];
        for (int l = 0; l < B; l++) T[j + (int64_t)(k + l) * ldt] = rho[j * B + l];
    }
}

// Repair path helpers: Rcc(0:l, l) += h(c0 .. c0+l) (the in-block coefficients
// of one CGS pass); the column's norm decides between scaling and a random
// replacement (flag).
__global__ void brepair_accum_kernel(const double *__restrict__ h, int c0, int l, int B, double *__restrict__ Rcc)
{
    for (int i = threadIdx.x; i < l; i += blockDim.x) Rcc[i + l * B] += h[c0 + i];
}

__global__ void brepair_norm_kernel(double *__restrict__ w, int64_t len, const double *__restrict__ nrm_in,
                                    int l, int B, double *__restrict__ Rcc, DevStatus *st, int parity,
                                    int *flag, int mode)
{
    // mode 0: a Lanczos column (breakdown test against the ||A|| estimate);
    // mode 1: a random replacement (needs norm > 1e-8).  *nrm_in = ||w||.
    const double nrm = *nrm_in;
    const double anorm = st->anorm[parity];
    const bool ok = mode == 0 ? (nrm > 1e-13 * anorm && isfinite(nrm)) : (nrm > 1e-8 && isfinite(nrm));
    if (!ok) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            *flag = 1;
            if (mode == 0) Rcc[l + l * B] = 0.0;
        }
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *flag = 0;
        if (mode == 0) {
            Rcc[l + l * B] = nrm;
            if (nrm > anorm) st->anorm[parity] = nrm;
        }
    }
    const double inv = 1.0 / nrm;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        w[i] *= inv;
}

// T block = Rcc R1 (both upper triangular; transposed into T for a V block)
__global__ void brepair_T_kernel(int B, const double *__restrict__ Rcc, const double *__restrict__ R1, double *T,
                                 int64_t ldt, int trans)
{
    if (threadIdx.x != 0) return;
    for (int l = 0; l < B; l++)
        for (int i = 0; i < B; i++) {
            double s = 0.0;
            for (int q = i; q <= l; q++) s += Rcc[i + q * B] * R1[q + l * B];
            const double v = i <= l ? s : 0.0;
            if (trans) T[l + (int64_t)i * ldt] = v;
            else T[i + (int64_t)l * ldt] = v;
        }
}

}  // namespace svdsc

// ============================================================ host driver

namespace {

struct BlockSide {
    double *W;      // basis (column-major)
    float *W32;     // FP32 shadow or null
    int64_t ld, len;
    double *X;      // row-major copy of the newest block
    float *X32;
    const Chunk *ch;
};

int nbk_of(int64_t len, int B) { return (int)((len + blk_rows(B) - 1) / blk_rows(B)); }

BlockSide side_of(svdsc_ctx *c, int side)
{
    BlockWork *w = c->bw;
    if (side == 0) return {c->U, c->U32, c->ldu, c->m, w->Xu, w->Xu32, &c->cm};
    return {c->V, c->V32, c->ldv, c->n, w->Xv, w->Xv32, &c->cn};
}

#define BCU(x)                                          \
    do {                                                \
        cudaError_t e_ = (x);                           \
        if (e_ != cudaSuccess) return SVDSC_ERR_CUDA;   \
    } while (0)

template <int B>
int spmm(svdsc_ctx *c, int trans, const void *X, const double *Z, int64_t ldz, const double *Cb, int ctrans,
         double *Y, int64_t ldy)
{
    const DevCSR &M = trans ? c->AT : c->A;
    const bool f32 = c->precision == SVDSC_MIXED;
    const int e0 = ph_begin(c);
    cudaError_t e = launch_spmm<B>(M, f32, X, Z, ldz, Cb, c->t_ld, ctrans, Y, ldy, poison_ptr(c), c->stream);
    const double bytes = (f32 ? 8.0 : 12.0) * M.nnz + 20.0 * M.m + (f32 ? 4.0 : 8.0) * B * M.n +
                         8.0 * B * M.m + (Z ? 8.0 * B * M.m : 0.0);
    ph_end(c, SVDSC_PH_SPMV, e0, 1, bytes, 2.0 * M.nnz * B);
    c->n_matvec += B;
    return e == cudaSuccess ? SVDSC_OK : SVDSC_ERR_CUDA;
}

// One CGS pass of the block Y (len x B, columns of the basis) against the
// first ncols columns of W; Pg: Gram partials of the new Y (second pass).
template <int B>
void bcgs_pass(svdsc_ctx *c, const BlockSide &S, bool f32pass, int ncols, double *Y)
{
    BlockWork *w = c->bw;
    const int nbk = nbk_of(S.len, B);
    const double L = (double)S.len;
    const size_t ysm = (f32pass ? sizeof(float) : sizeof(double)) * (size_t)blk_rows(B) * B;
    int e0 = ph_begin(c);
    if (f32pass) {
        static std::atomic<unsigned long long> a{0};
        set_smem_limit_once((const void *)bgemm_t_kernel<B, 4, float>, 200 * 1024, &a);
        bgemm_t_kernel<B, 4, float><<<nbk, kBlkThreads, ysm, c->stream>>>(S.W32, S.ld, ncols, Y, S.ld, S.len, nbk,
                                                                          w->P, poison_ptr(c));
    } else {
        static std::atomic<unsigned long long> a{0};
        set_smem_limit_once((const void *)bgemm_t_kernel<B, 2, double>, 200 * 1024, &a);
        bgemm_t_kernel<B, 2, double><<<nbk, kBlkThreads, ysm, c->stream>>>(S.W, S.ld, ncols, Y, S.ld, S.len, nbk,
                                                                           w->P, poison_ptr(c));
    }
    const double wsz = f32pass ? 4.0 : 8.0;
    ph_end(c, SVDSC_PH_GEMV_T, e0, 1, wsz * L * ncols + 8.0 * L * B, 2.0 * L * ncols * B);
    e0 = ph_begin(c);
    proj_reduce(w->P, nbk, ncols * B, w->H, poison_ptr(c), c->stream);
    ph_end(c, SVDSC_PH_VEC, e0, 1, 8.0 * nbk * ncols * B, (double)nbk * ncols * B);
    e0 = ph_begin(c);
    const size_t hsm = (f32pass ? sizeof(float) : sizeof(double)) * (size_t)ncols * B;
    if (f32pass) {
        static std::atomic<unsigned long long> a{0};
        set_smem_limit_once((const void *)bgemm_n_kernel<B, float>, 200 * 1024, &a);
        bgemm_n_kernel<B, float><<<nbk, kBlkThreads, hsm, c->stream>>>(S.W32, S.ld, ncols, w->H, Y, S.ld, S.len,
                                                                       poison_ptr(c));
    } else {
        static std::atomic<unsigned long long> a{0};
        set_smem_limit_once((const void *)bgemm_n_kernel<B, double>, 200 * 1024, &a);
        bgemm_n_kernel<B, double><<<nbk, kBlkThreads, hsm, c->stream>>>(S.W, S.ld, ncols, w->H, Y, S.ld, S.len,
                                                                        poison_ptr(c));
    }
    ph_end(c, SVDSC_PH_GEMV_N, e0, 1, wsz * L * ncols + 16.0 * L * B, 2.0 * L * ncols * B);
}

// Orthonormalizes the block at columns col..col+B of side `side` against the
// first col columns (CGS2) and within itself (CholQR2); the factor goes to T
// at (tr, tcol) (transposed for a V block).  `step` identifies the block for
// the repair path.
template <int B>
void block_orth(svdsc_ctx *c, int side, int col, int tr, int tcol, int step)
{
    BlockWork *w = c->bw;
    const BlockSide S = side_of(c, side);
    double *Y = S.W + (int64_t)col * S.ld;
    const int nbk = nbk_of(S.len, B);
    const double L = (double)S.len;
    if (col > 0) {
        bcgs_pass<B>(c, S, S.W32 != nullptr, col, Y);
        bcgs_pass<B>(c, S, false, col, Y);
    }
    double *T0 = c->T + tr + (int64_t)tcol * c->t_ld;
    const int trans = side == 1;
    const size_t gsm = sizeof(double) * (size_t)blk_rows(B) * B;
    static std::atomic<unsigned long long> ga{0};
    set_smem_limit_once((const void *)bgram_kernel<B>, 200 * 1024, &ga);
    const int e0 = ph_begin(c);
    bgram_kernel<B><<<nbk, kBlkThreads, gsm, c->stream>>>(Y, S.ld, S.len, nbk, w->P, poison_ptr(c));
    proj_reduce(w->P, nbk, B * B, w->G, poison_ptr(c), c->stream);
    bchol_kernel<<<1, 32, 0, c->stream>>>(B, w->G, w->R1, w->Rinv, nullptr, 1, T0, c->t_ld, trans, c->st,
                                          c->parity, step);
    btrsm_kernel<B><<<nbk, kBlkThreads, 0, c->stream>>>(Y, S.ld, S.len, w->Rinv, nullptr, nullptr, nullptr,
                                                        poison_ptr(c));
    bgram_kernel<B><<<nbk, kBlkThreads, gsm, c->stream>>>(Y, S.ld, S.len, nbk, w->P, poison_ptr(c));
    proj_reduce(w->P, nbk, B * B, w->G, poison_ptr(c), c->stream);
    bchol_kernel<<<1, 32, 0, c->stream>>>(B, w->G, w->R2, w->Rinv, w->R1, 2, T0, c->t_ld, trans, c->st,
                                          c->parity ^ 1, step);
    float *Y32 = S.W32 ? S.W32 + (int64_t)col * S.ld : nullptr;
    btrsm_kernel<B><<<nbk, kBlkThreads, 0, c->stream>>>(Y, S.ld, S.len, w->Rinv, Y32, S.X, S.X32, poison_ptr(c));
    ph_end(c, SVDSC_PH_VEC, e0, 8, 8.0 * L * B * 6 + (Y32 ? 4.0 * L * B : 0.0) + (S.X32 ? 4.0 * L * B : 0.0),
           L * B * (B + 1) + L * B * B);
    w->counts.push_back({c->n_matvec, c->n_steps + B});
    c->steps.push_back({side, col, c->parity});  // block start column, for the repair
    c->n_steps += B;
}

// Block Lanczos steps from cc columns until V holds tc + B columns.
template <int B>
int block_segment(svdsc_ctx *c, int cc, int tc)
{
    NvtxRange range("svdsc: block Lanczos segment");
    for (;;) {
        // Z = A^T U(:, cc-B:cc) - V(:, cc-B:cc) T(cc-B:cc, cc-B:cc)^T
        const void *Xu = c->precision == SVDSC_MIXED ? (const void *)c->bw->Xu32 : (const void *)c->bw->Xu;
        int rc = spmm<B>(c, 1, Xu, c->V + (int64_t)(cc - B) * c->ldv, c->ldv,
                         c->T + (cc - B) + (int64_t)(cc - B) * c->t_ld, 1, c->V + (int64_t)cc * c->ldv, c->ldv);
        if (rc) return rc;
        block_orth<B>(c, 1, cc, cc - B, cc, (int)c->steps.size());
        if (cc >= tc) break;
        // W = A V(:, cc:cc+B) - U(:, cc-B:cc) T(cc-B:cc, cc:cc+B)
        const void *Xv = c->precision == SVDSC_MIXED ? (const void *)c->bw->Xv32 : (const void *)c->bw->Xv;
        rc = spmm<B>(c, 0, Xv, c->U + (int64_t)(cc - B) * c->ldu, c->ldu,
                     c->T + (cc - B) + (int64_t)cc * c->t_ld, 0, c->U + (int64_t)cc * c->ldu, c->ldu);
        if (rc) return rc;
        block_orth<B>(c, 0, cc, cc, cc, (int)c->steps.size());
        cc += B;
    }
    return SVDSC_OK;
}

// Column-by-column QR of a flagged block (the oracle's path): each column is
// projected twice against all earlier columns of its basis (the in-block
// coefficients summed into Rcc), normalised, or replaced by a random vector
// orthogonalized against its predecessors; T gets Rcc R1.
template <int B>
int block_repair(svdsc_ctx *c, int side, int col, int tr, int tcol)
{
    BlockWork *w = c->bw;
    const BlockSide S = side_of(c, side);
    cudaStream_t s = c->stream;
    BCU(cudaMemsetAsync(w->Rcc, 0, sizeof(double) * B * B, s));
    for (int l = 0; l < B; l++) {
        double *y = S.W + (int64_t)(col + l) * S.ld;
        const int nc = col + l;
        for (int pass = 0; pass < 2 && nc > 0; pass++) {
            proj_partial(S.W, S.ld, nc, y, *S.ch, c->P, nullptr, s);
            proj_reduce(c->P, S.ch->nb, nc, c->h, nullptr, s);
            update_sub(S.W, S.ld, nc, c->h, y, *S.ch, pass == 1 ? c->Pn : nullptr, nullptr, s);
            if (l > 0) brepair_accum_kernel<<<1, 32, 0, s>>>(c->h, col, l, B, w->Rcc);
            ph_end(c, SVDSC_PH_OTHER, -1, l > 0 ? 4 : 3, 0.0, 0.0);
        }
        if (nc == 0) norm_partial(y, *S.ch, c->Pn, nullptr, s);
        norm_from_partials(c->Pn, S.ch->nbu, w->G, s);
        const int nb = (int)std::min<int64_t>((S.len + 255) / 256, 4 * 152);
        brepair_norm_kernel<<<nb, 256, 0, s>>>(y, S.len, w->G, l, B, w->Rcc, c->st, c->parity, w->flag, 0);
        ph_end(c, SVDSC_PH_OTHER, -1, 3, 0.0, 0.0);
        int hflag = 0;
        BCU(cudaMemcpyAsync(&hflag, w->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        BCU(cudaStreamSynchronize(s));
        for (int attempt = 0; attempt < 8 && hflag; attempt++) {
            c->breakdowns++;
            rng_normal_vec(c->seed, c->draws++, S.len, y, s);
            if (nc > 0) cgs2_fp64(c, S.W, S.ld, nc, y, *S.ch);
            else norm_partial(y, *S.ch, c->Pn, nullptr, s);
            norm_from_partials(c->Pn, S.ch->nbu, w->G, s);
            brepair_norm_kernel<<<nb, 256, 0, s>>>(y, S.len, w->G, l, B, w->Rcc, c->st, c->parity, w->flag, 1);
            ph_end(c, SVDSC_PH_OTHER, -1, 3, 0.0, 0.0);
            BCU(cudaMemcpyAsync(&hflag, w->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
            BCU(cudaStreamSynchronize(s));
        }
        if (hflag) return SVDSC_ERR_NONFINITE;
    }
    double *T0 = c->T + tr + (int64_t)tcol * c->t_ld;
    brepair_T_kernel<<<1, 32, 0, s>>>(B, w->Rcc, w->R1, T0, c->t_ld, side == 1);
    bcopy_rows_kernel<B><<<4 * 152, 256, 0, s>>>(S.W + (int64_t)col * S.ld, S.ld, S.len, S.X, S.X32,
                                                 S.W32 ? S.W32 + (int64_t)col * S.ld : nullptr);
    ph_end(c, SVDSC_PH_OTHER, -1, 2, 0.0, 0.0);
    BCU(cudaGetLastError());
    return SVDSC_OK;
}

// Waits for the issued work; while a block was flagged, repairs it and
// re-issues the rest of the segment.
template <int B>
int block_settle(svdsc_ctx *c, int tc)
{
    int rc = read_status(c);
    if (rc) return rc;
    int guard = 0;
    while (c->st_host->poison) {
        if (c->st_host->timeout) return SVDSC_ERR_TIMEOUT;
        if (++guard > 4 * (tc / B + 2)) return SVDSC_ERR_NONFINITE;
        const int sb = c->st_host->bd_step;
        if (sb < 0 || sb >= (int)c->steps.size()) return SVDSC_ERR_CUDA;
        const StepRec rec = c->steps[sb];
        c->steps.resize(sb + 1);
        c->bw->counts.resize(sb + 1);
        c->n_matvec = c->bw->counts[sb].first;   // the skipped launches after the block did not run
        c->n_steps = c->bw->counts[sb].second;
        DevStatus fresh = *c->st_host;
        fresh.poison = 0;
        fresh.bd_step = INT_MAX;
        fresh.nonfinite = 0;
        BCU(cudaMemcpyAsync(c->st, &fresh, sizeof(DevStatus), cudaMemcpyHostToDevice, c->stream));
        c->parity = rec.parity;
        const int col = rec.col;
        // a V block at col: T(col-B:col, col:col+B) (transposed); a U block: T(col:col+B, col:col+B)
        rc = block_repair<B>(c, rec.side, col, rec.side == 1 ? std::max(col - B, 0) : col, col);
        if (rc) return rc;
        // resume after the repaired block
        int next = col;
        if (rec.side == 1) {
            if (col < tc) {
                const void *Xv = c->precision == SVDSC_MIXED ? (const void *)c->bw->Xv32 : (const void *)c->bw->Xv;
                rc = spmm<B>(c, 0, Xv, c->U + (int64_t)(col - B) * c->ldu, c->ldu,
                             c->T + (col - B) + (int64_t)col * c->t_ld, 0, c->U + (int64_t)col * c->ldu, c->ldu);
                if (rc) return rc;
                block_orth<B>(c, 0, col, col, col, (int)c->steps.size());
                next = col + B;
                rc = block_segment<B>(c, next, tc);
            }
        } else {
            rc = block_segment<B>(c, col + B, tc);
        }
        if (rc) return rc;
        rc = read_status(c);
        if (rc) return rc;
    }
    if (c->st_host->timeout) return SVDSC_ERR_TIMEOUT;
    return SVDSC_OK;
}

}  // namespace

// Start block V(:, 0:B) (v0 n x B, or draws 0..B-1), orthonormalized; U(:, 0:B) R = A V(:, 0:B).
template <int B>
static int block_start(svdsc_ctx *c, const double *v0, int v0_on_device)
{
    cudaStream_t s = c->stream;
    BlockWork *w = c->bw;
    for (int l = 0; l < B; l++) {
        double *col = c->V + (int64_t)l * c->ldv;
        if (v0)
            BCU(cudaMemcpyAsync(col, v0 + (int64_t)l * c->n, sizeof(double) * c->n,
                                v0_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        else
            rng_normal_vec(c->seed, (uint64_t)l, c->n, col, s);
    }
    c->draws = B;
    ph_end(c, SVDSC_PH_OTHER, -1, v0 ? 0 : B, 0.0, 0.0);
    // the start block: any nonzero column counts as independent (anorm 0 here)
    block_orth<B>(c, 1, 0, 0, 0, 0);
    int rc = block_settle<B>(c, 0);
    if (rc) return rc;
    // its factor is not part of T: clear what the orthonormalization wrote
    BCU(cudaMemsetAsync(c->T, 0, sizeof(double) * (size_t)c->t_ld * c->t_ld, s));
    c->steps.clear();
    w->counts.clear();
    c->n_steps = 0;
    c->n_matvec = 0;
    c->breakdowns = 0;
    {
        DevStatus init;
        memset(&init, 0, sizeof(init));
        init.bd_step = INT_MAX;
        BCU(cudaMemcpyAsync(c->st, &init, sizeof(DevStatus), cudaMemcpyHostToDevice, s));
        c->parity = 0;
    }
    const void *Xv = c->precision == SVDSC_MIXED ? (const void *)w->Xv32 : (const void *)w->Xv;
    rc = spmm<B>(c, 0, Xv, nullptr, 0, nullptr, 0, c->U, c->ldu);
    if (rc) return rc;
    block_orth<B>(c, 0, 0, 0, 0, (int)c->steps.size());
    return SVDSC_OK;
}

template <int B>
static int solve_block_t(svdsc_ctx *c, int k, int t0, int t1, double tol, int maxit, const double *v0,
                         int v0_on_device, double **Uo, double **Vo, int *restarts_out, DevStatus *fin)
{
    cudaStream_t s = c->stream;
    BlockWork *w = c->bw;
    int rc = block_start<B>(c, v0, v0_on_device);
    if (rc) return rc;
    rc = block_segment<B>(c, B, t0);
    if (rc) return rc;
    rc = block_settle<B>(c, t0);
    if (rc) return rc;
    int tc = t0, restarts = 0;
    for (int it = 1; it <= maxit; it++) {
        {
            const int e0 = ph_begin(c);
            NvtxRange range("svdsc: projected SVD");
            BCU(small_svd(tc, c->T, c->t_ld, c->Sh, c->Uh, c->Vh, c->svd, c->st, s, nullptr));
            ph_end(c, SVDSC_PH_SVD, e0, 1, 0.0, 0.0);
        }
        {
            const int e0 = ph_begin(c);
            bresidual_kernel<<<1, 256, 0, s>>>(tc, k, B, tol, c->T, c->t_ld, c->Sh, c->Uh, c->res, w->rho, c->st,
                                               c->parity);
            ph_end(c, SVDSC_PH_OTHER, e0, 1, 0.0, 0.0);
        }
        BCU(cudaGetLastError());
        rc = read_status(c);
        if (rc) return rc;
        if (c->st_host->timeout) return SVDSC_ERR_TIMEOUT;
        if (c->st_host->converged || it == maxit) break;
        NvtxRange restart_range("svdsc: augmented restart");
        // U~_k = U(:, 0:tc) Uh(:, 0:k), V~_k = V(:, 0:tc) Vh(:, 0:k) into the other bases
        rc = gemm_tc(c, c->U, c->U32, c->ldu, c->m, tc, c->Uh, k, c->Ua, c->U32a);
        if (rc) return rc;
        rc = gemm_tc(c, c->V, c->V32, c->ldv, c->n, tc, c->Vh, k, c->Va, c->V32a);
        if (rc) return rc;
        // V(:, k:k+B) = V(:, tc:tc+B) (its row-major copy is still the newest V block's)
        BCU(cudaMemcpy2DAsync(c->Va + (int64_t)k * c->ldv, sizeof(double) * c->ldv, c->V + (int64_t)tc * c->ldv,
                              sizeof(double) * c->ldv, sizeof(double) * c->n, B, cudaMemcpyDeviceToDevice, s));
        if (c->V32)
            BCU(cudaMemcpy2DAsync(c->V32a + (int64_t)k * c->ldv, sizeof(float) * c->ldv,
                                  c->V32 + (int64_t)tc * c->ldv, sizeof(float) * c->ldv, sizeof(float) * c->n, B,
                                  cudaMemcpyDeviceToDevice, s));
        std::swap(c->U, c->Ua);
        std::swap(c->V, c->Va);
        std::swap(c->U32, c->U32a);
        std::swap(c->V32, c->V32a);
        brestart_T_kernel<<<1, 256, 0, s>>>(c->t_ld, k, B, c->T, c->Sh, w->rho);
        ph_end(c, SVDSC_PH_OTHER, -1, 1, 0.0, 0.0);
        // W = A V(:, k:k+B) - U~_k rho, orthonormalized against U~_k
        const void *Xv = c->precision == SVDSC_MIXED ? (const void *)w->Xv32 : (const void *)w->Xv;
        rc = spmm<B>(c, 0, Xv, nullptr, 0, nullptr, 0, c->U + (int64_t)k * c->ldu, c->ldu);
        if (rc) return rc;
        {
            const int e0 = ph_begin(c);
            const int nbk = nbk_of(c->m, B);
            static std::atomic<unsigned long long> a{0};
            set_smem_limit_once((const void *)bgemm_n_kernel<B, double>, 200 * 1024, &a);
            bgemm_n_kernel<B, double><<<nbk, kBlkThreads, sizeof(double) * (size_t)k * B, s>>>(
                c->U, c->ldu, k, w->rho, c->U + (int64_t)k * c->ldu, c->ldu, c->m, poison_ptr(c));
            ph_end(c, SVDSC_PH_GEMV_N, e0, 1, 8.0 * c->m * k + 16.0 * c->m * B, 2.0 * c->m * k * B);
        }
        block_orth<B>(c, 0, k, k, k, (int)c->steps.size());
        restarts++;
        tc = t1;
        rc = block_segment<B>(c, k + B, t1);
        if (rc) return rc;
        rc = block_settle<B>(c, t1);
        if (rc) return rc;
    }
    *fin = *c->st_host;
    *restarts_out = restarts;
    c->t = tc;  // size of the last projected matrix (reported in svdsc_info.t)
    // outputs of the last projected SVD
    rc = gemm_tc(c, c->U, c->U32, c->ldu, c->m, tc, c->Uh, k, c->Ua, nullptr);
    if (rc) return rc;
    rc = gemm_tc(c, c->V, c->V32, c->ldv, c->n, tc, c->Vh, k, c->Va, nullptr);
    if (rc) return rc;
    *Uo = c->Ua;
    *Vo = c->Va;
    return SVDSC_OK;
}

namespace svdsc {

void block_free(svdsc_ctx *c)
{
    BlockWork *w = c->bw;
    if (!w) return;
    cudaFree(w->Xu); cudaFree(w->Xv); cudaFree(w->Xu32); cudaFree(w->Xv32);
    cudaFree(w->P); cudaFree(w->H); cudaFree(w->G); cudaFree(w->R1); cudaFree(w->Rinv); cudaFree(w->R2);
    cudaFree(w->Rcc); cudaFree(w->rho); cudaFree(w->flag);
    delete w;
    c->bw = nullptr;
}

static int block_reserve(svdsc_ctx *c, int tcap, int k)
{
    const int B = c->block;
    BlockWork *w = c->bw;
    if (w && w->tcap >= tcap && w->b == B) return SVDSC_OK;
    cudaStreamSynchronize(c->stream);
    block_free(c);
    w = new (std::nothrow) BlockWork();
    if (!w) return SVDSC_ERR_NOMEM;
    c->bw = w;
    w->b = B;
    w->tcap = tcap;
    bool ok = true;
    auto alloc = [&](void **p, size_t bytes) {
        if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) ok = false;
    };
    const bool mixed = c->precision == SVDSC_MIXED;
    alloc((void **)&w->Xu, sizeof(double) * (size_t)c->m * B);
    alloc((void **)&w->Xv, sizeof(double) * (size_t)c->n * B);
    if (mixed) {
        alloc((void **)&w->Xu32, sizeof(float) * (size_t)c->m * B);
        alloc((void **)&w->Xv32, sizeof(float) * (size_t)c->n * B);
    }
    const int nbk = std::max(nbk_of(c->m, B), nbk_of(c->n, B));
    w->P_doubles = (size_t)nbk * std::max(tcap * B, B * B);
    alloc((void **)&w->P, sizeof(double) * w->P_doubles);
    alloc((void **)&w->H, sizeof(double) * (size_t)std::max(tcap, k) * B);
    alloc((void **)&w->G, sizeof(double) * B * B);
    alloc((void **)&w->R1, sizeof(double) * B * B);
    alloc((void **)&w->Rinv, sizeof(double) * B * B);
    alloc((void **)&w->R2, sizeof(double) * B * B);
    alloc((void **)&w->Rcc, sizeof(double) * B * B);
    alloc((void **)&w->rho, sizeof(double) * (size_t)tcap * B);
    alloc((void **)&w->flag, sizeof(int));
    if (!ok) {
        block_free(c);
        cudaGetLastError();
        return SVDSC_ERR_NOMEM;
    }
    return SVDSC_OK;
}

int solve_block(svdsc_ctx *c, int k, int p, double tol, int maxit, const double *v0, int v0_on_device,
                double **Uo, double **Vo, int *restarts, DevStatus *fin)
{
    const int B = c->block;
    const int t = (p < 0) ? std::max(15, 3 * k) : k + p;
    const int t0 = B * ((t + B - 1) / B), t1 = k + B * ((t - k + B - 1) / B);
    const int tmax = std::max(t0, t1);
    if (k + B > t1 || tmax > c->m || tmax + B > c->n || tmax > 448 || tmax + B > 512) return SVDSC_ERR_SIZE;
    int rc = reserve_ws(c, tmax + B);
    if (rc) return rc;
    rc = block_reserve(c, tmax + B, k);
    if (rc) return rc;
    c->t = tmax;  // workspace bookkeeping; the projected size varies (t0, t1)
    c->t_ld = tmax + B;
    c->k = k;
    BCU(cudaMemsetAsync(c->T, 0, sizeof(double) * (size_t)c->t_ld * c->t_ld, c->stream));
    switch (B) {
    case 2: rc = solve_block_t<2>(c, k, t0, t1, tol, maxit, v0, v0_on_device, Uo, Vo, restarts, fin); break;
    case 4: rc = solve_block_t<4>(c, k, t0, t1, tol, maxit, v0, v0_on_device, Uo, Vo, restarts, fin); break;
    case 8: rc = solve_block_t<8>(c, k, t0, t1, tol, maxit, v0, v0_on_device, Uo, Vo, restarts, fin); break;
    case 16: rc = solve_block_t<16>(c, k, t0, t1, tol, maxit, v0, v0_on_device, Uo, Vo, restarts, fin); break;
    default: return SVDSC_ERR_ARG;
    }
    return rc;
}

}  // namespace svdsc
