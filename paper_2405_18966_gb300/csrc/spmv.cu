// Products with A and A^T (Alg. 1 of the svds-C paper):
// a row-length-binned CSR SpMV (one launch covers every bin), dense
// column-major GEMV / GEMV-T, and the create-time preparation of CSR(A) and
// CSR(A^T) (0-based compaction, validation, deterministic transpose, bins).
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>
#include "internal.cuh"

namespace svdsc {

// ----------------------------------------------------------------- binned SpMV

template <int G, typename VT, typename XT, typename AT>
__device__ __forceinline__ AT spmv_row_group(const int64_t *__restrict__ row_ptr,
                                             const int32_t *__restrict__ col,
                                             const VT *__restrict__ val,
                                             const XT *__restrict__ x, int64_t r, int lg,
                                             unsigned gmask)
{
    const int64_t e0 = row_ptr[r], e1 = row_ptr[r + 1];
    AT a0 = AT(0), a1 = AT(0);
    int64_t e = e0 + lg;
    for (; e + 3 * G < e1; e += 4 * G) {  // four independent loads in flight per lane
        const int32_t c0 = __ldcs(col + e), c1 = __ldcs(col + e + G), c2 = __ldcs(col + e + 2 * G),
                      c3 = __ldcs(col + e + 3 * G);
        const VT v0 = __ldcs(val + e), v1 = __ldcs(val + e + G), v2 = __ldcs(val + e + 2 * G),
                 v3 = __ldcs(val + e + 3 * G);
        a0 += AT(v0) * AT(__ldg(x + c0));
        a1 += AT(v1) * AT(__ldg(x + c1));
        a0 += AT(v2) * AT(__ldg(x + c2));
        a1 += AT(v3) * AT(__ldg(x + c3));
    }
    for (; e < e1; e += G) a0 += AT(__ldg(val + e)) * AT(__ldg(x + __ldg(col + e)));
    AT s = a0 + a1;
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o);
    return s;
}

template <int G, typename VT, typename XT, typename AT>
__device__ __forceinline__ void spmv_bin(const int64_t *__restrict__ row_ptr,
                                         const int32_t *__restrict__ col,
                                         const VT *__restrict__ val, const XT *__restrict__ x,
                                         const int32_t *__restrict__ perm, int64_t row_begin,
                                         int64_t row_end, int64_t lb, const double *__restrict__ z,
                                         double coef, double *__restrict__ y)
{
    const int grp = threadIdx.x / G, lg = threadIdx.x % G;
    const int64_t idx = row_begin + lb * (kSpmvThreads / G) + grp;
    if (idx >= row_end) return;  // whole groups leave together
    const unsigned gmask = (G == 32) ? 0xffffffffu
                                     : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
    const int64_t r = perm[idx];
    AT s = spmv_row_group<G, VT, XT, AT>(row_ptr, col, val, x, r, lg, gmask);
    if (lg == 0) y[r] = double(s) - (z ? coef * z[r] : 0.0);
}

template <typename VT, typename XT, typename AT>
__global__ void __launch_bounds__(kSpmvThreads)
csr_spmv_binned(const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                const VT *__restrict__ val, const XT *__restrict__ x,
                const int32_t *__restrict__ perm, const __grid_constant__ Bins bins,
                const double *__restrict__ z,
                const double *__restrict__ coef_dev, double coef_h, double *__restrict__ y,
                const int *poison, int64_t sell_rows, int64_t sell_blocks,
                const int32_t *__restrict__ sell_perm, const int64_t *__restrict__ sell_off,
                const int32_t *__restrict__ sell_col, const VT *__restrict__ sell_val)
{
    if (poison && *(volatile const int *)poison) return;
    if ((int64_t)blockIdx.x < sell_blocks) {
        // SELL-32: one thread per row, slice-column-major storage
        const int64_t i = (int64_t)blockIdx.x * kSpmvThreads + threadIdx.x;
        if (i >= sell_rows) return;
        const int64_t sl = i >> 5;
        const int lane = (int)(i & 31);
        const int64_t off = sell_off[sl];
        const int w = (int)((sell_off[sl + 1] - off) >> 5);
        const int32_t *cp = sell_col + off + lane;
        const VT *vp = sell_val + off + lane;
        AT a0 = AT(0), a1 = AT(0), a2 = AT(0), a3 = AT(0);
        int j = 0;
        for (; j + 3 < w; j += 4) {
            // the matrix is streamed with evict-first loads so that the gathered
            // vector x stays resident in L2
            const int32_t c0 = __ldcs(cp + 32 * j), c1 = __ldcs(cp + 32 * (j + 1)), c2 = __ldcs(cp + 32 * (j + 2)),
                          c3 = __ldcs(cp + 32 * (j + 3));
            const VT v0 = __ldcs(vp + 32 * j), v1 = __ldcs(vp + 32 * (j + 1)), v2 = __ldcs(vp + 32 * (j + 2)),
                     v3 = __ldcs(vp + 32 * (j + 3));
            a0 += AT(v0) * AT(__ldg(x + c0));
            a1 += AT(v1) * AT(__ldg(x + c1));
            a2 += AT(v2) * AT(__ldg(x + c2));
            a3 += AT(v3) * AT(__ldg(x + c3));
        }
        for (; j < w; j++) a0 += AT(__ldcs(vp + 32 * j)) * AT(__ldg(x + __ldcs(cp + 32 * j)));
        const int64_t r = sell_perm[i];
        const double coef = coef_dev ? *coef_dev : coef_h;
        y[r] = double((a0 + a1) + (a2 + a3)) - (z ? coef * z[r] : 0.0);
        return;
    }
    const int64_t b = blockIdx.x - sell_blocks;
    int bin = 0;
#pragma unroll
    for (int i = 1; i < kNumBins; i++)
        if (b >= bins.block_start[i]) bin = i;
    const int64_t lb = b - bins.block_start[bin];
    const double coef = coef_dev ? *coef_dev : coef_h;
    const int64_t rb = bins.row_start[bin], re = bins.row_start[bin + 1];
    switch (bin) {
    case 0:
    case 1:
    case 2:
    case 3: spmv_bin<1, VT, XT, AT>(row_ptr, col, val, x, perm, rb, re, lb, z, coef, y); return;
    case 4: spmv_bin<2, VT, XT, AT>(row_ptr, col, val, x, perm, rb, re, lb, z, coef, y); return;
    case 5: spmv_bin<4, VT, XT, AT>(row_ptr, col, val, x, perm, rb, re, lb, z, coef, y); return;
    case 6: spmv_bin<8, VT, XT, AT>(row_ptr, col, val, x, perm, rb, re, lb, z, coef, y); return;
    case 7: spmv_bin<16, VT, XT, AT>(row_ptr, col, val, x, perm, rb, re, lb, z, coef, y); return;
    case 8: spmv_bin<32, VT, XT, AT>(row_ptr, col, val, x, perm, rb, re, lb, z, coef, y); return;
    default: break;
    }
    // a whole CTA per (very long) row
    const int64_t r = perm[rb + lb];
    const int64_t e0 = row_ptr[r], e1 = row_ptr[r + 1];
    AT s = AT(0);
    for (int64_t e = e0 + threadIdx.x; e < e1; e += kSpmvThreads)
        s += AT(__ldg(val + e)) * AT(__ldg(x + __ldg(col + e)));
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ AT red[kSpmvThreads / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        AT t = AT(0);
        for (int w = 0; w < kSpmvThreads / 32; w++) t += red[w];
        y[r] = double(t) - (z ? coef * z[r] : 0.0);
    }
}

static int64_t bin_blocks(const Bins &b) { return b.block_start[kNumBins]; }
static int64_t sell_blocks(const DevCSR &A) { return (A.sell_rows + kSpmvThreads - 1) / kSpmvThreads; }

cudaError_t csr_spmv_f64(const DevCSR &A, const double *x, const double *z, const double *coef_dev,
                         double coef_h, double *y, const int *poison, cudaStream_t s)
{
    const int64_t sb = sell_blocks(A);
    const int64_t nblk = sb + bin_blocks(A.bins);
    if (nblk == 0) return cudaSuccess;
    csr_spmv_binned<double, double, double><<<(unsigned)nblk, kSpmvThreads, 0, s>>>(
        A.row_ptr, A.col, A.val, x, A.perm, A.bins, z, coef_dev, coef_h, y, poison, A.sell_rows, sb,
        A.sell_perm, A.sell_off, A.sell_col, A.sell_val);
    return cudaGetLastError();
}

cudaError_t csr_spmv_f32(const DevCSR &A, const float *x, const double *z, const double *coef_dev,
                         double coef_h, double *y, const int *poison, cudaStream_t s)
{
    const int64_t sb = sell_blocks(A);
    const int64_t nblk = sb + bin_blocks(A.bins);
    if (nblk == 0) return cudaSuccess;
    csr_spmv_binned<float, float, float><<<(unsigned)nblk, kSpmvThreads, 0, s>>>(
        A.row_ptr, A.col, A.val32, x, A.perm, A.bins, z, coef_dev, coef_h, y, poison, A.sell_rows, sb,
        A.sell_perm, A.sell_off, A.sell_col, A.sell_val32);
    return cudaGetLastError();
}

// ----------------------------------------------------------------- dense GEMV
// y = A x: CTAs tile (512 rows) x (a slice of columns); partial sums per slice
// are added in slice order by a second kernel (deterministic).
constexpr int kGemvRowsPerCta = 512;

static void dense_n_shape(const DevDense &A, int64_t *cs, int *nslices)
{
    const int64_t rblocks = (A.m + kGemvRowsPerCta - 1) / kGemvRowsPerCta;
    int64_t want = (4 * 152 + rblocks - 1) / rblocks;
    int64_t maxs = (A.n + 15) / 16;
    int64_t ns = std::max<int64_t>(1, std::min(want, maxs));
    *cs = (A.n + ns - 1) / ns;
    *nslices = (int)((A.n + *cs - 1) / *cs);
}

static void dense_t_shape(const DevDense &A, int64_t *rc, int *nchunks)
{
    const int64_t ccta = (A.n + 7) / 8;
    int64_t want = (4 * 152 + ccta - 1) / ccta;
    int64_t maxc = std::max<int64_t>(1, (A.m + 2047) / 2048);
    int64_t nc = std::max<int64_t>(1, std::min(want, maxc));
    int64_t r = (A.m + nc - 1) / nc;
    r = (r + 1) & ~int64_t(1);
    *rc = r;
    *nchunks = (int)((A.m + r - 1) / r);
}

size_t dense_partial_doubles(const DevDense &A)
{
    int64_t cs, rc;
    int ns, nc;
    dense_n_shape(A, &cs, &ns);
    dense_t_shape(A, &rc, &nc);
    return (size_t)std::max<int64_t>((int64_t)ns * A.m, (int64_t)nc * A.n);
}

__global__ void __launch_bounds__(256)
gemv_n_partial(const double *__restrict__ A, int64_t ld, int64_t m, int64_t n,
               const double *__restrict__ x, int64_t cs, double *__restrict__ part,
               const int *poison)
{
    if (poison && *(volatile const int *)poison) return;
    const int64_t c0 = (int64_t)blockIdx.y * cs;
    const int64_t c1 = min(n, c0 + cs);
    const int64_t r = ((int64_t)blockIdx.x * 256 + threadIdx.x) * 2;
    if (r >= m) return;
    double a0 = 0.0, a1 = 0.0;
    if (r + 1 < m && (ld & 1) == 0) {
        const double *p = A + c0 * ld + r;
        int64_t c = c0;
        for (; c + 3 < c1; c += 4) {
            const double2 v0 = __ldg((const double2 *)(p));
            const double2 v1 = __ldg((const double2 *)(p + ld));
            const double2 v2 = __ldg((const double2 *)(p + 2 * ld));
            const double2 v3 = __ldg((const double2 *)(p + 3 * ld));
            const double x0 = __ldg(x + c), x1 = __ldg(x + c + 1), x2 = __ldg(x + c + 2),
                         x3 = __ldg(x + c + 3);
            a0 = fma(v0.x, x0, a0); a1 = fma(v0.y, x0, a1);
            a0 = fma(v1.x, x1, a0); a1 = fma(v1.y, x1, a1);
            a0 = fma(v2.x, x2, a0); a1 = fma(v2.y, x2, a1);
            a0 = fma(v3.x, x3, a0); a1 = fma(v3.y, x3, a1);
            p += 4 * ld;
        }
        for (; c < c1; c++, p += ld) {
            const double2 v = __ldg((const double2 *)p);
            const double xc = __ldg(x + c);
            a0 = fma(v.x, xc, a0); a1 = fma(v.y, xc, a1);
        }
        part[blockIdx.y * m + r] = a0;
        part[blockIdx.y * m + r + 1] = a1;
    } else {
        for (int64_t rr = r; rr < min(m, r + 2); rr++) {
            double a = 0.0;
            for (int64_t c = c0; c < c1; c++) a = fma(__ldg(A + c * ld + rr), __ldg(x + c), a);
            part[blockIdx.y * m + rr] = a;
        }
    }
}

__global__ void sum_slices(const double *__restrict__ part, int ns, int64_t len,
                           const double *__restrict__ z, const double *__restrict__ coef_dev,
                           double coef_h, double *__restrict__ y, const int *poison)
{
    if (poison && *(volatile const int *)poison) return;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= len) return;
    double s = 0.0;
    for (int i = 0; i < ns; i++) s += part[(int64_t)i * len + r];
    const double coef = coef_dev ? *coef_dev : coef_h;
    y[r] = s - (z ? coef * z[r] : 0.0);
}

cudaError_t dense_gemv_n(const DevDense &A, const double *x, const double *z, const double *coef_dev,
                         double coef_h, double *y, double *partial, const int *poison,
                         cudaStream_t s, int *launches)
{
    int64_t cs;
    int ns;
    dense_n_shape(A, &cs, &ns);
    dim3 grid((unsigned)((A.m + kGemvRowsPerCta - 1) / kGemvRowsPerCta), (unsigned)ns);
    gemv_n_partial<<<grid, 256, 0, s>>>(A.a, A.ld, A.m, A.n, x, cs, partial, poison);
    sum_slices<<<(unsigned)((A.m + 255) / 256), 256, 0, s>>>(partial, ns, A.m, z, coef_dev,
                                                            coef_h, y, poison);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

// z = A^T x: one warp per column over a chunk of rows.
__global__ void __launch_bounds__(256)
gemv_t_partial(const double *__restrict__ A, int64_t ld, int64_t m, int64_t n,
               const double *__restrict__ x, int64_t rc, double *__restrict__ part,
               const int *poison)
{
    if (poison && *(volatile const int *)poison) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * 8 + warp;
    if (c >= n) return;
    const int64_t r0 = (int64_t)blockIdx.y * rc;
    const int64_t r1 = min(m, r0 + rc);
    const double *col = A + c * ld;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    if ((ld & 1) == 0) {
        int64_t r = r0 + 2 * lane;
        for (; r + 65 < r1; r += 128) {
            const double2 v0 = __ldg((const double2 *)(col + r));
            const double2 v1 = __ldg((const double2 *)(col + r + 64));
            const double2 x0 = __ldg((const double2 *)(x + r));
            const double2 x1 = __ldg((const double2 *)(x + r + 64));
            a0 = fma(v0.x, x0.x, a0); a1 = fma(v0.y, x0.y, a1);
            a2 = fma(v1.x, x1.x, a2); a3 = fma(v1.y, x1.y, a3);
        }
        for (; r < r1; r += 64) {
            a0 = fma(__ldg(col + r), __ldg(x + r), a0);
            if (r + 1 < r1) a1 = fma(__ldg(col + r + 1), __ldg(x + r + 1), a1);
        }
    } else {
        for (int64_t r = r0 + lane; r < r1; r += 32) a0 = fma(__ldg(col + r), __ldg(x + r), a0);
    }
    double s = (a0 + a1) + (a2 + a3);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) part[blockIdx.y * n + c] = s;
}

cudaError_t dense_gemv_t(const DevDense &A, const double *x, const double *z, const double *coef_dev,
                         double coef_h, double *y, double *partial, const int *poison,
                         cudaStream_t s, int *launches)
{
    int64_t rc;
    int nc;
    dense_t_shape(A, &rc, &nc);
    dim3 grid((unsigned)((A.n + 7) / 8), (unsigned)nc);
    gemv_t_partial<<<grid, 256, 0, s>>>(A.a, A.ld, A.m, A.n, x, rc, partial, poison);
    sum_slices<<<(unsigned)((A.n + 255) / 256), 256, 0, s>>>(partial, nc, A.n, z, coef_dev,
                                                            coef_h, y, poison);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

// ------------------------------------------------------- create-time preparation

// out[0] = 0, out[i+1] = out[i] + len[i]  (lengths from begin/end arrays or counts)
__global__ void scan_tile_sums(const int64_t *__restrict__ len, int64_t n, int64_t *__restrict__ tile_sum)
{
    __shared__ int64_t red[32];
    const int64_t i0 = (int64_t)blockIdx.x * 1024;
    int64_t v = 0;
    for (int j = threadIdx.x; j < 1024; j += blockDim.x)
        if (i0 + j < n) v += len[i0 + j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < (int)(blockDim.x / 32); w++) t += red[w];
        tile_sum[blockIdx.x] = t;
    }
}

__global__ void scan_tiles_serial(int64_t *tile_sum, int64_t ntiles)
{
    // one thread: exclusive scan of the tile sums (ntiles <= a few 1e5)
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t acc = 0;
    for (int64_t i = 0; i < ntiles; i++) {
        int64_t v = tile_sum[i];
        tile_sum[i] = acc;
        acc += v;
    }
    tile_sum[ntiles] = acc;
}

__global__ void scan_tile_apply(const int64_t *__restrict__ len, int64_t n,
                                const int64_t *__restrict__ tile_off, int64_t *__restrict__ out)
{
    // 1024 elements per CTA of 1024 threads: Hillis-Steele in shared memory
    __shared__ int64_t buf[1024];
    const int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    buf[threadIdx.x] = (i < n) ? len[i] : 0;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int64_t t = (threadIdx.x >= (unsigned)o) ? buf[threadIdx.x - o] : 0;
        __syncthreads();
        buf[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i + 1] = tile_off[blockIdx.x] + buf[threadIdx.x];
    if (i == 0) out[0] = 0;
}

static cudaError_t exclusive_scan(const int64_t *len, int64_t n, int64_t *out, int64_t *tmp,
                                  cudaStream_t s)
{
    const int64_t ntiles = (n + 1023) / 1024;
    if (n == 0) return cudaMemsetAsync(out, 0, sizeof(int64_t), s);
    scan_tile_sums<<<(unsigned)ntiles, 256, 0, s>>>(len, n, tmp);
    scan_tiles_serial<<<1, 32, 0, s>>>(tmp, ntiles);
    scan_tile_apply<<<(unsigned)ntiles, 1024, 0, s>>>(len, n, tmp, out);
    return cudaGetLastError();
}

// Validation of the caller's CSR (begin/end per row, index base, extent).
__global__ void csr_validate(const int64_t *__restrict__ rb, const int64_t *__restrict__ re,
                             int64_t m, int64_t n, int64_t extent, int base,
                             const int32_t *__restrict__ col, int *bad, int64_t *len)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    const int64_t b = rb[r] - base, e = re[r] - base;
    if (b < 0 || e < b || e > extent) {
        atomicOr(bad, 1);
        len[r] = 0;
        return;
    }
    len[r] = e - b;
    for (int64_t j = b; j < e; j++) {
        const int64_t c = (int64_t)col[j] - base;
        if (c < 0 || c >= n) { atomicOr(bad, 2); return; }
    }
}

template <typename VT>
__global__ void csr_compact(const int64_t *__restrict__ rb, int64_t m, int base,
                            const int32_t *__restrict__ col_in, const VT *__restrict__ val_in,
                            const int64_t *__restrict__ rp_out, int32_t *__restrict__ col_out,
                            double *__restrict__ val64, float *__restrict__ val32, int *bad)
{
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= m) return;
    const int64_t b = rb[r] - base;
    const int64_t o = rp_out[r], len = rp_out[r + 1] - o;
    for (int64_t j = lane; j < len; j += 32) {
        const double v = (double)val_in[b + j];
        if (!isfinite(v)) atomicOr(bad, 4);
        col_out[o + j] = col_in[b + j] - base;
        if (val64) val64[o + j] = v;
        if (val32) val32[o + j] = (float)v;
    }
}

__global__ void col_count(const int32_t *__restrict__ col, int64_t nnz,
                          unsigned long long *__restrict__ cnt)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt + col[e], 1ull);
}

__global__ void col_scatter(const int32_t *__restrict__ col, int64_t nnz,
                            unsigned long long *__restrict__ cursor, int64_t *__restrict__ keys)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long pos = atomicAdd(cursor + col[e], 1ull);
        keys[pos] = e;
    }
}

// Sort the keys of each A^T row ascending (keys are distinct nnz positions of
// A, so the order is unique): short segments by one thread, longer ones by a
// CTA with a bitonic network (+inf padding, ascending comparators only).
__global__ void seg_sort_short(const int64_t *__restrict__ rp, const int32_t *__restrict__ segs,
                               int64_t nseg, int64_t *__restrict__ keys)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nseg) return;
    const int64_t s = segs[i];
    int64_t *k = keys + rp[s];
    const int64_t L = rp[s + 1] - rp[s];
    for (int64_t a = 1; a < L; a++) {
        const int64_t v = k[a];
        int64_t b = a - 1;
        while (b >= 0 && k[b] > v) { k[b + 1] = k[b]; b--; }
        k[b + 1] = v;
    }
}

__device__ void bitonic_sort_block(int64_t *k, int64_t L)
{
    int64_t P = 1;
    while (P < L) P <<= 1;
    for (int64_t size = 2; size <= P; size <<= 1) {
        // flip step: compare i with i ^ (size - 1)
        for (int64_t t = threadIdx.x; t < P / 2; t += blockDim.x) {
            const int64_t lo = (t / (size / 2)) * size + (t % (size / 2));
            const int64_t hi = lo ^ (size - 1);
            if (hi < L && k[lo] > k[hi]) { int64_t x = k[lo]; k[lo] = k[hi]; k[hi] = x; }
        }
        __syncthreads();
        for (int64_t j = size / 4; j >= 1; j >>= 1) {
            for (int64_t t = threadIdx.x; t < P / 2; t += blockDim.x) {
                const int64_t lo = (t / j) * 2 * j + (t % j);
                const int64_t hi = lo + j;
                if (hi < L && k[lo] > k[hi]) { int64_t x = k[lo]; k[lo] = k[hi]; k[hi] = x; }
            }
            __syncthreads();
        }
    }
}

constexpr int kSmemSortKeys = 4096;  // 32 KB of static shared memory

__global__ void __launch_bounds__(512)
seg_sort_block(const int64_t *__restrict__ rp, const int32_t *__restrict__ segs,
               int64_t *__restrict__ keys)
{
    __shared__ int64_t sk[kSmemSortKeys];
    const int64_t s = segs[blockIdx.x];
    int64_t *k = keys + rp[s];
    const int64_t L = rp[s + 1] - rp[s];
    if (L <= kSmemSortKeys) {
        for (int64_t j = threadIdx.x; j < L; j += blockDim.x) sk[j] = k[j];
        __syncthreads();
        bitonic_sort_block(sk, L);
        for (int64_t j = threadIdx.x; j < L; j += blockDim.x) k[j] = sk[j];
    } else {
        bitonic_sort_block(k, L);  // in global memory (very long columns only)
    }
}

__global__ void transpose_fill(const int64_t *__restrict__ keys, int64_t nnz,
                               const int64_t *__restrict__ rp, int64_t m,
                               const double *__restrict__ val64, const float *__restrict__ val32,
                               int32_t *__restrict__ colT, double *__restrict__ valT64,
                               float *__restrict__ valT32)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nnz;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = keys[j];
        // row of e: largest r with rp[r] <= e
        int64_t lo = 0, hi = m - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (rp[mid] <= e) lo = mid; else hi = mid - 1;
        }
        colT[j] = (int32_t)lo;
        if (valT64) valT64[j] = val64[e];
        if (valT32) valT32[j] = val32[e];
    }
}

#define PREP_TRY(x)                                    \
    do {                                               \
        cudaError_t e_ = (x);                          \
        if (e_ != cudaSuccess) { rc = SVDSC_ERR_CUDA; goto done; } \
    } while (0)

// Lanes per row are chosen so that each lane does >= 4 FMAs: on GB300 every
// warp-wide FP64 instruction occupies the FP64 pipe for 16 SM cycles, so a
// shuffle reduction over many lanes of a short row costs more than its FMAs.
// Lanes per row are chosen so that each lane does >= 4 FMAs: on GB300 every
// warp-wide FP64 instruction occupies the FP64 pipe for 16 SM cycles, so a
// shuffle reduction over many lanes of a short row costs more than its FMAs.
// Rows handled by one lane are further split by length (1, 2, 3-4, 5-8) so
// the lanes of a warp run loops of similar length.
static int bin_of(int64_t len)
{
    if (len <= 1) return 0;      // 1 lane per row
    if (len <= 2) return 1;
    if (len <= 4) return 2;
    if (len <= 8) return 3;
    if (len <= 16) return 4;     // 2
    if (len <= 32) return 5;     // 4
    if (len <= 64) return 6;     // 8
    if (len <= 128) return 7;    // 16
    if (len <= 4096) return 8;   // 32 (a warp)
    return 9;                    // a CTA
}

static int bin_lanes(int bin) { return bin <= 3 ? 1 : (bin == 9 ? kSpmvThreads : 1 << (bin - 3)); }

// Fills the padded SELL-32 arrays: thread per (slice, lane); lanes past the
// last row of the last slice are all padding.
__global__ void sell_fill_kernel(const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                 const double *__restrict__ val, const float *__restrict__ val32,
                                 const int32_t *__restrict__ sell_perm, const int64_t *__restrict__ sell_off,
                                 int64_t sell_rows, int64_t slices, int32_t *__restrict__ scol,
                                 double *__restrict__ sval, float *__restrict__ sval32)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= slices * 32) return;
    const int64_t sl = i >> 5;
    const int lane = (int)(i & 31);
    const int64_t off = sell_off[sl];
    const int w = (int)((sell_off[sl + 1] - off) >> 5);
    int64_t e0 = 0, len = 0;
    if (i < sell_rows) {
        const int64_t r = sell_perm[i];
        e0 = row_ptr[r];
        len = row_ptr[r + 1] - e0;
    }
    for (int j = 0; j < w; j++) {
        const int64_t d = off + (int64_t)j * 32 + lane;
        const bool real = j < len;
        scol[d] = real ? col[e0 + j] : 0;
        if (sval) sval[d] = real ? val[e0 + j] : 0.0;
        if (sval32) sval32[d] = real ? val32[e0 + j] : 0.f;
    }
}

// Rows with <= kSellMaxLen entries go to the SELL-32 part (sorted by length,
// descending, then by row); longer rows are grouped by bin (ascending row
// order inside a bin).  Uploads both layouts.
static int build_bins(DevCSR *A, const std::vector<int64_t> &rp, cudaStream_t s)
{
    const int64_t m = A->m;
    // SELL part: counting sort by length, descending
    std::vector<int64_t> lcnt(kSellMaxLen + 2, 0);
    for (int64_t r = 0; r < m; r++) {
        const int64_t L = rp[r + 1] - rp[r];
        if (L <= kSellMaxLen) lcnt[L]++;
    }
    std::vector<int64_t> lpos(kSellMaxLen + 2, 0);
    int64_t acc = 0;
    for (int L = kSellMaxLen; L >= 0; L--) { lpos[L] = acc; acc += lcnt[L]; }
    const int64_t sr = acc;
    std::vector<int32_t> sperm((size_t)std::max<int64_t>(sr, 1));
    for (int64_t r = 0; r < m; r++) {
        const int64_t L = rp[r + 1] - rp[r];
        if (L <= kSellMaxLen) sperm[lpos[L]++] = (int32_t)r;
    }
    const int64_t slices = (sr + 31) / 32;
    std::vector<int64_t> soff((size_t)slices + 1, 0);
    for (int64_t sl = 0; sl < slices; sl++) {
        const int32_t r = sperm[sl * 32];  // the longest row of the slice comes first
        soff[sl + 1] = soff[sl] + 32 * (rp[r + 1] - rp[r]);
    }
    A->sell_rows = sr;
    A->sell_slices = slices;
    const int64_t padded = soff[(size_t)slices];
    if (cudaMalloc(&A->sell_perm, sizeof(int32_t) * (size_t)std::max<int64_t>(sr, 1)) != cudaSuccess ||
        cudaMalloc(&A->sell_off, sizeof(int64_t) * (size_t)(slices + 1)) != cudaSuccess ||
        cudaMalloc(&A->sell_col, sizeof(int32_t) * (size_t)std::max<int64_t>(padded, 1)) != cudaSuccess)
        return SVDSC_ERR_NOMEM;
    if (A->val && cudaMalloc(&A->sell_val, sizeof(double) * (size_t)std::max<int64_t>(padded, 1)) != cudaSuccess)
        return SVDSC_ERR_NOMEM;
    if (A->val32 && cudaMalloc(&A->sell_val32, sizeof(float) * (size_t)std::max<int64_t>(padded, 1)) != cudaSuccess)
        return SVDSC_ERR_NOMEM;
    if (sr > 0 && cudaMemcpyAsync(A->sell_perm, sperm.data(), sizeof(int32_t) * (size_t)sr, cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
        return SVDSC_ERR_CUDA;
    if (cudaMemcpyAsync(A->sell_off, soff.data(), sizeof(int64_t) * (size_t)(slices + 1), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return SVDSC_ERR_CUDA;
    if (slices > 0)
        sell_fill_kernel<<<(unsigned)((slices * 32 + 255) / 256), 256, 0, s>>>(
            A->row_ptr, A->col, A->val, A->val32, A->sell_perm, A->sell_off, sr, slices, A->sell_col, A->sell_val,
            A->sell_val32);
    if (cudaGetLastError() != cudaSuccess) return SVDSC_ERR_CUDA;

    // binned part (rows longer than kSellMaxLen)
    std::vector<int64_t> cnt(kNumBins, 0);
    int64_t nlong = 0;
    for (int64_t r = 0; r < m; r++) {
        const int64_t L = rp[r + 1] - rp[r];
        if (L > kSellMaxLen) { cnt[bin_of(L)]++; nlong++; }
    }
    Bins b;
    b.row_start[0] = 0;
    for (int i = 0; i < kNumBins; i++) b.row_start[i + 1] = b.row_start[i] + cnt[i];
    b.block_start[0] = 0;
    for (int i = 0; i < kNumBins; i++) {
        const int64_t rows_per_block = kSpmvThreads / bin_lanes(i);
        b.block_start[i + 1] = b.block_start[i] + (cnt[i] + rows_per_block - 1) / rows_per_block;
    }
    if (b.block_start[kNumBins] + (sr + kSpmvThreads - 1) / kSpmvThreads > 0x7fffffff) return SVDSC_ERR_SIZE;
    std::vector<int32_t> perm((size_t)std::max<int64_t>(nlong, 1));
    std::vector<int64_t> pos(b.row_start, b.row_start + kNumBins);
    for (int64_t r = 0; r < m; r++) {
        const int64_t L = rp[r + 1] - rp[r];
        if (L > kSellMaxLen) perm[pos[bin_of(L)]++] = (int32_t)r;
    }
    A->bins = b;
    if (cudaMalloc(&A->perm, sizeof(int32_t) * (size_t)std::max<int64_t>(nlong, 1)) != cudaSuccess)
        return SVDSC_ERR_NOMEM;
    if (nlong > 0 && cudaMemcpyAsync(A->perm, perm.data(), sizeof(int32_t) * (size_t)nlong, cudaMemcpyHostToDevice,
                                     s) != cudaSuccess)
        return SVDSC_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SVDSC_ERR_CUDA;
    return SVDSC_OK;
}

void csr_free(DevCSR *A)
{
    cudaFree(A->sell_perm);
    cudaFree(A->sell_off);
    cudaFree(A->sell_col);
    cudaFree(A->sell_val);
    cudaFree(A->sell_val32);
    cudaFree(A->row_ptr);
    cudaFree(A->col);
    cudaFree(A->val);
    cudaFree(A->val32);
    cudaFree(A->perm);
    *A = DevCSR();
}

template <typename T>
static cudaError_t dev_copy_in(T **dst, const T *src, int64_t count, bool on_device, cudaStream_t s)
{
    cudaError_t e = cudaMalloc(dst, sizeof(T) * (size_t)std::max<int64_t>(count, 1));
    if (e != cudaSuccess) return e;
    if (count == 0) return cudaSuccess;
    return cudaMemcpyAsync(*dst, src, sizeof(T) * (size_t)count,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
}

int csr_prepare(const svdsc_matrix *in, bool want_f32, bool want_f64, DevCSR *A, DevCSR *AT,
                cudaStream_t s)
{
    int rc = SVDSC_OK;
    const int64_t m = in->m, n = in->n;
    const int base = in->index_base;
    const bool dev = in->on_device != 0;
    const bool four = (in->row_ptr == nullptr);
    int64_t *rb = nullptr, *re = nullptr, *len = nullptr, *tmp = nullptr, *keys = nullptr;
    int32_t *col_in = nullptr, *segs = nullptr;
    void *val_in = nullptr;
    int *bad = nullptr;
    unsigned long long *cnt = nullptr;
    int64_t extent = 0;
    std::vector<int64_t> hrp, hrpT;
    int hbad = 0;
    const size_t vsz = (in->value_type == SVDSC_F32) ? 4 : 8;
    *A = DevCSR();
    *AT = DevCSR();
    A->m = m; A->n = n;
    AT->m = n; AT->n = m;

    // 1. row begin/end on the device, and the extent of col_idx/values
    if (!four) {
        int64_t first = 0, last = 0;
        if (dev) {
            PREP_TRY(cudaMemcpyAsync(&first, in->row_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            PREP_TRY(cudaMemcpyAsync(&last, in->row_ptr + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            PREP_TRY(cudaStreamSynchronize(s));
        } else {
            first = in->row_ptr[0];
            last = in->row_ptr[m];
        }
        if (first != base || last < first) { rc = SVDSC_ERR_CSR; goto done; }
        extent = last - base;
        PREP_TRY(dev_copy_in(&rb, in->row_ptr, m + 1, dev, s));
        re = rb + 1;
    } else {
        if (!in->row_end || in->nnz < 0) { rc = SVDSC_ERR_ARG; goto done; }
        extent = in->nnz;
        PREP_TRY(dev_copy_in(&rb, in->row_begin, m, dev, s));
        PREP_TRY(dev_copy_in(&re, in->row_end, m, dev, s));
    }
    PREP_TRY(dev_copy_in(&col_in, in->col_idx, extent, dev, s));
    if (vsz == 8) PREP_TRY(dev_copy_in((double **)&val_in, (const double *)in->values, extent, dev, s));
    else PREP_TRY(dev_copy_in((float **)&val_in, (const float *)in->values, extent, dev, s));
    PREP_TRY(cudaMalloc(&bad, sizeof(int)));
    PREP_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
    PREP_TRY(cudaMalloc(&len, sizeof(int64_t) * (size_t)std::max<int64_t>(std::max(m, n), 1)));
    PREP_TRY(cudaMalloc(&tmp, sizeof(int64_t) * (size_t)((std::max(m, n) + 1023) / 1024 + 2)));

    // 2. validate and compute row lengths
    if (m > 0)
        csr_validate<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(rb, four ? re : rb + 1, m, n, extent,
                                                                 base, col_in, bad, len);
    PREP_TRY(cudaGetLastError());
    PREP_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    PREP_TRY(cudaStreamSynchronize(s));
    if (hbad) { rc = SVDSC_ERR_CSR; goto done; }

    // 3. compact to 0-based 3-array CSR in the working precision(s)
    PREP_TRY(cudaMalloc(&A->row_ptr, sizeof(int64_t) * (size_t)(m + 1)));
    PREP_TRY(exclusive_scan(len, m, A->row_ptr, tmp, s));
    hrp.resize((size_t)m + 1);
    PREP_TRY(cudaMemcpyAsync(hrp.data(), A->row_ptr, sizeof(int64_t) * (size_t)(m + 1),
                             cudaMemcpyDeviceToHost, s));
    PREP_TRY(cudaStreamSynchronize(s));
    A->nnz = hrp[(size_t)m];
    AT->nnz = A->nnz;
    if (A->nnz > 0x7fffffffLL * 16) { rc = SVDSC_ERR_SIZE; goto done; }
    PREP_TRY(cudaMalloc(&A->col, sizeof(int32_t) * (size_t)std::max<int64_t>(A->nnz, 1)));
    if (want_f64) PREP_TRY(cudaMalloc(&A->val, sizeof(double) * (size_t)std::max<int64_t>(A->nnz, 1)));
    if (want_f32) PREP_TRY(cudaMalloc(&A->val32, sizeof(float) * (size_t)std::max<int64_t>(A->nnz, 1)));
    if (m > 0) {
        const unsigned g = (unsigned)((m * 32 + 255) / 256);
        if (vsz == 8)
            csr_compact<double><<<g, 256, 0, s>>>(rb, m, base, col_in, (const double *)val_in,
                                                  A->row_ptr, A->col, A->val, A->val32, bad);
        else
            csr_compact<float><<<g, 256, 0, s>>>(rb, m, base, col_in, (const float *)val_in,
                                                 A->row_ptr, A->col, A->val, A->val32, bad);
        PREP_TRY(cudaGetLastError());
    }
    PREP_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    PREP_TRY(cudaStreamSynchronize(s));
    if (hbad & 4) { rc = SVDSC_ERR_NONFINITE; goto done; }
    cudaFree(rb); rb = nullptr;
    if (four) { cudaFree(re); }
    re = nullptr;
    cudaFree(col_in); col_in = nullptr;
    cudaFree(val_in); val_in = nullptr;

    // 4. CSR(A^T): count per column, scan, scatter nnz positions, sort each
    //    row of A^T by position (= by row of A), then gather
    PREP_TRY(cudaMalloc(&cnt, sizeof(unsigned long long) * (size_t)std::max<int64_t>(n, 1)));
    PREP_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * (size_t)std::max<int64_t>(n, 1), s));
    if (A->nnz > 0) col_count<<<4 * 152, 256, 0, s>>>(A->col, A->nnz, cnt);
    PREP_TRY(cudaGetLastError());
    PREP_TRY(cudaMalloc(&AT->row_ptr, sizeof(int64_t) * (size_t)(n + 1)));
    PREP_TRY(exclusive_scan((const int64_t *)cnt, n, AT->row_ptr, tmp, s));
    PREP_TRY(cudaMemcpyAsync(cnt, AT->row_ptr, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    PREP_TRY(cudaMalloc(&keys, sizeof(int64_t) * (size_t)std::max<int64_t>(A->nnz, 1)));
    if (A->nnz > 0) col_scatter<<<4 * 152, 256, 0, s>>>(A->col, A->nnz, cnt, keys);
    PREP_TRY(cudaGetLastError());
    hrpT.resize((size_t)n + 1);
    PREP_TRY(cudaMemcpyAsync(hrpT.data(), AT->row_ptr, sizeof(int64_t) * (size_t)(n + 1),
                             cudaMemcpyDeviceToHost, s));
    PREP_TRY(cudaStreamSynchronize(s));
    {
        std::vector<int32_t> shortv, longv;
        for (int64_t c = 0; c < n; c++) {
            const int64_t L = hrpT[(size_t)c + 1] - hrpT[(size_t)c];
            if (L <= 1) continue;
            if (L <= 32) shortv.push_back((int32_t)c); else longv.push_back((int32_t)c);
        }
        const size_t ns = shortv.size(), nl = longv.size();
        PREP_TRY(cudaMalloc(&segs, sizeof(int32_t) * std::max<size_t>(ns + nl, 1)));
        if (ns) PREP_TRY(cudaMemcpyAsync(segs, shortv.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, s));
        if (nl) PREP_TRY(cudaMemcpyAsync(segs + ns, longv.data(), sizeof(int32_t) * nl, cudaMemcpyHostToDevice, s));
        if (ns) seg_sort_short<<<(unsigned)((ns + 255) / 256), 256, 0, s>>>(AT->row_ptr, segs, (int64_t)ns, keys);
        if (nl) seg_sort_block<<<(unsigned)nl, 512, 0, s>>>(AT->row_ptr, segs + ns, keys);
        PREP_TRY(cudaGetLastError());
        PREP_TRY(cudaStreamSynchronize(s));  // host vectors above must outlive the copies
    }
    PREP_TRY(cudaMalloc(&AT->col, sizeof(int32_t) * (size_t)std::max<int64_t>(A->nnz, 1)));
    if (want_f64) PREP_TRY(cudaMalloc(&AT->val, sizeof(double) * (size_t)std::max<int64_t>(A->nnz, 1)));
    if (want_f32) PREP_TRY(cudaMalloc(&AT->val32, sizeof(float) * (size_t)std::max<int64_t>(A->nnz, 1)));
    if (A->nnz > 0)
        transpose_fill<<<8 * 152, 256, 0, s>>>(keys, A->nnz, A->row_ptr, m, A->val, A->val32,
                                               AT->col, AT->val, AT->val32);
    PREP_TRY(cudaGetLastError());

    // 5. bins of both
    rc = build_bins(A, hrp, s);
    if (rc != SVDSC_OK) goto done;
    rc = build_bins(AT, hrpT, s);
    if (rc != SVDSC_OK) goto done;
    PREP_TRY(cudaStreamSynchronize(s));

done:
    if (rb) cudaFree(rb);
    if (four && re) cudaFree(re);
    cudaFree(col_in);
    cudaFree(val_in);
    cudaFree(len);
    cudaFree(tmp);
    cudaFree(keys);
    cudaFree(segs);
    cudaFree(bad);
    cudaFree(cnt);
    if (rc != SVDSC_OK) {
        cudaStreamSynchronize(s);
        csr_free(A);
        csr_free(AT);
    }
    return rc;
}

}  // namespace svdsc
