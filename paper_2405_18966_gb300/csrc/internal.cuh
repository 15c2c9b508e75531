// Internal declarations shared by the svdsc CUDA translation units.
#pragma once
#include <atomic>
#include <cuda_runtime.h>
#include <stdint.h>
#include "../../include/svdsc.h"

namespace svdsc {

// Counter-based N(0,1) of the method's random vectors: SplitMix64 (Steele,
// Lea & Flood 2014) as the mixing function and the Box-Muller transform
// (1958).  Element j of draw d under seed: key = mix(seed); c = 2 (d 2^32 + j);
// U1, U2 from the top 53 bits of mix(key + c), mix(key + c + 1), offset by one
// half; z = sqrt(-2 ln U1) cos(2 pi U2).
__device__ __forceinline__ uint64_t splitmix_mix(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double normal_draw(uint64_t key, uint64_t draw, uint64_t j)
{
    const uint64_t c = 2ull * ((draw << 32) + j);
    const double u1 = ((double)(splitmix_mix(key + c) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    const double u2 = ((double)(splitmix_mix(key + c + 1ull) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

// Device-side status block of one context (device memory, read by the host at
// restart boundaries only).
struct DevStatus {
    int poison;        // a finalize met a breakdown or a non-finite norm: later kernels skip
    int bd_step;       // step id of the first such vector (INT32_MAX: none)
    int nonfinite;     // the bad norm was NaN/Inf
    int timeout;       // a bounded grid barrier ran out
    int converged;     // residual test: every res_j < tol
    int nconv;         // residual test: count of res_j < tol
    int svd_sweeps;    // sweeps of the last projected SVD (-1: sweep cap hit)
    int pad;
    double anorm[2];   // running max of alpha/beta/sigma, double-buffered by step parity
    double beta_t;     // T(t, t+1) at the last residual test
    double last_norm;  // norm of the last finalized vector
};

// Partial re-orthogonalization state (device memory).
struct PrState {
    double bytes_t, bytes_n, flops;  // algorithmic bytes / flops of the CGS2 passes that ran
    int gate;      // 1: the CGS2 kernels of the current vector skip their work
    int force_u;   // the next u vector is re-orthogonalized regardless of its estimates
    int force_v;   // likewise for the next v vector
    int n_reorth;  // vectors the estimates sent to CGS2 in this solve
};

// Raises a kernel's dynamic shared-memory limit once per device (function
// attributes belong to the device's context, so a process-wide flag would
// skip the second GPU); thread-safe.
inline cudaError_t set_smem_limit_once(const void *fn, int bytes, std::atomic<unsigned long long> *done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
    if (bit && (done->load() & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done->fetch_or(bit);
    return e;
}

// Row chunking of one vector length for the row-blocked kernels.
struct Chunk {
    int64_t len = 0;
    int64_t R = 0;   // rows per CTA (multiple of 64)
    int nb = 0;      // number of CTAs
    // layout of the FP64 GEMV-N (w -= W h), which also fixes the partial sums
    // of ||w||^2: nbu CTAs of thu threads, Ru rows each.  Every producer
    // (GEMV-N, norm_partial) and consumer (finalize, the estimate gate) of
    // those partials uses nbu, so the norm is summed in one fixed order.
    int64_t Ru = 0;
    int nbu = 0;
    int thu = 0;
};
Chunk make_chunk(int64_t len, int target_blocks);

// Row-length bins of a CSR matrix for the binned SpMV kernel.
constexpr int kNumBins = 10;  // lanes per row: 1 (four length classes), 2, 4, 8, 16, 32, a whole CTA
struct Bins {
    int64_t row_start[kNumBins + 1] = {0};    // offsets into perm
    int64_t block_start[kNumBins + 1] = {0};  // CTA offsets of each bin in the single launch
};

struct DevCSR {
    int64_t m = 0, n = 0, nnz = 0;
    int64_t *row_ptr = nullptr;  // m+1, 0-based
    int32_t *col = nullptr;      // nnz
    double *val = nullptr;       // nnz (FP64 contexts)
    float *val32 = nullptr;      // nnz (MIXED contexts)
    // SELL-32 part (Kreutzer et al., SELL-C-sigma with C = 32 and full sorting):
    // rows with at most kSellMaxLen entries, sorted by length (descending),
    // cut into slices of 32 rows, each slice padded to its longest row and
    // stored column-major, so one thread per row loads coalesced values.
    int64_t sell_rows = 0;
    int64_t sell_slices = 0;
    int32_t *sell_perm = nullptr;    // original row of each SELL row
    int64_t *sell_off = nullptr;     // element offset of each slice (sell_slices + 1)
    int32_t *sell_col = nullptr;
    double *sell_val = nullptr;
    float *sell_val32 = nullptr;
    // longer rows: grouped by row-length bin (warp / CTA per row)
    int32_t *perm = nullptr;     // rows grouped by bin, ascending inside a bin
    Bins bins;
};
constexpr int kSellMaxLen = 128;

struct DevDense {
    int64_t m = 0, n = 0, ld = 0;
    double *a = nullptr;
};

constexpr int kSpmvThreads = 256;
constexpr int kRowThreads = 512;
constexpr int kUpdSmallThreads = 256;               // FP64 GEMV-N small-CTA layout
constexpr int64_t kUpdSmallMinRows = 1336 * 512;    // rows from which it is used

// ---- products (spmv.cu)
// y = A x - coef * z (z may be null; coef from *coef_dev when non-null, else coef_h)
cudaError_t csr_spmv_f64(const DevCSR &A, const double *x, const double *z, const double *coef_dev,
                         double coef_h, double *y, const int *poison, cudaStream_t s);
cudaError_t csr_spmv_f32(const DevCSR &A, const float *x, const double *z, const double *coef_dev,
                         double coef_h, double *y, const int *poison, cudaStream_t s);
cudaError_t dense_gemv_n(const DevDense &A, const double *x, const double *z, const double *coef_dev,
                         double coef_h, double *y, double *partial, const int *poison,
                         cudaStream_t s, int *launches);
cudaError_t dense_gemv_t(const DevDense &A, const double *x, const double *z, const double *coef_dev,
                         double coef_h, double *y, double *partial, const int *poison,
                         cudaStream_t s, int *launches);
size_t dense_partial_doubles(const DevDense &A);
// create-time preparation
int csr_prepare(const svdsc_matrix *in, bool want_f32, bool want_f64, DevCSR *A, DevCSR *AT,
                cudaStream_t s);
void csr_free(DevCSR *A);

// ---- re-orthogonalization (reorth.cu)
void proj_partial(const double *W, int64_t ld, int ncols, const double *w, const Chunk &c,
                  double *P, const int *poison, cudaStream_t s);
void proj_partial_f32(const float *W32, int64_t ld, int ncols, const double *w, const Chunk &c,
                      double *P, const int *poison, cudaStream_t s);
void proj_reduce(const double *P, int nb, int ncols, double *h, const int *poison, cudaStream_t s);
void update_sub(const double *W, int64_t ld, int ncols, const double *h, double *w, const Chunk &c,
                double *Pn, const int *poison, cudaStream_t s);
void update_sub_f32(const float *W32, int64_t ld, int ncols, const double *h, double *w,
                    const Chunk &c, const int *poison, cudaStream_t s);
void norm_partial(const double *w, const Chunk &c, double *Pn, const int *poison, cudaStream_t s);
// *out = ||w||_2 from the partial sums norm_partial / the last GEMV-N pass left (nb = Chunk::nbu)
void norm_from_partials(const double *Pn, int nb, double *out, cudaStream_t s);
// mode: 0 = Lanczos vector (T entry := norm, breakdown check), 1 = plain normalise
// (no T entry), 2 = repair of a breakdown (T entry := 0, needs norm > 1e-8)
void finalize(double *w, const Chunk &c, const double *Pn, double *T_entry, DevStatus *st,
              int step, int parity, int mode, float *w32, cudaStream_t s);
void rng_normal_vec(uint64_t seed, uint64_t draw, int64_t len, double *x, cudaStream_t s);
// partial re-orthogonalization (side 1: v vector, 0: u vector; i, kk 1-based step / restart size)
// (bt, bn, fl: algorithmic GEMV-T / GEMV-N bytes and flops of the CGS2 if it runs)
void pr_omega(int side, int i, int kk, const double *T, int ldt, double *mu, double *nu, const Chunk &c,
              const double *Pn, const DevStatus *st, int parity, PrState *pr, double bt, double bn,
              double fl, cudaStream_t s);
void pr_restart(int t, int k, const double *Vh, double *mu, double *nu, PrState *pr, cudaStream_t s);
void pr_reset(int side, int col, double *mu, double *nu, PrState *pr, cudaStream_t s);
void copy_f64_to_f32(const double *x, float *y, int64_t len, cudaStream_t s);

// ---- projected SVD (small_svd.cu)
struct SvdWork {
    double *B = nullptr;       // t x t
    double *W = nullptr;       // t x t (right rotations)
    double *sig = nullptr;     // t
    int *rot = nullptr;        // per-sweep rotation counters
    unsigned *bar = nullptr;   // grid barrier: [count, generation]
    int max_sweeps = 60;
    int coop_blocks = 0;       // co-resident CTAs available for the multi-CTA kernel
};
cudaError_t small_svd(int t, const double *T, int64_t ldt, double *S, double *Uh, double *Vh,
                      SvdWork &w, DevStatus *st, cudaStream_t s, int *launches);
int small_svd_coop_capacity();
// self-tests of the bounded waits (each wait is made to run out on purpose)
cudaError_t probe_grid_barrier(unsigned *bar, DevStatus *st, cudaStream_t s);
cudaError_t probe_mbarrier(int *err, cudaStream_t s);

// ---- tensor-core restart GEMM (gemm_tc.cu)
size_t tc_gemm_ws_bytes(int t, int k);
cudaError_t tc_gemm(int mode, const double *W, const float *W32, int64_t ldw, int64_t rows, int t,
                    const double *Q, int64_t ldq, int k, double *C, int64_t ldc, float *C32, void *ws,
                    int *err, cudaStream_t s, int *launches);

}  // namespace svdsc
