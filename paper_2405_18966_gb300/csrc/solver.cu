// Host driver and C-ABI of the svdsc library: Alg. 2 of the svds-C paper
// (augmented-restart truncated SVD) with every numerical step on the device.
// The host issues kernels and reads a small status block once per restart
// round (convergence flag, breakdown marker); nothing else crosses to the host
// until the outputs are copied.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>
#include <nvtx3/nvToolsExt.h>
#include "context.cuh"

// ----------------------------------------------------------- small kernels

// Eq. (4) residuals res_j = |beta_t Uh(t,j)| / max(sigma_j, eps sigma_1), the
// restart coefficients rho_j = beta_t Uh(t,j) of Eq. (6), the convergence test
// of Alg. 2 and the ||A|| estimate.
__global__ void residual_kernel(int t, int k, double tol, const double *__restrict__ T,
                                const double *__restrict__ Sh, const double *__restrict__ Uh,
                                double *__restrict__ res, double *__restrict__ rho, DevStatus *st,
                                int parity, int imax)
{
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const double beta_t = T[(t - 1) + (int64_t)t * (t + 1)];
    const double s0 = Sh[imax];  // the largest Ritz value
    int local = 0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const double den = Sh[j] > DBL_EPSILON * s0 ? Sh[j] : DBL_EPSILON * s0;
        const double u = Uh[(t - 1) + (int64_t)j * t];
        const double r = den > 0.0 ? fabs(beta_t * u) / den : 0.0;
        res[j] = r;
        rho[j] = beta_t * u;
        local += (r < tol);
    }
    atomicAdd(&cnt, local);
    __syncthreads();
    if (threadIdx.x == 0) {
        st->nconv = cnt;
        st->converged = (cnt == k);
        st->beta_t = beta_t;
        if (s0 > st->anorm[parity]) st->anorm[parity] = s0;
    }
}

// Reverses the order of the t Ritz triplets (S ascending) so that the k
// smallest are the first k columns the residual test, restart and outputs use.
__global__ void reverse_triplets_kernel(int t, double *__restrict__ Sh, double *__restrict__ Uh,
                                        double *__restrict__ Vh)
{
    const int half = t / 2;
    const int64_t total = (int64_t)half * t;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(i / t), r = (int)(i % t);
        const int64_t a = r + (int64_t)j * t, b = r + (int64_t)(t - 1 - j) * t;
        double x = Uh[a]; Uh[a] = Uh[b]; Uh[b] = x;
        x = Vh[a]; Vh[a] = Vh[b]; Vh[b] = x;
    }
    if (blockIdx.x == 0)
        for (int j = threadIdx.x; j < half; j += blockDim.x) {
            const double x = Sh[j];
            Sh[j] = Sh[t - 1 - j];
            Sh[t - 1 - j] = x;
        }
}

// T <- 0; T(j,j) = sigma_j, T(j,k+1) = rho_j for j <= k  (the augmented restart of Alg. 2, Eq. 6)
__global__ void restart_T_kernel(int t, int k, double *__restrict__ T, const double *__restrict__ Sh,
                                 const double *__restrict__ rho)
{
    const int64_t ld = t + 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ld * ld;
         i += (int64_t)gridDim.x * blockDim.x)
        T[i] = 0.0;
    __syncthreads();
    if (blockIdx.x == 0)
        for (int j = threadIdx.x; j < k; j += blockDim.x) {
            T[j + j * ld] = Sh[j];
            T[j + (int64_t)k * ld] = rho[j];
        }
}

// In-place restart update W(:, 0:k) <- W(:, 0:t) Q(:, 0:k) of Alg. 2 (restart
// and final output, FP64 FMA).  A CTA owns a block of 32 rows and all k outputs of
// them, so it reads its rows completely before overwriting them.  Q is held in
// shared memory in chunks of KC rows.
constexpr int kGemmGroups = 8;   // warps per CTA; each covers 32 rows x (k / 8) columns
constexpr int kGemmMaxQ = 32;    // accumulators per thread => k <= 256

__global__ void __launch_bounds__(kGemmGroups * 32)
gemm_inplace_kernel(double *__restrict__ W, int64_t ld, int64_t rows, int t,
                    const double *__restrict__ Q, int64_t ldq, int k, int KC)
{
    extern __shared__ double Qs[];  // KC x k, ld KC
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const int nq = (k + kGemmGroups - 1) / kGemmGroups;
    for (int64_t rb = (int64_t)blockIdx.x * 32; rb < rows; rb += (int64_t)gridDim.x * 32) {
        double acc[kGemmMaxQ];
#pragma unroll
        for (int q = 0; q < kGemmMaxQ; q++) acc[q] = 0.0;
        const int64_t r = rb + lane;
        for (int c0 = 0; c0 < t; c0 += KC) {
            const int kc = min(KC, t - c0);
            __syncthreads();
            for (int i = threadIdx.x; i < kc * k; i += blockDim.x) {
                const int cc = i % kc, j = i / kc;
                Qs[cc + j * KC] = Q[(c0 + cc) + (int64_t)j * ldq];
            }
            __syncthreads();
            for (int cc = 0; cc < kc; cc++) {
                const double a = (r < rows) ? W[r + (int64_t)(c0 + cc) * ld] : 0.0;
#pragma unroll
                for (int q = 0; q < kGemmMaxQ; q++) {
                    if (q < nq) {
                        const int j = grp + kGemmGroups * q;
                        if (j < k) acc[q] = fma(a, Qs[cc + j * KC], acc[q]);
                    }
                }
            }
        }
        __syncthreads();  // every read of this row block precedes the writes
        if (r < rows) {
#pragma unroll
            for (int q = 0; q < kGemmMaxQ; q++) {
                const int j = grp + kGemmGroups * q;
                if (q < nq && j < k) W[r + (int64_t)j * ld] = acc[q];
            }
        }
    }
}

static int gemm_inplace(svdsc_ctx *c, double *W, int64_t ld, int64_t rows, int t, const double *Q,
                        int k)
{
    if (k > kGemmGroups * kGemmMaxQ) return SVDSC_ERR_SIZE;
    int KC = t;
    const int max_doubles = (200 * 1024) / 8;
    if ((int64_t)KC * k > max_doubles) KC = std::max(1, max_doubles / k);
    const size_t smem = sizeof(double) * (size_t)KC * k;
    static std::atomic<unsigned long long> attr_done{0};
    if (smem > 48 * 1024) CU(set_smem_limit_once((const void *)gemm_inplace_kernel, 200 * 1024, &attr_done));
    const int64_t blocks = std::min<int64_t>((rows + 31) / 32, 152 * (smem > 100 * 1024 ? 1 : 2));
    const int e0 = ph_begin(c);
    gemm_inplace_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), kGemmGroups * 32, smem, c->stream>>>(
        W, ld, rows, t, Q, t, k, KC);
    ph_end(c, SVDSC_PH_GEMM, e0, 1, 8.0 * rows * (t + k), 2.0 * rows * t * k);
    CU(cudaGetLastError());
    return SVDSC_OK;
}

// Out-of-place tensor-core update C = W Q (svdsc_gemm modes): FP64 digits, or
// three BF16 pieces of the FP32 shadow in the mixed form (C32 gets the shadow).
int gemm_tc(svdsc_ctx *c, const double *W, const float *W32, int64_t ld, int64_t rows, int t,
            const double *Q, int k, double *C, float *C32)
{
    const int mode = (c->precision == SVDSC_MIXED) ? 1 : 0;
    const int e0 = ph_begin(c);
    int nl = 0;
    cudaError_t e = tc_gemm(mode, W, W32, ld, rows, t, Q, t, k, C, ld, C32, c->gemm_ws, &c->st->timeout,
                            c->stream, &nl);
    const double wb = (W32 ? 4.0 : 8.0) * rows * t;
    const double prods = mode == 0 ? 36.0 : 6.0;  // BF16 products per multiply-add
    ph_end(c, SVDSC_PH_GEMM, e0, nl, wb + 8.0 * rows * k + (C32 ? 4.0 * rows * k : 0.0),
           2.0 * rows * (double)t * k * prods);
    return e == cudaSuccess ? SVDSC_OK : SVDSC_ERR_CUDA;
}

// Sign rule for returned pairs: the entry of v_j with the largest magnitude
// (lowest index on ties) is made positive, flipping u_j with it.
__global__ void __launch_bounds__(256)
sign_kernel(double *__restrict__ U, int64_t ldu, int64_t m, double *__restrict__ V, int64_t ldv,
            int64_t n)
{
    const int j = blockIdx.x;
    double *v = V + (int64_t)j * ldv;
    double best = -1.0;
    int64_t bi = 0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
        const double a = fabs(v[r]);
        if (a > best) { best = a; bi = r; }  // ascending r: first max kept
    }
    __shared__ double sb[256];
    __shared__ int64_t si[256];
    sb[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const double b2 = sb[threadIdx.x + o];
            const int64_t i2 = si[threadIdx.x + o];
            if (b2 > sb[threadIdx.x] || (b2 == sb[threadIdx.x] && i2 < si[threadIdx.x])) {
                sb[threadIdx.x] = b2;
                si[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    const bool flip = v[si[0]] < 0.0;
    __syncthreads();
    if (!flip) return;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) v[r] = -v[r];
    double *u = U + (int64_t)j * ldu;
    for (int64_t r = threadIdx.x; r < m; r += blockDim.x) u[r] = -u[r];
}

__global__ void check_finite_kernel(const double *__restrict__ a, int64_t ld, int64_t m, int64_t n,
                                    int *bad)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m * n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i % m, c = i / m;
        if (!isfinite(a[r + c * ld])) { atomicOr(bad, 1); return; }
    }
}

// ----------------------------------------------------------- host helpers

static void free_workspace(svdsc_ctx *c)
{
    cudaFree(c->U); cudaFree(c->V); cudaFree(c->T);
    cudaFree(c->U32); cudaFree(c->V32);
    cudaFree(c->Ua); cudaFree(c->Va); cudaFree(c->U32a); cudaFree(c->V32a); cudaFree(c->gemm_ws);
    c->Ua = c->Va = nullptr;
    c->U32a = c->V32a = nullptr;
    c->gemm_ws = nullptr;
    cudaFree(c->P); cudaFree(c->h); cudaFree(c->Pn);
    cudaFree(c->Sh); cudaFree(c->Uh); cudaFree(c->Vh); cudaFree(c->res); cudaFree(c->rho);
    cudaFree(c->svd.B); cudaFree(c->svd.W); cudaFree(c->svd.sig); cudaFree(c->svd.rot);
    cudaFree(c->svd.bar);
    cudaFree(c->mu); cudaFree(c->nu); cudaFree(c->pr);
    c->mu = c->nu = nullptr;
    c->pr = nullptr;
    c->U = c->V = c->T = c->P = c->h = c->Pn = c->Sh = c->Uh = c->Vh = c->res = c->rho = nullptr;
    c->U32 = c->V32 = nullptr;
    c->svd.B = c->svd.W = c->svd.sig = nullptr;
    c->svd.rot = nullptr;
    c->svd.bar = nullptr;
    c->t_cap = 0;
    block_free(c);
}

int reserve_ws(svdsc_ctx *c, int t)
{
    if (t <= c->t_cap) return SVDSC_OK;
    cudaStreamSynchronize(c->stream);
    free_workspace(c);
    const int64_t cols = t + 2;
    const int nbmax = std::max(c->cm.nb, c->cn.nb);
    bool ok = true;
    auto alloc = [&](void **p, size_t bytes) {
        if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) ok = false;
    };
    alloc((void **)&c->U, sizeof(double) * c->ldu * cols);
    alloc((void **)&c->V, sizeof(double) * c->ldv * cols);
    alloc((void **)&c->Ua, sizeof(double) * c->ldu * cols);
    alloc((void **)&c->Va, sizeof(double) * c->ldv * cols);
    alloc(&c->gemm_ws, tc_gemm_ws_bytes(t, t));
    alloc((void **)&c->T, sizeof(double) * (size_t)(t + 2) * (t + 2));
    if (c->precision == SVDSC_MIXED) {
        alloc((void **)&c->U32, sizeof(float) * c->ldu * cols);
        alloc((void **)&c->V32, sizeof(float) * c->ldv * cols);
        alloc((void **)&c->U32a, sizeof(float) * c->ldu * cols);
        alloc((void **)&c->V32a, sizeof(float) * c->ldv * cols);
    }
    alloc((void **)&c->P, sizeof(double) * (size_t)nbmax * cols);
    alloc((void **)&c->h, sizeof(double) * cols);
    alloc((void **)&c->mu, sizeof(double) * cols);
    alloc((void **)&c->nu, sizeof(double) * cols);
    alloc((void **)&c->pr, sizeof(PrState));
    alloc((void **)&c->Pn, sizeof(double) * std::max({nbmax, c->cm.nbu, c->cn.nbu}));
    alloc((void **)&c->Sh, sizeof(double) * t);
    alloc((void **)&c->Uh, sizeof(double) * (size_t)t * t);
    alloc((void **)&c->Vh, sizeof(double) * (size_t)t * t);
    alloc((void **)&c->res, sizeof(double) * t);
    alloc((void **)&c->rho, sizeof(double) * t);
    alloc((void **)&c->svd.B, sizeof(double) * (size_t)t * t);
    alloc((void **)&c->svd.W, sizeof(double) * (size_t)t * t);
    alloc((void **)&c->svd.sig, sizeof(double) * t);
    alloc((void **)&c->svd.rot, sizeof(int) * c->svd.max_sweeps);
    alloc((void **)&c->svd.bar, sizeof(unsigned) * (2 + (size_t)t));  // grid barrier + Jacobi column flags
    if (!ok) {
        free_workspace(c);
        cudaGetLastError();
        return SVDSC_ERR_NOMEM;
    }
    // zero the bases once so that stale columns never hold NaN
    if (cudaMemsetAsync(c->U, 0, sizeof(double) * c->ldu * cols, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->V, 0, sizeof(double) * c->ldv * cols, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->Ua, 0, sizeof(double) * c->ldu * cols, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->Va, 0, sizeof(double) * c->ldv * cols, c->stream) != cudaSuccess)
        return SVDSC_ERR_CUDA;
    c->t_cap = t;
    return SVDSC_OK;
}

// y = A x - coef z   (trans: A^T).  x32 is the FP32 copy of x in MIXED contexts.
static int apply_A(svdsc_ctx *c, int trans, const double *x, const float *x32, const double *z,
                   const double *coef_dev, double coef_h, double *y, const int *poison)
{
    cudaError_t e;
    const int e0 = ph_begin(c);
    int nl = 1;
    double bytes, flops;
    if (c->format == SVDSC_CSR) {
        const DevCSR &M = trans ? c->AT : c->A;
        const bool f32 = c->precision == SVDSC_MIXED;
        if (f32) e = csr_spmv_f32(M, x32, z, coef_dev, coef_h, y, poison, c->stream);
        else e = csr_spmv_f64(M, x, z, coef_dev, coef_h, y, poison, c->stream);
        bytes = (f32 ? 8.0 : 12.0) * M.nnz + 20.0 * M.m + (f32 ? 4.0 : 8.0) * M.n + (z ? 8.0 * M.m : 0.0);
        flops = 2.0 * M.nnz;
    } else {
        nl = 0;
        if (trans) e = dense_gemv_t(c->D, x, z, coef_dev, coef_h, y, c->dense_part, poison, c->stream, &nl);
        else e = dense_gemv_n(c->D, x, z, coef_dev, coef_h, y, c->dense_part, poison, c->stream, &nl);
        const double out = trans ? c->D.n : c->D.m, in = trans ? c->D.m : c->D.n;
        bytes = 8.0 * c->D.m * c->D.n + 8.0 * in + 8.0 * out + (z ? 8.0 * out : 0.0);
        flops = 2.0 * c->D.m * c->D.n;
    }
    ph_end(c, SVDSC_PH_SPMV, e0, nl, bytes, flops);
    c->n_matvec++;
    return e == cudaSuccess ? SVDSC_OK : SVDSC_ERR_CUDA;
}

// One CGS pass: h = W^T w, then w -= W h (Pn: partial sums of the new ||w||^2).
static void cgs_pass(svdsc_ctx *c, const double *W, const float *W32, int64_t ld, int ncols, double *w,
                     const Chunk &ch, double *Pn, const int *poison, bool count = true)
{
    cudaStream_t s = c->stream;
    // gated passes (partial re-orthogonalization) count their bytes on the device
    const double L = count ? (double)ch.len : 0.0, nc = ncols;
    const double wsz = W32 ? 4.0 : 8.0;
    int e0 = ph_begin(c);
    if (W32) proj_partial_f32(W32, ld, ncols, w, ch, c->P, poison, s);
    else proj_partial(W, ld, ncols, w, ch, c->P, poison, s);
    ph_end(c, SVDSC_PH_GEMV_T, e0, 1, wsz * L * nc + 8.0 * L, 2.0 * L * nc);
    e0 = ph_begin(c);
    proj_reduce(c->P, ch.nb, ncols, c->h, poison, s);
    ph_end(c, SVDSC_PH_VEC, e0, 1, 8.0 * ch.nb * nc, ch.nb * nc);
    e0 = ph_begin(c);
    if (W32) update_sub_f32(W32, ld, ncols, c->h, w, ch, poison, s);
    else update_sub(W, ld, ncols, c->h, w, ch, Pn, poison, s);
    ph_end(c, SVDSC_PH_GEMV_N, e0, 1, wsz * L * nc + 16.0 * L, 2.0 * L * nc);
}

// CGS2: w <- (I - W W^T)^2 w against ncols columns; leaves the partial sums
// of ||w||^2 in c->Pn.  MIXED: first pass on the FP32 shadow W32.
static void cgs2(svdsc_ctx *c, const double *W, const float *W32, int64_t ld, int ncols, double *w,
                 const Chunk &ch, const int *poison, bool count = true)
{
    if (ncols > 0) {
        cgs_pass(c, W, W32, ld, ncols, w, ch, nullptr, poison, count);
        cgs_pass(c, W, nullptr, ld, ncols, w, ch, c->Pn, poison, count);
    } else {
        const int e0 = ph_begin(c);
        norm_partial(w, ch, c->Pn, poison, c->stream);
        ph_end(c, SVDSC_PH_VEC, e0, 1, 8.0 * ch.len, 2.0 * ch.len);
    }
}

// CGS2 in FP64 against ncols columns (partial sums of ||w||^2 left in c->Pn).
void cgs2_fp64(svdsc_ctx *c, const double *W, int64_t ld, int ncols, double *w, const Chunk &ch)
{
    cgs2(c, W, nullptr, ld, ncols, w, ch, nullptr);
}

static void do_finalize(svdsc_ctx *c, int side, int col, double *T_entry, int mode)
{
    const Chunk &ch = side == 0 ? c->cm : c->cn;
    double *w = side == 0 ? colU(c, col) : colV(c, col);
    float *w32 = side == 0 ? colU32(c, col) : colV32(c, col);
    const int step = (int)c->steps.size();
    c->steps.push_back({side, col, c->parity});
    const int e0 = ph_begin(c);
    finalize(w, ch, c->Pn, T_entry, c->st, step, c->parity, mode, w32, c->stream);
    ph_end(c, SVDSC_PH_VEC, e0, 1, (w32 ? 20.0 : 16.0) * ch.len, ch.len);
    c->parity ^= 1;
    c->n_steps++;
}

// Re-orthogonalization of a new Lanczos vector w against the first ncols
// columns of its basis: always (CGS2), or, in the partial mode, behind the
// estimate-driven gate of pr_omega (side 1: v vector, 0: u vector).
static void reorth_vector(svdsc_ctx *c, int side, int ncols, double *w)
{
    const Chunk &ch = side ? c->cn : c->cm;
    const double *W = side ? c->V : c->U;
    const float *W32 = side ? c->V32 : c->U32;
    const int64_t ld = side ? c->ldv : c->ldu;
    if (!c->reorth) {
        cgs2(c, W, W32, ld, ncols, w, ch, poison_ptr(c));
        return;
    }
    const int e0 = ph_begin(c);
    norm_partial(w, ch, c->Pn, poison_ptr(c), c->stream);
    ph_end(c, SVDSC_PH_VEC, e0, 1, 8.0 * ch.len, 2.0 * ch.len);
    const int e1 = ph_begin(c);
    const double L = (double)ch.len, w1 = W32 ? 4.0 : 8.0;
    pr_omega(side, ncols, c->pr_kk, c->T, c->t + 1, c->mu, c->nu, ch, c->Pn, c->st, c->parity, c->pr,
             (w1 + 8.0) * L * ncols + 16.0 * L, (w1 + 8.0) * L * ncols + 32.0 * L, 4.0 * L * ncols,
             c->stream);
    ph_end(c, SVDSC_PH_OTHER, e1, 1, 0.0, 0.0);
    cgs2(c, W, W32, ld, ncols, w, ch, &c->pr->gate, false);
}

// v_{i+1} = A^T u_i - alpha_i v_i, re-orthogonalized against v_1..v_i, beta_i = ||.||  (Alg. 1)
static int issue_v(svdsc_ctx *c, int i)
{
    double *out = colV(c, i);
    int rc = apply_A(c, 1, colU(c, i - 1), colU32(c, i - 1), colV(c, i - 1), Tent(c, i - 1, i - 1), 0.0,
                     out, poison_ptr(c));
    if (rc) return rc;
    reorth_vector(c, 1, i, out);
    do_finalize(c, 1, i, Tent(c, i - 1, i), 0);
    return SVDSC_OK;
}

// u_{i+1} = A v_{i+1} - beta_i u_i, re-orthogonalized against u_1..u_i, alpha_{i+1}  (Alg. 1)
static int issue_u(svdsc_ctx *c, int i)
{
    double *out = colU(c, i);
    int rc = apply_A(c, 0, colV(c, i), colV32(c, i), colU(c, i - 1), Tent(c, i - 1, i), 0.0, out,
                     poison_ptr(c));
    if (rc) return rc;
    reorth_vector(c, 0, i, out);
    do_finalize(c, 0, i, Tent(c, i, i), 0);
    return SVDSC_OK;
}

// Alg. 1 loop for iterations i = s..t (u_{t+1} is not formed); if first_u,
// iteration s starts with its u half (the v half was already formed).
static int issue_segment(svdsc_ctx *c, int s, bool first_u)
{
    NvtxRange range("svdsc: Lanczos segment");
    for (int i = s; i <= c->t; i++) {
        if (!(first_u && i == s)) {
            int rc = issue_v(c, i);
            if (rc) return rc;
        }
        if (i < c->t) {
            int rc = issue_u(c, i);
            if (rc) return rc;
        }
    }
    return SVDSC_OK;
}

int read_status(svdsc_ctx *c)
{
    CU(cudaMemcpyAsync(c->st_host, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return SVDSC_OK;
}

// Waits for the issued work; while a Lanczos vector broke down, replaces it
// by a random vector orthogonalized against its predecessors (T entry 0) and
// re-issues the rest of the segment.
static int settle(svdsc_ctx *c)
{
    int rc = read_status(c);
    if (rc) return rc;
    int guard = 0;
    while (c->st_host->poison) {
        if (c->st_host->nonfinite) return SVDSC_ERR_NONFINITE;
        if (c->st_host->timeout) return SVDSC_ERR_TIMEOUT;
        if (++guard > 4 * (c->t + 2)) return SVDSC_ERR_NONFINITE;
        const int sb = c->st_host->bd_step;
        if (sb < 0 || sb >= (int)c->steps.size()) return SVDSC_ERR_CUDA;
        const StepRec rec = c->steps[sb];
        c->breakdowns++;
        bool repaired = false;
        for (int attempt = 0; attempt < 8 && !repaired; attempt++) {
            DevStatus fresh = *c->st_host;
            fresh.poison = 0;
            fresh.bd_step = INT_MAX;
            fresh.nonfinite = 0;
            CU(cudaMemcpyAsync(c->st, &fresh, sizeof(DevStatus), cudaMemcpyHostToDevice, c->stream));
            c->parity = rec.parity ^ 1;  // anorm slot written by the failed finalize
            double *w = rec.side == 0 ? colU(c, rec.col) : colV(c, rec.col);
            const Chunk &ch = rec.side == 0 ? c->cm : c->cn;
            rng_normal_vec(c->seed, c->draws++, ch.len, w, c->stream);
            ph_end(c, SVDSC_PH_OTHER, -1, 1, 0.0, 0.0);
            if (rec.side == 0) cgs2(c, c->U, nullptr, c->ldu, rec.col, w, ch, poison_ptr(c));
            else cgs2(c, c->V, nullptr, c->ldv, rec.col, w, ch, poison_ptr(c));
            double *Te = nullptr;
            if (rec.side == 0) Te = Tent(c, rec.col, rec.col);
            else Te = Tent(c, rec.col - 1, rec.col);
            do_finalize(c, rec.side, rec.col, Te, 2);
            if (c->reorth) {  // the repaired vector is orthogonal to its predecessors
                pr_reset(rec.side, rec.col, c->mu, c->nu, c->pr, c->stream);
                ph_end(c, SVDSC_PH_OTHER, -1, 1, 0.0, 0.0);
            }
            rc = read_status(c);
            if (rc) return rc;
            repaired = !c->st_host->poison;
            if (!repaired && c->st_host->nonfinite) return SVDSC_ERR_NONFINITE;
        }
        if (!repaired) return SVDSC_ERR_NONFINITE;
        // resume after the repaired vector
        if (rec.side == 1) rc = issue_segment(c, rec.col, true);
        else rc = issue_segment(c, rec.col + 1, false);
        if (rc) return rc;
        rc = read_status(c);
        if (rc) return rc;
    }
    if (c->st_host->timeout) return SVDSC_ERR_TIMEOUT;
    return SVDSC_OK;
}

// ----------------------------------------------------------------- C-ABI

extern "C" {

const char *svdsc_strerror(int status)
{
    switch (status) {
    case SVDSC_OK: return "ok";
    case SVDSC_NOT_CONVERGED: return "not every residual reached tol within maxit rounds";
    case SVDSC_ERR_ARG: return "bad argument";
    case SVDSC_ERR_SIZE: return "subspace dimension does not fit (need t <= m, t + 1 <= n, k <= 256)";
    case SVDSC_ERR_CSR: return "invalid CSR (row pointers or column indices)";
    case SVDSC_ERR_NOMEM: return "out of memory";
    case SVDSC_ERR_CUDA: return "CUDA runtime error";
    case SVDSC_ERR_TIMEOUT: return "a bounded device-side wait timed out";
    case SVDSC_ERR_NONFINITE: return "NaN or Inf in the matrix or a Lanczos vector";
    default: return "unknown status";
    }
}

int svdsc_destroy(svdsc_ctx *c)
{
    if (!c) return SVDSC_OK;
    cudaStreamSynchronize(c->stream);
    free_workspace(c);
    csr_free(&c->A);
    csr_free(&c->AT);
    cudaFree(c->D.a);
    cudaFree(c->dense_part);
    cudaFree(c->st);
    cudaFreeHost(c->st_host);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    delete c;
    return SVDSC_OK;
}

int svdsc_create(svdsc_ctx **out, const svdsc_matrix *A, const svdsc_options *opt, void *stream)
{
    NvtxRange range("svdsc_create");
    if (!out || !A) return SVDSC_ERR_ARG;
    *out = nullptr;
    if (A->m < 1 || A->n < 1) return SVDSC_ERR_ARG;
    if (A->format != SVDSC_CSR && A->format != SVDSC_DENSE) return SVDSC_ERR_ARG;
    const int prec = opt ? opt->precision : SVDSC_FP64;
    if (prec != SVDSC_FP64 && prec != SVDSC_MIXED) return SVDSC_ERR_ARG;
    if (A->format == SVDSC_CSR) {
        if (!A->col_idx || !A->values) return SVDSC_ERR_ARG;
        if (!A->row_ptr && !(A->row_begin && A->row_end)) return SVDSC_ERR_ARG;
        if (A->index_base != 0 && A->index_base != 1) return SVDSC_ERR_ARG;
        if (A->value_type != SVDSC_F64 && A->value_type != SVDSC_F32) return SVDSC_ERR_ARG;
        if (A->m > INT32_MAX || A->n > INT32_MAX) return SVDSC_ERR_SIZE;
    } else {
        if (!A->dense || A->ld < A->m) return SVDSC_ERR_ARG;
        if (prec == SVDSC_MIXED) return SVDSC_ERR_ARG;  // the mixed form is defined for CSR input
    }
    svdsc_ctx *c = new (std::nothrow) svdsc_ctx();
    if (!c) return SVDSC_ERR_NOMEM;
    c->stream = (cudaStream_t)stream;
    c->precision = prec;
    c->seed = opt ? opt->seed : 0;
    c->timing = opt ? (opt->timing != 0) : false;
    c->restart_gemm = opt ? opt->restart_gemm : 0;
    if (c->restart_gemm != 0 && c->restart_gemm != 1) { delete c; return SVDSC_ERR_ARG; }
    c->which = opt ? opt->which : SVDSC_LARGEST;
    if ((c->which != SVDSC_LARGEST && c->which != SVDSC_SMALLEST) ||
        (c->which == SVDSC_SMALLEST && A->m < A->n)) { delete c; return SVDSC_ERR_ARG; }
    c->reorth = opt ? opt->reorth : SVDSC_REORTH_FULL;
    if (c->reorth != SVDSC_REORTH_FULL && c->reorth != SVDSC_REORTH_PARTIAL) { delete c; return SVDSC_ERR_ARG; }
    c->block = (opt && opt->block > 1) ? opt->block : 1;
    if (opt && opt->block < 0) { delete c; return SVDSC_ERR_ARG; }
    if (c->block > 1 && ((c->block != 2 && c->block != 4 && c->block != 8 && c->block != 16) ||
                         A->format != SVDSC_CSR || c->which != SVDSC_LARGEST || c->reorth != SVDSC_REORTH_FULL ||
                         c->restart_gemm != 0)) { delete c; return SVDSC_ERR_ARG; }
    c->format = A->format;
    c->m = A->m;
    c->n = A->n;
    c->ldu = (A->m + 63) & ~int64_t(63);
    c->ldv = (A->n + 63) & ~int64_t(63);
    c->cm = make_chunk(A->m, 2 * 152);
    c->cn = make_chunk(A->n, 2 * 152);
    int rc = SVDSC_OK;
    if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return SVDSC_ERR_CUDA; }
    if (cudaMalloc(&c->st, sizeof(DevStatus)) != cudaSuccess ||
        cudaMallocHost(&c->st_host, sizeof(DevStatus)) != cudaSuccess) {
        svdsc_destroy(c);
        return SVDSC_ERR_NOMEM;
    }
    c->svd.coop_blocks = small_svd_coop_capacity();
    if (A->format == SVDSC_CSR) {
        rc = csr_prepare(A, prec == SVDSC_MIXED, prec == SVDSC_FP64, &c->A, &c->AT, c->stream);
    } else {
        c->D.m = A->m;
        c->D.n = A->n;
        c->D.ld = c->ldu;
        if (cudaMalloc(&c->D.a, sizeof(double) * (size_t)c->D.ld * A->n) != cudaSuccess) rc = SVDSC_ERR_NOMEM;
        if (!rc && cudaMemcpy2DAsync(c->D.a, sizeof(double) * c->D.ld, A->dense, sizeof(double) * A->ld,
                                     sizeof(double) * A->m, A->n,
                                     A->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                     c->stream) != cudaSuccess)
            rc = SVDSC_ERR_CUDA;
        if (!rc && cudaMalloc(&c->dense_part, sizeof(double) * dense_partial_doubles(c->D)) != cudaSuccess)
            rc = SVDSC_ERR_NOMEM;
        if (!rc) {
            int *bad = nullptr;
            int hbad = 0;
            if (cudaMalloc(&bad, sizeof(int)) != cudaSuccess) rc = SVDSC_ERR_NOMEM;
            if (!rc) {
                cudaMemsetAsync(bad, 0, sizeof(int), c->stream);
                check_finite_kernel<<<8 * 152, 256, 0, c->stream>>>(c->D.a, c->D.ld, c->D.m, c->D.n, bad);
                if (cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
                    cudaStreamSynchronize(c->stream) != cudaSuccess)
                    rc = SVDSC_ERR_CUDA;
                else if (hbad)
                    rc = SVDSC_ERR_NONFINITE;
                cudaFree(bad);
            }
        }
    }
    if (rc) {
        svdsc_destroy(c);
        cudaGetLastError();
        return rc;
    }
    *out = c;
    return SVDSC_OK;
}

int svdsc_reserve(svdsc_ctx *c, int t)
{
    if (!c || t < 1) return SVDSC_ERR_ARG;
    return reserve_ws(c, t);
}

int svdsc_solve(svdsc_ctx *c, int k, int p, double tol, int maxit, const double *v0, int v0_on_device,
                double *S, double *U, int64_t ldu, double *V, int64_t ldv, double *res,
                int out_on_device, svdsc_info *info)
{
    NvtxRange range("svdsc_solve");
    if (!c || k < 1 || !(tol > 0.0) || maxit < 1 || !S || !U || !V) return SVDSC_ERR_ARG;
    if (ldu < c->m || ldv < c->n) return SVDSC_ERR_ARG;
    const int t = (p < 0) ? std::max(15, 3 * k) : k + p;
    if (t < k || t > c->m || t + 1 > c->n || k > kGemmGroups * kGemmMaxQ) return SVDSC_ERR_SIZE;
    if (c->restart_gemm == 0 && t > 448) return SVDSC_ERR_SIZE;
    if (t > 512) return SVDSC_ERR_SIZE;  // projected SVD limit
    int rc = reserve_ws(c, t);
    if (rc) return rc;
    cudaStream_t s = c->stream;
    c->t = t;
    c->k = k;
    c->launches = 0;
    ph_reset(c);
    c->parity = 0;
    c->draws = 0;
    c->breakdowns = 0;
    c->n_matvec = 0;
    c->n_steps = 0;
    c->steps.clear();
    c->steps.reserve(4 * (size_t)t);
    c->pr_kk = 0;
    if (c->reorth) pr_reset(0, -1, c->mu, c->nu, c->pr, s);  // nu_1 = mu_1 = 1, counters cleared
    {
        DevStatus init;
        memset(&init, 0, sizeof(init));
        init.bd_step = INT_MAX;
        *c->st_host = init;
        CU(cudaMemcpyAsync(c->st, c->st_host, sizeof(DevStatus), cudaMemcpyHostToDevice, s));
    }
    CU(cudaMemsetAsync(c->T, 0, sizeof(double) * (size_t)(t + 1) * (t + 1), s));

    int restarts = 0;
    double *Uo = c->U, *Vo = c->V;
    DevStatus fin;
    if (c->block > 1) {
        rc = solve_block(c, k, p, tol, maxit, v0, v0_on_device, &Uo, &Vo, &restarts, &fin);
        if (rc) return rc;
    } else {
    // Alg. 1, start: v_1 (the caller's v0 or draw 0), normalised
    if (v0) CU(cudaMemcpyAsync(colV(c, 0), v0, sizeof(double) * c->n,
                               v0_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    else { rng_normal_vec(c->seed, 0, c->n, colV(c, 0), s); ph_end(c, SVDSC_PH_OTHER, -1, 1, 0.0, 0.0); }
    c->draws = 1;
    norm_partial(colV(c, 0), c->cn, c->Pn, nullptr, s);
    ph_end(c, SVDSC_PH_VEC, -1, 1, 8.0 * c->n, 2.0 * c->n);
    do_finalize(c, 1, 0, nullptr, 1);
    rc = read_status(c);
    if (rc) return rc;
    if (c->st_host->poison) {  // unusable v0: fall back to a random draw
        DevStatus fresh = *c->st_host;
        fresh.poison = 0;
        fresh.bd_step = INT_MAX;
        fresh.nonfinite = 0;
        CU(cudaMemcpyAsync(c->st, &fresh, sizeof(DevStatus), cudaMemcpyHostToDevice, s));
        c->parity = 0;
        rng_normal_vec(c->seed, c->draws++, c->n, colV(c, 0), s);
        norm_partial(colV(c, 0), c->cn, c->Pn, nullptr, s);
        ph_end(c, SVDSC_PH_OTHER, -1, 2, 0.0, 0.0);
        do_finalize(c, 1, 0, nullptr, 1);
    }
    c->steps.clear();   // step ids below index Lanczos vectors only
    c->n_steps = 0;
    // u_1 = A v_1, alpha_1
    rc = apply_A(c, 0, colV(c, 0), colV32(c, 0), nullptr, nullptr, 0.0, colU(c, 0), poison_ptr(c));
    if (rc) return rc;
    norm_partial(colU(c, 0), c->cm, c->Pn, poison_ptr(c), s);
    ph_end(c, SVDSC_PH_VEC, -1, 1, 8.0 * c->m, 2.0 * c->m);
    do_finalize(c, 0, 0, Tent(c, 0, 0), 0);
    // Alg. 2: LBP(A, t+1)
    rc = issue_segment(c, 1, false);
    if (rc) return rc;
    rc = settle(c);
    if (rc) return rc;

    for (int it = 1; it <= maxit; it++) {
        // Alg. 2: SVD of T(1:t,1:t)
        {
            const int e0 = ph_begin(c);
            NvtxRange range("svdsc: projected SVD");
            CU(small_svd(t, c->T, t + 1, c->Sh, c->Uh, c->Vh, c->svd, c->st, s, nullptr));
            int nl = 1;
            if (c->which == SVDSC_SMALLEST) {  // wanted (smallest) triplets first, ascending
                reverse_triplets_kernel<<<std::max(1, std::min(64, (t / 2 * t + 255) / 256)), 256, 0, s>>>(
                    t, c->Sh, c->Uh, c->Vh);
                nl++;
            }
            ph_end(c, SVDSC_PH_SVD, e0, nl, 0.0, 0.0);
        }
        // residual test (Eq. 4)
        {
            const int e0 = ph_begin(c);
            residual_kernel<<<1, 256, 0, s>>>(t, k, tol, c->T, c->Sh, c->Uh, c->res, c->rho, c->st, c->parity,
                                              c->which == SVDSC_SMALLEST ? t - 1 : 0);
            ph_end(c, SVDSC_PH_OTHER, e0, 1, 0.0, 0.0);
        }
        CU(cudaGetLastError());
        rc = read_status(c);
        if (rc) return rc;
        if (c->st_host->timeout) return SVDSC_ERR_TIMEOUT;
        if (c->st_host->converged || it == maxit) break;
        // augmented restart (Eq. 5-7)
        {
        NvtxRange restart_range("svdsc: augmented restart");
        if (c->restart_gemm == 0) {
            // U~_k = U(:,1:t) Uh(:,1:k), V~_k = V(:,1:t) Vh(:,1:k) into the other bases
            rc = gemm_tc(c, c->U, c->U32, c->ldu, c->m, t, c->Uh, k, c->Ua, c->U32a);
            if (rc) return rc;
            rc = gemm_tc(c, c->V, c->V32, c->ldv, c->n, t, c->Vh, k, c->Va, c->V32a);
            if (rc) return rc;
            // v_{k+1} = v_{t+1}
            CU(cudaMemcpyAsync(c->Va + (int64_t)k * c->ldv, colV(c, t), sizeof(double) * c->n,
                               cudaMemcpyDeviceToDevice, s));
            if (c->V32)
                CU(cudaMemcpyAsync(c->V32a + (int64_t)k * c->ldv, colV32(c, t), sizeof(float) * c->n,
                                   cudaMemcpyDeviceToDevice, s));
            std::swap(c->U, c->Ua);
            std::swap(c->V, c->Va);
            std::swap(c->U32, c->U32a);
            std::swap(c->V32, c->V32a);
        } else {
            rc = gemm_inplace(c, c->U, c->ldu, c->m, t, c->Uh, k);   // U~_k = U(:,1:t) Uh(:,1:k)
            if (rc) return rc;
            rc = gemm_inplace(c, c->V, c->ldv, c->n, t, c->Vh, k);   // V~_k = V(:,1:t) Vh(:,1:k)
            if (rc) return rc;
            CU(cudaMemcpyAsync(colV(c, k), colV(c, t), sizeof(double) * c->n, cudaMemcpyDeviceToDevice, s));
            if (c->precision == SVDSC_MIXED) {
                copy_f64_to_f32(c->U, c->U32, c->ldu * k, s);
                copy_f64_to_f32(c->V, c->V32, c->ldv * (k + 1), s);
                ph_end(c, SVDSC_PH_OTHER, -1, 2, 12.0 * (c->ldu * k + c->ldv * (k + 1)), 0.0);
            }
        }
        restart_T_kernel<<<1, 256, 0, s>>>(t, k, c->T, c->Sh, c->rho);
        ph_end(c, SVDSC_PH_OTHER, -1, 1, 0.0, 0.0);
        if (c->reorth) {
            pr_restart(t, k, c->Vh, c->mu, c->nu, c->pr, s);
            ph_end(c, SVDSC_PH_OTHER, -1, 1, 0.0, 0.0);
            c->pr_kk = k;
        }
        CU(cudaGetLastError());
        // u_{k+1} = A v_{k+1} - U~_k rho (Eq. 7), re-orthogonalized against U~_k
        rc = apply_A(c, 0, colV(c, k), colV32(c, k), nullptr, nullptr, 0.0, colU(c, k), poison_ptr(c));
        if (rc) return rc;
        {
            const int e0 = ph_begin(c);
            update_sub(c->U, c->ldu, k, c->rho, colU(c, k), c->cm, nullptr, poison_ptr(c), s);
            ph_end(c, SVDSC_PH_GEMV_N, e0, 1, 8.0 * c->m * k + 16.0 * c->m, 2.0 * c->m * k);
        }
        cgs2(c, c->U, c->U32, c->ldu, k, colU(c, k), c->cm, poison_ptr(c));
        do_finalize(c, 0, k, Tent(c, k, k), 0);
        restarts++;
        }
        // continue Alg. 1 from i = k+1
        rc = issue_segment(c, k + 1, false);
        if (rc) return rc;
        rc = settle(c);
        if (rc) return rc;
    }
    fin = *c->st_host;

    // outputs of Alg. 2 (into the spare bases or in place, then copied out)
    NvtxRange out_range("svdsc: outputs");
    if (c->restart_gemm == 0) {
        rc = gemm_tc(c, c->U, c->U32, c->ldu, c->m, t, c->Uh, k, c->Ua, nullptr);
        if (rc) return rc;
        rc = gemm_tc(c, c->V, c->V32, c->ldv, c->n, t, c->Vh, k, c->Va, nullptr);
        if (rc) return rc;
        Uo = c->Ua;
        Vo = c->Va;
    } else {
        rc = gemm_inplace(c, c->U, c->ldu, c->m, t, c->Uh, k);
        if (rc) return rc;
        rc = gemm_inplace(c, c->V, c->ldv, c->n, t, c->Vh, k);
        if (rc) return rc;
    }
    }  // single-vector form
    sign_kernel<<<k, 256, 0, s>>>(Uo, c->ldu, c->m, Vo, c->ldv, c->n);
    ph_end(c, SVDSC_PH_OTHER, -1, 1, 0.0, 0.0);
    CU(cudaGetLastError());
    const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CU(cudaMemcpyAsync(S, c->Sh, sizeof(double) * k, kind, s));
    if (res) CU(cudaMemcpyAsync(res, c->res, sizeof(double) * k, kind, s));
    CU(cudaMemcpy2DAsync(U, sizeof(double) * ldu, Uo, sizeof(double) * c->ldu, sizeof(double) * c->m, k,
                         kind, s));
    CU(cudaMemcpy2DAsync(V, sizeof(double) * ldv, Vo, sizeof(double) * c->ldv, sizeof(double) * c->n, k,
                         kind, s));
    CU(cudaStreamSynchronize(s));
    if (c->st_host->timeout) return SVDSC_ERR_TIMEOUT;
    rc = read_status(c);  // a CUDA error here is reported as such, not as a timeout
    if (rc) return rc;
    if (c->st_host->timeout) return SVDSC_ERR_TIMEOUT;
    if (info) {
        memset(info, 0, sizeof(*info));
        info->converged = fin.converged;
        info->nconv = fin.nconv;
        info->restarts = restarts;
        info->breakdowns = c->breakdowns;
        info->n_matvec = c->n_matvec;
        info->n_steps = c->n_steps;
        info->n_launches = c->launches;
        info->anorm_est = std::max(fin.anorm[0], fin.anorm[1]);
        info->beta_t = fin.beta_t;
        info->t = c->block > 1 ? c->t : t;
        for (int i = 0; i < SVDSC_NUM_PHASES; i++) {
            info->launches[i] = c->ph_launch[i];
            info->bytes[i] = c->ph_bytes[i];
            info->flops[i] = c->ph_flops[i];
        }
        // every Lanczos vector but u_1 (full), or the estimate-driven ones plus
        // the restart vectors (partial), whose CGS2 bytes were counted on the device
        info->n_reorth = c->n_steps - c->block;
        if (c->reorth) {
            PrState ps;
            CU(cudaMemcpy(&ps, c->pr, sizeof(PrState), cudaMemcpyDeviceToHost));
            info->n_reorth = ps.n_reorth + restarts;
            info->bytes[SVDSC_PH_GEMV_T] += ps.bytes_t;
            info->bytes[SVDSC_PH_GEMV_N] += ps.bytes_n;
            info->flops[SVDSC_PH_GEMV_T] += ps.flops;
            info->flops[SVDSC_PH_GEMV_N] += ps.flops;
        }
        for (const auto &r : c->recs) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, c->ev_pool[r.e0], c->ev_pool[r.e1]) == cudaSuccess)
                info->ms[r.ph] += ms;
        }
    }
    return fin.converged ? SVDSC_OK : SVDSC_NOT_CONVERGED;
}

int svdsc_matvec(svdsc_ctx *c, int trans, const double *x, const double *z, double coef, double *y)
{
    if (!c || !x || !y || (trans != 0 && trans != 1)) return SVDSC_ERR_ARG;
    float *x32 = nullptr;
    if (c->precision == SVDSC_MIXED) {
        const int64_t len = trans ? c->m : c->n;
        if (cudaMalloc(&x32, sizeof(float) * len) != cudaSuccess) return SVDSC_ERR_NOMEM;
        copy_f64_to_f32(x, x32, len, c->stream);
    }
    const int64_t saved = c->n_matvec;
    int rc = apply_A(c, trans, x, x32, z, nullptr, coef, y, nullptr);
    c->n_matvec = saved;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) rc = SVDSC_ERR_CUDA;
    cudaFree(x32);
    return rc;
}

int svdsc_cgs2(svdsc_ctx *c, int64_t len, int64_t ncols, const double *W, int64_t ldw, double *w,
               double *norm_out)
{
    if (!c || !W || !w || !norm_out || ncols < 0 || ldw < len) return SVDSC_ERR_ARG;
    if (((uintptr_t)W & 15) || ((uintptr_t)w & 15) || (ldw & 1)) return SVDSC_ERR_ARG;
    const Chunk *ch = (len == c->m) ? &c->cm : (len == c->n ? &c->cn : nullptr);
    if (!ch) return SVDSC_ERR_ARG;
    if (ncols > c->t_cap + 1) return SVDSC_ERR_SIZE;
    cgs2(c, W, nullptr, ldw, (int)ncols, w, *ch, nullptr);
    norm_from_partials(c->Pn, ch->nbu, norm_out, c->stream);
    if (cudaGetLastError() != cudaSuccess) return SVDSC_ERR_CUDA;
    return cudaStreamSynchronize(c->stream) == cudaSuccess ? SVDSC_OK : SVDSC_ERR_CUDA;
}

int svdsc_gemm(svdsc_ctx *c, int mode, int64_t rows, int t, int k, const double *W, int64_t ldw,
               const double *Q, int64_t ldq, double *C, int64_t ldc)
{
    if (!c || !W || !Q || !C || rows < 1 || t < 1 || k < 1 || k > t || ldw < rows || ldq < t || ldc < rows)
        return SVDSC_ERR_ARG;
    if (mode != 0 && mode != 1) return SVDSC_ERR_ARG;
    if (t > c->t_cap || (mode == 0 && t > 448)) return SVDSC_ERR_SIZE;
    int nl = 0;
    DevStatus init;
    memset(&init, 0, sizeof(init));
    init.bd_step = INT_MAX;
    CU(cudaMemcpyAsync(c->st, &init, sizeof(DevStatus), cudaMemcpyHostToDevice, c->stream));
    CU(tc_gemm(mode, W, nullptr, ldw, rows, t, Q, ldq, k, C, ldc, nullptr, c->gemm_ws, &c->st->timeout,
               c->stream, &nl));
    int rc = read_status(c);
    if (rc) return rc;
    return c->st_host->timeout ? SVDSC_ERR_TIMEOUT : SVDSC_OK;
}

int svdsc_selftest_wait(svdsc_ctx *c, int kind)
{
    if (!c || (kind != 0 && kind != 1)) return SVDSC_ERR_ARG;
    int rc = reserve_ws(c, 2);  // the status block and the barrier words
    if (rc) return rc;
    DevStatus init;
    memset(&init, 0, sizeof(init));
    init.bd_step = INT_MAX;
    CU(cudaMemcpyAsync(c->st, &init, sizeof(DevStatus), cudaMemcpyHostToDevice, c->stream));
    if (kind == 0) CU(probe_grid_barrier(c->svd.bar, c->st, c->stream));
    else CU(probe_mbarrier(&c->st->timeout, c->stream));
    rc = read_status(c);
    if (rc) return rc;
    const int ran_out = c->st_host->timeout;
    init.timeout = 0;  // leave the context as a solve expects it
    CU(cudaMemcpyAsync(c->st, &init, sizeof(DevStatus), cudaMemcpyHostToDevice, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return ran_out ? SVDSC_ERR_TIMEOUT : SVDSC_OK;
}

int svdsc_small_svd(svdsc_ctx *c, int t, const double *T, int64_t ldt, double *S, double *Uh, double *Vh)
{
    if (!c || t < 1 || !T || !S || !Uh || !Vh || ldt < t) return SVDSC_ERR_ARG;
    if (t > c->t_cap || t > 512) return SVDSC_ERR_SIZE;
    DevStatus init;
    memset(&init, 0, sizeof(init));
    init.bd_step = INT_MAX;
    CU(cudaMemcpyAsync(c->st, &init, sizeof(DevStatus), cudaMemcpyHostToDevice, c->stream));
    CU(small_svd(t, T, ldt, S, Uh, Vh, c->svd, c->st, c->stream, nullptr));
    int rc = read_status(c);
    if (rc) return rc;
    if (c->st_host->timeout) return SVDSC_ERR_TIMEOUT;
    return SVDSC_OK;
}

}  // extern "C"
