// Projected SVD of Alg. 2 (svds-C paper): [Uh, Sh, Vh] = svd(T(1:t,1:t))
// in FP64 on the device, by one-sided (Hestenes) Jacobi: columns of B = T V
// are rotated in pairs until mutually orthogonal; sigma_j = ||B(:,j)||,
// uh_j = B(:,j)/sigma_j, vh_j = the accumulated rotation.  Pairs are visited
// in round-robin (circle) order so that t/2 disjoint rotations run at once:
//   t <= 64 : one CTA, B and V in shared memory, one warp per pair;
//   t  > 64 : a cooperative multi-CTA kernel (one pair per CTA per round,
//             B and V in global memory, rounds ordered by per-column flags,
//             one bounded grid barrier per sweep),
// since GB300 has ~2 FP64 FMA/clk/SM and an O(t^3) sweep must be spread over
// many SMs.  The convergence test matches the CPU oracle's:
// |b_p . b_q| <= eps sqrt(t) ||b_p|| ||b_q||.
#include <cfloat>
#include <cstdint>
#include "internal.cuh"

namespace svdsc {

__device__ __forceinline__ void rr_pair(int slot, int round, int n2, int *p, int *q)
{
    auto player = [&](int pos) { return pos == 0 ? 0 : ((pos - 1 + round) % (n2 - 1)) + 1; };
    int a = player(slot), b = player(n2 - 1 - slot);
    *p = a < b ? a : b;
    *q = a < b ? b : a;
}

// Rotation of Golub & Van Loan (one-sided Jacobi) that zeroes gamma in
// [alpha gamma; gamma beta]; same skip test as the oracle.  With d = beta -
// alpha and zeta = d / (2 gamma), tan = sign(zeta) / (|zeta| + sqrt(1 +
// zeta^2)) is evaluated as sign(zeta) |2 gamma| / (|d| + sqrt(d^2 + 4
// gamma^2)) (numerator and denominator times |2 gamma|) and c = rsqrt(1 +
// tan^2): one square root, one division and one reciprocal square root on the
// critical path instead of three square roots and three divisions, which on
// GB300's narrow FP64 pipe are the longest part of a Jacobi round.  d and
// 2 gamma are first scaled by an exact power of two so their squares cannot
// overflow or lose everything to underflow.
__device__ __forceinline__ bool jacobi_rotation(double alpha, double beta, double gamma, double tol,
                                                double *c, double *s)
{
    if (gamma == 0.0 || fabs(gamma) <= tol * sqrt(alpha * beta)) return false;
    const double d = beta - alpha, g2 = 2.0 * gamma;
    const double mx = fmax(fabs(d), fabs(g2));
    if (!isfinite(mx)) return false;
    // 2^-floor(log2 mx) from the exponent field (mx > 0: g2 != 0), clamped to
    // the normal range: a subnormal mx (field 0) gets 2^1023, which brings it
    // above 2^-52, and mx >= 2^1023 gets 2^-1022, which leaves it below 4
    const int ex = (int)((unsigned long long)__double_as_longlong(mx) >> 52) & 0x7FF;
    const int fs = ex == 0 ? 2046 : (ex >= 2046 ? 1 : 2046 - ex);
    const double sc = __longlong_as_double((long long)fs << 52);
    const double ds = d * sc, gs = fabs(g2) * sc;
    const double r = sqrt(fma(ds, ds, gs * gs));
    // sign(zeta), with zeta = +-0 counted as positive like the unscaled form
    const bool neg = d != 0.0 && ((d > 0.0) != (gamma > 0.0));
    const double tt = (neg ? -gs : gs) / (fabs(ds) + r);
    *c = rsqrt(fma(tt, tt, 1.0));
    *s = *c * tt;
    return true;
}

// Completes columns with sigma == 0 to an orthonormal set: the first unit
// vectors that survive two Gram-Schmidt passes against the other columns
// (same rule as the oracle).  One CTA; Uh column-major t x t (ld t).
__device__ void complete_zero_columns(int t, double *Uh, const double *S)
{
    __shared__ double red[32];
    __shared__ double s_val;
    int next_e = 0;
    for (int j = 0; j < t; j++) {
        if (S[j] > 0.0) continue;
        double *u = Uh + (int64_t)j * t;
        while (next_e < t) {
            for (int r = threadIdx.x; r < t; r += blockDim.x) u[r] = (r == next_e) ? 1.0 : 0.0;
            next_e++;
            __syncthreads();
            for (int pass = 0; pass < 2; pass++) {
                for (int i = 0; i < t; i++) {
                    if (i == j || (S[i] == 0.0 && i > j)) continue;
                    const double *ui = Uh + (int64_t)i * t;
                    double d = 0.0;
                    for (int r = threadIdx.x; r < t; r += blockDim.x) d += ui[r] * u[r];
                    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
                    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        double tot = 0.0;
                        for (int w = 0; w < (int)(blockDim.x >> 5); w++) tot += red[w];
                        s_val = tot;
                    }
                    __syncthreads();
                    d = s_val;
                    for (int r = threadIdx.x; r < t; r += blockDim.x) u[r] -= d * ui[r];
                    __syncthreads();
                }
            }
            double q = 0.0;
            for (int r = threadIdx.x; r < t; r += blockDim.x) q += u[r] * u[r];
            for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = q;
            __syncthreads();
            if (threadIdx.x == 0) {
                double tot = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); w++) tot += red[w];
                s_val = sqrt(tot);
            }
            __syncthreads();
            const double nu = s_val;
            if (nu > 0.5) {
                for (int r = threadIdx.x; r < t; r += blockDim.x) u[r] /= nu;
                __syncthreads();
                break;
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------ one-CTA form
constexpr int kSmallT = 64;
constexpr int kSmallThreads = 1024;

__global__ void __launch_bounds__(kSmallThreads)
jacobi_small_kernel(int t, const double *__restrict__ T, int64_t ldt, double *__restrict__ S,
                    double *__restrict__ Uh, double *__restrict__ Vh, DevStatus *st, int max_sweeps)
{
    extern __shared__ double sm[];
    double *B = sm;                       // t x t, ld kSmallT
    double *W = sm + kSmallT * kSmallT;   // t x t, ld kSmallT
    __shared__ double sig[kSmallT];
    __shared__ int rot_count;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int i = threadIdx.x; i < t * t; i += blockDim.x) {
        const int r = i % t, c = i / t;
        B[r + c * kSmallT] = T[r + (int64_t)c * ldt];
        W[r + c * kSmallT] = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    const double tol = DBL_EPSILON * sqrt((double)t);
    const int n2 = t + (t & 1);
    int sweeps = 0;
    bool conv = false;
    while (sweeps < max_sweeps) {
        if (threadIdx.x == 0) rot_count = 0;
        __syncthreads();
        sweeps++;
        for (int round = 0; round < n2 - 1; round++) {
            for (int slot = warp; slot < n2 / 2; slot += nwarps) {
                int p, q;
                rr_pair(slot, round, n2, &p, &q);
                if (q >= t) continue;
                double *bp = B + p * kSmallT, *bq = B + q * kSmallT;
                double a = 0.0, b = 0.0, g = 0.0;
                for (int r = lane; r < t; r += 32) {
                    a += bp[r] * bp[r];
                    b += bq[r] * bq[r];
                    g += bp[r] * bq[r];
                }
                for (int o = 16; o > 0; o >>= 1) {
                    a += __shfl_xor_sync(0xffffffffu, a, o);
                    b += __shfl_xor_sync(0xffffffffu, b, o);
                    g += __shfl_xor_sync(0xffffffffu, g, o);
                }
                double c, s;
                if (!jacobi_rotation(a, b, g, tol, &c, &s)) continue;
                if (lane == 0) atomicAdd(&rot_count, 1);
                for (int r = lane; r < t; r += 32) {
                    const double x = bp[r], y = bq[r];
                    bp[r] = c * x - s * y;
                    bq[r] = s * x + c * y;
                }
                double *wp = W + p * kSmallT, *wq = W + q * kSmallT;
                for (int r = lane; r < t; r += 32) {
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
    // singular values, descending stable order, outputs
    for (int j = warp; j < t; j += nwarps) {
        double a = 0.0;
        for (int r = lane; r < t; r += 32) a += B[r + j * kSmallT] * B[r + j * kSmallT];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) sig[j] = sqrt(a);
    }
    __syncthreads();
    for (int j = warp; j < t; j += nwarps) {
        const double sj = sig[j];
        int rank = 0;
        for (int i = 0; i < t; i++) rank += (sig[i] > sj) || (sig[i] == sj && i < j);
        if (lane == 0) S[rank] = sj;
        for (int r = lane; r < t; r += 32) {
            Uh[r + (int64_t)rank * t] = sj > 0.0 ? B[r + j * kSmallT] / sj : 0.0;
            Vh[r + (int64_t)rank * t] = W[r + j * kSmallT];
        }
    }
    __syncthreads();
    if (sig[0] >= 0.0) {  // zero singular values are rare: check on the sorted list
        bool anyzero = false;
        for (int j = 0; j < t; j++) anyzero |= (sig[j] == 0.0);
        if (anyzero) complete_zero_columns(t, Uh, S);
    }
    if (threadIdx.x == 0) st->svd_sweeps = conv ? sweeps : -1;
}

// ------------------------------------------------------------ multi-CTA form
constexpr int kCoopThreads = 256;
constexpr int kCoopPer = 2;  // column elements per thread: t <= 512

// Bounded grid barrier for a cooperative launch (all CTAs co-resident).
// bar[0]: arrivals, bar[1]: generation.  Gives up after ~0.5-1 s of spinning,
// records the timeout and returns false.
__device__ bool grid_sync(unsigned *bar, unsigned nblk, int *timeout)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = bar + 1;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u);
        int ok = 1;
        if (arrived == nblk - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            unsigned long long spins = 0;
            while (*vgen == gen) {
                if (++spins > (1ull << 23)) { ok = 0; atomicExch(timeout, 1); break; }
                if (spins > 2048) __nanosleep(32);  // poll tightly first, then back off
            }
        }
        __threadfence();
        s_ok = ok && !*(volatile int *)timeout;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ double block_sum_coop(double v, double *red, double *out)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tsum = 0.0;
        for (int w = 0; w < kCoopThreads / 32; w++) tsum += red[w];
        *out = tsum;
    }
    __syncthreads();
    return *out;
}

__global__ void __launch_bounds__(kCoopThreads)
jacobi_coop_kernel(int t, const double *__restrict__ T, int64_t ldt, double *B, double *W,
                   double *sig, int *rot, unsigned *bar, DevStatus *st, int max_sweeps,
                   double *__restrict__ S, double *__restrict__ Uh, double *__restrict__ Vh)
{
    __shared__ double red[kCoopThreads / 32];
    __shared__ double sv;
    __shared__ double part[3][kCoopThreads];
    __shared__ double s_cs[2];
    __shared__ int s_rot;
    const unsigned nblk = gridDim.x;
    int *timeout = &st->timeout;
    // B = T, W = I
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)t * t;
         i += (int64_t)nblk * blockDim.x) {
        const int r = (int)(i % t), c = (int)(i / t);
        __stcg(B + i, T[r + (int64_t)c * ldt]);
        __stcg(W + i, (r == c) ? 1.0 : 0.0);
    }
    if (!grid_sync(bar, nblk, timeout)) return;
    const double tol = DBL_EPSILON * sqrt((double)t);
    const int n2 = t + (t & 1);
    const int nwrow = t < kCoopThreads ? (t + 31) / 32 : kCoopThreads / 32;  // warps holding rows
    // Rounds are ordered by per-column version flags instead of grid
    // barriers: flag[c] counts the rounds completed on column c, the CTA that
    // owns the pair (p, q) in global round R waits (bounded) for both flags to
    // reach R, rotates, and publishes R + 1.  Each column has exactly one
    // reader-writer per round, so no other ordering is needed; one grid
    // barrier per sweep remains for the convergence test.
    unsigned *flag = bar + 2;
    __shared__ int s_go;
    unsigned R = 0;
    int sweeps = 0;
    bool conv = false;
    while (sweeps < max_sweeps) {
        for (int round = 0; round < n2 - 1; round++, R++) {
            for (int slot = blockIdx.x; slot < n2 / 2; slot += nblk) {
                int p, q;
                rr_pair(slot, round, n2, &p, &q);
                const bool idle = q >= t;  // odd t: column p sits this round out
                if (threadIdx.x == 0) {
                    int ok = 1;
                    unsigned long long spins = 0;
                    // both flags are loaded before either is tested: one L2
                    // round trip per poll instead of two
                    for (;;) {
                        const unsigned fp = ld_acquire_u32(flag + p);
                        const unsigned fq = idle ? R : ld_acquire_u32(flag + q);
                        if (fp >= R && fq >= R) break;
                        if (++spins > (1ull << 24) || *(volatile int *)timeout) { ok = 0; break; }
                        if (spins > 256) __nanosleep(32);
                    }
                    if (!ok) atomicExch(timeout, 1);
                    s_go = ok;
                }
                __syncthreads();
                if (!s_go) return;
                if (idle) {
                    if (threadIdx.x == 0) st_release_u32(flag + p, R + 1);
                    __syncthreads();  // s_go is read by every thread before thread 0 rewrites it
                    continue;
                }
                double *bp = B + (int64_t)p * t, *bq = B + (int64_t)q * t;
                double *wp = W + (int64_t)p * t, *wq = W + (int64_t)q * t;
                // every element of both pairs of columns is loaded once, up front
                // (t <= kCoopThreads * kCoopPer), and kept in registers; warps
                // past the last row skip the FP64 work
                double xb[kCoopPer], yb[kCoopPer], xw[kCoopPer], yw[kCoopPer];
#pragma unroll
                for (int u = 0; u < kCoopPer; u++) {
                    const int r = threadIdx.x + u * kCoopThreads;
                    xb[u] = yb[u] = xw[u] = yw[u] = 0.0;
                    if (r < t) {
                        xb[u] = __ldcg(bp + r);
                        yb[u] = __ldcg(bq + r);
                        xw[u] = __ldcg(wp + r);
                        yw[u] = __ldcg(wq + r);
                    }
                }
                double a = 0.0, b = 0.0, g = 0.0;
#pragma unroll
                for (int u = 0; u < kCoopPer; u++) {
                    if (threadIdx.x + u * kCoopThreads < t) {
                        a += xb[u] * xb[u];
                        b += yb[u] * yb[u];
                        g += xb[u] * yb[u];
                    }
                }
                // GB300 issues FP64 at ~2 lanes/clk/SM, so the reduction and
                // the rotation are done by one warp, not by every warp of the
                // CTA: per-thread partials go through shared memory, warp 0
                // adds them up and reduces the three sums with one transposed
                // butterfly (6 FP64 adds instead of 3 x 5 per warp), and one
                // lane computes the rotation.
                part[0][threadIdx.x] = a;
                part[1][threadIdx.x] = b;
                part[2][threadIdx.x] = g;
                __syncthreads();
                if (threadIdx.x < 32) {
                    const int lane = threadIdx.x;
                    double v0 = part[0][lane], v1 = part[1][lane], v2 = part[2][lane];
                    for (int w = 1; w < nwrow; w++) {
                        v0 += part[0][lane + 32 * w];
                        v1 += part[1][lane + 32 * w];
                        v2 += part[2][lane + 32 * w];
                    }
                    // lanes with bit 4 clear gather (v0, v1), the others (v2, 0)
                    const bool h16 = (lane & 16) != 0;
                    double k0 = h16 ? v2 : v0, k1 = h16 ? 0.0 : v1;
                    const double s0 = h16 ? v0 : v2, s1 = h16 ? v1 : 0.0;
                    k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
                    k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
                    // bit 3 clear keeps the first of the two, set the second
                    const bool h8 = (lane & 8) != 0;
                    double k = h8 ? k1 : k0;
                    k += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
                    for (int o = 4; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
                    // lane 0: sum of v0 (alpha), lane 8: v1 (beta), lane 16: v2 (gamma)
                    const double beta = __shfl_sync(0xffffffffu, k, 8);
                    const double gamma = __shfl_sync(0xffffffffu, k, 16);
                    if (lane == 0) {
                        double c = 1.0, s = 0.0;
                        const bool do_rot = jacobi_rotation(k, beta, gamma, tol, &c, &s);
                        s_cs[0] = c;
                        s_cs[1] = s;
                        s_rot = do_rot;
                        if (do_rot) atomicAdd(rot + sweeps, 1);
                    }
                }
                __syncthreads();
                if (s_rot) {
                    const double c = s_cs[0], s = s_cs[1];
#pragma unroll
                    for (int u = 0; u < kCoopPer; u++) {
                        const int r = threadIdx.x + u * kCoopThreads;
                        if (r < t) {
                            __stcg(bp + r, c * xb[u] - s * yb[u]);
                            __stcg(bq + r, s * xb[u] + c * yb[u]);
                            __stcg(wp + r, c * xw[u] - s * yw[u]);
                            __stcg(wq + r, s * xw[u] + c * yw[u]);
                        }
                    }
                }
                __syncthreads();  // every store of the CTA precedes the release below
                if (threadIdx.x == 0) {
                    __threadfence();
                    st_release_u32(flag + p, R + 1);
                    st_release_u32(flag + q, R + 1);
                }
            }
        }
        if (!grid_sync(bar, nblk, timeout)) return;  // once per sweep: the rotation count is final
        const int done = (__ldcg(rot + sweeps) == 0);
        sweeps++;
        if (done) { conv = true; break; }
    }
    for (int j = blockIdx.x; j < t; j += nblk) {
        const double *bj = B + (int64_t)j * t;
        double a = 0.0;
        for (int r = threadIdx.x; r < t; r += kCoopThreads) {
            const double x = __ldcg(bj + r);
            a += x * x;
        }
        const double tot = block_sum_coop(a, red, &sv);
        if (threadIdx.x == 0) __stcg(sig + j, sqrt(tot));
    }
    if (!grid_sync(bar, nblk, timeout)) return;
    for (int j = blockIdx.x; j < t; j += nblk) {
        const double sj = __ldcg(sig + j);
        int rank = 0;
        for (int i = 0; i < t; i++) {
            const double si = __ldcg(sig + i);
            rank += (si > sj) || (si == sj && i < j);
        }
        if (threadIdx.x == 0) S[rank] = sj;
        for (int r = threadIdx.x; r < t; r += kCoopThreads) {
            Uh[r + (int64_t)rank * t] = sj > 0.0 ? __ldcg(B + r + (int64_t)j * t) / sj : 0.0;
            Vh[r + (int64_t)rank * t] = __ldcg(W + r + (int64_t)j * t);
        }
    }
    if (!grid_sync(bar, nblk, timeout)) return;
    if (blockIdx.x == 0) {
        bool anyzero = false;
        for (int j = 0; j < t; j++) anyzero |= (__ldcg(sig + j) == 0.0);
        if (anyzero) complete_zero_columns(t, Uh, S);
        if (threadIdx.x == 0) st->svd_sweeps = conv ? sweeps : -1;
    }
}

// Self-test of the bounded grid barrier: every CTA waits for one more arrival
// than the grid has, so the wait must run out; grid_sync records the timeout
// in the status block and each CTA returns.
__global__ void barrier_probe_kernel(unsigned *bar, DevStatus *st)
{
    grid_sync(bar, gridDim.x + 1, &st->timeout);
}

cudaError_t probe_grid_barrier(unsigned *bar, DevStatus *st, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    void *args[] = {&bar, &st};
    return cudaLaunchCooperativeKernel((const void *)barrier_probe_kernel, dim3(4), dim3(kCoopThreads), args,
                                       0, s);
}

int small_svd_coop_capacity()
{
    int dev = 0, nsm = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, jacobi_coop_kernel, kCoopThreads, 0) !=
        cudaSuccess)
        return 0;
    return nsm * per;
}

cudaError_t small_svd(int t, const double *T, int64_t ldt, double *S, double *Uh, double *Vh,
                      SvdWork &w, DevStatus *st, cudaStream_t s, int *launches)
{
    if (t <= kSmallT) {
        const size_t smem = 2 * sizeof(double) * kSmallT * kSmallT;
        static std::atomic<unsigned long long> attr_done{0};
        cudaError_t e = set_smem_limit_once((const void *)jacobi_small_kernel, (int)smem, &attr_done);
        if (e != cudaSuccess) return e;
        jacobi_small_kernel<<<1, kSmallThreads, smem, s>>>(t, T, ldt, S, Uh, Vh, st, 100);
        if (launches) (*launches)++;
        return cudaGetLastError();
    }
    if (t > kCoopThreads * kCoopPer) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(w.bar, 0, (2 + (size_t)t) * sizeof(unsigned), s);  // barrier + column flags
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(w.rot, 0, sizeof(int) * w.max_sweeps, s);
    if (e != cudaSuccess) return e;
    int nblk = (t + (t & 1)) / 2;
    if (nblk > w.coop_blocks) nblk = w.coop_blocks;
    if (nblk < 1) return cudaErrorInvalidConfiguration;
    int tt = t;
    int64_t ld = ldt;
    int ms = w.max_sweeps;
    void *args[] = {&tt, (void *)&T, &ld, &w.B, &w.W, &w.sig, &w.rot, &w.bar, &st, &ms, &S, &Uh, &Vh};
    e = cudaLaunchCooperativeKernel((const void *)jacobi_coop_kernel, dim3(nblk), dim3(kCoopThreads),
                                    args, 0, s);
    if (launches) (*launches)++;
    return e;
}

}  // namespace svdsc
