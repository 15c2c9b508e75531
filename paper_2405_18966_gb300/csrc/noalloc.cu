// CGS2 re-orthogonalization for callers that cannot allocate device memory.
//
// svdsc_cgs2 needs a context, and a context owns device memory obtained with
// cudaMalloc.  Some callers cannot do that: code that runs while a framework's
// caching allocator has reserved all device memory, real-time or serving loops
// whose memory budget is fixed before they start (cudaMalloc may synchronize
// the device and can fail mid-run), and libraries embedded in hosts that only
// hand them pre-allocated buffers.  svdsc_cgs2_noalloc does the same work as
// svdsc_cgs2 with its scratch (the per-chunk partial sums, the projection
// coefficients and the partial norms) in one file-scope __device__ array of
// fixed size.  Every GPU that loads this library holds that array until the
// process exits.  The paper has no counterpart of this entry point.
#include <mutex>
#include "internal.cuh"

namespace svdsc {

constexpr int64_t kNoAllocMaxCols = 512;   // ncols limit
constexpr int kNoAllocMaxChunks = 1024;    // row chunks of <= 4096 rows: len <= 4,194,304
constexpr int kNoAllocMaxNormParts = 8192; // GEMV-N CTAs of >= 512 rows at that length
constexpr size_t kNoAllocDoubles =
    (size_t)kNoAllocMaxChunks * kNoAllocMaxCols + kNoAllocMaxCols + kNoAllocMaxNormParts;
constexpr int kNoAllocMaxDevices = 64;

// 4.3 MB of scratch per device: P (ncols x chunks), h (ncols), Pn (GEMV-N CTAs).
static __device__ __align__(256) double g_cgs2_scratch[kNoAllocDoubles];

static std::mutex g_scratch_mu;
static double *g_scratch_addr[kNoAllocMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (the name itself is only a host-side stand-in).
static int scratch_address(double **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SVDSC_ERR_CUDA;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return SVDSC_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_cgs2_scratch) != cudaSuccess || !p) return SVDSC_ERR_CUDA;
        g_scratch_addr[dev] = (double *)p;
    }
    *out = g_scratch_addr[dev];
    return SVDSC_OK;
}

__global__ void noalloc_norm_kernel(const double *__restrict__ Pn, int nb, double *out)
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

}  // namespace svdsc

using namespace svdsc;

extern "C" int svdsc_cgs2_noalloc(int64_t len, int64_t ncols, const double *W, int64_t ldw, double *w,
                                  double *norm_out, void *stream)
{
    if (!w || !norm_out || len < 1 || ncols < 0 || (ncols > 0 && (!W || ldw < len)))
        return SVDSC_ERR_ARG;
    if (((uintptr_t)W & 15) || ((uintptr_t)w & 15) || (ncols > 0 && (ldw & 1))) return SVDSC_ERR_ARG;
    if (ncols > kNoAllocMaxCols) return SVDSC_ERR_SIZE;
    const Chunk ch = make_chunk(len, 2 * 152);
    if (ch.nb > kNoAllocMaxChunks || ch.nbu > kNoAllocMaxNormParts) return SVDSC_ERR_SIZE;
    double *base = nullptr;
    int rc = scratch_address(&base);
    if (rc != SVDSC_OK) return rc;
    double *P = base;
    double *h = base + (size_t)kNoAllocMaxChunks * kNoAllocMaxCols;
    double *Pn = h + kNoAllocMaxCols;
    cudaStream_t s = (cudaStream_t)stream;
    // every scratch element read below is written first in the same call, so
    // nothing left by an earlier call needs clearing
    if (ncols > 0) {
        for (int pass = 0; pass < 2; pass++) {
            proj_partial(W, ldw, (int)ncols, w, ch, P, nullptr, s);
            proj_reduce(P, ch.nb, (int)ncols, h, nullptr, s);
            update_sub(W, ldw, (int)ncols, h, w, ch, pass == 1 ? Pn : nullptr, nullptr, s);
        }
    } else {
        norm_partial(w, ch, Pn, nullptr, s);
    }
    noalloc_norm_kernel<<<1, 256, 0, s>>>(Pn, ch.nbu, norm_out);
    return cudaGetLastError() == cudaSuccess ? SVDSC_OK : SVDSC_ERR_CUDA;
}
