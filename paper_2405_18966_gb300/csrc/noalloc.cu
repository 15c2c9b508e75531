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
#include <cuda.h>  // CUcontext / CUresult types; the two driver calls come from cudaGetDriverEntryPointByVersion
#include "ctx_cache.h"
#include "internal.cuh"

namespace svdsc {

constexpr int64_t kNoAllocMaxCols = 512;   // ncols limit
constexpr int kNoAllocMaxChunks = 1024;    // row chunks of <= 4096 rows: len <= 4,194,304
constexpr int kNoAllocMaxNormParts = 8192; // GEMV-N CTAs of >= 512 rows at that length
constexpr size_t kNoAllocDoubles =
    (size_t)kNoAllocMaxChunks * kNoAllocMaxCols + kNoAllocMaxCols + kNoAllocMaxNormParts;

// 4.3 MB of scratch per context: P (ncols x chunks), h (ncols), Pn (GEMV-N CTAs).
static __device__ __align__(256) double g_cgs2_scratch[kNoAllocDoubles];

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

static std::mutex g_scratch_mu;
static CtxAddrCache<64> g_scratch_addr;  // context ID -> device address of g_cgs2_scratch

static bool driver_calls(CtxGetCurrentFn *cur, CtxGetIdFn *id)
{
    static std::once_flag once;
    static CtxGetCurrentFn f_cur = nullptr;
    static CtxGetIdFn f_id = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            f_cur = (CtxGetCurrentFn)p;
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            f_id = (CtxGetIdFn)p;
    });
    *cur = f_cur;
    *id = f_id;
    return f_cur && f_id;
}

// Device address of the scratch array in the current context.  The array is
// placed anew in every context that loads this module (after a device reset,
// or in a second context on the same device), so the address is cached per
// context ID and looked up (cudaGetSymbolAddress, with that context current)
// the first time a context calls.  That lookup is refused while `s` is being
// captured into a CUDA graph (SVDSC_ERR_ARG): make a context's first call
// outside any capture.
static int scratch_address(cudaStream_t s, double **out)
{
    CtxGetCurrentFn f_cur;
    CtxGetIdFn f_id;
    if (!driver_calls(&f_cur, &f_id)) return SVDSC_ERR_CUDA;
    CUcontext ctx = nullptr;
    if (f_cur(&ctx) != CUDA_SUCCESS) return SVDSC_ERR_CUDA;
    if (!ctx) {  // no context yet: the runtime creates the device's primary context on first use
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_cgs2_scratch) != cudaSuccess || !p) return SVDSC_ERR_CUDA;
        if (f_cur(&ctx) != CUDA_SUCCESS || !ctx) return SVDSC_ERR_CUDA;
    }
    unsigned long long id = 0;
    if (f_id(ctx, &id) != CUDA_SUCCESS) return SVDSC_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    void *p = g_scratch_addr.find(id);
    if (!p) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return SVDSC_ERR_CUDA;
        if (cs != cudaStreamCaptureStatusNone) return SVDSC_ERR_ARG;
        if (cudaGetSymbolAddress(&p, g_cgs2_scratch) != cudaSuccess || !p) return SVDSC_ERR_CUDA;
        g_scratch_addr.put(id, p);
    }
    *out = (double *)p;
    return SVDSC_OK;
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
    cudaStream_t s = (cudaStream_t)stream;
    double *base = nullptr;
    int rc = scratch_address(s, &base);
    if (rc != SVDSC_OK) return rc;
    double *P = base;
    double *h = base + (size_t)kNoAllocMaxChunks * kNoAllocMaxCols;
    double *Pn = h + kNoAllocMaxCols;
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
    norm_from_partials(Pn, ch.nbu, norm_out, s);
    return cudaGetLastError() == cudaSuccess ? SVDSC_OK : SVDSC_ERR_CUDA;
}
