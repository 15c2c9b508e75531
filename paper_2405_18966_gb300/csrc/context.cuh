// The solver context (svdsc_ctx) and the host helpers shared by the
// single-vector driver (solver.cu) and the block driver (block_solver.cu):
// per-phase launch accounting with optional CUDA events, column accessors.
#pragma once
#include <algorithm>
#include <cstdint>
#include <vector>
#include <nvtx3/nvToolsExt.h>
#include "internal.cuh"

namespace svdsc {
struct BlockWork;  // block-form workspace (block_solver.cu)
}
using namespace svdsc;

struct StepRec {
    int side;    // 0: u (column of U), 1: v (column of V)
    int col;     // column index created
    int parity;  // anorm parity used by its finalize
};

struct svdsc_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int precision = SVDSC_FP64;
    uint64_t seed = 0;
    int format = SVDSC_CSR;
    int64_t m = 0, n = 0;
    DevCSR A, AT;
    DevDense D;
    double *dense_part = nullptr;
    Chunk cm, cn;
    // workspace sized for t_cap
    int t_cap = 0;
    int64_t ldu = 0, ldv = 0;
    double *U = nullptr, *V = nullptr, *T = nullptr;
    float *U32 = nullptr, *V32 = nullptr;
    // second bases: the tensor-core restart GEMM writes out of place and the
    // two sets swap roles at every restart
    double *Ua = nullptr, *Va = nullptr;
    float *U32a = nullptr, *V32a = nullptr;
    void *gemm_ws = nullptr;
    int restart_gemm = 0;
    int which = 0;  // 0: k largest triplets, 1: k smallest
    int reorth = 0; // 0: CGS2 on every Lanczos vector, 1: partial (estimate-driven)
    double *mu = nullptr, *nu = nullptr;  // partial re-orthogonalization estimates (t + 2 each)
    PrState *pr = nullptr;
    int pr_kk = 0;  // size of the last augmented restart (spike column kk + 1 of T), 0 before
    int block = 1;  // Lanczos block size b (1: the single-vector method)
    BlockWork *bw = nullptr;
    int t_ld = 0;   // leading dimension of T in the block form
    double *P = nullptr, *h = nullptr, *Pn = nullptr;
    double *Sh = nullptr, *Uh = nullptr, *Vh = nullptr, *res = nullptr, *rho = nullptr;
    SvdWork svd;
    DevStatus *st = nullptr;
    DevStatus *st_host = nullptr;  // pinned
    // per-solve state
    int64_t launches = 0;
    int parity = 0;
    int t = 0, k = 0;
    uint64_t draws = 0;
    int breakdowns = 0;
    int64_t n_matvec = 0, n_steps = 0;
    std::vector<StepRec> steps;
    // per-phase accounting (svdsc_info.ms / launches / bytes / flops)
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    struct Rec { int ph, e0, e1; };
    std::vector<Rec> recs;
    int64_t ph_launch[SVDSC_NUM_PHASES] = {0};
    double ph_bytes[SVDSC_NUM_PHASES] = {0};
    double ph_flops[SVDSC_NUM_PHASES] = {0};
};

static inline int next_event(svdsc_ctx *c)
{
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        c->ev_pool.push_back(e);
    }
    return (int)c->ev_used++;
}

// Opens a timed region on the stream (returns -1 when timing is off).
static inline int ph_begin(svdsc_ctx *c)
{
    if (!c->timing) return -1;
    const int e = next_event(c);
    if (e >= 0) cudaEventRecord(c->ev_pool[e], c->stream);
    return e;
}

static inline void ph_end(svdsc_ctx *c, int ph, int e0, int nlaunch, double bytes, double flops)
{
    c->ph_launch[ph] += nlaunch;
    c->ph_bytes[ph] += bytes;
    c->ph_flops[ph] += flops;
    c->launches += nlaunch;
    if (e0 < 0) return;
    const int e1 = next_event(c);
    if (e1 < 0) return;
    cudaEventRecord(c->ev_pool[e1], c->stream);
    c->recs.push_back({ph, e0, e1});
}

static inline void ph_reset(svdsc_ctx *c)
{
    c->ev_used = 0;
    c->recs.clear();
    for (int i = 0; i < SVDSC_NUM_PHASES; i++) {
        c->ph_launch[i] = 0;
        c->ph_bytes[i] = 0.0;
        c->ph_flops[i] = 0.0;
    }
}

#define CU(x)                                          \
    do {                                               \
        cudaError_t e_ = (x);                          \
        if (e_ != cudaSuccess) return SVDSC_ERR_CUDA;  \
    } while (0)

// Named ranges for Nsight Systems timelines (no-ops unless a tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

static inline double *colU(svdsc_ctx *c, int j) { return c->U + (int64_t)j * c->ldu; }
static inline double *colV(svdsc_ctx *c, int j) { return c->V + (int64_t)j * c->ldv; }
static inline float *colU32(svdsc_ctx *c, int j) { return c->U32 ? c->U32 + (int64_t)j * c->ldu : nullptr; }
static inline float *colV32(svdsc_ctx *c, int j) { return c->V32 ? c->V32 + (int64_t)j * c->ldv : nullptr; }
static inline double *Tent(svdsc_ctx *c, int r, int col) { return c->T + r + (int64_t)col * (c->t + 1); }
static inline int *poison_ptr(svdsc_ctx *c) { return &c->st->poison; }


// solver.cu helpers used by the block form
int read_status(svdsc_ctx *c);
int reserve_ws(svdsc_ctx *c, int t);
int gemm_tc(svdsc_ctx *c, const double *W, const float *W32, int64_t ld, int64_t rows, int t, const double *Q,
            int k, double *C, float *C32);
void cgs2_fp64(svdsc_ctx *c, const double *W, int64_t ld, int ncols, double *w, const Chunk &ch);

namespace svdsc {
// block form (block_solver in block.cu): runs Alg. 2 with blocks of c->block
// columns up to the outputs of the last projected SVD (*Uo, *Vo: the spare
// bases holding U~_k, V~_k before the sign rule)
int solve_block(svdsc_ctx *c, int k, int p, double tol, int maxit, const double *v0, int v0_on_device,
                double **Uo, double **Vo, int *restarts, DevStatus *fin);
void block_free(svdsc_ctx *c);
}  // namespace svdsc
