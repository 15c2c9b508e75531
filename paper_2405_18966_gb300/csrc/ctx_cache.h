// A small table from CUDA context IDs to device addresses, used by
// svdsc_cgs2_noalloc to remember where its file-scope scratch array lives in
// each context.  A module's __device__ array is placed anew in every context
// that loads the module (after cudaDeviceReset, or in a second context on the
// same device), so the address must be keyed on the context, not on the
// device index.  Context IDs (cuCtxGetId) are unique for the life of the
// process, unlike context handles, which a new context may reuse.
//
// Plain C++ (no CUDA types) so that the keying can be checked on a machine
// without a GPU.  Not thread-safe by itself: the caller holds a lock.
#pragma once
#include <cstdint>

namespace svdsc {

template <int N>
struct CtxAddrCache {
    unsigned long long id[N] = {0};
    void *addr[N] = {nullptr};
    bool used[N] = {false};
    int next = 0;  // slot the next insertion overwrites once all are used

    // Address recorded for context `ctx_id`, or nullptr.
    void *find(unsigned long long ctx_id) const
    {
        for (int i = 0; i < N; i++)
            if (used[i] && id[i] == ctx_id) return addr[i];
        return nullptr;
    }

    // Records (or replaces) the address of context `ctx_id`; with every slot
    // in use, the oldest insertion is dropped.
    void put(unsigned long long ctx_id, void *a)
    {
        for (int i = 0; i < N; i++)
            if (used[i] && id[i] == ctx_id) { addr[i] = a; return; }
        id[next] = ctx_id;
        addr[next] = a;
        used[next] = true;
        next = (next + 1) % N;
    }

    // Forgets every context (the next call in each looks the address up again).
    void clear()
    {
        for (int i = 0; i < N; i++) used[i] = false;
        next = 0;
    }
};

}  // namespace svdsc
