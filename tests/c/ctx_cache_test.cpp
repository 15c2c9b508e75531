// Keying of the per-context address table used by svdsc_cgs2_noalloc
// (csrc/ctx_cache.h): addresses are found by context ID only, a context ID
// seen again after other contexts still finds its own entry, a replaced
// entry returns the new address, and the oldest entry goes when the table is
// full.  Plain C++, no GPU.
#include <cstdio>
#include "ctx_cache.h"

static int fails = 0;
#define CHECK(c)                                                  \
    do {                                                          \
        if (!(c)) { std::printf("FAIL line %d: %s\n", __LINE__, #c); fails++; } \
    } while (0)

int main()
{
    svdsc::CtxAddrCache<4> c;
    int a, b, d, e, f;
    CHECK(c.find(1) == nullptr);
    c.put(1, &a);  // context 1 on device 0
    c.put(2, &b);  // context 2 (a second context on the same device, or after a reset)
    CHECK(c.find(1) == &a);
    CHECK(c.find(2) == &b);
    CHECK(c.find(3) == nullptr);  // a context that never called: looked up afresh
    c.put(2, &d);                 // same context, new address: replaced, not duplicated
    CHECK(c.find(2) == &d);
    c.put(3, &e);
    c.put(4, &f);
    CHECK(c.find(1) == &a && c.find(3) == &e && c.find(4) == &f);
    c.put(5, &a);                 // table full: the oldest insertion (context 1) goes
    CHECK(c.find(1) == nullptr);
    CHECK(c.find(5) == &a && c.find(2) == &d);
    c.clear();
    CHECK(c.find(2) == nullptr && c.find(5) == nullptr);
    std::printf("%s (%d failures)\n", fails ? "FAILED" : "OK", fails);
    return fails ? 1 : 0;
}
