// debug.cuh -- index checks of the debug build of libprnu.
//
// Compiled with -DPRNU_DEBUG (libprnu_debug.so), PRNU_DCHECK(cond, index)
// evaluates cond in device code; the first check of a translation unit that
// fails records its source line and the offending index in that unit's
// device error word and the caller skips the access (no trap: the context
// stays usable).  prnu_debug_status reads and clears every unit's word.  In
// the release build PRNU_DCHECK is the constant true and costs nothing.
#pragma once

#include <cuda_runtime.h>

namespace prnu {

struct DebugWord {
    int hit;          // 0 until a check fails
    int line;         // source line of the first failed check
    long long index;  // the index it rejected
};
using DebugReader = cudaError_t (*)(DebugWord *out, bool clear);
// host registry of the translation units' readers (prnu_abi.cu)
void debug_register(const char *unit, DebugReader fn);

#ifdef PRNU_DEBUG
namespace {
__device__ DebugWord g_prnu_dbg;

__device__ __forceinline__ bool dcheck(bool ok, int line, long long idx) {
    if (!ok && atomicCAS(&g_prnu_dbg.hit, 0, 1) == 0) {
        g_prnu_dbg.line = line;
        g_prnu_dbg.index = idx;
    }
    return ok;
}

cudaError_t debug_read(DebugWord *out, bool clear) {
    cudaError_t e = cudaMemcpyFromSymbol(out, g_prnu_dbg, sizeof(DebugWord));
    if (e == cudaSuccess && clear) {
        const DebugWord z{0, 0, 0};
        e = cudaMemcpyToSymbol(g_prnu_dbg, &z, sizeof(DebugWord));
    }
    return e;
}

struct DebugReg {
    DebugReg() { debug_register(__BASE_FILE__, debug_read); }
};
DebugReg g_prnu_dbg_reg;
}  // namespace
#define PRNU_DCHECK(cond, idx) (::prnu::dcheck((cond), __LINE__, (long long)(idx)))
#else
#define PRNU_DCHECK(cond, idx) (true)
#endif

}  // namespace prnu
