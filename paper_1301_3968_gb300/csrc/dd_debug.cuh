// Bounds checks of the debug build (compiled with -DDD_DEBUG into libdd_debug.so).  A
// failed check records DD_ERR_ARG in the plan's device status word (the first error
// stays; dd_get_device_status reads and clears it) and the caller skips the access it
// guarded, so a bad table shows up as a status code instead of a fault: nothing traps.
// In the normal build every check is the constant true and compiles away.
#pragma once

#include <cstdint>

#include "dd.h"

namespace dd {

#ifdef DD_DEBUG
constexpr bool kDebug = true;
#else
constexpr bool kDebug = false;
#endif

__device__ __forceinline__ bool dbg_ok(bool cond, int32_t* status) {
    if (kDebug && !cond) {
        if (status) atomicCAS(status, 0, (int)DD_ERR_ARG);
        return false;
    }
    return true;
}

}  // namespace dd
