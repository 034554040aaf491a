// Device-side helpers shared by the kernel translation units (lsw_kernels.cu,
// lsw_panels.cu): bounds-checked accesses of the self-checking build.
#pragma once

#include <cstdint>

#include "lsw_internal.h"

namespace lsw {

// Checked accesses: plain loads/stores in the normal build; with -DLSW_CHECKED an
// index outside [0, n) records (kernel, line, block, index, bound) in the status
// block and the access is skipped (a load returns 0).  Never traps, never returns
// early, so barriers stay balanced.
static __device__ __noinline__ void lsw_report(int* st, int kid, int line, int64_t idx, int64_t n) {
    if ((atomicOr(st, ST_BAD_INDEX) & ST_BAD_INDEX) == 0) {
        st[1] = kid;
        st[2] = line;
        st[3] = static_cast<int>(blockIdx.x + 65536u * blockIdx.y);
        reinterpret_cast<long long*>(st + 4)[0] = idx;
        reinterpret_cast<long long*>(st + 4)[1] = n;
    }
}
#ifdef LSW_CHECKED
#define LD(p, i, n) ld_chk(p, static_cast<int64_t>(i), static_cast<int64_t>(n), ST_, KID, __LINE__)
#define ST(p, i, n, v) st_chk(p, static_cast<int64_t>(i), static_cast<int64_t>(n), v, ST_, KID, __LINE__)
#else
#define LD(p, i, n) ((p)[i])
#define ST(p, i, n, v) ((p)[i] = (v))
#endif
template <class T>
__device__ __forceinline__ T ld_chk(const T* p, int64_t i, int64_t n, int* st, int kid, int line) {
    if (i < 0 || i >= n) {
        lsw_report(st, kid, line, i, n);
        return T{};
    }
    return p[i];
}
template <class T, class V>
__device__ __forceinline__ void st_chk(T* p, int64_t i, int64_t n, V v, int* st, int kid, int line) {
    if (i < 0 || i >= n) {
        lsw_report(st, kid, line, i, n);
        return;
    }
    p[i] = static_cast<T>(v);
}

}  // namespace lsw
