// tcgen05 helpers shared by the kernel translation units (lsw_kernels.cu: the z stage
// and plane kernels; lsw_panels.cu: the H/S products): shared-memory operand layout and
// descriptors, the kind::f16 instruction descriptor, MMA issue and commit, mbarrier waits
// bounded in time, tensor-memory allocation and loads, and the split of FP32 values into
// bfloat16 parts.  Hand-written from the PTX ISA's description of these instructions.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

#include "lsw_device.h"

namespace lsw {

namespace tc {

constexpr int TILE = 128;       // real-space columns per tile (MMA M)
constexpr int HEAD = 512;       // shared header: mbarrier, tensor-memory address, taps
constexpr int TILES_PER_CTA = 16;
constexpr int MAX_KH = 64;      // largest half of K1 = 2 nz rounded up to 16 (nz <= 64)

__device__ __forceinline__ uint32_t saddr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// Byte offset of element (r, k) of an R x K bfloat16 operand in the canonical K-major
// layout without swizzle: core matrices of 8 rows x 16 bytes stored contiguously,
// K-adjacent core matrices 128 bytes apart (leading byte offset), 8-row groups K * 16
// bytes apart (stride byte offset).
__device__ __forceinline__ int core_off(int r, int k, int K) {
    return ((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}
// Shared-memory matrix descriptor of that layout (start address >> 4, leading byte
// offset >> 4 at bit 16, stride byte offset >> 4 at bit 32, descriptor version 1 at
// bit 46, no swizzle).
__device__ __forceinline__ uint64_t sdesc(uint32_t start, int K) {
    return static_cast<uint64_t>((start & 0x3FFFFu) >> 4) | (static_cast<uint64_t>(128 >> 4) << 16) |
           (static_cast<uint64_t>((K * 16) >> 4) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator (bit 4), bfloat16 A and B
// (bits 7, 10), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}
__device__ __forceinline__ void mma(uint32_t d, uint64_t da, uint64_t db, uint32_t id, int acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(da), "l"(db), "r"(id), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// generic-proxy shared-memory writes -> visible to the tensor cores (async proxy)
__device__ __forceinline__ void fence_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_init(uint32_t mbar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ uint64_t gtime() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
// Wait for phase `parity` of the mbarrier; false after about one second.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    const uint64_t t0 = gtime();
    for (int it = 0; it < (1 << 24); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (gtime() - t0 > 1000000000ull) return false;
    }
    return false;
}
__device__ __forceinline__ void tmem_alloc(uint32_t slot, int ncols) {   // one whole warp
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, int ncols) {    // one whole warp
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
// 8 consecutive FP32 columns of this thread's lane; the wait is in the same statement
// so no use of the registers can be scheduled before it.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t q[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(q[i]);
}
// (x0, x1) = sum of NS packed bfloat16 pairs (low half x0's part, high half x1's); each
// part rounds (to nearest) what the previous parts leave, and the subtraction is exact
// in FP32.
template <int NS>
__device__ __forceinline__ void split2(float x0, float x1, uint32_t (&w)[NS]) {
    float r0 = x0, r1 = x1;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const __nv_bfloat162 b = __floats2bfloat162_rn(r0, r1);
        w[i] = *reinterpret_cast<const uint32_t*>(&b);
        if (i + 1 < NS) {
            r0 -= __low2float(b);
            r1 -= __high2float(b);
        }
    }
}
// Split 8 values and store part i as one 16-byte row of a core matrix at
// base + i * part_bytes + off.
template <int NS>
__device__ __forceinline__ void put8(unsigned char* base, int part_bytes, int off, const float (&x)[8],
                                     [[maybe_unused]] int* st, [[maybe_unused]] int64_t room) {
    uint32_t w[4][NS];
#pragma unroll
    for (int e = 0; e < 4; ++e) split2<NS>(x[2 * e], x[2 * e + 1], w[e]);
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const int64_t at = static_cast<int64_t>(i) * part_bytes + off;
#ifdef LSW_CHECKED
        if (off < 0 || off + 16 > part_bytes || at + 16 > room) {
            lsw_report(st, 8, __LINE__, at, room);
            continue;
        }
#endif
        *reinterpret_cast<uint4*>(base + at) = make_uint4(w[0][i], w[1][i], w[2][i], w[3][i]);
    }
}
// Index pairs (part of the data operand, part of the filter operand) of the products.
template <int NS>
struct Terms;
template <>
struct Terms<2> {
    static constexpr int n = 3;
    __device__ static int a(int t) { return t == 2 ? 1 : 0; }
    __device__ static int b(int t) { return t == 1 ? 1 : 0; }
};
template <>
struct Terms<3> {
    static constexpr int n = 6;   // (0,0) (0,1) (1,0) (1,1) (0,2) (2,0)
    __device__ static int a(int t) { return t == 2 || t == 3 ? 1 : (t == 5 ? 2 : 0); }
    __device__ static int b(int t) { return t == 1 || t == 3 ? 1 : (t == 4 ? 2 : 0); }
};

}  // namespace tc

}  // namespace lsw
