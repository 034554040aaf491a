// sm_103a kernels of the localized Hamiltonian application and the sparse H/S build.
//
// H phi = L' (T + W^T M^T diag(V) M W) L phi   (Sec. II.A, II.B Eq. phi, III.B)
//
//   k_uncompress  compressed phi on L (segment keys) -> dense 8-type box D (L box)
//   k_fwd_xy      per coarse z plane: synthesis+magic along x then y, i.e. the
//                 combined filters (w*h), (w*g) (u_j = sum_i (w*h)_{j-2i} s_i + ...)
//   k_z           per (x', y') column: the same along z -> real-space u; v = V u
//                 (E_pot += V u^2); then the transposed filters back to coarse z on
//                 the L' box
//   k_kin_z       per (x, y) column of L: kinetic arm along z (T = -1/(2h^2) sum_d
//                 T_{b_d b'_d} along d, Galerkin blocks of the two-level basis) -> G
//   k_bwd_xy      per coarse z plane of L': transposed filters along y then x, plus
//                 the kinetic arms along x and y, plus G; written straight into the
//                 compressed H phi on the members of L'; E_kin partials
// (the sparse S_ab, H_ab build is in lsw_panels.cu)
//
// Density rho = sum_ab K_ab phi_a phi_b on the fine grid (Sec. II.A Eq. density):
//   k_z_dens      the forward half of k_z: real-space values u of every function into
//                 a store (after k_uncompress and k_fwd_xy)
//   k_density     per tile of grid points: sum over chunk pairs of the functions whose
//                 blocks meet the tile of K_ab u_a u_b, FP64 total per point
//
// All kernels are templated on the storage/compute type T (double or float); energy
// and matrix accumulations are FP64.  Device-side checks set bits of a status word
// (never trap).
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "lsw_internal.h"
#include "lsw_device.h"
#include "lsw_tc.h"

namespace lsw {

__constant__ double c_fwd_d[2][FWD_TAPS];
__constant__ float c_fwd_f[2][FWD_TAPS];
__constant__ double c_kin_d[4][KIN_TAPS];
__constant__ float c_kin_f[4][KIN_TAPS];
// Tap pairs for the packed (two-lane) FP32 FMA of the blocks below: the two outputs of a
// block that read the same input element, side by side.
__constant__ float2 c_fwd2_bwd[FWD_TAPS];          // (F_0[m], F_1[m])
__constant__ float2 c_fwd2_up[2][16];              // (F_b[2k], F_b[2k+1]), F_b[31] = 0
__constant__ float2 c_kin2[2][KIN_TAPS];           // (K_0(l), K_2(l)), (K_1(l), K_3(l))

template <class T>
struct Tab;
template <>
struct Tab<double> {
    __device__ static __forceinline__ double fwd(int b, int m) { return c_fwd_d[b][m]; }
    __device__ static __forceinline__ double kin(int k, int l) { return c_kin_d[k][l]; }
};
template <>
struct Tab<float> {
    __device__ static __forceinline__ float fwd(int b, int m) { return c_fwd_f[b][m]; }
    __device__ static __forceinline__ float kin(int k, int l) { return c_kin_f[k][l]; }
};

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

#define FWD(b, m) Tab<T>::fwd(b, m)
#ifdef LSW_CHECKED
#undef FWD
#define FWD(b, m) (((m) >= 0 && (m) < FWD_TAPS) ? Tab<T>::fwd(b, m) : (lsw_report(ST_, KID, __LINE__, (m), FWD_TAPS), T(0)))
#endif

// Element copy global -> shared without a register round trip (cp.async, 4 or 8 bytes):
// a staging loop issues all its copies back to back, so every load of a plane is in
// flight at once; cp_wait() completes this thread's copies (a barrier then publishes
// them to the block).  The checked build copies through the bounds-checked accessors.
#ifdef LSW_CHECKED
#define CPA(dst, di, dn, src, si, sn) ST(dst, di, dn, LD(src, si, sn))
#else
#define CPA(dst, di, dn, src, si, sn) cp_async(&(dst)[di], &(src)[si])
#endif
template <class T>
__device__ __forceinline__ void cp_async(T* dst, const T* src) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "cp.async element of 4 or 8 bytes");
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N committed groups of this thread's copies are still in flight
template <int N>
__device__ __forceinline__ void cp_wait_group() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// ---------------------------------------------------------------- uncompress / compress

template <class T>
__global__ void __launch_bounds__(256) k_uncompress(HphiLaunch a) {
    // Warp per (y, z) row of the L box: writes all 8 types of the row, the members' values
    // from the compressed phi (one coarse segment per row of the sphere, a few fine
    // segments) and zero elsewhere, so the box needs no separate clearing.
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = 1;
    const FnRec r = a.fn[blockIdx.y];
    const AtomRec& at = a.atoms[r.atom];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nx = r.n[0], nrows = r.n[1] * r.n[2];
    const int row = blockIdx.x * (blockDim.x >> 5) + warp;
    if (row >= nrows) return;
    const int64_t plane = static_cast<int64_t>(nx) * nrows;
    T* D = static_cast<T*>(a.ws) + r.ws_D + static_cast<int64_t>(row) * nx;
    const T* phi = static_cast<const T*>(a.phi) + r.off_phi;
    const int64_t phi_room = a.phi_n - r.off_phi;
    const int c0 = LD(a.rowptr, at.rowLc + row, a.rowptr_n), c1 = LD(a.rowptr, at.rowLc + row + 1, a.rowptr_n);
    const int f0 = LD(a.rowptr, at.rowLf + row, a.rowptr_n), f1 = LD(a.rowptr, at.rowLf + row + 1, a.rowptr_n);
    Seg cs{};
    cs.x0 = 1;
    cs.x1 = 0;                                         // empty unless the row has members
    if (c1 > c0) {
        cs = LD(a.seg, at.segLc + c0, a.seg_n);
        if (c1 - c0 > 1 || cs.x0 < 0 || cs.x1 >= nx || cs.row != row) {
            if (lane == 0) atomicOr(a.status, ST_BAD_SEG);
            return;
        }
    }
    for (int x = lane; x < nx; x += 32) {
        ST(D, x, 8 * plane - static_cast<int64_t>(row) * nx,
           (x >= cs.x0 && x <= cs.x1) ? LD(phi, cs.off + (x - cs.x0), phi_room) : T(0));
        // wavelet types: the fine segment of this row holding x, if any
        int64_t fo = -1;
        for (int q = f0; q < f1; ++q) {
            const Seg fs = LD(a.seg, at.segLf + q, a.seg_n);
            if (x >= fs.x0 && x <= fs.x1) fo = fs.off + (x - fs.x0);
        }
#pragma unroll
        for (int t = 1; t < 8; ++t)
            ST(D, t * plane + x, 8 * plane - static_cast<int64_t>(row) * nx,
               fo >= 0 ? LD(phi, at.ncL + static_cast<int64_t>(t - 1) * at.nfL + fo, phi_room) : T(0));
    }
}

// Division by a loop-invariant divisor d (1 <= d < 2^16) for dividends n < 2^16:
// q = umulhi(n, ceil(2^32 / d)) is exact there (the error term n / 2^32 < 2^-16 cannot
// reach the next integer).  Replaces the ~20-instruction integer division in index math.
struct FastDiv {
    uint32_t m;
    int d;
    __device__ __forceinline__ explicit FastDiv(int dd) : m(dd > 1 ? 0xFFFFFFFFu / static_cast<uint32_t>(dd) + 1u : 0u), d(dd) {}
    __device__ __forceinline__ int div(int n) const {
        return d > 1 ? static_cast<int>(__umulhi(static_cast<uint32_t>(n), m)) : n;
    }
};

// ---------------------------------------------------------------- register-blocked 1D blocks
//
// Forward (synthesis + magic filter, upsampling by 2): u[2p+e] = sum_{k} F_b[2k+e] in_b[p-k],
// k = 0..15 (e = 0) or 0..14 (e = 1), summed over the two input types b (s and d).  A
// block produces the 8 outputs 2p0 .. 2p0+7 from the window in_b[p0-15 .. p0+3] (19
// values per type) held in registers; taps are compile-time immediates.
constexpr int FB = 4;                 // coarse steps per forward block (8 outputs)
constexpr int FW = FB + 15;           // forward window
constexpr int BB = 4;                 // outputs per kinetic block
constexpr int KW = BB + 2 * KIN_HALF; // kinetic window
#ifndef LSW_Z_NB
#define LSW_Z_NB 4                    // outputs per backward block in the z stage (FP32)
#endif
#ifndef LSW_BWD_NB
#define LSW_BWD_NB 8                  // outputs per backward block in the plane kernel (FP32)
#endif
template <class T, int Stage>         // Stage 0: z stage, 1: backward plane kernel
struct Blk {                          // outputs per backward (decimating) block
    static constexpr int NB = sizeof(T) == 4 ? (Stage == 0 ? LSW_Z_NB : LSW_BWD_NB) : 4;
    static constexpr int W = 2 * NB + 29;
};
template <class T>
struct ZCols { static constexpr int C = sizeof(T) == 8 ? ZCOLS_F64 : ZCOLS_F32; };

// Window w[i] = p[off + (first + i) * stride] for positions first + i in [0, n), 0 outside.
// When the whole window is inside (the common, warp-uniform case) the loads carry no
// bounds test.
#ifdef LSW_CHECKED
#define WLD(p, i, room) ld_chk(p, static_cast<int64_t>(i), static_cast<int64_t>(room), st, 11, __LINE__)
#else
#define WLD(p, i, room) ((p)[i])
#endif
template <int N, class T>
__device__ __forceinline__ void win(T (&w)[N], const T* p, int64_t off, int stride, int first, int n,
                                    [[maybe_unused]] int64_t room, [[maybe_unused]] int* st) {
    if (first >= 0 && first + N <= n) {
        const T* q = p + off + static_cast<int64_t>(first) * stride;
#pragma unroll
        for (int i = 0; i < N; ++i) w[i] = WLD(q, static_cast<int64_t>(i) * stride, room - off - static_cast<int64_t>(first) * stride);
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const int pos = first + i;
            w[i] = (pos >= 0 && pos < n) ? WLD(p, off + static_cast<int64_t>(pos) * stride, room) : T(0);
        }
    }
}

// The same for a window in shared memory, with 32-bit offsets (shared addresses are
// 32-bit; keeping the index math in int lets loads fold their offsets).
template <int N, class T>
__device__ __forceinline__ void swin(T (&w)[N], const T* p, int off, int stride, int first, int n,
                                     [[maybe_unused]] int64_t room, [[maybe_unused]] int* st) {
    if (first >= 0 && first + N <= n) {
        const int b = off + first * stride;
#pragma unroll
        for (int i = 0; i < N; ++i) w[i] = WLD(p, b + i * stride, room);
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const int pos = first + i;
            w[i] = (pos >= 0 && pos < n) ? WLD(p, off + pos * stride, room) : T(0);
        }
    }
}

template <class T>
__device__ __forceinline__ void fwd_block(const T (&w0)[FW], const T (&w1)[FW], T (&u)[2 * FB]) {
#pragma unroll
    for (int j = 0; j < FB; ++j) {
        T ue = 0, uo = 0;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            ue += Tab<T>::fwd(0, 2 * k) * w0[j + 15 - k];
            ue += Tab<T>::fwd(1, 2 * k) * w1[j + 15 - k];
            if (k < 15) {
                uo += Tab<T>::fwd(0, 2 * k + 1) * w0[j + 15 - k];
                uo += Tab<T>::fwd(1, 2 * k + 1) * w1[j + 15 - k];
            }
        }
        u[2 * j] = ue;
        u[2 * j + 1] = uo;
    }
}

// Backward (transposed filters, decimation by 2): s_j = sum_m F_0[m] v[2j+m],
// d_j = sum_m F_1[m] v[2j+m], m = 0..30, from the window v[0 .. 2*NB+28].
template <class T, int NB>
__device__ __forceinline__ void bwd_block(const T (&w)[2 * NB + 29], T (&s)[NB], T (&d)[NB]) {
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        T a0 = 0, a1 = 0;
#pragma unroll
        for (int m = 0; m < FWD_TAPS; ++m) {
            a0 += Tab<T>::fwd(0, m) * w[2 * j + m];
            a1 += Tab<T>::fwd(1, m) * w[2 * j + m];
        }
        s[j] = a0;
        d[j] = a1;
    }
}

// Kinetic arm along one axis for the two types of a pair differing in that axis' bit:
// out_o[j] += sum_l K_{o,0}(l) in_0[j+14+l] + K_{o,1}(l) in_1[j+14+l], o = 0, 1.
template <class T>
__device__ __forceinline__ void kin_block(const T (&k0)[KW], const T (&k1)[KW], T (&o0)[BB], T (&o1)[BB]) {
#pragma unroll
    for (int j = 0; j < BB; ++j) {
        T a0 = 0, a1 = 0;
#pragma unroll
        for (int l = 0; l < KIN_TAPS; ++l) {
            a0 += Tab<T>::kin(0, l) * k0[j + l];
            a0 += Tab<T>::kin(1, l) * k1[j + l];
            a1 += Tab<T>::kin(2, l) * k0[j + l];
            a1 += Tab<T>::kin(3, l) * k1[j + l];
        }
        o0[j] = a0;
        o1[j] = a1;
    }
}

// FP32 versions on the packed two-lane FMA (__ffma2_rn: each lane one FMA rounded to
// nearest, so every accumulator sees the same operations in the same order as above and
// the results are the same bits).  The two lanes are the two outputs of a block that read
// the same input element.
#ifndef LSW_FFMA2
#define LSW_FFMA2 1
#endif
#if LSW_FFMA2
template <>
__device__ __forceinline__ void fwd_block<float>(const float (&w0)[FW], const float (&w1)[FW], float (&u)[2 * FB]) {
#pragma unroll
    for (int j = 0; j < FB; ++j) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float a = w0[j + 15 - k], b = w1[j + 15 - k];
            acc = __ffma2_rn(c_fwd2_up[0][k], make_float2(a, a), acc);
            acc = __ffma2_rn(c_fwd2_up[1][k], make_float2(b, b), acc);
        }
        u[2 * j] = acc.x;
        u[2 * j + 1] = acc.y;
    }
}
// The tap loop outside, the NB independent accumulators inside: each accumulator sees the
// same operations in the same order (same bits), and consecutive instructions belong to
// different dependency chains.
template <int NB>
__device__ __forceinline__ void bwd_block_f2(const float (&w)[2 * NB + 29], float (&s)[NB], float (&d)[NB]) {
    float2 acc[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) acc[j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 0; m < FWD_TAPS; ++m) {
        const float2 t = c_fwd2_bwd[m];
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const float a = w[2 * j + m];
            acc[j] = __ffma2_rn(t, make_float2(a, a), acc[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        s[j] = acc[j].x;
        d[j] = acc[j].y;
    }
}
template <>
__device__ __forceinline__ void bwd_block<float, 4>(const float (&w)[37], float (&s)[4], float (&d)[4]) {
    bwd_block_f2<4>(w, s, d);
}
template <>
__device__ __forceinline__ void bwd_block<float, 8>(const float (&w)[45], float (&s)[8], float (&d)[8]) {
    bwd_block_f2<8>(w, s, d);
}
template <>
__device__ __forceinline__ void kin_block<float>(const float (&k0)[KW], const float (&k1)[KW], float (&o0)[BB],
                                                 float (&o1)[BB]) {
    float2 acc[BB];
#pragma unroll
    for (int j = 0; j < BB; ++j) acc[j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int l = 0; l < KIN_TAPS; ++l) {
        const float2 t0 = c_kin2[0][l], t1 = c_kin2[1][l];
#pragma unroll
        for (int j = 0; j < BB; ++j) {
            const float a = k0[j + l], b = k1[j + l];
            acc[j] = __ffma2_rn(t0, make_float2(a, a), acc[j]);
            acc[j] = __ffma2_rn(t1, make_float2(b, b), acc[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < BB; ++j) {
        o0[j] = acc[j].x;
        o1[j] = acc[j].y;
    }
}
#endif

// ---------------------------------------------------------------- forward x, y

template <class T>
__device__ __forceinline__ void fwd_plane(const HphiLaunch& a, int fl, int z, int bz) {
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = 2;
    int* st = a.status;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const FnRec r = a.fn[fl];
    if (z >= r.n[2]) return;
    const int nx = r.n[0], ny = r.n[1], nz = r.n[2];
    const int X = 2 * nx + 29, Y = 2 * ny + 29;
    const int RS = nx | 1;                   // odd row stride: rows land in different banks
    T* in = sm;                              // [4][ny][RS], type tb = bx + 2 by
    T* mid = sm + 4 * ny * RS;               // [2][ny][X]
    const int64_t smem_n = static_cast<int64_t>(a.smem_fwd / sizeof(T));
    const int64_t mid_n = smem_n - 4 * ny * RS;
    const T* D = static_cast<const T*>(a.ws) + r.ws_D;
    const int64_t plane = static_cast<int64_t>(nx) * ny * nz;
    const int pn = nx * ny;
    {
        const FastDiv fd_pn(pn), fd_nx(nx);
        for (int i = threadIdx.x; i < 4 * pn; i += blockDim.x) {
            const int tb = fd_pn.div(i), rem = i - tb * pn;
            const int y = fd_nx.div(rem), x = rem - y * nx;
            CPA(in, (tb * ny + y) * RS + x, smem_n, D, (tb + 4 * bz) * plane + static_cast<int64_t>(z) * pn + rem,
                8 * plane);
        }
    }
    // x pass work list.  Row (by, y) holds the types (bz, by, 0), (bz, by, 1) of D, which are
    // zero off L's members in the row: the coarse segment where the pair holds type 0
    // (bz = 0, by = 0), else the fine segments.  Block blk (inputs x = 4 blk - 15 ..
    // 4 blk + 3) is computed for the rows whose nonzero range meets its window; per (by,
    // blk) the hull of those rows is listed (block-major, consecutive rows on consecutive
    // threads), and the rest of mid is zero.
    const int nbx = (nx + 15 + FB - 1) / FB;
    __shared__ int16_t ix0[2][256], ix1[2][256];
    __shared__ int hlo[128], hhi[128], hp[129];
    const bool listed = a.fwd_list && 2 * nbx <= 128 && ny <= 256;   // else every (row, block)
    if (listed) {
        const AtomRec& at = a.atoms[r.atom];
        for (int y = threadIdx.x; y < ny; y += blockDim.x) {
            const int64_t crow = at.rowLc + y + static_cast<int64_t>(ny) * z;
            const int64_t frow = at.rowLf + y + static_cast<int64_t>(ny) * z;
            const int c0 = LD(a.rowptr, crow, a.rowptr_n), c1 = LD(a.rowptr, crow + 1, a.rowptr_n);
            const int q0 = LD(a.rowptr, frow, a.rowptr_n), q1 = LD(a.rowptr, frow + 1, a.rowptr_n);
            const int cx0 = c1 > c0 ? LD(a.seg, at.segLc + c0, a.seg_n).x0 : -1;
            const int cx1 = c1 > c0 ? LD(a.seg, at.segLc + c1 - 1, a.seg_n).x1 : -1;
            const int fx0 = q1 > q0 ? LD(a.seg, at.segLf + q0, a.seg_n).x0 : -1;
            const int fx1 = q1 > q0 ? LD(a.seg, at.segLf + q1 - 1, a.seg_n).x1 : -1;
            ix0[0][y] = static_cast<int16_t>(bz == 0 ? cx0 : fx0);
            ix1[0][y] = static_cast<int16_t>(bz == 0 ? cx1 : fx1);
            ix0[1][y] = static_cast<int16_t>(fx0);
            ix1[1][y] = static_cast<int16_t>(fx1);
        }
        for (int e = threadIdx.x; e < 2 * nbx; e += blockDim.x) {
            hlo[e] = ny;
            hhi[e] = -1;
        }
        for (int i = threadIdx.x; i < 2 * ny * X; i += blockDim.x) ST(mid, i, mid_n, T(0));
    }
    __syncthreads();
    if (listed) {
        for (int row = threadIdx.x; row < 2 * ny; row += blockDim.x) {
            const int by = row >= ny, y = row - by * ny;
            const int x0 = ix0[by][y];
            if (x0 < 0) continue;
            const int k1 = min(nbx - 1, (ix1[by][y] + 15) / FB);
            for (int k = x0 / FB; k <= k1; ++k) {
                atomicMin(&hlo[by * nbx + k], y);
                atomicMax(&hhi[by * nbx + k], y);
            }
        }
    }
    cp_wait();
    __syncthreads();
    if (listed && threadIdx.x == 0) {
        hp[0] = 0;
        for (int e = 0; e < 2 * nbx; ++e) hp[e + 1] = hp[e] + max(0, hhi[e] - hlo[e] + 1);
    }
    __syncthreads();
    // x pass: rows (by, y), blocks of 8 outputs along x'
    {
        const FastDiv fd_2ny(2 * ny), fd_ny(ny);
        const int ntk = listed ? hp[2 * nbx] : 2 * ny * nbx;
        for (int task = threadIdx.x; task < ntk; task += blockDim.x) {
            int by, y, blk;
            if (listed) {
                int lo = 0, hi = 2 * nbx - 1;              // the entry e with hp[e] <= task < hp[e + 1]
                while (lo < hi) {
                    const int m = (lo + hi + 1) >> 1;
                    if (hp[m] <= task) lo = m;
                    else hi = m - 1;
                }
                by = lo >= nbx;
                blk = lo - by * nbx;
                y = hlo[lo] + (task - hp[lo]);
            } else {
                blk = fd_2ny.div(task);
                const int rw = task - blk * 2 * ny;
                by = fd_ny.div(rw);
                y = rw - by * ny;
            }
            const int row = by * ny + y;
            const int p0 = blk * FB;
            const int s0 = ((2 * by) * ny + y) * RS, d0 = s0 + ny * RS;
            T w0[FW], w1[FW], u[2 * FB];
            swin(w0, in, s0, 1, p0 - 15, nx, smem_n, st);
            swin(w1, in, d0, 1, p0 - 15, nx, smem_n, st);
            fwd_block(w0, w1, u);
#pragma unroll
            for (int k = 0; k < 2 * FB; ++k) {
                const int xo = 2 * p0 + k;
                if (xo < X) ST(mid, row * X + xo, mid_n, u[k]);
            }
        }
    }
    __syncthreads();
    // y pass: columns x', blocks of 8 outputs along y'
    T* Bf = static_cast<T*>(a.ws) + r.ws_Bf + (static_cast<int64_t>(bz) * nz + z) * Y * X;
    const int64_t bf_room = 2LL * nz * Y * X - (static_cast<int64_t>(bz) * nz + z) * Y * X;
    const int nby = (ny + 15 + FB - 1) / FB;
    const FastDiv fd_X(X);
    for (int task = threadIdx.x; task < X * nby; task += blockDim.x) {
        const int blk = fd_X.div(task), xo = task - blk * X;
        const int p0 = blk * FB;
        T w0[FW], w1[FW], u[2 * FB];
        swin(w0, mid, xo, X, p0 - 15, ny, mid_n, st);
        swin(w1, mid, ny * X + xo, X, p0 - 15, ny, mid_n, st);
        fwd_block(w0, w1, u);
#pragma unroll
        for (int k = 0; k < 2 * FB; ++k) {
            const int yo = 2 * p0 + k;
            if (yo < Y) ST(Bf, static_cast<int64_t>(yo) * X + xo, bf_room, u[k]);
        }
    }
}

// Item k of a persistent plane kernel: the next index of the queue counter (one atomic per
// CTA, broadcast through shared memory), so CTAs take the batch's planes largest first
// as they free up.  The caller's next barrier orders the read before the next write.
__device__ __forceinline__ int next_item(int* counter, int* s_item) {
    if (threadIdx.x == 0) *s_item = atomicAdd(counter, 1);
    __syncthreads();
    return *s_item;
}

// Persistent form (a.items_fwd set): a grid of as many CTAs as fit on the GPU loops over
// the batch's (function, z plane, z type) items; otherwise one CTA per grid slot
// (blockIdx.x = 2 z + b_z, blockIdx.y = function).
template <class T>
__global__ void __launch_bounds__(256) k_fwd_xy(HphiLaunch a) {
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = 2;
    if (a.items_fwd) {
        __shared__ int s_item;
        for (;;) {
            const int k = next_item(a.queue, &s_item);
            if (k >= a.n_items_fwd) break;
            const int code = LD(a.items_fwd, k, a.n_items_fwd);
            fwd_plane<T>(a, code >> 11, (code >> 1) & 1023, code & 1);
            __syncthreads();   // shared memory and s_item are reused by the next item
        }
    } else {
        fwd_plane<T>(a, blockIdx.y, blockIdx.x >> 1, blockIdx.x & 1);
    }
}

// ---------------------------------------------------------------- z stage with V

template <class T>
__global__ void __launch_bounds__(ZCols<T>::C) k_z(HphiLaunch a) {
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = 3;
    constexpr int NB = Blk<T, 0>::NB;
    constexpr int W = Blk<T, 0>::W;
    constexpr int C = ZCols<T>::C;       // columns per block = threads; a compile-time
                                         // stride turns window offsets into immediates
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const FnRec r = a.fn[blockIdx.y];
    const int nx = r.n[0], ny = r.n[1], nz = r.n[2];
    const int X = 2 * nx + 29, Y = 2 * ny + 29, Z = 2 * nz + 29;
    const int cols = X * Y;
    const int c = blockIdx.x * C + threadIdx.x;
    if (blockIdx.x * C >= cols) return;
    const bool valid = c < cols;
    const int t = threadIdx.x;
    T* cin = sm;                  // [2][nz][C]  (each thread owns its column)
    T* vs = sm + 2 * nz * C;      // [Z][C]
    [[maybe_unused]] const int64_t smem_n = static_cast<int64_t>(a.smem_z / sizeof(T));
    [[maybe_unused]] const int64_t vs_n = smem_n - 2 * nz * C;
    const T* Bf = static_cast<const T*>(a.ws) + r.ws_Bf;
    T epot_t = 0;   // per-thread partial in the kernel's precision (no FP64 in FP32 loops)
    if (valid) {
        // Stage the column's input and its slice of V first: all loads independent and
        // in flight together (the multiply below then reads V from shared memory).
        const int xo = c % X, yo = c / X;
        const int64_t jx = 2LL * r.lo[0] - V_REACH + xo - a.vlo[0];
        const int64_t jy = 2LL * r.lo[1] - V_REACH + yo - a.vlo[1];
        const int64_t jz0 = 2LL * r.lo[2] - V_REACH - a.vlo[2];
        const T* V = static_cast<const T*>(a.V);
        const int64_t vrow = jy * a.vn[0] + jx;
        const int64_t vstride = a.vn[0] * a.vn[1];
        for (int q = 0; q < 2 * nz; ++q)
            CPA(cin, q * C + t, smem_n, Bf, static_cast<int64_t>(q) * cols + c, 2LL * nz * cols);
        for (int zo = 0; zo < Z; ++zo)
            CPA(vs, zo * C + t, vs_n, V, (jz0 + zo) * vstride + vrow, a.v_n);
        cp_wait();   // each thread reads only its own column: no barrier needed
        for (int p0 = 0; 2 * p0 < Z; p0 += FB) {
            T w0[FW], w1[FW], u[2 * FB];
            const int q0 = p0 - 15;
            if (q0 >= 0 && q0 + FW <= nz) {
#pragma unroll
                for (int i = 0; i < FW; ++i) {
                    w0[i] = LD(cin, (q0 + i) * C + t, smem_n);
                    w1[i] = LD(cin, (nz + q0 + i) * C + t, smem_n);
                }
            } else {
#pragma unroll
                for (int i = 0; i < FW; ++i) {
                    const int q = q0 + i;
                    const bool ok = q >= 0 && q < nz;
                    w0[i] = ok ? LD(cin, q * C + t, smem_n) : T(0);
                    w1[i] = ok ? LD(cin, (nz + q) * C + t, smem_n) : T(0);
                }
            }
            fwd_block(w0, w1, u);
#pragma unroll
            for (int k = 0; k < 2 * FB; ++k) {
                const int zo = 2 * p0 + k;
                if (zo < Z) {
                    const T vv = LD(vs, zo * C + t, vs_n);
                    const T v = vv * u[k];
                    epot_t += v * u[k];
                    ST(vs, zo * C + t, vs_n, v);
                }
            }
        }
        const int nzp = r.np[2];
        const int dz = r.lop[2] - r.lo[2];
        T* Bb = static_cast<T*>(a.ws) + r.ws_Bb;
        for (int b0 = 0; b0 < nzp; b0 += NB) {
            T w[W], s[NB], d[NB];
            const int z0 = 2 * (b0 + dz);
            if (z0 >= 0 && z0 + W <= Z) {
#pragma unroll
                for (int i = 0; i < W; ++i) w[i] = LD(vs, (z0 + i) * C + t, vs_n);
            } else {
#pragma unroll
                for (int i = 0; i < W; ++i) {
                    const int zo = z0 + i;
                    w[i] = (zo >= 0 && zo < Z) ? LD(vs, zo * C + t, vs_n) : T(0);
                }
            }
            bwd_block<T, NB>(w, s, d);
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                const int b = b0 + j;
                if (b < nzp) {
                    ST(Bb, static_cast<int64_t>(b) * cols + c, 2LL * nzp * cols, s[j]);
                    ST(Bb, static_cast<int64_t>(nzp + b) * cols + c, 2LL * nzp * cols, d[j]);
                }
            }
        }
    }
    const double epot = warp_sum(static_cast<double>(epot_t));
    if ((threadIdx.x & 31) == 0 && epot != 0.0) atomicAdd(a.e_pot + r.f, epot);
}

// ---------------------------------------------------------------- density: real-space values

// The forward half of k_z for the density (Eq. density): per (x', y') column, synthesis +
// magic filter along z, and the real-space values u written to the function's block of
// the density store (no potential, no backward pass).
template <class T>
__global__ void __launch_bounds__(ZCols<T>::C) k_z_dens(HphiLaunch a) {
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = 12;
    constexpr int C = ZCols<T>::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* cin = reinterpret_cast<T*>(smem_raw);   // [2][nz][C] (each thread owns its column)
    const FnRec r = a.fn[blockIdx.y];
    const int nx = r.n[0], ny = r.n[1], nz = r.n[2];
    const int X = 2 * nx + 29, Y = 2 * ny + 29, Z = 2 * nz + 29;
    const int cols = X * Y;
    const int c = blockIdx.x * C + threadIdx.x;
    if (c >= cols) return;   // no barrier below: threads leave independently
    const int t = threadIdx.x;
    [[maybe_unused]] const int64_t smem_n = static_cast<int64_t>(a.smem_z / sizeof(T));
    const T* Bf = static_cast<const T*>(a.ws) + r.ws_Bf;
    const DensFn df = a.dfn[r.f];
    T* U = static_cast<T*>(a.U) + df.off;
    [[maybe_unused]] const int64_t room = a.U_n - df.off;
    for (int q = 0; q < 2 * nz; ++q)
        CPA(cin, q * C + t, smem_n, Bf, static_cast<int64_t>(q) * cols + c, 2LL * nz * cols);
    cp_wait();
    for (int p0 = 0; 2 * p0 < Z; p0 += FB) {
        T w0[FW], w1[FW], u[2 * FB];
        const int q0 = p0 - 15;
#pragma unroll
        for (int i = 0; i < FW; ++i) {
            const int q = q0 + i;
            const bool ok = q >= 0 && q < nz;
            w0[i] = ok ? LD(cin, q * C + t, smem_n) : T(0);
            w1[i] = ok ? LD(cin, (nz + q) * C + t, smem_n) : T(0);
        }
        fwd_block(w0, w1, u);
#pragma unroll
        for (int k = 0; k < 2 * FB; ++k) {
            const int zo = 2 * p0 + k;
            if (zo < Z) ST(U, static_cast<int64_t>(zo) * cols + c, room, u[k]);
        }
    }
}

// ---------------------------------------------------------------- z stage on tensor cores
//
// The z stage of k_z cast as two band-Toeplitz products per tile of 128 real-space
// columns c (the MMA rows, M = 128), with the filter matrices as the N x K operand:
//   U[c][o]  = sum_k A1[c][k] F1[o][k],   k = b nz + q,      F1[o][k] = F_b[o - 2q]
//   v[c][o]  = V(o, c) U[c][o]            (E_pot += v U)
//   Bb[c][j] = sum_o v[c][o] F2[j][o],    j = b' nz' + b,     F2[j][o] = F_b'[o - 2(b + dz)]
// F_b are the combined synthesis + magic filters (w*h), (w*g) of k_z.  Every FP32
// operand x is split into NS bfloat16 parts x = x_0 + x_1 (+ x_2) (each part the
// rounding of what the previous ones leave); the products of parts whose orders add up
// to at most NS - 1 are accumulated in FP32 in tensor memory: NS = 2 takes 3 products
// (relative error of a product about 2^-17), NS = 3 takes 6 (about 2^-24).
//
// One CTA of 8 warps loops over tiles of one function.  Warp w reads tensor-memory
// lanes 32 (w mod 4) .. + 31 (the hardware's lane quarters), so thread (w, lane) owns
// column 32 (w mod 4) + lane of the tile and half w / 4 of each K or N range.  Per tile:
// inputs (prefetched into registers during the previous tile) -> bfloat16 parts in
// shared memory; V of the tile -> shared memory by cp.async; forward MMAs; U from
// tensor memory -> v -> parts; backward MMAs; result from tensor memory -> Bb.  Waits on
// MMA completion are bounded (about 1 s) and end in a status bit, never a hang.

// (the tcgen05 helpers, namespace tc, are in lsw_tc.h)

// Dynamic shared memory of k_z_tc for a function with L extent nz, L' extent nzp
// (host mirror in lsw_host.cpp: ztc_smem).
template <int NS>
__global__ void __launch_bounds__(256, 1) k_z_tc(HphiLaunch a) {
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = 8;
    using tc::TILE;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const FnRec r = a.fn[blockIdx.y];
    const int nx = r.n[0], ny = r.n[1], nz = r.n[2];
    const int X = 2 * nx + 29, Y = 2 * ny + 29, Z = 2 * nz + 29;
    const int cols = X * Y;
    const int ntiles = (cols + TILE - 1) / TILE;
    if (static_cast<int>(blockIdx.x) >= ntiles) return;   // uniform over the CTA
    const int nzp = r.np[2], dz = r.lop[2] - r.lo[2];
    const int K1 = (2 * nz + 15) & ~15, N1 = (Z + 15) & ~15, K2 = N1, N2 = (2 * nzp + 15) & ~15;
    const int KA = max(K1, K2);
    const int A_PART = TILE * KA * 2, B1_PART = N1 * K1 * 2, B2_PART = N2 * K2 * 2;
    unsigned char* sA = smem_raw + tc::HEAD;
    unsigned char* sB1 = sA + NS * A_PART;
    unsigned char* sB2 = sB1 + NS * B1_PART;
    float* sV = reinterpret_cast<float*>(sB2 + NS * B2_PART);   // [Z][TILE]
    const int64_t room = static_cast<int64_t>(a.smem_ztc);
    [[maybe_unused]] const int64_t sv_n = (room - (reinterpret_cast<unsigned char*>(sV) - smem_raw)) / 4;
    int* st = a.status;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = (warp & 3) * 32 + lane;    // tile column = tensor-memory lane
    const int half = warp >> 2;
    const uint32_t mbar = tc::saddr(smem_raw);
    const uint32_t tslot = tc::saddr(smem_raw + 8);
    const int ncols = max(N1, N2) <= 128 ? 128 : 256;
    float* taps = reinterpret_cast<float*>(smem_raw + 16);     // [2][FWD_TAPS]
    if (warp == 0) tc::tmem_alloc(tslot, ncols);
    if (threadIdx.x == 32) tc::mbar_init(mbar);
    if (threadIdx.x >= 64 && threadIdx.x < 64 + 2 * FWD_TAPS) {
        const int i = threadIdx.x - 64;
        taps[i] = Tab<float>::fwd(i / FWD_TAPS, i % FWD_TAPS);
    }
    __syncthreads();

    // filter operands F1 (N1 x K1) and F2 (N2 x K2), zero outside the filter support
    for (int ci = threadIdx.x; ci < N1 * (K1 >> 3); ci += blockDim.x) {
        const int o = ci / (K1 >> 3), k0 = (ci - o * (K1 >> 3)) * 8;
        float x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = k0 + e, b = k >= nz ? 1 : 0, q = k - b * nz, m = o - 2 * q;
            x[e] = (k < 2 * nz && m >= 0 && m < FWD_TAPS) ? taps[b * FWD_TAPS + m] : 0.f;
        }
        tc::put8<NS>(sB1, B1_PART, tc::core_off(o, k0, K1), x, st, room - (sB1 - smem_raw));
    }
    for (int ci = threadIdx.x; ci < N2 * (K2 >> 3); ci += blockDim.x) {
        const int j = ci / (K2 >> 3), o0 = (ci - j * (K2 >> 3)) * 8;
        const int bp = j >= nzp ? 1 : 0, b = j - bp * nzp;
        float x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int o = o0 + e, m = o - 2 * (b + dz);
            x[e] = (j < 2 * nzp && o < Z && m >= 0 && m < FWD_TAPS) ? taps[bp * FWD_TAPS + m] : 0.f;
        }
        tc::put8<NS>(sB2, B2_PART, tc::core_off(j, o0, K2), x, st, room - (sB2 - smem_raw));
    }

    const float* Bf = static_cast<const float*>(a.ws) + r.ws_Bf;
    float* Bb = static_cast<float*>(a.ws) + r.ws_Bb;
    const float* V = static_cast<const float*>(a.V);
    const int64_t vstride = a.vn[0] * a.vn[1];
    const int64_t jz0 = 2LL * r.lo[2] - V_REACH - a.vlo[2];
    const int kh = K1 >> 1, k_lo = half * kh;          // this thread's half of K1
    const int nh1 = N1 >> 1, o_lo = half * nh1;        // its half of N1 (= K2)
    const int nh2 = N2 >> 1, j_lo = half * nh2;        // its half of N2
    float xin[tc::MAX_KH];
    auto load_in = [&](int tile) {
        const int c = tile * TILE + row;
        const bool ok = c < cols;
#pragma unroll
        for (int i0 = 0; i0 < tc::MAX_KH; i0 += 8) {
            if (i0 >= kh) break;            // uniform: whole chunks of 8 past the half are skipped
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int k = k_lo + i0 + e;
                xin[i0 + e] = (ok && k < 2 * nz) ? LD(Bf, static_cast<int64_t>(k) * cols + c, 2LL * nz * cols) : 0.f;
            }
        }
    };
    load_in(blockIdx.x);
    tc::fence_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(smem_raw + 8);
    const uint32_t tlane = tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16);
    uint32_t phase = 0;
    float epot_t = 0.f;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int c = tile * TILE + row;
        const bool valid = c < cols;
        // V(o, c) for o in this thread's half -> sV (cp.async; read back by this thread only)
        if (valid) {
            const int xo = c % X, yo = c / X;
            const int64_t vrow = (2LL * r.lo[1] - V_REACH + yo - a.vlo[1]) * a.vn[0] + (2LL * r.lo[0] - V_REACH + xo - a.vlo[0]);
            const int o1 = min(o_lo + nh1, Z);
#ifdef LSW_CHECKED
            for (int o = o_lo; o < o1; ++o) CPA(sV, o * TILE + row, sv_n, V, (jz0 + o) * vstride + vrow, a.v_n);
#else
            const float* vp = V + (jz0 + o_lo) * vstride + vrow;
            float* sp = sV + o_lo * TILE + row;
#pragma unroll 4
            for (int o = o_lo; o < o1; ++o, vp += vstride, sp += TILE) cp_async(sp, vp);
#endif
        }
        // inputs -> A1 parts (row `row`, k in this thread's half)
#pragma unroll
        for (int i = 0; i < tc::MAX_KH; i += 8) {
            if (i >= kh) break;
            float x[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) x[e] = xin[i + e];
            tc::put8<NS>(sA, A_PART, tc::core_off(row, k_lo + i, K1), x, st, room - (sA - smem_raw));
        }
        tc::fence_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (threadIdx.x == 0) {
            const uint32_t id = tc::idesc(TILE, N1);
            for (int s = 0; s < (K1 >> 4); ++s)
#pragma unroll
                for (int t = 0; t < tc::Terms<NS>::n; ++t)
                    tc::mma(tmem, tc::sdesc(tc::saddr(sA + tc::Terms<NS>::a(t) * A_PART + s * 256), K1),
                            tc::sdesc(tc::saddr(sB1 + tc::Terms<NS>::b(t) * B1_PART + s * 256), K1), id,
                            s > 0 || t > 0);
            tc::commit(mbar);
        }
        if (tile + static_cast<int>(gridDim.x) < ntiles) load_in(tile + gridDim.x);   // prefetch
        bool ok = tc::mbar_wait(mbar, phase);
        phase ^= 1;
        cp_wait();
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) atomicOr(st, ST_WAIT_TIMEOUT);
            break;
        }
        tc::fence_after();
        // U -> v = V U -> A2 parts (row `row`, o in this thread's half of K2 = N1)
        for (int ch = 0; ch < nh1; ch += 8) {
            float u[8], x[8];
            tc::tmem_ld8(tlane + o_lo + ch, u);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int o = o_lo + ch + e;
                const float v = (valid && o < Z) ? LD(sV, o * TILE + row, sv_n) * u[e] : 0.f;
                epot_t += v * u[e];
                x[e] = v;
            }
            tc::put8<NS>(sA, A_PART, tc::core_off(row, o_lo + ch, K2), x, st, room - (sA - smem_raw));
        }
        tc::fence_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (threadIdx.x == 0) {
            const uint32_t id = tc::idesc(TILE, N2);
            for (int s = 0; s < (K2 >> 4); ++s)
#pragma unroll
                for (int t = 0; t < tc::Terms<NS>::n; ++t)
                    tc::mma(tmem, tc::sdesc(tc::saddr(sA + tc::Terms<NS>::a(t) * A_PART + s * 256), K2),
                            tc::sdesc(tc::saddr(sB2 + tc::Terms<NS>::b(t) * B2_PART + s * 256), K2), id,
                            s > 0 || t > 0);
            tc::commit(mbar);
        }
        ok = tc::mbar_wait(mbar, phase);
        phase ^= 1;
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) atomicOr(st, ST_WAIT_TIMEOUT);
            break;
        }
        tc::fence_after();
        // result -> Bb (row j = b' nz' + b of the coarse z output, column c)
        const int j1 = valid ? min(j_lo + nh2, 2 * nzp) : j_lo;    // rows this thread stores
        for (int ch = 0; ch < nh2; ch += 8) {
            float d[8];
            tc::tmem_ld8(tlane + j_lo + ch, d);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int j = j_lo + ch + e;
                if (j < j1) ST(Bb, static_cast<int64_t>(j) * cols + c, 2LL * nzp * cols, d[e]);
            }
        }
        tc::fence_before();
        __syncthreads();   // every read of this tile's tensor memory and V is done
        tc::fence_after();
    }
    const double epot = warp_sum(static_cast<double>(epot_t));
    if (lane == 0 && epot != 0.0) atomicAdd(a.e_pot + r.f, epot);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_free(tmem, ncols);
}

// ---------------------------------------------------------------- forward x, y on tensor cores
//
// k_fwd_xy as two band-Toeplitz tensor-core products per (z, b_z) plane with split-
// bfloat16 operands (NS parts) and FP32 accumulation in tensor memory:
//   M1[y'][i] = sum_k Fy[y'][k] Din[k][i],   k = by n_y + y,  i = bx n_x + q,  Fy[y'][k] = F_by[y' - 2y]
//   U[y'][x'] = sum_i M1[y'][i] Fx[x'][i],   Fx[x'][i] = F_bx[x' - 2q]
// with Din[k][i] = D[bx + 2 by][z][y][q] of this plane; U is the plane of Bf.  Thread
// (warp w, lane l) owns row y' = 32 (w mod 4) + l of both products and half w / 4 of each
// K or N range.  256 threads; the operands take about 90 KB, so two blocks share an SM.
template <int NS>
__global__ void __launch_bounds__(256) k_fwd_xy_tc(HphiLaunch a) {
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = 2;
    int* st = a.status;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const FnRec r = a.fn[blockIdx.y];
    const int z = blockIdx.x >> 1, bz = blockIdx.x & 1;
    if (z >= r.n[2]) return;   // uniform over the CTA, before any allocation
    const int nx = r.n[0], ny = r.n[1], nz = r.n[2];
    const int X = 2 * nx + 29, Y = 2 * ny + 29;
    const int K1 = (2 * ny + 15) & ~15, N1 = (2 * nx + 15) & ~15, K2 = N1, N2 = (X + 15) & ~15;
    const int FY_PART = 128 * K1 * 2, FX_PART = N2 * K2 * 2, P_PART = N1 * K1 * 2, M_PART = 128 * K2 * 2;
    unsigned char* sFy = smem_raw + tc::HEAD;
    unsigned char* sFx = sFy + NS * FY_PART;
    unsigned char* sXr = sFx + NS * FX_PART;
    const int64_t room = static_cast<int64_t>(a.smem_fwd_tc);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = (warp & 3) * 32 + lane, half = warp >> 2;
    const uint32_t mbar = tc::saddr(smem_raw);
    float* taps = reinterpret_cast<float*>(smem_raw + 16);
    if (warp == 0) tc::tmem_alloc(tc::saddr(smem_raw + 8), 128);
    if (threadIdx.x == 32) tc::mbar_init(mbar);
    if (threadIdx.x >= 64 && threadIdx.x < 64 + 2 * FWD_TAPS) {
        const int i = threadIdx.x - 64;
        taps[i] = Tab<float>::fwd(i / FWD_TAPS, i % FWD_TAPS);
    }
    __syncthreads();
    // Fy[y'][k] = F_by[y' - 2y], k = by n_y + y
    for (int ci = threadIdx.x; ci < 128 * (K1 >> 3); ci += blockDim.x) {
        const int yo = ci / (K1 >> 3), k0 = (ci - yo * (K1 >> 3)) * 8;
        float x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = k0 + e, by = k >= ny ? 1 : 0, y = k - by * ny, m = yo - 2 * y;
            x[e] = (yo < Y && k < 2 * ny && m >= 0 && m < FWD_TAPS) ? taps[by * FWD_TAPS + m] : 0.f;
        }
        tc::put8<NS>(sFy, FY_PART, tc::core_off(yo, k0, K1), x, st, room - (sFy - smem_raw));
    }
    // Fx[x'][i] = F_bx[x' - 2q], i = bx n_x + q
    for (int ci = threadIdx.x; ci < N2 * (K2 >> 3); ci += blockDim.x) {
        const int xo = ci / (K2 >> 3), i0 = (ci - xo * (K2 >> 3)) * 8;
        float x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int i = i0 + e, bx = i >= nx ? 1 : 0, q = i - bx * nx, m = xo - 2 * q;
            x[e] = (xo < X && i < 2 * nx && m >= 0 && m < FWD_TAPS) ? taps[bx * FWD_TAPS + m] : 0.f;
        }
        tc::put8<NS>(sFx, FX_PART, tc::core_off(xo, i0, K2), x, st, room - (sFx - smem_raw));
    }
    // Din[k][i] as the N1 x K1 operand (row i, column k); consecutive threads take
    // consecutive q (contiguous in D)
    const float* D = static_cast<const float*>(a.ws) + r.ws_D;
    const int64_t plane = static_cast<int64_t>(nx) * ny * nz;
    for (int ci = threadIdx.x; ci < N1 * (K1 >> 3); ci += blockDim.x) {
        const int c = ci / N1, i = ci - c * N1, k0 = c * 8;
        const int bx = i >= nx ? 1 : 0, q = i - bx * nx;
        float x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = k0 + e, by = k >= ny ? 1 : 0, y = k - by * ny;
            x[e] = (i < 2 * nx && k < 2 * ny)
                       ? LD(D, (bx + 2 * by + 4 * bz) * plane + (static_cast<int64_t>(z) * ny + y) * nx + q, 8 * plane)
                       : 0.f;
        }
        tc::put8<NS>(sXr, P_PART, tc::core_off(i, k0, K1), x, st, room - (sXr - smem_raw));
    }
    tc::fence_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(smem_raw + 8);
    const uint32_t tlane = tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16);
    if (threadIdx.x == 0) {
        const uint32_t id = tc::idesc(128, N1);
        for (int k = 0; k < (K1 >> 4); ++k)
#pragma unroll
            for (int t = 0; t < tc::Terms<NS>::n; ++t)
                tc::mma(tmem, tc::sdesc(tc::saddr(sFy + tc::Terms<NS>::a(t) * FY_PART + k * 256), K1),
                        tc::sdesc(tc::saddr(sXr + tc::Terms<NS>::b(t) * P_PART + k * 256), K1), id, k > 0 || t > 0);
        tc::commit(mbar);
    }
    bool ok = tc::mbar_wait(mbar, 0);
    if (__syncthreads_and(ok)) {
        tc::fence_after();
        for (int c = half; c < (N1 >> 3); c += 2) {
            float u[8];
            tc::tmem_ld8(tlane + c * 8, u);
            tc::put8<NS>(sXr, M_PART, tc::core_off(row, c * 8, K2), u, st, room - (sXr - smem_raw));
        }
        tc::fence_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (threadIdx.x == 0) {
            const uint32_t id = tc::idesc(128, N2);
            for (int k = 0; k < (K2 >> 4); ++k)
#pragma unroll
                for (int t = 0; t < tc::Terms<NS>::n; ++t)
                    tc::mma(tmem, tc::sdesc(tc::saddr(sXr + tc::Terms<NS>::a(t) * M_PART + k * 256), K2),
                            tc::sdesc(tc::saddr(sFx + tc::Terms<NS>::b(t) * FX_PART + k * 256), K2), id,
                            k > 0 || t > 0);
            tc::commit(mbar);
        }
        ok = tc::mbar_wait(mbar, 1);
        if (__syncthreads_and(ok)) {
            tc::fence_after();
            float* Bf = static_cast<float*>(a.ws) + r.ws_Bf + (static_cast<int64_t>(bz) * nz + z) * Y * X;
            [[maybe_unused]] const int64_t bf_room = 2LL * nz * Y * X - (static_cast<int64_t>(bz) * nz + z) * Y * X;
            for (int c = half; c < (N2 >> 3); c += 2) {
                float u[8];
                tc::tmem_ld8(tlane + c * 8, u);
                if (row < Y) {
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        if (c * 8 + e < X) ST(Bf, static_cast<int64_t>(row) * X + c * 8 + e, bf_room, u[e]);
                }
            }
        } else if (threadIdx.x == 0) {
            atomicOr(st, ST_WAIT_TIMEOUT);
        }
    } else if (threadIdx.x == 0) {
        atomicOr(st, ST_WAIT_TIMEOUT);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_free(tmem, 128);
}

// ---------------------------------------------------------------- kinetic z arm

// Per (x, y) column of the L box and type pair (t, t + 4): the kinetic arm along z,
// written to G on the L' box column (G holds only this arm; the backward plane kernel
// adds the rest).  Runs before the backward plane kernel.  The column pair is staged in
// shared memory; a column pair that is zero (outside the L sphere, or wavelet types off
// the fine region) only clears its flag, and the plane kernel then skips its G.
template <class T>
__global__ void __launch_bounds__(128) k_kin_z(HphiLaunch a) {
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = 5;
    int* st = a.status;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const FnRec r = a.fn[blockIdx.y];
    const int nx = r.n[0], ny = r.n[1], nz = r.n[2];
    const int nxp = r.np[0], nyp = r.np[1], nzp = r.np[2];
    const int dx = r.lop[0] - r.lo[0], dy = r.lop[1] - r.lo[1], dz = r.lop[2] - r.lo[2];
    const int pn = nx * ny;
    if (static_cast<int>(blockIdx.x) * 128 >= pn) return;
    const int t = threadIdx.x;
    const int c = blockIdx.x * 128 + t;                    // column (x, y) of the L box
    const int tb = blockIdx.z;                             // type pair (tb, tb + 4)
    T* col = reinterpret_cast<T*>(smem_raw);               // [2][nz][128]: this thread's column pair
    [[maybe_unused]] const int64_t col_n = static_cast<int64_t>(a.smem_kin / sizeof(T));
    unsigned char* flag = reinterpret_cast<unsigned char*>(static_cast<T*>(a.ws) + r.ws_Gf) + tb * pn;
    T ekin_t = 0;
    if (c < pn) {
        const T* D = static_cast<const T*>(a.ws) + r.ws_D;
        const int64_t plane = static_cast<int64_t>(nx) * ny * nz;
        for (int q = 0; q < nz; ++q) {
            CPA(col, q * 128 + t, col_n, D, tb * plane + static_cast<int64_t>(q) * pn + c, 8 * plane);
            CPA(col, (nz + q) * 128 + t, col_n, D, (tb + 4) * plane + static_cast<int64_t>(q) * pn + c, 8 * plane);
        }
        cp_wait();
        bool nonzero = false;
        for (int q = 0; q < 2 * nz; ++q) nonzero |= LD(col, q * 128 + t, col_n) != T(0);
        ST(flag, c, 4LL * pn, nonzero ? 1 : 0);
        const int y = c / nx, x = c - y * nx;
        const int xb = x - dx, yb = y - dy;             // the same column in the L' box
        if (nonzero && xb >= 0 && xb < nxp && yb >= 0 && yb < nyp) {
            T* G = static_cast<T*>(a.ws) + r.ws_G;
            const int64_t gplane = static_cast<int64_t>(nxp) * nyp * nzp;
            const int64_t pnp = static_cast<int64_t>(nxp) * nyp;
            const int64_t gcol = static_cast<int64_t>(yb) * nxp + xb;
            const T ks = static_cast<T>(a.kin_scale);
            // the planes of this column the compressed H phi reads: the coarse members' z
            // range where the pair holds type 0 (tb = 0), else the fine members' z hull (the
            // D values of the pair are zero off those, so E_kin loses no term)
            int zlo = 0, zhi = nzp - 1;
            if (a.colz) {
                const ColZ cz = LD(a.colz, a.atoms[r.atom].colz + gcol, a.colz_n);
                zlo = tb == 0 ? cz.c0 : cz.f0;
                zhi = tb == 0 ? cz.c1 : cz.f1;
            }
            for (int b0 = zlo < 0 ? nzp : (zlo / BB) * BB; b0 <= zhi; b0 += BB) {
                T k0[KW], k1[KW], o0[BB], o1[BB];
                swin(k0, col, t, 128, b0 + dz - KIN_HALF, nz, col_n, st);
                swin(k1, col, nz * 128 + t, 128, b0 + dz - KIN_HALF, nz, col_n, st);
                kin_block(k0, k1, o0, o1);
#pragma unroll
                for (int j = 0; j < BB; ++j) {
                    const int b = b0 + j;
                    if (b < nzp) {
                        o0[j] *= ks;
                        o1[j] *= ks;
                        ST(G, tb * gplane + b * pnp + gcol, 8 * gplane, o0[j]);
                        ST(G, (tb + 4) * gplane + b * pnp + gcol, 8 * gplane, o1[j]);
                        const int zz = b + dz;
                        if (zz >= 0 && zz < nz) ekin_t += k0[KIN_HALF + j] * o0[j] + k1[KIN_HALF + j] * o1[j];
                    }
                }
            }
        }
    }
    const double ekin = warp_sum(static_cast<double>(ekin_t));
    if ((threadIdx.x & 31) == 0 && ekin != 0.0) atomicAdd(a.e_kin + r.f, ekin);
}

// ---------------------------------------------------------------- backward y, x + kinetic x, y + compress

// Per plane (z'', bz) of the L' box: transposed filters along y then x (potential part)
// plus the kinetic arms along x and y of the four output types with z bit bz, plus the
// z arm that k_kin_z left in G; the sum is written straight into the compressed H phi
// on the members of L' in this plane.  Only member rows (and, per row, the x range of
// its member segment: L' is a sphere clipped by the box) are computed; kinetic type
// pairs whose input rows or columns of D are all zero (wavelet types off the fine
// region) are skipped.  Each phase first lists its tasks in shared memory, so skipped
// work frees whole rounds.
constexpr int BWD_MAX_TASKS = 2048;
#ifndef LSW_BWD_MIN_BLOCKS
#define LSW_BWD_MIN_BLOCKS 2      // resident blocks per SM the FP32 version is compiled for
#endif

// Potential part of the backward plane kernel on the tensor cores (the two products
// described at k_bwd_xy): builds the filter operands Fy (128 x K1) and Fx (N2 x K2) and
// the plane operand P (N1 x K1: row x', column y') from Bb, runs both products and writes
// Gs[bx + 2 by][b][b2] for every b < n_y', b2 < n_x'.  512 threads.  Returns false (for
// every thread) if a completion wait ran out.
template <int NS>
__device__ bool bwd_tc_potential(const float* Bb, [[maybe_unused]] int64_t bb_room, int X, int Y, int nyp, int nxp,
                                 int dx, int dy, int K1, int N1, int K2, int N2, int FY_PART, int FX_PART,
                                 [[maybe_unused]] int XR, unsigned char* sFy, unsigned char* sFx, unsigned char* sXr,
                                 float* Gs, unsigned char* smem_raw, int64_t room, int* st) {
    [[maybe_unused]] int* ST_ = st;
    [[maybe_unused]] constexpr int KID = 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = (warp & 3) * 32 + lane, part = warp >> 2;
    const int P_PART = N1 * K1 * 2, M_PART = 128 * K2 * 2;
    const float* taps = reinterpret_cast<const float*>(smem_raw + 16);
    const uint32_t mbar = tc::saddr(smem_raw);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(smem_raw + 8);
    const uint32_t tlane = tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16);
    // Fy[j][y'] = F_by[y' - 2 (b + dy)], j = by n_y' + b
    for (int ci = threadIdx.x; ci < 128 * (K1 >> 3); ci += blockDim.x) {
        const int j = ci / (K1 >> 3), y0 = (ci - j * (K1 >> 3)) * 8;
        const int by = j >= nyp ? 1 : 0, b = j - by * nyp;
        float x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int m = y0 + e - 2 * (b + dy);
            x[e] = (j < 2 * nyp && y0 + e < Y && m >= 0 && m < FWD_TAPS) ? taps[by * FWD_TAPS + m] : 0.f;
        }
        tc::put8<NS>(sFy, FY_PART, tc::core_off(j, y0, K1), x, st, room - (sFy - smem_raw));
    }
    // Fx[i][x'] = F_bx[x' - 2 (b2 + dx)], i = bx n_x' + b2
    for (int ci = threadIdx.x; ci < N2 * (K2 >> 3); ci += blockDim.x) {
        const int i = ci / (K2 >> 3), x0 = (ci - i * (K2 >> 3)) * 8;
        const int bx = i >= nxp ? 1 : 0, b2 = i - bx * nxp;
        float x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int m = x0 + e - 2 * (b2 + dx);
            x[e] = (i < 2 * nxp && x0 + e < X && m >= 0 && m < FWD_TAPS) ? taps[bx * FWD_TAPS + m] : 0.f;
        }
        tc::put8<NS>(sFx, FX_PART, tc::core_off(i, x0, K2), x, st, room - (sFx - smem_raw));
    }
    // P[x'][y'] = Bb plane (y', x'); consecutive threads take consecutive x' (coalesced)
    for (int ci = threadIdx.x; ci < N1 * (K1 >> 3); ci += blockDim.x) {
        const int c = ci / N1, xo = ci - c * N1, y0 = c * 8;
        float x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e)
            x[e] = (xo < X && y0 + e < Y) ? LD(Bb, static_cast<int64_t>(y0 + e) * X + xo, bb_room) : 0.f;
        tc::put8<NS>(sXr, P_PART, tc::core_off(xo, y0, K1), x, st, room - (sXr - smem_raw));
    }
    tc::fence_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (threadIdx.x == 0) {
        const uint32_t id = tc::idesc(128, N1);
        for (int k = 0; k < (K1 >> 4); ++k)
#pragma unroll
            for (int t = 0; t < tc::Terms<NS>::n; ++t)
                tc::mma(tmem, tc::sdesc(tc::saddr(sFy + tc::Terms<NS>::a(t) * FY_PART + k * 256), K1),
                        tc::sdesc(tc::saddr(sXr + tc::Terms<NS>::b(t) * P_PART + k * 256), K1), id, k > 0 || t > 0);
        tc::commit(mbar);
    }
    bool ok = tc::mbar_wait(mbar, 0);
    if (!__syncthreads_and(ok)) return false;
    tc::fence_after();
    // M1 row `row` -> operand of the second product (the P operand is dead)
    for (int c = part; c < (N1 >> 3); c += 4) {
        float u[8];
        tc::tmem_ld8(tlane + c * 8, u);
        tc::put8<NS>(sXr, M_PART, tc::core_off(row, c * 8, K2), u, st, room - (sXr - smem_raw));
    }
    tc::fence_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (threadIdx.x == 0) {
        const uint32_t id = tc::idesc(128, N2);
        for (int k = 0; k < (K2 >> 4); ++k)
#pragma unroll
            for (int t = 0; t < tc::Terms<NS>::n; ++t)
                tc::mma(tmem, tc::sdesc(tc::saddr(sXr + tc::Terms<NS>::a(t) * M_PART + k * 256), K2),
                        tc::sdesc(tc::saddr(sFx + tc::Terms<NS>::b(t) * FX_PART + k * 256), K2), id, k > 0 || t > 0);
        tc::commit(mbar);
    }
    ok = tc::mbar_wait(mbar, 1);
    if (!__syncthreads_and(ok)) return false;
    tc::fence_after();
    // Q row `row` -> Gs (the M1 operand is dead)
    const int by = row >= nyp ? 1 : 0, b = row - by * nyp;
    [[maybe_unused]] const int64_t gs_n = 4LL * nyp * nxp;
    for (int c = part; c < (N2 >> 3); c += 4) {
        float q[8];
        tc::tmem_ld8(tlane + c * 8, q);
        if (row < 2 * nyp) {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int i = c * 8 + e;
                if (i < 2 * nxp) {
                    const int bx = i >= nxp ? 1 : 0, b2 = i - bx * nxp;
                    ST(Gs, ((bx + 2 * by) * nyp + b) * nxp + b2, gs_n, q[e]);
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    return true;
}

// NS = 0: the transposed y and x filters run on the FMA units (256 threads, several
// blocks per SM).  NS = 2, 3 (FP32 only): they run as two band-Toeplitz tensor-core
// products per plane with split-bfloat16 operands (NS parts) and FP32 accumulation in
// tensor memory, as in k_z_tc (512 threads, one block per SM):
//   M1[j][x'] = sum_y' Fy[j][y'] P[y'][x'],   j = by n_y' + b,  Fy[j][y'] = F_by[y' - 2(b + dy)]
//   Q[j][i]   = sum_x' M1[j][x'] Fx[i][x'],   i = bx n_x' + b2, Fx[i][x'] = F_bx[x' - 2(b2 + dx)]
// with P the plane of Bb; thread (warp w, lane l) owns row j = 32 (w mod 4) + l of both
// products and quarter w / 4 of each K or N range.
template <class T, int NS>
__device__ __forceinline__ void bwd_plane(const HphiLaunch& a, int fl, int zb, int bz) {
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = 4;
    int* st = a.status;
    constexpr int NB = Blk<T, 1>::NB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int16_t rx0[256], rx1[256];         // member x range per row (L' plane), -1: none
    __shared__ int roff[256];                      // coefficient offset of the row's coarse segment
    __shared__ int fr0[256], fr1[256];             // fine segment range of the row (L' keys)
    __shared__ int16_t fx0[256], fx1[256];         // hull of the row's fine members, -1: none
    __shared__ int cq0[64], cq1[64], pq[65];       // y pass, per block of NB rows: column range, prefix
    __shared__ int rq0[128], rq1[128], rqp[129];   // kinetic y arm, per (x type, block of BB rows): the same
    __shared__ int ntask, ntask2, ylo, yhi;
    __shared__ unsigned char rowf[4][128], colf[4][128];   // D plane: nonzero per (type, row / column)
    T* sm = reinterpret_cast<T*>(smem_raw);
    const FnRec r = a.fn[fl];
    if (zb >= r.np[2]) return;
    const AtomRec& at = a.atoms[r.atom];
    const int nx = r.n[0], ny = r.n[1], nz = r.n[2];
    const int X = 2 * nx + 29, Y = 2 * ny + 29;
    const int nxp = r.np[0], nyp = r.np[1], nzp = r.np[2];
    const int dx = r.lop[0] - r.lo[0], dy = r.lop[1] - r.lo[1], dz = r.lop[2] - r.lo[2];
    const int RS = nx | 1;
    const int plA = max(Y * X, 4 * nyp * nxp);
    // FMA layout: pl [Y][X] (later Gs [4][nyp][nxp]), mid [2][nyp][X], Dp [4][ny][RS]
    // tensor-core layout: header, Fy parts, Fx parts, a region holding the P operand, then
    // the M1 operand, then Gs; Dp
    const int K1 = (Y + 15) & ~15, N1 = (X + 15) & ~15, K2 = N1, N2 = (2 * nxp + 15) & ~15;
    const int FY_PART = 128 * K1 * 2, FX_PART = N2 * K2 * 2, P_PART = N1 * K1 * 2, M_PART = 128 * K2 * 2;
    const int XR = (max(max(NS * P_PART, NS * M_PART), 16 * nyp * nxp) + 15) & ~15;
    unsigned char* sFy = smem_raw + tc::HEAD;
    unsigned char* sFx = sFy + NS * FY_PART;
    unsigned char* sXr = sFx + NS * FX_PART;
    // task lists of the x pass and the kinetic x arm, later the plane's fine segments for
    // the compressed write: static shared memory in the FMA version; in the tensor-core
    // version the filter operands' region, dead once the potential part is done
    // (NS * FY_PART >= 2 * 128 * 16 * 2 bytes = BWD_MAX_TASKS ints; 16-byte aligned)
    int* task;
    if constexpr (NS == 0) {
        __shared__ __align__(16) int task_s[BWD_MAX_TASKS];
        task = task_s;
    } else {
        task = reinterpret_cast<int*>(sFy);
    }
    T* pl = sm;
    T* Gs = NS ? reinterpret_cast<T*>(sXr) : sm;
    // mid [2][nyp][X], later (when the host found room: a.gstage) the z-arm plane
    const int midA = (NS == 0 && a.gstage) ? max(2 * nyp * X, 4 * nyp * nxp) : 2 * nyp * X;
    T* mid = sm + plA;
    T* Dp = NS ? reinterpret_cast<T*>(sXr + XR) : mid + midA;
    const int64_t smem_n = static_cast<int64_t>((NS ? a.smem_bwd_tc : a.smem_bwd) / sizeof(T));
    if constexpr (NS > 0) {
        if ((threadIdx.x >> 5) == 0) tc::tmem_alloc(tc::saddr(smem_raw + 8), 128);
        if (threadIdx.x == 32) tc::mbar_init(tc::saddr(smem_raw));
        float* taps = reinterpret_cast<float*>(smem_raw + 16);
        if (threadIdx.x >= 64 && threadIdx.x < 64 + 2 * FWD_TAPS) {
            const int i = threadIdx.x - 64;
            taps[i] = Tab<float>::fwd(i / FWD_TAPS, i % FWD_TAPS);
        }
    }
    const int zL = zb + dz;
    const bool dplane = zL >= 0 && zL < nz;
    if (threadIdx.x == 0) {
        ylo = nyp;
        yhi = -1;
    }
    for (int i = threadIdx.x; i < 4 * 128; i += blockDim.x) {
        rowf[i >> 7][i & 127] = 0;
        colf[i >> 7][i & 127] = 0;
    }
    __syncthreads();
    // staging copies first (they fly while the row records below are read): group 1 the
    // Bb plane, group 2 the D plane and the z-arm column flags
    const T* Bb = static_cast<const T*>(a.ws) + r.ws_Bb + (static_cast<int64_t>(bz) * nzp + zb) * Y * X;
    const int64_t bb_room = 2LL * nzp * Y * X - (static_cast<int64_t>(bz) * nzp + zb) * Y * X;
    if constexpr (NS == 0)
        for (int i = threadIdx.x; i < Y * X; i += blockDim.x) CPA(pl, i, smem_n, Bb, i, bb_room);
    cp_commit();
    const T* D = static_cast<const T*>(a.ws) + r.ws_D;
    const int64_t plane = static_cast<int64_t>(nx) * ny * nz;
    const int pn = nx * ny;
    const int64_t dp_n = smem_n - (reinterpret_cast<unsigned char*>(Dp) - smem_raw) / static_cast<int64_t>(sizeof(T));
    if (dplane) {
        const FastDiv fd_pn(pn), fd_nx(nx);
        for (int i = threadIdx.x; i < 4 * pn; i += blockDim.x) {
            const int tb = fd_pn.div(i), rem = i - tb * pn;
            const int y = fd_nx.div(rem), x = rem - y * nx;
            CPA(Dp, (tb * ny + y) * RS + x, dp_n, D, (tb + 4 * bz) * plane + static_cast<int64_t>(zL) * pn + rem,
                8 * plane);
        }
    }
    // z-arm column flags of the L box (written by k_kin_z): staged, 4 bytes per copy, when
    // the host found room (a.gstage), else read from global memory
    const uint32_t* gsrc = reinterpret_cast<const uint32_t*>(static_cast<const T*>(a.ws) + r.ws_Gf);
    uint32_t* gfl = reinterpret_cast<uint32_t*>(Dp + 4 * ny * RS);
    [[maybe_unused]] const int64_t gfl_n = (smem_n * static_cast<int64_t>(sizeof(T)) -
                                            (reinterpret_cast<unsigned char*>(gfl) - smem_raw)) / 4;
    if (a.gstage)
        for (int i = threadIdx.x; i < pn; i += blockDim.x) CPA(gfl, i, gfl_n, gsrc, i, pn);
    cp_commit();
    // member x range of each row of this plane (coarse part of L')
    for (int y = threadIdx.x; y < nyp; y += blockDim.x) {
        const int64_t row = at.rowPc + y + static_cast<int64_t>(nyp) * zb;
        const int s0 = LD(a.rowptr, row, a.rowptr_n), s1 = LD(a.rowptr, row + 1, a.rowptr_n);
        int lo = -1, hi = -1, off = 0;
        if (s1 > s0) {
            const Seg sg = LD(a.seg, at.segPc + s0, a.seg_n);
            lo = sg.x0;
            off = sg.off;
            hi = LD(a.seg, at.segPc + s1 - 1, a.seg_n).x1;
            atomicMin(&ylo, y);
            atomicMax(&yhi, y);
        }
        rx0[y] = static_cast<int16_t>(lo);
        rx1[y] = static_cast<int16_t>(hi);
        roff[y] = off;
        const int64_t frow = at.rowPf + y + static_cast<int64_t>(nyp) * zb;
        const int q0 = LD(a.rowptr, frow, a.rowptr_n), q1 = LD(a.rowptr, frow + 1, a.rowptr_n);
        fr0[y] = q0;
        fr1[y] = q1;
        fx0[y] = static_cast<int16_t>(q1 > q0 ? LD(a.seg, at.segPf + q0, a.seg_n).x0 : -1);
        fx1[y] = static_cast<int16_t>(q1 > q0 ? LD(a.seg, at.segPf + q1 - 1, a.seg_n).x1 : -1);
    }
    cp_wait_group<1>();   // the Bb plane (group 2 may still be in flight)
    if (threadIdx.x == 0) ntask = ntask2 = 0;
    __syncthreads();
    const int64_t mid_n = 2LL * nyp * X;
    const int64_t gs_n = 4LL * nyp * nxp;
    const T ks = static_cast<T>(a.kin_scale);
    T ekin_t = 0;
    const int ylo_ = ylo, yhi_ = yhi;
    // The x range of row b whose outputs of the y-type pair `by` (types 2 by, 2 by + 1 of
    // this plane) the compressed write reads: the coarse members where the pair holds the
    // scaling type 0 (bz = 0, by = 0), else the hull of the row's fine members (the wavelet
    // types are stored on fine members only).  lo < 0: none.
    auto need = [&](int by, int b, int& lo, int& hi) {
        if (bz == 0 && by == 0) {
            lo = rx0[b];
            hi = rx1[b];
        } else {
            lo = fx0[b];
            hi = fx1[b];
        }
    };
    // ---- column ranges per row block, with their prefix sums, in one phase: the y pass's
    //      (FMA version; blocks of NB rows: for row b and pair by its blocks k = lo/NB ..
    //      hi/NB of the needed range read x' in [2 (k NB + dx), 2 (k NB + NB - 1 + dx) + 30])
    //      and the kinetic y arm's (per x type bx, the pair of types bx, bx + 2, and block
    //      of BB rows: the hull of the rows' needed ranges, the coarse members where the
    //      pair holds type 0, else the fine members)
    const int nbb = (yhi_ - ylo_ + NB) / NB;
    const int nbyk = (yhi_ - ylo_ + BB) / BB;
    if (yhi_ >= 0) {
        if (NS == 0 && static_cast<int>(threadIdx.x) < nbb) {
            const int q = threadIdx.x;
            int c0 = X, c1 = -1;
            for (int b = ylo_ + q * NB; b < min(ylo_ + (q + 1) * NB, yhi_ + 1); ++b)
                for (int by = 0; by < 2; ++by) {
                    int lo, hi;
                    need(by, b, lo, hi);
                    if (lo < 0) continue;
                    c0 = min(c0, 2 * ((lo / NB) * NB + dx));
                    c1 = max(c1, 2 * ((hi / NB) * NB + NB - 1 + dx) + 30);
                }
            cq0[q] = max(c0, 0);
            cq1[q] = min(c1, X - 1);
        }
        const int t2 = static_cast<int>(threadIdx.x) - 128;
        if (t2 >= 0 && t2 < 2 * nbyk) {
            const int bx = t2 >= nbyk, q = t2 - bx * nbyk;
            const bool coarse = bz == 0 && bx == 0;
            int c0 = nxp, c1 = -1;
            for (int b = ylo_ + q * BB; b < min(ylo_ + (q + 1) * BB, yhi_ + 1); ++b) {
                const int lo = coarse ? rx0[b] : fx0[b], hi = coarse ? rx1[b] : fx1[b];
                if (lo < 0) continue;
                c0 = min(c0, lo);
                c1 = max(c1, hi);
            }
            rq0[t2] = c0;
            rq1[t2] = c1;
        }
        __syncthreads();
        if (NS == 0 && threadIdx.x == 0) {
            pq[0] = 0;
            for (int q = 0; q < nbb; ++q) pq[q + 1] = pq[q] + max(0, cq1[q] - cq0[q] + 1);
        }
        if (threadIdx.x == 32) {
            rqp[0] = 0;
            for (int i = 0; i < 2 * nbyk; ++i) rqp[i + 1] = rqp[i] + max(0, rq1[i] - rq0[i] + 1);
        }
        __syncthreads();
    }
    if constexpr (NS > 0) {
        // ---- potential part on the tensor cores -> Gs (every row and column of the plane)
        if (yhi_ >= 0 && !bwd_tc_potential<NS>(reinterpret_cast<const float*>(Bb), bb_room, X, Y, nyp, nxp, dx, dy,
                                                K1, N1, K2, N2, FY_PART, FX_PART, XR, sFy, sFx, sXr,
                                                reinterpret_cast<float*>(Gs), smem_raw, smem_n * 4, st)) {
            if (threadIdx.x == 0) atomicOr(st, ST_WAIT_TIMEOUT);
        }
    }
    if (yhi_ >= 0) {
      if constexpr (NS == 0) {
        // ---- y pass: blocks of NB rows b within [ylo, yhi], per block only the columns
        //      listed above
        {
            const int ntk = pq[nbb];
            for (int tk = threadIdx.x; tk < ntk; tk += blockDim.x) {
                int q = 0;
                while (tk >= pq[q + 1]) ++q;
                const int xo = cq0[q] + (tk - pq[q]), b0 = ylo_ + q * NB;
                T w[2 * NB + 29], s[NB], d[NB];
                swin(w, pl, xo, X, 2 * (b0 + dy), Y, smem_n, st);
                bwd_block<T, NB>(w, s, d);
#pragma unroll
                for (int j = 0; j < NB; ++j) {
                    const int b = b0 + j;
                    if (b <= yhi_) {
                        ST(mid, static_cast<int64_t>(b) * X + xo, mid_n, s[j]);
                        ST(mid, static_cast<int64_t>(nyp + b) * X + xo, mid_n, d[j]);
                    }
                }
            }
        }
        __syncthreads();   // pl is dead from here on: Gs reuses it
        // ---- task list: (by, row b, x block of NB) intersecting the row's needed range
        for (int b = ylo_ + threadIdx.x; b <= yhi_; b += blockDim.x) {
            for (int by = 0; by < 2; ++by) {
                int lo, hi;
                need(by, b, lo, hi);
                if (lo < 0) continue;
                const int k0 = lo / NB, k1 = hi / NB;
                const int base = atomicAdd(&ntask, k1 - k0 + 1);
                for (int k = k0; k <= k1; ++k)
                    if (base + k - k0 < BWD_MAX_TASKS) task[base + k - k0] = (by << 24) | (b << 12) | k;
            }
        }
        __syncthreads();
        int nt = min(ntask, BWD_MAX_TASKS);
        if (ntask > BWD_MAX_TASKS && threadIdx.x == 0) atomicOr(a.status, ST_BAD_BOX);
        // ---- x pass (transposed filters) on the listed row blocks
        for (int it = threadIdx.x; it < nt; it += blockDim.x) {
            const int code = task[it];
            const int by = code >> 24, b = (code >> 12) & 4095, x0 = (code & 4095) * NB;
            const int row = by * nyp + b;
            T w[2 * NB + 29], s[NB], d[NB];
            swin(w, mid, row * X, 1, 2 * (x0 + dx), X, mid_n, st);
            bwd_block<T, NB>(w, s, d);
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                const int xb = x0 + j;
                if (xb < nxp) {
                    ST(Gs, ((0 + 2 * by) * nyp + b) * nxp + xb, gs_n, s[j]);
                    ST(Gs, ((1 + 2 * by) * nyp + b) * nxp + xb, gs_n, d[j]);
                }
            }
        }
      }
        // the D plane and the flags have landed (their copies flew during the passes above)
        cp_wait();
        __syncthreads();
        if (dplane) {   // zero flags of the staged D plane
            const FastDiv fd_pn(pn), fd_nx(nx);
            for (int i = threadIdx.x; i < 4 * pn; i += blockDim.x) {
                const int tb = fd_pn.div(i), rem = i - tb * pn;
                const int y = fd_nx.div(rem), x = rem - y * nx;
                if (LD(Dp, (tb * ny + y) * RS + x, dp_n) != T(0)) {
                    rowf[tb][y & 127] = 1;
                    colf[tb][x & 127] = 1;
                }
            }
        }
        if (NS == 0 && a.gstage) {
            // mid is dead: stage the z-arm plane G (types tb + 4 bz) for the compressed
            // write, in flight during the kinetic phases
            const T* G = static_cast<const T*>(a.ws) + r.ws_G;
            const int64_t gplane = static_cast<int64_t>(nxp) * nyp * nzp;
            const int pnp = nyp * nxp;
            const int r0 = ylo_ * nxp, r1 = (yhi_ + 1) * nxp;        // member rows only
            for (int tb = 0; tb < 4; ++tb)
                for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x)
                    CPA(mid, tb * pnp + i, midA, G, (tb + 4 * bz) * gplane + static_cast<int64_t>(zb) * pnp + i,
                        8 * gplane);
        }
        if (dplane) {
            int nt;
            __syncthreads();   // the D plane's zero flags
            // ---- kinetic x arm: (by, row b, x block of BB) over the needed range of rows whose
            //      D rows are nonzero
            for (int b = ylo_ + threadIdx.x; b <= yhi_; b += blockDim.x) {
                const int y = b + dy;
                if (y < 0 || y >= ny) continue;
                for (int by = 0; by < 2; ++by) {
                    if (!rowf[2 * by][y & 127] && !rowf[2 * by + 1][y & 127]) continue;
                    int lo, hi;
                    need(by, b, lo, hi);
                    if (lo < 0) continue;
                    const int k0 = lo / BB, k1 = hi / BB;
                    const int base = atomicAdd(&ntask2, k1 - k0 + 1);
                    for (int k = k0; k <= k1; ++k)
                        if (base + k - k0 < BWD_MAX_TASKS) task[base + k - k0] = (by << 24) | (b << 12) | k;
                }
            }
            __syncthreads();
            nt = min(ntask2, BWD_MAX_TASKS);
            if (ntask2 > BWD_MAX_TASKS && threadIdx.x == 0) atomicOr(a.status, ST_BAD_BOX);
            for (int it = threadIdx.x; it < nt; it += blockDim.x) {
                const int code = task[it];
                const int by = code >> 24, b = (code >> 12) & 4095, x0 = (code & 4095) * BB;
                const int y = b + dy;
                T k0[KW], k1[KW], o0[BB], o1[BB];
                const int r0 = ((2 * by) * ny + y) * RS, r1 = r0 + ny * RS;
                swin(k0, Dp, r0, 1, x0 + dx - KIN_HALF, nx, dp_n, st);
                swin(k1, Dp, r1, 1, x0 + dx - KIN_HALF, nx, dp_n, st);
                kin_block(k0, k1, o0, o1);
#pragma unroll
                for (int j = 0; j < BB; ++j) {
                    const int xb = x0 + j;
                    if (xb < nxp) {
                        o0[j] *= ks;
                        o1[j] *= ks;
                        const int64_t g0 = ((0 + 2 * by) * nyp + b) * nxp + xb;
                        const int64_t g1 = ((1 + 2 * by) * nyp + b) * nxp + xb;
                        ST(Gs, g0, gs_n, LD(Gs, g0, gs_n) + o0[j]);
                        ST(Gs, g1, gs_n, LD(Gs, g1, gs_n) + o1[j]);
                        const int x = x0 + dx + j;
                        if (x >= 0 && x < nx) ekin_t += k0[KIN_HALF + j] * o0[j] + k1[KIN_HALF + j] * o1[j];
                    }
                }
            }
            __syncthreads();   // the x arm's Gs updates are done
            // ---- kinetic y arm: tasks (x type bx, block q of BB rows, column) over the column
            //      ranges listed above, consecutive columns on consecutive threads
            nt = rqp[2 * nbyk];
            for (int it = threadIdx.x; it < nt; it += blockDim.x) {
                int lo = 0, hi = 2 * nbyk - 1;              // the entry i with rqp[i] <= it < rqp[i + 1]
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (rqp[mid] <= it) lo = mid;
                    else hi = mid - 1;
                }
                const int bx = lo >= nbyk, q = lo - bx * nbyk;
                const int xb = rq0[lo] + (it - rqp[lo]), b0 = ylo_ + q * BB;
                const int x = xb + dx;
                if (x < 0 || x >= nx) continue;
                if (!colf[bx][x & 127] && !colf[bx + 2][x & 127]) continue;
                T k0[KW], k1[KW], o0[BB], o1[BB];
                swin(k0, Dp, bx * ny * RS + x, RS, b0 + dy - KIN_HALF, ny, dp_n, st);
                swin(k1, Dp, (bx + 2) * ny * RS + x, RS, b0 + dy - KIN_HALF, ny, dp_n, st);
                kin_block(k0, k1, o0, o1);
#pragma unroll
                for (int j = 0; j < BB; ++j) {
                    const int b = b0 + j;
                    if (b <= yhi_) {
                        o0[j] *= ks;
                        o1[j] *= ks;
                        const int64_t g0 = (static_cast<int64_t>(bx + 0) * nyp + b) * nxp + xb;
                        const int64_t g1 = (static_cast<int64_t>(bx + 2) * nyp + b) * nxp + xb;
                        ST(Gs, g0, gs_n, LD(Gs, g0, gs_n) + o0[j]);
                        ST(Gs, g1, gs_n, LD(Gs, g1, gs_n) + o1[j]);
                        const int y = b + dy;
                        if (y >= 0 && y < ny) ekin_t += k0[KIN_HALF + j] * o0[j] + k1[KIN_HALF + j] * o1[j];
                    }
                }
            }
        }
    }
    cp_wait();
    __syncthreads();
    // ---- compress: members of this plane -> H phi (plus the z arm left in G by k_kin_z;
    //      the FMA path reads it from the plane staged in mid).  Coarse members (type 0)
    //      row by row, a warp per row (one segment of up to n_x' members each); fine members
    //      flattened over the CTA, one member per thread and type: the plane's fine
    //      segments (many short chords of the fine spheres) are staged in shared memory and
    //      each member finds its segment by a binary search, so every lane writes and
    //      consecutive lanes write consecutive H phi elements.
    if (yhi_ >= 0) {
        const T* G = static_cast<const T*>(a.ws) + r.ws_G;
        const unsigned char* gflag = reinterpret_cast<const unsigned char*>(a.gstage ? gfl : gsrc);
        const bool gsm = NS == 0 && a.gstage;               // the z-arm plane is in mid
        const int64_t gplane = static_cast<int64_t>(nxp) * nyp * nzp;
        T* out = static_cast<T*>(a.hphi) + r.off_hphi;
        const int64_t out_room = a.hphi_n - r.off_hphi;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (bz == 0) {   // scaling part s (type 0) on the coarse members
            for (int b = ylo_ + warp; b <= yhi_; b += (blockDim.x >> 5)) {
                if (rx0[b] < 0) continue;
                const int y = b + dy;
                const bool yin = y >= 0 && y < ny;
                const int64_t grow = (static_cast<int64_t>(zb) * nyp + b) * nxp;
                for (int xb = rx0[b] + lane; xb <= rx1[b]; xb += 32) {
                    const int x = xb + dx;
                    T v = LD(Gs, static_cast<int64_t>(b) * nxp + xb, gs_n);
                    if (yin && x >= 0 && x < nx && LD(gflag, y * nx + x, 4LL * pn))
                        v += gsm ? LD(mid, static_cast<int64_t>(b) * nxp + xb, midA) : LD(G, grow + xb, 8 * gplane);
                    ST(out, roff[b] + (xb - rx0[b]), out_room, v);
                }
            }
        }
        // wavelet parts on the fine members of this plane: segments [q0, q1) hold members
        // [m0, m1) of each type's block
        const int q0 = fr0[ylo_], q1 = fr1[yhi_];
        if (q1 > q0) {
            constexpr int SEG_CAP = BWD_MAX_TASKS / 4;    // Seg records in the task array
            int4* sseg = reinterpret_cast<int4*>(task);
            const int nq = q1 - q0;
            const bool staged = nq <= SEG_CAP;
            if (staged)
                for (int i = threadIdx.x; i < nq; i += blockDim.x) {
                    const Seg g = LD(a.seg, at.segPf + q0 + i, a.seg_n);
                    sseg[i] = make_int4(g.x0, g.x1, g.row, g.off);
                }
            __syncthreads();
            auto seg_at = [&](int i) -> int4 {
                if (staged) return sseg[i];
                const Seg g = LD(a.seg, at.segPf + q0 + i, a.seg_n);
                return make_int4(g.x0, g.x1, g.row, g.off);
            };
            const int4 sl = seg_at(nq - 1);
            const int m0 = seg_at(0).w, m1 = sl.w + (sl.y - sl.x + 1);
            const int64_t zrow = static_cast<int64_t>(nyp) * zb;
            for (int m = m0 + static_cast<int>(threadIdx.x); m < m1; m += blockDim.x) {
                int lo = 0, hi = nq - 1;                     // the segment with off <= m
                while (lo < hi) {
                    const int mid_ = (lo + hi + 1) >> 1;
                    if (seg_at(mid_).w <= m) lo = mid_;
                    else hi = mid_ - 1;
                }
                const int4 g = seg_at(lo);
                const int xb = g.x + (m - g.w);
                const int b = static_cast<int>(g.z - zrow);
                const int y = b + dy, x = xb + dx;
                const bool zin = y >= 0 && y < ny && x >= 0 && x < nx;
                const int64_t grow = (static_cast<int64_t>(zb) * nyp + b) * nxp;
#pragma unroll
                for (int tb = 0; tb < 4; ++tb) {
                    const int t = tb + 4 * bz;
                    if (t == 0) continue;
                    T v = LD(Gs, (static_cast<int64_t>(tb) * nyp + b) * nxp + xb, gs_n);
                    if (zin && LD(gflag, (t & 3) * pn + y * nx + x, 4LL * pn))
                        v += gsm ? LD(mid, (static_cast<int64_t>(tb) * nyp + b) * nxp + xb, midA)
                                 : LD(G, t * gplane + grow + xb, 8 * gplane);
                    ST(out, at.ncP + static_cast<int64_t>(t - 1) * at.nfP + m, out_room, v);
                }
            }
        }
    }
    const double ekin = warp_sum(static_cast<double>(ekin_t));
    if ((threadIdx.x & 31) == 0 && ekin != 0.0) atomicAdd(a.e_kin + r.f, ekin);
    if constexpr (NS > 0) {
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if ((threadIdx.x >> 5) == 0) tc::tmem_free(*reinterpret_cast<volatile uint32_t*>(smem_raw + 8), 128);
    }
}

// Persistent form of the FMA version (a.items_bwd set): the batch's (function, z'' plane,
// z type) items, largest first, from the second queue counter; otherwise (and always for
// the tensor-core versions) one CTA per grid slot (blockIdx.x = 2 z'' + b_z, blockIdx.y =
// function).
template <class T, int NS>
__global__ void __launch_bounds__(NS ? 512 : 256, NS ? 1 : (sizeof(T) == 4 ? LSW_BWD_MIN_BLOCKS : 1))
    k_bwd_xy(HphiLaunch a) {
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = 4;
    if (NS == 0 && a.items_bwd) {
        __shared__ int s_item;
        for (;;) {
            const int k = next_item(a.queue + 1, &s_item);
            if (k >= a.n_items_bwd) break;
            const int code = LD(a.items_bwd, k, a.n_items_bwd);
            bwd_plane<T, NS>(a, code >> 11, (code >> 1) & 1023, code & 1);
            __syncthreads();   // shared memory and s_item are reused by the next item
        }
    } else {
        bwd_plane<T, NS>(a, blockIdx.y, blockIdx.x >> 1, blockIdx.x & 1);
    }
}

// ---------------------------------------------------------------- density: pair products
//
// rho_j = sum_ab K_ab u_a(j) u_b(j) (Eq. density) per tile of DT_X x DT_Y x DT_Z grid
// points, over the functions whose real-space blocks meet the tile (App. D: the density
// is formed like the scalar products, from the functions present at each point).  The
// quadratic form depends only on the symmetric part of K, so the functions of a tile are
// taken in chunks of DT_MC and every pair of chunks A <= B once: the coefficient block is
// K_ab for A = B and K_ab + K_ba for A < B.  Each thread owns DT_PP points and keeps the
// B chunk's values there in registers; the coefficient block sits in shared memory and is
// read as a broadcast.  Products and the chunk-pair partial sums run in T, the total per
// point in FP64; every point of the grid is written (0 where no block reaches).

// K_ab from the pattern CSR (binary search of b in row a), 0 outside the pattern.
__device__ __forceinline__ double dens_k(const DensLaunch& a, int fa, int fb) {
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = 13;
    int64_t lo = LD(a.row_ptr, fa, a.rowp_n), hi = LD(a.row_ptr, fa + 1, a.rowp_n);
    const int64_t end = hi;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (LD(a.col, mid, a.nnz) < fb)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (lo < end && LD(a.col, lo, a.nnz) == fb) ? LD(a.K, lo, a.nnz) : 0.0;
}

// u_f at grid point (x, y, z); 0 outside f's block.
template <class T>
__device__ __forceinline__ T dens_u(const DensLaunch& a, const DensFn& df, int x, int y, int z) {
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = 13;
    const int lx = x - df.o[0], ly = y - df.o[1], lz = z - df.o[2];
    if (static_cast<unsigned>(lx) >= static_cast<unsigned>(df.d[0]) ||
        static_cast<unsigned>(ly) >= static_cast<unsigned>(df.d[1]) ||
        static_cast<unsigned>(lz) >= static_cast<unsigned>(df.d[2]))
        return T(0);
    const T* U = static_cast<const T*>(a.U);
    return LD(U, df.off + (static_cast<int64_t>(lz) * df.d[1] + ly) * df.d[0] + lx, a.U_n);
}

__device__ __forceinline__ void lds16(const float* p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
}
__device__ __forceinline__ void lds16(const double* p, double (&v)[2]) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    v[0] = t.x, v[1] = t.y;
}

template <class T>
__global__ void __launch_bounds__(DT_THREADS) k_density(DensLaunch a) {
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = 13;
    constexpr int VW = 16 / sizeof(T);
    __shared__ __align__(16) T kb[DT_MC * DT_MC];
    const int tile = blockIdx.x;
    const int tx = tile % a.ntile[0];
    const int ty = (tile / a.ntile[0]) % a.ntile[1];
    const int tz = tile / (a.ntile[0] * a.ntile[1]);
    const int64_t t0 = LD(a.tptr, tile, a.tptr_n);
    const int m = static_cast<int>(LD(a.tptr, tile + 1, a.tptr_n) - t0);
    int px[DT_PP], py[DT_PP], pz[DT_PP];
    double acc[DT_PP];
#pragma unroll
    for (int i = 0; i < DT_PP; ++i) {
        const int p = threadIdx.x + i * DT_THREADS;
        px[i] = tx * DT_X + p % DT_X;
        py[i] = ty * DT_Y + (p / DT_X) % DT_Y;
        pz[i] = tz * DT_Z + p / (DT_X * DT_Y);
        acc[i] = 0.0;
    }
    for (int cb = 0; cb < m; cb += DT_MC) {
        const int nb = min(DT_MC, m - cb);
        T ub[DT_MC][DT_PP];
#pragma unroll
        for (int j = 0; j < DT_MC; ++j) {
            if (j < nb) {
                const DensFn df = LD(a.fn, LD(a.tfn, t0 + cb + j, a.tfn_n), a.fn_n);
#pragma unroll
                for (int i = 0; i < DT_PP; ++i) ub[j][i] = dens_u<T>(a, df, px[i], py[i], pz[i]);
            } else {
#pragma unroll
                for (int i = 0; i < DT_PP; ++i) ub[j][i] = T(0);
            }
        }
        for (int ca = 0; ca <= cb; ca += DT_MC) {
            const int na = min(DT_MC, m - ca);
            __syncthreads();   // the previous block's readers are done
            for (int e = threadIdx.x; e < DT_MC * DT_MC; e += DT_THREADS) {
                const int ia = e / DT_MC, ib = e % DT_MC;
                double v = 0.0;
                if (ia < na && ib < nb) {
                    const int fa = LD(a.tfn, t0 + ca + ia, a.tfn_n);
                    const int fb = LD(a.tfn, t0 + cb + ib, a.tfn_n);
                    v = dens_k(a, fa, fb);
                    if (ca != cb) v += dens_k(a, fb, fa);
                }
                kb[e] = static_cast<T>(v);
            }
            __syncthreads();
            T part[DT_PP];
#pragma unroll
            for (int i = 0; i < DT_PP; ++i) part[i] = T(0);
            for (int ia = 0; ia < na; ++ia) {
                const DensFn df = LD(a.fn, LD(a.tfn, t0 + ca + ia, a.tfn_n), a.fn_n);
                T ua[DT_PP], z[DT_PP];
#pragma unroll
                for (int i = 0; i < DT_PP; ++i) {
                    ua[i] = dens_u<T>(a, df, px[i], py[i], pz[i]);
                    z[i] = T(0);
                }
                const T* row = kb + ia * DT_MC;
#pragma unroll
                for (int q = 0; q < DT_MC; q += VW) {
                    T k[VW];
                    lds16(row + q, k);
#pragma unroll
                    for (int w = 0; w < VW; ++w)
#pragma unroll
                        for (int i = 0; i < DT_PP; ++i) z[i] += k[w] * ub[q + w][i];
                }
#pragma unroll
                for (int i = 0; i < DT_PP; ++i) part[i] += ua[i] * z[i];
            }
#pragma unroll
            for (int i = 0; i < DT_PP; ++i) acc[i] += static_cast<double>(part[i]);
        }
    }
#pragma unroll
    for (int i = 0; i < DT_PP; ++i)
        if (px[i] < a.gn[0] && py[i] < a.gn[1] && pz[i] < a.gn[2])
            ST(a.rho, (pz[i] * a.gn[1] + py[i]) * a.gn[0] + px[i], a.rho_n, acc[i]);
}

// ---------------------------------------------------------------- peak probes
//
// Denominators of the rooflines, measured on the running GPU: a dependent-chain FMA
// loop (8 independent chains per thread, operands from memory so nothing folds) and a
// 16-byte streaming copy.

template <class T>
__global__ void __launch_bounds__(256) k_fma_peak(const T* in, T* out, int iters) {
    T x = in[0], y = in[1];
    T acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = in[2 + i] + static_cast<T>(threadIdx.x);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] = acc[i] * x + y;
    T sum = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) sum += acc[i];
    if (sum == static_cast<T>(-1.2345)) out[blockIdx.x * blockDim.x + threadIdx.x] = sum;   // keeps the loop live
}

__global__ void __launch_bounds__(256) k_copy_peak(const float4* __restrict__ src, float4* __restrict__ dst, int64_t n) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        dst[i] = src[i];
}

cudaError_t measure_peaks(int n_sm, double* fp32_tflops, double* fp64_tflops, double* copy_gbs) {
    cudaError_t e;
    const int64_t n4 = (1LL << 30) / 16;       // 1 GiB per buffer
    float4 *a = nullptr, *b = nullptr;
    double* io = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto done = [&](cudaError_t r) {
        if (a) cudaFree(a);
        if (b) cudaFree(b);
        if (io) cudaFree(io);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        return r;
    };
    if ((e = cudaMalloc(&a, n4 * 16)) != cudaSuccess) return done(e);
    if ((e = cudaMalloc(&b, n4 * 16)) != cudaSuccess) return done(e);
    if ((e = cudaMalloc(&io, 4096)) != cudaSuccess) return done(e);
    if ((e = cudaMemset(a, 0, n4 * 16)) != cudaSuccess) return done(e);
    {
        const double hv[10] = {0.999999, 1e-7, 1, 2, 3, 4, 5, 6, 7, 8};
        const float hf[10] = {0.999999f, 1e-7f, 1, 2, 3, 4, 5, 6, 7, 8};
        if ((e = cudaMemcpy(io, hv, sizeof(hv), cudaMemcpyHostToDevice)) != cudaSuccess) return done(e);
        if ((e = cudaMemcpy(reinterpret_cast<char*>(io) + 128, hf, sizeof(hf), cudaMemcpyHostToDevice)) != cudaSuccess)
            return done(e);
    }
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) return done(e);
    const int blocks = n_sm * 8;
    auto best_ms = [&](auto launch, float* out_ms) -> cudaError_t {
        float best = 1e30f;
        for (int r = 0; r < 6; ++r) {
            cudaEventRecord(e0);
            launch();
            cudaEventRecord(e1);
            cudaError_t le = cudaEventSynchronize(e1);
            if (le != cudaSuccess) return le;
            if ((le = cudaGetLastError()) != cudaSuccess) return le;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0) best = std::min(best, ms);
        }
        *out_ms = best;
        return cudaSuccess;
    };
    float ms;
    const int it32 = 1 << 16, it64 = 1 << 12;
    float* io32 = reinterpret_cast<float*>(reinterpret_cast<char*>(io) + 128);
    if ((e = best_ms([&] { k_fma_peak<float><<<blocks, 256>>>(io32, io32 + 64, it32); }, &ms)) != cudaSuccess)
        return done(e);
    *fp32_tflops = 2.0 * 8.0 * it32 * blocks * 256.0 / (ms * 1e-3) / 1e12;
    if ((e = best_ms([&] { k_fma_peak<double><<<blocks, 256>>>(io, io + 128, it64); }, &ms)) != cudaSuccess)
        return done(e);
    *fp64_tflops = 2.0 * 8.0 * it64 * blocks * 256.0 / (ms * 1e-3) / 1e12;
    if ((e = best_ms([&] { k_copy_peak<<<n_sm * 16, 256>>>(a, b, n4); }, &ms)) != cudaSuccess) return done(e);
    *copy_gbs = 2.0 * n4 * 16.0 / (ms * 1e-3) / 1e9;
    return done(cudaSuccess);
}

// ---------------------------------------------------------------- reformat

// Reuse of support functions on a shifted geometry: warp per destination segment of
// L_dst(f); each member point p takes the source value at p - shift(atom) if that point
// is a member of L_src(f) (coarse part for s, fine part for d^1..d^7), else 0.
template <class T>
__global__ void k_reformat(ReformatLaunch a) {
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = 10;
    const FnRec r = a.fn[blockIdx.y];
    const AtomRec& ad = a.atoms_dst[r.atom];
    const AtomRec& as = a.atoms_src[r.atom];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sidx = blockIdx.x * (blockDim.x >> 5) + warp;
    const int nseg = ad.nsegLc + ad.nsegLf;
    if (sidx >= nseg) return;
    const bool fine = sidx >= ad.nsegLc;
    const Seg sg = LD(a.seg_dst, fine ? ad.segLf + (sidx - ad.nsegLc) : ad.segLc + sidx, a.seg_dst_n);
    const int sx = a.shift[3 * r.atom], sy = a.shift[3 * r.atom + 1], sz = a.shift[3 * r.atom + 2];
    // destination row -> global (y, z)
    const int yl = sg.row % ad.n[1], zl = sg.row / ad.n[1];
    const int gy = ad.lo[1] + yl - sy, gz = ad.lo[2] + zl - sz;     // source row
    const int ys = gy - as.lo[1], zs = gz - as.lo[2];
    const bool row_in = ys >= 0 && zs >= 0 && ys < as.n[1] && zs < as.n[2];
    int s0 = 0, s1 = 0;
    if (row_in) {
        const int64_t rrow = (fine ? as.rowLf : as.rowLc) + ys + static_cast<int64_t>(as.n[1]) * zs;
        s0 = LD(a.rowptr_src, rrow, a.rowptr_src_n);
        s1 = LD(a.rowptr_src, rrow + 1, a.rowptr_src_n);
    }
    const T* src = static_cast<const T*>(a.phi_src) + LD(a.off_src, r.f, a.nfn + 1);
    T* dst = static_cast<T*>(a.phi_dst) + r.off_phi;
    const int64_t src_room = a.src_n - LD(a.off_src, r.f, a.nfn + 1);
    const int64_t dst_room = a.dst_n - r.off_phi;
    const int64_t seg0 = fine ? as.segLf : as.segLc;
    const int len = sg.x1 - sg.x0 + 1;
    for (int k = lane; k < len; k += 32) {
        const int xs = ad.lo[0] + sg.x0 + k - sx - as.lo[0];          // source box-local x
        int64_t off = -1;
        for (int q = s0; q < s1; ++q) {
            const Seg ss = LD(a.seg_src, seg0 + q, a.seg_src_n);
            if (xs >= ss.x0 && xs <= ss.x1) off = ss.off + (xs - ss.x0);
        }
        if (!fine) {
            ST(dst, sg.off + k, dst_room, off >= 0 ? LD(src, off, src_room) : T(0));
        } else {
#pragma unroll
            for (int t = 0; t < 7; ++t)
                ST(dst, ad.ncL + static_cast<int64_t>(t) * ad.nfL + sg.off + k, dst_room,
                   off >= 0 ? LD(src, as.ncL + static_cast<int64_t>(t) * as.nfL + off, src_room) : T(0));
        }
    }
}

cudaError_t enqueue_reformat(const ReformatLaunch& a, cudaStream_t s) {
    if (a.nfn == 0) return cudaSuccess;
    const dim3 grid((a.max_seg + 7) / 8, a.nfn);
    if (a.prec == 0)
        k_reformat<double><<<grid, 256, 0, s>>>(a);
    else
        k_reformat<float><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- fixed device scratch

// Workspace of lsw_apply_hamiltonian_noalloc: a file-scope device array, so that this
// entry point never allocates.  Every GPU that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of the array on `device` (which must be current).  The first call for
// a device looks the address up with cudaGetSymbolAddress (this may load the module, so
// it belongs before any stream capture); later calls return the cached address.
cudaError_t noalloc_scratch(int device, void** ptr) {
    static std::mutex mu;
    static void* addr[NOALLOC_MAX_DEVICES] = {};
    if (device < 0 || device >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (addr[device] == nullptr) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        addr[device] = p;
    }
    *ptr = addr[device];
    return cudaSuccess;
}

// Records of one batch of the allocation-free path, built on the device: boxes and
// offsets are copied from the system's resident per-function records (all[f0 ..
// f0 + nb)), and the workspace offsets are laid out again, function after function, in
// the order and sizes the host validated (D boxes first, then Bf, Bb, G and the z-arm
// flags of each function; every region a multiple of 64 elements).  One thread: nb is
// at most NOALLOC_MAX_BATCH.
__global__ void k_noalloc_records(const FnRec* __restrict__ all, int64_t f0, int nb, int64_t esize,
                                  FnRec* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    auto al = [](int64_t x) { return (x + ALIGN_ELEMS - 1) / ALIGN_ELEMS * ALIGN_ELEMS; };
    int64_t o = 0;
    for (int k = 0; k < nb; ++k) {
        FnRec r = all[f0 + k];
        r.ws_D = o;
        o += al(8LL * r.n[0] * r.n[1] * r.n[2]);
        out[k] = r;
    }
    for (int k = 0; k < nb; ++k) {
        FnRec& r = out[k];
        const int64_t X = 2 * r.n[0] + 29, Y = 2 * r.n[1] + 29;
        r.ws_Bf = o;
        o += al(2LL * r.n[2] * Y * X);
        r.ws_Bb = o;
        o += al(2LL * r.np[2] * Y * X);
        r.ws_G = o;
        o += al(8LL * r.np[0] * r.np[1] * r.np[2]);
        r.ws_Gf = o;
        o += al((4LL * r.n[0] * r.n[1] + esize - 1) / esize);
    }
}

cudaError_t enqueue_noalloc_records(const FnRec* all, int64_t f0, int nb, int64_t esize, FnRec* out, cudaStream_t s) {
    k_noalloc_records<<<1, 32, 0, s>>>(all, f0, nb, esize, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- host entry points

cudaError_t upload_filters(const FilterSet& fs, int device) {
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return e;
    float f32[2][FWD_TAPS];
    float k32[4][KIN_TAPS];
    for (int b = 0; b < 2; ++b)
        for (int i = 0; i < FWD_TAPS; ++i) f32[b][i] = static_cast<float>(fs.fwd[b][i]);
    for (int b = 0; b < 4; ++b)
        for (int i = 0; i < KIN_TAPS; ++i) k32[b][i] = static_cast<float>(fs.kin[b][i]);
    if ((e = cudaMemcpyToSymbol(c_fwd_d, fs.fwd, sizeof(fs.fwd))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_kin_d, fs.kin, sizeof(fs.kin))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_fwd_f, f32, sizeof(f32))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_kin_f, k32, sizeof(k32))) != cudaSuccess) return e;
    float2 bwd2[FWD_TAPS], up2[2][16], kin2[2][KIN_TAPS];
    for (int m = 0; m < FWD_TAPS; ++m) bwd2[m] = make_float2(f32[0][m], f32[1][m]);
    for (int b = 0; b < 2; ++b)
        for (int k = 0; k < 16; ++k) up2[b][k] = make_float2(f32[b][2 * k], 2 * k + 1 < FWD_TAPS ? f32[b][2 * k + 1] : 0.f);
    for (int l = 0; l < KIN_TAPS; ++l) {
        kin2[0][l] = make_float2(k32[0][l], k32[2][l]);
        kin2[1][l] = make_float2(k32[1][l], k32[3][l]);
    }
    if ((e = cudaMemcpyToSymbol(c_fwd2_bwd, bwd2, sizeof(bwd2))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_fwd2_up, up2, sizeof(up2))) != cudaSuccess) return e;
    return cudaMemcpyToSymbol(c_kin2, kin2, sizeof(kin2));
}

cudaError_t configure_kernels(size_t max_smem) {
    // dynamic shared memory may use what the kernel's static shared memory leaves
    cudaError_t e;
#define SETMAX(K)                                                                               \
    {                                                                                           \
        cudaFuncAttributes fa;                                                                  \
        if ((e = cudaFuncGetAttributes(&fa, K)) != cudaSuccess) return e;                       \
        const int m = static_cast<int>(max_smem - fa.sharedSizeBytes);                          \
        if ((e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, m)) != cudaSuccess) \
            return e;                                                                           \
    }
    SETMAX(k_fwd_xy<double>) SETMAX(k_fwd_xy<float>)
    SETMAX(k_z<double>) SETMAX(k_z<float>)
    SETMAX(k_kin_z<double>) SETMAX(k_kin_z<float>)
    SETMAX(k_z_tc<2>) SETMAX(k_z_tc<3>)
    SETMAX(k_fwd_xy_tc<2>) SETMAX(k_fwd_xy_tc<3>)
    SETMAX((k_bwd_xy<double, 0>)) SETMAX((k_bwd_xy<float, 0>))
    SETMAX((k_bwd_xy<float, 2>)) SETMAX((k_bwd_xy<float, 3>))
    SETMAX(k_z_dens<double>) SETMAX(k_z_dens<float>)
#undef SETMAX
    // the plans size the plane kernels' dynamic shared memory against these bounds
#define STATIC_BOUND(K, B)                                                                     \
    {                                                                                          \
        cudaFuncAttributes fa;                                                                 \
        if ((e = cudaFuncGetAttributes(&fa, K)) != cudaSuccess) return e;                      \
        if (fa.sharedSizeBytes > (B)) return cudaErrorInvalidConfiguration;                     \
    }
    STATIC_BOUND(k_fwd_xy<double>, FWD_STATIC_SMEM) STATIC_BOUND(k_fwd_xy<float>, FWD_STATIC_SMEM)
    STATIC_BOUND((k_bwd_xy<double, 0>), BWD_STATIC_SMEM) STATIC_BOUND((k_bwd_xy<float, 0>), BWD_STATIC_SMEM)
    STATIC_BOUND((k_bwd_xy<float, 2>), BWD_TC_STATIC_SMEM) STATIC_BOUND((k_bwd_xy<float, 3>), BWD_TC_STATIC_SMEM)
#undef STATIC_BOUND
    return cudaSuccess;
}

cudaError_t plane_kernel_blocks(int prec, size_t smem_fwd, size_t smem_bwd, int* fwd, int* bwd) {
    cudaError_t e;
    if (prec == 0) {
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(fwd, k_fwd_xy<double>, 256, smem_fwd)) != cudaSuccess)
            return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bwd, k_bwd_xy<double, 0>, 256, smem_bwd);
    }
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(fwd, k_fwd_xy<float>, 256, smem_fwd)) != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bwd, k_bwd_xy<float, 0>, 256, smem_bwd);
}

#define TRACED(TR, KIND, S, LAUNCH) \
    do {                                \
        trace_begin(TR, KIND, S);       \
        LAUNCH;                         \
        trace_end(TR, S);               \
    } while (0)

template <class T>
static cudaError_t hphi_batch(const HphiLaunch& a, cudaStream_t s) {
    const int nf = a.nfn;
    TRACED(a.tr, TK_UNCOMPRESS, s, (k_uncompress<T><<<dim3((a.max_rowsL + 7) / 8, nf), 256, 0, s>>>(a)));
    const dim3 gfwd = a.items_fwd ? dim3(a.grid_fwd) : dim3(2 * a.max_nz, nf);
    const dim3 gbwd = a.items_bwd ? dim3(a.grid_bwd) : dim3(2 * a.max_nzp, nf);
    if constexpr (sizeof(T) == 4) {
        if (a.xy_tc && a.zsplit == 3)
            TRACED(a.tr, TK_FWD_XY, s, (k_fwd_xy_tc<3><<<dim3(2 * a.max_nz, nf), 256, a.smem_fwd_tc, s>>>(a)));
        else if (a.xy_tc && a.zsplit == 2)
            TRACED(a.tr, TK_FWD_XY, s, (k_fwd_xy_tc<2><<<dim3(2 * a.max_nz, nf), 256, a.smem_fwd_tc, s>>>(a)));
        else
            TRACED(a.tr, TK_FWD_XY, s, (k_fwd_xy<T><<<gfwd, 256, a.smem_fwd, s>>>(a)));
    } else {
        TRACED(a.tr, TK_FWD_XY, s, (k_fwd_xy<T><<<gfwd, 256, a.smem_fwd, s>>>(a)));
    }
    if constexpr (sizeof(T) == 4) {
        if (a.zsplit) {
            // several tiles per CTA: the filter operands are built once per CTA
            const int gx = ((a.max_cols + tc::TILE - 1) / tc::TILE + tc::TILES_PER_CTA - 1) / tc::TILES_PER_CTA;
            if (a.zsplit == 3)
                TRACED(a.tr, TK_Z, s, (k_z_tc<3><<<dim3(gx, nf), 256, a.smem_ztc, s>>>(a)));
            else
                TRACED(a.tr, TK_Z, s, (k_z_tc<2><<<dim3(gx, nf), 256, a.smem_ztc, s>>>(a)));
        } else {
            TRACED(a.tr, TK_Z, s, (k_z<T><<<dim3((a.max_cols + a.zcols - 1) / a.zcols, nf), a.zcols, a.smem_z, s>>>(a)));
        }
    } else {
        TRACED(a.tr, TK_Z, s, (k_z<T><<<dim3((a.max_cols + a.zcols - 1) / a.zcols, nf), a.zcols, a.smem_z, s>>>(a)));
    }
    TRACED(a.tr, TK_KINETIC, s,
           (k_kin_z<T><<<dim3(static_cast<unsigned>((a.max_colsL + 127) / 128), nf, 4), 128, a.smem_kin, s>>>(a)));
    if constexpr (sizeof(T) == 4) {
        if (a.xy_tc && a.zsplit == 3)
            TRACED(a.tr, TK_BWD_XY, s, (k_bwd_xy<float, 3><<<dim3(2 * a.max_nzp, nf), 512, a.smem_bwd_tc, s>>>(a)));
        else if (a.xy_tc && a.zsplit == 2)
            TRACED(a.tr, TK_BWD_XY, s, (k_bwd_xy<float, 2><<<dim3(2 * a.max_nzp, nf), 512, a.smem_bwd_tc, s>>>(a)));
        else
            TRACED(a.tr, TK_BWD_XY, s, (k_bwd_xy<float, 0><<<gbwd, 256, a.smem_bwd, s>>>(a)));
    } else {
        TRACED(a.tr, TK_BWD_XY, s, (k_bwd_xy<T, 0><<<gbwd, 256, a.smem_bwd, s>>>(a)));
    }
    return cudaGetLastError();
}

cudaError_t enqueue_hphi_batch(const HphiLaunch& a, cudaStream_t s) {
    return a.prec == 0 ? hphi_batch<double>(a, s) : hphi_batch<float>(a, s);
}

// Density, per batch: uncompress, forward x, y (FMA plane kernel in every precision) and
// the density z stage writing u into the store.
template <class T>
static cudaError_t dens_batch(HphiLaunch a, cudaStream_t s) {
    const int nf = a.nfn;
    constexpr int C = ZCols<T>::C;
    a.items_fwd = a.items_bwd = nullptr;       // one CTA per grid slot here
    a.queue = nullptr;
    a.smem_z = sizeof(T) * 2 * static_cast<size_t>(a.max_nz) * C;
    TRACED(a.tr, TK_UNCOMPRESS, s, (k_uncompress<T><<<dim3((a.max_rowsL + 7) / 8, nf), 256, 0, s>>>(a)));
    TRACED(a.tr, TK_FWD_XY, s, (k_fwd_xy<T><<<dim3(2 * a.max_nz, nf), 256, a.smem_fwd, s>>>(a)));
    TRACED(a.tr, TK_DENS_U, s, (k_z_dens<T><<<dim3((a.max_cols + C - 1) / C, nf), C, a.smem_z, s>>>(a)));
    return cudaGetLastError();
}

cudaError_t enqueue_dens_batch(const HphiLaunch& a, cudaStream_t s) {
    return a.prec == 0 ? dens_batch<double>(a, s) : dens_batch<float>(a, s);
}

cudaError_t enqueue_density(const DensLaunch& a, cudaStream_t s) {
    const int64_t nt = static_cast<int64_t>(a.ntile[0]) * a.ntile[1] * a.ntile[2];
    if (nt == 0) return cudaSuccess;
    if (a.prec == 0)
        TRACED(a.tr, TK_DENSITY, s, (k_density<double><<<static_cast<unsigned>(nt), DT_THREADS, 0, s>>>(a)));
    else
        TRACED(a.tr, TK_DENSITY, s, (k_density<float><<<static_cast<unsigned>(nt), DT_THREADS, 0, s>>>(a)));
    return cudaGetLastError();
}


}  // namespace lsw
