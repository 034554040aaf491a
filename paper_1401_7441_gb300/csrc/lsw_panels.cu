// sm_103a kernels of the sparse S_ab / H_ab build in the "transposed" layout (App. D):
//
//   S_ab = <phi_a|phi_b>   over L(a) n L(b),     H_ab = <phi_a|H phi_b>   over L(a) n L'(b)
//   (Sec. II.A; the dot products of the coefficients both functions carry, Eq. phi)
//
// The grid is cut into tiles of T^3 coarse points.  App. D distributes the scalar
// products by regions of the cell, each region holding, for its grid points, the
// coefficients of every support function present there; here a tile plays the region:
//
//   k_pack       per (atom, side): for every tile its region touches (within the slab),
//                writes one panel row per function of the atom: the T^3 scaling values
//                of the tile's points, then the 7 wavelet values of each of the tile's
//                fine points, 0 where the function has no member (A side: phi on L; Q
//                side: H phi on L').  The region's row tables are staged in shared
//                memory, so a panel value costs one lookup, one load and one store.
//   k_panel_hs   per work item (tile, up to 64 A rows, up to 128 columns of [A; Q]): the
//                dense product of the A panel with the [A; Q] panel over the tile's
//                panel length, 4 x 8 outputs per thread in the system's precision, then
//                each pattern entry (a, b) gets its tile sum added to S_ab (column in A)
//                or H_ab (column in Q) in FP64.
#include <cstdint>

#include "lsw_device.h"
#include "lsw_internal.h"
#include "lsw_tc.h"

namespace lsw {

// ---------------------------------------------------------------- pack

constexpr int PK_THREADS = 512;   // 16 warps: many tiles' loads in flight per CTA

template <class T, bool Unpack>
__global__ void __launch_bounds__(PK_THREADS, 2) k_pack(PackLaunch a) {
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = Unpack ? 12 : 10;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int side = blockIdx.y;                       // 0: phi on L -> PA; 1: H phi on L' -> PQ
    if (side == 1 && a.hphi == nullptr) return;        // block-uniform, before any barrier
    [[maybe_unused]] T* out = static_cast<T*>(a.out);
    const int atom = LD(a.slab_atoms, blockIdx.x, a.n_slab_atoms);
    const AtomRec at = LD(a.atoms, atom, a.n_atoms);
    const PanelAtom pa = LD(a.patoms, atom, a.n_atoms);
    int lo[3], n[3], tlo[3], tn[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = side ? at.lop[d] : at.lo[d];
        n[d] = side ? at.np[d] : at.n[d];
        tlo[d] = side ? pa.tloB[d] : pa.tloA[d];
        tn[d] = side ? pa.tnB[d] : pa.tnA[d];
    }
    const int64_t tab = side ? pa.tabB : pa.tabA;
    const int64_t segc = side ? at.segPc : at.segLc, segf = side ? at.segPf : at.segLf;
    const int64_t rowc = side ? at.rowPc : at.rowLc, rowf = side ? at.rowPf : at.rowLf;
    const int nsegc = side ? at.nsegPc : at.nsegLc, nsegf = side ? at.nsegPf : at.nsegLf;
    const int nc = side ? at.ncP : at.ncL, nf = side ? at.nfP : at.nfL;
    const int nrows = n[1] * n[2];
    // row tables of the region: rows (y, z) -> segments (x0, x1, offset in the part)
    const int32_t* rpc;
    const int32_t* rpf;
    const Seg* sgc;
    const Seg* sgf;
    int64_t rp_n, sgc_n, sgf_n;                        // extents for the checked build
    if (a.smem) {
        int32_t* s_rpc = reinterpret_cast<int32_t*>(smem_raw);
        int32_t* s_rpf = s_rpc + nrows + 1;
        Seg* s_sgc = reinterpret_cast<Seg*>(smem_raw + ((8 * (static_cast<size_t>(nrows) + 1) + 15) / 16) * 16);
        Seg* s_sgf = s_sgc + nsegc;
        for (int i = threadIdx.x; i <= nrows; i += blockDim.x) {
            s_rpc[i] = LD(a.rowptr, rowc + i, a.rowptr_n);
            s_rpf[i] = LD(a.rowptr, rowf + i, a.rowptr_n);
        }
        for (int i = threadIdx.x; i < nsegc; i += blockDim.x) s_sgc[i] = LD(a.seg, segc + i, a.seg_n);
        for (int i = threadIdx.x; i < nsegf; i += blockDim.x) s_sgf[i] = LD(a.seg, segf + i, a.seg_n);
        __syncthreads();
        rpc = s_rpc;
        rpf = s_rpf;
        sgc = s_sgc;
        sgf = s_sgf;
        rp_n = nrows + 1;
        sgc_n = nsegc;
        sgf_n = nsegf;
    } else {
        rpc = a.rowptr + rowc;
        rpf = a.rowptr + rowf;
        sgc = a.seg + segc;
        sgf = a.seg + segf;
        rp_n = a.rowptr_n - rowc;
        sgc_n = a.seg_n - segc;
        sgf_n = a.seg_n - segf;
    }
    const T* __restrict__ src = static_cast<const T*>(side ? a.hphi : a.phi);
    const int64_t src_n = side ? a.hphi_n : a.phi_n;
    const int64_t* offs = side ? a.off_Lp : a.off_L;
    T* __restrict__ dst = static_cast<T*>(side ? a.PQ : a.PA);
    const int64_t dst_n = side ? a.PQ_n : a.PA_n;
    (void)dst;
    (void)src_n;
    const int TE = a.tile, T2 = TE * TE, T3 = T2 * TE;
    int64_t of4[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) of4[j] = j < pa.nsf ? LD(offs, pa.f0 + j, a.n_sf + 1) : 0;
    // tile-z layers of the box inside the slab; one warp per tile of the box
    const int z0 = max(tlo[2], a.tz0), z1 = min(tlo[2] + tn[2], a.tz1);
    const int nbox = tn[0] * tn[1] * max(0, z1 - z0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int e = warp; e < nbox; e += PK_THREADS / 32) {
        const int ex = e % tn[0], ey = (e / tn[0]) % tn[1], ez = z0 - tlo[2] + e / (tn[0] * tn[1]);
        const int2 ent = LD(a.ttab, tab + ex + static_cast<int64_t>(tn[0]) * (ey + static_cast<int64_t>(tn[1]) * ez),
                            a.ttab_n);
        if (ent.x < 0) continue;
        const PanelTile tl = LD(a.tiles, ent.x, a.n_tiles);
        const int kp = tl.kp;
        const int64_t base = (side ? tl.pQ : tl.pA) + static_cast<int64_t>(ent.y) * kp;
        // offset of panel entry k inside a compressed function of the atom (-1: not a member)
        auto rel_of = [&](int k) -> int64_t {
            int64_t rel = -1;
            int x = 0, y = 0, z = 0, t = 0;
            bool coarse = k < T3, valid = false;
            if (coarse) {
                x = tl.org[0] + k % TE - lo[0];
                y = tl.org[1] + (k / TE) % TE - lo[1];
                z = tl.org[2] + k / T2 - lo[2];
                valid = true;
            } else {
                const int q = (k - T3) / 7;
                t = (k - T3) - 7 * q;
                if (q < tl.nfine) {
                    const int code = LD(a.tile_fine, tl.fine0 + q, a.fine_n);
                    x = tl.org[0] + (code & 255) - lo[0];
                    y = tl.org[1] + ((code >> 8) & 255) - lo[1];
                    z = tl.org[2] + (code >> 16) - lo[2];
                    valid = true;
                }
            }
            if (valid && x >= 0 && y >= 0 && z >= 0 && x < n[0] && y < n[1] && z < n[2]) {
                const int row = y + n[1] * z;
                const int32_t* rp = coarse ? rpc : rpf;
                const Seg* sg = coarse ? sgc : sgf;
                const int s0 = LD(rp, row, rp_n), s1 = LD(rp, row + 1, rp_n);
                for (int s = s0; s < s1; ++s) {
                    const Seg g = LD(sg, s, coarse ? sgc_n : sgf_n);
                    if (x >= g.x0 && x <= g.x1) {
                        rel = coarse ? g.off + (x - g.x0) : nc + g.off + (x - g.x0) + static_cast<int64_t>(t) * nf;
                        break;
                    }
                }
            }
            return rel;
        };
        if constexpr (Unpack) {
            for (int k = lane; k < kp; k += 32) {
                // combination result: panel row of the A side (in the Q buffer) -> members of L
                const int64_t rel = rel_of(k);
                if (rel >= 0)
                    for (int j = 0; j < pa.nsf; ++j) {
                        const int64_t o = LD(offs, pa.f0 + j, a.n_sf + 1);
                        ST(out, o + rel, a.out_n, LD(static_cast<const T*>(a.PQ), base + static_cast<int64_t>(j) * kp + k, a.PQ_n));
                    }
            }
        } else {
            // 4 entries per lane and 4 functions at a time: 16 loads in flight before the stores
            for (int kb = lane; kb < kp; kb += 128) {
                int64_t rel[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) rel[u] = kb + 32 * u < kp ? rel_of(kb + 32 * u) : -1;
                for (int j0 = 0; j0 < pa.nsf; j0 += 4) {
                    T v[4][4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int64_t o = j0 + j < pa.nsf ? (j0 + j < 4 ? of4[j] : LD(offs, pa.f0 + j0 + j, a.n_sf + 1)) : 0;
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            v[u][j] = (rel[u] >= 0 && j0 + j < pa.nsf) ? LD(src, o + rel[u], src_n) : T(0);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if (kb + 32 * u < kp && j0 + j < pa.nsf)
                                ST(dst, base + static_cast<int64_t>(j0 + j) * kp + kb + 32 * u, dst_n, v[u][j]);
                }
            }
        }
    }
}

// ---------------------------------------------------------------- products

constexpr int PH_M = 64;        // A rows per item
constexpr int PH_N = 128;       // columns per item
constexpr int PH_KC = 32;       // panel entries per chunk
constexpr int PH_LDA = PH_M + 4;
constexpr int PH_LDC = PH_N + 4;

// 4 consecutive panel values (16-byte aligned): one float4, or two double2
template <class T>
struct Quad;
template <>
struct Quad<float> {
    float4 v;
    __device__ __forceinline__ void load(const float* p) { v = *reinterpret_cast<const float4*>(p); }
    __device__ __forceinline__ void zero() { v = make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ __forceinline__ float operator[](int i) const { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
};
template <>
struct Quad<double> {
    double2 v0, v1;
    __device__ __forceinline__ void load(const double* p) {
        v0 = reinterpret_cast<const double2*>(p)[0];
        v1 = reinterpret_cast<const double2*>(p)[1];
    }
    __device__ __forceinline__ void zero() { v0 = v1 = make_double2(0.0, 0.0); }
    __device__ __forceinline__ double operator[](int i) const { return i == 0 ? v0.x : i == 1 ? v0.y : i == 2 ? v1.x : v1.y; }
};

template <class T>
__device__ __forceinline__ void ld4(Quad<T>& q, const T* p, int64_t i, int64_t n, [[maybe_unused]] int* ST_,
                                    [[maybe_unused]] int kid) {
#ifdef LSW_CHECKED
    if (i < 0 || i + 4 > n || (i & 3)) {
        lsw_report(ST_, kid, __LINE__, i, n);
        q.zero();
        return;
    }
#endif
    q.load(p + i);
}

template <class T>
__global__ void __launch_bounds__(256) k_panel_hs(PanelHSLaunch a) {
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = 11;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sA = reinterpret_cast<T*>(smem_raw);            // [KC][LDA]: A rows, transposed
    T* sC = sA + PH_KC * PH_LDA;                       // [KC][LDC]: [A; Q] columns, transposed
    constexpr int SA_N = PH_KC * PH_LDA, SC_N = PH_KC * PH_LDC;
    const PanelItem it = LD(a.items, blockIdx.x, a.nitems);
    const PanelTile tl = LD(a.tiles, it.tile, a.n_tiles);
    const int kp = tl.kp;
    const T* PA = static_cast<const T*>(a.PA);
    const T* PQ = static_cast<const T*>(a.PQ);
    const int tid = threadIdx.x;
    // loaders: A row tid & 63 (k groups (tid >> 6) + 4m), C row tid & 127 (k groups (tid >> 7) + 2m)
    const int ra = tid & 63, ga = tid >> 6;
    const int rc = tid & 127, gc = tid >> 7;
    const bool a_ok = ra < it.na, c_ok = rc < it.nc;
    const int cc = it.c0 + rc;
    const bool c_in_a = cc < tl.nA;
    const int64_t offA = tl.pA + static_cast<int64_t>(it.a0 + ra) * kp;
    const int64_t offC = c_in_a ? tl.pA + static_cast<int64_t>(cc) * kp : tl.pQ + static_cast<int64_t>(cc - tl.nA) * kp;
    const int64_t nC = c_in_a ? a.PA_n : a.PQ_n;
    Quad<T> qa[2], qc[4];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int k = k0 + 4 * (ga + 4 * m);
            if (a_ok && k < kp) ld4(qa[m], PA, offA + k, a.PA_n, ST_, KID); else qa[m].zero();
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int k = k0 + 4 * (gc + 2 * m);
            if (c_ok && k < kp) ld4(qc[m], c_in_a ? PA : PQ, offC + k, nC, ST_, KID); else qc[m].zero();
        }
    };
    const int ti = tid >> 4, tj = tid & 15;
    const bool wide = it.nc > 64;                      // block-uniform: second column half in use
    T acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = T(0);
    fetch(0);
    for (int k0 = 0; k0 < kp; k0 += PH_KC) {
        // registers -> shared, transposed ([k][row])
#pragma unroll
        for (int m = 0; m < 2; ++m)
#pragma unroll
            for (int e = 0; e < 4; ++e) ST(sA, (4 * (ga + 4 * m) + e) * PH_LDA + ra, SA_N, qa[m][e]);
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int e = 0; e < 4; ++e) ST(sC, (4 * (gc + 2 * m) + e) * PH_LDC + rc, SC_N, qc[m][e]);
        __syncthreads();
        if (k0 + PH_KC < kp) fetch(k0 + PH_KC);         // next chunk in flight during the products
        const int kn = min(PH_KC, kp - k0);
#ifndef LSW_CHECKED
        if constexpr (sizeof(T) == 4) {
            // 16-byte shared loads (the 4 rows and 2 x 4 columns of this thread) and packed
            // two-lane FMAs (each lane one FMA rounded to nearest: the same bits as below)
#pragma unroll 4
            for (int k = 0; k < kn; ++k) {
                const float4 a4 = *reinterpret_cast<const float4*>(sA + k * PH_LDA + 4 * ti);
                const float4 c4 = *reinterpret_cast<const float4*>(sC + k * PH_LDC + 4 * tj);
                const float av[4] = {a4.x, a4.y, a4.z, a4.w};
                if (wide) {
                    const float4 d4 = *reinterpret_cast<const float4*>(sC + k * PH_LDC + 64 + 4 * tj);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float2 ai = make_float2(av[i], av[i]);
                        float2 r0 = __ffma2_rn(ai, make_float2(c4.x, c4.y), make_float2(acc[i][0], acc[i][1]));
                        float2 r1 = __ffma2_rn(ai, make_float2(c4.z, c4.w), make_float2(acc[i][2], acc[i][3]));
                        float2 r2 = __ffma2_rn(ai, make_float2(d4.x, d4.y), make_float2(acc[i][4], acc[i][5]));
                        float2 r3 = __ffma2_rn(ai, make_float2(d4.z, d4.w), make_float2(acc[i][6], acc[i][7]));
                        acc[i][0] = r0.x, acc[i][1] = r0.y, acc[i][2] = r1.x, acc[i][3] = r1.y;
                        acc[i][4] = r2.x, acc[i][5] = r2.y, acc[i][6] = r3.x, acc[i][7] = r3.y;
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float2 ai = make_float2(av[i], av[i]);
                        float2 r0 = __ffma2_rn(ai, make_float2(c4.x, c4.y), make_float2(acc[i][0], acc[i][1]));
                        float2 r1 = __ffma2_rn(ai, make_float2(c4.z, c4.w), make_float2(acc[i][2], acc[i][3]));
                        acc[i][0] = r0.x, acc[i][1] = r0.y, acc[i][2] = r1.x, acc[i][3] = r1.y;
                    }
                }
            }
        } else
#endif
        {
            for (int k = 0; k < kn; ++k) {
                T av[4], cv[8];
#pragma unroll
                for (int i = 0; i < 4; ++i) av[i] = LD(sA, k * PH_LDA + 4 * ti + i, SA_N);
#pragma unroll
                for (int j = 0; j < 4; ++j) cv[j] = LD(sC, k * PH_LDC + 4 * tj + j, SC_N);
                if (wide) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) cv[4 + j] = LD(sC, k * PH_LDC + 64 + 4 * tj + j, SC_N);
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 8; ++j) acc[i][j] = fma(av[i], cv[j], acc[i][j]);
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], cv[j], acc[i][j]);
                }
            }
        }
        __syncthreads();
    }
    // pattern positions: the CSR rows of this item's A functions in shared memory (rows
    // that do not fit are searched in global memory), then one FP64 atomic add per entry
    __shared__ int rofs[PH_M + 1];
    __shared__ int rlen[PH_M];
    __shared__ long long rbase[PH_M];
    int* rcols = reinterpret_cast<int*>(smem_raw);
    const int rcap = static_cast<int>((SA_N + SC_N) * sizeof(T) / sizeof(int));
    if (tid < it.na) {
        const int fa = LD(a.listA, tl.listA + it.a0 + tid, a.listA_n);
        const int64_t r0 = LD(a.row_ptr, fa, a.n_sf + 1), r1 = LD(a.row_ptr, fa + 1, a.n_sf + 1);
        rbase[tid] = r0;
        rlen[tid] = static_cast<int>(r1 - r0);
    }
    __syncthreads();
    if (tid == 0) {
        int o = 0;
        for (int i = 0; i < it.na; ++i) {
            rofs[i] = o;
            if (o + rlen[i] <= rcap) o += rlen[i];
            else rofs[i] = -1;
        }
    }
    __syncthreads();
    for (int i = tid >> 5; i < it.na; i += blockDim.x >> 5) {
        if (rofs[i] < 0) continue;
        for (int k = tid & 31; k < rlen[i]; k += 32) ST(rcols, rofs[i] + k, rcap, LD(a.col, rbase[i] + k, a.nnz));
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = 4 * ti + i;
        if (r >= it.na) continue;
        const int64_t r0 = rbase[r];
        const int ro = rofs[r], rl = rlen[r];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = j < 4 ? 4 * tj + j : 64 + 4 * tj + (j - 4);
            if (c >= it.nc) continue;
            const int cg = it.c0 + c;
            const bool isS = cg < tl.nA;
            const int fb = isS ? LD(a.listA, tl.listA + cg, a.listA_n) : LD(a.listB, tl.listB + (cg - tl.nA), a.listB_n);
            int lo = 0, hi = rl - 1;
            int64_t pos = -1;
            while (lo <= hi) {
                const int mid = (lo + hi) >> 1;
                const int cm = ro >= 0 ? LD(rcols, ro + mid, rcap) : LD(a.col, r0 + mid, a.nnz);
                if (cm == fb) {
                    pos = r0 + mid;
                    break;
                }
                if (cm < fb) lo = mid + 1;
                else hi = mid - 1;
            }
            if (pos < 0 || acc[i][j] == T(0)) continue;
            atomicAdd((isS ? a.S : a.H) + pos, static_cast<double>(acc[i][j]));
        }
    }
}

// ---------------------------------------------------------------- products on the tensor cores

// k_panel_hs for FP32 panels on the tensor cores: per work item (tile, up to 64 A rows,
// up to 128 columns of [A; Q]) the product D[c][a] = sum_k C[c][k] A[a][k] (C the [A; Q]
// rows, A the item's A rows) runs as tcgen05.mma kind::f16 with M = 128 (the C rows), N
// = the A rows rounded up to 16, K = 16 per instruction, from split-bfloat16 operands:
// each FP32 panel value is split into 3 bfloat16 parts (each part the rounding of what
// the previous ones leave) and the 6 products of parts whose orders add up to at most 2
// are accumulated in FP32 in tensor memory (relative error of a product about 2^-24).
// The tensor cores' FP32 accumulation rounds each addition (measured: about 3e-6 of a
// sum of 300 terms when every product goes into one accumulator, biased low), so the
// leading product (part 0 x part 0) of each chunk of 32 panel entries goes into an
// accumulator of its own, read into registers after the chunk (2 additions per chunk in
// tensor memory, the chunks summed in FP32 registers), while the 5 correction products,
// 2^-8 smaller, share one accumulator over the whole panel row.  The panel rows are
// K-major, the layout the instruction reads: thread t converts (row, 8 panel entries)
// units straight into the canonical core-matrix layout.  Two operand buffers (and two
// leading-product accumulators) alternate, so the conversion of one chunk overlaps the
// products of the previous one.  Waits on MMA completion are bounded (about 1 s) and end
// in a status bit.  The epilogue holds, per thread, the sums of its C row c = 32 (w mod
// 4) + l (warp w, lane l) over half w / 4 of the A rows, and adds each pattern entry as
// in k_panel_hs.
constexpr int PT_M = 128, PT_N = 64, PT_KC = 32, PT_NS = 3;
constexpr int PT_APART = PT_M * PT_KC * 2;                 // bytes of one bfloat16 part of the C operand
constexpr int PT_BPART = PT_N * PT_KC * 2;                 // ... of the A operand
constexpr int PT_STAGE = PT_NS * (PT_APART + PT_BPART);    // one buffer
constexpr int PT_SMEM = tc::HEAD + 2 * PT_STAGE;
constexpr int PT_TCOLS = 256;                              // tensor memory: lead[2] at 0, 64; corrections at 128
constexpr int PT_U = (PT_M + PT_N) * (PT_KC / 8) / 256;    // operand units per thread and chunk

__global__ void __launch_bounds__(256, 2) k_panel_hs_tc(PanelHSLaunch a) {
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = 21;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const PanelItem it = LD(a.items, blockIdx.x, a.nitems);
    const PanelTile tl = LD(a.tiles, it.tile, a.n_tiles);
    const int kp = tl.kp;
    const int nN = (it.na + 15) & ~15;                      // MMA N (A rows, padded)
    const float* PA = static_cast<const float*>(a.PA);
    const float* PQ = static_cast<const float*>(a.PQ);
    const uint32_t mb0 = tc::saddr(smem_raw), mb1 = tc::saddr(smem_raw + 8);
    if (warp == 0) tc::tmem_alloc(tc::saddr(smem_raw + 16), PT_TCOLS);
    if (tid == 32) {
        tc::mbar_init(mb0);
        tc::mbar_init(mb1);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(smem_raw + 16);
    unsigned char* stage[2] = {smem_raw + tc::HEAD, smem_raw + tc::HEAD + PT_STAGE};
    const int64_t room = PT_SMEM;
    const uint32_t id = tc::idesc(PT_M, nN);
    const int nch = (kp + PT_KC - 1) / PT_KC;
    // this thread's tensor-memory lane and columns of the accumulators
    const uint32_t tlane = tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16);
    const int jbase = (warp >> 2) * (PT_N / 2);
    const bool jlive = jbase < nN;                          // warp-uniform
    float sum[PT_N / 2];
#pragma unroll
    for (int j = 0; j < PT_N / 2; ++j) sum[j] = 0.f;
    auto read_lead = [&](int sbuf) {                        // sum += leading-product chunk in lead[sbuf]
        if (!jlive) return;
#pragma unroll
        for (int g = 0; g < PT_N / 16; ++g) {
            float v[8];
            tc::tmem_ld8(tlane + sbuf * PT_N + jbase + 8 * g, v);
#pragma unroll
            for (int e = 0; e < 8; ++e) sum[8 * g + e] += v[e];
        }
    };
    // operand units of a chunk: 128 C rows x 4 groups of 8 entries, then 64 A rows x 4
    // groups; thread t takes units t + 256 m, m < PT_U.  Unit uu is row (uu & 7) + 8 (uu >>
    // 5) and group (uu >> 3) & 3, so the 8 threads of a 16-byte store phase write the 8
    // rows of one core matrix: 128 contiguous bytes, every bank once (with the 4 groups of
    // a row on consecutive threads, the phase's rows fell 128 bytes apart, on 4 banks)
    Quad<float> pre[PT_U][2];
    auto unit = [&](int m, bool& isC, int& row, int& g) {
        const int u = tid + m * 256;
        isC = u < PT_M * (PT_KC / 8);
        const int uu = isC ? u : u - PT_M * (PT_KC / 8);
        row = (uu & 7) + 8 * (uu >> 5);
        g = (uu >> 3) & 3;
    };
    auto fetch = [&](int chn) {
        const int k0 = chn * PT_KC;
#pragma unroll
        for (int m = 0; m < PT_U; ++m) {
            bool isC;
            int row, g;
            unit(m, isC, row, g);
            const int k = k0 + 8 * g;
            bool have = k < kp;
            const float* src;
            int64_t off, n;
            if (isC) {
                const int cc = it.c0 + row;
                have = have && row < it.nc;
                const bool inA = cc < tl.nA;
                src = inA ? PA : PQ;
                off = inA ? tl.pA + static_cast<int64_t>(cc) * kp : tl.pQ + static_cast<int64_t>(cc - tl.nA) * kp;
                n = inA ? a.PA_n : a.PQ_n;
            } else {
                have = have && row < it.na;
                src = PA;
                off = tl.pA + static_cast<int64_t>(it.a0 + row) * kp;
                n = a.PA_n;
            }
            if (have) ld4(pre[m][0], src, off + k, n, ST_, KID);
            else pre[m][0].zero();
            if (have && k + 4 < kp) ld4(pre[m][1], src, off + k + 4, n, ST_, KID);
            else pre[m][1].zero();
        }
    };
    fetch(0);
    bool ok = true;
    uint32_t phase[2] = {0, 0};
    for (int ch = 0; ch < nch && ok; ++ch) {
        const int s = ch & 1;
        if (ch >= 2) {   // the products of chunk ch - 2 (this buffer, this lead accumulator) are done
            ok = tc::mbar_wait(s ? mb1 : mb0, phase[s]);
            phase[s] ^= 1;
            if (!__syncthreads_and(ok)) break;
            tc::fence_after();
            read_lead(s);
        }
        unsigned char* sA = stage[s];                        // C rows: M operand
        unsigned char* sB = stage[s] + PT_NS * PT_APART;     // A rows: N operand
        // this chunk's values are in registers (loaded during the previous chunk): split
        // and store them, then load the next chunk's (in flight during the products)
#pragma unroll
        for (int m = 0; m < PT_U; ++m) {
            bool isC;
            int row, g;
            unit(m, isC, row, g);
            float x[8];
#pragma unroll
            for (int e = 0; e < 4; ++e) x[e] = pre[m][0][e], x[4 + e] = pre[m][1][e];
            if (isC) tc::put8<PT_NS>(sA, PT_APART, tc::core_off(row, 8 * g, PT_KC), x, ST_, room - (sA - smem_raw));
            else tc::put8<PT_NS>(sB, PT_BPART, tc::core_off(row, 8 * g, PT_KC), x, ST_, room - (sB - smem_raw));
        }
        if (ch + 1 < nch) fetch(ch + 1);
        tc::fence_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (tid == 0) {
            for (int kk = 0; kk < PT_KC / 16; ++kk)
#pragma unroll
                for (int t = 0; t < tc::Terms<PT_NS>::n; ++t) {
                    const int pa_ = tc::Terms<PT_NS>::b(t), pb_ = tc::Terms<PT_NS>::a(t);
                    const bool lead = pa_ == 0 && pb_ == 0;
                    const uint32_t d = tmem + (lead ? static_cast<uint32_t>(s * PT_N) : 2u * PT_N);
                    tc::mma(d, tc::sdesc(tc::saddr(sA + pa_ * PT_APART + kk * 256), PT_KC),
                            tc::sdesc(tc::saddr(sB + pb_ * PT_BPART + kk * 256), PT_KC), id,
                            lead ? kk > 0 : (ch > 0 || kk > 0 || t > 1));
                }
            tc::commit(s ? mb1 : mb0);
        }
    }
    // the last two chunks' products
    if (ok) {
        for (int ch = (nch >= 2 ? nch - 2 : 0); ch < nch && ok; ++ch) {
            const int s = ch & 1;
            ok = tc::mbar_wait(s ? mb1 : mb0, phase[s]);
            phase[s] ^= 1;
            if (!__syncthreads_and(ok)) break;
            tc::fence_after();
            read_lead(s);
        }
    }
    if (!__syncthreads_and(ok)) {
        if (tid == 0) atomicOr(a.status, ST_WAIT_TIMEOUT);
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (warp == 0) tc::tmem_free(tmem, PT_TCOLS);
        return;
    }
    // the correction products
    if (jlive) {
#pragma unroll
        for (int g = 0; g < PT_N / 16; ++g) {
            float v[8];
            tc::tmem_ld8(tlane + 2 * PT_N + jbase + 8 * g, v);
#pragma unroll
            for (int e = 0; e < 8; ++e) sum[8 * g + e] += v[e];
        }
    }
    // pattern positions: the CSR rows of this item's A functions in the (now free) operand
    // buffers, rows that do not fit searched in global memory
    __shared__ int rofs[64 + 1];
    __shared__ int rlen[64];
    __shared__ long long rbase[64];
    int* rcols = reinterpret_cast<int*>(smem_raw + tc::HEAD);
    const int rcap = 2 * PT_STAGE / static_cast<int>(sizeof(int));
    if (tid < it.na) {
        const int fa = LD(a.listA, tl.listA + it.a0 + tid, a.listA_n);
        const int64_t r0 = LD(a.row_ptr, fa, a.n_sf + 1), r1 = LD(a.row_ptr, fa + 1, a.n_sf + 1);
        rbase[tid] = r0;
        rlen[tid] = static_cast<int>(r1 - r0);
    }
    __syncthreads();
    if (tid == 0) {
        int o = 0;
        for (int i = 0; i < it.na; ++i) {
            rofs[i] = o;
            if (o + rlen[i] <= rcap) o += rlen[i];
            else rofs[i] = -1;
        }
    }
    __syncthreads();
    for (int i = warp; i < it.na; i += blockDim.x >> 5) {
        if (rofs[i] < 0) continue;
        for (int k = lane; k < rlen[i]; k += 32) ST(rcols, rofs[i] + k, rcap, LD(a.col, rbase[i] + k, a.nnz));
    }
    __syncthreads();
    const int c = 32 * (warp & 3) + lane;                   // C row of this thread (tensor-memory lane)
    const int cg = it.c0 + c;
    if (jlive && c < it.nc) {
        const bool isS = cg < tl.nA;
        const int fb = isS ? LD(a.listA, tl.listA + cg, a.listA_n) : LD(a.listB, tl.listB + (cg - tl.nA), a.listB_n);
#pragma unroll
        for (int e = 0; e < PT_N / 2; ++e) {
            const int r = jbase + e;
            if (r >= it.na || sum[e] == 0.f) continue;
            const int64_t r0 = rbase[r];
            const int ro = rofs[r];
            int lo = 0, hi = rlen[r] - 1;
            int64_t pos = -1;
            while (lo <= hi) {
                const int mid = (lo + hi) >> 1;
                const int cm = ro >= 0 ? LD(rcols, ro + mid, rcap) : LD(a.col, r0 + mid, a.nnz);
                if (cm == fb) {
                    pos = r0 + mid;
                    break;
                }
                if (cm < fb) lo = mid + 1;
                else hi = mid - 1;
            }
            if (pos >= 0) atomicAdd((isS ? a.S : a.H) + pos, static_cast<double>(sum[e]));
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_free(tmem, PT_TCOLS);
}

// ---------------------------------------------------------------- sparse combination

// (M Phi)_a = P_L(a) sum_b M_ab phi_b (Sec. "Orthogonalization", Eq. gradient): per work
// item (tile, up to 64 A rows, up to 128 panel entries starting at c0), the A panel's
// rows combined with the coefficients M_ab of the tile's A functions (looked up in the
// pattern CSR, 0 outside it), written to the output panel at the A panel's place in the
// Q buffer; the unpack then copies each member of L(a) from the tile holding it.
template <class T>
__global__ void __launch_bounds__(256) k_panel_combine(PanelHSLaunch a) {
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = 13;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sM = reinterpret_cast<T*>(smem_raw);            // [KC][LDA]: M[a0 + i][j0 + j] at [j][i]
    T* sP = sM + PH_KC * PH_LDA;                       // [KC][LDC]: PA[j0 + j][c0 + c] at [j][c]
    constexpr int SM_N = PH_KC * PH_LDA, SP_N = PH_KC * PH_LDC;
    const PanelItem it = LD(a.items, blockIdx.x, a.nitems);
    const PanelTile tl = LD(a.tiles, it.tile, a.n_tiles);
    const int kp = tl.kp;
    const T* PA = static_cast<const T*>(a.PA);
    T* PO = static_cast<T*>(const_cast<void*>(a.PQ));
    const int tid = threadIdx.x;
    const int ti = tid >> 4, tj = tid & 15;
    const bool wide = it.nc > 64;
    T acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = T(0);
    for (int j0 = 0; j0 < tl.nA; j0 += PH_KC) {
        const int nj = min(PH_KC, tl.nA - j0);
        // coefficients: thread (i = tid & 63, j = tid >> 6 + 4 m)
        {
            const int i = tid & 63;
            int64_t r0 = 0, r1 = 0;
            if (i < it.na) {
                const int fa = LD(a.listA, tl.listA + it.a0 + i, a.listA_n);
                r0 = LD(a.row_ptr, fa, a.n_sf + 1);
                r1 = LD(a.row_ptr, fa + 1, a.n_sf + 1);
            }
            for (int j = tid >> 6; j < PH_KC; j += 4) {
                T m = T(0);
                if (i < it.na && j < nj) {
                    const int fb = LD(a.listA, tl.listA + j0 + j, a.listA_n);
                    int64_t lo = r0, hi = r1 - 1;
                    while (lo <= hi) {
                        const int64_t mid = (lo + hi) >> 1;
                        const int cm = LD(a.col, mid, a.nnz);
                        if (cm == fb) {
                            m = static_cast<T>(LD(a.M, mid, a.nnz));
                            break;
                        }
                        if (cm < fb) lo = mid + 1;
                        else hi = mid - 1;
                    }
                }
                ST(sM, j * PH_LDA + i, SM_N, m);
            }
        }
        // panel rows j0 .. j0 + nj, entries c0 .. c0 + nc: thread (row j = tid >> 3, quad q = tid & 7 + 8 m)
        {
            const int j = tid >> 3;
            for (int q = tid & 7; q < PH_N / 4; q += 8) {
                const int c = 4 * q;
                Quad<T> v;
                if (j < nj && c < it.nc) ld4(v, PA, tl.pA + static_cast<int64_t>(j0 + j) * kp + it.c0 + c, a.PA_n, ST_, KID);
                else v.zero();
#pragma unroll
                for (int e = 0; e < 4; ++e) ST(sP, j * PH_LDC + c + e, SP_N, v[e]);
            }
        }
        __syncthreads();
        for (int j = 0; j < nj; ++j) {
            T av[4], cv[8];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = LD(sM, j * PH_LDA + 4 * ti + i, SM_N);
#pragma unroll
            for (int c = 0; c < 4; ++c) cv[c] = LD(sP, j * PH_LDC + 4 * tj + c, SP_N);
            if (wide) {
#pragma unroll
                for (int c = 0; c < 4; ++c) cv[4 + c] = LD(sP, j * PH_LDC + 64 + 4 * tj + c, SP_N);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int c = 0; c < 8; ++c) acc[i][c] = fma(av[i], cv[c], acc[i][c]);
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[i][c] = fma(av[i], cv[c], acc[i][c]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = 4 * ti + i;
        if (r >= it.na) continue;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int cc = c < 4 ? 4 * tj + c : 64 + 4 * tj + (c - 4);
            if (cc >= it.nc) continue;
            ST(PO, tl.pA + static_cast<int64_t>(it.a0 + r) * kp + it.c0 + cc, a.PQ_n, acc[i][c]);
        }
    }
}

// ---------------------------------------------------------------- host entry points

#define TRACED(TR, KIND, S, LAUNCH) \
    do {                                \
        trace_begin(TR, KIND, S);       \
        LAUNCH;                         \
        trace_end(TR, S);               \
    } while (0)

size_t panel_hs_smem(int prec) {
    return static_cast<size_t>(PH_KC) * (PH_LDA + PH_LDC) * (prec == 0 ? sizeof(double) : sizeof(float));
}

cudaError_t configure_panel_kernels(size_t max_smem) {
    cudaError_t e;
    const void* ks[] = {reinterpret_cast<const void*>(k_pack<double, false>),
                        reinterpret_cast<const void*>(k_pack<float, false>),
                        reinterpret_cast<const void*>(k_pack<double, true>),
                        reinterpret_cast<const void*>(k_pack<float, true>),
                        reinterpret_cast<const void*>(k_panel_hs<double>),
                        reinterpret_cast<const void*>(k_panel_hs<float>),
                        reinterpret_cast<const void*>(k_panel_combine<double>),
                        reinterpret_cast<const void*>(k_panel_combine<float>),
                        reinterpret_cast<const void*>(k_panel_hs_tc)};
    for (const void* k : ks) {
        cudaFuncAttributes fa;
        if ((e = cudaFuncGetAttributes(&fa, k)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(max_smem - fa.sharedSizeBytes))) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

cudaError_t enqueue_pack(const PackLaunch& a, cudaStream_t s) {
    if (a.n_slab_atoms == 0) return cudaSuccess;
    const dim3 grid(static_cast<unsigned>(a.n_slab_atoms), a.hphi && !a.out ? 2 : 1);
    if (a.out) {
        if (a.prec == 0)
            TRACED(a.tr, TK_PACK, s, (k_pack<double, true><<<grid, PK_THREADS, a.smem, s>>>(a)));
        else
            TRACED(a.tr, TK_PACK, s, (k_pack<float, true><<<grid, PK_THREADS, a.smem, s>>>(a)));
    } else if (a.prec == 0) {
        TRACED(a.tr, TK_PACK, s, (k_pack<double, false><<<grid, PK_THREADS, a.smem, s>>>(a)));
    } else {
        TRACED(a.tr, TK_PACK, s, (k_pack<float, false><<<grid, PK_THREADS, a.smem, s>>>(a)));
    }
    return cudaGetLastError();
}

cudaError_t enqueue_panel_combine(const PanelHSLaunch& a, cudaStream_t s) {
    if (a.nitems == 0) return cudaSuccess;
    const size_t smem = panel_hs_smem(a.prec);
    if (a.prec == 0)
        TRACED(a.tr, TK_HS, s, (k_panel_combine<double><<<static_cast<unsigned>(a.nitems), 256, smem, s>>>(a)));
    else
        TRACED(a.tr, TK_HS, s, (k_panel_combine<float><<<static_cast<unsigned>(a.nitems), 256, smem, s>>>(a)));
    return cudaGetLastError();
}

// T_ab = (3 delta_ab - S_ab) / 2 on the pattern: the first-order Taylor S^-1/2 of the
// Loewdin step (Sec. "Orthogonalization")
__global__ void k_lowdin_coeffs(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                const double* __restrict__ S, double* __restrict__ T, int n_sf) {
    const int a = blockIdx.x * blockDim.y + threadIdx.y;
    if (a >= n_sf) return;
    for (int64_t k = row_ptr[a] + threadIdx.x; k < row_ptr[a + 1]; k += blockDim.x)
        T[k] = (3.0 * (col[k] == a ? 1.0 : 0.0) - S[k]) * 0.5;
}

cudaError_t enqueue_lowdin_coeffs(const int64_t* row_ptr, const int32_t* col, const double* S, double* T, int n_sf,
                                  cudaStream_t s) {
    if (n_sf == 0) return cudaSuccess;
    k_lowdin_coeffs<<<(n_sf + 7) / 8, dim3(32, 8), 0, s>>>(row_ptr, col, S, T, n_sf);
    return cudaGetLastError();
}

cudaError_t enqueue_panel_hs(const PanelHSLaunch& a, cudaStream_t s) {
    if (a.nitems == 0) return cudaSuccess;
    const size_t smem = panel_hs_smem(a.prec);
    if (a.prec != 0 && a.tc) {
        TRACED(a.tr, TK_HS, s, (k_panel_hs_tc<<<static_cast<unsigned>(a.nitems), 256, PT_SMEM, s>>>(a)));
        return cudaGetLastError();
    }
    if (a.prec == 0)
        TRACED(a.tr, TK_HS, s, (k_panel_hs<double><<<static_cast<unsigned>(a.nitems), 256, smem, s>>>(a)));
    else
        TRACED(a.tr, TK_HS, s, (k_panel_hs<float><<<static_cast<unsigned>(a.nitems), 256, smem, s>>>(a)));
    return cudaGetLastError();
}

}  // namespace lsw
