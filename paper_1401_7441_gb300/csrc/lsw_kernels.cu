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
//   k_bwd_xy      per coarse z plane of L': transposed filters along y then x -> G
//   k_kinetic     G += -1/(2h^2) sum_d T_{b_d b'_d} along d on D (E_kin = <phi|T phi>)
//   k_compress    G on the members of L' -> compressed H phi
//   k_hs          per grid tile (App. D "transposed" layout): panels of phi and
//                 H phi of the functions touching the tile; S_ab += <phi_a|phi_b>,
//                 H_ab += <phi_a|H phi_b> over the tile; FP64 accumulation
//
// All kernels are templated on the storage/compute type T (double or float); energy
// and matrix accumulations are FP64.  Device-side checks set bits of a status word
// (never trap).
#include <cstdint>

#include "lsw_internal.h"

namespace lsw {

__constant__ double c_fwd_d[2][FWD_TAPS];
__constant__ float c_fwd_f[2][FWD_TAPS];
__constant__ double c_kin_d[4][KIN_TAPS];
__constant__ float c_kin_f[4][KIN_TAPS];

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

// ---------------------------------------------------------------- uncompress / compress

template <class T>
__global__ void k_uncompress(HphiLaunch a) {
    const FnRec r = a.fn[blockIdx.y];
    const AtomRec& at = a.atoms[r.atom];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sidx = blockIdx.x * (blockDim.x >> 5) + warp;
    const int nseg = at.nsegLc + at.nsegLf;
    if (sidx >= nseg) return;
    const bool fine = sidx >= at.nsegLc;
    const Seg sg = a.seg[fine ? at.segLf + (sidx - at.nsegLc) : at.segLc + sidx];
    const int64_t plane = static_cast<int64_t>(r.n[0]) * r.n[1] * r.n[2];
    T* D = static_cast<T*>(a.ws) + r.ws_D;
    const T* phi = static_cast<const T*>(a.phi) + r.off_phi;
    const int len = sg.x1 - sg.x0 + 1;
    if (sg.x0 < 0 || sg.x1 >= r.n[0] || sg.row < 0 || sg.row >= r.n[1] * r.n[2]) {
        if (lane == 0) atomicOr(a.status, ST_BAD_SEG);
        return;
    }
    const int64_t base = static_cast<int64_t>(sg.row) * r.n[0] + sg.x0;
    for (int k = lane; k < len; k += 32) {
        if (!fine) {
            D[base + k] = phi[sg.off + k];
        } else {
#pragma unroll
            for (int t = 1; t < 8; ++t)
                D[t * plane + base + k] = phi[at.ncL + static_cast<int64_t>(t - 1) * at.nfL + sg.off + k];
        }
    }
}

template <class T>
__global__ void k_compress(HphiLaunch a) {
    const FnRec r = a.fn[blockIdx.y];
    const AtomRec& at = a.atoms[r.atom];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sidx = blockIdx.x * (blockDim.x >> 5) + warp;
    const int nseg = at.nsegPc + at.nsegPf;
    if (sidx >= nseg) return;
    const bool fine = sidx >= at.nsegPc;
    const Seg sg = a.seg[fine ? at.segPf + (sidx - at.nsegPc) : at.segPc + sidx];
    const int64_t plane = static_cast<int64_t>(r.np[0]) * r.np[1] * r.np[2];
    const T* G = static_cast<const T*>(a.ws) + r.ws_G;
    T* out = static_cast<T*>(a.hphi) + r.off_hphi;
    const int len = sg.x1 - sg.x0 + 1;
    if (sg.x0 < 0 || sg.x1 >= r.np[0] || sg.row < 0 || sg.row >= r.np[1] * r.np[2]) {
        if (lane == 0) atomicOr(a.status, ST_BAD_SEG);
        return;
    }
    const int64_t base = static_cast<int64_t>(sg.row) * r.np[0] + sg.x0;
    for (int k = lane; k < len; k += 32) {
        if (!fine) {
            out[sg.off + k] = G[base + k];
        } else {
#pragma unroll
            for (int t = 1; t < 8; ++t)
                out[at.ncP + static_cast<int64_t>(t - 1) * at.nfP + sg.off + k] = G[t * plane + base + k];
        }
    }
}

// ---------------------------------------------------------------- forward x, y

// first a with 0 <= o - 2a <= 30, clamped to 0
__device__ __forceinline__ int up_lo(int o) { return o >= 30 ? (o - 29) >> 1 : 0; }

template <class T>
__global__ void k_fwd_xy(HphiLaunch a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const FnRec r = a.fn[blockIdx.y];
    const int z = blockIdx.x >> 1, bz = blockIdx.x & 1;
    if (z >= r.n[2]) return;
    const int nx = r.n[0], ny = r.n[1], nz = r.n[2];
    const int X = 2 * nx + 29, Y = 2 * ny + 29;
    T* in = sm;                 // [4][ny][nx]
    T* mid = sm + 4 * ny * nx;  // [2][ny][X]
    const T* D = static_cast<const T*>(a.ws) + r.ws_D;
    const int64_t plane = static_cast<int64_t>(nx) * ny * nz;
    const int pn = nx * ny;
    for (int i = threadIdx.x; i < 4 * pn; i += blockDim.x) {
        const int tb = i / pn, rem = i - tb * pn;
        in[i] = D[(tb + 4 * bz) * plane + static_cast<int64_t>(z) * pn + rem];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * ny * X; i += blockDim.x) {
        const int by = i / (ny * X), rem = i - by * ny * X;
        const int y = rem / X, xo = rem - y * X;
        const T* s = in + (2 * by) * pn + y * nx;
        const T* d = s + pn;
        const int lo = up_lo(xo), hi = min(nx - 1, xo >> 1);
        T acc = 0;
        for (int q = lo; q <= hi; ++q) acc += Tab<T>::fwd(0, xo - 2 * q) * s[q] + Tab<T>::fwd(1, xo - 2 * q) * d[q];
        mid[i] = acc;
    }
    __syncthreads();
    T* Bf = static_cast<T*>(a.ws) + r.ws_Bf + (static_cast<int64_t>(bz) * nz + z) * Y * X;
    for (int i = threadIdx.x; i < Y * X; i += blockDim.x) {
        const int yo = i / X, xo = i - yo * X;
        const T* s = mid + xo;
        const T* d = mid + ny * X + xo;
        const int lo = up_lo(yo), hi = min(ny - 1, yo >> 1);
        T acc = 0;
        for (int q = lo; q <= hi; ++q)
            acc += Tab<T>::fwd(0, yo - 2 * q) * s[q * X] + Tab<T>::fwd(1, yo - 2 * q) * d[q * X];
        Bf[i] = acc;
    }
}

// ---------------------------------------------------------------- z stage with V

template <class T>
__global__ void k_z(HphiLaunch a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const FnRec r = a.fn[blockIdx.y];
    const int nx = r.n[0], ny = r.n[1], nz = r.n[2];
    const int X = 2 * nx + 29, Y = 2 * ny + 29, Z = 2 * nz + 29;
    const int cols = X * Y;
    const int C = a.zcols;
    const int c = blockIdx.x * C + threadIdx.x;
    if (blockIdx.x * C >= cols) return;
    const bool valid = c < cols;
    const int t = threadIdx.x;
    T* Bs = sm;              // [2][nz][C]
    T* vs = sm + 2 * nz * C;  // [Z][C]
    const T* Bf = static_cast<const T*>(a.ws) + r.ws_Bf;
    for (int q = 0; q < 2 * nz; ++q) Bs[q * C + t] = valid ? Bf[static_cast<int64_t>(q) * cols + c] : T(0);
    double epot = 0.0;
    if (valid) {
        const int xo = c % X, yo = c / X;
        const int64_t jx = 2LL * r.lo[0] - V_REACH + xo - a.vlo[0];
        const int64_t jy = 2LL * r.lo[1] - V_REACH + yo - a.vlo[1];
        const int64_t jz0 = 2LL * r.lo[2] - V_REACH - a.vlo[2];
        const T* V = static_cast<const T*>(a.V) + (jy + 0) * a.vn[0] + jx;
        const int64_t vstride = a.vn[0] * a.vn[1];
        for (int zo = 0; zo < Z; ++zo) {
            const int lo = up_lo(zo), hi = min(nz - 1, zo >> 1);
            T u = 0;
            for (int q = lo; q <= hi; ++q)
                u += Tab<T>::fwd(0, zo - 2 * q) * Bs[q * C + t] + Tab<T>::fwd(1, zo - 2 * q) * Bs[(nz + q) * C + t];
            const T vv = V[(jz0 + zo) * vstride];
            const T v = vv * u;
            epot += static_cast<double>(v) * static_cast<double>(u);
            vs[zo * C + t] = v;
        }
        const int nzp = r.np[2];
        const int dz = r.lop[2] - r.lo[2];
        T* Bb = static_cast<T*>(a.ws) + r.ws_Bb;
        for (int b = 0; b < nzp; ++b) {
            const int b2 = 2 * (b + dz);
            const int lo = max(0, b2), hi = min(Z - 1, b2 + 30);
            T s = 0, d = 0;
            for (int zo = lo; zo <= hi; ++zo) {
                const T v = vs[zo * C + t];
                s += Tab<T>::fwd(0, zo - b2) * v;
                d += Tab<T>::fwd(1, zo - b2) * v;
            }
            Bb[static_cast<int64_t>(b) * cols + c] = s;
            Bb[static_cast<int64_t>(nzp + b) * cols + c] = d;
        }
    }
    epot = warp_sum(epot);
    if ((threadIdx.x & 31) == 0 && epot != 0.0) atomicAdd(a.e_pot + r.f, epot);
}

// ---------------------------------------------------------------- backward y, x

template <class T>
__global__ void k_bwd_xy(HphiLaunch a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const FnRec r = a.fn[blockIdx.y];
    const int zb = blockIdx.x >> 1, bz = blockIdx.x & 1;
    if (zb >= r.np[2]) return;
    const int nx = r.n[0], ny = r.n[1];
    const int X = 2 * nx + 29, Y = 2 * ny + 29;
    const int nxp = r.np[0], nyp = r.np[1], nzp = r.np[2];
    const int dx = r.lop[0] - r.lo[0], dy = r.lop[1] - r.lo[1];
    T* pl = sm;           // [Y][X]
    T* mid = sm + Y * X;  // [2][nyp][X]
    const T* Bb = static_cast<const T*>(a.ws) + r.ws_Bb + (static_cast<int64_t>(bz) * nzp + zb) * Y * X;
    for (int i = threadIdx.x; i < Y * X; i += blockDim.x) pl[i] = Bb[i];
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * nyp * X; i += blockDim.x) {
        const int by = i / (nyp * X), rem = i - by * nyp * X;
        const int b = rem / X, xo = rem - b * X;
        const int b2 = 2 * (b + dy);
        const int lo = max(0, b2), hi = min(Y - 1, b2 + 30);
        T acc = 0;
        for (int yo = lo; yo <= hi; ++yo) acc += Tab<T>::fwd(by, yo - b2) * pl[yo * X + xo];
        mid[i] = acc;
    }
    __syncthreads();
    T* G = static_cast<T*>(a.ws) + r.ws_G;
    const int64_t plane = static_cast<int64_t>(nxp) * nyp * nzp;
    const int pn = nxp * nyp;
    for (int i = threadIdx.x; i < 4 * pn; i += blockDim.x) {
        const int tb = i / pn, rem = i - tb * pn;
        const int bx = tb & 1, by = tb >> 1;
        const int b = rem / nxp, xb = rem - b * nxp;
        const int b2 = 2 * (xb + dx);
        const int lo = max(0, b2), hi = min(X - 1, b2 + 30);
        const T* m = mid + (by * nyp + b) * X;
        T acc = 0;
        for (int xo = lo; xo <= hi; ++xo) acc += Tab<T>::fwd(bx, xo - b2) * m[xo];
        G[(tb + 4 * bz) * plane + static_cast<int64_t>(zb) * pn + rem] = acc;
    }
}

// ---------------------------------------------------------------- kinetic

template <class T>
__global__ void k_kinetic(HphiLaunch a) {
    const FnRec r = a.fn[blockIdx.y];
    const int nxp = r.np[0], nyp = r.np[1], nzp = r.np[2];
    const int64_t pn = static_cast<int64_t>(nxp) * nyp * nzp;
    const int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    double ekin = 0.0;
    if (p < pn) {
        const int xp = static_cast<int>(p % nxp), yp = static_cast<int>((p / nxp) % nyp), zp = static_cast<int>(p / (static_cast<int64_t>(nxp) * nyp));
        const int nx = r.n[0], ny = r.n[1], nz = r.n[2];
        const int q[3] = {xp + r.lop[0] - r.lo[0], yp + r.lop[1] - r.lo[1], zp + r.lop[2] - r.lo[2]};
        const int n[3] = {nx, ny, nz};
        const int64_t plane = static_cast<int64_t>(nx) * ny * nz;
        const int64_t stride[3] = {1, nx, static_cast<int64_t>(nx) * ny};
        const T* D = static_cast<const T*>(a.ws) + r.ws_D;
        T* G = static_cast<T*>(a.ws) + r.ws_G;
        // the point must lie within reach (14) of the L box along every axis but one
        int out_axes = 0;
        for (int d = 0; d < 3; ++d) out_axes += (q[d] < 0 || q[d] >= n[d]);
        const bool inside = out_axes == 0;
        if (out_axes <= 1) {
            for (int b = 0; b < 8; ++b) {
                T acc = 0;
                for (int d = 0; d < 3; ++d) {
                    // the other two coordinates must be inside the L box
                    bool ok = true;
                    for (int e = 0; e < 3; ++e)
                        if (e != d && (q[e] < 0 || q[e] >= n[e])) ok = false;
                    if (!ok) continue;
                    const int bit = (b >> d) & 1;
                    int64_t base = 0;
                    for (int e = 0; e < 3; ++e)
                        if (e != d) base += q[e] * stride[e];
                    const int l0 = max(-KIN_HALF, -q[d]), l1 = min(KIN_HALF, n[d] - 1 - q[d]);
                    for (int bp = 0; bp < 2; ++bp) {
                        const int src = (b & ~(1 << d)) | (bp << d);
                        const T* Dp = D + src * plane + base;
                        const int k = bit * 2 + bp;
                        for (int l = l0; l <= l1; ++l)
                            acc += Tab<T>::kin(k, l + KIN_HALF) * Dp[static_cast<int64_t>(q[d] + l) * stride[d]];
                    }
                }
                const T kv = static_cast<T>(a.kin_scale) * acc;
                G[b * pn + p] += kv;
                if (inside) {
                    const int64_t qi = q[0] + q[1] * stride[1] + q[2] * stride[2];
                    ekin += static_cast<double>(D[b * plane + qi]) * static_cast<double>(kv);
                }
            }
        }
    }
    ekin = warp_sum(ekin);
    if ((threadIdx.x & 31) == 0 && ekin != 0.0) atomicAdd(a.e_kin + r.f, ekin);
}

// ---------------------------------------------------------------- sparse H / S

constexpr int HS_BLK = 32;
constexpr int HS_KC = 64;

// value of one compressed vector at box-local (x, y, z) of a region part; 0 if absent
template <class T>
__device__ __forceinline__ const T* seg_find(const Seg* seg, const int32_t* rowptr, int64_t seg0, int64_t row0,
                                             const int32_t* lo, const int32_t* n, int gx, int gy, int gz,
                                             const T* base) {
    const int x = gx - lo[0], y = gy - lo[1], z = gz - lo[2];
    if (x < 0 || y < 0 || z < 0 || x >= n[0] || y >= n[1] || z >= n[2]) return nullptr;
    const int row = y + n[1] * z;
    const int s0 = rowptr[row0 + row], s1 = rowptr[row0 + row + 1];
    for (int s = s0; s < s1; ++s) {
        const Seg sg = seg[seg0 + s];
        if (x >= sg.x0 && x <= sg.x1) return base + sg.off + (x - sg.x0);
    }
    return nullptr;
}

template <class T>
__global__ void k_hs(HSLaunch a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* P = reinterpret_cast<T*>(smem_raw);       // [BLK][KC+1]  phi_a
    T* PB = P + HS_BLK * (HS_KC + 1);             // [BLK][KC+1]  phi_b
    T* Q = PB + HS_BLK * (HS_KC + 1);             // [BLK][KC+1]  H phi_b
    const HSWork w = a.work[blockIdx.x];
    const int* org = a.tile_org + 4 * w.tile;
    const int ox = org[0], oy = org[1], oz = org[2];
    const int f0 = org[3], f1 = org[7];
    const int T3 = a.tile * a.tile * a.tile;
    const int nfine = f1 - f0;
    const int tid = threadIdx.x;
    const int pi = tid >> 3, pj0 = (tid & 7) * 4;
    double sacc[4] = {0, 0, 0, 0}, hacc[4] = {0, 0, 0, 0};
    const int n_coarse_chunks = (T3 + HS_KC - 1) / HS_KC;
    const int fpc = HS_KC / 7;  // fine points per chunk
    const int n_fine_chunks = (nfine + fpc - 1) / fpc;
    const T* phi = static_cast<const T*>(a.phi);
    const T* hphi = static_cast<const T*>(a.hphi);
    for (int ch = 0; ch < n_coarse_chunks + n_fine_chunks; ++ch) {
        const bool coarse = ch < n_coarse_chunks;
        int kcount;
        if (coarse)
            kcount = min(HS_KC, T3 - ch * HS_KC);
        else
            kcount = 7 * min(fpc, nfine - (ch - n_coarse_chunks) * fpc);
        // gather: task = (slot, k-point); slots 0..na-1 -> A, na..na+nb-1 -> B
        const int npts = coarse ? kcount : kcount / 7;
        const int nslot = w.na + w.nb;
        for (int task = tid; task < nslot * npts; task += blockDim.x) {
            const int slot = task / npts, kp = task - slot * npts;
            int lx, ly, lz;
            if (coarse) {
                const int k = ch * HS_KC + kp;
                lx = k % a.tile;
                ly = (k / a.tile) % a.tile;
                lz = k / (a.tile * a.tile);
            } else {
                const int code = a.tile_fine[f0 + (ch - n_coarse_chunks) * fpc + kp];
                lx = code & 255;
                ly = (code >> 8) & 255;
                lz = code >> 16;
            }
            const int gx = ox + lx, gy = oy + ly, gz = oz + lz;
            const bool isA = slot < w.na;
            const int f = isA ? a.listA[w.a0 + slot] : a.listB[w.b0 + slot - w.na];
            const AtomRec& at = a.atoms[a.sf_atom[f]];
            const T* pL = phi + a.off_L[f];
            T* dstP = isA ? P + slot * (HS_KC + 1) : PB + (slot - w.na) * (HS_KC + 1);
            if (coarse) {
                const T* v = seg_find<T>(a.seg, a.rowptr, at.segLc, at.rowLc, at.lo, at.n, gx, gy, gz, pL);
                dstP[kp] = v ? *v : T(0);
                if (!isA) {
                    const T* hv = seg_find<T>(a.seg, a.rowptr, at.segPc, at.rowPc, at.lop, at.np, gx, gy, gz,
                                              hphi + a.off_Lp[f]);
                    Q[(slot - w.na) * (HS_KC + 1) + kp] = hv ? *hv : T(0);
                }
            } else {
                const T* v = seg_find<T>(a.seg, a.rowptr, at.segLf, at.rowLf, at.lo, at.n, gx, gy, gz, pL + at.ncL);
#pragma unroll
                for (int t = 0; t < 7; ++t) dstP[7 * kp + t] = v ? v[static_cast<int64_t>(t) * at.nfL] : T(0);
                if (!isA) {
                    const T* hv = seg_find<T>(a.seg, a.rowptr, at.segPf, at.rowPf, at.lop, at.np, gx, gy, gz,
                                              hphi + a.off_Lp[f] + at.ncP);
                    T* q = Q + (slot - w.na) * (HS_KC + 1) + 7 * kp;
#pragma unroll
                    for (int t = 0; t < 7; ++t) q[t] = hv ? hv[static_cast<int64_t>(t) * at.nfP] : T(0);
                }
            }
        }
        __syncthreads();
        if (pi < w.na) {
            T ps[4] = {0, 0, 0, 0}, ph[4] = {0, 0, 0, 0};
            const T* pa = P + pi * (HS_KC + 1);
            for (int k = 0; k < kcount; ++k) {
                const T va = pa[k];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    ps[u] += va * PB[(pj0 + u) * (HS_KC + 1) + k];
                    ph[u] += va * Q[(pj0 + u) * (HS_KC + 1) + k];
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                sacc[u] += static_cast<double>(ps[u]);
                hacc[u] += static_cast<double>(ph[u]);
            }
        }
        __syncthreads();
    }
    if (pi >= w.na) return;
    const int fa = a.listA[w.a0 + pi];
    const int64_t r0 = a.row_ptr[fa], r1 = a.row_ptr[fa + 1];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int j = pj0 + u;
        if (j >= w.nb) continue;
        const int fb = a.listB[w.b0 + j];
        int64_t lo = r0, hi = r1 - 1;
        int64_t pos = -1;
        while (lo <= hi) {
            const int64_t mid = (lo + hi) >> 1;
            const int cm = a.col[mid];
            if (cm == fb) {
                pos = mid;
                break;
            }
            if (cm < fb)
                lo = mid + 1;
            else
                hi = mid - 1;
        }
        if (pos < 0) continue;
        if (hacc[u] != 0.0) atomicAdd(a.H + pos, hacc[u]);
        if (sacc[u] != 0.0) atomicAdd(a.S + pos, sacc[u]);
    }
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
    return cudaMemcpyToSymbol(c_kin_f, k32, sizeof(k32));
}

cudaError_t configure_kernels(size_t max_smem) {
    cudaError_t e;
    const int m = static_cast<int>(max_smem);
#define SETMAX(K)                                                                             \
    if ((e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, m)) != cudaSuccess) \
        return e;
    SETMAX(k_fwd_xy<double>) SETMAX(k_fwd_xy<float>)
    SETMAX(k_z<double>) SETMAX(k_z<float>)
    SETMAX(k_bwd_xy<double>) SETMAX(k_bwd_xy<float>)
    SETMAX(k_hs<double>) SETMAX(k_hs<float>)
#undef SETMAX
    return cudaSuccess;
}

#define TRACED(TR, KIND, S, LAUNCH) \
    do {                                \
        trace_begin(TR, KIND, S);       \
        LAUNCH;                         \
        trace_end(TR, S);               \
    } while (0)

template <class T>
static cudaError_t hphi_batch(const HphiLaunch& a, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    TRACED(a.tr, TK_MEMSET, s, e = cudaMemsetAsync(a.ws, 0, static_cast<size_t>(a.ws_D_elems) * sizeof(T), s));
    if (e != cudaSuccess) return e;
    const int nf = a.nfn;
    TRACED(a.tr, TK_UNCOMPRESS, s, (k_uncompress<T><<<dim3((a.max_segL + 7) / 8, nf), 256, 0, s>>>(a)));
    TRACED(a.tr, TK_FWD_XY, s, (k_fwd_xy<T><<<dim3(2 * a.max_nz, nf), 256, a.smem_fwd, s>>>(a)));
    TRACED(a.tr, TK_Z, s, (k_z<T><<<dim3((a.max_cols + a.zcols - 1) / a.zcols, nf), a.zcols, a.smem_z, s>>>(a)));
    TRACED(a.tr, TK_BWD_XY, s, (k_bwd_xy<T><<<dim3(2 * a.max_nzp, nf), 256, a.smem_bwd, s>>>(a)));
    TRACED(a.tr, TK_KINETIC, s,
           (k_kinetic<T><<<dim3(static_cast<unsigned>((a.max_ptsP + 255) / 256), nf), 256, 0, s>>>(a)));
    TRACED(a.tr, TK_COMPRESS, s, (k_compress<T><<<dim3((a.max_segP + 7) / 8, nf), 256, 0, s>>>(a)));
    return cudaGetLastError();
}

cudaError_t enqueue_hphi_batch(const HphiLaunch& a, cudaStream_t s) {
    return a.prec == 0 ? hphi_batch<double>(a, s) : hphi_batch<float>(a, s);
}

cudaError_t enqueue_hs(const HSLaunch& a, cudaStream_t s) {
    const size_t es = a.prec == 0 ? sizeof(double) : sizeof(float);
    const size_t smem = 3 * HS_BLK * (HS_KC + 1) * es;
    if (a.prec == 0)
        TRACED(a.tr, TK_HS, s, (k_hs<double><<<a.nwork, 256, smem, s>>>(a)));
    else
        TRACED(a.tr, TK_HS, s, (k_hs<float><<<a.nwork, 256, smem, s>>>(a)));
    return cudaGetLastError();
}

}  // namespace lsw
