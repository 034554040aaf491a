// sm_103a kernels of the quartic confinement and the preconditioning equation (Sec.
// "Support function optimization": H_alpha = H_KS + a_alpha (r - R_alpha)^4 in the first
// iterations, "evaluated via convolutions in the same manner as the kinetic energy";
// Eq. precond: (-1/2 nabla^2 + a_alpha (r - R_alpha)^4 - eps_alpha) g_prec = -g).
//
// The operators act on a function's dense two-level box E = (L box widened by 14 on
// every side), 8 coefficient types t = bx + 2 by + 4 bz:
//   Q = a [ sum_d X_d^4 + 2 sum_{d<e} X_d^2 X_e^2 ],  X_d = x_d - R_d,
// each X_d^m a 1D operator along d between the scaling/wavelet functions of coarse
// points i, j (band |j - i| <= 14), its entries depending on i (tables built on the host
// from the moment overlaps F^p of the filter set); T = -1/(2h^2) sum_d K_d with the
// Galerkin kinetic blocks.
//
//   k_conf_load    compressed phi on L -> the E box (members; the box is zeroed before)
//   k_conf_op      out (+)= scale * (1D operator along one dimension) in, for every type
//   k_conf_store   E box -> compressed members of L or L' (optionally added to the target)
//   k_conf_boxdot  per function sum over the box of in * out (FP64)
//   k_conf_dot     per function dot product of two compressed vectors on L (FP64)
//   k_cg_*         the conjugate-gradient updates, one set of scalars per function
#include <cstdint>

#include "lsw_device.h"
#include "lsw_internal.h"

namespace lsw {

__device__ __forceinline__ double warp_sum_c(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ double block_sum_c(double v) {
    __shared__ double part[32];
    __syncthreads();
    v = warp_sum_c(v);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < static_cast<int>(blockDim.x >> 5); ++i) s += part[i];
    return s;
}

// Box geometry of function k of the batch: E extents and origin (global coarse index).
struct ConfBox {
    int e[3], o[3];
    int64_t vol;
};
__device__ __forceinline__ ConfBox conf_box(const AtomRec& at) {
    ConfBox b;
    for (int d = 0; d < 3; ++d) {
        b.e[d] = at.n[d] + 2 * KIN_HALF;
        b.o[d] = at.lo[d] - KIN_HALF;
    }
    b.vol = static_cast<int64_t>(b.e[0]) * b.e[1] * b.e[2];
    return b;
}

// compressed phi on L -> box (8 types); warp per row (y, z) of the L box
template <class T>
__global__ void __launch_bounds__(256) k_conf_load(ConfLaunch a, const T* __restrict__ src, T* __restrict__ box) {
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = 16;
    const int k = blockIdx.y;
    const int f = static_cast<int>(a.f0) + k;
    const AtomRec at = LD(a.atoms, LD(a.sf_atom, f, a.n_sf), a.n_atoms);
    const ConfBox B = conf_box(at);
    T* bx = box + static_cast<int64_t>(k) * a.box_stride;
    const int64_t off = LD(a.off_L, f, a.n_sf + 1);
    const int rows = at.n[1] * at.n[2];
    const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (warp >= rows) return;
    const int y = warp % at.n[1], z = warp / at.n[1];
    const int64_t rowbase = (static_cast<int64_t>(z + KIN_HALF) * B.e[1] + (y + KIN_HALF)) * B.e[0] + KIN_HALF;
    for (int part = 0; part < 2; ++part) {
        const int64_t r0 = part ? at.rowLf : at.rowLc, sg0 = part ? at.segLf : at.segLc;
        const int s0 = LD(a.rowptr, r0 + warp, a.rowptr_n), s1 = LD(a.rowptr, r0 + warp + 1, a.rowptr_n);
        for (int s = s0; s < s1; ++s) {
            const Seg g = LD(a.seg, sg0 + s, a.seg_n);
            for (int x = g.x0 + lane; x <= g.x1; x += 32) {
                const int64_t rel = g.off + (x - g.x0);
                if (part == 0) {
                    ST(bx, rowbase + x, a.box_stride, LD(src, off + rel, a.vec_n));
                } else {
                    for (int t = 1; t < 8; ++t)
                        ST(bx, t * B.vol + rowbase + x, a.box_stride,
                           LD(src, off + at.ncL + rel + static_cast<int64_t>(t - 1) * at.nfL, a.vec_n));
                }
            }
        }
    }
}

// out[t][p] (+)= scale * sum_{b'} sum_{l=-14..14} B_{b(t) b'}(i_p, l) in[t'(b')][p + l e_dim]
// kind 0: kinetic blocks (constant); 1, 2: the tables of X^2, X^4 along dim (per atom)
template <class T>
__global__ void __launch_bounds__(256) k_conf_op(ConfLaunch a, const T* __restrict__ in, T* __restrict__ out, int dim,
                                                 int kind, int accumulate, double scale, int use_a) {
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = 17;
    const int k = blockIdx.z;
    const int t = blockIdx.y;
    const int f = static_cast<int>(a.f0) + k;
    const int atom = LD(a.sf_atom, f, a.n_sf);
    const AtomRec at = LD(a.atoms, atom, a.n_atoms);
    const ConfBox B = conf_box(at);
    const int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (p >= B.vol) return;
    const int x = static_cast<int>(p % B.e[0]), y = static_cast<int>((p / B.e[0]) % B.e[1]),
              z = static_cast<int>(p / (static_cast<int64_t>(B.e[0]) * B.e[1]));
    const int c[3] = {x, y, z};
    const int i = c[dim];
    const int64_t stride = dim == 0 ? 1 : dim == 1 ? B.e[0] : static_cast<int64_t>(B.e[0]) * B.e[1];
    const int b = (t >> dim) & 1;
    const T* ib = in + static_cast<int64_t>(k) * a.box_stride;
    double acc = 0.0;
    for (int bp = 0; bp < 2; ++bp) {
        const int src = (t & ~(1 << dim)) | (bp << dim);
        const int64_t q0 = src * B.vol + p;
        if (kind == 0) {
            const double* taps = a.kin[b * 2 + bp];
            for (int l = -KIN_HALF; l <= KIN_HALF; ++l) {
                const int j = i + l;
                if (j < 0 || j >= B.e[dim]) continue;
                acc += taps[l + KIN_HALF] * static_cast<double>(LD(ib, q0 + l * stride, a.box_stride));
            }
        } else {
            // table entries [pair][i][l + 14] of X^m along dim for this atom
            int64_t base = LD(a.qtab_off, atom, a.n_atoms + 1);
            for (int d = 0; d < dim; ++d) base += 2LL * 4 * (at.n[d] + 2 * KIN_HALF) * KIN_TAPS;
            base += ((static_cast<int64_t>(kind - 1) * 4 + (b * 2 + bp)) * B.e[dim] + i) * KIN_TAPS;
            for (int l = -KIN_HALF; l <= KIN_HALF; ++l) {
                const int j = i + l;
                if (j < 0 || j >= B.e[dim]) continue;
                acc += LD(a.qtab, base + l + KIN_HALF, a.qtab_n) * static_cast<double>(LD(ib, q0 + l * stride, a.box_stride));
            }
        }
    }
    T* ob = out + static_cast<int64_t>(k) * a.box_stride;
    const int64_t qo = t * B.vol + p;
    const double v = scale * (use_a ? LD(a.acoef, f, a.n_sf) : 1.0) * acc;
    ST(ob, qo, a.box_stride, static_cast<T>(accumulate ? static_cast<double>(LD(ob, qo, a.box_stride)) + v : v));
}

// box -> compressed members of the region (0: L, 1: L'); dst (+)= box value
template <class T>
__global__ void __launch_bounds__(256) k_conf_store(ConfLaunch a, const T* __restrict__ box, T* __restrict__ dst,
                                                    int region, int accumulate) {
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = 18;
    const int k = blockIdx.y;
    const int f = static_cast<int>(a.f0) + k;
    const AtomRec at = LD(a.atoms, LD(a.sf_atom, f, a.n_sf), a.n_atoms);
    const ConfBox B = conf_box(at);
    const T* bx = box + static_cast<int64_t>(k) * a.box_stride;
    const int* n = region ? at.np : at.n;
    const int* lo = region ? at.lop : at.lo;
    const int64_t off = LD(region ? a.off_Lp : a.off_L, f, a.n_sf + 1);
    const int nc = region ? at.ncP : at.ncL, nf = region ? at.nfP : at.nfL;
    const int64_t dn = region ? a.dst_n : a.vec_n;
    const int rows = n[1] * n[2];
    const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (warp >= rows) return;
    const int y = warp % n[1], z = warp / n[1];
    const int by = lo[1] + y - B.o[1], bz = lo[2] + z - B.o[2];
    const bool yz_in = by >= 0 && by < B.e[1] && bz >= 0 && bz < B.e[2];
    for (int part = 0; part < 2; ++part) {
        const int64_t r0 = part ? (region ? at.rowPf : at.rowLf) : (region ? at.rowPc : at.rowLc);
        const int64_t sg0 = part ? (region ? at.segPf : at.segLf) : (region ? at.segPc : at.segLc);
        const int s0 = LD(a.rowptr, r0 + warp, a.rowptr_n), s1 = LD(a.rowptr, r0 + warp + 1, a.rowptr_n);
        for (int s = s0; s < s1; ++s) {
            const Seg g = LD(a.seg, sg0 + s, a.seg_n);
            for (int x = g.x0 + lane; x <= g.x1; x += 32) {
                const int bxx = lo[0] + x - B.o[0];
                const bool in_box = yz_in && bxx >= 0 && bxx < B.e[0];
                const int64_t pb = (static_cast<int64_t>(bz) * B.e[1] + by) * B.e[0] + bxx;
                const int64_t rel = g.off + (x - g.x0);
                for (int t = part ? 1 : 0; t < (part ? 8 : 1); ++t) {
                    const int64_t q = off + (part ? nc + rel + static_cast<int64_t>(t - 1) * nf : rel);
                    const T v = in_box ? LD(bx, t * B.vol + pb, a.box_stride) : T(0);
                    ST(dst, q, dn, accumulate ? static_cast<T>(LD(dst, q, dn) + v) : v);
                }
            }
        }
    }
}

// out += coef[f] * in over the whole box (the - eps P_L term of the preconditioning operator)
template <class T>
__global__ void __launch_bounds__(256) k_conf_axpy_box(ConfLaunch a, const T* __restrict__ in, T* __restrict__ out) {
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = 20;
    const int k = blockIdx.y;
    const int f = static_cast<int>(a.f0) + k;
    const AtomRec at = LD(a.atoms, LD(a.sf_atom, f, a.n_sf), a.n_atoms);
    const ConfBox B = conf_box(at);
    const T c = static_cast<T>(-LD(a.eps, f, a.n_sf));
    const T* ib = in + static_cast<int64_t>(k) * a.box_stride;
    T* ob = out + static_cast<int64_t>(k) * a.box_stride;
    for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < 8 * B.vol;
         p += static_cast<int64_t>(gridDim.x) * blockDim.x)
        ST(ob, p, a.box_stride, LD(ob, p, a.box_stride) + c * LD(ib, p, a.box_stride));
}

// e[f] (+)= sum over the box of x * y (x: the loaded phi, zero off its members)
template <class T>
__global__ void __launch_bounds__(256) k_conf_boxdot(ConfLaunch a, const T* __restrict__ x, const T* __restrict__ y,
                                                     double* __restrict__ e) {
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = 19;
    const int k = blockIdx.x;
    const int f = static_cast<int>(a.f0) + k;
    const AtomRec at = LD(a.atoms, LD(a.sf_atom, f, a.n_sf), a.n_atoms);
    const ConfBox B = conf_box(at);
    const T* xb = x + static_cast<int64_t>(k) * a.box_stride;
    const T* yb = y + static_cast<int64_t>(k) * a.box_stride;
    double v = 0.0;
    for (int64_t p = threadIdx.x; p < 8 * B.vol; p += blockDim.x)
        v += static_cast<double>(LD(xb, p, a.box_stride)) * static_cast<double>(LD(yb, p, a.box_stride));
    const double s = block_sum_c(v);
    if (threadIdx.x == 0) e[f] = s;
}

// out[f] = sum over the compressed vector of function f on L of x * y
template <class T>
__global__ void __launch_bounds__(256) k_conf_dot(ConfLaunch a, const T* __restrict__ x, const T* __restrict__ y,
                                                  double* __restrict__ out) {
    const int f = static_cast<int>(a.f0) + blockIdx.x;
    const AtomRec at = a.atoms[a.sf_atom[f]];
    const int64_t o = a.off_L[f], n = at.ncL + 7LL * at.nfL;
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v += static_cast<double>(x[o + i]) * static_cast<double>(y[o + i]);
    const double s = block_sum_c(v);
    if (threadIdx.x == 0) out[f] = s;
}

// x = 0, r = p = -g on the members of every function of the batch
template <class T>
__global__ void __launch_bounds__(256) k_cg_init(ConfLaunch a, const T* __restrict__ g, T* __restrict__ x, T* __restrict__ r,
                                                 T* __restrict__ p) {
    const int f = static_cast<int>(a.f0) + blockIdx.y;
    const AtomRec at = a.atoms[a.sf_atom[f]];
    const int64_t o = a.off_L[f], n = at.ncL + 7LL * at.nfL;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        x[o + i] = T(0);
        r[o + i] = -g[o + i];
        p[o + i] = -g[o + i];
    }
}

// alpha = rr / pAp (0 once rr = 0: the function's iteration has stopped);
// x += alpha p, r -= alpha Ap
template <class T>
__global__ void __launch_bounds__(256) k_cg_step1(ConfLaunch a, const double* __restrict__ rr, const double* __restrict__ pAp,
                                                  const T* __restrict__ p, const T* __restrict__ Ap, T* __restrict__ x,
                                                  T* __restrict__ r) {
    const int f = static_cast<int>(a.f0) + blockIdx.y;
    const AtomRec at = a.atoms[a.sf_atom[f]];
    const int64_t o = a.off_L[f], n = at.ncL + 7LL * at.nfL;
    const double alpha = rr[f] == 0.0 ? 0.0 : rr[f] / pAp[f];
    const T al = static_cast<T>(alpha);
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        x[o + i] = x[o + i] + al * p[o + i];
        r[o + i] = r[o + i] - al * Ap[o + i];
    }
}

// beta = rr_new / rr (0 once rr_new = 0); p = r + beta p; rr = rr_new; res = sqrt(rr_new)
template <class T>
__global__ void __launch_bounds__(256) k_cg_step2(ConfLaunch a, double* __restrict__ rr, const double* __restrict__ rr_new,
                                                  const T* __restrict__ r, T* __restrict__ p, double* __restrict__ res) {
    const int f = static_cast<int>(a.f0) + blockIdx.y;
    const AtomRec at = a.atoms[a.sf_atom[f]];
    const int64_t o = a.off_L[f], n = at.ncL + 7LL * at.nfL;
    const double beta = (rr[f] == 0.0 || rr_new[f] == 0.0) ? 0.0 : rr_new[f] / rr[f];
    const T be = static_cast<T>(beta);
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        p[o + i] = r[o + i] + be * p[o + i];
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (res) res[f] = sqrt(rr_new[f]);
    }
}

// rr[f] = rr_new[f] after every block of step 2 has read both (separate launch)
__global__ void k_cg_swap(ConfLaunch a, double* __restrict__ rr, const double* __restrict__ rr_new) {
    const int f = static_cast<int>(a.f0) + blockIdx.x * blockDim.x + threadIdx.x;
    if (f < a.f0 + a.nfn) rr[f] = rr_new[f];
}

// ---------------------------------------------------------------- host wrappers

// The operator on a batch of functions: vin (compressed on L) -> box; box_out =
// a_f Q (+ T, + (-eps_f) for the preconditioning operator); optionally <vin|box_out>
// per function and the store of box_out onto the members of L (region 0) or L' (1).
template <class T>
static cudaError_t conf_apply_t(const ConfLaunch& a, const void* vin, void* box_in, void* box_out, void* box_tmp,
                                void* dst, int region, int accumulate, bool precond, double* energy, cudaStream_t s) {
    const T* src = static_cast<const T*>(vin);
    T* bi = static_cast<T*>(box_in);
    T* bo = static_cast<T*>(box_out);
    T* bt = static_cast<T*>(box_tmp);
    cudaError_t e = cudaMemsetAsync(bi, 0, static_cast<size_t>(a.nfn) * a.box_stride * sizeof(T), s);
    if (e != cudaSuccess) return e;
    k_conf_load<T><<<dim3(static_cast<unsigned>((a.max_rows_L + 7) / 8), a.nfn), 256, 0, s>>>(a, src, bi);
    const dim3 g(static_cast<unsigned>((a.max_vol + 255) / 256), 8, a.nfn);
    // a sum_d X_d^4 (and, for the preconditioning operator, the kinetic arms)
    for (int d = 0; d < 3; ++d) {
        k_conf_op<T><<<g, 256, 0, s>>>(a, bi, bo, d, 2, d > 0, 1.0, 1);
        if (precond) k_conf_op<T><<<g, 256, 0, s>>>(a, bi, bo, d, 0, 1, a.kin_scale, 0);
    }
    // 2 a sum_{d<e} X_d^2 X_e^2
    for (int d = 0; d < 3; ++d)
        for (int e2 = d + 1; e2 < 3; ++e2) {
            k_conf_op<T><<<g, 256, 0, s>>>(a, bi, bt, e2, 1, 0, 1.0, 0);
            k_conf_op<T><<<g, 256, 0, s>>>(a, bt, bo, d, 1, 1, 2.0, 1);
        }
    if (precond) k_conf_axpy_box<T><<<dim3(64, a.nfn), 256, 0, s>>>(a, bi, bo);
    if (energy) k_conf_boxdot<T><<<a.nfn, 256, 0, s>>>(a, bi, bo, energy);
    if (dst)
        k_conf_store<T><<<dim3(static_cast<unsigned>(((region ? a.max_rows_P : a.max_rows_L) + 7) / 8), a.nfn), 256, 0, s>>>(
            a, bo, static_cast<T*>(dst), region, accumulate);
    return cudaGetLastError();
}

cudaError_t conf_apply(const ConfLaunch& a, const void* vin, void* box_in, void* box_out, void* box_tmp, void* dst,
                       int region, int accumulate, bool precond, double* energy, cudaStream_t s) {
    return a.prec == 0 ? conf_apply_t<double>(a, vin, box_in, box_out, box_tmp, dst, region, accumulate, precond, energy, s)
                       : conf_apply_t<float>(a, vin, box_in, box_out, box_tmp, dst, region, accumulate, precond, energy, s);
}

cudaError_t conf_cg_init(const ConfLaunch& a, const void* g, void* x, void* r, void* p, cudaStream_t s) {
    const dim3 gr(64, a.nfn);
    if (a.prec == 0)
        k_cg_init<double><<<gr, 256, 0, s>>>(a, static_cast<const double*>(g), static_cast<double*>(x),
                                             static_cast<double*>(r), static_cast<double*>(p));
    else
        k_cg_init<float><<<gr, 256, 0, s>>>(a, static_cast<const float*>(g), static_cast<float*>(x), static_cast<float*>(r),
                                            static_cast<float*>(p));
    return cudaGetLastError();
}

cudaError_t conf_dot(const ConfLaunch& a, const void* x, const void* y, double* out, cudaStream_t s) {
    if (a.prec == 0)
        k_conf_dot<double><<<a.nfn, 256, 0, s>>>(a, static_cast<const double*>(x), static_cast<const double*>(y), out);
    else
        k_conf_dot<float><<<a.nfn, 256, 0, s>>>(a, static_cast<const float*>(x), static_cast<const float*>(y), out);
    return cudaGetLastError();
}

cudaError_t conf_cg_step1(const ConfLaunch& a, const double* rr, const double* pAp, const void* p, const void* Ap, void* x,
                          void* r, cudaStream_t s) {
    const dim3 gr(64, a.nfn);
    if (a.prec == 0)
        k_cg_step1<double><<<gr, 256, 0, s>>>(a, rr, pAp, static_cast<const double*>(p), static_cast<const double*>(Ap),
                                              static_cast<double*>(x), static_cast<double*>(r));
    else
        k_cg_step1<float><<<gr, 256, 0, s>>>(a, rr, pAp, static_cast<const float*>(p), static_cast<const float*>(Ap),
                                             static_cast<float*>(x), static_cast<float*>(r));
    return cudaGetLastError();
}

cudaError_t conf_cg_step2(const ConfLaunch& a, double* rr, const double* rr_new, const void* r, void* p, double* res,
                          cudaStream_t s) {
    const dim3 gr(64, a.nfn);
    if (a.prec == 0)
        k_cg_step2<double><<<gr, 256, 0, s>>>(a, rr, rr_new, static_cast<const double*>(r), static_cast<double*>(p), res);
    else
        k_cg_step2<float><<<gr, 256, 0, s>>>(a, rr, rr_new, static_cast<const float*>(r), static_cast<float*>(p), res);
    k_cg_swap<<<(a.nfn + 127) / 128, 128, 0, s>>>(a, rr, rr_new);
    return cudaGetLastError();
}

}  // namespace lsw
