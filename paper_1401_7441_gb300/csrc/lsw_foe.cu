// sm_103a kernels of the Fermi operator expansion of the density kernel (App. "Fermi
// operator expansion"; Sec. "Density kernel optimization"), FP64 on the sparsity
// pattern of H and S (CSR: rows a, ascending columns b; the pattern is symmetric and
// holds the diagonal).  Every matrix is a vector of values on that pattern.
//
//   k_foe_prep    H~ = sigma (H - tau S) and the Taylor S^-1/2 = (3 I - S) / 2
//   k_triple      Y = X A X restricted to the pattern: per row i, w = X_i. A is summed
//                 exactly (over every column it reaches) in a per-CTA dense row of the
//                 scratch, then Y_il = sum_m w_m X_ml for the pattern's l
//   k_cheb        one Chebyshev step for every column l of the pattern:
//                 t_l^{j+1} = alpha H~' t_l^j - t_l^{j-1}, kept on pattern column l;
//                 the columns are stored transposed (column l of T on row l of the CSR),
//                 the entries of t_l^j are found through a map in shared memory
//   k_trace       sum of the diagonal entries (one CTA, fixed order)
//   k_axpy_t      K'(transposed) += c T_j(transposed)
//   k_transpose   values on (i, l) <- values on (l, i)
//   k_ebs         E_BS = sum_{il} K_il (H~_li / sigma + tau S_li) (one CTA, fixed order)
#include <cstdint>

#include "lsw_device.h"
#include "lsw_internal.h"

namespace lsw {

__global__ void k_foe_prep(const double* __restrict__ H, const double* __restrict__ S, const int64_t* __restrict__ row_ptr,
                           const int32_t* __restrict__ col, int n, double sigma, double tau, double* __restrict__ Ht,
                           double* __restrict__ X) {
    const int a = blockIdx.x * blockDim.y + threadIdx.y;
    if (a >= n) return;
    for (int64_t k = row_ptr[a] + threadIdx.x; k < row_ptr[a + 1]; k += blockDim.x) {
        Ht[k] = sigma * (H[k] - tau * S[k]);
        X[k] = 0.5 * (3.0 * (col[k] == a ? 1.0 : 0.0) - S[k]);
    }
}

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Y = X A X on the pattern; tpos[q] = position of the transposed entry of q.  Each CTA
// owns the dense row scratch w + blockIdx.x * n (zero on entry, zero again on exit).
__global__ void __launch_bounds__(256) k_triple(FoeLaunch a, const double* __restrict__ X, const double* __restrict__ A,
                                                double* __restrict__ Y) {
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = 14;
    double* w = a.scratch + static_cast<int64_t>(blockIdx.x) * a.n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = blockIdx.x; i < a.n; i += gridDim.x) {
        const int64_t r0 = LD(a.row_ptr, i, a.n + 1), r1 = LD(a.row_ptr, i + 1, a.n + 1);
        // w_m = sum_k X_ik A_km
        for (int64_t q = r0 + warp; q < r1; q += nw) {
            const int k = LD(a.col, q, a.nnz);
            const double x = LD(X, q, a.nnz);
            const int64_t s0 = LD(a.row_ptr, k, a.n + 1), s1 = LD(a.row_ptr, k + 1, a.n + 1);
            for (int64_t p = s0 + lane; p < s1; p += 32) {
                const int m = LD(a.col, p, a.nnz);
                atomicAdd(&w[m], x * LD(A, p, a.nnz));
            }
        }
        __syncthreads();
        // Y_il = sum_m w_m X_ml, m over row l of the transposed X (X_ml = X[tpos[q]])
        for (int64_t q = r0 + warp; q < r1; q += nw) {
            const int l = LD(a.col, q, a.nnz);
            const int64_t s0 = LD(a.row_ptr, l, a.n + 1), s1 = LD(a.row_ptr, l + 1, a.n + 1);
            double acc = 0.0;
            for (int64_t p = s0 + lane; p < s1; p += 32) {
                const int m = LD(a.col, p, a.nnz);
                acc += LD(w, m, a.n) * LD(X, LD(a.tpos, p, a.nnz), a.nnz);
            }
            acc = warp_sum_d(acc);
            if (lane == 0) ST(Y, q, a.nnz, acc);
        }
        __syncthreads();
        for (int64_t q = r0 + warp; q < r1; q += nw) {
            const int k = LD(a.col, q, a.nnz);
            const int64_t s0 = LD(a.row_ptr, k, a.n + 1), s1 = LD(a.row_ptr, k + 1, a.n + 1);
            for (int64_t p = s0 + lane; p < s1; p += 32) ST(w, LD(a.col, p, a.nnz), a.n, 0.0);
        }
        __syncthreads();
    }
}

// One Chebyshev step on every column (transposed storage: Tc[pos(l, k)] = T_kl):
//   Tn[pos(l, i)] = alpha sum_k Htp_ik Tc[pos(l, k)] - (Tp ? Tp[pos(l, i)] : 0)
// map (shared, a.n ints, -1 outside the column) gives the position of k in row l.
__global__ void __launch_bounds__(256) k_cheb(FoeLaunch a, const double* __restrict__ Htp, const double* __restrict__ Tc,
                                              const double* __restrict__ Tp, double alpha, double* __restrict__ Tn) {
    [[maybe_unused]] int* ST_ = a.status;
    [[maybe_unused]] constexpr int KID = 15;
    extern __shared__ int map[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = threadIdx.x; i < a.n; i += blockDim.x) map[i] = -1;
    __syncthreads();
    for (int l = blockIdx.x; l < a.n; l += gridDim.x) {
        const int64_t r0 = LD(a.row_ptr, l, a.n + 1), r1 = LD(a.row_ptr, l + 1, a.n + 1);
        for (int64_t q = r0 + threadIdx.x; q < r1; q += blockDim.x) ST(map, LD(a.col, q, a.nnz), a.n, static_cast<int>(q - r0));
        __syncthreads();
        for (int64_t q = r0 + warp; q < r1; q += nw) {
            const int i = LD(a.col, q, a.nnz);
            const int64_t s0 = LD(a.row_ptr, i, a.n + 1), s1 = LD(a.row_ptr, i + 1, a.n + 1);
            double acc = 0.0;
            for (int64_t p = s0 + lane; p < s1; p += 32) {
                const int j = LD(map, LD(a.col, p, a.nnz), a.n);
                if (j >= 0) acc += LD(Htp, p, a.nnz) * LD(Tc, r0 + j, a.nnz);
            }
            acc = warp_sum_d(acc);
            if (lane == 0) ST(Tn, q, a.nnz, alpha * acc - (Tp ? LD(Tp, q, a.nnz) : 0.0));
        }
        __syncthreads();
        for (int64_t q = r0 + threadIdx.x; q < r1; q += blockDim.x) ST(map, LD(a.col, q, a.nnz), a.n, -1);
        __syncthreads();
    }
}

__device__ double block_sum_d(double v) {
    __shared__ double part[32];
    v = warp_sum_d(v);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < static_cast<int>(blockDim.x >> 5); ++i) s += part[i];
    return s;
}

// out[0] = sum of the diagonal entries of T (positions diag[0 .. n))
__global__ void __launch_bounds__(1024) k_trace(const double* __restrict__ T, const int64_t* __restrict__ diag, int n,
                                                double* __restrict__ out) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += T[diag[i]];
    const double s = block_sum_d(v);
    if (threadIdx.x == 0) *out = s;
}

__global__ void k_axpy_t(double* __restrict__ K, const double* __restrict__ T, double c, int64_t nnz) {
    for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < nnz;
         k += static_cast<int64_t>(gridDim.x) * blockDim.x)
        K[k] += c * T[k];
}

__global__ void k_transpose(const double* __restrict__ src, const int64_t* __restrict__ tpos, double* __restrict__ dst,
                            int64_t nnz) {
    for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < nnz;
         k += static_cast<int64_t>(gridDim.x) * blockDim.x)
        dst[k] = src[tpos[k]];
}

// E_BS = sum over pattern entries (i, l) of K_il (Ht_li / sigma + tau S_li)
__global__ void __launch_bounds__(1024) k_ebs(const double* __restrict__ K, const double* __restrict__ Ht,
                                              const double* __restrict__ S, const int64_t* __restrict__ tpos, int64_t nnz,
                                              double sigma, double tau, double* __restrict__ out) {
    double v = 0.0;
    for (int64_t k = threadIdx.x; k < nnz; k += blockDim.x) {
        const int64_t t = tpos[k];
        v += K[k] * (Ht[t] / sigma + tau * S[t]);
    }
    const double s = block_sum_d(v);
    if (threadIdx.x == 0) *out = s;
}

// ---------------------------------------------------------------- host wrappers

cudaError_t configure_foe_kernels(size_t max_smem) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_cheb);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_cheb, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(max_smem - fa.sharedSizeBytes));
}

cudaError_t foe_prep(const FoeLaunch& a, const double* H, const double* S, double sigma, double tau, double* Ht,
                     double* X, cudaStream_t s) {
    k_foe_prep<<<(a.n + 7) / 8, dim3(32, 8), 0, s>>>(H, S, a.row_ptr, a.col, a.n, sigma, tau, Ht, X);
    return cudaGetLastError();
}

cudaError_t foe_triple(const FoeLaunch& a, const double* X, const double* A, double* Y, cudaStream_t s) {
    k_triple<<<a.triple_ctas, 256, 0, s>>>(a, X, A, Y);
    return cudaGetLastError();
}

cudaError_t foe_cheb(const FoeLaunch& a, const double* Htp, const double* Tc, const double* Tp, double alpha, double* Tn,
                     cudaStream_t s) {
    k_cheb<<<a.cheb_ctas, 256, static_cast<size_t>(a.n) * sizeof(int), s>>>(a, Htp, Tc, Tp, alpha, Tn);
    return cudaGetLastError();
}

cudaError_t foe_trace(const FoeLaunch& a, const double* T, double* out, cudaStream_t s) {
    k_trace<<<1, 1024, 0, s>>>(T, a.diag, a.n, out);
    return cudaGetLastError();
}

cudaError_t foe_axpy_t(const FoeLaunch& a, double* K, const double* T, double c, cudaStream_t s) {
    k_axpy_t<<<static_cast<unsigned>(std::min<int64_t>((a.nnz + 255) / 256, 8192)), 256, 0, s>>>(K, T, c, a.nnz);
    return cudaGetLastError();
}

cudaError_t foe_transpose(const FoeLaunch& a, const double* src, double* dst, cudaStream_t s) {
    k_transpose<<<static_cast<unsigned>(std::min<int64_t>((a.nnz + 255) / 256, 8192)), 256, 0, s>>>(src, a.tpos, dst, a.nnz);
    return cudaGetLastError();
}

cudaError_t foe_ebs(const FoeLaunch& a, const double* K, const double* Ht, const double* S, double sigma, double tau,
                    double* out, cudaStream_t s) {
    k_ebs<<<1, 1024, 0, s>>>(K, Ht, S, a.tpos, a.nnz, sigma, tau, out);
    return cudaGetLastError();
}

}  // namespace lsw
