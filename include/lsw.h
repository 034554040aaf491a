/*
 * lsw.h -- C ABI of the GB300 (sm_103a) library for the localized Hamiltonian
 * application and the sparse H_ab / S_ab build of Daubechies-wavelet linear-scaling
 * DFT (arXiv 1401.7441).
 *
 * Problem statement (Sec. III, Eq. loccon; Sec. III.B; Sec. II.A): support functions
 * phi_alpha, each stored on its localization region L(alpha) (a sphere of radius
 * R_cut around its atom on a two-resolution Daubechies-16 grid, Sec. II.B), and a
 * local potential V(r) on the real-space grid of spacing h/2.  Compute
 *     H phi_alpha = L'(alpha) H L(alpha) phi_alpha,   H = -1/2 nabla^2 + V,
 * with L' of radius R_cut + 8 grid points (Sec. III.B), and the sparse matrices
 *     S_ab = <phi_a|phi_b>,  H_ab = <phi_a|H phi_b>
 * on the pattern of pairs whose atoms lie within a cutoff (Sec. II.A; Sec. IV.A
 * "Suitability of the methods": sparse matrices in compressed form).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every call returns an lsw_status.  On failure nothing was enqueued, and
 *   lsw_last_error() returns a message for the calling thread.
 * - Grid: coarse point (i1, i2, i3), 0 <= i_d < N_d, sits at (i1 h, i2 h, i3 h);
 *   fine real-space point j sits at j h / 2.  Global index g = i1 + N1 (i2 + N2 i3).
 * - Membership (locregs, fine spheres, pattern) is inclusive, d^2 <= R^2, with d^2
 *   computed in IEEE FP64 as ((x-X)^2 + (y-Y)^2) + (z-Z)^2 without fused operations.
 * - The fine region is the union of every atom's fine sphere (LSW_FINE_UNION, Sec.
 *   II.B) or, per locreg, its own atom's sphere (LSW_FINE_OWN).
 * - Compressed layout of one support function on a region: the scaling coefficients
 *   s at the region's coarse points in key order, then seven planes d^1..d^7 at its
 *   fine points in key order; wavelet type l = bx + 2 by + 4 bz (b_d = 1: wavelet
 *   along dimension d).  Functions are numbered atom by atom; function f starts at
 *   element off[f] (multiples of 64 elements).
 * - Ownership: the caller owns every pointer it passes (device buffers may come
 *   from any allocator, e.g. PyTorch).  Host arrays returned by the library stay
 *   valid until the owning object is destroyed.  The library owns its keys, plans
 *   and device workspace (lsw_workspace_bytes).
 * - Asynchrony: device work is enqueued on the context's stream; calls return after
 *   enqueueing.  Only lsw_sync and lsw_step_host wait for the device.
 * - Device-side checks never trap: they set a status word that lsw_sync reports.
 */
#ifndef LSW_H
#define LSW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LSW_OK = 0,
    LSW_ERR_ARG = 1,          /* invalid argument (detected before any launch)   */
    LSW_ERR_OOM = 2,          /* device or host allocation failed                */
    LSW_ERR_CUDA = 3,         /* a CUDA runtime call failed                      */
    LSW_ERR_TIMEOUT = 4,      /* lsw_sync: the device did not finish in time     */
    LSW_ERR_STATE = 5,        /* wrong call order (e.g. no potential set)        */
    LSW_ERR_UNSUPPORTED = 6,  /* valid but outside what the library supports    */
    LSW_ERR_IO = 7            /* lsw_save / lsw_load: file cannot be written/read */
} lsw_status;

#define LSW_HOST_ONLY (-1)

/* Arithmetic of a system.  LSW_FP64 and LSW_FP32: phi, H phi, V and every convolution
 * in that type.  LSW_FP32_BF16X: FP32 storage and arithmetic, except the z-direction
 * combined synthesis + magic filter and its transpose (the band-Toeplitz passes of the
 * z stage, Sec. II.B), which run as split-bfloat16 products on the tensor cores with
 * FP32 accumulation: each FP32 operand is split into 2 bfloat16 parts and the 3
 * products of order <= 1 are summed (option "zsplit" = 3: 3 parts, 6 products, FP32
 * rounding level).  H, S and energies are FP64 accumulations in every mode. */
typedef enum { LSW_FP64 = 0, LSW_FP32 = 1, LSW_FP32_BF16X = 2 } lsw_precision;
typedef enum { LSW_REGION_L = 0, LSW_REGION_LP = 1 } lsw_region;
typedef enum { LSW_PART_COARSE = 0, LSW_PART_FINE = 1 } lsw_part;
typedef enum { LSW_FINE_UNION = 0, LSW_FINE_OWN = 1 } lsw_fine_mode;
typedef enum { LSW_PAIR_CUTOFF = 0, LSW_PAIR_SUM_OF_RADII = 1 } lsw_pair_mode;

/* Filter tables exported for cross-checks (lsw_filter_table, `which`). */
typedef enum {
    LSW_FILTER_H = 0,        /* low-pass h_j, j = -7..8 (least-asymmetric D16)       */
    LSW_FILTER_G = 1,        /* high-pass g_j = (-1)^j h_{1-j}, j = -7..8            */
    LSW_FILTER_MOMENTS = 2,  /* M_p = int x^p phi, p = 0..15                         */
    LSW_FILTER_MAGIC = 3,    /* magic filter w_l, l = -7..8                          */
    LSW_FILTER_KIN_R = 4,    /* r_l = int phi phi''(. - l), l = -14..14              */
    LSW_FILTER_KIN_HH = 5,   /* T_XY(l) = <X_0|d2/dx2|Y_l>, l = -14..14              */
    LSW_FILTER_KIN_HG = 6,
    LSW_FILTER_KIN_GH = 7,
    LSW_FILTER_KIN_GG = 8,
    LSW_FILTER_FWD_H = 9,    /* (w * h)_m = sum_k w_{m-k} h_k, m = -14..16           */
    LSW_FILTER_FWD_G = 10,   /* (w * g)_m, m = -14..16                               */
    LSW_FILTER_MOVL_0 = 11,  /* F^p(l) = int x^p phi(x) phi(x - l) dx, l = -14..14,   */
    LSW_FILTER_MOVL_1 = 12,  /* p = 0..4 (moment overlaps of the quartic confinement) */
    LSW_FILTER_MOVL_2 = 13,
    LSW_FILTER_MOVL_3 = 14,
    LSW_FILTER_MOVL_4 = 15
} lsw_filter;

typedef struct lsw_ctx_s* lsw_ctx;
typedef struct lsw_system_s* lsw_system;

/* Description of a system (all pointers host, read during lsw_system_create only). */
typedef struct {
    int32_t N[3];            /* coarse grid points per dimension (>= 1)              */
    double h;                /* coarse grid spacing, bohr (> 0)                      */
    int32_t n_atoms;         /* >= 1                                                 */
    const double* pos;       /* [n_atoms][3] atom centres, bohr, box coordinates     */
    const double* r_loc;     /* [n_atoms] locreg radius R_cut, bohr (> 0)            */
    const double* r_fine;    /* [n_atoms] fine-sphere radius, bohr (>= 0)            */
    const int32_t* n_sf;     /* [n_atoms] support functions on the atom (>= 0)       */
    double lprime_margin;    /* L' radius = R_cut + lprime_margin * h; 8 in Sec. III.B */
    double pair_cutoff;      /* LSW_PAIR_CUTOFF: bohr                                */
    int32_t pair_mode;       /* lsw_pair_mode                                        */
    int32_t fine_mode;       /* lsw_fine_mode                                        */
    int32_t precision;       /* lsw_precision of phi, H phi and the convolutions     */
} lsw_system_desc;

/* Message describing the last failure on this thread ("" if none).  Never NULL. */
const char* lsw_last_error(void);

/* Create a context on CUDA device `device`, enqueueing on `stream` (a cudaStream_t;
 * NULL = the legacy default stream, on which work is never captured into CUDA
 * graphs; pass a created stream to get graph replay).  device = LSW_HOST_ONLY
 * makes a host-only context: filters, geometry, keys and pattern are available, every
 * call that needs the device returns LSW_ERR_STATE.  Derives the filter tables (Sec. II.B readings:
 * least-asymmetric order-16 Daubechies factor, magic filter with the moments of phi,
 * Galerkin kinetic connection coefficients) in double-double arithmetic, rounds them
 * to FP64/FP32 once and uploads them.  *out receives the handle.
 * Errors: LSW_ERR_ARG (out NULL, bad device), LSW_ERR_CUDA. */
lsw_status lsw_ctx_create(int device, void* stream, lsw_ctx* out);

/* Destroy a context (all its systems must have been destroyed).  NULL is a no-op. */
lsw_status lsw_ctx_destroy(lsw_ctx ctx);

/* Copy filter table `which` (lsw_filter) to host `values` (capacity >= 32 doubles);
 * *first = index of values[0], *count = number of entries.  Host only. */
lsw_status lsw_filter_table(lsw_ctx ctx, int32_t which, int32_t* first, int32_t* count,
                            double* values);

/* Build a system: fine region, locregs L and L' of every atom (Eq. loccon, Sec. III.B),
 * their segment keys, the compressed layout, the pair pattern (CSR) and the device
 * plans and workspace.  Host work plus uploads; synchronous.
 * Errors: LSW_ERR_ARG (sizes, radii, NULL arrays), LSW_ERR_OOM, LSW_ERR_CUDA,
 * LSW_ERR_UNSUPPORTED (a locreg box too large for the on-chip pass tiles). */
lsw_status lsw_system_create(lsw_ctx ctx, const lsw_system_desc* desc, lsw_system* out);

/* Destroy a system after its device work has finished.  NULL is a no-op. */
lsw_status lsw_system_destroy(lsw_system sys);

/* Compressed layout: *n_sf functions; phi buffers hold total_L elements (of the
 * system precision), H phi buffers total_Lp; off_L / off_Lp are host arrays of
 * n_sf + 1 element offsets; sf_atom[f] is the atom of function f. */
lsw_status lsw_system_layout(lsw_system sys, int64_t* n_sf, int64_t* total_L,
                             int64_t* total_Lp, const int64_t** off_L,
                             const int64_t** off_Lp, const int32_t** sf_atom);

/* Segment keys of atom `atom`'s region (lsw_region) part (lsw_part): *nseg keys of
 * three int64 each (first g, last g inclusive, coefficient offset within the part),
 * sorted by g; a segment is a maximal run of members along i1. Host array. */
lsw_status lsw_system_keys(lsw_system sys, int32_t atom, int32_t region, int32_t part,
                           int64_t* nseg, const int64_t** keys);

/* Pair pattern: CSR with n_sf rows, columns ascending, *nnz entries; host arrays. */
lsw_status lsw_pattern(lsw_system sys, int64_t* nnz, const int64_t** row_ptr,
                       const int32_t** col);

/* Register the global potential: a device array of the system precision, stored
 * [k][j][i] (x fastest) over fine indices fine_lo[d] .. fine_lo[d]+fine_dims[d]-1.
 * It must cover [-14, 2 N_d + 14] in every dimension (every point the magic filter
 * reaches, free boundary).  The pointer is kept (not copied): the caller keeps the
 * buffer alive and unchanged while work that reads it is in flight.
 * Errors: LSW_ERR_ARG (NULL, coverage). */
lsw_status lsw_set_potential(lsw_system sys, const void* V_dev, const int64_t fine_lo[3],
                             const int64_t fine_dims[3]);

/* H phi for every support function (Sec. III.B): phi_dev (total_L elements, layout
 * off_L) -> hphi_dev (total_Lp elements, layout off_Lp), both of the system precision.
 * e_kin_dev / e_pot_dev (n_sf doubles each, may be NULL) receive <phi|T phi> and
 * <phi|V phi>.  Asynchronous.  phi and hphi must not overlap.
 * Errors: LSW_ERR_ARG (NULL buffers), LSW_ERR_STATE (no potential), LSW_ERR_CUDA. */
lsw_status lsw_apply_hamiltonian(lsw_system sys, const void* phi_dev, void* hphi_dev,
                                 double* e_kin_dev, double* e_pot_dev);

/* Allocation-free H phi.  The paper has no counterpart: this entry point exists for
 * callers that must not allocate device memory while they work - a serving process
 * that reserves its HBM budget up front and forbids allocation on the request path, or
 * an application whose device memory belongs to another allocator's pool (where a stray
 * cudaMalloc bypasses the pool's accounting and fails once the pool holds the memory).
 * Same arguments, layouts and results as lsw_apply_hamiltonian (tolerance of the
 * precision), computed batch by batch in a fixed 32 MiB device array that the library
 * defines at file scope: it calls no cudaMalloc, cudaFree or other allocating routine.
 * Limits and rules:
 * - Every GPU that loads the library holds the 32 MiB array until the process exits.
 * - The first call on a device looks up the array's device address (this may load the
 *   library's module); make that first call before any stream capture.
 * - All calls share the one array and leave the last call's contents in it; calls
 *   whose work overlaps on the GPU (other streams, other systems, other threads) race
 *   and produce wrong results: serialize them.
 * - Every support function is checked before anything is enqueued: one whose
 *   workspace (its dense L box, the two z-stage intermediates and its dense L' box)
 *   exceeds the array, or whose box exceeds the on-chip tiles, makes the call return
 *   LSW_ERR_UNSUPPORTED with nothing enqueued and the outputs untouched.
 * - Each batch's records are written into the array by a kernel from the system's
 *   resident records; the call reads no host memory on the device.
 * Asynchronous on the system's stream.
 * Errors: LSW_ERR_ARG (NULL buffers), LSW_ERR_STATE (no potential, host-only context),
 * LSW_ERR_UNSUPPORTED, LSW_ERR_CUDA. */
lsw_status lsw_apply_hamiltonian_noalloc(lsw_system sys, const void* phi_dev, void* hphi_dev,
                                         double* e_kin_dev, double* e_pot_dev);

/* Sparse matrices on the pattern (Sec. II.A): H_dev[k] = <phi_a|H phi_b> (raw, not
 * symmetrized) and S_dev[k] = <phi_a|phi_b> for the k-th pattern entry (a, b).  Computed
 * in the transposed layout of App. D: per tile of T^3 coarse points (option "tile"),
 * panels hold the coefficients of every function present there (phi on L, H phi on L'),
 * and each tile's contributions are a small dense product in the system's precision,
 * added to the FP64 values (FP64 accumulation across tiles in every precision).  The
 * panels live in a library buffer of one slab of tiles (option "slab_mb").
 * Asynchronous.
 * Errors: LSW_ERR_ARG (NULL), LSW_ERR_CUDA. */
lsw_status lsw_build_matrices(lsw_system sys, const void* phi_dev, const void* hphi_dev,
                              double* H_dev, double* S_dev);

/* Sparse combination of support functions (Sec. "Orthogonalization" and Sec. "Gradient
 * and preconditioning", Eq. gradient: sums over overlapping functions, then localized
 * onto each function's region):
 *     (M Phi)_a = L(a) sum_b M_ab phi_b
 * for M given as FP64 values on the pattern (lsw_pattern: M_dev[k] belongs to the k-th
 * entry (a, b); entries outside the pattern count as 0; M need not be symmetric).  Each
 * phi_b contributes its coefficients at its own members; the sum is read back at the
 * members of L(a) (scaling and wavelet parts).  phi_in_dev and phi_out_dev: compressed
 * support functions on L (layout off_L, system precision); they must not overlap.  Only
 * the members of each function are written (the alignment gaps keep their contents).
 * The work runs in the transposed layout of the H/S build (App. D): per tile of the
 * grid, the functions present there are combined as a small dense product (FP32 with
 * FP32 sums for reduced-precision systems, M rounded to FP32; FP64 otherwise).
 * Asynchronous.  Errors: LSW_ERR_ARG (NULL, overlapping buffers), LSW_ERR_STATE
 * (host-only context), LSW_ERR_CUDA. */
lsw_status lsw_combine(lsw_system sys, const double* M_dev, const void* phi_in_dev, void* phi_out_dev);

/* Loewdin re-orthonormalization with the first-order Taylor form of S^-1/2 (Sec.
 * "Orthogonalization": the functions stay close to orthonormal, so S^-1/2 is replaced by
 * (3 I - S) / 2):  phi'_a = L(a) sum_b (3 delta_ab - S_ab) / 2 phi_b, with S_dev the
 * overlap values on the pattern (as lsw_build_matrices writes them).  Same layouts and
 * rules as lsw_combine; the coefficients are formed on the device in a library buffer
 * (allocated at the first call, counted by lsw_workspace_bytes).  Asynchronous.
 * Errors: as lsw_combine. */
lsw_status lsw_lowdin_taylor(lsw_system sys, const double* S_dev, const void* phi_in_dev, void* phi_out_dev);

/* Fermi operator expansion of the density kernel (App. "Fermi operator expansion";
 * Sec. "Density kernel optimization"), on the pattern of lsw_pattern (symmetric, with the
 * diagonal), FP64 throughout:
 *   H~ = sigma (H - tau S), sigma = 2 / (e_max - e_min), tau = (e_min + e_max) / 2;
 *   H~' = X H~ X restricted to the pattern, X = (3 I - S) / 2 (first-order Taylor S^-1/2);
 *   K' = c_0/2 I + sum_{j=1}^{n_pl} c_j T_j(H~'), column by column with the recursion
 *   t^{j+1} = 2 H~' t^j - t^{j-1}, every column cut to its pattern column after each
 *   product (the linear-scaling evaluation); the c_j are those of the polynomial
 *   interpolating f(x) = 1/2 [1 - erf((x - sigma (mu - tau)) / (sigma de))] at the n_pl + 1
 *   Chebyshev nodes;
 *   mu by bisection on [e_min, e_max] until |Tr K' - n_el| <= tol (at most max_bisect
 *   steps; Tr K' for a trial mu comes from the traces of the T_j, computed once);
 *   K = X K' X restricted to the pattern; E_BS = Tr(K H~) / sigma + tau Tr(K S).
 * - H_dev, S_dev: FP64 values on the pattern (as lsw_build_matrices writes them);
 *   e_min, e_max: bounds of the spectrum of H c = e S c (the library does not compute
 *   them); n_el: the target of Tr K' (occupied orbitals, occupations in [0, 1]); de: the
 *   smearing width in the units of H.
 * - Kp_dev, K_dev: FP64 outputs on the pattern (nnz each).  *mu_out, *ebs_out, *trace_out
 *   (host, may be NULL) receive mu, E_BS and the final Tr K'.
 * Synchronous (the search of mu runs on the host from the device traces).  Work buffers
 * are allocated at the first call (lsw_workspace_bytes).
 * Errors: LSW_ERR_ARG (NULL, e_max <= e_min, de <= 0, n_pl < 1), LSW_ERR_STATE (host-only),
 * LSW_ERR_UNSUPPORTED (pattern not symmetric or without the diagonal; more functions than
 * the shared-memory column map holds), LSW_ERR_CUDA. */
lsw_status lsw_foe(lsw_system sys, const double* H_dev, const double* S_dev, double e_min, double e_max, double n_el,
                   int32_t n_pl, double de, double tol, int32_t max_bisect, double* Kp_dev, double* K_dev,
                   double* mu_out, double* ebs_out, double* trace_out);

/* Quartic confining potential (Sec. "Support function optimization": in the first
 * iterations each support function alpha sees its own Hamiltonian
 * H_alpha = H_KS + a_alpha (r - R_alpha)^4, R_alpha its atom's centre):
 *     hphi_dev += L'(alpha) a_alpha Q_alpha L(alpha) phi_alpha,
 *     e_conf_dev[alpha] = <phi_alpha | a_alpha Q_alpha | phi_alpha>,
 * Q_alpha the Galerkin matrix of (r - R_alpha)^4 = sum_d X_d^4 + 2 sum_{d<e} X_d^2 X_e^2 in
 * the two-level basis: each X_d^m a 1D operator along d between the scaling and wavelet
 * functions of coarse points i, j (|j - i| <= 14), its entries built from the moment
 * overlaps F^p of the filter set and the powers of (2 i + k - 2 R_d / h) (the text: "in
 * the same manner as the kinetic energy").  Call after lsw_apply_hamiltonian on the same
 * buffers to get H_alpha phi_alpha.  a_dev: n_sf FP64 prefactors (device); phi_dev on L,
 * hphi_dev on L' (layouts of lsw_system_layout, system precision); e_conf_dev: n_sf FP64
 * or NULL.  The first call builds the operator tables of every atom (host, then
 * uploaded; lsw_workspace_bytes) and the batch boxes.  Asynchronous.
 * Errors: LSW_ERR_ARG (NULL), LSW_ERR_STATE (host-only), LSW_ERR_CUDA. */
lsw_status lsw_add_confinement(lsw_system sys, const double* a_dev, const void* phi_dev, void* hphi_dev,
                               double* e_conf_dev);

/* One row of the 1D operator tables of lsw_add_confinement, for cross-checks (host, no
 * device work): out[l + 14] = <chi^b_i | (x_dim - R_dim)^m | chi^b'_{i+l}>, l = -14..14,
 * for coarse index i along dimension dim (0..2), m = 2 or 4, b, b' = 0 (scaling) or 1
 * (wavelet), R the centre of atom `atom`.  Errors: LSW_ERR_ARG. */
lsw_status lsw_confinement_row(lsw_system sys, int32_t atom, int32_t dim, int32_t m, int32_t b, int32_t bp, int64_t i,
                               double* out);

/* Preconditioning of the support-function gradient (Sec. "Gradient and preconditioning",
 * Eq. precond): for every function alpha, `iters` conjugate-gradient iterations from
 * g_prec = 0 on
 *     A g_prec = -g,   A = L(alpha) (-1/2 nabla^2 + a_alpha (r - R_alpha)^4 - eps_alpha) L(alpha),
 * the kinetic part by the Galerkin blocks, the quartic as in lsw_add_confinement.  The
 * iteration of each function is its own (its own step lengths); it stops changing once
 * its residual is exactly zero.  g_dev, gprec_dev: compressed on L (system precision),
 * not overlapping (only members are written); a_dev, eps_dev: n_sf FP64 (eps_alpha < 0
 * keeps A positive definite); res_dev: iters x n_sf FP64 residual 2-norms after each
 * iteration (row = iteration), or NULL.  Vectors in the system precision, dot products
 * in FP64.  Asynchronous.  Errors: LSW_ERR_ARG (NULL, overlap, iters < 1),
 * LSW_ERR_STATE (host-only), LSW_ERR_CUDA. */
lsw_status lsw_precondition(lsw_system sys, const double* a_dev, const double* eps_dev, const void* g_dev,
                            void* gprec_dev, int32_t iters, double* res_dev);

/* Electronic density (Sec. II.A, Eq. density; App. D forms it like the scalar
 * products): rho_j = sum_ab K_ab u_a(j) u_b(j) at every fine point x_j = j h/2 of the
 * grid block [fine_lo, fine_lo + fine_dims), where u_a = M W L phi_a are the real-space
 * values of support function a (uncompress, one-level synthesis, magic filter: the
 * values the potential step of lsw_apply_hamiltonian multiplies), defined on the fine
 * points [2 lo - 14, 2 hi + 16] of its locreg's coarse bounding box [lo, hi], 0 outside.
 * rho_j is the electron count carried by point j; the density there is rho_j / (h/2)^3.
 * - phi_dev: compressed support functions (layout of lsw_system_layout), FP64 for an
 *   FP64 system, FP32 otherwise.
 * - K_dev: FP64 values of the density kernel on the pattern (lsw_pattern): K_dev[k]
 *   belongs to the k-th entry (a, b); entries outside the pattern count as 0.  K need
 *   not be symmetric (the result depends only on its symmetric part).
 * - rho_dev: FP64 output, fine_dims[2] x fine_dims[1] x fine_dims[0] values stored
 *   [z][y][x] (x fastest), every point written.
 * - The grid must cover fine indices [-14, 2 N_d + 14] in every dimension (the points
 *   any block reaches), like the potential.
 * The real-space values are computed in the system's precision (FP64, or FP32 with FMA
 * arithmetic for LSW_FP32 and LSW_FP32_BF16X); the pair products of a point run in that
 * precision per group of 32 x 32 functions, the sum over groups in FP64.  The first
 * call for a grid builds per-tile function lists on the host and allocates a device
 * store of every function's real-space block (counted by lsw_workspace_bytes); later
 * calls on the same grid reuse them.  Asynchronous.
 * Errors: LSW_ERR_ARG (NULL, grid not covering), LSW_ERR_STATE (host-only context),
 * LSW_ERR_UNSUPPORTED (grid too large), LSW_ERR_OOM / LSW_ERR_CUDA. */
lsw_status lsw_build_density(lsw_system sys, const void* phi_dev, const double* K_dev, double* rho_dev,
                             const int64_t fine_lo[3], const int64_t fine_dims[3]);

/* Reuse support functions on a changed geometry (the paper moves them with the atoms
 * between geometry steps, section "Flexibility of the minimal basis formalism",
 * subsection "Geometry optimization", with an interpolation scheme it does not
 * specify; this library's reading: integer grid shifts only, no sub-grid interpolation).  `dst` and `src`
 * have the same atoms (in the same order, same functions per atom, same precision,
 * same device); dst's atom a is src's atom a moved by shift[3a..3a+2] grid points
 * (host array, typically the change of the atom's nearest grid point).  For every
 * function f and every member p of L_dst(f): phi_dst = phi_src at p - shift if that
 * point is a member of L_src(f) (coarse part for s, fine part for d^1..d^7), else 0.
 * phi_src uses src's layout, phi_dst dst's; they must not overlap.  Enqueued on dst's
 * stream after the work already enqueued on src's stream.
 * Errors: LSW_ERR_ARG (mismatched systems, NULL), LSW_ERR_STATE, LSW_ERR_CUDA. */
lsw_status lsw_reformat(lsw_system dst, lsw_system src, const int32_t* shift, const void* phi_src_dev,
                        void* phi_dst_dev);

/* Roofline denominators measured on the context's GPU (no counterpart in the paper):
 * FP32 and FP64 FMA rates of a dependent-chain FMA loop over every SM, TFLOP/s, and the
 * rate of a 16-byte streaming copy between two 1 GiB device buffers, GB/s (bytes read +
 * written).  Best of 5 timed repetitions each.  Synchronous: waits for the whole device,
 * allocates and frees 2 GiB.  Errors: LSW_ERR_ARG, LSW_ERR_STATE (host-only context),
 * LSW_ERR_CUDA. */
lsw_status lsw_measure_peaks(lsw_ctx ctx, double* fp32_tflops, double* fp64_tflops, double* copy_gbs);

/* Device memory of the system, bytes: what it holds, plus the H/S panel buffers of one
 * slab, which the first lsw_build_matrices, lsw_combine or lsw_lowdin_taylor allocates
 * (so a request loop can budget a system before it runs). */
lsw_status lsw_workspace_bytes(lsw_system sys, int64_t* bytes);

/* Wait for the system's enqueued work for at most timeout_s seconds (polling an
 * event; never blocks longer).  Returns LSW_ERR_TIMEOUT if still running,
 * LSW_ERR_CUDA on a device error, LSW_ERR_STATE if a device-side check fired. */
lsw_status lsw_sync(lsw_system sys, double timeout_s);

/* End-to-end step through host memory: copy phi from host (pinned or pageable),
 * apply H, build H_ab and S_ab, and copy the results back; returns when done.
 * hphi_host, e_kin_host and e_pot_host may be NULL (not copied back).  The copies are
 * pipelined with the H phi batches on two copy streams of the system: batch i's phi
 * goes up while batch i - 1 runs, and its H phi comes back while later batches run (with
 * pinned host buffers the copies overlap the kernels; pageable ones are still correct).
 * The H phi batches of this call are not captured in a CUDA graph; H/S is. */
lsw_status lsw_step_host(lsw_system sys, const void* phi_host, void* hphi_host,
                         double* H_host, double* S_host, double* e_kin_host,
                         double* e_pot_host);

/* Enqueue this system's future work on `stream` (a cudaStream_t of the system's
 * device; NULL = the legacy default stream) instead of its context's stream.  Waits
 * for the work already enqueued on the old stream.  Lets a server build systems on one
 * stream (creation waits for its uploads) and run each request on its own stream. */
lsw_status lsw_system_set_stream(lsw_system sys, void* stream);

/* Device trace of the enqueued kernels.  enable = 1 records a CUDA event pair around
 * every launch the system enqueues from now on (inside CUDA graphs as event-record
 * nodes); enable = 0 stops.  Waits for the stream and drops cached graphs. */
lsw_status lsw_profile(lsw_system sys, int32_t enable);

/* Summed device milliseconds and launch counts per kernel kind since the last read,
 * kinds in this order: 0 memset, 1 uncompress, 2 forward xy, 3 z stage with V,
 * 4 backward xy (with the compressed write), 5 kinetic z arm, 6 (unused), 7 H/S tiles,
 * 8 density real-space values, 9 density pair products.  Waits for the stream.  Writes
 * min(max_kinds, *n_kinds) entries of ms[] and launches[]; resets the totals. */
lsw_status lsw_profile_read(lsw_system sys, int32_t max_kinds, int32_t* n_kinds, double* ms,
                            int64_t* launches);

/* Checkpoint (no counterpart in the paper, which restarts from its own files): write
 * the system description and, if phi_dev is not NULL, the compressed support functions
 * (total_L values of the system precision, device) to `path`.  Waits for the system's
 * stream.  File: "LSWSAVE1", int32 version 1, then the lsw_system_desc fields, the
 * atom arrays, the "zsplit" value, int64 total_L, int64 has_phi, phi; little-endian.
 * Errors: LSW_ERR_ARG (NULL), LSW_ERR_IO, LSW_ERR_CUDA. */
lsw_status lsw_save(lsw_system sys, const void* phi_dev, const char* path);

/* Rebuild a saved system on `ctx` (same arithmetic as lsw_system_create, so keys,
 * layout and pattern are identical; "zsplit" is restored, the other options take
 * their defaults) and, if phi_dev is not NULL, copy the saved
 * support functions into it (device, total_L values; the file must hold them).  Pass
 * NULL first to learn total_L from lsw_system_layout, then lsw_load_phi.  Synchronous.
 * Errors: LSW_ERR_ARG, LSW_ERR_IO (unreadable or not a checkpoint), LSW_ERR_STATE (no
 * support functions in the file), and those of lsw_system_create. */
lsw_status lsw_load(lsw_ctx ctx, const char* path, lsw_system* out, void* phi_dev);

/* Copy the support functions saved in `path` into phi_dev (device, total_L values of
 * sys, which must have been built from that file).  Synchronous.
 * Errors: LSW_ERR_ARG, LSW_ERR_IO, LSW_ERR_STATE (file without support functions or of
 * another layout). */
lsw_status lsw_load_phi(lsw_system sys, const char* path, void* phi_dev);

/* Tuning knob by name: "batch" (functions per HPhi batch), "graph" (0/1, capture the
 * enqueued work in a CUDA graph), "tile" (H/S tile edge, coarse points, 2..8),
 * "hs_tc" (FP32 and split-bfloat16 systems: 1, the default, runs the per-tile H/S products
 * as split-bfloat16 tensor-core products, 3 parts per FP32 value and 6 products, FP32
 * accumulation in tensor memory; 0 runs them on the FMA units),
 * "hphi_limit" (lsw_apply_hamiltonian computes H phi and the energies of functions
 * 0 .. value - 1 only, leaving the others' outputs untouched; -1, the default: every
 * function; a rank of a sharded run numbers its own functions first),
 * "slab_mb" (H/S and combination: panel budget of one slab of tiles, MiB; the panels of
 * consecutive tile-z layers are built and consumed slab by slab, default 8192),
 * "persistent" (bit 0: the backward FMA plane kernel of H phi, bit 1: the forward one,
 * runs as a persistent grid, as many CTAs as fit on the GPU, taking the batch's
 * (function, plane) items largest first from a device queue; a clear bit: one CTA per
 * plane slot of a (planes, functions) grid; the default 1, the backward kernel only,
 * measured fastest; the results are the same bits), "fwd_list" (1, the default: the forward plane kernel's x
 * pass computes only the blocks whose input window meets the row's members of L and
 * zeroes the rest; 0: every block; the same bits),
 * "zsplit" (LSW_FP32_BF16X systems only: 2 or 3 bfloat16 parts per FP32 operand of the
 * tensor-core z stage), "xy_tc" (LSW_FP32_BF16X systems only: 1 runs the x and y passes
 * of the plane kernels as split-bfloat16 tensor-core products as well; 0, the default,
 * keeps them on the FMA units, which measured faster).
 * Errors: LSW_ERR_ARG (unknown name or value), LSW_ERR_STATE ("zsplit" or "xy_tc" on
 * another precision), LSW_ERR_UNSUPPORTED (the locregs do not fit the tensor-core tiles
 * in shared memory; the previous value stays). */
lsw_status lsw_set_option(lsw_system sys, const char* name, int64_t value);

#ifdef __cplusplus
}
#endif

#endif /* LSW_H */
