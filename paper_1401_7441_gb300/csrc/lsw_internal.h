// Internal declarations shared by the host code (lsw_host.cpp, lsw_filters.cpp) and
// the CUDA kernels (lsw_kernels.cu).  Not part of the public ABI (include/lsw.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

namespace lsw {

constexpr int D16 = 16;          // filter length 2m, m = 8 (Sec. II.B)
constexpr int H_LO = -7;         // h, g, magic filter indices -7..8
constexpr int KIN_HALF = 14;     // kinetic blocks l = -14..14
constexpr int KIN_TAPS = 2 * KIN_HALF + 1;
constexpr int FWD_LO = -14;      // combined filters (w * h), (w * g): m = -14..16
constexpr int FWD_TAPS = 31;
constexpr int MOVL_P = 5;        // moment overlaps F^p, p = 0..4 (quartic confinement)
constexpr int V_REACH = 14;      // real-space box of a coarse block [lo, hi]: [2lo-14, 2hi+16]
constexpr int ALIGN_ELEMS = 64;  // function offsets in the compressed arrays
constexpr int ZCOLS_F64 = 64;    // real-space columns per block of the z stage (FP64)
constexpr int ZCOLS_F32 = 128;   // (FP32)
constexpr size_t BWD_STATIC_SMEM = 16 * 1024 + 512;   // upper bound of k_bwd_xy's static shared memory
constexpr size_t BWD_TC_STATIC_SMEM = 8 * 1024 + 512; // ... of its tensor-core versions (checked at set-up)
constexpr size_t FWD_STATIC_SMEM = 4 * 1024;          // ... of k_fwd_xy

// Filter tables, FP64 (rounded once from double-double).
struct FilterSet {
    double h[D16], g[D16], moments[D16], magic[D16];
    double kin_r[KIN_TAPS];
    double kin[4][KIN_TAPS];     // hh, hg, gh, gg: <X_0|d2|Y_l>
    double fwd[2][FWD_TAPS];     // (w*h)_m, (w*g)_m
    double movl[5][KIN_TAPS];    // F^p(l) = int x^p phi(x) phi(x - l) dx, p = 0..4
};

// Derive the whole table (lsw_filters.cpp).  Returns false with a message on failure.
bool derive_filters(FilterSet* out, std::string* err);

// A run of members along x inside a box: x0..x1 inclusive (box-local), row = y + ny*z
// (box-local), off = coefficient offset of x0 within its part.
struct Seg {
    int32_t x0, x1, row, off;
};

// Geometry of one atom's locregs as seen by the kernels.
struct AtomRec {
    int32_t lo[3], n[3];         // L box (coarse bounding box of the L members)
    int32_t lop[3], np[3];       // L' box
    int32_t ncL, nfL, ncP, nfP;  // member counts (coarse, fine) of L and L'
    int32_t nsegLc, nsegLf, nsegPc, nsegPf;
    int64_t segLc, segLf, segPc, segPf;  // first index in the global Seg array
    int64_t rowLc, rowLf, rowPc, rowPf;  // first index of the per-row CSR (n_rows + 1)
    int64_t colz;                // first entry of the L' column table (n_x' n_y' ColZ)
};

// Per (x, y) column of an L' box (entry y n_x' + x): the z range of its coarse members and
// the z hull of its fine members, L' box coordinates; -1, -1: none.
struct ColZ {
    int16_t c0, c1, f0, f1;
};

// One support function's real-space block in the density store (Eq. density): the
// values u = M W L phi on the fine points [2 lo - 14, 2 hi + 16] of its L box, stored
// [Z][Y][X] (x fastest) from element `off`.
struct DensFn {
    int64_t off;
    int32_t o[3];                // block origin, as a fine index local to the density grid
    int32_t d[3];                // X, Y, Z = 2 n + 29
};

// Density tiles: DT_X x DT_Y x DT_Z fine points (x fastest), one CTA each.
constexpr int DT_X = 32, DT_Y = 4, DT_Z = 4;
constexpr int DT_THREADS = 256;
constexpr int DT_PP = DT_X * DT_Y * DT_Z / DT_THREADS;   // points per thread
constexpr int DT_MC = 32;                                 // functions per chunk

// One support function inside an H phi batch.
struct FnRec {
    int32_t f, atom;
    int32_t lo[3], n[3], lop[3], np[3];
    int64_t off_phi, off_hphi;
    int64_t ws_D, ws_Bf, ws_Bb, ws_G;    // element offsets inside the batch workspace
    int64_t ws_Gf;                       // element offset of the z-arm column flags (bytes
                                         // [4][n_x n_y]: 1 where the D column pair is nonzero)
};

// The "transposed" layout of the scalar products (App. D) on one GPU: the grid is cut
// into tiles of T^3 coarse points; every function whose region touches a tile gets a
// panel row there holding its coefficients on the tile's points (T^3 scaling values,
// then the 7 wavelet values of each of the tile's fine points, zero where the function
// has no member, padded to a multiple of 4).  Panels of phi on L (the "A" side) and of
// H phi on L' (the "Q" side) turn S_ab and H_ab into small dense products per tile.
struct PanelTile {
    int32_t org[3];              // tile origin (coarse grid)
    int32_t fine0, nfine;        // the tile's fine points: tile_fine[fine0 .. fine0 + nfine)
    int32_t nA, nB;              // functions whose L (A) / L' (Q) touch the tile
    int32_t kp;                  // panel row length
    int64_t listA, listB;        // first entry of the tile's functions in listA / listB
    int64_t pA, pQ;              // element offsets of the tile's panels in its slab's buffers
};
// Per atom: its tile boxes (tiles its L and L' touch) and, per tile of each box, the
// used-tile index and the slot of the atom's first function in that tile's list
// (int2 {tile, slot}, tile = -1 where the region does not touch the tile).
struct PanelAtom {
    int32_t tloA[3], tnA[3];     // tile box of L
    int32_t tloB[3], tnB[3];     // tile box of L'
    int64_t tabA, tabB;          // first entry of the boxes' tables in the tile-table array
    int32_t f0, nsf;             // the atom's functions f0 .. f0 + nsf - 1
};
// One product work item: tile, rows a0 .. a0+na of its A list, columns c0 .. c0+nc of
// the concatenated column list [A list (S_ab); B list (H_ab)].
struct PanelItem {
    int32_t tile, a0, na, c0, nc, pad;
};
// One slab of tiles (consecutive tile-z layers) whose panels fit the panel buffers.
struct PanelSlab {
    int32_t tz0, tz1;            // tile-z layers tz0 .. tz1 - 1
    int64_t u0, u1;              // used tiles
    int64_t i0, i1;              // product items
    int64_t ci0, ci1;            // combination items (tile, A rows, panel entries)
    int64_t s0, s1;              // entries of the slab-atom list (atoms whose L' meets the slab)
    int64_t elemsA, elemsQ;      // panel elements of the slab
    size_t smem_pack;            // dynamic shared memory of the pack kernel (0: tables read from global)
};

// Kernel kinds of the per-launch device trace (lsw_profile / lsw_profile_read).
enum TraceKind : int {
    TK_MEMSET = 0, TK_UNCOMPRESS, TK_FWD_XY, TK_Z, TK_BWD_XY, TK_KINETIC, TK_PACK, TK_HS,
    TK_DENS_U, TK_DENSITY, TK_COUNT
};

// Host-side recorder of CUDA event pairs around launches; NULL = no tracing.
struct Tracer;
void trace_begin(Tracer* tr, int kind, cudaStream_t s);
void trace_end(Tracer* tr, cudaStream_t s);

struct HphiLaunch {
    Tracer* tr;
    int prec;                    // 0 FP64, 1 FP32
    const FnRec* fn;             // device records of this batch
    int nfn;
    int max_nz, max_nzp;         // largest L / L' z extents in the batch
    int max_cols;                // largest (2ny+29)(2nx+29) in the batch
    int max_rowsP;               // largest ny'*nz' of L'
    int64_t max_ptsP;            // largest nx'*ny'*nz' of L'
    int max_colsP;               // largest nx'*ny' of L'
    int max_colsL;               // largest nx*ny of L
    int max_rowsL;               // largest ny*nz of L
    int max_segL;                // largest coarse+fine segment count of L
    int max_segP;
    size_t smem_fwd, smem_z, smem_bwd;
    int gstage;                  // 1: the plane kernel stages the z-arm plane and column flags
                                 // in shared memory (smem_bwd includes them); 0: reads them
                                 // from global memory (the boxes leave no room)
    int zcols;                   // columns per CTA of the z stage
    int zsplit;                  // 0: z stage on FMA units; 2 or 3: bfloat16 parts per
                                 // FP32 operand of the tensor-core z stage
    int xy_tc;                   // 1: the x, y passes run on the tensor-core plane kernels too
                                 // (with zsplit parts); 0: on the FMA plane kernels
    size_t smem_ztc;             // dynamic shared memory of the tensor-core z stage
    size_t smem_bwd_tc;          // dynamic shared memory of the tensor-core plane kernel
    size_t smem_fwd_tc;          // dynamic shared memory of the tensor-core forward plane kernel
    size_t smem_kin;             // dynamic shared memory of the kinetic z-arm kernel
    // persistent FMA plane kernels: the batch's items (function << 11 | plane << 1 | z type),
    // largest planes first, taken from queue[0] (forward) and queue[1] (backward), which
    // are zeroed before the batch; grid_* CTAs (as many as fit on the GPU).  NULL items:
    // one CTA per (2 planes + z type, function) grid slot.
    const int32_t* items_fwd;
    const int32_t* items_bwd;
    int n_items_fwd, n_items_bwd;
    int grid_fwd, grid_bwd;
    int* queue;
    int fwd_list;                // 1: the forward x pass computes only the blocks whose input
                                 // window meets the row's members (the rest of its plane is 0)
    const AtomRec* atoms;
    const Seg* seg;
    const int32_t* rowptr;
    const ColZ* colz;            // L' column tables (NULL: the kinetic z arm computes every plane)
    int64_t colz_n;
    const void* phi;
    void* hphi;
    double* e_kin;
    double* e_pot;
    const void* V;
    int64_t vlo[3], vn[3];
    void* ws;                    // batch workspace base
    int64_t ws_D_elems;          // D region size (memset)
    double kin_scale;            // -1 / (2 h^2)
    int* status;
    // extents used by the self-checking build (-DLSW_CHECKED)
    int64_t phi_n, hphi_n, v_n, ws_n, seg_n, rowptr_n;
    int n_atoms;
    // density: real-space store written by the density z stage (NULL otherwise)
    void* U;
    const DensFn* dfn;           // per function (indexed by FnRec::f)
    int64_t U_n;
};

// The density products rho_j = sum_ab K_ab u_a(j) u_b(j) over the tiles of the grid.
struct DensLaunch {
    Tracer* tr;
    int prec;
    const DensFn* fn;            // per function
    const void* U;               // real-space store
    const int64_t* tptr;         // [ntiles + 1]: functions of tile t are tfn[tptr[t] .. tptr[t+1])
    const int32_t* tfn;          // ascending within a tile
    const int64_t* row_ptr;      // pattern CSR
    const int32_t* col;
    const double* K;             // density kernel on the pattern
    double* rho;                 // [gz][gy][gx]
    int64_t gn[3];               // grid extents
    int32_t ntile[3];
    int* status;
    // extents used by the self-checking build (-DLSW_CHECKED)
    int64_t U_n, tfn_n, nnz, rho_n, fn_n, tptr_n, rowp_n;
};

// Pack: panels of one slab (grid: slab atoms x 2 sides).
struct PackLaunch {
    Tracer* tr;
    int prec;
    const PanelTile* tiles;
    const PanelAtom* patoms;
    const int2* ttab;            // per-atom tile tables
    const int32_t* slab_atoms;   // atoms of this slab
    int n_slab_atoms;
    int tz0, tz1;
    int tile;                    // tile edge T
    int64_t u0;                  // first used tile of the slab
    const int32_t* tile_fine;    // fine points of the tiles: local x | y << 8 | z << 16
    const AtomRec* atoms;
    const Seg* seg;
    const int32_t* rowptr;
    const int64_t* off_L;
    const int64_t* off_Lp;
    const void* phi;
    const void* hphi;            // NULL: pack the A side only
    void* PA;
    void* PQ;
    size_t smem;                 // dynamic shared memory: 0 = region tables read from global
    void* out;                   // unpack (combination): compressed output on L; NULL: pack
    int* status;
    int64_t phi_n, hphi_n, seg_n, rowptr_n, fine_n, ttab_n, PA_n, PQ_n, out_n;
    int n_atoms, n_tiles, n_sf;
};

// Product: S_ab and H_ab contributions of one slab's tiles, added to the CSR values
// (or, for the combination, the output panels of one slab's tiles).
struct PanelHSLaunch {
    Tracer* tr;
    int prec;
    const PanelTile* tiles;
    const PanelItem* items;
    int64_t nitems;
    const int32_t* listA;
    const int32_t* listB;
    const int64_t* row_ptr;      // pattern CSR
    const int32_t* col;
    const void* PA;
    const void* PQ;              // combination: the output panels (A layout) in the Q buffer
    double* H;
    double* S;
    const double* M;             // combination: coefficients on the pattern
    int tc;                      // 1: FP32 products on the tensor cores (split bfloat16)
    int* status;
    int64_t listA_n, listB_n, nnz, PA_n, PQ_n, n_tiles;
    int n_sf;
};

// Fermi operator expansion on the pattern (lsw_foe.cu): shared arguments.
struct FoeLaunch {
    int n;                       // functions (rows)
    int64_t nnz;
    const int64_t* row_ptr;      // pattern CSR (symmetric, with the diagonal)
    const int32_t* col;
    const int64_t* tpos;         // position of the transposed entry of each entry
    const int64_t* diag;         // position of the diagonal entry of each row
    double* scratch;             // triple_ctas dense rows of n values, zero between uses
    int triple_ctas, cheb_ctas;
    int* status;
};
cudaError_t configure_foe_kernels(size_t max_smem);
cudaError_t foe_prep(const FoeLaunch& a, const double* H, const double* S, double sigma, double tau, double* Ht,
                     double* X, cudaStream_t s);
cudaError_t foe_triple(const FoeLaunch& a, const double* X, const double* A, double* Y, cudaStream_t s);
cudaError_t foe_cheb(const FoeLaunch& a, const double* Htp, const double* Tc, const double* Tp, double alpha, double* Tn,
                     cudaStream_t s);
cudaError_t foe_trace(const FoeLaunch& a, const double* T, double* out, cudaStream_t s);
cudaError_t foe_axpy_t(const FoeLaunch& a, double* K, const double* T, double c, cudaStream_t s);
cudaError_t foe_transpose(const FoeLaunch& a, const double* src, double* dst, cudaStream_t s);
cudaError_t foe_ebs(const FoeLaunch& a, const double* K, const double* Ht, const double* S, double sigma, double tau,
                    double* out, cudaStream_t s);

// Quartic confinement and preconditioning (lsw_confine.cu): one batch of functions
// f0 .. f0 + nfn - 1, each on its dense box E = L box widened by 14 (8 types).
struct ConfLaunch {
    int prec;
    int64_t f0;
    int nfn;
    const int32_t* sf_atom;
    const AtomRec* atoms;
    const Seg* seg;
    const int32_t* rowptr;
    const int64_t* off_L;
    const int64_t* off_Lp;
    const double* qtab;          // per atom: [dim][m = 2, 4][b b'][i over E][l + 14] of X_d^m
    const int64_t* qtab_off;     // first table entry of each atom (n_atoms + 1)
    const double* acoef;         // a_f, the confinement prefactor of each function
    const double* eps;           // eps_f of the preconditioning equation (NULL otherwise)
    double kin[4][KIN_TAPS];     // kinetic blocks hh, hg, gh, gg
    double kin_scale;            // -1 / (2 h^2)
    int64_t box_stride;          // elements of one function's box (8 types)
    int max_rows_L, max_rows_P;  // largest ny * nz of L and of L' boxes in the batch
    int64_t max_vol;             // largest E volume in the batch
    int* status;
    int64_t qtab_n, seg_n, rowptr_n, vec_n, dst_n;
    int n_sf, n_atoms;
};
cudaError_t conf_apply(const ConfLaunch& a, const void* vin, void* box_in, void* box_out, void* box_tmp, void* dst,
                       int region, int accumulate, bool precond, double* energy, cudaStream_t s);
cudaError_t conf_cg_init(const ConfLaunch& a, const void* g, void* x, void* r, void* p, cudaStream_t s);
cudaError_t conf_dot(const ConfLaunch& a, const void* x, const void* y, double* out, cudaStream_t s);
cudaError_t conf_cg_step1(const ConfLaunch& a, const double* rr, const double* pAp, const void* p, const void* Ap, void* x,
                          void* r, cudaStream_t s);
cudaError_t conf_cg_step2(const ConfLaunch& a, double* rr, const double* rr_new, const void* r, void* p, double* res,
                          cudaStream_t s);

// Fixed device scratch of the allocation-free Hamiltonian entry point (lsw_kernels.cu).
constexpr size_t NOALLOC_SCRATCH_BYTES = static_cast<size_t>(32) << 20;   // 32 MiB
constexpr int NOALLOC_MAX_DEVICES = 64;
constexpr int NOALLOC_MAX_BATCH = 64;      // functions per batch (records kept in the scratch)
cudaError_t noalloc_scratch(int device, void** ptr);
// Batch records of the allocation-free path, built on the device from the system's
// resident records all[f0 .. f0 + nb) with the batch's own workspace offsets.
cudaError_t enqueue_noalloc_records(const FnRec* all, int64_t f0, int nb, int64_t esize, FnRec* out, cudaStream_t s);

// Support-function reuse across geometries (lsw_reformat).
struct ReformatLaunch {
    const FnRec* fn;             // destination records (boxes, offsets); unused ws fields
    int nfn;
    int max_seg;                 // largest coarse+fine segment count of a destination L
    const AtomRec* atoms_dst;
    const AtomRec* atoms_src;
    const Seg* seg_dst;
    const Seg* seg_src;
    const int32_t* rowptr_src;
    const int32_t* shift;        // [n_atoms][3] grid shift of each atom (dst = src + shift)
    const int64_t* off_src;      // source function offsets
    const void* phi_src;
    void* phi_dst;
    int prec;
    int* status;
    int64_t seg_dst_n, seg_src_n, rowptr_src_n, src_n, dst_n;
};
cudaError_t enqueue_reformat(const ReformatLaunch& a, cudaStream_t s);

// Device entry points (lsw_kernels.cu).
cudaError_t upload_filters(const FilterSet& fs, int device);
cudaError_t measure_peaks(int n_sm, double* fp32_tflops, double* fp64_tflops, double* copy_gbs);
cudaError_t configure_kernels(size_t max_smem);
// Resident CTAs per SM of the FMA plane kernels at these dynamic shared-memory sizes.
cudaError_t plane_kernel_blocks(int prec, size_t smem_fwd, size_t smem_bwd, int* fwd, int* bwd);
cudaError_t enqueue_hphi_batch(const HphiLaunch& a, cudaStream_t s);
cudaError_t enqueue_pack(const PackLaunch& a, cudaStream_t s);     // panels of a slab (lsw_panels.cu)
cudaError_t enqueue_panel_hs(const PanelHSLaunch& a, cudaStream_t s);   // S, H from the panels
cudaError_t enqueue_panel_combine(const PanelHSLaunch& a, cudaStream_t s);   // M Phi panels
cudaError_t enqueue_lowdin_coeffs(const int64_t* row_ptr, const int32_t* col, const double* S, double* T, int n_sf,
                                  cudaStream_t s);
cudaError_t configure_panel_kernels(size_t max_smem);
size_t panel_hs_smem(int prec);
cudaError_t enqueue_dens_batch(const HphiLaunch& a, cudaStream_t s);   // real-space values
cudaError_t enqueue_density(const DensLaunch& a, cudaStream_t s);      // pair products

// Status word bits set by device-side checks.
enum : int {
    ST_BAD_BOX = 1,
    ST_BAD_SEG = 2,
    ST_BAD_PAIR = 4,
    ST_BAD_INDEX = 8,   // self-checking build: an index fell outside its buffer
    ST_WAIT_TIMEOUT = 16,   // a bounded wait for tensor-core completion ran out
};

// Layout of the device status block (int32 words): [0] status bits, [1] first bad
// kernel id, [2] source line, [3] block, [4..5] index (int64), [6..7] bound (int64).
constexpr int STATUS_WORDS = 8;

}  // namespace lsw
