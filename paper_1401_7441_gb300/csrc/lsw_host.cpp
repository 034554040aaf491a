// Host side of the C ABI (include/lsw.h): contexts, locreg geometry and segment keys,
// compressed layout, pair pattern, device plans, graph capture and the call surface.
//
// Paper: Sec. II.B (two-resolution grid; fine region = union of the atoms' small
// spheres; box with its origin at a corner), Sec. III Eq. loccon (locreg projector
// L: coefficients kept within R_cut of the centre), Sec. III.B (L' with R_cut + 8
// grid points; H phi = L' H L phi), Sec. II.A / Sec. IV.A (sparse H and S in
// compressed form on the locreg-overlap pattern), App. D (the "transposed" layout:
// partial matrices per region of the cell, here one H/S work item per grid tile).
//
// Membership tests are done in IEEE FP64 without contraction (this file is compiled
// with -ffp-contract=off): d2 = ((x-X)*(x-X) + (y-Y)*(y-Y)) + (z-Z)*(z-Z), x = i*h.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "lsw.h"
#include "lsw_internal.h"

using namespace lsw;

namespace {

thread_local std::string g_err;

lsw_status fail(lsw_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

lsw_status cuda_fail(cudaError_t e, const char* what) {
    return fail(LSW_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CUDA_TRY(expr)                                       \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, #expr);  \
    } while (0)

struct DeviceBuf {
    void* p = nullptr;
    size_t bytes = 0;
    ~DeviceBuf() {
        if (p) cudaFree(p);
    }
    cudaError_t alloc(size_t b) {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = b;
        if (b == 0) return cudaSuccess;
        const cudaError_t e = cudaMalloc(&p, b);
        if (e != cudaSuccess) {         // returned to the caller, not left pending for a later check
            p = nullptr;
            bytes = 0;
            (void)cudaGetLastError();
        }
        return e;
    }
    template <class T>
    cudaError_t upload(const std::vector<T>& v, cudaStream_t s) {
        cudaError_t e = alloc(v.size() * sizeof(T));
        if (e != cudaSuccess || v.empty()) return e;
        e = cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return e;
        return cudaStreamSynchronize(s);
    }
};

struct RegionHost {
    std::vector<int64_t> g;     // ascending
    std::vector<int64_t> keys;  // 3 per segment: first g, last g, offset
};

struct LocregHost {
    RegionHost c, f;
    int32_t lo[3] = {0, 0, 0}, n[3] = {0, 0, 0};
};

}  // namespace

namespace lsw {
struct EvPair {
    int kind;
    cudaEvent_t a, b;
};
struct Tracer {
    std::vector<EvPair> ev;    // pairs recorded (or captured) so far
    size_t used = 0;           // pairs in use for the current enqueue sequence
    bool capturing = false;
    bool pending = false;      // recorded work not read yet
    int cur = -1;
    ~Tracer() {
        for (auto& p : ev) {
            cudaEventDestroy(p.a);
            cudaEventDestroy(p.b);
        }
    }
};
void trace_begin(Tracer* tr, int kind, cudaStream_t s) {
    if (!tr) return;
    if (tr->used == tr->ev.size()) {
        EvPair p{kind, nullptr, nullptr};
        cudaEventCreate(&p.a);
        cudaEventCreate(&p.b);
        tr->ev.push_back(p);
    }
    EvPair& p = tr->ev[tr->used];
    p.kind = kind;
    tr->cur = static_cast<int>(tr->used);
    if (tr->capturing)
        cudaEventRecordWithFlags(p.a, s, cudaEventRecordExternal);
    else
        cudaEventRecord(p.a, s);
}
void trace_end(Tracer* tr, cudaStream_t s) {
    if (!tr || tr->cur < 0) return;
    EvPair& p = tr->ev[tr->cur];
    if (tr->capturing)
        cudaEventRecordWithFlags(p.b, s, cudaEventRecordExternal);
    else
        cudaEventRecord(p.b, s);
    tr->used++;
    tr->cur = -1;
    tr->pending = true;
}
}  // namespace lsw

struct lsw_ctx_s {
    int device = 0;
    bool host_only = false;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    FilterSet filters;
    size_t max_smem = 0;
    int n_sm = 0;
    std::atomic<int> live_systems{0};
};

struct GraphKey {
    const void* a;
    const void* b;
    const void* c;
    const void* d;
    bool operator<(const GraphKey& o) const {
        if (a != o.a) return a < o.a;
        if (b != o.b) return b < o.b;
        if (c != o.c) return c < o.c;
        return d < o.d;
    }
};

struct Batch {
    int64_t fn0, nfn;
    HphiLaunch proto;
};

constexpr int64_t PANEL_SLAB_MB = 8192;   // default panel budget of one H/S slab (option "slab_mb")

struct lsw_system_s {
    lsw_ctx ctx = nullptr;
    cudaStream_t stream = nullptr;   // where this system's work is enqueued (ctx's by default)
    int32_t N[3];
    double h;
    int prec;              // storage / arithmetic type: LSW_FP64 or LSW_FP32
    int zsplit = 0;        // LSW_FP32_BF16X: bfloat16 parts of the tensor-core z stage
    int xy_tc = 0;         // option "xy_tc": x, y passes on the tensor-core plane kernels
    size_t esize;
    int32_t n_atoms;
    std::vector<double> pos, r_loc, r_fine;
    std::vector<int32_t> nsf;
    double margin, cutoff;
    int pair_mode, fine_mode;
    std::vector<uint8_t> fine_mask;
    std::vector<LocregHost> L, Lp;
    std::vector<int32_t> sf_atom;
    std::vector<int64_t> off_L, off_Lp;
    std::vector<int64_t> row_ptr;
    std::vector<int32_t> col;
    // device state
    DeviceBuf d_atoms, d_seg, d_rowptr, d_fn, d_offL, d_offLp, d_sfatom, d_rowp, d_col;
    DeviceBuf d_plane_items, d_queue;   // plane items of the persistent kernels, their queue counters
    DeviceBuf d_colz;                   // L' column tables (ColZ) of every atom
    cudaStream_t copy_in = nullptr, copy_out = nullptr;   // lsw_step_host's copy streams
    DeviceBuf d_tile_fine, d_listA, d_listB, d_ws, d_status, d_escratch;
    // H/S in the transposed layout: used tiles, per-atom tile tables, product items, the
    // atoms of each slab and the panel buffers of one slab (reused slab after slab)
    DeviceBuf d_ptiles, d_patoms, d_ttab, d_items, d_citems, d_slab_atoms, d_PA, d_PQ, d_mcoef;
    // Fermi operator expansion: transposed positions, diagonal positions, the identity on
    // the pattern, work matrices and the dense row scratch of the triple products
    DeviceBuf d_tpos, d_diag, d_ident, d_foe, d_foe_scratch;
    // confinement and preconditioning: per-atom tables of the 1D operators X_d^2, X_d^4,
    // the batch boxes, and the conjugate-gradient vectors and scalars
    DeviceBuf d_qtab, d_qtab_off, d_cbox, d_cg, d_cgs;
    int conf_batch = 0;
    std::vector<PanelSlab> slabs;
    DeviceBuf d_shift, d_fn_all;   // reformat: per-atom shifts, records of every function
    // density: real-space store, block records, tile lists (built for one grid)
    DeviceBuf d_U, d_dfn, d_tptr, d_tfn;
    bool dens_ready = false;
    int64_t dens_lo[3] = {0, 0, 0}, dens_n[3] = {0, 0, 0};
    int32_t dens_ntile[3] = {0, 0, 0};
    int64_t U_elems = 0;
    std::vector<Batch> batches;
    int64_t ws_elems = 0;
    int batch_size = 0;
    int tile = 4;
    int64_t slab_mb = PANEL_SLAB_MB;
    size_t panel_bytes_A = 0, panel_bytes_Q = 0;   // panel buffers of the H/S plan (allocated on first use)
    int64_t hphi_limit = -1;         // option "hphi_limit" (-1: every function)
    int hs_tc = 1;                   // option "hs_tc": FP32 H/S products on the tensor cores
    int persistent = 1;              // option "persistent": bit 0 the backward, bit 1 the forward
                                     // FMA plane kernel over item queues
    int fwd_list = 1;                // option "fwd_list": forward x pass over member blocks only
    int use_graph = 1;
    // potential
    const void* V = nullptr;
    int64_t vlo[3] = {0, 0, 0}, vn[3] = {0, 0, 0};
    // graphs (each with the event pairs captured into it when tracing is on)
    struct GraphEntry {
        cudaGraphExec_t exec = nullptr;
        std::unique_ptr<Tracer> tr;
    };
    std::map<GraphKey, GraphEntry> graphs_h, graphs_m, graphs_d;
    int profiling = 0;
    std::unique_ptr<Tracer> direct_tr;   // tracer of work enqueued without a graph
    double prof_ms[TK_COUNT] = {0};
    int64_t prof_n[TK_COUNT] = {0};
    // host-API buffers
    DeviceBuf d_phi, d_hphi, d_H, d_S, d_ek, d_ep;
    cudaEvent_t done = nullptr;
};

namespace {

inline double d2_of(double x, double y, double z, const double* c) {
    double dx = x - c[0];
    double dy = y - c[1];
    double dz = z - c[2];
    double a = dx * dx;
    double b = dy * dy;
    double s = a + b;
    double e = dz * dz;
    return s + e;
}

void sphere_bounds(const int32_t* N, double h, const double* c, double R, int* lo, int* hi) {
    for (int d = 0; d < 3; ++d) {
        lo[d] = std::max(0, static_cast<int>(std::floor((c[d] - R) / h)) - 1);
        hi[d] = std::min(N[d] - 1, static_cast<int>(std::ceil((c[d] + R) / h)) + 1);
    }
}

void build_locreg(lsw_system_s* s, const std::vector<uint8_t>& fine, int a, double R,
                  LocregHost* out) {
    const int32_t* N = s->N;
    const double* c = &s->pos[3 * a];
    const double R2 = R * R;
    int lo[3], hi[3];
    sphere_bounds(N, s->h, c, R, lo, hi);
    double rf2 = s->r_fine[a] * s->r_fine[a];
    out->c.g.clear();
    out->f.g.clear();
    out->c.keys.clear();
    out->f.keys.clear();
    const double rg = R / s->h + 1.0;                  // sphere radius in grid steps, rounded up
    out->c.g.reserve(static_cast<size_t>(4.2 * rg * rg * rg) + 64);
    int bl[3] = {N[0], N[1], N[2]}, bh[3] = {-1, -1, -1};
    const double h = s->h;
    for (int k = lo[2]; k <= hi[2]; ++k) {
        double z = static_cast<double>(k) * h;
        for (int j = lo[1]; j <= hi[1]; ++j) {
            double y = static_cast<double>(j) * h;
            // The members of a row are one interval of i: d2 grows with |x - c_x| and every
            // operation of d2_of is correctly rounded, hence monotone.  The point nearest
            // c_x decides whether the row has members; the chord estimates the ends, and
            // the exact test moves each end to the true boundary.
            auto in = [&](int i) { return d2_of(static_cast<double>(i) * h, y, z, c) <= R2; };
            const int mc = static_cast<int>(std::floor(c[0] / h));
            int m = -1;                                // a member next to the minimum of d2, if any
            for (int t = mc - 1; t <= mc + 1 && m < 0; ++t) {
                const int tt = std::min(std::max(t, lo[0]), hi[0]);
                if (in(tt)) m = tt;
            }
            if (m < 0) continue;
            const double dy = y - c[1], dz = z - c[2];
            const double w = std::sqrt(std::max(0.0, R2 - (dy * dy + dz * dz)));
            int ia = std::min(m, std::max(lo[0], static_cast<int>(std::ceil((c[0] - w) / h))));
            int ib = std::max(m, std::min(hi[0], static_cast<int>(std::floor((c[0] + w) / h))));
            while (ia > lo[0] && in(ia - 1)) --ia;
            while (!in(ia)) ++ia;                      // stops at m at the latest
            while (ib < hi[0] && in(ib + 1)) ++ib;
            while (!in(ib)) --ib;
            const int64_t g0 = static_cast<int64_t>(N[0]) * (j + static_cast<int64_t>(N[1]) * k);
            // keys: (first g, last g, offset of the first) per run of consecutive members
            // within one x row; the coarse members of the row are one run, the fine ones
            // one run per stretch of the fine region
            out->c.keys.push_back(g0 + ia);
            out->c.keys.push_back(g0 + ib);
            out->c.keys.push_back(static_cast<int64_t>(out->c.g.size()));
            int64_t run = -1;                          // first g of the open fine run
            for (int i = ia; i <= ib; ++i) {
                const int64_t g = g0 + i;
                out->c.g.push_back(g);
                bool isf;
                if (s->fine_mode == LSW_FINE_UNION)
                    isf = fine[g] != 0;
                else
                    isf = d2_of(static_cast<double>(i) * h, y, z, c) <= rf2;
                if (isf) {
                    if (run < 0) {
                        run = g;
                        out->f.keys.push_back(g);
                        out->f.keys.push_back(g);
                        out->f.keys.push_back(static_cast<int64_t>(out->f.g.size()));
                    }
                    out->f.keys[out->f.keys.size() - 2] = g;
                    out->f.g.push_back(g);
                } else {
                    run = -1;
                }
            }
            bl[0] = std::min(bl[0], ia), bh[0] = std::max(bh[0], ib);
            bl[1] = std::min(bl[1], j), bh[1] = std::max(bh[1], j);
            bl[2] = std::min(bl[2], k), bh[2] = std::max(bh[2], k);
        }
    }
    for (int d = 0; d < 3; ++d) {
        out->lo[d] = out->c.g.empty() ? 0 : bl[d];
        out->n[d] = out->c.g.empty() ? 0 : bh[d] - bl[d] + 1;
    }
}

// box-local segments and per-row CSR of one region part
void emit_segments(const int32_t* N, const LocregHost& loc, const RegionHost& r,
                   std::vector<Seg>* seg, std::vector<int32_t>* rowptr, int64_t* seg0,
                   int32_t* nseg, int64_t* row0) {
    *seg0 = static_cast<int64_t>(seg->size());
    *row0 = static_cast<int64_t>(rowptr->size());
    const int nrows = loc.n[1] * loc.n[2];
    std::vector<int32_t> cnt(nrows + 1, 0);
    const size_t ns = r.keys.size() / 3;
    for (size_t q = 0; q < ns; ++q) {
        int64_t g0 = r.keys[3 * q], g1 = r.keys[3 * q + 1], off = r.keys[3 * q + 2];
        int64_t i1 = g0 % N[0], i2 = (g0 / N[0]) % N[1], i3 = g0 / (static_cast<int64_t>(N[0]) * N[1]);
        Seg sg;
        sg.x0 = static_cast<int32_t>(i1 - loc.lo[0]);
        sg.x1 = static_cast<int32_t>(sg.x0 + (g1 - g0));
        sg.row = static_cast<int32_t>((i2 - loc.lo[1]) + static_cast<int64_t>(loc.n[1]) * (i3 - loc.lo[2]));
        sg.off = static_cast<int32_t>(off);
        seg->push_back(sg);
        cnt[sg.row + 1]++;
    }
    for (int i = 0; i < nrows; ++i) cnt[i + 1] += cnt[i];
    for (int i = 0; i <= nrows; ++i) rowptr->push_back(cnt[i]);
    *nseg = static_cast<int32_t>(ns);
}

template <class F>
void parallel_for(int n, F fn) {
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    if (n < 64 || nt == 1) {
        for (int i = 0; i < n; ++i) fn(i);
        return;
    }
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([&, t]() {
            for (int i = static_cast<int>(t); i < n; i += static_cast<int>(nt)) fn(i);
        });
    for (auto& x : th) x.join();
}

lsw_status build_pattern(lsw_system_s* s) {
    const int na = s->n_atoms;
    double cmax = s->cutoff;
    if (s->pair_mode == LSW_PAIR_SUM_OF_RADII) {
        double rm = 0.0;
        for (double r : s->r_loc) rm = std::max(rm, r);
        cmax = 2.0 * rm;
    }
    double cell = std::max(cmax, 1e-3);
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int a = 0; a < na; ++a)
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], s->pos[3 * a + d]);
            hi[d] = std::max(hi[d], s->pos[3 * a + d]);
        }
    int nc[3];
    for (int d = 0; d < 3; ++d) nc[d] = std::max(1, std::min(1024, static_cast<int>((hi[d] - lo[d]) / cell) + 1));
    auto cidx = [&](int a, int d) {
        int c = static_cast<int>((s->pos[3 * a + d] - lo[d]) / cell);
        return std::min(nc[d] - 1, std::max(0, c));
    };
    std::vector<std::vector<int>> cells(static_cast<size_t>(nc[0]) * nc[1] * nc[2]);
    for (int a = 0; a < na; ++a)
        cells[(static_cast<size_t>(cidx(a, 2)) * nc[1] + cidx(a, 1)) * nc[0] + cidx(a, 0)].push_back(a);
    std::vector<std::vector<int>> nb(na);
    parallel_for(na, [&](int a) {
        int c0 = cidx(a, 0), c1 = cidx(a, 1), c2 = cidx(a, 2);
        const double* pa = &s->pos[3 * a];
        for (int z = std::max(0, c2 - 1); z <= std::min(nc[2] - 1, c2 + 1); ++z)
            for (int y = std::max(0, c1 - 1); y <= std::min(nc[1] - 1, c1 + 1); ++y)
                for (int x = std::max(0, c0 - 1); x <= std::min(nc[0] - 1, c0 + 1); ++x)
                    for (int b : cells[(static_cast<size_t>(z) * nc[1] + y) * nc[0] + x]) {
                        double c = s->pair_mode == LSW_PAIR_SUM_OF_RADII ? s->r_loc[b] + s->r_loc[a]
                                                                          : s->cutoff;
                        if (d2_of(s->pos[3 * b], s->pos[3 * b + 1], s->pos[3 * b + 2], pa) <= c * c)
                            nb[a].push_back(b);
                    }
        std::sort(nb[a].begin(), nb[a].end());
    });
    std::vector<int64_t> first(na + 1, 0);
    for (int a = 0; a < na; ++a) first[a + 1] = first[a] + s->nsf[a];
    const int64_t nf = first[na];
    s->row_ptr.assign(nf + 1, 0);
    for (int64_t f = 0; f < nf; ++f) {
        int a = s->sf_atom[f];
        int64_t cnt = 0;
        for (int b : nb[a]) cnt += s->nsf[b];
        s->row_ptr[f + 1] = s->row_ptr[f] + cnt;
    }
    s->col.resize(s->row_ptr[nf]);
    for (int64_t f = 0; f < nf; ++f) {
        int a = s->sf_atom[f];
        int64_t k = s->row_ptr[f];
        for (int b : nb[a])
            for (int64_t q = first[b]; q < first[b + 1]; ++q) s->col[k++] = static_cast<int32_t>(q);
    }
    return LSW_OK;
}

int64_t align64(int64_t x) { return (x + ALIGN_ELEMS - 1) / ALIGN_ELEMS * ALIGN_ELEMS; }

// smem bytes of the three pass kernels for a function record (bwd: with the z-arm plane
// and flag staging; bwd_plain: without)
void pass_smem(const FnRec& r, size_t es, int zcols, size_t* fwd, size_t* z, size_t* bwd, size_t* bwd_plain) {
    const int64_t X = 2 * r.n[0] + 29, Y = 2 * r.n[1] + 29, Z = 2 * r.n[2] + 29;
    const int64_t RS = r.n[0] | 1;
    *fwd = es * static_cast<size_t>(4 * r.n[1] * RS + 2 * r.n[1] * X);
    *z = es * static_cast<size_t>((2 * r.n[2] + Z) * zcols);
    const int64_t plA = std::max<int64_t>(Y * X, 4LL * r.np[1] * r.np[0]);
    const int64_t midA = std::max<int64_t>(2LL * r.np[1] * X, 4LL * r.np[1] * r.np[0]);
    *bwd = es * static_cast<size_t>(plA + midA + 4 * r.n[1] * RS) +
           static_cast<size_t>((4 * r.n[0] * r.n[1] + 15) / 16 * 16);   // + z-arm column flags
    *bwd_plain = es * static_cast<size_t>(plA + 2 * r.np[1] * X + 4 * r.n[1] * RS);
}

// Dynamic shared memory of the tensor-core z stage for a function record and `parts`
// bfloat16 parts (mirror of the layout in k_z_tc: 512-byte header, data operand parts
// 128 x max(K1, K2), filter operand parts N1 x K1 and N2 x K2, V tile Z x 128 FP32).
size_t ztc_smem(const FnRec& r, int parts) {
    auto up16 = [](int64_t v) { return (v + 15) / 16 * 16; };
    const int64_t Z = 2 * r.n[2] + 29;
    const int64_t K1 = up16(2 * r.n[2]), N1 = up16(Z), K2 = N1, N2 = up16(2 * r.np[2]);
    const int64_t KA = std::max(K1, K2);
    return static_cast<size_t>(512 + parts * (128 * KA * 2 + N1 * K1 * 2 + N2 * K2 * 2) + Z * 128 * 4);
}
// Dynamic shared memory of the tensor-core backward plane kernel (mirror of k_bwd_xy's
// tensor-core layout: 512-byte header, Fy parts 128 x K1, Fx parts N2 x K2, one region
// for the P operand / M1 operand / Gs, the D plane).
size_t bwd_tc_smem(const FnRec& r, int parts) {
    auto up16 = [](int64_t v) { return (v + 15) / 16 * 16; };
    const int64_t X = 2 * r.n[0] + 29, Y = 2 * r.n[1] + 29;
    const int64_t K1 = up16(Y), N1 = up16(X), K2 = N1, N2 = up16(2 * r.np[0]);
    const int64_t XR = up16(std::max<int64_t>(std::max<int64_t>(parts * N1 * K1 * 2, parts * 128 * K2 * 2), 16LL * r.np[1] * r.np[0]));
    const int64_t RS = r.n[0] | 1;
    return static_cast<size_t>(512 + parts * 128 * K1 * 2 + parts * N2 * K2 * 2 + XR + 4 * r.n[1] * RS * 4 +
                               (4 * r.n[0] * r.n[1] + 15) / 16 * 16);
}
// Dynamic shared memory of the tensor-core forward plane kernel (mirror of k_fwd_xy_tc:
// 512-byte header, Fy parts 128 x K1, Fx parts N2 x K2, one region for the D-plane
// operand and then the M1 operand).
size_t fwd_tc_smem(const FnRec& r, int parts) {
    auto up16 = [](int64_t v) { return (v + 15) / 16 * 16; };
    const int64_t X = 2 * r.n[0] + 29;
    const int64_t K1 = up16(2 * r.n[1]), N1 = up16(2 * r.n[0]), K2 = N1, N2 = up16(X);
    return static_cast<size_t>(512 + parts * 128 * K1 * 2 + parts * N2 * K2 * 2 +
                               parts * std::max<int64_t>(N1 * K1 * 2, 128 * K2 * 2));
}
// Largest extents the tensor-core kernels take: z stage (register window of half of
// K1 <= 64, MMA N <= 256); plane kernels (MMA M = 128 rows: 2 n_y' and Y <= 128, N <= 128).
bool ztc_fits(const FnRec& r) { return r.n[2] <= 64 && 2 * r.np[2] <= 256; }
bool xytc_fits(const FnRec& r) {
    return 2 * r.n[0] + 29 <= 128 && 2 * r.n[1] + 29 <= 128 && 2 * r.np[1] <= 128 && 2 * r.np[0] <= 128;
}

lsw_status build_plans(lsw_system_s* s) {
    const int64_t nf = static_cast<int64_t>(s->sf_atom.size());
    const int zcols = s->prec == LSW_FP64 ? ZCOLS_F64 : ZCOLS_F32;
    std::vector<FnRec> recs(nf);
    for (int64_t f = 0; f < nf; ++f) {
        FnRec& r = recs[f];
        int a = s->sf_atom[f];
        r.f = static_cast<int32_t>(f);
        r.atom = a;
        for (int d = 0; d < 3; ++d) {
            r.lo[d] = s->L[a].lo[d];
            r.n[d] = s->L[a].n[d];
            r.lop[d] = s->Lp[a].lo[d];
            r.np[d] = s->Lp[a].n[d];
        }
        r.off_phi = s->off_L[f];
        r.off_hphi = s->off_Lp[f];
    }
    s->batches.clear();
    int64_t ws_max = 0;
    std::vector<int32_t> items;          // plane items of every batch
    std::vector<int64_t> item_off;       // per batch: first item, -1 without items
    // option "hphi_limit": H phi only for functions 0 .. limit - 1 (a rank of a sharded
    // run computes its own functions, which its sub-system numbers first)
    const int64_t nf_h = s->hphi_limit >= 0 ? std::min<int64_t>(nf, s->hphi_limit) : nf;
    for (int64_t f0 = 0; f0 < nf_h; f0 += s->batch_size) {
        Batch b;
        b.fn0 = f0;
        b.nfn = std::min<int64_t>(s->batch_size, nf_h - f0);
        HphiLaunch& p = b.proto;
        std::memset(&p, 0, sizeof(p));
        p.prec = s->prec;
        p.nfn = static_cast<int>(b.nfn);
        p.zcols = zcols;
        p.fwd_list = s->fwd_list;
        size_t smem_bwd_plain = 0;
        int64_t o = 0;
        for (int64_t f = f0; f < f0 + b.nfn; ++f) {
            recs[f].ws_D = o;
            o += align64(8LL * recs[f].n[0] * recs[f].n[1] * recs[f].n[2]);
        }
        p.ws_D_elems = o;
        for (int64_t f = f0; f < f0 + b.nfn; ++f) {
            const FnRec& r = recs[f];
            const int64_t X = 2 * r.n[0] + 29, Y = 2 * r.n[1] + 29;
            recs[f].ws_Bf = o;
            o += align64(2LL * r.n[2] * Y * X);
            recs[f].ws_Bb = o;
            o += align64(2LL * r.np[2] * Y * X);
            recs[f].ws_G = o;
            o += align64(8LL * r.np[0] * r.np[1] * r.np[2]);
            recs[f].ws_Gf = o;
            o += align64((4LL * r.n[0] * r.n[1] + static_cast<int64_t>(s->esize) - 1) / static_cast<int64_t>(s->esize));
        }
        ws_max = std::max(ws_max, o);
        for (int64_t f = f0; f < f0 + b.nfn; ++f) {
            const FnRec& r = recs[f];
            const LocregHost& Lh = s->L[r.atom];
            const LocregHost& Ph = s->Lp[r.atom];
            p.max_nz = std::max(p.max_nz, r.n[2]);
            p.max_nzp = std::max(p.max_nzp, r.np[2]);
            p.max_cols = std::max<int>(p.max_cols, (2 * r.n[1] + 29) * (2 * r.n[0] + 29));
            p.max_rowsP = std::max(p.max_rowsP, r.np[1] * r.np[2]);
            p.max_ptsP = std::max<int64_t>(p.max_ptsP, static_cast<int64_t>(r.np[0]) * r.np[1] * r.np[2]);
            p.max_colsP = std::max(p.max_colsP, r.np[0] * r.np[1]);
            p.max_colsL = std::max(p.max_colsL, r.n[0] * r.n[1]);
            p.max_rowsL = std::max(p.max_rowsL, r.n[1] * r.n[2]);
            p.max_segL = std::max<int>(p.max_segL, static_cast<int>((Lh.c.keys.size() + Lh.f.keys.size()) / 3));
            p.max_segP = std::max<int>(p.max_segP, static_cast<int>((Ph.c.keys.size() + Ph.f.keys.size()) / 3));
            size_t a1, a2, a3, a4;
            pass_smem(r, s->esize, zcols, &a1, &a2, &a3, &a4);
            p.smem_fwd = std::max(p.smem_fwd, a1);
            p.smem_z = std::max(p.smem_z, a2);
            p.smem_kin = std::max(p.smem_kin, static_cast<size_t>(2 * r.n[2] * 128) * (p.prec == 0 ? 8 : 4));
            p.smem_bwd = std::max(p.smem_bwd, a3);
            smem_bwd_plain = std::max(smem_bwd_plain, a4);
            if (s->zsplit) {
                if (!ztc_fits(r))
                    return fail(LSW_ERR_UNSUPPORTED, "locreg extents too large for the tensor-core kernels");
                p.smem_ztc = std::max(p.smem_ztc, ztc_smem(r, s->zsplit));
                if (s->xy_tc) {
                    if (!xytc_fits(r))
                        return fail(LSW_ERR_UNSUPPORTED, "locreg extents too large for the tensor-core plane kernels");
                    p.smem_bwd_tc = std::max(p.smem_bwd_tc, bwd_tc_smem(r, s->zsplit));
                    p.smem_fwd_tc = std::max(p.smem_fwd_tc, fwd_tc_smem(r, s->zsplit));
                }
            }
        }
        // stage the z-arm plane and flags when they fit beside the plane kernel's tiles
        p.gstage = p.smem_bwd + BWD_STATIC_SMEM <= s->ctx->max_smem ? 1 : 0;
        if (!p.gstage) p.smem_bwd = smem_bwd_plain;
        p.zsplit = s->zsplit;
        p.xy_tc = s->zsplit ? s->xy_tc : 0;
        if (p.smem_fwd + FWD_STATIC_SMEM > s->ctx->max_smem || p.smem_z > s->ctx->max_smem || p.smem_bwd + BWD_STATIC_SMEM > s->ctx->max_smem ||
            p.smem_ztc > s->ctx->max_smem || p.smem_kin > s->ctx->max_smem || p.smem_bwd_tc + BWD_TC_STATIC_SMEM > s->ctx->max_smem ||
            p.smem_fwd_tc > s->ctx->max_smem)
            return fail(LSW_ERR_UNSUPPORTED, "locreg box too large for the on-chip pass tiles (%zu/%zu/%zu/%zu > %zu bytes)",
                        p.smem_fwd, p.smem_z, p.smem_bwd, p.smem_ztc, s->ctx->max_smem);
        // persistent FMA plane kernels: the batch's (function, plane, z type) items, largest
        // planes first (stable in function and plane order), and as many CTAs as fit
        if (s->persistent && !(p.zsplit && p.xy_tc) && p.max_nzp < 1024 && p.max_nz < 1024) {
            auto add = [&](int which) {
                std::vector<std::pair<int64_t, int32_t>> it;
                for (int64_t f = f0; f < f0 + b.nfn; ++f) {
                    const FnRec& r = recs[f];
                    const int64_t X = 2 * r.n[0] + 29, Y = 2 * r.n[1] + 29;
                    const int planes = which == 0 ? r.n[2] : r.np[2];
                    const int64_t cost = which == 0 ? X * Y : X * Y + static_cast<int64_t>(r.np[0]) * r.np[1];
                    for (int z = 0; z < planes; ++z)
                        for (int bz = 0; bz < 2; ++bz)
                            it.emplace_back(-cost, static_cast<int32_t>(((f - f0) << 11) | (z << 1) | bz));
                }
                std::stable_sort(it.begin(), it.end(),
                                 [](const auto& u, const auto& v) { return u.first < v.first; });
                for (const auto& q : it) items.push_back(q.second);
                return static_cast<int>(it.size());
            };
            int bf = 0, bb = 0;
            CUDA_TRY(plane_kernel_blocks(p.prec, p.smem_fwd, p.smem_bwd, &bf, &bb));
            item_off.push_back(static_cast<int64_t>(items.size()));
            p.n_items_fwd = (s->persistent & 2) ? add(0) : 0;
            p.n_items_bwd = (s->persistent & 1) ? add(1) : 0;
            p.grid_fwd = std::max(1, std::min(p.n_items_fwd, std::max(1, bf) * s->ctx->n_sm));
            p.grid_bwd = std::max(1, std::min(p.n_items_bwd, std::max(1, bb) * s->ctx->n_sm));
        } else {
            item_off.push_back(-1);
        }
        s->batches.push_back(b);
    }
    s->ws_elems = ws_max;
    cudaStream_t st = s->stream;
    CUDA_TRY(s->d_fn.upload(recs, st));
    for (auto& b : s->batches) b.proto.fn = static_cast<const FnRec*>(s->d_fn.p) + b.fn0;
    if (!items.empty()) {
        CUDA_TRY(s->d_plane_items.upload(items, st));
        if (!s->d_queue.p) CUDA_TRY(s->d_queue.alloc(4 * sizeof(int)));
    }
    for (size_t i = 0; i < s->batches.size(); ++i) {
        HphiLaunch& p = s->batches[i].proto;
        if (item_off[i] < 0) continue;
        const int32_t* it = static_cast<const int32_t*>(s->d_plane_items.p) + item_off[i];
        p.items_fwd = p.n_items_fwd ? it : nullptr;
        p.items_bwd = p.n_items_bwd ? it + p.n_items_fwd : nullptr;
        p.queue = static_cast<int*>(s->d_queue.p);
    }
    CUDA_TRY(s->d_ws.alloc(static_cast<size_t>(ws_max) * s->esize));
    return LSW_OK;
}

// Plan of the H/S build in the transposed layout (App. D): tiles of T^3 coarse points;
// per tile the functions whose L (A list) and L' (B list) touch it, atom by atom in
// atom order (so an atom's functions sit in consecutive slots); the panel row length
// T^3 + 7 (fine points of the tile), rounded up to 4; per atom, the tile boxes of L and
// L' with the used-tile index and slot of each tile; product items of at most 64 A rows
// by 128 columns of [A; B]; slabs of consecutive tile-z layers whose panels fit
// the slab budget (option "slab_mb"; one layer at least), with the atoms whose L' meets
// each slab.

lsw_status build_hs_plan(lsw_system_s* s) {
    const int T = s->tile;
    const int32_t* N = s->N;
    const int nt[3] = {(N[0] + T - 1) / T, (N[1] + T - 1) / T, (N[2] + T - 1) / T};
    const int64_t ntiles = static_cast<int64_t>(nt[0]) * nt[1] * nt[2];
    const int na = s->n_atoms;
    auto tiles_of = [&](const RegionHost& r, std::vector<int64_t>* out) {
        out->clear();
        for (size_t q = 0; q < r.keys.size() / 3; ++q) {
            int64_t g0 = r.keys[3 * q], g1 = r.keys[3 * q + 1];
            int64_t i1 = g0 % N[0], i2 = (g0 / N[0]) % N[1], i3 = g0 / (static_cast<int64_t>(N[0]) * N[1]);
            int64_t x1 = i1 + (g1 - g0);
            for (int64_t tx = i1 / T; tx <= x1 / T; ++tx)
                out->push_back(tx + nt[0] * ((i2 / T) + static_cast<int64_t>(nt[1]) * (i3 / T)));
        }
        std::sort(out->begin(), out->end());
        out->erase(std::unique(out->begin(), out->end()), out->end());
    };
    std::vector<std::vector<int64_t>> tA(na), tB(na);
    parallel_for(na, [&](int a) {
        tiles_of(s->L[a].c, &tA[a]);
        tiles_of(s->Lp[a].c, &tB[a]);
    });
    std::vector<int64_t> first(na + 1, 0);
    for (int a = 0; a < na; ++a) first[a + 1] = first[a] + s->nsf[a];
    // tile -> functions (atom by atom), and each (atom, tile)'s first slot
    auto invert = [&](const std::vector<std::vector<int64_t>>& t, std::vector<int64_t>* ptr, std::vector<int32_t>* fl,
                      std::vector<std::vector<int32_t>>* slot) {
        ptr->assign(ntiles + 1, 0);
        for (int a = 0; a < na; ++a)
            for (int64_t x : t[a]) (*ptr)[x + 1] += s->nsf[a];
        for (int64_t i = 0; i < ntiles; ++i) (*ptr)[i + 1] += (*ptr)[i];
        fl->resize((*ptr)[ntiles]);
        slot->assign(na, {});
        std::vector<int64_t> fill(ptr->begin(), ptr->end() - 1);
        for (int a = 0; a < na; ++a) {
            (*slot)[a].resize(t[a].size());
            for (size_t i = 0; i < t[a].size(); ++i) {
                const int64_t x = t[a][i];
                (*slot)[a][i] = static_cast<int32_t>(fill[x] - (*ptr)[x]);
                for (int64_t f = first[a]; f < first[a + 1]; ++f) (*fl)[fill[x]++] = static_cast<int32_t>(f);
            }
        }
    };
    std::vector<int64_t> pA, pB;
    std::vector<int32_t> fA, fB;
    std::vector<std::vector<int32_t>> slotA, slotB;
    invert(tA, &pA, &fA, &slotA);
    invert(tB, &pB, &fB, &slotB);
    // used tiles (L of some function touches them; then so does its L'), in tile order
    std::vector<int64_t> used_of(ntiles, -1);
    std::vector<PanelTile> tiles;
    std::vector<int32_t> fine;
    for (int64_t t = 0; t < ntiles; ++t) {
        if (pA[t + 1] == pA[t]) continue;
        PanelTile pt;
        std::memset(&pt, 0, sizeof(pt));
        const int tx = static_cast<int>(t % nt[0]);
        const int ty = static_cast<int>((t / nt[0]) % nt[1]);
        const int tz = static_cast<int>(t / (static_cast<int64_t>(nt[0]) * nt[1]));
        pt.org[0] = tx * T;
        pt.org[1] = ty * T;
        pt.org[2] = tz * T;
        pt.fine0 = static_cast<int32_t>(fine.size());
        for (int z = 0; z < T; ++z)
            for (int y = 0; y < T; ++y)
                for (int x = 0; x < T; ++x) {
                    int64_t gx = tx * T + x, gy = ty * T + y, gz = tz * T + z;
                    if (gx >= N[0] || gy >= N[1] || gz >= N[2]) continue;
                    int64_t g = gx + static_cast<int64_t>(N[0]) * (gy + static_cast<int64_t>(N[1]) * gz);
                    if (s->fine_mask[g]) fine.push_back(x | (y << 8) | (z << 16));
                }
        pt.nfine = static_cast<int32_t>(fine.size()) - pt.fine0;
        pt.nA = static_cast<int32_t>(pA[t + 1] - pA[t]);
        pt.nB = static_cast<int32_t>(pB[t + 1] - pB[t]);
        pt.kp = (T * T * T + 7 * pt.nfine + 3) / 4 * 4;
        pt.listA = pA[t];
        pt.listB = pB[t];
        used_of[t] = static_cast<int64_t>(tiles.size());
        tiles.push_back(pt);
    }
    if (tiles.size() > static_cast<size_t>(INT32_MAX)) return fail(LSW_ERR_UNSUPPORTED, "too many H/S tiles");
    // per-atom tile tables over the tile boxes of L and L'
    std::vector<PanelAtom> patoms(na);
    std::vector<int64_t> tab_off(na + 1, 0);
    for (int a = 0; a < na; ++a) {
        PanelAtom& q = patoms[a];
        std::memset(&q, 0, sizeof(q));
        int64_t nA = 1, nB = 1;
        for (int d = 0; d < 3; ++d) {
            q.tloA[d] = s->L[a].lo[d] / T;
            q.tnA[d] = (s->L[a].lo[d] + s->L[a].n[d] - 1) / T - q.tloA[d] + 1;
            q.tloB[d] = s->Lp[a].lo[d] / T;
            q.tnB[d] = (s->Lp[a].lo[d] + s->Lp[a].n[d] - 1) / T - q.tloB[d] + 1;
            nA *= q.tnA[d];
            nB *= q.tnB[d];
        }
        if (tA[a].empty()) nA = 0, q.tnA[0] = q.tnA[1] = q.tnA[2] = 0;   // no table: nothing to pack
        if (tB[a].empty()) nB = 0, q.tnB[0] = q.tnB[1] = q.tnB[2] = 0;
        q.f0 = static_cast<int32_t>(first[a]);
        q.nsf = s->nsf[a];
        tab_off[a + 1] = tab_off[a] + nA + nB;
    }
    std::vector<int2> ttab(tab_off[na], make_int2(-1, 0));
    parallel_for(na, [&](int a) {
        PanelAtom& q = patoms[a];
        q.tabA = tab_off[a];
        q.tabB = tab_off[a] + static_cast<int64_t>(q.tnA[0]) * q.tnA[1] * q.tnA[2];
        auto put = [&](const std::vector<int64_t>& tl, const std::vector<int32_t>& sl, const int32_t* lo,
                       const int32_t* n, int64_t base) {
            for (size_t i = 0; i < tl.size(); ++i) {
                const int64_t t = tl[i];
                const int tx = static_cast<int>(t % nt[0]) - lo[0];
                const int ty = static_cast<int>((t / nt[0]) % nt[1]) - lo[1];
                const int tz = static_cast<int>(t / (static_cast<int64_t>(nt[0]) * nt[1])) - lo[2];
                ttab[base + tx + static_cast<int64_t>(n[0]) * (ty + static_cast<int64_t>(n[1]) * tz)] =
                    make_int2(static_cast<int32_t>(used_of[t]), sl[i]);
            }
        };
        put(tA[a], slotA[a], q.tloA, q.tnA, q.tabA);
        put(tB[a], slotB[a], q.tloB, q.tnB, q.tabB);
    });
    // slabs of tile-z layers and their panel offsets; product items
    s->slabs.clear();
    std::vector<PanelItem> items, citems;
    const size_t es = s->esize;
    size_t maxA = 0, maxQ = 0;
    {
        size_t u = 0;
        while (u < tiles.size()) {
            PanelSlab sl;
            std::memset(&sl, 0, sizeof(sl));
            sl.tz0 = tiles[u].org[2] / T;
            sl.u0 = static_cast<int64_t>(u);
            sl.i0 = static_cast<int64_t>(items.size());
            sl.ci0 = static_cast<int64_t>(citems.size());
            int64_t eA = 0, eQ = 0;
            int tz = sl.tz0;
            while (u < tiles.size()) {
                // take the whole next layer
                size_t v = u;
                int64_t lA = 0, lQ = 0;
                while (v < tiles.size() && tiles[v].org[2] / T == tz) {
                    lA += static_cast<int64_t>(tiles[v].nA) * tiles[v].kp;
                    lQ += static_cast<int64_t>(tiles[v].nB) * tiles[v].kp;
                    ++v;
                }
                if (u > static_cast<size_t>(sl.u0) &&
                    static_cast<size_t>(eA + lA + eQ + lQ) * es > static_cast<size_t>(s->slab_mb) << 20)
                    break;
                for (size_t w = u; w < v; ++w) {
                    PanelTile& pt = tiles[w];
                    pt.pA = eA;
                    pt.pQ = eQ;
                    eA += static_cast<int64_t>(pt.nA) * pt.kp;
                    eQ += static_cast<int64_t>(pt.nB) * pt.kp;
                    const int ncol = pt.nA + pt.nB;
                    for (int a0 = 0; a0 < pt.nA; a0 += 64)
                        for (int c0 = 0; c0 < ncol; c0 += 128) {
                            PanelItem it;
                            it.tile = static_cast<int32_t>(w);
                            it.a0 = a0;
                            it.na = std::min(64, pt.nA - a0);
                            it.c0 = c0;
                            it.nc = std::min(128, ncol - c0);
                            it.pad = 0;
                            items.push_back(it);
                        }
                    for (int a0 = 0; a0 < pt.nA; a0 += 64)
                        for (int c0 = 0; c0 < pt.kp; c0 += 128) {
                            PanelItem it;
                            it.tile = static_cast<int32_t>(w);
                            it.a0 = a0;
                            it.na = std::min(64, pt.nA - a0);
                            it.c0 = c0;
                            it.nc = std::min(128, pt.kp - c0);
                            it.pad = 0;
                            citems.push_back(it);
                        }
                }
                u = v;
                if (u < tiles.size()) tz = tiles[u].org[2] / T;
                else break;
            }
            sl.tz1 = u < tiles.size() ? tiles[u].org[2] / T : nt[2];
            sl.u1 = static_cast<int64_t>(u);
            sl.i1 = static_cast<int64_t>(items.size());
            sl.ci1 = static_cast<int64_t>(citems.size());
            sl.elemsA = eA;
            sl.elemsQ = eQ;
            maxA = std::max(maxA, static_cast<size_t>(eA));
            maxQ = std::max(maxQ, static_cast<size_t>(eQ));
            s->slabs.push_back(sl);
        }
    }
    // atoms of each slab (their L' tile box meets the slab's layers) and the pack kernel's
    // shared memory (the largest region tables of those atoms; 0 when they do not fit)
    std::vector<int32_t> slab_atoms;
    const size_t smem_cap = std::min<size_t>(s->ctx->max_smem, 100 * 1024);
    for (PanelSlab& sl : s->slabs) {
        sl.s0 = static_cast<int64_t>(slab_atoms.size());
        size_t need = 0;
        for (int a = 0; a < na; ++a) {
            if (tB[a].empty() || s->nsf[a] == 0) continue;   // no functions: no panel rows
            const PanelAtom& q = patoms[a];
            if (q.tloB[2] + q.tnB[2] <= sl.tz0 || q.tloB[2] >= sl.tz1) continue;
            slab_atoms.push_back(a);
            for (int side = 0; side < 2; ++side) {
                const LocregHost& R = side ? s->Lp[a] : s->L[a];
                const size_t rows = static_cast<size_t>(R.n[1]) * R.n[2];
                const size_t segs = (R.c.keys.size() + R.f.keys.size()) / 3;
                need = std::max(need, (8 * (rows + 1) + 15) / 16 * 16 + sizeof(Seg) * segs);
            }
        }
        sl.s1 = static_cast<int64_t>(slab_atoms.size());
        sl.smem_pack = need <= smem_cap ? need : 0;
    }
    cudaStream_t st = s->stream;
    CUDA_TRY(s->d_ptiles.upload(tiles, st));
    CUDA_TRY(s->d_patoms.upload(patoms, st));
    CUDA_TRY(s->d_ttab.upload(ttab, st));
    CUDA_TRY(s->d_items.upload(items, st));
    CUDA_TRY(s->d_citems.upload(citems, st));
    CUDA_TRY(s->d_slab_atoms.upload(slab_atoms, st));
    CUDA_TRY(s->d_tile_fine.upload(fine, st));
    CUDA_TRY(s->d_listA.upload(fA, st));
    CUDA_TRY(s->d_listB.upload(fB, st));
    // the panel buffers of one slab are allocated by the first call that uses them
    // (ensure_panels), so a system that is created but not yet run holds none;
    // lsw_workspace_bytes counts them either way
    CUDA_TRY(s->d_PA.alloc(0));
    CUDA_TRY(s->d_PQ.alloc(0));
    s->panel_bytes_A = std::max<size_t>(maxA, 4) * es;
    s->panel_bytes_Q = std::max<size_t>(maxQ, 4) * es;
    return LSW_OK;
}

lsw_status ensure_panels(lsw_system_s* s) {
    if (!s->d_PA.p) CUDA_TRY(s->d_PA.alloc(s->panel_bytes_A));
    if (!s->d_PQ.p) CUDA_TRY(s->d_PQ.alloc(s->panel_bytes_Q));
    return LSW_OK;
}

lsw_status upload_geometry(lsw_system_s* s) {
    std::vector<AtomRec> recs(s->n_atoms);
    std::vector<Seg> seg;
    std::vector<int32_t> rowptr;
    for (int a = 0; a < s->n_atoms; ++a) {
        AtomRec& r = recs[a];
        const LocregHost& L = s->L[a];
        const LocregHost& P = s->Lp[a];
        for (int d = 0; d < 3; ++d) {
            r.lo[d] = L.lo[d];
            r.n[d] = L.n[d];
            r.lop[d] = P.lo[d];
            r.np[d] = P.n[d];
        }
        r.ncL = static_cast<int32_t>(L.c.g.size());
        r.nfL = static_cast<int32_t>(L.f.g.size());
        r.ncP = static_cast<int32_t>(P.c.g.size());
        r.nfP = static_cast<int32_t>(P.f.g.size());
        emit_segments(s->N, L, L.c, &seg, &rowptr, &r.segLc, &r.nsegLc, &r.rowLc);
        emit_segments(s->N, L, L.f, &seg, &rowptr, &r.segLf, &r.nsegLf, &r.rowLf);
        emit_segments(s->N, P, P.c, &seg, &rowptr, &r.segPc, &r.nsegPc, &r.rowPc);
        emit_segments(s->N, P, P.f, &seg, &rowptr, &r.segPf, &r.nsegPf, &r.rowPf);
    }
    // L' column tables: per (x, y) column the z range of the coarse members and the z hull
    // of the fine members (the planes the compressed H phi reads there)
    int64_t ncz = 0;
    for (int a = 0; a < s->n_atoms; ++a) {
        recs[a].colz = ncz;
        ncz += static_cast<int64_t>(s->Lp[a].n[0]) * s->Lp[a].n[1];
    }
    std::vector<ColZ> colz(static_cast<size_t>(ncz), ColZ{-1, -1, -1, -1});
    parallel_for(s->n_atoms, [&](int a) {
        const LocregHost& P = s->Lp[a];
        ColZ* t = colz.data() + recs[a].colz;
        const int64_t N0 = s->N[0], N01 = static_cast<int64_t>(s->N[0]) * s->N[1];
        auto fold = [&](const RegionHost& r, bool fine) {       // one segment (x run of a row) at a time
            for (size_t q = 0; q < r.keys.size() / 3; ++q) {
                const int64_t g0 = r.keys[3 * q], g1 = r.keys[3 * q + 1];
                const int x0 = static_cast<int>(g0 % N0 - P.lo[0]);
                const int y = static_cast<int>((g0 / N0) % s->N[1] - P.lo[1]);
                const int16_t z = static_cast<int16_t>(g0 / N01 - P.lo[2]);
                ColZ* row = t + static_cast<int64_t>(y) * P.n[0];
                for (int x = x0; x <= x0 + static_cast<int>(g1 - g0); ++x) {
                    int16_t& lo = fine ? row[x].f0 : row[x].c0;
                    int16_t& hi = fine ? row[x].f1 : row[x].c1;
                    if (lo < 0 || z < lo) lo = z;
                    if (z > hi) hi = z;
                }
            }
        };
        fold(P.c, false);
        fold(P.f, true);
    });
    cudaStream_t st = s->stream;
    CUDA_TRY(s->d_colz.upload(colz, st));
    CUDA_TRY(s->d_atoms.upload(recs, st));
    CUDA_TRY(s->d_seg.upload(seg, st));
    CUDA_TRY(s->d_rowptr.upload(rowptr, st));
    CUDA_TRY(s->d_offL.upload(s->off_L, st));
    CUDA_TRY(s->d_offLp.upload(s->off_Lp, st));
    CUDA_TRY(s->d_sfatom.upload(s->sf_atom, st));
    CUDA_TRY(s->d_rowp.upload(s->row_ptr, st));
    CUDA_TRY(s->d_col.upload(s->col, st));
    return LSW_OK;
}

void drop_graphs(lsw_system_s* s) {
    for (auto& kv : s->graphs_h) cudaGraphExecDestroy(kv.second.exec);
    for (auto& kv : s->graphs_m) cudaGraphExecDestroy(kv.second.exec);
    for (auto& kv : s->graphs_d) cudaGraphExecDestroy(kv.second.exec);
    s->graphs_h.clear();
    s->graphs_m.clear();
    s->graphs_d.clear();
}

// fold the elapsed times of a tracer's recorded pairs into the system's totals
void harvest(lsw_system_s* s, Tracer* tr) {
    if (!tr || !tr->pending) return;
    for (size_t i = 0; i < tr->used; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, tr->ev[i].a, tr->ev[i].b) == cudaSuccess) {
            s->prof_ms[tr->ev[i].kind] += ms;
            s->prof_n[tr->ev[i].kind] += 1;
        }
    }
    tr->pending = false;
}

struct NoHook {
    cudaError_t operator()(size_t) const { return cudaSuccess; }
};

// The batches of H phi on the system's stream; before(i) and after(i) enqueue what batch
// i waits for and what waits for it (the host-buffer step's copies).
template <class Before, class After>
lsw_status enqueue_apply_hooked(lsw_system_s* s, Tracer* tr, const void* phi, void* hphi, double* ek, double* ep,
                                Before before, After after) {
    cudaStream_t st = s->stream;
    int64_t nf = static_cast<int64_t>(s->sf_atom.size());
    if (s->hphi_limit >= 0) nf = std::min<int64_t>(nf, s->hphi_limit);
    CUDA_TRY(cudaMemsetAsync(ek, 0, nf * sizeof(double), st));
    CUDA_TRY(cudaMemsetAsync(ep, 0, nf * sizeof(double), st));
    for (size_t bi = 0; bi < s->batches.size(); ++bi) {
        const Batch& b = s->batches[bi];
        CUDA_TRY(before(bi));
        HphiLaunch p = b.proto;
        p.tr = tr;
        p.atoms = static_cast<const AtomRec*>(s->d_atoms.p);
        p.seg = static_cast<const Seg*>(s->d_seg.p);
        p.rowptr = static_cast<const int32_t*>(s->d_rowptr.p);
        p.colz = static_cast<const ColZ*>(s->d_colz.p);
        p.colz_n = static_cast<int64_t>(s->d_colz.bytes / sizeof(ColZ));
        p.phi = phi;
        p.hphi = hphi;
        p.e_kin = ek;
        p.e_pot = ep;
        p.V = s->V;
        for (int d = 0; d < 3; ++d) {
            p.vlo[d] = s->vlo[d];
            p.vn[d] = s->vn[d];
        }
        p.ws = s->d_ws.p;
        p.kin_scale = -1.0 / (2.0 * s->h * s->h);
        p.status = static_cast<int*>(s->d_status.p);
        p.phi_n = s->off_L.back();
        p.hphi_n = s->off_Lp.back();
        p.v_n = s->vn[0] * s->vn[1] * s->vn[2];
        p.ws_n = s->ws_elems;
        p.seg_n = static_cast<int64_t>(s->d_seg.bytes / sizeof(Seg));
        p.rowptr_n = static_cast<int64_t>(s->d_rowptr.bytes / sizeof(int32_t));
        p.n_atoms = s->n_atoms;
        if (p.queue) CUDA_TRY(cudaMemsetAsync(p.queue, 0, 2 * sizeof(int), st));
        CUDA_TRY(enqueue_hphi_batch(p, st));
        CUDA_TRY(after(bi));
    }
    return LSW_OK;
}

lsw_status enqueue_apply(lsw_system_s* s, Tracer* tr, const void* phi, void* hphi, double* ek, double* ep) {
    return enqueue_apply_hooked(s, tr, phi, hphi, ek, ep, NoHook{}, NoHook{});
}

PackLaunch pack_launch(lsw_system_s* s, Tracer* tr, const PanelSlab& sl, const void* phi, const void* hphi, void* out) {
    PackLaunch k;
    std::memset(&k, 0, sizeof(k));
    k.tr = tr;
    k.prec = s->prec;
    k.tiles = static_cast<const PanelTile*>(s->d_ptiles.p);
    k.patoms = static_cast<const PanelAtom*>(s->d_patoms.p);
    k.ttab = static_cast<const int2*>(s->d_ttab.p);
    k.slab_atoms = static_cast<const int32_t*>(s->d_slab_atoms.p) + sl.s0;
    k.n_slab_atoms = static_cast<int>(sl.s1 - sl.s0);
    k.tz0 = sl.tz0;
    k.tz1 = sl.tz1;
    k.tile = s->tile;
    k.u0 = sl.u0;
    k.tile_fine = static_cast<const int32_t*>(s->d_tile_fine.p);
    k.atoms = static_cast<const AtomRec*>(s->d_atoms.p);
    k.seg = static_cast<const Seg*>(s->d_seg.p);
    k.rowptr = static_cast<const int32_t*>(s->d_rowptr.p);
    k.off_L = static_cast<const int64_t*>(s->d_offL.p);
    k.off_Lp = static_cast<const int64_t*>(s->d_offLp.p);
    k.phi = phi;
    k.hphi = hphi;
    k.PA = s->d_PA.p;
    k.PQ = s->d_PQ.p;
    k.smem = sl.smem_pack;
    k.out = out;
    k.status = static_cast<int*>(s->d_status.p);
    k.phi_n = s->off_L.back();
    k.hphi_n = s->off_Lp.back();
    k.out_n = s->off_L.back();
    k.seg_n = static_cast<int64_t>(s->d_seg.bytes / sizeof(Seg));
    k.rowptr_n = static_cast<int64_t>(s->d_rowptr.bytes / sizeof(int32_t));
    k.fine_n = static_cast<int64_t>(s->d_tile_fine.bytes / sizeof(int32_t));
    k.ttab_n = static_cast<int64_t>(s->d_ttab.bytes / sizeof(int2));
    k.PA_n = static_cast<int64_t>(s->d_PA.bytes / s->esize);
    k.PQ_n = static_cast<int64_t>(s->d_PQ.bytes / s->esize);
    k.n_atoms = s->n_atoms;
    k.n_tiles = static_cast<int>(s->d_ptiles.bytes / sizeof(PanelTile));
    k.n_sf = static_cast<int>(s->sf_atom.size());
    return k;
}

PanelHSLaunch product_launch(lsw_system_s* s, Tracer* tr, const PanelSlab& sl, bool combine) {
    PanelHSLaunch p;
    std::memset(&p, 0, sizeof(p));
    p.tr = tr;
    p.prec = s->prec;
    p.tiles = static_cast<const PanelTile*>(s->d_ptiles.p);
    p.items = static_cast<const PanelItem*>(combine ? s->d_citems.p : s->d_items.p) + (combine ? sl.ci0 : sl.i0);
    p.nitems = combine ? sl.ci1 - sl.ci0 : sl.i1 - sl.i0;
    p.listA = static_cast<const int32_t*>(s->d_listA.p);
    p.listB = static_cast<const int32_t*>(s->d_listB.p);
    p.row_ptr = static_cast<const int64_t*>(s->d_rowp.p);
    p.col = static_cast<const int32_t*>(s->d_col.p);
    p.PA = s->d_PA.p;
    p.PQ = s->d_PQ.p;
    p.status = static_cast<int*>(s->d_status.p);
    p.listA_n = static_cast<int64_t>(s->d_listA.bytes / sizeof(int32_t));
    p.listB_n = static_cast<int64_t>(s->d_listB.bytes / sizeof(int32_t));
    p.nnz = static_cast<int64_t>(s->col.size());
    p.PA_n = static_cast<int64_t>(s->d_PA.bytes / s->esize);
    p.PQ_n = static_cast<int64_t>(s->d_PQ.bytes / s->esize);
    p.n_tiles = static_cast<int64_t>(s->d_ptiles.bytes / sizeof(PanelTile));
    p.n_sf = static_cast<int>(s->sf_atom.size());
    p.tc = (s->prec != LSW_FP64 && s->hs_tc && !combine) ? 1 : 0;
    return p;
}

lsw_status enqueue_matrices(lsw_system_s* s, Tracer* tr, const void* phi, const void* hphi, double* H, double* S) {
    cudaStream_t st = s->stream;
    const int64_t nnz = static_cast<int64_t>(s->col.size());
    CUDA_TRY(cudaMemsetAsync(H, 0, nnz * sizeof(double), st));
    CUDA_TRY(cudaMemsetAsync(S, 0, nnz * sizeof(double), st));
    for (const PanelSlab& sl : s->slabs) {
        CUDA_TRY(enqueue_pack(pack_launch(s, tr, sl, phi, hphi, nullptr), st));
        PanelHSLaunch p = product_launch(s, tr, sl, false);
        p.H = H;
        p.S = S;
        CUDA_TRY(enqueue_panel_hs(p, st));
    }
    return LSW_OK;
}

// (M Phi)_a = P_L(a) sum_b M_ab phi_b, slab by slab: pack phi on L, combine the panels,
// unpack onto the members of L.
lsw_status enqueue_combine(lsw_system_s* s, Tracer* tr, const double* M, const void* phi, void* out) {
    cudaStream_t st = s->stream;
    for (const PanelSlab& sl : s->slabs) {
        CUDA_TRY(enqueue_pack(pack_launch(s, tr, sl, phi, nullptr, nullptr), st));
        PanelHSLaunch p = product_launch(s, tr, sl, true);
        p.M = M;
        CUDA_TRY(enqueue_panel_combine(p, st));
        CUDA_TRY(enqueue_pack(pack_launch(s, tr, sl, nullptr, nullptr, out), st));
    }
    return LSW_OK;
}

// Density plan for the grid [lo, lo + dims): each function's real-space block (origin on
// the grid, extents, offset in the store) and, per tile of the grid, the functions whose
// blocks meet it (ascending).  Allocates the store.
lsw_status build_density_plan(lsw_system_s* s, const int64_t* lo, const int64_t* dims) {
    const int64_t nf = static_cast<int64_t>(s->sf_atom.size());
    std::vector<DensFn> dfn(nf);
    int64_t off = 0;
    for (int64_t f = 0; f < nf; ++f) {
        const LocregHost& L = s->L[s->sf_atom[f]];
        DensFn& r = dfn[f];
        r.off = off;
        int64_t vol = 1;
        for (int d = 0; d < 3; ++d) {
            r.o[d] = static_cast<int32_t>(2LL * L.lo[d] - V_REACH - lo[d]);
            r.d[d] = 2 * L.n[d] + 29;
            vol *= r.d[d];
        }
        off += align64(vol);
    }
    const int tdim[3] = {DT_X, DT_Y, DT_Z};
    int32_t nt[3];
    for (int d = 0; d < 3; ++d) nt[d] = static_cast<int32_t>((dims[d] + tdim[d] - 1) / tdim[d]);
    const int64_t ntiles = static_cast<int64_t>(nt[0]) * nt[1] * nt[2];
    if (ntiles > (1LL << 31) - 1) return fail(LSW_ERR_UNSUPPORTED, "lsw_build_density: grid has too many tiles");
    std::vector<int64_t> tptr(ntiles + 1, 0);
    auto each_tile = [&](const DensFn& r, auto fn) {
        int32_t t0[3], t1[3];
        for (int d = 0; d < 3; ++d) {
            t0[d] = r.o[d] / tdim[d];
            t1[d] = (r.o[d] + r.d[d] - 1) / tdim[d];
        }
        for (int32_t z = t0[2]; z <= t1[2]; ++z)
            for (int32_t y = t0[1]; y <= t1[1]; ++y)
                for (int32_t x = t0[0]; x <= t1[0]; ++x) fn((static_cast<int64_t>(z) * nt[1] + y) * nt[0] + x);
    };
    for (int64_t f = 0; f < nf; ++f) each_tile(dfn[f], [&](int64_t t) { tptr[t + 1]++; });
    for (int64_t t = 0; t < ntiles; ++t) tptr[t + 1] += tptr[t];
    std::vector<int32_t> tfn(static_cast<size_t>(tptr[ntiles]));
    {
        std::vector<int64_t> fill(tptr.begin(), tptr.end() - 1);
        for (int64_t f = 0; f < nf; ++f)
            each_tile(dfn[f], [&](int64_t t) { tfn[fill[t]++] = static_cast<int32_t>(f); });
    }
    s->dens_ready = false;
    cudaStream_t st = s->stream;
    CUDA_TRY(s->d_dfn.upload(dfn, st));
    CUDA_TRY(s->d_tptr.upload(tptr, st));
    CUDA_TRY(s->d_tfn.upload(tfn, st));
    CUDA_TRY(s->d_U.alloc(static_cast<size_t>(off) * s->esize));
    s->U_elems = off;
    for (int d = 0; d < 3; ++d) {
        s->dens_lo[d] = lo[d];
        s->dens_n[d] = dims[d];
        s->dens_ntile[d] = nt[d];
    }
    s->dens_ready = true;
    return LSW_OK;
}

lsw_status enqueue_density_all(lsw_system_s* s, Tracer* tr, const void* phi, const double* K, double* rho) {
    cudaStream_t st = s->stream;
    for (const Batch& b : s->batches) {
        HphiLaunch p = b.proto;
        p.tr = tr;
        p.atoms = static_cast<const AtomRec*>(s->d_atoms.p);
        p.seg = static_cast<const Seg*>(s->d_seg.p);
        p.rowptr = static_cast<const int32_t*>(s->d_rowptr.p);
        p.phi = phi;
        p.ws = s->d_ws.p;
        p.status = static_cast<int*>(s->d_status.p);
        p.phi_n = s->off_L.back();
        p.ws_n = s->ws_elems;
        p.seg_n = static_cast<int64_t>(s->d_seg.bytes / sizeof(Seg));
        p.rowptr_n = static_cast<int64_t>(s->d_rowptr.bytes / sizeof(int32_t));
        p.n_atoms = s->n_atoms;
        p.U = s->d_U.p;
        p.dfn = static_cast<const DensFn*>(s->d_dfn.p);
        p.U_n = s->U_elems;
        CUDA_TRY(enqueue_dens_batch(p, st));
    }
    DensLaunch d;
    std::memset(&d, 0, sizeof(d));
    d.tr = tr;
    d.prec = s->prec;
    d.fn = static_cast<const DensFn*>(s->d_dfn.p);
    d.U = s->d_U.p;
    d.tptr = static_cast<const int64_t*>(s->d_tptr.p);
    d.tfn = static_cast<const int32_t*>(s->d_tfn.p);
    d.row_ptr = static_cast<const int64_t*>(s->d_rowp.p);
    d.col = static_cast<const int32_t*>(s->d_col.p);
    d.K = K;
    d.rho = rho;
    for (int k = 0; k < 3; ++k) {
        d.gn[k] = s->dens_n[k];
        d.ntile[k] = s->dens_ntile[k];
    }
    d.status = static_cast<int*>(s->d_status.p);
    d.U_n = s->U_elems;
    d.tfn_n = static_cast<int64_t>(s->d_tfn.bytes / sizeof(int32_t));
    d.nnz = static_cast<int64_t>(s->col.size());
    d.rho_n = s->dens_n[0] * s->dens_n[1] * s->dens_n[2];
    d.fn_n = static_cast<int64_t>(s->sf_atom.size());
    d.tptr_n = static_cast<int64_t>(s->d_tptr.bytes / sizeof(int64_t));
    d.rowp_n = static_cast<int64_t>(s->row_ptr.size());
    CUDA_TRY(enqueue_density(d, st));
    return LSW_OK;
}

// Run `enq(tracer)` directly, or through a cached CUDA graph keyed by the buffer
// pointers; with profiling on, event pairs are recorded around every launch (captured
// as external event-record nodes inside graphs).
template <class Enq>
lsw_status run_maybe_graph(lsw_system_s* s, std::map<GraphKey, lsw_system_s::GraphEntry>* cache, GraphKey key,
                           Enq enq) {
    cudaStream_t st = s->stream;
    if (!s->use_graph || st == nullptr) {
        Tracer* tr = nullptr;
        if (s->profiling) {
            if (!s->direct_tr) s->direct_tr.reset(new Tracer());
            tr = s->direct_tr.get();
            if (!tr->pending) tr->used = 0;
        }
        return enq(tr);
    }
    auto it = cache->find(key);
    if (it == cache->end()) {
        lsw_system_s::GraphEntry ge;
        if (s->profiling) {
            ge.tr.reset(new Tracer());
            ge.tr->capturing = true;
        }
        cudaGraph_t g = nullptr;
        CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        lsw_status rs = enq(ge.tr.get());
        cudaError_t ce = cudaStreamEndCapture(st, &g);
        if (ge.tr) {
            ge.tr->capturing = false;
            ge.tr->pending = false;
        }
        if (rs != LSW_OK) {
            if (g) cudaGraphDestroy(g);
            return rs;
        }
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
        ce = cudaGraphInstantiate(&ge.exec, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate");
        it = cache->emplace(key, std::move(ge)).first;
    }
    if (it->second.tr) harvest(s, it->second.tr.get());  // a previous replay not read yet
    CUDA_TRY(cudaGraphLaunch(it->second.exec, st));
    if (it->second.tr) it->second.tr->pending = true;
    return LSW_OK;
}

// Workspace elements of one function (D box; Bf, Bb, G and the z-arm flags), as laid out
// by k_noalloc_records.
void noalloc_sizes(const lsw_system_s* s, const FnRec& r, int64_t* sD, int64_t* sR) {
    const int64_t X = 2 * r.n[0] + 29, Y = 2 * r.n[1] + 29;
    const int64_t es = static_cast<int64_t>(s->esize);
    *sD = align64(8LL * r.n[0] * r.n[1] * r.n[2]);
    *sR = align64(2LL * r.n[2] * Y * X) + align64(2LL * r.np[2] * Y * X) + align64(8LL * r.np[0] * r.np[1] * r.np[2]) +
          align64((4LL * r.n[0] * r.n[1] + es - 1) / es);
}
FnRec noalloc_record(const lsw_system_s* s, int64_t f) {
    FnRec r;
    std::memset(&r, 0, sizeof(r));
    const int a = s->sf_atom[f];
    r.f = static_cast<int32_t>(f);
    r.atom = a;
    for (int d = 0; d < 3; ++d) {
        r.lo[d] = s->L[a].lo[d];
        r.n[d] = s->L[a].n[d];
        r.lop[d] = s->Lp[a].lo[d];
        r.np[d] = s->Lp[a].n[d];
    }
    r.off_phi = s->off_L[f];
    r.off_hphi = s->off_Lp[f];
    return r;
}
// Fold one function into a batch's launch extents and shared-memory sizes.
void noalloc_fold(const lsw_system_s* s, const FnRec& r, int zcols, HphiLaunch* p, size_t* smem_bwd_plain) {
    const LocregHost& Lh = s->L[r.atom];
    const LocregHost& Ph = s->Lp[r.atom];
    p->max_nz = std::max(p->max_nz, r.n[2]);
    p->max_nzp = std::max(p->max_nzp, r.np[2]);
    p->max_cols = std::max<int>(p->max_cols, (2 * r.n[1] + 29) * (2 * r.n[0] + 29));
    p->max_rowsP = std::max(p->max_rowsP, r.np[1] * r.np[2]);
    p->max_ptsP = std::max<int64_t>(p->max_ptsP, static_cast<int64_t>(r.np[0]) * r.np[1] * r.np[2]);
    p->max_colsP = std::max(p->max_colsP, r.np[0] * r.np[1]);
    p->max_colsL = std::max(p->max_colsL, r.n[0] * r.n[1]);
    p->max_rowsL = std::max(p->max_rowsL, r.n[1] * r.n[2]);
    p->max_segL = std::max<int>(p->max_segL, static_cast<int>((Lh.c.keys.size() + Lh.f.keys.size()) / 3));
    p->max_segP = std::max<int>(p->max_segP, static_cast<int>((Ph.c.keys.size() + Ph.f.keys.size()) / 3));
    size_t a1, a2, a3, a4;
    pass_smem(r, s->esize, zcols, &a1, &a2, &a3, &a4);
    p->smem_fwd = std::max(p->smem_fwd, a1);
    p->smem_z = std::max(p->smem_z, a2);
    p->smem_kin = std::max(p->smem_kin, static_cast<size_t>(2 * r.n[2] * 128) * (p->prec == 0 ? 8 : 4));
    p->smem_bwd = std::max(p->smem_bwd, a3);
    *smem_bwd_plain = std::max(*smem_bwd_plain, a4);
    if (s->zsplit) {
        p->smem_ztc = std::max(p->smem_ztc, ztc_smem(r, s->zsplit));
        if (s->xy_tc) {
            p->smem_bwd_tc = std::max(p->smem_bwd_tc, bwd_tc_smem(r, s->zsplit));
            p->smem_fwd_tc = std::max(p->smem_fwd_tc, fwd_tc_smem(r, s->zsplit));
        }
    }
}
// Choose the plane kernel's staging and check the tiles against the shared memory.
bool noalloc_finish(const lsw_system_s* s, HphiLaunch* p, size_t smem_bwd_plain) {
    const size_t mx = s->ctx->max_smem;
    p->gstage = p->smem_bwd + BWD_STATIC_SMEM <= mx ? 1 : 0;
    if (!p->gstage) p->smem_bwd = smem_bwd_plain;
    return !(p->smem_fwd + FWD_STATIC_SMEM > mx || p->smem_z > mx || p->smem_bwd + BWD_STATIC_SMEM > mx || p->smem_ztc > mx ||
             p->smem_kin > mx || p->smem_bwd_tc + BWD_TC_STATIC_SMEM > mx || p->smem_fwd_tc > mx);
}
}  // namespace

// ============================================================================ C ABI

extern "C" {

const char* lsw_last_error(void) { return g_err.c_str(); }

lsw_status lsw_ctx_create(int device, void* stream, lsw_ctx* out) {
    g_err.clear();
    if (!out) return fail(LSW_ERR_ARG, "lsw_ctx_create: out is NULL");
    *out = nullptr;
    if (device == LSW_HOST_ONLY) {
        std::unique_ptr<lsw_ctx_s> c(new (std::nothrow) lsw_ctx_s());
        if (!c) return fail(LSW_ERR_OOM, "lsw_ctx_create: host allocation");
        c->host_only = true;
        c->device = LSW_HOST_ONLY;
        std::string err;
        if (!derive_filters(&c->filters, &err)) return fail(LSW_ERR_STATE, "filter derivation: %s", err.c_str());
        *out = c.release();
        return LSW_OK;
    }
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(LSW_ERR_ARG, "lsw_ctx_create: device %d of %d", device, ndev);
    CUDA_TRY(cudaSetDevice(device));
    std::unique_ptr<lsw_ctx_s> c(new (std::nothrow) lsw_ctx_s());
    if (!c) return fail(LSW_ERR_OOM, "lsw_ctx_create: host allocation");
    c->device = device;
    std::string err;
    if (!derive_filters(&c->filters, &err)) return fail(LSW_ERR_STATE, "filter derivation: %s", err.c_str());
    int smem = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    CUDA_TRY(cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device));
    c->max_smem = static_cast<size_t>(smem);
    c->stream = static_cast<cudaStream_t>(stream);  // NULL: the legacy default stream
    CUDA_TRY(upload_filters(c->filters, device));
    CUDA_TRY(configure_kernels(c->max_smem));
    CUDA_TRY(configure_panel_kernels(c->max_smem));
    CUDA_TRY(configure_foe_kernels(c->max_smem));
    *out = c.release();
    return LSW_OK;
}

lsw_status lsw_ctx_destroy(lsw_ctx ctx) {
    g_err.clear();
    if (!ctx) return LSW_OK;
    if (ctx->live_systems != 0) return fail(LSW_ERR_STATE, "lsw_ctx_destroy: %d systems alive", ctx->live_systems.load());
    if (!ctx->host_only && ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return LSW_OK;
}

lsw_status lsw_filter_table(lsw_ctx ctx, int32_t which, int32_t* first, int32_t* count, double* values) {
    g_err.clear();
    if (!ctx || !first || !count || !values) return fail(LSW_ERR_ARG, "lsw_filter_table: NULL argument");
    const FilterSet& f = ctx->filters;
    const double* src = nullptr;
    int lo = 0, n = 0;
    switch (which) {
        case LSW_FILTER_H: src = f.h, lo = H_LO, n = D16; break;
        case LSW_FILTER_G: src = f.g, lo = H_LO, n = D16; break;
        case LSW_FILTER_MOMENTS: src = f.moments, lo = 0, n = D16; break;
        case LSW_FILTER_MAGIC: src = f.magic, lo = H_LO, n = D16; break;
        case LSW_FILTER_KIN_R: src = f.kin_r, lo = -KIN_HALF, n = KIN_TAPS; break;
        case LSW_FILTER_KIN_HH: case LSW_FILTER_KIN_HG: case LSW_FILTER_KIN_GH: case LSW_FILTER_KIN_GG:
            src = f.kin[which - LSW_FILTER_KIN_HH], lo = -KIN_HALF, n = KIN_TAPS; break;
        case LSW_FILTER_FWD_H: case LSW_FILTER_FWD_G:
            src = f.fwd[which - LSW_FILTER_FWD_H], lo = FWD_LO, n = FWD_TAPS; break;
        case LSW_FILTER_MOVL_0: case LSW_FILTER_MOVL_1: case LSW_FILTER_MOVL_2: case LSW_FILTER_MOVL_3:
        case LSW_FILTER_MOVL_4:
            src = f.movl[which - LSW_FILTER_MOVL_0], lo = -KIN_HALF, n = KIN_TAPS; break;
        default: return fail(LSW_ERR_ARG, "lsw_filter_table: unknown table %d", which);
    }
    *first = lo;
    *count = n;
    std::memcpy(values, src, n * sizeof(double));
    return LSW_OK;
}

lsw_status lsw_system_create(lsw_ctx ctx, const lsw_system_desc* d, lsw_system* out) {
    g_err.clear();
    if (!ctx || !d || !out) return fail(LSW_ERR_ARG, "lsw_system_create: NULL argument");
    *out = nullptr;
    if (d->N[0] < 1 || d->N[1] < 1 || d->N[2] < 1 || d->N[0] > 4096 || d->N[1] > 4096 || d->N[2] > 4096)
        return fail(LSW_ERR_ARG, "lsw_system_create: grid %d x %d x %d out of range", d->N[0], d->N[1], d->N[2]);
    if (static_cast<double>(d->N[0]) * d->N[1] * d->N[2] > 2.0e9)
        return fail(LSW_ERR_ARG, "lsw_system_create: grid has more than 2e9 points");
    if (!(d->h > 0) || !std::isfinite(d->h)) return fail(LSW_ERR_ARG, "lsw_system_create: h must be > 0");
    if (d->n_atoms < 1 || !d->pos || !d->r_loc || !d->r_fine || !d->n_sf)
        return fail(LSW_ERR_ARG, "lsw_system_create: no atoms or NULL atom arrays");
    if (d->precision != LSW_FP64 && d->precision != LSW_FP32 && d->precision != LSW_FP32_BF16X)
        return fail(LSW_ERR_ARG, "lsw_system_create: precision %d", d->precision);
    if (d->fine_mode != LSW_FINE_UNION && d->fine_mode != LSW_FINE_OWN)
        return fail(LSW_ERR_ARG, "lsw_system_create: fine_mode %d", d->fine_mode);
    if (d->pair_mode != LSW_PAIR_CUTOFF && d->pair_mode != LSW_PAIR_SUM_OF_RADII)
        return fail(LSW_ERR_ARG, "lsw_system_create: pair_mode %d", d->pair_mode);
    if (!(d->lprime_margin >= 0) || !std::isfinite(d->lprime_margin))
        return fail(LSW_ERR_ARG, "lsw_system_create: lprime_margin must be >= 0");
    if (d->pair_mode == LSW_PAIR_CUTOFF && (!(d->pair_cutoff >= 0) || !std::isfinite(d->pair_cutoff)))
        return fail(LSW_ERR_ARG, "lsw_system_create: pair_cutoff must be >= 0");
    for (int a = 0; a < d->n_atoms; ++a) {
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(d->pos[3 * a + k])) return fail(LSW_ERR_ARG, "atom %d: position not finite", a);
        if (!(d->r_loc[a] > 0) || !std::isfinite(d->r_loc[a])) return fail(LSW_ERR_ARG, "atom %d: r_loc must be > 0", a);
        if (!(d->r_fine[a] >= 0) || !std::isfinite(d->r_fine[a])) return fail(LSW_ERR_ARG, "atom %d: r_fine must be >= 0", a);
        if (d->n_sf[a] < 0 || d->n_sf[a] > 64) return fail(LSW_ERR_ARG, "atom %d: n_sf %d", a, d->n_sf[a]);
    }
    if (!ctx->host_only) CUDA_TRY(cudaSetDevice(ctx->device));
    std::unique_ptr<lsw_system_s> s(new (std::nothrow) lsw_system_s());
    if (!s) return fail(LSW_ERR_OOM, "lsw_system_create: host allocation");
    s->ctx = ctx;
    s->stream = ctx->stream;
    for (int k = 0; k < 3; ++k) s->N[k] = d->N[k];
    s->h = d->h;
    s->prec = d->precision == LSW_FP64 ? LSW_FP64 : LSW_FP32;
    s->zsplit = d->precision == LSW_FP32_BF16X ? 2 : 0;
    s->esize = s->prec == LSW_FP64 ? 8 : 4;
    s->n_atoms = d->n_atoms;
    s->pos.assign(d->pos, d->pos + 3 * d->n_atoms);
    s->r_loc.assign(d->r_loc, d->r_loc + d->n_atoms);
    s->r_fine.assign(d->r_fine, d->r_fine + d->n_atoms);
    s->nsf.assign(d->n_sf, d->n_sf + d->n_atoms);
    s->margin = d->lprime_margin;
    s->cutoff = d->pair_cutoff;
    s->pair_mode = d->pair_mode;
    s->fine_mode = d->fine_mode;
    s->batch_size = s->prec == LSW_FP64 ? 16 : 32;
    for (int a = 0; a < s->n_atoms; ++a)
        for (int k = 0; k < s->nsf[a]; ++k) s->sf_atom.push_back(a);
    if (s->sf_atom.empty()) return fail(LSW_ERR_ARG, "lsw_system_create: no support functions");
    try {
        // global fine region: union of the fine spheres (Sec. II.B)
        const int64_t npts = static_cast<int64_t>(s->N[0]) * s->N[1] * s->N[2];
        s->fine_mask.assign(npts, 0);
        for (int a = 0; a < s->n_atoms; ++a) {
            const double* c = &s->pos[3 * a];
            const double R = s->r_fine[a];
            const double R2 = R * R;
            int lo[3], hi[3];
            sphere_bounds(s->N, s->h, c, R, lo, hi);
            for (int k = lo[2]; k <= hi[2]; ++k)
                for (int j = lo[1]; j <= hi[1]; ++j)
                    for (int i = lo[0]; i <= hi[0]; ++i) {
                        double x = static_cast<double>(i) * s->h, y = static_cast<double>(j) * s->h,
                               z = static_cast<double>(k) * s->h;
                        if (d2_of(x, y, z, c) <= R2)
                            s->fine_mask[i + static_cast<int64_t>(s->N[0]) * (j + static_cast<int64_t>(s->N[1]) * k)] = 1;
                    }
        }
        s->L.resize(s->n_atoms);
        s->Lp.resize(s->n_atoms);
        lsw_system_s* sp = s.get();
        parallel_for(s->n_atoms, [&](int a) {
            build_locreg(sp, sp->fine_mask, a, sp->r_loc[a], &sp->L[a]);
            const double Rp = sp->r_loc[a] + sp->margin * sp->h;
            build_locreg(sp, sp->fine_mask, a, Rp, &sp->Lp[a]);
        });
        for (int a = 0; a < s->n_atoms; ++a)
            if (s->nsf[a] > 0 && s->L[a].c.g.empty())
                return fail(LSW_ERR_ARG, "atom %d: its locreg holds no grid point", a);
        const int64_t nf = static_cast<int64_t>(s->sf_atom.size());
        s->off_L.assign(nf + 1, 0);
        s->off_Lp.assign(nf + 1, 0);
        for (int64_t f = 0; f < nf; ++f) {
            int a = s->sf_atom[f];
            int64_t nL = static_cast<int64_t>(s->L[a].c.g.size() + 7 * s->L[a].f.g.size());
            int64_t nP = static_cast<int64_t>(s->Lp[a].c.g.size() + 7 * s->Lp[a].f.g.size());
            s->off_L[f + 1] = s->off_L[f] + align64(nL);
            s->off_Lp[f + 1] = s->off_Lp[f] + align64(nP);
        }
        lsw_status st = build_pattern(s.get());
        if (st != LSW_OK) return st;
        if (ctx->host_only) {
            ctx->live_systems++;
            *out = s.release();
            return LSW_OK;
        }
        st = upload_geometry(s.get());
        if (st != LSW_OK) return st;
        st = build_plans(s.get());
        if (st != LSW_OK) return st;
        st = build_hs_plan(s.get());
        if (st != LSW_OK) return st;
    } catch (const std::bad_alloc&) {
        return fail(LSW_ERR_OOM, "lsw_system_create: host allocation");
    }
    CUDA_TRY(s->d_status.alloc(STATUS_WORDS * sizeof(int)));
    CUDA_TRY(cudaMemset(s->d_status.p, 0, STATUS_WORDS * sizeof(int)));
    CUDA_TRY(s->d_escratch.alloc(2 * s->sf_atom.size() * sizeof(double)));
    CUDA_TRY(cudaEventCreateWithFlags(&s->done, cudaEventDisableTiming));
    ctx->live_systems++;
    *out = s.release();
    return LSW_OK;
}

lsw_status lsw_system_destroy(lsw_system sys) {
    g_err.clear();
    if (!sys) return LSW_OK;
    if (!sys->ctx->host_only) cudaSetDevice(sys->ctx->device);
    drop_graphs(sys);
    if (sys->done) cudaEventDestroy(sys->done);
    if (sys->copy_in) cudaStreamDestroy(sys->copy_in);
    if (sys->copy_out) cudaStreamDestroy(sys->copy_out);
    sys->ctx->live_systems--;
    delete sys;
    return LSW_OK;
}

lsw_status lsw_system_layout(lsw_system sys, int64_t* n_sf, int64_t* total_L, int64_t* total_Lp,
                             const int64_t** off_L, const int64_t** off_Lp, const int32_t** sf_atom) {
    g_err.clear();
    if (!sys) return fail(LSW_ERR_ARG, "lsw_system_layout: NULL system");
    if (n_sf) *n_sf = static_cast<int64_t>(sys->sf_atom.size());
    if (total_L) *total_L = sys->off_L.back();
    if (total_Lp) *total_Lp = sys->off_Lp.back();
    if (off_L) *off_L = sys->off_L.data();
    if (off_Lp) *off_Lp = sys->off_Lp.data();
    if (sf_atom) *sf_atom = sys->sf_atom.data();
    return LSW_OK;
}

lsw_status lsw_system_keys(lsw_system sys, int32_t atom, int32_t region, int32_t part, int64_t* nseg,
                           const int64_t** keys) {
    g_err.clear();
    if (!sys || !nseg || !keys) return fail(LSW_ERR_ARG, "lsw_system_keys: NULL argument");
    if (atom < 0 || atom >= sys->n_atoms) return fail(LSW_ERR_ARG, "lsw_system_keys: atom %d", atom);
    if (region != LSW_REGION_L && region != LSW_REGION_LP) return fail(LSW_ERR_ARG, "lsw_system_keys: region %d", region);
    if (part != LSW_PART_COARSE && part != LSW_PART_FINE) return fail(LSW_ERR_ARG, "lsw_system_keys: part %d", part);
    const LocregHost& L = region == LSW_REGION_L ? sys->L[atom] : sys->Lp[atom];
    const RegionHost& r = part == LSW_PART_COARSE ? L.c : L.f;
    *nseg = static_cast<int64_t>(r.keys.size() / 3);
    *keys = r.keys.data();
    return LSW_OK;
}

lsw_status lsw_pattern(lsw_system sys, int64_t* nnz, const int64_t** row_ptr, const int32_t** col) {
    g_err.clear();
    if (!sys) return fail(LSW_ERR_ARG, "lsw_pattern: NULL system");
    if (nnz) *nnz = static_cast<int64_t>(sys->col.size());
    if (row_ptr) *row_ptr = sys->row_ptr.data();
    if (col) *col = sys->col.data();
    return LSW_OK;
}

lsw_status lsw_set_potential(lsw_system sys, const void* V_dev, const int64_t fine_lo[3], const int64_t fine_dims[3]) {
    g_err.clear();
    if (sys && sys->ctx->host_only) return fail(LSW_ERR_STATE, "host-only context: no device work");
    if (!sys || !V_dev || !fine_lo || !fine_dims) return fail(LSW_ERR_ARG, "lsw_set_potential: NULL argument");
    for (int d = 0; d < 3; ++d) {
        const int64_t need_lo = -V_REACH, need_hi = 2LL * sys->N[d] + V_REACH;
        if (fine_dims[d] < 1 || fine_lo[d] > need_lo || fine_lo[d] + fine_dims[d] - 1 < need_hi)
            return fail(LSW_ERR_ARG, "lsw_set_potential: dimension %d covers [%lld, %lld], needs [%lld, %lld]", d,
                        static_cast<long long>(fine_lo[d]), static_cast<long long>(fine_lo[d] + fine_dims[d] - 1),
                        static_cast<long long>(need_lo), static_cast<long long>(need_hi));
    }
    if (sys->V != V_dev) drop_graphs(sys);
    for (int d = 0; d < 3; ++d) {
        if (sys->vlo[d] != fine_lo[d] || sys->vn[d] != fine_dims[d]) drop_graphs(sys);
        sys->vlo[d] = fine_lo[d];
        sys->vn[d] = fine_dims[d];
    }
    sys->V = V_dev;
    return LSW_OK;
}

lsw_status lsw_apply_hamiltonian(lsw_system sys, const void* phi, void* hphi, double* ek, double* ep) {
    g_err.clear();
    if (sys && sys->ctx->host_only) return fail(LSW_ERR_STATE, "host-only context: no device work");
    if (!sys || !phi || !hphi) return fail(LSW_ERR_ARG, "lsw_apply_hamiltonian: NULL buffer");
    if (!sys->V) return fail(LSW_ERR_STATE, "lsw_apply_hamiltonian: no potential (lsw_set_potential)");
    const int64_t nf = static_cast<int64_t>(sys->sf_atom.size());
    double* e0 = static_cast<double*>(sys->d_escratch.p);
    if (!ek) ek = e0;
    if (!ep) ep = e0 + nf;
    CUDA_TRY(cudaSetDevice(sys->ctx->device));
    (void)cudaGetLastError();   // an earlier call's error is not this call's
    GraphKey key{phi, hphi, ek, ep};
    return run_maybe_graph(sys, &sys->graphs_h, key, [&](Tracer* tr) { return enqueue_apply(sys, tr, phi, hphi, ek, ep); });
}

lsw_status lsw_build_matrices(lsw_system sys, const void* phi, const void* hphi, double* H, double* S) {
    g_err.clear();
    if (sys && sys->ctx->host_only) return fail(LSW_ERR_STATE, "host-only context: no device work");
    if (!sys || !phi || !hphi || !H || !S) return fail(LSW_ERR_ARG, "lsw_build_matrices: NULL buffer");
    CUDA_TRY(cudaSetDevice(sys->ctx->device));
    (void)cudaGetLastError();   // an earlier call's error is not this call's
    if (lsw_status e = ensure_panels(sys); e != LSW_OK) return e;
    GraphKey key{phi, hphi, H, S};
    return run_maybe_graph(sys, &sys->graphs_m, key, [&](Tracer* tr) { return enqueue_matrices(sys, tr, phi, hphi, H, S); });
}

lsw_status lsw_combine(lsw_system sys, const double* M, const void* phi_in, void* phi_out) {
    g_err.clear();
    if (sys && sys->ctx->host_only) return fail(LSW_ERR_STATE, "host-only context: no device work");
    if (!sys || !M || !phi_in || !phi_out) return fail(LSW_ERR_ARG, "lsw_combine: NULL buffer");
    if (phi_in == phi_out) return fail(LSW_ERR_ARG, "lsw_combine: input and output must not overlap");
    CUDA_TRY(cudaSetDevice(sys->ctx->device));
    (void)cudaGetLastError();   // an earlier call's error is not this call's
    if (lsw_status e = ensure_panels(sys); e != LSW_OK) return e;
    return enqueue_combine(sys, nullptr, M, phi_in, phi_out);
}

lsw_status lsw_lowdin_taylor(lsw_system sys, const double* S, const void* phi_in, void* phi_out) {
    g_err.clear();
    if (sys && sys->ctx->host_only) return fail(LSW_ERR_STATE, "host-only context: no device work");
    if (!sys || !S || !phi_in || !phi_out) return fail(LSW_ERR_ARG, "lsw_lowdin_taylor: NULL buffer");
    if (phi_in == phi_out) return fail(LSW_ERR_ARG, "lsw_lowdin_taylor: input and output must not overlap");
    CUDA_TRY(cudaSetDevice(sys->ctx->device));
    (void)cudaGetLastError();   // an earlier call's error is not this call's
    if (lsw_status e = ensure_panels(sys); e != LSW_OK) return e;
    const int64_t nnz = static_cast<int64_t>(sys->col.size());
    if (sys->d_mcoef.bytes < static_cast<size_t>(std::max<int64_t>(nnz, 1)) * sizeof(double)) {
        CUDA_TRY(cudaStreamSynchronize(sys->stream));
        CUDA_TRY(sys->d_mcoef.alloc(static_cast<size_t>(std::max<int64_t>(nnz, 1)) * sizeof(double)));
    }
    double* T = static_cast<double*>(sys->d_mcoef.p);
    CUDA_TRY(enqueue_lowdin_coeffs(static_cast<const int64_t*>(sys->d_rowp.p), static_cast<const int32_t*>(sys->d_col.p),
                                   S, T, static_cast<int>(sys->sf_atom.size()), sys->stream));
    return enqueue_combine(sys, nullptr, T, phi_in, phi_out);
}

lsw_status lsw_foe(lsw_system sys, const double* H, const double* S, double e_min, double e_max, double n_el,
                   int32_t n_pl, double de, double tol, int32_t max_bisect, double* Kp_out, double* K_out,
                   double* mu_out, double* ebs_out, double* trace_out) {
    g_err.clear();
    if (sys && sys->ctx->host_only) return fail(LSW_ERR_STATE, "host-only context: no device work");
    if (!sys || !H || !S || !Kp_out || !K_out) return fail(LSW_ERR_ARG, "lsw_foe: NULL buffer");
    if (!(e_max > e_min) || !(de > 0.0) || n_pl < 1 || max_bisect < 1 || !(tol >= 0.0))
        return fail(LSW_ERR_ARG, "lsw_foe: need e_max > e_min, de > 0, n_pl >= 1, max_bisect >= 1, tol >= 0");
    const int n = static_cast<int>(sys->sf_atom.size());
    const int64_t nnz = static_cast<int64_t>(sys->col.size());
    if (static_cast<size_t>(n) * sizeof(int) + 1024 > sys->ctx->max_smem)
        return fail(LSW_ERR_UNSUPPORTED, "lsw_foe: %d functions exceed the shared-memory column map", n);
    CUDA_TRY(cudaSetDevice(sys->ctx->device));
    (void)cudaGetLastError();   // an earlier call's error is not this call's
    cudaStream_t st = sys->stream;
    const int triple_ctas = std::max(1, std::min(n, 4 * sys->ctx->n_sm));
    if (sys->d_tpos.bytes == 0) {
        // transposed and diagonal positions of the pattern, the identity on it
        std::vector<int64_t> tpos(nnz), diag(n, -1);
        std::vector<double> ident(nnz, 0.0);
        for (int a = 0; a < n; ++a)
            for (int64_t k = sys->row_ptr[a]; k < sys->row_ptr[a + 1]; ++k) {
                const int b = sys->col[k];
                const int32_t* c0 = sys->col.data() + sys->row_ptr[b];
                const int32_t* c1 = sys->col.data() + sys->row_ptr[b + 1];
                const int32_t* it = std::lower_bound(c0, c1, a);
                if (it == c1 || *it != a) return fail(LSW_ERR_UNSUPPORTED, "lsw_foe: the pattern is not symmetric");
                tpos[k] = sys->row_ptr[b] + (it - c0);
                if (b == a) diag[a] = k, ident[k] = 1.0;
            }
        for (int a = 0; a < n; ++a)
            if (diag[a] < 0) return fail(LSW_ERR_UNSUPPORTED, "lsw_foe: the pattern lacks a diagonal entry");
        CUDA_TRY(sys->d_tpos.upload(tpos, st));
        CUDA_TRY(sys->d_diag.upload(diag, st));
        CUDA_TRY(sys->d_ident.upload(ident, st));
        CUDA_TRY(sys->d_foe.alloc(static_cast<size_t>(std::max<int64_t>(nnz, 1)) * 9 * sizeof(double) +
                                  static_cast<size_t>(n_pl + 1 + 2) * sizeof(double)));
        CUDA_TRY(sys->d_foe_scratch.alloc(static_cast<size_t>(triple_ctas) * n * sizeof(double)));
        CUDA_TRY(cudaMemsetAsync(sys->d_foe_scratch.p, 0, sys->d_foe_scratch.bytes, st));
    }
    if (sys->d_foe.bytes < static_cast<size_t>(std::max<int64_t>(nnz, 1)) * 9 * sizeof(double) +
                               static_cast<size_t>(n_pl + 3) * sizeof(double)) {
        CUDA_TRY(cudaStreamSynchronize(st));
        CUDA_TRY(sys->d_foe.alloc(static_cast<size_t>(std::max<int64_t>(nnz, 1)) * 9 * sizeof(double) +
                                  static_cast<size_t>(n_pl + 3) * sizeof(double)));
    }
    FoeLaunch f;
    f.n = n;
    f.nnz = nnz;
    f.row_ptr = static_cast<const int64_t*>(sys->d_rowp.p);
    f.col = static_cast<const int32_t*>(sys->d_col.p);
    f.tpos = static_cast<const int64_t*>(sys->d_tpos.p);
    f.diag = static_cast<const int64_t*>(sys->d_diag.p);
    f.scratch = static_cast<double*>(sys->d_foe_scratch.p);
    f.triple_ctas = triple_ctas;
    f.cheb_ctas = std::max(1, std::min(n, 2 * sys->ctx->n_sm));
    f.status = static_cast<int*>(sys->d_status.p);
    double* w = static_cast<double*>(sys->d_foe.p);
    double* Ht = w;
    double* X = w + nnz;
    double* Htp = w + 2 * nnz;
    double* T[3] = {w + 3 * nnz, w + 4 * nnz, w + 5 * nnz};
    double* Kc = w + 6 * nnz;
    double* tmp = w + 7 * nnz;
    double* tr_d = w + 9 * nnz;          // n_pl + 1 traces, then E_BS
    const double* I = static_cast<const double*>(sys->d_ident.p);
    const double sigma = 2.0 / (e_max - e_min), tau = 0.5 * (e_min + e_max);
    CUDA_TRY(foe_prep(f, H, S, sigma, tau, Ht, X, st));
    CUDA_TRY(foe_triple(f, X, Ht, Htp, st));
    // the Chebyshev recursion t^{j+1} = 2 H~' t^j - t^{j-1} on every pattern column;
    // pass 1 keeps the traces (for the search of mu), pass 2 sums K'
    auto recursion = [&](const std::vector<double>* c) -> lsw_status {
        const double* prev = I;
        double* cur = T[0];
        CUDA_TRY(foe_cheb(f, Htp, I, nullptr, 1.0, cur, st));
        if (c) CUDA_TRY(foe_axpy_t(f, Kc, cur, (*c)[1], st));
        else CUDA_TRY(foe_trace(f, cur, tr_d + 1, st));
        int slot = 1;
        for (int j = 2; j <= n_pl; ++j) {
            double* next = T[slot];
            CUDA_TRY(foe_cheb(f, Htp, cur, prev, 2.0, next, st));
            if (c) CUDA_TRY(foe_axpy_t(f, Kc, next, (*c)[j], st));
            else CUDA_TRY(foe_trace(f, next, tr_d + j, st));
            prev = cur;
            cur = next;
            slot = (slot + 1) % 3;
            if (T[slot] == prev) slot = (slot + 1) % 3;
        }
        return LSW_OK;
    };
    lsw_status e = recursion(nullptr);
    if (e != LSW_OK) return e;
    std::vector<double> tr(n_pl + 1);
    CUDA_TRY(cudaMemcpyAsync(tr.data() + 1, tr_d + 1, n_pl * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    tr[0] = static_cast<double>(n);
    // mu by bisection on [e_min, e_max]: Tr K' = c_0/2 Tr T_0 + sum_j c_j Tr T_j, the c_j
    // those of the polynomial interpolating 1/2 [1 - erf((x - sigma (mu - tau)) / (sigma de))]
    // at the n_pl + 1 Chebyshev nodes
    const int Nn = n_pl + 1;
    std::vector<double> c(Nn), cosj(static_cast<size_t>(Nn) * Nn), xk(Nn);
    for (int k = 0; k < Nn; ++k) {
        const double th = M_PI * (k + 0.5) / Nn;
        xk[k] = std::cos(th);
        for (int j = 0; j < Nn; ++j) cosj[static_cast<size_t>(j) * Nn + k] = std::cos(j * th);
    }
    double lo = e_min, hi = e_max, mu = 0.5 * (lo + hi), trace = 0.0;
    for (int it = 0; it < max_bisect; ++it) {
        mu = 0.5 * (lo + hi);
        const double m0 = sigma * (mu - tau), w0 = sigma * de;
        std::vector<double> fx(Nn);
        for (int k = 0; k < Nn; ++k) fx[k] = 0.5 * (1.0 - std::erf((xk[k] - m0) / w0));
        for (int j = 0; j < Nn; ++j) {
            double acc = 0.0;
            for (int k = 0; k < Nn; ++k) acc += fx[k] * cosj[static_cast<size_t>(j) * Nn + k];
            c[j] = 2.0 / Nn * acc;
        }
        trace = 0.5 * c[0] * tr[0];
        for (int j = 1; j < Nn; ++j) trace += c[j] * tr[j];
        if (std::fabs(trace - n_el) <= tol) break;
        if (trace < n_el) lo = mu;
        else hi = mu;
    }
    CUDA_TRY(cudaMemsetAsync(Kc, 0, nnz * sizeof(double), st));
    CUDA_TRY(foe_axpy_t(f, Kc, I, 0.5 * c[0], st));
    e = recursion(&c);
    if (e != LSW_OK) return e;
    CUDA_TRY(foe_transpose(f, Kc, Kp_out, st));        // K' (columns were kept on the CSR rows)
    CUDA_TRY(foe_triple(f, X, Kp_out, K_out, st));     // K = S^-1/2 K' S^-1/2 on the pattern
    CUDA_TRY(foe_ebs(f, K_out, Ht, S, sigma, tau, tr_d + n_pl + 1, st));
    double ebs = 0.0;
    CUDA_TRY(cudaMemcpyAsync(&ebs, tr_d + n_pl + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    (void)tmp;
    if (mu_out) *mu_out = mu;
    if (ebs_out) *ebs_out = ebs;
    if (trace_out) *trace_out = trace;
    return LSW_OK;
}

// ---------------------------------------------------------------- confinement (Sec. "Support function optimization")

namespace {
// Tables of the 1D operators (x - R_d)^m, m = 2, 4, between the scaling (b = 0) and
// wavelet (b = 1) functions of coarse points i, j = i + l (|l| <= 14) along each
// dimension of every atom's widened box (i over [lo_d - 14, lo_d + n_d + 13]):
//   <chi^b_i|(x - R)^m|chi^b'_j> = (h/2)^m sum_p C(m,p) sum_k X_k (2i + k - 2c)^(m-p) G^p_Y(l, k),
//   G^p_Y(l, k) = sum_k' Y_k' F^p(2l + k' - k),   c = R_d / h,  X, Y = h or g by b, b',
// F^p the moment overlaps of the filter set (the Galerkin matrix of the multiplication
// operator x^m in the two-level basis, expanded by the refinement equation).
// G[y][p][l + 14][k] = sum_k' Y_k' F^p(2l + k' - k)
std::vector<double> conf_G(const FilterSet& F) {
    const double* XY[2] = {F.h, F.g};
    std::vector<double> G(2 * MOVL_P * KIN_TAPS * D16, 0.0);
    for (int y = 0; y < 2; ++y)
        for (int p = 0; p < MOVL_P; ++p)
            for (int l = -KIN_HALF; l <= KIN_HALF; ++l)
                for (int k = 0; k < D16; ++k) {
                    double acc = 0.0;
                    for (int kp = 0; kp < D16; ++kp) {
                        const int idx = 2 * l + (kp + H_LO) - (k + H_LO);
                        if (idx < -KIN_HALF || idx > KIN_HALF) continue;
                        acc += XY[y][kp] * F.movl[p][idx + KIN_HALF];
                    }
                    G[((y * MOVL_P + p) * KIN_TAPS + (l + KIN_HALF)) * D16 + k] = acc;
                }
    return G;
}

// out[l + 14] = <chi^b_i|(x - R)^m|chi^b'_{i+l}>, l = -14..14, c = R / h
void conf_row(const FilterSet& F, const std::vector<double>& G, int m, int b, int bp, double gi, double c, double h,
              double* out) {
    const double* XY[2] = {F.h, F.g};
    const double hm = std::pow(h / 2.0, m);
    for (int l = -KIN_HALF; l <= KIN_HALF; ++l) {
        double acc = 0.0;
        double cp = 1.0;   // C(m, p)
        for (int p = 0; p <= m; ++p) {
            if (p > 0) cp = cp * (m - p + 1) / p;
            const double* Gp = &G[((bp * MOVL_P + p) * KIN_TAPS + (l + KIN_HALF)) * D16];
            double sk = 0.0;
            for (int k = 0; k < D16; ++k) {
                const double z = 2.0 * gi + (k + H_LO) - 2.0 * c;
                double zp = 1.0;
                for (int r = 0; r < m - p; ++r) zp *= z;
                sk += XY[b][k] * zp * Gp[k];
            }
            acc += cp * sk;
        }
        out[l + KIN_HALF] = hm * acc;
    }
}

lsw_status build_conf_tables(lsw_system_s* s) {
    const FilterSet& F = s->ctx->filters;
    const std::vector<double> G = conf_G(F);
    const int na = s->n_atoms;
    std::vector<int64_t> off(na + 1, 0);
    for (int a = 0; a < na; ++a) {
        int64_t n = 0;
        for (int d = 0; d < 3; ++d) n += 2LL * 4 * (s->L[a].n[d] + 2 * KIN_HALF) * KIN_TAPS;
        off[a + 1] = off[a] + n;
    }
    std::vector<double> tab(std::max<int64_t>(off[na], 1), 0.0);
    const double h = s->h;
    parallel_for(na, [&](int a) {
        int64_t base = off[a];
        for (int d = 0; d < 3; ++d) {
            const int E = s->L[a].n[d] + 2 * KIN_HALF;
            const double c = s->pos[3 * a + d] / h;
            for (int mi = 0; mi < 2; ++mi)
                for (int b = 0; b < 2; ++b)
                    for (int bp = 0; bp < 2; ++bp)
                        for (int i = 0; i < E; ++i)
                            conf_row(F, G, mi == 0 ? 2 : 4, b, bp, static_cast<double>(s->L[a].lo[d] - KIN_HALF + i), c, h,
                                     &tab[base + ((static_cast<int64_t>(mi) * 4 + (b * 2 + bp)) * E + i) * KIN_TAPS]);
            base += 2LL * 4 * E * KIN_TAPS;
        }
    });
    cudaStream_t st = s->stream;
    CUDA_TRY(s->d_qtab.upload(tab, st));
    CUDA_TRY(s->d_qtab_off.upload(off, st));
    return LSW_OK;
}

// Launch arguments of one batch [f0, f0 + nfn) of the confinement kernels.
ConfLaunch conf_launch(lsw_system_s* s, int64_t f0, int nfn, const double* acoef, const double* eps, int64_t box_stride) {
    ConfLaunch c;
    std::memset(&c, 0, sizeof(c));
    c.prec = s->prec;
    c.f0 = f0;
    c.nfn = nfn;
    c.sf_atom = static_cast<const int32_t*>(s->d_sfatom.p);
    c.atoms = static_cast<const AtomRec*>(s->d_atoms.p);
    c.seg = static_cast<const Seg*>(s->d_seg.p);
    c.rowptr = static_cast<const int32_t*>(s->d_rowptr.p);
    c.off_L = static_cast<const int64_t*>(s->d_offL.p);
    c.off_Lp = static_cast<const int64_t*>(s->d_offLp.p);
    c.qtab = static_cast<const double*>(s->d_qtab.p);
    c.qtab_off = static_cast<const int64_t*>(s->d_qtab_off.p);
    c.acoef = acoef;
    c.eps = eps;
    for (int b = 0; b < 4; ++b)
        for (int l = 0; l < KIN_TAPS; ++l) c.kin[b][l] = s->ctx->filters.kin[b][l];
    c.kin_scale = -1.0 / (2.0 * s->h * s->h);
    c.box_stride = box_stride;
    for (int64_t f = f0; f < f0 + nfn; ++f) {
        const int a = s->sf_atom[f];
        c.max_rows_L = std::max(c.max_rows_L, s->L[a].n[1] * s->L[a].n[2]);
        c.max_rows_P = std::max(c.max_rows_P, s->Lp[a].n[1] * s->Lp[a].n[2]);
        int64_t v = 1;
        for (int d = 0; d < 3; ++d) v *= s->L[a].n[d] + 2 * KIN_HALF;
        c.max_vol = std::max(c.max_vol, v);
    }
    c.status = static_cast<int*>(s->d_status.p);
    c.qtab_n = static_cast<int64_t>(s->d_qtab.bytes / sizeof(double));
    c.seg_n = static_cast<int64_t>(s->d_seg.bytes / sizeof(Seg));
    c.rowptr_n = static_cast<int64_t>(s->d_rowptr.bytes / sizeof(int32_t));
    c.vec_n = s->off_L.back();
    c.dst_n = s->off_Lp.back();
    c.n_sf = static_cast<int>(s->sf_atom.size());
    c.n_atoms = s->n_atoms;
    return c;
}

// Tables (first call) and batch boxes: three boxes per function of a batch, the batch
// sized to a budget of 2 GiB.  Returns the box stride (elements) and the batch size.
lsw_status conf_prepare(lsw_system_s* s, int64_t* box_stride, int* batch) {
    if (s->d_qtab.bytes == 0) {
        lsw_status e = build_conf_tables(s);
        if (e != LSW_OK) return e;
    }
    int64_t vmax = 0;
    for (int a = 0; a < s->n_atoms; ++a) {
        int64_t v = 1;
        for (int d = 0; d < 3; ++d) v *= s->L[a].n[d] + 2 * KIN_HALF;
        vmax = std::max(vmax, v);
    }
    *box_stride = align64(8 * vmax);
    const int64_t nf = static_cast<int64_t>(s->sf_atom.size());
    const size_t per = 3 * static_cast<size_t>(*box_stride) * s->esize;
    const int b = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>({64, nf, static_cast<int64_t>((size_t(2) << 30) / per)})));
    if (s->d_cbox.bytes < per * b) {
        CUDA_TRY(cudaStreamSynchronize(s->stream));
        CUDA_TRY(s->d_cbox.alloc(per * b));
    }
    *batch = b;
    return LSW_OK;
}
}  // namespace

lsw_status lsw_confinement_row(lsw_system sys, int32_t atom, int32_t dim, int32_t m, int32_t b, int32_t bp, int64_t i,
                               double* out) {
    g_err.clear();
    if (!sys || !out) return fail(LSW_ERR_ARG, "lsw_confinement_row: NULL argument");
    if (atom < 0 || atom >= sys->n_atoms || dim < 0 || dim > 2 || (m != 2 && m != 4) || b < 0 || b > 1 || bp < 0 || bp > 1)
        return fail(LSW_ERR_ARG, "lsw_confinement_row: argument out of range");
    const std::vector<double> G = conf_G(sys->ctx->filters);
    conf_row(sys->ctx->filters, G, m, b, bp, static_cast<double>(i), sys->pos[3 * atom + dim] / sys->h, sys->h, out);
    return LSW_OK;
}

lsw_status lsw_add_confinement(lsw_system sys, const double* a_dev, const void* phi, void* hphi, double* e_conf) {
    g_err.clear();
    if (sys && sys->ctx->host_only) return fail(LSW_ERR_STATE, "host-only context: no device work");
    if (!sys || !a_dev || !phi || !hphi) return fail(LSW_ERR_ARG, "lsw_add_confinement: NULL buffer");
    CUDA_TRY(cudaSetDevice(sys->ctx->device));
    (void)cudaGetLastError();   // an earlier call's error is not this call's
    int64_t stride = 0;
    int batch = 0;
    lsw_status e = conf_prepare(sys, &stride, &batch);
    if (e != LSW_OK) return e;
    const int64_t nf = static_cast<int64_t>(sys->sf_atom.size());
    unsigned char* box = static_cast<unsigned char*>(sys->d_cbox.p);
    const size_t bb = static_cast<size_t>(batch) * stride * sys->esize;
    for (int64_t f0 = 0; f0 < nf; f0 += batch) {
        const int nb = static_cast<int>(std::min<int64_t>(batch, nf - f0));
        ConfLaunch c = conf_launch(sys, f0, nb, a_dev, nullptr, stride);
        CUDA_TRY(conf_apply(c, phi, box, box + bb, box + 2 * bb, hphi, 1, 1, false, e_conf, sys->stream));
    }
    return LSW_OK;
}

lsw_status lsw_precondition(lsw_system sys, const double* a_dev, const double* eps_dev, const void* g, void* gprec,
                            int32_t iters, double* res) {
    g_err.clear();
    if (sys && sys->ctx->host_only) return fail(LSW_ERR_STATE, "host-only context: no device work");
    if (!sys || !a_dev || !eps_dev || !g || !gprec) return fail(LSW_ERR_ARG, "lsw_precondition: NULL buffer");
    if (g == gprec) return fail(LSW_ERR_ARG, "lsw_precondition: g and g_prec must not overlap");
    if (iters < 1) return fail(LSW_ERR_ARG, "lsw_precondition: iters %d", iters);
    CUDA_TRY(cudaSetDevice(sys->ctx->device));
    (void)cudaGetLastError();   // an earlier call's error is not this call's
    int64_t stride = 0;
    int batch = 0;
    lsw_status e = conf_prepare(sys, &stride, &batch);
    if (e != LSW_OK) return e;
    const int64_t nf = static_cast<int64_t>(sys->sf_atom.size());
    const int64_t nv = sys->off_L.back();
    const size_t vb = static_cast<size_t>(std::max<int64_t>(nv, 1)) * sys->esize;
    if (sys->d_cg.bytes < 3 * vb || sys->d_cgs.bytes < 4 * nf * sizeof(double)) {
        CUDA_TRY(cudaStreamSynchronize(sys->stream));
        CUDA_TRY(sys->d_cg.alloc(3 * vb));
        CUDA_TRY(sys->d_cgs.alloc(static_cast<size_t>(4 * std::max<int64_t>(nf, 1)) * sizeof(double)));
    }
    unsigned char* V = static_cast<unsigned char*>(sys->d_cg.p);
    void* r = V;
    void* p = V + vb;
    void* Ap = V + 2 * vb;
    double* sc = static_cast<double*>(sys->d_cgs.p);
    double* rr = sc;
    double* rr_new = sc + nf;
    double* pAp = sc + 2 * nf;
    unsigned char* box = static_cast<unsigned char*>(sys->d_cbox.p);
    const size_t bb = static_cast<size_t>(batch) * stride * sys->esize;
    cudaStream_t st = sys->stream;
    for (int64_t f0 = 0; f0 < nf; f0 += batch) {
        const int nb = static_cast<int>(std::min<int64_t>(batch, nf - f0));
        ConfLaunch c = conf_launch(sys, f0, nb, a_dev, eps_dev, stride);
        CUDA_TRY(conf_cg_init(c, g, gprec, r, p, st));
        CUDA_TRY(conf_dot(c, r, r, rr, st));
        for (int it = 0; it < iters; ++it) {
            // Ap = P_L (T + Q - eps) P_L p
            CUDA_TRY(conf_apply(c, p, box, box + bb, box + 2 * bb, Ap, 0, 0, true, nullptr, st));
            CUDA_TRY(conf_dot(c, p, Ap, pAp, st));
            CUDA_TRY(conf_cg_step1(c, rr, pAp, p, Ap, gprec, r, st));
            CUDA_TRY(conf_dot(c, r, r, rr_new, st));
            CUDA_TRY(conf_cg_step2(c, rr, rr_new, r, p, res ? res + static_cast<int64_t>(it) * nf : nullptr, st));
        }
    }
    return LSW_OK;
}

lsw_status lsw_build_density(lsw_system sys, const void* phi, const double* K, double* rho, const int64_t fine_lo[3],
                             const int64_t fine_dims[3]) {
    g_err.clear();
    if (sys && sys->ctx->host_only) return fail(LSW_ERR_STATE, "host-only context: no device work");
    if (!sys || !phi || !K || !rho || !fine_lo || !fine_dims) return fail(LSW_ERR_ARG, "lsw_build_density: NULL argument");
    for (int d = 0; d < 3; ++d) {
        const int64_t need_lo = -V_REACH, need_hi = 2LL * sys->N[d] + V_REACH;
        if (fine_dims[d] < 1 || fine_lo[d] > need_lo || fine_lo[d] + fine_dims[d] - 1 < need_hi)
            return fail(LSW_ERR_ARG, "lsw_build_density: dimension %d covers [%lld, %lld], needs [%lld, %lld]", d,
                        static_cast<long long>(fine_lo[d]), static_cast<long long>(fine_lo[d] + fine_dims[d] - 1),
                        static_cast<long long>(need_lo), static_cast<long long>(need_hi));
        if (fine_dims[d] > (1LL << 30)) return fail(LSW_ERR_ARG, "lsw_build_density: dimension %d too large", d);
    }
    CUDA_TRY(cudaSetDevice(sys->ctx->device));
    (void)cudaGetLastError();   // an earlier call's error is not this call's
    bool same = sys->dens_ready;
    for (int d = 0; d < 3; ++d) same = same && sys->dens_lo[d] == fine_lo[d] && sys->dens_n[d] == fine_dims[d];
    if (!same) {
        for (auto& kv : sys->graphs_d) cudaGraphExecDestroy(kv.second.exec);
        sys->graphs_d.clear();
        lsw_status rs = build_density_plan(sys, fine_lo, fine_dims);
        if (rs != LSW_OK) return rs;
    }
    GraphKey key{phi, K, rho, nullptr};
    return run_maybe_graph(sys, &sys->graphs_d, key, [&](Tracer* tr) { return enqueue_density_all(sys, tr, phi, K, rho); });
}

// Allocation-free variant of lsw_apply_hamiltonian.  Works like it, batch by batch, but
// every batch's workspace and its function records live in the library's fixed device
// array (noalloc_scratch).  Every function is checked against the array and the on-chip
// tiles before anything is enqueued; then, per batch, a one-thread kernel writes the
// batch's records into the head of the array from the system's resident records (no
// host memory is read by the device), and the existing batch kernels run on the rest.
lsw_status lsw_apply_hamiltonian_noalloc(lsw_system sys, const void* phi, void* hphi, double* ek, double* ep) {
    g_err.clear();
    if (!sys || !phi || !hphi) return fail(LSW_ERR_ARG, "lsw_apply_hamiltonian_noalloc: NULL buffer");
    if (sys->ctx->host_only) return fail(LSW_ERR_STATE, "host-only context: no device work");
    if (!sys->V) return fail(LSW_ERR_STATE, "lsw_apply_hamiltonian_noalloc: no potential (lsw_set_potential)");
    const size_t head = (NOALLOC_MAX_BATCH * sizeof(FnRec) + 255) / 256 * 256;
    const int64_t cap = static_cast<int64_t>((NOALLOC_SCRATCH_BYTES - head) / sys->esize);
    const int zcols = sys->prec == LSW_FP64 ? ZCOLS_F64 : ZCOLS_F32;
    const int64_t nf = static_cast<int64_t>(sys->sf_atom.size());
    // every function on its own must fit the array and the tiles: checked before any work
    for (int64_t f = 0; f < nf; ++f) {
        const FnRec r = noalloc_record(sys, f);
        int64_t sD, sR;
        noalloc_sizes(sys, r, &sD, &sR);
        if (sD + sR > cap)
            return fail(LSW_ERR_UNSUPPORTED,
                        "lsw_apply_hamiltonian_noalloc: support function %lld needs %lld bytes of workspace, more than "
                        "the %lld bytes the fixed device array leaves after its record head",
                        static_cast<long long>(f), static_cast<long long>((sD + sR) * static_cast<int64_t>(sys->esize)),
                        static_cast<long long>(cap * static_cast<int64_t>(sys->esize)));
        if (sys->zsplit && (!ztc_fits(r) || (sys->xy_tc && !xytc_fits(r))))
            return fail(LSW_ERR_UNSUPPORTED, "locreg extents too large for the tensor-core kernels");
        HphiLaunch p;
        std::memset(&p, 0, sizeof(p));
        p.prec = sys->prec;
        size_t plain = 0;
        noalloc_fold(sys, r, zcols, &p, &plain);
        if (!noalloc_finish(sys, &p, plain))
            return fail(LSW_ERR_UNSUPPORTED, "locreg box too large for the on-chip pass tiles");
    }
    CUDA_TRY(cudaSetDevice(sys->ctx->device));
    (void)cudaGetLastError();   // an earlier call's error is not this call's
    void* scratch = nullptr;
    CUDA_TRY(noalloc_scratch(sys->ctx->device, &scratch));
    cudaStream_t st = sys->stream;
    double* e0 = static_cast<double*>(sys->d_escratch.p);
    if (!ek) ek = e0;
    if (!ep) ep = e0 + nf;
    CUDA_TRY(cudaMemsetAsync(ek, 0, nf * sizeof(double), st));
    CUDA_TRY(cudaMemsetAsync(ep, 0, nf * sizeof(double), st));
    int64_t f = 0;
    while (f < nf) {
        HphiLaunch p;
        std::memset(&p, 0, sizeof(p));
        p.prec = sys->prec;
        p.zcols = zcols;
        size_t smem_bwd_plain = 0;
        int nb = 0;
        int64_t need = 0;
        while (f + nb < nf && nb < NOALLOC_MAX_BATCH) {
            const FnRec r = noalloc_record(sys, f + nb);
            int64_t sD, sR;
            noalloc_sizes(sys, r, &sD, &sR);
            if (need + sD + sR > cap) break;
            need += sD + sR;
            p.ws_D_elems += sD;
            noalloc_fold(sys, r, zcols, &p, &smem_bwd_plain);
            ++nb;
        }
        if (nb == 0 || !noalloc_finish(sys, &p, smem_bwd_plain))   // excluded by the checks above
            return fail(LSW_ERR_STATE, "lsw_apply_hamiltonian_noalloc: inconsistent batch plan");
        p.nfn = nb;
        p.zsplit = sys->zsplit;
        p.xy_tc = sys->zsplit ? sys->xy_tc : 0;
        CUDA_TRY(enqueue_noalloc_records(static_cast<const FnRec*>(sys->d_fn.p), f, nb,
                                         static_cast<int64_t>(sys->esize), static_cast<FnRec*>(scratch), st));
        p.fn = static_cast<const FnRec*>(scratch);
        p.atoms = static_cast<const AtomRec*>(sys->d_atoms.p);
        p.seg = static_cast<const Seg*>(sys->d_seg.p);
        p.rowptr = static_cast<const int32_t*>(sys->d_rowptr.p);
        p.phi = phi;
        p.hphi = hphi;
        p.e_kin = ek;
        p.e_pot = ep;
        p.V = sys->V;
        for (int d = 0; d < 3; ++d) {
            p.vlo[d] = sys->vlo[d];
            p.vn[d] = sys->vn[d];
        }
        p.ws = static_cast<unsigned char*>(scratch) + head;
        p.kin_scale = -1.0 / (2.0 * sys->h * sys->h);
        p.status = static_cast<int*>(sys->d_status.p);
        p.phi_n = sys->off_L.back();
        p.hphi_n = sys->off_Lp.back();
        p.v_n = sys->vn[0] * sys->vn[1] * sys->vn[2];
        p.ws_n = cap;
        p.seg_n = static_cast<int64_t>(sys->d_seg.bytes / sizeof(Seg));
        p.rowptr_n = static_cast<int64_t>(sys->d_rowptr.bytes / sizeof(int32_t));
        p.n_atoms = sys->n_atoms;
        CUDA_TRY(enqueue_hphi_batch(p, st));
        f += nb;
    }
    return LSW_OK;
}

lsw_status lsw_reformat(lsw_system dst, lsw_system src, const int32_t* shift, const void* phi_src, void* phi_dst) {
    g_err.clear();
    if (!dst || !src || !shift || !phi_src || !phi_dst) return fail(LSW_ERR_ARG, "lsw_reformat: NULL argument");
    if (dst->ctx->host_only || src->ctx->host_only) return fail(LSW_ERR_STATE, "host-only context: no device work");
    if (dst->ctx->device != src->ctx->device) return fail(LSW_ERR_ARG, "lsw_reformat: systems on different devices");
    if (dst->prec != src->prec) return fail(LSW_ERR_ARG, "lsw_reformat: precisions differ");
    if (dst->n_atoms != src->n_atoms || dst->nsf != src->nsf)
        return fail(LSW_ERR_ARG, "lsw_reformat: atoms or support functions per atom differ");
    if (phi_src == phi_dst) return fail(LSW_ERR_ARG, "lsw_reformat: source and destination overlap");
    CUDA_TRY(cudaSetDevice(dst->ctx->device));
    cudaStream_t st = dst->stream;
    const int64_t nf = static_cast<int64_t>(dst->sf_atom.size());
    // the source's stream must have finished writing phi_src: order the two streams
    if (src->stream != st) {
        CUDA_TRY(cudaEventRecord(src->done, src->stream));
        CUDA_TRY(cudaStreamWaitEvent(st, src->done, 0));
    }
    std::vector<int32_t> sh(shift, shift + 3 * dst->n_atoms);
    CUDA_TRY(dst->d_shift.upload(sh, st));
    if (!dst->d_fn_all.p) {
        std::vector<FnRec> recs(nf);
        for (int64_t f = 0; f < nf; ++f) {
            FnRec& r = recs[f];
            std::memset(&r, 0, sizeof(r));
            r.f = static_cast<int32_t>(f);
            r.atom = dst->sf_atom[f];
            for (int d = 0; d < 3; ++d) {
                r.lo[d] = dst->L[r.atom].lo[d];
                r.n[d] = dst->L[r.atom].n[d];
            }
            r.off_phi = dst->off_L[f];
        }
        CUDA_TRY(dst->d_fn_all.upload(recs, st));
    }
    ReformatLaunch p;
    std::memset(&p, 0, sizeof(p));
    p.fn = static_cast<const FnRec*>(dst->d_fn_all.p);
    p.nfn = static_cast<int>(nf);
    for (int a = 0; a < dst->n_atoms; ++a)
        p.max_seg = std::max<int>(p.max_seg, static_cast<int>((dst->L[a].c.keys.size() + dst->L[a].f.keys.size()) / 3));
    p.atoms_dst = static_cast<const AtomRec*>(dst->d_atoms.p);
    p.atoms_src = static_cast<const AtomRec*>(src->d_atoms.p);
    p.seg_dst = static_cast<const Seg*>(dst->d_seg.p);
    p.seg_src = static_cast<const Seg*>(src->d_seg.p);
    p.rowptr_src = static_cast<const int32_t*>(src->d_rowptr.p);
    p.shift = static_cast<const int32_t*>(dst->d_shift.p);
    p.off_src = static_cast<const int64_t*>(src->d_offL.p);
    p.phi_src = phi_src;
    p.phi_dst = phi_dst;
    p.prec = dst->prec;
    p.status = static_cast<int*>(dst->d_status.p);
    p.seg_dst_n = static_cast<int64_t>(dst->d_seg.bytes / sizeof(Seg));
    p.seg_src_n = static_cast<int64_t>(src->d_seg.bytes / sizeof(Seg));
    p.rowptr_src_n = static_cast<int64_t>(src->d_rowptr.bytes / sizeof(int32_t));
    p.src_n = src->off_L.back();
    p.dst_n = dst->off_L.back();
    CUDA_TRY(cudaMemsetAsync(phi_dst, 0, static_cast<size_t>(dst->off_L.back()) * dst->esize, st));
    CUDA_TRY(enqueue_reformat(p, st));
    return LSW_OK;
}

lsw_status lsw_measure_peaks(lsw_ctx ctx, double* fp32_tflops, double* fp64_tflops, double* copy_gbs) {
    g_err.clear();
    if (!ctx || !fp32_tflops || !fp64_tflops || !copy_gbs) return fail(LSW_ERR_ARG, "lsw_measure_peaks: NULL argument");
    if (ctx->host_only) return fail(LSW_ERR_STATE, "host-only context: no device work");
    CUDA_TRY(cudaSetDevice(ctx->device));
    CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(measure_peaks(ctx->n_sm, fp32_tflops, fp64_tflops, copy_gbs));
    return LSW_OK;
}

lsw_status lsw_workspace_bytes(lsw_system sys, int64_t* bytes) {
    g_err.clear();
    if (!sys || !bytes) return fail(LSW_ERR_ARG, "lsw_workspace_bytes: NULL argument");
    const DeviceBuf* bufs[] = {&sys->d_atoms, &sys->d_seg, &sys->d_rowptr, &sys->d_fn, &sys->d_offL, &sys->d_offLp,
                               &sys->d_sfatom, &sys->d_rowp, &sys->d_col, &sys->d_tile_fine,
                               &sys->d_listA, &sys->d_listB, &sys->d_ptiles, &sys->d_patoms, &sys->d_ttab,
                               &sys->d_items, &sys->d_citems, &sys->d_slab_atoms, &sys->d_PA, &sys->d_PQ, &sys->d_mcoef,
                               &sys->d_tpos, &sys->d_diag, &sys->d_ident, &sys->d_foe, &sys->d_foe_scratch,
                               &sys->d_qtab, &sys->d_qtab_off, &sys->d_cbox, &sys->d_cg, &sys->d_cgs,
                               &sys->d_ws, &sys->d_status, &sys->d_plane_items, &sys->d_queue, &sys->d_colz,
                               &sys->d_escratch, &sys->d_phi, &sys->d_hphi, &sys->d_H, &sys->d_S, &sys->d_ek,
                               &sys->d_ep, &sys->d_shift, &sys->d_fn_all, &sys->d_U, &sys->d_dfn,
                               &sys->d_tptr, &sys->d_tfn};
    int64_t b = 0;
    for (auto* p : bufs) b += static_cast<int64_t>(p->bytes);
    if (!sys->d_PA.p) b += static_cast<int64_t>(sys->panel_bytes_A);   // not allocated yet
    if (!sys->d_PQ.p) b += static_cast<int64_t>(sys->panel_bytes_Q);
    *bytes = b;
    return LSW_OK;
}

lsw_status lsw_sync(lsw_system sys, double timeout_s) {
    g_err.clear();
    if (sys && sys->ctx->host_only) return fail(LSW_ERR_STATE, "host-only context: no device work");
    if (!sys) return fail(LSW_ERR_ARG, "lsw_sync: NULL system");
    CUDA_TRY(cudaSetDevice(sys->ctx->device));
    (void)cudaGetLastError();   // an earlier call's error is not this call's
    CUDA_TRY(cudaEventRecord(sys->done, sys->stream));
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaEventQuery(sys->done);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_fail(e, "lsw_sync");
        double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > timeout_s) return fail(LSW_ERR_TIMEOUT, "lsw_sync: not finished after %.3f s", el);
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    int st[STATUS_WORDS] = {0};
    CUDA_TRY(cudaMemcpy(st, sys->d_status.p, sizeof(st), cudaMemcpyDeviceToHost));
    if (st[0] != 0) {
        cudaMemset(sys->d_status.p, 0, sizeof(st));
        long long idx, bound;
        std::memcpy(&idx, st + 4, 8);
        std::memcpy(&bound, st + 6, 8);
        return fail(LSW_ERR_STATE, "device-side check failed (status bits 0x%x; kernel %d line %d block %d index %lld bound %lld)",
                    st[0], st[1], st[2], st[3], idx, bound);
    }
    return LSW_OK;
}

lsw_status lsw_step_host(lsw_system sys, const void* phi_host, void* hphi_host, double* H_host, double* S_host,
                         double* ek_host, double* ep_host) {
    g_err.clear();
    if (sys && sys->ctx->host_only) return fail(LSW_ERR_STATE, "host-only context: no device work");
    if (!sys || !phi_host || !H_host || !S_host) return fail(LSW_ERR_ARG, "lsw_step_host: NULL argument");
    CUDA_TRY(cudaSetDevice(sys->ctx->device));
    (void)cudaGetLastError();   // an earlier call's error is not this call's
    const int64_t nf = static_cast<int64_t>(sys->sf_atom.size());
    const size_t bphi = static_cast<size_t>(sys->off_L.back()) * sys->esize;
    const size_t bhphi = static_cast<size_t>(sys->off_Lp.back()) * sys->esize;
    const size_t bnnz = sys->col.size() * sizeof(double);
    if (!sys->d_phi.p) {
        CUDA_TRY(sys->d_phi.alloc(bphi));
        CUDA_TRY(sys->d_hphi.alloc(bhphi));
        CUDA_TRY(sys->d_H.alloc(std::max<size_t>(bnnz, 8)));
        CUDA_TRY(sys->d_S.alloc(std::max<size_t>(bnnz, 8)));
        CUDA_TRY(sys->d_ek.alloc(nf * sizeof(double)));
        CUDA_TRY(sys->d_ep.alloc(nf * sizeof(double)));
    }
    // Pipelined: Phi goes up batch by batch on one copy stream, each H phi batch waiting only
    // for its own functions; H phi comes back batch by batch on another copy stream while
    // the later batches run; H and S follow the last batch (they need every function).
    // The H phi batches are enqueued directly (no graph: their waits are on events of
    // this call).
    if (!sys->V) return fail(LSW_ERR_STATE, "lsw_step_host: no potential (lsw_set_potential)");
    cudaStream_t st = sys->stream;
    if (!sys->copy_in) CUDA_TRY(cudaStreamCreateWithFlags(&sys->copy_in, cudaStreamNonBlocking));
    if (!sys->copy_out) CUDA_TRY(cudaStreamCreateWithFlags(&sys->copy_out, cudaStreamNonBlocking));
    const size_t nb = sys->batches.size();
    std::vector<cudaEvent_t> ev;
    struct EvGuard {
        std::vector<cudaEvent_t>* v;
        ~EvGuard() {
            for (cudaEvent_t e : *v) cudaEventDestroy(e);
        }
    } guard{&ev};
    auto event = [&](cudaEvent_t* e) -> cudaError_t {
        cudaError_t c = cudaEventCreateWithFlags(e, cudaEventDisableTiming);
        if (c == cudaSuccess) ev.push_back(*e);
        return c;
    };
    const size_t es = sys->esize;
    const int64_t* oL = sys->off_L.data();
    const int64_t* oP = sys->off_Lp.data();
    cudaEvent_t e_start, e_in_all, e_out_all;
    CUDA_TRY(event(&e_start));
    CUDA_TRY(event(&e_in_all));
    CUDA_TRY(event(&e_out_all));
    // the copies start after what the system's stream holds (a previous step's readers)
    CUDA_TRY(cudaEventRecord(e_start, st));
    CUDA_TRY(cudaStreamWaitEvent(sys->copy_in, e_start, 0));
    CUDA_TRY(cudaStreamWaitEvent(sys->copy_out, e_start, 0));
    std::vector<cudaEvent_t> e_in(nb), e_out(nb);
    int64_t done_in = 0;
    for (size_t i = 0; i < nb; ++i) {
        const Batch& b = sys->batches[i];
        const int64_t a = oL[b.fn0], e = oL[b.fn0 + b.nfn];
        CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(sys->d_phi.p) + a * es, static_cast<const char*>(phi_host) + a * es,
                                 static_cast<size_t>(e - a) * es, cudaMemcpyHostToDevice, sys->copy_in));
        CUDA_TRY(event(&e_in[i]));
        CUDA_TRY(cudaEventRecord(e_in[i], sys->copy_in));
        done_in = e;
    }
    if (static_cast<size_t>(done_in) * es < bphi)       // functions past "hphi_limit"
        CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(sys->d_phi.p) + done_in * es,
                                 static_cast<const char*>(phi_host) + done_in * es, bphi - done_in * es,
                                 cudaMemcpyHostToDevice, sys->copy_in));
    CUDA_TRY(cudaEventRecord(e_in_all, sys->copy_in));
    Tracer* tr = nullptr;
    if (sys->profiling) {
        if (!sys->direct_tr) sys->direct_tr.reset(new Tracer());
        tr = sys->direct_tr.get();
        if (!tr->pending) tr->used = 0;
    }
    int64_t done_out = 0;
    auto before = [&](size_t i) { return cudaStreamWaitEvent(st, e_in[i], 0); };
    auto after = [&](size_t i) -> cudaError_t {
        if (!hphi_host) return cudaSuccess;
        const Batch& b = sys->batches[i];
        const int64_t a = oP[b.fn0], e = oP[b.fn0 + b.nfn];
        cudaError_t c;
        if ((c = event(&e_out[i])) != cudaSuccess) return c;
        if ((c = cudaEventRecord(e_out[i], st)) != cudaSuccess) return c;
        if ((c = cudaStreamWaitEvent(sys->copy_out, e_out[i], 0)) != cudaSuccess) return c;
        done_out = e;
        return cudaMemcpyAsync(static_cast<char*>(hphi_host) + a * es, static_cast<const char*>(sys->d_hphi.p) + a * es,
                               static_cast<size_t>(e - a) * es, cudaMemcpyDeviceToHost, sys->copy_out);
    };
    lsw_status r = enqueue_apply_hooked(sys, tr, sys->d_phi.p, sys->d_hphi.p, static_cast<double*>(sys->d_ek.p),
                                        static_cast<double*>(sys->d_ep.p), before, after);
    if (r != LSW_OK) return r;
    CUDA_TRY(cudaStreamWaitEvent(st, e_in_all, 0));
    r = lsw_build_matrices(sys, sys->d_phi.p, sys->d_hphi.p, static_cast<double*>(sys->d_H.p),
                           static_cast<double*>(sys->d_S.p));
    if (r != LSW_OK) return r;
    CUDA_TRY(cudaMemcpyAsync(H_host, sys->d_H.p, bnnz, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(S_host, sys->d_S.p, bnnz, cudaMemcpyDeviceToHost, st));
    if (hphi_host && static_cast<size_t>(done_out) * es < bhphi)
        CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(hphi_host) + done_out * es,
                                 static_cast<const char*>(sys->d_hphi.p) + done_out * es, bhphi - done_out * es,
                                 cudaMemcpyDeviceToHost, st));
    if (ek_host) CUDA_TRY(cudaMemcpyAsync(ek_host, sys->d_ek.p, nf * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (ep_host) CUDA_TRY(cudaMemcpyAsync(ep_host, sys->d_ep.p, nf * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaEventRecord(e_out_all, sys->copy_out));
    CUDA_TRY(cudaStreamWaitEvent(st, e_out_all, 0));
    return lsw_sync(sys, 600.0);
}

lsw_status lsw_system_set_stream(lsw_system sys, void* stream) {
    g_err.clear();
    if (!sys) return fail(LSW_ERR_ARG, "lsw_system_set_stream: NULL system");
    if (sys->ctx->host_only) return fail(LSW_ERR_STATE, "host-only context: no device work");
    CUDA_TRY(cudaSetDevice(sys->ctx->device));
    (void)cudaGetLastError();   // an earlier call's error is not this call's
    CUDA_TRY(cudaStreamSynchronize(sys->stream));
    sys->stream = static_cast<cudaStream_t>(stream);
    return LSW_OK;
}

lsw_status lsw_profile(lsw_system sys, int32_t enable) {
    g_err.clear();
    if (!sys) return fail(LSW_ERR_ARG, "lsw_profile: NULL system");
    if (sys->ctx->host_only) return fail(LSW_ERR_STATE, "host-only context: no device work");
    if (enable != 0 && enable != 1) return fail(LSW_ERR_ARG, "lsw_profile: enable %d", enable);
    CUDA_TRY(cudaSetDevice(sys->ctx->device));
    (void)cudaGetLastError();   // an earlier call's error is not this call's
    CUDA_TRY(cudaStreamSynchronize(sys->stream));
    drop_graphs(sys);
    sys->direct_tr.reset();
    sys->profiling = enable;
    for (int k = 0; k < TK_COUNT; ++k) sys->prof_ms[k] = 0.0, sys->prof_n[k] = 0;
    return LSW_OK;
}

lsw_status lsw_profile_read(lsw_system sys, int32_t max_kinds, int32_t* n_kinds, double* ms, int64_t* launches) {
    g_err.clear();
    if (!sys || !n_kinds || !ms || !launches) return fail(LSW_ERR_ARG, "lsw_profile_read: NULL argument");
    if (sys->ctx->host_only) return fail(LSW_ERR_STATE, "host-only context: no device work");
    CUDA_TRY(cudaSetDevice(sys->ctx->device));
    (void)cudaGetLastError();   // an earlier call's error is not this call's
    CUDA_TRY(cudaStreamSynchronize(sys->stream));
    harvest(sys, sys->direct_tr.get());
    for (auto* c : {&sys->graphs_h, &sys->graphs_m})
        for (auto& kv : *c) harvest(sys, kv.second.tr.get());
    *n_kinds = TK_COUNT;
    for (int k = 0; k < TK_COUNT && k < max_kinds; ++k) {
        ms[k] = sys->prof_ms[k];
        launches[k] = sys->prof_n[k];
        sys->prof_ms[k] = 0.0;
        sys->prof_n[k] = 0;
    }
    return LSW_OK;
}

lsw_status lsw_set_option(lsw_system sys, const char* name, int64_t value) {
    g_err.clear();
    if (sys && sys->ctx->host_only) return fail(LSW_ERR_STATE, "host-only context: no device work");
    if (!sys || !name) return fail(LSW_ERR_ARG, "lsw_set_option: NULL argument");
    CUDA_TRY(cudaSetDevice(sys->ctx->device));
    (void)cudaGetLastError();   // an earlier call's error is not this call's
    if (std::strcmp(name, "batch") == 0) {
        if (value < 1 || value > 4096) return fail(LSW_ERR_ARG, "lsw_set_option: batch %lld", static_cast<long long>(value));
        CUDA_TRY(cudaStreamSynchronize(sys->stream));
        drop_graphs(sys);
        sys->batch_size = static_cast<int>(value);
        return build_plans(sys);
    }
    if (std::strcmp(name, "hs_tc") == 0) {
        if (value != 0 && value != 1) return fail(LSW_ERR_ARG, "lsw_set_option: hs_tc %lld", static_cast<long long>(value));
        CUDA_TRY(cudaStreamSynchronize(sys->stream));
        drop_graphs(sys);
        sys->hs_tc = static_cast<int>(value);
        return LSW_OK;
    }
    if (std::strcmp(name, "hphi_limit") == 0) {
        if (value < -1 || value > static_cast<int64_t>(sys->sf_atom.size()))
            return fail(LSW_ERR_ARG, "lsw_set_option: hphi_limit %lld", static_cast<long long>(value));
        CUDA_TRY(cudaStreamSynchronize(sys->stream));
        drop_graphs(sys);
        sys->hphi_limit = value;
        return build_plans(sys);
    }
    if (std::strcmp(name, "fwd_list") == 0) {
        if (value != 0 && value != 1) return fail(LSW_ERR_ARG, "lsw_set_option: fwd_list %lld", static_cast<long long>(value));
        CUDA_TRY(cudaStreamSynchronize(sys->stream));
        drop_graphs(sys);
        sys->fwd_list = static_cast<int>(value);
        return build_plans(sys);
    }
    if (std::strcmp(name, "persistent") == 0) {
        if (value < 0 || value > 3) return fail(LSW_ERR_ARG, "lsw_set_option: persistent %lld", static_cast<long long>(value));
        CUDA_TRY(cudaStreamSynchronize(sys->stream));
        drop_graphs(sys);
        sys->persistent = static_cast<int>(value);
        return build_plans(sys);
    }
    if (std::strcmp(name, "graph") == 0) {
        if (value != 0 && value != 1) return fail(LSW_ERR_ARG, "lsw_set_option: graph %lld", static_cast<long long>(value));
        sys->use_graph = static_cast<int>(value);
        return LSW_OK;
    }
    if (std::strcmp(name, "zsplit") == 0) {
        if (value != 2 && value != 3) return fail(LSW_ERR_ARG, "lsw_set_option: zsplit %lld", static_cast<long long>(value));
        if (!sys->zsplit) return fail(LSW_ERR_STATE, "lsw_set_option: zsplit needs an LSW_FP32_BF16X system");
        CUDA_TRY(cudaStreamSynchronize(sys->stream));
        drop_graphs(sys);
        const int old = sys->zsplit;
        sys->zsplit = static_cast<int>(value);
        lsw_status e = build_plans(sys);
        if (e != LSW_OK) {
            const std::string msg = g_err;
            sys->zsplit = old;
            if (build_plans(sys) != LSW_OK) return fail(LSW_ERR_STATE, "lsw_set_option: zsplit: cannot restore plans");
            return fail(e, "%s", msg.c_str());
        }
        return LSW_OK;
    }
    if (std::strcmp(name, "xy_tc") == 0) {
        if (value != 0 && value != 1) return fail(LSW_ERR_ARG, "lsw_set_option: xy_tc %lld", static_cast<long long>(value));
        if (!sys->zsplit) return fail(LSW_ERR_STATE, "lsw_set_option: xy_tc needs an LSW_FP32_BF16X system");
        CUDA_TRY(cudaStreamSynchronize(sys->stream));
        drop_graphs(sys);
        const int old = sys->xy_tc;
        sys->xy_tc = static_cast<int>(value);
        lsw_status e = build_plans(sys);
        if (e != LSW_OK) {
            const std::string msg = g_err;
            sys->xy_tc = old;
            if (build_plans(sys) != LSW_OK) return fail(LSW_ERR_STATE, "lsw_set_option: xy_tc: cannot restore plans");
            return fail(e, "%s", msg.c_str());
        }
        return LSW_OK;
    }
    if (std::strcmp(name, "slab_mb") == 0) {
        if (value < 1 || value > (int64_t(1) << 22)) return fail(LSW_ERR_ARG, "lsw_set_option: slab_mb %lld", static_cast<long long>(value));
        CUDA_TRY(cudaStreamSynchronize(sys->stream));
        drop_graphs(sys);
        sys->slab_mb = value;
        return build_hs_plan(sys);
    }
    if (std::strcmp(name, "tile") == 0) {
        if (value < 2 || value > 8) return fail(LSW_ERR_ARG, "lsw_set_option: tile %lld", static_cast<long long>(value));
        CUDA_TRY(cudaStreamSynchronize(sys->stream));
        drop_graphs(sys);
        sys->tile = static_cast<int>(value);
        return build_hs_plan(sys);
    }
    return fail(LSW_ERR_ARG, "lsw_set_option: unknown option '%s'", name);
}

}  // extern "C"

// ---------------------------------------------------------------- checkpoint

namespace {
const char kSaveMagic[8] = {'L', 'S', 'W', 'S', 'A', 'V', 'E', '1'};

struct FileCloser {
    FILE* f;
    ~FileCloser() {
        if (f) std::fclose(f);
    }
};

template <class V>
bool put(FILE* f, const V* p, size_t n) { return n == 0 || std::fwrite(p, sizeof(V), n, f) == n; }
template <class V>
bool get(FILE* f, V* p, size_t n) { return n == 0 || std::fread(p, sizeof(V), n, f) == n; }

// Reads the description part of a checkpoint; leaves the file at total_L.
lsw_status read_desc(FILE* f, const char* path, lsw_system_desc* d, std::vector<double>& pos, std::vector<double>& rl,
                     std::vector<double>& rf, std::vector<int32_t>& nsf, int32_t* zsplit) {
    char magic[8];
    int32_t version = 0;
    if (!get(f, magic, 8) || std::memcmp(magic, kSaveMagic, 8) != 0 || !get(f, &version, 1) || version != 1)
        return fail(LSW_ERR_IO, "lsw_load: %s is not a checkpoint of this library", path);
    std::memset(d, 0, sizeof(*d));
    bool ok = get(f, d->N, 3) && get(f, &d->h, 1) && get(f, &d->n_atoms, 1) && get(f, &d->lprime_margin, 1) &&
              get(f, &d->pair_cutoff, 1) && get(f, &d->pair_mode, 1) && get(f, &d->fine_mode, 1) &&
              get(f, &d->precision, 1) && get(f, zsplit, 1);
    if (!ok || d->n_atoms < 1 || d->n_atoms > (1 << 26)) return fail(LSW_ERR_IO, "lsw_load: %s: truncated header", path);
    const size_t n = static_cast<size_t>(d->n_atoms);
    pos.resize(3 * n);
    rl.resize(n);
    rf.resize(n);
    nsf.resize(n);
    if (!get(f, pos.data(), 3 * n) || !get(f, rl.data(), n) || !get(f, rf.data(), n) || !get(f, nsf.data(), n))
        return fail(LSW_ERR_IO, "lsw_load: %s: truncated atom arrays", path);
    d->pos = pos.data();
    d->r_loc = rl.data();
    d->r_fine = rf.data();
    d->n_sf = nsf.data();
    return LSW_OK;
}

// Reads total_L, has_phi and (if phi_dev) the values into phi_dev.
lsw_status read_phi(FILE* f, const char* path, lsw_system_s* s, void* phi_dev) {
    int64_t total = -1, has = 0;
    if (!get(f, &total, 1) || !get(f, &has, 1)) return fail(LSW_ERR_IO, "lsw_load: %s: truncated", path);
    if (total != s->off_L.back()) return fail(LSW_ERR_STATE, "lsw_load: %s holds another layout", path);
    if (!phi_dev) return LSW_OK;
    if (!has) return fail(LSW_ERR_STATE, "lsw_load: %s holds no support functions", path);
    if (s->ctx->host_only) return fail(LSW_ERR_STATE, "host-only context: no device work");
    std::vector<unsigned char> buf(static_cast<size_t>(total) * s->esize);
    if (!get(f, buf.data(), buf.size())) return fail(LSW_ERR_IO, "lsw_load: %s: truncated values", path);
    CUDA_TRY(cudaSetDevice(s->ctx->device));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    CUDA_TRY(cudaMemcpy(phi_dev, buf.data(), buf.size(), cudaMemcpyHostToDevice));
    return LSW_OK;
}
}  // namespace

extern "C" {

lsw_status lsw_save(lsw_system sys, const void* phi_dev, const char* path) {
    g_err.clear();
    if (!sys || !path) return fail(LSW_ERR_ARG, "lsw_save: NULL argument");
    if (phi_dev && sys->ctx->host_only) return fail(LSW_ERR_STATE, "host-only context: no device work");
    const int64_t total = sys->off_L.back();
    std::vector<unsigned char> buf;
    if (phi_dev) {
        buf.resize(static_cast<size_t>(total) * sys->esize);
        CUDA_TRY(cudaSetDevice(sys->ctx->device));
        (void)cudaGetLastError();   // an earlier call's error is not this call's
        CUDA_TRY(cudaStreamSynchronize(sys->stream));
        CUDA_TRY(cudaMemcpy(buf.data(), phi_dev, buf.size(), cudaMemcpyDeviceToHost));
    }
    FileCloser fc{std::fopen(path, "wb")};
    if (!fc.f) return fail(LSW_ERR_IO, "lsw_save: cannot open %s", path);
    const int32_t version = 1, na = sys->n_atoms;
    const int32_t prec = sys->zsplit ? LSW_FP32_BF16X : sys->prec, zs = sys->zsplit;
    const double h = sys->h, margin = sys->margin, cutoff = sys->cutoff;
    const int32_t pm = sys->pair_mode, fm = sys->fine_mode;
    const int64_t has = phi_dev ? 1 : 0;
    const bool ok = put(fc.f, kSaveMagic, 8) && put(fc.f, &version, 1) && put(fc.f, sys->N, 3) && put(fc.f, &h, 1) &&
                    put(fc.f, &na, 1) && put(fc.f, &margin, 1) && put(fc.f, &cutoff, 1) && put(fc.f, &pm, 1) &&
                    put(fc.f, &fm, 1) && put(fc.f, &prec, 1) && put(fc.f, &zs, 1) &&
                    put(fc.f, sys->pos.data(), sys->pos.size()) && put(fc.f, sys->r_loc.data(), sys->r_loc.size()) &&
                    put(fc.f, sys->r_fine.data(), sys->r_fine.size()) && put(fc.f, sys->nsf.data(), sys->nsf.size()) &&
                    put(fc.f, &total, 1) && put(fc.f, &has, 1) && put(fc.f, buf.data(), buf.size());
    if (!ok || std::fflush(fc.f) != 0) return fail(LSW_ERR_IO, "lsw_save: write to %s failed", path);
    return LSW_OK;
}

lsw_status lsw_load(lsw_ctx ctx, const char* path, lsw_system* out, void* phi_dev) {
    g_err.clear();
    if (!ctx || !path || !out) return fail(LSW_ERR_ARG, "lsw_load: NULL argument");
    *out = nullptr;
    FileCloser fc{std::fopen(path, "rb")};
    if (!fc.f) return fail(LSW_ERR_IO, "lsw_load: cannot open %s", path);
    lsw_system_desc d;
    std::vector<double> pos, rl, rf;
    std::vector<int32_t> nsf;
    int32_t zs = 0;
    lsw_status e = read_desc(fc.f, path, &d, pos, rl, rf, nsf, &zs);
    if (e != LSW_OK) return e;
    lsw_system s = nullptr;
    if ((e = lsw_system_create(ctx, &d, &s)) != LSW_OK) return e;
    if (zs == 3 && s->zsplit && !ctx->host_only) {
        if ((e = lsw_set_option(s, "zsplit", 3)) != LSW_OK) {
            lsw_system_destroy(s);
            return e;
        }
    } else if (zs == 3) {
        s->zsplit = 3;
    }
    if ((e = read_phi(fc.f, path, s, phi_dev)) != LSW_OK) {
        const std::string msg = g_err;
        lsw_system_destroy(s);
        return fail(e, "%s", msg.c_str());
    }
    *out = s;
    return LSW_OK;
}

lsw_status lsw_load_phi(lsw_system sys, const char* path, void* phi_dev) {
    g_err.clear();
    if (!sys || !path || !phi_dev) return fail(LSW_ERR_ARG, "lsw_load_phi: NULL argument");
    FileCloser fc{std::fopen(path, "rb")};
    if (!fc.f) return fail(LSW_ERR_IO, "lsw_load: cannot open %s", path);
    lsw_system_desc d;
    std::vector<double> pos, rl, rf;
    std::vector<int32_t> nsf;
    int32_t zs = 0;
    lsw_status e = read_desc(fc.f, path, &d, pos, rl, rf, nsf, &zs);
    if (e != LSW_OK) return e;
    if (d.n_atoms != sys->n_atoms) return fail(LSW_ERR_STATE, "lsw_load_phi: %s holds another system", path);
    return read_phi(fc.f, path, sys, phi_dev);
}

}  // extern "C"
