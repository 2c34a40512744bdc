// Runtime and C ABI of the library (declared in include/lbm.h): context,
// parameter validation, device buffers, batch work-list, CUDA-graph replay of
// time steps, tile autotuning, read-out and checkpoints.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/lbm.h"
#include "lbm_launch.h"
#include "lbm_step.cuh"

using namespace lbm;

namespace {

thread_local std::string g_last_error;

// NVTX range over one API call (shows up in Nsight Systems / Compute
// timelines; free when no tool is attached)
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                        \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

constexpr double kCs2 = 1.0 / 3.0;
constexpr int kGraphChunk = 32;  // steps per captured graph (even: parity is preserved)
constexpr uint32_t kStateMagic = 0x4c424d31u;  // "LBM1"
// staging of the init and read-out kernels (lattices are staged a group at
// a time): nodes per field and FP64 psi cells
constexpr long long kStageNodes = 1LL << 24;
constexpr long long kStageCells = 1LL << 25;
// blob kind word: the precision, LBM_INPLACE for in-place storage, and
// kBlobSwapped when an in-place state was saved in the swapped layout
constexpr uint32_t kBlobSwapped = 0x10000u;

struct HostLattice {
    lbm_lattice_desc desc;       // wall_mask pointer not kept
    std::vector<uint8_t> mask;   // nx*ny, empty if none
    Geom geom;
    double rho_ref;              // as used by the kernels (FP32-rounded for FP32_DEV)
    bool rho_ref_auto;
    long long n_fluid;
    long long c_off;             // element offset in the compact checkpoint layout
    std::vector<uint8_t> halo_mask;  // open in x: mask columns -2, -1, nx, nx + 1 (ny each)
};

}  // namespace

namespace lbm {
// Record an error message for lbm_last_error() from another translation unit.
int report_error(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace lbm

struct lbm_ctx {
    int n = 0;
    int precision = LBM_FP32_DEV;
    size_t elem = 4;
    std::vector<HostLattice> lats;
    long long total_nodes = 0, fluid_nodes = 0;
    long long total_elems = 0;   // elements per distribution array
    long long compact_elems = 0; // elements of the distribution in a checkpoint blob
    long long mask_bytes = 0;
    long long max_nodes = 0;

    void* f[2] = {nullptr, nullptr};
    int cur = 0;                 // buffer holding the state read by the next step
    // in-place storage: one distribution array (f[1] == f[0]); cur is the
    // layout of the state, 0 natural, 1 swapped (kLayoutNatural/Swapped)
    bool inplace = false;
    // the two distribution arrays exceed L2, so every step streams from DRAM:
    // the plain kernel then prefetches later tiles into L2 (StepArgs::ahead)
    bool streams_dram = false;
    uint8_t* d_mask = nullptr;
    Geom* d_geom = nullptr;
    Phys<float>* d_phys_f = nullptr;
    Phys<double>* d_phys_d = nullptr;
    Tile* d_tiles = nullptr;
    int n_tiles = 0;             // tiles of the plain kernel
    int n_edge = 0;              // the first n_edge of them: within two cells of an open x edge
    int part_done = 0;           // parts of a split step (lbm_step_part) launched so far
    // pipelined variants: the full wall-free tiles go to the persistent kernel
    // (d_fast, n_fast, pipe_grid CTAs), the rest (d_tiles) to the plain kernel
    // of the same node tile; TMA variants take the tiles two cells or more
    // from every lattice edge (d_tma, n_tma), the plain kernel the rest
    TileGeom* d_tgeo = nullptr;  // d_tiles with their lattices' geometry (plain kernel)
    FastTile* d_fast = nullptr;
    int n_fast = 0;
    int pipe_grid = 0;
    Tile* d_tma = nullptr;
    int n_tma = 0;
    // the plain kernel's list as a regular grid (tiles_x > 0), so that its
    // FP32 shapes of four nodes per thread find tiles without loading their
    // records (tile_at)
    TileGrid grid{};
    // TMA variants: tensor maps per variant (box shape) and source buffer,
    // encoded once and passed to every launch as kernel parameters.
    static constexpr int kMaxTma = 8;
    TmaMaps* h_maps[kMaxTma][2] = {};   // host copies passed at launch, by source buffer
    int tma_grid[kMaxTma] = {};
    // Clock cycles a TMA-variant mbarrier wait may take (about one second),
    // and bytes added to every stage's expected count (0). The environment
    // variables LBM_TMA_WAIT_CYCLES and LBM_TMA_EXTRA_TX, read when the context
    // is created, override them: a test sets a short limit and a few extra
    // bytes, so that the waits run out (their phase never completes, while
    // every copy does land) and the step reports LBM_ETIMEOUT without a fault.
    long long tma_wait_limit = 2000000000LL;
    unsigned tma_extra_tx = 0;
    // LBM_FAIL_ALLOC_AT=k (read at creation) makes the k-th device allocation
    // of the context fail as if the device were out of memory, so that a test
    // can check the error path and the clean-up without exhausting a GPU
    long long fail_alloc_at = 0, alloc_count = 0;
    int tile_index = 0;
    unsigned* d_status = nullptr;
    double* d_partials = nullptr;
    double* d_scalar = nullptr;
    // staging of the init and read-out kernels, for a group of lattices at a
    // time: d_io holds 4 fields of stage_nodes doubles, d_psi stage_cells
    // FP64 psi cells (the read-out's plane); in-place storage also keeps the
    // step's psi planes of every lattice in d_psi
    double* d_io = nullptr;
    double* d_psi = nullptr;
    long long stage_nodes = 0, stage_cells = 0;
    // per-lattice invalid-input flags of the init kernel: page-locked host
    // memory that the kernel writes through its mapped address (m_bad); a
    // flag equal to bad_gen was set by the current init call
    unsigned* h_bad = nullptr;
    unsigned* h_status = nullptr;  // page-locked copy of d_status (read_status)
    unsigned* m_bad = nullptr;
    unsigned bad_gen = 0;
    std::vector<Phys<double>> phys_d;
    PhysTable<float>* h_table = nullptr;  // FP32 parameters as a kernel argument (n <= kParamLattices)
    size_t device_bytes = 0;

    cudaStream_t stream = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // chunk graphs by starting buffer
    long long steps = 0;
    unsigned long long launches = 0;
};

namespace {

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

int validate_desc(const lbm_lattice_desc& d, int i) {
    if (d.nx < 1 || d.ny < 1) return fail(LBM_EINVAL, "lattice %d: nx=%d, ny=%d must be >= 1", i, d.nx, d.ny);
    long long plane = (long long)(d.ny + 2 * kGY) * round_up((long long)d.nx + kGX + 2, 32);
    if (9 * plane >= (1ll << 31))
        return fail(LBM_EINVAL, "lattice %d: %dx%d too large (9 stored planes must hold < 2^31 elements)", i,
                    d.nx, d.ny);
    const lbm_eos_params& e = d.eos;
    if (!(std::isfinite(e.a) && std::isfinite(e.b) && std::isfinite(e.R) && std::isfinite(e.T) &&
          std::isfinite(e.G)))
        return fail(LBM_EINVAL, "lattice %d: EOS parameters must be finite", i);
    if (e.kind < LBM_EOS_CS || e.kind > LBM_PSI_EXP) return fail(LBM_EINVAL, "lattice %d: unknown psi kind %d", i, e.kind);
    if (e.kind == LBM_PSI_EXP) {
        if (!(e.G != 0.0 && std::isfinite(e.G))) return fail(LBM_EINVAL, "lattice %d: G must be finite and nonzero", i);
        if (!(d.eps >= 0.0)) return fail(LBM_EINVAL, "lattice %d: eps must be >= 0 for psi of Eq. 12", i);
    } else {
        if (!(e.b > 0.0)) return fail(LBM_EINVAL, "lattice %d: b must be > 0", i);
        if (!(e.G < 0.0)) return fail(LBM_EINVAL, "lattice %d: G must be < 0 for psi of Eq. 13", i);
        if (!(e.R * e.T >= 0.0)) return fail(LBM_EINVAL, "lattice %d: R*T must be >= 0", i);
        if (e.kind == LBM_EOS_PR && !(e.a > 0.0 && e.R > 0.0 && e.T >= 0.0 && std::isfinite(e.omega)))
            return fail(LBM_EINVAL, "lattice %d: Peng-Robinson needs a > 0, R > 0, T >= 0, finite omega", i);
    }
    for (int k = 0; k < 9; ++k)
        if (!(d.s[k] >= 0.0 && d.s[k] < 2.0))
            return fail(LBM_EINVAL, "lattice %d: relaxation rate s[%d]=%g outside [0, 2)", i, k, d.s[k]);
    if (!std::isfinite(d.eps)) return fail(LBM_EINVAL, "lattice %d: eps must be finite", i);
    if (!std::isfinite(d.rho_ref)) return fail(LBM_EINVAL, "lattice %d: rho_ref must be finite", i);
    return LBM_OK;
}

void fill_phys(const HostLattice& L, Phys<double>& P) {
    const lbm_lattice_desc& d = L.desc;
    P.rho_ref = L.rho_ref;
    P.RT = d.eos.R * d.eos.T;
    P.a = d.eos.a;
    P.b4 = d.eos.b / 4.0;
    P.G = d.eos.G;
    P.kpsi = 2.0 / d.eos.G;  // c = 1
    P.cs2 = kCs2;
    for (int k = 0; k < 9; ++k) {
        P.s[k] = d.s[k];
        P.h[k] = 1.0 - 0.5 * d.s[k];
    }
    P.li_e = d.s[1] * 0.75 * d.eps;
    P.li_z = d.s[2] * 0.75 * d.eps;
    P.eos = d.eos.kind;
    P.b1 = d.eos.b;
    // Eq. 12's exponent is the mechanical-stability eps that Li's forcing
    // with this lattice's eps produces, -G eps (Li et al. 2013; = eps at the
    // paper's G = -1), so that psi'/psi^(1+e) = 1/rho^2 holds for the model
    const double e12 = -d.eos.G * d.eps;
    P.eps12 = e12;
    P.inv_eps12 = e12 != 0.0 ? 1.0 / e12 : 0.0;
    if (d.eos.kind == LBM_EOS_PR) {
        // a alpha(T): Tc from a = 0.45724 R^2 Tc^2 / pc and b = 0.0778 R Tc / pc
        const double Tc = 0.0778 * d.eos.a / (0.45724 * d.eos.b * d.eos.R);
        const double k = 0.37464 + 1.54226 * d.eos.omega - 0.26992 * d.eos.omega * d.eos.omega;
        const double s = 1.0 + k * (1.0 - std::sqrt(d.eos.T / Tc));
        P.a = d.eos.a * s * s;
    }
}

void to_float(const Phys<double>& D, Phys<float>& F) {
    F.rho_ref = (float)D.rho_ref;
    F.RT = (float)D.RT;
    F.a = (float)D.a;
    F.b4 = (float)D.b4;
    F.G = (float)D.G;
    F.kpsi = (float)D.kpsi;
    F.cs2 = (float)D.cs2;
    for (int k = 0; k < 9; ++k) {
        F.s[k] = (float)D.s[k];
        F.h[k] = (float)D.h[k];
    }
    F.li_e = (float)D.li_e;
    F.li_z = (float)D.li_z;
    F.b1 = (float)D.b1;
    F.eps12 = (float)D.eps12;
    F.inv_eps12 = (float)D.inv_eps12;
    F.eos = D.eos;
}

template <typename P>
int dev_alloc(lbm_ctx* c, P** ptr, size_t bytes) {
    if (c->fail_alloc_at > 0 && ++c->alloc_count == c->fail_alloc_at) {  // injected failure (tests)
        *ptr = nullptr;
        return fail(LBM_ENOMEM, "cudaMalloc(%zu bytes): injected failure (LBM_FAIL_ALLOC_AT)", bytes);
    }
    cudaError_t e = cudaMalloc((void**)ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return fail(LBM_ENOMEM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    c->device_bytes += bytes;
    return LBM_OK;
}

void drop_graphs(lbm_ctx* c) {
    for (auto& g : c->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

void free_ctx(lbm_ctx* c) {
    if (!c) return;
    drop_graphs(c);
    cudaFree(c->f[0]);
    if (c->f[1] != c->f[0]) cudaFree(c->f[1]);
    cudaFree(c->d_mask);
    cudaFree(c->d_geom);
    cudaFree(c->d_phys_f);
    cudaFree(c->d_phys_d);
    cudaFree(c->d_tiles);
    delete c->h_table;
    for (int v = 0; v < lbm_ctx::kMaxTma; ++v)
        for (int b = 0; b < 2; ++b) delete c->h_maps[v][b];
    cudaFree(c->d_fast);
    cudaFree(c->d_tma);
    cudaFree(c->d_tgeo);
    cudaFree(c->d_status);
    cudaFree(c->d_partials);
    cudaFree(c->d_scalar);
    cudaFree(c->d_io);
    cudaFree(c->d_psi);
    cudaFreeHost(c->h_bad);
    cudaFreeHost(c->h_status);
    delete c;
}

int total_tiles() { return kTileCount + tma_variant_count() + pipe_variant_count(); }
int pipe_first() { return kTileCount + tma_variant_count(); }
bool is_tma(int index) { return index >= kTileCount && index < pipe_first(); }
bool is_pipe(int index) { return index >= pipe_first(); }

void tile_shape(int index, int* tx, int* ty) {
    if (index < kTileCount) {
        *tx = kTiles[index][0];
        *ty = kTiles[index][1] * kTiles[index][2];
    } else if (is_tma(index)) {
        tma_variant_shape(index - kTileCount, tx, ty);
    } else {
        pipe_variant_shape(index - pipe_first(), tx, ty);
    }
}

// layout of the stored state (the step kernels' and read-outs' view of it)
int state_layout(const lbm_ctx* c) {
    if (!c->inplace) return kLayoutPull;
    return c->cur == 0 ? kLayoutNatural : kLayoutSwapped;
}

// kernel launches of one step with the current tile list
int launches_per_step(const lbm_ctx* c) {
    if (c->inplace) return 2;
    if (is_pipe(c->tile_index)) return (c->n_fast > 0 ? 1 : 0) + (c->n_tiles > 0 ? 1 : 0);
    if (is_tma(c->tile_index)) return (c->n_tma > 0 ? 1 : 0) + (c->n_tiles > 0 ? 1 : 0);
    return 1;
}

// Tensor maps for a TMA variant's box shape (built once per context and
// variant), and its persistent grid size.
int build_tma(lbm_ctx* c, int tile_index) {
    const int v = tile_index - kTileCount;
    if (v < 0 || v >= lbm_ctx::kMaxTma) return fail(LBM_EINVAL, "no TMA variant %d", tile_index);
    if (c->n > kTmaMaxLattices)
        return fail(LBM_EINVAL, "tile %d (TMA) takes batches of at most %d lattices", tile_index, kTmaMaxLattices);
    if (c->h_maps[v][0] == nullptr) {
        int tx = 0, ty = 0;
        tile_shape(tile_index, &tx, &ty);
        TmaMaps* m0 = new TmaMaps();
        TmaMaps* m1 = new TmaMaps();
        memset(m0, 0, sizeof(TmaMaps));
        memset(m1, 0, sizeof(TmaMaps));
        for (int l = 0; l < c->n; ++l) {
            CUtensorMap fm[2];
            if (!encode_lattice_maps(c->lats[l].geom, tx, ty, (const float*)c->f[0], (const float*)c->f[1],
                                     c->d_mask, fm, &m0->m[l])) {
                delete m0;
                delete m1;
                return fail(LBM_ECUDA, "cuTensorMapEncodeTiled failed for lattice %d", l);
            }
            m0->f[l] = fm[0];
            m1->f[l] = fm[1];
            m1->m[l] = m0->m[l];
        }
        c->h_maps[v][0] = m0;
        c->h_maps[v][1] = m1;
    }
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int per_sm = tma_blocks_per_sm(v);
    if (per_sm < 1) return fail(LBM_ECUDA, "TMA step variant %d cannot be resident on this device", tile_index);
    c->tma_grid[v] = std::min(c->n_tma, per_sm * sms);
    return LBM_OK;
}

// The plain kernel's list as a regular grid of tx x ty tiles, if it is one:
// every lattice with the same size and layout, no wall mask, not open in x,
// covered by whole tiles, lattices evenly spaced in the distribution arrays,
// and the list equal to the grid's order entry by entry (lattice by lattice,
// row by row). Otherwise tiles_x = 0.
TileGrid regular_grid(const lbm_ctx* c, const std::vector<Tile>& tiles, int tx, int ty) {
    TileGrid none{};
    if (c->n < 1) return none;
    const Geom& g0 = c->lats[0].geom;
    if (g0.nx % tx != 0 || g0.ny % ty != 0 || g0.flags != 0) return none;
    const long long stride = c->n > 1 ? c->lats[1].geom.f_off - g0.f_off : 0;
    for (int l = 0; l < c->n; ++l) {
        const Geom& g = c->lats[l].geom;
        if (g.nx != g0.nx || g.ny != g0.ny || g.pitch != g0.pitch || g.plane != g0.plane || g.flags != 0 ||
            g.f_off != g0.f_off + (long long)l * stride)
            return none;
    }
    const int tiles_x = g0.nx / tx, per_lat = tiles_x * (g0.ny / ty);
    if ((long long)per_lat * c->n != (long long)tiles.size()) return none;
    for (size_t k = 0; k < tiles.size(); ++k) {
        const int lat = (int)(k / per_lat), r = (int)(k % per_lat);
        const Tile& t = tiles[k];
        if (t.lat != lat || t.x0 != (r % tiles_x) * tx || t.y0 != (r / tiles_x) * ty || t.clear != 1) return none;
    }
    TileGrid grid{tiles_x, per_lat, stride, g0, 0, 0, 0, 0};
    div_magic_of(per_lat, &grid.m_lat, &grid.s_lat);
    div_magic_of(tiles_x, &grid.m_x, &grid.s_x);
    return grid;
}

// Work-lists of one step: every tile of every lattice, lattices in creation
// order, tiles row-major within a lattice (in the plain kernel's list, the
// tiles of its general path come first). The pipelined variants take the
// full wall-free Carnahan-Starling tiles, the TMA variants the tiles two
// cells or more from every edge of their lattice; the plain kernel of the
// same node tile takes the rest.
int build_tiles(lbm_ctx* c, int tile_index) {
    if (tile_index < 0 || tile_index >= total_tiles()) return fail(LBM_EINVAL, "no tile shape %d", tile_index);
    if (tile_index >= kTileCount && c->precision == LBM_FP64)
        return fail(LBM_EINVAL, "tile %d is an FP32-only variant; this context stores FP64", tile_index);
    if (tile_index >= kTileCount && c->inplace)
        return fail(LBM_EINVAL, "tile %d is a two-buffer variant; this context stores in place", tile_index);
    if (is_tma(tile_index) && c->n > kTmaMaxLattices)  // refused before the current tile list is replaced
        return fail(LBM_EINVAL, "tile %d (TMA) takes batches of at most %d lattices", tile_index, kTmaMaxLattices);
    const bool pipe = is_pipe(tile_index), tma = is_tma(tile_index);
    int tx = 0, ty = 0;
    tile_shape(tile_index, &tx, &ty);
    std::vector<Tile> tiles, inner_tiles;
    std::vector<FastTile> fast;
    for (int l = 0; l < c->n; ++l) {
        const HostLattice& L = c->lats[l];
        const Geom& g = L.geom;
        // solid cells of the periodic lattice summed over rectangles: a tile
        // whose cells and two-cell frame hold none takes the wall-free paths
        const int ex = g.nx + 4, ey = g.ny + 4;
        std::vector<int> sat;
        if (geom_mask(g)) {
            sat.assign((size_t)(ex + 1) * (ey + 1), 0);
            for (int j = 0; j < ey; ++j)
                for (int i = 0; i < ex; ++i) {
                    const int xs = ((i - 2) % g.nx + g.nx) % g.nx, ys = ((j - 2) % g.ny + g.ny) % g.ny;
                    sat[(size_t)(j + 1) * (ex + 1) + i + 1] = L.mask[(size_t)ys * g.nx + xs] +
                                                              sat[(size_t)j * (ex + 1) + i + 1] +
                                                              sat[(size_t)(j + 1) * (ex + 1) + i] -
                                                              sat[(size_t)j * (ex + 1) + i];
                }
        }
        for (int y0 = 0; y0 < g.ny; y0 += ty)
            for (int x0 = 0; x0 < g.nx; x0 += tx) {
                const bool full = x0 + tx <= g.nx && y0 + ty <= g.ny;
                bool clear = !geom_mask(g);
                if (geom_mask(g) && full) {  // frame [x0 - 2, x0 + tx + 2) x [y0 - 2, y0 + ty + 2)
                    const int i0 = x0, i1 = x0 + tx + 4, j0 = y0, j1 = y0 + ty + 4;
                    const int n = sat[(size_t)j1 * (ex + 1) + i1] - sat[(size_t)j0 * (ex + 1) + i1] -
                                  sat[(size_t)j1 * (ex + 1) + i0] + sat[(size_t)j0 * (ex + 1) + i0];
                    clear = n == 0;
                }
                // an x-slab's tiles within two cells of its x edges pull from
                // the frame (the halo): the general path, which does not wrap
                if (geom_open_x(g) && (x0 < 2 || x0 + tx > g.nx - 2)) clear = false;
                // no pull of the tile or of its halo ring crosses an edge
                const bool inner = x0 >= 2 && x0 + tx <= g.nx - 2 && y0 >= 2 && y0 + ty <= g.ny - 2;
                if (pipe && clear && full && g.nx >= 4 && g.ny >= 4 && L.desc.eos.kind == LBM_EOS_CS)
                    fast.push_back(
                        FastTile{g.f_off, (int)g.plane, g.pitch, g.nx, g.ny, l, x0, y0, inner ? 0 : 1, {0, 0}});
                else if (tma && inner)
                    inner_tiles.push_back(Tile{l, x0, y0, clear ? 1 : 0});
                else
                    tiles.push_back(Tile{l, x0, y0, clear ? 1 : 0});
            }
    }
    if (tiles.size() > (size_t)0x7fffffff || fast.size() > (size_t)0x7fffffff || inner_tiles.size() > (size_t)0x7fffffff)
        return fail(LBM_EINVAL, "too many tiles");
    // tiles that take the general path (walls nearby, partial tiles, other
    // EOS kinds, lattices under 4 x 4) run longer than fast-path tiles: put
    // them first, so that they start in the first wave instead of trailing
    // the last one (every tile is independent: the order changes no result)
    std::stable_partition(tiles.begin(), tiles.end(), [&](const Tile& t) {
        const Geom& g = c->lats[t.lat].geom;
        const bool full = t.x0 + tx <= g.nx && t.y0 + ty <= g.ny;
        const bool fast = t.clear && full && g.nx >= 4 && g.ny >= 4 && c->lats[t.lat].desc.eos.kind == LBM_EOS_CS;
        return !fast;
    });
    // the tiles within two cells of an open x edge (an x-slab's cuts) go
    // first of all: a split step (lbm_step_part) launches them apart, so
    // that the halo they feed can be exchanged while the rest runs
    auto open_edge = [&](const Tile& t) {
        const Geom& g = c->lats[t.lat].geom;
        return geom_open_x(g) && (t.x0 < 2 || t.x0 + tx > g.nx - 2);
    };
    std::stable_partition(tiles.begin(), tiles.end(), open_edge);
    const int n_edge = (int)std::count_if(tiles.begin(), tiles.end(), open_edge);
    std::vector<TileGeom> tgeo(tiles.size());
    for (size_t k = 0; k < tiles.size(); ++k) tgeo[k] = TileGeom{c->lats[tiles[k].lat].geom, tiles[k]};
    const TileGrid grid = regular_grid(c, tiles, tx, ty);
    Tile* d = nullptr;
    TileGeom* dg = nullptr;
    FastTile* df = nullptr;
    int rc = 0;
    if (!tiles.empty()) rc = dev_alloc(c, &d, tiles.size() * sizeof(Tile));
    if (!rc && !tiles.empty()) rc = dev_alloc(c, &dg, tgeo.size() * sizeof(TileGeom));
    if (!rc && !fast.empty()) rc = dev_alloc(c, &df, fast.size() * sizeof(FastTile));
    Tile* di = nullptr;
    if (!rc && !inner_tiles.empty()) rc = dev_alloc(c, &di, inner_tiles.size() * sizeof(Tile));
    if (rc) {
        if (d) {
            cudaFree(d);
            c->device_bytes -= tiles.size() * sizeof(Tile);
        }
        if (dg) {
            cudaFree(dg);
            c->device_bytes -= tgeo.size() * sizeof(TileGeom);
        }
        if (df) {
            cudaFree(df);
            c->device_bytes -= fast.size() * sizeof(FastTile);
        }
        return rc;
    }
    cudaError_t e = cudaSuccess;
    if (d) e = cudaMemcpy(d, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && dg) e = cudaMemcpy(dg, tgeo.data(), tgeo.size() * sizeof(TileGeom), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && df) e = cudaMemcpy(df, fast.data(), fast.size() * sizeof(FastTile), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && di)
        e = cudaMemcpy(di, inner_tiles.data(), inner_tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice);
    int per_sm = 0, sms = 0, dev = 0;
    if (e == cudaSuccess && pipe) {
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        per_sm = pipe_blocks_per_sm(tile_index - pipe_first(), c->n <= kParamLattices);
    }
    if (e != cudaSuccess || (pipe && per_sm < 1)) {
        cudaFree(d);
        cudaFree(dg);
        cudaFree(df);
        cudaFree(di);
        c->device_bytes -= tiles.size() * (sizeof(Tile) + sizeof(TileGeom)) + fast.size() * sizeof(FastTile) +
                           inner_tiles.size() * sizeof(Tile);
        return e != cudaSuccess ? cuda_fail(e, "tile list upload")
                                : fail(LBM_ECUDA, "pipelined variant %d cannot be resident on this device", tile_index);
    }
    if (c->d_tiles) {
        cudaFree(c->d_tiles);
        c->device_bytes -= (size_t)c->n_tiles * sizeof(Tile);
    }
    if (c->d_tgeo) {
        cudaFree(c->d_tgeo);
        c->device_bytes -= (size_t)c->n_tiles * sizeof(TileGeom);
    }
    if (c->d_fast) {
        cudaFree(c->d_fast);
        c->device_bytes -= (size_t)c->n_fast * sizeof(FastTile);
    }
    if (c->d_tma) {
        cudaFree(c->d_tma);
        c->device_bytes -= (size_t)c->n_tma * sizeof(Tile);
    }
    c->d_tiles = d;
    c->d_tgeo = dg;
    c->n_tiles = (int)tiles.size();
    c->n_edge = n_edge;
    c->d_fast = df;
    c->n_fast = (int)fast.size();
    c->pipe_grid = pipe ? (int)std::min<long long>(c->n_fast, (long long)per_sm * sms) : 0;
    c->d_tma = di;
    c->n_tma = (int)inner_tiles.size();
    c->grid = grid;
    c->tile_index = tile_index;
    drop_graphs(c);
    if (is_tma(tile_index)) return build_tma(c, tile_index);
    return LBM_OK;
}

// The mask plane of lattice l: its nodes, and in the frame their periodic
// images, or for a lattice open in x the halo mask columns x = -2, -1, nx,
// nx + 1 (rows wrap periodically in both cases).
cudaError_t upload_mask(lbm_ctx* c, int l) {
    const HostLattice& L = c->lats[l];
    if (L.mask.empty()) return cudaSuccess;
    const Geom& g = L.geom;
    std::vector<uint8_t> rows((size_t)g.plane, 0);
    for (int y = -kGY; y < g.ny + kGY; ++y)
        for (int x = -2; x < g.nx + 2; ++x) {
            const int ys = (int)(((long long)y % g.ny + g.ny) % g.ny);
            uint8_t v;
            if (geom_open_x(g) && (x < 0 || x >= g.nx)) {
                const int col = x < 0 ? x + 2 : x - g.nx + 2;  // -2, -1, nx, nx + 1 -> 0 .. 3
                v = L.halo_mask[(size_t)col * g.ny + ys];
            } else {
                const int xs = (int)(((long long)x % g.nx + g.nx) % g.nx);
                v = L.mask[(size_t)ys * g.nx + xs];
            }
            rows[(size_t)node_index(g, x, y)] = v;
        }
    return cudaMemcpy(c->d_mask + g.mask_off, rows.data(), rows.size(), cudaMemcpyHostToDevice);
}

bool any_open_x(const lbm_ctx* c) {
    for (const auto& L : c->lats)
        if (geom_open_x(L.geom)) return true;
    return false;
}

int upload_phys(lbm_ctx* c) {
    std::vector<Phys<float>> pf(c->n);
    for (int l = 0; l < c->n; ++l) {
        fill_phys(c->lats[l], c->phys_d[l]);
        to_float(c->phys_d[l], pf[l]);
    }
    CK(cudaMemcpy(c->d_phys_d, c->phys_d.data(), c->n * sizeof(Phys<double>), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_phys_f, pf.data(), c->n * sizeof(Phys<float>), cudaMemcpyHostToDevice));
    if (c->n <= kParamLattices) {
        if (!c->h_table) c->h_table = new PhysTable<float>();
        memset(c->h_table, 0, sizeof(PhysTable<float>));
        for (int l = 0; l < c->n; ++l) c->h_table->p[l] = pf[l];
    }
    return LBM_OK;
}

// One step launch from buffer `src` into buffer 1 - src.
LaunchSet launch_set(lbm_ctx* c, int lat0, int n_lat) {
    long long mx = 0, me = 0;
    for (int l = lat0; l < lat0 + n_lat; ++l) {
        const Geom& g = c->lats[l].geom;
        mx = std::max(mx, (long long)g.nx * g.ny);
        me = std::max(me, (long long)g.nx + g.ny);
    }
    return LaunchSet{c->d_geom, c->d_phys_d, c->d_mask, lat0, n_lat, mx, me, state_layout(c)};
}

// Parts of a time step: every tile, the tiles within two cells of an open
// x edge (the first n_edge of the plain list), or all the others.
constexpr int kPartAll = 3;
constexpr int kPartEdge = LBM_STEP_EDGE;
constexpr int kPartInterior = LBM_STEP_INTERIOR;

// One step launch (or one part of it) from buffer `src` into buffer 1 - src.
cudaError_t launch_one_step(lbm_ctx* c, int src, int part = kPartAll) {
    cudaError_t e = cudaSuccess;
    if (c->inplace) {
        if (!(part & kPartInterior)) return cudaSuccess;  // in place holds no open lattice: no edge part
        int tx = 0, ty = 0;
        tile_shape(c->tile_index, &tx, &ty);
        const int layout = src == 0 ? kLayoutNatural : kLayoutSwapped;
        if (c->precision == LBM_FP64)
            e = launch_step_inplace_f64(c->d_tgeo, c->n_tiles, tx, ty, c->d_phys_d, (double*)c->f[0], c->d_mask,
                                        c->d_psi, c->d_status, layout, c->stream);
        else
            e = launch_step_inplace_f32(c->d_tgeo, c->n_tiles, tx, ty, c->d_phys_f, (float*)c->f[0], c->d_mask,
                                        (float*)c->d_psi, c->d_status, layout, c->stream);
        return e;
    }
    // the plain kernel's share of this part: [first, first + count) of its list
    const int first = part == kPartInterior ? c->n_edge : 0;
    const int count = part == kPartEdge ? c->n_edge : (part == kPartInterior ? c->n_tiles - c->n_edge : c->n_tiles);
    const bool open = any_open_x(c);
    // the launch takes the plain kernel's whole list, in order
    const bool whole_list = first == 0 && count == c->n_tiles;
    if (c->precision == LBM_FP64) {
        StepArgs<double> a{c->d_tiles + first, c->d_geom, c->d_phys_d, (const double*)c->f[src],
                           (double*)c->f[1 - src], c->d_mask, c->d_status, c->d_tgeo + first, 0};
        return launch_step_f64(c->tile_index, count, a, c->stream, open);
    }
    StepArgs<float> a{c->d_tiles + first, c->d_geom, c->d_phys_f, (const float*)c->f[src], (float*)c->f[1 - src],
                      c->d_mask, c->d_status, c->d_tgeo + first, c->streams_dram ? 1 : 0};
    const TileGrid grid = whole_list && c->tile_index < kTileCount ? c->grid : TileGrid{};
    int plain_shape = c->tile_index;
    if (is_pipe(c->tile_index)) {
        const int v = c->tile_index - pipe_first();
        plain_shape = pipe_plain_partner(v);
        if (part & kPartInterior) {  // the persistent kernel's tiles are all interior
            const PhysTable<float>* table = c->n <= kParamLattices ? c->h_table : nullptr;
            PipeArgs pa{c->d_fast, c->n_fast, c->d_phys_f, (const float*)c->f[src], (float*)c->f[1 - src],
                        c->d_status};
            e = launch_step_pipe(v, c->pipe_grid, pa, table, c->stream);
        }
    } else if (c->tile_index >= kTileCount) {
        const int v = c->tile_index - kTileCount;
        plain_shape = tma_plain_partner(v);
        if (part & kPartInterior) {  // as are the TMA kernel's
            TmaArgs ta{c->d_tma, c->n_tma, c->d_geom, c->d_phys_f, (float*)c->f[1 - src], c->d_status,
                       c->tma_wait_limit, c->tma_extra_tx};
            e = launch_step_tma(v, c->tma_grid[v], ta, *c->h_maps[v][src], *c->h_table, c->stream);
        }
    }
    if (e == cudaSuccess && count > 0) e = launch_step_f32(plain_shape, count, a, c->h_table, grid, c->stream, open);
    return e;
}

bool capturable_stream(cudaStream_t s) {
    return s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
}

int ensure_graph(lbm_ctx* c, int src) {
    if (c->graph[src]) return LBM_OK;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < kGraphChunk && le == cudaSuccess; ++k) le = launch_one_step(c, (src + k) & 1);
    cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(le, "step launch during graph capture");
    }
    if (ee != cudaSuccess) return cuda_fail(ee, "cudaStreamEndCapture");
    cudaError_t ie = cudaGraphInstantiate(&c->graph[src], g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        c->graph[src] = nullptr;
        return cuda_fail(ie, "cudaGraphInstantiate");
    }
    return LBM_OK;
}

// Calls that replace the state or the tile lists wait for a split step's
// second part.
int check_whole_step(lbm_ctx* c, const char* what) {
    if (c->part_done) return fail(LBM_EINVAL, "%s: a split step (lbm_step_part) is half done", what);
    return LBM_OK;
}

int check_lat(lbm_ctx* c, int lat) {
    if (!c) return fail(LBM_EINVAL, "null context");
    if (lat < 0 || lat >= c->n) return fail(LBM_EINVAL, "lattice index %d outside [0, %d)", lat, c->n);
    return LBM_OK;
}

int status_code(unsigned flags) {
    if (flags & FLAG_TIMEOUT) return fail(LBM_ETIMEOUT, "a device-side wait of the step kernel gave up");
    if (flags & FLAG_NONFINITE) return fail(LBM_ENONFINITE, "a density or psi^2 became non-finite");
    if (flags & FLAG_PSI_CLAMPED)
        return fail(LBM_EPSI_DOMAIN, "psi^2 of Eq. 13 went negative and was clamped to 0");
    return LBM_OK;
}

// The status words after everything enqueued so far: one copy into
// page-locked memory and one synchronisation, which also completes the
// caller's own copies enqueued before (the read-outs rely on it).
int read_status(lbm_ctx* c, std::vector<unsigned>& out) {
    CK(cudaMemcpyAsync(c->h_status, c->d_status, c->n * sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    out.assign(c->h_status, c->h_status + c->n);
    return LBM_OK;
}

// Resolve an automatic FP32 deviation reference (the minimum density over
// fluid nodes) from lattice `lat`'s host field; the inputs themselves are
// validated on the device by the init kernel.
int resolve_rho_ref(lbm_ctx* c, int lat, const double* rho, bool* phys_changed) {
    HostLattice& L = c->lats[lat];
    if (!(c->precision == LBM_FP32_DEV && L.rho_ref_auto)) return LBM_OK;
    const long long n = (long long)L.geom.nx * L.geom.ny;
    const uint8_t* m = L.mask.empty() ? nullptr : L.mask.data();
    double rmin = HUGE_VAL;
    for (long long i = 0; i < n; ++i) {
        if (m && m[i]) continue;
        if (!(std::isfinite(rho[i]) && rho[i] > 0.0))
            return fail(LBM_EINVAL, "lattice %d: rho[%lld]=%g must be finite and > 0", lat, i, rho[i]);
        rmin = std::min(rmin, rho[i]);
    }
    L.rho_ref = std::isfinite(rmin) ? (double)(float)rmin : 0.0;
    L.rho_ref_auto = false;
    *phys_changed = true;
    return LBM_OK;
}


long long range_nodes(lbm_ctx* c, int lat0, int n_lat) {
    const Geom& last = c->lats[lat0 + n_lat - 1].geom;
    return last.node_off + (long long)last.nx * last.ny - c->lats[lat0].geom.node_off;
}

// First psi cell of lattice l in a plane that covers every lattice (the
// kernels place lattice l's plane at f_off / 9), and one past its last.
long long cell_lo(const lbm_ctx* c, int l) { return c->lats[l].geom.f_off / 9; }
long long cell_hi(const lbm_ctx* c, int l) { return c->lats[l].geom.f_off / 9 + c->lats[l].geom.plane; }

// End of the group of lattices starting at `l0` (at most `end`) whose nodes
// and psi cells fit the staging buffers; every lattice fits on its own.
int group_end(const lbm_ctx* c, int l0, int end) {
    int l1 = l0 + 1;
    while (l1 < end && range_nodes(const_cast<lbm_ctx*>(c), l0, l1 + 1 - l0) <= c->stage_nodes &&
           cell_hi(c, l1) - cell_lo(c, l0) <= c->stage_cells)
        ++l1;
    return l1;
}

// A staging array holding the group that starts at node `nodes` (cells:
// psi cell `cells`), shifted so that the kernels index it by geom.node_off
// (geom.f_off / 9).
template <typename P>
P* cell_base(P* p, long long cells) {
    return p ? (P*)((uintptr_t)p - (uintptr_t)(cells * (long long)sizeof(double))) : nullptr;
}

// Initial state of lattices [lat0, lat0 + n_lat) from host arrays that start
// at lattice lat0's first node: one upload per field, one kernel launch.
// Device address under which kernels reach a page-locked, mapped host
// buffer (memory from cudaHostAlloc / cudaHostRegister, e.g. a pinned torch
// tensor), or null for pageable memory. The density read-out writes such a
// buffer directly over the host link, with no staging copy.
const void* mapped_device_ptr(const void* p) {
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// `p` shifted back by `nodes` doubles: the base the kernels index by
// geom.node_off when `p` holds the range starting at node `nodes`
template <typename P>
P* node_base(P* p, long long nodes) {
    return p ? (P*)((uintptr_t)p - (uintptr_t)(nodes * (long long)sizeof(double))) : nullptr;
}

int init_range(lbm_ctx* c, int lat0, int n_lat, const double* rho, const double* ux, const double* uy) {
    bool changed = false;
    for (int l = lat0; l < lat0 + n_lat; ++l) {
        const long long o = c->lats[l].geom.node_off - c->lats[lat0].geom.node_off;
        int rc = resolve_rho_ref(c, l, rho + o, &changed);
        if (rc) return rc;
    }
    if (changed) {
        int rc = upload_phys(c);
        if (rc) return rc;
        drop_graphs(c);
    }
    // staged through the device buffer d_io, a group of lattices at a time:
    // a bulk copy, then the init kernel (faster than the kernel reading a
    // mapped host buffer in place, whose scattered reads each pay the host
    // link's latency)
    if (++c->bad_gen == 0) c->bad_gen = 1;  // 0 is the value of a flag never set
    const long long base = c->lats[lat0].geom.node_off;
    const long long S = c->stage_nodes;
    for (int a = lat0; a < lat0 + n_lat;) {
        const int b = group_end(c, a, lat0 + n_lat);
        const long long gb = c->lats[a].geom.node_off;
        const size_t bytes = (size_t)range_nodes(c, a, b - a) * sizeof(double);
        const long long o = gb - base;
        CK(cudaMemcpyAsync(c->d_io, rho + o, bytes, cudaMemcpyHostToDevice, c->stream));
        if (ux) CK(cudaMemcpyAsync(c->d_io + S, ux + o, bytes, cudaMemcpyHostToDevice, c->stream));
        if (uy) CK(cudaMemcpyAsync(c->d_io + 2 * S, uy + o, bytes, cudaMemcpyHostToDevice, c->stream));
        const double* k_rho = node_base(c->d_io, gb);
        const double* k_ux = ux ? node_base(c->d_io + S, gb) : nullptr;
        const double* k_uy = uy ? node_base(c->d_io + 2 * S, gb) : nullptr;
        const LaunchSet ls = launch_set(c, a, b - a);
        cudaError_t e;
        if (c->precision == LBM_FP64)
            e = launch_init_f64(ls, k_rho, k_ux, k_uy, (double*)c->f[c->cur], c->m_bad, c->bad_gen, c->stream);
        else
            e = launch_init_f32(ls, k_rho, k_ux, k_uy, (float*)c->f[c->cur], c->m_bad, c->bad_gen, c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "init kernel");
        c->launches += 1;
        a = b;
    }
    // the host arrays may be pageable and the staging buffer is reused: wait,
    // then report invalid input found by the init kernel
    CK(cudaStreamSynchronize(c->stream));
    for (int l = lat0; l < lat0 + n_lat; ++l)
        if (c->h_bad[l] == c->bad_gen)
            return fail(LBM_EINVAL,
                        "lattice %d: a fluid density is not finite and > 0, or a velocity is not finite "
                        "(the lattice's state is undefined until the next successful init)", l);
    return LBM_OK;
}

// Initial state of lattice `lat`, open in x, from host arrays of
// (nx + 2) x ny values (the neighbouring slabs' edge columns included),
// through a temporary device buffer.
int init_open(lbm_ctx* c, int lat, const double* rho, const double* ux, const double* uy) {
    HostLattice& L = c->lats[lat];
    const Geom& g = L.geom;
    const size_t n = (size_t)(g.nx + 2) * g.ny;
    const int nf = 1 + (ux ? 1 : 0) + (uy ? 1 : 0);
    double* d = nullptr;
    int rc = dev_alloc(c, &d, (size_t)nf * n * sizeof(double));
    if (rc) return rc;
    double* d_rho = d;
    double* d_ux = ux ? d + n : nullptr;
    double* d_uy = uy ? d + (ux ? 2 : 1) * n : nullptr;
    cudaError_t e = cudaMemcpyAsync(d_rho, rho, n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && ux) e = cudaMemcpyAsync(d_ux, ux, n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && uy) e = cudaMemcpyAsync(d_uy, uy, n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (++c->bad_gen == 0) c->bad_gen = 1;
    if (e == cudaSuccess) {
        if (c->precision == LBM_FP64)
            e = launch_init_open_f64(g, L.rho_ref, d_rho, d_ux, d_uy, c->d_mask, (double*)c->f[c->cur], c->m_bad,
                                     lat, c->bad_gen, c->stream);
        else
            e = launch_init_open_f32(g, L.rho_ref, d_rho, d_ux, d_uy, c->d_mask, (float*)c->f[c->cur], c->m_bad,
                                     lat, c->bad_gen, c->stream);
        if (e == cudaSuccess) c->launches += 1;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    c->device_bytes -= (size_t)nf * n * sizeof(double);
    if (e != cudaSuccess) return cuda_fail(e, "open-lattice init");
    if (c->h_bad[lat] == c->bad_gen)
        return fail(LBM_EINVAL,
                    "lattice %d: a fluid density is not finite and > 0, or a velocity is not finite "
                    "(the lattice's state is undefined until the next successful init)", lat);
    return LBM_OK;
}

// rho, v, p of lattices [lat0, lat0 + n_lat) into host arrays that start at
// lattice lat0's first node: per group of lattices that fits the staging
// buffers, one or two kernel launches and one download per field (density
// alone into a page-locked, mapped host buffer: one launch, no staging).
// Enqueued only: the caller synchronises before it returns the arrays.
int moments_range(lbm_ctx* c, int lat0, int n_lat, double* rho, double* ux, double* uy, double* p) {
    const long long S = c->stage_nodes;
    const long long base = c->lats[lat0].geom.node_off;
    const bool density_only = !ux && !uy && !p;
    double* m_rho = (double*)mapped_device_ptr(rho);
    cudaError_t e;
    if (density_only && m_rho) {
        const LaunchSet ls = launch_set(c, lat0, n_lat);
        double* out = node_base(m_rho, base);
        e = c->precision == LBM_FP64 ? launch_density_f64(ls, (const double*)c->f[c->cur], out, c->stream)
                                     : launch_density_f32(ls, (const float*)c->f[c->cur], out, c->stream);
        c->launches += 1;
        if (e != cudaSuccess) return cuda_fail(e, "moments kernels");
        return LBM_OK;
    }
    double* h[4] = {rho, ux, uy, p};
    for (int a = lat0; a < lat0 + n_lat;) {
        const int b = group_end(c, a, lat0 + n_lat);
        const long long gb = c->lats[a].geom.node_off;
        const LaunchSet ls = launch_set(c, a, b - a);
        double* d[4];
        for (int k = 0; k < 4; ++k) d[k] = node_base(c->d_io + k * S, gb);
        if (density_only) {
            e = c->precision == LBM_FP64 ? launch_density_f64(ls, (const double*)c->f[c->cur], d[0], c->stream)
                                         : launch_density_f32(ls, (const float*)c->f[c->cur], d[0], c->stream);
            c->launches += 1;
        } else {
            double* psi = cell_base(c->d_psi, cell_lo(c, a));
            e = c->precision == LBM_FP64
                    ? launch_moments_f64(ls, (const double*)c->f[c->cur], psi, d[0], d[1], d[2], d[3], c->stream)
                    : launch_moments_f32(ls, (const float*)c->f[c->cur], psi, d[0], d[1], d[2], d[3], c->stream);
            c->launches += 2;
        }
        if (e != cudaSuccess) return cuda_fail(e, "moments kernels");
        const size_t bytes = (size_t)range_nodes(c, a, b - a) * sizeof(double);
        for (int k = 0; k < 4; ++k)
            if (h[k]) CK(cudaMemcpyAsync(h[k] + (gb - base), c->d_io + k * S, bytes, cudaMemcpyDeviceToHost, c->stream));
        a = b;
    }
    return LBM_OK;  // the caller synchronises (read_status)
}

int create_common(int n, const lbm_lattice_desc* desc, int precision, lbm_ctx** out) {
    if (!out) return fail(LBM_EINVAL, "out is null");
    *out = nullptr;
    if (n < 1 || !desc) return fail(LBM_EINVAL, "need n >= 1 lattice descriptions");
    if (n > 65535) return fail(LBM_EINVAL, "n=%d lattices: at most 65535 per context", n);
    const bool inplace = (precision & LBM_INPLACE) != 0;
    precision &= ~LBM_INPLACE;
    if (precision != LBM_FP32_DEV && precision != LBM_FP32 && precision != LBM_FP64)
        return fail(LBM_EINVAL, "unknown precision %d", precision);
    for (int i = 0; i < n; ++i) {
        int rc = validate_desc(desc[i], i);
        if (rc) return rc;
    }
    int dev_count = 0;
    cudaError_t de = cudaGetDeviceCount(&dev_count);
    if (de != cudaSuccess || dev_count == 0) {
        cudaGetLastError();
        return fail(LBM_ECUDA, "no CUDA device available: %s", cudaGetErrorString(de));
    }

    lbm_ctx* c = new lbm_ctx();
    if (const char* w = getenv("LBM_TMA_WAIT_CYCLES")) c->tma_wait_limit = std::max(0LL, atoll(w));
    if (const char* x = getenv("LBM_TMA_EXTRA_TX")) c->tma_extra_tx = (unsigned)std::min(4096LL, std::max(0LL, atoll(x)));
    if (const char* a = getenv("LBM_FAIL_ALLOC_AT")) c->fail_alloc_at = std::max(0LL, atoll(a));
    c->n = n;
    c->precision = precision;
    c->inplace = inplace;
    c->elem = precision == LBM_FP64 ? 8 : 4;
    c->lats.resize(n);
    c->phys_d.resize(n);
    long long f_off = 0, m_off = 0, node_off = 0;
    for (int i = 0; i < n; ++i) {
        HostLattice& L = c->lats[i];
        L.desc = desc[i];
        L.desc.wall_mask = nullptr;
        Geom& g = L.geom;
        g.nx = desc[i].nx;
        g.ny = desc[i].ny;
        g.pitch = (int)round_up((long long)g.nx + kGX + 2, 32);
        g.plane = (long long)(g.ny + 2 * kGY) * g.pitch;
        g.f_off = f_off;
        g.node_off = node_off;
        const long long nn = (long long)g.nx * g.ny;
        L.n_fluid = nn;
        if (desc[i].wall_mask) {
            L.mask.assign(desc[i].wall_mask, desc[i].wall_mask + nn);
            for (auto& b : L.mask) b = b ? 1 : 0;
            L.n_fluid = 0;
            for (auto b : L.mask) L.n_fluid += (b == 0);
            g.flags = kGeomMask;
            g.mask_off = m_off;
            m_off += round_up(g.plane, 256);
        } else {
            g.flags = 0;
            g.mask_off = 0;
        }
        // keep each lattice's planes 256-byte aligned
        f_off += round_up(9 * g.plane, 64);
        L.c_off = c->compact_elems;
        c->compact_elems += round_up(9 * (long long)g.ny * round_up(g.nx, 32), 64);
        node_off += nn;
        c->total_nodes += nn;
        c->fluid_nodes += L.n_fluid;
        c->max_nodes = std::max(c->max_nodes, nn);
        if (precision == LBM_FP32_DEV) {
            L.rho_ref_auto = desc[i].rho_ref < 0.0;
            L.rho_ref = L.rho_ref_auto ? 0.0 : (double)(float)desc[i].rho_ref;
        } else {
            L.rho_ref_auto = false;
            L.rho_ref = 0.0;
        }
    }
    c->total_elems = f_off;
    c->mask_bytes = m_off;

    int rc = LBM_OK;
    const size_t fbytes = (size_t)c->total_elems * c->elem;
    if (!rc) rc = dev_alloc(c, &c->f[0], fbytes);
    if (!rc && !c->inplace) rc = dev_alloc(c, &c->f[1], fbytes);
    if (!rc) {
        int dev = 0, l2 = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) == cudaSuccess)
            c->streams_dram = 2 * fbytes > (size_t)l2;
    }
    if (!rc && c->inplace) c->f[1] = c->f[0];
    if (!rc && m_off > 0) rc = dev_alloc(c, &c->d_mask, (size_t)m_off);
    if (!rc) rc = dev_alloc(c, &c->d_geom, n * sizeof(Geom));
    if (!rc) rc = dev_alloc(c, &c->d_phys_f, n * sizeof(Phys<float>));
    if (!rc) rc = dev_alloc(c, &c->d_phys_d, n * sizeof(Phys<double>));
    if (!rc) rc = dev_alloc(c, &c->d_status, n * sizeof(unsigned));
    // reduction scratch: 4 partial sums per block and lattice, 3 totals per lattice
    if (!rc) rc = dev_alloc(c, &c->d_partials, 4 * (size_t)kMassBlocks * n * sizeof(double));
    if (!rc) rc = dev_alloc(c, &c->d_scalar, 3 * (size_t)n * sizeof(double));
    // staging for a group of lattices at a time: at least the largest
    // lattice, at most kStageNodes nodes (and kStageCells psi cells) unless
    // one lattice needs more
    long long max_plane = 0;
    for (const auto& L : c->lats) max_plane = std::max(max_plane, L.geom.plane);
    const long long total_cells = c->total_elems / 9 + 64;
    // LBM_STAGE_NODES / LBM_STAGE_CELLS (read here) lower the two limits, so
    // that a test can make small batches take several groups
    long long lim_nodes = kStageNodes, lim_cells = kStageCells;
    if (const char* v = getenv("LBM_STAGE_NODES")) lim_nodes = std::max(1LL, std::min(kStageNodes, atoll(v)));
    if (const char* v = getenv("LBM_STAGE_CELLS")) lim_cells = std::max(1LL, std::min(kStageCells, atoll(v)));
    c->stage_nodes = std::max(c->max_nodes, std::min(c->total_nodes, lim_nodes));
    c->stage_cells = std::max(max_plane, std::min(total_cells, lim_cells));
    if (!rc) rc = dev_alloc(c, &c->d_io, 4 * (size_t)c->stage_nodes * sizeof(double));
    // in place, the step also keeps one psi plane of every lattice here
    const size_t psi_bytes = std::max((size_t)c->stage_cells * sizeof(double),
                                      c->inplace ? (size_t)total_cells * c->elem : (size_t)0);
    if (!rc) rc = dev_alloc(c, &c->d_psi, psi_bytes);
    if (!rc && cudaHostAlloc((void**)&c->h_status, n * sizeof(unsigned), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        c->h_status = nullptr;
        rc = fail(LBM_ENOMEM, "cudaHostAlloc(%zu bytes) failed", n * sizeof(unsigned));
    }
    if (!rc && cudaHostAlloc((void**)&c->h_bad, n * sizeof(unsigned), cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        c->h_bad = nullptr;
        rc = fail(LBM_ENOMEM, "cudaHostAlloc(%zu bytes) failed", n * sizeof(unsigned));
    }
    if (!rc) {
        memset(c->h_bad, 0, n * sizeof(unsigned));
        if (cudaHostGetDevicePointer((void**)&c->m_bad, c->h_bad, 0) != cudaSuccess) {
            cudaGetLastError();
            rc = fail(LBM_ECUDA, "no device address for the page-locked flag buffer");
        }
    }
    if (rc) {
        free_ctx(c);
        return rc;
    }
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemset(c->f[0], 0, fbytes);
    if (e == cudaSuccess && c->f[1] != c->f[0]) e = cudaMemset(c->f[1], 0, fbytes);
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, n * sizeof(unsigned));
    if (e == cudaSuccess && m_off > 0) {
        e = cudaMemset(c->d_mask, 0, (size_t)m_off);
        for (int i = 0; i < n && e == cudaSuccess; ++i) e = upload_mask(c, i);
    }
    if (e == cudaSuccess) {
        std::vector<Geom> geoms(n);
        for (int i = 0; i < n; ++i) geoms[i] = c->lats[i].geom;
        e = cudaMemcpy(c->d_geom, geoms.data(), n * sizeof(Geom), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        rc = cuda_fail(e, "context set-up copy");
        free_ctx(c);
        return rc;
    }
    rc = upload_phys(c);
    if (!rc) rc = build_tiles(c, 0);
    if (rc) {
        free_ctx(c);
        return rc;
    }
    *out = c;
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_create(int nx, int ny, const lbm_eos_params* eos, const double relax_rates[9], double eps,
               const uint8_t* wall_mask, int precision, lbm_ctx** out) {
    g_last_error.clear();
    if (!eos || !relax_rates) return fail(LBM_EINVAL, "eos and relax_rates must not be null");
    lbm_lattice_desc d;
    d.nx = nx;
    d.ny = ny;
    d.eos = *eos;
    for (int k = 0; k < 9; ++k) d.s[k] = relax_rates[k];
    d.eps = eps;
    d.rho_ref = -1.0;  // FP32_DEV: minimum of the first density field
    d.wall_mask = wall_mask;
    return create_common(1, &d, precision, out);
}

int lbm_create_batch(int n, const lbm_lattice_desc* desc, int precision, lbm_ctx** out) {
    g_last_error.clear();
    return create_common(n, desc, precision, out);
}

int lbm_set_stream(lbm_ctx* c, void* stream) {
    if (!c) return fail(LBM_EINVAL, "null context");
    cudaStream_t s = (cudaStream_t)stream;
    if (s != c->stream) {
        drop_graphs(c);
        c->stream = s;
    }
    return LBM_OK;
}

int lbm_init_fields(lbm_ctx* c, int lat, const double* rho, const double* ux, const double* uy) {
    Range range("lbm_init_fields");
    int rc = check_lat(c, lat);
    if (!rc) rc = check_whole_step(c, "lbm_init_fields");
    if (rc) return rc;
    if (!rho) return fail(LBM_EINVAL, "rho must not be null");
    rc = geom_open_x(c->lats[lat].geom) ? init_open(c, lat, rho, ux, uy) : init_range(c, lat, 1, rho, ux, uy);
    if (rc) return rc;
    c->steps = 0;
    return LBM_OK;
}

int lbm_init_fields_all(lbm_ctx* c, const double* rho, const double* ux, const double* uy) {
    Range range("lbm_init_fields_all");
    if (!c) return fail(LBM_EINVAL, "null context");
    if (check_whole_step(c, "lbm_init_fields_all")) return LBM_EINVAL;
    if (!rho) return fail(LBM_EINVAL, "rho must not be null");
    if (any_open_x(c))
        return fail(LBM_EINVAL, "a lattice of this context is open in x: initialise it with lbm_init_fields "
                                "((nx + 2) x ny arrays)");
    int rc = init_range(c, 0, c->n, rho, ux, uy);
    if (rc) return rc;
    c->steps = 0;
    return LBM_OK;
}

int lbm_step(lbm_ctx* c, int n) {
    Range range("lbm_step");
    if (!c) return fail(LBM_EINVAL, "null context");
    if (n < 0) return fail(LBM_EINVAL, "n=%d must be >= 0", n);
    if (n > 1 && any_open_x(c))
        return fail(LBM_EINVAL, "n=%d: a lattice open in x needs its halo exchanged between steps; step one "
                                "at a time", n);
    if (n > 0 && c->part_done)
        return fail(LBM_EINVAL, "a split step (lbm_step_part) is half done: launch its other part first");
    int done = 0;
    if (capturable_stream(c->stream)) {
        while (n - done >= kGraphChunk) {
            int rc = ensure_graph(c, c->cur);
            if (rc) return rc;
            CK(cudaGraphLaunch(c->graph[c->cur], c->stream));
            c->launches += kGraphChunk * launches_per_step(c);
            done += kGraphChunk;
            c->steps += kGraphChunk;  // kGraphChunk is even: c->cur unchanged
        }
    }
    for (; done < n; ++done) {
        cudaError_t e = launch_one_step(c, c->cur);
        if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
        c->launches += launches_per_step(c);
        c->cur ^= 1;
        c->steps += 1;
    }
    return LBM_OK;
}

int lbm_step_part(lbm_ctx* c, int part) {
    Range range("lbm_step_part");
    if (!c) return fail(LBM_EINVAL, "null context");
    if (part != LBM_STEP_EDGE && part != LBM_STEP_INTERIOR)
        return fail(LBM_EINVAL, "part=%d must be LBM_STEP_EDGE or LBM_STEP_INTERIOR", part);
    if (c->part_done & part) return fail(LBM_EINVAL, "part %d of this step was launched already", part);
    cudaError_t e = launch_one_step(c, c->cur, part);
    if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
    c->launches += part == LBM_STEP_EDGE ? (c->n_edge > 0 ? 1 : 0) : launches_per_step(c);
    c->part_done |= part;
    if (c->part_done == (LBM_STEP_EDGE | LBM_STEP_INTERIOR)) {
        c->part_done = 0;
        c->cur ^= 1;
        c->steps += 1;
    }
    return LBM_OK;
}

int lbm_read_moments(lbm_ctx* c, int lat, double* rho, double* ux, double* uy, double* p) {
    Range range("lbm_read_moments");
    int rc = check_lat(c, lat);
    if (rc) return rc;
    rc = moments_range(c, lat, 1, rho, ux, uy, p);
    if (rc) return rc;
    std::vector<unsigned> st;
    rc = read_status(c, st);
    if (rc) return rc;
    return status_code(st[lat]);
}

int lbm_read_moments_all(lbm_ctx* c, double* rho, double* ux, double* uy, double* p) {
    Range range("lbm_read_moments_all");
    if (!c) return fail(LBM_EINVAL, "null context");
    int rc = moments_range(c, 0, c->n, rho, ux, uy, p);
    if (rc) return rc;
    std::vector<unsigned> st;
    rc = read_status(c, st);
    if (rc) return rc;
    unsigned all = 0;
    for (unsigned s : st) all |= s;
    return status_code(all);
}

int lbm_total_mass(lbm_ctx* c, int lat, double* mass) {
    Range range("lbm_total_mass");
    int rc = check_lat(c, lat);
    if (rc) return rc;
    if (!mass) return fail(LBM_EINVAL, "mass must not be null");
    const HostLattice& L = c->lats[lat];
    const uint8_t* dm = L.mask.empty() ? nullptr : c->d_mask + L.geom.mask_off;
    cudaError_t e;
    if (c->precision == LBM_FP64)
        e = launch_mass_f64(L.geom, L.rho_ref, L.n_fluid, (const double*)c->f[c->cur], dm, state_layout(c),
                            c->d_partials,
                            c->d_scalar, c->stream);
    else
        e = launch_mass_f32(L.geom, L.rho_ref, L.n_fluid, (const float*)c->f[c->cur], dm, state_layout(c),
                            c->d_partials,
                            c->d_scalar, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "mass kernels");
    c->launches += 2;
    CK(cudaMemcpyAsync(mass, c->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    std::vector<unsigned> st;
    rc = read_status(c, st);
    if (rc) return rc;
    return status_code(st[lat]);
}

namespace {

// Mass and momentum of lattices [lat0, lat0 + n_lat) into out[3k .. 3k + 2];
// the status bits of every lattice come back in st.
int totals_range(lbm_ctx* c, int lat0, int n_lat, double* out, std::vector<unsigned>& st) {
    const long long S = c->stage_nodes;
    for (int a = lat0; a < lat0 + n_lat;) {
        const int b = group_end(c, a, lat0 + n_lat);
        const long long gb = c->lats[a].geom.node_off;
        const LaunchSet ls = launch_set(c, a, b - a);
        double* psi = cell_base(c->d_psi, cell_lo(c, a));
        double* d[3];
        for (int k = 0; k < 3; ++k) d[k] = node_base(c->d_io + k * S, gb);
        cudaError_t e;
        if (c->precision == LBM_FP64)
            e = launch_totals_f64(ls, (const double*)c->f[c->cur], psi, d[0], d[1], d[2], c->d_partials,
                                  c->d_scalar + 3 * (a - lat0), c->stream);
        else
            e = launch_totals_f32(ls, (const float*)c->f[c->cur], psi, d[0], d[1], d[2], c->d_partials,
                                  c->d_scalar + 3 * (a - lat0), c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "totals kernels");
        c->launches += 3;
        a = b;
    }
    CK(cudaMemcpyAsync(out, c->d_scalar, 3 * (size_t)n_lat * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return read_status(c, st);
}

}  // namespace

int lbm_total_momentum(lbm_ctx* c, int lat, double* px, double* py) {
    Range range("lbm_total_momentum");
    int rc = check_lat(c, lat);
    if (rc) return rc;
    if (!px && !py) return fail(LBM_EINVAL, "px and py must not both be null");
    double t[3];
    std::vector<unsigned> st;
    rc = totals_range(c, lat, 1, t, st);
    if (rc) return rc;
    if (px) *px = t[1];
    if (py) *py = t[2];
    return status_code(st[lat]);
}

int lbm_totals_all(lbm_ctx* c, double* out) {
    Range range("lbm_totals_all");
    if (!c) return fail(LBM_EINVAL, "null context");
    if (!out) return fail(LBM_EINVAL, "out must not be null");
    std::vector<unsigned> st;
    int rc = totals_range(c, 0, c->n, out, st);
    if (rc) return rc;
    unsigned all = 0;
    for (unsigned s : st) all |= s;
    return status_code(all);
}

int lbm_status(lbm_ctx* c, int lat, uint32_t* flags) {
    int rc = check_lat(c, lat);
    if (rc) return rc;
    if (!flags) return fail(LBM_EINVAL, "flags must not be null");
    std::vector<unsigned> st;
    rc = read_status(c, st);
    if (rc) return rc;
    *flags = st[lat];
    return LBM_OK;
}

int lbm_clear_status(lbm_ctx* c) {
    if (!c) return fail(LBM_EINVAL, "null context");
    CK(cudaMemsetAsync(c->d_status, 0, c->n * sizeof(unsigned), c->stream));
    return LBM_OK;
}

int lbm_sync(lbm_ctx* c) {
    if (!c) return fail(LBM_EINVAL, "null context");
    std::vector<unsigned> st;
    int rc = read_status(c, st);
    if (rc) return rc;
    unsigned all = 0;
    for (unsigned s : st) all |= s;
    return status_code(all);
}

int lbm_state_size(lbm_ctx* c, size_t* bytes) {
    if (!c || !bytes) return fail(LBM_EINVAL, "null argument");
    *bytes = 4 * sizeof(uint32_t) + sizeof(long long) + c->n * sizeof(double) +
             (size_t)c->compact_elems * c->elem;
    return LBM_OK;
}

namespace {

uint32_t blob_kind(const lbm_ctx* c) {
    uint32_t k = (uint32_t)c->precision;
    if (c->inplace) k |= (uint32_t)LBM_INPLACE | (c->cur ? kBlobSwapped : 0u);
    return k;
}

// Copy every lattice's nodes between the device layout (frame, row
// pitch `pitch`) and the compact checkpoint layout (plane a of lattice l at
// c_off + a*ny*cpitch, node (x, y) at y*cpitch + x, cpitch = round_up(nx, 32)).
int copy_compact(lbm_ctx* c, char* host, bool to_host) {
    for (int l = 0; l < c->n; ++l) {
        const HostLattice& L = c->lats[l];
        const Geom& g = L.geom;
        const size_t cpitch = (size_t)round_up(g.nx, 32);
        for (int a = 0; a < 9; ++a) {
            char* h = host + ((size_t)L.c_off + (size_t)a * g.ny * cpitch) * c->elem;
            char* d = (char*)c->f[c->cur] + ((size_t)g.f_off + (size_t)a * g.plane + node_index(g, 0, 0)) * c->elem;
            if (to_host)
                CK(cudaMemcpy2DAsync(h, cpitch * c->elem, d, (size_t)g.pitch * c->elem, (size_t)g.nx * c->elem,
                                     (size_t)g.ny, cudaMemcpyDeviceToHost, c->stream));
            else
                CK(cudaMemcpy2DAsync(d, (size_t)g.pitch * c->elem, h, cpitch * c->elem, (size_t)g.nx * c->elem,
                                     (size_t)g.ny, cudaMemcpyHostToDevice, c->stream));
        }
    }
    return LBM_OK;
}

}  // namespace

int lbm_save_state(lbm_ctx* c, void* buf, size_t bytes) {
    Range range("lbm_save_state");
    size_t need = 0;
    int rc = lbm_state_size(c, &need);
    if (!rc) rc = check_whole_step(c, "lbm_save_state");
    if (rc) return rc;
    if (!buf || bytes < need) return fail(LBM_EINVAL, "state buffer needs %zu bytes, got %zu", need, bytes);
    char* p = (char*)buf;
    uint32_t hdr[4] = {kStateMagic, blob_kind(c), (uint32_t)c->n, (uint32_t)c->compact_elems};
    memcpy(p, hdr, sizeof(hdr));
    p += sizeof(hdr);
    memcpy(p, &c->steps, sizeof(long long));
    p += sizeof(long long);
    for (int l = 0; l < c->n; ++l) {
        memcpy(p, &c->lats[l].rho_ref, sizeof(double));
        p += sizeof(double);
    }
    memset(p, 0, (size_t)c->compact_elems * c->elem);
    rc = copy_compact(c, p, true);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_load_state(lbm_ctx* c, const void* buf, size_t bytes) {
    Range range("lbm_load_state");
    size_t need = 0;
    int rc = lbm_state_size(c, &need);
    if (!rc) rc = check_whole_step(c, "lbm_load_state");
    if (rc) return rc;
    if (!buf || bytes < need) return fail(LBM_EINVAL, "state blob has %zu bytes, need %zu", bytes, need);
    const char* p = (const char*)buf;
    uint32_t hdr[4];
    memcpy(hdr, p, sizeof(hdr));
    p += sizeof(hdr);
    const uint32_t kind = hdr[1] & ~kBlobSwapped;
    if (hdr[0] != kStateMagic || kind != (blob_kind(c) & ~kBlobSwapped) || hdr[2] != (uint32_t)c->n ||
        hdr[3] != (uint32_t)c->compact_elems)
        return fail(LBM_EINVAL, "state blob does not match this context (lattices or precision differ)");
    long long steps;
    memcpy(&steps, p, sizeof(long long));
    p += sizeof(long long);
    for (int l = 0; l < c->n; ++l) {
        memcpy(&c->lats[l].rho_ref, p, sizeof(double));
        c->lats[l].rho_ref_auto = false;
        p += sizeof(double);
    }
    rc = upload_phys(c);
    if (rc) return rc;
    drop_graphs(c);
    rc = copy_compact(c, const_cast<char*>(p), false);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->stream));
    c->steps = steps;
    if (c->inplace) c->cur = (hdr[1] & kBlobSwapped) ? 1 : 0;
    return LBM_OK;
}

int lbm_tile_count(void) { return total_tiles(); }

int lbm_tile_shape(int index, int* tx, int* ty) {
    if (index < 0 || index >= total_tiles())
        return fail(LBM_EINVAL, "tile index %d outside [0, %d)", index, total_tiles());
    int a = 0, b = 0;
    tile_shape(index, &a, &b);
    if (tx) *tx = a;
    if (ty) *ty = b;
    return LBM_OK;
}

int lbm_tile_kind(int index, int* kind) {
    if (index < 0 || index >= total_tiles())
        return fail(LBM_EINVAL, "tile index %d outside [0, %d)", index, total_tiles());
    if (!kind) return fail(LBM_EINVAL, "null argument");
    *kind = is_pipe(index) ? LBM_TILE_PIPELINED : is_tma(index) ? LBM_TILE_TMA : LBM_TILE_PLAIN;
    return LBM_OK;
}

int lbm_set_tile(lbm_ctx* c, int index) {
    if (!c) return fail(LBM_EINVAL, "null context");
    if (check_whole_step(c, "lbm_set_tile")) return LBM_EINVAL;
    if (index < 0 || index >= total_tiles())
        return fail(LBM_EINVAL, "tile index %d outside [0, %d)", index, total_tiles());
    if (index == c->tile_index) return LBM_OK;
    CK(cudaStreamSynchronize(c->stream));
    const int prev = c->tile_index;
    const int rc = build_tiles(c, index);
    if (rc != LBM_OK && c->tile_index != prev) {
        // a later stage failed after the list was replaced: go back to the
        // previous shape, keeping the first error's message
        const std::string msg = g_last_error;
        build_tiles(c, prev);
        g_last_error = msg;
    }
    return rc;
}

int lbm_autotune(lbm_ctx* c, int steps, int* best_index, double* ms) {
    Range range("lbm_autotune");
    if (!c) return fail(LBM_EINVAL, "null context");
    if (steps < 1) return fail(LBM_EINVAL, "steps=%d must be >= 1", steps);
    if (check_whole_step(c, "lbm_autotune")) return LBM_EINVAL;
    const size_t fbytes = (size_t)c->total_elems * c->elem;
    void* saved = nullptr;
    int rc = dev_alloc(c, &saved, fbytes);
    if (rc) return rc;
    std::vector<unsigned> saved_status(c->n);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const int cur0 = c->cur;
    const long long steps0 = c->steps;
    const int tile0 = c->tile_index;
    int best = tile0;
    double best_ms = 1e300;
    auto cleanup = [&]() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(saved);
        c->device_bytes -= fbytes;
    };
    cudaError_t e = cudaMemcpyAsync(saved, c->f[cur0], fbytes, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(saved_status.data(), c->d_status, c->n * sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "autotune set-up");
    }
    for (int t = 0; t < total_tiles(); ++t) {
        if ((t >= kTileCount && (c->precision == LBM_FP64 || c->inplace)) ||
            (is_tma(t) && c->n > kTmaMaxLattices)) {
            if (ms) ms[t] = -1.0;  // FP32 two-buffer variant, or too many lattices for it
            continue;
        }
        rc = build_tiles(c, t);
        if (rc) break;
        // warm-up launch, then the timed steps
        e = launch_one_step(c, c->cur);
        c->launches += launches_per_step(c);
        c->cur ^= 1;
        if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
        for (int k = 0; k < steps && e == cudaSuccess; ++k) {
            e = launch_one_step(c, c->cur);
            c->launches += launches_per_step(c);
            c->cur ^= 1;
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t_ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t_ms, e0, e1);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "autotune trial");
            break;
        }
        const double per = (double)t_ms / steps;
        if (ms) ms[t] = per;
        if (per < best_ms) {
            best_ms = per;
            best = t;
        }
        // restore the state for the next candidate
        e = cudaMemcpyAsync(c->f[cur0], saved, fbytes, cudaMemcpyDeviceToDevice, c->stream);
        c->cur = cur0;
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "autotune restore");
            break;
        }
    }
    if (!rc) {
        e = cudaMemcpyAsync(c->f[cur0], saved, fbytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->d_status, saved_status.data(), c->n * sizeof(unsigned), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "autotune final restore");
    }
    c->cur = cur0;
    c->steps = steps0;
    cleanup();
    if (rc) {
        build_tiles(c, tile0);
        return rc;
    }
    rc = build_tiles(c, best);
    if (rc) return rc;
    if (best_index) *best_index = best;
    return LBM_OK;
}

int lbm_get_state_view(lbm_ctx* c, int lat, lbm_state_view* view) {
    if (!view) return fail(LBM_EINVAL, "null argument");
    int rc = check_lat(c, lat);
    if (rc) return rc;
    const HostLattice& L = c->lats[lat];
    const Geom& g = L.geom;
    view->base = (char*)c->f[c->cur] + (size_t)g.f_off * c->elem;
    view->plane = g.plane;
    view->pitch = g.pitch;
    view->rows = (int)(g.plane / g.pitch);
    view->x0 = kGX;
    view->y0 = kGY;
    view->elem_bytes = c->elem;
    view->deviation = c->precision == LBM_FP32_DEV ? 1 : 0;
    view->rho_ref = c->precision == LBM_FP32_DEV ? L.rho_ref : 0.0;
    view->layout = state_layout(c);
    return LBM_OK;
}

int lbm_info(lbm_ctx* c, lbm_info_t* info) {
    if (!c || !info) return fail(LBM_EINVAL, "null argument");
    info->n_lattices = c->n;
    info->precision = c->precision;
    info->nodes = c->total_nodes;
    info->fluid_nodes = c->fluid_nodes;
    info->steps = c->steps;
    info->kernel_launches = c->launches;
    info->device_bytes = c->device_bytes;
    tile_shape(c->tile_index, &info->tile_x, &info->tile_y);
    info->n_tiles = c->n_tiles + c->n_fast + c->n_tma;
    info->graph_chunk = kGraphChunk;
    info->inplace = c->inplace ? 1 : 0;
    info->l2_prefetch = c->streams_dram && !c->inplace && c->precision != LBM_FP64 ? 1 : 0;
    info->tile_grid =
        c->grid.tiles_x > 0 && !c->inplace && c->precision != LBM_FP64 && c->tile_index < kTileCount ? 1 : 0;
    return LBM_OK;
}

int lbm_set_open_x(lbm_ctx* c, int lat, const uint8_t* halo_mask) {
    Range range("lbm_set_open_x");
    int rc = check_lat(c, lat);
    if (!rc) rc = check_whole_step(c, "lbm_set_open_x");
    if (rc) return rc;
    HostLattice& L = c->lats[lat];
    Geom& g = L.geom;
    if (c->inplace) return fail(LBM_EINVAL, "an x-slab needs two-buffer storage; this context stores in place");
    if (g.nx < 2) return fail(LBM_EINVAL, "lattice %d: an x-slab needs nx >= 2 (nx=%d)", lat, g.nx);
    if (c->precision == LBM_FP32_DEV && L.rho_ref_auto)
        return fail(LBM_EINVAL, "lattice %d: an x-slab needs an explicit rho_ref (>= 0) shared by every slab of "
                                "its lattice, so that their stored halos mean the same", lat);
    if (L.mask.empty()) {
        if (halo_mask)
            for (long long i = 0; i < 4LL * g.ny; ++i)
                if (halo_mask[i]) return fail(LBM_EINVAL, "lattice %d has no wall mask: halo_mask must be clear", lat);
    } else {
        L.halo_mask.assign((size_t)4 * g.ny, 0);
        for (int col = 0; col < 4; ++col)
            for (int y = 0; y < g.ny; ++y) {
                const int xe = col < 2 ? 0 : g.nx - 1;  // the edge column continued across the cut
                L.halo_mask[(size_t)col * g.ny + y] =
                    halo_mask ? (halo_mask[(size_t)col * g.ny + y] ? 1 : 0) : L.mask[(size_t)y * g.nx + xe];
            }
    }
    const int old_flags = g.flags;
    g.flags |= kGeomOpenX;
    cudaError_t e = upload_mask(c, lat);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_geom + lat, &g, sizeof(Geom), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        g.flags = old_flags;
        cudaMemcpy(c->d_geom + lat, &g, sizeof(Geom), cudaMemcpyHostToDevice);
        return cuda_fail(e, "x-slab set-up");
    }
    rc = build_tiles(c, c->tile_index);  // the tiles at the x edges now take the general path
    if (rc) {
        g.flags = old_flags;
        cudaMemcpy(c->d_geom + lat, &g, sizeof(Geom), cudaMemcpyHostToDevice);
        return rc;
    }
    return LBM_OK;
}

static int halo_call(lbm_ctx* c, int lat, int side, void* buf, bool pack, void* stream) {
    int rc = check_lat(c, lat);
    if (rc) return rc;
    if (!geom_open_x(c->lats[lat].geom)) return fail(LBM_EINVAL, "lattice %d is not open in x (lbm_set_open_x)", lat);
    if (side != 0 && side != 1) return fail(LBM_EINVAL, "side=%d must be 0 (left) or 1 (right)", side);
    if (!buf) return fail(LBM_EINVAL, "null halo buffer");
    // during a split step, the buffer that step writes (its edge part must
    // have run before a pack); else the state the next step reads
    int b = c->cur;
    if (c->part_done) {
        if (pack && !(c->part_done & LBM_STEP_EDGE))
            return fail(LBM_EINVAL, "halo pack during a split step needs its edge part first");
        b = 1 - c->cur;
    }
    const Geom& g = c->lats[lat].geom;
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    cudaError_t e = c->precision == LBM_FP64
                        ? launch_halo_f64(g, (double*)c->f[b], side, (double*)buf, pack, s)
                        : launch_halo_f32(g, (float*)c->f[b], side, (float*)buf, pack, s);
    if (e != cudaSuccess) return cuda_fail(e, pack ? "halo pack" : "halo unpack");
    c->launches += 1;
    return LBM_OK;
}

int lbm_halo_pack(lbm_ctx* c, int lat, int side, void* dev_out, void* cuda_stream) {
    Range range("lbm_halo_pack");
    return halo_call(c, lat, side, dev_out, true, cuda_stream);
}

int lbm_halo_unpack(lbm_ctx* c, int lat, int side, const void* dev_in, void* cuda_stream) {
    Range range("lbm_halo_unpack");
    return halo_call(c, lat, side, const_cast<void*>(dev_in), false, cuda_stream);
}

const char* lbm_last_error(void) { return g_last_error.c_str(); }

void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_ctx(c);
}

}  // extern "C"
