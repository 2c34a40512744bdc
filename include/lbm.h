/*
 * lbm.h - C ABI of the GB300 pseudopotential MRT lattice Boltzmann library.
 *
 * The library advances batches of independent two-dimensional D2Q9 lattices
 * with the scheme of Shan et al., "Pseudopotential MRT lattice Boltzmann
 * model for cavitation bubble collapse with high density ratio"
 * (arXiv:1605.01800):
 *   - MRT collision in moment space, Eq. 1-4, relaxation rates Lambda of Eq. 2;
 *   - the pseudopotential interaction force of Eq. 7 with psi of Eq. 13 and
 *     the Carnahan-Starling EOS of Eq. 15;
 *   - Li's modified forcing source of Eq. 14 (epsilon), velocity of Eq. 6;
 *   - streaming, Eq. 5, periodic in x and y, with no-slip halfway bounce-back
 *     at solid nodes (Sec. 4.1).
 * Lattice units: delta_x = delta_t = c = 1, c_s^2 = 1/3.
 *
 * Conventions shared by every entry point:
 *   - Every function returns LBM_OK (0) or an LBM_E* code; lbm_last_error()
 *     then holds a message for the calling thread.
 *   - Host arrays of one lattice are row-major nx*ny doubles (x fastest). The
 *     "_all" variants take the lattices of a batch concatenated in creation
 *     order (sum of nx*ny doubles).
 *   - Host pointers may be pageable or pinned; the library copies them
 *     (inputs) or fills them (outputs) and never keeps them. A page-locked
 *     (cudaHostAlloc / cudaHostRegister) density array given to a
 *     density-only lbm_read_moments* is written by the kernel in place, with
 *     no staging copy; the call still returns only once it is complete.
 *   - Device memory is owned by the context and released by lbm_destroy().
 *   - Work is enqueued on the context's stream (lbm_set_stream). Entry points
 *     that return data to the host synchronise that stream.
 *   - Device-side errors (psi^2 < 0 clamped, a non-finite density) are sticky
 *     per lattice; they are reported by lbm_status() and turn the return code
 *     of lbm_read_moments*, lbm_total_mass, lbm_total_momentum,
 *     lbm_totals_all and lbm_sync into
 *     LBM_EPSI_DOMAIN or LBM_ENONFINITE (the data is still written).
 *   - A context is not thread-safe; distinct contexts may be used from
 *     distinct threads.
 */
#ifndef PAPER_1605_01800_GB300_LBM_H
#define PAPER_1605_01800_GB300_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes -------------------------------------------------------- */
#define LBM_OK 0
#define LBM_EINVAL 1          /* invalid argument (message says which) */
#define LBM_ENOMEM 2          /* device or host allocation failed */
#define LBM_ECUDA 3           /* a CUDA runtime call failed */
#define LBM_EPSI_DOMAIN 4     /* psi^2 of Eq. 13 went negative somewhere and was clamped to 0 */
#define LBM_ENONFINITE 5      /* a density or psi^2 became NaN or infinite */
#define LBM_ETIMEOUT 6        /* a bounded device-side wait gave up (the step was not completed) */

/* ---- storage precision (lbm_create*, argument `precision`) --------------- */
#define LBM_FP32_DEV 0        /* FP32 storage and collision of f_a - w_a rho_ref */
#define LBM_FP32 1            /* FP32 storage of f_a (rho_ref forced to 0) */
#define LBM_FP64 2            /* FP64 storage and arithmetic */
/* OR'ed into `precision`: in-place storage (the AA pattern), one
 * distribution array instead of two (36 instead of 72 bytes per node in
 * FP32), for lattices that would not fit otherwise. Streaming (Eq. 5) is
 * folded into the stores of every other step, so the array alternates
 * between two layouts (lbm_state_view.layout). A step is two launches, psi
 * of every node into a scratch plane and then the collision in place, and
 * moves 116 bytes per node instead of 72. Results are bitwise those of
 * two-buffer storage. Not available with lbm_set_open_x; lbm_set_tile and
 * lbm_autotune take the LBM_TILE_PLAIN shapes only (others: LBM_EINVAL or
 * skipped). */
#define LBM_INPLACE 0x100

/* ---- sticky per-lattice status bits (lbm_status) ------------------------- */
#define LBM_FLAG_PSI_CLAMPED 1u
#define LBM_FLAG_NONFINITE 2u
#define LBM_FLAG_TIMEOUT 4u

typedef struct lbm_ctx lbm_ctx;

/* The pseudopotential psi of a lattice and the interaction strength G of
 * Eq. 7. `kind` selects psi:
 *   LBM_EOS_CS   Eq. 13 with the Carnahan-Starling EOS of Eq. 15 (the paper's):
 *                p = rho R T (1 + h + h^2 - h^3)/(1 - h)^3 - a rho^2, h = b rho / 4;
 *   LBM_EOS_VDW  Eq. 13 with van der Waals, p = rho R T/(1 - b rho) - a rho^2;
 *   LBM_EOS_PR   Eq. 13 with Peng-Robinson, p = rho R T/(1 - b rho)
 *                - a alpha(T) rho^2/(1 + 2 b rho - b^2 rho^2), alpha =
 *                (1 + k (1 - sqrt(T/Tc)))^2, k = 0.37464 + 1.54226 omega
 *                - 0.26992 omega^2, Tc = 0.0778 a / (0.45724 b R);
 *   LBM_PSI_EXP  Eq. 12 (the first strategy): psi = exp(-1/rho) for e = 0,
 *                (rho/(e + rho))^(1/e) otherwise, with e = -G eps: the
 *                mechanical-stability exponent that Li's term with the
 *                lattice's eps (Eq. 14) produces (e = eps at G = -1), so the
 *                model meets Eq. 11 by construction; a, b, R, T, omega
 *                unused; p of Eq. 10 is then the model's EOS (G < 0 with
 *                |G| large enough for two phases, e.g. -3).
 * For the Eq. 13 kinds G < 0 (the paper uses G = -1), b > 0, R T >= 0. The
 * fastest step paths take LBM_EOS_CS lattices; the others run the general
 * path. A zero-initialised `kind` and `omega` select the paper's EOS. */
#define LBM_EOS_CS 0
#define LBM_EOS_VDW 1
#define LBM_EOS_PR 2
#define LBM_PSI_EXP 3
typedef struct {
    double a, b, R, T, G;
    int kind;
    double omega;   /* Peng-Robinson acentric factor */
} lbm_eos_params;

/* One lattice of a batch.
 *   nx, ny     lattice size, each >= 1; 9 * ny * round_up(nx, 32) < 2^31.
 *   eos        psi (Eq. 13 with an EOS, or Eq. 12) and G.
 *   s          diagonal of Lambda (Eq. 2) in the moment order
 *              (rho, e, zeta, j_x, q_x, j_y, q_y, p_xx, p_xy); each in [0, 2).
 *   eps        epsilon of Li's term, Eq. 14.
 *   rho_ref    FP32_DEV only: the reference density of the stored deviation
 *              f_a - w_a rho_ref (rounded to FP32). > 0: used as given;
 *              0: plain FP32 storage; < 0: taken as the minimum of the first
 *              density field passed to lbm_init_fields* over fluid nodes.
 *              Any 0 <= rho_ref <= min(rho) stores every node at least as
 *              precisely as plain FP32, and the vapour of a two-phase field
 *              far more precisely. Ignored for LBM_FP32 and LBM_FP64.
 *   wall_mask  NULL (no solid nodes) or nx*ny bytes, nonzero = solid node. It
 *              is copied. Solid nodes are not updated; a fluid node's link
 *              that would stream into a solid node is reflected (halfway
 *              bounce-back), and a solid neighbour in the force sum of Eq. 7
 *              takes the psi of the fluid node being updated. */
typedef struct {
    int nx, ny;
    lbm_eos_params eos;
    double s[9];
    double eps;
    double rho_ref;
    const uint8_t* wall_mask;
} lbm_lattice_desc;

/* Context introspection (lbm_info). */
typedef struct {
    int n_lattices;
    int precision;
    long long nodes;           /* sum of nx*ny */
    long long fluid_nodes;     /* nodes that are not solid */
    long long steps;           /* time steps taken since the last init/load */
    unsigned long long kernel_launches; /* kernels this context has launched */
    size_t device_bytes;       /* device memory held by the context */
    int tile_x, tile_y;        /* node tile of one CTA of the step kernel */
    int n_tiles;               /* CTAs of one step launch */
    int graph_chunk;           /* steps per CUDA-graph replay in lbm_step */
    int inplace;               /* 1 for in-place storage (LBM_INPLACE) */
    int l2_prefetch;           /* 1 when the two distribution arrays exceed the
                                  device's L2: the FP32 step kernel then
                                  prefetches later tiles' populations into L2
                                  (no effect on results) */
    int tile_grid;             /* 1 when the plain kernel's tiles form a regular
                                  grid (every lattice alike, no walls, whole
                                  tiles), so that its shapes of four nodes per
                                  thread find tiles by arithmetic instead of
                                  loading their records (no effect on results) */
} lbm_info_t;

/* Where one lattice's current state lives on the device (lbm_state_view),
 * for zero-copy access from other device code, e.g. a PyTorch tensor built
 * through __cuda_array_interface__. Population a of node (x, y) (Eq. 1-5
 * numbering, 0 <= x < nx, 0 <= y < ny) is element
 *     a * plane + (y + y0) * pitch + (x + x0)
 * of the array at `base`. Each element is f_a - w_a rho_ref with FP32
 * deviation storage, and f_a with plain FP32 or FP64 storage. The frame
 * around the nodes (the other rows and columns of each plane) holds no
 * populations: no step reads it, so it may hold anything.
 * The view describes the buffer that the next step reads; a step writes
 * the other buffer and then reads from it (in place: the same array in the
 * other layout), so query again after lbm_step.
 * The memory belongs to the context (valid until lbm_destroy), and access
 * is ordered with the context's stream by the caller (lbm_sync). */
typedef struct {
    void* base;          /* device address of plane 0 */
    long long plane;     /* elements per plane = rows * pitch */
    int pitch;           /* elements per row */
    int rows;            /* rows per plane (ny plus the frame) */
    int x0, y0;          /* stored column and row of node (0, 0) */
    int elem_bytes;      /* 4 (FP32 storage) or 8 (FP64) */
    int deviation;       /* 1 for FP32 deviation storage */
    double rho_ref;      /* the deviation reference (0 for plain storage) */
    int layout;          /* what plane a at node x holds:
                          *   0  two-buffer storage: f*_a(x), the post-collision
                          *      value the next step pulls to x + e_a;
                          *   1  in-place storage, natural layout: f_a(x), already
                          *      streamed;
                          *   2  in-place storage, swapped layout: f*_opp(a)(x),
                          *      streaming pending (e_opp(a) = -e_a). */
} lbm_state_view;

/* Create a one-lattice context (the paper's single-domain runs, Sec. 3-4).
 * eps is the epsilon of Eq. 14; relax_rates the nine rates of Eq. 2. For
 * LBM_FP32_DEV the deviation reference is the minimum of the first density
 * field given to lbm_init_fields. The context starts in the rest state
 * rho = 0 until lbm_init_fields is called. */
int lbm_create(int nx, int ny, const lbm_eos_params* eos, const double relax_rates[9],
               double eps, const uint8_t* wall_mask, int precision, lbm_ctx** out);

/* Create a context advancing n (1 <= n <= 65535) independent lattices of any
 * sizes together: each lbm_step advances every lattice by one time step in one
 * launch. */
int lbm_create_batch(int n, const lbm_lattice_desc* desc, int precision, lbm_ctx** out);

/* Run the context's work on `cuda_stream` (a cudaStream_t, e.g. PyTorch's
 * torch.cuda.Stream().cuda_stream); NULL selects the legacy default stream,
 * on which lbm_step launches kernels one by one instead of replaying a graph. */
int lbm_set_stream(lbm_ctx* ctx, void* cuda_stream);

/* Set lattice `lat` to the equilibrium f_eq(rho, u) of Eq. 4 at every fluid
 * node (host arrays, nx*ny doubles; ux/uy may be NULL for u = 0) and reset the
 * step counter. The state is then the distribution at time 0 (before the
 * first collision). Densities must be > 0 and finite at fluid nodes. */
int lbm_init_fields(lbm_ctx* ctx, int lat, const double* rho, const double* ux, const double* uy);

/* lbm_init_fields for every lattice, inputs concatenated in creation order. */
int lbm_init_fields_all(lbm_ctx* ctx, const double* rho, const double* ux, const double* uy);

/* Advance every lattice by n >= 0 time steps (Eq. 1: collision, Eq. 3, then
 * streaming, Eq. 5). Asynchronous on the context's stream. With a non-default
 * stream, whole chunks of `graph_chunk` steps replay a captured CUDA graph. */
int lbm_step(lbm_ctx* ctx, int n);

/* One time step in two launches (asynchronous on the context's stream), for
 * overlapping an x-slab's halo exchange with the step:
 *   LBM_STEP_EDGE      the tiles within two cells of an open x edge (those
 *                      whose nodes the halo holds; none without x-slabs);
 *   LBM_STEP_INTERIOR  every other tile.
 * The step is complete (the state advances, the step count grows) once both
 * parts are launched, in either order; the result is bitwise lbm_step(ctx, 1).
 * Between the two parts the read-outs see the state before the step. While
 * a split step is half done, lbm_step, lbm_init_fields*, lbm_save_state,
 * lbm_load_state, lbm_set_tile, lbm_autotune and lbm_set_open_x return
 * LBM_EINVAL, as do another part value and a part launched twice. */
#define LBM_STEP_EDGE 1
#define LBM_STEP_INTERIOR 2
int lbm_step_part(lbm_ctx* ctx, int part);

/* Macroscopic fields of lattice `lat` at the current time: rho = sum_a f_a,
 * v of Eq. 6 (with the force of Eq. 7), p of Eq. 10. Host outputs of nx*ny
 * doubles; any may be NULL (with ux, uy and p all NULL only the density is
 * computed, by a lighter kernel, with the same values). Solid nodes read as 0.
 * Synchronises the stream. */
int lbm_read_moments(lbm_ctx* ctx, int lat, double* rho, double* ux, double* uy, double* p);

/* lbm_read_moments for every lattice, outputs concatenated in creation order. */
int lbm_read_moments_all(lbm_ctx* ctx, double* rho, double* ux, double* uy, double* p);

/* Total mass sum_x rho(x) over the fluid nodes of lattice `lat`, reduced in
 * FP64 in a fixed order (bitwise reproducible). Synchronises the stream. */
int lbm_total_mass(lbm_ctx* ctx, int lat, double* mass);

/* Total momentum of lattice `lat`: the sums over its fluid nodes of
 * j + F/2, the numerator of Eq. 6 (j = sum_a e_a f_a with the distribution as
 * lbm_read_moments gathers it, F the force of Eq. 7), i.e. the sums of rho v_x
 * and rho v_y. Reduced in FP64 in a fixed order (bitwise reproducible). px or
 * py may be NULL (not both: LBM_EINVAL). Without walls the total is invariant
 * under lbm_step up to rounding; walls exchange momentum with the fluid.
 * Three kernel launches; uses the read-out scratch; synchronises the stream.
 * Returns a lattice's sticky status like lbm_total_mass. */
int lbm_total_momentum(lbm_ctx* ctx, int lat, double* px, double* py);

/* Mass and momentum of every lattice in three launches for the whole batch:
 * out (host, 3 * n_lattices doubles) receives, for lattice k in creation
 * order, out[3k] = lbm_total_mass (bit for bit), out[3k + 1], out[3k + 2] =
 * lbm_total_momentum. 24 bytes per lattice come back to the host, so a
 * caller can monitor a large batch every K steps. Returns LBM_EINVAL for a
 * NULL out, else like lbm_read_moments_all. */
int lbm_totals_all(lbm_ctx* ctx, double* out);

/* Sticky status bits LBM_FLAG_* of lattice `lat` (0 if clean). Synchronises. */
int lbm_status(lbm_ctx* ctx, int lat, uint32_t* flags);

/* Clear the sticky status bits of every lattice. */
int lbm_clear_status(lbm_ctx* ctx);

/* Wait for the context's stream; returns a sticky device error if any. */
int lbm_sync(lbm_ctx* ctx);

/* Checkpoint: size in bytes of the state blob, and save/load of the raw
 * distributions plus the step counter. A blob loads only into a context
 * created with the same lattices and precision. */
int lbm_state_size(lbm_ctx* ctx, size_t* bytes);
int lbm_save_state(lbm_ctx* ctx, void* buf, size_t bytes);
int lbm_load_state(lbm_ctx* ctx, const void* buf, size_t bytes);

/* Select the CTA tile of the step kernel by index into the built-in list
 * (lbm_tile_count() entries; lbm_tile_shape gives each node tile, lbm_tile_kind
 * the kernel that runs it):
 *   LBM_TILE_PLAIN      one CTA per tile;
 *   LBM_TILE_TMA        TMA-staged persistent, FP32, batches of at most 64
 *                       lattices; it takes the tiles two cells or more from
 *                       every lattice edge, the plain kernel of the same shape
 *                       the others;
 *   LBM_TILE_PIPELINED  persistent with the next tile's loads in flight during
 *                       the collision, FP32; it takes the full wall-free tiles,
 *                       the plain kernel of the same shape the others.
 * Results are bitwise identical for every tile. An FP32-only index on an FP64
 * context is LBM_EINVAL. */
#define LBM_TILE_PLAIN 0
#define LBM_TILE_TMA 1
#define LBM_TILE_PIPELINED 2
int lbm_tile_count(void);
int lbm_tile_shape(int index, int* tile_x, int* tile_y);
int lbm_tile_kind(int index, int* kind);
int lbm_set_tile(lbm_ctx* ctx, int index);

/* Time every built-in tile on this context's lattices for `steps` steps each
 * (CUDA events on the context's stream), keep the fastest and report its
 * index and the per-step milliseconds of each candidate (ms may be NULL,
 * else lbm_tile_count() doubles). The state is saved before and restored
 * after, so the simulation is unchanged. */
int lbm_autotune(lbm_ctx* ctx, int steps, int* best_index, double* ms);

/* Context introspection. */
int lbm_info(lbm_ctx* ctx, lbm_info_t* info);

/* Fill *view for lattice `lat` (see lbm_state_view). LBM_EINVAL for a null
 * argument or a lattice index out of range. No device work, no sync. */
int lbm_get_state_view(lbm_ctx* ctx, int lat, lbm_state_view* view);

/* ---- one lattice split into x-slabs (one context or rank per slab) ------
 * The scheme's step reads, at a node, its neighbours' state up to two
 * columns away (the pull of Eq. 5 reaches one column, and the psi of Eq. 13
 * on the one-cell ring around a node's neighbours needs their pulled
 * density, which reaches the next). A lattice split at x cuts into slabs
 * therefore exchanges, per face and step, LBM_HALO_ROWS = 12 values per row:
 * the nine populations of the edge column (the neighbour's halo node there
 * pulls those that point across the cut or along it, and reads the others
 * back where a link comes from a solid cell), and the three of the next
 * column that point across the cut.
 *
 * Mark lattice `lat` as one such slab: its x edges are no longer periodic;
 * the pulls across them read the frame columns x = -2, -1 (left neighbour)
 * and nx, nx + 1 (right neighbour) of the state, which lbm_halo_unpack
 * fills. Rows stay periodic (and may carry walls). Call before
 * lbm_init_fields; nx >= 2; with LBM_FP32_DEV the lattice's rho_ref must be
 * given (>= 0) and equal in every slab of the lattice, so that the stored
 * deviations they exchange mean the same.
 *   halo_mask  NULL, or 4*ny bytes: the wall mask of columns -2, -1, nx and
 *              nx + 1 (ny rows each, in that order), i.e. the neighbouring
 *              slabs' edge columns. NULL takes each edge column of the
 *              lattice's own mask as continuing across the cut. Must be
 *              NULL or clear for a lattice without a wall mask.
 * Afterwards, for this lattice:
 *   - lbm_init_fields takes (nx + 2) x ny arrays (x = -1 .. nx, x fastest):
 *     the slab's own field with the neighbouring slabs' edge columns on
 *     either side; it also fills the frame, so the first step needs no
 *     exchange. lbm_init_fields_all is refused for such a context.
 *   - lbm_step(ctx, n) takes n <= 1: exchange the halos between steps.
 *   - the read-outs (lbm_read_moments*) pull across the cut too: exchange
 *     after the last step before reading.
 *   - a checkpoint holds the slab's own nodes; exchange after a load. */
#define LBM_HALO_ROWS 12
int lbm_set_open_x(lbm_ctx* ctx, int lat, const uint8_t* halo_mask);

/* Halo exchange of a slab (asynchronous on `cuda_stream`, NULL: the
 * context's stream; device buffers of LBM_HALO_ROWS*ny elements of the
 * storage type: 4-byte floats for the FP32 precisions, 8-byte doubles for
 * LBM_FP64; rows k*ny .. k*ny + ny - 1 hold value k of every row y).
 *   lbm_halo_pack    writes into dev_out what the neighbour on `side`
 *                    (0: left, x < 0; 1: right, x >= nx) pulls from this
 *                    slab's current state.
 *   lbm_halo_unpack  writes the halo packed by the neighbour on `side` (its
 *                    pack of the opposite side) into this slab's frame.
 * The transport between the two (NCCL send/recv, a peer copy, a host copy)
 * is the caller's, and so is the ordering of a stream other than the
 * context's with it. Per step: step, pack both sides, exchange, unpack both
 * sides. To overlap the exchange with the step, split the step with
 * lbm_step_part: launch LBM_STEP_EDGE, pack (on another stream, ordered after
 * it), exchange and unpack there while LBM_STEP_INTERIOR runs, and order the
 * next step after the unpack. During a split step the calls address the
 * buffer the step writes: a pack needs the edge part launched first; an
 * unpack writes the frame the next step reads (no part writes it).
 * LBM_EINVAL for a lattice not open in x, a side other than 0 or 1, a null
 * buffer, or a pack before a split step's edge part. */
int lbm_halo_pack(lbm_ctx* ctx, int lat, int side, void* dev_out, void* cuda_stream);
int lbm_halo_unpack(lbm_ctx* ctx, int lat, int side, const void* dev_in, void* cuda_stream);

/* Largest ny accepted by lbm_total_mass_fp32_noalloc. */
#define LBM_NOALLOC_MAX_NY 32768

/* Mass of one FP32-stored lattice without allocating any memory (the paper
 * has no counterpart: this serves callers that cannot allocate device memory
 * when they need the check, such as applications whose own allocator owns all
 * device memory, or loops that must not wait in the driver's allocator).
 *   f_dev      device pointer to the lattice's nine FP32 planes in the
 *              library's layout: plane a at f_dev + a*ny*pitch, node (x, y) at
 *              y*pitch + x, pitch = round_up(nx, 32) (the layout of a
 *              lbm_save_state blob's distribution section).
 *   nx, ny     lattice size, 1 <= ny <= LBM_NOALLOC_MAX_NY and
 *              9 * ny * round_up(nx, 32) < 2^31; other sizes are rejected with
 *              LBM_EINVAL.
 *   rho_ref    the deviation reference the values are stored against (0 for
 *              plain FP32 storage).
 *   mask_dev   NULL, or ny*pitch device bytes, nonzero = solid (not counted).
 *   mass_dev   device pointer to one double: receives the sum over fluid nodes
 *              of rho_ref + the nine stored values, reduced in FP64 in a fixed
 *              order.
 *   cuda_stream  stream to run on (NULL: legacy default stream); the call is
 *              asynchronous and returns LBM_OK once the work is enqueued.
 * The partial sums live in one fixed device array of LBM_NOALLOC_MAX_NY/8
 * doubles (32 KiB) that every device which loads the library holds until the
 * process exits; no cudaMalloc, cudaFree or allocating library call is made.
 * The first call on each device (and again under each new CUDA context, e.g.
 * after cudaDeviceReset) looks that array's device address up
 * (cudaGetSymbolAddress) with the device current; make that first call
 * before any stream capture. All calls share the array: calls whose work may
 * overlap on the GPU (different streams without ordering) race on it.
 * Errors: LBM_EINVAL for null pointers or sizes out of range; LBM_ECUDA, with
 * the CUDA error named, when a launch fails or when an error left by earlier
 * CUDA work is pending (that error is left in place, not cleared). */
int lbm_total_mass_fp32_noalloc(const float* f_dev, int nx, int ny, double rho_ref,
                                const uint8_t* mask_dev, double* mass_dev, void* cuda_stream);

/* Message of the last failed call on this thread ("" if none). */
const char* lbm_last_error(void);

/* Release the context and its device memory (NULL is ignored). */
void lbm_destroy(lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* PAPER_1605_01800_GB300_LBM_H */
