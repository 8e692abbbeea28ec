/*
 * lbm.h -- C ABI of liblbm.so: the D2Q9I lattice-BGK stream-and-collide update
 * on one GB300 (sm_103a), after PortLBM (arXiv 2607.20650).
 *
 * The method (Sec. 3.1): Eq. (1), the BGK lattice Boltzmann equation
 *   f_i(r + c_i, t + 1) = f_i(r, t) - (1/tau) [f_i(r, t) - f_i^eq(r, t)],
 * with the incompressible D2Q9I equilibrium of Eq. (2)
 *   f_i^eq = w_i [rho + 3 v.c_i + 9/2 (v.c_i)^2 - 3/2 v^2],  v = sum_i f_i c_i,
 * directions i = 0..8 = SW, S, SE, W, rest, E, NW, N, NE (Fig. 2), i.e.
 * c_i = (i%3 - 1, i/3 - 1), opposite(i) = 8 - i. Half-way bounce-back at
 * fluid-solid links; Sec. 3.1 boundary kinds plus the edge conditions below.
 *
 * Conventions shared by every call:
 *  - Node index n = y*nx + x (x fastest), 0 <= x < nx, 0 <= y < ny.
 *  - Populations are stored as deviations h_i = f_i - w_i from the rest
 *    weights ("shifted" storage) in every precision.
 *  - The stored state after k updates holds post-collision populations.
 *    "Moments of update k" are rho and v computed inside update k from the
 *    pulled pre-collision values, with v = sum_i f_i c_i + F/2 (Guo force).
 *  - Ownership: the library never allocates device memory. The caller
 *    passes one device workspace (size from lbm_workspace_bytes) and a CUDA
 *    stream (cudaStream_t as void*, NULL = legacy default stream); all
 *    device work is enqueued on that stream. Host arrays stay caller-owned;
 *    the mask is copied during lbm_create. Host-side handles are malloc'ed
 *    and freed by lbm_destroy / lbm_batch_destroy.
 *  - Errors: every call returns an lbm_status; nothing throws or exits.
 *    lbm_last_error() returns a thread-local message for the last failure.
 *  - The one device-side wait is NSOL's wait for its tile's tensor copy,
 *    bounded (LBM_ECUDA at the next check if it runs out); host waits are
 *    bounded by lbm_wait.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,        /* bad argument (message in lbm_last_error) */
    LBM_ENOMEM = 2,        /* workspace too small, or host allocation failed */
    LBM_ECUDA = 3,         /* a CUDA runtime call failed */
    LBM_EDIVERGED = 4,     /* a non-finite density was seen since the last check */
    LBM_ETIMEOUT = 5,      /* lbm_wait ran out of time; work is still in flight */
    LBM_EUNSUPPORTED = 6   /* valid but not implemented combination */
} lbm_status;

/* Population layouts of Sec. 3.2 / Fig. 2 (addresses in elements, N = nx*ny):
 *   STREAM    (SoA)   addr(n, i) = i*N + n
 *   BUNDLE    (SoAoS) addr(n, i) = (i/3)*3N + 3n + i%3
 *               bundles {SW,S,SE}, {W,rest,E}, {NW,N,NE}
 *   COLLISION (AoS)   addr(n, i) = 9n + i                                    */
typedef enum { LBM_LAYOUT_STREAM = 0, LBM_LAYOUT_BUNDLE = 1, LBM_LAYOUT_COLLISION = 2 } lbm_layout;

/* Algorithms of Sec. 3.3:
 *   LPTL linear pull, two lattices (1-D launch, block size from the runtime)
 *   NPTL 2-D tiles (tile_x * tile_y nodes, padded grid), pull, two lattices
 *   NPOL 2-D tiles, pull, one lattice: a node's pulled values are held in
 *        registers, a block barrier precedes the in-place writes, and values
 *        crossing tile edges travel through a buffer grid double-buffered by
 *        step parity
 *   NSOL 2-D tiles, swap streaming (one lattice, populations stored in
 *        opposite slots), in-tile exchanges in shared memory, the same buffer
 *        grid across tiles.
 * All four produce bit-identical states at equal storage precision.
 * Beyond the paper's four (Sec. 3.3 names it among state-of-the-art schemes,
 * Sec. 6 as future work):
 *   AA   in-place streaming with one lattice and no buffer grid (the AA
 *        pattern): updates alternate between a phase that pulls from and
 *        pushes to neighbours and a phase that only touches the node's own
 *        slots. Same bits as the others. The state (lbm_read_populations,
 *        lbm_write_populations, lbm_mass, lbm_force) is accessible after an
 *        even number of updates only (LBM_EINVAL otherwise); zero-gradient
 *        outflow is not supported (LBM_EUNSUPPORTED); not in batches.       */
typedef enum { LBM_LPTL = 0, LBM_NPTL = 1, LBM_NPOL = 2, LBM_NSOL = 3, LBM_AA = 4 } lbm_algo;

/* Storage precision of h; arithmetic is FP64 for F64 and FP32 otherwise. */
typedef enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16S = 2, LBM_BF16S = 3 } lbm_storage;

/* Rounding of the FP32 -> F16S/BF16S store: round-to-nearest-even, or
 * stochastic rounding keyed on (seed, update index, n, i), so results do not
 * depend on layout or algorithm. Ignored for F64 / F32.                      */
typedef enum { LBM_ROUND_RNE = 0, LBM_ROUND_SR = 1 } lbm_rounding;

/* Edge conditions. SOUTH/NORTH: PERIODIC (both), WALL, FREESLIP.
 * WEST: PERIODIC (with EAST), WALL, INLET_ZOUHE, INLET_EQ, INLET_EQ_NEUMANN, OUTFLOW_ZG.
 * EAST: PERIODIC (with WEST), WALL, OUTFLOW_ZG, OUTLET_PRESSURE.
 *   WALL        half-way bounce-back one half cell outside the edge
 *   FREESLIP    specular reflection: the value pulled across the edge is the
 *               neighbour row's mirror population of the node's own row
 *   INLET_ZOUHE incompressible Zou-He velocity inlet (u_in) in column 0
 *   INLET_EQ    column 0 set to f^eq(rho = 1, u_in) (Sec. 3.1 Dirichlet)
 *   OUTFLOW_ZG  zero gradient: the pulled source column is clamped
 *   INLET_EQ_NEUMANN  column 0 set to f^eq(rho of node (1, y) in the previous
 *               state, u_in): Sec. 3.1's equilibrium inlet with a Neumann
 *               density (one-lattice algorithms need tile_x >= 2; not AA)
 *   OUTLET_PRESSURE  Zou-He pressure outlet in column nx-1 (Sec. 3.1's
 *               "adapted Zou and He" outlet): rho = rho_out, v_y = 0       */
typedef enum {
    LBM_BC_PERIODIC = 0, LBM_BC_WALL = 1, LBM_BC_FREESLIP = 2,
    LBM_BC_INLET_ZOUHE = 3, LBM_BC_INLET_EQ = 4, LBM_BC_OUTFLOW_ZG = 5,
    LBM_BC_INLET_EQ_NEUMANN = 6, LBM_BC_OUTLET_PRESSURE = 7
} lbm_bc;

#define LBM_FLAG_NO_GRAPH 0x1u   /* lbm_step launches kernels one by one */
#define LBM_FLAG_TWO_NODES_PER_THREAD 0x2u  /* NPTL, F64/F32 storage, even tile_y: two nodes
                                               per thread, rows y and y + tile_y/2 (default:
                                               one node per thread) */
#define LBM_FLAG_NO_STAGING 0x4u  /* NPTL, collision layout: no shared-memory staging of
                                     row spans (default when tile_x % 32 == 0) */
#define LBM_FLAG_WIDE_OFFSETS 0x8u  /* D3Q19: 64-bit addressing for every pull, the path
                                       lattices too large for 32-bit offset tables take */
#define LBM_FLAG_NO_PREFETCH 0x10u  /* LPTL/NPTL/AA: no L2 prefetch of the records pulled
                                       by the blocks launched next (default: on for 32-bit
                                       storage in the stream and bundle layouts when a
                                       lattice exceeds the L2 cache) */
#define LBM_FLAG_NO_PAIRS 0x20u  /* LPTL/NPTL, F16S/BF16S storage: one node per thread
                                    with scalar FP32 arithmetic (default when nx is even,
                                    the layout is bundle and tile_x is even: two
                                    adjacent nodes per thread with packed FP32
                                    arithmetic; the results are bit-identical) */
#define LBM_FLAG_NO_TMA 0x40u  /* NSOL, F32 storage: stage each tile with per-thread loads
                                  (default when the layout is stream or bundle, nx and
                                  tile_x are multiples of 4 and the tile's rows fit one
                                  tensor copy: one tensor-memory-access copy of the tile's
                                  populations into shared memory per block; bit-identical) */

typedef struct lbm_params {
    int32_t nx, ny;          /* lattice size; nx*ny < 2^32 */
    double tau;              /* relaxation time, > 1/2 (omega = 1/tau in FP64) */
    double force[2];         /* Guo body force (lattice units) */
    double u_in[2];          /* inlet velocity for INLET_* edges */
    int32_t bc_west, bc_east, bc_south, bc_north;   /* lbm_bc */
    int32_t layout;          /* lbm_layout */
    int32_t algo;            /* lbm_algo */
    int32_t storage;         /* lbm_storage */
    int32_t rounding;        /* lbm_rounding */
    uint64_t seed;           /* stochastic-rounding seed */
    int32_t tile_x, tile_y;  /* NPTL/NPOL/NSOL tile (0, 0 = 32 x 8); tile_x*tile_y <= 512;
                                tile_x a multiple of 32 keeps warps on one row */
    uint32_t flags;          /* LBM_FLAG_* */
    double rho_out;          /* outlet density for OUTLET_PRESSURE (> 0) */
} lbm_params;

typedef struct lbm_lattice lbm_lattice;

/* Bytes of device workspace lbm_create needs for these parameters. */
lbm_status lbm_workspace_bytes(const lbm_params *p, size_t *bytes);

/* Lay a lattice out in d_workspace (>= lbm_workspace_bytes, 256-byte aligned,
 * caller-owned, must outlive the lattice). mask_host: N bytes, nonzero =
 * solid node (copied). A fluid node whose eight neighbours are all solid
 * or wall is treated as solid. State after create: rho = 1, v = 0. */
lbm_status lbm_create(const lbm_params *p, const uint8_t *mask_host, void *d_workspace,
                      size_t bytes, void *cuda_stream, lbm_lattice **out);

/* Initial state f = f^eq(rho, v) on fluid nodes (Eq. (2)), evaluated in FP64
 * and rounded once to the storage type. Host arrays of N doubles; NULL rho
 * means 1, NULL ux/uy mean 0. Resets the update counter. Synchronous. */
lbm_status lbm_init(lbm_lattice *L, const double *rho, const double *ux, const double *uy);

/* Enqueue nsteps updates (Eq. (1)) on the stream; asynchronous. With
 * want_moments != 0 the last update also stores its moments (rho, ux, uy) in
 * the workspace for lbm_read_moments / lbm_moments_device. Uses cached CUDA
 * graphs of whole step blocks unless LBM_FLAG_NO_GRAPH is set. */
lbm_status lbm_step(lbm_lattice *L, int64_t nsteps, uint32_t want_moments);

/* Synchronise the stream; LBM_EDIVERGED if a non-finite density was seen
 * (the flag is then cleared). */
lbm_status lbm_sync(lbm_lattice *L);

/* Wait at most timeout_s seconds for all enqueued work; LBM_ETIMEOUT if it is
 * still running (nothing is cancelled), otherwise as lbm_sync. */
lbm_status lbm_wait(lbm_lattice *L, double timeout_s);

/* Moments of the last update that stored them (or of lbm_init), as host
 * doubles, N each (solid nodes: rho = 1, v = 0); a NULL array is skipped.
 * Synchronous. Page-locked destinations (cudaHostAlloc, cudaHostRegister)
 * are written by the device directly; pageable ones of more than 64 MB per
 * field go through page-locked staging the lattice allocates on first use
 * (128 MB of host memory, freed by lbm_destroy). */
lbm_status lbm_read_moments(lbm_lattice *L, double *rho, double *ux, double *uy);

/* Same moments as FP32 device arrays (N each), enqueued on the stream. */
lbm_status lbm_moments_device(lbm_lattice *L, float *d_rho, float *d_ux, float *d_uy);

/* Total mass sum over fluid nodes of rho = 1 + sum_i h_i of the stored state,
 * reduced in FP64 on the GPU in a fixed order. Synchronous. */
lbm_status lbm_mass(lbm_lattice *L, double *out);

/* Momentum-exchange force on the body: sum over links from a fluid node x to
 * a node x + c_i with d_body[x + c_i] != 0 of 2 c_i f*_i(x), f* = w + h the
 * stored post-collision populations; FP64 on the GPU, fixed order.
 * d_body: device array of N bytes (NULL = every solid node). Synchronous. */
lbm_status lbm_force(lbm_lattice *L, const uint8_t *d_body, double out[2]);

/* Copy the state to / from host memory in canonical order h[i*N + n],
 * as = LBM_F64 (double) or LBM_F32 (float). Writes round to the storage
 * type (via FP32 for F16S/BF16S, nearest-even). Synchronous. */
lbm_status lbm_read_populations(lbm_lattice *L, void *host, int32_t as);
lbm_status lbm_write_populations(lbm_lattice *L, const void *host, int32_t as);

/* Face exchange between x-slabs of one lattice (the domain split behind the
 * multi-GPU extension of Sec. 6). A slab holds whole columns of the lattice
 * plus one ghost column on each face it shares with another slab; the pull
 * update (Eq. (1)) of the column next to a ghost column reads from it only the
 * three populations that cross the face, the directions with c_ix = sense
 * (sense = +1: SE, E, NE; -1: SW, W, NW, in that order, Fig. 2). After every
 * update, pack those three values of the sender's boundary column and unpack
 * them into the receiver's ghost column; the slabs' interiors then evolve
 * bit for bit like the undivided lattice (same storage, layout, algorithm;
 * with LBM_ROUND_SR the draws are keyed on each slab's own node index).
 *   x      column of this lattice, 0 <= x < nx
 *   sense  +1 or -1 (which three directions)
 *   d_buf  device buffer of 3 * ny stored values (8, 4, 2, 2 bytes each for
 *          F64, F32, F16S, BF16S), caller-owned; value k * ny + y is
 *          direction k of node (x, y), bits as stored.
 * lbm_face_pack copies the column of the current state into d_buf;
 * lbm_face_unpack copies d_buf into it (NPOL / NSOL: then refreshes the
 * buffer grid from the lattice). Both enqueue on the lattice's stream and
 * return at once. LBM_EINVAL: NULL argument, x or sense out of range, or the
 * AA algorithm (its stored state alternates between two forms). */
lbm_status lbm_face_pack(lbm_lattice *L, int32_t x, int32_t sense, void *d_buf);
lbm_status lbm_face_unpack(lbm_lattice *L, int32_t x, int32_t sense, const void *d_buf);

/* Every message of an exchange between lattices held by one process, in one
 * launch: message k copies the three populations crossing x -> x + sense[k]
 * of column xs[k] of src[k] into column xd[k] of dst[k] (what
 * lbm_face_pack of src[k] followed by lbm_face_unpack of dst[k] does, with
 * no buffer in between), then the buffer grid of every NPOL / NSOL receiver
 * is refreshed once. All arrays are host arrays of `count` entries,
 * 0 <= count <= 64; every lattice must have the same ny, storage, layout
 * and algorithm. Enqueued on cuda_stream (cudaStream_t as void*): the
 * caller orders it after the updates of every lattice involved, e.g. by
 * keeping them all on that stream. LBM_EINVAL: as lbm_face_pack, a count
 * out of range, or lattices that differ. */
lbm_status lbm_face_exchange(int32_t count, lbm_lattice *const *src, const int32_t *xs,
                             lbm_lattice *const *dst, const int32_t *xd, const int32_t *sense,
                             void *cuda_stream);

typedef struct lbm_info {
    int64_t cells, fluid_cells;
    int64_t steps;                 /* updates done since lbm_init */
    int32_t tile_x, tile_y;        /* tile used (LPTL: block size, 1) */
    int32_t aux;                   /* lbm_get_info: L2 prefetch distance (LPTL: nodes, NPTL
                                      and AA: rows; 0 = off); NSOL: 1 when tiles are staged
                                      by tensor copies (LBM_FLAG_NO_TMA); lbm3_get_info: see
                                      there */
    double bytes_per_update;       /* algorithmic DRAM bytes of one update */
    size_t workspace_bytes;
} lbm_info;
lbm_status lbm_get_info(lbm_lattice *L, lbm_info *out);

void lbm_destroy(lbm_lattice *L);
const char *lbm_last_error(void);

/* Element offset of population i of node n in a layout (host-side copy of
 * the device index map, for checks). Returns -1 on bad arguments. */
int64_t lbm_layout_index(int32_t layout, int64_t N, int64_t n, int32_t i);

/* Store codec on device arrays, enqueued on stream: d_in[k] (FP32) is
 * rounded to storage (F16S or BF16S) as population i = k % 9 of node
 * n = k / 9 at update index t (the keys of LBM_ROUND_SR), written to d_out
 * (2 bytes each), then decoded back to FP32 in d_back (may be NULL). */
lbm_status lbm_quantize(int32_t storage, int32_t rounding, uint64_t seed, int64_t t,
                        const float *d_in, void *d_out, float *d_back, int64_t count,
                        void *cuda_stream);

/* Total mass like lbm_mass, for callers that cannot provide device memory:
 * code hosted by a framework that owns every device allocation and forbids
 * direct cudaMalloc, or loops that must not incur an allocation's implicit
 * synchronisation. The paper has no counterpart; this is a library utility.
 * d_h: canonical FP32 deviations h[i*N + n] (9N floats, device).
 * d_solid: N bytes (device), nonzero = a node that is not counted. It must be
 * the effective solid set that lbm_mass skips: the given solid nodes plus
 * every fluid node whose eight pulls all bounce (no open neighbour; such a
 * node is treated as solid). A raw geometry mask counts each such enclosed
 * node as rho = 1 + sum(h) = 1, i.e. one more per node.
 * out: host double, written before return.
 * Allocates nothing: its scratch is a fixed device array inside the library
 * (one per GPU, kept until exit), so N is limited to 134,217,728 nodes
 * (LBM_EINVAL beyond). All calls share that array: calls whose GPU work
 * overlaps race. The first call on a device does the set-up: it looks the
 * array's device address up with that device current and keeps it for the
 * rest of the process; make that first call before any stream capture. The
 * kept address is not refreshed after cudaDeviceReset: do not call this
 * entry point after resetting the device in the same process. Every call
 * copies the result to host memory and synchronises cuda_stream before it
 * returns. The sum is the same quantity as lbm_mass in a different fixed
 * order: it agrees with lbm_mass to round-off, and repeated calls on the
 * same data return identical bits. */
lbm_status lbm_mass_f32_noalloc(const float *d_h, const uint8_t *d_solid, int64_t N, double *out,
                                void *cuda_stream);

/* ---------------------------------------------------------------- masks
 * Host-side generator of the benchmark families' solid masks (Sec. 4:
 * Hagen-Poiseuille channel, obstacles, porous media, a wing at an angle of
 * attack) for callers that do not build masks themselves. No GPU work. The
 * mask is row-major, mask[y nx + x] (3-D: mask[(z ny + y) nx + x]), 1 =
 * solid, caller-owned (nx * ny bytes), overwritten (lbm_mask_disc: ORed
 * into). Seeded generators draw from splitmix64 streams (Steele, Lea & Flood,
 * 2014) seeded with seed ^ mix(stream * gamma + gamma), doubles (x >> 11)
 * 2^-53: the same masks as the package's Python input generator. LBM_EINVAL
 * on a NULL mask, nx * ny >= 2^32 or out-of-range parameters.            */
/* Solid rows y = 0 and y = ny - 1. */
lbm_status lbm_mask_channel_walls(int32_t nx, int32_t ny, uint8_t *mask);
/* Nodes with (x - xc)^2 + (y - yc)^2 <= r^2 (integer node coordinates) set
 * to 1; periodic != 0 wraps the disc around the domain, else clips it. */
lbm_status lbm_mask_disc(int32_t nx, int32_t ny, double xc, double yc, double r, int32_t periodic,
                         uint8_t *mask);
/* Random overlapping discs on a periodic domain (stream 1: three uniforms
 * per disc, centre (u nx, v ny), radius rmin + (rmax - rmin) w, batches of
 * 256) until at least solid_fraction of the nodes are solid. The 134M-node
 * porous workload: 16384 x 8192, seed 3, radii 8-32, fraction 0.4. */
lbm_status lbm_mask_porous_discs(int32_t nx, int32_t ny, uint64_t seed, double rmin, double rmax,
                                 double solid_fraction, uint8_t *mask);
/* NACA 4-digit airfoil (camber m at chord fraction p, thickness t: 2412 is
 * 0.02, 0.4, 0.12) of the given chord in nodes, from the closed-form
 * thickness (closed trailing edge) and camber-line equations with n_points
 * cosine-spaced points per side, leading edge at (nx/4, ny/2), rotated
 * nose-up by aoa_deg about the quarter chord; nodes inside the outline
 * (even-odd rule) are solid. Transcendental functions come from the C
 * library, so a node within rounding distance of the outline may differ
 * from another implementation's. */
lbm_status lbm_mask_naca4(int32_t nx, int32_t ny, double chord, double m, double p, double t,
                          double aoa_deg, int32_t n_points, uint8_t *mask);
/* Random overlapping spheres on a periodic box (stream 5: four uniforms per
 * sphere, batches of 256) until at least solid_fraction is solid. */
lbm_status lbm3_mask_porous_spheres(int32_t nx, int32_t ny, int32_t nz, uint64_t seed, double rmin,
                                    double rmax, double solid_fraction, uint8_t *mask);

/* ---------------------------------------------------------------- batches
 * Many independent lattices advanced together, one persistent launch per
 * update over a packed list of tiles of every case, captured into CUDA
 * graphs. Per case: its own size, tau, force, inlet, edges and mask; layout,
 * algorithm and tile may be given or left to the autotuner (-1 / 0).
 * Results per case are bit-identical to a single-lattice run.               */
typedef struct lbm_batch lbm_batch;

#define LBM_AUTO (-1)

/* Measured cost table for the autotuner, filled by lbm_tune (or zeroed to
 * use the built-in model). ns_per_cell[storage-independent layout][algo],
 * ns_per_tile: per-tile overhead. */
typedef struct lbm_tuning {
    double ns_per_cell[3][4];
    double ns_per_tile;
    int32_t valid;
    int32_t reserved;
} lbm_tuning;

/* Time the batch kernel for every (layout, algo) on eight copies of a probe
 * case in the caller's workspace (at least lbm_tune_workspace_bytes(probe))
 * and fill *out. Synchronous. */
lbm_status lbm_tune_workspace_bytes(const lbm_params *probe, size_t *bytes);
lbm_status lbm_tune(const lbm_params *probe, const uint8_t *mask_host, void *d_workspace,
                    size_t bytes, void *cuda_stream, lbm_tuning *out);

/* Resolve LBM_AUTO layout/algo and 0 tiles of every case with the
 * autotuner (tuning may be NULL: built-in model); params is updated in
 * place. All cases must share storage type. One layout/algorithm pair is
 * given to every case (the batch then runs a kernel specialised for it)
 * unless per-case pairs are predicted faster by more than 1.6x, the
 * measured cost of the general mixed-pair kernel. */
lbm_status lbm_batch_plan(int32_t ncases, lbm_params *params, const lbm_tuning *tuning);

lbm_status lbm_batch_workspace_bytes(int32_t ncases, const lbm_params *params, size_t *bytes);
lbm_status lbm_batch_create(int32_t ncases, const lbm_params *params,
                            const uint8_t *const *masks_host, void *d_workspace, size_t bytes,
                            void *cuda_stream, lbm_batch **out);
/* Initial equilibrium of case c from host arrays (NULL = rho 1 / v 0). */
lbm_status lbm_batch_init(lbm_batch *B, int32_t c, const double *rho, const double *ux,
                          const double *uy);
lbm_status lbm_batch_step(lbm_batch *B, int64_t nsteps, uint32_t want_moments);
lbm_status lbm_batch_sync(lbm_batch *B);
lbm_status lbm_batch_read_moments(lbm_batch *B, int32_t c, double *rho, double *ux, double *uy);
lbm_status lbm_batch_read_populations(lbm_batch *B, int32_t c, void *host, int32_t as);
/* Entries in the packed work list (4 tiles of a two-lattice case or one tile
 * of a one-lattice case each), the persistent grid size, and total nodes. */
lbm_status lbm_batch_get_info(lbm_batch *B, int64_t *items, int32_t *grid, int64_t *cells);
void lbm_batch_destroy(lbm_batch *B);

/* ---------------------------------------------------------------- D3Q19
 * Three-dimensional lattices (Sec. 6 names the 3-D extension as future
 * work) with the method of Sec. 3.1: Eq. 1 BGK with the Eq. 2 incompressible
 * equilibrium (v = sum f c) on the 19 velocities of {-1,0,1}^3 with
 * |c|^2 <= 2, numbered lexicographically in (c_z, c_y, c_x): opposite(i) =
 * 18 - i, rest i = 9, weights 1/3, 1/18 (faces), 1/36 (edges). Node index
 * n = (z ny + y) nx + x; h = f - w is stored as in 2-D.
 * Layouts (lbm_layout): STREAM h[i N + n]; COLLISION h[19 n + i]; BUNDLE
 * groups the directions with the same (c_y, c_z), i.e. the same source row:
 * {0}, {1,2,3}, {4}, {5,6,7}, {8,9,10}, {11,12,13}, {14}, {15,16,17}, {18},
 * a group of size s starting at direction b stored at b N + s n + (i - b).
 * Algorithms: LPTL and NPTL (3-D tiles tile_x * tile_y * tile_z <= 512,
 * 0,0,0 = 128 x 1 x 1; tile_z <= 64), two lattices; NPOL (one lattice and a
 * buffer grid: per tile and parity, the five populations leaving each node
 * of each of the six tile faces, 2 x tiles x 10 (ty tz + tx tz + tx ty)
 * values); NSOL (one lattice, swap streaming: population i of a node kept
 * in its slot opp(i), the tile staged in shared memory, the same buffer
 * grid as NPOL); AA (the same tiles, one lattice, as in 2-D: populations and mass
 * accessible after an even number of updates only, LBM_EINVAL otherwise;
 * needs 32-bit offset tables, i.e. roughly 19 N < 2^31, LBM_EUNSUPPORTED
 * otherwise). All produce the same bits at equal storage. Faces per axis: PERIODIC or WALL
 * (half-way bounce-back); on x the west face may instead be an equilibrium
 * inlet (LBM_BC_INLET_EQ: the x = 0 plane set to f^eq(rho = 1, u_in) before
 * the collision, Sec. 3.1's Dirichlet equilibrium inlet) with the east face
 * bc_x_east a wall or a zero-gradient outflow (LBM_BC_OUTFLOW_ZG, the pulled
 * source plane clamped), or both x faces may be outflows; pulls are mapped
 * in z, then y, then x; inlet and outflow faces with LPTL and NPTL only
 * (LBM_EUNSUPPORTED otherwise). Solid mask nodes bounce back; a fluid node
 * whose 18 pulls all bounce is treated as solid. Storage, rounding, Guo
 * force, graphs and errors as in 2-D. Workspace: 2 x 19 N elements, 4 N
 * bytes of links, 4 N compute-type moments, small scratch.               */
typedef struct lbm3_params {
    int32_t nx, ny, nz;      /* lattice size; nx*ny*nz < 2^32 */
    double tau;              /* relaxation time, > 1/2 */
    double force[3];         /* Guo body force */
    int32_t bc_x, bc_y, bc_z;   /* LBM_BC_PERIODIC or LBM_BC_WALL, both faces of the axis;
                                   bc_x also LBM_BC_INLET_EQ or LBM_BC_INLET_ZOUHE (west face,
                                   see bc_x_east) or LBM_BC_OUTFLOW_ZG (both x faces) */
    int32_t layout, algo, storage, rounding;   /* algo: LBM_LPTL, LBM_NPTL, LBM_NPOL, LBM_NSOL
                                                  or LBM_AA */
    uint64_t seed;
    int32_t tile_x, tile_y, tile_z;
    uint32_t flags;          /* LBM_FLAG_NO_GRAPH, LBM_FLAG_WIDE_OFFSETS, LBM_FLAG_NO_PAIRS */
    int32_t bc_x_east;       /* east x face after an inlet west face: LBM_BC_OUTFLOW_ZG,
                                LBM_BC_WALL or LBM_BC_OUTLET_PRESSURE (ignored otherwise:
                                both x faces are bc_x) */
    double u_in[3];          /* inlet velocity for bc_x = LBM_BC_INLET_EQ or LBM_BC_INLET_ZOUHE */
    double rho_out;          /* outlet density for bc_x_east = LBM_BC_OUTLET_PRESSURE (> 0) */
} lbm3_params;

typedef struct lbm3_lattice lbm3_lattice;

lbm_status lbm3_workspace_bytes(const lbm3_params *p, size_t *bytes);
/* mask_host: N bytes, nonzero = solid (host, read during the call); the
 * workspace (256-byte aligned device memory of lbm3_workspace_bytes) and
 * the stream stay the caller's. Initial state: rho = 1, v = 0. */
lbm_status lbm3_create(const lbm3_params *p, const uint8_t *mask_host, void *d_workspace, size_t bytes,
                       void *cuda_stream, lbm3_lattice **out);
/* Equilibrium from host arrays of N doubles (each may be NULL: rho 1, v 0).
 * Synchronous; resets the update count. */
lbm_status lbm3_init(lbm3_lattice *L, const double *rho, const double *ux, const double *uy,
                     const double *uz);
/* Enqueue nsteps updates; with want_moments the last writes rho, v. */
lbm_status lbm3_step(lbm3_lattice *L, int64_t nsteps, uint32_t want_moments);
lbm_status lbm3_sync(lbm3_lattice *L);
/* Host arrays of N doubles (any may be NULL); solid nodes read rho 1, v 0. */
lbm_status lbm3_read_moments(lbm3_lattice *L, double *rho, double *ux, double *uy, double *uz);
/* Canonical host array [i N + n] (19 N values of type as). */
lbm_status lbm3_read_populations(lbm3_lattice *L, void *host, int32_t as);
lbm_status lbm3_write_populations(lbm3_lattice *L, const void *host, int32_t as);
/* Total mass sum over fluid nodes of sum_i f_i, accumulated in FP64. */
lbm_status lbm3_mass(lbm3_lattice *L, double *out);
/* Momentum-exchange force, as lbm_force in 3-D: sum over links from a fluid
 * node x to x + c_i with d_body[x + c_i] != 0 (links across a wall face
 * skipped) of 2 c_i f*_i(x), f* = w + h of the stored state; FP64, fixed
 * order. d_body: device array of N bytes (NULL = every solid node).
 * Synchronous; AA: after an even number of updates only. */
lbm_status lbm3_force(lbm3_lattice *L, const uint8_t *d_body, double out[3]);
/* cells, fluid_cells, steps, tile (tile_y = tile_y * tile_z), bytes per
 * update; aux bit 0: pulls use 64-bit addressing (large lattices or
 * LBM_FLAG_WIDE_OFFSETS; clear with the 32-bit offset tables); bit 1: LPTL
 * or NPTL with 16-bit storage update two x-adjacent nodes per thread
 * (stream or bundle layout, nx and tile_x even, 32-bit offset tables, no
 * LBM_FLAG_NO_PAIRS; bit-identical to one node per thread). */
lbm_status lbm3_get_info(lbm3_lattice *L, lbm_info *out);
void lbm3_destroy(lbm3_lattice *L);
int64_t lbm3_layout_index(int32_t layout, int64_t N, int64_t n, int32_t i);

/* Face exchange between x-slabs of a D3Q19 box, as lbm_face_pack /
 * lbm_face_unpack / lbm_face_exchange in 2-D: a slab holds whole x-planes
 * plus a ghost plane on each face it shares with another; after every update
 * the five populations with c_x = sense (in direction order) of the sender's
 * boundary plane x go into the receiver's ghost plane. d_buf: device buffer
 * of 5 * ny * nz stored values, value k * (ny nz) + (z ny + y) = direction k
 * of node (x, y, z), bits as stored. Same rules, errors and stream use as
 * the 2-D calls (AA refused; NPOL / NSOL receivers refresh their buffer
 * grid); every lattice of one lbm3_face_exchange has the same ny * nz,
 * storage, layout and algorithm. */
lbm_status lbm3_face_pack(lbm3_lattice *L, int32_t x, int32_t sense, void *d_buf);
lbm_status lbm3_face_unpack(lbm3_lattice *L, int32_t x, int32_t sense, const void *d_buf);
lbm_status lbm3_face_exchange(int32_t count, lbm3_lattice *const *src, const int32_t *xs,
                              lbm3_lattice *const *dst, const int32_t *xd, const int32_t *sense,
                              void *cuda_stream);

/* ---------------------------------------------------------------- D3Q19 batches
 * Many independent boxes advanced together: one launch per update over a
 * packed list of work items of every case (a tile for NPTL, NPOL and NSOL,
 * 256 consecutive nodes for LPTL), captured into CUDA graphs of 64 updates.
 * Per case: its own size, tau, force, faces, inlet/outlet, rounding, seed and
 * mask. Shared by every case (LBM_EINVAL otherwise): storage, layout,
 * algorithm (LPTL, NPTL, NPOL or NSOL; AA: LBM_EUNSUPPORTED) and, for the
 * tiled algorithms, the tile. Every case must fit the 32-bit offset tables
 * (roughly 19 N < 2^31, no LBM_FLAG_WIDE_OFFSETS; LBM_EUNSUPPORTED
 * otherwise). Results per case are bit-identical to a single-box run of the
 * same parameters, stochastic rounding included (the batch's update counter
 * starts at 0 like a box's).
 * Workspace: lbm3_batch_workspace_bytes of 256-byte aligned device memory,
 * the caller's, as is the stream. A divergence in any case is reported by
 * lbm3_batch_sync and the read calls as LBM_EDIVERGED.                    */
typedef struct lbm3_batch lbm3_batch;

lbm_status lbm3_batch_workspace_bytes(int32_t ncases, const lbm3_params *params, size_t *bytes);
/* params, masks_host: ncases entries; mask c holds nx ny nz bytes of case c
 * (nonzero = solid, host, read during the call). Initial state of every
 * case: rho = 1, v = 0. */
lbm_status lbm3_batch_create(int32_t ncases, const lbm3_params *params, const uint8_t *const *masks_host,
                             void *d_workspace, size_t bytes, void *cuda_stream, lbm3_batch **out);
/* Equilibrium of case c from host arrays (NULL: rho 1 / v 0); only before
 * the first lbm3_batch_step (LBM_EINVAL afterwards). Synchronous. */
lbm_status lbm3_batch_init(lbm3_batch *B, int32_t c, const double *rho, const double *ux, const double *uy,
                           const double *uz);
/* Enqueue nsteps updates of every case; with want_moments the last one
 * writes rho, v of every case. */
lbm_status lbm3_batch_step(lbm3_batch *B, int64_t nsteps, uint32_t want_moments);
lbm_status lbm3_batch_sync(lbm3_batch *B);
/* Case c, as lbm3_read_moments / lbm3_read_populations / lbm3_mass. */
lbm_status lbm3_batch_read_moments(lbm3_batch *B, int32_t c, double *rho, double *ux, double *uy, double *uz);
lbm_status lbm3_batch_read_populations(lbm3_batch *B, int32_t c, void *host, int32_t as);
lbm_status lbm3_batch_mass(lbm3_batch *B, int32_t c, double *out);
/* Work items per update, total nodes, total fluid nodes and algorithmic
 * bytes per update (the sum of the cases' lbm3_get_info figures); any
 * pointer may be NULL. */
lbm_status lbm3_batch_get_info(lbm3_batch *B, int64_t *items, int64_t *cells, int64_t *fluid_cells,
                               double *bytes_per_update);
void lbm3_batch_destroy(lbm3_batch *B);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
