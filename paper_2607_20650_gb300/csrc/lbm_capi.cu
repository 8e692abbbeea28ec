// C ABI of liblbm.so (declared in include/lbm.h): parameter checks, the
// workspace layout, update scheduling with cached CUDA graphs, host-side
// layout conversion for checkpoints, and the FP64 reductions.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "lbm.h"
#include "lbm_capi_internal.h"
#include "lbm_device.cuh"
#include "lbm_internal.h"

using namespace lbm;

// ------------------------------------------------------------ errors
static thread_local std::string g_last_error;

lbm_status lbm_fail(lbm_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

lbm_status lbm_cuda_fail(cudaError_t e, const char *where) {
    return lbm_fail(LBM_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

extern "C" const char *lbm_last_error(void) { return g_last_error.c_str(); }

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return lbm_cuda_fail(e_, #call); \
    } while (0)

// ------------------------------------------------------------ planning
const Ops *ops_for_storage(int storage) {
    switch (storage) {
        case LBM_F64: return &ops_f64();
        case LBM_F32: return &ops_f32();
        case LBM_F16S: return &ops_f16();
        case LBM_BF16S: return &ops_bf16();
    }
    return nullptr;
}

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

lbm_status lbm_check_params(const lbm_params *p) {
    if (!p) return lbm_fail(LBM_EINVAL, "params is NULL");
    if (p->nx < 1 || p->ny < 1) return lbm_fail(LBM_EINVAL, "nx, ny must be >= 1 (got %d, %d)", p->nx, p->ny);
    if ((uint64_t)p->nx * (uint64_t)p->ny >= (1ull << 32))
        return lbm_fail(LBM_EUNSUPPORTED, "nx*ny must be < 2^32");
    if (!(p->tau > 0.5)) return lbm_fail(LBM_EINVAL, "tau must be > 1/2 (got %g)", p->tau);
    if (!std::isfinite(p->force[0]) || !std::isfinite(p->force[1]) || !std::isfinite(p->u_in[0]) ||
        !std::isfinite(p->u_in[1]))
        return lbm_fail(LBM_EINVAL, "force and u_in must be finite");
    if (p->layout < 0 || p->layout > 2) return lbm_fail(LBM_EINVAL, "bad layout %d", p->layout);
    if (p->algo < 0 || p->algo > 4) return lbm_fail(LBM_EINVAL, "bad algo %d", p->algo);
    if (p->storage < 0 || p->storage > 3) return lbm_fail(LBM_EINVAL, "bad storage %d", p->storage);
    if (p->rounding < 0 || p->rounding > 1) return lbm_fail(LBM_EINVAL, "bad rounding %d", p->rounding);
    const int s = p->bc_south, nn = p->bc_north, w = p->bc_west, e = p->bc_east;
    auto ok_sn = [](int b) { return b == LBM_BC_PERIODIC || b == LBM_BC_WALL || b == LBM_BC_FREESLIP; };
    if (!ok_sn(s) || !ok_sn(nn)) return lbm_fail(LBM_EINVAL, "south/north must be PERIODIC, WALL or FREESLIP");
    if ((s == LBM_BC_PERIODIC) != (nn == LBM_BC_PERIODIC))
        return lbm_fail(LBM_EINVAL, "south and north must both be PERIODIC or neither");
    if (!(w >= 0 && w <= 6 && w != LBM_BC_FREESLIP))
        return lbm_fail(LBM_EINVAL,
                        "west must be PERIODIC, WALL, INLET_ZOUHE, INLET_EQ, INLET_EQ_NEUMANN or OUTFLOW_ZG");
    if (!(e == LBM_BC_PERIODIC || e == LBM_BC_WALL || e == LBM_BC_OUTFLOW_ZG || e == LBM_BC_OUTLET_PRESSURE))
        return lbm_fail(LBM_EINVAL, "east must be PERIODIC, WALL, OUTFLOW_ZG or OUTLET_PRESSURE");
    if (e == LBM_BC_OUTLET_PRESSURE && !(std::isfinite(p->rho_out) && p->rho_out > 0))
        return lbm_fail(LBM_EINVAL, "rho_out must be finite and > 0 (got %g)", p->rho_out);
    if (w == LBM_BC_INLET_EQ_NEUMANN && p->algo == LBM_AA)
        return lbm_fail(LBM_EUNSUPPORTED, "AA pattern: the Neumann inlet reads a neighbour that is updated in place");
    if ((w == LBM_BC_PERIODIC) != (e == LBM_BC_PERIODIC))
        return lbm_fail(LBM_EINVAL, "west and east must both be PERIODIC or neither");
    if ((w == LBM_BC_INLET_ZOUHE || w == LBM_BC_INLET_EQ || w == LBM_BC_INLET_EQ_NEUMANN ||
         e == LBM_BC_OUTLET_PRESSURE) && p->nx < 2)
        return lbm_fail(LBM_EINVAL, "an inlet or pressure outlet needs nx >= 2");
    if (p->algo == LBM_AA && (w == LBM_BC_OUTFLOW_ZG || e == LBM_BC_OUTFLOW_ZG))
        return lbm_fail(LBM_EUNSUPPORTED,
                        "AA pattern: zero-gradient outflow reads one slot from two nodes in place");
    return LBM_OK;
}

lbm_status lbm_plan(const lbm_params *p, Plan *pl) {
    lbm_status s = lbm_check_params(p);
    if (s != LBM_OK) return s;
    const Ops *ops = ops_for_storage(p->storage);
    const int64_t N = (int64_t)p->nx * p->ny;
    *pl = Plan();
    pl->N = N;
    pl->two = p->algo == LBM_LPTL || p->algo == LBM_NPTL;
    int tx = p->tile_x, ty = p->tile_y;
    if (p->algo == LBM_LPTL) {
        tx = 0;
        ty = 1;
    } else {
        if (tx == 0 && ty == 0) {
            tx = 32;
            ty = 8;
        }
        if (tx < 1 || ty < 1 || (int64_t)tx * ty > kMaxTileThreadsHost)
            return lbm_fail(LBM_EINVAL, "tile %dx%d: need tile_x, tile_y >= 1, tile_x*tile_y <= %d", tx, ty,
                            kMaxTileThreadsHost);
        if (p->bc_west == LBM_BC_INLET_EQ_NEUMANN && (p->algo == LBM_NPOL || p->algo == LBM_NSOL) && tx < 2)
            return lbm_fail(LBM_EINVAL, "the Neumann inlet needs tile_x >= 2 for one-lattice algorithms");
        pl->ntx = (p->nx + tx - 1) / tx;
        pl->nty = (p->ny + ty - 1) / ty;
        if (pl->nty > 65535) return lbm_fail(LBM_EUNSUPPORTED, "too many tile rows (%d)", pl->nty);
    }
    pl->tx = tx;
    pl->ty = ty;
    const size_t elem = ops->elem, comp = ops->compute;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    pl->pop[0] = take(9 * (size_t)N * elem);
    pl->pop[1] = pl->two ? take(9 * (size_t)N * elem) : (size_t)-1;
    pl->halo_grid = p->algo == LBM_NPOL || p->algo == LBM_NSOL;
    if (pl->halo_grid) {
        pl->halo_parity_elems = (int64_t)pl->ntx * pl->nty * 6 * (tx + ty);
        pl->halo = take(2 * (size_t)pl->halo_parity_elems * elem);
    } else {
        pl->halo = (size_t)-1;
    }
    pl->links = take((size_t)N);
    // Moments; also the staging area of lbm_init (>= 3 doubles per staged node).
    pl->mom_bytes = std::max(3 * (size_t)N * comp, 3 * sizeof(double) * (size_t)std::min<int64_t>(N, 1 << 16));
    pl->mom = take(pl->mom_bytes);
    pl->partials = take(sizeof(double) * (2 * kReduceBlocks + 4));
    pl->misc = take(256);
    pl->total = off;
    return LBM_OK;
}

// ------------------------------------------------------------ lattice
extern "C" lbm_status lbm_workspace_bytes(const lbm_params *p, size_t *bytes) {
    if (!bytes) return lbm_fail(LBM_EINVAL, "bytes is NULL");
    Plan pl;
    lbm_status s = lbm_plan(p, &pl);
    if (s != LBM_OK) return s;
    *bytes = pl.total;
    return LBM_OK;
}

// L2 prefetch distance of the two-lattice and AA kernels (LPTL: nodes, NPTL
// and AA: rows), 0 = off. On for 32-bit storage in the stream and bundle
// layouts when the lattice exceeds the L2 cache (the FP64 update is bound by
// FP64 arithmetic, the 16-bit one by instruction issue). The distance is
// 5/4 of the threads resident on the device: far enough that the prefetch
// lands before the block that pulls it starts, near enough that it is still
// in L2 then. Measured with FP32 storage, bundle layout, NPTL 32 x 4 on
// 134M- and 16.8M-node porous lattices (40 % solid discs): 0.8 to 1.7
// resident thread sets ahead gain 5 to 9 %, 3.4 sets nothing, 6.7 sets lose
// 18 %; on the 134M-node lattice without solids 0.8 sets gain 5 %, 1.3 sets
// 3 %, 2.1 sets lose 6 %.
#ifndef LBM_PF_PAIRS
#define LBM_PF_PAIRS 1
#endif
static uint32_t prefetch_distance(const lbm_params *p, int64_t N, size_t elem, int tile_x) {
    if (p->flags & LBM_FLAG_NO_PREFETCH) return 0;
    // 16-bit storage: only the node-pair kernel (LPTL/NPTL, bundle layout,
    // nx even) prefetches; its distance counts pairs of nodes. Measured on
    // the 134M-node porous lattice (FP16, NPTL 32 x 8): +6 %.
    const bool pairs = elem == 2 && LBM_PF_PAIRS && (p->algo == LBM_LPTL || p->algo == LBM_NPTL) &&
                       p->layout == LBM_LAYOUT_BUNDLE && p->nx % 2 == 0 &&
                       !(p->flags & LBM_FLAG_NO_PAIRS) && 9 * N < (int64_t(1) << 32) &&
                       (p->algo == LBM_LPTL || tile_x % 2 == 0);
    if (elem != 4 && !pairs) return 0;
    if ((p->algo != LBM_LPTL && p->algo != LBM_NPTL && p->algo != LBM_AA) || p->layout == LBM_LAYOUT_COLLISION)
        return 0;
    int dev = 0, sms = 0, threads = 0, l2 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&threads, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    if ((double)N * 9.0 * (double)elem <= (double)l2) return 0;
#ifndef LBM_PF_NUM
#define LBM_PF_NUM 5
#endif
    // pairs: LPTL distances count pairs (the kernel doubles them), NPTL rows
    const int64_t nodes = (int64_t)sms * threads * LBM_PF_NUM / 4 * (pairs && p->algo == LBM_NPTL ? 2 : 1);
    if (p->algo == LBM_LPTL) return nodes < N ? (uint32_t)nodes : 0;
    const int64_t rows = std::max<int64_t>(1, (nodes + p->nx / 2) / p->nx);
    return rows < p->ny ? (uint32_t)rows : 0;
}

// NSOL with FP32 storage stages each tile by one tensor copy (TMA) when the
// tile's rows are whole 16-byte units in a tensor the copy can describe:
// stream layout as a (nx, ny, 9) tensor, box (tx, ty, 9); bundle layout as
// (3 nx, ny, 3), box (3 tx, ty, 3). The copy's x coordinate (x0 or 3 x0) times
// 4 bytes is then a multiple of 16 for every tile, the row strides are
// multiples of 16 bytes, and tiles past the lattice edge read zeros. The
// encoder is the CUDA driver's, reached through the runtime; without it (or on any
// failure) the kernel stages with per-thread loads.
bool lbm_encode_f32_tensor_map(TmaDesc *out, int rank, void *base, const uint64_t *dims,
                                const uint64_t *strides, const uint32_t *box) {
    using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode encode = [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            (void)cudaGetLastError();
            fn = nullptr;
        }
        return (Encode)fn;
    }();
    if (!encode || rank < 1 || rank > 5 || ((uintptr_t)base) % 16) return false;
    cuuint64_t d[5], st[4];
    cuuint32_t bx[5], es[5];
    for (int k = 0; k < rank; ++k) {
        d[k] = dims[k];
        bx[k] = box[k];
        es[k] = 1;
        if (k + 1 < rank) st[k] = strides[k];
    }
    static_assert(sizeof(CUtensorMap) == sizeof(TmaDesc), "tensor map size");
    CUtensorMap m;
    if (encode(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, base, d, st, bx, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    memcpy(out->bytes, &m, sizeof(m));
    return true;
}

static void setup_tma(const lbm_params *p, const Plan &pl, HostArgs *h) {
    h->tma = 0;
    if (p->algo != LBM_NSOL || p->storage != LBM_F32 || (p->flags & LBM_FLAG_NO_TMA)) return;
    if (p->layout != LBM_LAYOUT_STREAM && p->layout != LBM_LAYOUT_BUNDLE) return;
    const bool bundle = p->layout == LBM_LAYOUT_BUNDLE;
    const int64_t row = bundle ? 3 * (int64_t)pl.tx : pl.tx;
    if (pl.tx % 4 || p->nx % 4 || row > 256 || pl.ty > 256) return;
    const uint64_t N = (uint64_t)pl.N, nx = (uint64_t)p->nx;
    const uint64_t dims[3] = {bundle ? 3 * nx : nx, (uint64_t)p->ny, bundle ? 3u : 9u};
    const uint64_t strides[2] = {dims[0] * 4, (bundle ? 3 * N : N) * 4};
    const uint32_t box[3] = {(uint32_t)row, (uint32_t)pl.ty, bundle ? 3u : 9u};
    h->tma = lbm_encode_f32_tensor_map(&h->tmap, 3, h->pop[0], dims, strides, box) ? 1 : 0;
}

void lbm_fill_args(const lbm_params *p, const Plan &pl, char *ws, const Ops *ops, HostArgs *h) {
    memset(h, 0, sizeof(*h));
    h->nx = p->nx;
    h->ny = p->ny;
    h->N = pl.N;
    h->bw = p->bc_west;
    h->be = p->bc_east;
    h->bs = p->bc_south;
    h->bn = p->bc_north;
    h->layout = p->layout;
    h->algo = p->algo;
    h->storage = p->storage;
    h->rounding = p->rounding;
    h->omega = 1.0 / p->tau;
    h->kf = 1.0 - 0.5 * h->omega;
    h->fx = p->force[0];
    h->fy = p->force[1];
    h->ux_in = p->u_in[0];
    h->uy_in = p->u_in[1];
    h->rho_out = p->bc_east == LBM_BC_OUTLET_PRESSURE ? p->rho_out : 1.0;
    h->seed = p->seed;
    h->tile_x = pl.tx;
    h->tile_y = pl.ty;
    h->ntx = pl.ntx;
    h->nty = pl.nty;
    ops->prepare();
    h->block_1d = p->algo == LBM_LPTL ? ops->lptl_block(p->layout) : 0;
    h->flags = p->flags;
    h->nx_magic = p->nx == 1 ? 0ull : (~0ull / (uint64_t)p->nx) + 1ull;
    h->pf = prefetch_distance(p, pl.N, ops->elem, pl.tx);
    h->links = (const uint8_t *)(ws + pl.links);
    h->pop[0] = ws + pl.pop[0];
    h->pop[1] = pl.two ? ws + pl.pop[1] : nullptr;
    h->halo = pl.halo_grid ? ws + pl.halo : nullptr;
    h->halo_parity_elems = pl.halo_parity_elems;
    h->mom = ws + pl.mom;
    h->err = (unsigned int *)(ws + pl.misc);
    h->tctr = (long long *)(ws + pl.misc + 64);
    setup_tma(p, pl, h);
}

extern "C" lbm_status lbm_create(const lbm_params *p, const uint8_t *mask_host, void *d_workspace,
                                 size_t bytes, void *cuda_stream, lbm_lattice **out) {
    if (!out) return lbm_fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    Plan pl;
    lbm_status s = lbm_plan(p, &pl);
    if (s != LBM_OK) return s;
    if (!d_workspace) return lbm_fail(LBM_EINVAL, "workspace is NULL");
    if (((uintptr_t)d_workspace) % 256) return lbm_fail(LBM_EINVAL, "workspace must be 256-byte aligned");
    if (bytes < pl.total)
        return lbm_fail(LBM_ENOMEM, "workspace too small: %zu bytes given, %zu needed", bytes, pl.total);
    if (!mask_host) return lbm_fail(LBM_EINVAL, "mask is NULL");
    lbm_lattice *L = (lbm_lattice *)calloc(1, sizeof(lbm_lattice));
    if (!L) return lbm_fail(LBM_ENOMEM, "host allocation failed");
    L->p = *p;
    L->pl = pl;
    L->ops = ops_for_storage(p->storage);
    L->stream = (cudaStream_t)cuda_stream;
    L->ws = (char *)d_workspace;
    L->graph_steps = 64;
    lbm_fill_args(p, pl, L->ws, L->ops, &L->h);
    L->partials = (double *)(L->ws + pl.partials);
    L->red_out = L->partials + 2 * kReduceBlocks;
    L->err = L->h.err;
    L->count = (unsigned long long *)(L->ws + pl.misc + 128);
    cudaError_t e = cudaStreamCreateWithFlags(&L->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        free(L);
        return lbm_cuda_fail(e, "cudaStreamCreateWithFlags");
    }
    // Mask -> device (staged in the moments region, >= N bytes) -> link bytes.
    const cudaStream_t st = L->stream;
    uint8_t *dmask = (uint8_t *)L->h.mom;
    s = LBM_OK;
#define CKD(call)                                  \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) {                   \
            s = lbm_cuda_fail(e_, #call);          \
            goto fail;                             \
        }                                          \
    } while (0)
    {
        unsigned long long fluid = 0;
        CKD(cudaMemcpyAsync(dmask, mask_host, (size_t)pl.N, cudaMemcpyHostToDevice, st));
        CKD(launch_links(p->nx, p->ny, p->bc_west, p->bc_east, p->bc_south, p->bc_north, dmask,
                         (uint8_t *)L->h.links, st));
        CKD(launch_count_fluid(L->h.links, pl.N, L->count, st));
        CKD(cudaMemcpyAsync(&fluid, L->count, sizeof(fluid), cudaMemcpyDeviceToHost, st));
        CKD(cudaStreamSynchronize(st));
        L->fluid = (int64_t)fluid;
    }
#undef CKD
    s = lbm_init(L, nullptr, nullptr, nullptr);
    if (s != LBM_OK) goto fail;
    *out = L;
    return LBM_OK;
fail:
    cudaStreamDestroy(L->cap);
    free(L);
    return s;
}

static void stage_free(lbm_lattice *L);

static void drop_graphs(lbm_lattice *L) {
    for (auto &g : L->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

extern "C" void lbm_destroy(lbm_lattice *L) {
    if (!L) return;
    cudaStreamSynchronize(L->stream);
    drop_graphs(L);
    stage_free(L);
    cudaStreamDestroy(L->cap);
    free(L);
}

// Zero the populations, write the equilibrium of (rho, u) chunk by chunk
// through the moments region, reset counters, record the init moments.
extern "C" lbm_status lbm_init(lbm_lattice *L, const double *rho, const double *ux, const double *uy) {
    if (!L) return lbm_fail(LBM_EINVAL, "lattice is NULL");
    const cudaStream_t st = L->stream;
    const Plan &pl = L->pl;
    const size_t popb = 9 * (size_t)pl.N * L->ops->elem;
    CK(cudaStreamSynchronize(st));
    CK(cudaMemsetAsync(L->h.pop[0], 0, popb, st));
    if (pl.two) CK(cudaMemsetAsync(L->h.pop[1], 0, popb, st));
    if (pl.halo_grid) CK(cudaMemsetAsync(L->h.halo, 0, 2 * (size_t)pl.halo_parity_elems * L->ops->elem, st));
    CK(cudaMemsetAsync(L->ws + pl.misc, 0, 256, st));
    L->cur = 0;
    L->steps = 0;
    if (rho || ux || uy) {
        const int64_t chunk = std::min<int64_t>(pl.N, (int64_t)(pl.mom_bytes / (3 * sizeof(double))));
        double *d = (double *)L->h.mom;
        for (int64_t n0 = 0; n0 < pl.N; n0 += chunk) {
            const int64_t c = std::min<int64_t>(chunk, pl.N - n0);
            double *dr = rho ? d : nullptr, *du = ux ? d + chunk : nullptr, *dv = uy ? d + 2 * chunk : nullptr;
            if (rho) CK(cudaMemcpyAsync(dr, rho + n0, c * sizeof(double), cudaMemcpyHostToDevice, st));
            if (ux) CK(cudaMemcpyAsync(du, ux + n0, c * sizeof(double), cudaMemcpyHostToDevice, st));
            if (uy) CK(cudaMemcpyAsync(dv, uy + n0, c * sizeof(double), cudaMemcpyHostToDevice, st));
            CK(L->ops->init(L->h, dr, du, dv, n0, c, st));
            CK(cudaStreamSynchronize(st));
        }
    }
    CK(L->ops->state_moments(L->h, 0, 0, st));
    if (pl.halo_grid) CK(L->ops->publish(L->h, 0, 0, st));
    CK(cudaStreamSynchronize(st));
    return LBM_OK;
}

// ------------------------------------------------------------ stepping
static cudaError_t launch_block(lbm_lattice *L, cudaStream_t st, int64_t count, int want_moments) {
    const int two = L->pl.two;
    int cur = L->cur;
    int64_t steps = L->steps;
    for (int64_t s = 0; s < count; ++s) {
        StepCall c{cur, (int)(steps & 1), (int)s, (want_moments && s == count - 1) ? 1 : 0};
        cudaError_t e = L->ops->step(L->h, c, st);
        if (e != cudaSuccess) return e;
        if (two) cur ^= 1;
        ++steps;
    }
    return launch_bump_counter(L->h.tctr, count, st);
}

static lbm_status get_graph(lbm_lattice *L, cudaGraphExec_t *out) {
    const int key = (L->pl.two ? L->cur : 0) * 2 + (L->pl.two ? 0 : (int)(L->steps & 1));
    if (!L->graph[key]) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(L->cap, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = launch_block(L, L->cap, L->graph_steps, 0);
        cudaError_t e2 = cudaStreamEndCapture(L->cap, &g);
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return lbm_cuda_fail(e, "capturing update kernels");
        }
        if (e2 != cudaSuccess) return lbm_cuda_fail(e2, "cudaStreamEndCapture");
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return lbm_cuda_fail(e, "cudaGraphInstantiate");
        L->graph[key] = ex;
    }
    *out = L->graph[key];
    return LBM_OK;
}

extern "C" lbm_status lbm_step(lbm_lattice *L, int64_t nsteps, uint32_t want_moments) {
    if (!L) return lbm_fail(LBM_EINVAL, "lattice is NULL");
    if (nsteps < 0) return lbm_fail(LBM_EINVAL, "nsteps must be >= 0");
    int64_t left = nsteps;
    const bool graphs = !(L->p.flags & LBM_FLAG_NO_GRAPH);
    // whole graph blocks; the last block runs directly when it must store moments
    while (graphs && (left > L->graph_steps || (left == L->graph_steps && !want_moments))) {
        cudaGraphExec_t ex;
        lbm_status s = get_graph(L, &ex);
        if (s != LBM_OK) return s;
        CK(cudaGraphLaunch(ex, L->stream));
        L->steps += L->graph_steps;  // even block: lattice and parity unchanged
        left -= L->graph_steps;
    }
    if (left > 0) {
        CK(launch_block(L, L->stream, left, want_moments ? 1 : 0));
        if (L->pl.two && (left & 1)) L->cur ^= 1;
        L->steps += left;
    }
    return LBM_OK;
}

static lbm_status check_err(lbm_lattice *L) {
    unsigned int flag = 0;
    CK(cudaMemcpy(&flag, L->err, sizeof(flag), cudaMemcpyDeviceToHost));
    if (flag) {
        CK(cudaMemset(L->err, 0, sizeof(unsigned int)));
        if (flag & 2u)
            return lbm_fail(LBM_ECUDA, "a tile's tensor copy did not complete within the wait limit");
        return lbm_fail(LBM_EDIVERGED, "non-finite density after %lld updates", (long long)L->steps);
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_sync(lbm_lattice *L) {
    if (!L) return lbm_fail(LBM_EINVAL, "lattice is NULL");
    CK(cudaStreamSynchronize(L->stream));
    return check_err(L);
}

extern "C" lbm_status lbm_wait(lbm_lattice *L, double timeout_s) {
    if (!L) return lbm_fail(LBM_EINVAL, "lattice is NULL");
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ev, L->stream);
    if (e != cudaSuccess) {
        cudaEventDestroy(ev);
        return lbm_cuda_fail(e, "cudaEventRecord");
    }
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        e = cudaEventQuery(ev);
        if (e != cudaErrorNotReady) break;
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el >= timeout_s) {
            cudaEventDestroy(ev);
            return lbm_fail(LBM_ETIMEOUT, "work still running after %.3f s", el);
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return lbm_cuda_fail(e, "cudaEventQuery");
    return lbm_sync(L);
}

// ------------------------------------------------------------ host loops
// Run fn(begin, end) over [0, count) on up to 16 host threads (large arrays
// only; the conversions below are independent per element).
template <class Fn>
static void parallel_for(int64_t count, Fn fn) {
    const int64_t grain = 1 << 20;
    int nt = (int)std::min<int64_t>(16, std::max<int64_t>(1, count / grain));
    const unsigned hw = std::thread::hardware_concurrency();
    if (hw > 0) nt = std::min<int>(nt, (int)hw);
    if (nt <= 1) {
        fn((int64_t)0, count);
        return;
    }
    std::vector<std::thread> th;
    const int64_t step = (count + nt - 1) / nt;
    for (int t = 0; t < nt; ++t) {
        const int64_t b = t * step, e = std::min(count, b + step);
        if (b < e) th.emplace_back(fn, b, e);
    }
    for (auto &x : th) x.join();
}

// ------------------------------------------------------------ read-out
// Device address of a page-locked, mapped host buffer (cudaHostAlloc,
// cudaHostRegister, torch pin_memory), or NULL for pageable memory.
static void *mapped_host(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// FP32 -> FP64 widening straight into mapped host memory (over the
// CPU-GPU link, no staging copy).
constexpr int kWidenBlocks = 1216;  // grid-stride; 8 blocks per SM on 152 SMs
__global__ void k_widen(const float *__restrict__ s, double *__restrict__ d, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) d[k] = (double)s[k];
}

// Page-locked staging for pageable destinations: two chunks, copied and
// widened alternately so the copy of one overlaps the widening of the other.
// A field of up to kStageBytes goes through an unpinned host buffer instead
// (one copy; pinning costs more than it saves there).
static constexpr size_t kStageBytes = (size_t)64 << 20;

static lbm_status stage_alloc(lbm_lattice *L) {
    if (L->stage) return LBM_OK;
    CK(cudaHostAlloc(&L->stage, 2 * kStageBytes, cudaHostAllocDefault));
    for (auto &e : L->stage_ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return LBM_OK;
}

static lbm_status widen_small(lbm_lattice *L, const float *src, double *dst, int64_t n) {
    std::unique_ptr<float[]> buf(new (std::nothrow) float[(size_t)n]);
    if (!buf) return lbm_fail(LBM_ENOMEM, "host allocation failed");
    CK(cudaMemcpyAsync(buf.get(), src, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, L->stream));
    CK(cudaStreamSynchronize(L->stream));
    const float *f = buf.get();
    parallel_for(n, [f, dst](int64_t lo, int64_t hi) {
        for (int64_t k = lo; k < hi; ++k) dst[k] = f[k];
    });
    return LBM_OK;
}

static void stage_free(lbm_lattice *L) {
    for (auto &e : L->stage_ev)
        if (e) cudaEventDestroy(e);
    if (L->stage) cudaFreeHost(L->stage);
    L->stage = nullptr;
}

static lbm_status widen_staged(lbm_lattice *L, const float *src, double *dst, int64_t n) {
    lbm_status s = stage_alloc(L);
    if (s != LBM_OK) return s;
    const int64_t chunk = (int64_t)(kStageBytes / sizeof(float));
    const int64_t nch = (n + chunk - 1) / chunk;
    auto issue = [&](int64_t c) -> cudaError_t {
        const int64_t b = c * chunk, m = std::min(chunk, n - b);
        float *slot = (float *)(L->stage + (size_t)(c & 1) * kStageBytes);
        cudaError_t e = cudaMemcpyAsync(slot, src + b, (size_t)m * sizeof(float), cudaMemcpyDeviceToHost,
                                        L->stream);
        return e != cudaSuccess ? e : cudaEventRecord(L->stage_ev[c & 1], L->stream);
    };
    for (int64_t c = 0; c < std::min<int64_t>(2, nch); ++c) CK(issue(c));
    for (int64_t c = 0; c < nch; ++c) {
        CK(cudaEventSynchronize(L->stage_ev[c & 1]));
        const int64_t b = c * chunk, m = std::min(chunk, n - b);
        const float *f = (const float *)(L->stage + (size_t)(c & 1) * kStageBytes);
        double *d = dst + b;
        parallel_for(m, [f, d](int64_t lo, int64_t hi) {
            for (int64_t k = lo; k < hi; ++k) d[k] = f[k];
        });
        if (c + 2 < nch) CK(issue(c + 2));   // this slot is free again
    }
    return LBM_OK;
}

// Copy one moments field of N values (device, FP32 or FP64) to host doubles.
static lbm_status moments_to_host(lbm_lattice *L, const void *dev, double *dst, int64_t N) {
    if (L->ops->compute == 8) {
        CK(cudaMemcpyAsync(dst, dev, (size_t)N * 8, cudaMemcpyDeviceToHost, L->stream));
        return LBM_OK;
    }
    if (double *d = (double *)mapped_host(dst)) {
        k_widen<<<kWidenBlocks, 256, 0, L->stream>>>((const float *)dev, d, N);
        CK(cudaGetLastError());
        return LBM_OK;
    }
    if ((size_t)N * sizeof(float) <= kStageBytes) return widen_small(L, (const float *)dev, dst, N);
    return widen_staged(L, (const float *)dev, dst, N);
}

extern "C" lbm_status lbm_read_moments(lbm_lattice *L, double *rho, double *ux, double *uy) {
    if (!L) return lbm_fail(LBM_EINVAL, "lattice is NULL");
    const int64_t N = L->pl.N;
    const size_t comp = L->ops->compute;
    double *dst[3] = {rho, ux, uy};
    for (int k = 0; k < 3; ++k) {
        if (!dst[k]) continue;
        const lbm_status s = moments_to_host(L, (const char *)L->h.mom + (size_t)k * N * comp, dst[k], N);
        if (s != LBM_OK) return s;
    }
    CK(cudaStreamSynchronize(L->stream));
    return check_err(L);
}

extern "C" lbm_status lbm_moments_device(lbm_lattice *L, float *r, float *u, float *v) {
    if (!L || !r || !u || !v) return lbm_fail(LBM_EINVAL, "NULL argument");
    CK(L->ops->moments_f32(L->h, r, u, v, L->stream));
    return LBM_OK;
}

// The AA pattern holds the canonical state (in opposite slots) only after an
// even number of updates.
static lbm_status aa_state_readable(lbm_lattice *L) {
    if (L->p.algo == LBM_AA && (L->steps & 1))
        return lbm_fail(LBM_EINVAL, "AA pattern: the state is readable after an even number of updates");
    return LBM_OK;
}

extern "C" lbm_status lbm_mass(lbm_lattice *L, double *out) {
    if (!L || !out) return lbm_fail(LBM_EINVAL, "NULL argument");
    if (aa_state_readable(L) != LBM_OK) return LBM_EINVAL;
    CK(L->ops->mass(L->h, L->cur, L->partials, kReduceBlocks, L->stream));
    CK(launch_sum_partials(L->partials, kReduceBlocks, 1, L->red_out, L->stream));
    CK(cudaMemcpyAsync(out, L->red_out, sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    CK(cudaStreamSynchronize(L->stream));
    return check_err(L);
}

extern "C" lbm_status lbm_force(lbm_lattice *L, const uint8_t *d_body, double out[2]) {
    if (!L || !out) return lbm_fail(LBM_EINVAL, "NULL argument");
    if (aa_state_readable(L) != LBM_OK) return LBM_EINVAL;
    CK(L->ops->force(L->h, L->cur, d_body, L->partials, kReduceBlocks, L->stream));
    CK(launch_sum_partials(L->partials, kReduceBlocks, 2, L->red_out, L->stream));
    CK(cudaMemcpyAsync(out, L->red_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    CK(cudaStreamSynchronize(L->stream));
    return check_err(L);
}

// Host conversion between raw storage and canonical h[i*N + n].
template <int LAY>
static int64_t host_addr(int64_t N, int64_t n, int i) {
    return addr<LAY>(N, n, i);
}

int64_t layout_addr(int layout, int64_t N, int64_t n, int i) {
    switch (layout) {
        case LBM_LAYOUT_STREAM: return host_addr<STREAM>(N, n, i);
        case LBM_LAYOUT_BUNDLE: return host_addr<BUNDLE>(N, n, i);
        case LBM_LAYOUT_COLLISION: return host_addr<COLLISION>(N, n, i);
    }
    return -1;
}

extern "C" int64_t lbm_layout_index(int32_t layout, int64_t N, int64_t n, int32_t i) {
    if (layout < 0 || layout > 2 || N < 1 || n < 0 || n >= N || i < 0 || i > 8) return -1;
    return layout_addr(layout, N, n, i);
}

static double raw_get(const unsigned char *raw, int storage, int64_t k) {
    switch (storage) {
        case LBM_F64: return ((const double *)raw)[k];
        case LBM_F32: return ((const float *)raw)[k];
        case LBM_F16S: return __half2float(((const __half *)raw)[k]);
        default: return __bfloat162float(((const __nv_bfloat16 *)raw)[k]);
    }
}

static void raw_set(unsigned char *raw, int storage, int64_t k, double v) {
    switch (storage) {
        case LBM_F64: ((double *)raw)[k] = v; break;
        case LBM_F32: ((float *)raw)[k] = (float)v; break;
        case LBM_F16S: ((__half *)raw)[k] = __float2half_rn((float)v); break;
        default: ((__nv_bfloat16 *)raw)[k] = __float2bfloat16_rn((float)v); break;
    }
}

lbm_status lbm_pops_to_host(const unsigned char *raw, int storage, int layout, int rev, int64_t N, void *host,
                            int32_t as) {
    for (int i = 0; i < 9; ++i) {
        const int slot = rev ? 8 - i : i;
        parallel_for(N, [=](int64_t b, int64_t e) {
            for (int64_t n = b; n < e; ++n) {
                const double v = raw_get(raw, storage, layout_addr(layout, N, n, slot));
                if (as == LBM_F64)
                    ((double *)host)[(int64_t)i * N + n] = v;
                else
                    ((float *)host)[(int64_t)i * N + n] = (float)v;
            }
        });
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_read_populations(lbm_lattice *L, void *host, int32_t as) {
    if (!L || !host) return lbm_fail(LBM_EINVAL, "NULL argument");
    if (aa_state_readable(L) != LBM_OK) return LBM_EINVAL;
    if (as != LBM_F64 && as != LBM_F32) return lbm_fail(LBM_EINVAL, "as must be LBM_F64 or LBM_F32");
    const int64_t N = L->pl.N;
    std::vector<unsigned char> raw(9 * (size_t)N * L->ops->elem);
    CK(cudaStreamSynchronize(L->stream));
    CK(cudaMemcpy(raw.data(), L->h.pop[L->cur], raw.size(), cudaMemcpyDeviceToHost));
    lbm_pops_to_host(raw.data(), L->p.storage, L->p.layout, L->p.algo == LBM_NSOL || L->p.algo == LBM_AA, N,
                     host, as);
    return check_err(L);
}

extern "C" lbm_status lbm_write_populations(lbm_lattice *L, const void *host, int32_t as) {
    if (!L || !host) return lbm_fail(LBM_EINVAL, "NULL argument");
    if (aa_state_readable(L) != LBM_OK) return LBM_EINVAL;
    if (as != LBM_F64 && as != LBM_F32) return lbm_fail(LBM_EINVAL, "as must be LBM_F64 or LBM_F32");
    const int64_t N = L->pl.N;
    std::vector<unsigned char> raw(9 * (size_t)N * L->ops->elem);
    const int rev = L->p.algo == LBM_NSOL || L->p.algo == LBM_AA;
    unsigned char *rawp = raw.data();
    const int storage = L->p.storage, layout = L->p.layout;
    for (int i = 0; i < 9; ++i) {
        const int slot = rev ? 8 - i : i;
        parallel_for(N, [=](int64_t b, int64_t e) {
            for (int64_t n = b; n < e; ++n) {
                const double v = as == LBM_F64 ? ((const double *)host)[(int64_t)i * N + n]
                                               : (double)((const float *)host)[(int64_t)i * N + n];
                raw_set(rawp, storage, layout_addr(layout, N, n, slot), v);
            }
        });
    }
    CK(cudaStreamSynchronize(L->stream));
    CK(cudaMemcpy(L->h.pop[L->cur], raw.data(), raw.size(), cudaMemcpyHostToDevice));
    CK(L->ops->zero_solid(L->h, L->cur, L->stream));
    if (L->pl.halo_grid) CK(L->ops->publish(L->h, L->cur, (int)(L->steps & 1), L->stream));
    CK(cudaStreamSynchronize(L->stream));
    return LBM_OK;
}

extern "C" lbm_status lbm_get_info(lbm_lattice *L, lbm_info *out) {
    if (!L || !out) return lbm_fail(LBM_EINVAL, "NULL argument");
    memset(out, 0, sizeof(*out));
    out->cells = L->pl.N;
    out->fluid_cells = L->fluid;
    out->steps = L->steps;
    out->tile_x = L->p.algo == LBM_LPTL ? L->h.block_1d : L->pl.tx;
    out->tile_y = L->p.algo == LBM_LPTL ? 1 : L->pl.ty;
    const double elem = (double)L->ops->elem;
    double bytes = (double)L->fluid * 18.0 * elem + (double)L->pl.N;  // 9 reads + 9 writes, link byte
    if (L->pl.halo_grid) bytes += 2.0 * (double)L->pl.halo_parity_elems * elem;  // buffer grid read + write
    out->bytes_per_update = bytes;
    out->workspace_bytes = L->pl.total;
    out->aux = L->p.algo == LBM_NSOL ? (int32_t)L->h.tma : (int32_t)L->h.pf;
    return LBM_OK;
}

extern "C" lbm_status lbm_quantize(int32_t storage, int32_t rounding, uint64_t seed, int64_t t,
                                   const float *d_in, void *d_out, float *d_back, int64_t count,
                                   void *cuda_stream) {
    if (storage != LBM_F16S && storage != LBM_BF16S)
        return lbm_fail(LBM_EINVAL, "quantize: storage must be F16S or BF16S");
    if (rounding < 0 || rounding > 1) return lbm_fail(LBM_EINVAL, "bad rounding");
    if (count < 0 || (count > 0 && (!d_in || !d_out))) return lbm_fail(LBM_EINVAL, "bad arrays");
    CK(launch_quantize(storage, rounding, seed, t, d_in, d_out, d_back, count, (cudaStream_t)cuda_stream));
    return LBM_OK;
}
