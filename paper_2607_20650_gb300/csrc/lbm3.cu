// D3Q19 boxes (the paper's 3-D future work, Sec. 6) behind the lbm3_* calls
// of include/lbm.h: workspace planning and validation, creation (link words
// of the mask on the GPU), init, updates (captured into CUDA graphs of 64),
// read-back, FP64 mass and momentum-exchange force. The kernels live in
// lbm3_kernels.cuh and are launched through the per-storage tables of
// lbm3_ops_*.cu.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "lbm.h"
#include "lbm3_internal.h"
#include "lbm3_kernels.cuh"
#include "lbm_capi_internal.h"
#include "lbm_internal.h"

namespace lbm {
namespace d3 {

__global__ void k3_links(Geo3 g, const uint8_t *mask, uint32_t *links) {
    const uint64_t N64 = (uint64_t)g.nx * g.ny * g.nz;
    const uint64_t n64 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n64 >= N64) return;
    const uint32_t n = (uint32_t)n64;
    if (mask[n]) {
        links[n] = SOLID;
        return;
    }
    const uint32_t nxy = (uint32_t)g.nx * (uint32_t)g.ny;
    const int z = (int)(n / nxy), r = (int)(n - (uint32_t)z * nxy);
    const int y = r / g.nx, x = r - y * g.nx;
    uint32_t bits = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (i == REST) continue;
        uint32_t s;
        if (!map3(g, x, y, z, i, s) || mask[s]) bits |= 1u << bit(i);
    }
    links[n] = bits;   // SOLID when every pull bounces (isolated node)
}

__global__ void k3_count(const uint32_t *links, uint32_t N, unsigned long long *out) {
    unsigned long long c = 0;
    for (uint64_t n = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (uint64_t)gridDim.x * blockDim.x)
        c += links[n] != SOLID;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, c);
}

__global__ void k3_sum3(const double *partials, int nb, double *out) {
    if (threadIdx.x || blockIdx.x) return;
    for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += partials[3 * b + k];
        out[k] = s;
    }
}

__global__ void k3_sum(const double *partials, int nb, double *out) {
    if (threadIdx.x || blockIdx.x) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partials[b];
    *out = s;
}

}  // namespace d3
}  // namespace lbm

using namespace lbm;
using namespace lbm::d3;

#define CK3(call)                                                 \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return lbm_cuda_fail(e_, #call);   \
    } while (0)

const Ops3 *ops3_for(int storage) {
    switch (storage) {
        case LBM_F64: return &ops3_f64();
        case LBM_F32: return &ops3_f32();
        case LBM_F16S: return &ops3_f16();
        default: return &ops3_bf16();
    }
}

lbm_status lbm3_plan(const lbm3_params *p, Plan3 *pl) {
    if (!p) return lbm_fail(LBM_EINVAL, "params is NULL");
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return lbm_fail(LBM_EINVAL, "nx, ny, nz must be >= 1");
    const uint64_t N = (uint64_t)p->nx * p->ny * p->nz;
    if (N >= (1ull << 32)) return lbm_fail(LBM_EUNSUPPORTED, "nx*ny*nz must be < 2^32");
    if (!(p->tau > 0.5)) return lbm_fail(LBM_EINVAL, "tau must be > 1/2");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(p->force[a])) return lbm_fail(LBM_EINVAL, "force must be finite");
    const int bc[3] = {p->bc_x, p->bc_y, p->bc_z};
    for (int a = 1; a < 3; ++a)
        if (bc[a] != LBM_BC_PERIODIC && bc[a] != LBM_BC_WALL)
            return lbm_fail(LBM_EINVAL, "D3Q19 y and z faces are PERIODIC or WALL");
    if (p->bc_x != LBM_BC_PERIODIC && p->bc_x != LBM_BC_WALL && !inlet3_kind(p->bc_x) &&
        p->bc_x != LBM_BC_OUTFLOW_ZG)
        return lbm_fail(LBM_EINVAL, "D3Q19 x faces: PERIODIC, WALL, INLET_EQ or INLET_ZOUHE (west) or OUTFLOW_ZG");
    if (inlet3_kind(p->bc_x) && p->bc_x_east != LBM_BC_WALL && p->bc_x_east != LBM_BC_OUTFLOW_ZG &&
        p->bc_x_east != LBM_BC_OUTLET_PRESSURE)
        return lbm_fail(LBM_EINVAL, "D3Q19 inlet: the east face (bc_x_east) is WALL, OUTFLOW_ZG or OUTLET_PRESSURE");
    if (inlet3_kind(p->bc_x) && p->bc_x_east == LBM_BC_OUTLET_PRESSURE && !(p->rho_out > 0.0 && std::isfinite(p->rho_out)))
        return lbm_fail(LBM_EINVAL, "D3Q19 pressure outlet: rho_out must be finite and > 0");
    const bool open_x = inlet3_kind(p->bc_x) || p->bc_x == LBM_BC_OUTFLOW_ZG;
    if (open_x && (p->algo == LBM_AA || p->algo == LBM_NPOL || p->algo == LBM_NSOL))
        return lbm_fail(LBM_EUNSUPPORTED, "D3Q19 inlet/outlet faces: LPTL or NPTL only");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(p->u_in[a])) return lbm_fail(LBM_EINVAL, "u_in must be finite");
    if (p->layout < 0 || p->layout > 2) return lbm_fail(LBM_EINVAL, "bad layout");
    if (p->algo != LBM_LPTL && p->algo != LBM_NPTL && p->algo != LBM_AA && p->algo != LBM_NPOL &&
        p->algo != LBM_NSOL)
        return lbm_fail(LBM_EUNSUPPORTED, "D3Q19: LPTL, NPTL, NPOL, NSOL or AA");
    if (p->storage < 0 || p->storage > 3) return lbm_fail(LBM_EINVAL, "bad storage");
    if (p->rounding < 0 || p->rounding > 1) return lbm_fail(LBM_EINVAL, "bad rounding");
    *pl = Plan3();
    pl->N = (int64_t)N;
    if (p->algo == LBM_NPTL || p->algo == LBM_AA || p->algo == LBM_NPOL || p->algo == LBM_NSOL) {
        int tx = p->tile_x, ty = p->tile_y, tz = p->tile_z;
        if (tx == 0 && ty == 0 && tz == 0) { tx = 128; ty = 1; tz = 1; }
        if (tx < 1 || ty < 1 || tz < 1 || tz > 64 || (int64_t)tx * ty * tz > 512)
            return lbm_fail(LBM_EINVAL, "tile must be positive, tile_z <= 64, tile_x*tile_y*tile_z <= 512");
        pl->tx = tx; pl->ty = ty; pl->tz = tz;
        pl->ntx = (p->nx + tx - 1) / tx;
        pl->nty = (p->ny + ty - 1) / ty;
        pl->ntz = (p->nz + tz - 1) / tz;
        if (pl->nty > 65535 || pl->ntz > 65535) return lbm_fail(LBM_EUNSUPPORTED, "too many tiles in y or z");
    }
    pl->elem = elem3_of(p->storage);
    pl->comp = comp3_of(p->storage);
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = (off + b + 255) / 256 * 256; return o; };
    pl->pop[0] = take(19 * (size_t)N * pl->elem);
    pl->one = (p->algo == LBM_AA || p->algo == LBM_NPOL || p->algo == LBM_NSOL) ? 1 : 0;
    if (p->algo == LBM_AA && (!lbm3_offsets_fit(p, (int64_t)N) || (p->flags & LBM_FLAG_WIDE_OFFSETS)))
        return lbm_fail(LBM_EUNSUPPORTED, "D3Q19 AA needs 32-bit offset tables (19 N well below 2^31)");
    pl->pop[1] = pl->one ? pl->pop[0] : take(19 * (size_t)N * pl->elem);
    if (p->algo == LBM_NPOL || p->algo == LBM_NSOL) {
        pl->halo_parity = (int64_t)pl->ntx * pl->nty * pl->ntz * Tile3{pl->tx, pl->ty, pl->tz}.per_tile();
        pl->halo = take(2 * (size_t)pl->halo_parity * pl->elem);
    }
    pl->links = take(4 * (size_t)N);
    pl->mom_bytes = std::max(4 * (size_t)N * pl->comp, 4 * sizeof(double) * (size_t)std::min<uint64_t>(N, 1 << 16));
    pl->mom = take(pl->mom_bytes);
    pl->partials = take(sizeof(double) * (3 * kReduceBlocks + 4));
    pl->misc = take(256);
    pl->total = off;
    return LBM_OK;
}

// Element offsets of the kernels' 32-bit tables: own slot, bounced pull and
// interior pull plus the largest periodic-face correction, per direction.
bool lbm3_offsets_fit(const lbm3_params *p, int64_t N) {
    const int64_t nx = p->nx, nxy = (int64_t)p->nx * p->ny, lim = (1ll << 31) - 64;
    for (int i = 0; i < 19; ++i) {
        const int ax = std::abs(lbm::d3::cx(i)), ay = std::abs(lbm::d3::cy(i)), az = std::abs(lbm::d3::cz(i));
        const int64_t d = lbm::d3::cz(i) * nxy + lbm::d3::cy(i) * nx + lbm::d3::cx(i);
        int64_t self, mul;
        if (p->layout == LBM_LAYOUT_STREAM) { self = i * N; mul = 1; }
        else if (p->layout == LBM_LAYOUT_COLLISION) { self = i; mul = 19; }
        else { self = lbm::d3::bundle_first(i) * N + (i - lbm::d3::bundle_first(i)); mul = lbm::d3::bundle_size(i); }
        const int64_t wrap = mul * (az * N + ay * nxy + ax * nx);
        const int64_t pull = self - mul * d;
        const int j = lbm::d3::opp(i);
        const int64_t selfj = p->layout == LBM_LAYOUT_STREAM ? j * N
                            : p->layout == LBM_LAYOUT_COLLISION ? j
                            : lbm::d3::bundle_first(j) * N + (j - lbm::d3::bundle_first(j));
        const int64_t push = selfj + mul * d;
        if (self > lim || pull + wrap > lim || pull - wrap < -lim) return false;
        if (push + wrap > lim || push - wrap < -lim) return false;
        if (mul * N > lim) return false;   // mult * n itself stays 32-bit
    }
    return true;
}

static cudaError_t launch3(lbm3_lattice *L, cudaStream_t st, int64_t count, int want_moments) {
    int cur = L->cur;
    for (int64_t k = 0; k < count; ++k) {
        const int mom = (want_moments && k == count - 1) ? 1 : 0;
        cudaError_t e = L->ops->step(L, st, cur, (int)k, mom);
        if (e != cudaSuccess) return e;
        cur ^= 1;
    }
    return launch_bump_counter(L->tctr, count, st);
}

extern "C" lbm_status lbm3_workspace_bytes(const lbm3_params *p, size_t *bytes) {
    if (!bytes) return lbm_fail(LBM_EINVAL, "bytes is NULL");
    Plan3 pl;
    lbm_status s = lbm3_plan(p, &pl);
    if (s == LBM_OK) *bytes = pl.total;
    return s;
}

extern "C" int64_t lbm3_layout_index(int32_t layout, int64_t N, int64_t n, int32_t i) {
    if (layout < 0 || layout > 2 || N < 1 || n < 0 || n >= N || i < 0 || i > 18) return -1;
    if (layout == LBM_LAYOUT_STREAM) return d3::addr<STREAM>(N, n, i);
    if (layout == LBM_LAYOUT_BUNDLE) return d3::addr<BUNDLE>(N, n, i);
    return d3::addr<COLLISION>(N, n, i);
}

extern "C" lbm_status lbm3_init(lbm3_lattice *L, const double *rho, const double *ux, const double *uy,
                                const double *uz) {
    if (!L) return lbm_fail(LBM_EINVAL, "lattice is NULL");
    const cudaStream_t st = L->stream;
    const Plan3 &pl = L->pl;
    CK3(cudaStreamSynchronize(st));
    CK3(cudaMemsetAsync(L->ws + pl.pop[0], 0, 19 * (size_t)pl.N * pl.elem, st));
    if (!pl.one) CK3(cudaMemsetAsync(L->ws + pl.pop[1], 0, 19 * (size_t)pl.N * pl.elem, st));
    CK3(cudaMemsetAsync(L->ws + pl.misc, 0, 256, st));
    if (pl.halo_parity) CK3(cudaMemsetAsync(L->ws + pl.halo, 0, 2 * (size_t)pl.halo_parity * pl.elem, st));
    L->cur = 0;
    L->steps = 0;
    if (rho || ux || uy || uz) {
        const int64_t chunk = std::min<int64_t>(pl.N, (int64_t)(pl.mom_bytes / (4 * sizeof(double))));
        double *d = (double *)(L->ws + pl.mom);
        const double *in[4] = {rho, ux, uy, uz};
        for (int64_t n0 = 0; n0 < pl.N; n0 += chunk) {
            const int64_t c = std::min<int64_t>(chunk, pl.N - n0);
            double *dv[4];
            for (int k = 0; k < 4; ++k) {
                dv[k] = in[k] ? d + k * chunk : nullptr;
                if (in[k]) CK3(cudaMemcpyAsync(dv[k], in[k] + n0, c * sizeof(double), cudaMemcpyHostToDevice, st));
            }
            CK3(L->ops->init(L, dv, (uint32_t)n0, (uint32_t)c, st));
            CK3(cudaStreamSynchronize(st));
        }
    }
    CK3(L->ops->state_moments(L, st));
    if (pl.halo_parity) CK3(L->ops->publish(L, 0, st));
    CK3(cudaStreamSynchronize(st));
    return LBM_OK;
}

extern "C" lbm_status lbm3_create(const lbm3_params *p, const uint8_t *mask_host, void *d_workspace,
                                  size_t bytes, void *cuda_stream, lbm3_lattice **out) {
    if (!out) return lbm_fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    Plan3 pl;
    lbm_status s = lbm3_plan(p, &pl);
    if (s != LBM_OK) return s;
    if (!d_workspace || ((uintptr_t)d_workspace) % 256)
        return lbm_fail(LBM_EINVAL, "workspace must be non-NULL and 256-byte aligned");
    if (bytes < pl.total) return lbm_fail(LBM_ENOMEM, "workspace too small: %zu given, %zu needed", bytes, pl.total);
    if (!mask_host) return lbm_fail(LBM_EINVAL, "mask is NULL");
    lbm3_lattice *L = new lbm3_lattice();
    L->p = *p;
    L->pl = pl;
    L->ws = (char *)d_workspace;
    L->stream = (cudaStream_t)cuda_stream;
    L->ops = ops3_for(p->storage);
    L->block_1d = L->ops->block_1d(p->layout);
    L->ops->prepare(p->algo);
    L->off32 = (lbm3_offsets_fit(p, pl.N) && !(p->flags & LBM_FLAG_WIDE_OFFSETS)) ? 1 : 0;
    L->err = (unsigned int *)(L->ws + pl.misc);
    L->tctr = (long long *)(L->ws + pl.misc + 64);
    cudaError_t e = cudaStreamCreateWithFlags(&L->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete L;
        return lbm_cuda_fail(e, "cudaStreamCreateWithFlags");
    }
    uint8_t *dmask = (uint8_t *)(L->ws + pl.mom);   // staged in the moments region (>= N bytes)
    unsigned long long *dcount = (unsigned long long *)(L->ws + pl.partials);
    unsigned long long fluid = 0;
    const Geo3 g{p->nx, p->ny, p->nz, p->bc_x, p->bc_y, p->bc_z, east3_kind(p)};
    e = cudaMemcpyAsync(dmask, mask_host, (size_t)pl.N, cudaMemcpyHostToDevice, L->stream);
    if (e == cudaSuccess) {
        k3_links<<<(unsigned)((pl.N + 255) / 256), 256, 0, L->stream>>>(g, dmask, (uint32_t *)(L->ws + pl.links));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(dcount, 0, sizeof(*dcount), L->stream);
    if (e == cudaSuccess) {
        k3_count<<<1024, 256, 0, L->stream>>>((const uint32_t *)(L->ws + pl.links), (uint32_t)pl.N, dcount);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&fluid, dcount, sizeof(fluid), cudaMemcpyDeviceToHost, L->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(L->stream);
    if (e != cudaSuccess) {
        cudaStreamDestroy(L->cap);
        delete L;
        return lbm_cuda_fail(e, "lbm3_create");
    }
    L->fluid = (int64_t)fluid;
    s = lbm3_init(L, nullptr, nullptr, nullptr, nullptr);
    if (s != LBM_OK) {
        cudaStreamDestroy(L->cap);
        delete L;
        return s;
    }
    *out = L;
    return LBM_OK;
}

extern "C" void lbm3_destroy(lbm3_lattice *L) {
    if (!L) return;
    cudaStreamSynchronize(L->stream);
    for (auto &gx : L->graph)
        if (gx) cudaGraphExecDestroy(gx);
    cudaStreamDestroy(L->cap);
    delete L;
}

extern "C" lbm_status lbm3_step(lbm3_lattice *L, int64_t nsteps, uint32_t want_moments) {
    if (!L) return lbm_fail(LBM_EINVAL, "lattice is NULL");
    if (nsteps < 0) return lbm_fail(LBM_EINVAL, "nsteps must be >= 0");
    const int64_t G = 64;
    int64_t left = nsteps;
    while (!(L->p.flags & LBM_FLAG_NO_GRAPH) && (left > G || (left == G && !want_moments))) {
        cudaGraphExec_t &ex = L->graph[L->cur];
        if (!ex) {
            cudaGraph_t gr = nullptr;
            CK3(cudaStreamBeginCapture(L->cap, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = launch3(L, L->cap, G, 0);
            cudaError_t e2 = cudaStreamEndCapture(L->cap, &gr);
            if (e != cudaSuccess) {
                if (gr) cudaGraphDestroy(gr);
                return lbm_cuda_fail(e, "capturing D3Q19 updates");
            }
            if (e2 != cudaSuccess) return lbm_cuda_fail(e2, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&ex, gr, 0);
            cudaGraphDestroy(gr);
            if (e != cudaSuccess) return lbm_cuda_fail(e, "cudaGraphInstantiate");
        }
        CK3(cudaGraphLaunch(ex, L->stream));
        L->steps += G;
        left -= G;
    }
    if (left > 0) {
        CK3(launch3(L, L->stream, left, want_moments ? 1 : 0));
        if (left & 1) L->cur ^= 1;
        L->steps += left;
    }
    return LBM_OK;
}

lbm_status lbm3_check(lbm3_lattice *L) {
    unsigned int flag = 0;
    CK3(cudaMemcpy(&flag, L->err, sizeof(flag), cudaMemcpyDeviceToHost));
    if (flag) {
        CK3(cudaMemset(L->err, 0, sizeof(flag)));
        return lbm_fail(LBM_EDIVERGED, "non-finite density after %lld updates", (long long)L->steps);
    }
    return LBM_OK;
}

extern "C" lbm_status lbm3_sync(lbm3_lattice *L) {
    if (!L) return lbm_fail(LBM_EINVAL, "lattice is NULL");
    CK3(cudaStreamSynchronize(L->stream));
    return lbm3_check(L);
}

extern "C" lbm_status lbm3_read_moments(lbm3_lattice *L, double *rho, double *ux, double *uy, double *uz) {
    if (!L) return lbm_fail(LBM_EINVAL, "lattice is NULL");
    const int64_t N = L->pl.N;
    std::vector<unsigned char> buf(4 * (size_t)N * L->pl.comp);
    CK3(cudaStreamSynchronize(L->stream));
    CK3(cudaMemcpy(buf.data(), L->ws + L->pl.mom, buf.size(), cudaMemcpyDeviceToHost));
    double *dst[4] = {rho, ux, uy, uz};
    for (int k = 0; k < 4; ++k) {
        if (!dst[k]) continue;
        if (L->pl.comp == 8) {
            memcpy(dst[k], buf.data() + (size_t)k * N * 8, (size_t)N * 8);
        } else {
            const float *f = (const float *)(buf.data() + (size_t)k * N * 4);
            for (int64_t n = 0; n < N; ++n) dst[k][n] = f[n];
        }
    }
    return lbm3_check(L);
}

static double get_raw(const unsigned char *raw, int storage, int64_t k) {
    switch (storage) {
        case LBM_F64: return ((const double *)raw)[k];
        case LBM_F32: return ((const float *)raw)[k];
        case LBM_F16S: return __half2float(((const __half *)raw)[k]);
        default: return __bfloat162float(((const __nv_bfloat16 *)raw)[k]);
    }
}

static void set_raw(unsigned char *raw, int storage, int64_t k, double v) {
    switch (storage) {
        case LBM_F64: ((double *)raw)[k] = v; break;
        case LBM_F32: ((float *)raw)[k] = (float)v; break;
        case LBM_F16S: ((__half *)raw)[k] = __float2half_rn((float)v); break;
        default: ((__nv_bfloat16 *)raw)[k] = __float2bfloat16_rn((float)v); break;
    }
}

// AA pattern: the array holds the canonical state only after an even number
// of updates.
static lbm_status state_readable(const lbm3_lattice *L) {
    if (L->p.algo == LBM_AA && (L->steps & 1))
        return lbm_fail(LBM_EINVAL, "AA pattern: the state is accessible after an even number of updates only");
    return LBM_OK;
}

extern "C" lbm_status lbm3_read_populations(lbm3_lattice *L, void *host, int32_t as) {
    if (!L || !host) return lbm_fail(LBM_EINVAL, "NULL argument");
    if (state_readable(L) != LBM_OK) return LBM_EINVAL;
    if (as != LBM_F64 && as != LBM_F32) return lbm_fail(LBM_EINVAL, "as must be LBM_F64 or LBM_F32");
    const int64_t N = L->pl.N;
    std::vector<unsigned char> raw(19 * (size_t)N * L->pl.elem);
    CK3(cudaStreamSynchronize(L->stream));
    CK3(cudaMemcpy(raw.data(), L->ws + L->pl.pop[L->cur], raw.size(), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 19; ++i)
        for (int64_t n = 0; n < N; ++n) {
            const double v = get_raw(raw.data(), L->p.storage,
                                     lbm3_layout_index(L->p.layout, N, n, L->p.algo == LBM_NSOL ? 18 - i : i));
            if (as == LBM_F64) ((double *)host)[(int64_t)i * N + n] = v;
            else ((float *)host)[(int64_t)i * N + n] = (float)v;
        }
    return lbm3_check(L);
}

extern "C" lbm_status lbm3_write_populations(lbm3_lattice *L, const void *host, int32_t as) {
    if (!L || !host) return lbm_fail(LBM_EINVAL, "NULL argument");
    if (state_readable(L) != LBM_OK) return LBM_EINVAL;
    if (as != LBM_F64 && as != LBM_F32) return lbm_fail(LBM_EINVAL, "as must be LBM_F64 or LBM_F32");
    const int64_t N = L->pl.N;
    std::vector<unsigned char> raw(19 * (size_t)N * L->pl.elem);
    for (int i = 0; i < 19; ++i)
        for (int64_t n = 0; n < N; ++n) {
            const double v = as == LBM_F64 ? ((const double *)host)[(int64_t)i * N + n]
                                           : (double)((const float *)host)[(int64_t)i * N + n];
            set_raw(raw.data(), L->p.storage, lbm3_layout_index(L->p.layout, N, n, L->p.algo == LBM_NSOL ? 18 - i : i),
                    v);
        }
    CK3(cudaStreamSynchronize(L->stream));
    CK3(cudaMemcpy(L->ws + L->pl.pop[L->cur], raw.data(), raw.size(), cudaMemcpyHostToDevice));
    if (L->pl.halo_parity) {   // NPOL: the next update reads parity cur of the buffer grid
        CK3(L->ops->publish(L, L->cur, L->stream));
        CK3(cudaStreamSynchronize(L->stream));
    }
    return LBM_OK;
}

extern "C" lbm_status lbm3_mass(lbm3_lattice *L, double *out) {
    if (!L || !out) return lbm_fail(LBM_EINVAL, "NULL argument");
    if (state_readable(L) != LBM_OK) return LBM_EINVAL;
    double *partials = (double *)(L->ws + L->pl.partials);
    CK3(L->ops->mass(L, partials, L->stream));
    k3_sum<<<1, 32, 0, L->stream>>>(partials, kReduceBlocks, partials + kReduceBlocks);
    CK3(cudaGetLastError());
    CK3(cudaMemcpyAsync(out, partials + kReduceBlocks, sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    CK3(cudaStreamSynchronize(L->stream));
    return lbm3_check(L);
}

extern "C" lbm_status lbm3_force(lbm3_lattice *L, const uint8_t *d_body, double out[3]) {
    if (!L || !out) return lbm_fail(LBM_EINVAL, "NULL argument");
    if (state_readable(L) != LBM_OK) return LBM_EINVAL;
    double *partials = (double *)(L->ws + L->pl.partials);
    CK3(L->ops->force(L, d_body, partials, L->stream));
    k3_sum3<<<1, 32, 0, L->stream>>>(partials, kReduceBlocks, partials + 3 * kReduceBlocks);
    CK3(cudaGetLastError());
    CK3(cudaMemcpyAsync(out, partials + 3 * kReduceBlocks, 3 * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    CK3(cudaStreamSynchronize(L->stream));
    return lbm3_check(L);
}

extern "C" lbm_status lbm3_get_info(lbm3_lattice *L, lbm_info *out) {
    if (!L || !out) return lbm_fail(LBM_EINVAL, "NULL argument");
    memset(out, 0, sizeof(*out));
    out->cells = L->pl.N;
    out->fluid_cells = L->fluid;
    out->steps = L->steps;
    out->tile_x = L->p.algo == LBM_LPTL ? L->block_1d : L->pl.tx;
    out->tile_y = L->p.algo == LBM_LPTL ? 1 : L->pl.ty * L->pl.tz;
    out->bytes_per_update = (double)L->fluid * 38.0 * (double)L->pl.elem + 4.0 * (double)L->pl.N;
    if (L->pl.halo_parity)   // NPOL/NSOL buffer grid: one parity read, the other written
        out->bytes_per_update += 2.0 * (double)L->pl.halo_parity * (double)L->pl.elem;
    out->workspace_bytes = L->pl.total;
    // bit 0: the 64-bit addressing path; bit 1: two nodes per thread (16-bit storage)
    const bool pairs = (L->p.storage == LBM_F16S || L->p.storage == LBM_BF16S) && L->off32 &&
                       (L->p.layout == LBM_LAYOUT_BUNDLE || L->p.layout == LBM_LAYOUT_STREAM) &&
                       L->p.nx % 2 == 0 && !(L->p.flags & LBM_FLAG_NO_PAIRS) &&
                       (L->p.algo == LBM_LPTL || (L->p.algo == LBM_NPTL && L->pl.tx % 2 == 0));
    out->aux = (L->off32 ? 0 : 1) | (pairs ? 2 : 0);
    return LBM_OK;
}
