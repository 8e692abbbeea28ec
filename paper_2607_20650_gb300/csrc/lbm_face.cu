// Face exchange between x-slabs of one lattice: the multi-GPU extension the
// paper names as future work (Sec. 6) splits the lattice into slabs of whole
// columns, each with a ghost column on every face it shares with another slab.
// One pull update (Eq. 1) of a slab's first interior column reads, from the
// ghost column beside it, only the three populations that cross that face
// (c_ix = +1 across a west face, -1 across an east face). So after every
// update the owner of the neighbouring column sends those three values per
// node, and the receiver writes them into its ghost column; the interior of
// every slab then evolves exactly as the same columns of the undivided
// lattice.
//
// lbm_face_pack copies the three populations of one column of the current
// state into a dense buffer (the message), lbm_face_unpack writes a buffer
// into one column; lbm_face_exchange does both for every message between
// lattices of one process in one launch (no intermediate buffer). The values
// are moved as stored (bit copies of the storage type), so the exchange is
// exact for every storage type and rounding mode.
#include <cuda_runtime.h>

#include <cstdint>

#include "lbm.h"
#include "lbm_capi_internal.h"

namespace {

constexpr int kMaxFaceMessages = 64;

// Element offsets of the three exchanged populations of node (x, y) are
// base[k] + (y * nx + x) * stride in every layout: the layouts of Fig. 2 are
// affine in the node index for a fixed storage slot.
struct FaceMap {
    int64_t base[3];
    int64_t stride;
    int64_t nx;
    int32_t x, ny;
};

template <class E>
__global__ void k_face(E *pop, E *buf, FaceMap m, int unpack) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * (int64_t)m.ny) return;
    const int k = (int)(t / m.ny);
    const int64_t y = t - (int64_t)k * m.ny;
    const int64_t idx = m.base[k] + (y * m.nx + m.x) * m.stride;
    if (unpack)
        pop[idx] = buf[t];
    else
        buf[t] = pop[idx];
}

cudaError_t launch_face(size_t elem, void *pop, void *buf, const FaceMap &m, int unpack, cudaStream_t st) {
    const unsigned threads = 256;
    const unsigned blocks = (unsigned)((3 * (int64_t)m.ny + threads - 1) / threads);
    switch (elem) {
        case 8: k_face<uint64_t><<<blocks, threads, 0, st>>>((uint64_t *)pop, (uint64_t *)buf, m, unpack); break;
        case 4: k_face<uint32_t><<<blocks, threads, 0, st>>>((uint32_t *)pop, (uint32_t *)buf, m, unpack); break;
        default: k_face<uint16_t><<<blocks, threads, 0, st>>>((uint16_t *)pop, (uint16_t *)buf, m, unpack); break;
    }
    return cudaGetLastError();
}

lbm_status face_map(lbm_lattice *L, int32_t x, int32_t sense, const void *buf, FaceMap *m) {
    if (!L || !buf) return lbm_fail(LBM_EINVAL, "NULL argument");
    if (L->p.algo == LBM_AA)
        return lbm_fail(LBM_EINVAL, "face exchange needs a state stored the same way after every update (not AA)");
    if (x < 0 || x >= L->p.nx) return lbm_fail(LBM_EINVAL, "column %d outside [0, %d)", x, L->p.nx);
    if (sense != 1 && sense != -1) return lbm_fail(LBM_EINVAL, "sense must be +1 or -1");
    // Directions with c_ix = sense in the order c_iy = -1, 0, +1 (Fig. 2:
    // i = 3 (c_iy + 1) + (c_ix + 1)); swap streaming stores direction i in
    // slot 8 - i.
    const int rev = L->p.algo == LBM_NSOL;
    const int64_t N = L->pl.N;
    for (int k = 0; k < 3; ++k) {
        const int i = 3 * k + (sense + 1);
        const int slot = rev ? 8 - i : i;
        m->base[k] = layout_addr(L->p.layout, N, 0, slot);
    }
    m->stride = layout_addr(L->p.layout, N, 1, 0) - layout_addr(L->p.layout, N, 0, 0);
    m->nx = L->p.nx;
    m->x = x;
    m->ny = L->p.ny;
    return LBM_OK;
}

// Direct column-to-ghost copies of up to kCopiesPerLaunch messages between
// lattices of one process (same storage, layout, ny): message blockIdx.y.
constexpr int kCopiesPerLaunch = 16;

struct FaceCopy {
    const void *src;
    void *dst;
    int64_t sbase[3], dbase[3];
    int64_t snx, dnx;
    int32_t xs, xd;
};

struct FaceCopies {
    FaceCopy m[kCopiesPerLaunch];
    int64_t stride;
    int32_t ny;
};

template <class E>
__global__ void k_face_copy(const FaceCopies c) {
    const FaceCopy &m = c.m[blockIdx.y];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * (int64_t)c.ny) return;
    const int k = (int)(t / c.ny);
    const int64_t y = t - (int64_t)k * c.ny;
    const E v = ((const E *)m.src)[m.sbase[k] + (y * m.snx + m.xs) * c.stride];
    ((E *)m.dst)[m.dbase[k] + (y * m.dnx + m.xd) * c.stride] = v;
}

cudaError_t launch_face_copy(size_t elem, const FaceCopies &c, int count, cudaStream_t st) {
    const unsigned threads = 256;
    const dim3 grid((unsigned)((3 * (int64_t)c.ny + threads - 1) / threads), (unsigned)count);
    switch (elem) {
        case 8: k_face_copy<uint64_t><<<grid, threads, 0, st>>>(c); break;
        case 4: k_face_copy<uint32_t><<<grid, threads, 0, st>>>(c); break;
        default: k_face_copy<uint16_t><<<grid, threads, 0, st>>>(c); break;
    }
    return cudaGetLastError();
}

}  // namespace

extern "C" lbm_status lbm_face_exchange(int32_t count, lbm_lattice *const *src, const int32_t *xs,
                                        lbm_lattice *const *dst, const int32_t *xd, const int32_t *sense,
                                        void *cuda_stream) {
    if (count < 0 || count > kMaxFaceMessages) return lbm_fail(LBM_EINVAL, "count %d outside [0, %d]", count,
                                                                kMaxFaceMessages);
    if (count == 0) return LBM_OK;
    if (!src || !xs || !dst || !xd || !sense) return lbm_fail(LBM_EINVAL, "NULL argument");
    FaceMap ms[kMaxFaceMessages], md[kMaxFaceMessages];
    for (int k = 0; k < count; ++k) {
        lbm_status s = face_map(src[k], xs[k], sense[k], src[k], &ms[k]);
        if (s == LBM_OK) s = face_map(dst[k], xd[k], sense[k], dst[k], &md[k]);
        if (s != LBM_OK) return s;
        const lbm_lattice *a = src[k], *b = dst[k], *r = src[0];
        if (a->p.storage != r->p.storage || b->p.storage != r->p.storage || a->p.layout != r->p.layout ||
            b->p.layout != r->p.layout || a->p.algo != r->p.algo || b->p.algo != r->p.algo ||
            a->p.ny != r->p.ny || b->p.ny != r->p.ny)
            return lbm_fail(LBM_EINVAL, "message %d: lattices differ in storage, layout, algorithm or ny", k);
    }
    const cudaStream_t st = (cudaStream_t)cuda_stream;
    for (int k0 = 0; k0 < count; k0 += kCopiesPerLaunch) {
        const int n = count - k0 < kCopiesPerLaunch ? count - k0 : kCopiesPerLaunch;
        FaceCopies c{};
        c.stride = ms[k0].stride;
        c.ny = src[0]->p.ny;
        for (int j = 0; j < n; ++j) {
            const int k = k0 + j;
            FaceCopy &m = c.m[j];
            m.src = src[k]->h.pop[src[k]->cur];
            m.dst = dst[k]->h.pop[dst[k]->cur];
            for (int d = 0; d < 3; ++d) {
                m.sbase[d] = ms[k].base[d];
                m.dbase[d] = md[k].base[d];
            }
            m.snx = ms[k].nx;
            m.dnx = md[k].nx;
            m.xs = ms[k].x;
            m.xd = md[k].x;
        }
        cudaError_t e = launch_face_copy(src[0]->ops->elem, c, n, st);
        if (e != cudaSuccess) return lbm_cuda_fail(e, "face exchange");
    }
    // Buffer grids of the receivers (NPOL / NSOL), once each.
    for (int k = 0; k < count; ++k) {
        bool seen = false;
        for (int j = 0; j < k; ++j) seen = seen || dst[j] == dst[k];
        lbm_lattice *L = dst[k];
        if (seen || !L->pl.halo_grid) continue;
        cudaError_t e = L->ops->publish(L->h, L->cur, (int)(L->steps & 1), st);
        if (e != cudaSuccess) return lbm_cuda_fail(e, "buffer grid refresh after face exchange");
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_face_pack(lbm_lattice *L, int32_t x, int32_t sense, void *d_buf) {
    FaceMap m;
    lbm_status s = face_map(L, x, sense, d_buf, &m);
    if (s != LBM_OK) return s;
    cudaError_t e = launch_face(L->ops->elem, L->h.pop[L->cur], d_buf, m, 0, L->stream);
    return e == cudaSuccess ? LBM_OK : lbm_cuda_fail(e, "face pack");
}

extern "C" lbm_status lbm_face_unpack(lbm_lattice *L, int32_t x, int32_t sense, const void *d_buf) {
    FaceMap m;
    lbm_status s = face_map(L, x, sense, d_buf, &m);
    if (s != LBM_OK) return s;
    cudaError_t e = launch_face(L->ops->elem, L->h.pop[L->cur], const_cast<void *>(d_buf), m, 1, L->stream);
    if (e != cudaSuccess) return lbm_cuda_fail(e, "face unpack");
    // The one-lattice algorithms read populations of another tile from the
    // buffer grid, which holds copies of every tile's edge values: refresh it
    // from the lattice so the next update sees the received column there too.
    if (L->pl.halo_grid) {
        e = L->ops->publish(L->h, L->cur, (int)(L->steps & 1), L->stream);
        if (e != cudaSuccess) return lbm_cuda_fail(e, "buffer grid refresh after face unpack");
    }
    return LBM_OK;
}
