// Face exchange between x-slabs of one lattice: the multi-GPU extension the
// paper names as future work (Sec. 6) splits the lattice into slabs of whole
// columns (D2Q9) or planes (D3Q19), each with a ghost column / plane on every
// face it shares with another slab. One pull update (Eq. 1) of a slab's first
// interior column reads, from the ghost beside it, only the populations that
// cross that face: the directions with c_ix = +1 across a west face, -1
// across an east face (three in D2Q9, five in D3Q19). So after every update
// the owner of the neighbouring column sends those values per node, and the
// receiver writes them into its ghost; the interior of every slab then
// evolves exactly as the same columns of the undivided lattice.
//
// lbm_face_pack / lbm3_face_pack copy the crossing populations of one column
// of the current state into a dense buffer (the message), the unpack calls
// write a buffer into one column, and lbm_face_exchange / lbm3_face_exchange
// do both for every message between lattices of one process in one launch
// (no intermediate buffer). The values are moved as stored (bit copies of the
// storage type), so the exchange is exact for every storage type and
// rounding mode.
#include <cuda_runtime.h>

#include <cstdint>

#include "lbm.h"
#include "lbm3_device.cuh"
#include "lbm3_internal.h"
#include "lbm_capi_internal.h"

namespace {

constexpr int kMaxFaceMessages = 64;
constexpr int kMaxFaceDirs = 5;

// Element offset of exchanged direction k of node n = r * nx + x (r: the row
// y in 2-D, z * ny + y in 3-D): base[k] + n * stride[k]. Every layout of
// Fig. 2 and of the D3Q19 extension is affine in n for a fixed storage slot.
struct FaceMap {
    int64_t base[kMaxFaceDirs];
    int64_t stride[kMaxFaceDirs];
    int64_t nx;
    int32_t x, rows, q;
};

template <class E>
__global__ void k_face(E *pop, E *buf, const FaceMap m, int unpack) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)m.q * m.rows) return;
    const int k = (int)(t / m.rows);
    const int64_t r = t - (int64_t)k * m.rows;
    const int64_t idx = m.base[k] + (r * m.nx + m.x) * m.stride[k];
    if (unpack)
        pop[idx] = buf[t];
    else
        buf[t] = pop[idx];
}

cudaError_t launch_face(size_t elem, void *pop, void *buf, const FaceMap &m, int unpack, cudaStream_t st) {
    const unsigned threads = 256;
    const unsigned blocks = (unsigned)(((int64_t)m.q * m.rows + threads - 1) / threads);
    switch (elem) {
        case 8: k_face<uint64_t><<<blocks, threads, 0, st>>>((uint64_t *)pop, (uint64_t *)buf, m, unpack); break;
        case 4: k_face<uint32_t><<<blocks, threads, 0, st>>>((uint32_t *)pop, (uint32_t *)buf, m, unpack); break;
        default: k_face<uint16_t><<<blocks, threads, 0, st>>>((uint16_t *)pop, (uint16_t *)buf, m, unpack); break;
    }
    return cudaGetLastError();
}

// Direct column-to-ghost copies of up to kCopiesPerLaunch messages between
// lattices of one process (same storage, layout, algorithm and rows):
// message blockIdx.y.
constexpr int kCopiesPerLaunch = 16;

struct FaceCopy {
    const void *src;
    void *dst;
    int64_t sbase[kMaxFaceDirs], dbase[kMaxFaceDirs], stride[kMaxFaceDirs];
    int64_t snx, dnx;
    int32_t xs, xd;
};

struct FaceCopies {  // 2.6 KB of kernel parameters
    FaceCopy m[kCopiesPerLaunch];
    int32_t rows, q;
};

template <class E>
__global__ void k_face_copy(const FaceCopies c) {
    const FaceCopy &m = c.m[blockIdx.y];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)c.q * c.rows) return;
    const int k = (int)(t / c.rows);
    const int64_t r = t - (int64_t)k * c.rows;
    const E v = ((const E *)m.src)[m.sbase[k] + (r * m.snx + m.xs) * m.stride[k]];
    ((E *)m.dst)[m.dbase[k] + (r * m.dnx + m.xd) * m.stride[k]] = v;
}

cudaError_t launch_face_copy(size_t elem, const FaceCopies &c, int count, cudaStream_t st) {
    const unsigned threads = 256;
    const dim3 grid((unsigned)(((int64_t)c.q * c.rows + threads - 1) / threads), (unsigned)count);
    switch (elem) {
        case 8: k_face_copy<uint64_t><<<grid, threads, 0, st>>>(c); break;
        case 4: k_face_copy<uint32_t><<<grid, threads, 0, st>>>(c); break;
        default: k_face_copy<uint16_t><<<grid, threads, 0, st>>>(c); break;
    }
    return cudaGetLastError();
}

// What the exchange needs to know of a lattice of either kind.
struct FaceLattice {
    int layout, algo, storage, nx, rows;
    int64_t N;
    size_t elem;
    void *pop;  // current state
    int q3;     // D3Q19
};

FaceLattice face_lattice(const lbm_lattice *L) {
    return FaceLattice{L->p.layout, L->p.algo, L->p.storage, L->p.nx, L->p.ny, L->pl.N, L->ops->elem,
                       L->h.pop[L->cur], 0};
}

FaceLattice face_lattice(const lbm3_lattice *L) {
    return FaceLattice{L->p.layout, L->p.algo, L->p.storage, L->p.nx, L->p.ny * L->p.nz, L->pl.N, L->pl.elem,
                       L->ws + L->pl.pop[L->cur], 1};
}

int64_t slot_addr(const FaceLattice &f, int64_t n, int slot) {
    return f.q3 ? lbm3_layout_index(f.layout, f.N, n, slot) : layout_addr(f.layout, f.N, n, slot);
}

// Directions with c_ix = sense, in direction order: D2Q9 (Fig. 2) SE, E, NE
// or SW, W, NW; D3Q19 the five with c_x = sense.
int face_dirs(int q3, int sense, int *dirs) {
    int q = 0;
    if (q3) {
        for (int i = 0; i < lbm::d3::Q; ++i)
            if (lbm::d3::cx(i) == sense) dirs[q++] = i;
    } else {
        for (int i = 0; i < 9; ++i)
            if (lbm::cx(i) == sense) dirs[q++] = i;
    }
    return q;
}

lbm_status face_map(const FaceLattice &f, int32_t x, int32_t sense, FaceMap *m) {
    if (f.algo == LBM_AA)
        return lbm_fail(LBM_EINVAL, "face exchange needs a state stored the same way after every update (not AA)");
    if (x < 0 || x >= f.nx) return lbm_fail(LBM_EINVAL, "column %d outside [0, %d)", x, f.nx);
    if (sense != 1 && sense != -1) return lbm_fail(LBM_EINVAL, "sense must be +1 or -1");
    int dirs[kMaxFaceDirs + 4];
    m->q = face_dirs(f.q3, sense, dirs);
    // Swap streaming stores direction i in the opposite slot.
    const int opp_base = f.q3 ? 18 : 8;
    for (int k = 0; k < m->q; ++k) {
        const int slot = f.algo == LBM_NSOL ? opp_base - dirs[k] : dirs[k];
        m->base[k] = slot_addr(f, 0, slot);
        m->stride[k] = slot_addr(f, 1, slot) - m->base[k];
    }
    m->nx = f.nx;
    m->x = x;
    m->rows = f.rows;
    return LBM_OK;
}

// The one-lattice algorithms read populations of another tile from the
// buffer grid, which holds copies of every tile's edge values: refresh it
// from the lattice so the next update sees the received column there too.
cudaError_t refresh_buffer_grid(lbm_lattice *L, cudaStream_t st) {
    if (!L->pl.halo_grid) return cudaSuccess;
    return L->ops->publish(L->h, L->cur, (int)(L->steps & 1), st);
}

cudaError_t refresh_buffer_grid(lbm3_lattice *L, cudaStream_t st) {
    if (!L->pl.halo_parity) return cudaSuccess;
    return L->ops->publish(L, L->cur, st);
}

cudaStream_t stream_of(const lbm_lattice *L) { return L->stream; }
cudaStream_t stream_of(const lbm3_lattice *L) { return L->stream; }

template <class Lat>
lbm_status face_pack(Lat *L, int32_t x, int32_t sense, void *d_buf, int unpack) {
    if (!L || !d_buf) return lbm_fail(LBM_EINVAL, "NULL argument");
    const FaceLattice f = face_lattice(L);
    FaceMap m;
    lbm_status s = face_map(f, x, sense, &m);
    if (s != LBM_OK) return s;
    cudaError_t e = launch_face(f.elem, f.pop, d_buf, m, unpack, stream_of(L));
    if (e == cudaSuccess && unpack) e = refresh_buffer_grid(L, stream_of(L));
    return e == cudaSuccess ? LBM_OK : lbm_cuda_fail(e, unpack ? "face unpack" : "face pack");
}

template <class Lat>
lbm_status face_exchange(int32_t count, Lat *const *src, const int32_t *xs, Lat *const *dst, const int32_t *xd,
                         const int32_t *sense, void *cuda_stream) {
    if (count < 0 || count > kMaxFaceMessages)
        return lbm_fail(LBM_EINVAL, "count %d outside [0, %d]", count, kMaxFaceMessages);
    if (count == 0) return LBM_OK;
    if (!src || !xs || !dst || !xd || !sense) return lbm_fail(LBM_EINVAL, "NULL argument");
    for (int k = 0; k < count; ++k)
        if (!src[k] || !dst[k]) return lbm_fail(LBM_EINVAL, "NULL lattice in message %d", k);
    FaceMap ms[kMaxFaceMessages], md[kMaxFaceMessages];
    const FaceLattice r = face_lattice(src[0]);
    for (int k = 0; k < count; ++k) {
        const FaceLattice a = face_lattice(src[k]), b = face_lattice(dst[k]);
        lbm_status s = face_map(a, xs[k], sense[k], &ms[k]);
        if (s == LBM_OK) s = face_map(b, xd[k], sense[k], &md[k]);
        if (s != LBM_OK) return s;
        if (a.storage != r.storage || b.storage != r.storage || a.layout != r.layout || b.layout != r.layout ||
            a.algo != r.algo || b.algo != r.algo || a.rows != r.rows || b.rows != r.rows)
            return lbm_fail(LBM_EINVAL, "message %d: lattices differ in storage, layout, algorithm or face size", k);
    }
    const cudaStream_t st = (cudaStream_t)cuda_stream;
    for (int k0 = 0; k0 < count; k0 += kCopiesPerLaunch) {
        const int n = count - k0 < kCopiesPerLaunch ? count - k0 : kCopiesPerLaunch;
        FaceCopies c{};
        c.rows = r.rows;
        c.q = ms[k0].q;  // the same for every message: 3 (D2Q9) or 5 (D3Q19)
        for (int j = 0; j < n; ++j) {
            const int k = k0 + j;
            FaceCopy &m = c.m[j];
            m.src = face_lattice(src[k]).pop;
            m.dst = face_lattice(dst[k]).pop;
            // same layout and direction set on both sides: the same strides
            for (int d = 0; d < kMaxFaceDirs; ++d) {
                m.sbase[d] = ms[k].base[d];
                m.dbase[d] = md[k].base[d];
                m.stride[d] = ms[k].stride[d];
            }
            m.snx = ms[k].nx;
            m.dnx = md[k].nx;
            m.xs = ms[k].x;
            m.xd = md[k].x;
        }
        cudaError_t e = launch_face_copy(r.elem, c, n, st);
        if (e != cudaSuccess) return lbm_cuda_fail(e, "face exchange");
    }
    // Buffer grids of the receivers (NPOL / NSOL), once each.
    for (int k = 0; k < count; ++k) {
        bool seen = false;
        for (int j = 0; j < k; ++j) seen = seen || dst[j] == dst[k];
        if (seen) continue;
        cudaError_t e = refresh_buffer_grid(dst[k], st);
        if (e != cudaSuccess) return lbm_cuda_fail(e, "buffer grid refresh after face exchange");
    }
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_face_pack(lbm_lattice *L, int32_t x, int32_t sense, void *d_buf) {
    return face_pack(L, x, sense, d_buf, 0);
}

extern "C" lbm_status lbm_face_unpack(lbm_lattice *L, int32_t x, int32_t sense, const void *d_buf) {
    return face_pack(L, x, sense, const_cast<void *>(d_buf), 1);
}

extern "C" lbm_status lbm_face_exchange(int32_t count, lbm_lattice *const *src, const int32_t *xs,
                                        lbm_lattice *const *dst, const int32_t *xd, const int32_t *sense,
                                        void *cuda_stream) {
    return face_exchange(count, src, xs, dst, xd, sense, cuda_stream);
}

extern "C" lbm_status lbm3_face_pack(lbm3_lattice *L, int32_t x, int32_t sense, void *d_buf) {
    return face_pack(L, x, sense, d_buf, 0);
}

extern "C" lbm_status lbm3_face_unpack(lbm3_lattice *L, int32_t x, int32_t sense, const void *d_buf) {
    return face_pack(L, x, sense, const_cast<void *>(d_buf), 1);
}

extern "C" lbm_status lbm3_face_exchange(int32_t count, lbm3_lattice *const *src, const int32_t *xs,
                                         lbm3_lattice *const *dst, const int32_t *xd, const int32_t *sense,
                                         void *cuda_stream) {
    return face_exchange(count, src, xs, dst, xd, sense, cuda_stream);
}
