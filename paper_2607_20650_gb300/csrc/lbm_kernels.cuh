// Kernel templates of the D2Q9I BGK update (PortLBM Sec. 3.3), instantiated
// once per storage type by lbm_ops_*.cu. Every update kernel pulls the nine
// incoming values of a node (Sec. 3.3, one-step pull), substitutes boundary
// values, and calls the same collide() so that all layouts and algorithms
// produce the same bits.
#pragma once

#include <cuda_runtime.h>

#include <cstring>
#include <type_traits>

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

constexpr int kMaxTileThreads = 512;

template <class S>
struct Step {
    using C = typename Codec<S>::C;
    Geo geo;
    uint32_t N;
    Consts<C> k;
    const uint8_t *links;
    const S *src;
    S *dst;
    const S *halo_rd;
    S *halo_wr;
    C *mom;
    unsigned int *err;
    const long long *tctr;
    int toff;
    int sr;
    uint64_t seed;
    int tx, ty, ntx;
    uint64_t nx_magic;
    int off32;  // 9N < 2^32: element offsets fit 32 bits
    int aos16;  // nx % 16 == 0: warp segments of 32 records start on 16-byte boundaries
    uint32_t pf;  // L2 prefetch distance of the two-lattice kernel: nodes (LPTL), rows (NPTL); 0 = off
    Consts2 k2;   // FP32 arithmetic: k with every constant duplicated for the packed node pairs
};

// Host: FP64 constants rounded once to the compute type.
template <class S>
Step<S> make_step(const HostArgs &h, const StepCall &c) {
    using C = typename Codec<S>::C;
    Step<S> a;
    a.geo = Geo{h.nx, h.ny, h.bw, h.be, h.bs, h.bn};
    a.N = (uint32_t)h.N;
    Consts<C> &k = a.k;
    k.omega = (C)h.omega;
    k.hfx = (C)(0.5 * h.fx);
    k.hfy = (C)(0.5 * h.fy);
    k.fx = (C)h.fx;
    k.fy = (C)h.fy;
    k.sF = (C)(h.fx + h.fy);
    k.dF = (C)(h.fx - h.fy);
    k.w0 = (C)(1.0 / 36.0);
    k.w1 = (C)(1.0 / 9.0);
    k.w4 = (C)(4.0 / 9.0);
    k.wl0 = (C)(1.0 / 36.0 - (double)k.w0);
    k.wl1 = (C)(1.0 / 9.0 - (double)k.w1);
    k.wl4 = (C)(4.0 / 9.0 - (double)k.w4);
    k.kw0 = (C)(h.kf / 36.0);
    k.kw1 = (C)(h.kf / 9.0);
    k.kw4 = (C)(4.0 * h.kf / 9.0);
    k.zh5 = (C)(2.0 / 3.0 * h.ux_in);
    k.zh8 = (C)(h.ux_in / 6.0 + h.uy_in / 2.0);
    k.zh2 = (C)(h.ux_in / 6.0 - h.uy_in / 2.0);
    k.drho_out = (C)(h.rho_out - 1.0);
    const double W[9] = {1.0 / 36, 1.0 / 9, 1.0 / 36, 1.0 / 9, 4.0 / 9,
                         1.0 / 9, 1.0 / 36, 1.0 / 9, 1.0 / 36};
    for (int i = 0; i < 9; ++i) {
        double cu = cx(i) * h.ux_in + cy(i) * h.uy_in;
        double usq = h.ux_in * h.ux_in + h.uy_in * h.uy_in;
        k.heq_in[i] = (C)(W[i] * (3.0 * cu + 4.5 * cu * cu - 1.5 * usq));
    }
    k.force = (h.fx != 0.0 || h.fy != 0.0) ? 1 : 0;
    a.links = h.links;
    a.src = (const S *)h.pop[c.src];
    a.dst = (S *)(h.pop[1] ? h.pop[c.src ^ 1] : h.pop[0]);
    S *halo = (S *)h.halo;
    a.halo_rd = halo ? halo + (int64_t)c.rd_parity * h.halo_parity_elems : nullptr;
    a.halo_wr = halo ? halo + (int64_t)(c.rd_parity ^ 1) * h.halo_parity_elems : nullptr;
    a.mom = c.want_moments ? (C *)h.mom : nullptr;
    a.err = h.err;
    a.tctr = h.tctr;
    a.toff = c.toff;
    a.sr = h.rounding;
    a.seed = h.seed;
    a.tx = h.tile_x;
    a.ty = h.tile_y;
    a.ntx = h.ntx;
    a.nx_magic = h.nx_magic;
    a.off32 = (9 * h.N) < (int64_t(1) << 32) ? 1 : 0;
    a.aos16 = (h.nx % 16 == 0) ? 1 : 0;
    a.pf = h.pf;
    if constexpr (sizeof(C) == 4) a.k2 = make_consts2(a.k);
    else memset(&a.k2, 0, sizeof(a.k2));
    return a;
}

template <class S, int L>
__device__ __forceinline__ typename Codec<S>::C ldp(const S *base, uint32_t N, uint32_t n, int i) {
    return Codec<S>::dec(base[addr<L>(N, n, i)]);
}

#ifndef LBM_LDG_HINT
#define LBM_LDG_HINT 0
#endif
#ifndef LBM_ST_HINT
#define LBM_ST_HINT 0
#endif
// Loads of the read-only source lattice and stores of the destination
// lattice of the two-lattice update. Stores default to plain stores, which
// measured 1 % faster than evict-first (st.global.cs) for the bundle layout
// at 32 registers; LBM_ST_HINT=1 makes every store evict-first, 2 only the
// bundle layout's; LBM_LDG_HINT=1 loads through the read-only path (no
// measured difference).
template <class S>
__device__ __forceinline__ S ld_src(const S *p) {
#if LBM_LDG_HINT == 1
    return __ldg(p);
#else
    return *p;
#endif
}
template <class S, int L>
__device__ __forceinline__ void st_dst(S *p, S v) {
#if LBM_ST_HINT == 1
    __stcs(p, v);
#elif LBM_ST_HINT == 2
    if (L == BUNDLE)
        __stcs(p, v);
    else
        *p = v;
#else
    *p = v;
#endif
}

// Density deviation of node n + 1 (the Neumann inlet's east neighbour) in a
// stored state, summed in canonical direction order; 0 if it is solid.
template <class S, int L>
__device__ __forceinline__ typename Codec<S>::C neighbour_drho(const Step<S> &a, const S *lat, uint32_t n,
                                                               int rev) {
    using C = typename Codec<S>::C;
    if (a.links[n + 1] == SOLID_LINKS) return C(0);
    C d = C(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) d = Ar<C>::add(d, ldp<S, L>(lat, a.N, n + 1, rev ? opp(i) : i));
    return d;
}

// Inlet substitution, collision, divergence flag, moments, and encoding of
// the nine post-collision values (canonical direction order) into e.
// drho_nb: density deviation of node (1, y) in the previous state, used by
// the Neumann equilibrium inlet only.
// Inlet (x = 0) and outlet (x = nx - 1) substitutions of the pulled values.
// drho_nb: density deviation of node (1, y) in the previous state, used by
// the Neumann equilibrium inlet only.
template <class S>
__device__ __forceinline__ void edge_substitute(const Step<S> &a, uint32_t x, typename Codec<S>::C *g,
                                                typename Codec<S>::C drho_nb) {
    using C = typename Codec<S>::C;
    using A = Ar<C>;
    if (x == 0) {
        if (a.geo.bw == INLET_ZOUHE) {
            zou_he(a.k, g);
        } else if (a.geo.bw == INLET_EQ) {
#pragma unroll
            for (int i = 0; i < 9; ++i) g[i] = a.k.heq_in[i];
        } else if (a.geo.bw == INLET_EQ_NEUMANN) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const C w = i == 4 ? a.k.w4 : ((i & 1) ? a.k.w1 : a.k.w0);
                g[i] = A::fma(w, drho_nb, a.k.heq_in[i]);
            }
        }
    }
    if (x == (uint32_t)a.geo.nx - 1 && a.geo.be == OUTLET_PRESSURE) zou_he_pressure(a.k, g);
}

// Edge substitutions (EDGE = true; false when the caller has applied them or
// guarantees 0 < x < nx - 1, which keeps them out of the interior hot path),
// collision, divergence flag, moments, and encoding of the nine
// post-collision values (canonical direction order) into e.
template <class S, bool EDGE = true>
__device__ __forceinline__ void collide_encode(const Step<S> &a, uint32_t x, uint32_t n,
                                               typename Codec<S>::C *g, S *e,
                                               typename Codec<S>::C drho_nb = 0) {
    using C = typename Codec<S>::C;
    using A = Ar<C>;
    if (EDGE) edge_substitute(a, x, g, drho_nb);
    C drho, ux, uy;
    collide<Codec<S>::narrow>(a.k, g, drho, ux, uy);
    if (!isfinite(drho)) atomicOr(a.err, 1u);
    if (a.mom) {
        a.mom[n] = A::add(C(1), drho);
        a.mom[a.N + n] = ux;
        a.mom[2 * a.N + n] = uy;
    }
    const bool sr = Codec<S>::narrow && a.sr;
    uint32_t nk = 0;
    if (sr) nk = node_key(step_key(a.seed, (uint32_t)(*a.tctr + a.toff)), n);
#pragma unroll
    for (int i = 0; i < 9; ++i) e[i] = Codec<S>::enc(g[i], sr, sr ? pop_rand(nk, i) : 0u);
}

// ------------------------------------------------------------ two lattices
// Element offset of population i of node 0 in layout L; the offset of node n
// is lay_mul<L>() * n + lay_base<L>(N, i) for every layout.
template <int L> __host__ __device__ constexpr uint32_t lay_mul() {
    return L == STREAM ? 1u : (L == BUNDLE ? 3u : 9u);
}
template <int L> __device__ __forceinline__ uint32_t lay_base(uint32_t N, int i) {
    return L == STREAM ? (uint32_t)i * N
                       : (L == BUNDLE ? (uint32_t)(i / 3) * 3u * N + (uint32_t)(i % 3) : (uint32_t)i);
}

// Whether a solid node rewrites its (zero) record because it shares a
// 32-byte DRAM sector with a fluid node's record, from the warp's fluid
// ballot F (lanes = consecutive nodes). Only the stream layout does it
// (aligned groups of 32/sizeof(S) lanes): measured +9 % for the stream
// two-lattice kernels on the porous medium, but -6 % (FP32) / -10 % (FP16)
// for the bundle layout, -27 % for the AA pattern on it and -2 % for the
// collision layout, where the partial-sector writes cost less than the
// extra zeros.
template <class S, int L>
__device__ __forceinline__ bool shares_sector(unsigned F, int lane) {
    if (L != STREAM) return false;
    constexpr int G = (int)(32 / sizeof(S)) < 32 ? (int)(32 / sizeof(S)) : 32;
    const unsigned m = G >= 32 ? 0xffffffffu : ((1u << G) - 1u) << (lane & ~(G - 1));
    return (F & m) != 0u;
}

template <class S, int L>
__device__ __forceinline__ void store_zero(S *dst, uint32_t N, uint32_t n, int off32) {
    const S z = Codec<S>::enc(typename Codec<S>::C(0), false, 0u);
    if (off32) {
        const uint32_t base = lay_mul<L>() * n;
#pragma unroll
        for (int i = 0; i < 9; ++i) st_dst<S, L>(dst + base + lay_base<L>(N, i), z);
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) dst[addr<L>(N, n, i)] = z;
    }
}

// Pulls of an interior node (requires 9N < 2^32): pointers to the node's
// own record and to the rows above and below, plus per-direction constant
// offsets (immediates for the bundle and collision layouts); each pull picks
// the pulled neighbour or, for a bounced link, the node's opposite slot.
template <class S, int L>
__device__ __forceinline__ void pull_interior(const S *src, uint32_t n, uint32_t nx, uint32_t N, uint32_t lk,
                                              typename Codec<S>::C *g) {
    const S *own = src + lay_mul<L>() * n;
    const S *rs = own + (ptrdiff_t)lay_mul<L>() * nx;  // row y+1: source of c_y = -1
    const S *rn = own - (ptrdiff_t)lay_mul<L>() * nx;  // row y-1: source of c_y = +1
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        if (i == 4) {
            g[i] = Codec<S>::dec(ld_src(own + (ptrdiff_t)lay_base<L>(N, 4)));
            continue;
        }
        const S *row = cy(i) < 0 ? rs : (cy(i) > 0 ? rn : own);
        const S *pp = row + ((ptrdiff_t)lay_base<L>(N, i) - (ptrdiff_t)lay_mul<L>() * cx(i));
        const S *pb = own + (ptrdiff_t)lay_base<L>(N, opp(i));
        g[i] = Codec<S>::dec(ld_src(((lk >> link_bit(i)) & 1u) ? pb : pp));
    }
}

template <class S, int L>
__device__ __forceinline__ void store_node(S *dst, uint32_t n, uint32_t N, int off32, const S *e) {
    if (off32) {
        S *od = dst + lay_mul<L>() * n;
#pragma unroll
        for (int i = 0; i < 9; ++i) st_dst<S, L>(od + (ptrdiff_t)lay_base<L>(N, i), e[i]);
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) dst[addr<L>(N, n, i)] = e[i];
    }
}

// Pull, collide and store one fluid node of the two-lattice update. Interior
// nodes take a path with 32-bit element offsets where each pull is one
// select between two uniform offsets (pulled neighbour or own opposite slot);
// nodes on the domain edge take the general mapping.
template <class S, int L>
__device__ __forceinline__ void two_lattice_fluid(const Step<S> &a, uint32_t x, uint32_t y, uint32_t n,
                                                  uint32_t lk) {
    using C = typename Codec<S>::C;
    const uint32_t nx = (uint32_t)a.geo.nx, ny = (uint32_t)a.geo.ny;
    S *__restrict__ dst = a.dst;
    const S *__restrict__ src = a.src;
    const bool interior = (x - 1u < nx - 2u) && (y - 1u < ny - 2u);
    C g[9];
    if (interior && a.off32) {
        pull_interior<S, L>(src, n, nx, a.N, lk, g);
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (i == 4) {
                g[i] = ldp<S, L>(src, a.N, n, 4);
                continue;
            }
            if ((lk >> link_bit(i)) & 1u) {
                g[i] = ldp<S, L>(src, a.N, n, opp(i));
            } else if (interior) {
                g[i] = ldp<S, L>(src, a.N, n - (uint32_t)(cy(i) * (int)nx + cx(i)), i);
            } else {
                int xs, ys, j;
                if (map_pull(a.geo, (int)x, (int)y, i, xs, ys, j) == PULL_NODE)
                    g[i] = ldp<S, L>(src, a.N, (uint32_t)ys * nx + (uint32_t)xs, j);
                else
                    g[i] = C(0);  // inlet unknown, reconstructed by edge_substitute
            }
        }
        const C dnb = (x == 0 && a.geo.bw == INLET_EQ_NEUMANN) ? neighbour_drho<S, L>(a, src, n, 0) : C(0);
        edge_substitute(a, x, g, dnb);
    }
    S e[9];
    collide_encode<S, false>(a, x, n, g, e);
    store_node<S, L>(dst, n, a.N, a.off32, e);
}

// One node of the two-lattice pull update (LPTL and NPTL). lane: the
// thread's lane (the zero fill below votes over the warp).
template <class S, int L>
__device__ __forceinline__ void two_lattice_node(const Step<S> &a, uint32_t x, uint32_t y, int lane) {
    const uint32_t n = y * (uint32_t)a.geo.nx + x;
    const uint32_t lk = a.links[n];
    const bool fluid = lk != SOLID_LINKS;
    const unsigned F = __ballot_sync(__activemask(), fluid);
    if (!fluid) {
        // Solid nodes hold h = 0 and are never read. Where a solid node's
        // record shares a DRAM sector with a fluid node's, store the zeros
        // again so the sector is written whole (no read-modify-write).
        if (shares_sector<S, L>(F, lane)) store_zero<S, L>(a.dst, a.N, n, a.off32);
        return;
    }
    two_lattice_fluid<S, L>(a, x, y, n, lk);
}

// NPTL with two nodes per thread, rows y and y + ty/2 of a tx x ty tile:
// both link bytes, then all eighteen pulls of interior nodes are issued
// before either collision, so one thread keeps twice the loads in flight.
template <class S, int L>
__global__ void __launch_bounds__(kMaxTileThreads) k_two_lattice2(const Step<S> a) {
    using C = typename Codec<S>::C;
    const uint32_t nx = (uint32_t)a.geo.nx, ny = (uint32_t)a.geo.ny;
    const uint32_t x = blockIdx.x * a.tx + threadIdx.x;
    const uint32_t ya = blockIdx.y * a.ty + threadIdx.y, yb = ya + (uint32_t)(a.ty >> 1);
    if (x >= nx || ya >= ny) return;
    const int lane = (int)((threadIdx.y * blockDim.x + threadIdx.x) & 31u);
    const bool hb = yb < ny;
    const uint32_t na = ya * nx + x, nb = yb * nx + x;
    const uint32_t lka = a.links[na];
    const uint32_t lkb = hb ? (uint32_t)a.links[nb] : SOLID_LINKS;
    const bool fa = lka != SOLID_LINKS, fb = lkb != SOLID_LINKS;
    const unsigned act = __activemask();
    const unsigned Fa = __ballot_sync(act, fa), Fb = __ballot_sync(act, hb && fb);
    if (!fa && shares_sector<S, L>(Fa, lane)) store_zero<S, L>(a.dst, a.N, na, a.off32);
    if (hb && !fb && shares_sector<S, L>(Fb, lane)) store_zero<S, L>(a.dst, a.N, nb, a.off32);
    const bool fast_a = fa && a.off32 && (x - 1u < nx - 2u) && (ya - 1u < ny - 2u);
    const bool fast_b = fb && a.off32 && (x - 1u < nx - 2u) && (yb - 1u < ny - 2u);
    C ga[9], gb[9];
    if (fast_a) pull_interior<S, L>(a.src, na, nx, a.N, lka, ga);
    if (fast_b) pull_interior<S, L>(a.src, nb, nx, a.N, lkb, gb);
    S e[9];
    if (fast_a) {
        collide_encode<S, false>(a, x, na, ga, e);
        store_node<S, L>(a.dst, na, a.N, a.off32, e);
    } else if (fa) {
        two_lattice_fluid<S, L>(a, x, ya, na, lka);
    }
    if (fast_b) {
        collide_encode<S, false>(a, x, nb, gb, e);
        store_node<S, L>(a.dst, nb, a.N, a.off32, e);
    } else if (fb) {
        two_lattice_fluid<S, L>(a, x, yb, nb, lkb);
    }
}

// Collision layout (9 contiguous values per node), NPTL: a warp owns 32
// consecutive nodes of a row. For warps of 32 fluid nodes away from the domain
// edges, the three source row spans (nodes x0-1 .. x0+32 of rows y+1, y, y-1)
// are staged in shared memory with 16-byte loads, the pulls read shared
// memory, and the 32 output records are written back with 16-byte stores.
// Other warps use the per-node path.
template <class S>
struct AosSpan {
    static constexpr int R = 9 * (int)sizeof(S);                    // record bytes
    static constexpr int CHUNKS = (34 * R + 15) / 16 + 1;           // 16-byte chunks per row span
    static constexpr int ROW_BYTES = CHUNKS * 16;
    static constexpr int WARP_BYTES = 3 * ROW_BYTES;
};

template <class S>
__global__ void __launch_bounds__(kMaxTileThreads, sizeof(S) == 8 ? 1 : 4) k_two_lattice_aos(const Step<S> a) {
    using C = typename Codec<S>::C;
    using SP = AosSpan<S>;
    extern __shared__ __align__(16) unsigned char smem_aos[];
    const uint32_t nx = (uint32_t)a.geo.nx, ny = (uint32_t)a.geo.ny;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const uint32_t x = blockIdx.x * a.tx + threadIdx.x;
    const uint32_t y = blockIdx.y * a.ty + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const uint32_t n = y * nx + x;
    const uint32_t lk = a.links[n];
    const bool fluid = lk != SOLID_LINKS;
    const unsigned act = __activemask();
    const unsigned F = __ballot_sync(act, fluid);
    const uint32_t x0 = x - (uint32_t)lane;   // first node of this warp's row segment
    // Staging pays off for warps of fluid nodes only (measured): with solid
    // nodes in the warp the spans carry unused records and the stores stay scalar.
    const bool staged = F == 0xffffffffu && a.off32 && a.aos16 && x0 >= 1u && x0 + 33u <= nx &&
                        y >= 1u && y + 2u <= ny;
    if (!staged) {
        if (!fluid) {
            if (shares_sector<S, COLLISION>(F, lane)) store_zero<S, COLLISION>(a.dst, a.N, n, a.off32);
            return;
        }
        two_lattice_fluid<S, COLLISION>(a, x, y, n, lk);
        return;
    }
    unsigned char *wbuf = smem_aos + (size_t)warp * SP::WARP_BYTES;
    const uint32_t n0 = y * nx + x0;
    const unsigned char *srcb = reinterpret_cast<const unsigned char *>(a.src);
    int shift[3];   // bytes from each staged span start to record (n0 - 1 - c_y nx)
#pragma unroll
    for (int r = 0; r < 3; ++r) {       // r = c_y + 1: source row y - c_y
        const uint64_t first = (uint64_t)SP::R * (uint64_t)(n0 - 1u - (uint32_t)((r - 1) * (int)nx));
        const uint64_t base = first & ~(uint64_t)15;
        shift[r] = (int)(first - base);
        const uint4 *g4 = reinterpret_cast<const uint4 *>(srcb + base);
        uint4 *s4 = reinterpret_cast<uint4 *>(wbuf + r * SP::ROW_BYTES);
#pragma unroll
        for (int k = lane; k < SP::CHUNKS; k += 32) s4[k] = __ldg(g4 + k);
    }
    __syncwarp();
    C g[9];
    if (fluid) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const S *pp = reinterpret_cast<const S *>(wbuf + (cy(i) + 1) * SP::ROW_BYTES + shift[cy(i) + 1]) +
                          (lane + 1 - cx(i)) * 9 + i;
            const S *pb = reinterpret_cast<const S *>(wbuf + SP::ROW_BYTES + shift[1]) + (lane + 1) * 9 + opp(i);
            g[i] = Codec<S>::dec(((lk >> link_bit(i)) & 1u) ? *pb : *pp);
        }
    }
    S e[9];
    if (fluid) collide_encode(a, x, n, g, e);
    if (F != 0xffffffffu) {
        if (fluid) {
            store_node<S, COLLISION>(a.dst, n, a.N, a.off32, e);
        } else if (shares_sector<S, COLLISION>(F, lane)) {
            store_zero<S, COLLISION>(a.dst, a.N, n, a.off32);
        }
        return;
    }
    __syncwarp();   // every lane has read its inputs; reuse the first span for the output
    S *out = reinterpret_cast<S *>(wbuf);
#pragma unroll
    for (int i = 0; i < 9; ++i) out[lane * 9 + i] = e[i];
    __syncwarp();
    uint4 *d4 = reinterpret_cast<uint4 *>(reinterpret_cast<unsigned char *>(a.dst) + (uint64_t)SP::R * n0);
    const uint4 *o4 = reinterpret_cast<const uint4 *>(wbuf);
    constexpr int OUT_CHUNKS = 32 * SP::R / 16;
#pragma unroll
    for (int k = lane; k < OUT_CHUNKS; k += 32) d4[k] = o4[k];
}

// L2 prefetch of one node's source record (stream and bundle layouts): one
// address per DRAM sector the record occupies, every value of the stream
// layout and the first value of each bundle (a bundle straddling two sectors
// has its second one fetched by the neighbour's prefetch).
template <class S, int L>
__device__ __forceinline__ void prefetch_record(const S *src, uint32_t N, uint32_t n) {
#pragma unroll
    for (int i = 0; i < 9; ++i)
        if (L == STREAM || i % 3 == 0)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(src + addr<L>(N, n, i)));
}

// LPTL (LINEAR: one node per thread over n, block size from the runtime) and
// NPTL (2-D tiles of tx x ty nodes over a padded grid).
//
// Blocks start in index order, so the node a.pf nodes (LPTL) or a.pf rows
// (NPTL) ahead belongs to a block that starts a few microseconds later. Each
// thread loads that node's link byte first and, once its own node is stored,
// prefetches the node's source record into L2 when it is fluid: the pulls of
// the later block then hit L2 instead of waiting on DRAM, and the prefetches
// keep more DRAM requests in flight than the pulls alone at full occupancy.
// Solid records are not fetched, so DRAM traffic does not grow. Only 32-bit
// storage in the stream and bundle layouts has it: the 16-bit update is bound
// by instruction issue (the prefetch cost 3 %), and the collision layout's
// LPTL form spills at 32 registers with it (its NPTL form is the staged
// kernel above).
template <class S, int L, bool LINEAR>
__global__ void __launch_bounds__(kMaxTileThreads, sizeof(S) == 8 ? 1 : 4) k_two_lattice(const Step<S> a) {
    const uint32_t nx = (uint32_t)a.geo.nx, ny = (uint32_t)a.geo.ny;
    constexpr bool PF = sizeof(S) == 4 && L != COLLISION;
    uint32_t x, y, np = 0;
    bool ahead;
    if (LINEAR) {
        const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
        if (n >= a.N) return;
        y = a.nx_magic ? (uint32_t)__umul64hi((unsigned long long)n, a.nx_magic) : n;
        x = n - y * nx;
        ahead = PF && a.pf != 0u && a.N - n > a.pf;
        np = n + a.pf;
    } else {
        x = blockIdx.x * a.tx + threadIdx.x;
        y = blockIdx.y * a.ty + threadIdx.y;
        if (x >= nx || y >= ny) return;
        ahead = PF && a.pf != 0u && ny - y > a.pf;
        np = (y + a.pf) * nx + x;
    }
    const uint32_t lkp = ahead ? (uint32_t)a.links[np] : SOLID_LINKS;
    two_lattice_node<S, L>(a, x, y, (int)((threadIdx.y * blockDim.x + threadIdx.x) & 31u));
    if (PF && lkp != SOLID_LINKS) prefetch_record<S, L>(a.src, a.N, np);
}

// ------------------------------------------------------------ node pairs
// Two-lattice update (LPTL, NPTL) for 16-bit storage with two horizontally
// adjacent nodes per thread, x even (nx even, so a pair never wraps a row).
// The 16-bit update is bound by instruction issue, not by DRAM, so the pair
// shares what one node per thread repeats: one 16-bit load brings both link
// bytes, the collision runs on packed FP32 pairs (collide2: each lane is the
// scalar collide() bit for bit), two results are rounded to 16 bits by one
// packed conversion, and the stores are 32-bit words. A pair's values of
// one direction are adjacent in the stream layout (i N + n, n even); in the
// bundle layout a pair's bundle is six adjacent values (3n even), stored as
// three words. A solid node of a pair holding a fluid one stores its zeros in
// the same words, so the pair's sector is written whole. Pairs touching the
// domain edge take the per-node path.
template <class S>
__device__ __forceinline__ uint32_t pack_rne(float lo, float hi) {
    uint32_t r;
    if constexpr (sizeof(S) == 2 && std::is_same<S, __half>::value)
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    else
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// Encoded 16-bit pair words for the nine directions: word i holds direction i
// of node a (low half) and node b (high half). A node with keep = false
// contributes +0.
template <class S>
__device__ __forceinline__ void encode_pair(const Step<S> &a, uint32_t n, const f2 *g, bool ka, bool kb,
                                            uint32_t *w) {
    const bool sr = a.sr != 0;
    if (!sr) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            float lo, hi;
            up2(g[i], lo, hi);
            w[i] = pack_rne<S>(ka ? lo : 0.0f, kb ? hi : 0.0f);
        }
    } else {
        // one packed stochastic conversion per direction: node a in the low
        // half, node b in the high half, each with its own draw (a solid
        // node's lane converts +0, which no draw changes)
        const uint32_t sk = step_key(a.seed, (uint32_t)(*a.tctr + a.toff));
        const uint32_t nka = node_key(sk, n), nkb = node_key(sk, n + 1);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            float lo, hi;
            up2(g[i], lo, hi);
            lo = ka ? lo : 0.0f;
            hi = kb ? hi : 0.0f;
            if constexpr (std::is_same<S, __half>::value)
                w[i] = sr_half2(hi, lo, pop_rand(nkb, i), pop_rand(nka, i));
            else
                w[i] = sr_bf162(hi, lo, pop_rand(nkb, i), pop_rand(nka, i));
        }
    }
}

// Store the pair words of nodes n, n + 1 (n even) in layout L (STREAM or BUNDLE).
template <class S, int L>
__device__ __forceinline__ void store_pair(S *dst, uint32_t N, uint32_t n, const uint32_t *w) {
    if (L == STREAM) {
#pragma unroll
        for (int i = 0; i < 9; ++i) *reinterpret_cast<uint32_t *>(dst + (uint32_t)i * N + n) = w[i];
    } else {
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            uint32_t *p = reinterpret_cast<uint32_t *>(dst + (uint32_t)b * 3u * N + 3u * n);
            const uint32_t w0 = w[3 * b], w1 = w[3 * b + 1], w2 = w[3 * b + 2];
            p[0] = (w0 & 0xFFFFu) | (w1 << 16);            // (a, 3b), (a, 3b+1)
            p[1] = (w2 & 0xFFFFu) | (w0 & 0xFFFF0000u);    // (a, 3b+2), (b, 3b)
            p[2] = (w1 >> 16) | (w2 & 0xFFFF0000u);        // (b, 3b+1), (b, 3b+2)
        }
    }
}

// L2 prefetch of a pair's source records (both nodes): one address per
// bundle, or per direction in the stream layout.
template <class S, int L>
__device__ __forceinline__ void prefetch_pair(const S *src, uint32_t N, uint32_t n) {
#pragma unroll
    for (int i = 0; i < 9; ++i)
        if (L == STREAM || i % 3 == 0)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(src + addr<L>(N, n, i)));
}

// One pair: both link bytes in lk2 (node n in the low byte).
template <class S, int L>
__device__ __forceinline__ void pair_update(const Step<S> &a, uint32_t x, uint32_t y, uint32_t n, uint32_t lk2,
                                            int lane) {
    const uint32_t nx = (uint32_t)a.geo.nx, ny = (uint32_t)a.geo.ny;
    const uint32_t lka = lk2 & 0xFFu, lkb = lk2 >> 8;
    const bool fa = lka != SOLID_LINKS, fb = lkb != SOLID_LINKS;
    const unsigned F = __ballot_sync(__activemask(), fa || fb);
    if (!fa && !fb) {
        // Stream layout: rewrite the zeros of a solid pair whose 32-byte
        // sector (16 nodes = 8 pairs) also holds fluid nodes.
        if (L == STREAM) {
            const unsigned m = 0xFFu << (lane & ~7);
            if (F & m) {
                const uint32_t z[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
                store_pair<S, L>(a.dst, a.N, n, z);
            }
        }
        return;
    }
    const bool interior = (x - 1u < nx - 3u) && (y - 1u < ny - 2u);
    if (!interior || !a.off32) {
        if (fa) two_lattice_fluid<S, L>(a, x, y, n, lka);
        else if (L == STREAM) store_zero<S, L>(a.dst, a.N, n, a.off32);
        if (fb) two_lattice_fluid<S, L>(a, x + 1u, y, n + 1u, lkb);
        else if (L == STREAM) store_zero<S, L>(a.dst, a.N, n + 1u, a.off32);
        return;
    }
    // both nodes' pulls, direction by direction, into packed pairs (node b's
    // values sit one record after node a's; a solid node's lane is +0)
    f2 g[9];
    {
        const S *own = a.src + lay_mul<L>() * n;
        const S *rs = own + (ptrdiff_t)lay_mul<L>() * nx;  // row y+1: source of c_y = -1
        const S *rn = own - (ptrdiff_t)lay_mul<L>() * nx;  // row y-1: source of c_y = +1
        constexpr ptrdiff_t m = lay_mul<L>();
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const S *pa, *pb;
            if (i == 4) {
                pa = own + (ptrdiff_t)lay_base<L>(a.N, 4);
                pb = pa + m;
            } else {
                const S *row = cy(i) < 0 ? rs : (cy(i) > 0 ? rn : own);
                const S *pp = row + ((ptrdiff_t)lay_base<L>(a.N, i) - m * cx(i));
                const S *po = own + (ptrdiff_t)lay_base<L>(a.N, opp(i));
                pa = ((lka >> link_bit(i)) & 1u) ? po : pp;
                pb = (((lkb >> link_bit(i)) & 1u) ? po : pp) + m;
            }
            const float va = fa ? Codec<S>::dec(ld_src(pa)) : 0.0f;
            const float vb = fb ? Codec<S>::dec(ld_src(pb)) : 0.0f;
            g[i] = pk2(va, vb);
        }
    }
    f2 drho2, ux2, uy2;
    collide2(a.k2, a.k.force, g, drho2, ux2, uy2);
    float da, db;
    up2(drho2, da, db);
    if ((fa && !isfinite(da)) || (fb && !isfinite(db))) atomicOr(a.err, 1u);
    if (a.mom) {
        const f2 r2 = add2(dup2(1.0f), drho2);
        if (fa && fb) {
            *reinterpret_cast<f2 *>(a.mom + n) = r2;
            *reinterpret_cast<f2 *>(a.mom + a.N + n) = ux2;
            *reinterpret_cast<f2 *>(a.mom + 2 * a.N + n) = uy2;
        } else {
            float r0, r1, u0, u1, v0, v1;
            up2(r2, r0, r1);
            up2(ux2, u0, u1);
            up2(uy2, v0, v1);
            const uint32_t m = fa ? n : n + 1u;
            a.mom[m] = fa ? r0 : r1;
            a.mom[a.N + m] = fa ? u0 : u1;
            a.mom[2 * a.N + m] = fa ? v0 : v1;
        }
    }
    if (L == BUNDLE && fa && fb && !a.sr) {
        // both fluid, nearest rounding: each 32-bit word of a bundle pair is
        // one packed conversion of the two values it holds
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            float a0, b0, a1, b1, a2, b2;
            up2(g[3 * b], a0, b0);
            up2(g[3 * b + 1], a1, b1);
            up2(g[3 * b + 2], a2, b2);
            uint32_t *p = reinterpret_cast<uint32_t *>(a.dst + (uint32_t)b * 3u * a.N + 3u * n);
            p[0] = pack_rne<S>(a0, a1);
            p[1] = pack_rne<S>(a2, b0);
            p[2] = pack_rne<S>(b1, b2);
        }
        return;
    }
    uint32_t w[9];
    encode_pair<S>(a, n, g, fa, fb, w);
    store_pair<S, L>(a.dst, a.N, n, w);
}

// a.pf: L2 prefetch distance as for the 32-bit kernel (pairs of nodes for
// LPTL, rows for NPTL; 0 = off): the link bytes of the pair that far ahead
// are loaded first, and after the pair is stored its source records are
// prefetched into L2 when either node is fluid.
// Measured on the 134M-node porous lattice (FP16, bundle, NPTL 32 x 8): 72
// registers unbounded gives 119 GLUPS, 48 (five blocks of 256) 144, 40 with
// spills 143; one node per thread 126.
#ifndef LBM_PAIR_MINB
#define LBM_PAIR_MINB 5
#endif
template <class S, int L, bool LINEAR>
__global__ void __launch_bounds__(kMaxTileThreads / 2, LBM_PAIR_MINB) k_two_lattice_pair(const Step<S> a) {
    const uint32_t nx = (uint32_t)a.geo.nx, ny = (uint32_t)a.geo.ny;
    uint32_t x, y, n, np;
    bool ahead;
    if (LINEAR) {
        n = 2u * (blockIdx.x * blockDim.x + threadIdx.x);
        if (n >= a.N) return;
        y = a.nx_magic ? (uint32_t)__umul64hi((unsigned long long)n, a.nx_magic) : n;
        x = n - y * nx;
        ahead = a.pf != 0u && a.N - n > 2u * a.pf;
        np = n + 2u * a.pf;
    } else {
        x = blockIdx.x * (uint32_t)a.tx + 2u * threadIdx.x;
        y = blockIdx.y * (uint32_t)a.ty + threadIdx.y;
        if (x >= nx || y >= ny) return;
        n = y * nx + x;
        ahead = a.pf != 0u && ny - y > a.pf;
        np = n + a.pf * nx;
    }
    const uint32_t lkp = ahead ? (uint32_t)*reinterpret_cast<const unsigned short *>(a.links + np) : 0xFFFFu;
    const uint32_t lk2 = *reinterpret_cast<const unsigned short *>(a.links + n);
    pair_update<S, L>(a, x, y, n, lk2, (int)((threadIdx.y * blockDim.x + threadIdx.x) & 31u));
    if (lkp != 0xFFFFu) prefetch_pair<S, L>(a.src, a.N, np);
}

// ------------------------------------------------------------ buffer grid
// Per tile and parity: east edge 3 x ty values (directions 2,5,8), west
// 3 x ty (0,3,6), north 3 x tx (6,7,8), south 3 x tx (0,1,2).
enum Edge { EDGE_E = 0, EDGE_W = 1, EDGE_N = 2, EDGE_S = 3 };

__device__ __forceinline__ int64_t halo_slot(int tx, int ty, int ntx, int bx, int by, int edge,
                                             int k, int pos) {
    int64_t base = (int64_t)(by * ntx + bx) * (6 * (tx + ty));
    switch (edge) {
        case EDGE_E: return base + k * ty + pos;
        case EDGE_W: return base + 3 * ty + k * ty + pos;
        case EDGE_N: return base + 6 * ty + k * tx + pos;
        default: return base + 6 * ty + 3 * tx + k * tx + pos;
    }
}

// Value S[(xs, ys)][j] of a node in another tile, as that tile published it.
template <class S>
__device__ __forceinline__ typename Codec<S>::C halo_read(const Step<S> &a, int xs, int ys, int j,
                                                          int bx) {
    const int bxs = xs / a.tx, bys = ys / a.ty;
    int64_t s;
    if (bxs != bx)
        s = halo_slot(a.tx, a.ty, a.ntx, bxs, bys, cx(j) > 0 ? EDGE_E : EDGE_W, j / 3, ys - bys * a.ty);
    else
        s = halo_slot(a.tx, a.ty, a.ntx, bxs, bys, cy(j) > 0 ? EDGE_N : EDGE_S, j % 3, xs - bxs * a.tx);
    return Codec<S>::dec(a.halo_rd[s]);
}

// Publish the populations of an edge node that leave its tile.
template <class S>
__device__ __forceinline__ void halo_publish(S *hw, int tx, int ty, int ntx, int bx, int by, int x,
                                             int y, int x0, int y0, int x1, int y1, const S *e) {
    S *t = hw + (int64_t)(by * ntx + bx) * (6 * (tx + ty));
    const int r = y - y0, c = x - x0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (x == x1) t[k * ty + r] = e[3 * k + 2];                  // east:  2, 5, 8
        if (x == x0) t[3 * ty + k * ty + r] = e[3 * k];             // west:  0, 3, 6
        if (y == y1) t[6 * ty + k * tx + c] = e[6 + k];             // north: 6, 7, 8
        if (y == y0) t[6 * ty + 3 * tx + k * tx + c] = e[k];        // south: 0, 1, 2
    }
}

// ------------------------------------------------------------ NPOL
// One lattice, pull: every node reads its nine incoming values (in-tile
// sources from the lattice, cross-tile sources from the buffer grid of the
// previous update), the block barrier separates all reads from the in-place
// writes, and edge nodes publish their outgoing values for the next update.

// Pulls of a node off the domain edge (32-bit offsets): every lane runs the
// interior pull (neighbour value, or the own opposite value of a bounced
// link) and, where the source lies across a tile edge, reads instead the
// source tile's publication of the previous update: its east/west edge when
// the tiles differ in x (the diagonal tile at a corner), else its north/south
// edge. Tile-edge nodes thus take no separate per-direction path, so a warp
// holding them does not run two.
template <class S, int L>
__device__ __forceinline__ void npol_pull(const Step<S> &a, int bx, int by, int lx, int ly, int x, int y,
                                          int x0, int x1, int y0, int y1, uint32_t n, uint32_t lk,
                                          typename Codec<S>::C *g) {
    const uint32_t nx = (uint32_t)a.geo.nx;
    const S *own = a.dst + lay_mul<L>() * n;
    const S *rs = own + (ptrdiff_t)lay_mul<L>() * nx;  // row y+1: source of c_y = -1
    const S *rn = own - (ptrdiff_t)lay_mul<L>() * nx;  // row y-1: source of c_y = +1
    const bool ex0 = x == x0, ex1 = x == x1, ey0 = y == y0, ey1 = y == y1;
    const int per = 6 * (a.tx + a.ty);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        if (i == 4) {
            g[i] = Codec<S>::dec(own[(ptrdiff_t)lay_base<L>(a.N, 4)]);
            continue;
        }
        const bool bounce = (lk >> link_bit(i)) & 1u;
        const S *row = cy(i) < 0 ? rs : (cy(i) > 0 ? rn : own);
        const S *p = bounce ? own + (ptrdiff_t)lay_base<L>(a.N, opp(i))
                            : row + ((ptrdiff_t)lay_base<L>(a.N, i) - (ptrdiff_t)lay_mul<L>() * cx(i));
        const bool crx = (cx(i) > 0 && ex0) || (cx(i) < 0 && ex1);
        const bool cry = (cy(i) > 0 && ey0) || (cy(i) < 0 && ey1);
        if (!bounce && (crx || cry)) {
            const int bxs = bx - (crx ? cx(i) : 0), bys = by - (cry ? cy(i) : 0);
            const S *t = a.halo_rd + (int64_t)(bys * a.ntx + bxs) * per;
            if (crx) {
                const int r = cry ? (cy(i) > 0 ? a.ty - 1 : 0) : ly - cy(i);
                p = t + (cx(i) > 0 ? 0 : 3 * a.ty) + (i / 3) * a.ty + r;
            } else {
                p = t + 6 * a.ty + (cy(i) > 0 ? 0 : 3 * a.tx) + (i % 3) * a.tx + (lx - cx(i));
            }
        }
        g[i] = Codec<S>::dec(*p);
    }
}

template <class S, int L>
__device__ __forceinline__ void npol_tile(const Step<S> &a, int bx, int by, int lx, int ly, int lane) {
    using C = typename Codec<S>::C;
    const int nx = a.geo.nx, ny = a.geo.ny;
    const int x0 = bx * a.tx, y0 = by * a.ty;
    const int x1 = min(x0 + a.tx, nx) - 1, y1 = min(y0 + a.ty, ny) - 1;
    const int x = x0 + lx, y = y0 + ly;
    const bool valid = lx < a.tx && ly < a.ty && x <= x1 && y <= y1;
    S *lat = a.dst;
    uint32_t n = 0, lk = SOLID_LINKS;
    if (valid) {
        n = (uint32_t)y * (uint32_t)nx + (uint32_t)x;
        lk = a.links[n];
    }
    const bool fluid = lk != SOLID_LINKS;
    const unsigned F = __ballot_sync(__activemask(), fluid);
    (void)F;
    const bool zero_fill = false;   // measured: NPOL is 5 % faster without the sector zero fill
    const bool inner = x > x0 && x < x1 && y > y0 && y < y1;
    const bool dom_inner = x > 0 && x < nx - 1 && y > 0 && y < ny - 1;
    C g[9];
    if (fluid && dom_inner && a.off32) {
        npol_pull<S, L>(a, bx, by, lx, ly, x, y, x0, x1, y0, y1, n, lk, g);
    } else if (fluid) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (i == 4) {
                g[i] = ldp<S, L>(lat, a.N, n, 4);
            } else if ((lk >> link_bit(i)) & 1u) {
                g[i] = ldp<S, L>(lat, a.N, n, opp(i));
            } else if (inner) {
                g[i] = ldp<S, L>(lat, a.N, n - (uint32_t)(cy(i) * nx + cx(i)), i);
            } else if (dom_inner) {
                // Tile edge inside the domain: the source is in this tile or in
                // the adjacent tile's buffer grid; the crossed edge follows from
                // c_i and the node's place on the tile edge.
                const int dbx = (cx(i) > 0 && x == x0) ? -1 : ((cx(i) < 0 && x == x1) ? 1 : 0);
                const int dby = (cy(i) > 0 && y == y0) ? -1 : ((cy(i) < 0 && y == y1) ? 1 : 0);
                if (dbx == 0 && dby == 0) {
                    g[i] = ldp<S, L>(lat, a.N, n - (uint32_t)(cy(i) * nx + cx(i)), i);
                } else {
                    const int64_t tb = (int64_t)((by + dby) * a.ntx + (bx + dbx)) * (6 * (a.tx + a.ty));
                    int off;
                    if (dbx != 0)  // east (c_x > 0) or west edge buffer, row of the source
                        off = (cx(i) > 0 ? 0 : 3 * a.ty) + (i / 3) * a.ty + (ly - cy(i) - dby * a.ty);
                    else           // north (c_y > 0) or south edge buffer, column of the source
                        off = 6 * a.ty + (cy(i) > 0 ? 0 : 3 * a.tx) + (i % 3) * a.tx + (lx - cx(i));
                    g[i] = Codec<S>::dec(a.halo_rd[tb + off]);
                }
            } else {
                int xs, ys, j;
                if (map_pull(a.geo, x, y, i, xs, ys, j) != PULL_NODE)
                    g[i] = C(0);
                else if (xs >= x0 && xs <= x1 && ys >= y0 && ys <= y1)
                    g[i] = ldp<S, L>(lat, a.N, (uint32_t)ys * (uint32_t)nx + (uint32_t)xs, j);
                else
                    g[i] = halo_read(a, xs, ys, j, bx);
            }
        }
    }
    const C dnb = (fluid && x == 0 && a.geo.bw == INLET_EQ_NEUMANN) ? neighbour_drho<S, L>(a, lat, n, 0) : C(0);
    __syncthreads();
    if (fluid) {
        S e[9];
        collide_encode(a, (uint32_t)x, n, g, e, dnb);
        store_node<S, L>(lat, n, a.N, a.off32, e);
        if (!inner) halo_publish(a.halo_wr, a.tx, a.ty, a.ntx, bx, by, x, y, x0, y0, x1, y1, e);
    } else if (zero_fill) {
        store_zero<S, L>(lat, a.N, n, a.off32);  // whole-sector writes, as in two_lattice_node
    }
}

template <class S, int L>
__global__ void __launch_bounds__(kMaxTileThreads, sizeof(S) == 8 ? 1 : 4) k_npol(const Step<S> a) {
    npol_tile<S, L>(a, blockIdx.x, blockIdx.y, threadIdx.x, threadIdx.y,
                    (int)((threadIdx.y * blockDim.x + threadIdx.x) & 31u));
}

// TMA: the tile's populations arrive by one tensor copy (FP32 storage, stream
// or bundle layout; tm is the kernel's tensor-map parameter) and keep the
// bundle interleave in shared memory; otherwise every fluid node stages its
// own nine values.
template <class S, int L, bool TMA = false>
__device__ __forceinline__ void nsol_tile(const Step<S> &a, int bx, int by, int lx, int ly, int lane,
                                          unsigned char *smem_raw, const TmaDesc *tm = nullptr) {
    using C = typename Codec<S>::C;
    const int T = a.tx * a.ty;
    C *sm = reinterpret_cast<C *>(smem_raw);
    // slot of direction s of tile node t among the staged values
    auto si = [T](int s, int t) { return (TMA && L == BUNDLE) ? (s / 3) * 3 * T + 3 * t + s % 3 : s * T + t; };
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + sizeof(C) * 9 * T);
    if constexpr (TMA) {
        if (lx == 0 && ly == 0)
            tma_issue_3d(tm, sm, bar, L == BUNDLE ? 3 * bx * a.tx : bx * a.tx, by * a.ty, 0,
                         (uint32_t)(sizeof(C) * 9 * T));
        __syncthreads();   // the barrier is initialised before anyone waits on it
    }
    const int nx = a.geo.nx, ny = a.geo.ny;
    const int x0 = bx * a.tx, y0 = by * a.ty;
    const int x1 = min(x0 + a.tx, nx) - 1, y1 = min(y0 + a.ty, ny) - 1;
    const bool member = lx < a.tx && ly < a.ty;  // thread has a slot in this tile
    const int tid = member ? ly * a.tx + lx : 0;
    const int x = x0 + lx, y = y0 + ly;
    const bool valid = member && x <= x1 && y <= y1;
    S *lat = a.dst;
    uint32_t n = 0, lk = SOLID_LINKS;
    if (valid) {
        n = (uint32_t)y * (uint32_t)nx + (uint32_t)x;
        lk = a.links[n];
    }
    const bool fluid = lk != SOLID_LINKS;
    const unsigned F = __ballot_sync(__activemask(), fluid);
    (void)F;
    const bool zero_fill = false;   // measured: NSOL is 2 % faster without the sector zero fill
    if (!TMA && fluid) {
#pragma unroll
        for (int s = 0; s < 9; ++s) sm[si(s, tid)] = ldp<S, L>(lat, a.N, n, s);
    }
    const C dnb = (fluid && x == 0 && a.geo.bw == INLET_EQ_NEUMANN) ? neighbour_drho<S, L>(a, lat, n, 1) : C(0);
    // Substitutions for pulls the in-tile exchange does not cover, read
    // before the first barrier: the lattice holds the previous state until
    // the stores after the last barrier, and other tiles' values come from
    // the buffer grid.
    C fix[9];
    unsigned fixmask = 0;
    const bool dom_inner = x > 0 && x < nx - 1 && y > 0 && y < ny - 1;
    if (fluid && dom_inner && !(x > x0 && x < x1 && y > y0 && y < y1)) {
        // Tile edge inside the domain: values from other tiles come from their
        // buffer grid (same slots as NPOL); in-tile sources are exchanged.
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            fix[i] = C(0);
            if (i == 4 || ((lk >> link_bit(i)) & 1u)) continue;
            const int dbx = (cx(i) > 0 && x == x0) ? -1 : ((cx(i) < 0 && x == x1) ? 1 : 0);
            const int dby = (cy(i) > 0 && y == y0) ? -1 : ((cy(i) < 0 && y == y1) ? 1 : 0);
            if (dbx == 0 && dby == 0) continue;
            const int64_t tb = (int64_t)((by + dby) * a.ntx + (bx + dbx)) * (6 * (a.tx + a.ty));
            const int off = dbx != 0
                ? (cx(i) > 0 ? 0 : 3 * a.ty) + (i / 3) * a.ty + (ly - cy(i) - dby * a.ty)
                : 6 * a.ty + (cy(i) > 0 ? 0 : 3 * a.tx) + (i % 3) * a.tx + (lx - cx(i));
            fixmask |= 1u << i;
            fix[i] = Codec<S>::dec(a.halo_rd[tb + off]);
        }
    } else if (fluid && !(x > x0 && x < x1 && y > y0 && y < y1)) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            fix[i] = C(0);
            if (i == 4 || ((lk >> link_bit(i)) & 1u)) continue;
            int xs, ys, j;
            const int kind = map_pull(a.geo, x, y, i, xs, ys, j);
            const bool in_tile = kind == PULL_NODE && xs >= x0 && xs <= x1 && ys >= y0 && ys <= y1;
            if (in_tile && j == i && xs == x - cx(i) && ys == y - cy(i)) continue;  // exchanged
            fixmask |= 1u << i;
            if (kind != PULL_NODE) continue;  // inlet unknown
            if (in_tile)
                fix[i] = ldp<S, L>(lat, a.N, (uint32_t)ys * (uint32_t)nx + (uint32_t)xs, opp(j));
            else
                fix[i] = halo_read(a, xs, ys, j, bx);
        }
    }
    if constexpr (TMA) {
        bool done = tma_wait(bar);
        if (!__syncthreads_and(done)) {
            // let a late copy land before the block's shared memory is released
            if (!done) done = tma_wait(bar);
            if (lx == 0 && ly == 0) atomicOr(a.err, 2u);
            return;
        }
    } else {
        __syncthreads();
    }
    if (fluid) {
        // partner x + c_i fluid <=> the pull of direction 8-i from it does not bounce
#pragma unroll
        for (int i = 5; i < 9; ++i) {
            const int px = lx + cx(i), py = ly + cy(i);
            if (px >= 0 && px < a.tx && py < a.ty && x0 + px <= x1 && y0 + py <= y1) {
                const int pt = py * a.tx + px;
                if (!((lk >> link_bit(opp(i))) & 1u)) {
                    C t = sm[si(opp(i), tid)];
                    sm[si(opp(i), tid)] = sm[si(i, pt)];
                    sm[si(i, pt)] = t;
                }
            }
        }
    }
    __syncthreads();
    if (fluid) {
        C g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = ((fixmask >> i) & 1u) ? fix[i] : sm[si(i, tid)];
        S e[9];
        collide_encode(a, (uint32_t)x, n, g, e, dnb);
#pragma unroll
        for (int i = 0; i < 9; ++i) lat[addr<L>(a.N, n, opp(i))] = e[i];
        if (!(x > x0 && x < x1 && y > y0 && y < y1))
            halo_publish(a.halo_wr, a.tx, a.ty, a.ntx, bx, by, x, y, x0, y0, x1, y1, e);
    } else if (zero_fill) {
        store_zero<S, L>(lat, a.N, n, a.off32);
    }
}

#ifndef LBM_NSOL_MINB
#define LBM_NSOL_MINB 4
#endif
template <class S, int L>
__global__ void __launch_bounds__(kMaxTileThreads, sizeof(S) == 8 ? 1 : LBM_NSOL_MINB) k_nsol(const Step<S> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    nsol_tile<S, L>(a, blockIdx.x, blockIdx.y, threadIdx.x, threadIdx.y,
                    (int)((threadIdx.y * blockDim.x + threadIdx.x) & 31u), smem_raw);
}

// NSOL with the tile staged by a tensor copy; shared memory: the tile's
// 9 T values, then the copy's mbarrier.
template <class S, int L>
__global__ void __launch_bounds__(kMaxTileThreads, LBM_NSOL_MINB)
    k_nsol_tma(const Step<S> a, const __grid_constant__ TmaDesc tm) {
    extern __shared__ __align__(128) unsigned char smem_tma[];
    nsol_tile<S, L, true>(a, blockIdx.x, blockIdx.y, threadIdx.x, threadIdx.y,
                          (int)((threadIdx.y * blockDim.x + threadIdx.x) & 31u), smem_tma, &tm);
}

// ------------------------------------------------------------ AA pattern
// In-place streaming with one lattice and no buffer grid (the AA pattern of
// Bailey et al., which Sec. 3.3 names as a state-of-the-art scheme). Updates
// alternate between two phases on the same array:
//  phase 0 (state: post-collision values in opposite slots, slot 8-i of x
//           holds S[x]_i): pull every value through the edge mapping,
//           collide, and store each result in the slot its puller reads next,
//           i.e. slot i of x + c_i (slot 8-i of x itself for a bounced link);
//  phase 1 (state: every node's pulled values in its own slots): read them,
//           collide, store the results in the node's opposite slots.
// Each slot is read and written by the same node within a phase, so no
// synchronisation is needed. Zero-gradient outflow reads one slot from two
// nodes and is not supported here.
template <class S, int L, int PHASE>
__device__ __forceinline__ void aa_node(const Step<S> &a, uint32_t x, uint32_t y, int lane) {
    constexpr int phase = PHASE;
    using C = typename Codec<S>::C;
    const uint32_t nx = (uint32_t)a.geo.nx, ny = (uint32_t)a.geo.ny;
    const uint32_t n = y * nx + x;
    const uint32_t lk = a.links[n];
    S *lat = a.dst;
    const bool fluid = lk != SOLID_LINKS;
    const unsigned F = __ballot_sync(__activemask(), fluid);
    if (!fluid) {
        if (shares_sector<S, L>(F, lane)) store_zero<S, L>(lat, a.N, n, a.off32);
        return;
    }
    C g[9];
    S e[9];
    if (phase == 1) {
        if (a.off32) {
            S *own = lat + lay_mul<L>() * n;
#pragma unroll
            for (int i = 0; i < 9; ++i) g[i] = Codec<S>::dec(own[(ptrdiff_t)lay_base<L>(a.N, i)]);
            collide_encode(a, x, n, g, e);
#pragma unroll
            for (int i = 0; i < 9; ++i) own[(ptrdiff_t)lay_base<L>(a.N, opp(i))] = e[i];
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) g[i] = ldp<S, L>(lat, a.N, n, i);
            collide_encode(a, x, n, g, e);
#pragma unroll
            for (int i = 0; i < 9; ++i) lat[addr<L>(a.N, n, opp(i))] = e[i];
        }
        return;
    }
    const bool interior = (x - 1u < nx - 2u) && (y - 1u < ny - 2u);
    if (interior && a.off32) {
        // 32-bit element indices with constant offsets: pull slot 8-i of
        // x - c_i (or own slot i when bounced), push to slot i of x + c_i (or
        // own slot 8-i). Each access is one select between two indices and one
        // widening address computation (measured 2 % faster than selecting
        // between 64-bit row pointers, at the same 40 registers).
        const uint32_t own = lay_mul<L>() * n;
        const uint32_t ra = own + lay_mul<L>() * nx;  // row y+1
        const uint32_t rb = own - lay_mul<L>() * nx;  // row y-1
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (i == 4) {
                g[i] = Codec<S>::dec(lat[own + lay_base<L>(a.N, 4)]);
                continue;
            }
            const uint32_t row = cy(i) < 0 ? ra : (cy(i) > 0 ? rb : own);
            const uint32_t ip = row + lay_base<L>(a.N, opp(i)) - (uint32_t)((int)lay_mul<L>() * cx(i));
            const uint32_t ib = own + lay_base<L>(a.N, i);
            g[i] = Codec<S>::dec(lat[((lk >> link_bit(i)) & 1u) ? ib : ip]);
        }
        collide_encode(a, x, n, g, e);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (i == 4) {
                lat[own + lay_base<L>(a.N, 4)] = e[4];
                continue;
            }
            const uint32_t row = cy(i) > 0 ? ra : (cy(i) < 0 ? rb : own);
            const uint32_t ip = row + lay_base<L>(a.N, i) + (uint32_t)((int)lay_mul<L>() * cx(i));
            const uint32_t ib = own + lay_base<L>(a.N, opp(i));
            lat[((lk >> link_bit(opp(i))) & 1u) ? ib : ip] = e[i];
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        if (i == 4) {
            g[i] = ldp<S, L>(lat, a.N, n, 4);
        } else if ((lk >> link_bit(i)) & 1u) {
            g[i] = ldp<S, L>(lat, a.N, n, i);  // slot i of x holds S[x]_{8-i}
        } else if (interior) {
            g[i] = ldp<S, L>(lat, a.N, n - (uint32_t)(cy(i) * (int)nx + cx(i)), opp(i));
        } else {
            int xs, ys, j;
            if (map_pull(a.geo, (int)x, (int)y, i, xs, ys, j) == PULL_NODE)
                g[i] = ldp<S, L>(lat, a.N, (uint32_t)ys * nx + (uint32_t)xs, opp(j));
            else
                g[i] = C(0);  // inlet unknown
        }
    }
    collide_encode(a, x, n, g, e);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        if (i == 4) {
            lat[addr<L>(a.N, n, 4)] = e[4];
        } else if ((lk >> link_bit(opp(i))) & 1u) {
            lat[addr<L>(a.N, n, opp(i))] = e[i];  // bounced back into this node
        } else if (interior) {
            lat[addr<L>(a.N, n + (uint32_t)(cy(i) * (int)nx + cx(i)), i)] = e[i];
        } else {
            // The neighbour x + c_i (wrapped across periodic edges) pulls
            // S[x]_i into slot i whenever it lies in the domain; otherwise the
            // puller is found through the edge mapping: every fluid node
            // within one cell whose mapped pull reads S[x]_i receives it.
            int tx_ = (int)x + cx(i), ty_ = (int)y + cy(i);
            bool in = true;
            if (tx_ < 0 || tx_ >= (int)nx) {
                if (a.geo.bw == PERIODIC) tx_ = tx_ < 0 ? tx_ + (int)nx : tx_ - (int)nx;
                else in = false;
            }
            if (ty_ < 0 || ty_ >= (int)ny) {
                if (a.geo.bs == PERIODIC) ty_ = ty_ < 0 ? ty_ + (int)ny : ty_ - (int)ny;
                else in = false;
            }
            if (in) {
                lat[addr<L>(a.N, (uint32_t)ty_ * nx + (uint32_t)tx_, i)] = e[i];
                continue;
            }
#pragma unroll 1
            for (int dy = -1; dy <= 1; ++dy)
#pragma unroll 1
                for (int dx = -1; dx <= 1; ++dx) {
                    int ux = (int)x + dx, uy = (int)y + dy;
                    if (ux < 0 || ux >= (int)nx) {
                        if (a.geo.bw != PERIODIC) continue;
                        ux = ux < 0 ? ux + (int)nx : ux - (int)nx;
                    }
                    if (uy < 0 || uy >= (int)ny) {
                        if (a.geo.bs != PERIODIC) continue;
                        uy = uy < 0 ? uy + (int)ny : uy - (int)ny;
                    }
                    const uint32_t m = (uint32_t)uy * nx + (uint32_t)ux;
                    const uint32_t ml = a.links[m];
                    if (ml == SOLID_LINKS) continue;
#pragma unroll 1
                    for (int k = 0; k < 9; ++k) {
                        if (k == 4 || ((ml >> link_bit(k)) & 1u)) continue;
                        int xs, ys, j;
                        if (map_pull(a.geo, ux, uy, k, xs, ys, j) == PULL_NODE && xs == (int)x &&
                            ys == (int)y && j == i)
                            lat[addr<L>(a.N, m, k)] = e[i];
                    }
                }
        }
    }
}

template <class S, int L, int PHASE>
__global__ void __launch_bounds__(kMaxTileThreads, sizeof(S) == 8 ? 1 : (PHASE == 0 || L == STREAM ? 3 : 4)) k_aa(const Step<S> a) {
    const uint32_t x = blockIdx.x * a.tx + threadIdx.x;
    const uint32_t y = blockIdx.y * a.ty + threadIdx.y;
    if (x >= (uint32_t)a.geo.nx || y >= (uint32_t)a.geo.ny) return;
    // L2 prefetch of the record a.pf rows ahead, as in the two-lattice kernel
    constexpr bool PF = sizeof(S) == 4 && L != COLLISION;
    const bool ahead = PF && a.pf != 0u && (uint32_t)a.geo.ny - y > a.pf;
    const uint32_t np = (y + a.pf) * (uint32_t)a.geo.nx + x;
    const uint32_t lkp = ahead ? (uint32_t)a.links[np] : SOLID_LINKS;
    aa_node<S, L, PHASE>(a, x, y, (int)((threadIdx.y * blockDim.x + threadIdx.x) & 31u));
    if (PF && lkp != SOLID_LINKS) prefetch_record<S, L>(a.dst, a.N, np);
}

// ------------------------------------------------------------ batches
// Many independent lattices advanced by one persistent launch per update.
// The work list holds one entry per work item of every case: four tiles of
// a two-lattice case (LPTL tile = 256 consecutive nodes), one tile of a
// one-lattice case. Blocks take entries round-robin; a block stages a case
// record in shared memory only when the case changes.
constexpr int kBatchThreads = 256;
constexpr int kBatchSuper = 4;  // tiles per work item of a two-lattice case

template <class S>
struct BatchCase {
    Step<S> st;                 // constants, links, tile shape of the case
    S *pop0, *pop1, *halo;      // pop1 == nullptr for one-lattice cases
    typename Codec<S>::C *mom;
    long long halo_parity_elems;
    unsigned long long ntx_magic;  // ceil(2^64 / ntx), 0 when ntx == 1
    int layout, algo;
};

struct BatchTile {
    uint32_t c;                 // case index
    uint32_t t;                 // work item within the case
};

template <class S, int L>
__device__ __forceinline__ void batch_item(const BatchCase<S> &bc, int algo, uint32_t t, int tid,
                                           unsigned char *smem) {
    const Step<S> &a = bc.st;
    const int lane = tid & 31;
    if (algo == LPTL) {
#pragma unroll 1
        for (int k = 0; k < kBatchSuper; ++k) {
            const uint32_t n = (t * kBatchSuper + k) * (uint32_t)kBatchThreads + (uint32_t)tid;
            if (n < a.N) {
                const uint32_t y = a.nx_magic ? (uint32_t)__umul64hi((unsigned long long)n, a.nx_magic) : n;
                two_lattice_node<S, L>(a, n - y * (uint32_t)a.geo.nx, y, lane);
            }
        }
        return;
    }
    const int lx = tid % a.tx, ly = tid / a.tx;
    if (algo == NPTL) {
        const uint32_t ntiles = (uint32_t)a.ntx * (uint32_t)((a.geo.ny + a.ty - 1) / a.ty);
#pragma unroll 1
        for (int k = 0; k < kBatchSuper; ++k) {
            const uint32_t tt = t * kBatchSuper + k;
            if (tt >= ntiles) break;
            const uint32_t by = bc.ntx_magic ? (uint32_t)__umul64hi((unsigned long long)tt, bc.ntx_magic) : tt;
            const uint32_t bx = tt - by * (uint32_t)a.ntx;
            const int x = (int)bx * a.tx + lx, y = (int)by * a.ty + ly;
            if (ly < a.ty && x < a.geo.nx && y < a.geo.ny) two_lattice_node<S, L>(a, x, y, lane);
        }
        return;
    }
    const int by = (int)(t / (uint32_t)a.ntx), bx = (int)(t - (uint32_t)by * (uint32_t)a.ntx);
    if (algo == NPOL)
        npol_tile<S, L>(a, bx, by, lx, ly, lane);
    else
        nsol_tile<S, L>(a, bx, by, lx, ly, lane, smem);
}

// LK / AK: the layout / algorithm shared by every case, or -1 (any).
// cur: source lattice of two-lattice cases, which equals the buffer-grid
// parity read by one-lattice cases (all cases start together at update 0).
template <class S, int LK, int AK>
__global__ void __launch_bounds__(kBatchThreads, LK < 0 ? 2 : (AK <= NPTL ? (sizeof(S) == 8 ? 4 : 6) : 3))
    k_batch(const BatchCase<S> *cases, const BatchTile *tiles, uint32_t ntiles, int cur, int toff,
            int want_moments) {
    using C = typename Codec<S>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(16) BatchCase<S> bc;
    const int tid = threadIdx.x;
    uint32_t have = 0xffffffffu;  // case staged in bc (same in every thread)
    for (uint32_t w = blockIdx.x; w < ntiles; w += gridDim.x) {
        const BatchTile bt = tiles[w];
        if (bt.c != have) {
            __syncthreads();  // every thread is done with the previous record
            const uint32_t *srcw = reinterpret_cast<const uint32_t *>(cases + bt.c);
            uint32_t *dstw = reinterpret_cast<uint32_t *>(&bc);
            for (int k = tid; k < (int)(sizeof(BatchCase<S>) / 4); k += kBatchThreads) dstw[k] = srcw[k];
            __syncthreads();
            if (tid == 0) {
                if (bc.pop1) {
                    bc.st.src = cur ? bc.pop1 : bc.pop0;
                    bc.st.dst = cur ? bc.pop0 : bc.pop1;
                } else {
                    bc.st.src = bc.pop0;
                    bc.st.dst = bc.pop0;
                    bc.st.halo_rd = bc.halo + (long long)cur * bc.halo_parity_elems;
                    bc.st.halo_wr = bc.halo + (long long)(cur ^ 1) * bc.halo_parity_elems;
                }
                bc.st.mom = want_moments ? (C *)bc.mom : nullptr;
                bc.st.toff = toff;
            }
            __syncthreads();
            have = bt.c;
        }
        const int algo = AK >= 0 ? AK : bc.algo;
        const int layout = LK >= 0 ? LK : bc.layout;
        switch (layout) {
            case STREAM: batch_item<S, STREAM>(bc, algo, bt.t, tid, smem); break;
            case BUNDLE: batch_item<S, BUNDLE>(bc, algo, bt.t, tid, smem); break;
            default: batch_item<S, COLLISION>(bc, algo, bt.t, tid, smem); break;
        }
        if (algo == NSOL) __syncthreads();  // shared-memory tile reused by the next item
    }
}

template <class S>
size_t batch_smem_bytes() {
    return sizeof(typename Codec<S>::C) * 9 * kBatchThreads + kBatchThreads;
}

// kind = layout * 4 + algo when every case shares them, else -1.
#define LBM_BATCH_KINDS(X, S)                                                              \
    X(S, -1, -1) X(S, 0, 0) X(S, 0, 1) X(S, 0, 2) X(S, 0, 3) X(S, 1, 0) X(S, 1, 1) X(S, 1, 2) \
        X(S, 1, 3) X(S, 2, 0) X(S, 2, 1) X(S, 2, 2) X(S, 2, 3)

template <class S>
cudaError_t op_batch_step(int kind, const void *cases, const void *tiles, uint32_t ntiles, int grid, int cur,
                          int toff, int want_moments, cudaStream_t st) {
    const size_t sm = batch_smem_bytes<S>();
    const auto *c = (const BatchCase<S> *)cases;
    const auto *t = (const BatchTile *)tiles;
#define LBM_BATCH_LAUNCH(S_, L_, A_)                                                       \
    if (kind == ((L_) < 0 ? -1 : (L_) * 4 + (A_))) {                                      \
        k_batch<S_, L_, A_><<<grid, kBatchThreads, sm, st>>>(c, t, ntiles, cur, toff, want_moments); \
        return cudaGetLastError();                                                          \
    }
    LBM_BATCH_KINDS(LBM_BATCH_LAUNCH, S)
#undef LBM_BATCH_LAUNCH
    return cudaErrorInvalidValue;
}

template <class S, int LK, int AK>
int batch_grid_of() {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<S, LK, AK>, kBatchThreads,
                                                      batch_smem_bytes<S>()) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return sms * (per_sm > 0 ? per_sm : 1);
}

template <class S>
int op_batch_grid(int kind) {
#define LBM_BATCH_GRID(S_, L_, A_) \
    if (kind == ((L_) < 0 ? -1 : (L_) * 4 + (A_))) return batch_grid_of<S_, L_, A_>();
    LBM_BATCH_KINDS(LBM_BATCH_GRID, S)
#undef LBM_BATCH_GRID
    return 0;
}

// Host: the device record of one case (pointers from its HostArgs).
template <class S>
void op_batch_case(const HostArgs &h, void *out) {
    BatchCase<S> c;
    memset(&c, 0, sizeof(c));
    c.st = make_step<S>(h, StepCall{0, 0, 0, 0});
    c.pop0 = (S *)h.pop[0];
    c.pop1 = (S *)h.pop[1];
    c.halo = (S *)h.halo;
    c.mom = (typename Codec<S>::C *)h.mom;
    c.halo_parity_elems = h.halo_parity_elems;
    c.ntx_magic = h.ntx > 1 ? (~0ull / (unsigned long long)h.ntx) + 1ull : 0ull;
    c.layout = h.layout;
    c.algo = h.algo;
    memcpy(out, &c, sizeof(c));
}

// ------------------------------------------------------------ state kernels
template <class S, int L>
__global__ void k_init(const Step<S> a, const double *rho, const double *ux, const double *uy,
                       uint32_t n0, uint32_t count, int rev) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const uint32_t n = n0 + t;
    if (a.links[n] == SOLID_LINKS) return;
    const double dr = rho ? rho[t] - 1.0 : 0.0;
    const double vx = ux ? ux[t] : 0.0, vy = uy ? uy[t] : 0.0;
    const double usq = vx * vx + vy * vy;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const double w = i == 4 ? 4.0 / 9.0 : ((i & 1) ? 1.0 / 9.0 : 1.0 / 36.0);
        const double cu = cx(i) * vx + cy(i) * vy;
        const double h = w * (dr + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
        typename Codec<S>::C hc = (typename Codec<S>::C)h;
        a.dst[addr<L>(a.N, n, rev ? opp(i) : i)] = Codec<S>::enc(hc, false, 0u);
    }
}

// Solid nodes hold h = 0 (restored after host writes of the state).
template <class S, int L>
__global__ void k_zero_solid(const Step<S> a, S *lat) {
    const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= a.N || a.links[n] != SOLID_LINKS) return;
    store_zero<S, L>(lat, a.N, n, a.off32);
}

// Copy every tile-edge node's outgoing values into one buffer-grid parity.
template <class S, int L>
__global__ void k_publish(const Step<S> a, S *hw, int rev) {
    const int nx = a.geo.nx, ny = a.geo.ny;
    const int bx = blockIdx.x, by = blockIdx.y;
    const int x0 = bx * a.tx, y0 = by * a.ty;
    const int x1 = min(x0 + a.tx, nx) - 1, y1 = min(y0 + a.ty, ny) - 1;
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x > x1 || y > y1) return;
    if (x > x0 && x < x1 && y > y0 && y < y1) return;
    const uint32_t n = (uint32_t)y * (uint32_t)nx + (uint32_t)x;
    if (a.links[n] == SOLID_LINKS) return;
    S e[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) e[i] = a.src[addr<L>(a.N, n, rev ? opp(i) : i)];
    halo_publish(hw, a.tx, a.ty, a.ntx, bx, by, x, y, x0, y0, x1, y1, e);
}

// Moments from a stored state: rho = 1 + sum h, v = sum h c (- F/2 for a
// post-collision state, since the collision adds F to sum f c), in the
// arithmetic type (used for the moments reported after lbm_init).
template <class S, int L>
__global__ void k_state_moments(const Step<S> a, int rev, int post) {
    using C = typename Codec<S>::C;
    using A = Ar<C>;
    const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= a.N) return;
    C *m = (C *)a.mom;
    if (a.links[n] == SOLID_LINKS) {
        m[n] = C(1);
        m[a.N + n] = C(0);
        m[2 * a.N + n] = C(0);
        return;
    }
    C h[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) h[i] = ldp<S, L>(a.src, a.N, n, rev ? opp(i) : i);
    C r = C(0), jx = C(0), jy = C(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        r = A::add(r, h[i]);
        if (cx(i) != 0) jx = cx(i) > 0 ? A::add(jx, h[i]) : A::sub(jx, h[i]);
        if (cy(i) != 0) jy = cy(i) > 0 ? A::add(jy, h[i]) : A::sub(jy, h[i]);
    }
    if (post) {
        jx = A::sub(jx, a.k.hfx);
        jy = A::sub(jy, a.k.hfy);
    }
    m[n] = A::add(C(1), r);
    m[a.N + n] = jx;
    m[2 * a.N + n] = jy;
}

// Deterministic FP64 block reduction (fixed grid and tree).
template <int W>
__device__ __forceinline__ void block_reduce_store(double (&v)[W], double *partials) {
    __shared__ double red[W][kReduceThreads];
    for (int w = 0; w < W; ++w) red[w][threadIdx.x] = v[w];
    __syncthreads();
    for (int s = kReduceThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int w = 0; w < W; ++w) red[w][threadIdx.x] += red[w][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int w = 0; w < W; ++w) partials[blockIdx.x * W + w] = red[w][0];
}

template <class S, int L>
__global__ void __launch_bounds__(kReduceThreads) k_mass(const Step<S> a, int rev, double *partials) {
    double acc[1] = {0.0};
    for (uint64_t n64 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; n64 < a.N;
         n64 += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t n = (uint32_t)n64;
        if (a.links[n] == SOLID_LINKS) continue;
        double r = 1.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) r += (double)ldp<S, L>(a.src, a.N, n, rev ? opp(i) : i);
        acc[0] += r;
    }
    block_reduce_store<1>(acc, partials);
}

template <class S, int L>
__global__ void __launch_bounds__(kReduceThreads) k_force(const Step<S> a, int rev, const uint8_t *body,
                                                          double *partials) {
    double acc[2] = {0.0, 0.0};
    const int nx = a.geo.nx, ny = a.geo.ny;
    for (uint64_t n64 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; n64 < a.N;
         n64 += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t n = (uint32_t)n64;
        if (a.links[n] == SOLID_LINKS) continue;
        const int y = a.nx_magic ? (int)__umul64hi((unsigned long long)n, a.nx_magic) : (int)n;
        const int x = (int)n - y * nx;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (i == 4) continue;
            int bx = x + cx(i), by = y + cy(i);
            if (bx < 0 || bx >= nx) {
                if (a.geo.bw != PERIODIC) continue;
                bx = bx < 0 ? bx + nx : bx - nx;
            }
            if (by < 0 || by >= ny) {
                if (a.geo.bs != PERIODIC) continue;
                by = by < 0 ? by + ny : by - ny;
            }
            const uint32_t m = (uint32_t)by * (uint32_t)nx + (uint32_t)bx;
            const bool hit = body ? body[m] != 0 : a.links[m] == SOLID_LINKS;
            if (!hit) continue;
            const double w = (i & 1) ? 1.0 / 9.0 : 1.0 / 36.0;
            const double f = w + (double)ldp<S, L>(a.src, a.N, n, rev ? opp(i) : i);
            acc[0] += 2.0 * cx(i) * f;
            acc[1] += 2.0 * cy(i) * f;
        }
    }
    block_reduce_store<2>(acc, partials);
}

template <class C>
__global__ void k_moments_f32(const C *mom, uint32_t N, float *r, float *u, float *v) {
    const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    r[n] = (float)mom[n];
    u[n] = (float)mom[N + n];
    v[n] = (float)mom[2 * (size_t)N + n];
}

// ------------------------------------------------------------ launchers
template <class S, int L>
int lptl_block() {
    static int block = [] {
        int minGrid = 0, b = 256;
        if (cudaOccupancyMaxPotentialBlockSize(&minGrid, &b, k_two_lattice<S, L, true>, 0,
                                               kMaxTileThreads) != cudaSuccess) {
            cudaGetLastError();
            b = 256;
        }
        return b;
    }();
    return block;
}

// Node pairs: 16-bit storage in the bundle layout, nx even, 32-bit offsets,
// unless LBM_FLAG_NO_PAIRS asks for one node per thread. (The stream layout
// measured 7 % slower with pairs than with one node per thread: nine
// separate arrays give each pair nine 32-bit stores and nine prefetches.)
template <class S, int L>
bool pairs_ok(const HostArgs &h) {
    return sizeof(S) == 2 && L == BUNDLE && (h.nx % 2) == 0 && (9 * h.N) < (int64_t(1) << 32) &&
           !(h.flags & 0x20u);
}

template <class S, int L>
cudaError_t step_layout(const HostArgs &h, const Step<S> &a, int phase, cudaStream_t st) {
    using C = typename Codec<S>::C;
    const dim3 tile(h.tile_x, h.tile_y), grid(h.ntx, h.nty);
    switch (h.algo) {
        case LPTL: {
            if constexpr (sizeof(S) == 2 && L == BUNDLE) {
                if (pairs_ok<S, L>(h)) {
                    const int b = 128;
                    const unsigned g = (unsigned)((h.N / 2 + b - 1) / b);
                    k_two_lattice_pair<S, L, true><<<g, b, 0, st>>>(a);
                    break;
                }
            }
            const int b = h.block_1d;
            const unsigned g = (unsigned)((h.N + b - 1) / b);
            k_two_lattice<S, L, true><<<g, b, 0, st>>>(a);
            break;
        }
        case NPTL:
            if (L == COLLISION && h.tile_x % 32 == 0 && !(h.flags & 4u)) {
                const size_t sm = (size_t)AosSpan<S>::WARP_BYTES * ((h.tile_x * h.tile_y + 31) / 32);
                k_two_lattice_aos<S><<<grid, tile, sm, st>>>(a);
                break;
            }
            if constexpr (sizeof(S) == 2 && L == BUNDLE) {
                if (pairs_ok<S, L>(h) && !(h.tile_x & 1)) {
                    k_two_lattice_pair<S, L, false><<<grid, dim3(h.tile_x / 2, h.tile_y), 0, st>>>(a);
                    break;
                }
            }
            // Two nodes per thread on request (4- and 8-byte storage): one node
            // per thread at 32 registers keeps full occupancy and measured faster.
            if (sizeof(S) >= 4 && h.tile_y >= 2 && !(h.tile_y & 1) && (h.flags & 2u))
                k_two_lattice2<S, L><<<grid, dim3(h.tile_x, h.tile_y / 2), 0, st>>>(a);
            else
                k_two_lattice<S, L, false><<<grid, tile, 0, st>>>(a);
            break;
        case NPOL: k_npol<S, L><<<grid, tile, 0, st>>>(a); break;
        case NSOL: {
            const size_t sm = sizeof(C) * 9 * h.tile_x * h.tile_y;
            if constexpr (std::is_same<S, float>::value && L != COLLISION) {
                if (h.tma) {
                    k_nsol_tma<S, L><<<grid, tile, sm + 16, st>>>(a, h.tmap);
                    break;
                }
            }
            k_nsol<S, L><<<grid, tile, sm, st>>>(a);
            break;
        }
        case AA:
            if (phase)
                k_aa<S, L, 1><<<grid, tile, 0, st>>>(a);
            else
                k_aa<S, L, 0><<<grid, tile, 0, st>>>(a);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <class S>
cudaError_t op_step(const HostArgs &h, const StepCall &c, cudaStream_t st) {
    const Step<S> a = make_step<S>(h, c);
    switch (h.layout) {
        case STREAM: return step_layout<S, STREAM>(h, a, c.rd_parity, st);
        case BUNDLE: return step_layout<S, BUNDLE>(h, a, c.rd_parity, st);
        case COLLISION: return step_layout<S, COLLISION>(h, a, c.rd_parity, st);
    }
    return cudaErrorInvalidValue;
}

#define LBM_LAYOUT_SWITCH(h, CALL)                          \
    switch ((h).layout) {                                   \
        case STREAM: { constexpr int L_ = STREAM; CALL; break; }       \
        case BUNDLE: { constexpr int L_ = BUNDLE; CALL; break; }       \
        case COLLISION: { constexpr int L_ = COLLISION; CALL; break; } \
        default: return cudaErrorInvalidValue;              \
    }

template <class S>
cudaError_t op_init(const HostArgs &h, const double *rho, const double *ux, const double *uy,
                    int64_t n0, int64_t count, cudaStream_t st) {
    const Step<S> a = make_step<S>(h, StepCall{1, 0, 0, 0});  // dst = pop[0]
    if (count <= 0) return cudaSuccess;
    const unsigned g = (unsigned)((count + 255) / 256);
    const int rev = h.algo == NSOL || h.algo == AA;
    LBM_LAYOUT_SWITCH(h, (k_init<S, L_><<<g, 256, 0, st>>>(a, rho, ux, uy, (uint32_t)n0,
                                                             (uint32_t)count, rev)));
    return cudaGetLastError();
}

template <class S>
cudaError_t op_publish(const HostArgs &h, int src, int parity, cudaStream_t st) {
    const Step<S> a = make_step<S>(h, StepCall{src, 0, 0, 0});
    S *hw = (S *)h.halo + (int64_t)parity * h.halo_parity_elems;
    const int rev = h.algo == NSOL || h.algo == AA;
    const dim3 tile(h.tile_x, h.tile_y), grid(h.ntx, h.nty);
    LBM_LAYOUT_SWITCH(h, (k_publish<S, L_><<<grid, tile, 0, st>>>(a, hw, rev)));
    return cudaGetLastError();
}

template <class S>
cudaError_t op_zero_solid(const HostArgs &h, int src, cudaStream_t st) {
    const Step<S> a = make_step<S>(h, StepCall{src, 0, 0, 0});
    const unsigned g = (unsigned)((h.N + 255) / 256);
    S *lat = (S *)h.pop[src];
    LBM_LAYOUT_SWITCH(h, (k_zero_solid<S, L_><<<g, 256, 0, st>>>(a, lat)));
    return cudaGetLastError();
}

template <class S>
cudaError_t op_state_moments(const HostArgs &h, int src, int post, cudaStream_t st) {
    Step<S> a = make_step<S>(h, StepCall{src, 0, 0, 1});
    const unsigned g = (unsigned)((h.N + 255) / 256);
    const int rev = h.algo == NSOL || h.algo == AA;
    LBM_LAYOUT_SWITCH(h, (k_state_moments<S, L_><<<g, 256, 0, st>>>(a, rev, post)));
    return cudaGetLastError();
}

template <class S>
cudaError_t op_mass(const HostArgs &h, int src, double *partials, int nblocks, cudaStream_t st) {
    const Step<S> a = make_step<S>(h, StepCall{src, 0, 0, 0});
    const int rev = h.algo == NSOL || h.algo == AA;
    LBM_LAYOUT_SWITCH(h, (k_mass<S, L_><<<nblocks, kReduceThreads, 0, st>>>(a, rev, partials)));
    return cudaGetLastError();
}

template <class S>
cudaError_t op_force(const HostArgs &h, int src, const uint8_t *body, double *partials, int nblocks,
                     cudaStream_t st) {
    const Step<S> a = make_step<S>(h, StepCall{src, 0, 0, 0});
    const int rev = h.algo == NSOL || h.algo == AA;
    LBM_LAYOUT_SWITCH(h, (k_force<S, L_><<<nblocks, kReduceThreads, 0, st>>>(a, rev, body, partials)));
    return cudaGetLastError();
}

template <class S>
cudaError_t op_moments_f32(const HostArgs &h, float *r, float *u, float *v, cudaStream_t st) {
    using C = typename Codec<S>::C;
    const unsigned g = (unsigned)((h.N + 255) / 256);
    k_moments_f32<C><<<g, 256, 0, st>>>((const C *)h.mom, (uint32_t)h.N, r, u, v);
    return cudaGetLastError();
}

template <class S>
int op_lptl_block(int layout) {
    switch (layout) {
        case STREAM: return lptl_block<S, STREAM>();
        case BUNDLE: return lptl_block<S, BUNDLE>();
        default: return lptl_block<S, COLLISION>();
    }
}

// Allow the staged collision-layout kernel more than the default 48 KB of
// dynamic shared memory (FP64: 7.4 KB per warp). Called at lattice creation.
template <class S>
void op_prepare() {
    static const bool done = [] {
        cudaFuncSetAttribute(k_two_lattice_aos<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             AosSpan<S>::WARP_BYTES * (kMaxTileThreads / 32));
        cudaGetLastError();
        return true;
    }();
    (void)done;
}

template <class S>
Ops make_ops() {
    Ops o;
    o.step = op_step<S>;
    o.init = op_init<S>;
    o.publish = op_publish<S>;
    o.zero_solid = op_zero_solid<S>;
    o.state_moments = op_state_moments<S>;
    o.mass = op_mass<S>;
    o.force = op_force<S>;
    o.moments_f32 = op_moments_f32<S>;
    o.lptl_block = op_lptl_block<S>;
    o.prepare = op_prepare<S>;
    o.batch_step = op_batch_step<S>;
    o.batch_grid = op_batch_grid<S>;
    o.batch_case = op_batch_case<S>;
    o.batch_case_bytes = sizeof(BatchCase<S>);
    o.elem = sizeof(S);
    o.compute = sizeof(typename Codec<S>::C);
    return o;
}

}  // namespace lbm
