// D3Q19 lattices (the paper's 3-D future work, Sec. 6) with the method of
// Sec. 3.1: two-lattice pull (LPTL: one node per thread over n; NPTL: 3-D
// tiles), the one-lattice NPOL pull and NSOL swap of Sec. 3.3 (tiles and a
// buffer grid), and the one-lattice AA pattern (Sec. 3.3 names it, Sec. 6
// lists it as future work), the three layouts generalised (stream, bundle =
// directions sharing a source row, collision), periodic or half-way wall
// faces, equilibrium or Zou-He inlet, zero-gradient outflow or Zou-He
// pressure outlet on x, bounce-back at solid nodes, Guo force,
// FP64/FP32/FP16/BF16 shifted storage, on-the-fly moments, FP64 mass and
// momentum-exchange force, CUDA graphs. C ABI: the lbm3_* calls of
// include/lbm.h.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "lbm.h"
#include "lbm3_device.cuh"
#include "lbm_capi_internal.h"
#include "lbm_internal.h"

namespace lbm {
namespace d3 {

struct Geo3 {
    int nx, ny, nz;
    int bx, by, bz;   // y, z: PERIODIC or WALL; x: the west face (also INLET_EQ, INLET_ZOUHE, OUTFLOW_ZG)
    int bxe;          // the east face (PERIODIC with bx, WALL, OUTFLOW_ZG or OUTLET_PRESSURE)
};

// Source node of the value pulled by (x, y, z) in direction i, or bounce
// (walls; the inlet face, whose plane is overwritten before the collision).
// Mapped in z, then y, then x; the outflow clamps the source plane.
__host__ __device__ __forceinline__ bool map3(const Geo3 &g, int x, int y, int z, int i, uint32_t &src) {
    int s[3] = {x - cx(i), y - cy(i), z - cz(i)};
    const int ext[3] = {g.nx, g.ny, g.nz};
    const int bc[3] = {g.bx, g.by, g.bz};
#pragma unroll
    for (int a = 2; a >= 1; --a) {
        if (s[a] < 0 || s[a] >= ext[a]) {
            if (bc[a] != PERIODIC) return false;
            s[a] = s[a] < 0 ? s[a] + ext[a] : s[a] - ext[a];
        }
    }
    if (s[0] < 0 || s[0] >= g.nx) {
        const int kind = s[0] < 0 ? g.bx : g.bxe;
        if (kind == PERIODIC) s[0] = s[0] < 0 ? s[0] + g.nx : s[0] - g.nx;
        else if (kind == OUTFLOW_ZG) s[0] = s[0] < 0 ? 0 : g.nx - 1;
        else return false;
    }
    src = ((uint32_t)s[2] * (uint32_t)g.ny + (uint32_t)s[1]) * (uint32_t)g.nx + (uint32_t)s[0];
    return true;
}

template <class S>
struct Step3 {
    using C = typename Codec<S>::C;
    Geo3 g;
    uint32_t N;
    Consts3<C> k;
    const uint32_t *links;
    const S *src;
    S *dst;
    C *mom;
    unsigned int *err;
    const long long *tctr;
    int toff;
    int sr;
    uint64_t seed;
    int tx, ty, tz;
    uint64_t nx_magic, nxy_magic;   // ceil(2^64 / nx), ceil(2^64 / (nx ny)); 0 for 1
    int zero_fill;                  // lanes of a warp hold consecutive nodes
    // 32-bit element offsets from the base of direction i at node n (base =
    // lattice + mult3(i) n): own slot i (os), slot i of node n - c_i before
    // any periodic correction (op), own slot opp(i) for a bounced pull (ob).
    int32_t os[Q], op[Q], ob[Q];
    int32_t oq[Q];   // AA push: slot opp(i) of node n + c_i, from the base of direction i
    // node-index corrections of a pull across the west (x = 0) / east face:
    // +nx / -nx periodic, +1 / -1 zero-gradient outflow (clamped source)
    int xlo_corr, xhi_corr;
    int inlet;       // x = 0 plane: 1 takes heq_in (equilibrium inlet), 2 Zou-He velocity inlet
    int outlet;      // x = nx - 1 plane: Zou-He pressure outlet
    int rev;         // NSOL: population i of a node is stored in its slot opp(i)
    C heq_in[Q];
    // Zou-He: U_x/3, (U_x + U_y)/6, (U_x - U_y)/6, (U_x + U_z)/6, (U_x - U_z)/6,
    // -U_y/3, -U_z/3, rho_out - 1
    C zh[8];
};

// Storage slot of population i in the stored state.
template <class S>
__host__ __device__ __forceinline__ int slot3(const Step3<S> &a, int i) {
    return a.rev ? opp(i) : i;
}

// Zou-He velocity inlet on the west face: the five populations with
// c_x = +1 (unknown, pulled from outside) follow from sum_i g_i c_i = U and
// bounce-back of the normal non-equilibrium part, with the transverse
// momenta T_y, T_z of the nine c_x = 0 populations:
//   g10 = g8 + U_x/3,  g13 = g5 + (U_x + U_y)/6 - N_y,  g7 = g11 + (U_x - U_y)/6 + N_y,
//   g17 = g1 + (U_x + U_z)/6 - N_z,  g3 = g15 + (U_x - U_z)/6 + N_z,
//   N_y = T_y/2 - U_y/3,  N_z = T_z/2 - U_z/3.
template <class S>
__device__ __forceinline__ void zou_he3(const Step3<S> &a, typename Codec<S>::C *g) {
    using C = typename Codec<S>::C;
    using A = Ar<C>;
    const C ty = A::sub(A::add(A::add(g[4], g[12]), g[18]), A::add(A::add(g[0], g[6]), g[14]));
    const C tz = A::sub(A::add(A::add(g[14], g[16]), g[18]), A::add(A::add(g[0], g[2]), g[4]));
    const C ny = A::fma(C(0.5), ty, a.zh[5]);
    const C nz = A::fma(C(0.5), tz, a.zh[6]);
    g[10] = A::add(g[8], a.zh[0]);
    g[13] = A::sub(A::add(g[5], a.zh[1]), ny);
    g[7] = A::add(A::add(g[11], a.zh[2]), ny);
    g[17] = A::sub(A::add(g[1], a.zh[3]), nz);
    g[3] = A::add(A::add(g[15], a.zh[4]), nz);
}

// Zou-He pressure outlet on the east face: rho = rho_out and v_y = v_z = 0
// fix the five c_x = -1 populations; u_x = 2 H+ + H0 - (rho_out - 1) from
// the known c_x = +1 (H+) and c_x = 0 (H0) deviations, then
//   g8 = g10 - u_x/3,  g11 = g7 - u_x/6 - T_y/2,  g5 = g13 - u_x/6 + T_y/2,
//   g15 = g3 - u_x/6 - T_z/2,  g1 = g17 - u_x/6 + T_z/2.
template <class S>
__device__ __forceinline__ void zou_he_pressure3(const Step3<S> &a, typename Codec<S>::C *g) {
    using C = typename Codec<S>::C;
    using A = Ar<C>;
    const C hp = A::add(A::add(A::add(A::add(g[3], g[7]), g[10]), g[13]), g[17]);
    C h0 = g[0];
    h0 = A::add(h0, g[2]);
    h0 = A::add(h0, g[4]);
    h0 = A::add(h0, g[6]);
    h0 = A::add(h0, g[9]);
    h0 = A::add(h0, g[12]);
    h0 = A::add(h0, g[14]);
    h0 = A::add(h0, g[16]);
    h0 = A::add(h0, g[18]);
    const C ux = A::sub(A::fma(C(2), hp, h0), a.zh[7]);
    const C ty = A::sub(A::add(A::add(g[4], g[12]), g[18]), A::add(A::add(g[0], g[6]), g[14]));
    const C tz = A::sub(A::add(A::add(g[14], g[16]), g[18]), A::add(A::add(g[0], g[2]), g[4]));
    const C u6 = A::mul(ux, C(1.0 / 6.0));
    g[8] = A::fma(C(-1.0 / 3.0), ux, g[10]);
    g[11] = A::fma(C(-0.5), ty, A::sub(g[7], u6));
    g[5] = A::fma(C(0.5), ty, A::sub(g[13], u6));
    g[15] = A::fma(C(-0.5), tz, A::sub(g[3], u6));
    g[1] = A::fma(C(0.5), tz, A::sub(g[17], u6));
}

// Inlet (x = 0) and outlet (x = nx - 1) substitutions of the pulled values.
template <class S>
__device__ __forceinline__ void faces3(const Step3<S> &a, uint32_t x, typename Codec<S>::C *g) {
    if (a.inlet && x == 0) {
        if (a.inlet == 1) {
#pragma unroll
            for (int i = 0; i < Q; ++i) g[i] = a.heq_in[i];
        } else {
            zou_he3(a, g);
        }
    }
    if (a.outlet && x == (uint32_t)a.g.nx - 1) zou_he_pressure3(a, g);
}

// Node stride of direction i's array in a layout: 1 (stream; one-direction
// bundles), 3 (three-direction bundles), 19 (collision).
template <int L>
__host__ __device__ constexpr uint32_t mult3(int i) {
    return L == STREAM ? 1u : (L == COLLISION ? 19u : (uint32_t)bundle_size(i));
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, uint64_t magic) {
    return magic ? (uint32_t)__umul64hi((unsigned long long)n, magic) : n;
}

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

// Store hint: 0 plain stores (measured fastest), 1 evict-first (.cs)
// everywhere, 2 evict-first for the bundle layout only.
#ifndef LBM3_ST_HINT
#define LBM3_ST_HINT 0
#endif
template <class S, int L>
__device__ __forceinline__ void st3(S *p, S v) {
    if (LBM3_ST_HINT == 1 || (LBM3_ST_HINT == 2 && L == BUNDLE))
        __stcs(p, v);
    else
        *p = v;
}

// Pulled values of fluid node n at (x, y, z) with link word lk: the
// neighbour's value, or the node's own opposite slot for a bounced link.
template <class S, int L, bool OFF32>
__device__ __forceinline__ void pull3(const Step3<S> &a, uint32_t x, uint32_t y, uint32_t z, uint32_t n,
                                      uint32_t lk, typename Codec<S>::C *g) {
    const uint32_t nx = (uint32_t)a.g.nx, ny = (uint32_t)a.g.ny, nz = (uint32_t)a.g.nz;
    const S *__restrict__ src = a.src;
    const bool interior = (x - 1u < nx - 2u) && (y - 1u < ny - 2u) && (z - 1u < nz - 2u);
    if (OFF32) {
        // Node-index corrections of a pull that leaves the box through a
        // periodic face (walls bounce, so their corrections go unused):
        // c = +1 pulls from coordinate -1 at the low face, c = -1 from the
        // extent at the high face.
        const int N = (int)a.N, nxy = (int)(nx * ny);
        const int xlo = x == 0 ? a.xlo_corr : 0, xhi = x == nx - 1 ? a.xhi_corr : 0;
        const int ylo = y == 0 ? nxy : 0, yhi = y == ny - 1 ? -nxy : 0;
        const int zlo = z == 0 ? N : 0, zhi = z == nz - 1 ? -N : 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const S *b = src + mult3<L>(i) * n;
            int o;
            if (i == REST) {
                o = a.os[i];
            } else if ((lk >> bit(i)) & 1u) {
                o = a.ob[i];
            } else {
                const int w = (cx(i) > 0 ? xlo : cx(i) < 0 ? xhi : 0) + (cy(i) > 0 ? ylo : cy(i) < 0 ? yhi : 0) +
                              (cz(i) > 0 ? zlo : cz(i) < 0 ? zhi : 0);
                o = a.op[i] + (int)mult3<L>(i) * w;
            }
            g[i] = Codec<S>::dec(b[o]);
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        uint32_t s = n;
        int j = i;
        if (i != REST) {
            if ((lk >> bit(i)) & 1u) {
                j = opp(i);
            } else if (interior) {
                s = n - (uint32_t)(((int64_t)cz(i) * ny + cy(i)) * (int64_t)nx + cx(i));
            } else {
                map3(a.g, (int)x, (int)y, (int)z, i, s);
            }
        }
        g[i] = Codec<S>::dec(src[addr<L>(a.N, s, j)]);
    }
}

// Collision, moments and the encoded stores of node n.
template <class S, int L, bool OFF32>
__device__ __forceinline__ void finish3(const Step3<S> &a, uint32_t n, typename Codec<S>::C *g) {
    using C = typename Codec<S>::C;
    using A = Ar<C>;
    C drho, ux, uy, uz;
    collide3(a.k, g, drho, ux, uy, uz);
    if (!isfinite(drho)) atomicOr(a.err, 1u);
    if (a.mom) {
        a.mom[n] = A::add(C(1), drho);
        a.mom[a.N + n] = ux;
        a.mom[2 * (size_t)a.N + n] = uy;
        a.mom[3 * (size_t)a.N + n] = uz;
    }
    const bool sr = Codec<S>::narrow && a.sr;
    uint32_t nk = 0;
    if (sr) nk = node_key(step_key(a.seed, (uint32_t)(*a.tctr + a.toff)), n);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        S *p = OFF32 ? a.dst + (mult3<L>(i) * n + (uint32_t)a.os[i]) : a.dst + addr<L>(a.N, n, i);
        st3<S, L>(p, Codec<S>::enc(g[i], sr, sr ? pop_rand(nk, i) : 0u));
    }
}

// Solid nodes hold zeros in both lattices and are not rewritten, except
// where their slots share a 32-byte sector with a fluid node's slots: there
// zeros complete the sector so that it is written whole instead of being
// read, merged and written back. F: ballot of fluid lanes, lanes holding
// consecutive nodes. Stream: aligned groups of 32/sizeof(S) nodes; bundle:
// those groups (single-direction bundles) and the lanes within
// ceil(32 / (3 sizeof(S))) (three-direction bundles); collision: +-1 lane.
template <class S, int L>
__device__ __forceinline__ bool shares3(unsigned F, int lane) {
    constexpr int G = (int)(32 / sizeof(S)) < 32 ? (int)(32 / sizeof(S)) : 32;
    const unsigned grp = G >= 32 ? 0xffffffffu : ((1u << G) - 1u) << (lane & ~(G - 1));
    constexpr int k = L == COLLISION ? 1 : (int)((32 + 3 * sizeof(S) - 1) / (3 * sizeof(S)));
    const int lo = lane - k < 0 ? 0 : lane - k;
    const int hi = lane + k > 31 ? 31 : lane + k;
    const int w = hi - lo + 1;
    const unsigned near = w >= 32 ? 0xffffffffu : ((1u << w) - 1u) << lo;
    const unsigned m = L == STREAM ? grp : (L == BUNDLE ? (grp | near) : near);
    return (F & m) != 0u;
}

template <class S, int L>
__device__ __forceinline__ void zero3(const Step3<S> &a, uint32_t n) {
    const S z = Codec<S>::enc(typename Codec<S>::C(0), false, 0u);
#pragma unroll
    for (int i = 0; i < Q; ++i) st3<S, L>(a.dst + addr<L>(a.N, n, i), z);
}

// LINEAR: one node per thread over n (LPTL); otherwise 3-D tiles (NPTL).
// OFF32: the offset tables fit 31 bits; every pull uses them (periodic wrap
// as node-index corrections); otherwise 64-bit addressing with the general
// edge mapping for nodes on the box faces.
template <class S, int L, bool LINEAR, bool OFF32>
__global__ void __launch_bounds__(512, sizeof(S) == 8 ? 2 : 3) k3_step(const Step3<S> a) {
    using C = typename Codec<S>::C;
    const uint32_t nx = (uint32_t)a.g.nx, ny = (uint32_t)a.g.ny, nz = (uint32_t)a.g.nz;
    uint32_t x, y, z;
    if (LINEAR) {
        const uint64_t n64 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (n64 >= a.N) return;
        const uint32_t n = (uint32_t)n64;
        z = fdiv(n, a.nxy_magic);
        const uint32_t r = n - z * nx * ny;
        y = fdiv(r, a.nx_magic);
        x = r - y * nx;
    } else {
        x = blockIdx.x * a.tx + threadIdx.x;
        y = blockIdx.y * a.ty + threadIdx.y;
        z = blockIdx.z * a.tz + threadIdx.z;
        if (x >= nx || y >= ny || z >= nz) return;
    }
    const uint32_t n = (z * ny + y) * nx + x;
    const uint32_t lk = a.links[n];
    const bool f = lk != SOLID;
#ifndef LBM3_NO_ZERO_FILL
    if (a.zero_fill) {
        const int lane = (int)(((threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x) & 31u);
        const unsigned F = __ballot_sync(__activemask(), f);
        if (!f && shares3<S, L>(F, lane)) zero3<S, L>(a, n);
    }
#endif
    if (!f) return;
    C g[Q];
    pull3<S, L, OFF32>(a, x, y, z, n, lk, g);
    faces3(a, x, g);
    finish3<S, L, OFF32>(a, n, g);
}

// AA pattern on one array. Even updates (PHASE 0) start from the canonical
// state (slot i of node n holds h_i(n)): each fluid node pulls as the
// two-lattice update does and writes its result for direction i into slot
// opp(i) of node n + c_i, the slot only this node read, or into its own slot
// i when that neighbour is solid or beyond a wall (the next update bounces it
// back from there). Odd updates (PHASE 1) read the node's own slots opp(i),
// collide, and write slot i: the canonical state again. Every slot has one
// reader and one writer per phase, and each thread reads all its slots
// before writing any. Requires the 32-bit offset tables.
template <class S, int L, int PHASE>
__global__ void __launch_bounds__(512, PHASE == 0 ? (sizeof(S) == 8 ? 1 : 2) : (sizeof(S) == 8 ? 2 : 3)) k3_aa(const Step3<S> a) {
    using C = typename Codec<S>::C;
    const uint32_t nx = (uint32_t)a.g.nx, ny = (uint32_t)a.g.ny, nz = (uint32_t)a.g.nz;
    const uint32_t x = blockIdx.x * a.tx + threadIdx.x;
    const uint32_t y = blockIdx.y * a.ty + threadIdx.y;
    const uint32_t z = blockIdx.z * a.tz + threadIdx.z;
    if (x >= nx || y >= ny || z >= nz) return;
    const uint32_t n = (z * ny + y) * nx + x;
    const uint32_t lk = a.links[n];
    if (lk == SOLID) return;
    S *lat = a.dst;
    C g[Q];
    if (PHASE == 0) {
        pull3<S, L, true>(a, x, y, z, n, lk, g);
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) g[i] = Codec<S>::dec(lat[mult3<L>(i) * n + (uint32_t)a.ob[i]]);
    }
    using A = Ar<C>;
    C drho, ux, uy, uz;
    collide3(a.k, g, drho, ux, uy, uz);
    if (!isfinite(drho)) atomicOr(a.err, 1u);
    if (a.mom) {
        a.mom[n] = A::add(C(1), drho);
        a.mom[a.N + n] = ux;
        a.mom[2 * (size_t)a.N + n] = uy;
        a.mom[3 * (size_t)a.N + n] = uz;
    }
    const bool sr = Codec<S>::narrow && a.sr;
    uint32_t nk = 0;
    if (sr) nk = node_key(step_key(a.seed, (uint32_t)(*a.tctr + a.toff)), n);
    // push corrections for a neighbour across a periodic face
    const int N = (int)a.N, nxy = (int)(nx * ny);
    const int xhi = x == nx - 1 ? -(int)nx : 0, xlo = x == 0 ? (int)nx : 0;
    const int yhi = y == ny - 1 ? -nxy : 0, ylo = y == 0 ? nxy : 0;
    const int zhi = z == nz - 1 ? -N : 0, zlo = z == 0 ? N : 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        S *b = lat + mult3<L>(i) * n;
        int o;
        if (PHASE == 1 || i == REST || ((lk >> bit(opp(i))) & 1u)) {
            o = a.os[i];
        } else {
            const int w = (cx(i) > 0 ? xhi : cx(i) < 0 ? xlo : 0) + (cy(i) > 0 ? yhi : cy(i) < 0 ? ylo : 0) +
                          (cz(i) > 0 ? zhi : cz(i) < 0 ? zlo : 0);
            o = a.oq[i] + (int)mult3<L>(i) * w;
        }
        st3<S, L>(b + o, Codec<S>::enc(g[i], sr, sr ? pop_rand(nk, i) : 0u));
    }
}

// ------------------------------------------------------------ NPOL (3-D)
// Buffer grid: per tile and parity, for each of the six tile faces the five
// populations that leave each face node through it (c_a = +1 for the high
// face of axis a, -1 for the low face). Face order x+, x-, y+, y-, z+, z-;
// a face of axis x holds ty tz slots per direction (position ly + ty lz),
// of axis y tx tz (lx + tx lz), of axis z tx ty (lx + tx ly).
struct Tile3 {
    int tx, ty, tz;
    __host__ __device__ int nodes(int axis) const { return axis == 0 ? ty * tz : (axis == 1 ? tx * tz : tx * ty); }
    __host__ __device__ int64_t per_tile() const { return 10ll * (nodes(0) + nodes(1) + nodes(2)); }
    __host__ __device__ int64_t face_off(int axis, int sign) const {
        int64_t o = 0;
        for (int a = 0; a < axis; ++a) o += 10ll * nodes(a);
        return o + (sign > 0 ? 0 : 5ll * nodes(axis));
    }
    __host__ __device__ int pos(int axis, int lx, int ly, int lz) const {
        return axis == 0 ? ly + ty * lz : (axis == 1 ? lx + tx * lz : lx + tx * ly);
    }
};

// Rank of direction i among the five directions with the same nonzero c_a.
__host__ __device__ constexpr int face_rank(int i, int axis) {
    int r = 0;
    for (int j = 0; j < i; ++j) {
        const int cj = axis == 0 ? cx(j) : (axis == 1 ? cy(j) : cz(j));
        const int ci = axis == 0 ? cx(i) : (axis == 1 ? cy(i) : cz(i));
        if (cj == ci) ++r;
    }
    return r;
}

// Publish the outgoing populations e (canonical order) of the node at local
// (lx, ly, lz) of tile t, whose bounds are lo[] .. hi[] (global).
template <class S>
__device__ __forceinline__ void publish3(S *hw, const Tile3 &T, int64_t t, const int *p, const int *lo,
                                         const int *hi, int lx, int ly, int lz, const S *e) {
    S *base = hw + t * T.per_tile();
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int pos = T.pos(a, lx, ly, lz);
        const int fn = T.nodes(a);
        if (p[a] == hi[a]) {
            S *f = base + T.face_off(a, 1);
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if ((a == 0 ? cx(i) : (a == 1 ? cy(i) : cz(i))) > 0) f[face_rank(i, a) * fn + pos] = e[i];
        }
        if (p[a] == lo[a]) {
            S *f = base + T.face_off(a, -1);
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if ((a == 0 ? cx(i) : (a == 1 ? cy(i) : cz(i))) < 0) f[face_rank(i, a) * fn + pos] = e[i];
        }
    }
}

// Pulls of a fluid node off the box faces with the 32-bit offset tables:
// every lane runs the interior pull (neighbour value, or the node's own
// opposite value for a bounced link) and, for a direction whose source lies
// in another tile, reads the source tile's publication of the previous
// update instead (the face of the first axis along which the tiles differ).
// Face nodes therefore run the same code as inner nodes plus a short
// address computation per crossing direction.
template <class S, int L>
__device__ __forceinline__ void npol3_pull(const Step3<S> &a, const S *hr, const Tile3 &T, const int *b,
                                           const int *nt, const int *tdim, const int *l, const int *p,
                                           const int *lo, const int *hi, uint32_t n, uint32_t lk,
                                           typename Codec<S>::C *g) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const S *base = a.src + mult3<L>(i) * n;
        if (i == REST) {
            g[i] = Codec<S>::dec(base[a.os[i]]);
            continue;
        }
        const bool bounce = (lk >> bit(i)) & 1u;
        const S *q = base + (bounce ? a.ob[i] : a.op[i]);
        const int c[3] = {cx(i), cy(i), cz(i)};
        bool cr[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) cr[k] = (c[k] > 0 && p[k] == lo[k]) || (c[k] < 0 && p[k] == hi[k]);
        if (!bounce && (cr[0] || cr[1] || cr[2])) {
            int bs[3], ls[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                bs[k] = cr[k] ? b[k] - c[k] : b[k];
                ls[k] = cr[k] ? (c[k] > 0 ? tdim[k] - 1 : 0) : l[k] - c[k];
            }
            const int ax = cr[0] ? 0 : (cr[1] ? 1 : 2);
            const int64_t ts = ((int64_t)bs[2] * nt[1] + bs[1]) * nt[0] + bs[0];
            q = hr + ts * T.per_tile() + T.face_off(ax, c[ax]) + (int64_t)face_rank(i, ax) * T.nodes(ax) +
                T.pos(ax, ls[0], ls[1], ls[2]);
        }
        g[i] = Codec<S>::dec(*q);
    }
}

// One lattice, pull: every node of the tile reads its 19 incoming values
// (sources in the tile from the lattice, from other tiles out of the buffer
// grid the previous update wrote), a block barrier separates all reads from
// the in-place writes, and face nodes publish their outgoing values.
template <class S, int L, bool OFF32>
__global__ void __launch_bounds__(512, sizeof(S) == 8 ? 1 : 2) k3_npol(const Step3<S> a, const S *hr, S *hw) {
    using C = typename Codec<S>::C;
    using A = Ar<C>;
    const Tile3 T{a.tx, a.ty, a.tz};
    const int ext[3] = {a.g.nx, a.g.ny, a.g.nz};
    const int b[3] = {(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z};
    const int tdim[3] = {a.tx, a.ty, a.tz};
    const int l[3] = {(int)threadIdx.x, (int)threadIdx.y, (int)threadIdx.z};
    int lo[3], hi[3], p[3];
    bool valid = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        lo[k] = b[k] * tdim[k];
        hi[k] = min(lo[k] + tdim[k], ext[k]) - 1;
        p[k] = lo[k] + l[k];
        valid = valid && p[k] <= hi[k];
    }
    const uint32_t nx = (uint32_t)ext[0], ny = (uint32_t)ext[1];
    S *lat = a.dst;
    uint32_t n = 0, lk = SOLID;
    if (valid) {
        n = ((uint32_t)p[2] * ny + (uint32_t)p[1]) * nx + (uint32_t)p[0];
        lk = a.links[n];
    }
    const bool fluid = lk != SOLID;
    const bool inner = p[0] > lo[0] && p[0] < hi[0] && p[1] > lo[1] && p[1] < hi[1] && p[2] > lo[2] && p[2] < hi[2];
    const int nt[3] = {(int)gridDim.x, (int)gridDim.y, (int)gridDim.z};
    const int64_t t = ((int64_t)b[2] * nt[1] + b[1]) * nt[0] + b[0];
    C g[Q];
    const bool box_inner = p[0] > 0 && p[0] < ext[0] - 1 && p[1] > 0 && p[1] < ext[1] - 1 && p[2] > 0 &&
                           p[2] < ext[2] - 1;
    if (fluid && inner) {
        pull3<S, L, OFF32>(a, (uint32_t)p[0], (uint32_t)p[1], (uint32_t)p[2], n, lk, g);
    } else if (OFF32 && fluid && box_inner) {
        npol3_pull<S, L>(a, hr, T, b, nt, tdim, l, p, lo, hi, n, lk, g);
    } else if (fluid) {
        // Per axis: does a pull with c = +1 (-1) leave the tile (the node is on
        // the tile's low (high) face)? Where the tile spans the whole axis, such
        // a pull wraps around the box inside the tile (periodic) or bounces.
        bool lof[3], hif[3];
        int wrap_lo[3], wrap_hi[3];   // node-index correction of an in-tile wrap
        int tprev[3], tnext[3], lprev[3];
        const int stride[3] = {1, (int)nx, (int)(nx * ny)};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lof[k] = p[k] == lo[k];
            hif[k] = p[k] == hi[k];
            wrap_lo[k] = p[k] == 0 ? ext[k] * stride[k] : 0;
            wrap_hi[k] = p[k] == ext[k] - 1 ? -ext[k] * stride[k] : 0;
            tprev[k] = b[k] == 0 ? nt[k] - 1 : b[k] - 1;
            tnext[k] = b[k] == nt[k] - 1 ? 0 : b[k] + 1;
            lprev[k] = min(tdim[k], ext[k] - tprev[k] * tdim[k]) - 1;
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (i == REST) {
                g[i] = Codec<S>::dec(lat[addr<L>(a.N, n, i)]);
                continue;
            }
            if ((lk >> bit(i)) & 1u) {
                g[i] = Codec<S>::dec(lat[addr<L>(a.N, n, opp(i))]);
                continue;
            }
            const int c[3] = {cx(i), cy(i), cz(i)};
            bool out = false;   // the source lies in another tile
            int shift = 0;      // node-index shift of the source (in-tile, wraps included)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (c[k] == 0) continue;
                const bool cross = c[k] > 0 ? lof[k] : hif[k];
                shift += -c[k] * stride[k];
                if (cross) {
                    if (nt[k] == 1) shift += c[k] > 0 ? wrap_lo[k] : wrap_hi[k];
                    else out = true;
                }
            }
            if (!out) {
                g[i] = Codec<S>::dec(lat[addr<L>(a.N, (uint32_t)((int64_t)n + shift), i)]);
            } else {
                // the value left the source tile through its face of the first
                // axis along which the tiles differ
                int bs[3], ls[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const bool cr = c[k] != 0 && (c[k] > 0 ? lof[k] : hif[k]) && nt[k] > 1;
                    if (!cr) {
                        bs[k] = b[k];
                        int sk = p[k] - c[k];
                        sk = sk < 0 ? sk + ext[k] : (sk >= ext[k] ? sk - ext[k] : sk);
                        ls[k] = sk - lo[k];
                    } else {
                        bs[k] = c[k] > 0 ? tprev[k] : tnext[k];
                        ls[k] = c[k] > 0 ? lprev[k] : 0;
                    }
                }
                const int ax = bs[0] != b[0] ? 0 : (bs[1] != b[1] ? 1 : 2);
                const int64_t ts = ((int64_t)bs[2] * nt[1] + bs[1]) * nt[0] + bs[0];
                const int64_t slot = ts * T.per_tile() + T.face_off(ax, c[ax]) +
                                     (int64_t)face_rank(i, ax) * T.nodes(ax) + T.pos(ax, ls[0], ls[1], ls[2]);
                g[i] = Codec<S>::dec(hr[slot]);
            }
        }
    }
    __syncthreads();
    if (!fluid) return;
    C drho, ux, uy, uz;
    collide3(a.k, g, drho, ux, uy, uz);
    if (!isfinite(drho)) atomicOr(a.err, 1u);
    if (a.mom) {
        a.mom[n] = A::add(C(1), drho);
        a.mom[a.N + n] = ux;
        a.mom[2 * (size_t)a.N + n] = uy;
        a.mom[3 * (size_t)a.N + n] = uz;
    }
    const bool sr = Codec<S>::narrow && a.sr;
    uint32_t nk = 0;
    if (sr) nk = node_key(step_key(a.seed, (uint32_t)(*a.tctr + a.toff)), n);
    S e[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        e[i] = Codec<S>::enc(g[i], sr, sr ? pop_rand(nk, i) : 0u);
        lat[addr<L>(a.N, n, i)] = e[i];
    }
    if (!inner) publish3(hw, T, t, p, lo, hi, l[0], l[1], l[2], e);
}

// ------------------------------------------------------------ NSOL (3-D)
// One lattice, swap streaming (Sec. 3.3): the stored state holds population
// i of every node in its slot opp(i). The tile's slots are staged in shared
// memory; for each of the nine positive directions i (i > 9: c lexically
// positive), slot opp(i) of node x is exchanged with slot i of x + c_i when
// x + c_i is in the tile and no bounce separates them. After the exchanges
// slot j of x holds the value x pulls in direction j (a bounced link keeps
// the node's own value, i.e. bounce-back). Pulls from other tiles come from
// the buffer grid, in the same format as NPOL's; pulls that wrap around a
// periodic face inside one tile are read from the staged slots before the
// exchange. Results are stored back into the opposite slots and face nodes
// publish their outgoing values. Shared memory: 19 planes of the tile's
// nodes (compute type).
template <class S>
size_t nsol3_smem_bytes(int tx, int ty, int tz) {
    return sizeof(typename Codec<S>::C) * (size_t)Q * (size_t)tx * ty * tz;
}

template <class S, int L>
__global__ void __launch_bounds__(512, sizeof(S) == 8 ? 1 : 2) k3_nsol(const Step3<S> a, const S *hr, S *hw) {
    using C = typename Codec<S>::C;
    using A = Ar<C>;
    extern __shared__ __align__(16) unsigned char smem_nsol3[];
    C *sm = reinterpret_cast<C *>(smem_nsol3);
    const Tile3 T{a.tx, a.ty, a.tz};
    const int TN = a.tx * a.ty * a.tz;
    const int ext[3] = {a.g.nx, a.g.ny, a.g.nz};
    const int b[3] = {(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z};
    const int tdim[3] = {a.tx, a.ty, a.tz};
    const int l[3] = {(int)threadIdx.x, (int)threadIdx.y, (int)threadIdx.z};
    const int tid = (l[2] * a.ty + l[1]) * a.tx + l[0];
    int lo[3], hi[3], p[3];
    bool valid = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        lo[k] = b[k] * tdim[k];
        hi[k] = min(lo[k] + tdim[k], ext[k]) - 1;
        p[k] = lo[k] + l[k];
        valid = valid && p[k] <= hi[k];
    }
    const uint32_t nx = (uint32_t)ext[0], ny = (uint32_t)ext[1];
    S *lat = a.dst;
    uint32_t n = 0, lk = SOLID;
    if (valid) {
        n = ((uint32_t)p[2] * ny + (uint32_t)p[1]) * nx + (uint32_t)p[0];
        lk = a.links[n];
    }
    const bool fluid = lk != SOLID;
    const bool inner = p[0] > lo[0] && p[0] < hi[0] && p[1] > lo[1] && p[1] < hi[1] && p[2] > lo[2] && p[2] < hi[2];
    const int nt[3] = {(int)gridDim.x, (int)gridDim.y, (int)gridDim.z};
    const int64_t t = ((int64_t)b[2] * nt[1] + b[1]) * nt[0] + b[0];
    if (fluid) {
#pragma unroll
        for (int s = 0; s < Q; ++s) sm[s * TN + tid] = Codec<S>::dec(lat[addr<L>(a.N, n, s)]);
    }
    __syncthreads();
    // Pulls the in-tile exchange does not cover: sources in another tile
    // (buffer grid) or reached through a periodic face inside this tile.
    C fix[Q];
    uint32_t fixmask = 0;
    if (fluid && !inner) {
        bool lof[3], hif[3];
        int tprev[3], tnext[3], lprev[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lof[k] = p[k] == lo[k];
            hif[k] = p[k] == hi[k];
            tprev[k] = b[k] == 0 ? nt[k] - 1 : b[k] - 1;
            tnext[k] = b[k] == nt[k] - 1 ? 0 : b[k] + 1;
            lprev[k] = min(tdim[k], ext[k] - tprev[k] * tdim[k]) - 1;
        }
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            fix[j] = C(0);
            if (j == REST || ((lk >> bit(j)) & 1u)) continue;
            const int c[3] = {cx(j), cy(j), cz(j)};
            bool cross = false, out = false;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (c[k] == 0) continue;
                if (c[k] > 0 ? lof[k] : hif[k]) {
                    cross = true;
                    if (nt[k] > 1) out = true;
                }
            }
            if (!cross) continue;   // adjacent in the tile: the exchange delivers it
            fixmask |= 1u << j;
            if (!out) {
                // wraps around a periodic face of an axis the tile spans whole
                int q[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    int sk = p[k] - c[k];
                    sk = sk < 0 ? sk + ext[k] : (sk >= ext[k] ? sk - ext[k] : sk);
                    q[k] = sk - lo[k];
                }
                fix[j] = sm[opp(j) * TN + (q[2] * a.ty + q[1]) * a.tx + q[0]];
            } else {
                int bs[3], ls[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const bool cr = c[k] != 0 && (c[k] > 0 ? lof[k] : hif[k]) && nt[k] > 1;
                    if (!cr) {
                        bs[k] = b[k];
                        int sk = p[k] - c[k];
                        sk = sk < 0 ? sk + ext[k] : (sk >= ext[k] ? sk - ext[k] : sk);
                        ls[k] = sk - lo[k];
                    } else {
                        bs[k] = c[k] > 0 ? tprev[k] : tnext[k];
                        ls[k] = c[k] > 0 ? lprev[k] : 0;
                    }
                }
                const int ax = bs[0] != b[0] ? 0 : (bs[1] != b[1] ? 1 : 2);
                const int64_t ts = ((int64_t)bs[2] * nt[1] + bs[1]) * nt[0] + bs[0];
                const int64_t slot = ts * T.per_tile() + T.face_off(ax, c[ax]) +
                                     (int64_t)face_rank(j, ax) * T.nodes(ax) + T.pos(ax, ls[0], ls[1], ls[2]);
                fix[j] = Codec<S>::dec(hr[slot]);
            }
        }
    }
    __syncthreads();
    if (fluid) {
#pragma unroll
        for (int i = REST + 1; i < Q; ++i) {
            if ((lk >> bit(opp(i))) & 1u) continue;   // bounced: no exchange
            const int c[3] = {cx(i), cy(i), cz(i)};
            bool in = true;
#pragma unroll
            for (int k = 0; k < 3; ++k) in = in && p[k] + c[k] >= lo[k] && p[k] + c[k] <= hi[k];
            if (!in) continue;
            const int pt = tid + (c[2] * a.ty + c[1]) * a.tx + c[0];
            const C v = sm[opp(i) * TN + tid];
            sm[opp(i) * TN + tid] = sm[i * TN + pt];
            sm[i * TN + pt] = v;
        }
    }
    __syncthreads();
    if (!fluid) return;
    C g[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) g[j] = ((fixmask >> j) & 1u) ? fix[j] : sm[j * TN + tid];
    C drho, ux, uy, uz;
    collide3(a.k, g, drho, ux, uy, uz);
    if (!isfinite(drho)) atomicOr(a.err, 1u);
    if (a.mom) {
        a.mom[n] = A::add(C(1), drho);
        a.mom[a.N + n] = ux;
        a.mom[2 * (size_t)a.N + n] = uy;
        a.mom[3 * (size_t)a.N + n] = uz;
    }
    const bool sr = Codec<S>::narrow && a.sr;
    uint32_t nk = 0;
    if (sr) nk = node_key(step_key(a.seed, (uint32_t)(*a.tctr + a.toff)), n);
    S e[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        e[i] = Codec<S>::enc(g[i], sr, sr ? pop_rand(nk, i) : 0u);
        lat[addr<L>(a.N, n, opp(i))] = e[i];
    }
    if (!inner) publish3(hw, T, t, p, lo, hi, l[0], l[1], l[2], e);
}

// Fill a buffer-grid parity from the stored state (after init or a write).
template <class S, int L>
__global__ void k3_publish(const Step3<S> a, S *hw) {
    const Tile3 T{a.tx, a.ty, a.tz};
    const int ext[3] = {a.g.nx, a.g.ny, a.g.nz};
    const int b[3] = {(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z};
    const int tdim[3] = {a.tx, a.ty, a.tz};
    const int l[3] = {(int)threadIdx.x, (int)threadIdx.y, (int)threadIdx.z};
    int lo[3], hi[3], p[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        lo[k] = b[k] * tdim[k];
        hi[k] = min(lo[k] + tdim[k], ext[k]) - 1;
        p[k] = lo[k] + l[k];
        if (p[k] > hi[k]) return;
    }
    const uint32_t n = (((uint32_t)p[2] * (uint32_t)ext[1]) + (uint32_t)p[1]) * (uint32_t)ext[0] + (uint32_t)p[0];
    if (a.links[n] == SOLID) return;
    const int64_t ntx = (ext[0] + a.tx - 1) / a.tx, nty = (ext[1] + a.ty - 1) / a.ty;
    const int64_t t = ((int64_t)b[2] * nty + b[1]) * ntx + b[0];
    S e[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) e[i] = a.dst[addr<L>(a.N, n, slot3(a, i))];
    publish3(hw, T, t, p, lo, hi, l[0], l[1], l[2], e);
}

template <class S, int L>
__global__ void k3_init(const Step3<S> a, const double *rho, const double *ux, const double *uy,
                        const double *uz, uint32_t n0, uint32_t count) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const uint32_t n = n0 + t;
    if (a.links[n] == SOLID) return;
    const double dr = rho ? rho[t] - 1.0 : 0.0;
    const double v[3] = {ux ? ux[t] : 0.0, uy ? uy[t] : 0.0, uz ? uz[t] : 0.0};
    const double usq = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const double w = sq(i) == 0 ? 1.0 / 3.0 : (sq(i) == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        const double cu = cx(i) * v[0] + cy(i) * v[1] + cz(i) * v[2];
        const double h = w * (dr + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
        a.dst[addr<L>(a.N, n, slot3(a, i))] = Codec<S>::enc((typename Codec<S>::C)h, false, 0u);
    }
}

template <class S, int L>
__global__ void k3_state_moments(const Step3<S> a) {
    using C = typename Codec<S>::C;
    using A = Ar<C>;
    const uint64_t n64 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n64 >= a.N) return;
    const uint32_t n = (uint32_t)n64;
    C *m = a.mom;
    if (a.links[n] == SOLID) {
        m[n] = C(1);
        m[a.N + n] = C(0);
        m[2 * (size_t)a.N + n] = C(0);
        m[3 * (size_t)a.N + n] = C(0);
        return;
    }
    C r = C(0), j[3] = {C(0), C(0), C(0)};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const C h = Codec<S>::dec(a.src[addr<L>(a.N, n, slot3(a, i))]);
        r = A::add(r, h);
        if (cx(i)) j[0] = cx(i) > 0 ? A::add(j[0], h) : A::sub(j[0], h);
        if (cy(i)) j[1] = cy(i) > 0 ? A::add(j[1], h) : A::sub(j[1], h);
        if (cz(i)) j[2] = cz(i) > 0 ? A::add(j[2], h) : A::sub(j[2], h);
    }
    m[n] = A::add(C(1), r);
    m[a.N + n] = j[0];
    m[2 * (size_t)a.N + n] = j[1];
    m[3 * (size_t)a.N + n] = j[2];
}

template <class S, int L>
__global__ void __launch_bounds__(kReduceThreads) k3_mass(const Step3<S> a, double *partials) {
    __shared__ double red[kReduceThreads];
    double acc = 0.0;
    for (uint64_t n64 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; n64 < a.N;
         n64 += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t n = (uint32_t)n64;
        if (a.links[n] == SOLID) continue;
        double r = 1.0;
#pragma unroll
        for (int i = 0; i < Q; ++i) r += (double)Codec<S>::dec(a.src[addr<L>(a.N, n, slot3(a, i))]);
        acc += r;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kReduceThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

// Momentum-exchange force: over fluid nodes and links into body nodes
// (d_body[m] != 0, or solid nodes when body is NULL; links across a
// non-periodic face are skipped), 2 c_i (w_i + h_i) of the stored state.
// Per-block partials of the three components, FP64.
template <class S, int L>
__global__ void __launch_bounds__(kReduceThreads) k3_force(const Step3<S> a, const uint8_t *body,
                                                           double *partials) {
    __shared__ double red[3][kReduceThreads];
    double acc[3] = {0.0, 0.0, 0.0};
    const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
    const int ext[3] = {nx, ny, nz};
    const int bc[3] = {a.g.bx, a.g.by, a.g.bz};
    for (uint64_t n64 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; n64 < a.N;
         n64 += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t n = (uint32_t)n64;
        if (a.links[n] == SOLID) continue;
        const uint32_t z = fdiv(n, a.nxy_magic);
        const uint32_t r = n - z * (uint32_t)nx * (uint32_t)ny;
        const uint32_t y = fdiv(r, a.nx_magic);
        const uint32_t x = r - y * (uint32_t)nx;
        const int p[3] = {(int)x, (int)y, (int)z};
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (i == REST) continue;
            const int c[3] = {cx(i), cy(i), cz(i)};
            int b[3];
            bool inside = true;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                b[k] = p[k] + c[k];
                if (b[k] < 0 || b[k] >= ext[k]) {
                    if (bc[k] != PERIODIC) inside = false;
                    b[k] = b[k] < 0 ? b[k] + ext[k] : b[k] - ext[k];
                }
            }
            if (!inside) continue;
            const uint32_t m = ((uint32_t)b[2] * (uint32_t)ny + (uint32_t)b[1]) * (uint32_t)nx + (uint32_t)b[0];
            const bool hit = body ? body[m] != 0 : a.links[m] == SOLID;
            if (!hit) continue;
            const double w = sq(i) == 1 ? 1.0 / 18.0 : 1.0 / 36.0;
            const double f = w + (double)Codec<S>::dec(a.src[addr<L>(a.N, n, slot3(a, i))]);
#pragma unroll
            for (int k = 0; k < 3; ++k) acc[k] += 2.0 * c[k] * f;
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = kReduceThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
#pragma unroll
            for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 3; ++k) partials[3 * blockIdx.x + k] = red[k][0];
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

// ------------------------------------------------------------ host side
namespace {

struct Plan3 {
    int64_t N = 0;
    int tx = 0, ty = 1, tz = 1, ntx = 0, nty = 0, ntz = 0;
    size_t elem = 0, comp = 0;
    size_t pop[2] = {0, 0}, links = 0, mom = 0, mom_bytes = 0, partials = 0, misc = 0, total = 0;
    int one = 0;   // one lattice (AA pattern, NPOL)
    size_t halo = 0;          // NPOL buffer grid (two parities)
    int64_t halo_parity = 0;  // elements per parity
};

size_t elem_of(int storage) { return storage == LBM_F64 ? 8 : storage == LBM_F32 ? 4 : 2; }
size_t comp_of(int storage) { return storage == LBM_F64 ? 8 : 4; }

bool offsets_fit(const lbm3_params *p, int64_t N);

bool inlet_kind(int bc) { return bc == LBM_BC_INLET_EQ || bc == LBM_BC_INLET_ZOUHE; }

// Kind of the east x face: bc_x_east after an inlet west face, else bc_x.
int east_kind(const lbm3_params *p) { return inlet_kind(p->bc_x) ? p->bc_x_east : p->bc_x; }

lbm_status plan3(const lbm3_params *p, Plan3 *pl) {
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
    if (p->bc_x != LBM_BC_PERIODIC && p->bc_x != LBM_BC_WALL && !inlet_kind(p->bc_x) &&
        p->bc_x != LBM_BC_OUTFLOW_ZG)
        return lbm_fail(LBM_EINVAL, "D3Q19 x faces: PERIODIC, WALL, INLET_EQ or INLET_ZOUHE (west) or OUTFLOW_ZG");
    if (inlet_kind(p->bc_x) && p->bc_x_east != LBM_BC_WALL && p->bc_x_east != LBM_BC_OUTFLOW_ZG &&
        p->bc_x_east != LBM_BC_OUTLET_PRESSURE)
        return lbm_fail(LBM_EINVAL, "D3Q19 inlet: the east face (bc_x_east) is WALL, OUTFLOW_ZG or OUTLET_PRESSURE");
    if (inlet_kind(p->bc_x) && p->bc_x_east == LBM_BC_OUTLET_PRESSURE && !(p->rho_out > 0.0 && std::isfinite(p->rho_out)))
        return lbm_fail(LBM_EINVAL, "D3Q19 pressure outlet: rho_out must be finite and > 0");
    const bool open_x = inlet_kind(p->bc_x) || p->bc_x == LBM_BC_OUTFLOW_ZG;
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
    pl->elem = elem_of(p->storage);
    pl->comp = comp_of(p->storage);
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = (off + b + 255) / 256 * 256; return o; };
    pl->pop[0] = take(19 * (size_t)N * pl->elem);
    pl->one = (p->algo == LBM_AA || p->algo == LBM_NPOL || p->algo == LBM_NSOL) ? 1 : 0;
    if (p->algo == LBM_AA && (!offsets_fit(p, (int64_t)N) || (p->flags & LBM_FLAG_WIDE_OFFSETS)))
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

uint64_t magic(uint64_t d) { return d <= 1 ? 0ull : (~0ull / d) + 1ull; }

// Element offsets of the kernels' 32-bit tables: own slot, bounced pull and
// interior pull plus the largest periodic-face correction, per direction.
bool offsets_fit(const lbm3_params *p, int64_t N) {
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

}  // namespace

struct lbm3_lattice {
    lbm3_params p;
    Plan3 pl;
    char *ws;
    cudaStream_t stream, cap;
    int cur;
    int64_t steps;
    int64_t fluid;
    int block_1d;
    int off32;   // 32-bit offset tables usable (19 N and the pull shifts fit 31 bits)
    cudaGraphExec_t graph[2];
};

template <class S>
static Step3<S> make3(const lbm3_lattice *L, int src, int toff, int mom) {
    using C = typename Codec<S>::C;
    Step3<S> a;
    const lbm3_params &p = L->p;
    a.g = Geo3{p.nx, p.ny, p.nz, p.bc_x, p.bc_y, p.bc_z, east_kind(&p)};
    a.xlo_corr = p.bc_x == LBM_BC_PERIODIC ? p.nx : (p.bc_x == LBM_BC_OUTFLOW_ZG ? 1 : 0);
    a.xhi_corr = a.g.bxe == LBM_BC_PERIODIC ? -p.nx : (a.g.bxe == LBM_BC_OUTFLOW_ZG ? -1 : 0);
    a.inlet = p.bc_x == LBM_BC_INLET_EQ ? 1 : (p.bc_x == LBM_BC_INLET_ZOUHE ? 2 : 0);
    a.outlet = (inlet_kind(p.bc_x) && p.bc_x_east == LBM_BC_OUTLET_PRESSURE) ? 1 : 0;
    a.rev = p.algo == LBM_NSOL ? 1 : 0;
    {
        const double U[3] = {p.u_in[0], p.u_in[1], p.u_in[2]};
        a.zh[0] = (C)(U[0] / 3.0);
        a.zh[1] = (C)((U[0] + U[1]) / 6.0);
        a.zh[2] = (C)((U[0] - U[1]) / 6.0);
        a.zh[3] = (C)((U[0] + U[2]) / 6.0);
        a.zh[4] = (C)((U[0] - U[2]) / 6.0);
        a.zh[5] = (C)(-U[1] / 3.0);
        a.zh[6] = (C)(-U[2] / 3.0);
        a.zh[7] = (C)(p.rho_out - 1.0);
    }
    {
        const double usq = p.u_in[0] * p.u_in[0] + p.u_in[1] * p.u_in[1] + p.u_in[2] * p.u_in[2];
        for (int i = 0; i < Q; ++i) {
            const double w = d3::sq(i) == 0 ? 1.0 / 3.0 : (d3::sq(i) == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
            const double cu = d3::cx(i) * p.u_in[0] + d3::cy(i) * p.u_in[1] + d3::cz(i) * p.u_in[2];
            a.heq_in[i] = (C)(w * (3.0 * cu + 4.5 * cu * cu - 1.5 * usq));
        }
    }
    a.N = (uint32_t)L->pl.N;
    const double om = 1.0 / p.tau, kf = 1.0 - 0.5 * om;
    a.k.omega = (C)om;
    for (int d = 0; d < 3; ++d) {
        a.k.hf[d] = (C)(0.5 * p.force[d]);
        a.k.f[d] = (C)p.force[d];
    }
    a.k.w0 = (C)(1.0 / 3.0);
    a.k.w1 = (C)(1.0 / 18.0);
    a.k.w2 = (C)(1.0 / 36.0);
    a.k.wl0 = (C)(1.0 / 3.0 - (double)a.k.w0);
    a.k.wl1 = (C)(1.0 / 18.0 - (double)a.k.w1);
    a.k.wl2 = (C)(1.0 / 36.0 - (double)a.k.w2);
    a.k.kw0 = (C)(kf / 3.0);
    a.k.kw1 = (C)(kf / 18.0);
    a.k.kw2 = (C)(kf / 36.0);
    a.k.force = (p.force[0] != 0.0 || p.force[1] != 0.0 || p.force[2] != 0.0) ? 1 : 0;
    for (int i = 0; i < Q; ++i)
        a.k.cF[i] = (C)(d3::cx(i) * p.force[0] + d3::cy(i) * p.force[1] + d3::cz(i) * p.force[2]);
    {
        const int64_t N = L->pl.N, nx = p.nx, nxy = (int64_t)p.nx * p.ny;
        for (int i = 0; i < Q; ++i) {
            const int64_t d = d3::cz(i) * nxy + d3::cy(i) * nx + d3::cx(i);   // node shift of the pull
            int64_t self, mul;
            if (p.layout == LBM_LAYOUT_STREAM) { self = i * N; mul = 1; }
            else if (p.layout == LBM_LAYOUT_COLLISION) { self = i; mul = 19; }
            else { self = bundle_first(i) * N + (i - bundle_first(i)); mul = bundle_size(i); }
            const int j = d3::opp(i);
            const int64_t selfj = p.layout == LBM_LAYOUT_STREAM ? j * N
                                : p.layout == LBM_LAYOUT_COLLISION ? j
                                : bundle_first(j) * N + (j - bundle_first(j));
            a.os[i] = (int32_t)self;
            a.op[i] = (int32_t)(self - mul * d);
            a.ob[i] = (int32_t)selfj;
            a.oq[i] = (int32_t)(selfj + mul * d);
        }
    }
    a.links = (const uint32_t *)(L->ws + L->pl.links);
    a.src = (const S *)(L->ws + L->pl.pop[L->pl.one ? 0 : src]);
    a.dst = (S *)(L->ws + L->pl.pop[L->pl.one ? 0 : src ^ 1]);
    a.mom = mom ? (C *)(L->ws + L->pl.mom) : nullptr;
    a.err = (unsigned int *)(L->ws + L->pl.misc);
    a.tctr = (const long long *)(L->ws + L->pl.misc + 64);
    a.toff = toff;
    a.sr = p.rounding;
    a.seed = p.seed;
    a.tx = L->pl.tx;
    a.ty = L->pl.ty;
    a.tz = L->pl.tz;
    a.nx_magic = magic((uint64_t)p.nx);
    a.nxy_magic = magic((uint64_t)p.nx * (uint64_t)p.ny);
    // measured: +7 % for the stream layout on a porous box, -3 % for the bundle layout
    a.zero_fill = (p.layout != LBM_LAYOUT_BUNDLE && (p.algo == LBM_LPTL || L->pl.tx % 32 == 0)) ? 1 : 0;
    return a;
}

#define LBM3_DISPATCH(L_, ...)                                                                  \
    switch ((L_)->p.storage) {                                                                   \
        case LBM_F64: { using S = double; __VA_ARGS__; break; }                                         \
        case LBM_F32: { using S = float; __VA_ARGS__; break; }                                          \
        case LBM_F16S: { using S = __half; __VA_ARGS__; break; }                                        \
        default: { using S = __nv_bfloat16; __VA_ARGS__; break; }                                       \
    }

template <class S, bool LINEAR, bool OFF32>
static void launch3k(const lbm3_lattice *L, const Step3<S> &a, dim3 grid, dim3 block, cudaStream_t st) {
    const int lay = L->p.layout;
    if (lay == LBM_LAYOUT_STREAM) k3_step<S, STREAM, LINEAR, OFF32><<<grid, block, 0, st>>>(a);
    else if (lay == LBM_LAYOUT_BUNDLE) k3_step<S, BUNDLE, LINEAR, OFF32><<<grid, block, 0, st>>>(a);
    else k3_step<S, COLLISION, LINEAR, OFF32><<<grid, block, 0, st>>>(a);
}

template <class S, int PHASE>
static void launch_aa(const lbm3_lattice *L, const Step3<S> &a, cudaStream_t st) {
    const dim3 g(L->pl.ntx, L->pl.nty, L->pl.ntz), b(L->pl.tx, L->pl.ty, L->pl.tz);
    const int lay = L->p.layout;
    if (lay == LBM_LAYOUT_STREAM) k3_aa<S, STREAM, PHASE><<<g, b, 0, st>>>(a);
    else if (lay == LBM_LAYOUT_BUNDLE) k3_aa<S, BUNDLE, PHASE><<<g, b, 0, st>>>(a);
    else k3_aa<S, COLLISION, PHASE><<<g, b, 0, st>>>(a);
}

template <class S>
static S *halo_parity(const lbm3_lattice *L, int parity) {
    return (S *)(L->ws + L->pl.halo) + (int64_t)parity * L->pl.halo_parity;
}

template <class S, bool OFF32>
static void launch_npol(const lbm3_lattice *L, const Step3<S> &a, int parity, cudaStream_t st) {
    const dim3 g(L->pl.ntx, L->pl.nty, L->pl.ntz), b(L->pl.tx, L->pl.ty, L->pl.tz);
    const S *hr = halo_parity<S>(L, parity);
    S *hw = halo_parity<S>(L, parity ^ 1);
    const int lay = L->p.layout;
    if (lay == LBM_LAYOUT_STREAM) k3_npol<S, STREAM, OFF32><<<g, b, 0, st>>>(a, hr, hw);
    else if (lay == LBM_LAYOUT_BUNDLE) k3_npol<S, BUNDLE, OFF32><<<g, b, 0, st>>>(a, hr, hw);
    else k3_npol<S, COLLISION, OFF32><<<g, b, 0, st>>>(a, hr, hw);
}

template <class S>
static void launch_nsol(const lbm3_lattice *L, const Step3<S> &a, int parity, cudaStream_t st) {
    const dim3 g(L->pl.ntx, L->pl.nty, L->pl.ntz), b(L->pl.tx, L->pl.ty, L->pl.tz);
    const size_t sm = nsol3_smem_bytes<S>(L->pl.tx, L->pl.ty, L->pl.tz);
    const S *hr = halo_parity<S>(L, parity);
    S *hw = halo_parity<S>(L, parity ^ 1);
    const int lay = L->p.layout;
    if (lay == LBM_LAYOUT_STREAM) k3_nsol<S, STREAM><<<g, b, sm, st>>>(a, hr, hw);
    else if (lay == LBM_LAYOUT_BUNDLE) k3_nsol<S, BUNDLE><<<g, b, sm, st>>>(a, hr, hw);
    else k3_nsol<S, COLLISION><<<g, b, sm, st>>>(a, hr, hw);
}

// Largest staged tile of the 3-D NSOL kernel (512 nodes) beyond the default
// 48 KB of dynamic shared memory (FP64: 76 KB).
template <class S>
static void nsol3_prepare() {
    static const bool done = [] {
        const int bytes = (int)nsol3_smem_bytes<S>(512, 1, 1);
        cudaFuncSetAttribute(k3_nsol<S, STREAM>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        cudaFuncSetAttribute(k3_nsol<S, BUNDLE>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        cudaFuncSetAttribute(k3_nsol<S, COLLISION>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        cudaGetLastError();
        return true;
    }();
    (void)done;
}

// NPOL: fill buffer-grid parity `parity` from the stored state.
template <class S>
static cudaError_t publish_state(const lbm3_lattice *L, int parity, cudaStream_t st) {
    const Step3<S> a = make3<S>(L, 0, 0, 0);
    const dim3 g(L->pl.ntx, L->pl.nty, L->pl.ntz), b(L->pl.tx, L->pl.ty, L->pl.tz);
    S *hw = halo_parity<S>(L, parity);
    const int lay = L->p.layout;
    if (lay == LBM_LAYOUT_STREAM) k3_publish<S, STREAM><<<g, b, 0, st>>>(a, hw);
    else if (lay == LBM_LAYOUT_BUNDLE) k3_publish<S, BUNDLE><<<g, b, 0, st>>>(a, hw);
    else k3_publish<S, COLLISION><<<g, b, 0, st>>>(a, hw);
    return cudaGetLastError();
}

// src: the update's parity (two lattices: the source lattice; AA: the phase;
// NPOL: the buffer-grid parity read).
template <class S>
static cudaError_t step3(const lbm3_lattice *L, cudaStream_t st, int src, int toff, int mom) {
    const Step3<S> a = make3<S>(L, src, toff, mom);
    if (L->p.algo == LBM_NPOL) {
        if (L->off32) launch_npol<S, true>(L, a, src, st);
        else launch_npol<S, false>(L, a, src, st);
    } else if (L->p.algo == LBM_NSOL) {
        launch_nsol<S>(L, a, src, st);
    } else if (L->p.algo == LBM_AA) {
        if (src == 0) launch_aa<S, 0>(L, a, st);
        else launch_aa<S, 1>(L, a, st);
    } else if (L->p.algo == LBM_LPTL) {
        const dim3 g((unsigned)((L->pl.N + L->block_1d - 1) / L->block_1d)), b(L->block_1d);
        if (L->off32) launch3k<S, true, true>(L, a, g, b, st);
        else launch3k<S, true, false>(L, a, g, b, st);
    } else {
        const dim3 g(L->pl.ntx, L->pl.nty, L->pl.ntz), b(L->pl.tx, L->pl.ty, L->pl.tz);
        if (L->off32) launch3k<S, false, true>(L, a, g, b, st);
        else launch3k<S, false, false>(L, a, g, b, st);
    }
    return cudaGetLastError();
}

static cudaError_t launch3(lbm3_lattice *L, cudaStream_t st, int64_t count, int want_moments) {
    int cur = L->cur;
    for (int64_t k = 0; k < count; ++k) {
        cudaError_t e = cudaSuccess;
        const int mom = (want_moments && k == count - 1) ? 1 : 0;
        LBM3_DISPATCH(L, e = step3<S>(L, st, cur, (int)k, mom));
        if (e != cudaSuccess) return e;
        cur ^= 1;
    }
    return launch_bump_counter((long long *)(L->ws + L->pl.misc + 64), count, st);
}

#define CK3(call)                                                 \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return lbm_cuda_fail(e_, #call);   \
    } while (0)

extern "C" lbm_status lbm3_workspace_bytes(const lbm3_params *p, size_t *bytes) {
    if (!bytes) return lbm_fail(LBM_EINVAL, "bytes is NULL");
    Plan3 pl;
    lbm_status s = plan3(p, &pl);
    if (s == LBM_OK) *bytes = pl.total;
    return s;
}

extern "C" int64_t lbm3_layout_index(int32_t layout, int64_t N, int64_t n, int32_t i) {
    if (layout < 0 || layout > 2 || N < 1 || n < 0 || n >= N || i < 0 || i > 18) return -1;
    if (layout == LBM_LAYOUT_STREAM) return d3::addr<STREAM>(N, n, i);
    if (layout == LBM_LAYOUT_BUNDLE) return d3::addr<BUNDLE>(N, n, i);
    return d3::addr<COLLISION>(N, n, i);
}

template <class S>
static int block_of(int layout) {
    auto pick = [](const void *k) {
        int mg = 0, b = 256;
        if (cudaOccupancyMaxPotentialBlockSize(&mg, &b, k, 0, 512) != cudaSuccess) {
            cudaGetLastError();
            b = 256;
        }
        return b;
    };
    if (layout == LBM_LAYOUT_STREAM) return pick((const void *)k3_step<S, STREAM, true, true>);
    if (layout == LBM_LAYOUT_BUNDLE) return pick((const void *)k3_step<S, BUNDLE, true, true>);
    return pick((const void *)k3_step<S, COLLISION, true, true>);
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
            const unsigned g = (unsigned)((c + 255) / 256);
            LBM3_DISPATCH(L, {
                const Step3<S> a = make3<S>(L, 1, 0, 0);   // dst = lattice 0
                if (L->p.layout == LBM_LAYOUT_STREAM)
                    k3_init<S, STREAM><<<g, 256, 0, st>>>(a, dv[0], dv[1], dv[2], dv[3], (uint32_t)n0, (uint32_t)c);
                else if (L->p.layout == LBM_LAYOUT_BUNDLE)
                    k3_init<S, BUNDLE><<<g, 256, 0, st>>>(a, dv[0], dv[1], dv[2], dv[3], (uint32_t)n0, (uint32_t)c);
                else
                    k3_init<S, COLLISION><<<g, 256, 0, st>>>(a, dv[0], dv[1], dv[2], dv[3], (uint32_t)n0, (uint32_t)c);
            });
            CK3(cudaGetLastError());
            CK3(cudaStreamSynchronize(st));
        }
    }
    const unsigned g = (unsigned)((pl.N + 255) / 256);
    LBM3_DISPATCH(L, {
        Step3<S> a = make3<S>(L, 0, 0, 1);
        if (L->p.layout == LBM_LAYOUT_STREAM) k3_state_moments<S, STREAM><<<g, 256, 0, st>>>(a);
        else if (L->p.layout == LBM_LAYOUT_BUNDLE) k3_state_moments<S, BUNDLE><<<g, 256, 0, st>>>(a);
        else k3_state_moments<S, COLLISION><<<g, 256, 0, st>>>(a);
    });
    CK3(cudaGetLastError());
    if (pl.halo_parity) LBM3_DISPATCH(L, CK3(publish_state<S>(L, 0, st)));
    CK3(cudaStreamSynchronize(st));
    return LBM_OK;
}

extern "C" lbm_status lbm3_create(const lbm3_params *p, const uint8_t *mask_host, void *d_workspace,
                                  size_t bytes, void *cuda_stream, lbm3_lattice **out) {
    if (!out) return lbm_fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    Plan3 pl;
    lbm_status s = plan3(p, &pl);
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
    LBM3_DISPATCH(L, L->block_1d = block_of<S>(p->layout));
    if (p->algo == LBM_NSOL) LBM3_DISPATCH(L, nsol3_prepare<S>());
    L->off32 = (offsets_fit(p, pl.N) && !(p->flags & LBM_FLAG_WIDE_OFFSETS)) ? 1 : 0;
    cudaError_t e = cudaStreamCreateWithFlags(&L->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete L;
        return lbm_cuda_fail(e, "cudaStreamCreateWithFlags");
    }
    uint8_t *dmask = (uint8_t *)(L->ws + pl.mom);   // staged in the moments region (>= N bytes)
    unsigned long long *dcount = (unsigned long long *)(L->ws + pl.partials);
    unsigned long long fluid = 0;
    const Geo3 g{p->nx, p->ny, p->nz, p->bc_x, p->bc_y, p->bc_z, east_kind(p)};
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

static lbm_status check3(lbm3_lattice *L) {
    unsigned int flag = 0;
    CK3(cudaMemcpy(&flag, L->ws + L->pl.misc, sizeof(flag), cudaMemcpyDeviceToHost));
    if (flag) {
        CK3(cudaMemset(L->ws + L->pl.misc, 0, sizeof(flag)));
        return lbm_fail(LBM_EDIVERGED, "non-finite density after %lld updates", (long long)L->steps);
    }
    return LBM_OK;
}

extern "C" lbm_status lbm3_sync(lbm3_lattice *L) {
    if (!L) return lbm_fail(LBM_EINVAL, "lattice is NULL");
    CK3(cudaStreamSynchronize(L->stream));
    return check3(L);
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
    return check3(L);
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
    return check3(L);
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
        LBM3_DISPATCH(L, CK3(publish_state<S>(L, L->cur, L->stream)));
        CK3(cudaStreamSynchronize(L->stream));
    }
    return LBM_OK;
}

extern "C" lbm_status lbm3_mass(lbm3_lattice *L, double *out) {
    if (!L || !out) return lbm_fail(LBM_EINVAL, "NULL argument");
    if (state_readable(L) != LBM_OK) return LBM_EINVAL;
    double *partials = (double *)(L->ws + L->pl.partials);
    LBM3_DISPATCH(L, {
        const Step3<S> a = make3<S>(L, L->cur, 0, 0);
        if (L->p.layout == LBM_LAYOUT_STREAM) k3_mass<S, STREAM><<<kReduceBlocks, kReduceThreads, 0, L->stream>>>(a, partials);
        else if (L->p.layout == LBM_LAYOUT_BUNDLE) k3_mass<S, BUNDLE><<<kReduceBlocks, kReduceThreads, 0, L->stream>>>(a, partials);
        else k3_mass<S, COLLISION><<<kReduceBlocks, kReduceThreads, 0, L->stream>>>(a, partials);
    });
    CK3(cudaGetLastError());
    k3_sum<<<1, 32, 0, L->stream>>>(partials, kReduceBlocks, partials + kReduceBlocks);
    CK3(cudaGetLastError());
    CK3(cudaMemcpyAsync(out, partials + kReduceBlocks, sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    CK3(cudaStreamSynchronize(L->stream));
    return check3(L);
}

extern "C" lbm_status lbm3_force(lbm3_lattice *L, const uint8_t *d_body, double out[3]) {
    if (!L || !out) return lbm_fail(LBM_EINVAL, "NULL argument");
    if (state_readable(L) != LBM_OK) return LBM_EINVAL;
    double *partials = (double *)(L->ws + L->pl.partials);
    LBM3_DISPATCH(L, {
        const Step3<S> a = make3<S>(L, L->cur, 0, 0);
        if (L->p.layout == LBM_LAYOUT_STREAM) k3_force<S, STREAM><<<kReduceBlocks, kReduceThreads, 0, L->stream>>>(a, d_body, partials);
        else if (L->p.layout == LBM_LAYOUT_BUNDLE) k3_force<S, BUNDLE><<<kReduceBlocks, kReduceThreads, 0, L->stream>>>(a, d_body, partials);
        else k3_force<S, COLLISION><<<kReduceBlocks, kReduceThreads, 0, L->stream>>>(a, d_body, partials);
    });
    CK3(cudaGetLastError());
    k3_sum3<<<1, 32, 0, L->stream>>>(partials, kReduceBlocks, partials + 3 * kReduceBlocks);
    CK3(cudaGetLastError());
    CK3(cudaMemcpyAsync(out, partials + 3 * kReduceBlocks, 3 * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    CK3(cudaStreamSynchronize(L->stream));
    return check3(L);
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
    out->aux = L->off32 ? 0 : 1;   // 1: the 64-bit addressing path
    return LBM_OK;
}
