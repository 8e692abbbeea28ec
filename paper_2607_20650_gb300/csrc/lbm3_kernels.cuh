// D3Q19 device code (the paper's 3-D future work, Sec. 6) with the method of
// Sec. 3.1: two-lattice pull (LPTL: one node per thread over n; NPTL: 3-D
// tiles), the one-lattice NPOL pull and NSOL swap of Sec. 3.3 (tiles and a
// buffer grid), the one-lattice AA pattern (named in Sec. 3.3, future work in
// Sec. 6), the three layouts generalised (stream, bundle = directions sharing
// a source row, collision), periodic or half-way wall faces, equilibrium or
// Zou-He inlet, zero-gradient outflow or Zou-He pressure outlet on x,
// bounce-back at solid nodes, Guo force, FP64/FP32/FP16/BF16 shifted
// storage, on-the-fly moments, FP64 mass and momentum-exchange force, and
// the batched form. Templates only: each storage type is instantiated in its
// own translation unit (lbm3_ops_*.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "lbm.h"
#include "lbm3_device.cuh"
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
    Consts3x2 k2;   // FP32 arithmetic: k duplicated for the packed node pairs
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

// (x, y, z) of node n.
template <class S>
__device__ __forceinline__ void node_xyz(const Step3<S> &a, uint32_t n, uint32_t &x, uint32_t &y, uint32_t &z) {
    const uint32_t nx = (uint32_t)a.g.nx, ny = (uint32_t)a.g.ny;
    z = fdiv(n, a.nxy_magic);
    const uint32_t r = n - z * nx * ny;
    y = fdiv(r, a.nx_magic);
    x = r - y * nx;
}

// One node of the two-lattice update (LPTL, NPTL) at (x, y, z) in the box.
// OFF32: the offset tables fit 31 bits; every pull uses them (periodic wrap
// as node-index corrections); otherwise 64-bit addressing with the general
// edge mapping for nodes on the box faces.
template <class S, int L, bool OFF32>
__device__ __forceinline__ void step3_node(const Step3<S> &a, uint32_t x, uint32_t y, uint32_t z) {
    using C = typename Codec<S>::C;
    const uint32_t nx = (uint32_t)a.g.nx, ny = (uint32_t)a.g.ny;
    const uint32_t n = (z * ny + y) * nx + x;
    const uint32_t lk = a.links[n];
    const bool f = lk != SOLID;
    if (a.zero_fill) {
        const int lane = (int)(((threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x) & 31u);
        const unsigned F = __ballot_sync(__activemask(), f);
        if (!f && shares3<S, L>(F, lane)) zero3<S, L>(a, n);
    }
    if (!f) return;
    C g[Q];
    pull3<S, L, OFF32>(a, x, y, z, n, lk, g);
    faces3(a, x, g);
    finish3<S, L, OFF32>(a, n, g);
}

// LINEAR: one node per thread over n (LPTL); otherwise 3-D tiles (NPTL).
template <class S, int L, bool LINEAR, bool OFF32>
__global__ void __launch_bounds__(512, sizeof(S) == 8 ? 2 : 3) k3_step(const Step3<S> a) {
    uint32_t x, y, z;
    if (LINEAR) {
        const uint64_t n64 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (n64 >= a.N) return;
        node_xyz(a, (uint32_t)n64, x, y, z);
    } else {
        x = blockIdx.x * a.tx + threadIdx.x;
        y = blockIdx.y * a.ty + threadIdx.y;
        z = blockIdx.z * a.tz + threadIdx.z;
        if (x >= (uint32_t)a.g.nx || y >= (uint32_t)a.g.ny || z >= (uint32_t)a.g.nz) return;
    }
    step3_node<S, L, OFF32>(a, x, y, z);
}

// Node pairs: two x-adjacent nodes (x even) per thread for 16-bit storage,
// each pulled as step3_node pulls it, the collision on packed FP32 pairs
// (collide3_2, bit-identical to collide3 lane by lane) and two values rounded
// per conversion, node a in the low half and node b in the high half of each
// 32-bit word. A solid partner's lane holds +0, which is what a solid node
// stores, so its words are written whole.
template <class S>
__device__ __forceinline__ uint32_t pack3_rne(float lo, float hi) {
    uint32_t r;
    if constexpr (std::is_same<S, __half>::value)
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    else
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// The words of nodes n, n + 1 (n even, N even): stream layout one word per
// direction; bundle layout one word per single-direction bundle and three per
// three-direction bundle (the six values a0 a1 a2 b0 b1 b2 are adjacent).
template <class S, int L>
__device__ __forceinline__ void store3_pair(S *dst, uint32_t N, uint32_t n, const uint32_t *w) {
    if (L == STREAM) {
#pragma unroll
        for (int i = 0; i < Q; ++i) *reinterpret_cast<uint32_t *>(dst + (uint32_t)i * N + n) = w[i];
        return;
    }
#pragma unroll
    for (int f = 0; f < Q; ++f) {
        if (bundle_first(f) != f) continue;
        if (bundle_size(f) == 1) {
            *reinterpret_cast<uint32_t *>(dst + (uint32_t)f * N + n) = w[f];
        } else {
            uint32_t *q = reinterpret_cast<uint32_t *>(dst + (uint32_t)f * N + 3u * n);
            q[0] = (w[f] & 0xFFFFu) | (w[f + 1] << 16);
            q[1] = (w[f + 2] & 0xFFFFu) | (w[f] & 0xFFFF0000u);
            q[2] = (w[f + 1] >> 16) | (w[f + 2] & 0xFFFF0000u);
        }
    }
}

// Pulls of a pair (pull3 of both nodes, direction by direction, into packed
// pairs): node a = (x, y, z) with x even, node b = (x + 1, y, z); only node a
// can lie on the west face and only node b on the east one. A solid node's
// lane is +0.
template <class S, int L>
__device__ __forceinline__ void pull3_pair(const Step3<S> &a, uint32_t x, uint32_t y, uint32_t z, uint32_t n,
                                           uint32_t lka, uint32_t lkb, bool fa, bool fb, f2 *g) {
    const uint32_t nx = (uint32_t)a.g.nx, ny = (uint32_t)a.g.ny, nz = (uint32_t)a.g.nz;
    const S *__restrict__ src = a.src;
    const int N = (int)a.N, nxy = (int)(nx * ny);
    const int xlo = x == 0 ? a.xlo_corr : 0, xhi = x + 1u == nx - 1 ? a.xhi_corr : 0;
    const int ylo = y == 0 ? nxy : 0, yhi = y == ny - 1 ? -nxy : 0;
    const int zlo = z == 0 ? N : 0, zhi = z == nz - 1 ? -N : 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const S *ba = src + mult3<L>(i) * n, *bb = ba + mult3<L>(i);
        int oa, ob;
        if (i == REST) {
            oa = ob = a.os[i];
        } else {
            const int wyz = (cy(i) > 0 ? ylo : cy(i) < 0 ? yhi : 0) + (cz(i) > 0 ? zlo : cz(i) < 0 ? zhi : 0);
            const int wa = (cx(i) > 0 ? xlo : 0) + wyz, wb = (cx(i) < 0 ? xhi : 0) + wyz;
            oa = ((lka >> bit(i)) & 1u) ? a.ob[i] : a.op[i] + (int)mult3<L>(i) * wa;
            ob = ((lkb >> bit(i)) & 1u) ? a.ob[i] : a.op[i] + (int)mult3<L>(i) * wb;
        }
        const float va = fa ? Codec<S>::dec(ba[oa]) : 0.0f;
        const float vb = fb ? Codec<S>::dec(bb[ob]) : 0.0f;
        g[i] = pk2(va, vb);
    }
}

template <class S, int L>
__device__ __forceinline__ void step3_pair(const Step3<S> &a, uint32_t x, uint32_t y, uint32_t z, uint32_t n) {
    const uint2 lk2 = *reinterpret_cast<const uint2 *>(a.links + n);   // n even: 8-byte aligned
    const bool fa = lk2.x != SOLID, fb = lk2.y != SOLID;
    if (!fa && !fb) return;
    f2 g[Q];
    pull3_pair<S, L>(a, x, y, z, n, lk2.x, lk2.y, fa, fb, g);
    // inlet / outlet planes (x = 0 holds node a, x = nx - 1 node b): the
    // substitutions of one node, on its lane
    const bool west = a.inlet && x == 0 && fa, east = a.outlet && x + 1u == (uint32_t)a.g.nx - 1 && fb;
    if (west || east) {
        float ga[Q], gb[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) up2(g[i], ga[i], gb[i]);
        if (west) faces3(a, x, ga);
        if (east) faces3(a, x + 1u, gb);
#pragma unroll
        for (int i = 0; i < Q; ++i) g[i] = pk2(ga[i], gb[i]);
    }
    f2 drho, ux, uy, uz;
    collide3_2(a.k2, a.k.force, g, drho, ux, uy, uz);
    float da, db;
    up2(drho, da, db);
    if ((fa && !isfinite(da)) || (fb && !isfinite(db))) atomicOr(a.err, 1u);
    if (a.mom) {
        float r[2], u[3][2];
        up2(add2(dup2(1.0f), drho), r[0], r[1]);
        up2(ux, u[0][0], u[0][1]);
        up2(uy, u[1][0], u[1][1]);
        up2(uz, u[2][0], u[2][1]);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (!(k ? fb : fa)) continue;
            a.mom[n + k] = r[k];
            a.mom[a.N + n + k] = u[0][k];
            a.mom[2 * (size_t)a.N + n + k] = u[1][k];
            a.mom[3 * (size_t)a.N + n + k] = u[2][k];
        }
    }
    uint32_t w[Q];
    if (!a.sr) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float lo, hi;
            up2(g[i], lo, hi);
            w[i] = pack3_rne<S>(fa ? lo : 0.0f, fb ? hi : 0.0f);
        }
    } else {
        const uint32_t sk = step_key(a.seed, (uint32_t)(*a.tctr + a.toff));
        const uint32_t nka = node_key(sk, n), nkb = node_key(sk, n + 1u);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float lo, hi;
            up2(g[i], lo, hi);
            lo = fa ? lo : 0.0f;
            hi = fb ? hi : 0.0f;
            if constexpr (std::is_same<S, __half>::value)
                w[i] = sr_half2(hi, lo, pop_rand(nkb, i), pop_rand(nka, i));
            else
                w[i] = sr_bf162(hi, lo, pop_rand(nkb, i), pop_rand(nka, i));
        }
    }
    store3_pair<S, L>(a.dst, a.N, n, w);
}

#ifndef LBM3_PAIR_MINB
#define LBM3_PAIR_MINB 4
#endif
// LINEAR: pairs over n (LPTL, 2 x blockDim nodes per block); otherwise tiles
// of tx x ty x tz nodes with blocks of tx/2 x ty x tz threads (NPTL).
template <class S, int L, bool LINEAR>
__global__ void __launch_bounds__(256, LBM3_PAIR_MINB) k3_step_pair(const Step3<S> a) {
    uint32_t x, y, z, n;
    if (LINEAR) {
        const uint64_t n64 = 2ull * ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x);
        if (n64 >= a.N) return;
        n = (uint32_t)n64;
        node_xyz(a, n, x, y, z);
    } else {
        x = blockIdx.x * a.tx + 2u * threadIdx.x;
        y = blockIdx.y * a.ty + threadIdx.y;
        z = blockIdx.z * a.tz + threadIdx.z;
        if (x >= (uint32_t)a.g.nx || y >= (uint32_t)a.g.ny || z >= (uint32_t)a.g.nz) return;
        n = (z * (uint32_t)a.g.ny + y) * (uint32_t)a.g.nx + x;
    }
    step3_pair<S, L>(a, x, y, z, n);
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
// Tile b (of nt per axis) of the update.
template <class S, int L, bool OFF32>
__device__ __forceinline__ void npol3_tile(const Step3<S> &a, const S *hr, S *hw, const int *b, const int *nt) {
    using C = typename Codec<S>::C;
    using A = Ar<C>;
    const Tile3 T{a.tx, a.ty, a.tz};
    const int ext[3] = {a.g.nx, a.g.ny, a.g.nz};
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

template <class S, int L, bool OFF32>
__global__ void __launch_bounds__(512, sizeof(S) == 8 ? 1 : 2) k3_npol(const Step3<S> a, const S *hr, S *hw) {
    const int b[3] = {(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z};
    const int nt[3] = {(int)gridDim.x, (int)gridDim.y, (int)gridDim.z};
    npol3_tile<S, L, OFF32>(a, hr, hw, b, nt);
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

// Tile b (of nt per axis) of the update; sm: the tile's 19 staged planes.
template <class S, int L>
__device__ __forceinline__ void nsol3_tile(const Step3<S> &a, const S *hr, S *hw, const int *b, const int *nt,
                                           typename Codec<S>::C *sm) {
    using C = typename Codec<S>::C;
    using A = Ar<C>;
    const Tile3 T{a.tx, a.ty, a.tz};
    const int TN = a.tx * a.ty * a.tz;
    const int ext[3] = {a.g.nx, a.g.ny, a.g.nz};
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

template <class S, int L>
__global__ void __launch_bounds__(512, sizeof(S) == 8 ? 1 : 2) k3_nsol(const Step3<S> a, const S *hr, S *hw) {
    extern __shared__ __align__(16) unsigned char smem_nsol3[];
    const int b[3] = {(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z};
    const int nt[3] = {(int)gridDim.x, (int)gridDim.y, (int)gridDim.z};
    nsol3_tile<S, L>(a, hr, hw, b, nt, reinterpret_cast<typename Codec<S>::C *>(smem_nsol3));
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

// ------------------------------------------------------------ batches (3-D)
// Many independent boxes advanced by one launch per update. Every case has a
// record with its kernel arguments for both update parities; the work list
// holds (case, local item) pairs, an item being one tile (NPTL, NPOL, NSOL)
// or one block of consecutive nodes (LPTL). A block copies its case's
// arguments into shared memory and runs the single-lattice code on its item,
// so each case's results are those of a single-lattice run bit for bit.
template <class S>
struct Case3 {
    Step3<S> a[2];               // source lattice (two lattices) or buffer-grid parity 0 / 1
    S *halo[2];                  // buffer-grid parities (NPOL, NSOL; else null)
    typename Codec<S>::C *mom;   // moments array of the case
    int nt[3];                   // tiles per axis
    int pad;
};

// Register budget: threads per block and resident blocks. The arguments are
// read from shared memory here, which takes registers: the single-box bound
// (three 512-thread blocks, 40 registers) made the two-lattice body spill
// about 200 bytes. LPTL items are 256 nodes: five blocks (48 registers, a
// few spilled bytes) measured 6 % faster than four (64).
__host__ __device__ constexpr int batch3_threads(int algo) { return algo == LBM_LPTL ? 256 : 512; }
__host__ __device__ constexpr int batch3_min_blocks(int algo, int elem) {
    return algo == LBM_LPTL ? 5 : (algo == LBM_NPTL ? 2 : (elem == 8 ? 1 : 2));
}

// src: update parity; toff: offset added to the update counter (stochastic
// rounding keys); mom: store the moments.
template <class S, int L, int ALGO, bool OFF32>
__global__ void __launch_bounds__(batch3_threads(ALGO), batch3_min_blocks(ALGO, sizeof(S)))
    k3_batch(const Case3<S> *cases, const uint2 *items, int src, int toff, int mom) {
    __shared__ __align__(16) unsigned char raw[sizeof(Step3<S>)];
    Step3<S> &a = *reinterpret_cast<Step3<S> *>(raw);
    const uint2 it = items[blockIdx.x];
    const Case3<S> &cs = cases[it.x];
    const int tid = (int)((threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x);
    const int nth = (int)(blockDim.x * blockDim.y * blockDim.z);
    {
        const uint32_t *from = reinterpret_cast<const uint32_t *>(&cs.a[src]);
        uint32_t *to = reinterpret_cast<uint32_t *>(raw);
        for (int k = tid; k < (int)(sizeof(Step3<S>) / 4); k += nth) to[k] = from[k];
    }
    __syncthreads();
    if (tid == 0) {
        a.toff = toff;
        a.mom = mom ? cs.mom : nullptr;
    }
    __syncthreads();
    if (ALGO == LBM_LPTL) {
        const uint64_t n64 = (uint64_t)it.y * (uint64_t)nth + (uint64_t)tid;
        if (n64 >= a.N) return;
        uint32_t x, y, z;
        node_xyz(a, (uint32_t)n64, x, y, z);
        step3_node<S, L, OFF32>(a, x, y, z);
        return;
    }
    const int nt[3] = {cs.nt[0], cs.nt[1], cs.nt[2]};
    const uint32_t t = it.y, txy = (uint32_t)nt[0] * (uint32_t)nt[1];
    const int b[3] = {(int)(t % (uint32_t)nt[0]), (int)((t % txy) / (uint32_t)nt[0]), (int)(t / txy)};
    if (ALGO == LBM_NPTL) {
        const uint32_t x = (uint32_t)b[0] * a.tx + threadIdx.x;
        const uint32_t y = (uint32_t)b[1] * a.ty + threadIdx.y;
        const uint32_t z = (uint32_t)b[2] * a.tz + threadIdx.z;
        if (x >= (uint32_t)a.g.nx || y >= (uint32_t)a.g.ny || z >= (uint32_t)a.g.nz) return;
        step3_node<S, L, OFF32>(a, x, y, z);
    } else if (ALGO == LBM_NPOL) {
        npol3_tile<S, L, OFF32>(a, cs.halo[src], cs.halo[src ^ 1], b, nt);
    } else {
        extern __shared__ __align__(16) unsigned char smem_batch3[];
        nsol3_tile<S, L>(a, cs.halo[src], cs.halo[src ^ 1], b, nt,
                         reinterpret_cast<typename Codec<S>::C *>(smem_batch3));
    }
}

}  // namespace d3
}  // namespace lbm
