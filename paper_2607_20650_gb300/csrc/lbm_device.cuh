// Device-side building blocks of the D2Q9I BGK update (PortLBM, Sec. 3):
// direction set, the three population layouts, storage codecs, the pull
// mapping at domain edges, and the one collision routine every kernel calls.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace lbm {

enum Layout : int { STREAM = 0, BUNDLE = 1, COLLISION = 2 };
enum Algo : int { LPTL = 0, NPTL = 1, NPOL = 2, NSOL = 3, AA = 4 };
enum Bc : int {
    PERIODIC = 0, WALL = 1, FREESLIP = 2, INLET_ZOUHE = 3, INLET_EQ = 4, OUTFLOW_ZG = 5,
    INLET_EQ_NEUMANN = 6, OUTLET_PRESSURE = 7
};
enum Pull : int { PULL_NODE = 0, PULL_BOUNCE = 1, PULL_UNKNOWN = 2 };

// Per-node link byte: bit b(i) set when the value pulled in direction i is
// bounced back (source solid or a wall edge); 0xFF marks a solid node.
constexpr uint8_t SOLID_LINKS = 0xFF;

// Fig. 2 order: i = 0..8 = SW, S, SE, W, rest, E, NW, N, NE.
__host__ __device__ constexpr int cx(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int cy(int i) { return i / 3 - 1; }
__host__ __device__ constexpr int opp(int i) { return 8 - i; }
__host__ __device__ constexpr int mir_y(int i) { return (i % 3) + 3 * (2 - i / 3); }
__host__ __device__ constexpr int link_bit(int i) { return i < 4 ? i : i - 1; }

// Layouts of Fig. 2 (element offsets, N nodes).
template <int L>
__host__ __device__ __forceinline__ int64_t addr(int64_t N, int64_t n, int i) {
    if (L == STREAM) return (int64_t)i * N + n;
    if (L == COLLISION) return n * 9 + i;
    return (int64_t)(i / 3) * 3 * N + n * 3 + (i % 3);
}

// ------------------------------------------------------------ arithmetic
// Explicitly rounded operations: no contraction or reassociation, so every
// kernel that calls collide() produces the same bits.
template <class C> struct Ar;
template <> struct Ar<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
};
template <> struct Ar<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
};

// ------------------------------------------------------------ hashing
// 32-bit integer finaliser "lowbias32" (C. Wellons, hash-prospector).
__host__ __device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}
__host__ __device__ __forceinline__ uint32_t step_key(uint64_t seed, uint32_t t) {
    return mix32((uint32_t)seed ^ mix32((uint32_t)(seed >> 32) ^ mix32(t)));
}
__host__ __device__ __forceinline__ uint32_t node_key(uint32_t skey, uint32_t n) {
    return mix32(n ^ skey);
}
__host__ __device__ __forceinline__ uint32_t pop_rand(uint32_t nkey, int i) {
    return mix32(nkey + (uint32_t)i * 0x9E3779B9U);
}

// ------------------------------------------------------------ codecs
// Stochastic rounding: with lo the value rounded toward zero and ulp the gap
// to the next magnitude, round away from zero iff u * ulp < |x| - |lo| for
// u = (r >> 8) * 2^-24. Every product and difference here is exact.
__device__ __forceinline__ __half sr_half(float x, uint32_t r) {
    __half lo = __float2half_rz(x);
    float alo = fabsf(__half2float(lo));
    float ax = fabsf(x);
    if (!(ax < 65504.0f) || ax == alo) return __float2half_rn(x);
    unsigned short mag = __half_as_ushort(lo) & 0x7FFFu;
    float ulp = __half2float(__ushort_as_half((unsigned short)(mag + 1))) - alo;
    float u = __fmul_rn(__fmul_rn((float)(r >> 8), ulp), 0x1p-24f);
    if (u < __fsub_rn(ax, alo)) mag = (unsigned short)(mag + 1);
    return __ushort_as_half((unsigned short)(mag | (x < 0.0f ? 0x8000u : 0u)));
}
__device__ __forceinline__ __nv_bfloat16 sr_bf16(float x, uint32_t r) {
    __nv_bfloat16 lo = __float2bfloat16_rz(x);
    float alo = fabsf(__bfloat162float(lo));
    float ax = fabsf(x);
    if (!(ax < 3.0e38f) || ax == alo) return __float2bfloat16_rn(x);
    unsigned short mag = __bfloat16_as_ushort(lo) & 0x7FFFu;
    float ulp = __bfloat162float(__ushort_as_bfloat16((unsigned short)(mag + 1))) - alo;
    float u = __fmul_rn(__fmul_rn((float)(r >> 8), ulp), 0x1p-24f);
    if (u < __fsub_rn(ax, alo)) mag = (unsigned short)(mag + 1);
    return __ushort_as_bfloat16((unsigned short)(mag | (x < 0.0f ? 0x8000u : 0u)));
}

template <class S> struct Codec;
template <> struct Codec<double> {
    using C = double;
    static constexpr bool narrow = false;
    static __device__ __forceinline__ double dec(double v) { return v; }
    static __device__ __forceinline__ double enc(double v, bool, uint32_t) { return v; }
};
template <> struct Codec<float> {
    using C = float;
    static constexpr bool narrow = false;
    static __device__ __forceinline__ float dec(float v) { return v; }
    static __device__ __forceinline__ float enc(float v, bool, uint32_t) { return v; }
};
template <> struct Codec<__half> {
    using C = float;
    static constexpr bool narrow = true;
    static __device__ __forceinline__ float dec(__half v) { return __half2float(v); }
    static __device__ __forceinline__ __half enc(float v, bool sr, uint32_t r) {
        return sr ? sr_half(v, r) : __float2half_rn(v);
    }
};
template <> struct Codec<__nv_bfloat16> {
    using C = float;
    static constexpr bool narrow = true;
    static __device__ __forceinline__ float dec(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 enc(float v, bool sr, uint32_t r) {
        return sr ? sr_bf16(v, r) : __float2bfloat16_rn(v);
    }
};

// ------------------------------------------------------------ edges
struct Geo {
    int nx, ny;
    int bw, be, bs, bn;
};

// Where the value pulled by node (x, y) in direction i comes from: first the
// y edge (periodic wrap, wall, or free-slip mirror onto the node's own row
// with direction mir_y(i)), then the x edge (wrap, wall, outflow clamp, or
// inlet = unknown).
__host__ __device__ __forceinline__ int map_pull(const Geo &g, int x, int y, int i, int &xs,
                                                 int &ys, int &j) {
    int sx = x - cx(i), sy = y - cy(i), d = i;
    if (sy < 0 || sy >= g.ny) {
        int bc = sy < 0 ? g.bs : g.bn;
        if (bc == PERIODIC) {
            sy = sy < 0 ? sy + g.ny : sy - g.ny;
        } else if (bc == FREESLIP) {
            sy = y;
            d = mir_y(i);
        } else {
            return PULL_BOUNCE;
        }
    }
    if (sx < 0 || sx >= g.nx) {
        int bc = sx < 0 ? g.bw : g.be;
        if (bc == PERIODIC) {
            sx = sx < 0 ? sx + g.nx : sx - g.nx;
        } else if (bc == OUTFLOW_ZG) {
            sx = sx < 0 ? 0 : g.nx - 1;
        } else if (bc == INLET_ZOUHE || bc == INLET_EQ || bc == INLET_EQ_NEUMANN || bc == OUTLET_PRESSURE) {
            return PULL_UNKNOWN;
        } else {
            return PULL_BOUNCE;
        }
    }
    xs = sx;
    ys = sy;
    j = d;
    return PULL_NODE;
}

// ------------------------------------------------------------ collision
template <class C> struct Consts {
    C omega;              // 1/tau
    C hfx, hfy;           // F/2
    C fx, fy, sF, dF;     // F, fx+fy, fx-fy
    C w0, w1, w4;         // 1/36, 1/9, 4/9
    C wl0, wl1, wl4;      // w - (C)w: the weights' rounding residuals (0 in FP64)
    C kw0, kw1, kw4;      // (1 - omega/2) * w
    C zh5, zh8, zh2;      // Zou-He: 2/3 Ux, Ux/6 + Uy/2, Ux/6 - Uy/2
    C drho_out;           // pressure outlet: rho_out - 1
    C heq_in[9];          // equilibrium inlet populations
    int force;            // F != 0
};

// Zou-He velocity inlet: the three populations entering from the west are
// fixed by sum_i g_i c_i = U and bounce-back of the normal non-equilibrium part.
template <class C>
__device__ __forceinline__ void zou_he(const Consts<C> &k, C *g) {
    using A = Ar<C>;
    C g1 = g[1], g7 = g[7];
    g[5] = A::add(g[3], k.zh5);
    g[8] = A::fma(C(0.5), A::sub(g1, g7), A::add(g[0], k.zh8));
    g[2] = A::fma(C(0.5), A::sub(g7, g1), A::add(g[6], k.zh2));
}

// Zou-He pressure outlet: rho = rho_out and v_y = 0, with bounce-back of the
// normal non-equilibrium part, fix the three populations entering from the east.
template <class C>
__device__ __forceinline__ void zou_he_pressure(const Consts<C> &k, C *g) {
    using A = Ar<C>;
    const C g1 = g[1], g7 = g[7];
    const C ux = A::sub(A::fma(C(2), A::add(A::add(g[2], g[5]), g[8]), A::add(A::add(g1, g[4]), g7)), k.drho_out);
    const C u6 = A::mul(ux, C(1.0 / 6.0));
    g[3] = A::fma(C(-2.0 / 3.0), ux, g[5]);
    g[6] = A::sub(A::fma(C(0.5), A::sub(g1, g7), g[2]), u6);
    g[0] = A::sub(A::fma(C(0.5), A::sub(g7, g1), g[8]), u6);
}

// Moments, Eq. (2) equilibrium in deviation form and Eq. (1) BGK relaxation
// with the Guo source, in one fixed operation order:
//   P_i   = drho - 3/2 u^2 + cu_i (3 + 9/2 cu_i)          (h_i^eq = w_i P_i)
//   h*_i  = g_i + omega (w_i P_i - g_i)                    (w P - g in one fma)
//           + (1 - omega/2) w_i [cF_i (3 + 9 cu_i) - 3 u.F]
// with cu_i = c_i.u, cF_i = c_i.F. g (pulled h values) is replaced by h*.
// In FP32, w_i P_i uses w_i as the rounded weight plus its residual: with
// the rounded weights alone, sum_i w_i c_i c_i misses 1/3 by ~1e-8, and the
// relaxation then adds or removes momentum omega * 1e-8 * u at every node
// and update, a drift that reaches 1e-3 in lift and drag over 25,000 updates.
template <class C>
__device__ __forceinline__ void collide(const Consts<C> &k, C *g, C &drho, C &ux, C &uy) {
    using A = Ar<C>;
    const C cw = A::add(A::add(g[0], g[3]), g[6]);   // c_x = -1 column
    const C cm = A::add(A::add(g[1], g[4]), g[7]);   // c_x =  0
    const C ce = A::add(A::add(g[2], g[5]), g[8]);   // c_x = +1
    const C rs = A::add(A::add(g[0], g[1]), g[2]);   // c_y = -1 row
    const C rn = A::add(A::add(g[6], g[7]), g[8]);   // c_y = +1
    drho = A::add(A::add(cw, cm), ce);
    ux = A::add(A::sub(ce, cw), k.hfx);
    uy = A::add(A::sub(rn, rs), k.hfy);
    const C usq = A::fma(ux, ux, A::mul(uy, uy));
    const C base = A::fma(C(-1.5), usq, drho);
    const C s = A::add(ux, uy), d = A::sub(ux, uy);
    const C cu[9] = {-s, -uy, d, -ux, C(0), ux, -d, uy, s};
    const C cF[9] = {-k.sF, -k.fy, k.dF, -k.fx, C(0), k.fx, -k.dF, k.fy, k.sF};
    const C m3uF = A::mul(C(-3), A::fma(ux, k.fx, A::mul(uy, k.fy)));
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const C w = i == 4 ? k.w4 : ((i & 1) ? k.w1 : k.w0);
        const C P = A::fma(cu[i], A::fma(C(4.5), cu[i], C(3)), base);
        C t = A::fma(w, P, -g[i]);
        if (sizeof(C) == 4) t = A::fma(i == 4 ? k.wl4 : ((i & 1) ? k.wl1 : k.wl0), P, t);
        C o = A::fma(k.omega, t, g[i]);
        if (k.force) {
            const C kw = i == 4 ? k.kw4 : ((i & 1) ? k.kw1 : k.kw0);
            o = A::fma(kw, A::fma(cF[i], A::fma(C(9), cu[i], C(3)), m3uF), o);
        }
        g[i] = o;
    }
}

}  // namespace lbm
