// Device-side building blocks of the D2Q9I BGK update (PortLBM, Sec. 3):
// direction set, the three population layouts, storage codecs, the pull
// mapping at domain edges, and the collision routine every kernel of a
// storage type calls.
#pragma once

#include <cstdint>
#include <cstring>
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
// Random word of population i of a node: the node's hashed key with a
// per-direction constant folded in, multiplied by an odd constant (a
// multiplicative hash); the stochastic rounding below uses its top bits.
__host__ __device__ __forceinline__ uint32_t pop_rand(uint32_t nkey, int i) {
    return (nkey ^ ((uint32_t)i * 0x9E3779B9U)) * 0x85EBCA6BU;
}

// ------------------------------------------------------------ codecs
// Stochastic rounding of FP32 values to 16 bits with the stochastic-rounding
// conversion of the sm_100 family (cvt.rs): a random integer, the top bits of
// the value's random word r (13 for FP16, 16 for BF16), is added to the top
// bits the conversion drops and the sum truncated, so the kept part
// increments exactly when those dropped bits plus the draw carry: away from
// zero with probability (|x| - |lo|) / ulp, lo the value rounded toward zero
// and ulp the gap to the next magnitude. BF16 drops 16 bits and FP16 13 in
// its normal range (|x| >= 2^-14), where this is exact; below 2^-14 FP16
// drops more than 13 bits and the probability is the dropped fraction cut to
// 13 bits (at most 2^-13 ulp low). The packed forms round two values: hi to
// the upper half (its draw in bits 28..16 for FP16, 31..16 for BF16), lo to
// the lower half (bits 12..0, 15..0), each exactly as the one-value form.
__device__ __forceinline__ uint32_t sr_half2(float hi, float lo, uint32_t r_hi, uint32_t r_lo) {
    const uint32_t draw = ((r_hi >> 19) << 16) | (r_lo >> 19);
    uint32_t d;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(draw));
    return d;
}
__device__ __forceinline__ uint32_t sr_bf162(float hi, float lo, uint32_t r_hi, uint32_t r_lo) {
    const uint32_t draw = (r_hi & 0xFFFF0000u) | (r_lo >> 16);
    uint32_t d;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(draw));
    return d;
}
__device__ __forceinline__ __half sr_half(float x, uint32_t r) {
    return __ushort_as_half((unsigned short)(sr_half2(0.0f, x, 0u, r) & 0xFFFFu));
}
__device__ __forceinline__ __nv_bfloat16 sr_bf16(float x, uint32_t r) {
    return __ushort_as_bfloat16((unsigned short)(sr_bf162(0.0f, x, 0u, r) & 0xFFFFu));
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

// ------------------------------------------------------------ tensor copies
// Tensor copy (TMA) of a tile into shared memory with an mbarrier that
// counts the bytes: one thread initialises the barrier, announces the bytes
// and issues the copy; every thread then waits on the barrier's phase 0 with
// an iteration limit.
constexpr int kTmaSpin = 1 << 20;

__device__ __forceinline__ void tma_issue_3d(const void *tm, void *dst, uint64_t *bar, int c0, int c1, int c2,
                                             uint32_t bytes) {
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar), d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(d),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(b)
        : "memory");
}

__device__ __forceinline__ bool tma_wait(uint64_t *bar) {
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    for (int it = 0; it < kTmaSpin; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(b)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// ------------------------------------------------------------ NSOL
// One lattice, swap streaming: populations are stored in opposite slots
// (slot s of node x holds f*_{8-s}(x)). Tiles are staged in shared memory;
// for each of the four positive directions i, slot 8-i of x is exchanged
// with slot i of x + c_i when both are fluid (no exchange = bounce-back).
// Values that enter through domain edges or from other tiles (buffer grid)
// are substituted afterwards.
// Two block barriers: after the staging (and the substitutions, read from
// the lattice and the buffer grid), and after the exchanges.
// smem_raw: 9 * tx * ty compute values.
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
// with the Guo source, in the fixed operation order of 32- and 64-bit
// storage:
//   P_i   = drho - 3/2 u^2 + cu_i (3 + 9/2 cu_i)          (h_i^eq = w_i P_i)
//   h*_i  = g_i + omega (w_i P_i - g_i)                    (w P - g in one fma)
//           + (1 - omega/2) w_i [cF_i (3 + 9 cu_i) - 3 u.F]
// with cu_i = c_i.u, cF_i = c_i.F. g (pulled h values) is replaced by h*.
// In FP32, w_i P_i uses w_i as the rounded weight plus its residual: with
// the rounded weights alone, sum_i w_i c_i c_i misses 1/3 by ~1e-8, and the
// relaxation then adds or removes momentum omega * 1e-8 * u at every node
// and update, a drift that reaches 1e-3 in lift and drag over 25,000 updates.
template <class C>
__device__ __forceinline__ void collide_signed(const Consts<C> &k, C *g, C &drho, C &ux, C &uy) {
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

// The same update in the fixed operation order of 16-bit storage:
//   P_i   = drho - 3/2 u^2 + cu_i (3 + 9/2 cu_i)          (h_i^eq = w_i P_i)
//   h*_i  = g_i - omega (g_i - w_i P_i)
//           + (1 - omega/2) w_i [cF_i (3 + 9 cu_i) - 3 u.F]
// with cu_i = c_i.u, cF_i = c_i.F. g (pulled h values) is replaced by h*.
// Every direction is written through the magnitude c = |cu_i| of its pair
// (u_x, u_y, u_x + u_y, u_x - u_y) and the sign sg of cu_i:
//   cu_i (3 + 9/2 cu_i) = c (9/2 c + 3 sg),  cF_i (3 + 9 cu_i) = cF+ (9 c + 3 sg)
// with cF+ = sg cF_i, so no operand is ever negated at run time and the
// packed two-node form below (collide2) performs the same rounded operations
// lane by lane. (On the 32-bit storage path this form measured 2 % slower
// than the signed one above, so each storage type keeps its own order; all
// kernels of one storage type share it and agree bit for bit.)
template <class C>
__device__ __forceinline__ C relax(const Consts<C> &k, C g, C c, C sg3, C base, C m3uF, C w, C wl, C kw,
                                   C cFp) {
    using A = Ar<C>;
    const C P = A::fma(c, A::fma(C(4.5), c, sg3), base);
    C t = A::fma(-w, P, g);                                // g - w P
    if (sizeof(C) == 4) t = A::fma(-wl, P, t);
    C o = A::fma(-k.omega, t, g);                          // g - omega (g - w P)
    if (k.force) o = A::fma(kw, A::fma(cFp, A::fma(C(9), c, sg3), m3uF), o);
    return o;
}

template <class C>
__device__ __forceinline__ void collide_paired(const Consts<C> &k, C *g, C &drho, C &ux, C &uy) {
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
    const C m3uF = A::mul(C(-3), A::fma(ux, k.fx, A::mul(uy, k.fy)));
    const C p3 = C(3), m3 = C(-3);
    g[0] = relax(k, g[0], s, m3, base, m3uF, k.w0, k.wl0, k.kw0, k.sF);
    g[1] = relax(k, g[1], uy, m3, base, m3uF, k.w1, k.wl1, k.kw1, k.fy);
    g[2] = relax(k, g[2], d, p3, base, m3uF, k.w0, k.wl0, k.kw0, k.dF);
    g[3] = relax(k, g[3], ux, m3, base, m3uF, k.w1, k.wl1, k.kw1, k.fx);
    {   // rest: cu = cF = 0, P = base
        C t = A::fma(-k.w4, base, g[4]);
        if (sizeof(C) == 4) t = A::fma(-k.wl4, base, t);
        C o = A::fma(-k.omega, t, g[4]);
        if (k.force) o = A::fma(k.kw4, m3uF, o);
        g[4] = o;
    }
    g[5] = relax(k, g[5], ux, p3, base, m3uF, k.w1, k.wl1, k.kw1, k.fx);
    g[6] = relax(k, g[6], d, m3, base, m3uF, k.w0, k.wl0, k.kw0, k.dF);
    g[7] = relax(k, g[7], uy, p3, base, m3uF, k.w1, k.wl1, k.kw1, k.fy);
    g[8] = relax(k, g[8], s, p3, base, m3uF, k.w0, k.wl0, k.kw0, k.sF);
}

// The operation order every kernel of a storage type uses: the signed order
// for 64- and 32-bit storage, the negation-free order (which the packed
// node-pair kernel reproduces lane by lane) for 16-bit storage.
template <bool NARROW, class C>
__device__ __forceinline__ void collide(const Consts<C> &k, C *g, C &drho, C &ux, C &uy) {
    if constexpr (NARROW)
        collide_paired(k, g, drho, ux, uy);
    else
        collide_signed(k, g, drho, ux, uy);
}

// ------------------------------------------------------------ packed pairs
// Two FP32 values (lanes: first node, second node) in one 64-bit register
// pair, operated on by sm_100-family packed FP32 instructions. Each lane is
// rounded exactly like the scalar __fadd_rn / __fmul_rn / __fmaf_rn.
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk2(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void up2(f2 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// The FP32 constants of Consts<float>, each duplicated into both lanes, with
// the signs collide() applies folded in.
struct Consts2 {
    f2 nomega, nw0, nw1, nw4, nwl0, nwl1, nwl4, kw0, kw1, kw4;
    f2 hfx, hfy, fx, fy, sF, dF;
    f2 c45, c3, cm3, c9, cm15;
};

__host__ __device__ inline f2 dup2(float v) {
    uint32_t b;
    memcpy(&b, &v, 4);
    return ((f2)b << 32) | (f2)b;
}

inline Consts2 make_consts2(const Consts<float> &k) {
    Consts2 q;
    q.nomega = dup2(-k.omega);
    q.nw0 = dup2(-k.w0); q.nw1 = dup2(-k.w1); q.nw4 = dup2(-k.w4);
    q.nwl0 = dup2(-k.wl0); q.nwl1 = dup2(-k.wl1); q.nwl4 = dup2(-k.wl4);
    q.kw0 = dup2(k.kw0); q.kw1 = dup2(k.kw1); q.kw4 = dup2(k.kw4);
    q.hfx = dup2(k.hfx); q.hfy = dup2(k.hfy); q.fx = dup2(k.fx); q.fy = dup2(k.fy);
    q.sF = dup2(k.sF); q.dF = dup2(k.dF);
    q.c45 = dup2(4.5f); q.c3 = dup2(3.0f); q.cm3 = dup2(-3.0f); q.c9 = dup2(9.0f); q.cm15 = dup2(-1.5f);
    return q;
}

__device__ __forceinline__ f2 relax2(const Consts2 &q, int force, f2 g, f2 c, f2 sg3, f2 base, f2 m3uF,
                                     f2 nw, f2 nwl, f2 kw, f2 cFp) {
    const f2 P = fma2(c, fma2(q.c45, c, sg3), base);
    f2 t = fma2(nw, P, g);
    t = fma2(nwl, P, t);
    f2 o = fma2(q.nomega, t, g);
    if (force) o = fma2(kw, fma2(cFp, fma2(q.c9, c, sg3), m3uF), o);
    return o;
}

// collide_paired<float>() for two nodes at once: the same rounded operations in the
// same order on each lane, so each lane's result is bit-identical to the
// scalar routine's.
__device__ __forceinline__ void collide2(const Consts2 &q, int force, f2 *g, f2 &drho, f2 &ux, f2 &uy) {
    const f2 cw = add2(add2(g[0], g[3]), g[6]);
    const f2 cm = add2(add2(g[1], g[4]), g[7]);
    const f2 ce = add2(add2(g[2], g[5]), g[8]);
    const f2 rs = add2(add2(g[0], g[1]), g[2]);
    const f2 rn = add2(add2(g[6], g[7]), g[8]);
    drho = add2(add2(cw, cm), ce);
    ux = add2(sub2(ce, cw), q.hfx);
    uy = add2(sub2(rn, rs), q.hfy);
    const f2 usq = fma2(ux, ux, mul2(uy, uy));
    const f2 base = fma2(q.cm15, usq, drho);
    const f2 s = add2(ux, uy), d = sub2(ux, uy);
    const f2 m3uF = mul2(q.cm3, fma2(ux, q.fx, mul2(uy, q.fy)));
    g[0] = relax2(q, force, g[0], s, q.cm3, base, m3uF, q.nw0, q.nwl0, q.kw0, q.sF);
    g[1] = relax2(q, force, g[1], uy, q.cm3, base, m3uF, q.nw1, q.nwl1, q.kw1, q.fy);
    g[2] = relax2(q, force, g[2], d, q.c3, base, m3uF, q.nw0, q.nwl0, q.kw0, q.dF);
    g[3] = relax2(q, force, g[3], ux, q.cm3, base, m3uF, q.nw1, q.nwl1, q.kw1, q.fx);
    {
        f2 t = fma2(q.nw4, base, g[4]);
        t = fma2(q.nwl4, base, t);
        f2 o = fma2(q.nomega, t, g[4]);
        if (force) o = fma2(q.kw4, m3uF, o);
        g[4] = o;
    }
    g[5] = relax2(q, force, g[5], ux, q.c3, base, m3uF, q.nw1, q.nwl1, q.kw1, q.fx);
    g[6] = relax2(q, force, g[6], d, q.cm3, base, m3uF, q.nw0, q.nwl0, q.kw0, q.dF);
    g[7] = relax2(q, force, g[7], uy, q.c3, base, m3uF, q.nw1, q.nwl1, q.kw1, q.fy);
    g[8] = relax2(q, force, g[8], s, q.c3, base, m3uF, q.nw0, q.nwl0, q.kw0, q.sF);
}

}  // namespace lbm
