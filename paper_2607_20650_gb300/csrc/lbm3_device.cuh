// D3Q19 building blocks: the three-dimensional extension the paper lists as
// future work (Sec. 6), with the method of Sec. 3.1 (Eq. 1 BGK, Eq. 2
// incompressible equilibrium with v = sum f c) on the 19 velocities of
// {-1,0,1}^3 with |c|^2 <= 2, ordered lexicographically in (c_z, c_y, c_x):
// opposite(i) = 18 - i, rest at i = 9, weights 1/3, 1/18 (faces), 1/36 (edges).
#pragma once

#include "lbm_device.cuh"

namespace lbm {
namespace d3 {

constexpr int Q = 19;
constexpr int REST = 9;
constexpr uint32_t SOLID = 0x3FFFFu;  // all 18 pulls bounce: solid (or isolated) node

__host__ __device__ constexpr int cx(int i) {
    return i == 0 || i == 4 || i == 14 || i == 18 ? 0
         : (i == 1 || i == 5 || i == 8 || i == 11 || i == 15) ? -1
         : (i == 3 || i == 7 || i == 10 || i == 13 || i == 17) ? 1 : 0;
}
__host__ __device__ constexpr int cy(int i) {
    return (i == 0 || (i >= 5 && i <= 7) || i == 14) ? -1 : ((i == 4 || (i >= 11 && i <= 13) || i == 18) ? 1 : 0);
}
__host__ __device__ constexpr int cz(int i) { return i <= 4 ? -1 : (i >= 14 ? 1 : 0); }
__host__ __device__ constexpr int opp(int i) { return 18 - i; }
__host__ __device__ constexpr int bit(int i) { return i < REST ? i : i - 1; }
__host__ __device__ constexpr int sq(int i) { return cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i); }

// Bundles: directions with the same (c_y, c_z) (the same source row), in
// order; first direction and size of the bundle that holds direction i.
__host__ __device__ constexpr int bundle_first(int i) {
    return i == 0 ? 0 : i <= 3 ? 1 : i == 4 ? 4 : i <= 7 ? 5 : i <= 10 ? 8 : i <= 13 ? 11 : i == 14 ? 14 : i <= 17 ? 15 : 18;
}
__host__ __device__ constexpr int bundle_size(int i) { return (i == 0 || i == 4 || i == 14 || i == 18) ? 1 : 3; }

// Element offset of population i of node n (N nodes): stream i N + n,
// collision 19 n + i, bundle first N + size n + (i - first).
template <int L>
__host__ __device__ __forceinline__ int64_t addr(int64_t N, int64_t n, int i) {
    if (L == STREAM) return (int64_t)i * N + n;
    if (L == COLLISION) return n * 19 + i;
    return (int64_t)bundle_first(i) * N + (int64_t)bundle_size(i) * n + (i - bundle_first(i));
}

template <class C> struct Consts3 {
    C omega;
    C hf[3];        // F/2
    C f[3];         // F
    C cF[Q];        // c_i . F
    C w0, w1, w2;   // 1/3, 1/18, 1/36
    C wl0, wl1, wl2;  // w - (C)w: rounding residuals of the weights (0 in FP64)
    C kw0, kw1, kw2;  // (1 - omega/2) w
    int force;
};

// Moments, Eq. 2 equilibrium (deviation form) and Eq. 1 BGK relaxation with
// the Guo source in one fixed operation order (shared by every D3Q19 kernel):
//   P_i  = drho - 3/2 u^2 + cu_i (3 + 9/2 cu_i),  h*_i = g_i + omega (w_i P_i - g_i)
//          + (1 - omega/2) w_i [cF_i (3 + 9 cu_i) - 3 u.F]
// with cu_i formed from the one or two nonzero components of c_i, and in
// FP32 w_i P_i formed with w_i as the rounded weight plus its residual (the
// rounded weights alone miss sum_i w_i c_i c_i = 1/3 by ~1e-8, which would
// make the relaxation a momentum source proportional to u).
template <class C>
__device__ __forceinline__ void collide3(const Consts3<C> &k, C *g, C &drho, C &ux, C &uy, C &uz) {
    using A = Ar<C>;
    C r = g[0];
#pragma unroll
    for (int i = 1; i < Q; ++i) r = A::add(r, g[i]);
    drho = r;
    // momentum: signed sums in direction order, starting from the first term
    C j[3];
    bool started[3] = {false, false, false};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int c[3] = {cx(i), cy(i), cz(i)};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (!c[a]) continue;
            if (!started[a]) {
                j[a] = c[a] > 0 ? g[i] : -g[i];
                started[a] = true;
            } else {
                j[a] = c[a] > 0 ? A::add(j[a], g[i]) : A::sub(j[a], g[i]);
            }
        }
    }
    ux = A::add(j[0], k.hf[0]);
    uy = A::add(j[1], k.hf[1]);
    uz = A::add(j[2], k.hf[2]);
    const C usq = A::fma(ux, ux, A::fma(uy, uy, A::mul(uz, uz)));
    const C base = A::fma(C(-1.5), usq, drho);
    const C m3uF = A::mul(C(-3), A::fma(ux, k.f[0], A::fma(uy, k.f[1], A::mul(uz, k.f[2]))));
    const C u[3] = {ux, uy, uz};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int c[3] = {cx(i), cy(i), cz(i)};
        C cu = C(0);
        bool any = false;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (!c[a]) continue;
            const C t = c[a] > 0 ? u[a] : -u[a];
            cu = any ? A::add(cu, t) : t;
            any = true;
        }
        const C w = sq(i) == 0 ? k.w0 : (sq(i) == 1 ? k.w1 : k.w2);
        const C P = any ? A::fma(cu, A::fma(C(4.5), cu, C(3)), base) : base;
        C t = A::fma(w, P, -g[i]);
        if (sizeof(C) == 4) t = A::fma(sq(i) == 0 ? k.wl0 : (sq(i) == 1 ? k.wl1 : k.wl2), P, t);
        C o = A::fma(k.omega, t, g[i]);
        if (k.force && any) {
            const C kw = sq(i) == 1 ? k.kw1 : k.kw2;
            o = A::fma(kw, A::fma(k.cF[i], A::fma(C(9), cu, C(3)), m3uF), o);
        } else if (k.force) {
            o = A::fma(k.kw0, m3uF, o);
        }
        g[i] = o;
    }
}

// The FP32 constants of Consts3<float>, each duplicated into both lanes of a
// packed pair, with the signs collide3_2 folds in.
struct Consts3x2 {
    f2 nomega, nw[3], nwl[3], kw[3];
    f2 hf[3], f[3], cF[Q];
    f2 c45, c3, c9, cm3, cm15, cm1;
};

inline Consts3x2 make_consts3x2(const Consts3<float> &k) {
    Consts3x2 q;
    q.nomega = dup2(-k.omega);
    const float w[3] = {k.w0, k.w1, k.w2}, wl[3] = {k.wl0, k.wl1, k.wl2}, kw[3] = {k.kw0, k.kw1, k.kw2};
    for (int s = 0; s < 3; ++s) {
        q.nw[s] = dup2(-w[s]);
        q.nwl[s] = dup2(-wl[s]);
        q.kw[s] = dup2(kw[s]);
        q.hf[s] = dup2(k.hf[s]);
        q.f[s] = dup2(k.f[s]);
    }
    for (int i = 0; i < Q; ++i) q.cF[i] = dup2(k.cF[i]);
    q.c45 = dup2(4.5f);
    q.c3 = dup2(3.0f);
    q.c9 = dup2(9.0f);
    q.cm3 = dup2(-3.0f);
    q.cm15 = dup2(-1.5f);
    q.cm1 = dup2(-1.0f);
    return q;
}

// collide3 on two nodes at once (packed FP32 pairs, fma.rn.f32x2 and
// friends): the same rounded operations lane by lane, so each lane equals
// the scalar collide3 bit for bit. The relaxation is written without
// negated operands, t' = fma(-w, P, g) = -fma(w, P, -g) and o =
// fma(-omega, t'', g), which IEEE rounding makes exact; a negative first
// term of a sum is an exact product with -1.
__device__ __forceinline__ void collide3_2(const Consts3x2 &q, int force, f2 *g, f2 &drho, f2 &ux, f2 &uy,
                                           f2 &uz) {
    f2 r = g[0];
#pragma unroll
    for (int i = 1; i < Q; ++i) r = add2(r, g[i]);
    drho = r;
    f2 j[3];
    bool started[3] = {false, false, false};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int c[3] = {cx(i), cy(i), cz(i)};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (!c[a]) continue;
            if (!started[a]) {
                j[a] = c[a] > 0 ? g[i] : mul2(g[i], q.cm1);
                started[a] = true;
            } else {
                j[a] = c[a] > 0 ? add2(j[a], g[i]) : sub2(j[a], g[i]);
            }
        }
    }
    ux = add2(j[0], q.hf[0]);
    uy = add2(j[1], q.hf[1]);
    uz = add2(j[2], q.hf[2]);
    const f2 usq = fma2(ux, ux, fma2(uy, uy, mul2(uz, uz)));
    const f2 base = fma2(q.cm15, usq, drho);
    const f2 m3uF = mul2(q.cm3, fma2(ux, q.f[0], fma2(uy, q.f[1], mul2(uz, q.f[2]))));
    const f2 u[3] = {ux, uy, uz};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int c[3] = {cx(i), cy(i), cz(i)};
        f2 cu = 0;
        bool any = false;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (!c[a]) continue;
            if (!any) cu = c[a] > 0 ? u[a] : mul2(u[a], q.cm1);
            else cu = c[a] > 0 ? add2(cu, u[a]) : sub2(cu, u[a]);
            any = true;
        }
        const int s = sq(i);
        const f2 P = any ? fma2(cu, fma2(q.c45, cu, q.c3), base) : base;
        f2 t = fma2(q.nw[s], P, g[i]);
        t = fma2(q.nwl[s], P, t);
        f2 o = fma2(q.nomega, t, g[i]);
        if (force && any) o = fma2(q.kw[s], fma2(q.cF[i], fma2(q.c9, cu, q.c3), m3uF), o);
        else if (force) o = fma2(q.kw[0], m3uF, o);
        g[i] = o;
    }
}

}  // namespace d3
}  // namespace lbm
