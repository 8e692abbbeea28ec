// Host launchers of the D3Q19 kernels for one storage type S: the kernel
// arguments of a box (make3), one update per algorithm, init, moments, mass,
// force and the batched update, gathered in an Ops3 table. Included only by
// the lbm3_ops_*.cu translation units, one per storage type.
#pragma once

#include <cstring>

#include "lbm3_internal.h"
#include "lbm3_kernels.cuh"

using namespace lbm;
using namespace lbm::d3;

namespace {

template <class S>
Step3<S> make3(const lbm3_lattice *L, int src, int toff, int mom) {
    using C = typename Codec<S>::C;
    Step3<S> a;
    const lbm3_params &p = L->p;
    a.g = Geo3{p.nx, p.ny, p.nz, p.bc_x, p.bc_y, p.bc_z, east3_kind(&p)};
    a.xlo_corr = p.bc_x == LBM_BC_PERIODIC ? p.nx : (p.bc_x == LBM_BC_OUTFLOW_ZG ? 1 : 0);
    a.xhi_corr = a.g.bxe == LBM_BC_PERIODIC ? -p.nx : (a.g.bxe == LBM_BC_OUTFLOW_ZG ? -1 : 0);
    a.inlet = p.bc_x == LBM_BC_INLET_EQ ? 1 : (p.bc_x == LBM_BC_INLET_ZOUHE ? 2 : 0);
    a.outlet = (inlet3_kind(p.bc_x) && p.bc_x_east == LBM_BC_OUTLET_PRESSURE) ? 1 : 0;
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
    a.err = L->err;
    a.tctr = L->tctr;
    a.toff = toff;
    a.sr = p.rounding;
    a.seed = p.seed;
    a.tx = L->pl.tx;
    a.ty = L->pl.ty;
    a.tz = L->pl.tz;
    a.nx_magic = magic3((uint64_t)p.nx);
    a.nxy_magic = magic3((uint64_t)p.nx * (uint64_t)p.ny);
    // measured: +7 % for the stream layout on a porous box, -3 % for the bundle layout
    a.zero_fill = (p.layout != LBM_LAYOUT_BUNDLE && (p.algo == LBM_LPTL || L->pl.tx % 32 == 0)) ? 1 : 0;
    if constexpr (std::is_same<C, float>::value) a.k2 = make_consts3x2(a.k);
    return a;
}

// Node pairs (k3_step_pair): 16-bit storage, stream or bundle layout, the
// 32-bit offset tables, nx even (and tile_x even for NPTL), unless
// LBM_FLAG_NO_PAIRS asks for one node per thread.
template <class S>
bool pairs3_ok(const lbm3_lattice *L) {
    const lbm3_params &p = L->p;
    return sizeof(S) == 2 && L->off32 && (p.layout == LBM_LAYOUT_BUNDLE || p.layout == LBM_LAYOUT_STREAM) &&
           p.nx % 2 == 0 && !(p.flags & LBM_FLAG_NO_PAIRS) && (p.algo == LBM_LPTL || L->pl.tx % 2 == 0);
}

template <class S, bool LINEAR>
void launch_pair3(const lbm3_lattice *L, const Step3<S> &a, cudaStream_t st) {
    dim3 g, b;
    if (LINEAR) {
        b = dim3(128);
        g = dim3((unsigned)((L->pl.N / 2 + 127) / 128));
    } else {
        b = dim3(L->pl.tx / 2, L->pl.ty, L->pl.tz);
        g = dim3(L->pl.ntx, L->pl.nty, L->pl.ntz);
    }
    if (L->p.layout == LBM_LAYOUT_STREAM) k3_step_pair<S, STREAM, LINEAR><<<g, b, 0, st>>>(a);
    else k3_step_pair<S, BUNDLE, LINEAR><<<g, b, 0, st>>>(a);
}

template <class S, bool LINEAR, bool OFF32>
void launch3k(const lbm3_lattice *L, const Step3<S> &a, dim3 grid, dim3 block, cudaStream_t st) {
    const int lay = L->p.layout;
    if (lay == LBM_LAYOUT_STREAM) k3_step<S, STREAM, LINEAR, OFF32><<<grid, block, 0, st>>>(a);
    else if (lay == LBM_LAYOUT_BUNDLE) k3_step<S, BUNDLE, LINEAR, OFF32><<<grid, block, 0, st>>>(a);
    else k3_step<S, COLLISION, LINEAR, OFF32><<<grid, block, 0, st>>>(a);
}

template <class S, int PHASE>
void launch_aa(const lbm3_lattice *L, const Step3<S> &a, cudaStream_t st) {
    const dim3 g(L->pl.ntx, L->pl.nty, L->pl.ntz), b(L->pl.tx, L->pl.ty, L->pl.tz);
    const int lay = L->p.layout;
    if (lay == LBM_LAYOUT_STREAM) k3_aa<S, STREAM, PHASE><<<g, b, 0, st>>>(a);
    else if (lay == LBM_LAYOUT_BUNDLE) k3_aa<S, BUNDLE, PHASE><<<g, b, 0, st>>>(a);
    else k3_aa<S, COLLISION, PHASE><<<g, b, 0, st>>>(a);
}

template <class S>
S *halo_parity(const lbm3_lattice *L, int parity) {
    return (S *)(L->ws + L->pl.halo) + (int64_t)parity * L->pl.halo_parity;
}

template <class S, bool OFF32>
void launch_npol(const lbm3_lattice *L, const Step3<S> &a, int parity, cudaStream_t st) {
    const dim3 g(L->pl.ntx, L->pl.nty, L->pl.ntz), b(L->pl.tx, L->pl.ty, L->pl.tz);
    const S *hr = halo_parity<S>(L, parity);
    S *hw = halo_parity<S>(L, parity ^ 1);
    const int lay = L->p.layout;
    if (lay == LBM_LAYOUT_STREAM) k3_npol<S, STREAM, OFF32><<<g, b, 0, st>>>(a, hr, hw);
    else if (lay == LBM_LAYOUT_BUNDLE) k3_npol<S, BUNDLE, OFF32><<<g, b, 0, st>>>(a, hr, hw);
    else k3_npol<S, COLLISION, OFF32><<<g, b, 0, st>>>(a, hr, hw);
}

template <class S>
void launch_nsol(const lbm3_lattice *L, const Step3<S> &a, int parity, cudaStream_t st) {
    const dim3 g(L->pl.ntx, L->pl.nty, L->pl.ntz), b(L->pl.tx, L->pl.ty, L->pl.tz);
    const size_t sm = nsol3_smem_bytes<S>(L->pl.tx, L->pl.ty, L->pl.tz);
    const S *hr = halo_parity<S>(L, parity);
    S *hw = halo_parity<S>(L, parity ^ 1);
    const int lay = L->p.layout;
    if (lay == LBM_LAYOUT_STREAM) k3_nsol<S, STREAM><<<g, b, sm, st>>>(a, hr, hw);
    else if (lay == LBM_LAYOUT_BUNDLE) k3_nsol<S, BUNDLE><<<g, b, sm, st>>>(a, hr, hw);
    else k3_nsol<S, COLLISION><<<g, b, sm, st>>>(a, hr, hw);
}

// Largest staged tile of the 3-D NSOL kernels (512 nodes) beyond the default
// 48 KB of dynamic shared memory (FP64: 76 KB), single and batched.
template <class S>
void nsol3_prepare() {
    static const bool done = [] {
        const int bytes = (int)nsol3_smem_bytes<S>(512, 1, 1);
        cudaFuncSetAttribute(k3_nsol<S, STREAM>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        cudaFuncSetAttribute(k3_nsol<S, BUNDLE>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        cudaFuncSetAttribute(k3_nsol<S, COLLISION>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        cudaFuncSetAttribute(k3_batch<S, STREAM, LBM_NSOL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        cudaFuncSetAttribute(k3_batch<S, BUNDLE, LBM_NSOL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        cudaFuncSetAttribute(k3_batch<S, COLLISION, LBM_NSOL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes);
        cudaGetLastError();
        return true;
    }();
    (void)done;
}

// NPOL: fill buffer-grid parity `parity` from the stored state.
template <class S>
cudaError_t publish_state(const lbm3_lattice *L, int parity, cudaStream_t st) {
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
cudaError_t step3(const lbm3_lattice *L, cudaStream_t st, int src, int toff, int mom) {
    const Step3<S> a = make3<S>(L, src, toff, mom);
    if (L->p.algo == LBM_NPOL) {
        if (L->off32) launch_npol<S, true>(L, a, src, st);
        else launch_npol<S, false>(L, a, src, st);
    } else if (L->p.algo == LBM_NSOL) {
        launch_nsol<S>(L, a, src, st);
    } else if (L->p.algo == LBM_AA) {
        if (src == 0) launch_aa<S, 0>(L, a, st);
        else launch_aa<S, 1>(L, a, st);
    } else if ((L->p.algo == LBM_LPTL || L->p.algo == LBM_NPTL) && pairs3_ok<S>(L)) {
        if constexpr (sizeof(S) == 2) {
            if (L->p.algo == LBM_LPTL) launch_pair3<S, true>(L, a, st);
            else launch_pair3<S, false>(L, a, st);
        }
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


template <class S, int L>
cudaError_t init_k(const lbm3_lattice *L_, const double *const dv[4], uint32_t n0, uint32_t c, cudaStream_t st) {
    const Step3<S> a = make3<S>(L_, 1, 0, 0);   // dst = lattice 0
    k3_init<S, L><<<(c + 255) / 256, 256, 0, st>>>(a, dv[0], dv[1], dv[2], dv[3], n0, c);
    return cudaGetLastError();
}

template <class S>
cudaError_t init3(const lbm3_lattice *L, const double *const dv[4], uint32_t n0, uint32_t c, cudaStream_t st) {
    if (L->p.layout == LBM_LAYOUT_STREAM) return init_k<S, STREAM>(L, dv, n0, c, st);
    if (L->p.layout == LBM_LAYOUT_BUNDLE) return init_k<S, BUNDLE>(L, dv, n0, c, st);
    return init_k<S, COLLISION>(L, dv, n0, c, st);
}

template <class S>
cudaError_t state_moments3(const lbm3_lattice *L, cudaStream_t st) {
    const Step3<S> a = make3<S>(L, 0, 0, 1);
    const unsigned g = (unsigned)((L->pl.N + 255) / 256);
    if (L->p.layout == LBM_LAYOUT_STREAM) k3_state_moments<S, STREAM><<<g, 256, 0, st>>>(a);
    else if (L->p.layout == LBM_LAYOUT_BUNDLE) k3_state_moments<S, BUNDLE><<<g, 256, 0, st>>>(a);
    else k3_state_moments<S, COLLISION><<<g, 256, 0, st>>>(a);
    return cudaGetLastError();
}

template <class S>
cudaError_t mass3(const lbm3_lattice *L, double *partials, cudaStream_t st) {
    const Step3<S> a = make3<S>(L, L->cur, 0, 0);
    if (L->p.layout == LBM_LAYOUT_STREAM) k3_mass<S, STREAM><<<kReduceBlocks, kReduceThreads, 0, st>>>(a, partials);
    else if (L->p.layout == LBM_LAYOUT_BUNDLE) k3_mass<S, BUNDLE><<<kReduceBlocks, kReduceThreads, 0, st>>>(a, partials);
    else k3_mass<S, COLLISION><<<kReduceBlocks, kReduceThreads, 0, st>>>(a, partials);
    return cudaGetLastError();
}

template <class S>
cudaError_t force3(const lbm3_lattice *L, const uint8_t *body, double *partials, cudaStream_t st) {
    const Step3<S> a = make3<S>(L, L->cur, 0, 0);
    if (L->p.layout == LBM_LAYOUT_STREAM)
        k3_force<S, STREAM><<<kReduceBlocks, kReduceThreads, 0, st>>>(a, body, partials);
    else if (L->p.layout == LBM_LAYOUT_BUNDLE)
        k3_force<S, BUNDLE><<<kReduceBlocks, kReduceThreads, 0, st>>>(a, body, partials);
    else
        k3_force<S, COLLISION><<<kReduceBlocks, kReduceThreads, 0, st>>>(a, body, partials);
    return cudaGetLastError();
}

template <class S>
int block3_of(int layout) {
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

template <class S>
void prepare3(int algo) {
    if (algo == LBM_NSOL) nsol3_prepare<S>();
}

// Device record of one case of a batch: its arguments for both parities.
template <class S>
void batch_case3(const lbm3_lattice *L, void *rec) {
    Case3<S> c;
    memset(&c, 0, sizeof(c));
    c.a[0] = make3<S>(L, 0, 0, 0);
    c.a[1] = make3<S>(L, 1, 0, 0);
    for (int p = 0; p < 2; ++p) c.halo[p] = L->pl.halo_parity ? halo_parity<S>(L, p) : nullptr;
    c.mom = (typename Codec<S>::C *)(L->ws + L->pl.mom);
    c.nt[0] = L->pl.ntx;
    c.nt[1] = L->pl.nty;
    c.nt[2] = L->pl.ntz;
    memcpy(rec, &c, sizeof(c));
}

template <class S, int L, int ALGO, bool OFF32>
void batch_k(const Batch3Launch &b, cudaStream_t st) {
    const dim3 block = ALGO == LBM_LPTL ? dim3((unsigned)b.block_1d) : dim3(b.tx, b.ty, b.tz);
    const size_t sm = ALGO == LBM_NSOL ? nsol3_smem_bytes<S>(b.tx, b.ty, b.tz) : 0;
    k3_batch<S, L, ALGO, OFF32><<<b.nitems, block, sm, st>>>((const Case3<S> *)b.cases, (const uint2 *)b.items,
                                                             b.src, b.toff, b.mom);
}

// Batches use the 32-bit offset tables (every case is checked to fit them).
template <class S, int L>
void batch_layout3(const Batch3Launch &b, cudaStream_t st) {
    switch (b.algo) {
        case LBM_LPTL: batch_k<S, L, LBM_LPTL, true>(b, st); break;
        case LBM_NPTL: batch_k<S, L, LBM_NPTL, true>(b, st); break;
        case LBM_NPOL: batch_k<S, L, LBM_NPOL, true>(b, st); break;
        default: batch_k<S, L, LBM_NSOL, false>(b, st); break;
    }
}

template <class S>
cudaError_t batch_step3(const Batch3Launch &b, cudaStream_t st) {
    if (b.layout == LBM_LAYOUT_STREAM) batch_layout3<S, STREAM>(b, st);
    else if (b.layout == LBM_LAYOUT_BUNDLE) batch_layout3<S, BUNDLE>(b, st);
    else batch_layout3<S, COLLISION>(b, st);
    return cudaGetLastError();
}

template <class S>
Ops3 make_ops3() {
    Ops3 o;
    o.step = step3<S>;
    o.init = init3<S>;
    o.state_moments = state_moments3<S>;
    o.publish = publish_state<S>;
    o.mass = mass3<S>;
    o.force = force3<S>;
    o.block_1d = block3_of<S>;
    o.prepare = prepare3<S>;
    o.case_bytes = sizeof(Case3<S>);
    o.batch_case = batch_case3<S>;
    o.batch_step = batch_step3<S>;
    return o;
}

}  // namespace
