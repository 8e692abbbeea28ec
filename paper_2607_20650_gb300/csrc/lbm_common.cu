// Kernels shared by all storage types: link bytes from the solid mask,
// fluid count, the second pass of the FP64 reductions, the update counter,
// and the standalone store codec.
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

// Link byte per node: bit link_bit(i) set when the value pulled in direction
// i bounces back (mapped source solid, or a wall edge); a solid node, or a
// fluid node all of whose eight pulls bounce, gets SOLID_LINKS.
__global__ void k_links(Geo g, const uint8_t *mask, uint8_t *links) {
    const uint32_t N = (uint32_t)g.nx * (uint32_t)g.ny;
    const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    if (mask[n]) {
        links[n] = SOLID_LINKS;
        return;
    }
    const int y = (int)(n / (uint32_t)g.nx), x = (int)(n - (uint32_t)y * (uint32_t)g.nx);
    uint32_t bits = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        if (i == 4) continue;
        int xs, ys, j;
        const int k = map_pull(g, x, y, i, xs, ys, j);
        const bool bounce =
            k == PULL_BOUNCE || (k == PULL_NODE && mask[(uint32_t)ys * (uint32_t)g.nx + (uint32_t)xs]);
        if (bounce) bits |= 1u << link_bit(i);
    }
    links[n] = (uint8_t)bits;  // 0xFF: isolated fluid node, treated as solid
}

__global__ void k_count_fluid(const uint8_t *links, uint32_t N, unsigned long long *out) {
    unsigned long long c = 0;
    for (uint64_t n = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (uint64_t)gridDim.x * blockDim.x)
        c += links[n] != SOLID_LINKS;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, c);
}

// Fixed-order sum of the per-block partials (one thread: deterministic).
__global__ void k_sum_partials(const double *partials, int nblocks, int width, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int w = 0; w < width; ++w) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partials[b * width + w];
        out[w] = s;
    }
}

__global__ void k_bump(long long *ctr, long long by) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *ctr += by;
}

template <class S>
__global__ void k_quantize(int sr, uint64_t seed, uint32_t t, const float *in, S *out, float *back,
                           int64_t count) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const uint32_t n = (uint32_t)(k / 9);
    const int i = (int)(k % 9);
    const uint32_t r = sr ? pop_rand(node_key(step_key(seed, t), n), i) : 0u;
    const S e = Codec<S>::enc(in[k], sr != 0, r);
    out[k] = e;
    if (back) back[k] = Codec<S>::dec(e);
}

cudaError_t launch_links(int nx, int ny, int bw, int be, int bs, int bn, const uint8_t *mask,
                         uint8_t *links, cudaStream_t st) {
    const uint64_t N = (uint64_t)nx * (uint64_t)ny;
    k_links<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(Geo{nx, ny, bw, be, bs, bn}, mask, links);
    return cudaGetLastError();
}

cudaError_t launch_count_fluid(const uint8_t *links, int64_t N, unsigned long long *out,
                               cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_count_fluid<<<1024, 256, 0, st>>>(links, (uint32_t)N, out);
    return cudaGetLastError();
}

cudaError_t launch_sum_partials(const double *partials, int nblocks, int width, double *out,
                                cudaStream_t st) {
    k_sum_partials<<<1, 32, 0, st>>>(partials, nblocks, width, out);
    return cudaGetLastError();
}

cudaError_t launch_bump_counter(long long *ctr, long long by, cudaStream_t st) {
    k_bump<<<1, 32, 0, st>>>(ctr, by);
    return cudaGetLastError();
}

cudaError_t launch_quantize(int storage, int rounding, uint64_t seed, int64_t t, const float *in,
                            void *out, float *back, int64_t count, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const unsigned g = (unsigned)((count + 255) / 256);
    if (storage == 2)
        k_quantize<__half><<<g, 256, 0, st>>>(rounding, seed, (uint32_t)t, in, (__half *)out, back, count);
    else if (storage == 3)
        k_quantize<__nv_bfloat16><<<g, 256, 0, st>>>(rounding, seed, (uint32_t)t, in,
                                                     (__nv_bfloat16 *)out, back, count);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace lbm
