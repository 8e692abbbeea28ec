// Host-side generator of the solid masks of the benchmark families (Sec. 4:
// Hagen-Poiseuille channel, obstacles in a channel, porous media, a wing at
// an angle of attack), for callers of the C ABI that do not build masks
// themselves. No GPU work and no lattice-Boltzmann arithmetic: a mask is an
// input of lbm_create / lbm3_create. The seeded generators produce the same
// masks as the package's Python input generator (the same splitmix64 streams
// and the same double-precision tests), so C and Python callers run the same
// workloads.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "lbm.h"
#include "lbm_capi_internal.h"

namespace {

// splitmix64 (Steele, Lea & Flood, OOPSLA 2014): one stream per use, seeded
// with seed ^ mix(stream_id * gamma + gamma); doubles are (x >> 11) 2^-53.
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct Stream {
    uint64_t state;
    Stream(uint64_t seed, uint64_t id) : state(seed ^ mix64(id * kGamma + kGamma)) {}
    double uniform() {
        state += kGamma;
        return (double)(mix64(state) >> 11) * 0x1p-53;
    }
};

inline int floor_i(double v) { return (int)std::floor(v); }
inline int ceil_i(double v) { return (int)std::ceil(v); }
inline int wrap(int v, int n) { return ((v % n) + n) % n; }

bool bad_size(int64_t nx, int64_t ny) { return nx < 1 || ny < 1 || nx * ny >= (int64_t(1) << 32); }

}  // namespace

extern "C" lbm_status lbm_mask_channel_walls(int32_t nx, int32_t ny, uint8_t *mask) {
    if (!mask || bad_size(nx, ny)) return lbm_fail(LBM_EINVAL, "lbm_mask_channel_walls: bad size or NULL mask");
    memset(mask, 0, (size_t)nx * ny);
    memset(mask, 1, (size_t)nx);
    memset(mask + (size_t)(ny - 1) * nx, 1, (size_t)nx);
    return LBM_OK;
}

extern "C" lbm_status lbm_mask_disc(int32_t nx, int32_t ny, double xc, double yc, double r, int32_t periodic,
                                    uint8_t *mask) {
    if (!mask || bad_size(nx, ny) || !(r >= 0.0) || !std::isfinite(xc) || !std::isfinite(yc))
        return lbm_fail(LBM_EINVAL, "lbm_mask_disc: bad arguments");
    const int x0 = floor_i(xc - r), x1 = ceil_i(xc + r), y0 = floor_i(yc - r), y1 = ceil_i(yc + r);
    for (int y = y0; y <= y1; ++y) {
        const double dy = (double)y - yc;
        for (int x = x0; x <= x1; ++x) {
            const double dx = (double)x - xc;
            if (!(dx * dx + dy * dy <= r * r)) continue;
            int X = x, Y = y;
            if (periodic) {
                X = wrap(x, nx);
                Y = wrap(y, ny);
            } else if (x < 0 || x >= nx || y < 0 || y >= ny) {
                continue;
            }
            mask[(size_t)Y * nx + X] = 1;
        }
    }
    return LBM_OK;
}

// Random overlapping discs on a periodic domain, added in the stream's order
// (centre u nx, v ny, radius rmin + (rmax - rmin) w, three uniforms per disc,
// drawn in batches of 256 discs) until the solid fraction is reached.
extern "C" lbm_status lbm_mask_porous_discs(int32_t nx, int32_t ny, uint64_t seed, double rmin, double rmax,
                                            double solid_fraction, uint8_t *mask) {
    if (!mask || bad_size(nx, ny) || !(rmin >= 0.0) || !(rmax >= rmin) || !(solid_fraction >= 0.0) ||
        !(solid_fraction < 1.0))
        return lbm_fail(LBM_EINVAL, "lbm_mask_porous_discs: bad arguments");
    memset(mask, 0, (size_t)nx * ny);
    Stream rng(seed, 1);
    const double target = solid_fraction * (double)nx * (double)ny;
    int64_t solid = 0;
    while ((double)solid < target) {
        double batch[3 * 256];
        for (double &v : batch) v = rng.uniform();
        for (int k = 0; k < 256; ++k) {
            const double xc = batch[3 * k] * nx, yc = batch[3 * k + 1] * ny;
            const double r = rmin + (rmax - rmin) * batch[3 * k + 2];
            const int x0 = floor_i(xc - r), x1 = ceil_i(xc + r), y0 = floor_i(yc - r), y1 = ceil_i(yc + r);
            for (int y = y0; y <= y1; ++y) {
                const double dy = (double)y - yc;
                for (int x = x0; x <= x1; ++x) {
                    const double dx = (double)x - xc;
                    if (!(dx * dx + dy * dy <= r * r)) continue;
                    uint8_t &m = mask[(size_t)wrap(y, ny) * nx + wrap(x, nx)];
                    solid += m == 0;
                    m = 1;
                }
            }
            if ((double)solid >= target) break;
        }
    }
    return LBM_OK;
}

// NACA 4-digit airfoil (camber m, its position p, thickness t; 2412 = 0.02,
// 0.4, 0.12) of the given chord from the closed-form thickness (closed
// trailing edge, last coefficient -0.1036) and camber-line equations, cosine
// spacing of n_points per side, leading edge at (nx/4, ny/2), rotated nose-up
// by aoa_deg about the quarter chord; nodes inside the outline (even-odd
// rule, scanlines) are solid.
extern "C" lbm_status lbm_mask_naca4(int32_t nx, int32_t ny, double chord, double m, double p, double t,
                                     double aoa_deg, int32_t n_points, uint8_t *mask) {
    if (!mask || bad_size(nx, ny) || !(chord > 0.0) || !(p > 0.0 && p < 1.0) || !(t > 0.0) || n_points < 3)
        return lbm_fail(LBM_EINVAL, "lbm_mask_naca4: bad arguments");
    const int n = n_points;
    std::vector<double> xu(n), yu(n), xl(n), yl(n);
    const double pi = 3.14159265358979323846;
    const double step = pi / (double)(n - 1);
    for (int k = 0; k < n; ++k) {
        const double beta = k == n - 1 ? pi : (double)k * step;   // evenly spaced, ends exact
        const double xc = 0.5 * (1.0 - std::cos(beta));
        const double yt = 5.0 * t * (0.2969 * std::sqrt(xc) - 0.1260 * xc - 0.3516 * (xc * xc) +
                                     0.2843 * std::pow(xc, 3.0) - 0.1036 * std::pow(xc, 4.0));
        double yc, dyc;
        if (xc < p) {
            yc = m / (p * p) * (2 * p * xc - xc * xc);
            dyc = 2 * m / (p * p) * (p - xc);
        } else {
            yc = m / ((1 - p) * (1 - p)) * ((1 - 2 * p) + 2 * p * xc - xc * xc);
            dyc = 2 * m / ((1 - p) * (1 - p)) * (p - xc);
        }
        const double th = std::atan(dyc);
        xu[k] = xc - yt * std::sin(th);
        yu[k] = yc + yt * std::cos(th);
        xl[k] = xc + yt * std::sin(th);
        yl[k] = yc - yt * std::cos(th);
    }
    // outline: upper surface trailing edge -> leading edge, then lower surface
    std::vector<double> px, py;
    px.reserve(2 * n);
    py.reserve(2 * n);
    for (int k = n - 1; k >= 0; --k) {
        px.push_back(xu[k] * chord);
        py.push_back(yu[k] * chord);
    }
    for (int k = 1; k < n; ++k) {
        px.push_back(xl[k] * chord);
        py.push_back(yl[k] * chord);
    }
    const double a = -(aoa_deg * (pi / 180.0)), ca = std::cos(a), sa = std::sin(a), qc = 0.25 * chord;
    double ymin = INFINITY, ymax = -INFINITY;
    for (size_t k = 0; k < px.size(); ++k) {
        const double x = px[k] - qc, y = py[k];
        px[k] = (x * ca - y * sa) + qc + nx / 4.0;
        py[k] = (x * sa + y * ca) + ny / 2.0;
        ymin = std::fmin(ymin, py[k]);
        ymax = std::fmax(ymax, py[k]);
    }
    memset(mask, 0, (size_t)nx * ny);
    const size_t np = px.size();
    std::vector<double> xs;
    for (int yy = std::max(0, floor_i(ymin)); yy <= std::min(ny - 1, ceil_i(ymax)); ++yy) {
        const double Y = (double)yy;
        xs.clear();
        for (size_t k = 0; k < np; ++k) {
            const size_t k1 = (k + 1) % np;
            const double y0 = py[k], y1 = py[k1];
            if ((y0 <= Y && y1 > Y) || (y1 <= Y && y0 > Y))
                xs.push_back(px[k] + (Y - y0) * (px[k1] - px[k]) / (y1 - y0));
        }
        std::sort(xs.begin(), xs.end());
        for (size_t k = 0; k + 1 < xs.size(); k += 2) {
            const int lo = std::max(0, ceil_i(xs[k])), hi = std::min(nx - 1, floor_i(xs[k + 1]));
            for (int x = lo; x <= hi; ++x) mask[(size_t)yy * nx + x] = 1;
        }
    }
    return LBM_OK;
}

// Random overlapping spheres on a periodic box (mask[(z ny + y) nx + x]),
// the 3-D counterpart of lbm_mask_porous_discs: four uniforms per sphere
// (centre u nx, v ny, s nz, radius rmin + (rmax - rmin) w), batches of 256.
extern "C" lbm_status lbm3_mask_porous_spheres(int32_t nx, int32_t ny, int32_t nz, uint64_t seed, double rmin,
                                               double rmax, double solid_fraction, uint8_t *mask) {
    if (!mask || nx < 1 || ny < 1 || nz < 1 || (int64_t)nx * ny * nz >= (int64_t(1) << 32) || !(rmin >= 0.0) ||
        !(rmax >= rmin) || !(solid_fraction >= 0.0) || !(solid_fraction < 1.0))
        return lbm_fail(LBM_EINVAL, "lbm3_mask_porous_spheres: bad arguments");
    memset(mask, 0, (size_t)nx * ny * nz);
    Stream rng(seed, 5);
    const double target = solid_fraction * (double)nx * (double)ny * (double)nz;
    int64_t solid = 0;
    while ((double)solid < target) {
        double batch[4 * 256];
        for (double &v : batch) v = rng.uniform();
        for (int k = 0; k < 256; ++k) {
            const double xc = batch[4 * k] * nx, yc = batch[4 * k + 1] * ny, zc = batch[4 * k + 2] * nz;
            const double r = rmin + (rmax - rmin) * batch[4 * k + 3];
            for (int z = floor_i(zc - r); z <= ceil_i(zc + r); ++z) {
                const double dz = (double)z - zc;
                for (int y = floor_i(yc - r); y <= ceil_i(yc + r); ++y) {
                    const double dy = (double)y - yc;
                    for (int x = floor_i(xc - r); x <= ceil_i(xc + r); ++x) {
                        const double dx = (double)x - xc;
                        if (!(dx * dx + dy * dy + dz * dz <= r * r)) continue;
                        uint8_t &mm = mask[((size_t)wrap(z, nz) * ny + wrap(y, ny)) * nx + wrap(x, nx)];
                        solid += mm == 0;
                        mm = 1;
                    }
                }
            }
            if ((double)solid >= target) break;
        }
    }
    return LBM_OK;
}
