/*
 * FP64 CPU oracle for the D2Q9I lattice-BGK stream-and-collide update.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call this file:
 * only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * leg use it. It shares no source with the CUDA path.
 *
 * What it computes (PortLBM, arXiv 2607.20650, Sec. 3.1):
 *   Eq. (1)  f_i(r + c_i, t + 1) = f_i(r, t) - (1/tau) [f_i(r, t) - f_i^eq(r, t)]
 *   Eq. (2)  f_i^eq = w_i [rho + 3 v.c_i + 9/2 (v.c_i)^2 - 3/2 v^2],
 *            v = sum_i f_i c_i   (D2Q9I: no division by rho),
 *            w_4 = 4/9, w_{1,3,5,7} = 1/9, w_{0,2,6,8} = 1/36.
 *   Directions (Fig. 2, the collision layout's order): i = 0..8 is
 *   SW, S, SE, W, rest, E, NW, N, NE, i.e. c_i = (i%3 - 1, i/3 - 1).
 *
 * Algorithm: the plain two-lattice one-step pull of Sec. 3.3 (every node pulls
 * c_i-neighbour values of the source lattice, collides, writes a second
 * lattice). One canonical storage order only: h[i*N + n], n = y*nx + x.
 *
 * Representation: populations are held as deviations h_i = f_i - w_i from the
 * rest weights. Since sum_i w_i = 1 and sum_i w_i c_i = 0, Eq. (2) becomes
 *   h_i^eq = w_i [(rho - 1) + 3 v.c_i + 9/2 (v.c_i)^2 - 3/2 v^2],
 * rho = 1 + sum_i h_i, v = sum_i h_i c_i, and Eq. (1) holds unchanged for h.
 * This is the same update; it only keeps the O(1) rest weight out of the
 * rounding (FP64 mass then drifts by 0 instead of ~1e-12 over 2e4 steps).
 *
 * Additions the paper does not print (readings, stated once here):
 *   - Guo body force F (not in the paper): v = sum_i h_i c_i + F/2 and the
 *     source (1 - omega/2) w_i [3 (c_i - v) + 9 (c_i.v) c_i] . F is added.
 *   - Sec. 3.1 boundary list: half-way bounce-back at fluid-solid links
 *     (the population arriving from a solid node is the node's own opposite
 *     population). Domain edges are periodic, a half-way wall, specular
 *     free-slip (south/north), an incompressible Zou-He velocity inlet or an
 *     equilibrium inlet with Dirichlet (rho = 1) or Neumann density (rho of
 *     node (1, y) in the previous state) (west), a zero-gradient outflow
 *     (source column clamped into the domain) or a Zou-He pressure outlet
 *     (rho = rho_out, v_y = 0) (east).
 *   - A fluid node whose eight pull sources are all solid or wall exchanges
 *     nothing with the flow; it is treated as solid.
 *   - Solid nodes hold h = 0 and are never written; their moments are
 *     reported as rho = 1, v = 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { BC_PERIODIC = 0, BC_WALL = 1, BC_FREESLIP = 2, BC_INLET_ZOUHE = 3,
       BC_INLET_EQ = 4, BC_OUTFLOW_ZG = 5, BC_INLET_EQ_NEUMANN = 6, BC_OUTLET_PRESSURE = 7 };
enum { PULL_NODE = 0, PULL_BOUNCE = 1, PULL_UNKNOWN = 2 };

typedef struct {
    int32_t nx, ny;
    double tau;            /* relaxation time; INFINITY gives omega = 0 */
    double fx, fy;         /* Guo body force */
    double ux_in, uy_in;   /* inlet velocity */
    int32_t bc_w, bc_e, bc_s, bc_n;
    double rho_out;        /* outlet density for BC_OUTLET_PRESSURE */
} oracle_params;

/* Fig. 2 direction order: c_i = (i%3 - 1, i/3 - 1). */
static const int CX[9] = {-1, 0, 1, -1, 0, 1, -1, 0, 1};
static const int CY[9] = {-1, -1, -1, 0, 0, 0, 1, 1, 1};
/* Eq. (2) weights. */
static const double W[9] = {1.0 / 36, 1.0 / 9, 1.0 / 36, 1.0 / 9, 4.0 / 9,
                            1.0 / 9, 1.0 / 36, 1.0 / 9, 1.0 / 36};

static int opposite(int i) { return 8 - i; }
/* The direction with the same c_x and the opposite c_y. */
static int mirror_y(int i) { return (i % 3) + 3 * (2 - i / 3); }

int oracle_omp_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Thread count of the following parallel loops (timing on one core). */
void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Eq. (2) in deviation form: h_i^eq for density deviation drho = rho - 1. */
void oracle_equilibrium(double drho, double ux, double uy, double *heq) {
    double usq = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        double cu = CX[i] * ux + CY[i] * uy;
        heq[i] = W[i] * (drho + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
    }
}

/*
 * Where the value pulled by node (x, y) in direction i comes from.
 * Sources outside the domain in y are mapped first (periodic wrap, wall,
 * or free-slip mirror onto the node's own row with direction mirror_y(i)),
 * then in x (periodic wrap, wall, outflow clamp, or inlet = unknown).
 */
static int pull_source(const oracle_params *p, int x, int y, int i,
                       int *xs, int *ys, int *j) {
    int sx = x - CX[i], sy = y - CY[i], d = i;
    if (sy < 0 || sy >= p->ny) {
        int bc = sy < 0 ? p->bc_s : p->bc_n;
        if (bc == BC_PERIODIC) {
            sy = (sy + p->ny) % p->ny;
        } else if (bc == BC_FREESLIP) {
            sy = y;
            d = mirror_y(i);
        } else {
            return PULL_BOUNCE;
        }
    }
    if (sx < 0 || sx >= p->nx) {
        int bc = sx < 0 ? p->bc_w : p->bc_e;
        if (bc == BC_PERIODIC) {
            sx = (sx + p->nx) % p->nx;
        } else if (bc == BC_OUTFLOW_ZG) {
            sx = sx < 0 ? 0 : p->nx - 1;
        } else if (bc == BC_INLET_ZOUHE || bc == BC_INLET_EQ || bc == BC_INLET_EQ_NEUMANN ||
                   bc == BC_OUTLET_PRESSURE) {
            return PULL_UNKNOWN;
        } else {
            return PULL_BOUNCE;
        }
    }
    *xs = sx;
    *ys = sy;
    *j = d;
    return PULL_NODE;
}

/* Solid as given, plus fluid nodes whose eight pull sources are all solid/wall. */
void oracle_effective_solid(const oracle_params *p, const uint8_t *mask, uint8_t *solid) {
    int nx = p->nx, ny = p->ny;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int64_t n = (int64_t)y * nx + x;
            if (mask[n]) { solid[n] = 1; continue; }
            int open = 0;
            for (int i = 0; i < 9; ++i) {
                if (i == 4) continue;
                int xs, ys, j;
                int k = pull_source(p, x, y, i, &xs, &ys, &j);
                if (k == PULL_UNKNOWN || (k == PULL_NODE && !mask[(int64_t)ys * nx + xs]))
                    open = 1;
            }
            solid[n] = open ? 0 : 1;
        }
}

/* Initial state: h = h^eq(rho - 1, v) on fluid nodes, 0 on solid nodes. */
void oracle_init(const oracle_params *p, const uint8_t *solid, const double *rho,
                 const double *ux, const double *uy, double *h) {
    int64_t N = (int64_t)p->nx * p->ny;
    for (int64_t n = 0; n < N; ++n) {
        double heq[9] = {0};
        if (!solid[n])
            oracle_equilibrium(rho ? rho[n] - 1.0 : 0.0, ux ? ux[n] : 0.0,
                               uy ? uy[n] : 0.0, heq);
        for (int i = 0; i < 9; ++i) h[i * N + n] = heq[i];
    }
}

/*
 * One update (pull, boundary substitution, moments, Eq. (1) with Eq. (2) and
 * the Guo source). Reads h_in, writes h_out; rho/ux/uy (may be NULL) receive
 * the moments computed inside this update from the pulled values.
 */
void oracle_step(const oracle_params *p, const uint8_t *solid, const double *h_in,
                 double *h_out, double *rho, double *ux, double *uy) {
    int nx = p->nx, ny = p->ny;
    int64_t N = (int64_t)nx * ny;
    double omega = 1.0 / p->tau;
    double fx = p->fx, fy = p->fy;

#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            int64_t n = (int64_t)y * nx + x;
            if (solid[n]) {
                if (rho) { rho[n] = 1.0; ux[n] = 0.0; uy[n] = 0.0; }
                continue;
            }
            double g[9];
            for (int i = 0; i < 9; ++i) {
                int xs, ys, j;
                int k = pull_source(p, x, y, i, &xs, &ys, &j);
                if (k == PULL_NODE && solid[(int64_t)ys * nx + xs]) k = PULL_BOUNCE;
                if (k == PULL_NODE)
                    g[i] = h_in[(int64_t)j * N + (int64_t)ys * nx + xs];
                else if (k == PULL_BOUNCE)
                    g[i] = h_in[(int64_t)opposite(i) * N + n];
                else
                    g[i] = NAN; /* filled by the inlet below */
            }
            if (x == 0 && p->bc_w == BC_INLET_ZOUHE) {
                /* Incompressible Zou-He velocity inlet: the three populations
                 * entering from the west follow from sum_i g_i c_i = U and
                 * bounce-back of the non-equilibrium normal part. */
                double Ux = p->ux_in, Uy = p->uy_in;
                g[5] = g[3] + (2.0 / 3.0) * Ux;
                g[8] = g[0] + 0.5 * (g[1] - g[7]) + Ux / 6.0 + Uy / 2.0;
                g[2] = g[6] + 0.5 * (g[7] - g[1]) + Ux / 6.0 - Uy / 2.0;
            } else if (x == 0 && p->bc_w == BC_INLET_EQ) {
                /* Equilibrium inlet with Dirichlet density rho = 1. */
                oracle_equilibrium(0.0, p->ux_in, p->uy_in, g);
            } else if (x == 0 && p->bc_w == BC_INLET_EQ_NEUMANN) {
                /* Equilibrium inlet, zero density gradient: rho of node (1, y)
                 * in the previous state (collision conserves mass, so the
                 * post-collision sum is that node's density). */
                double d = 0.0;
                int64_t m = n + 1;
                if (!solid[m])
                    for (int i = 0; i < 9; ++i) d += h_in[(int64_t)i * N + m];
                oracle_equilibrium(d, p->ux_in, p->uy_in, g);
            }
            if (x == nx - 1 && p->bc_e == BC_OUTLET_PRESSURE) {
                /* Zou-He pressure outlet: rho = rho_out and v_y = 0 fix the
                 * three populations entering from the east together with
                 * bounce-back of the normal non-equilibrium part. */
                double dr = p->rho_out - 1.0;
                double ux = 2.0 * (g[2] + g[5] + g[8]) + (g[1] + g[4] + g[7]) - dr;
                g[3] = g[5] - (2.0 / 3.0) * ux;
                g[6] = g[2] + 0.5 * (g[1] - g[7]) - ux / 6.0;
                g[0] = g[8] + 0.5 * (g[7] - g[1]) - ux / 6.0;
            }
            double drho = 0.0, jx = 0.0, jy = 0.0;
            for (int i = 0; i < 9; ++i) {
                drho += g[i];
                jx += g[i] * CX[i];
                jy += g[i] * CY[i];
            }
            double vx = jx + 0.5 * fx, vy = jy + 0.5 * fy;
            double heq[9];
            oracle_equilibrium(drho, vx, vy, heq);
            for (int i = 0; i < 9; ++i) {
                double cv = CX[i] * vx + CY[i] * vy;
                double cF = CX[i] * fx + CY[i] * fy;
                double vF = vx * fx + vy * fy;
                double src = (1.0 - 0.5 * omega) * W[i] * (3.0 * (cF - vF) + 9.0 * cv * cF);
                h_out[(int64_t)i * N + n] = g[i] - omega * (g[i] - heq[i]) + src;
            }
            if (rho) { rho[n] = 1.0 + drho; ux[n] = vx; uy[n] = vy; }
        }
    }
}

/* nsteps updates from h (in place); moments of the last update to rho/ux/uy. */
int oracle_run(const oracle_params *p, const uint8_t *solid, double *h, int64_t nsteps,
               double *rho, double *ux, double *uy) {
    int64_t N = (int64_t)p->nx * p->ny;
    double *tmp = (double *)malloc(sizeof(double) * 9 * N);
    if (!tmp) return -1;
    memcpy(tmp, h, sizeof(double) * 9 * N); /* solid nodes are never written */
    double *a = h, *b = tmp;
    for (int64_t t = 0; t < nsteps; ++t) {
        int last = (t == nsteps - 1);
        oracle_step(p, solid, a, b, last ? rho : NULL, last ? ux : NULL, last ? uy : NULL);
        double *s = a; a = b; b = s;
    }
    if (a != h) memcpy(h, a, sizeof(double) * 9 * N);
    free(tmp);
    return 0;
}

/* Total mass sum over fluid nodes of rho = 1 + sum_i h_i (compensated sum). */
double oracle_mass(const oracle_params *p, const uint8_t *solid, const double *h) {
    int64_t N = (int64_t)p->nx * p->ny;
    double s = 0.0, c = 0.0;
    for (int64_t n = 0; n < N; ++n) {
        if (solid[n]) continue;
        double r = 1.0;
        for (int i = 0; i < 9; ++i) r += h[(int64_t)i * N + n];
        double yk = r - c, tk = s + yk;
        c = (tk - s) - yk;
        s = tk;
    }
    return s;
}

/*
 * Momentum-exchange force on the nodes flagged in body (a subset of the solid
 * nodes): every link from a fluid node x to a body node x + c_i carries
 * 2 c_i f*_i(x), f* = w + h the stored post-collision populations.
 * Neighbours across a periodic edge wrap; other edges end the link.
 */
void oracle_force(const oracle_params *p, const uint8_t *solid, const uint8_t *body,
                  const double *h, double *F) {
    int nx = p->nx, ny = p->ny;
    int64_t N = (int64_t)nx * ny;
    double Fx = 0.0, Fy = 0.0;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int64_t n = (int64_t)y * nx + x;
            if (solid[n]) continue;
            for (int i = 0; i < 9; ++i) {
                if (i == 4) continue;
                int bx = x + CX[i], by = y + CY[i];
                if (bx < 0 || bx >= nx) {
                    if (p->bc_w != BC_PERIODIC) continue;
                    bx = (bx + nx) % nx;
                }
                if (by < 0 || by >= ny) {
                    if (p->bc_s != BC_PERIODIC) continue;
                    by = (by + ny) % ny;
                }
                int64_t m = (int64_t)by * nx + bx;
                if (!body[m]) continue;
                double f = W[i] + h[(int64_t)i * N + n];
                Fx += 2.0 * CX[i] * f;
                Fy += 2.0 * CY[i] * f;
            }
        }
    F[0] = Fx;
    F[1] = Fy;
}
