/*
 * FP64 CPU oracle for the D3Q19 incompressible lattice-BGK update: the
 * three-dimensional extension PortLBM names as future work (Sec. 6), built
 * with the same method as the D2Q9I update of Sec. 3.1.
 *
 * TEST INFRASTRUCTURE ONLY (see lbm_oracle.c); shares no source with the CUDA
 * path.
 *
 *   Eq. (1)  f_i(r + c_i, t + 1) = f_i(r, t) - (1/tau) [f_i(r, t) - f_i^eq(r, t)]
 *   Eq. (2)  f_i^eq = w_i [rho + 3 v.c_i + 9/2 (v.c_i)^2 - 3/2 v^2], v = sum_i f_i c_i
 *   D3Q19: c_i = the 19 vectors of {-1,0,1}^3 with |c|^2 <= 2 in lexicographic
 *   order of (c_z, c_y, c_x); opposite(i) = 18 - i; w = 1/3 (rest), 1/18
 *   (faces), 1/36 (edges).
 *
 * Two-lattice pull on the canonical layout h[i*N + n], n = (z*ny + y)*nx + x,
 * h = f - w. Faces: periodic or half-way wall per axis; on the x axis the
 * west face may instead be an equilibrium inlet (the x = 0 plane set to
 * f^eq(rho = 1, u_in) before the collision, the 3-D form of the 2-D
 * oracle's Dirichlet equilibrium inlet) or an incompressible Zou-He velocity
 * inlet, and the east face a zero-gradient outflow (the pulled source plane
 * x = nx clamped to nx - 1) or a Zou-He pressure outlet. Pulls are mapped in
 * z, then y, then x, as the 2-D oracle maps y before x. Solid nodes bounce
 * back; Guo body force as in the 2-D oracle. A fluid node all of whose 18
 * pulls bounce (or come from outside an inlet or outlet face) is treated as
 * solid.
 *
 * Zou-He faces in 3-D (the 2-D oracle's Sec. 3.1 inlet and "adapted Zou and
 * He" outlet, written for the 19 velocities). At the west face the five
 * populations with c_x = +1 are unknown; with T_y, T_z the y and z momentum
 * of the nine c_x = 0 populations, sum_i g_i c_i = U and bounce-back of the
 * normal non-equilibrium part give
 *   g(1,0,0)   = g(-1,0,0)  + U_x / 3
 *   g(1,+-1,0) = g(-1,-+1,0) + (U_x +- U_y) / 6 -+ (T_y / 2 - U_y / 3)
 *   g(1,0,+-1) = g(-1,0,-+1) + (U_x +- U_z) / 6 -+ (T_z / 2 - U_z / 3).
 * At the east face rho = rho_out and v_y = v_z = 0 fix the five c_x = -1
 * populations: with H+, H0 the sums of the known c_x = +1 and c_x = 0
 * deviations, u_x = 2 H+ + H0 - (rho_out - 1), and
 *   g(-1,0,0)   = g(1,0,0)   - u_x / 3
 *   g(-1,+-1,0) = g(1,-+1,0) - u_x / 6 -+ T_y / 2
 *   g(-1,0,+-1) = g(1,0,-+1) - u_x / 6 -+ T_z / 2.
 * Both hold unchanged for the deviations h (opposite weights are equal), and
 * summed over c_z they are the 2-D oracle's formulas.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { F3_PERIODIC = 0, F3_WALL = 1, F3_INLET_ZOUHE = 3, F3_INLET_EQ = 4, F3_OUTFLOW_ZG = 5,
       F3_OUTLET_PRESSURE = 7 };
enum { P3_NODE = 0, P3_BOUNCE = 1 };

typedef struct {
    int32_t nx, ny, nz;
    double tau;
    double fx, fy, fz;
    int32_t bc_x, bc_y, bc_z;   /* per axis: both faces periodic or both walls; bc_x: the west face */
    int32_t bc_xe;              /* east face: periodic (with bc_x), wall, zero-gradient outflow or
                                   pressure outlet */
    double ux_in, uy_in, uz_in; /* inlet velocity (bc_x = F3_INLET_EQ or F3_INLET_ZOUHE) */
    double rho_out;             /* outlet density (bc_xe = F3_OUTLET_PRESSURE) */
} oracle3_params;

static int C3[19][3];
static double W3[19];
static int tables_ready = 0;

static void tables(void) {
    if (tables_ready) return;
    int k = 0;
    for (int cz = -1; cz <= 1; ++cz)
        for (int cy = -1; cy <= 1; ++cy)
            for (int cx = -1; cx <= 1; ++cx) {
                int q = cx * cx + cy * cy + cz * cz;
                if (q > 2) continue;
                C3[k][0] = cx;
                C3[k][1] = cy;
                C3[k][2] = cz;
                W3[k] = q == 0 ? 1.0 / 3.0 : (q == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
                ++k;
            }
    tables_ready = 1;
}

void oracle3_directions(int32_t *c, double *w) {
    tables();
    for (int i = 0; i < 19; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = C3[i][a];
        w[i] = W3[i];
    }
}

void oracle3_equilibrium(double drho, double ux, double uy, double uz, double *heq) {
    tables();
    double usq = ux * ux + uy * uy + uz * uz;
    for (int i = 0; i < 19; ++i) {
        double cu = C3[i][0] * ux + C3[i][1] * uy + C3[i][2] * uz;
        heq[i] = W3[i] * (drho + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
    }
}

/* Source of the value pulled by (x, y, z) in direction i: z and y wrap or
 * bounce; x wraps, bounces, is clamped (outflow) or unknown (inlet or
 * pressure outlet, marked as a bounce: those values are replaced before the
 * collision). */
static int pull3(const oracle3_params *p, int x, int y, int z, int i, int64_t *src) {
    int s[3] = {x - C3[i][0], y - C3[i][1], z - C3[i][2]};
    const int ext[3] = {p->nx, p->ny, p->nz};
    const int bc[3] = {p->bc_x, p->bc_y, p->bc_z};
    for (int a = 2; a >= 1; --a) {
        if (s[a] < 0 || s[a] >= ext[a]) {
            if (bc[a] != F3_PERIODIC) return P3_BOUNCE;
            s[a] = (s[a] + ext[a]) % ext[a];
        }
    }
    if (s[0] < 0 || s[0] >= p->nx) {
        const int kind = s[0] < 0 ? p->bc_x : p->bc_xe;
        if (kind == F3_PERIODIC) s[0] = (s[0] + p->nx) % p->nx;
        else if (kind == F3_OUTFLOW_ZG) s[0] = s[0] < 0 ? 0 : p->nx - 1;
        else return P3_BOUNCE;   /* wall, or inlet (unknown) */
    }
    *src = ((int64_t)s[2] * p->ny + s[1]) * p->nx + s[0];
    return P3_NODE;
}

void oracle3_effective_solid(const oracle3_params *p, const uint8_t *mask, uint8_t *solid) {
    tables();
    int64_t n = 0;
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x, ++n) {
                if (mask[n]) { solid[n] = 1; continue; }
                int open = 0;
                for (int i = 0; i < 19; ++i) {
                    if (i == 9) continue;
                    int64_t s;
                    if (pull3(p, x, y, z, i, &s) == P3_NODE && !mask[s]) open = 1;
                }
                solid[n] = open ? 0 : 1;
            }
}

void oracle3_init(const oracle3_params *p, const uint8_t *solid, const double *rho, const double *ux,
                  const double *uy, const double *uz, double *h) {
    tables();
    int64_t N = (int64_t)p->nx * p->ny * p->nz;
    for (int64_t n = 0; n < N; ++n) {
        double heq[19] = {0};
        if (!solid[n])
            oracle3_equilibrium(rho ? rho[n] - 1.0 : 0.0, ux ? ux[n] : 0.0, uy ? uy[n] : 0.0,
                                uz ? uz[n] : 0.0, heq);
        for (int i = 0; i < 19; ++i) h[i * N + n] = heq[i];
    }
}

/* Index of the direction (cx, cy, cz). */
static int dir3(int cx, int cy, int cz) {
    for (int i = 0; i < 19; ++i)
        if (C3[i][0] == cx && C3[i][1] == cy && C3[i][2] == cz) return i;
    return -1;
}

/* y and z momentum of the nine populations with c_x = 0. */
static void transverse3(const double *g, double *ty, double *tz) {
    *ty = 0.0;
    *tz = 0.0;
    for (int i = 0; i < 19; ++i) {
        if (C3[i][0] != 0) continue;
        *ty += C3[i][1] * g[i];
        *tz += C3[i][2] * g[i];
    }
}

/* Zou-He velocity inlet on the west face (formulas in the header). */
static void zou_he_inlet3(const oracle3_params *p, double *g) {
    const double Ux = p->ux_in, Uy = p->uy_in, Uz = p->uz_in;
    double ty, tz;
    transverse3(g, &ty, &tz);
    const double ny_ = 0.5 * ty - Uy / 3.0, nz_ = 0.5 * tz - Uz / 3.0;
    g[dir3(1, 0, 0)] = g[dir3(-1, 0, 0)] + Ux / 3.0;
    g[dir3(1, 1, 0)] = g[dir3(-1, -1, 0)] + (Ux + Uy) / 6.0 - ny_;
    g[dir3(1, -1, 0)] = g[dir3(-1, 1, 0)] + (Ux - Uy) / 6.0 + ny_;
    g[dir3(1, 0, 1)] = g[dir3(-1, 0, -1)] + (Ux + Uz) / 6.0 - nz_;
    g[dir3(1, 0, -1)] = g[dir3(-1, 0, 1)] + (Ux - Uz) / 6.0 + nz_;
}

/* Zou-He pressure outlet on the east face (formulas in the header). */
static void zou_he_outlet3(const oracle3_params *p, double *g) {
    double hp = 0.0, h0 = 0.0;
    for (int i = 0; i < 19; ++i) {
        if (C3[i][0] > 0) hp += g[i];
        if (C3[i][0] == 0) h0 += g[i];
    }
    const double ux = 2.0 * hp + h0 - (p->rho_out - 1.0);
    double ty, tz;
    transverse3(g, &ty, &tz);
    g[dir3(-1, 0, 0)] = g[dir3(1, 0, 0)] - ux / 3.0;
    g[dir3(-1, 1, 0)] = g[dir3(1, -1, 0)] - ux / 6.0 - 0.5 * ty;
    g[dir3(-1, -1, 0)] = g[dir3(1, 1, 0)] - ux / 6.0 + 0.5 * ty;
    g[dir3(-1, 0, 1)] = g[dir3(1, 0, -1)] - ux / 6.0 - 0.5 * tz;
    g[dir3(-1, 0, -1)] = g[dir3(1, 0, 1)] - ux / 6.0 + 0.5 * tz;
}

void oracle3_step(const oracle3_params *p, const uint8_t *solid, const double *h_in, double *h_out,
                  double *rho, double *ux, double *uy, double *uz) {
    tables();
    const int64_t N = (int64_t)p->nx * p->ny * p->nz;
    const double omega = 1.0 / p->tau;
    const double F[3] = {p->fx, p->fy, p->fz};
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                const int64_t n = ((int64_t)z * p->ny + y) * p->nx + x;
                if (solid[n]) {
                    if (rho) { rho[n] = 1.0; ux[n] = 0.0; uy[n] = 0.0; uz[n] = 0.0; }
                    continue;
                }
                double g[19];
                for (int i = 0; i < 19; ++i) {
                    int64_t s = 0;
                    int k = pull3(p, x, y, z, i, &s);
                    if (k == P3_NODE && solid[s]) k = P3_BOUNCE;
                    g[i] = k == P3_NODE ? h_in[(int64_t)i * N + s] : h_in[(int64_t)(18 - i) * N + n];
                }
                if (x == 0 && p->bc_x == F3_INLET_EQ)   /* Dirichlet equilibrium inlet */
                    oracle3_equilibrium(0.0, p->ux_in, p->uy_in, p->uz_in, g);
                if (x == 0 && p->bc_x == F3_INLET_ZOUHE) zou_he_inlet3(p, g);
                if (x == p->nx - 1 && p->bc_xe == F3_OUTLET_PRESSURE) zou_he_outlet3(p, g);
                double drho = 0.0, j[3] = {0.0, 0.0, 0.0};
                for (int i = 0; i < 19; ++i) {
                    drho += g[i];
                    for (int a = 0; a < 3; ++a) j[a] += g[i] * C3[i][a];
                }
                double v[3];
                for (int a = 0; a < 3; ++a) v[a] = j[a] + 0.5 * F[a];
                double heq[19];
                oracle3_equilibrium(drho, v[0], v[1], v[2], heq);
                const double vF = v[0] * F[0] + v[1] * F[1] + v[2] * F[2];
                for (int i = 0; i < 19; ++i) {
                    double cv = C3[i][0] * v[0] + C3[i][1] * v[1] + C3[i][2] * v[2];
                    double cF = C3[i][0] * F[0] + C3[i][1] * F[1] + C3[i][2] * F[2];
                    double src = (1.0 - 0.5 * omega) * W3[i] * (3.0 * (cF - vF) + 9.0 * cv * cF);
                    h_out[(int64_t)i * N + n] = g[i] - omega * (g[i] - heq[i]) + src;
                }
                if (rho) { rho[n] = 1.0 + drho; ux[n] = v[0]; uy[n] = v[1]; uz[n] = v[2]; }
            }
}

int oracle3_run(const oracle3_params *p, const uint8_t *solid, double *h, int64_t nsteps, double *rho,
                double *ux, double *uy, double *uz) {
    int64_t N = (int64_t)p->nx * p->ny * p->nz;
    double *tmp = (double *)malloc(sizeof(double) * 19 * N);
    if (!tmp) return -1;
    memcpy(tmp, h, sizeof(double) * 19 * N);
    double *a = h, *b = tmp;
    for (int64_t t = 0; t < nsteps; ++t) {
        int last = t == nsteps - 1;
        oracle3_step(p, solid, a, b, last ? rho : NULL, last ? ux : NULL, last ? uy : NULL, last ? uz : NULL);
        double *s = a; a = b; b = s;
    }
    if (a != h) memcpy(h, a, sizeof(double) * 19 * N);
    free(tmp);
    return 0;
}

double oracle3_mass(const oracle3_params *p, const uint8_t *solid, const double *h) {
    int64_t N = (int64_t)p->nx * p->ny * p->nz;
    double s = 0.0, c = 0.0;
    for (int64_t n = 0; n < N; ++n) {
        if (solid[n]) continue;
        double r = 1.0;
        for (int i = 0; i < 19; ++i) r += h[(int64_t)i * N + n];
        double yk = r - c, tk = s + yk;
        c = (tk - s) - yk;
        s = tk;
    }
    return s;
}

/* Momentum-exchange force on a body (the 3-D form of the 2-D oracle's):
 * sum over fluid nodes x and directions i with x + c_i a body node of
 * 2 c_i f*_i(x), f* = w + h the stored post-collision populations; links
 * across a non-periodic face are skipped. */
void oracle3_force(const oracle3_params *p, const uint8_t *solid, const uint8_t *body, const double *h,
                   double *F) {
    tables();
    const int64_t N = (int64_t)p->nx * p->ny * p->nz;
    const int ext[3] = {p->nx, p->ny, p->nz};
    const int bc[3] = {p->bc_x, p->bc_y, p->bc_z};
    double acc[3] = {0.0, 0.0, 0.0};
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                const int64_t n = ((int64_t)z * p->ny + y) * p->nx + x;
                if (solid[n]) continue;
                for (int i = 0; i < 19; ++i) {
                    if (i == 9) continue;
                    int b[3] = {x + C3[i][0], y + C3[i][1], z + C3[i][2]};
                    int inside = 1;
                    for (int a = 0; a < 3; ++a) {
                        if (b[a] < 0 || b[a] >= ext[a]) {
                            const int kind = a == 0 ? (b[0] < 0 ? p->bc_x : p->bc_xe) : bc[a];
                            if (kind != F3_PERIODIC) inside = 0;
                            b[a] = (b[a] + ext[a]) % ext[a];
                        }
                    }
                    if (!inside) continue;
                    const int64_t m = ((int64_t)b[2] * p->ny + b[1]) * p->nx + b[0];
                    if (!body[m]) continue;
                    const double f = W3[i] + h[(int64_t)i * N + n];
                    for (int a = 0; a < 3; ++a) acc[a] += 2.0 * C3[i][a] * f;
                }
            }
    for (int a = 0; a < 3; ++a) F[a] = acc[a];
}
