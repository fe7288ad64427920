/*
 * pb_oracle.c -- plain FP64 CPU oracle for the linear finite-difference
 * Poisson-Boltzmann (FDPB) solve of Qi, Botello-Smith & Luo (arXiv:1704.02745).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file.  It shares no code, header or
 * constant table with the CUDA library; both read the same seeded input arrays.
 *
 * Everything is FP64, single-threaded, explicit loops, built with
 * -ffp-contract=off so that every product and sum is rounded on its own.
 *
 * Array layouts (x fastest, all dense, no padding):
 *   node arrays   (nz, ny, nx)        index i + nx*(j + ny*k)
 *   ex            (nz, ny, nx+1)      ex[.. + (i+1)] = eps on the edge between
 *                                     x-nodes i and i+1, for i = -1 .. nx-1
 *   ey            (nz, ny+1, nx)      ey[(k*(ny+1) + (j+1))*nx + i], j = -1 .. ny-1
 *   ez            (nz+1, ny, nx)      ez[((k+1)*ny + j)*nx + i],     k = -1 .. nz-1
 * Node (i,j,k) sits at origin + (i*h, j*h, k*h), computed as o + i*h; the
 * midpoint of an x-edge as o + (i + 0.5)*h.  Dirichlet values live on the ghost
 * layer i = -1, i = nx (and likewise in y, z); the seven-point stencil reads
 * only face ghosts.
 *
 * Periodic grids (the periodic boundary of the paper's Fig. 2) have period
 * n*h on each axis and no ghost layer: node i's neighbours are i-1 and i+1
 * modulo n, and the edge array entry at i = -1 repeats the edge between
 * nodes n-1 and 0 (entry n-1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_NOT_CONVERGED 5
#define OR_BREAKDOWN 6

typedef struct {
    int nx, ny, nz;
    double h;
    double ox, oy, oz;
    double eps_in, eps_out;
    double kappa_d;    /* inverse Debye length, 1/A (0 for no salt)            */
    double kbar2_h2;   /* eps_out * kappa_d^2 * h^2: the Boltzmann diagonal term */
    int kappa_mask;    /* 1: lambda = 0 inside atoms; 0: lambda = 1 everywhere */
    int periodic;      /* 1: periodic on every axis (no ghost layer)            */
} or_grid;

static long wrap(long i, long n) { return ((i % n) + n) % n; }

static size_t nid(const or_grid *g, long i, long j, long k) {
    return (size_t)i + (size_t)g->nx * ((size_t)j + (size_t)g->ny * (size_t)k);
}
static size_t exid(const or_grid *g, long i, long j, long k) { /* edge i..i+1 */
    return (size_t)(i + 1) + (size_t)(g->nx + 1) * ((size_t)j + (size_t)g->ny * (size_t)k);
}
static size_t eyid(const or_grid *g, long i, long j, long k) { /* edge j..j+1 */
    return (size_t)i + (size_t)g->nx * ((size_t)(j + 1) + (size_t)(g->ny + 1) * (size_t)k);
}
static size_t ezid(const or_grid *g, long i, long j, long k) { /* edge k..k+1 */
    return (size_t)i + (size_t)g->nx * ((size_t)j + (size_t)g->ny * (size_t)(k + 1));
}

/* Square of the inverse Debye length (1/A^2) of a 1:1 electrolyte of ionic
 * strength I (mol/L) in a solvent of relative permittivity eps_out at T (K):
 * kappa^2 = 2 N_A e^2 (1000 I) / (eps0 eps_out k_B T), in m^-2, times 1e-20.
 * The paper absorbs every coefficient of the Boltzmann term of Eq. (2) into
 * kappa^2 of Eq. (3); this is that coefficient for the linearised term. */
double or_kappa_debye2(double ionic_M, double temp_K, double eps_out) {
    const double NA = 6.02214076e23, E = 1.602176634e-19;
    const double EPS0 = 8.8541878128e-12, KB = 1.380649e-23;
    double num = 2.0 * NA * E * E * (1000.0 * ionic_M);
    double den = EPS0 * eps_out * KB * temp_K;
    return num / den * 1e-20;
}

/* ------------------------------------------------------------------------- */
/* O1. Grid setup: dielectric edges (Eq. 3's eps_i, eps_j, eps_k), the ion-   */
/* exclusion mask lambda (Eq. 1-2), grid charges q(i,j,k) and the right-hand  */
/* side b of Eq. (4) with the Debye-Hueckel boundary folded in.               */
/* ------------------------------------------------------------------------- */

static long lmax(long a, long b) { return a > b ? a : b; }
static long lmin(long a, long b) { return a < b ? a : b; }

/* Strict inside test of a point against one atom sphere: |m - x_a|^2 < r_a^2,
 * summed in the order dx*dx + dy*dy + dz*dz. */
static int inside(double mx, double my, double mz, double ax, double ay, double az, double r2) {
    double dx = mx - ax, dy = my - ay, dz = mz - az;
    double d2 = dx * dx + dy * dy;
    d2 = d2 + dz * dz;
    return d2 < r2;
}

/* Dielectric on every edge and lambda on every node.  An edge takes eps_in when
 * its midpoint lies strictly inside any atom sphere, else eps_out; a node gets
 * lambda = 0 when it lies strictly inside any atom sphere (kappa_mask on).
 * Each atom visits the edges and nodes of its bounding box (plus one spacing
 * of margin); the exact test decides. */
void or_dielectric(const or_grid *g, int n_atoms, const double *xyz, const double *rad,
                   double *ex, double *ey, double *ez, uint8_t *lam) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const double h = g->h;
    size_t nex = (size_t)(nx + 1) * ny * nz, ney = (size_t)nx * (ny + 1) * nz,
           nez = (size_t)nx * ny * (nz + 1), nn = (size_t)nx * ny * nz;
    for (size_t t = 0; t < nex; t++) ex[t] = g->eps_out;
    for (size_t t = 0; t < ney; t++) ey[t] = g->eps_out;
    for (size_t t = 0; t < nez; t++) ez[t] = g->eps_out;
    for (size_t t = 0; t < nn; t++) lam[t] = 1;
    for (int a = 0; a < n_atoms; a++) {
        double ax = xyz[3 * a], ay = xyz[3 * a + 1], az = xyz[3 * a + 2], r = rad[a];
        double r2 = r * r;
        /* node-index bounding box, one spacing of margin on each side */
        long i0 = (long)floor((ax - r - g->ox) / h) - 1, i1 = (long)ceil((ax + r - g->ox) / h) + 1;
        long j0 = (long)floor((ay - r - g->oy) / h) - 1, j1 = (long)ceil((ay + r - g->oy) / h) + 1;
        long k0 = (long)floor((az - r - g->oz) / h) - 1, k1 = (long)ceil((az + r - g->oz) / h) + 1;
        /* x-edges: i = -1 .. nx-1 (edge between i and i+1) */
        for (long k = lmax(k0, 0); k <= lmin(k1, nz - 1); k++)
            for (long j = lmax(j0, 0); j <= lmin(j1, ny - 1); j++)
                for (long i = lmax(i0, -1); i <= lmin(i1, nx - 1); i++) {
                    double mx = g->ox + ((double)i + 0.5) * h;
                    double my = g->oy + (double)j * h;
                    double mz = g->oz + (double)k * h;
                    if (inside(mx, my, mz, ax, ay, az, r2)) ex[exid(g, i, j, k)] = g->eps_in;
                }
        /* y-edges */
        for (long k = lmax(k0, 0); k <= lmin(k1, nz - 1); k++)
            for (long j = lmax(j0, -1); j <= lmin(j1, ny - 1); j++)
                for (long i = lmax(i0, 0); i <= lmin(i1, nx - 1); i++) {
                    double mx = g->ox + (double)i * h;
                    double my = g->oy + ((double)j + 0.5) * h;
                    double mz = g->oz + (double)k * h;
                    if (inside(mx, my, mz, ax, ay, az, r2)) ey[eyid(g, i, j, k)] = g->eps_in;
                }
        /* z-edges */
        for (long k = lmax(k0, -1); k <= lmin(k1, nz - 1); k++)
            for (long j = lmax(j0, 0); j <= lmin(j1, ny - 1); j++)
                for (long i = lmax(i0, 0); i <= lmin(i1, nx - 1); i++) {
                    double mx = g->ox + (double)i * h;
                    double my = g->oy + (double)j * h;
                    double mz = g->oz + ((double)k + 0.5) * h;
                    if (inside(mx, my, mz, ax, ay, az, r2)) ez[ezid(g, i, j, k)] = g->eps_in;
                }
        /* nodes */
        if (g->kappa_mask)
            for (long k = lmax(k0, 0); k <= lmin(k1, nz - 1); k++)
                for (long j = lmax(j0, 0); j <= lmin(j1, ny - 1); j++)
                    for (long i = lmax(i0, 0); i <= lmin(i1, nx - 1); i++) {
                        double mx = g->ox + (double)i * h;
                        double my = g->oy + (double)j * h;
                        double mz = g->oz + (double)k * h;
                        if (inside(mx, my, mz, ax, ay, az, r2)) lam[nid(g, i, j, k)] = 0;
                    }
    }
}

/* The same map on a periodic grid: an edge takes eps_in when some periodic
 * image of its midpoint lies strictly inside an atom sphere, a node gets
 * lambda = 0 likewise.  Each atom visits its bounding box in unwrapped
 * indices (no clamping); points are placed at their unwrapped coordinates
 * o + i*h (i + 0.5 for midpoints), tested against the atom, and the result
 * lands on the element at the wrapped index.  The entry at i = -1 then copies
 * the edge between nodes n-1 and 0. */
void or_dielectric_periodic(const or_grid *g, int n_atoms, const double *xyz, const double *rad,
                            double *ex, double *ey, double *ez, uint8_t *lam) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const double h = g->h;
    size_t nex = (size_t)(nx + 1) * ny * nz, ney = (size_t)nx * (ny + 1) * nz,
           nez = (size_t)nx * ny * (nz + 1), nn = (size_t)nx * ny * nz;
    for (size_t t = 0; t < nex; t++) ex[t] = g->eps_out;
    for (size_t t = 0; t < ney; t++) ey[t] = g->eps_out;
    for (size_t t = 0; t < nez; t++) ez[t] = g->eps_out;
    for (size_t t = 0; t < nn; t++) lam[t] = 1;
    for (int a = 0; a < n_atoms; a++) {
        double ax = xyz[3 * a], ay = xyz[3 * a + 1], az = xyz[3 * a + 2], r = rad[a];
        double r2 = r * r;
        long i0 = (long)floor((ax - r - g->ox) / h) - 1, i1 = (long)ceil((ax + r - g->ox) / h) + 1;
        long j0 = (long)floor((ay - r - g->oy) / h) - 1, j1 = (long)ceil((ay + r - g->oy) / h) + 1;
        long k0 = (long)floor((az - r - g->oz) / h) - 1, k1 = (long)ceil((az + r - g->oz) / h) + 1;
        for (long k = k0; k <= k1; k++)
            for (long j = j0; j <= j1; j++)
                for (long i = i0; i <= i1; i++) {
                    double nxc = g->ox + (double)i * h, nyc = g->oy + (double)j * h,
                           nzc = g->oz + (double)k * h;
                    long iw = wrap(i, nx), jw = wrap(j, ny), kw = wrap(k, nz);
                    /* the x-, y- and z-edges whose lower node is (i, j, k) */
                    if (inside(g->ox + ((double)i + 0.5) * h, nyc, nzc, ax, ay, az, r2))
                        ex[exid(g, iw, jw, kw)] = g->eps_in;
                    if (inside(nxc, g->oy + ((double)j + 0.5) * h, nzc, ax, ay, az, r2))
                        ey[eyid(g, iw, jw, kw)] = g->eps_in;
                    if (inside(nxc, nyc, g->oz + ((double)k + 0.5) * h, ax, ay, az, r2))
                        ez[ezid(g, iw, jw, kw)] = g->eps_in;
                    if (g->kappa_mask && inside(nxc, nyc, nzc, ax, ay, az, r2))
                        lam[nid(g, iw, jw, kw)] = 0;
                }
    }
    for (long k = 0; k < nz; k++)
        for (long j = 0; j < ny; j++) ex[exid(g, -1, j, k)] = ex[exid(g, nx - 1, j, k)];
    for (long k = 0; k < nz; k++)
        for (long i = 0; i < nx; i++) ey[eyid(g, i, -1, k)] = ey[eyid(g, i, ny - 1, k)];
    for (long j = 0; j < ny; j++)
        for (long i = 0; i < nx; i++) ez[ezid(g, i, j, -1)] = ez[ezid(g, i, j, nz - 1)];
}

/* Weighted harmonic average boundary dielectric (Sec. 2.7): each edge takes
 * 1 / (w/eps_in + (1-w)/eps_out), w the fraction of the edge (the segment
 * between its two nodes) strictly inside the union of the atom spheres;
 * w = 0 gives eps_out and w = 1 gives eps_in exactly.  Per edge, every atom
 * contributes the open interval of the segment parameter t in [0, 1] where
 * the segment is inside its sphere; the intervals are sorted by start (then
 * end) and merged, touching ones joined, and their lengths summed in order.
 * lambda as in or_dielectric.  Free-space boundary only. */
typedef struct { double lo, hi; } or_iv;
static int iv_cmp(const void *a, const void *b) {
    const or_iv *x = a, *y = b;
    if (x->lo != y->lo) return x->lo < y->lo ? -1 : 1;
    if (x->hi != y->hi) return x->hi < y->hi ? -1 : 1;
    return 0;
}
/* Fraction inside of the segment from (px, py, pz) along axis `ax` (0, 1, 2)
 * over one spacing h. */
static double edge_fraction(const or_grid *g, int n_atoms, const double *xyz, const double *rad,
                            double px, double py, double pz, int ax, or_iv *buf) {
    const double p[3] = {px, py, pz};
    int n = 0;
    for (int a = 0; a < n_atoms; a++) {
        const double *c = xyz + 3 * a;
        const int u = (ax + 1) % 3, v = (ax + 2) % 3;  /* the two other axes */
        double du = p[u] - c[u], dv = p[v] - c[v];
        double d2 = du * du + dv * dv;
        double s = rad[a] * rad[a] - d2;
        if (!(s > 0.0)) continue;
        double q = sqrt(s);
        double t0 = ((c[ax] - q) - p[ax]) / g->h, t1 = ((c[ax] + q) - p[ax]) / g->h;
        double lo = t0 > 0.0 ? t0 : 0.0, hi = t1 < 1.0 ? t1 : 1.0;
        if (lo < hi) { buf[n].lo = lo; buf[n].hi = hi; n++; }
    }
    if (n == 0) return 0.0;
    qsort(buf, (size_t)n, sizeof(or_iv), iv_cmp);
    double w = 0.0, lo = buf[0].lo, hi = buf[0].hi;
    for (int t = 1; t < n; t++) {
        if (buf[t].lo <= hi) { if (buf[t].hi > hi) hi = buf[t].hi; }
        else { w = w + (hi - lo); lo = buf[t].lo; hi = buf[t].hi; }
    }
    return w + (hi - lo);
}
static double harmonic_eps(const or_grid *g, double w) {
    if (w == 0.0) return g->eps_out;
    if (w == 1.0) return g->eps_in;
    return 1.0 / (w / g->eps_in + (1.0 - w) / g->eps_out);
}
void or_dielectric_harmonic(const or_grid *g, int n_atoms, const double *xyz, const double *rad,
                            double *ex, double *ey, double *ez, uint8_t *lam) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const double h = g->h;
    or_dielectric(g, n_atoms, xyz, rad, ex, ey, ez, lam); /* lambda (and a binary map, replaced) */
    or_iv *buf = malloc(sizeof(or_iv) * (size_t)(n_atoms > 0 ? n_atoms : 1));
    for (long k = 0; k < nz; k++)
        for (long j = 0; j < ny; j++)
            for (long i = -1; i < nx; i++)
                ex[exid(g, i, j, k)] = harmonic_eps(g, edge_fraction(g, n_atoms, xyz, rad,
                    g->ox + (double)i * h, g->oy + (double)j * h, g->oz + (double)k * h, 0, buf));
    for (long k = 0; k < nz; k++)
        for (long j = -1; j < ny; j++)
            for (long i = 0; i < nx; i++)
                ey[eyid(g, i, j, k)] = harmonic_eps(g, edge_fraction(g, n_atoms, xyz, rad,
                    g->ox + (double)i * h, g->oy + (double)j * h, g->oz + (double)k * h, 1, buf));
    for (long k = -1; k < nz; k++)
        for (long j = 0; j < ny; j++)
            for (long i = 0; i < nx; i++)
                ez[ezid(g, i, j, k)] = harmonic_eps(g, edge_fraction(g, n_atoms, xyz, rad,
                    g->ox + (double)i * h, g->oy + (double)j * h, g->oz + (double)k * h, 2, buf));
    free(buf);
}

/* Grid charges q(i,j,k) (Eq. 3: the charge within the cube centred on the
 * node) by trilinear spreading of each atom onto the 8 nodes of its cell:
 * f = (x - o)/h, i0 = floor(f), w = f - i0; corner weights w or 1 - w per axis,
 * product taken as ((q * wx) * wy) * wz, corners in (dk, dj, di) order, atoms
 * in input order.  An atom whose cell leaves the grid (i0 < 0 or i0+1 > n-1 on
 * any axis) is an argument error. */
int or_spread_charge(const or_grid *g, int n_atoms, const double *xyz, const double *q,
                     double *q_node) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    memset(q_node, 0, sizeof(double) * (size_t)nx * ny * nz);
    for (int a = 0; a < n_atoms; a++) {
        double fx = (xyz[3 * a] - g->ox) / g->h;
        double fy = (xyz[3 * a + 1] - g->oy) / g->h;
        double fz = (xyz[3 * a + 2] - g->oz) / g->h;
        double flx = floor(fx), fly = floor(fy), flz = floor(fz);
        if (!g->periodic && (!(flx >= 0.0 && flx + 1.0 <= nx - 1) ||
                             !(fly >= 0.0 && fly + 1.0 <= ny - 1) ||
                             !(flz >= 0.0 && flz + 1.0 <= nz - 1)))
            return OR_ERR_ARG;
        long i0 = (long)flx, j0 = (long)fly, k0 = (long)flz;
        double w[3][2];
        w[0][1] = fx - flx; w[0][0] = 1.0 - w[0][1];
        w[1][1] = fy - fly; w[1][0] = 1.0 - w[1][1];
        w[2][1] = fz - flz; w[2][0] = 1.0 - w[2][1];
        for (int dk = 0; dk < 2; dk++)
            for (int dj = 0; dj < 2; dj++)
                for (int di = 0; di < 2; di++) {
                    double c = q[a] * w[0][di];
                    c = c * w[1][dj];
                    c = c * w[2][dk];
                    /* periodic: the corners wrap around */
                    q_node[nid(g, wrap(i0 + di, nx), wrap(j0 + dj, ny), wrap(k0 + dk, nz))] += c;
                }
    }
    return OR_OK;
}

/* Debye-Hueckel potential at one point: sum_a q_a exp(-kappa r)/(eps_out r),
 * atoms in input order (no ion-size factor; plain Coulomb in eps_out when
 * kappa = 0). */
static double dh_point(const or_grid *g, int n_atoms, const double *xyz, const double *q,
                       double px, double py, double pz) {
    double s = 0.0;
    for (int a = 0; a < n_atoms; a++) {
        double dx = px - xyz[3 * a], dy = py - xyz[3 * a + 1], dz = pz - xyz[3 * a + 2];
        double d2 = dx * dx + dy * dy;
        d2 = d2 + dz * dz;
        double r = sqrt(d2);
        double t = q[a] * exp(-g->kappa_d * r);
        s += t / (g->eps_out * r);
    }
    return s;
}

/* The same sum at n arbitrary points (p: n x 3). */
void or_dh_points(const or_grid *g, int n_atoms, const double *xyz, const double *q, int n,
                  const double *p, double *out) {
    for (int t = 0; t < n; t++)
        out[t] = dh_point(g, n_atoms, xyz, q, p[3 * t], p[3 * t + 1], p[3 * t + 2]);
}

/* Potential on the ghost faces, in face order x-, x+, y-, y+, z-, z+; each
 * face stored (nz, ny) for x faces, (nz, nx) for y faces, (ny, nx) for z faces
 * (first index slowest). */
void or_dh_ghost(const or_grid *g, int n_atoms, const double *xyz, const double *q,
                 double *ghost) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const double h = g->h;
    size_t off = 0;
    for (int side = 0; side < 2; side++) {
        long gi = side ? nx : -1;
        for (long k = 0; k < nz; k++)
            for (long j = 0; j < ny; j++)
                ghost[off++] = dh_point(g, n_atoms, xyz, q, g->ox + (double)gi * h,
                                        g->oy + (double)j * h, g->oz + (double)k * h);
    }
    for (int side = 0; side < 2; side++) {
        long gj = side ? ny : -1;
        for (long k = 0; k < nz; k++)
            for (long i = 0; i < nx; i++)
                ghost[off++] = dh_point(g, n_atoms, xyz, q, g->ox + (double)i * h,
                                        g->oy + (double)gj * h, g->oz + (double)k * h);
    }
    for (int side = 0; side < 2; side++) {
        long gk = side ? nz : -1;
        for (long j = 0; j < ny; j++)
            for (long i = 0; i < nx; i++)
                ghost[off++] = dh_point(g, n_atoms, xyz, q, g->ox + (double)i * h,
                                        g->oy + (double)j * h, g->oz + (double)gk * h);
    }
}

/* Right-hand side of the h^2-scaled Eq. (3): b = (4 pi / h) q_node, then each
 * boundary row gains eps_edge * phi_ghost for every ghost neighbour, faces
 * folded in the order x-, x+, y-, y+, z-, z+ (the ghost unknown moved to the
 * right-hand side). */
void or_rhs(const or_grid *g, const double *q_node, const double *ghost, const double *ex,
            const double *ey, const double *ez, double *b) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const double c = 4.0 * M_PI / g->h;
    size_t nn = (size_t)nx * ny * nz, off = 0;
    for (size_t t = 0; t < nn; t++) b[t] = q_node[t] * c;
    if (g->periodic) return; /* no boundary to fold */
    for (int side = 0; side < 2; side++) {
        long i = side ? nx - 1 : 0, ie = side ? nx - 1 : -1;
        for (long k = 0; k < nz; k++)
            for (long j = 0; j < ny; j++) {
                double e = ex[exid(g, ie, j, k)];
                b[nid(g, i, j, k)] += e * ghost[off++];
            }
    }
    for (int side = 0; side < 2; side++) {
        long j = side ? ny - 1 : 0, je = side ? ny - 1 : -1;
        for (long k = 0; k < nz; k++)
            for (long i = 0; i < nx; i++) {
                double e = ey[eyid(g, i, je, k)];
                b[nid(g, i, j, k)] += e * ghost[off++];
            }
    }
    for (int side = 0; side < 2; side++) {
        long k = side ? nz - 1 : 0, ke = side ? nz - 1 : -1;
        for (long j = 0; j < ny; j++)
            for (long i = 0; i < nx; i++) {
                double e = ez[ezid(g, i, j, ke)];
                b[nid(g, i, j, k)] += e * ghost[off++];
            }
    }
}

/* Diagonal of A (h^2-scaled Eq. 3): the six edge eps summed in the order
 * x-, x+, y-, y+, z-, z+, then + kbar2_h2 * lambda. */
void or_diag(const or_grid *g, const double *ex, const double *ey, const double *ez,
             const uint8_t *lam, double *diag) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    for (long k = 0; k < nz; k++)
        for (long j = 0; j < ny; j++)
            for (long i = 0; i < nx; i++) {
                double d = ex[exid(g, i - 1, j, k)];
                d = d + ex[exid(g, i, j, k)];
                d = d + ey[eyid(g, i, j - 1, k)];
                d = d + ey[eyid(g, i, j, k)];
                d = d + ez[ezid(g, i, j, k - 1)];
                d = d + ez[ezid(g, i, j, k)];
                d = d + g->kbar2_h2 * (double)lam[nid(g, i, j, k)];
                diag[nid(g, i, j, k)] = d;
            }
}

/* ------------------------------------------------------------------------- */
/* O2. The operator of Eq. (3)-(4), h^2-scaled:                              */
/*   (A u)_c = diag_c u_c - sum over the six neighbours of eps_edge * u_nb,   */
/* with u = 0 on the ghost layer (its values already sit in b).              */
/* ------------------------------------------------------------------------- */
void or_apply(const or_grid *g, const double *ex, const double *ey, const double *ez,
              const double *diag, const double *u, double *au) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    for (long k = 0; k < nz; k++)
        for (long j = 0; j < ny; j++)
            for (long i = 0; i < nx; i++) {
                size_t c = nid(g, i, j, k);
                double s = 0.0;
                if (g->periodic) { /* every neighbour exists, modulo n */
                    s += ex[exid(g, i - 1, j, k)] * u[nid(g, wrap(i - 1, nx), j, k)];
                    s += ex[exid(g, i, j, k)] * u[nid(g, wrap(i + 1, nx), j, k)];
                    s += ey[eyid(g, i, j - 1, k)] * u[nid(g, i, wrap(j - 1, ny), k)];
                    s += ey[eyid(g, i, j, k)] * u[nid(g, i, wrap(j + 1, ny), k)];
                    s += ez[ezid(g, i, j, k - 1)] * u[nid(g, i, j, wrap(k - 1, nz))];
                    s += ez[ezid(g, i, j, k)] * u[nid(g, i, j, wrap(k + 1, nz))];
                } else {
                    if (i > 0) s += ex[exid(g, i - 1, j, k)] * u[nid(g, i - 1, j, k)];
                    if (i < nx - 1) s += ex[exid(g, i, j, k)] * u[nid(g, i + 1, j, k)];
                    if (j > 0) s += ey[eyid(g, i, j - 1, k)] * u[nid(g, i, j - 1, k)];
                    if (j < ny - 1) s += ey[eyid(g, i, j, k)] * u[nid(g, i, j + 1, k)];
                    if (k > 0) s += ez[ezid(g, i, j, k - 1)] * u[nid(g, i, j, k - 1)];
                    if (k < nz - 1) s += ez[ezid(g, i, j, k)] * u[nid(g, i, j, k + 1)];
                }
                au[c] = diag[c] * u[c] - s;
            }
}

static double dot(size_t n, const double *a, const double *b) {
    double s = 0.0;
    for (size_t t = 0; t < n; t++) s += a[t] * b[t];
    return s;
}

/* ------------------------------------------------------------------------- */
/* O3/O4. Conjugate gradient, Sec. 2.2.                                      */
/* precond = 1: the preconditioned listing with M = diag(A) (Jacobi, Sec.    */
/*   2.4): r0 = b - A phi0, z = M^-1 r, p0 = z; alpha = (r.z)/(p.Ap);         */
/*   phi += alpha p; r -= alpha Ap; z = M^-1 r; beta = (r.z)_new/(r.z)_old;  */
/*   p = z + beta p.                                                         */
/* precond = 0: the same recurrence with M = I (plain CG).  The plain listing */
/*   prints beta = +r^T A p / p^T A p with a recomputed residual; A-conjugate */
/*   directions need the Hestenes-Stiefel form used here, which is the       */
/*   preconditioned listing with M = I.                                      */
/* Stopping rule: ||r_l|| / ||b|| < tol on the recursive residual, tested    */
/* before every update, at l = 0 too.  The iteration count is the number of  */
/* alpha updates.  b = 0 returns phi = 0 with zero iterations.               */
/* ------------------------------------------------------------------------- */
int or_pcg(const or_grid *g, const double *ex, const double *ey, const double *ez,
           const double *diag, const double *b, double *phi, int precond, double tol,
           int max_iter, int *iters_out, double *relres_out) {
    size_t n = (size_t)g->nx * g->ny * g->nz;
    double *r = malloc(n * sizeof(double)), *z = malloc(n * sizeof(double));
    double *p = malloc(n * sizeof(double)), *ap = malloc(n * sizeof(double));
    int status = OR_OK, l = 0;
    double bnorm = sqrt(dot(n, b, b)), relres = 0.0;
    if (bnorm == 0.0) {
        for (size_t t = 0; t < n; t++) phi[t] = 0.0;
        goto done;
    }
    or_apply(g, ex, ey, ez, diag, phi, ap);
    for (size_t t = 0; t < n; t++) r[t] = b[t] - ap[t];
    for (size_t t = 0; t < n; t++) z[t] = precond ? r[t] / diag[t] : r[t];
    for (size_t t = 0; t < n; t++) p[t] = z[t];
    double rz = dot(n, r, z);
    for (;;) {
        relres = sqrt(dot(n, r, r)) / bnorm;
        if (relres < tol) break;
        if (l >= max_iter) { status = OR_NOT_CONVERGED; break; }
        or_apply(g, ex, ey, ez, diag, p, ap);
        double pap = dot(n, p, ap);
        if (!(pap > 0.0) || !isfinite(pap)) { status = OR_BREAKDOWN; break; }
        double alpha = rz / pap;
        for (size_t t = 0; t < n; t++) phi[t] += alpha * p[t];
        for (size_t t = 0; t < n; t++) r[t] -= alpha * ap[t];
        l++;
        for (size_t t = 0; t < n; t++) z[t] = precond ? r[t] / diag[t] : r[t];
        double rz_new = dot(n, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
        for (size_t t = 0; t < n; t++) p[t] = z[t] + beta * p[t];
    }
done:
    free(r); free(z); free(p); free(ap);
    *iters_out = l;
    *relres_out = relres;
    return status;
}

/* Electrostatic energy (kcal/mol) 1/2 * 332.0637 * sum_nodes q_node phi_node,
 * summed in node order; 332.0637 = e^2/(4 pi eps0 A) in kcal/mol (CODATA). */
double or_energy(const or_grid *g, const double *q_node, const double *phi) {
    size_t n = (size_t)g->nx * g->ny * g->nz;
    double s = 0.0;
    for (size_t t = 0; t < n; t++) s += q_node[t] * phi[t];
    return 0.5 * 332.0637 * s;
}

/* ------------------------------------------------------------------------- */
/* O6. Dense check for small grids: the explicit matrix A and an in-place    */
/* Cholesky solve A x = b (A overwritten by its factor L, lower triangle).   */
/* ------------------------------------------------------------------------- */
void or_dense_matrix(const or_grid *g, const double *ex, const double *ey, const double *ez,
                     const double *diag, double *A) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    size_t n = (size_t)nx * ny * nz;
    memset(A, 0, sizeof(double) * n * n);
    for (long k = 0; k < nz; k++)
        for (long j = 0; j < ny; j++)
            for (long i = 0; i < nx; i++) {
                size_t c = nid(g, i, j, k);
                A[c * n + c] = diag[c];
                if (g->periodic) { /* accumulate: on n = 2 two edges join the same pair */
                    A[c * n + nid(g, wrap(i - 1, nx), j, k)] -= ex[exid(g, i - 1, j, k)];
                    A[c * n + nid(g, wrap(i + 1, nx), j, k)] -= ex[exid(g, i, j, k)];
                    A[c * n + nid(g, i, wrap(j - 1, ny), k)] -= ey[eyid(g, i, j - 1, k)];
                    A[c * n + nid(g, i, wrap(j + 1, ny), k)] -= ey[eyid(g, i, j, k)];
                    A[c * n + nid(g, i, j, wrap(k - 1, nz))] -= ez[ezid(g, i, j, k - 1)];
                    A[c * n + nid(g, i, j, wrap(k + 1, nz))] -= ez[ezid(g, i, j, k)];
                    continue;
                }
                if (i > 0) A[c * n + nid(g, i - 1, j, k)] = -ex[exid(g, i - 1, j, k)];
                if (i < nx - 1) A[c * n + nid(g, i + 1, j, k)] = -ex[exid(g, i, j, k)];
                if (j > 0) A[c * n + nid(g, i, j - 1, k)] = -ey[eyid(g, i, j - 1, k)];
                if (j < ny - 1) A[c * n + nid(g, i, j + 1, k)] = -ey[eyid(g, i, j, k)];
                if (k > 0) A[c * n + nid(g, i, j, k - 1)] = -ez[ezid(g, i, j, k - 1)];
                if (k < nz - 1) A[c * n + nid(g, i, j, k + 1)] = -ez[ezid(g, i, j, k)];
            }
}

int or_cholesky_solve(int n, double *A, const double *b, double *x) {
    for (int j = 0; j < n; j++) {
        double d = A[(size_t)j * n + j];
        for (int t = 0; t < j; t++) d -= A[(size_t)j * n + t] * A[(size_t)j * n + t];
        if (!(d > 0.0)) return OR_BREAKDOWN;
        double ljj = sqrt(d);
        A[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; i++) {
            double s = A[(size_t)i * n + j];
            for (int t = 0; t < j; t++) s -= A[(size_t)i * n + t] * A[(size_t)j * n + t];
            A[(size_t)i * n + j] = s / ljj;
        }
    }
    for (int i = 0; i < n; i++) { /* L y = b */
        double s = b[i];
        for (int t = 0; t < i; t++) s -= A[(size_t)i * n + t] * x[t];
        x[i] = s / A[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) { /* L^T x = y */
        double s = x[i];
        for (int t = i + 1; t < n; t++) s -= A[(size_t)t * n + i] * x[t];
        x[i] = s / A[(size_t)i * n + i];
    }
    return OR_OK;
}
