/*
 * pic_oracle.c -- plain FP64 CPU oracle of the electromagnetic PIC step used for the
 * relativistic-beam Weibel problem of Karmakar, Kumar, Shvets, Polomarov & Pukhov,
 * "On collisions driven negative energy waves and Weibel instability of a relativistic
 * electron beam in a quasi-neutral plasma" (arXiv:0808.4078).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls this file;
 * only the tests, the package's smoke check and the benchmark's CPU-baseline leg do.  It
 * shares no code, header or constant with the CUDA library.
 *
 * What the paper fixes and what is a reading:
 *   - Geometry, species and neutralisation (simulation section: 2D plane transverse to the
 *     beam, no z dependence; immobile ions of density n0 = nb + np; beam current initially
 *     neutralised by the return current).  3D runs are the paper's 3D simulations.
 *   - Collisional drag on the return current: Eq. (3), d v_pz/dt + nu v_pz = ..., read as a
 *     per-cell relaxation of the background electrons' mean momentum at rate nu (Krook).
 *   - Field-energy diagnostic: integral of (e F_i / m c w_p)^2 dx dy per component
 *     (simulation section; the printed fraction is garbled and read as a ratio).
 *   - The paper names no PIC algorithm (its code, VLPL, is not described).  The discrete
 *     method is the textbook one: CIC shapes, Yee staggering, relativistic Boris push
 *     (Boris 1970), charge-conserving Esirkepov deposit (Esirkepov 2001), Yee FDTD (Yee 1966).
 *
 * Normalised units: time 1/w_p, length c/w_p, momentum u = gamma v / c, fields m c w_p / e,
 * density n0, current e n0 c.  Maxwell: dB/dt = -curl E, dE/dt = curl B - J.  Electrons have
 * q = -1, m = 1.  A macro-particle of weight w contributes density w (units n0) spread over
 * nodes by its shape; positions are kept in cell units X = x/dx in [0, nx).
 *
 * Order of one step n -> n+1 (the reading used throughout):
 *   diagnostics of (E^n, B^n, u^n)  ->  gather E^n, B^n at X^n  ->  Boris u^{n-1/2} -> u^{n+1/2}
 *   -> Krook drag with the cell mean <u> accumulated at (X^n, u^{n-1/2})  ->  X^{n+1}
 *   -> Esirkepov J^{n+1/2}  ->  B half step, E full step, B half step.
 *
 * Yee staggering (2D, arrays indexed [j][i]):  Ex(i+1/2,j) Ey(i,j+1/2) Ez(i,j)
 *   Bx(i,j+1/2) By(i+1/2,j) Bz(i+1/2,j+1/2);  J like E; rho at nodes (i,j).
 * 3D (arrays [k][j][i]): Ex(i+1/2,j,k) Ey(i,j+1/2,k) Ez(i,j,k+1/2)
 *   Bx(i,j+1/2,k+1/2) By(i+1/2,j,k+1/2) Bz(i+1/2,j+1/2,k).
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct orc_grid {
    int ndim;             /* 2 or 3 */
    int nx, ny, nz;       /* nz = 1 when ndim == 2 */
    double dx, dy, dz, dt;
    double *Ex, *Ey, *Ez; /* nx*ny*nz each */
    double *Bx, *By, *Bz;
    double *Jx, *Jy, *Jz; /* current density of the last step, J^{n+1/2} */
    int64_t step;         /* steps completed: keys the binary-collision draws of the next step */
    int j_filter;         /* 1: one binomial pass per axis on J before the field update */
} orc_grid;

typedef struct orc_species {
    double q, m, w;   /* charge (e), mass (m_e), density weight per macro-particle (n0) */
    double nu;        /* Krook rate on this species' cell-mean momentum; 0 = no drag */
    int64_t n;
    double *X, *Y, *Z;    /* positions in cell units; Z unused in 2D */
    double *ux, *uy, *uz;
    double *ubar;     /* 3*ncell cell-mean momentum (NGP) used by the drag; NULL if no drag */
    double *nu_cell;  /* ncell Krook rates replacing nu, looked up at the particle's cell at time
                         n (the closure-driven drag); negative rates act as 0; NULL = nu */
    double nu_coll;   /* binary electron-ion collision rate (momentum transfer); 0 = none */
    uint64_t seed;    /* key of the collision draws */
    int32_t index;    /* species index in the draws' counter */
} orc_species;

#define ORC_MAX_SPECIES 4
typedef struct orc_diag {
    double WE[3], WB[3];            /* sum F_i^2 dV over the grid at time n */
    double Ekin[ORC_MAX_SPECIES];   /* sum w (gamma(u^n) - 1) dV per species */
    double P[3];                    /* sum w u^n dV over all species */
} orc_diag;

static int64_t ncell_of(const orc_grid *g) { return (int64_t)g->nx * g->ny * g->nz; }

static int wrap(int i, int n) { i %= n; return i < 0 ? i + n : i; }

static int64_t idx2(const orc_grid *g, int i, int j) {
    return (int64_t)wrap(j, g->ny) * g->nx + wrap(i, g->nx);
}
static int64_t idx3(const orc_grid *g, int i, int j, int k) {
    return ((int64_t)wrap(k, g->nz) * g->ny + wrap(j, g->ny)) * g->nx + wrap(i, g->nx);
}

/* First-order (cloud-in-cell) shape: weight of a node at distance r (cells). */
static double cic(double r) { r = fabs(r); return r < 1.0 ? 1.0 - r : 0.0; }

static double wrap_pos(double X, int n) {
    if (X < 0.0) X += n;
    if (X >= n) X -= n;
    return X;
}

/* ---------------------------------------------------------------- field gather (CIC) */

/* Interpolate one staggered component: the lattice of F is shifted by (sx,sy[,sz]) cells
 * from the nodes; F is linearly interpolated on its own lattice. */
static double interp2(const orc_grid *g, const double *F, double X, double Y, double sx, double sy) {
    double xs = X - sx, ys = Y - sy;
    double fx0 = floor(xs), fy0 = floor(ys);
    double ax = xs - fx0, ay = ys - fy0;
    int i = (int)fx0, j = (int)fy0;
    return (1 - ax) * (1 - ay) * F[idx2(g, i, j)] + ax * (1 - ay) * F[idx2(g, i + 1, j)]
         + (1 - ax) * ay * F[idx2(g, i, j + 1)] + ax * ay * F[idx2(g, i + 1, j + 1)];
}

static double interp3(const orc_grid *g, const double *F, double X, double Y, double Z,
                      double sx, double sy, double sz) {
    double xs = X - sx, ys = Y - sy, zs = Z - sz;
    double fx0 = floor(xs), fy0 = floor(ys), fz0 = floor(zs);
    double a[2], b[2], c[2];
    int i = (int)fx0, j = (int)fy0, k = (int)fz0;
    a[1] = xs - fx0; a[0] = 1 - a[1];
    b[1] = ys - fy0; b[0] = 1 - b[1];
    c[1] = zs - fz0; c[0] = 1 - c[1];
    double s = 0.0;
    for (int dk = 0; dk < 2; dk++)
        for (int dj = 0; dj < 2; dj++)
            for (int di = 0; di < 2; di++)
                s += a[di] * b[dj] * c[dk] * F[idx3(g, i + di, j + dj, k + dk)];
    return s;
}

/* E and B at a particle position (cell units). */
void orc_gather(const orc_grid *g, double X, double Y, double Z, double EB[6]) {
    if (g->ndim == 2) {
        EB[0] = interp2(g, g->Ex, X, Y, 0.5, 0.0);
        EB[1] = interp2(g, g->Ey, X, Y, 0.0, 0.5);
        EB[2] = interp2(g, g->Ez, X, Y, 0.0, 0.0);
        EB[3] = interp2(g, g->Bx, X, Y, 0.0, 0.5);
        EB[4] = interp2(g, g->By, X, Y, 0.5, 0.0);
        EB[5] = interp2(g, g->Bz, X, Y, 0.5, 0.5);
    } else {
        EB[0] = interp3(g, g->Ex, X, Y, Z, 0.5, 0.0, 0.0);
        EB[1] = interp3(g, g->Ey, X, Y, Z, 0.0, 0.5, 0.0);
        EB[2] = interp3(g, g->Ez, X, Y, Z, 0.0, 0.0, 0.5);
        EB[3] = interp3(g, g->Bx, X, Y, Z, 0.0, 0.5, 0.5);
        EB[4] = interp3(g, g->By, X, Y, Z, 0.5, 0.0, 0.5);
        EB[5] = interp3(g, g->Bz, X, Y, Z, 0.5, 0.5, 0.0);
    }
}

/* ---------------------------------------------------------------- relativistic Boris */

/* u^{n-1/2} -> u^{n+1/2} under E, B (textbook relativistic Boris rotation). */
void orc_boris(double qm, double dt, const double EB[6], double u[3]) {
    double h = 0.5 * qm * dt;
    double um[3] = {u[0] + h * EB[0], u[1] + h * EB[1], u[2] + h * EB[2]};
    double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    double t[3] = {h * EB[3] / gm, h * EB[4] / gm, h * EB[5] / gm};
    double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    double s[3] = {2 * t[0] / (1 + t2), 2 * t[1] / (1 + t2), 2 * t[2] / (1 + t2)};
    double up[3] = {um[0] + (um[1] * t[2] - um[2] * t[1]),
                    um[1] + (um[2] * t[0] - um[0] * t[2]),
                    um[2] + (um[0] * t[1] - um[1] * t[0])};
    double upl[3] = {um[0] + (up[1] * s[2] - up[2] * s[1]),
                     um[1] + (up[2] * s[0] - up[0] * s[2]),
                     um[2] + (up[0] * s[1] - up[1] * s[0])};
    u[0] = upl[0] + h * EB[0];
    u[1] = upl[1] + h * EB[1];
    u[2] = upl[2] + h * EB[2];
}

/* ---------------------------------------------------------------- Esirkepov deposit */

/* Charge-conserving current of one particle moving X0 -> X1 (unwrapped, cell units) during
 * dt, CIC shape (Esirkepov 2001).  The 4-node window per axis starts one node below the old
 * cell.  Adds current density (units e n0 c) to J; qw = q * w. */
static void deposit_2d(orc_grid *g, double qw, double X0, double Y0, double X1, double Y1, double vz) {
    int bx = (int)floor(X0) - 1, by = (int)floor(Y0) - 1;
    double S0x[4], S1x[4], DSx[4], S0y[4], S1y[4], DSy[4];
    for (int k = 0; k < 4; k++) {
        S0x[k] = cic(X0 - (bx + k)); S1x[k] = cic(X1 - (bx + k)); DSx[k] = S1x[k] - S0x[k];
        S0y[k] = cic(Y0 - (by + k)); S1y[k] = cic(Y1 - (by + k)); DSy[k] = S1y[k] - S0y[k];
    }
    double cx = -qw * g->dx / g->dt, cy = -qw * g->dy / g->dt;
    /* J_x on x-edges (bx+k+1/2, by+l): running sum of W_x along x. */
    for (int l = 0; l < 4; l++) {
        double acc = 0.0;
        for (int k = 0; k < 3; k++) {
            acc += DSx[k] * (S0y[l] + 0.5 * DSy[l]);
            g->Jx[idx2(g, bx + k, by + l)] += cx * acc;
        }
    }
    /* J_y on y-edges (bx+k, by+l+1/2). */
    for (int k = 0; k < 4; k++) {
        double acc = 0.0;
        for (int l = 0; l < 3; l++) {
            acc += DSy[l] * (S0x[k] + 0.5 * DSx[k]);
            g->Jy[idx2(g, bx + k, by + l)] += cy * acc;
        }
    }
    /* Out-of-plane J_z at nodes: path-averaged shape product. */
    for (int l = 0; l < 4; l++)
        for (int k = 0; k < 4; k++) {
            double wz = S0x[k] * S0y[l] / 3.0 + S0x[k] * S1y[l] / 6.0
                      + S1x[k] * S0y[l] / 6.0 + S1x[k] * S1y[l] / 3.0;
            if (wz != 0.0) g->Jz[idx2(g, bx + k, by + l)] += qw * vz * wz;
        }
}

static void deposit_3d(orc_grid *g, double qw, const double P0[3], const double P1[3]) {
    int b[3];
    double S0[3][4], S1[3][4], DS[3][4];
    for (int a = 0; a < 3; a++) {
        b[a] = (int)floor(P0[a]) - 1;
        for (int k = 0; k < 4; k++) {
            S0[a][k] = cic(P0[a] - (b[a] + k));
            S1[a][k] = cic(P1[a] - (b[a] + k));
            DS[a][k] = S1[a][k] - S0[a][k];
        }
    }
    double c[3] = {-qw * g->dx / g->dt, -qw * g->dy / g->dt, -qw * g->dz / g->dt};
    /* W_a = DS_a * (S0_b S0_c + DS_b S0_c / 2 + S0_b DS_c / 2 + DS_b DS_c / 3), (a,b,c) cyclic;
     * J_a is the running sum of W_a along axis a. */
    for (int m = 0; m < 4; m++)
        for (int l = 0; l < 4; l++) {
            double acc = 0.0;
            for (int k = 0; k < 3; k++) {
                acc += DS[0][k] * (S0[1][l] * S0[2][m] + 0.5 * DS[1][l] * S0[2][m]
                                   + 0.5 * S0[1][l] * DS[2][m] + DS[1][l] * DS[2][m] / 3.0);
                g->Jx[idx3(g, b[0] + k, b[1] + l, b[2] + m)] += c[0] * acc;
            }
        }
    for (int m = 0; m < 4; m++)
        for (int k = 0; k < 4; k++) {
            double acc = 0.0;
            for (int l = 0; l < 3; l++) {
                acc += DS[1][l] * (S0[2][m] * S0[0][k] + 0.5 * DS[2][m] * S0[0][k]
                                   + 0.5 * S0[2][m] * DS[0][k] + DS[2][m] * DS[0][k] / 3.0);
                g->Jy[idx3(g, b[0] + k, b[1] + l, b[2] + m)] += c[1] * acc;
            }
        }
    for (int l = 0; l < 4; l++)
        for (int k = 0; k < 4; k++) {
            double acc = 0.0;
            for (int m = 0; m < 3; m++) {
                acc += DS[2][m] * (S0[0][k] * S0[1][l] + 0.5 * DS[0][k] * S0[1][l]
                                   + 0.5 * S0[0][k] * DS[1][l] + DS[0][k] * DS[1][l] / 3.0);
                g->Jz[idx3(g, b[0] + k, b[1] + l, b[2] + m)] += c[2] * acc;
            }
        }
}

/* ---------------------------------------------------------------- Yee FDTD */

static void yee_half_b(orc_grid *g, double h) {
    int nx = g->nx, ny = g->ny, nz = g->nz;
    if (g->ndim == 2) {
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                int64_t c = idx2(g, i, j);
                double dEz_dy = (g->Ez[idx2(g, i, j + 1)] - g->Ez[c]) / g->dy;
                double dEz_dx = (g->Ez[idx2(g, i + 1, j)] - g->Ez[c]) / g->dx;
                double dEy_dx = (g->Ey[idx2(g, i + 1, j)] - g->Ey[c]) / g->dx;
                double dEx_dy = (g->Ex[idx2(g, i, j + 1)] - g->Ex[c]) / g->dy;
                g->Bx[c] -= h * dEz_dy;
                g->By[c] += h * dEz_dx;
                g->Bz[c] -= h * (dEy_dx - dEx_dy);
            }
    } else {
        for (int k = 0; k < nz; k++)
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++) {
                    int64_t c = idx3(g, i, j, k);
                    double Ex = g->Ex[c], Ey = g->Ey[c], Ez = g->Ez[c];
                    double dEz_dy = (g->Ez[idx3(g, i, j + 1, k)] - Ez) / g->dy;
                    double dEy_dz = (g->Ey[idx3(g, i, j, k + 1)] - Ey) / g->dz;
                    double dEx_dz = (g->Ex[idx3(g, i, j, k + 1)] - Ex) / g->dz;
                    double dEz_dx = (g->Ez[idx3(g, i + 1, j, k)] - Ez) / g->dx;
                    double dEy_dx = (g->Ey[idx3(g, i + 1, j, k)] - Ey) / g->dx;
                    double dEx_dy = (g->Ex[idx3(g, i, j + 1, k)] - Ex) / g->dy;
                    g->Bx[c] -= h * (dEz_dy - dEy_dz);
                    g->By[c] -= h * (dEx_dz - dEz_dx);
                    g->Bz[c] -= h * (dEy_dx - dEx_dy);
                }
    }
}

static void yee_full_e(orc_grid *g, double dt) {
    int nx = g->nx, ny = g->ny, nz = g->nz;
    if (g->ndim == 2) {
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                int64_t c = idx2(g, i, j);
                double dBz_dy = (g->Bz[c] - g->Bz[idx2(g, i, j - 1)]) / g->dy;
                double dBz_dx = (g->Bz[c] - g->Bz[idx2(g, i - 1, j)]) / g->dx;
                double dBy_dx = (g->By[c] - g->By[idx2(g, i - 1, j)]) / g->dx;
                double dBx_dy = (g->Bx[c] - g->Bx[idx2(g, i, j - 1)]) / g->dy;
                g->Ex[c] += dt * (dBz_dy - g->Jx[c]);
                g->Ey[c] += dt * (-dBz_dx - g->Jy[c]);
                g->Ez[c] += dt * (dBy_dx - dBx_dy - g->Jz[c]);
            }
    } else {
        for (int k = 0; k < nz; k++)
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++) {
                    int64_t c = idx3(g, i, j, k);
                    double Bx = g->Bx[c], By = g->By[c], Bz = g->Bz[c];
                    double dBz_dy = (Bz - g->Bz[idx3(g, i, j - 1, k)]) / g->dy;
                    double dBy_dz = (By - g->By[idx3(g, i, j, k - 1)]) / g->dz;
                    double dBx_dz = (Bx - g->Bx[idx3(g, i, j, k - 1)]) / g->dz;
                    double dBz_dx = (Bz - g->Bz[idx3(g, i - 1, j, k)]) / g->dx;
                    double dBy_dx = (By - g->By[idx3(g, i - 1, j, k)]) / g->dx;
                    double dBx_dy = (Bx - g->Bx[idx3(g, i, j - 1, k)]) / g->dy;
                    g->Ex[c] += dt * (dBz_dy - dBy_dz - g->Jx[c]);
                    g->Ey[c] += dt * (dBx_dz - dBz_dx - g->Jy[c]);
                    g->Ez[c] += dt * (dBy_dx - dBx_dy - g->Jz[c]);
                }
    }
}

/* ---------------------------------------------------------------- current filter */

/* One 1-2-1 binomial pass along each axis of a periodic grid array (x, y, then z in 3D):
 * F_i <- (F_{i-1} + 2 F_i + F_{i+1}) / 4.  The smoothing that damps grid-scale current
 * (numerical Cherenkov control); the paper is silent on filtering. */
void orc_binomial(const orc_grid *g, double *F) {
    int nx = g->nx, ny = g->ny, nz = g->ndim == 3 ? g->nz : 1;
    int64_t nc = (int64_t)nx * ny * nz;
    double *t = malloc(sizeof(double) * (size_t)nc);
    if (!t) return;
    for (int axis = 0; axis < g->ndim; axis++) {
        memcpy(t, F, sizeof(double) * (size_t)nc);
        for (int k = 0; k < nz; k++)
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++) {
                    int64_t c = ((int64_t)k * ny + j) * nx + i, m, p;
                    if (axis == 0) {
                        m = ((int64_t)k * ny + j) * nx + (i + nx - 1) % nx;
                        p = ((int64_t)k * ny + j) * nx + (i + 1) % nx;
                    } else if (axis == 1) {
                        m = ((int64_t)k * ny + (j + ny - 1) % ny) * nx + i;
                        p = ((int64_t)k * ny + (j + 1) % ny) * nx + i;
                    } else {
                        m = ((int64_t)((k + nz - 1) % nz) * ny + j) * nx + i;
                        p = ((int64_t)((k + 1) % nz) * ny + j) * nx + i;
                    }
                    F[c] = 0.25 * (t[m] + 2.0 * t[c] + t[p]);
                }
    }
    free(t);
}

/* Yee step with the grid's current: B^n -> B^{n+1/2}, E^n -> E^{n+1}, B^{n+1/2} -> B^{n+1}. */
void orc_yee(orc_grid *g) {
    yee_half_b(g, 0.5 * g->dt);
    yee_full_e(g, g->dt);
    yee_half_b(g, 0.5 * g->dt);
}

/* ---------------------------------------------------------------- moments for the drag */

static int64_t ngp_cell(const orc_grid *g, const orc_species *s, int64_t p) {
    int i = (int)floor(s->X[p]), j = (int)floor(s->Y[p]);
    if (g->ndim == 2) return idx2(g, i, j);
    return idx3(g, i, j, (int)floor(s->Z[p]));
}

/* Cell-mean momentum of species s with nearest-grid-point (cell) assignment. */
int orc_moments(const orc_grid *g, orc_species *s) {
    if (!s->ubar) return 0;
    int64_t nc = ncell_of(g);
    double *cnt = calloc((size_t)nc, sizeof(double));
    if (!cnt) return -1;
    memset(s->ubar, 0, sizeof(double) * 3 * (size_t)nc);
    for (int64_t p = 0; p < s->n; p++) {
        int64_t c = ngp_cell(g, s, p);
        s->ubar[3 * c + 0] += s->ux[p];
        s->ubar[3 * c + 1] += s->uy[p];
        s->ubar[3 * c + 2] += s->uz[p];
        cnt[c] += 1.0;
    }
    for (int64_t c = 0; c < nc; c++)
        if (cnt[c] > 0)
            for (int a = 0; a < 3; a++) s->ubar[3 * c + a] /= cnt[c];
    free(cnt);
    return 0;
}

/* ---------------------------------------------------------------- diagnostics */

static void field_energy(const orc_grid *g, orc_diag *d) {
    int64_t nc = ncell_of(g);
    double dV = g->dx * g->dy * (g->ndim == 3 ? g->dz : 1.0);
    const double *F[6] = {g->Ex, g->Ey, g->Ez, g->Bx, g->By, g->Bz};
    for (int a = 0; a < 6; a++) {
        double s = 0.0;
        for (int64_t c = 0; c < nc; c++) s += F[a][c] * F[a][c];
        if (a < 3) d->WE[a] = s * dV; else d->WB[a - 3] = s * dV;
    }
}

/* ---------------------------------------------------------------- binary collisions */

/* Philox4x32-10, the counter-based generator of Salmon, Moraes, Dror & Shaw ("Parallel random
 * numbers: as easy as 1, 2, 3", SC'11): ten rounds of
 *   (hi0, lo0) = M0 * c0,  (hi1, lo1) = M1 * c2,  c = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
 * with M0 = 0xD2511F53, M1 = 0xCD9E8D57 and the key raised by the Weyl constants
 * (0x9E3779B9, 0xBB67AE85) between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0; c1 = lo1; c2 = hi0 ^ c3 ^ k1; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The draws of particle `id` of species `sp` at step `step`: counter (id, step lo, step hi, sp),
 * key = the seed's two halves. */
static void collision_draws(uint64_t seed, int64_t id, int64_t step, int32_t sp, uint32_t r[4]) {
    const uint32_t ctr[4] = {(uint32_t)id, (uint32_t)((uint64_t)step & 0xffffffffu),
                             (uint32_t)((uint64_t)step >> 32), (uint32_t)sp};
    const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, r);
}

static double unit_open(uint32_t x) { return ((double)x + 0.5) / 4294967296.0; }

/* Binary collision of an electron with an immobile ion over one step (Takizuka & Abe, J. Comput.
 * Phys. 25, 205 (1977), with an infinitely heavy partner so that the relative velocity is the
 * electron's own): u is turned by the scattering angle theta, tan(theta / 2) = delta ~
 * N(0, sigma^2), about a random azimuth phi ~ U[0, 2 pi); |u| is unchanged.  The mean momentum
 * then relaxes at <1 - cos theta> / dt = 2 sigma^2 / dt per step for small sigma, so
 * sigma^2 = nu dt / 2 gives the momentum-transfer rate nu (the reading of the collision rate).
 * r: four 32-bit draws (r0, r1 -> delta by Box-Muller, r2 -> phi). */
void orc_collide_ion(double u[3], double sigma, const uint32_t r[4]) {
    const double pi = 3.14159265358979323846;
    double delta = sigma * sqrt(-2.0 * log(unit_open(r[0]))) * cos(2.0 * pi * unit_open(r[1]));
    double phi = 2.0 * pi * unit_open(r[2]);
    double sn = 2.0 * delta / (1.0 + delta * delta), omc = 2.0 * delta * delta / (1.0 + delta * delta);
    double cp = cos(phi), sp = sin(phi);
    double uperp = sqrt(u[0] * u[0] + u[1] * u[1]);
    double umag = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double d[3];
    if (uperp > 0.0) {
        d[0] = (u[0] * u[2] / uperp) * sn * cp - (u[1] * umag / uperp) * sn * sp - u[0] * omc;
        d[1] = (u[1] * u[2] / uperp) * sn * cp + (u[0] * umag / uperp) * sn * sp - u[1] * omc;
        d[2] = -uperp * sn * cp - u[2] * omc;
    } else {
        d[0] = umag * sn * cp;
        d[1] = umag * sn * sp;
        d[2] = -u[2] * omc;
    }
    for (int a = 0; a < 3; a++) u[a] += d[a];
}

/* ---------------------------------------------------------------- one particle */

/* Advance one particle by one step: gather, Boris, drag, move.  Returns the unwrapped new
 * position in P1 and writes u.  ubar_c is the mean momentum of the particle's cell (NULL
 * for no drag), dragf = 1 - exp(-nu dt). */
static void push_one(const orc_grid *g, double qm, const double P0[3], double u[3],
                     const double *ubar_c, double dragf, const orc_species *coll, int64_t id,
                     double P1[3]) {
    double EB[6];
    orc_gather(g, P0[0], P0[1], P0[2], EB);
    orc_boris(qm, g->dt, EB, u);
    if (ubar_c && dragf != 0.0)
        for (int a = 0; a < 3; a++) u[a] -= dragf * ubar_c[a];
    if (coll && coll->nu_coll > 0.0) {
        uint32_t r[4];
        collision_draws(coll->seed, id, g->step, coll->index, r);
        orc_collide_ion(u, sqrt(0.5 * coll->nu_coll * g->dt), r);
    }
    double gam = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    P1[0] = P0[0] + g->dt * u[0] / gam / g->dx;
    P1[1] = P0[1] + g->dt * u[1] / gam / g->dy;
    P1[2] = g->ndim == 3 ? P0[2] + g->dt * u[2] / gam / g->dz : P0[2];
}

/* Single-particle step for sampled checks: X,u in/out; ubar_c as above. */
void orc_push_particle(const orc_grid *g, double qm, double nu, double *X, double *Y, double *Z,
                       double u[3], const double ubar_c[3]) {
    double P0[3] = {*X, *Y, Z ? *Z : 0.0}, P1[3];
    push_one(g, qm, P0, u, ubar_c, ubar_c ? 1.0 - exp(-nu * g->dt) : 0.0, NULL, 0, P1);
    *X = wrap_pos(P1[0], g->nx);
    *Y = wrap_pos(P1[1], g->ny);
    if (Z && g->ndim == 3) *Z = wrap_pos(P1[2], g->nz);
}

/* ---------------------------------------------------------------- full step */

/* Particle p of species s (index si): push, deposit into g's current, diagnostics into d (may
 * be NULL), cell-mean momentum sums into nsum/ncnt (NULL without drag). */
static void step_particle(const orc_grid *g, orc_species *s, int si, int64_t p, double qm, double qw,
                          double dragf, double dV, orc_diag *d, double *nsum, double *ncnt) {
    double P0[3] = {s->X[p], s->Y[p], g->ndim == 3 ? s->Z[p] : 0.0}, P1[3];
    double u0[3] = {s->ux[p], s->uy[p], s->uz[p]};
    double u[3] = {u0[0], u0[1], u0[2]};
    const double *ub = s->ubar ? &s->ubar[3 * ngp_cell(g, s, p)] : NULL;
    double df = dragf;
    if (s->ubar && s->nu_cell) {
        double r = s->nu_cell[ngp_cell(g, s, p)];
        df = r > 0.0 ? 1.0 - exp(-r * g->dt) : 0.0;
    }
    push_one(g, qm, P0, u, ub, df, s, p, P1);
    double gam = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    if (g->ndim == 2) deposit_2d((orc_grid *)g, qw, P0[0], P0[1], P1[0], P1[1], u[2] / gam);
    else deposit_3d((orc_grid *)g, qw, P0, P1);
    if (d) {
        /* time-n momentum: mean of u^{n-1/2} and u^{n+1/2} */
        double um[3] = {0.5 * (u0[0] + u[0]), 0.5 * (u0[1] + u[1]), 0.5 * (u0[2] + u[2])};
        double gmid = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
        d->Ekin[si] += s->w * (gmid - 1.0) * dV;
        for (int a = 0; a < 3; a++) d->P[a] += s->w * um[a] * dV;
    }
    s->X[p] = wrap_pos(P1[0], g->nx);
    s->Y[p] = wrap_pos(P1[1], g->ny);
    if (g->ndim == 3) s->Z[p] = wrap_pos(P1[2], g->nz);
    s->ux[p] = u[0]; s->uy[p] = u[1]; s->uz[p] = u[2];
    if (nsum) {
        /* cell of the new position: the next step's drag mean */
        int64_t c = ngp_cell(g, s, p);
        for (int a = 0; a < 3; a++) nsum[3 * c + a] += u[a];
        ncnt[c] += 1.0;
    }
}

#ifdef _OPENMP
/* The particle loop of one species on all threads (build with -fopenmp; used only to time the
 * oracle on every host core): each thread deposits into its own current and moment arrays,
 * summed afterwards in thread order.  The same per-particle arithmetic as the serial loop; sums
 * are taken in a different order. */
static int step_species_threads(orc_grid *g, orc_species *s, int si, double qm, double qw, double dragf,
                                double dV, orc_diag *d, double *nsum, double *ncnt) {
    const int64_t nc = ncell_of(g);
    const int T = omp_get_max_threads();
    double *J = calloc((size_t)T * 3 * (size_t)nc, sizeof(double));
    double *M = nsum ? calloc((size_t)T * 4 * (size_t)nc, sizeof(double)) : NULL;
    orc_diag *D = calloc((size_t)T, sizeof(orc_diag));
    if (!J || (nsum && !M) || !D) { free(J); free(M); free(D); return -1; }
#pragma omp parallel num_threads(T)
    {
        const int t = omp_get_thread_num();
        orc_grid gl = *g;
        gl.Jx = J + (size_t)t * 3 * nc;
        gl.Jy = gl.Jx + nc;
        gl.Jz = gl.Jy + nc;
        double *ns = M ? M + (size_t)t * 4 * nc : NULL, *nn = ns ? ns + 3 * nc : NULL;
#pragma omp for schedule(static)
        for (int64_t p = 0; p < s->n; p++)
            step_particle(&gl, s, si, p, qm, qw, dragf, dV, d ? &D[t] : NULL, ns, nn);
    }
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; c++)
        for (int t = 0; t < T; t++) {
            const double *Jt = J + (size_t)t * 3 * nc;
            g->Jx[c] += Jt[c];
            g->Jy[c] += Jt[nc + c];
            g->Jz[c] += Jt[2 * nc + c];
            if (M) {
                const double *Mt = M + (size_t)t * 4 * nc;
                for (int a = 0; a < 3; a++) nsum[3 * c + a] += Mt[3 * c + a];
                ncnt[c] += Mt[3 * nc + c];
            }
        }
    if (d)
        for (int t = 0; t < T; t++) {
            d->Ekin[si] += D[t].Ekin[si];
            for (int a = 0; a < 3; a++) d->P[a] += D[t].P[a];
        }
    free(J); free(M); free(D);
    return 0;
}
#endif

int orc_step(orc_grid *g, orc_species *sp, int nsp, orc_diag *d) {
    int64_t nc = ncell_of(g);
    double dV = g->dx * g->dy * (g->ndim == 3 ? g->dz : 1.0);
    if (nsp > ORC_MAX_SPECIES) return -1;
    if (d) {
        memset(d, 0, sizeof(*d));
        field_energy(g, d);
    }
    memset(g->Jx, 0, sizeof(double) * (size_t)nc);
    memset(g->Jy, 0, sizeof(double) * (size_t)nc);
    memset(g->Jz, 0, sizeof(double) * (size_t)nc);

    for (int si = 0; si < nsp; si++) {
        orc_species *s = &sp[si];
        double qm = s->q / s->m, qw = s->q * s->w;
        double dragf = (s->ubar && s->nu > 0.0) ? 1.0 - exp(-s->nu * g->dt) : 0.0;
        double *nsum = NULL, *ncnt = NULL;
        if (s->ubar) {
            nsum = calloc(3 * (size_t)nc, sizeof(double));
            ncnt = calloc((size_t)nc, sizeof(double));
            if (!nsum || !ncnt) { free(nsum); free(ncnt); return -1; }
        }
#ifdef _OPENMP
        if (omp_get_max_threads() > 1) {
            if (step_species_threads(g, s, si, qm, qw, dragf, dV, d, nsum, ncnt) != 0) {
                free(nsum); free(ncnt); return -1;
            }
        } else
#endif
        for (int64_t p = 0; p < s->n; p++)
            step_particle(g, s, si, p, qm, qw, dragf, dV, d, nsum, ncnt);
        if (nsum) {
            for (int64_t c = 0; c < nc; c++)
                for (int a = 0; a < 3; a++)
                    s->ubar[3 * c + a] = ncnt[c] > 0 ? nsum[3 * c + a] / ncnt[c] : 0.0;
            free(nsum); free(ncnt);
        }
    }
    if (g->j_filter) {
        orc_binomial(g, g->Jx);
        orc_binomial(g, g->Jy);
        orc_binomial(g, g->Jz);
    }
    orc_yee(g);
    return 0;
}

/* ---------------------------------------------------------------- charge density */

/* CIC charge density of the given species at the nodes (ions not included). */
void orc_rho(const orc_grid *g, const orc_species *sp, int nsp, double *rho) {
    memset(rho, 0, sizeof(double) * (size_t)ncell_of(g));
    for (int si = 0; si < nsp; si++) {
        const orc_species *s = &sp[si];
        double qw = s->q * s->w;
        for (int64_t p = 0; p < s->n; p++) {
            double X = s->X[p], Y = s->Y[p];
            int i = (int)floor(X), j = (int)floor(Y);
            double ax = X - i, ay = Y - j;
            if (g->ndim == 2) {
                rho[idx2(g, i, j)] += qw * (1 - ax) * (1 - ay);
                rho[idx2(g, i + 1, j)] += qw * ax * (1 - ay);
                rho[idx2(g, i, j + 1)] += qw * (1 - ax) * ay;
                rho[idx2(g, i + 1, j + 1)] += qw * ax * ay;
            } else {
                double Z = s->Z[p];
                int k = (int)floor(Z);
                double az = Z - k;
                for (int dk = 0; dk < 2; dk++)
                    for (int dj = 0; dj < 2; dj++)
                        for (int di = 0; di < 2; di++)
                            rho[idx3(g, i + di, j + dj, k + dk)] +=
                                qw * (di ? ax : 1 - ax) * (dj ? ay : 1 - ay) * (dk ? az : 1 - az);
            }
        }
    }
}

/* Current of a single particle's move, exposed for the deposit checks. */
void orc_deposit_move(orc_grid *g, double qw, const double P0[3], const double P1[3], double vz) {
    if (g->ndim == 2) deposit_2d(g, qw, P0[0], P0[1], P1[0], P1[1], vz);
    else deposit_3d(g, qw, P0, P1);
}

/* E and B at n positions (cell units), out[6 * p + c]; the same gather as the push. */
void orc_gather_many(const orc_grid *g, int64_t n, const double *X, const double *Y,
                     const double *Z, double *out) {
    for (int64_t p = 0; p < n; p++)
        orc_gather(g, X[p], Y[p], Z ? Z[p] : 0.0, out + 6 * p);
}
