/*
 * FP64 CPU oracle of the MHD-PIC cosmic-ray particle update
 * (Bai, Caprioli, Sironi & Spitkovsky, arXiv:1412.1087).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference the CUDA path is checked against.  It shares no code, header,
 * table or constant with the CUDA library.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the product path
 * never does.
 *
 * Everything is double precision, one particle at a time, in the order the
 * paper states the method:
 *   Section 2.1  eq:emf0, eq:lorentz2, eq:emfcr2   cell-centred electric field
 *   Section 2.2  eq:4vel, eq:parEk                  four-velocity, gamma, E_k
 *   Section 3    TSC (quadratic spline) interpolation and deposit
 *   App. A.1     eq:nJCR, eq:ng                     particle charge / current
 *   App. A.2     drift-kick-rotate-kick-drift Boris step, E-parallel cleaning
 *   App. A.3     corrector deposit of -dM, -dE_k at x^(n+1/2)
 *
 * Readings where the paper is garbled or silent:
 *   - Boris rotation vector b = (h/2) B / gamma (the standard half angle; the
 *     printed "b = h B / gamma" would double the rotation angle).
 *   - E-parallel cleaning E <- E - (E.B) B / |B|^2, skipped when |B| = 0.
 *   - TSC nodes are cell centres; s = (x - x0)/dx, i = floor(s),
 *     delta = s - i - 1/2, weights 1/2(1/2-delta)^2, 3/4-delta^2,
 *     1/2(1/2+delta)^2 on cells i-1, i, i+1.
 *   - Reflecting boundary: specular (x -> mirror, v_d -> -v_d); a stencil
 *     cell outside the wall is folded onto its mirror cell.  A particle that
 *     lands exactly on the upper wall is placed just inside it.
 *   - m_CR is a per-particle mass; charge and current deposits are divided
 *     by the cell volume dV, the corrector deposit is a momentum / energy
 *     and is divided by dV when it is applied to the gas.
 *   - The kinetic-energy difference E_k(v^(n+1)) - E_k(v^(n)) with
 *     E_k = v^2/(gamma+1) is evaluated as the sum of the changes of the two
 *     half kicks, each as (a-b).(a+b)/(gamma_a+gamma_b): the rotation keeps
 *     |v| exactly, so this equals the difference of the two energies without
 *     its cancellation.
 *   - Without an MHD solver only the corrector deposit is applied to the gas;
 *     the moments n_CR, J_CR deposited at the end of a step feed R, F_CR and
 *     the CR-Hall electric field of the next step.
 *
 * Array layouts: positions x[d*np + j] (d < ndim), four-velocities
 * v[d*np + j] (d < 3), cell arrays plane-major a[q*ncell + c] with
 * c = (k*ny + j)*nx + i.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t ndim;   /* 2 or 3 */
    int32_t n[3];   /* cells per dimension, n[2] = 1 in 2-D */
    double dx[3];   /* cell widths, dx[2] is the cell depth in 2-D */
    double x0[3];   /* lower corner */
    int32_t bc[3];  /* 0 periodic, 1 reflecting walls on both faces, 2 a reflecting wall at the
                       lower face and an open upper face (particles that cross it leave) */
} orc_grid;

typedef struct {
    double qm_cr;   /* (q/mc) of the CR particles */
    double qm_gas;  /* (q/mc)_g of the gas ions */
    double C;       /* artificial speed of light */
    double m_cr;    /* particle "mass" m_CR */
    int32_t hall;   /* 1: include the CR-Hall term in the electric field */
} orc_params;

/* ------------------------------------------------------------------ */
/* small vector helpers                                                */
/* ------------------------------------------------------------------ */

static double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static void cross3(const double a[3], const double b[3], double out[3])
{
    double r0 = a[1] * b[2] - a[2] * b[1];
    double r1 = a[2] * b[0] - a[0] * b[2];
    double r2 = a[0] * b[1] - a[1] * b[0];
    out[0] = r0;
    out[1] = r1;
    out[2] = r2;
}

static int64_t ncell_of(const orc_grid *g)
{
    return (int64_t)g->n[0] * g->n[1] * g->n[2];
}

static double cell_volume(const orc_grid *g)
{
    return g->dx[0] * g->dx[1] * g->dx[2];
}

/* Lorentz factor of a four-velocity v: gamma = sqrt(C^2 + v^2) / C (Section 2.2). */
double orc_gamma(const double v[3], double C)
{
    return sqrt(C * C + dot3(v, v)) / C;
}

/* Kinetic energy per unit mass E_k = (gamma - 1) C^2 = v^2 / (gamma + 1) (eq:parEk). */
double orc_kinetic_energy(const double v[3], double C)
{
    return dot3(v, v) / (orc_gamma(v, C) + 1.0);
}

/* ------------------------------------------------------------------ */
/* TSC shape (Section 3: second-order quadratic spline)                 */
/* ------------------------------------------------------------------ */

/* Weights of the three cell centres nearest to position s (cell units). */
void orc_tsc_weights(double s, int64_t *i, double w[3])
{
    double fi = floor(s);
    double delta = s - fi - 0.5;
    *i = (int64_t)fi;
    w[0] = 0.5 * (0.5 - delta) * (0.5 - delta);
    w[1] = 0.75 - delta * delta;
    w[2] = 0.5 * (0.5 + delta) * (0.5 + delta);
}

/* Map a stencil cell index onto the grid: periodic wrap or mirror fold; at an
 * open face the cells beyond it take the values of the last cell (and receive
 * its deposits). */
static int64_t map_index(const orc_grid *g, int d, int64_t i)
{
    int64_t n = g->n[d];
    if (g->bc[d] == 0) {
        int64_t r = i % n;
        return r < 0 ? r + n : r;
    }
    if (g->bc[d] == 2) {
        if (i < 0)
            i = -1 - i;
        return i >= n ? n - 1 : i;
    }
    /* reflecting: cell -1-k mirrors cell k, cell n+k mirrors cell n-1-k */
    for (;;) {
        if (i < 0)
            i = -1 - i;
        else if (i >= n)
            i = 2 * n - 1 - i;
        else
            return i;
    }
}

/* Stencil of one particle: up to 27 (cell, weight) pairs. Returns the count. */
static int stencil(const orc_grid *g, const double *xp, int64_t cells[27], double wts[27])
{
    int64_t base[3] = {0, 0, 0};
    double w[3][3] = {{0, 1, 0}, {0, 1, 0}, {0, 1, 0}};
    for (int d = 0; d < g->ndim; ++d) {
        double s = (xp[d] - g->x0[d]) / g->dx[d];
        orc_tsc_weights(s, &base[d], w[d]);
    }
    int m = 0;
    int kz = g->ndim == 3 ? 3 : 1;
    for (int c = 0; c < kz; ++c) {
        for (int b = 0; b < 3; ++b) {
            for (int a = 0; a < 3; ++a) {
                int64_t ii = map_index(g, 0, base[0] + a - 1);
                int64_t jj = map_index(g, 1, base[1] + b - 1);
                int64_t kk = 0;
                double wz = 1.0;
                if (g->ndim == 3) {
                    kk = map_index(g, 2, base[2] + c - 1);
                    wz = w[2][c];
                }
                cells[m] = (kk * g->n[1] + jj) * g->n[0] + ii;
                wts[m] = w[0][a] * w[1][b] * wz;
                ++m;
            }
        }
    }
    return m;
}

/* Interpolate nq cell-centred planes (plane-major) to one particle position. */
void orc_gather(const orc_grid *g, const double *xp, const double *planes, int nq, double *out)
{
    int64_t cells[27];
    double wts[27];
    int m = stencil(g, xp, cells, wts);
    int64_t nc = ncell_of(g);
    for (int q = 0; q < nq; ++q) {
        double acc = 0.0;
        for (int k = 0; k < m; ++k)
            acc += wts[k] * planes[q * nc + cells[k]];
        out[q] = acc;
    }
}

/* Deposit nq particle quantities onto nq cell planes with the same weights. */
void orc_deposit(const orc_grid *g, const double *xp, const double *q, int nq, double *planes)
{
    int64_t cells[27];
    double wts[27];
    int m = stencil(g, xp, cells, wts);
    int64_t nc = ncell_of(g);
    for (int k = 0; k < m; ++k)
        for (int a = 0; a < nq; ++a)
            planes[a * nc + cells[k]] += q[a] * wts[k];
}

/* ------------------------------------------------------------------ */
/* particle boundary                                                    */
/* ------------------------------------------------------------------ */

/*
 * Particle boundary.  Periodic wrap; reflecting walls (specular); with bc 2 a
 * reflecting wall at the lower face and an open upper face: a particle at or
 * beyond the open face is put just inside it and the call returns 1 (the
 * particle is leaving the box), else 0.
 */
int orc_boundary(const orc_grid *g, double *xp, double *v)
{
    int left = 0;
    for (int d = 0; d < g->ndim; ++d) {
        double lo = g->x0[d];
        double L = g->n[d] * g->dx[d];
        double hi = lo + L;
        if (g->bc[d] == 2 && xp[d] >= hi) {
            xp[d] = nextafter(hi, lo);
            left = 1;
        } else if (g->bc[d] == 0) {
            double r = xp[d] - lo;
            r -= L * floor(r / L);
            if (r >= L)
                r -= L;
            xp[d] = lo + r;
        } else {
            if (xp[d] < lo) {
                xp[d] = 2.0 * lo - xp[d];
                v[d] = -v[d];
            } else if (xp[d] >= hi) {
                xp[d] = 2.0 * hi - xp[d];
                v[d] = -v[d];
            }
            if (xp[d] >= hi)
                xp[d] = nextafter(hi, lo);
            if (xp[d] < lo)
                xp[d] = lo;
        }
    }
    return left;
}

/* ------------------------------------------------------------------ */
/* cell-centred electric field (Section 2.1, used as in Section 2.2)    */
/* ------------------------------------------------------------------ */

/*
 * E0 = -v_g x B (eq:emf0).  With the CR-Hall term:
 *   n_g = (q/mc)_g rho (eq:ng), R = n_CR / (n_g + n_CR) (eq:defR),
 *   F_CR = (1 - R)(n_CR E0 + J_CR x B) (eq:lorentz2),
 *   E = E0 - F_CR / n_g (eq:emfcr2).
 * mom_dep holds the charge and current densities (n, Jx, Jy, Jz) deposited at
 * the current particle positions.
 */
void orc_field_prep(const orc_grid *g, const orc_params *p, const double *rho, const double *mom,
                    const double *B, const double *mom_dep, double *E)
{
    int64_t nc = ncell_of(g);
    for (int64_t c = 0; c < nc; ++c) {
        double vg[3], Bc[3], E0[3];
        for (int d = 0; d < 3; ++d) {
            vg[d] = mom[d * nc + c] / rho[c];
            Bc[d] = B[d * nc + c];
        }
        double vxb[3];
        cross3(vg, Bc, vxb);
        for (int d = 0; d < 3; ++d)
            E0[d] = -vxb[d];
        if (p->hall) {
            double ng = p->qm_gas * rho[c];
            double n = mom_dep[c];
            double J[3] = {mom_dep[nc + c], mom_dep[2 * nc + c], mom_dep[3 * nc + c]};
            double R = n / (ng + n);
            double JxB[3];
            cross3(J, Bc, JxB);
            for (int d = 0; d < 3; ++d) {
                double F = (1.0 - R) * (n * E0[d] + JxB[d]);
                E[d * nc + c] = E0[d] - F / ng;
            }
        } else {
            for (int d = 0; d < 3; ++d)
                E[d * nc + c] = E0[d];
        }
    }
}

/* ------------------------------------------------------------------ */
/* moments deposit (Appendix A.1, eq:nJCR)                              */
/* ------------------------------------------------------------------ */

/* n_CR += (q/mc) m_CR W / dV,  J_CR += (q/mc) m_CR u W / dV at each position. */
void orc_deposit_moments(const orc_grid *g, const orc_params *p, int64_t np, const double *x,
                         const double *v, double *mom_dep)
{
    double dV = cell_volume(g);
    for (int64_t j = 0; j < np; ++j) {
        double xp[3] = {0, 0, 0}, vj[3];
        if (isnan(x[j]))
            continue;
        for (int d = 0; d < g->ndim; ++d)
            xp[d] = x[d * np + j];
        for (int d = 0; d < 3; ++d)
            vj[d] = v[d * np + j];
        double gam = orc_gamma(vj, p->C);
        double q[4];
        q[0] = p->qm_cr * p->m_cr / dV;
        for (int d = 0; d < 3; ++d)
            q[1 + d] = p->qm_cr * p->m_cr * (vj[d] / gam) / dV;
        orc_deposit(g, xp, q, 4, mom_dep);
    }
}

/* ------------------------------------------------------------------ */
/* particle step (Appendix A.2 and the corrector of Appendix A.3)       */
/* ------------------------------------------------------------------ */

/*
 * One drift-kick-rotate-kick-drift step of every particle with h = (q/mc) dt:
 *   x^(n+1/2) = x^(n) + u^(n) dt/2
 *   E, B interpolated at x^(n+1/2); E <- E - (E.B)B/|B|^2
 *   v^0 = v^(n) + (h/2) E
 *   gamma = gamma(v^0),  b = (h/2) B / gamma
 *   v^1 = v^0 + 2 (v^0 + v^0 x b) x b / (1 + b^2)
 *   v^(n+1) = v^1 + (h/2) E
 *   x^(n+1) = x^(n+1/2) + u^(n+1) dt/2
 * Corrector deposit at x^(n+1/2): corr += (-m dv, -m dE_k) (momentum, energy).
 * Moments deposit at x^(n+1): mom_dep += (n, J) of eq:nJCR.
 * corr holds 4 planes (Mx, My, Mz, E_k); mom_dep holds 4 planes (n, Jx, Jy, Jz).
 * Either deposit pointer may be NULL to skip it.
 * A particle whose first coordinate is NaN is removed (it left the box through
 * an open face) and is skipped.  A particle that reaches an open face at the
 * half step is held just inside it for the gather and the corrector deposit;
 * one that has reached it at the half or the full step is removed after its
 * corrector deposit: no moments deposit, x[0] set to NaN and v to 0 (so that
 * sums over the particles, such as orc_totals, leave it out).
 */
void orc_push(const orc_grid *g, const orc_params *p, double dt, int64_t np, double *x, double *v,
              const double *E, const double *B, double *corr, double *mom_dep)
{
    const double h = p->qm_cr * dt;
    const double C = p->C;
    const double m = p->m_cr;
    const double dV = cell_volume(g);
    int64_t nc = ncell_of(g);
    /* interleave E and B planes for one gather call */
    double *EB = (double *)malloc(sizeof(double) * 6 * (size_t)nc);
    memcpy(EB, E, sizeof(double) * 3 * (size_t)nc);
    memcpy(EB + 3 * nc, B, sizeof(double) * 3 * (size_t)nc);

    for (int64_t j = 0; j < np; ++j) {
        double xp[3] = {0, 0, 0}, vn[3];
        if (isnan(x[j]))
            continue;
        for (int d = 0; d < g->ndim; ++d)
            xp[d] = x[d * np + j];
        for (int d = 0; d < 3; ++d)
            vn[d] = v[d * np + j];

        /* drift to the half step */
        double g0 = orc_gamma(vn, C);
        for (int d = 0; d < g->ndim; ++d)
            xp[d] = xp[d] + 0.5 * dt * (vn[d] / g0);
        int leaving = orc_boundary(g, xp, vn);

        /* fields at x^(n+1/2) */
        double f[6];
        orc_gather(g, xp, EB, 6, f);
        double Ep[3] = {f[0], f[1], f[2]};
        double Bp[3] = {f[3], f[4], f[5]};
        double B2 = dot3(Bp, Bp);
        if (B2 > 0.0) {
            double eb = dot3(Ep, Bp) / B2;
            for (int d = 0; d < 3; ++d)
                Ep[d] -= eb * Bp[d];
        }

        /* kick - rotate - kick */
        double v0[3], v1[3], vnew[3], b[3], t[3], txb[3];
        for (int d = 0; d < 3; ++d)
            v0[d] = vn[d] + 0.5 * h * Ep[d];
        double gam = orc_gamma(v0, C);
        for (int d = 0; d < 3; ++d)
            b[d] = 0.5 * h * Bp[d] / gam;
        cross3(v0, b, t);
        for (int d = 0; d < 3; ++d)
            t[d] += v0[d];
        cross3(t, b, txb);
        double b2 = dot3(b, b);
        for (int d = 0; d < 3; ++d)
            v1[d] = v0[d] + 2.0 * txb[d] / (1.0 + b2);
        for (int d = 0; d < 3; ++d)
            vnew[d] = v1[d] + 0.5 * h * Ep[d];

        /* corrector deposit: -m (v^(n+1) - v^(n)), -m (E_k^(n+1) - E_k^(n)).
         * The rotation keeps |v^1| = |v^0|, so the energy change is the sum of
         * the two half-kick changes, E_k(a) - E_k(b) = (a-b).(a+b)/(gamma_a+gamma_b)
         * with a - b = (h/2)E each time. */
        double g1 = orc_gamma(vnew, C);
        if (corr) {
            double dv[3], s1[3], s0[3], e[3];
            for (int d = 0; d < 3; ++d) {
                dv[d] = vnew[d] - vn[d];
                e[d] = 0.5 * h * Ep[d];
                s1[d] = vnew[d] + v1[d];
                s0[d] = v0[d] + vn[d];
            }
            double dEk = dot3(e, s1) / (g1 + gam) + dot3(e, s0) / (gam + g0);
            double q[4] = {-m * dv[0], -m * dv[1], -m * dv[2], -m * dEk};
            orc_deposit(g, xp, q, 4, corr);
        }

        /* drift to the full step */
        for (int d = 0; d < g->ndim; ++d)
            xp[d] = xp[d] + 0.5 * dt * (vnew[d] / g1);
        leaving |= orc_boundary(g, xp, vnew);
        if (leaving) {
            x[j] = NAN;
            for (int d = 0; d < 3; ++d)
                v[d * np + j] = 0.0;
            continue;
        }

        if (mom_dep) {
            double q[4];
            q[0] = p->qm_cr * m / dV;
            for (int d = 0; d < 3; ++d)
                q[1 + d] = p->qm_cr * m * (vnew[d] / g1) / dV;
            orc_deposit(g, xp, q, 4, mom_dep);
        }

        for (int d = 0; d < g->ndim; ++d)
            x[d * np + j] = xp[d];
        for (int d = 0; d < 3; ++d)
            v[d * np + j] = vnew[d];
    }
    free(EB);
}

/* ------------------------------------------------------------------ */
/* feedback to the gas (Section 2.1 Newton's third law, App. A.3)       */
/* ------------------------------------------------------------------ */

/* rho v += corr_M / dV,  E_gas += corr_E / dV; the corrector planes are zeroed. */
void orc_apply_feedback(const orc_grid *g, double *mom, double *egas, double *corr)
{
    int64_t nc = ncell_of(g);
    double dV = cell_volume(g);
    for (int64_t c = 0; c < nc; ++c) {
        for (int d = 0; d < 3; ++d)
            mom[d * nc + c] += corr[d * nc + c] / dV;
        egas[c] += corr[3 * nc + c] / dV;
    }
    memset(corr, 0, sizeof(double) * 4 * (size_t)nc);
}

/* Totals of gas + CR momentum and energy: out = {Pgas x,y,z, Egas, Pcr x,y,z, Ecr}. */
void orc_totals(const orc_grid *g, const orc_params *p, int64_t np, const double *v,
                const double *mom, const double *egas, double out[8])
{
    int64_t nc = ncell_of(g);
    double dV = cell_volume(g);
    for (int k = 0; k < 8; ++k)
        out[k] = 0.0;
    for (int64_t c = 0; c < nc; ++c) {
        for (int d = 0; d < 3; ++d)
            out[d] += mom[d * nc + c] * dV;
        out[3] += egas[c] * dV;
    }
    for (int64_t j = 0; j < np; ++j) {
        double vj[3] = {v[j], v[np + j], v[2 * np + j]};
        for (int d = 0; d < 3; ++d)
            out[4 + d] += p->m_cr * vj[d];
        out[7] += p->m_cr * orc_kinetic_energy(vj, p->C);
    }
}

/* ------------------------------------------------------------------ */
/* full step: fields, push with both deposits, feedback                 */
/* ------------------------------------------------------------------ */

/*
 * mom_dep holds the moments of the current positions on entry and of the new
 * positions on return.  corr must be zero on entry and is zero on return.
 * E is caller-provided scratch of 3 planes.
 */
void orc_step(const orc_grid *g, const orc_params *p, double dt, int64_t np, double *x, double *v,
              const double *rho, double *mom, double *egas, const double *B, double *mom_dep,
              double *corr, double *E)
{
    int64_t nc = ncell_of(g);
    orc_field_prep(g, p, rho, mom, B, mom_dep, E);
    memset(mom_dep, 0, sizeof(double) * 4 * (size_t)nc);
    orc_push(g, p, dt, np, x, v, E, B, corr, mom_dep);
    orc_apply_feedback(g, mom, egas, corr);
}

/* ------------------------------------------------------------------ */
/* cell sort (the layout of the GPU build; the paper has no sort)        */
/* ------------------------------------------------------------------ */

/*
 * Sort key of a cell with coordinates (i, j, k) for bricks of bx*by*bz cells:
 * the brick number (bricks numbered x fastest) times the brick volume plus the
 * cell's x-fastest number inside its brick.  With a brick equal to the whole
 * grid the key is the linear cell index.
 */
int64_t orc_sort_nkeys(const orc_grid *g, const int32_t brick[3])
{
    int64_t nb = 1, vol = 1;
    for (int d = 0; d < 3; ++d) {
        nb *= (g->n[d] + brick[d] - 1) / brick[d];
        vol *= brick[d];
    }
    return nb * vol;
}

int64_t orc_sort_key(const orc_grid *g, const int32_t brick[3], int64_t cell)
{
    int64_t nx = g->n[0], ny = g->n[1];
    int64_t i = cell % nx;
    int64_t j = (cell / nx) % ny;
    int64_t k = cell / (nx * ny);
    int64_t nbx = (nx + brick[0] - 1) / brick[0];
    int64_t nby = (ny + brick[1] - 1) / brick[1];
    int64_t bid = ((k / brick[2]) * nby + j / brick[1]) * nbx + i / brick[0];
    int64_t in = ((k % brick[2]) * brick[1] + j % brick[1]) * brick[0] + i % brick[0];
    return bid * (int64_t)brick[0] * brick[1] * brick[2] + in;
}

/* Linear cell of each FP64 position: i_d = floor((x_d - x0_d) / dx_d). */
void orc_cells_of(const orc_grid *g, int64_t np, const double *x, int32_t *cell)
{
    for (int64_t j = 0; j < np; ++j) {
        int64_t idx[3] = {0, 0, 0};
        if (isnan(x[j])) {   /* a removed particle */
            cell[j] = -1;
            continue;
        }
        for (int d = 0; d < g->ndim; ++d) {
            int64_t i = (int64_t)floor((x[d * np + j] - g->x0[d]) / g->dx[d]);
            if (i < 0)
                i = 0;
            if (i >= g->n[d])
                i = g->n[d] - 1;
            idx[d] = i;
        }
        cell[j] = (int32_t)((idx[2] * g->n[1] + idx[1]) * g->n[0] + idx[0]);
    }
}

/*
 * Stable counting sort of particles by key.  perm[r] = index of the particle
 * that goes to rank r; counts[key] = particles with that key (nkeys entries).
 * Removed particles (cell -1) go after every key, in their input order.
 */
void orc_sort_cells(const orc_grid *g, const int32_t brick[3], int64_t np, const int32_t *cell,
                    int64_t *perm, int64_t *counts)
{
    int64_t nk = orc_sort_nkeys(g, brick);
    int64_t *start = (int64_t *)calloc((size_t)nk + 2, sizeof(int64_t));
    int64_t *cnt = (int64_t *)calloc((size_t)nk + 1, sizeof(int64_t));
    for (int64_t j = 0; j < np; ++j)
        cnt[cell[j] < 0 ? nk : orc_sort_key(g, brick, cell[j])] += 1;
    for (int64_t k = 0; k <= nk; ++k)
        start[k + 1] = start[k] + cnt[k];
    for (int64_t j = 0; j < np; ++j) {
        int64_t k = cell[j] < 0 ? nk : orc_sort_key(g, brick, cell[j]);
        perm[start[k]++] = j;
    }
    memcpy(counts, cnt, sizeof(int64_t) * (size_t)nk);
    free(start);
    free(cnt);
}

/* ------------------------------------------------------------------ */
/* diagnostics: spectra and E_max (Section 4.3, eq:dpdE, eq:emax),      */
/* the CR-Hall parameter map (Section 2.2, eq:defR, eq:lambda)           */
/* ------------------------------------------------------------------ */

/*
 * Spectrum of the particles inside a region.  The binned quantity of a
 * particle is q = E_k = v^2/(gamma+1) (kind 0, eq:parEk, gamma =
 * sqrt(C^2 + v^2)/C) or q = |v| (kind 1, momentum per unit mass), with
 * v^2 = (vx^2 + vy^2) + vz^2.  The particle counts in bin b when
 * edges[b] <= q < edges[b+1], and, when region is given, when
 * region[2d] <= x_d < region[2d+1] for every d < ndim.  sums[0] and sums[1]
 * are the sums of q^(n+1) and q^n over the same particles, each power a
 * product of n factors q taken left to right: for kind 0 their ratio is the
 * E_max of eq:emax.  f(E) of eq:dpdE is counts[b] / (edges[b+1] - edges[b])
 * per particle number.
 */
void orc_spectrum(const orc_grid *g, const orc_params *p, int64_t np, const double *x, const double *v,
                  int kind, int nbins, const double *edges, const double *region, int n_moment,
                  int64_t *counts, double *sums)
{
    memset(counts, 0, sizeof(int64_t) * (size_t)nbins);
    sums[0] = sums[1] = 0.0;
    for (int64_t j = 0; j < np; ++j) {
        int inside = !isnan(x[j]);   /* removed particles are not counted */
        if (region)
            for (int d = 0; d < g->ndim; ++d) {
                double xd = x[d * np + j];
                if (!(xd >= region[2 * d] && xd < region[2 * d + 1]))
                    inside = 0;
            }
        if (!inside)
            continue;
        double vx = v[j], vy = v[np + j], vz = v[2 * np + j];
        double v2 = vx * vx + vy * vy;
        v2 = v2 + vz * vz;
        double q;
        if (kind == 0) {
            double gam = sqrt(p->C * p->C + v2) / p->C;
            q = v2 / (gam + 1.0);
        } else {
            q = sqrt(v2);
        }
        if (!(q >= edges[0] && q < edges[nbins]))
            continue;
        int b = 0;
        while (b + 1 < nbins && edges[b + 1] <= q)   /* plain linear search */
            ++b;
        counts[b] += 1;
        double qn = 1.0;
        for (int k = 0; k < n_moment; ++k)
            qn = qn * q;
        sums[0] += qn * q;
        sums[1] += qn;
    }
}

/*
 * Lambda = R (u_CR - v_g) / v_A per cell (eq:lambda) with R = n_CR /
 * (n_g + n_CR) (eq:defR), n_g = (q/mc)_g rho (eq:ng), u_CR = J_CR / n_CR,
 * v_g = (rho v)/rho and v_A = |B| / sqrt(rho) (code units).  Written without
 * the division by n_CR: Lambda = (J_CR - n_CR v_g) / ((n_g + n_CR) v_A).
 * Cells with |B| = 0 get Lambda = 0.  mom_dep holds (n, Jx, Jy, Jz).
 */
void orc_lambda_map(const orc_grid *g, const orc_params *p, const double *rho, const double *mom,
                    const double *B, const double *mom_dep, double *lam)
{
    int64_t nc = ncell_of(g);
    for (int64_t c = 0; c < nc; ++c) {
        double Bc[3] = {B[c], B[nc + c], B[2 * nc + c]};
        double vA = sqrt(dot3(Bc, Bc)) / sqrt(rho[c]);
        double n = mom_dep[c];
        double ng = p->qm_gas * rho[c];
        for (int d = 0; d < 3; ++d) {
            double vg = mom[d * nc + c] / rho[c];
            double J = mom_dep[(1 + d) * nc + c];
            lam[d * nc + c] = vA > 0.0 ? (J - n * vg) / ((ng + n) * vA) : 0.0;
        }
    }
}

/* ------------------------------------------------------------------ */
/* coupled step: the predictor-corrector of App. A.3 (eq:scheme)        */
/* ------------------------------------------------------------------ */

/*
 * The gas part G(f, g) of eq:scheme, in one of two models:
 *   model 0  CR sources only: the gas momentum and energy change by the CR
 *            feedback alone and B stays as it is (no induction);
 *   model 1  plane-parallel linear MHD along x: with rho and B_x uniform and
 *            v_x = 0 to first order, the transverse parts of eq:gasmotion and
 *            eq:induction are
 *              d(rho v_y)/dt = B_x dB_y/dx,   d(rho v_z)/dt = B_x dB_z/dx,
 *              dB_y/dt = B_x dv_y/dx,         dB_z/dt = B_x dv_z/dx,
 *            plus, from -c curl of the CR-Hall field -F_CR/n_g (eq:emfcr2),
 *              dB_y/dt += -d(F_z/n_g)/dx,     dB_z/dt += d(F_y/n_g)/dx,
 *            with centred differences (a_{i+1} - a_{i-1}) / (2 dx) and x
 *            periodic.  The gas energy takes only the CR sources (the gas is
 *            isothermal in the paper's linear test, App. B.2).
 *
 * CR sources (eq:gasmotion, eq:engeq): momentum -F_CR with
 * F_CR = (1-R)(n_CR E0 + J_CR x B) (eq:lorentz2), energy -(1-R) J_CR.E0;
 * R = n_CR/(n_g + n_CR) with the CR-Hall term and R = 0 without it.
 */

/* F_CR and (1-R) J.E0 of one cell. */
static void cr_source(const orc_params *p, double rho, const double mom[3], const double B[3], const double md[4],
                      double F[3], double *P)
{
    double vg[3], vxb[3], E0[3], JxB[3];
    for (int d = 0; d < 3; ++d)
        vg[d] = mom[d] / rho;
    cross3(vg, B, vxb);
    for (int d = 0; d < 3; ++d)
        E0[d] = -vxb[d];
    double n = md[0];
    double J[3] = {md[1], md[2], md[3]};
    double R = p->hall ? n / (p->qm_gas * rho + n) : 0.0;
    cross3(J, B, JxB);
    for (int d = 0; d < 3; ++d)
        F[d] = (1.0 - R) * (n * E0[d] + JxB[d]);
    *P = (1.0 - R) * dot3(J, E0);
}

/* Cell of the x neighbour (s = -1 or +1) of cell c, x periodic. */
static int64_t x_neighbour(const orc_grid *g, int64_t c, int s)
{
    int64_t nx = g->n[0];
    int64_t i = c % nx;
    int64_t j = (i + s + nx) % nx;
    return c - i + j;
}

/*
 * Right-hand side of model 1 at state (rho, mom, B) with the CR-Hall field
 * H = F_CR / n_g per cell (3 planes, or NULL): dmom[3 planes], dB[3 planes].
 * Model 0 gives zeros.
 */
void orc_gas_rhs(const orc_grid *g, int model, const double *rho, const double *mom, const double *B,
                 const double *H, double *dmom, double *dB)
{
    int64_t nc = ncell_of(g);
    double h = 1.0 / (2.0 * g->dx[0]);
    for (int64_t c = 0; c < nc; ++c) {
        for (int d = 0; d < 3; ++d) {
            dmom[d * nc + c] = 0.0;
            dB[d * nc + c] = 0.0;
        }
        if (model != 1)
            continue;
        int64_t l = x_neighbour(g, c, -1), r = x_neighbour(g, c, 1);
        double Bx = B[c];
        for (int d = 1; d < 3; ++d) {
            dmom[d * nc + c] = Bx * (B[d * nc + r] - B[d * nc + l]) * h;
            dB[d * nc + c] = Bx * (mom[d * nc + r] / rho[r] - mom[d * nc + l] / rho[l]) * h;
        }
        if (H) {
            dB[nc + c] -= (H[2 * nc + r] - H[2 * nc + l]) * h;
            dB[2 * nc + c] += (H[nc + r] - H[nc + l]) * h;
        }
    }
}

/*
 * Predictor (eq:scheme, first line): g^(n+1/2) = g^n + G(f^n, g^n) dt/2 with
 * the CR sources from the moments mom_dep (n, J at x^n).  Writes the half
 * state (rho_h, mom_h, egas_h, B_h) and the cell-centred electric field E of
 * g^(n+1/2) (with the CR-Hall term from the same moments) for the push.
 * H is scratch of 3 planes.
 */
void orc_gas_predict(const orc_grid *g, const orc_params *p, int model, double dt, const double *rho,
                     const double *mom, const double *egas, const double *B, const double *mom_dep,
                     double *rho_h, double *mom_h, double *egas_h, double *B_h, double *E, double *H,
                     double *dmom, double *dB)
{
    int64_t nc = ncell_of(g);
    double *P = (double *)malloc(sizeof(double) * (size_t)nc);
    double *F = (double *)malloc(sizeof(double) * 3 * (size_t)nc);
    for (int64_t c = 0; c < nc; ++c) {
        double m[3] = {mom[c], mom[nc + c], mom[2 * nc + c]};
        double Bc[3] = {B[c], B[nc + c], B[2 * nc + c]};
        double md[4] = {mom_dep[c], mom_dep[nc + c], mom_dep[2 * nc + c], mom_dep[3 * nc + c]};
        double Fc[3];
        cr_source(p, rho[c], m, Bc, md, Fc, &P[c]);
        for (int d = 0; d < 3; ++d) {
            F[d * nc + c] = Fc[d];
            H[d * nc + c] = p->hall ? Fc[d] / (p->qm_gas * rho[c]) : 0.0;
        }
    }
    orc_gas_rhs(g, model, rho, mom, B, H, dmom, dB);
    for (int64_t c = 0; c < nc; ++c) {
        rho_h[c] = rho[c];
        for (int d = 0; d < 3; ++d) {
            mom_h[d * nc + c] = mom[d * nc + c] + 0.5 * dt * (dmom[d * nc + c] - F[d * nc + c]);
            B_h[d * nc + c] = B[d * nc + c] + 0.5 * dt * dB[d * nc + c];
        }
        egas_h[c] = egas[c] - 0.5 * dt * P[c];
    }
    free(P);
    free(F);
    orc_field_prep(g, p, rho_h, mom_h, B_h, mom_dep, E);
}

/*
 * Corrector (eq:scheme, third line): g^(n+1) = g^n + G((f^n + f^(n+1))/2,
 * g^(n+1/2)) dt, where the CR part is the corrector deposit corr (momentum and
 * energy given to the gas over the step, App. A.3) and the CR-Hall field uses
 * the force it implies, F_CR = -corr_M / (dV dt).  The gas arrays are updated
 * in place (rho is unchanged); corr is zeroed.  H, dmom, dB are scratch.
 */
void orc_gas_correct(const orc_grid *g, const orc_params *p, int model, double dt, const double *rho,
                     double *mom, double *egas, double *B, const double *rho_h, const double *mom_h,
                     const double *B_h, double *corr, double *H, double *dmom, double *dB)
{
    int64_t nc = ncell_of(g);
    double dV = cell_volume(g);
    for (int64_t c = 0; c < nc; ++c)
        for (int d = 0; d < 3; ++d)
            H[d * nc + c] = p->hall ? (-corr[d * nc + c] / (dV * dt)) / (p->qm_gas * rho_h[c]) : 0.0;
    orc_gas_rhs(g, model, rho_h, mom_h, B_h, H, dmom, dB);
    (void)rho;
    for (int64_t c = 0; c < nc; ++c) {
        for (int d = 0; d < 3; ++d) {
            mom[d * nc + c] += dt * dmom[d * nc + c] + corr[d * nc + c] / dV;
            B[d * nc + c] += dt * dB[d * nc + c];
        }
        egas[c] += corr[3 * nc + c] / dV;
    }
    memset(corr, 0, sizeof(double) * 4 * (size_t)nc);
}

/* ------------------------------------------------------------------ */
/* shock front tracking and CR injection (Section 5)                    */
/* ------------------------------------------------------------------ */

/*
 * Counter-based random numbers: Philox4x32 with 10 rounds (Salmon, Moraes,
 * Dror & Shaw 2011, "Parallel random numbers: as easy as 1, 2, 3").  A round
 * multiplies words 0 and 2 by the two round multipliers, mixes the high
 * halves with the other two words and the key, and the key advances by the
 * two Weyl constants between rounds.
 */
static void philox4x32(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0;
        x1 = y1;
        x2 = y2;
        x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
}

void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    philox4x32(ctr, key, out);
}

/* A 32-bit random word as a double in (0, 1). */
static double unit_open(uint32_t u)
{
    return ((double)u + 0.5) * (1.0 / 4294967296.0);
}

/*
 * Shock front along x (Section 5): the transverse average of v_x = (rho v_x)/rho
 * per x cell, smoothed with a Gaussian kernel of standard deviation 4 cells
 * (truncated at 3 standard deviations and at the box ends, renormalised); the
 * upstream value v_up is the smoothed value in the last cell (the inflow side);
 * the front x_s is where, coming from upstream, the smoothed v_x first falls to
 * 0.6 v_up in magnitude (linear interpolation between the two cell centres).
 * The tail x_t is the centre of the first cell at or below the front cell,
 * going downstream, whose smoothed pressure P = (gamma-1)(E - rho v^2/2 - B^2/2)
 * reaches 2/3 of P1 = r/(r-1) rho_up v_up^2 (eq:rh, r = (gamma+1)/(gamma-1),
 * rho_up the smoothed density of the last cell); x0 if none does.
 * out = {x_s (NaN without a front), x_t, rho_up, v_up}.
 */
void orc_front(const orc_grid *g, const double *rho, const double *mom, const double *egas, const double *B,
               double gamma_gas, double out[4])
{
    int64_t nx = g->n[0], nt = (int64_t)g->n[1] * g->n[2], nc = ncell_of(g);
    double *pv = (double *)calloc((size_t)nx, sizeof(double));
    double *pr = (double *)calloc((size_t)nx, sizeof(double));
    double *pp = (double *)calloc((size_t)nx, sizeof(double));
    for (int64_t t = 0; t < nt; ++t)
        for (int64_t i = 0; i < nx; ++i) {
            int64_t c = t * nx + i;
            double r = rho[c];
            double m[3] = {mom[c], mom[nc + c], mom[2 * nc + c]};
            double b[3] = {B[c], B[nc + c], B[2 * nc + c]};
            pv[i] += m[0] / r;
            pr[i] += r;
            pp[i] += (gamma_gas - 1.0) * (egas[c] - 0.5 * dot3(m, m) / r - 0.5 * dot3(b, b));
        }
    for (int64_t i = 0; i < nx; ++i) {
        pv[i] /= (double)nt;
        pr[i] /= (double)nt;
        pp[i] /= (double)nt;
    }
    double *sv = (double *)calloc((size_t)nx, sizeof(double));
    double *sr = (double *)calloc((size_t)nx, sizeof(double));
    double *sp = (double *)calloc((size_t)nx, sizeof(double));
    const double sig = 4.0;
    const int half = 12;
    for (int64_t i = 0; i < nx; ++i) {
        double ws = 0.0, a = 0.0, b = 0.0, c = 0.0;
        for (int k = -half; k <= half; ++k) {
            int64_t j = i + k;
            if (j < 0 || j >= nx)
                continue;
            double w = exp(-0.5 * (double)(k * k) / (sig * sig));
            ws += w;
            a += w * pv[j];
            b += w * pr[j];
            c += w * pp[j];
        }
        sv[i] = a / ws;
        sr[i] = b / ws;
        sp[i] = c / ws;
    }
    double vup = sv[nx - 1], rup = sr[nx - 1];
    double thr = 0.6 * fabs(vup);
    double xs = NAN;
    int64_t is = -1;
    if (vup != 0.0)
        for (int64_t i = nx - 2; i >= 0; --i)
            if (fabs(sv[i]) <= thr) {
                /* crossing between centres i and i+1 */
                double a = fabs(sv[i]), b = fabs(sv[i + 1]);
                double f = (thr - a) / (b - a);
                xs = g->x0[0] + ((double)i + 0.5 + f) * g->dx[0];
                is = i;
                break;
            }
    double xt = g->x0[0];
    if (is >= 0) {
        double r = (gamma_gas + 1.0) / (gamma_gas - 1.0);
        double P1 = r / (r - 1.0) * rup * vup * vup;
        for (int64_t i = is; i >= 0; --i)
            if (sp[i] >= (2.0 / 3.0) * P1) {
                xt = g->x0[0] + ((double)i + 0.5) * g->dx[0];
                break;
            }
    }
    out[0] = xs;
    out[1] = xt;
    out[2] = rup;
    out[3] = vup;
    free(pv);
    free(pr);
    free(pp);
    free(sv);
    free(sr);
    free(sp);
}

/*
 * CR injection at the front (Section 5).  front = {x_s, x_t, rho_up, v_up} of
 * orc_front; xs_prev the front of the previous call (NaN for none) gives the
 * front speed V = (x_s - xs_prev)/dt (0 without one).  The gas mass swept in
 * this step is rho_up (|v_up| + max(V, 0)) dt A (A the box's cross-section);
 * eta of it becomes CR particles of mass m_CR: N = floor(eta M / m_CR + carry),
 * the remainder carried to the next call.  Particle k gets the Philox words of
 * counter (k, call, 0, 0) and key (seed_lo, seed_hi): x = x_s, the transverse
 * coordinates uniform over the box, a direction uniform on the sphere
 * (cos theta = 2u - 1, phi = 2 pi u'), and kinetic energy per unit mass
 * E_k = energy_factor E_sh, E_sh = v_up^2/2, in the frame of the front
 * (gamma' = 1 + E_k/C^2, |v'| = C sqrt(gamma'^2 - 1)); its four-velocity is
 * boosted to the box by V along x (v_x = Gamma (v'_x + V gamma')).  The gas
 * gives the injected mass, momentum (m sum v) and energy (m sum E_k) evenly
 * from the cells whose centres lie in [x_t, x_s) (the front's own cell column
 * when there are none).  New particles go to x_new[d*cap + k], v_new[d*cap + k]
 * for k < N <= cap.  Returns N (0 without a front).
 */
int64_t orc_inject(const orc_grid *g, const orc_params *p, const double front[4], double xs_prev, double dt,
                   double eta, double energy_factor, uint64_t seed, uint32_t call, double *carry, int64_t cap,
                   double *x_new, double *v_new, double *rho, double *mom, double *egas)
{
    double xs = front[0], xt = front[1], rup = front[2], vup = front[3];
    if (isnan(xs))
        return 0;
    double V = isnan(xs_prev) ? 0.0 : (xs - xs_prev) / dt;
    double A = 1.0;
    for (int d = 1; d < 3; ++d)
        A *= (d < g->ndim ? g->n[d] * g->dx[d] : g->dx[d]);
    double M = rup * (fabs(vup) + (V > 0.0 ? V : 0.0)) * dt * A;
    double want = eta * M / p->m_cr + *carry;
    int64_t N = (int64_t)floor(want);
    *carry = want - (double)N;
    if (N > cap)
        N = cap;
    const double C = p->C;
    double Ek = energy_factor * 0.5 * vup * vup;
    double gp = 1.0 + Ek / (C * C);
    double vmag = C * sqrt(gp * gp - 1.0);
    double Gam = 1.0 / sqrt(1.0 - V * V / (C * C));
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    double Pin[3] = {0.0, 0.0, 0.0}, Ein = 0.0;
    for (int64_t k = 0; k < N; ++k) {
        uint32_t ctr[4] = {(uint32_t)k, call, 0u, 0u}, u[4];
        philox4x32(ctr, key, u);
        x_new[k] = xs;
        if (g->ndim >= 2)
            x_new[cap + k] = g->x0[1] + unit_open(u[0]) * g->n[1] * g->dx[1];
        if (g->ndim == 3)
            x_new[2 * cap + k] = g->x0[2] + unit_open(u[1]) * g->n[2] * g->dx[2];
        double mu = 2.0 * unit_open(u[2]) - 1.0;
        double ph = 6.283185307179586 * unit_open(u[3]);   /* 2 pi */
        double st = sqrt(1.0 - mu * mu);
        double vv[3] = {vmag * mu, vmag * st * cos(ph), vmag * st * sin(ph)};
        vv[0] = Gam * (vv[0] + V * gp);
        for (int d = 0; d < 3; ++d) {
            v_new[d * cap + k] = vv[d];
            Pin[d] += p->m_cr * vv[d];
        }
        Ein += p->m_cr * orc_kinetic_energy(vv, C);
    }
    /* compensation: the gas gives what the particles take */
    int64_t nx = g->n[0], nt = (int64_t)g->n[1] * g->n[2], nc = ncell_of(g);
    int64_t i0 = -1, i1 = -1;
    for (int64_t i = 0; i < nx; ++i) {
        double xc = g->x0[0] + ((double)i + 0.5) * g->dx[0];
        if (xc >= xt && xc < xs) {
            if (i0 < 0)
                i0 = i;
            i1 = i;
        }
    }
    if (i0 < 0) {
        i0 = i1 = (int64_t)floor((xs - g->x0[0]) / g->dx[0]);
        if (i0 >= nx)
            i0 = i1 = nx - 1;
    }
    double Vreg = (double)((i1 - i0 + 1) * nt) * cell_volume(g);
    double Min = (double)N * p->m_cr;
    for (int64_t t = 0; t < nt; ++t)
        for (int64_t i = i0; i <= i1; ++i) {
            int64_t c = t * nx + i;
            rho[c] -= Min / Vreg;
            for (int d = 0; d < 3; ++d)
                mom[d * nc + c] -= Pin[d] / Vreg;
            egas[c] -= Ein / Vreg;
        }
    return N;
}

/* ------------------------------------------------------------------ */
/* early-particle removal (Section 5)                                   */
/* ------------------------------------------------------------------ */

/*
 * The shock runs record the injection time t_i of every CR; because the
 * first CRs meet an upstream whose Bell instability has not grown yet, every
 * particle with t_i < t_early is removed at t = 2 t_i.  Called at time t (the
 * end of a step): each live particle with t_inj[j] < t_early and t >= 2
 * t_inj[j] is removed (x[0] = NaN, v = 0, as for a particle that left through
 * an open face).  Returns the number removed.
 */
int64_t orc_remove_early(int ndim, int64_t np, double *x, double *v, const double *t_inj, double t,
                         double t_early)
{
    (void)ndim;
    int64_t n = 0;
    for (int64_t j = 0; j < np; ++j) {
        if (isnan(x[j]))
            continue;
        if (t_inj[j] < t_early && t >= 2.0 * t_inj[j]) {
            x[j] = NAN;
            for (int d = 0; d < 3; ++d)
                v[d * np + j] = 0.0;
            ++n;
        }
    }
    return n;
}
