/*
 * wx_oracle.c -- plain FP64 CPU oracle of the weather step.
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU baseline).
 * Written for a reader checking it against the paper by eye: every formula
 * is evaluated in the order it is written in wx_oracle.h, with no blocking,
 * fusion or reordering.  Compile with -ffp-contract=off so that no multiply
 * and add are fused behind the reader's back.
 *
 * Sources of each piece:
 *   explicit Euler + kappa*Laplacian       paper Sec. 3.1, Eq. 1
 *   zero-flux vertical ends (1-5d rows)    paper appendix, diffusion listing
 *   periodic horizontal boundaries         paper Sec. 3.1 ("cyclic")
 *   out-of-place update, then swap         paper appendix, time-loop listing
 *   one column per thread for physics      paper Sec. 3.1 and Sec. 2.1
 *   advection, Thomas solve, k-scan        the step definition in the
 *                                          header comment (the paper names
 *                                          C-grid finite-volume dynamics and
 *                                          sequential K dependencies, Sec. 2)
 */
#include "wx_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 0; /* 0 = OpenMP default */

int wxo_threads(void) {
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

void wxo_set_threads(int n) { g_threads = n; }

#define IDX3(p, i, j, k) (((size_t)(k) * (size_t)(p)->ny + (size_t)(j)) * (size_t)(p)->nx + (size_t)(i))
#define IDX2(p, i, j) ((size_t)(j) * (size_t)(p)->nx + (size_t)(i))

/* Upwind face value for a face between a west/south cell L and an
 * east/north cell R carrying velocity u (positive towards R). */
static double upwind(double u, double phiL, double phiR) {
    return (u >= 0.0) ? phiL : phiR;
}

/* The dynamics tendency Dh + Dz + Adv of one field at one cell, as
 * defined in the header; phi* = phi + dt * tendency. */
static double dyn_tendency(const wxo_params *p, const double *phi, const double *U,
                           const double *V, int i, int j, int k) {
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const int ie = (i + 1) % nx, iw = (i - 1 + nx) % nx;
    const int jn = (j + 1) % ny, js = (j - 1 + ny) % ny;

    const double c = phi[IDX3(p, i, j, k)];
    const double pe = phi[IDX3(p, ie, j, k)];
    const double pw = phi[IDX3(p, iw, j, k)];
    const double pn = phi[IDX3(p, i, jn, k)];
    const double ps = phi[IDX3(p, i, js, k)];

    /* D1 horizontal diffusion */
    const double Dh = p->kappa_h / (p->h * p->h) * (pe + pw + pn + ps - 4.0 * c);

    /* D2 vertical diffusion, zero flux through bottom and top */
    double Fup = 0.0, Fdn = 0.0;
    if (k < nz - 1) {
        const double g = 0.5 * (p->dz[k] + p->dz[k + 1]);
        Fup = (phi[IDX3(p, i, j, k + 1)] - c) / g;
    }
    if (k > 0) {
        const double g = 0.5 * (p->dz[k - 1] + p->dz[k]);
        Fdn = (c - phi[IDX3(p, i, j, k - 1)]) / g;
    }
    const double Dz = p->kappa_h / p->dz[k] * (Fup - Fdn);

    /* D3 flux-form first-order upwind advection, C-grid face winds */
    double Adv = 0.0;
    if (p->advection) {
        const double Ue = U[IDX2(p, i, j)];
        const double Uw = U[IDX2(p, iw, j)];
        const double Vn = V[IDX2(p, i, j)];
        const double Vs = V[IDX2(p, i, js)];
        const double fe = Ue * upwind(Ue, c, pe);
        const double fw = Uw * upwind(Uw, pw, c);
        const double fn = Vn * upwind(Vn, c, pn);
        const double fs = Vs * upwind(Vs, ps, c);
        Adv = -(1.0 / p->h) * (fe - fw + fn - fs);
    }

    return Dh + Dz + Adv;
}

/* phi* for one field at one cell. */
static double dyn_cell(const wxo_params *p, const double *phi, const double *U,
                       const double *V, int i, int j, int k) {
    return phi[IDX3(p, i, j, k)] + p->dt * dyn_tendency(p, phi, U, V, i, j, k);
}

void wxo_dynamics(const wxo_params *p, const double *T, const double *q,
                  const double *U, const double *V, double *Ts, double *qs) {
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    int j;
#pragma omp parallel for schedule(static) num_threads(wxo_threads())
    for (j = 0; j < ny; ++j)
        for (int k = 0; k < nz; ++k)
            for (int i = 0; i < nx; ++i) {
                Ts[IDX3(p, i, j, k)] = dyn_cell(p, T, U, V, i, j, k);
                qs[IDX3(p, i, j, k)] = dyn_cell(p, q, U, V, i, j, k);
            }
}

void wxo_vdiff_coeffs(int nz, double dt, const double *dz,
                      const double *kappa_lev, double kappa_mult,
                      double *a, double *b, double *c) {
    for (int k = 0; k < nz; ++k) {
        a[k] = 0.0;
        c[k] = 0.0;
        if (k >= 1) {
            const double kap = kappa_mult * 0.5 * (kappa_lev[k - 1] + kappa_lev[k]);
            const double g = 0.5 * (dz[k - 1] + dz[k]);
            a[k] = -dt * kap / (dz[k] * g);
        }
        if (k <= nz - 2) {
            const double kap = kappa_mult * 0.5 * (kappa_lev[k] + kappa_lev[k + 1]);
            const double g = 0.5 * (dz[k] + dz[k + 1]);
            c[k] = -dt * kap / (dz[k] * g);
        }
        b[k] = 1.0 - a[k] - c[k];
    }
}

void wxo_thomas(int nz, const double *a, const double *b, const double *c,
                const double *r, double *x) {
    double *cp = (double *)malloc(sizeof(double) * (size_t)nz);
    double *dp = (double *)malloc(sizeof(double) * (size_t)nz);
    /* forward elimination */
    cp[0] = c[0] / b[0];
    dp[0] = r[0] / b[0];
    for (int k = 1; k < nz; ++k) {
        const double m = b[k] - a[k] * cp[k - 1];
        cp[k] = c[k] / m;
        dp[k] = (r[k] - a[k] * dp[k - 1]) / m;
    }
    /* back substitution */
    x[nz - 1] = dp[nz - 1];
    for (int k = nz - 2; k >= 0; --k) x[k] = dp[k] - cp[k] * x[k + 1];
    free(cp);
    free(dp);
}

void wxo_radiation(int nz, const double *qs, const double *alpha,
                   const double *dz, double S0, double q_ref, double *H) {
    double *dtau = (double *)malloc(sizeof(double) * (size_t)nz);
    for (int k = 0; k < nz; ++k) dtau[k] = alpha[k] * dz[k] * qs[k] / q_ref;
    /* top-down exclusive scan: tau_top(nz-1) = 0 */
    double tau_top = 0.0;
    for (int k = nz - 1; k >= 0; --k) {
        const double tau_bot = tau_top + dtau[k];
        H[k] = S0 * (exp(-tau_top) - exp(-tau_bot)) / dz[k];
        tau_top = tau_bot;
    }
    free(dtau);
}

/* Physics of one column: Thomas solve of T*, then radiative heating. */
static void physics_column(int nz, double dt, const double *dz,
                           const double *kappa_lev, double kmult,
                           const double *alpha, double S0, double q_ref,
                           const double *Ts, const double *qs, double *Tout,
                           double *H_out, double *vdiff_out, double *work) {
    double *a = work, *b = work + nz, *c = work + 2 * nz;
    double *x = work + 3 * nz, *H = work + 4 * nz;
    wxo_vdiff_coeffs(nz, dt, dz, kappa_lev, kmult, a, b, c);
    wxo_thomas(nz, a, b, c, Ts, x);
    wxo_radiation(nz, qs, alpha, dz, S0, q_ref, H);
    for (int k = 0; k < nz; ++k) {
        Tout[k] = x[k] + dt * H[k];
        if (H_out) H_out[k] = H[k];
        if (vdiff_out) vdiff_out[k] = (x[k] - Ts[k]) / dt;
    }
}

void wxo_physics_columns(int nz, long ncol, double dt, const double *dz,
                         const double *kappa_lev, const double *kappa_mult,
                         const double *alpha, double S0, double q_ref,
                         const double *Ts, const double *qs,
                         double *Tout, double *tend) {
    long col;
#pragma omp parallel num_threads(wxo_threads())
    {
        double *work = (double *)malloc(sizeof(double) * 5 * (size_t)nz);
#pragma omp for schedule(static)
        for (col = 0; col < ncol; ++col) {
            const double km = kappa_mult ? kappa_mult[col] : 1.0;
            physics_column(nz, dt, dz, kappa_lev, km, alpha, S0, q_ref,
                           Ts + col * nz, qs + col * nz, Tout + col * nz,
                           tend ? tend + col * 2 * nz : NULL,
                           tend ? tend + col * 2 * nz + nz : NULL, work);
        }
        free(work);
    }
}

static void physics_all(const wxo_params *p, const double *Ts, const double *qn, double *Tn);

void wxo_step(const wxo_params *p, const double *T, const double *q,
              const double *U, const double *V, double *Tn, double *qn) {
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const size_t n = (size_t)nx * ny * nz;
    double *Ts = (double *)malloc(sizeof(double) * n);
    wxo_dynamics(p, T, q, U, V, Ts, qn);
    physics_all(p, Ts, qn, Tn);
    free(Ts);
}

/* Column physics of every column: Tn from T* and q* (T^{n+1} = T* when the
 * physics is off). */
static void physics_all(const wxo_params *p, const double *Ts, const double *qn, double *Tn) {
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    if (!p->physics) {
        memcpy(Tn, Ts, sizeof(double) * (size_t)nx * ny * nz);
        return;
    }
    int j;
#pragma omp parallel num_threads(wxo_threads())
    {
        double *work = (double *)malloc(sizeof(double) * 8 * (size_t)nz);
        double *cT = work + 5 * nz, *cq = work + 6 * nz, *cout = work + 7 * nz;
#pragma omp for schedule(static)
        for (j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                for (int k = 0; k < nz; ++k) {
                    cT[k] = Ts[IDX3(p, i, j, k)];
                    cq[k] = qn[IDX3(p, i, j, k)];
                }
                const double km = p->kappa_mult ? p->kappa_mult[IDX2(p, i, j)] : 1.0;
                physics_column(nz, p->dt, p->dz, p->kappa_lev, km, p->alpha,
                               p->S0, p->q_ref, cT, cq, cout, NULL, NULL, work);
                for (int k = 0; k < nz; ++k) Tn[IDX3(p, i, j, k)] = cout[k];
            }
        free(work);
    }
}

/* One stage of the three-stage Runge-Kutta scheme: phi_out = phi_n +
 * c dt L(phi_s) for T and q. */
static void rk3_stage(const wxo_params *p, const double *Tn0, const double *qn0, const double *Ts,
                      const double *qs, const double *U, const double *V, double cdt, double *To,
                      double *qo) {
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    int j;
#pragma omp parallel for schedule(static) num_threads(wxo_threads())
    for (j = 0; j < ny; ++j)
        for (int k = 0; k < nz; ++k)
            for (int i = 0; i < nx; ++i) {
                To[IDX3(p, i, j, k)] = Tn0[IDX3(p, i, j, k)] + cdt * dyn_tendency(p, Ts, U, V, i, j, k);
                qo[IDX3(p, i, j, k)] = qn0[IDX3(p, i, j, k)] + cdt * dyn_tendency(p, qs, U, V, i, j, k);
            }
}

void wxo_step_rk3(const wxo_params *p, const double *T, const double *q,
                  const double *U, const double *V, double *Tn, double *qn) {
    const size_t n = (size_t)p->nx * p->ny * p->nz;
    double *w = (double *)malloc(sizeof(double) * 5 * n);
    double *T1 = w, *q1 = w + n, *T2 = w + 2 * n, *q2 = w + 3 * n, *T3 = w + 4 * n;
    rk3_stage(p, T, q, T, q, U, V, p->dt / 3.0, T1, q1);
    rk3_stage(p, T, q, T1, q1, U, V, p->dt / 2.0, T2, q2);
    rk3_stage(p, T, q, T2, q2, U, V, p->dt, T3, qn);
    physics_all(p, T3, qn, Tn);
    free(w);
}

void wxo_run_rk3(const wxo_params *p, int n_steps, double *T, double *q,
                 const double *U, const double *V) {
    const size_t n = (size_t)p->nx * p->ny * p->nz;
    double *Tn = (double *)malloc(sizeof(double) * n), *qn = (double *)malloc(sizeof(double) * n);
    for (int s = 0; s < n_steps; ++s) {
        wxo_step_rk3(p, T, q, U, V, Tn, qn);
        memcpy(T, Tn, sizeof(double) * n);
        memcpy(q, qn, sizeof(double) * n);
    }
    free(Tn);
    free(qn);
}

void wxo_step_columns(const wxo_params *p, const double *T, const double *q,
                      const double *U, const double *V, long ncol,
                      const int *ci, const int *cj, double *Tn, double *qn) {
    const int nz = p->nz;
    long col;
#pragma omp parallel num_threads(wxo_threads())
    {
        double *work = (double *)malloc(sizeof(double) * 7 * (size_t)nz);
        double *cT = work + 5 * nz, *cq = work + 6 * nz;
#pragma omp for schedule(static)
        for (col = 0; col < ncol; ++col) {
            const int i = ci[col], j = cj[col];
            for (int k = 0; k < nz; ++k) {
                cT[k] = dyn_cell(p, T, U, V, i, j, k);
                cq[k] = dyn_cell(p, q, U, V, i, j, k);
                qn[col * nz + k] = cq[k];
            }
            if (p->physics) {
                const double km = p->kappa_mult ? p->kappa_mult[IDX2(p, i, j)] : 1.0;
                physics_column(nz, p->dt, p->dz, p->kappa_lev, km, p->alpha, p->S0,
                               p->q_ref, cT, cq, Tn + col * nz, NULL, NULL, work);
            } else {
                for (int k = 0; k < nz; ++k) Tn[col * nz + k] = cT[k];
            }
        }
        free(work);
    }
}

double wxo_column_weighted_sum(const wxo_params *p, const double *phi) {
    double s = 0.0;
    for (int k = 0; k < p->nz; ++k)
        for (int j = 0; j < p->ny; ++j)
            for (int i = 0; i < p->nx; ++i) s += phi[IDX3(p, i, j, k)] * p->dz[k];
    return p->h * p->h * s;
}

void wxo_run(const wxo_params *p, int n_steps, double *T, double *q,
             const double *U, const double *V, double *mass_q,
             double *energy_T) {
    const size_t n = (size_t)p->nx * p->ny * p->nz;
    double *Tn = (double *)malloc(sizeof(double) * n);
    double *qn = (double *)malloc(sizeof(double) * n);
    double *Tc = T, *qc = q;
    for (int s = 0; s < n_steps; ++s) {
        wxo_step(p, Tc, qc, U, V, Tn, qn);
        /* swap: the new state becomes the current one (no copy) */
        double *t = Tc; Tc = Tn; Tn = t;
        t = qc; qc = qn; qn = t;
        if (mass_q) mass_q[s] = wxo_column_weighted_sum(p, qc);
        if (energy_T) energy_T[s] = wxo_column_weighted_sum(p, Tc);
    }
    if (Tc != T) {
        memcpy(T, Tc, sizeof(double) * n);
        memcpy(q, qc, sizeof(double) * n);
        free(Tc);
        free(qc);
    } else {
        free(Tn);
        free(qn);
    }
}

/* ---------------------------------------------------------------------
 * The paper's reduced weather application (appendix listings), step by
 * step in the listings' order: physics in place on every column, then the
 * four diffusion regions into the new array.
 * ------------------------------------------------------------------- */
#define PF_AT(p, E, i, j, k) (E)[((size_t)(k) * ((p)->ny + 2) + (size_t)(j)) * ((p)->nx + 2) + (size_t)(i)]

static void pf_physics(const wxo_pf_params *p, double *E) {
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    long col;
    const long ncol = (long)(nx + 2) * (ny + 2);
#pragma omp parallel for num_threads(wxo_threads()) schedule(static)
    for (col = 0; col < ncol; ++col) {
        const int i = (int)(col % (nx + 2)), j = (int)(col / (nx + 2));
        /* radiate: uniform heat input on every level */
        for (int k = 0; k < nz; ++k) PF_AT(p, E, i, j, k) = PF_AT(p, E, i, j, k) + p->radiation;
        /* exchange_heat_with_boundary at the surface, then at the top */
        {
            const double x = PF_AT(p, E, i, j, 0);
            const double flux = p->transfer * (x - p->T_surf);
            PF_AT(p, E, i, j, 0) = x - flux;
        }
        {
            const double x = PF_AT(p, E, i, j, nz - 1);
            const double flux = p->transfer * (x - p->T_pbl);
            PF_AT(p, E, i, j, nz - 1) = x - flux;
        }
    }
}

static void pf_diffuse(const wxo_pf_params *p, const double *E, double *En) {
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const double d = p->d;
    int j;
    /* inner region */
#pragma omp parallel for num_threads(wxo_threads()) schedule(static)
    for (j = 1; j <= ny; ++j)
        for (int i = 1; i <= nx; ++i)
            for (int k = 1; k < nz - 1; ++k)
                PF_AT(p, En, i, j, k) = PF_AT(p, E, i, j, k) * (1.0 - 6 * d) +
                                        d * (PF_AT(p, E, i - 1, j, k) + PF_AT(p, E, i + 1, j, k) +
                                             PF_AT(p, E, i, j - 1, k) + PF_AT(p, E, i, j + 1, k) +
                                             PF_AT(p, E, i, j, k - 1) + PF_AT(p, E, i, j, k + 1));
    /* bottom and top levels: one vertical neighbour */
#pragma omp parallel for num_threads(wxo_threads()) schedule(static)
    for (j = 1; j <= ny; ++j)
        for (int i = 1; i <= nx; ++i) {
            PF_AT(p, En, i, j, 0) = (1.0 - 5 * d) * PF_AT(p, E, i, j, 0) +
                                    d * (PF_AT(p, E, i - 1, j, 0) + PF_AT(p, E, i + 1, j, 0) +
                                         PF_AT(p, E, i, j - 1, 0) + PF_AT(p, E, i, j + 1, 0) +
                                         PF_AT(p, E, i, j, 1));
            PF_AT(p, En, i, j, nz - 1) = (1.0 - 5 * d) * PF_AT(p, E, i, j, nz - 1) +
                                         d * (PF_AT(p, E, i - 1, j, nz - 1) + PF_AT(p, E, i + 1, j, nz - 1) +
                                              PF_AT(p, E, i, j - 1, nz - 1) + PF_AT(p, E, i, j + 1, nz - 1) +
                                              PF_AT(p, E, i, j, nz - 2));
        }
    /* ghost rows j = 0 and j = ny+1 */
    for (int i = 0; i <= nx + 1; ++i)
        for (int k = 0; k < nz; ++k) {
            PF_AT(p, En, i, 0, k) = (1.0 - 2 * d) * PF_AT(p, E, i, 0, k) +
                                    d * (PF_AT(p, E, i, 1, k) + PF_AT(p, E, i, ny + 1, k));
            PF_AT(p, En, i, ny + 1, k) = (1.0 - 2 * d) * PF_AT(p, E, i, ny + 1, k) +
                                         d * (PF_AT(p, E, i, ny, k) + PF_AT(p, E, i, 0, k));
        }
    /* ghost columns i = 0 and i = nx+1 (the corners end with this rule) */
    for (j = 0; j <= ny + 1; ++j)
        for (int k = 0; k < nz; ++k) {
            PF_AT(p, En, 0, j, k) = (1.0 - 2 * d) * PF_AT(p, E, 0, j, k) +
                                    d * (PF_AT(p, E, 1, j, k) + PF_AT(p, E, nx + 1, j, k));
            PF_AT(p, En, nx + 1, j, k) = (1.0 - 2 * d) * PF_AT(p, E, nx + 1, j, k) +
                                         d * (PF_AT(p, E, nx, j, k) + PF_AT(p, E, 0, j, k));
        }
}

void wxo_pf_step(const wxo_pf_params *p, const double *E, double *En) {
    const size_t n = (size_t)(p->nx + 2) * (p->ny + 2) * p->nz;
    double *W = (double *)malloc(sizeof(double) * n);
    memcpy(W, E, sizeof(double) * n);
    pf_physics(p, W);
    pf_diffuse(p, W, En);
    free(W);
}

void wxo_pf_run(const wxo_pf_params *p, int n_steps, double *E) {
    const size_t n = (size_t)(p->nx + 2) * (p->ny + 2) * p->nz;
    double *En = (double *)malloc(sizeof(double) * n);
    for (int s = 0; s < n_steps; ++s) {
        pf_physics(p, E);
        pf_diffuse(p, E, En);
        memcpy(E, En, sizeof(double) * n);
    }
    free(En);
}
