/*
 * wx_oracle.h -- plain FP64 CPU oracle of one weather-model time step.
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the GPU path.  Only
 * the tests, the smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no source, header, table or helper with the CUDA library
 * and must never be called by the product path.
 *
 * What is computed (one step n -> n+1, dynamics first, then column physics):
 *
 *   Grid: cells (i,j,k), i in [0,nx), j in [0,ny), k in [0,nz), k = 0 at the
 *   bottom; horizontal spacing h, layer thickness dz[k]; periodic in i and j
 *   (the paper's Sec. 3.1 treats the KI/KJ boundaries cyclically), zero flux
 *   through the bottom and the top (the paper's diffusion listing in the
 *   appendix drops the missing vertical neighbour, 1-5d instead of 1-6d).
 *
 *   Dynamics for phi in {T, q} (paper Eq. 1 diffusion term, explicit Euler,
 *   Sec. 3.1; plus flux-form first-order upwind advection on a C grid,
 *   Sec. 2 describes ASUCA's C-grid finite-volume dynamics):
 *     Dh  = kappa_h/h^2 * (phi_E + phi_W + phi_N + phi_S - 4 phi)
 *     Dz  = kappa_h/dz_k * (F_{k+1/2} - F_{k-1/2}),
 *           F_{k+1/2} = (phi_{k+1} - phi_k)/g_{k+1/2},  g = (dz_k+dz_{k+1})/2,
 *           F_{-1/2} = F_{nz-1/2} = 0
 *     Adv = -(1/h) * (U_e phi_e - U_w phi_w + V_n phi_n - V_s phi_s),
 *           face value phi_f taken from the upwind cell: for a face
 *           between cells L (west/south) and R (east/north) it is phi_L
 *           when the face velocity is >= 0 and phi_R otherwise
 *     phi* = phi + dt*(Dh + Dz + Adv)
 *
 *   Column physics (one column at a time: the paper's run_physics, Sec. 3.1
 *   and the appendix listing "Physical processes"):
 *     implicit vertical diffusion of T*:  (I - dt L_v) T** = T*, solved with
 *     the Thomas algorithm, kappa_v(i,j,k) = kappa_mult(i,j)*kappa_lev(k),
 *     interface value = mean of the two adjacent levels;
 *     radiation: dtau_k = alpha_k dz_k q*_k / q_ref, tau_top(k) = sum of dtau
 *     above k, tau_bot(k) = tau_top(k) + dtau_k,
 *     H_k = S0 (exp(-tau_top) - exp(-tau_bot)) / dz_k;
 *     T^{n+1} = T** + dt H,   q^{n+1} = q*.
 *
 * All arrays are C order: 3D fields [nz][ny][nx], 2D fields [ny][nx], face
 * winds U[j][i] on the east face of cell (i,j), V[j][i] on the north face.
 */
#ifndef WX_ORACLE_H
#define WX_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny, nz;
    double dt, h, kappa_h, S0, q_ref;
    const double *dz;         /* [nz] layer thickness                      */
    const double *kappa_lev;  /* [nz] vertical diffusivity profile         */
    const double *alpha;      /* [nz] absorber coefficient                 */
    const double *kappa_mult; /* [ny*nx] per-column multiplier, NULL = 1   */
    int advection;            /* 0: winds ignored                          */
    int physics;              /* 0: T^{n+1} = T*, no Thomas, no radiation  */
} wxo_params;

/* Dynamics only: (T, q) at step n -> (Ts, qs) = (T*, q*). */
void wxo_dynamics(const wxo_params *p, const double *T, const double *q,
                  const double *U, const double *V, double *Ts, double *qs);

/* Coefficients of the implicit vertical-diffusion system of one column
 * (sub-diagonal a, diagonal b, super-diagonal c, each [nz]). */
void wxo_vdiff_coeffs(int nz, double dt, const double *dz,
                      const double *kappa_lev, double kappa_mult,
                      double *a, double *b, double *c);

/* Thomas algorithm: solve a_k x_{k-1} + b_k x_k + c_k x_{k+1} = r_k. */
void wxo_thomas(int nz, const double *a, const double *b, const double *c,
                const double *r, double *x);

/* Radiative heating H[nz] of one column from its q*[nz]. */
void wxo_radiation(int nz, const double *qs, const double *alpha,
                   const double *dz, double S0, double q_ref, double *H);

/* Column physics of ncol independent columns, arrays [ncol][nz]:
 * Tout = T** + dt H; tend (optional, [ncol][2][nz]) = (H, (T** - T*)/dt). */
void wxo_physics_columns(int nz, long ncol, double dt, const double *dz,
                         const double *kappa_lev, const double *kappa_mult,
                         const double *alpha, double S0, double q_ref,
                         const double *Ts, const double *qs,
                         double *Tout, double *tend);

/* One full step (dynamics then physics), out of place. */
void wxo_step(const wxo_params *p, const double *T, const double *q,
              const double *U, const double *V, double *Tn, double *qn);

/* The step's result at ncol sampled columns (i[c], j[c]) only: Tn, qn are
 * [ncol][nz].  Same arithmetic as wxo_step, for checks at sizes where the
 * full oracle step is too slow. */
void wxo_step_columns(const wxo_params *p, const double *T, const double *q,
                      const double *U, const double *V, long ncol,
                      const int *ci, const int *cj, double *Tn, double *qn);

/* n_steps steps with ping-pong buffers; T, q updated in place.  If
 * mass/energy are non-NULL they receive the sums after every step. */
void wxo_run(const wxo_params *p, int n_steps, double *T, double *q,
             const double *U, const double *V, double *mass_q,
             double *energy_T);

/* h^2 * sum over cells of phi*dz_k, accumulated in order k, j, i. */
double wxo_column_weighted_sum(const wxo_params *p, const double *phi);

/* Threads the oracle's parallel loops use (1 when built without OpenMP). */

/* The same step with the dynamics integrated by the three-stage
 * Runge-Kutta scheme of Wicker and Skamarock (2002), the time integrator
 * ASUCA uses (Sec. 2.1): with L the dynamics tendency (phi* = phi + dt L),
 *   phi1 = phi^n + dt/3 L(phi^n),  phi2 = phi^n + dt/2 L(phi1),
 *   phi3 = phi^n + dt L(phi2),
 * then the column physics on (T3, q3) as in wxo_step; q^{n+1} = q3. */
void wxo_step_rk3(const wxo_params *p, const double *T, const double *q,
                  const double *U, const double *V, double *Tn, double *qn);
void wxo_run_rk3(const wxo_params *p, int n_steps, double *T, double *q,
                 const double *U, const double *V);

/* ---------------------------------------------------------------------
 * The paper's reduced weather application, as its listings state it
 * (Sec. 3.1, Eq. 1; appendix: diffusion, physical processes, radiation,
 * heat exchange, time integration).  The field E has a ghost ring that is
 * state of its own: E[k][j][i] with i in [0, nx+2), j in [0, ny+2), k in
 * [0, nz) (k = 0 is the listing's level 1), nz >= 2.  One step:
 *   physics on every column (i, j) of the whole (nx+2) x (ny+2) plane:
 *     E(k) += radiation                                   (radiate)
 *     E(0)    -= transfer (E(0)    - T_surf)              (surface well)
 *     E(nz-1) -= transfer (E(nz-1) - T_pbl)               (planetary well)
 *   then diffusion into a new array (d = diffusion_velocity):
 *     interior i in 1..nx, j in 1..ny, 0 < k < nz-1:
 *       (1 - 6d) E + d (E_i-1 + E_i+1 + E_j-1 + E_j+1 + E_k-1 + E_k+1)
 *     k = 0 and k = nz-1, same i, j: (1 - 5d) E + d (4 horizontal + the
 *       one vertical neighbour)
 *     ghost rows j = 0, ny+1 for i in 0..nx+1, every k:
 *       (1 - 2d) E(i,0) + d (E(i,1) + E(i,ny+1)),
 *       (1 - 2d) E(i,ny+1) + d (E(i,ny) + E(i,0))
 *     ghost columns i = 0, nx+1 for j in 0..ny+1, every k (written last,
 *       so the four corner columns take this rule):
 *       (1 - 2d) E(0,j) + d (E(1,j) + E(nx+1,j)),
 *       (1 - 2d) E(nx+1,j) + d (E(nx,j) + E(0,j))
 * ------------------------------------------------------------------- */
typedef struct {
    int nx, ny, nz;
    double d;          /* diffusion_velocity */
    double radiation;  /* radiation_intensity, added every step */
    double transfer;   /* transfer_velocity of the two heat wells */
    double T_surf;     /* surface heat well (level 0) */
    double T_pbl;      /* planetary-boundary heat well (level nz-1) */
} wxo_pf_params;

/* One step E -> En (arrays of (nx+2)(ny+2)nz doubles, layout above). */
void wxo_pf_step(const wxo_pf_params *p, const double *E, double *En);
/* n steps in place (ping-pong through a scratch copy). */
void wxo_pf_run(const wxo_pf_params *p, int n_steps, double *E);

int wxo_threads(void);
void wxo_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
