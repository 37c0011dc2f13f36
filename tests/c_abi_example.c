/*
 * c_abi_example.c -- the C ABI used from plain C (C99, no CUDA headers, no
 * Python): create an FP64 context, set the parameters, load a smooth state
 * and a divergence-free wind, take ten steps on the default stream, read
 * the state back and check it.  Exit status 0 when every check passes.
 *
 * Checks (properties of the step that hold at any size):
 *  - every call returns WX_OK, and the result is finite;
 *  - the tracer's mass h^2 sum q dz is conserved by the dynamics (periodic
 *    in x and y, zero flux through bottom and top, divergence-free winds)
 *    to 1e-12 relative, and equals the library's own FP64 sum;
 *  - q stays inside its initial range (the explicit update is a convex
 *    combination under the positivity bound);
 *  - a state read back and loaded again reproduces the next step bit for
 *    bit (checkpoint / resume);
 *  - out-of-order and bad-argument calls return their status codes.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "wx.h"

#define NX 37
#define NY 29
#define NZ 8
#define N3 ((size_t)NX * NY * NZ)
#define N2 ((size_t)NX * NY)

static int failures = 0;

static void expect(int ok, const char *what) {
    if (!ok) {
        fprintf(stderr, "FAILED: %s\n", what);
        ++failures;
    }
}

static int call(wx_ctx *c, int rc, const char *what) {
    if (rc != WX_OK) fprintf(stderr, "%s -> %d (%s)\n", what, rc, wx_last_error(c));
    expect(rc == WX_OK, what);
    return rc;
}

static double mass(const double *q, const double *dz, double h) {
    double s = 0.0;
    for (int k = 0; k < NZ; ++k)
        for (size_t e = 0; e < N2; ++e) s += q[(size_t)k * N2 + e] * dz[k];
    return h * h * s;
}

int main(void) {
    const double pi = 3.14159265358979323846, h = 2.5;
    double dz[NZ], klev[NZ], alpha[NZ];
    for (int k = 0; k < NZ; ++k) {
        dz[k] = pow(1.05, k);
        klev[k] = 0.01 + 0.005 * k;
        alpha[k] = 0.01 * exp(-k / 8.0);
    }
    double *T = malloc(N3 * sizeof(double)), *q = malloc(N3 * sizeof(double));
    double *T1 = malloc(N3 * sizeof(double)), *q1 = malloc(N3 * sizeof(double));
    double *T2 = malloc(N3 * sizeof(double)), *q2 = malloc(N3 * sizeof(double));
    double *U = malloc(N2 * sizeof(double)), *V = malloc(N2 * sizeof(double));
    double *psi = malloc(N2 * sizeof(double));
    if (!T || !q || !T1 || !q1 || !T2 || !q2 || !U || !V || !psi) return 2;
    for (int k = 0; k < NZ; ++k)
        for (int j = 0; j < NY; ++j)
            for (int i = 0; i < NX; ++i) {
                const size_t e = ((size_t)k * NY + j) * NX + i;
                T[e] = 280.0 + 2.0 * cos(2 * pi * i / NX) * sin(2 * pi * j / NY) + 0.1 * k;
                q[e] = 0.01 + 0.005 * sin(2 * pi * (i + 2 * j) / NX) * cos(pi * (k + 0.5) / NZ);
            }
    /* streamfunction at cell corners; face winds as its differences, so the
       discrete divergence of every cell is zero */
    for (int j = 0; j < NY; ++j)
        for (int i = 0; i < NX; ++i) psi[(size_t)j * NX + i] = 4.0 * sin(2 * pi * i / NX) * cos(2 * pi * j / NY);
    for (int j = 0; j < NY; ++j)
        for (int i = 0; i < NX; ++i) {
            const int jm = (j + NY - 1) % NY, im = (i + NX - 1) % NX;
            U[(size_t)j * NX + i] = -(psi[(size_t)j * NX + i] - psi[(size_t)jm * NX + i]);
            V[(size_t)j * NX + i] = psi[(size_t)j * NX + i] - psi[(size_t)j * NX + im];
        }

    wx_ctx *c = NULL;
    if (call(NULL, wx_create(NX, NY, NZ, WX_F64, &c), "wx_create") != WX_OK) return 1;
    expect(wx_step(c, 1, NULL) == WX_ESTATE, "step before set_params -> WX_ESTATE");
    wx_params p;
    memset(&p, 0, sizeof p);
    p.dt = 0.1;
    p.h = h;
    p.kappa_h = 0.05;
    p.S0 = 1.0;
    p.q_ref = 0.01;
    p.dz = dz;
    p.kappa_lev = klev;
    p.alpha = alpha;
    p.kappa_mult = NULL;
    p.flags = WX_ADVECTION | WX_PHYSICS | WX_SUMS;
    call(c, wx_set_params(c, &p), "wx_set_params");
    wx_params bad = p;
    bad.dt = -1.0;
    expect(wx_set_params(c, &bad) == WX_EINVAL, "negative dt -> WX_EINVAL");
    call(c, wx_load_fields(c, T, q, U, V, 0), "wx_load_fields");
    call(c, wx_step(c, 10, NULL), "wx_step");
    call(c, wx_sync(c), "wx_sync");
    call(c, wx_read_fields(c, T1, q1), "wx_read_fields");

    double qmin = q[0], qmax = q[0];
    int finite = 1;
    for (size_t e = 0; e < N3; ++e) {
        qmin = fmin(qmin, q[e]);
        qmax = fmax(qmax, q[e]);
    }
    int inside = 1;
    for (size_t e = 0; e < N3; ++e) {
        finite = finite && isfinite(T1[e]) && isfinite(q1[e]);
        inside = inside && q1[e] >= qmin - 1e-15 && q1[e] <= qmax + 1e-15;
    }
    expect(finite, "finite state after ten steps");
    expect(inside, "q inside its initial range");
    const double m0 = mass(q, dz, h), m1 = mass(q1, dz, h);
    expect(fabs(m1 - m0) <= 1e-12 * fabs(m0), "tracer mass conserved");
    double ms[16], es[16];
    int n = 0;
    call(c, wx_get_sums(c, ms, es, 16, &n), "wx_get_sums");
    expect(n == 10, "ten sums recorded");
    expect(n > 0 && fabs(ms[n - 1] - m1) <= 1e-12 * fabs(m1), "library sum equals the host sum");

    /* checkpoint / resume: one more step, then the same step from the
       state read back and loaded again */
    call(c, wx_step(c, 1, NULL), "wx_step");
    call(c, wx_sync(c), "wx_sync");
    call(c, wx_read_fields(c, T2, q2), "wx_read_fields");
    call(c, wx_load_fields(c, T1, q1, U, V, 0), "wx_load_fields (resume)");
    call(c, wx_step(c, 1, NULL), "wx_step");
    call(c, wx_sync(c), "wx_sync");
    call(c, wx_read_fields(c, T1, q1), "wx_read_fields");
    expect(memcmp(T1, T2, N3 * sizeof(double)) == 0 && memcmp(q1, q2, N3 * sizeof(double)) == 0,
           "resume reproduces the step bit for bit");

    expect(wx_step(c, -1, NULL) == WX_EINVAL, "negative step count -> WX_EINVAL");
    wx_destroy(c);
    wx_destroy(NULL);
    free(T), free(q), free(T1), free(q1), free(T2), free(q2), free(U), free(V), free(psi);
    if (failures == 0) printf("c_abi_example: all checks passed\n");
    return failures ? 1 : 0;
}
