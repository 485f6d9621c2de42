/*
 * vlbm_oracle.c -- plain, slow FP64 CPU vielbein lattice Boltzmann on the sphere.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA library is
 * checked against.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg may load it.  It shares no code, header, table
 * generator or constant with the CUDA path (paper_2504_15574_gb300/csrc).
 *
 * What it computes (Ambrus, Busuioc, Gabbana et al., arXiv 2504.15574):
 *   - D2Q16 Gauss-Hermite product quadrature, Sec. 3.1 Eq. (GH_weights),
 *     App. A.2 Tab. velocity_set_Q=4;
 *   - moments n, n u, Eq. (f_moments_sum);
 *   - 3rd-order Hermite equilibrium, App. A.2 Eq. (feq_Q=4);
 *   - BGK collision, Sec. 3.2;
 *   - velocity-derivative kernels K^H, Ktilde^H, Sec. 3.3 Eqs. (KH), (KtildeH),
 *     applied as in Eq. (df): K acts on k_theta at fixed k_phi, Ktilde acts on
 *     k_phi at fixed k_theta (App. A.3);
 *   - flux-form advection on the cell-centred grid, Sec. 3.4-3.5
 *     Eqs. (discrete_coord_sphere), (discrete_advection_sphere);
 *   - WENO-5 fluxes, Eqs. (fluxes_W5), (WENO5_delta), (WENO5_sigma), or the
 *     first/second/third-order upwind fluxes U1-U3, Eq. (fluxes_U1-3);
 *   - optionally the "Komissarov" theta flux, Eqs. (Komissarov_scheme),
 *     (Komissarov_sin_cos): d/dcos(theta) of the interface flux times the
 *     interface sine, V = v_theta, reconstruction on f;
 *   - periodic phi and pole boundary conditions, Sec. 3.6 Eqs. (bcs_phi),
 *     (bcs_theta);
 *   - SSP-RK3 time stepping and the operator L[f], Sec. 3.7 Eq. (Lf).
 *
 * Readings taken where the paper is silent or ambiguous (each also listed in
 * the design notes of the repository):
 *   R1  the WENO weights carry a regulariser: wt_i = delta_i / (sigma_i + eps)^2.
 *   R2/R3  the theta flux is a finite-difference WENO on the nodal values
 *       g = sin(theta) f; the smoothness indicators are taken on g as well.
 *   R4  for negative advection velocity the stencil is mirrored.
 *   R5  ghost rows beyond a pole carry sin() of their own (negative) angle.
 *   R11 an initial temperature T != 1 uses the T-dependent 3rd-order Hermite
 *       projection of the Maxwellian; the BGK target stays at T0 = 1.
 *   R19 sin/cos tables are built on the northern half and mirrored; the
 *       equator row of an odd grid gets cos = 0 exactly.
 *   R8  the Komissarov interface angles are theta_{s+-1/2} = (s - 1/2 +- 1/2) dth
 *       for the 1-based row s (the printed sin((s+1) dth), sin(s dth) is off by
 *       one); its ghost rows take the mapped population f itself (no sine).
 *
 * Layout: populations f[k][i][j], k = 4*a + b (a = k_theta index, b = k_phi
 * index, velocities ascending), i = theta row 0..nt-1 (theta_i = (i+1/2) dth),
 * j = phi column 0..np-1 (phi_j = (j+1/2) dph), j fastest.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no FMA contraction,
 * so results do not depend on the thread count or the host ISA).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NV 4   /* largest quadrature order (Q = 4); Q = 3 uses the first 3 entries */
#define NK 16  /* largest population count Q^2 */

/* ------------------------------------------------------------------------- */
/* Velocity space: Gauss-Hermite Q = 4 (Sec. 3.1, App. A.2)                   */
/* ------------------------------------------------------------------------- */

/* Probabilists' Hermite polynomials H_0..H_5 (Eq. hermite_polynomials and the
 * recurrence H_{l+1} = x H_l - l H_{l-1}). */
static double hermite(int l, double x)
{
    double hm = 1.0, h = x;
    if (l == 0) return 1.0;
    for (int m = 1; m < l; ++m) {
        double hp = x * h - (double)m * hm;
        hm = h;
        h = hp;
    }
    return h;
}

static double factorial(int l)
{
    double r = 1.0;
    for (int m = 2; m <= l; ++m) r *= (double)m;
    return r;
}

/* Roots of H_Q in ascending order and the weights w = Q!/H_{Q+1}(v)^2 (Eq. GH_weights):
 * Q = 4, H_4(x) = x^4 - 6x^2 + 3 (App. A.2, Tab. velocity_set_Q=4); Q = 3, H_3(x) = x^3 - 3x,
 * v = (-sqrt 3, 0, sqrt 3) (App. A.1, Tab. velocity_set_Q=3). */
void vo_quadrature_q(int q, double *v, double *w)
{
    if (q == 3) {
        v[0] = -sqrt(3.0);
        v[1] = 0.0;
        v[2] = sqrt(3.0);
    } else {
        double big = sqrt(3.0 + sqrt(6.0));
        double small = sqrt(3.0 - sqrt(6.0));
        v[0] = -big;
        v[1] = -small;
        v[2] = small;
        v[3] = big;
    }
    for (int a = 0; a < q; ++a) {
        double h = hermite(q + 1, v[a]);
        w[a] = factorial(q) / (h * h);
    }
}

void vo_quadrature(double v[NV], double w[NV]) { vo_quadrature_q(4, v, w); }

/* Kernels of Eqs. (KH) and (KtildeH) for order Q, row-major K[k*Q + k']. */
void vo_kernels_q(int q, double *K, double *Kt)
{
    double v[NV], w[NV];
    vo_quadrature_q(q, v, w);
    for (int k = 0; k < q; ++k) {
        for (int kp = 0; kp < q; ++kp) {
            double sk = 0.0, skt = 0.0;
            for (int l = 0; l < q; ++l) {
                double hk = hermite(l + 1, v[k]);
                sk += hk * hermite(l, v[kp]) / factorial(l);
                double inner = hermite(l + 1, v[kp]);
                if (l > 0) inner += (double)l * hermite(l - 1, v[kp]);
                skt += hk * inner / factorial(l);
            }
            K[k * q + kp] = -w[k] * sk;
            Kt[k * q + kp] = -w[k] * skt;
        }
    }
}

void vo_kernels(double K[NV * NV], double Kt[NV * NV]) { vo_kernels_q(4, K, Kt); }

/* BGK target, T0 = 1: Eq. (feq_Q=4) to third order for Q = 4, Eq. (feq_Q=3) to second
 * order for Q = 3. */
static double feq_k(int q, double n, double wk, double va, double vb, double ut, double up)
{
    double xi = va * ut + vb * up;
    double u2 = ut * ut + up * up;
    if (q == 3) return n * wk * (1.0 + xi + 0.5 * (xi * xi - u2));
    return n * wk * (1.0 + xi + 0.5 * (xi * xi - u2) + xi * (xi * xi - 3.0 * u2) / 6.0);
}

/* Initial state for a temperature T (reading R11): the Hermite projection of
 * the Maxwellian with a^(2) = n[uu + (T-1) delta] and a^(3) = n[uuu + (T-1)(u delta)_sym]
 * (Eqs. feq_series, feq_discrete with the coefficients of a Maxwellian at temperature T),
 * to the order of the quadrature (third for Q = 4, second for Q = 3).  Reduces to feq_k
 * at T = 1. */
static double finit_k(int q, double n, double wk, double va, double vb, double ut, double up, double T)
{
    if (T == 1.0) return feq_k(q, n, wk, va, vb, ut, up);
    double xi = va * ut + vb * up;
    double u2 = ut * ut + up * up;
    double v2 = va * va + vb * vb;
    double dT = T - 1.0;
    double second = xi * xi - u2 + dT * (v2 - 2.0);
    if (q == 3) return n * wk * (1.0 + xi + 0.5 * second);
    double third = xi * (xi * xi - 3.0 * u2) + 3.0 * dT * xi * (v2 - 4.0);
    return n * wk * (1.0 + xi + 0.5 * second + third / 6.0);
}

void vo_equilibrium_q(int q, double n, double ut, double up, double T, double *out)
{
    double v[NV], w[NV];
    vo_quadrature_q(q, v, w);
    for (int a = 0; a < q; ++a)
        for (int b = 0; b < q; ++b)
            out[q * a + b] = finit_k(q, n, w[a] * w[b], v[a], v[b], ut, up, T);
}

void vo_equilibrium(double n, double ut, double up, double T, double out[NK])
{
    vo_equilibrium_q(4, n, ut, up, T, out);
}

/* ------------------------------------------------------------------------- */
/* WENO-5 (Eqs. fluxes_W5, WENO5_delta, WENO5_sigma; reading R1)              */
/* ------------------------------------------------------------------------- */

/* Reconstruction at the interface c+1/2 from the upwind-ordered values
 * (a, b, c, d, e) = (g_{s-2}, g_{s-1}, g_s, g_{s+1}, g_{s+2}). */
double vo_weno5(double a, double b, double c, double d, double e, double eps)
{
    double p1 = (2.0 * a - 7.0 * b + 11.0 * c) / 6.0;
    double p2 = (-b + 5.0 * c + 2.0 * d) / 6.0;
    double p3 = (2.0 * c + 5.0 * d - e) / 6.0;
    double d1a = a - 2.0 * b + c, d1b = a - 4.0 * b + 3.0 * c;
    double d2a = b - 2.0 * c + d, d2b = b - d;
    double d3a = c - 2.0 * d + e, d3b = 3.0 * c - 4.0 * d + e;
    double s1 = 13.0 / 12.0 * (d1a * d1a) + 0.25 * (d1b * d1b);
    double s2 = 13.0 / 12.0 * (d2a * d2a) + 0.25 * (d2b * d2b);
    double s3 = 13.0 / 12.0 * (d3a * d3a) + 0.25 * (d3b * d3b);
    double w1 = 0.1 / ((s1 + eps) * (s1 + eps));
    double w2 = 0.6 / ((s2 + eps) * (s2 + eps));
    double w3 = 0.3 / ((s3 + eps) * (s3 + eps));
    return (w1 * p1 + w2 * p2 + w3 * p3) / (w1 + w2 + w3);
}

/* ------------------------------------------------------------------------- */
/* Solver state                                                               */
/* ------------------------------------------------------------------------- */

enum { VO_WENO5 = 0, VO_U1 = 1, VO_U2 = 2, VO_U3 = 3 };

typedef struct vo_state {
    int q, nk;             /* quadrature order Q (3: D2Q9, 4: D2Q16) and Q^2 populations */
    int nt, np;
    double tau, dt, eps, R;
    int filter;            /* polar ring filter on/off (not in the paper) */
    int scheme;            /* VO_WENO5 (default), VO_U1, VO_U2, VO_U3 */
    int komissarov;        /* theta flux in the Komissarov form */
    double *sin_f, *cos_f; /* per theta interface i = 0..nt, theta = i dth */
    double dth, dph;
    double v[NV], w[NV];
    double K[NV * NV], Kt[NV * NV];
    double *sin_t, *cos_t, *cot_t; /* per row */
    int *fblock;           /* per row block size of the polar filter (1 = off) */
    double *f, *f1, *f2, *L;
    double *Ft, *Fp;       /* interface fluxes of the last operator call */
    double t;
    long long steps;
    double pole_budget;    /* accumulated dt * (RK-weighted pole mass flux) */
    double mass0;
} vo_state;

static size_t plane(const vo_state *o) { return (size_t)o->nt * (size_t)o->np; }

static size_t idx(const vo_state *o, int k, int i, int j)
{
    return ((size_t)k * (size_t)o->nt + (size_t)i) * (size_t)o->np + (size_t)j;
}

/* Block size of the polar ring filter for a row (not in the paper): the
 * smallest power of two b with b sin(theta) dph >= dth / FILTER_RATIO, capped so
 * that b divides np.  Rows where b = 1 are left alone. */
#ifndef FILTER_RATIO
#define FILTER_RATIO 4.0
#endif
static int filter_block(const vo_state *o, int i)
{
    if (!o->filter || o->np < 2) return 1;
    double want = o->dth / (FILTER_RATIO * o->sin_t[i] * o->dph);
    int b = 1;
    while ((double)b < want && b < o->np) b *= 2;
    while (o->np % b != 0) b /= 2;
    return b;
}

vo_state *vo_create_q(int q, int nt, int np, double tau, double dt, double eps, double R, int filter)
{
    if (q != 3 && q != 4) return NULL;
    if (nt < 6 || np < 1 || (np != 1 && np % 2 != 0)) return NULL;
    if (!(tau > 0.0) || !(dt > 0.0) || !(eps > 0.0) || !(R > 0.0)) return NULL;
    vo_state *o = (vo_state *)calloc(1, sizeof(vo_state));
    if (!o) return NULL;
    o->q = q;
    o->nk = q * q;
    o->nt = nt;
    o->np = np;
    o->tau = tau;
    o->dt = dt;
    o->eps = eps;
    o->R = R;
    o->filter = filter ? 1 : 0;
    o->dth = M_PI / (double)nt;
    o->dph = 2.0 * M_PI / (double)np;
    vo_quadrature_q(q, o->v, o->w);
    vo_kernels_q(q, o->K, o->Kt);
    o->sin_t = (double *)malloc(sizeof(double) * nt);
    o->cos_t = (double *)malloc(sizeof(double) * nt);
    o->cot_t = (double *)malloc(sizeof(double) * nt);
    o->sin_f = (double *)malloc(sizeof(double) * (nt + 1));
    o->cos_f = (double *)malloc(sizeof(double) * (nt + 1));
    o->fblock = (int *)malloc(sizeof(int) * nt);
    /* Eq. (discrete_coord_sphere); north half computed, south half mirrored. */
    for (int i = 0; i < nt; ++i) {
        int m = nt - 1 - i;
        if (i <= m) {
            double th = ((double)i + 0.5) * o->dth;
            o->sin_t[i] = sin(th);
            o->cos_t[i] = (i == m) ? 0.0 : cos(th);
        } else {
            o->sin_t[i] = o->sin_t[m];
            o->cos_t[i] = -o->cos_t[m];
        }
    }
    for (int i = 0; i < nt; ++i) o->cot_t[i] = o->cos_t[i] / o->sin_t[i];
    /* interfaces theta_i = i dth (reading R8), northern half computed and mirrored */
    if (o->sin_f && o->cos_f)
        for (int i = 0; i <= nt; ++i) {
            int m = nt - i;
            if (i <= m) {
                double th = (double)i * o->dth;
                o->sin_f[i] = (i == 0) ? 0.0 : sin(th);
                o->cos_f[i] = (i == m) ? 0.0 : cos(th);
            } else {
                o->sin_f[i] = o->sin_f[m];
                o->cos_f[i] = -o->cos_f[m];
            }
        }
    for (int i = 0; i < nt; ++i) o->fblock[i] = filter_block(o, i);
    size_t n = plane(o) * (size_t)o->nk;
    o->f = (double *)calloc(n, sizeof(double));
    o->f1 = (double *)calloc(n, sizeof(double));
    o->f2 = (double *)calloc(n, sizeof(double));
    o->L = (double *)calloc(n, sizeof(double));
    o->Ft = (double *)calloc((size_t)o->nk * (size_t)(nt + 1) * (size_t)np, sizeof(double));
    o->Fp = (double *)calloc((size_t)o->nk * (size_t)nt * (size_t)(np + 1), sizeof(double));
    if (!o->sin_t || !o->cos_t || !o->cot_t || !o->sin_f || !o->cos_f || !o->fblock || !o->f || !o->f1 ||
        !o->f2 || !o->L || !o->Ft || !o->Fp) {
        free(o->sin_t); free(o->cos_t); free(o->cot_t); free(o->sin_f); free(o->cos_f); free(o->fblock);
        free(o->f); free(o->f1); free(o->f2); free(o->L); free(o->Ft); free(o->Fp);
        free(o);
        return NULL;
    }
    return o;
}

vo_state *vo_create(int nt, int np, double tau, double dt, double eps, double R, int filter)
{
    return vo_create_q(4, nt, np, tau, dt, eps, R, filter);
}

void vo_destroy(vo_state *o)
{
    if (!o) return;
    free(o->sin_t); free(o->cos_t); free(o->cot_t); free(o->sin_f); free(o->cos_f); free(o->fblock);
    free(o->f); free(o->f1); free(o->f2); free(o->L); free(o->Ft); free(o->Fp);
    free(o);
}

/* Selects the advection scheme (VO_WENO5, VO_U1, VO_U2, VO_U3) and the Komissarov
 * theta flux; returns -1 for an unknown scheme. */
int vo_set_scheme(vo_state *o, int scheme, int komissarov)
{
    if (!o || scheme < VO_WENO5 || scheme > VO_U3) return -1;
    o->scheme = scheme;
    o->komissarov = komissarov ? 1 : 0;
    return 0;
}

void vo_geometry(const vo_state *o, double *sin_t, double *cos_t, int *fblock)
{
    for (int i = 0; i < o->nt; ++i) {
        if (sin_t) sin_t[i] = o->sin_t[i];
        if (cos_t) cos_t[i] = o->cos_t[i];
        if (fblock) fblock[i] = o->fblock[i];
    }
}

/* ------------------------------------------------------------------------- */
/* Boundary conditions (Sec. 3.6)                                             */
/* ------------------------------------------------------------------------- */

/* f at column j wrapped periodically, Eq. (bcs_phi). */
static int wrap_col(const vo_state *o, int j)
{
    int np = o->np;
    j %= np;
    if (j < 0) j += np;
    return j;
}

/* Nodal theta-flux variable g = sin(theta_i) f at any row i in [-3, nt+2].
 * Rows beyond a pole read the mirrored row on the opposite meridian
 * (column j + np/2) with the reversed velocity -v, i.e. population 15 - k,
 * Eq. (bcs_theta); sin() of the ghost's own angle is negative (reading R5). */
static double g_theta(const vo_state *o, const double *f, int k, int i, int j)
{
    int nt = o->nt;
    if (i >= 0 && i < nt) return o->sin_t[i] * f[idx(o, k, i, j)];
    int half = o->np / 2;
    int jj = wrap_col(o, j + half);
    int kk = o->nk - 1 - k;
    int ii;
    if (i < 0) ii = -1 - i;           /* theta_{-m} = -theta_{m-1} */
    else ii = 2 * nt - 1 - i;         /* theta beyond pi mirrors into the last rows */
    return -o->sin_t[ii] * f[idx(o, kk, ii, jj)];
}

/* f at any row i in [-3, nt+2] for the Komissarov theta flux: rows beyond a pole
 * read the mirrored row and population of Eq. (bcs_theta) without a sine. */
static double f_theta(const vo_state *o, const double *f, int k, int i, int j)
{
    int nt = o->nt;
    if (i >= 0 && i < nt) return f[idx(o, k, i, j)];
    int jj = wrap_col(o, j + o->np / 2);
    int ii = (i < 0) ? -1 - i : 2 * nt - 1 - i;
    return f[idx(o, o->nk - 1 - k, ii, jj)];
}

/* Interface value from the upwind-ordered values a..e (a furthest upwind, c the
 * upwind cell, d the downwind cell): WENO-5 of Eqs. (fluxes_W5)-(WENO5_sigma), or
 * the upwind stencils of Eq. (fluxes_U1-3): U1 c, U2 (3c - b)/2, U3 (2d + 5c - b)/6. */
static double recon(const vo_state *o, double a, double b, double c, double d, double e)
{
    switch (o->scheme) {
    case VO_U1: return c;
    case VO_U2: return 1.5 * c - 0.5 * b;
    case VO_U3: return (2.0 * d + 5.0 * c - b) / 6.0;
    default: return vo_weno5(a, b, c, d, e, o->eps);
    }
}

/* ------------------------------------------------------------------------- */
/* The operator L[g] of Eq. (Lf)                                              */
/* ------------------------------------------------------------------------- */

/* Theta flux through the interface between rows i-1 and i (i = 0..nt):
 * Eq. (discrete_advection_sphere), the reconstruction on g = sin(theta) f; or,
 * Komissarov form, v_theta sin(theta_i) times the reconstruction on f
 * (Eq. Komissarov_scheme with V = v_theta). */
static double flux_theta(const vo_state *o, const double *f, int k, int i, int j)
{
    double vth = o->v[k / o->q];
    double (*val)(const vo_state *, const double *, int, int, int) = o->komissarov ? f_theta : g_theta;
    double gh;
    if (vth > 0.0) {
        gh = recon(o, val(o, f, k, i - 3, j), val(o, f, k, i - 2, j), val(o, f, k, i - 1, j),
                   val(o, f, k, i, j), val(o, f, k, i + 1, j));
    } else {
        gh = recon(o, val(o, f, k, i + 2, j), val(o, f, k, i + 1, j), val(o, f, k, i, j),
                   val(o, f, k, i - 1, j), val(o, f, k, i - 2, j));
    }
    return o->komissarov ? vth * o->sin_f[i] * gh : vth * gh;
}

/* Phi flux through the interface between columns j-1 and j (j = 0..np). */
static double flux_phi(const vo_state *o, const double *f, int k, int i, int j)
{
    double vph = o->v[k % o->q];
    const double *row = f + idx(o, k, i, 0);
    double gh;
    if (vph > 0.0) {
        gh = recon(o, row[wrap_col(o, j - 3)], row[wrap_col(o, j - 2)], row[wrap_col(o, j - 1)],
                   row[wrap_col(o, j)], row[wrap_col(o, j + 1)]);
    } else {
        gh = recon(o, row[wrap_col(o, j + 2)], row[wrap_col(o, j + 1)], row[wrap_col(o, j)],
                   row[wrap_col(o, j - 1)], row[wrap_col(o, j - 2)]);
    }
    return vph * gh;
}

/* Evaluates L[g] into L and the interface fluxes into o->Ft / o->Fp.
 * Returns the rate of change of the total mass caused by the pole fluxes,
 * -R dph sum_{j,k} (F_{nt} - F_{0}). */
static double operator_L(vo_state *o, const double *g, double *L)
{
    int nt = o->nt, np = o->np;
    double R = o->R;

    /* interface fluxes */
#pragma omp parallel for schedule(static)
    for (int i = 0; i <= nt; ++i)
        for (int k = 0; k < o->nk; ++k)
            for (int j = 0; j < np; ++j)
                o->Ft[((size_t)k * (size_t)(nt + 1) + (size_t)i) * (size_t)np + (size_t)j] =
                    flux_theta(o, g, k, i, j);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nt; ++i)
        for (int k = 0; k < o->nk; ++k)
            for (int j = 0; j <= np; ++j)
                o->Fp[((size_t)k * (size_t)nt + (size_t)i) * (size_t)(np + 1) + (size_t)j] =
                    flux_phi(o, g, k, i, j);

#pragma omp parallel for schedule(static)
    for (int i = 0; i < nt; ++i) {
        for (int j = 0; j < np; ++j) {
            double gk[NK];
            for (int k = 0; k < o->nk; ++k) gk[k] = g[idx(o, k, i, j)];
            /* moments, Eq. (f_moments_sum), summed in ascending k */
            double n = 0.0, jt = 0.0, jp = 0.0;
            for (int k = 0; k < o->nk; ++k) {
                n += gk[k];
                jt += gk[k] * o->v[k / o->q];
                jp += gk[k] * o->v[k % o->q];
            }
            double ut = jt / n, up = jp / n;
            for (int k = 0; k < o->nk; ++k) {
                int q = o->q, a = k / q, b = k % q;
                double va = o->v[a], vb = o->v[b];
                double feq = feq_k(q, n, o->w[a] * o->w[b], va, vb, ut, up);
                /* velocity derivatives, Eq. (df) */
                double kg = 0.0, ktg = 0.0;
                for (int m = 0; m < q; ++m) {
                    kg += o->K[a * q + m] * gk[q * m + b];
                    ktg += o->Kt[b * q + m] * gk[q * a + m];
                }
                double force = o->cot_t[i] / R * (vb * vb * kg - va * ktg);
                double ftp = o->Ft[((size_t)k * (size_t)(nt + 1) + (size_t)(i + 1)) * (size_t)np + (size_t)j];
                double ftm = o->Ft[((size_t)k * (size_t)(nt + 1) + (size_t)i) * (size_t)np + (size_t)j];
                double fpp = o->Fp[((size_t)k * (size_t)nt + (size_t)i) * (size_t)(np + 1) + (size_t)(j + 1)];
                double fpm = o->Fp[((size_t)k * (size_t)nt + (size_t)i) * (size_t)(np + 1) + (size_t)j];
                /* Komissarov: -d/dcos(theta) of the interface fluxes (Eq. Komissarov_scheme) */
                double adv_t = o->komissarov ? -(ftp - ftm) / (R * (o->cos_f[i] - o->cos_f[i + 1]))
                                             : -(ftp - ftm) / (R * o->sin_t[i] * o->dth);
                double adv_p = -(fpp - fpm) / (R * o->sin_t[i] * o->dph);
                L[idx(o, k, i, j)] = adv_t + adv_p - force - (gk[k] - feq) / o->tau;
            }
        }
    }

    double s = 0.0;
    for (int k = 0; k < o->nk; ++k)
        for (int j = 0; j < np; ++j) {
            double fs = o->Ft[((size_t)k * (size_t)(nt + 1) + (size_t)nt) * (size_t)np + (size_t)j];
            double fn = o->Ft[((size_t)k * (size_t)(nt + 1)) * (size_t)np + (size_t)j];
            s += fs - fn;
        }
    return -R * o->dph * s;
}

/* Polar ring filter (not in the paper; optional): on every row whose block
 * size b > 1, replace each aligned block of b columns by its mean, per
 * population. */
static void polar_filter(vo_state *o, double *g)
{
    if (!o->filter) return;
    int nt = o->nt, np = o->np;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nt; ++i) {
        int b = o->fblock[i];
        if (b <= 1) continue;
        for (int k = 0; k < o->nk; ++k) {
            double *row = g + idx(o, k, i, 0);
            for (int j0 = 0; j0 < np; j0 += b) {
                double s = 0.0;
                for (int m = 0; m < b; ++m) s += row[j0 + m];
                double mean = s / (double)b;
                for (int m = 0; m < b; ++m) row[j0 + m] = mean;
            }
        }
    }
}

/* One SSP-RK3 step, Sec. 3.7. */
static void rk3_step(vo_state *o)
{
    size_t n = plane(o) * (size_t)o->nk;
    double dt = o->dt;
    double *f = o->f, *f1 = o->f1, *f2 = o->f2, *L = o->L;

    double m1 = operator_L(o, f, L);
#pragma omp parallel for schedule(static)
    for (size_t x = 0; x < n; ++x) f1[x] = f[x] + dt * L[x];
    polar_filter(o, f1);

    double m2 = operator_L(o, f1, L);
#pragma omp parallel for schedule(static)
    for (size_t x = 0; x < n; ++x) f2[x] = 0.75 * f[x] + 0.25 * f1[x] + 0.25 * dt * L[x];
    polar_filter(o, f2);

    double m3 = operator_L(o, f2, L);
#pragma omp parallel for schedule(static)
    for (size_t x = 0; x < n; ++x) f[x] = f[x] / 3.0 + 2.0 / 3.0 * f2[x] + 2.0 / 3.0 * dt * L[x];
    polar_filter(o, f);

    o->pole_budget += dt * (m1 / 6.0 + m2 / 6.0 + 2.0 * m3 / 3.0);
    o->t += dt;
    o->steps += 1;
}

/* ------------------------------------------------------------------------- */
/* Public entry points (mirror of the C ABI, prefixed vo_)                    */
/* ------------------------------------------------------------------------- */

static double total_mass(const vo_state *o, const double *f);

int vo_set_populations(vo_state *o, const double *src)
{
    if (!o || !src) return -1;
    memcpy(o->f, src, plane(o) * (size_t)o->nk * sizeof(double));
    o->t = 0.0;
    o->steps = 0;
    o->pole_budget = 0.0;
    o->mass0 = total_mass(o, o->f);
    return 0;
}

int vo_get_populations(const vo_state *o, double *dst)
{
    if (!o || !dst) return -1;
    memcpy(dst, o->f, plane(o) * (size_t)o->nk * sizeof(double));
    return 0;
}

int vo_init_moments(vo_state *o, const double *rho, const double *ut, const double *up, const double *T)
{
    if (!o || !rho || !ut || !up) return -1;
    for (int i = 0; i < o->nt; ++i)
        for (int j = 0; j < o->np; ++j) {
            size_t c = (size_t)i * (size_t)o->np + (size_t)j;
            double temp = T ? T[c] : 1.0;
            for (int a = 0; a < o->q; ++a)
                for (int b = 0; b < o->q; ++b)
                    o->f[idx(o, o->q * a + b, i, j)] =
                        finit_k(o->q, rho[c], o->w[a] * o->w[b], o->v[a], o->v[b], ut[c], up[c], temp);
        }
    o->t = 0.0;
    o->steps = 0;
    o->pole_budget = 0.0;
    o->mass0 = total_mass(o, o->f);
    return 0;
}

int vo_step(vo_state *o, int n)
{
    if (!o || n < 0) return -1;
    for (int s = 0; s < n; ++s) rk3_step(o);
    return 0;
}

int vo_moments(const vo_state *o, double *rho, double *ut, double *up, double *T)
{
    if (!o || !rho || !ut || !up) return -1;
    for (int i = 0; i < o->nt; ++i)
        for (int j = 0; j < o->np; ++j) {
            size_t c = (size_t)i * (size_t)o->np + (size_t)j;
            double n = 0.0, jt = 0.0, jp = 0.0;
            for (int k = 0; k < o->nk; ++k) {
                double fk = o->f[idx(o, k, i, j)];
                n += fk;
                jt += fk * o->v[k / o->q];
                jp += fk * o->v[k % o->q];
            }
            rho[c] = n;
            ut[c] = jt / n;
            up[c] = jp / n;
            if (T) {
                double e = 0.0;
                for (int k = 0; k < o->nk; ++k) {
                    double ct = o->v[k / o->q] - ut[c], cp = o->v[k % o->q] - up[c];
                    e += o->f[idx(o, k, i, j)] * (ct * ct + cp * cp);
                }
                T[c] = e / (2.0 * n);
            }
        }
    return 0;
}

/* Evaluates L[g] for a caller-supplied population array (layout [k][i][j]) and
 * returns the interface fluxes: Ft[k][i][j] for the interface between rows
 * i-1 and i (i = 0..nt), Fp[k][i][j] between columns j-1 and j (j = 0..np).
 * Any output pointer may be NULL. Returns the pole mass-flux rate. */
double vo_operator(vo_state *o, const double *g, double *L, double *Ft, double *Fp)
{
    double *Lbuf = L ? L : o->L;
    double m = operator_L(o, g, Lbuf);
    if (Ft) memcpy(Ft, o->Ft, sizeof(double) * (size_t)o->nk * (size_t)(o->nt + 1) * (size_t)o->np);
    if (Fp) memcpy(Fp, o->Fp, sizeof(double) * (size_t)o->nk * (size_t)o->nt * (size_t)(o->np + 1));
    return m;
}

static double total_mass(const vo_state *o, const double *f)
{
    double area = o->R * o->R * o->dth * o->dph;
    double m = 0.0;
    for (int i = 0; i < o->nt; ++i) {
        double row = 0.0;
        for (int j = 0; j < o->np; ++j) {
            double n = 0.0;
            for (int k = 0; k < o->nk; ++k) n += f[idx(o, k, i, j)];
            row += n;
        }
        m += o->sin_t[i] * row * area;
    }
    return m;
}

/* out[0] = mass, out[1..3] = Cartesian momentum, out[4] = energy
 * sum f |v|^2 / 2, out[5] = accumulated pole mass flux (dt-weighted),
 * out[6] = initial mass, out[7] = time, out[8] = steps, out[9] = 1 if any
 * population is not finite. Area element R^2 sin(theta) dth dph. */
int vo_diagnostics(const vo_state *o, double out[10])
{
    if (!o || !out) return -1;
    double area = o->R * o->R * o->dth * o->dph;
    double M = 0.0, Px = 0.0, Py = 0.0, Pz = 0.0, E = 0.0;
    int bad = 0;
    for (int i = 0; i < o->nt; ++i) {
        double st = o->sin_t[i], ct = o->cos_t[i];
        for (int j = 0; j < o->np; ++j) {
            double ph = ((double)j + 0.5) * o->dph;
            double sp = sin(ph), cp = cos(ph);
            double n = 0.0, jt = 0.0, jp = 0.0, e = 0.0;
            for (int k = 0; k < o->nk; ++k) {
                double fk = o->f[idx(o, k, i, j)];
                if (!isfinite(fk)) bad = 1;
                double va = o->v[k / o->q], vb = o->v[k % o->q];
                n += fk;
                jt += fk * va;
                jp += fk * vb;
                e += fk * (va * va + vb * vb);
            }
            double dA = st * area;
            M += n * dA;
            Px += (jt * ct * cp - jp * sp) * dA;
            Py += (jt * ct * sp + jp * cp) * dA;
            Pz += (-jt * st) * dA;
            E += 0.5 * e * dA;
        }
    }
    out[0] = M;
    out[1] = Px;
    out[2] = Py;
    out[3] = Pz;
    out[4] = E;
    out[5] = o->pole_budget;
    out[6] = o->mass0;
    out[7] = o->t;
    out[8] = (double)o->steps;
    out[9] = bad ? 1.0 : 0.0;
    return 0;
}
