/*
 * kt_oracle.c -- plain, slow, FP64 CPU oracle for per-cell implicit integration of
 * stiff thermochemical ODEs (Wang 2025, "The Kratos Framework ...", Sec. 2.2-2.3).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the package smoke check and the
 * benchmark's CPU-baseline / reference legs may load this library.  The CUDA
 * library never calls, links or includes it, and it shares no code, header or
 * table with the CUDA path: it has its own network parser, its own rate law,
 * Jacobian, Crout LU, Newton iteration, step control and projection.
 *
 * Everything is written the obvious way: row-major dense matrices, one cell at a
 * time, the algorithm's steps in the paper's order.  Threads (pthreads, dynamic
 * cell counter) only split independent cells.
 *
 * What is computed (each function cites the passage it follows):
 *   ko_rates       modified Arrhenius k(T) and dk/dT          Sec. 2.2.1 item 1
 *   cell_rates     + tabulated (reduced per cell) and photo    Sec. 2.2.1 items 2-3, Sec. 2.2.2,
 *                  rates k = F sigma (1 - e^-tau)/tau           Eq. photo-reaction-single
 *   ko_rhs         dn/dt = sum A n n + sum B n,  dT/dt        Eq. method-ode-thermochem
 *   ko_jacobian    mass-action + thermal-coupling partials    Eq. method-jacobian, Sec. 2.2.1
 *   ko_lu          Crout LU, implicit-scaled row pivoting     Algorithm lu-decomp, Sec. 2.3.2
 *   ko_lu_solve    forward / back substitution                Sec. 2.3.2
 *   ko_be_solve    one backward-Euler step by Newton          "semi-implicit" solver, Sec. 2.2
 *   ko_integrate   pre-process, adaptive sub-steps (step       Sec. 2.2.2, 2.2.3, 4.2
 *                  doubling), clip + conservation projection,
 *                  retry / revert
 *
 * Readings of the paper taken here (the paper is silent or garbled on these):
 *  - the implicit scheme is backward Euler solved by full Newton; the sub-step
 *    error is estimated by step doubling (one step h vs two steps h/2), the
 *    two-half-step result is kept, h_new = h*min(facmax, max(0.2, 0.9/sqrt(err)));
 *  - Newton converges when |delta_i| <= newton_atol_i + newton_rtol*|y_i| for all i;
 *    a Newton failure halves h;
 *  - Arrhenius: k = A (T/T_ref)^b exp(-theta/T); an exponent below -700 gives k = 0;
 *  - T is the energy variable with a heat capacity per volume C_V = sum_s cv_s n_s
 *    frozen at the cell's initial abundances, so dT/dt = -sum_s h_s dn_s/dt / C_V;
 *  - LU pivot ties go to the smallest row index; a zero pivot fails the Newton solve;
 *  - post-processing clips negatives to zero, then restores the element totals by
 *    the abundance-weighted least-squares correction dy = -diag(y) N^T lambda,
 *    (N diag(y) N^T) lambda = N y - b0, which keeps every relative change tiny;
 *  - retry: from the pre-processed input with h0 * retry_h_factor and
 *    facmax = retry_facmax; a second failure reverts to the pre-processed input.
 */
#include <ctype.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define KO_MAXN 80      /* unknowns per cell (species + T) */
#define KO_MAXE 8       /* elements */
#define KO_MAXSIDE 3    /* reactants / products per reaction */
#define KO_MAXTAB 64    /* tabulated reactions per network */
#define KO_MAXTN 64     /* temperature / density nodes of a rate table */

#define KO_OK 0
#define KO_EINVAL (-1)
#define KO_ENOMEM (-2)
#define KO_EPARSE (-4)
#define KO_ENETWORK (-5)

/* per-cell status */
#define KO_ST_OK 0
#define KO_ST_RETRIED 1
#define KO_ST_REVERTED 2
#define KO_ST_NONFINITE 3

typedef struct {
    int ns, ne, nr, energy;
    double t_ref, t_min, t_max;
    double *mass, *h, *cv;      /* [ns] */
    int *counts;                /* [ns*ne] */
    int *nin, *nout;            /* [nr] */
    int *in, *out;              /* [nr*KO_MAXSIDE] */
    double *A, *b, *theta;      /* [nr] */
    /* rate types (Sec. 2.2.1): 0 modified Arrhenius, 1 tabulated, 2 photo-reaction */
    int *rtype;                 /* [nr] */
    double *sig_r;              /* [nr]: photo cross-section of a type-2 reaction [cm^2] */
    double *sig_s;              /* [ns]: absorption cross-section of each species, the sum
                                   of its photo reactions' [cm^2] */
    int ntab, tab_nT, tab_nR;   /* tabulated reactions and their grid */
    double tab_T0, tab_T1, tab_R0, tab_R1;   /* log-spaced T and rho nodes, end points */
    int *tab_of;                /* [nr]: table row of a type-1 reaction, -1 otherwise */
    double *tab;                /* [ntab][nR][nT]: ln k at the nodes */
    int cvpoly;                 /* 1: heat capacities are two-range polynomials in T */
    double t_mid;               /* boundary of the two ranges [K] */
    double *cvp;                /* [ns*10]: cv_s(T) = sum_k cvp[10s+k] T^k below t_mid,
                                   sum_k cvp[10s+5+k] T^k from t_mid, J/(mol K) */
} ko_net;

/* Heat capacity per volume of one cell, C_V = sum_s cv_s n_s with the composition n0
 * frozen at the cell's pre-processed input (operator split; the paper's Jacobian
 * neglects dC_V/dn as well).  Constant networks: C_V = cv0.  Polynomial networks
 * (Sec. 4.2, NASA-style fits): C_V(T) = sum_s n0_s cv_s(T); with n0 NULL the constant
 * cv0 is used (single-step pins). */
typedef struct {
    double cv0;
    const double *n0;
} ko_heat;

typedef struct {
    double rtol, atol, h_init, h_min;
    double newton_rtol, newton_atol_frac;
    double facmax, retry_h_factor, retry_facmax;
    int max_substeps, max_newton;
    int adaptive;   /* 1: step-doubling control; 0: fixed steps of h_init (pins only) */
    int retry;      /* 1: retry once on failure */
    int atol_mode;  /* 0: atol absolute; 1: atol times the cell's initial element-0 total */
    int guess;      /* Newton start of the second half step: 0 its own start state;
                       2 the full step's result (same end time).  Changes only the
                       iteration count, not the root (to the Newton tolerance). */
    int scheme;     /* 0: backward Euler with step doubling; 1: TR-BDF2 */
} ko_options;

/* ------------------------------------------------------------------ parsing */

static int next_token(FILE *f, char *buf, int cap)
{
    int c, n = 0;
    for (;;) {
        c = fgetc(f);
        if (c == EOF) return 0;
        if (c == '#') {
            while (c != '\n' && c != EOF) c = fgetc(f);
            continue;
        }
        if (!isspace(c)) break;
    }
    while (c != EOF && !isspace(c) && c != '#') {
        if (n < cap - 1) buf[n++] = (char)c;
        c = fgetc(f);
    }
    if (c == '#') ungetc(c, f);
    buf[n] = 0;
    return 1;
}

static int expect(FILE *f, const char *word)
{
    char buf[256];
    return next_token(f, buf, sizeof buf) && strcmp(buf, word) == 0;
}

static int read_int(FILE *f, int *v)
{
    char buf[256], *end;
    if (!next_token(f, buf, sizeof buf)) return 0;
    long x = strtol(buf, &end, 10);
    if (*end) return 0;
    *v = (int)x;
    return 1;
}

static int read_dbl(FILE *f, double *v)
{
    char buf[256], *end;
    if (!next_token(f, buf, sizeof buf)) return 0;
    *v = strtod(buf, &end);
    return *end == 0;
}

void ko_free(ko_net *n)
{
    if (!n) return;
    free(n->mass); free(n->h); free(n->cv); free(n->counts);
    free(n->nin); free(n->nout); free(n->in); free(n->out);
    free(n->A); free(n->b); free(n->theta); free(n->cvp);
    free(n->rtype); free(n->sig_r); free(n->sig_s); free(n->tab_of); free(n->tab);
    free(n);
}

int ko_load(const char *path, ko_net **out)
{
    char buf[256];
    int version, i, j;
    FILE *f = fopen(path, "r");
    if (!f) return KO_EINVAL;
    ko_net *n = calloc(1, sizeof *n);
    if (!n) { fclose(f); return KO_ENOMEM; }
    int ok = expect(f, "kratos_network") && read_int(f, &version) && version == 1 &&
             expect(f, "name") && next_token(f, buf, sizeof buf) &&
             expect(f, "n_species") && read_int(f, &n->ns) &&
             expect(f, "n_elements") && read_int(f, &n->ne) &&
             expect(f, "n_reactions") && read_int(f, &n->nr) &&
             expect(f, "energy") && read_int(f, &n->energy) &&
             expect(f, "t_ref") && read_dbl(f, &n->t_ref) &&
             expect(f, "t_min") && read_dbl(f, &n->t_min) &&
             expect(f, "t_max") && read_dbl(f, &n->t_max) &&
             expect(f, "elements");
    if (ok && (n->ns < 1 || n->ne < 1 || n->ne > KO_MAXE || n->nr < 0 ||
               n->ns + (n->energy ? 1 : 0) > KO_MAXN || (n->energy != 0 && n->energy != 1)))
        ok = 0;
    if (!ok) { fclose(f); ko_free(n); return KO_EPARSE; }
    for (i = 0; i < n->ne && ok; i++) ok = next_token(f, buf, sizeof buf);
    n->mass = calloc(n->ns, sizeof(double));
    n->h = calloc(n->ns, sizeof(double));
    n->cv = calloc(n->ns, sizeof(double));
    n->counts = calloc((size_t)n->ns * n->ne, sizeof(int));
    n->nin = calloc(n->nr + 1, sizeof(int));
    n->nout = calloc(n->nr + 1, sizeof(int));
    n->in = calloc((size_t)(n->nr + 1) * KO_MAXSIDE, sizeof(int));
    n->out = calloc((size_t)(n->nr + 1) * KO_MAXSIDE, sizeof(int));
    n->A = calloc(n->nr + 1, sizeof(double));
    n->b = calloc(n->nr + 1, sizeof(double));
    n->theta = calloc(n->nr + 1, sizeof(double));
    if (!n->mass || !n->h || !n->cv || !n->counts || !n->nin || !n->nout || !n->in ||
        !n->out || !n->A || !n->b || !n->theta) {
        fclose(f); ko_free(n); return KO_ENOMEM;
    }
    for (i = 0; i < n->ns && ok; i++) {
        ok = expect(f, "species") && next_token(f, buf, sizeof buf) &&
             read_dbl(f, &n->mass[i]) && read_dbl(f, &n->h[i]) && read_dbl(f, &n->cv[i]);
        for (j = 0; j < n->ne && ok; j++) ok = read_int(f, &n->counts[i * n->ne + j]);
    }
    for (i = 0; i < n->nr && ok; i++) {
        int pair;
        ok = expect(f, "reaction") && read_int(f, &n->nin[i]) &&
             n->nin[i] >= 1 && n->nin[i] <= KO_MAXSIDE;
        for (j = 0; j < n->nin[i] && ok; j++)
            ok = read_int(f, &n->in[i * KO_MAXSIDE + j]) &&
                 n->in[i * KO_MAXSIDE + j] >= 0 && n->in[i * KO_MAXSIDE + j] < n->ns;
        ok = ok && read_int(f, &n->nout[i]) && n->nout[i] >= 0 && n->nout[i] <= KO_MAXSIDE;
        for (j = 0; j < n->nout[i] && ok; j++)
            ok = read_int(f, &n->out[i * KO_MAXSIDE + j]) &&
                 n->out[i * KO_MAXSIDE + j] >= 0 && n->out[i * KO_MAXSIDE + j] < n->ns;
        ok = ok && read_dbl(f, &n->A[i]) && read_dbl(f, &n->b[i]) &&
             read_dbl(f, &n->theta[i]) && read_int(f, &pair);
    }
    /* optional sections (heat capacities, photo-reactions, rate tables), then "end" */
    n->rtype = calloc(n->nr + 1, sizeof(int));
    n->sig_r = calloc(n->nr + 1, sizeof(double));
    n->sig_s = calloc(n->ns, sizeof(double));
    n->tab_of = malloc((n->nr + 1) * sizeof(int));
    if (!n->rtype || !n->sig_r || !n->sig_s || !n->tab_of) ok = 0;
    for (i = 0; ok && i < n->nr; i++) n->tab_of[i] = -1;
    while (ok) {
        ok = next_token(f, buf, sizeof buf);
        if (!ok || strcmp(buf, "end") == 0) break;
        if (strcmp(buf, "cv_poly") == 0 && !n->cvpoly) {
            n->cvpoly = 1;
            n->cvp = calloc((size_t)n->ns * 10, sizeof(double));
            ok = n->cvp != NULL && n->energy == 1 && read_dbl(f, &n->t_mid) && n->t_mid > 0.0;
            for (i = 0; i < n->ns && ok; i++) {
                int sp;
                ok = expect(f, "cvp") && read_int(f, &sp) && sp == i;
                for (j = 0; j < 10 && ok; j++) ok = read_dbl(f, &n->cvp[i * 10 + j]);
            }
        } else if (strcmp(buf, "photo") == 0) {
            /* photo <count>, then "ph <reaction> <cross-section>" (one reactant each) */
            int np;
            ok = read_int(f, &np) && np >= 0 && np <= n->nr;
            for (i = 0; i < np && ok; i++) {
                int r;
                double sg;
                ok = expect(f, "ph") && read_int(f, &r) && r >= 0 && r < n->nr && read_dbl(f, &sg) &&
                     sg >= 0.0 && n->nin[r] == 1 && n->rtype[r] == 0;
                if (ok) {
                    n->rtype[r] = 2;
                    n->sig_r[r] = sg;
                    n->sig_s[n->in[r * KO_MAXSIDE]] += sg;
                }
            }
        } else if (strcmp(buf, "rate_table") == 0 && !n->tab) {
            /* rate_table <nT> <T0> <T1> <nR> <rho0> <rho1> <count>, then per reaction
             * "tab <reaction>" and nR x nT values of ln k (rho-major) */
            ok = read_int(f, &n->tab_nT) && read_dbl(f, &n->tab_T0) && read_dbl(f, &n->tab_T1) &&
                 read_int(f, &n->tab_nR) && read_dbl(f, &n->tab_R0) && read_dbl(f, &n->tab_R1) &&
                 read_int(f, &n->ntab) && n->tab_nT >= 2 && n->tab_nT <= KO_MAXTN && n->tab_nR >= 1 &&
                 n->tab_nR <= KO_MAXTN && n->ntab >= 0 && n->ntab <= KO_MAXTAB && n->ntab <= n->nr &&
                 n->tab_T0 > 0.0 && n->tab_T1 > n->tab_T0 && n->tab_R0 > 0.0 &&
                 (n->tab_nR == 1 || n->tab_R1 > n->tab_R0);
            if (ok) n->tab = calloc((size_t)(n->ntab + 1) * n->tab_nR * n->tab_nT, sizeof(double));
            ok = ok && n->tab != NULL;
            for (i = 0; i < n->ntab && ok; i++) {
                int r, q, m = n->tab_nR * n->tab_nT;
                ok = expect(f, "tab") && read_int(f, &r) && r >= 0 && r < n->nr && n->rtype[r] == 0;
                if (ok) {
                    n->rtype[r] = 1;
                    n->tab_of[r] = i;
                }
                for (q = 0; q < m && ok; q++) ok = read_dbl(f, &n->tab[(size_t)i * m + q]);
            }
        } else {
            ok = 0;
        }
    }
    fclose(f);
    if (!ok) { ko_free(n); return KO_EPARSE; }
    /* every reaction must conserve every element (Eq. method-const-elem) */
    for (i = 0; i < n->nr; i++) {
        int e;
        for (e = 0; e < n->ne; e++) {
            int bal = 0;
            for (j = 0; j < n->nin[i]; j++) bal -= n->counts[n->in[i * KO_MAXSIDE + j] * n->ne + e];
            for (j = 0; j < n->nout[i]; j++) bal += n->counts[n->out[i * KO_MAXSIDE + j] * n->ne + e];
            if (bal != 0) { ko_free(n); return KO_ENETWORK; }
        }
    }
    *out = n;
    return KO_OK;
}

int ko_info(const ko_net *n, int *ns, int *ne, int *nr, int *energy)
{
    *ns = n->ns; *ne = n->ne; *nr = n->nr; *energy = n->energy;
    return KO_OK;
}

/* ------------------------------------------------------------------ rate law */

/* Modified Arrhenius coefficient (Sec. 2.2.1, item 1): k = A (T/T_ref)^b exp(-theta/T),
 * dk/dT = k (b + theta/T) / T.  Exponents below -700 are flushed to k = 0. */
int ko_rates(const ko_net *n, double T, double *k, double *dkdT)
{
    int r;
    if (!(T > 0.0)) return KO_EINVAL;
    double lt = log(T / n->t_ref);
    for (r = 0; r < n->nr; r++) {
        double arg = n->b[r] * lt - n->theta[r] / T;
        if (arg < -700.0) {
            k[r] = 0.0;
            dkdT[r] = 0.0;
        } else {
            k[r] = n->A[r] * exp(arg);
            dkdT[r] = k[r] * (n->b[r] + n->theta[r] / T) / T;
        }
    }
    return KO_OK;
}

/* C_V of the cell at temperature T and its derivative dC_V/dT (see ko_heat). */
static double heat_capacity(const ko_net *n, const ko_heat *hc, double T, double *dcv)
{
    int s, k;
    if (!n->cvpoly || !hc->n0) {
        *dcv = 0.0;
        return hc->cv0;
    }
    double c = 0.0, d = 0.0;
    for (s = 0; s < n->ns; s++) {
        const double *a = n->cvp + s * 10 + (T < n->t_mid ? 0 : 5);
        double v = 0.0, dv = 0.0, tk = 1.0;
        for (k = 0; k < 5; k++) {
            v += a[k] * tk;
            if (k < 4) dv += (k + 1) * a[k + 1] * tk;
            tk *= T;
        }
        c += hc->n0[s] * v;
        d += hc->n0[s] * dv;
    }
    *dcv = d;
    return c;
}

/* Per-cell radiation and table data: the photo flux factor F = L dl / dV and path
 * length dl of Eq. photo-reaction-single, and the cell's rate tables reduced to one
 * dimension in T at its density (Sec. 2.2.2, "rate table generation"). */
typedef struct {
    double flux, path;
    const double *ltab;         /* [ntab][nT] ln k at the T nodes */
} ko_rad;

/* Pre-processing of the tables: ln k at the T nodes for density rho, linear in ln rho
 * between the two bracketing density nodes (clamped to the grid). */
static void table_reduce(const ko_net *n, double rho, double *ltab)
{
    int t, j, nT = n->tab_nT, nR = n->tab_nR;
    double u = 0.0, w = 0.0;
    int i = 0;
    if (nR > 1) {
        u = (log(rho) - log(n->tab_R0)) / (log(n->tab_R1) - log(n->tab_R0)) * (nR - 1);
        if (!(u > 0.0)) u = 0.0;
        if (u > nR - 1) u = nR - 1;
        i = (int)floor(u);
        if (i > nR - 2) i = nR - 2;
        w = u - i;
    }
    for (t = 0; t < n->ntab; t++)
        for (j = 0; j < nT; j++) {
            const double *row = n->tab + ((size_t)t * nR + i) * nT;
            ltab[t * nT + j] = nR > 1 ? (1.0 - w) * row[j] + w * row[nT + j] : row[j];
        }
}

/* k and dk/dT of tabulated reaction t at T: ln k linear in ln T between the nodes
 * (so dk/dT = k (ln k_{j+1} - ln k_j) / (d ln T) / T), constant beyond the grid. */
static void table_eval(const ko_net *n, const double *ltab, int t, double T, double *k, double *dk)
{
    const double *L = ltab + t * n->tab_nT;
    int nT = n->tab_nT;
    double dl = (log(n->tab_T1) - log(n->tab_T0)) / (nT - 1);
    double v = (log(T) - log(n->tab_T0)) / dl;
    if (!(v > 0.0)) { *k = exp(L[0]); *dk = 0.0; return; }
    if (v >= nT - 1) { *k = exp(L[nT - 1]); *dk = 0.0; return; }
    int j = (int)floor(v);
    if (j > nT - 2) j = nT - 2;
    double fr = v - j;
    *k = exp(L[j] + fr * (L[j + 1] - L[j]));
    *dk = *k * ((L[j + 1] - L[j]) / dl) / T;
}

/* phi(tau) = (1 - exp(-tau)) / tau (Eq. photo-reaction-single) and its derivative;
 * below tau = 0.1 by their Taylor series (8 terms), where the closed forms cancel. */
static void photo_phi(double tau, double *phi, double *dphi)
{
    if (tau < 0.1) {
        /* phi = sum_k (-tau)^k / (k+1)!,  phi' = sum_{k>=1} (-1)^k k tau^(k-1) / (k+1)! */
        double p = 0.0, d = 0.0, pw = 1.0, pwm = 0.0, fact = 1.0;
        int k;
        for (k = 0; k < 9; k++) {
            fact *= (k + 1);
            double sg = (k & 1) ? -1.0 : 1.0;
            p += sg * pw / fact;
            if (k >= 1) d += sg * k * pwm / fact;
            pwm = pw;
            pw *= tau;
        }
        *phi = p;
        *dphi = d;
    } else {
        double e = exp(-tau);
        *phi = (1.0 - e) / tau;
        *dphi = (e * (1.0 + tau) - 1.0) / (tau * tau);
    }
}

/* Optical depth of the cell, tau = dl sum_s n_s sigma_s. */
static double optical_depth(const ko_net *n, const ko_rad *rd, const double *y)
{
    double s = 0.0;
    int i;
    for (i = 0; i < n->ns; i++) s += y[i] * n->sig_s[i];
    return rd->path * s;
}

/* Rate coefficients of one cell at state y and temperature T: modified Arrhenius,
 * tabulated (the cell's reduced tables) and photo-reactions k_r = F sigma_r phi(tau)
 * (Sec. 2.2.1 items 1-3; dk/dT = 0 for the latter). */
static int cell_rates(const ko_net *n, const ko_rad *rd, const double *y, double T, double *k, double *dk)
{
    int r, rc = ko_rates(n, T, k, dk);
    if (rc) return rc;
    if (!n->rtype) return KO_OK;
    double phi = 1.0, dphi = 0.0;
    int have_phi = 0;
    for (r = 0; r < n->nr; r++) {
        if (n->rtype[r] == 1) {
            table_eval(n, rd->ltab, n->tab_of[r], T, &k[r], &dk[r]);
        } else if (n->rtype[r] == 2) {
            if (!have_phi) {
                photo_phi(optical_depth(n, rd, y), &phi, &dphi);
                have_phi = 1;
            }
            k[r] = rd->flux * n->sig_r[r] * phi;
            dk[r] = 0.0;
        }
    }
    return KO_OK;
}

/* Right-hand side (Eq. method-ode-thermochem): each reaction's rate is
 * w_r = k_r * prod(reactant densities); every reactant occurrence loses w_r and
 * every product occurrence gains w_r.  With the energy equation the last unknown is
 * T and dT/dt = -sum_s h_s dn_s/dt / C_V(T). */
static void rhs(const ko_net *n, const double *y, const double *k, const ko_heat *hc, double *f)
{
    int N = n->ns + n->energy, r, j;
    for (j = 0; j < N; j++) f[j] = 0.0;
    for (r = 0; r < n->nr; r++) {
        double w = k[r];
        for (j = 0; j < n->nin[r]; j++) w *= y[n->in[r * KO_MAXSIDE + j]];
        for (j = 0; j < n->nin[r]; j++) f[n->in[r * KO_MAXSIDE + j]] -= w;
        for (j = 0; j < n->nout[r]; j++) f[n->out[r * KO_MAXSIDE + j]] += w;
    }
    if (n->energy) {
        double q = 0.0;
        for (j = 0; j < n->ns; j++) q += n->h[j] * f[j];
        double dcv;
        f[n->ns] = -q / heat_capacity(n, hc, y[n->ns], &dcv);
    }
}

/* Analytic Jacobian (Eq. method-jacobian and the mass-action derivative cases;
 * thermal coupling through dk/dT, with dC_V/dn neglected as the paper does).  With
 * C_V(T) the temperature row's T entry also carries -f_T C_V'(T) / C_V(T). */
static void jacobian(const ko_net *n, const double *y, const double *k, const double *dkdT,
                     const ko_heat *hc, const ko_rad *rd, double *J)
{
    int N = n->ns + n->energy, r, j, l, a;
    for (j = 0; j < N * N; j++) J[j] = 0.0;
    for (r = 0; r < n->nr; r++) {
        const int *in = n->in + r * KO_MAXSIDE, *out = n->out + r * KO_MAXSIDE;
        for (j = 0; j < n->nin[r]; j++) {
            /* d w_r / d y_m for the reactant occurrence j (m = in[j]) */
            double d = k[r];
            for (l = 0; l < n->nin[r]; l++)
                if (l != j) d *= y[in[l]];
            int m = in[j];
            for (a = 0; a < n->nin[r]; a++) J[in[a] * N + m] -= d;
            for (a = 0; a < n->nout[r]; a++) J[out[a] * N + m] += d;
        }
        if (n->energy) {
            double dT = dkdT[r];
            for (l = 0; l < n->nin[r]; l++) dT *= y[in[l]];
            for (a = 0; a < n->nin[r]; a++) J[in[a] * N + n->ns] -= dT;
            for (a = 0; a < n->nout[r]; a++) J[out[a] * N + n->ns] += dT;
        }
        if (n->rtype && n->rtype[r] == 2 && rd->path > 0.0) {
            /* photo rate w = F sigma_r phi(tau) n_i with tau = dl sum_m n_m sigma_m:
             * dw/dn_m also carries F sigma_r n_i phi'(tau) dl sigma_m (every absorber) */
            double phi, dphi;
            photo_phi(optical_depth(n, rd, y), &phi, &dphi);
            double g = rd->flux * n->sig_r[r] * y[in[0]] * dphi * rd->path;
            int m;
            for (m = 0; m < n->ns; m++) {
                double d = g * n->sig_s[m];
                if (d == 0.0) continue;
                J[in[0] * N + m] -= d;
                for (a = 0; a < n->nout[r]; a++) J[out[a] * N + m] += d;
            }
        }
    }
    if (n->energy) {
        int m;
        double dcv, cv = heat_capacity(n, hc, y[n->ns], &dcv);
        for (m = 0; m < N; m++) {
            double q = 0.0;
            for (j = 0; j < n->ns; j++) q += n->h[j] * J[j * N + m];
            J[n->ns * N + m] = -q / cv;
        }
        if (dcv != 0.0) {
            double f[KO_MAXN];
            rhs(n, y, k, hc, f);
            J[n->ns * N + n->ns] -= f[n->ns] * dcv / cv;
        }
    }
}

/* Parameters of one cell for the pins: the isothermal temperature, C_V (constant, or
 * the frozen composition n0 of C_V(T)), the density (rate tables) and the photo flux
 * factor and path length (photo-reactions). */
typedef struct {
    double T_iso, cvtot;
    const double *n0;
    double rho, flux, path;
} ko_cellpar;

static void par_setup(const ko_net *n, const ko_cellpar *p, ko_heat *hc, ko_rad *rd, double *ltab)
{
    hc->cv0 = p->cvtot;
    hc->n0 = p->n0;
    rd->flux = p->flux;
    rd->path = p->path;
    rd->ltab = ltab;
    if (n->ntab) table_reduce(n, p->rho, ltab);
}

/* Rate coefficients, f(y) and J(y) of one state (pins). */
int ko_rates_cell(const ko_net *n, const double *y, const ko_cellpar *p, double *k, double *dk)
{
    double ltab[KO_MAXTAB * KO_MAXTN];
    ko_heat hc;
    ko_rad rd;
    par_setup(n, p, &hc, &rd, ltab);
    return cell_rates(n, &rd, y, n->energy ? y[n->ns] : p->T_iso, k, dk);
}

int ko_rhs(const ko_net *n, const double *y, const ko_cellpar *p, double *f)
{
    double ltab[KO_MAXTAB * KO_MAXTN];
    double k[4096], dk[4096];
    ko_heat hc;
    ko_rad rd;
    if (n->nr > 4096) return KO_EINVAL;
    par_setup(n, p, &hc, &rd, ltab);
    int rc = cell_rates(n, &rd, y, n->energy ? y[n->ns] : p->T_iso, k, dk);
    if (rc) return rc;
    rhs(n, y, k, &hc, f);
    return KO_OK;
}

int ko_jacobian(const ko_net *n, const double *y, const ko_cellpar *p, double *J)
{
    double ltab[KO_MAXTAB * KO_MAXTN];
    double k[4096], dk[4096];
    ko_heat hc;
    ko_rad rd;
    if (n->nr > 4096) return KO_EINVAL;
    par_setup(n, p, &hc, &rd, ltab);
    int rc = cell_rates(n, &rd, y, n->energy ? y[n->ns] : p->T_iso, k, dk);
    if (rc) return rc;
    jacobian(n, y, k, dk, &hc, &rd, J);
    return KO_OK;
}

/* ------------------------------------------------------------------ linear algebra */

/* Crout LU with implicit-scaled partial pivoting (Algorithm lu-decomp; Numerical
 * Recipes' ludcmp, which the paper cites).  v_i is the largest |a_ij| of row i.  For
 * each column j: a_ij -= sum_{k < min(i,j)} a_ik a_kj for every row; the pivot row is
 * argmax_{i >= j} |a_ij| / v_i (ties: smallest i); rows j and i_max are swapped
 * (with their scales) and p_j = i_max; then a_ij /= a_jj for i > j.  Returns -1 on a
 * zero row or a zero pivot. */
int ko_lu(int N, double *a, int *perm)
{
    double v[KO_MAXN];
    int i, j, k;
    for (i = 0; i < N; i++) {
        double big = 0.0;
        for (j = 0; j < N; j++)
            if (fabs(a[i * N + j]) > big) big = fabs(a[i * N + j]);
        if (!(big > 0.0)) return -1;
        v[i] = big;
    }
    for (j = 0; j < N; j++) {
        for (i = 0; i < N; i++) {
            int kmax = i < j ? i : j;
            double s = a[i * N + j];
            for (k = 0; k < kmax; k++) s -= a[i * N + k] * a[k * N + j];
            a[i * N + j] = s;
        }
        int imax = j;
        double tmax = fabs(a[j * N + j]) / v[j];
        for (i = j + 1; i < N; i++) {
            double t = fabs(a[i * N + j]) / v[i];
            if (t > tmax) { tmax = t; imax = i; }
        }
        if (!(tmax > 0.0)) return -1;
        if (imax != j) {
            for (k = 0; k < N; k++) {
                double tmp = a[imax * N + k];
                a[imax * N + k] = a[j * N + k];
                a[j * N + k] = tmp;
            }
            double tv = v[imax]; v[imax] = v[j]; v[j] = tv;
        }
        perm[j] = imax;
        for (i = j + 1; i < N; i++) a[i * N + j] /= a[j * N + j];
    }
    return 0;
}

/* Solve with the factors of ko_lu: apply the row swaps in order, then forward
 * substitution with the unit-diagonal L and back substitution with U. */
void ko_lu_solve(int N, const double *a, const int *perm, double *x)
{
    int i, k;
    for (i = 0; i < N; i++) {
        double t = x[i]; x[i] = x[perm[i]]; x[perm[i]] = t;
    }
    for (i = 0; i < N; i++) {
        double s = x[i];
        for (k = 0; k < i; k++) s -= a[i * N + k] * x[k];
        x[i] = s;
    }
    for (i = N - 1; i >= 0; i--) {
        double s = x[i];
        for (k = i + 1; k < N; k++) s -= a[i * N + k] * x[k];
        x[i] = s / a[i * N + i];
    }
}

/* ------------------------------------------------------------------ integrator */

typedef struct {
    const ko_net *n;
    const ko_options *o;
    int N;
    double T_iso, cvtot;
    double n0[KO_MAXN];       /* pre-processed composition (C_V(T) of polynomial networks) */
    ko_heat hc;
    ko_rad rd;                /* photo flux factor and path length, reduced rate tables */
    double ltab[KO_MAXTAB * KO_MAXTN];
    double atol_s;            /* species absolute tolerance for this cell */
    double k[4096], dk[4096];
    double f[KO_MAXN], G[KO_MAXN], d[KO_MAXN];
    double M[KO_MAXN * KO_MAXN], J[KO_MAXN * KO_MAXN];
    int perm[KO_MAXN];
    long nnewton;
} ko_cell;

static double natol(const ko_cell *c, int i)
{
    return i < c->n->ns ? c->o->newton_atol_frac * c->atol_s : 0.0;
}

static double eatol(const ko_cell *c, int i)
{
    return i < c->n->ns ? c->atol_s : 0.0;
}

/* One backward-Euler step y = yn + h f(y), solved by full Newton from the guess in y:
 * M = I - h J(y), M delta = -(y - yn - h f(y)), y += delta, until every
 * |delta_i| <= natol_i + newton_rtol |y_i|.  Returns 0 on convergence.  The TR-BDF2
 * stages are equations of the same form, y = r + c f(y), with r and c given below. */
static int be_solve(ko_cell *c, const double *yn, double h, double *y)
{
    const ko_net *n = c->n;
    int N = c->N, it, i, j;
    for (it = 0; it < c->o->max_newton; it++) {
        c->nnewton++;
        double T = n->energy ? y[n->ns] : c->T_iso;
        if (!(T > 0.0)) return -1;
        cell_rates(n, &c->rd, y, T, c->k, c->dk);
        rhs(n, y, c->k, &c->hc, c->f);
        for (i = 0; i < N; i++) c->G[i] = y[i] - yn[i] - h * c->f[i];
        jacobian(n, y, c->k, c->dk, &c->hc, &c->rd, c->J);
        for (i = 0; i < N; i++)
            for (j = 0; j < N; j++)
                c->M[i * N + j] = (i == j ? 1.0 : 0.0) - h * c->J[i * N + j];
        if (ko_lu(N, c->M, c->perm)) return -1;
        for (i = 0; i < N; i++) c->d[i] = -c->G[i];
        ko_lu_solve(N, c->M, c->perm, c->d);
        int conv = 1;
        for (i = 0; i < N; i++) {
            y[i] += c->d[i];
            double tol = natol(c, i) + c->o->newton_rtol * fabs(y[i]);
            if (!(fabs(c->d[i]) <= tol)) conv = 0;
        }
        if (conv) return 0;
    }
    return -1;
}

/* Weighted RMS of the step-doubling difference, weights atol_i + rtol max(|y_i|,|y2_i|). */
static double err_norm(const ko_cell *c, const double *y, const double *y2, const double *yf)
{
    double s = 0.0;
    int i;
    for (i = 0; i < c->N; i++) {
        double sc = eatol(c, i) + c->o->rtol * fmax(fabs(y[i]), fabs(y2[i]));
        double e = (y2[i] - yf[i]) / sc;
        s += e * e;
    }
    return sqrt(s / c->N);
}

#define ADV_OK 0
#define ADV_FAIL 1

/* TR-BDF2 (Bank et al. 1985), the one-step scheme with one iteration matrix per step:
 * a trapezoidal stage to t + gamma h, then a BDF2 stage to t + h, gamma = 2 - sqrt(2).
 * Both stages are y = r + d h f(y) with d = gamma / 2:
 *   stage 1: r1 = y_n + d h f(y_n)                      -> y_g
 *   stage 2: r2 = w1 y_g - w0 y_n,  w1 = 1/(gamma(2-gamma)), w0 = (1-gamma)^2/(gamma(2-gamma))
 *                                                       -> y_{n+1}
 * The local error y(t+h) - y_{n+1} = C h^3 y''' + O(h^4), C = (-3 gamma^2 + 4 gamma - 2) /
 * (12 (2 - gamma)), is estimated from the quadratic through f at t, t + gamma h, t + h:
 *   est = 2 C h (f_n / gamma - f_g / (gamma (1 - gamma)) + f_{n+1} / (1 - gamma)),
 * where f_g and f_{n+1} follow from the stage equations (f_g = (y_g - y_n)/(d h) - f_n,
 * f_{n+1} = (y_{n+1} - r2)/(d h)).  Accept when the weighted RMS of est is <= 1; the next
 * step is h * min(facmax, max(0.2, 0.9 err^(-1/3))).  (Hosea and Shampine 1996 analyse
 * this pair; their stiff filter of the estimate is not applied.)
 * f_n is f(y_n) evaluated only on a cell's first step; after an accepted step it is the
 * stage relation's f_{n+1} of that step ("first same as last").  An evaluated f(y_n)
 * enters est with the factor ~0.47 h, and for a component with rate constant k its
 * rounding (a sum of large, nearly cancelling rates) is amplified by h k, which reaches
 * 1e10 on stiff networks: the decision err <= 1 would then follow rounding noise.  The
 * stage relation carries no such amplification (its error is the Newton tolerance). */
typedef struct {
    double g, d, w1, w0, C, a0, a1, a2;
} trbdf2_coef;

static trbdf2_coef trbdf2_coefficients(void)
{
    trbdf2_coef k;
    k.g = 2.0 - sqrt(2.0);
    k.d = 0.5 * k.g;
    k.w1 = 1.0 / (k.g * (2.0 - k.g));
    k.w0 = (1.0 - k.g) * (1.0 - k.g) / (k.g * (2.0 - k.g));
    k.C = (-3.0 * k.g * k.g + 4.0 * k.g - 2.0) / (12.0 * (2.0 - k.g));
    k.a0 = 1.0 / k.g;
    k.a1 = -1.0 / (k.g * (1.0 - k.g));
    k.a2 = 1.0 / (1.0 - k.g);
    return k;
}

/* One TR-BDF2 step of size h from yn with f0 = f_n: y1 receives y_{n+1}, est the local
 * error estimate and f1 the stage relation's f_{n+1}.  Returns 0, or -1 when a stage's
 * Newton iteration fails. */
static int trbdf2_step(ko_cell *c, const double *yn, const double *f0, double h, double *y1, double *est,
                       double *f1)
{
    const trbdf2_coef k = trbdf2_coefficients();
    int N = c->N, i;
    double r[KO_MAXN], yg[KO_MAXN];
    const double dh = k.d * h, inv = 1.0 / dh;
    for (i = 0; i < N; i++) r[i] = yn[i] + dh * f0[i];
    for (i = 0; i < N; i++) yg[i] = yn[i];
    if (be_solve(c, r, dh, yg)) return -1;
    for (i = 0; i < N; i++) r[i] = k.w1 * yg[i] - k.w0 * yn[i];
    for (i = 0; i < N; i++) y1[i] = yg[i];
    if (be_solve(c, r, dh, y1)) return -1;
    const double ce = 2.0 * k.C * h;
    for (i = 0; i < N; i++) {
        double fg = (yg[i] - yn[i]) * inv - f0[i];
        f1[i] = (y1[i] - r[i]) * inv;
        est[i] = ce * (k.a0 * f0[i] + k.a1 * fg + k.a2 * f1[i]);
    }
    return 0;
}

/* f(y) of the cell (rates at y's temperature); -1 for a non-positive temperature. */
static int cell_rhs(ko_cell *c, const double *y, double *f)
{
    const ko_net *n = c->n;
    double T = n->energy ? y[n->ns] : c->T_iso;
    if (!(T > 0.0)) return -1;
    cell_rates(n, &c->rd, y, T, c->k, c->dk);
    rhs(n, y, c->k, &c->hc, f);
    return 0;
}

/* Weighted RMS of the TR-BDF2 estimate, weights atol_i + rtol max(|y_n,i|, |y_{n+1},i|). */
static double est_norm(const ko_cell *c, const double *yn, const double *y1, const double *est)
{
    double s = 0.0;
    int i;
    for (i = 0; i < c->N; i++) {
        double sc = eatol(c, i) + c->o->rtol * fmax(fabs(yn[i]), fabs(y1[i]));
        double e = est[i] / sc;
        s += e * e;
    }
    return sqrt(s / c->N);
}

static int advance_trbdf2(ko_cell *c, double *y, double dt, double h0, double facmax, int *nsub)
{
    const ko_options *o = c->o;
    int N = c->N, i;
    double y1[KO_MAXN], est[KO_MAXN], f0[KO_MAXN], f1[KO_MAXN];
    double t = 0.0, h = h0;
    int nacc = 0, natt = 0, f0ok = 0;
    for (;;) {
        if (natt >= o->max_substeps) return ADV_FAIL;
        natt++;
        int last = 0;
        if (t + h >= dt * (1.0 - 1e-12)) { h = dt - t; last = 1; }
        if (!f0ok) {
            if (cell_rhs(c, y, f0)) {
                h *= 0.5;
                if (h < o->h_min) return ADV_FAIL;
                continue;
            }
            f0ok = 1;
        }
        if (trbdf2_step(c, y, f0, h, y1, est, f1)) {
            h *= 0.5;
            if (h < o->h_min) return ADV_FAIL;
            continue;
        }
        double err = o->adaptive ? est_norm(c, y, y1, est) : 0.0;
        if (err <= 1.0) {
            for (i = 0; i < N; i++) {
                y[i] = y1[i];
                f0[i] = f1[i];          /* first same as last */
            }
            nacc++;
            if (last) break;
            t += h;
            if (!o->adaptive) continue;
            double fac = err > 0.0 ? 0.9 / cbrt(err) : facmax;
            if (fac > facmax) fac = facmax;
            if (fac < 0.2) fac = 0.2;
            h *= fac;
        } else {
            double fac = 0.9 / cbrt(err);   /* NaN err falls through to the 0.2 clamp */
            if (!(fac >= 0.2)) fac = 0.2;
            h *= fac;
            if (h < o->h_min) return ADV_FAIL;
        }
    }
    *nsub = nacc;
    return ADV_OK;
}

/* Advance y over [0, dt] with adaptive sub-steps (or fixed steps when adaptive=0). */
static int advance(ko_cell *c, double *y, double dt, double h0, double facmax, int *nsub)
{
    const ko_options *o = c->o;
    int N = c->N, i;
    double yf[KO_MAXN], yh[KO_MAXN], y2[KO_MAXN];
    double t = 0.0, h = h0;
    int nacc = 0, natt = 0;
    if (o->scheme == 1) return advance_trbdf2(c, y, dt, h0, facmax, nsub);
    for (;;) {
        if (natt >= o->max_substeps) return ADV_FAIL;
        natt++;
        int last = 0;
        if (t + h >= dt * (1.0 - 1e-12)) { h = dt - t; last = 1; }
        if (!o->adaptive) {
            for (i = 0; i < N; i++) yf[i] = y[i];
            if (be_solve(c, y, h, yf)) return ADV_FAIL;
            for (i = 0; i < N; i++) y[i] = yf[i];
            nacc++;
            if (last) break;
            t += h;
            continue;
        }
        for (i = 0; i < N; i++) yf[i] = y[i];
        int ok = be_solve(c, y, h, yf) == 0;
        if (ok) {
            for (i = 0; i < N; i++) yh[i] = y[i];
            ok = be_solve(c, y, 0.5 * h, yh) == 0;
        }
        if (ok) {
            for (i = 0; i < N; i++) y2[i] = o->guess == 2 ? yf[i] : yh[i];
            ok = be_solve(c, yh, 0.5 * h, y2) == 0;
        }
        if (!ok) {
            h *= 0.5;
            if (h < o->h_min) return ADV_FAIL;
            continue;
        }
        double err = err_norm(c, y, y2, yf);
        if (err <= 1.0) {
            for (i = 0; i < N; i++) y[i] = y2[i];
            nacc++;
            if (last) break;
            t += h;
            double fac = err > 0.0 ? 0.9 / sqrt(err) : facmax;
            if (fac > facmax) fac = facmax;
            if (fac < 0.2) fac = 0.2;
            h *= fac;
        } else {
            double fac = 0.9 / sqrt(err);   /* NaN err falls through to the 0.2 clamp */
            if (!(fac >= 0.2)) fac = 0.2;
            h *= fac;
            if (h < o->h_min) return ADV_FAIL;
        }
    }
    *nsub = nacc;
    return ADV_OK;
}

/* Small dense solve for the projection (Gaussian elimination, partial pivoting). */
static int small_solve(int m, double *A, double *x)
{
    int i, j, k;
    for (k = 0; k < m; k++) {
        int p = k;
        for (i = k + 1; i < m; i++)
            if (fabs(A[i * m + k]) > fabs(A[p * m + k])) p = i;
        if (!(fabs(A[p * m + k]) > 0.0)) return -1;
        if (p != k) {
            for (j = 0; j < m; j++) { double t = A[k * m + j]; A[k * m + j] = A[p * m + j]; A[p * m + j] = t; }
            double t = x[k]; x[k] = x[p]; x[p] = t;
        }
        for (i = k + 1; i < m; i++) {
            double l = A[i * m + k] / A[k * m + k];
            for (j = k; j < m; j++) A[i * m + j] -= l * A[k * m + j];
            x[i] -= l * x[k];
        }
    }
    for (i = m - 1; i >= 0; i--) {
        double s = x[i];
        for (j = i + 1; j < m; j++) s -= A[i * m + j] * x[j];
        x[i] = s / A[i * m + i];
    }
    return 0;
}

/* Post-processing (Sec. 2.2.3): stage 1 clips negative abundances; the element
 * totals b0 of the initial state are then restored by y_s -= y_s (N^T lambda)_s with
 * (N diag(y) N^T) lambda = N y - b0.  An element with no abundance left must have a
 * zero defect; a relative correction >= 1 (it would empty a species) is a
 * conservation failure. */
static int post_process(const ko_cell *c, double *y, const double *b0)
{
    const ko_net *n = c->n;
    int ns = n->ns, ne = n->ne, s, e, f;
    double M[KO_MAXE * KO_MAXE], r[KO_MAXE];
    for (s = 0; s < ns; s++)
        if (y[s] < 0.0) y[s] = 0.0;
    for (e = 0; e < ne; e++) {
        double tot = 0.0;
        for (s = 0; s < ns; s++) tot += n->counts[s * ne + e] * y[s];
        r[e] = tot - b0[e];
        for (f = 0; f < ne; f++) {
            double m = 0.0;
            for (s = 0; s < ns; s++) m += (double)n->counts[s * ne + e] * n->counts[s * ne + f] * y[s];
            M[e * ne + f] = m;
        }
    }
    for (e = 0; e < ne; e++) {
        if (M[e * ne + e] == 0.0) {
            if (r[e] != 0.0) return -1;
            for (f = 0; f < ne; f++) M[e * ne + f] = M[f * ne + e] = 0.0;
            M[e * ne + e] = 1.0;
        }
    }
    if (small_solve(ne, M, r)) return -1;
    for (s = 0; s < ns; s++) {
        double corr = 0.0;
        for (e = 0; e < ne; e++) corr += n->counts[s * ne + e] * r[e];
        if (!(corr < 1.0)) return -1;
        y[s] -= y[s] * corr;
    }
    for (s = 0; s < c->N; s++)
        if (!isfinite(y[s])) return -1;
    return 0;
}

/* One cell: pre-process, integrate, post-process, retry / revert (Sec. 2.2.2-2.2.3). */
static void integrate_cell(const ko_net *n, const ko_options *o, double dt,
                           const double *yin, double Tin, double rho, double flux, double path,
                           double *yout, double *Tout,
                           int32_t *status, int32_t *nsub, int32_t *nnew, ko_cell *c)
{
    int ns = n->ns, N = ns + n->energy, s, e;
    double y0[KO_MAXN], y[KO_MAXN], b0[KO_MAXE];
    int finite = isfinite(Tin);
    for (s = 0; s < ns; s++) finite = finite && isfinite(yin[s]);
    c->n = n; c->o = o; c->N = N; c->nnewton = 0;
    /* pre-processing (Sec. 2.2.2): the cell's rate tables at its density */
    c->rd.flux = flux;
    c->rd.path = path;
    c->rd.ltab = c->ltab;
    if (n->ntab) table_reduce(n, rho, c->ltab);
    if (!finite) {
        for (s = 0; s < ns; s++) yout[s] = yin[s];
        *Tout = Tin; *status = KO_ST_NONFINITE; *nsub = 0; *nnew = 0;
        return;
    }
    /* pre-processing: floors and temperature limits */
    for (s = 0; s < ns; s++) y0[s] = yin[s] > 0.0 ? yin[s] : 0.0;
    double T0 = Tin < n->t_min ? n->t_min : (Tin > n->t_max ? n->t_max : Tin);
    if (n->energy) y0[ns] = T0;
    c->T_iso = T0;
    for (e = 0; e < n->ne; e++) {
        double t = 0.0;
        for (s = 0; s < ns; s++) t += n->counts[s * n->ne + e] * y0[s];
        b0[e] = t;
    }
    c->cvtot = 0.0;
    for (s = 0; s < ns; s++) c->cvtot += n->cv[s] * y0[s];
    for (s = 0; s < ns; s++) c->n0[s] = y0[s];
    c->hc.cv0 = c->cvtot;
    c->hc.n0 = c->n0;
    c->atol_s = o->atol;
    if (o->atol_mode == 1 && b0[0] > 0.0) c->atol_s = o->atol * b0[0];

    int st = KO_ST_OK, ns_ok = 0;
    for (s = 0; s < N; s++) y[s] = y0[s];
    int rc = advance(c, y, dt, o->h_init, o->facmax, &ns_ok);
    if (rc == ADV_OK) rc = post_process(c, y, b0) ? ADV_FAIL : ADV_OK;
    if (rc != ADV_OK && o->retry) {
        for (s = 0; s < N; s++) y[s] = y0[s];
        rc = advance(c, y, dt, o->h_init * o->retry_h_factor, o->retry_facmax, &ns_ok);
        if (rc == ADV_OK) rc = post_process(c, y, b0) ? ADV_FAIL : ADV_OK;
        st = KO_ST_RETRIED;
    }
    if (rc != ADV_OK) {
        for (s = 0; s < N; s++) y[s] = y0[s];
        st = KO_ST_REVERTED;
        ns_ok = 0;
    }
    for (s = 0; s < ns; s++) yout[s] = y[s];
    *Tout = n->energy ? y[ns] : T0;
    *status = st;
    *nsub = ns_ok;
    *nnew = c->nnewton > 2147483647L ? 2147483647 : (int32_t)c->nnewton;
}

typedef struct {
    const ko_net *n;
    const ko_options *o;
    double dt;
    int64_t ncells;
    const double *y, *T, *rho, *flux, *path;
    double *yo, *To;
    int32_t *st, *nsub, *nnew;
    int64_t next;
    pthread_mutex_t lock;
} ko_job;

static void *worker(void *arg)
{
    ko_job *jb = arg;
    ko_cell *c = malloc(sizeof *c);
    double yin[KO_MAXN], yout[KO_MAXN];
    int ns = jb->n->ns, s;
    if (!c) return NULL;
    for (;;) {
        pthread_mutex_lock(&jb->lock);
        int64_t i = jb->next++;
        pthread_mutex_unlock(&jb->lock);
        if (i >= jb->ncells) break;
        for (s = 0; s < ns; s++) yin[s] = jb->y[(int64_t)s * jb->ncells + i];
        double To;
        integrate_cell(jb->n, jb->o, jb->dt, yin, jb->T[i], jb->rho ? jb->rho[i] : 1.0,
                       jb->flux ? jb->flux[i] : 1.0, jb->path ? jb->path[i] : 0.0, yout, &To,
                       &jb->st[i], &jb->nsub[i], &jb->nnew[i], c);
        for (s = 0; s < ns; s++) jb->yo[(int64_t)s * jb->ncells + i] = yout[s];
        jb->To[i] = To;
    }
    free(c);
    return NULL;
}

/* Integrate ncells cells over dt.  y, y_out: [ns][ncells] SoA; T, T_out: [ncells].
 * rho (rate tables; NULL: 1), flux and path (photo-reactions, Eq. photo-reaction-single;
 * NULL: F = 1 and dl = 0, the optically thin limit k = sigma) are per cell.
 * nthreads <= 0 means 1. */
int ko_integrate_rad(const ko_net *n, int64_t ncells, const double *y, const double *T,
                     const double *rho, const double *flux, const double *path, double dt,
                     const ko_options *o, int nthreads, double *y_out, double *T_out,
                     int32_t *status, int32_t *nsub, int32_t *nnew)
{
    if (!n || !o || ncells < 0 || !(dt > 0.0) || !(o->atol > 0.0) || !(o->rtol > 0.0) ||
        o->max_newton < 1 || o->max_substeps < 1 || !(o->h_init > 0.0))
        return KO_EINVAL;
    if (ncells == 0) return KO_OK;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 512) nthreads = 512;
    ko_job jb = {n, o, dt, ncells, y, T, rho, flux, path, y_out, T_out, status, nsub, nnew, 0,
                 PTHREAD_MUTEX_INITIALIZER};
    pthread_t th[512];
    int t, started = 0;
    for (t = 1; t < nthreads; t++)
        if (pthread_create(&th[t], NULL, worker, &jb) == 0) started = t;
        else break;
    worker(&jb);
    for (t = 1; t <= started; t++) pthread_join(th[t], NULL);
    return KO_OK;
}

int ko_integrate(const ko_net *n, int64_t ncells, const double *y, const double *T,
                 const double *rho, double dt, const ko_options *o, int nthreads,
                 double *y_out, double *T_out, int32_t *status, int32_t *nsub, int32_t *nnew)
{
    return ko_integrate_rad(n, ncells, y, T, rho, NULL, NULL, dt, o, nthreads, y_out, T_out, status,
                            nsub, nnew);
}

/* One backward-Euler step of one cell (pins): y_out = root of y - yn - h f(y). */
int ko_be_step(const ko_net *n, const ko_options *o, const double *yn, double T_iso,
               double cvtot, double h, double *y_out, int *n_iter)
{
    ko_cell *c = malloc(sizeof *c);
    int i, rc;
    if (!c) return KO_ENOMEM;
    c->n = n; c->o = o; c->N = n->ns + n->energy; c->T_iso = T_iso; c->cvtot = cvtot;
    c->hc.cv0 = cvtot; c->hc.n0 = NULL;
    c->rd.flux = 1.0; c->rd.path = 0.0; c->rd.ltab = c->ltab;
    if (n->ntab) table_reduce(n, 1.0, c->ltab);
    c->atol_s = o->atol; c->nnewton = 0;
    for (i = 0; i < c->N; i++) y_out[i] = yn[i];
    rc = be_solve(c, yn, h, y_out);
    *n_iter = (int)c->nnewton;
    free(c);
    return rc;
}

/* Post-processing of one state (pins, Sec. 2.2.3): y[0..ns) is clipped and corrected
 * in place towards the element totals b0[0..ne); returns 0, or -1 when the correction
 * fails (a relative correction >= 1, an element with no abundance left but a nonzero
 * defect, or a non-finite result).  y must hold ns + energy entries. */
int ko_post_process(const ko_net *n, double *y, const double *b0)
{
    ko_cell *c = malloc(sizeof *c);
    int rc;
    if (!c) return KO_ENOMEM;
    c->n = n; c->o = NULL; c->N = n->ns + n->energy; c->nnewton = 0;
    rc = post_process(c, y, b0);
    free(c);
    return rc;
}

/* One TR-BDF2 step of one cell (pins): y_out = y_{n+1}, est_out = the local error
 * estimate.  Returns 0, or -1 when a stage's Newton iteration fails. */
int ko_trbdf2_step(const ko_net *n, const ko_options *o, const double *yn, double T_iso,
                   double cvtot, double h, double *y_out, double *est_out)
{
    ko_cell *c = malloc(sizeof *c);
    int rc;
    if (!c) return KO_ENOMEM;
    c->n = n; c->o = o; c->N = n->ns + n->energy; c->T_iso = T_iso; c->cvtot = cvtot;
    c->hc.cv0 = cvtot; c->hc.n0 = NULL;
    c->rd.flux = 1.0; c->rd.path = 0.0; c->rd.ltab = c->ltab;
    if (n->ntab) table_reduce(n, 1.0, c->ltab);
    c->atol_s = o->atol; c->nnewton = 0;
    double f0[KO_MAXN], f1[KO_MAXN];
    rc = cell_rhs(c, yn, f0);
    if (!rc) rc = trbdf2_step(c, yn, f0, h, y_out, est_out, f1);
    free(c);
    return rc;
}
