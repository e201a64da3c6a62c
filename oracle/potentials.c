/*
 * Oracle: brute-force FP64 interatomic energy, force and virial.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load it.  It shares no code
 * with the CUDA library.
 *
 * Conventions (paper Sec. II.B):
 *   - lattice matrix h has the lattice vectors h1, h2, h3 as ROWS; a
 *     Cartesian position is the row vector R = s h (s fractional);
 *   - r^{ij} = r^j - r^i (the vector from i to j);
 *   - U = sum_i U_i, U_i a function of the r^{ij} of i's neighbours (Eq. U);
 *   - force on i due to j: f^{ij} = dU_i/dr^{ij} - dU_j/dr^{ji}, taken from
 *     the derivation of Eq. V2 (the one-line definition printed before it has
 *     U_i and U_j swapped; the derivation fixes the meaning);
 *   - F_i = sum_j f^{ij};
 *   - virial V = -1/2 sum_{ij} r^{ij} (x) f^{ij}, i.e. V_mn = -1/2 sum r_m f_n.
 *
 * Neighbours: every atom j (including i itself) and every periodic shift
 * t in Z^3 with |r^j + t h - r^i| < rc, except (j == i, t == 0).  No minimum
 * image convention: when rc exceeds half a cell width one atom appears under
 * several shifts and every such image is a separate neighbour.  The integer
 * range of t along axis a is bounded exactly: the fractional component of a
 * vector d along a is d . g_a with |g_a| = 1/w_a (w_a = perpendicular cell
 * width), so |ds_a + t_a| < rc / w_a is necessary for |d| < rc.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------- 3x3 helpers (row-major, h[3*a + b] = component b of h_a) ---- */

static double det3(const double *m)
{
    return m[0] * (m[4] * m[8] - m[5] * m[7]) -
           m[1] * (m[3] * m[8] - m[5] * m[6]) +
           m[2] * (m[3] * m[7] - m[4] * m[6]);
}

static void inv3(const double *m, double *out)
{
    double d = det3(m);
    out[0] = (m[4] * m[8] - m[5] * m[7]) / d;
    out[1] = (m[2] * m[7] - m[1] * m[8]) / d;
    out[2] = (m[1] * m[5] - m[2] * m[4]) / d;
    out[3] = (m[5] * m[6] - m[3] * m[8]) / d;
    out[4] = (m[0] * m[8] - m[2] * m[6]) / d;
    out[5] = (m[2] * m[3] - m[0] * m[5]) / d;
    out[6] = (m[3] * m[7] - m[4] * m[6]) / d;
    out[7] = (m[1] * m[6] - m[0] * m[7]) / d;
    out[8] = (m[0] * m[4] - m[1] * m[3]) / d;
}

/* perpendicular width of the cell along each lattice direction:
 * w_a = volume / |h_b x h_c| */
static void perp_widths(const double *h, double *w)
{
    double vol = fabs(det3(h));
    for (int a = 0; a < 3; ++a) {
        const double *u = h + 3 * ((a + 1) % 3);
        const double *v = h + 3 * ((a + 2) % 3);
        double cx = u[1] * v[2] - u[2] * v[1];
        double cy = u[2] * v[0] - u[0] * v[2];
        double cz = u[0] * v[1] - u[1] * v[0];
        w[a] = vol / sqrt(cx * cx + cy * cy + cz * cz);
    }
}

/* ---------- neighbour enumeration ------------------------------------- */

typedef struct {
    int j;          /* neighbour atom index                               */
    int t[3];       /* periodic shift                                     */
    double r[3];    /* r^{ij} = r^j + t h - r^i                           */
    double d;       /* |r^{ij}|                                           */
} nbr_t;

/* Collect every (j, t) within rc of atom i.  Returns the count; *out is
 * realloc'ed as needed and owned by the caller. */
static int neighbours_of(int i, int n, const double *R, const double *h,
                         const double *hinv, const double *w, double rc,
                         nbr_t **out, int *cap)
{
    int cnt = 0;
    for (int j = 0; j < n; ++j) {
        double d0[3];
        for (int c = 0; c < 3; ++c) d0[c] = R[3 * j + c] - R[3 * i + c];
        double ds[3];
        for (int a = 0; a < 3; ++a)
            ds[a] = d0[0] * hinv[0 * 3 + a] + d0[1] * hinv[1 * 3 + a] +
                    d0[2] * hinv[2 * 3 + a];
        int lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            double lim = rc / w[a];
            lo[a] = (int)ceil(-lim - ds[a]);
            hi[a] = (int)floor(lim - ds[a]);
        }
        for (int t0 = lo[0]; t0 <= hi[0]; ++t0)
            for (int t1 = lo[1]; t1 <= hi[1]; ++t1)
                for (int t2 = lo[2]; t2 <= hi[2]; ++t2) {
                    if (j == i && t0 == 0 && t1 == 0 && t2 == 0) continue;
                    double r[3];
                    for (int c = 0; c < 3; ++c)
                        r[c] = d0[c] + t0 * h[0 * 3 + c] + t1 * h[1 * 3 + c] +
                               t2 * h[2 * 3 + c];
                    double d2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                    if (d2 >= rc * rc) continue;
                    if (cnt == *cap) {
                        *cap = *cap ? 2 * *cap : 64;
                        *out = (nbr_t *)realloc(*out, sizeof(nbr_t) * (size_t)*cap);
                    }
                    nbr_t *e = &(*out)[cnt++];
                    e->j = j;
                    e->t[0] = t0; e->t[1] = t1; e->t[2] = t2;
                    e->r[0] = r[0]; e->r[1] = r[1]; e->r[2] = r[2];
                    e->d = sqrt(d2);
                }
    }
    return cnt;
}

/* ---------- Lennard-Jones --------------------------------------------- */

/* phi(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6], minus phi(rc) when shift != 0.
 * U_i = 1/2 sum_j phi(r_ij).  For this pair form dU_i/dr^{ij} =
 * 1/2 phi'(r) r^{ij}/r and dU_j/dr^{ji} = -1/2 phi'(r) r^{ij}/r, so
 * f^{ij} = phi'(r) r^{ij} / r. */
static double lj_phi(double r, double eps, double sigma)
{
    double sr6 = pow(sigma / r, 6.0);
    return 4.0 * eps * (sr6 * sr6 - sr6);
}

static double lj_dphi(double r, double eps, double sigma)
{
    double sr6 = pow(sigma / r, 6.0);
    return 4.0 * eps * (-12.0 * sr6 * sr6 + 6.0 * sr6) / r;
}

/* Energy per atom e_atom[n], forces F[n*3], virial V[9] (row-major V_mn). */
int oracle_lj(int n, const double *R, const double *h, double eps, double sigma,
              double rc, int shift, double *e_atom, double *F, double *V)
{
    double hinv[9], w[3];
    inv3(h, hinv);
    perp_widths(h, w);
    double phic = shift ? lj_phi(rc, eps, sigma) : 0.0;
    nbr_t *nb = NULL;
    int cap = 0;
    memset(V, 0, 9 * sizeof(double));
    for (int i = 0; i < n; ++i) {
        int cnt = neighbours_of(i, n, R, h, hinv, w, rc, &nb, &cap);
        double ei = 0.0, fi[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < cnt; ++k) {
            double r = nb[k].d;
            ei += 0.5 * (lj_phi(r, eps, sigma) - phic);
            double dphi = lj_dphi(r, eps, sigma);
            double f[3];
            for (int c = 0; c < 3; ++c) {
                f[c] = dphi * nb[k].r[c] / r;  /* f^{ij} */
                fi[c] += f[c];
            }
            for (int m = 0; m < 3; ++m)
                for (int q = 0; q < 3; ++q)
                    V[3 * m + q] += -0.5 * nb[k].r[m] * f[q];
        }
        e_atom[i] = ei;
        for (int c = 0; c < 3; ++c) F[3 * i + c] = fi[c];
    }
    free(nb);
    return 0;
}

/* ---------- Tersoff (1988 form) -------------------------------------- */

typedef struct {
    double A, B, lambda1, lambda2, beta, n, c, d, h, R, D;
} tersoff_params;

/* cutoff f_C: 1 below R-D, 1/2 - 1/2 sin(pi/2 (r-R)/D) inside, 0 above */
static double ters_fc(const tersoff_params *p, double r)
{
    if (r < p->R - p->D) return 1.0;
    if (r > p->R + p->D) return 0.0;
    return 0.5 - 0.5 * sin(0.5 * M_PI * (r - p->R) / p->D);
}

static double ters_dfc(const tersoff_params *p, double r)
{
    if (r < p->R - p->D || r > p->R + p->D) return 0.0;
    return -0.25 * M_PI / p->D * cos(0.5 * M_PI * (r - p->R) / p->D);
}

/* angular term g(theta) = 1 + c^2/d^2 - c^2 / (d^2 + (h - cos theta)^2),
 * written exactly as Tersoff publishes it; dg/dcos theta. */
static double ters_g(const tersoff_params *p, double cs)
{
    double c2 = p->c * p->c, d2 = p->d * p->d, u = p->h - cs;
    return 1.0 + c2 / d2 - c2 / (d2 + u * u);
}

static double ters_dg(const tersoff_params *p, double cs)
{
    double c2 = p->c * p->c, d2 = p->d * p->d, u = p->h - cs;
    double den = d2 + u * u;
    return -2.0 * c2 * u / (den * den);
}

/* b = (1 + beta^n zeta^n)^(-1/2n) and db/dzeta (0 when zeta == 0) */
static void ters_b(const tersoff_params *p, double zeta, double *b, double *db)
{
    if (zeta <= 0.0) { *b = 1.0; *db = 0.0; return; }
    double x = pow(p->beta * zeta, p->n);
    *b = pow(1.0 + x, -1.0 / (2.0 * p->n));
    *db = -0.5 / p->n * pow(1.0 + x, -1.0 / (2.0 * p->n) - 1.0) * p->n * x / zeta;
}

/* cos(angle between vectors a and b) and d cos / d a */
static double cos_and_grad(const double *a, double la, const double *b, double lb,
                           double *grad)
{
    double cs = (a[0] * b[0] + a[1] * b[1] + a[2] * b[2]) / (la * lb);
    for (int c = 0; c < 3; ++c) grad[c] = b[c] / (la * lb) - cs * a[c] / (la * la);
    return cs;
}

/* Site energy U_i and its partials P[k] = dU_i/dr^{i,nb_k} for every
 * neighbour entry k of atom i.
 *   U_i = 1/2 sum_j fC(r_ij) [A e^{-l1 r_ij} - b_ij B e^{-l2 r_ij}]
 *   zeta_ij = sum_{k != j} fC(r_ik) g(cos theta_ijk)   (lambda3 = 0) */
static double ters_site(const tersoff_params *p, const nbr_t *nb, int cnt, double *P)
{
    double U = 0.0;
    for (int q = 0; q < 3 * cnt; ++q) P[q] = 0.0;
    for (int j = 0; j < cnt; ++j) {
        double rij = nb[j].d;
        double fc = ters_fc(p, rij), dfc = ters_dfc(p, rij);
        double fr = p->A * exp(-p->lambda1 * rij);
        double dfr = -p->lambda1 * fr;
        double fa = -p->B * exp(-p->lambda2 * rij);
        double dfa = -p->lambda2 * fa;
        double zeta = 0.0;
        for (int k = 0; k < cnt; ++k) {
            if (k == j) continue;
            double g_[3];
            double cs = cos_and_grad(nb[j].r, rij, nb[k].r, nb[k].d, g_);
            zeta += ters_fc(p, nb[k].d) * ters_g(p, cs);
        }
        double b, db;
        ters_b(p, zeta, &b, &db);
        U += 0.5 * fc * (fr + b * fa);
        /* radial part through r_ij itself */
        double radial = 0.5 * (dfc * (fr + b * fa) + fc * (dfr + b * dfa));
        for (int c = 0; c < 3; ++c) P[3 * j + c] += radial * nb[j].r[c] / rij;
        /* through b_ij: d zeta_ij / d r^{ij} and d zeta_ij / d r^{ik} */
        double pref = 0.5 * fc * fa * db;
        if (pref == 0.0) continue;
        for (int k = 0; k < cnt; ++k) {
            if (k == j) continue;
            double rik = nb[k].d;
            double gj[3], gk[3];
            double cs = cos_and_grad(nb[j].r, rij, nb[k].r, rik, gj);
            cos_and_grad(nb[k].r, rik, nb[j].r, rij, gk);
            double fck = ters_fc(p, rik), dfck = ters_dfc(p, rik);
            double gval = ters_g(p, cs), dg = ters_dg(p, cs);
            for (int c = 0; c < 3; ++c) {
                P[3 * j + c] += pref * fck * dg * gj[c];
                P[3 * k + c] += pref * (dfck * gval * nb[k].r[c] / rik + fck * dg * gk[c]);
            }
        }
    }
    return U;
}

/* Full-system Tersoff: e_atom[n], F[n*3], V[9]. */
int oracle_tersoff(int n, const double *R, const double *h, const double *par,
                   double *e_atom, double *F, double *V)
{
    tersoff_params p;
    memcpy(&p, par, sizeof(p));
    double hinv[9], w[3];
    inv3(h, hinv);
    perp_widths(h, w);
    double rc = p.R + p.D;
    /* per-site neighbour lists and partials */
    nbr_t **nbl = (nbr_t **)calloc((size_t)n, sizeof(nbr_t *));
    int *cnt = (int *)calloc((size_t)n, sizeof(int));
    double **P = (double **)calloc((size_t)n, sizeof(double *));
    for (int i = 0; i < n; ++i) {
        int cap = 0;
        cnt[i] = neighbours_of(i, n, R, h, hinv, w, rc, &nbl[i], &cap);
        P[i] = (double *)malloc(sizeof(double) * 3 * (size_t)(cnt[i] > 0 ? cnt[i] : 1));
        e_atom[i] = ters_site(&p, nbl[i], cnt[i], P[i]);
    }
    memset(V, 0, 9 * sizeof(double));
    int status = 0;
    for (int i = 0; i < n; ++i) {
        double fi[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < cnt[i]; ++k) {
            const nbr_t *e = &nbl[i][k];
            /* the reverse entry: atom i seen from e->j under shift -t */
            int found = -1;
            for (int q = 0; q < cnt[e->j]; ++q) {
                const nbr_t *r = &nbl[e->j][q];
                if (r->j == i && r->t[0] == -e->t[0] && r->t[1] == -e->t[1] &&
                    r->t[2] == -e->t[2]) { found = q; break; }
            }
            if (found < 0) { status = -1; continue; }
            double f[3];
            for (int c = 0; c < 3; ++c) {
                f[c] = P[i][3 * k + c] - P[e->j][3 * found + c];
                fi[c] += f[c];
            }
            for (int m = 0; m < 3; ++m)
                for (int q = 0; q < 3; ++q) V[3 * m + q] += -0.5 * e->r[m] * f[q];
        }
        for (int c = 0; c < 3; ++c) F[3 * i + c] = fi[c];
    }
    for (int i = 0; i < n; ++i) { free(nbl[i]); free(P[i]); }
    free(nbl); free(cnt); free(P);
    return status;
}

/* Sampled Tersoff forces for large systems: F_i for the atoms idx[0..ns-1]
 * only.  F_i = sum_j [dU_i/dr^{ij} - dU_j/dr^{ji}] needs the sites i and
 * every neighbour j of i, each found by the same brute-force search. */
int oracle_tersoff_sampled(int n, const double *R, const double *h, const double *par,
                           int ns, const int *idx, double *F)
{
    tersoff_params p;
    memcpy(&p, par, sizeof(p));
    double hinv[9], w[3];
    inv3(h, hinv);
    perp_widths(h, w);
    double rc = p.R + p.D;
    int status = 0;
    nbr_t *ni = NULL, *nj = NULL;
    int capi = 0, capj = 0;
    for (int s = 0; s < ns; ++s) {
        int i = idx[s];
        int ci = neighbours_of(i, n, R, h, hinv, w, rc, &ni, &capi);
        double *Pi = (double *)malloc(sizeof(double) * 3 * (size_t)(ci > 0 ? ci : 1));
        ters_site(&p, ni, ci, Pi);
        double fi[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < ci; ++k) {
            int j = ni[k].j;
            int cj = neighbours_of(j, n, R, h, hinv, w, rc, &nj, &capj);
            double *Pj = (double *)malloc(sizeof(double) * 3 * (size_t)(cj > 0 ? cj : 1));
            ters_site(&p, nj, cj, Pj);
            int found = -1;
            for (int q = 0; q < cj; ++q)
                if (nj[q].j == i && nj[q].t[0] == -ni[k].t[0] &&
                    nj[q].t[1] == -ni[k].t[1] && nj[q].t[2] == -ni[k].t[2]) {
                    found = q;
                    break;
                }
            if (found < 0) status = -1;
            else
                for (int c = 0; c < 3; ++c) fi[c] += Pi[3 * k + c] - Pj[3 * found + c];
            free(Pj);
        }
        for (int c = 0; c < 3; ++c) F[3 * s + c] = fi[c];
        free(Pi);
    }
    free(ni);
    free(nj);
    return status;
}

/* Sampled LJ forces: F_i = sum over (j, t) of phi'(r) r^{ij}/r. */
int oracle_lj_sampled(int n, const double *R, const double *h, double eps, double sigma,
                      double rc, int ns, const int *idx, double *F)
{
    double hinv[9], w[3];
    inv3(h, hinv);
    perp_widths(h, w);
    nbr_t *nb = NULL;
    int cap = 0;
    for (int s = 0; s < ns; ++s) {
        int i = idx[s];
        int cnt = neighbours_of(i, n, R, h, hinv, w, rc, &nb, &cap);
        double fi[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < cnt; ++k) {
            double dphi = lj_dphi(nb[k].d, eps, sigma);
            for (int c = 0; c < 3; ++c) fi[c] += dphi * nb[k].r[c] / nb[k].d;
        }
        for (int c = 0; c < 3; ++c) F[3 * s + c] = fi[c];
    }
    free(nb);
    return 0;
}

/* Number of neighbour entries of atom i (diagnostics and tests). */
int oracle_count_neighbours(int n, const double *R, const double *h, double rc, int i)
{
    double hinv[9], w[3];
    inv3(h, hinv);
    perp_widths(h, w);
    nbr_t *nb = NULL;
    int cap = 0;
    int cnt = neighbours_of(i, n, R, h, hinv, w, rc, &nb, &cap);
    free(nb);
    return cnt;
}
