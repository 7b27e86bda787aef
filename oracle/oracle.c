/*
 * FP64 CPU oracle for real-space grid integration with numeric atom-centred orbitals.
 *
 * TEST INFRASTRUCTURE ONLY. This file is compiled into liboracle.so and is called by the
 * tests, by the package's smoke check and by the benchmark's CPU-baseline leg. The CUDA
 * library never includes, links or calls it, and it shares no code with that library.
 *
 * What it computes (all in IEEE FP64, compiled with -ffp-contract=off, no fast-math):
 *   - basis functions phi_i(r) = R_f(|r - R_A|) Y_lm(r^) and their gradients, with the
 *     radial part a natural cubic spline through the tabulated R_f on a logarithmic grid
 *     and Y_lm real, orthonormal spherical harmonics evaluated through spherical
 *     coordinates (theta = acos(z/r), phi = atan2(y,x)) and the associated-Legendre
 *     recurrence. (Sec. 3.2.1: NAO basis functions confined to a cutoff radius.)
 *   - the Hamiltonian matrix as the plain discrete definition (Eq. H_int_aims with the
 *     symmetric kinetic form of Eq. RealSpaceHamNonPeriodic):
 *         H_ij = sum_p w_p [ phi_i v_p phi_j + 1/2 grad phi_i . grad phi_j ]
 *     summed point by point over the basis functions that are non-zero at p;
 *   - the density as the plain definition (Eq. Density): n_p = sum_ij phi_i P_ij phi_j;
 *   - the electron count N_e = sum_p w_p n_p;
 *   - the density gradient and Hessian (Sec. 2: the derivatives of Eq. Density needed by GGA
 *     functionals and by forces and stresses), the Hessian from second derivatives of the basis
 *     functions written in Cartesian form, phi = g(r) S_lm(x, y, z) with g = R / r^l and the real
 *     solid harmonic S_lm = r^l Y_lm expanded into monomials by the closed formula of Helgaker,
 *     Jorgensen, Olsen, "Molecular Electronic-Structure Theory" (2000), Eq. 6.4.48 (Racah
 *     normalisation there, times sqrt((2l+1)/(4 pi)) here);
 *   - the batch partition (Sec. 3.3.1, grid-adapted cut planes) and the per-batch reduced
 *     basis sets nnz(B) (Sec. 3.3.2), both under the integer rules stated at each function.
 * Cross-point sums use Neumaier's compensated summation (Neumaier 1974).
 *
 * Readings of the paper used here (the paper is silent on them):
 *   - radial spline: natural cubic spline in the index coordinate s = ln(r/r0)/Delta;
 *     for r < r0 the radial part is taken at r0 (value and derivative); R = 0 for r >= rc;
 *   - real Y_lm without the Condon-Shortley phase; m > 0 carries cos(m phi), m < 0 carries
 *     sin(|m| phi); basis order is atom, then species radial function, then m = -l..l;
 *   - a point that coincides with a nucleus is an error (status -2); a point on the polar
 *     axis of an atom (sin theta < 1e-12) is reported through the pole counter and its
 *     angular gradient is not formed (status -3), because the spherical formula divides
 *     by sin theta there.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_LMAX 6

typedef struct {
    int32_t n_atoms;
    const double *atom_xyz;       /* [n_atoms*3] */
    const int32_t *atom_species;  /* [n_atoms] */
    int32_t n_species;
    const int32_t *species_fn_offset; /* [n_species+1] */
    const int32_t *fn_l;          /* [n_fn] */
    const double *fn_cutoff;      /* [n_fn] */
    int32_t n_rgrid;
    double r0, r_last;
    const double *fn_table;       /* [n_fn*n_rgrid] R_f(r_k) */
    const double *spline_M;       /* [n_fn*n_rgrid] second derivatives in s (from or_spline_M) */
} or_sys;

/* ------------------------------------------------------------------------------------ */
/* compensated summation                                                                */
/* ------------------------------------------------------------------------------------ */
static inline void neu_add(double *s, double *c, double x) {
    double t = *s + x;
    if (fabs(*s) >= fabs(x)) *c += (*s - t) + x;
    else *c += (x - t) + *s;
    *s = t;
}

/* ------------------------------------------------------------------------------------ */
/* natural cubic spline in the index coordinate                                         */
/* ------------------------------------------------------------------------------------ */
/* Second derivatives M_k of the natural cubic spline through (k, y_k), k = 0..n-1:
 * M_{k-1} + 4 M_k + M_{k+1} = 6 (y_{k+1} - 2 y_k + y_{k-1}),  M_0 = M_{n-1} = 0,
 * solved with the Thomas algorithm. */
int or_spline_M(const double *y, int32_t n, double *M) {
    if (n < 2) return -1;
    M[0] = 0.0;
    M[n - 1] = 0.0;
    if (n == 2) return 0;
    int32_t m = n - 2; /* unknowns M_1..M_{n-2} */
    double *c = (double *)malloc(sizeof(double) * (size_t)m);
    double *d = (double *)malloc(sizeof(double) * (size_t)m);
    if (!c || !d) { free(c); free(d); return -1; }
    for (int32_t i = 0; i < m; i++) {
        int32_t k = i + 1;
        double rhs = 6.0 * (y[k + 1] - 2.0 * y[k] + y[k - 1]);
        if (i == 0) {
            c[i] = 1.0 / 4.0;
            d[i] = rhs / 4.0;
        } else {
            double den = 4.0 - c[i - 1];
            c[i] = 1.0 / den;
            d[i] = (rhs - d[i - 1]) / den;
        }
    }
    M[m] = d[m - 1];
    for (int32_t i = m - 2; i >= 0; i--) M[i + 1] = d[i] - c[i] * M[i + 2];
    free(c);
    free(d);
    return 0;
}

/* Value and d/ds of the spline at s (segment k = floor(s), clamped to [0, n-2]). */
static void spline_eval(const double *y, const double *M, int32_t n, double s, double *val, double *dval) {
    int32_t k = (int32_t)floor(s);
    if (k < 0) k = 0;
    if (k > n - 2) k = n - 2;
    double t = s - (double)k;
    double u = 1.0 - t;
    *val = u * y[k] + t * y[k + 1] + ((u * u * u - u) * M[k] + (t * t * t - t) * M[k + 1]) / 6.0;
    *dval = (y[k + 1] - y[k]) + ((1.0 - 3.0 * u * u) * M[k] + (3.0 * t * t - 1.0) * M[k + 1]) / 6.0;
}

/* R_f(r) and dR_f/dr. Zero for r >= rc_f; the radial part is taken at r0 for r < r0. */
void or_radial(const or_sys *S, int32_t f, double r, double *R, double *dR) {
    if (r >= S->fn_cutoff[f]) { *R = 0.0; *dR = 0.0; return; }
    double delta = log(S->r_last / S->r0) / (double)(S->n_rgrid - 1);
    double rr = r < S->r0 ? S->r0 : r;
    double s = log(rr / S->r0) / delta;
    double v, dv;
    spline_eval(S->fn_table + (size_t)f * S->n_rgrid, S->spline_M + (size_t)f * S->n_rgrid, S->n_rgrid, s, &v, &dv);
    *R = v;
    *dR = dv / (rr * delta);
}

/* R_f(r) with dR_f/dr and d^2R_f/dr^2 (same conventions as or_radial). With s = ln(r/r0)/Delta,
 * ds/dr = 1/(r Delta) and d^2s/dr^2 = -1/(r^2 Delta), so R'' = v_ss / (r Delta)^2 - v_s / (r^2 Delta);
 * the spline's second derivative in s is the linear interpolation of M between the knots.     */
void or_radial2(const or_sys *S, int32_t f, double r, double *R, double *dR, double *d2R) {
    if (r >= S->fn_cutoff[f]) { *R = 0.0; *dR = 0.0; *d2R = 0.0; return; }
    double delta = log(S->r_last / S->r0) / (double)(S->n_rgrid - 1);
    double rr = r < S->r0 ? S->r0 : r;
    double s = log(rr / S->r0) / delta;
    const double *y = S->fn_table + (size_t)f * S->n_rgrid, *M = S->spline_M + (size_t)f * S->n_rgrid;
    double v, dv;
    spline_eval(y, M, S->n_rgrid, s, &v, &dv);
    int32_t k = (int32_t)floor(s);
    if (k < 0) k = 0;
    if (k > S->n_rgrid - 2) k = S->n_rgrid - 2;
    double t = s - (double)k;
    double vss = (1.0 - t) * M[k] + t * M[k + 1];
    *R = v;
    *dR = dv / (rr * delta);
    *d2R = vss / ((rr * delta) * (rr * delta)) - dv / (rr * rr * delta);
}

/* ------------------------------------------------------------------------------------ */
/* real spherical harmonics through spherical coordinates                               */
/* ------------------------------------------------------------------------------------ */
static double factorial(int n) { double f = 1.0; for (int i = 2; i <= n; i++) f *= (double)i; return f; }

/* Associated Legendre functions without the Condon-Shortley phase, P[l][m] for 0<=m<=l<=L,
 * at x = cos(theta), st = sin(theta):
 *   P_m^m = (2m-1)!! st^m,  P_{m+1}^m = (2m+1) x P_m^m,
 *   (l-m) P_l^m = (2l-1) x P_{l-1}^m - (l+m-1) P_{l-2}^m.                               */
static void legendre(int L, double x, double st, double P[OR_LMAX + 2][OR_LMAX + 2]) {
    memset(P, 0, sizeof(double) * (OR_LMAX + 2) * (OR_LMAX + 2));
    double pmm = 1.0;
    for (int m = 0; m <= L; m++) {
        if (m > 0) pmm *= (double)(2 * m - 1) * st;
        P[m][m] = pmm;
        if (m + 1 <= L) P[m + 1][m] = (double)(2 * m + 1) * x * pmm;
        for (int l = m + 2; l <= L; l++)
            P[l][m] = ((double)(2 * l - 1) * x * P[l - 1][m] - (double)(l + m - 1) * P[l - 2][m]) / (double)(l - m);
    }
}

/* Y_lm(theta, phi) for m = -l..l, with dY/dtheta and (1/sin theta) dY/dphi.
 * Y_l0 = K_l0 P_l^0; Y_lm = sqrt2 K_lm P_l^m cos(m phi); Y_l,-m = sqrt2 K_lm P_l^m sin(m phi);
 * K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!).
 * dP_l^0/dtheta = -P_l^1;  dP_l^m/dtheta = ((l+m)(l-m+1) P_l^{m-1} - P_l^{m+1}) / 2 for m >= 1. */
static void ylm_sph(int l, double theta, double phi, double *Y, double *dYt, double *dYp_over_st) {
    double x = cos(theta), st = sin(theta);
    double P[OR_LMAX + 2][OR_LMAX + 2];
    legendre(l + 1 <= OR_LMAX + 1 ? l + 1 : OR_LMAX + 1, x, st, P);
    for (int m = 0; m <= l; m++) {
        double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - m) / factorial(l + m));
        double dP;
        if (m == 0) dP = -P[l][1];
        else dP = 0.5 * ((double)(l + m) * (double)(l - m + 1) * P[l][m - 1] - (m + 1 <= l ? P[l][m + 1] : 0.0));
        if (m == 0) {
            Y[l] = K * P[l][0];
            dYt[l] = K * dP;
            dYp_over_st[l] = 0.0;
        } else {
            double c = cos(m * phi), s = sin(m * phi);
            double Pm_over_st = st > 0.0 ? P[l][m] / st : 0.0;
            Y[l + m] = M_SQRT2 * K * P[l][m] * c;
            Y[l - m] = M_SQRT2 * K * P[l][m] * s;
            dYt[l + m] = M_SQRT2 * K * dP * c;
            dYt[l - m] = M_SQRT2 * K * dP * s;
            dYp_over_st[l + m] = -M_SQRT2 * K * Pm_over_st * (double)m * s;
            dYp_over_st[l - m] = M_SQRT2 * K * Pm_over_st * (double)m * c;
        }
    }
}

/* Public helper for the tests: Y_lm (m=-l..l, 2l+1 values) at direction (x,y,z), any length. */
int or_ylm(int32_t l, double x, double y, double z, double *Y) {
    if (l < 0 || l > OR_LMAX) return -1;
    double r = sqrt(x * x + y * y + z * z);
    if (r == 0.0) return -2;
    double dt[2 * OR_LMAX + 1], dp[2 * OR_LMAX + 1];
    ylm_sph(l, acos(z / r), atan2(y, x), Y, dt, dp);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* real solid harmonics as polynomials (for second derivatives)                          */
/* ------------------------------------------------------------------------------------ */
static double binom(int n, int k) { return (k < 0 || k > n) ? 0.0 : factorial(n) / (factorial(k) * factorial(n - k)); }

typedef struct {
    int n;
    double c[64];
    int e[64][3];  /* exponents of x, y, z */
} or_poly;

/* S_lm(x, y, z) = r^l Y_lm as a sum of monomials (Helgaker et al. Eq. 6.4.48):
 *   S = sqrt((2l+1)/(4 pi)) N_lm sum_t sum_u sum_v C_tuv x^(2t+|m|-2(u+v)) y^(2(u+v)) z^(l-2t-|m|),
 *   C_tuv = (-1)^(t+v-v_m) 4^-t binom(l,t) binom(l-t,|m|+t) binom(t,u) binom(|m|,2v),
 *   N_lm = sqrt(2 (l+|m|)! (l-|m|)! / 2^delta_m0) / (2^|m| l!),
 * t = 0..floor((l-|m|)/2), u = 0..t, 2v = 0, 2, .. <= |m| (m >= 0, v_m = 0) or 1, 3, .. <= |m|
 * (m < 0, v_m = 1/2). Index w = 2v below.                                                    */
static void solid_poly(int l, int m, or_poly *P) {
    int am = m < 0 ? -m : m;
    double N = sqrt(2.0 * factorial(l + am) * factorial(l - am) / (m == 0 ? 2.0 : 1.0)) / (pow(2.0, am) * factorial(l));
    double norm = sqrt((2.0 * l + 1.0) / (4.0 * M_PI)) * N;
    P->n = 0;
    for (int t = 0; t <= (l - am) / 2; t++)
        for (int u = 0; u <= t; u++)
            for (int w = (m < 0 ? 1 : 0); w <= am; w += 2) {
                int sgn_exp = t + (m < 0 ? (w - 1) / 2 : w / 2);
                double C = ((sgn_exp & 1) ? -1.0 : 1.0) * pow(0.25, t) * binom(l, t) * binom(l - t, am + t) * binom(t, u) *
                           binom(am, w);
                P->c[P->n] = norm * C;
                P->e[P->n][0] = 2 * t + am - 2 * u - w;
                P->e[P->n][1] = 2 * u + w;
                P->e[P->n][2] = l - 2 * t - am;
                P->n++;
            }
}

static double ipow(double x, int k) { double r = 1.0; for (int i = 0; i < k; i++) r *= x; return r; }

/* value, gradient [3] and Hessian [6] (xx, xy, xz, yy, yz, zz) of a polynomial at (x, y, z) */
static void poly_eval2(const or_poly *P, const double q[3], double *v, double g[3], double h[6]) {
    *v = 0.0;
    for (int c = 0; c < 3; c++) g[c] = 0.0;
    for (int c = 0; c < 6; c++) h[c] = 0.0;
    static const int hp[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    for (int i = 0; i < P->n; i++) {
        const int *e = P->e[i];
        double f[3], d1[3], d2[3];
        for (int c = 0; c < 3; c++) {
            f[c] = ipow(q[c], e[c]);
            d1[c] = e[c] >= 1 ? (double)e[c] * ipow(q[c], e[c] - 1) : 0.0;
            d2[c] = e[c] >= 2 ? (double)(e[c] * (e[c] - 1)) * ipow(q[c], e[c] - 2) : 0.0;
        }
        *v += P->c[i] * f[0] * f[1] * f[2];
        g[0] += P->c[i] * d1[0] * f[1] * f[2];
        g[1] += P->c[i] * f[0] * d1[1] * f[2];
        g[2] += P->c[i] * f[0] * f[1] * d1[2];
        for (int k = 0; k < 6; k++) {
            int a = hp[k][0], b = hp[k][1];
            double prod = P->c[i];
            for (int c = 0; c < 3; c++) {
                int order = (c == a) + (c == b);
                prod *= order == 0 ? f[c] : order == 1 ? d1[c] : d2[c];
            }
            h[k] += prod;
        }
    }
}

/* Public helper for the tests: S_lm (m=-l..l) with gradients [2l+1][3] and Hessians [2l+1][6]
 * at (x, y, z). */
int or_solid(int32_t l, double x, double y, double z, double *S, double *G, double *Hs) {
    if (l < 0 || l > OR_LMAX) return -1;
    double q[3] = {x, y, z};
    for (int m = -l; m <= l; m++) {
        or_poly P;
        solid_poly(l, m, &P);
        poly_eval2(&P, q, S + (l + m), G + 3 * (l + m), Hs + 6 * (l + m));
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* basis functions                                                                      */
/* ------------------------------------------------------------------------------------ */
int64_t or_n_basis(const or_sys *S) {
    int64_t nb = 0;
    for (int32_t a = 0; a < S->n_atoms; a++) {
        int32_t sp = S->atom_species[a];
        for (int32_t f = S->species_fn_offset[sp]; f < S->species_fn_offset[sp + 1]; f++) nb += 2 * S->fn_l[f] + 1;
    }
    return nb;
}

/* All basis functions that are non-zero at point p (r < rc of their radial function), in
 * ascending basis order, with phi and grad phi.  Returns the count, or a negative status.
 * pole_count is incremented for each atom whose polar axis the point lies on.            */
static int64_t point_basis(const or_sys *S, const double p[3], int64_t *idx, double *phi, double *grad,
                           int64_t *pole_count, int all) {
    int64_t cnt = 0, base = 0;
    for (int32_t a = 0; a < S->n_atoms; a++) {
        int32_t sp = S->atom_species[a];
        double dx = p[0] - S->atom_xyz[3 * a + 0];
        double dy = p[1] - S->atom_xyz[3 * a + 1];
        double dz = p[2] - S->atom_xyz[3 * a + 2];
        double r = sqrt(dx * dx + dy * dy + dz * dz);
        int have_angles = 0;
        double theta = 0, ph = 0, st = 0, ct = 0, sp_ = 0, cp = 0;
        for (int32_t f = S->species_fn_offset[sp]; f < S->species_fn_offset[sp + 1]; f++) {
            int l = S->fn_l[f];
            int nm = 2 * l + 1;
            if (!(r < S->fn_cutoff[f])) {
                if (all) {
                    for (int m = 0; m < nm; m++) {
                        idx[cnt] = base + m; phi[cnt] = 0.0;
                        grad[3 * cnt] = grad[3 * cnt + 1] = grad[3 * cnt + 2] = 0.0; cnt++;
                    }
                }
                base += nm;
                continue;
            }
            if (r == 0.0) return -2;
            if (!have_angles) {
                theta = acos(dz / r);
                ph = atan2(dy, dx);
                st = sin(theta); ct = cos(theta); sp_ = sin(ph); cp = cos(ph);
                if (st < 1e-12) { (*pole_count)++; return -3; }
                have_angles = 1;
            }
            double R, dR;
            or_radial(S, f, r, &R, &dR);
            double Y[2 * OR_LMAX + 1], dYt[2 * OR_LMAX + 1], dYp[2 * OR_LMAX + 1];
            ylm_sph(l, theta, ph, Y, dYt, dYp);
            /* grad = R' Y r_hat + (R/r) [dY/dtheta theta_hat + (1/sin) dY/dphi phi_hat] */
            double rh[3] = {st * cp, st * sp_, ct};
            double th[3] = {ct * cp, ct * sp_, -st};
            double fh[3] = {-sp_, cp, 0.0};
            for (int m = 0; m < nm; m++) {
                idx[cnt] = base + m;
                phi[cnt] = R * Y[m];
                for (int c = 0; c < 3; c++)
                    grad[3 * cnt + c] = dR * Y[m] * rh[c] + (R / r) * (dYt[m] * th[c] + dYp[m] * fh[c]);
                cnt++;
            }
            base += nm;
        }
    }
    return cnt;
}

/* Dense phi [n_pts][nb] and grad [n_pts][nb][3] for every basis function (zeros included). */
int or_eval_dense(const or_sys *S, int64_t n_pts, const double *pts, double *phi, double *grad, int64_t *pole_count) {
    int64_t nb = or_n_basis(S);
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nb > 0 ? nb : 1));
    if (!idx) return -1;
    for (int64_t p = 0; p < n_pts; p++) {
        int64_t c = point_basis(S, pts + 3 * p, idx, phi + p * nb, grad + 3 * p * nb, pole_count, 1);
        if (c < 0) { free(idx); return (int)c; }
    }
    free(idx);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Hamiltonian (Eq. H_int_aims) and density (Eq. Density): plain point-by-point sums   */
/* ------------------------------------------------------------------------------------ */
/* H [nb*nb] (full, both triangles formed independently) and the error denominator
 * A_ij = sum_p w_p [ |phi_i v phi_j| + 1/2 |grad phi_i . grad phi_j| ].
 * terms: bit 0 = potential term (v == NULL means v = 1), bit 1 = kinetic term.           */
int or_hamiltonian_tau(const or_sys *S, int64_t n_pts, const double *pts, const double *w, const double *v,
                       const double *vtau, uint32_t terms, double *H, double *A, int64_t *pole_count);

int or_hamiltonian(const or_sys *S, int64_t n_pts, const double *pts, const double *w, const double *v,
                   uint32_t terms, double *H, double *A, int64_t *pole_count) {
    return or_hamiltonian_tau(S, n_pts, pts, w, v, NULL, terms & 3u, H, A, pole_count);
}

/* With the meta-GGA kinetic-energy-density term (Sec. 3.4: the tau-dependent part of the
 * exchange-correlation potential, an extra weighted gradient product): terms bit 4 adds
 *     w_p vtau_p 1/2 grad phi_i . grad phi_j
 * to each point's contribution (vtau required then).                                      */
int or_hamiltonian_tau(const or_sys *S, int64_t n_pts, const double *pts, const double *w, const double *v,
                       const double *vtau, uint32_t terms, double *H, double *A, int64_t *pole_count) {
    int64_t nb = or_n_basis(S);
    size_t nn = (size_t)nb * (size_t)nb;
    double *Hc = (double *)calloc(nn ? nn : 1, sizeof(double));
    double *Ac = (double *)calloc(nn ? nn : 1, sizeof(double));
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nb ? nb : 1));
    double *phi = (double *)malloc(sizeof(double) * (size_t)(nb ? nb : 1));
    double *grad = (double *)malloc(sizeof(double) * 3 * (size_t)(nb ? nb : 1));
    if (!Hc || !Ac || !idx || !phi || !grad) { free(Hc); free(Ac); free(idx); free(phi); free(grad); return -1; }
    memset(H, 0, nn * sizeof(double));
    memset(A, 0, nn * sizeof(double));
    int pot = (terms & 1u) != 0, kin = (terms & 2u) != 0, tau = (terms & 4u) != 0 && vtau != NULL;
    int status = 0;
    for (int64_t p = 0; p < n_pts; p++) {
        int64_t cnt = point_basis(S, pts + 3 * p, idx, phi, grad, pole_count, 0);
        if (cnt < 0) { status = (int)cnt; break; }
        double wp = w[p], vp = v ? v[p] : 1.0;
        for (int64_t a = 0; a < cnt; a++) {
            size_t row = (size_t)idx[a] * (size_t)nb;
            for (int64_t b = 0; b < cnt; b++) {
                double tv = pot ? wp * (phi[a] * vp * phi[b]) : 0.0;
                double gg = grad[3 * a] * grad[3 * b] + grad[3 * a + 1] * grad[3 * b + 1] + grad[3 * a + 2] * grad[3 * b + 2];
                double tk = kin ? wp * 0.5 * gg : 0.0;
                double tt = tau ? wp * vtau[p] * 0.5 * gg : 0.0;
                size_t e = row + (size_t)idx[b];
                neu_add(&H[e], &Hc[e], tv + tk + tt);
                neu_add(&A[e], &Ac[e], fabs(tv) + fabs(tk) + fabs(tt));
            }
        }
    }
    for (size_t e = 0; e < nn; e++) { H[e] += Hc[e]; A[e] += Ac[e]; }
    free(Hc); free(Ac); free(idx); free(phi); free(grad);
    return status;
}

/* phi and grad phi of the single basis function (atom a, radial function f, m) at p.
 * Same formulas as point_basis; returns 0 or a negative status.                        */
static int basis_one(const or_sys *S, int32_t a, int32_t f, int32_t m, const double p[3], double *phi, double g[3],
                     int64_t *pole_count) {
    double dx = p[0] - S->atom_xyz[3 * a + 0];
    double dy = p[1] - S->atom_xyz[3 * a + 1];
    double dz = p[2] - S->atom_xyz[3 * a + 2];
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    *phi = 0.0; g[0] = g[1] = g[2] = 0.0;
    if (!(r < S->fn_cutoff[f])) return 0;
    if (r == 0.0) return -2;
    double theta = acos(dz / r), ph = atan2(dy, dx);
    double st = sin(theta), ct = cos(theta), sp_ = sin(ph), cp = cos(ph);
    if (st < 1e-12) { (*pole_count)++; return -3; }
    int l = S->fn_l[f];
    double R, dR;
    or_radial(S, f, r, &R, &dR);
    double Y[2 * OR_LMAX + 1], dYt[2 * OR_LMAX + 1], dYp[2 * OR_LMAX + 1];
    ylm_sph(l, theta, ph, Y, dYt, dYp);
    double rh[3] = {st * cp, st * sp_, ct};
    double th[3] = {ct * cp, ct * sp_, -st};
    double fh[3] = {-sp_, cp, 0.0};
    int k = m + l;
    *phi = R * Y[k];
    for (int c = 0; c < 3; c++) g[c] = dR * Y[k] * rh[c] + (R / r) * (dYt[k] * th[c] + dYp[k] * fh[c]);
    return 0;
}

/* H and A restricted to a list of basis functions F (the block H[F,F]), from the same
 * definition: every point is visited and only the listed functions are evaluated.       */
int or_hamiltonian_block(const or_sys *S, int64_t n_pts, const double *pts, const double *w, const double *v,
                         uint32_t terms, int32_t nF, const int64_t *F, double *H, double *A, int64_t *pole_count) {
    int64_t nb = or_n_basis(S);
    size_t nn = (size_t)nF * (size_t)nF;
    double *Hc = (double *)calloc(nn ? nn : 1, sizeof(double));
    double *Ac = (double *)calloc(nn ? nn : 1, sizeof(double));
    int32_t *fa = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nF ? nF : 1));
    int32_t *ff = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nF ? nF : 1));
    int32_t *fm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nF ? nF : 1));
    double *fp = (double *)malloc(sizeof(double) * (size_t)(nF ? nF : 1));
    double *fg = (double *)malloc(sizeof(double) * 3 * (size_t)(nF ? nF : 1));
    if (!Hc || !Ac || !fa || !ff || !fm || !fp || !fg) {
        free(Hc); free(Ac); free(fa); free(ff); free(fm); free(fp); free(fg); return -1;
    }
    /* decode each listed index into (atom, radial function, m) by walking the basis order */
    for (int32_t q = 0; q < nF; q++) {
        int64_t base = 0;
        fa[q] = -1;
        for (int32_t a = 0; a < S->n_atoms && fa[q] < 0; a++) {
            int32_t sp = S->atom_species[a];
            for (int32_t f = S->species_fn_offset[sp]; f < S->species_fn_offset[sp + 1]; f++) {
                int nm = 2 * S->fn_l[f] + 1;
                if (F[q] >= base && F[q] < base + nm) { fa[q] = a; ff[q] = f; fm[q] = (int32_t)(F[q] - base) - S->fn_l[f]; break; }
                base += nm;
            }
        }
        if (fa[q] < 0 || F[q] >= nb) { free(Hc); free(Ac); free(fa); free(ff); free(fm); free(fp); free(fg); return -1; }
    }
    memset(H, 0, nn * sizeof(double));
    memset(A, 0, nn * sizeof(double));
    int pot = (terms & 1u) != 0, kin = (terms & 2u) != 0;
    int status = 0;
    for (int64_t p = 0; p < n_pts && !status; p++) {
        for (int32_t q = 0; q < nF && !status; q++)
            status = basis_one(S, fa[q], ff[q], fm[q], pts + 3 * p, &fp[q], &fg[3 * q], pole_count);
        if (status) break;
        double wp = w[p], vp = v ? v[p] : 1.0;
        for (int32_t a = 0; a < nF; a++) {
            if (fp[a] == 0.0 && fg[3 * a] == 0.0 && fg[3 * a + 1] == 0.0 && fg[3 * a + 2] == 0.0) continue;
            for (int32_t b = 0; b < nF; b++) {
                double tv = pot ? wp * (fp[a] * vp * fp[b]) : 0.0;
                double gg = fg[3 * a] * fg[3 * b] + fg[3 * a + 1] * fg[3 * b + 1] + fg[3 * a + 2] * fg[3 * b + 2];
                double tk = kin ? wp * 0.5 * gg : 0.0;
                size_t e = (size_t)a * (size_t)nF + (size_t)b;
                neu_add(&H[e], &Hc[e], tv + tk);
                neu_add(&A[e], &Ac[e], fabs(tv) + fabs(tk));
            }
        }
    }
    for (size_t e = 0; e < nn; e++) { H[e] += Hc[e]; A[e] += Ac[e]; }
    free(Hc); free(Ac); free(fa); free(ff); free(fm); free(fp); free(fg);
    return status;
}

/* n_p = sum_ij phi_i P_ij phi_j over the functions non-zero at p; D_p = sum_ij |phi_i P_ij phi_j|;
 * N_e = sum_p w_p n_p (w may be NULL, then N_e is not formed).                           */
int or_density(const or_sys *S, int64_t n_pts, const double *pts, const double *w, const double *P,
               double *n, double *D, double *Ne, int64_t *pole_count) {
    int64_t nb = or_n_basis(S);
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nb ? nb : 1));
    double *phi = (double *)malloc(sizeof(double) * (size_t)(nb ? nb : 1));
    double *grad = (double *)malloc(sizeof(double) * 3 * (size_t)(nb ? nb : 1));
    if (!idx || !phi || !grad) { free(idx); free(phi); free(grad); return -1; }
    double nes = 0.0, nec = 0.0;
    int status = 0;
    for (int64_t p = 0; p < n_pts; p++) {
        int64_t cnt = point_basis(S, pts + 3 * p, idx, phi, grad, pole_count, 0);
        if (cnt < 0) { status = (int)cnt; break; }
        double s = 0.0, c = 0.0, ds = 0.0, dc = 0.0;
        for (int64_t a = 0; a < cnt; a++) {
            const double *row = P + (size_t)idx[a] * (size_t)nb;
            for (int64_t b = 0; b < cnt; b++) {
                double t = phi[a] * row[idx[b]] * phi[b];
                neu_add(&s, &c, t);
                neu_add(&ds, &dc, fabs(t));
            }
        }
        n[p] = s + c;
        if (D) D[p] = ds + dc;
        if (w) neu_add(&nes, &nec, w[p] * n[p]);
    }
    if (Ne) *Ne = nes + nec;
    free(idx); free(phi); free(grad);
    return status;
}

/* Gradient of the density (Sec. 2, the density gradients needed by GGA functionals, "straightforward
 * extensions of Eq. Density"): differentiating n = sum_ij phi_i P_ij phi_j gives
 *     grad n = sum_ij P_ij (grad phi_i phi_j + phi_i grad phi_j) = 2 sum_ij grad phi_i P_ij phi_j
 * for symmetric P. g[3p + c] is component c at point p; Dg[3p + c] = 2 sum_ij |d_c phi_i P_ij phi_j|
 * (the sum of the term magnitudes, the error denominator). Compensated sums.                 */
int or_density_gradient(const or_sys *S, int64_t n_pts, const double *pts, const double *P, double *g,
                        double *Dg, int64_t *pole_count) {
    int64_t nb = or_n_basis(S);
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nb ? nb : 1));
    double *phi = (double *)malloc(sizeof(double) * (size_t)(nb ? nb : 1));
    double *grad = (double *)malloc(sizeof(double) * 3 * (size_t)(nb ? nb : 1));
    if (!idx || !phi || !grad) { free(idx); free(phi); free(grad); return -1; }
    int status = 0;
    for (int64_t p = 0; p < n_pts; p++) {
        int64_t cnt = point_basis(S, pts + 3 * p, idx, phi, grad, pole_count, 0);
        if (cnt < 0) { status = (int)cnt; break; }
        for (int c = 0; c < 3; c++) {
            double s = 0.0, e = 0.0, ds = 0.0, de = 0.0;
            for (int64_t a = 0; a < cnt; a++) {
                const double *row = P + (size_t)idx[a] * (size_t)nb;
                for (int64_t b = 0; b < cnt; b++) {
                    double t = 2.0 * grad[3 * a + c] * row[idx[b]] * phi[b];
                    neu_add(&s, &e, t);
                    neu_add(&ds, &de, fabs(t));
                }
            }
            g[3 * p + c] = s + e;
            if (Dg) Dg[3 * p + c] = ds + de;
        }
    }
    free(idx); free(phi); free(grad);
    return status;
}

/* All basis functions non-zero at p with phi, gradient [3] and Hessian [6] (xx, xy, xz, yy, yz,
 * zz), in ascending basis order, in Cartesian form: with x = p - R_A, r = |x|, phi = g S_lm,
 * g = R / r^l,
 *   d_a phi     = g' (x_a / r) S + g d_a S,
 *   d_a d_b phi = g'' (x_a x_b / r^2) S + g' (delta_ab / r - x_a x_b / r^3) S
 *                 + (g' / r)(x_b d_a S + x_a d_b S) + g d_a d_b S,
 *   g' = R' / r^l - l R / r^(l+1),  g'' = R'' / r^l - 2 l R' / r^(l+1) + l (l+1) R / r^(l+2).
 * When all is set, every basis function is listed (zeros beyond the cutoff). Returns the count,
 * or -2 for a point on a nucleus.                                                              */
static int64_t point_basis2(const or_sys *S, const double p[3], int64_t *idx, double *phi, double *grad,
                            double *hess, int all) {
    static const int hp[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    int64_t cnt = 0, base = 0;
    for (int32_t a = 0; a < S->n_atoms; a++) {
        int32_t sp = S->atom_species[a];
        double x[3] = {p[0] - S->atom_xyz[3 * a + 0], p[1] - S->atom_xyz[3 * a + 1], p[2] - S->atom_xyz[3 * a + 2]};
        double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        for (int32_t f = S->species_fn_offset[sp]; f < S->species_fn_offset[sp + 1]; f++) {
            int l = S->fn_l[f];
            int nm = 2 * l + 1;
            if (!(r < S->fn_cutoff[f])) {
                if (all)
                    for (int m = 0; m < nm; m++) {
                        idx[cnt] = base + m; phi[cnt] = 0.0;
                        for (int c = 0; c < 3; c++) grad[3 * cnt + c] = 0.0;
                        for (int c = 0; c < 6; c++) hess[6 * cnt + c] = 0.0;
                        cnt++;
                    }
                base += nm;
                continue;
            }
            if (r == 0.0) return -2;
            double R, dR, d2R;
            or_radial2(S, f, r, &R, &dR, &d2R);
            double rl = ipow(r, l);
            double g = R / rl;
            double g1 = dR / rl - (double)l * R / (rl * r);
            double g2 = d2R / rl - 2.0 * (double)l * dR / (rl * r) + (double)(l * (l + 1)) * R / (rl * r * r);
            for (int m = -l; m <= l; m++) {
                or_poly P;
                solid_poly(l, m, &P);
                double Sv, Sg[3], Sh[6];
                poly_eval2(&P, x, &Sv, Sg, Sh);
                idx[cnt] = base + (m + l);
                phi[cnt] = g * Sv;
                for (int c = 0; c < 3; c++) grad[3 * cnt + c] = g1 * (x[c] / r) * Sv + g * Sg[c];
                for (int k = 0; k < 6; k++) {
                    int ia = hp[k][0], ib = hp[k][1];
                    double dab = ia == ib ? 1.0 : 0.0;
                    hess[6 * cnt + k] = g2 * (x[ia] * x[ib] / (r * r)) * Sv + g1 * (dab / r - x[ia] * x[ib] / (r * r * r)) * Sv +
                                        (g1 / r) * (x[ib] * Sg[ia] + x[ia] * Sg[ib]) + g * Sh[k];
                }
                cnt++;
            }
            base += nm;
        }
    }
    return cnt;
}

/* Dense phi [n_pts][nb], grad [n_pts][nb][3] and Hessian [n_pts][nb][6] through the Cartesian
 * form (point_basis2). */
int or_eval_dense2(const or_sys *S, int64_t n_pts, const double *pts, double *phi, double *grad, double *hess) {
    int64_t nb = or_n_basis(S);
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nb > 0 ? nb : 1));
    if (!idx) return -1;
    for (int64_t p = 0; p < n_pts; p++) {
        int64_t c = point_basis2(S, pts + 3 * p, idx, phi + p * nb, grad + 3 * p * nb, hess + 6 * p * nb, 1);
        if (c < 0) { free(idx); return (int)c; }
    }
    free(idx);
    return 0;
}

/* Hessian of the density (Sec. 2: needed for forces and stresses; six components, each a
 * "straightforward extension" of Eq. Density). Differentiating n = sum_ij phi_i P_ij phi_j twice:
 *   d_a d_b n = sum_ij P_ij (d_a d_b phi_i phi_j + d_a phi_i d_b phi_j + d_b phi_i d_a phi_j
 *                            + phi_i d_a d_b phi_j),
 * h[6p + k] for k = xx, xy, xz, yy, yz, zz; Dh = the sum of the four terms' magnitudes.
 * Compensated sums.                                                                          */
int or_density_hessian(const or_sys *S, int64_t n_pts, const double *pts, const double *P, double *h, double *Dh) {
    static const int hp[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    int64_t nb = or_n_basis(S);
    size_t nn = (size_t)(nb ? nb : 1);
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * nn);
    double *phi = (double *)malloc(sizeof(double) * nn);
    double *grad = (double *)malloc(sizeof(double) * 3 * nn);
    double *hs = (double *)malloc(sizeof(double) * 6 * nn);
    if (!idx || !phi || !grad || !hs) { free(idx); free(phi); free(grad); free(hs); return -1; }
    int status = 0;
    for (int64_t p = 0; p < n_pts; p++) {
        int64_t cnt = point_basis2(S, pts + 3 * p, idx, phi, grad, hs, 0);
        if (cnt < 0) { status = (int)cnt; break; }
        for (int k = 0; k < 6; k++) {
            int ia = hp[k][0], ib = hp[k][1];
            double sv = 0.0, se = 0.0, dv = 0.0, de = 0.0;
            for (int64_t a = 0; a < cnt; a++) {
                const double *row = P + (size_t)idx[a] * (size_t)nb;
                for (int64_t b = 0; b < cnt; b++) {
                    double pij = row[idx[b]];
                    double t[4] = {pij * hs[6 * a + k] * phi[b], pij * grad[3 * a + ia] * grad[3 * b + ib],
                                   pij * grad[3 * a + ib] * grad[3 * b + ia], pij * phi[a] * hs[6 * b + k]};
                    for (int u = 0; u < 4; u++) {
                        neu_add(&sv, &se, t[u]);
                        neu_add(&dv, &de, fabs(t[u]));
                    }
                }
            }
            h[6 * p + k] = sv + se;
            if (Dh) Dh[6 * p + k] = dv + de;
        }
    }
    free(idx); free(phi); free(grad); free(hs);
    return status;
}

/* Local Pulay force terms (Sec. 2, Eq. for F^{P,local}: -2 sum_ij int [grad_at phi_i] n_ij h_KS phi_j
 * + 2 sum_ij int [grad_at phi_i] q_ij phi_j, with q the energy-weighted density matrix). The
 * library assembles matrix elements with basis-function indices first ("initially assembling
 * matrix elements", Sec. "Density and Density Derivatives"):
 *     M^c_ij = sum_p w_p d_c phi_i (h phi_j),  h phi_j = -1/2 lap phi_j + v phi_j,
 *     S^c_ij = sum_p w_p d_c phi_i phi_j                       (c = x, y, z),
 * M[c nb^2 + i nb + j]; AM, AS the sums of the term magnitudes (may be NULL). The Laplacian is
 * the trace of the Cartesian basis Hessian (point_basis2). Compensated sums.                   */
int or_pulay_matrices(const or_sys *S, int64_t n_pts, const double *pts, const double *w, const double *v,
                      double *M, double *Sm, double *AM, double *AS) {
    int64_t nb = or_n_basis(S);
    size_t nn = (size_t)nb * (size_t)nb, n1 = (size_t)(nb ? nb : 1);
    double *cM = (double *)calloc(3 * (nn ? nn : 1), sizeof(double));
    double *cS = (double *)calloc(3 * (nn ? nn : 1), sizeof(double));
    double *cAM = (double *)calloc(3 * (nn ? nn : 1), sizeof(double));
    double *cAS = (double *)calloc(3 * (nn ? nn : 1), sizeof(double));
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * n1);
    double *phi = (double *)malloc(sizeof(double) * n1);
    double *grad = (double *)malloc(sizeof(double) * 3 * n1);
    double *hs = (double *)malloc(sizeof(double) * 6 * n1);
    double *hphi = (double *)malloc(sizeof(double) * n1);
    double *dummyM = AM ? AM : cAM, *dummyS = AS ? AS : cAS;
    int status = 0;
    if (!cM || !cS || !cAM || !cAS || !idx || !phi || !grad || !hs || !hphi) { status = -1; goto done; }
    memset(M, 0, 3 * nn * sizeof(double));
    memset(Sm, 0, 3 * nn * sizeof(double));
    if (AM) memset(AM, 0, 3 * nn * sizeof(double));
    if (AS) memset(AS, 0, 3 * nn * sizeof(double));
    for (int64_t p = 0; p < n_pts; p++) {
        int64_t cnt = point_basis2(S, pts + 3 * p, idx, phi, grad, hs, 0);
        if (cnt < 0) { status = (int)cnt; break; }
        double wp = w[p], vp = v ? v[p] : 1.0;
        for (int64_t b = 0; b < cnt; b++) hphi[b] = -0.5 * (hs[6 * b + 0] + hs[6 * b + 3] + hs[6 * b + 5]) + vp * phi[b];
        for (int c = 0; c < 3; c++)
            for (int64_t a = 0; a < cnt; a++) {
                size_t row = (size_t)c * nn + (size_t)idx[a] * (size_t)nb;
                for (int64_t b = 0; b < cnt; b++) {
                    size_t e = row + (size_t)idx[b];
                    double tm = wp * (grad[3 * a + c] * hphi[b]);
                    double ts = wp * (grad[3 * a + c] * phi[b]);
                    neu_add(&M[e], &cM[e], tm);
                    neu_add(&Sm[e], &cS[e], ts);
                    if (AM) AM[e] += fabs(tm);
                    if (AS) AS[e] += fabs(ts);
                }
            }
    }
    for (size_t e = 0; e < 3 * nn; e++) { M[e] += cM[e]; Sm[e] += cS[e]; }
    (void)dummyM; (void)dummyS;
done:
    free(cM); free(cS); free(cAM); free(cAS); free(idx); free(phi); free(grad); free(hs); free(hphi);
    return status;
}

/* The local Pulay forces point by point from their definition (no matrix elements):
 *   F_at = -2 sum_ij sum_p w_p [d/dR_at phi_i] n_ij (h phi_j) + 2 sum_ij sum_p w_p [d/dR_at phi_i] q_ij phi_j,
 * d/dR_at phi_i = -grad phi_i for a function on atom at (0 otherwise); F[3 at + c].          */
int or_pulay_forces(const or_sys *S, int64_t n_pts, const double *pts, const double *w, const double *v,
                    const double *nmat, const double *qmat, double *F) {
    int64_t nb = or_n_basis(S);
    size_t n1 = (size_t)(nb ? nb : 1);
    int32_t *atom_of = (int32_t *)malloc(sizeof(int32_t) * n1);
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * n1);
    double *phi = (double *)malloc(sizeof(double) * n1);
    double *grad = (double *)malloc(sizeof(double) * 3 * n1);
    double *hs = (double *)malloc(sizeof(double) * 6 * n1);
    double *hphi = (double *)malloc(sizeof(double) * n1);
    double *acc = (double *)calloc(3 * (size_t)(S->n_atoms ? S->n_atoms : 1), sizeof(double));
    double *cacc = (double *)calloc(3 * (size_t)(S->n_atoms ? S->n_atoms : 1), sizeof(double));
    int status = 0;
    if (!atom_of || !idx || !phi || !grad || !hs || !hphi || !acc || !cacc) { status = -1; goto done2; }
    {
        int64_t k = 0;
        for (int32_t a = 0; a < S->n_atoms; a++) {
            int32_t sp = S->atom_species[a];
            for (int32_t f = S->species_fn_offset[sp]; f < S->species_fn_offset[sp + 1]; f++)
                for (int m = 0; m < 2 * S->fn_l[f] + 1; m++) atom_of[k++] = a;
        }
    }
    for (int64_t p = 0; p < n_pts; p++) {
        int64_t cnt = point_basis2(S, pts + 3 * p, idx, phi, grad, hs, 0);
        if (cnt < 0) { status = (int)cnt; break; }
        double wp = w[p], vp = v ? v[p] : 1.0;
        for (int64_t b = 0; b < cnt; b++) hphi[b] = -0.5 * (hs[6 * b + 0] + hs[6 * b + 3] + hs[6 * b + 5]) + vp * phi[b];
        for (int64_t a = 0; a < cnt; a++) {
            const double *nr = nmat + (size_t)idx[a] * (size_t)nb, *qr = qmat + (size_t)idx[a] * (size_t)nb;
            int32_t at = atom_of[idx[a]];
            for (int c = 0; c < 3; c++) {
                double dRphi = -grad[3 * a + c];
                for (int64_t b = 0; b < cnt; b++) {
                    double t = -2.0 * wp * dRphi * nr[idx[b]] * hphi[b] + 2.0 * wp * dRphi * qr[idx[b]] * phi[b];
                    neu_add(&acc[3 * at + c], &cacc[3 * at + c], t);
                }
            }
        }
    }
    for (int32_t a = 0; a < 3 * S->n_atoms; a++) F[a] = acc[a] + cacc[a];
done2:
    free(atom_of); free(idx); free(phi); free(grad); free(hs); free(hphi); free(acc); free(cacc);
    return status;
}

/* Periodic Hamiltonian at crystal momentum k (Eq. HamPeriodic with the Bloch basis of
 * Eq. Bloch-basis, chi_ik(r) = sum_T e^{i k.T} phi_i(r - T)), directly from its definition: at
 * every point r of the unit cell the Bloch functions and their gradients are summed over the
 * lattice translations T = n1 a1 + n2 a2 + n3 a3, |n_c| <= nrange, then
 *     h_ij(k) = sum_p w_p [ conj(chi_i) v chi_j (POTENTIAL) + 1/2 conj(grad chi_i) . grad chi_j (KINETIC) ]
 * over the unit cell's points. S describes the unit cell's atoms and basis; lattice = rows a1, a2,
 * a3. Hk[2 (i nb + j)] = (re, im); Ak the sums of the term magnitudes (may be NULL).           */
int or_periodic_h(const or_sys *S, const double *lattice, int32_t nrange, int64_t n_pts, const double *pts,
                  const double *w, const double *v, const double *k, uint32_t terms, double *Hk, double *Ak) {
    int64_t nb = or_n_basis(S);
    size_t n1 = (size_t)(nb ? nb : 1);
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * n1);
    double *phi = (double *)malloc(sizeof(double) * n1), *grad = (double *)malloc(sizeof(double) * 3 * n1);
    double *cr = (double *)malloc(sizeof(double) * n1), *ci = (double *)malloc(sizeof(double) * n1);
    double *gr = (double *)malloc(sizeof(double) * 3 * n1), *gi = (double *)malloc(sizeof(double) * 3 * n1);
    double *cH = (double *)calloc(2 * n1 * n1, sizeof(double));
    int64_t pole = 0;
    int status = 0;
    int pot = (terms & 1u) != 0, kin = (terms & 2u) != 0;
    if (!idx || !phi || !grad || !cr || !ci || !gr || !gi || !cH) { status = -1; goto done3; }
    memset(Hk, 0, 2 * (size_t)nb * (size_t)nb * sizeof(double));
    if (Ak) memset(Ak, 0, (size_t)nb * (size_t)nb * sizeof(double));
    for (int64_t p = 0; p < n_pts; p++) {
        for (int64_t a = 0; a < nb; a++) { cr[a] = ci[a] = 0.0; gr[3 * a] = gr[3 * a + 1] = gr[3 * a + 2] = 0.0; gi[3 * a] = gi[3 * a + 1] = gi[3 * a + 2] = 0.0; }
        for (int n0 = -nrange; n0 <= nrange; n0++)
            for (int n1_ = -nrange; n1_ <= nrange; n1_++)
                for (int n2 = -nrange; n2 <= nrange; n2++) {
                    double T[3];
                    for (int c = 0; c < 3; c++) T[c] = n0 * lattice[c] + n1_ * lattice[3 + c] + n2 * lattice[6 + c];
                    double q[3] = {pts[3 * p] - T[0], pts[3 * p + 1] - T[1], pts[3 * p + 2] - T[2]};
                    int64_t cnt = point_basis(S, q, idx, phi, grad, &pole, 0);
                    if (cnt < 0) { status = (int)cnt; goto done3; }
                    double ph = k[0] * T[0] + k[1] * T[1] + k[2] * T[2];
                    double c_ = cos(ph), s_ = sin(ph);
                    for (int64_t a = 0; a < cnt; a++) {
                        int64_t i = idx[a];
                        cr[i] += c_ * phi[a];
                        ci[i] += s_ * phi[a];
                        for (int c = 0; c < 3; c++) { gr[3 * i + c] += c_ * grad[3 * a + c]; gi[3 * i + c] += s_ * grad[3 * a + c]; }
                    }
                }
        double wp = w[p], vp = v ? v[p] : 1.0;
        for (int64_t i = 0; i < nb; i++)
            for (int64_t j = 0; j < nb; j++) {
                /* conj(x_i) y_j = (xr - i xi)(yr + i yi) */
                double tr = 0.0, ti = 0.0, ta = 0.0;
                if (pot) {
                    double re = cr[i] * cr[j] + ci[i] * ci[j], im = cr[i] * ci[j] - ci[i] * cr[j];
                    tr += wp * vp * re; ti += wp * vp * im;
                    ta += fabs(wp * vp) * sqrt(cr[i] * cr[i] + ci[i] * ci[i]) * sqrt(cr[j] * cr[j] + ci[j] * ci[j]);
                }
                if (kin) {
                    double re = 0.0, im = 0.0, mag = 0.0;
                    for (int c = 0; c < 3; c++) {
                        re += gr[3 * i + c] * gr[3 * j + c] + gi[3 * i + c] * gi[3 * j + c];
                        im += gr[3 * i + c] * gi[3 * j + c] - gi[3 * i + c] * gr[3 * j + c];
                        mag += sqrt(gr[3 * i + c] * gr[3 * i + c] + gi[3 * i + c] * gi[3 * i + c]) *
                               sqrt(gr[3 * j + c] * gr[3 * j + c] + gi[3 * j + c] * gi[3 * j + c]);
                    }
                    tr += 0.5 * wp * re; ti += 0.5 * wp * im; ta += 0.5 * fabs(wp) * mag;
                }
                size_t e = (size_t)i * (size_t)nb + (size_t)j;
                neu_add(&Hk[2 * e], &cH[2 * e], tr);
                neu_add(&Hk[2 * e + 1], &cH[2 * e + 1], ti);
                if (Ak) Ak[e] += ta;
            }
    }
    for (size_t e = 0; e < 2 * (size_t)nb * (size_t)nb; e++) Hk[e] += cH[e];
done3:
    free(idx); free(phi); free(grad); free(cr); free(ci); free(gr); free(gi); free(cH);
    return status;
}

/* Brute force for tiny inputs: phi for every basis function at every point (zeros
 * included) and a triple loop over p, i, j, with no batching and no relevance pruning.   */
int or_bruteforce(const or_sys *S, int64_t n_pts, const double *pts, const double *w, const double *v,
                  const double *P, double *H, double *n, int64_t *pole_count) {
    int64_t nb = or_n_basis(S);
    double *phi = (double *)malloc(sizeof(double) * (size_t)(n_pts * nb + 1));
    double *grad = (double *)malloc(sizeof(double) * 3 * (size_t)(n_pts * nb + 1));
    if (!phi || !grad) { free(phi); free(grad); return -1; }
    int st = or_eval_dense(S, n_pts, pts, phi, grad, pole_count);
    if (st) { free(phi); free(grad); return st; }
    for (int64_t i = 0; i < nb; i++)
        for (int64_t j = 0; j < nb; j++) {
            double s = 0.0, c = 0.0;
            for (int64_t p = 0; p < n_pts; p++) {
                const double *fi = phi + p * nb, *gi = grad + 3 * p * nb;
                double t = w[p] * (fi[i] * v[p] * fi[j] +
                                   0.5 * (gi[3 * i] * gi[3 * j] + gi[3 * i + 1] * gi[3 * j + 1] + gi[3 * i + 2] * gi[3 * j + 2]));
                neu_add(&s, &c, t);
            }
            H[i * nb + j] = s + c;
        }
    for (int64_t p = 0; p < n_pts; p++) {
        double s = 0.0, c = 0.0;
        const double *f = phi + p * nb;
        for (int64_t i = 0; i < nb; i++)
            for (int64_t j = 0; j < nb; j++) neu_add(&s, &c, f[i] * P[i * nb + j] * f[j]);
        n[p] = s + c;
    }
    free(phi); free(grad);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* batch partition (Sec. 3.3.1)                                                         */
/* ------------------------------------------------------------------------------------ */
/* Rule: split(S) with n = |S|, k = ceil(n/B). If k <= 1, S is one batch (in its current
 * order). Otherwise take the axis of largest bounding-box extent (max - min in FP64; ties
 * go x < y < z), stable-sort S by (coordinate, point index), put the first
 * n_L = floor(n * floor(k/2) / k) points left, recurse left then right. Batches are
 * numbered in that depth-first order.                                                     */
typedef struct { double key; int64_t idx; } or_keyed;

static int cmp_keyed(const void *a, const void *b) {
    const or_keyed *x = (const or_keyed *)a, *y = (const or_keyed *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

typedef struct {
    const double *xyz;
    int64_t B;
    int64_t *perm;
    int64_t pos;
    int64_t *offsets;
    int64_t nbatch;
    or_keyed *tmp;
} or_part;

static void split(or_part *st, int64_t *S, int64_t n) {
    int64_t k = (n + st->B - 1) / st->B;
    if (k <= 1) {
        for (int64_t i = 0; i < n; i++) st->perm[st->pos + i] = S[i];
        st->pos += n;
        st->nbatch++;
        st->offsets[st->nbatch] = st->pos;
        return;
    }
    double ext[3];
    for (int c = 0; c < 3; c++) {
        double lo = st->xyz[3 * S[0] + c], hi = lo;
        for (int64_t i = 1; i < n; i++) {
            double v = st->xyz[3 * S[i] + c];
            if (v < lo) lo = v;
            if (v > hi) hi = v;
        }
        ext[c] = hi - lo;
    }
    int ax = 0;
    if (ext[1] > ext[ax]) ax = 1;
    if (ext[2] > ext[ax]) ax = 2;
    for (int64_t i = 0; i < n; i++) { st->tmp[i].key = st->xyz[3 * S[i] + ax]; st->tmp[i].idx = S[i]; }
    qsort(st->tmp, (size_t)n, sizeof(or_keyed), cmp_keyed);
    for (int64_t i = 0; i < n; i++) S[i] = st->tmp[i].idx;
    int64_t kL = k / 2;
    int64_t nL = (n * kL) / k;
    split(st, S, nL);
    split(st, S + nL, n - nL);
}

/* offsets must hold ceil(n/B)+1 entries, perm n entries. Returns the number of batches. */
int64_t or_partition(int64_t n_pts, const double *xyz, int64_t B, int64_t *offsets, int64_t *perm) {
    if (n_pts <= 0 || B <= 0) return -1;
    int64_t *S = (int64_t *)malloc(sizeof(int64_t) * (size_t)n_pts);
    or_keyed *tmp = (or_keyed *)malloc(sizeof(or_keyed) * (size_t)n_pts);
    if (!S || !tmp) { free(S); free(tmp); return -1; }
    for (int64_t i = 0; i < n_pts; i++) S[i] = i;
    or_part st = {xyz, B, perm, 0, offsets, 0, tmp};
    offsets[0] = 0;
    split(&st, S, n_pts);
    free(S);
    free(tmp);
    return st.nbatch;
}

/* ------------------------------------------------------------------------------------ */
/* reduced basis per batch, nnz(B) (Sec. 3.3.2)                                          */
/* ------------------------------------------------------------------------------------ */
/* Rule: basis function (atom A, radial function f, m) is relevant to batch b iff some
 * point p of b has r2 < rc_f * rc_f with r2 = (dx*dx + dy*dy) + dz*dz, each operation a
 * separately rounded FP64 operation (no fused multiply-add). Indices ascending.
 * With rel_idx == NULL only the offsets are written. Returns the total count.           */
int64_t or_relevance(const or_sys *S, const double *pts, int64_t n_batches, const int64_t *offsets,
                     const int64_t *perm, int64_t *rel_offsets, int32_t *rel_idx) {
    int64_t total = 0;
    rel_offsets[0] = 0;
    for (int64_t b = 0; b < n_batches; b++) {
        int64_t base = 0;
        for (int32_t a = 0; a < S->n_atoms; a++) {
            int32_t sp = S->atom_species[a];
            double minr2 = INFINITY;
            for (int64_t q = offsets[b]; q < offsets[b + 1]; q++) {
                const double *p = pts + 3 * perm[q];
                double dx = p[0] - S->atom_xyz[3 * a + 0];
                double dy = p[1] - S->atom_xyz[3 * a + 1];
                double dz = p[2] - S->atom_xyz[3 * a + 2];
                double r2 = (dx * dx + dy * dy) + dz * dz;
                if (r2 < minr2) minr2 = r2;
            }
            for (int32_t f = S->species_fn_offset[sp]; f < S->species_fn_offset[sp + 1]; f++) {
                int nm = 2 * S->fn_l[f] + 1;
                double rc = S->fn_cutoff[f];
                if (minr2 < rc * rc) {
                    for (int m = 0; m < nm; m++) {
                        if (rel_idx) rel_idx[total] = (int32_t)(base + m);
                        total++;
                    }
                }
                base += nm;
            }
        }
        rel_offsets[b + 1] = total;
    }
    return total;
}
