/*
 * oracle.c -- plain FP64 brute-force oracle for real-space grid integration.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path; the two meet only through the
 * seeded inputs (geometry, radial tables, V, D values).
 *
 * What it computes (paper Section 2.2), all sums in FP64 with Neumaier
 * compensation, every sum taken in a fixed order (deterministic for any
 * thread count):
 *   - pattern: all blocks (I, J, T) with |R_J + T - R_I| < rc_I + rc_J (the
 *     overlapping-pair sparsity of Section 2.2), sorted by (I, J, t1, t2, t3);
 *   - H^V_IJ(T)[mu,nu] = sum_g sum_T1 phi_Imu(r_g - R_I - T1) V_g
 *                          phi_Jnu(r_g - R_J - T1 - T) dV            (Eq. 2);
 *   - rho_g = sum over neighbour pairs ((I,T1),(J,T2)) of
 *             phi_Imu D_IJ(T2-T1)[mu,nu] phi_Jnu                     (Eq. 3);
 *   - F_I = -dE/dR_I at fixed V with E = sum_g V_g rho_g dV:
 *           F_I = 2 dV sum_g V_g sum_{T1, mu in I} grad phi_Imu G_Imu  (Eq. 4,
 *           read as the exact derivative of the discrete energy);
 *   - per-atom virial Pi_I[a][b] = 2 dV sum_g V_g sum grad_a phi_Imu d_b G_Imu,
 *     with d = r - R_I - T1; stress = -sum_I Pi_I / Omega           (Eq. 5,
 *     read as the strain derivative at fixed V_g and dV).
 * G_Imu(r) = sum over neighbours (J,T2) of r and nu of D_IJ(T2-T1)[mu,nu] phi_Jnu.
 *
 * Basis (Section 2.1): phi_{l m}(d) = R_l(|d|) Y_lm(d/|d|) for |d| < rc, else 0.
 * R is the cubic Hermite interpolant of the tabulated (y_k, y'_k) on knots
 * r_k = k dr.  Y_lm are real, normalised, without the Condon-Shortley phase,
 * m = -l..l, written as solid harmonics S_lm = r^l Y_lm:
 *   l=1: (y, z, x) sqrt(3/4pi)
 *   l=2: xy, yz, (3z^2-r^2)/2*..., xz, (x^2-y^2)/2*...
 *   l=3: the seven real cubic harmonics.
 * Orbital order inside an atom: l ascending, then radial functions in input
 * order, then m = -l..l.
 * Grid: r_g = sum_i (g_i/n_i) a_i, dV = Omega / N_g.
 *
 * Every grid sum is taken over grid points in infinite space
 * (r = sum_i (k_i/n_i) a_i for any integer k_i, V periodic), which is the same
 * sum as the (g, T1) double sum above.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXL 3
#define ORC_MAXORB 64

typedef struct {
    int n_radial;
    int n_orb;
    double rc;
    /* per radial function */
    int* l;
    int* nk;
    double* dr;
    double** y;
    double** dy;
    /* per orbital: radial index, l, m */
    int* orb_rad;
    int* orb_l;
    int* orb_m;
} orc_species;

typedef struct {
    int n_atoms;
    double* pos;   /* n*3 */
    int* sp;       /* n */
    double A[3][3];    /* rows a_i */
    double Ainv[3][3]; /* A^{-1}: fractional f = r A^{-1} */
    double h[3];       /* interplanar spacings of the cell */
    double omega, dV;
    int n[3];
    int n_species;
    orc_species* species;
    /* pattern */
    int64_t n_blocks;
    int64_t* blocks;   /* n_blocks*5: I, J, t1, t2, t3 */
    int64_t* offsets;  /* n_blocks+1 */
    int64_t* row_start; /* n_atoms+1 */
    int error;
} orc_ctx;

/* ---------------------------------------------------------------- helpers */
static inline void neu_add(double* s, double* c, double x) {
    double t = *s + x;
    if (fabs(*s) >= fabs(x)) *c += (*s - t) + x;
    else *c += (x - t) + *s;
    *s = t;
}

static double det3(double a[3][3]) {
    return a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1])
         - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0])
         + a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
}

static void inv3(double a[3][3], double out[3][3]) {
    double d = det3(a);
    out[0][0] = (a[1][1] * a[2][2] - a[1][2] * a[2][1]) / d;
    out[0][1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) / d;
    out[0][2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) / d;
    out[1][0] = (a[1][2] * a[2][0] - a[1][0] * a[2][2]) / d;
    out[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) / d;
    out[1][2] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) / d;
    out[2][0] = (a[1][0] * a[2][1] - a[1][1] * a[2][0]) / d;
    out[2][1] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) / d;
    out[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) / d;
}

/* fractional coordinates f_i = sum_j r_j Ainv[j][i] */
static inline void to_frac(const orc_ctx* c, const double r[3], double f[3]) {
    for (int i = 0; i < 3; ++i) f[i] = r[0] * c->Ainv[0][i] + r[1] * c->Ainv[1][i] + r[2] * c->Ainv[2][i];
}

/* grid point in infinite space: r = sum_i (k_i / n_i) a_i */
static inline void grid_point(const orc_ctx* c, const int64_t k[3], double r[3]) {
    double f0 = (double)k[0] / c->n[0], f1 = (double)k[1] / c->n[1], f2 = (double)k[2] / c->n[2];
    for (int j = 0; j < 3; ++j) r[j] = f0 * c->A[0][j] + f1 * c->A[1][j] + f2 * c->A[2][j];
}

static inline int64_t pmod(int64_t a, int64_t n) { int64_t m = a % n; return m < 0 ? m + n : m; }

static inline double v_at(const orc_ctx* c, const double* V, const int64_t k[3]) {
    int64_t g0 = pmod(k[0], c->n[0]), g1 = pmod(k[1], c->n[1]), g2 = pmod(k[2], c->n[2]);
    return V[(g0 * c->n[1] + g1) * c->n[2] + g2];
}

/* ------------------------------------------------------- radial functions */
/* Cubic Hermite interpolation of (y_k, y'_k) on knots k*dr: value and derivative. */
static void hermite(const orc_species* s, int ir, double r, double* R, double* dR) {
    double dr = s->dr[ir];
    int nk = s->nk[ir];
    double x = r / dr;
    int64_t k = (int64_t)floor(x);
    if (k >= nk - 1) { *R = 0.0; *dR = 0.0; return; }
    if (k < 0) k = 0;
    double t = x - (double)k;
    double t2 = t * t, t3 = t2 * t;
    double h00 = 2.0 * t3 - 3.0 * t2 + 1.0;
    double h10 = t3 - 2.0 * t2 + t;
    double h01 = -2.0 * t3 + 3.0 * t2;
    double h11 = t3 - t2;
    double d00 = 6.0 * t2 - 6.0 * t;
    double d10 = 3.0 * t2 - 4.0 * t + 1.0;
    double d01 = -6.0 * t2 + 6.0 * t;
    double d11 = 3.0 * t2 - 2.0 * t;
    const double* y = s->y[ir];
    const double* yp = s->dy[ir];
    *R = h00 * y[k] + h10 * dr * yp[k] + h01 * y[k + 1] + h11 * dr * yp[k + 1];
    *dR = (d00 * y[k] + d10 * dr * yp[k] + d01 * y[k + 1] + d11 * dr * yp[k + 1]) / dr;
}

/* ------------------------------------------------ real solid harmonics */
/* S_lm(x,y,z) = r^l Y_lm and its gradient, m = -l..l at index m+l. */
static void solid_harmonics(int l, double x, double y, double z, double* S, double (*G)[3]) {
    const double pi = 3.14159265358979323846;
    if (l == 0) {
        double c0 = sqrt(1.0 / (4.0 * pi));
        S[0] = c0; G[0][0] = G[0][1] = G[0][2] = 0.0;
    } else if (l == 1) {
        double c1 = sqrt(3.0 / (4.0 * pi));
        S[0] = c1 * y; G[0][0] = 0; G[0][1] = c1; G[0][2] = 0;
        S[1] = c1 * z; G[1][0] = 0; G[1][1] = 0; G[1][2] = c1;
        S[2] = c1 * x; G[2][0] = c1; G[2][1] = 0; G[2][2] = 0;
    } else if (l == 2) {
        double a = sqrt(15.0 / (4.0 * pi)), b = sqrt(5.0 / (16.0 * pi)), c = sqrt(15.0 / (16.0 * pi));
        S[0] = a * x * y;      G[0][0] = a * y;   G[0][1] = a * x;  G[0][2] = 0;
        S[1] = a * y * z;      G[1][0] = 0;       G[1][1] = a * z;  G[1][2] = a * y;
        S[2] = b * (2.0 * z * z - x * x - y * y);
        G[2][0] = -2.0 * b * x; G[2][1] = -2.0 * b * y; G[2][2] = 4.0 * b * z;
        S[3] = a * x * z;      G[3][0] = a * z;   G[3][1] = 0;      G[3][2] = a * x;
        S[4] = c * (x * x - y * y);
        G[4][0] = 2.0 * c * x; G[4][1] = -2.0 * c * y; G[4][2] = 0;
    } else {
        double a = sqrt(35.0 / (32.0 * pi)), b = sqrt(105.0 / (4.0 * pi)), c = sqrt(21.0 / (32.0 * pi));
        double d = sqrt(7.0 / (16.0 * pi)), e = sqrt(105.0 / (16.0 * pi));
        S[0] = a * y * (3.0 * x * x - y * y);
        G[0][0] = a * 6.0 * x * y; G[0][1] = a * (3.0 * x * x - 3.0 * y * y); G[0][2] = 0;
        S[1] = b * x * y * z;
        G[1][0] = b * y * z; G[1][1] = b * x * z; G[1][2] = b * x * y;
        S[2] = c * y * (4.0 * z * z - x * x - y * y);
        G[2][0] = c * (-2.0 * x * y); G[2][1] = c * (4.0 * z * z - x * x - 3.0 * y * y); G[2][2] = c * 8.0 * y * z;
        S[3] = d * z * (2.0 * z * z - 3.0 * x * x - 3.0 * y * y);
        G[3][0] = d * (-6.0 * x * z); G[3][1] = d * (-6.0 * y * z); G[3][2] = d * (6.0 * z * z - 3.0 * x * x - 3.0 * y * y);
        S[4] = c * x * (4.0 * z * z - x * x - y * y);
        G[4][0] = c * (4.0 * z * z - 3.0 * x * x - y * y); G[4][1] = c * (-2.0 * x * y); G[4][2] = c * 8.0 * x * z;
        S[5] = e * z * (x * x - y * y);
        G[5][0] = e * 2.0 * x * z; G[5][1] = e * (-2.0 * y * z); G[5][2] = e * (x * x - y * y);
        S[6] = a * x * (x * x - 3.0 * y * y);
        G[6][0] = a * (3.0 * x * x - 3.0 * y * y); G[6][1] = a * (-6.0 * x * y); G[6][2] = 0;
    }
}

/* phi and (optionally) grad phi of every orbital of species s at displacement d.
   Returns 0 (and writes nothing) when |d| >= rc. */
static int eval_orbitals(const orc_species* s, const double d[3], double* phi, double (*gphi)[3]) {
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double r = sqrt(r2);
    if (r >= s->rc) return 0;
    double u[64], du[64];
    int small = r < 1e-12;
    for (int ir = 0; ir < s->n_radial; ++ir) {
        double R, dR;
        int l = s->l[ir];
        if (small) {
            /* limits at the atom centre: phi(0) = R(0) Y00 for l = 0, zero otherwise;
               grad phi(0) = R'(0) grad S_1m for l = 1, zero otherwise. */
            u[ir] = (l == 0) ? s->y[ir][0] : (l == 1 ? s->dy[ir][0] : 0.0);
            du[ir] = 0.0;
            continue;
        }
        hermite(s, ir, r, &R, &dR);
        double rl = 1.0;
        for (int q = 0; q < l; ++q) rl *= r;
        /* u = R / r^l, u' = R'/r^l - l R / r^(l+1) */
        u[ir] = R / rl;
        du[ir] = dR / rl - (double)l * R / (rl * r);
    }
    double S[7], G[7][3];
    int o = 0;
    while (o < s->n_orb) {
        int ir = s->orb_rad[o], l = s->orb_l[o];
        solid_harmonics(l, d[0], d[1], d[2], S, G);
        for (int m = 0; m < 2 * l + 1; ++m, ++o) {
            if (small && l >= 1) phi[o] = 0.0;
            else phi[o] = u[ir] * S[m];
            if (gphi) {
                if (small) {
                    for (int a = 0; a < 3; ++a) gphi[o][a] = (l == 1) ? u[ir] * G[m][a] : 0.0;
                } else {
                    for (int a = 0; a < 3; ++a)
                        gphi[o][a] = du[ir] * (d[a] / r) * S[m] + u[ir] * G[m][a];
                }
            }
        }
    }
    return 1;
}

/* ------------------------------------------------------------ context */
void orc_destroy(orc_ctx* c);

/* Species are described by flat arrays:
 *   rc[s], n_radial[s]; radials of all species concatenated in species order:
 *   rad_l[i], rad_nk[i], rad_dr[i]; y and dy concatenated (rad_nk[i] each). */
orc_ctx* orc_create(int n_atoms, const double* pos, const int* sp, const double* cell,
                    const int* grid, int n_species, const double* rc, const int* n_radial,
                    const int* rad_l, const int* rad_nk, const double* rad_dr,
                    const double* y, const double* dy) {
    orc_ctx* c = (orc_ctx*)calloc(1, sizeof(orc_ctx));
    c->n_atoms = n_atoms;
    c->pos = (double*)malloc(sizeof(double) * 3 * (n_atoms > 0 ? n_atoms : 1));
    c->sp = (int*)malloc(sizeof(int) * (n_atoms > 0 ? n_atoms : 1));
    memcpy(c->pos, pos, sizeof(double) * 3 * n_atoms);
    memcpy(c->sp, sp, sizeof(int) * n_atoms);
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) c->A[i][j] = cell[3 * i + j];
    inv3(c->A, c->Ainv);
    c->omega = fabs(det3(c->A));
    for (int i = 0; i < 3; ++i) {
        double b2 = c->Ainv[0][i] * c->Ainv[0][i] + c->Ainv[1][i] * c->Ainv[1][i] + c->Ainv[2][i] * c->Ainv[2][i];
        c->h[i] = 1.0 / sqrt(b2);
        c->n[i] = grid[i];
    }
    c->dV = c->omega / ((double)grid[0] * grid[1] * grid[2]);
    c->n_species = n_species;
    c->species = (orc_species*)calloc(n_species, sizeof(orc_species));
    int ri = 0;
    int64_t yoff = 0;
    for (int s = 0; s < n_species; ++s) {
        orc_species* S = &c->species[s];
        S->rc = rc[s];
        S->n_radial = n_radial[s];
        S->l = (int*)malloc(sizeof(int) * S->n_radial);
        S->nk = (int*)malloc(sizeof(int) * S->n_radial);
        S->dr = (double*)malloc(sizeof(double) * S->n_radial);
        S->y = (double**)malloc(sizeof(double*) * S->n_radial);
        S->dy = (double**)malloc(sizeof(double*) * S->n_radial);
        int norb = 0;
        for (int k = 0; k < S->n_radial; ++k, ++ri) {
            S->l[k] = rad_l[ri];
            S->nk[k] = rad_nk[ri];
            S->dr[k] = rad_dr[ri];
            S->y[k] = (double*)malloc(sizeof(double) * rad_nk[ri]);
            S->dy[k] = (double*)malloc(sizeof(double) * rad_nk[ri]);
            memcpy(S->y[k], y + yoff, sizeof(double) * rad_nk[ri]);
            memcpy(S->dy[k], dy + yoff, sizeof(double) * rad_nk[ri]);
            yoff += rad_nk[ri];
            norb += 2 * rad_l[ri] + 1;
            if (rad_l[ri] < 0 || rad_l[ri] > ORC_MAXL) c->error = 1;
        }
        if (norb > ORC_MAXORB || S->n_radial > 64) c->error = 1;
        S->n_orb = norb;
        S->orb_rad = (int*)malloc(sizeof(int) * (norb > 0 ? norb : 1));
        S->orb_l = (int*)malloc(sizeof(int) * (norb > 0 ? norb : 1));
        S->orb_m = (int*)malloc(sizeof(int) * (norb > 0 ? norb : 1));
        int o = 0;
        for (int l = 0; l <= ORC_MAXL; ++l)
            for (int k = 0; k < S->n_radial; ++k)
                if (S->l[k] == l)
                    for (int m = -l; m <= l; ++m) { S->orb_rad[o] = k; S->orb_l[o] = l; S->orb_m[o] = m; ++o; }
    }
    /* ---- pattern: all (I, J, T) with |R_J + T - R_I| < rc_I + rc_J, sorted ---- */
    int64_t* cnt = (int64_t*)calloc(n_atoms + 1, sizeof(int64_t));
    int64_t** rows = (int64_t**)calloc(n_atoms > 0 ? n_atoms : 1, sizeof(int64_t*));
#pragma omp parallel for schedule(dynamic, 1)
    for (int I = 0; I < n_atoms; ++I) {
        int64_t cap = 64, nrow = 0;
        int64_t* row = (int64_t*)malloc(sizeof(int64_t) * 4 * cap);
        double rcI = c->species[c->sp[I]].rc;
        for (int J = 0; J < n_atoms; ++J) {
            double rcJ = c->species[c->sp[J]].rc;
            double cut = rcI + rcJ;
            double dd[3] = {c->pos[3 * J] - c->pos[3 * I], c->pos[3 * J + 1] - c->pos[3 * I + 1],
                            c->pos[3 * J + 2] - c->pos[3 * I + 2]};
            double f[3];
            to_frac(c, dd, f);
            int64_t lo[3], hi[3];
            /* R_J + T - R_I within 'cut': -f_i - cut/h_i <= t_i <= -f_i + cut/h_i */
            for (int i = 0; i < 3; ++i) {
                lo[i] = (int64_t)ceil(-f[i] - cut / c->h[i]) - 1;
                hi[i] = (int64_t)floor(-f[i] + cut / c->h[i]) + 1;
            }
            for (int64_t t0 = lo[0]; t0 <= hi[0]; ++t0)
                for (int64_t t1 = lo[1]; t1 <= hi[1]; ++t1)
                    for (int64_t t2 = lo[2]; t2 <= hi[2]; ++t2) {
                        double v[3];
                        for (int j = 0; j < 3; ++j)
                            v[j] = dd[j] + t0 * c->A[0][j] + t1 * c->A[1][j] + t2 * c->A[2][j];
                        double dist = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                        if (dist < cut) {
                            if (nrow == cap) { cap *= 2; row = (int64_t*)realloc(row, sizeof(int64_t) * 4 * cap); }
                            row[4 * nrow] = J; row[4 * nrow + 1] = t0; row[4 * nrow + 2] = t1; row[4 * nrow + 3] = t2;
                            ++nrow;
                        }
                    }
        }
        rows[I] = row;
        cnt[I] = nrow;
    }
    c->row_start = (int64_t*)malloc(sizeof(int64_t) * (n_atoms + 1));
    c->row_start[0] = 0;
    for (int I = 0; I < n_atoms; ++I) c->row_start[I + 1] = c->row_start[I] + cnt[I];
    c->n_blocks = c->row_start[n_atoms];
    c->blocks = (int64_t*)malloc(sizeof(int64_t) * 5 * (c->n_blocks > 0 ? c->n_blocks : 1));
    c->offsets = (int64_t*)malloc(sizeof(int64_t) * (c->n_blocks + 1));
    int64_t b = 0, off = 0;
    for (int I = 0; I < n_atoms; ++I) {
        for (int64_t q = 0; q < cnt[I]; ++q, ++b) {
            int J = (int)rows[I][4 * q];
            c->blocks[5 * b] = I;
            c->blocks[5 * b + 1] = J;
            c->blocks[5 * b + 2] = rows[I][4 * q + 1];
            c->blocks[5 * b + 3] = rows[I][4 * q + 2];
            c->blocks[5 * b + 4] = rows[I][4 * q + 3];
            c->offsets[b] = off;
            off += (int64_t)c->species[c->sp[I]].n_orb * c->species[c->sp[J]].n_orb;
        }
        free(rows[I]);
    }
    c->offsets[c->n_blocks] = off;
    free(rows);
    free(cnt);
    return c;
}

void orc_destroy(orc_ctx* c) {
    if (!c) return;
    for (int s = 0; s < c->n_species; ++s) {
        orc_species* S = &c->species[s];
        for (int k = 0; k < S->n_radial; ++k) { free(S->y[k]); free(S->dy[k]); }
        free(S->l); free(S->nk); free(S->dr); free(S->y); free(S->dy);
        free(S->orb_rad); free(S->orb_l); free(S->orb_m);
    }
    free(c->species); free(c->pos); free(c->sp);
    free(c->blocks); free(c->offsets); free(c->row_start);
    free(c);
}

int orc_error(const orc_ctx* c) { return c->error; }
int64_t orc_n_blocks(const orc_ctx* c) { return c->n_blocks; }
int64_t orc_n_values(const orc_ctx* c) { return c->offsets[c->n_blocks]; }
void orc_blocks(const orc_ctx* c, int64_t* out_blocks, int64_t* out_offsets) {
    memcpy(out_blocks, c->blocks, sizeof(int64_t) * 5 * c->n_blocks);
    memcpy(out_offsets, c->offsets, sizeof(int64_t) * (c->n_blocks + 1));
}
double orc_dV(const orc_ctx* c) { return c->dV; }
double orc_omega(const orc_ctx* c) { return c->omega; }
int orc_n_orb(const orc_ctx* c, int species) { return c->species[species].n_orb; }

/* block index of (I, J, T) in the sorted pattern, or -1 */
static int64_t find_block(const orc_ctx* c, int64_t I, int64_t J, int64_t t0, int64_t t1, int64_t t2) {
    if (I < 0 || I >= c->n_atoms) return -1;
    int64_t lo = c->row_start[I], hi = c->row_start[I + 1] - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        const int64_t* k = c->blocks + 5 * mid;
        int cmp;
        if (k[1] != J) cmp = k[1] < J ? -1 : 1;
        else if (k[2] != t0) cmp = k[2] < t0 ? -1 : 1;
        else if (k[3] != t1) cmp = k[3] < t1 ? -1 : 1;
        else if (k[4] != t2) cmp = k[4] < t2 ? -1 : 1;
        else return mid;
        if (cmp < 0) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* integer box of grid indices k (infinite space) around centre p within radius rad */
static void grid_box(const orc_ctx* c, const double p[3], double rad, int64_t lo[3], int64_t hi[3]) {
    double f[3];
    to_frac(c, p, f);
    for (int i = 0; i < 3; ++i) {
        double w = rad / c->h[i];
        lo[i] = (int64_t)ceil((f[i] - w) * c->n[i]) - 1;
        hi[i] = (int64_t)floor((f[i] + w) * c->n[i]) + 1;
    }
}

/* ------------------------------------------------------------- H^V (Eq. 2) */
/* home index of grid point k (infinite space) in the cell's grid, C order */
static inline int64_t home_index(const orc_ctx* c, const int64_t k[3]) {
    return (pmod(k[0], c->n[0]) * c->n[1] + pmod(k[1], c->n[1])) * c->n[2] + pmod(k[2], c->n[2]);
}

/* mask (nullable): only grid points whose home index g has mask[g] != 0 enter the sum */
static void h_block(const orc_ctx* c, const double* V, int64_t b, double* out, const unsigned char* mask) {
    int64_t I = c->blocks[5 * b], J = c->blocks[5 * b + 1];
    int64_t T[3] = {c->blocks[5 * b + 2], c->blocks[5 * b + 3], c->blocks[5 * b + 4]};
    const orc_species* SI = &c->species[c->sp[I]];
    const orc_species* SJ = &c->species[c->sp[J]];
    int ni = SI->n_orb, nj = SJ->n_orb;
    double RJ[3];
    for (int j = 0; j < 3; ++j)
        RJ[j] = c->pos[3 * J + j] + T[0] * c->A[0][j] + T[1] * c->A[1][j] + T[2] * c->A[2][j];
    const double* RI = c->pos + 3 * I;
    double* s = (double*)calloc((size_t)ni * nj, sizeof(double));
    double* cmp = (double*)calloc((size_t)ni * nj, sizeof(double));
    int64_t lo[3], hi[3];
    grid_box(c, RI, SI->rc, lo, hi);
    double phiI[ORC_MAXORB], phiJ[ORC_MAXORB];
    for (int64_t k0 = lo[0]; k0 <= hi[0]; ++k0)
        for (int64_t k1 = lo[1]; k1 <= hi[1]; ++k1)
            for (int64_t k2 = lo[2]; k2 <= hi[2]; ++k2) {
                int64_t k[3] = {k0, k1, k2};
                if (mask && !mask[home_index(c, k)]) continue;
                double r[3], dI[3], dJ[3];
                grid_point(c, k, r);
                for (int j = 0; j < 3; ++j) { dI[j] = r[j] - RI[j]; dJ[j] = r[j] - RJ[j]; }
                if (!eval_orbitals(SI, dI, phiI, NULL)) continue;
                if (!eval_orbitals(SJ, dJ, phiJ, NULL)) continue;
                double w = v_at(c, V, k) * c->dV;
                for (int mu = 0; mu < ni; ++mu)
                    for (int nu = 0; nu < nj; ++nu)
                        neu_add(&s[mu * nj + nu], &cmp[mu * nj + nu], phiI[mu] * w * phiJ[nu]);
            }
    for (int q = 0; q < ni * nj; ++q) out[q] = s[q] + cmp[q];
    free(s);
    free(cmp);
}

/* Full H on the oracle's own pattern and layout. */
void orc_vlocal(const orc_ctx* c, const double* V, double* H) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < c->n_blocks; ++b) h_block(c, V, b, H + c->offsets[b], NULL);
}

/* H restricted to the grid points with mask[g] != 0 (a shard of the grid): the sum of Eq. 2
   over those points only, so that the shards of a partition of the grid add up to H. */
void orc_vlocal_masked(const orc_ctx* c, const double* V, const unsigned char* mask, double* H) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < c->n_blocks; ++b) h_block(c, V, b, H + c->offsets[b], mask);
}

/* Selected blocks (rows of sel: I, J, t1, t2, t3), written back to back.
   Returns -1 if a requested block is not in the pattern. */
int orc_vlocal_blocks(const orc_ctx* c, const double* V, int64_t n_sel, const int64_t* sel, double* out) {
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (n_sel > 0 ? n_sel : 1));
    int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (n_sel + 1));
    pos[0] = 0;
    for (int64_t q = 0; q < n_sel; ++q) {
        idx[q] = find_block(c, sel[5 * q], sel[5 * q + 1], sel[5 * q + 2], sel[5 * q + 3], sel[5 * q + 4]);
        if (idx[q] < 0) { free(idx); free(pos); return -1; }
        pos[q + 1] = pos[q] + (c->offsets[idx[q] + 1] - c->offsets[idx[q]]);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < n_sel; ++q) h_block(c, V, idx[q], out + pos[q], NULL);
    free(idx);
    free(pos);
    return 0;
}

/* -------------------------------------------------- neighbours of a point */
typedef struct {
    int n;
    int cap;
    int* atom;
    int64_t* t;      /* 3 per entry */
    double* phi;     /* ORC_MAXORB per entry */
} nbr_list;

static void nbr_init(nbr_list* L) { L->n = 0; L->cap = 64; L->atom = malloc(sizeof(int) * 64);
    L->t = malloc(sizeof(int64_t) * 3 * 64); L->phi = malloc(sizeof(double) * ORC_MAXORB * 64); }
static void nbr_free(nbr_list* L) { free(L->atom); free(L->t); free(L->phi); }

/* All (J, T) with |r - R_J - T| < rc_J, with phi_J at that displacement.
   Plain loop over every atom and every candidate image. */
static void neighbours(const orc_ctx* c, const double r[3], nbr_list* L) {
    L->n = 0;
    for (int J = 0; J < c->n_atoms; ++J) {
        const orc_species* S = &c->species[c->sp[J]];
        double d0[3] = {r[0] - c->pos[3 * J], r[1] - c->pos[3 * J + 1], r[2] - c->pos[3 * J + 2]};
        double f[3];
        to_frac(c, d0, f);
        int64_t lo[3], hi[3];
        for (int i = 0; i < 3; ++i) {
            lo[i] = (int64_t)ceil(f[i] - S->rc / c->h[i]) - 1;
            hi[i] = (int64_t)floor(f[i] + S->rc / c->h[i]) + 1;
        }
        for (int64_t t0 = lo[0]; t0 <= hi[0]; ++t0)
            for (int64_t t1 = lo[1]; t1 <= hi[1]; ++t1)
                for (int64_t t2 = lo[2]; t2 <= hi[2]; ++t2) {
                    double d[3];
                    for (int j = 0; j < 3; ++j) d[j] = d0[j] - (t0 * c->A[0][j] + t1 * c->A[1][j] + t2 * c->A[2][j]);
                    if (L->n == L->cap) {
                        L->cap *= 2;
                        L->atom = realloc(L->atom, sizeof(int) * L->cap);
                        L->t = realloc(L->t, sizeof(int64_t) * 3 * L->cap);
                        L->phi = realloc(L->phi, sizeof(double) * ORC_MAXORB * L->cap);
                    }
                    if (!eval_orbitals(S, d, L->phi + (size_t)ORC_MAXORB * L->n, NULL)) continue;
                    L->atom[L->n] = J;
                    L->t[3 * L->n] = t0; L->t[3 * L->n + 1] = t1; L->t[3 * L->n + 2] = t2;
                    L->n++;
                }
    }
}

/* ------------------------------------------------------------ rho (Eq. 3) */
static double rho_point(const orc_ctx* c, const double* D, const int64_t k[3], nbr_list* L, int* err) {
    double r[3];
    grid_point(c, k, r);
    neighbours(c, r, L);
    double s = 0.0, cmp = 0.0;
    for (int a = 0; a < L->n; ++a) {
        int I = L->atom[a];
        int ni = c->species[c->sp[I]].n_orb;
        const double* pa = L->phi + (size_t)ORC_MAXORB * a;
        for (int b = 0; b < L->n; ++b) {
            int J = L->atom[b];
            int nj = c->species[c->sp[J]].n_orb;
            const double* pb = L->phi + (size_t)ORC_MAXORB * b;
            int64_t blk = find_block(c, I, J, L->t[3 * b] - L->t[3 * a], L->t[3 * b + 1] - L->t[3 * a + 1],
                                     L->t[3 * b + 2] - L->t[3 * a + 2]);
            if (blk < 0) { *err = 1; continue; }
            const double* Db = D + c->offsets[blk];
            for (int mu = 0; mu < ni; ++mu)
                for (int nu = 0; nu < nj; ++nu) neu_add(&s, &cmp, pa[mu] * Db[mu * nj + nu] * pb[nu]);
        }
    }
    return s + cmp;
}

/* rho on the full grid, C order [n1][n2][n3]. D on the oracle's layout. */
int orc_rho(const orc_ctx* c, const double* D, double* rho) {
    int err = 0;
#pragma omp parallel reduction(| : err)
    {
        nbr_list L;
        nbr_init(&L);
#pragma omp for schedule(dynamic, 64)
        for (int64_t g = 0; g < (int64_t)c->n[0] * c->n[1] * c->n[2]; ++g) {
            int64_t k[3] = {g / ((int64_t)c->n[1] * c->n[2]), (g / c->n[2]) % c->n[1], g % c->n[2]};
            rho[g] = rho_point(c, D, k, &L, &err);
        }
        nbr_free(&L);
    }
    return err ? -1 : 0;
}

/* rho at selected grid points (rows of idx: g1, g2, g3). */
int orc_rho_points(const orc_ctx* c, const double* D, int64_t n_pts, const int64_t* idx, double* out) {
    int err = 0;
#pragma omp parallel reduction(| : err)
    {
        nbr_list L;
        nbr_init(&L);
#pragma omp for schedule(dynamic, 16)
        for (int64_t q = 0; q < n_pts; ++q) out[q] = rho_point(c, D, idx + 3 * q, &L, &err);
        nbr_free(&L);
    }
    return err ? -1 : 0;
}

/* E = sum_g V_g rho_g dV from the full rho. */
int orc_energy(const orc_ctx* c, const double* V, const double* D, double* E) {
    int64_t ng = (int64_t)c->n[0] * c->n[1] * c->n[2];
    double* rho = (double*)malloc(sizeof(double) * ng);
    int rc = orc_rho(c, D, rho);
    double s = 0.0, cmp = 0.0;
    for (int64_t g = 0; g < ng; ++g) neu_add(&s, &cmp, V[g] * rho[g] * c->dV);
    *E = s + cmp;
    free(rho);
    return rc;
}

/* ----------------------------------------------------- force and virial */
/* F_I (3) and per-atom virial Pi_I (3x3, row a = derivative direction,
   column b = displacement component) for the selected atoms.
   Sum over grid points in infinite space within rc_I of R_I; parallel over
   the first grid index with per-slice compensated partial sums that are
   added in slice order, so the result does not depend on the thread count. */
static int force_impl(const orc_ctx* c, const double* V, const double* D, int n_sel, const int* atoms,
                      double* F, double* virial, const unsigned char* mask) {
    int err = 0;
    for (int q = 0; q < n_sel; ++q) {
        int I = atoms[q];
        const orc_species* SI = &c->species[c->sp[I]];
        int ni = SI->n_orb;
        const double* RI = c->pos + 3 * I;
        int64_t lo[3], hi[3];
        grid_box(c, RI, SI->rc, lo, hi);
        int64_t ns = hi[0] - lo[0] + 1;
        double* part = (double*)calloc((size_t)ns * 24, sizeof(double)); /* 12 sums + 12 compensations */
#pragma omp parallel reduction(| : err)
        {
            nbr_list L;
            nbr_init(&L);
            double phiI[ORC_MAXORB], gI[ORC_MAXORB][3], G[ORC_MAXORB];
#pragma omp for schedule(dynamic, 1)
            for (int64_t k0 = lo[0]; k0 <= hi[0]; ++k0) {
                double* ps = part + 24 * (k0 - lo[0]);
                for (int64_t k1 = lo[1]; k1 <= hi[1]; ++k1)
                    for (int64_t k2 = lo[2]; k2 <= hi[2]; ++k2) {
                        int64_t k[3] = {k0, k1, k2};
                        if (mask && !mask[home_index(c, k)]) continue;
                        double r[3], d[3];
                        grid_point(c, k, r);
                        for (int j = 0; j < 3; ++j) d[j] = r[j] - RI[j];
                        if (!eval_orbitals(SI, d, phiI, gI)) continue;
                        neighbours(c, r, &L);
                        for (int mu = 0; mu < ni; ++mu) G[mu] = 0.0;
                        /* G_Imu = sum_{(J,T2)} sum_nu D_IJ(T2)[mu,nu] phi_Jnu; compensated per mu */
                        double Gs[ORC_MAXORB], Gc[ORC_MAXORB];
                        for (int mu = 0; mu < ni; ++mu) { Gs[mu] = 0.0; Gc[mu] = 0.0; }
                        for (int b = 0; b < L.n; ++b) {
                            int J = L.atom[b];
                            int nj = c->species[c->sp[J]].n_orb;
                            int64_t blk = find_block(c, I, J, L.t[3 * b], L.t[3 * b + 1], L.t[3 * b + 2]);
                            if (blk < 0) { err = 1; continue; }
                            const double* Db = D + c->offsets[blk];
                            const double* pb = L.phi + (size_t)ORC_MAXORB * b;
                            for (int mu = 0; mu < ni; ++mu)
                                for (int nu = 0; nu < nj; ++nu) neu_add(&Gs[mu], &Gc[mu], Db[mu * nj + nu] * pb[nu]);
                        }
                        for (int mu = 0; mu < ni; ++mu) G[mu] = Gs[mu] + Gc[mu];
                        double w = 2.0 * v_at(c, V, k) * c->dV;
                        for (int mu = 0; mu < ni; ++mu)
                            for (int a = 0; a < 3; ++a) {
                                double ga = w * gI[mu][a] * G[mu];
                                neu_add(&ps[a], &ps[12 + a], ga);
                                for (int bb = 0; bb < 3; ++bb)
                                    neu_add(&ps[3 + 3 * a + bb], &ps[12 + 3 + 3 * a + bb], ga * d[bb]);
                            }
                    }
            }
            nbr_free(&L);
        }
        double s[12], cm[12];
        for (int e = 0; e < 12; ++e) { s[e] = 0.0; cm[e] = 0.0; }
        for (int64_t sl = 0; sl < ns; ++sl)
            for (int e = 0; e < 12; ++e) {
                neu_add(&s[e], &cm[e], part[24 * sl + e]);
                neu_add(&s[e], &cm[e], part[24 * sl + 12 + e]);
            }
        for (int a = 0; a < 3; ++a) F[3 * q + a] = s[a] + cm[a];
        if (virial)
            for (int e = 0; e < 9; ++e) virial[9 * q + e] = s[3 + e] + cm[3 + e];
        free(part);
    }
    return err ? -1 : 0;
}

int orc_force(const orc_ctx* c, const double* V, const double* D, int n_sel, const int* atoms,
              double* F, double* virial) {
    return force_impl(c, V, D, n_sel, atoms, F, virial, NULL);
}

/* F_I and Pi_I from the grid points with mask[g] != 0 only (a shard of the grid). */
int orc_force_masked(const orc_ctx* c, const double* V, const double* D, const unsigned char* mask, int n_sel,
                     const int* atoms, double* F, double* virial) {
    return force_impl(c, V, D, n_sel, atoms, F, virial, mask);
}

/* phi and grad phi of one species at displacements d (n x 3); for tests of
   the basis itself. Rows beyond rc are zero. */
void orc_eval_orbitals(const orc_ctx* c, int species, int64_t n, const double* d, double* phi, double* gphi) {
    const orc_species* S = &c->species[species];
    for (int64_t q = 0; q < n; ++q) {
        double p[ORC_MAXORB], g[ORC_MAXORB][3];
        if (!eval_orbitals(S, d + 3 * q, p, g)) {
            for (int o = 0; o < S->n_orb; ++o) { p[o] = 0; g[o][0] = g[o][1] = g[o][2] = 0; }
        }
        for (int o = 0; o < S->n_orb; ++o) {
            phi[q * S->n_orb + o] = p[o];
            if (gphi) for (int a = 0; a < 3; ++a) gphi[(q * S->n_orb + o) * 3 + a] = g[o][a];
        }
    }
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
