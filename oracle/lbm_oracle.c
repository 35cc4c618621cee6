/*
 * Oracle: a plain, slow FP64 CPU restatement of the wind-turbine LBM + actuator
 * line method (arxiv 2402.13171).  TEST INFRASTRUCTURE ONLY: it exists so the
 * CUDA path can be checked against something written directly from the
 * mathematics.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline legs may load it; the product library never does, and this file
 * shares no code, header, table or constant with the CUDA path.
 *
 * Every function follows one passage of the paper (section / equation) or,
 * where the paper is silent, one stated reading:
 *   - D3Q27 stencil, moments with force half-shift ........ Sec. 2.1 (moments)
 *   - lattice Boltzmann equation with source term ......... Sec. 2.1, Eq. (lbm)
 *   - Guo forcing, collide/stream split ................... Sec. 2.1
 *   - cumulant collision (Geier et al. 2015) .............. Sec. 2.1
 *   - blade-line kinematics (Line::update) ................ Sec. 3.3, Algorithm 2
 *   - trilinear interpolation of rho and u ................ Sec. 2.2
 *   - force regularisation f_eps = f (x) eta_eps ........... Sec. 2.2
 *     (Gaussian kernel, or the discrete delta of Roma et al. 1999 that Sec. 2.2 names)
 *   - blade-element force F = 1/2 rho u_rel^2 w l (...) .... Sec. 2.2, element-force equation
 *   - tabulated polars C_L(alpha), C_D(alpha) ............. Sec. 2.2
 *   - Glauert tip-loss factor (optional) .................. Sec. 2.2, Sec. 5
 * Readings (paper silent): Gaussian regularisation with per-axis 3*eps cut-off
 * and per-axis renormalisation (the Roma delta needs neither); lagged force in
 * the velocity sample; Smagorinsky BGK variant (Hou et al. 1996);
 * inlet/outlet/no-slip boundary rules; inflow noise from splitmix64.  Each is
 * stated at its function.
 *
 * Velocity ordering: q = (cz+1)*9 + (cy+1)*3 + (cx+1), so q = 13 is the rest
 * population and opposite(q) = 26 - q.  Moment multi-indices (a,b,c) use the
 * same packing m = c*9 + b*3 + a.  Arrays of PDFs are [q][z][y][x], x fastest.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NQ 27

static int cx_of(int q) { return q % 3 - 1; }
static int cy_of(int q) { return (q / 3) % 3 - 1; }
static int cz_of(int q) { return q / 9 - 1; }
static int opp_of(int q) { return 26 - q; }

/* One-dimensional D1Q3 weights; the D3Q27 weight is their product. */
static double w1d(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
static double w_of(int q) { return w1d(cx_of(q)) * w1d(cy_of(q)) * w1d(cz_of(q)); }

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Equilibria                                                                */
/* ------------------------------------------------------------------------ */

/* Product-form D3Q27 equilibrium: f_q = rho * prod_a phi(c_qa, u_a) with the
 * one-dimensional factors chosen so that phi has zeroth moment 1, first moment
 * u and second central moment 1/3 (c_s^2).  Reading for the cumulant scheme:
 * its equilibrium has vanishing cumulants above second order. */
static double phi1d(int c, double u)
{
    if (c == 0) return 2.0 / 3.0 - u * u;
    return 0.5 * (1.0 / 3.0 + u * u + c * u);
}

void or_equilibrium(double rho, const double u[3], double feq[NQ])
{
    for (int q = 0; q < NQ; ++q)
        feq[q] = rho * phi1d(cx_of(q), u[0]) * phi1d(cy_of(q), u[1]) * phi1d(cz_of(q), u[2]);
}

/* Second-order polynomial equilibrium of the BGK (SRT) variant. */
void or_equilibrium_poly(double rho, const double u[3], double feq[NQ])
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int q = 0; q < NQ; ++q) {
        double cu = cx_of(q) * u[0] + cy_of(q) * u[1] + cz_of(q) * u[2];
        feq[q] = w_of(q) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

/* Macroscopic density and velocity with the Guo half-force shift:
 * rho = sum f, rho u = sum c f + F/2 (Sec. 2.1; the printed F dt/(2 rho) is read
 * as F dt / 2, the dimensionally consistent Guo 2002 form). */
void or_macroscopic(const double f[NQ], const double F[3], double* rho, double u[3])
{
    double r = 0, j[3] = {0, 0, 0};
    for (int q = 0; q < NQ; ++q) {
        r += f[q];
        j[0] += cx_of(q) * f[q];
        j[1] += cy_of(q) * f[q];
        j[2] += cz_of(q) * f[q];
    }
    *rho = r;
    for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * F[a]) / r;
}

/* ------------------------------------------------------------------------ */
/* Central moments <-> populations                                          */
/* ------------------------------------------------------------------------ */

/* A(u)[m][j] = (c_j - u)^m for the one-dimensional velocities c_j = j-1. */
static void axis_matrix(double u, double A[3][3])
{
    for (int j = 0; j < 3; ++j) {
        double d = (double)(j - 1) - u;
        A[0][j] = 1.0;
        A[1][j] = d;
        A[2][j] = d * d;
    }
}

static void invert3(const double A[3][3], double B[3][3])
{
    double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
               - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
               + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    B[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / det;
    B[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
    B[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
    B[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / det;
    B[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
    B[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
    B[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / det;
    B[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
    B[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
}

/* kappa_{abc} = sum_q (c_qx-u_x)^a (c_qy-u_y)^b (c_qz-u_z)^c f_q. */
void or_central_moments(const double f[NQ], const double u[3], double kappa[NQ])
{
    double Ax[3][3], Ay[3][3], Az[3][3];
    axis_matrix(u[0], Ax);
    axis_matrix(u[1], Ay);
    axis_matrix(u[2], Az);
    for (int m = 0; m < NQ; ++m) {
        int a = m % 3, b = (m / 3) % 3, c = m / 9;
        double s = 0;
        for (int q = 0; q < NQ; ++q)
            s += Ax[a][q % 3] * Ay[b][(q / 3) % 3] * Az[c][q / 9] * f[q];
        kappa[m] = s;
    }
}

/* Inverse of or_central_moments: the moment map is the tensor product of the
 * three one-dimensional maps A(u), so its inverse is the tensor product of
 * their inverses. */
void or_populations_from_central(const double kappa[NQ], const double u[3], double f[NQ])
{
    double Ax[3][3], Ay[3][3], Az[3][3], Bx[3][3], By[3][3], Bz[3][3];
    axis_matrix(u[0], Ax);
    axis_matrix(u[1], Ay);
    axis_matrix(u[2], Az);
    invert3(Ax, Bx);
    invert3(Ay, By);
    invert3(Az, Bz);
    for (int q = 0; q < NQ; ++q) {
        int jx = q % 3, jy = (q / 3) % 3, jz = q / 9;
        double s = 0;
        for (int m = 0; m < NQ; ++m)
            s += Bx[jx][m % 3] * By[jy][(m / 3) % 3] * Bz[jz][m / 9] * kappa[m];
        f[q] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* Central moments <-> cumulants                                            */
/* ------------------------------------------------------------------------ */
/*
 * Cumulants follow the zero-mean moment-cumulant relation: a normalised
 * central moment k_m = kappa_m / rho equals the sum, over every partition of
 * the multiset of axis labels of m into blocks of size >= 2, of the product of
 * the cumulants of the blocks (singleton blocks are absent because the moments
 * are central).  This is the relation that defines the cumulants of Geier et
 * al. 2015 in terms of central moments; the first-order central moments are
 * not part of it (they carry only the force half-shift and are handled by the
 * collision directly).  Cumulants are returned rho-weighted: C_m = rho c_m.
 */

typedef struct {
    int target;      /* moment index m */
    int nfac;        /* number of blocks (2 or 3) */
    int fac[3];      /* moment index of each block */
} or_term;

static or_term g_terms[1024];
static int g_nterms = 0;
static int g_first[NQ + 1]; /* terms of target m are g_terms[g_first[m] .. g_first[m+1]) */
static int g_terms_ready = 0;

static int order_of(int m) { return m % 3 + (m / 3) % 3 + m / 9; }

static void build_partition_terms(void)
{
    if (g_terms_ready) return;
    int n_terms = 0;
    for (int m = 0; m < NQ; ++m) {
        int a = m % 3, b = (m / 3) % 3, c = m / 9;
        int n = a + b + c;
        g_first[m] = n_terms;
        if (n < 4) continue; /* orders 2, 3 have only the single-block partition */
        int label[6], k = 0;
        for (int i = 0; i < a; ++i) label[k++] = 0;
        for (int i = 0; i < b; ++i) label[k++] = 1;
        for (int i = 0; i < c; ++i) label[k++] = 2;
        /* enumerate set partitions by restricted growth strings */
        int rg[6] = {0, 0, 0, 0, 0, 0};
        for (;;) {
            int nb = 0;
            for (int i = 0; i < n; ++i) if (rg[i] + 1 > nb) nb = rg[i] + 1;
            int size[6] = {0}, cnt[6][3];
            memset(cnt, 0, sizeof cnt);
            for (int i = 0; i < n; ++i) {
                size[rg[i]]++;
                cnt[rg[i]][label[i]]++;
            }
            int ok = nb >= 2;
            for (int bb = 0; bb < nb; ++bb) if (size[bb] < 2) ok = 0;
            if (ok) {
                or_term t;
                t.target = m;
                t.nfac = nb;
                for (int bb = 0; bb < nb; ++bb) t.fac[bb] = cnt[bb][2] * 9 + cnt[bb][1] * 3 + cnt[bb][0];
                for (int bb = nb; bb < 3; ++bb) t.fac[bb] = 0;
                g_terms[n_terms++] = t;
            }
            /* next restricted growth string */
            int i = n - 1;
            for (; i >= 1; --i) {
                int mx = 0;
                for (int j = 0; j < i; ++j) if (rg[j] > mx) mx = rg[j];
                if (rg[i] <= mx) { rg[i]++; for (int j = i + 1; j < n; ++j) rg[j] = 0; break; }
            }
            if (i < 1) break;
        }
    }
    g_first[NQ] = n_terms;
    g_nterms = n_terms;
    g_terms_ready = 1;
}

int or_partition_term_count(void)
{
    build_partition_terms();
    return g_nterms;
}

void or_cumulants_from_central(const double kappa[NQ], double C[NQ])
{
    build_partition_terms();
    double rho = kappa[0];
    double k[NQ], c[NQ];
    for (int m = 0; m < NQ; ++m) k[m] = kappa[m] / rho;
    /* increasing order: every block of a multi-block partition has lower order */
    for (int ord = 0; ord <= 6; ++ord) {
        for (int m = 0; m < NQ; ++m) {
            if (order_of(m) != ord) continue;
            double s = k[m];
            for (int t = g_first[m]; t < g_first[m + 1]; ++t) {
                double p = 1.0;
                for (int i = 0; i < g_terms[t].nfac; ++i) p *= c[g_terms[t].fac[i]];
                s -= p;
            }
            c[m] = s;
        }
    }
    for (int m = 0; m < NQ; ++m) C[m] = rho * c[m];
    C[0] = rho;
}

void or_central_from_cumulants(const double C[NQ], double kappa[NQ])
{
    build_partition_terms();
    double rho = C[0];
    double c[NQ];
    for (int m = 0; m < NQ; ++m) c[m] = C[m] / rho;
    for (int m = 0; m < NQ; ++m) {
        double s = c[m];
        for (int t = g_first[m]; t < g_first[m + 1]; ++t) {
            double p = 1.0;
            for (int i = 0; i < g_terms[t].nfac; ++i) p *= c[g_terms[t].fac[i]];
            s += p;
        }
        kappa[m] = rho * s;
    }
    kappa[0] = rho;
}

/* ------------------------------------------------------------------------ */
/* Collision operators                                                       */
/* ------------------------------------------------------------------------ */

#define MI(a, b, c) ((c) * 9 + (b) * 3 + (a))

/*
 * Cumulant collision (Sec. 2.1, Geier et al. 2015) with forcing by the
 * velocity shift.  rates[0] = omega1 (shear: off-diagonal and deviatoric
 * second-order cumulants), rates[1] = omega2 (bulk: trace), rates[2..9] =
 * omega3..omega10 for the third- to sixth-order groups of Geier 2015:
 *   omega3: C120+C102, C210+C012, C201+C021   omega4: the differences
 *   omega5: C111
 *   omega6: C220-2C202+C022, C220+C202-2C022   omega7: C220+C202+C022
 *   omega8: C211, C121, C112   omega9: C221, C212, C122   omega10: C222
 * Equilibria: trace -> rho, every other group -> 0.
 * Forcing: u = (sum c f + F/2)/rho; the pre-collision first central moments
 * are -F/2 and the post-collision ones are set to +F/2, which adds exactly F
 * to the momentum (the Guo force model in central-moment form).
 */
void or_collide_cumulant(const double f[NQ], const double F[3], const double rates[10], double fout[NQ])
{
    double rho, u[3], kap[NQ], C[NQ], Cs[NQ], kaps[NQ];
    or_macroscopic(f, F, &rho, u);
    or_central_moments(f, u, kap);
    or_cumulants_from_central(kap, C);
    memcpy(Cs, C, sizeof Cs);

    double w1 = rates[0], w2 = rates[1];
    const double* wh = rates + 2; /* wh[0] = omega3 ... wh[7] = omega10 */

    /* second order */
    Cs[MI(1, 1, 0)] = (1 - w1) * C[MI(1, 1, 0)];
    Cs[MI(1, 0, 1)] = (1 - w1) * C[MI(1, 0, 1)];
    Cs[MI(0, 1, 1)] = (1 - w1) * C[MI(0, 1, 1)];
    double Dxy = C[MI(2, 0, 0)] - C[MI(0, 2, 0)];
    double Dxz = C[MI(2, 0, 0)] - C[MI(0, 0, 2)];
    double T = C[MI(2, 0, 0)] + C[MI(0, 2, 0)] + C[MI(0, 0, 2)];
    Dxy *= (1 - w1);
    Dxz *= (1 - w1);
    T = T + w2 * (rho - T);
    Cs[MI(2, 0, 0)] = (T + Dxy + Dxz) / 3.0;
    Cs[MI(0, 2, 0)] = (T - 2 * Dxy + Dxz) / 3.0;
    Cs[MI(0, 0, 2)] = (T + Dxy - 2 * Dxz) / 3.0;

    /* third order */
    {
        const int pairs[3][2] = {{MI(1, 2, 0), MI(1, 0, 2)}, {MI(2, 1, 0), MI(0, 1, 2)}, {MI(2, 0, 1), MI(0, 2, 1)}};
        for (int p = 0; p < 3; ++p) {
            double s = (1 - wh[0]) * (C[pairs[p][0]] + C[pairs[p][1]]);
            double d = (1 - wh[1]) * (C[pairs[p][0]] - C[pairs[p][1]]);
            Cs[pairs[p][0]] = 0.5 * (s + d);
            Cs[pairs[p][1]] = 0.5 * (s - d);
        }
        Cs[MI(1, 1, 1)] = (1 - wh[2]) * C[MI(1, 1, 1)];
    }
    /* fourth order */
    {
        double c220 = C[MI(2, 2, 0)], c202 = C[MI(2, 0, 2)], c022 = C[MI(0, 2, 2)];
        double A = (1 - wh[3]) * (c220 - 2 * c202 + c022);
        double B = (1 - wh[3]) * (c220 + c202 - 2 * c022);
        double S = (1 - wh[4]) * (c220 + c202 + c022);
        Cs[MI(2, 2, 0)] = (A + B + S) / 3.0;
        Cs[MI(2, 0, 2)] = (S - A) / 3.0;
        Cs[MI(0, 2, 2)] = (S - B) / 3.0;
        Cs[MI(2, 1, 1)] = (1 - wh[5]) * C[MI(2, 1, 1)];
        Cs[MI(1, 2, 1)] = (1 - wh[5]) * C[MI(1, 2, 1)];
        Cs[MI(1, 1, 2)] = (1 - wh[5]) * C[MI(1, 1, 2)];
    }
    /* fifth and sixth order */
    Cs[MI(2, 2, 1)] = (1 - wh[6]) * C[MI(2, 2, 1)];
    Cs[MI(2, 1, 2)] = (1 - wh[6]) * C[MI(2, 1, 2)];
    Cs[MI(1, 2, 2)] = (1 - wh[6]) * C[MI(1, 2, 2)];
    Cs[MI(2, 2, 2)] = (1 - wh[7]) * C[MI(2, 2, 2)];

    /* forcing: first central moments -F/2 -> +F/2 */
    Cs[MI(1, 0, 0)] = 0.5 * F[0];
    Cs[MI(0, 1, 0)] = 0.5 * F[1];
    Cs[MI(0, 0, 1)] = 0.5 * F[2];

    or_central_from_cumulants(Cs, kaps);
    or_populations_from_central(kaps, u, fout);
}

/*
 * BGK (single relaxation time) with a Smagorinsky eddy viscosity and the Guo
 * source term -- the second collision operator of the solver (a reading: the
 * paper describes only the cumulant scheme).  tau_eff follows the closed form
 * of Hou et al. 1996, tau = (tau0 + sqrt(tau0^2 + 18 sqrt(2) C^2 |Pi|/rho))/2,
 * with Pi = sum c c (f - feq) + (u F + F u)/2 the force-corrected
 * non-equilibrium momentum flux; S_q = (1 - omega/2) w_q [3(c-u) + 9 (c.u) c].F.
 */
void or_collide_srt_smag(const double f[NQ], const double F[3], double nu, double smag_c, double fout[NQ])
{
    double rho, u[3], feq[NQ];
    or_macroscopic(f, F, &rho, u);
    or_equilibrium_poly(rho, u, feq);
    double Pi[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0;
            for (int q = 0; q < NQ; ++q) {
                int c[3] = {cx_of(q), cy_of(q), cz_of(q)};
                s += c[a] * c[b] * (f[q] - feq[q]);
            }
            Pi[a][b] = s + 0.5 * (u[a] * F[b] + u[b] * F[a]);
        }
    double P2 = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) P2 += Pi[a][b] * Pi[a][b];
    double tau0 = 3.0 * nu + 0.5;
    double tau = 0.5 * (tau0 + sqrt(tau0 * tau0 + 18.0 * sqrt(2.0) * smag_c * smag_c * sqrt(P2) / rho));
    double om = 1.0 / tau;
    for (int q = 0; q < NQ; ++q) {
        int c[3] = {cx_of(q), cy_of(q), cz_of(q)};
        double cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
        double s = 0;
        for (int a = 0; a < 3; ++a) s += (3.0 * (c[a] - u[a]) + 9.0 * cu * c[a]) * F[a];
        fout[q] = f[q] - om * (f[q] - feq[q]) + (1.0 - 0.5 * om) * w_of(q) * s;
    }
}

/* Relaxation rate of the shear cumulants from the lattice viscosity:
 * nu = c_s^2 (1/omega - 1/2) with c_s^2 = 1/3. */
double or_omega_from_nu(double nu) { return 1.0 / (3.0 * nu + 0.5); }

/* ------------------------------------------------------------------------ */
/* Domain, boundaries, inflow                                                */
/* ------------------------------------------------------------------------ */

enum { OR_BC_PERIODIC = 0, OR_BC_INOUT = 1, OR_BC_NOSLIP = 2, OR_BC_FREESLIP = 3 };
enum { OR_COLL_CUMULANT = 0, OR_COLL_SRT_SMAG = 1 };

typedef struct {
    int nx, ny, nz;
    int collision;
    double nu, smag_c;
    int bc[3];
    double body_force[3];
    int inflow_kind;          /* 0 uniform, 1 log law in z */
    double u_ref[3];
    double z0, z_ref;
    double noise_rel;
    unsigned long long seed;
} or_domain;

/* splitmix64 (Steele, Lea, Flood 2014): the k-th output (k >= 1) of the
 * generator whose state starts at `seed` is mix(seed + k * 0x9E3779B97F4A7C15). */
uint64_t or_splitmix64(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + k * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Uniform variate in [-1, 1) from the top 53 bits. */
static double uniform_pm1(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0; }

/* Inflow velocity of inlet column (y, z) at step n (reading of the configured
 * "uniform inflow with seeded white noise"): the mean profile (uniform u_ref,
 * or u_ref scaled by ln(z_c/z0)/ln(z_ref/z0) at z_c = z + 1/2), plus, for each
 * component a, noise_rel * |u_ref| * xi with xi in [-1, 1) the
 * (counter+1)-th splitmix64 output, counter = ((n*nz + z)*ny + y)*3 + a. */
void or_inflow_velocity(const or_domain* d, long step, int y, int z, double u[3])
{
    double scale = 1.0;
    if (d->inflow_kind == 1) scale = log((z + 0.5) / d->z0) / log(d->z_ref / d->z0);
    double U0 = sqrt(d->u_ref[0] * d->u_ref[0] + d->u_ref[1] * d->u_ref[1] + d->u_ref[2] * d->u_ref[2]);
    for (int a = 0; a < 3; ++a) {
        uint64_t counter = (((uint64_t)step * (uint64_t)d->nz + (uint64_t)z) * (uint64_t)d->ny + (uint64_t)y) * 3u + (uint64_t)a;
        double xi = uniform_pm1(or_splitmix64(d->seed, counter + 1));
        u[a] = d->u_ref[a] * scale + d->noise_rel * U0 * xi;
    }
}

static size_t cell_index(const or_domain* d, int x, int y, int z)
{
    return ((size_t)z * d->ny + y) * d->nx + x;
}

/*
 * Pull streaming with boundary rules (Sec. 2.1 streaming step; boundary rules
 * are a reading): the pre-collision population q of cell x is the
 * post-collision population q of cell x - c_q, except
 *   - no-slip axis, source outside [0, N): halfway bounce-back, the cell's own
 *     post-collision population of the opposite direction;
 *   - free-slip axis, source outside [0, N): specular reflection, the
 *     post-collision population of the mirrored direction (that velocity
 *     component negated) at the source moved back onto the cell's own index
 *     along that axis (the other components still shift);
 *   - periodic axis: the source index wraps;
 *   - x inflow (source x < 0): equilibrium at rho = 1 and the inflow velocity
 *     of the source column at this step (of the mirrored direction, after a
 *     free-slip reflection);
 *   - x outflow (source x >= nx): zero-gradient, the source is moved to the
 *     last plane x = nx-1.
 * The rules apply in this order: no-slip, free-slip, periodic wrap, x in/out.
 */
void or_pull_cell(const or_domain* d, const double* fsrc, long step, int x, int y, int z, double out[NQ])
{
    size_t N = (size_t)d->nx * d->ny * d->nz;
    int n[3] = {d->nx, d->ny, d->nz};
    int p[3] = {x, y, z};
    for (int q = 0; q < NQ; ++q) {
        int c[3] = {cx_of(q), cy_of(q), cz_of(q)};
        int s[3];
        int wall = 0;
        for (int a = 0; a < 3; ++a) {
            s[a] = p[a] - c[a];
            if (d->bc[a] == OR_BC_NOSLIP && (s[a] < 0 || s[a] >= n[a])) wall = 1;
        }
        if (wall) {
            out[q] = fsrc[(size_t)opp_of(q) * N + cell_index(d, x, y, z)];
            continue;
        }
        int cm[3] = {c[0], c[1], c[2]}; /* direction whose population is read */
        for (int a = 0; a < 3; ++a)
            if (d->bc[a] == OR_BC_FREESLIP && (s[a] < 0 || s[a] >= n[a])) {
                cm[a] = -c[a];
                s[a] = p[a];
            }
        int qm = (cm[2] + 1) * 9 + (cm[1] + 1) * 3 + (cm[0] + 1);
        for (int a = 0; a < 3; ++a)
            if (d->bc[a] == OR_BC_PERIODIC) s[a] = ((s[a] % n[a]) + n[a]) % n[a];
        if (d->bc[0] == OR_BC_INOUT) {
            if (s[0] < 0) {
                double uin[3], feq[NQ];
                or_inflow_velocity(d, step, s[1], s[2], uin);
                or_equilibrium(1.0, uin, feq);
                out[q] = feq[qm];
                continue;
            }
            if (s[0] >= n[0]) s[0] = n[0] - 1;
        }
        out[q] = fsrc[(size_t)qm * N + cell_index(d, s[0], s[1], s[2])];
    }
}

static void collide(const or_domain* d, const double f[NQ], const double F[3], double out[NQ])
{
    if (d->collision == OR_COLL_CUMULANT) {
        double rates[10];
        rates[0] = or_omega_from_nu(d->nu);
        for (int i = 1; i < 10; ++i) rates[i] = 1.0; /* bulk and higher orders: full relaxation */
        or_collide_cumulant(f, F, rates, out);
    } else {
        or_collide_srt_smag(f, F, d->nu, d->smag_c, out);
    }
}

/* ------------------------------------------------------------------------ */
/* Actuator line                                                             */
/* ------------------------------------------------------------------------ */

typedef struct {
    double hub[3];
    double radius;
    int n_blades, n_elements;
    double epsilon;
    double omega;             /* rotor speed, rad per step, about +axis */
    double yaw, pitch, theta0;
    double chord_root, chord_tip;
    const double* twist;      /* n_elements or NULL */
    int n_polar;
    const double* alpha;      /* ascending, radians */
    const double* cl;
    const double* cd;
    int kernel;               /* OR_KERNEL_GAUSS or OR_KERNEL_ROMA */
    int tip_loss;             /* 1: Glauert tip-loss factor on the element forces */
} or_turbine;

enum { OR_KERNEL_GAUSS = 0, OR_KERNEL_ROMA = 1 };

static void matmul3(const double A[3][3], const double B[3][3], double C[3][3])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += A[i][k] * B[k][j];
            C[i][j] = s;
        }
}

static void matvec3(const double A[3][3], const double v[3], double r[3])
{
    for (int i = 0; i < 3; ++i) r[i] = A[i][0] * v[0] + A[i][1] * v[1] + A[i][2] * v[2];
}

static void rot_x(double t, double R[3][3])
{
    double c = cos(t), s = sin(t);
    double M[3][3] = {{1, 0, 0}, {0, c, -s}, {0, s, c}};
    memcpy(R, M, sizeof M);
}

static void rot_z(double t, double R[3][3])
{
    double c = cos(t), s = sin(t);
    double M[3][3] = {{c, -s, 0}, {s, c, 0}, {0, 0, 1}};
    memcpy(R, M, sizeof M);
}

/*
 * Blade-line kinematics following Algorithm 2 (Line::update) for the flat
 * hub -> blade topology: the hub frame T_p is the yaw rotation about z, the
 * blade's fixed offset T_r is a rotation by 2 pi b / B about the rotor axis
 * (local x), and R is the rotation by theta0 + omega * n about the same axis.
 * Element k sits at p = hub + T_c (0, r_k, 0) with r_k = (k + 1/2) R / N_e.
 * Its velocity is omega e_axis x (p - hub).  Outputs: position, velocity, the
 * axis, radial and tangential unit vectors (e_t = e_axis x e_r) and r_k.
 */
void or_element_kinematics(const or_turbine* t, long step, int b, int k,
                           double pos[3], double vel[3], double e_axis[3], double e_r[3], double e_t[3], double* r_out)
{
    double Tp[3][3], Tr[3][3], R[3][3], tmp[3][3], Tc[3][3];
    rot_z(t->yaw, Tp);
    rot_x(2.0 * M_PI * b / t->n_blades, Tr);
    double theta = t->theta0 + t->omega * (double)step;
    rot_x(theta, R);
    matmul3(Tp, Tr, tmp);
    matmul3(tmp, R, Tc);
    double r = (k + 0.5) * t->radius / t->n_elements;
    double local[3] = {0, r, 0}, rel[3];
    matvec3(Tc, local, rel);
    double ex[3] = {1, 0, 0}, ey[3] = {0, 1, 0}, ez[3] = {0, 0, 1};
    double er[3], ea[3], et[3];
    matvec3(Tc, ey, er);
    matvec3(Tc, ex, ea);
    matvec3(Tc, ez, et); /* Tc e_z = Tc (e_x x e_y) = e_axis x e_r for a rotation */
    for (int a = 0; a < 3; ++a) {
        pos[a] = t->hub[a] + rel[a];
        e_axis[a] = ea[a];
        e_r[a] = er[a];
        e_t[a] = et[a];
    }
    double w[3] = {t->omega * ea[0], t->omega * ea[1], t->omega * ea[2]};
    vel[0] = w[1] * rel[2] - w[2] * rel[1];
    vel[1] = w[2] * rel[0] - w[0] * rel[2];
    vel[2] = w[0] * rel[1] - w[1] * rel[0];
    *r_out = r;
}

/* Linear interpolation in an ascending table, clamped at both ends. */
double or_table_lookup(const double* xs, const double* ys, int n, double x)
{
    if (x <= xs[0]) return ys[0];
    if (x >= xs[n - 1]) return ys[n - 1];
    for (int i = 0; i + 1 < n; ++i) {
        if (x >= xs[i] && x <= xs[i + 1]) {
            double t = (x - xs[i]) / (xs[i + 1] - xs[i]);
            return ys[i] + t * (ys[i + 1] - ys[i]);
        }
    }
    return ys[n - 1];
}

/*
 * Trilinear interpolation of rho and u at point p (Sec. 2.2).  At each of the
 * eight surrounding cells the pre-collision populations are pulled from the
 * current array (with boundary rules) and rho, u = (sum c f + F/2)/rho are
 * formed with the force field of the previous step; then rho and u are blended
 * with the trilinear weights.
 */
void or_sample(const or_domain* d, const double* fsrc, const double* force_prev, long step,
               const double p[3], double* rho_out, double u_out[3])
{
    size_t N = (size_t)d->nx * d->ny * d->nz;
    int n[3] = {d->nx, d->ny, d->nz};
    int i0[3];
    double t[3];
    for (int a = 0; a < 3; ++a) {
        i0[a] = (int)floor(p[a]);
        t[a] = p[a] - i0[a];
    }
    double rho = 0, u[3] = {0, 0, 0};
    for (int corner = 0; corner < 8; ++corner) {
        int o[3] = {corner & 1, (corner >> 1) & 1, (corner >> 2) & 1};
        int cpos[3];
        double wgt = 1.0;
        for (int a = 0; a < 3; ++a) {
            cpos[a] = i0[a] + o[a];
            if (d->bc[a] == OR_BC_PERIODIC) cpos[a] = ((cpos[a] % n[a]) + n[a]) % n[a];
            else if (cpos[a] < 0) cpos[a] = 0;
            else if (cpos[a] >= n[a]) cpos[a] = n[a] - 1;
            wgt *= o[a] ? t[a] : 1.0 - t[a];
        }
        double f[NQ];
        or_pull_cell(d, fsrc, step, cpos[0], cpos[1], cpos[2], f);
        size_t ci = cell_index(d, cpos[0], cpos[1], cpos[2]);
        double F[3];
        for (int a = 0; a < 3; ++a) F[a] = d->body_force[a] + (force_prev ? force_prev[(size_t)a * N + ci] : 0.0);
        double r, uc[3];
        or_macroscopic(f, F, &r, uc);
        rho += wgt * r;
        for (int a = 0; a < 3; ++a) u[a] += wgt * uc[a];
    }
    *rho_out = rho;
    for (int a = 0; a < 3; ++a) u_out[a] = u[a];
}

/*
 * Glauert's tip-loss factor (Sec. 2.2 names tip-loss models as an option of
 * the actuator line; the validation of Sec. 5 turns the Glauert type off),
 * in Prandtl's form: for B blades of radius R, an element at radius r and
 * inflow angle phi,
 *   F = (2/pi) arccos(exp(-B (R - r) / (2 r |sin phi|))),
 * the factor on the element force.  F -> 1 as sin phi -> 0 (the exponent's
 * limit), and F = 0 at the tip.
 */
double or_tip_loss(int n_blades, double R, double r, double phi)
{
    double s = fabs(sin(phi));
    if (s == 0.0) return 1.0;
    double f = n_blades * (R - r) / (2.0 * r * s);
    return 2.0 / M_PI * acos(exp(-f));
}

/*
 * Blade-element forces (Sec. 2.2): with u sampled at the element, the
 * relative velocity u_rel = u - v has its radial part removed; the inflow
 * angle is phi = atan2(u_rel.e_axis, -u_rel.e_t) and alpha = phi - twist -
 * pitch.  C_L, C_D come from the tables; e_D = u_rel/|u_rel|, e_L = e_D x e_r;
 * F_blade = 1/2 rho |u_rel|^2 c l (C_L e_L + C_D e_D) with chord c(r) varying
 * linearly from root to tip and l = R / N_e.  The force on the fluid is
 * -F_blade.  With the tip-loss option F_blade is scaled by or_tip_loss.
 * Thrust = sum F_blade . e_axis, torque = sum ((p-hub) x F_blade) . e_axis.
 * Outputs per element (blade-major): pos, F_blade, alpha, and the two rotor
 * loads.
 */
void or_alm_forces(const or_domain* d, const or_turbine* t, const double* fsrc, const double* force_prev, long step,
                   double* pos_out, double* force_out, double* alpha_out, double loads[2])
{
    double thrust = 0, torque = 0;
    double len = t->radius / t->n_elements;
    for (int b = 0; b < t->n_blades; ++b) {
        for (int k = 0; k < t->n_elements; ++k) {
            int e = b * t->n_elements + k;
            double p[3], v[3], ea[3], er[3], et[3], r;
            or_element_kinematics(t, step, b, k, p, v, ea, er, et, &r);
            double rho, u[3];
            or_sample(d, fsrc, force_prev, step, p, &rho, u);
            double ur[3];
            for (int a = 0; a < 3; ++a) ur[a] = u[a] - v[a];
            double urad = ur[0] * er[0] + ur[1] * er[1] + ur[2] * er[2];
            for (int a = 0; a < 3; ++a) ur[a] -= urad * er[a];
            double uax = ur[0] * ea[0] + ur[1] * ea[1] + ur[2] * ea[2];
            double utan = ur[0] * et[0] + ur[1] * et[1] + ur[2] * et[2];
            double phi = atan2(uax, -utan);
            double twist = t->twist ? t->twist[k] : 0.0;
            double alpha = phi - twist - t->pitch;
            double CL = or_table_lookup(t->alpha, t->cl, t->n_polar, alpha);
            double CD = or_table_lookup(t->alpha, t->cd, t->n_polar, alpha);
            double chord = t->chord_root + (t->chord_tip - t->chord_root) * r / t->radius;
            double mag2 = ur[0] * ur[0] + ur[1] * ur[1] + ur[2] * ur[2];
            double Fb[3] = {0, 0, 0};
            if (mag2 > 0) {
                double mag = sqrt(mag2);
                double eD[3] = {ur[0] / mag, ur[1] / mag, ur[2] / mag};
                double eL[3] = {eD[1] * er[2] - eD[2] * er[1], eD[2] * er[0] - eD[0] * er[2], eD[0] * er[1] - eD[1] * er[0]};
                double s = 0.5 * rho * mag2 * chord * len;
                if (t->tip_loss) s *= or_tip_loss(t->n_blades, t->radius, r, phi);
                for (int a = 0; a < 3; ++a) Fb[a] = s * (CL * eL[a] + CD * eD[a]);
            }
            double rel[3] = {p[0] - t->hub[0], p[1] - t->hub[1], p[2] - t->hub[2]};
            double mom[3] = {rel[1] * Fb[2] - rel[2] * Fb[1], rel[2] * Fb[0] - rel[0] * Fb[2], rel[0] * Fb[1] - rel[1] * Fb[0]};
            thrust += Fb[0] * ea[0] + Fb[1] * ea[1] + Fb[2] * ea[2];
            torque += mom[0] * ea[0] + mom[1] * ea[1] + mom[2] * ea[2];
            if (pos_out) for (int a = 0; a < 3; ++a) pos_out[3 * e + a] = p[a];
            if (force_out) for (int a = 0; a < 3; ++a) force_out[3 * e + a] = Fb[a];
            if (alpha_out) alpha_out[e] = alpha;
        }
    }
    loads[0] = thrust;
    loads[1] = torque;
}

/*
 * Gaussian force regularisation f_eps = f (x) eta_eps (Sec. 2.2), reading:
 * eta_eps(d) = prod_a g(d_a) with g(s) = exp(-s^2/eps^2)/(eps sqrt(pi)) for
 * |s| <= 3 eps and 0 beyond; each axis factor is renormalised so that its sum
 * over the integer lattice points is exactly 1, which makes the spread force
 * of every element sum to the element force.  Weight of cell x:
 * prod_a g(x_a - p_a) / sum_i g(i - p_a).
 */
double or_gauss_axis_sum(double p, double eps)
{
    int lo = (int)ceil(p - 3.0 * eps), hi = (int)floor(p + 3.0 * eps);
    double s = 0;
    for (int i = lo; i <= hi; ++i) {
        double dd = i - p;
        s += exp(-dd * dd / (eps * eps)) / (eps * sqrt(M_PI));
    }
    return s;
}

/*
 * The discrete delta of Roma, Peskin and Berger (1999), which Sec. 2.2 uses
 * for the spreading: the three-point function
 *   phi(r) = (1 + sqrt(1 - 3 r^2)) / 3                  for |r| <= 1/2,
 *   phi(r) = (5 - 3 |r| - sqrt(1 - 3 (1 - |r|)^2)) / 6   for 1/2 <= |r| <= 3/2,
 *   phi(r) = 0                                           beyond,
 * built so that its samples at the integers shifted by any r sum to 1, have
 * zero first moment and squares summing to 1/2.  The 3-D weight of cell x is
 * prod_a phi(x_a - p_a); it needs no renormalisation (the conservation Sec. 2.2
 * notes) and epsilon plays no part.
 */
double or_roma_phi(double r)
{
    double a = fabs(r);
    if (a <= 0.5) return (1.0 + sqrt(1.0 - 3.0 * a * a)) / 3.0;
    if (a <= 1.5) return (5.0 - 3.0 * a - sqrt(1.0 - 3.0 * (1.0 - a) * (1.0 - a))) / 6.0;
    return 0.0;
}

/* Per-axis support [lo, hi] of an element at p: |i - p| <= 3 eps (Gaussian)
 * or <= 3/2 (Roma). */
static void support_1d(int kernel, double p, double eps, int* lo, int* hi)
{
    double cut = kernel == OR_KERNEL_ROMA ? 1.5 : 3.0 * eps;
    *lo = (int)ceil(p - cut);
    *hi = (int)floor(p + cut);
}

/* Normaliser of an element at p: the product of the Gaussian's axis sums
 * (1 for Roma). */
static double reg_norm(int kernel, const double p[3], double eps)
{
    if (kernel == OR_KERNEL_ROMA) return 1.0;
    return or_gauss_axis_sum(p[0], eps) * or_gauss_axis_sum(p[1], eps) * or_gauss_axis_sum(p[2], eps);
}

/* Regularisation weight of cell c for an element at p with normaliser S. */
static double reg_weight(int kernel, const double p[3], double eps, double S, const int c[3])
{
    double d[3] = {c[0] - p[0], c[1] - p[1], c[2] - p[2]};
    if (kernel == OR_KERNEL_ROMA) return or_roma_phi(d[0]) * or_roma_phi(d[1]) * or_roma_phi(d[2]);
    double g = 1.0 / (eps * eps * eps * M_PI * sqrt(M_PI));
    return g * exp(-(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) / (eps * eps)) / S;
}

/* Adds -F_k * weight(x) of every element, in element order, to force[3][N].
 * The whole support of every element must lie inside the domain. */
void or_spread(const or_domain* d, const double* pos, const double* fblade, int n_el, double eps, int kernel,
               double* force)
{
    size_t N = (size_t)d->nx * d->ny * d->nz;
    for (int e = 0; e < n_el; ++e) {
        const double* p = pos + 3 * e;
        int lo[3], hi[3], c[3];
        for (int a = 0; a < 3; ++a) support_1d(kernel, p[a], eps, lo + a, hi + a);
        double S = reg_norm(kernel, p, eps);
        for (c[2] = lo[2]; c[2] <= hi[2]; ++c[2])
            for (c[1] = lo[1]; c[1] <= hi[1]; ++c[1])
                for (c[0] = lo[0]; c[0] <= hi[0]; ++c[0]) {
                    double wgt = reg_weight(kernel, p, eps, S, c);
                    size_t ci = cell_index(d, c[0], c[1], c[2]);
                    for (int a = 0; a < 3; ++a) force[(size_t)a * N + ci] += -fblade[3 * e + a] * wgt;
                }
    }
}

/* Spread force at one cell (x, y, z): the same sum as or_spread, restricted to
 * a single cell, in element order. */
void or_spread_at(const double* pos, const double* fblade, int n_el, double eps, int kernel, int x, int y, int z,
                  double out[3])
{
    out[0] = out[1] = out[2] = 0;
    int c[3] = {x, y, z};
    for (int e = 0; e < n_el; ++e) {
        const double* p = pos + 3 * e;
        int inside = 1;
        for (int a = 0; a < 3; ++a) {
            int lo, hi;
            support_1d(kernel, p[a], eps, &lo, &hi);
            if (c[a] < lo || c[a] > hi) inside = 0;
        }
        if (!inside) continue;
        double wgt = reg_weight(kernel, p, eps, reg_norm(kernel, p, eps), c);
        for (int a = 0; a < 3; ++a) out[a] += -fblade[3 * e + a] * wgt;
    }
}

/* ------------------------------------------------------------------------ */
/* One time step                                                             */
/* ------------------------------------------------------------------------ */

/*
 * Step n -> n+1 in the order of the coupled scheme:
 *  1. blade kinematics at t = n;
 *  2. sample rho, u at every element from the current array (force of the
 *     previous step in the half shift);
 *  3. element forces and FP64 rotor loads;
 *  4. spread -F of every element into the ALM force field falm_out;
 *  5. pull streaming with boundary rules (inflow noise of step n);
 *  6. collision with F = body force + falm_out;
 *  7. store into fdst.
 * falm_prev: ALM force field of the previous step (NULL = zero).  loads:
 * 2 doubles per turbine.  elem_pos / elem_force: 3 doubles per element,
 * turbines in order (may be NULL).  Steps 5-7 run on planes z_begin .. z_end-1
 * only (a bounded sample for CPU timing); or_step runs all planes.
 */
void or_step_planes(const or_domain* d, const or_turbine* turbs, int n_turb, const double* fsrc, double* fdst,
                    const double* falm_prev, double* falm_out, long step, double* loads, double* elem_pos,
                    double* elem_force, int z_begin, int z_end)
{
    build_partition_terms();
    size_t N = (size_t)d->nx * d->ny * d->nz;
    memset(falm_out, 0, sizeof(double) * 3 * N);
    int off = 0;
    for (int ti = 0; ti < n_turb; ++ti) {
        const or_turbine* t = turbs + ti;
        int ne = t->n_blades * t->n_elements;
        double* pos = (double*)malloc(sizeof(double) * 3 * ne);
        double* fb = (double*)malloc(sizeof(double) * 3 * ne);
        or_alm_forces(d, t, fsrc, falm_prev, step, pos, fb, NULL, loads + 2 * ti);
        or_spread(d, pos, fb, ne, t->epsilon, t->kernel, falm_out);
        if (elem_pos) memcpy(elem_pos + 3 * off, pos, sizeof(double) * 3 * ne);
        if (elem_force) memcpy(elem_force + 3 * off, fb, sizeof(double) * 3 * ne);
        off += ne;
        free(pos);
        free(fb);
    }
#pragma omp parallel for schedule(static)
    for (int z = z_begin; z < z_end; ++z) {
        for (int y = 0; y < d->ny; ++y) {
            for (int x = 0; x < d->nx; ++x) {
                double f[NQ], fo[NQ], F[3];
                size_t ci = cell_index(d, x, y, z);
                or_pull_cell(d, fsrc, step, x, y, z, f);
                for (int a = 0; a < 3; ++a) F[a] = d->body_force[a] + falm_out[(size_t)a * N + ci];
                collide(d, f, F, fo);
                for (int q = 0; q < NQ; ++q) fdst[(size_t)q * N + ci] = fo[q];
            }
        }
    }
}

/* The whole lattice (planes 0 .. nz-1). */
void or_step(const or_domain* d, const or_turbine* turbs, int n_turb, const double* fsrc, double* fdst,
             const double* falm_prev, double* falm_out, long step, double* loads, double* elem_pos, double* elem_force)
{
    or_step_planes(d, turbs, n_turb, fsrc, fdst, falm_prev, falm_out, step, loads, elem_pos, elem_force, 0, d->nz);
}

/* Post-collision update of a single cell (pull + collide) for sampled checks. */
void or_update_cell(const or_domain* d, const double* fsrc, const double F[3], long step, int x, int y, int z, double out[NQ])
{
    build_partition_terms();
    double f[NQ];
    or_pull_cell(d, fsrc, step, x, y, z, f);
    collide(d, f, F, out);
}

/* Moments of a stored post-collision field: rho = sum f*, and, since the
 * collision adds F to the momentum, u = (sum c f* - F/2)/rho, which is the
 * velocity the last collision used.  F = body force + falm (falm may be NULL). */
void or_moments(const or_domain* d, const double* f, const double* falm, double* rho_out, double* u_out)
{
    size_t N = (size_t)d->nx * d->ny * d->nz;
#pragma omp parallel for schedule(static)
    for (long long ci = 0; ci < (long long)N; ++ci) {
        double r = 0, j[3] = {0, 0, 0};
        for (int q = 0; q < NQ; ++q) {
            double v = f[(size_t)q * N + ci];
            r += v;
            j[0] += cx_of(q) * v;
            j[1] += cy_of(q) * v;
            j[2] += cz_of(q) * v;
        }
        rho_out[ci] = r;
        for (int a = 0; a < 3; ++a) {
            double F = d->body_force[a] + (falm ? falm[(size_t)a * N + ci] : 0.0);
            u_out[(size_t)a * N + ci] = (j[a] - 0.5 * F) / r;
        }
    }
}

/* f = feq(rho, u) + fneq at every cell, the product-form equilibrium.
 * rho: N values; u: 3 planes; fneq: 27 planes or NULL. */
void or_init_fields(const or_domain* d, const double* rho, const double* u, const float* fneq, double* f)
{
    size_t N = (size_t)d->nx * d->ny * d->nz;
#pragma omp parallel for schedule(static)
    for (long long ci = 0; ci < (long long)N; ++ci) {
        double uu[3] = {u[ci], u[N + ci], u[2 * N + ci]}, feq[NQ];
        or_equilibrium(rho[ci], uu, feq);
        for (int q = 0; q < NQ; ++q) f[(size_t)q * N + ci] = feq[q] + (fneq ? (double)fneq[(size_t)q * N + ci] : 0.0);
    }
}
