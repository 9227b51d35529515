/*
 * skyrme_oracle.c -- plain FP64 CPU reference of the arrested Newton flow of
 * the Skyrme model in sigma-model form (arXiv 2604.25876).
 *
 * TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's
 * CPU-baseline leg are its only users.  It is deliberately slow and literal:
 * every formula is written the way the paper states it (nested sums, explicit
 * Levi-Civita symbols), with no blocking, fusion or reordering.  Summations
 * over the lattice are Neumaier-compensated per x-plane and then over planes,
 * so the result does not depend on the number of OpenMP threads.
 *
 * Paper passages followed:
 *   Section 2.1, Eq. "SkyrmeEnergy_phi"   energy density (e2, e4, e0)
 *   Section 2.1, Eq. "B0_components"      baryon density
 *   Section 3,   Eq. "Newton_flow"        second-order flow with projection
 *   Section 3,   Eq. "Sigma model EL equations"  dE/dphi^A
 *   Section 3,   first/second-derivative 4th-order stencils
 *   Section 3,   arrest rule, normalisation after each update, vacuum box
 *   Section 4.1  rational-map ansatz, Table 1 (the B = 1 to 4 maps; the
 *                degree-3 constant a, given by reference only, is i: the
 *                tetrahedral map)
 *   Section 4.2  product ansatz, Eq. "Product ansatz"
 *   Section 5.6  virial V = integral of T_kk
 *   Section 7.8  extension models: the modified-pion, loosely and lightly
 *                bound potentials and the BPS sextic term
 *
 * Readings where the paper is silent or ambiguous (each is a choice the CUDA
 * library makes the same way):
 *   - mixed derivative d_i d_j: tensor product of the first-derivative
 *     stencil along i and along j (16 taps, radius 2);
 *   - baryon density sign: B0 = -(1/12 pi^2) eps^{ijk} eps_{ABCD} phi^A
 *     d_i phi^B d_j phi^C d_k phi^D with eps_{0123} = +1, so that the
 *     hedgehog with f(0) = pi and the R(z) = z map has B = +1 as Table 1
 *     states;
 *   - the arrest compares the static energy of phi_n with that of phi_{n-1}
 *     (strictly larger => velocity zeroed), the field is kept, and the update
 *     is symplectic Euler: v += dt F, phi = normalise(phi + dt v);
 *   - energies are h^3 times the sum over interior sites;
 *   - delta is the largest |F| over interior sites;
 *   - virial V = -E2 + E4 - 3 E0 (Derrick scaling of the three terms, which
 *     equals the integral of T_kk of Eq. "Stress tensor" for static fields);
 *     with the sextic term V = -E2 + E4 - 3 E0 + 3 E6 (E6 scales as lambda^3);
 *   - the sextic term's c6 4 pi^4 (B0)^2 enters the static energy density
 *     with a plus sign (a static energy bounded below for c6 >= 0), and the
 *     flow sees only its static energy (the flow's kinetic term is the plain
 *     sum of squared velocities);
 *   - E0 is the sum of all four potentials.
 */
#include "skyrme_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static size_t site_index(const int n[3], int x, int y, int z)
{
    return (((size_t)x * (size_t)n[1]) + (size_t)y) * (size_t)n[2] + (size_t)z;
}

static int is_interior(const int n[3], int x, int y, int z)
{
    return x >= 2 && x <= n[0] - 3 && y >= 2 && y <= n[1] - 3 && z >= 2 &&
           z <= n[2] - 3;
}

/* Neumaier (improved Kahan) running sum. */
typedef struct { double s, c; } nsum;
static void nsum_add(nsum *a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v))
        a->c += (a->s - t) + v;
    else
        a->c += (v - t) + a->s;
    a->s = t;
}
static double nsum_get(const nsum *a) { return a->s + a->c; }

/* ------------------------------------------------------------------------
 * Section 3: fourth-order stencils, weights for offsets -2, -1, 0, +1, +2.
 *   d_x phi_i   ~ ( phi_{i-2}/12 - 2 phi_{i-1}/3 + 2 phi_{i+1}/3 - phi_{i+2}/12 ) / h
 *   d_xx phi_i  ~ ( -phi_{i-2}/12 + 4 phi_{i-1}/3 - 5 phi_i/2 + 4 phi_{i+1}/3
 *                   - phi_{i+2}/12 ) / h^2
 * ------------------------------------------------------------------------ */
static const double FIRST[5] = {1.0 / 12.0, -2.0 / 3.0, 0.0, 2.0 / 3.0,
                                -1.0 / 12.0};
static const double SECOND[5] = {-1.0 / 12.0, 4.0 / 3.0, -5.0 / 2.0, 4.0 / 3.0,
                                 -1.0 / 12.0};

void orc_site_derivatives(const int n[3], double h, const double *phi, int x,
                          int y, int z, double d1[3][4], double d2[3][4],
                          double dm[3][4])
{
    const int unit[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    const int pair[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    int i, A, k, l, p;

    for (i = 0; i < 3; i++) {
        for (A = 0; A < 4; A++) {
            double s1 = 0.0, s2 = 0.0;
            for (k = 0; k < 5; k++) {
                int o = k - 2;
                size_t s = site_index(n, x + o * unit[i][0], y + o * unit[i][1],
                                      z + o * unit[i][2]);
                s1 += FIRST[k] * phi[4 * s + A];
                s2 += SECOND[k] * phi[4 * s + A];
            }
            d1[i][A] = s1 / h;
            d2[i][A] = s2 / (h * h);
        }
    }
    /* mixed derivative: first-derivative stencil along i applied to the
     * first-derivative stencil along j (16 taps). */
    for (p = 0; p < 3; p++) {
        int a = pair[p][0], b = pair[p][1];
        for (A = 0; A < 4; A++) {
            double s = 0.0;
            for (k = 0; k < 5; k++) {
                for (l = 0; l < 5; l++) {
                    int oa = k - 2, ob = l - 2;
                    size_t q;
                    if (FIRST[k] == 0.0 || FIRST[l] == 0.0) continue;
                    q = site_index(n, x + oa * unit[a][0] + ob * unit[b][0],
                                   y + oa * unit[a][1] + ob * unit[b][1],
                                   z + oa * unit[a][2] + ob * unit[b][2]);
                    s += FIRST[k] * FIRST[l] * phi[4 * q + A];
                }
            }
            dm[p][A] = s / (h * h);
        }
    }
}

/* Levi-Civita symbols as explicit permutation lists. */
static int perm_sign(const int *p, int len)
{
    int s = 1, i, j;
    for (i = 0; i < len; i++)
        for (j = i + 1; j < len; j++)
            if (p[i] > p[j]) s = -s;
    return s;
}

/* Levi-Civita symbol eps_{abcd} with eps_{0123} = +1 (0 for a repeated index). */
static int levi4(int a, int b, int c, int d)
{
    int p[4];
    if (a == b || a == c || a == d || b == c || b == d || c == d) return 0;
    p[0] = a;
    p[1] = b;
    p[2] = c;
    p[3] = d;
    return perm_sign(p, 4);
}

/* Section 7.8, BPS sextic term.  With the rows R_0 = phi, R_1 = d_x phi,
 * R_2 = d_y phi, R_3 = d_z phi and D = eps_{ABCD} R_0^A R_1^B R_2^C R_3^D,
 * B0 = -D / (2 pi^2), so the static density c6 4 pi^4 (B0)^2 is c6 D^2.  Its
 * Euler-Lagrange gradient, written out by the chain rule:
 *   G6_A = d(c6 D^2)/dphi^A - d_i [ d(c6 D^2)/d(d_i phi^A) ]
 *        = 2 c6 [ D C_0^A - sum_i ( (d_i D) C_{1+i}^A + D d_i C_{1+i}^A ) ]
 * with the cofactors C_r^A = dD/dR_r^A, d_i D = sum_r C_r . d_i R_r and
 * d_i C_r^A = sum_{s != r} (d^2 D / dR_r^A dR_s^B) d_i R_s^B, where
 * d_i R_0 = d_i phi and d_i R_{1+j} = d_i d_j phi (H[i][j]). */
static void sextic_gradient(const double phi[4], const double d1[3][4],
                            const double H[3][3][4], double c6, double G6[4])
{
    const double *R[4];
    double dR[3][4][4];       /* dR[i][r][A] = d_i R_r^A */
    double C[4][4];           /* dD / dR_r^A */
    double C2[4][4][4][4];    /* d^2 D / dR_r^A dR_s^B, r != s */
    double D = 0.0, dD[3], dC[3][4][4];
    int idx[4], i, r, s, A, B, k;

    R[0] = phi;
    R[1] = d1[0];
    R[2] = d1[1];
    R[3] = d1[2];
    memset(C, 0, sizeof(C));
    memset(C2, 0, sizeof(C2));
    for (idx[0] = 0; idx[0] < 4; idx[0]++)
        for (idx[1] = 0; idx[1] < 4; idx[1]++)
            for (idx[2] = 0; idx[2] < 4; idx[2]++)
                for (idx[3] = 0; idx[3] < 4; idx[3]++) {
                    const int e = levi4(idx[0], idx[1], idx[2], idx[3]);
                    if (e == 0) continue;
                    D += e * R[0][idx[0]] * R[1][idx[1]] * R[2][idx[2]] * R[3][idx[3]];
                    for (r = 0; r < 4; r++) {
                        double prod = e;
                        for (k = 0; k < 4; k++)
                            if (k != r) prod *= R[k][idx[k]];
                        C[r][idx[r]] += prod;
                        for (s = 0; s < 4; s++) {
                            double p2 = e;
                            if (s == r) continue;
                            for (k = 0; k < 4; k++)
                                if (k != r && k != s) p2 *= R[k][idx[k]];
                            C2[r][s][idx[r]][idx[s]] += p2;
                        }
                    }
                }
    for (i = 0; i < 3; i++)
        for (A = 0; A < 4; A++) {
            dR[i][0][A] = d1[i][A];
            for (r = 1; r < 4; r++) dR[i][r][A] = H[i][r - 1][A];
        }
    for (i = 0; i < 3; i++) {
        dD[i] = 0.0;
        for (r = 0; r < 4; r++)
            for (A = 0; A < 4; A++) dD[i] += C[r][A] * dR[i][r][A];
        for (r = 0; r < 4; r++)
            for (A = 0; A < 4; A++) {
                double t = 0.0;
                for (s = 0; s < 4; s++) {
                    if (s == r) continue;
                    for (B = 0; B < 4; B++) t += C2[r][s][A][B] * dR[i][s][B];
                }
                dC[i][r][A] = t;
            }
    }
    for (A = 0; A < 4; A++) {
        double div = 0.0;
        for (i = 0; i < 3; i++) div += dD[i] * C[1 + i][A] + D * dC[i][1 + i][A];
        G6[A] = 2.0 * c6 * (D * C[0][A] - div);
    }
}

void orc_site_terms(const double phi[4], const double d1[3][4],
                    const double d2[3][4], const double dm[3][4], double m,
                    double G[4], double F[4], double dens[4])
{
    orc_model md;
    double d5[5];
    int q;
    md.mx = m;
    md.my = md.mz = md.mw = md.c6 = 0.0;
    orc_site_terms_model(phi, d1, d2, dm, &md, G, F, d5);
    for (q = 0; q < 4; q++) dens[q] = d5[q];
}

void orc_site_terms_model(const double phi[4], const double d1[3][4],
                          const double d2[3][4], const double dm[3][4],
                          const orc_model *md, double G[4], double F[4],
                          double dens[5])
{
    const double m = md->mx;
    double H[3][3][4]; /* d_i d_j phi^A */
    double a[3][3];    /* d_i phi . d_j phi */
    double tra, Gphi, sumsq;
    int i, j, k, A, B;

    for (A = 0; A < 4; A++) {
        H[0][0][A] = d2[0][A];
        H[1][1][A] = d2[1][A];
        H[2][2][A] = d2[2][A];
        H[0][1][A] = H[1][0][A] = dm[0][A];
        H[0][2][A] = H[2][0][A] = dm[1][A];
        H[1][2][A] = H[2][1][A] = dm[2][A];
    }
    for (i = 0; i < 3; i++)
        for (j = 0; j < 3; j++) {
            double s = 0.0;
            for (B = 0; B < 4; B++) s += d1[i][B] * d1[j][B];
            a[i][j] = s;
        }
    tra = a[0][0] + a[1][1] + a[2][2]; /* (d_j phi^B)^2 */

    /* Eq. "Sigma model EL equations":
     * dE/dphi^A = -2 { d_ii phi^A [1 + (d_j phi^B)^2]
     *                + d_i phi^A (d_ij phi^B d_j phi^B - d_jj phi^B d_i phi^B)
     *                - d_ij phi^A (d_i phi^B d_j phi^B) + m^2 delta^A_0 } */
    for (A = 0; A < 4; A++) {
        double t1 = 0.0, t2 = 0.0, t3 = 0.0;
        for (i = 0; i < 3; i++) t1 += H[i][i][A] * (1.0 + tra);
        for (i = 0; i < 3; i++) {
            double inner = 0.0;
            for (j = 0; j < 3; j++)
                for (B = 0; B < 4; B++)
                    inner += H[i][j][B] * d1[j][B] - H[j][j][B] * d1[i][B];
            t2 += d1[i][A] * inner;
        }
        for (i = 0; i < 3; i++)
            for (j = 0; j < 3; j++) t3 += H[i][j][A] * a[i][j];
        G[A] = -2.0 * (t1 + t2 - t3 + (A == 0 ? m * m : 0.0));
    }
    /* Section 7.8 potentials m_y^2 (1 - phi0^2) + m_z^2 (1 - phi0)^2
     * + (1/2) m_w^2 (1 - phi0)^4: their derivatives in phi^0 */
    {
        const double u = 1.0 - phi[0];
        G[0] += -2.0 * md->my * md->my * phi[0] - 2.0 * md->mz * md->mz * u
                - 2.0 * md->mw * md->mw * u * u * u;
    }
    if (md->c6 != 0.0) {
        double G6[4];
        sextic_gradient(phi, d1, (const double(*)[3][4])H, md->c6, G6);
        for (A = 0; A < 4; A++) G[A] += G6[A];
    }

    /* Eq. "Newton_flow": phi_tt^A = -dE/dphi^A + (dE/dphi^B phi^B) phi^A */
    Gphi = 0.0;
    for (B = 0; B < 4; B++) Gphi += G[B] * phi[B];
    for (A = 0; A < 4; A++) F[A] = -G[A] + Gphi * phi[A];

    /* Eq. "SkyrmeEnergy_phi" split into its three terms */
    sumsq = 0.0;
    for (i = 0; i < 3; i++)
        for (j = 0; j < 3; j++) sumsq += a[i][j] * a[i][j];
    dens[0] = tra;
    dens[1] = 0.5 * (tra * tra - sumsq);
    {
        const double u = 1.0 - phi[0];
        dens[2] = 2.0 * m * m * u + md->my * md->my * (1.0 - phi[0] * phi[0])
                  + md->mz * md->mz * u * u + 0.5 * md->mw * md->mw * u * u * u * u;
    }

    /* Eq. "B0_components" (sign reading in the file header) */
    {
        static const int p3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2},
                                     {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
        int p4[24][4], np4 = 0, q0, q1, q2, q3;
        double s = 0.0;
        for (q0 = 0; q0 < 4; q0++)
            for (q1 = 0; q1 < 4; q1++)
                for (q2 = 0; q2 < 4; q2++)
                    for (q3 = 0; q3 < 4; q3++)
                        if (q0 != q1 && q0 != q2 && q0 != q3 && q1 != q2 &&
                            q1 != q3 && q2 != q3) {
                            p4[np4][0] = q0;
                            p4[np4][1] = q1;
                            p4[np4][2] = q2;
                            p4[np4][3] = q3;
                            np4++;
                        }
        for (i = 0; i < 6; i++) {
            int e3 = perm_sign(p3[i], 3);
            for (k = 0; k < 24; k++) {
                int e4 = perm_sign(p4[k], 4);
                s += (double)(e3 * e4) * phi[p4[k][0]] * d1[p3[i][0]][p4[k][1]] *
                     d1[p3[i][1]][p4[k][2]] * d1[p3[i][2]][p4[k][3]];
            }
        }
        dens[3] = -s / (12.0 * M_PI * M_PI);
    }
    /* Section 7.8: c6 4 pi^4 (B0)^2 */
    dens[4] = md->c6 * 4.0 * M_PI * M_PI * M_PI * M_PI * dens[3] * dens[3];
}

/* ------------------------------------------------------------------------
 * whole-lattice passes
 * ------------------------------------------------------------------------ */
typedef struct {
    nsum e[5];
    double fmax;
    int bad;
} plane_acc;

/* Per-site work for one x-plane; writes G/F/dens (e2, e4, e0, b) when
 * requested and sums e2, e4, e0, b, e6. */
static void plane_pass(const int n[3], double h, const orc_model *md, const double *phi,
                       int x, double *G, double *F, double *dens,
                       plane_acc *acc)
{
    int y, z, q;
    memset(acc, 0, sizeof(*acc));
    for (y = 2; y <= n[1] - 3; y++)
        for (z = 2; z <= n[2] - 3; z++) {
            double d1[3][4], d2[3][4], dm[3][4], g[4], f[4], d[5], fn;
            size_t s = site_index(n, x, y, z);
            orc_site_derivatives(n, h, phi, x, y, z, d1, d2, dm);
            orc_site_terms_model(&phi[4 * s], d1, d2, dm, md, g, f, d);
            for (q = 0; q < 4; q++) {
                if (G) G[4 * s + q] = g[q];
                if (F) F[4 * s + q] = f[q];
                if (dens) dens[4 * s + q] = d[q];
                if (!isfinite(f[q]) || !isfinite(d[q])) acc->bad = 1;
            }
            for (q = 0; q < 5; q++) nsum_add(&acc->e[q], d[q]);
            fn = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2] + f[3] * f[3]);
            if (fn > acc->fmax) acc->fmax = fn;
        }
}

static void zero_boundary(const int n[3], double *arr)
{
    int x, y, z;
    if (!arr) return;
    for (x = 0; x < n[0]; x++)
        for (y = 0; y < n[1]; y++)
            for (z = 0; z < n[2]; z++)
                if (!is_interior(n, x, y, z))
                    memset(&arr[4 * site_index(n, x, y, z)], 0,
                           4 * sizeof(double));
}

/* Sum the per-plane accumulators in plane order: sums = {e2, e4, e0, b, e6}. */
static void lattice_pass(const int n[3], double h, const orc_model *md, const double *phi,
                         double *G, double *F, double *dens, double sums[5],
                         double *fmax, int *bad)
{
    int x, q;
    int nx = n[0];
    plane_acc *acc = (plane_acc *)calloc((size_t)nx, sizeof(plane_acc));
    nsum tot[5];
#pragma omp parallel for schedule(dynamic, 1)
    for (x = 2; x <= nx - 3; x++) plane_pass(n, h, md, phi, x, G, F, dens, &acc[x]);
    memset(tot, 0, sizeof(tot));
    *fmax = 0.0;
    *bad = 0;
    for (x = 2; x <= nx - 3; x++) {
        for (q = 0; q < 5; q++) nsum_add(&tot[q], nsum_get(&acc[x].e[q]));
        if (acc[x].fmax > *fmax) *fmax = acc[x].fmax;
        if (acc[x].bad) *bad = 1;
    }
    for (q = 0; q < 5; q++) sums[q] = nsum_get(&tot[q]);
    free(acc);
}

static orc_model standard_model(double m)
{
    orc_model md;
    md.mx = m;
    md.my = md.mz = md.mw = md.c6 = 0.0;
    return md;
}

void orc_forces_model(const int n[3], double h, const orc_model *md, const double *phi,
                      double *G, double *F, double *dens)
{
    double sums[5], fmax;
    int bad;
    zero_boundary(n, G);
    zero_boundary(n, F);
    zero_boundary(n, dens);
    lattice_pass(n, h, md, phi, G, F, dens, sums, &fmax, &bad);
}

void orc_forces(const int n[3], double h, double m, const double *phi,
                double *G, double *F, double *dens)
{
    const orc_model md = standard_model(m);
    orc_forces_model(n, h, &md, phi, G, F, dens);
}

void orc_energy_model(const int n[3], double h, const orc_model *md, const double *phi,
                      double out[7])
{
    double sums[5], fmax, h3 = h * h * h;
    int bad;
    lattice_pass(n, h, md, phi, NULL, NULL, NULL, sums, &fmax, &bad);
    out[1] = h3 * sums[0];
    out[2] = h3 * sums[1];
    out[3] = h3 * sums[2];
    out[4] = h3 * sums[4];
    out[0] = out[1] + out[2] + out[3] + out[4];
    out[5] = h3 * sums[3];
    out[6] = -out[1] + out[2] - 3.0 * out[3] + 3.0 * out[4];
}

void orc_energy(const int n[3], double h, double m, const double *phi,
                double out[6])
{
    const orc_model md = standard_model(m);
    double o7[7];
    orc_energy_model(n, h, &md, phi, o7);
    out[0] = o7[0];
    out[1] = o7[1];
    out[2] = o7[2];
    out[3] = o7[3];
    out[4] = o7[5];
    out[5] = o7[6];
}

int orc_anf_step_model(const int n[3], double h, const orc_model *md, double dt, int mode,
                       double *phi, double *v, double *work, double *E_prev,
                       orc_report *rep)
{
    double sums[5], fmax, h3 = h * h * h, E, E2, E4, E0, E6;
    int bad, arrested = 0, x;
    size_t nsite = (size_t)n[0] * n[1] * n[2];

    zero_boundary(n, work);
    lattice_pass(n, h, md, phi, NULL, work, NULL, sums, &fmax, &bad);
    E2 = h3 * sums[0];
    E4 = h3 * sums[1];
    E0 = h3 * sums[2];
    E6 = h3 * sums[4];
    E = E2 + E4 + E0 + E6;

    /* arrest: the static energy rose, so the fictitious velocity is zeroed
     * while the field is kept (Section 3). */
    if (mode == ORC_ARRESTED && E > *E_prev) {
        memset(v, 0, 4 * nsite * sizeof(double));
        arrested = 1;
    }

#pragma omp parallel for schedule(static)
    for (x = 2; x <= n[0] - 3; x++) {
        int y, z, q;
        for (y = 2; y <= n[1] - 3; y++)
            for (z = 2; z <= n[2] - 3; z++) {
                size_t s = site_index(n, x, y, z);
                double t[4], nrm = 0.0;
                for (q = 0; q < 4; q++) {
                    if (mode == ORC_GRADIENT) {
                        t[q] = phi[4 * s + q] + dt * work[4 * s + q];
                    } else {
                        v[4 * s + q] = v[4 * s + q] + dt * work[4 * s + q];
                        t[q] = phi[4 * s + q] + dt * v[4 * s + q];
                    }
                    nrm += t[q] * t[q];
                }
                nrm = sqrt(nrm);
                for (q = 0; q < 4; q++) phi[4 * s + q] = t[q] / nrm;
            }
    }

    *E_prev = E;
    if (rep) {
        rep->E = E;
        rep->E2 = E2;
        rep->E4 = E4;
        rep->E0 = E0;
        rep->B = h3 * sums[3];
        rep->virial = -E2 + E4 - 3.0 * E0 + 3.0 * E6;
        rep->delta = fmax;
        rep->arrested = arrested;
        rep->E6 = E6;
    }
    return (bad || !isfinite(E)) ? -1 : 0;
}

int orc_anf_step(const int n[3], double h, double m, double dt, int mode,
                 double *phi, double *v, double *work, double *E_prev,
                 orc_report *rep)
{
    const orc_model md = standard_model(m);
    return orc_anf_step_model(n, h, &md, dt, mode, phi, v, work, E_prev, rep);
}

long long orc_flow_model(const int n[3], double h, const orc_model *md, double dt, int mode,
                         int nsteps, double *phi, double *v, double *work,
                         double *E_prev, orc_report *reps)
{
    long long arrests = 0;
    int s;
    for (s = 0; s < nsteps; s++) {
        orc_report r;
        if (orc_anf_step_model(n, h, md, dt, mode, phi, v, work, E_prev, &r) != 0) {
            if (reps) reps[s] = r;
            return -1;
        }
        arrests += r.arrested;
        if (reps) reps[s] = r;
    }
    return arrests;
}

long long orc_flow(const int n[3], double h, double m, double dt, int mode,
                   int nsteps, double *phi, double *v, double *work,
                   double *E_prev, orc_report *reps)
{
    const orc_model md = standard_model(m);
    return orc_flow_model(n, h, &md, dt, mode, nsteps, phi, v, work, E_prev, reps);
}

/* ------------------------------------------------------------------------
 * Section 4: initial fields
 * ------------------------------------------------------------------------ */
static double coord(const int n[3], double h, int axis, int i)
{
    return ((double)i - 0.5 * (double)(n[axis] - 1)) * h;
}

void orc_apply_vacuum_boundary(const int n[3], double *phi)
{
    int x, y, z;
    for (x = 0; x < n[0]; x++)
        for (y = 0; y < n[1]; y++)
            for (z = 0; z < n[2]; z++)
                if (!is_interior(n, x, y, z)) {
                    double *p = &phi[4 * site_index(n, x, y, z)];
                    p[0] = 1.0;
                    p[1] = p[2] = p[3] = 0.0;
                }
}

void orc_seed_vacuum(const int n[3], double *phi)
{
    size_t s, ns = (size_t)n[0] * n[1] * n[2];
    for (s = 0; s < ns; s++) {
        phi[4 * s] = 1.0;
        phi[4 * s + 1] = phi[4 * s + 2] = phi[4 * s + 3] = 0.0;
    }
}

/* complex helpers (plain structs, no <complex.h> to keep the C obvious) */
typedef struct { double re, im; } cplx;
static cplx cmul(cplx a, cplx b)
{
    cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
    return r;
}
static cplx cadd(cplx a, cplx b)
{
    cplx r = {a.re + b.re, a.im + b.im};
    return r;
}

/* Unit vector n_R = (2 Re R, 2 Im R, 1 - |R|^2)/(1 + |R|^2) of Section 4.1,
 * written with R = P/Q in homogeneous form so that no division by zero can
 * occur: n_R = (2 Re(P conj Q), 2 Im(P conj Q), |Q|^2 - |P|^2)/(|P|^2+|Q|^2).
 * The Riemann-sphere coordinate z = tan(theta/2) e^{i varphi} = (x+iy)/(r+z3)
 * is represented by the pair (Z1, Z0) with z = Z1/Z0; for z3 < 0 the
 * equivalent pair (r - z3, x - iy) is used, which avoids cancellation. */
static void rational_map_direction(int B, double x, double y, double z3,
                                   double r, double nhat[3])
{
    cplx Z1, Z0, P, Q;
    double den;
    if (z3 >= 0.0) {
        Z1.re = x; Z1.im = y;
        Z0.re = r + z3; Z0.im = 0.0;
    } else {
        Z1.re = r - z3; Z1.im = 0.0;
        Z0.re = x; Z0.im = -y;
    }
    if (B == 1) { /* R(z) = z */
        P = Z1;
        Q = Z0;
    } else if (B == 2) { /* R(z) = z^2 */
        P = cmul(Z1, Z1);
        Q = cmul(Z0, Z0);
    } else if (B == 3) { /* R(z) = (sqrt3 a z^2 - 1) / (z (z^2 - sqrt3 a)), a = i (tetrahedral) */
        cplx Z1s = cmul(Z1, Z1), Z0s = cmul(Z0, Z0);
        cplx c = {0.0, sqrt(3.0)};
        cplx t = cmul(c, Z1s);             /* sqrt3 i z1^2 */
        cplx u = cmul(c, Z0s);             /* sqrt3 i z0^2 */
        P.re = cmul(t, Z0).re - cmul(Z0s, Z0).re;  /* z0 (sqrt3 i z1^2 - z0^2) */
        P.im = cmul(t, Z0).im - cmul(Z0s, Z0).im;
        Q.re = cmul(Z1, cadd(Z1s, (cplx){-u.re, -u.im})).re;  /* z1 (z1^2 - sqrt3 i z0^2) */
        Q.im = cmul(Z1, cadd(Z1s, (cplx){-u.re, -u.im})).im;
    } else { /* B = 4: R(z) = (z^4 + 2 sqrt3 i z^2 + 1)/(z^4 - 2 sqrt3 i z^2 + 1) */
        cplx Z1s = cmul(Z1, Z1), Z0s = cmul(Z0, Z0);
        cplx Z14 = cmul(Z1s, Z1s), Z04 = cmul(Z0s, Z0s);
        cplx mid = cmul(Z1s, Z0s);
        cplx c = {0.0, 2.0 * sqrt(3.0)};
        cplx cm = {0.0, -2.0 * sqrt(3.0)};
        P = cadd(cadd(Z14, cmul(c, mid)), Z04);
        Q = cadd(cadd(Z14, cmul(cm, mid)), Z04);
    }
    den = P.re * P.re + P.im * P.im + Q.re * Q.re + Q.im * Q.im;
    if (den == 0.0) {
        nhat[0] = nhat[1] = nhat[2] = 0.0;
        return;
    }
    /* P conj(Q) */
    nhat[0] = 2.0 * (P.re * Q.re + P.im * Q.im) / den;
    nhat[1] = 2.0 * (P.im * Q.re - P.re * Q.im) / den;
    nhat[2] = (Q.re * Q.re + Q.im * Q.im - P.re * P.re - P.im * P.im) / den;
}

int orc_seed_rational_map(const int n[3], double h, int B,
                          double profile_scale, double *phi)
{
    int x;
    if (B < 1 || B > 4) return -1;
#pragma omp parallel for schedule(static)
    for (x = 0; x < n[0]; x++) {
        int y, z;
        for (y = 0; y < n[1]; y++)
            for (z = 0; z < n[2]; z++) {
                double cx = coord(n, h, 0, x), cy = coord(n, h, 1, y),
                       cz = coord(n, h, 2, z);
                double r = sqrt(cx * cx + cy * cy + cz * cz);
                double f = M_PI * exp(-r / profile_scale);
                double nh[3];
                double *p = &phi[4 * site_index(n, x, y, z)];
                rational_map_direction(B, cx, cy, cz, r, nh);
                /* U = exp(i f n.tau) = cos f + i sin f n.tau */
                p[0] = cos(f);
                p[1] = sin(f) * nh[0];
                p[2] = sin(f) * nh[1];
                p[3] = sin(f) * nh[2];
            }
    }
    orc_apply_vacuum_boundary(n, phi);
    return 0;
}

/* Section 4.1 with the placement convention of the configuration files
 * (Section 7.3): the rational-map Skyrmion of degree B moved to X and
 * rotated by R (row-major, x' = R x), U(x) = U_B(R^T (x - X)). */
int orc_rational_map_field(const int n[3], double h, int B, double profile_scale,
                           const double X[3], const double R[9], double *phi)
{
    int x;
    if (B < 1 || B > 4) return -1;
#pragma omp parallel for schedule(static)
    for (x = 0; x < n[0]; x++) {
        int y, z, i;
        for (y = 0; y < n[1]; y++)
            for (z = 0; z < n[2]; z++) {
                const double d[3] = {coord(n, h, 0, x) - X[0], coord(n, h, 1, y) - X[1],
                                     coord(n, h, 2, z) - X[2]};
                double q[3], r, f, nh[3];
                double *p = &phi[4 * site_index(n, x, y, z)];
                for (i = 0; i < 3; i++) q[i] = R[i] * d[0] + R[3 + i] * d[1] + R[6 + i] * d[2];
                r = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
                f = M_PI * exp(-r / profile_scale);
                rational_map_direction(B, q[0], q[1], q[2], r, nh);
                p[0] = cos(f);
                p[1] = sin(f) * nh[0];
                p[2] = sin(f) * nh[1];
                p[3] = sin(f) * nh[2];
            }
    }
    return 0;
}

/* Quaternion product in the U = phi^0 + i phi^a tau^a representation:
 * (a0, a)(b0, b) = (a0 b0 - a.b, a0 b + b0 a - a x b), which follows from
 * tau^a tau^b = delta^{ab} + i eps^{abc} tau^c. */
static void qmul(const double a[4], const double b[4], double out[4])
{
    double r[4];
    r[0] = a[0] * b[0] - (a[1] * b[1] + a[2] * b[2] + a[3] * b[3]);
    r[1] = a[0] * b[1] + b[0] * a[1] - (a[2] * b[3] - a[3] * b[2]);
    r[2] = a[0] * b[2] + b[0] * a[2] - (a[3] * b[1] - a[1] * b[3]);
    r[3] = a[0] * b[3] + b[0] * a[3] - (a[1] * b[2] - a[2] * b[1]);
    memcpy(out, r, sizeof(r));
}

/* Section 4.2, Eq. "Product ansatz": the ordered product a b of two fields,
 * site by site. */
void orc_field_product(const int n[3], const double *a, const double *b, double *out)
{
    const long long ns = (long long)n[0] * n[1] * n[2];
    long long s;
#pragma omp parallel for schedule(static)
    for (s = 0; s < ns; s++) qmul(&a[4 * s], &b[4 * s], &out[4 * s]);
}

void orc_seed_product(const int n[3], double h, int K, const double *pos,
                      const double *quat, double profile_scale,
                      int symmetrise, double *phi)
{
    int x;
#pragma omp parallel for schedule(static)
    for (x = 0; x < n[0]; x++) {
        int y, z, k, q;
        double *U = (double *)malloc(4 * (size_t)(K > 0 ? K : 1) * sizeof(double));
        for (y = 0; y < n[1]; y++)
            for (z = 0; z < n[2]; z++) {
                double fwd[4] = {1, 0, 0, 0}, rev[4] = {1, 0, 0, 0};
                double *p = &phi[4 * site_index(n, x, y, z)];
                for (k = 0; k < K; k++) {
                    double dx = coord(n, h, 0, x) - pos[3 * k];
                    double dy = coord(n, h, 1, y) - pos[3 * k + 1];
                    double dz = coord(n, h, 2, z) - pos[3 * k + 2];
                    double r = sqrt(dx * dx + dy * dy + dz * dz);
                    double f = M_PI * exp(-r / profile_scale);
                    double u0[4], A[4], Ad[4], t[4];
                    u0[0] = cos(f);
                    if (r > 0.0) {
                        u0[1] = sin(f) * dx / r;
                        u0[2] = sin(f) * dy / r;
                        u0[3] = sin(f) * dz / r;
                    } else {
                        u0[1] = u0[2] = u0[3] = 0.0;
                    }
                    /* A U A^dagger with A = q0 + i q.tau, A^dagger = q0 - i q.tau */
                    for (q = 0; q < 4; q++) A[q] = quat[4 * k + q];
                    Ad[0] = A[0];
                    Ad[1] = -A[1];
                    Ad[2] = -A[2];
                    Ad[3] = -A[3];
                    qmul(A, u0, t);
                    qmul(t, Ad, &U[4 * k]);
                }
                for (k = 0; k < K; k++) qmul(fwd, &U[4 * k], fwd);
                for (k = K - 1; k >= 0; k--) qmul(rev, &U[4 * k], rev);
                if (symmetrise) {
                    double s[4], nrm = 0.0;
                    for (q = 0; q < 4; q++) {
                        s[q] = fwd[q] + rev[q];
                        nrm += s[q] * s[q];
                    }
                    nrm = sqrt(nrm);
                    if (nrm < 1e-12) {
                        for (q = 0; q < 4; q++) p[q] = fwd[q];
                    } else {
                        for (q = 0; q < 4; q++) p[q] = s[q] / nrm;
                    }
                } else {
                    for (q = 0; q < 4; q++) p[q] = fwd[q];
                }
            }
        free(U);
    }
    orc_apply_vacuum_boundary(n, phi);
}

/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014), in counter form: the i-th
 * output of the generator whose state starts at `seed`. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * UINT64_C(0x9E3779B97F4A7C15);
    z = (z ^ (z >> 30)) * UINT64_C(0xBF58476D1CE4E5B9);
    z = (z ^ (z >> 27)) * UINT64_C(0x94D049BB133111EB);
    return z ^ (z >> 31);
}

/* Box-Muller: u1 in (0, 1], u2 in [0, 1) from the top 53 bits. */
double orc_normal(uint64_t seed, uint64_t i)
{
    double u1 = ((double)(orc_splitmix64(seed, 2 * i) >> 11) + 1.0) *
                (1.0 / 9007199254740992.0);
    double u2 = (double)(orc_splitmix64(seed, 2 * i + 1) >> 11) *
                (1.0 / 9007199254740992.0);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

/* Separable discrete Gaussian smoothing of a 4-component field (the noise
 * recipe's smoothing step): weights exp(-(k h)^2 / (2 sigma^2)) for
 * |k| <= K = ceil(4 sigma / h), divided by their sum; applied along x, then
 * y, then z, with sites outside the box contributing zero. */
void orc_gaussian_smooth(const int n[3], double h, double sigma, const double *in,
                         double *out)
{
    size_t ns = (size_t)n[0] * n[1] * n[2];
    int K = (int)ceil(4.0 * sigma / h), k, axis, x;
    double *w = (double *)malloc((size_t)(2 * K + 1) * sizeof(double));
    double *a = (double *)malloc(4 * ns * sizeof(double));
    double *b = (double *)calloc(4 * ns, sizeof(double));
    double wsum = 0.0;

    memcpy(a, in, 4 * ns * sizeof(double));
    for (k = -K; k <= K; k++) {
        w[k + K] = exp(-(k * h) * (k * h) / (2.0 * sigma * sigma));
        wsum += w[k + K];
    }
    for (k = 0; k <= 2 * K; k++) w[k] /= wsum;

    for (axis = 0; axis < 3; axis++) {
#pragma omp parallel for schedule(static)
        for (x = 0; x < n[0]; x++) {
            int y, z, c, kk;
            for (y = 0; y < n[1]; y++)
                for (z = 0; z < n[2]; z++) {
                    double acc[4] = {0, 0, 0, 0};
                    for (kk = -K; kk <= K; kk++) {
                        int xx = x, yy = y, zz = z;
                        if (axis == 0) xx += kk;
                        if (axis == 1) yy += kk;
                        if (axis == 2) zz += kk;
                        if (xx < 0 || xx >= n[0] || yy < 0 || yy >= n[1] ||
                            zz < 0 || zz >= n[2])
                            continue;
                        for (c = 0; c < 4; c++)
                            acc[c] += w[kk + K] *
                                      a[4 * site_index(n, xx, yy, zz) + c];
                    }
                    for (c = 0; c < 4; c++)
                        b[4 * site_index(n, x, y, z) + c] = acc[c];
                }
        }
        memcpy(a, b, 4 * ns * sizeof(double));
    }
    memcpy(out, a, 4 * ns * sizeof(double));
    free(w);
    free(a);
    free(b);
}

/* The noise 4-vector field of the smoothed-noise seed before it is added to
 * the vacuum: i.i.d. N(0,1) components (orc_normal with counter 4 s + c at
 * site s) at sites within `radius` of the origin and 0 elsewhere, smoothed
 * by orc_gaussian_smooth, then each component divided by its standard
 * deviation over the ball sites. */
void orc_noise_components(const int n[3], double h, double radius, double sigma,
                          uint64_t seed, double *a)
{
    size_t ns = (size_t)n[0] * n[1] * n[2], s;
    int x, q;
    double *raw = (double *)calloc(4 * ns, sizeof(double));
    nsum mean[4], var[4];
    double count = 0.0;

    /* i.i.d. N(0,1) per component inside the ball */
#pragma omp parallel for schedule(static)
    for (x = 0; x < n[0]; x++) {
        int y, z, c;
        for (y = 0; y < n[1]; y++)
            for (z = 0; z < n[2]; z++) {
                double cx = coord(n, h, 0, x), cy = coord(n, h, 1, y),
                       cz = coord(n, h, 2, z);
                size_t si = site_index(n, x, y, z);
                if (cx * cx + cy * cy + cz * cz <= radius * radius)
                    for (c = 0; c < 4; c++)
                        raw[4 * si + c] = orc_normal(seed, 4 * (uint64_t)si + c);
            }
    }

    orc_gaussian_smooth(n, h, sigma, raw, a);
    free(raw);

    /* unit standard deviation per component over the ball sites */
    memset(mean, 0, sizeof(mean));
    memset(var, 0, sizeof(var));
    for (s = 0; s < ns; s++) {
        int xs = (int)(s / ((size_t)n[1] * n[2]));
        int ys = (int)((s / (size_t)n[2]) % (size_t)n[1]);
        int zs = (int)(s % (size_t)n[2]);
        double cx = coord(n, h, 0, xs), cy = coord(n, h, 1, ys),
               cz = coord(n, h, 2, zs);
        if (cx * cx + cy * cy + cz * cz <= radius * radius) {
            for (q = 0; q < 4; q++) nsum_add(&mean[q], a[4 * s + q]);
            count += 1.0;
        }
    }
    for (s = 0; s < ns; s++) {
        int xs = (int)(s / ((size_t)n[1] * n[2]));
        int ys = (int)((s / (size_t)n[2]) % (size_t)n[1]);
        int zs = (int)(s % (size_t)n[2]);
        double cx = coord(n, h, 0, xs), cy = coord(n, h, 1, ys),
               cz = coord(n, h, 2, zs);
        if (cx * cx + cy * cy + cz * cz <= radius * radius)
            for (q = 0; q < 4; q++) {
                double d = a[4 * s + q] - nsum_get(&mean[q]) / count;
                nsum_add(&var[q], d * d);
            }
    }
    for (q = 0; q < 4; q++) {
        double sd = count > 0.0 ? sqrt(nsum_get(&var[q]) / count) : 0.0;
        if (sd > 0.0)
            for (s = 0; s < ns; s++) a[4 * s + q] /= sd;
    }
}

void orc_seed_noise(const int n[3], double h, double radius, double sigma,
                    uint64_t seed, double *phi)
{
    size_t ns = (size_t)n[0] * n[1] * n[2], s;
    double *a = (double *)malloc(4 * ns * sizeof(double));

    orc_noise_components(n, h, radius, sigma, seed, a);

    /* phi = normalise(vacuum + noise) */
    for (s = 0; s < ns; s++) {
        double t[4], nrm;
        t[0] = 1.0 + a[4 * s];
        t[1] = a[4 * s + 1];
        t[2] = a[4 * s + 2];
        t[3] = a[4 * s + 3];
        nrm = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2] + t[3] * t[3]);
        if (nrm < 1e-12) {
            phi[4 * s] = 1.0;
            phi[4 * s + 1] = phi[4 * s + 2] = phi[4 * s + 3] = 0.0;
        } else {
            int q;
            for (q = 0; q < 4; q++) phi[4 * s + q] = t[q] / nrm;
        }
    }
    orc_apply_vacuum_boundary(n, phi);
    free(a);
}

/* ------------------------------------------------------------------------
 * Section 5: physical properties of a static configuration
 *
 * Written in the paper's su(2) notation: U = phi^0 1 + i phi^a tau^a as a
 * 2x2 complex matrix, the left currents L_k = U^dagger d_k U (Eq. "Stress
 * tensor"), the isospin currents T_j = (i/2) U^dagger [tau^j, U], and traces
 * of explicit 2x2 products.  r = x - X_c with X_c of Eq. "CoM".
 * ------------------------------------------------------------------------ */
typedef struct {
    cplx a[2][2];
} mat2;

static mat2 m2_zero(void)
{
    mat2 r;
    memset(&r, 0, sizeof(r));
    return r;
}

static mat2 m2_mul(mat2 p, mat2 q)
{
    mat2 r = m2_zero();
    int i, j, k;
    for (i = 0; i < 2; i++)
        for (j = 0; j < 2; j++)
            for (k = 0; k < 2; k++) r.a[i][j] = cadd(r.a[i][j], cmul(p.a[i][k], q.a[k][j]));
    return r;
}

static mat2 m2_lin(double s, mat2 p, double t, mat2 q) /* s p + t q */
{
    mat2 r;
    int i, j;
    for (i = 0; i < 2; i++)
        for (j = 0; j < 2; j++) {
            r.a[i][j].re = s * p.a[i][j].re + t * q.a[i][j].re;
            r.a[i][j].im = s * p.a[i][j].im + t * q.a[i][j].im;
        }
    return r;
}

static mat2 m2_adjoint(mat2 p)
{
    mat2 r;
    int i, j;
    for (i = 0; i < 2; i++)
        for (j = 0; j < 2; j++) {
            r.a[i][j].re = p.a[j][i].re;
            r.a[i][j].im = -p.a[j][i].im;
        }
    return r;
}

static mat2 m2_times_i(mat2 p) /* i p */
{
    mat2 r;
    int i, j;
    for (i = 0; i < 2; i++)
        for (j = 0; j < 2; j++) {
            r.a[i][j].re = -p.a[i][j].im;
            r.a[i][j].im = p.a[i][j].re;
        }
    return r;
}

static mat2 m2_commutator(mat2 p, mat2 q) { return m2_lin(1.0, m2_mul(p, q), -1.0, m2_mul(q, p)); }

static double m2_retrace(mat2 p) { return p.a[0][0].re + p.a[1][1].re; }

/* Pauli matrices tau^1, tau^2, tau^3 */
static mat2 pauli(int a)
{
    mat2 r = m2_zero();
    if (a == 0) {
        r.a[0][1].re = 1.0;
        r.a[1][0].re = 1.0;
    } else if (a == 1) {
        r.a[0][1].im = -1.0;
        r.a[1][0].im = 1.0;
    } else {
        r.a[0][0].re = 1.0;
        r.a[1][1].re = -1.0;
    }
    return r;
}

/* q^0 1 + i q^a tau^a for a real 4-vector q */
static mat2 quaternion_matrix(const double q[4])
{
    mat2 r = m2_zero();
    int a;
    r.a[0][0].re = q[0];
    r.a[1][1].re = q[0];
    for (a = 0; a < 3; a++) r = m2_lin(1.0, r, q[a + 1], m2_times_i(pauli(a)));
    return r;
}

static int levi3(int i, int j, int k)
{
    if (i == j || j == k || i == k) return 0;
    return ((i == 0 && j == 1) || (i == 1 && j == 2) || (i == 2 && j == 0)) ? 1 : -1;
}

/* sums of one x-plane: pass 0 {b, x b, y b, z b}; pass 1 everything else */
enum { OBS_B = 0, OBS_XB = 1, OBS_E = 4, OBS_R2B = 5, OBS_Q = 6, OBS_U = 15, OBS_V = 24,
       OBS_W = 33, OBS_D = 42, OBS_N = 43 };

static void observables_plane(const int n[3], double h, double m, const double *phi, int x,
                              int pass, const double X[3], nsum *acc)
{
    int y, z, i, j, k, l, mm, nn, p, a;
    mat2 tau[3];
    for (a = 0; a < 3; a++) tau[a] = pauli(a);
    for (y = 2; y <= n[1] - 3; y++)
        for (z = 2; z <= n[2] - 3; z++) {
            double d1[3][4], d2[3][4], dm[3][4], g[4], f[4], dens[4], xv[3], r[3], r2;
            size_t s = site_index(n, x, y, z);
            const double *ph = &phi[4 * s];
            orc_site_derivatives(n, h, phi, x, y, z, d1, d2, dm);
            orc_site_terms(ph, d1, d2, dm, m, g, f, dens);
            xv[0] = coord(n, h, 0, x);
            xv[1] = coord(n, h, 1, y);
            xv[2] = coord(n, h, 2, z);
            if (pass == 0) {
                nsum_add(&acc[OBS_B], dens[3]);
                for (i = 0; i < 3; i++) nsum_add(&acc[OBS_XB + i], xv[i] * dens[3]);
                continue;
            }
            r2 = 0.0;
            for (i = 0; i < 3; i++) {
                r[i] = xv[i] - X[i];
                r2 += r[i] * r[i];
            }
            {
                mat2 U = quaternion_matrix(ph), Ud = m2_adjoint(U), L[3], T[3];
                double Tij[3][3], Tkk, lag, tr_ll = 0.0, tr_cc = 0.0;
                /* L_k is su(2)-valued; the lattice derivative of phi has a small
                 * component along phi, which shows up as a multiple of the
                 * identity in U^dagger d_k U: keep its traceless part */
                for (k = 0; k < 3; k++) {
                    mat2 full = m2_mul(Ud, quaternion_matrix(d1[k]));
                    const double half_tr = 0.5 * m2_retrace(full);
                    full.a[0][0].re -= half_tr;
                    full.a[1][1].re -= half_tr;
                    L[k] = full;
                }
                for (j = 0; j < 3; j++)
                    T[j] = m2_lin(0.5, m2_times_i(m2_mul(Ud, m2_commutator(tau[j], U))), 0.0, U);
                /* static Lagrangian density: (1/2) Tr(L_k L_k) + (1/16) Tr([L_i,L_j]^2) - m^2 Tr(1 - U) */
                for (k = 0; k < 3; k++) tr_ll += m2_retrace(m2_mul(L[k], L[k]));
                for (i = 0; i < 3; i++)
                    for (j = 0; j < 3; j++) {
                        mat2 c = m2_commutator(L[i], L[j]);
                        tr_cc += m2_retrace(m2_mul(c, c));
                    }
                lag = 0.5 * tr_ll + tr_cc / 16.0 - m * m * (2.0 - m2_retrace(U));
                /* Eq. "Stress tensor", spatial static part */
                for (i = 0; i < 3; i++)
                    for (j = 0; j < 3; j++) {
                        double t = -m2_retrace(m2_mul(L[i], L[j]));
                        for (k = 0; k < 3; k++)
                            t -= 0.25 * m2_retrace(m2_mul(m2_commutator(L[i], L[k]),
                                                          m2_commutator(L[j], L[k])));
                        Tij[i][j] = t + (i == j ? lag : 0.0);
                    }
                Tkk = Tij[0][0] + Tij[1][1] + Tij[2][2];
                nsum_add(&acc[OBS_E], dens[0] + dens[1] + dens[2]);
                nsum_add(&acc[OBS_R2B], r2 * dens[3]);
                /* Eq. "Q tensor" with rho = B0 / 2 */
                for (i = 0; i < 3; i++)
                    for (j = 0; j < 3; j++)
                        nsum_add(&acc[OBS_Q + 3 * i + j],
                                 (3.0 * r[i] * r[j] - (i == j ? r2 : 0.0)) * 0.5 * dens[3]);
                /* Eqs. "U inertia tensor", "V inertia tensor", "W inertia tensor" */
                for (i = 0; i < 3; i++)
                    for (j = 0; j < 3; j++) {
                        double u = m2_retrace(m2_mul(T[i], T[j])), v = 0.0, w = 0.0;
                        for (k = 0; k < 3; k++)
                            u += 0.25 * m2_retrace(m2_mul(m2_commutator(L[k], T[i]),
                                                          m2_commutator(L[k], T[j])));
                        for (l = 0; l < 3; l++)
                            for (mm = 0; mm < 3; mm++)
                                for (nn = 0; nn < 3; nn++)
                                    for (p = 0; p < 3; p++) {
                                        double e = (double)(levi3(i, l, mm) * levi3(j, nn, p));
                                        double t;
                                        if (e == 0.0) continue;
                                        t = m2_retrace(m2_mul(L[mm], L[p]));
                                        for (k = 0; k < 3; k++)
                                            t += 0.25 * m2_retrace(m2_mul(m2_commutator(L[k], L[mm]),
                                                                          m2_commutator(L[k], L[p])));
                                        v += e * r[l] * r[nn] * t;
                                    }
                        for (l = 0; l < 3; l++)
                            for (mm = 0; mm < 3; mm++) {
                                double e = (double)levi3(j, l, mm), t;
                                if (e == 0.0) continue;
                                t = m2_retrace(m2_mul(T[i], L[mm]));
                                for (k = 0; k < 3; k++)
                                    t += 0.25 * m2_retrace(m2_mul(m2_commutator(L[k], T[i]),
                                                                  m2_commutator(L[k], L[mm])));
                                w += e * r[l] * t;
                            }
                        nsum_add(&acc[OBS_U + 3 * i + j], -u);
                        nsum_add(&acc[OBS_V + 3 * i + j], -v);
                        nsum_add(&acc[OBS_W + 3 * i + j], w);
                    }
                /* Eq. "D-term" integrand */
                {
                    double q = 0.0;
                    for (i = 0; i < 3; i++)
                        for (j = 0; j < 3; j++) q += r[i] * r[j] * Tij[i][j];
                    nsum_add(&acc[OBS_D], q - r2 * Tkk / 3.0);
                }
            }
        }
}

void orc_observables(const int n[3], double h, double m, const double *phi, orc_observables_t *out)
{
    int x, q, i, j;
    const int nx = n[0];
    const double h3 = h * h * h;
    double X[3] = {0.0, 0.0, 0.0}, tot[OBS_N];
    nsum *acc = (nsum *)calloc((size_t)nx * OBS_N, sizeof(nsum));
    int pass;
    for (pass = 0; pass < 2; pass++) {
        nsum sum[OBS_N];
        memset(acc, 0, (size_t)nx * OBS_N * sizeof(nsum));
#pragma omp parallel for schedule(dynamic, 1)
        for (x = 2; x <= nx - 3; x++) observables_plane(n, h, m, phi, x, pass, X, &acc[(size_t)x * OBS_N]);
        memset(sum, 0, sizeof(sum));
        for (x = 2; x <= nx - 3; x++)
            for (q = 0; q < OBS_N; q++) nsum_add(&sum[q], nsum_get(&acc[(size_t)x * OBS_N + q]));
        for (q = 0; q < OBS_N; q++) tot[q] = h3 * nsum_get(&sum[q]);
        if (pass == 0) {
            out->B = tot[OBS_B];
            for (i = 0; i < 3; i++) X[i] = out->X[i] = tot[OBS_XB + i] / tot[OBS_B];
        }
    }
    out->E = tot[OBS_E];
    out->R = sqrt(tot[OBS_R2B] / out->B);
    for (i = 0; i < 3; i++)
        for (j = 0; j < 3; j++) {
            out->Q[i][j] = tot[OBS_Q + 3 * i + j];
            out->U[i][j] = tot[OBS_U + 3 * i + j];
            out->V[i][j] = tot[OBS_V + 3 * i + j];
            out->W[i][j] = tot[OBS_W + 3 * i + j];
        }
    out->D = -2.0 * out->E / 5.0 * tot[OBS_D];
    free(acc);
}

/* ------------------------------------------------------------------------
 * Section 6.2 (ray tracing): a headless volume render of the baryon density
 *
 * The volume holds, per site, {B0 / max B0, unit pion vector} (zero pions where
 * the pion vector vanishes); B0 is the flow's baryon density at interior
 * sites and 0 on the boundary layers.  Rays (perspective camera, fixed step)
 * sample it by trilinear interpolation; the transfer function and the
 * front-to-back compositing are those the paper states.  Readings are in the
 * header file.
 * ------------------------------------------------------------------------ */
void orc_render_volume_from_field(const int n[3], double h, const double *phi, double *vol)
{
    size_t total = (size_t)n[0] * n[1] * n[2], s;
    double bmax = 0.0;
    int x;
    double *b = (double *)calloc(total, sizeof(double));
#pragma omp parallel for schedule(static)
    for (x = 2; x <= n[0] - 3; x++) {
        int y, z;
        for (y = 2; y <= n[1] - 3; y++)
            for (z = 2; z <= n[2] - 3; z++) {
                double d1[3][4], d2[3][4], dm[3][4], g[4], f[4], dens[4];
                size_t i = site_index(n, x, y, z);
                orc_site_derivatives(n, h, phi, x, y, z, d1, d2, dm);
                orc_site_terms(&phi[4 * i], d1, d2, dm, 0.0, g, f, dens);
                b[i] = dens[3];
            }
    }
    for (s = 0; s < total; s++)
        if (b[s] > bmax) bmax = b[s];
    for (s = 0; s < total; s++) {
        const double *p = &phi[4 * s];
        const double np = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
        int a;
        vol[4 * s] = bmax > 0.0 ? b[s] / bmax : 0.0;
        for (a = 1; a < 4; a++) vol[4 * s + a] = np > 0.0 ? p[a] / np : 0.0;
    }
    free(b);
}

/* trilinear interpolation of the 4-component volume at lattice coordinates g */
void orc_render_sample(const int n[3], const double *vol, const double g[3], double out[4])
{
    int i0[3], c, a;
    double w[3];
    for (a = 0; a < 3; a++) {
        double t = g[a];
        if (t < 0.0) t = 0.0;
        if (t > (double)(n[a] - 1)) t = (double)(n[a] - 1);
        i0[a] = (int)floor(t);
        if (i0[a] > n[a] - 2) i0[a] = n[a] - 2;
        w[a] = t - (double)i0[a];
    }
    for (c = 0; c < 4; c++) out[c] = 0.0;
    for (a = 0; a < 8; a++) {
        const int dx = a & 1, dy = (a >> 1) & 1, dz = (a >> 2) & 1;
        const double wt = (dx ? w[0] : 1.0 - w[0]) * (dy ? w[1] : 1.0 - w[1]) * (dz ? w[2] : 1.0 - w[2]);
        const double *v = &vol[4 * site_index(n, i0[0] + dx, i0[1] + dy, i0[2] + dz)];
        for (c = 0; c < 4; c++) out[c] += wt * v[c];
    }
}

void orc_render_volume(const int n[3], const double *vol, const orc_render_params *rp,
                       double *rgba)
{
    double half[3], s = 0.0;
    int a, px;
    for (a = 0; a < 3; a++) {
        half[a] = 0.5 * (double)(n[a] - 1);
        if (half[a] > s) s = half[a];
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (px = 0; px < rp->width * rp->height; px++) {
        const int ix = px % rp->width, iy = px / rp->width;
        const double aspect = (double)rp->width / (double)rp->height;
        const double u = (2.0 * (ix + 0.5) / rp->width - 1.0) * aspect;
        const double v = 2.0 * (iy + 0.5) / rp->height - 1.0;
        double dv[3] = {u, v, -ORC_RENDER_FOCAL}, ov[3] = {0.0, 0.0, ORC_RENDER_EYE};
        double o[3], d[3], nd = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
        double tnear = -1e300, tfar = 1e300, sum[4] = {0.0, 0.0, 0.0, 0.0}, t;
        int i, j, c;
        for (i = 0; i < 3; i++) dv[i] /= nd;
        /* view space -> box space: o = R ov, d = R dv (R row-major) */
        for (i = 0; i < 3; i++) {
            o[i] = 0.0;
            d[i] = 0.0;
            for (j = 0; j < 3; j++) {
                o[i] += rp->view[3 * i + j] * ov[j];
                d[i] += rp->view[3 * i + j] * dv[j];
            }
        }
        /* slab intersection with the box |p_i| <= half_i / s */
        for (i = 0; i < 3; i++) {
            const double b = half[i] / s;
            if (d[i] != 0.0) {
                double t0 = (-b - o[i]) / d[i], t1 = (b - o[i]) / d[i];
                if (t0 > t1) {
                    const double tmp = t0;
                    t0 = t1;
                    t1 = tmp;
                }
                if (t0 > tnear) tnear = t0;
                if (t1 < tfar) tfar = t1;
            } else if (o[i] < -b || o[i] > b) {
                tnear = 1.0;
                tfar = 0.0;
            }
        }
        if (tnear < 0.0) tnear = 0.0;
        for (t = tnear; t <= tfar; t += rp->step) {
            double p[3], g[3], smp[4], input, col[4];
            for (i = 0; i < 3; i++) {
                p[i] = o[i] + t * d[i];
                g[i] = p[i] * s + half[i];
            }
            orc_render_sample(n, vol, g, smp);
            input = (smp[0] - rp->levelset) * rp->transfer_scale;
            if (input < 0.0) continue; /* rejected */
            /* colour = input^2 (pion_1, pion_2, pion_3, 1 / input) */
            col[0] = input * input * smp[1];
            col[1] = input * input * smp[2];
            col[2] = input * input * smp[3];
            col[3] = input;
            for (c = 0; c < 4; c++) sum[c] += col[c] * (1.0 - sum[3]);
            if (sum[3] > ORC_RENDER_ALPHA_STOP) break;
        }
        for (c = 0; c < 4; c++) {
            double val = sum[c] * rp->brightness;
            rgba[4 * (size_t)px + c] = val < 0.0 ? 0.0 : (val > 1.0 ? 1.0 : val);
        }
    }
}
