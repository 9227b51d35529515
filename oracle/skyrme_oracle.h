/*
 * skyrme_oracle.h -- plain FP64 CPU reference of the arrested-Newton-flow step
 * of the 3D Skyrme model in sigma-model form (arXiv 2604.25876, Sections 2-4).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA library.
 * Only tests, the smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code, header, table or helper with the CUDA path.
 *
 * Conventions (all arrays are host memory, caller-owned):
 *   - lattice n[3] = {Nx, Ny, Nz}; site (x,y,z) has linear index
 *     ((x*Ny)+y)*Nz+z, z fastest (Section 7.5.1, the text file format).
 *   - a field is 4 doubles per site (phi^0, phi^1, phi^2, phi^3), AoS.
 *   - coordinates x_i = (i - (N-1)/2) * h on every axis.
 *   - interior sites have every index in [2, N-3]; the two outer layers are
 *     the fixed vacuum phi = (1,0,0,0) (Section 3, vacuum boundary).
 */
#ifndef SKYRME_ORACLE_H
#define SKYRME_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- per-site building blocks (Section 3 and Section 2.1) ---- */

/* 4th-order finite differences at interior site (x,y,z):
 *   d1[i][A] = d_i phi^A, d2[i][A] = d_ii phi^A,
 *   dm[p][A] = d_i d_j phi^A for the pairs p = (x,y), (x,z), (y,z). */
void orc_site_derivatives(const int n[3], double h, const double *phi,
                          int x, int y, int z,
                          double d1[3][4], double d2[3][4], double dm[3][4]);

/* Euler-Lagrange gradient G = dE/dphi (Eq. "Sigma model EL equations"),
 * tangent force F = -G + (G.phi) phi (Eq. "Newton_flow"), and the site
 * densities dens = {e2, e4, e0, b}: the quadratic, quartic and mass parts of
 * Eq. "SkyrmeEnergy_phi" and the baryon density of Eq. "B0_components". */
void orc_site_terms(const double phi[4], const double d1[3][4],
                    const double d2[3][4], const double dm[3][4], double m,
                    double G[4], double F[4], double dens[4]);

/* ---- extension models (Section 7.8) ----
 * The potential is 2 mx^2 (1 - phi0) + my^2 (1 - phi0^2) + mz^2 (1 - phi0)^2
 * + (1/2) mw^2 (1 - phi0)^4 (standard, modified pion, loosely bound and
 * lightly bound), and the BPS sextic term adds c6 4 pi^4 (B0)^2 to the static
 * energy density.  {m, 0, 0, 0, 0} is the standard model of Section 2.1. */
typedef struct {
    double mx, my, mz, mw, c6;
} orc_model;

/* As orc_site_terms for a model: dens = {e2, e4, e0, b, e6}, e0 the sum of
 * the four potentials, e6 = c6 4 pi^4 b^2. */
void orc_site_terms_model(const double phi[4], const double d1[3][4],
                          const double d2[3][4], const double dm[3][4],
                          const orc_model *md, double G[4], double F[4],
                          double dens[5]);

/* ---- whole-lattice operations ---- */

/* G, F and densities at every interior site (zero on the boundary layers).
 * Any output pointer may be NULL. */
void orc_forces(const int n[3], double h, double m, const double *phi,
                double *G, double *F, double *dens);

/* out = {E, E2, E4, E0, B, V}: h^3 * sums over interior sites;
 * V = -E2 + E4 - 3 E0 (the virial, Section 5.6). */
void orc_energy(const int n[3], double h, double m, const double *phi,
                double out[6]);

/* Model versions: dens keeps {e2, e4, e0, b} per site (e6 = c6 4 pi^4 b^2);
 * out = {E, E2, E4, E0, E6, B, V}, E = E2 + E4 + E0 + E6 and
 * V = -E2 + E4 - 3 E0 + 3 E6. */
void orc_forces_model(const int n[3], double h, const orc_model *md, const double *phi,
                      double *G, double *F, double *dens);
void orc_energy_model(const int n[3], double h, const orc_model *md, const double *phi,
                      double out[7]);

/* Section 5 observables of a static field (h^3 times sums over interior
 * sites; r = x - X_c):
 *   B        baryon number (Eq. "B0_components" summed);
 *   X[3]     centre of mass, Eq. "CoM";
 *   R        RMS radius, Eq. "RMS radius";
 *   Q        quadrupole, Eq. "Q tensor" with rho = B0 / 2;
 *   U, V, W  isospin, spin and mixed inertia tensors, Eqs. "U/V/W inertia
 *            tensor" (W[i][j]: i isospin, j space);
 *   D        monopole D-term, Eq. "D-term", with E the static energy;
 *   E        static energy (Eq. "SkyrmeEnergy_phi" summed). */
typedef struct {
    double B, X[3], R, Q[3][3], U[3][3], V[3][3], W[3][3], D, E;
} orc_observables_t;
void orc_observables(const int n[3], double h, double m, const double *phi,
                     orc_observables_t *out);

/* Section 6.2 (ray tracing), headless.
 *   orc_render_volume_from_field: vol (4 doubles per site) = {B0 / max B0,
 *     pion / |pion|}, B0 the flow's baryon density (0 on the boundary layers,
 *     and the first component 0 everywhere when max B0 <= 0).
 *   orc_render_volume: one RGBA (4 doubles, each in [0, 1]) per pixel, row by
 *     row from the bottom (y up).  Readings where the paper is silent:
 *     - the box: lattice coordinates g map to box coordinates (g - (n-1)/2)/s,
 *       s the largest (n_i - 1)/2, so the longest axis spans [-1, 1];
 *     - the camera: eye at (0, 0, ORC_RENDER_EYE) in view space, pixel (u, v)
 *       in [-aspect, aspect] x [-1, 1] looking along (u, v, -ORC_RENDER_FOCAL);
 *       view is the row-major rotation taking view-space vectors to box space;
 *     - samples at t = t_near + k step along the unit ray inside the box,
 *       trilinear interpolation of all four volume components (clamped to the
 *       lattice);
 *     - input = (b - levelset) * transfer_scale, skipped when negative;
 *       colour = input^2 (pion_1, pion_2, pion_3, 1/input);
 *     - front-to-back compositing: sum += colour (1 - sum_alpha), stopped
 *       once sum_alpha > ORC_RENDER_ALPHA_STOP;
 *     - the result times brightness, each component clamped to [0, 1]. */
#define ORC_RENDER_EYE 4.0
#define ORC_RENDER_FOCAL 2.0
#define ORC_RENDER_ALPHA_STOP 0.95
typedef struct {
    int width, height;
    double view[9];
    double levelset, transfer_scale, brightness, step;
} orc_render_params;
void orc_render_volume_from_field(const int n[3], double h, const double *phi, double *vol);
void orc_render_volume(const int n[3], const double *vol, const orc_render_params *rp,
                       double *rgba);
/* the trilinear sample of the volume at lattice coordinates g (clamped) */
void orc_render_sample(const int n[3], const double *vol, const double g[3], double out[4]);

typedef struct {
    double E, E2, E4, E0, B, virial; /* of the field at the start of the step */
    double delta;                    /* max over interior sites of |F|      */
    int arrested;                    /* 1 when the velocity was zeroed       */
    double E6;                       /* sextic part of E (0 without it)      */
} orc_report;

enum { ORC_NEWTON = 0, ORC_ARRESTED = 1, ORC_GRADIENT = 2 };

/* One flow iteration (Section 3), in place on phi and v.
 *   mode ORC_ARRESTED: E_n of phi_n is compared with *E_prev; when E_n is
 *     strictly larger, v is set to zero everywhere; then
 *     v <- v + dt F(phi_n), phi <- normalise(phi_n + dt v).
 *   mode ORC_NEWTON: the same without the arrest test.
 *   mode ORC_GRADIENT: phi <- normalise(phi_n + dt F(phi_n)); v untouched.
 * *E_prev is replaced by E_n.  work holds 4 doubles per site (F).
 * Returns 0, or -1 when a non-finite value appeared. */
int orc_anf_step(const int n[3], double h, double m, double dt, int mode,
                 double *phi, double *v, double *work, double *E_prev,
                 orc_report *rep);

/* nsteps iterations; reps (nullable) receives one report per iteration.
 * Returns the number of arrests, or -1 on a non-finite value. */
long long orc_flow(const int n[3], double h, double m, double dt, int mode,
                   int nsteps, double *phi, double *v, double *work,
                   double *E_prev, orc_report *reps);

/* Model versions of the step and the flow (E includes E6). */
int orc_anf_step_model(const int n[3], double h, const orc_model *md, double dt, int mode,
                       double *phi, double *v, double *work, double *E_prev,
                       orc_report *rep);
long long orc_flow_model(const int n[3], double h, const orc_model *md, double dt, int mode,
                         int nsteps, double *phi, double *v, double *work,
                         double *E_prev, orc_report *reps);

/* ---- initial fields (Section 4) ---- */

void orc_seed_vacuum(const int n[3], double *phi);
/* phi = (cos f, sin f n_R(z)) with f(r) = pi exp(-r/profile_scale) and the
 * rational map of degree B (Table 1: 1: R=z; 2: z^2; 3: the tetrahedral map
 * with a = i; 4: the cubic map), centred at
 * the origin. */
int orc_seed_rational_map(const int n[3], double h, int B,
                          double profile_scale, double *phi);
/* Product ansatz of K isorotated 1-Skyrmions (Eq. "Product ansatz"):
 * U_k = A_k U_hedgehog(x - X_k) A_k^dagger, pos[k][3], quat[k][4] (unit).
 * symmetrise = 1: phi = normalise(U_1..U_K + U_K..U_1). */
void orc_seed_product(const int n[3], double h, int K, const double *pos,
                      const double *quat, double profile_scale,
                      int symmetrise, double *phi);
/* Smoothed-noise start: i.i.d. N(0,1) per component inside the ball
 * r <= radius, convolved with a Gaussian of width sigma (truncated at
 * 4 sigma), each component rescaled to unit standard deviation over the ball
 * sites, phi = normalise((1,0,0,0) + noise). */
void orc_seed_noise(const int n[3], double h, double radius, double sigma,
                    uint64_t seed, double *phi);
/* The seed's noise before it is added to the vacuum (4 components per
 * site): the ball's i.i.d. normals, smoothed, rescaled per component. */
void orc_noise_components(const int n[3], double h, double radius, double sigma,
                          uint64_t seed, double *noise);
/* The seed's smoothing step on any 4-component field: separable Gaussian
 * weights exp(-(k h)^2 / 2 sigma^2), |k| <= ceil(4 sigma / h), normalised to
 * sum 1, along x then y then z, zero outside the box. */
void orc_gaussian_smooth(const int n[3], double h, double sigma, const double *in,
                         double *out);
/* Overwrite the two outer layers with the vacuum. */
void orc_apply_vacuum_boundary(const int n[3], double *phi);

/* A rational-map Skyrmion (B = 1 to 4, profile pi exp(-r / profile_scale))
 * moved to X and rotated by the row-major rotation R: U(x) = U_B(R^T (x - X))
 * at every site, boundary layers included (the configuration-file placement
 * of Section 7.3).  Returns -1 for another B. */
int orc_rational_map_field(const int n[3], double h, int B, double profile_scale,
                           const double X[3], const double R[9], double *phi);
/* The ordered product ansatz of Section 4.2: out = a b site by site (out may
 * alias a or b). */
void orc_field_product(const int n[3], const double *a, const double *b, double *out);

/* SplitMix64 counter stream: value number i of stream `seed`. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t i);
/* Standard normal number i of stream `seed` (Box-Muller on two uniforms). */
double orc_normal(uint64_t seed, uint64_t i);

#ifdef __cplusplus
}
#endif
#endif
