/*
 * skyrme.h -- C ABI of the GB300 arrested-Newton-flow library for the 3D
 * Skyrme model in sigma-model form (arXiv 2604.25876).
 *
 * Every compute step runs in hand-written sm_103a CUDA kernels.  The caller
 * owns all memory: field, velocity and scratch buffers are device pointers it
 * allocated (for example with PyTorch), streams are cudaStream_t values passed
 * as void*.  The library keeps no global state between calls, never allocates
 * on the flow path, and synchronises a stream only when a host-side result
 * (a report or an energy) is requested.  Errors are status codes; nothing is
 * thrown across the ABI and nothing aborts the process.
 *
 * Device: every call works on the current CUDA device.  Device buffers passed
 * to it must live on that device (or be managed or mapped host memory that it
 * can address); a buffer of another GPU, or plain host memory, is rejected
 * with SKYRME_EINVAL after the other argument checks and before any launch.
 *
 * Lattice layout (Section 7.5.1, the text/binary file formats): site (x,y,z)
 * of an n[0] x n[1] x n[2] lattice has index ((x*n[1])+y)*n[2]+z, z fastest.
 * Each site holds the 4 components (phi^0, phi^1, phi^2, phi^3) contiguously:
 * a float4 (precision 32) or double4 (precision 64).  Site coordinates are
 * x_i = (i - (n-1)/2) h.  Interior sites have every index in [2, n-3]; the two
 * outer layers hold the fixed vacuum (1,0,0,0) and a zero velocity
 * (Section 3: vacuum boundary, stencil radius 2).
 */
#ifndef SKYRME_H
#define SKYRME_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SKYRME_ABI_VERSION 5

typedef enum {
    SKYRME_OK = 0,
    SKYRME_EINVAL = 1,      /* invalid size, spacing, precision, mode, or a null/misaligned pointer */
    SKYRME_ENOMEM = 2,      /* a caller-provided buffer is smaller than required */
    SKYRME_ECUDA = 3,       /* a CUDA runtime call failed (the message is in skyrme_last_cuda_error) */
    SKYRME_ENONFINITE = 4,  /* a NaN/Inf appeared in a force, density or energy sum */
    SKYRME_ETIMEOUT = 5,    /* a bounded device-side wait gave up */
    SKYRME_EUNSUPPORTED = 6 /* the request is valid but not implemented for this precision or model */
} skyrme_status;

/* Flow equations of Section 3.  ARRESTED is the arrested Newton flow
 * (velocity zeroed whenever the static energy rises), NEWTON the same flow
 * without arrest, GRADIENT the first-order flow phi_t = F. */
typedef enum { SKYRME_NEWTON = 0, SKYRME_ARRESTED = 1, SKYRME_GRADIENT = 2 } skyrme_flow_mode;

/* The model (Section 2.1, extended by the options of Section 7.8):
 *   static energy density  e2 + e4 + e0 + e6, with
 *   e0 = 2 m^2 (1 - phi^0) + m_y^2 (1 - (phi^0)^2) + m_z^2 (1 - phi^0)^2
 *        + (1/2) m_w^2 (1 - phi^0)^4
 *        (standard pion mass, modified pion mass, loosely bound and lightly
 *        bound potentials) and
 *   e6 = c6 4 pi^4 (B0)^2  (the BPS sextic term, B0 of Eq. "B0_components").
 * All five coefficients are finite and >= 0; m_y = m_z = m_w = c6 = 0 is the
 * standard model.  A lattice with any of the four extension coefficients
 * non-zero is an "extended" lattice: the Section 5 observables reject it with
 * SKYRME_EUNSUPPORTED, and so does the batched flow when c6 != 0 (batches
 * take the standard model and the potentials).  An FP32 flow runs on the
 * streaming FP32 kernel with any of the terms; an FP64 flow runs on the tile
 * kernels. */
typedef struct {
    int n[3];       /* sites per axis (x slowest, z fastest); each >= 5 */
    double h;       /* lattice spacing, > 0, equal on every axis */
    double m;       /* pion mass of the 2 m^2 (1 - phi^0) potential (Eq. SkyrmeEnergy_phi) */
    int precision;  /* 32: float4 field and velocity, FP64 sums; 64: double4 */
    double m_y;     /* modified pion mass: m_y^2 (1 - (phi^0)^2) */
    double m_z;     /* loosely bound potential: m_z^2 (1 - phi^0)^2 */
    double m_w;     /* lightly bound potential: (1/2) m_w^2 (1 - phi^0)^4 */
    double c6;      /* BPS sextic term: c6 4 pi^4 (B0)^2 */
} skyrme_lattice;

enum {
    SKYRME_SEED_VACUUM = 0,        /* phi = (1,0,0,0) everywhere */
    SKYRME_SEED_RATIONAL_MAP = 1,  /* Section 4.1, degree B in {1, 2, 3, 4} (Table 1; the
                                      degree-3 constant a = i, tetrahedral), centred */
    SKYRME_SEED_PRODUCT = 2,       /* Section 4.2, Eq. "Product ansatz" of B isorotated hedgehogs */
    SKYRME_SEED_NOISE = 3          /* vacuum + Gaussian-smoothed N(0,1) noise in a ball, normalised */
};

typedef struct {
    int kind;                    /* SKYRME_SEED_* */
    int B;                       /* rational-map degree, or number of product constituents */
    double profile_scale;        /* profile f(r) = pi exp(-r / profile_scale), > 0 */
    const double *positions;     /* host, B x 3: constituent centres (PRODUCT) */
    const double *quaternions;   /* host, B x 4: unit (q0, q1, q2, q3), A_k = q0 + i q.tau (PRODUCT) */
    int symmetrise;              /* PRODUCT: 1 -> normalise(U_1..U_B + U_B..U_1), 0 -> U_1..U_B */
    double radius;               /* NOISE: ball radius carrying the noise */
    double sigma;                /* NOISE: Gaussian smoothing width (physical units), truncated at 4 sigma */
    uint64_t seed;               /* NOISE: SplitMix64 stream; normal number k of site s, component c
                                    uses stream values 2k and 2k+1 with k = 4 s + c (Box-Muller) */
} skyrme_seed;

/* Caller-owned device buffers of one lattice.  phi[i] and vel[i] each hold
 * n[0]*n[1]*n[2] sites (16 or 32 bytes per site) and must be 16-byte (FP32)
 * or 32-byte (FP64) aligned.  scratch holds skyrme_scratch_bytes() bytes,
 * 256-byte aligned; it carries the flow's control block (current buffer,
 * previous energy, counters) so that stepping needs no host round trip. */
typedef struct {
    void *phi[2];
    void *vel[2];
    void *scratch;
    size_t scratch_bytes;
} skyrme_state;

/* Result of the latest flow iteration, read back from the control block. */
typedef struct {
    double E, E2, E4, E0;  /* static energy of the field at the start of the
                              iteration and its quadratic, quartic and potential
                              parts (E = E2 + E4 + E0 + E6) */
    double B;              /* baryon number, Eq. "B0_components" integrated */
    double virial;         /* V = -E2 + E4 - 3 E0 + 3 E6 (Section 5.6, Derrick scaling) */
    double delta;          /* max over interior sites of |F| (the residual of Section 3) */
    double rms_force;      /* sqrt(mean |F|^2) over interior sites */
    long long steps;       /* iterations completed since the field was set */
    long long arrests;     /* iterations whose velocity was zeroed */
    long long fixups;      /* speculative updates corrected after the energy was known */
    int cur;               /* index (0/1) of the buffers holding the current field */
    int status;            /* sticky device-side status (skyrme_status) */
    double E6;             /* sextic part of E (0 without the sextic term) */
} skyrme_report;

/* ---- queries ---- */
int skyrme_abi_version(void);
const char *skyrme_status_string(int status);
/* Text of the most recent failing CUDA call made by this thread ("" if none). */
const char *skyrme_last_cuda_error(void);
/* Bytes of scratch a lattice needs (0 when the lattice is invalid). */
size_t skyrme_scratch_bytes(const skyrme_lattice *lat);

/* ---- set-up ----
 * skyrme_init_field: writes the seed field of Section 4 into phi[0] and
 * phi[1], zeroes vel[0] and vel[1], resets the control block (E_prev = +inf,
 * counters zero, cur = 0).  PRODUCT reads its host arrays before returning.
 * Asynchronous on `stream`. */
skyrme_status skyrme_init_field(const skyrme_lattice *lat, const skyrme_seed *seed,
                                skyrme_state *st, void *stream);
/* skyrme_load_field: the caller has written a field into phi[0]; it is
 * copied to phi[1], its outer layers are set to the vacuum, velocities are
 * zeroed and the control block reset, as after skyrme_init_field. */
skyrme_status skyrme_load_field(const skyrme_lattice *lat, skyrme_state *st, void *stream);

/* ---- the flow (Section 3) ----
 * nsteps iterations of `mode` with time step dt > 0.  One iteration computes
 * the 4th-order derivatives of phi_n, the Euler-Lagrange gradient G, the
 * tangent force F = -G + (G.phi) phi, the energy E_n; in ARRESTED mode the
 * velocity is zeroed when E_n > E_{n-1}; then v += dt F, phi = (phi + dt v)/|.|
 * at interior sites.  `report` (nullable, host) receives the latest
 * iteration's results, which synchronises the stream.  Returns
 * SKYRME_ENONFINITE (sticky) once a non-finite value has appeared.
 * From 256 iterations on, on a stream that is not being captured, the call
 * captures 128 iterations into a CUDA graph on a stream of its own and
 * replays it on `stream` (fewer GPU cycles per launch); the graph and that
 * stream are host and driver resources released before the call returns. */
skyrme_status skyrme_flow_step(const skyrme_lattice *lat, double dt, int nsteps, int mode,
                               skyrme_state *st, skyrme_report *report, void *stream);
/* skyrme_flow_host: one job on host data through a device state: the field
 * field_in (host; n0*n1*n2 sites of 4 components in the lattice's precision,
 * index ((x*n1)+y)*n2+z) is loaded as by skyrme_load_field (vacuum outer
 * layers, zero velocity, a fresh control block): a pinned buffer is read by
 * the load kernel over the host link, any other is copied into phi[0] first;
 * then nsteps iterations run as skyrme_flow_step runs them (Section 3),
 * and the final field is copied to field_out (host, same layout; it may be
 * field_in).  Every iteration flips the current buffers, so the result is
 * phi[nsteps & 1]; the copies are queued behind the flow on `stream` without
 * a wait in between.  `report` (nullable) as for skyrme_flow_step.  The call
 * synchronises the stream before returning.  Host buffers may be pageable;
 * pinned ones move at the host link's full rate.  SKYRME_EINVAL for a null
 * buffer or the arguments skyrme_flow_step rejects. */
skyrme_status skyrme_flow_host(const skyrme_lattice *lat, double dt, int nsteps, int mode,
                               skyrme_state *st, const void *field_in, void *field_out,
                               skyrme_report *report, void *stream);

/* ---- work split of a single FP32 lattice's step ----
 * The FP32 step streams the lattice as columns of 16 x 32 interior (y, z)
 * sites along x, one persistent CTA per SM; each site of Section 3's
 * iteration is computed the same way whatever the split, so the fields do
 * not depend on it (the energy sums' order does, by FP64 rounding).
 *   SKYRME_SPLIT_BALANCED: contiguous (column, x-plane) ranges, column by
 *     column, with about the same number of streamed planes per CTA (a run
 *     of r centres streams r + 4 planes).
 *   SKYRME_SPLIT_LOCKSTEP: waves of whole columns (CTA b streams columns
 *     b, b + G, ... for G CTAs), then the remaining columns' heads (one CTA
 *     each) beside their tails (split over the other CTAs), so that
 *     neighbouring columns are streamed at the same x and the halo rows they
 *     share come from L2 instead of DRAM.
 *   SKYRME_SPLIT_AUTO (the default): the split measured fastest, BALANCED
 *     (LOCKSTEP moves fewer DRAM bytes but ran slower on every lattice too
 *     large for L2).
 * skyrme_set_single_split sets the policy for the process (SKYRME_EINVAL for
 * another value); launches and graphs take the policy in force when they are
 * issued or captured.  skyrme_single_split returns it.
 * skyrme_single_split_runs (host only, no device needed): the runs that
 * `policy` gives an n[0] x n[1] x n[2] lattice on min(grid, units) CTAs
 * (grid <= 256): for run k, runs[4k..4k+3] = {CTA, column, first interior
 * plane, end plane (exclusive)}, column = (y tile) * ceil((n[2]-4)/32) +
 * (z tile), planes counted from the first interior plane, each CTA's runs
 * in the order it streams them.  Writes at most `cap` runs, returns the
 * number of runs (-1 for invalid arguments); *chosen (nullable) receives the
 * split taken (BALANCED or LOCKSTEP). */
typedef enum {
    SKYRME_SPLIT_AUTO = 0,
    SKYRME_SPLIT_BALANCED = 1,
    SKYRME_SPLIT_LOCKSTEP = 2
} skyrme_single_split_policy;
skyrme_status skyrme_set_single_split(int policy);
int skyrme_single_split(void);
int skyrme_single_split_runs(const int n[3], int grid, int policy, int *runs, int cap,
                             int *chosen);
/* ---- x-slab decomposition of one lattice ----
 * The step is a radius-2 stencil (Section 3: the 4th-order first, second and
 * mixed differences reach two sites along each axis), and the arrest rule
 * (Section 3) compares the static energy of the WHOLE lattice with the
 * previous iteration's.  A lattice of N sites along x can therefore be cut
 * into slabs of whole interior x-planes, each held by its own skyrme_state
 * (on its own GPU or not), if every iteration
 *   1. steps each slab with the prediction of the arrest decision that all
 *      slabs share, leaving an 8-double record of the slab's sums instead of
 *      deciding (skyrme_slab_step),
 *   2. gives every slab the records of all slabs, in slab order (an
 *      all-gather between ranks),
 *   3. makes the decision over the whole lattice in every slab and applies
 *      the arrest fix-up (skyrme_slab_finish), and
 *   4. exchanges halos: each slab's two ghost planes on a side shared with a
 *      neighbour receive that neighbour's two nearest interior planes of the
 *      new field (the buffer the state's `cur` now names: after k iterations
 *      from a load or seed, cur = k mod 2).
 * A slab's lattice is the slab's p interior planes plus two ghost planes on
 * each side: n = {p + 4, N1, N2}, with h, m, precision and the model of the
 * whole lattice.  On a side that is the whole lattice's boundary the ghost
 * planes are its two vacuum layers and never change.  The per-site results
 * are those of the whole-lattice flow (the same kernels and per-site
 * arithmetic); the energy sums differ only by summation order.  Load each
 * slab with skyrme_load_field (which writes the vacuum into all outer
 * layers), then run step 4 once before the first iteration.
 *   skyrme_slab_step: one iteration of the slab as in skyrme_flow_step, up to
 *     the decision.  `record` (device, 8-byte aligned, 8 doubles) receives
 *     {sum e2, sum e4, sum e0, sum b, sum |F|^2, max |F|^2, interior sites,
 *     sum e6} over the slab's interior sites (e0 holding the whole
 *     potential density, b the baryon density).  Asynchronous.
 *   skyrme_slab_finish: sums `nslabs` records (device, 8 doubles each, slab
 *     order; 1 <= nslabs <= 4096) in that order, forms E_n, B, the virial and
 *     delta of the whole lattice, makes the arrest decision and the report's
 *     bookkeeping in the slab's control block, and (ARRESTED mode) corrects
 *     a mispredicted decision at the slab's sites.  dt and mode must be
 *     those of the skyrme_slab_step call.  Asynchronous.
 * Both return SKYRME_EINVAL for bad arguments, as skyrme_flow_step does. */
skyrme_status skyrme_slab_step(const skyrme_lattice *slab, double dt, int mode, skyrme_state *st,
                               double *record, void *stream);
skyrme_status skyrme_slab_finish(const skyrme_lattice *slab, double dt, int mode, skyrme_state *st,
                                 const double *records, int nslabs, void *stream);

/* ---- reduction diagnostic (FP32 streaming path) ----
 * skyrme_step_densities: one iteration exactly as skyrme_flow_step runs it
 * (the FP32 streaming kernel: precision 32 and c6 = 0, else
 * SKYRME_EUNSUPPORTED), which also writes, for every interior site, the FP32
 * per-site values that this iteration's energy and charge sums add up, as a
 * float4 in the site layout: {e2, e4, u, det} with e2 = tr a, e4 of
 * Eq. "SkyrmeEnergy_phi", det = det[phi, d_x phi, d_y phi, d_z phi] (the
 * baryon density is -det / 2 pi^2, Eq. "B0_components") and u the potential
 * term (1 - phi^0 for the standard model, whose density is 2 m^2 u; the whole
 * potential density with the Section 7.8 potentials).  Other sites of `dens`
 * (device, 16-byte aligned, n[0]*n[1]*n[2] float4) are not written.  With
 * them a test can compare the iteration's reported E_n, B and virial with an
 * exact sum of the very values the kernel summed, which isolates the error
 * of the reduction.  `report` as for skyrme_flow_step.  The paper has no
 * counterpart. */
skyrme_status skyrme_step_densities(const skyrme_lattice *lat, double dt, int mode,
                                    skyrme_state *st, void *dens, skyrme_report *report,
                                    void *stream);

/* ---- the flow as a CUDA graph ----
 * skyrme_graph_create captures `nsteps` iterations exactly as
 * skyrme_flow_step launches them (the step kernel and, where it has one, the
 * arrest fix-up check) on `stream`, which must be a stream that can be captured
 * (not the legacy default stream), and instantiates the graph.  The flow
 * state lives on the device, so one graph advances the flow by nsteps
 * iterations every time it is launched, for as long as the state's buffers
 * exist.  Creation and destruction allocate host and driver resources; a
 * launch does not.  skyrme_graph_destroy releases them (NULL is accepted). */
typedef struct skyrme_graph skyrme_graph;
skyrme_status skyrme_graph_create(const skyrme_lattice *lat, double dt, int nsteps, int mode,
                                  skyrme_state *st, void *stream, skyrme_graph **out);
skyrme_status skyrme_graph_launch(skyrme_graph *g, void *stream);
skyrme_status skyrme_graph_destroy(skyrme_graph *g);

/* skyrme_graph_create_until: a graph that, on each launch, relaxes the flow
 * until it has converged, without returning to the host: a device-side WHILE
 * node repeats `chunk` iterations (as skyrme_flow_step launches them)
 * followed by a check, for as long as
 *   - the last iteration's delta = max over interior sites of |F| (the
 *     convergence residual of Sections 3 and 7.9, taken as the largest
 *     force) is above tol,
 *   - fewer than max_steps iterations have run since this launch began, and
 *   - no error has been recorded in the state.
 * The flow therefore stops at the first chunk boundary where delta <= tol,
 * or at the first one at or after max_steps; read the result with
 * skyrme_read_report.  Arguments as for skyrme_graph_create, plus tol >= 0
 * (finite), max_steps >= 1 and chunk >= 1 (SKYRME_EINVAL otherwise).  The
 * same stream-capture requirements apply. */
skyrme_status skyrme_graph_create_until(const skyrme_lattice *lat, double dt, int mode, double tol,
                                        long long max_steps, int chunk, skyrme_state *st,
                                        void *stream, skyrme_graph **out);

/* ---- batched flow (FP32) ----
 * Many independent lattices, of uneven sizes, advanced together: every step
 * is one persistent launch over all of their work (plus, in ARRESTED mode,
 * one fix-up check launch), and each lattice's energy sums and arrest
 * decision close as soon as the CTAs that touched it are done.  Each lattice
 * keeps its own skyrme_state (initialise it with skyrme_init_field or
 * skyrme_load_field; read its results with skyrme_read_report).  Lattices
 * may differ in size, spacing, pion mass and Section 7.8 potentials; the
 * sextic term is not taken (SKYRME_EUNSUPPORTED).
 *   skyrme_batch_scratch_bytes: size of the caller-owned batch scratch
 *     (lattice table, the CTAs' unit ranges of a balanced split and per-CTA
 *     partial records), 256-byte aligned.
 *   skyrme_batch_create: validates the states (precision 32 only), encodes
 *     the lattice table for the default tile shape and uploads it (a
 *     synchronous copy); the handle owns no device memory.
 *   skyrme_batch_step: nsteps iterations, asynchronous.
 *   skyrme_batch_autotune: times every candidate tile shape, each with both
 *     work splits, on these lattices with `trials` dry steps each (outputs
 *     go to the inactive buffers; the flows do not advance) and keeps the
 *     fastest pair; best_tile is its tile shape.
 *   skyrme_batch_set_tile / skyrme_batch_tile: choose or query the tile
 *     shape (0: 8x32, 1: 4x32, 2: 16x16, 3: 8x16, 4: 16x32 interior sites per CTA) and
 *     the persistent grid.
 *   skyrme_batch_set_split / skyrme_batch_split: how the (column, x-plane)
 *     work of the concatenated lattices is divided among the persistent
 *     CTAs: balanced = 1 (the default) gives each CTA about the same number
 *     of streamed planes (a run of r centres streams r + 4), balanced = 0
 *     the same number of centres.  Results are the same either way (each
 *     site's arithmetic does not depend on the split; the sums' order
 *     does).  Both re-encode the table (a synchronous copy): re-capture
 *     graphs afterwards.
 *   skyrme_batch_graph_create: capture nsteps batched iterations as a
 *     skyrme_graph (launch and destroy it with skyrme_graph_launch /
 *     skyrme_graph_destroy).  Re-capture after changing the tile shape. */
typedef struct skyrme_batch skyrme_batch;
size_t skyrme_batch_scratch_bytes(int ninst, const skyrme_lattice *lats);
skyrme_status skyrme_batch_create(int ninst, const skyrme_lattice *lats, skyrme_state *states,
                                  const double *dt, int mode, void *scratch, size_t scratch_bytes,
                                  skyrme_batch **out);
skyrme_status skyrme_batch_step(skyrme_batch *b, int nsteps, void *stream);
skyrme_status skyrme_batch_autotune(skyrme_batch *b, int trials, void *stream, int *best_tile,
                                    double *best_ms);
skyrme_status skyrme_batch_set_tile(skyrme_batch *b, int tile);
skyrme_status skyrme_batch_set_split(skyrme_batch *b, int balanced);
skyrme_status skyrme_batch_split(const skyrme_batch *b, int *balanced);
skyrme_status skyrme_batch_tile(const skyrme_batch *b, int *tile, int *ty, int *tz, int *grid);
skyrme_status skyrme_batch_graph_create(skyrme_batch *b, int nsteps, void *stream,
                                        skyrme_graph **out);
skyrme_status skyrme_batch_destroy(skyrme_batch *b);

/* Copy the control block to the host (synchronises the stream). */
skyrme_status skyrme_read_report(const skyrme_lattice *lat, const skyrme_state *st,
                                 skyrme_report *report, void *stream);

/* ---- reductions of the current field (synchronise the stream) ----
 * out6 = {E, E2, E4, E0, B, V}: h^3 times FP64 sums over interior sites of
 * the densities of Eq. SkyrmeEnergy_phi (with the model's e0 and e6) and
 * Eq. B0_components; E and V include the sextic part, which
 * skyrme_sextic_energy returns on its own. */
skyrme_status skyrme_energy(const skyrme_lattice *lat, skyrme_state *st, double out6[6],
                            void *stream);
skyrme_status skyrme_baryon_number(const skyrme_lattice *lat, skyrme_state *st, double *B,
                                   void *stream);
skyrme_status skyrme_virial(const skyrme_lattice *lat, skyrme_state *st, double *V,
                            void *stream);
skyrme_status skyrme_sextic_energy(const skyrme_lattice *lat, skyrme_state *st, double *E6,
                                   void *stream);

/* ---- Section 5 observables of the current field ----
 * skyrme_observables: h^3-weighted sums over interior sites of
 *   B        the baryon number (Eq. "B0_components");
 *   X        the centre of mass, Eq. "CoM" (x_i = (i - (n_i - 1)/2) h);
 *   R        the RMS radius, Eq. "RMS radius", about X;
 *   Q        the quadrupole tensor, Eq. "Q tensor", with rho = B0/2;
 *   U, V, W  the isospin, spin and mixed inertia tensors, Eqs. "U/V/W
 *            inertia tensor" (W[i][j]: i isospin, j space); the lattice
 *            current L_k is the traceless part of U^dagger d_k U;
 *   D        the monopole D-term, Eq. "D-term", about X;
 *   E        the static energy used by D (Eq. "SkyrmeEnergy_phi").
 * All moments are taken about X.  Two passes over the field in FP64 (whatever
 * its precision), in a fixed order; uses the state's scratch; synchronises
 * `stream`.  SKYRME_EINVAL when B is 0 (no centre of mass), SKYRME_ENONFINITE
 * when a sum is not finite; `out` is zeroed in both cases. */
typedef struct {
    double B, X[3], R, Q[3][3], U[3][3], V[3][3], W[3][3], D, E;
} skyrme_observables_t;
skyrme_status skyrme_observables(const skyrme_lattice *lat, skyrme_state *st,
                                 skyrme_observables_t *out, void *stream);

/* ---- headless volume render of the baryon density (Section 6.2) ----
 * The paper ray-traces B0 in an OpenGL viewer; here the picture is written to
 * a caller-owned device RGBA buffer (one float4 per pixel, each channel in
 * [0, 1], rows from the bottom of the image, y up).
 *
 * skyrme_render_volume: the volume of the current field, one record of four
 *   doubles per site in the field's site order: {B0 / max B0, pion / |pion|}.
 *   B0 is the lattice baryon density of Eq. "B0_components" at interior
 *   sites and 0 on the two boundary layers; max B0 is taken over the lattice,
 *   and B0 / max B0 is 0 everywhere when max B0 <= 0.  The pion unit vector
 *   (phi_1, phi_2, phi_3) / |pion| is 0 where the pion is 0.  `vol` is a
 *   device buffer of at least skyrme_render_volume_bytes(lat) bytes, 32-byte
 *   aligned, owned by the caller.  Uses the state's scratch; asynchronous.
 *
 * skyrme_render_rays: ray-march a volume of that layout (device, n[0]*n[1]*n[2]
 *   records, 32-byte aligned, n[i] >= 2) into `rgba` (device, width*height
 *   float4, 16-byte aligned, owned by the caller).  Camera and box:
 *   - the lattice box is scaled so that its longest axis spans [-1, 1], lattice
 *     coordinate g mapping to (g - (n-1)/2) / s, s = max (n_i - 1)/2;
 *   - the eye is at (0, 0, 4) in view space; pixel (u, v) in [-aspect, aspect]
 *     x [-1, 1] looks along (u, v, -2); `view` is the row-major rotation that
 *     takes view-space vectors to box space;
 *   - samples at t = t_near + k step along the unit ray inside the box take a
 *     trilinear interpolation of all four components, clamped to the lattice;
 *   - input = (b - levelset) transfer_scale, skipped when negative; colour =
 *     input^2 (pion_1, pion_2, pion_3, 1 / input), composited front to back
 *     (sum += colour (1 - sum_alpha)), stopping once sum_alpha > 0.95;
 *   - the pixel is sum * brightness clamped to [0, 1].
 *   SKYRME_EINVAL for width or height < 1, more than SKYRME_RENDER_MAX_PIXELS
 *   pixels, step outside [SKYRME_RENDER_MIN_STEP, 1], non-finite values, a
 *   view that is not a rotation (rows orthonormal to 1e-9), or null or
 *   misaligned pointers.  Asynchronous.
 *
 * skyrme_render: skyrme_render_volume into `work` followed by
 *   skyrme_render_rays. */
#define SKYRME_RENDER_MAX_PIXELS (1LL << 26)
#define SKYRME_RENDER_MIN_STEP 1e-4
typedef struct {
    int width, height;
    double view[9];
    double levelset, transfer_scale, brightness, step;
} skyrme_render_params;
size_t skyrme_render_volume_bytes(const skyrme_lattice *lat);
skyrme_status skyrme_render_volume(const skyrme_lattice *lat, skyrme_state *st, void *vol,
                                   size_t vol_bytes, void *stream);
skyrme_status skyrme_render_rays(const int n[3], const void *vol,
                                 const skyrme_render_params *params, float *rgba, void *stream);
skyrme_status skyrme_render(const skyrme_lattice *lat, skyrme_state *st,
                            const skyrme_render_params *params, void *work, size_t work_bytes,
                            float *rgba, void *stream);

/* ---- per-site values of the current field (asynchronous) ----
 * force (device, nullable): F at interior sites, 0 on the boundary layers,
 * same site layout and precision as phi.  dens (device, nullable): per site
 * {e2, e4, e0, b} in the same precision (e0 the model's whole potential; the
 * sextic density is c6 4 pi^4 b^2). */
skyrme_status skyrme_forces(const skyrme_lattice *lat, skyrme_state *st, void *force,
                            void *dens, void *stream);

/* ---- allocation-free variant ----
 * skyrme_energy_static: the six values of skyrme_energy (E, E2, E4, E0, B, V)
 * for the field `phi` (device; n[0]*n[1]*n[2] sites in the layout and
 * precision described above), for callers that cannot allocate device memory:
 * for example code whose device memory is all owned by a host application's
 * own pool, or a plug-in that may only use the buffers it is handed.  It needs
 * no skyrme_state and no scratch buffer: its scratch is a fixed 128 KiB array
 * inside the library, which every GPU that loads the library keeps until the
 * process exits.  The paper has no counterpart; this is a packaging variant of
 * the reduction above.
 *   - Lattices with more than 2048 interior x-planes (n[0] - 4 > 2048) do not
 *     fit the array and are rejected with SKYRME_EINVAL, as are misaligned or
 *     null pointers.
 *   - `phi` must be on the current device (SKYRME_EINVAL otherwise).  Every
 *     call looks up the array's device address in the current context (a
 *     host-side lookup that allocates nothing), so a context that was reset
 *     or replaced under the same device never receives a stale address.
 *   - Every call on a device shares the array and leaves its contents behind;
 *     each call clears what must start at zero.  Calls that overlap on the
 *     GPU (on other streams or host threads) race, so the caller serialises
 *     them.
 *   - It allocates nothing (no cudaMalloc or cudaFree, no library allocator)
 *     and synchronises `stream` to return the values on the host. */
skyrme_status skyrme_energy_static(const skyrme_lattice *lat, const void *phi, double out6[6],
                                   void *stream);

/* ---- measurement diagnostic ----
 * skyrme_measure_fma_peak: the device's fused multiply-add throughput in
 * TFLOP/s (an FMA counts as 2 operations), measured by timing long chains of
 * independent FMAs on every SM: kind SKYRME_PEAK_FP32 uses the packed FP32
 * pair instruction the FP32 step kernel uses, SKYRME_PEAK_FP64 the FP64 FMA.
 * These are the ALU roofline denominators of the step kernels; the paper has
 * no counterpart.  Launches a few kernels on `stream` (about 1 ms) and
 * synchronises it.  SKYRME_EINVAL for another kind or a null pointer. */
typedef enum { SKYRME_PEAK_FP32 = 0, SKYRME_PEAK_FP64 = 1 } skyrme_peak_kind;
skyrme_status skyrme_measure_fma_peak(int kind, double *tflops, void *stream);

/* ---- failure detection ----
 * skyrme_selftest_wait: exercises the bounded device-side wait that the step
 * kernels use on their TMA plane copies.  One thread waits on a shared-memory
 * mbarrier that nothing completes, gives up after limit_seconds
 * (0 < limit_seconds <= 10, else SKYRME_EINVAL) and records the timeout in
 * the state's control block, as a step kernel does when a copy never lands.
 * Synchronises `stream` and returns the recorded status: SKYRME_ETIMEOUT.
 * The status is sticky in the state (flow calls and skyrme_read_report see
 * it) until skyrme_init_field or skyrme_load_field resets the control block;
 * the CUDA context stays usable. */
skyrme_status skyrme_selftest_wait(const skyrme_lattice *lat, skyrme_state *st,
                                   double limit_seconds, void *stream);

#ifdef __cplusplus
}
#endif
#endif
