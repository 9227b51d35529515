// observables.cu -- Section 5 observables of the current field: centre of
// mass (Eq. "CoM"), RMS radius (Eq. "RMS radius"), quadrupole (Eq. "Q tensor"
// with rho = B0 / 2), the inertia tensors U, V, W (Eqs. "U/V/W inertia
// tensor") and the monopole D-term (Eq. "D-term").
//
// The paper writes these with su(2) currents.  For U = phi^0 + i phi^a tau^a
// they reduce to 4-vector algebra with
//   d_k       the tangent part of the lattice derivative, d_k phi - (phi . d_k phi) phi
//             (the lattice L_k = U^dagger d_k U is taken as its traceless part),
//   A_ij      = d_i . d_j,
//   K_a       = (0, e_a x pi)                      (isorotation about axis a),
//   G_b       = -sum_nl eps_bnl r_n d_l             (rotation about axis b, r = x - X_c),
// as
//   U_ab = 2 sum [K_a.K_b (1 + tr A) - sum_k (K_a.d_k)(K_b.d_k)],
//   V_ab = the same with G_a, G_b,
//   W_ab = -2 sum [K_a.G_b (1 + tr A) - sum_k (K_a.d_k)(G_b.d_k)],
//   T_ij = 2 A_ij (1 + tr A) - 2 (A A)_ij - delta_ij (tr A + (tr^2 A - tr A^2)/2 + e0),
// which is what T = a U a/2 + b V b/2 - a W b means for the kinetic energy of
// the model's Lagrangian.  The baryon density and the energy density are those
// of the flow (Eqs. "B0_components" and "SkyrmeEnergy_phi" with the lattice
// derivatives).  All arithmetic is FP64 whatever the field's precision; the
// sums run in a fixed order (persistent CTAs, one partial record each, then
// one CTA summing the records), so repeated calls are bitwise equal.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "lattice_sites.cuh"
#include "skyrme_device.cuh"
#include "skyrme_internal.h"

namespace skyrme {

constexpr int kObsCtas = 152;
constexpr int kObsThreads = 256;
constexpr int kObsSums = 32;  // doubles per record

// record layout
enum {
    O_B = 0, O_XB = 1,  // pass 0: b, x b, y b, z b
    O_E = 0, O_R2B = 1, O_Q = 2, O_U = 8, O_V = 14, O_W = 20, O_D = 29,  // pass 1
};

template <typename T> struct ObsArgs {
    const vec4_t<T> *phi[2];
    const Ctrl *ctrl;
    double *parts;  // kObsCtas records of kObsSums doubles, then the totals
    int n0, n1, n2;
    double w1, w2;  // first-derivative weights / h
    double h, m;
    double X[3];    // centre of mass (pass 1)
};

template <typename T, int PASS>
__global__ void __launch_bounds__(kObsThreads) k_observables(ObsArgs<T> a)
{
    const int cur = __ldcg(&a.ctrl->cur);
    const vec4_t<T> *phi = cur ? a.phi[1] : a.phi[0];
    const int ix = a.n0 - 4, iy = a.n1 - 4, iz = a.n2 - 4;
    const long long total = (long long)ix * iy * iz;
    const size_t sx = (size_t)a.n1 * a.n2, sy = (size_t)a.n2;
    double acc[kObsSums];
#pragma unroll
    for (int q = 0; q < kObsSums; ++q) acc[q] = 0.0;

    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < total;
         s += (long long)gridDim.x * blockDim.x) {
        const int z = 2 + (int)(s % iz);
        const int y = 2 + (int)((s / iz) % iy);
        const int x = 2 + (int)(s / ((long long)iz * iy));
        const size_t c = x * sx + y * sy + z;
        double ph[4], d[3][4];
        load_site(phi, c, ph);
        site_first_derivatives(phi, c, sx, sy, a.w1, a.w2, d);
        const double b = baryon_density(ph, d);
        const double xv[3] = {((double)x - 0.5 * (a.n0 - 1)) * a.h, ((double)y - 0.5 * (a.n1 - 1)) * a.h,
                              ((double)z - 0.5 * (a.n2 - 1)) * a.h};
        if (PASS == 0) {
            acc[O_B] += b;
#pragma unroll
            for (int i = 0; i < 3; ++i) acc[O_XB + i] += xv[i] * b;
            continue;
        }
        // energy density of the flow (raw lattice derivatives)
        double ar[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                ar[i][j] = d[i][0] * d[j][0] + d[i][1] * d[j][1] + d[i][2] * d[j][2] + d[i][3] * d[j][3];
        const double tra_r = ar[0][0] + ar[1][1] + ar[2][2];
        double sq_r = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) sq_r += ar[i][j] * ar[i][j];
        const double e0 = 2.0 * a.m * a.m * (1.0 - ph[0]);
        acc[O_E] += tra_r + 0.5 * (tra_r * tra_r - sq_r) + e0;
        // tangent derivatives and their products
        double dt[3][4], A[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double pk = ph[0] * d[k][0] + ph[1] * d[k][1] + ph[2] * d[k][2] + ph[3] * d[k][3];
#pragma unroll
            for (int c4 = 0; c4 < 4; ++c4) dt[k][c4] = d[k][c4] - pk * ph[c4];
        }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                A[i][j] = dt[i][0] * dt[j][0] + dt[i][1] * dt[j][1] + dt[i][2] * dt[j][2] + dt[i][3] * dt[j][3];
        const double trA = A[0][0] + A[1][1] + A[2][2];
        const double one_tr = 1.0 + trA;
        double r[3], r2 = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            r[i] = xv[i] - a.X[i];
            r2 += r[i] * r[i];
        }
        acc[O_R2B] += r2 * b;
        // Q_ij, symmetric: xx yy zz xy xz yz
        {
            const int qi[6] = {0, 1, 2, 0, 0, 1}, qj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
            for (int t = 0; t < 6; ++t)
                acc[O_Q + t] += (3.0 * r[qi[t]] * r[qj[t]] - (qi[t] == qj[t] ? r2 : 0.0)) * 0.5 * b;
        }
        // generators: K_a = (0, e_a x pi), G_b = -sum eps_bnl r_n d_l
        double K[3][4], G[3][4];
        {
            const double pi1 = ph[1], pi2 = ph[2], pi3 = ph[3];
            K[0][0] = 0.0, K[0][1] = 0.0, K[0][2] = -pi3, K[0][3] = pi2;
            K[1][0] = 0.0, K[1][1] = pi3, K[1][2] = 0.0, K[1][3] = -pi1;
            K[2][0] = 0.0, K[2][1] = -pi2, K[2][2] = pi1, K[2][3] = 0.0;
#pragma unroll
            for (int c4 = 0; c4 < 4; ++c4) {
                // -(e_b x r) . d: (e_x x r) = (0, -r_z, r_y), (e_y x r) = (r_z, 0, -r_x), (e_z x r) = (-r_y, r_x, 0)
                G[0][c4] = -(-r[2] * dt[1][c4] + r[1] * dt[2][c4]);
                G[1][c4] = -(r[2] * dt[0][c4] - r[0] * dt[2][c4]);
                G[2][c4] = -(-r[1] * dt[0][c4] + r[0] * dt[1][c4]);
            }
        }
        double Kd[3][3], Gd[3][3];  // K_a . d_k, G_b . d_k
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                Kd[i][k] = K[i][0] * dt[k][0] + K[i][1] * dt[k][1] + K[i][2] * dt[k][2] + K[i][3] * dt[k][3];
                Gd[i][k] = G[i][0] * dt[k][0] + G[i][1] * dt[k][1] + G[i][2] * dt[k][2] + G[i][3] * dt[k][3];
            }
        {
            const int qi[6] = {0, 1, 2, 0, 0, 1}, qj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
            for (int t = 0; t < 6; ++t) {
                const int i = qi[t], j = qj[t];
                const double kk = K[i][0] * K[j][0] + K[i][1] * K[j][1] + K[i][2] * K[j][2] + K[i][3] * K[j][3];
                const double gg = G[i][0] * G[j][0] + G[i][1] * G[j][1] + G[i][2] * G[j][2] + G[i][3] * G[j][3];
                acc[O_U + t] += 2.0 * (kk * one_tr - (Kd[i][0] * Kd[j][0] + Kd[i][1] * Kd[j][1] + Kd[i][2] * Kd[j][2]));
                acc[O_V + t] += 2.0 * (gg * one_tr - (Gd[i][0] * Gd[j][0] + Gd[i][1] * Gd[j][1] + Gd[i][2] * Gd[j][2]));
            }
        }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const double kg = K[i][0] * G[j][0] + K[i][1] * G[j][1] + K[i][2] * G[j][2] + K[i][3] * G[j][3];
                acc[O_W + 3 * i + j] -= 2.0 * (kg * one_tr - (Kd[i][0] * Gd[j][0] + Kd[i][1] * Gd[j][1] + Kd[i][2] * Gd[j][2]));
            }
        // stress tensor of the static field and the D-term integrand
        {
            double AA[3][3], sqA = 0.0;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    AA[i][j] = A[i][0] * A[0][j] + A[i][1] * A[1][j] + A[i][2] * A[2][j];
                    sqA += A[i][j] * A[i][j];
                }
            const double lag = -(trA + 0.5 * (trA * trA - sqA) + e0);
            double rTr = 0.0, Tkk = 0.0;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const double Tij = 2.0 * A[i][j] * one_tr - 2.0 * AA[i][j] + (i == j ? lag : 0.0);
                    rTr += r[i] * r[j] * Tij;
                    if (i == j) Tkk += Tij;
                }
            acc[O_D] += rTr - r2 * Tkk / 3.0;
        }
    }

    // block sums in a fixed order: each warp by shuffles, then warp 0 over the warps
    __shared__ double red[kObsThreads / 32][kObsSums];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kObsSums; ++q) {
        double v = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < kObsSums) {
        double v = 0.0;
        for (int w = 0; w < kObsThreads / 32; ++w) v += red[w][threadIdx.x];
        a.parts[(size_t)blockIdx.x * kObsSums + threadIdx.x] = v;
    }
}

// totals[q] = sum over the records in record order
__global__ void k_observables_total(double *parts, int nrec)
{
    const int q = threadIdx.x;
    if (q >= kObsSums) return;
    double v = 0.0;
    for (int i = 0; i < nrec; ++i) v += parts[(size_t)i * kObsSums + q];
    parts[(size_t)nrec * kObsSums + q] = v;
}

template <typename T>
static skyrme_status run_pass(int pass, ObsArgs<T> a, double *host_tot, cudaStream_t s)
{
    if (pass == 0)
        k_observables<T, 0><<<kObsCtas, kObsThreads, 0, s>>>(a);
    else
        k_observables<T, 1><<<kObsCtas, kObsThreads, 0, s>>>(a);
    if (cudaGetLastError() != cudaSuccess) return SKYRME_ECUDA;
    k_observables_total<<<1, 32, 0, s>>>(a.parts, kObsCtas);
    if (cudaGetLastError() != cudaSuccess) return SKYRME_ECUDA;
    if (cudaMemcpyAsync(host_tot, a.parts + (size_t)kObsCtas * kObsSums, kObsSums * sizeof(double),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return SKYRME_ECUDA;
    return SKYRME_OK;
}

template <typename T>
static skyrme_status observables_impl(const skyrme_lattice &lat, const FlowArgs &fa,
                                      skyrme_observables_t *out, cudaStream_t s)
{
    ObsArgs<T> a;
    a.phi[0] = static_cast<const vec4_t<T> *>(fa.phi[0]);
    a.phi[1] = static_cast<const vec4_t<T> *>(fa.phi[1]);
    a.ctrl = static_cast<const Ctrl *>(fa.ctrl);
    a.parts = fa.energy_parts;
    a.n0 = lat.n[0];
    a.n1 = lat.n[1];
    a.n2 = lat.n[2];
    a.w1 = 2.0 / 3.0 / lat.h;
    a.w2 = -1.0 / 12.0 / lat.h;
    a.h = lat.h;
    a.m = lat.m;
    a.X[0] = a.X[1] = a.X[2] = 0.0;
    const double h3 = lat.h * lat.h * lat.h;
    double tot[kObsSums];
    skyrme_status rc = run_pass<T>(0, a, tot, s);
    if (rc != SKYRME_OK) return rc;
    out->B = h3 * tot[O_B];
    if (!(out->B != 0.0) || !isfinite(out->B)) {
        // no baryon density: no centre of mass to take moments about
        memset(out, 0, sizeof(*out));
        return isfinite(tot[O_B]) ? SKYRME_EINVAL : SKYRME_ENONFINITE;
    }
    for (int i = 0; i < 3; ++i) a.X[i] = out->X[i] = h3 * tot[O_XB + i] / out->B;
    rc = run_pass<T>(1, a, tot, s);
    if (rc != SKYRME_OK) return rc;
    out->E = h3 * tot[O_E];
    out->R = sqrt(h3 * tot[O_R2B] / out->B);
    const int qi[6] = {0, 1, 2, 0, 0, 1}, qj[6] = {0, 1, 2, 1, 2, 2};
    for (int t = 0; t < 6; ++t) {
        out->Q[qi[t]][qj[t]] = out->Q[qj[t]][qi[t]] = h3 * tot[O_Q + t];
        out->U[qi[t]][qj[t]] = out->U[qj[t]][qi[t]] = h3 * tot[O_U + t];
        out->V[qi[t]][qj[t]] = out->V[qj[t]][qi[t]] = h3 * tot[O_V + t];
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) out->W[i][j] = h3 * tot[O_W + 3 * i + j];
    out->D = -2.0 * out->E / 5.0 * h3 * tot[O_D];
    if (!isfinite(out->E) || !isfinite(out->D) || !isfinite(out->R)) return SKYRME_ENONFINITE;
    return SKYRME_OK;
}

skyrme_status compute_observables(const skyrme_lattice &lat, const FlowArgs &a,
                                  skyrme_observables_t *out, cudaStream_t s)
{
    return lat.precision == 64 ? observables_impl<double>(lat, a, out, s)
                               : observables_impl<float>(lat, a, out, s);
}

size_t observables_parts_bytes() { return (size_t)(kObsCtas + 1) * kObsSums * sizeof(double); }

}  // namespace skyrme
