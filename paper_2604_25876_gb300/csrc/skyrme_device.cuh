// skyrme_device.cuh -- device-side building blocks shared by the kernels of
// the arrested-Newton-flow library: vector types, the control block that
// carries the flow state across launches, the per-site physics (Section 3,
// Eq. "Sigma model EL equations", Eq. "Newton_flow"; Section 2.1,
// Eq. "SkyrmeEnergy_phi", Eq. "B0_components") and the deterministic block
// reductions.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace skyrme {

// ---------------------------------------------------------------- vectors
// One lattice site: 4 components, 16 bytes (float4) or 32 bytes (dvec4).
struct __align__(32) dvec4 {
    double x, y, z, w;
};
template <typename T> struct V4;
template <> struct V4<float> { using type = float4; };
template <> struct V4<double> { using type = dvec4; };
template <typename T> using vec4_t = typename V4<T>::type;

template <typename T> __device__ __forceinline__ vec4_t<T> load4(const vec4_t<T> *p);
template <> __device__ __forceinline__ float4 load4<float>(const float4 *p) { return *p; }
template <> __device__ __forceinline__ dvec4 load4<double>(const dvec4 *p)
{
    const double2 *q = reinterpret_cast<const double2 *>(p);
    const double2 a = q[0], b = q[1];
    return dvec4{a.x, a.y, b.x, b.y};
}
template <typename T> __device__ __forceinline__ void store4(vec4_t<T> *p, vec4_t<T> v);
template <> __device__ __forceinline__ void store4<float>(float4 *p, float4 v) { *p = v; }
template <> __device__ __forceinline__ void store4<double>(dvec4 *p, dvec4 v)
{
    double2 *q = reinterpret_cast<double2 *>(p);
    q[0] = make_double2(v.x, v.y);
    q[1] = make_double2(v.z, v.w);
}

template <typename T> __device__ __forceinline__ vec4_t<T> make4(T a, T b, T c, T d);
template <> __device__ __forceinline__ float4 make4<float>(float a, float b, float c, float d)
{
    return make_float4(a, b, c, d);
}
template <> __device__ __forceinline__ dvec4 make4<double>(double a, double b, double c, double d)
{
    return dvec4{a, b, c, d};
}

// ---------------------------------------------------------- control block
// Lives at the start of the caller's scratch buffer.  Written by the last
// CTA of each step launch; read by the next launch.
struct Ctrl {
    double E_prev;        // energy of the previous iteration's start field
    double last[8];       // E, E2, E4, E0, B, virial, delta, rms |F|
    long long steps;
    long long arrests;
    long long fixups;
    int cur;              // buffers holding the current field
    int pred;             // predicted arrest of the next iteration
    int fix;              // 0, or +1/-1: velocity correction the fix-up applies
    int status;           // sticky status (0 or an error code)
    unsigned int done;    // arrival counter of the step launch
    unsigned int edone;   // arrival counter of the energy launch
    double energy[8];     // E, E2, E4, E0, B, V, max|F|, rms|F| of skyrme_energy
    int hist;             // last 4 arrest decisions (bit 0 = latest)
    int pad_i;
    unsigned char pht[16];  // 2-bit saturating counters indexed by hist
    long long until_start;  // steps when a run-to-tolerance graph launch began
    double e6_last;         // sextic energy of the latest iteration's start field
    double e6_energy;       // sextic energy of skyrme_energy
};
static_assert(sizeof(Ctrl) <= 512, "control block must fit its 512-byte slot");
static_assert(offsetof(Ctrl, pht) % 16 == 0, "pht is read as one 16-byte word");

constexpr int kCtrlBytes = 512;
constexpr int kPartialDoubles = 8;  // per CTA: e2, e4, e0, b, sum|F|^2, max|F|^2, nsites, e6

enum Mode { MODE_NEWTON = 0, MODE_ARRESTED = 1, MODE_GRADIENT = 2 };
enum DevStatus { DEV_OK = 0, DEV_NONFINITE = 4, DEV_TIMEOUT = 5 };

// --------------------------------------------------------- stencil weights
// Section 3: first derivative (-phi_{+2} + 8 phi_{+1} - 8 phi_{-1} + phi_{-2})/(12 h),
// second derivative (-phi_{+2} + 16 phi_{+1} - 30 phi_0 + 16 phi_{-1} - phi_{-2})/(12 h^2),
// mixed derivative: first-derivative stencil along i of the one along j.
template <typename T> struct W {
    static constexpr T c1 = T(2) / T(3);
    static constexpr T c2 = T(-1) / T(12);
    static constexpr T s1 = T(4) / T(3);
    static constexpr T s2 = T(-1) / T(12);
    static constexpr T s0 = T(-5) / T(2);
};

// Unscaled symmetric stencils on scalars: fd1 = c1 (p1 - m1) + c2 (p2 - m2)
template <typename T>
__device__ __forceinline__ T fd1(T m2v, T m1v, T p1v, T p2v)
{
    return W<T>::c1 * (p1v - m1v) + W<T>::c2 * (p2v - m2v);
}
template <typename T>
__device__ __forceinline__ T fd2(T m2v, T m1v, T c, T p1v, T p2v)
{
    return W<T>::s1 * (p1v + m1v) + W<T>::s2 * (p2v + m2v) + W<T>::s0 * c;
}

// ------------------------------------------------------ 1 - phi^0
// 1 - phi^0 of a unit 4-vector, the variable of the pion-mass potential
// (Eq. "SkyrmeEnergy_phi") and of the Section 7.8 potentials.  Near the
// vacuum phi^0 -> 1 and the difference cancels: an FP32 phi^0 holds it only to
// its spacing of 6e-8 next to 1, and over a large near-vacuum lattice those
// per-site errors add up to a bias of the potential energy (2e-4 of E ~ 10 on
// a 112^3 lattice with h = 0.15).  In FP32 it is therefore taken, for
// phi^0 >= 0, as |pi|^2 / (1 + phi^0) with pi = (phi^1, phi^2, phi^3), which
// FP32 holds to full relative precision; for phi^0 < 0 there is no
// cancellation.  FP64 uses the difference as written.
// Reciprocal on the special-function unit (at most 1 ulp from 1/x for
// normal x); the denominators it gets here lie in [1, 2].
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
template <typename T> __device__ __forceinline__ T one_minus_phi0(const T phi[4])
{
    if constexpr (sizeof(T) == 4) {
        const T pi2 = phi[1] * phi[1] + phi[2] * phi[2] + phi[3] * phi[3];
        return phi[0] >= T(0) ? pi2 * rcp_approx(T(1) + phi[0]) : T(1) - phi[0];
    } else {
        return T(1) - phi[0];
    }
}
// 1 - (phi^0)^2 = u (2 - u) with u = 1 - phi^0 (same reasoning)
template <typename T> __device__ __forceinline__ T one_minus_phi0_sq(const T phi[4], T u)
{
    if constexpr (sizeof(T) == 4) return u * (T(2) - u);
    else return T(1) - phi[0] * phi[0];
}

// ------------------------------------------------------ extension models
// Section 7.8 options beyond the standard pion mass: squared masses of the
// modified pion, loosely and lightly bound potentials and the sextic
// coefficient.
template <typename T> struct ExtModel {
    T my2, mz2, mw2, c6;
};

// Scales of the unscaled derivatives the tile kernels carry: u_i = 12h d_i phi
// and N_ij = -12h^2 d_ij phi, so d_i phi = k1 u_i with k1 = 1/(12h).
template <typename T> struct StencilScale {
    T k1sq, k1cu, k1qu, k1sx;  // k1^2, k1^3, k1^4, k1^6
    T B;                       // k1^2 / (12h^2) = 12 k1^4 = 1/(1728 h^4)
    T K144;                    // 144 h^2 = 1/k1^2
};

// Adds the extension terms to the Euler-Lagrange gradient G (before the
// tangent projection); returns their potential density in e0x, the sextic
// density in e6 and 1 - phi^0 in u.
//   potentials: d/dphi^0 of m_y^2 (1 - phi0^2) + m_z^2 u^2 + m_w^2 u^4 / 2, u = 1 - phi0;
//   sextic, with D = det[phi, u, v, w] (u, v, w = d_x, d_y, d_z phi) and
//   e6 = c6 4 pi^4 (B0)^2 = c6 D^2: the Euler-Lagrange operator of c6 D^2 is
//     2 c6 [ 4 D P - sum_i (d_i D) Q_i ],  P = dD/dphi, Q_i = dD/d(d_i phi),
//   d_i D = sum_j Q_j . d_i d_j phi.  The 4 D P collects D P and the divergence
//   of the cofactors, sum_i d_i Q_i = -3 P (the d_i d_j phi parts cancel in
//   pairs because d_i d_j = d_j d_i on the lattice too).
// P and the Q_i are the cofactor rows of M = [phi; d_x phi; d_y phi; d_z phi],
// formed from the 2x2 minors s_AB of the rows (phi, d_x phi) and c_AB of
// (d_y phi, d_z phi) (AB = 01, 02, 03, 12, 13, 23) that the charge density's
// determinant D = det M uses too, three products each.  Here in the unscaled
// derivatives u, N (StencilScale): D, P, Q_i carry k1^3, k1^3, k1^2 and d_i D
// carries -k1^2/(12h^2) = -12 k1^4, so the bracket is k1^6 [4 D P + 12 sum_i
// dD_i Q_i] in the unscaled values.
template <typename T>
__device__ __forceinline__ void extension_terms(const T phi[4], const T d1[3][4], const T d2[3][4],
                                                const T dm[3][4], const ExtModel<T> &x,
                                                const StencilScale<T> &sc, const T (&sm)[6],
                                                const T (&cm)[6], T D, T G[4], T &e0x, T &e6,
                                                T &u)
{
    u = one_minus_phi0<T>(phi);
    const T u2 = u * u;
    G[0] -= T(2) * (x.my2 * phi[0] + x.mz2 * u + x.mw2 * u2 * u);
    e0x = x.my2 * one_minus_phi0_sq<T>(phi, u) + x.mz2 * u2 + T(0.5) * x.mw2 * u2 * u2;
    e6 = T(0);
    // potentials only (a uniform branch): the FP64 kernels skip the sextic
    // arithmetic; FP32 flows without the sextic term run on the streaming kernel
    if constexpr (sizeof(T) == 8)
        if (x.c6 == T(0)) return;
    const T s01 = sm[0], s02 = sm[1], s03 = sm[2], s12 = sm[3], s13 = sm[4], s23 = sm[5];
    const T c01 = cm[0], c02 = cm[1], c03 = cm[2], c12 = cm[3], c13 = cm[4], c23 = cm[5];
    const T *p = phi, *uu = d1[0], *v = d1[1], *w = d1[2];
    const T P[4] = {uu[1] * c23 - uu[2] * c13 + uu[3] * c12, -uu[0] * c23 + uu[2] * c03 - uu[3] * c02,
                    uu[0] * c13 - uu[1] * c03 + uu[3] * c01, -uu[0] * c12 + uu[1] * c02 - uu[2] * c01};
    const T Q0[4] = {-p[1] * c23 + p[2] * c13 - p[3] * c12, p[0] * c23 - p[2] * c03 + p[3] * c02,
                     -p[0] * c13 + p[1] * c03 - p[3] * c01, p[0] * c12 - p[1] * c02 + p[2] * c01};
    const T Q1[4] = {w[1] * s23 - w[2] * s13 + w[3] * s12, -w[0] * s23 + w[2] * s03 - w[3] * s02,
                     w[0] * s13 - w[1] * s03 + w[3] * s01, -w[0] * s12 + w[1] * s02 - w[2] * s01};
    const T Q2[4] = {-v[1] * s23 + v[2] * s13 - v[3] * s12, v[0] * s23 - v[2] * s03 + v[3] * s02,
                     -v[0] * s13 + v[1] * s03 - v[3] * s01, v[0] * s12 - v[1] * s02 + v[2] * s01};
    auto dot = [](const T *a, const T *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + a[3] * b[3]; };
    // mixed derivatives arrive as M = -12 N (site_physics)
    constexpr T kM = T(-1.0 / 12.0);
    const T dD0 = fma(kM, dot(Q1, dm[0]) + dot(Q2, dm[1]), dot(Q0, d2[0]));
    const T dD1 = fma(kM, dot(Q0, dm[0]) + dot(Q2, dm[2]), dot(Q1, d2[1]));
    const T dD2 = fma(kM, dot(Q0, dm[1]) + dot(Q1, dm[2]), dot(Q2, d2[2]));
    const T two_c6 = T(2) * x.c6 * sc.k1sx, four_D = T(4) * D;
#pragma unroll
    for (int A = 0; A < 4; ++A)
        G[A] += two_c6 * (four_D * P[A] + T(12) * (dD0 * Q0[A] + dD1 * Q1[A] + dD2 * Q2[A]));
    e6 = x.c6 * sc.k1sx * D * D;
}

// ------------------------------------------------------------ site physics
// Inputs: phi (4) and its derivatives without their 1/h factors (StencilScale):
// u[i][A] = 12h d_i phi^A, the negated pure second derivatives
// N2[i][A] = -12h^2 d_ii phi^A and the mixed ones M[p][A] = 144h^2 d_p phi^A
// = -12 N_p for p = xy, xz, yz (the -1/12 rides on factors formed anyway).  Outputs: tangent force F (4) and densities
// {e2, e4, e0, b}; with EXT the extension terms of `ext` are included (e0 then
// holds the whole potential) and the sextic density goes to e6.
// With a_ij = k1^2 A_ij (A_ij = u_i.u_j), d_ij phi = -N_ij / (12h^2) and
// B = k1^2 / (12h^2), the brace of the Euler-Lagrange equation is
// -B [L_N (144h^2 + tr A) + sum_i u_i C_i - H], L_N = sum_i N_ii,
// C_i = sum_{j != i} N_ij.u_j - (sum_{j != i} N_jj).u_i (the j = i terms of
// g_i and of the Laplacian's part cancel) and H = sum_ij N_ij A_ij, so that
// G = -2 brace - 2 m^2 e_0 = 2 B [...] - 2 m^2 e_0.
template <typename T, bool EXT = false>
__device__ __forceinline__ void site_physics(const T phi[4], const T d1[3][4], const T d2[3][4],
                                             const T dm[3][4], T m2, const StencilScale<T> &sc,
                                             T F[4], T dens[4], const ExtModel<T> *ext = nullptr,
                                             T *e6 = nullptr)
{
    auto dot = [](const T *a, const T *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + a[3] * b[3]; };
    const T a00 = dot(d1[0], d1[0]), a11 = dot(d1[1], d1[1]), a22 = dot(d1[2], d1[2]);
    const T a01 = dot(d1[0], d1[1]), a02 = dot(d1[0], d1[2]), a12 = dot(d1[1], d1[2]);
    const T tra = a00 + a11 + a22;
    T L[4], L12[4], L02[4], L01[4];
#pragma unroll
    for (int A = 0; A < 4; ++A) {
        L12[A] = d2[1][A] + d2[2][A];
        L02[A] = d2[0][A] + d2[2][A];
        L01[A] = d2[0][A] + d2[1][A];
        L[A] = d2[0][A] + L12[A];
    }
    constexpr T kM = T(-1.0 / 12.0);  // N_ij = kM M_ij
    const T c0 = fma(kM, dot(dm[0], d1[1]) + dot(dm[1], d1[2]), -dot(L12, d1[0]));
    const T c1 = fma(kM, dot(dm[0], d1[0]) + dot(dm[2], d1[2]), -dot(L02, d1[1]));
    const T c2 = fma(kM, dot(dm[1], d1[0]) + dot(dm[2], d1[1]), -dot(L01, d1[2]));
    const T k_tra = sc.K144 + tra;
    // 2 a_ij for the mixed terms, with kM
    const T b01 = T(-1.0 / 6.0) * a01, b02 = T(-1.0 / 6.0) * a02, b12 = T(-1.0 / 6.0) * a12;
    const T twoB = T(2) * sc.B;
    T G[4];
#pragma unroll
    for (int A = 0; A < 4; ++A) {
        // N_ij^A A_ij over all i, j (symmetric)
        const T Ha = d2[0][A] * a00 + d2[1][A] * a11 + d2[2][A] * a22 + dm[0][A] * b01 +
                     dm[1][A] * b02 + dm[2][A] * b12;
        const T bracket = L[A] * k_tra + d1[0][A] * c0 + d1[1][A] * c1 + d1[2][A] * c2 - Ha;
        G[A] = twoB * bracket;
    }
    G[0] -= T(2) * m2;
    // D = det[phi, d_x phi, d_y phi, d_z phi] by the 2x2 minors of the rows
    // (phi, d_x phi) and (d_y phi, d_z phi): formed here when the sextic
    // cofactors need them, at the end otherwise (shorter live ranges)
    T sm[6], cm[6], det = T(0);
    auto minors = [&]() {
        const T *r0 = phi, *r1 = d1[0], *r2 = d1[1], *r3 = d1[2];
        sm[0] = r0[0] * r1[1] - r1[0] * r0[1], sm[1] = r0[0] * r1[2] - r1[0] * r0[2];
        sm[2] = r0[0] * r1[3] - r1[0] * r0[3], sm[3] = r0[1] * r1[2] - r1[1] * r0[2];
        sm[4] = r0[1] * r1[3] - r1[1] * r0[3], sm[5] = r0[2] * r1[3] - r1[2] * r0[3];
        cm[0] = r2[0] * r3[1] - r3[0] * r2[1], cm[1] = r2[0] * r3[2] - r3[0] * r2[2];
        cm[2] = r2[0] * r3[3] - r3[0] * r2[3], cm[3] = r2[1] * r3[2] - r3[1] * r2[2];
        cm[4] = r2[1] * r3[3] - r3[1] * r2[3], cm[5] = r2[2] * r3[3] - r3[2] * r2[3];
        det = sm[0] * cm[5] - sm[1] * cm[4] + sm[2] * cm[3] + sm[3] * cm[2] - sm[4] * cm[1] +
              sm[5] * cm[0];
    };
    T e0x = T(0), u0 = T(0);
    if constexpr (EXT) {
        minors();
        extension_terms<T>(phi, d1, d2, dm, *ext, sc, sm, cm, det, G, e0x, *e6, u0);
    }
    const T Gphi = G[0] * phi[0] + G[1] * phi[1] + G[2] * phi[2] + G[3] * phi[3];
#pragma unroll
    for (int A = 0; A < 4; ++A) F[A] = Gphi * phi[A] - G[A];

    // e2 = tr a = k1^2 tr A, e4 = k1^4 (tr A^2 - A_ij A_ij) / 2
    dens[0] = sc.k1sq * tra;
    const T sq = a00 * a00 + a11 * a11 + a22 * a22 + T(2) * (a01 * a01 + a02 * a02 + a12 * a12);
    dens[1] = sc.k1qu * (T(0.5) * (tra * tra - sq));
    if constexpr (EXT) dens[2] = T(2) * m2 * u0 + e0x;
    else dens[2] = T(2) * m2 * one_minus_phi0<T>(phi);
    // b = -(1/2 pi^2) D, D = k1^3 det of the unscaled rows
    if constexpr (!EXT) minors();
    dens[3] = (T(-0.050660591821168885) * sc.k1cu) * det;  // -1/(2 pi^2)
}

// ------------------------------------------------------ block reductions
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Reduce NQ values per thread (sums, except index MAXQ which is a max) over
// the block; thread 0 ends with the totals in out[].  Fixed order: the result
// is bitwise reproducible for a given launch shape.  red must hold
// NQ * (blockDim/32) doubles.
template <int NQ, int MAXQ>
__device__ __forceinline__ void block_reduce(double (&v)[NQ], double *red, double (&out)[NQ])
{
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int lane = tid & 31, warp = tid >> 5;
    const int nw = (blockDim.x * blockDim.y * blockDim.z) >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = (q == MAXQ) ? warp_max(v[q]) : warp_sum(v[q]);
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) red[q * nw + warp] = v[q];
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double acc = red[q * nw];
            for (int w = 1; w < nw; ++w)
                acc = (q == MAXQ) ? fmax(acc, red[q * nw + w]) : acc + red[q * nw + w];
            out[q] = acc;
        }
    }
}

// Block reduction through shared memory with one warp per quantity: every
// thread parks its NQ values in buf (NQ * blockDim doubles), then warp q sums
// quantity q (a max for MAXQ) lane-strided and with a butterfly.  Far fewer
// FP64 instructions than a shuffle tree in every warp, which matters on a
// GPU whose FP64 pipe is narrow.  Needs at least NQ warps; fixed order.
template <int NQ, int MAXQ>
__device__ __forceinline__ void block_reduce_wide(const double (&v)[NQ], double *buf,
                                                  double (&out)[NQ])
{
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int lane = tid & 31, warp = tid >> 5;
    __syncthreads();  // buf may alias memory the block was still reading
#pragma unroll
    for (int q = 0; q < NQ; ++q) buf[q * nthr + tid] = v[q];
    __syncthreads();
    double r = 0.0;
    if (warp < NQ) {
        const double *col = buf + warp * nthr;
        r = col[lane];
        for (int i = lane + 32; i < nthr; i += 32) r = (warp == MAXQ) ? fmax(r, col[i]) : r + col[i];
        r = (warp == MAXQ) ? warp_max(r) : warp_sum(r);
    }
    __syncthreads();
    if (warp < NQ && lane == 0) buf[warp] = r;
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) out[q] = buf[q];
    }
}

// Sum the per-CTA partial records (count nparts) in a fixed order: warp q
// handles field q of every record (field 5 is a max).  The totals land in
// tot[] of thread 0; red must hold kPartialDoubles doubles.
__device__ __forceinline__ void reduce_partials(const double *parts, int nparts, double *red,
                                                double (&tot)[kPartialDoubles])
{
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
    __syncthreads();
    for (int q = warp; q < kPartialDoubles; q += nw) {
        double r = (q == 5) ? 0.0 : 0.0;
        for (int i = lane; i < nparts; i += 32) {
            const double x = __ldcg(parts + (size_t)i * kPartialDoubles + q);
            r = (q == 5) ? fmax(r, x) : r + x;
        }
        r = (q == 5) ? warp_max(r) : warp_sum(r);
        if (lane == 0) red[q] = r;
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < kPartialDoubles; ++q) tot[q] = red[q];
    }
}

// End-of-step bookkeeping, run by thread 0 of the last CTA to arrive (or,
// for a lattice split into x-slabs, by the one-thread kernel that combines the
// slabs' records).
// tot = {sum e2, sum e4, sum e0, sum b, sum |F|^2, max |F|^2, n_sites, sum e6}.
__device__ __forceinline__ void finish_step(Ctrl *c, const double (&tot)[kPartialDoubles],
                                            double h3, int mode, int pred)
{
    const double E2 = h3 * tot[0], E4 = h3 * tot[1], E0 = h3 * tot[2], E6 = h3 * tot[7];
    const double E = E2 + E4 + E0 + E6;
    const double B = h3 * tot[3];
    const double delta = sqrt(tot[5]);
    const double rms = tot[6] > 0.0 ? sqrt(tot[4] / tot[6]) : 0.0;
    int actual = 0;
    if (mode == MODE_ARRESTED) actual = (E > c->E_prev) ? 1 : 0;
    const int fix = (actual == pred) ? 0 : (actual ? -1 : +1);
    c->fix = fix;
    // two-level adaptive prediction of the next decision: the last four
    // decisions select a 2-bit saturating counter (learns runs and the
    // alternating arrest pattern of a nearly converged flow)
    {
        const int h = c->hist & 15;
        int ctr = c->pht[h];
        ctr = actual ? (ctr < 3 ? ctr + 1 : 3) : (ctr > 0 ? ctr - 1 : 0);
        c->pht[h] = (unsigned char)ctr;
        const int hn = ((h << 1) | actual) & 15;
        c->hist = hn;
        c->pred = c->pht[hn] >= 2 ? 1 : 0;
    }
    c->arrests += actual;
    c->fixups += (fix != 0);
    c->E_prev = E;
    c->steps += 1;
    c->cur ^= 1;
    c->last[0] = E;
    c->last[1] = E2;
    c->last[2] = E4;
    c->last[3] = E0;
    c->last[4] = B;
    c->last[5] = -E2 + E4 - 3.0 * E0 + 3.0 * E6;
    c->e6_last = E6;
    c->last[6] = delta;
    c->last[7] = rms;
    if (!(isfinite(E) && isfinite(B) && isfinite(tot[4]))) c->status = DEV_NONFINITE;
    c->done = 0;
}

}  // namespace skyrme
