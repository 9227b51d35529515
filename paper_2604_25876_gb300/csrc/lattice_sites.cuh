// lattice_sites.cuh -- FP64 per-site helpers shared by the diagnostic passes
// over the current field (observables, volume render): site loads widened to
// double and the lattice baryon density.
#pragma once

#include "skyrme_device.cuh"

namespace skyrme {

__device__ __forceinline__ void load_site(const float4 *p, size_t i, double v[4])
{
    const float4 q = __ldg(p + i);
    v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
}
__device__ __forceinline__ void load_site(const dvec4 *p, size_t i, double v[4])
{
    const dvec4 q = p[i];
    v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
}

// First lattice derivatives d[k][A] (k = x, y, z) of the site at linear index
// c: 4th-order central stencil, weights w1 = 2/(3h), w2 = -1/(12h).
template <typename V>
__device__ __forceinline__ void site_first_derivatives(const V *phi, size_t c, size_t sx, size_t sy,
                                                       double w1, double w2, double d[3][4])
{
    const size_t st[3] = {sx, sy, 1};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double m2v[4], m1v[4], p1v[4], p2v[4];
        load_site(phi, c - 2 * st[k], m2v);
        load_site(phi, c - st[k], m1v);
        load_site(phi, c + st[k], p1v);
        load_site(phi, c + 2 * st[k], p2v);
#pragma unroll
        for (int A = 0; A < 4; ++A) d[k][A] = w1 * (p1v[A] - m1v[A]) + w2 * (p2v[A] - m2v[A]);
    }
}

// Baryon density -det[phi, d_x phi, d_y phi, d_z phi] / (2 pi^2), the 4x4
// determinant expanded in 2x2 minors of the first two and last two columns.
__device__ __forceinline__ double baryon_density(const double ph[4], const double d[3][4])
{
    const double s0 = ph[0] * d[0][1] - d[0][0] * ph[1], s1 = ph[0] * d[0][2] - d[0][0] * ph[2];
    const double s2 = ph[0] * d[0][3] - d[0][0] * ph[3], s3 = ph[1] * d[0][2] - d[0][1] * ph[2];
    const double s4 = ph[1] * d[0][3] - d[0][1] * ph[3], s5 = ph[2] * d[0][3] - d[0][2] * ph[3];
    const double q5 = d[1][2] * d[2][3] - d[2][2] * d[1][3], q4 = d[1][1] * d[2][3] - d[2][1] * d[1][3];
    const double q3 = d[1][1] * d[2][2] - d[2][1] * d[1][2], q2 = d[1][0] * d[2][3] - d[2][0] * d[1][3];
    const double q1 = d[1][0] * d[2][2] - d[2][0] * d[1][2], q0 = d[1][0] * d[2][1] - d[2][0] * d[1][1];
    return -0.050660591821168885 * (s0 * q5 - s1 * q4 + s2 * q3 + s3 * q2 - s4 * q1 + s5 * q0);
}

}  // namespace skyrme
