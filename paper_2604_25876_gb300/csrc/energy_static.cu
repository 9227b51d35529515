// energy_static.cu -- skyrme_energy_static: the energy / baryon-number /
// virial reduction of skyrme_energy, for callers that cannot allocate device
// memory.
//
// Some callers have no way to obtain scratch memory.  Two examples: code
// running inside a host application that owns every device allocation
// through its own pool, and plug-ins that may only use buffers handed to
// them.  This entry point needs nothing but the field.  Its scratch is the
// file-scope array below: every GPU that loads the library holds those
// 128 KiB until the process exits.
//
// One CTA reduces one interior x-plane into an FP64 partial record; the last
// CTA to finish sums the records in plane order, so the result does not
// depend on the launch and matches skyrme_energy up to summation order.
#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>

#include "skyrme_device.cuh"
#include "skyrme_internal.h"

namespace skyrme {

constexpr int kStaticMaxPlanes = 2048;  // interior x-planes (n[0] - 4) supported
constexpr size_t kStaticHeaderBytes = 256;
constexpr size_t kStaticScratchBytes =
    kStaticHeaderBytes + (size_t)kStaticMaxPlanes * kPartialDoubles * sizeof(double);

// Shared by every call on a device; keeps the last call's contents.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

struct StaticHeader {
    unsigned int counter;  // CTAs finished (cleared before every launch)
    unsigned int pad[15];
    double result[8];      // E, E2, E4, E0, B, V
};
static_assert(sizeof(StaticHeader) <= kStaticHeaderBytes, "header must fit");

template <typename T>
__global__ void __launch_bounds__(256) k_energy_static(const vec4_t<T> *__restrict__ phi, int n0,
                                                       int n1, int n2, T inv_h, T m2,
                                                       ExtModel<T> ext, bool extended, double h3,
                                                       unsigned char *scratch)
{
    StaticHeader *hdr = reinterpret_cast<StaticHeader *>(scratch);
    double *records = reinterpret_cast<double *>(scratch + kStaticHeaderBytes);
    const int x = 2 + blockIdx.x;
    const int iy = n1 - 4, iz = n2 - 4;
    const size_t sy = (size_t)n2, sx = (size_t)n1 * n2;
    double acc[5] = {0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < iy * iz; i += blockDim.x) {
        const int y = 2 + i / iz, z = 2 + i % iz;
        const size_t s = (size_t)x * sx + (size_t)y * sy + z;
        const vec4_t<T> c = load4<T>(phi + s);
        const size_t step[3] = {sx, sy, 1};
        T d1[3][4];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const vec4_t<T> m2v = load4<T>(phi + s - 2 * step[a]), m1v = load4<T>(phi + s - step[a]);
            const vec4_t<T> p1v = load4<T>(phi + s + step[a]), p2v = load4<T>(phi + s + 2 * step[a]);
            d1[a][0] = fd1<T>(m2v.x, m1v.x, p1v.x, p2v.x) * inv_h;
            d1[a][1] = fd1<T>(m2v.y, m1v.y, p1v.y, p2v.y) * inv_h;
            d1[a][2] = fd1<T>(m2v.z, m1v.z, p1v.z, p2v.z) * inv_h;
            d1[a][3] = fd1<T>(m2v.w, m1v.w, p1v.w, p2v.w) * inv_h;
        }
        T a_[3][3];
#pragma unroll
        for (int i2 = 0; i2 < 3; ++i2)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                a_[i2][j] = d1[i2][0] * d1[j][0] + d1[i2][1] * d1[j][1] + d1[i2][2] * d1[j][2] +
                            d1[i2][3] * d1[j][3];
        const T tra = a_[0][0] + a_[1][1] + a_[2][2];
        T sq = T(0);
#pragma unroll
        for (int i2 = 0; i2 < 3; ++i2)
#pragma unroll
            for (int j = 0; j < 3; ++j) sq += a_[i2][j] * a_[i2][j];
        const T ph[4] = {c.x, c.y, c.z, c.w};
        // det[phi, d_x phi, d_y phi, d_z phi] by 2x2 minors of rows (phi, d_x), (d_y, d_z)
        const T *r0 = ph, *r1 = d1[0], *r2 = d1[1], *r3 = d1[2];
        const T det = (r0[0] * r1[1] - r1[0] * r0[1]) * (r2[2] * r3[3] - r3[2] * r2[3]) -
                      (r0[0] * r1[2] - r1[0] * r0[2]) * (r2[1] * r3[3] - r3[1] * r2[3]) +
                      (r0[0] * r1[3] - r1[0] * r0[3]) * (r2[1] * r3[2] - r3[1] * r2[2]) +
                      (r0[1] * r1[2] - r1[1] * r0[2]) * (r2[0] * r3[3] - r3[0] * r2[3]) -
                      (r0[1] * r1[3] - r1[1] * r0[3]) * (r2[0] * r3[2] - r3[0] * r2[2]) +
                      (r0[2] * r1[3] - r1[2] * r0[3]) * (r2[0] * r3[1] - r3[0] * r2[1]);
        acc[0] += (double)tra;
        acc[1] += (double)(T(0.5) * (tra * tra - sq));
        const T u = one_minus_phi0<T>(ph);
        T e0 = T(2) * m2 * u;
        if (extended) {
            // Section 7.8 potentials and the sextic term c6 4 pi^4 (B0)^2 = c6 det^2
            e0 += ext.my2 * one_minus_phi0_sq<T>(ph, u) + ext.mz2 * u * u + T(0.5) * ext.mw2 * u * u * u * u;
            acc[4] += (double)(ext.c6 * det * det);
        }
        acc[2] += (double)e0;
        acc[3] += (double)det;
    }
    __shared__ double red[5 * 8];
    __shared__ int s_last;
    double tot[5];
    block_reduce<5, -1>(acc, red, tot);
    if (threadIdx.x == 0) {
        double *rec = records + (size_t)blockIdx.x * kPartialDoubles;
        for (int q = 0; q < 5; ++q) rec[q] = tot[q];
        __threadfence();
        s_last = (atomicAdd(&hdr->counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    double sum[5] = {0, 0, 0, 0, 0};
    for (unsigned int b = 0; b < gridDim.x; ++b)
        for (int q = 0; q < 5; ++q) sum[q] += __ldcg(records + (size_t)b * kPartialDoubles + q);
    const double E2 = h3 * sum[0], E4 = h3 * sum[1], E0 = h3 * sum[2], E6 = h3 * sum[4];
    hdr->result[0] = E2 + E4 + E0 + E6;
    hdr->result[1] = E2;
    hdr->result[2] = E4;
    hdr->result[3] = E0;
    hdr->result[4] = h3 * sum[3] * -0.050660591821168885;  // b = -det / (2 pi^2)
    hdr->result[5] = -E2 + E4 - 3.0 * E0 + 3.0 * E6;
    hdr->counter = 0;
}

// Device address of the static scratch in the current context.  Module
// symbols belong to a context, and a context can be replaced under the same
// device ordinal (cudaDeviceReset, or a host application that binds its own
// context), so the address is looked up on every call rather than cached:
// the lookup is host-side and allocates nothing.
static void *static_scratch_address(cudaError_t *err)
{
    void *p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_static_scratch);
    return *err == cudaSuccess ? p : nullptr;
}

}  // namespace skyrme

using namespace skyrme;

extern "C" skyrme_status skyrme_energy_static(const skyrme_lattice *lat, const void *phi,
                                              double out6[6], void *stream)
{
    if (!lattice_ok(lat) || !phi || !out6) return SKYRME_EINVAL;
    // one partial record per interior x-plane must fit the static scratch
    if (lat->n[0] - 4 > kStaticMaxPlanes) return SKYRME_EINVAL;
    const size_t align = lat->precision == 64 ? 32 : 16;
    if ((uintptr_t)phi % align) return SKYRME_EINVAL;
    // the field must be on the current device, where the scratch is looked up
    // and the kernel runs
    skyrme_status rc = on_current_device(&phi, 1);
    if (rc != SKYRME_OK) return rc;
    cudaError_t e;
    void *scratch = static_scratch_address(&e);
    if (!scratch) return SKYRME_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the arrival counter and the results must start from zero on every call
    if (cudaMemsetAsync(scratch, 0, kStaticHeaderBytes, s) != cudaSuccess) return SKYRME_ECUDA;
    const double h = lat->h;
    const unsigned grid = (unsigned)(lat->n[0] - 4);
    unsigned char *sp = static_cast<unsigned char *>(scratch);
    const bool ext = lattice_extended(*lat);
    if (lat->precision == 64) {
        const ExtModel<double> x{lat->m_y * lat->m_y, lat->m_z * lat->m_z, lat->m_w * lat->m_w,
                                 lat->c6};
        k_energy_static<double><<<grid, 256, 0, s>>>(static_cast<const dvec4 *>(phi), lat->n[0],
                                                     lat->n[1], lat->n[2], 1.0 / h,
                                                     lat->m * lat->m, x, ext, h * h * h, sp);
    } else {
        const ExtModel<float> x{(float)(lat->m_y * lat->m_y), (float)(lat->m_z * lat->m_z),
                                (float)(lat->m_w * lat->m_w), (float)lat->c6};
        k_energy_static<float><<<grid, 256, 0, s>>>(static_cast<const float4 *>(phi), lat->n[0],
                                                    lat->n[1], lat->n[2], (float)(1.0 / h),
                                                    (float)(lat->m * lat->m), x, ext, h * h * h, sp);
    }
    if (cudaGetLastError() != cudaSuccess) return SKYRME_ECUDA;
    double res[8];
    if (cudaMemcpyAsync(res, sp + offsetof(StaticHeader, result), 6 * sizeof(double),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SKYRME_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SKYRME_ECUDA;
    for (int i = 0; i < 6; ++i) out6[i] = res[i];
    if (!isfinite(res[0]) || !isfinite(res[4])) return SKYRME_ENONFINITE;
    return SKYRME_OK;
}
