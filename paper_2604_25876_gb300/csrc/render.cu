// render.cu -- headless volume render of the baryon density (Section 6.2,
// ray tracing).  The picture goes to a caller-owned device RGBA buffer in
// place of a GL pixel buffer.
//
//   1. k_render_volume: one FP64 record per site, {B0, pion / |pion|}, in the
//      caller's volume buffer.  B0 uses the flow's lattice derivatives at
//      interior sites and is 0 on the boundary layers.  Max B0 is an atomic
//      max on the bit pattern, since positive doubles order like their bits.
//   2. k_render_normalise: B0 / max B0, or 0 everywhere when max B0 <= 0.
//   3. k_render_rays: one thread per pixel.
//      - A perspective ray crosses the lattice box in fixed steps.
//      - Each step takes trilinear samples of all four components.
//      - The transfer input is (b - levelset) scale; negative inputs are
//        skipped.
//      - The colour is input^2 (pion, 1/input).
//      - Compositing is front to back and stops once alpha exceeds 0.95.
//      - The result is multiplied by brightness and clamped to [0, 1].
// The ray arithmetic is FP64, compiled without multiply-add contraction.
// That way the skip and stop decisions round the same way as a plain C
// restatement compiled with contraction off.  Only the output is FP32.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "lattice_sites.cuh"
#include "skyrme_device.cuh"
#include "skyrme_internal.h"

namespace skyrme {

constexpr double kRenderEye = 4.0;     // eye on the view-space z axis
constexpr double kRenderFocal = 2.0;   // image plane distance (vertical half-extent 1)
constexpr double kRenderAlphaStop = 0.95;

template <typename V>
__global__ void k_render_volume(const V *phi0, const V *phi1, const Ctrl *ctrl, int n0, int n1,
                                int n2, double w1, double w2, dvec4 *vol,
                                unsigned long long *bmax_bits)
{
    const V *phi = __ldcg(&ctrl->cur) ? phi1 : phi0;
    const long long total = (long long)n0 * n1 * n2;
    const size_t sx = (size_t)n1 * n2, sy = (size_t)n2;
    double local_max = 0.0;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < total;
         s += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(s % n2), y = (int)((s / n2) % n1), x = (int)(s / ((long long)n2 * n1));
        double ph[4];
        load_site(phi, (size_t)s, ph);
        double b = 0.0;
        if (x >= 2 && x <= n0 - 3 && y >= 2 && y <= n1 - 3 && z >= 2 && z <= n2 - 3) {
            double d[3][4];
            site_first_derivatives(phi, (size_t)s, sx, sy, w1, w2, d);
            b = baryon_density(ph, d);
        }
        const double np = sqrt(ph[1] * ph[1] + ph[2] * ph[2] + ph[3] * ph[3]);
        dvec4 out;
        out.x = b;
        out.y = np > 0.0 ? ph[1] / np : 0.0;
        out.z = np > 0.0 ? ph[2] / np : 0.0;
        out.w = np > 0.0 ? ph[3] / np : 0.0;
        vol[s] = out;
        local_max = fmax(local_max, b);
    }
    for (int o = 16; o > 0; o >>= 1) local_max = fmax(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
    if ((threadIdx.x & 31) == 0 && local_max > 0.0)
        atomicMax(bmax_bits, (unsigned long long)__double_as_longlong(local_max));
}

__global__ void k_render_normalise(dvec4 *vol, long long total, const unsigned long long *bmax_bits)
{
    const double bmax = __longlong_as_double((long long)*bmax_bits);
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < total;
         s += (long long)gridDim.x * blockDim.x)
        vol[s].x = bmax > 0.0 ? vol[s].x / bmax : 0.0;
}

struct RayParams {
    int width, height;
    int n[3];
    long long max_samples;  // per ray, a bound the valid parameters never reach
    double view[9];
    double levelset, scale, brightness, step;
};

// Trilinear interpolation of the four components at lattice coordinates g,
// clamped to the lattice.
__device__ __forceinline__ void trilinear(const dvec4 *vol, const int n[3], const double g[3],
                                          double out[4])
{
    int i0[3];
    double w[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double t = fmin(fmax(g[a], 0.0), (double)(n[a] - 1));
        i0[a] = min((int)floor(t), n[a] - 2);
        w[a] = t - (double)i0[a];
    }
    out[0] = out[1] = out[2] = out[3] = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        const double wt = (dx ? w[0] : 1.0 - w[0]) * (dy ? w[1] : 1.0 - w[1]) * (dz ? w[2] : 1.0 - w[2]);
        const dvec4 v = vol[((size_t)(i0[0] + dx) * n[1] + (i0[1] + dy)) * n[2] + (i0[2] + dz)];
        out[0] += wt * v.x;
        out[1] += wt * v.y;
        out[2] += wt * v.z;
        out[3] += wt * v.w;
    }
}

__global__ void __launch_bounds__(128) k_render_rays(const __grid_constant__ RayParams rp,
                                                     const dvec4 *vol, float4 *rgba)
{
    const int px = blockIdx.x * blockDim.x + threadIdx.x;
    if (px >= rp.width * rp.height) return;
    const int ix = px % rp.width, iy = px / rp.width;
    // box: lattice coordinate g <-> (g - (n-1)/2) / s, the longest axis spans [-1, 1]
    double half[3], s = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        half[a] = 0.5 * (double)(rp.n[a] - 1);
        s = fmax(s, half[a]);
    }
    const double aspect = (double)rp.width / (double)rp.height;
    double dv[3] = {(2.0 * (ix + 0.5) / rp.width - 1.0) * aspect, 2.0 * (iy + 0.5) / rp.height - 1.0,
                    -kRenderFocal};
    const double nd = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
#pragma unroll
    for (int i = 0; i < 3; ++i) dv[i] /= nd;
    // view space -> box space through the row-major rotation
    const double ov[3] = {0.0, 0.0, kRenderEye};
    double o[3], d[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        o[i] = 0.0, d[i] = 0.0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            o[i] += rp.view[3 * i + j] * ov[j];
            d[i] += rp.view[3 * i + j] * dv[j];
        }
    }
    // slab intersection with |p_i| <= half_i / s
    double tnear = -1e300, tfar = 1e300;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
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
    double sum[4] = {0.0, 0.0, 0.0, 0.0};
    long long k = 0;
    for (double t = tnear; t <= tfar && k < rp.max_samples; t += rp.step, ++k) {
        double g[3], smp[4];
#pragma unroll
        for (int i = 0; i < 3; ++i) g[i] = (o[i] + t * d[i]) * s + half[i];
        trilinear(vol, rp.n, g, smp);
        const double input = (smp[0] - rp.levelset) * rp.scale;
        if (input < 0.0) continue;
        const double col[4] = {input * input * smp[1], input * input * smp[2], input * input * smp[3],
                               input};
        const double keep = 1.0 - sum[3];
#pragma unroll
        for (int c = 0; c < 4; ++c) sum[c] += col[c] * keep;
        if (sum[3] > kRenderAlphaStop) break;
    }
    double v[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        v[c] = sum[c] * rp.brightness;
        v[c] = v[c] < 0.0 ? 0.0 : (v[c] > 1.0 ? 1.0 : v[c]);
    }
    rgba[px] = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
}

bool render_params_valid(const skyrme_render_params &p)
{
    if (p.width < 1 || p.height < 1 || (long long)p.width * p.height > SKYRME_RENDER_MAX_PIXELS)
        return false;
    if (!(p.step >= SKYRME_RENDER_MIN_STEP && p.step <= 1.0)) return false;
    if (!isfinite(p.levelset) || !isfinite(p.transfer_scale) || !isfinite(p.brightness)) return false;
    // view: a rotation (orthonormal rows) to 1e-9
    for (int i = 0; i < 9; ++i)
        if (!isfinite(p.view[i])) return false;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double dot = 0.0;
            for (int k = 0; k < 3; ++k) dot += p.view[3 * i + k] * p.view[3 * j + k];
            if (fabs(dot - (i == j ? 1.0 : 0.0)) > 1e-9) return false;
        }
    return true;
}

cudaError_t launch_render_volume(const skyrme_lattice &lat, const FlowArgs &a, void *vol,
                                 void *bmax_scratch, cudaStream_t s)
{
    const long long total = (long long)lat.n[0] * lat.n[1] * lat.n[2];
    auto *bits = static_cast<unsigned long long *>(bmax_scratch);
    cudaError_t e = cudaMemsetAsync(bits, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const double w1 = 2.0 / 3.0 / lat.h, w2 = -1.0 / 12.0 / lat.h;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 8);
    dvec4 *v = static_cast<dvec4 *>(vol);
    const Ctrl *ctrl = static_cast<const Ctrl *>(a.ctrl);
    if (lat.precision == 64)
        k_render_volume<dvec4><<<blocks, 256, 0, s>>>(static_cast<const dvec4 *>(a.phi[0]),
                                                     static_cast<const dvec4 *>(a.phi[1]), ctrl,
                                                     lat.n[0], lat.n[1], lat.n[2], w1, w2, v, bits);
    else
        k_render_volume<float4><<<blocks, 256, 0, s>>>(static_cast<const float4 *>(a.phi[0]),
                                                      static_cast<const float4 *>(a.phi[1]), ctrl,
                                                      lat.n[0], lat.n[1], lat.n[2], w1, w2, v, bits);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_render_normalise<<<blocks, 256, 0, s>>>(v, total, bits);
    return cudaGetLastError();
}

cudaError_t launch_render_rays(const int n[3], const void *vol, const skyrme_render_params &p,
                               float *rgba, cudaStream_t s)
{
    RayParams rp;
    rp.width = p.width;
    rp.height = p.height;
    for (int i = 0; i < 3; ++i) rp.n[i] = n[i];
    for (int i = 0; i < 9; ++i) rp.view[i] = p.view[i];
    rp.levelset = p.levelset;
    rp.scale = p.transfer_scale;
    rp.brightness = p.brightness;
    rp.step = p.step;
    // a chord of the box is at most 2 sqrt(3) long
    rp.max_samples = (long long)ceil(3.5 / p.step) + 2;
    const int pixels = p.width * p.height;
    k_render_rays<<<(pixels + 127) / 128, 128, 0, s>>>(rp, static_cast<const dvec4 *>(vol),
                                                       reinterpret_cast<float4 *>(rgba));
    return cudaGetLastError();
}

}  // namespace skyrme
