// init_fields.cu -- initial fields of Section 4 built on the device:
// rational-map Skyrmions (Section 4.1, Table 1 degrees 1 to 4), the product
// ansatz of isorotated 1-Skyrmions (Section 4.2, Eq. "Product ansatz",
// optionally symmetrised by renormalising U_1..U_K + U_K..U_1), and a
// smoothed-noise start (vacuum plus Gaussian-smoothed N(0,1) noise inside a
// ball, each component scaled to unit standard deviation over the ball).
//
// The noise uses the SplitMix64 generator (Steele, Lea and Flood 2014) in
// counter form with Box-Muller normals; the two velocity buffers serve as
// temporaries and are zeroed afterwards.
#include <cuda_runtime.h>
#include <math.h>

#include "skyrme_device.cuh"
#include "skyrme_internal.h"

namespace skyrme {

constexpr int kMaxConstituents = 64;
constexpr int kMaxHalfWidth = 96;  // smoothing taps on each side

struct ProductArgs {
    int K;
    int symmetrise;
    double scale;
    double pos[kMaxConstituents][3];
    double quat[kMaxConstituents][4];
};

struct SmoothArgs {
    int half;
    double w[2 * kMaxHalfWidth + 1];
};

__device__ __forceinline__ double coord(int i, int n, double h) { return ((double)i - 0.5 * (double)(n - 1)) * h; }

__device__ __forceinline__ bool interior(int x, int y, int z, int n0, int n1, int n2)
{
    return x >= 2 && x <= n0 - 3 && y >= 2 && y <= n1 - 3 && z >= 2 && z <= n2 - 3;
}

// (a0, a)(b0, b) = (a0 b0 - a.b, a0 b + b0 a - a x b) for U = a0 + i a.tau
__device__ __forceinline__ void su2_mul(const double a[4], const double b[4], double r[4])
{
    const double r0 = a[0] * b[0] - (a[1] * b[1] + a[2] * b[2] + a[3] * b[3]);
    const double r1 = a[0] * b[1] + b[0] * a[1] - (a[2] * b[3] - a[3] * b[2]);
    const double r2 = a[0] * b[2] + b[0] * a[2] - (a[3] * b[1] - a[1] * b[3]);
    const double r3 = a[0] * b[3] + b[0] * a[3] - (a[1] * b[2] - a[2] * b[1]);
    r[0] = r0; r[1] = r1; r[2] = r2; r[3] = r3;
}

template <typename T>
__device__ __forceinline__ void put(vec4_t<T> *p, const double v[4])
{
    store4<T>(p, make4<T>((T)v[0], (T)v[1], (T)v[2], (T)v[3]));
}

// Riemann-sphere direction of R(z) = P/Q in homogeneous form; z = Z1/Z0 with
// (Z1, Z0) = (x + i y, r + z3) for z3 >= 0 and the equivalent (r - z3, x - i y)
// otherwise.
__device__ void rm_direction(int B, double x, double y, double z3, double r, double nh[3])
{
    double z1r, z1i, z0r, z0i;
    if (z3 >= 0.0) { z1r = x; z1i = y; z0r = r + z3; z0i = 0.0; }
    else { z1r = r - z3; z1i = 0.0; z0r = x; z0i = -y; }
    double pr, pi, qr, qi;
    if (B == 1) { pr = z1r; pi = z1i; qr = z0r; qi = z0i; }
    else if (B == 2) {  // R = z^2
        pr = z1r * z1r - z1i * z1i; pi = 2 * z1r * z1i;
        qr = z0r * z0r - z0i * z0i; qi = 2 * z0r * z0i;
    } else if (B == 3) {
        // R = (sqrt3 i z^2 - 1) / (z (z^2 - sqrt3 i)):
        // P = z0 (sqrt3 i z1^2 - z0^2), Q = z1 (z1^2 - sqrt3 i z0^2)
        const double c = sqrt(3.0);
        const double a2r = z1r * z1r - z1i * z1i, a2i = 2 * z1r * z1i;
        const double b2r = z0r * z0r - z0i * z0i, b2i = 2 * z0r * z0i;
        const double ar = -c * a2i - b2r, ai = c * a2r - b2i;
        const double cr = a2r + c * b2i, ci = a2i - c * b2r;
        pr = z0r * ar - z0i * ai; pi = z0r * ai + z0i * ar;
        qr = z1r * cr - z1i * ci; qi = z1r * ci + z1i * cr;
    } else {
        // z1^2, z0^2, z1^4, z0^4, z1^2 z0^2
        const double a2r = z1r * z1r - z1i * z1i, a2i = 2 * z1r * z1i;
        const double b2r = z0r * z0r - z0i * z0i, b2i = 2 * z0r * z0i;
        const double a4r = a2r * a2r - a2i * a2i, a4i = 2 * a2r * a2i;
        const double b4r = b2r * b2r - b2i * b2i, b4i = 2 * b2r * b2i;
        const double mr = a2r * b2r - a2i * b2i, mi = a2r * b2i + a2i * b2r;
        const double k = 2.0 * sqrt(3.0);
        // P = z1^4 + i k z1^2 z0^2 + z0^4 ; Q = z1^4 - i k z1^2 z0^2 + z0^4
        pr = a4r - k * mi + b4r; pi = a4i + k * mr + b4i;
        qr = a4r + k * mi + b4r; qi = a4i - k * mr + b4i;
    }
    const double den = pr * pr + pi * pi + qr * qr + qi * qi;
    if (den == 0.0) { nh[0] = nh[1] = nh[2] = 0.0; return; }
    nh[0] = 2.0 * (pr * qr + pi * qi) / den;
    nh[1] = 2.0 * (pi * qr - pr * qi) / den;
    nh[2] = (qr * qr + qi * qi - pr * pr - pi * pi) / den;
}

template <typename T> __global__ void k_fill_vacuum(vec4_t<T> *phi, size_t total)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x)
        store4<T>(phi + i, make4<T>(T(1), T(0), T(0), T(0)));
}

template <typename T>
__global__ void k_seed_rm(vec4_t<T> *phi, int n0, int n1, int n2, double h, int B, double scale)
{
    const size_t total = (size_t)n0 * n1 * n2;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int z = (int)(i % n2), y = (int)((i / n2) % n1), x = (int)(i / ((size_t)n2 * n1));
        const double cx = coord(x, n0, h), cy = coord(y, n1, h), cz = coord(z, n2, h);
        const double r = sqrt(cx * cx + cy * cy + cz * cz);
        const double f = M_PI * exp(-r / scale);
        double nh[3];
        rm_direction(B, cx, cy, cz, r, nh);
        const double sf = sin(f);
        const double v[4] = {cos(f), sf * nh[0], sf * nh[1], sf * nh[2]};
        put<T>(phi + i, v);
    }
}

template <typename T>
__global__ void k_seed_product(vec4_t<T> *phi, int n0, int n1, int n2, double h, ProductArgs a)
{
    const size_t total = (size_t)n0 * n1 * n2;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int z = (int)(i % n2), y = (int)((i / n2) % n1), x = (int)(i / ((size_t)n2 * n1));
        const double cx = coord(x, n0, h), cy = coord(y, n1, h), cz = coord(z, n2, h);
        double fwd[4] = {1, 0, 0, 0}, rev[4] = {1, 0, 0, 0};
        // forward product U_1 U_2 ... U_K; the reverse product is accumulated
        // by left multiplication: U_K ... U_1
        for (int k = 0; k < a.K; ++k) {
            const double dx = cx - a.pos[k][0], dy = cy - a.pos[k][1], dz = cz - a.pos[k][2];
            const double r = sqrt(dx * dx + dy * dy + dz * dz);
            const double f = M_PI * exp(-r / a.scale);
            const double sf = sin(f);
            double u[4] = {cos(f), 0.0, 0.0, 0.0};
            if (r > 0.0) { u[1] = sf * dx / r; u[2] = sf * dy / r; u[3] = sf * dz / r; }
            const double A[4] = {a.quat[k][0], a.quat[k][1], a.quat[k][2], a.quat[k][3]};
            const double Ad[4] = {A[0], -A[1], -A[2], -A[3]};
            double t[4], uk[4];
            su2_mul(A, u, t);
            su2_mul(t, Ad, uk);
            su2_mul(fwd, uk, fwd);
            su2_mul(uk, rev, rev);
        }
        double out[4];
        if (a.symmetrise) {
            double s[4] = {fwd[0] + rev[0], fwd[1] + rev[1], fwd[2] + rev[2], fwd[3] + rev[3]};
            const double nrm = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + s[3] * s[3]);
            if (nrm < 1e-12) { for (int q = 0; q < 4; ++q) out[q] = fwd[q]; }
            else { for (int q = 0; q < 4; ++q) out[q] = s[q] / nrm; }
        } else {
            for (int q = 0; q < 4; ++q) out[q] = fwd[q];
        }
        put<T>(phi + i, out);
    }
}

// ------------------------------------------------------------------ noise
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double normal_at(uint64_t seed, uint64_t k)
{
    const double scale = 1.0 / 9007199254740992.0;  // 2^-53
    const double u1 = ((double)(splitmix64_at(seed, 2 * k) >> 11) + 1.0) * scale;
    const double u2 = (double)(splitmix64_at(seed, 2 * k + 1) >> 11) * scale;
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

template <typename T>
__global__ void k_noise(vec4_t<T> *out, int n0, int n1, int n2, double h, double radius,
                        uint64_t seed)
{
    const size_t total = (size_t)n0 * n1 * n2;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int z = (int)(i % n2), y = (int)((i / n2) % n1), x = (int)(i / ((size_t)n2 * n1));
        const double cx = coord(x, n0, h), cy = coord(y, n1, h), cz = coord(z, n2, h);
        double v[4] = {0, 0, 0, 0};
        if (cx * cx + cy * cy + cz * cz <= radius * radius)
            for (int c = 0; c < 4; ++c) v[c] = normal_at(seed, 4ull * i + (uint64_t)c);
        put<T>(out + i, v);
    }
}

// One separable Gaussian pass along `axis`; zero outside the lattice.
template <typename T>
__global__ void k_smooth(const vec4_t<T> *src, vec4_t<T> *dst, int n0, int n1, int n2, int axis,
                         SmoothArgs w)
{
    const size_t total = (size_t)n0 * n1 * n2;
    const int nax = axis == 0 ? n0 : (axis == 1 ? n1 : n2);
    const size_t stride = axis == 0 ? (size_t)n1 * n2 : (axis == 1 ? (size_t)n2 : 1);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int z = (int)(i % n2), y = (int)((i / n2) % n1), x = (int)(i / ((size_t)n2 * n1));
        const int c = axis == 0 ? x : (axis == 1 ? y : z);
        double acc[4] = {0, 0, 0, 0};
        for (int k = -w.half; k <= w.half; ++k) {
            const int cc = c + k;
            if (cc < 0 || cc >= nax) continue;
            const vec4_t<T> s = load4<T>(src + (size_t)((long long)i + (long long)k * (long long)stride));
            const double wk = w.w[k + w.half];
            acc[0] += wk * (double)s.x;
            acc[1] += wk * (double)s.y;
            acc[2] += wk * (double)s.z;
            acc[3] += wk * (double)s.w;
        }
        put<T>(dst + i, acc);
    }
}

// Moments over the ball: pass 0 sums the values (and the count), pass 1 the
// squared deviations from the mean.  Per-block partials, fixed-order finish.
template <typename T>
__global__ void k_ball_moments(const vec4_t<T> *src, int n0, int n1, int n2, double h,
                               double radius, int pass, double *parts, double *stats,
                               unsigned int *counter)
{
    const size_t total = (size_t)n0 * n1 * n2;
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double mean[4] = {0, 0, 0, 0};
    if (pass == 1)
        for (int c = 0; c < 4; ++c) mean[c] = stats[c];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int z = (int)(i % n2), y = (int)((i / n2) % n1), x = (int)(i / ((size_t)n2 * n1));
        const double cx = coord(x, n0, h), cy = coord(y, n1, h), cz = coord(z, n2, h);
        if (cx * cx + cy * cy + cz * cz > radius * radius) continue;
        const vec4_t<T> s = load4<T>(src + i);
        const double a[4] = {(double)s.x, (double)s.y, (double)s.z, (double)s.w};
        for (int c = 0; c < 4; ++c) {
            const double d = a[c] - mean[c];
            v[c] += pass == 0 ? a[c] : d * d;
        }
        v[4] += 1.0;
    }
    __shared__ double red[8 * 8];
    __shared__ int s_last;
    double out[8];
    block_reduce<8, -1>(v, red, out);
    if (threadIdx.x == 0) {
        for (int q = 0; q < 8; ++q) parts[(size_t)blockIdx.x * 8 + q] = out[q];
        __threadfence();
        s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x == 0) {
        double tot[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (unsigned int b = 0; b < gridDim.x; ++b)
            for (int q = 0; q < 8; ++q) tot[q] += __ldcg(parts + (size_t)b * 8 + q);
        const double cnt = tot[4];
        for (int c = 0; c < 4; ++c) {
            if (pass == 0) stats[c] = cnt > 0 ? tot[c] / cnt : 0.0;
            else stats[4 + c] = cnt > 0 ? sqrt(tot[c] / cnt) : 0.0;
        }
        *counter = 0;
    }
}

template <typename T>
__global__ void k_noise_finish(vec4_t<T> *phi, const vec4_t<T> *noise, size_t total,
                               const double *stats)
{
    double sd[4];
    for (int c = 0; c < 4; ++c) sd[c] = stats[4 + c] > 0.0 ? stats[4 + c] : 1.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const vec4_t<T> s = load4<T>(noise + i);
        const double t[4] = {1.0 + (double)s.x / sd[0], (double)s.y / sd[1], (double)s.z / sd[2],
                             (double)s.w / sd[3]};
        const double nrm = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2] + t[3] * t[3]);
        double o[4] = {1, 0, 0, 0};
        if (nrm >= 1e-12)
            for (int c = 0; c < 4; ++c) o[c] = t[c] / nrm;
        put<T>(phi + i, o);
    }
}

static int grid_for(size_t total)
{
    size_t b = (total + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    return (int)(b < 1 ? 1 : b);
}

template <typename T>
static cudaError_t seed_impl(const skyrme_lattice &lat, const skyrme_seed &sd, const FlowArgs &a,
                             cudaStream_t s)
{
    vec4_t<T> *phi0 = static_cast<vec4_t<T> *>(a.phi[0]);
    const int n0 = lat.n[0], n1 = lat.n[1], n2 = lat.n[2];
    const size_t total = (size_t)n0 * n1 * n2;
    const int g = grid_for(total);
    switch (sd.kind) {
    case SKYRME_SEED_VACUUM:
        k_fill_vacuum<T><<<g, 256, 0, s>>>(phi0, total);
        break;
    case SKYRME_SEED_RATIONAL_MAP:
        k_seed_rm<T><<<g, 256, 0, s>>>(phi0, n0, n1, n2, lat.h, sd.B, sd.profile_scale);
        break;
    case SKYRME_SEED_PRODUCT: {
        ProductArgs pa;
        pa.K = sd.B;
        pa.symmetrise = sd.symmetrise;
        pa.scale = sd.profile_scale;
        for (int k = 0; k < sd.B; ++k) {
            for (int c = 0; c < 3; ++c) pa.pos[k][c] = sd.positions[3 * k + c];
            for (int c = 0; c < 4; ++c) pa.quat[k][c] = sd.quaternions[4 * k + c];
        }
        k_seed_product<T><<<g, 256, 0, s>>>(phi0, n0, n1, n2, lat.h, pa);
        break;
    }
    case SKYRME_SEED_NOISE: {
        vec4_t<T> *t0 = static_cast<vec4_t<T> *>(a.vel[0]);
        vec4_t<T> *t1 = static_cast<vec4_t<T> *>(a.vel[1]);
        SmoothArgs w;
        w.half = (int)ceil(4.0 * sd.sigma / lat.h);
        double wsum = 0.0;
        for (int k = -w.half; k <= w.half; ++k) {
            w.w[k + w.half] = exp(-(k * lat.h) * (k * lat.h) / (2.0 * sd.sigma * sd.sigma));
            wsum += w.w[k + w.half];
        }
        for (int k = 0; k <= 2 * w.half; ++k) w.w[k] /= wsum;
        k_noise<T><<<g, 256, 0, s>>>(t0, n0, n1, n2, lat.h, sd.radius, sd.seed);
        k_smooth<T><<<g, 256, 0, s>>>(t0, t1, n0, n1, n2, 0, w);
        k_smooth<T><<<g, 256, 0, s>>>(t1, t0, n0, n1, n2, 1, w);
        k_smooth<T><<<g, 256, 0, s>>>(t0, t1, n0, n1, n2, 2, w);
        Ctrl *c = static_cast<Ctrl *>(a.ctrl);
        double *stats = c->energy;  // 8 doubles: mean[4], sd[4]
        unsigned int *ctr = &c->edone;
        k_ball_moments<T><<<g, 256, 0, s>>>(t1, n0, n1, n2, lat.h, sd.radius, 0, a.energy_parts,
                                            stats, ctr);
        k_ball_moments<T><<<g, 256, 0, s>>>(t1, n0, n1, n2, lat.h, sd.radius, 1, a.energy_parts,
                                            stats, ctr);
        k_noise_finish<T><<<g, 256, 0, s>>>(phi0, t1, total, stats);
        break;
    }
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_seed(const skyrme_lattice &lat, const skyrme_seed &seed, const FlowArgs &a,
                        cudaStream_t s)
{
    if (lat.precision == 64) return seed_impl<double>(lat, seed, a, s);
    return seed_impl<float>(lat, seed, a, s);
}

int max_constituents() { return kMaxConstituents; }
int max_smoothing_half_width() { return kMaxHalfWidth; }

}  // namespace skyrme
