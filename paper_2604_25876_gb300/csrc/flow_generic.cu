// flow_generic.cu -- tile-staged kernels of the arrested Newton flow in either
// precision: the fused step (derivatives + Euler-Lagrange gradient + tangent
// projection + velocity/field update + renormalisation + energy sums), the
// speculative-arrest fix-up, the energy reduction and the per-site force dump.
//
// One CTA owns a TX x TY x TZ block of interior sites and stages the field
// with a 2-site halo in shared memory (Section 3: stencil radius 2).  The
// FP64 path is bound by the FP64 pipe, so this straightforward staging is its
// production kernel; FP32 has a dedicated streaming kernel elsewhere.
//
// Arrest without a host round trip: the energy E_n of phi_n is only known
// after every CTA has finished, but the update needs to know whether v_n is
// zeroed.  Each step therefore applies the decision predicted from the
// previous iteration (ctrl.pred); the last CTA compares E_n with E_{n-1},
// and when the prediction was wrong it sets ctrl.fix = +-1 so that the
// pointwise fix-up kernel rewrites v_{n+1} = v' -+ v_n and
// phi_{n+1} = normalise(phi_n + dt v_{n+1}) from the untouched old buffers.
#include <cuda_runtime.h>

#include <algorithm>

#include "skyrme_device.cuh"
#include "skyrme_internal.h"

namespace skyrme {

// Tile geometry: TX x TY x TZ interior sites per CTA, one thread per site,
// 256 threads either way.  TZ = 32 (2 x 4 x 32) in general; TZ = 16
// (2 x 8 x 16) for lattices whose z-interior pads less to 16 than to 32
// (a 44-site interior: 8% idle lanes instead of 31%).  S* are the haloed
// extents, DXN / DYN / TILEN the entries of d_x phi, d_y phi and the field
// tile in shared memory.
template <int TZ_> struct TileG {
    static constexpr int TX = 2, TZ = TZ_, TY = 256 / (TX * TZ_);
    static constexpr int SX = TX + 4, SY = TY + 4, SZ = TZ + 4;
    static constexpr int DXN = TX * SY * SZ, DYN = TX * TY * SZ, TILEN = SX * SY * SZ;
};
constexpr int GTHREADS = 256;

template <typename T> struct FlowParams {
    vec4_t<T> *phi[2];
    vec4_t<T> *vel[2];
    Ctrl *ctrl;
    double *parts;
    int n0, n1, n2;
    T m2, dt;
    ExtModel<T> ext;     // Section 7.8 extension terms (used by EXT instantiations)
    StencilScale<T> sc;  // scales of the unscaled derivatives
    double h3;
    int mode;
    double *slab_rec;  // x-slab: the step's record goes here, the decision is made later
};

template <typename T> __device__ __forceinline__ T comp(const vec4_t<T> &v, int A)
{
    return A == 0 ? v.x : (A == 1 ? v.y : (A == 2 ? v.z : v.w));
}

__device__ __forceinline__ size_t site_index(int x, int y, int z, int n1, int n2)
{
    return ((size_t)x * n1 + y) * (size_t)n2 + z;
}

// Stage the field tile with its halo; entries outside the lattice are left
// unwritten (only sites outside the interior would read them).
template <int TZ, typename T>
__device__ __forceinline__ void load_tile(vec4_t<T> *tile, const vec4_t<T> *phi, int x0, int y0,
                                          int z0, int n0, int n1, int n2)
{
    using G = TileG<TZ>;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    for (int i = tid; i < G::TILEN; i += GTHREADS) {
        const int lz = i % G::SZ, ly = (i / G::SZ) % G::SY, lx = i / (G::SZ * G::SY);
        const int x = x0 - 2 + lx, y = y0 - 2 + ly, z = z0 - 2 + lz;
        if (x < n0 && y < n1 && z < n2) tile[i] = load4<T>(phi + site_index(x, y, z, n1, n2));
    }
}

// The same staging with asynchronous copies (cp.async, 16 bytes per site of
// an FP32 field), committed as one group: the copies of the next tile fly
// while the current one is computed.
template <int TZ>
__device__ __forceinline__ void load_tile_async(float4 *tile, const float4 *phi, int x0, int y0,
                                                int z0, int n0, int n1, int n2)
{
    using G = TileG<TZ>;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    for (int i = tid; i < G::TILEN; i += GTHREADS) {
        const int lz = i % G::SZ, ly = (i / G::SZ) % G::SY, lx = i / (G::SZ * G::SY);
        const int x = x0 - 2 + lx, y = y0 - 2 + ly, z = z0 - 2 + lz;
        if (x < n0 && y < n1 && z < n2) {
            const unsigned dst = static_cast<unsigned>(__cvta_generic_to_shared(tile + i));
            const size_t src = __cvta_generic_to_global(phi + site_index(x, y, z, n1, n2));
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void wait_tile_async()
{
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// The Section 3 stencils without their 1/h factors (StencilScale carries
// them): u = 8 (p1 - m1) - (p2 - m2) = 12h d phi; the pure second derivative
// negated, N = (p2 + m2) + 30 c - 16 (p1 + m1) = -12h^2 dd phi; and the mixed
// one as the same first-derivative stencil of the u of the other direction,
// M = 8 (p1 - m1) - (p2 - m2) = 144h^2 d_ij phi = -12 N_ij.
template <typename T> __device__ __forceinline__ T sd1u(T m2v, T m1v, T p1v, T p2v)
{
    return fma(T(8), p1v - m1v, m2v - p2v);
}
template <typename T> __device__ __forceinline__ T sd2n(T m2v, T m1v, T c, T p1v, T p2v)
{
    return fma(T(-16), p1v + m1v, fma(T(30), c, p2v + m2v));
}
template <typename T>
__device__ __forceinline__ vec4_t<T> sd1uv(const vec4_t<T> &m2v, const vec4_t<T> &m1v,
                                           const vec4_t<T> &p1v, const vec4_t<T> &p2v)
{
    return make4<T>(sd1u<T>(m2v.x, m1v.x, p1v.x, p2v.x), sd1u<T>(m2v.y, m1v.y, p1v.y, p2v.y),
                    sd1u<T>(m2v.z, m1v.z, p1v.z, p2v.z), sd1u<T>(m2v.w, m1v.w, p1v.w, p2v.w));
}

// Shared-memory layout of the tile kernels: the haloed field tile, then
// d_x phi on the interior x-planes of the tile over (y, z) widened by 2, then
// d_y phi on the interior (x, y) rows of the tile over z widened by 2.  The
// mixed derivatives are first-derivative stencils of these (Section 3,
// the mixed stencil being the product of two first-derivative stencils:
// d_xy = d_y(d_x phi), d_xz = d_z(d_x phi), d_yz = d_z(d_y phi)),
// which costs a quarter of the FP64 operations of the 16-tap sums.
// FP32 kernels keep two field tiles, the next one arriving by cp.async.
template <typename T> constexpr int kTileBufs = sizeof(T) == 4 ? 2 : 1;
template <typename T, int TZ> constexpr size_t tile_smem_bytes()
{
    using G = TileG<TZ>;
    return (size_t)(kTileBufs<T> * G::TILEN + G::DXN + G::DYN) * sizeof(vec4_t<T>);
}

// Stage u_x and u_y (12h d_x phi, 12h d_y phi) of the tile (all threads),
// from the loaded tile.  Entries whose stencil leaves the lattice hold
// garbage that only sites outside the interior read.
template <int TZ, typename T>
__device__ __forceinline__ void stage_first_derivatives(const vec4_t<T> *tile, vec4_t<T> *dxs,
                                                        vec4_t<T> *dys)
{
    using G = TileG<TZ>;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    auto P = [&](int tx, int ty, int tz) -> const vec4_t<T> & { return tile[(tx * G::SY + ty) * G::SZ + tz]; };
    for (int i = tid; i < G::DXN; i += GTHREADS) {
        const int lz = i % G::SZ, ly = (i / G::SZ) % G::SY, lx = i / (G::SZ * G::SY);
        dxs[i] = sd1uv<T>(P(lx, ly, lz), P(lx + 1, ly, lz), P(lx + 3, ly, lz), P(lx + 4, ly, lz));
    }
    for (int i = tid; i < G::DYN; i += GTHREADS) {
        const int lz = i % G::SZ, ly = (i / G::SZ) % G::TY, lx = i / (G::SZ * G::TY);
        dys[i] = sd1uv<T>(P(lx + 2, ly, lz), P(lx + 2, ly + 1, lz), P(lx + 2, ly + 3, lz),
                          P(lx + 2, ly + 4, lz));
    }
}

// All derivatives of the site at local interior coordinate (lx, ly, lz),
// without their 1/h factors (u, N of the unscaled stencils above).
template <int TZ, typename T>
__device__ __forceinline__ void tile_derivatives(const vec4_t<T> *tile, const vec4_t<T> *dxs,
                                                 const vec4_t<T> *dys, int lx, int ly, int lz,
                                                 const FlowParams<T> &p, T phi[4], T d1[3][4],
                                                 T d2[3][4], T dm[3][4])
{
    using G = TileG<TZ>;
    auto P = [&](int dx, int dy, int dz) -> vec4_t<T> {
        return tile[((lx + 2 + dx) * G::SY + (ly + 2 + dy)) * G::SZ + (lz + 2 + dz)];
    };
    // d_x phi at (lx, ly + 2 + dy, lz + 2 + dz) and d_y phi at (lx, ly, lz + 2 + dz)
    auto DX = [&](int dy, int dz) -> vec4_t<T> { return dxs[(lx * G::SY + ly + 2 + dy) * G::SZ + lz + 2 + dz]; };
    auto DY = [&](int dz) -> vec4_t<T> { return dys[(lx * G::TY + ly) * G::SZ + lz + 2 + dz]; };
    (void)p;
    const vec4_t<T> c = P(0, 0, 0);
    const int off[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const vec4_t<T> m2v = P(-2 * off[i][0], -2 * off[i][1], -2 * off[i][2]);
        const vec4_t<T> m1v = P(-off[i][0], -off[i][1], -off[i][2]);
        const vec4_t<T> p1v = P(off[i][0], off[i][1], off[i][2]);
        const vec4_t<T> p2v = P(2 * off[i][0], 2 * off[i][1], 2 * off[i][2]);
#pragma unroll
        for (int A = 0; A < 4; ++A) {
            if (i == 2)
                d1[i][A] = sd1u<T>(comp<T>(m2v, A), comp<T>(m1v, A), comp<T>(p1v, A), comp<T>(p2v, A));
            d2[i][A] = sd2n<T>(comp<T>(m2v, A), comp<T>(m1v, A), comp<T>(c, A), comp<T>(p1v, A),
                               comp<T>(p2v, A));
        }
    }
    const vec4_t<T> dx0 = DX(0, 0), dy0 = DY(0);
    const vec4_t<T> xym2 = DX(-2, 0), xym1 = DX(-1, 0), xyp1 = DX(1, 0), xyp2 = DX(2, 0);
    const vec4_t<T> xzm2 = DX(0, -2), xzm1 = DX(0, -1), xzp1 = DX(0, 1), xzp2 = DX(0, 2);
    const vec4_t<T> yzm2 = DY(-2), yzm1 = DY(-1), yzp1 = DY(1), yzp2 = DY(2);
#pragma unroll
    for (int A = 0; A < 4; ++A) {
        phi[A] = comp<T>(c, A);
        d1[0][A] = comp<T>(dx0, A);
        d1[1][A] = comp<T>(dy0, A);
        dm[0][A] = sd1u<T>(comp<T>(xym2, A), comp<T>(xym1, A), comp<T>(xyp1, A), comp<T>(xyp2, A));
        dm[1][A] = sd1u<T>(comp<T>(xzm2, A), comp<T>(xzm1, A), comp<T>(xzp1, A), comp<T>(xzp2, A));
        dm[2][A] = sd1u<T>(comp<T>(yzm2, A), comp<T>(yzm1, A), comp<T>(yzp1, A), comp<T>(yzp2, A));
    }
}

template <typename T>
__device__ __forceinline__ void normalise_store(vec4_t<T> *dst, const T t[4])
{
    const T nn = t[0] * t[0] + t[1] * t[1] + t[2] * t[2] + t[3] * t[3];
    const T r = rsqrt(nn);  // within an ulp of 1/sqrt, without its division
    store4<T>(dst, make4<T>(t[0] * r, t[1] * r, t[2] * r, t[3] * r));
}

// Per-CTA partial record + last-CTA finish.  acc = {e2, e4, e0, b, |F|^2,
// |F|^2 (max), e6}; the sextic sum is reduced only when EXT.
template <typename T, bool EXT>
__device__ __forceinline__ void reduce_and_finish(const FlowParams<T> &p, double (&acc)[7],
                                                  bool energy_only, int pred)
{
    __shared__ double red[8 * (GTHREADS / 32)];
    __shared__ int s_last;
    constexpr int NQ = EXT ? 7 : 6;
    double tot6[NQ];
    block_reduce<NQ, 5>(*reinterpret_cast<double(*)[NQ]>(acc), red, tot6);
    const int nblocks = gridDim.x * gridDim.y * gridDim.z;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    if (tid == 0) {
        double *rec = p.parts + (size_t)bid * kPartialDoubles;
#pragma unroll
        for (int q = 0; q < 6; ++q) rec[q] = tot6[q];
        rec[6] = 0.0;
        rec[7] = EXT ? tot6[NQ - 1] : 0.0;
        __threadfence();
        unsigned int *ctr = energy_only ? &p.ctrl->edone : &p.ctrl->done;
        const unsigned int t = atomicAdd(ctr, 1u);
        s_last = (t == (unsigned int)(nblocks - 1));
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double tot[kPartialDoubles];
    reduce_partials(p.parts, nblocks, red, tot);
    if (tid == 0) {
        const double nsites = (double)(p.n0 - 4) * (double)(p.n1 - 4) * (double)(p.n2 - 4);
        tot[6] = nsites;
        if (energy_only) {
            Ctrl *c = p.ctrl;
            const double E2 = p.h3 * tot[0], E4 = p.h3 * tot[1], E0 = p.h3 * tot[2];
            const double E6 = p.h3 * tot[7];
            c->energy[0] = E2 + E4 + E0 + E6;
            c->energy[1] = E2;
            c->energy[2] = E4;
            c->energy[3] = E0;
            c->energy[4] = p.h3 * tot[3];
            c->energy[5] = -E2 + E4 - 3.0 * E0 + 3.0 * E6;
            c->e6_energy = E6;
            c->energy[6] = sqrt(tot[5]);
            c->energy[7] = sqrt(tot[4] / nsites);
            if (!(isfinite(c->energy[0]) && isfinite(c->energy[4]))) c->status = DEV_NONFINITE;
            c->edone = 0;
        } else if (p.slab_rec) {
            // one x-slab of a larger lattice: the arrest decision needs every
            // slab's sums, so this step only leaves its record
#pragma unroll
            for (int q = 0; q < kPartialDoubles; ++q) p.slab_rec[q] = tot[q];
            p.ctrl->done = 0;
        } else {
            finish_step(p.ctrl, tot, p.h3, p.mode, pred);
        }
    }
}

// Resident 256-thread CTAs per SM the register allocation is sized for:
// three for FP32 (24 warps to hide the latency of the tile loads), two for the
// standard FP64 kernels, one for the extended FP64 kernels (bound by the FP64
// pipe either way).
template <typename T, bool EXT>
constexpr int kTileMinBlocks = sizeof(T) == 4 ? 3 : (EXT ? 1 : 2);

// kind 0: fused step; kind 1: energy only; kind 2: per-site dump.
// EXT: the Section 7.8 extension terms are included.
template <typename T, int KIND, bool EXT, int TZ>
__global__ void __launch_bounds__(GTHREADS, kTileMinBlocks<T, EXT>) k_tile(FlowParams<T> p, vec4_t<T> *fout,
                                                   vec4_t<T> *dout)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    vec4_t<T> *tiles = reinterpret_cast<vec4_t<T> *>(smem_raw);
    using G = TileG<TZ>;
    vec4_t<T> *dxs = tiles + kTileBufs<T> * G::TILEN;
    vec4_t<T> *dys = dxs + G::DXN;
    const int cur = __ldcg(&p.ctrl->cur);
    const int pred = (KIND == 0 && p.mode == MODE_ARRESTED) ? __ldcg(&p.ctrl->pred) : 0;
    // buffers selected by value (a run-time index into the parameter copies it to the stack)
    const vec4_t<T> *phi = cur ? p.phi[1] : p.phi[0];
    const vec4_t<T> *vin = cur ? p.vel[1] : p.vel[0];
    vec4_t<T> *phi_out = cur ? p.phi[0] : p.phi[1];
    vec4_t<T> *vel_out = cur ? p.vel[0] : p.vel[1];
    const int lz = threadIdx.x, ly = threadIdx.y, lx = threadIdx.z;
    // persistent CTAs walk the tiles z-fastest, so CTAs in flight share halos in L2
    const int nz = (p.n2 - 4 + G::TZ - 1) / G::TZ, ny = (p.n1 - 4 + G::TY - 1) / G::TY;
    const int ntiles = nz * ny * ((p.n0 - 4 + G::TX - 1) / G::TX);
    // Per-thread sums {e2, e4, e0, b, |F|^2, max |F|^2, e6}.  The FP32 kernels
    // add in FP32 over at most kFoldTiles tiles and then fold into FP64, so
    // that the FP64 pipe (1/64 of the FP32 rate) does a few operations per
    // thread instead of seven per site; FP64 kernels add in FP64 directly.
    // In FP32 the energy, charge and sextic sums are compensated: each
    // addition's rounding error (Knuth's two-sum, exact) is added to comp[],
    // so part + comp carries no FP32 reduction error into the FP64 totals.
    constexpr int kFoldTiles = sizeof(T) == 4 ? 32 : 1;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    T part[7] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
    T comp[7] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
    int pending = 0;
    auto add = [&](int q, T x) {
        if constexpr (sizeof(T) == 4) {
            const T t = __fadd_rn(part[q], x);
            const T bb = __fsub_rn(t, part[q]);
            comp[q] = __fadd_rn(comp[q], __fadd_rn(__fsub_rn(part[q], __fsub_rn(t, bb)),
                                                   __fsub_rn(x, bb)));
            part[q] = t;
        } else {
            part[q] += x;
        }
    };
    auto fold = [&]() {
#pragma unroll
        for (int q = 0; q < 7; ++q)
            acc[q] = (q == 5) ? fmax(acc[q], (double)part[q])
                              : acc[q] + (double)part[q] + (double)comp[q];
#pragma unroll
        for (int q = 0; q < 7; ++q) part[q] = T(0), comp[q] = T(0);
        pending = 0;
    };
    auto x0_of = [&](int t) { return 2 + (t / (nz * ny)) * G::TX; };
    auto y0_of = [&](int t) { return 2 + ((t / nz) % ny) * G::TY; };
    auto z0_of = [&](int t) { return 2 + (t % nz) * G::TZ; };
    if constexpr (kTileBufs<T> == 2) {
        if (blockIdx.x < ntiles)
            load_tile_async<TZ>(tiles, phi, x0_of(blockIdx.x), y0_of(blockIdx.x), z0_of(blockIdx.x),
                            p.n0, p.n1, p.n2);
    }
    int buf = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, buf ^= (kTileBufs<T> - 1)) {
        const int x0 = x0_of(t), y0 = y0_of(t), z0 = z0_of(t);
        vec4_t<T> *tile = tiles + buf * G::TILEN;
        if constexpr (kTileBufs<T> == 2) {
            wait_tile_async();  // this thread's copies of tile t have landed
            // every thread's copies have landed, and every thread is done with
            // the other buffer and with the staged derivatives of tile t - grid
            __syncthreads();
            const int tn = t + gridDim.x;
            if (tn < ntiles)
                load_tile_async<TZ>(tiles + (buf ^ 1) * G::TILEN, phi, x0_of(tn), y0_of(tn), z0_of(tn),
                                p.n0, p.n1, p.n2);
        } else {
            __syncthreads();  // the previous tile's readers are done with shared memory
            load_tile<TZ, T>(tile, phi, x0, y0, z0, p.n0, p.n1, p.n2);
            __syncthreads();
        }
        stage_first_derivatives<TZ, T>(tile, dxs, dys);
        __syncthreads();
        const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
        if (!((x <= p.n0 - 3) && (y <= p.n1 - 3) && (z <= p.n2 - 3))) continue;
        T ph[4], d1[3][4], d2[3][4], dm[3][4], F[4], dens[4], e6 = T(0);
        tile_derivatives<TZ, T>(tile, dxs, dys, lx, ly, lz, p, ph, d1, d2, dm);
        site_physics<T, EXT>(ph, d1, d2, dm, p.m2, p.sc, F, dens, &p.ext, &e6);
        const size_t s = site_index(x, y, z, p.n1, p.n2);
        if (KIND == 0) {
            T tv[4];
            if (p.mode == MODE_GRADIENT) {
#pragma unroll
                for (int A = 0; A < 4; ++A) tv[A] = ph[A] + p.dt * F[A];
            } else {
                T v[4] = {T(0), T(0), T(0), T(0)};
                if (!pred) {
                    const vec4_t<T> vv = load4<T>(vin + s);
                    v[0] = vv.x; v[1] = vv.y; v[2] = vv.z; v[3] = vv.w;
                }
#pragma unroll
                for (int A = 0; A < 4; ++A) {
                    v[A] = v[A] + p.dt * F[A];
                    tv[A] = ph[A] + p.dt * v[A];
                }
                store4<T>(vel_out + s, make4<T>(v[0], v[1], v[2], v[3]));
            }
            normalise_store<T>(phi_out + s, tv);
        } else if (KIND == 2) {
            if (fout) store4<T>(fout + s, make4<T>(F[0], F[1], F[2], F[3]));
            if (dout) store4<T>(dout + s, make4<T>(dens[0], dens[1], dens[2], dens[3]));
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) add(q, dens[q]);
        const T f2 = F[0] * F[0] + F[1] * F[1] + F[2] * F[2] + F[3] * F[3];
        part[4] += f2;
        part[5] = part[5] > f2 ? part[5] : f2;
        if constexpr (EXT) add(6, e6);
        if (++pending == kFoldTiles) fold();
    }
    if (pending) fold();
    if (KIND == 2) return;
    reduce_and_finish<T, EXT>(p, acc, KIND == 1, pred);
}

// Pointwise correction of a mispredicted arrest decision: the step ran with
// the predicted rule, the finished step stored fix = -1 (velocity should have
// been zeroed) or +1 (it should have been kept), and the site update is redone
// from the previous buffers: v = v_new + fix v_old, phi = normalise(phi_old + dt v).
// One warp per z-row of interior sites; each lane stages the loads of
// kFixUnroll sites before its stores so that many loads are in flight.
template <typename T> __global__ void __launch_bounds__(512, 2) k_fixup(FlowParams<T> p)
{
    constexpr int kFixUnroll = sizeof(T) == 4 ? 2 : 1;
    const int fix = __ldcg(&p.ctrl->fix);
    if (fix == 0) return;
    const int nb = __ldcg(&p.ctrl->cur);  // new buffers (already flipped)
    const int ob = nb ^ 1;
    const int iy = p.n1 - 4, iz = p.n2 - 4, rows = (p.n0 - 4) * iy;
    const T sgn = T(fix);
    const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
    // buffer selection by value: a run-time index into the parameter would copy it to the stack
    vec4_t<T> *vnew = ob ? p.vel[0] : p.vel[1];
    vec4_t<T> *pnew = ob ? p.phi[0] : p.phi[1];
    const vec4_t<T> *vold = ob ? p.vel[1] : p.vel[0];
    const vec4_t<T> *pold = ob ? p.phi[1] : p.phi[0];
    for (int row = blockIdx.x * warps + (threadIdx.x >> 5); row < rows; row += gridDim.x * warps) {
        const int xr = row / iy;
        const size_t base = site_index(2 + xr, 2 + (row - xr * iy), 2, p.n1, p.n2);
        for (int z0 = 0; z0 < iz; z0 += 32 * kFixUnroll) {
            vec4_t<T> vn[kFixUnroll], vo[kFixUnroll], fo[kFixUnroll];
#pragma unroll
            for (int k = 0; k < kFixUnroll; ++k) {
                const int z = z0 + 32 * k + lane;
                if (z < iz) {
                    vn[k] = load4<T>(vnew + base + z);
                    vo[k] = load4<T>(vold + base + z);
                    fo[k] = load4<T>(pold + base + z);
                }
            }
#pragma unroll
            for (int k = 0; k < kFixUnroll; ++k) {
                const int z = z0 + 32 * k + lane;
                if (z < iz) {
                    const T v0 = vn[k].x + sgn * vo[k].x, v1 = vn[k].y + sgn * vo[k].y;
                    const T v2 = vn[k].z + sgn * vo[k].z, v3 = vn[k].w + sgn * vo[k].w;
                    const T t0 = fo[k].x + p.dt * v0, t1 = fo[k].y + p.dt * v1;
                    const T t2 = fo[k].z + p.dt * v2, t3 = fo[k].w + p.dt * v3;
                    store4<T>(vnew + base + z, make4<T>(v0, v1, v2, v3));
                    const T r = T(1) / sqrt(t0 * t0 + t1 * t1 + t2 * t2 + t3 * t3);
                    store4<T>(pnew + base + z, make4<T>(t0 * r, t1 * r, t2 * r, t3 * r));
                }
            }
        }
    }
}

// phi[1] <- phi[0] (read from src instead when it is given: a caller's field
// in pinned host memory, read over the host link); outer layers <- vacuum in
// both; velocities <- 0.
template <typename T> __global__ void k_load_finish(FlowParams<T> p, const vec4_t<T> *src)
{
    const vec4_t<T> *in = src ? src : p.phi[0];
    const size_t total = (size_t)p.n0 * p.n1 * p.n2;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int z = (int)(i % p.n2);
        const int y = (int)((i / p.n2) % p.n1);
        const int x = (int)(i / ((size_t)p.n2 * p.n1));
        const bool inner = x >= 2 && x <= p.n0 - 3 && y >= 2 && y <= p.n1 - 3 && z >= 2 &&
                           z <= p.n2 - 3;
        vec4_t<T> f = inner ? load4<T>(in + i) : make4<T>(T(1), T(0), T(0), T(0));
        store4<T>(p.phi[0] + i, f);
        store4<T>(p.phi[1] + i, f);
        store4<T>(p.vel[0] + i, make4<T>(T(0), T(0), T(0), T(0)));
        store4<T>(p.vel[1] + i, make4<T>(T(0), T(0), T(0), T(0)));
    }
}

__global__ void k_reset_ctrl(Ctrl *c)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        c->E_prev = __longlong_as_double(0x7ff0000000000000LL);  // +inf
        for (int i = 0; i < 8; ++i) c->last[i] = 0.0, c->energy[i] = 0.0;
        c->steps = 0;
        c->arrests = 0;
        c->fixups = 0;
        c->cur = 0;
        c->pred = 0;
        c->fix = 0;
        c->status = 0;
        c->done = 0;
        c->edone = 0;
        c->hist = 0;
        for (int i = 0; i < 16; ++i) c->pht[i] = 1;  // weakly "no arrest"
        c->until_start = 0;
        c->e6_last = 0.0;
        c->e6_energy = 0.0;
    }
}

// Run-to-tolerance graphs: a WHILE node repeats a body of `chunk` iterations.
// k_until_arm (in front of the node) records the step count and enters the
// loop; k_until_check (last in the body) keeps it going while the last
// iteration's delta = max |F| is above tol, fewer than max_steps iterations
// have run since the launch began, and no error was recorded.
__global__ void k_until_arm(Ctrl *c, cudaGraphConditionalHandle h)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        c->until_start = c->steps;
        cudaGraphSetConditional(h, c->status == 0 ? 1u : 0u);
    }
}
__global__ void k_until_check(Ctrl *c, cudaGraphConditionalHandle h, double tol, long long max_steps)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const bool more = c->status == 0 && !(c->last[6] <= tol) &&
                          c->steps - c->until_start < max_steps;
        cudaGraphSetConditional(h, more ? 1u : 0u);
    }
}

cudaError_t launch_until_arm(void *ctrl, unsigned long long handle, cudaStream_t s)
{
    k_until_arm<<<1, 32, 0, s>>>(static_cast<Ctrl *>(ctrl), handle);
    return cudaGetLastError();
}
cudaError_t launch_until_check(void *ctrl, unsigned long long handle, double tol,
                               long long max_steps, cudaStream_t s)
{
    k_until_check<<<1, 32, 0, s>>>(static_cast<Ctrl *>(ctrl), handle, tol, max_steps);
    return cudaGetLastError();
}

// ------------------------------------------------------------- launchers
// The persistent grid of the tile kernels never exceeds kTileGridCap CTAs
// (the partial-record space of the scratch holds at least that many).
constexpr int kTileGridCap = 152 * 8;

template <int TZ> static TileGeom tile_geometry_tz(const skyrme_lattice &lat)
{
    using G = TileG<TZ>;
    TileGeom g;
    const int ix = lat.n[0] - 4, iy = lat.n[1] - 4, iz = lat.n[2] - 4;
    const long long ntiles = (long long)((iz + G::TZ - 1) / G::TZ) * ((iy + G::TY - 1) / G::TY) *
                             ((ix + G::TX - 1) / G::TX);
    g.nblocks = (int)std::min<long long>(ntiles, kTileGridCap);
    g.grid = dim3(g.nblocks);
    g.block = dim3(G::TZ, G::TY, G::TX);
    g.smem = lat.precision == 64 ? tile_smem_bytes<double, TZ>() : tile_smem_bytes<float, TZ>();
    g.tz = TZ;
    return g;
}

// The 16-wide z tile is taken only where it leaves fewer idle lanes than the
// 32-wide one (it pays more halo per site where both pad alike).
TileGeom tile_geometry(const skyrme_lattice &lat)
{
    const int iz = lat.n[2] - 4;
    const int pad32 = (iz + 31) / 32 * 32 - iz, pad16 = (iz + 15) / 16 * 16 - iz;
    return pad16 < pad32 ? tile_geometry_tz<16>(lat) : tile_geometry_tz<32>(lat);
}

template <typename T> static FlowParams<T> make_params(const FlowArgs &a, double *parts)
{
    FlowParams<T> p;
    p.phi[0] = static_cast<vec4_t<T> *>(a.phi[0]);
    p.phi[1] = static_cast<vec4_t<T> *>(a.phi[1]);
    p.vel[0] = static_cast<vec4_t<T> *>(a.vel[0]);
    p.vel[1] = static_cast<vec4_t<T> *>(a.vel[1]);
    p.ctrl = static_cast<Ctrl *>(a.ctrl);
    p.parts = parts;
    p.n0 = a.n[0];
    p.n1 = a.n[1];
    p.n2 = a.n[2];
    {
        const double k1 = 1.0 / (12.0 * a.h);
        p.sc.k1sq = T(k1 * k1);
        p.sc.k1cu = T(k1 * k1 * k1);
        p.sc.k1qu = T(k1 * k1 * k1 * k1);
        p.sc.k1sx = T(k1 * k1 * k1 * k1 * k1 * k1);
        p.sc.B = T(12.0 * k1 * k1 * k1 * k1);
        p.sc.K144 = T(144.0 * a.h * a.h);
    }
    p.m2 = T(a.m * a.m);
    p.ext.my2 = T(a.my * a.my);
    p.ext.mz2 = T(a.mz * a.mz);
    p.ext.mw2 = T(a.mw * a.mw);
    p.ext.c6 = T(a.c6);
    p.dt = T(a.dt);
    p.h3 = a.h * a.h * a.h;
    p.mode = a.mode;
    p.slab_rec = a.slab_rec;
    return p;
}

template <typename T, int KIND, bool EXT, int TZ>
static cudaError_t launch_tile_geom(const TileGeom &g, const FlowParams<T> &p, vec4_t<T> *fo,
                                    vec4_t<T> *dout, cudaStream_t s)
{
    // resident CTAs of this instantiation on the whole GPU (queried once)
    static thread_local int resident = 0;
    if (!resident) {
        cudaError_t e = cudaFuncSetAttribute(k_tile<T, KIND, EXT, TZ>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)tile_smem_bytes<T, TZ>());
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per_sm = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile<T, KIND, EXT, TZ>,
                                                          GTHREADS, tile_smem_bytes<T, TZ>());
        if (e != cudaSuccess) return e;
        resident = std::max(1, sms * std::max(1, per_sm));
    }
    const int grid = std::min(g.nblocks, resident);
    k_tile<T, KIND, EXT, TZ><<<grid, g.block, g.smem, s>>>(p, fo, dout);
    return cudaGetLastError();
}

template <typename T, int KIND, bool EXT>
static cudaError_t launch_tile_model(const skyrme_lattice &lat, const FlowParams<T> &p,
                                     vec4_t<T> *fo, vec4_t<T> *dout, cudaStream_t s)
{
    const TileGeom g = tile_geometry(lat);
    return g.tz == 16 ? launch_tile_geom<T, KIND, EXT, 16>(g, p, fo, dout, s)
                      : launch_tile_geom<T, KIND, EXT, 32>(g, p, fo, dout, s);
}

template <typename T, int KIND>
static cudaError_t launch_tile(const skyrme_lattice &lat, const FlowParams<T> &p, vec4_t<T> *fo,
                               vec4_t<T> *dout, cudaStream_t s)
{
    return lattice_extended(lat) ? launch_tile_model<T, KIND, true>(lat, p, fo, dout, s)
                                 : launch_tile_model<T, KIND, false>(lat, p, fo, dout, s);
}

cudaError_t launch_step(const skyrme_lattice &lat, const FlowArgs &a, cudaStream_t s)
{
    if (lat.precision == 64)
        return launch_tile<double, 0>(lat, make_params<double>(a, a.step_parts), nullptr, nullptr, s);
    return launch_tile<float, 0>(lat, make_params<float>(a, a.step_parts), nullptr, nullptr, s);
}

cudaError_t launch_energy(const skyrme_lattice &lat, const FlowArgs &a, cudaStream_t s)
{
    if (lat.precision == 64)
        return launch_tile<double, 1>(lat, make_params<double>(a, a.energy_parts), nullptr, nullptr, s);
    return launch_tile<float, 1>(lat, make_params<float>(a, a.energy_parts), nullptr, nullptr, s);
}

cudaError_t launch_forces(const skyrme_lattice &lat, const FlowArgs &a, void *force, void *dens,
                          cudaStream_t s)
{
    if (lat.precision == 64)
        return launch_tile<double, 2>(lat, make_params<double>(a, a.energy_parts),
                                      static_cast<dvec4 *>(force), static_cast<dvec4 *>(dens), s);
    return launch_tile<float, 2>(lat, make_params<float>(a, a.energy_parts),
                                 static_cast<float4 *>(force), static_cast<float4 *>(dens), s);
}

static int pointwise_blocks(size_t total)
{
    size_t b = (total + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t launch_fixup(const skyrme_lattice &lat, const FlowArgs &a, cudaStream_t s)
{
    // mostly an early exit: one wave of 512-thread blocks, 16 rows each at most per pass
    const long long rows = (long long)(lat.n[0] - 4) * (lat.n[1] - 4);
    const int blocks = (int)std::max(1LL, std::min(304LL, (rows + 15) / 16));
    if (lat.precision == 64)
        k_fixup<double><<<blocks, 512, 0, s>>>(make_params<double>(a, a.step_parts));
    else
        k_fixup<float><<<blocks, 512, 0, s>>>(make_params<float>(a, a.step_parts));
    return cudaGetLastError();
}

cudaError_t launch_load_finish(const skyrme_lattice &lat, const FlowArgs &a, cudaStream_t s,
                               const void *src)
{
    const size_t total = (size_t)lat.n[0] * lat.n[1] * lat.n[2];
    if (lat.precision == 64)
        k_load_finish<double><<<pointwise_blocks(total), 256, 0, s>>>(
            make_params<double>(a, a.step_parts), static_cast<const vec4_t<double> *>(src));
    else
        k_load_finish<float><<<pointwise_blocks(total), 256, 0, s>>>(
            make_params<float>(a, a.step_parts), static_cast<const vec4_t<float> *>(src));
    return cudaGetLastError();
}

cudaError_t launch_reset_ctrl(void *ctrl, cudaStream_t s)
{
    k_reset_ctrl<<<1, 32, 0, s>>>(static_cast<Ctrl *>(ctrl));
    return cudaGetLastError();
}

// The arrest decision of a lattice cut into x-slabs (Section 3 arrest rule on
// the whole lattice's energy): the slabs' records {e2, e4, e0, b, |F|^2,
// max |F|^2, sites, e6} are combined in slab order, so every slab (every rank)
// that combines the same records reaches the same decision, predictor state
// and report; then the end-of-step bookkeeping of a whole lattice runs.
__global__ void k_slab_decide(Ctrl *c, const double *__restrict__ recs, int nslabs, double h3,
                              int mode)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double tot[kPartialDoubles];
#pragma unroll
    for (int q = 0; q < kPartialDoubles; ++q) tot[q] = 0.0;
    for (int sl = 0; sl < nslabs; ++sl)
#pragma unroll
        for (int q = 0; q < kPartialDoubles; ++q) {
            const double v = recs[(size_t)sl * kPartialDoubles + q];
            tot[q] = (q == 5) ? fmax(tot[q], v) : tot[q] + v;
        }
    const int pred = (mode == MODE_ARRESTED) ? c->pred : 0;
    finish_step(c, tot, h3, mode, pred);
}

cudaError_t launch_slab_decide(void *ctrl, const double *records, int nslabs, double h3, int mode,
                               cudaStream_t s)
{
    k_slab_decide<<<1, 32, 0, s>>>(static_cast<Ctrl *>(ctrl), records, nslabs, h3, mode);
    return cudaGetLastError();
}

}  // namespace skyrme
