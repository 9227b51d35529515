// flow_f32.cu -- FP32 streaming step kernel of the arrested Newton flow.
//
// Same iteration as the tile kernel (Section 3: 4th-order first, second and
// mixed derivatives, Euler-Lagrange gradient, tangent projection of
// Eq. "Newton_flow", v += dt F, phi = normalise(phi + dt v); Section 2.1
// densities summed in FP64), organised for GB300:
//
//  * two persistent CTAs per SM (16 warps); the CTAs split the (column,
//    x-plane) work of the lattice evenly.  A column is an 8 x 32 block of interior (y, z)
//    sites; a CTA marches along x through contiguous runs of planes.
//  * each x-plane of the column tile, with its 2-site halo (12 x 36 sites,
//    6.9 KB), is streamed into a 4-slot shared-memory ring by TMA
//    (cp.async.bulk.tensor.3d) and an mbarrier per slot; every wait is
//    bounded and reports SKYRME_ETIMEOUT instead of hanging.
//  * in-plane derivatives (d_y, d_z, d_yy, d_zz) come from the staged plane;
//    d_yz = d_z(d_y phi) uses a shared-memory exchange of d_y phi (with the
//    4 z-halo columns computed by 4 lanes per warp); d_x, d_xx, d_xy = d_x(d_y
//    phi), d_xz = d_x(d_z phi) come from a 5-plane register ring of (phi, d_y
//    phi, d_z phi) that the x-loop cycles through (unrolled by 5 so no
//    register is ever moved).  The in-plane contractions a plane contributes
//    to its own centre two planes later wait in a per-thread shared-memory
//    ring, and the velocity of each centre plane arrives by TMA together with
//    the field plane two planes ahead: this keeps the kernel at 128 registers,
//    two CTAs (16 warps) per SM.
//  * 4-vector arithmetic uses the packed FP32 pair instructions of sm_100+
//    (__ffma2_rn / __fadd2_rn / __fmul2_rn): two components per instruction.
//  * per-site densities are summed in FP32 over at most 20 consecutive planes
//    and then accumulated in FP64; the block and grid reductions are FP64 in
//    a fixed order, as in the tile kernel.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdlib.h>

#include "skyrme_device.cuh"
#include "skyrme_internal.h"

namespace skyrme {

constexpr int FTY = 8, FTZ = 32;
constexpr int FTHREADS = FTY * FTZ;  // 256: warp w owns row w of the tile
constexpr int FSY = FTY + 4, FSZ = FTZ + 4;
constexpr int NSLOT = 4;
constexpr unsigned PLANE_BYTES = FSY * FSZ * 16;   // 6912
constexpr unsigned VPLANE_BYTES = FTY * FTZ * 16;  // 4096
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s per plane copy

struct F32Params {
    float4 *phi[2];
    float4 *vel[2];
    Ctrl *ctrl;
    double *parts;
    int n0, n1, n2;
    int nzt;                // column tiles along z
    int nix;                // interior planes along x
    long long units;        // columns * nix
    float c1, c2;           // first-derivative weights / h
    float s1, s2, s0;       // second-derivative weights / h^2
    float m2, dt;
    double h3;
    int mode;
};

struct __align__(128) F32Smem {
    float4 plane[NSLOT][FSY][FSZ];   // haloed field planes (TMA)
    float4 vpl[NSLOT][FTY][FTZ];     // velocity planes of the centre sites (TMA)
    float4 dy[2][FTY][FSZ];          // d_y phi exchange for d_yz
    float4 inpl[3][4][FTHREADS];     // per-thread in-plane values of the last 3 planes
    unsigned long long bar[NSLOT];
    double red[8 * (FTHREADS / 32)];
    int flag;
    int last;
};

// ------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait: false when the phase did not complete within limit_ns.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity,
                                          unsigned long long limit_ns = kWaitLimitNs)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (global_ns() - t0 < limit_ns)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_plane(void *dst, const CUtensorMap *map,
                                          unsigned long long *bar, int c0, int c1, int c2)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

// ------------------------------------------------- packed 4-vector helpers
struct P4 {
    float2 a, b;  // components (0,1) and (2,3)
};
__device__ __forceinline__ float2 bc(float s) { return make_float2(s, s); }
__device__ __forceinline__ P4 ld4(const float4 &v) { return {make_float2(v.x, v.y), make_float2(v.z, v.w)}; }
__device__ __forceinline__ float4 st4(const P4 &v) { return make_float4(v.a.x, v.a.y, v.b.x, v.b.y); }
__device__ __forceinline__ P4 add(const P4 &u, const P4 &v) { return {__fadd2_rn(u.a, v.a), __fadd2_rn(u.b, v.b)}; }
// u - v
__device__ __forceinline__ P4 sub(const P4 &u, const P4 &v)
{
    return {__ffma2_rn(v.a, bc(-1.f), u.a), __ffma2_rn(v.b, bc(-1.f), u.b)};
}
__device__ __forceinline__ P4 mul(float2 s, const P4 &v) { return {__fmul2_rn(s, v.a), __fmul2_rn(s, v.b)}; }
__device__ __forceinline__ P4 fma(float2 s, const P4 &v, const P4 &c)
{
    return {__ffma2_rn(s, v.a, c.a), __ffma2_rn(s, v.b, c.b)};
}
__device__ __forceinline__ float2 dot2(const P4 &u, const P4 &v, float2 acc)
{
    return __ffma2_rn(u.b, v.b, __ffma2_rn(u.a, v.a, acc));
}
__device__ __forceinline__ float hsum(float2 t) { return t.x + t.y; }
__device__ __forceinline__ float dot(const P4 &u, const P4 &v)
{
    return hsum(__ffma2_rn(u.b, v.b, __fmul2_rn(u.a, v.a)));
}
// first derivative c1 (p1 - m1) + c2 (p2 - m2)
__device__ __forceinline__ P4 fd1(const P4 &m2, const P4 &m1, const P4 &p1, const P4 &p2, float c1,
                                  float c2)
{
    return fma(bc(c2), sub(p2, m2), mul(bc(c1), sub(p1, m1)));
}
// second derivative s1 (p1 + m1) + s2 (p2 + m2) + s0 c
__device__ __forceinline__ P4 fd2(const P4 &m2, const P4 &m1, const P4 &c, const P4 &p1,
                                  const P4 &p2, float s1, float s2, float s0)
{
    return fma(bc(s0), c, fma(bc(s2), add(p2, m2), mul(bc(s1), add(p1, m1))));
}

// Per-plane values of one column kept in the register x-ring.
struct PlaneVals {
    P4 phi, dy, dz;
};

struct Acc {
    float e2, e4, e0, b, f2, fmax2;
};

__device__ __forceinline__ void flush(double (&acc)[6], Acc &a)
{
    acc[0] += (double)a.e2;
    acc[1] += (double)a.e4;
    acc[2] += (double)a.e0;
    acc[3] += (double)a.b;
    acc[4] += (double)a.f2;
    acc[5] = fmax(acc[5], (double)a.fmax2);
    a = {0, 0, 0, 0, 0, 0};
}

// ------------------------------------------------------------------ kernel
__global__ void __launch_bounds__(FTHREADS, 2)
    k_step_f32(const __grid_constant__ CUtensorMap map0, const __grid_constant__ CUtensorMap map1,
               const __grid_constant__ CUtensorMap vmap0, const __grid_constant__ CUtensorMap vmap1,
               F32Params p)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    F32Smem &sm = *reinterpret_cast<F32Smem *>(smem_raw);
    const int tid = threadIdx.x;
    const int ty = tid >> 5, tz = tid & 31;
    Ctrl *ctrl = p.ctrl;
    const int cur = __ldcg(&ctrl->cur);
    const int pred = (p.mode == MODE_ARRESTED) ? __ldcg(&ctrl->pred) : 0;
    const CUtensorMap *map = cur ? &map1 : &map0;
    const CUtensorMap *vmap = cur ? &vmap1 : &vmap0;
    float4 *__restrict__ phiout = p.phi[cur ^ 1];
    float4 *__restrict__ vout = p.vel[cur ^ 1];
    const bool use_v = (p.mode != MODE_GRADIENT) && !pred;
    const float dt = p.dt, dt2 = 2.0f * p.dt;

    if (tid == 0) {
        for (int s = 0; s < NSLOT; ++s) mbar_init(&sm.bar[s], 1);
        mbar_fence_init();
        sm.flag = 0;
    }
    __syncthreads();

    double acc_d[6] = {0, 0, 0, 0, 0, 0};
    Acc a32 = {0, 0, 0, 0, 0, 0};
    uint32_t g = 0;  // planes consumed by this CTA (ring sequence number)
    bool failed = false;

    const long long u0 = p.units * blockIdx.x / gridDim.x;
    const long long u1 = p.units * (blockIdx.x + 1) / gridDim.x;
    const size_t plane_stride = (size_t)p.n1 * p.n2;

    for (long long us = u0; us < u1 && !failed;) {
        const long long col = us / p.nix;
        const long long ue = min(u1, (col + 1) * (long long)p.nix);
        const int xs = 2 + (int)(us - col * p.nix);
        const int xe = 2 + (int)(ue - col * p.nix);  // exclusive
        us = ue;
        const int y0 = 2 + (int)(col / p.nzt) * FTY, z0 = 2 + (int)(col % p.nzt) * FTZ;
        const int y = y0 + ty, z = z0 + tz;
        const bool valid = (y <= p.n1 - 3) && (z <= p.n2 - 3);
        const size_t col_off = (size_t)y * p.n2 + z;
        const int pf = xs - 2, pl = xe + 1;  // planes needed by this run
        // plane q travels with the velocity of centre q - 2 (when that is a centre)
        auto issue = [&](int q, int slot) {
            const bool wv = use_v && q - 2 >= xs && q - 2 < xe;
            mbar_expect_tx(&sm.bar[slot], PLANE_BYTES + (wv ? VPLANE_BYTES : 0u));
            tma_plane(&sm.plane[slot][0][0], map, &sm.bar[slot], 4 * (z0 - 2), y0 - 2, q);
            if (wv) tma_plane(&sm.vpl[slot][0][0], vmap, &sm.bar[slot], 4 * z0, y0, q - 2);
        };
        if (tid == 0)
            for (int q = 0; q < NSLOT && pf + q <= pl; ++q) issue(pf + q, (g + q) % NSLOT);
        PlaneVals ring[5];
        int nouter = 0;
        for (int base = pf; base <= pl && !failed; base += 5) {
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const int pp = base + k;
                if (pp > pl) break;
                const int s = g % NSLOT;
                const uint32_t par = (g / NSLOT) & 1u;
                if (!mbar_wait(&sm.bar[s], par)) sm.flag = 1;
                // ---- arrival of plane pp: in-plane first and second derivatives
                const float4(*P)[FSZ] = sm.plane[s];
                const P4 c = ld4(P[ty + 2][tz + 2]);
                const P4 ym2 = ld4(P[ty][tz + 2]), ym1 = ld4(P[ty + 1][tz + 2]);
                const P4 yp1 = ld4(P[ty + 3][tz + 2]), yp2 = ld4(P[ty + 4][tz + 2]);
                const P4 zm2 = ld4(P[ty + 2][tz]), zm1 = ld4(P[ty + 2][tz + 1]);
                const P4 zp1 = ld4(P[ty + 2][tz + 3]), zp2 = ld4(P[ty + 2][tz + 4]);
                const P4 dy = fd1(ym2, ym1, yp1, yp2, p.c1, p.c2);
                const P4 dz = fd1(zm2, zm1, zp1, zp2, p.c1, p.c2);
                const P4 dyy = fd2(ym2, ym1, c, yp1, yp2, p.s1, p.s2, p.s0);
                const P4 dzz = fd2(zm2, zm1, c, zp1, zp2, p.s1, p.s2, p.s0);
                float4(*DY)[FSZ] = sm.dy[g & 1];
                DY[ty][tz + 2] = st4(dy);
                if (tz < 4) {  // z-halo columns of d_y phi for this row
                    const int hc = tz < 2 ? tz : FTZ + tz;
                    DY[ty][hc] = st4(fd1(ld4(P[ty][hc]), ld4(P[ty + 1][hc]), ld4(P[ty + 3][hc]),
                                         ld4(P[ty + 4][hc]), p.c1, p.c2));
                }
                ring[k].phi = c;
                ring[k].dy = dy;
                ring[k].dz = dz;

                // ---- centre x = pp - 2: x-derivatives, physics, update
                const int x = pp - 2;
                if (x >= xs) {
                    const PlaneVals &M2 = ring[(k + 1) % 5], &M1 = ring[(k + 2) % 5];
                    const PlaneVals &C = ring[(k + 3) % 5], &Q1 = ring[(k + 4) % 5];
                    const PlaneVals &Q2 = ring[k];
                    const float4 *rec = &sm.inpl[(g + 1) % 3][0][tid];  // plane x = pp - 2
                    const P4 lin = ld4(rec[0]), qin = ld4(rec[FTHREADS]);
                    const float4 r2 = rec[2 * FTHREADS];
                    const float Cgy = r2.x, Cgz = r2.y, Cayy = r2.z, Cazz = r2.w;
                    const float Cayz = rec[3 * FTHREADS].x;
                    const P4 ph = C.phi;
                    const P4 dx = fd1(M2.phi, M1.phi, Q1.phi, Q2.phi, p.c1, p.c2);
                    const P4 dxx = fd2(M2.phi, M1.phi, ph, Q1.phi, Q2.phi, p.s1, p.s2, p.s0);
                    const P4 dxy = fd1(M2.dy, M1.dy, Q1.dy, Q2.dy, p.c1, p.c2);
                    const P4 dxz = fd1(M2.dz, M1.dz, Q1.dz, Q2.dz, p.c1, p.c2);
                    const P4 dyc = C.dy, dzc = C.dz;
                    const float axx = dot(dx, dx), axy = dot(dx, dyc), axz = dot(dx, dzc);
                    const float tra = axx + Cayy + Cazz;
                    const P4 L = add(dxx, lin);
                    // g_i = sum_j d_ij phi.d_j phi; c_i = g_i - Laplacian.d_i phi
                    const float gx = hsum(dot2(dxz, dzc, dot2(dxy, dyc,
                                                   __ffma2_rn(dxx.b, dx.b, __fmul2_rn(dxx.a, dx.a)))));
                    const float gy = dot(dxy, dx) + Cgy;
                    const float gz = dot(dxz, dx) + Cgz;
                    const float ccx = gx - dot(L, dx), ccy = gy - dot(L, dyc), ccz = gz - dot(L, dzc);
                    // d_ij phi a_ij summed over i, j
                    const P4 Ha = fma(bc(2.f * axz), dxz, fma(bc(2.f * axy), dxy, fma(bc(axx), dxx, qin)));
                    // brace of the Euler-Lagrange equation; G = -2 (brace + m^2 e_0)
                    P4 br = fma(bc(ccz), dzc, fma(bc(ccy), dyc, fma(bc(ccx), dx,
                                fma(bc(1.f + tra), L, mul(bc(-1.f), Ha)))));
                    br.a.x += p.m2;
                    // F = -G + (G.phi) phi = 2 (br - (br.phi) phi)
                    const float bp = dot(br, ph);
                    const P4 Fh = fma(bc(-bp), ph, br);
                    const float f2 = 4.f * dot(Fh, Fh);
                    P4 t, vnew;
                    if (p.mode == MODE_GRADIENT) {
                        t = fma(bc(dt2), Fh, ph);
                    } else {
                        const P4 vo = use_v ? ld4(sm.vpl[s][ty][tz]) : P4{bc(0.f), bc(0.f)};
                        vnew = fma(bc(dt2), Fh, vo);
                        t = fma(bc(dt), vnew, ph);
                    }
                    const float r = rsqrtf(dot(t, t));
                    const P4 pn = mul(bc(r), t);
                    const float sq = axx * axx + Cayy * Cayy + Cazz * Cazz +
                                     2.f * (axy * axy + axz * axz + Cayz * Cayz);
                    const float e4 = 0.5f * (tra * tra - sq);
                    // det[phi, d_x phi, d_y phi, d_z phi] by 2x2 minors of rows (phi, d_x) and (d_y, d_z)
                    const float s0 = ph.a.x * dx.a.y - dx.a.x * ph.a.y;
                    const float2 s12 = __ffma2_rn(bc(-dx.a.x), ph.b, __fmul2_rn(bc(ph.a.x), dx.b));
                    const float2 s34 = __ffma2_rn(bc(-dx.a.y), ph.b, __fmul2_rn(bc(ph.a.y), dx.b));
                    const float s5 = ph.b.x * dx.b.y - dx.b.x * ph.b.y;
                    const float q0 = dyc.a.x * dzc.a.y - dzc.a.x * dyc.a.y;
                    const float2 q12 = __ffma2_rn(bc(-dzc.a.x), dyc.b, __fmul2_rn(bc(dyc.a.x), dzc.b));
                    const float2 q34 = __ffma2_rn(bc(-dzc.a.y), dyc.b, __fmul2_rn(bc(dyc.a.y), dzc.b));
                    const float q5 = dyc.b.x * dzc.b.y - dzc.b.x * dyc.b.y;
                    const float det = s0 * q5 - s12.x * q34.y + s12.y * q34.x + s34.x * q12.y -
                                      s34.y * q12.x + s5 * q0;
                    if (valid) {
                        const size_t si = (size_t)x * plane_stride + col_off;
                        __stcs(phiout + si, st4(pn));
                        if (p.mode != MODE_GRADIENT) __stcs(vout + si, st4(vnew));
                        a32.e2 += tra;
                        a32.e4 += e4;
                        a32.e0 += 1.f - ph.a.x;
                        a32.b += det;
                        a32.f2 += f2;
                        a32.fmax2 = fmaxf(a32.fmax2, f2);
                    }
                }
                __syncthreads();
                if (sm.flag) {
                    failed = true;
                    break;
                }
                // slot s is free again: stream plane pp + NSLOT (and its velocity) into it
                if (tid == 0 && pp + NSLOT <= pl) issue(pp + NSLOT, s);
                // ---- in-plane values of plane pp for its own centre, two planes on
                const P4 dyz = fd1(ld4(DY[ty][tz]), ld4(DY[ty][tz + 1]), ld4(DY[ty][tz + 3]),
                                   ld4(DY[ty][tz + 4]), p.c1, p.c2);
                const float ayy = dot(dy, dy), azz = dot(dz, dz), ayz = dot(dy, dz);
                const P4 lin = add(dyy, dzz);
                const P4 qin = fma(bc(2.f * ayz), dyz, fma(bc(azz), dzz, mul(bc(ayy), dyy)));
                const float gyv = hsum(dot2(dyz, dz, __ffma2_rn(dyy.b, dy.b, __fmul2_rn(dyy.a, dy.a))));
                const float gzv = hsum(dot2(dzz, dz, __ffma2_rn(dyz.b, dy.b, __fmul2_rn(dyz.a, dy.a))));
                float4 *wrec = &sm.inpl[g % 3][0][tid];
                wrec[0] = st4(lin);
                wrec[FTHREADS] = st4(qin);
                wrec[2 * FTHREADS] = make_float4(gyv, gzv, ayy, azz);
                wrec[3 * FTHREADS] = make_float4(ayz, 0.f, 0.f, 0.f);
                ++g;
            }
            // FP32 partial sums cover at most 20 planes before entering FP64
            if ((++nouter & 3) == 0) flush(acc_d, a32);
        }
        flush(acc_d, a32);
    }

    if (failed) {
        // a plane copy never landed: record it, let in-flight copies finish
        // (bounded), and leave without touching the reduction counter
        if (tid == 0) {
            atomicExch(&ctrl->status, (int)DEV_TIMEOUT);
            for (int s = 0; s < NSLOT; ++s) {
                (void)mbar_wait(&sm.bar[s], 0, 50000000ull);
                (void)mbar_wait(&sm.bar[s], 1, 50000000ull);
            }
        }
        return;
    }

    // ---- block and grid reductions (FP64, fixed order)
    acc_d[2] *= 2.0 * (double)p.m2;     // e0 = 2 m^2 (1 - phi^0)
    acc_d[3] *= -0.050660591821168885;  // b = -det / (2 pi^2)
    double tot6[6];
    block_reduce<6, 5>(acc_d, sm.red, tot6);
    if (tid == 0) {
        double *rec = p.parts + (size_t)blockIdx.x * kPartialDoubles;
        for (int q = 0; q < 6; ++q) rec[q] = tot6[q];
        rec[6] = rec[7] = 0.0;
        __threadfence();
        sm.last = (atomicAdd(&ctrl->done, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!sm.last) return;
    __threadfence();
    double tot[kPartialDoubles];
    reduce_partials(p.parts, gridDim.x, sm.red, tot);
    if (tid == 0) {
        tot[6] = (double)(p.n0 - 4) * (double)(p.n1 - 4) * (double)(p.n2 - 4);
        finish_step(ctrl, tot, p.h3, p.mode, pred);
    }
}

// ------------------------------------------------------------------- host
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    }
    return fn;
}

// 3D view (4 n2 floats, n1, n0) of a float4 site array; one box is a
// box_z-float by box_y-row tile of a single x-plane.
static bool make_plane_map(CUtensorMap *m, const void *base, const skyrme_lattice &lat,
                           unsigned box_z, unsigned box_y)
{
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)4 * lat.n[2], (cuuint64_t)lat.n[1], (cuuint64_t)lat.n[0]};
    const cuuint64_t strides[2] = {(cuuint64_t)lat.n[2] * 16, (cuuint64_t)lat.n[1] * lat.n[2] * 16};
    const cuuint32_t box[3] = {box_z, box_y, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

static int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 152;
    return n > 0 ? n : 152;
}

bool f32_fast_path_available(const skyrme_lattice &lat)
{
    // the streaming kernel needs 16-byte aligned TMA rows (always true for
    // float4 sites) and a driver that exposes the tensor-map encoder
    return lat.precision == 32 && encode_fn() != nullptr;
}

int f32_fast_blocks(const skyrme_lattice &lat)
{
    (void)lat;
    return 1216;  // upper bound on the persistent grid (one CTA per SM)
}

cudaError_t launch_step_f32_fast(const skyrme_lattice &lat, const FlowArgs &a, cudaStream_t s)
{
    CUtensorMap m0, m1, v0, v1;
    if (!make_plane_map(&m0, a.phi[0], lat, 4 * FSZ, FSY) ||
        !make_plane_map(&m1, a.phi[1], lat, 4 * FSZ, FSY) ||
        !make_plane_map(&v0, a.vel[0], lat, 4 * FTZ, FTY) ||
        !make_plane_map(&v1, a.vel[1], lat, 4 * FTZ, FTY))
        return cudaErrorInvalidValue;
    static thread_local int smem_set_device = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (smem_set_device != dev) {
        cudaError_t e = cudaFuncSetAttribute(k_step_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(F32Smem));
        if (e != cudaSuccess) return e;
        smem_set_device = dev;
    }
    F32Params p;
    p.phi[0] = static_cast<float4 *>(a.phi[0]);
    p.phi[1] = static_cast<float4 *>(a.phi[1]);
    p.vel[0] = static_cast<float4 *>(a.vel[0]);
    p.vel[1] = static_cast<float4 *>(a.vel[1]);
    p.ctrl = static_cast<Ctrl *>(a.ctrl);
    p.parts = a.step_parts;
    p.n0 = lat.n[0];
    p.n1 = lat.n[1];
    p.n2 = lat.n[2];
    const int nyt = (lat.n[1] - 4 + FTY - 1) / FTY;
    p.nzt = (lat.n[2] - 4 + FTZ - 1) / FTZ;
    p.nix = lat.n[0] - 4;
    p.units = (long long)nyt * p.nzt * p.nix;
    const double ih = 1.0 / lat.h, ih2 = ih * ih;
    p.c1 = (float)(2.0 / 3.0 * ih);
    p.c2 = (float)(-1.0 / 12.0 * ih);
    p.s1 = (float)(4.0 / 3.0 * ih2);
    p.s2 = (float)(-1.0 / 12.0 * ih2);
    p.s0 = (float)(-2.5 * ih2);
    p.m2 = (float)(lat.m * lat.m);
    p.dt = (float)a.dt;
    p.h3 = lat.h * lat.h * lat.h;
    p.mode = a.mode;
    long long grid = 2LL * sm_count();
    if (grid > p.units) grid = p.units;
    if (grid > f32_fast_blocks(lat)) grid = f32_fast_blocks(lat);
    if (grid < 1) grid = 1;
    k_step_f32<<<(unsigned)grid, FTHREADS, sizeof(F32Smem), s>>>(m0, m1, v0, v1, p);
    return cudaGetLastError();
}

}  // namespace skyrme
