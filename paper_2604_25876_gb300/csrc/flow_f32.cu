// flow_f32.cu -- FP32 streaming step kernel of the arrested Newton flow, for
// one lattice or a batch of independent lattices of uneven sizes.
//
// Same iteration as the tile kernel (Section 3: 4th-order first, second and
// mixed derivatives, Euler-Lagrange gradient, tangent projection of
// Eq. "Newton_flow", v += dt F, phi = normalise(phi + dt v); Section 2.1
// densities), organised for GB300:
//
//  * persistent CTAs (as many as fit: one per SM for a single lattice, with
//    16 x 32 columns) split the (column, x-plane) work of every lattice in
//    the batch.  A column is a TY x TZ block of interior (y, z) sites; a CTA
//    marches along x through contiguous runs of planes, crossing from one
//    lattice into the next.  A batch is split evenly by units; a single
//    lattice by streamed planes, a run of r centres streaming r + 4 planes,
//    so that CTAs whose range spans two columns get fewer centres.  Each lattice's energy sums close as soon as the CTAs that
//    touched it are done (per-lattice arrival counter, last-CTA finish), so
//    lattices of different sizes need no global barrier.
//  * each x-plane of the column tile, with its 2-site halo, is streamed into
//    a shared-memory ring (8 slots for a single lattice's 16 x 32 tile, else
//    4) by TMA (cp.async.bulk.tensor.3d) with an
//    mbarrier per slot; every wait is bounded and reports SKYRME_ETIMEOUT
//    instead of hanging.  Warps consume the planes independently: the last
//    warp to be done with a slot (a shared-memory counter) streams the next
//    plane into it, so the only CTA-wide barriers are at the ends of runs.
//  * the in-plane values a plane contributes to its own centre two planes
//    later (13 per site) wait in tensor memory: each warp keeps a 3-slot ring
//    of them in its TMEM lanes (tcgen05.st / tcgen05.ld), which takes them
//    off the shared-memory pipe and out of shared memory.
//  * derivatives are carried without their 1/(12h), 1/(12h^2) factors (the
//    first-derivative stencil is then 3 instructions per component pair, the
//    second 4); the factors move into the time step, the mass terms and the
//    FP64 scale of the sums.
//  * in-plane derivatives (d_y, d_z, d_yy, d_zz) come from the staged plane;
//    d_yz = d_z(d_y phi) uses a per-warp shared-memory exchange of d_y phi
//    (each warp computes the 4 z-halo columns of its own rows, one
//    component per lane); d_x, d_xx,
//    d_xy = d_x(d_y phi), d_xz = d_x(d_z phi) come from a 5-plane register
//    ring of (phi, d_y phi, d_z phi) that the x-loop cycles through (unrolled
//    by 5 so no register is ever moved).  The velocity of each centre plane
//    arrives by TMA together with the field plane two planes ahead.
//  * 4-vector arithmetic uses the packed FP32 pair instructions of sm_100+
//    (__ffma2_rn / __fadd2_rn / __fmul2_rn): two components per instruction;
//    stencil weights are stored as (w, w) pairs.
//  * per-site energy and charge densities enter compensated FP32 sums
//    (Knuth's error-free two-sum at every addition, the rounding errors summed
//    exactly beside them), folded every 40 planes into double-float (hi, lo)
//    pairs kept in shared memory; block and per-lattice reductions are
//    double-float in a fixed order, and the arrest comparison is made in FP64
//    on the rounded totals.
//  * the tile shape (TY, TZ) is a template parameter; the batch autotuner
//    times the candidates on the actual lattices and keeps the fastest.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdlib.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string.h>

#include <vector>

#include "skyrme_device.cuh"
#include "skyrme_internal.h"

namespace skyrme {

// Depth of the TMA plane ring: 8 slots for the 512-thread tile of a single
// lattice (one CTA per SM; more copies in flight), 4 for the smaller tiles
// that share an SM and for the sextic variant (its register spills live in
// the L1 share of the SM's shared-memory array).  A power of two keeps the
// slot arithmetic to shifts.
template <int TY, int TZ, bool SEX = false> constexpr int nslot()
{
    return TY * TZ >= 512 && !SEX ? 8 : 4;
}
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s per plane copy

// One lattice of a step launch: a kernel parameter for a single lattice, an
// entry of a device table for a batch.
struct InstDesc {
    CUtensorMap map[2];   // haloed field planes of phi[0], phi[1]
    CUtensorMap vmap[2];  // centre-site velocity planes of vel[0], vel[1]
    float4 *phi[2];
    float4 *vel[2];
    Ctrl *ctrl;
    double *parts;         // per-CTA partial records of this lattice
    long long unit_start;  // first global work unit (column-plane) of the lattice
    long long units;       // columns * interior planes
    int n0, n1, n2;
    int nzt, nix;          // column tiles along z, interior planes along x
    int cta_first, cta_count;
    // Time steps as (w, w) pairs: the packed FP32 instructions take them as
    // one 64-bit operand.  The kernels carry the derivatives without their
    // 1/(12h), 1/(12h^2) factors: u_i = 12h d_i phi = 8 (p1 - m1) - (p2 - m2),
    // and every second derivative negated on one scale, N_ij = -12h^2 d_ij phi:
    // the pure ones as (p2 + m2) + 30 c - 16 (p1 + m1), the mixed N_yz (and
    // N_xy, N_xz in the sextic variant) as -(2/3)(p1 - m1) + (1/12)(p2 - m2)
    // of the u_i; the other kernels take N_xy, N_xz as -1/12 of the
    // first-derivative stencil of u_y, u_z along x, the factor applied where
    // they enter (weights the same for every lattice: kW8 ... kXm2).  The
    // force then comes out as F / B,
    // B = 1/(1728 h^4); B moves into the time step and the mass terms, and
    // the sums are scaled in the finish.
    float2 dt, dt2;        // dt and 2 dt B
    float m2;              // m^2 (potential energy density)
    float bm2;             // m^2 / B (its force term)
    float negK;            // -144 h^2: the quadratic term of the force against the quartic ones
    // Section 7.8 potentials (the POT kernels): squared masses of the
    // modified-pion, loosely and lightly bound terms, and the same / B
    float my2, mz2, mw2;
    float bmy2, bmz2, bmw2;
    float e0_scale;        // E0 = h^3 e0_scale sum(e0 slot): 2 m^2 (standard) or 1 (POT)
    float c6;              // Section 7.8 sextic coefficient (the SEX kernels)
    float c6b;             // c6 / (144 h^2): the sextic force term's weight
    float dk2, dk3, dk4;   // DUMP kernels: (12h)^-2, ^-3, ^-4 to the densities they write
    // (hi, lo) factors of the sums: e2 (12h)^-2, e4 (12h)^-4, det (12h)^-3,
    // e6 (12h)^-6, |F|^2 B^2 (all 1 but |F|^2 in the DUMP kernels, whose
    // per-site densities are already scaled)
    float2 s_e2, s_e4, s_b, s_e6, s_f;
    float h3_hi, h3_lo;    // h^3 as an unevaluated float sum
    int mode;
    double *slab_rec;      // x-slab of a larger lattice: record out, no decision (else null)
    float4 *dump;          // DUMP kernels: per-site densities the step sums
    int fuse_fix;          // single lattice, ARRESTED: the step corrects its own mispredictions
};

// Unit ranges of the CTAs of a single-lattice launch.
//   n > 0, the balanced split: CTA b streams units [start[b], start[b + 1])
//     (column-major), the ranges balanced by their plane count (units plus
//     the pipeline fill of every run) rather than by units.
//   n = 0: the even split of the units.
//   n = -2, the lockstep schedule: lw waves of whole columns (CTA b streams
//     columns b, b + lg, ..., b + (lw - 1) lg, every CTA at the same x), then
//     of the lr remaining columns CTA b < lr streams the head x < la of
//     column lw lg + b while CTAs b >= lr stream the tails x >= la, tail units
//     start[b] .. start[b + 1] (tail by tail).  Neighbouring columns are
//     streamed side by side, so the halo rows they share are read from L2.
constexpr int kSplitMax = 256;
struct CtaSplit {
    int n;
    int lw, lr, la, lg;
    int start[kSplitMax + 1];
};

// Units of CTA b under the lockstep schedule, and the run that starts at its
// unit o (of o1): column, first interior plane (0-based) and length.
__host__ __device__ __forceinline__ int lock_units(const CtaSplit &sp, int b, int nix)
{
    return sp.lw * nix + (b < sp.lr ? sp.la : sp.start[b + 1] - sp.start[b]);
}
__host__ __device__ __forceinline__ void lock_run(const CtaSplit &sp, int b, int nix, int o, int o1,
                                                  int &col, int &xl, int &len)
{
    const int wu = sp.lw * nix;
    if (o < wu) {
        const int w = o / nix;
        col = w * sp.lg + b;
        xl = o - w * nix;
        len = nix - xl;
    } else if (b < sp.lr) {
        col = sp.lw * sp.lg + b;
        xl = o - wu;
        len = sp.la - xl;
    } else {
        const int tn = nix - sp.la, t = sp.start[b] + (o - wu), c2 = t / tn;
        col = sp.lw * sp.lg + c2;
        xl = sp.la + (t - c2 * tn);
        len = nix - xl;
    }
    len = len < o1 - o ? len : o1 - o;
}

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
// The same wait that also gives up once *flag is set (another warp's wait
// failed); the flag is read only when the phase is not complete at once.
__device__ __forceinline__ bool mbar_wait_flag(unsigned long long *bar, uint32_t parity,
                                               const volatile int *flag)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (*flag == 0 && global_ns() - t0 < kWaitLimitNs)
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


// ------------------------------------------------- tensor memory helpers
// Tensor memory (256 KiB per SM: 128 lanes x 512 columns of 32 bits) holds
// each thread's ring of in-plane records.  Warp 0 allocates the CTA's
// columns when the kernel starts and frees them when it ends, on every path
// (tcgen05.alloc / tcgen05.dealloc).  A warp can address only the 32 lanes of
// its quarter of a warpgroup, 32 * (warp % 4); among the warps sharing those
// lanes, warp w owns columns [C * (w / 4), C * (w / 4) + C) with
// C = tmem_cols_per_warp.
// Thread t of a warp reads and writes its own lane (the 32x32b shapes).
// One in-plane record: 16 columns (12 values used), or 32 (24 used) in the
// sextic kernels, which also carry d_yy, d_zz and d_yz phi to the centre.
template <bool SEX> constexpr int rec_cols() { return SEX ? 32 : 16; }
// the sextic variant also keeps the d_z phi part of its x-ring (5 planes of
// 4 values) in tensor memory, after its 3 records, for the registers; its
// warps' column ranges are padded to 128 (4 warps share a lane quarter: 512)
// so that every record starts on a 32-column boundary
constexpr int kDzCol = 3 * 32;
template <bool SEX> constexpr int tmem_cols_per_warp()
{
    return SEX ? 128 : 3 * rec_cols<SEX>();  // 3 records in flight (+ the d_z ring)
}
template <int NW, bool SEX = false> constexpr uint32_t tmem_cols()
{
    constexpr int need = ((NW + 3) / 4) * tmem_cols_per_warp<SEX>();
    static_assert(need <= 512, "the warps' TMEM columns exceed the SM's 512");
    return need <= 32 ? 32 : need <= 64 ? 64 : need <= 128 ? 128 : need <= 256 ? 256 : 512;
}
__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// Stores and loads of 8, 4 and 1 consecutive columns of this thread's TMEM
// lane (32x32b shapes).  Loaded values are usable only after a wait, so they
// pass through the wait's own operands (no use can be scheduled before it).
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float *v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]) : "memory");
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const float *v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]) : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];" : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]) : "r"(taddr) : "memory");
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float *v)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];" : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "r"(taddr) : "memory");
}
__device__ __forceinline__ void tmem_wait_ld16(float (&v)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]), "+f"(v[6]), "+f"(v[7]), "+f"(v[8]), "+f"(v[9]), "+f"(v[10]), "+f"(v[11]), "+f"(v[12]), "+f"(v[13]), "+f"(v[14]), "+f"(v[15]) : : "memory");
}
__device__ __forceinline__ void tmem_wait_ld12(float (&v)[12])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]), "+f"(v[6]), "+f"(v[7]), "+f"(v[8]), "+f"(v[9]), "+f"(v[10]), "+f"(v[11]) : : "memory");
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
// The unscaled stencils' weights, the same for every lattice (compile-time
// constants: the compiler takes them from its constant bank instead of
// registers, which matters in the batched kernels, whose lattice
// descriptors live in global memory)
__device__ __forceinline__ float2 kW8() { return make_float2(8.f, 8.f); }
__device__ __forceinline__ float2 kWm16() { return make_float2(-16.f, -16.f); }
__device__ __forceinline__ float2 kW30() { return make_float2(30.f, 30.f); }
__device__ __forceinline__ float2 kXm1() { return make_float2(-2.f / 3.f, -2.f / 3.f); }
__device__ __forceinline__ float2 kXm2() { return make_float2(1.f / 12.f, 1.f / 12.f); }

// weighted first difference c1 (p1 - m1) + c2 (p2 - m2) (the mixed second
// derivatives, of the u_i)
__device__ __forceinline__ P4 fd1(const P4 &m2, const P4 &m1, const P4 &p1, const P4 &p2, float2 c1,
                                  float2 c2)
{
    return fma(c2, sub(p2, m2), mul(c1, sub(p1, m1)));
}
// 12h d phi = 8 (p1 - m1) - (p2 - m2), w8 = (8, 8)
__device__ __forceinline__ P4 fd1u(const P4 &m2, const P4 &m1, const P4 &p1, const P4 &p2,
                                   float2 w8)
{
    return fma(w8, sub(p1, m1), sub(m2, p2));
}
// -12h^2 d^2 phi = (p2 + m2) + 30 c - 16 (p1 + m1), wm16 = (-16, -16), w30 = (30, 30)
__device__ __forceinline__ P4 fd2n(const P4 &m2, const P4 &m1, const P4 &c, const P4 &p1,
                                   const P4 &p2, float2 wm16, float2 w30)
{
    return fma(wm16, add(p1, m1), fma(w30, c, add(p2, m2)));
}

// ------------------------------------------------- double-float sums
// The streaming kernel keeps its energy, charge and force sums as unevaluated
// sums hi + lo of two floats (|lo| <= ulp(hi)/2), combined with the error-free
// two-sum and FMA two-product transformations (Knuth, Dekker): about 48
// significant bits on the FP32 pipe.  GB300's FP64 pipe issues 2 operations
// per SM and cycle, so FP64 reductions at the end of a launch sit on the
// critical path; these do not.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ DF quick_two_sum(float a, float b)  // |a| >= |b|
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_add(DF a, DF b)
{
    float s, e, t, f;
    two_sum(a.hi, b.hi, s, e);
    two_sum(a.lo, b.lo, t, f);
    DF r = quick_two_sum(s, __fadd_rn(e, t));
    return quick_two_sum(r.hi, __fadd_rn(r.lo, f));
}
__device__ __forceinline__ DF df_add(DF a, float x)
{
    float s, e;
    two_sum(a.hi, x, s, e);
    return quick_two_sum(s, __fadd_rn(e, a.lo));
}
__device__ __forceinline__ DF df_mul(DF a, DF b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = __fmaf_rn(a.hi, b.hi, -p);
    return quick_two_sum(p, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e)));
}
__device__ __forceinline__ DF df_neg(DF a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ double df_value(DF a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ DF df_shfl_xor(DF a, int o)
{
    return {__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

// the six sums of a step: e2, e4, the potential (1 - phi^0 for the standard
// model), det, |F|^2 and the sextic density e6 (zero without the sextic
// term); plus max |F|^2
constexpr int kSums = 6;

// A thread's running sums between two flushes.  The energy and charge
// densities are added with Knuth's error-free two-sum, two quantities per
// packed instruction: s holds the FP32 sums of (e2, e4) and (e0, det), c the
// exact sums of the rounding errors of every addition into s (each error is
// itself exact, so s + c is the exact sum up to the rounding of the few
// additions into c).  The per-site sums therefore carry no FP32 reduction
// error into the energy of the arrest test or the baryon number.  |F|^2 is a
// plain FP32 sum (it feeds only the reported residual).
struct Acc {
    float2 s24, c24;  // (e2, e4) and their compensation
    float2 s0b, c0b;  // (e0, det) and their compensation
    float s6, c6;     // e6 and its compensation (the sextic kernels)
    float f2, fmax2;
};

// the same for one quantity
__device__ __forceinline__ void two_sum_acc1(float &s, float &c, float x)
{
    const float t = __fadd_rn(s, x);
    const float bb = __fsub_rn(t, s);
    c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(x, bb)));
    s = t;
}

// s + x with the rounding error of the addition added to c (two quantities)
__device__ __forceinline__ void two_sum_acc(float2 &s, float2 &c, float2 x)
{
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 t = __fadd2_rn(s, x);
    const float2 bb = __ffma2_rn(s, m1, t);                      // t - s
    const float2 ea = __ffma2_rn(__ffma2_rn(bb, m1, t), m1, s);  // s - (t - bb)
    const float2 eb = __ffma2_rn(bb, m1, x);                     // x - bb
    c = __fadd2_rn(c, __fadd2_rn(ea, eb));
    s = t;
}

// Fold a thread's running sums into its double-float sums, which live in
// shared memory (acc: kSums arrays of stride nthreads, at this thread's slot).
__device__ __forceinline__ void flush(DF *acc, float *amax, int nthreads, Acc &a)
{
    acc[0] = df_add(df_add(acc[0], a.s24.x), a.c24.x);
    acc[nthreads] = df_add(df_add(acc[nthreads], a.s24.y), a.c24.y);
    acc[2 * nthreads] = df_add(df_add(acc[2 * nthreads], a.s0b.x), a.c0b.x);
    acc[3 * nthreads] = df_add(df_add(acc[3 * nthreads], a.s0b.y), a.c0b.y);
    acc[4 * nthreads] = df_add(acc[4 * nthreads], a.f2);
    acc[5 * nthreads] = df_add(df_add(acc[5 * nthreads], a.s6), a.c6);
    *amax = fmaxf(*amax, a.fmax2);
    a = Acc{};
}

__device__ __forceinline__ void zero_sums(DF *acc, float *amax, int nthreads)
{
#pragma unroll
    for (int q = 0; q < kSums; ++q) acc[q * nthreads] = DF{0.f, 0.f};
    *amax = 0.f;
}
__device__ __forceinline__ void load_sums(const DF *acc, const float *amax, int nthreads,
                                          DF (&v)[kSums], float &m)
{
#pragma unroll
    for (int q = 0; q < kSums; ++q) v[q] = acc[q * nthreads];
    m = *amax;
}

// Block sum of the per-thread double-float sums (and max of amax) in a fixed
// shuffle order; thread 0 ends with the totals.  buf: kSums * NW DFs, amx: NW.
template <int NW, typename Sync>
__device__ __forceinline__ void block_reduce_df(DF (&v)[kSums], float amax, DF *buf, float *amx,
                                                DF (&tot)[kSums], float &tmax, int tid, Sync sync)
{
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int q = 0; q < kSums; ++q) v[q] = df_add(v[q], df_shfl_xor(v[q], o));
        amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    }
    sync();  // buf may still be read by an earlier reduction
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < kSums; ++q) buf[q * NW + warp] = v[q];
        amx[warp] = amax;
    }
    sync();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < kSums; ++q) v[q] = lane < NW ? buf[q * NW + lane] : DF{0.f, 0.f};
        amax = lane < NW ? amx[lane] : 0.f;
#pragma unroll
        for (int o = NW / 2; o > 0; o >>= 1) {
#pragma unroll
            for (int q = 0; q < kSums; ++q) v[q] = df_add(v[q], df_shfl_xor(v[q], o));
            amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        }
#pragma unroll
        for (int q = 0; q < kSums; ++q) tot[q] = v[q];
        tmax = amax;
    }
}

// Pairwise sum of x[0..K) into x[0] (K a power of two): a tree of depth log2 K
template <int K> __device__ __forceinline__ void df_tree(DF (&x)[K])
{
#pragma unroll
    for (int w = 1; w < K; w <<= 1) {
#pragma unroll
        for (int k = 0; k + w < K; k += 2 * w) x[k] = df_add(x[k], x[k + w]);
    }
}

// Block sum of the per-thread double-float sums kept in shared memory
// (accs: kSums arrays of NT, amaxs: NT) for CTAs of at least kSums + 1 warps:
// warp q sums quantity q, each lane its NT / 32 entries as a pairwise tree,
// then a butterfly; warp kSums takes the max.  Fixed order; thread 0 ends
// with the totals.  The caller has synchronised after the last write to accs.
template <int NT>
__device__ __forceinline__ void block_reduce_df_smem(const DF *accs, const float *amaxs, DF *red,
                                                     float *mred, DF (&tot)[kSums], float &tmax,
                                                     int tid)
{
    constexpr int K = NT / 32;
    static_assert(K > kSums && (K & (K - 1)) == 0, "one warp per quantity, a power-of-two tree");
    const int lane = tid & 31, warp = tid >> 5;
    if (warp < kSums) {
        const DF *a = accs + warp * NT + lane;
        DF x[K];
#pragma unroll
        for (int k = 0; k < K; ++k) x[k] = a[32 * k];
        df_tree<K>(x);
        DF v = x[0];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
        if (lane == 0) red[warp] = v;
    } else if (warp == kSums) {
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) m = fmaxf(m, amaxs[lane + 32 * k]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) *mred = m;
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < kSums; ++q) tot[q] = red[q];
        tmax = *mred;
    }
}

// Per-plane values of one column kept in the register x-ring.
struct PlaneVals {
    P4 phi, dy, dz;
};

template <int TY, int TZ, bool SEX = false> struct __align__(128) StepSmem {
    float4 plane[nslot<TY, TZ, SEX>()][TY + 4][TZ + 4];  // haloed field planes (TMA)
    float4 vpl[nslot<TY, TZ, SEX>()][TY][TZ];            // velocity planes of the centre sites (TMA)
    float4 dy[2][TY][TZ + 4];             // d_y phi exchange for d_yz
    int rel[nslot<TY, TZ, SEX>()];        // warps done with the plane in each slot
    DF accs[kSums][TY * TZ];              // per-thread double-float sums (kept out of registers)
    float amaxs[TY * TZ];                 // per-thread max |F|^2
    unsigned long long bar[nslot<TY, TZ, SEX>()];
    DF dfred[kSums * (TY * TZ / 32)];
    float mxred[TY * TZ / 32];
    int flag;
    int last;
    int fixv;                             // the decided correction (fused arrest fix-up)
    int cur_used;                         // ... the buffers the step read
    long long steps0;                     // ... and the step count before the step
    uint32_t tmem;                        // TMEM base address of the CTA's allocation
};

// Dynamic shared memory requested by a step CTA: its StepSmem, padded so
// that one CTA more than the SM's 512 TMEM columns can serve would need more
// than the SM's 228 KiB of shared memory, and so never becomes resident
// (tcgen05.alloc in that CTA would otherwise wait for a co-resident CTA to
// free its columns).
template <int TY, int TZ, bool SEX = false> constexpr size_t step_smem_bytes()
{
    constexpr size_t per_sm = 228 * 1024;
    constexpr int max_ctas = 512 / tmem_cols<TY * TZ / 32, SEX>();
    constexpr size_t floor_bytes = per_sm / (max_ctas + 1) + 1;  // max_ctas + 1 never fit
    return sizeof(StepSmem<TY, TZ, SEX>) > floor_bytes ? sizeof(StepSmem<TY, TZ, SEX>) : floor_bytes;
}

struct CtaSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// ------------------------------------------------- the plane pipeline
// Arrival of a haloed plane P: in-plane first and second y/z derivatives of
// the tile's centre column, d_y phi (each warp fills the z-halo of its own
// rows) into DY for the mixed d_yz of this plane.
template <int TY, int TZ>
__device__ __forceinline__ void arrive_plane(const float4 (*P)[TZ + 4], float4 (*DY)[TZ + 4],
                                             const InstDesc &D, int halo_off, int ty, int tz,
                                             PlaneVals &rv, P4 &dyy, P4 &dzz)
{
    const float2 w8 = kW8(), wm16 = kWm16(), w30 = kW30();
    const P4 c = ld4(P[ty + 2][tz + 2]);
    const P4 ym2 = ld4(P[ty][tz + 2]), ym1 = ld4(P[ty + 1][tz + 2]);
    const P4 yp1 = ld4(P[ty + 3][tz + 2]), yp2 = ld4(P[ty + 4][tz + 2]);
    const P4 zm2 = ld4(P[ty + 2][tz]), zm1 = ld4(P[ty + 2][tz + 1]);
    const P4 zp1 = ld4(P[ty + 2][tz + 3]), zp2 = ld4(P[ty + 2][tz + 4]);
    const P4 dy = fd1u(ym2, ym1, yp1, yp2, w8);
    const P4 dz = fd1u(zm2, zm1, zp1, zp2, w8);
    dyy = fd2n(ym2, ym1, c, yp1, yp2, wm16, w30);
    dzz = fd2n(zm2, zm1, c, zp1, zp2, wm16, w30);
    DY[ty][tz + 2] = st4(dy);
    {  // each warp fills the z-halo columns of u_y of its own rows, one
       // component per lane (a packed 4-vector stencil would idle 28 lanes);
       // the same roundings as fd1u
        // (halo_off: the lane's float offset in both arrays)
        constexpr int RS = 4 * (TZ + 4);  // floats per haloed row
        {
            const float *pc = reinterpret_cast<const float *>(P) + halo_off;
            const float m2 = pc[0], m1 = pc[RS], p1 = pc[3 * RS], p2 = pc[4 * RS];
            reinterpret_cast<float *>(DY)[halo_off] = __fmaf_rn(w8.x, __fsub_rn(p1, m1), __fsub_rn(m2, p2));
        }
    }
    rv.phi = c;
    rv.dy = dy;
    rv.dz = dz;
}

// In-plane values of a plane for its own centre two planes later: d_yz, the
// y/z parts of a_ij, of the Laplacian, of d_ij phi a_ij and of g_y, g_z.
template <int TY, int TZ, bool SEX = false>
__device__ __forceinline__ void plane_record(const float4 (*DY)[TZ + 4], const InstDesc &D, int ty,
                                             int tz, const PlaneVals &rv, const P4 &dyy,
                                             const P4 &dzz, uint32_t trec)
{
    constexpr int THREADS = TY * TZ;
    const P4 dy = rv.dy, dz = rv.dz;
    const P4 dyz = fd1(ld4(DY[ty][tz]), ld4(DY[ty][tz + 1]), ld4(DY[ty][tz + 3]), ld4(DY[ty][tz + 4]),
                       kXm1(), kXm2());
    const float ayy = dot(dy, dy), azz = dot(dz, dz), ayz = dot(dy, dz);
    const P4 lin = add(dyy, dzz);
    const P4 qin = fma(bc(2.f * ayz), dyz, fma(bc(azz), dzz, mul(bc(ayy), dyy)));
    const float gyv = hsum(dot2(dyz, dz, __ffma2_rn(dyy.b, dy.b, __fmul2_rn(dyy.a, dy.a))));
    const float gzv = hsum(dot2(dzz, dz, __ffma2_rn(dyz.b, dy.b, __fmul2_rn(dyz.a, dy.a))));
    // the centre needs a_yy, a_zz, a_yz only as a_yy + a_zz (in tr a) and
    // a_yy^2 + a_zz^2 + 2 a_yz^2 (in the quartic density)
    const float asum = ayy + azz;
    const float asq = fmaf(2.f * ayz, ayz, fmaf(azz, azz, ayy * ayy));
    // columns 0-7 lin, qin; 8-11 g_y, g_z, a_yy + a_zz, a_yy^2 + a_zz^2 + 2 a_yz^2
    const float r[12] = {lin.a.x, lin.a.y, lin.b.x, lin.b.y, qin.a.x, qin.a.y, qin.b.x, qin.b.y,
                         gyv, gzv, asum, asq};
    (void)THREADS;
    tmem_st8(trec, r);
    tmem_st4(trec + 8, r + 8);
    if constexpr (SEX) {
        // columns 16-27: N_yy, N_zz, N_yz
        const float r2[12] = {dyy.a.x, dyy.a.y, dyy.b.x, dyy.b.y, dzz.a.x, dzz.a.y, dzz.b.x, dzz.b.y,
                              dyz.a.x, dyz.a.y, dyz.b.x, dyz.b.y};
        tmem_st8(trec + 16, r2);
        tmem_st4(trec + 24, r2 + 8);
    }
}

// One centre site: x-derivatives from the register ring (M2, M1, C, Q1, Q2 in
// streaming order; xc1, xc2 are the mixed-derivative weights along x), the
// Euler-Lagrange force of Eq. (3.3) projected on the tangent space, the
// symplectic update with renormalisation, and the energy, charge and force
// densities into a32 (valid sites only).
template <int TY, int TZ, bool POT = false, bool DUMP = false, bool SEX = false>
__device__ __forceinline__ void centre_site(const InstDesc &D, const PlaneVals &M2,
                                            const PlaneVals &M1, const PlaneVals &C,
                                            const PlaneVals &Q1, const PlaneVals &Q2, float2 xc1,
                                            float2 xc2, uint32_t trec, uint4 tdz,
                                            const float4 *vp,
                                            bool use_v, bool valid, float4 *phiout, float4 *vout,
                                            size_t si, Acc &a32)
{
    constexpr int THREADS = TY * TZ;
    const int mode = D.mode;
    const float2 dt = D.dt, dt2 = D.dt2;
    float rv[12];
    tmem_wait_st();  // this thread's earlier record stores have landed
    tmem_ld8(trec, rv);
    tmem_ld4(trec + 8, rv + 8);
    // the sextic variant's d_z phi of M2, M1, C, Q1 (tdz: their columns)
    float zv[16];
    if constexpr (SEX) {
        tmem_ld4(tdz.x, zv);
        tmem_ld4(tdz.y, zv + 4);
        tmem_ld4(tdz.z, zv + 8);
        tmem_ld4(tdz.w, zv + 12);
    }
    tmem_wait_ld12(rv);
    if constexpr (SEX) tmem_wait_ld16(zv);
    auto zp4 = [&](int i) -> P4 {
        return {make_float2(zv[4 * i], zv[4 * i + 1]), make_float2(zv[4 * i + 2], zv[4 * i + 3])};
    };
    const P4 zM2 = SEX ? zp4(0) : M2.dz, zM1 = SEX ? zp4(1) : M1.dz;
    const P4 zC = SEX ? zp4(2) : C.dz, zQ1 = SEX ? zp4(3) : Q1.dz;

    const P4 lin = {make_float2(rv[0], rv[1]), make_float2(rv[2], rv[3])};
    const P4 qin = {make_float2(rv[4], rv[5]), make_float2(rv[6], rv[7])};
    const float Cgy = rv[8], Cgz = rv[9], Casum = rv[10], Casq = rv[11];
    (void)THREADS;
    const P4 ph = C.phi;
    // u_x and the negated second derivatives N_xx, N_xy, N_xz (the scales
    // are those of the descriptor's stencil weights)
    const P4 dx = fd1u(M2.phi, M1.phi, Q1.phi, Q2.phi, kW8());
    const P4 dxx = fd2n(M2.phi, M1.phi, ph, Q1.phi, Q2.phi, kWm16(), kW30());
    // the mixed derivatives along x: the sextic variant takes them on the
    // N scale (weights xc1, xc2); the others as the first-derivative
    // stencil of the u_i, M_xi = 144h^2 d_xi phi = -12 N_xi, with the
    // factor kS = -1/12 applied where they enter
    constexpr float kS = SEX ? 1.f : -1.f / 12.f;
    const P4 dxy = SEX ? fd1(M2.dy, M1.dy, Q1.dy, Q2.dy, xc1, xc2) : fd1u(M2.dy, M1.dy, Q1.dy, Q2.dy, kW8());
    const P4 dxz = SEX ? fd1(zM2, zM1, zQ1, Q2.dz, xc1, xc2) : fd1u(zM2, zM1, zQ1, Q2.dz, kW8());
    const P4 dyc = C.dy, dzc = zC;
    const float axx = dot(dx, dx), axy = dot(dx, dyc), axz = dot(dx, dzc);
    const float tra = axx + Casum;
    const P4 L = add(dxx, lin);  // -12h^2 Laplacian phi
    // g_i = sum_j d_ij phi.d_j phi and c_i = g_i - Laplacian.d_i phi, both
    // negated; nc_i = -c_i
    float gx;
    if constexpr (SEX) {
        gx = hsum(dot2(dxz, dzc, dot2(dxy, dyc, __ffma2_rn(dxx.b, dx.b, __fmul2_rn(dxx.a, dx.a)))));
    } else {
        const float2 gxm = dot2(dxz, dzc, __ffma2_rn(dxy.b, dyc.b, __fmul2_rn(dxy.a, dyc.a)));
        gx = hsum(__ffma2_rn(bc(kS), gxm, __ffma2_rn(dxx.b, dx.b, __fmul2_rn(dxx.a, dx.a))));
    }
    const float gy = fmaf(kS, dot(dxy, dx), Cgy);
    const float gz = fmaf(kS, dot(dxz, dx), Cgz);
    const float ncx = dot(L, dx) - gx, ncy = dot(L, dyc) - gy, ncz = dot(L, dzc) - gz;
    // -d_ij phi a_ij summed over i, j
    const P4 Ha = fma(bc(2.f * kS * axz), dxz, fma(bc(2.f * kS * axy), dxy, fma(bc(axx), dxx, qin)));
    // brace of the Euler-Lagrange equation / B; G = -2 B (brace + m^2 e_0 / B)
    P4 br = fma(bc(ncz), dzc, fma(bc(ncy), dyc, fma(bc(ncx), dx, fma(bc(D.negK - tra), L, Ha))));
    br.a.x += D.bm2;
    // 1 - phi^0 from the pion components where it cancels (phi^0 >= 0)
    auto one_minus_phi0 = [&]() {
        const float2 pq = __fmul2_rn(ph.b, ph.b);
        const float pi2 = fmaf(ph.a.y, ph.a.y, pq.x + pq.y);
        return ph.a.x >= 0.f ? pi2 * rcp_approx(1.f + ph.a.x) : 1.f - ph.a.x;
    };
    float u = 0.f;
    if constexpr (POT) {
        // d/dphi^0 of the Section 7.8 potentials m_y^2 (1 - phi0^2) + m_z^2 u^2
        // + m_w^2 u^4 / 2, u = 1 - phi^0, in the brace (G = -2 brace)
        u = one_minus_phi0();
        br.a.x += fmaf(D.bmy2, ph.a.x, u * fmaf(D.bmw2 * u, u, D.bmz2));
    }
    // det[phi, d_x phi, d_y phi, d_z phi] by the 2x2 minors s_AB of rows
    // (phi, d_x) and c_AB of rows (d_y, d_z): {q_s0, s12, s34, q_s5} =
    // {s01, (s02, s03), (s12, s13), s23}, {q0, q12, q34, q5} likewise for c
    const float q_s0 = ph.a.x * dx.a.y - dx.a.x * ph.a.y;
    const float2 s12 = __ffma2_rn(bc(-dx.a.x), ph.b, __fmul2_rn(bc(ph.a.x), dx.b));
    const float2 s34 = __ffma2_rn(bc(-dx.a.y), ph.b, __fmul2_rn(bc(ph.a.y), dx.b));
    const float q_s5 = ph.b.x * dx.b.y - dx.b.x * ph.b.y;
    const float q0 = dyc.a.x * dzc.a.y - dzc.a.x * dyc.a.y;
    const float2 q12 = __ffma2_rn(bc(-dzc.a.x), dyc.b, __fmul2_rn(bc(dyc.a.x), dzc.b));
    const float2 q34 = __ffma2_rn(bc(-dzc.a.y), dyc.b, __fmul2_rn(bc(dyc.a.y), dzc.b));
    const float q5 = dyc.b.x * dzc.b.y - dzc.b.x * dyc.b.y;
    const float det = q_s0 * q5 - s12.x * q34.y + s12.y * q34.x + s34.x * q12.y - s34.y * q12.x + q_s5 * q0;
    float e6 = 0.f;
    if constexpr (SEX) {
        // Section 7.8 sextic term c6 D^2, D = det[phi, d_x phi, d_y phi, d_z phi]
        // (= c6 4 pi^4 (B0)^2): its Euler-Lagrange gradient is
        // 2 c6 [4 D P - sum_i (d_i D) Q_i] with P = dD/dphi, Q_i = dD/d(d_i phi)
        // and d_i D = sum_j Q_j . d_i d_j phi; in the brace (G = -2 brace) it
        // enters as -c6 [...].  From the u_i and N_ij (D, P, Q, d_i D carry
        // (12h)^-3, ^-3, ^-2 and -(12h)^-2 (12h^2)^-1) the bracket is
        // (12h)^-4 (12h^2)^-1 [D P / 3 + sum_i dDn_i Q_i], which enters the
        // brace / B with the weight -c6 / (144 h^2).
        float rs[12];  // N_yy, N_zz, N_yz of the centre plane
        tmem_ld8(trec + 16, rs);
        tmem_ld4(trec + 24, rs + 8);
        tmem_wait_ld12(rs);
        // the cofactor rows of M = [phi; u; v; w] (rows): P = dD/dphi and
        // q_i = dD/d(u_i), each a sum of three products of an entry of the
        // other row of its pair with the minors of the opposite pair
        const float s01 = q_s0, s02 = s12.x, s03 = s12.y, s12v = s34.x, s13 = s34.y, s23 = q_s5;
        const float c01 = q0, c02 = q12.x, c03 = q12.y, c12 = q34.x, c13 = q34.y, c23 = q5;
        const float u0 = dx.a.x, u1 = dx.a.y, u2 = dx.b.x, u3 = dx.b.y;
        const float p0 = ph.a.x, p1 = ph.a.y, p2 = ph.b.x, p3 = ph.b.y;
        const float v0 = dyc.a.x, v1 = dyc.a.y, v2 = dyc.b.x, v3 = dyc.b.y;
        const float w0 = dzc.a.x, w1 = dzc.a.y, w2 = dzc.b.x, w3 = dzc.b.y;
        const P4 pp = {make_float2(fmaf(u3, c12, fmaf(-u2, c13, u1 * c23)),
                                   fmaf(-u3, c02, fmaf(u2, c03, -u0 * c23))),
                       make_float2(fmaf(u3, c01, fmaf(-u1, c03, u0 * c13)),
                                   fmaf(-u2, c01, fmaf(u1, c02, -u0 * c12)))};
        const P4 qx = {make_float2(fmaf(-p3, c12, fmaf(p2, c13, -p1 * c23)),
                                   fmaf(p3, c02, fmaf(-p2, c03, p0 * c23))),
                       make_float2(fmaf(-p3, c01, fmaf(p1, c03, -p0 * c13)),
                                   fmaf(p2, c01, fmaf(-p1, c02, p0 * c12)))};
        const P4 qy = {make_float2(fmaf(w3, s12v, fmaf(-w2, s13, w1 * s23)),
                                   fmaf(-w3, s02, fmaf(w2, s03, -w0 * s23))),
                       make_float2(fmaf(w3, s01, fmaf(-w1, s03, w0 * s13)),
                                   fmaf(-w2, s01, fmaf(w1, s02, -w0 * s12v)))};
        const P4 qz = {make_float2(fmaf(-v3, s12v, fmaf(v2, s13, -v1 * s23)),
                                   fmaf(v3, s02, fmaf(-v2, s03, v0 * s23))),
                       make_float2(fmaf(-v3, s01, fmaf(v1, s03, -v0 * s13)),
                                   fmaf(v2, s01, fmaf(-v1, s02, v0 * s12v)))};
        const float Dd = det;
        const P4 dyy = {make_float2(rs[0], rs[1]), make_float2(rs[2], rs[3])};
        const P4 dzz = {make_float2(rs[4], rs[5]), make_float2(rs[6], rs[7])};
        const P4 dyz = {make_float2(rs[8], rs[9]), make_float2(rs[10], rs[11])};
        const float dDx = hsum(dot2(qz, dxz, dot2(qy, dxy, __ffma2_rn(qx.b, dxx.b, __fmul2_rn(qx.a, dxx.a)))));
        const float dDy = hsum(dot2(qz, dyz, dot2(qy, dyy, __ffma2_rn(qx.b, dxy.b, __fmul2_rn(qx.a, dxy.a)))));
        const float dDz = hsum(dot2(qz, dzz, dot2(qy, dyz, __ffma2_rn(qx.b, dxz.b, __fmul2_rn(qx.a, dxz.a)))));
        const P4 sx = fma(bc(dDz), qz, fma(bc(dDy), qy, fma(bc(dDx), qx, mul(bc(Dd * (1.f / 3.f)), pp))));
        br = fma(bc(-D.c6b), sx, br);
        e6 = D.c6 * Dd * Dd;
    }

    // F = -G + (G.phi) phi = 2 B (br - (br.phi) phi); dt2 = 2 dt B
    const float bp = dot(br, ph);
    const P4 Fh = fma(bc(-bp), ph, br);
    const float f2 = 4.f * dot(Fh, Fh);
    P4 t, vnew;
    if (mode == MODE_GRADIENT) {
        t = fma(dt2, Fh, ph);
    } else {
        const P4 vo = use_v ? ld4(*vp) : P4{bc(0.f), bc(0.f)};
        vnew = fma(dt2, Fh, vo);
        t = fma(dt, vnew, ph);
    }
    const float r = rsqrtf(dot(t, t));
    const P4 pn = mul(bc(r), t);
    const float sq = fmaf(axx, axx, Casq) + 2.f * fmaf(axy, axy, axz * axz);
    const float e4 = 0.5f * (tra * tra - sq);
    if (valid) {
        __stcs(phiout + si, st4(pn));
        if (mode != MODE_GRADIENT) __stcs(vout + si, st4(vnew));
        float e0v;
        if constexpr (POT) {
            // the whole potential: 2 m^2 u + m_y^2 u (2 - u) + m_z^2 u^2 + m_w^2 u^4 / 2
            const float u2 = u * u;
            e0v = fmaf(2.f * D.m2, u, fmaf(D.my2, u * (2.f - u), u2 * fmaf(0.5f * D.mw2, u2, D.mz2)));
        } else {
            e0v = one_minus_phi0();
        }
        if constexpr (DUMP) {
            // the densities in lattice units; the sums take the same values
            const float e2s = tra * D.dk2, e4s = e4 * D.dk4, dets = det * D.dk3;
            __stcs(D.dump + si, make_float4(e2s, e4s, e0v, dets));
            two_sum_acc(a32.s24, a32.c24, make_float2(e2s, e4s));
            two_sum_acc(a32.s0b, a32.c0b, make_float2(e0v, dets));
        } else {
            two_sum_acc(a32.s24, a32.c24, make_float2(tra, e4));
            two_sum_acc(a32.s0b, a32.c0b, make_float2(e0v, det));
        }
        if constexpr (SEX) two_sum_acc1(a32.s6, a32.c6, e6);
        a32.f2 += f2;
        a32.fmax2 = fmaxf(a32.fmax2, f2);
    }
}

// One site of the correction of a mispredicted arrest decision:
// v = v_new + sgn v_old, phi = normalise(phi_old + dt v).  Every operation is
// rounded explicitly, so that every path that corrects a site (the fix-up
// kernels, the step's own correction, an x-slab's fix-up) gives the same bits.
__device__ __forceinline__ void arrest_fix_site(const float4 &vn, const float4 &vo,
                                                const float4 &fo, float sgn, float dt, float4 &v,
                                                float4 &p)
{
    v = make_float4(__fmaf_rn(sgn, vo.x, vn.x), __fmaf_rn(sgn, vo.y, vn.y),
                    __fmaf_rn(sgn, vo.z, vn.z), __fmaf_rn(sgn, vo.w, vn.w));
    const float4 t = make_float4(__fmaf_rn(dt, v.x, fo.x), __fmaf_rn(dt, v.y, fo.y),
                                 __fmaf_rn(dt, v.z, fo.z), __fmaf_rn(dt, v.w, fo.w));
    const float r =
        rsqrtf(__fmaf_rn(t.w, t.w, __fmaf_rn(t.z, t.z, __fmaf_rn(t.y, t.y, __fmul_rn(t.x, t.x)))));
    p = make_float4(__fmul_rn(t.x, r), __fmul_rn(t.y, r), __fmul_rn(t.z, r), __fmul_rn(t.w, r));
}

__device__ __forceinline__ void write_record(const InstDesc &D, int slot, const DF (&tot)[kSums], float tmax)
{
    float4 *recp = reinterpret_cast<float4 *>(D.parts + (size_t)slot * kPartialDoubles);
    recp[0] = make_float4(tot[0].hi, tot[0].lo, tot[1].hi, tot[1].lo);
    recp[1] = make_float4(tot[2].hi, tot[2].lo, tot[3].hi, tot[3].lo);
    recp[2] = make_float4(tot[4].hi, tot[4].lo, tmax, 0.f);
    recp[3] = make_float4(tot[5].hi, tot[5].lo, 0.f, 0.f);
}

__device__ __forceinline__ void st_release_s64(long long *p, long long v)
{
    asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// Arrival at a lattice's counter: releases this thread's earlier stores (the
// CTA record) and acquires every earlier arrival's
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned *p, unsigned v)
{
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// End of a step for one lattice, run by every thread of the last CTA to
// leave it.  The CTA records {e2, e4, 1 - phi^0, det, |F|^2} (as hi, lo float
// pairs) and max |F|^2 are summed in a fixed order.  Thread 0 then forms the
// energy of Eq. (2.4), applies the arrest rule of Section 4 in FP64
// (E_n > E_{n-1}: the velocity is zeroed), scores the prediction the launch
// ran with, updates the two-level predictor (the last four decisions select a
// 2-bit saturating counter) and publishes the step; meanwhile thread 32 forms
// the reported energies, the charge of Eq. (2.6), the virial and the force
// norms, which nothing in the launch waits for.
template <int NW, typename Sync>
__device__ __forceinline__ void finish_lattice(const InstDesc &D, Ctrl *c, int cur, int mode,
                                               int pred, int dry, DF *buf, float *amx, int tid,
                                               Sync sync)
{
    // thread 0 fetches the control fields it needs while the block sums the records
    double E_prev = 0.0;
    int hist = 0;
    uint4 pht4 = make_uint4(0u, 0u, 0u, 0u);
    long long steps = 0, arrests = 0, fixups = 0;
    if (tid == 0 && !dry) {
        E_prev = __ldcg(&c->E_prev);
        hist = __ldcg(&c->hist);
        pht4 = __ldcg(reinterpret_cast<const uint4 *>(c->pht));
        steps = __ldcg(&c->steps);
        arrests = __ldcg(&c->arrests);
        fixups = __ldcg(&c->fixups);
    }
    DF t[kSums];
    float tmax = 0.f;
    if constexpr (NW > kSums) {
        // warp q sums quantity q of every record straight from global memory
        // (eight independent loads per lane and pass, a pairwise tree, then a
        // butterfly); warp kSums takes the max
        const int lane = tid & 31, warp = tid >> 5;
        // float offsets in a record: e2 0, e4 2, e0 4, det 6, |F|^2 8, e6 12; max 10
        const int off = warp < 5 ? 2 * warp : (warp == 5 ? 12 : 10);
        const float *base = reinterpret_cast<const float *>(D.parts) + off;
        constexpr int kRec = 2 * kPartialDoubles;                 // floats per record
        if (warp < kSums) {
            DF acc = {0.f, 0.f};
            for (int i0 = 0; i0 < D.cta_count; i0 += 256) {
                DF x[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int i = i0 + lane + 32 * k;
                    float2 r = make_float2(0.f, 0.f);
                    if (i < D.cta_count)
                        r = __ldcg(reinterpret_cast<const float2 *>(base + (size_t)i * kRec));
                    x[k] = DF{r.x, r.y};
                }
                df_tree<8>(x);
                acc = df_add(acc, x[0]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc = df_add(acc, df_shfl_xor(acc, o));
            if (lane == 0) buf[warp] = acc;
        } else if (warp == kSums) {
            float m = 0.f;
            for (int i = lane; i < D.cta_count; i += 32)
                m = fmaxf(m, __ldcg(base + (size_t)i * kRec));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0) *amx = m;
        }
        sync();
        if (tid != 0 && tid != 32) return;
#pragma unroll
        for (int q = 0; q < kSums; ++q) t[q] = buf[q];
        tmax = *amx;
    } else {
        DF v[kSums] = {};
        float amax = 0.f;
        for (int i = tid; i < D.cta_count; i += NW * 32) {
            const float4 *r = reinterpret_cast<const float4 *>(D.parts + (size_t)i * kPartialDoubles);
            const float4 a = __ldcg(r), b = __ldcg(r + 1), e = __ldcg(r + 2), f = __ldcg(r + 3);
            v[0] = df_add(v[0], DF{a.x, a.y});
            v[1] = df_add(v[1], DF{a.z, a.w});
            v[2] = df_add(v[2], DF{b.x, b.y});
            v[3] = df_add(v[3], DF{b.z, b.w});
            v[4] = df_add(v[4], DF{e.x, e.y});
            v[5] = df_add(v[5], DF{f.x, f.y});
            amax = fmaxf(amax, e.z);
        }
        block_reduce_df<NW>(v, amax, buf, amx, t, tmax, tid, sync);
        if (tid != 0) return;
    }
    const bool reporter = NW > kSums ? tid == 32 : tid == 0;
    const bool decider = tid == 0;
    if (dry) {
        if (decider) c->done = 0;
        return;
    }
    // the sums in lattice units (the step sums unscaled densities)
    t[0] = df_mul(DF{D.s_e2.x, D.s_e2.y}, t[0]);
    t[1] = df_mul(DF{D.s_e4.x, D.s_e4.y}, t[1]);
    t[3] = df_mul(DF{D.s_b.x, D.s_b.y}, t[3]);
    t[4] = df_mul(DF{D.s_f.x, D.s_f.y}, t[4]);
    t[5] = df_mul(DF{D.s_e6.x, D.s_e6.y}, t[5]);
    const double fmax2 = (double)tmax * ((double)D.s_f.x + (double)D.s_f.y);
    constexpr double kB = -0.050660591821168885;  // b = -det / (2 pi^2)
    const DF bfac = {(float)kB, (float)(kB - (double)(float)kB)};
    if (D.slab_rec) {
        // one x-slab of a larger lattice: leave this slab's record for the
        // decision over all slabs, {e2, e4, e0, b, |F|^2, max |F|^2, sites, e6}
        if (!decider) return;
        double *r = D.slab_rec;
        r[0] = df_value(t[0]);
        r[1] = df_value(t[1]);
        r[2] = df_value(df_mul(DF{D.e0_scale, 0.f}, t[2]));
        r[3] = df_value(df_mul(bfac, t[3]));
        r[4] = df_value(t[4]);
        r[5] = fmax2;
        r[6] = (double)(D.n0 - 4) * (double)(D.n1 - 4) * (double)(D.n2 - 4);
        r[7] = df_value(t[5]);
        c->done = 0;
        return;
    }
    const DF h3 = {D.h3_hi, D.h3_lo};
    const DF E2 = df_mul(h3, t[0]), E4 = df_mul(h3, t[1]);
    const DF E0 = df_mul(h3, df_mul(DF{D.e0_scale, 0.f}, t[2]));  // 2 m^2 sum(1 - phi^0), or the potentials' sum
    const DF E6 = df_mul(h3, t[5]);  // the sextic term (zero without it)
    const DF E = df_add(df_add(df_add(E2, E4), E0), E6);
    const double Ed = df_value(E);
    if (decider) {
        const int actual = (mode == MODE_ARRESTED && Ed > E_prev) ? 1 : 0;
        const int fix = (actual == pred) ? 0 : (actual ? -1 : +1);
        // counter i of the 16 is byte i of pht4 (read by shifts, no local copy)
        auto counter = [&](int i) {
            const unsigned w = i < 8 ? (i < 4 ? pht4.x : pht4.y) : (i < 12 ? pht4.z : pht4.w);
            return (int)((w >> (8 * (i & 3))) & 0xffu);
        };
        const int h = hist & 15;
        int ctr = counter(h);
        ctr = actual ? (ctr < 3 ? ctr + 1 : 3) : (ctr > 0 ? ctr - 1 : 0);
        const int hn = ((h << 1) | actual) & 15;
        c->pht[h] = (unsigned char)ctr;
        c->hist = hn;
        c->pred = (h == hn ? ctr : counter(hn)) >= 2 ? 1 : 0;
        c->fix = fix;
        c->arrests = arrests + actual;
        c->fixups = fixups + (fix != 0);
        c->E_prev = Ed;
        c->cur = cur ^ 1;
        c->done = 0;
        // the step count goes last, released: CTAs that correct their own
        // sites wait for it, and then see every field above
        st_release_s64(&c->steps, steps + 1);
    }
    if (reporter) {
        const DF B = df_mul(h3, df_mul(bfac, t[3]));
        // Derrick scaling: -E2 + E4 - 3 E0 + 3 E6
        const DF V = df_add(df_add(df_add(df_neg(E2), E4), df_mul(DF{-3.f, 0.f}, E0)),
                            df_mul(DF{3.f, 0.f}, E6));
        const double nsites = (double)(D.n0 - 4) * (double)(D.n1 - 4) * (double)(D.n2 - 4);
        c->last[0] = Ed;
        c->last[1] = df_value(E2);
        c->last[2] = df_value(E4);
        c->last[3] = df_value(E0);
        c->last[4] = df_value(B);
        c->last[5] = df_value(V);
        c->last[6] = sqrt(fmax2);
        c->last[7] = sqrt(df_value(t[4]) / nsites);
        c->e6_last = df_value(E6);
        if (!(isfinite(Ed) && isfinite(B.hi) && isfinite(t[4].hi))) c->status = DEV_NONFINITE;
    }
}

__device__ __forceinline__ long long ld_acquire_s64(const long long *p)
{
    long long v;
    asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// The step's own correction of a mispredicted arrest decision, at the sites
// this CTA updated (units [u0, u1) of the single lattice D, whose step read
// buffers `cur`): v = v' + fix v_old, phi = normalise(phi_old + dt v) by
// arrest_fix_site.  Each thread corrects the very sites it wrote, four planes
// of loads in flight at a time.
// (Its unit arithmetic is 32-bit: a 64-bit division here made the compiler
// spill the main loop's registers.)
template <int TY, int TZ>
__device__ __forceinline__ void correct_own_sites(const InstDesc &D, const CtaSplit &sp,
                                                  long long u0, long long u1,
                                                  int cur, int fix, int ty, int tz)
{
    // buffers selected by value, not by a run-time index into the parameter
    const float4 *__restrict__ vo_p = cur ? D.vel[1] : D.vel[0];
    const float4 *__restrict__ fo_p = cur ? D.phi[1] : D.phi[0];
    float4 *__restrict__ vn_p = cur ? D.vel[0] : D.vel[1];
    float4 *__restrict__ fn_p = cur ? D.phi[0] : D.phi[1];
    const size_t ps = (size_t)D.n1 * D.n2;
    const float sgn = (float)fix, dt = D.dt.x;
    // a single lattice's units (columns x interior planes) fit in an int
    const int nix = D.nix, nzt = D.nzt, w1 = (int)(u1 - D.unit_start);
    for (int us = (int)(u0 - D.unit_start); us < w1;) {
        int col, xs, xe;
        if (sp.n == -2) {
            int xl, len;
            lock_run(sp, blockIdx.x, nix, us, w1, col, xl, len);
            xs = 2 + xl;
            xe = xs + len;
            us += len;
        } else {
            col = us / nix;
            const int ue = min(w1, (col + 1) * nix);
            xs = 2 + (us - col * nix);
            xe = 2 + (ue - col * nix);
            us = ue;
        }
        const int y = 2 + (col / nzt) * TY + ty, z = 2 + (col % nzt) * TZ + tz;
        if (y > D.n1 - 3 || z > D.n2 - 3) continue;
        size_t si = (size_t)xs * ps + (size_t)y * D.n2 + z;
        int x = xs;
        for (; x + 4 <= xe; x += 4, si += 4 * ps) {
            float4 vn[4], vo[4], fo[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                vn[k] = __ldcg(vn_p + si + k * ps);
                vo[k] = __ldcs(vo_p + si + k * ps);
                fo[k] = __ldcs(fo_p + si + k * ps);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float4 v, p;
                arrest_fix_site(vn[k], vo[k], fo[k], sgn, dt, v, p);
                vn_p[si + k * ps] = v;
                fn_p[si + k * ps] = p;
            }
        }
        for (; x < xe; ++x, si += ps) {
            float4 v, p;
            arrest_fix_site(__ldcg(vn_p + si), __ldcs(vo_p + si), __ldcs(fo_p + si), sgn, dt, v, p);
            vn_p[si] = v;
            fn_p[si] = p;
        }
    }
}

// The step for every lattice of the launch, two CTAs per SM.  BATCHED:
// lattices come from `table` (ninst entries, ordered by unit_start); otherwise
// from `one`.  dry != 0 (autotuning): outputs land in the inactive buffers and
// the control blocks are left as they were.
template <int TY, int TZ, bool BATCHED, bool POT = false, bool DUMP = false, bool SEX = false>
__global__ void __launch_bounds__(TY *TZ, 512 / (TY * TZ))
    k_step_f32(const __grid_constant__ InstDesc one, const __grid_constant__ CtaSplit split,
               const InstDesc *__restrict__ table, int ninst, long long total_units, int dry)
{
    constexpr int THREADS = TY * TZ;
    constexpr int NSLOT = nslot<TY, TZ, SEX>();
    constexpr unsigned PLANE_BYTES = (TY + 4) * (TZ + 4) * 16;
    constexpr unsigned VPLANE_BYTES = TY * TZ * 16;
    using Smem = StepSmem<TY, TZ, SEX>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    const int tid = threadIdx.x;
    const int ty = tid / TZ, tz = tid % TZ;
    // the d_y halo column this lane fills in every plane: one component of
    // the two z-halo columns at each end of the warp's rows (16 lanes per row)
    int halo_off;
    {
        constexpr int ROWS = 32 / TZ;
        const int lane = (tid & 31) % (16 * ROWS);  // the spare lanes repeat the first ones
        const int hr = (tid >> 5) * ROWS + (lane >> 4), ci = (lane >> 2) & 3, k = lane & 3;
        const int hc = ci < 2 ? ci : TZ + ci;
        halo_off = 4 * (hr * (TZ + 4) + hc) + k;
    }
    // a single lattice's next step may start its prologue as soon as an SM
    // frees up (its grid-dependency wait below keeps it off this step's data)
    if constexpr (!BATCHED) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    int cur0 = 0, pred0 = 0;

    if (tid == 0) {
        for (int s = 0; s < NSLOT; ++s) {
            mbar_init(&sm.bar[s], 1);
            sm.rel[s] = 0;
        }
        mbar_fence_init();
        sm.flag = 0;
    }
    constexpr uint32_t TCOLS = tmem_cols<THREADS / 32, SEX>();
    constexpr int RECC = rec_cols<SEX>();
    if (tid < 32) tmem_alloc(&sm.tmem, TCOLS);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if constexpr (!BATCHED) {
        // the previous launch (its field, velocity and control block) is
        // complete and visible from here on
        asm volatile("griddepcontrol.wait;" ::: "memory");
        cur0 = __ldcg(&one.ctrl->cur);
        pred0 = one.mode == MODE_ARRESTED ? __ldcg(&one.ctrl->pred) : 0;
        // the step count before this step, for the fused correction (kept in
        // shared memory, out of the main loop's registers)
        if (one.fuse_fix && tid == 0) sm.steps0 = __ldcg(&one.ctrl->steps);
    }
    const uint32_t twarp = sm.tmem + ((uint32_t)(32 * ((tid >> 5) & 3)) << 16) +
                           (uint32_t)(tmem_cols_per_warp<SEX>() * ((tid >> 5) >> 2));

    // unit ranges: a single lattice's listed in the parameter; a batch's,
    // when balanced (split.n < 0), in device memory right after its table;
    // else the even split
    const bool listed = !BATCHED && split.n > 0;
    const int *bstart = reinterpret_cast<const int *>(table + ninst);
    const bool blisted = BATCHED && split.n < 0;
    const bool locked = !BATCHED && split.n == -2;
    const long long u0 = locked ? 0
                         : listed ? split.start[blockIdx.x]
                         : blisted ? bstart[blockIdx.x]
                                   : total_units * blockIdx.x / gridDim.x;
    const long long u1 = locked ? lock_units(split, blockIdx.x, one.nix)
                         : listed ? split.start[blockIdx.x + 1]
                         : blisted ? bstart[blockIdx.x + 1]
                                   : total_units * (blockIdx.x + 1) / gridDim.x;
    int inst = 0;
    if (BATCHED)
        while (inst + 1 < ninst && table[inst + 1].unit_start <= u0) ++inst;
    uint32_t g = 0;   // planes consumed by this CTA (ring sequence number)
    uint32_t g3 = 0;  // g % 3, the in-plane record slot of plane g
    bool failed = false;

    for (long long us = u0; us < u1 && !failed; ++inst) {
        // for a single lattice D names the kernel parameter itself, so its
        // fields stay constant-bank operands instead of occupying registers
        const InstDesc &D = BATCHED ? table[inst] : one;
        const long long seg_hi = min(u1, D.unit_start + D.units);
        Ctrl *ctrl = D.ctrl;
        const int cur = BATCHED ? __ldcg(&ctrl->cur) : cur0;
        if (!BATCHED && tid == 0) sm.cur_used = cur;
        const int pred = BATCHED ? ((D.mode == MODE_ARRESTED) ? __ldcg(&ctrl->pred) : 0) : pred0;
        const CUtensorMap *map = &D.map[cur];
        const CUtensorMap *vmap = &D.vmap[cur];
        float4 *__restrict__ phiout = D.phi[cur ^ 1];
        float4 *__restrict__ vout = D.vel[cur ^ 1];
        const int mode = D.mode;
        const bool use_v = (mode != MODE_GRADIENT) && !pred;
        const int nix = D.nix, nzt = D.nzt, n1 = D.n1, n2 = D.n2;
        const size_t plane_stride = (size_t)n1 * n2;
        DF *acc = &sm.accs[0][tid];
        float *amax = &sm.amaxs[tid];
        zero_sums(acc, amax, THREADS);
        Acc a32 = {};

        while (us < seg_hi && !failed) {
            long long col;
            int xs, xe;  // xe exclusive
            if (locked) {
                int c, xl, len;
                lock_run(split, blockIdx.x, nix, (int)us, (int)seg_hi, c, xl, len);
                col = c;
                xs = 2 + xl;
                xe = xs + len;
                us += len;
            } else {
                const long long local = us - D.unit_start;
                col = local / nix;
                const long long ue = min(seg_hi, D.unit_start + (col + 1) * (long long)nix);
                xs = 2 + (int)(local - col * nix);
                xe = 2 + (int)(ue - D.unit_start - col * nix);
                us = ue;
            }
            const int y0 = 2 + (int)(col / nzt) * TY, z0 = 2 + (int)(col % nzt) * TZ;
            const int y = y0 + ty, z = z0 + tz;
            const bool valid = (y <= n1 - 3) && (z <= n2 - 3);
            const size_t col_off = (size_t)y * n2 + z;
            const int pf = xs - 2, pl = xe + 1;  // planes needed by this run
            // plane q travels with the velocity of centre q - 2 (when that is a centre)
            auto issue = [&](int q, int slot) {
                const bool wv = use_v && q - 2 >= xs && q - 2 < xe;
                mbar_expect_tx(&sm.bar[slot], PLANE_BYTES + (wv ? VPLANE_BYTES : 0u));
                tma_plane(&sm.plane[slot][0][0], map, &sm.bar[slot], 4 * (z0 - 2), y0 - 2, q);
                if (wv) tma_plane(&sm.vpl[slot][0][0], vmap, &sm.bar[slot], 4 * z0, y0, q - 2);
            };
            if (tid == 0) {
                // the slots were last read through the generic proxy (the run
                // before this one, ordered by the closing barrier): order those
                // reads before the copies' async-proxy writes
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                for (int q = 0; q < NSLOT && pf + q <= pl; ++q) issue(pf + q, (g + q) % NSLOT);
            }
            PlaneVals ring[5];
            int nouter = 0;
            size_t si = (size_t)(pf - 2) * plane_stride + col_off;  // of the centre x = pp - 2
            for (int base = pf; base <= pl && !failed; base += 5) {
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    const int pp = base + k;
                    if (pp > pl) break;
                    const int s = g % NSLOT;
                    const uint32_t par = (g / NSLOT) & 1u;
                    // a copy that never lands fails the step; the waits of the
                    // group of five that follow give up at once
                    if (!mbar_wait_flag(&sm.bar[s], par, &sm.flag)) sm.flag = 1;
                    float4(*DY)[TZ + 4] = sm.dy[g & 1];
                    P4 dyy, dzz;
                    arrive_plane<TY, TZ>(sm.plane[s], DY, D, halo_off, ty, tz, ring[k], dyy, dzz);
                    // ---- centre x = pp - 2, whose in-plane record is that of plane g - 2
                    const uint32_t g3n = g3 == 2 ? 0 : g3 + 1;  // (g + 1) % 3 == (g - 2) % 3
                    const int x = pp - 2;
                    __syncwarp();
                    if (x >= xs)
                        centre_site<TY, TZ, POT, DUMP, SEX>(D, ring[(k + 1) % 5], ring[(k + 2) % 5], ring[(k + 3) % 5],
                                            ring[(k + 4) % 5], ring[k], kXm1(), kXm2(),
                                            twarp + RECC * g3n,
                                            make_uint4(twarp + kDzCol + 4 * ((k + 1) % 5),
                                                       twarp + kDzCol + 4 * ((k + 2) % 5),
                                                       twarp + kDzCol + 4 * ((k + 3) % 5),
                                                       twarp + kDzCol + 4 * ((k + 4) % 5)),
                                            &sm.vpl[s][ty][tz], use_v,
                                            valid, phiout, vout, si, a32);
                    // this warp is done with slot s; the last warp to leave it streams
                    // plane pp + NSLOT (and its velocity) into it
                    __syncwarp();
                    if ((tid & 31) == 0) {
                        __threadfence_block();
                        if (atomicAdd(&sm.rel[s], 1) == THREADS / 32 - 1) {
                            sm.rel[s] = 0;
                            __threadfence_block();
                            if (pp + NSLOT <= pl) {
                                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                                issue(pp + NSLOT, s);
                            }
                        }
                    }
                    plane_record<TY, TZ, SEX>(DY, D, ty, tz, ring[k], dyy, dzz, twarp + RECC * g3);
                    if constexpr (SEX) {
                        const float zr[4] = {ring[k].dz.a.x, ring[k].dz.a.y, ring[k].dz.b.x, ring[k].dz.b.y};
                        tmem_st4(twarp + kDzCol + 4 * k, zr);
                    }
                    ++g;
                    g3 = g3n;
                    si += plane_stride;
                }
                // a failed copy is noticed once per group of five planes
                if (*(volatile int *)&sm.flag) failed = true;
                // FP32 partial sums cover at most 40 planes before entering the double-float sums
                if ((++nouter & 7) == 0) flush(acc, amax, THREADS, a32);
            }
            flush(acc, amax, THREADS, a32);
            // every warp is done with the run's planes before its slots are reused
            __syncthreads();
            failed = sm.flag != 0;
        }
        if (failed) break;

        // ---- this CTA is done with lattice D: block reduction, per-lattice finish
        DF tot[kSums];
        float tmax = 0.f;
        if constexpr (THREADS / 32 > kSums && THREADS % 64 == 0) {
            // the accumulators were last written before the run's closing barrier
            block_reduce_df_smem<THREADS>(&sm.accs[0][0], sm.amaxs, sm.dfred, sm.mxred, tot, tmax,
                                          tid);
        } else {
            DF mine[kSums];
            float mmax;
            load_sums(acc, amax, THREADS, mine, mmax);
            block_reduce_df<THREADS / 32>(mine, mmax, sm.dfred, sm.mxred, tot, tmax, tid,
                                          CtaSync{});
        }
        if (tid == 0) {
            write_record(D, (int)blockIdx.x - D.cta_first, tot, tmax);
            sm.last = (atom_add_acq_rel(&ctrl->done, 1u) == (unsigned)(D.cta_count - 1));
        }
        // the last CTA's threads read the records after thread 0's acquire
        __syncthreads();
        if (sm.last)
            finish_lattice<THREADS / 32>(D, ctrl, cur, mode, pred, dry, sm.dfred, sm.mxred, tid,
                                         CtaSync{});
        __syncthreads();
    }

    if constexpr (!BATCHED) {
        if (one.fuse_fix && !failed) {
            // the arrest decision is made by the last CTA to finish; every CTA
            // (all resident: a cooperative launch of at most one per SM) waits
            // for it, bounded, and corrects its own sites when the decision the
            // step ran with was wrong
            if (tid == 0) {
                const long long steps0 = sm.steps0;
                long long st = ld_acquire_s64(&one.ctrl->steps);
                if (st == steps0) {
                    const unsigned long long t0 = global_ns();
                    do {
                        st = ld_acquire_s64(&one.ctrl->steps);
                    } while (st == steps0 && global_ns() - t0 < kWaitLimitNs);
                }
                sm.fixv = (st == steps0) ? 2 : __ldcg(&one.ctrl->fix);
            }
            __syncthreads();
            const int fx = sm.fixv;
            if (fx == 2) {
                if (tid == 0) atomicExch(&one.ctrl->status, (int)DEV_TIMEOUT);
            } else if (fx != 0) {
                const bool listed2 = split.n > 0, locked2 = split.n == -2;
                const long long v0 = locked2 ? 0
                                     : listed2 ? split.start[blockIdx.x] : total_units * blockIdx.x / gridDim.x;
                const long long v1 = locked2 ? lock_units(split, blockIdx.x, one.nix)
                                     : listed2 ? split.start[blockIdx.x + 1]
                                               : total_units * (blockIdx.x + 1) / gridDim.x;
                correct_own_sites<TY, TZ>(one, split, v0, v1, sm.cur_used, fx, tid / TZ, tid % TZ);
            }
        }
    }

    if (failed) {
        // a plane copy never landed: record it, let in-flight copies finish
        // (bounded), and leave without closing the lattice's reduction
        if (tid == 0) {
            const InstDesc &Df = BATCHED ? table[inst] : one;
            atomicExch(&Df.ctrl->status, (int)DEV_TIMEOUT);
            for (int s = 0; s < NSLOT; ++s) {
                (void)mbar_wait(&sm.bar[s], 0, 50000000ull);
                (void)mbar_wait(&sm.bar[s], 1, 50000000ull);
            }
        }
    }
    // every warp is done with its TMEM columns: free the allocation
    tmem_wait_st();
    tmem_fence_before();
    __syncthreads();
    if (tid < 32) {
        tmem_fence_after();
        tmem_dealloc(sm.tmem, TCOLS);
    }
}

// Pointwise correction of a mispredicted arrest decision (the finished step
// stored fix = -1: the velocity should have been zeroed, +1: kept): the site
// update is redone from the previous buffers, v = v_new + fix v_old,
// phi = normalise(phi_old + dt v).  Warps of the grid share the z-rows of
// interior sites; each lane stages two sites' loads before its stores.
__device__ __forceinline__ void fixup_rows(float4 *const (&phi)[2], float4 *const (&vel)[2],
                                           int cur, int n0, int n1, int n2, float dt, int fix,
                                           int wg, int ws)
{
    const int nb = cur, ob = cur ^ 1;  // cur was already flipped by the finished step
    const float4 *__restrict__ vnp = vel[nb];
    const float4 *__restrict__ vop = vel[ob];
    const float4 *__restrict__ fop = phi[ob];
    float4 *__restrict__ vst = vel[nb];
    float4 *__restrict__ fst = phi[nb];
    const int iy = n1 - 4, iz = n2 - 4, rows = (n0 - 4) * iy;
    const float sgn = (float)fix;
    const int lane = threadIdx.x & 31;
    for (int row = wg; row < rows; row += ws) {
        const int xr = row / iy;
        const size_t base = ((size_t)(2 + xr) * n1 + (2 + row - xr * iy)) * n2 + 2;
        for (int z0 = 0; z0 < iz; z0 += 64) {
            float4 vn[2], vo[2], fo[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int z = z0 + 32 * k + lane;
                if (z < iz) {
                    vn[k] = vnp[base + z];
                    vo[k] = __ldcs(vop + base + z);
                    fo[k] = __ldcs(fop + base + z);
                }
            }
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int z = z0 + 32 * k + lane;
                if (z < iz) {
                    float4 v, p;
                    arrest_fix_site(vn[k], vo[k], fo[k], sgn, dt, v, p);
                    vst[base + z] = v;
                    fst[base + z] = p;
                }
            }
        }
    }
}

struct FixDesc {
    float4 *phi[2];
    float4 *vel[2];
    Ctrl *ctrl;
    int n0, n1, n2;
    float dt;
};

// one lattice; mostly an early exit
__global__ void __launch_bounds__(512, 2) k_fixup_one(const __grid_constant__ FixDesc d)
{
    const int fix = __ldcg(&d.ctrl->fix);
    if (fix == 0) return;
    const int warps = blockDim.x >> 5;
    fixup_rows(d.phi, d.vel, __ldcg(&d.ctrl->cur), d.n0, d.n1, d.n2, d.dt, fix,
               blockIdx.x * warps + (threadIdx.x >> 5), gridDim.x * warps);
}

// every lattice of a batch: each warp reads 32 lattices' flags at once and
// the whole grid then corrects, one after another, the lattices that need it
__global__ void __launch_bounds__(512, 2) k_fixup_batch(const InstDesc *__restrict__ table, int ninst)
{
    const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
    const int wg = blockIdx.x * warps + (threadIdx.x >> 5), ws = gridDim.x * warps;
    for (int i0 = 0; i0 < ninst; i0 += 32) {
        int fix = 0, cur = 0;
        if (i0 + lane < ninst) {
            const Ctrl *c = table[i0 + lane].ctrl;
            fix = __ldcg(&c->fix);
            cur = __ldcg(&c->cur);
        }
        unsigned need = __ballot_sync(0xffffffffu, fix != 0);
        while (need) {
            const int j = __ffs(need) - 1;
            need &= need - 1;
            const int f = __shfl_sync(0xffffffffu, fix, j), cj = __shfl_sync(0xffffffffu, cur, j);
            const InstDesc &D = table[i0 + j];
            fixup_rows(D.phi, D.vel, cj, D.n0, D.n1, D.n2, D.dt.x, f, wg, ws);
        }
    }
}

// ---------------------------------------------------- tensor maps
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


// ------------------------------------------------------------------- host
static int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 152;
    return n > 0 ? n : 152;
}

constexpr int kMaxGrid = 1216;  // persistent CTAs per launch (partial records per lattice)

struct TileShape {
    int ty, tz;
};
// Autotuner candidates: (rows, columns) of interior sites per CTA
static const TileShape kTiles[] = {{8, 32}, {4, 32}, {16, 16}, {8, 16}, {16, 32}};
constexpr int kNumTiles = 5;
// a single lattice runs one 512-thread CTA of 16 x 32 columns per SM: with no
// per-plane barrier its 16 warps cost nothing extra, and the haloed plane is
// 1.41x the sites it updates instead of 1.69x for 8 x 32 (measured 3-3.5%
// faster than two 8 x 32 CTAs per SM on 128^3, 256^3 and 512^3)
constexpr int kSingleTile = 4;

template <int TY, int TZ, bool B, bool POT = false, bool DUMP = false, bool SEX = false>
static void *kernel_ptr()
{
    return reinterpret_cast<void *>(&k_step_f32<TY, TZ, B, POT, DUMP, SEX>);
}

template <int TY, int TZ, bool B, bool POT = false>
static cudaError_t launch_shape(const InstDesc &one, const CtaSplit &split, const InstDesc *table,
                                int ninst, long long units, int grid, int dry, cudaStream_t s)
{
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lock(mu);
        if (dev < 64 && !done[dev]) {
            cudaError_t e = cudaFuncSetAttribute(k_step_f32<TY, TZ, B, POT>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)step_smem_bytes<TY, TZ>());
            if (e != cudaSuccess) return e;
            done[dev] = true;
        }
    }
    k_step_f32<TY, TZ, B, POT><<<(unsigned)grid, TY * TZ, step_smem_bytes<TY, TZ>(), s>>>(
        one, split, table, ninst, units, dry);
    return cudaGetLastError();
}

template <bool B, bool POT = false>
static cudaError_t launch_tile(int tile, const InstDesc &one, const CtaSplit &split,
                               const InstDesc *table, int ninst, long long units, int grid, int dry,
                               cudaStream_t s)
{
    switch (tile) {
    case 0: return launch_shape<8, 32, B, POT>(one, split, table, ninst, units, grid, dry, s);
    case 1: return launch_shape<4, 32, B, POT>(one, split, table, ninst, units, grid, dry, s);
    case 2: return launch_shape<16, 16, B, POT>(one, split, table, ninst, units, grid, dry, s);
    case 4: return launch_shape<16, 32, B, POT>(one, split, table, ninst, units, grid, dry, s);
    default: return launch_shape<8, 16, B, POT>(one, split, table, ninst, units, grid, dry, s);
    }
}

// Persistent CTAs of one tile shape that fit on the device.
template <int TY, int TZ, bool B> static int occupancy_of()
{
    int n = 0;
    cudaFuncSetAttribute(k_step_f32<TY, TZ, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)step_smem_bytes<TY, TZ>());
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_f32<TY, TZ, B>, TY * TZ,
                                                      step_smem_bytes<TY, TZ>()) != cudaSuccess)
        n = 1;
    return n > 0 ? n : 1;
}

static int blocks_per_sm(int tile, bool batched)
{
    static std::mutex mu;
    static int cache[2][kNumTiles] = {{0}};
    std::lock_guard<std::mutex> lock(mu);
    int &c = cache[batched][tile];
    if (!c) {
        switch (tile * 2 + (batched ? 1 : 0)) {
        case 0: c = occupancy_of<8, 32, false>(); break;
        case 1: c = occupancy_of<8, 32, true>(); break;
        case 2: c = occupancy_of<4, 32, false>(); break;
        case 3: c = occupancy_of<4, 32, true>(); break;
        case 4: c = occupancy_of<16, 16, false>(); break;
        case 5: c = occupancy_of<16, 16, true>(); break;
        case 6: c = occupancy_of<8, 16, false>(); break;
        case 7: c = occupancy_of<8, 16, true>(); break;
        case 8: c = occupancy_of<16, 32, false>(); break;
        default: c = occupancy_of<16, 32, true>(); break;
        }
    }
    return c;
}


// Lattice description for a tile shape; the work partition is filled later.
// pot_sums: the lattice runs in a potentials instantiation (its e0 slot
// then holds the whole potential density, whatever the lattice's model).
static bool fill_desc(InstDesc &d, const skyrme_lattice &lat, const skyrme_state &st, Ctrl *ctrl,
                      double dt, int mode, int tile, bool pot_sums = false)
{
    const int ty = kTiles[tile].ty, tz = kTiles[tile].tz;
    memset(&d, 0, sizeof(d));
    for (int i = 0; i < 2; ++i) {
        if (!make_plane_map(&d.map[i], st.phi[i], lat, 4 * (tz + 4), ty + 4)) return false;
        if (!make_plane_map(&d.vmap[i], st.vel[i], lat, 4 * tz, ty)) return false;
        d.phi[i] = static_cast<float4 *>(st.phi[i]);
        d.vel[i] = static_cast<float4 *>(st.vel[i]);
    }
    d.ctrl = ctrl;
    d.n0 = lat.n[0];
    d.n1 = lat.n[1];
    d.n2 = lat.n[2];
    const int nyt = (lat.n[1] - 4 + ty - 1) / ty;
    d.nzt = (lat.n[2] - 4 + tz - 1) / tz;
    d.nix = lat.n[0] - 4;
    d.units = (long long)nyt * d.nzt * d.nix;
    auto pair = [](double w) { return make_float2((float)w, (float)w); };
    auto split = [](double w) {  // (hi, lo) with hi + lo = w to about 48 bits
        const float hi = (float)w;
        return make_float2(hi, (float)(w - (double)hi));
    };
    // unscaled stencils: u = 12h d phi, N = -12h^2 d^2 phi; the force scale
    // B = k1^2 k2 with k1 = 1/(12h), k2 = 1/(12h^2)
    const double k1 = 1.0 / (12.0 * lat.h), k2 = 1.0 / (12.0 * lat.h * lat.h), B = k1 * k1 * k2;
    d.m2 = (float)(lat.m * lat.m);
    d.bm2 = (float)(lat.m * lat.m / B);
    d.negK = (float)(-1.0 / (k1 * k1));
    d.my2 = (float)(lat.m_y * lat.m_y);
    d.mz2 = (float)(lat.m_z * lat.m_z);
    d.mw2 = (float)(lat.m_w * lat.m_w);
    d.bmy2 = (float)(lat.m_y * lat.m_y / B);
    d.bmz2 = (float)(lat.m_z * lat.m_z / B);
    d.bmw2 = (float)(lat.m_w * lat.m_w / B);
    d.e0_scale = pot_sums || lattice_potentials(lat) || lat.c6 != 0.0 ? 1.f : 2.f * d.m2;
    d.c6 = (float)lat.c6;
    d.c6b = (float)(lat.c6 * k1 * k1);
    d.dk2 = (float)(k1 * k1);
    d.dk3 = (float)(k1 * k1 * k1);
    d.dk4 = (float)(k1 * k1 * k1 * k1);
    d.s_e2 = split(k1 * k1);
    d.s_e4 = split(k1 * k1 * k1 * k1);
    d.s_b = split(k1 * k1 * k1);
    d.s_e6 = split(k1 * k1 * k1 * k1 * k1 * k1);
    d.s_f = split(B * B);
    d.dt = make_float2((float)dt, (float)dt);
    d.dt2 = pair(2.0 * dt * B);
    const double h3 = lat.h * lat.h * lat.h;
    d.h3_hi = (float)h3;
    d.h3_lo = (float)(h3 - (double)d.h3_hi);
    d.mode = mode;
    return true;
}

// Split total units over `grid` CTAs and record, for each lattice, the CTAs
// that touch it; partial records are laid out lattice after lattice.
static void partition(std::vector<InstDesc> &ds, int grid, double *parts,
                      const int *starts = nullptr)
{
    long long total = 0;
    for (auto &d : ds) {
        d.unit_start = total;
        total += d.units;
    }
    size_t off = 0;
    for (auto &d : ds) {
        const long long lo = d.unit_start, hi = d.unit_start + d.units;
        int first = -1, count = 0;
        for (int b = 0; b < grid; ++b) {
            const long long b0 = starts ? starts[b] : total * b / grid;
            const long long b1 = starts ? starts[b + 1] : total * (b + 1) / grid;
            if (b1 > lo && b0 < hi) {
                if (first < 0) first = b;
                ++count;
            }
        }
        d.cta_first = first;
        d.cta_count = count;
        d.parts = parts + off * kPartialDoubles;
        off += (size_t)count;
    }
}

static long long total_units(const std::vector<InstDesc> &ds)
{
    long long t = 0;
    for (auto &d : ds) t += d.units;
    return t;
}

static int grid_for(int tile, bool batched, long long units)
{
    long long g = (long long)sm_count() * blocks_per_sm(tile, batched);
    g = std::min<long long>(g, units);
    g = std::min<long long>(g, kMaxGrid);
    return (int)std::max<long long>(g, 1);
}

bool f32_fast_path_available(const skyrme_lattice &lat)
{
    // the streaming kernel needs the driver's tensor-map encoder
    return lat.precision == 32 && encode_fn() != nullptr;
}

int f32_fast_blocks(const skyrme_lattice &lat)
{
    (void)lat;
    return kMaxGrid;
}

// The even split (batched launches).
static const CtaSplit kEvenSplit = {};

// Pipeline fill of a run, in planes: its first centre needs planes x - 2 ..
// x + 2, so a run of r centres streams r + 4 planes.
constexpr int kRunFill = 4;

// Greedy cover of `units` (columns of nix planes, one after the other) by CTAs
// that each stream at most `cap` planes, a run costing its centres plus the
// fill.  Fills `start` and returns the CTAs used (INT_MAX when more than
// max_ctas would be needed).
static int greedy_split(long long units, int nix, double cap, int max_ctas, int *start)
{
    long long pos = 0;
    int b = 0;
    while (pos < units) {
        if (b >= max_ctas) return 0x7fffffff;
        start[b++] = (int)pos;
        double budget = cap;
        bool first = true;
        while (pos < units) {
            const long long col_end = (pos / nix + 1) * (long long)nix;
            long long take = (long long)(budget - kRunFill);
            if (first) take = std::max(take, 1LL);  // every CTA streams at least one centre
            take = std::min(take, col_end - pos);
            if (take <= 0) break;
            pos += take;
            budget -= (double)(kRunFill + take);
            first = false;
            if (pos < col_end) break;  // the budget ran out inside the column
        }
    }
    start[b] = (int)pos;
    return b;
}

// Unit ranges for `grid` CTAs whose largest plane count is as small as the
// greedy cover allows (bisection on the cap).
static bool balanced_split(long long units, int nix, int grid, CtaSplit &out)
{
    out = CtaSplit{};
    if (grid <= 0 || grid > kSplitMax || units > 0x7fffffffLL || units < grid) return false;
    double lo = (double)units / grid, hi = (double)units / grid + 2.0 * kRunFill + nix;
    for (int it = 0; it < 48; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (greedy_split(units, nix, mid, grid, out.start) <= grid) hi = mid;
        else lo = mid;
    }
    out.n = greedy_split(units, nix, hi, grid, out.start);
    if (out.n > grid) out.n = 0;
    return out.n > 0;
}

// Largest plane count of a cover (unit starts of n CTAs over columns of nix
// planes).
static long long max_planes(const int *start, int n, int nix)
{
    long long m = 0;
    for (int b = 0; b < n; ++b) {
        long long p = 0;
        for (long long u = start[b]; u < start[b + 1];) {
            const long long e = std::min<long long>(start[b + 1], (u / nix + 1) * nix);
            p += e - u + kRunFill;
            u = e;
        }
        m = std::max(m, p);
    }
    return m;
}

// The lockstep schedule (n = -2) of ncol = units / nix columns for `grid`
// CTAs: W = ncol / grid waves of whole columns, then the R = ncol % grid
// remaining columns' heads (x < a, one per CTA b < R) and tails (x >= a, a
// balanced cover over the other CTAs), the head length a chosen so that the
// heads' planes match the tails' largest.  Without waves, CTAs left without
// a tail are not launched (lg: the CTAs to launch), so every launched CTA
// streams at least one plane.  Returns the largest plane count of a CTA, or
// -1 when the geometry has no such schedule.
static long long lock_split(long long units, int nix, int grid, CtaSplit &out)
{
    out = CtaSplit{};
    const long long ncol = nix > 0 ? units / nix : 0;
    if (grid <= 0 || grid > kSplitMax || units > 0x7fffffffLL || ncol * nix != units || ncol == 0)
        return -1;
    const int W = (int)(ncol / grid), R = (int)(ncol % grid);
    out.n = -2;
    out.lw = W;
    out.lr = R;
    out.lg = grid;
    const long long wave = (long long)W * (nix + kRunFill);
    if (R == 0) return wave;
    std::vector<int> ts(grid - R + 1);
    int used = 0;  // tail CTAs given units by the last cover
    auto tails = [&](int a) -> long long {
        const int tn = nix - a, nt = grid - R;
        const long long tu = (long long)R * tn;
        double lo = (double)tu / nt, hi = lo + 2.0 * kRunFill + tn;
        for (int it = 0; it < 40; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (greedy_split(tu, tn, mid, nt, ts.data()) <= nt) hi = mid;
            else lo = mid;
        }
        const int n = greedy_split(tu, tn, hi, nt, ts.data());
        if (n > nt) return -1;
        for (int k = n + 1; k <= nt; ++k) ts[k] = ts[n];
        used = n;
        return max_planes(ts.data(), n, tn);
    };
    // the smallest a whose heads reach the tails' largest plane count, or
    // the one before it
    int lo = 1, hi = nix - 1;
    while (lo < hi) {
        const int mid = (lo + hi) / 2;
        const long long t = tails(mid);
        if (t >= 0 && t <= mid + kRunFill) hi = mid;
        else lo = mid + 1;
    }
    long long best = -1;
    int best_a = 0;
    for (int a = std::max(1, lo - 1); a <= std::min(nix - 1, lo); ++a) {
        const long long t = tails(a);
        if (t < 0) continue;
        const long long m = std::max<long long>(t, a + kRunFill);
        if (best < 0 || m < best) best = m, best_a = a;
    }
    if (best < 0) return -1;
    (void)tails(best_a);
    out.la = best_a;
    for (int k = 0; k <= grid - R; ++k) out.start[R + k] = ts[k];
    if (W == 0) out.lg = R + used;
    return wave + best;
}

// Single-lattice split policy (skyrme_set_single_split): process-wide.
static std::atomic<int> g_single_split{SKYRME_SPLIT_AUTO};

// The split of a single lattice's units among at most `grid` CTAs under
// `policy`; *ctas receives the CTAs to launch.  AUTO takes the balanced
// split: the lockstep schedule cuts the DRAM traffic (1.31x -> 1.02x of the
// algorithmic bytes on 256^3) but measured slower wherever the step is not
// L2-resident (256^3: 57.8 against 59.4, 512^3: 62.2 against 64.3
// Gsite-updates/s), and equal on 128^3.  Cached for the last geometry and
// policy.
static void plan_single(long long units, int nix, int grid, int policy, CtaSplit &out, int *ctas)
{
    static thread_local long long key_units = -1;
    static thread_local int key_nix = -1, key_grid = -1, key_policy = -1, key_ctas = 0;
    static thread_local CtaSplit cached;
    if (units == key_units && nix == key_nix && grid == key_grid && policy == key_policy) {
        out = cached;
        *ctas = key_ctas;
        return;
    }
    CtaSplit bal, lk;
    const bool have_bal = balanced_split(units, nix, grid, bal);
    long long lk_max = -1;
    if (policy == SKYRME_SPLIT_LOCKSTEP) lk_max = lock_split(units, nix, grid, lk);
    const bool use_lock = policy == SKYRME_SPLIT_LOCKSTEP && lk_max >= 0;
    if (use_lock) {
        out = lk;
        *ctas = lk.lg;
    } else if (have_bal) {
        out = bal;
        *ctas = bal.n;
    } else {
        out = CtaSplit{};
        *ctas = grid;
    }
    key_units = units, key_nix = nix, key_grid = grid, key_policy = policy, key_ctas = *ctas;
    cached = out;
}

// The same cover for a batch: the lattices' columns concatenated, each
// lattice with its own column length (interior planes).
static int greedy_split_batch(const std::vector<InstDesc> &ds, long long units, double cap,
                              int max_ctas, int *start)
{
    long long pos = 0;
    int b = 0;
    size_t i = 0;
    while (pos < units) {
        if (b >= max_ctas) return 0x7fffffff;
        start[b++] = (int)pos;
        double budget = cap;
        bool first = true;
        while (pos < units) {
            while (pos >= ds[i].unit_start + ds[i].units) ++i;
            const long long nix = ds[i].nix;
            const long long col_end = ds[i].unit_start + ((pos - ds[i].unit_start) / nix + 1) * nix;
            long long take = (long long)(budget - kRunFill);
            if (first) take = std::max(take, 1LL);
            take = std::min(take, col_end - pos);
            if (take <= 0) break;
            pos += take;
            budget -= (double)(kRunFill + take);
            first = false;
            if (pos < col_end) break;
        }
    }
    start[b] = (int)pos;
    return b;
}

// Unit ranges of at most `grid` CTAs over a batch whose largest plane count
// is as small as the greedy cover allows; the number of ranges, or 0.
// ds[].unit_start must be set.
static int balanced_split_batch(const std::vector<InstDesc> &ds, int grid, std::vector<int> &start)
{
    const long long units = total_units(ds);
    start.assign((size_t)grid + 1, 0);
    if (grid <= 0 || units > 0x7fffffffLL || units < grid) return 0;
    long long maxnix = 1;
    for (auto &d : ds) maxnix = std::max<long long>(maxnix, d.nix);
    double lo = (double)units / grid, hi = (double)units / grid + 2.0 * kRunFill + (double)maxnix;
    for (int it = 0; it < 48; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (greedy_split_batch(ds, units, mid, grid, start.data()) <= grid) hi = mid;
        else lo = mid;
    }
    const int n = greedy_split_batch(ds, units, hi, grid, start.data());
    return n <= grid ? n : 0;
}

// Self-test of the bounded wait the step kernels use on their TMA copies:
// thread 0 waits on a shared-memory mbarrier that nothing ever completes,
// gives up after limit_ns, and records SKYRME_ETIMEOUT in the control block,
// as a step kernel does when a plane copy never lands.  Nothing faults or
// hangs: the kernel returns after the limit.
__global__ void k_wait_selftest(Ctrl *c, unsigned long long limit_ns)
{
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(&bar, 0, limit_ns)) atomicExch(&c->status, (int)DEV_TIMEOUT);
}

cudaError_t launch_wait_selftest(void *ctrl, unsigned long long limit_ns, cudaStream_t s)
{
    k_wait_selftest<<<1, 32, 0, s>>>(static_cast<Ctrl *>(ctrl), limit_ns);
    return cudaGetLastError();
}

// nsteps iterations of a single lattice: one step launch each (a whole
// lattice in ARRESTED mode corrects its own mispredicted decisions inside
// it; an x-slab's correction follows the decision over all slabs).  The
// tensor maps and the work split are the same for every iteration, so they
// are prepared once per call; the loop only launches.
cudaError_t launch_iterations_f32_fast(const skyrme_lattice &lat, const FlowArgs &a, int nsteps,
                                       cudaStream_t s)
{
    if (nsteps <= 0) return cudaSuccess;
    const int tile = kSingleTile;
    skyrme_state st;
    for (int i = 0; i < 2; ++i) {
        st.phi[i] = a.phi[i];
        st.vel[i] = a.vel[i];
    }
    std::vector<InstDesc> ds(1);
    if (!fill_desc(ds[0], lat, st, static_cast<Ctrl *>(a.ctrl), a.dt, a.mode, tile))
        return cudaErrorInvalidValue;
    int grid = grid_for(tile, false, ds[0].units);
    CtaSplit split;
    plan_single(ds[0].units, ds[0].nix, grid, g_single_split.load(), split, &grid);
    partition(ds, grid, a.step_parts, split.n > 0 ? split.start : nullptr);

    ds[0].slab_rec = a.slab_rec;
    ds[0].dump = static_cast<float4 *>(a.dump);
    if (a.dump) {
        // the dump kernels scale each site's densities and sum the scaled values
        ds[0].s_e2 = ds[0].s_e4 = ds[0].s_b = make_float2(1.f, 0.f);
    }
    // ARRESTED whole lattices correct their own mispredicted decisions inside
    // the step (the CTAs wait for the last one's decision, so the launch is
    // cooperative: every CTA resident at once); an x-slab's decision and
    // fix-up come after the decision over all slabs
    const bool fused = a.mode == SKYRME_ARRESTED && !a.slab_rec;
    ds[0].fuse_fix = fused ? 1 : 0;
    // the instantiation: the standard model, the Section 7.8 potentials, the
    // sextic term (with any potentials), each also with the density dump
    // (not for the sextic term)
    const bool sex = lat.c6 != 0.0;
    const bool pot = sex || lattice_potentials(lat);
    const bool dump = a.dump != nullptr;
    if (sex && dump) return cudaErrorInvalidValue;
    void *kern = sex ? kernel_ptr<16, 32, false, true, false, true>()
               : pot ? (dump ? kernel_ptr<16, 32, false, true, true>() : kernel_ptr<16, 32, false, true>())
                     : (dump ? kernel_ptr<16, 32, false, false, true>() : kernel_ptr<16, 32, false>());
    const size_t smem = sex ? step_smem_bytes<16, 32, true>() : step_smem_bytes<16, 32>();
    {
        static std::mutex mu;
        static bool done[5][64] = {{false}};
        const int which = sex ? 4 : (pot ? 2 : 0) + (dump ? 1 : 0);
        int dev = 0;
        cudaGetDevice(&dev);
        std::lock_guard<std::mutex> lock(mu);
        if (dev < 64 && !done[which][dev]) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
            done[which][dev] = true;
        }
    }
    const InstDesc *tab = nullptr;
    int ninst = 1, dry = 0;
    long long units = ds[0].units;
    void *args[] = {(void *)&ds[0], (void *)&split, (void *)&tab, (void *)&ninst, (void *)&units,
                    (void *)&dry};
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = fused ? 1 : 0;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = fused ? 1 : 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(16 * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    for (int k = 0; k < nsteps; ++k) {
        const cudaError_t e = cudaLaunchKernelExC(&cfg, kern, args);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_fixup_f32_fast(const skyrme_lattice &lat, const FlowArgs &a, cudaStream_t s)
{
    FixDesc fx;
    for (int i = 0; i < 2; ++i) {
        fx.phi[i] = static_cast<float4 *>(a.phi[i]);
        fx.vel[i] = static_cast<float4 *>(a.vel[i]);
    }
    fx.ctrl = static_cast<Ctrl *>(a.ctrl);
    fx.n0 = lat.n[0];
    fx.n1 = lat.n[1];
    fx.n2 = lat.n[2];
    fx.dt = (float)a.dt;
    const long long rows = (long long)(lat.n[0] - 4) * (lat.n[1] - 4);
    const int fix_blocks = (int)std::max(1LL, std::min((long long)sm_count() * 2, (rows + 15) / 16));
    k_fixup_one<<<fix_blocks, 512, 0, s>>>(fx);
    return cudaGetLastError();
}

}  // namespace skyrme

// ---------------------------------------------------------- batch C ABI
using namespace skyrme;

struct skyrme_batch {
    int ninst = 0;
    int mode = 0;
    int tile = 0;
    int grid = 1;
    long long units = 0;
    std::vector<skyrme_lattice> lats;
    std::vector<skyrme_state> states;
    std::vector<double> dt;
    InstDesc *d_table = nullptr;  // in the caller's batch scratch
    double *d_parts = nullptr;
    int fixup_blocks = 1;
    bool pot = false;  // some lattice has a Section 7.8 potential: the POT kernels
    int split = 1;     // CTA ranges balanced by streamed planes (1) or even by units (0)
};

// The lattice table, followed by the CTAs' unit ranges of a balanced split
static size_t table_bytes(int ninst)
{
    return ((size_t)ninst * sizeof(InstDesc) + (kMaxGrid + 1) * sizeof(int) + 255) & ~(size_t)255;
}
static size_t batch_parts_bytes(int ninst)
{
    return ((size_t)(kMaxGrid + ninst) * kPartialDoubles * sizeof(double) + 255) & ~(size_t)255;
}

// Encode the lattice table for tile shape `tile` and split mode `split` and
// upload it (with the CTAs' unit ranges when the split is balanced).
static skyrme_status upload_table(skyrme_batch *b, int tile, int split)
{
    std::vector<InstDesc> ds(b->ninst);
    for (int i = 0; i < b->ninst; ++i) {
        Ctrl *ctrl = static_cast<Ctrl *>(b->states[i].scratch);
        if (!fill_desc(ds[i], b->lats[i], b->states[i], ctrl, b->dt[i], b->mode, tile, b->pot))
            return SKYRME_EINVAL;
    }
    const long long units = total_units(ds);
    int grid = grid_for(tile, true, units);
    long long pos = 0;
    for (auto &d : ds) {
        d.unit_start = pos;
        pos += d.units;
    }
    std::vector<int> starts;
    const int n = split ? balanced_split_batch(ds, grid, starts) : 0;
    if (n > 0) grid = n;
    partition(ds, grid, b->d_parts, n > 0 ? starts.data() : nullptr);
    const size_t tb = ds.size() * sizeof(InstDesc);
    std::vector<unsigned char> host(tb + (n > 0 ? (size_t)(n + 1) * sizeof(int) : 0));
    memcpy(host.data(), ds.data(), tb);
    if (n > 0) memcpy(host.data() + tb, starts.data(), (size_t)(n + 1) * sizeof(int));
    if (cudaMemcpy(b->d_table, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return SKYRME_ECUDA;
    b->tile = tile;
    b->split = n > 0 ? 1 : 0;
    b->grid = grid;
    b->units = units;
    return SKYRME_OK;
}

static skyrme_status batch_launch(skyrme_batch *b, int nsteps, int dry, cudaStream_t s)
{
    InstDesc dummy;
    memset(&dummy, 0, sizeof(dummy));
    // split.n = -1: the ranges follow the table in device memory
    static const CtaSplit kBatchListed = {-1};
    const CtaSplit &sp = b->split ? kBatchListed : kEvenSplit;
    for (int k = 0; k < nsteps; ++k) {
        const cudaError_t e =
            b->pot ? launch_tile<true, true>(b->tile, dummy, sp, b->d_table, b->ninst, b->units,
                                             b->grid, dry, s)
                   : launch_tile<true>(b->tile, dummy, sp, b->d_table, b->ninst, b->units, b->grid,
                                       dry, s);
        if (e != cudaSuccess) return SKYRME_ECUDA;
        if (!dry && b->mode == MODE_ARRESTED) {
            k_fixup_batch<<<(unsigned)b->fixup_blocks, 512, 0, s>>>(b->d_table, b->ninst);
            if (cudaGetLastError() != cudaSuccess) return SKYRME_ECUDA;
        }
    }
    return SKYRME_OK;
}

namespace skyrme {
bool state_ok_for_batch(const skyrme_lattice *lat, const skyrme_state *st);
skyrme_status make_graph(skyrme_batch *b, int nsteps, cudaStream_t s, skyrme_graph **out);
}  // namespace skyrme

extern "C" {

size_t skyrme_batch_scratch_bytes(int ninst, const skyrme_lattice *lats)
{
    if (ninst < 1 || !lats) return 0;
    return table_bytes(ninst) + batch_parts_bytes(ninst);
}

skyrme_status skyrme_batch_create(int ninst, const skyrme_lattice *lats, skyrme_state *states,
                                  const double *dt, int mode, void *scratch, size_t scratch_bytes,
                                  skyrme_batch **out)
{
    if (!out) return SKYRME_EINVAL;
    *out = nullptr;
    if (ninst < 1 || !lats || !states || !dt || !scratch) return SKYRME_EINVAL;
    if (mode != MODE_NEWTON && mode != MODE_ARRESTED && mode != MODE_GRADIENT) return SKYRME_EINVAL;
    if ((uintptr_t)scratch % 256) return SKYRME_EINVAL;
    if (scratch_bytes < skyrme_batch_scratch_bytes(ninst, lats)) return SKYRME_ENOMEM;
    for (int i = 0; i < ninst; ++i) {
        if (lats[i].precision != 32) return SKYRME_EUNSUPPORTED;
        if (!state_ok_for_batch(&lats[i], &states[i])) return SKYRME_EINVAL;
        if (!(dt[i] > 0.0)) return SKYRME_EINVAL;
    }
    // batches run the standard model and the Section 7.8 potentials; the
    // sextic term runs on single lattices
    bool pot = false;
    for (int i = 0; i < ninst; ++i) {
        if (lats[i].c6 != 0.0) return SKYRME_EUNSUPPORTED;
        pot = pot || lattice_potentials(lats[i]);
    }
    if (!f32_fast_path_available(lats[0])) return SKYRME_EUNSUPPORTED;
    {
        const void *p = scratch;
        skyrme_status rc = on_current_device(&p, 1);
        if (rc != SKYRME_OK) return rc;
    }
    for (int i = 0; i < ninst; ++i) {
        const void *p[5] = {states[i].phi[0], states[i].phi[1], states[i].vel[0], states[i].vel[1],
                            states[i].scratch};
        skyrme_status rc = on_current_device(p, 5);
        if (rc != SKYRME_OK) return rc;
    }
    skyrme_batch *b = new skyrme_batch();
    b->ninst = ninst;
    b->mode = mode;
    b->fixup_blocks = sm_count() * 2;
    b->pot = pot;
    b->lats.assign(lats, lats + ninst);
    b->states.assign(states, states + ninst);
    b->dt.assign(dt, dt + ninst);
    b->d_table = static_cast<InstDesc *>(scratch);
    b->d_parts = reinterpret_cast<double *>(static_cast<char *>(scratch) + table_bytes(ninst));
    skyrme_status rc = upload_table(b, 0, 1);
    if (rc != SKYRME_OK) {
        delete b;
        return rc;
    }
    *out = b;
    return SKYRME_OK;
}

skyrme_status skyrme_batch_step(skyrme_batch *b, int nsteps, void *stream)
{
    if (!b || nsteps < 0) return SKYRME_EINVAL;
    return batch_launch(b, nsteps, 0, static_cast<cudaStream_t>(stream));
}

skyrme_status skyrme_batch_set_tile(skyrme_batch *b, int tile)
{
    if (!b || tile < 0 || tile >= kNumTiles) return SKYRME_EINVAL;
    return upload_table(b, tile, b->split);
}

skyrme_status skyrme_batch_set_split(skyrme_batch *b, int balanced)
{
    if (!b || (balanced != 0 && balanced != 1)) return SKYRME_EINVAL;
    return upload_table(b, b->tile, balanced);
}

skyrme_status skyrme_batch_split(const skyrme_batch *b, int *balanced)
{
    if (!b || !balanced) return SKYRME_EINVAL;
    *balanced = b->split;
    return SKYRME_OK;
}

skyrme_status skyrme_set_single_split(int policy)
{
    if (policy != SKYRME_SPLIT_AUTO && policy != SKYRME_SPLIT_BALANCED &&
        policy != SKYRME_SPLIT_LOCKSTEP)
        return SKYRME_EINVAL;
    g_single_split.store(policy);
    return SKYRME_OK;
}

int skyrme_single_split(void) { return g_single_split.load(); }

int skyrme_single_split_runs(const int n[3], int grid, int policy, int *runs, int cap,
                             int *chosen)
{
    if (!n || grid <= 0 || grid > kSplitMax || cap < 0 || (cap > 0 && !runs)) return -1;
    if (policy != SKYRME_SPLIT_AUTO && policy != SKYRME_SPLIT_BALANCED &&
        policy != SKYRME_SPLIT_LOCKSTEP)
        return -1;
    if (n[0] < 5 || n[1] < 5 || n[2] < 5) return -1;
    // the single lattice's 16 x 32 columns
    const int nyt = (n[1] - 4 + 15) / 16, nzt = (n[2] - 4 + 31) / 32, nix = n[0] - 4;
    const long long units = (long long)nyt * nzt * nix;
    if (units > 0x7fffffffLL) return -1;
    grid = (int)std::min<long long>(grid, units);
    CtaSplit sp;
    int ctas = grid;
    plan_single(units, nix, grid, policy, sp, &ctas);
    if (chosen) *chosen = sp.n == -2 ? SKYRME_SPLIT_LOCKSTEP : SKYRME_SPLIT_BALANCED;
    // walk every CTA's units as the step kernel does
    int count = 0;
    for (int b = 0; b < ctas; ++b) {
        const bool locked = sp.n == -2;
        const long long u0 = locked ? 0 : sp.n > 0 ? sp.start[b] : units * b / ctas;
        const long long u1 = locked ? lock_units(sp, b, nix) : sp.n > 0 ? sp.start[b + 1]
                                                                         : units * (b + 1) / ctas;
        for (long long us = u0; us < u1;) {
            int col, xs, xe;
            if (locked) {
                int xl, len;
                lock_run(sp, b, nix, (int)us, (int)u1, col, xl, len);
                xs = xl;
                xe = xl + len;
                us += len;
            } else {
                col = (int)(us / nix);
                const long long ue = std::min<long long>(u1, (long long)(col + 1) * nix);
                xs = (int)(us - (long long)col * nix);
                xe = (int)(ue - (long long)col * nix);
                us = ue;
            }
            if (count < cap) {
                runs[4 * count + 0] = b;
                runs[4 * count + 1] = col;
                runs[4 * count + 2] = xs;
                runs[4 * count + 3] = xe;
            }
            ++count;
        }
    }
    return count;
}

skyrme_status skyrme_batch_autotune(skyrme_batch *b, int trials, void *stream, int *best_tile,
                                    double *best_ms)
{
    if (!b || trials < 1) return SKYRME_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SKYRME_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SKYRME_ECUDA;
    }
    int best = -1, best_split = 1;
    float best_t = 0.f;
    skyrme_status rc = SKYRME_OK;
    // every tile shape, each with the even and the plane-balanced split
    for (int c = 0; c < 2 * kNumTiles && rc == SKYRME_OK; ++c) {
        const int t = c / 2, sp = c % 2;
        rc = upload_table(b, t, sp);
        if (rc != SKYRME_OK) break;
        if (sp && !b->split) continue;  // no balanced cover for this geometry
        rc = batch_launch(b, 1, 1, s);  // warm-up (dry: the flow does not advance)
        if (rc != SKYRME_OK) break;
        cudaEventRecord(e0, s);
        rc = batch_launch(b, trials, 1, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = SKYRME_ECUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= (float)trials;
        if (rc == SKYRME_OK && (best < 0 || ms < best_t)) {
            best = t;
            best_split = sp;
            best_t = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SKYRME_OK) return rc;
    rc = upload_table(b, best, best_split);
    if (rc != SKYRME_OK) return rc;
    if (best_tile) *best_tile = best;
    if (best_ms) *best_ms = best_t;
    return SKYRME_OK;
}

skyrme_status skyrme_batch_tile(const skyrme_batch *b, int *tile, int *ty, int *tz, int *grid)
{
    if (!b) return SKYRME_EINVAL;
    if (tile) *tile = b->tile;
    if (ty) *ty = kTiles[b->tile].ty;
    if (tz) *tz = kTiles[b->tile].tz;
    if (grid) *grid = b->grid;
    return SKYRME_OK;
}

skyrme_status skyrme_batch_graph_create(skyrme_batch *b, int nsteps, void *stream, skyrme_graph **out)
{
    if (!b || nsteps < 1 || !out) return SKYRME_EINVAL;
    return make_graph(b, nsteps, static_cast<cudaStream_t>(stream), out);
}

skyrme_status skyrme_batch_destroy(skyrme_batch *b)
{
    delete b;
    return SKYRME_OK;
}

}  // extern "C"

namespace skyrme {
skyrme_status batch_capture(skyrme_batch *b, int nsteps, cudaStream_t s)
{
    return batch_launch(b, nsteps, 0, s);
}
}  // namespace skyrme
