// skyrme_internal.h -- host-side declarations shared by the library's
// translation units (launchers and the scratch layout).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "skyrme.h"

namespace skyrme {

// Scratch layout: [control block 512 B][step partials][energy partials]
struct ScratchLayout {
    size_t ctrl_off = 0;
    size_t step_off = 0;
    size_t energy_off = 0;
    size_t total = 0;
    int max_blocks = 0;
};

// Launch geometry of a lattice for the generic tile kernels.
struct TileGeom {
    dim3 grid;
    dim3 block;
    int nblocks;
    size_t smem;
    int tz;  // z extent of the tile: 32, or 16 where that pads the lattice less
};

TileGeom tile_geometry(const skyrme_lattice &lat);
ScratchLayout scratch_layout(const skyrme_lattice &lat);

struct FlowArgs {
    void *phi[2];
    void *vel[2];
    void *ctrl;
    double *step_parts;
    double *energy_parts;
    int n[3];
    double h, m, dt;
    double my, mz, mw, c6;  // Section 7.8 extension coefficients
    int mode;
    // x-slab of a larger lattice: the step writes its 8-double record here and
    // leaves the arrest decision to launch_slab_decide (null: a whole lattice)
    double *slab_rec = nullptr;
    // FP32 streaming step only: per-site densities the step summed (float4
    // per site, null: none)
    void *dump = nullptr;
};

// A lattice with any Section 7.8 extension term switched on.
inline bool lattice_extended(const skyrme_lattice &lat)
{
    return lat.m_y != 0.0 || lat.m_z != 0.0 || lat.m_w != 0.0 || lat.c6 != 0.0;
}

// A lattice with a Section 7.8 potential switched on (m_y, m_z or m_w).
inline bool lattice_potentials(const skyrme_lattice &lat)
{
    return lat.m_y != 0.0 || lat.m_z != 0.0 || lat.m_w != 0.0;
}

// Argument checks shared by the entry points (api.cu): lattice sizes, spacing
// and coefficients; every non-null pointer on the current device.
bool lattice_ok(const skyrme_lattice *lat);
skyrme_status on_current_device(const void *const *ptrs, int n);

// Kernels (asynchronous, return the launch error)
cudaError_t launch_step(const skyrme_lattice &lat, const FlowArgs &a, cudaStream_t s);
cudaError_t launch_fixup(const skyrme_lattice &lat, const FlowArgs &a, cudaStream_t s);
cudaError_t launch_energy(const skyrme_lattice &lat, const FlowArgs &a, cudaStream_t s);
cudaError_t launch_forces(const skyrme_lattice &lat, const FlowArgs &a, void *force, void *dens,
                          cudaStream_t s);
// src (nullable): a device-accessible copy of the field to read instead of phi[0]
cudaError_t launch_load_finish(const skyrme_lattice &lat, const FlowArgs &a, cudaStream_t s,
                               const void *src = nullptr);
cudaError_t launch_reset_ctrl(void *ctrl, cudaStream_t s);
// Sum nslabs slab records (8 doubles each, slab order) and run the lattice's
// end-of-step bookkeeping: arrest decision, predictor, fix flag, buffer flip.
cudaError_t launch_slab_decide(void *ctrl, const double *records, int nslabs, double h3, int mode,
                               cudaStream_t s);
// The FP32 streaming path's arrest fix-up (the whole-lattice flow's own).
cudaError_t launch_fixup_f32_fast(const skyrme_lattice &lat, const FlowArgs &a, cudaStream_t s);
cudaError_t launch_until_arm(void *ctrl, unsigned long long handle, cudaStream_t s);
cudaError_t launch_until_check(void *ctrl, unsigned long long handle, double tol,
                               long long max_steps, cudaStream_t s);

// Section 5 observables (observables.cu)
skyrme_status compute_observables(const skyrme_lattice &lat, const FlowArgs &a,
                                  skyrme_observables_t *out, cudaStream_t s);
size_t observables_parts_bytes();

// Volume render of the baryon density (render.cu)
bool render_params_valid(const skyrme_render_params &p);
cudaError_t launch_render_volume(const skyrme_lattice &lat, const FlowArgs &a, void *vol,
                                 void *bmax_scratch, cudaStream_t s);
cudaError_t launch_render_rays(const int n[3], const void *vol, const skyrme_render_params &p,
                               float *rgba, cudaStream_t s);

// Seeds (init_fields.cu)
cudaError_t launch_seed(const skyrme_lattice &lat, const skyrme_seed &seed, const FlowArgs &a,
                        cudaStream_t s);

}  // namespace skyrme
