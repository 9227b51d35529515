// api.cu -- the extern "C" entry points of include/skyrme.h: argument
// validation, the scratch layout, kernel launches and report read-back.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>

#include "skyrme_device.cuh"
#include "skyrme_internal.h"

namespace skyrme {
int max_constituents();
int max_smoothing_half_width();
bool f32_fast_path_available(const skyrme_lattice &lat);
cudaError_t launch_wait_selftest(void *ctrl, unsigned long long limit_ns, cudaStream_t s);
cudaError_t launch_iterations_f32_fast(const skyrme_lattice &lat, const FlowArgs &a, int nsteps,
                                       cudaStream_t s);
int f32_fast_blocks(const skyrme_lattice &lat);
}  // namespace skyrme

using namespace skyrme;

struct skyrme_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int nsteps = 0;
};

static thread_local std::string g_last_cuda_error;

static skyrme_status cuda_fail(cudaError_t e, const char *what)
{
    g_last_cuda_error = std::string(what) + ": " + cudaGetErrorString(e);
    return SKYRME_ECUDA;
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t _e = (call);                         \
        if (_e != cudaSuccess) return cuda_fail(_e, what); \
    } while (0)

namespace skyrme {
bool lattice_ok(const skyrme_lattice *lat)
{
    if (!lat) return false;
    for (int i = 0; i < 3; ++i)
        if (lat->n[i] < 5 || lat->n[i] > 4096) return false;
    if (!(lat->h > 0.0) || !isfinite(lat->h) || !isfinite(lat->m) || lat->m < 0.0) return false;
    const double ext[4] = {lat->m_y, lat->m_z, lat->m_w, lat->c6};
    for (double v : ext)
        if (!isfinite(v) || v < 0.0) return false;
    if (lat->precision != 32 && lat->precision != 64) return false;
    const double sites = (double)lat->n[0] * lat->n[1] * lat->n[2];
    return sites < 4.0e9;
}

// Device buffers must live on the current device: the kernels are launched
// there, and a buffer of another GPU would be read across devices (a fault
// when peer access is off).  Host memory the device cannot address is
// rejected too.  Managed and mapped host memory pass.
skyrme_status on_current_device(const void *const *ptrs, int n)
{
    int dev = -1;
    CK(cudaGetDevice(&dev), "current device");
    for (int i = 0; i < n; ++i) {
        if (!ptrs[i]) continue;
        cudaPointerAttributes at;
        CK(cudaPointerGetAttributes(&at, ptrs[i]), "pointer attributes");
        if (at.type == cudaMemoryTypeUnregistered) return SKYRME_EINVAL;
        if (at.type == cudaMemoryTypeDevice && at.device != dev) return SKYRME_EINVAL;
    }
    return SKYRME_OK;
}
}  // namespace skyrme

static skyrme_status state_on_device(const skyrme_state *st)
{
    const void *p[5] = {st->phi[0], st->phi[1], st->vel[0], st->vel[1], st->scratch};
    return on_current_device(p, 5);
}

#define CKDEV(expr)                          \
    do {                                     \
        skyrme_status _r = (expr);           \
        if (_r != SKYRME_OK) return _r;      \
    } while (0)

static size_t site_bytes(const skyrme_lattice &lat) { return lat.precision == 64 ? 32 : 16; }

namespace skyrme {
ScratchLayout scratch_layout(const skyrme_lattice &lat)
{
    ScratchLayout L;
    const TileGeom g = tile_geometry(lat);
    int blocks = g.nblocks;
    if (lat.precision == 32) blocks = std::max(blocks, f32_fast_blocks(lat));
    blocks = std::max(blocks, 152 * 8);  // pointwise reductions of the seed pass
    L.max_blocks = blocks;
    L.ctrl_off = 0;
    L.step_off = kCtrlBytes;
    const size_t part = ((size_t)blocks * kPartialDoubles * sizeof(double) + 255) & ~(size_t)255;
    L.energy_off = L.step_off + part;
    L.total = L.energy_off + part;
    return L;
}
}  // namespace skyrme

static skyrme_status check_state(const skyrme_lattice *lat, const skyrme_state *st)
{
    if (!lattice_ok(lat) || !st) return SKYRME_EINVAL;
    const size_t align = site_bytes(*lat) == 32 ? 32 : 16;
    for (int i = 0; i < 2; ++i) {
        if (!st->phi[i] || !st->vel[i]) return SKYRME_EINVAL;
        if (((uintptr_t)st->phi[i] % align) || ((uintptr_t)st->vel[i] % align)) return SKYRME_EINVAL;
    }
    if (!st->scratch || ((uintptr_t)st->scratch % 256)) return SKYRME_EINVAL;
    if (st->scratch_bytes < scratch_layout(*lat).total) return SKYRME_ENOMEM;
    if (st->phi[0] == st->phi[1] || st->vel[0] == st->vel[1]) return SKYRME_EINVAL;
    return SKYRME_OK;
}

namespace skyrme {
bool state_ok_for_batch(const skyrme_lattice *lat, const skyrme_state *st)
{
    return check_state(lat, st) == SKYRME_OK;
}
skyrme_status batch_capture(skyrme_batch *b, int nsteps, cudaStream_t s);

// Capture nsteps batched iterations into a graph.
skyrme_status make_graph(skyrme_batch *b, int nsteps, cudaStream_t s, skyrme_graph **out)
{
    *out = nullptr;
    skyrme_graph *g = new skyrme_graph();
    g->nsteps = nsteps;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        delete g;
        return cuda_fail(e, "begin stream capture");
    }
    skyrme_status rc = batch_capture(b, nsteps, s);
    e = cudaStreamEndCapture(s, &g->graph);
    if (rc != SKYRME_OK || e != cudaSuccess) {
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return rc != SKYRME_OK ? rc : cuda_fail(e, "end stream capture");
    }
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g->graph);
        delete g;
        return cuda_fail(e, "instantiate graph");
    }
    // upload now, so that the first launch does not pay for it
    (void)cudaGraphUpload(g->exec, s);
    *out = g;
    return SKYRME_OK;
}
}  // namespace skyrme

static FlowArgs make_args(const skyrme_lattice &lat, const skyrme_state &st, double dt, int mode)
{
    const ScratchLayout L = scratch_layout(lat);
    FlowArgs a;
    for (int i = 0; i < 2; ++i) {
        a.phi[i] = st.phi[i];
        a.vel[i] = st.vel[i];
    }
    char *base = static_cast<char *>(st.scratch);
    a.ctrl = base + L.ctrl_off;
    a.step_parts = reinterpret_cast<double *>(base + L.step_off);
    a.energy_parts = reinterpret_cast<double *>(base + L.energy_off);
    for (int i = 0; i < 3; ++i) a.n[i] = lat.n[i];
    a.h = lat.h;
    a.m = lat.m;
    a.my = lat.m_y;
    a.mz = lat.m_z;
    a.mw = lat.m_w;
    a.c6 = lat.c6;
    a.dt = dt;
    a.mode = mode;
    return a;
}

static skyrme_status copy_ctrl(const skyrme_state &st, Ctrl *host, cudaStream_t s)
{
    CK(cudaMemcpyAsync(host, st.scratch, sizeof(Ctrl), cudaMemcpyDeviceToHost, s), "read control block");
    CK(cudaStreamSynchronize(s), "synchronise");
    return SKYRME_OK;
}

static void fill_report(const Ctrl &c, skyrme_report *r)
{
    r->E = c.last[0];
    r->E2 = c.last[1];
    r->E4 = c.last[2];
    r->E0 = c.last[3];
    r->B = c.last[4];
    r->virial = c.last[5];
    r->delta = c.last[6];
    r->rms_force = c.last[7];
    r->steps = c.steps;
    r->arrests = c.arrests;
    r->fixups = c.fixups;
    r->cur = c.cur;
    r->status = c.status;
    r->E6 = c.e6_last;
}

extern "C" {

int skyrme_abi_version(void) { return SKYRME_ABI_VERSION; }

const char *skyrme_status_string(int status)
{
    switch (status) {
    case SKYRME_OK: return "ok";
    case SKYRME_EINVAL: return "invalid argument";
    case SKYRME_ENOMEM: return "buffer too small";
    case SKYRME_ECUDA: return "CUDA error";
    case SKYRME_ENONFINITE: return "non-finite value detected";
    case SKYRME_ETIMEOUT: return "device wait timed out";
    case SKYRME_EUNSUPPORTED: return "unsupported";
    default: return "unknown status";
    }
}

const char *skyrme_last_cuda_error(void) { return g_last_cuda_error.c_str(); }

size_t skyrme_scratch_bytes(const skyrme_lattice *lat)
{
    if (!lattice_ok(lat)) return 0;
    return scratch_layout(*lat).total;
}

skyrme_status skyrme_init_field(const skyrme_lattice *lat, const skyrme_seed *seed,
                                skyrme_state *st, void *stream)
{
    skyrme_status rc = check_state(lat, st);
    if (rc != SKYRME_OK) return rc;
    if (!seed) return SKYRME_EINVAL;
    switch (seed->kind) {
    case SKYRME_SEED_VACUUM: break;
    case SKYRME_SEED_RATIONAL_MAP:
        if (seed->B < 1 || seed->B > 4 || !(seed->profile_scale > 0.0)) return SKYRME_EINVAL;
        break;
    case SKYRME_SEED_PRODUCT:
        if (seed->B < 1 || seed->B > max_constituents() || !seed->positions || !seed->quaternions ||
            !(seed->profile_scale > 0.0))
            return SKYRME_EINVAL;
        for (int k = 0; k < 4 * seed->B; ++k)
            if (!isfinite(seed->quaternions[k])) return SKYRME_EINVAL;
        for (int k = 0; k < 3 * seed->B; ++k)
            if (!isfinite(seed->positions[k])) return SKYRME_EINVAL;
        break;
    case SKYRME_SEED_NOISE:
        if (!(seed->radius > 0.0) || !(seed->sigma > 0.0)) return SKYRME_EINVAL;
        if (ceil(4.0 * seed->sigma / lat->h) > max_smoothing_half_width()) return SKYRME_EINVAL;
        break;
    default: return SKYRME_EINVAL;
    }
    CKDEV(state_on_device(st));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FlowArgs a = make_args(*lat, *st, 0.0, MODE_ARRESTED);
    CK(launch_reset_ctrl(a.ctrl, s), "reset control block");
    CK(launch_seed(*lat, *seed, a, s), "seed kernels");
    CK(launch_load_finish(*lat, a, s), "finish field");
    return SKYRME_OK;
}

skyrme_status skyrme_load_field(const skyrme_lattice *lat, skyrme_state *st, void *stream)
{
    skyrme_status rc = check_state(lat, st);
    if (rc != SKYRME_OK) return rc;
    CKDEV(state_on_device(st));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FlowArgs a = make_args(*lat, *st, 0.0, MODE_ARRESTED);
    CK(launch_reset_ctrl(a.ctrl, s), "reset control block");
    CK(launch_load_finish(*lat, a, s), "finish field");
    return SKYRME_OK;
}

// FP32 flows run on the streaming kernel (the standard model, the Section 7.8
// potentials and the sextic term)
static bool fp32_streaming(const skyrme_lattice &lat)
{
    return lat.precision == 32 && f32_fast_path_available(lat);
}

static skyrme_status launch_iterations(const skyrme_lattice &lat, const FlowArgs &a, int nsteps,
                                       cudaStream_t s)
{
    // FP32: the streaming kernel (the standard model, the Section 7.8
    // potentials, the sextic term); FP64: the tile kernels
    if (fp32_streaming(lat)) {
        CK(launch_iterations_f32_fast(lat, a, nsteps, s), "step and fix-up kernels (fp32)");
        return SKYRME_OK;
    }
    for (int k = 0; k < nsteps; ++k) {
        CK(launch_step(lat, a, s), "step kernel");
        // an x-slab's fix-up follows the decision over all slabs
        if (a.mode == SKYRME_ARRESTED && !a.slab_rec) CK(launch_fixup(lat, a, s), "fix-up kernel");
    }
    return SKYRME_OK;
}


// skyrme_flow_step's iterations.  A stream launch costs the GPU about 2.5 us
// and a kernel node of a graph about 0.8 us, and every iteration is two
// launches, so a long call captures kGraphChunk iterations once, on a stream
// of its own, and replays that graph on the caller's stream; the graph and
// the stream are released before the call returns (a graph still running is
// freed when it completes).  Short calls, and calls on a stream that is
// being captured, launch directly.
constexpr int kGraphChunk = 128;

static skyrme_status run_iterations(const skyrme_lattice &lat, const FlowArgs &a, int nsteps,
                                    cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (nsteps < 2 * kGraphChunk || cudaStreamIsCapturing(s, &cs) != cudaSuccess ||
        cs != cudaStreamCaptureStatusNone) {
        (void)cudaGetLastError();
        return launch_iterations(lat, a, nsteps, s);
    }
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "create capture stream");
    skyrme_status rc = SKYRME_OK;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = launch_iterations(lat, a, kGraphChunk, cap);
        const cudaError_t ee = cudaStreamEndCapture(cap, &graph);
        if (rc == SKYRME_OK && ee == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        else if (ee != cudaSuccess) e = ee;
    }
    if (rc == SKYRME_OK && e == cudaSuccess) {
        for (int k = 0; k + kGraphChunk <= nsteps && e == cudaSuccess; k += kGraphChunk)
            e = cudaGraphLaunch(exec, s);
        if (e == cudaSuccess) rc = launch_iterations(lat, a, nsteps % kGraphChunk, s);
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    if (rc != SKYRME_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "flow iterations as a graph");
    return SKYRME_OK;
}

static bool mode_ok(int mode)
{
    return mode == SKYRME_NEWTON || mode == SKYRME_ARRESTED || mode == SKYRME_GRADIENT;
}


skyrme_status skyrme_flow_step(const skyrme_lattice *lat, double dt, int nsteps, int mode,
                               skyrme_state *st, skyrme_report *report, void *stream)
{
    skyrme_status rc = check_state(lat, st);
    if (rc != SKYRME_OK) return rc;
    if (!(dt > 0.0) || !isfinite(dt) || nsteps < 0) return SKYRME_EINVAL;
    if (!mode_ok(mode)) return SKYRME_EINVAL;
    CKDEV(state_on_device(st));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FlowArgs a = make_args(*lat, *st, dt, mode);
    rc = run_iterations(*lat, a, nsteps, s);
    if (rc != SKYRME_OK) return rc;
    if (report) {
        Ctrl c;
        rc = copy_ctrl(*st, &c, s);
        if (rc != SKYRME_OK) return rc;
        fill_report(c, report);
        if (c.status) return static_cast<skyrme_status>(c.status);
    }
    return SKYRME_OK;
}

skyrme_status skyrme_flow_host(const skyrme_lattice *lat, double dt, int nsteps, int mode,
                               skyrme_state *st, const void *field_in, void *field_out,
                               skyrme_report *report, void *stream)
{
    skyrme_status rc = check_state(lat, st);
    if (rc != SKYRME_OK) return rc;
    if (!field_in || !field_out) return SKYRME_EINVAL;
    if (!(dt > 0.0) || !isfinite(dt) || nsteps < 0 || !mode_ok(mode)) return SKYRME_EINVAL;
    CKDEV(state_on_device(st));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)lat->n[0] * lat->n[1] * lat->n[2] * 4 * (lat->precision == 64 ? 8 : 4);
    // a pinned input is read by the load kernel itself over the host link (the
    // copy engine moves it no faster), so the upload and the load are one pass;
    // any other input is copied into phi[0] first
    const void *direct = nullptr;
    {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, field_in) == cudaSuccess && at.type == cudaMemoryTypeHost &&
            at.devicePointer && (reinterpret_cast<uintptr_t>(at.devicePointer) % 32) == 0)
            direct = at.devicePointer;
        (void)cudaGetLastError();
    }
    if (direct) {
        FlowArgs l = make_args(*lat, *st, 0.0, MODE_ARRESTED);
        CK(launch_reset_ctrl(l.ctrl, s), "reset control block");
        CK(launch_load_finish(*lat, l, s, direct), "load field from host");
    } else {
        CK(cudaMemcpyAsync(st->phi[0], field_in, bytes, cudaMemcpyHostToDevice, s), "upload field");
        rc = skyrme_load_field(lat, st, stream);
        if (rc != SKYRME_OK) return rc;
    }
    FlowArgs a = make_args(*lat, *st, dt, mode);
    rc = run_iterations(*lat, a, nsteps, s);
    if (rc != SKYRME_OK) return rc;
    // the load leaves cur = 0 and every iteration flips it
    const int cur = nsteps & 1;
    CK(cudaMemcpyAsync(field_out, st->phi[cur], bytes, cudaMemcpyDeviceToHost, s), "download field");
    Ctrl c;
    rc = copy_ctrl(*st, &c, s);
    if (rc != SKYRME_OK) return rc;
    if (report) fill_report(c, report);
    if (c.status) return static_cast<skyrme_status>(c.status);
    if (c.cur != cur) return SKYRME_ECUDA;  // not reached: a step that did not flip set a status
    return SKYRME_OK;
}

skyrme_status skyrme_step_densities(const skyrme_lattice *lat, double dt, int mode,
                                    skyrme_state *st, void *dens, skyrme_report *report,
                                    void *stream)
{
    skyrme_status rc = check_state(lat, st);
    if (rc != SKYRME_OK) return rc;
    if (!(dt > 0.0) || !isfinite(dt) || !mode_ok(mode)) return SKYRME_EINVAL;
    if (!dens || ((uintptr_t)dens % 16)) return SKYRME_EINVAL;
    if (!fp32_streaming(*lat) || lat->c6 != 0.0) return SKYRME_EUNSUPPORTED;
    CKDEV(state_on_device(st));
    {
        const void *p = dens;
        CKDEV(on_current_device(&p, 1));
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FlowArgs a = make_args(*lat, *st, dt, mode);
    a.dump = dens;
    rc = launch_iterations(*lat, a, 1, s);
    if (rc != SKYRME_OK) return rc;
    if (report) {
        Ctrl c;
        rc = copy_ctrl(*st, &c, s);
        if (rc != SKYRME_OK) return rc;
        fill_report(c, report);
        if (c.status) return static_cast<skyrme_status>(c.status);
    }
    return SKYRME_OK;
}

skyrme_status skyrme_slab_step(const skyrme_lattice *slab, double dt, int mode, skyrme_state *st,
                               double *record, void *stream)
{
    skyrme_status rc = check_state(slab, st);
    if (rc != SKYRME_OK) return rc;
    if (!(dt > 0.0) || !isfinite(dt) || !mode_ok(mode)) return SKYRME_EINVAL;
    if (!record || ((uintptr_t)record % 8)) return SKYRME_EINVAL;
    CKDEV(state_on_device(st));
    {
        const void *p = record;
        CKDEV(on_current_device(&p, 1));
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FlowArgs a = make_args(*slab, *st, dt, mode);
    a.slab_rec = record;
    return launch_iterations(*slab, a, 1, s);
}

skyrme_status skyrme_slab_finish(const skyrme_lattice *slab, double dt, int mode, skyrme_state *st,
                                 const double *records, int nslabs, void *stream)
{
    skyrme_status rc = check_state(slab, st);
    if (rc != SKYRME_OK) return rc;
    if (!(dt > 0.0) || !isfinite(dt) || !mode_ok(mode)) return SKYRME_EINVAL;
    if (!records || ((uintptr_t)records % 8) || nslabs < 1 || nslabs > 4096) return SKYRME_EINVAL;
    CKDEV(state_on_device(st));
    {
        const void *p = records;
        CKDEV(on_current_device(&p, 1));
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FlowArgs a = make_args(*slab, *st, dt, mode);
    CK(launch_slab_decide(a.ctrl, records, nslabs, slab->h * slab->h * slab->h, mode, s),
       "slab decision kernel");
    if (mode == SKYRME_ARRESTED) {
        if (fp32_streaming(*slab)) CK(launch_fixup_f32_fast(*slab, a, s), "fix-up kernel (fp32)");
        else CK(launch_fixup(*slab, a, s), "fix-up kernel");
    }
    return SKYRME_OK;
}

skyrme_status skyrme_graph_create(const skyrme_lattice *lat, double dt, int nsteps, int mode,
                                  skyrme_state *st, void *stream, skyrme_graph **out)
{
    if (!out) return SKYRME_EINVAL;
    *out = nullptr;
    skyrme_status rc = check_state(lat, st);
    if (rc != SKYRME_OK) return rc;
    if (!(dt > 0.0) || !isfinite(dt) || nsteps < 1 || !mode_ok(mode)) return SKYRME_EINVAL;
    CKDEV(state_on_device(st));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FlowArgs a = make_args(*lat, *st, dt, mode);
    skyrme_graph *g = new skyrme_graph();
    g->nsteps = nsteps;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        delete g;
        return cuda_fail(e, "begin stream capture");
    }
    rc = launch_iterations(*lat, a, nsteps, s);
    e = cudaStreamEndCapture(s, &g->graph);
    if (rc != SKYRME_OK || e != cudaSuccess) {
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return rc != SKYRME_OK ? rc : cuda_fail(e, "end stream capture");
    }
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g->graph);
        delete g;
        return cuda_fail(e, "instantiate graph");
    }
    // upload now, so that the first launch does not pay for it
    (void)cudaGraphUpload(g->exec, s);
    *out = g;
    return SKYRME_OK;
}

// The flow run to a tolerance: arm kernel, then WHILE { chunk iterations;
// check kernel } captured into the node's body through a second stream.
skyrme_status skyrme_graph_create_until(const skyrme_lattice *lat, double dt, int mode, double tol,
                                        long long max_steps, int chunk, skyrme_state *st,
                                        void *stream, skyrme_graph **out)
{
    if (!out) return SKYRME_EINVAL;
    *out = nullptr;
    skyrme_status rc = check_state(lat, st);
    if (rc != SKYRME_OK) return rc;
    if (!(dt > 0.0) || !isfinite(dt) || !mode_ok(mode) || !(tol >= 0.0) || !isfinite(tol) ||
        max_steps < 1 || chunk < 1)
        return SKYRME_EINVAL;
    CKDEV(state_on_device(st));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FlowArgs a = make_args(*lat, *st, dt, mode);
    cudaStream_t body = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&body, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "create body stream");
    skyrme_graph *g = new skyrme_graph();
    g->nsteps = 0;
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(body);
        delete g;
        return cuda_fail(e, "begin stream capture");
    }
    rc = [&]() -> skyrme_status {
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg = nullptr;
        CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg), "capture info");
        cudaGraphConditionalHandle h;
        CK(cudaGraphConditionalHandleCreate(&h, cg, 0, 0), "conditional handle");
        CK(launch_until_arm(a.ctrl, h, s), "arm kernel");
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, &deps, nullptr, &ndeps), "capture info");
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cn;
        CK(cudaGraphAddNode(&cn, cg, deps, nullptr, ndeps, &cp), "while node");
        CK(cudaStreamUpdateCaptureDependencies(s, &cn, nullptr, 1, cudaStreamSetCaptureDependencies),
           "capture dependencies");
        CK(cudaStreamBeginCaptureToGraph(body, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal),
           "begin body capture");
        skyrme_status brc = launch_iterations(*lat, a, chunk, body);
        if (brc == SKYRME_OK && launch_until_check(a.ctrl, h, tol, max_steps, body) != cudaSuccess)
            brc = cuda_fail(cudaGetLastError(), "check kernel");
        cudaGraph_t done = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(body, &done);
        if (brc != SKYRME_OK) return brc;
        CK(ee, "end body capture");
        return SKYRME_OK;
    }();
    e = cudaStreamEndCapture(s, &g->graph);
    cudaStreamDestroy(body);
    if (rc != SKYRME_OK || e != cudaSuccess) {
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return rc != SKYRME_OK ? rc : cuda_fail(e, "end stream capture");
    }
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g->graph);
        delete g;
        return cuda_fail(e, "instantiate graph");
    }
    // upload now, so that the first launch does not pay for it
    (void)cudaGraphUpload(g->exec, s);
    *out = g;
    return SKYRME_OK;
}

skyrme_status skyrme_graph_launch(skyrme_graph *g, void *stream)
{
    if (!g || !g->exec) return SKYRME_EINVAL;
    CK(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)), "launch graph");
    return SKYRME_OK;
}

skyrme_status skyrme_graph_destroy(skyrme_graph *g)
{
    if (!g) return SKYRME_OK;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return SKYRME_OK;
}

skyrme_status skyrme_selftest_wait(const skyrme_lattice *lat, skyrme_state *st,
                                   double limit_seconds, void *stream)
{
    skyrme_status rc = check_state(lat, st);
    if (rc != SKYRME_OK) return rc;
    if (!(limit_seconds > 0.0) || !(limit_seconds <= 10.0)) return SKYRME_EINVAL;
    CKDEV(state_on_device(st));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(launch_wait_selftest(st->scratch, (unsigned long long)(limit_seconds * 1e9), s),
       "wait self-test kernel");
    Ctrl c;
    rc = copy_ctrl(*st, &c, s);
    if (rc != SKYRME_OK) return rc;
    return static_cast<skyrme_status>(c.status);
}

skyrme_status skyrme_read_report(const skyrme_lattice *lat, const skyrme_state *st,
                                 skyrme_report *report, void *stream)
{
    skyrme_status rc = check_state(lat, st);
    if (rc != SKYRME_OK) return rc;
    if (!report) return SKYRME_EINVAL;
    CKDEV(state_on_device(st));
    Ctrl c;
    rc = copy_ctrl(*st, &c, static_cast<cudaStream_t>(stream));
    if (rc != SKYRME_OK) return rc;
    fill_report(c, report);
    return SKYRME_OK;
}

skyrme_status skyrme_energy(const skyrme_lattice *lat, skyrme_state *st, double out6[6],
                            void *stream)
{
    skyrme_status rc = check_state(lat, st);
    if (rc != SKYRME_OK) return rc;
    if (!out6) return SKYRME_EINVAL;
    CKDEV(state_on_device(st));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FlowArgs a = make_args(*lat, *st, 0.0, MODE_ARRESTED);
    CK(launch_energy(*lat, a, s), "energy kernel");
    Ctrl c;
    rc = copy_ctrl(*st, &c, s);
    if (rc != SKYRME_OK) return rc;
    for (int i = 0; i < 6; ++i) out6[i] = c.energy[i];
    if (!isfinite(out6[0]) || !isfinite(out6[4])) return SKYRME_ENONFINITE;
    return SKYRME_OK;
}

skyrme_status skyrme_baryon_number(const skyrme_lattice *lat, skyrme_state *st, double *B,
                                   void *stream)
{
    if (!B) return SKYRME_EINVAL;
    double e[6];
    skyrme_status rc = skyrme_energy(lat, st, e, stream);
    if (rc == SKYRME_OK) *B = e[4];
    return rc;
}

skyrme_status skyrme_virial(const skyrme_lattice *lat, skyrme_state *st, double *V, void *stream)
{
    if (!V) return SKYRME_EINVAL;
    double e[6];
    skyrme_status rc = skyrme_energy(lat, st, e, stream);
    if (rc == SKYRME_OK) *V = e[5];
    return rc;
}

skyrme_status skyrme_sextic_energy(const skyrme_lattice *lat, skyrme_state *st, double *E6,
                                   void *stream)
{
    if (!E6) return SKYRME_EINVAL;
    skyrme_status rc = check_state(lat, st);
    if (rc != SKYRME_OK) return rc;
    CKDEV(state_on_device(st));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FlowArgs a = make_args(*lat, *st, 0.0, MODE_ARRESTED);
    CK(launch_energy(*lat, a, s), "energy kernel");
    Ctrl c;
    rc = copy_ctrl(*st, &c, s);
    if (rc != SKYRME_OK) return rc;
    *E6 = c.e6_energy;
    return isfinite(*E6) ? SKYRME_OK : SKYRME_ENONFINITE;
}

skyrme_status skyrme_observables(const skyrme_lattice *lat, skyrme_state *st,
                                 skyrme_observables_t *out, void *stream)
{
    skyrme_status rc = check_state(lat, st);
    if (rc != SKYRME_OK) return rc;
    if (!out) return SKYRME_EINVAL;
    // Section 5 gives the currents and the stress tensor of the standard model
    if (lattice_extended(*lat)) return SKYRME_EUNSUPPORTED;
    const ScratchLayout L = scratch_layout(*lat);
    if (L.total - L.energy_off < observables_parts_bytes()) return SKYRME_ENOMEM;
    CKDEV(state_on_device(st));
    FlowArgs a = make_args(*lat, *st, 0.0, MODE_ARRESTED);
    return compute_observables(*lat, a, out, static_cast<cudaStream_t>(stream));
}

skyrme_status skyrme_forces(const skyrme_lattice *lat, skyrme_state *st, void *force, void *dens,
                            void *stream)
{
    skyrme_status rc = check_state(lat, st);
    if (rc != SKYRME_OK) return rc;
    const size_t align = site_bytes(*lat);
    if (((uintptr_t)force % align) || ((uintptr_t)dens % align)) return SKYRME_EINVAL;
    CKDEV(state_on_device(st));
    {
        const void *p[2] = {force, dens};
        CKDEV(on_current_device(p, 2));
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FlowArgs a = make_args(*lat, *st, 0.0, MODE_ARRESTED);
    const size_t bytes = (size_t)lat->n[0] * lat->n[1] * lat->n[2] * site_bytes(*lat);
    if (force) CK(cudaMemsetAsync(force, 0, bytes, s), "clear force buffer");
    if (dens) CK(cudaMemsetAsync(dens, 0, bytes, s), "clear density buffer");
    CK(launch_forces(*lat, a, force, dens, s), "force kernel");
    return SKYRME_OK;
}

size_t skyrme_render_volume_bytes(const skyrme_lattice *lat)
{
    if (!lattice_ok(lat)) return 0;
    return (size_t)lat->n[0] * lat->n[1] * lat->n[2] * 4 * sizeof(double);
}

skyrme_status skyrme_render_volume(const skyrme_lattice *lat, skyrme_state *st, void *vol,
                                   size_t vol_bytes, void *stream)
{
    skyrme_status rc = check_state(lat, st);
    if (rc != SKYRME_OK) return rc;
    if (!vol || ((uintptr_t)vol % 32)) return SKYRME_EINVAL;
    if (vol_bytes < skyrme_render_volume_bytes(lat)) return SKYRME_ENOMEM;
    CKDEV(state_on_device(st));
    CKDEV(on_current_device(&vol, 1));
    const ScratchLayout L = scratch_layout(*lat);
    FlowArgs a = make_args(*lat, *st, 0.0, MODE_ARRESTED);
    void *bmax = static_cast<char *>(st->scratch) + L.energy_off;
    CK(launch_render_volume(*lat, a, vol, bmax, static_cast<cudaStream_t>(stream)), "render volume");
    return SKYRME_OK;
}

skyrme_status skyrme_render_rays(const int n[3], const void *vol,
                                 const skyrme_render_params *params, float *rgba, void *stream)
{
    if (!n || !params || !vol || !rgba) return SKYRME_EINVAL;
    if (((uintptr_t)vol % 32) || ((uintptr_t)rgba % 16)) return SKYRME_EINVAL;
    for (int i = 0; i < 3; ++i)
        if (n[i] < 2 || n[i] > (1 << 20)) return SKYRME_EINVAL;
    if (!render_params_valid(*params)) return SKYRME_EINVAL;
    {
        const void *p[2] = {vol, rgba};
        CKDEV(on_current_device(p, 2));
    }
    CK(launch_render_rays(n, vol, *params, rgba, static_cast<cudaStream_t>(stream)), "render rays");
    return SKYRME_OK;
}

skyrme_status skyrme_render(const skyrme_lattice *lat, skyrme_state *st,
                            const skyrme_render_params *params, void *work, size_t work_bytes,
                            float *rgba, void *stream)
{
    skyrme_status rc = check_state(lat, st);
    if (rc != SKYRME_OK) return rc;
    if (!params || !render_params_valid(*params) || !rgba || ((uintptr_t)rgba % 16))
        return SKYRME_EINVAL;
    rc = skyrme_render_volume(lat, st, work, work_bytes, stream);
    if (rc != SKYRME_OK) return rc;
    return skyrme_render_rays(lat->n, work, params, rgba, stream);
}

}  // extern "C"
