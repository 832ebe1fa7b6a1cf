// md_api.cu -- the C ABI of libmd (declared in include/md.h): handle life cycle, device
// layout, CUDA-graph capture of the time step, state transfer and getters.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <vector>

#include "md_internal.h"

#define MD_ABI_VERSION 7

namespace {

thread_local std::string g_init_error;

// device-side state transfer between the caller's AoS order and the slot order; the
// positions live in one of two buffers (d0, d1), chosen by the buffer counter st->ph.
// diff (may be NULL) is set when any value differs bit for bit from the one it replaces.
__global__ void k_state_in(const double *stage, double *d0, double *d1, const DevStatus *st, const int32_t *orig,
                           int slot_off, int n, size_t S, int32_t *diff)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double *dst = (st->ph & 1) ? d1 : d0;
    int s = slot_off + i;
    int o = orig[s];
    bool same = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double v = stage[3 * (size_t)o + k];
        same &= __double_as_longlong(v) == __double_as_longlong(dst[k * S + s]);
        dst[k * S + s] = v;
    }
    if (diff && !same) *diff = 1;
}

// md_set_state: the drift the last force pass made is kept when no velocity changed
__global__ void k_keep_drift(int32_t *drift_ok, const int32_t *vdiff)
{
    *drift_ok = *vdiff == 0 ? 1 : 0;
}

// md_step's checkpoint (recovery from a list overflow): every replica's positions and
// velocities in caller order (replica r from 3 real_off), from the state buffer
__global__ void k_ckpt_save(DevArgs a, double *cx, double *cv)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.S) return;
    const RepDev &R = a.rep[a.tile_rep[s / MD_TILE]];
    if (s - R.slot_off >= R.n_atoms) return;
    const size_t S = a.S, o = 3 * ((size_t)R.real_off + a.orig[s]);
    const double *x = a.xs[a.st->ph & 1];
#pragma unroll
    for (int k = 0; k < 3; ++k) { cx[o + k] = x[k * S + s]; cv[o + k] = a.v[k * S + s]; }
}

// the checkpoint back into the current slot order, positions into both buffers
__global__ void k_ckpt_restore(DevArgs a, const double *cx, const double *cv)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.S) return;
    const RepDev &R = a.rep[a.tile_rep[s / MD_TILE]];
    if (s - R.slot_off >= R.n_atoms) return;
    const size_t S = a.S, o = 3 * ((size_t)R.real_off + a.orig[s]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        a.xs[0][k * S + s] = cx[o + k];
        a.xs[1][k * S + s] = cx[o + k];
        a.v[k * S + s] = cv[o + k];
    }
}

// the per-atom virial of replica r into caller order, 6 per atom
__global__ void k_vir_out(const double *vir, double *stage, const int32_t *orig, int slot_off, int n, size_t S)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int s = slot_off + i;
    int o = orig[s];
#pragma unroll
    for (int k = 0; k < 6; ++k) stage[6 * (size_t)o + k] = vir[k * S + s];
}

__global__ void k_state_out(const double *s0, const double *s1, const DevStatus *st, double *stage,
                            const int32_t *orig, int slot_off, int n, size_t S)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *src = (st->ph & 1) ? s1 : s0;
    int s = slot_off + i;
    int o = orig[s];
#pragma unroll
    for (int k = 0; k < 3; ++k) stage[3 * (size_t)o + k] = src[k * S + s];
}

}  // namespace

// small device-to-host readbacks land in pinned memory (a copy into pageable memory goes
// through a driver bounce buffer and costs more than the copy itself)
struct HostPin {
    DevStatus st{};
    RepEnergy E;
    RepState rs;
    int32_t flag, verlet;
    int32_t need_changed[2];   // md_set_state: DevStatus any_rebuild, changed
    int32_t one;               // 1, the source of a device flag set from the host
};

struct md_handle {
    cudaStream_t stream = nullptr;       // caller's stream
    cudaStream_t cap = nullptr;          // private stream used only for graph capture
    cudaStream_t cap2 = nullptr;         // second capture stream: k_morse_mixed beside k_density
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaStream_t xfer = nullptr;         // md_set_state: the velocities' upload beside the list test
    cudaEvent_t xev0 = nullptr, xev1 = nullptr;
    int32_t *vdiff = nullptr;            // md_set_state: k_state_in's velocity comparison
    md_options opt{};
    md_params pot_h{};
    PotDev pot{};
    LaunchCfg cfg{1, 128, 0};
    DevArgs a{};
    std::vector<RepDev> rep;
    std::vector<int32_t> c_orig;          // indenter slot -> caller indenter id (within replica)
    int n_rep = 0;
    int64_t n_cr = 0, n_c = 0;
    Cf64 *tab64 = nullptr;
    float4 *tab32 = nullptr;
    double *stage = nullptr;              // 6 * max replica atoms doubles (x, then v)
    std::vector<void *> allocs;
    // step graphs: exec1 / execU one / `unroll` steps after a step (mixed: drift made), execE
    // the same single step with the energies (the last step of an md_step call); execF /
    // execFE mixed precision's first step when no drift is known to be ready (DEC_AUTO: it
    // runs k_verlet1 unless the device's flag says one is), without / with the energies
    cudaGraphExec_t exec1 = nullptr, execU = nullptr, execE = nullptr;
    cudaGraphExec_t execF = nullptr, execFE = nullptr;
    // md_step_io's last step (captured on first use): execE / execFE with an external event,
    // xready, recorded once the step's Task 3 has made x(t + dt); [0] when a drift is known to
    // be ready or in FP64, [1] mixed precision's first step that reads the drift flag (DEC_AUTO)
    cudaGraphExec_t execIO[2] = {nullptr, nullptr};
    cudaEvent_t xready = nullptr;
    bool drift = false;   // mixed: the last force kernel made the next step's Task 3 (mirrors drift_ok)
    HostPin *hp = nullptr;
    int unroll = 1;
    bool forces_valid = false;
    bool energies_valid = false;   // the energy sums belong to the current state
    std::vector<cudaEvent_t> ev;
    std::string err;
    // md_step's checkpoint (allocated on first use): positions and velocities of all replicas
    // in caller order, the per-replica and global device state
    double *ck_x = nullptr, *ck_v = nullptr;
    RepState *ck_rs = nullptr;
    DevStatus *ck_st = nullptr;
    int32_t last_max_cnt = 0, last_max_cntc = 0;   // list maxima of the last status read
};

namespace {

int fail(md_t *h, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else g_init_error = buf;
    return code;
}

#define CU(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(h, MD_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

template <class T>
int dalloc(md_t *h, T **p, size_t n)
{
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
    if (e != cudaSuccess) return fail(h, MD_ERR_CUDA, "cudaMalloc(%zu bytes): %s", n * sizeof(T), cudaGetErrorString(e));
    h->allocs.push_back(*p);
    e = cudaMemset(*p, 0, n * sizeof(T));
    if (e != cudaSuccess) return fail(h, MD_ERR_CUDA, "cudaMemset: %s", cudaGetErrorString(e));
    return MD_OK;
}

int cu_check(md_t *h, cudaError_t e, const char *what)
{
    if (e != cudaSuccess) return fail(h, MD_ERR_CUDA, "%s failed: %s", what, cudaGetErrorString(e));
    return MD_OK;
}

int read_status(md_t *h, DevStatus *st)
{
    CU(cudaMemcpyAsync(&h->hp->st, h->a.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    *st = h->hp->st;
    h->last_max_cnt = st->max_cnt;
    h->last_max_cntc = st->max_cntc;
    return MD_OK;
}

int status_to_code(md_t *h, const DevStatus &st)
{
    if (st.err & MDE_LOST) return fail(h, MD_ERR_LOST_ATOM, "an atom left the cell-grid domain along a non-periodic axis or became NaN");
    if (st.err & MDE_OVERFLOW) return fail(h, MD_ERR_NBR_OVERFLOW, "Cr-Cr neighbour list overflow: %d > kmax %d", st.max_cnt, h->a.kmax);
    if (st.err & MDE_COVERFLOW) return fail(h, MD_ERR_NBR_OVERFLOW, "Cr-C neighbour list overflow: %d > kcmax %d", st.max_cntc, h->a.kcmax);
    if (st.err & MDE_SKIN) return fail(h, MD_ERR_SKIN_VIOLATION, "an atom moved more than skin/2 between fixed-interval rebuilds");
    if (st.err & MDE_SCHED) return fail(h, MD_ERR_STATE, "internal: a step found no drift from the last force kernel");
    if (st.err & MDE_LISTCHECK)
        return fail(h, MD_ERR_STATE, "list check after a build: %llu out of range, %llu over capacity, %llu wrong "
                    "direction, %llu beyond the radius, %llu missing, %llu one-way, %llu bad Cr-C, %llu inner not in Verlet",
                    st.chk[0], st.chk[1], st.chk[2], st.chk[3], st.chk[4], st.chk[5], st.chk[6], st.chk[7]);
    return MD_OK;
}

int clear_err(md_t *h)
{
    CU(cudaMemsetAsync(&h->a.st->err, 0, sizeof(int32_t), h->stream));
    return MD_OK;
}

// density and forces at the current positions (no integration); in mixed precision the force
// kernel also makes the next step's drift from this state, so that the next step needs no
// k_verlet1.  before_force: an event the force kernel waits for (it reads the velocities).
// energies = false leaves the energy sums stale (md_get_energy then evaluates them).
int forces_now(md_t *h, cudaStream_t s, cudaEvent_t before_force = nullptr, bool energies = true)
{
    const bool mixed = h->a.mixed != 0;
    const int en = energies || !mixed;   // the FP64 kernels always sum the energies
    if (mixed) CU(launch_drift_prep(h->a, s));
    CU(launch_density(h->a, h->pot, h->cfg, en, s));
    if (before_force) CU(cudaStreamWaitEvent(s, before_force, 0));
    CU(launch_force(h->a, h->pot, h->cfg, mixed ? 2 : 0, en, s));
    h->drift = mixed;
    if (en) CU(launch_reduce(h->a, h->cfg, s));
    h->energies_valid = en != 0;
    return MD_OK;
}

int rebuild_now(md_t *h)
{
    h->drift = false;   // k_build_done voids a drift made before the build
    CU(launch_decide(h->a, DEC_BUILD, 0, 0, h->stream));
    CU(launch_rebuild(h->a, h->stream));
    return MD_OK;
}

void destroy_graphs(md_t *h);

// replace a device array by a larger one (the contents are not kept: a list build follows).
// The step graphs hold the old pointer: they are destroyed here and rebuilt by the caller.
template <class T>
int regrow(md_t *h, T **p, size_t n)
{
    destroy_graphs(h);
    auto it = std::find(h->allocs.begin(), h->allocs.end(), (void *)*p);
    if (it != h->allocs.end()) {
        CU(cudaStreamSynchronize(h->stream));
        cudaFree(*p);
        h->allocs.erase(it);
    }
    return dalloc(h, p, n);
}

// list capacities grown past the counts of an overflowing build (by a quarter, at least
// 16 / 32 entries: lists that overflowed in a compressing film tend to keep growing);
// *grew = false when the status shows no overflow to grow for
int grow_lists(md_t *h, const DevStatus &st, bool *grew)
{
    int rc;
    *grew = false;
    if ((st.err & MDE_OVERFLOW) && st.max_cnt > h->a.kmax) {
        const int k = std::max(st.max_cnt + 16, st.max_cnt + st.max_cnt / 4);
        if ((rc = regrow(h, &h->a.nbr, (size_t)k * h->a.S))) return rc;
        const int kin = (k + h->cfg.tpa - 1) / h->cfg.tpa * h->cfg.tpa;
        if (h->a.mixed && (rc = regrow(h, &h->a.inner, (size_t)kin * h->a.S))) return rc;
        h->a.kmax = k;
        h->a.kinner = kin;
        *grew = true;
    }
    if ((st.err & MDE_COVERFLOW) && st.max_cntc > h->a.kcmax) {
        const int k = std::max(st.max_cntc + 32, st.max_cntc + st.max_cntc / 4);
        if ((rc = regrow(h, &h->a.nbrc, (size_t)k * h->a.S))) return rc;
        h->a.kcmax = k;
        *grew = true;
    }
    return MD_OK;
}

// grow the list capacities when the last build overflowed (outside md_step only)
int rebuild_growing(md_t *h)
{
    for (int attempt = 0; attempt < 4; ++attempt) {
        int rc = clear_err(h);
        if (rc) return rc;
        if ((rc = rebuild_now(h))) return rc;
        DevStatus st{};
        if ((rc = read_status(h, &st))) return rc;
        bool grew = false;
        if ((rc = grow_lists(h, st, &grew))) return rc;
        if (!grew) return status_to_code(h, st);
    }
    return fail(h, MD_ERR_NBR_OVERFLOW, "neighbour capacity kept growing");
}

void destroy_graphs(md_t *h)
{
    if (h->exec1) cudaGraphExecDestroy(h->exec1);
    if (h->execU) cudaGraphExecDestroy(h->execU);
    if (h->execE) cudaGraphExecDestroy(h->execE);
    if (h->execF) cudaGraphExecDestroy(h->execF);
    if (h->execFE) cudaGraphExecDestroy(h->execFE);
    for (auto &e : h->execIO)
        if (e) cudaGraphExecDestroy(e);
    h->exec1 = h->execU = h->execE = h->execF = h->execFE = h->execIO[0] = h->execIO[1] = nullptr;
}

// One graph of `nsteps` whole time steps: per step k_decide -> IF(rebuild) [list build] ->
// k_verlet1 -> k_density (beside k_morse) -> k_force; k_decide sets the step's conditional.
// In mixed precision the force kernel drifts the positions for the next step, and k_verlet1
// runs only after a rebuild (inside the IF), except in a first step with first_full set
// (after md_build_neighbors, md_set_state, ...): there k_decide (DEC_AUTO) sets a second
// conditional, IF(rebuild or no drift ready) [k_verlet1], from the device's drift flag.
// The energy sums (k_reduce) run once after the last step of an md_step call; with
// last_energy the graph's last force kernel writes the partials they add.  xev: recorded
// (an external event node) in every step once x(t + dt) is final, after Task 3 and any
// list build.
int capture(md_t *h, int nsteps, bool first_full, bool last_energy, cudaGraphExec_t *out,
            cudaEvent_t xev = nullptr)
{
    cudaGraph_t g = nullptr;
    CU(cudaGraphCreate(&g, 0));
    std::vector<cudaGraphNode_t> deps;
    const cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
    for (int k = 0; k < nsteps; ++k) {
        const int dm = !h->a.mixed ? DEC_FULL : (first_full && k == 0) ? DEC_AUTO : DEC_DRIFT;
        const int en = last_energy && k == nsteps - 1;
        cudaGraphConditionalHandle hc, hv = 0;
        CU(cudaGraphConditionalHandleCreate(&hc, g, 0, cudaGraphCondAssignDefault));
        if (dm == DEC_AUTO) CU(cudaGraphConditionalHandleCreate(&hv, g, 0, cudaGraphCondAssignDefault));
        CU(cudaStreamBeginCaptureToGraph(h->cap, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), mode));
        CU(launch_decide(h->a, dm, 1, hc, h->cap, hv));
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t *d = nullptr;
        size_t nd = 0;
        CU(cudaStreamGetCaptureInfo(h->cap, &cs, nullptr, nullptr, &d, nullptr, &nd));
        std::vector<cudaGraphNode_t> cur(d, d + nd);
        CU(cudaStreamEndCapture(h->cap, &g));
        alignas(cudaGraphNodeParams) unsigned char cpbuf[sizeof(cudaGraphNodeParams)];
        memset(cpbuf, 0, sizeof cpbuf);
        cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(cpbuf);
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = hc;
        cp.conditional.type = cudaGraphCondTypeIf;
        cp.conditional.size = 1;
        cudaGraphNode_t cn;
        CU(cudaGraphAddNode(&cn, g, cur.data(), nullptr, cur.size(), &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        CU(cudaStreamBeginCaptureToGraph(h->cap, body, nullptr, nullptr, 0, mode));
        CU(launch_rebuild(h->a, h->cap));
        if (dm == DEC_DRIFT) CU(launch_verlet1(h->a, h->cap));   // the drift was made before the build
        CU(cudaStreamEndCapture(h->cap, &body));
        if (dm == DEC_AUTO) {   // IF(rebuild or no drift ready) [k_verlet1]
            alignas(cudaGraphNodeParams) unsigned char vpbuf[sizeof(cudaGraphNodeParams)];
            memset(vpbuf, 0, sizeof vpbuf);
            cudaGraphNodeParams &vp = *reinterpret_cast<cudaGraphNodeParams *>(vpbuf);
            vp.type = cudaGraphNodeTypeConditional;
            vp.conditional.handle = hv;
            vp.conditional.type = cudaGraphCondTypeIf;
            vp.conditional.size = 1;
            cudaGraphNode_t cv;
            CU(cudaGraphAddNode(&cv, g, &cn, nullptr, 1, &vp));
            cudaGraph_t vbody = vp.conditional.phGraph_out[0];
            CU(cudaStreamBeginCaptureToGraph(h->cap, vbody, nullptr, nullptr, 0, mode));
            CU(launch_verlet1(h->a, h->cap));
            CU(cudaStreamEndCapture(h->cap, &vbody));
            cn = cv;
        }
        CU(cudaStreamBeginCaptureToGraph(h->cap, g, &cn, nullptr, 1, mode));
        if (dm == DEC_FULL) CU(launch_verlet1(h->a, h->cap));
        if (xev) CU(cudaEventRecordWithFlags(xev, h->cap, cudaEventRecordExternal));
        if (h->a.mixed) {   // the Morse sums need only this step's positions: beside k_density
            CU(cudaEventRecord(h->fork, h->cap));
            CU(cudaStreamWaitEvent(h->cap2, h->fork, 0));
            CU(launch_morse(h->a, h->pot, h->cap2));
            CU(cudaEventRecord(h->join, h->cap2));
            CU(launch_density(h->a, h->pot, h->cfg, en, h->cap));
            CU(cudaStreamWaitEvent(h->cap, h->join, 0));
            CU(launch_force_split(h->a, h->pot, h->cfg, 1, en, 0, h->cap));
        } else {
            CU(launch_density(h->a, h->pot, h->cfg, en, h->cap));
            CU(launch_force(h->a, h->pot, h->cfg, 1, en, h->cap));
        }
        CU(cudaStreamGetCaptureInfo(h->cap, &cs, nullptr, nullptr, &d, nullptr, &nd));
        deps.assign(d, d + nd);
        CU(cudaStreamEndCapture(h->cap, &g));
    }
    cudaError_t e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(h, MD_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    return MD_OK;
}

int build_graphs(md_t *h)
{
    destroy_graphs(h);
    if (!h->opt.use_graph) return MD_OK;
    int rc;
    if ((rc = capture(h, 1, false, false, &h->exec1))) return rc;
    if ((rc = capture(h, 1, false, true, &h->execE))) return rc;
    if (h->unroll > 1 && (rc = capture(h, h->unroll, false, false, &h->execU))) return rc;
    if (h->a.mixed) {
        if ((rc = capture(h, 1, true, false, &h->execF))) return rc;
        if ((rc = capture(h, 1, true, true, &h->execFE))) return rc;
    }
    return MD_OK;
}

// the per-step sequence with direct launches (no graph); the host reads the rebuild flag.
// energies: the force kernel writes the energy partials (needed by the step k_reduce follows)
int step_direct(md_t *h, cudaEvent_t *ev, bool *rebuilt, bool energies)
{
    cudaStream_t s = h->stream;
    if (ev) CU(cudaEventRecord(ev[0], s));
    CU(launch_decide(h->a, h->drift ? DEC_DRIFT : (h->a.mixed ? DEC_AUTO : DEC_FULL), 0, 0, s));
    if (ev) CU(cudaEventRecord(ev[1], s));
    CU(cudaMemcpyAsync(&h->hp->flag, &h->a.st->any_rebuild, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(&h->hp->verlet, &h->a.st->run_verlet, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    const int32_t flag = h->hp->flag, verlet = h->hp->verlet;
    if (ev) CU(cudaEventRecord(ev[2], s));
    if (flag) CU(launch_rebuild(h->a, s));
    if (ev) CU(cudaEventRecord(ev[3], s));
    if (verlet) CU(launch_verlet1(h->a, s));
    if (ev) CU(cudaEventRecord(ev[4], s));
    CU(launch_density(h->a, h->pot, h->cfg, energies ? 1 : 0, s));
    if (ev) CU(cudaEventRecord(ev[5], s));
    if (h->a.mixed) CU(launch_morse(h->a, h->pot, s));
    if (ev) CU(cudaEventRecord(ev[6], s));
    CU(launch_force_split(h->a, h->pot, h->cfg, 1, energies ? 1 : 0, 0, s));
    if (ev) CU(cudaEventRecord(ev[7], s));
    h->drift = h->a.mixed != 0;
    if (rebuilt) *rebuilt = flag != 0;
    return MD_OK;
}

int check_replica(md_t *h, int32_t r)
{
    if (!h) return MD_ERR_ARG;
    if (r < 0 || r >= h->n_rep) return fail(h, MD_ERR_ARG, "replica %d out of range [0, %d)", r, h->n_rep);
    return MD_OK;
}

}  // namespace

extern "C" {

int md_version(void) { return MD_ABI_VERSION; }

const char *md_last_error(const md_t *h)
{
    if (!h) return g_init_error.c_str();
    return h->err.c_str();
}

void md_free(md_t *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    destroy_graphs(h);
    for (auto e : h->ev) cudaEventDestroy(e);
    for (void *p : h->allocs) cudaFree(p);
    if (h->tab64) cudaFree(h->tab64);
    if (h->tab32) cudaFree(h->tab32);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->cap2) cudaStreamDestroy(h->cap2);
    if (h->fork) cudaEventDestroy(h->fork);
    if (h->join) cudaEventDestroy(h->join);
    if (h->xfer) { cudaStreamSynchronize(h->xfer); cudaStreamDestroy(h->xfer); }
    if (h->xev0) cudaEventDestroy(h->xev0);
    if (h->xev1) cudaEventDestroy(h->xev1);
    if (h->xready) cudaEventDestroy(h->xready);
    if (h->hp) cudaFreeHost(h->hp);
    delete h;
}

int md_init(const md_system *sys, int32_t n_replicas, const md_options *opt, void *cuda_stream, md_t **out)
{
    md_t *h = nullptr;
    if (out) *out = nullptr;
    if (!sys || !opt || !out || n_replicas < 1 || !opt->pot)
        return fail(nullptr, MD_ERR_ARG, "md_init: null argument or n_replicas < 1");
    if (opt->precision != MD_FP64 && opt->precision != MD_MIXED)
        return fail(nullptr, MD_ERR_ARG, "md_init: precision must be MD_FP64 or MD_MIXED");
    if (!(opt->skin >= 0.0) || opt->rebuild_every < 0 || !isfinite(opt->inner_skin))
        return fail(nullptr, MD_ERR_ARG, "md_init: skin must be >= 0, rebuild_every >= 0 and inner_skin finite");
    // threads per atom by default: the smallest of 1, 2, 4, 8 that puts at least 64Ki threads
    // on the atoms of all replicas (a small system's atoms then share their lists among
    // more lanes: 1 024 atoms run 1.4x, a 2 331-atom cube at the long cut-off 2.5x faster)
    int64_t n_all = 0;
    for (int32_t r = 0; r < n_replicas; ++r) n_all += sys[r].n_cr > 0 ? sys[r].n_cr : 0;
    int tpa = opt->tpa;
    if (!tpa) for (tpa = 1; tpa < 8 && n_all * tpa < 65536; tpa *= 2) {}
    int block = opt->block ? opt->block : 128;
    if (!(tpa == 1 || tpa == 2 || tpa == 4 || tpa == 8) || block < 32 || block > 256 || block % 32 ||
        MD_TILE % (block / tpa) != 0)
        return fail(nullptr, MD_ERR_ARG, "md_init: tpa must be 1, 2, 4 or 8 and block a multiple of 32 in [32, 256] with %d %% (block/tpa) == 0", MD_TILE);
    for (int32_t r = 0; r < n_replicas; ++r) {   // host-side checks before any device work
        const md_system &y = sys[r];
        if (y.n_cr < 1 || y.n_c < 0 || !y.x_cr || !y.v_cr || (y.n_c > 0 && !y.x_c) || !(y.dt > 0) || !(y.mass_cr > 0))
            return fail(nullptr, MD_ERR_ARG, "md_init: replica %d: need n_cr >= 1, positions, velocities, dt > 0, mass > 0", r);
    }
    h = new md_t();
    h->stream = (cudaStream_t)cuda_stream;
    h->opt = *opt;
    h->pot_h = *opt->pot;
    h->opt.pot = &h->pot_h;
    h->cfg.tpa = tpa;
    h->cfg.block = block;
    h->n_rep = n_replicas;
    int rc = MD_OK;
#define INIT_FAIL(code_expr)                    \
    do {                                        \
        int c_ = (code_expr);                   \
        if (c_) {                               \
            g_init_error = h->err;              \
            md_free(h);                         \
            return c_;                          \
        }                                       \
    } while (0)

#define CUI(call) INIT_FAIL(cu_check(h, (call), #call))
    char ebuf[256] = {0};
    rc = md_build_pot(&h->pot_h, &h->pot, &h->tab64, &h->tab32, ebuf, sizeof ebuf);
    if (rc) { h->err = ebuf; INIT_FAIL(rc); }

    const double cut = h->pot_h.rc + opt->skin, cutc = h->pot_h.rc_morse + opt->skin;
    // ---- layout
    int64_t slots = 0, cells = 0, ccells = 0, real = 0, cslots = 0, ncen = 0;
    size_t max_n = 1;
    h->rep.resize(n_replicas);
    for (int r = 0; r < n_replicas; ++r) {
        const md_system &y = sys[r];
        RepDev &R = h->rep[r];
        memset(&R, 0, sizeof R);
        if (y.n_cr < 1 || y.n_c < 0 || !y.x_cr || !y.v_cr || (y.n_c > 0 && !y.x_c) || !(y.dt > 0) || !(y.mass_cr > 0))
            INIT_FAIL(fail(h, MD_ERR_ARG, "replica %d: need n_cr >= 1, positions, velocities, dt > 0, mass > 0", r));
        for (int k = 0; k < 3; ++k) {
            R.lo[k] = y.box_lo[k]; R.hi[k] = y.box_hi[k]; R.L[k] = y.box_hi[k] - y.box_lo[k];
            R.per[k] = y.periodic[k] ? 1 : 0;
            if (!(R.L[k] > 0)) INIT_FAIL(fail(h, MD_ERR_ARG, "replica %d: box_hi must exceed box_lo", r));
            int n = (int)floor(R.L[k] / cut);
            if (n < 1) n = 1;
            if (R.per[k] && n < 3)
                INIT_FAIL(fail(h, MD_ERR_ARG, "replica %d: periodic axis %d is %.3f A, shorter than 3 cells of rc + skin = %.3f A", r, k, R.L[k], cut));
            if (n > (1 << MD_CELL_BITS) - 1)
                INIT_FAIL(fail(h, MD_ERR_ARG, "replica %d: axis %d needs %d cells, more than %d", r, k, n, (1 << MD_CELL_BITS) - 1));
            R.nc[k] = n;
            R.w[k] = R.L[k] / n;
            R.iw[k] = 1.0 / R.w[k];
            R.iL[k] = 1.0 / R.L[k];
            R.lo32[k] = (float)R.lo[k];
            R.L32[k] = (float)R.L[k];
            R.iL32[k] = (float)(1.0 / R.L[k]);
        }
        R.cell_off = (int32_t)cells;
        for (int k = 0; k < 3; ++k) R.nbk[k] = (R.nc[k] + 1) / 2;
        R.n_cells = 8 * R.nbk[0] * R.nbk[1] * R.nbk[2];
        cells += R.n_cells;
        R.slot_off = (int32_t)slots;
        R.n_atoms = y.n_cr;
        R.n_slots = (y.n_cr + MD_TILE - 1) / MD_TILE * MD_TILE;
        h->cfg.max_rep_slots = std::max(h->cfg.max_rep_slots, R.n_slots);
        R.real_off = (int32_t)real;
        slots += R.n_slots;
        real += y.n_cr;
        max_n = std::max(max_n, (size_t)y.n_cr);
        int nmob = 0;
        for (int i = 0; i < y.n_cr; ++i) nmob += (y.fixed && y.fixed[i]) ? 0 : 1;
        R.n_mobile = nmob;
        R.v_ind = y.v_indenter; R.dt = y.dt; R.mass = y.mass_cr; R.acc_per_f = MD_ACC / y.mass_cr;
        R.hk = 0.5 * R.dt * R.acc_per_f;
        for (int k = 0; k < 3; ++k) { R.cen_off[k] = (int32_t)ncen; ncen += R.nc[k]; }
        double ztop = -1e300;
        for (int i = 0; i < y.n_cr; ++i) ztop = std::max(ztop, y.x_cr[3 * i + 2]);
        R.z_surface0 = ztop;
        // indenter grid over the bounding box of x_c
        R.c_off = (int32_t)cslots;
        R.n_c = y.n_c;
        R.ccell_off = (int32_t)ccells;
        if (y.n_c > 0) {
            double bl[3], bh[3];
            for (int k = 0; k < 3; ++k) { bl[k] = 1e300; bh[k] = -1e300; }
            for (int c = 0; c < y.n_c; ++c)
                for (int k = 0; k < 3; ++k) { bl[k] = std::min(bl[k], y.x_c[3 * c + k]); bh[k] = std::max(bh[k], y.x_c[3 * c + k]); }
            R.zc_min0 = bl[2];
            for (int k = 0; k < 3; ++k) {
                double ext = (bh[k] - bl[k]) + 1e-6;
                int n = (int)floor(ext / cutc);
                if (n < 1) n = 1;
                if (n > 64) n = 64;   // one 64-bit cell set per axis in k_nbrc
                R.cg_n[k] = n; R.cg_w[k] = ext / n; R.cg_lo[k] = bl[k] - 0.5e-6;
                R.cg_ctr32[k] = (float)(R.cg_lo[k] + 0.5 * n * R.cg_w[k]);
                R.cg_half32[k] = (float)(0.5 * n * R.cg_w[k]);
                if (R.per[k] && !(R.L[k] > 2.0 * cutc))
                    INIT_FAIL(fail(h, MD_ERR_ARG, "replica %d: periodic length %.2f A on axis %d must exceed twice the Morse reach rc_morse + skin = %.2f A", r, R.L[k], k, cutc));
            }
            ccells += R.cg_n[0] * R.cg_n[1] * R.cg_n[2];
        }
        cslots += y.n_c;
    }
    if (slots >= (int64_t)1 << MD_J_BITS || cells >= (int64_t)1 << 31)
        INIT_FAIL(fail(h, MD_ERR_ARG, "too many atom slots (%lld) for the %d-bit neighbour entries", (long long)slots, MD_J_BITS));
    h->n_cr = real; h->n_c = cslots;
    const int S = (int)slots;
    DevArgs &a = h->a;
    a.S = S; a.n_rep = n_replicas; a.total_cells = (int)cells;
    a.kmax = opt->kmax > 0 ? opt->kmax : 80;
    a.kcmax = opt->kcmax > 0 ? opt->kcmax : 160;
    a.mixed = opt->precision == MD_MIXED;
    a.rebuild_every = opt->rebuild_every;
    a.debug = opt->debug_checks != 0;
    a.skin = opt->skin; a.cut = cut; a.cutc = cutc; a.cut2 = cut * cut; a.cutc2 = cutc * cutc;
    {
        // unit of the fixed-point cell-relative positions: the largest power of two
        // u = 2^-k A with (2 w_max + 2 skin + 4 A) / u < 2^30, so that every displacement
        // within a 27-cell stencil, and any drift before a rebuild, fits in 32 bits with a
        // margin of two (k = 26, u = 1.5e-8 A, for 5.6 A cells)
        double wmax = 0.0;
        for (const RepDev &R : h->rep)
            for (int k = 0; k < 3; ++k) wmax = std::max(wmax, R.w[k]);
        int qk = (int)floor(log2(1073741824.0 / (2.0 * wmax + 2.0 * opt->skin + 4.0)));
        qk = std::min(std::max(qk, 8), 30);
        const double qu = ldexp(1.0, -qk);
        a.qu = (float)qu;
        a.qinv = ldexp(1.0, qk);
        // cells of width wc = Wq u (w rounded to the unit), centres lo + (c + 1/2) wc; a pair
        // through a periodic face adds DLq = (L - nc wc) / u rounded (an error below u/2)
        for (RepDev &R : h->rep)
            for (int k = 0; k < 3; ++k) {
                R.Wq[k] = (int32_t)llround(R.w[k] / qu);
                R.wc[k] = R.Wq[k] * qu;
                R.w32[k] = (float)R.wc[k];
                R.DLq[k] = (int32_t)llround((R.L[k] - R.nc[k] * R.wc[k]) / qu);
                R.dL32[k] = (float)(R.DLq[k] * qu);
                R.pad32[k] = (float)(1e-4 + (R.nc[k] + 1) * fabs(R.w[k] - R.wc[k]));
            }
    }
    {
        // inner list: entries within rc + d (FP32 test); rebuilt once an atom has moved
        // (FP32 estimate, error < 1e-6 A) more than (d - 1e-4) / 2 since its last build, so
        // every pair then within rc was within rc + d - 1e-4 + 2e-6 at the build
        const double d = opt->inner_skin > 0 ? opt->inner_skin : MD_INNER_SKIN;
        if (opt->inner_skin < 0) {   // every step, radius rc
            a.rin2 = (float)(h->pot_h.rc * h->pot_h.rc);
            a.ithr2 = -1.0f;
        } else {
            const double rin = h->pot_h.rc + d, half = 0.5 * (d - 1e-4);
            a.rin2 = (float)(rin * rin);
            a.ithr2 = (float)(half * half);
        }
    }
    a.C = (int)cslots;
    a.max_blocks = S / (block / tpa) + 1;

    // ---- device memory
    RepDev *d_rep; RepState *d_rs; RepEnergy *d_en; DevStatus *d_st;
    int32_t *d_tile_rep, *d_cell_rep;
    INIT_FAIL(dalloc(h, &d_rep, n_replicas));
    INIT_FAIL(dalloc(h, &d_rs, n_replicas));
    INIT_FAIL(dalloc(h, &d_en, n_replicas));
    INIT_FAIL(dalloc(h, &d_st, 1));
    INIT_FAIL(dalloc(h, &d_tile_rep, S / MD_TILE));
    INIT_FAIL(dalloc(h, &d_cell_rep, cells));
    a.rep = d_rep; a.rs = d_rs; a.en = d_en; a.st = d_st; a.tile_rep = d_tile_rep; a.cell_rep = d_cell_rep;
    // two position buffers in mixed precision: the force epilogue drifts the positions it
    // has just used to the other one (one buffer in FP64, where k_verlet1 runs every step)
    INIT_FAIL(dalloc(h, &a.xs[0], 3 * (size_t)S));
    if (a.mixed) INIT_FAIL(dalloc(h, &a.xs[1], 3 * (size_t)S)); else a.xs[1] = a.xs[0];
    INIT_FAIL(dalloc(h, &a.v, 3 * (size_t)S));
    INIT_FAIL(dalloc(h, &a.vh, 3 * (size_t)S));
    INIT_FAIL(dalloc(h, &a.F, 3 * (size_t)S));
    INIT_FAIL(dalloc(h, &a.xb, 3 * (size_t)S));
    INIT_FAIL(dalloc(h, &a.p4[0], S));
    if (a.mixed) INIT_FAIL(dalloc(h, &a.p4[1], S)); else a.p4[1] = a.p4[0];
    INIT_FAIL(dalloc(h, &a.fm64, S));
    INIT_FAIL(dalloc(h, &a.fm32, S));
    INIT_FAIL(dalloc(h, &a.cellc, S));
    INIT_FAIL(dalloc(h, &a.orig, S));
    INIT_FAIL(dalloc(h, &a.fixed, S));
    INIT_FAIL(dalloc(h, &a.nbr, (size_t)a.kmax * S));
    INIT_FAIL(dalloc(h, &a.cnt, S));
    a.kinner = (a.kmax + tpa - 1) / tpa * tpa;
    INIT_FAIL(dalloc(h, &a.inner, a.mixed ? (size_t)a.kinner * S : 1));
    INIT_FAIL(dalloc(h, &a.icnt, S));
    INIT_FAIL(dalloc(h, &a.nbrc, (size_t)a.kcmax * S));
    INIT_FAIL(dalloc(h, &a.cntc, S));
    INIT_FAIL(dalloc(h, &a.cand, S));
    INIT_FAIL(dalloc(h, &a.near, S));
    INIT_FAIL(dalloc(h, &a.fmorse, S));
    if (a.mixed) INIT_FAIL(dalloc(h, &a.pin, S));
    if (a.mixed) INIT_FAIL(dalloc(h, &a.pb, S));
    INIT_FAIL(dalloc(h, &a.key, S));
    INIT_FAIL(dalloc(h, &a.perm, S));
    INIT_FAIL(dalloc(h, &a.cell_count, cells));
    INIT_FAIL(dalloc(h, &a.cell_start, cells));
    INIT_FAIL(dalloc(h, &a.cell_fill, cells));
    INIT_FAIL(dalloc(h, &a.scan_blk, cells / 1024 + 2));
    INIT_FAIL(dalloc(h, &a.sx, 3 * (size_t)S));
    INIT_FAIL(dalloc(h, &a.sv, 3 * (size_t)S));
    INIT_FAIL(dalloc(h, &a.sF, 3 * (size_t)S));
    INIT_FAIL(dalloc(h, &a.sorig, S));
    INIT_FAIL(dalloc(h, &a.sfixed, S));
    INIT_FAIL(dalloc(h, &a.part, 6 * (size_t)a.max_blocks));
    INIT_FAIL(dalloc(h, &a.rsum, 6 * (size_t)MD_RED_CHUNKS * n_replicas));
    double *d_xc0; int32_t *d_ccs, *d_ccc;
    float4 *d_xc32;
    INIT_FAIL(dalloc(h, &d_xc0, 3 * (size_t)(cslots > 0 ? cslots : 1)));
    INIT_FAIL(dalloc(h, &d_xc32, (size_t)(cslots > 0 ? cslots : 1)));
    a.xc32 = d_xc32;
    INIT_FAIL(dalloc(h, &d_ccs, ccells > 0 ? ccells : 1));
    INIT_FAIL(dalloc(h, &d_ccc, ccells > 0 ? ccells : 1));
    a.xc0 = d_xc0; a.ccell_start = d_ccs; a.ccell_count = d_ccc;
    INIT_FAIL(dalloc(h, &h->stage, 6 * max_n));
    INIT_FAIL(dalloc(h, &h->vdiff, 1));
    double *d_cen;
    INIT_FAIL(dalloc(h, &d_cen, ncen));
    a.cen = d_cen;
    {
        std::vector<double> hc(ncen);
        for (int r = 0; r < n_replicas; ++r)
            for (int k = 0; k < 3; ++k)
                for (int c = 0; c < h->rep[r].nc[k]; ++c)
                    hc[h->rep[r].cen_off[k] + c] = h->rep[r].lo[k] + (c + 0.5) * h->rep[r].wc[k];
        CUI(cudaMemcpy(d_cen, hc.data(), ncen * sizeof(double), cudaMemcpyHostToDevice));
    }

    // ---- host staging in slot order (initial slot order = caller order)
    {
        std::vector<double> hx(3 * (size_t)S, 0.0), hv(3 * (size_t)S, 0.0);
        std::vector<int32_t> horig(S, 0), htile(S / MD_TILE), hcell(cells);
        std::vector<uint8_t> hfix(S, 1);
        std::vector<double> hxc(3 * (size_t)(cslots > 0 ? cslots : 1), 0.0);
        std::vector<float4> hxc32((size_t)(cslots > 0 ? cslots : 1));
        std::vector<int32_t> hccs(ccells > 0 ? ccells : 1, 0), hccc(ccells > 0 ? ccells : 1, 0);
        h->c_orig.assign(cslots > 0 ? cslots : 1, 0);
        std::vector<RepState> hrs(n_replicas);
        for (int r = 0; r < n_replicas; ++r) {
            const md_system &y = sys[r];
            const RepDev &R = h->rep[r];
            for (int t = R.slot_off / MD_TILE; t < (R.slot_off + R.n_slots) / MD_TILE; ++t) htile[t] = r;
            for (int c = R.cell_off; c < R.cell_off + R.n_cells; ++c) hcell[c] = r;
            for (int i = 0; i < y.n_cr; ++i) {
                int s = R.slot_off + i;
                for (int k = 0; k < 3; ++k) {
                    hx[(size_t)k * S + s] = y.x_cr[3 * i + k];
                    hv[(size_t)k * S + s] = y.v_cr[3 * i + k];
                }
                horig[s] = i;
                hfix[s] = (y.fixed && y.fixed[i]) ? 1 : 0;
                if (hfix[s]) for (int k = 0; k < 3; ++k) hv[(size_t)k * S + s] = 0.0;
            }
            // indenter: counting sort by indenter cell (static, once)
            if (y.n_c > 0) {
                int nc3 = R.cg_n[0] * R.cg_n[1] * R.cg_n[2];
                std::vector<int32_t> key(y.n_c), cnt(nc3, 0), start(nc3 + 1, 0);
                for (int c = 0; c < y.n_c; ++c) {
                    int q[3];
                    for (int k = 0; k < 3; ++k) {
                        int t = (int)floor((y.x_c[3 * c + k] - R.cg_lo[k]) / R.cg_w[k]);
                        q[k] = std::min(std::max(t, 0), R.cg_n[k] - 1);
                    }
                    key[c] = (q[2] * R.cg_n[1] + q[1]) * R.cg_n[0] + q[0];
                    cnt[key[c]]++;
                }
                for (int k = 0; k < nc3; ++k) start[k + 1] = start[k] + cnt[k];
                std::vector<int32_t> fill(start.begin(), start.end() - 1);
                for (int c = 0; c < y.n_c; ++c) {
                    int t = R.c_off + fill[key[c]]++;
                    for (int k = 0; k < 3; ++k) hxc[(size_t)k * cslots + t] = y.x_c[3 * c + k];
                    hxc32[t] = make_float4((float)(y.x_c[3 * c] - R.cg_lo[0]), (float)(y.x_c[3 * c + 1] - R.cg_lo[1]),
                                           (float)(y.x_c[3 * c + 2] - R.cg_lo[2]), 0.0f);
                    h->c_orig[t] = c;
                }
                for (int k = 0; k < nc3; ++k) { hccs[R.ccell_off + k] = R.c_off + start[k]; hccc[R.ccell_off + k] = cnt[k]; }
            }
            hrs[r].z_ind = y.z_indenter0;
            hrs[r].z_build = y.z_indenter0;
        }
        CUI(cudaMemcpy(a.xs[0], hx.data(), hx.size() * sizeof(double), cudaMemcpyHostToDevice));   // ph = 0
        CUI(cudaMemcpy(a.v, hv.data(), hv.size() * sizeof(double), cudaMemcpyHostToDevice));
        CUI(cudaMemcpy(a.orig, horig.data(), S * sizeof(int32_t), cudaMemcpyHostToDevice));
        CUI(cudaMemcpy(a.fixed, hfix.data(), S, cudaMemcpyHostToDevice));
        CUI(cudaMemcpy(d_tile_rep, htile.data(), htile.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        CUI(cudaMemcpy(d_cell_rep, hcell.data(), hcell.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        CUI(cudaMemcpy(d_rep, h->rep.data(), n_replicas * sizeof(RepDev), cudaMemcpyHostToDevice));
        CUI(cudaMemcpy(d_rs, hrs.data(), n_replicas * sizeof(RepState), cudaMemcpyHostToDevice));
        if (cslots > 0) {
            CUI(cudaMemcpy(d_xc0, hxc.data(), 3 * (size_t)cslots * sizeof(double), cudaMemcpyHostToDevice));
            CUI(cudaMemcpy(d_xc32, hxc32.data(), (size_t)cslots * sizeof(float4), cudaMemcpyHostToDevice));
            CUI(cudaMemcpy(d_ccs, hccs.data(), ccells * sizeof(int32_t), cudaMemcpyHostToDevice));
            CUI(cudaMemcpy(d_ccc, hccc.data(), ccells * sizeof(int32_t), cudaMemcpyHostToDevice));
        }
    }
    CUI(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
    CUI(cudaStreamCreateWithFlags(&h->cap2, cudaStreamNonBlocking));
    CUI(cudaStreamCreateWithFlags(&h->xfer, cudaStreamNonBlocking));
    CUI(cudaEventCreateWithFlags(&h->xev0, cudaEventDisableTiming));
    CUI(cudaEventCreateWithFlags(&h->xev1, cudaEventDisableTiming));
    CUI(cudaEventCreateWithFlags(&h->xready, cudaEventDisableTiming));
    CUI(cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming));
    CUI(cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming));
    CUI(cudaHostAlloc((void **)&h->hp, sizeof(HostPin), cudaHostAllocDefault));
    *h->hp = HostPin{};
    h->hp->one = 1;
    h->ev.resize(8);
    for (auto &e : h->ev) CUI(cudaEventCreate(&e));
    h->unroll = 8;

    // ---- first list build and forces at t = 0
    INIT_FAIL(rebuild_growing(h));
    INIT_FAIL(forces_now(h, h->stream));
    {
        DevStatus st{};
        INIT_FAIL(read_status(h, &st));
        INIT_FAIL(status_to_code(h, st));
        st.rebuilds = 0; st.step = 0; st.since_build = 0;
        CUI(cudaMemcpy(a.st, &st, sizeof st, cudaMemcpyHostToDevice));
    }
    h->forces_valid = true;
    INIT_FAIL(build_graphs(h));
    CUI(cudaStreamSynchronize(h->stream));
    *out = h;
    return MD_OK;
#undef INIT_FAIL
#undef CUI
}

int md_build_neighbors(md_t *h)
{
    if (!h) return MD_ERR_ARG;
    size_t kmax0 = h->a.kmax, kc0 = h->a.kcmax;
    int rc = rebuild_growing(h);
    if (rc) return rc;
    if ((size_t)h->a.kmax != kmax0 || (size_t)h->a.kcmax != kc0) {
        if ((rc = build_graphs(h))) return rc;
    }
    CU(cudaStreamSynchronize(h->stream));
    return MD_OK;
}

int md_compute_forces(md_t *h)
{
    if (!h) return MD_ERR_ARG;
    int rc = forces_now(h, h->stream);
    if (rc) return rc;
    CU(cudaStreamSynchronize(h->stream));
    h->forces_valid = true;
    return MD_OK;
}

static int ensure_forces(md_t *h)
{
    if (h->forces_valid) return MD_OK;
    int rc = md_build_neighbors(h);
    if (rc) return rc;
    rc = forces_now(h, h->stream);
    if (rc) return rc;
    h->forces_valid = true;
    return MD_OK;
}

// md_step's checkpoint: every replica's positions and velocities in caller order and the
// device state words, queued on the stream (copies within the device)
static int save_checkpoint(md_t *h)
{
    if (!h->ck_x) {
        int rc;
        if ((rc = dalloc(h, &h->ck_x, 3 * (size_t)h->n_cr)) || (rc = dalloc(h, &h->ck_v, 3 * (size_t)h->n_cr)) ||
            (rc = dalloc(h, &h->ck_rs, h->n_rep)) || (rc = dalloc(h, &h->ck_st, 1)))
            return rc;
    }
    k_ckpt_save<<<(h->a.S + 255) / 256, 256, 0, h->stream>>>(h->a, h->ck_x, h->ck_v);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(h->ck_rs, h->a.rs, h->n_rep * sizeof(RepState), cudaMemcpyDeviceToDevice, h->stream));
    CU(cudaMemcpyAsync(h->ck_st, h->a.st, sizeof(DevStatus), cudaMemcpyDeviceToDevice, h->stream));
    return MD_OK;
}

// after a list overflow inside md_step: capacities grown past the overflowing counts, every
// replica back at the checkpoint, lists rebuilt there, forces and the step graphs renewed
static int restore_checkpoint(md_t *h, const DevStatus &st)
{
    bool grew = false;
    int rc = grow_lists(h, st, &grew);
    if (rc) return rc;
    k_ckpt_restore<<<(h->a.S + 255) / 256, 256, 0, h->stream>>>(h->a, h->ck_x, h->ck_v);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(h->a.rs, h->ck_rs, h->n_rep * sizeof(RepState), cudaMemcpyDeviceToDevice, h->stream));
    CU(cudaMemcpyAsync(h->a.st, h->ck_st, sizeof(DevStatus), cudaMemcpyDeviceToDevice, h->stream));
    // the FP32 copies of the positions belong to the abandoned steps: the build bins in FP64
    CU(cudaMemsetAsync(&h->a.st->pos4_ok, 0, sizeof(int32_t), h->stream));
    if ((rc = rebuild_growing(h))) return rc;
    if ((rc = forces_now(h, h->stream))) return rc;
    h->forces_valid = true;
    return build_graphs(h);
}

// io_last (graphs only): the last step is md_step_io's graph, which records h->xready once
// that step's positions are final
static int run_steps(md_t *h, int64_t n, bool io_last = false)
{
    int rc;
    if (h->opt.use_graph && h->exec1 && n > 0) {
        // steps 0 .. n-2 without the energies, step n-1 with them (k_reduce follows)
        int64_t k = 0;
        if (h->a.mixed && !h->drift) {
            CU(cudaGraphLaunch(n == 1 ? (io_last ? h->execIO[1] : h->execFE) : h->execF, h->stream));
            k = 1;
        }
        h->drift = h->a.mixed != 0;
        if (h->execU)
            for (; k + h->unroll <= n - 1; k += h->unroll) CU(cudaGraphLaunch(h->execU, h->stream));
        for (; k < n - 1; ++k) CU(cudaGraphLaunch(h->exec1, h->stream));
        if (k < n) CU(cudaGraphLaunch(io_last ? h->execIO[0] : h->execE, h->stream));
    } else {
        for (int64_t k = 0; k < n; ++k)
            if ((rc = step_direct(h, nullptr, nullptr, k == n - 1))) return rc;
    }
    if (n > 0) {
        CU(launch_reduce(h->a, h->cfg, h->stream));
        h->energies_valid = true;
    }
    return MD_OK;
}

// the longest list of the last build came within 1/8 of its capacity (8 entries at least):
// between builds the longest lists of a film grow by a few entries (thermal motion, an
// indenter's compression), so a build inside a short call overflows only from there
static bool near_capacity(const md_t *h)
{
    const auto near = [](int64_t m, int64_t k) { return m + std::max<int64_t>(8, k / 8) > k; };
    return near(h->last_max_cnt, h->a.kmax) || near(h->last_max_cntc, h->a.kcmax);
}

int md_step(md_t *h, int64_t n)
{
    if (!h) return MD_ERR_ARG;
    if (n < 0) return fail(h, MD_ERR_ARG, "md_step: n < 0");
    for (int attempt = 0;; ++attempt) {
        int rc = ensure_forces(h);
        if (rc) return rc;
        if ((rc = clear_err(h))) return rc;
        // a copy to come back to if a list build inside the call overflows: for calls long
        // enough to amortise it, or when the last build came near a capacity
        const bool ck = n > 0 && attempt < 8 && (n >= 16 || near_capacity(h));
        if (ck && (rc = save_checkpoint(h))) return rc;
        if ((rc = run_steps(h, n))) return rc;
        DevStatus st{};
        if ((rc = read_status(h, &st))) return rc;
        // after an overflowing build the lists miss pairs, so whatever else the rest of the
        // call raised (a lost atom, a skin violation) may be its consequence: go back and
        // redo it; an error of its own comes back in the redo and is reported then
        if (!ck || !(st.err & (MDE_OVERFLOW | MDE_COVERFLOW))) return status_to_code(h, st);
        if ((rc = restore_checkpoint(h, st))) return rc;   // then the n steps again
    }
}

int md_step_profiled(md_t *h, int64_t n, md_phase_times *out)
{
    if (!h || !out) return MD_ERR_ARG;
    int rc = ensure_forces(h);
    if (rc) return rc;
    if ((rc = clear_err(h))) return rc;
    memset(out, 0, sizeof *out);
    for (int64_t k = 0; k < n; ++k) {
        bool rebuilt = false;
        if ((rc = step_direct(h, h->ev.data(), &rebuilt, k == n - 1))) return rc;
        CU(cudaEventSynchronize(h->ev[7]));
        float ms[7];
        for (int p = 0; p < 7; ++p) CU(cudaEventElapsedTime(&ms[p], h->ev[p], h->ev[p + 1]));
        out->skin += ms[0];
        out->rebuild += ms[2];
        out->verlet1 += ms[3];
        out->density += ms[4];
        out->morse += ms[5];
        out->force += ms[6];
        out->steps += 1;
        out->rebuilds += rebuilt ? 1 : 0;
    }
    if (n > 0) {
        CU(cudaEventRecord(h->ev[0], h->stream));
        CU(launch_reduce(h->a, h->cfg, h->stream));
        CU(cudaEventRecord(h->ev[1], h->stream));
        CU(cudaEventSynchronize(h->ev[1]));
        float ms;
        CU(cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]));
        out->reduce += ms;
        h->energies_valid = true;
    }
    DevStatus st{};
    if ((rc = read_status(h, &st))) return rc;
    return status_to_code(h, st);
}

static void fill_energy(const md_t *h, int32_t r, md_energy *out);

int md_get_energy(md_t *h, int32_t r, md_energy *out)
{
    int rc = check_replica(h, r);
    if (rc) return rc;
    if (!out) return fail(h, MD_ERR_ARG, "md_get_energy: null output");
    if (!h->energies_valid) {   // a state set since the last sums: evaluate them now
        if ((rc = ensure_forces(h))) return rc;
        if (!h->energies_valid && (rc = forces_now(h, h->stream))) return rc;
    }
    CU(cudaMemcpyAsync(&h->hp->E, h->a.en + r, sizeof(RepEnergy), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(&h->hp->rs, h->a.rs + r, sizeof(RepState), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(&h->hp->st, h->a.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    fill_energy(h, r, out);
    return MD_OK;
}

// md_energy of replica r from the sums, replica state and status read into pinned memory
static void fill_energy(const md_t *h, int32_t r, md_energy *out)
{
    const RepEnergy E = h->hp->E;
    const RepState rs = h->hp->rs;
    const DevStatus st = h->hp->st;
    const RepDev &R = h->rep[r];
    out->embed = E.embed; out->pair = E.pair; out->mterm = E.mterm; out->morse = E.morse;
    out->kinetic = E.kinetic;
    out->potential = E.embed + E.pair + E.mterm + E.morse;
    out->total = out->potential + E.kinetic;
    out->temperature = R.n_mobile > 0 ? 2.0 * E.kinetic / (3.0 * MD_KB * R.n_mobile) : 0.0;
    out->load = E.load;
    out->z_indenter = rs.z_ind;
    out->depth = R.n_c > 0 ? R.z_surface0 - (R.zc_min0 + rs.z_ind) : 0.0;
    out->step = st.step;
    out->rebuilds = st.rebuilds;
}

// queue the gather of one per-atom array of replica r into caller order (stage half `half`
// of the staging buffer) and its copy to out3n, on stream s (default: the handle's); the
// caller synchronises
static int fetch_async(md_t *h, int32_t r, const double *s0, const double *s1, double *out3n, int half,
                       cudaStream_t s = nullptr)
{
    const RepDev &R = h->rep[r];
    int n = R.n_atoms;
    if (!s) s = h->stream;
    double *stage = h->stage + 3 * (size_t)n * half;
    k_state_out<<<(n + 255) / 256, 256, 0, s>>>(s0, s1, h->a.st, stage, h->a.orig, R.slot_off, n, h->a.S);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(out3n, stage, 3 * (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s));
    return MD_OK;
}

static int fetch(md_t *h, int32_t r, const double *s0, const double *s1, double *out3n)
{
    int rc = fetch_async(h, r, s0, s1, out3n, 0);
    if (rc) return rc;
    CU(cudaStreamSynchronize(h->stream));
    return MD_OK;
}

int md_get_forces(md_t *h, int32_t r, double *out3n)
{
    int rc = check_replica(h, r);
    if (rc) return rc;
    if (!out3n) return fail(h, MD_ERR_ARG, "md_get_forces: null output");
    return fetch(h, r, h->a.F, h->a.F, out3n);
}

int md_get_indenter_load(md_t *h, int32_t r, double *load_z, double *depth)
{
    md_energy e;
    int rc = md_get_energy(h, r, &e);
    if (rc) return rc;
    if (load_z) *load_z = e.load;
    if (depth) *depth = e.depth;
    return MD_OK;
}

int md_get_state(md_t *h, int32_t r, double *x3n, double *v3n, double *z_ind, int64_t *step)
{
    int rc = check_replica(h, r);
    if (rc) return rc;
    // both gathers and copies queued, one synchronisation: the gather of v runs while x is
    // on its way
    if (x3n && (rc = fetch_async(h, r, h->a.xs[0], h->a.xs[1], x3n, 0))) return rc;
    if (v3n && (rc = fetch_async(h, r, h->a.v, h->a.v, v3n, 1))) return rc;
    if (z_ind || step) {
        CU(cudaMemcpyAsync(&h->hp->rs, h->a.rs + r, sizeof(RepState), cudaMemcpyDeviceToHost, h->stream));
        CU(cudaMemcpyAsync(&h->hp->st, h->a.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream));
    }
    CU(cudaStreamSynchronize(h->stream));
    if (z_ind) *z_ind = h->hp->rs.z_ind;
    if (step) *step = h->hp->st.step;
    return MD_OK;
}

// page-locked host memory (the copy engine reads it after the call that queued the copy)
static bool host_pinned(const void *p)
{
    cudaPointerAttributes at;
    if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost;
}

// md_set_state; wait_v: return only once the velocities are read from v3n (the public
// call: the caller may write v3n when it returns); md_step_io synchronises later itself
static int set_state_impl(md_t *h, int32_t r, const double *x3n, const double *v3n, double z_ind, int64_t step,
                          bool wait_v)
{
    int rc = check_replica(h, r);
    if (rc) return rc;
    const RepDev &R = h->rep[r];
    int n = R.n_atoms;
    const bool had_forces = h->forces_valid;
    const bool had_drift = h->drift;
    h->drift = false;   // k_state_prep voids the drift made from the old state
    if (x3n) CU(cudaMemcpyAsync(h->stage, x3n, 3 * (size_t)n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    // The velocities go up on the transfer stream once the positions are up (one copy at a
    // time fills the link) and the work queued before this call is done; the list test,
    // the pair positions and the density, which do not read v, run meanwhile.  Every
    // reader of v below waits for xev1.
    CU(cudaEventRecord(h->xev0, h->stream));
    if (v3n) {
        double *st2 = h->stage + 3 * (size_t)n;
        CU(cudaStreamWaitEvent(h->xfer, h->xev0, 0));
        CU(cudaMemcpyAsync(st2, v3n, 3 * (size_t)n * sizeof(double), cudaMemcpyHostToDevice, h->xfer));
        CU(cudaMemsetAsync(h->vdiff, 0, sizeof(int32_t), h->xfer));
        k_state_in<<<(n + 255) / 256, 256, 0, h->xfer>>>(st2, h->a.v, h->a.v, h->a.st, h->a.orig, R.slot_off, n,
                                                         h->a.S, h->vdiff);
        CU(cudaGetLastError());
        CU(cudaEventRecord(h->xev1, h->xfer));
    }
    h->forces_valid = false;
    // The lists stay valid when the new state passes the rebuild test md_step applies
    // (max |x - x_build| and the indenter's travel against the skin): the positions, their
    // pos4 and both displacement tests come out of one pass, and the inner list is rebuilt
    // by the density pass if its own test fails.  Otherwise (or when positions leave their
    // periodic image, become NaN, ...) a full rebuild.
    CU(launch_state_set(h->a, r, R.slot_off, n, z_ind, (long long)step, x3n ? h->stage : nullptr, h->stream));
    static_assert(offsetof(DevStatus, changed) == offsetof(DevStatus, any_rebuild) + sizeof(int32_t), "layout");
    CU(cudaMemcpyAsync(h->hp->need_changed, &h->a.st->any_rebuild, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost,
                       h->stream));
    CU(cudaStreamSynchronize(h->stream));
    const int32_t need = h->hp->need_changed[0], changed = h->hp->need_changed[1];
    if (need) {   // the list build moves the velocities with the atoms
        if (v3n) CU(cudaStreamWaitEvent(h->stream, h->xev1, 0));
        return ensure_forces(h);
    }
    if (had_forces && !changed) {
        // the same positions and indenter displacement: the forces of the state hold (they
        // do not depend on the velocities), and md_get_energy sums the energies anew (the
        // kinetic term).  With the same velocities too, bit for bit, the next step's Task 3
        // that the last force pass made (mixed precision) holds as well: it is what
        // k_verlet1 would make again from the same x, v and F, so it is kept (k_state_prep
        // voided it; nothing else of it was touched).  The device sets its flag again when
        // k_state_in found every velocity the same, without a wait here: the host then
        // does not know, and the next step's graph (DEC_AUTO) reads the flag.  Otherwise
        // the next step makes its own drift from the velocities now set.
        if (v3n) CU(cudaStreamWaitEvent(h->stream, h->xev1, 0));
        if (had_drift) {
            if (v3n) {
                k_keep_drift<<<1, 1, 0, h->stream>>>(&h->a.st->drift_ok, h->vdiff);
                CU(cudaGetLastError());
            } else {
                CU(cudaMemcpyAsync(&h->a.st->drift_ok, &h->hp->one, sizeof(int32_t), cudaMemcpyHostToDevice,
                                   h->stream));
                h->drift = true;
            }
        }
        h->forces_valid = true;
        h->energies_valid = false;
        // a page-locked v3n is still being read by the copy engine when this returns: the
        // public call waits for it (a pageable one was copied before cudaMemcpyAsync returned)
        if (wait_v && v3n && host_pinned(v3n)) CU(cudaStreamSynchronize(h->xfer));
        return MD_OK;
    }
    int rc2;
    // the energy sums are left to md_get_energy: a caller that sets a state and steps on
    // reads those of the step
    if ((rc2 = forces_now(h, h->stream, v3n ? h->xev1 : nullptr, false))) return rc2;
    DevStatus st{};
    if ((rc2 = read_status(h, &st))) return rc2;
    if ((rc2 = status_to_code(h, st))) return rc2;
    h->forces_valid = true;
    return MD_OK;
}

int md_set_state(md_t *h, int32_t r, const double *x3n, const double *v3n, double z_ind, int64_t step)
{
    return set_state_impl(h, r, x3n, v3n, z_ind, step, true);
}

int md_step_io(md_t *h, int32_t r, const double *x3n, const double *v3n, double z_ind, int64_t step, int64_t n,
               double *x_out, double *v_out, md_energy *e_out)
{
    int rc = check_replica(h, r);
    if (rc) return rc;
    if (!x3n || !v3n || !x_out || !v_out || !e_out) return fail(h, MD_ERR_ARG, "md_step_io: null argument");
    if (n < 1) return fail(h, MD_ERR_ARG, "md_step_io: n < 1");
    if ((rc = set_state_impl(h, r, x3n, v3n, z_ind, step, false))) return rc;
    if ((rc = ensure_forces(h))) return rc;
    // direct launches: the calls in turn
    if (!h->opt.use_graph || !h->exec1) {
        if ((rc = md_step(h, n))) return rc;
        if ((rc = md_get_state(h, r, x_out, v_out, nullptr, nullptr))) return rc;
        return md_get_energy(h, r, e_out);
    }
    const int w = (n == 1 && h->a.mixed && !h->drift) ? 1 : 0;
    if (!h->execIO[w] && (rc = capture(h, 1, w == 1, true, &h->execIO[w], h->xready))) return rc;
    if ((rc = clear_err(h))) return rc;
    // md_step's checkpoint policy; after an overflowing build the checkpoint is restored and
    // md_step runs the n steps with its recovery
    const bool ck = n >= 16 || near_capacity(h);
    if (ck && (rc = save_checkpoint(h))) return rc;
    if ((rc = run_steps(h, n, true))) return rc;
    // x(t + n dt) is final once the last step's Task 3 (and list build) is done: its gather
    // and copy run on the transfer stream beside that step's density and force passes
    CU(cudaStreamWaitEvent(h->xfer, h->xready, 0));
    if ((rc = fetch_async(h, r, h->a.xs[0], h->a.xs[1], x_out, 0, h->xfer))) return rc;
    // v(t + n dt) and the sums after the force pass and k_reduce (queued by run_steps)
    if ((rc = fetch_async(h, r, h->a.v, h->a.v, v_out, 1))) return rc;
    CU(cudaMemcpyAsync(&h->hp->E, h->a.en + r, sizeof(RepEnergy), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(&h->hp->rs, h->a.rs + r, sizeof(RepState), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(&h->hp->st, h->a.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->xfer));
    CU(cudaStreamSynchronize(h->stream));
    const DevStatus st = h->hp->st;
    h->last_max_cnt = st.max_cnt;
    h->last_max_cntc = st.max_cntc;
    if (ck && (st.err & (MDE_OVERFLOW | MDE_COVERFLOW))) {
        if ((rc = restore_checkpoint(h, st))) return rc;
        if ((rc = md_step(h, n))) return rc;
        if ((rc = md_get_state(h, r, x_out, v_out, nullptr, nullptr))) return rc;
        return md_get_energy(h, r, e_out);
    }
    if ((rc = status_to_code(h, st))) return rc;
    fill_energy(h, r, e_out);
    return MD_OK;
}

int md_get_virial(md_t *h, int32_t r, double *out6n)
{
    int rc = check_replica(h, r);
    if (rc) return rc;
    if (!out6n) return fail(h, MD_ERR_ARG, "md_get_virial: null output");
    if ((rc = ensure_forces(h))) return rc;
    if (!h->a.vir && (rc = dalloc(h, &h->a.vir, 6 * (size_t)h->a.S))) return rc;
    // a force evaluation first: F'(rho), M'(P) and the inner list then belong to the current
    // slot order and positions whatever call came before (a list build permutes the slots)
    if ((rc = forces_now(h, h->stream))) return rc;
    CU(launch_virial(h->a, h->pot, h->cfg, h->stream));
    const RepDev &R = h->rep[r];
    const int n = R.n_atoms;
    k_vir_out<<<(n + 255) / 256, 256, 0, h->stream>>>(h->a.vir, h->stage, h->a.orig, R.slot_off, n, h->a.S);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(out6n, h->stage, 6 * (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    DevStatus st{};
    if ((rc = read_status(h, &st))) return rc;
    return status_to_code(h, st);
}

int md_set_indenter_velocity(md_t *h, int32_t r, double v_ind)
{
    int rc = check_replica(h, r);
    if (rc) return rc;
    if (!(v_ind == v_ind)) return fail(h, MD_ERR_ARG, "md_set_indenter_velocity: v_ind is NaN");
    h->rep[r].v_ind = v_ind;
    RepDev *d = const_cast<RepDev *>(h->a.rep) + r;
    CU(cudaMemcpyAsync(&d->v_ind, &h->rep[r].v_ind, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    // the drift made for the next step took its displacement threshold from the old path:
    // void it on the device too (a first step in DEC_AUTO reads the device's flag)
    CU(cudaMemsetAsync(&h->a.st->drift_ok, 0, sizeof(int32_t), h->stream));
    CU(cudaStreamSynchronize(h->stream));
    h->drift = false;
    return MD_OK;
}

int md_get_neighbors(md_t *h, int32_t r, int32_t which, int32_t *cell_xyz, int32_t *cnt, int32_t *nbr, int32_t kmax)
{
    int rc = check_replica(h, r);
    if (rc) return rc;
    if (!cnt || (nbr && kmax < 1)) return fail(h, MD_ERR_ARG, "md_get_neighbors: cnt required, kmax >= 1 with nbr");
    const RepDev &R = h->rep[r];
    int n = R.n_atoms, S = h->a.S;
    int K = which ? h->a.kcmax : h->a.kmax;
    std::vector<int32_t> orig(n), c(n), cellc(n), list;
    CU(cudaMemcpy(orig.data(), h->a.orig + R.slot_off, n * sizeof(int32_t), cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(c.data(), (which ? h->a.cntc : h->a.cnt) + R.slot_off, n * sizeof(int32_t), cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(cellc.data(), h->a.cellc + R.slot_off, n * sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (nbr) {
        list.resize((size_t)K * n);
        for (int k = 0; k < K; ++k)
            CU(cudaMemcpy(list.data() + (size_t)k * n, (which ? h->a.nbrc : h->a.nbr) + (size_t)k * S + R.slot_off,
                          n * sizeof(int32_t), cudaMemcpyDeviceToHost));
    }
    const int M = (1 << MD_CELL_BITS) - 1;
    for (int i = 0; i < n; ++i) {
        int o = orig[i];
        cnt[o] = c[i];
        if (cell_xyz) {
            cell_xyz[3 * o] = cellc[i] & M;
            cell_xyz[3 * o + 1] = (cellc[i] >> MD_CELL_BITS) & M;
            cell_xyz[3 * o + 2] = (cellc[i] >> (2 * MD_CELL_BITS)) & M;
        }
        if (nbr) {
            int m = std::min(c[i], kmax);
            for (int k = 0; k < m; ++k) {
                int e = list[(size_t)k * n + i];
                nbr[(size_t)o * kmax + k] = which ? h->c_orig[e] : orig[(int)((unsigned)e & MD_J_MASK) - R.slot_off];
            }
        }
    }
    return MD_OK;
}

int md_check_lists(md_t *h, double radius, int64_t *out8)
{
    if (!h || !out8) return MD_ERR_ARG;
    CU(launch_check_lists(h->a, radius, h->stream));
    DevStatus st{};
    int rc = read_status(h, &st);
    if (rc) return rc;
    for (int t = 0; t < MD_NCHK; ++t) out8[t] = (int64_t)st.chk[t];
    // the violation bit belongs to this call, not to the steps: clear it again
    return clear_err(h);
}

int md_get_info(md_t *h, int64_t *out9)
{
    if (!h || !out9) return MD_ERR_ARG;
    DevStatus st{};
    int rc = read_status(h, &st);
    if (rc) return rc;
    out9[0] = h->n_rep; out9[1] = h->n_cr; out9[2] = h->n_c; out9[3] = h->a.S; out9[4] = h->a.total_cells;
    out9[5] = h->a.kmax; out9[6] = h->a.kcmax; out9[7] = st.max_cnt; out9[8] = st.max_cntc;
    return MD_OK;
}

}  // extern "C"

// ============================================================================ FP64 FMA probe

namespace {
// eight independent FMA chains per thread; the result is stored so that nothing is elided
__global__ void __launch_bounds__(256) k_fp64_fma_probe(double *out, int iters, double b, double c)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double a0 = t * 1e-9, a1 = a0 + 1.0, a2 = a0 + 2.0, a3 = a0 + 3.0, a4 = a0 + 4.0, a5 = a0 + 5.0,
           a6 = a0 + 6.0, a7 = a0 + 7.0;
    for (int i = 0; i < iters; ++i) {
        a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
        a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
    }
    out[t] = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
}
}  // namespace

extern "C" int md_probe_fp64_fma(double *flops_per_s, double *ms)
{
    if (!flops_per_s) return MD_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MD_ERR_CUDA;
    const int blocks = sms * 8, threads = 256, iters = 4096;
    double *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t st = nullptr;
    int rc = MD_OK;
    float t = 0.f;
    if (cudaMalloc((void **)&out, sizeof(double) * (size_t)blocks * threads) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = MD_ERR_CUDA;
    } else {
        k_fp64_fma_probe<<<blocks, threads, 0, st>>>(out, iters, 0.999999, 1e-7);   // warm-up
        cudaEventRecord(e0, st);
        for (int k = 0; k < 5; ++k) k_fp64_fma_probe<<<blocks, threads, 0, st>>>(out, iters, 0.999999, 1e-7);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess ||
            cudaGetLastError() != cudaSuccess)
            rc = MD_ERR_CUDA;
    }
    if (rc == MD_OK) {
        *flops_per_s = 5.0 * 2.0 * 8.0 * iters * (double)blocks * threads / (t * 1e-3);
        if (ms) *ms = t / 5.0;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    return rc;
}

// ============================================================================ md_forces_small

namespace {

constexpr int SMALL_MAX_DEVICES = 64;
std::atomic<double *> g_small_scratch_ptr[SMALL_MAX_DEVICES];   // per device, set on first use

int small_reject(char *errbuf, size_t errlen, int code, const char *fmt, ...)
{
    if (errbuf && errlen) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(errbuf, errlen, fmt, ap);
        va_end(ap);
    }
    return code;
}

}  // namespace

extern "C" int md_forces_small(const md_params *params, int32_t n_cr, const double *x_cr, int32_t n_c,
                               const double *x_c, const double box_lo[3], const double box_hi[3],
                               const int32_t periodic[3], double *F, double *energy, void *stream,
                               char *errbuf, size_t errlen)
{
    if (errbuf && errlen) errbuf[0] = '\0';
    if (!params || !box_lo || !box_hi || !periodic)
        return small_reject(errbuf, errlen, MD_ERR_ARG, "md_forces_small: params, box_lo, box_hi, periodic are required");
    if (n_cr < 0 || n_cr > MD_SMALL_MAX_ATOMS || n_c < 0 || n_c > MD_SMALL_MAX_ATOMS)
        return small_reject(errbuf, errlen, MD_ERR_ARG,
                            "md_forces_small: n_cr = %d, n_c = %d; each must be in 0..%d (the size of its static scratch)",
                            (int)n_cr, (int)n_c, MD_SMALL_MAX_ATOMS);
    if (n_cr > 0 && (!x_cr || !F || !energy))
        return small_reject(errbuf, errlen, MD_ERR_ARG, "md_forces_small: x_cr, F and energy are required when n_cr > 0");
    if (n_c > 0 && !x_c)
        return small_reject(errbuf, errlen, MD_ERR_ARG, "md_forces_small: x_c is required when n_c > 0");
    PotDev P;
    char pmsg[160];
    int rc = md_pot_forms(params, &P, pmsg, sizeof pmsg);
    if (rc != MD_OK) return small_reject(errbuf, errlen, rc, "md_forces_small: %s", pmsg);
    SmallArgs g;
    memset(&g, 0, sizeof g);
    const double reach = std::max(params->rc, params->rc_morse);
    for (int k = 0; k < 3; ++k) {
        g.L[k] = box_hi[k] - box_lo[k];
        g.per[k] = periodic[k] ? 1 : 0;
        if (g.per[k] && !(g.L[k] > 2.0 * reach))
            return small_reject(errbuf, errlen, MD_ERR_ARG,
                                "md_forces_small: periodic axis %d is %.3f A; it must exceed twice the cut-off %.3f A", k, g.L[k], reach);
        g.iL[k] = g.per[k] ? 1.0 / g.L[k] : 0.0;
    }
    // set-up, once per device: the scratch address
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return small_reject(errbuf, errlen, MD_ERR_CUDA, "md_forces_small: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= SMALL_MAX_DEVICES)
        return small_reject(errbuf, errlen, MD_ERR_ARG, "md_forces_small: device %d beyond the %d supported", dev, SMALL_MAX_DEVICES);
    double *scratch = g_small_scratch_ptr[dev].load();
    if (!scratch) {
        size_t nd = 0;
        e = small_setup(&scratch, &nd);
        if (e != cudaSuccess || !scratch)
            return small_reject(errbuf, errlen, MD_ERR_CUDA, "md_forces_small: scratch look-up failed: %s", cudaGetErrorString(e));
        g_small_scratch_ptr[dev].store(scratch);
    }
    if (n_cr == 0) return MD_OK;
    g.n = n_cr; g.n_c = n_c;
    g.nb = (n_cr + MD_SMALL_BLOCK - 1) / MD_SMALL_BLOCK;
    g.x = x_cr; g.xc = x_c; g.F = F; g.energy = energy;
    g.fm = scratch;
    g.part = scratch + 2 * (size_t)MD_SMALL_MAX_ATOMS;
    e = launch_small(g, P, (cudaStream_t)stream);
    if (e != cudaSuccess) return small_reject(errbuf, errlen, MD_ERR_CUDA, "md_forces_small: launch failed: %s", cudaGetErrorString(e));
    return MD_OK;
}
