// C ABI of the library (include/fmm2d.h): plans, workspace, the evaluation
// sequence of Sec. 3.1 / Fig. 3 recorded into a CUDA graph, and the
// accuracy yardsticks.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "fmm2d_internal.cuh"

using namespace fmm2d;

namespace {

thread_local std::string g_last_error;

fmm2d_status fail(fmm2d_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

fmm2d_status cuda_fail(cudaError_t e, const char* where) {
    return fail(e == cudaErrorMemoryAllocation ? FMM2D_OUT_OF_MEMORY : FMM2D_CUDA_ERROR,
                std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

int status_from_flags(int flags) {
    if (flags & kFlagNonfinite) return FMM2D_NONFINITE;
    if (flags & kFlagOutOfDomain) return FMM2D_OUT_OF_DOMAIN;
    if (flags & kFlagInvalid) return FMM2D_INVALID_ARG;
    if (flags & kFlagTimeout) return FMM2D_TIMEOUT;
    return FMM2D_OK;
}

}  // namespace

static constexpr int kPhases = FMM2D_NUM_PHASES;

struct fmm2d_plan {
    fmm2d_params prm{};
    Geometry geo{};
    int device = 0;
    size_t elem = 0;  // bytes per real
    // workspace
    void* ws = nullptr;
    SortBuffers sb{};
    void* particles = nullptr;
    void* me = nullptr;
    void* le = nullptr;
    double* tab64 = nullptr;
    float* tab32 = nullptr;
    int* d_status = nullptr;
    uint32_t* p2p_counter = nullptr;  // near-field work counter (in the status slot)
    int* h_status = nullptr;
    // host-call staging
    void* st_xy = nullptr;
    void* st_gamma = nullptr;
    void* st_uv = nullptr;
    void* st_u1 = nullptr;  // first-stage velocities of a convection step
    // pipelined host evaluations (fmm2d_velocity_host_many), allocated on first use:
    // two input and two output staging sets, copy streams and their events
    void* pipe_buf = nullptr;
    void* pipe_in_xy[2]{}, *pipe_in_g[2]{}, *pipe_out[2]{};
    cudaStream_t pipe_h2d = nullptr, pipe_d2h = nullptr;
    cudaEvent_t pipe_staged[2]{}, pipe_consumed[2]{}, pipe_result[2]{}, pipe_drained[2]{};
    // one recorded evaluation per staging set (reading its inputs and writing
    // its output set directly), for n = pipe_n
    cudaGraph_t pipe_graph[2]{};
    cudaGraphExec_t pipe_exec[2]{};
    int64_t pipe_n = -1;
    // graph cache
    cudaStream_t cap = nullptr;
    // FP32 forms: the far field's branch of the graph and its fork/join events
    cudaStream_t cap2 = nullptr;
    float* uv_sorted = nullptr;  // FP32 forms: near-field velocities in sorted order
    RingStrips strips{};         // FP32 forms with a cutoff: the ring strips (else null)
    bool use_strips = true;      // gather the ring from them (else from whole leaves)
    uint64_t l2_bytes = 0;       // the device's L2 size
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool overlapped = false;  // the recorded graph runs far and near fields side by side
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void* g_xy = nullptr;
    const void* g_gamma = nullptr;
    void* g_uv = nullptr;
    int64_t g_n = -1;
    // timing
    int ring = 0;
    int64_t calls = 0;
    std::vector<cudaEvent_t> ev;        // ring * (kPhases + 1)
    cudaEvent_t ev_mark[kPhases + 1]{}; // placeholders captured into the graph
    cudaGraphNode_t ev_node[kPhases + 1]{};
    bool graph_timed = false;
    int kernel_nodes = -1;
    // tensor-core M2L (FMM2D_FP32_TC)
    void* tc_ws = nullptr;
    float* me_hi = nullptr;
    float* me_lo = nullptr;
    float* bimg = nullptr;  // operator stages
    int4* tiles = nullptr;
    M2LTcConfig tc{};
    M2LTcMaps* maps = nullptr;
    uint32_t spin = 0;  // poll limit of its device waits (0: the default)
};

namespace {

// The ring strips the near field uses (null: whole leaves).
RingStrips strips_of(const fmm2d_plan* pl) {
    return pl->use_strips ? pl->strips : RingStrips{nullptr, nullptr};
}

// out = x + dt u (u2 null) or x + dt (u + u2) / 2, over m reals: the
// position updates of a convection step.
template <typename R>
__global__ void convect_update_kernel(int64_t m, R* __restrict__ out, const R* __restrict__ x,
                                      R dt, const R* __restrict__ u, const R* __restrict__ u2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const R v = u2 ? R(0.5) * (u[i] + u2[i]) : u[i];
        out[i] = x[i] + dt * v;
    }
}

cudaError_t launch_convect_update(size_t elem, int64_t m, void* out, const void* x, double dt,
                                  const void* u, const void* u2, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    const int64_t want = (m + 255) / 256;
    const unsigned blocks = (unsigned)(want < 4096 ? want : 4096);
    if (elem == 8)
        convect_update_kernel<double><<<blocks, 256, 0, s>>>(
            m, static_cast<double*>(out), static_cast<const double*>(x), dt,
            static_cast<const double*>(u), static_cast<const double*>(u2));
    else
        convect_update_kernel<float><<<blocks, 256, 0, s>>>(
            m, static_cast<float*>(out), static_cast<const float*>(x), (float)dt,
            static_cast<const float*>(u), static_cast<const float*>(u2));
    return cudaGetLastError();
}

template <typename R>
Tables<R> tables_of(const fmm2d_plan* pl);
template <>
Tables<double> tables_of<double>(const fmm2d_plan* pl) {
    int64_t per = (int64_t)pl->geo.P * pl->geo.P * 2;
    return {pl->tab64, pl->tab64 + 4 * per, pl->tab64 + 8 * per};
}
template <>
Tables<float> tables_of<float>(const fmm2d_plan* pl) {
    int64_t per = (int64_t)pl->geo.P * pl->geo.P * 2;
    return {pl->tab32, pl->tab32 + 4 * per, pl->tab32 + 8 * per};
}

// Record phase-boundary event `k` (external record node inside a graph).
cudaError_t mark(fmm2d_plan* pl, int k, cudaStream_t s) {
    if (!pl->ring) return cudaSuccess;
    return cudaEventRecordWithFlags(pl->ev_mark[k], s, cudaEventRecordExternal);
}

// The evaluation sequence of Sec. 3.1 on stream s.
template <typename R>
cudaError_t enqueue(fmm2d_plan* pl, int64_t n, const R* xy, const R* gamma, R* uv,
                    cudaStream_t s) {
    const Geometry& g = pl->geo;
    Tables<R> t = tables_of<R>(pl);
    R* me = static_cast<R*>(pl->me);
    R* le = static_cast<R*>(pl->le);
    cudaError_t e;
#define STEP(x)                         \
    if ((e = (x)) != cudaSuccess) return e;
    STEP(mark(pl, 0, s));
    STEP(launch_tree_build<R>(g, n, xy, gamma, pl->sb, pl->particles, s));
    STEP(mark(pl, 1, s));
    const uint32_t* skeys = pl->sb.keys[sort_passes(2 * g.L) & 1];
    if (sizeof(R) == 4 && g.L >= 2 && pl->cap2 && n > 0) {
        // FP32 forms: the near field (without its far part) starts with the
        // tree done, on the whole persistent grid; the far field runs on a
        // second branch of the graph, its kernels filling the SMs that the
        // near field's last work items leave idle; L2P adds the far part once
        // both are done (the fused kernel's sum, bit for bit).  Measured
        // against the sequential order: 7% faster at 2^20 particles (L = 7),
        // 3% at 2^24.  A timed graph (phase marks on) runs the same kernels
        // one after another instead, so that each phase is the duration of
        // its own kernels, not of their wait for room on the GPU.
        float* uvf = reinterpret_cast<float*>(uv);
        const bool fork = pl->ring == 0;
        // the near parts go to a sorted-order buffer (coalesced) while it and
        // the velocities fit in half the L2; beyond that the partial-sector
        // writes of the scattered final store reach memory, and reading the
        // near parts back at the input indices costs less (measured at 2^24:
        // 1.2% of the step)
        const bool sorted = (uint64_t)n * 4 * sizeof(float) <= pl->l2_bytes / 2;
        auto near_only = [&]() {
            return launch_near_only_f32(g, pl->prm.sigma, n, pl->particles, skeys,
                                        pl->sb.leaf_start, pl->p2p_counter,
                                        sorted ? pl->uv_sorted : uvf, sorted, strips_of(pl), s);
        };
        cudaStream_t s2 = s;
        if (fork) {
            STEP(cudaEventRecord(pl->ev_fork, s));
            STEP(cudaStreamWaitEvent(pl->cap2, pl->ev_fork, 0));
            STEP(near_only());
            s2 = pl->cap2;
        }
        STEP(launch_p2m<R>(g, pl->particles, pl->sb.leaf_start, t, me, s2));
        STEP(mark(pl, 2, s2));
        if (g.L >= 4) STEP(launch_m2m<R>(g, t, me, s2));
        STEP(mark(pl, 3, s2));
        if (pl->prm.precision == FMM2D_FP32_TC) {
            STEP(launch_m2l_tc(g, pl->tc, *pl->maps, pl->tiles,
                               reinterpret_cast<const float*>(me), pl->me_hi, pl->me_lo,
                               pl->bimg, reinterpret_cast<float*>(le), pl->d_status, pl->spin,
                               s2));
        } else {
            STEP(launch_m2l<R>(g, t, me, le, s2));
        }
        STEP(mark(pl, 4, s2));
        if (g.L >= 4) STEP(launch_l2l<R>(g, t, le, s2));
        STEP(mark(pl, 5, s2));
        if (fork) {
            STEP(cudaEventRecord(pl->ev_join, s2));
            STEP(cudaStreamWaitEvent(s, pl->ev_join, 0));
        } else {
            STEP(near_only());
        }
        STEP(launch_l2p_f32(g, pl->prm.sigma, n, pl->particles, pl->sb.leaf_start,
                            reinterpret_cast<const float*>(le),
                            reinterpret_cast<const float*>(t.l2l),
                            sorted ? pl->uv_sorted : nullptr, uvf, s));
        STEP(mark(pl, 6, s));
        pl->overlapped = fork;
        return cudaSuccess;
    }
    pl->overlapped = false;
    if (g.L >= 2) STEP(launch_p2m<R>(g, pl->particles, pl->sb.leaf_start, t, me, s));
    STEP(mark(pl, 2, s));
    if (g.L >= 4) STEP(launch_m2m<R>(g, t, me, s));
    STEP(mark(pl, 3, s));
    if (g.L >= 2) {
        if (pl->prm.precision == FMM2D_FP32_TC) {
            STEP(launch_m2l_tc(g, pl->tc, *pl->maps, pl->tiles,
                               reinterpret_cast<const float*>(me), pl->me_hi, pl->me_lo,
                               pl->bimg, reinterpret_cast<float*>(le), pl->d_status, pl->spin,
                               s));
        } else {
            STEP(launch_m2l<R>(g, t, me, le, s));
        }
    }
    STEP(mark(pl, 4, s));
    if (g.L >= 4) STEP(launch_l2l<R>(g, t, le, s));
    STEP(mark(pl, 5, s));
    STEP(launch_p2p_l2p<R>(g, pl->prm.sigma, n, pl->particles, skeys, pl->sb.leaf_start,
                           pl->p2p_counter, le, t.l2l, uv, s));
    STEP(mark(pl, 6, s));
    return cudaSuccess;
}

// Partial evaluations for a split of one evaluation over several devices,
// launched directly on the caller's stream (not recorded in the graph):
// upward (tree, P2M, M2M; the multipoles copied to me_out), or the rest of
// the evaluation from a complete multipole array me_in (tree, M2L, L2L, near
// field and L2P), the steps of Sec. 3.1 in the same order.
template <typename R>
cudaError_t enqueue_partial(fmm2d_plan* pl, bool upward, int64_t n, const R* xy, const R* gamma,
                            const R* me_in, R* me_out, R* uv, cudaStream_t s) {
    const Geometry& g = pl->geo;
    Tables<R> t = tables_of<R>(pl);
    R* me = static_cast<R*>(pl->me);
    R* le = static_cast<R*>(pl->le);
    const size_t me_bytes = (size_t)g.nboxes * 2 * g.P * sizeof(R);
    cudaError_t e;
    STEP(launch_tree_build<R>(g, n, xy, gamma, pl->sb, pl->particles, s));
    const uint32_t* skeys = pl->sb.keys[sort_passes(2 * g.L) & 1];
    if (upward) {
        if (g.L >= 2) {
            STEP(launch_p2m<R>(g, pl->particles, pl->sb.leaf_start, t, me, s));
            if (g.L >= 4) STEP(launch_m2m<R>(g, t, me, s));
            STEP(cudaMemcpyAsync(me_out, me, me_bytes, cudaMemcpyDeviceToDevice, s));
        }
        return cudaSuccess;
    }
    if (g.L >= 2) {
        STEP(cudaMemcpyAsync(me, me_in, me_bytes, cudaMemcpyDeviceToDevice, s));
        if (pl->prm.precision == FMM2D_FP32_TC) {
            STEP(launch_m2l_tc(g, pl->tc, *pl->maps, pl->tiles,
                               reinterpret_cast<const float*>(me), pl->me_hi, pl->me_lo,
                               pl->bimg, reinterpret_cast<float*>(le), pl->d_status, pl->spin,
                               s));
        } else {
            STEP(launch_m2l<R>(g, t, me, le, s));
        }
        if (g.L >= 4) STEP(launch_l2l<R>(g, t, le, s));
    }
    if (sizeof(R) == 4 && g.L >= 2 && n > 0) {
        float* uvf = reinterpret_cast<float*>(uv);
        const bool sorted = (uint64_t)n * 4 * sizeof(float) <= pl->l2_bytes / 2;
        STEP(launch_near_only_f32(g, pl->prm.sigma, n, pl->particles, skeys, pl->sb.leaf_start,
                                  pl->p2p_counter, sorted ? pl->uv_sorted : uvf, sorted,
                                  strips_of(pl), s));
        STEP(launch_l2p_f32(g, pl->prm.sigma, n, pl->particles, pl->sb.leaf_start,
                            reinterpret_cast<const float*>(le),
                            reinterpret_cast<const float*>(t.l2l),
                            sorted ? pl->uv_sorted : nullptr, uvf, s));
        return cudaSuccess;
    }
    STEP(launch_p2p_l2p<R>(g, pl->prm.sigma, n, pl->particles, skeys, pl->sb.leaf_start,
                           pl->p2p_counter, le, t.l2l, uv, s));
    return cudaSuccess;
}
#undef STEP

void drop_main_graph(fmm2d_plan* pl) {
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    pl->exec = nullptr;
    pl->graph = nullptr;
    pl->g_n = -1;
}

// Every recorded evaluation (a setting recorded in the kernels changed).
void drop_graph(fmm2d_plan* pl) {
    drop_main_graph(pl);
    for (int b = 0; b < 2; ++b) {
        if (pl->pipe_exec[b]) cudaGraphExecDestroy(pl->pipe_exec[b]);
        if (pl->pipe_graph[b]) cudaGraphDestroy(pl->pipe_graph[b]);
        pl->pipe_exec[b] = nullptr;
        pl->pipe_graph[b] = nullptr;
    }
    pl->pipe_n = -1;
}

fmm2d_status record_graph(fmm2d_plan* pl, int64_t n, const void* xy, const void* gamma, void* uv) {
    drop_main_graph(pl);
    CK(cudaStreamBeginCapture(pl->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = pl->elem == 8
                        ? enqueue<double>(pl, n, static_cast<const double*>(xy),
                                          static_cast<const double*>(gamma),
                                          static_cast<double*>(uv), pl->cap)
                        : enqueue<float>(pl, n, static_cast<const float*>(xy),
                                         static_cast<const float*>(gamma), static_cast<float*>(uv),
                                         pl->cap);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(pl->cap, &graph);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(e, "kernel launch during capture");
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
    pl->graph = graph;
    CK(cudaGraphInstantiate(&pl->exec, graph, 0));
    {
        size_t count = 0;
        CK(cudaGraphGetNodes(graph, nullptr, &count));
        std::vector<cudaGraphNode_t> nodes(count);
        CK(cudaGraphGetNodes(graph, nodes.data(), &count));
        int kernels = 0;
        for (size_t i = 0; i < count; ++i) {
            cudaGraphNodeType ty;
            CK(cudaGraphNodeGetType(nodes[i], &ty));
            kernels += ty == cudaGraphNodeTypeKernel;
        }
        pl->kernel_nodes = kernels;
    }
    pl->graph_timed = pl->ring > 0;
    if (pl->graph_timed) {
        // find the event-record nodes of the phase marks
        size_t count = 0;
        CK(cudaGraphGetNodes(graph, nullptr, &count));
        std::vector<cudaGraphNode_t> nodes(count);
        CK(cudaGraphGetNodes(graph, nodes.data(), &count));
        for (auto& nd : pl->ev_node) nd = nullptr;
        for (size_t i = 0; i < count; ++i) {
            cudaGraphNodeType ty;
            CK(cudaGraphNodeGetType(nodes[i], &ty));
            if (ty != cudaGraphNodeTypeEventRecord) continue;
            cudaEvent_t evn;
            CK(cudaGraphEventRecordNodeGetEvent(nodes[i], &evn));
            for (int k = 0; k <= kPhases; ++k)
                if (evn == pl->ev_mark[k]) pl->ev_node[k] = nodes[i];
        }
        for (int k = 0; k <= kPhases; ++k)
            if (!pl->ev_node[k]) return fail(FMM2D_CUDA_ERROR, "timing node missing from graph");
    }
    pl->g_xy = xy;
    pl->g_gamma = gamma;
    pl->g_uv = uv;
    pl->g_n = n;
    return FMM2D_OK;
}

fmm2d_status run(fmm2d_plan* pl, int64_t n, const void* xy, const void* gamma, void* uv,
                 cudaStream_t stream) {
    bool timed = pl->ring > 0;
    if (!pl->exec || pl->g_xy != xy || pl->g_gamma != gamma || pl->g_uv != uv || pl->g_n != n ||
        pl->graph_timed != timed) {
        fmm2d_status st = record_graph(pl, n, xy, gamma, uv);
        if (st != FMM2D_OK) return st;
    }
    if (timed) {
        int slot = (int)(pl->calls % pl->ring);
        for (int k = 0; k <= kPhases; ++k)
            CK(cudaGraphExecEventRecordNodeSetEvent(pl->exec, pl->ev_node[k],
                                                    pl->ev[slot * (kPhases + 1) + k]));
    }
    CK(cudaGraphLaunch(pl->exec, stream));
    pl->calls++;
    return FMM2D_OK;
}

bool valid_params(const fmm2d_params* p, std::string* why) {
    if (!p) return *why = "null params", false;
    if (p->p < 1 || p->p > kMaxP) return *why = "p must be in [1, 32]", false;
    if (p->L < 0 || p->L > kMaxL) return *why = "L must be in [0, 12]", false;
    if (!(p->sigma > 0.0) || !std::isfinite(p->sigma)) return *why = "sigma must be > 0", false;
    if (!(p->W > 0.0) || !std::isfinite(p->W) || !std::isfinite(p->x0) || !std::isfinite(p->y0))
        return *why = "root box must be finite with W > 0", false;
    if (p->precision < FMM2D_FP64 || p->precision > FMM2D_FP32_TC)
        return *why = "unknown precision", false;
    if (p->max_n < 0 || p->max_n > (int64_t)0xFFFFFFFF) return *why = "max_n out of range", false;
    // the kernels correct the ring of leaves at Chebyshev distance 2 only
    if (!(p->cutoff >= 0.0) || !std::isfinite(p->cutoff) ||
        (p->L >= 2 && p->cutoff > 2.0 * p->W / ldexp(1.0, p->L)))
        return *why = "cutoff must be in [0, 2 W / 2^L]", false;
    return true;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

extern "C" {

const char* fmm2d_status_string(fmm2d_status s) {
    switch (s) {
        case FMM2D_OK: return "ok";
        case FMM2D_INVALID_ARG: return "invalid argument";
        case FMM2D_OUT_OF_DOMAIN: return "particle outside the root box";
        case FMM2D_NONFINITE: return "non-finite input";
        case FMM2D_CUDA_ERROR: return "CUDA error";
        case FMM2D_TIMEOUT: return "device wait timed out";
        case FMM2D_OUT_OF_MEMORY: return "out of device memory";
        case FMM2D_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char* fmm2d_last_error(void) { return g_last_error.c_str(); }

fmm2d_status fmm2d_plan_create(fmm2d_plan** out, const fmm2d_params* prm) {
    if (!out) return fail(FMM2D_INVALID_ARG, "null output pointer");
    *out = nullptr;
    std::string why;
    if (!valid_params(prm, &why)) return fail(FMM2D_INVALID_ARG, why);
    auto* pl = new fmm2d_plan();
    pl->prm = *prm;
    pl->elem = prm->precision == FMM2D_FP64 ? 8 : 4;
    Geometry& g = pl->geo;
    g.x0 = prm->x0;
    g.y0 = prm->y0;
    g.W = prm->W;
    g.L = prm->L;
    g.p = prm->p;
    g.P = prm->p <= 16 ? 16 : 32;
    int64_t acc = 0;
    for (int l = 0; l <= kMaxL + 1; ++l) g.level_base[l] = 0;
    for (int l = 2; l <= g.L + 1; ++l) {
        g.level_base[l] = acc;
        if (l <= g.L) acc += (int64_t)1 << (2 * l);
    }
    g.nboxes = acc;
    g.scale = ldexp(1.0, g.L) / g.W;
    g.cutoff = prm->cutoff;

    auto cleanup = [&](fmm2d_status s) {
        fmm2d_plan_destroy(pl);
        return s;
    };
    if (cudaGetDevice(&pl->device) != cudaSuccess)
        return cleanup(fail(FMM2D_CUDA_ERROR, "no current CUDA device"));

    int64_t nmax = prm->max_n > 0 ? prm->max_n : 1;
    int64_t nblocks = (nmax + kSortTile - 1) / kSortTile;
    int64_t nleaf = (int64_t)1 << (2 * g.L);
    size_t psize = pl->elem == 8 ? sizeof(ParticleD) : sizeof(float4);
    // the FP32 near field gathers its cutoff ring from per-side strips of the
    // ring leaves (4 records per particle; positions below 2^32)
    const bool strips = pl->elem == 4 && prm->cutoff > 0.0 && g.L >= 2 && nmax < ((int64_t)1 << 30);
    size_t tab_count = (size_t)(8 + kOffsetSlots) * g.P * g.P * 2;
    size_t sizes[] = {
        align256(nmax * 4), align256(nmax * 4), align256(nmax * 4), align256(nmax * 4),
        align256(nmax * 4),                                   // keys x2, vals x2, perm
        align256(((size_t)kRadix * nblocks + kRadix) * 4),    // hist + digit totals
        align256((size_t)(nleaf + 1) * 4),                    // leaf_start
        align256(nmax * psize),                               // particles
        align256((size_t)(g.nboxes > 0 ? g.nboxes : 1) * 2 * g.P * pl->elem),  // me
        align256((size_t)(g.nboxes > 0 ? g.nboxes : 1) * 2 * g.P * pl->elem),  // le
        align256(tab_count * 8),                              // tables fp64
        align256(tab_count * 4),                              // tables fp32
        align256((size_t)(2 * g.P + 1) * (2 * g.P + 1) * 8),  // binomials
        256,                                                  // status, work counter
        align256(((size_t)1 << g.L) * sizeof(float4)),        // leaf-centre table
        align256(pl->elem == 4 ? nmax * 2 * sizeof(float) : 0),  // near field, sorted order
        align256(strips ? (size_t)nmax * 4 * sizeof(float4) : 0),  // ring strips
        align256(strips ? (size_t)nleaf * 4 * 4 : 0),               // their counts
    };
    size_t total = 0;
    for (size_t s : sizes) total += s;
    cudaError_t e = cudaMalloc(&pl->ws, total);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "workspace cudaMalloc"));
    char* p = static_cast<char*>(pl->ws);
    void* slots[18];
    static_assert(sizeof(sizes) / sizeof(sizes[0]) == 18, "one size per slot");
    for (int i = 0; i < 18; ++i) {
        slots[i] = p;
        p += sizes[i];
    }
    pl->sb.keys[0] = (uint32_t*)slots[0];
    pl->sb.keys[1] = (uint32_t*)slots[1];
    pl->sb.vals[0] = (uint32_t*)slots[2];
    pl->sb.vals[1] = (uint32_t*)slots[3];
    pl->sb.perm = (uint32_t*)slots[4];
    pl->sb.hist = (uint32_t*)slots[5];
    pl->sb.leaf_start = (uint32_t*)slots[6];
    pl->particles = slots[7];
    pl->me = slots[8];
    pl->le = slots[9];
    pl->tab64 = (double*)slots[10];
    pl->tab32 = (float*)slots[11];
    double* binom = (double*)slots[12];
    pl->d_status = (int*)slots[13];
    pl->p2p_counter = reinterpret_cast<uint32_t*>(static_cast<char*>(slots[13]) + 128);
    pl->sb.status = pl->d_status;
    float4* centres = (float4*)slots[14];
    pl->uv_sorted = (float*)slots[15];
    if (strips) pl->strips = RingStrips{(float4*)slots[16], (uint32_t*)slots[17]};

    e = cudaHostAlloc((void**)&pl->h_status, sizeof(int), cudaHostAllocDefault);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaHostAlloc"));
    e = cudaStreamCreateWithFlags(&pl->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaStreamCreate"));
    {
        int dev = 0, l2 = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
        pl->l2_bytes = (uint64_t)(l2 > 0 ? l2 : 0);
    }
    if (prm->precision != FMM2D_FP64) {  // the far field's branch of the graph
        e = cudaStreamCreateWithFlags(&pl->cap2, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->ev_join, cudaEventDisableTiming);
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "graph branch set-up"));
    }
    e = cudaMemsetAsync(pl->d_status, 0, sizeof(int), pl->cap);
    if (e == cudaSuccess) {
        int64_t per = (int64_t)g.P * g.P * 2;
        e = launch_build_tables(g.p, g.P, pl->tab64, pl->tab64 + 4 * per, pl->tab64 + 8 * per,
                                binom, pl->cap);
    }
    if (e == cudaSuccess) e = launch_tables_to_f32(pl->tab64, pl->tab32, (int64_t)tab_count, pl->cap);
    if (e == cudaSuccess) e = launch_centre_table(g, centres, pl->cap);
    if (e == cudaSuccess) e = cudaStreamSynchronize(pl->cap);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "table build"));
    g.centre_tab = centres;  // the kernels read leaf centres from the table
    for (int k = 0; k <= kPhases; ++k) {
        e = cudaEventCreate(&pl->ev_mark[k]);
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaEventCreate"));
    }
    if (prm->precision == FMM2D_FP32_TC && g.L >= 2) {
        static bool configured = false;
        if (!configured) {
            e = m2l_tc_configure();
            if (e != cudaSuccess) return cleanup(cuda_fail(e, "tensor-core M2L configuration"));
            configured = true;
        }
        M2LTcConfig cfg = m2l_tc_plan(g, nullptr);  // tile count first (no device work)
        std::vector<int4> tiles(2 * (size_t)cfg.ntiles);  // two records per tile
        cfg = m2l_tc_plan(g, tiles.data());
        size_t me_floats = (size_t)g.nboxes * 2 * cfg.Pk;
        size_t bytes = align256(me_floats * 4) * 2 + align256((size_t)cfg.b_floats * 4) +
                       align256((size_t)cfg.ntiles * 2 * sizeof(int4));
        e = cudaMalloc(&pl->tc_ws, bytes);
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "tensor-core workspace cudaMalloc"));
        char* q = static_cast<char*>(pl->tc_ws);
        pl->me_hi = (float*)q;
        q += align256(me_floats * 4);
        pl->me_lo = (float*)q;
        q += align256(me_floats * 4);
        pl->bimg = (float*)q;
        q += align256((size_t)cfg.b_floats * 4);
        pl->tiles = (int4*)q;
        pl->maps = new M2LTcMaps();
        int64_t per = (int64_t)g.P * g.P * 2;
        e = m2l_tc_prepare(g, cfg, pl->tab64 + 8 * per, pl->me_hi, pl->me_lo, pl->bimg, pl->maps,
                           pl->cap);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(pl->tiles, tiles.data(), (size_t)cfg.ntiles * 2 * sizeof(int4),
                                cudaMemcpyHostToDevice, pl->cap);
        if (e == cudaSuccess) e = cudaStreamSynchronize(pl->cap);
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "tensor-core M2L set-up"));
        pl->tc = cfg;
    }
    *out = pl;
    return FMM2D_OK;
}

void fmm2d_plan_destroy(fmm2d_plan* pl) {
    if (!pl) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(pl->device);
    cudaDeviceSynchronize();
    drop_graph(pl);
    for (auto ev : pl->ev) cudaEventDestroy(ev);
    for (auto ev : pl->ev_mark)
        if (ev) cudaEventDestroy(ev);
    if (pl->cap) cudaStreamDestroy(pl->cap);
    if (pl->cap2) cudaStreamDestroy(pl->cap2);
    if (pl->ev_fork) cudaEventDestroy(pl->ev_fork);
    if (pl->ev_join) cudaEventDestroy(pl->ev_join);
    if (pl->h_status) cudaFreeHost(pl->h_status);
    if (pl->st_xy) cudaFree(pl->st_xy);
    if (pl->pipe_buf) cudaFree(pl->pipe_buf);
    if (pl->pipe_h2d) cudaStreamDestroy(pl->pipe_h2d);
    if (pl->pipe_d2h) cudaStreamDestroy(pl->pipe_d2h);
    for (int b = 0; b < 2; ++b)
        for (cudaEvent_t ev : {pl->pipe_staged[b], pl->pipe_consumed[b], pl->pipe_result[b],
                               pl->pipe_drained[b]})
            if (ev) cudaEventDestroy(ev);
    if (pl->tc_ws) cudaFree(pl->tc_ws);
    delete pl->maps;
    if (pl->ws) cudaFree(pl->ws);
    cudaSetDevice(cur);
    delete pl;
}

fmm2d_status fmm2d_velocity(fmm2d_plan* pl, int64_t n, const void* xy, const void* gamma,
                            void* uv, cudaStream_t stream) {
    if (!pl) return fail(FMM2D_INVALID_ARG, "null plan");
    if (n < 0 || n > pl->prm.max_n) return fail(FMM2D_INVALID_ARG, "n out of [0, max_n]");
    if (n > 0 && (!xy || !gamma || !uv)) return fail(FMM2D_INVALID_ARG, "null buffer");
    return run(pl, n, xy, gamma, uv, stream);
}

fmm2d_status fmm2d_plan_check(fmm2d_plan* pl, cudaStream_t stream) {
    if (!pl) return fail(FMM2D_INVALID_ARG, "null plan");
    CK(cudaMemcpyAsync(pl->h_status, pl->d_status, sizeof(int), cudaMemcpyDeviceToHost, stream));
    CK(cudaMemsetAsync(pl->d_status, 0, sizeof(int), stream));
    CK(cudaStreamSynchronize(stream));
    int st = status_from_flags(*pl->h_status);
    if (st != FMM2D_OK) return fail((fmm2d_status)st, "device reported an input error");
    return FMM2D_OK;
}

// Staging buffers for max_n particles (allocated on first use).
static fmm2d_status ensure_staging(fmm2d_plan* pl) {
    if (pl->st_xy) return FMM2D_OK;
    size_t nm = (size_t)(pl->prm.max_n > 0 ? pl->prm.max_n : 1);
    size_t bxy = align256(2 * nm * pl->elem), bg = align256(nm * pl->elem);
    void* buf = nullptr;
    CK(cudaMalloc(&buf, 3 * bxy + bg));
    pl->st_xy = buf;
    pl->st_gamma = static_cast<char*>(buf) + bxy;
    pl->st_uv = static_cast<char*>(buf) + bxy + bg;
    pl->st_u1 = static_cast<char*>(buf) + 2 * bxy + bg;
    return FMM2D_OK;
}

int64_t fmm2d_plan_multipole_reals(const fmm2d_plan* pl) {
    return pl ? pl->geo.nboxes * 2 * pl->geo.P : -1;
}

fmm2d_status fmm2d_multipoles(fmm2d_plan* pl, int64_t n, const void* xy, const void* gamma,
                              void* me_dev, cudaStream_t stream) {
    if (!pl) return fail(FMM2D_INVALID_ARG, "null plan");
    if (n < 0 || n > pl->prm.max_n) return fail(FMM2D_INVALID_ARG, "n out of [0, max_n]");
    if ((n > 0 && (!xy || !gamma)) || (pl->geo.nboxes > 0 && !me_dev))
        return fail(FMM2D_INVALID_ARG, "null buffer");
    cudaError_t e = pl->elem == 8
                        ? enqueue_partial<double>(pl, true, n, static_cast<const double*>(xy),
                                                  static_cast<const double*>(gamma), nullptr,
                                                  static_cast<double*>(me_dev), nullptr, stream)
                        : enqueue_partial<float>(pl, true, n, static_cast<const float*>(xy),
                                                 static_cast<const float*>(gamma), nullptr,
                                                 static_cast<float*>(me_dev), nullptr, stream);
    if (e != cudaSuccess) return cuda_fail(e, "multipoles");
    return FMM2D_OK;
}

fmm2d_status fmm2d_velocity_from_multipoles(fmm2d_plan* pl, int64_t n, const void* xy,
                                            const void* gamma, const void* me_dev, void* uv,
                                            cudaStream_t stream) {
    if (!pl) return fail(FMM2D_INVALID_ARG, "null plan");
    if (n < 0 || n > pl->prm.max_n) return fail(FMM2D_INVALID_ARG, "n out of [0, max_n]");
    if ((n > 0 && (!xy || !gamma || !uv)) || (pl->geo.nboxes > 0 && !me_dev))
        return fail(FMM2D_INVALID_ARG, "null buffer");
    cudaError_t e = pl->elem == 8
                        ? enqueue_partial<double>(pl, false, n, static_cast<const double*>(xy),
                                                  static_cast<const double*>(gamma),
                                                  static_cast<const double*>(me_dev), nullptr,
                                                  static_cast<double*>(uv), stream)
                        : enqueue_partial<float>(pl, false, n, static_cast<const float*>(xy),
                                                 static_cast<const float*>(gamma),
                                                 static_cast<const float*>(me_dev), nullptr,
                                                 static_cast<float*>(uv), stream);
    if (e != cudaSuccess) return cuda_fail(e, "velocity_from_multipoles");
    return FMM2D_OK;
}

fmm2d_status fmm2d_velocity_host(fmm2d_plan* pl, int64_t n, const void* xy_host,
                                 const void* gamma_host, void* uv_host, cudaStream_t stream) {
    if (!pl) return fail(FMM2D_INVALID_ARG, "null plan");
    if (n < 0 || n > pl->prm.max_n) return fail(FMM2D_INVALID_ARG, "n out of [0, max_n]");
    if (n > 0 && (!xy_host || !gamma_host || !uv_host)) return fail(FMM2D_INVALID_ARG, "null buffer");
    fmm2d_status sst = ensure_staging(pl);
    if (sst != FMM2D_OK) return sst;
    if (n > 0) {
        CK(cudaMemcpyAsync(pl->st_xy, xy_host, 2 * n * pl->elem, cudaMemcpyHostToDevice, stream));
        CK(cudaMemcpyAsync(pl->st_gamma, gamma_host, n * pl->elem, cudaMemcpyHostToDevice, stream));
    }
    fmm2d_status st = run(pl, n, pl->st_xy, pl->st_gamma, pl->st_uv, stream);
    if (st != FMM2D_OK) return st;
    if (n > 0)
        CK(cudaMemcpyAsync(uv_host, pl->st_uv, 2 * n * pl->elem, cudaMemcpyDeviceToHost, stream));
    return fmm2d_plan_check(pl, stream);
}

// Staging sets, streams and events of the pipelined host evaluations.
static fmm2d_status ensure_pipe(fmm2d_plan* pl) {
    if (pl->pipe_buf) return FMM2D_OK;
    size_t nm = (size_t)(pl->prm.max_n > 0 ? pl->prm.max_n : 1);
    size_t bxy = align256(2 * nm * pl->elem), bg = align256(nm * pl->elem);
    void* buf = nullptr;
    CK(cudaMalloc(&buf, 2 * (2 * bxy + bg)));
    pl->pipe_buf = buf;
    char* p = static_cast<char*>(buf);
    for (int b = 0; b < 2; ++b) {
        pl->pipe_in_xy[b] = p;
        pl->pipe_in_g[b] = p + bxy;
        pl->pipe_out[b] = p + bxy + bg;
        p += 2 * bxy + bg;
    }
    CK(cudaStreamCreateWithFlags(&pl->pipe_h2d, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&pl->pipe_d2h, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
        CK(cudaEventCreateWithFlags(&pl->pipe_staged[b], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&pl->pipe_consumed[b], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&pl->pipe_result[b], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&pl->pipe_drained[b], cudaEventDisableTiming));
    }
    return FMM2D_OK;
}

fmm2d_status fmm2d_velocity_host_many(fmm2d_plan* pl, int count, int64_t n,
                                      const void* const* xy_host, const void* const* gamma_host,
                                      void* const* uv_host, cudaStream_t stream) {
    if (!pl) return fail(FMM2D_INVALID_ARG, "null plan");
    if (count < 0) return fail(FMM2D_INVALID_ARG, "count < 0");
    if (n < 0 || n > pl->prm.max_n) return fail(FMM2D_INVALID_ARG, "n out of [0, max_n]");
    if (count > 0 && n > 0) {
        if (!xy_host || !gamma_host || !uv_host) return fail(FMM2D_INVALID_ARG, "null buffer");
        for (int k = 0; k < count; ++k)
            if (!xy_host[k] || !gamma_host[k] || !uv_host[k])
                return fail(FMM2D_INVALID_ARG, "null buffer");
    }
    if (count == 0 || n == 0) {
        for (int k = 0; k < count; ++k) {
            fmm2d_status st = run(pl, 0, nullptr, nullptr, nullptr, stream);
            if (st != FMM2D_OK) return st;
        }
        return fmm2d_plan_check(pl, stream);
    }
    fmm2d_status sst = ensure_staging(pl);
    if (sst != FMM2D_OK) return sst;
    sst = ensure_pipe(pl);
    if (sst != FMM2D_OK) return sst;
    const size_t bxy = 2 * (size_t)n * pl->elem, bg = (size_t)n * pl->elem;
    // one recorded evaluation per staging set, so that no copy between the
    // staging sets and the plan's buffers is needed (not with phase timing,
    // whose marks belong to the plan's own graph)
    const bool direct = pl->ring == 0;
    if (direct && pl->pipe_n != n) {
        for (int b = 0; b < 2; ++b) {
            fmm2d_status st = record_graph(pl, n, pl->pipe_in_xy[b], pl->pipe_in_g[b],
                                           pl->pipe_out[b]);
            if (st != FMM2D_OK) return st;
            if (pl->pipe_exec[b]) cudaGraphExecDestroy(pl->pipe_exec[b]);
            if (pl->pipe_graph[b]) cudaGraphDestroy(pl->pipe_graph[b]);
            pl->pipe_graph[b] = pl->graph;  // moved out of the plan's own cache
            pl->pipe_exec[b] = pl->exec;
            pl->graph = nullptr;
            pl->exec = nullptr;
            pl->g_n = -1;
        }
        pl->pipe_n = n;
    }
    // the copy streams start after whatever `stream` has queued before this call
    CK(cudaEventRecord(pl->pipe_consumed[0], stream));
    CK(cudaEventRecord(pl->pipe_consumed[1], stream));
    CK(cudaEventRecord(pl->pipe_drained[0], stream));
    CK(cudaEventRecord(pl->pipe_drained[1], stream));
    for (int k = 0; k < count; ++k) {
        const int b = k & 1;
        // inputs of set k into staging set b once set k - 2 has left it
        CK(cudaStreamWaitEvent(pl->pipe_h2d, pl->pipe_consumed[b], 0));
        CK(cudaMemcpyAsync(pl->pipe_in_xy[b], xy_host[k], bxy, cudaMemcpyHostToDevice,
                           pl->pipe_h2d));
        CK(cudaMemcpyAsync(pl->pipe_in_g[b], gamma_host[k], bg, cudaMemcpyHostToDevice,
                           pl->pipe_h2d));
        CK(cudaEventRecord(pl->pipe_staged[b], pl->pipe_h2d));
        if (direct) {
            // set b's own graph: reads staging set b, writes output set b once
            // set k - 2's velocities have been read back from it
            CK(cudaStreamWaitEvent(stream, pl->pipe_staged[b], 0));
            CK(cudaStreamWaitEvent(stream, pl->pipe_drained[b], 0));
            CK(cudaGraphLaunch(pl->pipe_exec[b], stream));
            pl->calls++;
            CK(cudaEventRecord(pl->pipe_consumed[b], stream));
            CK(cudaEventRecord(pl->pipe_result[b], stream));
            CK(cudaStreamWaitEvent(pl->pipe_d2h, pl->pipe_result[b], 0));
            CK(cudaMemcpyAsync(uv_host[k], pl->pipe_out[b], bxy, cudaMemcpyDeviceToHost,
                               pl->pipe_d2h));
            CK(cudaEventRecord(pl->pipe_drained[b], pl->pipe_d2h));
            continue;
        }
        // the evaluation reads the plan's fixed buffers (one recorded graph)
        CK(cudaStreamWaitEvent(stream, pl->pipe_staged[b], 0));
        CK(cudaMemcpyAsync(pl->st_xy, pl->pipe_in_xy[b], bxy, cudaMemcpyDeviceToDevice, stream));
        CK(cudaMemcpyAsync(pl->st_gamma, pl->pipe_in_g[b], bg, cudaMemcpyDeviceToDevice, stream));
        CK(cudaEventRecord(pl->pipe_consumed[b], stream));
        fmm2d_status st = run(pl, n, pl->st_xy, pl->st_gamma, pl->st_uv, stream);
        if (st != FMM2D_OK) return st;
        // velocities of set k into output set b once set k - 2's have been read back
        CK(cudaStreamWaitEvent(stream, pl->pipe_drained[b], 0));
        CK(cudaMemcpyAsync(pl->pipe_out[b], pl->st_uv, bxy, cudaMemcpyDeviceToDevice, stream));
        CK(cudaEventRecord(pl->pipe_result[b], stream));
        CK(cudaStreamWaitEvent(pl->pipe_d2h, pl->pipe_result[b], 0));
        CK(cudaMemcpyAsync(uv_host[k], pl->pipe_out[b], bxy, cudaMemcpyDeviceToHost,
                           pl->pipe_d2h));
        CK(cudaEventRecord(pl->pipe_drained[b], pl->pipe_d2h));
    }
    CK(cudaStreamSynchronize(pl->pipe_d2h));
    CK(cudaStreamSynchronize(pl->pipe_h2d));
    return fmm2d_plan_check(pl, stream);
}

fmm2d_status fmm2d_convect(fmm2d_plan* pl, int64_t n, void* xy, const void* gamma, double dt,
                           int order, cudaStream_t stream) {
    if (!pl) return fail(FMM2D_INVALID_ARG, "null plan");
    if (n < 0 || n > pl->prm.max_n) return fail(FMM2D_INVALID_ARG, "n out of [0, max_n]");
    if (n > 0 && (!xy || !gamma)) return fail(FMM2D_INVALID_ARG, "null buffer");
    if (order != 1 && order != 2) return fail(FMM2D_INVALID_ARG, "order must be 1 or 2");
    if (!std::isfinite(dt)) return fail(FMM2D_INVALID_ARG, "dt must be finite");
    fmm2d_status st = ensure_staging(pl);
    if (st != FMM2D_OK) return st;
    if (n == 0) return FMM2D_OK;
    // both evaluations read the staging positions and write the staging
    // velocities, so the plan's recorded graph serves both
    const size_t e = pl->elem, bytes = 2 * (size_t)n * e;
    CK(cudaMemcpyAsync(pl->st_xy, xy, bytes, cudaMemcpyDeviceToDevice, stream));
    st = run(pl, n, pl->st_xy, gamma, pl->st_uv, stream);
    if (st != FMM2D_OK) return st;
    if (order == 1) {
        CK(launch_convect_update(e, 2 * n, xy, xy, dt, pl->st_uv, nullptr, stream));
        return FMM2D_OK;
    }
    // Heun: x* = x + dt u(x), x' = x + dt (u(x) + u(x*)) / 2
    CK(cudaMemcpyAsync(pl->st_u1, pl->st_uv, bytes, cudaMemcpyDeviceToDevice, stream));
    CK(launch_convect_update(e, 2 * n, pl->st_xy, xy, dt, pl->st_u1, nullptr, stream));
    st = run(pl, n, pl->st_xy, gamma, pl->st_uv, stream);
    if (st != FMM2D_OK) return st;
    CK(launch_convect_update(e, 2 * n, xy, xy, dt, pl->st_u1, pl->st_uv, stream));
    return FMM2D_OK;
}

fmm2d_status fmm2d_velocity_targets(fmm2d_plan* pl, int64_t n, const void* xy,
                                    const void* gamma, int64_t m, const void* txy, void* tuv,
                                    cudaStream_t stream) {
    if (!pl) return fail(FMM2D_INVALID_ARG, "null plan");
    if (n < 0 || m < 0 || n + m > pl->prm.max_n)
        return fail(FMM2D_INVALID_ARG, "need n, m >= 0 and n + m <= max_n");
    if ((n > 0 && (!xy || !gamma)) || (m > 0 && (!txy || !tuv)))
        return fail(FMM2D_INVALID_ARG, "null buffer");
    fmm2d_status sst = ensure_staging(pl);
    if (sst != FMM2D_OK) return sst;
    // particles, then the targets as particles of zero circulation: they
    // induce nothing and receive the velocity at their positions
    char* sxy = static_cast<char*>(pl->st_xy);
    char* sg = static_cast<char*>(pl->st_gamma);
    const size_t e = pl->elem;
    if (n > 0) {
        CK(cudaMemcpyAsync(sxy, xy, 2 * n * e, cudaMemcpyDeviceToDevice, stream));
        CK(cudaMemcpyAsync(sg, gamma, n * e, cudaMemcpyDeviceToDevice, stream));
    }
    if (m > 0) {
        CK(cudaMemcpyAsync(sxy + 2 * n * e, txy, 2 * m * e, cudaMemcpyDeviceToDevice, stream));
        CK(cudaMemsetAsync(sg + n * e, 0, m * e, stream));  // +0.0 in either precision
    }
    fmm2d_status st = run(pl, n + m, pl->st_xy, pl->st_gamma, pl->st_uv, stream);
    if (st != FMM2D_OK) return st;
    if (m > 0)
        CK(cudaMemcpyAsync(tuv, static_cast<char*>(pl->st_uv) + 2 * n * e, 2 * m * e,
                           cudaMemcpyDeviceToDevice, stream));
    return FMM2D_OK;
}

fmm2d_status fmm2d_tree_debug(fmm2d_plan* pl, uint32_t* keys, uint32_t* perm,
                              uint32_t* leaf_start, cudaStream_t stream) {
    if (!pl) return fail(FMM2D_INVALID_ARG, "null plan");
    if (pl->g_n < 0) return fail(FMM2D_INVALID_ARG, "no evaluation has run on this plan");
    int64_t n = pl->g_n;
    int bits = 2 * pl->geo.L;
    const uint32_t* sorted = pl->sb.keys[sort_passes(bits) & 1];
    if (keys && n > 0)
        CK(cudaMemcpyAsync(keys, sorted, n * 4, cudaMemcpyDeviceToDevice, stream));
    if (perm && n > 0)
        CK(cudaMemcpyAsync(perm, pl->sb.perm, n * 4, cudaMemcpyDeviceToDevice, stream));
    if (leaf_start)
        CK(cudaMemcpyAsync(leaf_start, pl->sb.leaf_start, (((size_t)1 << (2 * pl->geo.L)) + 1) * 4,
                           cudaMemcpyDeviceToDevice, stream));
    return FMM2D_OK;
}

fmm2d_status fmm2d_direct_sampled(fmm2d_plan* pl, int kernel, int64_t n, const void* xy,
                                  const void* gamma, int64_t s, const int64_t* targets,
                                  double* uv_ref, cudaStream_t stream) {
    if (!pl) return fail(FMM2D_INVALID_ARG, "null plan");
    if (kernel != 0 && kernel != 1) return fail(FMM2D_INVALID_ARG, "kernel must be 0 or 1");
    if (n < 0 || s < 0) return fail(FMM2D_INVALID_ARG, "negative size");
    if (s > 0 && (!xy || !gamma || !targets || !uv_ref))
        return fail(FMM2D_INVALID_ARG, "null buffer");
    cudaError_t e =
        pl->elem == 8
            ? launch_direct_sampled<double>(pl->geo, pl->prm.sigma, kernel, n,
                                            static_cast<const double*>(xy),
                                            static_cast<const double*>(gamma), s, targets, uv_ref,
                                            pl->d_status, stream)
            : launch_direct_sampled<float>(pl->geo, pl->prm.sigma, kernel, n,
                                           static_cast<const float*>(xy),
                                           static_cast<const float*>(gamma), s, targets, uv_ref,
                                           pl->d_status, stream);
    if (e != cudaSuccess) return cuda_fail(e, "direct_sampled launch");
    return FMM2D_OK;
}

fmm2d_status fmm2d_error_stats(fmm2d_plan* pl, int64_t n, const void* xy, const void* uv,
                               int64_t s, const int64_t* targets, const double* uv_ref,
                               double* stats, double* leaf_err, cudaStream_t stream) {
    if (!pl) return fail(FMM2D_INVALID_ARG, "null plan");
    if (n < 0 || s < 0) return fail(FMM2D_INVALID_ARG, "negative size");
    if (!stats || (s > 0 && (!xy || !uv || !targets || !uv_ref)))
        return fail(FMM2D_INVALID_ARG, "null buffer");
    cudaError_t e =
        pl->elem == 8
            ? launch_error_stats<double>(pl->geo, n, static_cast<const double*>(xy),
                                         static_cast<const double*>(uv), s, targets, uv_ref, stats,
                                         leaf_err, pl->d_status, stream)
            : launch_error_stats<float>(pl->geo, n, static_cast<const float*>(xy),
                                        static_cast<const float*>(uv), s, targets, uv_ref, stats,
                                        leaf_err, pl->d_status, stream);
    if (e != cudaSuccess) return cuda_fail(e, "error_stats launch");
    return FMM2D_OK;
}

fmm2d_status fmm2d_plan_set_timing(fmm2d_plan* pl, int ring) {
    if (!pl) return fail(FMM2D_INVALID_ARG, "null plan");
    if (ring < 0 || ring > 4096) return fail(FMM2D_INVALID_ARG, "ring must be in [0, 4096]");
    CK(cudaDeviceSynchronize());
    for (auto ev : pl->ev) cudaEventDestroy(ev);
    pl->ev.clear();
    pl->ring = 0;
    pl->calls = 0;
    for (int i = 0; i < ring * (kPhases + 1); ++i) {
        cudaEvent_t ev;
        CK(cudaEventCreate(&ev));
        pl->ev.push_back(ev);
    }
    pl->ring = ring;
    drop_graph(pl);
    return FMM2D_OK;
}

fmm2d_status fmm2d_plan_phase_ms(fmm2d_plan* pl, int age, double* ms) {
    if (!pl || !ms) return fail(FMM2D_INVALID_ARG, "null argument");
    if (!pl->ring) return fail(FMM2D_INVALID_ARG, "timing is off");
    if (age < 0 || age >= pl->ring || age >= pl->calls)
        return fail(FMM2D_INVALID_ARG, "no such call in the timing ring");
    int slot = (int)((pl->calls - 1 - age) % pl->ring);
    cudaEvent_t* e = &pl->ev[slot * (kPhases + 1)];
    CK(cudaEventSynchronize(e[kPhases]));
    for (int k = 0; k < kPhases; ++k) {
        float t = 0.f;
        // side by side (pl->overlapped): the near field runs from the end of
        // the tree to the end of L2P, the far-field phases on their branch
        const bool near = pl->overlapped && k == kPhases - 1;
        CK(cudaEventElapsedTime(&t, e[near ? 1 : k], e[k + 1]));
        ms[k] = t;
    }
    return FMM2D_OK;
}

int fmm2d_plan_kernels_per_call(const fmm2d_plan* pl) { return pl ? pl->kernel_nodes : -1; }

fmm2d_status fmm2d_plan_set_ring_strips(fmm2d_plan* pl, int enable) {
    if (!pl) return fail(FMM2D_INVALID_ARG, "null plan");
    pl->use_strips = enable != 0;
    drop_graph(pl);  // the strips are kernel arguments recorded in the graph
    return FMM2D_OK;
}

fmm2d_status fmm2d_plan_set_spin_limit(fmm2d_plan* pl, uint32_t polls) {
    if (!pl) return fail(FMM2D_INVALID_ARG, "null plan");
    pl->spin = polls;
    drop_graph(pl);  // the limit is a kernel argument recorded in the graph
    return FMM2D_OK;
}

}  // extern "C"
