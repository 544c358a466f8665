// Batched evaluation: many independent FMM evaluations of uneven size,
// expansion order and depth -- a parameter sweep like the paper's study of
// about a thousand runs (Sec. 5) -- executed as one packed problem.
//
// Instances are packed back to back in the caller's arrays and into one
// global leaf index space, so one stable radix sort builds every quadtree.
// Each step of Sec. 3.1 is one launch over all instances (per expansion
// stride class P = 16 or 32, and per level where levels depend on each
// other); the near field is one persistent launch whose warps pull leaves
// from a work counter, largest instances first.  The whole sequence is
// recorded once into a CUDA graph and replayed.  An autotuner times the
// candidate launch shapes of the two heaviest steps on the batch itself.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "fmm2d_internal.cuh"

using namespace fmm2d;

namespace {

thread_local std::string g_batch_error;

fmm2d_status bfail(fmm2d_status s, const std::string& m) {
    g_batch_error = m;
    return s;
}
#define BCK(call)                                                                        \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return bfail(e_ == cudaErrorMemoryAllocation ? FMM2D_OUT_OF_MEMORY           \
                                                         : FMM2D_CUDA_ERROR,             \
                         std::string(#call) + ": " + cudaGetErrorString(e_));            \
    } while (0)

size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

struct fmm2d_batch_plan {
    int count = 0;
    int device = 0;
    std::vector<BatchInst> inst;  // host copies
    int64_t ntotal = 0;
    uint32_t nleaf_total = 0;
    int key_bits = 1;
    int max_L = 0;
    // device
    void* ws = nullptr;
    BatchInst* d_inst = nullptr;
    int64_t* d_offsets = nullptr;
    void* d_keyparams = nullptr;
    void* d_near = nullptr;
    int32_t* d_leaf_inst = nullptr;
    uint32_t* d_counter = nullptr;
    int* d_status = nullptr;
    int* h_status = nullptr;
    SortBuffers sb{};
    void* particles = nullptr;
    float* me = nullptr;
    float* le = nullptr;
    double* tab64[2] = {nullptr, nullptr};
    float* tab32[2] = {nullptr, nullptr};
    bool has_class[2] = {false, false};
    BatchLists lists[2]{};
    // launch shapes (autotuned; the near field's default is the residency
    // limit of its kernels, which the autotuner picked on every sweep measured)
    int p2p_ctas_per_sm = 6;
    int m2l_threads = 128;
    // FP32_TC: one tensor-core M2L class per Pk (operator stages and tile
    // policy autotuned); FP32: M2L on the CUDA cores
    int precision = FMM2D_FP32;
    std::vector<M2LTcBatchClass> tc;
    int tc_b_stages = 0;  // 0: as many as shared memory holds
    int tc_policy = 0;
    bool any_cutoff = false;
    RingStrips strips{};  // with a cutoff: the near field's ring strips
    // windows of 32 sorted positions holding particles of instances whose
    // sparse leaves take the near field's per-target-lane pass
    uint32_t* lane_win = nullptr;
    uint32_t lane_win_count = 0;
    // graph
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void* g_xy = nullptr;
    const void* g_gamma = nullptr;
    void* g_uv = nullptr;
    int kernel_nodes = -1;
};

namespace {

int class_of(int P) { return P <= 16 ? 0 : 1; }

const float* tab_m2m(const fmm2d_batch_plan* b, int c) { return b->tab32[c]; }
const float* tab_l2l(const fmm2d_batch_plan* b, int c) {
    int P = c ? 32 : 16;
    return b->tab32[c] + (int64_t)4 * P * P * 2;
}
const float* tab_m2l(const fmm2d_batch_plan* b, int c) {
    int P = c ? 32 : 16;
    return b->tab32[c] + (int64_t)8 * P * P * 2;
}

// The batch's steps on stream s; with `ev` (6 events) each phase boundary is
// recorded: tree, P2M + M2M, M2L, L2L, near field with L2P.
cudaError_t enqueue_batch(fmm2d_batch_plan* b, const float* xy, const float* gamma, float* uv,
                          cudaStream_t s, cudaEvent_t* ev = nullptr) {
    cudaError_t e;
#define BSTEP(x) \
    if ((e = (x)) != cudaSuccess) return e;
#define BMARK(k) \
    if (ev) BSTEP(cudaEventRecord(ev[k], s));
    BMARK(0);
    BSTEP(launch_batch_tree(b->d_keyparams, b->d_offsets, b->count, b->ntotal, b->key_bits,
                            b->nleaf_total, xy, gamma, b->sb, b->particles, s));
    BMARK(1);
    for (int c = 0; c < 2; ++c)
        if (b->has_class[c])
            BSTEP(launch_batch_p2m(b->d_inst, b->lists[c], c ? 32 : 16, b->particles,
                                   b->sb.leaf_start, tab_m2m(b, c), b->me, s));
    for (int l = b->max_L - 2; l >= 2; --l)
        for (int c = 0; c < 2; ++c)
            if (b->has_class[c])
                BSTEP(launch_batch_m2m(b->d_inst, b->lists[c], c ? 32 : 16, l, tab_m2m(b, c),
                                       b->me, s));
    BMARK(2);
    if (b->precision == FMM2D_FP32_TC) {
        for (const M2LTcBatchClass& c : b->tc)
            BSTEP(launch_m2l_tc_batch(c, b->d_inst, b->me, b->le, b->d_status, 0, s));
    } else {
        for (int c = 0; c < 2; ++c)
            if (b->has_class[c])
                BSTEP(launch_batch_m2l(b->d_inst, b->lists[c], c ? 32 : 16, b->m2l_threads,
                                       tab_m2l(b, c), b->me, b->le, s));
    }
    BMARK(3);
    for (int l = 3; l <= b->max_L - 1; ++l)
        for (int c = 0; c < 2; ++c)
            if (b->has_class[c])
                BSTEP(launch_batch_l2l(b->d_inst, b->lists[c], c ? 32 : 16, l, tab_l2l(b, c),
                                       b->le, s));
    BMARK(4);
    BSTEP(launch_batch_p2p(b->d_inst, b->d_near, b->d_leaf_inst, (uint32_t)b->ntotal,
                           b->d_counter, b->p2p_ctas_per_sm, b->particles,
                           b->sb.keys[sort_passes(b->key_bits) & 1], b->sb.leaf_start, b->le,
                           b->has_class[0] ? tab_l2l(b, 0) : nullptr,
                           b->has_class[1] ? tab_l2l(b, 1) : nullptr, uv, b->any_cutoff, b->strips,
                           b->nleaf_total, b->lane_win, b->lane_win_count, s));
    BMARK(5);
#undef BMARK
#undef BSTEP
    return cudaSuccess;
}

void drop_batch_graph(fmm2d_batch_plan* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->g_xy = nullptr;
}

fmm2d_status record_batch_graph(fmm2d_batch_plan* b, const float* xy, const float* gamma,
                                float* uv) {
    drop_batch_graph(b);
    BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_batch(b, xy, gamma, uv, b->cap);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return bfail(FMM2D_CUDA_ERROR, std::string("batch launch: ") + cudaGetErrorString(e));
    }
    if (e2 != cudaSuccess)
        return bfail(FMM2D_CUDA_ERROR, std::string("end capture: ") + cudaGetErrorString(e2));
    b->graph = graph;
    BCK(cudaGraphInstantiate(&b->exec, graph, 0));
    size_t count = 0;
    BCK(cudaGraphGetNodes(graph, nullptr, &count));
    std::vector<cudaGraphNode_t> nodes(count);
    BCK(cudaGraphGetNodes(graph, nodes.data(), &count));
    int kernels = 0;
    for (size_t i = 0; i < count; ++i) {
        cudaGraphNodeType ty;
        BCK(cudaGraphNodeGetType(nodes[i], &ty));
        kernels += ty == cudaGraphNodeTypeKernel;
    }
    b->kernel_nodes = kernels;
    b->g_xy = xy;
    b->g_gamma = gamma;
    b->g_uv = uv;
    return FMM2D_OK;
}

bool valid_instance(const fmm2d_instance& in, std::string* why) {
    if (in.n < 0) return *why = "instance n < 0", false;
    if (in.p < 1 || in.p > kMaxP) return *why = "instance p must be in [1, 32]", false;
    if (in.L < 0 || in.L > kMaxL) return *why = "instance L must be in [0, 12]", false;
    if (!(in.sigma > 0.0) || !std::isfinite(in.sigma)) return *why = "instance sigma", false;
    if (!(in.W > 0.0) || !std::isfinite(in.W) || !std::isfinite(in.x0) || !std::isfinite(in.y0))
        return *why = "instance root box", false;
    // the kernels correct the ring of leaves at Chebyshev distance 2 only
    if (!(in.cutoff >= 0.0) || !std::isfinite(in.cutoff) ||
        (in.L >= 2 && in.cutoff > 2.0 * in.W / ldexp(1.0, in.L)))
        return *why = "instance cutoff must be in [0, 2 W / 2^L]", false;
    return true;
}

// (Re)build the tensor-core M2L classes with the given operator stages and
// tile policy: the instances with L >= 2 grouped by Pk = p rounded up to 4.
cudaError_t build_tc_classes(fmm2d_batch_plan* b, int b_stages, int policy) {
    for (auto& c : b->tc) m2l_tc_batch_destroy(&c);
    b->tc.clear();
    for (int Pk = 4; Pk <= kMaxP; Pk += 4) {
        std::vector<int> ids;
        for (int i = 0; i < b->count; ++i) {
            const Geometry& g = b->inst[i].g;
            if (g.L >= 2 && ((g.p + 3) & ~3) == Pk) ids.push_back(i);
        }
        if (ids.empty()) continue;
        const int P = Pk <= 16 ? 16 : 32;
        const int c = class_of(P);
        const int64_t per = (int64_t)P * P * 2;
        M2LTcBatchClass cls;
        cudaError_t e = m2l_tc_batch_create(b->inst.data(), ids.data(), (int)ids.size(), Pk, P,
                                            b->tab64[c] + 8 * per, b_stages, policy, &cls,
                                            b->cap);
        if (e != cudaSuccess) return e;
        b->tc.push_back(cls);
    }
    b->tc_b_stages = b_stages;
    b->tc_policy = policy;
    return cudaSuccess;
}

}  // namespace

extern "C" {

const char* fmm2d_batch_last_error(void) { return g_batch_error.c_str(); }

fmm2d_status fmm2d_batch_plan_create(fmm2d_batch_plan** out, int count,
                                     const fmm2d_instance* in) {
    return fmm2d_batch_plan_create_ex(out, count, in, FMM2D_FP32);
}

fmm2d_status fmm2d_batch_plan_create_ex(fmm2d_batch_plan** out, int count,
                                        const fmm2d_instance* in, int precision) {
    if (!out) return bfail(FMM2D_INVALID_ARG, "null output pointer");
    if (precision != FMM2D_FP32 && precision != FMM2D_FP32_TC)
        return bfail(FMM2D_INVALID_ARG, "batch precision must be FMM2D_FP32 or FMM2D_FP32_TC");
    *out = nullptr;
    if (count < 1 || !in) return bfail(FMM2D_INVALID_ARG, "count must be >= 1 with instances");
    std::string why;
    int64_t ntotal = 0;
    uint64_t nleaf = 0;
    for (int i = 0; i < count; ++i) {
        if (!valid_instance(in[i], &why))
            return bfail(FMM2D_INVALID_ARG, why + " (instance " + std::to_string(i) + ")");
        ntotal += in[i].n;
        nleaf += 1ull << (2 * in[i].L);
    }
    if (ntotal >= (int64_t)0xFFFFFFFF || nleaf >= 0xFFFFFFFFull)
        return bfail(FMM2D_INVALID_ARG, "batch too large for 32-bit keys and indices");

    auto* b = new fmm2d_batch_plan();
    auto cleanup = [&](fmm2d_status st) {
        fmm2d_batch_plan_destroy(b);
        return st;
    };
    cudaGetDevice(&b->device);
    b->count = count;
    b->precision = precision;
    b->ntotal = ntotal;
    b->nleaf_total = (uint32_t)nleaf;
    while ((1ull << b->key_bits) < nleaf) ++b->key_bits;
    b->inst.resize(count);
    std::vector<int64_t> offsets(count + 1, 0);
    int64_t exp_total = 0, off = 0;
    uint32_t leaf_base = 0;
    for (int i = 0; i < count; ++i) {
        BatchInst& bi = b->inst[i];
        Geometry& g = bi.g;
        g = Geometry{};
        g.x0 = in[i].x0;
        g.y0 = in[i].y0;
        g.W = in[i].W;
        g.L = in[i].L;
        g.p = in[i].p;
        g.P = in[i].p <= 16 ? 16 : 32;
        int64_t acc = 0;
        for (int l = 2; l <= g.L + 1; ++l) {
            g.level_base[l] = acc;
            if (l <= g.L) acc += (int64_t)1 << (2 * l);
        }
        g.nboxes = acc;
        g.scale = ldexp(1.0, g.L) / g.W;
        g.cutoff = g.L >= 2 ? in[i].cutoff : 0.0;  // Sec. 4.1 (0: the plain 3x3 rule)
        if (g.cutoff > 0.0) b->any_cutoff = true;
        bi.offset = off;
        bi.n = in[i].n;
        bi.exp_off = exp_total;
        bi.leaf_base = leaf_base;
        bi.sigma = in[i].sigma;
        offsets[i] = off;
        off += in[i].n;
        exp_total += (acc * 2 * g.P + 31) / 32 * 32;
        leaf_base += 1u << (2 * g.L);
        b->max_L = std::max(b->max_L, g.L);
        if (g.L >= 2) b->has_class[class_of(g.P)] = true;
    }
    offsets[count] = off;

    // work lists (host)
    std::vector<int32_t> quad_inst[2], m2l_inst[2], lvl_m2m[2][kMaxL + 1], lvl_l2l[2][kMaxL + 1];
    std::vector<uint32_t> quad_local[2];
    std::vector<int64_t> m2l_prefix[2];
    for (int c = 0; c < 2; ++c) m2l_prefix[c].push_back(0);
    std::vector<int32_t> leaf_inst(nleaf);
    for (int i = 0; i < count; ++i) {
        const Geometry& g = b->inst[i].g;
        for (uint32_t k = 0; k < (1u << (2 * g.L)); ++k) leaf_inst[b->inst[i].leaf_base + k] = i;
        if (g.L < 2) continue;
        int c = class_of(g.P);
        m2l_inst[c].push_back(i);
        m2l_prefix[c].push_back(m2l_prefix[c].back() + g.nboxes);
        for (int l = 2; l <= g.L - 2; ++l) lvl_m2m[c][l].push_back(i);
        for (int l = 3; l <= g.L - 1; ++l) lvl_l2l[c][l].push_back(i);
    }
    // P2M parent boxes per class: first those of the instances with at most 32
    // particles per leaf on average (one warp per box), then the others
    int64_t nquads_warp[2] = {0, 0};
    for (int pass = 0; pass < 2; ++pass)
        for (int i = 0; i < count; ++i) {
            const Geometry& g = b->inst[i].g;
            if (g.L < 2 || near_lane_path(b->inst[i].n, g.L) != (pass == 0)) continue;
            const int c = class_of(g.P);
            for (uint32_t q = 0; q < (1u << (2 * (g.L - 1))); ++q) {
                quad_inst[c].push_back(i);
                quad_local[c].push_back(q);
            }
            if (pass == 0) nquads_warp[c] = (int64_t)quad_inst[c].size();
        }
    // one device allocation
    int64_t nmax = ntotal > 0 ? ntotal : 1;
    int64_t nblocks = (nmax + kSortTile - 1) / kSortTile;
    size_t tab_count[2] = {(size_t)(8 + kOffsetSlots) * 16 * 16 * 2,
                           (size_t)(8 + kOffsetSlots) * 32 * 32 * 2};
    std::vector<size_t> sizes = {
        a256(sizeof(BatchInst) * count), a256(8 * (count + 1)), a256(batch_key_params_bytes(count)),
        a256(batch_near_bytes(count)), a256(4 * nleaf), 256,  // counter
        256,                                                                   // status
        a256(4 * nmax), a256(4 * nmax), a256(4 * nmax), a256(4 * nmax), a256(4 * nmax),
        a256(4 * ((size_t)kRadix * nblocks + kRadix)), a256(4 * (nleaf + 1)), a256(16 * nmax),
        a256(4 * (size_t)std::max<int64_t>(exp_total, 1)),
        a256(4 * (size_t)std::max<int64_t>(exp_total, 1)), a256(8 * tab_count[0]),
        a256(8 * tab_count[1]), a256(4 * tab_count[0]), a256(4 * tab_count[1]),
        a256(8 * 65 * 65)};  // binomial scratch
    // leaf centres per instance and axis index (FP32 hi/lo pairs, formed once
    // with the single plans' FP64 arithmetic: the same bits, and no FP64 in
    // the kernels that read them)
    std::vector<int64_t> centre_off(count + 1, 0);
    for (int i = 0; i < count; ++i)
        centre_off[i + 1] = centre_off[i] + ((int64_t)1 << b->inst[i].g.L);
    sizes.push_back(a256(sizeof(float4) * (size_t)centre_off[count]));
    // ring strips of the cutoff: 4 records per particle, 4 counts per leaf
    const bool want_strips = b->any_cutoff && nmax < ((int64_t)1 << 30);
    sizes.push_back(a256(want_strips ? 16 * 4 * (size_t)nmax : 0));
    sizes.push_back(a256(want_strips ? 16 * (size_t)nleaf : 0));
    // the per-target-lane pass's queue, when an instance has sparse leaves
    std::vector<uint32_t> lane_win;  // each window once, in increasing order
    for (int i = 0; i < count; ++i) {
        const BatchInst& bi = b->inst[i];
        if (bi.n == 0 || !near_lane_path(bi.n, bi.g.L)) continue;
        const uint32_t w0 = (uint32_t)(offsets[i] / 32);
        const uint32_t w1 = (uint32_t)((offsets[i] + bi.n - 1) / 32);
        for (uint32_t w = lane_win.empty() ? w0 : std::max(w0, lane_win.back() + 1); w <= w1; ++w)
            lane_win.push_back(w);
    }
    sizes.push_back(a256(4 * lane_win.size()));
    size_t lists_bytes = 0;
    for (int c = 0; c < 2; ++c) {
        lists_bytes += a256(4 * quad_inst[c].size() + 4) * 2 + a256(4 * m2l_inst[c].size() + 4) +
                       a256(8 * m2l_prefix[c].size());
        for (int l = 0; l <= kMaxL; ++l)
            lists_bytes += a256(4 * lvl_m2m[c][l].size() + 4) + a256(4 * lvl_l2l[c][l].size() + 4);
    }
    size_t total = lists_bytes;
    for (size_t v : sizes) total += v;
    cudaError_t e = cudaMalloc(&b->ws, total);
    if (e != cudaSuccess) return cleanup(bfail(FMM2D_OUT_OF_MEMORY, "batch workspace"));
    char* p = static_cast<char*>(b->ws);
    auto take = [&](size_t bytes) {
        char* r = p;
        p += bytes;
        return r;
    };
    size_t k = 0;
    b->d_inst = (BatchInst*)take(sizes[k++]);
    b->d_offsets = (int64_t*)take(sizes[k++]);
    b->d_keyparams = take(sizes[k++]);
    b->d_near = take(sizes[k++]);
    b->d_leaf_inst = (int32_t*)take(sizes[k++]);
    b->d_counter = (uint32_t*)take(sizes[k++]);
    b->d_status = (int*)take(sizes[k++]);
    b->sb.keys[0] = (uint32_t*)take(sizes[k++]);
    b->sb.keys[1] = (uint32_t*)take(sizes[k++]);
    b->sb.vals[0] = (uint32_t*)take(sizes[k++]);
    b->sb.vals[1] = (uint32_t*)take(sizes[k++]);
    b->sb.perm = (uint32_t*)take(sizes[k++]);
    b->sb.hist = (uint32_t*)take(sizes[k++]);
    b->sb.leaf_start = (uint32_t*)take(sizes[k++]);
    b->particles = take(sizes[k++]);
    b->me = (float*)take(sizes[k++]);
    b->le = (float*)take(sizes[k++]);
    b->tab64[0] = (double*)take(sizes[k++]);
    b->tab64[1] = (double*)take(sizes[k++]);
    b->tab32[0] = (float*)take(sizes[k++]);
    b->tab32[1] = (float*)take(sizes[k++]);
    double* binom = (double*)take(sizes[k++]);
    float4* centres = (float4*)take(sizes[k++]);
    for (int i = 0; i < count; ++i) b->inst[i].g.centre_tab = centres + centre_off[i];
    {
        float4* rec = (float4*)take(sizes[k++]);
        uint32_t* cnt = (uint32_t*)take(sizes[k++]);
        if (want_strips) b->strips = RingStrips{rec, cnt};
    }
    {
        uint32_t* q = (uint32_t*)take(sizes[k++]);
        if (!lane_win.empty()) {
            b->lane_win = q;
            b->lane_win_count = (uint32_t)lane_win.size();
        }
    }
    b->sb.status = b->d_status;

    e = cudaHostAlloc((void**)&b->h_status, sizeof(int), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cleanup(bfail(FMM2D_CUDA_ERROR, "batch stream / host memory"));
    cudaStream_t s = b->cap;
    auto up = [&](void* dst, const void* src, size_t bytes) {
        return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
    };
    for (int i = 0; i < count && e == cudaSuccess; ++i)
        e = launch_centre_table(b->inst[i].g, centres + centre_off[i], s);
    if (e == cudaSuccess) e = up(b->d_inst, b->inst.data(), sizeof(BatchInst) * count);
    if (e == cudaSuccess) e = up(b->d_offsets, offsets.data(), 8 * (count + 1));
    if (e == cudaSuccess) e = up(b->d_leaf_inst, leaf_inst.data(), 4 * nleaf);
    if (e == cudaSuccess) e = up(b->lane_win, lane_win.data(), 4 * (size_t)b->lane_win_count);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_status, 0, sizeof(int), s);
    for (int c = 0; c < 2 && e == cudaSuccess; ++c) {
        BatchLists& bl = b->lists[c];
        int32_t* qi = (int32_t*)take(a256(4 * quad_inst[c].size() + 4));
        uint32_t* ql = (uint32_t*)take(a256(4 * quad_local[c].size() + 4));
        int32_t* mi = (int32_t*)take(a256(4 * m2l_inst[c].size() + 4));
        int64_t* mp = (int64_t*)take(a256(8 * m2l_prefix[c].size()));
        e = up(qi, quad_inst[c].data(), 4 * quad_inst[c].size());
        if (e == cudaSuccess) e = up(ql, quad_local[c].data(), 4 * quad_local[c].size());
        if (e == cudaSuccess) e = up(mi, m2l_inst[c].data(), 4 * m2l_inst[c].size());
        if (e == cudaSuccess) e = up(mp, m2l_prefix[c].data(), 8 * m2l_prefix[c].size());
        bl.quad_inst = qi;
        bl.quad_local = ql;
        bl.nquads = (int64_t)quad_inst[c].size();
        bl.nquads_warp = nquads_warp[c];
        bl.m2l_inst = mi;
        bl.m2l_prefix = mp;
        bl.m2l_count = (int)m2l_inst[c].size();
        bl.m2l_total = m2l_prefix[c].back();
        for (int l = 0; l <= kMaxL && e == cudaSuccess; ++l) {
            int32_t* a = (int32_t*)take(a256(4 * lvl_m2m[c][l].size() + 4));
            int32_t* d = (int32_t*)take(a256(4 * lvl_l2l[c][l].size() + 4));
            e = up(a, lvl_m2m[c][l].data(), 4 * lvl_m2m[c][l].size());
            if (e == cudaSuccess) e = up(d, lvl_l2l[c][l].data(), 4 * lvl_l2l[c][l].size());
            bl.m2m_inst[l] = a;
            bl.m2m_count[l] = (int)lvl_m2m[c][l].size();
            bl.l2l_inst[l] = d;
            bl.l2l_count[l] = (int)lvl_l2l[c][l].size();
        }
    }
    for (int c = 0; c < 2 && e == cudaSuccess; ++c) {
        int P = c ? 32 : 16;
        int64_t per = (int64_t)P * P * 2;
        // full tables (p = P); every kernel masks coefficients >= the instance's p
        e = launch_build_tables(P, P, b->tab64[c], b->tab64[c] + 4 * per, b->tab64[c] + 8 * per,
                                binom, s);
        if (e == cudaSuccess) e = launch_tables_to_f32(b->tab64[c], b->tab32[c], tab_count[c], s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = batch_key_params(b->inst.data(), count, b->d_keyparams, s);
    if (e == cudaSuccess) e = batch_near_fill(b->inst.data(), count, b->d_near, s);
    if (e == cudaSuccess && precision == FMM2D_FP32_TC) {
        static bool configured = false;
        if (!configured) {
            e = m2l_tc_configure();
            configured = e == cudaSuccess;
        }
        if (e == cudaSuccess) e = build_tc_classes(b, 0, 0);
    }
    if (e != cudaSuccess)
        return cleanup(bfail(FMM2D_CUDA_ERROR, std::string("batch set-up: ") +
                                                   cudaGetErrorString(e)));
    *out = b;
    return FMM2D_OK;
}

void fmm2d_batch_plan_destroy(fmm2d_batch_plan* b) {
    if (!b) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    drop_batch_graph(b);
    for (auto& c : b->tc) m2l_tc_batch_destroy(&c);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->h_status) cudaFreeHost(b->h_status);
    if (b->ws) cudaFree(b->ws);
    cudaSetDevice(cur);
    delete b;
}

fmm2d_status fmm2d_batch_velocity(fmm2d_batch_plan* b, const float* xy, const float* gamma,
                                  float* uv, cudaStream_t stream) {
    if (!b) return bfail(FMM2D_INVALID_ARG, "null plan");
    if (b->ntotal > 0 && (!xy || !gamma || !uv)) return bfail(FMM2D_INVALID_ARG, "null buffer");
    if (!b->exec || b->g_xy != xy || b->g_gamma != gamma || b->g_uv != uv) {
        fmm2d_status st = record_batch_graph(b, xy, gamma, uv);
        if (st != FMM2D_OK) return st;
    }
    BCK(cudaGraphLaunch(b->exec, stream));
    return FMM2D_OK;
}

fmm2d_status fmm2d_batch_check(fmm2d_batch_plan* b, cudaStream_t stream) {
    if (!b) return bfail(FMM2D_INVALID_ARG, "null plan");
    BCK(cudaMemcpyAsync(b->h_status, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, stream));
    BCK(cudaMemsetAsync(b->d_status, 0, sizeof(int), stream));
    BCK(cudaStreamSynchronize(stream));
    int f = *b->h_status;
    if (f & (1 << FMM2D_NONFINITE)) return bfail(FMM2D_NONFINITE, "non-finite input");
    if (f & (1 << FMM2D_OUT_OF_DOMAIN)) return bfail(FMM2D_OUT_OF_DOMAIN, "outside a root box");
    if (f & (1 << FMM2D_INVALID_ARG)) return bfail(FMM2D_INVALID_ARG, "invalid sample index");
    if (f & (1 << FMM2D_TIMEOUT)) return bfail(FMM2D_TIMEOUT, "device wait timed out");
    return FMM2D_OK;
}

fmm2d_status fmm2d_batch_autotune(fmm2d_batch_plan* b, const float* xy, const float* gamma,
                                  float* uv, cudaStream_t stream) {
    if (!b) return bfail(FMM2D_INVALID_ARG, "null plan");
    if (b->ntotal > 0 && (!xy || !gamma || !uv)) return bfail(FMM2D_INVALID_ARG, "null buffer");
    cudaStream_t s = b->cap;
    BCK(cudaStreamSynchronize(stream));
    // one full evaluation so that every step sees real data
    BCK(enqueue_batch(b, xy, gamma, uv, s));
    cudaEvent_t t0, t1;
    BCK(cudaEventCreate(&t0));
    BCK(cudaEventCreate(&t1));
    // best of three timings; a candidate whose launch fails is never chosen
    auto time_it = [&](auto&& launch) -> float {
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(t0, s);
            cudaError_t le = launch();
            cudaEventRecord(t1, s);
            cudaEventSynchronize(t1);
            if (le != cudaSuccess || cudaGetLastError() != cudaSuccess) return 1e30f;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, t0, t1);
            best = std::min(best, ms);
        }
        return best;
    };
    // near field: persistent CTAs per SM (shared memory allows at most 6)
    float best = 1e30f;
    int best_cps = b->p2p_ctas_per_sm;
    for (int cps : {2, 3, 4, 5, 6}) {
        float ms = time_it([&] {
            return launch_batch_p2p(b->d_inst, b->d_near, b->d_leaf_inst, (uint32_t)b->ntotal,
                                    b->d_counter, cps, b->particles,
                                    b->sb.keys[sort_passes(b->key_bits) & 1],
                                    b->sb.leaf_start, b->le,
                                    b->has_class[0] ? tab_l2l(b, 0) : nullptr,
                                    b->has_class[1] ? tab_l2l(b, 1) : nullptr, uv,
                                    b->any_cutoff, b->strips, b->nleaf_total, b->lane_win,
                                    b->lane_win_count, s);
        });
        if (ms < best) {
            best = ms;
            best_cps = cps;
        }
    }
    // FP32_TC: the tensor-core M2L's shapes -- operator stages in flight
    // (2, 3, 4 or as many as shared memory holds) and the tile policy (the
    // fewest tiles, or the widest rows) -- timed over every class
    if (b->precision == FMM2D_FP32_TC) {
        float tbest = 1e30f;
        int bst = 0, bpol = 0;
        for (int pol : {0, 1})
            for (int st : {2, 3, 4, 0}) {
                if (build_tc_classes(b, st, pol) != cudaSuccess) continue;
                float ms = time_it([&] {
                    cudaError_t r = cudaSuccess;
                    for (const M2LTcBatchClass& c : b->tc)
                        if (r == cudaSuccess)
                            r = launch_m2l_tc_batch(c, b->d_inst, b->me, b->le, b->d_status, 0,
                                                    s);
                    return r;
                });
                if (ms < tbest) {
                    tbest = ms;
                    bst = st;
                    bpol = pol;
                }
            }
        if (build_tc_classes(b, bst, bpol) != cudaSuccess)
            return bfail(FMM2D_CUDA_ERROR, "tensor-core M2L classes");
    }
    // M2L: block size of the box-parallel contraction
    best = 1e30f;
    int best_threads = b->m2l_threads;
    for (int th : {64, 128, 256}) {  // the kernel is compiled for at most 256 threads
        float ms = time_it([&] {
            cudaError_t r = cudaSuccess;
            for (int c = 0; c < 2 && r == cudaSuccess; ++c)
                if (b->has_class[c])
                    r = launch_batch_m2l(b->d_inst, b->lists[c], c ? 32 : 16, th, tab_m2l(b, c),
                                         b->me, b->le, s);
            return r;
        });
        if (ms < best) {
            best = ms;
            best_threads = th;
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    BCK(cudaGetLastError());
    b->p2p_ctas_per_sm = best_cps;
    b->m2l_threads = best_threads;
    drop_batch_graph(b);
    // leave the caller's output consistent with the chosen shapes
    BCK(enqueue_batch(b, xy, gamma, uv, s));
    BCK(cudaStreamSynchronize(s));
    return FMM2D_OK;
}

fmm2d_status fmm2d_batch_direct_sampled(fmm2d_batch_plan* b, int kernel, const float* xy,
                                        const float* gamma, int64_t s_count,
                                        const int64_t* targets, double* uv_ref,
                                        cudaStream_t stream) {
    if (!b) return bfail(FMM2D_INVALID_ARG, "null plan");
    if (kernel != 0 && kernel != 1) return bfail(FMM2D_INVALID_ARG, "kernel must be 0 or 1");
    if (s_count < 0 || (s_count > 0 && (!xy || !gamma || !targets || !uv_ref)))
        return bfail(FMM2D_INVALID_ARG, "bad sample arguments");
    BCK(launch_batch_direct(b->d_inst, b->d_offsets, b->count, kernel, xy, gamma, s_count, targets,
                            uv_ref, b->d_status, stream));
    return FMM2D_OK;
}

fmm2d_status fmm2d_batch_error_stats(fmm2d_batch_plan* b, const float* xy, const float* uv,
                                     int64_t s_count, const int64_t* targets,
                                     const double* uv_ref, double* stats, double* leaf_err,
                                     cudaStream_t stream) {
    if (!b) return bfail(FMM2D_INVALID_ARG, "null plan");
    if (!stats || s_count < 0 || (s_count > 0 && (!xy || !uv || !targets || !uv_ref)))
        return bfail(FMM2D_INVALID_ARG, "bad statistics arguments");
    BCK(launch_batch_error(b->d_inst, b->d_offsets, b->count, xy, uv, s_count, targets, uv_ref,
                           stats, leaf_err, b->nleaf_total, b->d_status, stream));
    return FMM2D_OK;
}

fmm2d_status fmm2d_batch_info(const fmm2d_batch_plan* b, int64_t* n_total, int64_t* leaves_total,
                              int* kernels_per_call, int* p2p_ctas_per_sm, int* m2l_threads) {
    if (!b) return bfail(FMM2D_INVALID_ARG, "null plan");
    if (n_total) *n_total = b->ntotal;
    if (leaves_total) *leaves_total = b->nleaf_total;
    if (kernels_per_call) *kernels_per_call = b->kernel_nodes;
    if (p2p_ctas_per_sm) *p2p_ctas_per_sm = b->p2p_ctas_per_sm;
    if (m2l_threads) *m2l_threads = b->m2l_threads;
    return FMM2D_OK;
}

fmm2d_status fmm2d_batch_profile(fmm2d_batch_plan* b, const float* xy, const float* gamma,
                                 float* uv, double* ms, cudaStream_t stream) {
    if (!b || !ms) return bfail(FMM2D_INVALID_ARG, "null argument");
    if (b->ntotal > 0 && (!xy || !gamma || !uv)) return bfail(FMM2D_INVALID_ARG, "null buffer");
    cudaEvent_t ev[6] = {};
    for (auto& x : ev) BCK(cudaEventCreate(&x));
    BCK(cudaStreamSynchronize(stream));
    cudaError_t e = enqueue_batch(b, xy, gamma, uv, b->cap, ev);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->cap);
    for (int k = 0; k < 5 && e == cudaSuccess; ++k) {
        float t = 0.f;
        e = cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
        ms[k] = t;
    }
    for (auto& x : ev) cudaEventDestroy(x);
    BCK(e);
    return FMM2D_OK;
}

fmm2d_status fmm2d_batch_info_tc(const fmm2d_batch_plan* b, int* classes, int* tiles,
                                 int* b_stages, int* tile_policy) {
    if (!b) return bfail(FMM2D_INVALID_ARG, "null plan");
    int t = 0;
    for (const M2LTcBatchClass& c : b->tc) t += c.cfg.ntiles;
    if (classes) *classes = (int)b->tc.size();
    if (tiles) *tiles = t;
    if (b_stages) *b_stages = b->tc.empty() ? 0 : b->tc[0].cfg.b_stages;
    if (tile_policy) *tile_policy = b->tc_policy;
    return FMM2D_OK;
}

fmm2d_status fmm2d_batch_tree_debug(fmm2d_batch_plan* b, uint32_t* keys, uint32_t* perm,
                                    uint32_t* leaf_start, cudaStream_t stream) {
    if (!b) return bfail(FMM2D_INVALID_ARG, "null plan");
    int passes = sort_passes(b->key_bits);
    if (keys && b->ntotal > 0)
        BCK(cudaMemcpyAsync(keys, b->sb.keys[passes & 1], 4 * b->ntotal, cudaMemcpyDeviceToDevice,
                            stream));
    if (perm && b->ntotal > 0)
        BCK(cudaMemcpyAsync(perm, b->sb.perm, 4 * b->ntotal, cudaMemcpyDeviceToDevice, stream));
    if (leaf_start)
        BCK(cudaMemcpyAsync(leaf_start, b->sb.leaf_start, 4 * ((size_t)b->nleaf_total + 1),
                            cudaMemcpyDeviceToDevice, stream));
    return FMM2D_OK;
}

}  // extern "C"
