// Upward sweep (Sec. 3.1, Fig. 3): P2M at the leaves, then M2M for levels
// L-1 .. 2.  Expansions are box-size scaled (see tables.cu):
//   P2M  a~_m = sum_{i in leaf} c_i zeta_i^m,  c_i = -j Gamma_i / 2pi,
//        zeta_i = (z_i - z_leaf) / s_leaf                          (Eq. 20-21)
//   M2M  parent b~_n = sum_quadrants sum_{k<=n} M2M[q]_{nk} a~_k(child)  (Sec. 3.3.2)
// Launches: the P2M kernel runs one CTA per parent box (four warps, one per
// child leaf) and also forms the parent's expansion at level L-1 from the
// four children in shared memory.  Levels L-2 .. 5 take one launch each;
// levels 4 .. 2 (at most 336 boxes) run in one single-CTA launch with a
// barrier between levels.  The 4-quadrant M2M table is staged in shared
// memory by every kernel that loops over it.
// The leaf centre is formed once per warp in FP64 and held as an FP32 hi/lo
// pair, so that zeta = ((x - c_hi) - c_lo) / s is accurate to FP32 relative
// to the leaf size and the expansion is centred where the translation
// tables assume.
#include "fmm2d_internal.cuh"

namespace fmm2d {
namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr int kTopLevel = 2;  // levels <= kTopLevel run in the single-CTA kernel

// P2M of one leaf by one warp: lanes stride over the leaf's particles,
// accumulate all coefficients, then reduce across the warp.  Writes the
// leaf's expansion to me and a copy to kid (2 PMAX reals) for the parent's
// translation.  Leaf keys are offset by leaf_base in leaf_start (zero for a
// single evaluation).
template <typename R, int PMAX>
__device__ __forceinline__ void p2m_leaf(const typename ParticleOf<R>::type* __restrict__ sp,
                                         const uint32_t* __restrict__ leaf_start,
                                         uint32_t leaf_base, uint32_t leaf, const Geometry& g,
                                         R* __restrict__ me, R* kid) {
    using C = typename Cplx<R>::T;
    const int lane = threadIdx.x & 31;
    const uint32_t ix = morton_compact(leaf), iy = morton_compact(leaf >> 1);
    const uint32_t b = leaf_start[leaf_base + leaf], e = leaf_start[leaf_base + leaf + 1];
    const double scale = g.scale;
    R cxh, cxl, cyh, cyl;
    if (sizeof(R) == 4) {
        float a0, a1, a2, a3;
        leaf_centre_hilo(g, ix, iy, &a0, &a1, &a2, &a3);
        cxh = a0;
        cxl = a1;
        cyh = a2;
        cyl = a3;
    } else {
        cxh = (R)(g.x0 + ((double)ix + 0.5) / scale);
        cyh = (R)(g.y0 + ((double)iy + 0.5) / scale);
        cxl = cyl = R(0);
    }
    const R inv_s = (R)scale;
    const R inv2pi = (R)(1.0 / kTwoPi);
    C acc[PMAX];
#pragma unroll
    for (int m = 0; m < PMAX; ++m) acc[m] = cmake<C>(R(0), R(0));
    for (uint32_t r = b + lane; r < e; r += 32) {
        auto q = sp[r];
        C zeta = cmake<C>(((q.x - cxh) - cxl) * inv_s, ((q.y - cyh) - cyl) * inv_s);
        C pw = cmake<C>(R(0), -q.z * inv2pi);  // c_i = -j Gamma / 2pi
#pragma unroll
        for (int m = 0; m < PMAX; ++m) {
            if (m < g.p) {
                acc[m].x += pw.x;
                acc[m].y += pw.y;
                pw = cmul(pw, zeta);
            }
        }
    }
    // Butterfly reduce-scatter of the warp's 2 PMAX partial sums: at each of
    // five steps a lane keeps half of its live values and adds its partner's
    // copy of that half.  Lane l ends with the warp totals of reals
    // [l W, (l + 1) W), W = 2 PMAX / 32: one real for PMAX = 16, one complex
    // coefficient for PMAX = 32.
    constexpr int N = 2 * PMAX;
    R v[N];
#pragma unroll
    for (int m = 0; m < PMAX; ++m) {
        v[2 * m] = acc[m].x;
        v[2 * m + 1] = acc[m].y;
    }
#pragma unroll
    for (int step = 0; step < 5; ++step) {
        const int o = 16 >> step;
        const int half = (N >> step) >> 1;
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const R send = upper ? v[i] : v[i + half];
            const R keep = upper ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    constexpr int W = N / 32;
    R* dst = me + box_slot(g.level_base, g.L, ix, iy) * (2 * g.P);
#pragma unroll
    for (int j = 0; j < W; ++j) {
        dst[lane * W + j] = v[j];
        kid[lane * W + j] = v[j];
    }
}

// One warp per leaf, four sibling leaves per CTA (p2m_leaf), then the parent.
// `quad` is the parent box (Morton key at level L-1).
template <typename R, int PMAX>
__device__ __forceinline__ void p2m_quad(const typename ParticleOf<R>::type* __restrict__ sp,
                                         const uint32_t* __restrict__ leaf_start,
                                         uint32_t leaf_base, uint32_t quad, const Geometry& g,
                                         const R* __restrict__ m2m, bool fuse_parent,
                                         R* __restrict__ me,
                                         typename Cplx<R>::T (*child_me)[PMAX],
                                         typename Cplx<R>::T (*part)[PMAX]) {
    using C = typename Cplx<R>::T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t leaf = quad * 4 + warp;
    const uint32_t ix = morton_compact(leaf), iy = morton_compact(leaf >> 1);
    p2m_leaf<R, PMAX>(sp, leaf_start, leaf_base, leaf, g, me,
                      reinterpret_cast<R*>(child_me[warp]));
    if (!fuse_parent) return;  // uniform over the CTA
    __syncthreads();
    // parent at level L-1: warp q translates its own child quadrant q (one
    // chain of P steps per warp instead of one of 4 P in a single warp, which
    // held each CTA for most of its time), then warp 0 adds the four
    // contributions in quadrant order
    if (lane < g.P) {
        const C* tq = reinterpret_cast<const C*>(m2m) + (int64_t)warp * g.P * g.P;
        C acc_q = cmake<C>(R(0), R(0));
#pragma unroll
        for (int k = 0; k < PMAX; ++k)
            if (k < g.P) acc_q = cfma(tq[k * g.P + lane], child_me[warp][k], acc_q);
        part[warp][lane] = acc_q;
    }
    __syncthreads();
    if (warp == 0 && lane < g.P) {
        C out = part[0][lane];
        for (int q = 1; q < 4; ++q) out = cmake<C>(out.x + part[q][lane].x, out.y + part[q][lane].y);
        if (lane >= g.p) out = cmake<C>(R(0), R(0));
        reinterpret_cast<C*>(me + box_slot(g.level_base, g.L - 1, ix >> 1, iy >> 1) *
                                      (2 * g.P))[lane] = out;
    }
}

template <typename R, int PMAX>
__global__ void __launch_bounds__(128)
p2m_kernel(const typename ParticleOf<R>::type* __restrict__ sp,
           const uint32_t* __restrict__ leaf_start, Geometry g, const R* __restrict__ m2m,
           bool fuse_parent, R* __restrict__ me) {
    __shared__ typename Cplx<R>::T child_me[4][PMAX], part[4][PMAX];
    p2m_quad<R, PMAX>(sp, leaf_start, 0, blockIdx.x, g, m2m, fuse_parent, me, child_me, part);
}

// One warp per parent box (batched instances of at most 32 particles per leaf
// on average, whose boxes are mostly sparse).  A sparse box, every child
// leaf holding at most kQuadSparse particles, is formed with eight lanes per
// child (child q in lanes 8q .. 8q + 7, its particle j in lane 8q + j)
// instead of a warp per child with most lanes idle; another box one child
// after the other (p2m_leaf).  Either way the expansions are p2m_quad's, bit
// for bit: in the sparse form a lane's one particle enters its coefficients
// as 0 + c zeta^m as there, and the sum over a child's eight lanes pairs
// lanes as the last three steps of p2m_quad's butterfly do (its first two
// steps only add the zeros of its empty lanes, exactly; no partial sum is
// -0, since each starts from +0).  The parent's translation runs the same
// chains (child q, coefficient n) and adds the four in quadrant order.
constexpr uint32_t kQuadSparse = 8;

template <int PMAX>
__device__ __forceinline__ void p2m_quad_warp(const float4* __restrict__ sp,
                                              const uint32_t* __restrict__ leaf_start,
                                              uint32_t leaf_base, uint32_t quad,
                                              const Geometry& g, const float* __restrict__ m2m,
                                              bool fuse_parent, float* __restrict__ me,
                                              float2 (*child_me)[PMAX], float2 (*part)[PMAX]) {
    const int lane = threadIdx.x & 31;
    const uint32_t* cnt = leaf_start + leaf_base + quad * 4;
    const uint32_t s0 = cnt[0], s1 = cnt[1], s2 = cnt[2], s3 = cnt[3], s4 = cnt[4];
    const bool sparse = s1 - s0 <= kQuadSparse && s2 - s1 <= kQuadSparse &&
                        s3 - s2 <= kQuadSparse && s4 - s3 <= kQuadSparse;
    __syncwarp();  // earlier readers of child_me are done
    if (sparse) {
        const int q = lane >> 3, j = lane & 7;
        const uint32_t leaf = quad * 4 + q;
        const uint32_t ix = morton_compact(leaf), iy = morton_compact(leaf >> 1);
        const uint32_t b = leaf_start[leaf_base + leaf], e = leaf_start[leaf_base + leaf + 1];
        float cxh, cxl, cyh, cyl;  // the lane's own leaf centre (no warp broadcast)
        if (g.centre_tab) {
            const float4 tx = g.centre_tab[ix], ty = g.centre_tab[iy];
            cxh = tx.x;
            cxl = tx.y;
            cyh = ty.z;
            cyl = ty.w;
        } else {
            centre_hilo_1d(g.x0, g.W, g.L, ix, &cxh, &cxl);
            centre_hilo_1d(g.y0, g.W, g.L, iy, &cyh, &cyl);
        }
        const float inv_s = (float)g.scale;
        const float inv2pi = (float)(1.0 / kTwoPi);
        float2 acc[PMAX];
#pragma unroll
        for (int m = 0; m < PMAX; ++m) acc[m] = make_float2(0.f, 0.f);
        if (b + j < e) {
            const float4 rec = sp[b + j];
            const float2 zeta =
                make_float2(((rec.x - cxh) - cxl) * inv_s, ((rec.y - cyh) - cyl) * inv_s);
            float2 pw = make_float2(0.f, -rec.z * inv2pi);  // c_i = -j Gamma / 2pi
#pragma unroll
            for (int m = 0; m < PMAX; ++m) {
                if (m < g.p) {
                    acc[m].x += pw.x;
                    acc[m].y += pw.y;
                    pw = cmul(pw, zeta);
                }
            }
        }
        // reduce-scatter over the child's eight lanes: lane j keeps reals
        // [j W8, (j + 1) W8) of the child's 2 PMAX
        constexpr int N = 2 * PMAX;
        float v[N];
#pragma unroll
        for (int m = 0; m < PMAX; ++m) {
            v[2 * m] = acc[m].x;
            v[2 * m + 1] = acc[m].y;
        }
#pragma unroll
        for (int step = 0; step < 3; ++step) {
            const int o = 4 >> step;
            const int half = (N >> step) >> 1;
            const bool upper = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < half; ++i) {
                const float send = upper ? v[i] : v[i + half];
                const float keep = upper ? v[i + half] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
        constexpr int W8 = N / 8;
        float* dst = me + box_slot(g.level_base, g.L, ix, iy) * (2 * g.P);
        float* kid = reinterpret_cast<float*>(child_me[q]);
#pragma unroll
        for (int t = 0; t < W8; ++t) {
            dst[j * W8 + t] = v[t];
            kid[j * W8 + t] = v[t];
        }
    } else {
        for (int q = 0; q < 4; ++q)
            p2m_leaf<float, PMAX>(sp, leaf_start, leaf_base, quad * 4 + q, g, me,
                                  reinterpret_cast<float*>(child_me[q]));
    }
    if (!fuse_parent) return;  // uniform over the warp
    __syncwarp();
    // parent at level L-1: the four children's translations, chain (cq, n).
    // An empty child's expansion is +0 throughout, and so is its chain's
    // result (each step adds +0): it is written without the chain.
    const unsigned empty = (s1 == s0 ? 1u : 0u) | (s2 == s1 ? 2u : 0u) | (s3 == s2 ? 4u : 0u) |
                           (s4 == s3 ? 8u : 0u);
    for (int c = lane; c < 4 * PMAX; c += 32) {
        const int cq = c / PMAX, n = c % PMAX;
        if (n < g.P && ((empty >> cq) & 1u)) {
            part[cq][n] = make_float2(0.f, 0.f);
        } else if (n < g.P) {
            const float2* tq = reinterpret_cast<const float2*>(m2m) + (int64_t)cq * g.P * g.P;
            float2 acc_q = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < PMAX; ++k)
                if (k < g.P) acc_q = cfma(tq[k * g.P + n], child_me[cq][k], acc_q);
            part[cq][n] = acc_q;
        }
    }
    __syncwarp();
    if (lane < g.P) {
        float2 out = part[0][lane];
        for (int k = 1; k < 4; ++k)
            out = make_float2(out.x + part[k][lane].x, out.y + part[k][lane].y);
        if (lane >= g.p) out = make_float2(0.f, 0.f);
        const uint32_t px = morton_compact(quad), py = morton_compact(quad >> 1);
        reinterpret_cast<float2*>(me + box_slot(g.level_base, g.L - 1, px, py) *
                                           (2 * g.P))[lane] = out;
    }
}

// Batched: one CTA per parent box of the class's other instances (the quads
// from nquads_warp on).
template <int PMAX>
__global__ void __launch_bounds__(128)
p2m_batch_kernel(const float4* __restrict__ sp, const uint32_t* __restrict__ leaf_start,
                 const BatchInst* __restrict__ inst, const int32_t* __restrict__ quad_inst,
                 const uint32_t* __restrict__ quad_local, int64_t first,
                 const float* __restrict__ m2m, float* __restrict__ me) {
    __shared__ float2 child_me[4][PMAX], part[4][PMAX];
    const int64_t qi = first + blockIdx.x;
    const BatchInst& b = inst[quad_inst[qi]];
    p2m_quad<float, PMAX>(sp, leaf_start, b.leaf_base, quad_local[qi], b.g, m2m, b.g.L >= 3,
                          me + b.exp_off, child_me, part);
}

// Batched, instances of at most 32 particles per leaf on average: one warp
// per parent box (p2m_quad_warp), four per CTA, quads [0, count).
template <int PMAX>
__global__ void __launch_bounds__(128)
p2m_batch_warp_kernel(const float4* __restrict__ sp, const uint32_t* __restrict__ leaf_start,
                      const BatchInst* __restrict__ inst, const int32_t* __restrict__ quad_inst,
                      const uint32_t* __restrict__ quad_local, int64_t count,
                      const float* __restrict__ m2m, float* __restrict__ me) {
    __shared__ float2 child_me[4][4][PMAX], part[4][4][PMAX];
    const int warp = threadIdx.x >> 5;
    const int64_t qi = (int64_t)blockIdx.x * 4 + warp;
    if (qi >= count) return;  // uniform over the warp
    const BatchInst& b = inst[quad_inst[qi]];
    p2m_quad_warp<PMAX>(sp, leaf_start, b.leaf_base, quad_local[qi], b.g, m2m, b.g.L >= 3,
                        me + b.exp_off, child_me[warp], part[warp]);
}

// M2M of one box with G lanes (lane n computes b~_n); children read by lane k
// and broadcast with shuffles, the table from shared memory.
template <typename R, int G>
__device__ __forceinline__ void m2m_box(const Geometry& g, int level, int64_t slot, bool valid,
                                        const typename Cplx<R>::T* tab, R* __restrict__ me) {
    using C = typename Cplx<R>::T;
    const int n = (threadIdx.x & 31) % G;
    uint32_t ix, iy;
    slot_box(g.level_base, level, slot, &ix, &iy);
    C acc = cmake<C>(R(0), R(0));
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t cx = 2 * ix + (q & 1), cy = 2 * iy + (q >> 1);
        const C* child = reinterpret_cast<const C*>(me + box_slot(g.level_base, level + 1, cx, cy) *
                                                             (2 * g.P));
        C a_own = child[n];
#pragma unroll
        for (int k = 0; k < G; ++k) {  // entries with k >= p are zero
            C ak = cshfl(a_own, k, G);
            acc = cfma(tab[(q * G + k) * G + n], ak, acc);
        }
    }
    if (n >= g.p) acc = cmake<C>(R(0), R(0));  // coefficients >= p stay zero
    if (valid) reinterpret_cast<C*>(me + slot * (2 * g.P))[n] = acc;
}

template <typename R, int G>
__device__ __forceinline__ void stage_table(const R* __restrict__ src, typename Cplx<R>::T* dst) {
    using C = typename Cplx<R>::T;
    const C* s = reinterpret_cast<const C*>(src);
    for (int i = threadIdx.x; i < 4 * G * G; i += blockDim.x) dst[i] = s[i];
    __syncthreads();
}

// One level, G lanes per box.
template <typename R, int G>
__global__ void __launch_bounds__(256)
m2m_level_kernel(Geometry g, int level, const R* __restrict__ m2m, R* __restrict__ me) {
    using C = typename Cplx<R>::T;
    __shared__ C tab[4 * G * G];
    stage_table<R, G>(m2m, tab);
    int64_t gid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
    int64_t nb = (int64_t)1 << (2 * level);
    bool valid = gid < nb;
    m2m_box<R, G>(g, level, g.level_base[level] + (valid ? gid : 0), valid, tab, me);
}

// Levels lhi .. 2 in one CTA, a barrier between levels.
template <typename R, int G>
__global__ void __launch_bounds__(1024)
m2m_top_kernel(Geometry g, int lhi, const R* __restrict__ m2m, R* __restrict__ me) {
    using C = typename Cplx<R>::T;
    __shared__ C tab[4 * G * G];
    stage_table<R, G>(m2m, tab);
    for (int level = lhi; level >= 2; --level) {
        int64_t nb = (int64_t)1 << (2 * level);
        for (int64_t base = 0; base < nb * G; base += blockDim.x) {
            int64_t gid = (base + threadIdx.x) / G;
            bool valid = gid < nb;
            m2m_box<R, G>(g, level, g.level_base[level] + (valid ? gid : 0), valid, tab, me);
        }
        __syncthreads();
    }
}

// Batched M2M at one level: G lanes per box, boxes of the listed instances.
template <int G>
__global__ void __launch_bounds__(256)
m2m_batch_kernel(const BatchInst* __restrict__ inst, const int32_t* __restrict__ list, int count,
                 int level, const float* __restrict__ m2m, float* __restrict__ me) {
    __shared__ float2 tab[4 * G * G];
    stage_table<float, G>(m2m, tab);
    const int64_t per = (int64_t)1 << (2 * level);
    const int64_t gid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
    const bool valid = gid < per * count;
    const int64_t g0 = valid ? gid : 0;
    const BatchInst& b = inst[list[g0 / per]];
    m2m_box<float, G>(b.g, level, b.g.level_base[level] + g0 % per, valid, tab, me + b.exp_off);
}

}  // namespace

cudaError_t launch_batch_p2m(const BatchInst* inst, const BatchLists& bl, int P,
                             const void* particles, const uint32_t* leaf_start, const float* m2m,
                             float* me, cudaStream_t s) {
    if (bl.nquads == 0) return cudaSuccess;
    const float4* sp = reinterpret_cast<const float4*>(particles);
    const int64_t nw = bl.nquads_warp, nc = bl.nquads - bl.nquads_warp;
    if (nw > 0) {
        const unsigned blocks = (unsigned)((nw + 3) / 4);
        if (P <= 16)
            p2m_batch_warp_kernel<16><<<blocks, 128, 0, s>>>(sp, leaf_start, inst, bl.quad_inst,
                                                             bl.quad_local, nw, m2m, me);
        else
            p2m_batch_warp_kernel<32><<<blocks, 128, 0, s>>>(sp, leaf_start, inst, bl.quad_inst,
                                                             bl.quad_local, nw, m2m, me);
    }
    if (nc > 0) {
        if (P <= 16)
            p2m_batch_kernel<16><<<(unsigned)nc, 128, 0, s>>>(sp, leaf_start, inst, bl.quad_inst,
                                                              bl.quad_local, nw, m2m, me);
        else
            p2m_batch_kernel<32><<<(unsigned)nc, 128, 0, s>>>(sp, leaf_start, inst, bl.quad_inst,
                                                              bl.quad_local, nw, m2m, me);
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_m2m(const BatchInst* inst, const BatchLists& bl, int P, int level,
                             const float* m2m, float* me, cudaStream_t s) {
    const int count = bl.m2m_count[level];
    if (count == 0) return cudaSuccess;
    const int64_t threads = ((int64_t)1 << (2 * level)) * count * P;
    const int blocks = (int)((threads + 255) / 256);
    if (P <= 16)
        m2m_batch_kernel<16><<<blocks, 256, 0, s>>>(inst, bl.m2m_inst[level], count, level, m2m,
                                                   me);
    else
        m2m_batch_kernel<32><<<blocks, 256, 0, s>>>(inst, bl.m2m_inst[level], count, level, m2m,
                                                   me);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_p2m(const Geometry& g, const void* particles, const uint32_t* leaf_start,
                       const Tables<R>& t, R* me, cudaStream_t s) {
    using P = typename ParticleOf<R>::type;
    int64_t nleaf = (int64_t)1 << (2 * g.L);
    int blocks = (int)(nleaf / 4);
    bool fuse = g.L >= 3;
    if (g.P <= 16)
        p2m_kernel<R, 16><<<blocks, 128, 0, s>>>(reinterpret_cast<const P*>(particles), leaf_start,
                                                 g, t.m2m, fuse, me);
    else
        p2m_kernel<R, 32><<<blocks, 128, 0, s>>>(reinterpret_cast<const P*>(particles), leaf_start,
                                                 g, t.m2m, fuse, me);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_m2m(const Geometry& g, const Tables<R>& t, R* me, cudaStream_t s) {
    // level L-1 was formed by the P2M kernel
    for (int level = g.L - 2; level > kTopLevel; --level) {
        int64_t threads = ((int64_t)1 << (2 * level)) * g.P;
        int blocks = (int)((threads + 255) / 256);
        if (g.P <= 16)
            m2m_level_kernel<R, 16><<<blocks, 256, 0, s>>>(g, level, t.m2m, me);
        else
            m2m_level_kernel<R, 32><<<blocks, 256, 0, s>>>(g, level, t.m2m, me);
    }
    int lhi = g.L - 2 < kTopLevel ? g.L - 2 : kTopLevel;
    if (lhi >= 2) {
        if (g.P <= 16)
            m2m_top_kernel<R, 16><<<1, 1024, 0, s>>>(g, lhi, t.m2m, me);
        else
            m2m_top_kernel<R, 32><<<1, 1024, 0, s>>>(g, lhi, t.m2m, me);
    }
    return cudaGetLastError();
}

template cudaError_t launch_p2m<float>(const Geometry&, const void*, const uint32_t*,
                                       const Tables<float>&, float*, cudaStream_t);
template cudaError_t launch_p2m<double>(const Geometry&, const void*, const uint32_t*,
                                        const Tables<double>&, double*, cudaStream_t);
template cudaError_t launch_m2m<float>(const Geometry&, const Tables<float>&, float*,
                                       cudaStream_t);
template cudaError_t launch_m2m<double>(const Geometry&, const Tables<double>&, double*,
                                        cudaStream_t);

}  // namespace fmm2d
