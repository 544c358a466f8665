// Downward sweep, L2L part (Sec. 3.3.3): for levels 3..L each box adds its
// parent's complete local expansion, re-expanded about its own centre:
//   L~_n(child) += sum_{k>=n} L2L[q]_{nk} L~_k(parent),  q = child quadrant.
// Level l runs after level l-1 is complete.  Levels 3 .. L-1 run two to a
// launch (a 4 x 4 block of boxes and then its 8 x 8 children per CTA), an
// odd last level alone; the leaf level is folded into the near-field or L2P
// kernel, which forms each leaf's expansion from its own M2L part and its
// parent's.  The
// 4-quadrant L2L table is staged in shared memory.
#include "fmm2d_internal.cuh"

namespace fmm2d {
namespace {

constexpr int kTopLevel = 2;  // the coarsest level with local expansions (M2L only)

template <typename R, int G>
__device__ __forceinline__ void l2l_box(const Geometry& g, int level, int64_t slot, bool valid,
                                        const typename Cplx<R>::T* tab, R* __restrict__ le) {
    using C = typename Cplx<R>::T;
    const int n = (threadIdx.x & 31) % G;
    uint32_t ix, iy;
    slot_box(g.level_base, level, slot, &ix, &iy);
    const int q = (int)(((iy & 1u) << 1) | (ix & 1u));
    const C* parent = reinterpret_cast<const C*>(
        le + box_slot(g.level_base, level - 1, ix >> 1, iy >> 1) * (2 * g.P));
    C l_own = parent[n];
    C acc = cmake<C>(R(0), R(0));
#pragma unroll
    for (int k = 0; k < G; ++k) {  // entries with k >= p or k < n are zero
        C lk = cshfl(l_own, k, G);
        acc = cfma(tab[(q * G + k) * G + n], lk, acc);
    }
    if (n >= g.p) acc = cmake<C>(R(0), R(0));  // coefficients >= p stay zero
    if (valid) {
        C* dst = reinterpret_cast<C*>(le + slot * (2 * g.P));
        C v = dst[n];
        v.x += acc.x;
        v.y += acc.y;
        dst[n] = v;
    }
}

template <typename R, int G>
__device__ __forceinline__ void stage_l2l_table(const R* __restrict__ src,
                                                typename Cplx<R>::T* dst) {
    using C = typename Cplx<R>::T;
    const C* s = reinterpret_cast<const C*>(src);
    for (int i = threadIdx.x; i < 4 * G * G; i += blockDim.x) dst[i] = s[i];
    __syncthreads();
}

template <typename R, int G>
__global__ void __launch_bounds__(256)
l2l_level_kernel(Geometry g, int level, const R* __restrict__ l2l, R* __restrict__ le) {
    using C = typename Cplx<R>::T;
    __shared__ C tab[4 * G * G];
    stage_l2l_table<R, G>(l2l, tab);
    int64_t gid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
    int64_t nb = (int64_t)1 << (2 * level);
    bool valid = gid < nb;
    l2l_box<R, G>(g, level, g.level_base[level] + (valid ? gid : 0), valid, tab, le);
}

// Two consecutive levels in one launch: a CTA takes a 4 x 4 block of boxes at
// `level`, then the 8 x 8 block of their children at level + 1, with a CTA
// barrier between (the children read their parents' expansions, which this
// CTA has just completed).  The per-box arithmetic is l2l_box's, so the
// expansions are those of two single-level launches bit for bit; the launch
// saved shortens the far-field branch, whose last kernels can end after the
// near field.
template <typename R, int G>
__global__ void __launch_bounds__(256)
l2l_two_level_kernel(Geometry g, int level, const R* __restrict__ l2l, R* __restrict__ le) {
    using C = typename Cplx<R>::T;
    __shared__ C tab[4 * G * G];
    stage_l2l_table<R, G>(l2l, tab);
    constexpr int kPer = 256 / G;  // boxes per sweep of the CTA
    const uint32_t tiles = 1u << (level - 2);  // 4 x 4 blocks per axis at `level`
    const uint32_t tx = blockIdx.x % tiles, ty = blockIdx.x / tiles;
    const int b = threadIdx.x / G;
#pragma unroll 1
    for (int b0 = 0; b0 < 16; b0 += kPer) {
        const uint32_t ix = 4 * tx + ((b0 + b) & 3), iy = 4 * ty + ((b0 + b) >> 2);
        l2l_box<R, G>(g, level, box_slot(g.level_base, level, ix, iy), true, tab, le);
    }
    __syncthreads();  // this CTA's boxes at `level` are complete
#pragma unroll 1
    for (int b0 = 0; b0 < 64; b0 += kPer) {
        const uint32_t ix = 8 * tx + ((b0 + b) & 7), iy = 8 * ty + ((b0 + b) >> 3);
        l2l_box<R, G>(g, level + 1, box_slot(g.level_base, level + 1, ix, iy), true, tab, le);
    }
}

// Batched L2L at one level: G lanes per box, boxes of the listed instances.
template <int G>
__global__ void __launch_bounds__(256)
l2l_batch_kernel(const BatchInst* __restrict__ inst, const int32_t* __restrict__ list, int count,
                 int level, const float* __restrict__ l2l, float* __restrict__ le) {
    __shared__ float2 tab[4 * G * G];
    stage_l2l_table<float, G>(l2l, tab);
    const int64_t per = (int64_t)1 << (2 * level);
    const int64_t gid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
    const bool valid = gid < per * count;
    const int64_t g0 = valid ? gid : 0;
    const BatchInst& b = inst[list[g0 / per]];
    l2l_box<float, G>(b.g, level, b.g.level_base[level] + g0 % per, valid, tab, le + b.exp_off);
}

}  // namespace

cudaError_t launch_batch_l2l(const BatchInst* inst, const BatchLists& bl, int P, int level,
                             const float* l2l, float* le, cudaStream_t s) {
    const int count = bl.l2l_count[level];
    if (count == 0) return cudaSuccess;
    const int64_t threads = ((int64_t)1 << (2 * level)) * count * P;
    const int blocks = (int)((threads + 255) / 256);
    if (P <= 16)
        l2l_batch_kernel<16><<<blocks, 256, 0, s>>>(inst, bl.l2l_inst[level], count, level, l2l,
                                                   le);
    else
        l2l_batch_kernel<32><<<blocks, 256, 0, s>>>(inst, bl.l2l_inst[level], count, level, l2l,
                                                   le);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_l2l(const Geometry& g, const Tables<R>& t, R* le, cudaStream_t s) {
    int level = kTopLevel + 1;
    for (; level + 1 <= g.L - 1; level += 2) {  // levels in pairs
        const unsigned blocks = 1u << (2 * (level - 2));
        if (g.P <= 16)
            l2l_two_level_kernel<R, 16><<<blocks, 256, 0, s>>>(g, level, t.l2l, le);
        else
            l2l_two_level_kernel<R, 32><<<blocks, 256, 0, s>>>(g, level, t.l2l, le);
    }
    if (level <= g.L - 1) {  // an odd level left over
        int64_t threads = ((int64_t)1 << (2 * level)) * g.P;
        int blocks = (int)((threads + 255) / 256);
        if (g.P <= 16)
            l2l_level_kernel<R, 16><<<blocks, 256, 0, s>>>(g, level, t.l2l, le);
        else
            l2l_level_kernel<R, 32><<<blocks, 256, 0, s>>>(g, level, t.l2l, le);
    }
    return cudaGetLastError();
}

template cudaError_t launch_l2l<float>(const Geometry&, const Tables<float>&, float*,
                                       cudaStream_t);
template cudaError_t launch_l2l<double>(const Geometry&, const Tables<double>&, double*,
                                        cudaStream_t);

}  // namespace fmm2d
