// M2L on CUDA cores (Eq. 22), for the FP64 path and the plain FP32 path.
//
// For every box b of levels 2..L, its local expansion is the sum over the
// interaction list -- children of the parent's neighbours that are not in
// b's local list (Sec. 3.3.1) -- of the translated multipole expansions:
//   L~_n(b) = sum_{s in IL(b)} sum_k M2L[off(s,b)]_{nk} a~_k(s)
// With box-size scaling the matrix depends only on the offset (dx, dy) of s
// from b, one of 40 in [-3, 3]^2 with max(|dx|, |dy|) >= 2.  All levels are
// independent given the multipole expansions, so one launch covers them.
// The result is assigned (not accumulated): L2L later adds the parent part.
#include "fmm2d_internal.cuh"

namespace fmm2d {
namespace {

// One target box, G lanes (lane n computes L~_n).
template <typename R, int G>
__device__ __forceinline__ void m2l_box(const Geometry& g, int64_t slot, bool valid,
                                        const R* __restrict__ m2l, const R* __restrict__ me,
                                        R* __restrict__ le) {
    using C = typename Cplx<R>::T;
    int lane = threadIdx.x & 31;
    int n = lane % G;
    unsigned seg = segment_mask(G);
    int l = slot_level(g.level_base, g.L, slot);
    uint32_t ix, iy;
    slot_box(g.level_base, l, slot, &ix, &iy);
    int nb = 1 << l;
    const C* tab = reinterpret_cast<const C*>(m2l);
    C acc = cmake<C>(R(0), R(0));
    for (int dy = -3; dy <= 3; ++dy) {
        int sy = (int)iy + dy;
        if (sy < 0 || sy >= nb || abs((sy >> 1) - (int)(iy >> 1)) > 1) continue;
        for (int dx = -3; dx <= 3; ++dx) {
            int sx = (int)ix + dx;
            if (sx < 0 || sx >= nb || abs((sx >> 1) - (int)(ix >> 1)) > 1) continue;
            if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;  // local list
            const C* src = reinterpret_cast<const C*>(
                me + box_slot(g.level_base, l, (uint32_t)sx, (uint32_t)sy) * (2 * g.P));
            C a_own = src[n];
            const C* t = tab + (int64_t)offset_slot(dx, dy) * G * G;
#pragma unroll
            for (int k = 0; k < G; ++k) {  // entries with k >= p are zero
                C ak = cshfl(a_own, k, G, seg);
                acc = cfma(t[k * G + n], ak, acc);
            }
        }
    }
    if (n >= g.p) acc = cmake<C>(R(0), R(0));  // coefficients >= p stay zero
    if (valid) reinterpret_cast<C*>(le + slot * (2 * g.P))[n] = acc;
}

template <typename R, int G>
__global__ void __launch_bounds__(128)
m2l_kernel(Geometry g, const R* __restrict__ m2l, const R* __restrict__ me, R* __restrict__ le) {
    int64_t gid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
    bool valid = gid < g.nboxes;
    m2l_box<R, G>(g, g.level_base[2] + (valid ? gid : 0), valid, m2l, me, le);
}

// Batched: every box of every listed instance (levels 2..L), G lanes each.
template <int G>
__global__ void __launch_bounds__(256)
m2l_batch_kernel(const BatchInst* __restrict__ inst, const int32_t* __restrict__ list,
                 const int64_t* __restrict__ prefix, int count, int64_t total,
                 const float* __restrict__ m2l, const float* __restrict__ me,
                 float* __restrict__ le) {
    const int64_t gid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
    const bool valid = gid < total;
    const int64_t g0 = valid ? gid : 0;
    int lo = 0, hi = count;  // prefix[lo] <= g0 < prefix[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (prefix[mid] <= g0) lo = mid;
        else hi = mid;
    }
    const BatchInst& b = inst[list[lo]];
    m2l_box<float, G>(b.g, b.g.level_base[2] + (g0 - prefix[lo]), valid, m2l, me + b.exp_off,
                      le + b.exp_off);
}

}  // namespace

template <typename R>
cudaError_t launch_m2l(const Geometry& g, const Tables<R>& t, const R* me, R* le, cudaStream_t s) {
    if (g.L < 2) return cudaSuccess;
    int64_t threads = g.nboxes * g.P;
    int blocks = (int)((threads + 127) / 128);
    if (g.P <= 16)
        m2l_kernel<R, 16><<<blocks, 128, 0, s>>>(g, t.m2l, me, le);
    else
        m2l_kernel<R, 32><<<blocks, 128, 0, s>>>(g, t.m2l, me, le);
    return cudaGetLastError();
}

cudaError_t launch_batch_m2l(const BatchInst* inst, const BatchLists& bl, int P, int threads,
                             const float* m2l, const float* me, float* le, cudaStream_t s) {
    if (bl.m2l_count == 0) return cudaSuccess;
    const int64_t lanes = bl.m2l_total * P;
    const int blocks = (int)((lanes + threads - 1) / threads);
    if (P <= 16)
        m2l_batch_kernel<16><<<blocks, threads, 0, s>>>(inst, bl.m2l_inst, bl.m2l_prefix,
                                                       bl.m2l_count, bl.m2l_total, m2l, me, le);
    else
        m2l_batch_kernel<32><<<blocks, threads, 0, s>>>(inst, bl.m2l_inst, bl.m2l_prefix,
                                                       bl.m2l_count, bl.m2l_total, m2l, me, le);
    return cudaGetLastError();
}

template cudaError_t launch_m2l<float>(const Geometry&, const Tables<float>&, const float*, float*,
                                       cudaStream_t);
template cudaError_t launch_m2l<double>(const Geometry&, const Tables<double>&, const double*,
                                        double*, cudaStream_t);

}  // namespace fmm2d
