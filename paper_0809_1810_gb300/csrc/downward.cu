// Downward sweep, L2L part (Sec. 3.3.3): for levels 3..L each box adds its
// parent's complete local expansion, re-expanded about its own centre:
//   L~_n(child) += sum_{k>=n} L2L[q]_{nk} L~_k(parent),  q = child quadrant.
// Level l runs after level l-1 is complete, one launch per level.
#include "fmm2d_internal.cuh"

namespace fmm2d {
namespace {

template <typename R, int G>
__global__ void __launch_bounds__(128)
l2l_kernel(Geometry g, int level, const R* __restrict__ l2l, R* __restrict__ le) {
    using C = typename Cplx<R>::T;  // G = P lanes per box (16 or 32)
    int lane = threadIdx.x & 31;
    int n = lane % G;
    int64_t gid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
    int64_t nb = (int64_t)1 << (2 * level);
    bool valid = gid < nb;
    int64_t slot = g.level_base[level] + (valid ? gid : 0);
    uint32_t ix, iy;
    slot_box(g.level_base, level, slot, &ix, &iy);
    int q = (int)(((iy & 1u) << 1) | (ix & 1u));
    const C* parent = reinterpret_cast<const C*>(
        le + box_slot(g.level_base, level - 1, ix >> 1, iy >> 1) * (2 * g.P));
    C l_own = parent[n];
    const C* t = reinterpret_cast<const C*>(l2l) + (int64_t)q * G * G;
    C acc = cmake<C>(R(0), R(0));
#pragma unroll
    for (int k = 0; k < G; ++k) {  // entries with k >= p are zero
        C lk = cshfl(l_own, k, G);
        acc = cfma(t[k * G + n], lk, acc);
    }
    if (valid) {
        C* dst = reinterpret_cast<C*>(le + slot * (2 * g.P));
        C v = dst[n];
        v.x += acc.x;
        v.y += acc.y;
        dst[n] = v;
    }
}

}  // namespace

template <typename R>
cudaError_t launch_l2l(const Geometry& g, int level, const Tables<R>& t, R* le, cudaStream_t s) {
    int64_t nb = (int64_t)1 << (2 * level);
    int blocks = (int)((nb * g.P + 127) / 128);
    if (g.P <= 16)
        l2l_kernel<R, 16><<<blocks, 128, 0, s>>>(g, level, t.l2l, le);
    else
        l2l_kernel<R, 32><<<blocks, 128, 0, s>>>(g, level, t.l2l, le);
    return cudaGetLastError();
}

template cudaError_t launch_l2l<float>(const Geometry&, int, const Tables<float>&, float*,
                                       cudaStream_t);
template cudaError_t launch_l2l<double>(const Geometry&, int, const Tables<double>&, double*,
                                        cudaStream_t);

}  // namespace fmm2d
