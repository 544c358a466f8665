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

template <typename R, int G>
__global__ void __launch_bounds__(128)
m2l_kernel(Geometry g, const R* __restrict__ m2l, const R* __restrict__ me, R* __restrict__ le) {
    using C = typename Cplx<R>::T;  // G = P lanes per target box (16 or 32)
    int lane = threadIdx.x & 31;
    int n = lane % G;
    unsigned seg = segment_mask(G);
    int64_t gid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
    bool valid = gid < g.nboxes;
    int64_t slot = g.level_base[2] + (valid ? gid : 0);
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
    if (valid) reinterpret_cast<C*>(le + slot * (2 * g.P))[n] = acc;
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

template cudaError_t launch_m2l<float>(const Geometry&, const Tables<float>&, const float*, float*,
                                       cudaStream_t);
template cudaError_t launch_m2l<double>(const Geometry&, const Tables<double>&, const double*,
                                        double*, cudaStream_t);

}  // namespace fmm2d
