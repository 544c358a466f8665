// Upward sweep (Sec. 3.1, Fig. 3): P2M at the leaves, then M2M for levels
// L-1 .. 2.  Expansions are box-size scaled (see tables.cu):
//   P2M  a~_m = sum_{i in leaf} c_i zeta_i^m,  c_i = -j Gamma_i / 2pi,
//        zeta_i = (z_i - z_leaf) / s_leaf                          (Eq. 20-21)
//   M2M  parent b~_n = sum_quadrants sum_{k<=n} M2M[q]_{nk} a~_k(child)  (Sec. 3.3.2)
// The leaf centre is formed once per leaf in FP64 and held as an FP32 hi/lo
// pair, so that zeta = ((x - c_hi) - c_lo) / s is accurate to FP32 relative
// to the leaf size and the expansion is centred where the translation
// tables assume.
#include "fmm2d_internal.cuh"

namespace fmm2d {
namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

// One warp per leaf; lanes stride over the leaf's particles, accumulate all
// p coefficients, then reduce across the warp.
template <typename R, int PMAX>
__global__ void __launch_bounds__(128)
p2m_kernel(const typename ParticleOf<R>::type* __restrict__ sp,
           const uint32_t* __restrict__ leaf_start, Geometry g, double scale, R* __restrict__ me) {
    using C = typename Cplx<R>::T;
    int lane = threadIdx.x & 31;
    int64_t leaf = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nleaf = (int64_t)1 << (2 * g.L);
    if (leaf >= nleaf) return;
    uint32_t ix = morton_compact((uint32_t)leaf), iy = morton_compact((uint32_t)leaf >> 1);
    uint32_t b = leaf_start[leaf], e = leaf_start[leaf + 1];
    double cx = g.x0 + ((double)ix + 0.5) / scale, cy = g.y0 + ((double)iy + 0.5) / scale;
    R cxh = (R)cx, cyh = (R)cy;
    R cxl = (R)(cx - (double)cxh), cyl = (R)(cy - (double)cyh);
    R inv_s = (R)scale;
    C acc[PMAX];
#pragma unroll
    for (int m = 0; m < PMAX; ++m) acc[m] = cmake<C>(R(0), R(0));
    for (uint32_t r = b + lane; r < e; r += 32) {
        auto q = sp[r];
        C zeta = cmake<C>(((q.x - cxh) - cxl) * inv_s, ((q.y - cyh) - cyl) * inv_s);
        C pw = cmake<C>(R(0), -q.z * (R)(1.0 / kTwoPi));  // c_i = -j Gamma / 2pi
#pragma unroll
        for (int m = 0; m < PMAX; ++m) {
            if (m < g.p) {
                acc[m].x += pw.x;
                acc[m].y += pw.y;
                pw = cmul(pw, zeta);
            }
        }
    }
#pragma unroll
    for (int m = 0; m < PMAX; ++m) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc[m].x += __shfl_xor_sync(0xffffffffu, acc[m].x, o);
            acc[m].y += __shfl_xor_sync(0xffffffffu, acc[m].y, o);
        }
    }
    R* dst = me + box_slot(g.level_base, g.L, ix, iy) * (2 * g.P);
#pragma unroll
    for (int m = 0; m < PMAX; ++m) {
        if ((m & 31) == lane && m < g.P) {
            dst[2 * m] = acc[m].x;
            dst[2 * m + 1] = acc[m].y;
        }
    }
}

// One group of P lanes per parent box at `level`; lane n computes b~_n.
template <typename R, int G>
__global__ void __launch_bounds__(128)
m2m_kernel(Geometry g, int level, const R* __restrict__ m2m, R* __restrict__ me) {
    using C = typename Cplx<R>::T;  // G = P lanes per box (16 or 32)
    int lane = threadIdx.x & 31;
    int n = lane % G;
    int64_t gid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
    int64_t nb = (int64_t)1 << (2 * level);
    bool valid = gid < nb;
    int64_t slot = g.level_base[level] + (valid ? gid : 0);
    uint32_t ix, iy;
    slot_box(g.level_base, level, slot, &ix, &iy);
    const C* tab = reinterpret_cast<const C*>(m2m);
    C acc = cmake<C>(R(0), R(0));
    for (int q = 0; q < 4; ++q) {
        uint32_t cx = 2 * ix + (q & 1), cy = 2 * iy + (q >> 1);
        const C* child = reinterpret_cast<const C*>(me + box_slot(g.level_base, level + 1, cx, cy) *
                                                             (2 * g.P));
        C a_own = child[n];
        const C* tq = tab + (int64_t)q * G * G;
#pragma unroll
        for (int k = 0; k < G; ++k) {  // entries with k >= p are zero
            C ak = cshfl(a_own, k, G);
            acc = cfma(tq[k * G + n], ak, acc);
        }
    }
    if (valid) reinterpret_cast<C*>(me + slot * (2 * g.P))[n] = acc;
}

}  // namespace

template <typename R>
cudaError_t launch_p2m(const Geometry& g, const void* particles, const uint32_t* leaf_start, R* me,
                       cudaStream_t s) {
    using P = typename ParticleOf<R>::type;
    int64_t nleaf = (int64_t)1 << (2 * g.L);
    int blocks = (int)((nleaf * 32 + 127) / 128);
    double scale = ldexp(1.0, g.L) / g.W;
    if (g.P <= 16)
        p2m_kernel<R, 16><<<blocks, 128, 0, s>>>(reinterpret_cast<const P*>(particles), leaf_start,
                                                 g, scale, me);
    else
        p2m_kernel<R, 32><<<blocks, 128, 0, s>>>(reinterpret_cast<const P*>(particles), leaf_start,
                                                 g, scale, me);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_m2m(const Geometry& g, int level, const Tables<R>& t, R* me, cudaStream_t s) {
    int64_t nb = (int64_t)1 << (2 * level);
    int64_t threads = nb * g.P;
    int blocks = (int)((threads + 127) / 128);
    if (g.P <= 16)
        m2m_kernel<R, 16><<<blocks, 128, 0, s>>>(g, level, t.m2m, me);
    else
        m2m_kernel<R, 32><<<blocks, 128, 0, s>>>(g, level, t.m2m, me);
    return cudaGetLastError();
}

template cudaError_t launch_p2m<float>(const Geometry&, const void*, const uint32_t*, float*,
                                       cudaStream_t);
template cudaError_t launch_p2m<double>(const Geometry&, const void*, const uint32_t*, double*,
                                        cudaStream_t);
template cudaError_t launch_m2m<float>(const Geometry&, int, const Tables<float>&, float*,
                                       cudaStream_t);
template cudaError_t launch_m2m<double>(const Geometry&, int, const Tables<double>&, double*,
                                        cudaStream_t);

}  // namespace fmm2d
