// Accuracy yardsticks in double precision (Sec. 5: the FMM result is
// compared with a direct sum and errors are normalised by the maximum speed).
//
// direct_sampled: velocity at s sampled particles by direct summation over
// all n particles, self term excluded (Eq. 9):
//   kernel 0: K_sigma of Eq. 6 for every pair (Eq. 7)
//   kernel 1: K_sigma for pairs in each other's 3x3 leaf neighbourhood (and,
//             with a cutoff a, for every pair closer than a) and the singular
//             kernel of Eq. 27 for the rest -- the sum the FMM converges to as
//             p grows (Eq. 10, Sec. 4.1)
// error_stats: max |du|, max |u_ref|, sum |du|^2, sum |u_ref|^2 and the
// per-leaf max |du| over the sampled particles.
#include "fmm2d_internal.cuh"

namespace fmm2d {
namespace {

constexpr int kTargetsPerBlock = 16;
constexpr int kSlices = 16;  // threads per target
constexpr int kTile = 256;   // source particles per shared-memory tile

__device__ inline int leaf_index(double x, double lo, double scale, double top) {
    double f = floor((x - lo) * scale);
    if (!(f >= 0.0)) f = 0.0;
    if (f > top) f = top;
    return (int)f;
}

template <typename R>
__global__ void __launch_bounds__(kTargetsPerBlock* kSlices)
direct_kernel(int kernel, int64_t n, const R* __restrict__ xy, const R* __restrict__ gamma,
              int64_t s_count, const int64_t* __restrict__ targets, double inv2s2, double a2,
              double x0, double y0, double scale, double top, double* __restrict__ uv_ref,
              int* status) {
    __shared__ double sx[kTile], sy[kTile], sg[kTile];
    __shared__ int sl[kTile], sm[kTile];
    __shared__ double red[2][kSlices][kTargetsPerBlock];
    const int t = threadIdx.x % kTargetsPerBlock;
    const int slice = threadIdx.x / kTargetsPerBlock;
    const int64_t ti = blockIdx.x * (int64_t)kTargetsPerBlock + t;
    int64_t i = -1;
    if (ti < s_count) {
        i = targets[ti];
        if (i < 0 || i >= n) {
            if (slice == 0) atomicOr(status, kFlagInvalid);
            i = -1;
        }
    }
    double xi = 0.0, yi = 0.0;
    int li = 0, mi = 0;
    if (i >= 0) {
        xi = (double)xy[2 * i];
        yi = (double)xy[2 * i + 1];
        li = leaf_index(xi, x0, scale, top);
        mi = leaf_index(yi, y0, scale, top);
    }
    double au = 0.0, av = 0.0;
    for (int64_t base = 0; base < n; base += kTile) {
        __syncthreads();
        for (int q = threadIdx.x; q < kTile; q += blockDim.x) {
            int64_t j = base + q;
            if (j < n) {
                double x = (double)xy[2 * j], y = (double)xy[2 * j + 1];
                sx[q] = x;
                sy[q] = y;
                sg[q] = (double)gamma[j];
                sl[q] = leaf_index(x, x0, scale, top);
                sm[q] = leaf_index(y, y0, scale, top);
            } else {
                sx[q] = 0.0;
                sy[q] = 0.0;
                sg[q] = 0.0;
                sl[q] = -100;
                sm[q] = -100;
            }
        }
        __syncthreads();
        if (i < 0) continue;
        for (int q = slice; q < kTile; q += kSlices) {
            int64_t j = base + q;
            if (j == i || j >= n) continue;
            double dx = xi - sx[q], dy = yi - sy[q];
            double r2 = dx * dx + dy * dy;
            if (r2 == 0.0) continue;  // K_sigma(0) = 0 by its limit
            bool near = kernel == 0 || (abs(sl[q] - li) <= 1 && abs(sm[q] - mi) <= 1) || r2 < a2;
            double f = near ? -expm1(-r2 * inv2s2) / r2 : 1.0 / r2;
            double w = sg[q] * f;
            au = fma(-dy, w, au);
            av = fma(dx, w, av);
        }
    }
    red[0][slice][t] = au;
    red[1][slice][t] = av;
    __syncthreads();
    if (slice == 0 && ti < s_count) {
        double u = 0.0, v = 0.0;
        for (int k = 0; k < kSlices; ++k) {
            u += red[0][k][t];
            v += red[1][k][t];
        }
        const double inv2pi = 1.0 / 6.283185307179586476925286766559;
        uv_ref[2 * ti] = u * inv2pi;
        uv_ref[2 * ti + 1] = v * inv2pi;
    }
}

// Non-negative doubles order like their bit patterns.
__device__ inline void atomic_max_nonneg(double* addr, double v) {
    atomicMax(reinterpret_cast<unsigned long long*>(addr),
              (unsigned long long)__double_as_longlong(v));
}

template <typename R>
__global__ void error_kernel(int64_t n, const R* __restrict__ xy, const R* __restrict__ uv,
                             int64_t s_count, const int64_t* __restrict__ targets,
                             const double* __restrict__ uv_ref, double* stats, double* leaf_err,
                             double x0, double y0, double scale, double top, int* status) {
    double emax = 0.0, rmax = 0.0, esum = 0.0, rsum = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < s_count;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = targets[t];
        if (i < 0 || i >= n) {
            atomicOr(status, kFlagInvalid);
            continue;
        }
        double ru = uv_ref[2 * t], rv = uv_ref[2 * t + 1];
        double du = (double)uv[2 * i] - ru, dv = (double)uv[2 * i + 1] - rv;
        double e2 = du * du + dv * dv, r2 = ru * ru + rv * rv;
        double e = sqrt(e2), r = sqrt(r2);
        if (!(e == e)) e = __longlong_as_double(0x7ff0000000000000LL);  // NaN counts as infinite
        emax = fmax(emax, e);
        rmax = fmax(rmax, r);
        esum += e2;
        rsum += r2;
        if (leaf_err) {
            uint32_t lx = (uint32_t)leaf_index((double)xy[2 * i], x0, scale, top);
            uint32_t ly = (uint32_t)leaf_index((double)xy[2 * i + 1], y0, scale, top);
            atomic_max_nonneg(&leaf_err[morton_key(lx, ly)], e);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
        rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
        esum += __shfl_xor_sync(0xffffffffu, esum, o);
        rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(&stats[0], emax);
        atomic_max_nonneg(&stats[1], rmax);
        atomicAdd(&stats[2], esum);
        atomicAdd(&stats[3], rsum);
    }
}

__device__ inline int find_instance(const int64_t* __restrict__ offsets, int count, int64_t i) {
    int lo = 0, hi = count;  // offsets[lo] <= i < offsets[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (offsets[mid] <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Batched direct sums: one warp per sampled target, over its own instance.
__global__ void __launch_bounds__(256)
batch_direct_kernel(const BatchInst* __restrict__ inst, const int64_t* __restrict__ offsets,
                    int count, int kernel, const float* __restrict__ xy,
                    const float* __restrict__ gamma, int64_t s_count,
                    const int64_t* __restrict__ targets, double* __restrict__ uv_ref,
                    int* status) {
    const int lane = threadIdx.x & 31;
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (t >= s_count) return;
    const int64_t i = targets[t];
    if (i < 0 || i >= offsets[count]) {
        if (lane == 0) atomicOr(status, kFlagInvalid);
        return;
    }
    const BatchInst& b = inst[find_instance(offsets, count, i)];
    const double top = ldexp(1.0, b.g.L) - 1.0;
    const double xi = (double)xy[2 * i], yi = (double)xy[2 * i + 1];
    const int li = leaf_index(xi, b.g.x0, b.g.scale, top), mi = leaf_index(yi, b.g.y0, b.g.scale, top);
    const double inv2s2 = 1.0 / (2.0 * b.sigma * b.sigma);
    double au = 0.0, av = 0.0;
    for (int64_t j = b.offset + lane; j < b.offset + b.n; j += 32) {
        if (j == i) continue;
        const double x = (double)xy[2 * j], y = (double)xy[2 * j + 1];
        const double dx = xi - x, dy = yi - y, r2 = dx * dx + dy * dy;
        if (r2 == 0.0) continue;  // K_sigma(0) = 0 by its limit
        bool near = kernel == 0;
        if (!near) {
            const int lj = leaf_index(x, b.g.x0, b.g.scale, top);
            const int mj = leaf_index(y, b.g.y0, b.g.scale, top);
            near = (abs(lj - li) <= 1 && abs(mj - mi) <= 1) ||
                   (b.g.L >= 2 && r2 < b.g.cutoff * b.g.cutoff);  // Sec. 4.1 cutoff
        }
        const double f = near ? -expm1(-r2 * inv2s2) / r2 : 1.0 / r2;
        const double w = (double)gamma[j] * f;
        au = fma(-dy, w, au);
        av = fma(dx, w, av);
    }
    for (int o = 16; o > 0; o >>= 1) {
        au += __shfl_xor_sync(0xffffffffu, au, o);
        av += __shfl_xor_sync(0xffffffffu, av, o);
    }
    if (lane == 0) {
        const double inv2pi = 1.0 / 6.283185307179586476925286766559;
        uv_ref[2 * t] = au * inv2pi;
        uv_ref[2 * t + 1] = av * inv2pi;
    }
}

// Batched error statistics: 4 doubles per instance (max |du|, max |u_ref|,
// sum |du|^2, sum |u_ref|^2) and the max |du| per global leaf.
__global__ void batch_error_kernel(const BatchInst* __restrict__ inst,
                                   const int64_t* __restrict__ offsets, int count,
                                   const float* __restrict__ xy, const float* __restrict__ uv,
                                   int64_t s_count, const int64_t* __restrict__ targets,
                                   const double* __restrict__ uv_ref, double* stats,
                                   double* leaf_err, int* status) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < s_count;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = targets[t];
        if (i < 0 || i >= offsets[count]) {
            atomicOr(status, kFlagInvalid);
            continue;
        }
        const int k = find_instance(offsets, count, i);
        const BatchInst& b = inst[k];
        double ru = uv_ref[2 * t], rv = uv_ref[2 * t + 1];
        double du = (double)uv[2 * i] - ru, dv = (double)uv[2 * i + 1] - rv;
        double e = sqrt(du * du + dv * dv), r = sqrt(ru * ru + rv * rv);
        if (!(e == e)) e = __longlong_as_double(0x7ff0000000000000LL);
        atomic_max_nonneg(&stats[4 * k], e);
        atomic_max_nonneg(&stats[4 * k + 1], r);
        atomicAdd(&stats[4 * k + 2], e * e);
        atomicAdd(&stats[4 * k + 3], r * r);
        if (leaf_err) {
            const double top = ldexp(1.0, b.g.L) - 1.0;
            uint32_t lx = (uint32_t)leaf_index((double)xy[2 * i], b.g.x0, b.g.scale, top);
            uint32_t ly = (uint32_t)leaf_index((double)xy[2 * i + 1], b.g.y0, b.g.scale, top);
            atomic_max_nonneg(&leaf_err[b.leaf_base + morton_key(lx, ly)], e);
        }
    }
}

}  // namespace

cudaError_t launch_batch_direct(const BatchInst* inst, const int64_t* dev_offsets, int count,
                                int kernel, const float* xy, const float* gamma, int64_t s_count,
                                const int64_t* targets, double* uv_ref, int* status,
                                cudaStream_t s) {
    if (s_count == 0) return cudaSuccess;
    int64_t blocks = (s_count * 32 + 255) / 256;
    batch_direct_kernel<<<(unsigned)blocks, 256, 0, s>>>(inst, dev_offsets, count, kernel, xy,
                                                         gamma, s_count, targets, uv_ref, status);
    return cudaGetLastError();
}

cudaError_t launch_batch_error(const BatchInst* inst, const int64_t* dev_offsets, int count,
                               const float* xy, const float* uv, int64_t s_count,
                               const int64_t* targets, const double* uv_ref, double* stats,
                               double* leaf_err, uint32_t nleaf_total, int* status,
                               cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(stats, 0, 4 * sizeof(double) * count, s);
    if (e == cudaSuccess && leaf_err)
        e = cudaMemsetAsync(leaf_err, 0, sizeof(double) * nleaf_total, s);
    if (e != cudaSuccess || s_count == 0) return e;
    int64_t blocks = (s_count + 255) / 256;
    if (blocks > 2048) blocks = 2048;
    batch_error_kernel<<<(unsigned)blocks, 256, 0, s>>>(inst, dev_offsets, count, xy, uv, s_count,
                                                        targets, uv_ref, stats, leaf_err, status);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_direct_sampled(const Geometry& g, double sigma, int kernel, int64_t n,
                                  const R* xy, const R* gamma, int64_t s_count,
                                  const int64_t* targets, double* uv_ref, int* status,
                                  cudaStream_t s) {
    if (s_count == 0) return cudaSuccess;
    int64_t blocks = (s_count + kTargetsPerBlock - 1) / kTargetsPerBlock;
    direct_kernel<R><<<(unsigned)blocks, kTargetsPerBlock * kSlices, 0, s>>>(
        kernel, n, xy, gamma, s_count, targets, 1.0 / (2.0 * sigma * sigma),
        g.L >= 2 ? g.cutoff * g.cutoff : 0.0, g.x0, g.y0, ldexp(1.0, g.L) / g.W,
        ldexp(1.0, g.L) - 1.0, uv_ref, status);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_error_stats(const Geometry& g, int64_t n, const R* xy, const R* uv,
                               int64_t s_count, const int64_t* targets, const double* uv_ref,
                               double* stats, double* leaf_err, int* status, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(stats, 0, 4 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    if (leaf_err) {
        e = cudaMemsetAsync(leaf_err, 0, sizeof(double) << (2 * g.L), s);
        if (e != cudaSuccess) return e;
    }
    if (s_count == 0) return cudaSuccess;
    int64_t blocks = (s_count + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    error_kernel<R><<<(unsigned)blocks, 256, 0, s>>>(n, xy, uv, s_count, targets, uv_ref, stats,
                                                     leaf_err, g.x0, g.y0, ldexp(1.0, g.L) / g.W,
                                                     ldexp(1.0, g.L) - 1.0, status);
    return cudaGetLastError();
}

#define INST(R)                                                                                  \
    template cudaError_t launch_direct_sampled<R>(const Geometry&, double, int, int64_t, const R*, \
                                                  const R*, int64_t, const int64_t*, double*,   \
                                                  int*, cudaStream_t);                          \
    template cudaError_t launch_error_stats<R>(const Geometry&, int64_t, const R*, const R*,      \
                                               int64_t, const int64_t*, const double*, double*,  \
                                               double*, int*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace fmm2d
