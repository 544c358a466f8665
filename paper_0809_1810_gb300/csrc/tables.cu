// Translation-operator tables, built on the device in double precision.
//
// Expansions are scaled by box size so that coefficients stay O(1) at any
// level (s = box width at the level of the expansion):
//   ME  a~_k = sum_i c_i ((z_i - z_c) / s)^k,   c_i = -j Gamma_i / 2pi   (Eq. 20)
//   LE  L~_n = s^(n+1) L_n,   w(y) = (1/s) sum_n L~_n ((y - z_c) / s)^n
// With that scaling every translation matrix depends only on the relative
// position of the two boxes, not on the level:
//   M2M  (Sec. 3.3.2, exact binomial shift)  child quadrant (cx, cy),
//        t = (z_child - z_parent) / s_parent = ((2cx-1) + j(2cy-1)) / 4,
//        b~_n = sum_{k<=n} C(n,k) t^(n-k) 2^-k a~_k
//   L2L  (Sec. 3.3.3)  t = (z_child - z_parent) / s_child = ((2cx-1) + j(2cy-1)) / 2,
//        L~'_n = sum_{k>=n} C(k,n) t^(k-n) 2^-(k+1) L~_k
//   M2L  (Eq. 22)  source box offset (dx, dy) from the target, tau = -(dx + j dy),
//        L~_n = sum_k (-1)^n C(n+k,k) tau^-(n+k+1) a~_k
// Entries with n or k >= p are zero, so padded coefficients stay zero.
#include "fmm2d_internal.cuh"

namespace fmm2d {
namespace {

struct C64 {
    double re, im;
};
__device__ inline C64 cmul(C64 a, C64 b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ inline C64 cinv(C64 a) {
    double d = a.re * a.re + a.im * a.im;
    return {a.re / d, -a.im / d};
}
__device__ inline C64 cpow(C64 a, int m) {
    C64 r{1.0, 0.0};
    for (int i = 0; i < m; ++i) r = cmul(r, a);
    return r;
}

// Pascal's triangle C[n][k], n, k <= nmax, one block; each row from the last.
__global__ void binomial_kernel(double* C, int nmax) {
    int ld = nmax + 1;
    for (int k = threadIdx.x; k < ld * ld; k += blockDim.x) C[k] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) C[0] = 1.0;
    __syncthreads();
    for (int n = 1; n <= nmax; ++n) {
        for (int k = threadIdx.x; k <= n; k += blockDim.x) {
            double left = k > 0 ? C[(n - 1) * ld + k - 1] : 0.0;
            double up = k < n ? C[(n - 1) * ld + k] : 0.0;
            C[n * ld + k] = left + up;
        }
        __syncthreads();
    }
}

// One thread per (matrix, k, n) entry of the three tables.
__global__ void tables_kernel(int p, int P, const double* C, int ld, double* m2m, double* l2l,
                              double* m2l) {
    int64_t per = (int64_t)P * P;
    int64_t total = (4 + 4 + kOffsetSlots) * per;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t mat = e / per;
        int k = (int)((e % per) / P);
        int n = (int)(e % P);
        C64 v{0.0, 0.0};
        double* dst;
        if (mat < 4) {
            int cx = (int)(mat & 1), cy = (int)(mat >> 1);
            if (n < p && k < p && k <= n) {
                C64 t{(2 * cx - 1) * 0.25, (2 * cy - 1) * 0.25};
                C64 tp = cpow(t, n - k);
                double f = C[n * ld + k] * ldexp(1.0, -k);
                v = {f * tp.re, f * tp.im};
            }
            dst = m2m + mat * per * 2;
        } else if (mat < 8) {
            int q = (int)(mat - 4);
            int cx = q & 1, cy = q >> 1;
            if (n < p && k < p && k >= n) {
                C64 t{(2 * cx - 1) * 0.5, (2 * cy - 1) * 0.5};
                C64 tp = cpow(t, k - n);
                double f = C[k * ld + n] * ldexp(1.0, -(k + 1));
                v = {f * tp.re, f * tp.im};
            }
            dst = l2l + q * per * 2;
        } else {
            int slot = (int)(mat - 8);
            int dx = slot % 7 - 3, dy = slot / 7 - 3;
            bool far = (dx < -1 || dx > 1 || dy < -1 || dy > 1);
            if (far && n < p && k < p) {
                C64 tau{(double)-dx, (double)-dy};
                C64 tp = cpow(cinv(tau), n + k + 1);
                double f = ((n & 1) ? -1.0 : 1.0) * C[(n + k) * ld + k];
                v = {f * tp.re, f * tp.im};
            }
            dst = m2l + slot * per * 2;
        }
        int64_t off = ((int64_t)k * P + n) * 2;
        dst[off] = v.re;
        dst[off + 1] = v.im;
    }
}

__global__ void to_f32_kernel(const double* src, float* dst, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

// One thread per axis index: the same FP64 arithmetic as the direct
// computation (centre_hilo_1d), so the table holds the same bits.
__global__ void centre_table_kernel(Geometry g, float4* tab) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (1u << g.L)) return;
    float4 v;
    centre_hilo_1d(g.x0, g.W, g.L, i, &v.x, &v.y);
    centre_hilo_1d(g.y0, g.W, g.L, i, &v.z, &v.w);
    tab[i] = v;
}

}  // namespace

cudaError_t launch_centre_table(const Geometry& g, float4* tab, cudaStream_t s) {
    const int n = 1 << g.L;
    centre_table_kernel<<<(n + 255) / 256, 256, 0, s>>>(g, tab);
    return cudaGetLastError();
}

cudaError_t launch_build_tables(int p, int P, double* m2m, double* l2l, double* m2l,
                                double* binom_scratch, cudaStream_t s) {
    int nmax = 2 * P;
    binomial_kernel<<<1, 256, 0, s>>>(binom_scratch, nmax);
    int64_t total = (int64_t)(4 + 4 + kOffsetSlots) * P * P;
    int blocks = (int)((total + 255) / 256);
    tables_kernel<<<blocks, 256, 0, s>>>(p, P, binom_scratch, nmax + 1, m2m, l2l, m2l);
    return cudaGetLastError();
}

cudaError_t launch_tables_to_f32(const double* src, float* dst, int64_t count, cudaStream_t s) {
    int blocks = (int)((count + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    to_f32_kernel<<<blocks, 256, 0, s>>>(src, dst, count);
    return cudaGetLastError();
}

}  // namespace fmm2d
