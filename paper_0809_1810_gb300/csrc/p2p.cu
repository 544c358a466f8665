// Evaluation step (Sec. 3.1, Eq. 10): for every particle i of a leaf b,
//   far part   w = (1/s) sum_n L~_n(b) zeta^n,  zeta = (z_i - z_b)/s   (L2P)
//              u_far = (Re w, -Im w)                                (Eq. 16 with -j)
//   near part  sum_{j in local list of b, j != i} Gamma_j K_sigma(x_i - x_j)   (Eq. 6)
// The local list is the leaf and its up to 8 neighbours (Sec. 3.3.1).  The
// self term drops out without a test: K_sigma's direction vector (-dy, dx)
// is exactly zero at zero separation, and its radial factor stays finite.
//
// One CTA per target leaf.  Source records of the 3x3 neighbourhood are
// staged in shared memory in chunks; each target is handled by `ns` adjacent
// lanes that split the sources and combine with warp shuffles.  Velocities
// are written straight to the input order through the record's index.
//
// FP32 radial factor.  With q = r^2 / 2 sigma^2 and q2 = q / ln 2,
//   (1 - e^-q) / r^2 = g(q2) / (2 sigma^2 ln 2),  g(q2) = (1 - 2^-q2) / q2.
// For q >= 1, g = (1 - ex2(-q2)) * rcp(q2) on the MUFU unit; for q < 1 the
// subtraction would cancel, so g is summed from its Taylor series
//   g(q2) = sum_k (-1)^k ln2^(k+1) q2^k / (k+1)!   (truncated after q2^9,
// relative truncation error below 5e-8 on [0, 1/ln 2)).
// Each lane accumulates kInner pairs in a fresh register, then adds that
// partial sum to its running sum with Neumaier's compensated addition, so
// the FP32 rounding of a near sum stays at the level of one kInner-term sum
// however many sources the local list holds.
#include "fmm2d_internal.cuh"

namespace fmm2d {
namespace {

constexpr int kThreads = 128;
constexpr int kChunk = 1024;   // source records per shared-memory chunk
constexpr int kInner = 16;     // pairs per first-level partial sum
constexpr int kMaxSlices = 8;  // lanes per target when a leaf holds few particles
constexpr int kPad = kInner * kMaxSlices;
constexpr int kSeries = 10;    // Taylor coefficients of g

struct NearF32 {
    float c2;              // log2(e) / (2 sigma^2)
    float qthr;            // 1 / ln 2  (q = 1)
    float k0;              // 1 / (4 pi sigma^2 ln 2)
    float coef[kSeries];   // Taylor coefficients of g in q2
};
struct NearF64 {
    double inv2s2;  // 1 / (2 sigma^2)
    double k0;      // 1 / (2 pi)
};

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Radial weight Gamma_j * (1 - e^-q)/r^2 up to the constant k0.
__device__ __forceinline__ float radial(const NearF32& nm, float r2) {
    float q2 = r2 * nm.c2;
    float naive = (1.0f - ex2_approx(-q2)) * rcp_approx(q2);
    float ser = nm.coef[kSeries - 1];
#pragma unroll
    for (int k = kSeries - 2; k >= 0; --k) ser = fmaf(ser, q2, nm.coef[k]);
    return q2 < nm.qthr ? ser : naive;
}
__device__ __forceinline__ double radial(const NearF64& nm, double r2) {
    return r2 > 0.0 ? -expm1(-r2 * nm.inv2s2) / r2 : 0.0;
}
__device__ __forceinline__ float k0_of(const NearF32& nm) { return nm.k0; }

// Neumaier's compensated summation step: s + c tracks the exact sum.
template <typename R>
__device__ __forceinline__ void neumaier_add(R& s, R& c, R x) {
    R t = s + x;
    c += (fabs(s) >= fabs(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
}
__device__ __forceinline__ double k0_of(const NearF64& nm) { return nm.k0; }

template <typename R, typename NM>
__global__ void __launch_bounds__(kThreads)
p2p_l2p_kernel(const typename ParticleOf<R>::type* __restrict__ sp,
               const uint32_t* __restrict__ leaf_start, Geometry g, double scale, NM nm,
               const R* __restrict__ le, R* __restrict__ uv) {
    using PT = ParticleOf<R>;
    using P = typename PT::type;
    using C = typename Cplx<R>::T;
    __shared__ P src[kChunk + kPad];
    __shared__ C le_s[kMaxP];
    __shared__ uint32_t rbeg[9], rpre[10];

    const int tid = threadIdx.x;
    const uint32_t leaf = blockIdx.x;
    const uint32_t ix = morton_compact(leaf), iy = morton_compact(leaf >> 1);
    const uint32_t t0 = leaf_start[leaf], t1 = leaf_start[leaf + 1];
    if (t0 == t1) return;
    const int nl = 1 << g.L;
    if (tid < 9) {
        int sx = (int)ix + tid % 3 - 1, sy = (int)iy + tid / 3 - 1;
        uint32_t b = 0, len = 0;
        if (sx >= 0 && sy >= 0 && sx < nl && sy < nl) {
            uint32_t k = morton_key((uint32_t)sx, (uint32_t)sy);
            b = leaf_start[k];
            len = leaf_start[k + 1] - b;
        }
        rbeg[tid] = b;
        rpre[tid + 1] = len;
    }
    const bool far = g.L >= 2;
    if (far && tid < g.P)
        le_s[tid] = reinterpret_cast<const C*>(le + box_slot(g.level_base, g.L, ix, iy) *
                                                        (2 * g.P))[tid];
    __syncthreads();
    if (tid == 0) {
        rpre[0] = 0;
        for (int r = 0; r < 9; ++r) rpre[r + 1] += rpre[r];
    }
    __syncthreads();
    const uint32_t total = rpre[9];
    const uint32_t nt = t1 - t0;

    for (uint32_t tb = 0; tb < nt; tb += kThreads) {
        const uint32_t ntc = min(nt - tb, (uint32_t)kThreads);
        const int ns = ntc <= 16 ? 8 : ntc <= 32 ? 4 : ntc <= 64 ? 2 : 1;
        const uint32_t tl = tid / ns;
        const int sl = tid % ns;
        const bool active = tl < ntc;
        P self = active ? sp[t0 + tb + tl] : P{};
        const R xi = self.x, yi = self.y;
        R au = R(0), av = R(0), cu = R(0), cv = R(0);
        for (uint32_t cb = 0; cb < total; cb += kChunk) {
            const uint32_t cnt = min(total - cb, (uint32_t)kChunk);
            const uint32_t step = kInner * ns;
            const uint32_t cpad = (cnt + step - 1) / step * step;
            __syncthreads();
            for (uint32_t v = tid; v < cpad; v += kThreads) {
                P rec{};
                if (v < cnt) {
                    uint32_t gv = cb + v;
                    int r = 0;
                    while (gv >= rpre[r + 1]) ++r;
                    rec = sp[rbeg[r] + (gv - rpre[r])];
                }
                src[v] = rec;
            }
            __syncthreads();
            for (uint32_t j0 = sl; j0 < cpad; j0 += step) {
                R iu = R(0), iv = R(0);
#pragma unroll
                for (int t = 0; t < kInner; ++t) {
                    const P s = src[j0 + t * ns];
                    const R dx = xi - s.x, dy = yi - s.y;
                    const R r2 = dx * dx + dy * dy;
                    const R w = s.z * radial(nm, r2);
                    iu = fma(-dy, w, iu);
                    iv = fma(dx, w, iv);
                }
                neumaier_add(au, cu, iu);
                neumaier_add(av, cv, iv);
            }
        }
        au += cu;
        av += cv;
        for (int o = 1; o < ns; o <<= 1) {
            au += __shfl_xor_sync(0xffffffffu, au, o);
            av += __shfl_xor_sync(0xffffffffu, av, o);
        }
        if (active && sl == 0) {
            R u = k0_of(nm) * au, v = k0_of(nm) * av;
            if (far) {
                double xi_d = ((double)self.x - g.x0) * scale - ((double)ix + 0.5);
                double eta_d = ((double)self.y - g.y0) * scale - ((double)iy + 0.5);
                C zeta = cmake<C>((R)xi_d, (R)eta_d);
                C w = le_s[g.p - 1];
                for (int m = g.p - 2; m >= 0; --m) {
                    C t = cmul(w, zeta);
                    w = cmake<C>(t.x + le_s[m].x, t.y + le_s[m].y);
                }
                u += (R)scale * w.x;
                v -= (R)scale * w.y;
            }
            uint32_t idx = PT::index(self);
            uv[2 * (int64_t)idx] = u;
            uv[2 * (int64_t)idx + 1] = v;
        }
    }
}

}  // namespace

template <>
cudaError_t launch_p2p_l2p<float>(const Geometry& g, double sigma, const void* particles,
                                  const uint32_t* leaf_start, const float* le, float* uv,
                                  cudaStream_t s) {
    const double ln2 = 0.69314718055994530942;
    const double pi = 3.14159265358979323846;
    NearF32 nm;
    nm.c2 = (float)(1.0 / (2.0 * sigma * sigma * ln2));
    nm.qthr = (float)(1.0 / ln2);
    nm.k0 = (float)(1.0 / (4.0 * pi * sigma * sigma * ln2));
    double lk = ln2, fact = 1.0;
    for (int k = 0; k < kSeries; ++k) {  // (-1)^k ln2^(k+1) / (k+1)!
        fact *= (double)(k + 1);
        nm.coef[k] = (float)(((k & 1) ? -1.0 : 1.0) * lk / fact);
        lk *= ln2;
    }
    unsigned nleaf = 1u << (2 * g.L);
    p2p_l2p_kernel<float, NearF32><<<nleaf, kThreads, 0, s>>>(
        reinterpret_cast<const float4*>(particles), leaf_start, g, ldexp(1.0, g.L) / g.W, nm, le,
        uv);
    return cudaGetLastError();
}

template <>
cudaError_t launch_p2p_l2p<double>(const Geometry& g, double sigma, const void* particles,
                                   const uint32_t* leaf_start, const double* le, double* uv,
                                   cudaStream_t s) {
    NearF64 nm;
    nm.inv2s2 = 1.0 / (2.0 * sigma * sigma);
    nm.k0 = 1.0 / (2.0 * 3.14159265358979323846);
    unsigned nleaf = 1u << (2 * g.L);
    p2p_l2p_kernel<double, NearF64><<<nleaf, kThreads, 0, s>>>(
        reinterpret_cast<const ParticleD*>(particles), leaf_start, g, ldexp(1.0, g.L) / g.W, nm,
        le, uv);
    return cudaGetLastError();
}

}  // namespace fmm2d
