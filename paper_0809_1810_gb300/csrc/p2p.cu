// Evaluation step (Sec. 3.1, Eq. 10): for every particle i of a leaf b,
//   far part   w = (1/s) sum_n L~_n(b) zeta^n,  zeta = (z_i - z_b)/s   (L2P)
//              u_far = (Re w, -Im w)                                (Eq. 16 with -j)
//   near part  sum_{j in local list of b, j != i} Gamma_j K_sigma(x_i - x_j)   (Eq. 6)
// The local list is the leaf and its up to 8 neighbours (Sec. 3.3.1).  The
// self term drops out without a test: K_sigma's direction vector (-dy, dx)
// is exactly zero at zero separation, and its radial factor stays finite.
//
// FP64: one CTA per target leaf.  Source records of the 3x3 neighbourhood
// are staged in shared memory in chunks; each target is handled by `ns`
// adjacent lanes that split the sources and combine with warp shuffles.
// Velocities are written straight to the input order through the record's
// index.  The radial factor is (1 - e^-q)/r^2 with q = r^2 / 2 sigma^2,
// formed with expm1 so that it keeps full precision for small q.  The FP32
// kernel (further down) has its own work split and radial factor.
#include <algorithm>
#include <type_traits>

#include "fmm2d_internal.cuh"

namespace fmm2d {
namespace {

constexpr int kThreads = 128;
constexpr int kChunk = 1024;   // source records per shared-memory chunk
constexpr int kInner = 16;     // pairs per first-level partial sum
constexpr int kMaxSlices = 8;  // lanes per target when a leaf holds few particles
constexpr int kPad = kInner * kMaxSlices;

struct NearF64 {
    double inv2s2;  // 1 / (2 sigma^2)
    double k0;      // 1 / (2 pi)
    double a2;      // cutoff a^2 (0: none)
    uint32_t ring_mask;  // ring leaves that can hold a pair closer than a
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
__device__ __forceinline__ double radial(const NearF64& nm, double r2) {
    return r2 > 0.0 ? -expm1(-r2 * nm.inv2s2) / r2 : 0.0;
}
// Cutoff correction for a ring pair (Sec. 4.1): the far field applied the
// singular 1/r^2 to it; closer than a, K_sigma - K' = -e^-q / r^2 restores
// the regularised kernel.
__device__ __forceinline__ double radial_cut(const NearF64& nm, double r2) {
    return r2 < nm.a2 && r2 > 0.0 ? -exp(-r2 * nm.inv2s2) / r2 : 0.0;
}

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
               const R* __restrict__ le, const R* __restrict__ l2l, R* __restrict__ uv) {
    using PT = ParticleOf<R>;
    using P = typename PT::type;
    using C = typename Cplx<R>::T;
    __shared__ P src[kChunk + kPad];
    __shared__ C le_s[kMaxP];
    __shared__ uint32_t rbeg[25], rpre[26];  // 3x3 block, then the ring (cutoff)

    const int tid = threadIdx.x;
    const uint32_t leaf = blockIdx.x;
    const uint32_t ix = morton_compact(leaf), iy = morton_compact(leaf >> 1);
    const uint32_t t0 = leaf_start[leaf], t1 = leaf_start[leaf + 1];
    if (t0 == t1) return;
    const int nl = 1 << g.L;
    if (tid < 25) {
        int dx = tid % 3 - 1, dy = tid / 3 - 1;
        if (tid >= 9) ring_offset(tid - 9, &dx, &dy);
        const int sx = (int)ix + dx, sy = (int)iy + dy;
        uint32_t b = 0, len = 0;
        const bool want = tid < 9 || ((nm.ring_mask >> (tid - 9)) & 1u);
        if (want && sx >= 0 && sy >= 0 && sx < nl && sy < nl) {
            uint32_t k = morton_key((uint32_t)sx, (uint32_t)sy);
            b = leaf_start[k];
            len = leaf_start[k + 1] - b;
        }
        rbeg[tid] = b;
        rpre[tid + 1] = len;
    }
    const bool far = g.L >= 2;
    if (far && tid < g.P) {  // the leaf's LE: its M2L part plus L2L of its parent's
        C v = reinterpret_cast<const C*>(le + box_slot(g.level_base, g.L, ix, iy) * (2 * g.P))[tid];
        if (g.L >= 3) {
            const C* par = reinterpret_cast<const C*>(
                le + box_slot(g.level_base, g.L - 1, ix >> 1, iy >> 1) * (2 * g.P));
            const C* t = reinterpret_cast<const C*>(l2l) +
                         (int64_t)(((iy & 1u) << 1) | (ix & 1u)) * g.P * g.P;
            for (int k = 0; k < g.P; ++k) v = cfma(t[k * g.P + tid], par[k], v);
        }
        le_s[tid] = v;
    }
    __syncthreads();
    if (tid == 0) {
        rpre[0] = 0;
        for (int r = 0; r < 25; ++r) rpre[r + 1] += rpre[r];
    }
    __syncthreads();
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
        // phase 0: the 3x3 local list with K_sigma; phase 1: the ring with
        // the cutoff correction (empty without a cutoff)
        for (int ph = 0; ph < 2; ++ph) {
            const uint32_t lo = ph ? rpre[9] : 0u, hi = ph ? rpre[25] : rpre[9];
            for (uint32_t cb = lo; cb < hi; cb += kChunk) {
                const uint32_t cnt = min(hi - cb, (uint32_t)kChunk);
                const uint32_t step = kInner * ns;
                const uint32_t cpad = (cnt + step - 1) / step * step;
                __syncthreads();
                for (uint32_t v = tid; v < cpad; v += kThreads) {
                    P rec{};
                    if (v < cnt) {
                        uint32_t gv = cb + v;
                        int r = ph ? 9 : 0;
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
                        const R w = s.z * (ph ? radial_cut(nm, r2) : radial(nm, r2));
                        iu = fma(-dy, w, iu);
                        iv = fma(dx, w, iv);
                    }
                    neumaier_add(au, cu, iu);
                    neumaier_add(av, cv, iv);
                }
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

// ---------------------------------------------------------------------------
// FP32 near field, the dominant kernel of the FP32 form.
//
// Work split: targets in sorted (leaf) order.  A leaf's targets form rounds
// of 32 and chunks of 64 or 128 from its first target; persistent warps pull
// windows of the sorted order from a counter and run every chunk that starts
// inside (see WorkSplit), so a crowded leaf spreads over many warps instead
// of holding one warp while the rest of the GPU idles, and the last items are
// short.  For each chunk the warp gathers the leaf's local list -- the 9
// source ranges of the 3x3 neighbourhood, coalesced loads -- into a
// per-warp shared-memory buffer, sorted by a ballot compaction into a near
// band (front) and a far band (back): a source farther than sqrt(qthr)
// scaled units from the leaf's square is at q2 >= qthr from every target of
// the leaf, so the far band never needs the polynomial.
// Targets go in passes of 32 T (T = 4, 2, 1 per lane); all lanes read the
// same source (a shared-memory broadcast).  In a leaf's last round of at
// most 16 targets, ns adjacent lanes share a target and split its sources
// (combined by shuffles).  Band loops are straight-line code (no per-pair
// branches).  Lists longer than the buffer are processed in parts.
//
// Pair arithmetic in scaled leaf-relative FP32 coordinates X = (x - centre)
// sc, so that q2 = |X_i - X_j|^2 = r^2 / (2 sigma^2 ln 2).
// Radial factor g(q2) = (1 - 2^-q2) / q2: MUFU ex2 and rcp for
// q2 >= kPolyEdge; below it the subtraction 1 - 2^-q2 would cancel, and a
// cubic interpolating g at the Chebyshev nodes of [0, kPolyEdge] takes over
// (interpolation error 8e-9, below FP32 rounding), fitted on the host when
// the kernel is launched.  At q2 = kPolyEdge the MUFU form is within 6e-7
// of g (two ulp of ex2 over 1 - 2^-q2 = 0.099), and the few pairs that close
// to a target carry a small share of its velocity.
// Sums: blocks of sources into fresh registers, then Neumaier-compensated
// addition into the running sums.  A whole chunk (128 targets) gives each
// lane four targets and gathers each part of the local list once; full
// passes of 64 targets give each lane two; one shared-memory read of a
// source serves that many pairs.
// ---------------------------------------------------------------------------
constexpr int kLeafWarps = 4;
constexpr uint32_t kTicket = 128;  // largest sorted-target window (a power of two)
#ifndef FMM2D_P2P_LIST_CAP
#define FMM2D_P2P_LIST_CAP 560  // 37 KB of shared memory per CTA: 6 CTAs per SM
#endif
constexpr int kListCap = FMM2D_P2P_LIST_CAP;  // source records per warp buffer
static_assert(kListCap % 2 == 0, "the source lists hold whole pairs");
constexpr int kF32Deg = 3;
constexpr double kPolyEdge = 0.15;  // q2 below which the polynomial is used

struct NearF32v3 {
    float sc;                 // coordinate scale: q2 = |dX|^2 with X = (x - centre) sc
    float qthr;               // polynomial below, MUFU at and above (q2 = kPolyEdge)
    float kvel;               // 1 / (4 pi sigma^2 ln 2 sc): sum -> velocity
    float kzeta;              // 1 / (sc s): scaled coordinate -> zeta
    float inv_s;              // 1 / s (leaf width)
    float half_leaf;          // s sc / 2, half the leaf in scaled units
    float band2;              // squared scaled distance to the leaf square below
                              // which a source may be at q2 < qthr of a target
    float qa;                 // cutoff a^2 in scaled units, a^2 sc^2 (0: none)
    float band_a2;            // qa with a margin: ring sources nearer the leaf square
    float wstrip;             // ring strips: the band along a side of a leaf (scaled
                              // width) holding every source the leaf two leaves away
                              // on that side keeps (0: no cutoff)
    uint32_t ring_mask;       // ring leaves (bit r, ring_offset order) nearer than a
    uint32_t lane_nt;         // leaves of at most this many targets go to the
                              // per-target-lane pass (0: none)
    float coef[kF32Deg + 1];  // g(q2) ~ sum_k coef[k] q2^k on [0, qthr)
};

// Packed FP32 pairs (f32x2): one instruction applies the same operation to
// the two halves of a register pair, so the pair arithmetic of two sources
// against one target takes one issue slot per step instead of two.
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
    float2 r;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " sub.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) {
    float2 r;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " mul.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
// a * b + c, rounded once per half
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
    float2 r;
    asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " mov.b64 rc, {%6, %7};\n fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}
__device__ __forceinline__ float2 f2_dup(float v) { return make_float2(v, v); }

// Source lists hold sources in pairs: pair k occupies buf[2k] = (x_a, x_b,
// y_a, y_b) and buf[2k + 1] = (Gamma_a, Gamma_b, -Gamma_a, -Gamma_b), in
// scaled leaf-relative coordinates; source j is half j & 1 of pair j >> 1.
// A band of odd length is completed by a dummy source of zero circulation
// far from every target (q2 ~ 1e36: its weight is exactly zero).
constexpr float kFarAway = 1e18f;
__device__ __forceinline__ void put_source(float4* buf, uint32_t j, float x, float y, float g) {
    float* p0 = reinterpret_cast<float*>(buf + 2 * (j >> 1));
    const uint32_t h = j & 1u;
    p0[h] = x;
    p0[2 + h] = y;
    p0[4 + h] = g;
    p0[6 + h] = -g;
}
__device__ __forceinline__ void put_dummy(float4* buf, uint32_t j) {
    put_source(buf, j, kFarAway, kFarAway, 0.f);
}

// Pair modes of the band loops: far band, near band (polynomial below the
// edge), ring pairs under the cutoff.
constexpr int kFar = 0, kNearBand = 1, kRing = 2;

// Two sources (a pair of the list) against one target at (tx, tx), (ty, ty):
// the velocity sums of the two halves, iu = sum Gamma g(q2) (-dy) and
// iv = sum Gamma g(q2) dx with dx = x_t - x_s, dy = y_t - y_s.
// Radial weight Gamma g(q2) = fma(-Gamma, e, Gamma) rcp(q2), e = 2^-q2
// (Gamma (1 - e)/q2 with the circulation folded into the subtraction: one
// instruction fewer than forming 1 - e first, and one rounding fewer).  Near
// band: below qthr the cubic in q2 times Gamma instead.  Ring: the cutoff
// correction of Sec. 4.1 -- the far field applied the singular kernel, and
// closer than a, -Gamma 2^-q2 / q2 restores K_sigma; zero beyond a.
template <int kMode>
__device__ __forceinline__ void pair_sources(const NearF32v3& nm, const float4 P0, const float4 P1,
                                             float2 tx, float2 ty, float2& iu, float2& iv) {
    const float2 dx = f2_sub(tx, make_float2(P0.x, P0.y));
    const float2 ndy = f2_sub(make_float2(P0.z, P0.w), ty);  // -dy
    const float2 q = f2_fma(ndy, ndy, f2_mul(dx, dx));
    const float2 e = make_float2(ex2_approx(-q.x), ex2_approx(-q.y));
    const float2 r = make_float2(rcp_approx(q.x), rcp_approx(q.y));
    float2 w;
    if (kMode == kRing) {
        w = f2_mul(f2_mul(make_float2(P1.z, P1.w), e), r);
        w.x = q.x < nm.qa ? w.x : 0.f;
        w.y = q.y < nm.qa ? w.y : 0.f;
    } else {
        const float2 g = make_float2(P1.x, P1.y);
        w = f2_mul(f2_fma(make_float2(P1.z, P1.w), e, g), r);
        if (kMode == kNearBand) {
            float2 poly = f2_dup(nm.coef[kF32Deg]);
#pragma unroll
            for (int k = kF32Deg - 1; k >= 0; --k) poly = f2_fma(poly, q, f2_dup(nm.coef[k]));
            const float2 wn = f2_mul(g, poly);
            w.x = q.x < nm.qthr ? wn.x : w.x;
            w.y = q.y < nm.qthr ? wn.y : w.y;
        }
    }
    iu = f2_fma(ndy, w, iu);
    iv = f2_fma(dx, w, iv);
}

// Pairs [lo, hi) of the list against the lane's target when ns > 1 lanes
// share a target (sl = this lane's slot; a leaf's last round of at most 16
// targets): blocks of kInner pairs into fresh sums, then compensated.
template <int kMode>
__device__ __forceinline__ void band_loop_split(const float4* list, uint32_t lo, uint32_t hi,
                                                int ns, int sl, const NearF32v3& nm, float x,
                                                float y, float& su, float& sv, float& cu,
                                                float& cv) {
    const float2 tx = f2_dup(x), ty = f2_dup(y);
    float2 iu = make_float2(0.f, 0.f), iv = make_float2(0.f, 0.f);
    int cnt = 0;
#pragma unroll 1
    for (uint32_t kk = lo; kk < hi; kk += ns) {
        const uint32_t k = kk + sl;
        // past the end: a pair of dummies (zero circulation, far away)
        float4 P0 = make_float4(kFarAway, kFarAway, kFarAway, kFarAway);
        float4 P1 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < hi) {
            P0 = list[2 * k];
            P1 = list[2 * k + 1];
        }
        pair_sources<kMode>(nm, P0, P1, tx, ty, iu, iv);
        if (++cnt == kInner / 2) {
            neumaier_add(su, cu, iu.x + iu.y);
            neumaier_add(sv, cv, iv.x + iv.y);
            iu = iv = make_float2(0.f, 0.f);
            cnt = 0;
        }
    }
    neumaier_add(su, cu, iu.x + iu.y);
    neumaier_add(sv, cv, iv.x + iv.y);
}

// Pairs [lo, hi) of the list against T targets per lane (passes of 32 T
// targets): blocks of kInnerT / 2 pairs into fresh sums, then compensated.
// One shared-memory read of a pair serves 2 T source-target pairs.  Each
// target sees the same sequence of operations whatever T is, so a target's
// velocity does not depend on how its rounds were grouped into passes.
constexpr int kInnerT = 64;

template <int T>
struct SumT {
    float su[T], sv[T], cu[T], cv[T];
};

template <int kMode, int T>
__device__ __forceinline__ void band_loopT(const float4* list, uint32_t lo, uint32_t hi,
                                           const NearF32v3& nm, const float (&x)[T],
                                           const float (&y)[T], SumT<T>& S) {
    // pairs per iteration (two at one and two targets per lane, one at four)
    constexpr int kUnroll = T >= 4 ? 1 : 2;
    float2 tx[T], ty[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        tx[t] = f2_dup(x[t]);
        ty[t] = f2_dup(y[t]);
    }
    uint32_t k = lo;
    while (k < hi) {
        const uint32_t e = min(k + (uint32_t)(kInnerT / 2), hi);
        float2 iu[T], iv[T];
#pragma unroll
        for (int t = 0; t < T; ++t) iu[t] = iv[t] = make_float2(0.f, 0.f);
#pragma unroll 1
        for (; k + kUnroll <= e; k += kUnroll) {
#pragma unroll
            for (int q = 0; q < kUnroll; ++q) {
                const float4 P0 = list[2 * (k + q)], P1 = list[2 * (k + q) + 1];
#pragma unroll
                for (int t = 0; t < T; ++t)
                    pair_sources<kMode>(nm, P0, P1, tx[t], ty[t], iu[t], iv[t]);
            }
        }
        for (; k < e; ++k) {
            const float4 P0 = list[2 * k], P1 = list[2 * k + 1];
#pragma unroll
            for (int t = 0; t < T; ++t) pair_sources<kMode>(nm, P0, P1, tx[t], ty[t], iu[t], iv[t]);
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            neumaier_add(S.su[t], S.cu[t], iu[t].x + iu[t].y);
            neumaier_add(S.sv[t], S.cv[t], iv[t].x + iv[t].y);
        }
    }
}

// Band boundaries in pairs: the near band [0, near_pairs(nn)) and the far band
// [far_first(nf), kListCap / 2) of a buffer holding nn near and nf far sources.
__device__ __forceinline__ uint32_t near_pairs(uint32_t nn) { return (nn + 1) >> 1; }
__device__ __forceinline__ uint32_t far_first(uint32_t nf) {
    return ((uint32_t)kListCap - nf - (nf & 1u)) >> 1;
}
// Sources gathered into a buffer at a time: room for a dummy in each band.
constexpr uint32_t kListChunk = kListCap - 2;
// gathers of at most this many records walk one index space over the ranges
// (built into the batched kernel (kFlat), whose sparse instances have lists of
// a few records per range; in the single-evaluation kernel the extra code
// slowed the near field at 64 particles per leaf by 7%)
constexpr uint32_t kSmallList = 64;

struct LeafCtx {
    uint32_t t0, nt;           // the leaf's targets in sorted order
    const float* le_leaf;      // its local expansion (null when L < 2)
    float cxh, cxl, cyh, cyl;  // leaf centre as FP32 hi/lo
    const uint32_t* rbeg;      // the 9 source ranges (shared memory)
    const uint32_t* rpre;      // prefix sums of their lengths (10 entries)
    uint32_t ctotal;           // ring sources under a cutoff (0: none)
    const uint32_t* cbeg;      // the 16 ring ranges (shared memory)
    const uint32_t* cpre;      // prefix sums of their lengths (17 entries)
};

// The two vectors a leaf's local expansion is formed from: its M2L part and
// its parent's expansion (lane k < P holds coefficient k; zero elsewhere).
struct LeafLeParts {
    float2 own, par;
};

__device__ __forceinline__ LeafLeParts leaf_le_load(const Geometry& g, const float* __restrict__ le,
                                                    uint32_t lx, uint32_t ly) {
    const int lane = threadIdx.x & 31;
    LeafLeParts q{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    if (lane < g.P) {
        q.own = reinterpret_cast<const float2*>(
            le + box_slot(g.level_base, g.L, lx, ly) * (2 * g.P))[lane];
        if (g.L >= 3)
            q.par = reinterpret_cast<const float2*>(
                le + box_slot(g.level_base, g.L - 1, lx >> 1, ly >> 1) * (2 * g.P))[lane];
    }
    return q;
}

// The leaf's local expansion, written to `out` (P coefficients, shared
// memory): its M2L part plus the L2L of its parent's (Sec. 3.3.3).  One warp.
__device__ __forceinline__ void leaf_le_finish(const Geometry& g, const float* __restrict__ l2l,
                                               uint32_t lx, uint32_t ly, const LeafLeParts& q,
                                               float2* out) {
    const int lane = threadIdx.x & 31;
    float2 v = q.own;
    if (g.L >= 3) {
        const float2* t = reinterpret_cast<const float2*>(l2l) +
                          (int64_t)(((ly & 1u) << 1) | (lx & 1u)) * g.P * g.P;
        for (int k = 0; k < g.P; ++k) {
            float2 pk = cshfl(q.par, k, 32);
            if (lane < g.P) v = cfma(t[k * g.P + lane], pk, v);
        }
    }
    if (lane >= g.p) v = make_float2(0.f, 0.f);
    __syncwarp();  // earlier readers of `out` are done
    if (lane < g.P) out[lane] = v;
    __syncwarp();
}

// leaf_le_finish for P = 16, the loop unrolled so that the translation
// table's loads are issued together (the same operations in the same order).
__device__ __forceinline__ void leaf_le_finish16(const Geometry& g, const float* __restrict__ l2l,
                                                 uint32_t lx, uint32_t ly, const LeafLeParts& q,
                                                 float2* out) {
    const int lane = threadIdx.x & 31;
    float2 v = q.own;
    if (g.L >= 3) {
        const float2* t = reinterpret_cast<const float2*>(l2l) +
                          (int64_t)(((ly & 1u) << 1) | (lx & 1u)) * 16 * 16;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            float2 pk = cshfl(q.par, k, 32);
            if (lane < 16) v = cfma(t[k * 16 + lane], pk, v);
        }
    }
    if (lane >= g.p) v = make_float2(0.f, 0.f);
    __syncwarp();  // earlier readers of `out` are done
    if (lane < 16) out[lane] = v;
    __syncwarp();
}

// leaf_le_finish for P = 32, the loop unrolled by eight so that the table's
// loads are issued eight at a time (the same operations in the same order).
__device__ __forceinline__ void leaf_le_finish32(const Geometry& g, const float* __restrict__ l2l,
                                                 uint32_t lx, uint32_t ly, const LeafLeParts& q,
                                                 float2* out) {
    const int lane = threadIdx.x & 31;
    float2 v = q.own;
    if (g.L >= 3) {
        const float2* t = reinterpret_cast<const float2*>(l2l) +
                          (int64_t)(((ly & 1u) << 1) | (lx & 1u)) * 32 * 32;
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            float2 pk = cshfl(q.par, k, 32);
            v = cfma(t[k * 32 + lane], pk, v);
        }
    }
    if (lane >= g.p) v = make_float2(0.f, 0.f);
    __syncwarp();  // earlier readers of `out` are done
    out[lane] = v;
    __syncwarp();
}

__device__ __forceinline__ void leaf_le_build(const Geometry& g, const float* __restrict__ le,
                                              const float* __restrict__ l2l, uint32_t lx,
                                              uint32_t ly, float2* out) {
    leaf_le_finish(g, l2l, lx, ly, leaf_le_load(g, le, lx, ly), out);
}

// The same by the unrolled form of its expansion width (P is 16 or 32): the
// batched near-field kernel builds one per leaf, and with a few particles per
// leaf the chain of P table products is most of a leaf's time.  (The
// single-evaluation kernels leave the expansion to l2p_f32_kernel.)
__device__ __forceinline__ void leaf_le_build_unrolled(const Geometry& g,
                                                       const float* __restrict__ le,
                                                       const float* __restrict__ l2l,
                                                       uint32_t lx, uint32_t ly, float2* out) {
    const LeafLeParts q = leaf_le_load(g, le, lx, ly);
    if (g.P == 16) leaf_le_finish16(g, l2l, lx, ly, q, out);
    else if (g.P == 32) leaf_le_finish32(g, l2l, lx, ly, q, out);
    else leaf_le_finish(g, l2l, lx, ly, q, out);
}

// L2P (Eq. 12) added to a target's velocity: w = (1/s) sum_n L~_n zeta^n at
// zeta = (z - z_leaf) / s, from the target's scaled leaf-relative (x, y).
__device__ __forceinline__ void l2p_add(int p, float kzeta, float inv_s, const float2* Lc,
                                        float x, float y, float& u, float& v) {
    float2 zeta = make_float2(x * kzeta, y * kzeta);
    float2 w = Lc[p - 1];
    for (int m = p - 2; m >= 0; --m) {
        float2 t = cmul(w, zeta);
        float2 lm = Lc[m];
        w = make_float2(t.x + lm.x, t.y + lm.y);
    }
    u = fmaf(inv_s, w.x, u);
    v = fmaf(-inv_s, w.y, v);
}

// Far field of a target in a lane-pass leaf (Eq. 12), from the two parts the
// leaf's local expansion is the sum of: its own M2L part (level L, `own`) at
// zeta = (z - z_leaf)/s, and its parent's complete expansion (level L - 1,
// `par`; null at L = 2) at zeta_p = (z - z_parent)/(2 s) = (zeta + t)/2,
// t = (z_leaf - z_parent)/s = (+-1/2, +-1/2) by the leaf's quadrant (cx, cy).
// The L2L shift of a polynomial is exact, so this is the value of the leaf's
// expansion up to rounding, without the P^2 products of forming it.
__device__ __forceinline__ void l2p_two_levels(int p, float kzeta, float inv_s,
                                               const float2* own, const float2* par,
                                               uint32_t cx, uint32_t cy, float x, float y,
                                               float& u, float& v) {
    const float2 zeta = make_float2(x * kzeta, y * kzeta);
    float2 w = own[p - 1];
    for (int m = p - 2; m >= 0; --m) {
        const float2 t = cmul(w, zeta);
        const float2 lm = own[m];
        w = make_float2(t.x + lm.x, t.y + lm.y);
    }
    u = fmaf(inv_s, w.x, u);
    v = fmaf(-inv_s, w.y, v);
    if (par) {
        const float2 zp = make_float2((zeta.x + (cx ? 0.5f : -0.5f)) * 0.5f,
                                      (zeta.y + (cy ? 0.5f : -0.5f)) * 0.5f);
        float2 wp = par[p - 1];
        for (int m = p - 2; m >= 0; --m) {
            const float2 t = cmul(wp, zp);
            const float2 lm = par[m];
            wp = make_float2(t.x + lm.x, t.y + lm.y);
        }
        const float hs = 0.5f * inv_s;  // 1 / s_parent
        u = fmaf(hs, wp.x, u);
        v = fmaf(-hs, wp.y, v);
    }
}

// A lane-pass leaf's two expansion parts into shared memory (own[0 .. P),
// par[0 .. P)), one warp; par only with a parent (L >= 3).
__device__ __forceinline__ void stage_two_levels(const Geometry& g, const float* __restrict__ le,
                                                 uint32_t lx, uint32_t ly, float2* own,
                                                 float2* par) {
    const int lane = threadIdx.x & 31;
    if (lane < g.P) {
        own[lane] = reinterpret_cast<const float2*>(
            le + box_slot(g.level_base, g.L, lx, ly) * (2 * g.P))[lane];
        if (g.L >= 3)
            par[lane] = reinterpret_cast<const float2*>(
                le + box_slot(g.level_base, g.L - 1, lx >> 1, ly >> 1) * (2 * g.P))[lane];
    }
}

// Gather local-list records [cb, cb + cnt) (cnt <= kListChunk) into the
// warp's buffer in scaled leaf-relative coordinates: nn near-band sources
// from the front (sources 0, 1, ...), nf far-band sources from the back
// (sources kListCap - 1, kListCap - 2, ...), each band completed to whole
// pairs by a dummy.
template <bool kFlat>
__device__ __forceinline__ void gather_bands(const float4* __restrict__ sp, const LeafCtx& c,
                                             const NearF32v3& nm, uint32_t cb, uint32_t cnt,
                                             float4* buf, uint32_t& nn, uint32_t& nf) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    nn = 0;
    nf = 0;
    __syncwarp();  // earlier readers of the buffer are done
    const uint32_t ce = cb + cnt;
    if constexpr (kFlat) {
        if (cnt <= kSmallList) {
            // few records (sparse leaves): one index space over the 9 ranges,
            // each lane finding its record's range, so that the list takes one
            // or two batches instead of one per range; the same records in the
            // same order
            for (uint32_t g0 = cb; g0 < ce; g0 += 32) {
                const uint32_t gv = g0 + lane;
                float rx = 0.f, ry = 0.f, rg = 0.f;
                bool ok = gv < ce, near = false;
                if (ok) {
                    int r = 0;
                    while (gv >= c.rpre[r + 1]) ++r;
                    float4 q = sp[c.rbeg[r] - c.rpre[r] + gv];
                    rx = ((q.x - c.cxh) - c.cxl) * nm.sc;
                    ry = ((q.y - c.cyh) - c.cyl) * nm.sc;
                    rg = q.z;
                    float ex = fmaxf(fabsf(rx) - nm.half_leaf, 0.f);
                    float ey = fmaxf(fabsf(ry) - nm.half_leaf, 0.f);
                    near = fmaf(ex, ex, ey * ey) < nm.band2;
                }
                const unsigned bn = __ballot_sync(0xffffffffu, near);
                const unsigned bf = __ballot_sync(0xffffffffu, ok && !near);
                if (near) put_source(buf, nn + __popc(bn & lt), rx, ry, rg);
                else if (ok) put_source(buf, kListCap - 1 - (nf + __popc(bf & lt)), rx, ry, rg);
                nn += __popc(bn);
                nf += __popc(bf);
            }
            cnt = 0;  // done: the range loop below has nothing left
        }
    }
    // range by range (no per-record range search); records keep their order
    for (int r = 0; (!kFlat || cnt > 0) && r < 9; ++r) {
        const uint32_t lo = max(c.rpre[r], cb), hi = min(c.rpre[r + 1], ce);
        const uint32_t base = c.rbeg[r] - c.rpre[r];
        for (uint32_t g0 = lo; g0 < hi; g0 += 32) {
            const uint32_t gv = g0 + lane;
            float rx = 0.f, ry = 0.f, rg = 0.f;
            bool ok = gv < hi, near = false;
            if (ok) {
                float4 q = sp[base + gv];
                rx = ((q.x - c.cxh) - c.cxl) * nm.sc;
                ry = ((q.y - c.cyh) - c.cyl) * nm.sc;
                rg = q.z;
                float ex = fmaxf(fabsf(rx) - nm.half_leaf, 0.f);
                float ey = fmaxf(fabsf(ry) - nm.half_leaf, 0.f);
                near = fmaf(ex, ex, ey * ey) < nm.band2;
            }
            const unsigned bn = __ballot_sync(0xffffffffu, near);
            const unsigned bf = __ballot_sync(0xffffffffu, ok && !near);
            if (near) put_source(buf, nn + __popc(bn & lt), rx, ry, rg);
            else if (ok) put_source(buf, kListCap - 1 - (nf + __popc(bf & lt)), rx, ry, rg);
            nn += __popc(bn);
            nf += __popc(bf);
        }
    }
    if (lane == 0) {
        if (nn & 1u) put_dummy(buf, nn);
        if (nf & 1u) put_dummy(buf, kListCap - 1 - nf);
    }
    __syncwarp();
}

// Gather the ring sources [cb, cb + cnt) (cnt <= kListChunk) that lie within
// the cutoff of the leaf square (only those can be closer than a to a
// target) into sources [0, nc) of buf, in scaled leaf-relative coordinates,
// completed to whole pairs by a dummy.
template <bool kFlat>
__device__ __forceinline__ void gather_ring(const float4* __restrict__ sp, const LeafCtx& c,
                                            const NearF32v3& nm, uint32_t cb, uint32_t cnt,
                                            float4* buf, uint32_t& nc) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    nc = 0;
    __syncwarp();  // earlier readers of the buffer are done
    const uint32_t ce = cb + cnt;
    if constexpr (kFlat) {
        if (cnt <= kSmallList) {  // few records: one index space over the 16 ranges
            for (uint32_t g0 = cb; g0 < ce; g0 += 32) {
                const uint32_t gv = g0 + lane;
                float rx = 0.f, ry = 0.f, rg = 0.f;
                bool keep = false;
                if (gv < ce) {
                    int r = 0;
                    while (gv >= c.cpre[r + 1]) ++r;
                    float4 q = sp[c.cbeg[r] - c.cpre[r] + gv];
                    rx = ((q.x - c.cxh) - c.cxl) * nm.sc;
                    ry = ((q.y - c.cyh) - c.cyl) * nm.sc;
                    rg = q.z;
                    float ex = fmaxf(fabsf(rx) - nm.half_leaf, 0.f);
                    float ey = fmaxf(fabsf(ry) - nm.half_leaf, 0.f);
                    keep = fmaf(ex, ex, ey * ey) < nm.band_a2;
                }
                const unsigned bk = __ballot_sync(0xffffffffu, keep);
                if (keep) put_source(buf, nc + __popc(bk & lt), rx, ry, rg);
                nc += __popc(bk);
            }
            cnt = 0;
        }
    }
    for (int r = 0; (!kFlat || cnt > 0) && r < 16; ++r) {
        const uint32_t lo = max(c.cpre[r], cb), hi = min(c.cpre[r + 1], ce);
        const uint32_t base = c.cbeg[r] - c.cpre[r];
        for (uint32_t g0 = lo; g0 < hi; g0 += 32) {
            const uint32_t gv = g0 + lane;
            float rx = 0.f, ry = 0.f, rg = 0.f;
            bool keep = false;
            if (gv < hi) {
                float4 q = sp[base + gv];
                rx = ((q.x - c.cxh) - c.cxl) * nm.sc;
                ry = ((q.y - c.cyh) - c.cyl) * nm.sc;
                rg = q.z;
                float ex = fmaxf(fabsf(rx) - nm.half_leaf, 0.f);
                float ey = fmaxf(fabsf(ry) - nm.half_leaf, 0.f);
                keep = fmaf(ex, ex, ey * ey) < nm.band_a2;
            }
            const unsigned bk = __ballot_sync(0xffffffffu, keep);
            if (keep) put_source(buf, nc + __popc(bk & lt), rx, ry, rg);
            nc += __popc(bk);
        }
    }
    if (lane == 0 && (nc & 1u)) put_dummy(buf, nc);
    __syncwarp();
}

// Targets [a, b) of one leaf (positions within the leaf) against its local
// list, by one warp.  `leaf` is the leaf's Morton key; leaf_start is indexed
// by leaf_base + key (zero for a single evaluation).  buf, ranges (9 local
// ranges and 10 prefix sums; with kCut, then 16 ring ranges and 17 prefix
// sums) and leaf_le are this warp's shared memory.  kCut compiles in the
// cutoff ring; without it the kernel carries no ring code at all.  kMaxT is
// the widest pass compiled in: 4 when chunks of 128 targets occur, else 2.
// The cutoff kernel's hot code outgrows the instruction cache (its leading
// stall is instruction fetch); with kMaxT = 2 it also runs a leaf's last
// round of at most 16 targets as a one-per-lane pass, without the split
// path: 10% faster at 64 targets per leaf.  (The plain kernel keeps both:
// there the narrower build measured slower.)
template <bool kCut, int kMaxT = 4, bool kSorted = false, bool kFlat = false>
__device__ __forceinline__ void p2p_chunk_f32(const float4* __restrict__ sp,
                                              const uint32_t* __restrict__ leaf_start,
                                              uint32_t leaf_base, uint32_t leaf, uint32_t a,
                                              uint32_t b, const Geometry& g,
                                             const NearF32v3& nm, const float* __restrict__ le,
                                             const float* __restrict__ l2l,
                                             float* __restrict__ uv, float4* buf,
                                             uint32_t* ranges, float2* leaf_le,
                                             const RingStrips& rs) {
    const int lane = threadIdx.x & 31;
    const int nl = 1 << g.L;
    const uint32_t lx = morton_compact(leaf), ly = morton_compact(leaf >> 1);
    LeafCtx c;
    c.t0 = leaf_start[leaf_base + leaf];
    c.nt = leaf_start[leaf_base + leaf + 1] - c.t0;
    if (a >= b) return;
    uint32_t* rbeg = ranges;
    uint32_t* rpre = ranges + 9;
    {  // lane r < 9 reads range r
        uint32_t b = 0, len = 0;
        if (lane < 9) {
            int sx = (int)lx + lane % 3 - 1, sy = (int)ly + lane / 3 - 1;
            if (sx >= 0 && sy >= 0 && sx < nl && sy < nl) {
                uint32_t k = leaf_base + morton_key((uint32_t)sx, (uint32_t)sy);
                b = leaf_start[k];
                len = leaf_start[k + 1] - b;
            }
        }
        uint32_t incl = len;  // inclusive prefix over lanes 0..8
        for (int o = 1; o < 16; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        __syncwarp();  // earlier readers of ranges are done
        if (lane < 9) {
            rbeg[lane] = b;
            rpre[lane + 1] = incl;
        }
        if (lane == 0) rpre[0] = 0;
        __syncwarp();
    }
    c.rbeg = rbeg;
    c.rpre = rpre;
    c.ctotal = 0;
    c.cbeg = ranges + 19;
    c.cpre = ranges + 35;
    if (kCut) {  // lane r < 16 reads ring range r (leaves wholly beyond a skipped)
        uint32_t b = 0, len = 0;
        if (lane < 16 && ((nm.ring_mask >> lane) & 1u)) {
            int dx, dy;
            ring_offset(lane, &dx, &dy);
            const int sx = (int)lx + dx, sy = (int)ly + dy;
            if (sx >= 0 && sy >= 0 && sx < nl && sy < nl) {
                uint32_t k = leaf_base + morton_key((uint32_t)sx, (uint32_t)sy);
                b = leaf_start[k];
                len = leaf_start[k + 1] - b;
                if (rs.rec && nm.wstrip > 0.f) {  // the ring leaf's strip facing this leaf
                    const uint32_t sd = dx == 2 ? 0u : dx == -2 ? 1u : dy == 2 ? 2u : 3u;
                    b = 4u * b + sd * len;
                    len = rs.n[4u * k + sd];
                }
            }
        }
        uint32_t incl = len;
        for (int o = 1; o < 16; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        uint32_t* cb = ranges + 19;
        uint32_t* cp = ranges + 35;
        if (lane < 16) {
            cb[lane] = b;
            cp[lane + 1] = incl;
        }
        if (lane == 0) cp[0] = 0;
        c.ctotal = __shfl_sync(0xffffffffu, incl, 15);
        __syncwarp();
    }
    leaf_centre_hilo(g, lx, ly, &c.cxh, &c.cxl, &c.cyh, &c.cyl);
    c.le_leaf = nullptr;
    if (g.L >= 2 && le) {  // null le: near field only, the far field is added later
        if constexpr (kFlat) leaf_le_build_unrolled(g, le, l2l, lx, ly, leaf_le);
        else leaf_le_build(g, le, l2l, lx, ly, leaf_le);
        c.le_leaf = reinterpret_cast<const float*>(leaf_le);
    }
    const float4* rsrc = rs.rec && nm.wstrip > 0.f ? rs.rec : sp;  // where the ring ranges point
    const uint32_t total = rpre[9];
    const bool one_chunk = total <= kListChunk && (!kCut || c.ctotal == 0);  // ring reuses buf
    uint32_t nn = 0, nf = 0;
    if (one_chunk) gather_bands<kFlat>(sp, c, nm, 0, total, buf, nn, nf);

    // far field (L2P, Eq. 12) plus near sum -> velocity of one target, at
    // its input index or (kSorted, near part alone) at its sorted position
    // ks, coalesced, for the L2P kernel that follows
    auto finish = [&](const float4& rec, uint32_t ks, float x, float y, float su, float sv) {
        float u = __fmul_rn(nm.kvel, su), v = __fmul_rn(nm.kvel, sv);
        if (c.le_leaf)
            l2p_add(g.p, nm.kzeta, nm.inv_s, reinterpret_cast<const float2*>(c.le_leaf), x, y,
                    u, v);
        const uint32_t o = kSorted ? ks : __float_as_uint(rec.w);
        uv[2 * (int64_t)o] = u;
        uv[2 * (int64_t)o + 1] = v;
    };

    // passes of 32 T targets, T per lane (targets tb + lane + 32 t); in a
    // leaf's last round fewer than 32 targets may be active
    auto pass = [&](auto tag, uint32_t tb, uint32_t active) {
        constexpr int T = decltype(tag)::value;
        float4 rec[T];
        float x[T], y[T];
        SumT<T> S;
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const uint32_t k = 32 * t + lane;
            rec[t] = sp[c.t0 + tb + (k < active ? k : 0)];
            x[t] = ((rec[t].x - c.cxh) - c.cxl) * nm.sc;
            y[t] = ((rec[t].y - c.cyh) - c.cyl) * nm.sc;
            S.su[t] = S.sv[t] = S.cu[t] = S.cv[t] = 0.f;
        }
        for (uint32_t cb = 0; cb < total; cb += kListChunk) {
            if (!one_chunk)
                gather_bands<kFlat>(sp, c, nm, cb, min(kListChunk, total - cb), buf, nn, nf);
            band_loopT<kNearBand, T>(buf, 0, near_pairs(nn), nm, x, y, S);
            band_loopT<kFar, T>(buf, far_first(nf), kListCap / 2, nm, x, y, S);
        }
        if (kCut)
            for (uint32_t cb = 0; cb < c.ctotal; cb += kListChunk) {  // cutoff ring
                uint32_t nc;
                gather_ring<kFlat>(rsrc, c, nm, cb, min(kListChunk, c.ctotal - cb), buf, nc);
                band_loopT<kRing, T>(buf, 0, near_pairs(nc), nm, x, y, S);
            }
#pragma unroll
        for (int t = 0; t < T; ++t)
            if (32 * t + lane < active)
                finish(rec[t], c.t0 + tb + 32 * t + lane, x[t], y[t], S.su[t] + S.cu[t],
                       S.sv[t] + S.cv[t]);
    };
    uint32_t tb = a;
    if (kMaxT >= 4 && b - tb == 128) {  // 128 targets: four per lane, the list gathered once
        pass(std::integral_constant<int, 4>{}, tb, 128u);
        tb = b;
    }
    // passes of 64 targets, two per lane, and at a chunk's end passes of 49
    // to 63 (one gather of the list for what would otherwise be two rounds;
    // the last round then keeps more than 16 targets, as a leaf's last round
    // of at most 16 takes the split path below in whichever work item it
    // falls)
    for (; tb + 48 < b; tb += 64) pass(std::integral_constant<int, 2>{}, tb, min(64u, b - tb));
    // rounds of 17..32 targets, one per lane
    for (; tb + 16 < b; tb += 32) pass(std::integral_constant<int, 1>{}, tb, min(32u, b - tb));
    if (tb < b) {  // a leaf's last round of at most 16 targets: ns lanes per target
        const uint32_t tc = b - tb;
        const int ns = (int)(32u / tc);  // lanes per target, 2..32
        const uint32_t tl = lane / ns;
        const int sl = lane % ns;
        const bool active = tl < tc;
        const float4 rec = sp[c.t0 + tb + (active ? tl : 0)];
        const float x = ((rec.x - c.cxh) - c.cxl) * nm.sc, y = ((rec.y - c.cyh) - c.cyl) * nm.sc;
        float su = 0.f, sv = 0.f, cu = 0.f, cv = 0.f;
        for (uint32_t cb = 0; cb < total; cb += kListChunk) {
            if (!one_chunk)
                gather_bands<kFlat>(sp, c, nm, cb, min(kListChunk, total - cb), buf, nn, nf);
            band_loop_split<kNearBand>(buf, 0, near_pairs(nn), ns, sl, nm, x, y, su, sv, cu, cv);
            band_loop_split<kFar>(buf, far_first(nf), kListCap / 2, ns, sl, nm, x, y, su, sv, cu,
                                  cv);
        }
        if (kCut)
            for (uint32_t cb = 0; cb < c.ctotal; cb += kListChunk) {  // cutoff ring
                uint32_t nc;
                gather_ring<kFlat>(rsrc, c, nm, cb, min(kListChunk, c.ctotal - cb), buf, nc);
                band_loop_split<kRing>(buf, 0, near_pairs(nc), ns, sl, nm, x, y, su, sv, cu, cv);
            }
        su += cu;
        sv += cv;
        // the target's ns partial sums, a segmented tree: after the step of
        // width o, lane sl holds the sum of lanes sl .. sl + 2o - 1 of its
        // segment (clipped at ns)
        for (int o = 1; o < ns; o <<= 1) {
            const float pu = __shfl_down_sync(0xffffffffu, su, o);
            const float pv = __shfl_down_sync(0xffffffffu, sv, o);
            if (sl + o < ns) {
                su += pu;
                sv += pv;
            }
        }
        if (active && sl == 0) finish(rec, c.t0 + tb + tl, x, y, su, sv);
    }
    __syncwarp();  // the buffer may be reused by this warp's next chunk
}

// Work items of one near-field pass over n sorted targets.  Items
// [0, nbig) are windows of `span` positions (128, or 64 when there are few
// windows per resident warp), covering [0, nbig span); the rest are windows of
// 32 positions covering [nbig span, n).  A big window runs every chunk (span
// targets from a multiple of span past its leaf's first target) that starts
// inside it; a small window runs every round (32 targets from a multiple of
// 32 past the leaf's first target) that starts inside it and whose chunk
// starts at or after nbig span (earlier chunks are a big window's).  Small
// items at the end keep the last warps' work short; neither the window size
// nor the split changes a target's arithmetic, only how rounds are grouped.
struct WorkSplit {
    uint32_t n, span, nbig, items;
};

// The small items cover about half a window per resident warp (the spread
// of the warps' finishing times), at most a quarter of the windows.  Windows
// of 128 targets give each lane four targets but take a warp long to finish;
// with fewer than 8 of them per warp the tail would dominate, and windows of
// 64 are used.
static WorkSplit work_split(uint64_t n, uint64_t warps) {
    const uint32_t span = (n + kTicket - 1) / kTicket >= 8 * warps ? kTicket : kTicket / 2;
    const uint64_t windows = (n + span - 1) / span;
    const uint64_t nbig = windows - std::min(windows / 4, warps / 2 + 1);
    const uint64_t rest = n - std::min<uint64_t>(n, nbig * span);
    return WorkSplit{(uint32_t)n, span, (uint32_t)nbig, (uint32_t)(nbig + (rest + 31) / 32)};
}

// Sparse leaves (Sec. 3.3.1's local lists of a few particles each): with at
// most kLaneMaxT targets a leaf would leave most of a warp idle, and its
// fixed costs (the ranges of its 25 neighbours, the gathers, its local
// expansion) outweigh its pairs.  In an evaluation whose mean occupancy is
// at most kLaneMean particles per leaf, such leaves are skipped here and
// taken by the per-target-lane pass (p2p_lane_kernel), which gives each of
// their targets a lane.  The choice depends on the leaf's count and the
// evaluation's n and L alone, so a target gets the same arithmetic in a
// single and a batched evaluation, whatever warp it lands in.
constexpr uint32_t kLaneMaxT = 16;
constexpr int64_t kLaneMean = 32;

// f(key, a, b) for every chunk or round that item w owns: key the leaf index
// into leaf_start, [a, b) its targets within the leaf.  Warp-uniform calls.
// kSkip: leaves of nt <= kLaneMaxT targets whose gate(key) (the evaluation's
// bound, 0 or kLaneMaxT) admits them are left to the per-target-lane pass
// (the kernels are compiled with and without the test: its registers cost
// the dense evaluations that never use it).
template <bool kSkip, typename Gate, typename F>
__device__ __forceinline__ void for_each_piece(const uint32_t* __restrict__ skeys,
                                               const uint32_t* __restrict__ leaf_start,
                                               const WorkSplit& ws, uint32_t w, Gate&& gate,
                                               F&& f) {
    const int lane = threadIdx.x & 31;
    const bool big = w < ws.nbig;
    const uint32_t split = ws.nbig * ws.span;
    const uint32_t r0 = big ? w * ws.span : split + (w - ws.nbig) * 32u;
    const uint32_t span = big ? ws.span : 32u;
    const uint32_t r1 = min(r0 + span, ws.n);
    for (uint32_t base = r0; base < r1; base += 32) {
        const uint32_t r = base + lane;
        uint32_t key = 0, first = 0, nt = 0;
        bool starts = false;
        if (r < r1) {
            key = skeys[r];
            first = leaf_start[key];
            const uint32_t off = r - first;
            starts = (off & (span - 1)) == 0 &&
                     (big || first + (off & ~(ws.span - 1)) >= split);
            if (kSkip && starts) {
                nt = leaf_start[key + 1] - first;
                if (nt <= kLaneMaxT && nt <= gate(key)) starts = false;
            }
        }
        unsigned m = __ballot_sync(0xffffffffu, starts);
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            const uint32_t k = __shfl_sync(0xffffffffu, key, src);
            const uint32_t f0 = __shfl_sync(0xffffffffu, first, src);
            const uint32_t a = base + (uint32_t)src - f0;
            const uint32_t ntk =
                kSkip ? __shfl_sync(0xffffffffu, nt, src) : leaf_start[k + 1] - f0;
            f(k, a, min(a + span, ntk));
        }
    }
}

// Persistent: as many CTAs as fit on the GPU at once; each warp pulls work
// items from a counter (zeroed before the launch) until none is left, so
// crowded windows balance against light ones and no SM idles behind a
// partial last wave.
template <bool kCut, int kMaxT, bool kSorted, bool kSkip>
__global__ void __launch_bounds__(kLeafWarps * 32, 6)
p2p_l2p_f32_kernel(const float4* __restrict__ sp, const uint32_t* __restrict__ skeys,
                   const uint32_t* __restrict__ leaf_start, WorkSplit ws, uint32_t* counter,
                   Geometry g, NearF32v3 nm, const float* __restrict__ le,
                   const float* __restrict__ l2l, float* __restrict__ uv, RingStrips rs) {
    __shared__ float4 lists[kLeafWarps][kListCap];
    __shared__ uint32_t ranges[kLeafWarps][kCut ? 52 : 20];
    __shared__ float2 leaf_le[kLeafWarps][kMaxP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto gate = [&](uint32_t) { return nm.lane_nt; };
    for (;;) {
        uint32_t w = 0;
        if (lane == 0) w = atomicAdd(counter, 1u);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= ws.items) break;
        for_each_piece<kSkip>(skeys, leaf_start, ws, w, gate,
                              [&](uint32_t leaf, uint32_t a, uint32_t b) {
            p2p_chunk_f32<kCut, kMaxT, kSorted>(sp, leaf_start, 0, leaf, a, b, g, nm, le, l2l,
                                                uv, lists[warp], ranges[warp], leaf_le[warp], rs);
        });
    }
}

// Per-instance near-field constants of a batched evaluation.
struct NearInst {
    float sc, kvel, kzeta, inv_s, half_leaf;
    float qa, band_a2;   // the instance's cutoff of Sec. 4.1 (0: none)
    float wstrip;        // its ring strips' width
    uint32_t ring_mask;  // its ring leaves nearer than a
    uint32_t lane_nt;    // its sparse leaves' bound for the per-target-lane pass
};

// Ring strips of the cutoff (Sec. 4.1), one warp per leaf: the leaf's
// records within wstrip of each side (scaled leaf-relative coordinates; 0
// left, 1 right, 2 bottom, 3 top), compacted in sorted order to
// rs.rec[4 t0 + side n ...], their counts to rs.n[4 leaf + side].  A ring leaf
// two leaves away can keep (closer than the cutoff to its square, with the
// near-field kernel's margin) only sources of this leaf's strip on the side
// facing it, so the near field gathers the strip instead of the whole leaf:
// the same kept sources in the same order.  kBatch: leaf is a global leaf of
// a batch (its instance's geometry and constants); otherwise of one tree.
template <bool kBatch>
__global__ void __launch_bounds__(kLeafWarps * 32)
ring_strips_kernel(const float4* __restrict__ sp, const uint32_t* __restrict__ leaf_start,
                   uint32_t nleaf, Geometry g1, NearF32v3 nm1,
                   const BatchInst* __restrict__ inst, const NearInst* __restrict__ near_inst,
                   const int32_t* __restrict__ leaf_inst, RingStrips rs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t leaf = blockIdx.x * kLeafWarps + warp;
    if (leaf >= nleaf) return;  // warp-uniform
    const unsigned lt = (1u << lane) - 1u;
    float sc = nm1.sc, hl = nm1.half_leaf, w = nm1.wstrip;
    uint32_t local = leaf;
    const Geometry* g = &g1;
    if (kBatch) {
        const int i = leaf_inst[leaf];
        const NearInst ni = near_inst[i];
        if (ni.ring_mask == 0 || !(ni.wstrip > 0.f)) return;  // its strips are never read
        sc = ni.sc;
        hl = ni.half_leaf;
        w = ni.wstrip;
        g = &inst[i].g;
        local = leaf - inst[i].leaf_base;
    }
    const uint32_t t0 = leaf_start[leaf], n = leaf_start[leaf + 1] - t0;
    float cxh, cxl, cyh, cyl;
    leaf_centre_hilo(*g, morton_compact(local), morton_compact(local >> 1), &cxh, &cxl, &cyh,
                     &cyl);
    const float lo = w - hl, hi = hl - w;  // X < lo: left strip; X > hi: right strip
    uint32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
    float4* out = rs.rec + 4 * (int64_t)t0;
    for (uint32_t g0 = 0; g0 < n; g0 += 32) {
        const uint32_t k = g0 + lane;
        const bool in = k < n;
        float4 rec = make_float4(0.f, 0.f, 0.f, 0.f);
        float X = 0.f, Y = 0.f;
        if (in) {
            rec = sp[t0 + k];
            X = ((rec.x - cxh) - cxl) * sc;
            Y = ((rec.y - cyh) - cyl) * sc;
        }
        auto put = [&](bool f, uint32_t side, uint32_t& cnt) {
            const unsigned m = __ballot_sync(0xffffffffu, f);
            if (f) out[side * n + cnt + __popc(m & lt)] = rec;
            cnt += __popc(m);
        };
        put(in && X < lo, 0u, c0);
        put(in && X > hi, 1u, c1);
        put(in && Y < lo, 2u, c2);
        put(in && Y > hi, 3u, c3);
    }
    if (lane < 4) rs.n[4 * leaf + lane] = lane == 0 ? c0 : lane == 1 ? c1 : lane == 2 ? c2 : c3;
}

// Batched and persistent: warps pull work items over the global sorted order
// (all instances, packed) from a work counter.  kCut compiles in the cutoff
// ring of Sec. 4.1 for batches where some instance has a cutoff (the others
// have an empty ring and skip it).
template <bool kCut, bool kSkip>
__global__ void __launch_bounds__(kLeafWarps * 32, 6)
p2p_batch_kernel(const float4* __restrict__ sp, const uint32_t* __restrict__ skeys,
                 const uint32_t* __restrict__ leaf_start, const BatchInst* __restrict__ inst,
                 const NearInst* __restrict__ near_inst, const int32_t* __restrict__ leaf_inst,
                 WorkSplit ws, uint32_t* counter, NearF32v3 shared_nm,
                 const float* __restrict__ le, const float* __restrict__ l2l16,
                 const float* __restrict__ l2l32, float* __restrict__ uv, RingStrips rs) {
    __shared__ float4 lists[kLeafWarps][kListCap];
    __shared__ uint32_t ranges[kLeafWarps][kCut ? 52 : 20];
    __shared__ float2 leaf_le[kLeafWarps][kMaxP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto gate = [&](uint32_t gleaf) { return near_inst[leaf_inst[gleaf]].lane_nt; };
    for (;;) {
        uint32_t w = 0;
        if (lane == 0) w = atomicAdd(counter, 1u);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= ws.items) break;
        for_each_piece<kSkip>(skeys, leaf_start, ws, w, gate,
                              [&](uint32_t gleaf, uint32_t a, uint32_t e) {
            const int i = leaf_inst[gleaf];
            const BatchInst& b = inst[i];
            NearF32v3 nm = shared_nm;
            const NearInst ni = near_inst[i];
            nm.sc = ni.sc;
            nm.kvel = ni.kvel;
            nm.kzeta = ni.kzeta;
            nm.inv_s = ni.inv_s;
            nm.half_leaf = ni.half_leaf;
            nm.qa = ni.qa;
            nm.band_a2 = ni.band_a2;
            nm.wstrip = ni.wstrip;
            nm.ring_mask = ni.ring_mask;
            p2p_chunk_f32<kCut, kCut ? 2 : 4, false, true>(sp, leaf_start, b.leaf_base,
                                                           gleaf - b.leaf_base, a,
                                              e, b.g, nm, le + b.exp_off,
                                              b.g.P <= 16 ? l2l16 : l2l32, uv, lists[warp],
                                              ranges[warp], leaf_le[warp], rs);
        });
    }
}

// ---------------------------------------------------------------------------
// Per-target-lane pass over the targets of sparse leaves.
//
// Warps take windows of 32 sorted positions (a CTA four consecutive ones, so
// that its warps read neighbouring records and share them in L1); a lane
// whose target lies in a leaf of at most kLaneMaxT targets (in a sparse
// evaluation) walks that target's local list itself: the 9 ranges of its
// leaf's 3x3 neighbourhood, then (with a cutoff) the ring leaves that come
// within the cutoff of the target, reading the sorted records from global
// memory (the lanes of one leaf read the same records: one broadcast), two
// records per step as one packed pair.  Every pair of the 3x3 block takes
// the near-band form (the polynomial below qthr), every ring pair the cutoff
// correction.  The walk's trip count is the warp's longest list; a lane past
// its own end evaluates dummies (zero circulation, far away).  Sums: blocks
// of kLanePairs pairs into fresh registers, then compensated.  Far field
// (when le is given): the leaf's two expansion parts, staged once per warp
// in shared memory, evaluated by each lane (l2p_two_levels).  A target's
// arithmetic does not depend on which warp or lane takes it.
// ---------------------------------------------------------------------------
constexpr int kLaneRanges = 25;      // 9 local + 16 ring
constexpr uint32_t kLanePairs = 32;  // pairs per first-level partial sum
constexpr int kLaneSlots = 12;       // leaves' expansion parts staged at a time

// Per warp: the lanes' source ranges while the sums run, then the two
// expansion parts of the warp's leaves (6.4 KB: with 7 CTAs of 4 warps,
// 179 KB of shared memory per SM, the rest left to L1 for the records).
union LaneSmem {
    struct {
        uint32_t beg[kLaneRanges][32];  // range r of lane l at [r][l]
        uint32_t end[kLaneRanges][32];
    } r;
    struct {
        float2 own[kMaxP + 1];  // padded: lanes of different leaves in different banks
        float2 par[kMaxP + 1];
    } le[kLaneSlots];
};

// The windows of 32 sorted positions a lane pass visits: win[0 .. count)
// (window w covers positions 32 w .. 32 w + 31 below n), or with win null
// windows 0 .. count - 1.
struct LaneWindows {
    const uint32_t* win;
    uint32_t count;
    uint32_t n;
};

// Leaf centre as FP32 hi/lo pairs for the calling lane alone (the table, or
// the FP64 formula the table is built with: the same values).
__device__ __forceinline__ void lane_centre_hilo(const Geometry& g, uint32_t ix, uint32_t iy,
                                                 float* cxh, float* cxl, float* cyh,
                                                 float* cyl) {
    if (g.centre_tab) {
        const float4 a = g.centre_tab[ix], b = g.centre_tab[iy];
        *cxh = a.x;
        *cxl = a.y;
        *cyh = b.z;
        *cyl = b.w;
    } else {
        centre_hilo_1d(g.x0, g.W, g.L, ix, cxh, cxl);
        centre_hilo_1d(g.y0, g.W, g.L, iy, cyh, cyl);
    }
}

// The lane's records against its target, two per step for `steps` steps
// (the warp's longest walk): `left` records from the non-empty ranges
// r0, r0 + 1, ... (compacted in shared memory).  Past its own end a lane
// evaluates dummies.
template <int kMode>
__device__ __forceinline__ void lane_walk(const float4* __restrict__ sp, const LaneSmem& sm,
                                          int r0, uint32_t left, uint32_t steps,
                                          const NearF32v3& nm, float2 ch, float2 cl, float x,
                                          float y, float& su, float& sv, float& cu, float& cv) {
    const int lane = threadIdx.x & 31;
    int r = r0;
    uint32_t pos = sm.r.beg[r][lane], end = sm.r.end[r][lane];
    // the record at pos (false: the lane's list is done), then the walk moves
    // on, to the next range at the end of this one (branch-free)
    auto take = [&](uint32_t& at) {
        at = pos;
        const bool v = left > 0;
        left -= v ? 1u : 0u;
        ++pos;
        const bool adv = pos == end;
        r += adv ? 1 : 0;
        const int rr = min(r, kLaneRanges - 1);
        const uint32_t nb = sm.r.beg[rr][lane], ne = sm.r.end[rr][lane];
        pos = adv ? nb : pos;
        end = adv ? ne : end;
        return v;
    };
    const float2 tx = f2_dup(x), ty = f2_dup(y), scv = f2_dup(nm.sc);
#pragma unroll 1
    for (uint32_t k0 = 0; k0 < steps; k0 += kLanePairs) {
        const uint32_t k1 = min(k0 + kLanePairs, steps);
        float2 iu = make_float2(0.f, 0.f), iv = iu;
#pragma unroll 2  // two steps' loads in flight: 5% faster than one
        for (uint32_t k = k0; k < k1; ++k) {
            uint32_t ia, ib;
            const bool va = take(ia), vb = take(ib);
            const float4 qa = sp[va ? ia : 0u], qb = sp[vb ? ib : 0u];  // both loads in flight
            // scaled leaf-relative (x, y) of each, ((x - c_hi) - c_lo) sc, packed
            const float2 da = f2_mul(f2_sub(f2_sub(make_float2(qa.x, qa.y), ch), cl), scv);
            const float2 db = f2_mul(f2_sub(f2_sub(make_float2(qb.x, qb.y), ch), cl), scv);
            const float xa = va ? da.x : kFarAway, ya = va ? da.y : kFarAway;
            const float xb = vb ? db.x : kFarAway, yb = vb ? db.y : kFarAway;
            const float ga = va ? qa.z : 0.f, gb = vb ? qb.z : 0.f;
            pair_sources<kMode>(nm, make_float4(xa, xb, ya, yb), make_float4(ga, gb, -ga, -gb),
                                tx, ty, iu, iv);
        }
        neumaier_add(su, cu, iu.x + iu.y);
        neumaier_add(sv, cv, iv.x + iv.y);
    }
}

// Persistent over the windows.  kBatch: the targets belong to the instances
// of a batch (each lane its own instance's geometry and constants);
// otherwise to one evaluation (g, nm).  kSorted: near parts alone at the
// sorted positions (le null); otherwise at the input indices.
template <bool kBatch, bool kCut, bool kSorted>
__global__ void __launch_bounds__(kLeafWarps * 32, 7)  // 72 registers: 2% faster than 6 CTAs
p2p_lane_kernel(const float4* __restrict__ sp, const uint32_t* __restrict__ skeys,
                const uint32_t* __restrict__ leaf_start, LaneWindows lw, Geometry g,
                NearF32v3 nm, const BatchInst* __restrict__ inst,
                const NearInst* __restrict__ near_inst, const int32_t* __restrict__ leaf_inst,
                const float* __restrict__ le, const float* __restrict__ l2l16,
                const float* __restrict__ l2l32, float* __restrict__ uv) {
    __shared__ LaneSmem smem[kLeafWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    LaneSmem& sm = smem[warp];
    for (uint32_t gw = blockIdx.x * kLeafWarps + warp; gw < lw.count;
         gw += gridDim.x * kLeafWarps) {
        const uint32_t r = (lw.win ? lw.win[gw] : gw) * 32u + lane;
        // the target's leaf and evaluation: geometry, constants, first leaf
        uint32_t key = 0, nt = 0;
        if (r < lw.n) {
            key = skeys[r];
            nt = leaf_start[key + 1] - leaf_start[key];
        }
        int ii = 0;
        uint32_t leaf_base = 0, gate = nm.lane_nt;
        NearF32v3 m = nm;
        const Geometry* gp = &g;
        if constexpr (kBatch) {
            ii = leaf_inst[key];
            const NearInst ni = near_inst[ii];
            m.sc = ni.sc;
            m.kvel = ni.kvel;
            m.kzeta = ni.kzeta;
            m.inv_s = ni.inv_s;
            m.qa = ni.qa;
            m.ring_mask = ni.ring_mask;
            m.half_leaf = ni.half_leaf;
            m.band_a2 = ni.band_a2;
            gate = ni.lane_nt;
            leaf_base = inst[ii].leaf_base;
            gp = &inst[ii].g;
        }
        const bool active = r < lw.n && nt <= kLaneMaxT && nt <= gate;
        if (!__any_sync(0xffffffffu, active)) continue;
        const int L = gp->L;
        const int nl = 1 << L;
        const uint32_t leaf = key - leaf_base;
        const uint32_t lx = morton_compact(leaf), ly = morton_compact(leaf >> 1);
        const float4 rec = sp[r < lw.n ? r : 0u];
        float cxh, cxl, cyh, cyl;
        lane_centre_hilo(*gp, lx, ly, &cxh, &cxl, &cyh, &cyl);
        const float x = ((rec.x - cxh) - cxl) * m.sc, y = ((rec.y - cyh) - cyl) * m.sc;

        // the lane's non-empty ranges, compacted: the 3x3 block in row order
        // from slot 0, then the ring from slot 9
        __syncwarp();  // the warp's previous readers of sm are done
        uint32_t tot_l = 0, tot_r = 0;
        int nr = 0;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const int sx = (int)lx + q % 3 - 1, sy = (int)ly + q / 3 - 1;
            uint32_t b = 0, e = 0;
            if (active && sx >= 0 && sy >= 0 && sx < nl && sy < nl) {
                const uint32_t k = leaf_base + morton_key((uint32_t)sx, (uint32_t)sy);
                b = leaf_start[k];
                e = leaf_start[k + 1];
            }
            if (e > b) {
                sm.r.beg[nr][lane] = b;
                sm.r.end[nr][lane] = e;
                ++nr;
            }
            tot_l += e - b;
        }
        if (kCut) {
            nr = 9;
            sm.r.beg[9][lane] = 0;  // an empty ring reads one dummy range
            sm.r.end[9][lane] = 0;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                int dx, dy;
                ring_offset(q, &dx, &dy);
                const int sx = (int)lx + dx, sy = (int)ly + dy;
                uint32_t b = 0, e = 0;
                // a ring leaf farther than the cutoff from the target itself holds
                // no pair under it (band_a2's 2% margin covers the roundings)
                const float ex =
                    fmaxf(fabsf(x - (float)(2 * dx) * m.half_leaf) - m.half_leaf, 0.f);
                const float ey =
                    fmaxf(fabsf(y - (float)(2 * dy) * m.half_leaf) - m.half_leaf, 0.f);
                if (active && ((m.ring_mask >> q) & 1u) && sx >= 0 && sy >= 0 && sx < nl &&
                    sy < nl && fmaf(ex, ex, ey * ey) < m.band_a2) {
                    const uint32_t k = leaf_base + morton_key((uint32_t)sx, (uint32_t)sy);
                    b = leaf_start[k];
                    e = leaf_start[k + 1];
                }
                if (e > b) {
                    sm.r.beg[nr][lane] = b;
                    sm.r.end[nr][lane] = e;
                    ++nr;
                }
                tot_r += e - b;
            }
        }
        __syncwarp();
        const float2 ch = make_float2(cxh, cyh), cl = make_float2(cxl, cyl);
        float su = 0.f, sv = 0.f, cu = 0.f, cv = 0.f;
        lane_walk<kNearBand>(sp, sm, 0, tot_l, __reduce_max_sync(0xffffffffu, (tot_l + 1) >> 1),
                             m, ch, cl, x, y, su, sv, cu, cv);
        if (kCut) {
            const uint32_t steps = __reduce_max_sync(0xffffffffu, (tot_r + 1) >> 1);
            if (steps) lane_walk<kRing>(sp, sm, 9, tot_r, steps, m, ch, cl, x, y, su, sv, cu, cv);
        }
        su += cu;
        sv += cv;
        float u = __fmul_rn(m.kvel, su), v = __fmul_rn(m.kvel, sv);

        if (le) {  // far field: each leaf's two expansion parts staged once per warp
            const uint32_t prev = __shfl_up_sync(0xffffffffu, key, 1);
            const bool lead = active && (lane == 0 || prev != key);
            const unsigned lm = __ballot_sync(0xffffffffu, lead);
            const unsigned upto = lane == 31 ? 0xffffffffu : (2u << lane) - 1u;
            const int mine = __popc(lm & upto) - 1;  // this lane's leaf among the leaders
            const unsigned far = __ballot_sync(0xffffffffu, L >= 2);
            unsigned todo = lm;
            for (int base = 0; todo; base += kLaneSlots) {  // kLaneSlots leaves at a time
                __syncwarp();  // earlier readers of sm are done
                for (int sj = 0; sj < kLaneSlots && todo; ++sj, todo &= todo - 1) {
                    const int j = __ffs(todo) - 1;
                    if (!((far >> j) & 1u)) continue;
                    const uint32_t jlx = __shfl_sync(0xffffffffu, lx, j);
                    const uint32_t jly = __shfl_sync(0xffffffffu, ly, j);
                    if constexpr (kBatch) {
                        const BatchInst& b = inst[__shfl_sync(0xffffffffu, ii, j)];
                        stage_two_levels(b.g, le + b.exp_off, jlx, jly, sm.le[sj].own,
                                         sm.le[sj].par);
                    } else {
                        stage_two_levels(g, le, jlx, jly, sm.le[sj].own, sm.le[sj].par);
                    }
                }
                __syncwarp();
                if (active && L >= 2 && mine >= base && mine < base + kLaneSlots) {
                    const int sl = mine - base;
                    l2p_two_levels(gp->p, m.kzeta, m.inv_s, sm.le[sl].own,
                                   L >= 3 ? sm.le[sl].par : nullptr, lx & 1u, ly & 1u, x, y, u,
                                   v);
                }
            }
        }
        if (active) {
            const uint32_t o = kSorted ? r : __float_as_uint(rec.w);
            uv[2 * (int64_t)o] = u;
            uv[2 * (int64_t)o + 1] = v;
        }
    }
}

// Polynomial interpolating g(q2) = (1 - 2^-q2)/q2 at the Chebyshev nodes of
// [0, a]; coefficients of q2^k.  Solved in double by Gaussian elimination
// with partial pivoting on the scaled variable u = q2 / a.  Returns the
// largest relative error on a fine grid (double evaluation).
double fit_near_polynomial(double a, double* coef) {
    const int n = kF32Deg + 1;
    const double pi = 3.14159265358979323846, ln2 = 0.69314718055994530942;
    auto gfun = [&](double x) { return x > 0.0 ? -expm1(-x * ln2) / x : ln2; };
    double A[kF32Deg + 1][kF32Deg + 2];
    for (int i = 0; i < n; ++i) {
        double u = 0.5 * (cos(pi * (i + 0.5) / n) + 1.0);
        double pw = 1.0;
        for (int k = 0; k < n; ++k) {
            A[i][k] = pw;
            pw *= u;
        }
        A[i][n] = gfun(a * u);
    }
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        for (int k = 0; k <= n; ++k) {
            double t = A[c][k];
            A[c][k] = A[piv][k];
            A[piv][k] = t;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double f = A[r][c] / A[c][c];
            for (int k = c; k <= n; ++k) A[r][k] -= f * A[c][k];
        }
    }
    double scale = 1.0;
    for (int k = 0; k < n; ++k) {
        coef[k] = A[k][n] / A[k][k] / scale;
        scale *= a;
    }
    double worst = 0.0;
    for (int i = 0; i <= 4000; ++i) {
        double x = a * i / 4000.0, p = coef[n - 1];
        for (int k = n - 2; k >= 0; --k) p = p * x + coef[k];
        worst = fmax(worst, fabs(p - gfun(x)) / gfun(x));
    }
    return worst;
}

}  // namespace

// Ring leaves that can hold a source closer than the cutoff to some point of
// the target leaf: ring leaf (dx, dy) is (max(|dx| - 1, 0), max(|dy| - 1, 0))
// leaf widths from the leaf square.  Zero without a cutoff or below L = 2.
static uint32_t ring_mask(const Geometry& g) {
    if (g.L < 2 || !(g.cutoff > 0.0)) return 0;
    const double w = g.W / ldexp(1.0, g.L);
    uint32_t m = 0;
    for (int r = 0; r < 16; ++r) {
        int dx, dy;
        ring_offset(r, &dx, &dy);
        const double gx = std::max(std::abs(dx) - 1, 0) * w, gy = std::max(std::abs(dy) - 1, 0) * w;
        if (gx * gx + gy * gy < g.cutoff * g.cutoff * (1.0 + 1e-12)) m |= 1u << r;
    }
    return m;
}

// Near-field constants of an evaluation (formed in double, rounded once).
static NearF32v3 near_constants(double sigma, const Geometry& g, bool* ok) {
    const double ln2 = 0.69314718055994530942;
    const double pi = 3.14159265358979323846;
    NearF32v3 nm;
    double qthr = kPolyEdge;
    double box = g.W / ldexp(1.0, g.L);
    nm.sc = (float)sqrt(1.0 / (2.0 * sigma * sigma * ln2));
    nm.qthr = (float)qthr;
    nm.kvel = (float)(1.0 / (4.0 * pi * sigma * sigma * ln2 * (double)nm.sc));
    nm.kzeta = (float)(1.0 / ((double)nm.sc * box));
    nm.inv_s = (float)(1.0 / box);
    nm.half_leaf = (float)(0.5 * box * (double)nm.sc);
    nm.band2 = (float)(qthr * 1.02);  // q2 < qthr needs |dX|^2 < qthr; 2% margin for rounding
    const double qa = g.L >= 2 ? g.cutoff * g.cutoff * (double)nm.sc * (double)nm.sc : 0.0;
    nm.qa = (float)qa;
    nm.band_a2 = (float)(qa * 1.02);
    // a source of a ring leaf two leaves to the right is kept when its
    // distance to the target leaf's square, at least its distance from its
    // own leaf's left side plus one leaf width, is below sqrt(band_a2): the
    // strip is sqrt(band_a2) less a leaf wide (a margin of 1e-3 half-leaves
    // covers the rounding of the two leaves' frames)
    const double hl = 0.5 * box * (double)nm.sc;
    const double wstrip = sqrt(qa * 1.02) - 2.0 * hl + 1e-3 * hl;
    // strips pay while they are narrow: at most half a leaf (a up to 1.5 leaf
    // widths); wider, their writes cost more than the gathers they save, and
    // the ring is gathered from whole leaves (wstrip 0)
    nm.wstrip = qa > 0.0 && wstrip <= hl ? (float)wstrip : 0.f;
    nm.ring_mask = ring_mask(g);
    nm.lane_nt = 0;  // set by the launch from its particle count
    double coef[kF32Deg + 1];
    *ok = fit_near_polynomial(qthr, coef) <= 1e-8;
    for (int k = 0; k <= kF32Deg; ++k) nm.coef[k] = (float)coef[k];
    return nm;
}

// CTAs of `kernel` resident on the whole GPU at once (at least one).
static unsigned resident_ctas(const void* kernel) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kLeafWarps * 32, 0);
    return (unsigned)std::max(1, sms * std::max(per_sm, 1));
}

bool near_lane_path(int64_t n, int L) { return n > 0 && n <= (kLaneMean << (2 * L)); }

// The FP32 near field's launches: for a sparse evaluation (near_lane_path)
// the per-target-lane pass over every window of 32 sorted positions, then
// the warp path on the whole persistent grid (all CTAs that fit on the GPU
// at once; work counter zeroed first), skipping the lane pass's leaves.
// With le null they write the near part alone, at the input indices or
// (sorted_out) in sorted order.
static cudaError_t launch_near_f32(const Geometry& g, double sigma, int64_t n,
                                   const void* particles, const uint32_t* skeys,
                                   const uint32_t* leaf_start, uint32_t* counter,
                                   const float* le, const float* l2l, float* uv, bool sorted_out,
                                   RingStrips rs, cudaStream_t s) {
    bool ok;
    NearF32v3 nm = near_constants(sigma, g, &ok);
    if (!ok) return cudaErrorInvalidValue;
    if (n == 0) return cudaSuccess;
    const bool lanes = near_lane_path(n, g.L);
    if (lanes) nm.lane_nt = kLaneMaxT;
    const bool cut = nm.ring_mask != 0;  // some ring leaf can hold a pair closer than a
    const float4* sp = reinterpret_cast<const float4*>(particles);
    cudaError_t e;
    if (lanes) {
        const LaneWindows lw{nullptr, (uint32_t)((n + 31) / 32), (uint32_t)n};
        auto run = [&](auto kernel) {
            const unsigned lb = (unsigned)std::min<uint64_t>(
                resident_ctas(reinterpret_cast<const void*>(kernel)),
                (lw.count + kLeafWarps - 1) / kLeafWarps);
            kernel<<<dim3(lb), dim3(kLeafWarps * 32), 0, s>>>(sp, skeys, leaf_start, lw, g, nm,
                                                              nullptr, nullptr, nullptr, le,
                                                              l2l, nullptr, uv);
            return cudaGetLastError();
        };
        if (cut)
            e = sorted_out ? run(p2p_lane_kernel<false, true, true>)
                           : run(p2p_lane_kernel<false, true, false>);
        else
            e = sorted_out ? run(p2p_lane_kernel<false, false, true>)
                           : run(p2p_lane_kernel<false, false, false>);
        if (e != cudaSuccess) return e;
    }
    auto kernel_of = [&](int max_t) {
        return cut ? (max_t >= 4
                          ? reinterpret_cast<const void*>(p2p_l2p_f32_kernel<true, 4, false, false>)
                          : reinterpret_cast<const void*>(p2p_l2p_f32_kernel<true, 2, false, false>))
                   : reinterpret_cast<const void*>(p2p_l2p_f32_kernel<false, 4, false, false>);
    };
    const unsigned resident = resident_ctas(kernel_of(4));
    const WorkSplit ws = work_split((uint64_t)n, (uint64_t)resident * kLeafWarps);
    // chunks of 128 only with 128-target windows; the plain kernel stays wide
    const int max_t = ws.span >= 128 || !cut ? 4 : 2;
    if (resident_ctas(kernel_of(max_t)) != resident) return cudaErrorInvalidConfiguration;
    const unsigned needed = (ws.items + kLeafWarps - 1) / kLeafWarps;
    const unsigned blocks = std::min(needed, resident);
    e = cudaMemsetAsync(counter, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    if (!cut || !rs.n || !(nm.wstrip > 0.f)) rs.rec = nullptr;
    if (rs.rec) {
        const uint32_t nleaf = 1u << (2 * g.L);
        ring_strips_kernel<false><<<(nleaf + kLeafWarps - 1) / kLeafWarps, kLeafWarps * 32, 0, s>>>(
            sp, leaf_start, nleaf, g, nm, nullptr, nullptr, nullptr, rs);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    auto go = [&](auto kernel) {
        if (resident_ctas(reinterpret_cast<const void*>(kernel)) != resident)
            return cudaErrorInvalidConfiguration;
        kernel<<<dim3(blocks), dim3(kLeafWarps * 32), 0, s>>>(sp, skeys, leaf_start, ws, counter,
                                                              g, nm, le, l2l, uv, rs);
        return cudaGetLastError();
    };
    // the kernel for (cut, max_t, sorted_out), skipping the lane pass's leaves
    // when there is one
    auto pick = [&](auto skip) {
        constexpr bool kS = decltype(skip)::value;
        if (cut && max_t >= 4)
            return sorted_out ? go(p2p_l2p_f32_kernel<true, 4, true, kS>)
                              : go(p2p_l2p_f32_kernel<true, 4, false, kS>);
        if (cut)
            return sorted_out ? go(p2p_l2p_f32_kernel<true, 2, true, kS>)
                              : go(p2p_l2p_f32_kernel<true, 2, false, kS>);
        return sorted_out ? go(p2p_l2p_f32_kernel<false, 4, true, kS>)
                          : go(p2p_l2p_f32_kernel<false, 4, false, kS>);
    };
    return lanes ? pick(std::true_type{}) : pick(std::false_type{});
}

template <>
cudaError_t launch_p2p_l2p<float>(const Geometry& g, double sigma, int64_t n,
                                  const void* particles, const uint32_t* skeys,
                                  const uint32_t* leaf_start, uint32_t* counter, const float* le,
                                  const float* l2l, float* uv, cudaStream_t s) {
    return launch_near_f32(g, sigma, n, particles, skeys, leaf_start, counter, le, l2l, uv, false,
                           RingStrips{nullptr, nullptr}, s);
}

cudaError_t launch_near_only_f32(const Geometry& g, double sigma, int64_t n,
                                 const void* particles, const uint32_t* skeys,
                                 const uint32_t* leaf_start, uint32_t* counter, float* out,
                                 bool sorted_out, RingStrips strips, cudaStream_t s) {
    return launch_near_f32(g, sigma, n, particles, skeys, leaf_start, counter, nullptr, nullptr,
                           out, sorted_out, strips, s);
}

// L2P after a near-field-only pass: one warp per leaf adds the leaf's local
// expansion to each of its targets' near-field velocities and writes the sums
// at the targets' input indices, with the operations the fused kernel applies
// (leaf_le_load/finish, l2p_add), so the sum is the same bit for bit.  The
// kernel is bound by the latency of its loads.  kSorted: the near parts are
// read in sorted order (coalesced), and the loads that depend on the leaf
// alone (its expansion parts, centre and target range), then the lane's
// first two targets, are all issued before the expansion is formed.
// Otherwise the near parts are read back at the targets' input indices, leaf
// by leaf.
template <bool kSorted, bool kLanes>
__global__ void __launch_bounds__(kLeafWarps * 32)
l2p_f32_kernel(const float4* __restrict__ sp, const uint32_t* __restrict__ leaf_start, Geometry g,
               float sc, float kzeta, float inv_s, const float* __restrict__ le,
               const float* __restrict__ l2l, const float2* __restrict__ uvs,
               float* __restrict__ uv, uint32_t lane_nt) {
    __shared__ float2 leaf_le[kLeafWarps][kMaxP];
    __shared__ float2 parts[kLeafWarps][kLanes ? 2 : 1][kLanes ? kMaxP : 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t leaf = blockIdx.x * kLeafWarps + warp;
    if (leaf >= (1u << (2 * g.L))) return;  // warp-uniform
    const uint32_t lx = morton_compact(leaf), ly = morton_compact(leaf >> 1);
    float cxh, cxl, cyh, cyl;
    const bool uv8 = (reinterpret_cast<uintptr_t>(uv) & 7u) == 0;  // one 8-byte store
    auto add = [&](const float4& rec, float u, float v) {
        const float x = ((rec.x - cxh) - cxl) * sc, y = ((rec.y - cyh) - cyl) * sc;
        l2p_add(g.p, kzeta, inv_s, leaf_le[warp], x, y, u, v);
        const uint32_t idx = __float_as_uint(rec.w);
        if (kSorted && uv8) {
            *reinterpret_cast<float2*>(uv + 2 * (int64_t)idx) = make_float2(u, v);
        } else {
            uv[2 * (int64_t)idx] = u;
            uv[2 * (int64_t)idx + 1] = v;
        }
    };
    // a leaf of the per-target-lane pass: its far field as that pass forms it
    // (the expansion's two parts, l2p_two_levels)
    auto lane_leaf = [&](uint32_t t0, uint32_t t1) {
        stage_two_levels(g, le, lx, ly, parts[warp][0], parts[warp][kLanes ? 1 : 0]);
        __syncwarp();
        for (uint32_t k = t0 + lane; k < t1; k += 32) {
            const float4 rec = sp[k];
            const uint32_t idx = __float_as_uint(rec.w);
            float u, v;
            if (kSorted) {
                const float2 w = uvs[k];
                u = w.x;
                v = w.y;
            } else {
                u = uv[2 * (int64_t)idx];
                v = uv[2 * (int64_t)idx + 1];
            }
            const float x = ((rec.x - cxh) - cxl) * sc, y = ((rec.y - cyh) - cyl) * sc;
            l2p_two_levels(g.p, kzeta, inv_s, parts[warp][0],
                           g.L >= 3 ? parts[warp][kLanes ? 1 : 0] : nullptr, lx & 1u, ly & 1u,
                           x, y, u, v);
            if (kSorted && uv8) {
                *reinterpret_cast<float2*>(uv + 2 * (int64_t)idx) = make_float2(u, v);
            } else {
                uv[2 * (int64_t)idx] = u;
                uv[2 * (int64_t)idx + 1] = v;
            }
        }
    };
    if (!kSorted) {
        const uint32_t t0 = leaf_start[leaf], t1 = leaf_start[leaf + 1];
        if (t0 == t1) return;
        leaf_centre_hilo(g, lx, ly, &cxh, &cxl, &cyh, &cyl);
        if (kLanes && t1 - t0 <= lane_nt) {
            lane_leaf(t0, t1);
            return;
        }
        leaf_le_build(g, le, l2l, lx, ly, leaf_le[warp]);
        for (uint32_t k = t0 + lane; k < t1; k += 32) {
            const float4 rec = sp[k];
            const uint32_t idx = __float_as_uint(rec.w);
            add(rec, uv[2 * (int64_t)idx], uv[2 * (int64_t)idx + 1]);
        }
        return;
    }
    const LeafLeParts q = leaf_le_load(g, le, lx, ly);
    leaf_centre_hilo(g, lx, ly, &cxh, &cxl, &cyh, &cyl);
    const uint32_t t0 = leaf_start[leaf], t1 = leaf_start[leaf + 1];
    if (t0 == t1) return;
    if (kLanes && t1 - t0 <= lane_nt) {
        lane_leaf(t0, t1);
        return;
    }
    const uint32_t k0 = t0 + lane, k1 = k0 + 32;
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
    float2 w0 = make_float2(0.f, 0.f), w1 = w0;
    if (k0 < t1) {
        r0 = sp[k0];
        w0 = uvs[k0];
    }
    if (k1 < t1) {
        r1 = sp[k1];
        w1 = uvs[k1];
    }
    if (g.P == 16)
        leaf_le_finish16(g, l2l, lx, ly, q, leaf_le[warp]);
    else if (g.P == 32)
        leaf_le_finish32(g, l2l, lx, ly, q, leaf_le[warp]);
    else
        leaf_le_finish(g, l2l, lx, ly, q, leaf_le[warp]);
    if (k0 < t1) add(r0, w0.x, w0.y);
    if (k1 < t1) add(r1, w1.x, w1.y);
    for (uint32_t k = k1 + 32; k < t1; k += 32) {
        const float2 w = uvs[k];
        add(sp[k], w.x, w.y);
    }
}

cudaError_t launch_l2p_f32(const Geometry& g, double sigma, int64_t n, const void* particles,
                           const uint32_t* leaf_start, const float* le, const float* l2l,
                           const float* uv_sorted, float* uv, cudaStream_t s) {
    if (g.L < 2) return cudaSuccess;
    bool ok;
    const NearF32v3 nm = near_constants(sigma, g, &ok);
    if (!ok) return cudaErrorInvalidValue;
    const uint32_t lane_nt = near_lane_path(n, g.L) ? kLaneMaxT : 0u;
    const unsigned blocks = (unsigned)(((uint64_t)1 << (2 * g.L)) / kLeafWarps);
    const float4* sp = reinterpret_cast<const float4*>(particles);
    const float2* uvs = reinterpret_cast<const float2*>(uv_sorted);
    // the lane pass's leaves compiled in only where there are some: their
    // branch costs the dense evaluations that never take it
    auto run = [&](auto kernel) {
        kernel<<<blocks, kLeafWarps * 32, 0, s>>>(sp, leaf_start, g, nm.sc, nm.kzeta, nm.inv_s, le,
                                                  l2l, uvs, uv, lane_nt);
    };
    if (uv_sorted)
        lane_nt ? run(l2p_f32_kernel<true, true>) : run(l2p_f32_kernel<true, false>);
    else
        lane_nt ? run(l2p_f32_kernel<false, true>) : run(l2p_f32_kernel<false, false>);
    return cudaGetLastError();
}

size_t batch_near_bytes(int count) { return sizeof(NearInst) * (size_t)count; }

cudaError_t batch_near_fill(const BatchInst* host_inst, int count, void* dev_near,
                            cudaStream_t s) {
    NearInst* h = new NearInst[count];
    bool ok = true;
    for (int i = 0; i < count; ++i) {
        bool oki;
        NearF32v3 nm = near_constants(host_inst[i].sigma, host_inst[i].g, &oki);
        ok = ok && oki;
        const uint32_t lane_nt =
            near_lane_path(host_inst[i].n, host_inst[i].g.L) ? kLaneMaxT : 0u;
        h[i] = NearInst{nm.sc, nm.kvel,    nm.kzeta,  nm.inv_s,     nm.half_leaf,
                        nm.qa, nm.band_a2, nm.wstrip, nm.ring_mask, lane_nt};
    }
    cudaError_t e = ok ? cudaMemcpyAsync(dev_near, h, sizeof(NearInst) * count,
                                         cudaMemcpyHostToDevice, s)
                       : cudaErrorInvalidValue;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    delete[] h;
    return e;
}

cudaError_t launch_batch_p2p(const BatchInst* inst, const void* near_inst,
                             const int32_t* leaf_inst, uint32_t ntotal, uint32_t* counter,
                             int ctas_per_sm, const void* particles, const uint32_t* skeys,
                             const uint32_t* leaf_start, const float* le, const float* l2l16,
                             const float* l2l32, float* uv, bool cut, RingStrips strips,
                             uint32_t nleaf_total, const uint32_t* lane_win,
                             uint32_t lane_win_count, cudaStream_t s) {
    if (ntotal == 0) return cudaSuccess;
    Geometry g1{};
    g1.W = 2.0;
    g1.L = 0;
    bool ok;
    NearF32v3 shared_nm = near_constants(1.0, g1, &ok);  // sigma-independent parts
    if (!ok) return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    unsigned blocks = (unsigned)(sms * ctas_per_sm);
    const float4* sp = reinterpret_cast<const float4*>(particles);
    const NearInst* ni = static_cast<const NearInst*>(near_inst);
    cudaError_t e;
    // the per-target-lane pass over the windows of the sparse instances
    const bool lanes = lane_win && lane_win_count > 0;
    if (lanes) {
        const LaneWindows lw{lane_win, lane_win_count, ntotal};
        auto run = [&](auto kernel) {
            const unsigned lb = (unsigned)std::min<uint64_t>(
                resident_ctas(reinterpret_cast<const void*>(kernel)),
                (lw.count + kLeafWarps - 1) / kLeafWarps);
            kernel<<<dim3(lb), dim3(kLeafWarps * 32), 0, s>>>(sp, skeys, leaf_start, lw,
                                                              Geometry{}, shared_nm, inst, ni,
                                                              leaf_inst, le, l2l16, l2l32, uv);
            return cudaGetLastError();
        };
        e = cut ? run(p2p_lane_kernel<true, true, false>) : run(p2p_lane_kernel<true, false, false>);
        if (e != cudaSuccess) return e;
    }
    e = cudaMemsetAsync(counter, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    if (!cut || !strips.n) strips.rec = nullptr;
    if (strips.rec) {
        ring_strips_kernel<true><<<(nleaf_total + kLeafWarps - 1) / kLeafWarps, kLeafWarps * 32, 0,
                                   s>>>(reinterpret_cast<const float4*>(particles), leaf_start,
                                        nleaf_total, Geometry{}, shared_nm, inst,
                                        static_cast<const NearInst*>(near_inst), leaf_inst, strips);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const WorkSplit ws = work_split(ntotal, (uint64_t)blocks * kLeafWarps);
    auto dense = [&](auto kernel) {
        kernel<<<blocks, kLeafWarps * 32, 0, s>>>(sp, skeys, leaf_start, inst, ni, leaf_inst, ws,
                                                  counter, shared_nm, le, l2l16, l2l32, uv,
                                                  strips);
        return cudaGetLastError();
    };
    if (cut)
        return lanes ? dense(p2p_batch_kernel<true, true>) : dense(p2p_batch_kernel<true, false>);
    return lanes ? dense(p2p_batch_kernel<false, true>) : dense(p2p_batch_kernel<false, false>);
}

template <>
cudaError_t launch_p2p_l2p<double>(const Geometry& g, double sigma, int64_t n,
                                   const void* particles, const uint32_t* skeys,
                                   const uint32_t* leaf_start, uint32_t* counter,
                                   const double* le, const double* l2l, double* uv,
                                   cudaStream_t s) {
    (void)n;
    (void)skeys;
    (void)counter;  // one CTA per leaf
    NearF64 nm;
    nm.inv2s2 = 1.0 / (2.0 * sigma * sigma);
    nm.k0 = 1.0 / (2.0 * 3.14159265358979323846);
    nm.a2 = g.L >= 2 ? g.cutoff * g.cutoff : 0.0;
    nm.ring_mask = ring_mask(g);
    unsigned nleaf = 1u << (2 * g.L);
    p2p_l2p_kernel<double, NearF64><<<nleaf, kThreads, 0, s>>>(
        reinterpret_cast<const ParticleD*>(particles), leaf_start, g, ldexp(1.0, g.L) / g.W, nm,
        le, l2l, uv);
    return cudaGetLastError();
}

}  // namespace fmm2d
