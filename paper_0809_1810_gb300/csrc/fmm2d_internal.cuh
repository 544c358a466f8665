// Internal declarations shared by the CUDA translation units of the library.
// Not part of the ABI: everything callers see is in include/fmm2d.h.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fmm2d.h"

namespace fmm2d {

constexpr int kMaxP = 32;      // largest expansion order served
constexpr int kMaxL = 12;      // deepest quadtree level served
constexpr int kRadixBits = 8;  // radix sort digit width
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;
// keys per thread per tile: 2048-key tiles sort 2^24 keys 10-15% faster than
// 4096-key ones (more CTAs in flight) and 2^20 keys as fast
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;

// Device-side status flags (bitwise OR of 1 << fmm2d_status).
constexpr int kFlagOutOfDomain = 1 << FMM2D_OUT_OF_DOMAIN;
constexpr int kFlagNonfinite = 1 << FMM2D_NONFINITE;
constexpr int kFlagInvalid = 1 << FMM2D_INVALID_ARG;
constexpr int kFlagTimeout = 1 << FMM2D_TIMEOUT;

// Offset tables index the 7 x 7 source-minus-target box offsets (dx, dy) in
// [-3, 3]^2; the 40 with max(|dx|, |dy|) >= 2 are M2L offsets.
constexpr int kOffsetSlots = 49;
__host__ __device__ inline int offset_slot(int dx, int dy) { return (dy + 3) * 7 + (dx + 3); }

// Sorted particle record: position, circulation and input index.
struct __align__(32) ParticleD {
    double x, y, z, w;  // position, circulation, input index (an integer below 2^53)
};
template <typename R>
struct ParticleOf;
template <>
struct ParticleOf<float> {
    using type = float4;  // (x, y, Gamma, input index as uint bits)
    __device__ static inline type make(float x, float y, float g, uint32_t i) {
        return make_float4(x, y, g, __uint_as_float(i));
    }
    __device__ static inline uint32_t index(const type& q) { return __float_as_uint(q.w); }
};
template <>
struct ParticleOf<double> {
    using type = ParticleD;
    __device__ static inline type make(double x, double y, double g, uint32_t i) {
        return ParticleD{x, y, g, (double)i};
    }
    __device__ static inline uint32_t index(const type& q) { return (uint32_t)q.w; }
};

// Geometry shared by the kernels of one evaluation.
struct Geometry {
    double x0, y0, W;  // root box
    int L;             // leaf level
    int p;             // expansion terms
    int P;             // padded terms per box in expansion arrays (16 or 32)
    int64_t level_base[kMaxL + 2];  // first box slot of level l (l >= 2)
    int64_t nboxes;    // box slots over levels 2..L
    double scale;      // 2^L / W, inverse leaf width (formed on the host)
    double cutoff;     // a of Sec. 4.1 (0: none): pairs closer than a keep K_sigma
    // leaf centres per axis index as FP32 hi/lo pairs, (x hi, x lo, y hi, y lo)
    // at index i, built once per plan (null: computed where needed)
    const float4* centre_tab;
};

// The 16 leaves at Chebyshev distance 2 (the ring around the 3x3 block that a
// cutoff of at most two leaf widths can reach): offset of ring leaf r.
__host__ __device__ inline void ring_offset(int r, int* dx, int* dy) {
    if (r < 5) *dx = r - 2, *dy = -2;
    else if (r < 10) *dx = r - 7, *dy = 2;
    else if (r < 13) *dx = -2, *dy = r - 11;
    else *dx = 2, *dy = r - 14;
}

// Expansion-array slot of box (ix, iy) at level l >= 2.  Each level is
// stored as four parity planes (ix & 1, iy & 1), each a row-major grid of
// (2^(l-1))^2 boxes, so that a fixed box offset maps a run of same-parity
// target boxes onto a run of source boxes.
__host__ __device__ inline int64_t box_slot(const int64_t* level_base, int l, uint32_t ix,
                                            uint32_t iy) {
    uint32_t h = 1u << (l - 1);
    uint32_t plane = ((iy & 1u) << 1) | (ix & 1u);
    return level_base[l] + ((int64_t)(plane * h + (iy >> 1)) * h + (ix >> 1));
}

__host__ __device__ inline uint32_t morton_spread(uint32_t v) {
    v &= 0xFFFFu;
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

__host__ __device__ inline uint32_t morton_compact(uint32_t v) {
    v &= 0x55555555u;
    v = (v | (v >> 1)) & 0x33333333u;
    v = (v | (v >> 2)) & 0x0F0F0F0Fu;
    v = (v | (v >> 4)) & 0x00FF00FFu;
    v = (v | (v >> 8)) & 0x0000FFFFu;
    return v;
}

__host__ __device__ inline uint32_t morton_key(uint32_t ix, uint32_t iy) {
    return morton_spread(ix) | (morton_spread(iy) << 1);
}

// Translation tables in the precision of the evaluation, complex entries as
// (re, im) pairs, each matrix stored [k][n] (input index major) so that the
// lanes of a warp, one per output coefficient n, read consecutive entries.
template <typename R>
struct Tables {
    const R* m2m;  // [4 quadrants][P][P] complex: child quadrant (cy*2+cx)
    const R* l2l;  // [4 quadrants][P][P] complex
    const R* m2l;  // [49 offset slots][P][P] complex
};

// Host launchers (one translation unit each).
cudaError_t launch_build_tables(int p, int P, double* m2m, double* l2l, double* m2l,
                                double* binom_scratch, cudaStream_t s);
cudaError_t launch_tables_to_f32(const double* src, float* dst, int64_t count, cudaStream_t s);
// Leaf-centre table of a plan: entry i = (x hi, x lo, y hi, y lo) of the
// centre coordinates x0 + (i + 1/2) s and y0 + (i + 1/2) s, i < 2^L.
cudaError_t launch_centre_table(const Geometry& g, float4* tab, cudaStream_t s);

// Sorted keys after an LSD sort of key_bits-bit keys (kRadixBits per pass):
// the buffer the last pass wrote.
inline int sort_passes(int key_bits) {
    return key_bits <= kRadixBits ? 1 : (key_bits + kRadixBits - 1) / kRadixBits;
}

struct SortBuffers {
    uint32_t* keys[2];
    uint32_t* vals[2];
    uint32_t* hist;      // kRadix * nblocks
    uint32_t* leaf_start;
    uint32_t* perm;      // sorted input index
    int* status;
};

template <typename R>
cudaError_t launch_tree_build(const Geometry& g, int64_t n, const R* xy, const R* gamma,
                              SortBuffers& sb, void* particles, cudaStream_t s);

template <typename R>
cudaError_t launch_p2m(const Geometry& g, const void* particles, const uint32_t* leaf_start,
                       const Tables<R>& t, R* me, cudaStream_t s);
template <typename R>
cudaError_t launch_m2m(const Geometry& g, const Tables<R>& t, R* me, cudaStream_t s);
template <typename R>
cudaError_t launch_m2l(const Geometry& g, const Tables<R>& t, const R* me, R* le, cudaStream_t s);
template <typename R>
cudaError_t launch_l2l(const Geometry& g, const Tables<R>& t, R* le, cudaStream_t s);
template <typename R>
cudaError_t launch_p2p_l2p(const Geometry& g, double sigma, int64_t n, const void* particles,
                           const uint32_t* skeys, const uint32_t* leaf_start, uint32_t* counter,
                           const R* le, const R* l2l, R* uv, cudaStream_t s);
// The FP32 near field without its far part, written to `out` (2 floats per
// target) at the input indices or (sorted_out) in sorted order, and the L2P
// that adds the far part afterwards -- reading the near parts in sorted order
// from uv_sorted, or from uv itself when uv_sorted is null -- and writes the
// velocities to uv at the input indices (the fused kernel's sum, bit for bit).
// Ring strips of the cutoff (Sec. 4.1) for the FP32 near field: per leaf
// and side (0 left, 1 right, 2 bottom, 3 top), the leaf's records within
// reach of the leaf two leaves away on that side, in sorted order, at
// rec[4 t0 + side n_leaf ...] (t0 the leaf's first sorted position), their
// counts at n[4 leaf + side].  rec holds 4 records per particle, n 4 counts
// per leaf.  Null rec: the ring is gathered from whole leaves (the same
// sources, in the same order).
struct RingStrips {
    float4* rec;
    uint32_t* n;
};

cudaError_t launch_near_only_f32(const Geometry& g, double sigma, int64_t n,
                                 const void* particles, const uint32_t* skeys,
                                 const uint32_t* leaf_start, uint32_t* counter, float* out,
                                 bool sorted_out, RingStrips strips, cudaStream_t s);
cudaError_t launch_l2p_f32(const Geometry& g, double sigma, int64_t n, const void* particles,
                           const uint32_t* leaf_start, const float* le, const float* l2l,
                           const float* uv_sorted, float* uv, cudaStream_t s);

// ---------------------------------------------------------------------------
// Batched evaluation: many instances in one packed problem.  Instance i owns
// particles [offset, offset + n) of the packed arrays, leaves
// [leaf_base, leaf_base + 4^L) of one global leaf index space (its keys are
// leaf_base + Morton key, so one stable sort groups every instance), and the
// expansion block starting at element exp_off of the ME and LE arrays.
// ---------------------------------------------------------------------------
struct BatchInst {
    Geometry g;          // the instance's geometry; level_base relative to exp_off
    int64_t offset;      // first particle in the packed arrays
    int64_t n;           // particle count
    int64_t exp_off;     // first element of its expansion block
    uint32_t leaf_base;  // global index of its leaf 0
    double sigma;        // core size
};

// Per-class work lists built on the host (class = expansion stride P, 16 or
// 32): the instances that take part in a step, and flattened index spaces.
struct BatchLists {
    const int32_t* quad_inst;    // P2M: instance of every parent box (level L-1) of the class
    const uint32_t* quad_local;  // its local index (Morton key at level L-1)
    int64_t nquads;
    int64_t nquads_warp;         // the first ones: instances of at most 32 particles
                                 // per leaf on average (one warp per box)
    const int32_t* m2l_inst;     // M2L: instances of the class ...
    const int64_t* m2l_prefix;   // ... and the prefix of their box counts (levels 2..L)
    int m2l_count;
    int64_t m2l_total;
    const int32_t* m2m_inst[kMaxL + 1];  // M2M at level l: instances with 2 <= l <= L - 2
    int m2m_count[kMaxL + 1];
    const int32_t* l2l_inst[kMaxL + 1];  // L2L at level l: instances with 3 <= l <= L - 1
    int l2l_count[kMaxL + 1];
};

cudaError_t batch_key_params(const BatchInst* host_inst, int count, void* dev_params,
                             cudaStream_t s);
size_t batch_key_params_bytes(int count);
cudaError_t launch_batch_tree(const void* dev_key_params, const int64_t* dev_offsets, int count,
                              int64_t ntotal, int key_bits, uint32_t nleaf_total, const float* xy,
                              const float* gamma, SortBuffers& sb, void* particles,
                              cudaStream_t s);
cudaError_t launch_batch_p2m(const BatchInst* inst, const BatchLists& bl, int P,
                             const void* particles, const uint32_t* leaf_start, const float* m2m,
                             float* me, cudaStream_t s);
cudaError_t launch_batch_m2m(const BatchInst* inst, const BatchLists& bl, int P, int level,
                             const float* m2m, float* me, cudaStream_t s);
cudaError_t launch_batch_m2l(const BatchInst* inst, const BatchLists& bl, int P, int threads,
                             const float* m2l, const float* me, float* le, cudaStream_t s);
cudaError_t launch_batch_l2l(const BatchInst* inst, const BatchLists& bl, int P, int level,
                             const float* l2l, float* le, cudaStream_t s);
size_t batch_near_bytes(int count);
cudaError_t batch_near_fill(const BatchInst* host_inst, int count, void* dev_near,
                            cudaStream_t s);
cudaError_t launch_batch_p2p(const BatchInst* inst, const void* near_inst,
                             const int32_t* leaf_inst, uint32_t ntotal, uint32_t* counter,
                             int ctas_per_sm, const void* particles, const uint32_t* skeys,
                             const uint32_t* leaf_start, const float* le, const float* l2l16,
                             const float* l2l32, float* uv, bool cut, RingStrips strips,
                             uint32_t nleaf_total, const uint32_t* lane_win,
                             uint32_t lane_win_count, cudaStream_t s);
// Whether an evaluation of n particles over 4^L leaves sends its sparse
// leaves to the per-target-lane pass of the FP32 near field.  A batch lists
// the windows of 32 sorted positions that hold such instances' particles
// (lane_win, lane_win_count; null: none).
bool near_lane_path(int64_t n, int L);
cudaError_t launch_batch_direct(const BatchInst* inst, const int64_t* dev_offsets, int count,
                                int kernel, const float* xy, const float* gamma, int64_t s_count,
                                const int64_t* targets, double* uv_ref, int* status,
                                cudaStream_t s);
cudaError_t launch_batch_error(const BatchInst* inst, const int64_t* dev_offsets, int count,
                               const float* xy, const float* uv, int64_t s_count,
                               const int64_t* targets, const double* uv_ref, double* stats,
                               double* leaf_err, uint32_t nleaf_total, int* status,
                               cudaStream_t s);

// Tensor-core M2L (m2l_tc.cu).  The 27 interaction-list boxes of each of the
// four children of a target parent are the children of the parent's 8
// neighbours, so per neighbour offset D the operator is one dense block
// matrix [4 target children x 2Pk] x [4 source children x 2Pk] (zero blocks
// for adjacent children, which the near field takes), Pk = p rounded up to a
// multiple of 4.  Multipole hi/lo parts are kept per level in a layout made
// for TMA boxes of a tile's source halo: [parity plane][k-group of 4 reals]
// [row][column][4 reals]; one 4-D map per level and part.
struct M2LTcMaps {
    CUtensorMap me_hi[kMaxL + 1];
    CUtensorMap me_lo[kMaxL + 1];
};
// Per-plan configuration of the tensor-core M2L.
struct M2LTcConfig {
    int Pk;             // p rounded up to a multiple of 4 (4..32)
    int ntiles;         // CTAs: tiles of target parents over levels 2..L
    int halo_bytes;     // shared memory of one halo slot (hi or lo part)
    int b_stages;       // operator stages in flight
    int smem;           // dynamic shared memory per CTA
    int64_t b_floats;   // size of the operator image
};
// Default bound on the polls of one device wait in the tensor-core M2L: long
// enough never to expire in a correct run, short enough that a hung pipeline
// returns FMM2D_TIMEOUT instead of holding the GPU.
constexpr uint32_t kSpinDefault = 1u << 26;
cudaError_t m2l_tc_configure();
// Host-side plan of the tiles and shared memory (no device work); tiles_host
// (optional) receives two int4 records per tile.
M2LTcConfig m2l_tc_plan(const Geometry& g, int4* tiles_host);
// Tensor maps, tile list upload and the operator image (FP64 tables split
// into TF32 hi/lo, laid out as the kernel's shared-memory stages).
cudaError_t m2l_tc_prepare(const Geometry& g, const M2LTcConfig& cfg, const double* m2l64,
                           float* me_hi, float* me_lo, float* bimg, M2LTcMaps* maps,
                           cudaStream_t s);
// The tensor-core M2L of a batch: one class per Pk (p rounded up to 4) over
// every instance of the batch with that Pk and L >= 2.  Its multipole hi/lo
// parts are stacked per level over the instances deep enough (an instance
// slot dimension in the level's tensor map), so one launch serves them all.
struct M2LTcBatchClass {
    int Pk = 0, P = 0;
    M2LTcConfig cfg{};
    M2LTcMaps* maps = nullptr;
    void* ws = nullptr;          // one device allocation for everything below
    int4* tiles = nullptr;       // two records per tile
    float* hi = nullptr;
    float* lo = nullptr;
    float* bimg = nullptr;
    int32_t* inst = nullptr;     // the class's instances
    int64_t* box_prefix = nullptr;  // prefix of their box counts
    int64_t* dst_base = nullptr;    // per instance and level: float4 offset in hi / lo
    int count = 0;
    int64_t boxes = 0;
};
// ids: the class's instances (L >= 2, Pk = (p + 3) & ~3); m2l64 the FP64
// M2L table of stride P built for p = P.  `tile_policy` 0: the fewest tiles
// per level; 1: the widest rows (the autotuner's alternative).
cudaError_t m2l_tc_batch_create(const BatchInst* host_inst, const int* ids, int nids, int Pk,
                                int P, const double* m2l64, int b_stages, int tile_policy,
                                M2LTcBatchClass* out, cudaStream_t s);
void m2l_tc_batch_destroy(M2LTcBatchClass* c);
cudaError_t launch_m2l_tc_batch(const M2LTcBatchClass& c, const BatchInst* d_inst,
                                const float* me, float* le, int* status, uint32_t spin,
                                cudaStream_t s);
cudaError_t launch_m2l_tc(const Geometry& g, const M2LTcConfig& cfg, const M2LTcMaps& maps,
                          const int4* tiles, const float* me, float* me_hi, float* me_lo,
                          const float* bimg, float* le, int* status, uint32_t spin,
                          cudaStream_t s);

template <typename R>
cudaError_t launch_direct_sampled(const Geometry& g, double sigma, int kernel, int64_t n,
                                  const R* xy, const R* gamma, int64_t s_count,
                                  const int64_t* targets, double* uv_ref, int* status,
                                  cudaStream_t s);
template <typename R>
cudaError_t launch_error_stats(const Geometry& g, int64_t n, const R* xy, const R* uv,
                               int64_t s_count, const int64_t* targets, const double* uv_ref,
                               double* stats, double* leaf_err, int* status, cudaStream_t s);

}  // namespace fmm2d

namespace fmm2d {

// Complex arithmetic on (re, im) pairs of the evaluation's precision.
template <typename R>
struct Cplx;
template <>
struct Cplx<float> {
    using T = float2;
};
template <>
struct Cplx<double> {
    using T = double2;
};
template <typename T>
__host__ __device__ inline T cmake(decltype(T().x) re, decltype(T().x) im) {
    T r;
    r.x = re;
    r.y = im;
    return r;
}
// Products the compiler may not fuse into a neighbouring addition: with the
// fused steps spelled out, every kernel that inlines a routine rounds it the
// same way (batched and single evaluations agree bit for bit).
__device__ inline float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ inline double mul_rn(double a, double b) { return __dmul_rn(a, b); }
template <typename T>
__device__ inline T cmul(T a, T b) {
    return cmake<T>(fma(a.x, b.x, -mul_rn(a.y, b.y)), fma(a.x, b.y, mul_rn(a.y, b.x)));
}
// acc + a * b
template <typename T>
__device__ inline T cfma(T a, T b, T acc) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
    return acc;
}
template <typename T>
__device__ inline T cshfl(T v, int src, int width, unsigned mask = 0xffffffffu) {
    v.x = __shfl_sync(mask, v.x, src, width);
    v.y = __shfl_sync(mask, v.y, src, width);
    return v;
}
// Lanes of the G-lane segment (G = 16 or 32) that holds the calling lane.
__device__ inline unsigned segment_mask(int G) {
    int lane = threadIdx.x & 31;
    return G == 32 ? 0xffffffffu : (0xffffu << (lane & 16));
}

// Leaf-centre coordinate x0 + (i + 1/2) s, s = W 2^-L, formed in FP64 with
// every rounding explicit (no contraction, so the per-plan table and the
// direct computation agree bit for bit), split into an FP32 hi/lo pair.
__device__ inline void centre_hilo_1d(double x0, double W, int L, uint32_t i, float* hi,
                                      float* lo) {
    const double s = W * ldexp(1.0, -L);
    const double c = __dadd_rn(x0, __dmul_rn((double)i + 0.5, s));
    *hi = (float)c;
    *lo = (float)__dsub_rn(c, (double)*hi);
}

// Centre of leaf (ix, iy) as FP32 hi/lo pairs: from the plan's table when it
// has one, else computed in FP64 by lane 0 of the warp and broadcast (FP64 is
// slow on this part).  Every lane of the warp must call it.
__device__ inline void leaf_centre_hilo(const Geometry& g, uint32_t ix, uint32_t iy, float* cxh,
                                        float* cxl, float* cyh, float* cyl) {
    if (g.centre_tab) {
        const float4 a = g.centre_tab[ix], b = g.centre_tab[iy];
        *cxh = a.x;
        *cxl = a.y;
        *cyh = b.z;
        *cyl = b.w;
        return;
    }
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if ((threadIdx.x & 31) == 0) {
        centre_hilo_1d(g.x0, g.W, g.L, ix, &v[0], &v[1]);
        centre_hilo_1d(g.y0, g.W, g.L, iy, &v[2], &v[3]);
    }
    *cxh = __shfl_sync(0xffffffffu, v[0], 0);
    *cxl = __shfl_sync(0xffffffffu, v[1], 0);
    *cyh = __shfl_sync(0xffffffffu, v[2], 0);
    *cyl = __shfl_sync(0xffffffffu, v[3], 0);
}

// Decode the box of level l held by expansion slot `slot` (inverse of box_slot).
__device__ inline int slot_level(const int64_t* level_base, int L, int64_t slot) {
    int l = 2;
    while (l < L && slot >= level_base[l + 1]) ++l;
    return l;
}
__device__ inline void slot_box(const int64_t* level_base, int l, int64_t slot, uint32_t* ix,
                                uint32_t* iy) {
    int64_t r = slot - level_base[l];
    uint32_t h = 1u << (l - 1);
    uint32_t plane = (uint32_t)(r / ((int64_t)h * h));
    uint32_t rem = (uint32_t)(r % ((int64_t)h * h));
    *ix = ((rem % h) << 1) | (plane & 1u);
    *iy = ((rem / h) << 1) | (plane >> 1);
}

}  // namespace fmm2d
