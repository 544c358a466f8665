// Quadtree build (Sec. 3.3, Fig. 6): Morton keys of the leaves at level L,
// a stable LSD radix sort of (key, input index), the gather of the sorted
// particle records, and the leaf ranges.
//
// Leaf coordinate along an axis: floor((x - x0) * (2^L / W)) in FP64,
// clamped into [0, 2^L - 1]; the upper edge of the root box belongs to the
// last leaf.  Key = leaf x index in the even bits, y index in the odd bits.
// The sort is stable, so particles of one leaf keep their input order and
// the permutation is unique.
//
// Radix pass (8-bit digit): per-tile digit counts -> exclusive scan over
// (digit, tile) -> scatter.  Within a tile each warp owns a contiguous run of
// keys and ranks equal digits with __match_any_sync, which preserves input
// order; warps are then offset per digit in warp order.
#include <mutex>

#include "fmm2d_internal.cuh"

namespace fmm2d {
namespace {

struct KeyParams {
    double x0, y0, x1, y1;  // closed root box
    double scale;           // 2^L / W
    double top;             // 2^L - 1
    // FP32 fast path for float inputs: the FP32 estimate of (x - x0) 2^L / W
    // is trusted when it lies farther than `margin` cells from every cell
    // edge; otherwise the FP64 expression decides.  Domain bounds are the
    // float values that bracket the closed root box exactly.
    bool fast;
    float x0f, y0f, scalef, margin;
    float lox, hix, loy, hiy;
};

__device__ inline uint32_t leaf_coord(double x, double lo, double hi, double scale, double top,
                                      int* flags) {
    if (!(x >= lo && x <= hi)) *flags |= (x != x) ? kFlagNonfinite : kFlagOutOfDomain;
    double f = floor((x - lo) * scale);
    if (!(f >= 0.0)) f = 0.0;  // also maps NaN to 0 so that no index runs wild
    if (f > top) f = top;
    return (uint32_t)f;
}

// The defining FP64 expression, for coordinates near a cell edge.  Not
// inlined: as a short inline branch it was evaluated for every coordinate
// (the FP64 pipe, about 1/64 of the FP32 rate here, then limited the kernel).
__device__ __noinline__ uint32_t leaf_coord_fp64(float x, double lo_d, double scale, double top) {
    double fd = floor(((double)x - lo_d) * scale);
    if (!(fd >= 0.0)) fd = 0.0;
    if (fd > top) fd = top;
    return (uint32_t)fd;
}

__device__ inline uint32_t leaf_coord_f32(float x, float lo, float hi, float x0f, float scalef,
                                          float margin, double lo_d, double scale, double top,
                                          int* flags) {
    if (!(x >= lo && x <= hi)) *flags |= (x != x) ? kFlagNonfinite : kFlagOutOfDomain;
    float f = (x - x0f) * scalef;
    float fl = floorf(f);
    float fr = f - fl;
    if (fr > margin && fr < 1.0f - margin && fl >= 0.0f && fl <= (float)top)
        return (uint32_t)fl;
    return leaf_coord_fp64(x, lo_d, scale, top);
}

// Keys of one tile plus the histogram of the first digit.
template <typename R>
__global__ void __launch_bounds__(kSortThreads)
keys_hist_kernel(int64_t n, const R* __restrict__ xy, const R* __restrict__ gamma, KeyParams kp,
                 uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                 uint32_t* __restrict__ hist, int nblocks, int* status) {
    __shared__ uint32_t cnt[kRadix];
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) cnt[d] = 0;
    __syncthreads();
    int flags = 0;
    int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
    for (int it = 0; it < kSortItems; ++it) {
        int64_t i = base + it * kSortThreads + threadIdx.x;
        if (i < n) {
            uint32_t ix, iy;
            if (sizeof(R) == 4 && kp.fast) {
                float x = (float)xy[2 * i], y = (float)xy[2 * i + 1];
                if (!isfinite((float)gamma[i])) flags |= kFlagNonfinite;
                ix = leaf_coord_f32(x, kp.lox, kp.hix, kp.x0f, kp.scalef, kp.margin, kp.x0,
                                    kp.scale, kp.top, &flags);
                iy = leaf_coord_f32(y, kp.loy, kp.hiy, kp.y0f, kp.scalef, kp.margin, kp.y0,
                                    kp.scale, kp.top, &flags);
            } else {
                double x = (double)xy[2 * i], y = (double)xy[2 * i + 1];
                if (!isfinite((double)gamma[i])) flags |= kFlagNonfinite;
                ix = leaf_coord(x, kp.x0, kp.x1, kp.scale, kp.top, &flags);
                iy = leaf_coord(y, kp.y0, kp.y1, kp.scale, kp.top, &flags);
            }
            uint32_t k = morton_key(ix, iy);
            keys[i] = k;
            vals[i] = (uint32_t)i;
            atomicAdd(&cnt[k & (kRadix - 1)], 1u);
        }
    }
    if (flags) atomicOr(status, flags);
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x)
        hist[(int64_t)d * nblocks + blockIdx.x] = cnt[d];
}

__global__ void __launch_bounds__(kSortThreads)
hist_kernel(int64_t n, const uint32_t* __restrict__ keys, int shift, uint32_t* __restrict__ hist,
            int nblocks) {
    __shared__ uint32_t cnt[kRadix];
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) cnt[d] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
    for (int it = 0; it < kSortItems; ++it) {
        int64_t i = base + it * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x)
        hist[(int64_t)d * nblocks + blockIdx.x] = cnt[d];
}

// Exclusive scan of each digit's per-tile counts in place (one CTA per
// digit, counts stored digit-major), and the digit's total count.
__global__ void __launch_bounds__(256)
scan_digits_kernel(uint32_t* __restrict__ hist, int nblocks, uint32_t* __restrict__ digit_total) {
    __shared__ uint32_t warp_sums[8];
    uint32_t* row = hist + (int64_t)blockIdx.x * nblocks;
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t carry = 0;
    for (int base = 0; base < nblocks; base += 256) {
        int i = base + threadIdx.x;
        uint32_t v = i < nblocks ? row[i] : 0u;
        uint32_t incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        uint32_t before = 0, tile = 0;
        for (int w = 0; w < 8; ++w) {
            uint32_t ws = warp_sums[w];
            if (w < warp) before += ws;
            tile += ws;
        }
        if (i < nblocks) row[i] = carry + before + incl - v;
        carry += tile;
        __syncthreads();
    }
    if (threadIdx.x == 0) digit_total[blockIdx.x] = carry;
}

// Block-wide exclusive scan of one value per thread (kSortThreads threads);
// returns the exclusive prefix, writes the block total to *total.
__device__ inline uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_tmp, uint32_t* total) {
    constexpr int kWarps = kSortThreads / 32;
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tmp[warp] = incl;
    __syncthreads();
    uint32_t before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        uint32_t ws = warp_tmp[w];
        before += w < warp ? ws : 0u;
        all += ws;
    }
    *total = all;
    __syncthreads();  // warp_tmp may be reused
    return before + incl - v;
}

// Stable scatter of one tile.  Keys are first ranked within the tile (each
// warp owns a contiguous run and ranks equal digits with __match_any_sync,
// which keeps input order), staged in shared memory in tile-sorted order,
// then written out as contiguous per-digit runs (coalesced).  With kLast the
// pass is the final one and also writes the permutation and the sorted
// particle records.
template <typename R, bool kLast>
__global__ void __launch_bounds__(kSortThreads)
scatter_kernel(int64_t n, const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
               int shift, const uint32_t* __restrict__ offsets,
               const uint32_t* __restrict__ digit_total, int nblocks,
               uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
               const R* __restrict__ xy, const R* __restrict__ gamma,
               typename ParticleOf<R>::type* __restrict__ particles) {
    constexpr int kWarps = kSortThreads / 32;
    constexpr int kPerWarp = kSortTile / kWarps;  // contiguous keys per warp
    constexpr int kIters = kPerWarp / 32;
    __shared__ uint32_t wcnt[kWarps][kRadix];
    __shared__ uint32_t gbase[kRadix];  // where the tile's digit-d run starts overall
    __shared__ uint32_t tbase[kRadix];  // where it starts within the tile
    __shared__ uint32_t tmp[kWarps];
    __shared__ uint32_t skey[kSortTile], sval[kSortTile];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = lane; d < kRadix; d += 32) wcnt[warp][d] = 0;
    __syncwarp();
    const int64_t tile0 = (int64_t)blockIdx.x * kSortTile;
    const int64_t base = tile0 + (int64_t)warp * kPerWarp;
    uint32_t key[kIters], val[kIters], rank[kIters];
    const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int it = 0; it < kIters; ++it) {
        int64_t i = base + it * 32 + lane;
        bool ok = i < n;
        key[it] = ok ? keys_in[i] : 0u;
        val[it] = ok ? vals_in[i] : 0u;
        uint32_t d = ok ? ((key[it] >> shift) & (kRadix - 1)) : (uint32_t)kRadix;  // sentinel
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = ok ? wcnt[warp][d] : 0u;
        __syncwarp();
        if (ok && (peers & lt_mask) == 0) wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
        rank[it] = before + __popc(peers & lt_mask);
    }
    __syncthreads();
    static_assert(kRadix == kSortThreads, "one thread per digit");
    {
        const int d = threadIdx.x;
        uint32_t cnt = 0;  // the tile's count of digit d; warps offset in warp order
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            uint32_t c = wcnt[w][d];
            wcnt[w][d] = cnt;
            cnt += c;
        }
        uint32_t all;
        uint32_t dstart = block_exclusive_scan(digit_total[d], tmp, &all);
        tbase[d] = block_exclusive_scan(cnt, tmp, &all);
        gbase[d] = dstart + offsets[(int64_t)d * nblocks + blockIdx.x];
    }
    __syncthreads();
    // stage in tile-sorted order
#pragma unroll
    for (int it = 0; it < kIters; ++it) {
        int64_t i = base + it * 32 + lane;
        if (i < n) {
            uint32_t d = (key[it] >> shift) & (kRadix - 1);
            uint32_t lp = tbase[d] + wcnt[warp][d] + rank[it];
            skey[lp] = key[it];
            sval[lp] = val[it];
        }
    }
    __syncthreads();
    const int tile_n = (int)min((int64_t)kSortTile, n - tile0);
    for (int lp = threadIdx.x; lp < tile_n; lp += kSortThreads) {
        uint32_t k = skey[lp], v = sval[lp];
        uint32_t d = (k >> shift) & (kRadix - 1);
        uint32_t pos = gbase[d] + (uint32_t)lp - tbase[d];
        keys_out[pos] = k;
        vals_out[pos] = v;
        if (kLast)
            particles[pos] = ParticleOf<R>::make(xy[2 * (int64_t)v], xy[2 * (int64_t)v + 1],
                                                 gamma[v], v);
    }
}

// leaf_start[k] = first sorted position whose key is >= k, k = 0 .. 4^L.
__global__ void leaf_bounds_kernel(int64_t n, const uint32_t* __restrict__ skeys, uint32_t nleaf,
                                   uint32_t* __restrict__ leaf_start) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= n;
         r += (int64_t)gridDim.x * blockDim.x) {
        int64_t prev = r == 0 ? -1 : (int64_t)skeys[r - 1];
        int64_t cur = r == n ? (int64_t)nleaf : (int64_t)skeys[r];
        for (int64_t k = prev + 1; k <= cur; ++k) leaf_start[k] = (uint32_t)r;
    }
}

// Key parameters for root box (x0, y0, W) at level L.  The FP32 fast path
// is enabled for float inputs when its error bound stays well below a cell.
KeyParams make_key_params(double x0, double y0, double W, int L) {
    KeyParams kp;
    kp.x0 = x0;
    kp.y0 = y0;
    kp.x1 = x0 + W;
    kp.y1 = y0 + W;
    kp.scale = ldexp(1.0, L) / W;
    kp.top = ldexp(1.0, L) - 1.0;
    kp.x0f = (float)x0;
    kp.y0f = (float)y0;
    kp.scalef = (float)kp.scale;
    // |error of the FP32 estimate| <= 2^-24 (4 * 2^L + max|x0,y0| * 2^L / W) cells
    double err = ldexp(4.0 * ldexp(1.0, L) + fmax(fabs(x0), fabs(y0)) * kp.scale, -24);
    kp.margin = (float)(2.0 * err);
    kp.fast = 2.0 * err < 0.05;
    auto up = [](double v) {  // smallest float >= v
        float f = (float)v;
        return (double)f < v ? nextafterf(f, INFINITY) : f;
    };
    auto down = [](double v) {  // largest float <= v
        float f = (float)v;
        return (double)f > v ? nextafterf(f, -INFINITY) : f;
    };
    kp.lox = up(kp.x0);
    kp.hix = down(kp.x1);
    kp.loy = up(kp.y0);
    kp.hiy = down(kp.y1);
    return kp;
}

}  // namespace

template <typename R>
cudaError_t launch_tree_build(const Geometry& g, int64_t n, const R* xy, const R* gamma,
                              SortBuffers& sb, void* particles, cudaStream_t s) {
    using P = typename ParticleOf<R>::type;
    uint32_t nleaf = 1u << (2 * g.L);
    if (n == 0) {
        leaf_bounds_kernel<<<1, 32, 0, s>>>(0, sb.keys[0], nleaf, sb.leaf_start);
        return cudaGetLastError();
    }
    KeyParams kp = make_key_params(g.x0, g.y0, g.W, g.L);
    int nblocks = (int)((n + kSortTile - 1) / kSortTile);
    int bits = 2 * g.L;
    int passes = sort_passes(bits);
    uint32_t* digit_total = sb.hist + (int64_t)kRadix * nblocks;
    keys_hist_kernel<R><<<nblocks, kSortThreads, 0, s>>>(n, xy, gamma, kp, sb.keys[0], sb.vals[0],
                                                         sb.hist, nblocks, sb.status);
    for (int q = 0; q < passes; ++q) {
        int src = q & 1, dst = src ^ 1;
        int shift = q * kRadixBits;
        if (q > 0)
            hist_kernel<<<nblocks, kSortThreads, 0, s>>>(n, sb.keys[src], shift, sb.hist, nblocks);
        scan_digits_kernel<<<kRadix, 256, 0, s>>>(sb.hist, nblocks, digit_total);
        if (q == passes - 1)
            scatter_kernel<R, true><<<nblocks, kSortThreads, 0, s>>>(
                n, sb.keys[src], sb.vals[src], shift, sb.hist, digit_total, nblocks, sb.keys[dst],
                sb.perm, xy, gamma, reinterpret_cast<P*>(particles));
        else
            scatter_kernel<R, false><<<nblocks, kSortThreads, 0, s>>>(
                n, sb.keys[src], sb.vals[src], shift, sb.hist, digit_total, nblocks, sb.keys[dst],
                sb.vals[dst], xy, gamma, reinterpret_cast<P*>(particles));
    }
    const uint32_t* sorted = sb.keys[passes & 1];
    int lb_blocks = (int)((n + 1 + 255) / 256);
    if (lb_blocks > 2048) lb_blocks = 2048;
    leaf_bounds_kernel<<<lb_blocks, 256, 0, s>>>(n, sorted, nleaf, sb.leaf_start);
    return cudaGetLastError();
}

template cudaError_t launch_tree_build<float>(const Geometry&, int64_t, const float*, const float*,
                                              SortBuffers&, void*, cudaStream_t);
template cudaError_t launch_tree_build<double>(const Geometry&, int64_t, const double*,
                                               const double*, SortBuffers&, void*, cudaStream_t);


// ---------------------------------------------------------------------------
// Batched tree build: keys of all instances in one global leaf index space
// (instance i's keys are leaf_base_i + its Morton keys), then the same stable
// radix sort, record gather and leaf ranges as a single evaluation.
// ---------------------------------------------------------------------------
namespace {

struct BatchKeyParams {
    KeyParams kp;
    uint32_t leaf_base;
    int L;
};

__global__ void __launch_bounds__(kSortThreads)
batch_keys_hist_kernel(int64_t n, const float* __restrict__ xy, const float* __restrict__ gamma,
                       const BatchKeyParams* __restrict__ bkp, const int64_t* __restrict__ offsets,
                       int count, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                       uint32_t* __restrict__ hist, int nblocks, int* status) {
    __shared__ uint32_t cnt[kRadix];
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) cnt[d] = 0;
    __syncthreads();
    int flags = 0;
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int it = 0; it < kSortItems; ++it) {
        int64_t i = base + it * kSortThreads + threadIdx.x;
        if (i < n) {
            int lo = 0, hi = count;  // offsets[lo] <= i < offsets[hi]
            while (hi - lo > 1) {
                int mid = (lo + hi) >> 1;
                if (offsets[mid] <= i) lo = mid;
                else hi = mid;
            }
            const BatchKeyParams& b = bkp[lo];
            const KeyParams& kp = b.kp;
            float x = xy[2 * i], y = xy[2 * i + 1];
            if (!isfinite(gamma[i])) flags |= kFlagNonfinite;
            uint32_t ix, iy;
            if (kp.fast) {
                ix = leaf_coord_f32(x, kp.lox, kp.hix, kp.x0f, kp.scalef, kp.margin, kp.x0,
                                    kp.scale, kp.top, &flags);
                iy = leaf_coord_f32(y, kp.loy, kp.hiy, kp.y0f, kp.scalef, kp.margin, kp.y0,
                                    kp.scale, kp.top, &flags);
            } else {
                ix = leaf_coord((double)x, kp.x0, kp.x1, kp.scale, kp.top, &flags);
                iy = leaf_coord((double)y, kp.y0, kp.y1, kp.scale, kp.top, &flags);
            }
            uint32_t k = b.leaf_base + morton_key(ix, iy);
            keys[i] = k;
            vals[i] = (uint32_t)i;
            atomicAdd(&cnt[k & (kRadix - 1)], 1u);
        }
    }
    if (flags) atomicOr(status, flags);
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x)
        hist[(int64_t)d * nblocks + blockIdx.x] = cnt[d];
}

}  // namespace

size_t batch_key_params_bytes(int count) { return sizeof(BatchKeyParams) * (size_t)count; }

cudaError_t batch_key_params(const BatchInst* host_inst, int count, void* dev_params,
                             cudaStream_t s) {
    static_assert(sizeof(BatchKeyParams) % 8 == 0, "aligned records");
    BatchKeyParams* h = new BatchKeyParams[count];
    for (int i = 0; i < count; ++i) {
        const Geometry& g = host_inst[i].g;
        h[i].kp = make_key_params(g.x0, g.y0, g.W, g.L);
        h[i].leaf_base = host_inst[i].leaf_base;
        h[i].L = g.L;
    }
    cudaError_t e = cudaMemcpyAsync(dev_params, h, sizeof(BatchKeyParams) * count,
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    delete[] h;
    return e;
}

cudaError_t launch_batch_tree(const void* dev_key_params, const int64_t* dev_offsets, int count,
                              int64_t ntotal, int key_bits, uint32_t nleaf_total, const float* xy,
                              const float* gamma, SortBuffers& sb, void* particles,
                              cudaStream_t s) {
    if (ntotal == 0) {
        leaf_bounds_kernel<<<1, 32, 0, s>>>(0, sb.keys[0], nleaf_total, sb.leaf_start);
        return cudaGetLastError();
    }
    int nblocks = (int)((ntotal + kSortTile - 1) / kSortTile);
    int passes = sort_passes(key_bits);
    uint32_t* digit_total = sb.hist + (int64_t)kRadix * nblocks;
    batch_keys_hist_kernel<<<nblocks, kSortThreads, 0, s>>>(
        ntotal, xy, gamma, static_cast<const BatchKeyParams*>(dev_key_params), dev_offsets, count,
        sb.keys[0], sb.vals[0], sb.hist, nblocks, sb.status);
    for (int q = 0; q < passes; ++q) {
        int src = q & 1, dst = src ^ 1;
        int shift = q * kRadixBits;
        if (q > 0)
            hist_kernel<<<nblocks, kSortThreads, 0, s>>>(ntotal, sb.keys[src], shift, sb.hist,
                                                         nblocks);
        scan_digits_kernel<<<kRadix, 256, 0, s>>>(sb.hist, nblocks, digit_total);
        if (q == passes - 1)
            scatter_kernel<float, true><<<nblocks, kSortThreads, 0, s>>>(
                ntotal, sb.keys[src], sb.vals[src], shift, sb.hist, digit_total, nblocks,
                sb.keys[dst], sb.perm, xy, gamma, reinterpret_cast<float4*>(particles));
        else
            scatter_kernel<float, false><<<nblocks, kSortThreads, 0, s>>>(
                ntotal, sb.keys[src], sb.vals[src], shift, sb.hist, digit_total, nblocks,
                sb.keys[dst], sb.vals[dst], xy, gamma, reinterpret_cast<float4*>(particles));
    }
    const uint32_t* sorted = sb.keys[passes & 1];
    int lb_blocks = (int)((ntotal + 1 + 255) / 256);
    if (lb_blocks > 4096) lb_blocks = 4096;
    leaf_bounds_kernel<<<lb_blocks, 256, 0, s>>>(ntotal, sorted, nleaf_total, sb.leaf_start);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Tree build without allocation (fmm2d_tree_build_noalloc).
//
// For callers that cannot allocate device memory.  The scratch the build
// needs (two key/value ping-pong buffers, the digit counts and a status
// word) lives in one file-scope device array of fixed size, so the call
// itself allocates nothing.  Every GPU that loads the library holds this
// array (about 4.3 MB) until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kNoAllocMaxN = int64_t(1) << 18;  // particles per call at most
constexpr int64_t kNoAllocMaxBlocks = (kNoAllocMaxN + kSortTile - 1) / kSortTile;
constexpr size_t kNoAllocWords = 4 * kNoAllocMaxN + kRadix * kNoAllocMaxBlocks + kRadix + 64;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocWords];

std::mutex g_noalloc_mu;
uint32_t* g_noalloc_ptr[kNoAllocMaxDevices] = {};
unsigned long long g_noalloc_ctx[kNoAllocMaxDevices] = {};  // context id the address belongs to

// Unique id of the calling thread's current context (driver entry points;
// 0 if they are unavailable).  A context torn down and created again (for
// example after cudaDeviceReset) gets a new id, and the module holding the
// scratch array is loaded again, possibly at another address.
unsigned long long current_context_id() {
    typedef CUresult (*GetCurrentFn)(CUcontext*);
    typedef CUresult (*GetIdFn)(CUcontext, unsigned long long*);
    static GetCurrentFn get_current = nullptr;
    static GetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        cudaDriverEntryPointQueryResult q;
        void* f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetIdFn>(f);
        looked_up = true;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx &&
        get_id(ctx, &id) == CUDA_SUCCESS)
        return id;
    return 0;
}

// Device address of the scratch array in the current device's context.  In
// host code the array's name is only a host-side stand-in, so the address is
// asked of the runtime once per device (with that device current) and kept
// together with the id of the context it belongs to; a call in another
// context of that device (the old one reset) asks again.  Without a
// context id (none current yet on this thread, or no driver entry point) the
// address is asked again on that call.
cudaError_t noalloc_scratch(uint32_t** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev] || ctx == 0 || g_noalloc_ctx[dev] != ctx) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<uint32_t*>(p);
        g_noalloc_ctx[dev] = ctx;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

template <typename R>
cudaError_t tree_build_noalloc(int64_t n, const R* xy, const R* gamma, int L, double x0,
                               double y0, double W, uint32_t* keys_out, uint32_t* perm_out,
                               uint32_t* leaf_start_out, int* flags_out, uint32_t* scratch,
                               cudaStream_t s) {
    uint32_t* kA = scratch;
    uint32_t* vA = kA + kNoAllocMaxN;
    uint32_t* kB = vA + kNoAllocMaxN;
    uint32_t* vB = kB + kNoAllocMaxN;
    uint32_t* hist = vB + kNoAllocMaxN;
    uint32_t* digit_total = hist + kRadix * kNoAllocMaxBlocks;
    int* status = flags_out ? flags_out : reinterpret_cast<int*>(digit_total + kRadix);
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);  // flags start clear
    if (e != cudaSuccess) return e;
    uint32_t nleaf = 1u << (2 * L);
    if (n == 0) {
        leaf_bounds_kernel<<<1, 32, 0, s>>>(0, keys_out, nleaf, leaf_start_out);
        return cudaGetLastError();
    }
    KeyParams kp = make_key_params(x0, y0, W, L);
    int nblocks = (int)((n + kSortTile - 1) / kSortTile);
    int bits = 2 * L;
    int passes = sort_passes(bits);
    keys_hist_kernel<R><<<nblocks, kSortThreads, 0, s>>>(n, xy, gamma, kp, kA, vA, hist, nblocks,
                                                         status);
    for (int q = 0; q < passes; ++q) {
        bool even = (q & 1) == 0;
        uint32_t* sk = even ? kA : kB;
        uint32_t* sv = even ? vA : vB;
        bool last = q == passes - 1;
        uint32_t* dk = last ? keys_out : (even ? kB : kA);
        uint32_t* dv = last ? perm_out : (even ? vB : vA);
        int shift = q * kRadixBits;
        if (q > 0) hist_kernel<<<nblocks, kSortThreads, 0, s>>>(n, sk, shift, hist, nblocks);
        scan_digits_kernel<<<kRadix, 256, 0, s>>>(hist, nblocks, digit_total);
        scatter_kernel<R, false><<<nblocks, kSortThreads, 0, s>>>(
            n, sk, sv, shift, hist, digit_total, nblocks, dk, dv, xy, gamma, nullptr);
    }
    int lb_blocks = (int)((n + 1 + 255) / 256);
    leaf_bounds_kernel<<<lb_blocks, 256, 0, s>>>(n, keys_out, nleaf, leaf_start_out);
    return cudaGetLastError();
}

}  // namespace
}  // namespace fmm2d

extern "C" fmm2d_status fmm2d_tree_build_noalloc(int precision, int64_t n, const void* xy_dev,
                                                 const void* gamma_dev, int L, double x0,
                                                 double y0, double W, uint32_t* keys_dev,
                                                 uint32_t* perm_dev, uint32_t* leaf_start_dev,
                                                 int* flags_dev, cudaStream_t stream) {
    using namespace fmm2d;
    if (precision < FMM2D_FP64 || precision > FMM2D_FP32_TC) return FMM2D_INVALID_ARG;
    if (L < 0 || L > kMaxL || !(W > 0.0) || !isfinite(W) || !isfinite(x0) || !isfinite(y0))
        return FMM2D_INVALID_ARG;
    if (n < 0 || n > kNoAllocMaxN) return FMM2D_INVALID_ARG;  // beyond the static scratch
    if (!leaf_start_dev || (n > 0 && (!xy_dev || !gamma_dev || !keys_dev || !perm_dev)))
        return FMM2D_INVALID_ARG;
    uint32_t* scratch = nullptr;
    if (noalloc_scratch(&scratch) != cudaSuccess) return FMM2D_CUDA_ERROR;
    cudaError_t e =
        precision == FMM2D_FP64
            ? tree_build_noalloc<double>(n, static_cast<const double*>(xy_dev),
                                         static_cast<const double*>(gamma_dev), L, x0, y0, W,
                                         keys_dev, perm_dev, leaf_start_dev, flags_dev, scratch,
                                         stream)
            : tree_build_noalloc<float>(n, static_cast<const float*>(xy_dev),
                                        static_cast<const float*>(gamma_dev), L, x0, y0, W,
                                        keys_dev, perm_dev, leaf_start_dev, flags_dev, scratch,
                                        stream);
    return e == cudaSuccess ? FMM2D_OK : FMM2D_CUDA_ERROR;
}

