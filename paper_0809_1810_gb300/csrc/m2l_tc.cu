// M2L (Eq. 22) as a dense contraction on the 5th-generation tensor cores,
// in 3xTF32 split products with FP32 accumulation in tensor memory.
//
// With box-size-scaled expansions the M2L operator of a source box at offset
// (dx, dy) from the target is one fixed complex P x P matrix (tables.cu).
// Written over real numbers (re/im interleaved), the local expansions of a
// tile of 128 same-parity target boxes are
//   LE[128 x 2P] = sum_{27 offsets} ME_shifted[128 x 2P] * B_offset[2P x 2P].
// The expansion arrays are stored as four parity planes per level, each a
// row-major grid, so for a fixed offset the 128 source rows of a tile form a
// rectangle of one source plane: one TMA box, with the domain edge
// zero-filled by the copy engine.
//
// Precision: x = hi + lo with hi = tf32(x) (round to nearest) and
// lo = tf32(x - hi); D = A_hi B_hi + A_hi B_lo + A_lo B_hi, so the products
// carry ~22 bits.  The tensor core's accumulation truncates, and its error
// grows with the number of MMAs summed into one accumulator, so the products
// go to 8 accumulators in tensor memory -- the A_hi B_hi products of the 27
// offsets spread round-robin over 7, all correction products (small) in the
// 8th -- and the epilogue adds the 8 with round-to-nearest FP32 adds.  The
// multipole expansions are split by m2l_split_kernel, the matrices once per
// plan by m2l_tc_tables_kernel.
//
// CTA = 4 warps.  Warp 0 lane 0 issues the TMA copies into an S-stage ring,
// warp 1 lane 0 issues tcgen05.mma (M = 128, N = 2P, K = 8) and commits each
// stage back to the producer; all 128 threads then read the accumulator
// rows from tensor memory (thread t = row t) and store the local expansions.
// Every wait on an mbarrier is bounded; on expiry the kernel records
// FMM2D_TIMEOUT in the status word, drains what it issued, frees tensor
// memory and returns.
#include <cuda.h>

#include "fmm2d_internal.cuh"

namespace fmm2d {
namespace {

constexpr uint32_t kSpinLimit = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)),
                 "r"(bytes)
                 : "memory");
}
// Bounded wait for the phase with parity `phase` to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t phase) {
    for (uint32_t it = 0; it < kSpinLimit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(b)), "r"(phase)
            : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}
// Shared-memory matrix descriptor: K-major operand in the 128-byte swizzled
// canonical layout (rows of 128 B, 8-row groups 1024 B apart).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;            // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset between 8-row groups
    d |= (uint64_t)1 << 46;            // descriptor version
    d |= (uint64_t)2 << 61;            // 128-byte swizzle
    return d;
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Instruction descriptor: D f32, A and B tf32, both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_tf32(uint32_t n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

constexpr int kAccs = 8;       // accumulators in tensor memory
constexpr int kMainAccs = 7;   // for A_hi B_hi; the last one takes the corrections

// KC K-chunks of 32 floats (2P = 32 KC), ST pipeline stages.  At 2P = 32 a
// stage is 40 KB: two stages let two CTAs share an SM (many tiles), four
// keep more loads in flight for one CTA per SM (fewer tiles than SMs).  At
// 2P = 64 a stage is 96 KB and two fit.
template <int KC, int ST>
struct TcShape {
    static constexpr int kN = 32 * KC;                    // 2P columns
    static constexpr int kTmemCols = kAccs * kN;          // 256 or 512 (power of two)
    static constexpr int kStages = ST;
    static constexpr int kABytes = 128 * 128;             // one 128 x 32-float K chunk
    static constexpr int kBBytes = kN * 128;              // one kN x 32-float K chunk
    static constexpr int kStageBytes = 2 * KC * (kABytes + kBBytes);
    static constexpr int kSmem = kStages * kStageBytes + 1024;  // + alignment slack
};

__global__ void __launch_bounds__(256)
m2l_split_kernel(const float* __restrict__ me, float* __restrict__ hi, float* __restrict__ lo,
                 int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        float x = me[i];
        float h = tf32_rna(x);
        hi[i] = h;
        lo[i] = tf32_rna(x - h);
    }
}

// B^T of every offset slot, real-ified: for complex T[n][k] (stored [k][n]),
// Bt[2n][2k] = Re T, Bt[2n][2k+1] = -Im T, Bt[2n+1][2k] = Im T, Bt[2n+1][2k+1] = Re T.
__global__ void m2l_tc_tables_kernel(const double* __restrict__ m2l64, int P,
                                     float* __restrict__ bhi, float* __restrict__ blo) {
    const int n2 = 2 * P;
    const int64_t total = (int64_t)kOffsetSlots * n2 * n2;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int slot = (int)(e / (n2 * n2));
        int row = (int)((e / n2) % n2);  // n'
        int col = (int)(e % n2);         // k'
        int n = row >> 1, k = col >> 1;
        const double* t = m2l64 + (((int64_t)slot * P + k) * P + n) * 2;
        double re = t[0], im = t[1];
        double v = (row & 1) == 0 ? ((col & 1) == 0 ? re : -im) : ((col & 1) == 0 ? im : re);
        float h = tf32_rna((float)v);
        bhi[e] = h;
        blo[e] = tf32_rna((float)(v - (double)h));
    }
}

template <int KC, int ST>
__global__ void __launch_bounds__(128, 1)
m2l_tc_kernel(const __grid_constant__ M2LTcMaps maps, const int4* __restrict__ tiles, Geometry g,
              float* __restrict__ le, int* status) {
    using S = TcShape<KC, ST>;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[S::kStages], empty[S::kStages], done;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int4 tile = tiles[blockIdx.x];
    const int level = tile.x, plane = tile.y, X0 = tile.z, Y0 = tile.w;
    const int px = plane & 1, py = plane >> 1;
    const int Wh = 1 << (level - 1);
    const int bw = Wh < 128 ? Wh : 128;
    const int bh = (128 / bw) < Wh ? (128 / bw) : Wh;
    const uint32_t a_box_bytes = 128u * (uint32_t)(bw * bh);
    const uint32_t stage_tx = 2u * KC * (a_box_bytes + (uint32_t)S::kBBytes);

    if (tid == 0) {
        for (int s = 0; s < S::kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile(
            "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                smem_u32(&tmem_base)),
            "r"((uint32_t)S::kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;

    // the 27 interaction offsets of this parity: children of the parent's
    // neighbours outside the local list (Sec. 3.3.1)
    auto offset_of = [&](int i, int* dx, int* dy) {
        int c = 0;
        for (int yy = -2 - py; yy <= 3 - py; ++yy)
            for (int xx = -2 - px; xx <= 3 - px; ++xx) {
                if (xx >= -1 && xx <= 1 && yy >= -1 && yy <= 1) continue;
                if (c == i) {
                    *dx = xx;
                    *dy = yy;
                    return;
                }
                ++c;
            }
    };
    constexpr int kOffsets = 27;

    if (warp == 0 && lane == 0) {  // TMA producer
        int issued = 0;
        for (int i = 0; i < kOffsets; ++i) {
            const int s = i % S::kStages;
            if (i >= S::kStages && !mbar_wait(&empty[s], ((i / S::kStages) - 1) & 1)) {
                atomicOr(status, kFlagTimeout);
                abort_flag = 1;
                break;
            }
            int dx, dy;
            offset_of(i, &dx, &dy);
            const int sxp = (px + dx) & 1, syp = (py + dy) & 1;
            const int ox = (px + dx - sxp) / 2, oy = (py + dy - syp) / 2;  // exact halving
            const int splane = syp * 2 + sxp;
            const int slot = offset_slot(dx, dy);
            uint8_t* st = smem + s * S::kStageBytes;
            mbar_expect_tx(&full[s], stage_tx);
            for (int kc = 0; kc < KC; ++kc) {
                tma_load_4d(st + kc * S::kABytes, &maps.me_hi[level], kc * 32, X0 + ox, Y0 + oy,
                            splane, &full[s]);
                tma_load_4d(st + (KC + kc) * S::kABytes, &maps.me_lo[level], kc * 32, X0 + ox,
                            Y0 + oy, splane, &full[s]);
                uint8_t* sb = st + 2 * KC * S::kABytes;
                tma_load_3d(sb + kc * S::kBBytes, &maps.b_hi, kc * 32, 0, slot, &full[s]);
                tma_load_3d(sb + (KC + kc) * S::kBBytes, &maps.b_lo, kc * 32, 0, slot, &full[s]);
            }
            ++issued;
        }
        // on abort, wait (bounded) for the copies still in flight: the last
        // load armed on each stage
        if (abort_flag)
            for (int i = (issued > S::kStages ? issued - S::kStages : 0); i < issued; ++i)
                mbar_wait(&full[i % S::kStages], (i / S::kStages) & 1);
    } else if (warp == 1 && lane == 0) {  // MMA issuer
        constexpr uint32_t idesc = idesc_tf32(S::kN);
        bool ok = true;
        for (int i = 0; i < kOffsets && ok; ++i) {
            const int s = i % S::kStages;
            if (!mbar_wait(&full[s], (i / S::kStages) & 1)) {
                atomicOr(status, kFlagTimeout);
                abort_flag = 1;
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t st = smem_u32(smem + s * S::kStageBytes);
            for (int kc = 0; kc < KC; ++kc) {
                const uint32_t a_hi = st + kc * S::kABytes, a_lo = st + (KC + kc) * S::kABytes;
                const uint32_t b0 = st + 2 * KC * S::kABytes;
                const uint32_t b_hi = b0 + kc * S::kBBytes, b_lo = b0 + (KC + kc) * S::kBBytes;
                const uint32_t acc_main = tmem + (uint32_t)((i % kMainAccs) * S::kN);
                const uint32_t acc_corr = tmem + (uint32_t)(kMainAccs * S::kN);
#pragma unroll
                for (int k8 = 0; k8 < 4; ++k8) {
                    const uint32_t off = k8 * 32;  // 8 tf32 = 32 bytes along K
                    const uint64_t dah = sdesc_sw128(a_hi + off), dal = sdesc_sw128(a_lo + off);
                    const uint64_t dbh = sdesc_sw128(b_hi + off), dbl = sdesc_sw128(b_lo + off);
                    const bool first = kc == 0 && k8 == 0;  // first product of the accumulator
                    mma_tf32(acc_main, dah, dbh, idesc, !(first && i < kMainAccs));
                    mma_tf32(acc_corr, dah, dbl, idesc, !(first && i == 0));
                    mma_tf32(acc_corr, dal, dbh, idesc, 1);
                }
            }
            mma_commit(&empty[s]);  // frees the stage once these MMAs have read it
        }
        if (ok) mma_commit(&done);
    }
    __syncwarp();
    // epilogue: thread t holds accumulator row t (TMEM lane t)
    const bool ok = mbar_wait(&done, 0);
    if (!ok) atomicOr(status, kFlagTimeout);
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int m = tid;
    const int ix_local = m % bw, iy_local = m / bw;
    const int IX = X0 + ix_local, IY = Y0 + iy_local;
    const bool valid = ok && m < bw * bh && IX < Wh && IY < Wh;
    float* dst = le + (g.level_base[level] + ((int64_t)(plane * Wh + IY) * Wh + IX)) * (2 * g.P);
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
    for (int c0 = 0; c0 < S::kN; c0 += 32) {
        float sum[32];
        uint32_t r[32];
        tmem_ld32(lane_base + (uint32_t)(kMainAccs * S::kN + c0), r);  // corrections first
#pragma unroll
        for (int j = 0; j < 32; ++j) sum[j] = __uint_as_float(r[j]);
        for (int a = 0; a < kMainAccs; ++a) {
            tmem_ld32(lane_base + (uint32_t)(a * S::kN + c0), r);
#pragma unroll
            for (int j = 0; j < 32; ++j) sum[j] += __uint_as_float(r[j]);
        }
        if (valid) {
            float4* d4 = reinterpret_cast<float4*>(dst + c0);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                d4[j] = make_float4(sum[4 * j], sum[4 * j + 1], sum[4 * j + 2], sum[4 * j + 3]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)S::kTmemCols));
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

}  // namespace

int m2l_tc_smem_bytes(int P) { return P <= 16 ? TcShape<1, 4>::kSmem : TcShape<2, 2>::kSmem; }

cudaError_t m2l_tc_prepare(const Geometry& g, const double* m2l64, float* me_hi, float* me_lo,
                           float* bhi, float* blo, M2LTcMaps* maps, int4* tiles_host,
                           int* ntiles, cudaStream_t s) {
    EncodeTiledFn enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    const int n2 = 2 * g.P;
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int l = 2; l <= g.L; ++l) {
        const cuuint64_t Wh = 1ull << (l - 1);
        const cuuint64_t dims[4] = {(cuuint64_t)n2, Wh, Wh, 4};
        const cuuint64_t strides[3] = {(cuuint64_t)n2 * 4, (cuuint64_t)n2 * 4 * Wh,
                                       (cuuint64_t)n2 * 4 * Wh * Wh};
        const cuuint32_t bw = Wh < 128 ? (cuuint32_t)Wh : 128u;
        const cuuint32_t bh = (128u / bw) < Wh ? 128u / bw : (cuuint32_t)Wh;
        const cuuint32_t box[4] = {32, bw, bh, 1};
        for (int which = 0; which < 2; ++which) {
            float* base = (which ? me_lo : me_hi) + g.level_base[l] * n2;
            CUresult r = enc(which ? &maps->me_lo[l] : &maps->me_hi[l],
                             CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
        }
    }
    {
        const cuuint64_t dims[3] = {(cuuint64_t)n2, (cuuint64_t)n2, (cuuint64_t)kOffsetSlots};
        const cuuint64_t strides[2] = {(cuuint64_t)n2 * 4, (cuuint64_t)n2 * n2 * 4};
        const cuuint32_t box[3] = {32, (cuuint32_t)n2, 1};
        for (int which = 0; which < 2; ++which) {
            CUresult r = enc(which ? &maps->b_lo : &maps->b_hi, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                             which ? blo : bhi, dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
        }
    }
    int count = 0;
    for (int l = 2; l <= g.L; ++l) {
        const int Wh = 1 << (l - 1);
        const int bw = Wh < 128 ? Wh : 128;
        const int bh = (128 / bw) < Wh ? 128 / bw : Wh;
        for (int pl = 0; pl < 4; ++pl)
            for (int y = 0; y < Wh; y += bh)
                for (int x = 0; x < Wh; x += bw) {
                    if (tiles_host) tiles_host[count] = make_int4(l, pl, x, y);
                    ++count;
                }
    }
    *ntiles = count;
    int64_t total = (int64_t)kOffsetSlots * n2 * n2;
    int blocks = (int)((total + 255) / 256);
    m2l_tc_tables_kernel<<<blocks, 256, 0, s>>>(m2l64, g.P, bhi, blo);
    return cudaGetLastError();
}

cudaError_t launch_m2l_tc(const Geometry& g, const M2LTcMaps& maps, const int4* tiles, int ntiles,
                          const float* me, float* me_hi, float* me_lo, float* le, int* status,
                          cudaStream_t s) {
    if (g.L < 2) return cudaSuccess;
    const int64_t count = g.nboxes * 2 * g.P;
    int blocks = (int)((count + 255) / 256);
    if (blocks > 8192) blocks = 8192;
    m2l_split_kernel<<<blocks, 256, 0, s>>>(me, me_hi, me_lo, count);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (g.P > 16)
        m2l_tc_kernel<2, 2><<<ntiles, 128, TcShape<2, 2>::kSmem, s>>>(maps, tiles, g, le, status);
    else if (ntiles <= sms)
        m2l_tc_kernel<1, 4><<<ntiles, 128, TcShape<1, 4>::kSmem, s>>>(maps, tiles, g, le, status);
    else
        m2l_tc_kernel<1, 2><<<ntiles, 128, TcShape<1, 2>::kSmem, s>>>(maps, tiles, g, le, status);
    return cudaGetLastError();
}

cudaError_t m2l_tc_configure() {
    cudaError_t e = cudaFuncSetAttribute(m2l_tc_kernel<1, 4>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TcShape<1, 4>::kSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(m2l_tc_kernel<1, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 TcShape<1, 2>::kSmem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(m2l_tc_kernel<2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                TcShape<2, 2>::kSmem);
}

}  // namespace fmm2d
