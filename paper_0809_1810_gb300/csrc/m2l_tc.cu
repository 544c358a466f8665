// M2L (Eq. 22) over the interaction lists (Sec. 3.3.1) as a dense
// contraction on the 5th-generation tensor cores, in 3xTF32 split products
// with FP32 accumulation in tensor memory.
//
// Formulation.  With box-size-scaled expansions the M2L operator between two
// boxes of one level depends only on their offset (tables.cu), and the
// interaction list of a box is the children of its parent's neighbours that
// are not its own neighbours.  So for a target parent T and each of its 8
// neighbour offsets D, the local expansions of T's four children receive
//   LE[T, 4 x 2Pk] += ME[T + D, 4 x 2Pk] * B_D[4 x 2Pk, 4 x 2Pk]
// where B_D holds the scaled child-offset matrices (real-ified: re/im
// interleaved) and zero blocks where the two children are adjacent (those
// pairs belong to the near field or to a finer level), Pk = p rounded up to
// a multiple of 4.  One tile of 128 target parents is the GEMM
//   D[128 x N] = sum over (D, source child, k) of A * B,   N = 8 Pk <= 256,
// one column per real coefficient of the four children.
//
// Data reuse.  A tile is a tw x th rectangle of target parents; its source
// parents are the (tw+2) x (th+2) halo around it.  The halo is loaded once
// per K chunk by TMA into shared memory in the no-swizzle K-major layout,
// whose rows sit 16 bytes apart within a k-group (4 reals): target parent
// (x, y) is MMA row m = y Hw + x (Hw = tw + 2), and the source parent at
// offset D is halo row m + (Hw + 1) + D_y Hw + D_x, so the 8 offsets read the
// same halo through descriptors whose start address moves by whole rows.
// MMA rows that fall on halo columns are computed and discarded.  The
// operator stages (B_D for one source child and K chunk, hi and lo) are
// stored in global memory exactly as the kernel's shared-memory slots hold
// them and arrive by plain bulk copies.
//
// Precision: x = hi + lo with hi = tf32(x) (round to nearest) and lo =
// tf32(x - hi); D = A_hi B_hi + A_hi B_lo + A_lo B_hi.  The tensor core's
// accumulation truncates and its error grows with the number of MMAs summed
// into one accumulator, so the A_hi B_hi products go to chains of 16 MMAs (two
// K chunks of the 8 offsets) in a tensor-memory accumulator that the epilogue
// warps drain into FP32 registers with round-to-nearest adds (two such
// accumulators alternate when tensor memory has room for them); the small
// correction products all go to one accumulator, added at the end.
//
// CTA = 10 warps.  Warp 8 lane 0 issues the TMA halo boxes and the bulk
// copies of the operator stages into rings of shared-memory slots; warp 9
// lane 0 issues tcgen05.mma (M = 128, N = 8 Pk, K = 8) and commits every slot
// back to the producer; warps 0-7 drain the accumulators (warp w reads tensor
// memory lanes 32 (w % 4) + [0, 32), column half w / 4) and store the local
// expansions.  Every wait on an mbarrier is bounded by a poll limit; when one
// runs out the kernel records FMM2D_TIMEOUT, stops issuing, waits with the
// default limit for the copies it issued and for the MMAs it issued (the MMA
// thread commits them to `done` on every path), then frees tensor memory and
// returns.
#include <cuda.h>

#include <algorithm>
#include <climits>
#include <vector>

#include "fmm2d_internal.cuh"

namespace fmm2d {
namespace {

constexpr int kThreads = 320;
constexpr int kEpiWarps = 8;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kProducerWarp = 8;
constexpr int kMmaWarp = 9;
constexpr int kHaloSlots = 4;
constexpr int kMaxBStages = 24;
constexpr int kChainSteps = 2;          // K chunks per main-accumulator chain: 16 MMAs
constexpr uint32_t kPollNs = 32;        // suspend hint of one poll
// dynamic shared memory a CTA opts into: the 227 KB per block less room for
// the kernel's static barriers
constexpr int kSmemLimit = 226 * 1024;

// Tensor-memory columns of a CTA: a power of two >= 32 covering the main
// accumulators and the correction accumulator.
__host__ __device__ constexpr uint32_t tmem_cols(int n_cols) {
    return n_cols <= 32 ? 32u : n_cols <= 64 ? 64u : n_cols <= 128 ? 128u : n_cols <= 256 ? 256u
                                                                                       : 512u;
}

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
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
// Wait for the phase with parity `phase`: at most `limit` polls of about
// kPollNs each; gives up early once `abort` is set (null: never).
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t phase, uint32_t limit,
                                          volatile int* abort) {
    {  // non-blocking first test: a phase already complete costs no suspension
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(b)), "r"(phase)
            : "memory");
        if (done) return true;
    }
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(b)), "r"(phase), "r"(kPollNs)
            : "memory");
        if (ok) return true;
        if (abort && *abort) return false;
    }
    return false;
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(dst),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// Shared-memory matrix descriptor, K-major operand in the no-swizzle layout:
// core matrices of 8 rows x 16 bytes, rows 16 bytes apart (stride byte offset
// 128 between 8-row groups), k-groups `kstride` bytes apart (leading byte
// offset).  Any 16-byte-aligned start address is legal, so the operand can
// begin at any row.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t kstride) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((kstride >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)(128 >> 4) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version; swizzle bits 0 = none
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
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
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

// Parent offsets per operator stage: enough MMAs (3 per offset) between two
// barrier round trips of the issuing thread to keep the tensor pipe busy,
// within shared memory (a stage is 64 N bytes per offset).
__host__ __device__ constexpr int offsets_per_stage(int n_cols) { return n_cols <= 192 ? 4 : 2; }

// Neighbour offset d (0..7) of a parent: the 3 x 3 block without its centre.
__host__ __device__ inline void parent_offset(int d, int* dx, int* dy) {
    const int idx = d < 4 ? d : d + 1;
    *dx = idx % 3 - 1;
    *dy = idx / 3 - 1;
}

struct M2LTcArgs {
    // two records per CTA: (level, X0, Y0, tw | th << 8) and (slot, LE offset
    // low, high word, p): the instance slot of the level's halo map, the
    // first real of the level's local expansions in `le`, and the instance's
    // expansion terms (local-expansion coefficients from p up are stored as
    // zero, as an operator built for that p gives them)
    const int4* tiles;
    const float* bimg;  // operator stages
    float* le;
    int* status;
    int P;           // terms per box in the expansion arrays
    int halo_bytes;  // one halo slot (hi or lo part)
    int b_stages;    // operator slots
    uint32_t spin;   // poll limit of the pipeline waits
};

// Multipoles split into TF32 hi/lo parts in the halo layout: box b of level
// l (parity plane, row Y, column X of its plane) goes to
// [level_base[l] KG + ((plane KG + kg) G + Y) G + X] (float4 units), kg the
// k-group of 4 reals, KG = Pk / 2, G = 2^(l-1).
__global__ void __launch_bounds__(256)
m2l_tc_split_kernel(const float* __restrict__ me, float4* __restrict__ hi,
                    float4* __restrict__ lo, Geometry g, int Pk) {
    const int KG = Pk / 2;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < g.nboxes;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int l = slot_level(g.level_base, g.L, b);
        const int64_t G = (int64_t)1 << (l - 1);
        const int64_t r = b - g.level_base[l];
        const int64_t plane = r / (G * G), rem = r % (G * G);
        const float4* src = reinterpret_cast<const float4*>(me + b * (2 * g.P));
        const int64_t out0 = g.level_base[l] * KG + (plane * KG * G) * G + rem;
        for (int kg = 0; kg < KG; ++kg) {
            const float4 v = src[kg];
            float4 h, o;
            h.x = tf32_rna(v.x);
            h.y = tf32_rna(v.y);
            h.z = tf32_rna(v.z);
            h.w = tf32_rna(v.w);
            o.x = tf32_rna(v.x - h.x);
            o.y = tf32_rna(v.y - h.y);
            o.z = tf32_rna(v.z - h.z);
            o.w = tf32_rna(v.w - h.w);
            const int64_t at = out0 + (int64_t)kg * G * G;
            hi[at] = h;
            lo[at] = o;
        }
    }
}

// The batch form: box r of class instance j (instance inst[j]) goes to its
// instance slot's block of the level's stacked arrays, dst_base[j][level].
__global__ void __launch_bounds__(256)
m2l_tc_split_batch_kernel(const BatchInst* __restrict__ insts, const int32_t* __restrict__ ids,
                          const int64_t* __restrict__ prefix, const int64_t* __restrict__ dst_base,
                          int count, int64_t boxes, int Pk, const float* __restrict__ me,
                          float4* __restrict__ hi, float4* __restrict__ lo) {
    const int KG = Pk / 2;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < boxes;
         b += (int64_t)gridDim.x * blockDim.x) {
        int lo_j = 0, hi_j = count;  // prefix[lo_j] <= b < prefix[hi_j]
        while (hi_j - lo_j > 1) {
            const int mid = (lo_j + hi_j) >> 1;
            if (prefix[mid] <= b) lo_j = mid;
            else hi_j = mid;
        }
        const BatchInst& in = insts[ids[lo_j]];
        const int64_t r = b - prefix[lo_j];
        const int l = slot_level(in.g.level_base, in.g.L, r);
        const int64_t G = (int64_t)1 << (l - 1);
        const int64_t q = r - in.g.level_base[l];
        const int64_t plane = q / (G * G), rem = q % (G * G);
        const float4* src = reinterpret_cast<const float4*>(me + in.exp_off + r * (2 * in.g.P));
        const int64_t out0 = dst_base[(int64_t)lo_j * (kMaxL + 1) + l] + (plane * KG * G) * G + rem;
        const int nr = 2 * in.g.p;  // reals of the instance's p terms; the rest read as zero
        for (int kg = 0; kg < KG; ++kg) {
            float4 v = src[kg];
            if (4 * kg >= nr) v.x = 0.f;
            if (4 * kg + 1 >= nr) v.y = 0.f;
            if (4 * kg + 2 >= nr) v.z = 0.f;
            if (4 * kg + 3 >= nr) v.w = 0.f;
            float4 h, o;
            h.x = tf32_rna(v.x);
            h.y = tf32_rna(v.y);
            h.z = tf32_rna(v.z);
            h.w = tf32_rna(v.w);
            o.x = tf32_rna(v.x - h.x);
            o.y = tf32_rna(v.y - h.y);
            o.z = tf32_rna(v.z - h.z);
            o.w = tf32_rna(v.w - h.w);
            const int64_t at = out0 + (int64_t)kg * G * G;
            hi[at] = h;
            lo[at] = o;
        }
    }
}

// Operator image: stage s = (source child sp, K chunk kc, parent offset d)
// in the order the kernel consumes them, s = (sp KC + kc) 8 + d.  A stage is
// 16 N floats: the hi part then the lo part, each two k-groups of N rows x 4
// reals (row = target child tp x 2Pk + real output index n', column the real
// input index k' = 8 kc + 4 group + j).  Entry: the real-ified scaled M2L
// matrix of child offset 2D + sp - tp (source minus target), zero for
// adjacent children and for n or k >= p; for complex T[n][k] (stored
// [k][n]), Bt[2n][2k] = Re T, Bt[2n][2k+1] = -Im T, Bt[2n+1][2k] = Im T,
// Bt[2n+1][2k+1] = Re T.
__global__ void m2l_tc_bimg_kernel(const double* __restrict__ m2l64, int P, int p, int Pk,
                                   float* __restrict__ bimg) {
    const int N = 8 * Pk, KC = Pk / 4;
    const int64_t per_stage = (int64_t)N * 8;
    const int64_t total = (int64_t)4 * KC * 8 * per_stage;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int stage = (int)(e / per_stage);
        const int rem = (int)(e % per_stage);
        const int row = rem / 8, kk = rem % 8;
        const int h = stage / 8, d = stage % 8;
        const int sp = h / KC, kc = h % KC;
        const int tp = row / (2 * Pk), np = row % (2 * Pk);
        const int kp = kc * 8 + kk;
        int Dx, Dy;
        parent_offset(d, &Dx, &Dy);
        const int ox = 2 * Dx + (sp & 1) - (tp & 1), oy = 2 * Dy + (sp >> 1) - (tp >> 1);
        double v = 0.0;
        const int n = np >> 1, k = kp >> 1;
        if ((ox < -1 || ox > 1 || oy < -1 || oy > 1) && n < p && k < p) {
            const double* t = m2l64 + (((int64_t)offset_slot(ox, oy) * P + k) * P + n) * 2;
            const double re = t[0], im = t[1];
            v = (np & 1) == 0 ? ((kp & 1) == 0 ? re : -im) : ((kp & 1) == 0 ? im : re);
        }
        const float hv = tf32_rna((float)v);
        const float lv = tf32_rna((float)(v - (double)hv));
        const int grp = kk / 4, j = kk % 4;
        float* st = bimg + (int64_t)stage * 16 * N;
        st[grp * 4 * N + row * 4 + j] = hv;
        st[8 * N + grp * 4 * N + row * 4 + j] = lv;
    }
}

template <int PK4>
__global__ void __launch_bounds__(kThreads, 1)
m2l_parent_tc_kernel(const __grid_constant__ M2LTcMaps maps, const M2LTcArgs a) {
    constexpr int Pk = 4 * PK4;
    constexpr int N = 8 * Pk;          // MMA columns: 4 children x 2Pk reals
    constexpr int HALF = N / 2;        // columns per epilogue thread
    constexpr int KG = Pk / 2;         // k-groups of 4 reals per child
    constexpr int KC = Pk / 4;         // K chunks of 8 reals (one MMA) per child
    constexpr int kSteps = 4 * KC;     // halo steps: (source child, K chunk)
    constexpr int NB = 3 * N <= 512 ? 2 : 1;  // main accumulators
    constexpr uint32_t kTmemCols = tmem_cols((NB + 1) * N);
    constexpr int kChains = (kSteps + kChainSteps - 1) / kChainSteps;
    constexpr int kGD = offsets_per_stage(N);   // parent offsets per operator stage
    constexpr int kSPH = 8 / kGD;              // operator stages per halo step
    constexpr uint32_t kBOff = 64u * N;        // one offset: hi and lo, 2 k-groups x N x 16 B
    constexpr uint32_t kBStage = kGD * kBOff;
    constexpr uint32_t idesc = idesc_tf32(N);

    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t halo_full[kHaloSlots], halo_empty[kHaloSlots];
    __shared__ __align__(8) uint64_t b_full[kMaxBStages], b_empty[kMaxBStages];
    __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], done;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t s_halo = smem_u32(smem);
    const uint32_t s_b = s_halo + 2u * kHaloSlots * (uint32_t)a.halo_bytes;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int4 tile = a.tiles[2 * blockIdx.x], tile2 = a.tiles[2 * blockIdx.x + 1];
    const int level = tile.x, X0 = tile.y, Y0 = tile.z;
    const int tw = tile.w & 0xFF, th = (tile.w >> 8) & 0xFF;
    const int slot = tile2.x, p_terms = tile2.w;
    const int64_t le_off = (int64_t)(uint32_t)tile2.y | ((int64_t)(uint32_t)tile2.z << 32);
    const int Hw = tw + 2, Hh = th + 2;
    const int G = 1 << (level - 1);
    const uint32_t box_bytes = 32u * (uint32_t)(Hw * Hh);  // 2 k-groups x Hw x Hh x 16 B
    const uint32_t kstride_a = 16u * (uint32_t)(Hw * Hh);

    if (tid == 0) {
        for (int s = 0; s < kHaloSlots; ++s) {
            mbar_init(&halo_full[s], 1);
            mbar_init(&halo_empty[s], 1);
        }
        for (int s = 0; s < a.b_stages; ++s) {
            mbar_init(&b_full[s], 1);
            mbar_init(&b_empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&acc_full[s], 1);
            mbar_init(&acc_empty[s], kEpiThreads);
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
            "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;

    if (warp == kProducerWarp) {
        if (lane == 0) {
            int h_issued = 0, b_issued = 0;
            bool ok = true;
            for (int h = 0; h < kSteps && ok; ++h) {
                const int sp = h / KC, kc = h % KC, hs = h % kHaloSlots;
                if (h >= kHaloSlots &&
                    !mbar_wait(&halo_empty[hs], ((h / kHaloSlots) - 1) & 1, a.spin, &abort_flag)) {
                    ok = false;
                    break;
                }
                mbar_expect_tx(&halo_full[hs], 2 * box_bytes);
                const uint32_t dst = s_halo + (uint32_t)(2 * hs) * (uint32_t)a.halo_bytes;
                // the halo's columns X0 - 1 .. X0 + tw as one run of 4 Hw reals
                // (a multiple of 4: 16-byte aligned; -4 reads the zero fill)
                tma_load_4d(dst, &maps.me_hi[level], 4 * (X0 - 1), Y0 - 1, sp * KG + 2 * kc,
                            slot, &halo_full[hs]);
                tma_load_4d(dst + (uint32_t)a.halo_bytes, &maps.me_lo[level], 4 * (X0 - 1),
                            Y0 - 1, sp * KG + 2 * kc, slot, &halo_full[hs]);
                ++h_issued;
                for (int j = 0; j < kSPH; ++j) {
                    const int b = h * kSPH + j, bs = b % a.b_stages;
                    if (b >= a.b_stages && !mbar_wait(&b_empty[bs], ((b / a.b_stages) - 1) & 1,
                                                      a.spin, &abort_flag)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&b_full[bs], kBStage);
                    bulk_load(s_b + (uint32_t)bs * kBStage, a.bimg + (int64_t)b * (kBStage / 4),
                              kBStage, &b_full[bs]);
                    ++b_issued;
                }
            }
            if (!ok) {
                atomicOr(a.status, kFlagTimeout);
                abort_flag = 1;
                // the copies still in flight land in this CTA's shared memory:
                // wait for the last one armed on each slot before leaving
                for (int i = max(0, h_issued - kHaloSlots); i < h_issued; ++i)
                    mbar_wait(&halo_full[i % kHaloSlots], (i / kHaloSlots) & 1, kSpinDefault,
                              nullptr);
                for (int i = max(0, b_issued - a.b_stages); i < b_issued; ++i)
                    mbar_wait(&b_full[i % a.b_stages], (i / a.b_stages) & 1, kSpinDefault,
                              nullptr);
            }
        }
    } else if (warp == kMmaWarp) {
        if (lane == 0) {
            // halo row of the source parent at each offset, in 16-byte units
            uint32_t shift16[8];
#pragma unroll
            for (int d = 0; d < 8; ++d) {
                int dx, dy;
                parent_offset(d, &dx, &dy);
                shift16[d] = (uint32_t)((Hw + 1) + dy * Hw + dx);
            }
            bool ok = true;
            for (int h = 0; h < kSteps && ok; ++h) {
                const int hs = h % kHaloSlots;
                const int c = h / kChainSteps, cpos = h % kChainSteps, buf = c % NB;
                if (cpos == 0 && c >= NB &&
                    !mbar_wait(&acc_empty[buf], ((c / NB) - 1) & 1, a.spin, &abort_flag)) {
                    ok = false;
                    break;
                }
                if (!mbar_wait(&halo_full[hs], (h / kHaloSlots) & 1, a.spin, &abort_flag)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t hbase = s_halo + (uint32_t)(2 * hs) * (uint32_t)a.halo_bytes;
                const uint64_t ah0 = sdesc(hbase, kstride_a);
                const uint64_t al0 = sdesc(hbase + (uint32_t)a.halo_bytes, kstride_a);
                const uint32_t acc_main = tmem + (uint32_t)(buf * N);
                const uint32_t acc_corr = tmem + (uint32_t)(NB * N);
                for (int j = 0; j < kSPH; ++j) {
                    const int b = h * kSPH + j, bs = b % a.b_stages;
                    if (!mbar_wait(&b_full[bs], (b / a.b_stages) & 1, a.spin, &abort_flag)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint64_t b0 = sdesc(s_b + (uint32_t)bs * kBStage, 16u * N);
#pragma unroll
                    for (int e = 0; e < kGD; ++e) {
                        const int d = j * kGD + e;
                        // the offset's rows of the halo: a start address moved by
                        // whole 16-byte rows (descriptor address field in 16 B)
                        const uint64_t ah = ah0 + (uint64_t)shift16[d];
                        const uint64_t al = al0 + (uint64_t)shift16[d];
                        const uint64_t bh = b0 + (uint64_t)(e * (kBOff >> 4));
                        const uint64_t bl = bh + (uint64_t)((32u * N) >> 4);
                        mma_tf32(acc_main, ah, bh, idesc, !(cpos == 0 && d == 0));
                        mma_tf32(acc_corr, ah, bl, idesc, !(h == 0 && d == 0));
                        mma_tf32(acc_corr, al, bh, idesc, 1u);
                    }
                    mma_commit(&b_empty[bs]);  // frees the slot once these MMAs have read it
                }
                if (!ok) break;
                mma_commit(&halo_empty[hs]);
                if (cpos == kChainSteps - 1 || h == kSteps - 1) mma_commit(&acc_full[buf]);
            }
            if (!ok) {
                atomicOr(a.status, kFlagTimeout);
                abort_flag = 1;
            }
            mma_commit(&done);  // every MMA issued above, on every path
        }
    } else {  // epilogue warps 0..7
        const int q = warp & 3, hh = warp >> 2;
        const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(hh * HALF);
        float sum[HALF];
#pragma unroll
        for (int j = 0; j < HALF; ++j) sum[j] = 0.f;
        bool ok = true;
        for (int c = 0; c < kChains; ++c) {
            const int buf = c % NB;
            const bool w = mbar_wait(&acc_full[buf], (c / NB) & 1, a.spin, &abort_flag);
            if (!__all_sync(0xffffffffu, w)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int j = 0; j < HALF; j += 16) {
                uint32_t r[16];
                tmem_ld16(tbase + (uint32_t)(buf * N + j), r);
#pragma unroll
                for (int i = 0; i < 16; ++i) sum[j + i] += __uint_as_float(r[i]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            mbar_arrive(&acc_empty[buf]);
        }
        if (!ok) {
            if (lane == 0) atomicOr(a.status, kFlagTimeout);
            abort_flag = 1;
        }
        // the MMAs' completion, on every path, before tensor memory is read
        // again or freed
        const bool dn = mbar_wait(&done, 0, kSpinDefault, nullptr);
        const bool aborted = abort_flag != 0;
        ok = __all_sync(0xffffffffu, ok && dn && !aborted);
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (ok) {
#pragma unroll
            for (int j = 0; j < HALF; j += 16) {
                uint32_t r[16];
                tmem_ld16(tbase + (uint32_t)(NB * N + j), r);
#pragma unroll
                for (int i = 0; i < 16; ++i) sum[j + i] += __uint_as_float(r[i]);
            }
            const int m = q * 32 + lane;  // accumulator row = tensor-memory lane
            const int x = m % Hw, y = m / Hw;
            const int X = X0 + x, Y = Y0 + y;
            if (x < tw && y < th && X < G && Y < G) {
#pragma unroll
                for (int t2 = 0; t2 < 2; ++t2) {
                    const int tp = 2 * hh + t2;  // target child (parity plane)
                    float4* d4 = reinterpret_cast<float4*>(
                        a.le + le_off + ((int64_t)(tp * G + Y) * G + X) * (2 * a.P));
                    const int nr = 2 * p_terms;  // reals kept
#pragma unroll
                    for (int j = 0; j < Pk / 2; ++j) {
                        const float* v = &sum[t2 * 2 * Pk + 4 * j];
                        d4[j] = make_float4(4 * j < nr ? v[0] : 0.f, 4 * j + 1 < nr ? v[1] : 0.f,
                                            4 * j + 2 < nr ? v[2] : 0.f,
                                            4 * j + 3 < nr ? v[3] : 0.f);
                    }
                    for (int j = Pk / 2; j < a.P / 2; ++j) d4[j] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols));
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

// Tile of target parents at a level of G x G parents: the tw x th rectangle
// (th (tw + 2) <= 128 MMA rows, tw <= 62) with the fewest tiles, then the
// smallest halo.
// Policy 1 (an autotuner candidate) takes the widest rows instead.
void choose_tile(int G, int* tw_out, int* th_out, int policy = 0) {
    if (policy == 1) {
        *tw_out = std::min(G, 62);
        *th_out = std::min(G, 128 / (*tw_out + 2));
        return;
    }
    long best = LONG_MAX, best_halo = LONG_MAX;
    int btw = 1, bth = 1;
    for (int tw = 1; tw <= G && tw <= 62; ++tw) {  // box inner extent 4 (tw + 2) <= 256
        const int Hw = tw + 2;
        const int th = std::min(G, 128 / Hw);
        if (th < 1) break;
        const long tiles = (long)((G + tw - 1) / tw) * ((G + th - 1) / th);
        const long halo = (long)Hw * (th + 2);
        if (tiles < best || (tiles == best && halo < best_halo)) {
            best = tiles;
            best_halo = halo;
            btw = tw;
            bth = th;
        }
    }
    *tw_out = btw;
    *th_out = bth;
}

template <int PK4>
cudaError_t launch_pk(const M2LTcConfig& cfg, const M2LTcMaps& maps, const M2LTcArgs& a,
                      cudaStream_t s) {
    m2l_parent_tc_kernel<PK4><<<cfg.ntiles, kThreads, cfg.smem, s>>>(maps, a);
    return cudaGetLastError();
}

template <int PK4>
cudaError_t configure_pk() {
    return cudaFuncSetAttribute(m2l_parent_tc_kernel<PK4>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
}

}  // namespace

namespace {
// Shared memory of a configuration whose largest halo needs `halo_rows`
// 16-byte rows per slot: the halo ring, then as many operator stages as fit
// (at most `want` when want > 0).
void finish_config(M2LTcConfig* c, int halo_rows, int want) {
    const int N = 8 * c->Pk;
    c->halo_bytes = ((halo_rows * 16) + 127) & ~127;
    const int stage = 64 * N * offsets_per_stage(N);
    const int budget = kSmemLimit - 1024 - 2 * kHaloSlots * c->halo_bytes;
    c->b_stages = std::min(kMaxBStages, budget / stage);
    if (want > 0) c->b_stages = std::min(c->b_stages, want);
    c->smem = 2 * kHaloSlots * c->halo_bytes + c->b_stages * stage + 1024;
    c->b_floats = (int64_t)4 * (c->Pk / 4) * 8 * 16 * N;
}
// rows one halo slot must hold for tiles tw x th: the TMA box (2 k-groups)
// and the furthest row an MMA reads (k-group 1, offset (1, 1), row 127)
int halo_rows_of(int tw, int th) {
    const int Hw = tw + 2, Hh = th + 2;
    return std::max(2 * Hw * Hh, Hw * Hh + 2 * Hw + 130);
}
}  // namespace

M2LTcConfig m2l_tc_plan(const Geometry& g, int4* tiles_host) {
    M2LTcConfig c{};
    c.Pk = (g.p + 3) & ~3;
    int count = 0, halo_rows = 0;
    for (int l = 2; l <= g.L; ++l) {
        const int G = 1 << (l - 1);
        int tw, th;
        choose_tile(G, &tw, &th);
        halo_rows = std::max(halo_rows, halo_rows_of(tw, th));
        const int64_t le_off = g.level_base[l] * 2 * g.P;
        for (int y = 0; y < G; y += th)
            for (int x = 0; x < G; x += tw) {
                if (tiles_host) {
                    tiles_host[2 * count] = make_int4(l, x, y, tw | (th << 8));
                    tiles_host[2 * count + 1] =
                        make_int4(0, (int)(uint32_t)le_off, (int)(uint32_t)(le_off >> 32), g.p);
                }
                ++count;
            }
    }
    c.ntiles = count;
    finish_config(&c, halo_rows, 0);
    return c;
}

cudaError_t m2l_tc_configure() {
    cudaError_t e = configure_pk<1>();
    if (e == cudaSuccess) e = configure_pk<2>();
    if (e == cudaSuccess) e = configure_pk<3>();
    if (e == cudaSuccess) e = configure_pk<4>();
    if (e == cudaSuccess) e = configure_pk<5>();
    if (e == cudaSuccess) e = configure_pk<6>();
    if (e == cudaSuccess) e = configure_pk<7>();
    if (e == cudaSuccess) e = configure_pk<8>();
    return e;
}

cudaError_t m2l_tc_prepare(const Geometry& g, const M2LTcConfig& cfg, const double* m2l64,
                           float* me_hi, float* me_lo, float* bimg, M2LTcMaps* maps,
                           cudaStream_t s) {
    EncodeTiledFn enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    if (cfg.b_stages < 2 || cfg.b_stages > kMaxBStages || cfg.Pk < 4 || cfg.Pk > kMaxP)
        return cudaErrorInvalidValue;
    const int KG = cfg.Pk / 2;
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int l = 2; l <= g.L; ++l) {
        const cuuint64_t G = 1ull << (l - 1);
        int tw, th;
        choose_tile((int)G, &tw, &th);
        // a row of the level's plane (G columns x 4 reals) is one contiguous
        // run: the box's inner extent is the halo's 4 Hw reals (16 Hw bytes),
        // landing as [k-group][row][column][4 reals] like the 4-D view would
        const cuuint64_t dims[4] = {4 * G, G, (cuuint64_t)4 * KG, 1};
        const cuuint64_t strides[3] = {16 * G, 16 * G * G, 16 * G * G * 4 * KG};
        const cuuint32_t box[4] = {(cuuint32_t)(4 * (tw + 2)), (cuuint32_t)(th + 2), 2, 1};
        for (int which = 0; which < 2; ++which) {
            float* base = (which ? me_lo : me_hi) + g.level_base[l] * 2 * cfg.Pk;
            CUresult r = enc(which ? &maps->me_lo[l] : &maps->me_hi[l],
                             CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
        }
    }
    const int64_t total = cfg.b_floats / 2;  // one thread per (stage, row, k) entry
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 8192);
    m2l_tc_bimg_kernel<<<blocks, 256, 0, s>>>(m2l64, g.P, g.p, cfg.Pk, bimg);
    return cudaGetLastError();
}

cudaError_t launch_m2l_tc(const Geometry& g, const M2LTcConfig& cfg, const M2LTcMaps& maps,
                          const int4* tiles, const float* me, float* me_hi, float* me_lo,
                          const float* bimg, float* le, int* status, uint32_t spin,
                          cudaStream_t s) {
    if (g.L < 2) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>((g.nboxes + 255) / 256, 4096);
    m2l_tc_split_kernel<<<blocks, 256, 0, s>>>(me, reinterpret_cast<float4*>(me_hi),
                                               reinterpret_cast<float4*>(me_lo), g, cfg.Pk);
    M2LTcArgs a{};
    a.tiles = tiles;
    a.bimg = bimg;
    a.le = le;
    a.status = status;
    a.P = g.P;
    a.halo_bytes = cfg.halo_bytes;
    a.b_stages = cfg.b_stages;
    a.spin = spin ? spin : kSpinDefault;
    switch (cfg.Pk / 4) {
        case 1: return launch_pk<1>(cfg, maps, a, s);
        case 2: return launch_pk<2>(cfg, maps, a, s);
        case 3: return launch_pk<3>(cfg, maps, a, s);
        case 4: return launch_pk<4>(cfg, maps, a, s);
        case 5: return launch_pk<5>(cfg, maps, a, s);
        case 6: return launch_pk<6>(cfg, maps, a, s);
        case 7: return launch_pk<7>(cfg, maps, a, s);
        case 8: return launch_pk<8>(cfg, maps, a, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t m2l_tc_batch_create(const BatchInst* host_inst, const int* ids, int nids, int Pk,
                                int P, const double* m2l64, int b_stages, int tile_policy,
                                M2LTcBatchClass* out, cudaStream_t s) {
    EncodeTiledFn enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    if (nids < 1 || Pk < 4 || Pk > kMaxP || (Pk & 3)) return cudaErrorInvalidValue;
    M2LTcBatchClass c;
    c.Pk = Pk;
    c.P = P;
    c.count = nids;
    c.cfg.Pk = Pk;
    const int KG = Pk / 2;
    int maxL = 0;
    for (int j = 0; j < nids; ++j) maxL = std::max(maxL, host_inst[ids[j]].g.L);
    // stacked layout: level l holds one block of KG x 4^l float4 per instance
    // with L >= l, in class order
    std::vector<int> nslot(kMaxL + 1, 0);
    for (int l = 2; l <= maxL; ++l)
        for (int j = 0; j < nids; ++j) nslot[l] += host_inst[ids[j]].g.L >= l;
    std::vector<int64_t> lvl(kMaxL + 2, 0);
    for (int l = 2; l <= maxL; ++l) lvl[l + 1] = lvl[l] + (int64_t)nslot[l] * KG * (1ll << (2 * l));
    const int64_t total4 = lvl[maxL + 1];
    std::vector<int64_t> dst((size_t)nids * (kMaxL + 1), 0), prefix(nids + 1, 0);
    std::vector<int> next(kMaxL + 1, 0);
    std::vector<std::vector<int>> slot_inst(kMaxL + 1);
    for (int j = 0; j < nids; ++j) {
        const BatchInst& in = host_inst[ids[j]];
        prefix[j + 1] = prefix[j] + in.g.nboxes;
        for (int l = 2; l <= in.g.L; ++l) {
            dst[(size_t)j * (kMaxL + 1) + l] = lvl[l] + (int64_t)next[l] * KG * (1ll << (2 * l));
            slot_inst[l].push_back(ids[j]);
            ++next[l];
        }
    }
    c.boxes = prefix[nids];
    std::vector<int4> tiles;
    int halo_rows = 0;
    std::vector<int> tws(kMaxL + 1, 0), ths(kMaxL + 1, 0);
    for (int l = 2; l <= maxL; ++l) {
        if (!nslot[l]) continue;
        const int G = 1 << (l - 1);
        choose_tile(G, &tws[l], &ths[l], tile_policy);
        halo_rows = std::max(halo_rows, halo_rows_of(tws[l], ths[l]));
        for (int sl = 0; sl < nslot[l]; ++sl) {
            const BatchInst& in = host_inst[slot_inst[l][sl]];
            const int64_t le_off = in.exp_off + in.g.level_base[l] * 2 * P;
            for (int y = 0; y < G; y += ths[l])
                for (int x = 0; x < G; x += tws[l]) {
                    tiles.push_back(make_int4(l, x, y, tws[l] | (ths[l] << 8)));
                    tiles.push_back(make_int4(sl, (int)(uint32_t)le_off,
                                              (int)(uint32_t)(le_off >> 32), in.g.p));
                }
        }
    }
    c.cfg.ntiles = (int)(tiles.size() / 2);
    finish_config(&c.cfg, halo_rows, b_stages);
    if (c.cfg.b_stages < 2) return cudaErrorInvalidValue;
    auto a256 = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const size_t sz[] = {a256(tiles.size() * sizeof(int4)), a256((size_t)total4 * 16),
                         a256((size_t)total4 * 16), a256((size_t)c.cfg.b_floats * 4),
                         a256(4 * (size_t)nids), a256(8 * (size_t)(nids + 1)),
                         a256(dst.size() * 8)};
    size_t bytes = 0;
    for (size_t v : sz) bytes += v;
    cudaError_t e = cudaMalloc(&c.ws, bytes);
    if (e != cudaSuccess) return e;
    char* q = static_cast<char*>(c.ws);
    c.tiles = (int4*)q;
    q += sz[0];
    c.hi = (float*)q;
    q += sz[1];
    c.lo = (float*)q;
    q += sz[2];
    c.bimg = (float*)q;
    q += sz[3];
    c.inst = (int32_t*)q;
    q += sz[4];
    c.box_prefix = (int64_t*)q;
    q += sz[5];
    c.dst_base = (int64_t*)q;
    e = cudaMemcpyAsync(c.tiles, tiles.data(), tiles.size() * sizeof(int4),
                        cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c.inst, ids, 4 * (size_t)nids, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c.box_prefix, prefix.data(), 8 * (size_t)(nids + 1),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c.dst_base, dst.data(), dst.size() * 8, cudaMemcpyHostToDevice, s);
    c.maps = new M2LTcMaps();
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int l = 2; l <= maxL && e == cudaSuccess; ++l) {
        if (!nslot[l]) continue;
        const cuuint64_t G = 1ull << (l - 1);
        const cuuint64_t dims[4] = {4 * G, G, (cuuint64_t)4 * KG, (cuuint64_t)nslot[l]};
        const cuuint64_t strides[3] = {16 * G, 16 * G * G, 16 * G * G * 4 * KG};
        const cuuint32_t box[4] = {(cuuint32_t)(4 * (tws[l] + 2)), (cuuint32_t)(ths[l] + 2), 2,
                                   1};
        for (int which = 0; which < 2 && e == cudaSuccess; ++which) {
            float* base = (which ? c.lo : c.hi) + lvl[l] * 4;
            CUresult r = enc(which ? &c.maps->me_lo[l] : &c.maps->me_hi[l],
                             CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) e = cudaErrorInvalidValue;
        }
    }
    if (e == cudaSuccess) {
        const int64_t entries = c.cfg.b_floats / 2;
        const int blocks = (int)std::min<int64_t>((entries + 255) / 256, 8192);
        // the full operator (p = Pk): coefficients from the instance's p up
        // are zero in its multipoles and masked in its local expansions
        m2l_tc_bimg_kernel<<<blocks, 256, 0, s>>>(m2l64, P, Pk, Pk, c.bimg);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        m2l_tc_batch_destroy(&c);
        return e;
    }
    *out = c;
    return cudaSuccess;
}

void m2l_tc_batch_destroy(M2LTcBatchClass* c) {
    if (c->ws) cudaFree(c->ws);
    delete c->maps;
    *c = M2LTcBatchClass();
}

cudaError_t launch_m2l_tc_batch(const M2LTcBatchClass& c, const BatchInst* d_inst,
                                const float* me, float* le, int* status, uint32_t spin,
                                cudaStream_t s) {
    if (c.count == 0 || c.cfg.ntiles == 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>((c.boxes + 255) / 256, 4096);
    m2l_tc_split_batch_kernel<<<blocks, 256, 0, s>>>(d_inst, c.inst, c.box_prefix, c.dst_base,
                                                      c.count, c.boxes, c.Pk, me,
                                                      reinterpret_cast<float4*>(c.hi),
                                                      reinterpret_cast<float4*>(c.lo));
    M2LTcArgs a{};
    a.tiles = c.tiles;
    a.bimg = c.bimg;
    a.le = le;
    a.status = status;
    a.P = c.P;
    a.halo_bytes = c.cfg.halo_bytes;
    a.b_stages = c.cfg.b_stages;
    a.spin = spin ? spin : kSpinDefault;
    switch (c.Pk / 4) {
        case 1: return launch_pk<1>(c.cfg, *c.maps, a, s);
        case 2: return launch_pk<2>(c.cfg, *c.maps, a, s);
        case 3: return launch_pk<3>(c.cfg, *c.maps, a, s);
        case 4: return launch_pk<4>(c.cfg, *c.maps, a, s);
        case 5: return launch_pk<5>(c.cfg, *c.maps, a, s);
        case 6: return launch_pk<6>(c.cfg, *c.maps, a, s);
        case 7: return launch_pk<7>(c.cfg, *c.maps, a, s);
        case 8: return launch_pk<8>(c.cfg, *c.maps, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fmm2d
