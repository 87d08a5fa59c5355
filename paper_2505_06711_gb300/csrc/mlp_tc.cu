// Per-element atomic networks on the 5th-generation tensor cores (tcgen05),
// BF16 (or split BF16, or FP8 E4M3: see the FP8 section below) operands, FP32
// accumulation in tensor memory (TMEM).
//
// Sec. 2.1, Eq. 2: c^{t+1}_i = M^t_{Z_i}(rho^t_i), 48 -> 64 -> 64 -> 8, and the
// energy network 48 -> 64 -> 64 -> 1, SiLU between layers; the reverse pass
// (Eqs. 4-5) needs rhobar = J^T ybar only (a vector-Jacobian product).
//
// One CTA of 128 threads takes a tile of 128 consecutive atoms of one element
// (atoms are stored element-major).  Per layer, thread 0 issues
// tcgen05.mma.cta_group::1.kind::f16 (M = 128, K = 16 per instruction) with A
// (activations) and B (weights, N x K) in shared memory in the K-major
// no-swizzle core-matrix layout and D in TMEM; tcgen05.commit arrives on an
// mbarrier that all threads wait on.  Thread r then reads TMEM lane r
// (tcgen05.ld 32x32b), applies bias and SiLU (or its derivative) in FP32,
// rounds to BF16 and writes the next layer's A tile.  Weight images are laid
// out once on the host in the same core-matrix layout and copied to shared
// memory with bulk asynchronous copies (cp.async.bulk, TMA engine).  The BF16
// forward keeps SiLU'(z1), SiLU'(z2) of every row for the backward, which then
// needs three products and the backward weight image only.
//
// Two precisions share the kernels:
//   plain BF16 (SPLIT = false): one MMA per K step, BF16 operands;
//   split BF16 (SPLIT = true): every operand is a BF16 pair x = hi + lo and
//     each K step issues hi*hi + hi*lo + lo*hi, still BF16 tensor-core MMAs
//     with FP32 accumulation but with ~16 significant bits per operand.  In a
//     crystal every atom feeds the networks nearly the same inputs, so plain
//     BF16 rounding shifts every atomic energy the same way; the split form
//     removes that shift.
//
// Core-matrix layout of an R x K BF16 tile: 8 x 8 blocks of 128 contiguous
// bytes (8 rows of 16 bytes); block (r/8, k/8) at byte (r/8 * K/8 + k/8) * 128.
// Descriptor: LBO = 128 B (next block along K), SBO = 16 K bytes (next 8-row
// group).
//
// Every wait is bounded: after kSpinLimit polls a CTA records FLAG_TIMEOUT in
// the context flags, waits (bounded) until every MMA it issued and its weight
// copy have completed, frees its TMEM and returns (reann_ctx_check reports
// REANN_E_TIMEOUT).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"

namespace reann {
namespace {

constexpr int kThreads = 128;
constexpr int kRows = 128;
constexpr uint32_t kTmemCols = 256;
constexpr long long kSpinLimit = 1ll << 26;

// ------------------------------------------------------------- PTX glue ---
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// K-major, no swizzle, sm_100-family descriptor (version field = 1 at bit 46)
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;  // base offset 0, relative LBO, layout type 0 (no swizzle)
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
    return (1u << 4)                      // D format F32
           | (1u << 7)                    // A format BF16
           | (1u << 10)                   // B format BF16
           | ((uint32_t)(N >> 3) << 17)   // N / 8
           | ((uint32_t)(M >> 4) << 24);  // M / 16
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes)
                 : "memory");
}

// bounded wait for phase `parity`; returns false when `limit` polls ran out
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, long long limit = kSpinLimit) {
    const uint32_t a = smem_addr(mbar);
    for (long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// global -> shared bulk copy (TMA engine), completion counted on the mbarrier
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(mbar))
        : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float silu(float z) { return z / (1.f + expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
    const float s = 1.f / (1.f + expf(-z));
    return s * (1.f + z * (1.f - s));
}

// Write 8 values (k = 8 kc .. 8 kc + 7) of row r into a core-matrix tile with K
// columns: the BF16 rounding into `hi` and, when `lo` is given, the BF16
// rounding of the remainder into `lo` (so that hi + lo carries ~16 bits).
__device__ __forceinline__ void put8(uint8_t* hi, uint8_t* lo, int K, int r, int kc, const float* v) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * p], v[2 * p + 1]);
        h[p] = *reinterpret_cast<const uint32_t*>(&b);
        if (lo) {
            const float2 f = __bfloat1622float2(b);
            const __nv_bfloat162 c = __floats2bfloat162_rn(v[2 * p] - f.x, v[2 * p + 1] - f.y);
            l[p] = *reinterpret_cast<const uint32_t*>(&c);
        }
    }
    const size_t off = (size_t)((r >> 3) * (K >> 3) + kc) * 128 + (r & 7) * 16;
    *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    if (lo) *reinterpret_cast<uint4*>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// 16 KiB weight images per (layer, element), laid out by the host:
//   forward  (W1^T 64x48 | W2^T 64x64 | W3^T 16x64), backward (W3 64x16 | W2 64x64 | W1 48x64);
// in memory: forward hi | forward lo | backward hi | backward lo (lo = BF16 remainder).
constexpr uint32_t kImg = 16384;
constexpr uint32_t kF_W1t = 0, kF_W2t = 6144, kF_W3t = 14336;
constexpr uint32_t kB_W3p = 0, kB_W2 = 2048, kB_W1 = 10240;

// shared-memory layouts (bytes); lo tiles exist only in the split form
template <bool SPLIT>
struct FwdSmem {
    static constexpr uint32_t S = SPLIT ? 2 : 1;
    static constexpr uint32_t W = 0, A = kImg * S, H = A + 12288 * S, BAR = H + 16384 * S;
    static constexpr uint32_t WLO = W + kImg, ALO = A + 12288, HLO = H + 16384;
    static constexpr int BYTES = BAR + 64;
    static constexpr int REQUEST = 110 * 1024;  // > 1/3 of an SM's shared memory: at most 2 CTAs (2 x 256 TMEM columns)
};
template <bool SPLIT>
struct BwdSmem {
    static constexpr uint32_t S = SPLIT ? 2 : 1;
    static constexpr uint32_t WF = 0, WB = kImg * S, A = 2 * kImg * S, H = A + 12288 * S, Y = H + 16384 * S,
                              BAR = Y + 4096 * S;
    static constexpr uint32_t WFLO = WF + kImg, WBLO = WB + kImg, ALO = A + 12288, HLO = H + 16384, YLO = Y + 4096;
    static constexpr int BYTES = BAR + 64;
    static constexpr int REQUEST = SPLIT ? 132 * 1024 : 110 * 1024;  // split: one CTA per SM
};
static_assert(FwdSmem<true>::BYTES <= FwdSmem<true>::REQUEST, "forward shared memory");
static_assert(BwdSmem<true>::BYTES <= BwdSmem<true>::REQUEST, "backward shared memory");

struct TcNet {
    const uint8_t* img;  // forward hi | forward lo | backward hi | backward lo
    const float *b1, *b2, *b3;
    const uint8_t* img8;  // FP8: forward | backward
    const float* s8;      // FP8: s(W1), s(W2), s(W3)
};
struct TcLayer {
    TcNet e[MAX_ELEM];
};

__device__ __forceinline__ uint32_t lane_addr(uint32_t tmem, int warp, int col) {
    return tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)col;
}

// uniform bounded wait: every thread polls; the CTA agrees on the outcome
__device__ __forceinline__ bool wait_all(uint64_t* bar, uint32_t parity, long long limit = kSpinLimit) {
    const bool ok = mbar_wait(bar, parity, limit);
    return __syncthreads_and(ok);
}

// After a wait ran out (bar[0]: the weight copy, bar[1]: MMA completion, bar[2]:
// spare): record FLAG_TIMEOUT, then make sure nothing this CTA started is still in
// flight before the caller releases its TMEM and shared memory.  Thread 0 commits
// every tcgen05 operation it issued to the spare barrier (it arrives once all of
// them completed, at once when there were none); when the weight copy was not seen
// to land, its barrier is waited for again.  Both waits are bounded; if either runs
// out as well, FLAG_TIMEOUT_DRAIN is recorded too (the CTA still frees its TMEM and
// returns, and the host reports that the device state is suspect).
__device__ __forceinline__ void fail(int* flags, uint64_t* bar, bool weights_landed) {
    if (threadIdx.x == 0) {
        atomicOr(&flags[FLAG_TIMEOUT], 1);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_addr(&bar[2]))
                     : "memory");
    }
    bool drained = mbar_wait(&bar[2], 0);
    if (!weights_landed) drained = mbar_wait(&bar[0], 0) && drained;
    if (!__syncthreads_and(drained) && threadIdx.x == 0) atomicOr(&flags[FLAG_TIMEOUT_DRAIN], 1);
}

// rows [row0, row0 + nrows) of a row-major FP32 [.][48] array -> BF16 core-matrix tile(s) (K = 48)
__device__ __forceinline__ void load_x_tile(uint8_t* hi, uint8_t* lo, const float* __restrict__ x, const Tile& tl,
                                            int r) {
#pragma unroll
    for (int kc = 0; kc < NFEAT / 8; ++kc) {
        float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (r < tl.nrows) {
            const float4 a = *reinterpret_cast<const float4*>(x + (size_t)(tl.row0 + r) * NFEAT + 8 * kc);
            const float4 b = *reinterpret_cast<const float4*>(x + (size_t)(tl.row0 + r) * NFEAT + 8 * kc + 4);
            v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
        }
        put8(hi, lo, NFEAT, r, kc, v);
    }
}

// D[cols] (+)= A (K = 16 ks_count) x B^T for one 128-row tile; split form adds hi*lo + lo*hi
template <bool SPLIT>
__device__ __forceinline__ void issue(uint32_t tmem_d, const uint8_t* A, const uint8_t* Alo, int KA,
                                      const uint8_t* B, const uint8_t* Blo, int N, int ks_count) {
    const uint32_t idesc = make_idesc(kRows, N);
    const uint32_t a0 = smem_addr(A), b0 = smem_addr(B);
    const uint32_t a1 = SPLIT ? smem_addr(Alo) : 0u, b1 = SPLIT ? smem_addr(Blo) : 0u;
    for (int ks = 0; ks < ks_count; ++ks) {
        const uint64_t ah = make_desc(a0 + ks * 256, 128, 16 * KA), bh = make_desc(b0 + ks * 256, 128, 16 * KA);
        mma_bf16(tmem_d, ah, bh, idesc, ks > 0 ? 1u : 0u);
        if (SPLIT) {
            mma_bf16(tmem_d, ah, make_desc(b1 + ks * 256, 128, 16 * KA), idesc, 1u);
            mma_bf16(tmem_d, make_desc(a1 + ks * 256, 128, 16 * KA), bh, idesc, 1u);
        }
    }
}

// between "threads wrote shared memory / read TMEM" and "thread 0 issues MMAs"
__device__ __forceinline__ void handoff() {
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

__device__ __forceinline__ uint32_t setup(uint32_t* tslot, uint64_t* bar) {
    if ((threadIdx.x >> 5) == 0) tmem_alloc(tslot, kTmemCols);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return *tslot;
}

__device__ __forceinline__ void teardown(uint32_t tmem) {
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) tmem_dealloc(tmem, kTmemCols);
}

// TMEM columns [c, c + 64) of this lane -> act(v + bias) -> row r of an A tile (K = 64);
// with dsave (the row's 64 values for this layer), SiLU'(v + bias) is kept there for the
// reverse pass
template <bool SPLIT>
__device__ __forceinline__ void silu_to_tile(uint32_t tmem, int warp, int c, const float* __restrict__ bias,
                                             uint8_t* hi, uint8_t* lo, int r, float* __restrict__ dsave = nullptr) {
    float v[16], h[16];
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 16) {
        tmem_ld16(lane_addr(tmem, warp, c + c0), v);
#pragma unroll
        for (int i = 0; i < 16; ++i) h[i] = silu(v[i] + bias[c0 + i]);
        put8(hi, SPLIT ? lo : nullptr, 64, r, c0 / 8, h);
        put8(hi, SPLIT ? lo : nullptr, 64, r, c0 / 8 + 1, h + 8);
        if (dsave) {
#pragma unroll
            for (int i = 0; i < 16; ++i) h[i] = dsilu(v[i] + bias[c0 + i]);
            float4* d = reinterpret_cast<float4*>(dsave + c0);
#pragma unroll
            for (int q = 0; q < 4; ++q) d[q] = make_float4(h[4 * q], h[4 * q + 1], h[4 * q + 2], h[4 * q + 3]);
        }
    }
}

// g (columns [cg, cg + 64)) * silu'(z + bias) (z in columns [cz, cz + 64)) -> row r of an A tile
template <bool SPLIT>
__device__ __forceinline__ void dsilu_to_tile(uint32_t tmem, int warp, int cg, int cz, const float* __restrict__ bias,
                                              uint8_t* hi, uint8_t* lo, int r) {
    float g[16], z[16], h[16];
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 16) {
        tmem_ld16(lane_addr(tmem, warp, cg + c0), g);
        tmem_ld16(lane_addr(tmem, warp, cz + c0), z);
#pragma unroll
        for (int i = 0; i < 16; ++i) h[i] = g[i] * dsilu(z[i] + bias[c0 + i]);
        put8(hi, SPLIT ? lo : nullptr, 64, r, c0 / 8, h);
        put8(hi, SPLIT ? lo : nullptr, 64, r, c0 / 8 + 1, h + 8);
    }
}

// 64 saved SiLU' values of a row into registers (zeros for rows past the tile's
// end); issued a stage ahead so that the loads overlap the previous product
__device__ __forceinline__ void load64(const float* __restrict__ p, float* d) {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const float4 x = p ? __ldg(reinterpret_cast<const float4*>(p) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        d[4 * q] = x.x, d[4 * q + 1] = x.y, d[4 * q + 2] = x.z, d[4 * q + 3] = x.w;
    }
}

// g (TMEM columns [cg, cg + 64)) * the row's saved SiLU' values sd -> row r of an A tile
template <bool SPLIT>
__device__ __forceinline__ void scale_to_tile(uint32_t tmem, int warp, int cg, const float* sd, uint8_t* hi,
                                              uint8_t* lo, int r) {
    float g[16], h[16];
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 16) {
        tmem_ld16(lane_addr(tmem, warp, cg + c0), g);
#pragma unroll
        for (int i = 0; i < 16; ++i) h[i] = g[i] * sd[c0 + i];
        put8(hi, SPLIT ? lo : nullptr, 64, r, c0 / 8, h);
        put8(hi, SPLIT ? lo : nullptr, 64, r, c0 / 8 + 1, h + 8);
    }
}

// forward: TMEM columns [0,64) z1, [64,128) z2, [128,144) y.  With dsave, row i's
// SiLU'(z1), SiLU'(z2) go to dsave[i][0..63], dsave[i][64..127] for the reverse pass.
template <int OUT, bool SPLIT>
__global__ void __launch_bounds__(kThreads, 1) k_mlp_tc_fwd(TcLayer nets, const Tile* __restrict__ tiles,
                                                           const float* __restrict__ rho, float* __restrict__ out,
                                                           int out_stride, int* __restrict__ flags, GhostOut gh,
                                                           float* __restrict__ dsave) {
    using L = FwdSmem<SPLIT>;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::BAR);  // [0] weights, [1] MMA
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 3);
    const int tid = threadIdx.x, warp = tid >> 5, r = tid;
    const Tile tl = tiles[blockIdx.x];
    if (tl.nrows <= 0) return;  // padding entry of a fixed-size tile list (before any TMEM allocation)
    const TcNet& w = nets.e[tl.elem];
    float* drow = dsave && r < tl.nrows ? dsave + (size_t)(tl.row0 + r) * (H1 + H2) : nullptr;
    const uint32_t tmem = setup(tslot, bar);
    if (tid == 0) {
        mbar_expect_tx(&bar[0], kImg * L::S);
        bulk_g2s(smem + L::W, w.img, kImg * L::S, &bar[0]);  // forward hi (| lo)
    }
    load_x_tile(smem + L::A, SPLIT ? smem + L::ALO : nullptr, rho, tl, r);
    handoff();
    bool ok = wait_all(&bar[0], 0);
    if (!ok) {
        fail(flags, bar, false);
    } else {
        if (tid == 0) {  // z1 = x W1
            issue<SPLIT>(tmem, smem + L::A, smem + L::ALO, NFEAT, smem + L::W + kF_W1t, smem + L::WLO + kF_W1t, H1,
                         NFEAT / 16);
            mma_commit(&bar[1]);
        }
        ok = wait_all(&bar[1], 0);
        if (!ok) fail(flags, bar, true);
    }
    if (ok) {
        tc_fence_after();
        silu_to_tile<SPLIT>(tmem, warp, 0, w.b1, smem + L::H, smem + L::HLO, r, drow);
        handoff();
        if (tid == 0) {  // z2 = h1 W2
            issue<SPLIT>(tmem + 64, smem + L::H, smem + L::HLO, H1, smem + L::W + kF_W2t, smem + L::WLO + kF_W2t, H2,
                         H1 / 16);
            mma_commit(&bar[1]);
        }
        ok = wait_all(&bar[1], 1);
        if (!ok) fail(flags, bar, true);
    }
    if (ok) {
        tc_fence_after();
        silu_to_tile<SPLIT>(tmem, warp, 64, w.b2, smem + L::H, smem + L::HLO, r, drow ? drow + H1 : nullptr);
        handoff();
        if (tid == 0) {  // y = h2 W3 (N padded to 16)
            issue<SPLIT>(tmem + 128, smem + L::H, smem + L::HLO, H2, smem + L::W + kF_W3t, smem + L::WLO + kF_W3t, 16,
                         H2 / 16);
            mma_commit(&bar[1]);
        }
        ok = wait_all(&bar[1], 0);
        if (!ok) fail(flags, bar, true);
    }
    if (ok) {
        tc_fence_after();
        float v[16];
        tmem_ld16(lane_addr(tmem, warp, 128), v);
        if (r < tl.nrows) {
            const int64_t row = tl.row0 + r;
            float* o = out + (size_t)row * out_stride;
#pragma unroll
            for (int i = 0; i < OUT; ++i) o[i] = v[i] + w.b3[i];
            if (OUT > 1 && gh.goff)  // the row's ghost images get the same coefficients
                for (int64_t g = gh.goff[row]; g < gh.goff[row + 1] && g < gh.gcap; ++g) {
                    float* go = out + (size_t)(gh.base + g) * out_stride;
#pragma unroll
                    for (int i = 0; i < OUT; ++i) go[i] = v[i] + w.b3[i];
                }
        }
    }
    teardown(tmem);
}

// rhobar = J^T ybar with SiLU'(z1), SiLU'(z2) saved by the forward (dsave, 128
// floats per row): three products, nothing recomputed, only the backward weight
// image staged.  TMEM columns: [128,192) ybar W3^T then rhobar (48), [192,256)
// z2bar W2^T.
template <int OUT, bool SPLIT>
__global__ void __launch_bounds__(kThreads, 1) k_mlp_tc_bwd(TcLayer nets, const Tile* __restrict__ tiles,
                                                           const float* __restrict__ dsave,
                                                           const float* __restrict__ ybar,
                                                           float* __restrict__ rhobar, int* __restrict__ flags) {
    using L = BwdSmem<SPLIT>;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 3);
    const int tid = threadIdx.x, warp = tid >> 5, r = tid;
    const Tile tl = tiles[blockIdx.x];
    if (tl.nrows <= 0) return;  // padding entry of a fixed-size tile list (before any TMEM allocation)
    const TcNet& w = nets.e[tl.elem];
    const float* drow = r < tl.nrows ? dsave + (size_t)(tl.row0 + r) * (H1 + H2) : nullptr;
    const uint32_t tmem = setup(tslot, bar);
    if (tid == 0) {
        mbar_expect_tx(&bar[0], kImg * L::S);
        bulk_g2s(smem + L::WB, w.img + 2 * kImg, kImg * L::S, &bar[0]);  // backward hi (| lo)
    }
    {
        float y[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) y[i] = 0.f;
        if (r < tl.nrows) {
            if (OUT == 1)
                y[0] = 1.f;  // d eps_i / d eps_i
            else
#pragma unroll
                for (int i = 0; i < OUT; ++i) y[i] = ybar[(size_t)(tl.row0 + r) * OUT + i];
        }
        put8(smem + L::Y, SPLIT ? smem + L::YLO : nullptr, 16, r, 0, y);
        put8(smem + L::Y, SPLIT ? smem + L::YLO : nullptr, 16, r, 1, y + 8);
    }
    float sd[64];
    load64(drow ? drow + H1 : nullptr, sd);  // SiLU'(z2)
    handoff();
    bool ok = wait_all(&bar[0], 0);
    if (!ok) {
        fail(flags, bar, false);
    } else {
        if (tid == 0) {  // ybar W3^T
            issue<SPLIT>(tmem + 128, smem + L::Y, smem + L::YLO, 16, smem + L::WB + kB_W3p, smem + L::WBLO + kB_W3p,
                         H2, 1);
            mma_commit(&bar[1]);
        }
        ok = wait_all(&bar[1], 0);
        if (!ok) fail(flags, bar, true);
    }
    if (ok) {
        tc_fence_after();
        scale_to_tile<SPLIT>(tmem, warp, 128, sd, smem + L::H, smem + L::HLO, r);  // z2bar
        handoff();
        if (tid == 0) {  // z2bar W2^T
            issue<SPLIT>(tmem + 192, smem + L::H, smem + L::HLO, H2, smem + L::WB + kB_W2, smem + L::WBLO + kB_W2, H1,
                         H2 / 16);
            mma_commit(&bar[1]);
        }
        load64(drow, sd);  // SiLU'(z1), while the product runs
        ok = wait_all(&bar[1], 1);
        if (!ok) fail(flags, bar, true);
    }
    if (ok) {
        tc_fence_after();
        scale_to_tile<SPLIT>(tmem, warp, 192, sd, smem + L::H, smem + L::HLO, r);  // z1bar
        handoff();
        if (tid == 0) {  // rhobar = z1bar W1^T
            issue<SPLIT>(tmem + 128, smem + L::H, smem + L::HLO, H1, smem + L::WB + kB_W1, smem + L::WBLO + kB_W1,
                         NFEAT, H1 / 16);
            mma_commit(&bar[1]);
        }
        ok = wait_all(&bar[1], 0);
        if (!ok) fail(flags, bar, true);
    }
    if (ok) {
        tc_fence_after();
        float v[16];
#pragma unroll
        for (int c0 = 0; c0 < NFEAT; c0 += 16) {
            tmem_ld16(lane_addr(tmem, warp, 128 + c0), v);
            if (r < tl.nrows) {
                float4* dst = reinterpret_cast<float4*>(rhobar + (size_t)(tl.row0 + r) * NFEAT + c0);
#pragma unroll
                for (int q = 0; q < 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
        }
    }
    teardown(tmem);
}

// ------------------------------------------------------------------ FP8 ---
// E4M3 operands (tcgen05.mma kind::f8f6f4, K = 32 per instruction), FP32
// accumulation in TMEM.  Weights are E4M3 images of W / s(W), one scale per
// matrix (host-built); each 128-row activation tile is divided by its own
// scale s = max |x| / 448 (a block-wide maximum) before rounding to E4M3
// (cvt.rn.satfinite), and the accumulator is multiplied back by s(tile) s(W).
// 8-bit core-matrix layout: 8 x 16 blocks of 128 bytes, block (r/8, k/16) at
// (r/8 * K/16 + k/16) * 128; descriptor LBO = 128 B, SBO = 8 K bytes.
constexpr uint32_t kF8_W1t = 0, kF8_W2t = 4096, kF8_W3t = 8192;  // forward image
constexpr uint32_t kF8_W3 = 0, kF8_W2 = 2048, kF8_W1 = 6144;     // backward image

// kind::f8f6f4 instruction descriptor: D = F32, A = B = E4M3 (format 0), both K-major
__host__ __device__ constexpr uint32_t make_idesc_e4m3(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_e4m3(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// D[cols] = A (K = 32 ks_count) x B^T (B: N x K), E4M3 tiles with K = KA columns
__device__ __forceinline__ void issue8(uint32_t tmem_d, const uint8_t* A, int KA, const uint8_t* B, int N,
                                       int ks_count) {
    const uint32_t idesc = make_idesc_e4m3(kRows, N);
    const uint32_t a0 = smem_addr(A), b0 = smem_addr(B);
    for (int ks = 0; ks < ks_count; ++ks)
        mma_e4m3(tmem_d, make_desc(a0 + ks * 256, 128, 8 * KA), make_desc(b0 + ks * 256, 128, 8 * KA), idesc,
                 ks > 0 ? 1u : 0u);
}

// max over the CTA's 128 threads (every thread calls it)
__device__ __forceinline__ float block_max(float m, float* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    const float r = fmaxf(fmaxf(red[0], red[1]), fmaxf(red[2], red[3]));
    __syncthreads();  // red is reused by the next call
    return r;
}

// the tile's scale (max |x| maps to 448, the largest finite E4M3 value)
__device__ __forceinline__ float tile_scale(float amax) { return amax > 0.f ? amax / 448.f : 1.f; }

// row r (K values, already divided by the tile's scale) -> E4M3 core-matrix tile with K columns
template <int K>
__device__ __forceinline__ void put_row_e4m3(uint8_t* tile, int r, const float* v) {
#pragma unroll
    for (int kc = 0; kc < K / 16; ++kc) {
        uint32_t w[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            uint16_t lo, hi;  // cvt puts its first source in the upper byte
            asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(lo) : "f"(v[16 * kc + 4 * p + 1]), "f"(v[16 * kc + 4 * p]));
            asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;"
                : "=h"(hi)
                : "f"(v[16 * kc + 4 * p + 3]), "f"(v[16 * kc + 4 * p + 2]));
            w[p] = (uint32_t)lo | ((uint32_t)hi << 16);
        }
        *reinterpret_cast<uint4*>(tile + ((size_t)((r >> 3) * (K / 16) + kc) * 128 + (r & 7) * 16)) =
            make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// scale the rows of a tile by the tile's max, write them as E4M3; returns the scale
template <int K>
__device__ __forceinline__ float quantize_rows(uint8_t* tile, int r, float* v, float* red) {
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) m = fmaxf(m, fabsf(v[k]));
    const float s = tile_scale(block_max(m, red)), inv = 1.f / s;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] *= inv;
    put_row_e4m3<K>(tile, r, v);
    return s;
}

// 64 TMEM columns [c, c + 64) of this lane, times `scale`
__device__ __forceinline__ void tmem_row64(uint32_t tmem, int warp, int c, float scale, float* v) {
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 16) {
        tmem_ld16(lane_addr(tmem, warp, c + c0), v + c0);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[c0 + i] *= scale;
    }
}

struct F8Fwd {  // shared memory (bytes)
    static constexpr uint32_t W = 0, A = kF8Fwd, H = A + 128 * 64, RED = H + 128 * 64, BAR = RED + 64;
    static constexpr int BYTES = BAR + 64;
    static constexpr int REQUEST = 110 * 1024;  // at most 2 CTAs (2 x 256 TMEM columns) per SM
};
struct F8Bwd {
    static constexpr uint32_t WF = 0, WB = kF8Fwd, A = kF8Img, H = A + 128 * 64, Y = H + 128 * 64,
                              RED = Y + 128 * 32, BAR = RED + 64;
    static constexpr int BYTES = BAR + 64;
    static constexpr int REQUEST = 110 * 1024;
};
static_assert(F8Fwd::BYTES <= F8Fwd::REQUEST && F8Bwd::BYTES <= F8Bwd::REQUEST, "FP8 shared memory");
static_assert(kF8Fwd % 128 == 0 && kF8Img % 128 == 0, "FP8 tiles stay 128 B aligned");

// rows [row0, row0 + nrows) of a row-major FP32 [.][48] array, zero-padded to 64 columns
__device__ __forceinline__ void load_x_row64(const float* __restrict__ x, const Tile& tl, int r, float* v) {
#pragma unroll
    for (int k = 0; k < 64; ++k) v[k] = 0.f;
    if (r < tl.nrows) {
#pragma unroll
        for (int k = 0; k < NFEAT; k += 4) {
            const float4 a = *reinterpret_cast<const float4*>(x + (size_t)(tl.row0 + r) * NFEAT + k);
            v[k] = a.x, v[k + 1] = a.y, v[k + 2] = a.z, v[k + 3] = a.w;
        }
    }
}

// forward: TMEM columns [0,64) z1, [64,128) z2, [128,144) y
template <int OUT>
__global__ void __launch_bounds__(kThreads, 1) k_mlp_f8_fwd(TcLayer nets, const Tile* __restrict__ tiles,
                                                           const float* __restrict__ rho, float* __restrict__ out,
                                                           int out_stride, int* __restrict__ flags, GhostOut gh) {
    using L = F8Fwd;
    extern __shared__ __align__(1024) uint8_t smem[];
    float* red = reinterpret_cast<float*>(smem + L::RED);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::BAR);  // [0] weights, [1] MMA
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 3);
    const int tid = threadIdx.x, warp = tid >> 5, r = tid;
    const Tile tl = tiles[blockIdx.x];
    if (tl.nrows <= 0) return;  // padding entry of a fixed-size tile list (before any TMEM allocation)
    const TcNet& w = nets.e[tl.elem];
    const uint32_t tmem = setup(tslot, bar);
    if (tid == 0) {
        mbar_expect_tx(&bar[0], kF8Fwd);
        bulk_g2s(smem + L::W, w.img8, kF8Fwd, &bar[0]);
    }
    const float sw1 = w.s8[0], sw2 = w.s8[1], sw3 = w.s8[2];
    float v[64];
    load_x_row64(rho, tl, r, v);
    const float sx = quantize_rows<64>(smem + L::A, r, v, red);
    handoff();
    bool ok = wait_all(&bar[0], 0);
    float sh = 1.f;
    if (!ok) {
        fail(flags, bar, false);
    } else {
        if (tid == 0) {  // z1 = x W1
            issue8(tmem, smem + L::A, 64, smem + L::W + kF8_W1t, H1, 2);
            mma_commit(&bar[1]);
        }
        ok = wait_all(&bar[1], 0);
        if (!ok) fail(flags, bar, true);
    }
    if (ok) {
        tc_fence_after();
        tmem_row64(tmem, warp, 0, sx * sw1, v);
#pragma unroll
        for (int i = 0; i < 64; ++i) v[i] = silu(v[i] + w.b1[i]);
        sh = quantize_rows<64>(smem + L::H, r, v, red);
        handoff();
        if (tid == 0) {  // z2 = h1 W2
            issue8(tmem + 64, smem + L::H, 64, smem + L::W + kF8_W2t, H2, 2);
            mma_commit(&bar[1]);
        }
        ok = wait_all(&bar[1], 1);
        if (!ok) fail(flags, bar, true);
    }
    if (ok) {
        tc_fence_after();
        tmem_row64(tmem, warp, 64, sh * sw2, v);
#pragma unroll
        for (int i = 0; i < 64; ++i) v[i] = silu(v[i] + w.b2[i]);
        sh = quantize_rows<64>(smem + L::H, r, v, red);
        handoff();
        if (tid == 0) {  // y = h2 W3 (N padded to 16)
            issue8(tmem + 128, smem + L::H, 64, smem + L::W + kF8_W3t, 16, 2);
            mma_commit(&bar[1]);
        }
        ok = wait_all(&bar[1], 0);
        if (!ok) fail(flags, bar, true);
    }
    if (ok) {
        tc_fence_after();
        float y[16];
        tmem_ld16(lane_addr(tmem, warp, 128), y);
        if (r < tl.nrows) {
            const int64_t row = tl.row0 + r;
            float* o = out + (size_t)row * out_stride;
#pragma unroll
            for (int i = 0; i < OUT; ++i) o[i] = y[i] * (sh * sw3) + w.b3[i];
            if (OUT > 1 && gh.goff)  // the row's ghost images get the same coefficients
                for (int64_t g = gh.goff[row]; g < gh.goff[row + 1] && g < gh.gcap; ++g) {
                    float* go = out + (size_t)(gh.base + g) * out_stride;
#pragma unroll
                    for (int i = 0; i < OUT; ++i) go[i] = y[i] * (sh * sw3) + w.b3[i];
                }
        }
    }
    teardown(tmem);
}

// rhobar = J^T ybar, recomputing z1, z2.  TMEM columns: [0,64) z1, [64,128) z2,
// [128,192) ybar W3^T then rhobar (48), [192,256) z2bar W2^T.
template <int OUT>
__global__ void __launch_bounds__(kThreads, 1) k_mlp_f8_bwd(TcLayer nets, const Tile* __restrict__ tiles,
                                                           const float* __restrict__ rho,
                                                           const float* __restrict__ ybar,
                                                           float* __restrict__ rhobar, int* __restrict__ flags) {
    using L = F8Bwd;
    extern __shared__ __align__(1024) uint8_t smem[];
    float* red = reinterpret_cast<float*>(smem + L::RED);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 3);
    const int tid = threadIdx.x, warp = tid >> 5, r = tid;
    const Tile tl = tiles[blockIdx.x];
    if (tl.nrows <= 0) return;  // padding entry of a fixed-size tile list (before any TMEM allocation)
    const TcNet& w = nets.e[tl.elem];
    const uint32_t tmem = setup(tslot, bar);
    if (tid == 0) {
        mbar_expect_tx(&bar[0], kF8Img);
        bulk_g2s(smem + L::WF, w.img8, kF8Img, &bar[0]);  // forward | backward
    }
    const float sw1 = w.s8[0], sw2 = w.s8[1], sw3 = w.s8[2];
    float v[64];
    load_x_row64(rho, tl, r, v);
    const float sx = quantize_rows<64>(smem + L::A, r, v, red);
    float y[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) y[i] = 0.f;
    if (r < tl.nrows) {
        if (OUT == 1)
            y[0] = 1.f;  // d eps_i / d eps_i
        else
#pragma unroll
            for (int i = 0; i < OUT; ++i) y[i] = ybar[(size_t)(tl.row0 + r) * OUT + i];
    }
    const float sy = quantize_rows<32>(smem + L::Y, r, y, red);
    handoff();
    float sh1 = 1.f, sg = 1.f;
    bool ok = wait_all(&bar[0], 0);
    if (!ok) {
        fail(flags, bar, false);
    } else {
        if (tid == 0) {
            issue8(tmem, smem + L::A, 64, smem + L::WF + kF8_W1t, H1, 2);         // z1
            issue8(tmem + 128, smem + L::Y, 32, smem + L::WB + kF8_W3, H2, 1);    // ybar W3^T
            mma_commit(&bar[1]);
        }
        ok = wait_all(&bar[1], 0);
        if (!ok) fail(flags, bar, true);
    }
    if (ok) {
        tc_fence_after();
        tmem_row64(tmem, warp, 0, sx * sw1, v);
#pragma unroll
        for (int i = 0; i < 64; ++i) v[i] = silu(v[i] + w.b1[i]);
        sh1 = quantize_rows<64>(smem + L::H, r, v, red);
        handoff();
        if (tid == 0) {  // z2
            issue8(tmem + 64, smem + L::H, 64, smem + L::WF + kF8_W2t, H2, 2);
            mma_commit(&bar[1]);
        }
        ok = wait_all(&bar[1], 1);
        if (!ok) fail(flags, bar, true);
    }
    if (ok) {
        tc_fence_after();
        float z[64];
        tmem_row64(tmem, warp, 128, sy * sw3, v);  // ybar W3^T
        tmem_row64(tmem, warp, 64, sh1 * sw2, z);  // z2 (without b2)
#pragma unroll
        for (int i = 0; i < 64; ++i) v[i] *= dsilu(z[i] + w.b2[i]);  // z2bar
        sg = quantize_rows<64>(smem + L::H, r, v, red);
        handoff();
        if (tid == 0) {  // z2bar W2^T
            issue8(tmem + 192, smem + L::H, 64, smem + L::WB + kF8_W2, H1, 2);
            mma_commit(&bar[1]);
        }
        ok = wait_all(&bar[1], 0);
        if (!ok) fail(flags, bar, true);
    }
    if (ok) {
        tc_fence_after();
        float z[64];
        tmem_row64(tmem, warp, 192, sg * sw2, v);  // z2bar W2^T
        tmem_row64(tmem, warp, 0, sx * sw1, z);    // z1 (without b1)
#pragma unroll
        for (int i = 0; i < 64; ++i) v[i] *= dsilu(z[i] + w.b1[i]);  // z1bar
        sg = quantize_rows<64>(smem + L::H, r, v, red);
        handoff();
        if (tid == 0) {  // rhobar = z1bar W1^T
            issue8(tmem + 128, smem + L::H, 64, smem + L::WB + kF8_W1, NFEAT, 2);
            mma_commit(&bar[1]);
        }
        ok = wait_all(&bar[1], 1);
        if (!ok) fail(flags, bar, true);
    }
    if (ok) {
        tc_fence_after();
        float g[16];
#pragma unroll
        for (int c0 = 0; c0 < NFEAT; c0 += 16) {
            tmem_ld16(lane_addr(tmem, warp, 128 + c0), g);
            if (r < tl.nrows) {
                float4* dst = reinterpret_cast<float4*>(rhobar + (size_t)(tl.row0 + r) * NFEAT + c0);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    dst[q] = make_float4(g[4 * q] * (sg * sw1), g[4 * q + 1] * (sg * sw1), g[4 * q + 2] * (sg * sw1),
                                         g[4 * q + 3] * (sg * sw1));
            }
        }
    }
    teardown(tmem);
}

// The bounded-wait exit with nothing in flight: allocate TMEM, wait `polls` times on
// an mbarrier that nothing arrives on, then fail() (flag, drain, release) as the
// network kernels do when a wait runs out.
__global__ void __launch_bounds__(kThreads, 1) k_wait_selftest(int* __restrict__ flags, long long polls) {
    __shared__ __align__(8) uint64_t bar[4];
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 3);
    const uint32_t tmem = setup(tslot, bar);
    if (!wait_all(&bar[1], 0, polls)) fail(flags, bar, true);
    teardown(tmem);
}

TcLayer layer_of(const TcTable& t, int layer) {
    TcLayer l;
    for (int e = 0; e < MAX_ELEM; ++e) {
        const TcImg& i = t.img[layer][e];
        l.e[e] = TcNet{i.img, i.b1, i.b2, i.b3, i.img8, i.s8};
    }
    return l;
}

template <int OUT, bool SPLIT>
void set_attrs() {
    cudaFuncSetAttribute(k_mlp_tc_fwd<OUT, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         FwdSmem<SPLIT>::REQUEST);
    cudaFuncSetAttribute(k_mlp_tc_bwd<OUT, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         BwdSmem<SPLIT>::REQUEST);
}

void ensure_tc_attrs() {
    // once per device, safe under concurrent first calls
    static std::mutex mu;
    static uint64_t done = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 64 && ((done >> dev) & 1)) return;
    set_attrs<1, false>();
    set_attrs<NPHI, false>();
    set_attrs<1, true>();
    set_attrs<NPHI, true>();
    cudaFuncSetAttribute(k_mlp_f8_fwd<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, F8Fwd::REQUEST);
    cudaFuncSetAttribute(k_mlp_f8_fwd<NPHI>, cudaFuncAttributeMaxDynamicSharedMemorySize, F8Fwd::REQUEST);
    cudaFuncSetAttribute(k_mlp_f8_bwd<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, F8Bwd::REQUEST);
    cudaFuncSetAttribute(k_mlp_f8_bwd<NPHI>, cudaFuncAttributeMaxDynamicSharedMemorySize, F8Bwd::REQUEST);
    if (dev < 64) done |= (uint64_t)1 << dev;
}

template <int OUT, bool SPLIT>
void fwd_launch(cudaStream_t s, int nt, const TcLayer& l, const Tile* tiles, const float* rho, float* out,
                int out_stride, int* flags, GhostOut gh, float* dsave) {
    k_mlp_tc_fwd<OUT, SPLIT><<<nt, kThreads, FwdSmem<SPLIT>::REQUEST, s>>>(l, tiles, rho, out, out_stride, flags, gh,
                                                                          dsave);
}

template <int OUT, bool SPLIT>
void bwd_launch(cudaStream_t s, int nt, const TcLayer& l, const Tile* tiles, const float* dsave, const float* ybar,
                float* rhobar, int* flags) {
    k_mlp_tc_bwd<OUT, SPLIT><<<nt, kThreads, BwdSmem<SPLIT>::REQUEST, s>>>(l, tiles, dsave, ybar, rhobar, flags);
}

}  // namespace

cudaError_t launch_mlp_fwd_tc(cudaStream_t s, const reann_nlist* nl, const TcTable& nets, int t, bool energy,
                              int precision, const float* rho, float* out, int out_stride, int* flags, GhostOut gh,
                              float* dsave) {
    const int nt = (int)nl->tiles128_h.size();
    if (nt == 0) return cudaSuccess;
    ensure_tc_attrs();
    const TcLayer l = layer_of(nets, t);
    if (precision == REANN_MLP_FP8) {
        if (energy)
            k_mlp_f8_fwd<1><<<nt, kThreads, F8Fwd::REQUEST, s>>>(l, nl->tiles128, rho, out, out_stride, flags, gh);
        else
            k_mlp_f8_fwd<NPHI><<<nt, kThreads, F8Fwd::REQUEST, s>>>(l, nl->tiles128, rho, out, out_stride, flags, gh);
        return cudaGetLastError();
    }
    const bool split = precision == REANN_MLP_BF16X3;
    if (energy)
        (split ? fwd_launch<1, true> : fwd_launch<1, false>)(s, nt, l, nl->tiles128, rho, out, out_stride, flags, gh,
                                                             dsave);
    else
        (split ? fwd_launch<NPHI, true> : fwd_launch<NPHI, false>)(s, nt, l, nl->tiles128, rho, out, out_stride,
                                                                    flags, gh, dsave);
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(cudaStream_t s, int* flags, long long polls) {
    k_wait_selftest<<<1, kThreads, 0, s>>>(flags, polls);
    return cudaGetLastError();
}

cudaError_t launch_mlp_bwd_tc(cudaStream_t s, const reann_nlist* nl, const TcTable& nets, int t, bool energy,
                              int precision, const float* rho, const float* dsave, const float* ybar, float* rhobar,
                              int* flags) {
    const int nt = (int)nl->tiles128_h.size();
    if (nt == 0) return cudaSuccess;
    ensure_tc_attrs();
    const TcLayer l = layer_of(nets, t);
    if (precision == REANN_MLP_FP8) {
        if (energy)
            k_mlp_f8_bwd<1><<<nt, kThreads, F8Bwd::REQUEST, s>>>(l, nl->tiles128, rho, ybar, rhobar, flags);
        else
            k_mlp_f8_bwd<NPHI><<<nt, kThreads, F8Bwd::REQUEST, s>>>(l, nl->tiles128, rho, ybar, rhobar, flags);
        return cudaGetLastError();
    }
    const bool split = precision == REANN_MLP_BF16X3;
    if (!dsave) return cudaErrorInvalidValue;  // the BF16 backward reads the forward's SiLU' values
    if (energy)
        (split ? bwd_launch<1, true> : bwd_launch<1, false>)(s, nt, l, nl->tiles128, dsave, ybar, rhobar, flags);
    else
        (split ? bwd_launch<NPHI, true> : bwd_launch<NPHI, false>)(s, nt, l, nl->tiles128, dsave, ybar, rhobar,
                                                                    flags);
    return cudaGetLastError();
}

}  // namespace reann
