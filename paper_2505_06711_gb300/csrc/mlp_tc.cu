// Per-element atomic networks on the 5th-generation tensor cores (tcgen05):
// BF16, split BF16 (hi + lo) or FP8 E4M3 operands, FP32 accumulation in tensor
// memory (TMEM).
//
// Sec. 2.1, Eq. 2: c^{t+1}_i = M^t_{Z_i}(rho^t_i), 48 -> 64 -> 64 -> 8, and the
// energy network 48 -> 64 -> 64 -> 1, SiLU between layers; the reverse pass
// (Eqs. 3-5) needs rhobar = J^T ybar only (a vector-Jacobian product), and the
// backward kernel goes on to the first step of the density adjoint (bbar of
// Eq. 1's squares) and writes the adjoint records the edge kernel reads.
//
// Tiles and threads.  One CTA of 512 threads (16 warps) takes a tile of 128
// consecutive atoms of one element (atoms are stored element-major).  Warp w
// reads TMEM lanes 32 (w % 4) .. + 31 (its row quarter) and columns
// [16 (w / 4), + 16) of a 64-wide layer, so each row is handled by four threads
// and each thread holds 16 values of its row (many warps per tile hide the
// latency of the per-row epilogue work, which outweighs the products at this
// network width).  Thread 0 issues
// tcgen05.mma.cta_group::1 (M = 128) with A (activations) and B (weights, N x K)
// in shared memory in the K-major no-swizzle core-matrix layout and D in TMEM;
// tcgen05.commit arrives on an mbarrier that all threads wait on.
//
// Anchored products.  Before each product the tile subtracts an anchor from
// its activations and only the deviation is rounded to the low-precision type:
//   x W = (x - xbar) W + xbar W,
// xbar the column mean of the tile's valid rows (FP32) and xbar W computed in
// FP32 from the FP32 weights while the tensor-core product runs.  The identity
// is exact, so the network computes Eq. 2 unchanged; rounding now acts on
// deviations from the tile mean, which are small wherever atoms see similar
// environments (a crystal), and the weight rounding acts on deviations that sum
// to zero over the tile instead of shifting every atom alike.  The output
// layer (64 -> 8 or 1) and the first backward product ybar W3^T are FP32 SIMT.
// Forward: rho -> [anchor] z1 -> SiLU -> [anchor] z2 -> SiLU -> FP32 W3.
// Backward: ybar -> FP32 W3^T (x SiLU'(z2)) -> [anchor] W2^T (x SiLU'(z1)) ->
// [anchor] W1^T = rhobar, with SiLU'(z1), SiLU'(z2) saved by the forward.
//
// Precisions (template P):
//   P_BF16   one kind::f16 MMA per K step of 16, BF16 operands;
//   P_SPLIT  every operand a BF16 pair x = hi + lo, hi*hi + hi*lo + lo*hi per K
//            step (about 16 significant bits per operand);
//   P_FP8    kind::f8f6f4, E4M3 operands, K step 32; each activation row is
//            divided by its own power-of-two scale (row max |x| / 448 rounded
//            up to a power of two, so the division is exact) and each weight
//            row of B (an output unit) by its own scale max |w| / 448
//            (host-built); the accumulator is multiplied back by both.
//
// Core-matrix layouts.  BF16 R x K tile: 8 x 8 blocks of 128 contiguous bytes
// (8 rows of 16 bytes), block (r/8, k/8) at (r/8 * K/8 + k/8) * 128;
// descriptor LBO = 128 B (next block along K), SBO = 16 K bytes (next 8 rows).
// E4M3 R x K tile: 8 x 16 blocks, block (r/8, k/16) at (r/8 * K/16 + k/16) * 128;
// LBO = 128 B, SBO = 8 K bytes.
//
// Every mbarrier wait is bounded: after kSpinLimit polls a CTA records
// FLAG_TIMEOUT in the context flags, waits (bounded) until every MMA it issued
// and its bulk copies have completed, frees its TMEM and returns
// (reann_ctx_check reports REANN_E_TIMEOUT).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>

#include "bulk.cuh"
#include "common.cuh"

namespace reann {
namespace {

constexpr int kThreads = 512;
constexpr int kRows = 128;
constexpr uint32_t kTmemCols = 128;
constexpr long long kSpinLimit = bulk::kSpinLimit;

enum Prec { P_BF16 = 0, P_SPLIT = 1, P_FP8 = 2 };

// the networks of one layer, one per element (kernel parameter)
struct TcLayer {
    TcImg e[MAX_ELEM];
};

// ------------------------------------------------------------- PTX glue ---
using bulk::bulk_g2s;
using bulk::fence_async_smem;
using bulk::mbar_expect_tx;
using bulk::mbar_init;
using bulk::mbar_wait;
using bulk::smem_addr;

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

// kind::f8f6f4 instruction descriptor: D = F32, A = B = E4M3 (format 0), both K-major
__host__ __device__ constexpr uint32_t make_idesc_e4m3(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_e4m3(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar))
                 : "memory");
}

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
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
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

// 32 consecutive FP32 columns of this thread's TMEM lane (one load, one wait)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// TMEM address of lane quarter q (a warp's w % 4), column col
__device__ __forceinline__ uint32_t lane_addr(uint32_t tmem, int q, int col) {
    return tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)col;
}

// SiLU(z) = z s and SiLU'(z) = s (1 + z (1 - s)), s = 1 / (1 + exp(-z)), with
// the fast exponential and division intrinsics (a few units in the last place,
// far below the rounding of the tensor-core operands); h receives SiLU, the
// result is SiLU'.  For z below about -88, exp(-z) is infinite and s = 0.
__device__ __forceinline__ float silu_fast(float z, float& h) {
    const float s = __fdividef(1.f, 1.f + __expf(-z));
    h = z * s;
    return s * fmaf(z, 1.f - s, 1.f);
}

// --------------------------------------------------- operand tiles (smem) ---
// 8 values (k = 8 kc .. 8 kc + 7) of row r into a BF16 core-matrix tile with K
// columns; with lo, the BF16 rounding of the remainder goes to the lo tile
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

// 16 values (k = 16 kc .. 16 kc + 15, already divided by the row's scale) of row r
// into an E4M3 core-matrix tile with K columns (round to nearest even, saturating)
__device__ __forceinline__ void put16_e4m3(uint8_t* tile, int K, int r, int kc, const float* v) {
    uint32_t w[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        uint16_t lo, hi;  // cvt puts its first source in the upper byte
        asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(lo) : "f"(v[4 * p + 1]), "f"(v[4 * p]));
        asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(hi) : "f"(v[4 * p + 3]), "f"(v[4 * p + 2]));
        w[p] = (uint32_t)lo | ((uint32_t)hi << 16);
    }
    *reinterpret_cast<uint4*>(tile + ((size_t)((r >> 3) * (K / 16) + kc) * 128 + (r & 7) * 16)) =
        make_uint4(w[0], w[1], w[2], w[3]);
}

// power-of-two scale s with max |x| / s in [224, 448) (1 for an all-zero row):
// dividing by it and multiplying back are exact
__device__ __forceinline__ float pow2_scale(float amax) {
    if (!(amax > 0.f)) return 1.f;
    int e;
    frexpf(amax * (1.f / 448.f), &e);
    return ldexpf(1.f, e);
}

// This thread's 16 values of row r (columns [16 cq, 16 cq + 16) of K = 64) into
// the A tile(s) of precision P.  FP8: the row's scale from the four quarters of
// the row (exchanged through rmax, one __syncthreads, which every thread of the
// CTA must reach) is returned; else 1.
template <int P>
__device__ __forceinline__ float put_quarter_row(uint8_t* A, uint8_t* Alo, int r, int cq, float* v, float* rmax) {
    if (P == P_FP8) {
        float m = 0.f;
#pragma unroll
        for (int i = 0; i < 16; ++i) m = fmaxf(m, fabsf(v[i]));
        rmax[cq * kRows + r] = m;
        __syncthreads();
        const float s = pow2_scale(fmaxf(fmaxf(rmax[r], rmax[kRows + r]), fmaxf(rmax[2 * kRows + r], rmax[3 * kRows + r])));
        const float inv = 1.f / s;
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] *= inv;
        put16_e4m3(A, 64, r, cq, v);
        return s;
    }
    put8(A, P == P_SPLIT ? Alo : nullptr, 64, r, 2 * cq, v);
    put8(A, P == P_SPLIT ? Alo : nullptr, 64, r, 2 * cq + 1, v + 8);
    return 1.f;
}

// D (TMEM) = A (K columns) x B^T (B: N rows of K) for one 128-row tile
template <int P>
__device__ __forceinline__ void issue(uint32_t tmem_d, const uint8_t* A, const uint8_t* Alo, int K, const uint8_t* B,
                                      const uint8_t* Blo, int N) {
    const uint32_t a0 = smem_addr(A), b0 = smem_addr(B);
    if (P == P_FP8) {
        const uint32_t idesc = make_idesc_e4m3(kRows, N);
        for (int ks = 0; ks < K / 32; ++ks)
            mma_e4m3(tmem_d, make_desc(a0 + ks * 256, 128, 8 * K), make_desc(b0 + ks * 256, 128, 8 * K), idesc,
                     ks > 0 ? 1u : 0u);
        return;
    }
    const uint32_t idesc = make_idesc(kRows, N);
    const uint32_t a1 = P == P_SPLIT ? smem_addr(Alo) : 0u, b1 = P == P_SPLIT ? smem_addr(Blo) : 0u;
    for (int ks = 0; ks < K / 16; ++ks) {
        const uint64_t ah = make_desc(a0 + ks * 256, 128, 16 * K), bh = make_desc(b0 + ks * 256, 128, 16 * K);
        mma_bf16(tmem_d, ah, bh, idesc, ks > 0 ? 1u : 0u);
        if (P == P_SPLIT) {
            mma_bf16(tmem_d, ah, make_desc(b1 + ks * 256, 128, 16 * K), idesc, 1u);
            mma_bf16(tmem_d, make_desc(a1 + ks * 256, 128, 16 * K), bh, idesc, 1u);
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

// bar[0]: bulk copies, bar[1]: MMA completion, bar[2]: drain after a timeout
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

// uniform bounded wait: every thread polls; the CTA agrees on the outcome
__device__ __forceinline__ bool wait_all(uint64_t* bar, uint32_t parity, long long limit = kSpinLimit) {
    const bool ok = mbar_wait(bar, parity, limit);
    return __syncthreads_and(ok);
}

// After a wait ran out: record FLAG_TIMEOUT, then make sure nothing this CTA
// started is still in flight before the caller releases its TMEM and shared
// memory.  Thread 0 commits every tcgen05 operation it issued to the spare
// barrier bar[2] (it arrives once all of them completed, at once when there
// were none); when the bulk copies were not seen to land, their barrier is
// waited for again.  Both waits are bounded; if either runs out as well,
// FLAG_TIMEOUT_DRAIN is recorded too (the CTA still frees its TMEM and
// returns, and the host reports that the device state is suspect).
__device__ __forceinline__ void fail(int* flags, uint64_t* bar, bool copies_landed) {
    if (threadIdx.x == 0) {
        atomicOr(&flags[FLAG_TIMEOUT], 1);
        mma_commit(&bar[2]);
    }
    bool drained = mbar_wait(&bar[2], 0);
    if (!copies_landed) drained = mbar_wait(&bar[0], 0) && drained;
    if (!__syncthreads_and(drained) && threadIdx.x == 0) atomicOr(&flags[FLAG_TIMEOUT_DRAIN], 1);
}

// One butterfly reduce-scatter stage over CNT values: lanes with bit CNT/2 set
// keep the upper half, and each kept value adds its partner lane's.
template <int CNT>
__device__ __forceinline__ void rs_stage(float* v, int lane) {
    constexpr int H = CNT / 2;
    const bool upper = lane & H;
#pragma unroll
    for (int k = 0; k < H; ++k) {
        const float send = upper ? v[k] : v[k + H];
        const float keep = upper ? v[k + H] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, H);
    }
}

// Column means over the tile's rows of a 64-wide layer held as 16 values per
// thread (rows past the tile's end must hold zeros).  In each warp the stages
// 16, 8, 4, 2 leave lane l with column c0 + (l % 16) summed over its half-warp,
// one more shuffle adds the other half; the 4 row quarters are then added in a
// fixed order, so the result is deterministic.
__device__ __forceinline__ void tile_mean64(const float* v, float* psum, float* mean, int q, int c0, int lane,
                                            float inv_n) {
    float t[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) t[i] = v[i];
    rs_stage<16>(t, lane);
    rs_stage<8>(t, lane);
    rs_stage<4>(t, lane);
    rs_stage<2>(t, lane);
    t[0] += __shfl_xor_sync(0xffffffffu, t[0], 16);
    if (lane < 16) psum[q * 64 + c0 + lane] = t[0];
    __syncthreads();
    const int c = threadIdx.x;
    if (c < 64) mean[c] = ((psum[c] + psum[64 + c]) + (psum[128 + c] + psum[192 + c])) * inv_n;
    __syncthreads();
}

// Anchor products x W in FP32 with all 512 threads: thread t takes output
// j = t % 64 and the eighth p8 = t / 64 of the K inputs.  Its K/8 weights are
// loaded in one unrolled batch (wq_load, issued early so the loads overlap other
// work), the partial dot product goes to part[p8][j], and after a
// __syncthreads the eight partials are added in a fixed order (wq_sum).
template <int K>
struct WQ {
    float w[K / 8];
};
template <int K>
__device__ __forceinline__ void wq_load(WQ<K>& r, const float* __restrict__ W, int ldw, int nout) {
    const int j = threadIdx.x & 63, p8 = threadIdx.x >> 6;
#pragma unroll
    for (int i = 0; i < K / 8; ++i) r.w[i] = j < nout ? __ldg(W + (size_t)(K / 8 * p8 + i) * ldw + j) : 0.f;
}
template <int K>
__device__ __forceinline__ void wq_part(const WQ<K>& r, const float* x, float* part) {
    const int j = threadIdx.x & 63, p8 = threadIdx.x >> 6;
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < K / 8; ++i) s = fmaf(x[K / 8 * p8 + i], r.w[i], s);
    part[p8 * 64 + j] = s;
}
// after a __syncthreads: out[j] = bias[j] + the eight partials (bias may be null), j < nout
__device__ __forceinline__ void wq_sum(const float* part, const float* bias, float* out, int nout) {
    const int j = threadIdx.x;
    if (j < nout)
        out[j] = (bias ? bias[j] : 0.f) + (((part[j] + part[64 + j]) + (part[128 + j] + part[192 + j])) +
                                           ((part[256 + j] + part[320 + j]) + (part[384 + j] + part[448 + j])));
}

// 16 consecutive floats of shared memory (16 B aligned) into registers
__device__ __forceinline__ void lds16(const float* p, float* v) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 x = reinterpret_cast<const float4*>(p)[k];
        v[4 * k] = x.x, v[4 * k + 1] = x.y, v[4 * k + 2] = x.z, v[4 * k + 3] = x.w;
    }
}

// 16 consecutive floats of global memory (16 B aligned) into registers, zeros when !ok
__device__ __forceinline__ void ldg16(const float* p, bool ok, float* v) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 x = ok ? __ldg(reinterpret_cast<const float4*>(p) + k) : make_float4(0.f, 0.f, 0.f, 0.f);
        v[4 * k] = x.x, v[4 * k + 1] = x.y, v[4 * k + 2] = x.z, v[4 * k + 3] = x.w;
    }
}

// ------------------------------------------------------------- layouts ---
// FP32 parameter / scratch area (float offsets); every block starts on 16 B
enum FwdPar {
    F_B1 = 0, F_B2 = 64, F_B3 = 128, F_W3 = 136, F_S1 = 648, F_S2 = 712, F_RB = 776, F_Z1 = 840, F_HB = 904,
    F_Z2 = 968, F_PS = 1032, F_RM = 1288, F_ZP = 1800, F_END = 2312
};
enum BwdPar {
    B_W3 = 0, B_WC = 512, B_S2 = 896, B_S1 = 960, B_VB2 = 1024, B_U2 = 1088, B_VB1 = 1152, B_RA = 1216,
    B_PS = 1280, B_RM = 1536, B_ZP = 2048, B_END = 2560
};

constexpr uint32_t img_bytes(int P) { return P == P_FP8 ? 8192u : 14336u; }  // W1^T | W2^T  (bwd: W2 | W1)
constexpr uint32_t a_bytes(int P) { return P == P_FP8 ? 8192u : 16384u; }     // one 128 x 64 activation tile
constexpr uint32_t nsplit(int P) { return P == P_SPLIT ? 2u : 1u; }
constexpr uint32_t rup(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }
constexpr uint32_t umax(uint32_t a, uint32_t b) { return a > b ? a : b; }

template <int P>
struct FwdL {
    static constexpr uint32_t WB = img_bytes(P), AB = a_bytes(P), NS = nsplit(P);
    static constexpr uint32_t W2T = P == P_FP8 ? 4096u : 6144u;  // W2^T inside the image
    // X: the tile's input rows (FP32, bulk copy); once the first A tile is written the same
    // bytes hold the output layer's partial sums (OP: 4 column quarters x 128 rows x 8)
    static constexpr uint32_t W = 0, A = rup(W + WB * NS, 1024), X = rup(A + AB * NS, 1024),
                              PAR = X + umax(kRows * NFEAT * 4, 4 * kRows * 8 * 4), SE = PAR + F_END * 4,
                              BAR = SE + kRows * 8;
    static constexpr int BYTES = BAR + 64;
};
template <int P>
struct BwdL {
    static constexpr uint32_t WB = img_bytes(P), AB = a_bytes(P), NS = nsplit(P);
    static constexpr uint32_t W1B = P == P_FP8 ? 4096u : 8192u;  // W1 inside the backward image
    static constexpr uint32_t W = 0, A = rup(W + WB * NS, 1024);
    static constexpr uint32_t REC = 0;  // record staging, once the products are done
    static constexpr int kLdR = NFEAT + 1;  // rhobar staging stride (floats)
    static constexpr uint32_t RB = rup(umax(A + AB * NS, (uint32_t)(kRows * kRecLd * 4)), 1024),
                              PAR = rup(RB + kRows * kLdR * 4, 16), BAR = PAR + B_END * 4;
    static constexpr int BYTES = BAR + 64;
};
static_assert(FwdL<P_SPLIT>::BYTES <= 113 * 1024 && BwdL<P_SPLIT>::BYTES <= 113 * 1024, "two CTAs per SM");
static_assert(FwdL<P_BF16>::BYTES <= 113 * 1024 && FwdL<P_FP8>::BYTES <= 113 * 1024, "two CTAs per SM");
static_assert(BwdL<P_BF16>::BYTES <= 113 * 1024 && BwdL<P_FP8>::BYTES <= 113 * 1024, "two CTAs per SM");

// ------------------------------------------------------------- forward ---
// rho tile -> c (out_stride, ghost images too) or eps (and the tile's FP64
// energy sum in epart); dsave[row] = SiLU'(z1) (64) | SiLU'(z2) (64).
template <int OUT, int P>
__global__ void __launch_bounds__(kThreads, 2) k_tc_fwd(TcLayer nets, const Tile* __restrict__ tiles,
                                                       const float* __restrict__ rho, float* __restrict__ out,
                                                       int out_stride, int* __restrict__ flags, GhostOut gh,
                                                       float* __restrict__ dsave, double* __restrict__ epart) {
    pdl_enter();
    using L = FwdL<P>;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 3);
    float* par = reinterpret_cast<float*>(smem + L::PAR);
    const float* sX = reinterpret_cast<const float*>(smem + L::X);
    float* sOP = reinterpret_cast<float*>(smem + L::X);  // after the first A tile
    uint8_t* sA = smem + L::A;
    uint8_t* sAlo = P == P_SPLIT ? smem + L::A + L::AB : nullptr;
    const uint8_t* sW = smem + L::W;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, q = warp & 3, cq = warp >> 2;
    const int r = 32 * q + lane, c0 = 16 * cq;
    const Tile tl = tiles[blockIdx.x];
    if (tl.nrows <= 0) {  // padding entry of a fixed-size tile list (before any TMEM allocation)
        if (OUT == 1 && epart && tid == 0) epart[blockIdx.x] = 0.0;
        return;
    }
    const bool valid = r < tl.nrows;
    const int64_t row = tl.row0 + r;
    const float inv_n = 1.f / (float)tl.nrows;
    const TcImg& w = nets.e[tl.elem];
    int64_t g_lo = 0, g_hi = 0;  // the row's ghost images (loaded now, used by the output stage)
    if (OUT > 1 && gh.goff && valid) {
        g_lo = gh.goff[row];
        g_hi = min((int64_t)gh.goff[row + 1], gh.gcap);
    }
    const uint32_t tmem = setup(tslot, bar);
    if (tid == 0) {
        const uint32_t xb = (uint32_t)tl.nrows * NFEAT * 4;
        const uint8_t* img = P == P_FP8 ? w.wf8 : w.wf;
        mbar_expect_tx(&bar[0], L::WB * L::NS + xb);
        bulk_g2s(smem + L::W, img, L::WB, &bar[0]);
        if (P == P_SPLIT) bulk_g2s(smem + L::W + L::WB, img + L::WB, L::WB, &bar[0]);
        bulk_g2s(smem + L::X, rho + (size_t)tl.row0 * NFEAT, xb, &bar[0]);
    }
    if (tid < 64) {
        par[F_B1 + tid] = w.b1[tid];
        par[F_B2 + tid] = w.b2[tid];
        if (P == P_FP8) {
            par[F_S1 + tid] = w.s8[tid];
            par[F_S2 + tid] = w.s8[64 + tid];
        }
    }
    if (tid < OUT) par[F_B3 + tid] = w.b3[tid];
    for (int i = tid; i < H2 * OUT; i += kThreads) par[F_W3 + (i / OUT) * 8 + i % OUT] = w.W3[i];
    WQ<NFEAT> wq1;  // this thread's eighth of W1 for the anchor zhat1 = rho-bar W1 + b1
    wq_load<NFEAT>(wq1, w.W1, H1, H1);
    bool ok = wait_all(&bar[0], 0);
    if (!ok) fail(flags, bar, false);
    float sx = 1.f, sh = 1.f;
    float v[16], a[16];
    if (ok) {
        // this quarter row of rho (features [16 cq, 16 cq + 16); the fourth quarter and rows
        // past the tile's end hold zeros), then rho-bar: the column means of the valid rows
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 x = (valid && cq < 3) ? reinterpret_cast<const float4*>(sX + r * NFEAT + c0)[k]
                                               : make_float4(0.f, 0.f, 0.f, 0.f);
            v[4 * k] = x.x, v[4 * k + 1] = x.y, v[4 * k + 2] = x.z, v[4 * k + 3] = x.w;
        }
        tile_mean64(v, par + F_PS, par + F_RB, q, c0, lane, inv_n);
        // A0 = rho - rho-bar: BF16 tiles have K = 48 (the fourth quarter writes nothing),
        // E4M3 tiles K = 64 (48 + zeros)
        float xb[16];
        lds16(par + F_RB + c0, xb);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = (valid && cq < 3) ? v[i] - xb[i] : 0.f;
        if (P == P_FP8) {
            sx = put_quarter_row<P>(sA, nullptr, r, cq, v, par + F_RM);
        } else if (cq < 3) {
            put8(sA, sAlo, NFEAT, r, 2 * cq, v);
            put8(sA, sAlo, NFEAT, r, 2 * cq + 1, v + 8);
        }
        handoff();
        if (tid == 0) {  // z1 - zhat1 = (rho - rho-bar) W1
            if (P == P_FP8)
                issue<P>(tmem, sA, nullptr, 64, sW, nullptr, H1);
            else
                issue<P>(tmem, sA, sAlo, NFEAT, sW, P == P_SPLIT ? sW + L::WB : nullptr, H1);
            mma_commit(&bar[1]);
        }
        wq_part<NFEAT>(wq1, par + F_RB, par + F_ZP);  // zhat1 = rho-bar W1 + b1 (FP32) while the product runs
        ok = wait_all(&bar[1], 0);
        if (!ok) fail(flags, bar, true);
        wq_sum(par + F_ZP, par + F_B1, par + F_Z1, H1);
        __syncthreads();
    }
    if (ok) {
        tc_fence_after();
        tmem_ld16(lane_addr(tmem, q, c0), a);
        float zb[16], sc[16];
        lds16(par + F_Z1 + c0, zb);
        if (P == P_FP8) lds16(par + F_S1 + c0, sc);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float z = (P == P_FP8 ? a[i] * (sx * sc[i]) : a[i]) + zb[i];
            a[i] = silu_fast(z, v[i]);  // a: SiLU'(z1), v: h1
            if (!valid) v[i] = 0.f;
        }
        if (valid && dsave) {
            float4* d = reinterpret_cast<float4*>(dsave + (size_t)row * (H1 + H2) + c0);
#pragma unroll
            for (int k = 0; k < 4; ++k) d[k] = make_float4(a[4 * k], a[4 * k + 1], a[4 * k + 2], a[4 * k + 3]);
        }
        WQ<H1> wq2;  // this thread's eighth of W2 for zhat2 = h1-bar W2 + b2
        wq_load<H1>(wq2, w.W2, H2, H2);
        tile_mean64(v, par + F_PS, par + F_HB, q, c0, lane, inv_n);  // h1-bar
        lds16(par + F_HB + c0, zb);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = valid ? v[i] - zb[i] : 0.f;
        sh = put_quarter_row<P>(sA, sAlo, r, cq, v, par + F_RM);
        handoff();
        if (tid == 0) {  // z2 - zhat2 = (h1 - h1-bar) W2
            issue<P>(tmem + 64, sA, sAlo, 64, sW + L::W2T, P == P_SPLIT ? sW + L::WB + L::W2T : nullptr, H2);
            mma_commit(&bar[1]);
        }
        wq_part<H1>(wq2, par + F_HB, par + F_ZP);
        ok = wait_all(&bar[1], 1);
        if (!ok) fail(flags, bar, true);
        wq_sum(par + F_ZP, par + F_B2, par + F_Z2, H2);
        __syncthreads();
    }
    if (ok) {
        tc_fence_after();
        tmem_ld16(lane_addr(tmem, q, 64 + c0), a);
        float zb[16], sc[16];
        lds16(par + F_Z2 + c0, zb);
        if (P == P_FP8) lds16(par + F_S2 + c0, sc);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float z = (P == P_FP8 ? a[i] * (sh * sc[i]) : a[i]) + zb[i];
            a[i] = silu_fast(z, v[i]);  // a: SiLU'(z2), v: h2
        }
        if (valid && dsave) {
            float4* d = reinterpret_cast<float4*>(dsave + (size_t)row * (H1 + H2) + H1 + c0);
#pragma unroll
            for (int k = 0; k < 4; ++k) d[k] = make_float4(a[4 * k], a[4 * k + 1], a[4 * k + 2], a[4 * k + 3]);
        }
        // output layer in FP32: this quarter row's partial dot products, then the four quarters
        float y[OUT];
#pragma unroll
        for (int o = 0; o < OUT; ++o) y[o] = 0.f;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            if (OUT == 1) {
                y[0] = fmaf(v[i], par[F_W3 + (c0 + i) * 8], y[0]);
            } else {
                const float4 wa = *reinterpret_cast<const float4*>(par + F_W3 + (c0 + i) * 8);
                const float4 wb = *reinterpret_cast<const float4*>(par + F_W3 + (c0 + i) * 8 + 4);
                const float wv[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
                for (int o = 0; o < OUT; ++o) y[o] = fmaf(v[i], wv[o], y[o]);
            }
        }
        if (OUT == 1) {
            sOP[cq * kRows + r] = y[0];
        } else {
            float4* d = reinterpret_cast<float4*>(sOP + (cq * kRows + r) * 8);
            d[0] = make_float4(y[0], y[1], y[2], y[3]);
            d[1] = make_float4(y[4], y[5], y[6], y[7]);
        }
        __syncthreads();
        if (OUT == 1) {
            double* sE = reinterpret_cast<double*>(smem + L::SE);
            if (cq == 0) {
                const float e =
                    ((sOP[r] + sOP[kRows + r]) + (sOP[2 * kRows + r] + sOP[3 * kRows + r])) + par[F_B3];
                if (valid) out[(size_t)row * out_stride] = e;
                sE[r] = valid ? (double)e : 0.0;
            }
            if (epart) {  // the tile's energy in FP64, summed in a fixed order
                __syncthreads();
                if (tid < 32) {
                    double x = (sE[tid] + sE[tid + 32]) + (sE[tid + 64] + sE[tid + 96]);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                    if (tid == 0) epart[blockIdx.x] = x;
                }
            }
        } else if (valid) {
            float c[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int o = 2 * cq + k;
                c[k] = ((sOP[r * 8 + o] + sOP[(kRows + r) * 8 + o]) +
                        (sOP[(2 * kRows + r) * 8 + o] + sOP[(3 * kRows + r) * 8 + o])) +
                       par[F_B3 + o];
            }
            const float2 cv = make_float2(c[0], c[1]);
            *reinterpret_cast<float2*>(out + (size_t)row * out_stride + 2 * cq) = cv;
            for (int64_t g = g_lo; g < g_hi; ++g)  // the row's ghost images get the same coefficients (Fig. 4a)
                *reinterpret_cast<float2*>(out + (size_t)(gh.base + g) * out_stride + 2 * cq) = cv;
        }
    }
    teardown(tmem);
}

// ------------------------------------------------------------ backward ---
// rhobar = J^T ybar of the tile's rows (ybar: c-bar rows, or 1 for the energy
// network), then the bbar step of Eq. 1's squares for the same rows,
//   bbar_{a,m} = sum_k 2 w_a g_{a,k} rhobar_{l(a),k} W_{l,m,k},  g = b W (b: checkpoint bck),
// written as the rows' adjoint records (bbar with the layer's c; ghost images too).
template <int OUT, int P>
__global__ void __launch_bounds__(kThreads, 2) k_tc_bwd(TcLayer nets, const Tile* __restrict__ tiles,
                                                       const float* __restrict__ dsave, const float* __restrict__ ybar,
                                                       const float* __restrict__ Wc, const float* __restrict__ bck,
                                                       const float* __restrict__ coef, float* __restrict__ rec,
                                                       GhostOut gh, int* __restrict__ flags) {
    pdl_enter();
    using L = BwdL<P>;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 3);
    float* par = reinterpret_cast<float*>(smem + L::PAR);
    float* sRB = reinterpret_cast<float*>(smem + L::RB);
    uint8_t* sA = smem + L::A;
    uint8_t* sAlo = P == P_SPLIT ? smem + L::A + L::AB : nullptr;
    const uint8_t* sW = smem + L::W;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, q = warp & 3, cq = warp >> 2;
    const int r = 32 * q + lane, c0 = 16 * cq;
    const Tile tl = tiles[blockIdx.x];
    if (tl.nrows <= 0) return;  // padding entry of a fixed-size tile list (before any TMEM allocation)
    const bool valid = r < tl.nrows;
    const int64_t row = tl.row0 + r;
    const float inv_n = 1.f / (float)tl.nrows;
    const TcImg& w = nets.e[tl.elem];
    const uint32_t tmem = setup(tslot, bar);
    if (tid == 0) {
        const uint8_t* img = P == P_FP8 ? w.wb8 : w.wb;
        mbar_expect_tx(&bar[0], L::WB * L::NS);
        bulk_g2s(smem + L::W, img, L::WB, &bar[0]);
        if (P == P_SPLIT) bulk_g2s(smem + L::W + L::WB, img + L::WB, L::WB, &bar[0]);
    }
    for (int i = tid; i < H2 * OUT; i += kThreads) par[B_W3 + (i / OUT) * 8 + i % OUT] = w.W3[i];
    if (tid < (LMAX + 1) * NPHI * NORB) {  // transposed per l: [l][k][m]
        const int i = tid, l = i / (NPHI * NORB), m = (i / NORB) % NPHI, k = i % NORB;
        par[B_WC + (l * NORB + k) * NPHI + m] = Wc[i];
    }
    if (P == P_FP8 && tid < 64) {
        par[B_S2 + tid] = w.s8[128 + tid];
        if (tid < NFEAT) par[B_S1 + tid] = w.s8[192 + tid];
    }
    WQ<H2> wq;  // this thread's eighth of W2^T for the anchor u2-hat = v2-bar W2^T
    wq_load<H2>(wq, w.W2t, H1, H1);
    float yb[OUT];
#pragma unroll
    for (int o = 0; o < OUT; ++o)  // d eps_i / d eps_i = 1 for the energy network
        yb[o] = OUT == 1 ? 1.f : (valid ? __ldg(ybar + (size_t)row * OUT + o) : 0.f);
    float sd[16], v[16], a[16];
    ldg16(dsave + (size_t)row * (H1 + H2) + H1 + c0, valid, sd);  // SiLU'(z2) of this quarter row
    __syncthreads();
    // v2 = (ybar W3^T) * SiLU'(z2) in FP32
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        float u = 0.f;
        if (OUT == 1) {
            u = yb[0] * par[B_W3 + (c0 + i) * 8];
        } else {
            const float4 wa = *reinterpret_cast<const float4*>(par + B_W3 + (c0 + i) * 8);
            const float4 wb = *reinterpret_cast<const float4*>(par + B_W3 + (c0 + i) * 8 + 4);
            const float wv[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
            for (int o = 0; o < OUT; ++o) u = fmaf(yb[o], wv[o], u);
        }
        v[i] = valid ? u * sd[i] : 0.f;
    }
    tile_mean64(v, par + B_PS, par + B_VB2, q, c0, lane, inv_n);
    wq_part<H2>(wq, par + B_VB2, par + B_ZP);  // u2-hat partials (summed after the next barrier)
    lds16(par + B_VB2 + c0, a);
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = valid ? v[i] - a[i] : 0.f;
    float sa = put_quarter_row<P>(sA, sAlo, r, cq, v, par + B_RM);
    handoff();
    bool ok = wait_all(&bar[0], 0);
    if (!ok) fail(flags, bar, false);
    if (ok) {
        if (tid == 0) {  // u2 - u2-hat = (v2 - v2-bar) W2^T, B = W2 (rows h1 unit, K = h2 unit)
            issue<P>(tmem, sA, sAlo, 64, sW, P == P_SPLIT ? sW + L::WB : nullptr, H1);
            mma_commit(&bar[1]);
        }
        ldg16(dsave + (size_t)row * (H1 + H2) + c0, valid, sd);  // SiLU'(z1), while the product runs
        // u2-hat = v2-bar W2^T: sum_q W2[u][q] v2-bar[q] = sum_q W2t[q][u] v2-bar[q]
        wq_sum(par + B_ZP, nullptr, par + B_U2, H1);
        ok = wait_all(&bar[1], 0);
        if (!ok) fail(flags, bar, true);
    }
    if (ok) {
        tc_fence_after();
        tmem_ld16(lane_addr(tmem, q, c0), a);
        float ub[16], sc[16];
        lds16(par + B_U2 + c0, ub);
        if (P == P_FP8) lds16(par + B_S2 + c0, sc);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float u = (P == P_FP8 ? a[i] * (sa * sc[i]) : a[i]) + ub[i];
            v[i] = valid ? u * sd[i] : 0.f;  // v1 = u2 * SiLU'(z1)
        }
        WQ<H1> wq1;  // this thread's eighth of W1^T for rhobar-hat = v1-bar W1^T
        wq_load<H1>(wq1, w.W1t, NFEAT, NFEAT);
        tile_mean64(v, par + B_PS, par + B_VB1, q, c0, lane, inv_n);
        wq_part<H1>(wq1, par + B_VB1, par + B_ZP);
        lds16(par + B_VB1 + c0, ub);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = valid ? v[i] - ub[i] : 0.f;
        sa = put_quarter_row<P>(sA, sAlo, r, cq, v, par + B_RM);
        handoff();
        if (tid == 0) {  // rhobar - rhobar-hat = (v1 - v1-bar) W1^T, B = W1 (rows feature, K = h1 unit)
            issue<P>(tmem + 64, sA, sAlo, 64, sW + L::W1B, P == P_SPLIT ? sW + L::WB + L::W1B : nullptr, NFEAT);
            mma_commit(&bar[1]);
        }
        // rhobar-hat = v1-bar W1^T: sum_u W1[f][u] v1-bar[u] = sum_u W1t[u][f] v1-bar[u]
        wq_sum(par + B_ZP, nullptr, par + B_RA, NFEAT);
        ok = wait_all(&bar[1], 1);
        if (!ok) fail(flags, bar, true);
    }
    if (ok) {
        tc_fence_after();
        // rhobar of the row, features [16 cq, 16 cq + 16) from the first three column quarters
        if (cq < 3) {
            tmem_ld16(lane_addr(tmem, q, 64 + c0), a);
            float ra[16], sc[16];
            lds16(par + B_RA + c0, ra);
            if (P == P_FP8) lds16(par + B_S1 + c0, sc);
#pragma unroll
            for (int i = 0; i < 16; ++i) sRB[r * L::kLdR + c0 + i] = (P == P_FP8 ? a[i] * (sa * sc[i]) : a[i]) + ra[i];
        }
        __syncthreads();  // the products are done: the image and A tiles become the record staging area
        float* sRec = reinterpret_cast<float*>(smem + L::REC);
        if (valid) {
            const float* rb = sRB + r * L::kLdR;
            // record values v = cq, cq + 4, cq + 8: angular terms a < 10, then c (10) and zero (11)
#pragma unroll 1
            for (int vv = cq; vv < NREC / NPHI; vv += 4) {
                float o[NPHI];
                if (vv >= NANG) {
                    rec_tail(coef, row, vv, o);
                    stage_rec(sRec, r, vv, o);
                    continue;
                }
                const int a_ = vv, l = ang_l(a_);
                const float4 b0 = __ldg(reinterpret_cast<const float4*>(bck + (size_t)row * NB + a_ * NPHI));
                const float4 b1 = __ldg(reinterpret_cast<const float4*>(bck + (size_t)row * NB + a_ * NPHI + 4));
                const float bm[NPHI] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int m = 0; m < NPHI; ++m) o[m] = 0.f;
                const float two_w = 2.f * ang_w(a_);
                const float* wl = par + B_WC + l * NORB * NPHI;
                const float* rl = rb + l * NORB;
#pragma unroll 4
                for (int k = 0; k < NORB; ++k) {
                    const float4 w0 = *reinterpret_cast<const float4*>(wl + k * NPHI);
                    const float4 w1 = *reinterpret_cast<const float4*>(wl + k * NPHI + 4);
                    const float wm[NPHI] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
                    float g = 0.f;
#pragma unroll
                    for (int m = 0; m < NPHI; ++m) g = fmaf(bm[m], wm[m], g);
                    const float gb = two_w * g * rl[k];
#pragma unroll
                    for (int m = 0; m < NPHI; ++m) o[m] = fmaf(gb, wm[m], o[m]);
                }
                stage_rec(sRec, r, a_, o);
            }
        }
        __syncthreads();
        flush_rec(sRec, tl.nrows, tl.row0, rec, gh, tid, kThreads);  // ghost images get the rows' records too
    }
    teardown(tmem);
}

// The bounded-wait exit with nothing in flight: allocate TMEM, wait `polls` times on
// an mbarrier that nothing arrives on, then fail() (flag, drain, release) as the
// network kernels do when a wait runs out.
__global__ void __launch_bounds__(kThreads, 1) k_wait_selftest(int* __restrict__ flags, long long polls) {
    pdl_enter();
    __shared__ __align__(8) uint64_t bar[4];
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 3);
    const uint32_t tmem = setup(tslot, bar);
    if (!wait_all(&bar[1], 0, polls)) fail(flags, bar, true);
    teardown(tmem);
}

TcLayer layer_of(const TcTable& t, int layer) {
    TcLayer l;
    for (int e = 0; e < MAX_ELEM; ++e) l.e[e] = t.img[layer][e];
    return l;
}

template <int OUT, int P>
void set_attrs() {
    cudaFuncSetAttribute(k_tc_fwd<OUT, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, FwdL<P>::BYTES);
    cudaFuncSetAttribute(k_tc_bwd<OUT, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, BwdL<P>::BYTES);
}

void ensure_tc_attrs() {
    // once per device, safe under concurrent first calls
    static std::mutex mu;
    static uint64_t done = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 64 && ((done >> dev) & 1)) return;
    set_attrs<1, P_BF16>();
    set_attrs<NPHI, P_BF16>();
    set_attrs<1, P_SPLIT>();
    set_attrs<NPHI, P_SPLIT>();
    set_attrs<1, P_FP8>();
    set_attrs<NPHI, P_FP8>();
    if (dev < 64) done |= (uint64_t)1 << dev;
}

int prec_of(int precision) {
    return precision == REANN_MLP_FP8 ? P_FP8 : (precision == REANN_MLP_BF16X3 ? P_SPLIT : P_BF16);
}

template <int OUT, int P>
void fwd_launch(cudaStream_t s, int nt, const TcLayer& l, const Tile* tiles, const float* rho, float* out,
                int out_stride, int* flags, GhostOut gh, float* dsave, double* epart) {
    k_tc_fwd<OUT, P><<<nt, kThreads, FwdL<P>::BYTES, s>>>(l, tiles, rho, out, out_stride, flags, gh, dsave, epart);
}

template <int OUT, int P>
void bwd_launch(cudaStream_t s, int nt, const TcLayer& l, const Tile* tiles, const float* dsave, const float* ybar,
                const float* Wc, const float* bck, const float* coef, float* rec, GhostOut gh, int* flags) {
    k_tc_bwd<OUT, P><<<nt, kThreads, BwdL<P>::BYTES, s>>>(l, tiles, dsave, ybar, Wc, bck, coef, rec, gh, flags);
}

}  // namespace

cudaError_t launch_mlp_fwd_tc(cudaStream_t s, const reann_nlist* nl, const TcTable& nets, int t, bool energy,
                              int precision, const float* rho, float* out, int out_stride, int* flags, GhostOut gh,
                              float* dsave, double* epart) {
    const int nt = (int)tiles128_of(nl);
    if (nt == 0) return cudaSuccess;
    if (!dsave) return cudaErrorInvalidValue;
    ensure_tc_attrs();
    const TcLayer l = layer_of(nets, t);
    using F = void (*)(cudaStream_t, int, const TcLayer&, const Tile*, const float*, float*, int, int*, GhostOut,
                       float*, double*);
    static const F table[2][3] = {{fwd_launch<NPHI, P_BF16>, fwd_launch<NPHI, P_SPLIT>, fwd_launch<NPHI, P_FP8>},
                                  {fwd_launch<1, P_BF16>, fwd_launch<1, P_SPLIT>, fwd_launch<1, P_FP8>}};
    table[energy ? 1 : 0][prec_of(precision)](s, nt, l, nl->tiles128, rho, out, out_stride, flags, gh, dsave,
                                              energy ? epart : nullptr);
    return cudaGetLastError();
}

cudaError_t launch_mlp_bwd_tc(cudaStream_t s, const reann_nlist* nl, const TcTable& nets, int t, bool energy,
                              int precision, const float* dsave, const float* ybar, const float* Wc, const float* bck,
                              const float* coef, float* rec, GhostOut gh, int* flags) {
    const int nt = (int)tiles128_of(nl);
    if (nt == 0) return cudaSuccess;
    if (!dsave) return cudaErrorInvalidValue;  // the backward reads the forward's SiLU' values
    ensure_tc_attrs();
    const TcLayer l = layer_of(nets, t);
    using F = void (*)(cudaStream_t, int, const TcLayer&, const Tile*, const float*, const float*, const float*,
                       const float*, const float*, float*, GhostOut, int*);
    static const F table[2][3] = {{bwd_launch<NPHI, P_BF16>, bwd_launch<NPHI, P_SPLIT>, bwd_launch<NPHI, P_FP8>},
                                  {bwd_launch<1, P_BF16>, bwd_launch<1, P_SPLIT>, bwd_launch<1, P_FP8>}};
    table[energy ? 1 : 0][prec_of(precision)](s, nt, l, nl->tiles128, dsave, ybar, Wc, bck, coef, rec, gh, flags);
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(cudaStream_t s, int* flags, long long polls) {
    k_wait_selftest<<<1, kThreads, 0, s>>>(flags, polls);
    return cudaGetLastError();
}

}  // namespace reann
