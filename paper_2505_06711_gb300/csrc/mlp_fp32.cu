// Per-element atomic networks in plain FP32 (SIMT FMA), forward and
// input-gradient backward.
//
// Sec. 2.1, Eq. 2: c^{t+1}_i = M^t_{Z_i}(rho^t_i) (48 -> 64 -> 64 -> 8), and the
// energy network eps_i = M^{T-1}_{Z_i}(rho^{T-1}_i) (48 -> 64 -> 64 -> 1), SiLU
// between layers.  The reverse pass (Eqs. 4-5) needs only the input gradient
// rhobar = J^T ybar (a vector-Jacobian product, Sec. 2.2), never weight
// gradients.
//
// Atoms are stored element-major, so a tile of 64 consecutive rows uses one
// element's weights.  A block of 256 threads computes a 64x64 layer output as
// 16x16 threads x (4 rows x 4 columns), reading float4 fragments of the
// row-major activations and weights from shared memory.  The forward keeps one
// activation buffer (48 KB of shared memory: four blocks per SM) and writes
// SiLU'(z1), SiLU'(z2) of every row; the backward reads them instead of
// recomputing the forward, and with the 48-feature networks also takes the
// bbar step of Eq. 1's squares and writes the adjoint records (69 KB: three
// blocks per SM).
#include <cuda_runtime.h>

#include <mutex>

#include "bulk.cuh"
#include "common.cuh"

namespace reann {
namespace {

constexpr int kT = 256;       // threads per block
constexpr int kR = MLP_TILE;  // 64 rows per tile
constexpr int LDH = H1 + 4;     // 68
// input rows of FIN features are held with stride FIN (one bulk copy of the
// tile's contiguous rows) in the buffer that later holds h1 (stride LDH)
template <int FIN>
__host__ __device__ constexpr int ldx() { return FIN; }
template <int FIN>
__host__ __device__ constexpr int abuf() { return kR * (ldx<FIN>() > LDH ? ldx<FIN>() : LDH); }

struct NetsOfLayer {
    NetDev e[MAX_ELEM];
};

// SiLU(z) = z s and SiLU'(z) = s (1 + z (1 - s)) from one correctly rounded
// reciprocal s = 1 / (1 + exp(-z)); h receives SiLU, the result is SiLU'
__device__ __forceinline__ float silu_d(float z, float& h) {
    const float s = __frcp_rn(1.f + expf(-z));
    h = z * s;
    return s * fmaf(z, 1.f - s, 1.f);
}

// Wait (bounded) for the tile's bulk copies on `bar`; all threads agree.  Thread 0
// initialised `bar` and issued the copies before it reaches the first barrier
// here, so no thread polls the mbarrier before its initialisation.  When the
// wait runs out: record FLAG_TIMEOUT, wait once more for the copies in flight
// (FLAG_TIMEOUT_DRAIN if they still have not landed) and return false.
__device__ __forceinline__ bool staged(uint64_t* bar, int* flags) {
    __syncthreads();
    if (__syncthreads_and(bulk::mbar_wait(bar, 0))) return true;
    if (threadIdx.x == 0) atomicOr(&flags[FLAG_TIMEOUT], 1);
    const bool drained = __syncthreads_and(bulk::mbar_wait(bar, 0));
    if (!drained && threadIdx.x == 0) atomicOr(&flags[FLAG_TIMEOUT_DRAIN], 1);
    return false;
}

__device__ __forceinline__ void copy_f4(float* dst, const float* src, int count, int tid) {
    const float4* s = reinterpret_cast<const float4*>(src);
    float4* d = reinterpret_cast<float4*>(dst);
    for (int i = tid; i < count / 4; i += kT) d[i] = s[i];
}

// acc[i][j] += sum_k A[(4ty+i)*LDA + k] * B[k*LDB + 4tx + j], K multiple of 4
template <int K, int LDA, int LDB>
__device__ __forceinline__ void mma_4x4(const float* A, const float* B, int ty, int tx, float acc[4][4]) {
#pragma unroll 4
    for (int k = 0; k < K; k += 4) {
        float4 a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = *reinterpret_cast<const float4*>(A + (4 * ty + i) * LDA + k);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) b[kk] = *reinterpret_cast<const float4*>(B + (k + kk) * LDB + 4 * tx);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float av[4] = {a[i].x, a[i].y, a[i].z, a[i].w};
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                acc[i][0] = fmaf(av[kk], b[kk].x, acc[i][0]);
                acc[i][1] = fmaf(av[kk], b[kk].y, acc[i][1]);
                acc[i][2] = fmaf(av[kk], b[kk].z, acc[i][2]);
                acc[i][3] = fmaf(av[kk], b[kk].w, acc[i][3]);
            }
        }
    }
}

template <int FIN>
__device__ __forceinline__ void load_rows(float* sX, const float* src, int row0, int nrows, int tid) {
    // 64 rows x FIN floats -> sX[r][FIN + 4]
    for (int t = tid; t < kR * (FIN / 4); t += kT) {
        const int r = t / (FIN / 4), c = t % (FIN / 4);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < nrows) v = *reinterpret_cast<const float4*>(src + (size_t)(row0 + r) * FIN + 4 * c);
        *reinterpret_cast<float4*>(sX + r * ldx<FIN>() + 4 * c) = v;
    }
}

// Sum of 4 * OUT partial values over the 16 lanes of a half-warp (the tx of one
// ty), as a butterfly reduce-scatter: with NV = 32 lane tx ends with values
// 2 tx and 2 tx + 1, with NV = 4 every lane ends with value tx / 4.
template <int NV>
__device__ __forceinline__ void reduce16(float v[NV], int tx) {
    int cnt = NV;
#pragma unroll
    for (int off = 8; off >= 1; off >>= 1) {
        if (cnt > 1) {
            const bool upper = tx & off;
            const int half = cnt / 2;
#pragma unroll
            for (int k = 0; k < NV / 2; ++k) {
                if (k < half) {
                    const float send = upper ? v[k] : v[k + half];
                    const float keep = upper ? v[k + half] : v[k];
                    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
                }
            }
            cnt = half;
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], off);
        }
    }
}

// W3 (64 x OUT) in shared memory with row k = 4 tx + j stored at (j * 16 + tx):
// the 16 lanes of a half-warp read 16 different rows without bank conflicts
template <int OUT>
__device__ __forceinline__ int w3_row(int k) {
    return (k & 3) * 16 + (k >> 2);
}

// ----------------------------------------------------------- forward ---
// Shared memory: weights (31 KB) and one 64 x 68 activation buffer that holds
// the input rows, then h1; h2 stays in registers and the output layer is a
// half-warp reduction, so four blocks fit on an SM.  With dsave, the row's
// SiLU derivatives are kept for the reverse pass: dsave[row][0..63] =
// SiLU'(z1), dsave[row][64..127] = SiLU'(z2).
constexpr int kSave = H1 + H2;
template <int OUT, int FIN>
__global__ void __launch_bounds__(kT) k_mlp_fwd(NetsOfLayer nets, const Tile* __restrict__ tiles,
                                               const float* __restrict__ rho, float* __restrict__ out,
                                               int out_stride, GhostOut gh, float* __restrict__ dsave,
                                               double* __restrict__ epart, int* __restrict__ flags) {
    pdl_enter();
    __shared__ __align__(8) uint64_t bar;
    extern __shared__ __align__(16) float sm[];
    float* sW1 = sm;                 // FIN x 64
    float* sW2 = sW1 + FIN * H1;     // 64 x 64
    float* sW3 = sW2 + H1 * H2;      // 64 x OUT (8 reserved), rows permuted (w3_row)
    float* sb1 = sW3 + H2 * 8;       // 64
    float* sb2 = sb1 + H1;           // 64
    float* sb3 = sb2 + H2;           // 8
    float* sA = sb3 + 8;             // input rows (stride FIN + 4), then h1 (stride LDH)
    const int tid = threadIdx.x;
    const Tile tl = tiles[blockIdx.x];
    if (tl.nrows <= 0) {  // padding entry of a fixed-size tile list
        if (OUT == 1 && epart && tid == 0) epart[blockIdx.x] = 0.0;
        return;
    }
    const NetDev& w = nets.e[tl.elem];
    if (tid == 0) {  // W1, W2 and the tile's input rows by bulk copies (TMA engine)
        bulk::mbar_init(&bar, 1);
        bulk::mbar_init_fence();
        const uint32_t xb = (uint32_t)tl.nrows * FIN * 4;
        bulk::mbar_expect_tx(&bar, (FIN * H1 + H1 * H2) * 4 + xb);
        bulk::bulk_g2s(sW1, w.W1, FIN * H1 * 4, &bar);
        bulk::bulk_g2s(sW2, w.W2, H1 * H2 * 4, &bar);
        bulk::bulk_g2s(sA, rho + (size_t)tl.row0 * FIN, xb, &bar);
    }
    for (int i = tid; i < H2 * OUT; i += kT) sW3[w3_row<OUT>(i / OUT) * OUT + i % OUT] = w.W3[i];
    for (int i = tid; i < H1; i += kT) sb1[i] = w.b1[i];
    for (int i = tid; i < H2; i += kT) sb2[i] = w.b2[i];
    if (tid < OUT) sb3[tid] = w.b3[tid];
    for (int i = tl.nrows * FIN + tid; i < kR * FIN; i += kT) sA[i] = 0.f;  // rows past the tile's end
    if (!staged(&bar, flags)) return;
    const int ty = tid >> 4, tx = tid & 15;
    float acc[4][4];
    // layer 1
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = sb1[4 * tx + j];
    mma_4x4<FIN, ldx<FIN>(), H1>(sA, sW1, ty, tx, acc);
    float ds[4][4];  // SiLU'(z1) (acc becomes h1)
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) ds[i][j] = silu_d(acc[i][j], acc[i][j]);
    if (dsave)
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (4 * ty + i < tl.nrows)
                *reinterpret_cast<float4*>(dsave + (size_t)(tl.row0 + 4 * ty + i) * kSave + 4 * tx) =
                    make_float4(ds[i][0], ds[i][1], ds[i][2], ds[i][3]);
    __syncthreads();  // every thread is done reading the input rows
#pragma unroll
    for (int i = 0; i < 4; ++i)
        *reinterpret_cast<float4*>(sA + (4 * ty + i) * LDH + 4 * tx) =
            make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    __syncthreads();
    // layer 2 (h2 stays in registers)
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = sb2[4 * tx + j];
    mma_4x4<H1, LDH, H2>(sA, sW2, ty, tx, acc);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) ds[i][j] = silu_d(acc[i][j], acc[i][j]);  // acc becomes h2
    if (dsave)
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (4 * ty + i < tl.nrows)
                *reinterpret_cast<float4*>(dsave + (size_t)(tl.row0 + 4 * ty + i) * kSave + H1 + 4 * tx) =
                    make_float4(ds[i][0], ds[i][1], ds[i][2], ds[i][3]);
    // layer 3: per-thread partial dot products over its 4 columns, reduced over tx
    float v[4 * OUT];
#pragma unroll
    for (int q = 0; q < 4 * OUT; ++q) v[q] = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float* w3 = sW3 + (j * 16 + tx) * OUT;
#pragma unroll
        for (int o = 0; o < OUT; ++o) {
            const float wv = w3[o];
#pragma unroll
            for (int i = 0; i < 4; ++i) v[i * OUT + o] = fmaf(acc[i][j], wv, v[i * OUT + o]);
        }
    }
    reduce16<4 * OUT>(v, tx);
    if (OUT == 1) {
        const int r = 4 * ty + (tx >> 2);
        const float e = v[0] + sb3[0];
        if ((tx & 3) == 0 && r < tl.nrows) out[(size_t)(tl.row0 + r) * out_stride] = e;
        if (epart) {  // the tile's energy in FP64, summed in a fixed order
            __syncthreads();  // every thread is done with the activation buffer
            double* sE = reinterpret_cast<double*>(sA);
            if ((tx & 3) == 0) sE[r] = r < tl.nrows ? (double)e : 0.0;
            __syncthreads();
            if (tid < 32) {
                double x = sE[tid] + sE[tid + 32];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                if (tid == 0) epart[blockIdx.x] = x;
            }
        }
    } else {
        const int r = 4 * ty + (tx >> 2), o = 2 * (tx & 3);
        if (r < tl.nrows) {
            const int64_t i = tl.row0 + r;
            const float y0 = v[0] + sb3[o], y1 = v[1] + sb3[o + 1];
            float* dst = out + (size_t)i * out_stride + o;
            dst[0] = y0;
            dst[1] = y1;
            if (gh.goff)  // the row's ghost images get the same coefficients (Fig. 4a)
                for (int64_t g = gh.goff[i]; g < gh.goff[i + 1] && g < gh.gcap; ++g) {
                    float* gd = out + (size_t)(gh.base + g) * out_stride + o;
                    gd[0] = y0;
                    gd[1] = y1;
                }
        }
    }
}

// ---------------------------------------------------------- backward ---
// rhobar = W1 (s1 * (W2 (s2 * (W3 ybar))))   per row, with s1 = SiLU'(z1) and
// s2 = SiLU'(z2) kept by the forward (dsave), so nothing is recomputed.
// Shared memory: the transposed weights, ybar, one 64 x 68 buffer (z2bar, then
// z1bar) and, with BBAR, the rhobar rows and the contraction weights.
//
// BBAR (Eq. 1's squares only): instead of writing rhobar, go on to the density
// adjoint's first step for the tile's rows, bbar_{a,m} = sum_k 2 w_a g_{a,k}
// rhobar_{l,k} W_{l,m,k} with g = b W recomputed from the b checkpoint (bck), and
// write the rows' adjoint records, bbar with the layer's c (the separate bbar
// kernel's work, without the rhobar round trip).
__device__ __forceinline__ float4 ld_save(const float* dsave, const Tile& tl, int r, int col) {
    if (r >= tl.nrows) return make_float4(0.f, 0.f, 0.f, 0.f);
    return __ldg(reinterpret_cast<const float4*>(dsave + (size_t)(tl.row0 + r) * kSave + col));
}

template <int OUT, int FIN, bool BBAR>
__global__ void __launch_bounds__(kT, 3) k_mlp_bwd(NetsOfLayer nets, const Tile* __restrict__ tiles,
                                               const float* __restrict__ dsave, const float* __restrict__ ybar,
                                               float* __restrict__ rhobar, const float* __restrict__ Wt,
                                               const float* __restrict__ bck, const float* __restrict__ coef,
                                               float* __restrict__ rec, GhostOut gh, int* __restrict__ flags) {
    pdl_enter();
    __shared__ __align__(8) uint64_t bar;
    extern __shared__ __align__(16) float sm[];
    float* sW1t = sm;                 // W1^T: 64 x FIN
    float* sW2t = sW1t + H1 * FIN;    // W2^T: 64 x 64
    float* sW3t = sW2t + H1 * H2;     // W3^T: OUT x 64 (8 rows reserved)
    float* sY = sW3t + 8 * H2;        // 64 x 8
    float* sG = sY + kR * 8;          // z2bar, then z1bar (stride LDH)
    float* sR = sG + kR * LDH;        // rhobar rows (BBAR, stride LDH)
    float* sWc = sR + kR * LDH;       // (L+1) x N_orb x N_phi contraction W^t, transposed per l (BBAR)
    const int tid = threadIdx.x;
    const Tile tl = tiles[blockIdx.x];
    if (tl.nrows <= 0) return;  // padding entry of a fixed-size tile list
    const int ty = tid >> 4, tx = tid & 15;
    // the thread's SiLU'(z2), in flight while the weights are staged
    float4 s2[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) s2[i] = ld_save(dsave, tl, 4 * ty + i, H1 + 4 * tx);
    const NetDev& w = nets.e[tl.elem];
    if (tid == 0) {  // W1^T, W2^T, W3^T by bulk copies (TMA engine)
        bulk::mbar_init(&bar, 1);
        bulk::mbar_init_fence();
        bulk::mbar_expect_tx(&bar, (H1 * FIN + H1 * H2 + OUT * H2) * 4);
        bulk::bulk_g2s(sW1t, w.W1t, H1 * FIN * 4, &bar);
        bulk::bulk_g2s(sW2t, w.W2t, H1 * H2 * 4, &bar);
        bulk::bulk_g2s(sW3t, w.W3t, OUT * H2 * 4, &bar);
    }
    if (BBAR)  // transposed per l: sWc[(l N_orb + k) N_phi + m] = W_{l,m,k}
        for (int i = tid; i < (LMAX + 1) * NPHI * NORB; i += kT) {
            const int l = i / (NPHI * NORB), m = (i / NORB) % NPHI, k = i % NORB;
            sWc[(l * NORB + k) * NPHI + m] = Wt[i];
        }
    for (int i = tid; i < kR * OUT; i += kT) {
        const int r = i / OUT, o = i % OUT;
        sY[r * 8 + o] = (OUT == 1) ? 1.f : (r < tl.nrows ? ybar[(size_t)(tl.row0 + r) * OUT + o] : 0.f);
    }
    if (!staged(&bar, flags)) return;
    // z2bar = (ybar W3^T) * s2 -> sG
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int o = 0; o < OUT; ++o) {
            const float y = sY[(4 * ty + i) * 8 + o];
            const float4 wv = *reinterpret_cast<const float4*>(sW3t + o * H2 + 4 * tx);
            v[0] = fmaf(y, wv.x, v[0]);
            v[1] = fmaf(y, wv.y, v[1]);
            v[2] = fmaf(y, wv.z, v[2]);
            v[3] = fmaf(y, wv.w, v[3]);
        }
        *reinterpret_cast<float4*>(sG + (4 * ty + i) * LDH + 4 * tx) =
            make_float4(v[0] * s2[i].x, v[1] * s2[i].y, v[2] * s2[i].z, v[3] * s2[i].w);
    }
    float4 s1[4];  // SiLU'(z1), in flight during the z1bar product
#pragma unroll
    for (int i = 0; i < 4; ++i) s1[i] = ld_save(dsave, tl, 4 * ty + i, 4 * tx);
    __syncthreads();
    // z1bar = (z2bar W2^T) * s1
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    mma_4x4<H2, LDH, H1>(sG, sW2t, ty, tx, acc);
    __syncthreads();  // everyone is done reading z2bar
#pragma unroll
    for (int i = 0; i < 4; ++i)
        *reinterpret_cast<float4*>(sG + (4 * ty + i) * LDH + 4 * tx) = make_float4(
            acc[i][0] * s1[i].x, acc[i][1] * s1[i].y, acc[i][2] * s1[i].z, acc[i][3] * s1[i].w);
    __syncthreads();
    // rhobar = z1bar W1^T  (64 x FIN): FIN / 4 column groups of 4 over the 16 tx
    for (int cg = tx; cg < FIN / 4; cg += 16) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        mma_4x4<H1, LDH, FIN>(sG, sW1t, ty, cg, acc);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = 4 * ty + i;
            if (BBAR) {
                *reinterpret_cast<float4*>(sR + r * LDH + 4 * cg) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
            } else if (r < tl.nrows) {
                *reinterpret_cast<float4*>(rhobar + (size_t)(tl.row0 + r) * FIN + 4 * cg) =
                    make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
            }
        }
    }
    if (!BBAR) return;
    __syncthreads();
    // four threads per row, record values v = q, q + 4, q + 8 (angular terms, then c and 0),
    // staged in shared memory (W1^T, W2^T are no longer needed) and stored as whole lines
    float* sRec = sW1t;
    const int r = tid >> 2, q = tid & 3;
    const size_t row = (size_t)(tl.row0 + r);
    const float* rb = sR + r * LDH;
#pragma unroll 1
    for (int v = q; v < NREC / NPHI && r < tl.nrows; v += 4) {
        float o[NPHI];
        if (v >= NANG) {
            rec_tail(coef, row, v, o);
            stage_rec(sRec, r, v, o);
            continue;
        }
        const int a = v, l = ang_l(a);
        const float4 b0 = __ldg(reinterpret_cast<const float4*>(bck + row * NB + a * NPHI));
        const float4 b1 = __ldg(reinterpret_cast<const float4*>(bck + row * NB + a * NPHI + 4));
        const float bm[NPHI] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int m = 0; m < NPHI; ++m) o[m] = 0.f;
        const float two_w = 2.f * ang_w(a);
        const float* wl = sWc + l * NORB * NPHI;
#pragma unroll 4
        for (int k = 0; k < NORB; ++k) {
            const float4 w0 = *reinterpret_cast<const float4*>(wl + k * NPHI);
            const float4 w1 = *reinterpret_cast<const float4*>(wl + k * NPHI + 4);
            const float wm[NPHI] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
            float g = 0.f;
#pragma unroll
            for (int m = 0; m < NPHI; ++m) g = fmaf(bm[m], wm[m], g);
            const float gb = two_w * g * rb[l * NORB + k];
#pragma unroll
            for (int m = 0; m < NPHI; ++m) o[m] = fmaf(gb, wm[m], o[m]);
        }
        stage_rec(sRec, r, v, o);
    }
    __syncthreads();
    flush_rec(sRec, tl.nrows, tl.row0, rec, gh, tid, kT);  // ghost images get the rows' records too (reverse exchange)
}

static_assert(NFEAT * H1 + H1 * H2 >= kR * kRecLd, "record staging must fit in the W1, W2 region");

template <int FIN>
constexpr size_t fwd_smem() { return sizeof(float) * (FIN * H1 + H1 * H2 + H2 * 8 + H1 + H2 + 8 + abuf<FIN>()); }
template <int FIN, bool BBAR>
constexpr size_t bwd_smem() {
    return sizeof(float) * (H1 * FIN + H1 * H2 + 8 * H2 + kR * 8 + kR * LDH +
                            (BBAR ? kR * LDH + (LMAX + 1) * NPHI * NORB : 0));
}
void ensure_attrs() {
    // once per device, safe under concurrent first calls
    static std::mutex mu;
    static uint64_t done = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 64 && ((done >> dev) & 1)) return;
#define REANN_SMEM(K, BYTES) cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(BYTES))
    REANN_SMEM((k_mlp_fwd<1, NFEAT>), fwd_smem<NFEAT>());
    REANN_SMEM((k_mlp_fwd<NPHI, NFEAT>), fwd_smem<NFEAT>());
    REANN_SMEM((k_mlp_fwd<1, NFEAT_P>), fwd_smem<NFEAT_P>());
    REANN_SMEM((k_mlp_fwd<NPHI, NFEAT_P>), fwd_smem<NFEAT_P>());
    REANN_SMEM((k_mlp_bwd<1, NFEAT, false>), (bwd_smem<NFEAT, false>()));
    REANN_SMEM((k_mlp_bwd<NPHI, NFEAT, false>), (bwd_smem<NFEAT, false>()));
    REANN_SMEM((k_mlp_bwd<1, NFEAT, true>), (bwd_smem<NFEAT, true>()));
    REANN_SMEM((k_mlp_bwd<NPHI, NFEAT, true>), (bwd_smem<NFEAT, true>()));
    REANN_SMEM((k_mlp_bwd<1, NFEAT_P, false>), (bwd_smem<NFEAT_P, false>()));
    REANN_SMEM((k_mlp_bwd<NPHI, NFEAT_P, false>), (bwd_smem<NFEAT_P, false>()));
#undef REANN_SMEM
    if (dev < 64) done |= (uint64_t)1 << dev;
}

NetsOfLayer layer_nets(const NetTable& t, int layer) {
    NetsOfLayer n;
    for (int e = 0; e < MAX_ELEM; ++e) n.e[e] = t.net[layer][e];
    return n;
}

}  // namespace

cudaError_t launch_mlp_fwd_f32(cudaStream_t s, const reann_nlist* nl, const NetTable& nets, int t, bool energy,
                               const float* rho, float* out, int out_stride, bool pairs, GhostOut gh, float* dsave,
                               double* epart, int* flags) {
    const int nt = (int)tiles_of(nl);
    if (nt == 0) return cudaSuccess;
    ensure_attrs();
    const NetsOfLayer ln = layer_nets(nets, t);
#define REANN_FWD(O, F) \
    k_mlp_fwd<O, F><<<nt, kT, fwd_smem<F>(), s>>>(ln, nl->tiles, rho, out, out_stride, gh, dsave, epart, flags)
    if (pairs) {
        if (energy)
            REANN_FWD(1, NFEAT_P);
        else
            REANN_FWD(NPHI, NFEAT_P);
    } else {
        if (energy)
            REANN_FWD(1, NFEAT);
        else
            REANN_FWD(NPHI, NFEAT);
    }
#undef REANN_FWD
    return cudaGetLastError();
}

cudaError_t launch_mlp_bwd_f32(cudaStream_t s, const reann_nlist* nl, const NetTable& nets, int t, bool energy,
                               const float* dsave, const float* ybar, float* rhobar, int* flags, bool pairs,
                               const float* Wt, const float* bck, const float* coef, float* rec, GhostOut gh) {
    const int nt = (int)tiles_of(nl);
    if (nt == 0) return cudaSuccess;
    ensure_attrs();
    const NetsOfLayer ln = layer_nets(nets, t);
#define REANN_BWD(O, F, B)                                                                                      \
    k_mlp_bwd<O, F, B><<<nt, kT, bwd_smem<F, B>(), s>>>(ln, nl->tiles, dsave, ybar, rhobar, B ? Wt : nullptr, \
                                                        B ? bck : nullptr, B ? coef : nullptr, B ? rec : nullptr, \
                                                        B ? gh : GhostOut{}, flags)
    if (pairs) {
        if (energy)
            REANN_BWD(1, NFEAT_P, false);
        else
            REANN_BWD(NPHI, NFEAT_P, false);
    } else if (rec) {
        if (energy)
            REANN_BWD(1, NFEAT, true);
        else
            REANN_BWD(NPHI, NFEAT, true);
    } else {
        if (energy)
            REANN_BWD(1, NFEAT, false);
        else
            REANN_BWD(NPHI, NFEAT, false);
    }
#undef REANN_BWD
    return cudaGetLastError();
}

}  // namespace reann
