// Periodic neighbour list with a skin and the ghost (periodic-image) map.
//
// Sec. 2.2: one neighbour list of radius r_c serves every message-passing
// layer; Sec. 1 motivates the skin (rebuild only after atoms moved skin/2).
// On one GPU the paper's ghost atoms (Fig. 3a, Fig. 4a) become ghost slots
// N..N+G-1: every periodic image that lies within r_c + skin of the cell,
// pointing at its owner atom and carrying an integer image shift.
//
// Build (all deterministic):
//   1. wrap positions into the cell in FP64 and key every atom by
//      (element, cell bin) -- on the first build and every 8th rebuild; the
//      rebuilds in between keep the previous internal order (k_wrap_keep);
//   2. counting sort by key -> internal order (element-major so the atomic
//      networks see contiguous per-element tiles, spatially sorted inside an
//      element so neighbour gathers stay local);
//   3. enumerate ghost images (count while gathering, scan, fill while keying);
//   4. bin owned + ghost slots into an extended cell grid (counting sort);
//   5. warp per owned atom: scan the stencil bins (in a rectangular cell each
//      column trimmed to the sphere), FP32 pre-test with a margin, FP64 exact
//      test for pairs near r_c + skin, ballot-compacted writes into a
//      fixed-stride row.
// The first build sizes the ghost and row capacities (one host round trip);
// every later rebuild re-runs the same kernels into the resident buffers
// without allocating or synchronising, so it can sit inside a CUDA graph.
// The FP64 test follows one fixed arithmetic order (no FMA contraction):
//   r = (x_w,o - x_w,i) + S(n), S(n)_d = (n0 H0d + n1 H1d) + n2 H2d,
//   d^2 = (r0 r0 + r1 r1) + r2 r2 < (r_c + skin)^2.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace reann {
namespace {

constexpr int kScanThreads = 256;
// Per-slot kernels whose time goes to FP64 arithmetic (wrapping, image shifts, halo tests) run
// in 64-thread blocks: 24,576 atoms then spread over all SMs' FP64 units (256-thread blocks
// left a third of the SMs without work)
constexpr int kFp64Threads = 64;

__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }

// n h rounded as the FP64 product, without the FP64 multiply for the image shifts -1, 0, 1
// (0 h is a zero with the sign of h): GB300's FP64 pipe is narrow, and the rebuild's
// per-slot kernels are bound by it
__device__ __forceinline__ double smul(int n, double h) {
    if (n == 0) return copysign(0.0, h);
    if (n == 1) return h;
    if (n == -1) return -h;
    return dmul((double)n, h);
}

__device__ __forceinline__ void shift_vec(const CellGeom& g, int n0, int n1, int n2, double s[3]) {
#pragma unroll
    for (int d = 0; d < 3; ++d) s[d] = dadd(dadd(smul(n0, g.h[d]), smul(n1, g.h[3 + d])), smul(n2, g.h[6 + d]));
}
// the same vector with plain FP64 products (bitwise equal): for the neighbour search's
// boundary test, where the lanes of a warp hold different shifts and branches diverge
__device__ __forceinline__ void shift_vec_mul(const CellGeom& g, int n0, int n1, int n2, double s[3]) {
#pragma unroll
    for (int d = 0; d < 3; ++d)
        s[d] = dadd(dadd(dmul((double)n0, g.h[d]), dmul((double)n1, g.h[3 + d])), dmul((double)n2, g.h[6 + d]));
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ int pack_shift(int a, int b, int c) { return (a + 128) | ((b + 128) << 8) | ((c + 128) << 16); }
__device__ __forceinline__ void unpack_shift(int p, int& a, int& b, int& c) {
    a = (p & 255) - 128;
    b = ((p >> 8) & 255) - 128;
    c = ((p >> 16) & 255) - 128;
}

// ghosts in use: the device count clamped to the capacity
__device__ __forceinline__ int64_t ghosts_in_use(const int32_t* g_count, int64_t g_cap) {
    const int64_t g = *g_count;
    return g < g_cap ? g : g_cap;
}

// 1. wrap + key (caller order)
// Wrap one position into the cell in FP64 (fixed operation order): fractional
// coordinates f = x . hinv, integer shift m = floor(f), wrapped Cartesian
// x - m.H and fractional f - m; `bad` for a non-finite or absurd position.
__device__ __forceinline__ void wrap_one(const CellGeom& g, const double x_in[3], double xw[3], double fw[3], int m[3],
                                         bool& bad) {
    double x[3] = {x_in[0], x_in[1], x_in[2]};
    double fr[3];
    bad = !(isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2]));
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        fr[k] = dadd(dadd(dmul(x[0], g.hinv[k]), dmul(x[1], g.hinv[3 + k])), dmul(x[2], g.hinv[6 + k]));
        if (!isfinite(fr[k]) || fabs(fr[k]) > 1e9) bad = true;
    }
    if (bad) {
#pragma unroll
        for (int k = 0; k < 3; ++k) fr[k] = 0.0, x[k] = 0.0;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) m[k] = (int)floor(fr[k]);
    double s[3];
    shift_vec(g, m[0], m[1], m[2], s);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        xw[k] = dsub(x[k], s[k]);
        fw[k] = dsub(fr[k], (double)m[k]);
    }
}

__global__ void k_wrap_key(const int* __restrict__ gate, int64_t n, const double* __restrict__ pos, const int32_t* __restrict__ species, int n_elem,
                           CellGeom g, double* __restrict__ xw, double* __restrict__ fw, int32_t* __restrict__ mw,
                           int32_t* __restrict__ key, int32_t* __restrict__ counts, int* __restrict__ flags,
                           double* __restrict__ ref) {
    pdl_enter();
    if (gate && *gate == 0) return;  // rebuild (or this rebuild's sort) not needed
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
    // the positions of this build, for the moved-by-more-than-skin/2 test
    ref[3 * i] = x[0];
    ref[3 * i + 1] = x[1];
    ref[3 * i + 2] = x[2];
    int sp = species[i];
    if (sp < 0 || sp >= n_elem) {
        atomicOr(&flags[FLAG_SPECIES], 1);
        sp = 0;
    }
    double xwi[3], f[3];
    int m[3];
    bool bad;
    wrap_one(g, x, xwi, f, m, bad);
    if (bad) atomicOr(&flags[FLAG_GEOM], 1);
    int b[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        xw[3 * i + k] = xwi[k];
        fw[3 * i + k] = f[k];
        mw[3 * i + k] = m[k];
        b[k] = clampi((int)floor(f[k] * g.nb[k]), 0, g.nb[k] - 1);
    }
    int nbins = g.nb[0] * g.nb[1] * g.nb[2];
    const int k = sp * nbins + (b[0] * g.nb[1] + b[1]) * g.nb[2] + b[2];
    key[i] = k;
    atomicAdd(&counts[k], 1);  // the counting sort's histogram
}

// ---- deterministic counting sort ------------------------------------------

// Exclusive scan of `in` (n entries, int32) into out[0..n], one launch over
// tiles of kScanTile entries, one block per tile, joined by decoupled look-back
// (D. Merrill and M. Garland, Single-pass Parallel Prefix Scan with Decoupled
// Look-back, NVIDIA technical report NVR-2016-002): a block takes its tile
// number from a ticket counter (so every lower tile's block has started),
// publishes its tile's sum, walks back over the published words of the tiles
// before it (one warp, 32 words per read) until one carries an inclusive
// prefix, and publishes its own inclusive prefix.  A tile is loaded and stored
// coalesced through shared memory (padded one word per 32 against bank
// conflicts), each thread scans kScanPer consecutive entries, and a two-level
// warp scan joins the threads.
// The status words (scan_tiles(n) + 2: one per tile, the ticket, the count of
// finished blocks) start at zero; the last block to finish sets them back to
// zero.  A wait on a lower tile is bounded (kScanSpin polls, seconds): when it
// runs out the block sets FLAG_TIMEOUT and goes on with a wrong carry.
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;
constexpr int32_t kScanAgg = 1 << 30, kScanIncl = (int32_t)0x80000000u, kScanVal = (1 << 30) - 1;
constexpr long long kScanSpin = 1ll << 22;

__global__ void __launch_bounds__(kScanThreads) k_scan(const int* __restrict__ gate, int64_t n,
                                                       const int32_t* __restrict__ in, int32_t* __restrict__ out,
                                                       int32_t* __restrict__ status, int* __restrict__ flags) {
    pdl_enter();
    if (gate && *gate == 0) return;  // rebuild not needed this step
    __shared__ int32_t buf[kScanTile + kScanTile / 32];
    __shared__ int32_t warp_sums[kScanThreads / 32];
    __shared__ int32_t s_tile, s_carry;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int nb = (int)gridDim.x;
    if (tid == 0) s_tile = atomicAdd(&status[nb], 1);
    __syncthreads();
    const int tile = s_tile;
    const int64_t base = (int64_t)tile * kScanTile;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        const int x = k * kScanThreads + tid;
        buf[x + x / 32] = base + x < n ? in[base + x] : 0;
    }
    __syncthreads();
    int32_t v[kScanPer];
    int32_t local = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        const int x = tid * kScanPer + k;
        v[k] = buf[x + x / 32];
        local += v[k];
    }
    int32_t incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[w] = incl;
    __syncthreads();
    if (w == 0) {
        int32_t t = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kScanThreads / 32) warp_sums[lane] = t;  // inclusive
    }
    __syncthreads();
    const int32_t total = warp_sums[kScanThreads / 32 - 1];
    if (w == 0) {  // look-back by one warp: lane l reads the word of tile top - l
        int32_t carry = 0;
        if (tile == 0) {
            if (lane == 0) atomicExch(&status[0], kScanIncl | total);
        } else {
            if (lane == 0) atomicExch(&status[tile], kScanAgg | total);
            bool late = false;
            for (int top = tile - 1; top >= 0; top -= 32) {
                const int q = top - lane;
                int32_t word = kScanIncl;  // below tile 0: an inclusive zero
                if (q >= 0) {
                    long long spins = 0;
                    do {
                        word = *reinterpret_cast<volatile int32_t*>(status + q);
                    } while (word == 0 && ++spins <= kScanSpin);
                    if (word == 0) {
                        late = true;
                        word = kScanIncl;
                    }
                }
                // the nearest tile with an inclusive prefix ends the walk
                const unsigned inc = __ballot_sync(0xffffffffu, (word & kScanIncl) != 0);
                const int stop = inc ? __ffs(inc) - 1 : 31;
                int32_t val = lane <= stop ? (word & kScanVal) : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
                carry += val;
                if (inc) break;
            }
            if (__any_sync(0xffffffffu, late) && lane == 0) atomicOr(&flags[FLAG_TIMEOUT], 1);
            if (lane == 0) atomicExch(&status[tile], kScanIncl | (carry + total));
        }
        if (lane == 0) s_carry = carry;
    }
    __syncthreads();
    int32_t run = s_carry + (w > 0 ? warp_sums[w - 1] : 0) + incl - local;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        const int x = tid * kScanPer + k;
        buf[x + x / 32] = run;
        run += v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        const int x = k * kScanThreads + tid;
        if (base + x < n) out[base + x] = buf[x + x / 32];
    }
    if (tid == 0) {
        if (tile == nb - 1) out[n] = s_carry + total;
        __threadfence();
        if (atomicAdd(&status[nb + 1], 1) == nb - 1) {  // every block is past its look-back
            for (int q = 0; q < nb + 2; ++q) status[q] = 0;
        }
    }
}

inline int64_t scan_tiles(int64_t n) { return n > 0 ? (n + kScanTile - 1) / kScanTile : 1; }
inline int64_t scan_status_words(int64_t n) { return scan_tiles(n) + 2; }

// out[0..n] = exclusive scan of in[0..n), out[n] the total; status: scan_status_words(n)
// zeroed words
static void scan_exclusive(cudaStream_t s, const int* gate, int64_t n, const int32_t* in, int32_t* out,
                           int32_t* status, int* flags) {
    launch_pdl(k_scan, (unsigned)scan_tiles(n), kScanThreads, 0, s, gate, n, in, out, status, flags);
}

__global__ void k_scatter(const int* __restrict__ gate, int64_t n, const int32_t* __restrict__ key,
                          const int32_t* __restrict__ start, int32_t* __restrict__ counts,
                          int32_t* __restrict__ order) {
    pdl_enter();
    if (gate && *gate == 0) return;  // rebuild not needed this step
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = key[i];
    // counting the histogram back down: the bucket's entries take its slots from the top,
    // and the counts end at zero, ready for the next sort's histogram
    int p = start[k] + atomicSub(&counts[k], 1) - 1;
    order[p] = (int32_t)i;
}

// Deterministic placement inside each bucket: the entry at position p of the
// atomic-order scatter moves to start[b] + (number of entries of its bucket with
// a smaller index).  One thread per entry, each scanning its own bucket (buckets
// hold tens of entries); entries of buckets >= sorted_keys keep their position.
// With `pin`, the entry's FP32 position follows it into sorted order, its index
// carried in .w (bit pattern), so that the search reads candidates contiguously.
__global__ void k_bucket_rank(const int* __restrict__ gate, int64_t n, const int32_t* __restrict__ key,
                              const int32_t* __restrict__ start, const int32_t* __restrict__ scattered,
                              int64_t sorted_keys, int32_t* __restrict__ order, const float4* __restrict__ pin,
                              float4* __restrict__ pout) {
    pdl_enter();
    if (gate && *gate == 0) return;  // rebuild not needed this step
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int32_t v = scattered[p];
    const int32_t b = key[v];
    int64_t dst = p;
    if (b < sorted_keys) {
        const int lo = start[b], hi = start[b + 1];
        int rank = 0;
        for (int q = lo; q < hi; ++q) rank += scattered[q] < v;
        dst = lo + rank;
    }
    order[dst] = v;
    if (pin) {
        const float4 x = pin[v];
        pout[dst] = make_float4(x.x, x.y, x.z, __int_as_float(v));
    }
}

// an axis's image interval [lo, hi] in one word (|lo|, |hi| < 128)
__device__ __forceinline__ int32_t pack_halo(int lo, int hi) { return (lo + 128) | ((hi + 128) << 8); }
__device__ __forceinline__ void unpack_halo(int32_t p, int& lo, int& hi) {
    lo = (p & 255) - 128;
    hi = ((p >> 8) & 255) - 128;
}

// admissible image shifts of one axis: those keeping f + a within (-reach, 1 + reach),
// an interval because the test is monotone in a
__device__ __forceinline__ void halo_interval(const CellGeom& g, int k, double f, int& lo, int& hi) {
    lo = 1;
    hi = 0;
    for (int a = -g.nmax[k]; a <= g.nmax[k]; ++a) {
        const double v = f + a;
        if (v > -g.reach[k] && v < 1.0 + g.reach[k]) {
            if (lo > hi) lo = a;
            hi = a;
        }
    }
}

// 2. gather per-atom arrays into internal order
// (also each atom's number of ghost images: the product of its per-axis intervals
// minus the zero shift, which wrapped coordinates in [0, 1) always admit)
__global__ void k_gather_internal(const int* __restrict__ gate, int64_t n, CellGeom g, const int32_t* __restrict__ perm,
                                  const double* __restrict__ xw_c, const double* __restrict__ fw_c,
                                  const int32_t* __restrict__ mw_c, const int32_t* __restrict__ sp_c,
                                  double* __restrict__ xw, double* __restrict__ fw, int32_t* __restrict__ mw,
                                  int32_t* __restrict__ sp, int32_t* __restrict__ gcnt, int32_t* __restrict__ halo) {
    pdl_enter();
    if (gate && *gate == 0) return;  // rebuild not needed this step
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = perm[i];
    int cnt = 1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        xw[3 * i + k] = xw_c[3 * (int64_t)c + k];
        const double f = fw_c[3 * (int64_t)c + k];
        fw[3 * i + k] = f;
        mw[3 * i + k] = mw_c[3 * (int64_t)c + k];
        int lo, hi;
        halo_interval(g, k, f, lo, hi);
        halo[3 * i + k] = pack_halo(lo, hi);
        cnt *= hi - lo + 1;
    }
    sp[i] = sp_c[c];
    gcnt[i] = cnt - 1;
}

// Rebuilds between sorts: every kResortPeriod-th rebuild sorts the owned atoms
// again; the others keep the internal order of the last sort, and only wrap the
// new positions (straight into internal order) and count their ghost images.
// The list itself (ghosts, extended bins, search) is rebuilt in full either way.
// state[0] counts rebuilds since the last sort; state[1] gates the sort path and
// state[2] the keep-order path for this rebuild (both 0 when it is gated off).
constexpr int kResortPeriod = 8;

__global__ void k_rebuild_gates(const int* __restrict__ gate, int* __restrict__ state) {
    pdl_enter();
    const bool run = !gate || *gate != 0;
    const bool sort = run && state[0] >= kResortPeriod;
    if (run) state[0] = sort ? 1 : state[0] + 1;
    state[1] = sort ? 1 : 0;
    state[2] = run && !sort ? 1 : 0;
}

// the keep-order path: wrap the caller-order positions of the internal atoms i
// (the same arithmetic as k_wrap_key) and count their ghost images
__global__ void k_wrap_keep(const int* __restrict__ gate, int64_t n, CellGeom g, const double* __restrict__ pos,
                            const int32_t* __restrict__ perm, double* __restrict__ xw, double* __restrict__ fw,
                            int32_t* __restrict__ mw, int32_t* __restrict__ gcnt, int32_t* __restrict__ halo,
                            int* __restrict__ flags, double* __restrict__ ref) {
    pdl_enter();
    if (gate && *gate == 0) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t c = perm[i];
    const double x[3] = {pos[3 * c], pos[3 * c + 1], pos[3 * c + 2]};
    ref[3 * c] = x[0];
    ref[3 * c + 1] = x[1];
    ref[3 * c + 2] = x[2];
    double xwi[3], f[3];
    int m[3];
    bool bad;
    wrap_one(g, x, xwi, f, m, bad);
    if (bad) atomicOr(&flags[FLAG_GEOM], 1);
    int cnt = 1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        xw[3 * i + k] = xwi[k];
        fw[3 * i + k] = f[k];
        mw[3 * i + k] = m[k];
        int lo, hi;
        halo_interval(g, k, f[k], lo, hi);
        halo[3 * i + k] = pack_halo(lo, hi);
        cnt *= hi - lo + 1;
    }
    gcnt[i] = cnt - 1;
}

// 3-4. ghost images (fractional coordinate within (-reach, 1 + reach) on every
// axis) and the extended binning of owned + ghost slots.
// Extended key and FP32 position of slot (owner o, image shift (a, b, c)):
__device__ __forceinline__ void ext_slot(const CellGeom& g, const double* __restrict__ xw, const double* __restrict__ fw,
                                         int64_t o, int a, int b, int c, int32_t* __restrict__ key,
                                         int32_t* __restrict__ counts, float4* __restrict__ p32, int64_t s) {
    double f[3] = {fw[3 * o] + a, fw[3 * o + 1] + b, fw[3 * o + 2] + c};
    int bx[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) bx[k] = clampi((int)floor(f[k] * g.ns[k]) + g.pad[k], 0, g.nbx[k] - 1);
    const int k = (bx[0] * g.nbx[1] + bx[1]) * g.nbx[2] + bx[2];
    key[s] = k;
    atomicAdd(&counts[k], 1);  // the extended sort's histogram
    double sv[3];
    shift_vec(g, a, b, c, sv);
    p32[s] = make_float4((float)(xw[3 * o] + sv[0]), (float)(xw[3 * o + 1] + sv[1]), (float)(xw[3 * o + 2] + sv[2]), 0.f);
}

// ext_slot for the atom itself (shift 0): f + 0 and x + 0 without the FP64 adds (they
// differ at most in the sign of a zero, which no bin or distance sees)
__device__ __forceinline__ void ext_slot_self(const CellGeom& g, const double* __restrict__ xw,
                                              const double* __restrict__ fw, int64_t o, int32_t* __restrict__ key,
                                              int32_t* __restrict__ counts, float4* __restrict__ p32) {
    int bx[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) bx[k] = clampi((int)floor(fw[3 * o + k] * g.ns[k]) + g.pad[k], 0, g.nbx[k] - 1);
    const int k = (bx[0] * g.nbx[1] + bx[1]) * g.nbx[2] + bx[2];
    key[o] = k;
    atomicAdd(&counts[k], 1);
    p32[o] = make_float4((float)xw[3 * o], (float)xw[3 * o + 1], (float)xw[3 * o + 2], 0.f);
}

// 3-4. ghost images and the extended binning, one thread per slot of [0, n + g_cap):
// owned slot i keys itself and fills its images' slots [goff[i], goff[i+1])
// (owner, shift, key, FP32 position) in the order a, b, c of the per-axis
// intervals; unused ghost capacity sorts last.
__global__ void k_ghosts_ext(const int* __restrict__ gate, int64_t n, CellGeom g, const double* __restrict__ xw,
                             const double* __restrict__ fw, const int32_t* __restrict__ goff, int64_t g_cap,
                             int32_t* __restrict__ owner, int32_t* __restrict__ shift, int32_t* __restrict__ key,
                             int32_t* __restrict__ counts, float4* __restrict__ p32, int32_t dead_key,
                             const int32_t* __restrict__ halo, int* __restrict__ flags) {
    pdl_enter();
    if (gate && *gate == 0) return;  // rebuild not needed this step
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n + g_cap) return;
    if (s >= n) {
        if (s >= n + ghosts_in_use(goff + n, g_cap)) {
            key[s] = dead_key;
            atomicAdd(&counts[dead_key], 1);
            p32[s] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        return;  // slots in use are written by their owners
    }
    ext_slot_self(g, xw, fw, s, key, counts, p32);
    int lo[3], hi[3];  // the intervals the wrap computed
#pragma unroll
    for (int k = 0; k < 3; ++k) unpack_halo(halo[3 * s + k], lo[k], hi[k]);
    int64_t q = goff[s];
    for (int a = lo[0]; a <= hi[0]; ++a)
        for (int b = lo[1]; b <= hi[1]; ++b)
            for (int c = lo[2]; c <= hi[2]; ++c) {
                if (a == 0 && b == 0 && c == 0) continue;
                if (q < g_cap) {
                    owner[q] = (int32_t)s;
                    shift[q] = pack_shift(a, b, c);
                    ext_slot(g, xw, fw, s, a, b, c, key, counts, p32, n + q);
                } else {
                    atomicOr(&flags[FLAG_GHOST_OVERFLOW], 1);
                }
                ++q;
            }
}

// 5. neighbour search: one warp per owned atom.  For each (x, y) column of the
// stencil the z-run of bins is one contiguous range of the bin-sorted slots;
// lane l takes column l of a batch of 32, a warp scan of the run lengths
// concatenates them, and the warp walks the concatenation 32 candidates at a
// time (a binary search over the scanned lengths maps a candidate to its
// column), reading the sorted FP32 positions with their slot index in .w.
// Candidates come in the same order as a bin-by-bin walk (x, then y, then z).
__global__ void __launch_bounds__(256) k_nbr_search(const int* __restrict__ gate, int64_t n, CellGeom g,
                                                   const double* __restrict__ xw, const int32_t* __restrict__ owner,
                                                   const int32_t* __restrict__ shift, const float4* __restrict__ p32,
                                                   const float4* __restrict__ p32s, const int32_t* __restrict__ bstart,
                                                   const int32_t* __restrict__ ekey,
                                                   int stride, int32_t* __restrict__ nbr, int32_t* __restrict__ cnt_out,
                                                   int* __restrict__ flags) {
    pdl_enter();
    if (gate && *gate == 0) return;  // rebuild not needed this step
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    const float4 pi = p32[i];
    const double xi[3] = {xw[3 * i], xw[3 * i + 1], xw[3 * i + 2]};
    // the atom's own bin, as the extended keying computed it (its FP64 floor, evaluated by
    // every lane here, kept a third of GB300's narrow FP64 pipe busy)
    int b[3];
    {
        const int key = ekey[i];
        b[2] = key % g.nbx[2];
        b[1] = (key / g.nbx[2]) % g.nbx[1];
        b[0] = key / (g.nbx[2] * g.nbx[1]);
    }
    const int x0 = max(0, b[0] - g.sw[0]), x1 = min(g.nbx[0] - 1, b[0] + g.sw[0]);
    const int y0 = max(0, b[1] - g.sw[1]), y1 = min(g.nbx[1] - 1, b[1] + g.sw[1]);
    const int z0 = max(0, b[2] - g.sw[2]), z1 = min(g.nbx[2] - 1, b[2] + g.sw[2]);
    const int ny = y1 - y0 + 1, ncol = (x1 - x0 + 1) * ny;
    const float lo2 = g.rcut2_f - g.margin, hi2 = g.rcut2_f + g.margin;
    int count = 0;
    int32_t* row = nbr + (size_t)i * stride;
    for (int cb = 0; cb < ncol; cb += 32) {
        int st = 0, len = 0;
        if (cb + lane < ncol) {
            const int col = cb + lane;
            const int bx = x0 + col / ny, by = y0 + col % ny;
            const int bin0 = (bx * g.nbx[1] + by) * g.nbx[2];
            int za = z0, zb = z1;
            if (g.ortho) {
                // rectangular cell: bin b of axis k spans [(b - pad) w, (b - pad + 1) w) in Cartesian
                // coordinates; keep the z-bins within sqrt(r^2 - rho^2) of the atom, rho being the
                // atom's distance to the column.  FP32 (the FP64 units are slow) with 2e-3 A of slack,
                // far above the rounding of coordinates and bin edges.
                constexpr float kSlack = 2e-3f;
                const float lx = (bx - g.pad[0]) * g.binw[0], ly = (by - g.pad[1]) * g.binw[1];
                const float dx = fmaxf(0.f, fmaxf(lx - pi.x, pi.x - (lx + g.binw[0])) - kSlack);
                const float dy = fmaxf(0.f, fmaxf(ly - pi.y, pi.y - (ly + g.binw[1])) - kSlack);
                const float rho2 = dx * dx + dy * dy;
                if (rho2 >= g.rcut2_f) {
                    zb = za - 1;
                } else {
                    const float hz = sqrtf(g.rcut2_f - rho2) + kSlack;
                    za = max(z0, (int)floorf((pi.z - hz) * g.binw_inv[2]) + g.pad[2]);
                    zb = min(z1, (int)floorf((pi.z + hz) * g.binw_inv[2]) + g.pad[2]);
                }
            }
            if (za <= zb) {
                st = bstart[bin0 + za];
                len = bstart[bin0 + zb + 1] - st;
            }
        }
        int pref = len;  // inclusive scan of the run lengths
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, pref, o);
            if (lane >= o) pref += y;
        }
        const int total = __shfl_sync(FULL, pref, 31);
        for (int t0 = 0; t0 < total; t0 += 32) {
            const int t = t0 + lane;
            // column r of candidate t: the first lane whose inclusive prefix exceeds t
            int lo = 0, hi = 31;
#pragma unroll
            for (int step = 0; step < 5; ++step) {
                const int mid = (lo + hi) >> 1;
                if (__shfl_sync(FULL, pref, mid) > t) hi = mid;
                else lo = mid + 1;
            }
            const int r = min(lo, 31);
            const int c = __shfl_sync(FULL, st, r) + t - (__shfl_sync(FULL, pref, r) - __shfl_sync(FULL, len, r));
            bool hit = false;
            int j = -1;
            if (t < total) {
                const float4 pj = p32s[c];
                j = __float_as_int(pj.w);
                if (j != (int)i) {
                    const float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
                    const float d2 = dx * dx + dy * dy + dz * dz;
                    if (d2 < lo2 && d2 > 1e-4f) {
                        hit = true;
                    } else if (d2 <= hi2) {
                        // exact FP64 decision (and the coincident-atom check)
                        int64_t o = j;
                        int a0 = 0, a1 = 0, a2 = 0;
                        if (j >= n) {
                            o = owner[j - n];
                            unpack_shift(shift[j - n], a0, a1, a2);
                        }
                        double sv[3];
                        shift_vec_mul(g, a0, a1, a2, sv);
                        double rr[3];
#pragma unroll
                        for (int k = 0; k < 3; ++k) rr[k] = dadd(dsub(xw[3 * o + k], xi[k]), sv[k]);
                        const double dd = dadd(dadd(dmul(rr[0], rr[0]), dmul(rr[1], rr[1])), dmul(rr[2], rr[2]));
                        hit = dd < g.rcut2;
                        if (dd < 1e-16) atomicOr(&flags[FLAG_GEOM], 2);
                    }
                }
            }
            const unsigned m = __ballot_sync(FULL, hit);
            if (hit) {
                const int p = count + __popc(m & ((1u << lane) - 1u));
                if (p < stride) row[p] = j;
            }
            count += __popc(m);
        }
    }
    if (lane == 0) {
        cnt_out[i] = min(count, stride);
        if (count > stride) atomicOr(&flags[FLAG_NBR_OVERFLOW], 1);
        atomicMax(&flags[FLAG_MAXNBR], count);
    }
}

// per evaluation: refresh owned + ghost positions (FP64 -> hi/lo FP32 pair)
// (with c0, also the first layer's coefficients c0[species] of every slot)
__global__ void k_refresh(int64_t n, const int32_t* __restrict__ g_count, int64_t g_cap, CellGeom g,
                          const double* __restrict__ pos, const int32_t* __restrict__ perm,
                          const int32_t* __restrict__ wrapm, const int32_t* __restrict__ owner,
                          const int32_t* __restrict__ shift, float4* __restrict__ hi, float4* __restrict__ lo,
                          const int32_t* __restrict__ species, const float* __restrict__ c0,
                          float* __restrict__ coef) {
    pdl_enter();
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n + ghosts_in_use(g_count, g_cap)) return;
    int64_t o = s;
    int a = 0, b = 0, c = 0;
    if (s >= n) {
        o = owner[s - n];
        unpack_shift(shift[s - n], a, b, c);
    }
    const int64_t cidx = perm[o];
    double sm[3], sv[3];
    shift_vec(g, wrapm[3 * o], wrapm[3 * o + 1], wrapm[3 * o + 2], sm);
    shift_vec(g, a, b, c, sv);
    double x[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) x[k] = (pos[3 * cidx + k] - sm[k]) + sv[k];
    float h[3], l[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        h[k] = (float)x[k];
        l[k] = (float)(x[k] - (double)h[k]);
    }
    hi[s] = make_float4(h[0], h[1], h[2], 0.f);
    lo[s] = make_float4(l[0], l[1], l[2], 0.f);
    if (c0) {
        const float4* src = reinterpret_cast<const float4*>(c0 + species[o] * NPHI);
        float4* dst = reinterpret_cast<float4*>(coef + (size_t)s * NPHI);
        dst[0] = src[0];
        dst[1] = src[1];
    }
}

// per evaluation: live (d < r_c) entries of every row, moved to the row's front
__global__ void __launch_bounds__(256) k_live(int64_t n, int stride, float rc2, float band,
                                             const int32_t* __restrict__ nbr,
                                             const int32_t* __restrict__ cnt, const float4* __restrict__ hi,
                                             const float4* __restrict__ lo, int32_t* __restrict__ live,
                                             int32_t* __restrict__ live_cnt, int* __restrict__ flags) {
    pdl_enter();
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    const float4 hi_i = hi[i], lo_i = lo[i];
    const int c = cnt[i];
    const int32_t* row = nbr + (size_t)i * stride;
    int32_t* out = live + (size_t)i * stride;
    int count = 0;
    for (int base = 0; base < c; base += 32) {
        const int e = base + lane;
        bool keep = false;
        int j = 0;
        if (e < c) {
            j = row[e];
            // the high parts decide unless d^2 is within `band` of rc2 (or tiny): then the hi + lo
            // difference decides, as it always did, so the decision is the same with half the loads
            const float4 hj = hi[j];
            const float xh = hj.x - hi_i.x, yh = hj.y - hi_i.y, zh = hj.z - hi_i.z;
            const float d2h = xh * xh + yh * yh + zh * zh;
            if (d2h < rc2 - band && d2h > 0.01f) {
                keep = true;
            } else if (d2h > rc2 + band) {
                keep = false;
            } else {
                const float4 lj = lo[j];
                const float x = (hj.x - hi_i.x) + (lj.x - lo_i.x);
                const float y = (hj.y - hi_i.y) + (lj.y - lo_i.y);
                const float z = (hj.z - hi_i.z) + (lj.z - lo_i.z);
                const float d2 = x * x + y * y + z * z;
                keep = d2 < rc2;
                if (!(d2 > 1e-16f)) {
                    keep = false;
                    atomicOr(&flags[FLAG_GEOM], 4);
                }
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) out[count + __popc(m & ((1u << lane) - 1u))] = j;
        count += __popc(m);
    }
    if (lane == 0) live_cnt[i] = count;
}

// largest displacement since the build: flag when any atom moved more than half the skin
__global__ void k_moved(int64_t n, const double* __restrict__ pos, const double* __restrict__ ref, double thr2,
                        int* __restrict__ moved) {
    pdl_enter();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double dx = pos[3 * i] - ref[3 * i], dy = pos[3 * i + 1] - ref[3 * i + 1], dz = pos[3 * i + 2] - ref[3 * i + 2];
    if (!(dx * dx + dy * dy + dz * dz <= thr2)) atomicOr(moved, 1);
}


inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// Counting sort of n keys in [0, nkeys) whose histogram `counts` the kernel that
// produced the keys has filled: order = indices sorted by (key, index) within the
// first `sorted_keys` buckets (later buckets hold unused capacity whose order does
// not matter); start = bucket offsets.  The scatter counts the histogram back down
// to zero for the next sort.
static cudaError_t counting_sort(cudaStream_t s, const int* gate, int64_t n, int64_t nkeys, const int32_t* key,
                                 int32_t* counts, int32_t* start, int32_t* scattered, int32_t* order,
                                 int64_t sorted_keys, int32_t* tsum, int* flags, const float4* pin = nullptr,
                                 float4* pout = nullptr) {
    scan_exclusive(s, gate, nkeys, counts, start, tsum, flags);
    if (n > 0) {
        launch_pdl(k_scatter, blocks_for(n, 256), 256, 0, s, gate, n, key, start, counts, scattered);
        launch_pdl(k_bucket_rank, blocks_for(n, 256), 256, 0, s, gate, n, key, start, scattered, sorted_keys, order,
                   pin, pout);
    }
    return cudaGetLastError();
}

void* nlist_alloc_bytes(reann_nlist* nl, size_t bytes) {
    void* p = nullptr;
    bytes = std::max<size_t>(bytes, 1);
    const cudaError_t e = nl->mem_pool ? cudaMallocFromPoolAsync(&p, bytes, nl->mem_pool, nl->alloc_stream)
                                       : cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    nl->allocs.push_back(p);
    return p;
}

template <typename T>
static T* dalloc(reann_nlist* nl, size_t count) {
    return nlist_alloc<T>(nl, count);
}

static int64_t owned_keys(const reann_nlist* nl) {
    const CellGeom& g = nl->geom;
    return (int64_t)g.nb[0] * g.nb[1] * g.nb[2] * nl->n_elem;
}
static int64_t ext_bins(const reann_nlist* nl) {
    const CellGeom& g = nl->geom;
    return (int64_t)g.nbx[0] * g.nbx[1] * g.nbx[2];
}

// steps 1-3a: wrap, sort, gather, ghost count + scan (goff[n] = ghost count on the device)
// sort_gate: the sort path (nullptr: always); keep_gate: the keep-order path (nullptr:
// never); gate: the rest of the rebuild (nullptr: always)
static cudaError_t stage_sort_and_count(cudaStream_t s, reann_nlist* nl, const double* pos, int* flags,
                                        const int* sort_gate, const int* keep_gate, const int* gate) {
    const int64_t n = nl->n;
    NlistScratch& w = nl->w;
    launch_pdl(k_wrap_key, blocks_for(n, kFp64Threads), kFp64Threads, 0, s, sort_gate, n, pos, w.species_c,
               nl->n_elem, nl->geom, w.xw_c, w.fw_c, w.mw_c, w.key, w.counts, flags, nl->pos_ref);
    counting_sort(s, sort_gate, n, owned_keys(nl), w.key, w.counts, w.start, w.scat, nl->perm, owned_keys(nl),
                  w.tsum, flags);
    launch_pdl(k_gather_internal, blocks_for(n, kFp64Threads), kFp64Threads, 0, s, sort_gate, n, nl->geom, nl->perm,
               w.xw_c, w.fw_c, w.mw_c, w.species_c, w.xw, w.fw, nl->wrapm, nl->species, w.gcnt, w.halo);
    if (keep_gate)
        launch_pdl(k_wrap_keep, blocks_for(n, kFp64Threads), kFp64Threads, 0, s, keep_gate, n, nl->geom, pos,
                   nl->perm, w.xw, w.fw, nl->wrapm, w.gcnt, w.halo, flags, nl->pos_ref);
    scan_exclusive(s, gate, n, w.gcnt, w.goff, w.tsum, flags);
    return cudaGetLastError();
}

// steps 3b-4: ghost fill and the extended bins (needs the ghost capacity)
static cudaError_t stage_ghosts_and_bins(cudaStream_t s, reann_nlist* nl, int* flags, const int* gate) {
    const int64_t n = nl->n, next = n + nl->g_cap;
    NlistScratch& w = nl->w;
    const int64_t nx = ext_bins(nl);
    launch_pdl(k_ghosts_ext, blocks_for(next, kFp64Threads), kFp64Threads, 0, s, gate, n, nl->geom, w.xw, w.fw,
               w.goff, nl->g_cap, nl->g_owner, nl->g_shift, w.ekey, w.ecounts, w.p32, (int32_t)nx, w.halo, flags);
    counting_sort(s, gate, next, nx + 1, w.ekey, w.ecounts, w.estart, w.escat, w.eorder, nx, w.etsum, flags,
                  w.p32, w.p32s);
    return cudaGetLastError();
}

static cudaError_t stage_search(cudaStream_t s, reann_nlist* nl, int* flags, const int* gate) {
    const int64_t n = nl->n;
    NlistScratch& w = nl->w;
    launch_pdl(k_nbr_search, blocks_for(n * 32, 256), 256, 0, s, gate, n, nl->geom, w.xw, nl->g_owner,
               nl->g_shift, w.p32, w.p32s, w.estart, w.ekey, nl->stride, nl->nbr, nl->nbr_cnt, flags);
    return cudaGetLastError();
}

int build_nlist_device(reann_ctx* ctx, reann_nlist* nl, const double* pos, const int32_t* species) {
    cudaStream_t s = ctx->stream;
    const int64_t n = nl->n;
    NlistScratch& w = nl->w;
    const int64_t nkeys = owned_keys(nl);
    if (n >= (int64_t(1) << 28))  // the scans' status words carry sums below 2^30 (atoms + ghost capacity)
        return set_error(ctx, REANN_E_ARG, "more than 2^28 atoms in one list");
    w.xw_c = dalloc<double>(nl, 3 * n);
    w.fw_c = dalloc<double>(nl, 3 * n);
    w.mw_c = dalloc<int32_t>(nl, 3 * n);
    w.key = dalloc<int32_t>(nl, n);
    w.counts = dalloc<int32_t>(nl, nkeys);
    w.start = dalloc<int32_t>(nl, nkeys + 1);
    w.xw = dalloc<double>(nl, 3 * n);
    w.fw = dalloc<double>(nl, 3 * n);
    w.gcnt = dalloc<int32_t>(nl, n);
    w.halo = dalloc<int32_t>(nl, 3 * n);
    w.goff = dalloc<int32_t>(nl, n + 1);
    w.species_c = dalloc<int32_t>(nl, n);
    w.scat = dalloc<int32_t>(nl, n);
    w.rb_state = dalloc<int32_t>(nl, 4);
    w.tsum = dalloc<int32_t>(nl, std::max(scan_status_words(nkeys), scan_status_words(n)));
    nl->perm = dalloc<int32_t>(nl, n);
    nl->species = dalloc<int32_t>(nl, n);
    nl->wrapm = dalloc<int32_t>(nl, 3 * n);
    nl->pos_ref = dalloc<double>(nl, 3 * n);
    if (!w.xw_c || !w.fw_c || !w.mw_c || !w.key || !w.counts || !w.start || !w.xw || !w.fw || !w.gcnt || !w.goff ||
        !w.halo ||
        !w.species_c || !w.scat || !nl->perm || !nl->species || !nl->wrapm || !nl->pos_ref || !w.rb_state ||
        !w.tsum)
        return set_error(ctx, REANN_E_NOMEM, "neighbour-list allocation failed");
    {
        const int32_t state0[4] = {1, 0, 0, 0};  // this build sorts; rebuilds count from 1
        REANN_CUDA_TRY(ctx, cudaMemcpyAsync(w.rb_state, state0, sizeof(state0), cudaMemcpyHostToDevice, s));
        REANN_CUDA_TRY(ctx, cudaStreamSynchronize(s));  // state0 lives on this stack frame
    }
    REANN_CUDA_TRY(ctx, cudaMemcpyAsync(w.species_c, species, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    REANN_CUDA_TRY(ctx, cudaMemsetAsync(w.counts, 0, sizeof(int32_t) * nkeys, s));  // kept zero between sorts
    REANN_CUDA_TRY(ctx, cudaMemsetAsync(w.tsum, 0,
                                        sizeof(int32_t) * std::max(scan_status_words(nkeys), scan_status_words(n)), s));
    REANN_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_flags, 0, sizeof(int) * NFLAGS, s));
    REANN_CUDA_TRY(ctx, stage_sort_and_count(s, nl, pos, ctx->d_flags, nullptr, nullptr, nullptr));
    // sizes: element ranges of the internal order and the ghost count
    std::vector<int32_t> es(nl->n_elem + 1);
    const int64_t nbins = nkeys / nl->n_elem;
    for (int e = 0; e <= nl->n_elem; ++e)
        REANN_CUDA_TRY(ctx, cudaMemcpyAsync(&es[e], w.start + (int64_t)e * nbins, sizeof(int32_t),
                                            cudaMemcpyDeviceToHost, s));
    int32_t G = 0;
    REANN_CUDA_TRY(ctx, cudaMemcpyAsync(&G, w.goff + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    REANN_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_flags, ctx->d_flags, sizeof(int) * NFLAGS, cudaMemcpyDeviceToHost, s));
    REANN_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (ctx->h_flags[FLAG_SPECIES]) return set_error(ctx, REANN_E_ARG, "species index out of range");
    if (ctx->h_flags[FLAG_GEOM]) return set_error(ctx, REANN_E_GEOM, "non-finite atom position");
    for (int e = 0; e <= nl->n_elem; ++e) nl->elem_start[e] = es[e];
    nl->g = G;
    nl->ghosts_by_owner = true;  // k_ghosts enumerates each atom's images contiguously at goff[i]
    // capacity with headroom so that rebuilds after atom motion fit
    nl->g_cap = G + G / 4 + 64;
    const int64_t next = n + nl->g_cap;
    const int64_t nx = ext_bins(nl);
    nl->g_owner = dalloc<int32_t>(nl, nl->g_cap);
    nl->g_shift = dalloc<int32_t>(nl, nl->g_cap);
    w.ekey = dalloc<int32_t>(nl, next);
    w.p32 = dalloc<float4>(nl, next);
    w.p32s = dalloc<float4>(nl, next);
    w.ecounts = dalloc<int32_t>(nl, nx + 1);
    w.estart = dalloc<int32_t>(nl, nx + 2);
    w.eorder = dalloc<int32_t>(nl, next);
    w.escat = dalloc<int32_t>(nl, next);
    w.etsum = dalloc<int32_t>(nl, scan_status_words(nx + 1));
    if (!nl->g_owner || !nl->g_shift || !w.ekey || !w.p32 || !w.p32s || !w.ecounts || !w.estart || !w.eorder ||
        !w.escat || !w.etsum)
        return set_error(ctx, REANN_E_NOMEM, "ghost allocation failed");
    REANN_CUDA_TRY(ctx, cudaMemsetAsync(w.ecounts, 0, sizeof(int32_t) * (nx + 1), s));  // kept zero between sorts
    REANN_CUDA_TRY(ctx, cudaMemsetAsync(w.etsum, 0, sizeof(int32_t) * scan_status_words(nx + 1), s));
    REANN_CUDA_TRY(ctx, stage_ghosts_and_bins(s, nl, ctx->d_flags, nullptr));
    // row capacity: expected neighbours from the number density, with headroom
    const CellGeom& g = nl->geom;
    const double vol = std::fabs(g.h[0] * (g.h[4] * g.h[8] - g.h[5] * g.h[7]) -
                                 g.h[1] * (g.h[3] * g.h[8] - g.h[5] * g.h[6]) +
                                 g.h[2] * (g.h[3] * g.h[7] - g.h[4] * g.h[6]));
    const double expect = (double)n / vol * 4.18879020478639 * std::pow(g.rcut2, 1.5);
    int stride = (int)std::min<double>(1 << 20, std::ceil((1.5 * expect + 32) / 8.0) * 8);
    for (int attempt = 0; attempt < 2; ++attempt) {
        nl->stride = stride;
        nl->nbr = dalloc<int32_t>(nl, (size_t)n * stride);
        nl->nbr_cnt = dalloc<int32_t>(nl, n);
        if (!nl->nbr || !nl->nbr_cnt) return set_error(ctx, REANN_E_NOMEM, "neighbour-list allocation failed");
        REANN_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_flags, 0, sizeof(int) * NFLAGS, s));
        REANN_CUDA_TRY(ctx, stage_search(s, nl, ctx->d_flags, nullptr));
        REANN_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_flags, ctx->d_flags, sizeof(int) * NFLAGS, cudaMemcpyDeviceToHost, s));
        REANN_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        if (ctx->h_flags[FLAG_GEOM]) return set_error(ctx, REANN_E_GEOM, "coincident atoms (distance < 1e-8 A)");
        if (ctx->h_flags[FLAG_GHOST_OVERFLOW]) return set_error(ctx, REANN_E_CAPACITY, "ghost capacity exceeded");
        nl->max_count = ctx->h_flags[FLAG_MAXNBR];
        if (!ctx->h_flags[FLAG_NBR_OVERFLOW]) break;
        if (attempt == 1) return set_error(ctx, REANN_E_CAPACITY, "neighbour capacity exceeded");
        // grow to the observed maximum (plus headroom for later motion) and search again
        stride = ((ctx->h_flags[FLAG_MAXNBR] + ctx->h_flags[FLAG_MAXNBR] / 8 + 16 + 7) / 8) * 8;
    }
    return REANN_OK;
}

// gate == nullptr: always rebuild; otherwise every kernel returns at once unless *gate != 0
cudaError_t launch_rebuild(cudaStream_t s, reann_nlist* nl, const double* pos, int* flags, const int* gate) {
    launch_pdl(k_rebuild_gates, 1, 1, 0, s, gate, nl->w.rb_state);
    cudaError_t e = stage_sort_and_count(s, nl, pos, flags, nl->w.rb_state + 1, nl->w.rb_state + 2, gate);
    if (e == cudaSuccess) e = stage_ghosts_and_bins(s, nl, flags, gate);
    if (e == cudaSuccess) e = stage_search(s, nl, flags, gate);
    return e;
}

cudaError_t launch_moved(cudaStream_t s, const reann_nlist* nl, const double* pos, int* moved) {
    const double half = 0.5 * nl->skin;
    launch_pdl(k_moved, blocks_for(nl->n, kFp64Threads), kFp64Threads, 0, s, nl->n, pos, nl->pos_ref, half * half,
               moved);
    return cudaGetLastError();
}

const int32_t* ghost_count_ptr(const reann_nlist* nl) { return nl->w.goff + nl->n; }

cudaError_t launch_refresh_positions(cudaStream_t s, const reann_nlist* nl, const double* pos, const float* c0) {
    const int64_t total = nl->n + nl->g_cap;
    launch_pdl(k_refresh, blocks_for(total, kFp64Threads), kFp64Threads, 0, s, nl->n, ghost_count_ptr(nl), nl->g_cap,
               nl->geom, pos, nl->perm, nl->wrapm, nl->g_owner, nl->g_shift, nl->pos_hi, nl->pos_lo, nl->species, c0,
               nl->coef);
    return cudaGetLastError();
}

cudaError_t launch_live_edges(cudaStream_t s, const reann_nlist* nl, float rc2, int* flags) {
    const int64_t nr = rows_of(nl);
    if (nr == 0) return cudaSuccess;
    // the band bounds the low parts' share of d^2 with room to spare: the search's FP32 margin
    // (16 r_cut ulp(largest coordinate) + 1e-4 A^2) plus 0.05 A^2
    const float band = nl->geom.margin + 0.05f;
    launch_pdl(k_live, blocks_for(nr * 32, 256), 256, 0, s, nr, nl->stride, rc2, band, nl->nbr, nl->nbr_cnt,
               nl->pos_hi, nl->pos_lo, nl->live, nl->live_cnt, flags);
    return cudaGetLastError();
}

int export_nlist(reann_ctx* ctx, const reann_nlist* nl, int64_t cap, int32_t* oi, int32_t* oj, int32_t* on,
                 int64_t* count) {
    cudaStream_t s = ctx->stream;
    const int64_t n = nl->n;
    int32_t G = 0;
    REANN_CUDA_TRY(ctx, cudaMemcpyAsync(&G, ghost_count_ptr(nl), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    REANN_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    const int64_t g = std::min<int64_t>(G, nl->g_cap);
    std::vector<int32_t> nbr((size_t)n * nl->stride), cnt(n), perm(n), wm(3 * n), own(g), sh(g);
    REANN_CUDA_TRY(ctx, cudaMemcpyAsync(nbr.data(), nl->nbr, sizeof(int32_t) * nbr.size(), cudaMemcpyDeviceToHost, s));
    REANN_CUDA_TRY(ctx, cudaMemcpyAsync(cnt.data(), nl->nbr_cnt, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    REANN_CUDA_TRY(ctx, cudaMemcpyAsync(perm.data(), nl->perm, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    REANN_CUDA_TRY(ctx, cudaMemcpyAsync(wm.data(), nl->wrapm, sizeof(int32_t) * 3 * n, cudaMemcpyDeviceToHost, s));
    if (g > 0) {
        REANN_CUDA_TRY(ctx, cudaMemcpyAsync(own.data(), nl->g_owner, sizeof(int32_t) * g, cudaMemcpyDeviceToHost, s));
        REANN_CUDA_TRY(ctx, cudaMemcpyAsync(sh.data(), nl->g_shift, sizeof(int32_t) * g, cudaMemcpyDeviceToHost, s));
    }
    REANN_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    int64_t q = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int e = 0; e < cnt[i]; ++e) {
            int64_t slot = nbr[(size_t)i * nl->stride + e];
            int64_t o = slot;
            int a[3] = {0, 0, 0};
            if (slot >= n) {
                o = own[slot - n];
                int p = sh[slot - n];
                a[0] = (p & 255) - 128;
                a[1] = ((p >> 8) & 255) - 128;
                a[2] = ((p >> 16) & 255) - 128;
            }
            if (q < cap) {
                oi[q] = perm[i];
                oj[q] = perm[o];
                for (int k = 0; k < 3; ++k) on[3 * q + k] = a[k] - wm[3 * o + k] + wm[3 * i + k];
            }
            ++q;
        }
    }
    *count = q;
    return REANN_OK;
}

}  // namespace reann
