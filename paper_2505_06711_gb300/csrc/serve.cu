// Kernels of the serving pool: many independent structures packed into one
// resident reann_nlist-shaped pool so that one evaluation covers all of them.
//
// Pool index space: owned slots [0, NO) followed by ghost slots [NO, NO + NG).
// A structure admitted into owned range [ob, ob + n) and ghost range
// [gb, gb + g) has its neighbour rows copied with every entry remapped
// (local owned j -> ob + j, local ghost N + q -> NO + gb + q), its positions
// written once as hi/lo FP32 pairs, its ghosts pointed at ob + owner, and its
// output destination (the pool's perm) set to ob + caller index.  Slots that
// hold no structure have no neighbours and write their outputs to a sink row.
#include <cuda_runtime.h>

#include "common.cuh"

namespace reann {
namespace {

__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }

__device__ __forceinline__ void shift_vec(const CellGeom& g, int n0, int n1, int n2, double s[3]) {
#pragma unroll
    for (int d = 0; d < 3; ++d)
        s[d] = dadd(dadd(dmul((double)n0, g.h[d]), dmul((double)n1, g.h[3 + d])), dmul((double)n2, g.h[6 + d]));
}

__device__ __forceinline__ void hilo(const double x[3], float4& hi, float4& lo) {
    float h[3], l[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        h[k] = (float)x[k];
        l[k] = (float)(x[k] - (double)h[k]);
    }
    hi = make_float4(h[0], h[1], h[2], 0.f);
    lo = make_float4(l[0], l[1], l[2], 0.f);
}

struct PackSrc {
    int64_t n, g;                // atoms, ghosts of the structure
    int stride;                  // its row capacity
    const int32_t* nbr;          // n x stride local slots
    const int32_t* cnt;          // n
    const int32_t* species;      // n (internal order)
    const int32_t* perm;         // n internal -> caller
    const int32_t* wrapm;        // n x 3
    const int32_t* owner;        // g
    const int32_t* shift;        // g packed
    const double* pos;           // caller order FP64
    CellGeom geom;
};

struct PackDst {
    int64_t no, ob, gb;  // pool owned size, owned base, ghost base
    int stride;
    int32_t *nbr, *cnt, *species, *perm, *owner;
    float4 *hi, *lo;
};

// owned atoms: rows (remapped), species, destination, positions
__global__ void k_pack_owned(PackSrc s, PackDst d) {
    pdl_enter();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    const int c = s.cnt[i];
    const int32_t* src = s.nbr + (size_t)i * s.stride;
    int32_t* dst = d.nbr + (size_t)(d.ob + i) * d.stride;
    for (int e = 0; e < c; ++e) {
        const int64_t j = src[e];
        dst[e] = (int32_t)(j < s.n ? d.ob + j : d.no + d.gb + (j - s.n));
    }
    d.cnt[d.ob + i] = c;
    d.species[d.ob + i] = s.species[i];
    d.perm[d.ob + i] = (int32_t)(d.ob + s.perm[i]);
    const int64_t ci = s.perm[i];
    double sm[3], x[3];
    shift_vec(s.geom, s.wrapm[3 * i], s.wrapm[3 * i + 1], s.wrapm[3 * i + 2], sm);
#pragma unroll
    for (int k = 0; k < 3; ++k) x[k] = s.pos[3 * ci + k] - sm[k];
    hilo(x, d.hi[d.ob + i], d.lo[d.ob + i]);
}

// ghost slots: owner (pool index) and image position
__global__ void k_pack_ghosts(PackSrc s, PackDst d) {
    pdl_enter();
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= s.g) return;
    const int64_t o = s.owner[q];
    const int p = s.shift[q];
    const int a = (p & 255) - 128, b = ((p >> 8) & 255) - 128, c = ((p >> 16) & 255) - 128;
    d.owner[d.gb + q] = (int32_t)(d.ob + o);
    const int64_t co = s.perm[o];
    double sm[3], sv[3], x[3];
    shift_vec(s.geom, s.wrapm[3 * o], s.wrapm[3 * o + 1], s.wrapm[3 * o + 2], sm);
    shift_vec(s.geom, a, b, c, sv);
#pragma unroll
    for (int k = 0; k < 3; ++k) x[k] = (s.pos[3 * co + k] - sm[k]) + sv[k];
    hilo(x, d.hi[d.no + d.gb + q], d.lo[d.no + d.gb + q]);
}

// a released owned range: no neighbours, outputs to the sink row
__global__ void k_release(int64_t ob, int64_t n, int32_t sink, int32_t* __restrict__ cnt, int32_t* __restrict__ perm) {
    pdl_enter();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    cnt[ob + i] = 0;
    perm[ob + i] = sink;
}

// structures just evaluated: drop their neighbours and send their outputs to the
// sink so that later pool launches leave their result rows untouched
__global__ void k_retire(const int4* __restrict__ seg, int32_t sink, int32_t* __restrict__ cnt,
                         int32_t* __restrict__ perm) {
    pdl_enter();
    const int4 sg = seg[blockIdx.x];
    for (int i = threadIdx.x; i < sg.y; i += blockDim.x) {
        cnt[sg.x + i] = 0;
        perm[sg.x + i] = sink;
    }
}

// per-structure FP64 energy: one block per segment, fixed summation order
__global__ void __launch_bounds__(256) k_segment_energy(const int4* __restrict__ seg, const float* __restrict__ eps,
                                                        double* __restrict__ energies) {
    pdl_enter();
    __shared__ double sm[256];
    const int4 sg = seg[blockIdx.x];  // x = owned base, y = atoms, z = output index
    double s = 0.0;
    for (int i = threadIdx.x; i < sg.y; i += 256) s += (double)eps[sg.x + i];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && sg.y >= 0) energies[sg.z] = sm[0];
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_pack(cudaStream_t s, const reann_nlist* src, const double* caller_pos, reann_nlist* pool,
                        int64_t ob, int64_t gb) {
    PackSrc a{src->n,       src->g,     src->stride, src->nbr,      src->nbr_cnt, src->species,
              src->perm,    src->wrapm, src->g_owner, src->g_shift, caller_pos,   src->geom};
    PackDst b{pool->n, ob, gb, pool->stride, pool->nbr, pool->nbr_cnt, pool->species, pool->perm, pool->g_owner,
              pool->pos_hi, pool->pos_lo};
    launch_pdl(k_pack_owned, blocks_for(src->n, 128), 128, 0, s, a, b);
    if (src->g > 0) launch_pdl(k_pack_ghosts, blocks_for(src->g, 256), 256, 0, s, a, b);
    return cudaGetLastError();
}

cudaError_t launch_release(cudaStream_t s, reann_nlist* pool, int64_t ob, int64_t n) {
    if (n > 0) launch_pdl(k_release, blocks_for(n, 256), 256, 0, s, ob, n, (int32_t)pool->n, pool->nbr_cnt, pool->perm);
    return cudaGetLastError();
}

cudaError_t launch_retire(cudaStream_t s, const int4* seg, int nseg, reann_nlist* pool) {
    if (nseg > 0) launch_pdl(k_retire, nseg, 256, 0, s, seg, (int32_t)pool->n, pool->nbr_cnt, pool->perm);
    return cudaGetLastError();
}

cudaError_t launch_segment_energy(cudaStream_t s, const int4* seg, int nseg, const float* eps, double* energies) {
    if (nseg > 0) launch_pdl(k_segment_energy, nseg, 256, 0, s, seg, eps, energies);
    return cudaGetLastError();
}

}  // namespace reann
