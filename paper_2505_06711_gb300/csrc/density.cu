// Edge kernels of the REANN message-passing layer and its adjoint.
//
// Forward (Sec. 2.1, Eq. 1), per owned atom i and layer t:
//   b_{i,a,m} = sum_{j live} c^t_{j,m} phi_m(d_ij) A_a(r_ij)
//   g_{i,a,k} = sum_m b_{i,a,m} W^t_{l(a),m,k}
//   rho_{i,l,k} = sum_{a in l} w_a g_{i,a,k}^2
// Reverse (Sec. 2.2, Eqs. 3-5), per layer, given rhobar:
//   gbar = 2 w_a g rhobar,  bbar_{a,m} = sum_k gbar_{a,k} W_{l(a),m,k}
//   and, gathering over atom k's own (symmetric, full) list with r = r_j - r_k:
//     dE/dr_k = -sum_j sum_{a,m} [bbar_{k,a,m} c_{j,m} + (-1)^l bbar_{j,a,m} c_{k,m}] grad_r(phi_m A_a)(r)
//     cbar_{k,m} = sum_j phi_m(d) sum_a (-1)^l bbar_{j,a,m} A_a(r)
//   (the second term of each line is the reverse edge j -> k, written with
//   A_a(-r) = (-1)^l A_a(r); ghost slots j carry their owner's bbar, which is
//   the paper's ghost-gradient exchange as a vector-Jacobian product, Sec. 2.2).
// No atomics: every output row is written by the lanes of its own centre atom.
//
// Forward layout: a quad of 4 lanes per centre atom (8 atoms per warp).  Each
// lane walks every 4th live neighbour, whose hi/lo FP32 position (32 B) and
// coefficients (32 B) are copied into shared memory with cp.async one edge
// ahead, and accumulates the 80 products in registers; a butterfly
// reduce-scatter leaves 20 of the 80 b values in each lane, which then
// contracts its 4 orbitals from shared memory.  The adjoint gathers each
// neighbour's 384 B adjoint record (bbar and c) and uses 8 lanes per atom
// instead (below).
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"

namespace reann {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kWarps = 4;          // warps per block
constexpr int kFwdStages = 2;      // forward: a lane's next kFwdStages - 1 edges are in flight (3, 4 measured slower)
constexpr int kAtomsPerWarp = 8;   // quads per warp
constexpr int kBStride = 84;       // padded per-atom row in shared memory (16 B aligned)


struct Edge {
    float x, y, z, d;
    float phi[NPHI];
};

// exp(a) for |a| < 80 by Cody-Waite range reduction (W. J. Cody and W. Waite,
// Software Manual for the Elementary Functions, 1980): a = k ln2 + r with ln2
// split into a short high part (k ln2_hi exact) and a correction, |r| <= ln2/2,
// then the degree-7 Taylor polynomial of exp(r) (truncation < 6e-9 relative) in
// Horner form and an exact scaling by 2^k.  Measured on the GPU against FP64 its
// mean relative error is ~1e-9 (unbiased), so the m-fold Gaussian recurrence
// below does not turn a one-sided rounding habit into a shift of every phi_m.
__device__ __forceinline__ float exp_cw(float a) {
    a = fminf(fmaxf(a, -87.f), 88.f);  // keeps 2^k a normal float
    const float k = rintf(a * 1.44269504f);
    float r = fmaf(-k, 0.693145751953125f, a);
    r = fmaf(-k, 1.428606820309417e-06f, r);
    float p = 1.f / 5040.f;
    p = fmaf(p, r, 1.f / 720.f);
    p = fmaf(p, r, 1.f / 120.f);
    p = fmaf(p, r, 1.f / 24.f);
    p = fmaf(p, r, 1.f / 6.f);
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.f);
    p = fmaf(p, r, 1.f);
    return p * __int_as_float(((int)k + 127) << 23);
}

// Gaussians by the equal-spacing recurrence exp(-a(d-mu_{m+1})^2) = exp(-a(d-mu_m)^2) q kappa_m,
// q = exp(2 a Delta d): two exponentials per edge instead of eight.  The constants
// a, 2 a Delta and kappa_m enter as float pairs (see Radial).
__device__ __forceinline__ void gaussians(const Radial& R, float d, float gs[NPHI]) {
    const float dd = d * d;
    gs[0] = exp_cw(-fmaf(R.alpha_hi, dd, R.alpha_lo * dd));
    const float q = exp_cw(fmaf(R.tad_hi, d, R.tad_lo * d));
#pragma unroll
    for (int m = 0; m + 1 < NPHI; ++m) {
        const float p = gs[m] * q;
        gs[m + 1] = fmaf(p, R.kap_hi[m], p * R.kap_lo[m]);
    }
}

// f_c(d) = (cos(pi d/r_c)/2 + 1/2)^2 evaluated as cos^4(pi x / 2), x = d / r_c
// taken with 1/r_c as a float pair (d inv_hi + d inv_lo: within an ulp of the
// correctly rounded quotient and without the one-sided error of a rounded 1/r_c,
// which near r_c, where the cutoff's logarithmic derivative is large, would
// bias every atom), no rounded pi constant, and no cancellation of 1/2 + cos/2
// near d = r_c.  dfc = -(2 pi / r_c) cos^3 sin (half angle).
__device__ __forceinline__ void cutoff(const Radial& R, float d, float& fc, float& dfc) {
    float s, c;
    const float x = fmaf(d, R.inv_rc_hi, d * R.inv_rc_lo);
    sincospif(0.5f * x, &s, &c);
    const float c2 = c * c;
    fc = c2 * c2;
    const float u = -6.28318530717959f * c2 * c * s;
    dfc = fmaf(u, R.inv_rc_hi, u * R.inv_rc_lo);
}

__device__ __forceinline__ void monomials(float x, float y, float z, float A[NANG]) {
    A[0] = 1.f;
    A[1] = x;
    A[2] = y;
    A[3] = z;
    A[4] = x * x;
    A[5] = y * y;
    A[6] = z * z;
    A[7] = x * y;
    A[8] = x * z;
    A[9] = y * z;
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }

// Orbital pair (k, k'), k <= k', of pair feature p = 0..35 (row-major over k)
__constant__ unsigned char c_pair_k[NORB_P * (NORB_P + 1) / 2];
__constant__ unsigned char c_pair_k2[NORB_P * (NORB_P + 1) / 2];

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// ------------------------------------------------------------- forward ---
// PAIRS = false: Eq. 1, rho_{l,k} = sum_{a in l} w_a g_{a,k}^2 over 16 orbitals.
// PAIRS = true: the orbital-pair products rho_{l,(k,k')} = sum_{a in l} w_a g_{a,k} g_{a,k'},
// k <= k' over 8 orbitals (108 features).
template <bool PAIRS>
__global__ void __launch_bounds__(kWarps * 32, 16 / kWarps) k_density_fwd(int64_t n, int stride, Radial R,
                                                            const int32_t* __restrict__ live,
                                                            const int32_t* __restrict__ live_cnt,
                                                            const float4* __restrict__ phi_hi,
                                                            const float4* __restrict__ plo,
                                                            const float* __restrict__ coef,
                                                            const float* __restrict__ Wt, float* __restrict__ rho,
                                                            float* __restrict__ bck) {
    pdl_enter();
    constexpr int KO = PAIRS ? NORB_P : NORB;
    __shared__ __align__(16) float sW[(LMAX + 1) * NPHI * KO];
    // During the edge loop: kFwdStages stages of a lane's next neighbours (hi, lo
    // position and c of j), [stage][part][thread] float4; afterwards the b rows.
    constexpr int kStage = kFwdStages * 4 * kWarps * 32 * 4;
    static_assert(kStage >= kWarps * kAtomsPerWarp * kBStride, "b rows must fit in the staging area");
    __shared__ __align__(16) float sU[kStage];
    float4* stg = reinterpret_cast<float4*>(sU);
    for (int i = threadIdx.x; i < (LMAX + 1) * NPHI * KO; i += blockDim.x) sW[i] = Wt[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, q = lane & 3, slot = lane >> 2;
    const int64_t atom = ((int64_t)blockIdx.x * kWarps + warp) * kAtomsPerWarp + slot;
    const bool valid = atom < n;

    float acc[NB];
#pragma unroll
    for (int v = 0; v < NB; ++v) acc[v] = 0.f;
    if (valid) {
        const float4 hi_i = phi_hi[atom], lo_i = plo[atom];
        const int cnt = live_cnt[atom];
        const int32_t* row = live + (size_t)atom * stride;
        constexpr int kT = kWarps * 32;
        auto stage = [&](int st, int j) {
            float4* d = stg + st * 4 * kT + threadIdx.x;
            cp_async16(d, phi_hi + j);
            cp_async16(d + kT, plo + j);
            cp_async16(d + 2 * kT, coef + (size_t)j * NPHI);
            cp_async16(d + 3 * kT, coef + (size_t)j * NPHI + 4);
        };
        // the lane's edges e = q, q + 4, ...: the copies of the next kFwdStages - 1 edges
        // are in flight while edge e is computed, and the index after them is loaded
        constexpr int NST = kFwdStages;
#pragma unroll
        for (int p = 0; p < NST - 1; ++p) {
            if (q + 4 * p < cnt) stage(p, row[q + 4 * p]);
            cp_async_commit();
        }
        int j_nx = q + 4 * (NST - 1) < cnt ? row[q + 4 * (NST - 1)] : 0;
        int st = 0;  // stage of edge e
        for (int e = q; e < cnt; e += 4) {
            const int e_st = e + 4 * (NST - 1);  // the edge copied now, into the stage edge e - 4 used
            if (e_st < cnt) stage(st == 0 ? NST - 1 : st - 1, j_nx);
            cp_async_commit();
            j_nx = e_st + 4 < cnt ? row[e_st + 4] : 0;
            cp_async_wait<NST - 1>();  // edge e's stage has landed
            const float4* src = stg + st * 4 * kT + threadIdx.x;
            const float4 hj = src[0], lj = src[kT], c0 = src[2 * kT], c1 = src[3 * kT];
            st = st == NST - 1 ? 0 : st + 1;
            const float x = (hj.x - hi_i.x) + (lj.x - lo_i.x);
            const float y = (hj.y - hi_i.y) + (lj.y - lo_i.y);
            const float z = (hj.z - hi_i.z) + (lj.z - lo_i.z);
            const float d = sqrtf(x * x + y * y + z * z);
            float gs[NPHI], fc, dfc;
            gaussians(R, d, gs);
            cutoff(R, d, fc, dfc);
            const float cj[NPHI] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
            float tm[NPHI];
#pragma unroll
            for (int m = 0; m < NPHI; ++m) tm[m] = cj[m] * gs[m] * fc;
            float A[NANG];
            monomials(x, y, z, A);
#pragma unroll
            for (int a = 0; a < NANG; ++a)
#pragma unroll
                for (int m = 0; m < NPHI; ++m) acc[a * NPHI + m] = fmaf(tm[m], A[a], acc[a * NPHI + m]);
        }
    }
    cp_async_wait_all();
    __syncthreads();  // the staging area becomes the b rows
    // butterfly reduce-scatter over the quad: lane q keeps b[20q, 20q+20)
    float r1[NB / 2];
    const bool hi_half = (q >> 1) & 1;
#pragma unroll
    for (int v = 0; v < NB / 2; ++v) {
        const float send = hi_half ? acc[v] : acc[NB / 2 + v];
        const float keep = hi_half ? acc[NB / 2 + v] : acc[v];
        r1[v] = keep + __shfl_xor_sync(FULL, send, 2);
    }
    float r2[NB / 4];
    const bool odd = q & 1;
#pragma unroll
    for (int v = 0; v < NB / 4; ++v) {
        const float send = odd ? r1[v] : r1[NB / 4 + v];
        const float keep = odd ? r1[NB / 4 + v] : r1[v];
        r2[v] = keep + __shfl_xor_sync(FULL, send, 1);
    }
    float* sb = sU + (warp * kAtomsPerWarp + slot) * kBStride;
#pragma unroll
    for (int v = 0; v < NB / 4; v += 4) {
        const float4 w4 = make_float4(r2[v], r2[v + 1], r2[v + 2], r2[v + 3]);
        *reinterpret_cast<float4*>(sb + 20 * q + v) = w4;
        if (valid) *reinterpret_cast<float4*>(bck + (size_t)atom * NB + 20 * q + v) = w4;
    }
    __syncwarp();
    if constexpr (PAIRS) {
        // g_{a,k} = sum_m b_{a,m} W_{l,m,k}: lane q the orbitals 2q, 2q+1 of every a,
        // into the b row's place (after all four lanes have read it); then lane q
        // the 27 features 27q .. 27q+26
        float g[NANG][2];
#pragma unroll
        for (int a = 0; a < NANG; ++a) {
            const int l = ang_l(a);
            const float4 b0 = ld4(sb + a * NPHI), b1 = ld4(sb + a * NPHI + 4);
            const float bm[NPHI] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
            g[a][0] = g[a][1] = 0.f;
#pragma unroll
            for (int m = 0; m < NPHI; ++m) {
                const float2 w = *reinterpret_cast<const float2*>(sW + (l * NPHI + m) * KO + 2 * q);
                g[a][0] = fmaf(bm[m], w.x, g[a][0]);
                g[a][1] = fmaf(bm[m], w.y, g[a][1]);
            }
        }
        __syncwarp();
#pragma unroll
        for (int a = 0; a < NANG; ++a)
            *reinterpret_cast<float2*>(sb + a * NORB_P + 2 * q) = make_float2(g[a][0], g[a][1]);
        __syncwarp();
        if (!valid) return;
        constexpr int KP = NORB_P * (NORB_P + 1) / 2;
        for (int f = 27 * q; f < 27 * q + 27; ++f) {
            const int l = f / KP, p = f - l * KP;
            const int k = c_pair_k[p], k2 = c_pair_k2[p];
            const int a0 = l == 0 ? 0 : (l == 1 ? 1 : 4), a1 = l == 0 ? 1 : (l == 1 ? 4 : NANG);
            float acc_f = 0.f;
            for (int a = a0; a < a1; ++a) acc_f = fmaf(ang_w(a) * sb[a * NORB_P + k], sb[a * NORB_P + k2], acc_f);
            rho[(size_t)atom * NFEAT_P + f] = acc_f;
        }
        return;
    }
    if (!valid) return;
    // contraction over m and the squared multinomial sum; lane q owns orbitals 4q..4q+3
    float racc[LMAX + 1][4];
#pragma unroll
    for (int l = 0; l <= LMAX; ++l)
#pragma unroll
        for (int k = 0; k < 4; ++k) racc[l][k] = 0.f;
#pragma unroll
    for (int a = 0; a < NANG; ++a) {
        const int l = ang_l(a);
        const float4 b0 = ld4(sb + a * NPHI), b1 = ld4(sb + a * NPHI + 4);
        const float bm[NPHI] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
        float g[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int m = 0; m < NPHI; ++m) {
            const float4 w = ld4(sW + (l * NPHI + m) * NORB + 4 * q);
            g[0] = fmaf(bm[m], w.x, g[0]);
            g[1] = fmaf(bm[m], w.y, g[1]);
            g[2] = fmaf(bm[m], w.z, g[2]);
            g[3] = fmaf(bm[m], w.w, g[3]);
        }
        const float wa = ang_w(a);
#pragma unroll
        for (int k = 0; k < 4; ++k) racc[l][k] = fmaf(wa * g[k], g[k], racc[l][k]);
    }
#pragma unroll
    for (int l = 0; l <= LMAX; ++l)
        *reinterpret_cast<float4*>(rho + (size_t)atom * NFEAT + l * NORB + 4 * q) =
            make_float4(racc[l][0], racc[l][1], racc[l][2], racc[l][3]);
}

// -------------------------------------------------------------- bbar -----
// bbar_{a,m} = sum_k gbar_{a,k} W_{l(a),m,k}, g recomputed from the b checkpoint, with
//   squares:  gbar_{a,k} = 2 w_a g_{a,k} rhobar_{l,k}
//   pairs:    gbar_{a,k} = w_a sum_k' R_{kk'} g_{a,k'},  R_{kk'} = rhobar_{l,(min,max)} (x 2 on the diagonal)
// written into the atom's adjoint record with the layer's c (values 10, 11 of
// the record); 4 threads per atom take values q, q + 4, q + 8.  The block's
// kBbarAtoms records are staged in shared memory and stored as whole lines.
constexpr int kBbarAtoms = 16;  // small blocks (64 threads): 4x finer balancing than 64 atoms, ~1.5 % per BF16 step
template <bool PAIRS>
__global__ void __launch_bounds__(4 * kBbarAtoms) k_bbar(int64_t n, const float* __restrict__ Wt, const float* __restrict__ bck,
                                              const float* __restrict__ rhobar, const float* __restrict__ coef,
                                              float* __restrict__ rec, GhostOut gh) {
    pdl_enter();
    constexpr int KO = PAIRS ? NORB_P : NORB;
    __shared__ __align__(16) float sW[(LMAX + 1) * NPHI * KO];
    __shared__ __align__(16) float sRec[kBbarAtoms * kRecLd];
    for (int i = threadIdx.x; i < (LMAX + 1) * NPHI * KO; i += blockDim.x) sW[i] = Wt[i];
    __syncthreads();
    const int64_t atom0 = (int64_t)blockIdx.x * kBbarAtoms;
    const int r = threadIdx.x >> 2, q = threadIdx.x & 3;
    const int64_t atom = atom0 + r;
    const int nrows = n - atom0 < kBbarAtoms ? (int)(n - atom0) : kBbarAtoms;
#pragma unroll 1
    for (int v = q; v < NREC / NPHI && r < nrows; v += 4) {
        float out[NPHI];
        if (v >= NANG) {
            rec_tail(coef, atom, v, out);
            stage_rec(sRec, r, v, out);
            continue;
        }
        const int a = v, l = ang_l(a);
        const float4 b0 = ldg4(bck + (size_t)atom * NB + a * NPHI), b1 = ldg4(bck + (size_t)atom * NB + a * NPHI + 4);
        const float bm[NPHI] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int m = 0; m < NPHI; ++m) out[m] = 0.f;
        if constexpr (PAIRS) {
            constexpr int KP = NORB_P * (NORB_P + 1) / 2;
            float g[NORB_P], gb[NORB_P];
#pragma unroll
            for (int k = 0; k < NORB_P; ++k) {
                g[k] = 0.f;
                gb[k] = 0.f;
#pragma unroll
                for (int m = 0; m < NPHI; ++m) g[k] = fmaf(bm[m], sW[(l * NPHI + m) * KO + k], g[k]);
            }
            const float* rb = rhobar + (size_t)atom * NFEAT_P + l * KP;
            int p = 0;
#pragma unroll
            for (int k = 0; k < NORB_P; ++k)
#pragma unroll
                for (int k2 = k; k2 < NORB_P; ++k2, ++p) {
                    const float rv = __ldg(rb + p);
                    gb[k] = fmaf(rv, g[k2], gb[k]);
                    gb[k2] = fmaf(rv, g[k], gb[k2]);
                }
            const float wa = ang_w(a);
#pragma unroll
            for (int m = 0; m < NPHI; ++m)
#pragma unroll
                for (int k = 0; k < NORB_P; ++k) out[m] = fmaf(wa * gb[k], sW[(l * NPHI + m) * KO + k], out[m]);
        } else {
            bbar_term(bm, 2.f * ang_w(a), sW + l * NPHI * NORB, rhobar + (size_t)atom * NFEAT + l * NORB, out);
        }
        stage_rec(sRec, r, v, out);
    }
    __syncthreads();
    flush_rec(sRec, nrows, atom0, rec, gh, threadIdx.x, blockDim.x);
}

// ---------------------------------------------------------- adjoint ------

// Reverse pass (header formulas), laid out for coalesced gathers: 8
// lanes per centre atom k (4 atoms per warp), lane m owning radial channel m.
// Per batch of 8 live edges each lane first computes the geometry of one edge
// (d, f_c, f_c', the 8 Gaussians) into shared memory; then every lane walks the
// 8 edges and, for its channel m, gathers bbar_{j,a,m} (a = 0..9) and c_{j,m}
// from j's adjoint record (3 float4 loads per lane; per load the 8 lanes read
// one full 128 B line of the record), and accumulates its share of dE/dr_k;
// cbar_{k,m} is lane m's own sum.  The force is reduced over the 8 lanes once
// per atom.  Each record is gathered just before its edge is computed: without
// records held in registers ahead of use the kernel fits 64 registers and 32
// warps per SM (prefetching one edge ahead took 80 registers and 24 warps, and
// was 3 % slower).
constexpr int kAdjWarps = 2;  // small blocks: the block scheduler balances the SMs at fine grain
constexpr int kAdjGroups = 4;  // centre atoms per warp
// Edge record in shared memory: x y z 1/d | d fc fc' - | g_0..g_7 (16 floats).
// Strides chosen bank-conflict free: a record every 20 floats (8 lanes' float4
// stores hit 32 distinct banks), a group every 168 floats (the 4 groups'
// reads of g_m land on disjoint banks).
constexpr int kGeoStride = 20;
constexpr int kGroupStride = 8 * kGeoStride + 8;

// With forces set (the last reverse layer), the kernel also writes F = -dE/dr
// and the atomic energies in caller order (perm: internal -> caller index);
// with first set (the first reverse layer), grad and vir are written, not
// accumulated.
struct Outputs {
    const int32_t* perm;
    const float* eps;
    float* forces;
    float* atom_energy;
    bool first;
};

// WANT_VIR: also W -= (dE/dr_e) r_e^T over the atom's own edges (their
// bbar_k c_j terms: every directed edge once) into vir (N x 9, accumulated
// over the layers like grad).
template <bool WANT_CBAR, bool WANT_VIR>
__global__ void __launch_bounds__(kAdjWarps * 32) k_density_adj8(int64_t n, int stride, Radial R,
                                                                const int32_t* __restrict__ live,
                                                                const int32_t* __restrict__ live_cnt,
                                                                const float4* __restrict__ phi_hi,
                                                                const float4* __restrict__ plo,
                                                                const float* __restrict__ rec,
                                                                float* __restrict__ cbar, float* __restrict__ grad,
                                                                float* __restrict__ vir, Outputs out) {
    pdl_enter();
    __shared__ __align__(16) float sGeo[kAdjWarps][kAdjGroups * kGroupStride];
    __shared__ __align__(16) float4 sPos[2][kAdjWarps * 32];  // a lane's next edge: hi, lo position of j
    __shared__ __align__(16) float4 sCen[kAdjWarps * kAdjGroups][2];  // hi, lo position of the centre atom
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, m = lane & 7, grp = lane >> 3;
    const int64_t atom = ((int64_t)blockIdx.x * kAdjWarps + warp) * kAdjGroups + grp;
    const bool valid = atom < n;
    // the 12 values of channel m in an atom's record: bbar_{0..9,m}, c_m, 0
    auto load_rec = [&](int64_t r, float* v) {
        const float* p = rec + (size_t)r * NREC + 4 * m;
#pragma unroll
        for (int line = 0; line < 3; ++line) {
            const float4 x = ldg4(p + line * 4 * NPHI);
            v[4 * line] = x.x, v[4 * line + 1] = x.y, v[4 * line + 2] = x.z, v[4 * line + 3] = x.w;
        }
    };
    float bk[12];
    int cnt = 0;
    const int32_t* row = live;
    float4* cen = sCen[warp * kAdjGroups + grp];
    if (valid) {
        load_rec(atom, bk);
        cnt = live_cnt[atom];
        if (m < 2) cen[m] = (m == 0 ? phi_hi : plo)[atom];
        row = live + (size_t)atom * stride;
    } else {
#pragma unroll
        for (int a = 0; a < 12; ++a) bk[a] = 0.f;
    }
    const float ck = bk[NANG];
    int cmax = cnt;
    cmax = max(cmax, __shfl_xor_sync(FULL, cmax, 8));
    cmax = max(cmax, __shfl_xor_sync(FULL, cmax, 16));
    __syncwarp();  // the centre positions are visible to the group
    const float mu_hi = R.mu_hi[m], mu_lo = R.mu_lo[m], two_alpha = 2.f * R.alpha_hi;
    float* geo = sGeo[warp] + grp * kGroupStride;
    float4* my_hi = &sPos[0][threadIdx.x];
    float4* my_lo = &sPos[1][threadIdx.x];
    float gx = 0.f, gy = 0.f, gz = 0.f, cb = 0.f;
    float w[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) w[q] = 0.f;
    // Pipeline across batches of 8 edges: while batch b is computed, the
    // positions of batch b + 1 are copied into shared memory (cp.async) and the
    // indices of batch b + 2 are loaded.
    int j_cur = 0;
    if (m < cnt) {
        j_cur = row[m];
        cp_async16(my_hi, phi_hi + j_cur);
        cp_async16(my_lo, plo + j_cur);
    }
    cp_async_commit();
    int j_nx = 8 + m < cnt ? row[8 + m] : 0;
    for (int e0 = 0; e0 < cmax; e0 += 8) {
        const int ns = cnt - e0;
        // geometry of edge e0 + m, one edge per lane, from the staged positions
        cp_async_wait_all();
        if (m < ns) {
            const float4 hj = *my_hi, lj = *my_lo, hi_i = cen[0], lo_i = cen[1];
            const float x = (hj.x - hi_i.x) + (lj.x - lo_i.x);
            const float y = (hj.y - hi_i.y) + (lj.y - lo_i.y);
            const float z = (hj.z - hi_i.z) + (lj.z - lo_i.z);
            const float d = sqrtf(x * x + y * y + z * z);
            float gs[NPHI], fc, dfc;
            gaussians(R, d, gs);
            cutoff(R, d, fc, dfc);
            float* g = geo + m * kGeoStride;
            *reinterpret_cast<float4*>(g) = make_float4(x, y, z, 1.f / d);
            *reinterpret_cast<float4*>(g + 4) = make_float4(d, fc, dfc, __int_as_float(j_cur));
            *reinterpret_cast<float4*>(g + 8) = make_float4(gs[0], gs[1], gs[2], gs[3]);
            *reinterpret_cast<float4*>(g + 12) = make_float4(gs[4], gs[5], gs[6], gs[7]);
        }
        __syncwarp();
        // this lane's slot has been read (its values are used above): stage the next batch
        if (8 + m < ns) {
            cp_async16(my_hi, phi_hi + j_nx);
            cp_async16(my_lo, plo + j_nx);
        }
        cp_async_commit();
        const int j_nx2 = 16 + m < ns ? row[e0 + 16 + m] : 0;
        auto gather = [&](int s, float* bj) {
            if (s < ns) load_rec(__float_as_int(geo[s * kGeoStride + 7]), bj);
        };
        auto edge = [&](int s, const float* bj) {
            if (s >= ns) return;
            const float cj = bj[NANG];
            const float* g = geo + s * kGeoStride;
            const float4 g0 = *reinterpret_cast<const float4*>(g);
            const float4 g1 = *reinterpret_cast<const float4*>(g + 4);
            const float gsm = g[8 + m];
            const float x = g0.x, y = g0.y, z = g0.z, inv_d = g0.w;
            const float d = g1.x, fc = g1.y, dfc = g1.z;
            const float phi = gsm * fc;
            const float dphi = gsm * (dfc - two_alpha * ((d - mu_hi) - mu_lo) * fc);  // d - mu_m as a float pair
            // Gk = sum_a bbar_k grad A_a,  Gj = sum_a (-1)^l bbar_j grad A_a
            const float x2 = 2.f * x, y2 = 2.f * y, z2 = 2.f * z;
            const float gkx = fmaf(z, bk[8], fmaf(y, bk[7], fmaf(x2, bk[4], bk[1])));
            const float gky = fmaf(z, bk[9], fmaf(x, bk[7], fmaf(y2, bk[5], bk[2])));
            const float gkz = fmaf(y, bk[9], fmaf(x, bk[8], fmaf(z2, bk[6], bk[3])));
            const float gjx = fmaf(z, bj[8], fmaf(y, bj[7], fmaf(x2, bj[4], -bj[1])));
            const float gjy = fmaf(z, bj[9], fmaf(x, bj[7], fmaf(y2, bj[5], -bj[2])));
            const float gjz = fmaf(y, bj[9], fmaf(x, bj[8], fmaf(z2, bj[6], -bj[3])));
            // Sk = sum_a A_a bbar_k,  Sj = sum_a (-1)^l A_a bbar_j  (also cbar's edge term): both are
            // quadratics P(r) = p0 + l.r + r^T M r, and P = p0 + (r . (l + grad P)) / 2
            const float Sk = fmaf(0.5f, fmaf(z, bk[3] + gkz, fmaf(y, bk[2] + gky, x * (bk[1] + gkx))), bk[0]);
            const float Sj = fmaf(0.5f, fmaf(z, gjz - bj[3], fmaf(y, gjy - bj[2], x * (gjx - bj[1]))), bj[0]);
            // radial part (d phi / dd) A along r/d, angular part phi grad A
            const float sc = fmaf(cj * dphi, Sk, ck * dphi * Sj) * inv_d;
            const float qv = cj * phi, qt = ck * phi;
            gx -= fmaf(sc, x, fmaf(qv, gkx, qt * gjx));
            gy -= fmaf(sc, y, fmaf(qv, gky, qt * gjy));
            gz -= fmaf(sc, z, fmaf(qv, gkz, qt * gjz));
            if (WANT_CBAR) cb = fmaf(phi, Sj, cb);
            if (WANT_VIR) {
                // dE/dr_e of this edge: the bbar_k c_j part
                const float sa = cj * dphi * Sk * inv_d;
                const float t3[3] = {fmaf(sa, x, qv * gkx), fmaf(sa, y, qv * gky), fmaf(sa, z, qv * gkz)};
                const float r3[3] = {x, y, z};
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) w[3 * a + b] = fmaf(-t3[a], r3[b], w[3 * a + b]);
            }
        };
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            float bj[12];
            gather(s, bj);
            edge(s, bj);
        }
        __syncwarp();
        j_cur = j_nx;
        j_nx = j_nx2;
    }
#pragma unroll
    for (int o = 1; o <= 4; o <<= 1) {
        gx += __shfl_xor_sync(FULL, gx, o);
        gy += __shfl_xor_sync(FULL, gy, o);
        gz += __shfl_xor_sync(FULL, gz, o);
    }
    if (WANT_VIR) {
#pragma unroll
        for (int o = 1; o <= 4; o <<= 1)
#pragma unroll
            for (int q = 0; q < 9; ++q) w[q] += __shfl_xor_sync(FULL, w[q], o);
    }
    if (!valid) return;
    if (m == 0) {
        float* gr = grad + (size_t)atom * 3;
        if (out.first) {  // the first reverse layer starts the sums (no memset)
            gr[0] = gx;
            gr[1] = gy;
            gr[2] = gz;
        } else {
            gr[0] += gx;
            gr[1] += gy;
            gr[2] += gz;
        }
        if (out.forces) {  // the last layer: F = -dE/dr and eps_i in caller order
            const int64_t c = out.perm[atom];
            out.forces[3 * c] = -gr[0];
            out.forces[3 * c + 1] = -gr[1];
            out.forces[3 * c + 2] = -gr[2];
            if (out.atom_energy) out.atom_energy[c] = out.eps[atom];
        }
        if (WANT_VIR) {
            float* vr = vir + (size_t)atom * 9;
#pragma unroll
            for (int q = 0; q < 9; ++q) vr[q] = out.first ? w[q] : vr[q] + w[q];
        }
    }
    if (WANT_CBAR) cbar[(size_t)atom * NPHI + m] = cb;
}

// ------------------------------------------------------- small kernels ---
__device__ __forceinline__ int64_t ghosts_in_use(const int32_t* g_count, int64_t g_cap) {
    const int64_t g = *g_count;
    return g < g_cap ? g : g_cap;
}

// first-layer coefficients c0 of owned rows [0, n_rows) and ghost slots n + [0, g_rows)
__global__ void k_init_coef(int64_t n, int64_t n_rows, int64_t g_rows, const int32_t* __restrict__ g_count,
                            int64_t g_cap, const int32_t* __restrict__ species, const int32_t* __restrict__ owner,
                            const float* __restrict__ c0, float* __restrict__ coef) {
    pdl_enter();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t s, o;
    if (t < n_rows) {
        s = o = t;
    } else {
        const int64_t gi = t - n_rows;
        if (gi >= g_rows || gi >= ghosts_in_use(g_count, g_cap)) return;
        s = n + gi;
        o = owner[gi];
    }
    const int e = species[o];
    const float4* src = reinterpret_cast<const float4*>(c0 + e * NPHI);
    float4* dst = reinterpret_cast<float4*>(coef + (size_t)s * NPHI);
    dst[0] = src[0];
    dst[1] = src[1];
}

// ghost rows <- owner rows (the per-layer ghost refresh of Fig. 4a), width in floats, multiple of 4
__global__ void k_gather_rows(int64_t n, const int32_t* __restrict__ g_count, int64_t g_cap, int w4,
                              const int32_t* __restrict__ owner, float* __restrict__ base) {
    pdl_enter();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ghosts_in_use(g_count, g_cap) * w4) return;
    const int64_t gi = t / w4;
    const int c = (int)(t - gi * w4);
    float4* b = reinterpret_cast<float4*>(base);
    b[(n + gi) * w4 + c] = b[(int64_t)owner[gi] * w4 + c];
}

constexpr int kSumThreads = 256, kSumPer = 8;

__global__ void __launch_bounds__(kSumThreads) k_energy_partial(int64_t n, const float* __restrict__ eps,
                                                               double* __restrict__ partial) {
    pdl_enter();
    __shared__ double sm[kSumThreads];
    const int64_t base = (int64_t)blockIdx.x * kSumThreads * kSumPer;
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kSumPer; ++k) {
        const int64_t i = base + k * kSumThreads + threadIdx.x;
        if (i < n) s += (double)eps[i];
    }
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = kSumThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

__global__ void __launch_bounds__(kSumThreads) k_energy_final(int np, const double* __restrict__ partial,
                                                             double* __restrict__ energy) {
    pdl_enter();
    __shared__ double sm[kSumThreads];
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += kSumThreads) s += partial[i];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = kSumThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) energy[0] = sm[0];
}

// FP64 sum of the per-atom virials (N x 9): partial sums per 2048 atoms, then one block
__global__ void __launch_bounds__(kSumThreads) k_virial_partial(int64_t n, const float* __restrict__ vir,
                                                               double* __restrict__ partial) {
    pdl_enter();
    __shared__ double sm[kSumThreads];
    const int64_t base = (int64_t)blockIdx.x * kSumThreads * kSumPer;
    for (int c = 0; c < 9; ++c) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < kSumPer; ++k) {
            const int64_t i = base + k * kSumThreads + threadIdx.x;
            if (i < n) s += (double)vir[9 * i + c];
        }
        sm[threadIdx.x] = s;
        __syncthreads();
        for (int o = kSumThreads / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[9 * blockIdx.x + c] = sm[0];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kSumThreads) k_virial_final(int np, const double* __restrict__ partial,
                                                             double* __restrict__ out) {
    pdl_enter();
    __shared__ double sm[kSumThreads];
    for (int c = 0; c < 9; ++c) {
        double s = 0.0;
        for (int i = threadIdx.x; i < np; i += kSumThreads) s += partial[9 * i + c];
        sm[threadIdx.x] = s;
        __syncthreads();
        for (int o = kSumThreads / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[c] = sm[0];
        __syncthreads();
    }
}

__global__ void k_unpermute_rows(int64_t n, int width, const int32_t* __restrict__ perm, const float* __restrict__ src,
                                 int src_stride, float* __restrict__ dst) {
    pdl_enter();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * width) return;
    const int64_t i = t / width;
    const int c = (int)(t - i * width);
    dst[(int64_t)perm[i] * width + c] = src[i * src_stride + c];
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_init_coef(cudaStream_t s, const reann_nlist* nl, const float* c0) {
    const int64_t nr = rows_of(nl), gr = ghost_rows_of(nl);
    if (nr + gr == 0) return cudaSuccess;
    launch_pdl(k_init_coef, blocks_for(nr + gr, 256), 256, 0, s, nl->n, nr, gr, ghost_count_ptr(nl), nl->g_cap,
               nl->species, nl->g_owner, c0, nl->coef);
    return cudaGetLastError();
}

cudaError_t launch_gather_ghost_rows(cudaStream_t s, const reann_nlist* nl, float* base, int width) {
    const int64_t gr = ghost_rows_of(nl);
    if (gr == 0) return cudaSuccess;
    const int w4 = width / 4;
    launch_pdl(k_gather_rows, blocks_for(gr * w4, 256), 256, 0, s, nl->n, ghost_count_ptr(nl), gr, w4, nl->g_owner,
               base);
    return cudaGetLastError();
}

// Preferred shared-memory carveout (percent of the 228 KB maximum) of the edge
// kernels; the rest of the 256 KB per SM serves as L1 for the neighbour
// gathers.  40 % (a 100 KB configuration) holds four forward blocks and 50 %
// (132 KB) sixteen adjoint blocks, their occupancy limits by registers (60 % and
// 80 % were 1 % and 4 % slower for the adjoint); on the
// 24,576-atom water box this is 2 % faster for the forward than the driver's
// choice, and a 0 % hint (fewer resident blocks) 1.5-6 x slower.
constexpr int kFwdCarveout = 40;
constexpr int kAdjCarveout = 50;
static void ensure_edge_attrs() {
    static std::mutex mu;
    static uint64_t done = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 64 && ((done >> dev) & 1)) return;
    const auto carve = [](const void* k, int pct) {
        if (pct >= 0) cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    };
    carve((const void*)k_density_fwd<false>, kFwdCarveout);
    carve((const void*)k_density_fwd<true>, kFwdCarveout);
    carve((const void*)k_density_adj8<false, false>, kAdjCarveout);
    carve((const void*)k_density_adj8<false, true>, kAdjCarveout);
    carve((const void*)k_density_adj8<true, false>, kAdjCarveout);
    carve((const void*)k_density_adj8<true, true>, kAdjCarveout);
    if (dev < 64) done |= (uint64_t)1 << dev;
}

cudaError_t launch_density_fwd(cudaStream_t s, const reann_nlist* nl, const Radial& r, const float* W, const float* coef,
                               float* rho, float* bck, bool pairs) {
    ensure_edge_attrs();
    const int64_t per_block = kWarps * kAtomsPerWarp;
    const int64_t nr = rows_of(nl);
    if (nr == 0) return cudaSuccess;
    const unsigned nb = blocks_for(nr, per_block);
    if (pairs)
        launch_pdl(k_density_fwd<true>, nb, kWarps * 32, 0, s, nr, nl->stride, r, nl->live, nl->live_cnt, nl->pos_hi,
                   nl->pos_lo, coef, W, rho, bck);
    else
        launch_pdl(k_density_fwd<false>, nb, kWarps * 32, 0, s, nr, nl->stride, r, nl->live, nl->live_cnt, nl->pos_hi,
                   nl->pos_lo, coef, W, rho, bck);
    return cudaGetLastError();
}

cudaError_t launch_bbar(cudaStream_t s, const reann_nlist* nl, const float* W, const float* bck, const float* rhobar,
                        const float* coef, float* rec, bool pairs, GhostOut gh) {
    const int64_t nr = rows_of(nl);
    if (nr == 0) return cudaSuccess;
    if (pairs)
        launch_pdl(k_bbar<true>, blocks_for(nr, kBbarAtoms), 4 * kBbarAtoms, 0, s, nr, W, bck, rhobar, coef, rec, gh);
    else
        launch_pdl(k_bbar<false>, blocks_for(nr, kBbarAtoms), 4 * kBbarAtoms, 0, s, nr, W, bck, rhobar, coef, rec, gh);
    return cudaGetLastError();
}

cudaError_t upload_pair_table() {
    unsigned char k1[NORB_P * (NORB_P + 1) / 2], k2[NORB_P * (NORB_P + 1) / 2];
    int p = 0;
    for (int a = 0; a < NORB_P; ++a)
        for (int b = a; b < NORB_P; ++b, ++p) {
            k1[p] = (unsigned char)a;
            k2[p] = (unsigned char)b;
        }
    cudaError_t e = cudaMemcpyToSymbol(c_pair_k, k1, sizeof(k1));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_pair_k2, k2, sizeof(k2));
    return e;
}

cudaError_t launch_density_adj(cudaStream_t s, const reann_nlist* nl, const Radial& r, const float* rec, float* cbar,
                               float* grad, bool want_cbar, int* flags, float* vir, float* forces, float* atom_energy,
                               bool first) {
    const Outputs out{forces ? nl->perm : nullptr, forces ? nl->eps : nullptr, forces, atom_energy, first};
    (void)flags;
    ensure_edge_attrs();
    const int64_t per_block = kAdjWarps * kAdjGroups;
    const int64_t nr = rows_of(nl);
    if (nr == 0) return cudaSuccess;
    const unsigned nb = blocks_for(nr, per_block);
#define REANN_ADJ(C, V)                                                                                              \
    launch_pdl(k_density_adj8<C, V>, nb, kAdjWarps * 32, 0, s, nr, nl->stride, r, nl->live, nl->live_cnt,       \
               nl->pos_hi, nl->pos_lo, rec, cbar, grad, vir, out)
    if (want_cbar && vir)
        REANN_ADJ(true, true);
    else if (want_cbar)
        REANN_ADJ(true, false);
    else if (vir)
        REANN_ADJ(false, true);
    else
        REANN_ADJ(false, false);
#undef REANN_ADJ
    return cudaGetLastError();
}

cudaError_t launch_virial_sum(cudaStream_t s, const reann_nlist* nl, const float* vir, double* partial, double* out) {
    const int np = (int)blocks_for(nl->n, kSumThreads * kSumPer);
    launch_pdl(k_virial_partial, np, kSumThreads, 0, s, nl->n, vir, partial);
    launch_pdl(k_virial_final, 1, kSumThreads, 0, s, np, partial, out);
    return cudaGetLastError();
}

cudaError_t launch_energy_sum(cudaStream_t s, const reann_nlist* nl, double* energy) {
    const int np = (int)blocks_for(nl->n, kSumThreads * kSumPer);
    launch_pdl(k_energy_partial, np, kSumThreads, 0, s, nl->n, nl->eps, nl->partial);
    launch_pdl(k_energy_final, 1, kSumThreads, 0, s, np, nl->partial, energy);
    return cudaGetLastError();
}

cudaError_t launch_energy_final(cudaStream_t s, const double* partial, int np, double* energy) {
    launch_pdl(k_energy_final, 1, kSumThreads, 0, s, np, partial, energy);
    return cudaGetLastError();
}

cudaError_t launch_unpermute_rows(cudaStream_t s, const reann_nlist* nl, const float* src, int src_stride, float* dst,
                                  int width) {
    launch_pdl(k_unpermute_rows, blocks_for(nl->n * width, 256), 256, 0, s, nl->n, width, nl->perm, src, src_stride,
               dst);
    return cudaGetLastError();
}

}  // namespace reann
