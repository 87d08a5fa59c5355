// Internal declarations shared by the library's translation units.
// Fixed model shape (Sec. 2.1): N_phi = 8 primitive Gaussians, L = 2
// (10 Cartesian terms x^lx y^ly z^lz), N_orb = 16 orbitals, F = 48 features,
// atomic networks 48 -> 64 -> 64 -> {8 | 1}.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/reann.h"

namespace reann {

constexpr int NPHI = 8;
constexpr int NANG = 10;  // angular terms for L = 2
constexpr int LMAX = 2;
constexpr int NORB = 16;
constexpr int NFEAT = (LMAX + 1) * NORB;  // 48
// orbital-pair-product features: 8 orbitals, (L+1) 8 (8+1)/2 = 108 features
constexpr int NORB_P = 8;
constexpr int NFEAT_P = (LMAX + 1) * NORB_P * (NORB_P + 1) / 2;
constexpr int NB = NANG * NPHI;           // 80 per-atom density partials b_{a,m}
// Adjoint record of an atom (the reverse pass's per-atom row): 3 lines of
// 128 B, line v / 4 holding value v of channel m at float 4 m + v % 4, with
// values v = 0..9 the adjoint bbar_{a = v, m}, v = 10 the coefficient c_m of
// the layer and v = 11 zero.  Channel m's 12 values are then 3 aligned float4s,
// one per line, so the 8 lanes of an atom read one full line per load.
constexpr int NREC = 3 * 4 * NPHI;  // 96 floats
__host__ __device__ constexpr int rec_at(int v, int m) { return (v >> 2) * (4 * NPHI) + 4 * m + (v & 3); }
constexpr int H1 = 64;
constexpr int H2 = 64;
constexpr int MAX_ELEM = 8;
constexpr int MLP_TILE = 64;  // rows per FP32 network tile

// Internal angular order: 1, x, y, z, xx, yy, zz, xy, xz, yz.
// l(a), multinomial weight l!/(lx! ly! lz!) and parity (-1)^l.
#ifdef __CUDACC__
__device__ __forceinline__ int ang_l(int a) { return a == 0 ? 0 : (a < 4 ? 1 : 2); }
__device__ __forceinline__ float ang_w(int a) { return a >= 7 ? 2.f : 1.f; }
__device__ __forceinline__ float ang_sign(int a) { return (a >= 1 && a <= 3) ? -1.f : 1.f; }

// Programmatic dependent launch.  A kernel started by launch_pdl() may become
// resident while the previous kernel on its stream is still draining; before
// it reads or writes global memory that an earlier kernel of the stream reads
// or writes, and on every path before it exits, it runs pdl_enter():
// griddepcontrol.wait returns once every prerequisite grid has completed and
// its writes are visible (so completion stays transitive along the stream),
// and launch_dependents then lets the next kernel be scheduled early.  Without
// a programmatic prerequisite both instructions return at once.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
#endif

// Device-side error flags (ctx->d_flags)
enum Flag {
    FLAG_GEOM = 0,
    FLAG_NBR_OVERFLOW = 1,
    FLAG_GHOST_OVERFLOW = 2,
    FLAG_MAXNBR = 3,
    FLAG_SPECIES = 4,
    FLAG_MOVED = 5,
    FLAG_TIMEOUT = 6,
    FLAG_TIMEOUT_DRAIN = 7,  // after a timeout, the CTA's own MMAs or copies did not complete either
    NFLAGS = 8
};

// Ghost slots filled by their owners: ghost slot g (row base + g) copies owned
// row i for g in [goff[i], goff[i+1]) (the single-domain list enumerates each
// atom's images contiguously), g < gcap.  goff == nullptr: the caller gathers.
struct GhostOut {
    const int32_t* goff = nullptr;
    int64_t base = 0, gcap = 0;
};

#ifdef __CUDACC__
// Staging of a tile's records in shared memory: row stride 100 floats, so that
// the 4 threads of a row writing value v of channel m (8 rows per warp) hit 32
// distinct banks, and every row starts on a 16 B boundary.
constexpr int kRecLd = NREC + 4;
__device__ __forceinline__ void stage_rec(float* __restrict__ sRec, int r, int v, const float val[NPHI]) {
#pragma unroll
    for (int m = 0; m < NPHI; ++m) sRec[r * kRecLd + rec_at(v, m)] = val[m];
}
// Copies the staged records of rows row0 .. row0 + nrows - 1 to global memory
// with float4 stores (whole 128 B lines), and to the rows' ghost images when
// gh.goff is set.
__device__ __forceinline__ void flush_rec(const float* __restrict__ sRec, int nrows, int64_t row0,
                                          float* __restrict__ rec, const GhostOut& gh, int tid, int nthreads) {
    constexpr int W4 = NREC / 4;
    for (int i = tid; i < nrows * W4; i += nthreads) {
        const int r = i / W4, c = i - r * W4;
        const float4 x = *reinterpret_cast<const float4*>(sRec + r * kRecLd + 4 * c);
        const int64_t row = row0 + r;
        reinterpret_cast<float4*>(rec + (size_t)row * NREC)[c] = x;
        if (gh.goff)
            for (int64_t g = gh.goff[row]; g < gh.goff[row + 1] && g < gh.gcap; ++g)
                reinterpret_cast<float4*>(rec + (size_t)(gh.base + g) * NREC)[c] = x;
    }
}

// The bbar step of one angular term a of one atom (Eq. 1's squares):
//   bbar_{a,m} = sum_k W_{l,m,k} gbar_{a,k},  gbar_{a,k} = 2 w_a rhobar_{l,k} sum_m' b_{a,m'} W_{l,m',k}
// bm = b_{a,0..7}, Wl = W_{l} (N_phi x N_orb, row-major, 16 B aligned), rb = rhobar_{l,0..15}
// (16 B aligned); blocked over 4 orbitals (W fragments are float4 loads, read again
// for the second product rather than held in registers).
__device__ __forceinline__ void bbar_term(const float bm[NPHI], float two_w, const float* Wl, const float* rb,
                                          float out[NPHI]) {
#pragma unroll
    for (int m = 0; m < NPHI; ++m) out[m] = 0.f;
#pragma unroll
    for (int k4 = 0; k4 < NORB; k4 += 4) {
        float g[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int m = 0; m < NPHI; ++m) {
            const float4 w = *reinterpret_cast<const float4*>(Wl + m * NORB + k4);
            g[0] = fmaf(bm[m], w.x, g[0]);
            g[1] = fmaf(bm[m], w.y, g[1]);
            g[2] = fmaf(bm[m], w.z, g[2]);
            g[3] = fmaf(bm[m], w.w, g[3]);
        }
        const float4 r = *reinterpret_cast<const float4*>(rb + k4);
        const float gb[4] = {two_w * g[0] * r.x, two_w * g[1] * r.y, two_w * g[2] * r.z, two_w * g[3] * r.w};
#pragma unroll
        for (int m = 0; m < NPHI; ++m) {
            const float4 w = *reinterpret_cast<const float4*>(Wl + m * NORB + k4);
            out[m] = fmaf(gb[0], w.x, fmaf(gb[1], w.y, fmaf(gb[2], w.z, fmaf(gb[3], w.w, out[m]))));
        }
    }
}

// Values 10 and 11 of the record: the layer's coefficients c_m of `row`, and zero.
__device__ __forceinline__ void rec_tail(const float* __restrict__ coef, int64_t row, int v, float val[NPHI]) {
    if (v == NANG) {
        const float4 c0 = __ldg(reinterpret_cast<const float4*>(coef + (size_t)row * NPHI));
        const float4 c1 = __ldg(reinterpret_cast<const float4*>(coef + (size_t)row * NPHI + 4));
        val[0] = c0.x, val[1] = c0.y, val[2] = c0.z, val[3] = c0.w;
        val[4] = c1.x, val[5] = c1.y, val[6] = c1.z, val[7] = c1.w;
    } else {
#pragma unroll
        for (int m = 0; m < NPHI; ++m) val[m] = 0.f;
    }
}
#endif

// Named regions of the optional per-kernel event profile (reann_ctx_profile).
enum ProfRegion {
    PR_REBUILD = 0,
    PR_REFRESH,
    PR_LIVE,
    PR_INIT,
    PR_GATHER,
    PR_DENSITY_FWD,
    PR_MLP_FWD,
    PR_ENERGY,
    PR_MLP_BWD,
    PR_BBAR,
    PR_DENSITY_ADJ,
    PR_OUTPUT,
    PR_COUNT
};

// Constants of the radial basis, passed by value to kernels.  Constants that
// enter every edge identically are split into a float pair (hi + lo) so that
// their FP32 rounding does not bias all atoms the same way (in a crystal every
// atom sees the same neighbour shells, so a rounded constant would shift every
// atomic energy by the same amount).
struct Radial {
    float rc, rc2;
    float inv_rc_hi, inv_rc_lo;  // 1 / r_c as a float pair
    float alpha_hi, alpha_lo;  // alpha
    float tad_hi, tad_lo;      // 2 alpha Delta, Delta = r_c / (N_phi - 1)
    float mu_hi[NPHI], mu_lo[NPHI];      // Gaussian centres m Delta
    float kap_hi[NPHI], kap_lo[NPHI];    // exp(-alpha Delta^2 (2m+1)) for the Gaussian recurrence
};

// Cell geometry for the neighbour build (FP64) and ghost refresh.
struct CellGeom {
    double h[9];     // rows = lattice vectors
    double hinv[9];  // frac = x . hinv
    double reach[3]; // r_cut / width_k + margin (fractional units)
    int nmax[3];     // largest |image shift| per axis
    int nb[3];       // owned bins per axis (internal order), width >= r_cut
    int ns[3];       // search bins per axis, width >= r_cut / 2
    int pad[3];      // extra search bins per side for ghosts
    int nbx[3];      // ns + 2 pad
    int sw[3];       // stencil half-width in search bins per axis
    int ortho;       // rectangular cell with a positive diagonal: the search trims each stencil column
    float binw[3];   // search-bin widths (A) of a rectangular cell, and their inverses
    float binw_inv[3];
    double rcut2;    // (r_c + skin)^2
    float rcut2_f;
    float margin;    // FP32 pre-test band around rcut2 (A^2) decided in FP64
};

struct Model {
    int n_elem, T;
    double r_c, alpha;
    bool pairs = false;  // orbital-pair-product features instead of Eq. 1's squares
    int n_orb() const { return pairs ? NORB_P : NORB; }
    int n_feat() const { return pairs ? NFEAT_P : NFEAT; }
    std::vector<float> params;  // host copy, flat layout of reann.h
};

// Per-layer/element network weights on the device.
struct NetDev {
    const float* W1;  // [48][64]
    const float* b1;  // [64]
    const float* W2;  // [64][64]
    const float* b2;  // [64]
    const float* W3;  // [64][out]
    const float* b3;  // [out]
    const float* W1t; // [64][48]
    const float* W2t; // [64][64]
    const float* W3t; // [out][64]
};

struct NetTable {
    NetDev net[8][MAX_ELEM];  // [t][e]
};

struct Tile {
    int elem, row0, nrows, pad;
};

// Weights of one (layer, element) network for the tensor-core path.  B
// operands (N rows of K, K-major core-matrix layout, see mlp_tc.cu):
//   BF16  forward  W1^T (64 x 48) | W2^T (64 x 64)   14336 B, hi then lo (BF16
//         backward W2   (64 x 64) | W1   (48 x 64)   rounding of w - hi) each
//   FP8   forward  W1^T (64 x 64, K padded) | W2^T (64 x 64)     8192 B
//         backward W2   (64 x 64)           | W1   (48 x 64)     7168 B
// with every B row divided by its own scale max |w| / 448 (s8).  The FP32
// copies serve the anchors and the FP32 output layer.
struct TcImg {
    const uint8_t* wf;   // BF16 forward images (hi | lo)
    const uint8_t* wb;   // BF16 backward images (hi | lo)
    const uint8_t* wf8;  // FP8 forward image
    const uint8_t* wb8;  // FP8 backward image
    const float *W1, *W2, *W3, *W1t, *W2t, *b1, *b2, *b3;
    const float* s8;     // FP8 B-row scales: forward W1^T (64), W2^T (64), backward W2 (64), W1 (48)
};
constexpr uint32_t kBfImg = 14336;
constexpr uint32_t kF8Fwd = 8192;
constexpr uint32_t kF8Bwd = 7168;
constexpr uint32_t kF8Img = kF8Fwd + kF8Bwd;
constexpr int kF8Scales = 64 + 64 + 64 + 48;
struct TcTable {
    TcImg img[8][MAX_ELEM];
};

// Resident scratch of the neighbour build, kept so that rebuilds neither
// allocate nor synchronise.
struct NlistScratch {
    double *xw_c = nullptr, *fw_c = nullptr, *xw = nullptr, *fw = nullptr;  // wrapped Cartesian / fractional
    int32_t *mw_c = nullptr, *key = nullptr, *counts = nullptr, *start = nullptr;
    int32_t *gcnt = nullptr, *goff = nullptr;  // ghosts per atom and offsets; goff[n] = ghost count
    int32_t* halo = nullptr;                    // per atom and axis: the image interval (pack_halo)
    int32_t* species_c = nullptr;              // caller-order species
    int32_t *ekey = nullptr, *ecounts = nullptr, *estart = nullptr, *eorder = nullptr;
    int32_t *scat = nullptr, *escat = nullptr;  // atomic-order scatter before the in-bucket ranking
    int32_t *tsum = nullptr, *etsum = nullptr;  // look-back status words of the scans (owned / extended)
    int32_t* rb_state = nullptr;  // rebuilds since the last sort, sort gate, keep-order gate
    float4* p32 = nullptr;   // FP32 positions of owned + ghost slots for the pre-test
    float4* p32s = nullptr;  // the same in bin-sorted order, slot index in .w
};

// A call replayed as a CUDA graph: the arguments it was captured with (key),
// and whether the same call has run once uncaptured (seen) or cannot be
// captured (nograph).
struct GraphSlot {
    const void* key[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int ikey[4] = {0, 0, 0, 0};
    bool seen = false, nograph = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};
enum GraphSlotId { GS_REBUILD = 0, GS_EVAL, GS_HOST_REBUILD, GS_HOST_EVAL, GS_COUNT };

}  // namespace reann

struct reann_model {
    reann::Model m;
};

struct reann_nlist {
    int64_t n = 0, g = 0, g_cap = 0;  // atoms, ghosts, ghost capacity
    // Bounds of the work an evaluation launches for (a serving pool sets them per launch
    // to the rows and ghost slots in use, rounded up to a size class; -1: all): owned rows
    // [0, n_rows), ghost slots [n, n + g_rows), network tiles [0, tiles_active) and
    // [0, tiles128_active) of the tile lists.
    int64_t n_rows = -1, g_rows = -1;
    int64_t tiles_active = -1, tiles128_active = -1;
    int stride = 0;                   // neighbour row capacity
    int max_count = 0;                // longest row found by the first build
    int n_elem = 0, T = 0;
    int n_feat = reann::NFEAT;        // features per atom of the model the buffers were sized for
    double r_c = 0, skin = 0;
    reann::CellGeom geom{};
    int elem_start[reann::MAX_ELEM + 1] = {0};
    std::vector<reann::Tile> tiles_h;
    // device arrays
    int32_t* perm = nullptr;       // internal -> caller
    int32_t* species = nullptr;    // internal order
    int32_t* wrapm = nullptr;      // N x 3 wrap shifts m (x_w = x - m.H), internal order
    int32_t* g_owner = nullptr;    // g_cap
    int32_t* g_shift = nullptr;    // g_cap, packed (n0+128) | (n1+128)<<8 | (n2+128)<<16
    int32_t* nbr = nullptr;        // N x stride ext slots
    int32_t* nbr_cnt = nullptr;    // N
    int32_t* live = nullptr;       // N x stride, live (d < r_c) entries first
    int32_t* live_cnt = nullptr;   // N
    reann::Tile* tiles = nullptr;  // MLP tiles (64 rows, FP32 networks)
    std::vector<reann::Tile> tiles128_h;
    reann::Tile* tiles128 = nullptr;  // 128-row tiles of the tensor-core networks
    double* pos_ref = nullptr;     // N x 3 FP64 caller positions at build (caller order)
    // per-evaluation state (resident)
    float4* pos_hi = nullptr;      // N + g_cap
    float4* pos_lo = nullptr;      // N + g_cap
    float* coef = nullptr;         // T x (N + g_cap) x 8
    float* rho = nullptr;          // T x N x 48
    float* bck = nullptr;          // T x N x 80
    float* eps = nullptr;          // N
    float* rhobar = nullptr;       // N x 48
    float* dsave = nullptr;        // T x N x 128 SiLU'(z1), SiLU'(z2) of the FP32 networks
    float* bbar = nullptr;         // (N + g_cap) x 96 adjoint records (bbar, c)
    float* cbar = nullptr;         // N x 8
    float* grad = nullptr;         // N x 3
    float* vir = nullptr;          // N x 9 per-atom virial (allocated on first request)
    double* vir_partial = nullptr; // virial partial sums
    double* partial = nullptr;     // energy partial sums
    int n_partial = 0;
    reann::NlistScratch w;
    // host-buffer entry point staging
    double* h2d_pos = nullptr;     // N x 3
    double* d_energy = nullptr;    // 1
    float* d_forces = nullptr;     // N x 3
    // MD state: forces of the current positions, per-step energies, rebuild gate, graph
    float* md_forces = nullptr;    // N x 3 (caller order)
    double* md_scalars = nullptr;  // [0] E_pot, [1] E_kin, [2] xi, [3] eta, [4] velocity scale
    double* md_partial = nullptr;
    int* md_ints = nullptr;        // [0] rebuild gate, [1] step counter, [2] rebuild count
    bool md_forces_valid = false;
    const double* md_forces_at = nullptr;  // positions the forces belong to
    cudaGraph_t md_graph = nullptr;
    cudaGraphExec_t md_exec = nullptr;
    reann::GraphSlot graphs[reann::GS_COUNT];  // rebuild / evaluation calls replayed as graphs
    const void* md_key[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    double md_dt = 0.0;
    double md_kt = 0.0, md_tau = 0.0;  // thermostat of the captured step (tau 0: NVE)
    int md_precision = -1, md_nsteps = -1;
    // spatial decomposition into virtual ranks (reann_build_nlist_decomposed):
    // per rank its local atoms, ghost slots, and ghost slots owned by another rank
    bool decomposed = false;
    bool ghosts_by_owner = false;  // ghost slots of owned row i are [goff[i], goff[i+1]) (single-domain build)
    int rank_grid[3] = {1, 1, 1};
    std::vector<int64_t> rank_local, rank_ghost, rank_remote;
    std::vector<void*> allocs;
    // stream-ordered allocation (serving builds): blocks come from mem_pool on
    // alloc_stream and go back with cudaFreeAsync on the same stream, so neither
    // side waits for unrelated device work; null pool: cudaMalloc / cudaFree
    cudaMemPool_t mem_pool = nullptr;
    cudaStream_t alloc_stream = nullptr;
};

struct reann_ctx {
    reann::Model model;
    cudaStream_t stream = nullptr;
    int device = 0;
    int precision = REANN_MLP_FP32;
    reann::Radial radial{};
    float* d_params = nullptr;     // model parameters (FP32, flat + transposed copies)
    reann::NetTable nets{};
    const float* d_c0 = nullptr;   // [n_elem][8]
    const float* d_W = nullptr;    // [T][3][8][16]
    void* d_bf16 = nullptr;        // BF16 weight images for the tensor-core networks
    void* d_fp8 = nullptr;         // FP8 E4M3 weight images for the tensor-core networks
    reann::TcTable tc{};
    int* d_flags = nullptr;        // reann::NFLAGS ints
    int* h_flags = nullptr;        // pinned mirror
    std::string err;
    int num_sms = 0;
    // a non-blocking stream the MD step graph and the replayed rebuild / evaluation graphs run on
    cudaStream_t md_stream = nullptr;
    cudaEvent_t md_ev[2] = {nullptr, nullptr};
    // optional per-region event profile
    bool prof_on = false;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_recs;
    std::vector<cudaEvent_t> prof_pool;
    double prof_ms[reann::PR_COUNT] = {0};
    int64_t prof_n[reann::PR_COUNT] = {0};
};

namespace reann {

// the launch bounds of an evaluation of nl (see reann_nlist::n_rows)
inline int64_t rows_of(const reann_nlist* nl) { return nl->n_rows >= 0 ? nl->n_rows : nl->n; }
inline int64_t ghost_rows_of(const reann_nlist* nl) { return nl->g_rows >= 0 ? nl->g_rows : nl->g_cap; }
inline int64_t tiles_of(const reann_nlist* nl) {
    return nl->tiles_active >= 0 ? nl->tiles_active : (int64_t)nl->tiles_h.size();
}
inline int64_t tiles128_of(const reann_nlist* nl) {
    return nl->tiles128_active >= 0 ? nl->tiles128_active : (int64_t)nl->tiles128_h.size();
}

int set_error(reann_ctx* ctx, int code, const std::string& msg);

// Launches k with the programmatic-stream-serialization attribute; every
// kernel of the library calls pdl_enter() first.  In a captured graph the
// attribute becomes a programmatic edge.  The network kernels are launched
// without it: their grids are one wave of tiles, and blocks that become
// resident while the previous kernel drains pile up on the SMs that freed
// first (measured: FP32 step 0.489 -> 0.502 ms with them, 0.489 -> 0.487 ms
// for the edge and rebuild kernels alone).
template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A... args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, static_cast<P>(args)...);
}

#define REANN_CUDA_TRY(ctx, expr)                                                                   \
    do {                                                                                            \
        cudaError_t _e = (expr);                                                                    \
        if (_e != cudaSuccess)                                                                      \
            return ::reann::set_error((ctx), REANN_E_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)

// ---- launchers (defined in the .cu files) ----
// neighbour list (nlist.cu)
int build_nlist_device(reann_ctx* ctx, reann_nlist* nl, const double* pos, const int32_t* species);
cudaError_t launch_rebuild(cudaStream_t s, reann_nlist* nl, const double* pos, int* flags, const int* gate);
cudaError_t launch_moved(cudaStream_t s, const reann_nlist* nl, const double* pos, int* moved);

// serving pool (serve.cu)
cudaError_t launch_pack(cudaStream_t s, const reann_nlist* src, const double* caller_pos, reann_nlist* pool,
                        int64_t ob, int64_t gb);
void* nlist_alloc_bytes(reann_nlist* nl, size_t bytes);
template <typename T>
inline T* nlist_alloc(reann_nlist* nl, size_t count) {
    return static_cast<T*>(nlist_alloc_bytes(nl, count * sizeof(T)));
}
cudaError_t launch_release(cudaStream_t s, reann_nlist* pool, int64_t ob, int64_t n);
cudaError_t launch_retire(cudaStream_t s, const int4* seg, int nseg, reann_nlist* pool);
cudaError_t launch_segment_energy(cudaStream_t s, const int4* seg, int nseg, const float* eps, double* energies);

// velocity Verlet (md.cu)
cudaError_t launch_kick(cudaStream_t s, int64_t n, double* vel, const float* forces, const double* mass,
                        double half_dt, const double* scale = nullptr);
cudaError_t launch_scale(cudaStream_t s, int64_t n, double* vel, const double* scale);
cudaError_t launch_nh_half(cudaStream_t s, double* scalars, double dt, double gkt, double q);
cudaError_t launch_drift(cudaStream_t s, int64_t n, double* pos, const double* vel, double dt);
cudaError_t launch_ekin(cudaStream_t s, int64_t n, const double* vel, const double* mass, double* partial,
                        double* out);
cudaError_t launch_record(cudaStream_t s, int* counter, const double* scalars, double* epot_out, double* ekin_out,
                          double* bath_out, double gkt, double q, int n_steps, const int* gate, int* rebuilds);
const int32_t* ghost_count_ptr(const reann_nlist* nl);
// with c0: also the first layer's coefficients of every slot (k_init_coef's work)
cudaError_t launch_refresh_positions(cudaStream_t s, const reann_nlist* nl, const double* pos,
                                     const float* c0 = nullptr);
cudaError_t launch_live_edges(cudaStream_t s, const reann_nlist* nl, float rc2, int* flags);
int export_nlist(reann_ctx* ctx, const reann_nlist* nl, int64_t cap, int32_t* i, int32_t* j, int32_t* n, int64_t* count);

// density (density.cu)
cudaError_t launch_init_coef(cudaStream_t s, const reann_nlist* nl, const float* c0);
cudaError_t launch_gather_ghost_rows(cudaStream_t s, const reann_nlist* nl, float* base, int width);
cudaError_t launch_density_fwd(cudaStream_t s, const reann_nlist* nl, const Radial& r, const float* W, const float* coef,
                               float* rho, float* bck, bool pairs = false);
cudaError_t launch_bbar(cudaStream_t s, const reann_nlist* nl, const float* W, const float* bck, const float* rhobar,
                        const float* coef, float* rec, bool pairs = false, GhostOut gh = {});
// forces / atom_energy (caller order): the last reverse layer writes the outputs itself;
// first: the first reverse layer writes grad (and vir) instead of accumulating
cudaError_t launch_density_adj(cudaStream_t s, const reann_nlist* nl, const Radial& r, const float* rec, float* cbar,
                               float* grad, bool want_cbar, int* flags, float* vir = nullptr,
                               float* forces = nullptr, float* atom_energy = nullptr, bool first = false);
cudaError_t upload_pair_table();
cudaError_t launch_virial_sum(cudaStream_t s, const reann_nlist* nl, const float* vir, double* partial, double* out);
cudaError_t launch_energy_sum(cudaStream_t s, const reann_nlist* nl, double* energy);
cudaError_t launch_unpermute_rows(cudaStream_t s, const reann_nlist* nl, const float* src, int src_stride, float* dst,
                                  int width);

// atomic networks, FP32 SIMT (mlp_fp32.cu)
// dsave (N x 128, optional): the forward keeps SiLU'(z1), SiLU'(z2) of every row for the backward;
// epart (energy network, optional): one FP64 energy partial sum per tile (reann_nlist::tiles order)
cudaError_t launch_mlp_fwd_f32(cudaStream_t s, const reann_nlist* nl, const NetTable& nets, int t, bool energy,
                               const float* rho, float* out, int out_stride, bool pairs, GhostOut gh, float* dsave,
                               double* epart, int* flags);
// total energy from np partial sums, in a fixed order
cudaError_t launch_energy_final(cudaStream_t s, const double* partial, int np, double* energy);
// atomic networks on tcgen05 tensor cores (mlp_tc.cu), precision REANN_MLP_BF16,
// REANN_MLP_BF16X3 or REANN_MLP_FP8.  The forward keeps SiLU'(z1), SiLU'(z2) of every
// row in dsave (128 floats per row) and, for the energy network, writes one FP64
// energy partial per 128-row tile to epart (nullable); the backward reads dsave, takes
// the bbar step and writes the adjoint records (rec, ghost images through gh).
cudaError_t launch_mlp_fwd_tc(cudaStream_t s, const reann_nlist* nl, const TcTable& nets, int t, bool energy,
                              int precision, const float* rho, float* out, int out_stride, int* flags,
                              GhostOut gh, float* dsave, double* epart);
cudaError_t launch_mlp_bwd_tc(cudaStream_t s, const reann_nlist* nl, const TcTable& nets, int t, bool energy,
                              int precision, const float* dsave, const float* ybar, const float* Wc, const float* bck,
                              const float* coef, float* rec, GhostOut gh, int* flags);
// one CTA that waits, `polls` times, on an mbarrier nothing arrives on and then takes
// the bounded-wait exit of the tensor-core kernels (reann_ctx_wait_selftest)
cudaError_t launch_wait_selftest(cudaStream_t s, int* flags, long long polls);

cudaError_t launch_mlp_bwd_f32(cudaStream_t s, const reann_nlist* nl, const NetTable& nets, int t, bool energy,
                               const float* dsave, const float* ybar, float* rhobar, int* flags, bool pairs = false,
                               const float* Wt = nullptr, const float* bck = nullptr, const float* coef = nullptr,
                               float* rec = nullptr, GhostOut gh = {});

}  // namespace reann
