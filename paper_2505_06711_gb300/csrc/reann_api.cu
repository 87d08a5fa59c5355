// Host side of the C ABI declared in include/reann.h: argument checks, model
// upload, neighbour-list objects and the order of kernels of one energy +
// force evaluation (T forward layers, then T reverse layers, Sec. 2.1-2.2).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <unordered_map>
#include <vector>

#include "common.cuh"

using namespace reann;

namespace reann {

int set_error(reann_ctx* ctx, int code, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return code;
}

}  // namespace reann

namespace {

constexpr int64_t expected_params(int n_elem, int T, bool pairs = false) {
    const int ko = pairs ? NORB_P : NORB, nf = pairs ? NFEAT_P : NFEAT;
    int64_t n = (int64_t)n_elem * NPHI + (int64_t)T * (LMAX + 1) * NPHI * ko;
    for (int t = 0; t < T; ++t) {
        const int out = (t == T - 1) ? 1 : NPHI;
        n += (int64_t)n_elem * (nf * H1 + H1 + H1 * H2 + H2 + H2 * out + out);
    }
    return n;
}

// cell inverse: frac = x . hinv, with hinv = adj(H) / det(H)
bool cell_inverse(const double* h, double* hinv, double* det_out) {
    const double det = h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) +
                       h[2] * (h[3] * h[7] - h[4] * h[6]);
    if (!(std::fabs(det) > 1e-12) || !std::isfinite(det)) return false;
    hinv[0] = (h[4] * h[8] - h[5] * h[7]) / det;
    hinv[1] = (h[2] * h[7] - h[1] * h[8]) / det;
    hinv[2] = (h[1] * h[5] - h[2] * h[4]) / det;
    hinv[3] = (h[5] * h[6] - h[3] * h[8]) / det;
    hinv[4] = (h[0] * h[8] - h[2] * h[6]) / det;
    hinv[5] = (h[2] * h[3] - h[0] * h[5]) / det;
    hinv[6] = (h[3] * h[7] - h[4] * h[6]) / det;
    hinv[7] = (h[1] * h[6] - h[0] * h[7]) / det;
    hinv[8] = (h[0] * h[4] - h[1] * h[3]) / det;
    *det_out = det;
    return true;
}

int make_geometry(reann_ctx* ctx, const double* cell, double r_cut, CellGeom* g) {
    std::memset(g, 0, sizeof(*g));
    for (int i = 0; i < 9; ++i) {
        if (!std::isfinite(cell[i])) return set_error(ctx, REANN_E_GEOM, "non-finite cell");
        g->h[i] = cell[i];
    }
    double det = 0;
    if (!cell_inverse(g->h, g->hinv, &det)) return set_error(ctx, REANN_E_GEOM, "singular cell");
    double maxc = r_cut;
    for (int k = 0; k < 3; ++k) {
        const double* u = g->h + 3 * ((k + 1) % 3);
        const double* v = g->h + 3 * ((k + 2) % 3);
        const double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
        const double w = std::fabs(det) / std::sqrt(cx * cx + cy * cy + cz * cz);
        const double delta = r_cut / w;
        g->reach[k] = delta + 1e-6;
        g->nmax[k] = (int)std::ceil(g->reach[k]);
        if (g->nmax[k] > 100) return set_error(ctx, REANN_E_GEOM, "cell too thin for the cutoff");
        g->nb[k] = std::max(1, std::min(1024, (int)std::floor(w / r_cut)));
        // half-width search bins: a 5 x 5 x 5 stencil covers 42 % less volume than 3 x 3 x 3 full bins
        g->ns[k] = std::max(1, std::min(1024, (int)std::floor(2.0 * w / r_cut)));
        g->sw[k] = std::max(1, (int)std::ceil(delta * g->ns[k] - 1e-9));
        g->pad[k] = (int)std::ceil(g->reach[k] * g->ns[k]) + 1;
        g->nbx[k] = g->ns[k] + 2 * g->pad[k];
        maxc += std::fabs(g->h[k]) + std::fabs(g->h[3 + k]) + std::fabs(g->h[6 + k]);
    }
    g->ortho = g->h[1] == 0.0 && g->h[2] == 0.0 && g->h[3] == 0.0 && g->h[5] == 0.0 && g->h[6] == 0.0 &&
               g->h[7] == 0.0 && g->h[0] > 0.0 && g->h[4] > 0.0 && g->h[8] > 0.0;
    for (int k = 0; k < 3; ++k) {
        g->binw[k] = (float)(g->h[4 * k] / g->ns[k]);
        g->binw_inv[k] = (float)(g->ns[k] / g->h[4 * k]);
    }
    g->rcut2 = r_cut * r_cut;
    g->rcut2_f = (float)g->rcut2;
    // FP32 positions carry up to half an ulp of the largest coordinate each
    const double ulp = maxc * std::ldexp(1.0, -23);
    g->margin = (float)(16.0 * r_cut * ulp + 1e-4);
    return REANN_OK;
}

template <typename T>
T* nl_alloc(reann_nlist* nl, size_t count) {
    return nlist_alloc<T>(nl, count);
}

// ranges: (element, first row, end row) of the network tiles; default the element ranges
int alloc_eval_buffers(reann_ctx* ctx, reann_nlist* nl, const std::vector<std::array<int, 3>>* ranges = nullptr) {
    const int64_t n = nl->n, ne = nl->n + nl->g_cap, T = nl->T;
    nl->live = nl_alloc<int32_t>(nl, (size_t)n * nl->stride);
    nl->live_cnt = nl_alloc<int32_t>(nl, n);
    nl->pos_hi = nl_alloc<float4>(nl, ne);
    nl->pos_lo = nl_alloc<float4>(nl, ne);
    nl->coef = nl_alloc<float>(nl, (size_t)T * ne * NPHI);
    nl->n_feat = ctx->model.n_feat();
    nl->rho = nl_alloc<float>(nl, (size_t)T * n * nl->n_feat);
    nl->bck = nl_alloc<float>(nl, (size_t)T * n * NB);
    nl->eps = nl_alloc<float>(nl, n);
    nl->rhobar = nl_alloc<float>(nl, (size_t)n * nl->n_feat);
    nl->dsave = nl_alloc<float>(nl, (size_t)T * n * (H1 + H2));
    nl->bbar = nl_alloc<float>(nl, (size_t)ne * NREC);  // adjoint records (bbar with c)
    nl->cbar = nl_alloc<float>(nl, (size_t)n * NPHI);
    nl->grad = nl_alloc<float>(nl, (size_t)n * 3);
    // element tiles of the atomic networks
    std::vector<std::array<int, 3>> own;
    if (!ranges) {
        for (int e = 0; e < nl->n_elem; ++e) own.push_back({e, nl->elem_start[e], nl->elem_start[e + 1]});
        ranges = &own;
    }
    nl->tiles_h.clear();
    nl->tiles128_h.clear();
    for (const auto& rg : *ranges) {
        for (int r = rg[1]; r < rg[2]; r += MLP_TILE) nl->tiles_h.push_back(Tile{rg[0], r, std::min(MLP_TILE, rg[2] - r), 0});
        for (int r = rg[1]; r < rg[2]; r += 128) nl->tiles128_h.push_back(Tile{rg[0], r, std::min(128, rg[2] - r), 0});
    }
    nl->tiles = nl_alloc<Tile>(nl, nl->tiles_h.size());
    // energy partial sums: per 2048 atoms, or per network tile when the energy network sums them
    nl->n_partial = (int)std::max<int64_t>((n + 2047) / 2048, (int64_t)nl->tiles_h.size());
    nl->partial = nl_alloc<double>(nl, nl->n_partial);
    nl->tiles128 = nl_alloc<Tile>(nl, nl->tiles128_h.size());
    if (!nl->tiles128) return set_error(ctx, REANN_E_NOMEM, "evaluation buffers: out of device memory");
    if (!nl->tiles128_h.empty())
        REANN_CUDA_TRY(ctx, cudaMemcpyAsync(nl->tiles128, nl->tiles128_h.data(), sizeof(Tile) * nl->tiles128_h.size(),
                                            cudaMemcpyHostToDevice, ctx->stream));
    if (!nl->live || !nl->live_cnt || !nl->pos_hi || !nl->pos_lo || !nl->coef || !nl->rho || !nl->bck || !nl->eps ||
        !nl->rhobar || !nl->dsave || !nl->bbar || !nl->cbar || !nl->grad || !nl->partial || !nl->tiles)
        return set_error(ctx, REANN_E_NOMEM, "evaluation buffers: out of device memory");
    if (!nl->tiles_h.empty())
        REANN_CUDA_TRY(ctx, cudaMemcpyAsync(nl->tiles, nl->tiles_h.data(), sizeof(Tile) * nl->tiles_h.size(),
                                            cudaMemcpyHostToDevice, ctx->stream));
    // unused ghost capacity keeps finite values; no live edges before the first evaluation
    REANN_CUDA_TRY(ctx, cudaMemsetAsync(nl->bbar, 0, sizeof(float) * ne * NREC, ctx->stream));
    REANN_CUDA_TRY(ctx, cudaMemsetAsync(nl->live_cnt, 0, sizeof(int32_t) * n, ctx->stream));
    return REANN_OK;
}

void free_nlist(reann_nlist* nl) {
    if (!nl) return;
    if (nl->md_exec) cudaGraphExecDestroy(nl->md_exec);
    if (nl->md_graph) cudaGraphDestroy(nl->md_graph);
    for (GraphSlot& g : nl->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
    }
    for (void* p : nl->allocs) {
        if (nl->mem_pool)
            cudaFreeAsync(p, nl->alloc_stream);
        else
            cudaFree(p);
    }
    delete nl;
}

// FP32 -> BF16, round to nearest even
uint16_t to_bf16(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

float from_bf16(uint16_t h) {
    const uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// Append an R x K BF16 tile (src row-major with leading dimension ld, entries
// beyond rows x cols zero) in the K-major core-matrix layout used by
// tcgen05.mma: 8 x 8 blocks of 128 bytes, block (r/8, k/8) at (r/8 * K/8 + k/8).
// With lo = true the tile holds the BF16 rounding of w - bf16(w) instead.
void push_core(std::vector<uint16_t>& dst, const float* src, int ld, int rows, int cols, int R, int K,
               bool lo = false) {
    const size_t base = dst.size();
    dst.resize(base + (size_t)R * K, 0);
    for (int r = 0; r < R; ++r)
        for (int k = 0; k < K; ++k) {
            const float v = (r < rows && k < cols) ? src[(size_t)r * ld + k] : 0.f;
            const uint16_t h = to_bf16(v);
            dst[base + ((size_t)(r / 8) * (K / 8) + k / 8) * 64 + (r % 8) * 8 + (k % 8)] =
                lo ? to_bf16(v - from_bf16(h)) : h;
        }
}

// FP32 -> FP8 E4M3 (1 sign, 4 exponent bits with bias 7, 3 mantissa bits; no
// infinities, largest finite 448, subnormals down to 2^-9), round to nearest
// even, saturating at +-448.
uint8_t to_e4m3(float x) {
    const uint8_t sign = std::signbit(x) ? 0x80 : 0x00;
    const double a = std::fabs((double)x);
    if (!(a == a)) return 0x7F;
    if (a >= 448.0) return sign | 0x7E;
    int e = 0;
    (void)std::frexp(a, &e);  // a = f 2^e, f in [0.5, 1): the leading bit has weight 2^(e - 1)
    int ex = e - 1;           // unbiased exponent of a
    if (a == 0.0 || ex < -6) {  // subnormal range: multiples of 2^-9
        const double m = std::nearbyint(a * 512.0);  // default rounding: ties to even
        if (m >= 8.0) return sign | 0x08;            // rounds up to the smallest normal 2^-6
        return sign | (uint8_t)m;
    }
    double m = std::nearbyint((a / std::ldexp(1.0, ex) - 1.0) * 8.0);
    if (m >= 8.0) {
        m = 0.0;
        ++ex;
    }
    if (ex > 8 || (ex == 8 && m > 6.0)) return sign | 0x7E;
    return sign | (uint8_t)((ex + 7) << 3) | (uint8_t)m;
}

// Append an R x K FP8 E4M3 tile of src (row-major with leading dimension ld,
// entries beyond rows x cols zero), row r divided by scale[r], in the K-major
// core-matrix layout of 8-bit tcgen05.mma operands: 8 x 16 blocks of 128 bytes
// (8 rows of 16 bytes), block (r/8, k/16) at (r/8 * K/16 + k/16) * 128.
void push_core8(std::vector<uint8_t>& dst, const float* src, int ld, int rows, int cols, int R, int K,
                const float* scale) {
    const size_t base = dst.size();
    dst.resize(base + (size_t)R * K, 0);
    for (int r = 0; r < R; ++r)
        for (int k = 0; k < K; ++k) {
            const float v = (r < rows && k < cols) ? src[(size_t)r * ld + k] / scale[r] : 0.f;
            dst[base + ((size_t)(r / 8) * (K / 16) + k / 16) * 128 + (r % 8) * 16 + (k % 16)] = to_e4m3(v);
        }
}

// E4M3 scale of each of the `rows` rows of src (row-major, `cols` used of
// leading dimension ld): max |w| / 448 in FP32, so that each row's largest
// weight maps to the largest finite E4M3 value (1 for a zero row).  Exact
// per-row maxima keep the weight rounding markedly smaller than power-of-two
// scales do (measured: 5-10 x smaller energy error of the FP8 networks).
void fp8_row_scales(const float* src, int ld, int rows, int cols, float* out) {
    for (int r = 0; r < rows; ++r) {
        float m = 0.f;
        for (int k = 0; k < cols; ++k) m = std::max(m, std::fabs(src[(size_t)r * ld + k]));
        out[r] = m > 0.f ? m / 448.f : 1.f;
    }
}

// pad to a multiple of 4 floats so that float4 loads stay aligned
void push_block(std::vector<float>& dst, const float* src, size_t count) {
    dst.insert(dst.end(), src, src + count);
    while (dst.size() % 4) dst.push_back(0.f);
}

}  // namespace

// ===================================================================== ABI ==

extern "C" int reann_model_create_ex(int n_elem, int T, int n_phi, int l_max, int n_orb, int h1, int h2, double r_c,
                                     double alpha, int feature_pairs, const float* params, int64_t n_params,
                                     reann_model** out) {
    if (!out || !params || (feature_pairs != 0 && feature_pairs != 1)) return REANN_E_ARG;
    *out = nullptr;
    const bool pairs = feature_pairs == 1;
    if (n_elem < 1 || n_elem > MAX_ELEM || T < 1 || T > 8 || n_phi != NPHI || l_max != LMAX ||
        n_orb != (pairs ? NORB_P : NORB) || h1 != H1 || h2 != H2 || !(r_c > 0) || !(alpha > 0) ||
        !std::isfinite(r_c) || !std::isfinite(alpha) || alpha * r_c * r_c > 80.0)
        return REANN_E_ARG;
    if (n_params != expected_params(n_elem, T, pairs)) return REANN_E_ARG;
    for (int64_t i = 0; i < n_params; ++i)
        if (!std::isfinite(params[i])) return REANN_E_ARG;
    reann_model* m = new (std::nothrow) reann_model;
    if (!m) return REANN_E_NOMEM;
    m->m.n_elem = n_elem;
    m->m.T = T;
    m->m.r_c = r_c;
    m->m.alpha = alpha;
    m->m.pairs = pairs;
    m->m.params.assign(params, params + n_params);
    *out = m;
    return REANN_OK;
}

extern "C" int reann_model_create(int n_elem, int T, int n_phi, int l_max, int n_orb, int h1, int h2, double r_c,
                                  double alpha, const float* params, int64_t n_params, reann_model** out) {
    return reann_model_create_ex(n_elem, T, n_phi, l_max, n_orb, h1, h2, r_c, alpha, 0, params, n_params, out);
}

extern "C" void reann_model_free(reann_model* model) { delete model; }

extern "C" int reann_ctx_create(const reann_model* model, void* cuda_stream, reann_ctx** out) {
    if (!out || !model) return REANN_E_ARG;
    *out = nullptr;
    reann_ctx* ctx = new (std::nothrow) reann_ctx;
    if (!ctx) return REANN_E_NOMEM;
    ctx->model = model->m;
    ctx->stream = (cudaStream_t)cuda_stream;
    auto fail = [&](int code) {
        reann_ctx_free(ctx);
        return code;
    };
    if (cudaGetDevice(&ctx->device) != cudaSuccess) return fail(REANN_E_CUDA);
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    const Model& M = ctx->model;
    // radial constants (Sec. 2.1: Gaussian-type orbitals; centres linspace(0, r_c, N_phi))
    Radial& R = ctx->radial;
    auto split = [](double v, float& hi, float& lo) {
        hi = (float)v;
        lo = (float)(v - (double)hi);
    };
    R.rc = (float)M.r_c;
    R.rc2 = (float)(M.r_c * M.r_c);
    split(1.0 / M.r_c, R.inv_rc_hi, R.inv_rc_lo);
    split(M.alpha, R.alpha_hi, R.alpha_lo);
    const double delta = M.r_c / (NPHI - 1);
    split(2.0 * M.alpha * delta, R.tad_hi, R.tad_lo);
    for (int m = 0; m < NPHI; ++m) {
        split(m * delta, R.mu_hi[m], R.mu_lo[m]);
        split(std::exp(-M.alpha * delta * delta * (2 * m + 1)), R.kap_hi[m], R.kap_lo[m]);
    }
    // device image of the parameters: c0, W, then per (t, e) W1 b1 W2 b2 W3 b3 W1t W2t W3t
    std::vector<float> img;
    const float* p = M.params.data();
    std::vector<size_t> off_c0(1), off_W(1);
    off_c0[0] = img.size();
    push_block(img, p, (size_t)M.n_elem * NPHI);
    p += M.n_elem * NPHI;
    off_W[0] = img.size();
    const int KO = M.n_orb(), NF = M.n_feat();
    push_block(img, p, (size_t)M.T * (LMAX + 1) * NPHI * KO);
    p += M.T * (LMAX + 1) * NPHI * KO;
    struct Off {
        size_t W1 = 0, b1 = 0, W2 = 0, b2 = 0, W3 = 0, b3 = 0, W1t = 0, W2t = 0, W3t = 0, s8 = 0;
    };
    std::vector<Off> offs((size_t)M.T * M.n_elem);
    std::vector<uint16_t> tcimg;  // per (t, e): forward hi | forward lo | backward hi | backward lo, 16 KiB each
    std::vector<uint8_t> f8img;   // per (t, e): forward | backward FP8 images, kF8Img bytes
    for (int t = 0; t < M.T; ++t) {
        const int outd = (t == M.T - 1) ? 1 : NPHI;
        for (int e = 0; e < M.n_elem; ++e) {
            Off& o = offs[(size_t)t * M.n_elem + e];
            const float* W1 = p;
            const float* b1 = W1 + NF * H1;
            const float* W2 = b1 + H1;
            const float* b2 = W2 + H1 * H2;
            const float* W3 = b2 + H2;
            const float* b3 = W3 + H2 * outd;
            p = b3 + outd;
            o.W1 = img.size(); push_block(img, W1, NF * H1);
            o.b1 = img.size(); push_block(img, b1, H1);
            o.W2 = img.size(); push_block(img, W2, H1 * H2);
            o.b2 = img.size(); push_block(img, b2, H2);
            o.W3 = img.size(); push_block(img, W3, H2 * outd);
            o.b3 = img.size(); push_block(img, b3, outd);
            std::vector<float> tr;
            tr.resize(H1 * NF);
            for (int f = 0; f < NF; ++f)
                for (int q = 0; q < H1; ++q) tr[q * NF + f] = W1[f * H1 + q];
            o.W1t = img.size(); push_block(img, tr.data(), tr.size());
            tr.assign(H2 * H1, 0.f);
            for (int u = 0; u < H1; ++u)
                for (int q = 0; q < H2; ++q) tr[q * H1 + u] = W2[u * H2 + q];
            o.W2t = img.size(); push_block(img, tr.data(), tr.size());
            tr.assign(outd * H2, 0.f);
            for (int u = 0; u < H2; ++u)
                for (int q = 0; q < outd; ++q) tr[q * H2 + u] = W3[u * outd + q];
            o.W3t = img.size(); push_block(img, tr.data(), tr.size());
            // tensor-core B operands (N x K, K-major), for the 48-feature networks only
            if (M.pairs) continue;
            std::vector<float> w1t(H1 * NFEAT), w2t(H2 * H1);
            for (int f = 0; f < NFEAT; ++f)
                for (int q = 0; q < H1; ++q) w1t[q * NFEAT + f] = W1[f * H1 + q];
            for (int u = 0; u < H1; ++u)
                for (int q = 0; q < H2; ++q) w2t[q * H1 + u] = W2[u * H2 + q];
            for (int lo = 0; lo < 2; ++lo) {                                    // BF16 forward: hi, lo
                push_core(tcimg, w1t.data(), NFEAT, H1, NFEAT, H1, NFEAT, lo);  //   W1^T 64 x 48
                push_core(tcimg, w2t.data(), H1, H2, H1, H2, H1, lo);           //   W2^T 64 x 64
            }
            for (int lo = 0; lo < 2; ++lo) {                                    // BF16 backward: hi, lo
                push_core(tcimg, W2, H2, H1, H2, H1, H2, lo);                   //   W2   64 x 64
                push_core(tcimg, W1, H1, NFEAT, H1, NFEAT, H1, lo);             //   W1   48 x 64
            }
            // FP8 E4M3 images, one scale per B row (K a multiple of 32: 48 -> 64)
            float sc[kF8Scales];
            fp8_row_scales(w1t.data(), NFEAT, H1, NFEAT, sc);
            fp8_row_scales(w2t.data(), H1, H2, H1, sc + 64);
            fp8_row_scales(W2, H2, H1, H2, sc + 128);
            fp8_row_scales(W1, H1, NFEAT, H1, sc + 192);
            push_core8(f8img, w1t.data(), NFEAT, H1, NFEAT, H1, 64, sc);  // forward: W1^T (K padded to 64)
            push_core8(f8img, w2t.data(), H1, H2, H1, H2, H1, sc + 64);   //          W2^T
            push_core8(f8img, W2, H2, H1, H2, H1, H2, sc + 128);          // backward: W2
            push_core8(f8img, W1, H1, NFEAT, H1, NFEAT, H1, sc + 192);    //           W1
            o.s8 = img.size();
            push_block(img, sc, kF8Scales);
        }
    }
    if (tcimg.empty()) tcimg.resize(1);
    if (f8img.empty()) f8img.resize(16);
    if (cudaMalloc(&ctx->d_fp8, f8img.size()) != cudaSuccess) return fail(REANN_E_NOMEM);
    if (cudaMemcpy(ctx->d_fp8, f8img.data(), f8img.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(REANN_E_CUDA);
    if (cudaMalloc(&ctx->d_bf16, tcimg.size() * sizeof(uint16_t)) != cudaSuccess) return fail(REANN_E_NOMEM);
    if (cudaMemcpy(ctx->d_bf16, tcimg.data(), tcimg.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) !=
        cudaSuccess)
        return fail(REANN_E_CUDA);
    if (cudaMalloc(&ctx->d_params, img.size() * sizeof(float)) != cudaSuccess) return fail(REANN_E_NOMEM);
    if (cudaMemcpy(ctx->d_params, img.data(), img.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(REANN_E_CUDA);
    const float* base = ctx->d_params;
    ctx->d_c0 = base + off_c0[0];
    ctx->d_W = base + off_W[0];
    for (int t = 0; t < M.T; ++t)
        for (int e = 0; e < M.n_elem; ++e) {
            const Off& o = offs[(size_t)t * M.n_elem + e];
            ctx->nets.net[t][e] = NetDev{base + o.W1, base + o.b1, base + o.W2, base + o.b2, base + o.W3,
                                         base + o.b3, base + o.W1t, base + o.W2t, base + o.W3t};
            const uint8_t* ib =
                static_cast<const uint8_t*>(ctx->d_bf16) + (M.pairs ? 0 : ((size_t)t * M.n_elem + e) * 4 * kBfImg);
            const uint8_t* i8 =
                static_cast<const uint8_t*>(ctx->d_fp8) + (M.pairs ? 0 : ((size_t)t * M.n_elem + e) * kF8Img);
            TcImg& ti = ctx->tc.img[t][e];
            ti.wf = ib;
            ti.wb = ib + 2 * kBfImg;
            ti.wf8 = i8;
            ti.wb8 = i8 + kF8Fwd;
            ti.W1 = base + o.W1, ti.W2 = base + o.W2, ti.W3 = base + o.W3;
            ti.W1t = base + o.W1t, ti.W2t = base + o.W2t;
            ti.b1 = base + o.b1, ti.b2 = base + o.b2, ti.b3 = base + o.b3;
            ti.s8 = base + o.s8;
        }
    if (M.pairs && upload_pair_table() != cudaSuccess) return fail(REANN_E_CUDA);
    if (cudaMalloc(&ctx->d_flags, sizeof(int) * NFLAGS) != cudaSuccess) return fail(REANN_E_NOMEM);
    if (cudaMemset(ctx->d_flags, 0, sizeof(int) * NFLAGS) != cudaSuccess) return fail(REANN_E_CUDA);
    if (cudaMallocHost(&ctx->h_flags, sizeof(int) * NFLAGS) != cudaSuccess) return fail(REANN_E_NOMEM);
    *out = ctx;
    return REANN_OK;
}

extern "C" void reann_ctx_free(reann_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto& r : ctx->prof_recs) {
        cudaEventDestroy(r.second.first);
        cudaEventDestroy(r.second.second);
    }
    for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
    if (ctx->md_stream) {
        cudaStreamSynchronize(ctx->md_stream);
        cudaStreamDestroy(ctx->md_stream);
    }
    for (cudaEvent_t e : ctx->md_ev)
        if (e) cudaEventDestroy(e);
    if (ctx->d_params) cudaFree(ctx->d_params);
    if (ctx->d_bf16) cudaFree(ctx->d_bf16);
    if (ctx->d_fp8) cudaFree(ctx->d_fp8);
    if (ctx->d_flags) cudaFree(ctx->d_flags);
    if (ctx->h_flags) cudaFreeHost(ctx->h_flags);
    delete ctx;
}

extern "C" int reann_ctx_set_mlp_precision(reann_ctx* ctx, int precision) {
    if (!ctx) return REANN_E_ARG;
    if (precision != REANN_MLP_FP32 && precision != REANN_MLP_BF16 && precision != REANN_MLP_BF16X3 &&
        precision != REANN_MLP_FP8)
        return set_error(ctx, REANN_E_ARG, "unsupported network precision");
    if (precision != REANN_MLP_FP32 && ctx->model.pairs)
        return set_error(ctx, REANN_E_ARG, "tensor-core networks are built for the 48-feature models only");
    ctx->precision = precision;
    return REANN_OK;
}

extern "C" const char* reann_last_error(const reann_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

namespace {

// enqueue the read-back of the device flags and their reset on the context stream
int enqueue_flags_readback(reann_ctx* ctx) {
    REANN_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_flags, ctx->d_flags, sizeof(int) * NFLAGS, cudaMemcpyDeviceToHost,
                                        ctx->stream));
    REANN_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_flags, 0, sizeof(int) * NFLAGS, ctx->stream));
    return REANN_OK;
}

// the status the flags read back by enqueue_flags_readback report (after a synchronisation)
int flags_status(reann_ctx* ctx) {
    REANN_CUDA_TRY(ctx, cudaGetLastError());
    const int geom = ctx->h_flags[FLAG_GEOM], cap = ctx->h_flags[FLAG_NBR_OVERFLOW] | ctx->h_flags[FLAG_GHOST_OVERFLOW];
    const int timeout = ctx->h_flags[FLAG_TIMEOUT], drain = ctx->h_flags[FLAG_TIMEOUT_DRAIN];
    if (geom) return set_error(ctx, REANN_E_GEOM, "coincident or non-finite atoms in an evaluation");
    if (cap) return set_error(ctx, REANN_E_CAPACITY, "neighbour or ghost capacity exceeded");
    if (drain)
        return set_error(ctx, REANN_E_TIMEOUT,
                         "a bounded device wait ran out and the kernel's own tensor-core work or copy did not "
                         "complete either: results are invalid and the device state is suspect");
    if (timeout) return set_error(ctx, REANN_E_TIMEOUT, "a bounded device wait ran out (tensor-core network)");
    return REANN_OK;
}

}  // namespace

extern "C" int reann_ctx_wait_selftest(reann_ctx* ctx, int64_t polls) {
    if (!ctx) return REANN_E_ARG;
    if (polls < 1 || polls > (int64_t(1) << 26))
        return set_error(ctx, REANN_E_ARG, "polls must be in [1, 2^26]");
    REANN_CUDA_TRY(ctx, launch_wait_selftest(ctx->stream, ctx->d_flags, (long long)polls));
    return REANN_OK;
}

extern "C" int reann_ctx_check(reann_ctx* ctx) {
    if (!ctx) return REANN_E_ARG;
    if (int rc = enqueue_flags_readback(ctx)) return rc;
    REANN_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return flags_status(ctx);
}

namespace {

// neighbour list and ghost map only (no per-structure evaluation buffers)
int build_list(reann_ctx* ctx, int64_t n_atoms, const double* pos, const int32_t* species, const double* cell,
               double r_c, double skin, bool eval_buffers, reann_nlist** out, cudaMemPool_t mem_pool = nullptr) {
    if (!ctx || !out) return REANN_E_ARG;
    *out = nullptr;
    if (n_atoms < 1 || n_atoms > (int64_t)1 << 28 || !pos || !species || !cell || !(skin >= 0) || !std::isfinite(skin))
        return set_error(ctx, REANN_E_ARG, "bad argument to reann_build_nlist");
    if (r_c != ctx->model.r_c) return set_error(ctx, REANN_E_MISMATCH, "r_c differs from the model cutoff");
    reann_nlist* nl = new (std::nothrow) reann_nlist;
    if (!nl) return set_error(ctx, REANN_E_NOMEM, "host allocation failed");
    nl->n = n_atoms;
    nl->n_elem = ctx->model.n_elem;
    nl->T = ctx->model.T;
    nl->r_c = r_c;
    nl->skin = skin;
    nl->mem_pool = mem_pool;
    nl->alloc_stream = ctx->stream;
    int rc = make_geometry(ctx, cell, r_c + skin, &nl->geom);
    if (!rc) rc = build_nlist_device(ctx, nl, pos, species);
    if (!rc && eval_buffers) rc = alloc_eval_buffers(ctx, nl);
    if (rc) {
        cudaStreamSynchronize(ctx->stream);
        free_nlist(nl);
        return rc;
    }
    *out = nl;
    return REANN_OK;
}

}  // namespace

extern "C" int reann_build_nlist(reann_ctx* ctx, int64_t n_atoms, const double* pos, const int32_t* species,
                                 const double* cell, double r_c, double skin, reann_nlist** out) {
    return build_list(ctx, n_atoms, pos, species, cell, r_c, skin, true, out);
}

// ------------------------------------------------ spatial decomposition ---
// Virtual ranks on one device (Sec. 2.2, Figs. 3-5).  The single-domain list is
// built first and read back; every atom is assigned to the subdomain of its
// wrapped fractional coordinates; atoms are re-ordered rank-major (element-
// major inside a rank, the spatial order kept); every neighbour entry that is
// not a zero-shift atom of the same rank becomes a ghost slot of that rank,
// one slot per distinct (owner, image shift) in order of first use.  The rows
// keep their entries' order, and a ghost slot receives bit-identical copies of
// its owner's position, coefficients and bbar, so each atom's arithmetic is
// the single-domain arithmetic.
namespace {

constexpr int32_t kZeroShift = 128 | (128 << 8) | (128 << 16);

int build_decomposed(reann_ctx* ctx, reann_nlist* src, const int32_t ranks[3], reann_nlist** out) {
    cudaStream_t s = ctx->stream;
    const int64_t n = src->n;
    const int stride = src->stride;
    int32_t G = 0;
    std::vector<int32_t> nbr((size_t)n * stride), cnt(n), perm(n), spc(n), wm(3 * n);
    std::vector<double> fw(3 * n), pref(3 * n);
    REANN_CUDA_TRY(ctx, cudaMemcpyAsync(&G, src->w.goff + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    REANN_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    std::vector<int32_t> own(std::max<int32_t>(G, 1)), sh(std::max<int32_t>(G, 1));
    REANN_CUDA_TRY(ctx, cudaMemcpyAsync(nbr.data(), src->nbr, sizeof(int32_t) * nbr.size(), cudaMemcpyDeviceToHost, s));
    REANN_CUDA_TRY(ctx, cudaMemcpyAsync(cnt.data(), src->nbr_cnt, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    REANN_CUDA_TRY(ctx, cudaMemcpyAsync(perm.data(), src->perm, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    REANN_CUDA_TRY(ctx, cudaMemcpyAsync(spc.data(), src->species, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    REANN_CUDA_TRY(ctx, cudaMemcpyAsync(wm.data(), src->wrapm, sizeof(int32_t) * 3 * n, cudaMemcpyDeviceToHost, s));
    REANN_CUDA_TRY(ctx, cudaMemcpyAsync(fw.data(), src->w.fw, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
    REANN_CUDA_TRY(ctx, cudaMemcpyAsync(pref.data(), src->pos_ref, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
    if (G > 0) {
        REANN_CUDA_TRY(ctx, cudaMemcpyAsync(own.data(), src->g_owner, sizeof(int32_t) * G, cudaMemcpyDeviceToHost, s));
        REANN_CUDA_TRY(ctx, cudaMemcpyAsync(sh.data(), src->g_shift, sizeof(int32_t) * G, cudaMemcpyDeviceToHost, s));
    }
    REANN_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    // subdomain of every atom (internal order)
    const int K = ranks[0] * ranks[1] * ranks[2];
    std::vector<int32_t> rank(n);
    for (int64_t i = 0; i < n; ++i) {
        int b[3];
        for (int k = 0; k < 3; ++k)
            b[k] = std::min(ranks[k] - 1, std::max(0, (int)std::floor(fw[3 * i + k] * ranks[k])));
        rank[i] = (b[0] * ranks[1] + b[1]) * ranks[2] + b[2];
    }
    // rank-major, then element-major; the existing (spatially sorted) order inside
    std::vector<int64_t> order(n), newidx(n);
    std::iota(order.begin(), order.end(), (int64_t)0);
    const int ne = src->n_elem;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        return (int64_t)rank[a] * ne + spc[a] < (int64_t)rank[b] * ne + spc[b];
    });
    for (int64_t p = 0; p < n; ++p) newidx[order[p]] = p;
    // ghost slots per rank and remapped rows (ghost entries first as -(local id + 1))
    std::vector<std::unordered_map<int64_t, int32_t>> gmap(K);
    std::vector<std::vector<int32_t>> gown(K), gsh(K);
    std::vector<int32_t> row_new((size_t)n * stride, 0), cnt_new(n);
    for (int64_t p = 0; p < n; ++p) {
        const int64_t i = order[p];
        const int r = rank[i];
        cnt_new[p] = cnt[i];
        for (int e = 0; e < cnt[i]; ++e) {
            const int64_t sl = nbr[(size_t)i * stride + e];
            int64_t o = sl;
            int32_t shift = kZeroShift;
            if (sl >= n) {
                o = own[sl - n];
                shift = sh[sl - n];
            }
            int32_t entry;
            if (shift == kZeroShift && rank[o] == r) {
                entry = (int32_t)newidx[o];
            } else {
                const int64_t key = (o << 24) | (int64_t)(shift & 0xFFFFFF);
                auto it = gmap[r].find(key);
                int32_t id;
                if (it == gmap[r].end()) {
                    id = (int32_t)gown[r].size();
                    gmap[r].emplace(key, id);
                    gown[r].push_back((int32_t)newidx[o]);
                    gsh[r].push_back(shift);
                } else {
                    id = it->second;
                }
                entry = -(id + 1);
            }
            row_new[(size_t)p * stride + e] = entry;
        }
    }
    std::vector<int64_t> gbase(K + 1, 0);
    for (int r = 0; r < K; ++r) gbase[r + 1] = gbase[r] + (int64_t)gown[r].size();
    const int64_t Gt = gbase[K];
    if (n + Gt > ((int64_t)1 << 31) - 1) return set_error(ctx, REANN_E_CAPACITY, "decomposed list too large");
    for (int64_t p = 0; p < n; ++p) {
        const int r = rank[order[p]];
        for (int e = 0; e < cnt_new[p]; ++e) {
            int32_t& v = row_new[(size_t)p * stride + e];
            if (v < 0) v = (int32_t)(n + gbase[r] + (-v - 1));
        }
    }
    std::vector<int32_t> g_own(std::max<int64_t>(Gt, 1)), g_sh(std::max<int64_t>(Gt, 1));
    for (int r = 0; r < K; ++r)
        for (size_t q = 0; q < gown[r].size(); ++q) {
            g_own[gbase[r] + q] = gown[r][q];
            g_sh[gbase[r] + q] = gsh[r][q];
        }
    std::vector<int32_t> perm_new(n), spc_new(n), wm_new(3 * n), goff(n + 1, 0);
    for (int64_t p = 0; p < n; ++p) {
        const int64_t i = order[p];
        perm_new[p] = perm[i];
        spc_new[p] = spc[i];
        for (int k = 0; k < 3; ++k) wm_new[3 * p + k] = wm[3 * i + k];
    }
    goff[n] = (int32_t)Gt;
    // tiles: one run per (rank, element)
    std::vector<std::array<int, 3>> ranges;
    for (int64_t p = 0; p < n;) {
        int64_t q = p;
        while (q < n && rank[order[q]] == rank[order[p]] && spc_new[q] == spc_new[p]) ++q;
        ranges.push_back({spc_new[p], (int)p, (int)q});
        p = q;
    }
    // the new list
    reann_nlist* nl = new (std::nothrow) reann_nlist;
    if (!nl) return set_error(ctx, REANN_E_NOMEM, "host allocation failed");
    nl->n = n;
    nl->g = nl->g_cap = Gt;
    nl->stride = stride;
    nl->max_count = src->max_count;
    nl->n_elem = ne;
    nl->T = src->T;
    nl->r_c = src->r_c;
    nl->skin = src->skin;
    nl->geom = src->geom;
    for (int e = 0; e <= MAX_ELEM; ++e) nl->elem_start[e] = 0;
    nl->decomposed = true;
    for (int k = 0; k < 3; ++k) nl->rank_grid[k] = ranks[k];
    nl->rank_local.assign(K, 0);
    nl->rank_ghost.assign(K, 0);
    nl->rank_remote.assign(K, 0);
    for (int64_t i = 0; i < n; ++i) nl->rank_local[rank[i]]++;
    for (int r = 0; r < K; ++r) {
        nl->rank_ghost[r] = (int64_t)gown[r].size();
        for (int32_t o : gown[r]) nl->rank_remote[r] += rank[order[o]] != r;
    }
    auto fail = [&](int code, const char* msg) {
        cudaStreamSynchronize(s);
        free_nlist(nl);
        return set_error(ctx, code, msg);
    };
    nl->perm = nl_alloc<int32_t>(nl, n);
    nl->species = nl_alloc<int32_t>(nl, n);
    nl->wrapm = nl_alloc<int32_t>(nl, 3 * n);
    nl->g_owner = nl_alloc<int32_t>(nl, std::max<int64_t>(Gt, 1));
    nl->g_shift = nl_alloc<int32_t>(nl, std::max<int64_t>(Gt, 1));
    nl->nbr = nl_alloc<int32_t>(nl, (size_t)n * stride);
    nl->nbr_cnt = nl_alloc<int32_t>(nl, n);
    nl->w.goff = nl_alloc<int32_t>(nl, n + 1);
    nl->pos_ref = nl_alloc<double>(nl, 3 * n);
    if (!nl->perm || !nl->species || !nl->wrapm || !nl->g_owner || !nl->g_shift || !nl->nbr || !nl->nbr_cnt ||
        !nl->w.goff || !nl->pos_ref)
        return fail(REANN_E_NOMEM, "decomposed list: out of device memory");
    bool ok = cudaMemcpyAsync(nl->perm, perm_new.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(nl->species, spc_new.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(nl->wrapm, wm_new.data(), sizeof(int32_t) * 3 * n, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(nl->g_owner, g_own.data(), sizeof(int32_t) * g_own.size(), cudaMemcpyHostToDevice, s) ==
                  cudaSuccess &&
              cudaMemcpyAsync(nl->g_shift, g_sh.data(), sizeof(int32_t) * g_sh.size(), cudaMemcpyHostToDevice, s) ==
                  cudaSuccess &&
              cudaMemcpyAsync(nl->nbr, row_new.data(), sizeof(int32_t) * row_new.size(), cudaMemcpyHostToDevice, s) ==
                  cudaSuccess &&
              cudaMemcpyAsync(nl->nbr_cnt, cnt_new.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(nl->w.goff, goff.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, s) ==
                  cudaSuccess &&
              cudaMemcpyAsync(nl->pos_ref, pref.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s) == cudaSuccess;
    if (!ok) return fail(REANN_E_CUDA, "decomposed list: upload failed");
    if (int rc = alloc_eval_buffers(ctx, nl, &ranges)) {
        cudaStreamSynchronize(s);
        free_nlist(nl);
        return rc;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(REANN_E_CUDA, "decomposed list: upload failed");
    *out = nl;
    return REANN_OK;
}

}  // namespace

extern "C" int reann_build_nlist_decomposed(reann_ctx* ctx, int64_t n_atoms, const double* pos, const int32_t* species,
                                            const double* cell, double r_c, double skin, const int32_t ranks[3],
                                            reann_nlist** out) {
    if (!ctx || !out || !ranks) return set_error(ctx, REANN_E_ARG, "null argument");
    *out = nullptr;
    for (int k = 0; k < 3; ++k)
        if (ranks[k] < 1 || ranks[k] > 64) return set_error(ctx, REANN_E_ARG, "ranks per axis must be in 1..64");
    reann_nlist* src = nullptr;
    int rc = build_list(ctx, n_atoms, pos, species, cell, r_c, skin, false, &src);
    if (rc) return rc;
    rc = build_decomposed(ctx, src, ranks, out);
    cudaStreamSynchronize(ctx->stream);
    free_nlist(src);
    return rc;
}

extern "C" int reann_decomp_info(const reann_nlist* nl, int32_t* n_ranks, int64_t* local, int64_t* ghosts,
                                 int64_t* remote) {
    if (!nl) return REANN_E_ARG;
    const int K = nl->decomposed ? (int)nl->rank_local.size() : 1;
    if (n_ranks) *n_ranks = K;
    for (int r = 0; r < K; ++r) {
        if (local) local[r] = nl->decomposed ? nl->rank_local[r] : nl->n;
        if (ghosts) ghosts[r] = nl->decomposed ? nl->rank_ghost[r] : nl->g;
        if (remote) remote[r] = nl->decomposed ? nl->rank_remote[r] : 0;
    }
    return REANN_OK;
}

extern "C" void reann_nlist_free(reann_nlist* nl) { free_nlist(nl); }

extern "C" int reann_nlist_info(const reann_nlist* nl, int64_t* n_atoms, int64_t* n_ghosts, int64_t* n_pairs,
                                int64_t* n_live) {
    if (!nl) return REANN_E_ARG;
    if (n_atoms) *n_atoms = nl->n;
    if (n_ghosts) {
        int32_t g = 0;
        if (cudaMemcpy(&g, ghost_count_ptr(nl), sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
            return REANN_E_CUDA;
        *n_ghosts = std::min<int64_t>(g, nl->g_cap);
    }
    auto sum_counts = [&](const int32_t* d, int64_t* out) {
        std::vector<int32_t> cnt(nl->n);
        if (cudaMemcpy(cnt.data(), d, sizeof(int32_t) * nl->n, cudaMemcpyDeviceToHost) != cudaSuccess)
            return REANN_E_CUDA;
        int64_t s = 0;
        for (int32_t c : cnt) s += c;
        *out = s;
        return REANN_OK;
    };
    if (n_pairs && sum_counts(nl->nbr_cnt, n_pairs)) return REANN_E_CUDA;
    if (n_live && sum_counts(nl->live_cnt, n_live)) return REANN_E_CUDA;
    return REANN_OK;
}

extern "C" int reann_nlist_export(reann_ctx* ctx, const reann_nlist* nl, int64_t cap, int32_t* i, int32_t* j,
                                  int32_t* n, int64_t* count) {
    if (!ctx || !nl || !count || cap < 0 || (cap > 0 && (!i || !j || !n))) return REANN_E_ARG;
    return export_nlist(ctx, nl, cap, i, j, n, count);
}

namespace {

// ---- optional per-region event profile -----------------------------------
cudaEvent_t prof_event(reann_ctx* ctx) {
    if (!ctx->prof_pool.empty()) {
        cudaEvent_t e = ctx->prof_pool.back();
        ctx->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct ProfScope {
    reann_ctx* ctx;
    int region;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(reann_ctx* c, int r) : ctx(c), region(r) {
        if (!ctx->prof_on) return;
        a = prof_event(ctx);
        b = prof_event(ctx);
        cudaEventRecord(a, ctx->stream);
    }
    ~ProfScope() {
        if (!ctx->prof_on || !a) return;
        cudaEventRecord(b, ctx->stream);
        ctx->prof_recs.push_back({region, {a, b}});
    }
};

// harvest recorded event pairs into the per-region totals (synchronous)
void prof_collect(reann_ctx* ctx) {
    if (ctx->prof_recs.empty()) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto& r : ctx->prof_recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.second.first, r.second.second) == cudaSuccess) {
            ctx->prof_ms[r.first] += ms;
            ctx->prof_n[r.first] += 1;
        }
        ctx->prof_pool.push_back(r.second.first);
        ctx->prof_pool.push_back(r.second.second);
    }
    ctx->prof_recs.clear();
}

const char* kRegionNames[PR_COUNT] = {"nlist_rebuild", "refresh_positions", "live_edges",   "init_coef",
                                      "ghost_gather",  "density_fwd",       "mlp_fwd",      "energy_sum",
                                      "mlp_bwd",       "bbar",              "density_adj",  "scatter_outputs"};

// pos == nullptr: positions already in place (serving pool); seg != nullptr: one FP64
// energy per segment (structure) into energy[seg.z] instead of one total;
// virial != nullptr: the 3 x 3 FP64 virial (and, with atom_virial, the per-atom
// virials in caller order); the buffers must have been sized (ensure_virial).
int run_energy_forces(reann_ctx* ctx, reann_nlist* nl, const double* pos, int T, double* energy, float* forces,
                      float* atom_energy, const int4* seg = nullptr, int nseg = 0, double* virial = nullptr,
                      float* atom_virial = nullptr) {
    cudaStream_t s = ctx->stream;
    const int64_t n = nl->n, ne = nl->n + nl->g_cap;
    float* vir = virial ? nl->vir : nullptr;
    if (pos) {
        ProfScope p(ctx, PR_REFRESH);  // positions and the first layer's coefficients
        REANN_CUDA_TRY(ctx, launch_refresh_positions(s, nl, pos, ctx->d_c0));
    } else {
        ProfScope p(ctx, PR_INIT);
        REANN_CUDA_TRY(ctx, launch_init_coef(s, nl, ctx->d_c0));
    }
    {
        ProfScope p(ctx, PR_LIVE);
        REANN_CUDA_TRY(ctx, launch_live_edges(s, nl, ctx->radial.rc2, ctx->d_flags));
    }
    const bool pairs = ctx->model.pairs;
    const size_t lw = (size_t)(LMAX + 1) * NPHI * ctx->model.n_orb();
    const int64_t nf = nl->n_feat;
    // single-domain lists: owners write their ghost rows (no gather launches); otherwise gather
    const GhostOut gh = nl->ghosts_by_owner ? GhostOut{nl->w.goff, n, nl->g_cap} : GhostOut{};
    // forward: Eq. 1 then Eq. 2, re-using the same list in every layer (Sec. 2.2)
    for (int t = 0; t < T; ++t) {
        float* coef_t = nl->coef + (size_t)t * ne * NPHI;
        float* rho_t = nl->rho + (size_t)t * n * nf;
        float* bck_t = nl->bck + (size_t)t * n * NB;
        if (t > 0 && !gh.goff) {
            ProfScope p(ctx, PR_GATHER);  // ghost slots receive their owners' coefficients (Fig. 4a)
            REANN_CUDA_TRY(ctx, launch_gather_ghost_rows(s, nl, coef_t, NPHI));
        }
        {
            ProfScope p(ctx, PR_DENSITY_FWD);
            REANN_CUDA_TRY(ctx, launch_density_fwd(s, nl, ctx->radial, ctx->d_W + t * lw, coef_t, rho_t, bck_t, pairs));
        }
        ProfScope p(ctx, PR_MLP_FWD);
        const bool energy_net = t == T - 1;
        // the FP32 energy network also sums the tiles' energies (unless per-structure sums are wanted)
        double* epart = energy_net && !seg ? nl->partial : nullptr;
        float* out = energy_net ? nl->eps : nl->coef + (size_t)(t + 1) * ne * NPHI;
        const int out_stride = energy_net ? 1 : NPHI;
        if (ctx->precision != REANN_MLP_FP32)
            REANN_CUDA_TRY(ctx, launch_mlp_fwd_tc(s, nl, ctx->tc, t, energy_net, ctx->precision, rho_t, out,
                                                  out_stride, ctx->d_flags, gh,
                                                  nl->dsave + (size_t)t * n * (H1 + H2), epart));
        else
            REANN_CUDA_TRY(ctx, launch_mlp_fwd_f32(s, nl, ctx->nets, t, energy_net, rho_t, out, out_stride, pairs, gh,
                                                  nl->dsave + (size_t)t * n * (H1 + H2), epart, ctx->d_flags));
    }
    {
        ProfScope p(ctx, PR_ENERGY);
        if (seg)
            REANN_CUDA_TRY(ctx, launch_segment_energy(s, seg, nseg, nl->eps, energy));
        else  // the energy network summed its tiles (64-row FP32 tiles or 128-row tensor-core tiles)
            REANN_CUDA_TRY(ctx, launch_energy_final(s, nl->partial,
                                                    (int)(ctx->precision == REANN_MLP_FP32 ? tiles_of(nl)
                                                                                           : tiles128_of(nl)),
                                                    energy));
    }
    // reverse: Eqs. 3-5, one vector-Jacobian product per layer
    for (int t = T - 1; t >= 0; --t) {
        const float* coef_t = nl->coef + (size_t)t * ne * NPHI;
        const float* bck_t = nl->bck + (size_t)t * n * NB;
        const float* dsave_t = nl->dsave + (size_t)t * n * (H1 + H2);
        {
            ProfScope p(ctx, PR_MLP_BWD);
            if (ctx->precision != REANN_MLP_FP32)  // the tensor-core backward networks also take the bbar step
                REANN_CUDA_TRY(ctx, launch_mlp_bwd_tc(s, nl, ctx->tc, t, t == T - 1, ctx->precision, dsave_t,
                                                      nl->cbar, ctx->d_W + t * lw, bck_t, coef_t, nl->bbar, gh,
                                                      ctx->d_flags));
            else if (!pairs)  // the FP32 backward networks also take the bbar step (fused)
                REANN_CUDA_TRY(ctx, launch_mlp_bwd_f32(s, nl, ctx->nets, t, t == T - 1, dsave_t, nl->cbar,
                                                       nl->rhobar, ctx->d_flags, false, ctx->d_W + t * lw, bck_t,
                                                       coef_t, nl->bbar, gh));
            else
                REANN_CUDA_TRY(ctx, launch_mlp_bwd_f32(s, nl, ctx->nets, t, t == T - 1, dsave_t, nl->cbar,
                                                       nl->rhobar, ctx->d_flags, true));
        }
        if (pairs) {
            ProfScope p(ctx, PR_BBAR);
            REANN_CUDA_TRY(ctx, launch_bbar(s, nl, ctx->d_W + t * lw, bck_t, nl->rhobar, coef_t, nl->bbar, pairs, gh));
        }
        if (!gh.goff) {
            ProfScope p(ctx, PR_GATHER);  // ghost slots receive their owners' adjoints (vector-Jacobian product)
            REANN_CUDA_TRY(ctx, launch_gather_ghost_rows(s, nl, nl->bbar, NREC));
        }
        ProfScope p(ctx, PR_DENSITY_ADJ);
        REANN_CUDA_TRY(ctx, launch_density_adj(s, nl, ctx->radial, nl->bbar, nl->cbar, nl->grad, t >= 1,
                                               ctx->d_flags, vir, t == 0 ? forces : nullptr,
                                               t == 0 ? atom_energy : nullptr, t == T - 1));
    }
    ProfScope p(ctx, PR_OUTPUT);
    if (vir) {
        REANN_CUDA_TRY(ctx, launch_virial_sum(s, nl, vir, nl->vir_partial, virial));
        if (atom_virial) REANN_CUDA_TRY(ctx, launch_unpermute_rows(s, nl, vir, 9, atom_virial, 9));
    }
    return REANN_OK;
}

int ensure_virial(reann_ctx* ctx, reann_nlist* nl) {
    if (nl->vir) return REANN_OK;
    nl->vir = nl_alloc<float>(nl, (size_t)nl->n * 9);
    nl->vir_partial = nl_alloc<double>(nl, (size_t)9 * ((nl->n + 2047) / 2048 + 1));
    if (!nl->vir || !nl->vir_partial) return set_error(ctx, REANN_E_NOMEM, "virial buffers: out of device memory");
    return REANN_OK;
}

int run_rebuild(reann_ctx* ctx, reann_nlist* nl, const double* pos) {
    if (nl->decomposed)
        return set_error(ctx, REANN_E_ARG, "a decomposed list is not rebuilt in place: build it anew");
    ProfScope p(ctx, PR_REBUILD);
    REANN_CUDA_TRY(ctx, launch_rebuild(ctx->stream, nl, pos, ctx->d_flags, nullptr));
    return REANN_OK;
}

// Runs fn() on the context's own non-blocking stream (created on first use),
// ordered after the work already on the caller's stream and before any work
// the caller enqueues later; CUDA graphs are captured and replayed there.
template <class F>
int on_graph_stream(reann_ctx* ctx, F fn) {
    if (!ctx->md_stream) {
        REANN_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->md_stream, cudaStreamNonBlocking));
        REANN_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->md_ev[0], cudaEventDisableTiming));
        REANN_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->md_ev[1], cudaEventDisableTiming));
    }
    cudaStream_t user = ctx->stream;
    REANN_CUDA_TRY(ctx, cudaEventRecord(ctx->md_ev[0], user));
    REANN_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->md_stream, ctx->md_ev[0], 0));
    ctx->stream = ctx->md_stream;
    const int rc = fn();
    ctx->stream = user;
    REANN_CUDA_TRY(ctx, cudaEventRecord(ctx->md_ev[1], ctx->md_stream));
    REANN_CUDA_TRY(ctx, cudaStreamWaitEvent(user, ctx->md_ev[1], 0));
    return rc;
}

// Runs body(), which only enqueues work on ctx->stream whose launch sequence
// is fixed by the list, the context and the key.  The first call with a key
// runs directly (one-time set-up happens there); the second captures it into
// a CUDA graph; later calls replay the graph.  With per-region profiling on,
// every call runs directly.
template <class F>
int run_graphed(reann_ctx* ctx, reann_nlist* nl, GraphSlotId slot, const void* const key[6], const int ikey[4],
                F body) {
    if (ctx->prof_on) return body();
    GraphSlot& gs = nl->graphs[slot];
    const bool same = gs.seen && std::memcmp(gs.key, key, sizeof(gs.key)) == 0 &&
                      std::memcmp(gs.ikey, ikey, sizeof(gs.ikey)) == 0;
    if (!same) {
        if (gs.exec) cudaGraphExecDestroy(gs.exec);
        if (gs.graph) cudaGraphDestroy(gs.graph);
        gs = GraphSlot{};
        std::memcpy(gs.key, key, sizeof(gs.key));
        std::memcpy(gs.ikey, ikey, sizeof(gs.ikey));
        gs.seen = true;
        return body();
    }
    if (gs.nograph) return body();
    return on_graph_stream(ctx, [&]() -> int {
        cudaStream_t s = ctx->stream;
        if (!gs.exec) {
            REANN_CUDA_TRY(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            const int rc = body();
            cudaGraph_t g = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(s, &g);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (ec != cudaSuccess || cudaGraphInstantiate(&gs.exec, g, 0) != cudaSuccess) {
                // not capturable: run directly from now on
                if (g) cudaGraphDestroy(g);
                gs.exec = nullptr;
                gs.nograph = true;
                (void)cudaGetLastError();
                return body();
            }
            gs.graph = g;
        }
        REANN_CUDA_TRY(ctx, cudaGraphLaunch(gs.exec, s));
        return REANN_OK;
    });
}

int graphed_rebuild(reann_ctx* ctx, reann_nlist* nl, const double* pos, GraphSlotId slot) {
    if (nl->decomposed) return run_rebuild(ctx, nl, pos);  // refused, with its message
    const void* key[6] = {pos, nullptr, nullptr, nullptr, nullptr, nullptr};
    const int ikey[4] = {0, 0, 0, 0};
    return run_graphed(ctx, nl, slot, key, ikey, [&] { return run_rebuild(ctx, nl, pos); });
}

int graphed_eval(reann_ctx* ctx, reann_nlist* nl, const double* pos, int T, double* energy, float* forces,
                 float* atom_energy, double* virial, float* atom_virial, GraphSlotId slot) {
    const void* key[6] = {pos, energy, forces, atom_energy, virial, atom_virial};
    const int ikey[4] = {T, ctx->precision, 0, 0};
    return run_graphed(ctx, nl, slot, key, ikey, [&] {
        return run_energy_forces(ctx, nl, pos, T, energy, forces, atom_energy, nullptr, 0, virial, atom_virial);
    });
}

}  // namespace

extern "C" int reann_nlist_rebuild(reann_ctx* ctx, reann_nlist* nl, const double* pos) {
    if (!ctx || !nl || !pos) return set_error(ctx, REANN_E_ARG, "null argument");
    return graphed_rebuild(ctx, nl, pos, GS_REBUILD);
}

extern "C" int reann_energy_forces(reann_ctx* ctx, reann_nlist* nl, const double* pos, int T, double* energy,
                                   float* forces, float* atom_energy) {
    if (!ctx || !nl || !pos || !energy || !forces) return set_error(ctx, REANN_E_ARG, "null argument");
    if (T != ctx->model.T || T != nl->T) return set_error(ctx, REANN_E_MISMATCH, "T differs from the model");
    return graphed_eval(ctx, nl, pos, T, energy, forces, atom_energy, nullptr, nullptr, GS_EVAL);
}

extern "C" int reann_energy_forces_virial(reann_ctx* ctx, reann_nlist* nl, const double* pos, int T, double* energy,
                                          float* forces, float* atom_energy, double* virial, float* atom_virial) {
    if (!ctx || !nl || !pos || !energy || !forces || !virial) return set_error(ctx, REANN_E_ARG, "null argument");
    if (T != ctx->model.T || T != nl->T) return set_error(ctx, REANN_E_MISMATCH, "T differs from the model");
    if (int rc = ensure_virial(ctx, nl)) return rc;
    return graphed_eval(ctx, nl, pos, T, energy, forces, atom_energy, virial, atom_virial, GS_EVAL);
}

extern "C" int reann_energy_forces_host(reann_ctx* ctx, reann_nlist* nl, const double* pos, int T, double* energy,
                                        float* forces, int rebuild) {
    if (!ctx || !nl || !pos || !energy || !forces) return set_error(ctx, REANN_E_ARG, "null argument");
    if (T != ctx->model.T || T != nl->T) return set_error(ctx, REANN_E_MISMATCH, "T differs from the model");
    cudaStream_t s = ctx->stream;
    const int64_t n = nl->n;
    if (!nl->h2d_pos) {
        nl->h2d_pos = nl_alloc<double>(nl, 3 * n);
        nl->d_forces = nl_alloc<float>(nl, 3 * n);
        nl->d_energy = nl_alloc<double>(nl, 1);
        if (!nl->h2d_pos || !nl->d_forces || !nl->d_energy) return set_error(ctx, REANN_E_NOMEM, "staging buffers");
    }
    REANN_CUDA_TRY(ctx, cudaMemcpyAsync(nl->h2d_pos, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
    if (rebuild) {
        int rc = graphed_rebuild(ctx, nl, nl->h2d_pos, GS_HOST_REBUILD);
        if (rc) return rc;
    } else {
        REANN_CUDA_TRY(ctx, launch_moved(s, nl, nl->h2d_pos, ctx->d_flags + FLAG_MOVED));
        REANN_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_flags, ctx->d_flags, sizeof(int) * NFLAGS, cudaMemcpyDeviceToHost, s));
        REANN_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        if (ctx->h_flags[FLAG_MOVED]) {
            int zero = 0;
            REANN_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->d_flags + FLAG_MOVED, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
            int rc = run_rebuild(ctx, nl, nl->h2d_pos);
            if (rc) return rc;
        }
    }
    int rc = graphed_eval(ctx, nl, nl->h2d_pos, T, nl->d_energy, nl->d_forces, nullptr, nullptr, nullptr, GS_HOST_EVAL);
    if (rc) return rc;
    REANN_CUDA_TRY(ctx, cudaMemcpyAsync(forces, nl->d_forces, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, s));
    REANN_CUDA_TRY(ctx, cudaMemcpyAsync(energy, nl->d_energy, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (int rc2 = enqueue_flags_readback(ctx)) return rc2;  // the flags come back with the results:
    REANN_CUDA_TRY(ctx, cudaStreamSynchronize(s));           // one synchronisation per call
    return flags_status(ctx);
}

namespace {

// enqueue one velocity-Verlet step on ctx->stream (captured into the step graph)
// Nose-Hoover parameters: kT (eV), Q = g kT tau^2, g = 3N - 3; tau = 0: NVE
struct Thermo {
    double kt = 0.0, tau = 0.0, gkt = 0.0, q = 0.0;
    bool on() const { return tau > 0.0; }
};

Thermo make_thermo(int64_t n, double temperature_k, double tau_fs) {
    Thermo th;
    if (tau_fs > 0.0) {
        th.kt = 8.617333262e-5 * temperature_k;
        th.tau = tau_fs;
        th.gkt = (double)(3 * n - 3) * th.kt;
        th.q = th.gkt * tau_fs * tau_fs;
    }
    return th;
}

int md_step_body(reann_ctx* ctx, reann_nlist* nl, double* pos, double* vel, const double* mass, double dt,
                 int n_steps, double* e_pot, double* e_kin, const Thermo& th, double* e_bath) {
    cudaStream_t s = ctx->stream;
    const int64_t n = nl->n;
    int* gate = nl->md_ints;
    double* sc = nl->md_scalars;
    if (th.on()) REANN_CUDA_TRY(ctx, launch_nh_half(s, sc, dt, th.gkt, th.q));
    REANN_CUDA_TRY(ctx, launch_kick(s, n, vel, nl->md_forces, mass, 0.5 * dt, th.on() ? sc + 4 : nullptr));
    REANN_CUDA_TRY(ctx, launch_drift(s, n, pos, vel, dt));
    REANN_CUDA_TRY(ctx, cudaMemsetAsync(gate, 0, sizeof(int), s));
    REANN_CUDA_TRY(ctx, launch_moved(s, nl, pos, gate));
    REANN_CUDA_TRY(ctx, launch_rebuild(s, nl, pos, ctx->d_flags, gate));  // kernels return at once unless gate != 0
    int rc = run_energy_forces(ctx, nl, pos, nl->T, nl->md_scalars, nl->md_forces, nullptr);
    if (rc) return rc;
    REANN_CUDA_TRY(ctx, launch_kick(s, n, vel, nl->md_forces, mass, 0.5 * dt));
    REANN_CUDA_TRY(ctx, launch_ekin(s, n, vel, mass, nl->md_partial, sc + 1));
    if (th.on()) {
        REANN_CUDA_TRY(ctx, launch_nh_half(s, sc, dt, th.gkt, th.q));
        REANN_CUDA_TRY(ctx, launch_scale(s, n, vel, sc + 4));
    }
    REANN_CUDA_TRY(ctx, launch_record(s, nl->md_ints + 1, sc, e_pot, e_kin, e_bath, th.gkt, th.q, n_steps, gate,
                                      nl->md_ints + 2));
    return REANN_OK;
}

int md_run(reann_ctx* ctx, reann_nlist* nl, double* pos, double* vel, const double* mass, double dt, int n_steps,
           double* e_pot, double* e_kin, const Thermo& th, double* e_bath) {
    cudaStream_t s = ctx->stream;
    const int64_t n = nl->n;
    if (!nl->md_forces) {
        nl->md_forces = nl_alloc<float>(nl, 3 * n);
        nl->md_scalars = nl_alloc<double>(nl, 8);
        nl->md_partial = nl_alloc<double>(nl, (n + 2047) / 2048);
        nl->md_ints = nl_alloc<int>(nl, 3);
        if (!nl->md_forces || !nl->md_scalars || !nl->md_partial || !nl->md_ints)
            return set_error(ctx, REANN_E_NOMEM, "MD buffers: out of device memory");
        REANN_CUDA_TRY(ctx, cudaMemsetAsync(nl->md_ints, 0, 3 * sizeof(int), s));
        REANN_CUDA_TRY(ctx, cudaMemsetAsync(nl->md_scalars, 0, 8 * sizeof(double), s));  // xi = eta = 0
    }
    int* gate = nl->md_ints;
    // forces at the starting positions (rebuilding first if atoms moved beyond skin/2)
    if (!nl->md_forces_valid || nl->md_forces_at != pos || nl->md_precision != ctx->precision) {
        REANN_CUDA_TRY(ctx, cudaMemsetAsync(gate, 0, sizeof(int), s));
        REANN_CUDA_TRY(ctx, launch_moved(s, nl, pos, gate));
        REANN_CUDA_TRY(ctx, launch_rebuild(s, nl, pos, ctx->d_flags, gate));
        int rc = run_energy_forces(ctx, nl, pos, nl->T, nl->md_scalars, nl->md_forces, nullptr);
        if (rc) return rc;
        nl->md_forces_valid = true;
        nl->md_forces_at = pos;
    }
    // the thermostat's first half step needs K of the current velocities
    if (th.on()) REANN_CUDA_TRY(ctx, launch_ekin(s, n, vel, mass, nl->md_partial, nl->md_scalars + 1));
    const void* key[6] = {pos, vel, mass, e_pot, e_kin, e_bath};
    const bool same = nl->md_exec && std::memcmp(key, nl->md_key, sizeof(key)) == 0 && nl->md_dt == dt &&
                      nl->md_precision == ctx->precision && nl->md_nsteps == n_steps && nl->md_kt == th.kt &&
                      nl->md_tau == th.tau;
    if (!same) {
        if (nl->md_exec) cudaGraphExecDestroy(nl->md_exec);
        if (nl->md_graph) cudaGraphDestroy(nl->md_graph);
        nl->md_exec = nullptr;
        nl->md_graph = nullptr;
        REANN_CUDA_TRY(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        const int rc = md_step_body(ctx, nl, pos, vel, mass, dt, n_steps, e_pot, e_kin, th, e_bath);
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(s, &g);
        if (rc || ec != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return rc ? rc : set_error(ctx, REANN_E_CUDA, std::string("MD step capture: ") + cudaGetErrorString(ec));
        }
        nl->md_graph = g;
        REANN_CUDA_TRY(ctx, cudaGraphInstantiate(&nl->md_exec, g, 0));
        std::memcpy(nl->md_key, key, sizeof(key));
        nl->md_dt = dt;
        nl->md_precision = ctx->precision;
        nl->md_nsteps = n_steps;
        nl->md_kt = th.kt;
        nl->md_tau = th.tau;
    }
    REANN_CUDA_TRY(ctx, cudaMemsetAsync(nl->md_ints + 1, 0, sizeof(int), s));
    for (int k = 0; k < n_steps; ++k) REANN_CUDA_TRY(ctx, cudaGraphLaunch(nl->md_exec, s));
    return REANN_OK;
}

}  // namespace

namespace {

int md_entry(reann_ctx* ctx, reann_nlist* nl, double* pos, double* vel, const double* mass, double dt_fs, int n_steps,
             double* e_pot, double* e_kin, const Thermo& th, double* e_bath);

}  // namespace

extern "C" int reann_md_step(reann_ctx* ctx, reann_nlist* nl, double* pos, double* vel, const double* mass,
                             double dt_fs, int n_steps, double* e_pot, double* e_kin) {
    if (!ctx || !nl) return set_error(ctx, REANN_E_ARG, "bad argument to reann_md_step");
    return md_entry(ctx, nl, pos, vel, mass, dt_fs, n_steps, e_pot, e_kin, Thermo{}, nullptr);
}

extern "C" int reann_md_step_nvt(reann_ctx* ctx, reann_nlist* nl, double* pos, double* vel, const double* mass,
                                 double dt_fs, int n_steps, double temperature_k, double tau_fs, double* e_pot,
                                 double* e_kin, double* e_bath) {
    if (!ctx || !nl || !(temperature_k > 0) || !std::isfinite(temperature_k) || !(tau_fs > 0) ||
        !std::isfinite(tau_fs) || nl->n < 2)
        return set_error(ctx, REANN_E_ARG, "bad argument to reann_md_step_nvt");
    return md_entry(ctx, nl, pos, vel, mass, dt_fs, n_steps, e_pot, e_kin, make_thermo(nl->n, temperature_k, tau_fs),
                    e_bath);
}

namespace {

int md_entry(reann_ctx* ctx, reann_nlist* nl, double* pos, double* vel, const double* mass, double dt_fs, int n_steps,
             double* e_pot, double* e_kin, const Thermo& th, double* e_bath) {
    if (!ctx || !nl || !pos || !vel || !mass || !(dt_fs > 0) || !std::isfinite(dt_fs) || n_steps < 0)
        return set_error(ctx, REANN_E_ARG, "bad argument to reann_md_step");
    if (nl->decomposed) return set_error(ctx, REANN_E_ARG, "MD needs device rebuilds: use a single-domain list");
    if (n_steps == 0) return REANN_OK;
    // run on the graph stream, ordered after and before the caller's stream
    const bool prof = ctx->prof_on;
    ctx->prof_on = false;
    const int rc = on_graph_stream(
        ctx, [&] { return md_run(ctx, nl, pos, vel, mass, dt_fs, n_steps, e_pot, e_kin, th, e_bath); });
    ctx->prof_on = prof;
    return rc;
}

}  // namespace

extern "C" int reann_md_info(reann_ctx* ctx, const reann_nlist* nl, int64_t* steps, int64_t* rebuilds) {
    if (!ctx || !nl) return REANN_E_ARG;
    int h[3] = {0, 0, 0};
    if (nl->md_ints) {
        REANN_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        REANN_CUDA_TRY(ctx, cudaMemcpy(h, nl->md_ints, sizeof(h), cudaMemcpyDeviceToHost));
    }
    if (steps) *steps = h[1];
    if (rebuilds) *rebuilds = h[2];
    return REANN_OK;
}

extern "C" int reann_ctx_profile(reann_ctx* ctx, int enable) {
    if (!ctx) return REANN_E_ARG;
    prof_collect(ctx);
    ctx->prof_on = enable != 0;
    for (int r = 0; r < PR_COUNT; ++r) {
        ctx->prof_ms[r] = 0.0;
        ctx->prof_n[r] = 0;
    }
    return REANN_OK;
}

extern "C" int reann_profile_regions(void) { return PR_COUNT; }

extern "C" const char* reann_profile_region_name(int region) {
    return (region >= 0 && region < PR_COUNT) ? kRegionNames[region] : "";
}

extern "C" int reann_ctx_profile_read(reann_ctx* ctx, double* total_ms, int64_t* launches) {
    if (!ctx || !total_ms || !launches) return REANN_E_ARG;
    prof_collect(ctx);
    for (int r = 0; r < PR_COUNT; ++r) {
        total_ms[r] = ctx->prof_ms[r];
        launches[r] = ctx->prof_n[r];
    }
    return REANN_OK;
}

extern "C" int reann_get_layer(reann_ctx* ctx, const reann_nlist* nl, int layer, float* rho, float* coef) {
    if (!ctx || !nl || layer < 0 || layer >= nl->T) return set_error(ctx, REANN_E_ARG, "bad layer");
    const int64_t n = nl->n, ne = nl->n + nl->g_cap;
    if (rho)
        REANN_CUDA_TRY(ctx, launch_unpermute_rows(ctx->stream, nl, nl->rho + (size_t)layer * n * nl->n_feat, nl->n_feat,
                                                  rho, nl->n_feat));
    if (coef)
        REANN_CUDA_TRY(ctx, launch_unpermute_rows(ctx->stream, nl, nl->coef + (size_t)layer * ne * NPHI, NPHI, coef, NPHI));
    return REANN_OK;
}

// ================================================================ serving ==

namespace {

// first-fit allocator of [start, start + len) ranges with coalescing
struct RangeAlloc {
    std::vector<std::pair<int64_t, int64_t>> free;  // sorted (start, len)
    void init(int64_t n) { free.assign(1, {0, n}); }
    bool take(int64_t len, int64_t* start) {
        if (len == 0) {
            *start = 0;
            return true;
        }
        for (size_t k = 0; k < free.size(); ++k)
            if (free[k].second >= len) {
                *start = free[k].first;
                free[k].first += len;
                free[k].second -= len;
                if (free[k].second == 0) free.erase(free.begin() + k);
                return true;
            }
        return false;
    }
    void give(int64_t start, int64_t len) {
        if (len == 0) return;
        auto it = std::lower_bound(free.begin(), free.end(), std::make_pair(start, (int64_t)0));
        it = free.insert(it, {start, len});
        size_t k = it - free.begin();
        if (k + 1 < free.size() && free[k].first + free[k].second == free[k + 1].first) {
            free[k].second += free[k + 1].second;
            free.erase(free.begin() + k + 1);
        }
        if (k > 0 && free[k - 1].first + free[k - 1].second == free[k].first) {
            free[k - 1].second += free[k].second;
            free.erase(free.begin() + k);
        }
    }
};

struct ServeSlot {
    bool used = false, pending = false, retired = false;
    int64_t ob = 0, n = 0, gb = 0, g = 0;
    std::vector<Tile> t64, t128;
};

}  // namespace

struct reann_serve {
    std::mutex mu;  // slots, ranges, staging and the pool stream; builds run outside it
    reann_ctx* ctx = nullptr;
    reann_nlist* pool = nullptr;
    int max_slots = 0;
    RangeAlloc owned, ghost;
    std::vector<ServeSlot> slots;
    int4* d_seg = nullptr;
    int4* h_seg = nullptr;  // pinned staging
    Tile *h_t64 = nullptr, *h_t128 = nullptr;
    cudaStream_t stream = nullptr;
    cudaMemPool_t build_pool = nullptr;  // stream-ordered blocks of the per-submission lists
    cudaEvent_t staged = nullptr, done = nullptr, user_ready = nullptr;
    std::vector<std::pair<reann_nlist*, cudaEvent_t>> deferred;  // built lists freed once their pack has run
    // one captured pass per size class k: owned rows [0, n >> k), ghost slots [0, g_cap >> k)
    static constexpr int kClasses = 8;
    static constexpr int64_t kMinRows = 2048;
    cudaGraph_t graph[kClasses] = {};
    cudaGraphExec_t exec[kClasses] = {};
    int graph_precision = -1;
    const void* graph_out[2] = {nullptr, nullptr};
};

namespace {

void serve_reap(reann_serve* srv, bool wait) {
    for (size_t k = 0; k < srv->deferred.size();) {
        auto& d = srv->deferred[k];
        if (wait) cudaEventSynchronize(d.second);
        if (cudaEventQuery(d.second) == cudaSuccess) {
            d.first->alloc_stream = srv->stream;  // its last readers ran there
            free_nlist(d.first);
            cudaEventDestroy(d.second);
            srv->deferred.erase(srv->deferred.begin() + k);
        } else {
            ++k;
        }
    }
}

// one evaluation of every structure in the segment table, then their retirement
int pool_pass(reann_ctx* ctx, reann_serve* srv, double* energies, float* forces) {
    reann_nlist* p = srv->pool;
    int rc = run_energy_forces(ctx, p, nullptr, p->T, energies, forces, nullptr, srv->d_seg, srv->max_slots);
    if (!rc) REANN_CUDA_TRY(ctx, launch_retire(ctx->stream, srv->d_seg, srv->max_slots, p));
    return rc;
}

}  // namespace

extern "C" void reann_serve_free(reann_serve* srv) {
    if (!srv) return;
    if (srv->stream) cudaStreamSynchronize(srv->stream);
    serve_reap(srv, true);
    if (srv->stream) cudaStreamSynchronize(srv->stream);
    if (srv->build_pool) cudaMemPoolDestroy(srv->build_pool);
    for (int k = 0; k < reann_serve::kClasses; ++k) {
        if (srv->exec[k]) cudaGraphExecDestroy(srv->exec[k]);
        if (srv->graph[k]) cudaGraphDestroy(srv->graph[k]);
    }
    free_nlist(srv->pool);
    if (srv->d_seg) cudaFree(srv->d_seg);
    if (srv->h_seg) cudaFreeHost(srv->h_seg);
    if (srv->h_t64) cudaFreeHost(srv->h_t64);
    if (srv->h_t128) cudaFreeHost(srv->h_t128);
    for (cudaEvent_t e : {srv->staged, srv->done, srv->user_ready})
        if (e) cudaEventDestroy(e);
    if (srv->stream) cudaStreamDestroy(srv->stream);
    delete srv;
}

extern "C" int reann_serve_create(reann_ctx* ctx, int64_t max_atoms, int64_t max_ghosts, int max_structures,
                                  int stride, reann_serve** out) {
    if (!ctx || !out || max_atoms < 1 || max_ghosts < 0 || max_structures < 1 || stride < 8 || stride > 4096 ||
        max_atoms > ((int64_t)1 << 28))
        return set_error(ctx, REANN_E_ARG, "bad argument to reann_serve_create");
    *out = nullptr;
    reann_serve* srv = new (std::nothrow) reann_serve;
    if (!srv) return set_error(ctx, REANN_E_NOMEM, "host allocation failed");
    auto fail = [&](int code, const char* msg) {
        reann_serve_free(srv);
        return set_error(ctx, code, msg);
    };
    srv->ctx = ctx;
    srv->max_slots = max_structures;
    srv->slots.resize(max_structures);
    srv->owned.init(max_atoms);
    srv->ghost.init(max_ghosts);
    reann_nlist* p = new (std::nothrow) reann_nlist;
    if (!p) return fail(REANN_E_NOMEM, "host allocation failed");
    srv->pool = p;
    p->n = max_atoms;
    p->g = p->g_cap = max_ghosts;
    p->stride = stride;
    p->n_elem = ctx->model.n_elem;
    p->T = ctx->model.T;
    p->r_c = ctx->model.r_c;
    p->perm = nl_alloc<int32_t>(p, max_atoms);
    p->species = nl_alloc<int32_t>(p, max_atoms);
    p->g_owner = nl_alloc<int32_t>(p, max_ghosts);
    p->nbr = nl_alloc<int32_t>(p, (size_t)max_atoms * stride);
    p->nbr_cnt = nl_alloc<int32_t>(p, max_atoms);
    p->w.goff = nl_alloc<int32_t>(p, max_atoms + 1);
    if (!p->perm || !p->species || !p->g_owner || !p->nbr || !p->nbr_cnt || !p->w.goff)
        return fail(REANN_E_NOMEM, "serving pool: out of device memory");
    if (alloc_eval_buffers(ctx, p)) return fail(REANN_E_NOMEM, "serving pool: out of device memory");
    // tile lists of fixed capacity (padding entries have nrows = 0)
    const int64_t cap64 = max_atoms / MLP_TILE + (int64_t)max_structures * p->n_elem + 1;
    const int64_t cap128 = max_atoms / 128 + (int64_t)max_structures * p->n_elem + 1;
    p->tiles_h.assign(cap64, Tile{0, 0, 0, 0});
    p->tiles128_h.assign(cap128, Tile{0, 0, 0, 0});
    p->tiles = nl_alloc<Tile>(p, cap64);
    p->tiles128 = nl_alloc<Tile>(p, cap128);
    if (!p->tiles || !p->tiles128 || cudaMalloc(&srv->d_seg, sizeof(int4) * max_structures) != cudaSuccess ||
        cudaMallocHost(&srv->h_seg, sizeof(int4) * max_structures) != cudaSuccess ||
        cudaMallocHost(&srv->h_t64, sizeof(Tile) * cap64) != cudaSuccess ||
        cudaMallocHost(&srv->h_t128, sizeof(Tile) * cap128) != cudaSuccess)
        return fail(REANN_E_NOMEM, "serving pool: out of memory");
    if (cudaStreamCreateWithFlags(&srv->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&srv->staged, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&srv->done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&srv->user_ready, cudaEventDisableTiming) != cudaSuccess)
        return fail(REANN_E_CUDA, "serving pool: stream/event creation failed");
    {
        int dev = 0;
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        if (cudaGetDevice(&dev) != cudaSuccess) return fail(REANN_E_CUDA, "serving pool: no current device");
        props.location.id = dev;
        uint64_t keep = UINT64_MAX;  // released blocks stay mapped for the next submission
        if (cudaMemPoolCreate(&srv->build_pool, &props) != cudaSuccess ||
            cudaMemPoolSetAttribute(srv->build_pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess)
            return fail(REANN_E_CUDA, "serving pool: memory pool creation failed");
    }
    // empty pool: no neighbours, outputs to the sink row, every ghost slot "in use" (all point at atom 0)
    std::vector<int32_t> sink(max_atoms, (int32_t)max_atoms), goff(max_atoms + 1, 0);
    goff[max_atoms] = (int32_t)max_ghosts;
    bool ok = cudaMemcpy(p->perm, sink.data(), sizeof(int32_t) * max_atoms, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(p->w.goff, goff.data(), sizeof(int32_t) * (max_atoms + 1), cudaMemcpyHostToDevice) ==
                  cudaSuccess &&
              cudaMemset(p->nbr_cnt, 0, sizeof(int32_t) * max_atoms) == cudaSuccess &&
              cudaMemset(p->species, 0, sizeof(int32_t) * max_atoms) == cudaSuccess &&
              cudaMemset(p->g_owner, 0, sizeof(int32_t) * std::max<int64_t>(max_ghosts, 1)) == cudaSuccess &&
              cudaMemset(p->pos_hi, 0, sizeof(float4) * (max_atoms + max_ghosts)) == cudaSuccess &&
              cudaMemset(p->pos_lo, 0, sizeof(float4) * (max_atoms + max_ghosts)) == cudaSuccess &&
              cudaDeviceSynchronize() == cudaSuccess;
    if (!ok) return fail(REANN_E_CUDA, "serving pool: initialisation failed");
    *out = srv;
    return REANN_OK;
}

extern "C" int reann_serve_submit(reann_serve* srv, reann_ctx* build_ctx, int64_t n_atoms, const double* pos,
                                  const int32_t* species, const double* cell, double skin, int* slot) {
    if (!srv || !build_ctx || !slot) return REANN_E_ARG;
    reann_ctx* ctx = srv->ctx;
    if (build_ctx->model.T != ctx->model.T || build_ctx->model.n_elem != ctx->model.n_elem ||
        build_ctx->model.r_c != ctx->model.r_c)
        return set_error(ctx, REANN_E_MISMATCH, "build context holds a different model");
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        serve_reap(srv, false);
        // refuse early when no structure slot or owned range can take it (ghosts are known only after the build)
        bool slot_free = false;
        for (const ServeSlot& sl : srv->slots) slot_free |= !sl.used;
        int64_t widest = 0;
        for (auto& r : srv->owned.free) widest = std::max(widest, r.second);
        if (!slot_free || widest < n_atoms) return set_error(ctx, REANN_E_NOMEM, "serving pool full (admission refused)");
    }
    reann_nlist* tmp = nullptr;
    int rc = build_list(build_ctx, n_atoms, pos, species, cell, ctx->model.r_c, skin, false, &tmp, srv->build_pool);
    std::lock_guard<std::mutex> lock(srv->mu);
    if (rc) return set_error(ctx, rc, std::string("structure build: ") + build_ctx->err);
    if (tmp->max_count > srv->pool->stride) {
        free_nlist(tmp);
        return set_error(ctx, REANN_E_CAPACITY, "a neighbour row is longer than the pool stride");
    }
    int s = -1;
    for (int k = 0; k < srv->max_slots; ++k)
        if (!srv->slots[k].used) {
            s = k;
            break;
        }
    int64_t ob = 0, gb = 0;
    if (s < 0 || !srv->owned.take(tmp->n, &ob)) {
        free_nlist(tmp);
        return set_error(ctx, REANN_E_NOMEM, "serving pool full (admission refused)");
    }
    if (!srv->ghost.take(tmp->g, &gb)) {
        srv->owned.give(ob, tmp->n);
        free_nlist(tmp);
        return set_error(ctx, REANN_E_NOMEM, "serving pool full (admission refused)");
    }
    ServeSlot& sl = srv->slots[s];
    sl.used = true;
    sl.pending = true;
    sl.ob = ob;
    sl.n = tmp->n;
    sl.gb = gb;
    sl.g = tmp->g;
    sl.t64.clear();
    sl.t128.clear();
    for (int e = 0; e < tmp->n_elem; ++e) {
        for (int r = tmp->elem_start[e]; r < tmp->elem_start[e + 1]; r += MLP_TILE)
            sl.t64.push_back(Tile{e, (int)(ob + r), std::min(MLP_TILE, tmp->elem_start[e + 1] - r), 0});
        for (int r = tmp->elem_start[e]; r < tmp->elem_start[e + 1]; r += 128)
            sl.t128.push_back(Tile{e, (int)(ob + r), std::min(128, tmp->elem_start[e + 1] - r), 0});
    }
    // pack on the pool stream (ordered with launches); the built list lives until the pack has run
    REANN_CUDA_TRY(ctx, launch_pack(srv->stream, tmp, tmp->pos_ref, srv->pool, ob, gb));
    cudaEvent_t ev = nullptr;
    REANN_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    REANN_CUDA_TRY(ctx, cudaEventRecord(ev, srv->stream));
    srv->deferred.push_back({tmp, ev});
    *slot = s;
    return REANN_OK;
}

extern "C" int reann_serve_launch(reann_serve* srv, double* energies, float* forces, int* slots, int* count) {
    if (!srv || !energies || !forces || !count) return REANN_E_ARG;
    std::lock_guard<std::mutex> lock(srv->mu);
    reann_ctx* ctx = srv->ctx;
    reann_nlist* p = srv->pool;
    // the pinned staging buffers of the previous launch must have been copied
    REANN_CUDA_TRY(ctx, cudaEventSynchronize(srv->staged));
    size_t n64 = 0, n128 = 0;
    int nseg = 0;
    int64_t hi = 0, ghi = 0;  // owned rows and ghost slots the launched structures occupy
    for (int k = 0; k < srv->max_slots; ++k) {
        ServeSlot& sl = srv->slots[k];
        if (!sl.used || !sl.pending) continue;
        hi = std::max<int64_t>(hi, sl.ob + sl.n);
        ghi = std::max<int64_t>(ghi, sl.gb + sl.g);
        for (const Tile& t : sl.t64) srv->h_t64[n64++] = t;
        for (const Tile& t : sl.t128) srv->h_t128[n128++] = t;
        srv->h_seg[nseg] = make_int4((int)sl.ob, (int)sl.n, k, 0);
        if (slots) slots[nseg] = k;
        ++nseg;
        sl.pending = false;
        sl.retired = true;  // by the pass below
    }
    *count = nseg;
    if (nseg == 0) return REANN_OK;
    for (size_t k = n64; k < p->tiles_h.size(); ++k) srv->h_t64[k] = Tile{0, 0, 0, 0};
    for (size_t k = n128; k < p->tiles128_h.size(); ++k) srv->h_t128[k] = Tile{0, 0, 0, 0};
    for (int k = nseg; k < srv->max_slots; ++k) srv->h_seg[k] = make_int4(0, -1, 0, 0);
    cudaStream_t s = srv->stream;
    REANN_CUDA_TRY(ctx, cudaEventRecord(srv->user_ready, ctx->stream));
    REANN_CUDA_TRY(ctx, cudaStreamWaitEvent(s, srv->user_ready, 0));
    REANN_CUDA_TRY(ctx, cudaMemcpyAsync(p->tiles, srv->h_t64, sizeof(Tile) * p->tiles_h.size(), cudaMemcpyHostToDevice, s));
    REANN_CUDA_TRY(ctx, cudaMemcpyAsync(p->tiles128, srv->h_t128, sizeof(Tile) * p->tiles128_h.size(),
                                        cudaMemcpyHostToDevice, s));
    REANN_CUDA_TRY(ctx, cudaMemcpyAsync(srv->d_seg, srv->h_seg, sizeof(int4) * srv->max_slots, cudaMemcpyHostToDevice, s));
    REANN_CUDA_TRY(ctx, cudaEventRecord(srv->staged, s));
    // One evaluation of the pool, sized to the work: size class k covers owned rows
    // [0, n >> k) and ghost slots [0, g_cap >> k), the smallest class holding every
    // launched structure (free and retired rows inside it have no neighbours).  Each
    // class is captured once per (precision, outputs) and replayed.
    int cls = 0, ncls = 1;
    while (ncls < reann_serve::kClasses && (p->n >> ncls) >= reann_serve::kMinRows) ++ncls;
    while (cls + 1 < ncls && (p->n >> (cls + 1)) >= hi && (p->g_cap >> (cls + 1)) >= ghi) ++cls;
    const auto set_class = [&](int k) {
        const int64_t rows = p->n >> k;
        p->n_rows = rows;
        p->g_rows = p->g_cap >> k;
        // tiles of the launched structures: at most rows / tile + one partial tile per element and structure
        const int64_t ms = std::min<int64_t>(srv->max_slots, rows) * p->n_elem + 1;
        p->tiles_active = std::min<int64_t>((int64_t)p->tiles_h.size(), rows / MLP_TILE + ms);
        p->tiles128_active = std::min<int64_t>((int64_t)p->tiles128_h.size(), rows / 128 + ms);
    };
    set_class(cls);
    cudaStream_t user = ctx->stream;
    const bool prof = ctx->prof_on;
    ctx->stream = s;
    ctx->prof_on = false;
    int rc = REANN_OK;
    if (srv->graph_precision != ctx->precision || srv->graph_out[0] != energies || srv->graph_out[1] != forces) {
        for (int k = 0; k < reann_serve::kClasses; ++k) {  // another key: every class is captured again
            if (srv->exec[k]) cudaGraphExecDestroy(srv->exec[k]);
            if (srv->graph[k]) cudaGraphDestroy(srv->graph[k]);
            srv->exec[k] = nullptr;
            srv->graph[k] = nullptr;
        }
        srv->graph_precision = ctx->precision;
        srv->graph_out[0] = energies;
        srv->graph_out[1] = forces;
    }
    if (!srv->exec[cls]) {
        // this launch runs directly (which also sets kernel attributes outside capture);
        // then every size class is captured, so that no later launch pays for a capture
        rc = pool_pass(ctx, srv, energies, forces);
        for (int k = 0; k < ncls && !rc; ++k) {
            if (srv->exec[k]) continue;
            set_class(k);
            if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                rc = set_error(ctx, REANN_E_CUDA, "serving graph capture failed");
                break;
            }
            rc = pool_pass(ctx, srv, energies, forces);
            cudaGraph_t g = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(s, &g);
            if (!rc && ec == cudaSuccess && cudaGraphInstantiate(&srv->exec[k], g, 0) == cudaSuccess) {
                srv->graph[k] = g;
            } else {
                if (g) cudaGraphDestroy(g);
                srv->exec[k] = nullptr;
                if (!rc) rc = set_error(ctx, REANN_E_CUDA, "serving graph capture failed");
            }
        }
    } else if (cudaGraphLaunch(srv->exec[cls], s) != cudaSuccess) {
        rc = set_error(ctx, REANN_E_CUDA, "serving graph launch failed");
    }
    p->n_rows = p->g_rows = p->tiles_active = p->tiles128_active = -1;
    ctx->stream = user;
    ctx->prof_on = prof;
    REANN_CUDA_TRY(ctx, cudaEventRecord(srv->done, s));
    REANN_CUDA_TRY(ctx, cudaStreamWaitEvent(user, srv->done, 0));
    serve_reap(srv, false);
    return rc;
}

extern "C" int reann_serve_release(reann_serve* srv, int slot) {
    if (!srv) return REANN_E_ARG;
    std::lock_guard<std::mutex> lock(srv->mu);
    if (slot < 0 || slot >= srv->max_slots || !srv->slots[slot].used) return REANN_E_ARG;
    ServeSlot& sl = srv->slots[slot];
    if (!sl.retired) REANN_CUDA_TRY(srv->ctx, launch_release(srv->stream, srv->pool, sl.ob, sl.n));
    srv->owned.give(sl.ob, sl.n);
    srv->ghost.give(sl.gb, sl.g);
    sl = ServeSlot{};
    return REANN_OK;
}

extern "C" int reann_serve_slot(reann_serve* srv, int slot, int64_t* atom_offset, int64_t* n_atoms) {
    if (!srv) return REANN_E_ARG;
    std::lock_guard<std::mutex> lock(srv->mu);
    if (slot < 0 || slot >= srv->max_slots || !srv->slots[slot].used) return REANN_E_ARG;
    if (atom_offset) *atom_offset = srv->slots[slot].ob;
    if (n_atoms) *n_atoms = srv->slots[slot].n;
    return REANN_OK;
}

extern "C" int reann_serve_usage(reann_serve* srv, int64_t* free_atoms, int64_t* free_ghosts, int* free_slots) {
    if (!srv) return REANN_E_ARG;
    std::lock_guard<std::mutex> lock(srv->mu);
    int64_t fa = 0, fg = 0;
    for (auto& r : srv->owned.free) fa = std::max(fa, r.second);
    for (auto& r : srv->ghost.free) fg = std::max(fg, r.second);
    int fs = 0;
    for (auto& sl : srv->slots) fs += !sl.used;
    if (free_atoms) *free_atoms = fa;
    if (free_ghosts) *free_ghosts = fg;
    if (free_slots) *free_slots = fs;
    return REANN_OK;
}
