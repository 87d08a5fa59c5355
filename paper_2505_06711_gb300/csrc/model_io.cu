// Model files: reann_model_load / reann_model_save.
//
// A model is the shape of Eqs. 1-2 (elements, layers T, N_phi Gaussians, L,
// orbitals, hidden widths, r_c, alpha, feature kind) and the flat FP32
// parameter vector of reann_model_create.  The file stores exactly that, in
// little-endian byte order whatever the host's:
//
//   offset  size  field
//        0     8  magic "REANNMDL"
//        8     4  uint32 format version (1)
//       12    32  int32 n_elem, T, n_phi, l_max, n_orb, h1, h2, feature_pairs
//       44     4  uint32 reserved (0)
//       48     8  float64 r_c
//       56     8  float64 alpha
//       64     8  int64 n_params
//       72  4 n_params  float32 parameters
//
// The loader reads the whole file, checks the magic, the version, that the
// size is exactly 72 + 4 n_params bytes, and hands the values to
// reann_model_create_ex, which validates the shape and the parameter count.
// Host only: no CUDA call.
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

namespace {

constexpr char kMagic[8] = {'R', 'E', 'A', 'N', 'N', 'M', 'D', 'L'};
constexpr uint32_t kVersion = 1;
constexpr size_t kHeader = 72;

uint32_t get_u32(const unsigned char* p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
uint64_t get_u64(const unsigned char* p) { return (uint64_t)get_u32(p) | ((uint64_t)get_u32(p + 4) << 32); }
int32_t get_i32(const unsigned char* p) {
    const uint32_t u = get_u32(p);
    int32_t v;
    std::memcpy(&v, &u, 4);
    return v;
}
double get_f64(const unsigned char* p) {
    const uint64_t u = get_u64(p);
    double v;
    std::memcpy(&v, &u, 8);
    return v;
}
void put_u32(std::vector<unsigned char>& b, uint32_t v) {
    for (int k = 0; k < 4; ++k) b.push_back((unsigned char)((v >> (8 * k)) & 0xFFu));
}
void put_u64(std::vector<unsigned char>& b, uint64_t v) {
    put_u32(b, (uint32_t)(v & 0xFFFFFFFFu));
    put_u32(b, (uint32_t)(v >> 32));
}
void put_i32(std::vector<unsigned char>& b, int32_t v) {
    uint32_t u;
    std::memcpy(&u, &v, 4);
    put_u32(b, u);
}
void put_f64(std::vector<unsigned char>& b, double v) {
    uint64_t u;
    std::memcpy(&u, &v, 8);
    put_u64(b, u);
}

bool read_file(const char* path, std::vector<unsigned char>& out) {
    FILE* f = std::fopen(path, "rb");
    if (!f) return false;
    unsigned char buf[1 << 16];
    size_t got;
    bool ok = true;
    while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0) out.insert(out.end(), buf, buf + got);
    if (std::ferror(f)) ok = false;
    std::fclose(f);
    return ok;
}

}  // namespace

extern "C" int reann_model_load(const char* path, reann_model** out) {
    if (!path || !out) return REANN_E_ARG;
    *out = nullptr;
    std::vector<unsigned char> b;
    if (!read_file(path, b)) return REANN_E_ARG;
    if (b.size() < kHeader || std::memcmp(b.data(), kMagic, 8) != 0 || get_u32(b.data() + 8) != kVersion)
        return REANN_E_ARG;
    int32_t h[8];
    for (int k = 0; k < 8; ++k) h[k] = get_i32(b.data() + 12 + 4 * k);
    const double r_c = get_f64(b.data() + 48), alpha = get_f64(b.data() + 56);
    const int64_t n_params = (int64_t)get_u64(b.data() + 64);
    if (n_params < 1 || (uint64_t)n_params > (uint64_t)(b.size() - kHeader) / 4 ||
        b.size() != kHeader + 4 * (size_t)n_params)
        return REANN_E_ARG;  // truncated, padded or inconsistent
    std::vector<float> params((size_t)n_params);
    for (int64_t i = 0; i < n_params; ++i) {
        const uint32_t u = get_u32(b.data() + kHeader + 4 * (size_t)i);
        std::memcpy(&params[(size_t)i], &u, 4);
    }
    return reann_model_create_ex(h[0], h[1], h[2], h[3], h[4], h[5], h[6], r_c, alpha, h[7], params.data(),
                                 n_params, out);
}

extern "C" int reann_model_save(const reann_model* model, const char* path) {
    if (!model || !path) return REANN_E_ARG;
    const reann::Model& m = model->m;
    std::vector<unsigned char> b;
    b.reserve(kHeader + 4 * m.params.size());
    b.insert(b.end(), kMagic, kMagic + 8);
    put_u32(b, kVersion);
    const int32_t h[8] = {m.n_elem, m.T, reann::NPHI, reann::LMAX, m.n_orb(), reann::H1, reann::H2,
                          m.pairs ? 1 : 0};
    for (int k = 0; k < 8; ++k) put_i32(b, h[k]);
    put_u32(b, 0u);
    put_f64(b, m.r_c);
    put_f64(b, m.alpha);
    put_u64(b, (uint64_t)m.params.size());
    for (float x : m.params) {
        uint32_t u;
        std::memcpy(&u, &x, 4);
        put_u32(b, u);
    }
    FILE* f = std::fopen(path, "wb");
    if (!f) return REANN_E_ARG;
    const bool ok = std::fwrite(b.data(), 1, b.size(), f) == b.size();
    const bool closed = std::fclose(f) == 0;
    return ok && closed ? REANN_OK : REANN_E_ARG;
}
