// reann_energy_sum_noalloc: the FP64 total-energy reduction without any
// device allocation.
//
// Some callers must not allocate device memory at the moment they need a total
// energy: force back-ends hosted as plugins by a molecular-dynamics engine
// whose force callback may not allocate (the engine owns the device-memory
// budget and its pools), and latency-critical callbacks that avoid cudaMalloc
// because it can synchronise the device.  This entry point sums per-atom
// energies that such a caller already holds, in FP64, using a fixed scratch
// array compiled into the library instead of memory allocated per call.
//
// Scratch: g_energy_partials below, kMaxPartials doubles (32 KiB), one per
// block of 2048 atoms, so at most kMaxAtoms = 8,388,608 atoms per call.  Every
// GPU that loads the library holds this array until the process exits.  Every
// call shares it and it keeps the last call's contents; each call writes every
// partial it later reads, so nothing needs clearing, but two calls that overlap
// on the GPU (different streams, or different host threads on one device) race
// on it and must be serialised by the caller.  The array's device address is
// looked up once per device (first call) and cached for the process lifetime.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/reann.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 8;
constexpr int64_t kAtomsPerBlock = (int64_t)kThreads * kPerThread;  // 2048
constexpr int kMaxPartials = 4096;
constexpr int64_t kMaxAtoms = kAtomsPerBlock * kMaxPartials;  // 8,388,608
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_energy_partials[kMaxPartials];

// device address of g_energy_partials, resolved once per device (host code may
// not use the symbol itself: on the host it names a stand-in, not device memory)
std::mutex g_mutex;
double* g_partials_addr[kMaxDevices] = {nullptr};

__global__ void __launch_bounds__(kThreads) k_partial(int64_t n, const float* __restrict__ eps,
                                                      double* __restrict__ partial) {
    __shared__ double sm[kThreads];
    const int64_t base = (int64_t)blockIdx.x * kAtomsPerBlock;
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
        if (i < n) s += (double)eps[i];
    }
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

__global__ void __launch_bounds__(kThreads) k_final(int np, const double* __restrict__ partial,
                                                    double* __restrict__ energy) {
    __shared__ double sm[kThreads];
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += kThreads) s += partial[i];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) energy[0] = sm[0];
}

// once per device, with that device current
int partials_on_current_device(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return REANN_E_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return REANN_E_ARG;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_partials_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_energy_partials) != cudaSuccess || !p) return REANN_E_CUDA;
        g_partials_addr[dev] = static_cast<double*>(p);
    }
    *out = g_partials_addr[dev];
    return REANN_OK;
}

}  // namespace

extern "C" int reann_energy_sum_noalloc(const float* atom_energy, int64_t n_atoms, double* energy,
                                        void* cuda_stream) {
    if (!energy || n_atoms < 0 || (n_atoms > 0 && !atom_energy)) return REANN_E_ARG;
    if (n_atoms > kMaxAtoms) return REANN_E_CAPACITY;
    double* partials = nullptr;
    const int rc = partials_on_current_device(&partials);
    if (rc != REANN_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int np = (int)((n_atoms + kAtomsPerBlock - 1) / kAtomsPerBlock);
    if (np > 0) {
        k_partial<<<np, kThreads, 0, s>>>(n_atoms, atom_energy, partials);
        if (cudaGetLastError() != cudaSuccess) return REANN_E_CUDA;
    }
    k_final<<<1, kThreads, 0, s>>>(np, partials, energy);
    return cudaGetLastError() == cudaSuccess ? REANN_OK : REANN_E_CUDA;
}

extern "C" int64_t reann_energy_sum_noalloc_max_atoms(void) { return kMaxAtoms; }
