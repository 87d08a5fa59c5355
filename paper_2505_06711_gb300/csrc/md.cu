// Velocity-Verlet integration in FP64 around the REANN force evaluation, NVE
// or NVT with one Nose-Hoover thermostat.
//
// One MD step (captured once as a CUDA graph and replayed):
//   [NVT: thermostat half step, v *= s]
//   v += (dt/2) F/m;  x += dt v;  rebuild the neighbour list if any atom moved
//   more than skin/2 since the last build (gated kernels, no host round trip);
//   E, F = REANN(x);  v += (dt/2) F/m;  K = sum m v^2 / 2 (FP64);
//   [NVT: thermostat half step, v *= s];  record E, K (and the bath energy).
// Thermostat half step of length dt/2 (time-reversible Trotter splitting of
// the Nose-Hoover equations xi' = (2K - g kT)/Q, eta' = xi, v' = -xi v):
//   xi += (dt/4) G(K);  eta += (dt/2) xi;  s = exp(-(dt/2) xi);  K *= s^2;
//   xi += (dt/4) G(K),  with G(K) = (2K - g kT)/Q, Q = g kT tau^2, g = 3N - 3.
// The conserved quantity is E + K + Q xi^2 / 2 + g kT eta.
// Units: A, fs, amu, eV; 1 eV/(A amu) = 9.648533212e-3 A/fs^2.
#include <cuda_runtime.h>

#include "common.cuh"

namespace reann {
namespace {

constexpr double kAccel = 9.648533212e-3;  // (eV/A)/amu -> A/fs^2
constexpr int kThreads = 256, kPer = 8;

// v = s v + (dt/2) F/m, s read from the device (1 without a thermostat)
__global__ void k_kick(int64_t n, double* __restrict__ vel, const float* __restrict__ forces,
                       const double* __restrict__ mass, double half_dt, const double* __restrict__ scale) {
    pdl_enter();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * n) return;
    const double v = scale ? vel[t] * *scale : vel[t];
    vel[t] = v + half_dt * kAccel * (double)forces[t] / mass[t / 3];
}

__global__ void k_scale(int64_t n, double* __restrict__ vel, const double* __restrict__ scale) {
    pdl_enter();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < 3 * n) vel[t] *= *scale;
}

// thermostat half step on the device scalars: sc[1] K, sc[2] xi, sc[3] eta, sc[4] s
__global__ void k_nh_half(double* __restrict__ sc, double dt, double gkt, double q) {
    pdl_enter();
    double K = sc[1], xi = sc[2], eta = sc[3];
    xi += 0.25 * dt * (2.0 * K - gkt) / q;
    eta += 0.5 * dt * xi;
    const double s = exp(-0.5 * dt * xi);
    K *= s * s;
    xi += 0.25 * dt * (2.0 * K - gkt) / q;
    sc[1] = K;
    sc[2] = xi;
    sc[3] = eta;
    sc[4] = s;
}

__global__ void k_drift(int64_t n, double* __restrict__ pos, const double* __restrict__ vel, double dt) {
    pdl_enter();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < 3 * n) pos[t] += dt * vel[t];
}

// kinetic energy in eV, two-level FP64 tree (fixed order, deterministic)
__global__ void __launch_bounds__(kThreads) k_ekin_partial(int64_t n, const double* __restrict__ vel,
                                                           const double* __restrict__ mass,
                                                           double* __restrict__ partial) {
    pdl_enter();
    __shared__ double sm[kThreads];
    const int64_t base = (int64_t)blockIdx.x * kThreads * kPer;
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int64_t i = base + k * kThreads + threadIdx.x;
        if (i < n) {
            const double vx = vel[3 * i], vy = vel[3 * i + 1], vz = vel[3 * i + 2];
            s += 0.5 * mass[i] * (vx * vx + vy * vy + vz * vz) / kAccel;
        }
    }
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

__global__ void __launch_bounds__(kThreads) k_ekin_final(int np, const double* __restrict__ partial,
                                                         double* __restrict__ out) {
    pdl_enter();
    __shared__ double sm[kThreads];
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += kThreads) s += partial[i];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sm[0];
}

// append this step's energies at the device step counter, count rebuilds; the
// bath energy Q xi^2 / 2 + g kT eta from the thermostat scalars
__global__ void k_record(int* __restrict__ counter, const double* __restrict__ sc, double* __restrict__ epot_out,
                         double* __restrict__ ekin_out, double* __restrict__ bath_out, double gkt, double q,
                         int n_steps, const int* __restrict__ gate, int* __restrict__ rebuilds) {
    pdl_enter();
    const int k = *counter;
    if (k < n_steps) {
        if (epot_out) epot_out[k] = sc[0];
        if (ekin_out) ekin_out[k] = sc[1];
        if (bath_out) bath_out[k] = 0.5 * q * sc[2] * sc[2] + gkt * sc[3];
    }
    *counter = k + 1;
    if (*gate) *rebuilds += 1;
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_kick(cudaStream_t s, int64_t n, double* vel, const float* forces, const double* mass,
                        double half_dt, const double* scale) {
    launch_pdl(k_kick, blocks_for(3 * n, 256), 256, 0, s, n, vel, forces, mass, half_dt, scale);
    return cudaGetLastError();
}

cudaError_t launch_scale(cudaStream_t s, int64_t n, double* vel, const double* scale) {
    launch_pdl(k_scale, blocks_for(3 * n, 256), 256, 0, s, n, vel, scale);
    return cudaGetLastError();
}

cudaError_t launch_nh_half(cudaStream_t s, double* scalars, double dt, double gkt, double q) {
    launch_pdl(k_nh_half, 1, 1, 0, s, scalars, dt, gkt, q);
    return cudaGetLastError();
}

cudaError_t launch_drift(cudaStream_t s, int64_t n, double* pos, const double* vel, double dt) {
    launch_pdl(k_drift, blocks_for(3 * n, 256), 256, 0, s, n, pos, vel, dt);
    return cudaGetLastError();
}

cudaError_t launch_ekin(cudaStream_t s, int64_t n, const double* vel, const double* mass, double* partial,
                        double* out) {
    const int np = (int)blocks_for(n, kThreads * kPer);
    launch_pdl(k_ekin_partial, np, kThreads, 0, s, n, vel, mass, partial);
    launch_pdl(k_ekin_final, 1, kThreads, 0, s, np, partial, out);
    return cudaGetLastError();
}

cudaError_t launch_record(cudaStream_t s, int* counter, const double* scalars, double* epot_out, double* ekin_out,
                          double* bath_out, double gkt, double q, int n_steps, const int* gate, int* rebuilds) {
    launch_pdl(k_record, 1, 1, 0, s, counter, scalars, epot_out, ekin_out, bath_out, gkt, q, n_steps, gate, rebuilds);
    return cudaGetLastError();
}

}  // namespace reann
