// noalloc.cu -- lbmd_particle_sums_static: the particle-momentum and
// kinetic-energy reduction of lbmd_observables, for caller-owned device
// arrays, with no device allocation at all.
//
// Who needs it: callers that must not allocate device memory -- code running
// while a framework captures the stream into a CUDA graph and forbids
// allocation during capture, code living inside a framework whose caching
// allocator owns the device memory budget (a raw cudaMalloc there can fail or
// fragment its pool), and latency-critical paths where cudaMalloc is too slow
// or may synchronise the device.  Instead of a scratch buffer from
// cudaMalloc, the per-block partial sums live in one file-scope __device__
// array of fixed size (g_partials, 32 KB), which every GPU that loads this
// library holds until the process exits.
#include <mutex>

#include "lbmd_ctx.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int64_t NA_PER_BLOCK = 4096;  // particles per block
constexpr int NA_MAX_BLOCKS = 1024;     // rows of the scratch array
constexpr int NA_MAX_DEVICES = 64;

// scratch: one row of 4 partial sums per block
__device__ __align__(256) double g_partials[NA_MAX_BLOCKS * 4];

double *g_partials_addr[NA_MAX_DEVICES];  // device address per device id
std::mutex g_setup_mutex;

__global__ void __launch_bounds__(NA_THREADS)
    particle_sums_partial_kernel(const double *vel, const double *mass, int64_t n, double *partials) {
    __shared__ double sh[4][NA_THREADS];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    const int64_t lo = (int64_t)blockIdx.x * NA_PER_BLOCK;
    const int64_t hi = lo + NA_PER_BLOCK < n ? lo + NA_PER_BLOCK : n;
    for (int64_t p = lo + threadIdx.x; p < hi; p += NA_THREADS) {
        const double m = mass ? mass[p] : 1.0;
        const double vx = vel[3 * p], vy = vel[3 * p + 1], vz = vel[3 * p + 2];
        v[0] += m * vx;
        v[1] += m * vy;
        v[2] += m * vz;
        v[3] += m * (vx * vx + vy * vy + vz * vz);
    }
    for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] = v[c];
    __syncthreads();
    for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 4) partials[4 * (int64_t)blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

// rows 0..blocks-1 added in order; every row is rewritten by the call that
// reads it, so no clearing is needed between calls
__global__ void particle_sums_final_kernel(const double *partials, int blocks, double *out) {
    const int c = threadIdx.x;
    if (c >= 4) return;
    double s = 0.0;
    for (int b = 0; b < blocks; ++b) s += partials[4 * b + c];
    out[c] = s;
}

}  // namespace

extern "C" lbmd_status lbmd_particle_sums_static(const double *vel, const double *mass, int64_t n, double *out,
                                                 void *stream) {
    if (n < 0 || !out || (n > 0 && !vel)) {
        lbmd_set_global_error("lbmd_particle_sums_static: bad arguments");
        return LBMD_ERR_ARG;
    }
    if (n > (int64_t)NA_MAX_BLOCKS * NA_PER_BLOCK) {
        lbmd_set_global_error("lbmd_particle_sums_static: more than 4194304 particles (fixed scratch size)");
        return LBMD_ERR_CAPACITY;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        lbmd_set_global_error("lbmd_particle_sums_static: no usable current device");
        return LBMD_ERR_CUDA;
    }
    double *partials = nullptr;
    {
        // once per device, with that device current: the device address of
        // the scratch array (its host-side name is only a stand-in)
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_partials_addr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_partials);
            if (e != cudaSuccess || !ptr) {
                lbmd_set_global_error(std::string("lbmd_particle_sums_static: cudaGetSymbolAddress: ") +
                                      cudaGetErrorString(e));
                return LBMD_ERR_CUDA;
            }
            g_partials_addr[dev] = static_cast<double *>(ptr);
        }
        partials = g_partials_addr[dev];
    }
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = (int)((n + NA_PER_BLOCK - 1) / NA_PER_BLOCK);
    if (blocks > 0) particle_sums_partial_kernel<<<blocks, NA_THREADS, 0, s>>>(vel, mass, n, partials);
    particle_sums_final_kernel<<<1, 32, 0, s>>>(partials, blocks, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        lbmd_set_global_error(std::string("lbmd_particle_sums_static: ") + cudaGetErrorString(e));
        return LBMD_ERR_CUDA;
    }
    return LBMD_OK;
}
