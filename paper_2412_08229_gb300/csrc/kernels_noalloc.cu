// kernels_noalloc.cu - kinetic energy of a caller-held population state without any
// device allocation.
//
// Some callers cannot call cudaMalloc: code running inside a CUDA graph that is being
// captured, a host framework whose memory comes from its own pool and forbids
// allocations on its hot path, or an embedding that owns every device byte. This entry
// point serves them. Its only scratch (the per-block partial sums of the reduction) is
// a file-scope __device__ array of fixed size that every GPU loading this library holds
// until the process exits. Host code must not hand the array's name to a kernel (in
// host code the name is a host-side stand-in, not a device address): the device
// address is looked up once per device with cudaGetSymbolAddress and passed to the
// kernels.
#include <mutex>

#include "internal.h"

namespace lbm {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaCellsPerThread = 16;
constexpr long long kNaCellsPerBlock = static_cast<long long>(kNaThreads) * kNaCellsPerThread;  // 4096
constexpr int kNaMaxPartials = 4096;                                                           // 32 KB
constexpr long long kNaMaxCells = kNaCellsPerBlock * kNaMaxPartials;  // 16,777,216 = 256^3
constexpr int kNaMaxDevices = 64;

// One partial sum per block; every call overwrites exactly the slots it later reads.
__device__ __align__(256) double g_ke_scratch[kNaMaxPartials];

double* scratch_address(int device, cudaError_t* err) {
    static std::mutex mu;
    static double* addr[kNaMaxDevices] = {};
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device]) {
        void* p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_ke_scratch);
        if (*err != cudaSuccess) return nullptr;
        addr[device] = static_cast<double*>(p);
    }
    return addr[device];
}

__device__ __forceinline__ double na_block_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    if (w == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// Block b sums (1/2)|u|^2 over cells [b*4096, b*4096 + 4096) of absolute populations f
// (27 planes, velocity order of include/lbm.h): rho = sum f, rho u = sum c f.
__global__ void __launch_bounds__(kNaThreads) ke_abs_partial_kernel(const float* __restrict__ f, long long ncell,
                                                                    double* partials) {
    __shared__ double sh[kNaThreads / 32];
    double acc = 0.0;
    const long long base = static_cast<long long>(blockIdx.x) * kNaCellsPerBlock;
    for (int k = 0; k < kNaCellsPerThread; ++k) {
        const long long cell = base + static_cast<long long>(k) * kNaThreads + threadIdx.x;
        if (cell >= ncell) break;
        float rho = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const float v = __ldg(f + static_cast<size_t>(i) * ncell + cell);
            rho += v;
            jx += cx_of(i) * v;
            jy += cy_of(i) * v;
            jz += cz_of(i) * v;
        }
        const double ux = jx / rho, uy = jy / rho, uz = jz / rho;
        acc += 0.5 * (ux * ux + uy * uy + uz * uz);
    }
    acc = na_block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kNaThreads) ke_abs_sum_kernel(const double* partials, int n, double scale,
                                                                double* out) {
    __shared__ double sh[kNaThreads / 32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partials[i];
    acc = na_block_sum(acc, sh);
    if (threadIdx.x == 0) *out = acc * scale;
}

// Device or managed memory that the current device `dev` can address directly: device
// memory must live on `dev` itself (another GPU's memory would fault without peer access).
bool on_device(const void* p, int dev) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace
}  // namespace lbm

extern "C" lbm_status lbm_kinetic_energy_noalloc(const float* f, int nx, int ny, int nz, double* ke, void* stream) {
    using namespace lbm;
    if (!f || !ke || nx < 1 || ny < 1 || nz < 1) return LBM_ERR_ARG;
    const long long ncell = static_cast<long long>(nx) * ny * nz;
    if (ncell > kNaMaxCells) return LBM_ERR_ARG;  // the scratch holds 4096 partials of 4096 cells
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return LBM_ERR_CUDA;
    if (!on_device(f, dev) || !on_device(ke, dev)) return LBM_ERR_ARG;
    cudaError_t e = cudaSuccess;
    double* scratch = scratch_address(dev, &e);
    if (!scratch) return LBM_ERR_CUDA;
    const int blocks = static_cast<int>((ncell + kNaCellsPerBlock - 1) / kNaCellsPerBlock);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ke_abs_partial_kernel<<<blocks, kNaThreads, 0, s>>>(f, ncell, scratch);
    ke_abs_sum_kernel<<<1, kNaThreads, 0, s>>>(scratch, blocks, 1.0 / static_cast<double>(ncell), ke);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
