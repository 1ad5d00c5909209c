// kernels_diag.cu - energy spectrum E(kappa) of the velocity field (Sec. II.D uses it in
// the loss; Sec. III.A plots it): u^ = FFT(u)/N^3 with a mixed radix-2/3 Stockham FFT
// in shared memory (FP32), then |u^|^2/2 binned into integer shells with FP64 atomics.
//
// The FFT is the autosort formulation of Govindaraju et al., "High performance discrete
// Fourier transforms on graphics processors" (SC 2008): stage s with radix R reads
// x[j + r n/R], twiddles by exp(-2 pi i (j mod Ns) r / (Ns R)), applies an R-point DFT
// and writes y[(j / Ns) Ns R + (j mod Ns) + r Ns], Ns being the product of the radices
// of the earlier stages.
#include "cell.cuh"

namespace lbm {

bool fft_size_ok(int n) {
    if (n < 1 || n > 2048) return false;  // two line buffers of n float2 in 32 KB of shared memory
    while (n % 2 == 0) n /= 2;
    if (n % 3 == 0) n /= 3;
    return n == 1;
}

static Dims full_dims(const Dims& d, int bc) {
    const int m = bc == LBM_BC_MIRROR ? 2 : 1;
    Dims f{d.nx * m, d.ny * m, d.nz * m, 0};
    f.ncell = static_cast<long long>(f.nx) * f.ny * f.nz;
    return f;
}

size_t spectrum_work_elems(const Dims& d, int bc) { return 3 * static_cast<size_t>(full_dims(d, bc).ncell); }

// Velocity of every node of the (possibly unfolded) box as complex values, component-major.
// Mirror octants unfold by the Taylor-Green parities: u_a is odd under the reflection of
// axis a and even under the other two.
template <int STORAGE, int BC>
__global__ void build_velocity_kernel(const Dims d, const Dims f, const void* src, float2* work) {
    const long long cell = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (cell >= d.ncell) return;
    int x, y, z;
    cell_coords(cell, d, x, y, z);
    float df[Q], m[Q];
    load_pulled<STORAGE, BC>(src, d, x, y, z, df);
    const float drho = moments_from_dev(df, m);
    const Macro q = macro_from_moments(m, drho);
    const float u[3] = {q.ux, q.uy, q.uz};
    const int reps = BC == LBM_BC_MIRROR ? 8 : 1;
    for (int r = 0; r < reps; ++r) {
        const int mx = r & 1, my = (r >> 1) & 1, mz = (r >> 2) & 1;
        const int X = mx ? f.nx - 1 - x : x, Y = my ? f.ny - 1 - y : y, Z = mz ? f.nz - 1 - z : z;
        const long long o = (static_cast<long long>(Z) * f.ny + Y) * f.nx + X;
        const int flips[3] = {mx, my, mz};
#pragma unroll
        for (int a = 0; a < 3; ++a) work[a * f.ncell + o] = make_float2(flips[a] ? -u[a] : u[a], 0.0f);
    }
}

// One block transforms one line of length n (<= 2048) with the given element stride.
// Line index l enumerates (component, the two other coordinates).
__global__ void fft_line_kernel(float2* data, int n, long long stride, int inner, long long inner_stride,
                                long long outer_stride, int radix_mask, int nstages) {
    extern __shared__ float2 sm[];
    float2* a = sm;
    float2* b = sm + n;
    const long long l = blockIdx.x;
    const long long base = (l % inner) * inner_stride + (l / inner) * outer_stride;
    for (int i = threadIdx.x; i < n; i += blockDim.x) a[i] = data[base + i * stride];
    __syncthreads();
    int Ns = 1;
    for (int s = 0; s < nstages; ++s) {
        const int R = ((radix_mask >> s) & 1) ? 3 : 2;
        const int nb = n / R;
        for (int j = threadIdx.x; j < nb; j += blockDim.x) {
            const int k = j % Ns;
            float2 v[3];
            for (int r = 0; r < R; ++r) v[r] = a[j + r * nb];
            for (int r = 1; r < R; ++r) {
                float sn, cs;
                sincospif(-2.0f * static_cast<float>(k * r) / static_cast<float>(Ns * R), &sn, &cs);
                const float2 t = v[r];
                v[r] = make_float2(t.x * cs - t.y * sn, t.x * sn + t.y * cs);
            }
            float2 V[3];
            if (R == 2) {
                V[0] = make_float2(v[0].x + v[1].x, v[0].y + v[1].y);
                V[1] = make_float2(v[0].x - v[1].x, v[0].y - v[1].y);
            } else {
                // X_p = sum_q v_q exp(-2 pi i p q / 3), exp(-2 pi i/3) = -1/2 - i sqrt3/2
                const float h = 0.8660254037844386f;
                const float2 s12 = make_float2(v[1].x + v[2].x, v[1].y + v[2].y);
                const float2 d12 = make_float2(v[1].x - v[2].x, v[1].y - v[2].y);
                V[0] = make_float2(v[0].x + s12.x, v[0].y + s12.y);
                const float2 m = make_float2(v[0].x - 0.5f * s12.x, v[0].y - 0.5f * s12.y);
                // -i h d12 = (h d12.y, -h d12.x)
                V[1] = make_float2(m.x + h * d12.y, m.y - h * d12.x);
                V[2] = make_float2(m.x - h * d12.y, m.y + h * d12.x);
            }
            const int o = (j / Ns) * Ns * R + k;
            for (int r = 0; r < R; ++r) b[o + r * Ns] = V[r];
        }
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) data[base + i * stride] = a[i];
}

// Shell of an integer |k|^2: the n with n^2 - n + 1 <= k2 <= n^2 + n (nearest integer |k|).
__device__ __forceinline__ int shell_of(long long k2) {
    long long n = static_cast<long long>(sqrt(static_cast<double>(k2)));
    while (n * n + n < k2) ++n;
    while (n > 0 && (n - 1) * (n - 1) + (n - 1) >= k2) --n;
    return static_cast<int>(n);
}

__device__ __forceinline__ int freq(int i, int n) { return i < (n + 1) / 2 ? i : i - n; }

constexpr int kBinThreads = 256;
constexpr int kMaxSmemBins = 1024;

__global__ void __launch_bounds__(kBinThreads) bin_kernel(const Dims f, const float2* work, double* E,
                                                          int nbins, double* total, double inv_n2) {
    __shared__ double sbin[kMaxSmemBins];
    __shared__ double stot;
    const int nb = nbins < kMaxSmemBins ? nbins : kMaxSmemBins;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) sbin[i] = 0.0;
    if (threadIdx.x == 0) stot = 0.0;
    __syncthreads();
    double tacc = 0.0;
    for (long long c = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; c < f.ncell;
         c += static_cast<long long>(gridDim.x) * blockDim.x) {
        int x, y, z;
        cell_coords(c, f, x, y, z);
        const long long kx = freq(x, f.nx), ky = freq(y, f.ny), kz = freq(z, f.nz);
        double e = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float2 v = work[a * f.ncell + c];
            e += static_cast<double>(v.x) * v.x + static_cast<double>(v.y) * v.y;
        }
        e *= 0.5 * inv_n2;
        tacc += e;
        const int s = shell_of(kx * kx + ky * ky + kz * kz);
        if (s < nb) atomicAdd(&sbin[s], e);
        else if (s < nbins) atomicAdd(&E[s], e);
    }
    atomicAdd(&stot, tacc);
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
        if (sbin[i] != 0.0) atomicAdd(&E[i], sbin[i]);
    if (threadIdx.x == 0 && total) atomicAdd(total, stot);
}

// The shell of every wave vector of an nx x ny x nz box in FFT order (x fastest), by the
// same shell_of and freq the binning uses (exported for checks of the binning rule).
__global__ void __launch_bounds__(256) shell_index_kernel(const Dims f, int* out) {
    for (long long c = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; c < f.ncell;
         c += static_cast<long long>(gridDim.x) * blockDim.x) {
        int x, y, z;
        cell_coords(c, f, x, y, z);
        const long long kx = freq(x, f.nx), ky = freq(y, f.ny), kz = freq(z, f.nz);
        out[c] = shell_of(kx * kx + ky * ky + kz * kz);
    }
}

static int radix_mask(int n, int* nst) {
    int mask = 0, s = 0;
    // radix-3 stages first, then radix-2 (any order is valid for the autosort scheme)
    while (n % 3 == 0) { mask |= 1 << s; ++s; n /= 3; }
    while (n % 2 == 0) { ++s; n /= 2; }
    *nst = s;
    return mask;
}

static cudaError_t fft_axis(float2* data, const Dims& f, int axis, cudaStream_t s) {
    int n, inner;
    long long stride, inner_stride, outer_stride;
    const long long nx = f.nx, ny = f.ny, nz = f.nz;
    if (axis == 0) { n = f.nx; stride = 1; inner = f.ny * f.nz * 3; inner_stride = nx; outer_stride = 0; }
    else if (axis == 1) { n = f.ny; stride = nx; inner = f.nx; inner_stride = 1; outer_stride = nx * ny; }
    else { n = f.nz; stride = nx * ny; inner = f.nx * f.ny; inner_stride = 1; outer_stride = nx * ny * nz; }
    if (n == 1) return cudaSuccess;
    int nst = 0;
    const int mask = radix_mask(n, &nst);
    long long lines = 3LL * f.ncell / n;
    if (axis == 0) { inner = static_cast<int>(lines); }
    const int threads = n / 2 < 256 ? (n / 2 < 32 ? 32 : n / 2) : 256;
    const size_t smem = 2 * n * sizeof(float2);
    fft_line_kernel<<<static_cast<unsigned>(lines), threads, smem, s>>>(data, n, stride, inner, inner_stride,
                                                                        outer_stride, mask, nst);
    return cudaGetLastError();
}

namespace {

struct GuardRegions {
    const unsigned char* r[4];
};

// block b checks region b byte by byte
__global__ void __launch_bounds__(256) guard_check_kernel(const GuardRegions g, int* bad) {
    const unsigned char* r = g.r[blockIdx.x];
    int n = 0;
    for (size_t i = threadIdx.x; i < kGuardBytes; i += blockDim.x) n += r[i] != kGuardPattern;
    if (n) atomicAdd(&bad[blockIdx.x], n);
}

}  // namespace

cudaError_t launch_guard_check(const unsigned char* const regions[4], int* bad, cudaStream_t s) {
    const GuardRegions g{{regions[0], regions[1], regions[2], regions[3]}};
    guard_check_kernel<<<4, 256, 0, s>>>(g, bad);
    return cudaGetLastError();
}

cudaError_t launch_spectrum_shells(const Dims& f, int* out, cudaStream_t s) {
    long long blocks = (f.ncell + 255) / 256;
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    shell_index_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(f, out);
    return cudaGetLastError();
}

cudaError_t launch_spectrum(const Dims& d, int storage, int bc, const void* src, float2* work, double* E,
                            int nbins, double* ke, cudaStream_t s) {
    const Dims f = full_dims(d, bc);
    const dim3 grid(static_cast<unsigned>((d.ncell + 127) / 128));
#define LBM_BUILD(S_, B_) build_velocity_kernel<S_, B_><<<grid, 128, 0, s>>>(d, f, src, work)
    if (storage == LBM_STORE_F32) { if (bc == LBM_BC_PERIODIC) LBM_BUILD(LBM_STORE_F32, LBM_BC_PERIODIC); else LBM_BUILD(LBM_STORE_F32, LBM_BC_MIRROR); }
    else if (storage == LBM_STORE_F16_DEV) { if (bc == LBM_BC_PERIODIC) LBM_BUILD(LBM_STORE_F16_DEV, LBM_BC_PERIODIC); else LBM_BUILD(LBM_STORE_F16_DEV, LBM_BC_MIRROR); }
    else { if (bc == LBM_BC_PERIODIC) LBM_BUILD(LBM_STORE_BF16_DEV, LBM_BC_PERIODIC); else LBM_BUILD(LBM_STORE_BF16_DEV, LBM_BC_MIRROR); }
#undef LBM_BUILD
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int ax = 0; ax < 3; ++ax) {
        e = fft_axis(work, f, ax, s);
        if (e != cudaSuccess) return e;
    }
    e = cudaMemsetAsync(E, 0, sizeof(double) * nbins, s);
    if (e != cudaSuccess) return e;
    if (ke) {
        e = cudaMemsetAsync(ke, 0, sizeof(double), s);
        if (e != cudaSuccess) return e;
    }
    const double n = static_cast<double>(f.ncell);
    long long blocks = (f.ncell + kBinThreads - 1) / kBinThreads;
    if (blocks > 152 * 8) blocks = 152 * 8;
    bin_kernel<<<static_cast<unsigned>(blocks), kBinThreads, 0, s>>>(f, work, E, nbins, ke, 1.0 / (n * n));
    return cudaGetLastError();
}

}  // namespace lbm
