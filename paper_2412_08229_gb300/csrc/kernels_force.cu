// kernels_force.cu - Alvelius spectral forcing (Sec. II.C) on the 16 half-space modes with
// 1 <= |k| <= 2 (32 modes with their conjugates).
//
// Per step of a single context: (1) force_coeffs turns the projection u^(k) of the previous
// step's velocity and that step's random phases into F^(k) and clears the projection sums;
// (2) the step kernel synthesises F(x) = sum 2 Re(F^ e^{ik.x}) per cell, applies the
// Kupershtokh source and adds its pre-collision velocity's projection to the sums
// (force.cuh). Batches keep a stored force field (force_synth) and a projection pass
// (force_project) around their persistent step kernel. Grid coordinates are x_j = 2 pi j / N,
// u^(k) = N^-3 sum_x u(x) e^{-ik.x}.
// What does not change from step to step is computed once on the host in FP64: the unit
// vectors and amplitude of every mode (force_mode_consts), the per-axis phase factors
// e^{i 2 pi k j / N}, k = 1, 2 (force_phase_table), and, when the draws are queued, the
// sines and cosines of the random phases; the coefficient kernel is then sums, products,
// one square root and divisions.
#include <cmath>
#include <vector>

#include "force.cuh"

namespace lbm {

ForceModes forced_modes() {
    ForceModes m{};
    for (int i = 0; i < kForcedModes; ++i)
        for (int a = 0; a < 3; ++a) m.k[i][a] = kModeTable.k[i][a];
    return m;
}

namespace {
constexpr int kProjThreads = 256;
}  // namespace

void force_phase_table(const Dims& d, float2* out) {
    const int n[3] = {d.nx, d.ny, d.nz};
    int off = 0;
    for (int a = 0; a < 3; ++a) {
        for (int j = 0; j < n[a]; ++j)
            for (int k = 1; k <= 2; ++k) {
                const double ph = 2.0 * 3.14159265358979323846 * static_cast<double>((k * j) % n[a]) / n[a];
                out[off + 2 * j + (k - 1)] = make_float2(static_cast<float>(std::cos(ph)), static_cast<float>(std::sin(ph)));
            }
        off += 2 * n[a];
    }
}

// Per mode (Sec. II.C): the unit vectors e1 = (ky, -kx, 0)/kh (reading: the printed e1 is not
// normal to k), e2 = (kx kz, ky kz, -kh^2)/(|k| kh), e1 = (1,0,0), e2 = (0,1,0) when kx = ky = 0;
// and the amplitude sqrt(F(|k|) / (2 pi |k|^2)), F(k) = A exp(-(k - kf)^2 / c), A = P divided by
// the integral of the Gaussian over [ka, kb] (the continuous integral, reading).
void force_mode_consts(const ForceParams& fp, double* out) {
    const double sc = std::sqrt(fp.c);
    const double integral = 0.5 * std::sqrt(3.14159265358979323846 * fp.c) *
                            (std::erf((fp.kb - fp.kf) / sc) - std::erf((fp.ka - fp.kf) / sc));
    const double A = fp.power / integral;
    for (int m = 0; m < kForcedModes; ++m) {
        const double kx = kModeTable.k[m][0], ky = kModeTable.k[m][1], kz = kModeTable.k[m][2];
        const double kk = std::sqrt(kx * kx + ky * ky + kz * kz), kh = std::sqrt(kx * kx + ky * ky);
        double* o = out + m * kForceConsts;
        if (kh == 0.0) {
            const double e1[3] = {1, 0, 0}, e2[3] = {0, 1, 0};
            for (int a = 0; a < 3; ++a) { o[a] = e1[a]; o[3 + a] = e2[a]; }
        } else {
            o[0] = ky / kh; o[1] = -kx / kh; o[2] = 0.0;
            o[3] = kx * kz / (kk * kh); o[4] = ky * kz / (kk * kh); o[5] = -kh / kk;
        }
        const double Fk = A * std::exp(-((kk - fp.kf) * (kk - fp.kf)) / fp.c);
        o[6] = std::sqrt(Fk / (2.0 * 3.14159265358979323846 * kk * kk));
    }
}

void force_draw_trig(const double* phi, const double* psi, double* row) {
    for (int m = 0; m < kForcedModes; ++m) {
        row[m] = std::sin(2.0 * phi[m]);                      // g_A = sin 2 phi
        row[kForcedModes + m] = std::cos(2.0 * phi[m]);       // g_B = cos 2 phi
        row[2 * kForcedModes + m] = std::sin(psi[m]);
        row[3 * kForcedModes + m] = std::cos(psi[m]);
    }
}

// 2^S with S = 62 - ceil(log2(ncell + 31)): at most ceil(ncell / 32) warp sums of
// magnitude <= 32 each, so every partial sum stays below 2^62.
float force_proj_scale(long long ncell) {
    int bits = 0;
    while ((1LL << bits) < ncell + 31) ++bits;
    return std::ldexp(1.0f, 62 - bits);
}

// The fixed-point sums to u^(k): sum x 2^-S / ncell.
double force_proj_unit(long long ncell) {
    return 1.0 / (static_cast<double>(force_proj_scale(ncell)) * static_cast<double>(ncell));
}

int force_project_blocks(const Dims& d) {
    const long long b = (d.ncell + kProjThreads - 1) / kProjThreads;
    return static_cast<int>(b < 2 * 152 ? (b < 1 ? 1 : b) : 2 * 152);
}

namespace {

// Block b of nb adds the projection of the cells b * 256 + k * nb * 256 + (0..255), read
// from the velocity planes u, to proj (the same fixed-point sums a forced step kernel adds).
__device__ __forceinline__ void project_block(const Dims& d, const float* __restrict__ u, const float2* tab,
                                              unsigned long long* proj, float scale, int b, int nb) {
    __shared__ unsigned long long red[frc::kProjValues];
    for (int i = threadIdx.x; i < frc::kProjValues; i += blockDim.x) red[i] = 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    long long acc[3] = {0, 0, 0};
    for (long long base = static_cast<long long>(b) * kProjThreads; base < d.ncell;
         base += static_cast<long long>(nb) * kProjThreads) {
        const long long c = base + threadIdx.x;
        frc::Cx p[kForcedModes];
        float v[3] = {0.0f, 0.0f, 0.0f};
        int x = 0, y = 0, z = 0;
        if (c < d.ncell) {
            cell_coords(c, d, x, y, z);
            v[0] = u[c];
            v[1] = u[d.ncell + c];
            v[2] = u[2 * d.ncell + c];
        }
        frc::cell_phases(x, y, z, d, tab, p);
        frc::project_warp(v[0], v[1], v[2], p, lane, acc, scale);
    }
    frc::proj_to_shared(red, acc, lane);
    __syncthreads();
    frc::proj_to_global(red, proj);
}

__global__ void __launch_bounds__(kProjThreads) force_project_kernel(const Dims d, const float* __restrict__ u,
                                                                     const float2* tab, unsigned long long* proj,
                                                                     float scale) {
    project_block(d, u, tab, proj, scale, blockIdx.x, gridDim.x);
}

// The projections of several instances: grid (blocks, instances).
__global__ void __launch_bounds__(kProjThreads) force_project_batch_kernel(const ForceBatchItem* items) {
    const ForceBatchItem& it = items[blockIdx.y];
    project_block(it.d, it.u, it.tab, it.proj, it.scale, blockIdx.x, gridDim.x);
}

}  // namespace

cudaError_t launch_force_project(const Dims& d, const float* u, const float2* tab, unsigned long long* proj,
                                 float scale, cudaStream_t s) {
    force_project_kernel<<<force_project_blocks(d), kProjThreads, 0, s>>>(d, u, tab, proj, scale);
    return cudaGetLastError();
}

namespace {

// One thread per mode, from the projection u^(k): F^(k) = A_ran e1 + B_ran e2 (Sec. II.C),
// with the constants of force_mode_consts (k: e1, e2, amp) and a row of draws as
// force_draw_trig lays it out. theta1 = atan2(num, den) (reading; the leading "e" of the
// printed tan theta1 is a typo) enters only through cos theta1 = den / h and sin theta1 =
// num / h, h = |(num, den)| (theta1 = 0 when both vanish), and theta2 = theta1 + psi through
// the angle-sum formulas.
__device__ void force_mode(int m, const double* uh, const double* row, const double* consts, double* fhat) {
    const double* k = consts + m * kForceConsts;
    const double *e1 = k, *e2 = k + 3;
    double x1r = 0, x1i = 0, x2r = 0, x2i = 0;
    for (int a = 0; a < 3; ++a) {
        x1r += uh[2 * a] * e1[a];
        x1i += uh[2 * a + 1] * e1[a];
        x2r += uh[2 * a] * e2[a];
        x2i += uh[2 * a + 1] * e2[a];
    }
    const double gA = row[m], gB = row[kForcedModes + m];
    const double sp = row[2 * kForcedModes + m], cp = row[3 * kForcedModes + m];
    const double num = gA * x1r + gB * (sp * x2i + cp * x2r);
    const double den = -gA * x1i + gB * (sp * x2r - cp * x2i);
    const double h = sqrt(num * num + den * den);
    const double c1 = h > 0.0 ? den / h : 1.0, s1 = h > 0.0 ? num / h : 0.0;
    const double c2 = c1 * cp - s1 * sp, s2 = s1 * cp + c1 * sp;
    const double amp = k[6];
    const double ar = amp * c1 * gA, ai = amp * s1 * gA;
    const double br = amp * c2 * gB, bi = amp * s2 * gB;
    for (int a = 0; a < 3; ++a) {
        fhat[m * 6 + 2 * a] = ar * e1[a] + br * e2[a];
        fhat[m * 6 + 2 * a + 1] = ai * e1[a] + bi * e2[a];
    }
}

// u^(k_m) from the fixed-point sums: uh[2 a + c] = proj[32 a + 2 m + c] * unit.
__device__ __forceinline__ void mode_projection(int m, const unsigned long long* proj, double unit, double* uh) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 2; ++c)
            uh[2 * a + c] = static_cast<double>(static_cast<long long>(proj[32 * a + 2 * m + c])) * unit;
}

constexpr int kCoeffThreads = 128;
static_assert(kCoeffThreads >= frc::kProjValues, "one thread per projection sum clears them");

// Thread m < 16 forms F^ of mode m; after a barrier the sums are cleared for the step that
// follows, and the indexed form advances the device step counter.
__device__ __forceinline__ void coeffs_block(unsigned long long* proj, double unit, const double* row,
                                             const double* consts, double* fhat) {
    const int m = threadIdx.x;
    if (m < kForcedModes) {
        double uh[6];
        mode_projection(m, proj, unit, uh);
        force_mode(m, uh, row, consts, fhat);
    }
    __syncthreads();
    if (threadIdx.x < frc::kProjValues) proj[threadIdx.x] = 0ull;
}

__global__ void __launch_bounds__(kCoeffThreads) force_coeffs_kernel(unsigned long long* proj, double unit,
                                                                     const double* row, const double* consts,
                                                                     double* fhat) {
    coeffs_block(proj, unit, row, consts, fhat);
}

// The row of draws chosen by a device step counter, for CUDA graphs replayed many times:
// row = min(head + *counter, rows - 1); the counter is advanced after it was read.
__global__ void __launch_bounds__(kCoeffThreads) force_coeffs_indexed_kernel(
    unsigned long long* proj, double unit, const double* draws, long long* counter, long long head, long long rows,
    const double* consts, double* fhat) {
    long long row = head + *counter;
    if (row > rows - 1) row = rows - 1;
    coeffs_block(proj, unit, draws + row * kDrawRow, consts, fhat);
    if (threadIdx.x == 0) *counter += 1;
}

// The coefficients of several instances, one block per instance; the draw row is
// head + *counter (clamped to the rows allocated), as for graph replays.
__global__ void __launch_bounds__(kCoeffThreads) force_coeffs_batch_kernel(const ForceBatchItem* items,
                                                                           const long long* counter) {
    const ForceBatchItem& it = items[blockIdx.x];
    long long row = it.head + *counter;
    if (row > it.rows - 1) row = it.rows - 1;
    coeffs_block(it.proj, it.unit, it.draws + row * kDrawRow, it.consts, it.fhat);
}

__global__ void counter_increment_kernel(long long* counter) { *counter += 1; }
__global__ void counter_set_kernel(long long* counter, long long v) { *counter = v; }

}  // namespace

cudaError_t launch_force_coeffs(unsigned long long* proj, double unit, const double* row, const double* consts,
                                double* fhat, cudaStream_t s) {
    force_coeffs_kernel<<<1, kCoeffThreads, 0, s>>>(proj, unit, row, consts, fhat);
    return cudaGetLastError();
}

cudaError_t launch_force_coeffs_indexed(unsigned long long* proj, double unit, const double* draws,
                                        long long* counter, long long head, long long rows, const double* consts,
                                        double* fhat, cudaStream_t s) {
    force_coeffs_indexed_kernel<<<1, kCoeffThreads, 0, s>>>(proj, unit, draws, counter, head, rows, consts, fhat);
    return cudaGetLastError();
}

cudaError_t launch_counter_increment(long long* counter, cudaStream_t s) {
    counter_increment_kernel<<<1, 1, 0, s>>>(counter);
    return cudaGetLastError();
}

cudaError_t launch_counter_set(long long* counter, long long v, cudaStream_t s) {
    counter_set_kernel<<<1, 1, 0, s>>>(counter, v);
    return cudaGetLastError();
}

namespace {

// The stored force field F(x) (3 planes) for the step kernels of batches and the adjoint.
__device__ __forceinline__ void synth_cell(const Dims& d, const float* fh2, const float2* tab,
                                           float* __restrict__ force, long long c) {
    int x, y, z;
    cell_coords(c, d, x, y, z);
    frc::Cx p[kForcedModes];
    frc::cell_phases(x, y, z, d, tab, p);
    float F[3];
    frc::synth_force(fh2, p, F);
#pragma unroll
    for (int a = 0; a < 3; ++a) force[a * d.ncell + c] = F[a];
}

__global__ void __launch_bounds__(128) force_synth_kernel(const Dims d, const double* __restrict__ fhat,
                                                           const float2* tab, float* __restrict__ force) {
    __shared__ float fh2[kForcedModes * 6];
    frc::load_fh2(fhat, fh2);
    __syncthreads();
    const long long c = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (c < d.ncell) synth_cell(d, fh2, tab, force, c);
}

// The force fields of several instances: grid (blocks of the largest, instances).
__global__ void __launch_bounds__(128) force_synth_batch_kernel(const ForceBatchItem* items) {
    const ForceBatchItem& it = items[blockIdx.y];
    if (static_cast<long long>(blockIdx.x) * blockDim.x >= it.d.ncell) return;
    __shared__ float fh2[kForcedModes * 6];
    frc::load_fh2(it.fhat, fh2);
    __syncthreads();
    const long long c = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (c < it.d.ncell) synth_cell(it.d, fh2, it.tab, it.force, c);
}

}  // namespace

cudaError_t launch_force_synth(const Dims& d, const double* fhat, const float2* tab, float* force, cudaStream_t s) {
    force_synth_kernel<<<static_cast<unsigned>((d.ncell + 127) / 128), 128, 0, s>>>(d, fhat, tab, force);
    return cudaGetLastError();
}

cudaError_t launch_force_batch(const ForceBatchItem* d_items, int n, int max_proj_blocks, long long max_cells,
                               const long long* counter, int stage, cudaStream_t s) {
    if (n < 1) return cudaSuccess;
    if (stage == 0) {
        force_coeffs_batch_kernel<<<n, kCoeffThreads, 0, s>>>(d_items, counter);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const unsigned gx = static_cast<unsigned>((max_cells + 127) / 128);
        force_synth_batch_kernel<<<dim3(gx, n), 128, 0, s>>>(d_items);
    } else {
        force_project_batch_kernel<<<dim3(max_proj_blocks, n), kProjThreads, 0, s>>>(d_items);
    }
    return cudaGetLastError();
}

}  // namespace lbm
