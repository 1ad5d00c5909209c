// kernels_force.cu - Alvelius spectral forcing (Sec. II.C) on the 16 half-space modes with
// 1 <= |k| <= 2 (32 modes with their conjugates).
//
// Per step: (1) force_coeffs turns the projection u^(k) of the previous step's velocity and
// that step's random phases into F^(k); (2) force_synth writes F(x) = sum 2 Re(F^ e^{ik.x});
// (3) the step kernel applies the Kupershtokh source with F and writes its pre-collision
// velocity; (4) force_project forms the FP64 partial sums of u^(k) for the next step.
// Grid coordinates are x_j = 2 pi j / N, u^(k) = N^-3 sum_x u(x) e^{-ik.x}.
// What does not change from step to step is computed once on the host in FP64: the unit
// vectors and amplitude of every mode (force_mode_consts), the per-axis phase factors
// e^{i 2 pi k j / N}, k = 1, 2 (force_phase_table), and, when the draws are queued, the
// sines and cosines of the random phases; the coefficient kernel is then sums, products,
// one square root and divisions.
#include <cmath>
#include <vector>

#include "cell.cuh"

namespace lbm {

// The forced modes, sorted by (|k|^2, kz, ky, kx): every integer k in the half space
// (kz > 0, or kz = 0 and ky > 0, or kz = ky = 0 and kx > 0) with 1 <= |k|^2 <= 4.
struct ModeTable {
    int k[kForcedModes][3];
};

constexpr ModeTable make_mode_table() {
    ModeTable m{};
    int n = 0;
    for (int k2 = 1; k2 <= 4; ++k2)
        for (int kz = -2; kz <= 2; ++kz)
            for (int ky = -2; ky <= 2; ++ky)
                for (int kx = -2; kx <= 2; ++kx) {
                    if (kx * kx + ky * ky + kz * kz != k2) continue;
                    const bool half = kz > 0 || (kz == 0 && ky > 0) || (kz == 0 && ky == 0 && kx > 0);
                    if (!half || n >= kForcedModes) continue;
                    m.k[n][0] = kx;
                    m.k[n][1] = ky;
                    m.k[n][2] = kz;
                    ++n;
                }
    return m;
}

constexpr ModeTable kModeTable = make_mode_table();

ForceModes forced_modes() {
    ForceModes m{};
    for (int i = 0; i < kForcedModes; ++i)
        for (int a = 0; a < 3; ++a) m.k[i][a] = kModeTable.k[i][a];
    return m;
}

namespace {

constexpr int kProjThreads = 256;
constexpr int kProjCellsPerThread = 4;  // cells per thread between the block reductions

struct Cx {
    float re, im;
};

__device__ __forceinline__ Cx cmul(Cx a, Cx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }

// exp(i 2 pi k j / n) for k = 1, 2 along one axis, from the axis's phase table
__device__ __forceinline__ void axis_phases(const float2* tab, int j, Cx& e1, Cx& e2) {
    const float2 a = __ldg(&tab[2 * j]), b = __ldg(&tab[2 * j + 1]);
    e1 = Cx{a.x, a.y};
    e2 = Cx{b.x, b.y};
}

// exp(i K 2 pi j / n) from the axis table: K in -2..2, 0 -> not a factor
template <int K>
__device__ __forceinline__ Cx axis_factor(const Cx& e1, const Cx& e2) {
    if constexpr (K == 1) return e1;
    else if constexpr (K == 2) return e2;
    else if constexpr (K == -1) return Cx{e1.re, -e1.im};
    else return Cx{e2.re, -e2.im};
}

// exp(i k_m . x) for mode M, x_j = 2 pi j / n per axis (Sec. II.C), as a product of the
// per-axis factors: the phases of all 16 modes cost 6 sincospif per cell
template <int M>
__device__ __forceinline__ Cx mode_phase(const Cx* ex, const Cx* ey, const Cx* ez) {
    constexpr int kx = kModeTable.k[M][0], ky = kModeTable.k[M][1], kz = kModeTable.k[M][2];
    Cx p{1.0f, 0.0f};
    bool first = true;
    if constexpr (kx != 0) {
        p = axis_factor<kx>(ex[0], ex[1]);
        first = false;
    }
    if constexpr (ky != 0) {
        const Cx f = axis_factor<ky>(ey[0], ey[1]);
        p = first ? f : cmul(p, f);
        first = false;
    }
    if constexpr (kz != 0) {
        const Cx f = axis_factor<kz>(ez[0], ez[1]);
        p = first ? f : cmul(p, f);
    }
    return p;
}

// tab: the phase tables of the x, y and z axes one after another (2 entries per node)
__device__ __forceinline__ void cell_axis_phases(long long c, const Dims& d, const float2* tab, Cx* ex, Cx* ey,
                                                 Cx* ez) {
    int x, y, z;
    cell_coords(c, d, x, y, z);
    axis_phases(tab, x, ex[0], ex[1]);
    axis_phases(tab + 2 * d.nx, y, ey[0], ey[1]);
    axis_phases(tab + 2 * (d.nx + d.ny), z, ez[0], ez[1]);
}

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

int force_project_blocks(const Dims& d) {
    const long long per_block = static_cast<long long>(kProjThreads) * kProjCellsPerThread;
    const long long b = (d.ncell + per_block - 1) / per_block;
    return static_cast<int>(b < 2 * 152 ? (b < 1 ? 1 : b) : 2 * 152);
}

// One pass over the cells for all 16 modes by block b of nb: partials[(mode * nb + b) * 6 +
// 2a + {0: re, 1: im}] of u_a(x) e^{-i k.x}. FP32 per thread, FP32 warp sums, FP64 across
// warps (and, in force_coeffs, across blocks).
__device__ __forceinline__ void project_block(const Dims& d, const float* __restrict__ u, const float2* tab,
                                              double* partials, int b, int nb) {
    __shared__ double sh[kProjThreads / 32][kForcedModes * 6];
    float acc[kForcedModes * 6];
#pragma unroll
    for (int q = 0; q < kForcedModes * 6; ++q) acc[q] = 0.0f;
    for (long long c = static_cast<long long>(b) * kProjThreads + threadIdx.x; c < d.ncell;
         c += static_cast<long long>(nb) * kProjThreads) {
        Cx ex[2], ey[2], ez[2];
        cell_axis_phases(c, d, tab, ex, ey, ez);
        const float v[3] = {u[c], u[d.ncell + c], u[2 * d.ncell + c]};
        static_for<kForcedModes>([&](auto Mc) {
            constexpr int m = decltype(Mc)::value;
            const Cx p = mode_phase<m>(ex, ey, ez);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                acc[m * 6 + 2 * a] = fmaf(v[a], p.re, acc[m * 6 + 2 * a]);          // Re(u e^{-i phi})
                acc[m * 6 + 2 * a + 1] = fmaf(-v[a], p.im, acc[m * 6 + 2 * a + 1]); // Im(u e^{-i phi})
            }
        });
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < kForcedModes * 6; ++q) {
        float v = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (l == 0) sh[w][q] = v;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kForcedModes * 6; q += blockDim.x) {
        double v = 0.0;
        for (int i = 0; i < (kProjThreads >> 5); ++i) v += sh[i][q];
        const int m = q / 6, j = q % 6;
        partials[(static_cast<long long>(m) * nb + b) * 6 + j] = v;
    }
}

__global__ void __launch_bounds__(kProjThreads) force_project_kernel(const Dims d, const float* __restrict__ u,
                                                                     const float2* tab, double* partials) {
    project_block(d, u, tab, partials, blockIdx.x, gridDim.x);
}

// The projections of several instances: grid (max blocks, instances), idle blocks return.
__global__ void __launch_bounds__(kProjThreads) force_project_batch_kernel(const ForceBatchItem* items) {
    const ForceBatchItem& it = items[blockIdx.y];
    if (static_cast<int>(blockIdx.x) >= it.nblocks) return;
    project_block(it.d, it.u, it.tab, it.partials, blockIdx.x, it.nblocks);
}

cudaError_t launch_force_project(const Dims& d, const float* u, const float2* tab, double* partials, int nblocks,
                                 cudaStream_t s) {
    force_project_kernel<<<nblocks, kProjThreads, 0, s>>>(d, u, tab, partials);
    return cudaGetLastError();
}

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

// u^(k_m) = inv_cells * (sum of the block partials of mode m), summed by one warp in a
// fixed order (lane-strided, then a butterfly), so every lane holds the same bits.
__device__ __forceinline__ void mode_projection(int m, const double* partials, int nblocks, double inv_cells,
                                                int lane, double* uh) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        double v = 0.0;
        for (int b = lane; b < nblocks; b += 32) v += partials[(static_cast<long long>(m) * nblocks + b) * 6 + q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        uh[q] = v * inv_cells;
    }
}

constexpr int kCoeffThreads = 32 * kForcedModes;  // one warp per mode

__global__ void __launch_bounds__(kCoeffThreads) force_coeffs_kernel(const double* partials, int nblocks,
                                                                     double inv_cells, const double* row,
                                                                     const double* consts, double* fhat) {
    const int m = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double uh[6];
    mode_projection(m, partials, nblocks, inv_cells, lane, uh);
    if (lane == 0) force_mode(m, uh, row, consts, fhat);
}

cudaError_t launch_force_coeffs(const double* partials, int nblocks, double inv_cells, const double* row,
                                const double* consts, double* fhat, cudaStream_t s) {
    force_coeffs_kernel<<<1, kCoeffThreads, 0, s>>>(partials, nblocks, inv_cells, row, consts, fhat);
    return cudaGetLastError();
}

// The same with the row of draws chosen by a device step counter, for CUDA graphs replayed
// many times: row = min(head + *counter, rows - 1).
__global__ void __launch_bounds__(kCoeffThreads) force_coeffs_indexed_kernel(
    const double* partials, int nblocks, double inv_cells, const double* draws, const long long* counter,
    long long head, long long rows, const double* consts, double* fhat) {
    const int m = threadIdx.x >> 5, lane = threadIdx.x & 31;
    long long row = head + *counter;
    if (row > rows - 1) row = rows - 1;
    double uh[6];
    mode_projection(m, partials, nblocks, inv_cells, lane, uh);
    if (lane == 0) force_mode(m, uh, draws + row * kDrawRow, consts, fhat);
}

cudaError_t launch_force_coeffs_indexed(const double* partials, int nblocks, double inv_cells, const double* draws,
                                        const long long* counter, long long head, long long rows,
                                        const double* consts, double* fhat, cudaStream_t s) {
    force_coeffs_indexed_kernel<<<1, kCoeffThreads, 0, s>>>(partials, nblocks, inv_cells, draws, counter, head, rows,
                                                            consts, fhat);
    return cudaGetLastError();
}

// The coefficients of several instances, one block per instance; the draw row is
// head + *counter (clamped to the rows allocated), as for graph replays.
__global__ void __launch_bounds__(kCoeffThreads) force_coeffs_batch_kernel(const ForceBatchItem* items,
                                                                           const long long* counter) {
    const ForceBatchItem& it = items[blockIdx.x];
    const int m = threadIdx.x >> 5, lane = threadIdx.x & 31;
    long long row = it.head + *counter;
    if (row > it.rows - 1) row = it.rows - 1;
    double uh[6];
    mode_projection(m, it.partials, it.nblocks, it.inv_cells, lane, uh);
    if (lane == 0) force_mode(m, uh, it.draws + row * kDrawRow, it.consts, it.fhat);
}

__global__ void counter_increment_kernel(long long* counter) { *counter += 1; }
__global__ void counter_set_kernel(long long* counter, long long v) { *counter = v; }

cudaError_t launch_counter_increment(long long* counter, cudaStream_t s) {
    counter_increment_kernel<<<1, 1, 0, s>>>(counter);
    return cudaGetLastError();
}

cudaError_t launch_counter_set(long long* counter, long long v, cudaStream_t s) {
    counter_set_kernel<<<1, 1, 0, s>>>(counter, v);
    return cudaGetLastError();
}

// F(x) = sum_m 2 Re(F^_m e^{i k_m . x}) at cell c (fh: F^ as floats in shared memory)
__device__ __forceinline__ void synth_cell(const Dims& d, const float* fh, const float2* tab, float* __restrict__ force,
                                           long long c) {
    Cx ex[2], ey[2], ez[2];
    cell_axis_phases(c, d, tab, ex, ey, ez);
    float F[3] = {0, 0, 0};
    static_for<kForcedModes>([&](auto Mc) {
        constexpr int m = decltype(Mc)::value;
        const Cx p = mode_phase<m>(ex, ey, ez);
#pragma unroll
        for (int a = 0; a < 3; ++a) F[a] += 2.0f * (fh[m * 6 + 2 * a] * p.re - fh[m * 6 + 2 * a + 1] * p.im);
    });
#pragma unroll
    for (int a = 0; a < 3; ++a) force[a * d.ncell + c] = F[a];
}

__global__ void __launch_bounds__(128) force_synth_kernel(const Dims d, const double* __restrict__ fhat,
                                                           const float2* tab, float* __restrict__ force) {
    __shared__ float fh[kForcedModes * 6];
    for (int i = threadIdx.x; i < kForcedModes * 6; i += blockDim.x) fh[i] = static_cast<float>(fhat[i]);
    __syncthreads();
    const long long c = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (c < d.ncell) synth_cell(d, fh, tab, force, c);
}

// The force fields of several instances: grid (blocks of the largest, instances).
__global__ void __launch_bounds__(128) force_synth_batch_kernel(const ForceBatchItem* items) {
    const ForceBatchItem& it = items[blockIdx.y];
    if (static_cast<long long>(blockIdx.x) * blockDim.x >= it.d.ncell) return;
    __shared__ float fh[kForcedModes * 6];
    for (int i = threadIdx.x; i < kForcedModes * 6; i += blockDim.x) fh[i] = static_cast<float>(it.fhat[i]);
    __syncthreads();
    const long long c = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (c < it.d.ncell) synth_cell(it.d, fh, it.tab, it.force, c);
}

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
