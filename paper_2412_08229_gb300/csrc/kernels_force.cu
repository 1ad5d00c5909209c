// kernels_force.cu - Alvelius spectral forcing (Sec. II.C) on the 16 half-space modes with
// 1 <= |k| <= 2 (32 modes with their conjugates).
//
// Per step: (1) force_coeffs turns the projection u^(k) of the previous step's velocity and
// that step's random phases into F^(k); (2) force_synth writes F(x) = sum 2 Re(F^ e^{ik.x});
// (3) the step kernel applies the Kupershtokh source with F and writes its pre-collision
// velocity; (4) force_project forms the FP64 partial sums of u^(k) for the next step.
// Grid coordinates are x_j = 2 pi j / N, u^(k) = N^-3 sum_x u(x) e^{-ik.x}.
#include <cmath>

#include "cell.cuh"

namespace lbm {

ForceModes forced_modes() {
    ForceModes m{};
    int n = 0;
    // sorted by (|k|^2, kz, ky, kx): enumerate |k|^2 = 1..4, then kz, ky, kx ascending
    for (int k2 = 1; k2 <= 4; ++k2)
        for (int kz = -2; kz <= 2; ++kz)
            for (int ky = -2; ky <= 2; ++ky)
                for (int kx = -2; kx <= 2; ++kx) {
                    if (kx * kx + ky * ky + kz * kz != k2) continue;
                    const bool half = kz > 0 || (kz == 0 && ky > 0) || (kz == 0 && ky == 0 && kx > 0);
                    if (!half) continue;
                    if (n < kForcedModes) {
                        m.k[n][0] = kx;
                        m.k[n][1] = ky;
                        m.k[n][2] = kz;
                    }
                    ++n;
                }
    return m;
}

constexpr int kProjThreads = 256;

int force_project_blocks(const Dims& d) {
    long long b = (d.ncell + kProjThreads - 1) / kProjThreads;
    return static_cast<int>(b < 152 ? b : 152);
}

// phase of mode k at cell (x,y,z) in units of pi: 2 (kx x/nx + ky y/ny + kz z/nz) mod 2
__device__ __forceinline__ float phase_pi(const int* k, int x, int y, int z, const Dims& d) {
    double a = static_cast<double>(k[0] * x) / d.nx + static_cast<double>(k[1] * y) / d.ny +
               static_cast<double>(k[2] * z) / d.nz;
    a -= floor(a);
    return static_cast<float>(2.0 * a);
}

// grid (nblocks, 16 modes); partials[(mode * nblocks + block) * 6 + 2a + {0: re, 1: im}]
__global__ void __launch_bounds__(kProjThreads) force_project_kernel(const Dims d, const ForceModes modes,
                                                                     const float* __restrict__ u,
                                                                     double* partials) {
    __shared__ double sh[6][kProjThreads / 32];
    const int mode = blockIdx.y;
    float acc[6] = {0, 0, 0, 0, 0, 0};
    for (long long c = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; c < d.ncell;
         c += static_cast<long long>(gridDim.x) * blockDim.x) {
        int x, y, z;
        cell_coords(c, d, x, y, z);
        float sn, cs;
        sincospif(phase_pi(modes.k[mode], x, y, z, d), &sn, &cs);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float v = u[a * d.ncell + c];
            acc[2 * a] += v * cs;       // Re(u e^{-i phi}) = u cos
            acc[2 * a + 1] -= v * sn;   // Im(u e^{-i phi}) = -u sin
        }
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        double v = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (l == 0) sh[q][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double v = 0.0;
        for (int i = 0; i < (kProjThreads >> 5); ++i) v += sh[threadIdx.x][i];
        partials[(static_cast<long long>(mode) * gridDim.x + blockIdx.x) * 6 + threadIdx.x] = v;
    }
}

cudaError_t launch_force_project(const Dims& d, const float* u, double* partials, int nblocks, cudaStream_t s) {
    force_project_kernel<<<dim3(nblocks, kForcedModes), kProjThreads, 0, s>>>(d, forced_modes(), u, partials);
    return cudaGetLastError();
}

// One thread per mode: F^(k) = A_ran e1 + B_ran e2 (Sec. II.C). Readings: e1 = (ky, -kx, 0)/kh
// (the printed e1 is not normal to k), e1 = (1,0,0) and e2 = (0,1,0) when kx = ky = 0,
// theta1 = atan2(num, den), dt = 1, A from the continuous Gaussian integral over [ka, kb].
__global__ void force_coeffs_kernel(const ForceModes modes, const double* partials, int nblocks,
                                    double inv_cells, const double* phi, const double* psi,
                                    const ForceParams fp, double* fhat) {
    const int m = threadIdx.x;
    if (m >= kForcedModes) return;
    double uh[6];
    for (int q = 0; q < 6; ++q) {
        double v = 0.0;
        for (int b = 0; b < nblocks; ++b) v += partials[(static_cast<long long>(m) * nblocks + b) * 6 + q];
        uh[q] = v * inv_cells;
    }
    const double kx = modes.k[m][0], ky = modes.k[m][1], kz = modes.k[m][2];
    const double kk = sqrt(kx * kx + ky * ky + kz * kz);
    const double kh = sqrt(kx * kx + ky * ky);
    double e1[3], e2[3];
    if (kh == 0.0) {
        e1[0] = 1; e1[1] = 0; e1[2] = 0;
        e2[0] = 0; e2[1] = 1; e2[2] = 0;
    } else {
        e1[0] = ky / kh; e1[1] = -kx / kh; e1[2] = 0.0;
        e2[0] = kx * kz / (kk * kh); e2[1] = ky * kz / (kk * kh); e2[2] = -kh / kk;
    }
    double x1r = 0, x1i = 0, x2r = 0, x2i = 0;
    for (int a = 0; a < 3; ++a) {
        x1r += uh[2 * a] * e1[a];
        x1i += uh[2 * a + 1] * e1[a];
        x2r += uh[2 * a] * e2[a];
        x2i += uh[2 * a + 1] * e2[a];
    }
    const double gA = sin(2.0 * phi[m]), gB = cos(2.0 * phi[m]);
    const double sp = sin(psi[m]), cp = cos(psi[m]);
    const double num = gA * x1r + gB * (sp * x2i + cp * x2r);
    const double den = -gA * x1i + gB * (sp * x2r - cp * x2i);
    const double th1 = atan2(num, den);
    const double th2 = th1 + psi[m];
    const double sc = sqrt(fp.c);
    const double integral = 0.5 * sqrt(3.14159265358979323846 * fp.c) * (erf((fp.kb - fp.kf) / sc) - erf((fp.ka - fp.kf) / sc));
    const double A = fp.power / integral;
    const double Fk = A * exp(-((kk - fp.kf) * (kk - fp.kf)) / fp.c);
    const double amp = sqrt(Fk / (2.0 * 3.14159265358979323846 * kk * kk));
    const double ar = amp * cos(th1) * gA, ai = amp * sin(th1) * gA;
    const double br = amp * cos(th2) * gB, bi = amp * sin(th2) * gB;
    for (int a = 0; a < 3; ++a) {
        fhat[m * 6 + 2 * a] = ar * e1[a] + br * e2[a];
        fhat[m * 6 + 2 * a + 1] = ai * e1[a] + bi * e2[a];
    }
}

cudaError_t launch_force_coeffs(const double* partials, int nblocks, double inv_cells, const double* phi,
                                const double* psi, ForceParams fp, double* fhat, cudaStream_t s) {
    force_coeffs_kernel<<<1, 32, 0, s>>>(forced_modes(), partials, nblocks, inv_cells, phi, psi, fp, fhat);
    return cudaGetLastError();
}

__global__ void force_synth_kernel(const Dims d, const ForceModes modes, const double* __restrict__ fhat,
                                   float* __restrict__ force) {
    __shared__ float fh[kForcedModes * 6];
    for (int i = threadIdx.x; i < kForcedModes * 6; i += blockDim.x) fh[i] = static_cast<float>(fhat[i]);
    __syncthreads();
    const long long c = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (c >= d.ncell) return;
    int x, y, z;
    cell_coords(c, d, x, y, z);
    float F[3] = {0, 0, 0};
#pragma unroll 4
    for (int m = 0; m < kForcedModes; ++m) {
        float sn, cs;
        sincospif(phase_pi(modes.k[m], x, y, z, d), &sn, &cs);
#pragma unroll
        for (int a = 0; a < 3; ++a) F[a] += 2.0f * (fh[m * 6 + 2 * a] * cs - fh[m * 6 + 2 * a + 1] * sn);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) force[a * d.ncell + c] = F[a];
}

cudaError_t launch_force_synth(const Dims& d, const double* fhat, float* force, cudaStream_t s) {
    force_synth_kernel<<<static_cast<unsigned>((d.ncell + 127) / 128), 128, 0, s>>>(d, forced_modes(), fhat, force);
    return cudaGetLastError();
}

}  // namespace lbm
