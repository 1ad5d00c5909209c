// kernels_step.cu - the fused pull-stream-collide step (Sec. II.A-B) with the BGK, KBC
// and FP32 neural-collision operators, plus state set/get, macroscopic fields and the
// FP64 kinetic-energy reduction.
//
// One thread per cell; consecutive threads take consecutive x, so every one of the 27
// population loads and stores of a warp is a contiguous run of one plane (shifted by
// c_x for the loads). In the pull scheme every stored value is read exactly once per
// step, so there is no reuse for shared-memory staging to capture; the +-1 shift along
// x is absorbed by L1/L2 sectors that neighbouring warps share.
#include <atomic>

#include "force.cuh"
#include "internal.h"

namespace lbm {

constexpr int kStepThreads = 128;

// ---------------------------------------------------------------------------
// FP32 invariant network N_Phi (Sec. II.B, eq. gconv_m) evaluated per cell.
// The 48 elements of O_h are (axis permutation p, sign vector s). For element (p, s)
// the network input in the printed moment order is P_g m; with the columns of W1
// rearranged per p (W1p, built on the host from the group tables) the first layer
// reads sgn(s, t) * m_t in tensor order t, where sgn flips the moments that are odd
// in a reflected axis: sgn(s, t) = (-1)^popcount(s & c(t)) with c(t) the parity class of
// t (which axes t is odd in). Grouping the first layer's sum by class, the 8 sign
// vectors of one permutation are an 8-point Walsh-Hadamard transform of the 8 class
// sums y_c = sum_{t in class c} W1p[:, t] m_t: 20 x 27 MAC and 20 x 24 additions per
// permutation instead of 8 x 20 x 27 MAC. The relu'd first-layer outputs of the 8 sign
// vectors are staged in shared memory, one column per thread, and read back per sign
// vector for the layers after it. The output layer is affine, so the group mean is taken
// on the last hidden layer first (h2, or h3 for the 1484-parameter network with a third
// hidden layer).
// ---------------------------------------------------------------------------
constexpr int kNcoThreads = 64;  // block of the FP32 network kernel: 8 x 20 x 64 floats of staging

__device__ __forceinline__ int odd_mask(int t) {
    return ((ex_of(t) == 1) << 2) | ((ey_of(t) == 1) << 1) | (ez_of(t) == 1);
}

__device__ __forceinline__ void nco_rates_f32(const float* m, const NetParams& net, float* rates) {
    __shared__ float h1s[8 * kHidden * kNcoThreads];  // [s][j][thread]: each thread its own column
    float* col = h1s + threadIdx.x;
    float acc[kHidden];
#pragma unroll
    for (int j = 0; j < kHidden; ++j) acc[j] = 0.0f;
#pragma unroll 1
    for (int p = 0; p < 6; ++p) {
#pragma unroll
        for (int j = 0; j < kHidden; ++j) {
            float y[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) y[c] = 0.0f;
#pragma unroll
            for (int t = 0; t < Q; ++t) y[odd_mask(t)] = fmaf(net.W1p[p][j][t], m[t], y[odd_mask(t)]);
            // H[s] = sum_c (-1)^popcount(s & c) y[c], in place
#pragma unroll
            for (int bit = 1; bit < 8; bit <<= 1)
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    if (!(c & bit)) {
                        const float u = y[c], v = y[c | bit];
                        y[c] = u + v;
                        y[c | bit] = u - v;
                    }
#pragma unroll
            for (int sv = 0; sv < 8; ++sv) col[(sv * kHidden + j) * kNcoThreads] = fmaxf(y[sv] + net.b1[j], 0.0f);
        }
#pragma unroll 1
        for (int sv = 0; sv < 8; ++sv) {
            float h1[kHidden];
#pragma unroll
            for (int j = 0; j < kHidden; ++j) h1[j] = col[(sv * kHidden + j) * kNcoThreads];
            if (net.deep) {  // 27-20-20-20-4: a third hidden layer before the group sum
                float h2[kHidden];
#pragma unroll
                for (int j = 0; j < kHidden; ++j) {
                    float a = net.b2[j];
#pragma unroll
                    for (int k = 0; k < kHidden; ++k) a = fmaf(net.W2[j][k], h1[k], a);
                    h2[j] = fmaxf(a, 0.0f);
                }
#pragma unroll
                for (int j = 0; j < kHidden; ++j) {
                    float a = net.bd[j];
#pragma unroll
                    for (int k = 0; k < kHidden; ++k) a = fmaf(net.Wd[j][k], h2[k], a);
                    acc[j] += fmaxf(a, 0.0f);
                }
            } else {
#pragma unroll
                for (int j = 0; j < kHidden; ++j) {
                    float a = net.b2[j];
#pragma unroll
                    for (int k = 0; k < kHidden; ++k) a = fmaf(net.W2[j][k], h1[k], a);
                    acc[j] += fmaxf(a, 0.0f);
                }
            }
        }
    }
#pragma unroll
    for (int n = 0; n < kOut; ++n) {
        float a = 0.0f;
#pragma unroll
        for (int j = 0; j < kHidden; ++j) a = fmaf(net.W3[n][j], acc[j], a);
        rates[n] = rate_from_output(a * (1.0f / 48.0f) + net.b3[n]);
    }
}

// Collision of one cell's pulled deviations df, in place; reports a density outside the
// window and returns the cell's pre-collision macroscopic state.
template <int OP>
__device__ __forceinline__ Macro collide_cell(const StepArgs& a, float* df, const NetParams* net) {
    Macro q;
    if constexpr (OP == LBM_OP_KBC) {  // needs only rho, u and the second-order moments
        float s2[6];
        q = kbc_moments(df, s2);
        if (!(q.rho >= a.rho_min && q.rho <= a.rho_max)) atomicOr(a.status, 1);
        collide_kbc(df, s2, q, a.tau);
    } else {
        float m[Q];
        const float drho = moments_from_dev(df, m);
        q = macro_from_moments(m, drho);
        if (!(q.rho >= a.rho_min && q.rho <= a.rho_max)) atomicOr(a.status, 1);
        const float omega = 1.0f / a.tau;
        if constexpr (OP == LBM_OP_BGK) {
            collide_bgk(df, q, omega);
        } else if constexpr (OP == LBM_OP_REG) {  // orders 3..6 relaxed with rate 1
            const float ones[kOut] = {1.0f, 1.0f, 1.0f, 1.0f};
            collide_mrt(df, m, q, omega, ones);
        } else {
            float rates[kOut];
            nco_rates_f32(m, *net, rates);
            collide_mrt(df, m, q, omega, rates);
        }
    }
    return q;
}

template <int OP, int STORAGE, int BC>
__device__ __forceinline__ void step_body(const StepArgs& a, const NetParams* net) {
    const long long cell = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (cell >= a.d.ncell) return;
    int x, y, z;
    cell_coords(cell, a.d, x, y, z);
    float df[Q];
    load_pulled_offsets<STORAGE, BC>(a.src, a.d, x, y, z, df);
    collide_cell<OP>(a, df, net);
    store_cell<STORAGE>(a.dst, a.d, cell, df);
}

// The forced step (Sec. II.A source, Sec. II.C force) on a grid that strides over the
// cells: per cell the force F(x) is synthesised from the step's 16 coefficients and the
// phase tables and added as the Kupershtokh source after the collision, and the
// pre-collision velocity is added to the fixed-point projection sums of the next step's
// coefficients (force.cuh). Every lane of a warp takes part in the projection; lanes past
// the last cell contribute zero.
template <int OP, int STORAGE, int BC>
__device__ __forceinline__ void step_body_forced(const StepArgs& a, const FusedForce& ff, const NetParams* net) {
    __shared__ float fh2[kForcedModes * 6];
    __shared__ unsigned long long red[frc::kProjValues];
    frc::load_fh2(ff.fhat, fh2);
    for (int i = threadIdx.x; i < frc::kProjValues; i += blockDim.x) red[i] = 0ull;
    __syncthreads();
    const bool project = ff.proj != nullptr;
    const int lane = threadIdx.x & 31;
    long long acc[3] = {0, 0, 0};
    for (long long base = static_cast<long long>(blockIdx.x) * blockDim.x; base < a.d.ncell;
         base += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long cell = base + threadIdx.x;
        const bool valid = cell < a.d.ncell;
        int x = 0, y = 0, z = 0;
        float df[Q];
        Macro q{};
        if (valid) {
            cell_coords(cell, a.d, x, y, z);
            load_pulled_offsets<STORAGE, BC>(a.src, a.d, x, y, z, df);
            q = collide_cell<OP>(a, df, net);
        }
        frc::Cx p[kForcedModes];
        frc::cell_phases(x, y, z, a.d, ff.tab, p);
        if (valid) {
            float F[3];
            frc::synth_force(fh2, p, F);
            add_kupershtokh(df, q, F[0], F[1], F[2]);
            store_cell<STORAGE>(a.dst, a.d, cell, df);
        }
        if (project) frc::project_warp(q.ux, q.uy, q.uz, p, lane, acc, ff.scale);
    }
    if (project) {
        frc::proj_to_shared(red, acc, lane);
        __syncthreads();
        frc::proj_to_global(red, ff.proj);
    }
}

template <int OP, int STORAGE, int BC, bool FORCED>
__global__ void __launch_bounds__(kStepThreads, OP == LBM_OP_KBC && !FORCED ? 7 : 1)
    step_kernel(const StepArgs a, const FusedForce ff) {
    if constexpr (FORCED) step_body_forced<OP, STORAGE, BC>(a, ff, nullptr);
    else step_body<OP, STORAGE, BC>(a, nullptr);
}

template <int STORAGE, int BC, bool FORCED>
__global__ void __launch_bounds__(kNcoThreads) step_nco_f32_kernel(const StepArgs a,
                                                                    const __grid_constant__ NetParams net,
                                                                    const FusedForce ff) {
    if constexpr (FORCED) step_body_forced<LBM_OP_NCO, STORAGE, BC>(a, ff, &net);
    else step_body<LBM_OP_NCO, STORAGE, BC>(a, &net);
}

// Blocks of a forced launch: as many as are resident at once (the grid strides over the
// cells), at most one per 128 cells.
template <typename K>
static unsigned forced_grid(K kernel, int threads, std::atomic<int>& occ, long long ncell) {
    int n = occ.load(std::memory_order_relaxed);
    if (n == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, 0) != cudaSuccess || n < 1) {
            cudaGetLastError();
            n = 1;
        }
        occ.store(n, std::memory_order_relaxed);
    }
    const long long need = (ncell + threads - 1) / threads;
    const long long res = static_cast<long long>(n) * sm_count();
    return static_cast<unsigned>(need < res ? need : res);
}

template <int OP, int STORAGE, int BC, bool FORCED>
static cudaError_t launch_op(const StepArgs& a, const FusedForce& ff, cudaStream_t s) {
    unsigned grid = static_cast<unsigned>((a.d.ncell + kStepThreads - 1) / kStepThreads);
    if constexpr (FORCED) {
        static std::atomic<int> occ{0};
        grid = forced_grid(step_kernel<OP, STORAGE, BC, true>, kStepThreads, occ, a.d.ncell);
    }
    step_kernel<OP, STORAGE, BC, FORCED><<<grid, kStepThreads, 0, s>>>(a, ff);
    return cudaGetLastError();
}

template <int STORAGE, int BC, bool FORCED>
static cudaError_t launch_step_t(const StepArgs& a, const FusedForce& ff, int op, const NetParams* net,
                                 cudaStream_t s) {
    if (op == LBM_OP_BGK) return launch_op<LBM_OP_BGK, STORAGE, BC, FORCED>(a, ff, s);
    if (op == LBM_OP_KBC) return launch_op<LBM_OP_KBC, STORAGE, BC, FORCED>(a, ff, s);
    if (op == LBM_OP_REG) return launch_op<LBM_OP_REG, STORAGE, BC, FORCED>(a, ff, s);
    unsigned grid = static_cast<unsigned>((a.d.ncell + kNcoThreads - 1) / kNcoThreads);
    if constexpr (FORCED) {
        static std::atomic<int> occ{0};
        grid = forced_grid(step_nco_f32_kernel<STORAGE, BC, true>, kNcoThreads, occ, a.d.ncell);
    }
    step_nco_f32_kernel<STORAGE, BC, FORCED><<<grid, kNcoThreads, 0, s>>>(a, *net, ff);
    return cudaGetLastError();
}

// Forcing runs on periodic boxes only (contexts refuse it on the other boundaries).
template <int STORAGE>
static cudaError_t launch_step_s(const StepArgs& a, const FusedForce* ff, int op, int bc, const NetParams* net,
                                 cudaStream_t s) {
    const FusedForce none{};
    if (ff) {
        if (bc != LBM_BC_PERIODIC) return cudaErrorInvalidValue;
        return launch_step_t<STORAGE, LBM_BC_PERIODIC, true>(a, *ff, op, net, s);
    }
    if (bc == LBM_BC_PERIODIC) return launch_step_t<STORAGE, LBM_BC_PERIODIC, false>(a, none, op, net, s);
    if (bc == LBM_BC_TGV_REDUCED) return launch_step_t<STORAGE, LBM_BC_TGV_REDUCED, false>(a, none, op, net, s);
    return launch_step_t<STORAGE, LBM_BC_MIRROR, false>(a, none, op, net, s);
}

cudaError_t launch_step(const StepArgs& a, const FusedForce* ff, int op, int storage, int bc, int net_prec,
                        const NetParams* net, const void* tc_weights, int tc_shape, long long wait_cycles,
                        cudaStream_t s) {
    if (op == LBM_OP_NCO && net_prec == LBM_NET_BF16)
        return launch_step_nco_tc(a, ff, storage, bc, net && net->deep, tc_shape, wait_cycles, tc_weights, s);
    if (op == LBM_OP_NCO && net_prec == LBM_NET_BF16X3)
        return launch_step_nco_tc3(a, ff, storage, bc, net && net->deep, tc_weights, wait_cycles, s);
    switch (storage) {
        case LBM_STORE_F32: return launch_step_s<LBM_STORE_F32>(a, ff, op, bc, net, s);
        case LBM_STORE_F16_DEV: return launch_step_s<LBM_STORE_F16_DEV>(a, ff, op, bc, net, s);
        default: return launch_step_s<LBM_STORE_BF16_DEV>(a, ff, op, bc, net, s);
    }
}

// ---------------------------------------------------------------------------
// State initialisation and access. The stored buffer holds post-collision values
// f*(x, t-1); the pre-collision state is f_i(x, t) = f*_{ip}(src(x, i)), the pull map.
// Writing a given state scatters through the same map (a bijection), so reading it
// back is exact.
// ---------------------------------------------------------------------------
template <int STORAGE, int BC>
__global__ void init_eq_kernel(const Dims d, const float* __restrict__ rho, const float* __restrict__ u,
                               void* dst) {
    const long long cell = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (cell >= d.ncell) return;
    int x, y, z;
    cell_coords(cell, d, x, y, z);
    Macro q;
    q.rho = rho[cell];
    q.drho = q.rho - 1.0f;
    q.ux = u[cell];
    q.uy = u[d.ncell + cell];
    q.uz = u[2 * d.ncell + cell];
    using S = Store<STORAGE>;
    typename S::T* base = static_cast<typename S::T*>(dst);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        int ip, s;
        pull_source<BC>(x, y, z, i, d, ip, s);
        S::st(base + static_cast<size_t>(ip) * d.ncell + s, feq_dev(i, q));
    }
}

template <int STORAGE, int BC>
__global__ void set_state_kernel(const Dims d, const float* __restrict__ f, void* dst) {
    const long long cell = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (cell >= d.ncell) return;
    int x, y, z;
    cell_coords(cell, d, x, y, z);
    using S = Store<STORAGE>;
    typename S::T* base = static_cast<typename S::T*>(dst);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        int ip, s;
        pull_source<BC>(x, y, z, i, d, ip, s);
        S::st(base + static_cast<size_t>(ip) * d.ncell + s, f[static_cast<size_t>(i) * d.ncell + cell] - wgt(i));
    }
}

template <int STORAGE, int BC>
__global__ void get_state_kernel(const Dims d, const void* src, float* __restrict__ f) {
    const long long cell = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (cell >= d.ncell) return;
    int x, y, z;
    cell_coords(cell, d, x, y, z);
    float df[Q];
    load_pulled<STORAGE, BC>(src, d, x, y, z, df);
#pragma unroll
    for (int i = 0; i < Q; ++i) f[static_cast<size_t>(i) * d.ncell + cell] = wgt(i) + df[i];
}

template <int STORAGE, int BC>
__global__ void macroscopic_kernel(const Dims d, const void* src, float* __restrict__ rho,
                                   float* __restrict__ u) {
    const long long cell = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (cell >= d.ncell) return;
    int x, y, z;
    cell_coords(cell, d, x, y, z);
    float df[Q], m[Q];
    load_pulled<STORAGE, BC>(src, d, x, y, z, df);
    const float drho = moments_from_dev(df, m);
    const Macro q = macro_from_moments(m, drho);
    if (rho) rho[cell] = q.rho;
    if (u) {
        u[cell] = q.ux;
        u[d.ncell + cell] = q.uy;
        u[2 * d.ncell + cell] = q.uz;
    }
}

// k = (1/2) <|u|^2>: per-block FP64 partial sums, then one block adds the partials.
constexpr int kKeThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    v = 0.0;
    if (threadIdx.x < (blockDim.x >> 5)) v = sh[threadIdx.x];
    if (w == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

template <int STORAGE, int BC>
__global__ void __launch_bounds__(kKeThreads) ke_partial_kernel(const Dims d, const void* src,
                                                                double* partials) {
    __shared__ double sh[kKeThreads / 32];
    double acc = 0.0;
    for (long long cell = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; cell < d.ncell;
         cell += static_cast<long long>(gridDim.x) * blockDim.x) {
        int x, y, z;
        cell_coords(cell, d, x, y, z);
        float df[Q], m[Q];
        load_pulled<STORAGE, BC>(src, d, x, y, z, df);
        const float drho = moments_from_dev(df, m);
        const Macro q = macro_from_moments(m, drho);
        acc += 0.5 * (static_cast<double>(q.ux) * q.ux + static_cast<double>(q.uy) * q.uy +
                      static_cast<double>(q.uz) * q.uz);
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kKeThreads) sum_partials_kernel(const double* partials, int n,
                                                                  double scale, double* out) {
    __shared__ double sh[kKeThreads / 32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partials[i];
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) *out = acc * scale;
}

int kinetic_energy_blocks(const Dims& d) {
    const long long need = (d.ncell + kKeThreads - 1) / kKeThreads;
    return static_cast<int>(need < 152 * 8 ? need : 152 * 8);
}

// --- dispatch helpers --------------------------------------------------------
#define LBM_DISPATCH_SB(storage, bc, KERNEL_CALL)                                              \
    do {                                                                                       \
        if (storage == LBM_STORE_F32) {                                                        \
            if (bc == LBM_BC_PERIODIC) { constexpr int S_ = LBM_STORE_F32, B_ = LBM_BC_PERIODIC; KERNEL_CALL; } \
            else if (bc == LBM_BC_TGV_REDUCED) { constexpr int S_ = LBM_STORE_F32, B_ = LBM_BC_TGV_REDUCED; KERNEL_CALL; } \
            else { constexpr int S_ = LBM_STORE_F32, B_ = LBM_BC_MIRROR; KERNEL_CALL; }        \
        } else if (storage == LBM_STORE_F16_DEV) {                                             \
            if (bc == LBM_BC_PERIODIC) { constexpr int S_ = LBM_STORE_F16_DEV, B_ = LBM_BC_PERIODIC; KERNEL_CALL; } \
            else if (bc == LBM_BC_TGV_REDUCED) { constexpr int S_ = LBM_STORE_F16_DEV, B_ = LBM_BC_TGV_REDUCED; KERNEL_CALL; } \
            else { constexpr int S_ = LBM_STORE_F16_DEV, B_ = LBM_BC_MIRROR; KERNEL_CALL; }    \
        } else {                                                                               \
            if (bc == LBM_BC_PERIODIC) { constexpr int S_ = LBM_STORE_BF16_DEV, B_ = LBM_BC_PERIODIC; KERNEL_CALL; } \
            else if (bc == LBM_BC_TGV_REDUCED) { constexpr int S_ = LBM_STORE_BF16_DEV, B_ = LBM_BC_TGV_REDUCED; KERNEL_CALL; } \
            else { constexpr int S_ = LBM_STORE_BF16_DEV, B_ = LBM_BC_MIRROR; KERNEL_CALL; }   \
        }                                                                                      \
    } while (0)

static dim3 cell_grid(const Dims& d, int threads) {
    return dim3(static_cast<unsigned>((d.ncell + threads - 1) / threads));
}

cudaError_t launch_init_eq(const Dims& d, int storage, int bc, const float* rho, const float* u,
                           void* dst, cudaStream_t s) {
    LBM_DISPATCH_SB(storage, bc, (init_eq_kernel<S_, B_><<<cell_grid(d, 128), 128, 0, s>>>(d, rho, u, dst)));
    return cudaGetLastError();
}

cudaError_t launch_set_state(const Dims& d, int storage, int bc, const float* f, void* dst, cudaStream_t s) {
    LBM_DISPATCH_SB(storage, bc, (set_state_kernel<S_, B_><<<cell_grid(d, 128), 128, 0, s>>>(d, f, dst)));
    return cudaGetLastError();
}

cudaError_t launch_get_state(const Dims& d, int storage, int bc, const void* src, float* f, cudaStream_t s) {
    LBM_DISPATCH_SB(storage, bc, (get_state_kernel<S_, B_><<<cell_grid(d, 128), 128, 0, s>>>(d, src, f)));
    return cudaGetLastError();
}

cudaError_t launch_macroscopic(const Dims& d, int storage, int bc, const void* src, float* rho, float* u,
                               cudaStream_t s) {
    LBM_DISPATCH_SB(storage, bc, (macroscopic_kernel<S_, B_><<<cell_grid(d, 128), 128, 0, s>>>(d, src, rho, u)));
    return cudaGetLastError();
}

cudaError_t launch_kinetic_energy(const Dims& d, int storage, int bc, const void* src, double* partials,
                                  int npartials, double* out, cudaStream_t s) {
    LBM_DISPATCH_SB(storage, bc,
                    (ke_partial_kernel<S_, B_><<<npartials, kKeThreads, 0, s>>>(d, src, partials)));
    sum_partials_kernel<<<1, kKeThreads, 0, s>>>(partials, npartials, 1.0 / static_cast<double>(d.ncell), out);
    return cudaGetLastError();
}

}  // namespace lbm
