// kernels_adjoint.cu - the hand-written adjoint (vector-Jacobian product) of one fused
// pull-stream + neural-collision step (Sec. II.A-B), FP32 on the CUDA cores.
//
// Forward step t: f_{t+1}[x][i] = C(f_t)[src(x,i)][ip(x,i)] (pull map, a bijection), with
// C(f) = M^-1 m*, m* = m - S_theta(m) (m - m^eq(m)), m = M f (eq. omegatheta).
// Adjoint, per cell y:
//   lam*[y][j] = lam_{t+1}[x][i] for the (x, i) that pulls (y, j)  (push with reflection);
//   mu* = M^-T lam*;                                 cotangent of m*
//   dL/dm = diag(1 - s) mu* + omega_nu (dm^eq/dm)^T mu*_(order 2) + (dtheta-network term);
//   the learned rates omega_n = 1/tau_n(tau~_n), tau~ = (1/48) sum_g Phi(P_g m), get the
//   cotangent -sum_{order(e)=n} mu*_e m_e and are backpropagated through the sigmoid,
//   the group mean and the 48 copies of Phi (weights and inputs);
//   lam_t[y] = M^T dL/dm.
// Weight gradients: per group element the block stages (delta h2, h1, delta h1, x) of its
// 128 cells in shared memory and accumulates register-blocked outer products, flushed
// to FP64 global accumulators with atomics. Layout of the accumulator (doubles):
// [dW1p (6 x 20 x 27, the W1 columns rearranged per axis permutation) | db1 | dW2 | db2 |
//  dW3 | db3]; the host folds dW1p back to the printed column order of W1.
#include "cell.cuh"

namespace lbm {

constexpr int kAdjThreads = 128;
constexpr int kGradW1p = 6 * kHidden * Q;                  // 3240
constexpr int kGradOffB1 = kGradW1p;
constexpr int kGradOffW2 = kGradOffB1 + kHidden;
constexpr int kGradOffB2 = kGradOffW2 + kHidden * kHidden;
constexpr int kGradOffW3 = kGradOffB2 + kHidden;
constexpr int kGradOffB3 = kGradOffW3 + kOut * kHidden;
constexpr int kGradLen = kGradOffB3 + kOut;               // 3764

int adjoint_grad_len() { return kGradLen; }

__device__ __forceinline__ int adj_odd_mask(int t) {
    return ((ex_of(t) == 1) << 2) | ((ey_of(t) == 1) << 1) | (ez_of(t) == 1);
}

// Inverse of the pull map: the (x, i) whose pulled value is population j of cell y.
template <int BC>
__device__ __forceinline__ void push_target(int y0, int y1, int y2, int j, const Dims& d, int& i, int& dst) {
    const int c[3] = {cx_of(j), cy_of(j), cz_of(j)};
    const int n[3] = {d.nx, d.ny, d.nz};
    const int y[3] = {y0, y1, y2};
    int x[3], ci[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int t = y[a] + c[a];
        if (BC == LBM_BC_PERIODIC) {
            t = t < 0 ? t + n[a] : (t >= n[a] ? t - n[a] : t);
            x[a] = t;
            ci[a] = c[a];
        } else {
            const bool out = t < 0 || t >= n[a];
            x[a] = out ? y[a] : t;
            ci[a] = out ? -c[a] : c[a];
        }
    }
    i = 9 * (ci[2] + 1) + 3 * (ci[1] + 1) + (ci[0] + 1);
    dst = (x[2] * d.ny + x[1]) * d.nx + x[0];
}

struct AdjArgs {
    Dims d;
    const void* state;   // stored buffer whose pull image is f_t
    const float* lam_in; // lam_{t+1}: 27 planes
    float* lam_out;      // lam_t: 27 planes
    double* grad;        // kGradLen accumulators
    float tau;
};

// Shared staging of one group element for the whole block.
struct AdjStage {
    float dh2[kAdjThreads][kHidden];
    float h1x[kAdjThreads][24];   // h1 (20), 1 (bias), pad
    float dh1[kAdjThreads][kHidden];
    float xm[kAdjThreads][28];    // signed moments (27, tensor order), 1 (bias)
};  // 47104 bytes; after the group loop h1x holds (gbar (4), h2 sum / 48 (20)) per cell

struct AdjShared {
    AdjStage st;
    NetParams net;                   // weights, read with run-time group indices
    float tail[kAdjThreads][24];     // per cell: gbar (4), h2 sum / 48 (20)
};
constexpr size_t kAdjSmem = sizeof(AdjShared);

template <int STORAGE, int BC>
__global__ void __launch_bounds__(kAdjThreads, 1) adjoint_step_kernel(const AdjArgs a,
                                                                      const __grid_constant__ NetParams netp) {
    extern __shared__ __align__(16) uint8_t adj_smem_raw[];
    AdjShared& sh = *reinterpret_cast<AdjShared*>(adj_smem_raw);
    AdjStage& st = sh.st;
    const NetParams& net = sh.net;
    const int tid = threadIdx.x;
    {
        const float* srcw = reinterpret_cast<const float*>(&netp);
        float* dstw = reinterpret_cast<float*>(&sh.net);
        for (int i = tid; i < static_cast<int>(sizeof(NetParams) / 4); i += kAdjThreads) dstw[i] = srcw[i];
        __syncthreads();
    }
    const long long cell = static_cast<long long>(blockIdx.x) * kAdjThreads + tid;
    const bool valid = cell < a.d.ncell;

    // ---- forward recompute of this cell
    float m[Q];
    float drho = 0.0f;
    float lam[Q];
    int x = 0, y = 0, z = 0;
    if (valid) {
        cell_coords(cell, a.d, x, y, z);
        float df[Q];
        load_pulled<STORAGE, BC>(a.state, a.d, x, y, z, df);
        drho = moments_from_dev(df, m);
#pragma unroll
        for (int jj = 0; jj < Q; ++jj) {
            int i, dst;
            push_target<BC>(x, y, z, jj, a.d, i, dst);
            lam[jj] = a.lam_in[static_cast<size_t>(i) * a.d.ncell + dst];
        }
    } else {
#pragma unroll
        for (int e = 0; e < Q; ++e) {
            m[e] = 0.0f;
            lam[e] = 0.0f;
        }
        m[0] = 1.0f;
    }
    const Macro q = macro_from_moments(m, drho);

    float hsum[kHidden];
#pragma unroll
    for (int j = 0; j < kHidden; ++j) hsum[j] = 0.0f;
#pragma unroll 1
    for (int g = 0; g < 48; ++g) {
        const int p = g >> 3, s = g & 7;
        float xs[Q];
#pragma unroll
        for (int t = 0; t < Q; ++t) xs[t] = (__popc(s & adj_odd_mask(t)) & 1) ? -m[t] : m[t];
        float h1[kHidden];
#pragma unroll 2
        for (int j = 0; j < kHidden; ++j) {
            float acc = net.b1[j];
#pragma unroll
            for (int t = 0; t < Q; ++t) acc = fmaf(net.W1p[p][j][t], xs[t], acc);
            h1[j] = fmaxf(acc, 0.0f);
        }
#pragma unroll 2
        for (int j = 0; j < kHidden; ++j) {
            float acc = net.b2[j];
#pragma unroll
            for (int k = 0; k < kHidden; ++k) acc = fmaf(net.W2[j][k], h1[k], acc);
            hsum[j] += fmaxf(acc, 0.0f);
        }
    }
    float ttil[kOut], tau_n[kOut], rates[kOut];
#pragma unroll
    for (int n = 0; n < kOut; ++n) {
        float acc = 0.0f;
#pragma unroll
        for (int j = 0; j < kHidden; ++j) acc = fmaf(net.W3[n][j], hsum[j], acc);
        ttil[n] = acc * (1.0f / 48.0f) + net.b3[n];
        tau_n[n] = 0.5f / (1.0f + expf(ttil[n])) + 0.5f;
        rates[n] = 1.0f / tau_n[n];
    }
#pragma unroll
    for (int j = 0; j < kHidden; ++j) sh.tail[tid][4 + j] = hsum[j] * (1.0f / 48.0f);

    // ---- cotangents in moment space
    populations_transpose_inplace(lam);  // lam now holds mu* = M^-T lam* (tensor order)
    const float omega_nu = 1.0f / a.tau;
    float dm[Q];
    float gw[kOut] = {0.0f, 0.0f, 0.0f, 0.0f};
    const float rho = m[0];
    const float mx = m[1], my = m[3], mz = m[9];
    const float irho = 1.0f / rho;
#pragma unroll
    for (int e = 0; e < Q; ++e) dm[e] = 0.0f;
#pragma unroll
    for (int e = 0; e < Q; ++e) {
        const int n = order_of(e);
        const float mu = lam[e];
        if (n <= 1) {
            dm[e] += mu;
        } else if (n == 2) {
            dm[e] += (1.0f - omega_nu) * mu;
            // m^eq_e = m_a m_b / m_0 for the axes a, b of component e
            const int ex = ex_of(e), ey = ey_of(e), ez = ez_of(e);
            int ia = -1, ib = -1;
            const int cnt[3] = {ex, ey, ez};
            const int idx[3] = {1, 3, 9};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (cnt[k] == 2) { ia = idx[k]; ib = idx[k]; }
                if (cnt[k] == 1) { if (ia < 0) ia = idx[k]; else ib = idx[k]; }
            }
            const float ma = m[ia], mb = m[ib];
            const float c = omega_nu * mu;
            dm[ia] += c * mb * irho;
            dm[ib] += c * ma * irho;
            dm[0] -= c * ma * mb * irho * irho;
        } else {
            dm[e] += (1.0f - rates[n - 3]) * mu;
            gw[n - 3] -= mu * m[e];
        }
    }
    (void)mx; (void)my; (void)mz;
    // d omega / d tau~ = sigma (1 - sigma) / (2 tau_n^2), sigma = 1 / (1 + e^{tau~})
    float gbar[kOut];
#pragma unroll
    for (int n = 0; n < kOut; ++n) {
        const float sg = 1.0f / (1.0f + expf(ttil[n]));
        gbar[n] = valid ? gw[n] * sg * (1.0f - sg) / (2.0f * tau_n[n] * tau_n[n]) : 0.0f;
        sh.tail[tid][n] = gbar[n];
    }
    // layer-3 cotangent into h2 (the same for every group element): W3^T gbar / 48
    float v3[kHidden];
#pragma unroll
    for (int j = 0; j < kHidden; ++j) {
        float acc = 0.0f;
#pragma unroll
        for (int n = 0; n < kOut; ++n) acc = fmaf(net.W3[n][j], gbar[n], acc);
        v3[j] = acc * (1.0f / 48.0f);
    }

    // ---- backward through the 48 copies of Phi, with block-level weight gradients
    // thread roles in the outer-product accumulation
    const bool w2_role = tid < 40;                 // dW2|db2: rows 2r.., cols 6c.. (20 x 24)
    const bool w1_role = tid >= 40 && tid < 110;   // dW1p|db1: rows 2r.., cols 4c.. (20 x 28)
    const int w2_r = (tid % 10) * 2, w2_c = (tid / 10) * 6;
    const int w1_r = ((tid - 40) % 10) * 2, w1_c = ((tid - 40) / 10) * 4;
    float acc2[2][6], acc1[2][4];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
#pragma unroll
        for (int v = 0; v < 6; ++v) acc2[u][v] = 0.0f;
#pragma unroll
        for (int v = 0; v < 4; ++v) acc1[u][v] = 0.0f;
    }
#pragma unroll 1
    for (int g = 0; g < 48; ++g) {
        const int p = g >> 3, s = g & 7;
        float xs[Q];
#pragma unroll
        for (int t = 0; t < Q; ++t) xs[t] = (__popc(s & adj_odd_mask(t)) & 1) ? -m[t] : m[t];
        float h1[kHidden];
#pragma unroll 2
        for (int j = 0; j < kHidden; ++j) {
            float acc = net.b1[j];
#pragma unroll
            for (int t = 0; t < Q; ++t) acc = fmaf(net.W1p[p][j][t], xs[t], acc);
            h1[j] = fmaxf(acc, 0.0f);
        }
        float dh2[kHidden];
#pragma unroll 2
        for (int j = 0; j < kHidden; ++j) {
            float acc = net.b2[j];
#pragma unroll
            for (int k = 0; k < kHidden; ++k) acc = fmaf(net.W2[j][k], h1[k], acc);
            dh2[j] = acc > 0.0f ? v3[j] : 0.0f;
        }
        float dh1[kHidden];
#pragma unroll 2
        for (int k = 0; k < kHidden; ++k) {
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < kHidden; ++j) acc = fmaf(net.W2[j][k], dh2[j], acc);
            dh1[k] = h1[k] > 0.0f ? acc : 0.0f;
        }
#pragma unroll 3
        for (int t = 0; t < Q; ++t) {
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < kHidden; ++j) acc = fmaf(net.W1p[p][j][t], dh1[j], acc);
            dm[t] += ((__popc(s & adj_odd_mask(t)) & 1) ? -acc : acc);
        }
        // stage this group element for the weight-gradient outer products
#pragma unroll
        for (int j = 0; j < kHidden; ++j) {
            st.dh2[tid][j] = dh2[j];
            st.h1x[tid][j] = h1[j];
            st.dh1[tid][j] = dh1[j];
        }
        st.h1x[tid][kHidden] = 1.0f;
#pragma unroll
        for (int k = kHidden + 1; k < 24; ++k) st.h1x[tid][k] = 0.0f;
#pragma unroll
        for (int t = 0; t < Q; ++t) st.xm[tid][t] = xs[t];
        st.xm[tid][Q] = 1.0f;
        __syncthreads();
        if (w2_role) {
            for (int c = 0; c < kAdjThreads; ++c) {
                const float r0 = st.dh2[c][w2_r], r1 = st.dh2[c][w2_r + 1];
#pragma unroll
                for (int v = 0; v < 6; ++v) {
                    const float cv = st.h1x[c][w2_c + v];
                    acc2[0][v] = fmaf(r0, cv, acc2[0][v]);
                    acc2[1][v] = fmaf(r1, cv, acc2[1][v]);
                }
            }
        } else if (w1_role) {
            for (int c = 0; c < kAdjThreads; ++c) {
                const float r0 = st.dh1[c][w1_r], r1 = st.dh1[c][w1_r + 1];
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const float cv = st.xm[c][w1_c + v];
                    acc1[0][v] = fmaf(r0, cv, acc1[0][v]);
                    acc1[1][v] = fmaf(r1, cv, acc1[1][v]);
                }
            }
        }
        __syncthreads();
        if (s == 7 && w1_role) {  // the eight elements of axis permutation p are done
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int j = w1_r + u, col = w1_c + v;
                    if (col < Q) atomicAdd(&a.grad[p * kHidden * Q + j * Q + col], static_cast<double>(acc1[u][v]));
                    else if (col == Q) atomicAdd(&a.grad[kGradOffB1 + j], static_cast<double>(acc1[u][v]));
                    acc1[u][v] = 0.0f;
                }
        }
    }
    if (w2_role) {
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int v = 0; v < 6; ++v) {
                const int j = w2_r + u, col = w2_c + v;
                if (col < kHidden) atomicAdd(&a.grad[kGradOffW2 + j * kHidden + col], static_cast<double>(acc2[u][v]));
                else if (col == kHidden) atomicAdd(&a.grad[kGradOffB2 + j], static_cast<double>(acc2[u][v]));
            }
    }
    // layer 3: dW3[n][j] += gbar_n * hsum_j / 48, db3[n] += gbar_n (block sums via shared memory)
    __syncthreads();
    if (tid < kOut * (kHidden + 1)) {
        const int n = tid / (kHidden + 1), j = tid % (kHidden + 1);
        float acc = 0.0f;
        for (int c = 0; c < kAdjThreads; ++c) acc = fmaf(sh.tail[c][n], j < kHidden ? sh.tail[c][4 + j] : 1.0f, acc);
        if (j < kHidden) atomicAdd(&a.grad[kGradOffW3 + n * kHidden + j], static_cast<double>(acc));
        else atomicAdd(&a.grad[kGradOffB3 + n], static_cast<double>(acc));
    }

    // ---- lam_t = M^T dL/dm
    if (valid) {
        moments_transpose_inplace(dm);
#pragma unroll
        for (int i = 0; i < Q; ++i) a.lam_out[static_cast<size_t>(i) * a.d.ncell + cell] = dm[i];
    }
}

// lam_T[i] = sum_a dL/du_a (c_ia - u_a) / rho + dL/drho for the state whose pull image is f_T.
template <int STORAGE, int BC>
__global__ void adjoint_seed_kernel(const Dims d, const void* state, const float* __restrict__ du,
                                    const float* __restrict__ drho_in, float* lam) {
    const long long cell = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (cell >= d.ncell) return;
    int x, y, z;
    cell_coords(cell, d, x, y, z);
    float df[Q], m[Q];
    load_pulled<STORAGE, BC>(state, d, x, y, z, df);
    const float dr = moments_from_dev(df, m);
    const Macro q = macro_from_moments(m, dr);
    const float gx = du ? du[cell] : 0.0f, gy = du ? du[d.ncell + cell] : 0.0f, gz = du ? du[2 * d.ncell + cell] : 0.0f;
    const float gr = drho_in ? drho_in[cell] : 0.0f;
    const float ir = 1.0f / q.rho;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float v = (gx * (cx_of(i) - q.ux) + gy * (cy_of(i) - q.uy) + gz * (cz_of(i) - q.uz)) * ir + gr;
        lam[static_cast<size_t>(i) * d.ncell + cell] = v;
    }
}

cudaError_t launch_adjoint_seed(const Dims& d, int storage, int bc, const void* state, const float* du,
                                const float* drho, float* lam, cudaStream_t s) {
    const dim3 grid(static_cast<unsigned>((d.ncell + 127) / 128));
    if (storage != LBM_STORE_F32) return cudaErrorInvalidValue;
    if (bc == LBM_BC_PERIODIC) adjoint_seed_kernel<LBM_STORE_F32, LBM_BC_PERIODIC><<<grid, 128, 0, s>>>(d, state, du, drho, lam);
    else adjoint_seed_kernel<LBM_STORE_F32, LBM_BC_MIRROR><<<grid, 128, 0, s>>>(d, state, du, drho, lam);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_step(const Dims& d, int storage, int bc, const void* state, const float* lam_in,
                                float* lam_out, double* grad, float tau, const NetParams& net, cudaStream_t s) {
    if (storage != LBM_STORE_F32) return cudaErrorInvalidValue;
    AdjArgs a{d, state, lam_in, lam_out, grad, tau};
    const dim3 grid(static_cast<unsigned>((d.ncell + kAdjThreads - 1) / kAdjThreads));
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(adjoint_step_kernel<LBM_STORE_F32, LBM_BC_PERIODIC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kAdjSmem));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(adjoint_step_kernel<LBM_STORE_F32, LBM_BC_MIRROR>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kAdjSmem));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (bc == LBM_BC_PERIODIC) adjoint_step_kernel<LBM_STORE_F32, LBM_BC_PERIODIC><<<grid, kAdjThreads, kAdjSmem, s>>>(a, net);
    else adjoint_step_kernel<LBM_STORE_F32, LBM_BC_MIRROR><<<grid, kAdjThreads, kAdjSmem, s>>>(a, net);
    return cudaGetLastError();
}

// Fold the accumulator into the flat parameter order W1, b1, W2, b2, W3, b3 (W1 in the
// printed column order): dW1[j][k] = sum_p dW1p[p][j][t_p(k)].
void adjoint_fold_gradient(const double* acc, float* out) {
    const GroupTables& g = group_tables();
    for (int j = 0; j < kHidden; ++j)
        for (int k = 0; k < Q; ++k) {
            double v = 0.0;
            for (int p = 0; p < 6; ++p) v += acc[p * kHidden * Q + j * Q + g.mperm_t[p * 8][kPrinted.e[k]]];
            out[j * Q + k] = static_cast<float>(v);
        }
    float* o = out + kHidden * Q;
    for (int j = 0; j < kHidden; ++j) *o++ = static_cast<float>(acc[kGradOffB1 + j]);
    for (int j = 0; j < kHidden * kHidden; ++j) *o++ = static_cast<float>(acc[kGradOffW2 + j]);
    for (int j = 0; j < kHidden; ++j) *o++ = static_cast<float>(acc[kGradOffB2 + j]);
    for (int j = 0; j < kOut * kHidden; ++j) *o++ = static_cast<float>(acc[kGradOffW3 + j]);
    for (int j = 0; j < kOut; ++j) *o++ = static_cast<float>(acc[kGradOffB3 + j]);
}

}  // namespace lbm
