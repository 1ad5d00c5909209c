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
// The 48 elements are taken per axis permutation p: for its 8 sign vectors s the first layer
// is an 8-point Walsh-Hadamard transform of the parity-class partial sums of W1p m (the
// forward kernel's form), and so are the first layer's cotangents: with E[c][j] =
// sum_s (-1)^popcount(s & c) delta h1[s][j], the cotangent of m_t is sum_j W1p[j][t]
// E[c(t)][j] and dW1p[j][t] = sum over cells of m_t E[c(t)][j], c(t) the parity class of
// moment t. Each thread keeps the 8 x 20 values of its cell (h1, then delta h1, then E) in
// a row of shared memory. Weight gradients: per sign vector the block stages (delta h2, h1;
// with the third hidden layer also delta h3, h2) of its 128 cells and accumulates
// register-blocked outer products, per permutation (E, m) for the first layer, flushed to
// FP64 global accumulators with atomics.
// Layout of the accumulator (doubles): [dW1p (6 x 20 x 27, the W1 columns rearranged per
// axis permutation) | db1 | dW2 | db2 | (dWd | dbd, third hidden layer) | dW3 | db3]; the
// host folds dW1p back to the printed column order of W1.
//
// Observations of the kinetic energy k = (1/2)<|u|^2> at intermediate steps (the loss of
// Sec. IV is a function of k(t)) enter as extra seeds added to lam_t when the reverse
// sweep passes step t: dk/df_i = (1/cells) sum_a u_a (c_ia - u_a) / rho.
#include "cell.cuh"

namespace lbm {

constexpr int kAdjThreads = 128;

template <bool DEEP>
struct GradLayout {
    static constexpr int kB1 = 6 * kHidden * Q;                 // dW1p first
    static constexpr int kW2 = kB1 + kHidden;
    static constexpr int kB2 = kW2 + kHidden * kHidden;
    static constexpr int kWd = kB2 + kHidden;                   // third hidden layer
    static constexpr int kBd = kWd + kHidden * kHidden;
    static constexpr int kW3 = DEEP ? kBd + kHidden : kB2 + kHidden;
    static constexpr int kB3 = kW3 + kOut * kHidden;
    static constexpr int kLen = kB3 + kOut;                     // 3764 or 4184
};

int adjoint_grad_len(bool deep) { return deep ? GradLayout<true>::kLen : GradLayout<false>::kLen; }

__device__ __forceinline__ int adj_odd_mask(int t) {
    return ((ex_of(t) == 1) << 2) | ((ey_of(t) == 1) << 1) | (ez_of(t) == 1);
}

// y[s] <- sum_c (-1)^popcount(s & c) y[c], in place (its own inverse up to a factor 8)
__device__ __forceinline__ void wht8(float* y) {
#pragma unroll
    for (int bit = 1; bit < 8; bit <<= 1)
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if (!(c & bit)) {
                const float u = y[c], v = y[c | bit];
                y[c] = u + v;
                y[c | bit] = u - v;
            }
}

// a thread's row of first-layer values: [s * kHidden + j], padded so that the rows of a
// warp's threads fall in different banks
constexpr int kHbStride = 8 * kHidden + 1;

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
        } else if (BC == LBM_BC_TGV_REDUCED) {
            x[a] = t;
            ci[a] = c[a];
        } else {
            const bool out = t < 0 || t >= n[a];
            x[a] = out ? y[a] : t;
            ci[a] = out ? -c[a] : c[a];
        }
    }
    i = 9 * (ci[2] + 1) + 3 * (ci[1] + 1) + (ci[0] + 1);
    if (BC == LBM_BC_TGV_REDUCED) {
        // Appendix A: a population leaving the domain towards the block r of q = y + c_j
        // re-enters as its image under the flow symmetry g_r = (A, t) of that block: at
        // g_r(q) with velocity A c_j. This inverts the pull, which takes the source
        // g_r(x - c_i) for a source outside the domain: g_r is the only symmetry mapping
        // block r onto the domain, so g_r^-1 is the one for the block g_r(domain).
        const int nn = d.nx;
        const int rx = x[0] < 0 ? -1 : (x[0] >= nn ? 1 : 0), ry = x[1] < 0 ? -1 : (x[1] >= nn ? 1 : 0),
                  rz = x[2] < 0 ? -1 : (x[2] >= nn ? 1 : 0);
        if (rx | ry | rz) {
            const SymRegion& g = d.sym[9 * (rz + 1) + 3 * (ry + 1) + (rx + 1)];
            const int q2[3] = {2 * x[0] + 1, 2 * x[1] + 1, 2 * x[2] + 1};
            int xi[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                int v = g.sign[a] * q2[g.perm[a]] + 2 * nn * g.k[a];
                v %= 8 * nn;
                if (v < 0) v += 8 * nn;
                xi[a] = (v - 1) >> 1;
            }
            x[0] = xi[0];
            x[1] = xi[1];
            x[2] = xi[2];
            i = g.pmap[j];
        }
    }
    dst = (x[2] * d.ny + x[1]) * d.nx + x[0];
}

struct AdjArgs {
    Dims d;
    const void* state;   // stored buffer whose pull image is f_t
    const float* lam_in; // lam_{t+1}: 27 planes
    float* lam_out;      // lam_t: 27 planes
    double* grad;        // GradLayout<DEEP>::kLen accumulators
    float tau;
    const float* force;  // forced step: the force field of step t (3 planes), else null
    int nparts;          // blocks per tile, each backpropagating 6 / nparts axis permutations
};

// Shared staging of one group element for the whole block (the last two arrays only with
// the third hidden layer).
template <bool DEEP>
struct AdjStage {
    float dh2[kAdjThreads][kHidden];
    float h1x[kAdjThreads][24];   // h1 (20), 1 (bias), pad
    float xm[kAdjThreads][28];    // moments (27, tensor order), 1 (bias)
    float dh3[DEEP ? kAdjThreads : 1][kHidden];
    float h2x[DEEP ? kAdjThreads : 1][24];  // h2 (20), 1 (bias), pad
};

template <bool DEEP>
struct AdjShared {
    AdjStage<DEEP> st;
    float hb[kAdjThreads * kHbStride];  // per cell: h1, delta h1, then E of the 8 sign vectors
    NetParams net;                      // weights, read with run-time group indices
    float tail[kAdjThreads][24];        // per cell: gbar (4), group mean of the last hidden layer (20)
};

template <int STORAGE, int BC, bool DEEP>
__global__ void __launch_bounds__(kAdjThreads, 1) adjoint_step_kernel(const AdjArgs a,
                                                                      const __grid_constant__ NetParams netp) {
    using GL = GradLayout<DEEP>;
    extern __shared__ __align__(16) uint8_t adj_smem_raw[];
    AdjShared<DEEP>& sh = *reinterpret_cast<AdjShared<DEEP>*>(adj_smem_raw);
    AdjStage<DEEP>& st = sh.st;
    const NetParams& net = sh.net;
    const int tid = threadIdx.x;
    {
        const float* srcw = reinterpret_cast<const float*>(&netp);
        float* dstw = reinterpret_cast<float*>(&sh.net);
        for (int i = tid; i < static_cast<int>(sizeof(NetParams) / 4); i += kAdjThreads) dstw[i] = srcw[i];
        __syncthreads();
    }
    // small grids: nparts blocks share a tile, block `part` backpropagating the group
    // elements of axis permutations [part, part + 1) * 6 / nparts; every part recomputes the
    // forward, part 0 alone adds the relaxation terms and the output-layer gradient
    const long long tile = blockIdx.x / a.nparts;
    const int part = static_cast<int>(blockIdx.x % a.nparts);
    const int p_begin = part * (6 / a.nparts), p_end = p_begin + 6 / a.nparts;
    const long long cell = tile * kAdjThreads + tid;
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

    // this thread's row of first-layer values; first_layer(p) fills it with relu(W1p x^(s) +
    // b1) of the 8 sign vectors s of permutation p
    float* hb = sh.hb + tid * kHbStride;
    auto first_layer = [&](int p) {
#pragma unroll 2
        for (int j = 0; j < kHidden; ++j) {
            float y[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) y[c] = 0.0f;
#pragma unroll
            for (int t = 0; t < Q; ++t) y[adj_odd_mask(t)] = fmaf(net.W1p[p][j][t], m[t], y[adj_odd_mask(t)]);
            wht8(y);
#pragma unroll
            for (int sv = 0; sv < 8; ++sv) hb[sv * kHidden + j] = fmaxf(y[sv] + net.b1[j], 0.0f);
        }
    };

    // group sum of the last hidden layer (h2, or h3 with the third hidden layer)
    float hsum[kHidden];
#pragma unroll
    for (int j = 0; j < kHidden; ++j) hsum[j] = 0.0f;
#pragma unroll 1
    for (int p = 0; p < 6; ++p) {
        first_layer(p);
#pragma unroll 1
        for (int sv = 0; sv < 8; ++sv) {
            float h1[kHidden];
#pragma unroll
            for (int j = 0; j < kHidden; ++j) h1[j] = hb[sv * kHidden + j];
            if constexpr (DEEP) {
                float h2[kHidden];
#pragma unroll 2
                for (int j = 0; j < kHidden; ++j) {
                    float acc = net.b2[j];
#pragma unroll
                    for (int k = 0; k < kHidden; ++k) acc = fmaf(net.W2[j][k], h1[k], acc);
                    h2[j] = fmaxf(acc, 0.0f);
                }
#pragma unroll 2
                for (int j = 0; j < kHidden; ++j) {
                    float acc = net.bd[j];
#pragma unroll
                    for (int k = 0; k < kHidden; ++k) acc = fmaf(net.Wd[j][k], h2[k], acc);
                    hsum[j] += fmaxf(acc, 0.0f);
                }
            } else {
#pragma unroll 2
                for (int j = 0; j < kHidden; ++j) {
                    float acc = net.b2[j];
#pragma unroll
                    for (int k = 0; k < kHidden; ++k) acc = fmaf(net.W2[j][k], h1[k], acc);
                    hsum[j] += fmaxf(acc, 0.0f);
                }
            }
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
            int ia = -1, ib = -1, axa = 0, axb = 0;
            const int cnt[3] = {ex, ey, ez};
            const int idx[3] = {1, 3, 9};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (cnt[k] == 2) { ia = idx[k]; ib = idx[k]; axa = axb = k; }
                if (cnt[k] == 1) {
                    if (ia < 0) { ia = idx[k]; axa = k; }
                    else { ib = idx[k]; axb = k; }
                }
            }
            const float ma = m[ia], mb = m[ib];
            const float c = omega_nu * mu;
            dm[ia] += c * mb * irho;
            dm[ib] += c * ma * irho;
            dm[0] -= c * ma * mb * irho * irho;
            if (a.force && valid) {
                // Kupershtokh source (Sec. II.A) in moment space: its only state-dependent part
                // is order 2, dm*_ab = 3 ((j + F)_a (j + F)_b - j_a j_b) / rho with m_a = sqrt3 j_a,
                // i.e. (sqrt3 (m_a F_b + F_a m_b) + 3 F_a F_b) / rho; the force is an input
                const float Fa = a.force[static_cast<size_t>(axa) * a.d.ncell + cell];
                const float Fb = a.force[static_cast<size_t>(axb) * a.d.ncell + cell];
                const float src = (kSqrt3 * (ma * Fb + Fa * mb) + 3.0f * Fa * Fb) * irho;
                dm[ia] += mu * kSqrt3 * Fb * irho;
                dm[ib] += mu * kSqrt3 * Fa * irho;
                dm[0] -= mu * src * irho;
            }
        } else {
            dm[e] += (1.0f - rates[n - 3]) * mu;
            gw[n - 3] -= mu * m[e];
        }
    }
    if (part != 0) {  // the relaxation's own terms belong to part 0; the rates' cotangent gw to all
#pragma unroll
        for (int e = 0; e < Q; ++e) dm[e] = 0.0f;
    }
    // d omega / d tau~ = sigma (1 - sigma) / (2 tau_n^2), sigma = 1 / (1 + e^{tau~})
    float gbar[kOut];
#pragma unroll
    for (int n = 0; n < kOut; ++n) {
        const float sg = 1.0f / (1.0f + expf(ttil[n]));
        gbar[n] = valid ? gw[n] * sg * (1.0f - sg) / (2.0f * tau_n[n] * tau_n[n]) : 0.0f;
        sh.tail[tid][n] = gbar[n];
    }
    // cotangent of the last hidden layer (the same for every group element): W3^T gbar / 48
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
    const bool w2_role = tid < 40;                 // dW2|db2 (and dWd|dbd): rows 2r.., cols 6c.. (20 x 24)
    const bool w1_role = tid >= 40 && tid < 110;   // dW1p|db1: rows 2r.., cols 4c.. (20 x 28)
    const int w2_r = (tid % 10) * 2, w2_c = (tid / 10) * 6;
    const int w1_r = ((tid - 40) % 10) * 2, w1_c = ((tid - 40) / 10) * 4;
    float acc2[2][6], accd[2][6], acc1[2][4];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
#pragma unroll
        for (int v = 0; v < 6; ++v) {
            acc2[u][v] = 0.0f;
            accd[u][v] = 0.0f;
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) acc1[u][v] = 0.0f;
    }
    // the moments and the bias input of every cell, for the first layer's weight gradient
#pragma unroll
    for (int t = 0; t < Q; ++t) st.xm[tid][t] = m[t];
    st.xm[tid][Q] = 1.0f;
    // the first-layer gradient columns of this thread and their parity classes (the bias
    // column Q belongs to class 0: all its signs are +)
    int w1_cls[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int col = w1_role ? w1_c + v : 0;
        w1_cls[v] = col < Q ? adj_odd_mask(col) : 0;
    }
#pragma unroll 1
    for (int p = p_begin; p < p_end; ++p) {
        first_layer(p);
#pragma unroll 1
        for (int sv = 0; sv < 8; ++sv) {
            float h1[kHidden];
#pragma unroll
            for (int j = 0; j < kHidden; ++j) h1[j] = hb[sv * kHidden + j];
            float dh2[kHidden];
            if constexpr (DEEP) {
                float h2[kHidden];
#pragma unroll 2
                for (int j = 0; j < kHidden; ++j) {
                    float acc = net.b2[j];
#pragma unroll
                    for (int k = 0; k < kHidden; ++k) acc = fmaf(net.W2[j][k], h1[k], acc);
                    h2[j] = fmaxf(acc, 0.0f);
                }
                float dh3[kHidden];
#pragma unroll 2
                for (int j = 0; j < kHidden; ++j) {
                    float acc = net.bd[j];
#pragma unroll
                    for (int k = 0; k < kHidden; ++k) acc = fmaf(net.Wd[j][k], h2[k], acc);
                    dh3[j] = acc > 0.0f ? v3[j] : 0.0f;
                }
#pragma unroll 2
                for (int k = 0; k < kHidden; ++k) {
                    float acc = 0.0f;
#pragma unroll
                    for (int j = 0; j < kHidden; ++j) acc = fmaf(net.Wd[j][k], dh3[j], acc);
                    dh2[k] = h2[k] > 0.0f ? acc : 0.0f;
                }
#pragma unroll
                for (int j = 0; j < kHidden; ++j) {
                    st.dh3[tid][j] = dh3[j];
                    st.h2x[tid][j] = h2[j];
                }
                st.h2x[tid][kHidden] = 1.0f;
#pragma unroll
                for (int k = kHidden + 1; k < 24; ++k) st.h2x[tid][k] = 0.0f;
            } else {
#pragma unroll 2
                for (int j = 0; j < kHidden; ++j) {
                    float acc = net.b2[j];
#pragma unroll
                    for (int k = 0; k < kHidden; ++k) acc = fmaf(net.W2[j][k], h1[k], acc);
                    dh2[j] = acc > 0.0f ? v3[j] : 0.0f;
                }
            }
            // delta h1 replaces h1 in this thread's row
#pragma unroll 2
            for (int k = 0; k < kHidden; ++k) {
                float acc = 0.0f;
#pragma unroll
                for (int j = 0; j < kHidden; ++j) acc = fmaf(net.W2[j][k], dh2[j], acc);
                hb[sv * kHidden + k] = h1[k] > 0.0f ? acc : 0.0f;
            }
            // stage this sign vector for the second-layer weight-gradient outer products
#pragma unroll
            for (int j = 0; j < kHidden; ++j) {
                st.dh2[tid][j] = dh2[j];
                st.h1x[tid][j] = h1[j];
            }
            st.h1x[tid][kHidden] = 1.0f;
#pragma unroll
            for (int k = kHidden + 1; k < 24; ++k) st.h1x[tid][k] = 0.0f;
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
                    if constexpr (DEEP) {
                        const float d0 = st.dh3[c][w2_r], d1 = st.dh3[c][w2_r + 1];
#pragma unroll
                        for (int v = 0; v < 6; ++v) {
                            const float cv = st.h2x[c][w2_c + v];
                            accd[0][v] = fmaf(d0, cv, accd[0][v]);
                            accd[1][v] = fmaf(d1, cv, accd[1][v]);
                        }
                    }
                }
            }
            __syncthreads();
        }
        // E[c][j] = sum_s (-1)^popcount(s & c) delta h1[s][j], in place, and the first
        // layer's cotangent of m: sum_s sgn(s, t) (W1p^T delta h1[s])_t = (W1p^T E[c(t)])_t
#pragma unroll 2
        for (int j = 0; j < kHidden; ++j) {
            float e[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) e[c] = hb[c * kHidden + j];
            wht8(e);
#pragma unroll
            for (int c = 0; c < 8; ++c) hb[c * kHidden + j] = e[c];
#pragma unroll
            for (int t = 0; t < Q; ++t) dm[t] = fmaf(net.W1p[p][j][t], e[adj_odd_mask(t)], dm[t]);
        }
        __syncthreads();  // every cell's E is in place
        if (w1_role) {  // dW1p[j][t] += sum over cells of E[c(t)][j] m_t (db1 through the bias column)
            for (int c = 0; c < kAdjThreads; ++c) {
                const float* ec = sh.hb + c * kHbStride;
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const float cv = st.xm[c][w1_c + v];
                    acc1[0][v] = fmaf(ec[w1_cls[v] * kHidden + w1_r], cv, acc1[0][v]);
                    acc1[1][v] = fmaf(ec[w1_cls[v] * kHidden + w1_r + 1], cv, acc1[1][v]);
                }
            }
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int j = w1_r + u, col = w1_c + v;
                    if (col < Q) atomicAdd(&a.grad[p * kHidden * Q + j * Q + col], static_cast<double>(acc1[u][v]));
                    else if (col == Q) atomicAdd(&a.grad[GL::kB1 + j], static_cast<double>(acc1[u][v]));
                    acc1[u][v] = 0.0f;
                }
        }
        __syncthreads();  // the rows are refilled by the next permutation
    }
    if (w2_role) {
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int v = 0; v < 6; ++v) {
                const int j = w2_r + u, col = w2_c + v;
                if (col < kHidden) atomicAdd(&a.grad[GL::kW2 + j * kHidden + col], static_cast<double>(acc2[u][v]));
                else if (col == kHidden) atomicAdd(&a.grad[GL::kB2 + j], static_cast<double>(acc2[u][v]));
                if constexpr (DEEP) {
                    if (col < kHidden) atomicAdd(&a.grad[GL::kWd + j * kHidden + col], static_cast<double>(accd[u][v]));
                    else if (col == kHidden) atomicAdd(&a.grad[GL::kBd + j], static_cast<double>(accd[u][v]));
                }
            }
    }
    // output layer: dW3[n][j] += gbar_n * hmean_j, db3[n] += gbar_n (block sums via shared memory)
    __syncthreads();
    if (part == 0 && tid < kOut * (kHidden + 1)) {
        const int n = tid / (kHidden + 1), j = tid % (kHidden + 1);
        float acc = 0.0f;
        for (int c = 0; c < kAdjThreads; ++c) acc = fmaf(sh.tail[c][n], j < kHidden ? sh.tail[c][4 + j] : 1.0f, acc);
        if (j < kHidden) atomicAdd(&a.grad[GL::kW3 + n * kHidden + j], static_cast<double>(acc));
        else atomicAdd(&a.grad[GL::kB3 + n], static_cast<double>(acc));
    }

    // ---- lam_t = M^T dL/dm (summed over the parts of a tile into a zeroed buffer)
    if (valid) {
        moments_transpose_inplace(dm);
        float* out = a.lam_out + cell;
        if (a.nparts == 1) {
#pragma unroll
            for (int i = 0; i < Q; ++i) out[static_cast<size_t>(i) * a.d.ncell] = dm[i];
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) atomicAdd(out + static_cast<size_t>(i) * a.d.ncell, dm[i]);
        }
    }
}

// lam[i] (=, or += when accumulate) sum_a g_a (c_ia - u_a) / rho + dL/drho for the state
// whose pull image is f, with g_a = dL/du_a + ke_scale u_a: the cotangent of the
// macroscopic fields, and of the kinetic energy k = (1/2)<|u|^2> with ke_scale =
// (dL/dk) / cells.
template <int STORAGE, int BC>
__global__ void adjoint_seed_kernel(const Dims d, const void* state, const float* __restrict__ du,
                                    const float* __restrict__ drho_in, float ke_scale, int accumulate,
                                    float* lam) {
    const long long cell = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (cell >= d.ncell) return;
    int x, y, z;
    cell_coords(cell, d, x, y, z);
    float df[Q], m[Q];
    load_pulled<STORAGE, BC>(state, d, x, y, z, df);
    const float dr = moments_from_dev(df, m);
    const Macro q = macro_from_moments(m, dr);
    const float gx = (du ? du[cell] : 0.0f) + ke_scale * q.ux;
    const float gy = (du ? du[d.ncell + cell] : 0.0f) + ke_scale * q.uy;
    const float gz = (du ? du[2 * d.ncell + cell] : 0.0f) + ke_scale * q.uz;
    const float gr = drho_in ? drho_in[cell] : 0.0f;
    const float ir = 1.0f / q.rho;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float v = (gx * (cx_of(i) - q.ux) + gy * (cy_of(i) - q.uy) + gz * (cz_of(i) - q.uz)) * ir + gr;
        float* o = lam + static_cast<size_t>(i) * d.ncell + cell;
        *o = accumulate ? *o + v : v;
    }
}

cudaError_t launch_adjoint_seed(const Dims& d, int storage, int bc, const void* state, const float* du,
                                const float* drho, float ke_scale, bool accumulate, float* lam, cudaStream_t s) {
    const dim3 grid(static_cast<unsigned>((d.ncell + 127) / 128));
    if (storage != LBM_STORE_F32) return cudaErrorInvalidValue;
    const int acc = accumulate ? 1 : 0;
    if (bc == LBM_BC_PERIODIC)
        adjoint_seed_kernel<LBM_STORE_F32, LBM_BC_PERIODIC><<<grid, 128, 0, s>>>(d, state, du, drho, ke_scale, acc, lam);
    else if (bc == LBM_BC_MIRROR)
        adjoint_seed_kernel<LBM_STORE_F32, LBM_BC_MIRROR><<<grid, 128, 0, s>>>(d, state, du, drho, ke_scale, acc, lam);
    else if (bc == LBM_BC_TGV_REDUCED)
        adjoint_seed_kernel<LBM_STORE_F32, LBM_BC_TGV_REDUCED><<<grid, 128, 0, s>>>(d, state, du, drho, ke_scale, acc, lam);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <int BC, bool DEEP>
static cudaError_t launch_adjoint_step_t(const AdjArgs& a, const NetParams& net, cudaStream_t s) {
    constexpr size_t smem = sizeof(AdjShared<DEEP>);
    static std::atomic<unsigned long long> attr{0};  // one set of per-device flags per instantiation
    {
        const cudaError_t e = ensure_dynamic_smem(adjoint_step_kernel<LBM_STORE_F32, BC, DEEP>, static_cast<int>(smem),
                                                  attr);
        if (e != cudaSuccess) return e;
    }
    const long long tiles = (a.d.ncell + kAdjThreads - 1) / kAdjThreads;
    if (a.nparts > 1) {
        const cudaError_t e = cudaMemsetAsync(a.lam_out, 0, sizeof(float) * Q * static_cast<size_t>(a.d.ncell), s);
        if (e != cudaSuccess) return e;
    }
    const dim3 grid(static_cast<unsigned>(tiles * a.nparts));
    adjoint_step_kernel<LBM_STORE_F32, BC, DEEP><<<grid, kAdjThreads, smem, s>>>(a, net);
    return cudaGetLastError();
}

template <bool DEEP>
static cudaError_t launch_adjoint_step_bc(const AdjArgs& a, int bc, const NetParams& net, cudaStream_t s) {
    switch (bc) {
        case LBM_BC_PERIODIC: return launch_adjoint_step_t<LBM_BC_PERIODIC, DEEP>(a, net, s);
        case LBM_BC_MIRROR: return launch_adjoint_step_t<LBM_BC_MIRROR, DEEP>(a, net, s);
        case LBM_BC_TGV_REDUCED: return launch_adjoint_step_t<LBM_BC_TGV_REDUCED, DEEP>(a, net, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_adjoint_step(const Dims& d, int storage, int bc, const void* state, const float* lam_in,
                                float* lam_out, double* grad, float tau, const float* force, const NetParams& net,
                                cudaStream_t s) {
    if (storage != LBM_STORE_F32) return cudaErrorInvalidValue;
    // grids of fewer tiles than SMs (the small domains of training): split the 6 axis
    // permutations of a tile over 2, 3 or 6 blocks so that every SM gets work; from one tile
    // per SM on, the forward that every part recomputes costs more than it brings
    // (measured: 16^3 with 32 tiles, 6 parts, 1.74 x faster; 32^3 with 256 tiles, 2 parts,
    // 15 % slower)
    const long long tiles = (d.ncell + kAdjThreads - 1) / kAdjThreads;
    const long long want = sm_count();
    const int nparts = tiles >= want ? 1 : tiles * 2 >= want ? 2 : tiles * 3 >= want ? 3 : 6;
    AdjArgs a{d, state, lam_in, lam_out, grad, tau, force, nparts};
    return net.deep ? launch_adjoint_step_bc<true>(a, bc, net, s) : launch_adjoint_step_bc<false>(a, bc, net, s);
}

// Fold the accumulator into the flat parameter order W1, b1, W2, b2, (Wd, bd), W3, b3 (W1
// in the printed column order): dW1[j][k] = sum_p dW1p[p][j][t_p(k)].
template <bool DEEP>
static void fold_gradient(const double* acc, float* out) {
    using GL = GradLayout<DEEP>;
    const GroupTables& g = group_tables();
    for (int j = 0; j < kHidden; ++j)
        for (int k = 0; k < Q; ++k) {
            double v = 0.0;
            for (int p = 0; p < 6; ++p) v += acc[p * kHidden * Q + j * Q + g.mperm_t[p * 8][kPrinted.e[k]]];
            out[j * Q + k] = static_cast<float>(v);
        }
    float* o = out + kHidden * Q;
    for (int j = 0; j < kHidden; ++j) *o++ = static_cast<float>(acc[GL::kB1 + j]);
    for (int j = 0; j < kHidden * kHidden; ++j) *o++ = static_cast<float>(acc[GL::kW2 + j]);
    for (int j = 0; j < kHidden; ++j) *o++ = static_cast<float>(acc[GL::kB2 + j]);
    if (DEEP) {
        for (int j = 0; j < kHidden * kHidden; ++j) *o++ = static_cast<float>(acc[GL::kWd + j]);
        for (int j = 0; j < kHidden; ++j) *o++ = static_cast<float>(acc[GL::kBd + j]);
    }
    for (int j = 0; j < kOut * kHidden; ++j) *o++ = static_cast<float>(acc[GL::kW3 + j]);
    for (int j = 0; j < kOut; ++j) *o++ = static_cast<float>(acc[GL::kB3 + j]);
}

void adjoint_fold_gradient(const double* acc, bool deep, float* out) {
    if (deep) fold_gradient<true>(acc, out);
    else fold_gradient<false>(acc, out);
}

}  // namespace lbm
