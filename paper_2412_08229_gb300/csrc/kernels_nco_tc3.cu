// kernels_nco_tc3.cu - the fused neural-collision step with the invariant network of
// Sec. II.B (eq. gconv_m) on the tcgen05 tensor cores to FP32-class accuracy.
//
// Every operand x is split into two BF16 numbers, x = x_hi + x_lo with x_hi = bf16(x) and
// x_lo = bf16(x - x_hi), and every product is formed in the FP32 accumulator as
// a_hi b_hi + a_hi b_lo + a_lo b_hi (three MMAs per K slice). The dropped a_lo b_lo term
// and the residual of the split are below 2^-16 of |a||b| per product, against 2^-8 for a
// plain BF16 product; sums and the relu and sigmoid stages are FP32.
//
// Per tile of 128 cells (one cell per thread and TMEM lane), 12 chunks of 4 group elements:
//   L1  D1[128 x 80] = A1 . B1_c^T, A1 = (m in the printed order, 1, 0...) split, in TMEM;
//       B1_c rows (g, j) = ((W1 P_g)[j,:], b1[j]) split, in shared memory;
//   per pair of elements g: A2_g = split(relu(D1_g), 1, 0...) into TMEM,
//       L2  D2_g[128 x 32] = A2_g . B2^T (B2 rows (W2[j,:], b2[j]) split);
//       with the third hidden layer the same once more with (W_d, b_d);
//   L3  on the CUDA cores: h = sum_g relu(D2_g) in FP32, tau~ = W3 h / 48 + b3;
//   relaxation as in the CUDA-core FP32 step: f* - w = (f - w) - M^-1 S (m - m^eq), the
//   loaded deviations kept in registers so that mass and momentum are not re-synthesised.
// Two warpgroups per CTA (one persistent CTA per SM), each owning whole tiles and 256 of
// the 512 TMEM columns: D1 [0, 80), the pair's D2 [80, 144), A1 hi/lo [144, 176), the
// pair's A2 hi/lo [176, 240). Only the weights live in shared memory (128 KB). Waits on
// MMA completion are bounded; a timeout ends the kernel early (LBM_ERR_TIMEOUT).
#include "force.cuh"
#include "tc_common.cuh"

namespace lbm {
using namespace tc;
using namespace tcc;

namespace {

constexpr int kTile = 128;
constexpr int kG = 48;
constexpr int kChunkG = 4;
constexpr int kChunks = kG / kChunkG;   // 12
constexpr int kN1 = kChunkG * kHidden;  // 80
constexpr int kK1 = 32;                 // 27 moments + bias input + pad
constexpr int kN2 = 32;                 // 20 hidden + pad
constexpr int kK2 = 32;                 // 20 hidden + bias input + pad
constexpr int kWGs = 2;

// weight image (shared-memory image): B1 hi | B1 lo | B2 hi | B2 lo | B2d hi | B2d lo | W3 | b3
constexpr uint32_t kB1ChunkBytes = kN1 * kK1 * 2;       // 5120
constexpr uint32_t kB1Bytes = kChunks * kB1ChunkBytes;  // 61440
constexpr uint32_t kB2Bytes = kN2 * kK2 * 2;            // 2048
constexpr uint32_t kB1HiOff = 0;
constexpr uint32_t kB1LoOff = kB1HiOff + kB1Bytes;
constexpr uint32_t kB2HiOff = kB1LoOff + kB1Bytes;
constexpr uint32_t kB2LoOff = kB2HiOff + kB2Bytes;
constexpr uint32_t kB2dHiOff = kB2LoOff + kB2Bytes;     // third hidden layer (deep network)
constexpr uint32_t kB2dLoOff = kB2dHiOff + kB2Bytes;
constexpr uint32_t kW3Off = kB2dLoOff + kB2Bytes;       // 80 floats
constexpr uint32_t kB3Off = kW3Off + kOut * kHidden * 4;
constexpr uint32_t kWeightBytes = kB3Off + 16;          // 131408
static_assert(kWeightBytes % 16 == 0, "weight image copies in 16-byte vectors");
constexpr uint32_t kBarOff = kWeightBytes;
// forced steps: 2 F^ as floats and the block's projection sums after the barriers
constexpr uint32_t kFhOff = kBarOff + 2 * kWGs * 8 + 16;
constexpr uint32_t kRedOff = kFhOff + 6 * kForcedModes * 4;
constexpr uint32_t kSmemBytes = kRedOff + frc::kProjValues * 8;
static_assert(kSmemBytes <= 227 * 1024, "shared memory budget");

constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kTmemPerWg = kTmemCols / kWGs;       // 256
constexpr uint32_t kD1Col = 0;                          // 80 columns
constexpr uint32_t kD2Col = 80;                         // two elements x 32
constexpr uint32_t kA1Col = 144;                        // hi (16) then lo (16)
constexpr uint32_t kA2Col = 176;                        // per element of the pair: hi (16) then lo (16)
static_assert(kA2Col + 2 * 32 <= kTmemPerWg && kD2Col + 2 * kN2 <= kA1Col && kN1 <= kD2Col, "TMEM layout");

// (x0, x1) = hi + lo as packed BF16 pairs (x0 in bits 0..15): hi rounds x to nearest,
// lo rounds the exact FP32 remainder x - hi.
__device__ __forceinline__ void split_pack(float x0, float x1, uint32_t& hi, uint32_t& lo) {
    hi = pack_bf16(x0, x1);
    const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xFFFF0000u);
    lo = pack_bf16(x0 - h0, x1 - h1);
}

template <int STORAGE, int BC, bool FORCED, bool DEEP>
__global__ void __launch_bounds__(kWGs * 128, 1) nco_tc3_kernel(const StepArgs a, const uint8_t* __restrict__ wimg,
                                                                 int ntiles, long long limit, const FusedForce ff) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const int tid = threadIdx.x;
    const int wg = tid >> 7;
    const int r = tid & 127;
    const int warp = tid >> 5;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kBarOff);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(smem + kBarOff + 2 * kWGs * 8);
    float* fh2 = reinterpret_cast<float*>(smem + kFhOff);
    unsigned long long* red = reinterpret_cast<unsigned long long*>(smem + kRedOff);

    // ---- set-up: weights to shared memory, barriers, TMEM
    for (uint32_t i = tid * 16; i < kWeightBytes; i += kWGs * 128 * 16)
        *reinterpret_cast<uint4*>(smem + i) = *reinterpret_cast<const uint4*>(wimg + i);
    if (FORCED) {
        frc::load_fh2(ff.fhat, fh2);
        if (tid < frc::kProjValues) red[tid] = 0ull;
    }
    if (tid == 0) {
        for (int b = 0; b < 2 * kWGs; ++b) mbar_init(&bars[b], 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(tmem_holder, kTmemCols);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    const uint32_t tmem = *tmem_holder + static_cast<uint32_t>(wg) * kTmemPerWg;
    const uint32_t lane = static_cast<uint32_t>((warp & 3) * 32) << 16;
    const uint32_t sW = smem_u32(smem);
    const float* W3 = reinterpret_cast<const float*>(smem + kW3Off);
    const float* b3 = reinterpret_cast<const float*>(smem + kB3Off);
    uint64_t* bar1 = &bars[2 * wg];
    uint64_t* bar2 = &bars[2 * wg + 1];
    const int bid = 1 + wg;
    uint32_t ph1 = 0, ph2 = 0;
    constexpr uint32_t id1 = idesc_bf16(128, kN1), id2 = idesc_bf16(128, kN2);
    const float omega_nu = 1.0f / a.tau;

    // relu of 20 accumulator columns -> split (relu(h), 1, 0...) as TMEM row r of an A operand
    auto relu_split_to_tmem = [&](uint32_t src, uint32_t dst) {
        uint32_t v[kHidden];
        tmem_ld16(src, v);
        tmem_ld4(src + 16, v + 16);
        tmem_ld_wait();
        uint32_t hi[16], lo[16];
#pragma unroll
        for (int i = 0; i < 10; ++i)
            split_pack(fmaxf(as_f(v[2 * i]), 0.0f), fmaxf(as_f(v[2 * i + 1]), 0.0f), hi[i], lo[i]);
        hi[10] = kBf16One;
        lo[10] = 0u;
#pragma unroll
        for (int i = 11; i < 16; ++i) hi[i] = lo[i] = 0u;
        tmem_st16(dst, hi);
        tmem_st16(dst + 16, lo);
    };
    // D (+)= A . B^T in split form over K = 32: three MMAs per K slice
    auto mma_split = [&](uint32_t d, uint32_t a_col, uint32_t b_hi, uint32_t b_lo, uint32_t kbytes, uint32_t idesc) {
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            const uint64_t dh = smem_desc(b_hi + kk * 256, 128, kbytes);
            const uint64_t dl = smem_desc(b_lo + kk * 256, 128, kbytes);
            mma_bf16_ta(d, a_col + kk * 8, dh, idesc, kk);
            mma_bf16_ta(d, a_col + kk * 8, dl, idesc, 1);
            mma_bf16_ta(d, a_col + 16 + kk * 8, dh, idesc, 1);
        }
    };
    bool ok = true;
    bool last_wait_l2 = false;  // the barrier of the last wait: its phase ph ^ 1 is the one a timeout leaves running
    long long pacc[3] = {0, 0, 0};  // forced steps: fixed-point projection sums of this thread's lane

    for (int tile = blockIdx.x * kWGs + wg; tile < ntiles; tile += gridDim.x * kWGs) {
        const long long cell = static_cast<long long>(tile) * kTile + r;
        const bool valid = cell < a.d.ncell;
        float m[Q];
        float df[Q];  // kept for the incremental relaxation, as in the CUDA-core FP32 step
        float drho = 0.0f;
        Macro q{1.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (valid) {
            int x, y, z;
            cell_coords(cell, a.d, x, y, z);
            load_pulled<STORAGE, BC>(a.src, a.d, x, y, z, df);
            drho = moments_from_dev(df, m);
            q = macro_from_moments(m, drho);
            if (!(q.rho >= a.rho_min && q.rho <= a.rho_max)) atomicOr(a.status, 1);
        } else {
#pragma unroll
            for (int e = 0; e < Q; ++e) m[e] = df[e] = 0.0f;
            m[0] = 1.0f;
        }
        {  // A1 row r: the raw moments in the printed order of Sec. II.B, the bias input 1, split
            uint32_t hi[16], lo[16];
            static_for<13>([&](auto K) {
                constexpr int k = decltype(K)::value;
                split_pack(m[kPrintedE<2 * k>], m[kPrintedE<2 * k + 1>], hi[k], lo[k]);
            });
            split_pack(m[kPrintedE<26>], 1.0f, hi[13], lo[13]);
            hi[14] = hi[15] = lo[14] = lo[15] = 0u;
            tmem_st16(tmem + lane + kA1Col, hi);
            tmem_st16(tmem + lane + kA1Col + 16, lo);
            tmem_st_wait();
        }
        tc_fence_before();
        if (!(ok = wg_sync_and(bid, ok))) break;

        float acc[kHidden];
#pragma unroll
        for (int j = 0; j < kHidden; ++j) acc[j] = 0.0f;
        for (int c = 0; c < kChunks; ++c) {
            // ---- layer 1 for four group elements
            if (r == 0) {
                tc_fence_after();
                mma_split(tmem + kD1Col, tmem + kA1Col, sW + kB1HiOff + c * kB1ChunkBytes,
                          sW + kB1LoOff + c * kB1ChunkBytes, 128 * kK1 / 8, id1);
                mma_commit(bar1);
            }
            last_wait_l2 = false;
            bool w_ok = wait_phase(bar1, ph1, limit);
            ph1 ^= 1u;
            tc_fence_after();
#pragma unroll 1
            for (int pr = 0; pr < kChunkG / 2; ++pr) {
                // ---- layer 2 for the pair (2 pr, 2 pr + 1)
#pragma unroll
                for (int e = 0; e < 2; ++e)
                    relu_split_to_tmem(tmem + lane + kD1Col + kHidden * (2 * pr + e), tmem + lane + kA2Col + 32 * e);
                tmem_st_wait();
                tc_fence_before();
                if (!(ok = wg_sync_and(bid, w_ok))) break;
                if (r == 0) {
                    tc_fence_after();
#pragma unroll
                    for (int e = 0; e < 2; ++e)
                        mma_split(tmem + kD2Col + kN2 * e, tmem + kA2Col + 32 * e, sW + kB2HiOff, sW + kB2LoOff,
                                  128 * kK2 / 8, id2);
                    mma_commit(bar2);
                }
                last_wait_l2 = true;
                w_ok = wait_phase(bar2, ph2, limit);
                ph2 ^= 1u;
                tc_fence_after();
                if constexpr (DEEP) {  // third hidden layer: split relu(h2) into A2, W_d written over D2
#pragma unroll
                    for (int e = 0; e < 2; ++e)
                        relu_split_to_tmem(tmem + lane + kD2Col + kN2 * e, tmem + lane + kA2Col + 32 * e);
                    tmem_st_wait();
                    tc_fence_before();
                    if (!(ok = wg_sync_and(bid, w_ok))) break;
                    if (r == 0) {
                        tc_fence_after();
#pragma unroll
                        for (int e = 0; e < 2; ++e)
                            mma_split(tmem + kD2Col + kN2 * e, tmem + kA2Col + 32 * e, sW + kB2dHiOff,
                                      sW + kB2dLoOff, 128 * kK2 / 8, id2);
                        mma_commit(bar2);
                    }
                    last_wait_l2 = true;
                    w_ok = wait_phase(bar2, ph2, limit);
                    ph2 ^= 1u;
                    tc_fence_after();
                }
#pragma unroll
                for (int e = 0; e < 2; ++e) {  // output-layer input: the last relu(h) summed over the group
                    uint32_t v[kHidden];
                    tmem_ld16(tmem + lane + kD2Col + kN2 * e, v);
                    tmem_ld4(tmem + lane + kD2Col + kN2 * e + 16, v + 16);
                    tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < kHidden; j += 2) add2_relu(acc[j], acc[j + 1], as_f(v[j]), as_f(v[j + 1]));
                }
                tc_fence_before();
                if (!(ok = wg_sync_and(bid, w_ok))) break;  // D2 and A2 read before they are rewritten
            }
            if (!ok) break;
        }
        if (!ok) break;
        frc::Cx ph[kForcedModes];  // forced steps: the phases of the 16 modes at this cell
        if (FORCED) {
            int x = 0, y = 0, z = 0;
            if (valid) cell_coords(cell, a.d, x, y, z);
            frc::cell_phases(x, y, z, a.d, ff.tab, ph);
        }
        if (valid) {
            float rates[kOut];
#pragma unroll
            for (int n = 0; n < kOut; ++n) {
                float t = 0.0f;
#pragma unroll
                for (int j = 0; j < kHidden; ++j) t = fmaf(W3[n * kHidden + j], acc[j], t);
                rates[n] = rate_from_output(t * (1.0f / 48.0f) + b3[n]);
            }
            // f* - w = (f - w) - M^-1 S (m - m^eq): the conserved moments are not re-synthesised
            collide_mrt(df, m, q, omega_nu, rates);
            if (FORCED) {  // F(x) from this step's coefficients
                float F[3];
                frc::synth_force(fh2, ph, F);
                add_kupershtokh(df, q, F[0], F[1], F[2]);
            }
            store_cell<STORAGE>(a.dst, a.d, cell, df);
        }
        if (FORCED && ff.proj) frc::project_warp(q.ux, q.uy, q.uz, ph, tid & 31, pacc, ff.scale);
    }
    if (FORCED && ff.proj) frc::proj_to_shared(red, pacc, tid & 31);
    bool drained = true;
    if (!ok && r == 0) {
        atomicOr(a.status, 2);
        // At most one commit is outstanding: wait, with the full limit, for the phase the
        // warpgroup gave up on, so that no MMA still uses TMEM when it is released.
        drained = last_wait_l2 ? wait_phase(bar2, ph2 ^ 1u) : wait_phase(bar1, ph1 ^ 1u);
    }
    tc_fence_before();
    if (!__syncthreads_and(drained)) {
        if (threadIdx.x == 0) atomicOr(a.status, 4);  // MMAs still running: TMEM is left allocated
        return;
    }
    if (FORCED && ff.proj && ok) frc::proj_to_global(red, ff.proj);
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(*tmem_holder, kTmemCols);
    }
}

template <int STORAGE, int BC, bool FORCED, bool DEEP>
cudaError_t launch_tc3_t(const StepArgs& a, const FusedForce& ff, const void* w, long long wait, cudaStream_t s) {
    static std::atomic<unsigned long long> attr{0};
    const cudaError_t e = ensure_dynamic_smem(nco_tc3_kernel<STORAGE, BC, FORCED, DEEP>, static_cast<int>(kSmemBytes),
                                              attr);
    if (e != cudaSuccess) return e;
    const int ntiles = static_cast<int>((a.d.ncell + kTile - 1) / kTile);
    int grid = (ntiles + kWGs - 1) / kWGs;
    if (grid > sm_count()) grid = sm_count();
    if (grid < 1) return cudaSuccess;
    nco_tc3_kernel<STORAGE, BC, FORCED, DEEP><<<grid, kWGs * 128, kSmemBytes, s>>>(a, static_cast<const uint8_t*>(w),
                                                                                   ntiles, wait, ff);
    return cudaGetLastError();
}

template <int STORAGE, int BC, bool FORCED>
cudaError_t launch_tc3_f(const StepArgs& a, const FusedForce& ff, bool deep, const void* w, long long wait,
                         cudaStream_t s) {
    return deep ? launch_tc3_t<STORAGE, BC, FORCED, true>(a, ff, w, wait, s)
                : launch_tc3_t<STORAGE, BC, FORCED, false>(a, ff, w, wait, s);
}

template <int STORAGE>
cudaError_t launch_tc3_b(const StepArgs& a, const FusedForce* ff, int bc, bool deep, const void* w, long long wait,
                         cudaStream_t s) {
    const FusedForce nf{};
    if (ff) {  // forcing runs on periodic boxes only
        if (bc != LBM_BC_PERIODIC) return cudaErrorInvalidValue;
        return launch_tc3_f<STORAGE, LBM_BC_PERIODIC, true>(a, *ff, deep, w, wait, s);
    }
    if (bc == LBM_BC_TGV_REDUCED) return launch_tc3_f<STORAGE, LBM_BC_TGV_REDUCED, false>(a, nf, deep, w, wait, s);
    return bc == LBM_BC_PERIODIC ? launch_tc3_f<STORAGE, LBM_BC_PERIODIC, false>(a, nf, deep, w, wait, s)
                                 : launch_tc3_f<STORAGE, LBM_BC_MIRROR, false>(a, nf, deep, w, wait, s);
}

}  // namespace

size_t nco_tc3_weight_bytes() { return kWeightBytes; }

void nco_tc3_pack_weights(const float* theta, bool deep, void* out) {
    const float* W1 = theta;  // (20, 27), printed moment order
    const float* b1 = W1 + kHidden * Q;
    const float* W2 = b1 + kHidden;
    const float* b2 = W2 + kHidden * kHidden;
    const float* Wd = b2 + kHidden;  // deep network: the third hidden layer comes next
    const float* bd = Wd + kHidden * kHidden;
    const float* W3 = deep ? bd + kHidden : b2 + kHidden;
    const float* b3 = W3 + kOut * kHidden;
    uint8_t* img = static_cast<uint8_t*>(out);
    std::memset(img, 0, kWeightBytes);
    // v = hi + lo in BF16 at (row, k) of the K-major images at hi_base and lo_base
    auto put = [&](uint32_t hi_base, uint32_t lo_base, int row, int k, int K, float v) {
        const uint16_t h = f2bf(v);
        const uint32_t hb = static_cast<uint32_t>(h) << 16;
        float hv;
        std::memcpy(&hv, &hb, 4);
        const uint16_t l = f2bf(v - hv);
        std::memcpy(img + hi_base + kmajor_offset(row, k, K), &h, 2);
        std::memcpy(img + lo_base + kmajor_offset(row, k, K), &l, 2);
    };
    const GroupTables& gt = group_tables();
    for (int g = 0; g < kG; ++g) {
        const int c = g / kChunkG, gl = g % kChunkG;
        const uint32_t hb = kB1HiOff + c * kB1ChunkBytes, lb = kB1LoOff + c * kB1ChunkBytes;
        for (int j = 0; j < kHidden; ++j) {
            const int row = gl * kHidden + j;
            // (W1 P_g m)_j = sum_k W1[j][k] msign[g][k] m[mperm[g][k]] (printed order)
            for (int k = 0; k < Q; ++k) {
                const int e = kPrinted.e[k];
                int kp = 0;
                for (int t = 0; t < Q; ++t)
                    if (kPrinted.e[t] == gt.mperm_t[g][e]) kp = t;
                put(hb, lb, row, kp, kK1, W1[j * Q + k] * static_cast<float>(gt.msign_t[g][e]));
            }
            put(hb, lb, row, Q, kK1, b1[j]);
        }
    }
    for (int j = 0; j < kHidden; ++j) {
        for (int k = 0; k < kHidden; ++k) put(kB2HiOff, kB2LoOff, j, k, kK2, W2[j * kHidden + k]);
        put(kB2HiOff, kB2LoOff, j, kHidden, kK2, b2[j]);
        if (deep) {
            for (int k = 0; k < kHidden; ++k) put(kB2dHiOff, kB2dLoOff, j, k, kK2, Wd[j * kHidden + k]);
            put(kB2dHiOff, kB2dLoOff, j, kHidden, kK2, bd[j]);
        }
    }
    std::memcpy(img + kW3Off, W3, kOut * kHidden * sizeof(float));
    std::memcpy(img + kB3Off, b3, kOut * sizeof(float));
}

cudaError_t launch_step_nco_tc3(const StepArgs& a, const FusedForce* ff, int storage, int bc, bool deep, const void* w,
                                long long wait_cycles, cudaStream_t s) {
    switch (storage) {
        case LBM_STORE_F32: return launch_tc3_b<LBM_STORE_F32>(a, ff, bc, deep, w, wait_cycles, s);
        case LBM_STORE_F16_DEV: return launch_tc3_b<LBM_STORE_F16_DEV>(a, ff, bc, deep, w, wait_cycles, s);
        default: return launch_tc3_b<LBM_STORE_BF16_DEV>(a, ff, bc, deep, w, wait_cycles, s);
    }
}

}  // namespace lbm
