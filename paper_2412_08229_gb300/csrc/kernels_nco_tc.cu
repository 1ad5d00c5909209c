// kernels_nco_tc.cu - the fused neural-collision step with the invariant network of
// Sec. II.B (eq. gconv_m) on the tcgen05 tensor cores: BF16 operands in shared memory,
// FP32 accumulators in tensor memory (TMEM).
//
// Per tile of 128 cells (M = 128, one cell per thread and TMEM lane) the 48 elements g of
// O_h are walked in 12 chunks of 4:
//   L1  D1[128 x 80]  = A1[128 x 32] . B1_c^T   A1 = (m in the printed order, 1, 0...),
//                                              B1_c rows (g, j) = ((W1 P_g)[j,:], b1[j]);
//   L2  D2_g[128 x 32] = A2_g . B2^T            A2_g = (relu(D1_g), 1, 0...), B2 rows j =
//                                              (W2[j,:], b2[j]); written over D1's columns;
//   L3  on the CUDA cores: h = sum_g relu(D2_g) in FP32 registers (packed FP32 adds),
//       tau~ = W3 h / 48 + b3 (layer 3 is affine, so the group mean moves inside it).
// Design notes from measurements on GB300 (M = 128, K = 16, BF16):
//  * the tensor pipe spends 40 (N <= 32) to 52 (N = 80) cycles on an MMA whose A operand
//    is in shared memory (reading the 4 KB A tile dominates), 18-24 cycles (N <= 48) when
//    A is in TMEM; one issuing thread starts at most one MMA every ~61 cycles;
//  * timestamps inside this kernel at 256^3: a warpgroup spends ~45k cycles on a tile,
//    43% of it in MMA round trips (issue to completion seen: ~600 cycles for L1, ~1000
//    for the eight L2 MMAs, which queue behind the other warpgroups' MMAs), 28% in the
//    epilogues, 12% in barriers and 15% in the per-cell load, moments, relaxation and store;
//  * layouts that move A2/A3 into TMEM need more than the 128 TMEM columns a warpgroup has
//    when four warpgroups share an SM, and the variants that fit (pairs of elements, or
//    three elements with a block-diagonal L2) trade cheaper MMAs for more round trips and
//    measured slower; so did layer 3 on the tensor pipe (8 more MMAs per chunk) and L2
//    issued from four warps.
// Each warpgroup owns whole tiles, issues its own MMAs from one thread and synchronises
// with named barriers; the warpgroups of a CTA (one persistent CTA per SM) interleave on
// the tensor pipe and hide each other's latency. This kernel steps the deep network and
// batches (kernels_nco_tcp.cu steps single instances of the two-layer network). Waits on
// MMA completion are bounded in time by the compile-time default; a timeout ends the
// kernel early and is reported as LBM_ERR_TIMEOUT. Shared-memory operands use the K-major,
// no-swizzle core-matrix layout of tc_ptx.cuh.
#include <cstring>

#include "force.cuh"
#include "tc_common.cuh"

namespace lbm {
using namespace tc;
using namespace tcc;

namespace {

constexpr int kTile = 128;
constexpr int kG = 48;
constexpr int kChunkG = 4;
constexpr int kChunks = kG / kChunkG;       // 12
constexpr int kN1 = kChunkG * kHidden;      // 80
constexpr int kK1 = 32;                     // 27 moments + bias input + pad
constexpr int kN2 = 32;                     // 20 hidden + pad
constexpr int kK2 = 32;                     // 20 hidden + bias input + pad

// packed weight image = shared-memory image: B1 (12 chunks), B2, W3 and b3 as floats
constexpr uint32_t kB1ChunkBytes = kN1 * kK1 * 2;       // 5120
constexpr uint32_t kB1Bytes = kChunks * kB1ChunkBytes;  // 61440
constexpr uint32_t kB2Bytes = kN2 * kK2 * 2;            // 2048
constexpr uint32_t kB1Off = 0;
constexpr uint32_t kB2Off = kB1Off + kB1Bytes;
constexpr uint32_t kB2dOff = kB2Off + kB2Bytes;           // third hidden layer (deep network)
constexpr uint32_t kW3Off = kB2dOff + kB2Bytes;           // 80 floats
constexpr uint32_t kB3Off = kW3Off + kOut * kHidden * 4;  // 4 floats
constexpr uint32_t kWeightBytes = kB3Off + 16;            // 65872, a multiple of 16
static_assert(kWeightBytes % 16 == 0, "weight image copies in 16-byte vectors");

constexpr uint32_t kA1Bytes = kTile * kK1 * 2;           // 8192
constexpr uint32_t kA2GBytes = kTile * kK2 * 2;          // 8192 per group element
constexpr uint32_t kA2Bytes = kChunkG * kA2GBytes;       // 32768
constexpr uint32_t kWgBytes = kA1Bytes + kA2Bytes;       // 40960
constexpr uint32_t kWgOff = (kWeightBytes + 1023) / 1024 * 1024;
template <int NWG> constexpr uint32_t bar_off() { return kWgOff + NWG * kWgBytes; }
// forced steps: 2 F^ as floats and the block's projection sums after the barriers
template <int NWG> constexpr uint32_t fh_off() { return bar_off<NWG>() + 2 * NWG * 8 + 16; }
template <int NWG> constexpr uint32_t red_off() { return fh_off<NWG>() + 6 * kForcedModes * 4; }
template <int NWG> constexpr uint32_t smem_bytes() { return red_off<NWG>() + frc::kProjValues * 8; }

static_assert(smem_bytes<4>() <= 227 * 1024, "shared memory budget");
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kTmemPerWg = 128;                      // D1 (80) then D2 (4 x 32) in place
static_assert(kChunkG * kN2 <= kTmemPerWg && kN1 <= kTmemPerWg, "TMEM budget");

template <int STORAGE, int BC, bool FORCED, int kWGs, bool BATCHED, bool DEEP>
__global__ void __launch_bounds__(kWGs * 128, 1) nco_tc_kernel(const StepArgs a0, const BatchTiles bt,
                                                                const uint8_t* __restrict__ wimg, int ntiles,
                                                                const FusedForce ff) {
    extern __shared__ __align__(1024) uint8_t smem[];
    constexpr int kThreads = kWGs * 128;
    const int tid = threadIdx.x;
    const int wg = tid >> 7;
    const int r = tid & 127;
    const int warp = tid >> 5;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + bar_off<kWGs>());
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(smem + bar_off<kWGs>() + 2 * kWGs * 8);
    float* fh2 = reinterpret_cast<float*>(smem + fh_off<kWGs>());
    unsigned long long* red = reinterpret_cast<unsigned long long*>(smem + red_off<kWGs>());

    // ---- set-up: weights to shared memory, zeroed operand buffers, barriers, TMEM
    for (uint32_t i = tid * 16; i < kWeightBytes; i += kThreads * 16)
        *reinterpret_cast<uint4*>(smem + i) = *reinterpret_cast<const uint4*>(wimg + i);
    for (uint32_t i = kWgOff + tid * 16; i < bar_off<kWGs>(); i += kThreads * 16)
        *reinterpret_cast<uint4*>(smem + i) = make_uint4(0, 0, 0, 0);
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
    const uint32_t sB1 = smem_u32(smem + kB1Off), sB2 = smem_u32(smem + kB2Off), sB2d = smem_u32(smem + kB2dOff);
    const uint32_t sA1 = smem_u32(smem + kWgOff + wg * kWgBytes);
    const uint32_t sA2 = sA1 + kA1Bytes;
    const float* W3 = reinterpret_cast<const float*>(smem + kW3Off);
    const float* b3 = reinterpret_cast<const float*>(smem + kB3Off);
    uint64_t* bar1 = &bars[2 * wg];
    uint64_t* bar2 = &bars[2 * wg + 1];
    const int bid = 1 + wg;
    uint32_t ph1 = 0, ph2 = 0;
    constexpr uint32_t id1 = idesc_bf16(128, kN1), id2 = idesc_bf16(128, kN2);
    // 20 accumulator columns of one group element -> (relu(.) in BF16, 1, 0...) as row r of
    // the next layer's K-major operand
    auto relu_to_operand = [&](uint32_t taddr, uint32_t gb) {
        uint32_t v[kHidden];
        tmem_ld16(taddr, v);
        tmem_ld4(taddr + 16, v + 16);
        tmem_ld_wait();
        uint32_t h[10];
#pragma unroll
        for (int i = 0; i < 10; ++i) h[i] = pack_bf16_relu(as_f(v[2 * i]), as_f(v[2 * i + 1]));
        st_shared_v4(gb + kmajor_offset(r, 0, kK2), h[0], h[1], h[2], h[3]);
        st_shared_v4(gb + kmajor_offset(r, 8, kK2), h[4], h[5], h[6], h[7]);
        st_shared_v4(gb + kmajor_offset(r, 16, kK2), h[8], h[9], kBf16One, 0u);
    };
    bool ok = true;
    bool last_wait_l2 = false;  // the barrier of the last wait: its phase ph ^ 1 is the one a timeout leaves running
    long long pacc[3] = {0, 0, 0};  // forced steps: fixed-point projection sums of this thread's lane

    for (int gtile = blockIdx.x * kWGs + wg; gtile < ntiles; gtile += gridDim.x * kWGs) {
        int tile = gtile;
        StepArgs a = a0;
        if (BATCHED) {  // the instance owning this tile
            const int i = __ldg(&bt.tile_inst[gtile]);
            a = bt.inst[i];
            tile = gtile - static_cast<int>(__ldg(&bt.tile_begin[i]));
        }
        const float omega_nu = 1.0f / a.tau;
        const long long cell = static_cast<long long>(tile) * kTile + r;
        const bool valid = cell < a.d.ncell;
        float m[Q];
        float drho = 0.0f;
        Macro q{1.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (valid) {
            int x, y, z;
            cell_coords(cell, a.d, x, y, z);
            float df[Q];
            load_pulled<STORAGE, BC>(a.src, a.d, x, y, z, df);
            drho = moments_from_dev(df, m);
            q = macro_from_moments(m, drho);
            if (!(q.rho >= a.rho_min && q.rho <= a.rho_max)) atomicOr(a.status, 1);
            if (BATCHED && a.u_out) {
                a.u_out[cell] = q.ux;
                a.u_out[a.d.ncell + cell] = q.uy;
                a.u_out[2 * a.d.ncell + cell] = q.uz;
            }
        } else {
#pragma unroll
            for (int e = 0; e < Q; ++e) m[e] = 0.0f;
            m[0] = 1.0f;
        }
        {  // A1 row r: the raw moments in the printed order of Sec. II.B, then the bias input 1
            uint32_t p[16];
            static_for<13>([&](auto K) {
                constexpr int k = decltype(K)::value;
                p[k] = pack_bf16(m[kPrintedE<2 * k>], m[kPrintedE<2 * k + 1>]);
            });
            p[13] = pack_bf16(m[kPrintedE<26>], 1.0f);
            p[14] = 0u;
            p[15] = 0u;
#pragma unroll
            for (int kc = 0; kc < 4; ++kc)
                st_shared_v4(sA1 + kmajor_offset(r, 8 * kc, kK1), p[4 * kc], p[4 * kc + 1], p[4 * kc + 2], p[4 * kc + 3]);
        }
        fence_proxy_async_smem();
        tc_fence_before();
        if (!(ok = wg_sync_and(bid, ok))) break;

        float acc[kHidden];
#pragma unroll
        for (int j = 0; j < kHidden; ++j) acc[j] = 0.0f;
        for (int c = 0; c < kChunks; ++c) {
            // ---- layer 1 for four group elements
            if (r == 0) {
                tc_fence_after();
#pragma unroll
                for (int kk = 0; kk < kK1 / 16; ++kk)
                    mma_bf16(tmem, smem_desc(sA1 + kk * 256, 128, 128 * kK1 / 8),
                             smem_desc(sB1 + c * kB1ChunkBytes + kk * 256, 128, 128 * kK1 / 8), id1, kk);
                mma_commit(bar1);
            }
            last_wait_l2 = false;
            bool w_ok = wait_phase(bar1, ph1);
            ph1 ^= 1u;
            tc_fence_after();
#pragma unroll
            for (int g = 0; g < kChunkG; ++g) relu_to_operand(tmem + lane + kHidden * g, sA2 + g * kA2GBytes);
            fence_proxy_async_smem();
            tc_fence_before();
            if (!(ok = wg_sync_and(bid, w_ok))) break;

            // ---- layer 2: one MMA pair per group element, written over D1
            if (r == 0) {
                tc_fence_after();
#pragma unroll
                for (int g = 0; g < kChunkG; ++g)
#pragma unroll
                    for (int kk = 0; kk < kK2 / 16; ++kk)
                        mma_bf16(tmem + kN2 * g, smem_desc(sA2 + g * kA2GBytes + kk * 256, 128, 128 * kK2 / 8),
                                 smem_desc(sB2 + kk * 256, 128, 128 * kK2 / 8), id2, kk);
                mma_commit(bar2);
            }
            last_wait_l2 = true;
            w_ok = wait_phase(bar2, ph2);
            ph2 ^= 1u;
            tc_fence_after();
            if constexpr (DEEP) {  // third hidden layer: relu(h2) into A2, then W_d written over D2
#pragma unroll
                for (int g = 0; g < kChunkG; ++g) relu_to_operand(tmem + lane + kN2 * g, sA2 + g * kA2GBytes);
                fence_proxy_async_smem();
                tc_fence_before();
                if (!(ok = wg_sync_and(bid, w_ok))) break;
                if (r == 0) {
                    tc_fence_after();
#pragma unroll
                    for (int g = 0; g < kChunkG; ++g)
#pragma unroll
                        for (int kk = 0; kk < kK2 / 16; ++kk)
                            mma_bf16(tmem + kN2 * g, smem_desc(sA2 + g * kA2GBytes + kk * 256, 128, 128 * kK2 / 8),
                                     smem_desc(sB2d + kk * 256, 128, 128 * kK2 / 8), id2, kk);
                    mma_commit(bar2);
                }
                last_wait_l2 = true;
                w_ok = wait_phase(bar2, ph2);
                ph2 ^= 1u;
                tc_fence_after();
            }
#pragma unroll
            for (int g = 0; g < kChunkG; ++g) {  // output-layer input: the last relu(h) summed over the group
                uint32_t v[kHidden];
                tmem_ld16(tmem + lane + kN2 * g, v);
                tmem_ld4(tmem + lane + kN2 * g + 16, v + 16);
                tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < kHidden; j += 2) add2_relu(acc[j], acc[j + 1], as_f(v[j]), as_f(v[j + 1]));
            }
            tc_fence_before();
            if (!(ok = wg_sync_and(bid, w_ok))) break;  // D2 read before the next layer 1 overwrites it
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
            float df[Q];
            relax_to_populations(m, drho, q, omega_nu, rates, df);
            if (FORCED) {  // F(x) from this step's coefficients
                float F[3];
                frc::synth_force(fh2, ph, F);
                add_kupershtokh(df, q, F[0], F[1], F[2]);
            } else if (BATCHED && a.force) {
                add_kupershtokh(df, q, a.force[cell], a.force[a.d.ncell + cell], a.force[2 * a.d.ncell + cell]);
            }
            store_cell<STORAGE>(a.dst, a.d, cell, df);
        }
        if (FORCED && ff.proj) frc::project_warp(q.ux, q.uy, q.uz, ph, tid & 31, pacc, ff.scale);
    }
    if (FORCED && ff.proj) frc::proj_to_shared(red, pacc, tid & 31);
    bool drained = true;
    if (!ok && r == 0) {
        atomicOr(a0.status, 2);
        // At most one commit is outstanding (every commit is waited on before the next MMA
        // is issued): wait, with the full limit, for the phase the warpgroup gave up on, so
        // that no MMA still writes TMEM when it is released.
        drained = last_wait_l2 ? wait_phase(bar2, ph2 ^ 1u) : wait_phase(bar1, ph1 ^ 1u);
    }
    tc_fence_before();
    if (!__syncthreads_and(drained)) {
        if (tid == 0) atomicOr(a0.status, 4);  // MMAs still running: TMEM is left allocated
        return;
    }
    if (FORCED && ff.proj && ok) frc::proj_to_global(red, ff.proj);
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(*tmem_holder, kTmemCols);
    }
}

// ---------------------------------------------------------------------------
// Self-test: one CTA multiplies deterministic BF16 matrices with tcgen05 in the two shapes
// the network uses (M = 128 with N/K = 80/32 and 32/32) and in N/K = 16/80, and compares
// every result with a CUDA-core FP32 dot product of the same BF16 values.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float test_val(uint32_t which, uint32_t row, uint32_t k) {
    uint32_t h = which * 0x9E3779B1u ^ (row * 0x85EBCA77u) ^ (k * 0xC2B2AE3Du);
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    // small integers / 8: exactly representable in BF16, exact products and sums in FP32
    return static_cast<float>(static_cast<int>(h % 17u) - 8) * 0.125f;
}

__global__ void __launch_bounds__(128, 1) tc_selftest_kernel(float* max_err, int* status) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const int r = threadIdx.x;
    const int warp = r >> 5;
    // regions: A(128 x 80) 20480 B, B(80 x 80) 12800 B, bars, holder
    const uint32_t sA = smem_u32(smem), sB = smem_u32(smem + 20480);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 20480 + 12800);
    uint32_t* holder = reinterpret_cast<uint32_t*>(smem + 20480 + 12800 + 8);
    if (r == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(holder, 128);
    struct Shape { int N, K; };
    const Shape shapes[3] = {{80, 32}, {32, 32}, {16, 80}};
    float worst = 0.0f;
    uint32_t ph = 0;
    bool ok = true;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *holder;
    for (int s = 0; s < 3; ++s) {
        const int N = shapes[s].N, K = shapes[s].K;
        // A row r and B rows (r < N) in the K-major core-matrix layout
        for (int k = 0; k < K; k += 2) {
            const uint32_t pa = pack_bf16(test_val(2 * s, r, k), test_val(2 * s, r, k + 1));
            asm volatile("st.shared.b32 [%0], %1;" ::"r"(sA + kmajor_offset(r, k, K)), "r"(pa) : "memory");
            if (r < N) {
                const uint32_t pb = pack_bf16(test_val(2 * s + 1, r, k), test_val(2 * s + 1, r, k + 1));
                asm volatile("st.shared.b32 [%0], %1;" ::"r"(sB + kmajor_offset(r, k, K)), "r"(pb) : "memory");
            }
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (r == 0) {
            tc_fence_after();
            for (int kk = 0; kk < K / 16; ++kk)
                mma_bf16(tmem, smem_desc(sA + kk * 256, 128, 16 * K), smem_desc(sB + kk * 256, 128, 16 * K),
                         idesc_bf16(128, N), kk);
            mma_commit(bar);
        }
        const bool w = wait_phase(bar, ph);
        ok = __syncthreads_and(w) && ok;  // uniform across the CTA
        if (!ok) break;
        ph ^= 1u;
        tc_fence_after();
        for (int n0 = 0; n0 < N; n0 += 16) {
            uint32_t v[16];
            tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + n0, v);
            tmem_ld_wait();
            for (int j = 0; j < 16 && n0 + j < N; ++j) {
                float ref = 0.0f;
                for (int k = 0; k < K; ++k) ref += test_val(2 * s, r, k) * test_val(2 * s + 1, n0 + j, k);
                worst = fmaxf(worst, fabsf(as_f(v[j]) - ref));
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    bool drained = true;
    if (!ok && r == 0) {
        atomicOr(status, 2);
        drained = wait_phase(bar, ph);  // the phase given up on: its MMAs must finish before TMEM is released
    }
    atomicMax(reinterpret_cast<int*>(max_err), __float_as_int(worst));
    tc_fence_before();
    if (!__syncthreads_and(drained)) {
        if (r == 0) atomicOr(status, 4);
        return;
    }
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 128);
    }
}


template <int STORAGE, int BC, bool FORCED, int NWG, bool BATCHED, bool DEEP = false>
cudaError_t launch_tc_t(const StepArgs& a, const BatchTiles& bt, const void* w, int ntiles, const FusedForce& ff,
                        cudaStream_t s) {
    static std::atomic<unsigned long long> attr{0};
    const cudaError_t e = ensure_dynamic_smem(nco_tc_kernel<STORAGE, BC, FORCED, NWG, BATCHED, DEEP>,
                                              static_cast<int>(smem_bytes<NWG>()), attr);
    if (e != cudaSuccess) return e;
    int grid = (ntiles + NWG - 1) / NWG;
    if (grid > sm_count()) grid = sm_count();
    if (grid < 1) return cudaSuccess;
    nco_tc_kernel<STORAGE, BC, FORCED, NWG, BATCHED, DEEP>
        <<<grid, NWG * 128, smem_bytes<NWG>(), s>>>(a, bt, static_cast<const uint8_t*>(w), ntiles, ff);
    return cudaGetLastError();
}

template <int STORAGE, int BC, bool FORCED>
cudaError_t launch_tc_f(const StepArgs& a, const FusedForce& ff, bool deep, const void* w, cudaStream_t s) {
    const int ntiles = static_cast<int>((a.d.ncell + kTile - 1) / kTile);
    const BatchTiles none{nullptr, nullptr, nullptr, 0};
    return deep ? launch_tc_t<STORAGE, BC, FORCED, 4, false, true>(a, none, w, ntiles, ff, s)
                : launch_tc_t<STORAGE, BC, FORCED, 4, false>(a, none, w, ntiles, ff, s);
}

template <int STORAGE>
cudaError_t launch_tc_b(const StepArgs& a, const FusedForce* ff, int bc, bool deep, const void* w, cudaStream_t s) {
    const FusedForce nf{};
    if (ff) {  // forcing runs on periodic boxes only
        if (bc != LBM_BC_PERIODIC) return cudaErrorInvalidValue;
        return launch_tc_f<STORAGE, LBM_BC_PERIODIC, true>(a, *ff, deep, w, s);
    }
    if (bc == LBM_BC_TGV_REDUCED) return launch_tc_f<STORAGE, LBM_BC_TGV_REDUCED, false>(a, nf, deep, w, s);
    return bc == LBM_BC_PERIODIC ? launch_tc_f<STORAGE, LBM_BC_PERIODIC, false>(a, nf, deep, w, s)
                                 : launch_tc_f<STORAGE, LBM_BC_MIRROR, false>(a, nf, deep, w, s);
}

template <int STORAGE>
cudaError_t launch_tc_batch_s(const StepArgs& status_args, const BatchTiles& bt, long long ntiles, int nwg,
                              const void* w, cudaStream_t s) {
    const int nt = static_cast<int>(ntiles);
    const FusedForce nf{};
    switch (nwg) {
        case 2: return launch_tc_t<STORAGE, LBM_BC_PERIODIC, false, 2, true>(status_args, bt, w, nt, nf, s);
        case 3: return launch_tc_t<STORAGE, LBM_BC_PERIODIC, false, 3, true>(status_args, bt, w, nt, nf, s);
        default: return launch_tc_t<STORAGE, LBM_BC_PERIODIC, false, 4, true>(status_args, bt, w, nt, nf, s);
    }
}

}  // namespace

bool nco_tc_supported(int, int) { return true; }
// The image holds this kernel's layout (deep network, batches) followed by the pair layout
// of the pipelined kernel (kernels_nco_tcp.cu), which steps single two-layer instances.
size_t nco_tc_weight_bytes() { return kWeightBytes + nco_tcp_weight_bytes(); }

void nco_tc_pack_weights(const float* theta, bool deep, void* out) {
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
    auto put = [&](uint32_t base, int row, int k, int K, float v) {
        const uint16_t b = f2bf(v);
        std::memcpy(img + base + kmajor_offset(row, k, K), &b, 2);
    };
    const GroupTables& gt = group_tables();
    for (int g = 0; g < kG; ++g) {
        const int c = g / kChunkG, gl = g % kChunkG;
        for (int j = 0; j < kHidden; ++j) {
            const int row = gl * kHidden + j;
            // (W1 P_g m)_j = sum_k W1[j][k] msign[g][k] m[mperm[g][k]] (printed order)
            for (int k = 0; k < Q; ++k) {
                const int e = kPrinted.e[k];
                int kp = 0;
                for (int t = 0; t < Q; ++t)
                    if (kPrinted.e[t] == gt.mperm_t[g][e]) kp = t;
                put(kB1Off + c * kB1ChunkBytes, row, kp, kK1, W1[j * Q + k] * static_cast<float>(gt.msign_t[g][e]));
            }
            put(kB1Off + c * kB1ChunkBytes, row, Q, kK1, b1[j]);
        }
    }
    for (int j = 0; j < kHidden; ++j) {
        for (int k = 0; k < kHidden; ++k) put(kB2Off, j, k, kK2, W2[j * kHidden + k]);
        put(kB2Off, j, kHidden, kK2, b2[j]);
        if (deep) {
            for (int k = 0; k < kHidden; ++k) put(kB2dOff, j, k, kK2, Wd[j * kHidden + k]);
            put(kB2dOff, j, kHidden, kK2, bd[j]);
        }
    }
    std::memcpy(img + kW3Off, W3, kOut * kHidden * sizeof(float));
    std::memcpy(img + kB3Off, b3, kOut * sizeof(float));
    if (!deep) nco_tcp_pack_weights(theta, img + kWeightBytes);
}

cudaError_t launch_step_nco_tc(const StepArgs& a, const FusedForce* ff, int storage, int bc, bool deep, int tc_shape,
                               long long wait_cycles, const void* w, cudaStream_t s) {
    if (!deep && tc_shape == 0)
        return launch_step_nco_tcp(a, ff, storage, bc, static_cast<const uint8_t*>(w) + kWeightBytes, wait_cycles, s);
    switch (storage) {
        case LBM_STORE_F32: return launch_tc_b<LBM_STORE_F32>(a, ff, bc, deep, w, s);
        case LBM_STORE_F16_DEV: return launch_tc_b<LBM_STORE_F16_DEV>(a, ff, bc, deep, w, s);
        default: return launch_tc_b<LBM_STORE_BF16_DEV>(a, ff, bc, deep, w, s);
    }
}

cudaError_t launch_step_nco_tc_batch(const StepArgs* d_inst, const long long* d_tile_begin, const int* d_tile_inst,
                                     int ninst, long long ntiles, int storage, int tc_shape, int* status, const void* w,
                                     cudaStream_t s) {
    if (tc_shape == 0)
        return launch_step_nco_tcp_batch(d_inst, d_tile_begin, d_tile_inst, ninst, ntiles, storage, status,
                                         static_cast<const uint8_t*>(w) + kWeightBytes, s);
    StepArgs sa{};
    sa.status = status;
    const BatchTiles bt{d_inst, d_tile_begin, d_tile_inst, ninst};
    switch (storage) {
        case LBM_STORE_F32: return launch_tc_batch_s<LBM_STORE_F32>(sa, bt, ntiles, tc_shape, w, s);
        case LBM_STORE_F16_DEV: return launch_tc_batch_s<LBM_STORE_F16_DEV>(sa, bt, ntiles, tc_shape, w, s);
        default: return launch_tc_batch_s<LBM_STORE_BF16_DEV>(sa, bt, ntiles, tc_shape, w, s);
    }
}

cudaError_t run_tc_selftest(float* d_err, int* d_status, cudaStream_t s) {
    const uint32_t smem = 20480 + 12800 + 64;
    tc_selftest_kernel<<<1, 128, smem, s>>>(d_err, d_status);
    return cudaGetLastError();
}

}  // namespace lbm
