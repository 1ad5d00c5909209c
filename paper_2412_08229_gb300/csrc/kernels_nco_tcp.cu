// kernels_nco_tcp.cu - the fused neural-collision step with the invariant network of
// Sec. II.B (eq. gconv_m) on the tcgen05 tensor cores, pipelined over pairs of group
// elements with every MMA operand A and accumulator in tensor memory (TMEM).
//
// One persistent CTA per SM runs two tile pipelines; a pipeline is two warpgroups that
// share one tile of 128 cells (one cell per thread and TMEM lane). The 48 elements g of
// O_h form 24 pairs (2P, 2P + 1); warpgroup s of a pipeline takes the pairs P = 2i + s,
// i = 0..11, each with its own TMEM regions:
//   L1  D1[128 x 48] = A1[128 x 32] . B1_P^T  A1 = (m in the printed order, 1, 0, 0) in TMEM,
//                                            B1_P rows (e, j) = ((W1 P_g)[j,:], b1[j]), g = 2P + e;
//   L2  D2[128 x 48] = A2[128 x 48] . B2^T    A2 = (relu(h_a), 1, 0, 0, 0, relu(h_b), 1, 0, 0, 0)
//                                            in TMEM (BF16), B2 = the block-diagonal pair of
//                                            (W2 | b2), so one chain of three MMAs serves both;
//   L3  on the CUDA cores: h = sum_g relu(D2) in FP32, tau~ = W3 h / 48 + b3 (layer 3 is
//       affine, so the group mean moves inside it).
// Per pair a warpgroup converts D1 to A2 (relu, BF16), lets its L2 issuer start layer 2 and
// its L1 issuer start layer 1 of its next pair into the freed D1, then folds D2 into its
// group sum while the tensor pipe runs that layer 1. TMEM per pipeline (256 of the SM's 512
// columns): D1[2] at 0 and 48, D2[2] at 96 and 144, A1 at 192, A2[2] at 208 and 232.
// At a tile boundary warpgroup 0 loads the next tile (populations, moments, A1) while
// warpgroup 1 adds warpgroup 0's group sums to its own, forms the rates and relaxes and
// stores the previous tile (the moments pass through shared memory, double-buffered).
// The handoffs between the warpgroups never let a barrier run two phases ahead of its
// waiter (a parity wait cannot tell those apart): warpgroup 1 releases A1 once per tile
// (after its last layer-1 MMA of the tile completed), and the group sums go through one
// barrier per tile parity, as their buffers do. Every wait is bounded in clock cycles; a wait that runs out latches a status flag, the
// warpgroups leave their loops, each MMA issuer waits (full limit) for its last commit, and
// TMEM is released only when every issuer drained. B operands use the K-major, no-swizzle
// core-matrix layout of tc_ptx.cuh.
#include <cstring>

#include "force.cuh"
#include "tc_common.cuh"

namespace lbm {
using namespace tc;
using namespace tcc;

namespace {

constexpr int kTile = 128;
constexpr int kG = 48;
constexpr int kPairs = kG / 2;          // 24 pairs of group elements
constexpr int kPairsPerWg = kPairs / 2;  // 12
constexpr int kN = 48;                   // 2 elements x 20 hidden units + 8 padding rows
constexpr int kK1 = 32;                  // 27 moments + bias input + pad
constexpr int kK2 = 48;                  // 2 x (20 hidden + bias input + 3 pad)
constexpr int kPipes = 2;
constexpr int kThreads = kPipes * 256;

// weight image = shared-memory image: 24 B1 pairs, the block-diagonal B2, W3 and b3 (floats)
constexpr uint32_t kB1PairBytes = kN * kK1 * 2;  // 3072
constexpr uint32_t kB1Off = 0;
constexpr uint32_t kB2Off = kB1Off + kPairs * kB1PairBytes;  // 73728
constexpr uint32_t kB2Bytes = kN * kK2 * 2;                  // 4608
constexpr uint32_t kW3Off = kB2Off + kB2Bytes;
constexpr uint32_t kB3Off = kW3Off + kOut * kHidden * 4;
constexpr uint32_t kWeightBytes = kB3Off + 16;  // 78672
static_assert(kWeightBytes % 16 == 0, "weight image copies in 16-byte vectors");

// per pipeline: moments and rho - 1 of two tiles, warpgroup 0's group sums of two tiles
constexpr int kMVals = Q + 1;
constexpr uint32_t kMBufBytes = kMVals * kTile * 4;     // 14336
constexpr uint32_t kAccBufBytes = kHidden * kTile * 4;  // 10240
constexpr uint32_t kPipeBytes = 2 * kMBufBytes + 2 * kAccBufBytes;
constexpr uint32_t kPipeOff = (kWeightBytes + 1023) / 1024 * 1024;
constexpr uint32_t kBarOff = kPipeOff + kPipes * kPipeBytes;
// l1[2], l2[2] (commits); A1 written; group sums written, one per tile parity; A1 free
constexpr int kBarsPerPipe = 8;
// forced steps: 2 F^ as floats and the block's projection sums
constexpr uint32_t kFhOff = kBarOff + kPipes * kBarsPerPipe * 8 + 16;
constexpr uint32_t kRedOff = kFhOff + 6 * kForcedModes * 4;
constexpr uint32_t kSmemBytes = kRedOff + frc::kProjValues * 8;
static_assert(kSmemBytes <= 227 * 1024, "shared memory budget");

constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kTmemPerPipe = 256;
constexpr uint32_t kD1Col = 0, kD2Col = 96, kA1Col = 192, kA2Col = 208;  // + 48 s, + 48 s, -, + 24 s
static_assert(kA2Col + 2 * 24 == kTmemPerPipe, "TMEM budget of a pipeline");

template <int STORAGE, int BC, bool FORCED, bool BATCHED>
__global__ void __launch_bounds__(kThreads, 1) nco_tcp_kernel(const StepArgs a0, const BatchTiles bt,
                                                              const uint8_t* __restrict__ wimg, int ntiles,
                                                              long long limit, const FusedForce ff) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane_id = tid & 31;
    const int pipe = tid >> 8;
    const int s = (tid >> 7) & 1;  // warpgroup within the pipeline
    const int r = tid & 127;       // cell of the tile, TMEM lane
    const int wq = warp & 3;       // TMEM lane quarter of this warp
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kBarOff) + pipe * kBarsPerPipe;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(smem + kBarOff + kPipes * kBarsPerPipe * 8);
    float* fh2 = reinterpret_cast<float*>(smem + kFhOff);
    unsigned long long* red = reinterpret_cast<unsigned long long*>(smem + kRedOff);

    // ---- set-up: weights to shared memory, barriers, TMEM
    for (uint32_t i = tid * 16; i < kWeightBytes; i += kThreads * 16)
        *reinterpret_cast<uint4*>(smem + i) = *reinterpret_cast<const uint4*>(wimg + i);
    if (FORCED) {
        frc::load_fh2(ff.fhat, fh2);
        if (tid < frc::kProjValues) red[tid] = 0ull;
    }
    if (tid == 0) {
        for (int p = 0; p < kPipes; ++p) {
            uint64_t* b = reinterpret_cast<uint64_t*>(smem + kBarOff) + p * kBarsPerPipe;
            for (int k = 0; k < 4; ++k) mbar_init(&b[k], 1);  // one tcgen05.commit each
            mbar_init(&b[4], 128);                             // warpgroup 0 wrote A1
            mbar_init(&b[5], 128);                             // warpgroup 0 wrote its group sums (even tile)
            mbar_init(&b[6], 128);                             // ... (odd tile)
            mbar_init(&b[7], 128);                             // warpgroup 1's last layer 1 of a tile completed
        }
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(tmem_holder, kTmemCols);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    uint64_t* bar_l1 = &bars[s];       // this warpgroup's layer-1 commits
    uint64_t* bar_l2 = &bars[2 + s];   // this warpgroup's layer-2 commits
    uint64_t* bar_a1 = &bars[4];
    uint64_t* bar_acc = &bars[5];      // + (tile & 1)
    uint64_t* bar_a1free = &bars[7];   // warpgroup 1 no longer reads the tile's A1
    const uint32_t tbase = *tmem_holder + static_cast<uint32_t>(pipe) * kTmemPerPipe;
    const uint32_t lanes = static_cast<uint32_t>(wq * 32) << 16;
    const uint32_t tD1 = tbase + kD1Col + 48 * s, tD2 = tbase + kD2Col + 48 * s;
    const uint32_t tA1 = tbase + kA1Col, tA2 = tbase + kA2Col + 24 * s;
    const uint32_t sB1 = smem_u32(smem + kB1Off), sB2 = smem_u32(smem + kB2Off);
    const float* W3 = reinterpret_cast<const float*>(smem + kW3Off);
    const float* b3 = reinterpret_cast<const float*>(smem + kB3Off);
    float* mbuf = reinterpret_cast<float*>(smem + kPipeOff + pipe * kPipeBytes);
    float* accbuf = reinterpret_cast<float*>(smem + kPipeOff + pipe * kPipeBytes + 2 * kMBufBytes);
    const int bid = 1 + 2 * pipe + s;
    const bool l2_issuer = wq == 0 && lane_id == 0;
    const bool l1_issuer = wq == 1 && lane_id == 0;
    constexpr uint32_t idesc = idesc_bf16(128, kN);

    // forced steps: warpgroup 0's fixed-point projection sums of the velocities it loads
    long long pacc[3] = {0, 0, 0};
    // completions waited on (the parity of the next wait) and commits made (the drain)
    uint32_t n_l1 = 0, n_l2 = 0, n_a1 = 0, c_l1 = 0, c_l2 = 0;
    auto issue_l1 = [&](int P) {
#pragma unroll
        for (int kk = 0; kk < kK1 / 16; ++kk)
            mma_bf16_ta(tD1, tA1 + 8 * kk, smem_desc(sB1 + P * kB1PairBytes + kk * 256, 128, 128 * kK1 / 8), idesc,
                        kk);
        mma_commit(bar_l1);
        ++c_l1;
    };
    bool ok = true;
    int it = 0;
    for (int gtile = blockIdx.x * kPipes + pipe; gtile < ntiles; gtile += gridDim.x * kPipes, ++it) {
        int tile = gtile;
        StepArgs a = a0;
        if (BATCHED) {  // the instance owning this tile
            const int inst = __ldg(&bt.tile_inst[gtile]);
            a = bt.inst[inst];
            tile = gtile - static_cast<int>(__ldg(&bt.tile_begin[inst]));
        }
        const long long cell = static_cast<long long>(tile) * kTile + r;
        const bool valid = cell < a.d.ncell;
        bool w = true;
        if (s == 0) {
            // A1 is free once warpgroup 1's last layer-1 MMA of the previous tile has completed,
            // which warpgroup 1 signals once per tile, so the barrier is at most one phase
            // ahead of or behind this wait (the result is made uniform: the A1 store below is
            // a warp-collective instruction)
            if (it > 0)
                w = wg_sync_and(bid, wait_phase(bar_a1free, static_cast<uint32_t>(it - 1) & 1u, limit));
            float m[Q];
            float drho = 0.0f;
            int x = 0, y = 0, z = 0;
            Macro q{};
            if (valid) {
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
            float* mb = mbuf + (it & 1) * kMVals * kTile;
#pragma unroll
            for (int e = 0; e < Q; ++e) mb[e * kTile + r] = m[e];
            mb[Q * kTile + r] = drho;
            uint32_t p[16];  // A1 row r: the raw moments in the printed order of Sec. II.B, then the bias input 1
            static_for<13>([&](auto K) {
                constexpr int k = decltype(K)::value;
                p[k] = pack_bf16(m[kPrintedE<2 * k>], m[kPrintedE<2 * k + 1>]);
            });
            p[13] = pack_bf16(m[kPrintedE<26>], 1.0f);
            p[14] = 0u;
            p[15] = 0u;
            if (w) {  // the previous tile's layer 1 may still read A1 otherwise
                tmem_st16(tA1 + lanes, p);
                tmem_st_wait();
            }
            tc_fence_before();
            mbar_arrive(bar_a1);
            if (FORCED && ff.proj) {  // this tile's velocities into the next step's projection
                frc::Cx ph[kForcedModes];
                frc::cell_phases(x, y, z, a.d, ff.tab, ph);
                frc::project_warp(q.ux, q.uy, q.uz, ph, lane_id, pacc, ff.scale);
            }
        }
        {
            const bool wa = wait_phase(bar_a1, n_a1 & 1u, limit);
            ++n_a1;
            if (!(ok = wg_sync_and(bid, ok && w && wa))) break;
        }
        if (l1_issuer) {
            tc_fence_after();
            issue_l1(s);
        }
        float acc[kHidden];
#pragma unroll
        for (int j = 0; j < kHidden; ++j) acc[j] = 0.0f;
        bool w2 = true;
        for (int i = 0; i < kPairsPerWg; ++i) {
            const bool w1 = wait_phase(bar_l1, n_l1 & 1u, limit);
            ++n_l1;
            tc_fence_after();
            if (s == 1 && i == kPairsPerWg - 1) mbar_arrive(bar_a1free);  // its last layer 1 read A1
            {  // D1 of the pair -> (relu in BF16, 1, 0) per element = A2
                uint32_t v[40];
                tmem_ld16(tD1 + lanes, v);
                tmem_ld16(tD1 + lanes + 16, v + 16);
                tmem_ld8(tD1 + lanes + 32, v + 32);
                tmem_ld_wait();
                uint32_t h[24];
#pragma unroll
                for (int k = 0; k < 10; ++k) {
                    h[k] = pack_bf16_relu(as_f(v[2 * k]), as_f(v[2 * k + 1]));
                    h[12 + k] = pack_bf16_relu(as_f(v[20 + 2 * k]), as_f(v[21 + 2 * k]));
                }
                h[10] = kBf16One;
                h[11] = 0u;
                h[22] = kBf16One;
                h[23] = 0u;
                // three 8-column stores: A2 of warpgroup 1 starts 8-, not 16-column aligned
                tmem_st8(tA2 + lanes, h);
                tmem_st8(tA2 + lanes + 8, h + 8);
                tmem_st8(tA2 + lanes + 16, h + 16);
                tmem_st_wait();
            }
            tc_fence_before();
            if (!(ok = wg_sync_and(bid, ok && w1 && w2))) break;
            if (l2_issuer) {
                tc_fence_after();
#pragma unroll
                for (int kk = 0; kk < kK2 / 16; ++kk)
                    mma_bf16_ta(tD2, tA2 + 8 * kk, smem_desc(sB2 + kk * 256, 128, 128 * kK2 / 8), idesc, kk);
                mma_commit(bar_l2);
                ++c_l2;
            }
            if (l1_issuer && i + 1 < kPairsPerWg) {
                tc_fence_after();
                issue_l1(2 * (i + 1) + s);
            }
            w2 = wait_phase(bar_l2, n_l2 & 1u, limit);
            ++n_l2;
            tc_fence_after();
            {  // relu of the pair's layer-2 outputs, summed over the group
                uint32_t v[40];
                tmem_ld16(tD2 + lanes, v);
                tmem_ld16(tD2 + lanes + 16, v + 16);
                tmem_ld8(tD2 + lanes + 32, v + 32);
                tmem_ld_wait();
                tc_fence_before();  // D2 read before this warpgroup's next layer 2 overwrites it
#pragma unroll
                for (int j = 0; j < kHidden; j += 2) {
                    add2_relu(acc[j], acc[j + 1], as_f(v[j]), as_f(v[j + 1]));
                    add2_relu(acc[j], acc[j + 1], as_f(v[kHidden + j]), as_f(v[kHidden + j + 1]));
                }
            }
        }
        if (!ok) break;
        if (!(ok = wg_sync_and(bid, w2))) break;
        float* ab = accbuf + (it & 1) * kHidden * kTile;
        if (s == 0) {  // hand this warpgroup's group sums to warpgroup 1
#pragma unroll
            for (int j = 0; j < kHidden; ++j) ab[j * kTile + r] = acc[j];
            mbar_arrive(bar_acc + (it & 1));
        } else {
            // one barrier per tile parity (as for the buffers): warpgroup 0 may hand over the
            // next tile's sums before this wait, but not the one after (it needs bar_a1free)
            const bool wa = wait_phase(bar_acc + (it & 1), static_cast<uint32_t>(it >> 1) & 1u, limit);
            if (!(ok = wg_sync_and(bid, wa))) break;
            if (valid) {
                float rates[kOut];
#pragma unroll
                for (int n = 0; n < kOut; ++n) {
                    float t = 0.0f;
#pragma unroll
                    for (int j = 0; j < kHidden; ++j) t = fmaf(W3[n * kHidden + j], acc[j] + ab[j * kTile + r], t);
                    rates[n] = rate_from_output(t * (1.0f / 48.0f) + b3[n]);
                }
                const float* mb = mbuf + (it & 1) * kMVals * kTile;
                float m[Q];
#pragma unroll
                for (int e = 0; e < Q; ++e) m[e] = mb[e * kTile + r];
                const float drho = mb[Q * kTile + r];
                const Macro q = macro_from_moments(m, drho);
                float df[Q];
                relax_to_populations(m, drho, q, 1.0f / a.tau, rates, df);
                if (FORCED) {  // F(x) from this step's coefficients
                    int x, y, z;
                    cell_coords(cell, a.d, x, y, z);
                    frc::Cx ph[kForcedModes];
                    frc::cell_phases(x, y, z, a.d, ff.tab, ph);
                    float F[3];
                    frc::synth_force(fh2, ph, F);
                    add_kupershtokh(df, q, F[0], F[1], F[2]);
                } else if (BATCHED && a.force) {
                    add_kupershtokh(df, q, a.force[cell], a.force[a.d.ncell + cell], a.force[2 * a.d.ncell + cell]);
                }
                store_cell<STORAGE>(a.dst, a.d, cell, df);
            }
        }
    }
    if (FORCED && ff.proj && s == 0) frc::proj_to_shared(red, pacc, lane_id);
    bool drained = true;
    if (!ok) {
        if (r == 0) atomicOr(a0.status, 2);
        // wait, with the full limit, for the last commit of each issuer: no MMA may still use
        // TMEM when it is released
        if (l1_issuer && c_l1 > 0) drained = wait_phase(bar_l1, (c_l1 - 1u) & 1u);
        if (l2_issuer && c_l2 > 0) drained = wait_phase(bar_l2, (c_l2 - 1u) & 1u);
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

template <int STORAGE, int BC, bool FORCED, bool BATCHED>
cudaError_t launch_tcp_t(const StepArgs& a, const BatchTiles& bt, const void* w, int ntiles, long long wait,
                         const FusedForce& ff, cudaStream_t s) {
    static std::atomic<unsigned long long> attr{0};
    const cudaError_t e =
        ensure_dynamic_smem(nco_tcp_kernel<STORAGE, BC, FORCED, BATCHED>, static_cast<int>(kSmemBytes), attr);
    if (e != cudaSuccess) return e;
    int grid = (ntiles + kPipes - 1) / kPipes;
    if (grid > sm_count()) grid = sm_count();
    if (grid < 1) return cudaSuccess;
    nco_tcp_kernel<STORAGE, BC, FORCED, BATCHED>
        <<<grid, kThreads, kSmemBytes, s>>>(a, bt, static_cast<const uint8_t*>(w), ntiles, wait, ff);
    return cudaGetLastError();
}

template <int STORAGE>
cudaError_t launch_tcp_b(const StepArgs& a, const FusedForce* ff, int bc, const void* w, long long wait,
                         cudaStream_t s) {
    const int ntiles = static_cast<int>((a.d.ncell + kTile - 1) / kTile);
    const BatchTiles none{nullptr, nullptr, nullptr, 0};
    const FusedForce nf{};
    if (ff) {  // forcing runs on periodic boxes only
        if (bc != LBM_BC_PERIODIC) return cudaErrorInvalidValue;
        return launch_tcp_t<STORAGE, LBM_BC_PERIODIC, true, false>(a, none, w, ntiles, wait, *ff, s);
    }
    if (bc == LBM_BC_TGV_REDUCED)
        return launch_tcp_t<STORAGE, LBM_BC_TGV_REDUCED, false, false>(a, none, w, ntiles, wait, nf, s);
    return bc == LBM_BC_PERIODIC ? launch_tcp_t<STORAGE, LBM_BC_PERIODIC, false, false>(a, none, w, ntiles, wait, nf, s)
                                 : launch_tcp_t<STORAGE, LBM_BC_MIRROR, false, false>(a, none, w, ntiles, wait, nf, s);
}

}  // namespace

size_t nco_tcp_weight_bytes() { return kWeightBytes; }

void nco_tcp_pack_weights(const float* theta, void* out) {
    const float* W1 = theta;  // (20, 27), printed moment order
    const float* b1 = W1 + kHidden * Q;
    const float* W2 = b1 + kHidden;
    const float* b2 = W2 + kHidden * kHidden;
    const float* W3 = b2 + kHidden;
    const float* b3 = W3 + kOut * kHidden;
    uint8_t* img = static_cast<uint8_t*>(out);
    std::memset(img, 0, kWeightBytes);
    auto put = [&](uint32_t base, int row, int k, int K, float v) {
        const uint16_t b = f2bf(v);
        std::memcpy(img + base + kmajor_offset(row, k, K), &b, 2);
    };
    const GroupTables& gt = group_tables();
    for (int g = 0; g < kG; ++g) {
        const uint32_t base = kB1Off + (g / 2) * kB1PairBytes;
        for (int j = 0; j < kHidden; ++j) {
            const int row = (g % 2) * kHidden + j;
            // (W1 P_g m)_j = sum_k W1[j][k] msign[g][k] m[mperm[g][k]] (printed order)
            for (int k = 0; k < Q; ++k) {
                const int e = kPrinted.e[k];
                int kp = 0;
                for (int t = 0; t < Q; ++t)
                    if (kPrinted.e[t] == gt.mperm_t[g][e]) kp = t;
                put(base, row, kp, kK1, W1[j * Q + k] * static_cast<float>(gt.msign_t[g][e]));
            }
            put(base, row, Q, kK1, b1[j]);
        }
    }
    for (int j = 0; j < kHidden; ++j)
        for (int half = 0; half < 2; ++half) {  // block diagonal: element a at K 0..20, element b at K 24..44
            const int row = half * kHidden + j, k0 = half * 24;
            for (int k = 0; k < kHidden; ++k) put(kB2Off, row, k0 + k, kK2, W2[j * kHidden + k]);
            put(kB2Off, row, k0 + kHidden, kK2, b2[j]);
        }
    std::memcpy(img + kW3Off, W3, kOut * kHidden * sizeof(float));
    std::memcpy(img + kB3Off, b3, kOut * sizeof(float));
}

cudaError_t launch_step_nco_tcp_batch(const StepArgs* d_inst, const long long* d_tile_begin, const int* d_tile_inst,
                                      int ninst, long long ntiles, int storage, int* status, const void* w,
                                      cudaStream_t s) {
    StepArgs sa{};
    sa.status = status;
    const BatchTiles bt{d_inst, d_tile_begin, d_tile_inst, ninst};
    const int nt = static_cast<int>(ntiles);
    const FusedForce nf{};
    switch (storage) {
        case LBM_STORE_F32:
            return launch_tcp_t<LBM_STORE_F32, LBM_BC_PERIODIC, false, true>(sa, bt, w, nt, kDefaultWaitCycles, nf, s);
        case LBM_STORE_F16_DEV:
            return launch_tcp_t<LBM_STORE_F16_DEV, LBM_BC_PERIODIC, false, true>(sa, bt, w, nt, kDefaultWaitCycles, nf, s);
        default:
            return launch_tcp_t<LBM_STORE_BF16_DEV, LBM_BC_PERIODIC, false, true>(sa, bt, w, nt, kDefaultWaitCycles, nf, s);
    }
}

cudaError_t launch_step_nco_tcp(const StepArgs& a, const FusedForce* ff, int storage, int bc, const void* w,
                                long long wait_cycles, cudaStream_t s) {
    switch (storage) {
        case LBM_STORE_F32: return launch_tcp_b<LBM_STORE_F32>(a, ff, bc, w, wait_cycles, s);
        case LBM_STORE_F16_DEV: return launch_tcp_b<LBM_STORE_F16_DEV>(a, ff, bc, w, wait_cycles, s);
        default: return launch_tcp_b<LBM_STORE_BF16_DEV>(a, ff, bc, w, wait_cycles, s);
    }
}

}  // namespace lbm
