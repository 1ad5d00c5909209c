// internal.h - shared declarations of the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "d3q27.cuh"

namespace lbm {

constexpr int kHidden = 20;
constexpr int kOut = 4;
constexpr int kNumTheta = 27 * 20 + 20 + 20 * 20 + 20 + 20 * 4 + 4;  // 1064 (Sec. II.B)
constexpr int kNumThetaDeep = kNumTheta + 20 * 20 + 20;  // 1484: a third hidden layer of 20 (Sec. IV)
constexpr int kForcedModes = 16;  // half-space integer modes with 1 <= |k| <= 2

// Network parameters handed to the FP32 step kernel by value (they live in the
// kernel's constant parameter bank, so FFMAs read them without loads).
// W1p[p] = W1 with its columns rearranged for axis permutation p: the input of
// group element (p, s) is then sgn(s, t) * m_t in tensor order t (see nco_f32).
struct NetParams {
    float W1p[6][kHidden][Q];
    float b1[kHidden];
    float W2[kHidden][kHidden];
    float b2[kHidden];
    float W3[kOut][kHidden];  // output layer
    float b3[kOut];
    float Wd[kHidden][kHidden];  // third hidden layer (deep network only)
    float bd[kHidden];
    int deep;                    // 1: 27-20-20-20-4, 0: 27-20-20-4
};

// One symmetry g = (A, t) of the Taylor-Green flow that maps the block of the periodic
// box next to the reduced domain [0, pi/2]^3 in direction (rx, ry, rz) onto the domain:
// (A x)_a = sign[a] x_perm[a], t_a = k[a] pi/2; pmap[i] = index of A c_i.
struct SymRegion {
    signed char perm[3], sign[3], k[3], pad;
    unsigned char pmap[27], pad2;
};

// SMs of the current device (grid sizing), looked up once per device
inline int sm_count() {
    static std::atomic<int> cache[64];
    int dev = 0;
    cudaGetDevice(&dev);
    const int slot = dev & 63;
    int n = cache[slot].load(std::memory_order_relaxed);
    if (n <= 0) {
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
        cache[slot].store(n, std::memory_order_relaxed);
    }
    return n;
}

// The dynamic shared-memory limit of a kernel is a per-device setting: raise it once per
// device (bit `device` of `done`). Threads may race here; setting it twice is harmless.
template <typename F>
inline cudaError_t ensure_dynamic_smem(F* kernel, int bytes, std::atomic<unsigned long long>& done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

// Limit of each wait of the tensor-core kernels on MMA completion, in SM clock cycles
// (about 1 s at 2 GHz): a wait that runs out ends the kernel early with a status flag.
constexpr long long kDefaultWaitCycles = 2000000000LL;

struct Dims {
    int nx, ny, nz;
    long long ncell;
    const SymRegion* sym = nullptr;  // reduced Taylor-Green domain: 27 regions (device memory)
};

// The 27 region entries (index 9 (rz+1) + 3 (ry+1) + (rx+1); the centre is unused) of the
// reduced Taylor-Green domain, derived from the flow's symmetry group (host).
bool tgv_reduced_table(SymRegion* out27);

struct StepArgs {
    Dims d;
    const void* src;       // 27 planes, storage type
    void* dst;             // 27 planes, storage type
    const float* force;    // stored force field, 3 planes, or nullptr (batches and the adjoint)
    float* u_out;          // 3 planes of the pre-collision bare velocity, or nullptr (batches)
    int* status;           // latched error flags
    float tau;
    float rho_min, rho_max;
};

struct FusedForce;  // the in-kernel forcing of a forced step (declared with the forcing below)

// Kernel launchers (kernels_step.cu)
// tc_shape selects the tile shape of the BF16 tensor-core network (0: pairs of group
// elements across two warpgroups, kernels_nco_tcp.cu, two-layer network only; 2, 3, 4:
// chunks of four elements per warpgroup, kernels_nco_tc.cu, with that many warpgroups per
// SM in batches). The per-tile arithmetic of one shape does not depend on the warpgroup count.
// wait_cycles: limit of the main MMA-completion waits of the pair-pipelined and split
// tensor-core kernels (kept out of StepArgs: a larger argument block made the CUDA-core
// network kernel spill).
// ff: the in-kernel forcing of a forced step (nullptr: unforced; a.force is then not read).
cudaError_t launch_step(const StepArgs& a, const FusedForce* ff, int op, int storage, int bc, int net_prec,
                        const NetParams* net, const void* tc_weights, int tc_shape, long long wait_cycles,
                        cudaStream_t s);
cudaError_t launch_init_eq(const Dims& d, int storage, int bc, const float* rho, const float* u,
                           void* dst, cudaStream_t s);
cudaError_t launch_set_state(const Dims& d, int storage, int bc, const float* f, void* dst,
                             cudaStream_t s);
cudaError_t launch_get_state(const Dims& d, int storage, int bc, const void* src, float* f,
                             cudaStream_t s);
cudaError_t launch_macroscopic(const Dims& d, int storage, int bc, const void* src, float* rho,
                               float* u, cudaStream_t s);
cudaError_t launch_kinetic_energy(const Dims& d, int storage, int bc, const void* src,
                                  double* partials, int npartials, double* out, cudaStream_t s);
int kinetic_energy_blocks(const Dims& d);

// Tensor-core network (kernels_nco_tc.cu)
size_t nco_tc_weight_bytes();
void nco_tc_pack_weights(const float* theta, bool deep, void* host_out);  // host-side packing
cudaError_t launch_step_nco_tc(const StepArgs& a, const FusedForce* ff, int storage, int bc, bool deep, int tc_shape,
                               long long wait_cycles, const void* tc_weights, cudaStream_t s);
bool nco_tc_supported(int storage, int bc);
// Pipelined tensor-core step of the two-layer network (kernels_nco_tcp.cu); its weights are
// the second part of the nco_tc image.
size_t nco_tcp_weight_bytes();
void nco_tcp_pack_weights(const float* theta, void* host_out);
cudaError_t launch_step_nco_tcp(const StepArgs& a, const FusedForce* ff, int storage, int bc, const void* tc_weights,
                                long long wait_cycles, cudaStream_t s);
// Split-BF16 (three-product) tensor-core network of FP32-class accuracy (kernels_nco_tc3.cu)
size_t nco_tc3_weight_bytes();
void nco_tc3_pack_weights(const float* theta, bool deep, void* host_out);
cudaError_t launch_step_nco_tc3(const StepArgs& a, const FusedForce* ff, int storage, int bc, bool deep,
                                const void* tc_weights, long long wait_cycles, cudaStream_t s);
cudaError_t run_tc_selftest(float* d_err, int* d_status, cudaStream_t s);
// One persistent launch over the tiles of a batch of instances (periodic, same storage).
cudaError_t launch_step_nco_tc_batch(const StepArgs* d_inst, const long long* d_tile_begin, const int* d_tile_inst,
                                     int ninst, long long ntiles, int storage, int tc_shape, int* status, const void* w,
                                     cudaStream_t s);
cudaError_t launch_step_nco_tcp_batch(const StepArgs* d_inst, const long long* d_tile_begin, const int* d_tile_inst,
                                      int ninst, long long ntiles, int storage, int* status, const void* w,
                                      cudaStream_t s);

// Spectrum (kernels_diag.cu)
bool fft_size_ok(int n);
cudaError_t launch_spectrum(const Dims& d, int storage, int bc, const void* src, float2* work,
                            double* E, int nbins, double* ke, cudaStream_t s);
size_t spectrum_work_elems(const Dims& d, int bc);
cudaError_t launch_spectrum_shells(const Dims& f, int* out, cudaStream_t s);

// Guard regions around the population buffers (kernels_diag.cu): bytes of the four regions
// that differ from the pattern are counted per region into bad[4] (zeroed by the caller).
constexpr size_t kGuardBytes = 4096;
constexpr unsigned char kGuardPattern = 0xA5;
cudaError_t launch_guard_check(const unsigned char* const regions[4], int* bad, cudaStream_t s);

// Forcing (kernels_force.cu)
struct ForceModes {
    int k[kForcedModes][3];
};
ForceModes forced_modes();
struct ForceParams {
    double power, kf, c, ka, kb;
};
constexpr int kForceConsts = 7;                // per mode: e1 (3), e2 (3), amplitude
constexpr int kDrawRow = 4 * kForcedModes;     // per step: sin 2 phi, cos 2 phi, sin psi, cos psi of every mode
// Host: the per-mode constants (kForcedModes x kForceConsts doubles), the phase tables of
// the three axes (2 (nx + ny + nz) float2: e^{i 2 pi k j / n} for k = 1, 2), and one row of
// draws from the random phases phi, psi (kForcedModes each).
void force_mode_consts(const ForceParams& fp, double* out);
void force_phase_table(const Dims& d, float2* out);
void force_draw_trig(const double* phi, const double* psi, double* row);
// Projection u^(k) of a step's velocity, accumulated as 96 fixed-point sums (force.cuh):
// proj[32 a + 2 m + c] = sum over warps of round(2^S x warp sum of Re/Im u_a e^{-ik_m.x}).
float force_proj_scale(long long ncell);   // 2^S
double force_proj_unit(long long ncell);   // 2^-S / ncell: a sum times unit is u^(k)
int force_project_blocks(const Dims& d);
// Adds the projection of the velocity planes u to proj (the caller clears proj first).
cudaError_t launch_force_project(const Dims& d, const float* u, const float2* tab, unsigned long long* proj,
                                 float scale, cudaStream_t s);
// F^ of one step from proj and one row of draws; clears proj for the next step's sums.
cudaError_t launch_force_coeffs(unsigned long long* proj, double unit, const double* row, const double* consts,
                                double* fhat, cudaStream_t s);
// The same with row = min(head + *counter, rows - 1), then *counter += 1 (graph replays).
cudaError_t launch_force_coeffs_indexed(unsigned long long* proj, double unit, const double* draws,
                                        long long* counter, long long head, long long rows, const double* consts,
                                        double* fhat, cudaStream_t s);
cudaError_t launch_force_synth(const Dims& d, const double* fhat, const float2* tab, float* force, cudaStream_t s);
// The in-kernel forcing of a single context's forced step: F(x) from fhat and the phase
// tables, the step's velocity projected into proj (nullptr: not projected, as in the
// adjoint's recomputed steps).
struct FusedForce {
    const double* fhat;        // 16 x 6 coefficients of this step, fhat[6 m + 2 a + c]
    const float2* tab;         // per-axis phase tables (force_phase_table)
    unsigned long long* proj;  // fixed-point projection sums, or nullptr
    float scale;               // force_proj_scale(ncell)
};
// One forced instance of a batch (device array of these for the batched launches).
struct ForceBatchItem {
    Dims d;
    const float* u;            // velocity written by the step kernel (projection input)
    float* force;              // 3 planes
    unsigned long long* proj;  // its projection sums
    float scale;               // force_proj_scale(ncell)
    double unit;               // force_proj_unit(ncell)
    const double* draws;       // rows of kDrawRow doubles (force_draw_trig)
    long long head;            // draw row of the step the device counter calls 0
    long long rows;            // rows allocated (clamp)
    const double* consts;      // force_mode_consts of the instance
    const float2* tab;         // its phase tables
    double* fhat;              // 16 x 6 coefficients
};
// stage 0: coefficients then force fields of every item; stage 1: the projections.
cudaError_t launch_force_batch(const ForceBatchItem* d_items, int n, int max_proj_blocks, long long max_cells,
                               const long long* counter, int stage, cudaStream_t s);
cudaError_t launch_counter_increment(long long* counter, cudaStream_t s);
cudaError_t launch_counter_set(long long* counter, long long v, cudaStream_t s);

// Adjoint of the NCO step (kernels_adjoint.cu), FP32 storage only; periodic, mirror and
// reduced Taylor-Green boundaries; two or three hidden layers (net.deep)
int adjoint_grad_len(bool deep);
cudaError_t launch_adjoint_seed(const Dims& d, int storage, int bc, const void* state, const float* du,
                                const float* drho, float ke_scale, bool accumulate, float* lam, cudaStream_t s);
cudaError_t launch_adjoint_step(const Dims& d, int storage, int bc, const void* state, const float* lam_in,
                                float* lam_out, double* grad, float tau, const float* force, const NetParams& net,
                                cudaStream_t s);
void adjoint_fold_gradient(const double* acc, bool deep, float* out);

// Host-side group tables and parameter packing (lbm_abi.cu)
const GroupTables& group_tables();
void make_net_params(const float* theta, bool deep, NetParams* out);

}  // namespace lbm
