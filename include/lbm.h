/*
 * lbm.h - C ABI of the GB300 (sm_103a) D3Q27 neural-collision lattice Boltzmann library.
 *
 * Method: arXiv 2412.08229, Bedrunka et al., "Machine Learning Enhanced Collision
 * Operator for the Lattice Boltzmann Method Based on Invariant Networks".
 *
 * Conventions shared by every call
 *  - Every call returns an lbm_status; 0 is success, negative values are errors. No
 *    call throws, aborts or exits. lbm_last_error(ctx) returns a message for the last
 *    failure on that context (valid until the next call on it).
 *  - Grid fields are structure-of-arrays, x fastest: a scalar field is nx*ny*nz values
 *    at index (z*ny + y)*nx + x; a vector field stores its three components one after
 *    the other (component-major); populations store 27 such planes in the velocity
 *    order below.
 *  - Velocity order: index i = 9*(cz+1) + 3*(cy+1) + (cx+1) for c_i = (cx,cy,cz) in
 *    {-1,0,1}^3 (lexicographic over z, y, x); 13 is the rest velocity and 26-i is the
 *    opposite of i. Moment order: the Hermite rows as printed in Sec. II.B (last row
 *    xxyyzz).
 *  - Field pointers may be device memory or host memory (pageable or pinned); the
 *    library tells them apart with cudaPointerGetAttributes. Calls whose outputs land
 *    in host memory synchronise the context's stream before returning; all other work
 *    is asynchronous on that stream. The caller owns every pointer it passes.
 *  - The context owns its population buffers and any scratch it needs. After
 *    lbm_create, buffers are allocated on first use and kept: the staging buffer for
 *    host fields, the FFT work of lbm_energy_spectrum, the growing queue of forcing
 *    draws, and for training the checkpoints and force coefficients of a recording and
 *    the adjoint's work buffers (these from the library's stream-ordered pool, without a
 *    device-wide synchronisation).
 */
#ifndef NCO_LBM_H
#define NCO_LBM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef int lbm_status;

enum {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,       /* invalid argument or unsupported combination            */
    LBM_ERR_CUDA = -2,      /* a CUDA runtime call failed (message in lbm_last_error)  */
    LBM_ERR_OOM = -3,       /* device allocation failed                                */
    LBM_ERR_UNSTABLE = -4,  /* NaN/Inf or density outside [rho_min, rho_max] was seen  */
    LBM_ERR_TIMEOUT = -5,   /* a bounded device wait ran out                           */
    LBM_ERR_STATE = -6      /* call out of order (e.g. NCO step before nco_set_weights)*/
};

/* Collision operators (Sec. II.A-B; KBC and the regularised REG are compared in Sec. III.A and
 * Sec. IV: REG relaxes the second-order moments with 1/tau and removes orders 3..6). */
enum { LBM_OP_BGK = 0, LBM_OP_KBC = 1, LBM_OP_NCO = 2, LBM_OP_REG = 3 };

/* Population storage: FP32, or 16-bit deviations f_i - w_i (FP16 or BF16). */
enum { LBM_STORE_F32 = 0, LBM_STORE_F16_DEV = 1, LBM_STORE_BF16_DEV = 2 };

/* Precision of the NCO network: FP32 on CUDA cores; BF16 operands on the tcgen05 tensor
 * cores with FP32 accumulation; or split BF16 on the tensor cores (every operand x =
 * x_hi + x_lo in BF16, products a_hi b_hi + a_hi b_lo + a_lo b_hi accumulated in FP32:
 * below 2^-16 relative per product, FP32-class, at three MMAs per one of LBM_NET_BF16). */
enum { LBM_NET_F32 = 0, LBM_NET_BF16 = 1, LBM_NET_BF16X3 = 2 };

/* Boundaries: fully periodic; specular mirror planes on all six faces with the nodes half
 * a spacing inside (the Taylor-Green octant [0, pi]^3); or the reduced Taylor-Green domain
 * of Appendix A, [0, pi/2]^3 with nodes at (j + 1/2) pi / (2N) on a cube of N^3 nodes,
 * whose faces, edges and corners map a population leaving the domain onto the node and
 * direction the flow's symmetries (reflections, rotations, the x-y exchange) prescribe.
 * The reduced domain holds a flow with the Taylor-Green symmetries only; it takes no
 * spectral forcing, spectrum or adjoint (LBM_ERR_ARG). */
enum { LBM_BC_PERIODIC = 0, LBM_BC_MIRROR = 1, LBM_BC_TGV_REDUCED = 2 };

typedef struct lbm_config {
    int nx, ny, nz;         /* grid size, each >= 1; nx*ny*nz*27 < 2^31              */
    double nu;              /* lattice viscosity, > 0; tau = 3 nu + 1/2 (Sec. II.B)  */
    int op;                 /* LBM_OP_*                                               */
    int storage;            /* LBM_STORE_*                                            */
    int net_precision;      /* LBM_NET_* (NCO only)                                   */
    int boundary;           /* LBM_BC_*                                               */
    int forcing;            /* 0: none; 1: Alvelius spectral forcing (Sec. II.C)      */
    double force_power;     /* P, power input per unit time (lattice units)          */
    double force_kf, force_c, force_ka, force_kb; /* Gaussian shell of forced modes  */
    double rho_min, rho_max;/* stability window for LBM_ERR_UNSTABLE (0,0: 0.5..2)   */
} lbm_config;

typedef struct lbm_ctx lbm_ctx;

/* Create a solver on the current CUDA device. stream: a cudaStream_t passed as void*
 * (NULL = legacy default stream); every kernel of this context runs on it.
 * Allocates two population buffers (27*cells elements of the storage type each).
 * Errors: LBM_ERR_ARG for bad sizes/enums, LBM_ERR_OOM, LBM_ERR_CUDA. */
lbm_status lbm_create(const lbm_config* cfg, void* stream, lbm_ctx** out);

/* Free everything the context owns (the pool buffers in order on the context's stream,
 * which must still exist). Accepts NULL. */
lbm_status lbm_destroy(lbm_ctx* ctx);

/* Message of the last failed call on ctx ("" if none); a static string if ctx is NULL. */
const char* lbm_last_error(const lbm_ctx* ctx);

/* Set the state to the equilibrium f_i = f^eq_i(rho, u) (Sec. II.A, Eq.
 * EquilibriumDistribution) at time 0. rho: cells values; u: 3*cells values (SoA). */
lbm_status lbm_init(lbm_ctx* ctx, const float* rho, const float* u);

/* Set / read the pre-collision populations f_i(x, t) (absolute values, not deviations):
 * 27*cells floats, SoA in the velocity order. */
lbm_status lbm_set_state(lbm_ctx* ctx, const float* f);
lbm_status lbm_get_state(lbm_ctx* ctx, float* f);

/* The stored state itself, for checkpoints that resume bit for bit: 27 planes of
 * lbm_raw_state_bytes(ctx) / 27 bytes each in the context's storage type, as the next step
 * reads them (every storage holds deviations f - w, so the FP32 values of lbm_get_state,
 * w + (f - w), need not give back the same bits). Host or device memory; the calls
 * synchronise the stream. lbm_set_raw_state then treats the state as lbm_set_state does
 * (the step counter restarts and a forced context projects the restored state). */
long long lbm_raw_state_bytes(const lbm_ctx* ctx);
lbm_status lbm_get_raw_state(lbm_ctx* ctx, void* buf);
lbm_status lbm_set_raw_state(lbm_ctx* ctx, const void* buf);

/* Advance nsteps >= 0 steps of f_i(x + c_i, t + 1) = f_i + Omega_i + S_i (Sec. II.A):
 * one fused pull-stream-collide kernel per step. A forced step adds one small kernel
 * before it that turns the previous step's velocity projection and this step's draws into
 * the 16 force coefficients; the step kernel synthesises the force and projects its
 * velocity itself (no force or velocity field is stored).
 * Asynchronous. Density and NaN checks run inside the step kernel and latch a device
 * flag that lbm_check reports. LBM_ERR_STATE for an NCO context without weights, or a
 * forced context without enough random draws. */
lbm_status lbm_step(lbm_ctx* ctx, int nsteps);

/* Synchronise the stream and report LBM_ERR_UNSTABLE if any step so far saw a
 * non-finite value or a density outside the window, LBM_ERR_TIMEOUT if a wait of a
 * tensor-core step kernel on MMA completion ran out (the kernel then stopped early and the
 * state is not a valid step; lbm_last_error says whether the MMAs drained, in which case
 * the tensor memory was released). Every flag stays latched for the context's lifetime. */
lbm_status lbm_check(lbm_ctx* ctx);

/* Guard regions, a check of out-of-bounds writes that needs no sanitizer: 4 KB of a fixed
 * byte pattern sit before and after each of the context's two population buffers, which
 * every step, init and state kernel writes. lbm_check_guards synchronises the stream and
 * returns LBM_OK if all four regions still hold the pattern, else LBM_ERR_STATE with the
 * region and the count of changed bytes in lbm_last_error. lbm_selftest_guards changes one
 * guard byte (a plain memset of the context's own allocation), checks that
 * lbm_check_guards reports it, restores it and checks again: LBM_OK when both checks
 * answered as they should. */
lbm_status lbm_check_guards(lbm_ctx* ctx);
lbm_status lbm_selftest_guards(lbm_ctx* ctx);

/* Limit, in SM clock cycles, of each wait of the context's tensor-core step kernel on MMA
 * completion (the two-layer BF16 network and the split-BF16 network; default 2e9, about
 * 1 s at 2 GHz; the deep BF16 network and batches keep the default). A wait that
 * runs out ends the step kernel early with the LBM_ERR_TIMEOUT flag; before releasing its
 * tensor memory the kernel still waits, with the default limit, for the MMAs it had
 * started. 0 gives up at the first wait. For failure-detection tests; not part of the
 * method (the paper has no counterpart). LBM_ERR_ARG for cycles < 0. */
lbm_status lbm_set_wait_limit(lbm_ctx* ctx, long long cycles);

/* Density and bare velocity u = j / rho of the current pre-collision state
 * (Sec. II.A). rho: cells values (may be NULL); u: 3*cells values (may be NULL). */
lbm_status lbm_macroscopic(lbm_ctx* ctx, float* rho, float* u);

/* Kinetic energy k = (1/2) <|u|^2> of the current state, reduced in FP64 on the GPU.
 * ke: one double, host or device. */
lbm_status lbm_kinetic_energy(lbm_ctx* ctx, double* ke);

/* Energy spectrum of the current velocity field (Sec. II.D uses E(kappa)):
 * u^ = FFT(u)/cells per component (FP32 FFT), E[n] = sum over |k| rounding to n of
 * (1/2)|u^(k)|^2, accumulated in FP64. With mirror boundaries the field is first
 * unfolded to the full (2nx,2ny,2nz) box by the Taylor-Green parities. E: nbins
 * doubles (host or device); bins past the largest shell are zero. ke (may be NULL):
 * the kinetic energy from the same pass. Needs nx, ny, nz each a power of two times
 * 1 or 3 (FFT radices 2 and 3), at most 2048, else LBM_ERR_ARG. */
lbm_status lbm_energy_spectrum(lbm_ctx* ctx, double* E, int nbins, double* ke);

/* Network parameters of Phi (Sec. II.B: 27 -> 20 -> 20 -> 4, ReLU, 1064 values)
 * flattened as W1, b1, W2, b2, W3, b3 with each W row-major (out, in); or the deeper
 * network with a third hidden layer of 20 (Sec. IV: 27 -> 20 -> 20 -> 20 -> 4, 1484
 * values, W1, b1, W2, b2, W3, b3, W4, b4). theta: n floats in host or device memory;
 * n must be 1064 or 1484, else LBM_ERR_ARG. The adjoint and batches take the 1064-value
 * network only. */
lbm_status nco_set_weights(lbm_ctx* ctx, const float* theta, int n);

/* Start recording for nco_backward: from now on lbm_step keeps a device copy of the
 * state every k >= 1 steps (the current state is the first). Covers NCO contexts with
 * FP32 storage and FP32 network (either network depth; periodic, mirror or reduced
 * Taylor-Green boundary), else LBM_ERR_ARG. In a forced context every step's force is
 * recorded too (its 16 mode coefficients) and enters the adjoint as an input of that step:
 * the adjoint differentiates the Kupershtokh source through rho and u, not the force's own
 * dependence on the flow (the stirring is redrawn every step). Recording allocates one state-sized
 * buffer per checkpoint and ends at the next lbm_init / lbm_set_state. The weights must
 * not change between recording and the reverse pass. Checkpoints and the adjoint's work
 * buffers come from a stream-ordered memory pool the library keeps per device: memory a
 * finished recording or reverse pass releases stays reserved there for the next one (of
 * any context on that device) and goes back to the device when a context that used the
 * pool is destroyed (lbm_destroy trims the pool's unused memory). */
lbm_status lbm_record_begin(lbm_ctx* ctx, int k);

/* Reverse pass of the unrolled simulation since lbm_record_begin: the hand-written
 * adjoint (vector-Jacobian product) of each pull-stream + NCO collision step (Sec. II.A-B,
 * eqs. omegatheta and gconv_m; on the reduced Taylor-Green domain the streaming adjoint
 * is the inverse of the symmetry pull of Appendix A), segment by segment from the
 * checkpoints, recomputing the k states of a segment before walking it backwards.
 * Inputs: the cotangents of the final macroscopic fields, dL_du (3*cells) and/or dL_drho
 * (cells), host or device (either may be NULL, not both). Outputs (each may be NULL):
 * dL_dtheta, 1064 or 1484 floats (the count nco_set_weights was given) in its layout;
 * dL_df0, 27*cells floats, the cotangent of the populations at lbm_record_begin.
 * Synchronous. Allocates k + 2 state-sized work buffers on first use. LBM_ERR_STATE
 * without a recording or weights. */
lbm_status nco_backward(lbm_ctx* ctx, const float* dL_du, const float* dL_drho, float* dL_dtheta, float* dL_df0);

/* nco_backward for a loss that also depends on the kinetic energy k = (1/2)<|u|^2> (cell
 * mean, no density weight; lbm_kinetic_energy's definition) at recorded steps, as the
 * dissipation-rate loss of the time-dependent training does (Sec. IV: the MSE of -dk/dt
 * against a reference at 100 points of t in [0, 15], -dk/dt from k by finite differences;
 * the loss and its dL/dk are the caller's). obs_step[j] (host, 0 <= obs_step[j] <= the steps
 * taken since lbm_record_begin; repeats add up) and dL_dk[j] (host doubles) for j <
 * nobs; each adds dL/dk_j * dk/df to the cotangent of the state after obs_step[j] steps.
 * dL_du / dL_drho as in nco_backward, both may be NULL when nobs > 0. Same outputs,
 * buffers and errors as nco_backward; LBM_ERR_ARG for a step out of range or a
 * non-finite dL_dk. */
lbm_status nco_backward_ke(lbm_ctx* ctx, int nobs, const int* obs_step, const double* dL_dk, const float* dL_du,
                           const float* dL_drho, float* dL_dtheta, float* dL_df0);

/* Random phases of the spectral force for the next nsteps steps (Sec. II.C):
 * phi in [0, pi), psi in [0, 2 pi), each nsteps*16 doubles (host), one row of the 16
 * half-space modes per step, modes ordered by (|k|^2, kz, ky, kx). Appends to the
 * queue the next lbm_step calls consume. */
lbm_status lbm_force_draws(lbm_ctx* ctx, const double* phi, const double* psi, int nsteps);

/* The forcing state that lbm_get_state's populations do not hold (Sec. II.C): the
 * projection of the last step's pre-collision velocity onto the 16 forced modes, from which
 * the next step's force coefficients are formed, as 96 fixed-point sums (64-bit integers
 * whose scale depends on the grid size only). Saved next to lbm_get_raw_state's state, and
 * with the draws of the steps still to come queued again with lbm_force_draws, it resumes a
 * forced run bit for bit: restore with lbm_set_raw_state first (which projects the restored
 * state itself), then lbm_set_force_state. sums: 96 int64, host or device memory (the calls
 * synchronise the context's stream). LBM_ERR_STATE for an unforced context. */
lbm_status lbm_get_force_state(lbm_ctx* ctx, long long* sums);
lbm_status lbm_set_force_state(lbm_ctx* ctx, const long long* sums);

/* The library's own O_h tables (no device work, no context). R: 48*9 ints, row-major
 * 3x3 signed permutation matrices with (R c)_a = s_a c_{p(a)}; vperm: 48*27 with
 * c[vperm[g][i]] = R_g c_i; mperm, msign: 48*27 with (M Pi_g f)_k =
 * msign[g][k] * (M f)_{mperm[g][k]} in the printed moment order (Sec. II.B). Any
 * pointer may be NULL. */
lbm_status lbm_group_tables(int* R, int* vperm, int* mperm, int* msign);

/* The library's symmetry table of the reduced Taylor-Green domain (Appendix A; no device
 * work, no context): for each of the 27 blocks r = 9 (rz+1) + 3 (ry+1) + (rx+1) around
 * [0, pi/2]^3 (r = 13 is the domain itself, all zeros), the flow symmetry (A, t) that maps
 * the block back onto the domain: A as a 3x3 row-major integer matrix in A (27*9 ints),
 * t in units of pi/2 in k (27*3 ints, 0..3), and pmap (27*27 ints) with c[pmap[r][i]] =
 * A c_i. LBM_ERR_STATE if the derivation fails. Any pointer may be NULL. */
lbm_status lbm_tgv_reduced_table(int* A, int* k, int* pmap);

/* The energy-spectrum shell of every wave vector of an nx x ny x nz box (tools call, no
 * context, current device, synchronous), computed by the device code lbm_energy_spectrum
 * bins with: wave numbers k in FFT order (0, 1, ..., -1 per axis, x fastest) and shell n
 * with n^2 - n + 1 <= |k|^2 <= n^2 + n, the nearest integer to |k| (the reading of the
 * spectrum E(kappa) of Sec. II.D, which the paper uses without defining its bins).
 * shell: host memory, nx*ny*nz ints. LBM_ERR_ARG for empty or >= 2^31-cell boxes or a
 * NULL pointer, LBM_ERR_OOM / LBM_ERR_CUDA if the temporary device buffer fails. */
lbm_status lbm_spectrum_shells(int nx, int ny, int nz, int* shell);

/* Tensor-core self-test (no context, current device, synchronous): one CTA multiplies
 * fixed BF16 matrices with tcgen05.mma in the three shapes the network uses (M=128;
 * N/K = 80/32, 32/32, 16/80) and compares every product with a CUDA-core FP32 dot
 * product of the same values. max_err (host): the largest absolute difference, 0 when
 * the layouts are right (the test values make every product and sum exact).
 * LBM_ERR_TIMEOUT if an MMA completion wait ran out, LBM_ERR_CUDA on a runtime error. */
lbm_status lbm_selftest_tensor_cores(double* max_err);

/* Kinetic energy k = (1/2) <|u|^2> of populations the caller holds, with no device
 * allocation at all. The paper has no counterpart; this entry point is for callers
 * that cannot call cudaMalloc (for instance code whose device memory all comes from a
 * host framework's own pool, or that runs where an allocation would break its
 * contract) but still own their inputs and outputs.
 * f: device memory of the current device (or managed memory), 27*nx*ny*nz floats of
 * absolute pre-collision populations in the layout of lbm_get_state. ke: device memory of
 * the current device (or managed) for one double. stream: a cudaStream_t
 * passed as void* (NULL = legacy default stream). Asynchronous; no synchronisation.
 * Scratch: a fixed 32 KB array of 4096 partial sums in the library's device memory,
 * held by every GPU that loads the library until the process exits. It limits the
 * grid to nx*ny*nz <= 256^3 cells; larger grids, non-positive sizes, and NULL pointers
 * or pointers that are not memory of the current device return LBM_ERR_ARG before any
 * device work. The first call on a
 * device looks the scratch address up (cudaGetSymbolAddress) and caches it, so make
 * that first call before any stream capture. All calls share the one array: calls
 * that overlap on the GPU (other streams, other threads) race and must be ordered by
 * the caller. Every slot a call reads it has written first, so nothing needs clearing.
 * LBM_ERR_CUDA if a runtime call or launch fails. */
lbm_status lbm_kinetic_energy_noalloc(const float* f, int nx, int ny, int nz, double* ke, void* stream);

/* ---- Batches: many independent NCO instances in one persistent launch ----
 * All instances must use the NCO operator with the BF16 tensor-core network, periodic
 * boundaries and one common storage format; their grids, viscosities and forcing may
 * differ. The batch shares one network (lbm_batch_set_weights). Each step runs the
 * forcing kernels of the forced instances, one persistent tensor-core kernel over the
 * 128-cell tiles of every instance, and the forcing projections. */
typedef struct lbm_batch lbm_batch;

/* Create n instances from cfgs[0..n-1] on `stream` (a cudaStream_t as void*; NULL makes
 * the batch create and own a blocking stream, since graphs cannot be captured on the
 * legacy default stream). LBM_ERR_ARG for an unsupported configuration. */
lbm_status lbm_batch_create(int n, const lbm_config* cfgs, void* stream, lbm_batch** out);
lbm_status lbm_batch_destroy(lbm_batch* b);
const char* lbm_batch_last_error(const lbm_batch* b);

/* The i-th instance as an ordinary context (for lbm_init, lbm_force_draws,
 * lbm_macroscopic, ...). It stays owned by the batch. */
lbm_status lbm_batch_get(lbm_batch* b, int i, lbm_ctx** out);

/* Network parameters for every instance (as nco_set_weights). */
lbm_status lbm_batch_set_weights(lbm_batch* b, const float* theta, int n);

/* Autotuner of the tile shape of the batched network kernel: time it on the current state
 * without advancing it in each shape and keep the fastest; *choice (may be NULL) receives
 * the shape. Shapes: 0 = pairs of group elements shared by two warpgroups per tile (two
 * tiles in flight per SM, every MMA operand A in tensor memory, the default); 2, 3, 4 =
 * chunks of four group elements per warpgroup with that many warpgroups (tiles in flight)
 * per SM. The shapes differ in the rounding order of the network's FP32 sums (all within
 * the BF16 network's accuracy). The shape applies to the batch's instances also when one is
 * stepped alone with lbm_step, so every instance stays bit-identical to its own steps.
 * Synchronous. */
lbm_status lbm_batch_autotune(lbm_batch* b, int* choice);

/* Set the tile shape (0, 2, 3 or 4, as lbm_batch_autotune chooses) without timing; for
 * example a choice made earlier. LBM_ERR_ARG for any other value. */
lbm_status lbm_batch_set_tile_shape(lbm_batch* b, int shape);

/* Advance every instance nsteps steps. use_graph != 0 captures one step per buffer parity
 * into CUDA graphs on the first call (and again whenever an instance's buffers or random
 * draw queue changed) and replays them; use_graph == 0 launches directly. Forced instances
 * need nsteps random draws queued (LBM_ERR_STATE otherwise). Asynchronous. */
lbm_status lbm_batch_step(lbm_batch* b, int nsteps, int use_graph);

/* Synchronise and report the first error flag of the batch or of any instance. */
lbm_status lbm_batch_check(lbm_batch* b);

/* Library version string. */
const char* lbm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NCO_LBM_H */
