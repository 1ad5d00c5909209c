// lbm_abi.cu - the C ABI of include/lbm.h: context life cycle, argument checks, host/device
// marshalling and the per-step launch sequence. Every entry point catches its own errors and
// returns an lbm_status; nothing here throws across the ABI.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

using namespace lbm;

struct lbm_ctx {
    lbm_config cfg{};
    Dims d{};
    cudaStream_t stream = nullptr;
    int device = 0;
    size_t elem = 4;
    void* buf[2] = {nullptr, nullptr};
    void* buf_base[2] = {nullptr, nullptr};  // allocations: kGuardBytes, buf[p], kGuardBytes
    int cur = 0;
    float tau = 0.5f;
    bool have_weights = false;
    NetParams* net = nullptr;  // host copy handed to FP32 NCO launches by value
    void* tc_w = nullptr;      // device: packed BF16 operands of the tensor-core network
    int* d_status = nullptr;
    double* d_partials = nullptr;
    int npart = 0;
    double* d_scalar = nullptr;
    float* d_stage = nullptr;  // device staging for host-memory fields (lazy)
    size_t stage_elems = 0;
    float2* d_fft = nullptr;   // spectrum work (lazy)
    size_t fft_elems = 0;
    double* d_E = nullptr;
    int E_cap = 0;
    // forcing
    float* d_force = nullptr;
    float* d_u = nullptr;
    unsigned long long* d_fproj = nullptr;  // fixed-point projection sums of the next step's forcing
    float fscale = 0.0f;                     // force_proj_scale(ncell)
    double funit = 0.0;                      // force_proj_unit(ncell)
    int fblocks = 0;                         // blocks of a separate projection pass (batches)
    double* d_fhat = nullptr;
    double* d_draws = nullptr;  // queued draws, one row of kDrawRow per step (force_draw_trig)
    double* d_fconst = nullptr;  // per-mode forcing constants (force_mode_consts)
    float2* d_ftab = nullptr;    // per-axis phase tables (force_phase_table)
    SymRegion* d_sym = nullptr;  // reduced Taylor-Green domain: symmetry table (27 regions)
    long long draws_cap = 0, draws_head = 0, draws_tail = 0;  // rows
    long long t = 0;
    // recording for nco_backward: checkpoint every rec_k steps since lbm_record_begin
    int rec_k = 0;
    long long rec_steps = 0;
    std::vector<void*> ckpts;
    std::vector<double*> rec_fhat;  // forced contexts: the force coefficients of every recorded step
    std::vector<void*> adj_work;   // states of one segment (rec_k buffers), allocated by nco_backward
    float* adj_lam[2] = {nullptr, nullptr};
    double* adj_grad = nullptr;
    int adj_grad_len = 0;
    long long wait_cycles = kDefaultWaitCycles;  // limit of the tensor-core kernels' MMA waits
    int tc_shape = 0;  // tile shape of the BF16 tensor-core network (a batch's autotuned choice)
    // one step per buffer parity captured in CUDA graphs (lbm_step with nsteps >= 2, not
    // recording): captured on a private stream, launched on `stream`; a forced step reads its
    // row of draws at graph_head + *d_counter
    cudaStream_t gstream = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    long long* d_counter = nullptr;
    long long graph_head = 0;
    const double* graph_draws = nullptr;
    long long graph_cap = 0;
    std::string err;
};

static void drop_step_graphs(lbm_ctx* c) {
    for (cudaGraphExec_t& g : c->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

// Makes a context's device current for the duration of an entry point and restores the
// caller's afterwards, so that launches, pool allocations and copies land on that GPU.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        int cur = 0;
        if (cudaGetDevice(&cur) == cudaSuccess && cur != dev && cudaSetDevice(dev) == cudaSuccess) prev = cur;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard&) = delete;
    DeviceGuard& operator=(const DeviceGuard&) = delete;
};

namespace {

const char* kNoCtxError = "invalid context (NULL)";

lbm_status fail(lbm_ctx* c, lbm_status code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

lbm_status cuda_fail(lbm_ctx* c, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(c, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, m);
}

#define LBM_CK(ctx, call)                                         \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);  \
    } while (0)

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at{};
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t storage_bytes(int storage) { return storage == LBM_STORE_F32 ? 4 : 2; }

lbm_status ensure_stage(lbm_ctx* c, size_t elems) {
    if (c->stage_elems >= elems) return LBM_OK;
    if (c->d_stage) cudaFree(c->d_stage);
    c->d_stage = nullptr;
    c->stage_elems = 0;
    LBM_CK(c, cudaMalloc(&c->d_stage, elems * sizeof(float)));
    c->stage_elems = elems;
    return LBM_OK;
}

// Bring a caller field of `elems` floats to the device (copy if it is host memory).
lbm_status device_input(lbm_ctx* c, const float* p, size_t elems, size_t stage_off, const float** out) {
    if (is_device_ptr(p)) {
        *out = p;
        return LBM_OK;
    }
    LBM_CK(c, cudaMemcpyAsync(c->d_stage + stage_off, p, elems * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    *out = c->d_stage + stage_off;
    return LBM_OK;
}

}  // namespace

namespace lbm {

const GroupTables& group_tables() {
    static const GroupTables t = make_group();
    return t;
}

static int tensor_to_printed(int e) {
    for (int k = 0; k < Q; ++k)
        if (kPrinted.e[k] == e) return k;
    return -1;
}

// Appendix A: the reduced Taylor-Green domain. The symmetries (A, t) of the flow
// u = (sin x cos y cos z, -cos x sin y cos z, 0) with A a signed permutation (a symmetry of
// the lattice) and t in (pi/2) Z^3 are found by testing every candidate on fixed
// pseudo-random points; there are 64 modulo the 2 pi period, and [0, pi/2]^3 is a
// fundamental domain. Each of the 26 neighbouring blocks is mapped back by exactly one.
bool tgv_reduced_table(SymRegion* out) {
    constexpr double kPi = 3.14159265358979323846;
    auto tgv = [](const double* p, double* u) {
        u[0] = std::sin(p[0]) * std::cos(p[1]) * std::cos(p[2]);
        u[1] = -std::cos(p[0]) * std::sin(p[1]) * std::cos(p[2]);
        u[2] = 0.0;
    };
    double pts[64][3];
    uint64_t st = 0x9E3779B97F4A7C15ull;
    for (auto& p : pts)
        for (double& v : p) {
            st = st * 6364136223846793005ull + 1442695040888963407ull;
            v = static_cast<double>(st >> 11) * (1.0 / 9007199254740992.0) * 2.0 * kPi;
        }
    struct G { int perm[3], sign[3], k[3]; };
    std::vector<G> group;
    const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (const auto& pm : perms)
        for (int sb = 0; sb < 8; ++sb)
            for (int kk = 0; kk < 64; ++kk) {
                G g{};
                for (int a = 0; a < 3; ++a) {
                    g.perm[a] = pm[a];
                    g.sign[a] = (sb >> a) & 1 ? -1 : 1;
                }
                g.k[0] = kk & 3;
                g.k[1] = (kk >> 2) & 3;
                g.k[2] = kk >> 4;
                bool ok = true;
                for (const auto& p : pts) {
                    double q[3], uq[3], up[3];
                    for (int a = 0; a < 3; ++a) q[a] = g.sign[a] * p[g.perm[a]] + g.k[a] * kPi / 2;
                    tgv(q, uq);
                    tgv(p, up);
                    for (int a = 0; a < 3; ++a)
                        if (std::fabs(uq[a] - g.sign[a] * up[g.perm[a]]) > 1e-9) ok = false;
                    if (!ok) break;
                }
                if (ok) group.push_back(g);
            }
    if (group.size() != 64) return false;
    for (int r = 0; r < 27; ++r) {
        SymRegion& e = out[r];
        e = SymRegion{};
        const int rv[3] = {r % 3 - 1, (r / 3) % 3 - 1, r / 9 - 1};
        if (r == 13) continue;  // the domain itself
        int found = 0;
        for (const G& g : group) {
            bool inside = true;
            for (int a = 0; a < 3; ++a) {  // centre of the neighbouring block, in units of pi/2
                double v = g.sign[a] * (rv[g.perm[a]] + 0.5) + g.k[a];
                v = std::fmod(v, 4.0);
                if (v < 0) v += 4.0;
                inside = inside && v > 0.0 && v < 1.0;
            }
            if (!inside) continue;
            ++found;
            for (int a = 0; a < 3; ++a) {
                e.perm[a] = static_cast<signed char>(g.perm[a]);
                e.sign[a] = static_cast<signed char>(g.sign[a]);
                e.k[a] = static_cast<signed char>(g.k[a]);
            }
            for (int i = 0; i < Q; ++i) {
                const int c[3] = {cx_of(i), cy_of(i), cz_of(i)};
                int ac[3];
                for (int a = 0; a < 3; ++a) ac[a] = g.sign[a] * c[g.perm[a]];
                e.pmap[i] = static_cast<unsigned char>(9 * (ac[2] + 1) + 3 * (ac[1] + 1) + (ac[0] + 1));
            }
        }
        if (found != 1) return false;
    }
    return true;
}

void make_net_params(const float* theta, bool deep, NetParams* out) {
    const float* W1 = theta;                 // (20, 27) printed column order
    const float* b1 = W1 + kHidden * Q;
    const float* W2 = b1 + kHidden;
    const float* b2 = W2 + kHidden * kHidden;
    const float* Wd = b2 + kHidden;          // deep network: the third hidden layer comes next
    const float* bd = Wd + kHidden * kHidden;
    const float* W3 = deep ? bd + kHidden : b2 + kHidden;
    const float* b3 = W3 + kOut * kHidden;
    const GroupTables& g = group_tables();
    for (int p = 0; p < 6; ++p) {
        const int gp = p * 8;  // element with axis permutation p and no reflection
        for (int j = 0; j < kHidden; ++j)
            for (int k = 0; k < Q; ++k) {
                const int t = g.mperm_t[gp][kPrinted.e[k]];
                out->W1p[p][j][t] = W1[j * Q + k];
            }
    }
    std::memcpy(out->b1, b1, sizeof(out->b1));
    std::memcpy(out->W2, W2, sizeof(out->W2));
    std::memcpy(out->b2, b2, sizeof(out->b2));
    std::memcpy(out->W3, W3, sizeof(out->W3));
    std::memcpy(out->b3, b3, sizeof(out->b3));
    out->deep = deep ? 1 : 0;
    if (deep) {
        std::memcpy(out->Wd, Wd, sizeof(out->Wd));
        std::memcpy(out->bd, bd, sizeof(out->bd));
    } else {
        std::memset(out->Wd, 0, sizeof(out->Wd));
        std::memset(out->bd, 0, sizeof(out->bd));
    }
}

}  // namespace lbm

extern "C" {

const char* lbm_version(void) { return "nco-lbm-gb300 0.1 (sm_103a)"; }

const char* lbm_last_error(const lbm_ctx* ctx) { return ctx ? ctx->err.c_str() : kNoCtxError; }

lbm_status lbm_tgv_reduced_table(int* A, int* k, int* pmap) {
    SymRegion t[27];
    if (!tgv_reduced_table(t)) return LBM_ERR_STATE;
    for (int r = 0; r < 27; ++r) {
        if (A) {
            for (int a = 0; a < 9; ++a) A[r * 9 + a] = 0;
            if (r != 13)
                for (int a = 0; a < 3; ++a) A[r * 9 + a * 3 + t[r].perm[a]] = t[r].sign[a];
        }
        if (k)
            for (int a = 0; a < 3; ++a) k[r * 3 + a] = t[r].k[a];
        if (pmap)
            for (int i = 0; i < Q; ++i) pmap[r * Q + i] = t[r].pmap[i];
    }
    return LBM_OK;
}

lbm_status lbm_group_tables(int* R, int* vperm, int* mperm, int* msign) {
    const GroupTables& g = group_tables();
    for (int a = 0; a < 48; ++a) {
        if (R)
            for (int k = 0; k < 9; ++k) R[a * 9 + k] = g.R[a][k];
        for (int k = 0; k < Q; ++k) {
            if (vperm) vperm[a * Q + k] = g.vperm[a][k];
            const int e = kPrinted.e[k];
            if (mperm) mperm[a * Q + k] = tensor_to_printed(g.mperm_t[a][e]);
            if (msign) msign[a * Q + k] = g.msign_t[a][e];
        }
    }
    return LBM_OK;
}

lbm_status lbm_spectrum_shells(int nx, int ny, int nz, int* shell) {
    if (!shell || nx < 1 || ny < 1 || nz < 1) return LBM_ERR_ARG;
    const long long n = static_cast<long long>(nx) * ny * nz;
    if (n >= (1LL << 31)) return LBM_ERR_ARG;
    int* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(int) * static_cast<size_t>(n));
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
    e = launch_spectrum_shells(Dims{nx, ny, nz, n}, d, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(shell, d, sizeof(int) * static_cast<size_t>(n), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

lbm_status lbm_selftest_tensor_cores(double* max_err) {
    if (!max_err) return LBM_ERR_ARG;
    float* d_err = nullptr;
    int* d_status = nullptr;
    lbm_status st = LBM_OK;
    if (cudaMalloc(&d_err, sizeof(float)) != cudaSuccess || cudaMalloc(&d_status, sizeof(int)) != cudaSuccess) {
        st = LBM_ERR_OOM;
    } else {
        float herr = 0.0f;
        int hst = 0;
        cudaError_t e = cudaMemset(d_err, 0, sizeof(float));
        if (e == cudaSuccess) e = cudaMemset(d_status, 0, sizeof(int));
        if (e == cudaSuccess) e = run_tc_selftest(d_err, d_status, nullptr);
        if (e == cudaSuccess) e = cudaMemcpy(&herr, d_err, sizeof(float), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(&hst, d_status, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = LBM_ERR_CUDA;
        else if (hst & 2) st = LBM_ERR_TIMEOUT;
        *max_err = herr;
    }
    if (d_err) cudaFree(d_err);
    if (d_status) cudaFree(d_status);
    return st;
}

// Recorded force coefficients: blocks of kFhatBlock steps x kFhatDoubles (16 modes x 3
// complex components).
constexpr int kFhatDoubles = kForcedModes * 6;
constexpr long long kFhatBlock = 512;

static double* rec_fhat_at(lbm_ctx* c, long long t) {
    return c->rec_fhat[static_cast<size_t>(t / kFhatBlock)] + (t % kFhatBlock) * kFhatDoubles;
}

// Recording and adjoint buffers come from the library's own stream-ordered pool (one per
// device, created on first use, keeping released memory for reuse): a checkpoint every k
// steps then costs no device-wide synchronisation, so contexts stepped side by side on
// their own streams do not stall one another, and repeated training steps reuse memory.
// lbm_destroy gives the pool's unused memory back to the device (pool_trim).
static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[64] = {};

static cudaError_t pool_alloc(const lbm_ctx* c, void** p, size_t bytes, cudaStream_t s) {
    const int dev = c->device;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        if (!g_pools[dev]) {
            cudaMemPoolProps props{};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            cudaError_t e = cudaMemPoolCreate(&pool, &props);
            if (e != cudaSuccess) return e;
            uint64_t keep = UINT64_MAX;
            e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            if (e != cudaSuccess) return e;
            g_pools[dev] = pool;
        }
        pool = g_pools[dev];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

// Release the pool's memory that no allocation holds (other contexts' buffers stay).
static void pool_trim(int dev) {
    if (dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (g_pools[dev]) cudaMemPoolTrimTo(g_pools[dev], 0);
}

static void free_recording(lbm_ctx* c) {
    for (void* p : c->ckpts) cudaFreeAsync(p, c->stream);
    c->ckpts.clear();
    for (double* p : c->rec_fhat) cudaFreeAsync(p, c->stream);
    c->rec_fhat.clear();
    c->rec_k = 0;
    c->rec_steps = 0;
}

static void free_adjoint(lbm_ctx* c) {
    for (void* p : c->adj_work) cudaFreeAsync(p, c->stream);
    c->adj_work.clear();
    for (float*& p : c->adj_lam) {
        if (p) cudaFreeAsync(p, c->stream);
        p = nullptr;
    }
    if (c->adj_grad) cudaFreeAsync(c->adj_grad, c->stream);
    c->adj_grad = nullptr;
    c->adj_grad_len = 0;
}

lbm_status lbm_destroy(lbm_ctx* c) {
    if (!c) return LBM_OK;
    DeviceGuard guard(c->device);
    const bool pooled = !c->ckpts.empty() || !c->rec_fhat.empty() || !c->adj_work.empty() || c->adj_grad ||
                        c->adj_lam[0] || c->adj_lam[1];
    free_recording(c);
    free_adjoint(c);
    void* devs[] = {c->buf_base[0], c->buf_base[1], c->tc_w, c->d_status, c->d_partials, c->d_scalar, c->d_stage,
                    c->d_fft, c->d_E, c->d_force, c->d_u, c->d_fproj, c->d_fhat, c->d_draws, c->d_sym,
                    c->d_fconst, c->d_ftab};
    for (void* p : devs)
        if (p) cudaFree(p);
    if (pooled) {  // the stream-ordered frees above must have run before the pool can give memory back
        cudaStreamSynchronize(c->stream);
        pool_trim(c->device);
    }
    drop_step_graphs(c);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    if (c->d_counter) cudaFree(c->d_counter);
    delete c->net;
    delete c;
    return LBM_OK;
}

lbm_status lbm_create(const lbm_config* cfg, void* stream, lbm_ctx** out) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (!cfg) return LBM_ERR_ARG;
    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_ERR_OOM;
    c->cfg = *cfg;
    const long long n = static_cast<long long>(cfg->nx) * cfg->ny * cfg->nz;
    auto bad = [&](const char* m) {
        std::fprintf(stderr, "lbm_create: %s\n", m);
        lbm_destroy(c);
        return LBM_ERR_ARG;
    };
    if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1) return bad("grid sizes must be >= 1");
    if (n * Q >= (1LL << 31)) return bad("27*cells must stay below 2^31");
    if (!(cfg->nu > 0.0)) return bad("nu must be > 0");
    if (cfg->op < LBM_OP_BGK || cfg->op > LBM_OP_REG) return bad("unknown operator");
    if (cfg->storage < LBM_STORE_F32 || cfg->storage > LBM_STORE_BF16_DEV) return bad("unknown storage");
    if (cfg->net_precision != LBM_NET_F32 && cfg->net_precision != LBM_NET_BF16 &&
        cfg->net_precision != LBM_NET_BF16X3)
        return bad("unknown network precision");
    if (cfg->boundary != LBM_BC_PERIODIC && cfg->boundary != LBM_BC_MIRROR && cfg->boundary != LBM_BC_TGV_REDUCED)
        return bad("unknown boundary");
    if (cfg->boundary == LBM_BC_TGV_REDUCED && (cfg->ny != cfg->nx || cfg->nz != cfg->nx))
        return bad("the reduced Taylor-Green domain is a cube");
    if (cfg->forcing != 0 && cfg->forcing != 1) return bad("unknown forcing");
    if (cfg->forcing == 1 && cfg->boundary != LBM_BC_PERIODIC) return bad("spectral forcing needs periodic boundaries");
    if (cfg->op == LBM_OP_NCO && cfg->net_precision == LBM_NET_BF16 && !nco_tc_supported(cfg->storage, cfg->boundary))
        return bad("tensor-core network not available for this storage/boundary");
    c->d = Dims{cfg->nx, cfg->ny, cfg->nz, n};
    c->stream = static_cast<cudaStream_t>(stream);
    c->tau = static_cast<float>(3.0 * cfg->nu + 0.5);
    if (c->cfg.rho_min == 0.0 && c->cfg.rho_max == 0.0) {
        c->cfg.rho_min = 0.5;
        c->cfg.rho_max = 2.0;
    }
    c->elem = storage_bytes(cfg->storage);
    cudaError_t e = cudaGetDevice(&c->device);
    lbm_status st = LBM_OK;
    auto alloc = [&](void** p, size_t bytes) {
        if (st != LBM_OK) return;
        cudaError_t ee = cudaMalloc(p, bytes);
        if (ee != cudaSuccess) st = cuda_fail(c, ee, "cudaMalloc");
    };
    if (e != cudaSuccess) st = cuda_fail(c, e, "cudaGetDevice");
    const size_t state_bytes = static_cast<size_t>(n) * Q * c->elem;
    for (int p = 0; p < 2; ++p) {  // each buffer between two guard regions of a fixed pattern
        alloc(&c->buf_base[p], state_bytes + 2 * kGuardBytes);
        if (c->buf_base[p]) {
            unsigned char* base = static_cast<unsigned char*>(c->buf_base[p]);
            c->buf[p] = base + kGuardBytes;
            cudaError_t ee = cudaMemset(base, kGuardPattern, kGuardBytes);
            if (ee == cudaSuccess) ee = cudaMemset(base + kGuardBytes + state_bytes, kGuardPattern, kGuardBytes);
            if (ee != cudaSuccess && st == LBM_OK) st = cuda_fail(c, ee, "cudaMemset");
        }
    }
    alloc(reinterpret_cast<void**>(&c->d_status), sizeof(int));
    c->npart = kinetic_energy_blocks(c->d);
    alloc(reinterpret_cast<void**>(&c->d_partials), sizeof(double) * c->npart);
    alloc(reinterpret_cast<void**>(&c->d_scalar), sizeof(double) * 2);
    if (cfg->op == LBM_OP_NCO && cfg->net_precision == LBM_NET_BF16) alloc(&c->tc_w, nco_tc_weight_bytes());
    if (cfg->op == LBM_OP_NCO && cfg->net_precision == LBM_NET_BF16X3) alloc(&c->tc_w, nco_tc3_weight_bytes());
    if (cfg->boundary == LBM_BC_TGV_REDUCED) {
        SymRegion table[27];
        if (!tgv_reduced_table(table) && st == LBM_OK) st = fail(c, LBM_ERR_STATE, "reduced Taylor-Green table");
        alloc(reinterpret_cast<void**>(&c->d_sym), sizeof(table));
        if (st == LBM_OK) {
            cudaError_t ee = cudaMemcpy(c->d_sym, table, sizeof(table), cudaMemcpyHostToDevice);
            if (ee != cudaSuccess) st = cuda_fail(c, ee, "cudaMemcpy");
        }
        c->d.sym = c->d_sym;
    }
    if (cfg->forcing == 1) {
        alloc(reinterpret_cast<void**>(&c->d_force), sizeof(float) * 3 * n);
        alloc(reinterpret_cast<void**>(&c->d_u), sizeof(float) * 3 * n);
        c->fblocks = force_project_blocks(c->d);
        c->fscale = force_proj_scale(c->d.ncell);
        c->funit = force_proj_unit(c->d.ncell);
        alloc(reinterpret_cast<void**>(&c->d_fproj), sizeof(unsigned long long) * 6 * kForcedModes);
        alloc(reinterpret_cast<void**>(&c->d_fhat), sizeof(double) * kForcedModes * 6);
        alloc(reinterpret_cast<void**>(&c->d_fconst), sizeof(double) * kForcedModes * kForceConsts);
        alloc(reinterpret_cast<void**>(&c->d_ftab), sizeof(float2) * 2 * (cfg->nx + cfg->ny + cfg->nz));
        if (st == LBM_OK) {
            std::vector<double> consts(kForcedModes * kForceConsts);
            force_mode_consts(ForceParams{cfg->force_power, cfg->force_kf, cfg->force_c, cfg->force_ka, cfg->force_kb},
                              consts.data());
            std::vector<float2> tab(2 * static_cast<size_t>(cfg->nx + cfg->ny + cfg->nz));
            force_phase_table(c->d, tab.data());
            cudaError_t ee = cudaMemcpy(c->d_fconst, consts.data(), sizeof(double) * consts.size(), cudaMemcpyHostToDevice);
            if (ee == cudaSuccess)
                ee = cudaMemcpy(c->d_ftab, tab.data(), sizeof(float2) * tab.size(), cudaMemcpyHostToDevice);
            if (ee != cudaSuccess) st = cuda_fail(c, ee, "cudaMemcpy");
        }
    }
    if (st == LBM_OK) {
        cudaError_t ee = cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
        if (ee == cudaSuccess) ee = cudaMemsetAsync(c->buf[0], 0, static_cast<size_t>(n) * Q * c->elem, c->stream);
        if (ee != cudaSuccess) st = cuda_fail(c, ee, "cudaMemsetAsync");
    }
    if (st != LBM_OK) {
        std::fprintf(stderr, "lbm_create: %s\n", c->err.c_str());
        lbm_destroy(c);
        return st;
    }
    *out = c;
    return LBM_OK;
}

static lbm_status after_state_change(lbm_ctx* c) {
    c->t = 0;
    free_recording(c);
    if (c->cfg.forcing == 1) {
        // the force of step 0 uses the projection of the initial field (Sec. II.C reading)
        LBM_CK(c, launch_macroscopic(c->d, c->cfg.storage, c->cfg.boundary, c->buf[c->cur], nullptr, c->d_u, c->stream));
        LBM_CK(c, cudaMemsetAsync(c->d_fproj, 0, sizeof(unsigned long long) * 6 * kForcedModes, c->stream));
        LBM_CK(c, launch_force_project(c->d, c->d_u, c->d_ftab, c->d_fproj, c->fscale, c->stream));
    }
    return LBM_OK;
}

lbm_status lbm_init(lbm_ctx* c, const float* rho, const float* u) {
    if (!c) return LBM_ERR_ARG;
    DeviceGuard guard(c->device);
    if (!rho || !u) return fail(c, LBM_ERR_ARG, "lbm_init: rho and u are required");
    const size_t n = static_cast<size_t>(c->d.ncell);
    const bool host = !is_device_ptr(rho) || !is_device_ptr(u);
    if (host) {
        lbm_status st = ensure_stage(c, 4 * n);
        if (st) return st;
    }
    const float *dr = nullptr, *du = nullptr;
    lbm_status st = device_input(c, rho, n, 0, &dr);
    if (st) return st;
    st = device_input(c, u, 3 * n, n, &du);
    if (st) return st;
    LBM_CK(c, launch_init_eq(c->d, c->cfg.storage, c->cfg.boundary, dr, du, c->buf[c->cur], c->stream));
    return after_state_change(c);
}

lbm_status lbm_set_state(lbm_ctx* c, const float* f) {
    if (!c) return LBM_ERR_ARG;
    DeviceGuard guard(c->device);
    if (!f) return fail(c, LBM_ERR_ARG, "lbm_set_state: f is required");
    const size_t n = static_cast<size_t>(c->d.ncell);
    const float* df = f;
    if (!is_device_ptr(f)) {
        lbm_status st = ensure_stage(c, Q * n);
        if (st) return st;
        st = device_input(c, f, Q * n, 0, &df);
        if (st) return st;
    }
    LBM_CK(c, launch_set_state(c->d, c->cfg.storage, c->cfg.boundary, df, c->buf[c->cur], c->stream));
    return after_state_change(c);
}

lbm_status lbm_get_state(lbm_ctx* c, float* f) {
    if (!c) return LBM_ERR_ARG;
    DeviceGuard guard(c->device);
    if (!f) return fail(c, LBM_ERR_ARG, "lbm_get_state: f is required");
    const size_t n = static_cast<size_t>(c->d.ncell);
    if (is_device_ptr(f)) {
        LBM_CK(c, launch_get_state(c->d, c->cfg.storage, c->cfg.boundary, c->buf[c->cur], f, c->stream));
        return LBM_OK;
    }
    lbm_status st = ensure_stage(c, Q * n);
    if (st) return st;
    LBM_CK(c, launch_get_state(c->d, c->cfg.storage, c->cfg.boundary, c->buf[c->cur], c->d_stage, c->stream));
    LBM_CK(c, cudaMemcpyAsync(f, c->d_stage, Q * n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    LBM_CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status nco_set_weights(lbm_ctx* c, const float* theta, int n) {
    if (!c) return LBM_ERR_ARG;
    DeviceGuard guard(c->device);
    if (!theta || (n != kNumTheta && n != kNumThetaDeep))
        return fail(c, LBM_ERR_ARG, "nco_set_weights: expected 1064 (two hidden layers) or 1484 (three) parameters");
    const bool deep = n == kNumThetaDeep;
    std::vector<float> h(n);
    if (is_device_ptr(theta)) {
        LBM_CK(c, cudaMemcpyAsync(h.data(), theta, sizeof(float) * n, cudaMemcpyDeviceToHost, c->stream));
        LBM_CK(c, cudaStreamSynchronize(c->stream));
    } else {
        std::memcpy(h.data(), theta, sizeof(float) * n);
    }
    if (!c->net) {
        c->net = new (std::nothrow) NetParams();
        if (!c->net) return fail(c, LBM_ERR_OOM, "nco_set_weights: host allocation failed");
    }
    make_net_params(h.data(), deep, c->net);
    drop_step_graphs(c);  // the FP32 network's parameters are kernel arguments of the captured steps
    if (c->tc_w) {
        const bool split = c->cfg.net_precision == LBM_NET_BF16X3;
        std::vector<unsigned char> packed(split ? nco_tc3_weight_bytes() : nco_tc_weight_bytes());
        if (split) nco_tc3_pack_weights(h.data(), deep, packed.data());
        else nco_tc_pack_weights(h.data(), deep, packed.data());
        LBM_CK(c, cudaMemcpyAsync(c->tc_w, packed.data(), packed.size(), cudaMemcpyHostToDevice, c->stream));
        LBM_CK(c, cudaStreamSynchronize(c->stream));  // `packed` is pageable and goes out of scope
    }
    c->have_weights = true;
    return LBM_OK;
}

long long lbm_raw_state_bytes(const lbm_ctx* c) {
    return c ? c->d.ncell * Q * static_cast<long long>(c->elem) : 0;
}

lbm_status lbm_get_raw_state(lbm_ctx* c, void* buf) {
    if (!c) return LBM_ERR_ARG;
    DeviceGuard guard(c->device);
    if (!buf) return fail(c, LBM_ERR_ARG, "lbm_get_raw_state: buf is required");
    LBM_CK(c, cudaMemcpyAsync(buf, c->buf[c->cur], static_cast<size_t>(lbm_raw_state_bytes(c)), cudaMemcpyDefault,
                              c->stream));
    LBM_CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status lbm_set_raw_state(lbm_ctx* c, const void* buf) {
    if (!c) return LBM_ERR_ARG;
    DeviceGuard guard(c->device);
    if (!buf) return fail(c, LBM_ERR_ARG, "lbm_set_raw_state: buf is required");
    LBM_CK(c, cudaMemcpyAsync(c->buf[c->cur], buf, static_cast<size_t>(lbm_raw_state_bytes(c)), cudaMemcpyDefault,
                              c->stream));
    LBM_CK(c, cudaStreamSynchronize(c->stream));
    return after_state_change(c);
}

lbm_status lbm_get_force_state(lbm_ctx* c, long long* sums) {
    if (!c) return LBM_ERR_ARG;
    DeviceGuard guard(c->device);
    if (c->cfg.forcing != 1) return fail(c, LBM_ERR_STATE, "lbm_get_force_state: context is not forced");
    if (!sums) return fail(c, LBM_ERR_ARG, "lbm_get_force_state: sums is required");
    LBM_CK(c, cudaMemcpyAsync(sums, c->d_fproj, sizeof(long long) * 6 * kForcedModes, cudaMemcpyDefault, c->stream));
    LBM_CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status lbm_set_force_state(lbm_ctx* c, const long long* sums) {
    if (!c) return LBM_ERR_ARG;
    DeviceGuard guard(c->device);
    if (c->cfg.forcing != 1) return fail(c, LBM_ERR_STATE, "lbm_set_force_state: context is not forced");
    if (!sums) return fail(c, LBM_ERR_ARG, "lbm_set_force_state: sums is required");
    LBM_CK(c, cudaMemcpyAsync(c->d_fproj, sums, sizeof(long long) * 6 * kForcedModes, cudaMemcpyDefault, c->stream));
    LBM_CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status lbm_force_draws(lbm_ctx* c, const double* phi, const double* psi, int nsteps) {
    if (!c) return LBM_ERR_ARG;
    DeviceGuard guard(c->device);
    if (c->cfg.forcing != 1) return fail(c, LBM_ERR_STATE, "lbm_force_draws: context is not forced");
    if (nsteps < 0 || (nsteps > 0 && (!phi || !psi))) return fail(c, LBM_ERR_ARG, "lbm_force_draws: bad arguments");
    if (nsteps == 0) return LBM_OK;
    constexpr size_t row = kDrawRow;  // doubles per step
    if (c->draws_tail + nsteps > c->draws_cap) {
        const long long pending = c->draws_tail - c->draws_head;
        long long cap = std::max<long long>(2 * c->draws_cap, pending + nsteps);
        double* nb = nullptr;
        LBM_CK(c, cudaMalloc(&nb, sizeof(double) * row * cap));
        if (pending > 0)
            LBM_CK(c, cudaMemcpyAsync(nb, c->d_draws + c->draws_head * row, sizeof(double) * row * pending,
                                      cudaMemcpyDeviceToDevice, c->stream));
        LBM_CK(c, cudaStreamSynchronize(c->stream));
        if (c->d_draws) cudaFree(c->d_draws);
        c->d_draws = nb;
        c->draws_cap = cap;
        c->draws_head = 0;
        c->draws_tail = pending;
    }
    std::vector<double> rows(row * static_cast<size_t>(nsteps));
    for (int t = 0; t < nsteps; ++t)
        force_draw_trig(phi + static_cast<size_t>(t) * kForcedModes, psi + static_cast<size_t>(t) * kForcedModes,
                        rows.data() + static_cast<size_t>(t) * row);
    LBM_CK(c, cudaMemcpyAsync(c->d_draws + c->draws_tail * row, rows.data(), sizeof(double) * rows.size(),
                              cudaMemcpyHostToDevice, c->stream));
    LBM_CK(c, cudaStreamSynchronize(c->stream));  // `rows` is pageable and goes out of scope
    c->draws_tail += nsteps;
    return LBM_OK;
}

// One step's device work from buffer parity p on stream s. A forced step is two launches:
// the forcing coefficients from the projection sums of the step before (draw row `row`, or
// with `indexed` the row graph_head + *d_counter, advancing the counter), then the step
// kernel, which synthesises the force per cell and adds its velocity's projection to the
// sums for the next step.
static lbm_status enqueue_step(lbm_ctx* c, int p, cudaStream_t s, const double* row, bool indexed) {
    StepArgs a{};
    a.d = c->d;
    a.src = c->buf[p];
    a.dst = c->buf[1 - p];
    a.status = c->d_status;
    a.tau = c->tau;
    a.rho_min = static_cast<float>(c->cfg.rho_min);
    a.rho_max = static_cast<float>(c->cfg.rho_max);
    const bool forced = c->cfg.forcing == 1;
    FusedForce ff{};
    if (forced) {
        if (indexed)
            LBM_CK(c, launch_force_coeffs_indexed(c->d_fproj, c->funit, c->d_draws, c->d_counter, c->graph_head,
                                                  c->draws_cap, c->d_fconst, c->d_fhat, s));
        else
            LBM_CK(c, launch_force_coeffs(c->d_fproj, c->funit, row, c->d_fconst, c->d_fhat, s));
        ff = FusedForce{c->d_fhat, c->d_ftab, c->d_fproj, c->fscale};
    }
    LBM_CK(c, launch_step(a, forced ? &ff : nullptr, c->cfg.op, c->cfg.storage, c->cfg.boundary,
                          c->cfg.net_precision, c->net, c->tc_w, c->tc_shape, c->wait_cycles, s));
    return LBM_OK;
}

// Capture one step per buffer parity unless the graphs in hand still fit (a forced step's
// graph depends on the draw queue it reads).
static lbm_status ensure_step_graphs(lbm_ctx* c) {
    const bool forced = c->cfg.forcing == 1;
    if (c->graph[0] && (!forced || (c->graph_draws == c->d_draws && c->graph_cap == c->draws_cap))) return LBM_OK;
    drop_step_graphs(c);
    if (!c->gstream) LBM_CK(c, cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
    if (forced && !c->d_counter) LBM_CK(c, cudaMalloc(reinterpret_cast<void**>(&c->d_counter), sizeof(long long)));
    c->graph_head = c->draws_head;
    c->graph_draws = c->d_draws;
    c->graph_cap = c->draws_cap;
    for (int p = 0; p < 2; ++p) {
        cudaGraph_t g = nullptr;
        LBM_CK(c, cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal));
        const lbm_status st = enqueue_step(c, p, c->gstream, nullptr, true);
        const cudaError_t ce = cudaStreamEndCapture(c->gstream, &g);
        if (st) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (ce != cudaSuccess) return cuda_fail(c, ce, "graph capture");
        const cudaError_t ie = cudaGraphInstantiate(&c->graph[p], g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) return cuda_fail(c, ie, "graph instantiate");
    }
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* c, int nsteps) {
    if (!c) return LBM_ERR_ARG;
    if (nsteps < 0) return fail(c, LBM_ERR_ARG, "lbm_step: nsteps < 0");
    if (c->cfg.op == LBM_OP_NCO && !c->have_weights) return fail(c, LBM_ERR_STATE, "lbm_step: call nco_set_weights first");
    const bool forced = c->cfg.forcing == 1;
    if (forced && (c->draws_tail - c->draws_head) < nsteps)
        return fail(c, LBM_ERR_STATE, "lbm_step: not enough random draws queued (lbm_force_draws)");
    DeviceGuard guard(c->device);
    // steps after the first of a call replay CUDA graphs, unless a recording needs its
    // per-step host work (the first step runs directly: it also sets the kernels' attributes)
    const bool graphs = nsteps >= 2 && c->rec_k == 0;
    for (int k = 0; k < nsteps; ++k) {
        if (graphs && k == 1) {
            lbm_status st = ensure_step_graphs(c);
            if (st) return st;
            if (forced) LBM_CK(c, launch_counter_set(c->d_counter, c->draws_head - c->graph_head, c->stream));
            for (; k < nsteps; ++k) {
                LBM_CK(c, cudaGraphLaunch(c->graph[c->cur], c->stream));
                c->cur = 1 - c->cur;
                ++c->t;
                if (forced) ++c->draws_head;
            }
            break;
        }
        const double* row = forced ? c->d_draws + c->draws_head * kDrawRow : nullptr;
        lbm_status st = enqueue_step(c, c->cur, c->stream, row, false);
        if (st) return st;
        if (forced) {
            ++c->draws_head;
            if (c->rec_k > 0) {  // keep this step's force for the reverse sweep
                const long long t = c->rec_steps;
                if (static_cast<size_t>(t / kFhatBlock) >= c->rec_fhat.size()) {
                    double* p = nullptr;
                    LBM_CK(c, pool_alloc(c, reinterpret_cast<void**>(&p), sizeof(double) * kFhatDoubles * kFhatBlock,
                                         c->stream));
                    c->rec_fhat.push_back(p);
                }
                LBM_CK(c, cudaMemcpyAsync(rec_fhat_at(c, t), c->d_fhat, sizeof(double) * kFhatDoubles,
                                          cudaMemcpyDeviceToDevice, c->stream));
            }
        }
        c->cur = 1 - c->cur;
        ++c->t;
        if (c->rec_k > 0 && (++c->rec_steps) % c->rec_k == 0) {
            const size_t bytes = static_cast<size_t>(c->d.ncell) * Q * c->elem;
            void* p = nullptr;
            LBM_CK(c, pool_alloc(c, &p, bytes, c->stream));
            c->ckpts.push_back(p);
            LBM_CK(c, cudaMemcpyAsync(p, c->buf[c->cur], bytes, cudaMemcpyDeviceToDevice, c->stream));
        }
    }
    return LBM_OK;
}

// The four guard regions: before and after each population buffer.
static void guard_regions(const lbm_ctx* c, const unsigned char* r[4]) {
    const size_t state_bytes = static_cast<size_t>(c->d.ncell) * Q * c->elem;
    for (int p = 0; p < 2; ++p) {
        const unsigned char* base = static_cast<const unsigned char*>(c->buf_base[p]);
        r[2 * p] = base;
        r[2 * p + 1] = base + kGuardBytes + state_bytes;
    }
}

lbm_status lbm_check_guards(lbm_ctx* c) {
    if (!c) return LBM_ERR_ARG;
    DeviceGuard guard(c->device);
    const unsigned char* r[4];
    guard_regions(c, r);
    int* d_bad = nullptr;
    LBM_CK(c, pool_alloc(c, reinterpret_cast<void**>(&d_bad), 4 * sizeof(int), c->stream));
    int bad[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemsetAsync(d_bad, 0, sizeof(bad), c->stream);
    if (e == cudaSuccess) e = launch_guard_check(r, d_bad, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, c->stream);
    cudaFreeAsync(d_bad, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_check_guards");
    static const char* names[4] = {"before buffer 0", "after buffer 0", "before buffer 1", "after buffer 1"};
    for (int k = 0; k < 4; ++k)
        if (bad[k])
            return fail(c, LBM_ERR_STATE, std::string("lbm_check_guards: guard region ") + names[k] + ": " +
                                              std::to_string(bad[k]) + " bytes changed (an out-of-bounds write)");
    return LBM_OK;
}

lbm_status lbm_selftest_guards(lbm_ctx* c) {
    if (!c) return LBM_ERR_ARG;
    DeviceGuard guard(c->device);
    const unsigned char* r[4];
    guard_regions(c, r);
    unsigned char* probe = const_cast<unsigned char*>(r[3]) + kGuardBytes / 2;  // inside the last region
    LBM_CK(c, cudaMemsetAsync(probe, static_cast<unsigned char>(~kGuardPattern), 1, c->stream));
    const lbm_status seen = lbm_check_guards(c);
    LBM_CK(c, cudaMemsetAsync(probe, kGuardPattern, 1, c->stream));
    const lbm_status clean = lbm_check_guards(c);
    if (seen != LBM_ERR_STATE) return fail(c, LBM_ERR_STATE, "lbm_selftest_guards: a changed guard byte went unseen");
    if (clean != LBM_OK) return clean;
    return LBM_OK;
}

lbm_status lbm_set_wait_limit(lbm_ctx* c, long long cycles) {
    if (!c) return LBM_ERR_ARG;
    if (cycles < 0) return fail(c, LBM_ERR_ARG, "lbm_set_wait_limit: cycles must be >= 0");
    c->wait_cycles = cycles;
    drop_step_graphs(c);  // the captured steps hold the old limit
    return LBM_OK;
}

lbm_status lbm_record_begin(lbm_ctx* c, int k) {
    if (!c) return LBM_ERR_ARG;
    DeviceGuard guard(c->device);
    if (k < 1) return fail(c, LBM_ERR_ARG, "lbm_record_begin: k must be >= 1");
    if (c->cfg.op != LBM_OP_NCO || c->cfg.net_precision != LBM_NET_F32 || c->cfg.storage != LBM_STORE_F32)
        return fail(c, LBM_ERR_ARG, "lbm_record_begin: the adjoint covers NCO with FP32 storage and network");
    free_recording(c);
    c->rec_k = k;
    const size_t bytes = static_cast<size_t>(c->d.ncell) * Q * c->elem;
    void* p = nullptr;
    LBM_CK(c, pool_alloc(c, &p, bytes, c->stream));
    c->ckpts.push_back(p);
    LBM_CK(c, cudaMemcpyAsync(p, c->buf[c->cur], bytes, cudaMemcpyDeviceToDevice, c->stream));
    return LBM_OK;
}

}  // extern "C"

// The reverse sweep shared by nco_backward and nco_backward_ke. kscale[t] (t = 0..T) is
// (dL/dk_t) / cells for the kinetic-energy observations, empty without any.
static lbm_status backward_sweep(lbm_ctx* c, const char* who, const float* dL_du, const float* dL_drho,
                                 const std::vector<double>& kscale, float* dL_dtheta, float* dL_df0) {
    DeviceGuard guard(c->device);
    const std::string w(who);
    if (c->rec_k < 1 || c->ckpts.empty()) return fail(c, LBM_ERR_STATE, w + ": call lbm_record_begin before stepping");
    if (!c->have_weights) return fail(c, LBM_ERR_STATE, w + ": no network weights");
    const bool deep = c->net->deep != 0;
    const bool forced = c->cfg.forcing == 1;
    const size_t n = static_cast<size_t>(c->d.ncell);
    const size_t bytes = n * Q * c->elem;
    const int k = c->rec_k;
    const long long T = c->rec_steps;
    auto scale_at = [&](long long t) { return kscale.empty() ? 0.0f : static_cast<float>(kscale[static_cast<size_t>(t)]); };
    // work buffers, kept for the next call
    while (c->adj_work.size() < static_cast<size_t>(k)) {
        void* p = nullptr;
        LBM_CK(c, pool_alloc(c, &p, bytes, c->stream));
        c->adj_work.push_back(p);
    }
    for (float*& p : c->adj_lam)
        if (!p) LBM_CK(c, pool_alloc(c, reinterpret_cast<void**>(&p), n * Q * sizeof(float), c->stream));
    const int glen = adjoint_grad_len(deep);
    if (c->adj_grad_len < glen) {
        if (c->adj_grad) cudaFreeAsync(c->adj_grad, c->stream);
        c->adj_grad = nullptr;
        c->adj_grad_len = 0;
        LBM_CK(c, pool_alloc(c, reinterpret_cast<void**>(&c->adj_grad), sizeof(double) * glen, c->stream));
        c->adj_grad_len = glen;
    }
    LBM_CK(c, cudaMemsetAsync(c->adj_grad, 0, sizeof(double) * glen, c->stream));
    // incoming cotangents (host or device)
    const bool hu = dL_du && !is_device_ptr(dL_du), hr = dL_drho && !is_device_ptr(dL_drho);
    if (hu || hr) {
        lbm_status st = ensure_stage(c, 4 * n);
        if (st) return st;
    }
    const float *du = dL_du, *dr = dL_drho;
    if (hu) {
        LBM_CK(c, cudaMemcpyAsync(c->d_stage, dL_du, 3 * n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        du = c->d_stage;
    }
    if (hr) {
        LBM_CK(c, cudaMemcpyAsync(c->d_stage + 3 * n, dL_drho, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        dr = c->d_stage + 3 * n;
    }
    int li = 0;  // adj_lam[li] holds lam_{t+1}
    LBM_CK(c, launch_adjoint_seed(c->d, c->cfg.storage, c->cfg.boundary, c->buf[c->cur], du, dr, scale_at(T), false,
                                  c->adj_lam[li], c->stream));
    const long long nseg = (T + k - 1) / k;
    for (long long sgi = nseg - 1; sgi >= 0; --sgi) {
        const long long a0 = sgi * k, b0 = std::min<long long>(a0 + k, T);
        // restore the checkpoint of step a0 and recompute the states of the segment
        LBM_CK(c, cudaMemcpyAsync(c->adj_work[0], c->ckpts[static_cast<size_t>(sgi)], bytes, cudaMemcpyDeviceToDevice,
                                  c->stream));
        for (long long t = a0; t < b0 - 1; ++t) {
            StepArgs a{};
            a.d = c->d;
            a.src = c->adj_work[static_cast<size_t>(t - a0)];
            a.dst = c->adj_work[static_cast<size_t>(t - a0 + 1)];
            a.status = c->d_status;
            a.tau = c->tau;
            a.rho_min = static_cast<float>(c->cfg.rho_min);
            a.rho_max = static_cast<float>(c->cfg.rho_max);
            // the recorded force of step t (the forward's projection is not needed again)
            const FusedForce ff{forced ? rec_fhat_at(c, t) : nullptr, c->d_ftab, nullptr, c->fscale};
            LBM_CK(c, launch_step(a, forced ? &ff : nullptr, c->cfg.op, c->cfg.storage, c->cfg.boundary,
                                  c->cfg.net_precision, c->net, c->tc_w, c->tc_shape, c->wait_cycles, c->stream));
        }
        for (long long t = b0 - 1; t >= a0; --t) {
            void* state_t = c->adj_work[static_cast<size_t>(t - a0)];
            if (forced) LBM_CK(c, launch_force_synth(c->d, rec_fhat_at(c, t), c->d_ftab, c->d_force, c->stream));
            LBM_CK(c, launch_adjoint_step(c->d, c->cfg.storage, c->cfg.boundary, state_t, c->adj_lam[li],
                                          c->adj_lam[1 - li], c->adj_grad, c->tau, forced ? c->d_force : nullptr,
                                          *c->net, c->stream));
            li = 1 - li;
            const float ks = scale_at(t);
            if (ks != 0.0f)
                LBM_CK(c, launch_adjoint_seed(c->d, c->cfg.storage, c->cfg.boundary, state_t, nullptr, nullptr, ks, true,
                                              c->adj_lam[li], c->stream));
        }
    }
    if (dL_dtheta) {
        const int nth = deep ? kNumThetaDeep : kNumTheta;
        std::vector<double> acc(glen);
        std::vector<float> out(nth);
        LBM_CK(c, cudaMemcpyAsync(acc.data(), c->adj_grad, sizeof(double) * glen, cudaMemcpyDeviceToHost, c->stream));
        LBM_CK(c, cudaStreamSynchronize(c->stream));
        adjoint_fold_gradient(acc.data(), deep, out.data());
        if (is_device_ptr(dL_dtheta)) {
            LBM_CK(c, cudaMemcpyAsync(dL_dtheta, out.data(), sizeof(float) * nth, cudaMemcpyHostToDevice, c->stream));
            LBM_CK(c, cudaStreamSynchronize(c->stream));
        } else {
            std::memcpy(dL_dtheta, out.data(), sizeof(float) * nth);
        }
    }
    if (dL_df0) {
        LBM_CK(c, cudaMemcpyAsync(dL_df0, c->adj_lam[li], n * Q * sizeof(float), cudaMemcpyDefault, c->stream));
    }
    LBM_CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

extern "C" {

lbm_status nco_backward(lbm_ctx* c, const float* dL_du, const float* dL_drho, float* dL_dtheta, float* dL_df0) {
    if (!c) return LBM_ERR_ARG;
    if (!dL_du && !dL_drho) return fail(c, LBM_ERR_ARG, "nco_backward: dL_du or dL_drho is required");
    return backward_sweep(c, "nco_backward", dL_du, dL_drho, {}, dL_dtheta, dL_df0);
}

lbm_status nco_backward_ke(lbm_ctx* c, int nobs, const int* obs_step, const double* dL_dk, const float* dL_du,
                           const float* dL_drho, float* dL_dtheta, float* dL_df0) {
    if (!c) return LBM_ERR_ARG;
    if (nobs < 0 || (nobs > 0 && (!obs_step || !dL_dk)))
        return fail(c, LBM_ERR_ARG, "nco_backward_ke: nobs >= 0 steps and cotangents required");
    if (nobs == 0 && !dL_du && !dL_drho)
        return fail(c, LBM_ERR_ARG, "nco_backward_ke: no observation and no field cotangent");
    const long long T = c->rec_steps;
    std::vector<double> kscale(static_cast<size_t>(T) + 1, 0.0);
    for (int j = 0; j < nobs; ++j) {
        if (obs_step[j] < 0 || obs_step[j] > T)
            return fail(c, LBM_ERR_ARG, "nco_backward_ke: observation step outside [0, steps recorded]");
        if (!std::isfinite(dL_dk[j])) return fail(c, LBM_ERR_ARG, "nco_backward_ke: non-finite dL/dk");
        kscale[static_cast<size_t>(obs_step[j])] += dL_dk[j] / static_cast<double>(c->d.ncell);
    }
    return backward_sweep(c, "nco_backward_ke", dL_du, dL_drho, kscale, dL_dtheta, dL_df0);
}

lbm_status lbm_check(lbm_ctx* c) {
    if (!c) return LBM_ERR_ARG;
    DeviceGuard guard(c->device);
    int h = 0;
    LBM_CK(c, cudaMemcpyAsync(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LBM_CK(c, cudaStreamSynchronize(c->stream));
    if (h & 4)
        return fail(c, LBM_ERR_TIMEOUT, "tensor-core MMAs still ran after a timed-out wait and its drain; "
                                        "their tensor memory was left allocated");
    if (h & 2) return fail(c, LBM_ERR_TIMEOUT, "a tensor-core completion wait ran out (kernel stopped early)");
    if (h & 1) return fail(c, LBM_ERR_UNSTABLE, "non-finite value or density outside [rho_min, rho_max]");
    return LBM_OK;
}

lbm_status lbm_macroscopic(lbm_ctx* c, float* rho, float* u) {
    if (!c) return LBM_ERR_ARG;
    DeviceGuard guard(c->device);
    const size_t n = static_cast<size_t>(c->d.ncell);
    const bool hr = rho && !is_device_ptr(rho), hu = u && !is_device_ptr(u);
    if (hr || hu) {
        lbm_status st = ensure_stage(c, 4 * n);
        if (st) return st;
    }
    float* dr = hr ? c->d_stage : rho;
    float* du = hu ? c->d_stage + n : u;
    LBM_CK(c, launch_macroscopic(c->d, c->cfg.storage, c->cfg.boundary, c->buf[c->cur], dr, du, c->stream));
    if (hr) LBM_CK(c, cudaMemcpyAsync(rho, dr, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    if (hu) LBM_CK(c, cudaMemcpyAsync(u, du, 3 * n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    if (hr || hu) LBM_CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status lbm_kinetic_energy(lbm_ctx* c, double* ke) {
    if (!c) return LBM_ERR_ARG;
    DeviceGuard guard(c->device);
    if (!ke) return fail(c, LBM_ERR_ARG, "lbm_kinetic_energy: ke is required");
    const bool dev = is_device_ptr(ke);
    double* out = dev ? ke : c->d_scalar;
    LBM_CK(c, launch_kinetic_energy(c->d, c->cfg.storage, c->cfg.boundary, c->buf[c->cur], c->d_partials, c->npart,
                                    out, c->stream));
    if (!dev) {
        LBM_CK(c, cudaMemcpyAsync(ke, out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        LBM_CK(c, cudaStreamSynchronize(c->stream));
    }
    return LBM_OK;
}

lbm_status lbm_energy_spectrum(lbm_ctx* c, double* E, int nbins, double* ke) {
    if (!c) return LBM_ERR_ARG;
    DeviceGuard guard(c->device);
    if (!E || nbins < 1) return fail(c, LBM_ERR_ARG, "lbm_energy_spectrum: E and nbins >= 1 are required");
    if (c->cfg.boundary == LBM_BC_TGV_REDUCED)
        return fail(c, LBM_ERR_ARG, "lbm_energy_spectrum: not available on the reduced Taylor-Green domain");
    const int mul = c->cfg.boundary == LBM_BC_MIRROR ? 2 : 1;
    if (!fft_size_ok(mul * c->d.nx) || !fft_size_ok(mul * c->d.ny) || !fft_size_ok(mul * c->d.nz))
        return fail(c, LBM_ERR_ARG, "lbm_energy_spectrum: sizes must be 2^a or 3*2^a (a >= 0)");
    const size_t need = spectrum_work_elems(c->d, c->cfg.boundary);
    if (c->fft_elems < need) {
        if (c->d_fft) cudaFree(c->d_fft);
        c->d_fft = nullptr;
        c->fft_elems = 0;
        LBM_CK(c, cudaMalloc(&c->d_fft, need * sizeof(float2)));
        c->fft_elems = need;
    }
    if (c->E_cap < nbins) {
        if (c->d_E) cudaFree(c->d_E);
        c->d_E = nullptr;
        c->E_cap = 0;
        LBM_CK(c, cudaMalloc(&c->d_E, sizeof(double) * nbins));
        c->E_cap = nbins;
    }
    const bool dev = is_device_ptr(E);
    const bool kdev = ke && is_device_ptr(ke);
    double* dE = dev ? E : c->d_E;
    double* dke = ke ? (kdev ? ke : c->d_scalar) : nullptr;
    LBM_CK(c, launch_spectrum(c->d, c->cfg.storage, c->cfg.boundary, c->buf[c->cur], c->d_fft, dE, nbins, dke,
                              c->stream));
    if (!dev) LBM_CK(c, cudaMemcpyAsync(E, dE, sizeof(double) * nbins, cudaMemcpyDeviceToHost, c->stream));
    if (ke && !kdev) LBM_CK(c, cudaMemcpyAsync(ke, dke, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (!dev || (ke && !kdev)) LBM_CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// Batches: independent NCO instances of uneven size stepped by one persistent launch.
// ---------------------------------------------------------------------------
}  // extern "C"

struct lbm_batch {
    std::vector<lbm_ctx*> ctx;
    cudaStream_t stream = nullptr;
    int storage = 0;
    int shape = 0;                     // tile shape of the batched kernel (autotuned; see lbm.h)
    StepArgs* d_inst = nullptr;        // two descriptor sets: [0] current buffers, [1] swapped
    long long* d_tile_begin = nullptr;
    int* d_tile_inst = nullptr;        // instance of every global tile
    long long ntiles = 0;
    ForceBatchItem* d_fitems = nullptr;  // the forced instances' forcing descriptors
    int nforced = 0;
    int max_proj_blocks = 0;
    long long max_forced_cells = 0;
    int* d_status = nullptr;
    long long* d_counter = nullptr;    // steps replayed since the graphs were captured
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // one step from descriptor set 0 / 1
    int graph_shape = -1;              // tile shape the graphs were captured with
    std::vector<long long> desc_sig;   // instance buffers and draw queues the descriptors hold
    long long steps_since_upload = 0;  // the device step counter
    int phase = 0;                     // descriptor set of the next step
    bool have_weights = false;
    bool own_stream = false;
    std::string err;
};

namespace {

lbm_status bfail(lbm_batch* b, lbm_status code, const std::string& m) {
    if (b) b->err = m;
    return code;
}

#define LBM_BCK(b, call)                                                                   \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,  \
                         std::string(#call) + ": " + cudaGetErrorString(e_));              \
    } while (0)

StepArgs instance_args(const lbm_ctx* c, int parity) {
    StepArgs a{};
    a.d = c->d;
    const int cur = parity ? 1 - c->cur : c->cur;
    a.src = c->buf[cur];
    a.dst = c->buf[1 - cur];
    a.force = c->cfg.forcing ? c->d_force : nullptr;
    a.u_out = c->cfg.forcing ? c->d_u : nullptr;
    a.status = c->d_status;
    a.tau = c->tau;
    a.rho_min = static_cast<float>(c->cfg.rho_min);
    a.rho_max = static_cast<float>(c->cfg.rho_max);
    return a;
}

// What the device descriptors depend on. The draw head enters as head - steps since the
// upload, which batch steps leave unchanged and a direct lbm_step of an instance moves.
std::vector<long long> batch_signature(const lbm_batch* b) {
    std::vector<long long> sig;
    for (const lbm_ctx* c : b->ctx) {
        sig.push_back(reinterpret_cast<long long>(c->buf[c->cur]));
        sig.push_back(reinterpret_cast<long long>(c->d_draws));
        sig.push_back(c->draws_cap);
        sig.push_back(c->draws_head - b->steps_since_upload);
    }
    return sig;
}

lbm_status upload_descriptors(lbm_batch* b) {
    const size_t n = b->ctx.size();
    std::vector<StepArgs> h(2 * n);
    for (size_t i = 0; i < n; ++i) {
        h[i] = instance_args(b->ctx[i], 0);
        h[n + i] = instance_args(b->ctx[i], 1);
    }
    LBM_BCK(b, cudaMemcpyAsync(b->d_inst, h.data(), sizeof(StepArgs) * 2 * n, cudaMemcpyHostToDevice, b->stream));
    std::vector<ForceBatchItem> fi;
    for (lbm_ctx* c : b->ctx) {
        if (!c->cfg.forcing) continue;
        ForceBatchItem it{};
        it.d = c->d;
        it.u = c->d_u;
        it.force = c->d_force;
        it.proj = c->d_fproj;
        it.scale = c->fscale;
        it.unit = c->funit;
        it.draws = c->d_draws;
        it.head = c->draws_head;
        it.rows = c->draws_cap;
        it.consts = c->d_fconst;
        it.tab = c->d_ftab;
        it.fhat = c->d_fhat;
        fi.push_back(it);
    }
    if (!fi.empty())
        LBM_BCK(b, cudaMemcpyAsync(b->d_fitems, fi.data(), sizeof(ForceBatchItem) * fi.size(), cudaMemcpyHostToDevice,
                                   b->stream));
    LBM_BCK(b, cudaMemsetAsync(b->d_counter, 0, sizeof(long long), b->stream));
    LBM_BCK(b, cudaStreamSynchronize(b->stream));
    b->phase = 0;
    b->steps_since_upload = 0;
    b->desc_sig = batch_signature(b);
    return LBM_OK;
}

// Enqueue one batch step with descriptor set `phase`: the forcing coefficients and force
// fields of every forced instance (draw row = its head + the device step counter), the
// persistent step kernel over all tiles, the forcing projections, the counter increment.
lbm_status enqueue_batch_step(lbm_batch* b, int phase) {
    const size_t n = b->ctx.size();
    LBM_BCK(b, launch_force_batch(b->d_fitems, b->nforced, b->max_proj_blocks, b->max_forced_cells, b->d_counter, 0,
                                  b->stream));
    LBM_BCK(b, launch_step_nco_tc_batch(b->d_inst + phase * n, b->d_tile_begin, b->d_tile_inst, static_cast<int>(n),
                                        b->ntiles, b->storage, b->shape, b->d_status, b->ctx[0]->tc_w, b->stream));
    LBM_BCK(b, launch_force_batch(b->d_fitems, b->nforced, b->max_proj_blocks, b->max_forced_cells, b->d_counter, 1,
                                  b->stream));
    if (b->nforced > 0) LBM_BCK(b, launch_counter_increment(b->d_counter, b->stream));
    return LBM_OK;
}

void advance_host_state(lbm_batch* b, int nsteps) {
    for (lbm_ctx* c : b->ctx) {
        if (nsteps & 1) c->cur = 1 - c->cur;
        c->t += nsteps;
        if (c->cfg.forcing) c->draws_head += nsteps;
    }
    b->steps_since_upload += nsteps;
    b->phase ^= nsteps & 1;
}

void destroy_graphs(lbm_batch* b) {
    for (cudaGraphExec_t& g : b->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

}  // namespace

extern "C" {

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : kNoCtxError; }

lbm_status lbm_batch_destroy(lbm_batch* b) {
    if (!b) return LBM_OK;
    destroy_graphs(b);
    for (lbm_ctx* c : b->ctx) lbm_destroy(c);
    void* devs[] = {b->d_inst, b->d_tile_begin, b->d_tile_inst, b->d_fitems, b->d_status, b->d_counter};
    for (void* p : devs)
        if (p) cudaFree(p);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return LBM_OK;
}

lbm_status lbm_batch_create(int n, const lbm_config* cfgs, void* stream, lbm_batch** out) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (n < 1 || !cfgs) return LBM_ERR_ARG;
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ERR_OOM;
    b->stream = static_cast<cudaStream_t>(stream);
    if (!b->stream) {  // graphs cannot be captured on the legacy default stream
        if (cudaStreamCreate(&b->stream) != cudaSuccess) {
            delete b;
            return LBM_ERR_CUDA;
        }
        b->own_stream = true;
    }
    b->storage = cfgs[0].storage;
    for (int i = 0; i < n; ++i) {
        const lbm_config& c = cfgs[i];
        if (c.op != LBM_OP_NCO || c.net_precision != LBM_NET_BF16 || c.boundary != LBM_BC_PERIODIC ||
            c.storage != b->storage) {
            std::fprintf(stderr, "lbm_batch_create: instance %d must be NCO, BF16 network, periodic, common storage\n", i);
            lbm_batch_destroy(b);
            return LBM_ERR_ARG;
        }
        lbm_ctx* ctx = nullptr;
        const lbm_status st = lbm_create(&c, b->stream, &ctx);
        if (st != LBM_OK) {
            lbm_batch_destroy(b);
            return st;
        }
        b->ctx.push_back(ctx);
    }
    std::vector<long long> tb(n + 1, 0);
    for (int i = 0; i < n; ++i) tb[i + 1] = tb[i] + (b->ctx[i]->d.ncell + 127) / 128;
    b->ntiles = tb[n];
    std::vector<int> ti(static_cast<size_t>(b->ntiles));
    for (int i = 0; i < n; ++i)
        for (long long t = tb[i]; t < tb[i + 1]; ++t) ti[static_cast<size_t>(t)] = i;
    for (lbm_ctx* c : b->ctx)
        if (c->cfg.forcing) {
            ++b->nforced;
            b->max_proj_blocks = std::max(b->max_proj_blocks, c->fblocks);
            b->max_forced_cells = std::max(b->max_forced_cells, c->d.ncell);
        }
    auto alloc = [&](void** p, size_t bytes) { return cudaMalloc(p, bytes); };
    if (alloc(reinterpret_cast<void**>(&b->d_inst), sizeof(StepArgs) * 2 * n) != cudaSuccess ||
        alloc(reinterpret_cast<void**>(&b->d_tile_begin), sizeof(long long) * (n + 1)) != cudaSuccess ||
        alloc(reinterpret_cast<void**>(&b->d_tile_inst), sizeof(int) * ti.size()) != cudaSuccess ||
        alloc(reinterpret_cast<void**>(&b->d_fitems), sizeof(ForceBatchItem) * std::max(1, b->nforced)) != cudaSuccess ||
        alloc(reinterpret_cast<void**>(&b->d_status), sizeof(int)) != cudaSuccess ||
        alloc(reinterpret_cast<void**>(&b->d_counter), sizeof(long long)) != cudaSuccess) {
        lbm_batch_destroy(b);
        return LBM_ERR_OOM;
    }
    if (cudaMemcpy(b->d_tile_begin, tb.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_tile_inst, ti.data(), sizeof(int) * ti.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->d_status, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(b->d_counter, 0, sizeof(long long)) != cudaSuccess) {
        lbm_batch_destroy(b);
        return LBM_ERR_CUDA;
    }
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_get(lbm_batch* b, int i, lbm_ctx** out) {
    if (!b || !out || i < 0 || i >= static_cast<int>(b->ctx.size())) return LBM_ERR_ARG;
    *out = b->ctx[i];
    return LBM_OK;
}

lbm_status lbm_batch_set_weights(lbm_batch* b, const float* theta, int n) {
    if (!b) return LBM_ERR_ARG;
    if (n != kNumTheta) return bfail(b, LBM_ERR_ARG, "lbm_batch_set_weights: batches take the 1064-parameter network");
    for (lbm_ctx* c : b->ctx) {
        const lbm_status st = nco_set_weights(c, theta, n);
        if (st != LBM_OK) return bfail(b, st, c->err);
    }
    b->have_weights = true;
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int nsteps, int use_graph) {
    if (!b) return LBM_ERR_ARG;
    if (nsteps < 0) return bfail(b, LBM_ERR_ARG, "lbm_batch_step: nsteps < 0");
    if (!b->have_weights) return bfail(b, LBM_ERR_STATE, "lbm_batch_step: call lbm_batch_set_weights first");
    for (lbm_ctx* c : b->ctx)
        if (c->cfg.forcing && c->draws_tail - c->draws_head < nsteps)
            return bfail(b, LBM_ERR_STATE, "lbm_batch_step: a forced instance has too few random draws queued");
    if (nsteps == 0) return LBM_OK;
    // the batch's own kernels must not run while earlier work of the instances is pending
    LBM_BCK(b, cudaStreamSynchronize(b->stream));
    lbm_status st;
    if (use_graph && (!b->graph[0] || b->graph_shape != b->shape)) {
        // capture one step per descriptor set; the kernels read the descriptors and the
        // step counter from device memory, so the graphs outlive re-uploads
        destroy_graphs(b);
        LBM_BCK(b, launch_step_nco_tc_batch(b->d_inst, b->d_tile_begin, b->d_tile_inst, static_cast<int>(b->ctx.size()),
                                            0, b->storage, b->shape, b->d_status, b->ctx[0]->tc_w,
                                            b->stream));  // sets the kernel attributes, no work
        for (int p = 0; p < 2; ++p) {
            cudaGraph_t g = nullptr;
            LBM_BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            st = enqueue_batch_step(b, p);
            cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
            if (st) return st;
            if (ce != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
            ce = cudaGraphInstantiate(&b->graph[p], g, 0);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
        }
        b->graph_shape = b->shape;
    }
    if (b->desc_sig.empty() || batch_signature(b) != b->desc_sig) {
        st = upload_descriptors(b);  // buffers or draw queues changed outside the batch
        if (st) return st;
    }
    for (int k = 0; k < nsteps; ++k) {
        const int p = b->phase ^ (k & 1);
        if (use_graph) LBM_BCK(b, cudaGraphLaunch(b->graph[p], b->stream));
        else if ((st = enqueue_batch_step(b, p))) return st;
    }
    advance_host_state(b, nsteps);
    b->desc_sig = batch_signature(b);
    return LBM_OK;
}

// The tile shape of a batch applies to its instances too, so that an instance stepped alone
// with lbm_step follows the same per-tile arithmetic as in the batch.
static void apply_shape(lbm_batch* b, int shape) {
    if (shape != b->shape) destroy_graphs(b);
    b->shape = shape;
    for (lbm_ctx* c : b->ctx) {
        if (c->tc_shape != shape) drop_step_graphs(c);
        c->tc_shape = shape;
    }
}

lbm_status lbm_batch_set_tile_shape(lbm_batch* b, int shape) {
    if (!b) return LBM_ERR_ARG;
    if (shape != 0 && (shape < 2 || shape > 4)) return bfail(b, LBM_ERR_ARG, "lbm_batch_set_tile_shape: shape 0, 2, 3 or 4");
    apply_shape(b, shape);
    return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch* b, int* choice) {
    if (!b) return LBM_ERR_ARG;
    if (!b->have_weights) return bfail(b, LBM_ERR_STATE, "lbm_batch_autotune: call lbm_batch_set_weights first");
    lbm_status st = upload_descriptors(b);
    if (st) return st;
    const int cands[4] = {0, 2, 3, 4};  // pairs across two warpgroups; chunks of four with 2, 3, 4 warpgroups
    float best = 1e30f;
    int best_shape = 0;
    cudaEvent_t e0, e1;
    LBM_BCK(b, cudaEventCreate(&e0));
    LBM_BCK(b, cudaEventCreate(&e1));
    for (int shape : cands) {
        // the step kernel alone, reading the current buffers and writing the spare ones:
        // the state does not advance
        for (int rep = 0; rep < 2; ++rep)
            LBM_BCK(b, launch_step_nco_tc_batch(b->d_inst, b->d_tile_begin, b->d_tile_inst, static_cast<int>(b->ctx.size()),
                                                b->ntiles, b->storage, shape, b->d_status, b->ctx[0]->tc_w, b->stream));
        LBM_BCK(b, cudaEventRecord(e0, b->stream));
        for (int rep = 0; rep < 3; ++rep)
            LBM_BCK(b, launch_step_nco_tc_batch(b->d_inst, b->d_tile_begin, b->d_tile_inst, static_cast<int>(b->ctx.size()),
                                                b->ntiles, b->storage, shape, b->d_status, b->ctx[0]->tc_w, b->stream));
        LBM_BCK(b, cudaEventRecord(e1, b->stream));
        LBM_BCK(b, cudaEventSynchronize(e1));
        float ms = 0.0f;
        LBM_BCK(b, cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
            best = ms;
            best_shape = shape;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    apply_shape(b, best_shape);
    if (choice) *choice = best_shape;
    return LBM_OK;
}

lbm_status lbm_batch_check(lbm_batch* b) {
    if (!b) return LBM_ERR_ARG;
    int h = 0;
    LBM_BCK(b, cudaMemcpyAsync(&h, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    LBM_BCK(b, cudaStreamSynchronize(b->stream));
    if (h & 2) return bfail(b, LBM_ERR_TIMEOUT, "a tensor-core completion wait ran out");
    for (lbm_ctx* c : b->ctx) {
        const lbm_status st = lbm_check(c);
        if (st != LBM_OK) return bfail(b, st, c->err);
    }
    return LBM_OK;
}

}  // extern "C"
