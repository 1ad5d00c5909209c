// tc_common.cuh - helpers shared by the tensor-core NCO kernels (kernels_nco_tc.cu,
// kernels_nco_tc3.cu): bounded mbarrier waits, warpgroup barriers, BF16 rounding on the
// host, packed FP32 adds and the relaxation back to populations.
#pragma once
#include <cstring>

#include "cell.cuh"
#include "tc_ptx.cuh"

namespace lbm {
namespace tcc {
using namespace tc;

constexpr uint32_t kBf16One = 0x3F80u;

// Tiles of a batch of instances: instance i owns global tiles [tile_begin[i], tile_begin[i+1]).
struct BatchTiles {
    const StepArgs* inst;          // device array, ninst entries
    const long long* tile_begin;   // device array, ninst + 1 entries
    const int* tile_inst;          // device array: the instance of every global tile
    int ninst;
};

// FP32 -> BF16 bits, round to nearest even (host-side weight packing)
inline uint16_t f2bf(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    const uint32_t r = 0x7FFFu + ((u >> 16) & 1u);
    return static_cast<uint16_t>((u + r) >> 16);
}

// Wait until the phase of `bar` with this parity has completed, for at most `limit` SM
// clock cycles (0: give up at once). Returns false when the limit runs out first.
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity, long long limit = kDefaultWaitCycles) {
    if (limit <= 0) return false;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// Barrier over one warpgroup that also ANDs a per-thread flag; the result is uniform.
__device__ __forceinline__ bool wg_sync_and(int id, bool ok) {
    uint32_t out;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.b32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(out)
        : "r"(static_cast<int>(ok)), "r"(id)
        : "memory");
    return out != 0;
}

__device__ __forceinline__ float as_f(uint32_t u) { return __uint_as_float(u); }


// f* from moments: m*_e = m_e - s_e (m_e - m^eq_e) (Sec. II.B, eq. omegatheta), then
// df* = M^-1 m* - w, with the zeroth moment carried as rho - 1 for precision.
__device__ __forceinline__ void relax_to_populations(const float* m, float drho, const Macro& q, float omega_nu,
                                                     const float* rates, float* df) {
#pragma unroll
    for (int e = 0; e < Q; ++e) {
        const int n = order_of(e);
        if (e == 0) df[e] = drho;
        else if (n == 1) df[e] = m[e];
        else if (n == 2) df[e] = m[e] - omega_nu * (m[e] - meq2(e, q));
        else df[e] = m[e] - rates[n - 3] * m[e];
    }
    populations_inplace(df);
}

// (a0, a1) += (relu(b0), relu(b1)) with one packed FP32 add
__device__ __forceinline__ void add2_relu(float& a0, float& a1, float b0, float b1) {
    b0 = fmaxf(b0, 0.0f);
    b1 = fmaxf(b1, 0.0f);
    asm("{\n\t.reg .b64 x, y;\n\tmov.b64 x, {%0, %1};\n\tmov.b64 y, {%2, %3};\n\t"
        "add.rn.f32x2 x, x, y;\n\tmov.b64 {%0, %1}, x;\n\t}"
        : "+f"(a0), "+f"(a1)
        : "f"(b0), "f"(b1));
}

}  // namespace tcc
}  // namespace lbm
