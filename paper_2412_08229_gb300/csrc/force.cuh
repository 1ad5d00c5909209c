// force.cuh - per-cell pieces of the Alvelius spectral forcing (Sec. II.C) shared by the
// forcing kernels and the forced step kernels: the phases e^{i k.x} of the 16 forced modes
// from per-axis tables, the force F(x) = sum_m 2 Re(F^_m e^{i k_m.x}) and the projection
// u^(k) = N^-3 sum_x u(x) e^{-i k.x} of the step's velocity.
//
// Every product and sum here is written with an explicit rounding (fmaf, __fmul_rn,
// __fadd_rn), so that the compiler cannot contract it differently in different kernels:
// the force a step kernel synthesises is bit-identical to the stored field of
// force_synth, and a projection formed inside a step kernel is bit-identical to one
// formed by force_project.
//
// Projection: each warp sums its 32 cells' values (the 32 cells are always an aligned run
// of consecutive cells) with a fixed butterfly, rounds the warp sums to fixed point (the
// scale 2^S of force_proj_scale) and adds them as 64-bit integers. Integer sums do not
// depend on the order of addition, so the result is the same whatever grid, kernel or
// interleaving of warps produced it. Value q = 32 a + 2 m + c holds axis a, mode m and
// c = 0: Re, 1: Im of u_a e^{-i k_m.x}.
#pragma once

#include "cell.cuh"

namespace lbm {

// The forced modes, sorted by (|k|^2, kz, ky, kx): every integer k in the half space
// (kz > 0, or kz = 0 and ky > 0, or kz = ky = 0 and kx > 0) with 1 <= |k|^2 <= 4.
struct ModeTable {
    int k[kForcedModes][3];
};

constexpr ModeTable make_mode_table() {
    ModeTable m{};
    int n = 0;
    for (int k2 = 1; k2 <= 4; ++k2)
        for (int kz = -2; kz <= 2; ++kz)
            for (int ky = -2; ky <= 2; ++ky)
                for (int kx = -2; kx <= 2; ++kx) {
                    if (kx * kx + ky * ky + kz * kz != k2) continue;
                    const bool half = kz > 0 || (kz == 0 && ky > 0) || (kz == 0 && ky == 0 && kx > 0);
                    if (!half || n >= kForcedModes) continue;
                    m.k[n][0] = kx;
                    m.k[n][1] = ky;
                    m.k[n][2] = kz;
                    ++n;
                }
    return m;
}

constexpr ModeTable kModeTable = make_mode_table();

namespace frc {

constexpr int kProjValues = 3 * 2 * kForcedModes;  // 96

struct Cx {
    float re, im;
};

__device__ __forceinline__ Cx cmul(Cx a, Cx b) {
    return {__fsub_rn(__fmul_rn(a.re, b.re), __fmul_rn(a.im, b.im)),
            __fadd_rn(__fmul_rn(a.re, b.im), __fmul_rn(a.im, b.re))};
}

// exp(i K 2 pi j / n) from one axis's factors e1 = exp(i 2 pi j / n), e2 = exp(i 4 pi j / n)
template <int K>
__device__ __forceinline__ Cx axis_factor(const Cx& e1, const Cx& e2) {
    if constexpr (K == 1) return e1;
    else if constexpr (K == 2) return e2;
    else if constexpr (K == -1) return Cx{e1.re, -e1.im};
    else return Cx{e2.re, -e2.im};
}

// exp(i k_m . x) for mode M, x_j = 2 pi j / n per axis, as a product of per-axis factors
template <int M>
__device__ __forceinline__ Cx mode_phase(const Cx* ex, const Cx* ey, const Cx* ez) {
    constexpr int kx = kModeTable.k[M][0], ky = kModeTable.k[M][1], kz = kModeTable.k[M][2];
    Cx p{1.0f, 0.0f};
    bool first = true;
    if constexpr (kx != 0) {
        p = axis_factor<kx>(ex[0], ex[1]);
        first = false;
    }
    if constexpr (ky != 0) {
        const Cx f = axis_factor<ky>(ey[0], ey[1]);
        p = first ? f : cmul(p, f);
        first = false;
    }
    if constexpr (kz != 0) {
        const Cx f = axis_factor<kz>(ez[0], ez[1]);
        p = first ? f : cmul(p, f);
    }
    return p;
}

// The phases of all 16 modes at grid node (x, y, z); tab holds the tables of the x, y and
// z axes one after another (2 entries per node: k = 1, 2).
__device__ __forceinline__ void cell_phases(int x, int y, int z, const Dims& d, const float2* tab, Cx* p) {
    Cx ex[2], ey[2], ez[2];
    const float4 tx = __ldg(reinterpret_cast<const float4*>(tab) + x);
    const float4 ty = __ldg(reinterpret_cast<const float4*>(tab + 2 * d.nx) + y);
    const float4 tz = __ldg(reinterpret_cast<const float4*>(tab + 2 * (d.nx + d.ny)) + z);
    ex[0] = Cx{tx.x, tx.y};
    ex[1] = Cx{tx.z, tx.w};
    ey[0] = Cx{ty.x, ty.y};
    ey[1] = Cx{ty.z, ty.w};
    ez[0] = Cx{tz.x, tz.y};
    ez[1] = Cx{tz.z, tz.w};
    static_for<kForcedModes>([&](auto Mc) {
        constexpr int m = decltype(Mc)::value;
        p[m] = mode_phase<m>(ex, ey, ez);
    });
}

// fh2 = 2 F^ as floats, fh2[6 m + 2 a + c]; F_a = sum_m (2 Re F^ cos - 2 Im F^ sin) in mode order
__device__ __forceinline__ void synth_force(const float* fh2, const Cx* p, float* F) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float s = 0.0f;
#pragma unroll
        for (int m = 0; m < kForcedModes; ++m) {
            s = fmaf(fh2[m * 6 + 2 * a], p[m].re, s);
            s = fmaf(-fh2[m * 6 + 2 * a + 1], p[m].im, s);
        }
        F[a] = s;
    }
}

// Loads 2 F^ (FP64, fhat[6 m + 2 a + c]) into shared memory as floats; the caller syncs.
__device__ __forceinline__ void load_fh2(const double* fhat, float* fh2) {
    for (int i = threadIdx.x; i < 6 * kForcedModes; i += blockDim.x) fh2[i] = static_cast<float>(2.0 * fhat[i]);
}

// v[0..2H) of this lane -> v[0..H): lane bit H picks which half it keeps; the kept half
// gets the partner's copy of it added (partner = lane ^ H).
template <int H>
__device__ __forceinline__ void halve(float* v, int lane) {
    const bool hi = (lane & H) != 0;
#pragma unroll
    for (int i = 0; i < H; ++i) {
        const float keep = hi ? v[H + i] : v[i];
        const float send = hi ? v[i] : v[H + i];
        v[i] = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, H));
    }
}

// Value 2 m + c of axis a for one lane: c = 0: u_a Re p_m, c = 1: -u_a Im p_m.
__device__ __forceinline__ float proj_value(float ua, const Cx& p, int c) {
    return c == 0 ? __fmul_rn(ua, p.re) : __fmul_rn(-ua, p.im);
}

// The projection of one cell per lane (u = 0 for a lane without a cell), added to the
// lane's fixed-point accumulators: after the call lane l has added the warp's sum of
// value 32 a + l to acc[a]. All 32 lanes must call it together. Per axis the 32 values
// are summed over the warp by halving (offsets 16, 8, 4, 2, 1); the first halving is
// taken while the values are formed, so that only 16 of them are live at a time.
__device__ __forceinline__ void project_warp(float ux, float uy, float uz, const Cx* p, int lane, long long* acc,
                                             float scale) {
    const bool hi = (lane & 16) != 0;
#pragma unroll 1
    for (int a = 0; a < 3; ++a) {
        const float ua = a == 0 ? ux : (a == 1 ? uy : uz);
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {  // values i (modes 0..7) and 16 + i (modes 8..15)
            const float lo = proj_value(ua, p[i >> 1], i & 1);
            const float up = proj_value(ua, p[8 + (i >> 1)], i & 1);
            const float keep = hi ? up : lo;
            const float send = hi ? lo : up;
            v[i] = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, 16));
        }
        halve<8>(v, lane);
        halve<4>(v, lane);
        halve<2>(v, lane);
        halve<1>(v, lane);
        const float w = fminf(fmaxf(v[0], -32.0f), 32.0f);  // |u| < 1 in any stable state
        const long long iw = __float2ll_rn(w * scale);       // w * 2^S is exact
        if (a == 0) acc[0] += iw;
        else if (a == 1) acc[1] += iw;
        else acc[2] += iw;
    }
}

// A block's accumulators: every projecting lane adds its three values to red[96] (zeroed
// before), then after a barrier threads 0..95 add red to the context's sums.
__device__ __forceinline__ void proj_to_shared(unsigned long long* red, const long long* acc, int lane) {
#pragma unroll
    for (int a = 0; a < 3; ++a) atomicAdd(&red[32 * a + lane], static_cast<unsigned long long>(acc[a]));
}

__device__ __forceinline__ void proj_to_global(const unsigned long long* red, unsigned long long* proj) {
    for (int i = threadIdx.x; i < kProjValues; i += blockDim.x)
        if (red[i] != 0ull) atomicAdd(&proj[i], red[i]);
}

}  // namespace frc
}  // namespace lbm
