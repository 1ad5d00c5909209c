// cell.cuh - per-cell device building blocks shared by the step kernels:
// storage conversion, the pull map (periodic or mirror), moments, equilibrium,
// the MRT relaxation (Sec. II.B), BGK (Sec. II.A), KBC and the Kupershtokh source.
//
// Populations are carried as deviations df_i = f_i - w_i in every storage format, so
// rho - 1 and all non-equilibrium moments are formed from small numbers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"

namespace lbm {

template <int STORAGE> struct Store;
template <> struct Store<LBM_STORE_F32> {
    using T = float;
    static __device__ __forceinline__ float ld(const T* p) { return __ldg(p); }
    static __device__ __forceinline__ void st(T* p, float v) { *p = v; }
};
template <> struct Store<LBM_STORE_F16_DEV> {
    using T = __half;
    static __device__ __forceinline__ float ld(const T* p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void st(T* p, float v) { *p = __float2half_rn(v); }
};
template <> struct Store<LBM_STORE_BF16_DEV> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float ld(const T* p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ void st(T* p, float v) { *p = __float2bfloat16_rn(v); }
};

__device__ __forceinline__ float wgt(int i) { return static_cast<float>(weight(i)); }

// Pull map of the streaming step (Sec. II.A): population i of cell (x,y,z) at t+1 is
// population ip of cell `src` at t (post-collision). Periodic: src = x - c_i wrapped.
// Mirror (Appendix A, octant with nodes half a spacing from the planes): when x - c_i
// leaves the box along an axis, the source is the node itself with that velocity
// component reflected.
template <int BC>
__device__ __forceinline__ void pull_source(int x, int y, int z, int i, const Dims& d, int& ip,
                                            int& src) {
    const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
    int sx = x - cx, sy = y - cy, sz = z - cz;
    if (BC == LBM_BC_PERIODIC) {
        sx = sx < 0 ? sx + d.nx : (sx >= d.nx ? sx - d.nx : sx);
        sy = sy < 0 ? sy + d.ny : (sy >= d.ny ? sy - d.ny : sy);
        sz = sz < 0 ? sz + d.nz : (sz >= d.nz ? sz - d.nz : sz);
        ip = i;
    } else {
        const bool fx = sx < 0 || sx >= d.nx, fy = sy < 0 || sy >= d.ny, fz = sz < 0 || sz >= d.nz;
        sx = fx ? x : sx;
        sy = fy ? y : sy;
        sz = fz ? z : sz;
        ip = 9 * ((fz ? -cz : cz) + 1) + 3 * ((fy ? -cy : cy) + 1) + ((fx ? -cx : cx) + 1);
    }
    src = (sz * d.ny + sy) * d.nx + sx;
}

__device__ __forceinline__ void cell_coords(long long cell, const Dims& d, int& x, int& y, int& z) {
    const int c = static_cast<int>(cell);
    x = c % d.nx;
    const int yz = c / d.nx;
    y = yz % d.ny;
    z = yz / d.ny;
}

template <int STORAGE, int BC>
__device__ __forceinline__ void load_pulled(const void* src, const Dims& d, int x, int y, int z,
                                            float* df) {
    using S = Store<STORAGE>;
    const typename S::T* base = static_cast<const typename S::T*>(src);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        int ip, s;
        pull_source<BC>(x, y, z, i, d, ip, s);
        df[i] = S::ld(base + static_cast<size_t>(ip) * d.ncell + s);
    }
}

template <int STORAGE>
__device__ __forceinline__ void store_cell(void* dst, const Dims& d, long long cell, const float* df) {
    using S = Store<STORAGE>;
    typename S::T* base = static_cast<typename S::T*>(dst);
#pragma unroll
    for (int i = 0; i < Q; ++i) S::st(base + static_cast<size_t>(i) * d.ncell + cell, df[i]);
}

// Macroscopic fields from the raw moment vector in tensor order (m[0] = rho,
// m[1], m[3], m[9] = sqrt3 j_x, j_y, j_z).
struct Macro {
    float rho, drho, ux, uy, uz;
};

__device__ __forceinline__ Macro macro_from_moments(const float* m, float drho) {
    Macro r;
    r.rho = m[0];
    r.drho = drho;
    const float s = (1.0f / kSqrt3) / r.rho;
    r.ux = m[1] * s;
    r.uy = m[3] * s;
    r.uz = m[9] * s;
    return r;
}

// m = M f in tensor order from deviations; returns rho - 1 separately.
__device__ __forceinline__ float moments_from_dev(const float* df, float* m) {
#pragma unroll
    for (int i = 0; i < Q; ++i) m[i] = df[i];
    moments_inplace(m);
    const float drho = m[0];
    m[0] = 1.0f + drho;  // M w = e_0
    return drho;
}

// f^eq_i - w_i for the quadratic equilibrium (Sec. II.A, Eq. EquilibriumDistribution).
__device__ __forceinline__ float feq_dev(int i, const Macro& q) {
    const float cu = cx_of(i) * q.ux + cy_of(i) * q.uy + cz_of(i) * q.uz;
    const float usq = q.ux * q.ux + q.uy * q.uy + q.uz * q.uz;
    return wgt(i) * (q.drho + q.rho * (3.0f * cu + 4.5f * cu * cu - 1.5f * usq));
}

// Second-order equilibrium moment 3 rho u_a u_b of tensor component e (order 2).
__device__ __forceinline__ float meq2(int e, const Macro& q) {
    const int ex = ex_of(e), ey = ey_of(e), ez = ez_of(e);
    const float u[3] = {q.ux, q.uy, q.uz};
    int a = -1, b = -1;
    const int cnt[3] = {ex, ey, ez};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (cnt[k] == 2) { a = k; b = k; }
        if (cnt[k] == 1) { if (a < 0) a = k; else b = k; }
    }
    return 3.0f * q.rho * u[a] * u[b];
}

// BGK: f* = f - (f - f^eq)/tau (Sec. II.A).
__device__ __forceinline__ void collide_bgk(float* df, const Macro& q, float omega) {
#pragma unroll
    for (int i = 0; i < Q; ++i) df[i] -= omega * (df[i] - feq_dev(i, q));
}

// Generalised MRT of Sec. II.B, eq. omegatheta: f* = f - M^-1 S (m - m^eq) with
// S = 1 on orders 0-1, omega_nu on order 2, rates[n-3] on order n >= 3.
__device__ __forceinline__ void collide_mrt(float* df, const float* m, const Macro& q,
                                            float omega_nu, const float* rates) {
    float y[Q];
#pragma unroll
    for (int e = 0; e < Q; ++e) {
        const int n = order_of(e);
        if (n <= 1) y[e] = 0.0f;
        else if (n == 2) y[e] = omega_nu * (m[e] - meq2(e, q));
        else y[e] = rates[n - 3] * m[e];
    }
    populations_inplace(y);
#pragma unroll
    for (int i = 0; i < Q; ++i) df[i] -= y[i];
}

// KBC (Karlin, Boesch, Chikatamarla 2014; cited in Sec. III.A): Ds = order-2 part and
// Dh = orders 3..6 of the non-equilibrium, beta = 1/(2 tau),
// gamma = 1/beta - (2 - 1/beta) <Ds|Dh>/<Dh|Dh>, <X|Y> = sum X Y / f^eq,
// f* = f - beta (2 Ds + gamma Dh); gamma = 2 when <Dh|Dh> < 1e-30.
__device__ __forceinline__ void collide_kbc(float* df, const float* m, const Macro& q, float tau) {
    float ds[Q], dh[Q];
#pragma unroll
    for (int e = 0; e < Q; ++e) {
        const int n = order_of(e);
        ds[e] = (n == 2) ? (m[e] - meq2(e, q)) : 0.0f;
        dh[e] = (n >= 3) ? m[e] : 0.0f;
    }
    populations_inplace(ds);
    populations_inplace(dh);
    float sh = 0.0f, hh = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        // hardware reciprocal (about 1 ulp): the weights 1/f^eq only shape gamma
        const float inv_feq = __frcp_rn(wgt(i) + feq_dev(i, q));
        const float dhw = dh[i] * inv_feq;
        sh = fmaf(ds[i], dhw, sh);
        hh = fmaf(dh[i], dhw, hh);
    }
    const float beta = 0.5f / tau;
    const float ib = 2.0f * tau;
    const float gamma = (hh >= 1e-30f) ? ib - (2.0f - ib) * __fdividef(sh, hh) : 2.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) df[i] -= beta * (2.0f * ds[i] + gamma * dh[i]);
}

// Kupershtokh source S_i = f^eq(rho, u + du) - f^eq(rho, u), du = F / rho (Sec. II.A).
// c v for one lattice component c in {-1, 0, 1}, exactly
__device__ __forceinline__ float lattice_dot1(int c, float v) { return c == 0 ? 0.0f : (c > 0 ? v : -v); }

__device__ __forceinline__ float lattice_dot(int i, float vx, float vy, float vz) {
    return __fadd_rn(__fadd_rn(lattice_dot1(cx_of(i), vx), lattice_dot1(cy_of(i), vy)), lattice_dot1(cz_of(i), vz));
}

// Exact-difference source f_i += f_i^eq(rho, u + F/rho) - f_i^eq(rho, u) (Sec. II.A, eq. for
// the Kupershtokh force term, dt = 1). Written with explicit round-to-nearest intrinsics so
// that every kernel that inlines it rounds identically (no context-dependent contraction).
__device__ __forceinline__ void add_kupershtokh(float* df, const Macro& q, float Fx, float Fy, float Fz) {
    const float ir = 1.0f / q.rho;
    const float dx = __fmul_rn(Fx, ir), dy = __fmul_rn(Fy, ir), dz = __fmul_rn(Fz, ir);
    const float vx = __fadd_rn(q.ux, dx), vy = __fadd_rn(q.uy, dy), vz = __fadd_rn(q.uz, dz);
    const float vsq = __fmaf_rn(vx, vx, __fmaf_rn(vy, vy, __fmul_rn(vz, vz)));
    const float usq = __fmaf_rn(q.ux, q.ux, __fmaf_rn(q.uy, q.uy, __fmul_rn(q.uz, q.uz)));
    const float dusq = __fsub_rn(vsq, usq);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float cu = lattice_dot(i, q.ux, q.uy, q.uz);
        const float cd = lattice_dot(i, dx, dy, dz);
        const float cv = __fadd_rn(cu, cd);
        const float quad = __fsub_rn(__fmul_rn(cv, cv), __fmul_rn(cu, cu));
        const float t = __fmaf_rn(3.0f, cd, __fmaf_rn(4.5f, quad, __fmul_rn(-1.5f, dusq)));
        df[i] = __fmaf_rn(__fmul_rn(wgt(i), q.rho), t, df[i]);
    }
}

// tau_n = 1/(2(1 + e^{tau~})) + 1/2 and omega_n = 1/tau_n (Sec. II.B).
__device__ __forceinline__ float rate_from_output(float t) {
    const float tau_n = 0.5f / (1.0f + expf(t)) + 0.5f;
    return 1.0f / tau_n;
}

}  // namespace lbm
