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
    } else if (BC == LBM_BC_TGV_REDUCED) {
        // Appendix A: a source outside [0, pi/2]^3 lies in one of the 26 neighbouring
        // blocks; the flow symmetry g = (A, t) of that block brings it back. In doubled
        // units of the spacing h (node j at 2j + 1, t = 2N k, period 8N), the image of
        // coordinate s is sign * (2 s_perm + 1) + 2N k.
        const int n = d.nx;
        const int rx = sx < 0 ? -1 : (sx >= n ? 1 : 0), ry = sy < 0 ? -1 : (sy >= n ? 1 : 0),
                  rz = sz < 0 ? -1 : (sz >= n ? 1 : 0);
        ip = i;
        if (rx | ry | rz) {
            const SymRegion& g = d.sym[9 * (rz + 1) + 3 * (ry + 1) + (rx + 1)];
            const int s2[3] = {2 * sx + 1, 2 * sy + 1, 2 * sz + 1};
            int j[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                int v = g.sign[a] * s2[g.perm[a]] + 2 * n * g.k[a];
                v %= 8 * n;
                if (v < 0) v += 8 * n;
                j[a] = (v - 1) >> 1;
            }
            sx = j[0];
            sy = j[1];
            sz = j[2];
            ip = g.pmap[i];
        }
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

// The same pull with, for periodic boxes, the wrapped source offsets of the three axes
// formed once per cell (fewer instructions per load; more registers live, which the
// register-lean step kernels can afford and the tensor-core kernel cannot).
template <int STORAGE, int BC>
__device__ __forceinline__ void load_pulled_offsets(const void* src, const Dims& d, int x, int y, int z,
                                                    float* df) {
    using S = Store<STORAGE>;
    const typename S::T* base = static_cast<const typename S::T*>(src);
    if constexpr (BC == LBM_BC_PERIODIC) {
        // source offsets along each axis for c = +1 (from the cell below) and c = -1
        // (from the cell above), wrapped once per cell instead of once per population
        const int nxy = d.nx * d.ny;
        const int ox[2] = {x == 0 ? d.nx - 1 : -1, x == d.nx - 1 ? 1 - d.nx : 1};
        const int oy[2] = {y == 0 ? (d.ny - 1) * d.nx : -d.nx, y == d.ny - 1 ? (1 - d.ny) * d.nx : d.nx};
        const int oz[2] = {z == 0 ? (d.nz - 1) * nxy : -nxy, z == d.nz - 1 ? (1 - d.nz) * nxy : nxy};
        const int cell = (z * d.ny + y) * d.nx + x;
        static_for<Q>([&](auto Ic) {
            constexpr int i = decltype(Ic)::value;
            constexpr int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
            int s = cell;
            if constexpr (cx != 0) s += ox[cx > 0 ? 0 : 1];
            if constexpr (cy != 0) s += oy[cy > 0 ? 0 : 1];
            if constexpr (cz != 0) s += oz[cz > 0 ? 0 : 1];
            df[i] = S::ld(base + static_cast<size_t>(i) * d.ncell + s);
        });
    } else {
        load_pulled<STORAGE, BC>(src, d, x, y, z, df);
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

// BGK: f* = f - (f - f^eq)/tau (Sec. II.A). Velocities i and 26 - i are opposite, so
// f^eq - w of the pair is e_i +- o_i with the even part e_i = w_i (drho + rho (4.5 (c_i.u)^2
// - 1.5 u^2)) and the odd part o_i = 3 w_i rho c_i.u: each pair's equilibrium costs one
// c_i.u, one square and two products.
__device__ __forceinline__ void collide_bgk(float* df, const Macro& q, float omega) {
    // f* - w = (1 - omega) (f - w) + omega (f^eq - w), with omega folded into the factors of
    // f^eq - w (its even and odd parts per velocity pair)
    const float usq = q.ux * q.ux + q.uy * q.uy + q.uz * q.uz;
    const float base = omega * fmaf(-1.5f * q.rho, usq, q.drho);
    const float r45 = (4.5f * omega) * q.rho, r3 = (3.0f * omega) * q.rho;
    const float keep = 1.0f - omega;
#pragma unroll
    for (int i = 0; i < Q / 2; ++i) {
        const float cu = cx_of(i) * q.ux + cy_of(i) * q.uy + cz_of(i) * q.uz;
        const float even = wgt(i) * fmaf(r45 * cu, cu, base);
        const float odd = (wgt(i) * r3) * cu;
        df[i] = fmaf(keep, df[i], even + odd);
        df[Q - 1 - i] = fmaf(keep, df[Q - 1 - i], even - odd);
    }
    df[Q / 2] = fmaf(keep, df[Q / 2], wgt(Q / 2) * base);
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
// Dh = orders 3..6 of the non-equilibrium part in population space (Hermite basis),
// beta = 1/(2 tau),
// gamma = 1/beta - (2 - 1/beta) <Ds|Dh>/<Dh|Dh>, <X|Y> = sum X Y / f^eq,
// f* = f - beta (2 Ds + gamma Dh); gamma = 2 when <Dh|Dh> < 1e-30.
// The quadratic f^eq has no Hermite moments above order 2 on D3Q27 (the three-point rule
// is exact to degree 5 per axis), so f - f^eq = Ds + Dh and Dh = (f - f^eq) - Ds: only the
// six second-order non-equilibrium moments are transformed back,
//   Ds_i = w_i [ sum_a He2(c_ia) s_aa / 2 + sum_{a<b} 3 c_ia c_ib s_ab ],
// and Ds, f^eq are recomputed in a second pass instead of being held in 54 registers.
template <int I>
__device__ __forceinline__ float kbc_ds_unweighted(const float* s) {  // s: xx, yy, zz, xy, xz, yz
    constexpr int cx = cx_of(I), cy = cy_of(I), cz = cz_of(I);
    constexpr float hx = 0.5f * (3 * cx * cx - 1), hy = 0.5f * (3 * cy * cy - 1), hz = 0.5f * (3 * cz * cz - 1);
    float t = hx * s[0] + hy * s[1] + hz * s[2];
    if constexpr (cx * cy != 0) t += (3.0f * cx * cy) * s[3];
    if constexpr (cx * cz != 0) t += (3.0f * cx * cz) * s[4];
    if constexpr (cy * cz != 0) t += (3.0f * cy * cz) * s[5];
    return t;
}
template <int I>
__device__ __forceinline__ float kbc_ds(const float* s) {
    return wgt(I) * kbc_ds_unweighted<I>(s);
}

// Velocity index i = 9 (c_z + 1) + 3 (c_y + 1) + (c_x + 1): the x-row (c_y, c_z) holds
// c_x = -1, 0, +1 at 9 (c_z + 1) + 3 (c_y + 1) + 0, 1, 2.
static_assert(cx_of(0) == -1 && cx_of(2) == 1 && cy_of(0) == -1 && cy_of(6) == 1 && cz_of(0) == -1 &&
                  cz_of(18) == 1,
              "velocity index order");

// rho - 1, u and the six second-order non-equilibrium moments s = m_2 - m^eq_2 (xx, yy,
// zz, xy, xz, yz; m_aa = sum (3 c_a^2 - 1) f, m_ab = sum 3 c_a c_b f) straight from the
// deviations, without the full 27-moment transform, summed axis by axis: over c_x within
// each x-row, then over c_y within each z-plane, then over c_z (about 75 operations).
__device__ __forceinline__ Macro kbc_moments(const float* df, float* s) {
    // per plane c_z: sum f, sum c_x f, sum c_y f, sum c_y^2 f, sum c_x c_y f, sum c_x^2 f
    float p0[3], p1[3], py[3], pyy[3], pxy[3], p2[3];
#pragma unroll
    for (int z = 0; z < 3; ++z) {
        float s0[3], s1[3], s2[3];  // per row c_y: sum f, sum c_x f, sum c_x^2 f
#pragma unroll
        for (int y = 0; y < 3; ++y) {
            const int b = 9 * z + 3 * y;
            s2[y] = df[b] + df[b + 2];
            s1[y] = df[b + 2] - df[b];
            s0[y] = s2[y] + df[b + 1];
        }
        py[z] = s0[2] - s0[0];
        pyy[z] = s0[0] + s0[2];
        p0[z] = pyy[z] + s0[1];
        p1[z] = (s1[0] + s1[2]) + s1[1];
        pxy[z] = s1[2] - s1[0];
        p2[z] = (s2[0] + s2[2]) + s2[1];
    }
    const float d0 = (p0[0] + p0[2]) + p0[1];
    const float jx = (p1[0] + p1[2]) + p1[1];
    const float jy = (py[0] + py[2]) + py[1];
    const float jz = p0[2] - p0[0];
    const float mxx = fmaf(3.0f, (p2[0] + p2[2]) + p2[1], -d0);
    const float myy = fmaf(3.0f, (pyy[0] + pyy[2]) + pyy[1], -d0);
    const float mzz = fmaf(3.0f, p0[0] + p0[2], -d0);
    const float mxy = 3.0f * ((pxy[0] + pxy[2]) + pxy[1]);
    const float mxz = 3.0f * (p1[2] - p1[0]);
    const float myz = 3.0f * (py[2] - py[0]);
    Macro q;
    q.drho = d0;
    q.rho = 1.0f + d0;
    const float ir = 1.0f / q.rho;
    q.ux = jx * ir;
    q.uy = jy * ir;
    q.uz = jz * ir;
    const float r3 = 3.0f * q.rho;
    s[0] = mxx - r3 * q.ux * q.ux;
    s[1] = myy - r3 * q.uy * q.uy;
    s[2] = mzz - r3 * q.uz * q.uz;
    s[3] = mxy - r3 * q.ux * q.uy;
    s[4] = mxz - r3 * q.ux * q.uz;
    s[5] = myz - r3 * q.uy * q.uz;
    return q;
}

// The even and odd parts of f^eq - w for velocity I and its opposite 26 - I:
// f^eq_I - w_I = even + odd, f^eq_{26-I} - w_I = even - odd (w is even in c).
struct FeqPair {
    float even, odd;
};

template <int I>
__device__ __forceinline__ FeqPair feq_pair(const Macro& q, float base, float r45, float r3) {
    const float cu = cx_of(I) * q.ux + cy_of(I) * q.uy + cz_of(I) * q.uz;
    return {wgt(I) * fmaf(r45 * cu, cu, base), (wgt(I) * r3) * cu};
}

// s: the six second-order non-equilibrium moments of kbc_moments. Ds is quadratic in c, so
// velocities I and 26 - I share it; f^eq is formed from its even and odd parts per pair.
__device__ __forceinline__ void collide_kbc(float* df, const float* s, const Macro& q, float tau) {
    const float usq = q.ux * q.ux + q.uy * q.uy + q.uz * q.uz;
    float sh = 0.0f, hh = 0.0f;
    {
        const float base = fmaf(-1.5f * q.rho, usq, q.drho);
        const float r45 = 4.5f * q.rho, r3 = 3.0f * q.rho;
        // fast reciprocal (a couple of ulp): the weights 1/f^eq only shape gamma
        static_for<Q / 2>([&](auto Ic) {
            constexpr int i = decltype(Ic)::value, o = Q - 1 - i;
            const FeqPair e = feq_pair<i>(q, base, r45, r3);
            const float ds = kbc_ds<i>(s);
            const float fa = e.even + e.odd, fb = e.even - e.odd;
            const float dha = (df[i] - fa) - ds, dhb = (df[o] - fb) - ds;
            const float wa = dha * __fdividef(1.0f, wgt(i) + fa), wb = dhb * __fdividef(1.0f, wgt(i) + fb);
            sh = fmaf(ds, wa + wb, sh);
            hh = fmaf(dha, wa, hh);
            hh = fmaf(dhb, wb, hh);
        });
        constexpr int r = Q / 2;  // the rest velocity
        const float fr = wgt(r) * base;
        const float dsr = kbc_ds<r>(s);
        const float dhr = (df[r] - fr) - dsr;
        const float wr = dhr * __fdividef(1.0f, wgt(r) + fr);
        sh = fmaf(dsr, wr, sh);
        hh = fmaf(dhr, wr, hh);
    }
    const float beta = 0.5f / tau;
    const float ib = 2.0f * tau;
    const float gamma = (hh >= 1e-30f) ? ib - (2.0f - ib) * __fdividef(sh, hh) : 2.0f;
    // second pass: recompute f^eq and Ds (opaque copies of the inputs keep the compiler
    // from holding the first pass's values in registers instead)
    Macro q2 = q;
    float s2[6];
    float usq2 = usq;
    asm volatile("" : "+f"(q2.rho), "+f"(q2.drho), "+f"(q2.ux), "+f"(q2.uy), "+f"(q2.uz), "+f"(usq2));
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        s2[k] = s[k];
        asm volatile("" : "+f"(s2[k]));
    }
    // f* = f - beta (2 Ds + gamma Dh) with Dh = f - f^eq - Ds, written per population as
    // A (f - w) + B (f^eq - w) + C Ds with A = 1 - beta gamma, B = beta gamma, C = -beta (2 - gamma);
    // B and C are folded into the weight of each velocity pair
    const float base = fmaf(-1.5f * q2.rho, usq2, q2.drho);
    const float r45 = 4.5f * q2.rho, r3 = 3.0f * q2.rho;
    const float B = beta * gamma, A = 1.0f - B, C = -beta * (2.0f - gamma);
    const float Br3 = B * r3;
    static_for<Q / 2>([&](auto Ic) {
        constexpr int i = decltype(Ic)::value, o = Q - 1 - i;
        const float cu = cx_of(i) * q2.ux + cy_of(i) * q2.uy + cz_of(i) * q2.uz;
        const float even = (wgt(i) * B) * fmaf(r45 * cu, cu, base);  // B (f^eq - w), even part
        const float odd = (wgt(i) * Br3) * cu;                         // B (f^eq - w), odd part
        const float p = fmaf(wgt(i) * C, kbc_ds_unweighted<i>(s2), even);  // + C Ds
        df[i] = fmaf(A, df[i], p + odd);
        df[o] = fmaf(A, df[o], p - odd);
    });
    constexpr int r = Q / 2;
    const float dsr = kbc_ds<r>(s2);
    df[r] = fmaf(A, df[r], fmaf(C, dsr, B * (wgt(r) * base)));
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
