// d3q27.cuh - D3Q27 lattice, Hermite moment transforms and O_h tables for the
// CUDA library (host + device).
//
// Velocity index i = 9*(cz+1) + 3*(cy+1) + (cx+1). Moments are kept in "tensor"
// index e = 9*ez + 3*ey + ex, where e_a in {0,1,2} is how often axis a appears in
// the Hermite component (Sec. II.B lists the 27 components; each is a product of the
// 1-D Hermite polynomials He_0 = 1, He_1 = xi, He_2 = xi^2 - 1 at xi = sqrt(3) c).
// kPrinted[k] maps the printed row order of M (Sec. II.B) to the tensor index.
#pragma once

#include <cstdint>
#include <type_traits>
#include <utility>

namespace lbm {

constexpr int Q = 27;
constexpr float kSqrt3 = 1.7320508075688772f;

__host__ __device__ constexpr int cx_of(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int cy_of(int i) { return (i / 3) % 3 - 1; }
__host__ __device__ constexpr int cz_of(int i) { return i / 9 - 1; }

// 1-D three-point Gauss-Hermite weights 1/6, 2/3, 1/6; D3Q27 weights are products.
__host__ __device__ constexpr double w1d(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
__host__ __device__ constexpr double weight(int i) {
    return w1d(cx_of(i)) * w1d(cy_of(i)) * w1d(cz_of(i));
}

// Printed row order of M in Sec. II.B, as the axis letters of each component
// (the last printed row is garbled; xxyyzz is the only sixth-order component).
struct MomentName { const char* s; };
constexpr MomentName kNames[Q] = {
    {""}, {"x"}, {"y"}, {"z"}, {"xx"}, {"xy"}, {"xz"}, {"yy"}, {"yz"}, {"zz"},
    {"xxy"}, {"xxz"}, {"xyy"}, {"xyz"}, {"xzz"}, {"yyz"}, {"yzz"},
    {"xxyy"}, {"xxyz"}, {"xxzz"}, {"xyyz"}, {"xyzz"}, {"yyzz"},
    {"xxyyz"}, {"xxyzz"}, {"xyyzz"}, {"xxyyzz"}};

constexpr int count_axis(const char* s, char a) {
    int n = 0;
    for (; *s; ++s) n += (*s == a);
    return n;
}

struct PrintedTable { int e[Q]; int order[Q]; };
constexpr PrintedTable make_printed() {
    PrintedTable t{};
    for (int k = 0; k < Q; ++k) {
        int ex = count_axis(kNames[k].s, 'x'), ey = count_axis(kNames[k].s, 'y'),
            ez = count_axis(kNames[k].s, 'z');
        t.e[k] = 9 * ez + 3 * ey + ex;
        t.order[k] = ex + ey + ez;
    }
    return t;
}
constexpr PrintedTable kPrinted = make_printed();

// Tensor index of printed moment K as a compile-time constant usable in device code.
template <int K>
constexpr int kPrintedE = kPrinted.e[K];

// Compile-time loop: f(std::integral_constant<int, I>) for I = 0..N-1.
template <typename F, int... I>
__host__ __device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

__host__ __device__ constexpr int ex_of(int e) { return e % 3; }
__host__ __device__ constexpr int ey_of(int e) { return (e / 3) % 3; }
__host__ __device__ constexpr int ez_of(int e) { return e / 9; }
__host__ __device__ constexpr int order_of(int e) { return ex_of(e) + ey_of(e) + ez_of(e); }

// ---------------------------------------------------------------------------
// Moment transform m = M f and its inverse, as three 1-D passes.
// Along one axis the values a = f(c=-1), b = f(0), c = f(+1) map to
//   He_0: a + b + c,  He_1: sqrt3 (c - a),  He_2: 2 (a + c) - b,
// and back (M^-1 = W M^T N^-1 with 1-D norms 1, 1, 2):
//   f(-1) = (m0 - sqrt3 m1 + m2)/6, f(0) = (2 m0 - m2)/3, f(+1) = (m0 + sqrt3 m1 + m2)/6.
// In place on a 27-array; stride selects the axis (1: x, 3: y, 9: z).
// ---------------------------------------------------------------------------
template <int STRIDE, typename T>
__host__ __device__ __forceinline__ void fwd_axis(T* v) {
#pragma unroll
    for (int o = 0; o < 9; ++o) {
        // the 9 lines along this axis: base index with this axis' digit = 0
        const int hi = (STRIDE == 1) ? 3 * o : (STRIDE == 3) ? (o / 3) * 9 + (o % 3) : o;
        T a = v[hi], b = v[hi + STRIDE], c = v[hi + 2 * STRIDE];
        T s = a + c;
        v[hi] = s + b;
        v[hi + STRIDE] = T(kSqrt3) * (c - a);
        v[hi + 2 * STRIDE] = T(2) * s - b;
    }
}

template <int STRIDE, typename T>
__host__ __device__ __forceinline__ void inv_axis(T* v) {
#pragma unroll
    for (int o = 0; o < 9; ++o) {
        const int hi = (STRIDE == 1) ? 3 * o : (STRIDE == 3) ? (o / 3) * 9 + (o % 3) : o;
        T m0 = v[hi], m1 = v[hi + STRIDE], m2 = v[hi + 2 * STRIDE];
        T p = m0 + m2;
        T q = T(kSqrt3) * m1;
        v[hi] = (p - q) * T(1.0 / 6.0);
        v[hi + STRIDE] = (T(2) * m0 - m2) * T(1.0 / 3.0);
        v[hi + 2 * STRIDE] = (p + q) * T(1.0 / 6.0);
    }
}

// Transposes of the two per-axis transforms (for adjoints). fwdT applies T^T with
// T = [[1,1,1],[-sqrt3,0,sqrt3],[2,-1,2]] (rows He_0..2, columns c = -1,0,1); invT applies
// (T^-1)^T with T^-1 the per-axis inverse above.
template <int STRIDE, typename T>
__host__ __device__ __forceinline__ void fwdT_axis(T* v) {
#pragma unroll
    for (int o = 0; o < 9; ++o) {
        const int hi = (STRIDE == 1) ? 3 * o : (STRIDE == 3) ? (o / 3) * 9 + (o % 3) : o;
        T m0 = v[hi], m1 = v[hi + STRIDE], m2 = v[hi + 2 * STRIDE];
        T q = T(kSqrt3) * m1;
        v[hi] = m0 - q + T(2) * m2;
        v[hi + STRIDE] = m0 - m2;
        v[hi + 2 * STRIDE] = m0 + q + T(2) * m2;
    }
}

template <int STRIDE, typename T>
__host__ __device__ __forceinline__ void invT_axis(T* v) {
#pragma unroll
    for (int o = 0; o < 9; ++o) {
        const int hi = (STRIDE == 1) ? 3 * o : (STRIDE == 3) ? (o / 3) * 9 + (o % 3) : o;
        T a = v[hi], b = v[hi + STRIDE], c = v[hi + 2 * STRIDE];
        v[hi] = (a + c) * T(1.0 / 6.0) + b * T(2.0 / 3.0);
        v[hi + STRIDE] = (c - a) * T(kSqrt3 / 6.0);
        v[hi + 2 * STRIDE] = (a + c) * T(1.0 / 6.0) - b * T(1.0 / 3.0);
    }
}

// M^T applied to a moment-space vector (tensor order in, velocity order out), in place.
template <typename T>
__host__ __device__ __forceinline__ void moments_transpose_inplace(T* v) {
    fwdT_axis<1>(v);
    fwdT_axis<3>(v);
    fwdT_axis<9>(v);
}
// (M^-1)^T applied to a population-space vector (velocity order in, tensor order out).
template <typename T>
__host__ __device__ __forceinline__ void populations_transpose_inplace(T* v) {
    invT_axis<1>(v);
    invT_axis<3>(v);
    invT_axis<9>(v);
}

// f (velocity order) -> m (tensor order), in place.
template <typename T>
__host__ __device__ __forceinline__ void moments_inplace(T* v) {
    fwd_axis<1>(v);
    fwd_axis<3>(v);
    fwd_axis<9>(v);
}
// m (tensor order) -> f (velocity order), in place.
template <typename T>
__host__ __device__ __forceinline__ void populations_inplace(T* v) {
    inv_axis<1>(v);
    inv_axis<3>(v);
    inv_axis<9>(v);
}

// ---------------------------------------------------------------------------
// O_h: 48 signed permutation matrices. Enumeration: axis permutations p in
// lexicographic order, then sign vectors s with bit a set meaning s_a = -1;
// R[a][p[a]] = s_a, i.e. (R c)_a = s_a c_{p(a)}.
// Action on moments (derived from m^(g) = M Pi_g f with (Pi_g f)_i = f_{pi(i)},
// c_{pi(i)} = R c_i, and He_n(-xi) = (-1)^n He_n(xi)):
//   (P_g m)_e = prod_b s_b^[e_{p(b)} == 1] * m_{e'},  e'_b = e_{p(b)}.
// ---------------------------------------------------------------------------
struct GroupTables {
    int R[48][9];
    int vperm[48][Q];
    int mperm_t[48][Q];  // tensor-index moment permutation
    int msign_t[48][Q];
};

constexpr int kPerms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

constexpr GroupTables make_group() {
    GroupTables t{};
    for (int pi = 0; pi < 6; ++pi)
        for (int sb = 0; sb < 8; ++sb) {
            const int g = pi * 8 + sb;
            int s[3] = {(sb & 4) ? -1 : 1, (sb & 2) ? -1 : 1, (sb & 1) ? -1 : 1};
            const int* p = kPerms[pi];
            for (int k = 0; k < 9; ++k) t.R[g][k] = 0;
            for (int a = 0; a < 3; ++a) t.R[g][3 * a + p[a]] = s[a];
            for (int i = 0; i < Q; ++i) {
                int c[3] = {cx_of(i), cy_of(i), cz_of(i)};
                int rc[3] = {s[0] * c[p[0]], s[1] * c[p[1]], s[2] * c[p[2]]};
                t.vperm[g][i] = 9 * (rc[2] + 1) + 3 * (rc[1] + 1) + (rc[0] + 1);
            }
            for (int e = 0; e < Q; ++e) {
                int ev[3] = {ex_of(e), ey_of(e), ez_of(e)};
                int ep[3] = {ev[p[0]], ev[p[1]], ev[p[2]]};
                int sign = 1;
                for (int b = 0; b < 3; ++b)
                    if (ep[b] == 1) sign *= s[b];
                t.mperm_t[g][e] = 9 * ep[2] + 3 * ep[1] + ep[0];
                t.msign_t[g][e] = sign;
            }
        }
    return t;
}

}  // namespace lbm
