// btdf_device.cuh - device-side building blocks shared by the forward
// kernels of one time step and the kernels of its discrete adjoint: storage
// formats, the moments and equilibrium algebra relative to the reference
// velocity, and the pulls with boundary rules.
#pragma once

#include "btdf_internal.cuh"

namespace btdf {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---- storage formats --------------------------------------------------------

template <typename T> struct Io;

// FP32 storage: N = 4 -> one 16-byte vector, N = 2 -> one 8-byte vector.
template <> struct Io<float> {
    template <int N>
    static __device__ __forceinline__ void ldv(const float* p, float (&o)[N]) {
        if constexpr (N == 4) {
            const float4 v = *reinterpret_cast<const float4*>(p);
            o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
        } else if constexpr (N == 1) {
            o[0] = *p;
        } else {
            const float2 v = *reinterpret_cast<const float2*>(p);
            o[0] = v.x; o[1] = v.y;
        }
    }
    template <int N>
    static __device__ __forceinline__ void stv(float* p, const float (&o)[N]) {
        if constexpr (N == 4) *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
        else if constexpr (N == 1) *p = o[0];
        else *reinterpret_cast<float2*>(p) = make_float2(o[0], o[1]);
    }
    static __device__ __forceinline__ float ld1(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ float ld1s(const float* p) { return *p; }
};

// 16-bit storage (FP16 or BF16): pairs converted with the paired intrinsics.
template <typename H, typename H2> struct Io16 {
    static __device__ __forceinline__ float2 to2(unsigned u);
    static __device__ __forceinline__ unsigned from2(float a, float b);
};
// FP16 stores the deviations scaled by 2^10: the bulk of the lattice sits
// 1e-6 .. 1e-3 away from the reference equilibrium, where unscaled FP16 would
// be subnormal; the largest deviations (~0.1 near a body at start-up) stay far
// below FP16's range after scaling.  Power-of-two scaling is exact.
constexpr float kHalfScale = kF16Scale;
constexpr float kHalfInvScale = 1.0f / 1024.0f;
template <> __device__ __forceinline__ float2 Io16<__half, __half2>::to2(unsigned u) {
    const float2 v = __half22float2(*reinterpret_cast<const __half2*>(&u));
    return make_float2(v.x * kHalfInvScale, v.y * kHalfInvScale);
}
template <> __device__ __forceinline__ unsigned Io16<__half, __half2>::from2(float a, float b) {
    const __half2 h = __floats2half2_rn(a * kHalfScale, b * kHalfScale);
    return *reinterpret_cast<const unsigned*>(&h);
}
template <> __device__ __forceinline__ float2 Io16<__nv_bfloat16, __nv_bfloat162>::to2(unsigned u) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
}
template <> __device__ __forceinline__ unsigned Io16<__nv_bfloat16, __nv_bfloat162>::from2(float a,
                                                                                             float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const unsigned*>(&h);
}

template <typename H, typename H2> struct IoHalf {
    using C = Io16<H, H2>;
    template <int N>
    static __device__ __forceinline__ void ldv(const H* p, float (&o)[N]) {
        if constexpr (N == 4) {
            const uint2 r = *reinterpret_cast<const uint2*>(p);
            const float2 a = C::to2(r.x), b = C::to2(r.y);
            o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
        } else if constexpr (N == 1) {
            o[0] = C::to2((unsigned)*reinterpret_cast<const unsigned short*>(p)).x;
        } else {
            const unsigned r = *reinterpret_cast<const unsigned*>(p);
            const float2 a = C::to2(r);
            o[0] = a.x; o[1] = a.y;
        }
    }
    template <int N>
    static __device__ __forceinline__ void stv(H* p, const float (&o)[N]) {
        if constexpr (N == 4) {
            uint2 r;
            r.x = C::from2(o[0], o[1]);
            r.y = C::from2(o[2], o[3]);
            *reinterpret_cast<uint2*>(p) = r;
        } else if constexpr (N == 1) {
            *reinterpret_cast<unsigned short*>(p) = (unsigned short)(C::from2(o[0], 0.0f) & 0xffffu);
        } else {
            *reinterpret_cast<unsigned*>(p) = C::from2(o[0], o[1]);
        }
    }
    static __device__ __forceinline__ float ld1(const H* p);
    static __device__ __forceinline__ float ld1s(const H* p);
};
template <> __device__ __forceinline__ float IoHalf<__half, __half2>::ld1(const __half* p) {
    return __half2float(__ldg(p)) * kHalfInvScale;
}
template <> __device__ __forceinline__ float IoHalf<__nv_bfloat16, __nv_bfloat162>::ld1(
    const __nv_bfloat16* p) {
    return __bfloat162float(__ldg(p));
}
template <> __device__ __forceinline__ float IoHalf<__half, __half2>::ld1s(const __half* p) {
    return __half2float(*p) * kHalfInvScale;
}
template <> __device__ __forceinline__ float IoHalf<__nv_bfloat16, __nv_bfloat162>::ld1s(
    const __nv_bfloat16* p) {
    return __bfloat162float(*p);
}
template <> struct Io<__half> : IoHalf<__half, __half2> {};
template <> struct Io<__nv_bfloat16> : IoHalf<__nv_bfloat16, __nv_bfloat162> {};

// Stored-scale access for the LBM kernels: populations exactly as stored,
// so FP16 keeps its 2^10 factor.  Those kernels carry the factor through the
// streaming and fold it into the moments and the collision constants instead
// of scaling every population on the way in and out; kScale is the stored
// value of a unit deviation.  Power-of-two scaling is exact, so the results
// are the same as with the scaled access.
template <typename T> struct Raw : Io<T> {
    static constexpr float kScale = 1.0f;
};
template <> struct Raw<__half> {
    static constexpr float kScale = kHalfScale;
    static __device__ __forceinline__ float2 to2(unsigned u) {
        return __half22float2(*reinterpret_cast<const __half2*>(&u));
    }
    static __device__ __forceinline__ unsigned from2(float a, float b) {
        const __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<const unsigned*>(&h);
    }
    template <int N>
    static __device__ __forceinline__ void ldv(const __half* p, float (&o)[N]) {
        if constexpr (N == 4) {
            const uint2 r = *reinterpret_cast<const uint2*>(p);
            const float2 a = to2(r.x), b = to2(r.y);
            o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
        } else if constexpr (N == 1) {
            o[0] = __half2float(*p);
        } else {
            const float2 a = to2(*reinterpret_cast<const unsigned*>(p));
            o[0] = a.x; o[1] = a.y;
        }
    }
    template <int N>
    static __device__ __forceinline__ void stv(__half* p, const float (&o)[N]) {
        if constexpr (N == 4) {
            *reinterpret_cast<uint2*>(p) = make_uint2(from2(o[0], o[1]), from2(o[2], o[3]));
        } else if constexpr (N == 1) {
            *p = __float2half_rn(o[0]);
        } else {
            *reinterpret_cast<unsigned*>(p) = from2(o[0], o[1]);
        }
    }
    static __device__ __forceinline__ float ld1(const __half* p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ float ld1s(const __half* p) { return __half2float(*p); }
};

template <typename T>
__device__ __forceinline__ void store_scalar(T* p, float v);
template <> __device__ __forceinline__ void store_scalar<float>(float* p, float v) { *p = v; }
template <> __device__ __forceinline__ void store_scalar<__half>(__half* p, float v) {
    *p = __float2half_rn(v * kHalfScale);
}
template <> __device__ __forceinline__ void store_scalar<__nv_bfloat16>(__nv_bfloat16* p, float v) {
    *p = __float2bfloat16_rn(v);
}

// ---- reference-equilibrium algebra ----------------------------------------

// Velocity part of the equilibrium (Eq. 6 with rho factored out),
// P_a(u) = 3 e.u + 4.5 (e.u)^2 - 1.5 u^2.
__device__ __forceinline__ float eq_part(int a, float ux, float uy) {
    const float eu = ex(a) * ux + ey(a) * uy;
    return eu * (3.0f + 4.5f * eu) - 1.5f * (ux * ux + uy * uy);
}

// P_a(U_r + du) - P_a(U_r), written so that no O(|U_r|) terms cancel.
__device__ __forceinline__ float eq_part_diff(int a, float urx, float ury, float dux, float duy) {
    const float eU = ex(a) * urx + ey(a) * ury;
    const float ed = ex(a) * dux + ey(a) * duy;
    return ed * (3.0f + 4.5f * (2.0f * eU + ed)) -
           1.5f * (2.0f * (urx * dux + ury * duy) + dux * dux + duy * duy);
}

// Density deviation and velocity deviation du* = u* - U_r of one node from
// its stored deviations (Eqs. 9-10): with J = sum_a e_a d_a,
// rho u* = U_r + J, hence du* = (J - drho U_r) / rho.
struct Moments {
    float drho, rho, inv, dux, duy;
};

// Every product that meets a sum is written as an explicit rounded operation
// (__fmaf_rn, __fmul_rn), so the compiler cannot contract differently in
// different kernels and all launch shapes give bitwise identical results.
// d may hold the deviations times a power of two; s (its inverse, a
// compile-time constant at every call) scales the sums back exactly.
__device__ __forceinline__ Moments moments(const float d[9], float urx, float ury, float s = 1.0f) {
    Moments m;
    m.drho = (((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8]) * s;
    m.rho = 1.0f + m.drho;
    m.inv = __fdividef(1.0f, m.rho);
    const float jx = ((d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7])) * s;
    const float jy = ((d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8])) * s;
    m.dux = __fmul_rn(__fmaf_rn(-m.drho, urx, jx), m.inv);
    m.duy = __fmul_rn(__fmaf_rn(-m.drho, ury, jy), m.inv);
    return m;
}

// ---- packed FP32x2 arithmetic (two nodes per instruction) -------------------

// One instruction, two IEEE round-to-nearest operations: the same values as
// the scalar __fadd_rn / __fmul_rn / __fmaf_rn on each half.
__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// moments() for two nodes at once, operation for operation.
struct Moments2 {
    float2 drho, rho, inv, dux, duy;
};
__device__ __forceinline__ Moments2 moments2(const float2 d[9], float urx, float ury, float s = 1.0f) {
    Moments2 m;
    float2 r = add2(add2(add2(d[0], d[1]), add2(d[2], d[3])), add2(add2(d[4], d[5]), add2(d[6], d[7])));
    r = add2(r, d[8]);
    float2 jx = add2(add2(sub2(d[1], d[3]), sub2(d[5], d[6])), sub2(d[8], d[7]));
    float2 jy = sub2(add2(sub2(d[2], d[4]), add2(d[5], d[6])), add2(d[7], d[8]));
    if (s != 1.0f) {
        r = mul2(r, f2(s));
        jx = mul2(jx, f2(s));
        jy = mul2(jy, f2(s));
    }
    m.drho = r;
    m.rho = add2(f2(1.0f), r);
    m.inv = make_float2(__fdividef(1.0f, m.rho.x), __fdividef(1.0f, m.rho.y));
    m.dux = mul2(fma2(m.drho, f2(-urx), jx), m.inv);
    m.duy = mul2(fma2(m.drho, f2(-ury), jy), m.inv);
    return m;
}

// edot() for two nodes; nx, ny are -x, -y.
__device__ __forceinline__ float2 edot2(int a, float2 x, float2 y, float2 nx, float2 ny) {
    const float2 sx = ex(a) > 0 ? x : nx, sy = ey(a) > 0 ? y : ny;
    return ex(a) == 0 ? (ey(a) == 0 ? f2(0.0f) : sy) : (ey(a) == 0 ? sx : add2(sx, sy));
}

// ---- pulls with boundary rules ---------------------------------------------

// Source of population a at node (x, y) under the rules of the y boundaries:
// plane, row and x shift to read from, and the constant to add (bounce-back
// swaps a population for its opposite, whose reference equilibrium differs by
// -6 w_a e_a.U_r; specular reflection keeps e.U_r since U_r has no normal part).
__device__ __forceinline__ void y_source(int a, int y, const LatticeParams& p, int& pa, int& sy,
                                         int& dx, float& add) {
    pa = a;
    sy = y - ey(a);
    dx = -ex(a);
    add = 0.0f;
    if (sy < 0 || sy >= p.ny) {
        if (p.bcy == kBcyPeriodic) {
            sy = sy < 0 ? p.ny - 1 : 0;
        } else if (p.bcy == kBcyFreeslip) {   // half-way specular reflection
            sy = y;
            pa = mirror_y(a);
        } else {                              // half-way bounce-back
            sy = y;
            pa = opposite(a);
            dx = 0;
            add = -6.0f * wt(a) * (ex(a) * p.urx + ey(a) * p.ury);
        }
    }
}

// Post-streaming deviations at one node, interior and wall rules only.
template <typename T>
__device__ void pull_raw(const T* __restrict__ g, const LatticeParams& p, int x, int y, float f[9]) {
#pragma unroll
    for (int a = 0; a < 9; a++) {
        int pa, sy, dx;
        float add;
        y_source(a, y, p, pa, sy, dx, add);
        int sx = x + dx;
        if (sx < 0 || sx >= p.nx) {
            if (p.bcx == kBcxPeriodic) sx = sx < 0 ? sx + p.nx : sx - p.nx;
            else sx = sx < 0 ? 0 : p.nx - 1;   // only reached for columns the caller overrides
        }
        f[a] = Io<T>::ld1(g + p.poff[pa] + (unsigned)sy * p.rs + (unsigned)sx) + add;
    }
}

// Prescribed-velocity box: outer node (x, y) by extrapolation from the
// nearest interior node (the diagonal one at corners) to the node's boundary
// velocity.  Kept out of line: the box is a test configuration, and inlining
// it into every row-end path of the LBM kernels overflows the instruction
// cache of the common path.
template <typename T>
__device__ __noinline__ void pull_box_node(const T* __restrict__ g, const LatticeParams& p, int x, int y,
                                           float* f) {
    const int xn = min(max(x, 1), p.nx - 2), yn = min(max(y, 1), p.ny - 2);
    float f1[9];
    pull_raw<T>(g, p, xn, yn, f1);
    const Moments m = moments(f1, p.urx, p.ury);
    const float2 ub = p.box[perimeter_index(x, y, p.nx, p.ny)];
    const float inx = ub.x - p.urx, iny = ub.y - p.ury;
#pragma unroll
    for (int a = 0; a < 9; a++)
        f[a] = f1[a] + wt(a) * m.rho *
                           (eq_part_diff(a, p.urx, p.ury, inx, iny) -
                            eq_part_diff(a, p.urx, p.ury, m.dux, m.duy));
}

// Post-streaming deviations with the boundary rules of the x ends: inlet
// column by non-equilibrium extrapolation from column 1 to u = (u_in, 0),
// f(0) = f(1) + f_eq(rho_1, u_in) - f_eq(rho_1, u*_1); outlet column copied
// from column nx-2, or, with the convective outlet, relaxed towards it from
// the previous step's outlet column.  The prescribed-velocity box is applied
// by read_node and by the LBM kernels through pull_box_node.
template <typename T>
__device__ void pull_node(const T* __restrict__ g, const LatticeParams& p, int x, int y, float f[9]) {
    if (p.bcx == kBcxInout && x == 0) {
        float f1[9];
        pull_raw<T>(g, p, 1, y, f1);
        const Moments m = moments(f1, p.urx, p.ury);
        const float inx = p.u_in - p.urx, iny = -p.ury;
#pragma unroll
        for (int a = 0; a < 9; a++)
            f[a] = f1[a] + wt(a) * m.rho *
                               (eq_part_diff(a, p.urx, p.ury, inx, iny) -
                                eq_part_diff(a, p.urx, p.ury, m.dux, m.duy));
    } else if (p.bcx == kBcxInout && x == p.nx - 1) {
        pull_raw<T>(g, p, p.nx - 2, y, f);
        if (p.outlet != nullptr) {
            // convective outlet, implicit upwind: (old + U f(N-1)) / (1 + U)
#pragma unroll
            for (int a = 0; a < 9; a++)
                f[a] = __fmaf_rn(p.uc_new, f[a], __fmul_rn(p.uc_old, p.outlet[a * p.ny + y]));
        }
    } else {
        pull_raw<T>(g, p, x, y, f);
    }
}

template <typename T>
__device__ __forceinline__ void read_node(const T* __restrict__ g, const LatticeParams& p, bool pull,
                                          int x, int y, float f[9]) {
    if (pull) {
        if (p.box != nullptr && (x == 0 || x == p.nx - 1 || y == 0 || y == p.ny - 1))
            pull_box_node<T>(g, p, x, y, f);
        else
            pull_node<T>(g, p, x, y, f);
    } else {
#pragma unroll
        for (int a = 0; a < 9; a++) f[a] = Io<T>::ld1(g + p.poff[a] + (unsigned)y * p.rs + (unsigned)x);
    }
}

// read_node for the IB stage, which reads one node per lane: the nine source
// offsets of the pull are formed first (selects, no memory traffic) and the
// nine loads are then issued back to back, so their latencies overlap instead
// of queueing behind the stores of an out-of-line call.  The arithmetic is
// pull_raw's (load plus the bounce-back constant); the inlet and outlet
// columns and the box's outer nodes keep their own paths.
template <typename T>
__device__ __forceinline__ void gather_node(const T* __restrict__ g, const LatticeParams& p, bool pull,
                                            int x, int y, float f[9]) {
    if (!pull) {
        unsigned off[9];
#pragma unroll
        for (int a = 0; a < 9; a++) off[a] = p.poff[a] + (unsigned)y * p.rs + (unsigned)x;
#pragma unroll
        for (int a = 0; a < 9; a++) f[a] = Io<T>::ld1(g + off[a]);
        return;
    }
    if ((p.box != nullptr && (x == 0 || x == p.nx - 1 || y == 0 || y == p.ny - 1)) ||
        (p.bcx == kBcxInout && (x == 0 || x == p.nx - 1))) {
        read_node<T>(g, p, true, x, y, f);
        return;
    }
    unsigned off[9];
    float add[9];
#pragma unroll
    for (int a = 0; a < 9; a++) {
        int pa, sy, dx;
        y_source(a, y, p, pa, sy, dx, add[a]);
        int sx = x + dx;
        if (sx < 0 || sx >= p.nx) sx = sx < 0 ? sx + p.nx : sx - p.nx;   // periodic x only here
        off[a] = p.poff[pa] + (unsigned)sy * p.rs + (unsigned)sx;
    }
    float v[9];
#pragma unroll
    for (int a = 0; a < 9; a++) v[a] = Io<T>::ld1(g + off[a]);
#pragma unroll
    for (int a = 0; a < 9; a++) f[a] = v[a] + add[a];
}

// Lanes per marker: S*S support nodes rounded up to a power of two.
template <int S> struct Group { static constexpr int G = (S * S <= 4) ? 4 : 16; };

template <typename T, int S>
__device__ __forceinline__ long long ib_marker_index() {
    constexpr int G = Group<S>::G;
    constexpr int MPW = 32 / G;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    return wid * MPW + (threadIdx.x & 31) / G;
}

}  // namespace
}  // namespace btdf
