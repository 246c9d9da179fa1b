// btdf_kernels.cu - sm_103a kernels of one BTDF-IB/LBM time step
// (Jiang & Liu, arXiv 1806.09403, Algorithm 1).
//
// State.  After every step the buffer holds the post-collision populations
// g = f' (Eq. 5 right-hand side) as deviations from the lattice weights,
// structure-of-arrays [9][ny][nxp].  The post-streaming populations of the
// next step are obtained by a pull, f_a(x) = g_a(x - e_a), with the boundary
// rules applied inside the pull.  Right after initialisation (or loading a
// checkpoint) the buffer holds post-streaming populations instead and the
// first step reads them in place ("local" mode).
//
// Kernels per step:
//   ib_force       marker-parallel: pull the populations at every support
//                  node, rho and u* (Eqs. 9-10), interpolate (Eq. 14), force
//                  F_b = 2 rho_l (U_b - U*_l) (Eq. 20); the last block to
//                  finish reduces the force on every body in FP64 (Eq. 27).
//                  With NF > 1 it runs NF times (Algorithm 1 step 3); pass k
//                  adds the force field of passes < k to u* (Eq. 11).
//   collide_stream node-parallel, one warp per 128-node row segment: pull,
//                  node-centric spread of F_b onto band nodes (Eq. 15),
//                  u = u* + f / (2 rho) (Eq. 11), f_eq (Eq. 6), Guo term
//                  (Eq. 7), BGK collision (Eq. 5), vector stores.
#include "btdf_internal.cuh"

namespace btdf {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---- storage formats --------------------------------------------------------

template <typename T> struct Io;

template <> struct Io<float> {
    static __device__ __forceinline__ float4 ld4(const float* p) {
        return __ldg(reinterpret_cast<const float4*>(p));
    }
    static __device__ __forceinline__ float ld1(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ void st4(float* p, float4 v) {
        *reinterpret_cast<float4*>(p) = v;
    }
    static __device__ __forceinline__ float cvt(float v) { return v; }
};

template <> struct Io<__half> {
    static __device__ __forceinline__ float4 ld4(const __half* p) {
        uint2 r = __ldg(reinterpret_cast<const uint2*>(p));
        float2 a = __half22float2(*reinterpret_cast<__half2*>(&r.x));
        float2 b = __half22float2(*reinterpret_cast<__half2*>(&r.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    static __device__ __forceinline__ float ld1(const __half* p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void st4(__half* p, float4 v) {
        __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
        uint2 r;
        r.x = *reinterpret_cast<unsigned*>(&a);
        r.y = *reinterpret_cast<unsigned*>(&b);
        *reinterpret_cast<uint2*>(p) = r;
    }
};

template <> struct Io<__nv_bfloat16> {
    static __device__ __forceinline__ float4 ld4(const __nv_bfloat16* p) {
        uint2 r = __ldg(reinterpret_cast<const uint2*>(p));
        float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&r.x));
        float2 b = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&r.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    static __device__ __forceinline__ float ld1(const __nv_bfloat16* p) {
        return __bfloat162float(__ldg(p));
    }
    static __device__ __forceinline__ void st4(__nv_bfloat16* p, float4 v) {
        __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
        uint2 r;
        r.x = *reinterpret_cast<unsigned*>(&a);
        r.y = *reinterpret_cast<unsigned*>(&b);
        *reinterpret_cast<uint2*>(p) = r;
    }
};

template <typename T>
__device__ __forceinline__ void store_scalar(T* p, float v);
template <> __device__ __forceinline__ void store_scalar<float>(float* p, float v) { *p = v; }
template <> __device__ __forceinline__ void store_scalar<__half>(__half* p, float v) {
    *p = __float2half_rn(v);
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

__device__ __forceinline__ Moments moments(const float d[9], float urx, float ury) {
    Moments m;
    m.drho = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
    m.rho = 1.0f + m.drho;
    m.inv = 1.0f / m.rho;
    const float jx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
    const float jy = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
    m.dux = (jx - m.drho * urx) * m.inv;
    m.duy = (jy - m.drho * ury) * m.inv;
    return m;
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
        f[a] = Io<T>::ld1(g + pa * p.plane + (long long)sy * p.nxp + sx) + add;
    }
}

// Post-streaming deviations with every boundary rule: inlet column by
// non-equilibrium extrapolation from column 1 to u = (u_in, 0),
// f(0) = f(1) + f_eq(rho_1, u_in) - f_eq(rho_1, u*_1); outlet column copied
// from column nx-2.
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
    } else {
        pull_raw<T>(g, p, x, y, f);
    }
}

template <typename T>
__device__ __forceinline__ void read_node(const T* __restrict__ g, const LatticeParams& p, bool pull,
                                          int x, int y, float f[9]) {
    if (pull) {
        pull_node<T>(g, p, x, y, f);
    } else {
#pragma unroll
        for (int a = 0; a < 9; a++) f[a] = Io<T>::ld1(g + a * p.plane + (long long)y * p.nxp + x);
    }
}

// ---- the fused LBM kernel ----------------------------------------------------

// One warp per 128-node row segment, 4 consecutive nodes per lane.  All nine
// vector loads (and the one scalar per shifted plane that lane 0 / lane 31
// needs from the neighbouring segment) are issued before any is used; the
// values that cross lanes come by shuffle.  Row-end nodes are recomputed by
// pull_node, which carries every boundary rule.
template <typename T, bool kPull>
__global__ void __launch_bounds__(kThreads)
collide_stream_kernel(const T* __restrict__ gin, T* __restrict__ gout, LatticeParams p) {
    const int lane = threadIdx.x & 31;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0 && p.step != nullptr) *p.step += 1ull;
    const int y = (int)(wid / p.nseg);
    if (y >= p.ny) return;                       // whole warps only
    const int s = (int)(wid - (long long)y * p.nseg);
    const int x0 = s * kSeg + kNodesPerLane * lane;
    const bool live = x0 < p.nxp;

    float4 v[9];
    float edge[9], add[9];
    int shift[9];
#pragma unroll
    for (int a = 0; a < 9; a++) {
        const T* row;
        int dx = 0;
        add[a] = 0.0f;
        if (kPull) {
            int pa, sy;
            y_source(a, y, p, pa, sy, dx, add[a]);
            row = gin + pa * p.plane + (long long)sy * p.nxp;
        } else {
            row = gin + a * p.plane + (long long)y * p.nxp;
        }
        shift[a] = dx;
        v[a] = live ? Io<T>::ld4(row + x0) : make_float4(0.f, 0.f, 0.f, 0.f);
        edge[a] = 0.0f;
        if (dx < 0 && lane == 0 && live && x0 > 0) edge[a] = Io<T>::ld1(row + x0 - 1);
        if (dx > 0 && lane == 31 && live && x0 + 4 < p.nxp) edge[a] = Io<T>::ld1(row + x0 + 4);
    }
    float f[9][4];
#pragma unroll
    for (int a = 0; a < 9; a++) {
        float4 w = v[a];
        if (shift[a] < 0) {
            float prev = __shfl_up_sync(kFull, w.w, 1);
            if (lane == 0) prev = edge[a];
            w = make_float4(prev, w.x, w.y, w.z);
        } else if (shift[a] > 0) {
            float next = __shfl_down_sync(kFull, w.x, 1);
            if (lane == 31) next = edge[a];
            w = make_float4(w.y, w.z, w.w, next);
        }
        f[a][0] = w.x + add[a];
        f[a][1] = w.y + add[a];
        f[a][2] = w.z + add[a];
        f[a][3] = w.w + add[a];
    }
    if (kPull && live && (x0 == 0 || x0 + 3 >= p.nx - 1) && x0 < p.nx) {
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int x = x0 + i;
            if (x == 0 || x == p.nx - 1) {
                float fe[9];
                pull_node<T>(gin, p, x, y, fe);
#pragma unroll
                for (int a = 0; a < 9; a++) f[a][i] = fe[a];
            }
        }
    }

    // Force density on this lane's nodes: node-centric spread (Eq. 15) of the
    // Lagrangian forces over band segments, plus the uniform body force.
    float Fx[4], Fy[4];
    bool forced = (p.gx != 0.f) || (p.gy != 0.f);
#pragma unroll
    for (int i = 0; i < 4; i++) {
        Fx[i] = 0.0f;
        Fy[i] = 0.0f;
    }
    if (p.seg_index != nullptr) {
        const int seg = __ldg(p.seg_index + (long long)y * p.nseg + s);
        if (seg >= 0) {
            forced = true;
            if (live) {
                const int* ptr = p.seg_ptr + (long long)seg * (kSeg + 1) + kNodesPerLane * lane;
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const int b = __ldg(ptr + i), e = __ldg(ptr + i + 1);
                    for (int k = b; k < e; k++) {
                        const CsrEntry c = p.csr[k];
                        const float2 F = p.F[c.marker];
                        Fx[i] += c.w * F.x;
                        Fy[i] += c.w * F.y;
                    }
                }
            }
        }
    }

    // Moments and velocity correction u = u* + f / (2 rho) (Eq. 11).
    float drho[4], rho[4], dux[4], duy[4], ux[4], uy[4], usq[4], pd0[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        float d[9];
#pragma unroll
        for (int a = 0; a < 9; a++) d[a] = f[a][i];
        const Moments m = moments(d, p.urx, p.ury);
        Fx[i] += p.gx;
        Fy[i] += p.gy;
        float du = m.dux, dv = m.duy;
        if (forced) {
            du += 0.5f * Fx[i] * m.inv;
            dv += 0.5f * Fy[i] * m.inv;
        }
        drho[i] = m.drho;
        rho[i] = m.rho;
        dux[i] = du;
        duy[i] = dv;
        ux[i] = p.urx + du;
        uy[i] = p.ury + dv;
        usq[i] = 1.5f * (ux[i] * ux[i] + uy[i] * uy[i]);
        pd0[i] = 1.5f * (2.0f * (p.urx * du + p.ury * dv) + du * du + dv * dv);
    }

    // Collision (Eqs. 5-7) in deviation form, one population at a time:
    //   d_eq = f_eq(rho, u) - f_eq(1, U_r) = w [drho (1 + P(u)) + P(u) - P(U_r)]
    //   d'   = d - (d - d_eq) / tau + F_a
    const long long base = (long long)y * p.nxp + x0;
    const bool store = live && x0 < p.nx;
#pragma unroll
    for (int a = 0; a < 9; a++) {
        const float eU = ex(a) * p.urx + ey(a) * p.ury;
        float o[4];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const float ed = ex(a) * dux[i] + ey(a) * duy[i];
            const float eu = eU + ed;
            const float pu = eu * (3.0f + 4.5f * eu) - usq[i];                 // P(u)
            const float pdiff = ed * (3.0f + 4.5f * (2.0f * eU + ed)) - pd0[i];  // P(u) - P(U_r)
            const float deq = wt(a) * (drho[i] * (1.0f + pu) + pdiff);            // Eq. 6
            float r = f[a][i] - p.omega * (f[a][i] - deq);                        // Eq. 5
            if (forced) {                                                         // Eq. 7
                const float t = 3.0f * ((ex(a) - ux[i]) * Fx[i] + (ey(a) - uy[i]) * Fy[i]) +
                                9.0f * eu * (ex(a) * Fx[i] + ey(a) * Fy[i]);
                r += p.guo * wt(a) * t;
            }
            o[i] = r;
        }
        if (store) Io<T>::st4(gout + a * p.plane + base, make_float4(o[0], o[1], o[2], o[3]));
    }
    (void)rho;
}

// ---- the IB stage -------------------------------------------------------------

// Lanes per marker: S*S support nodes rounded up to a power of two.
template <int S> struct Group { static constexpr int G = (S * S <= 4) ? 4 : 16; };

template <typename T, int S>
__global__ void __launch_bounds__(kThreads)
ib_force_kernel(const T* __restrict__ g, LatticeParams p, IbParams q, int pull) {
    constexpr int G = Group<S>::G;
    constexpr int MPW = 32 / G;
    const int lane = threadIdx.x & 31;
    const int li = lane % G;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long m = wid * MPW + lane / G;

    // Weighted sums over the support (Eq. 14) of the density deviation and
    // of the velocity deviation u* - U_r.
    float wr = 0.f, wu = 0.f, wv = 0.f;
    if (m < q.nmark && li < S * S) {
        const int xi = li % S, yi = li / S;
        const Marker* mk = q.mk + m;
        const float w = __ldg(&mk->w[li]);
        if (w != 0.f) {
            const int x = __ldg(&mk->xs[xi]), y = __ldg(&mk->ys[yi]);
            float d[9];
            read_node<T>(g, p, pull != 0, x, y, d);
            const Moments mo = moments(d, p.urx, p.ury);
            float du = mo.dux, dv = mo.duy;
            if (q.F_prev != nullptr) {
                // Force field of the earlier passes at this node (Eq. 15) and
                // the corresponding velocity update (Eq. 11, Algorithm 1 3(d)).
                const int seg = __ldg(p.seg_index + (long long)y * p.nseg + x / kSeg);
                float fx = 0.f, fy = 0.f;
                if (seg >= 0) {
                    const int* ptr = p.seg_ptr + (long long)seg * (kSeg + 1) + (x % kSeg);
                    const int b = __ldg(ptr), e = __ldg(ptr + 1);
                    for (int k = b; k < e; k++) {
                        const CsrEntry c = p.csr[k];
                        const float2 F = q.F_prev[c.marker];
                        fx += c.w * F.x;
                        fy += c.w * F.y;
                    }
                }
                du += 0.5f * fx * mo.inv;
                dv += 0.5f * fy * mo.inv;
            }
            wr = w * mo.drho;
            wu = w * du;
            wv = w * dv;
        }
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        wr += __shfl_xor_sync(kFull, wr, off);
        wu += __shfl_xor_sync(kFull, wu, off);
        wv += __shfl_xor_sync(kFull, wv, off);
    }
    if (li == 0 && m < q.nmark) {
        const MarkerAux ax = q.aux[m];
        const float rl = ax.wsum + wr;                   // D_I rho
        const float dFx = 2.0f * rl * (ax.ubx_rel - wu);   // Eq. 20 (dt = 1):
        const float dFy = 2.0f * rl * (ax.uby_rel - wv);   // U_b - D_I u*, relative to U_r
        float2 F = make_float2(dFx, dFy);
        if (q.F_prev != nullptr) {
            const float2 P = q.F_prev[m];
            F.x += P.x;
            F.y += P.y;
        }
        q.F_out[m] = F;
        if (q.first_pass) {
            q.Us[m] = make_float2(p.urx * ax.wsum + wu, p.ury * ax.wsum + wv);
            q.rhol[m] = rl;
        }
        if (!(rl > 0.f) || !isfinite(dFx) || !isfinite(dFy)) atomicOr(q.status, kStatusUnstable);
    }
    if (!q.last_pass) return;

    // Force on each body (Eq. 27), reduced in FP64 by the last block to finish.
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(q.ticket, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const unsigned long long step = *q.step;
    const long long slot = (long long)(step % (unsigned long long)q.hist_len) * q.nbody;
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int b = warp; b < q.nbody; b += nwarps) {
        double sx = 0.0, sy = 0.0;
        for (int k = q.body_ptr[b] + lane; k < q.body_ptr[b + 1]; k += 32) {
            const float2 F = __ldcg(q.F_out + k);
            sx += (double)F.x;
            sy += (double)F.y;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            sx += __shfl_xor_sync(kFull, sx, off);
            sy += __shfl_xor_sync(kFull, sy, off);
        }
        if (lane == 0) {
            const double sc = q.body_scale[b];
            q.hist[slot + b] = make_double2(-sx * sc, -sy * sc);
        }
    }
    if (threadIdx.x == 0) *q.ticket = 0u;
}

// ---- initialisation and read-back ------------------------------------------------

template <typename T>
__global__ void init_kernel(T* g, LatticeParams p, const double* rho, const double* ux,
                            const double* uy) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (long long)p.nx * p.ny) return;
    const int y = (int)(n / p.nx), x = (int)(n - (long long)y * p.nx);
    const double r = rho[n], u = ux[n], v = uy[n];
    const double usq = u * u + v * v;
    const double Ux = p.urx, Uy = p.ury;
    for (int a = 0; a < 9; a++) {
        const double eu = ex(a) * u + ey(a) * v;
        const double eU = ex(a) * Ux + ey(a) * Uy;
        const double w = a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
        const double pu = 3.0 * eu + 4.5 * eu * eu - 1.5 * usq;
        const double pU = 3.0 * eU + 4.5 * eU * eU - 1.5 * (Ux * Ux + Uy * Uy);
        // f_eq(rho, u) - f_eq(1, U_r) = w [(rho - 1)(1 + P(u)) + P(u) - P(U_r)], Eq. 6
        const double dev = w * ((r - 1.0) * (1.0 + pu) + (pu - pU));
        store_scalar<T>(g + a * p.plane + (long long)y * p.nxp + x, (float)dev);
    }
}

template <typename T>
__global__ void read_field_kernel(const T* __restrict__ g, LatticeParams p, int pull, int kind,
                                  float* dst) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nn = (long long)p.nx * p.ny;
    if (n >= nn) return;
    const int y = (int)(n / p.nx), x = (int)(n - (long long)y * p.nx);
    float d[9];
    read_node<T>(g, p, pull != 0, x, y, d);
    if (kind == 3) {
        for (int a = 0; a < 9; a++)
            dst[a * nn + n] = wt(a) * (1.0f + eq_part(a, p.urx, p.ury)) + d[a];
        return;
    }
    const Moments m = moments(d, p.urx, p.ury);
    if (kind == 0) dst[n] = m.rho;
    else if (kind == 1) dst[n] = p.urx + m.dux;
    else dst[n] = p.ury + m.duy;
}

inline unsigned blocks_for(long long threads) {
    return (unsigned)((threads + kThreads - 1) / kThreads);
}

template <typename T>
cudaError_t collide_stream_t(bool pull, const void* gin, void* gout, const LatticeParams& p,
                             cudaStream_t st) {
    const long long threads = (long long)p.ny * p.nseg * 32;
    const unsigned nb = blocks_for(threads);
    if (pull)
        collide_stream_kernel<T, true><<<nb, kThreads, 0, st>>>((const T*)gin, (T*)gout, p);
    else
        collide_stream_kernel<T, false><<<nb, kThreads, 0, st>>>((const T*)gin, (T*)gout, p);
    return cudaGetLastError();
}

template <typename T, int S>
cudaError_t ib_force_ts(bool pull, const void* g, const LatticeParams& p, const IbParams& q,
                        cudaStream_t st) {
    constexpr int MPW = 32 / Group<S>::G;
    const long long warps = (q.nmark + MPW - 1) / MPW;
    const unsigned nb = blocks_for(warps * 32);
    ib_force_kernel<T, S><<<nb, kThreads, 0, st>>>((const T*)g, p, q, pull ? 1 : 0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t ib_force_t(bool pull, int width, const void* g, const LatticeParams& p,
                       const IbParams& q, cudaStream_t st) {
    switch (width) {
    case 2: return ib_force_ts<T, 2>(pull, g, p, q, st);
    case 3: return ib_force_ts<T, 3>(pull, g, p, q, st);
    case 4: return ib_force_ts<T, 4>(pull, g, p, q, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_collide_stream(int storage, bool pull, const void* gin, void* gout,
                                  const LatticeParams& p, cudaStream_t st) {
    switch (storage) {
    case kStoreF32: return collide_stream_t<float>(pull, gin, gout, p, st);
    case kStoreF16: return collide_stream_t<__half>(pull, gin, gout, p, st);
    case kStoreBF16: return collide_stream_t<__nv_bfloat16>(pull, gin, gout, p, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ib_force(int storage, bool pull, int width, const void* g, const LatticeParams& p,
                            const IbParams& q, cudaStream_t st) {
    if (q.nmark <= 0) return cudaSuccess;
    switch (storage) {
    case kStoreF32: return ib_force_t<float>(pull, width, g, p, q, st);
    case kStoreF16: return ib_force_t<__half>(pull, width, g, p, q, st);
    case kStoreBF16: return ib_force_t<__nv_bfloat16>(pull, width, g, p, q, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_init_equilibrium(int storage, void* g, const LatticeParams& p, const double* rho,
                                    const double* ux, const double* uy, cudaStream_t st) {
    const unsigned nb = blocks_for((long long)p.nx * p.ny);
    switch (storage) {
    case kStoreF32: init_kernel<float><<<nb, kThreads, 0, st>>>((float*)g, p, rho, ux, uy); break;
    case kStoreF16: init_kernel<__half><<<nb, kThreads, 0, st>>>((__half*)g, p, rho, ux, uy); break;
    case kStoreBF16:
        init_kernel<__nv_bfloat16><<<nb, kThreads, 0, st>>>((__nv_bfloat16*)g, p, rho, ux, uy);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_read_field(int storage, bool pull, const void* g, const LatticeParams& p, int kind,
                              float* dst, cudaStream_t st) {
    const unsigned nb = blocks_for((long long)p.nx * p.ny);
    const int pl = pull ? 1 : 0;
    switch (storage) {
    case kStoreF32:
        read_field_kernel<float><<<nb, kThreads, 0, st>>>((const float*)g, p, pl, kind, dst);
        break;
    case kStoreF16:
        read_field_kernel<__half><<<nb, kThreads, 0, st>>>((const __half*)g, p, pl, kind, dst);
        break;
    case kStoreBF16:
        read_field_kernel<__nv_bfloat16>
            <<<nb, kThreads, 0, st>>>((const __nv_bfloat16*)g, p, pl, kind, dst);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace btdf
