// btdf_kernels.cu - sm_103a kernels of one BTDF-IB/LBM time step
// (Jiang & Liu, arXiv 1806.09403, Algorithm 1).
//
// State.  After every step the buffer holds the post-collision populations
// g = f' (Eq. 5 right-hand side) as deviations f_a - f_eq_a(1, U_r) from the
// equilibrium of the reference state (unit density, reference velocity U_r),
// structure-of-arrays, planar [9][ny][nxp] or row-interleaved [ny][9][nxp].
// The post-streaming populations of the next step are obtained by a pull,
// f_a(x) = g_a(x - e_a), with the boundary rules applied inside the pull.  Right after initialisation (or loading a
// checkpoint) the buffer holds post-streaming populations instead and the
// first step reads them in place ("local" mode).
//
// Kernels per step:
//   ib_force       marker-parallel: pull the populations at every support
//                  node, rho and u* (Eqs. 9-10), interpolate (Eq. 14), force
//                  F_b = 2 rho_l (U_b - U*_l) (Eq. 20).  With NF > 1 it runs
//                  NF times (Algorithm 1 step 3); pass k adds the force field
//                  of passes < k to u* (Eq. 11).
//   collide_stream node-parallel, one warp per 128-node row segment: pull,
//                  node-centric spread of F_b onto band nodes (Eq. 15),
//                  u = u* + f / (2 rho) (Eq. 11), f_eq (Eq. 6), Guo term
//                  (Eq. 7), BGK collision (Eq. 5), vector stores; block 0
//                  then reduces the force on every body in FP64 (Eq. 27)
//                  once the IB kernel has finished.
#include "btdf_internal.cuh"
#include "btdf_device.cuh"

#include <cuda.h>

#include <algorithm>

namespace btdf {
namespace {

// ---- the fused LBM kernel ----------------------------------------------------

// Force on every body (Eq. 27) from the Lagrangian forces of this step, in
// FP64, and the step counter.  Run by block 0 of the LBM kernel (after its
// lattice work; first, in the persistent warp-specialized kernel) once the IB
// kernel has finished.  FP64 arithmetic is slow on this part and, on small
// lattices, this reduction is on the step's critical path: one warp per body
// and no work for absent bodies.
__device__ void body_forces_and_step(const LatticeParams& p) {
    __shared__ unsigned long long s_step;
    if (p.nbody > 0) cudaGridDependencySynchronize();
    if (threadIdx.x == 0) s_step = p.step != nullptr ? *p.step : 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const long long slot = (long long)(s_step % (unsigned long long)(p.hist_len > 0 ? p.hist_len : 1)) *
                           p.nbody;
    for (int b = warp; b < p.nbody; b += nwarps) {
        double sx = 0.0, sy = 0.0;
        for (int k = p.body_ptr[b] + lane; k < p.body_ptr[b + 1]; k += 32) {
            const float2 F = p.F[k];
            sx += (double)F.x;
            sy += (double)F.y;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            sx += __shfl_xor_sync(kFull, sx, off);
            sy += __shfl_xor_sync(kFull, sy, off);
        }
        if (lane == 0) {
            const double sc = p.body_scale[b];
            p.hist[slot + b] = make_double2(-sx * sc, -sy * sc);
        }
    }
    if (threadIdx.x == 0 && p.step != nullptr) *p.step = s_step + 1ull;
}

// Second half of one lattice segment, shared by the LBM kernels: the spread
// force on this lane's nodes, the moments, the collision and the stores.
// f holds the post-streaming deviations of nodes x0 .. x0+NPL-1 of row y;
// xw is the first node of the warp's segment.
// Band segment of row y that holds node xw (-1: none); loaded by the callers
// before their population loads so that its latency overlaps them.
__device__ __forceinline__ int band_segment(const LatticeParams& p, int y, int xw) {
    return p.seg_index != nullptr ? __ldg(p.seg_index + y * p.nseg + xw / kSeg) : -1;
}

template <typename T, int NPL>
__device__ __forceinline__ void collide_store(float (&f)[9][NPL], T* __restrict__ gout,
                                              const LatticeParams& p, int y, int xw, int x0,
                                              bool live, int seg) {
    const unsigned rowoff = (unsigned)y * p.rs + (unsigned)x0;
    // Convective outlet: keep this step's post-streaming outlet column for
    // the next step's boundary rule.
    if (p.outlet != nullptr && live && x0 + NPL > p.nx - 1 && x0 <= p.nx - 1) {
        const int i = p.nx - 1 - x0;
#pragma unroll
        for (int a = 0; a < 9; a++) {
            float v = f[a][0];
#pragma unroll
            for (int k = 1; k < NPL; k++)
                if (k == i) v = f[a][k];
            p.outlet[a * p.ny + y] = v * (1.0f / Raw<T>::kScale);
        }
    }
    // Force density on this lane's nodes: node-centric spread (Eq. 15) of the
    // Lagrangian forces over band segments (after the IB kernel has finished),
    // plus the uniform body force.
    float Fx[NPL], Fy[NPL];
#pragma unroll
    for (int i = 0; i < NPL; i++) {
        Fx[i] = 0.0f;
        Fy[i] = 0.0f;
    }
    bool forced = (p.gx != 0.f) || (p.gy != 0.f);
    {
        const int bs = xw / kSeg;
        if (seg >= 0) {
            forced = true;
            cudaGridDependencySynchronize();
            if (live) {
                const int* ptr = p.seg_ptr + (long long)seg * (kSeg + 1) + (x0 - bs * kSeg);
#pragma unroll
                for (int i = 0; i < NPL; i++) {
                    const int b = __ldg(ptr + i), e = __ldg(ptr + i + 1);
                    float sx = 0.f, sy = 0.f;
                    for (int k = b; k < e; k++) {
                        const CsrEntry c = p.csr[k];
                        const float2 F = p.F[c.marker];
                        sx = __fmaf_rn(c.w, F.x, sx);
                        sy = __fmaf_rn(c.w, F.y, sy);
                    }
                    Fx[i] = sx;
                    Fy[i] = sy;
                }
            }
        }
    }

    // Moments (Eqs. 9-10) and the velocity correction u = u* + f / (2 rho)
    // (Eq. 11), as deviations from the reference state.
    float drho[NPL], rho[NPL], du[NPL], dv[NPL], pd0[NPL], uF[NPL], inv[NPL];
    if constexpr (NPL % 2 == 0) {
        // node pairs through the packed FP32x2 instructions
#pragma unroll
        for (int j = 0; j < NPL; j += 2) {
            float2 d[9];
#pragma unroll
            for (int a = 0; a < 9; a++) d[a] = make_float2(f[a][j], f[a][j + 1]);
            const Moments2 m = moments2(d, p.urx, p.ury, 1.0f / Raw<T>::kScale);
            drho[j] = m.drho.x; drho[j + 1] = m.drho.y;
            rho[j] = m.rho.x; rho[j + 1] = m.rho.y;
            inv[j] = m.inv.x; inv[j + 1] = m.inv.y;
            du[j] = m.dux.x; du[j + 1] = m.dux.y;
            dv[j] = m.duy.x; dv[j + 1] = m.duy.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < NPL; i++) {
            float d[9];
#pragma unroll
            for (int a = 0; a < 9; a++) d[a] = f[a][i];
            const Moments m = moments(d, p.urx, p.ury, 1.0f / Raw<T>::kScale);
            drho[i] = m.drho;
            rho[i] = m.rho;
            inv[i] = m.inv;
            du[i] = m.dux;
            dv[i] = m.duy;
        }
    }
#pragma unroll
    for (int i = 0; i < NPL; i++) {
        uF[i] = 0.0f;
        if (forced) {
            Fx[i] += p.gx;
            Fy[i] += p.gy;
            du[i] = __fmaf_rn(__fmul_rn(0.5f, Fx[i]), inv[i], du[i]);
            dv[i] = __fmaf_rn(__fmul_rn(0.5f, Fy[i]), inv[i], dv[i]);
            uF[i] = __fmaf_rn(p.urx + du[i], Fx[i], __fmul_rn(p.ury + dv[i], Fy[i]));
        }
    }
    // 1.5 (2 U_r.du + du^2), the velocity part shared by all populations
    auto velocity_term = [&]() {
#pragma unroll
        for (int i = 0; i < NPL; i++) {
            float t = __fmaf_rn(du[i], du[i], __fmul_rn(dv[i], dv[i]));
            t = __fmaf_rn(2.0f * p.urx, du[i], t);
            t = __fmaf_rn(2.0f * p.ury, dv[i], t);
            pd0[i] = __fmul_rn(1.5f, t);
        }
    };

    // Collision (Eqs. 5-7), one population at a time, in the form
    //   d_eq / w = drho (1 + P(U_r)) + rho (P(u) - P(U_r))
    //   P(u) - P(U_r) = ed (3 + 9 e.U_r + 4.5 ed) - 1.5 (2 U_r.du + du^2),  ed = e.du
    //   d' = (1 - 1/tau) d + (w / tau) d_eq / w
    //        + (1 - 1/(2 tau)) w [e.F (3 + 9 e.u) - 3 u.F]
    T* const out = gout + rowoff;
    const bool store = live && x0 < p.nx;
    if (NPL % 2 == 0 && !forced) {
        constexpr int NP = NPL / 2 > 0 ? NPL / 2 : 1;
        float2 U[NP], V[NP], nU[NP], nV[NP], D[NP], R[NP], P[NP];
#pragma unroll
        for (int j = 0; j < NP; j++) {
            U[j] = make_float2(du[2 * j], du[2 * j + 1]);
            V[j] = make_float2(dv[2 * j], dv[2 * j + 1]);
            nU[j] = mul2(U[j], f2(-1.0f));
            nV[j] = mul2(V[j], f2(-1.0f));
            D[j] = make_float2(drho[2 * j], drho[2 * j + 1]);
            R[j] = make_float2(rho[2 * j], rho[2 * j + 1]);
            // -pd0 of velocity_term for the pair (-1.5 t is exactly -(1.5 t))
            float2 t = fma2(U[j], U[j], mul2(V[j], V[j]));
            t = fma2(f2(2.0f * p.urx), U[j], t);
            t = fma2(f2(2.0f * p.ury), V[j], t);
            P[j] = mul2(f2(-1.5f), t);
        }
#pragma unroll
        for (int a = 0; a < 9; a++) {
            float o[NPL];
#pragma unroll
            for (int j = 0; j < NP; j++) {
                const float2 ed = edot2(a, U[j], V[j], nU[j], nV[j]);
                const float2 pdiff = fma2(ed, fma2(f2(4.5f), ed, p.c1p[a]), P[j]);
                const float2 deqw = fma2(R[j], pdiff, mul2(p.krp[a], D[j]));
                const float2 r = fma2(p.womp[a], deqw, mul2(p.omop, make_float2(f[a][2 * j], f[a][2 * j + 1])));
                o[2 * j] = r.x;
                o[2 * j + 1] = r.y;
            }
            if (store) Raw<T>::template stv<NPL>(out + p.poff[a], o);
        }
    } else if (!forced) {
        velocity_term();
#pragma unroll
        for (int a = 0; a < 9; a++) {
            float o[NPL];
#pragma unroll
            for (int i = 0; i < NPL; i++) {
                const float ed = edot(a, du[i], dv[i]);
                const float pdiff = __fmaf_rn(ed, __fmaf_rn(4.5f, ed, p.c1[a]), -pd0[i]);
                const float deqw = __fmaf_rn(rho[i], pdiff, __fmul_rn(p.kr[a], drho[i]));
                o[i] = __fmaf_rn(p.wom[a], deqw, __fmul_rn(p.one_m_omega, f[a][i]));
            }
            if (store) Raw<T>::template stv<NPL>(out + p.poff[a], o);
        }
    } else {
        velocity_term();
#pragma unroll
        for (int a = 0; a < 9; a++) {
            float o[NPL];
#pragma unroll
            for (int i = 0; i < NPL; i++) {
                const float ed = edot(a, du[i], dv[i]);
                const float pdiff = __fmaf_rn(ed, __fmaf_rn(4.5f, ed, p.c1[a]), -pd0[i]);
                const float deqw = __fmaf_rn(rho[i], pdiff, __fmul_rn(p.kr[a], drho[i]));
                float r = __fmaf_rn(p.wom[a], deqw, __fmul_rn(p.one_m_omega, f[a][i]));
                const float eF = edot(a, Fx[i], Fy[i]);
                const float eu = p.eur[a] + ed;
                const float g = __fmaf_rn(eF, __fmaf_rn(9.0f, eu, 3.0f), __fmul_rn(-3.0f, uF[i]));
                o[i] = __fmaf_rn(p.wg[a], g, r);
            }
            if (store) Raw<T>::template stv<NPL>(out + p.poff[a], o);
        }
    }
}

// One row segment of 32 * NPL nodes: NPL consecutive nodes per lane.  All
// nine vector loads (and the one scalar per shifted plane that lane 0 /
// lane 31 needs from the neighbouring segment) are issued before any is used;
// the values that cross lanes come by shuffle.  Row-end nodes are recomputed
// by pull_node, which carries every boundary rule.  Offsets are 32-bit
// element offsets (the lattice holds fewer than 2^32 / 9 nodes).
template <typename T, bool kPull, int NPL>
__device__ __forceinline__ void lbm_segment(const T* __restrict__ gin, T* __restrict__ gout,
                                            const LatticeParams& p, int y, int xw, int lane,
                                            int seg) {
    const int x0 = xw + NPL * lane;
    const bool live = x0 < p.nxp;
    const bool lane0 = lane == 0, lane31 = lane == 31;

    float f[9][NPL];
    if (!kPull || (y > 0 && y < p.ny - 1)) {
        // Interior row: every source row is y - e_y and every shift -e_x is
        // known at compile time.  Lanes past the padded row end load a valid
        // vector and never store.
        const int x0c = live ? x0 : p.nxp - NPL;
        const unsigned rowc = (unsigned)y * p.rs + (unsigned)x0c;
#pragma unroll
        for (int a = 0; a < 9; a++) {
            const int dx = kPull ? -ex(a) : 0, dy = kPull ? -ey(a) : 0;
            const unsigned off = p.poff[a] + rowc + (unsigned)(dy * (int)p.rs);
            Raw<T>::template ldv<NPL>(gin + off, f[a]);
            float edge = 0.0f;
            if (dx < 0 && lane0 && x0 > 0) edge = Raw<T>::ld1(gin + (off - 1));
            if (dx > 0 && lane31 && x0 + NPL < p.nxp) edge = Raw<T>::ld1(gin + (off + NPL));
            if (dx < 0) {
                float prev = __shfl_up_sync(kFull, f[a][NPL - 1], 1);
                if (lane0) prev = edge;
#pragma unroll
                for (int i = NPL - 1; i > 0; i--) f[a][i] = f[a][i - 1];
                f[a][0] = prev;
            } else if (dx > 0) {
                float next = __shfl_down_sync(kFull, f[a][0], 1);
                if (lane31) next = edge;
#pragma unroll
                for (int i = 0; i < NPL - 1; i++) f[a][i] = f[a][i + 1];
                f[a][NPL - 1] = next;
            }
        }
    } else {
    const unsigned rowoff = (unsigned)y * p.rs + (unsigned)x0;
    float edge[9];
    int shift[9];
#pragma unroll
    for (int a = 0; a < 9; a++) {
        unsigned off;
        int dx = 0;
        if (kPull) {
            int pa = a, sy = y - ey(a);
            dx = -ex(a);
            if (sy < 0 || sy >= p.ny) {
                float unused;
                y_source(a, y, p, pa, sy, dx, unused);
            }
            off = p.poff[pa] + (unsigned)sy * p.rs + (unsigned)x0;
        } else {
            off = p.poff[a] + rowoff;
        }
        shift[a] = dx;
        if (live) {
            Raw<T>::template ldv<NPL>(gin + off, f[a]);
        } else {
#pragma unroll
            for (int i = 0; i < NPL; i++) f[a][i] = 0.0f;
        }
        edge[a] = 0.0f;
        if (dx < 0 && lane0 && live && x0 > 0) edge[a] = Raw<T>::ld1(gin + (off - 1));
        if (dx > 0 && lane31 && live && x0 + NPL < p.nxp) edge[a] = Raw<T>::ld1(gin + (off + NPL));
    }
#pragma unroll
    for (int a = 0; a < 9; a++) {
        if (shift[a] < 0) {
            float prev = __shfl_up_sync(kFull, f[a][NPL - 1], 1);
            if (lane0) prev = edge[a];
#pragma unroll
            for (int i = NPL - 1; i > 0; i--) f[a][i] = f[a][i - 1];
            f[a][0] = prev;
        } else if (shift[a] > 0) {
            float next = __shfl_down_sync(kFull, f[a][0], 1);
            if (lane31) next = edge[a];
#pragma unroll
            for (int i = 0; i < NPL - 1; i++) f[a][i] = f[a][i + 1];
            f[a][NPL - 1] = next;
        }
    }
    }
    if (kPull && p.bcy == kBcyNoslip && (y == 0 || y == p.ny - 1)) {
        // bounce-back swapped these populations for their opposites
#pragma unroll
        for (int a = 0; a < 9; a++) {
            const int sy = y - ey(a);
            if (sy < 0 || sy >= p.ny) {
                const float add = -6.0f * wt(a) * p.eur[a] * Raw<T>::kScale;
#pragma unroll
                for (int i = 0; i < NPL; i++) f[a][i] += add;
            }
        }
    }
    if (kPull && p.box != nullptr) {
        // prescribed-velocity box: the lane's outer nodes (the first and last
        // rows, the two end columns), each through one out-of-line call
        if (live && (y == 0 || y == p.ny - 1 || x0 == 0 || x0 + NPL - 1 >= p.nx - 1)) {
#pragma unroll
            for (int i = 0; i < NPL; i++) {
                const int x = x0 + i;
                if (x < p.nx && (y == 0 || y == p.ny - 1 || x == 0 || x == p.nx - 1)) {
                    float fe[9];
                    pull_box_node<T>(gin, p, x, y, fe);
#pragma unroll
                    for (int a = 0; a < 9; a++) f[a][i] = fe[a] * Raw<T>::kScale;
                }
            }
        }
    } else if (kPull && live && x0 < p.nx && (x0 == 0 || x0 + NPL - 1 >= p.nx - 1)) {
#pragma unroll
        for (int i = 0; i < NPL; i++) {
            const int x = x0 + i;
            if (x == 0 || x == p.nx - 1) {
                float fe[9];
                pull_node<T>(gin, p, x, y, fe);
#pragma unroll
                for (int a = 0; a < 9; a++) f[a][i] = fe[a] * Raw<T>::kScale;
            }
        }
    }

    collide_store<T, NPL>(f, gout, p, y, xw, x0, live, seg);
}

// Each warp walks the row segments with a grid stride, stepping its (row,
// segment) pair without integer division.  The host normally launches one
// segment per warp, so the block scheduler balances the SMs; a capped grid
// makes the kernel persistent.
template <typename T, bool kPull, int NPL, int MINB>
__global__ void __launch_bounds__(lbm_block_threads(sizeof(T), NPL, MINB),
                                  MINB * kThreads / lbm_block_threads(sizeof(T), NPL, MINB))
collide_stream_kernel(const T* __restrict__ gin, T* __restrict__ gout, LatticeParams p) {
    // The next step's IB kernel may launch once every block has started: it
    // only loads its marker tables before waiting for this grid to finish.
    cudaTriggerProgrammaticLaunchCompletion();
    constexpr int SW = 32 * NPL;
    const int lane = threadIdx.x & 31;
    const int nsegw = (p.nxp + SW - 1) / SW;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int y0 = (int)((__umulhi((unsigned)w0, p.wmul) + (unsigned)w0) >> p.wshift);
    const int s0 = w0 - y0 * nsegw;
    // Band segments wait for the IB kernel's forces inside lbm_segment; the
    // body-force reduction comes after block 0's lattice work, when the IB
    // kernel has long finished.
    // L2 prefetch of the segment a later wave of warps will process: its
    // loads then hit L2 instead of waiting on DRAM (one instruction per warp).
    if (p.pf_ahead > 0) {
        const int u2 = w0 + p.pf_ahead;
        if (u2 < (int)p.nwork) {
            const int y2 = (int)((__umulhi((unsigned)u2, p.wmul) + (unsigned)u2) >> p.wshift);
            const int x2 = (u2 - y2 * nsegw) * SW;
            constexpr int LE = 128 / (int)sizeof(T);            // elements per 128-byte line
            constexpr int LINES = (SW + LE - 1) / LE;
            for (int k = lane; k < 9 * LINES; k += 32) {
                const int a = k / LINES, xl = x2 + (k - a * LINES) * LE;
                if (xl < p.nxp) {
                    const T* addr = gin + p.poff[a] + (unsigned)y2 * p.rs + (unsigned)xl;
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(addr));
                }
            }
        }
    }
    int y = y0, s = s0;
    while (y < p.ny) {
        const int seg = band_segment(p, y, s * SW);
        lbm_segment<T, kPull, NPL>(gin, gout, p, y, s * SW, lane, seg);
        s += p.wds;
        y += p.wdy;
        if (s >= nsegw) {
            s -= nsegw;
            y += 1;
        }
    }
    if (blockIdx.x == 0) body_forces_and_step(p);
}

// ---- the software-pipelined LBM kernel ------------------------------------------

// Raw loads of one interior row segment: the nine vectors and the one value
// per shifted plane that lane 0 / lane 31 needs beyond the segment.
template <int NPL>
struct RawSeg {
    float v[9][NPL];
    float e[9];
};

template <typename T, int NPL>
__device__ __forceinline__ void issue_interior(const T* __restrict__ gin, const LatticeParams& p, int y,
                                               int xw, int lane, RawSeg<NPL>& r) {
    const int x0 = xw + NPL * lane;
    const int x0c = x0 < p.nxp ? x0 : p.nxp - NPL;
    const unsigned rowc = (unsigned)y * p.rs + (unsigned)x0c;
#pragma unroll
    for (int a = 0; a < 9; a++) {
        const int dx = -ex(a), dy = -ey(a);
        const unsigned off = p.poff[a] + rowc + (unsigned)(dy * (int)p.rs);
        Raw<T>::template ldv<NPL>(gin + off, r.v[a]);
        r.e[a] = 0.0f;
        if (dx < 0 && lane == 0 && x0 > 0) r.e[a] = Raw<T>::ld1(gin + (off - 1));
        if (dx > 0 && lane == 31 && x0 + NPL < p.nxp) r.e[a] = Raw<T>::ld1(gin + (off + NPL));
    }
}

template <int NPL>
__device__ __forceinline__ void shift_interior(RawSeg<NPL>& r, int lane, float (&f)[9][NPL]) {
#pragma unroll
    for (int a = 0; a < 9; a++) {
        const int dx = -ex(a);
#pragma unroll
        for (int i = 0; i < NPL; i++) f[a][i] = r.v[a][i];
        if (dx < 0) {
            float prev = __shfl_up_sync(kFull, f[a][NPL - 1], 1);
            if (lane == 0) prev = r.e[a];
#pragma unroll
            for (int i = NPL - 1; i > 0; i--) f[a][i] = f[a][i - 1];
            f[a][0] = prev;
        } else if (dx > 0) {
            float next = __shfl_down_sync(kFull, f[a][0], 1);
            if (lane == 31) next = r.e[a];
#pragma unroll
            for (int i = 0; i < NPL - 1; i++) f[a][i] = f[a][i + 1];
            f[a][NPL - 1] = next;
        }
    }
}

// Same schedule as collide_stream_kernel, but each warp issues the loads of
// its next interior segment before computing the current one, so memory
// latency overlaps arithmetic.  Wall rows take the direct path.
template <typename T, int NPL>
__global__ void __launch_bounds__(kThreads, 2)
collide_stream_pf_kernel(const T* __restrict__ gin, T* __restrict__ gout, LatticeParams p) {
    cudaTriggerProgrammaticLaunchCompletion();   // as in collide_stream_kernel
    constexpr int SW = 32 * NPL;
    const int lane = threadIdx.x & 31;
    const int nsegw = (p.nxp + SW - 1) / SW;
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int y = w0 / nsegw, s = w0 - y * nsegw;
    const int dy = nw / nsegw, ds = nw - dy * nsegw;
    RawSeg<NPL> cur;
    bool interior = y > 0 && y < p.ny - 1;
    if (y < p.ny && interior) issue_interior<T, NPL>(gin, p, y, s * SW, lane, cur);
    while (y < p.ny) {
        int yn = y + dy, sn = s + ds;
        if (sn >= nsegw) {
            sn -= nsegw;
            yn += 1;
        }
        const bool n_interior = yn > 0 && yn < p.ny - 1;
        RawSeg<NPL> nxt;
        if (yn < p.ny && n_interior) issue_interior<T, NPL>(gin, p, yn, sn * SW, lane, nxt);
        const int xw = s * SW;
        if (interior) {
            const int x0 = xw + NPL * lane;
            const bool live = x0 < p.nxp;
            const int seg = band_segment(p, y, xw);
            float f[9][NPL];
            shift_interior<NPL>(cur, lane, f);
            if (live && x0 < p.nx && (x0 == 0 || x0 + NPL - 1 >= p.nx - 1)) {
#pragma unroll
                for (int i = 0; i < NPL; i++) {
                    const int x = x0 + i;
                    if (x == 0 || x == p.nx - 1) {
                        float fe[9];
                        pull_node<T>(gin, p, x, y, fe);
#pragma unroll
                        for (int a = 0; a < 9; a++) f[a][i] = fe[a] * Raw<T>::kScale;
                    }
                }
            }
            collide_store<T, NPL>(f, gout, p, y, xw, x0, live, seg);
        } else {
            lbm_segment<T, true, NPL>(gin, gout, p, y, xw, lane, band_segment(p, y, xw));
        }
        cur = nxt;
        y = yn;
        s = sn;
        interior = n_interior;
    }
    if (blockIdx.x == 0) body_forces_and_step(p);
}

// ---- the TMA-tiled LBM kernel ---------------------------------------------------

// Tiles of 128 nodes x TH rows.  One elected thread streams each tile's nine
// population planes, with a one-row and a 16-byte-column halo, from global
// into shared memory with a single 3-D cp.async.bulk.tensor load per tile;
// S tiles are in flight per CTA, tracked by one mbarrier per stage.  Warp w
// of the CTA then computes row y0 + w of the tile from shared memory (x and
// y neighbours included) and stores its post-collision populations straight
// to global memory with vector stores.  Nodes the tile cannot serve (periodic
// wrap rows, the two row ends) fall back to global loads.
template <typename T, int TH, int S>
struct TmaCfg {
    static constexpr int TW = kSeg;                  // 32 lanes x 4 nodes
    static constexpr int H = 16 / (int)sizeof(T);    // halo columns: 16 bytes
    static constexpr int BX = TW + 2 * H;
    static constexpr int BY = TH + 2;
    static constexpr int STAGE_BYTES = 9 * BY * BX * (int)sizeof(T);
    static constexpr int STAGE_STRIDE = (STAGE_BYTES + 1023) / 1024 * 1024;
    static constexpr int SMEM = S * STAGE_STRIDE + 1024 + 64;
};

// Wait bound for one stage (about a second of polling); past it the kernel
// records a timeout and leaves instead of spinning on.
constexpr unsigned kWaitLimit = 1u << 22;

__device__ __forceinline__ unsigned smem_u32(const void* ptr) {
    return (unsigned)__cvta_generic_to_shared(ptr);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity,
                                                  unsigned limit = kWaitLimit) {
    for (unsigned i = 0; i < limit; i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, unsigned long long* bar,
                                            int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

template <typename T, int TH, int S>
__device__ __forceinline__ void tma_issue(const CUtensorMap* map, unsigned char* stages,
                                          unsigned long long* bars, int stage, int t, int ntx) {
    using C = TmaCfg<T, TH, S>;
    const int tx = t % ntx, ty = t / ntx;
    mbar_expect_tx(&bars[stage], C::STAGE_BYTES);
    // x starts 16 bytes left of the tile (aligned); rows start one above it.
    // Coordinates off the lattice read as zero and are never used.
    tma_load_3d(stages + stage * C::STAGE_STRIDE, map, &bars[stage], tx * C::TW - C::H, ty * TH - 1, 0);
}

// One row of a TMA tile (warp `warp` of the tile's TH rows): the nine
// pulled planes from the shared-memory stage (x and y neighbours included;
// wrap rows of a periodic lattice and the two row ends from global memory),
// then collide_store.  C is the tile configuration (TmaCfg); seg is the row's
// band segment (band_segment()).
template <typename T, typename C>
__device__ __forceinline__ void tma_tile_row(const T* __restrict__ tile, const T* __restrict__ gin,
                                             T* __restrict__ gout, const LatticeParams& p, int x0t,
                                             int y0, int warp, int lane, int seg) {
    const int y = y0 + warp;
    if (y < p.ny) {
        const int x0 = x0t + 4 * lane;
        const bool live = x0 < p.nxp;
        float f[9][4];
        if (y > 0 && y < p.ny - 1) {
            // Interior row: all nine sources in the tile, shifts known at
            // compile time.
#pragma unroll
            for (int a = 0; a < 9; a++) {
                const int dx = -ex(a);
                const T* srow = tile + (a * C::BY + warp + 1 - ey(a)) * C::BX + C::H;
                Raw<T>::template ldv<4>(srow + 4 * lane, f[a]);
                if (dx < 0) {
                    float prev = __shfl_up_sync(kFull, f[a][3], 1);
                    if (lane == 0) prev = Raw<T>::ld1s(srow - 1);
                    f[a][3] = f[a][2]; f[a][2] = f[a][1]; f[a][1] = f[a][0]; f[a][0] = prev;
                } else if (dx > 0) {
                    float next = __shfl_down_sync(kFull, f[a][0], 1);
                    if (lane == 31) next = Raw<T>::ld1s(srow + C::TW);
                    f[a][0] = f[a][1]; f[a][1] = f[a][2]; f[a][2] = f[a][3]; f[a][3] = next;
                }
            }
        } else {
#pragma unroll
        for (int a = 0; a < 9; a++) {
            int pa = a, sy = y - ey(a), dx = -ex(a);
            if (sy < 0 || sy >= p.ny) {
                float unused;
                y_source(a, y, p, pa, sy, dx, unused);
            }
            const int r = sy - y0 + 1;                  // row inside the tile
            float v[4];
            if (r >= 0 && r < C::BY) {                  // from shared memory
                const T* srow = tile + (pa * C::BY + r) * C::BX + C::H;
                Raw<T>::template ldv<4>(srow + 4 * lane, v);   // same bank group per lane
                if (dx < 0) {
                    float prev = __shfl_up_sync(kFull, v[3], 1);
                    if (lane == 0) prev = Raw<T>::ld1s(srow - 1);
                    v[3] = v[2]; v[2] = v[1]; v[1] = v[0]; v[0] = prev;
                } else if (dx > 0) {
                    float next = __shfl_down_sync(kFull, v[0], 1);
                    if (lane == 31) next = Raw<T>::ld1s(srow + C::TW);
                    v[0] = v[1]; v[1] = v[2]; v[2] = v[3]; v[3] = next;
                }
            } else {                                    // periodic wrap row: global
                const T* grow = gin + p.poff[pa] + (unsigned)sy * p.rs;
                if (live) Raw<T>::template ldv<4>(grow + x0, v);
                else v[0] = v[1] = v[2] = v[3] = 0.0f;
                if (dx < 0) {
                    float prev = __shfl_up_sync(kFull, v[3], 1);
                    if (lane == 0) prev = (live && x0 > 0) ? Raw<T>::ld1(grow + x0 - 1) : 0.0f;
                    v[3] = v[2]; v[2] = v[1]; v[1] = v[0]; v[0] = prev;
                } else if (dx > 0) {
                    float next = __shfl_down_sync(kFull, v[0], 1);
                    if (lane == 31) next = (live && x0 + 4 < p.nxp) ? Raw<T>::ld1(grow + x0 + 4) : 0.0f;
                    v[0] = v[1]; v[1] = v[2]; v[2] = v[3]; v[3] = next;
                }
            }
#pragma unroll
            for (int i = 0; i < 4; i++) f[a][i] = v[i];
        }
        }
        if (p.bcy == kBcyNoslip && (y == 0 || y == p.ny - 1)) {
#pragma unroll
            for (int a = 0; a < 9; a++) {
                const int sy = y - ey(a);
                if (sy < 0 || sy >= p.ny) {
                    const float add = -6.0f * wt(a) * p.eur[a] * Raw<T>::kScale;
#pragma unroll
                    for (int i = 0; i < 4; i++) f[a][i] += add;
                }
            }
        }
        if (live && x0 < p.nx && (x0 == 0 || x0 + 3 >= p.nx - 1)) {
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int x = x0 + i;
                if (x == 0 || x == p.nx - 1) {
                    float fe[9];
                    pull_node<T>(gin, p, x, y, fe);
#pragma unroll
                    for (int a = 0; a < 9; a++) f[a][i] = fe[a] * Raw<T>::kScale;
                }
            }
        }
        collide_store<T, 4>(f, gout, p, y, x0t, x0, live, seg);
    }
}

template <typename T, int TH, int S>
__global__ void __launch_bounds__(32 * TH, TH == 8 ? 2 : 1)
collide_stream_tma_kernel(const __grid_constant__ CUtensorMap tmap, const T* __restrict__ gin,
                          T* __restrict__ gout, LatticeParams p) {
    cudaTriggerProgrammaticLaunchCompletion();   // as in collide_stream_kernel
    using C = TmaCfg<T, TH, S>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* stages =
        (unsigned char*)(((unsigned long long)smem_raw + 1023ull) & ~1023ull);
    unsigned long long* bars = (unsigned long long*)(stages + S * C::STAGE_STRIDE);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const int ntx = (p.nxp + C::TW - 1) / C::TW;
    const int ntiles = ntx * ((p.ny + TH - 1) / TH);
    if (tid == 0) {
        for (int st = 0; st < S; st++) mbar_init(&bars[st], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0)
        for (int k = 0; k < S; k++) {
            const int t = blockIdx.x + k * gridDim.x;
            if (t < ntiles) tma_issue<T, TH, S>(&tmap, stages, bars, k, t, ntx);
        }

    int issued = S;        // tiles whose loads were issued (bounded by ntiles below)
    for (int k = 0;; k++) {
        const int t = blockIdx.x + k * gridDim.x;
        if (t >= ntiles) break;
        const int st = k % S;
        // p.wait_polls >= 0 shortens this wait (a test of the timeout path);
        // the drain below always keeps the full bound
        const bool ok = mbar_wait_bounded(&bars[st], (unsigned)((k / S) & 1),
                                          p.wait_polls < 0 ? kWaitLimit : (unsigned)p.wait_polls);
        if (!__syncthreads_and(ok)) {
            // A copy did not land: record it and drain the others (bounded).
            if (tid == 0) {
                atomicOr(p.status, kStatusTimeout);
                for (int j = k; j < issued; j++) {
                    if (blockIdx.x + j * gridDim.x >= ntiles) break;
                    mbar_wait_bounded(&bars[j % S], (unsigned)((j / S) & 1));
                }
            }
            return;
        }
        const T* tile = (const T*)(stages + st * C::STAGE_STRIDE);
        const int y0 = (t / ntx) * TH, x0t = (t % ntx) * C::TW;
        const int seg = y0 + warp < p.ny ? band_segment(p, y0 + warp, x0t) : -1;
        tma_tile_row<T, C>(tile, gin, gout, p, x0t, y0, warp, lane, seg);
        // Every thread is done with this stage: refill it with tile k + S.
        __syncthreads();
        if (tid == 0) {
            const int t2 = blockIdx.x + (k + S) * gridDim.x;
            if (t2 < ntiles) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                tma_issue<T, TH, S>(&tmap, stages, bars, st, t2, ntx);
                issued = k + S + 1;
            }
        }
    }
    if (blockIdx.x == 0) body_forces_and_step(p);
}

// ---- the warp-specialized TMA LBM kernel ----------------------------------------

// The tiles of collide_stream_tma_kernel, handed out dynamically: warp TH of
// the CTA is the producer, warps 0..TH-1 compute rows.  The producer takes
// tile indices from a global ticket counter (p.sched[0], one stage use
// ahead), waits until the consumers have released the stage it refills (one
// "empty" mbarrier per stage, TH arrivals), writes the tile index beside the
// stage, issues the tile's 3-D load on the stage's "full" mbarrier, looks up
// the band segment of each of the tile's rows into shared memory and adds the
// stage's second arrival.  Consumer warps walk the stages in order: wait for
// "full", compute their row, arrive on "empty".  No CTA-wide barrier sits
// between tiles, so a warp can run up to S tiles ahead of the slowest, and
// tiles go to CTAs as they free up (the block scheduler's balancing, in a
// persistent grid).  A ticket past the last tile makes the producer post
// index -1, which ends the consumers.  The last CTA to finish resets both
// counters (p.sched[1] counts finished CTAs) for the next launch.
//
// Every wait is bounded.  A consumer that gives up records BTDF_ETIMEOUT and
// raises a shared halt flag that ends every other wait of the CTA; the
// producer then waits (with the full bound) for each of its copies still in
// flight before the CTA exits.
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait on phase `parity` of `bar` that also ends when *halt is set.
__device__ __forceinline__ bool mbar_wait_haltable(unsigned long long* bar, unsigned parity,
                                                    unsigned limit, const volatile int* halt) {
    for (unsigned i = 0; i < limit; i++) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*halt) return false;
    }
    return false;
}

template <typename T, int TH, int S, int MINB>
__global__ void __launch_bounds__(32 * (TH + 1), MINB)
collide_stream_tma_ws_kernel(const __grid_constant__ CUtensorMap tmap, const T* __restrict__ gin,
                             T* __restrict__ gout, LatticeParams p) {
    cudaTriggerProgrammaticLaunchCompletion();   // as in collide_stream_kernel
    using C = TmaCfg<T, TH, S>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* stages =
        (unsigned char*)(((unsigned long long)smem_raw + 1023ull) & ~1023ull);
    unsigned long long* full = (unsigned long long*)(stages + S * C::STAGE_STRIDE);
    unsigned long long* empty = full + S;
    volatile int* tile_of = (volatile int*)(empty + S);   // [S] tile index per stage
    volatile int* halt = tile_of + S;
    volatile int* seg_of = halt + 1;                       // [S][TH] band segment per row
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const int ntx = (p.nxp + C::TW - 1) / C::TW;
    const int ntiles = ntx * ((p.ny + TH - 1) / TH);
    if (tid == 0) {
        for (int st = 0; st < S; st++) {
            mbar_init(&full[st], 2);   // the copy's arrival and the band segments'
            mbar_init(&empty[st], TH);
        }
        *halt = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // Block 0 reduces the body forces first: the other CTAs take the tiles
    // meanwhile, whereas after its last tile the reduction (a dependent chain
    // of loads per body) would be the launch's tail.
    if (blockIdx.x == 0) body_forces_and_step(p);
    // p.wait_polls >= 0 shortens the consumers' waits (a test of the timeout
    // path); the producer's drain always keeps the full bound
    const unsigned limit = p.wait_polls < 0 ? kWaitLimit : (unsigned)p.wait_polls;

    if (warp == TH) {
        // Producer warp.  Lane 0 holds the ticket of the next stage use
        // (taken one use ahead, so the atomic's latency overlaps the wait for
        // a free stage) and issues the copy; then lanes 0..TH-1 look up the
        // band segment of each row of the tile, so that the consumers find it
        // in shared memory beside the tile, and lane 0 adds the stage's
        // second arrival.
        int k = 0;   // stage uses so far
        int t_next = lane == 0 ? (int)atomicAdd(&p.sched[0], 1u) : 0;
        for (;; k++) {
            const int st = k % S;
            if (k >= S) {
                bool ok = mbar_wait_haltable(&empty[st], (unsigned)((k / S - 1) & 1), kWaitLimit, halt);
                ok = __all_sync(kFull, ok);
                if (!ok) {
                    if (lane == 0 && !*halt) {
                        atomicOr(p.status, kStatusTimeout);
                        *halt = 1;
                    }
                    break;
                }
                if (lane == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            }
            if (__any_sync(kFull, *halt != 0)) break;
            int t = __shfl_sync(kFull, t_next, 0);
            if (t >= ntiles) t = -1;
            if (lane == 0) {
                tile_of[st] = t;
                if (t < 0) {
                    mbar_arrive(&full[st]);
                } else {
                    tma_issue<T, TH, S>(&tmap, stages, full, st, t, ntx);
                    t_next = (int)atomicAdd(&p.sched[0], 1u);
                }
            }
            if (t >= 0 && lane < TH) {
                const int y = (t / ntx) * TH + lane;
                seg_of[st * TH + lane] = y < p.ny ? band_segment(p, y, (t % ntx) * C::TW) : -1;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&full[st]);
            if (t < 0) {
                k++;
                break;
            }
        }
        // After a halt, wait for the copies that may still be landing: the
        // last use of each stage.
        if (lane == 0 && *halt)
            for (int j = k - S < 0 ? 0 : k - S; j < k; j++)
                mbar_wait_bounded(&full[j % S], (unsigned)((j / S) & 1));
    } else {
        for (int k = 0;; k++) {
            const int st = k % S;
            bool ok = mbar_wait_haltable(&full[st], (unsigned)((k / S) & 1), limit, halt);
            ok = __all_sync(kFull, ok);
            if (!ok) {
                if (lane == 0 && !*halt) {
                    atomicOr(p.status, kStatusTimeout);
                    *halt = 1;
                }
                break;
            }
            const int t = tile_of[st];
            if (t < 0) break;
            const int seg = seg_of[st * TH + warp];
            const T* tile = (const T*)(stages + st * C::STAGE_STRIDE);
            tma_tile_row<T, C>(tile, gin, gout, p, (t % ntx) * C::TW, (t / ntx) * TH, warp, lane, seg);
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[st]);
        }
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&p.sched[1], 1u) == gridDim.x - 1) {
            p.sched[0] = 0u;
            p.sched[1] = 0u;
        }
    }
}

// ---- the IB stage -------------------------------------------------------------

// Marker-parallel: one lane per support node, G lanes per marker.  Each lane
// pulls the 9 populations of its node, forms rho and u* (Eqs. 9-10) and its
// weighted share of the interpolation (Eq. 14); a segmented shuffle reduction
// completes D_I rho and D_I u*, and the group's first lane writes
// F_b = 2 rho_l (U_b - D_I u*) (Eq. 20).  Launched as a programmatic
// dependent of the previous LBM kernel, it loads its marker tables while that
// kernel drains and waits for it before the pulls; right after that wait it
// lets its own dependent, the next LBM kernel, launch: only band nodes there
// wait for these forces.

// Body of the IB kernel for marker m of this lane's group, on the lattice
// described by p whose populations start at g.
template <typename T, int S>
__device__ __forceinline__ void ib_force_body(const T* __restrict__ g, const LatticeParams& p,
                                              const IbParams& q, int pull, long long m) {
    constexpr int G = Group<S>::G;
    const int lane = threadIdx.x & 31;
    const int li = lane % G;
    const bool head = li == 0 && m < q.nmark;

    // Static marker data first: no kernel of the step writes it.
    MarkerAux ax{};
    if (head) ax = q.aux[m];
    const bool act = m < q.nmark && li < S * S;
    float w = 0.f;
    int x = 0, y = 0;
    if (act) {
        const Marker* mk = q.mk + m;
        w = __ldg(&mk->w[li]);
        x = __ldg(&mk->xs[li % S]);
        y = __ldg(&mk->ys[li / S]);
    }
    // The populations (previous LBM kernel) and the forces of earlier passes
    // (previous IB kernel) come from the preceding launch: wait for it (a
    // no-op unless this grid was launched as its programmatic dependent),
    // then let the dependent LBM kernel launch.
    cudaGridDependencySynchronize();
    cudaTriggerProgrammaticLaunchCompletion();
    float2 Fp = make_float2(0.f, 0.f);
    if (head && q.F_prev != nullptr) Fp = q.F_prev[m];
    // Weighted sums over the support (Eq. 14) of the density deviation and
    // of the velocity deviation u* - U_r.
    float wr = 0.f, wu = 0.f, wv = 0.f;
    if (act) {
        if (w != 0.f) {
            float d[9];
            gather_node<T>(g, p, pull != 0, x, y, d);
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
                        fx = __fmaf_rn(c.w, F.x, fx);
                        fy = __fmaf_rn(c.w, F.y, fy);
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
    if (head) {
        const float rl = ax.wsum + wr;                      // D_I rho
        const float dFx = 2.0f * rl * (ax.ubx_rel - wu);    // Eq. 20 (dt = 1):
        const float dFy = 2.0f * rl * (ax.uby_rel - wv);    // U_b - D_I u*, relative to U_r
        q.F_out[m] = make_float2(Fp.x + dFx, Fp.y + dFy);
        if (q.first_pass) {
            q.Us[m] = make_float2(p.urx * ax.wsum + wu, p.ury * ax.wsum + wv);
            q.rhol[m] = rl;
        }
        if (!(rl > 0.f) || !isfinite(dFx) || !isfinite(dFy)) atomicOr(q.status, kStatusUnstable);
    }
}

template <typename T, int S>
__global__ void __launch_bounds__(kThreads)
ib_force_kernel(const T* __restrict__ g, LatticeParams p, IbParams q, int pull) {
    ib_force_body<T, S>(g, p, q, pull, ib_marker_index<T, S>());
}

// Batched form: the markers of all lattices in one launch; MarkerAux.body
// holds the lattice index, whose description and population offset the
// lanes of that marker use.
template <typename T, int S>
__global__ void __launch_bounds__(kThreads)
ib_force_batch_kernel(const T* __restrict__ g, const LatticeParams* __restrict__ descs,
                      const unsigned long long* __restrict__ case_off, IbParams q, int pull) {
    const long long m = ib_marker_index<T, S>();
    const int c = q.aux[m < q.nmark ? m : q.nmark - 1].body;
    ib_force_body<T, S>(g + case_off[c], descs[c], q, pull, m);
}

// ---- the batched LBM kernel ---------------------------------------------------

// Many independent lattices in one persistent launch.  Work units are blocks
// of 8 rows of one lattice (one row per warp, all of its segments); each CTA
// owns a contiguous range of units chosen on the host to balance segment
// counts, and keeps the description of its current lattice in shared memory.
// Body forces of all lattices are reduced in FP64 across the CTAs at the
// end; the last CTA to finish advances the step counter.
template <typename T, bool kPull, int NPL, int MINB>
__global__ void __launch_bounds__(kThreads, MINB)
collide_stream_batch_kernel(const T* __restrict__ gin, T* __restrict__ gout, BatchLbm b) {
    constexpr int SW = 32 * NPL;
    constexpr int kWords = (int)(sizeof(LatticeParams) / sizeof(int));
    __shared__ __align__(16) LatticeParams sp;
    __shared__ unsigned long long s_step;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) s_step = *b.step;
    __syncthreads();
    int cur = -1;
    unsigned long long off = 0;
    const int u0 = b.cta_units[blockIdx.x], u1 = b.cta_units[blockIdx.x + 1];
    for (int u = u0; u < u1; u++) {
        const int2 un = b.units[u];
        if (un.x != cur) {
            __syncthreads();
            const int* src = reinterpret_cast<const int*>(b.descs + un.x);
            int* dst = reinterpret_cast<int*>(&sp);
            for (int k = tid; k < kWords; k += blockDim.x) dst[k] = src[k];
            __syncthreads();
            cur = un.x;
            off = b.case_off[cur];
        }
        const int y = un.y + warp;
        if (y < sp.ny) {
            const int nsegw = (sp.nxp + SW - 1) / SW;
            for (int s = 0; s < nsegw; s++) {
                const int seg = band_segment(sp, y, s * SW);
                lbm_segment<T, kPull, NPL>(gin + off, gout + off, sp, y, s * SW, lane, seg);
            }
        }
    }
    if (b.nbody > 0) {
        cudaGridDependencySynchronize();
        const int nwarps = blockDim.x >> 5;
        const long long slot =
            (long long)(s_step % (unsigned long long)(b.hist_len > 0 ? b.hist_len : 1)) * b.nbody;
        for (int bb = blockIdx.x * nwarps + warp; bb < b.nbody; bb += gridDim.x * nwarps) {
            double sx = 0.0, sy = 0.0;
            for (int k = b.body_rng[2 * bb] + lane; k < b.body_rng[2 * bb + 1]; k += 32) {
                const float2 F = b.F[k];
                sx += (double)F.x;
                sy += (double)F.y;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                sx += __shfl_xor_sync(kFull, sx, o);
                sy += __shfl_xor_sync(kFull, sy, o);
            }
            if (lane == 0) {
                const double sc = b.body_scale[bb];
                b.hist[slot + bb] = make_double2(-sx * sc, -sy * sc);
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(b.done, 1u) == gridDim.x - 1) {
            *b.step = s_step + 1ull;
            *b.done = 0u;
        }
    }
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
        store_scalar<T>(g + p.poff[a] + (unsigned)y * p.rs + (unsigned)x, (float)dev);
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

// Division of the warp index by nsegw as a multiply and a shift (Granlund
// and Montgomery, "Division by invariant integers using multiplication",
// 1994): with s = ceil(log2 d) and m = floor(2^32 (2^s - d) / d) + 1,
// n / d = (umulhi(n, m) + n) >> s for every n < 2^31.
inline void set_warp_map(LatticeParams& p, int nsegw, long long nw) {
    const unsigned long long d = (unsigned long long)nsegw;
    int s = 0;
    while ((1ull << s) < d) s++;
    p.wmul = (unsigned)((((1ull << s) - d) << 32) / d + 1ull);
    p.wshift = s;
    p.wdy = (int)(nw / nsegw);
    p.wds = (int)(nw - (long long)p.wdy * nsegw);
}

inline unsigned blocks_for(long long threads) {
    return (unsigned)((threads + kThreads - 1) / kThreads);
}

template <typename T, int NPL, int MB>
cudaError_t collide_stream_tn(bool pull, const void* gin, void* gout, LatticeParams p, int grid,
                              bool pdl, cudaStream_t st) {
    constexpr int SW = 32 * NPL;
    constexpr int BT = lbm_block_threads(sizeof(T), NPL, MB);
    const int nsegw = (p.nxp + SW - 1) / SW;
    p.nwork = (long long)p.ny * nsegw;
    const long long need = (p.nwork * 32 + BT - 1) / BT;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::min<long long>(need, (long long)grid));
    cfg.blockDim = dim3(BT);
    cfg.dynamicSmemBytes = 0;
    const long long nw = (long long)cfg.gridDim.x * (BT / 32);
    set_warp_map(p, nsegw, nw);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    const T* a = (const T*)gin;
    T* b = (T*)gout;
    if (pull) return cudaLaunchKernelEx(&cfg, collide_stream_kernel<T, true, NPL, MB>, a, b, p);
    return cudaLaunchKernelEx(&cfg, collide_stream_kernel<T, false, NPL, MB>, a, b, p);
}

template <typename T, int NPL>
cudaError_t collide_stream_pf_tn(const void* gin, void* gout, LatticeParams p, int grid, bool pdl,
                                 cudaStream_t st) {
    constexpr int SW = 32 * NPL;
    p.nwork = (long long)p.ny * ((p.nxp + SW - 1) / SW);
    const long long need = (p.nwork * 32 + kThreads - 1) / kThreads;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::min<long long>(need, (long long)grid));
    cfg.blockDim = dim3(kThreads);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, collide_stream_pf_kernel<T, NPL>, (const T*)gin, (T*)gout, p);
}

template <typename T, int NPL>
int pf_blocks_tn() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, collide_stream_pf_kernel<T, NPL>, kThreads, 0);
    return n;
}

// Register variants: nodes per lane and the resident blocks per SM the
// register budget is cut for, counted in 256-thread blocks (3 x 256 threads
// <= 80 registers, 4 <= 64, 5 <= 48, 6 <= 40); where lbm_block_threads
// picks 128-thread blocks, twice as many are resident.
template <typename T>
cudaError_t collide_stream_t(bool pull, int variant, const void* gin, void* gout, const LatticeParams& p,
                             int grid, bool pdl, cudaStream_t st) {
    switch (variant) {
    case kVarReg4Pf:
        if (pull) return collide_stream_pf_tn<T, 4>(gin, gout, p, grid, pdl, st);
        return collide_stream_tn<T, 4, 3>(pull, gin, gout, p, grid, pdl, st);
    case kVarReg2Pf:
        if (pull) return collide_stream_pf_tn<T, 2>(gin, gout, p, grid, pdl, st);
        return collide_stream_tn<T, 2, 4>(pull, gin, gout, p, grid, pdl, st);
    case kVarReg2: return collide_stream_tn<T, 2, 4>(pull, gin, gout, p, grid, pdl, st);
    case kVarReg1: return collide_stream_tn<T, 1, 6>(pull, gin, gout, p, grid, pdl, st);
    case kVarReg2Occ:
    case kVarReg2OccPf: return collide_stream_tn<T, 2, 5>(pull, gin, gout, p, grid, pdl, st);
    case kVarReg4L2Pf: return collide_stream_tn<T, 4, 3>(pull, gin, gout, p, grid, pdl, st);
    default: return collide_stream_tn<T, 4, 3>(pull, gin, gout, p, grid, pdl, st);
    }
}

template <typename T, int NPL, int MB>
int blocks_per_sm_tn(bool pull) {
    int n = 0;
    if (pull)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, collide_stream_kernel<T, true, NPL, MB>,
                                                      lbm_block_threads(sizeof(T), NPL, MB), 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, collide_stream_kernel<T, false, NPL, MB>,
                                                      lbm_block_threads(sizeof(T), NPL, MB), 0);
    return n > 0 ? n : 1;
}

template <typename T>
int blocks_per_sm_t(bool pull, int variant) {
    switch (variant) {
    case kVarReg4Pf: return pull ? pf_blocks_tn<T, 4>() : blocks_per_sm_tn<T, 4, 3>(pull);
    case kVarReg2Pf: return pull ? pf_blocks_tn<T, 2>() : blocks_per_sm_tn<T, 2, 4>(pull);
    case kVarReg2: return blocks_per_sm_tn<T, 2, 4>(pull);
    case kVarReg1: return blocks_per_sm_tn<T, 1, 6>(pull);
    case kVarReg2Occ:
    case kVarReg2OccPf: return blocks_per_sm_tn<T, 2, 5>(pull);
    case kVarReg4L2Pf: return blocks_per_sm_tn<T, 4, 3>(pull);
    default: return blocks_per_sm_tn<T, 4, 3>(pull);
    }
}

template <typename T, int TH, int S>
cudaError_t tma_tn(const CUtensorMap* map, const void* gin, void* gout, const LatticeParams& p,
                   int grid, bool pdl, cudaStream_t st) {
    using C = TmaCfg<T, TH, S>;
    auto kern = collide_stream_tma_kernel<T, TH, S>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    const long long ntiles = (long long)((p.nxp + C::TW - 1) / C::TW) * ((p.ny + TH - 1) / TH);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::min<long long>(ntiles, (long long)grid));
    cfg.blockDim = dim3(32 * TH);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, *map, (const T*)gin, (T*)gout, p);
}

template <typename T, int TH, int S>
int tma_blocks_tn() {
    using C = TmaCfg<T, TH, S>;
    auto kern = collide_stream_tma_kernel<T, TH, S>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM) != cudaSuccess)
        return 0;
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, 32 * TH, C::SMEM);
    return n;
}

// Shared memory of the warp-specialized kernel: the stages, alignment slack
// and the full / empty barriers, tile indices, halt flag and band segments.
template <typename T, int TH, int S>
constexpr int ws_smem() {
    return S * TmaCfg<T, TH, S>::STAGE_STRIDE + 1024 + S * (20 + 4 * TH) + 16;
}

template <typename T, int TH, int S, int MINB>
cudaError_t tma_ws_tn(const CUtensorMap* map, const void* gin, void* gout, const LatticeParams& p,
                      int grid, bool pdl, cudaStream_t st) {
    using C = TmaCfg<T, TH, S>;
    if (p.sched == nullptr) return cudaErrorInvalidValue;
    auto kern = collide_stream_tma_ws_kernel<T, TH, S, MINB>;
    constexpr int smem = ws_smem<T, TH, S>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const long long ntiles = (long long)((p.nxp + C::TW - 1) / C::TW) * ((p.ny + TH - 1) / TH);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::min<long long>(ntiles, (long long)grid));
    cfg.blockDim = dim3(32 * (TH + 1));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, *map, (const T*)gin, (T*)gout, p);
}

template <typename T, int TH, int S, int MINB>
int tma_ws_blocks_tn() {
    auto kern = collide_stream_tma_ws_kernel<T, TH, S, MINB>;
    constexpr int smem = ws_smem<T, TH, S>();
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return 0;
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, 32 * (TH + 1), smem);
    return n;
}

template <typename T>
cudaError_t tma_t(int variant, const CUtensorMap* map, const void* gin, void* gout,
                  const LatticeParams& p, int grid, bool pdl, cudaStream_t st) {
    switch (variant) {
    case kVarTma8x2: return tma_tn<T, 8, 2>(map, gin, gout, p, grid, pdl, st);
    case kVarTma8x3: return tma_tn<T, 8, 3>(map, gin, gout, p, grid, pdl, st);
    case kVarTma16x2: return tma_tn<T, 16, 2>(map, gin, gout, p, grid, pdl, st);
    case kVarTmaWs8x2: return tma_ws_tn<T, 8, 2, 3>(map, gin, gout, p, grid, pdl, st);
    case kVarTmaWs7x3: return tma_ws_tn<T, 7, 3, 3>(map, gin, gout, p, grid, pdl, st);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
int tma_blocks_t(int variant) {
    switch (variant) {
    case kVarTma8x2: return tma_blocks_tn<T, 8, 2>();
    case kVarTma8x3: return tma_blocks_tn<T, 8, 3>();
    case kVarTma16x2: return tma_blocks_tn<T, 16, 2>();
    case kVarTmaWs8x2: return tma_ws_blocks_tn<T, 8, 2, 3>();
    case kVarTmaWs7x3: return tma_ws_blocks_tn<T, 7, 3, 3>();
    default: return 0;
    }
}

template <typename T, int S>
cudaError_t ib_force_ts(bool pull, const void* g, const LatticeParams& p, const IbParams& q, bool pdl,
                        cudaStream_t st) {
    constexpr int MPW = 32 / Group<S>::G;
    const long long warps = (q.nmark + MPW - 1) / MPW;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks_for(warps * 32));
    cfg.blockDim = dim3(kThreads);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, ib_force_kernel<T, S>, (const T*)g, p, q, pull ? 1 : 0);
}

template <typename T>
cudaError_t ib_force_t(bool pull, int width, const void* g, const LatticeParams& p,
                       const IbParams& q, bool pdl, cudaStream_t st) {
    switch (width) {
    case 2: return ib_force_ts<T, 2>(pull, g, p, q, pdl, st);
    case 3: return ib_force_ts<T, 3>(pull, g, p, q, pdl, st);
    case 4: return ib_force_ts<T, 4>(pull, g, p, q, pdl, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

template <typename T, int NPL>
cudaError_t batch_lbm_tn(bool pull, const void* gin, void* gout, const BatchLbm& b, int grid, bool pdl,
                         cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    constexpr int MB = NPL == 4 ? 3 : 4;
    if (pull)
        return cudaLaunchKernelEx(&cfg, collide_stream_batch_kernel<T, true, NPL, MB>, (const T*)gin,
                                  (T*)gout, b);
    return cudaLaunchKernelEx(&cfg, collide_stream_batch_kernel<T, false, NPL, MB>, (const T*)gin,
                              (T*)gout, b);
}

template <typename T, int NPL>
int batch_blocks_tn() {
    int n = 0, m = 0;
    constexpr int MB = NPL == 4 ? 3 : 4;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, collide_stream_batch_kernel<T, true, NPL, MB>,
                                                  kThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, collide_stream_batch_kernel<T, false, NPL, MB>,
                                                  kThreads, 0);
    return std::max(1, std::min(n, m));
}

template <typename T, int S>
cudaError_t ib_batch_ts(bool pull, const void* g, const LatticeParams* descs,
                        const unsigned long long* case_off, const IbParams& q, cudaStream_t st) {
    constexpr int MPW = 32 / Group<S>::G;
    const long long warps = (q.nmark + MPW - 1) / MPW;
    const unsigned nb = blocks_for(warps * 32);
    ib_force_batch_kernel<T, S><<<nb, kThreads, 0, st>>>((const T*)g, descs, case_off, q, pull ? 1 : 0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t ib_batch_t(bool pull, int width, const void* g, const LatticeParams* descs,
                       const unsigned long long* case_off, const IbParams& q, cudaStream_t st) {
    switch (width) {
    case 2: return ib_batch_ts<T, 2>(pull, g, descs, case_off, q, st);
    case 3: return ib_batch_ts<T, 3>(pull, g, descs, case_off, q, st);
    case 4: return ib_batch_ts<T, 4>(pull, g, descs, case_off, q, st);
    default: return cudaErrorInvalidValue;
    }
}


cudaError_t launch_collide_stream_batch(int storage, bool pull, int npl, const void* gin, void* gout,
                                        const BatchLbm& b, int grid, bool pdl, cudaStream_t st) {
    switch (storage) {
    case kStoreF32:
        return npl == 2 ? batch_lbm_tn<float, 2>(pull, gin, gout, b, grid, pdl, st)
                        : batch_lbm_tn<float, 4>(pull, gin, gout, b, grid, pdl, st);
    case kStoreF16:
        return npl == 2 ? batch_lbm_tn<__half, 2>(pull, gin, gout, b, grid, pdl, st)
                        : batch_lbm_tn<__half, 4>(pull, gin, gout, b, grid, pdl, st);
    case kStoreBF16:
        return npl == 2 ? batch_lbm_tn<__nv_bfloat16, 2>(pull, gin, gout, b, grid, pdl, st)
                        : batch_lbm_tn<__nv_bfloat16, 4>(pull, gin, gout, b, grid, pdl, st);
    default: return cudaErrorInvalidValue;
    }
}

int collide_stream_batch_blocks_per_sm(int storage, int npl) {
    switch (storage) {
    case kStoreF16: return npl == 2 ? batch_blocks_tn<__half, 2>() : batch_blocks_tn<__half, 4>();
    case kStoreBF16:
        return npl == 2 ? batch_blocks_tn<__nv_bfloat16, 2>() : batch_blocks_tn<__nv_bfloat16, 4>();
    default: return npl == 2 ? batch_blocks_tn<float, 2>() : batch_blocks_tn<float, 4>();
    }
}

cudaError_t launch_ib_force_batch(int storage, bool pull, int width, const void* g,
                                  const LatticeParams* descs, const unsigned long long* case_off,
                                  const IbParams& q, cudaStream_t st) {
    if (q.nmark <= 0) return cudaSuccess;
    switch (storage) {
    case kStoreF32: return ib_batch_t<float>(pull, width, g, descs, case_off, q, st);
    case kStoreF16: return ib_batch_t<__half>(pull, width, g, descs, case_off, q, st);
    case kStoreBF16: return ib_batch_t<__nv_bfloat16>(pull, width, g, descs, case_off, q, st);
    default: return cudaErrorInvalidValue;
    }
}


cudaError_t launch_collide_stream(int storage, bool pull, int variant, const void* gin, void* gout,
                                  const LatticeParams& p, int grid, bool pdl, cudaStream_t st) {
    switch (storage) {
    case kStoreF32: return collide_stream_t<float>(pull, variant, gin, gout, p, grid, pdl, st);
    case kStoreF16: return collide_stream_t<__half>(pull, variant, gin, gout, p, grid, pdl, st);
    case kStoreBF16: return collide_stream_t<__nv_bfloat16>(pull, variant, gin, gout, p, grid, pdl, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_collide_stream_tma(int storage, int variant, const CUtensorMap* map, const void* gin,
                                      void* gout, const LatticeParams& p, int grid, bool pdl,
                                      cudaStream_t st) {
    switch (storage) {
    case kStoreF32: return tma_t<float>(variant, map, gin, gout, p, grid, pdl, st);
    case kStoreF16: return tma_t<__half>(variant, map, gin, gout, p, grid, pdl, st);
    case kStoreBF16: return tma_t<__nv_bfloat16>(variant, map, gin, gout, p, grid, pdl, st);
    default: return cudaErrorInvalidValue;
    }
}

int collide_stream_tma_blocks_per_sm(int storage, int variant) {
    switch (storage) {
    case kStoreF16: return tma_blocks_t<__half>(variant);
    case kStoreBF16: return tma_blocks_t<__nv_bfloat16>(variant);
    default: return tma_blocks_t<float>(variant);
    }
}

int tma_box_rows(int variant) {
    return variant == kVarTma16x2 ? 18 : variant == kVarTmaWs7x3 ? 9 : 10;
}
int tma_halo(int storage) { return storage == kStoreF32 ? 4 : 8; }

int collide_stream_block_threads(int storage, int variant) {
    if (variant == kVarTma8x2 || variant == kVarTma8x3 || variant == kVarTma16x2 ||
        variant == kVarTmaWs8x2 || variant == kVarTmaWs7x3)
        return -1;   // the TMA kernels size their own blocks
    if (variant == kVarReg4Pf || variant == kVarReg2Pf) return kThreads;
    const int eb = storage == kStoreF32 ? 4 : 2;
    switch (variant) {
    case kVarReg2: return lbm_block_threads(eb, 2, 4);
    case kVarReg1: return lbm_block_threads(eb, 1, 6);
    case kVarReg2Occ:
    case kVarReg2OccPf: return lbm_block_threads(eb, 2, 5);
    default: return lbm_block_threads(eb, 4, 3);
    }
}

int collide_stream_blocks_per_sm(int storage, bool pull, int variant) {
    switch (storage) {
    case kStoreF16: return blocks_per_sm_t<__half>(pull, variant);
    case kStoreBF16: return blocks_per_sm_t<__nv_bfloat16>(pull, variant);
    default: return blocks_per_sm_t<float>(pull, variant);
    }
}

cudaError_t launch_ib_force(int storage, bool pull, int width, const void* g, const LatticeParams& p,
                            const IbParams& q, bool pdl, cudaStream_t st) {
    if (q.nmark <= 0) return cudaSuccess;
    switch (storage) {
    case kStoreF32: return ib_force_t<float>(pull, width, g, p, q, pdl, st);
    case kStoreF16: return ib_force_t<__half>(pull, width, g, p, q, pdl, st);
    case kStoreBF16: return ib_force_t<__nv_bfloat16>(pull, width, g, p, q, pdl, st);
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
