// btdf_adjoint.cu - discrete adjoint of one BTDF-IB/LBM time step (FP32
// storage, NF = 1).
//
// The forward step n maps the post-collision state g^n to g^{n+1}:
//   f = Pull(g^n) with the boundary rules,
//   rho_e, u*_e from f at the support nodes (Eqs. 9-10),
//   rho_l = sum_e W_le rho_e,  U*_l = sum_e W_le u*_e            (Eq. 14),
//   F_l = 2 rho_l (U_b - U*_l)                                    (Eq. 20),
//   F(x) = sum_l c_l W_lx F_l + body force,  c_l = drs_l ds_l      (Eq. 15),
//   g^{n+1}(x) = BGK collision of f(x) with the Guo term of F(x)   (Eqs. 5-7, 11),
// and the objective collects sum_l dJ/dF_l . F_l.  Given
// lam = dJ/dg^{n+1} the three kernels below form gbar = dJ/dg^n and
// accumulate dJ/dX_l, dJ/dY_l and the inlet part of dJ/dU_in:
//   (A) node-parallel: adjoint of the collision, the inlet extrapolation and
//       the outlet copy folded into columns 1 and nx-2; ordinary nodes push
//       dJ/df back through the pull, band nodes park it with dJ/dF(x);
//   (B) marker-parallel: adjoint of the force law and of spreading and
//       interpolation with respect to the forces and the marker positions;
//   (C) band-node-parallel: adjoint of the interpolation added to the parked
//       dJ/df, then the push.
// The pull reads every stored population at most once, so its adjoint is a
// scatter with a unique writer per entry: plain stores into a zeroed buffer.
#include "btdf_internal.cuh"
#include "btdf_device.cuh"

namespace btdf {
namespace {

// Node force of the step at (x, y) (Eq. 15 plus the uniform body force) and
// the node's band slot (-1: not in a band segment).
__device__ __forceinline__ void node_force(const LatticeParams& p, int x, int y, float& Fx, float& Fy,
                                           int& slot) {
    Fx = 0.f;
    Fy = 0.f;
    slot = -1;
    if (p.seg_index != nullptr) {
        const int seg = __ldg(p.seg_index + y * p.nseg + x / kSeg);
        if (seg >= 0) {
            slot = seg * kSeg + (x % kSeg);
            const int* ptr = p.seg_ptr + (long long)seg * (kSeg + 1) + (x % kSeg);
            const int b = __ldg(ptr), e = __ldg(ptr + 1);
            for (int k = b; k < e; k++) {
                const CsrEntry c = p.csr[k];
                const float2 F = p.F[c.marker];
                Fx = __fmaf_rn(c.w, F.x, Fx);
                Fy = __fmaf_rn(c.w, F.y, Fy);
            }
        }
    }
    Fx += p.gx;
    Fy += p.gy;
}

// Adjoint of the collision (Eqs. 5-7 with Eq. 11) at one node.  With full
// populations f, rho = sum f, m = rho u = sum e f + F/2 and B = 1 - omega/2:
//   g'_a = (1 - omega) f_a + omega w_a [rho + 3 e.m + (4.5 (e.m)^2 - 1.5 m.m) / rho]
//          + B w_a [3 e.F - 3 m.F / rho + 9 (e.m)(e.F) / rho].
// Given lam_a = dJ/dg'_a returns fb_b = dJ/df_b and (Fbx, Fby) = dJ/dF.
__device__ void adj_collide(const LatticeParams& p, const float d[9], float Fx, float Fy,
                            const float lam[9], float fb[9], float& Fbx, float& Fby) {
    float rho = 0.f, jx = 0.f, jy = 0.f;
#pragma unroll
    for (int a = 0; a < 9; a++) {
        const float fa = d[a] + wt(a) * (1.0f + eq_part(a, p.urx, p.ury));   // full population
        rho += fa;
        jx += ex(a) * fa;
        jy += ey(a) * fa;
    }
    const float om = p.omega, B = 1.0f - 0.5f * om;
    const float mx = jx + 0.5f * Fx, my = jy + 0.5f * Fy;
    const float ir = 1.0f / rho, ir2 = ir * ir;
    const float m2 = mx * mx + my * my, mF = mx * Fx + my * Fy;
    float rb = 0.f, mbx = 0.f, mby = 0.f, Fex = 0.f, Fey = 0.f;
#pragma unroll
    for (int a = 0; a < 9; a++) {
        const float l = lam[a] * wt(a);
        const float em = ex(a) * mx + ey(a) * my, eF = ex(a) * Fx + ey(a) * Fy;
        // d/drho
        rb += l * (om * (1.0f - (4.5f * em * em - 1.5f * m2) * ir2) + B * (3.0f * mF - 9.0f * em * eF) * ir2);
        // d/dm
        const float cm = om * (3.0f + 9.0f * em * ir) + B * 9.0f * eF * ir;
        mbx += l * (cm * ex(a) - (om * 3.0f * mx + B * 3.0f * Fx) * ir);
        mby += l * (cm * ey(a) - (om * 3.0f * my + B * 3.0f * Fy) * ir);
        // d/dF at fixed m
        const float ce = B * (3.0f + 9.0f * em * ir);
        Fex += l * (ce * ex(a) - B * 3.0f * mx * ir);
        Fey += l * (ce * ey(a) - B * 3.0f * my * ir);
    }
#pragma unroll
    for (int b = 0; b < 9; b++) fb[b] = (1.0f - om) * lam[b] + rb + ex(b) * mbx + ey(b) * mby;
    Fbx = Fex + 0.5f * mbx;   // m depends on F through F/2
    Fby = Fey + 0.5f * mby;
}

// dJ/df at node (x, y) from lam = dJ/dg' there.
__device__ void adj_node(const float* __restrict__ g, const float* __restrict__ lam,
                         const LatticeParams& p, bool pull, int x, int y, float fb[9], float& Fbx,
                         float& Fby, int& slot) {
    float d[9], l[9];
    read_node<float>(g, p, pull, x, y, d);
#pragma unroll
    for (int a = 0; a < 9; a++) l[a] = __ldg(lam + p.poff[a] + (unsigned)y * p.rs + (unsigned)x);
    float Fx, Fy;
    node_force(p, x, y, Fx, Fy, slot);
    adj_collide(p, d, Fx, Fy, l, fb, Fbx, Fby);
}

// Adjoint of the pull at node (x, y): f_a(x) was read from one stored entry
// g_pa(src); dJ/df_a goes back there.
__device__ void adj_push(float* __restrict__ gbar, const LatticeParams& p, bool pull, int x, int y,
                         const float fb[9]) {
#pragma unroll
    for (int a = 0; a < 9; a++) {
        int pa = a, sy = y, dx = 0;
        if (pull) {
            float unused;
            y_source(a, y, p, pa, sy, dx, unused);
        }
        int sx = x + dx;
        if (sx < 0 || sx >= p.nx) {
            if (p.bcx != kBcxPeriodic) continue;   // only the overridden edge columns read outside
            sx = sx < 0 ? sx + p.nx : sx - p.nx;
        }
        gbar[p.poff[pa] + (unsigned)sy * p.rs + (unsigned)sx] = fb[a];
    }
}

// (A) one thread per node.
__global__ void __launch_bounds__(kThreads)
adj_collide_kernel(const float* __restrict__ g, const float* __restrict__ lam, float* __restrict__ gbar,
                   LatticeParams p, AdjParams q, int pull) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (long long)p.nx * p.ny) return;
    const int y = (int)(n / p.nx), x = (int)(n - (long long)y * p.nx);
    const bool inout = pull && p.bcx == kBcxInout;
    if (inout && (x == 0 || x == p.nx - 1)) return;   // folded into columns 1 and nx-2
    float fb[9], Fbx, Fby;
    int slot;
    adj_node(g, lam, p, pull != 0, x, y, fb, Fbx, Fby, slot);
    if (inout && x == 1) {
        // Inlet by non-equilibrium extrapolation from column 1 (post-stream
        // f1, pre-force u1 = J1 / rho1):
        //   f_a(0) = f1_a + w_a [rho1 P_a(U_in) - 3 e.J1 - (4.5 (e.J1)^2 - 1.5 J1.J1) / rho1].
        float f0b[9], unused_x, unused_y;
        int unused_s;
        adj_node(g, lam, p, true, 0, y, f0b, unused_x, unused_y, unused_s);
        float f1[9];
        pull_raw<float>(g, p, 1, y, f1);
        float r1 = 0.f, jx = 0.f, jy = 0.f;
#pragma unroll
        for (int a = 0; a < 9; a++) {
            const float fa = f1[a] + wt(a) * (1.0f + eq_part(a, p.urx, p.ury));
            r1 += fa;
            jx += ex(a) * fa;
            jy += ey(a) * fa;
        }
        const float ir = 1.0f / r1, U = p.u_in;
        const float j2 = jx * jx + jy * jy;
        float sb = 0.f, sjx = 0.f, sjy = 0.f, dU = 0.f;
#pragma unroll
        for (int a = 0; a < 9; a++) {
            const float l = f0b[a] * wt(a);
            const float ej = ex(a) * jx + ey(a) * jy;
            const float PU = 3.0f * ex(a) * U + 4.5f * ex(a) * ex(a) * U * U - 1.5f * U * U;
            sb += l * (PU + (4.5f * ej * ej - 1.5f * j2) * ir * ir);       // d/drho1
            const float cj = 3.0f + 9.0f * ej * ir;
            sjx += l * (cj * ex(a) - 3.0f * jx * ir);                        // d/dJ1
            sjy += l * (cj * ey(a) - 3.0f * jy * ir);
            dU += l * r1 * (3.0f * ex(a) + 9.0f * ex(a) * ex(a) * U - 3.0f * U);   // d/dU_in
        }
#pragma unroll
        for (int b = 0; b < 9; b++) fb[b] += f0b[b] + sb - (ex(b) * sjx + ey(b) * sjy);
        atomicAdd(q.dU, (double)dU);
    }
    if (inout && x == p.nx - 2) {
        float fob[9], unused_x, unused_y;
        int unused_s;
        adj_node(g, lam, p, true, p.nx - 1, y, fob, unused_x, unused_y, unused_s);   // f(nx-1) = f(nx-2)
#pragma unroll
        for (int b = 0; b < 9; b++) fb[b] += fob[b];
    }
    if (slot >= 0) {
#pragma unroll
        for (int b = 0; b < 9; b++) q.fbar_band[(long long)slot * 9 + b] = fb[b];
        q.Fbar_band[slot] = make_float2(Fbx, Fby);
        return;
    }
    adj_push(gbar, p, pull != 0, x, y, fb);
}

// (B) marker-parallel, G lanes per marker (one per support node).  The
// interpolation is recomputed from g^n; then
//   dJ/dF_l   = c_l sum_e W_le dJ/dF(e) + (objective weight of F_l),
//   dJ/dU*_l  = -2 rho_l dJ/dF_l,   dJ/drho_l = 2 (U_b - U*_l) . dJ/dF_l,
// and, W_le depending on the marker position through delta(x_e - X) delta(y_e - Y),
//   dJ/dX_l  += sum_e dW_le/dX_l [dJ/dU*_l . u*_e + dJ/drho_l rho_e + c_l F_l . dJ/dF(e)]
// (the same with Y).  dJ/drho_l and dJ/dU*_l go to (C) through mbar.
template <int S>
__global__ void __launch_bounds__(kThreads)
adj_ib_kernel(const float* __restrict__ g, LatticeParams p, AdjParams q, int pull) {
    constexpr int G = Group<S>::G;
    const long long m = ib_marker_index<float, S>();
    const int lane = threadIdx.x & 31;
    const int li = lane % G;
    const bool valid = m < q.nmark;
    const long long mm = valid ? m : 0;
    const MarkerAux ax = q.aux[mm];
    const AdjMarker am = q.am[mm];
    const float c = q.cscale[mm];
    float w = 0.f, dwx = 0.f, dwy = 0.f, rho = 1.f, dux = 0.f, duy = 0.f, drho = 0.f;
    float Fex = 0.f, Fey = 0.f;
    if (valid && li < S * S) {
        const int xi = li % S, yi = li / S;
        const Marker* mk = q.mk + mm;
        w = __ldg(&mk->w[li]);
        dwx = am.dwx[xi] * am.wy[yi];
        dwy = am.wx[xi] * am.dwy[yi];
        if (w != 0.f || dwx != 0.f || dwy != 0.f) {
            const int x = __ldg(&mk->xs[xi]), y = __ldg(&mk->ys[yi]);
            float d[9];
            read_node<float>(g, p, pull != 0, x, y, d);
            const Moments mo = moments(d, p.urx, p.ury);
            rho = mo.rho;
            drho = mo.drho;
            dux = mo.dux;
            duy = mo.duy;
            const int seg = __ldg(p.seg_index + y * p.nseg + x / kSeg);
            if (seg >= 0) {
                const float2 fe = q.Fbar_band[seg * kSeg + (x % kSeg)];
                Fex = fe.x;
                Fey = fe.y;
            }
        }
    }
    float sr = w * drho, su = w * dux, sv = w * duy, sfx = w * Fex, sfy = w * Fey;
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        sr += __shfl_xor_sync(kFull, sr, off);
        su += __shfl_xor_sync(kFull, su, off);
        sv += __shfl_xor_sync(kFull, sv, off);
        sfx += __shfl_xor_sync(kFull, sfx, off);
        sfy += __shfl_xor_sync(kFull, sfy, off);
    }
    const float rl = ax.wsum + sr;                              // rho_l
    const float vx = ax.ubx_rel - su, vy = ax.uby_rel - sv;     // U_b - U*_l
    const float Flx = 2.0f * rl * vx, Fly = 2.0f * rl * vy;     // F_l
    const float2 ow = q.objw[mm];
    const float Fbx = c * sfx + ow.x, Fby = c * sfy + ow.y;     // dJ/dF_l
    const float ubx = -2.0f * rl * Fbx, uby = -2.0f * rl * Fby; // dJ/dU*_l
    const float rb = 2.0f * (vx * Fbx + vy * Fby);              // dJ/drho_l
    const float h = ubx * (p.urx + dux) + uby * (p.ury + duy) + rb * rho + c * (Flx * Fex + Fly * Fey);
    float gX = dwx * h, gY = dwy * h;
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        gX += __shfl_xor_sync(kFull, gX, off);
        gY += __shfl_xor_sync(kFull, gY, off);
    }
    if (valid && li == 0) {
        q.dJdX[mm] += (double)gX;
        q.dJdY[mm] += (double)gY;
        q.mbar[mm] = make_float4(rb, ubx, uby, 0.f);
    }
}

// (C) one thread per node of a band segment: adds the adjoint of the
// interpolation of the markers covering the node (rho = sum f,
// u* = sum e f / rho, so d/df_b = rho_bar + (e_b - u*) . U*_bar / rho),
// then pushes like (A).
__global__ void __launch_bounds__(kThreads)
adj_band_kernel(const float* __restrict__ g, float* __restrict__ gbar, LatticeParams p, AdjParams q,
                int pull) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)q.nband * kSeg) return;
    const int seg = (int)(t / kSeg), i = (int)(t % kSeg);
    const int key = q.band_keys[seg];
    const int y = key / p.nseg, x = (key - y * p.nseg) * kSeg + i;
    if (x >= p.nx) return;
    if (pull && p.bcx == kBcxInout && (x == 0 || x == p.nx - 1)) return;   // folded in (A)
    float fb[9];
#pragma unroll
    for (int b = 0; b < 9; b++) fb[b] = q.fbar_band[t * 9 + b];
    const int* ptr = p.seg_ptr + (long long)seg * (kSeg + 1) + i;
    const int kb = __ldg(ptr), ke = __ldg(ptr + 1);
    if (ke > kb) {
        float rb = 0.f, ubx = 0.f, uby = 0.f;
        for (int k = kb; k < ke; k++) {
            const CsrEntry c = p.csr[k];
            const float W = c.w / q.cscale[c.marker];
            const float4 mb = q.mbar[c.marker];
            rb = __fmaf_rn(W, mb.x, rb);
            ubx = __fmaf_rn(W, mb.y, ubx);
            uby = __fmaf_rn(W, mb.z, uby);
        }
        float d[9];
        read_node<float>(g, p, pull != 0, x, y, d);
        const Moments mo = moments(d, p.urx, p.ury);
        const float ux = p.urx + mo.dux, uy = p.ury + mo.duy;
        const float jbx = ubx * mo.inv, jby = uby * mo.inv;
        const float rbar = rb - (ux * ubx + uy * uby) * mo.inv;
#pragma unroll
        for (int b = 0; b < 9; b++) fb[b] += rbar + ex(b) * jbx + ey(b) * jby;
    }
    adj_push(gbar, p, pull != 0, x, y, fb);
}

inline unsigned blocks_of(long long threads) { return (unsigned)((threads + kThreads - 1) / kThreads); }

}  // namespace

cudaError_t launch_adjoint_step(const float* g, const float* lam, float* gbar, const LatticeParams& p,
                                const AdjParams& q, int width, bool pull, cudaStream_t st) {
    const int pl = pull ? 1 : 0;
    adj_collide_kernel<<<blocks_of((long long)p.nx * p.ny), kThreads, 0, st>>>(g, lam, gbar, p, q, pl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || q.nmark <= 0) return e;
    const int G = width * width <= 4 ? 4 : 16;
    const long long lanes = ((long long)q.nmark + 32 / G - 1) / (32 / G) * 32;
    switch (width) {
    case 2: adj_ib_kernel<2><<<blocks_of(lanes), kThreads, 0, st>>>(g, p, q, pl); break;
    case 3: adj_ib_kernel<3><<<blocks_of(lanes), kThreads, 0, st>>>(g, p, q, pl); break;
    case 4: adj_ib_kernel<4><<<blocks_of(lanes), kThreads, 0, st>>>(g, p, q, pl); break;
    default: return cudaErrorInvalidValue;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    adj_band_kernel<<<blocks_of((long long)q.nband * kSeg), kThreads, 0, st>>>(g, gbar, p, q, pl);
    return cudaGetLastError();
}

}  // namespace btdf
