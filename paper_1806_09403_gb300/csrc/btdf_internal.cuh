// btdf_internal.cuh - structures shared by the host side and the kernels of
// the BTDF-IB/LBM library (not part of the public C ABI).
#pragma once

#include <algorithm>
#include <cstdint>
#include <vector>
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

namespace btdf {

// One warp owns a run of kSeg consecutive nodes of one lattice row: 32 lanes
// x 4 nodes, so every population plane is read and written with 16-byte
// (FP32) or 8-byte (FP16/BF16) vectors.
constexpr int kSeg = 128;
constexpr int kNodesPerLane = 4;
constexpr int kThreads = 256;
// Threads per block of the register LBM kernels (npl nodes per lane, minb
// resident 256-thread blocks per SM): 128 with 16-bit storage (measured 5%
// faster on 8192 x 4096 FP16, equal at 1600 x 800) and for the FP32 kernel of
// 2 nodes per lane at 64 registers (2% faster at 1600 x 800); 256 for the
// other FP32 kernels (the 128-thread form of the 5-block kernel was 11% slower
// on 8192 x 4096).
__host__ __device__ constexpr int lbm_block_threads(int elem_bytes, int npl, int minb) {
    return (elem_bytes == 2 || (npl == 2 && minb == 4)) ? 128 : 256;
}

// D2Q9 velocities and weights (Eq. 8 and the weights stated below Eq. 7).
__host__ __device__ constexpr int ex(int a) {
    return (a == 1 || a == 5 || a == 8) ? 1 : ((a == 3 || a == 6 || a == 7) ? -1 : 0);
}
__host__ __device__ constexpr int ey(int a) {
    return (a == 2 || a == 5 || a == 6) ? 1 : ((a == 4 || a == 7 || a == 8) ? -1 : 0);
}
// e_a . (x, y), leaving out the zero components: IEEE arithmetic keeps a
// 0 * x term, so writing ex(a) * x + ey(a) * y costs an instruction per axis
// population for nothing.  The value is the same (one rounding of the exact
// sum for the diagonals).
__host__ __device__ constexpr float edot(int a, float x, float y) {
    return ex(a) == 0 ? (ey(a) == 0 ? 0.0f : (ey(a) > 0 ? y : -y))
                      : (ey(a) == 0 ? (ex(a) > 0 ? x : -x)
                                    : (ex(a) > 0 ? x : -x) + (ey(a) > 0 ? y : -y));
}
__host__ __device__ constexpr float wt(int a) {
    return a == 0 ? 4.0f / 9.0f : (a < 5 ? 1.0f / 9.0f : 1.0f / 36.0f);
}
// Population with the normal (y) component reversed: specular reflection.
__host__ __device__ constexpr int mirror_y(int a) {
    return a == 2 ? 4 : a == 4 ? 2 : a == 5 ? 8 : a == 8 ? 5 : a == 6 ? 7 : a == 7 ? 6 : a;
}
// Population with both components reversed: bounce-back.
__host__ __device__ constexpr int opposite(int a) {
    return a == 0 ? 0 : (a <= 4 ? ((a + 1) % 4) + 1 : ((a - 3) % 4) + 5);
}

enum : int { kBcxPeriodic = 0, kBcxInout = 1 };

// Index of outer node (x, y) in the perimeter order of the prescribed-velocity
// box: row 0 (x = 0..nx-1), row ny-1 (x = 0..nx-1), column 0 (y = 1..ny-2),
// column nx-1 (y = 1..ny-2); 2 nx + 2 (ny - 2) entries.
__host__ __device__ inline int perimeter_index(int x, int y, int nx, int ny) {
    if (y == 0) return x;
    if (y == ny - 1) return nx + x;
    if (x == 0) return 2 * nx + (y - 1);
    return 2 * nx + (ny - 2) + (y - 1);
}
enum : int { kBcyPeriodic = 0, kBcyFreeslip = 1, kBcyNoslip = 2 };
enum : int { kStoreF32 = 0, kStoreF16 = 1, kStoreBF16 = 2 };
// FP16 storage holds the deviations times 2^10 (see Io<__half>).
constexpr float kF16Scale = 1024.0f;
// Stored value of a unit deviation for a storage format.
inline double store_scale(int storage) { return storage == kStoreF16 ? (double)kF16Scale : 1.0; }

// Static per-marker data evaluated once on the host in FP64 (Eq. 14):
// support node coordinates (wrapped on periodic axes, clamped and given zero
// weight where a bounded axis cuts the support) and the 2-D weights
// w[j*S + i] = delta(x_i - X) delta(y_j - Y).
struct Marker {
    int xs[4];
    int ys[4];
    float w[16];
};

// Per-marker values the IB kernel needs besides the weights.  Velocities are
// stored relative to the reference velocity U_r (see LatticeParams):
// ub_rel = U_b - U_r * wsum, with wsum = sum of the marker's weights (1 unless
// a bounded lattice edge clips the support), both evaluated in FP64.
struct MarkerAux {
    float ubx_rel, uby_rel;
    float wsum;
    int body;
};

// One term of the node-centric spread (Eq. 15): the marker and its
// pre-multiplied weight delta*delta*drs*ds (dh = 1).
struct CsrEntry {
    int marker;
    float w;
};

struct LatticeParams {
    int nx, ny, nxp, nseg;
    long long plane;           // elements per population plane (nxp * ny)
    unsigned rs;               // elements between consecutive rows of one plane
    long long nwork;           // warp row segments of the LBM kernel
    // Warp-to-segment map of the register LBM kernels, set for each launch:
    // warp w starts at row w / nsegw, computed as (umulhi(w, wmul) + w) >> wshift,
    // and steps wdy rows plus wds segments per grid stride.
    unsigned wmul;
    int wshift, wdy, wds;
    unsigned poff[9];          // element offset of population plane a (row 0, x 0)
    int bcx, bcy;
    float omega;               // 1 / tau
    float one_m_omega;         // 1 - 1 / tau
    float guo;                 // 1 - 1 / (2 tau)
    float u_in;
    // Reference velocity U_r = (urx, ury): the buffers store
    // d_a = f_a - f_eq_a(1, U_r), so FP32 rounding scales with the departure
    // of the flow from the free stream rather than with the flow itself.
    float urx, ury;
    // Per-population constants of the collision in that form:
    //   c1 = 3 + 9 e.U_r,  k = 1 + P_a(U_r),  wom = w_a / tau,  wg = w_a (1 - 1/(2 tau)),
    // wom and wg times the storage scale (2^10 for FP16, else 1): the LBM
    // kernels collide the populations at their stored scale.
    float eur[9], c1[9], kr[9], wom[9], wg[9];
    // The same constants duplicated into pairs for the packed FP32x2
    // arithmetic of two nodes at once (c1, kr, wom), and 1 - 1/tau.
    float2 c1p[9], krp[9], womp[9];
    float2 omop;
    float gx, gy;              // uniform body force
    // Convective outlet (null: zero-gradient): the outlet column's
    // post-streaming deviations of the previous step, [9][ny], and the
    // weights of f(N, t+1) = old / (1 + U) + U / (1 + U) f(N-1, t+1).
    float* outlet;
    float uc_old, uc_new;
    // Prescribed-velocity box (null: none): every outer node gets the
    // velocity box[perimeter_index(x, y)] by non-equilibrium extrapolation
    // from its nearest interior node.
    const float2* box;
    const int* seg_index;      // [ny * nseg] band segment id or -1 (null: no band)
    const int* seg_ptr;        // [nband * (kSeg + 1)] CSR row pointers per node
    const CsrEntry* csr;
    const float2* F;           // Lagrangian forces of the step (sum of passes)
    unsigned long long* step;  // device step counter, advanced by the LBM kernel
    // Register variants: prefetch into L2 the row segment this many units
    // ahead (about half a wave of resident warps later; 0: off).
    int pf_ahead;
    int* status;               // sticky device status bits
    // Polls before a TMA stage wait gives up (< 0: the default bound of about
    // a second); set by btdf_set_wait_limit to exercise the timeout path.
    int wait_polls;
    // Tile tickets of the warp-specialized TMA kernel: [0] next tile, [1]
    // CTAs finished; both zero between launches (null: kernel unavailable).
    unsigned* sched;
    // Force on each body (Eq. 27), reduced in FP64 by block 0 of the LBM kernel.
    int nbody;
    int hist_len;
    const int* body_ptr;       // [nbody + 1] marker ranges
    const double* body_scale;  // ds * drs per body
    double2* hist;             // [hist_len * nbody]
};

struct IbParams {
    int nmark;
    const Marker* mk;
    const MarkerAux* aux;
    const float2* F_prev;      // forces accumulated by earlier passes (null on pass 1)
    float2* F_out;             // F_prev + this pass's increment
    float2* Us;                // D_I u* of pass 1 (diagnostic)
    float* rhol;               // D_I rho (diagnostic)
    int first_pass;
    int* status;               // sticky device status bits
};

enum : int { kStatusUnstable = 1, kStatusTimeout = 2 };

// Batched LBM launch: many lattices, one persistent grid.
struct BatchLbm {
    const LatticeParams* descs;             // per lattice
    const unsigned long long* case_off;     // element offset of each lattice's populations
    const int2* units;                      // (lattice, first row) of each 8-row block
    const int* cta_units;                   // [grid + 1] first unit of each CTA
    int nbody;
    int hist_len;
    const int* body_rng;                    // [2 * nbody] first and end flat marker index
    const double* body_scale;               // ds * drs per body
    double2* hist;                          // [hist_len * nbody]
    const float2* F;                        // Lagrangian forces of the step
    unsigned long long* step;               // step counter, advanced by the last CTA
    unsigned int* done;                     // CTAs finished this launch, reset by the last
};

// Launchers implemented in btdf_kernels.cu.
// variant: one of the register variants below (the software-pipelined ones
// fall back to their plain form for an in-place step); grid: upper bound on
// the blocks; pdl: launch as a programmatic dependent of the preceding IB
// kernel (its non-band work overlaps the IB stage).
cudaError_t launch_collide_stream(int storage, bool pull, int variant, const void* gin, void* gout,
                                  const LatticeParams& p, int grid, bool pdl, cudaStream_t st);
int collide_stream_blocks_per_sm(int storage, bool pull, int variant);
// Threads per block of a collide-stream variant for a storage format.
int collide_stream_block_threads(int storage, int variant);

// Kernel variants of the LBM step (btdf_tune): register-pipelined warps with
// 4 or 2 nodes per lane, or TMA-tiled CTAs (tile rows x pipeline stages).
enum : int {
    kVarAuto = 0,
    kVarReg4 = 1,
    kVarReg2 = 2,
    kVarTma8x2 = 3,
    kVarTma8x3 = 4,
    kVarTma16x2 = 5,
    kVarReg4Pf = 6,
    kVarReg2Pf = 7,
    kVarReg1 = 8,      // 1 node per lane, 6 blocks per SM (<= 40 registers)
    kVarReg2Occ = 9,   // 2 nodes per lane, 5 blocks per SM (<= 48 registers)
    kVarReg2OccPf = 10, // as 9, each warp also prefetches a later row segment into L2
    kVarReg4L2Pf = 11, // as 1, with the L2 prefetch of 10
    kVarTmaWs8x2 = 12, // TMA tiles of 8 rows, a producer warp, 2 stages, <= 72 registers
    kVarTmaWs7x3 = 13, // TMA tiles of 7 rows, a producer warp, 3 stages, <= 80 registers
    kVarCount = 14
};
// map: 3-D tensor map (x, y, population) of the input buffer with box
// (128 + 2 * tma_halo(storage), tma_box_rows(variant), 9).
cudaError_t launch_collide_stream_tma(int storage, int variant, const CUtensorMap* map, const void* gin,
                                      void* gout, const LatticeParams& p, int grid, bool pdl,
                                      cudaStream_t st);
int collide_stream_tma_blocks_per_sm(int storage, int variant);
cudaError_t launch_collide_stream_batch(int storage, bool pull, int npl, const void* gin, void* gout,
                                        const BatchLbm& b, int grid, bool pdl, cudaStream_t st);
int collide_stream_batch_blocks_per_sm(int storage, int npl);
cudaError_t launch_ib_force_batch(int storage, bool pull, int width, const void* g,
                                  const LatticeParams* descs, const unsigned long long* case_off,
                                  const IbParams& q, cudaStream_t st);
int tma_box_rows(int variant);
int tma_halo(int storage);

// Statistic of the autotuners: the mean of the middle half of the per-step
// times (all of them below four).  CUDA event times come in steps of about a
// microsecond on this hardware, so the median of a few dozen steps ties
// variants that differ by less; the mean resolves below that step, and
// dropping the outer quarters keeps it robust to outliers.
inline float interquartile_mean(std::vector<float> t) {
    std::sort(t.begin(), t.end());
    const size_t n = t.size(), lo = n >= 4 ? n / 4 : 0, hi = n >= 4 ? n - n / 4 : n;
    double s = 0.0;
    for (size_t i = lo; i < hi; i++) s += t[i];
    return hi > lo ? (float)(s / (double)(hi - lo)) : 0.0f;
}
// pdl: launch as a programmatic dependent of the preceding kernel (the IB
// kernel loads its marker tables, then waits for that kernel's results).
cudaError_t launch_ib_force(int storage, bool pull, int width, const void* g,
                            const LatticeParams& p, const IbParams& q, bool pdl, cudaStream_t st);
cudaError_t launch_init_equilibrium(int storage, void* g, const LatticeParams& p,
                                    const double* rho, const double* ux, const double* uy,
                                    cudaStream_t st);
cudaError_t launch_read_field(int storage, bool pull, const void* g, const LatticeParams& p,
                              int kind, float* dst, cudaStream_t st);

// Evicts the L2 cache before a timed launch (btdf_api.cu): writes `bytes`
// of `buf`, then reads them back so the lines left behind are clean.
cudaError_t launch_l2_flush(void* buf, size_t bytes, cudaStream_t st);
// Bytes of scratch that evict the whole L2 of the current device.
size_t l2_flush_bytes();

// ---- discrete adjoint ----

// Per-marker 1-D weights and their derivatives with respect to the marker
// position: W = wx[i] wy[j], dW/dX = dwx[i] wy[j], dW/dY = wx[i] dwy[j].
struct AdjMarker {
    float wx[4], wy[4], dwx[4], dwy[4];
};

struct AdjParams {
    int nmark, nband;
    const Marker* mk;
    const MarkerAux* aux;
    const AdjMarker* am;
    const float* cscale;       // drs * ds of each marker's body
    const int* band_keys;      // [nband] y * nseg + segment
    float* fbar_band;          // [nband * kSeg * 9] dJ/df parked at band nodes
    float2* Fbar_band;         // [nband * kSeg] dJ/dF (node force) at band nodes
    float4* mbar;              // [nmark] (dJ/drho_l, dJ/dU*_l)
    const float2* objw;        // [nmark] explicit dJ/dF_l of the objective
    double* dJdX;              // [nmark] accumulated over the window
    double* dJdY;
    double* dU;                // inlet part of dJ/dU_in
};

// Launcher implemented in btdf_adjoint.cu: g = g^n (pull: post-collision,
// else post-streaming), lam = dJ/dg^{n+1}, gbar = dJ/dg^n (zeroed by the
// caller); p.F must hold the Lagrangian forces F^n of the step.
cudaError_t launch_adjoint_step(const float* g, const float* lam, float* gbar, const LatticeParams& p,
                                const AdjParams& q, int width, bool pull, cudaStream_t st);

// ---- host-side static tables (btdf_tables.cu) ----

// One rigid body as seen by the table builder; tag goes to MarkerAux.body.
struct BodyDesc {
    int n;
    double ds, drs;
    const double *X, *Y, *Ubx, *Uby;   // velocities may be null (at rest)
    int tag;
};

struct HostTables {
    std::vector<Marker> mk;
    std::vector<MarkerAux> aux;
    std::vector<double> wsum;          // FP64 sum of each marker's weights
    std::vector<int> seg_index;        // [ny * nseg]
    std::vector<long long> seg_keys;   // y * nseg + segment, ascending
    std::vector<int> seg_ptr;          // [nband * (kSeg + 1)]
    std::vector<CsrEntry> csr;         // marker indices offset by marker_base
};

double delta_fn(int kind, double r);
double delta_deriv(int kind, double r);
void build_adjoint_markers(int nx, int ny, int delta, int width, bool px, bool py,
                           const std::vector<BodyDesc>& bodies, std::vector<AdjMarker>& out);
void build_marker_tables(int nx, int ny, int nseg, int delta, int width, bool px, bool py,
                         double u_in, const std::vector<BodyDesc>& bodies, int marker_base,
                         HostTables& t);

}  // namespace btdf
