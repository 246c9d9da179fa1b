// btdf_api.cu - host side of the C ABI declared in include/btdf.h.
//
// Holds the context, validates configurations, evaluates the static marker
// weights in FP64 (Eq. 14 with the delta functions of Eqs. 37-39), builds the
// node-centric spreading table (Eq. 15), orders the kernels of a time step
// (Algorithm 1) and replays them through CUDA graphs.
#include "btdf.h"
#include "btdf_internal.cuh"

#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

static_assert(btdf::kVarCount == BTDF_VARIANT_COUNT, "variant count of the C ABI");

namespace btdf {
namespace {

__global__ void l2_read_kernel(const float4* __restrict__ buf, size_t n, float* __restrict__ sink) {
    float acc = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float4 v = buf[i];
        acc += (v.x + v.y) + (v.z + v.w);
    }
    if (acc != 0.f) sink[0] = acc;   // the buffer is zero: never taken, keeps the loads live
}

}  // namespace

cudaError_t launch_l2_flush(void* buf, size_t bytes, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(buf, 0, bytes, st);
    if (e != cudaSuccess) return e;
    const size_t n = bytes / sizeof(float4) - 1;   // the last float4 is the sink
    l2_read_kernel<<<1024, kThreads, 0, st>>>((const float4*)buf, n, (float*)buf + 4 * n);
    return cudaGetLastError();
}

// Immersed-boundary force density of the step whose Lagrangian forces
// p.F holds (Eq. 15): the same node-centric gather the LBM kernel applies.
__global__ void force_field_kernel(LatticeParams p, int comp, float* __restrict__ dst) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (long long)p.nx * p.ny) return;
    const int y = (int)(n / p.nx), x = (int)(n - (long long)y * p.nx);
    float f = 0.0f;
    if (p.seg_index != nullptr) {
        const int seg = p.seg_index[y * p.nseg + x / kSeg];
        if (seg >= 0) {
            const int* ptr = p.seg_ptr + (long long)seg * (kSeg + 1) + (x % kSeg);
            for (int k = ptr[0]; k < ptr[1]; k++) {
                const CsrEntry c = p.csr[k];
                const float2 F = p.F[c.marker];
                f = __fmaf_rn(c.w, comp == 0 ? F.x : F.y, f);
            }
        }
    }
    dst[n] = f;
}

cudaError_t launch_force_field(const LatticeParams& p, int comp, float* dst, cudaStream_t st) {
    const long long nn = (long long)p.nx * p.ny;
    force_field_kernel<<<(unsigned)((nn + kThreads - 1) / kThreads), kThreads, 0, st>>>(p, comp, dst);
    return cudaGetLastError();
}

size_t l2_flush_bytes() {
    int dev = 0, l2 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess)
        l2 = 128 << 20;
    return (size_t)std::max(l2, 1 << 20) * 4;
}

}  // namespace btdf

using namespace btdf;

namespace {

constexpr int kGraphSteps = 64;          // steps per replayed CUDA graph (even)
constexpr int kFullGrid = 1 << 30;       // grid cap meaning "one row segment per warp"
constexpr int kStageSlots = 4;           // pinned staging slots for marker velocities
constexpr uint64_t kStateMagic = 0x3230465444544242ull;   // "BBTDTF02"

struct Body {
    int first = 0, n = 0;
    double ds = 0.0, drs = 0.0;
    std::vector<double> X, Y, Ubx, Uby;
    std::vector<double> wsum;      // sum of each marker's weights (filled by rebuild)
};

// Checkpoint header (48 bytes).  u_ref is the reference velocity the stored
// deviations are relative to (the creation-time u_in of the context).
struct StateHeader {
    uint64_t magic;
    int32_t nx, ny, nxp, storage;
    int32_t poststream, layout;
    int64_t steps;
    double u_ref;
};
static_assert(sizeof(StateHeader) == 48, "checkpoint header layout");

int support_width(int kind) { return kind == 2 ? 2 : kind == 3 ? 3 : (kind == 4 || kind == 5) ? 4 : 0; }

// Solid-shell thickness drs/dh suggested in Sec. 4.4 (the cosine kernel has
// the 4-point support and takes the 4-point value).
double paper_drs(int kind) { return kind == 2 ? 1.4 : kind == 3 ? 1.9 : 2.6; }

size_t elem_bytes(int storage) { return storage == kStoreF32 ? 4 : 2; }

// Device buffers and bookkeeping of one adjoint window (btdf_adjoint_*).
struct AdjointTape {
    bool pending = false;        // a forward window whose checkpoints are valid
    bool post0 = false;          // the window starts from post-streaming populations
    int64_t nsteps = 0;
    int every = 0, nck = 0;      // checkpoint spacing and count
    int body = -1;
    double dref = 0.0, J = 0.0;
    size_t state_elems = 0;      // floats per state
    float* ck = nullptr;         // [nck] states g^{j every}
    float* seg = nullptr;        // [every] states of the segment being reversed
    float* lam[2] = {nullptr, nullptr};
    float2* Fall = nullptr;      // [nsteps * nmark] Lagrangian forces of every step
    float2* Us = nullptr;        // IB diagnostics of the recomputed steps (unused)
    float* rhol = nullptr;
    AdjMarker* am = nullptr;
    float* cscale = nullptr;
    float2* objw = nullptr;
    int* band_keys = nullptr;
    float* fbar_band = nullptr;
    float2* Fbar_band = nullptr;
    float4* mbar = nullptr;
    double* acc = nullptr;       // [2 nmark + 1]: dJ/dX, dJ/dY, inlet part of dJ/dU
    size_t bytes = 0;
    long long gen = 0;           // bumped whenever the buffers are reallocated
    // The window's forward pass and its reverse sweep as CUDA graphs, valid
    // while `key` (window shape, buffers, markers, inflow) is unchanged.
    cudaGraphExec_t fwd = nullptr, bwd = nullptr;
    std::vector<double> fwd_key, bwd_key;
    int cap_ck = 0, cap_every = 0;
    int64_t cap_F = 0;
    int cap_mark = 0, cap_band = 0;
};

}  // namespace

struct btdf_ctx {
    btdf_config cfg{};
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    int nxp = 0, nseg = 0, width = 0;
    long long plane = 0;
    size_t elem = 4;
    void* g[2] = {nullptr, nullptr};
    int cur = 0;
    bool poststream = true;
    bool has_fields = false;
    int64_t steps = 0;
    int64_t hist_from = 0;

    std::vector<Body> bodies;
    int nmark = 0, nband = 0;
    // All marker data below (tables, forces, diagnostics, body tables,
    // spreading table, force history) are carved from one device arena.
    void* d_arena = nullptr;
    Marker* d_mk = nullptr;
    MarkerAux* d_aux = nullptr;
    float2* d_F[2] = {nullptr, nullptr};
    float2* d_Us = nullptr;
    float* d_rhol = nullptr;
    int* d_seg_index = nullptr;
    int* d_seg_ptr = nullptr;
    CsrEntry* d_csr = nullptr;
    int* d_body_ptr = nullptr;
    double* d_body_scale = nullptr;
    double2* d_hist = nullptr;
    unsigned long long* d_step = nullptr;
    int* d_status = nullptr;
    unsigned* d_sched = nullptr;         // tile tickets of the warp-specialized TMA kernel
    float* d_outlet = nullptr;         // [9][ny] previous outlet column (convective outlet)
    float2* d_box = nullptr;           // perimeter velocities of the prescribed-velocity box
    std::vector<MarkerAux> aux_host;
    // Pinned host staging, so per-step host <-> device copies are true DMA
    // transfers and a step's inputs and outputs need one synchronization.
    // kStageSlots x [nmark] marker velocities on their way to the device;
    // slot k is reused once its upload (aux_ev[k]) has run, so the host can
    // prepare a few steps ahead of the device.
    MarkerAux* aux_pin = nullptr;
    cudaEvent_t aux_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    int aux_slot = 0;
    int* status_pin = nullptr;         // device status word
    void* pin = nullptr;               // force-history read-back
    size_t pin_cap = 0;

    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    long long pf_grid[2] = {1, 1};                 // software-pipelined kernel [npl 4/2]
    long long pf_units[2][2] = {};                 // L2 prefetch distance of variants 10, 11 [local/pull]
    long long tma_grid[kVarCount] = {};  // persistent grid of each TMA variant
    int variant = kVarAuto;              // LBM kernel variant (btdf_tune)
    int grid_override = 0;               // 0: SMs x resident blocks
    bool tma_ok = false;                 // tensor maps encoded
    CUtensorMap tmap[2][3];              // [buffer][box of 10 / 18 / 9 rows]

    bool prof = false;
    std::vector<cudaEvent_t> ev;         // 3 per profiled step
    size_t ev_used = 0;

    size_t dev_bytes = 0;
    size_t marker_bytes = 0;           // part of dev_bytes held by marker data
    std::string err;

    // Reference velocity U_r = (u_ref, 0) of the stored deviations: the
    // creation-time inflow speed; btdf_set_inflow changes only cfg.u_in.
    double u_ref = 0.0;
    std::vector<int> band_keys;        // y * nseg + segment of each band segment
    long long marker_gen = 0;          // bumped by every rebuild of the marker tables
    AdjointTape tape;
    double2* tune_hist = nullptr;      // one-slot force ring used while btdf_autotune times steps
    int wait_polls = -1;               // btdf_set_wait_limit (< 0: default bound)
};

namespace {

int fail(btdf_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_fail(btdf_ctx* c, cudaError_t e, const char* where) {
    return fail(c, BTDF_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);   \
    } while (0)

template <typename P>
cudaError_t dalloc(btdf_ctx* ctx, P** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e == cudaSuccess) ctx->dev_bytes += bytes;
    else cudaGetLastError();   // allocation errors are not sticky; clear them
    return e;
}

template <typename P>
void dfree(btdf_ctx* ctx, P*& p) {
    (void)ctx;
    if (p) cudaFree((void*)p);
    p = nullptr;
}

void drop_graphs(btdf_ctx* ctx) {
    for (auto& g : ctx->gexec)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

void free_markers(btdf_ctx* ctx) {
    for (cudaEvent_t e : ctx->aux_ev)
        if (e) cudaEventSynchronize(e);
    if (ctx->aux_pin) cudaFreeHost(ctx->aux_pin);
    ctx->aux_pin = nullptr;
    ctx->dev_bytes -= ctx->marker_bytes;
    ctx->marker_bytes = 0;
    dfree(ctx, ctx->d_arena);
    ctx->d_mk = nullptr;
    ctx->d_aux = nullptr;
    ctx->d_F[0] = ctx->d_F[1] = nullptr;
    ctx->d_Us = nullptr;
    ctx->d_rhol = nullptr;
    ctx->d_seg_index = nullptr;
    ctx->d_seg_ptr = nullptr;
    ctx->d_csr = nullptr;
    ctx->d_body_ptr = nullptr;
    ctx->d_body_scale = nullptr;
    ctx->d_hist = nullptr;
}

// Sub-buffers of one device allocation, each 256-byte aligned.
struct Arena {
    size_t size = 0;
    template <typename P>
    size_t take(size_t bytes) {
        const size_t off = size;
        size = (size + bytes + 255) / 256 * 256;
        return off;
    }
};

void free_tape(btdf_ctx* ctx) {
    AdjointTape& T = ctx->tape;
    if (T.fwd) cudaGraphExecDestroy(T.fwd);
    if (T.bwd) cudaGraphExecDestroy(T.bwd);
    const long long gen = T.gen;
    dfree(ctx, T.ck);
    dfree(ctx, T.seg);
    dfree(ctx, T.lam[0]);
    dfree(ctx, T.lam[1]);
    dfree(ctx, T.Fall);
    dfree(ctx, T.Us);
    dfree(ctx, T.rhol);
    dfree(ctx, T.am);
    dfree(ctx, T.cscale);
    dfree(ctx, T.objw);
    dfree(ctx, T.band_keys);
    dfree(ctx, T.fbar_band);
    dfree(ctx, T.Fbar_band);
    dfree(ctx, T.mbar);
    dfree(ctx, T.acc);
    ctx->dev_bytes -= T.bytes;
    T = AdjointTape{};
    T.gen = gen + 1;
}

bool is_tma(int v) {
    return v == kVarTma8x2 || v == kVarTma8x3 || v == kVarTma16x2 || v == kVarTmaWs8x2 || v == kVarTmaWs7x3;
}

// Variant 0 (automatic): the autotuner's usual picks on a GB300 with the L2
// flushed per step.  From 2^23 nodes up the lattice streams from DRAM: the
// prefetching 4-node kernel for FP32 (0.342 against 0.36-0.40 ms for variant
// 2 on 8192 x 4096) and the warp-specialized TMA kernel for 16-bit storage
// (0.220 against 0.260 ms).  Below, the step is latency-bound and the
// register kernels with one row segment per warp win (variant 12 takes 25
// against 20 us on 1600 x 800).
int auto_variant(const btdf_ctx* ctx) {
    const bool big = (long long)ctx->cfg.nx * ctx->cfg.ny >= (1LL << 23);
    if (ctx->cfg.storage == kStoreF32) return big ? kVarReg4L2Pf : kVarReg2;
    return big && ctx->tma_ok ? kVarTmaWs8x2 : kVarReg4L2Pf;
}

// Tensor map of a TMA variant: boxes of 10, 18 and 9 rows.
int tmap_index(int v) { return v == kVarTma16x2 ? 1 : v == kVarTmaWs7x3 ? 2 : 0; }

LatticeParams lattice_params(const btdf_ctx* ctx) {
    LatticeParams p{};
    p.nx = ctx->cfg.nx;
    p.ny = ctx->cfg.ny;
    p.nxp = ctx->nxp;
    p.nseg = ctx->nseg;
    p.plane = ctx->plane;
    // the convective outlet is the in/out channel plus an outlet column buffer
    // the box overrides every outer node; its raw pulls wrap like a periodic lattice
    const bool box = ctx->cfg.bc_x == BTDF_BCX_BOX;
    p.bcx = box ? kBcxPeriodic : ctx->cfg.bc_x == BTDF_BCX_CONVECTIVE ? kBcxInout : ctx->cfg.bc_x;
    p.bcy = box ? kBcyPeriodic : ctx->cfg.bc_y;
    p.box = ctx->d_box;
    p.outlet = ctx->d_outlet;
    p.uc_old = (float)(1.0 / (1.0 + ctx->cfg.u_in));
    p.uc_new = (float)(ctx->cfg.u_in / (1.0 + ctx->cfg.u_in));
    p.omega = (float)(1.0 / ctx->cfg.tau);
    p.guo = (float)(1.0 - 0.5 / ctx->cfg.tau);
    p.u_in = (float)ctx->cfg.u_in;
    p.urx = (float)ctx->u_ref;   // reference velocity of the stored deviations
    p.ury = 0.0f;
    {
        const double tau = ctx->cfg.tau, Ux = ctx->u_ref, Uy = 0.0;
        p.one_m_omega = (float)(1.0 - 1.0 / tau);
        for (int a = 0; a < 9; a++) {
            const double w = a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
            const double eU = ex(a) * Ux + ey(a) * Uy;
            p.eur[a] = (float)eU;
            p.c1[a] = (float)(3.0 + 9.0 * eU);
            p.kr[a] = (float)(1.0 + 3.0 * eU + 4.5 * eU * eU - 1.5 * (Ux * Ux + Uy * Uy));
            p.wom[a] = (float)(w / tau * store_scale(ctx->cfg.storage));
            p.wg[a] = (float)(w * (1.0 - 0.5 / tau) * store_scale(ctx->cfg.storage));
        }
        for (int a = 0; a < 9; a++) {
            p.c1p[a] = make_float2(p.c1[a], p.c1[a]);
            p.krp[a] = make_float2(p.kr[a], p.kr[a]);
            p.womp[a] = make_float2(p.wom[a], p.wom[a]);
        }
        p.omop = make_float2(p.one_m_omega, p.one_m_omega);
    }
    p.nwork = (long long)ctx->cfg.ny * ctx->nseg;
    // planar: [9][ny][nxp]; row-interleaved: [ny][9][nxp]
    p.rs = ctx->cfg.layout == BTDF_LAYOUT_ROWS ? 9u * (unsigned)ctx->nxp : (unsigned)ctx->nxp;
    for (int a = 0; a < 9; a++)
        p.poff[a] = ctx->cfg.layout == BTDF_LAYOUT_ROWS ? (unsigned)(a * ctx->nxp) : (unsigned)(a * ctx->plane);
    p.gx = (float)ctx->cfg.gx;
    p.gy = (float)ctx->cfg.gy;
    p.seg_index = ctx->nmark > 0 ? ctx->d_seg_index : nullptr;
    p.seg_ptr = ctx->d_seg_ptr;
    p.csr = ctx->d_csr;
    p.F = ctx->d_F[(ctx->cfg.nf - 1) % 2];
    p.step = ctx->d_step;
    p.status = ctx->d_status;
    p.wait_polls = ctx->wait_polls;
    p.sched = ctx->d_sched;
    p.nbody = ctx->nmark > 0 ? (int)ctx->bodies.size() : 0;
    p.hist_len = ctx->cfg.history_len;
    p.body_ptr = ctx->d_body_ptr;
    p.body_scale = ctx->d_body_scale;
    p.hist = ctx->d_hist;
    if (ctx->tune_hist) {   // timing steps must not overwrite the force history
        p.hist_len = 1;
        p.hist = ctx->tune_hist;
    }
    return p;
}

cudaEvent_t next_event(btdf_ctx* ctx) {
    if (ctx->ev_used == ctx->ev.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        ctx->ev.push_back(e);
    }
    return ctx->ev[ctx->ev_used++];
}

// Issues the kernels of one time step reading buffer `cur` (Algorithm 1).
int enqueue_step(btdf_ctx* ctx, cudaStream_t st, bool pull, int cur, bool prof) {
    const LatticeParams p = lattice_params(ctx);
    cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
    if (prof) {
        e0 = next_event(ctx);
        e1 = next_event(ctx);
        e2 = next_event(ctx);
        if (!e0 || !e1 || !e2) return fail(ctx, BTDF_ECUDA, "cudaEventCreate failed");
        CK(cudaEventRecord(e0, st));
    }
    if (ctx->nmark > 0) {
        for (int k = 1; k <= ctx->cfg.nf; k++) {
            IbParams q{};
            q.nmark = ctx->nmark;
            q.mk = ctx->d_mk;
            q.aux = ctx->d_aux;
            q.F_prev = k == 1 ? nullptr : ctx->d_F[(k - 2) % 2];
            q.F_out = ctx->d_F[(k - 1) % 2];
            q.Us = ctx->d_Us;
            q.rhol = ctx->d_rhol;
            q.first_pass = k == 1;
            q.status = ctx->d_status;
            // Without profiling events in between, each IB pass is a
            // programmatic dependent of the kernel before it: it loads its
            // marker tables while that kernel drains, then waits for it.
            CK(launch_ib_force(ctx->cfg.storage, pull, ctx->width, ctx->g[cur], p, q, !prof, st));
        }
    }
    if (prof) CK(cudaEventRecord(e1, st));
    // Without profiling events in between, the LBM kernel is a programmatic
    // dependent of the IB kernel: its band nodes wait for the forces, the rest
    // of the lattice overlaps the IB stage.
    const bool pdl = ctx->nmark > 0 && !prof;
    int v = ctx->variant == kVarAuto ? auto_variant(ctx) : ctx->variant;
    if (is_tma(v) && (!pull || !ctx->tma_ok)) v = kVarReg4;   // TMA kernel pulls only
    // the box's first and last rows are rebuilt in the register kernels only
    if (ctx->d_box && (is_tma(v) || v == kVarReg4Pf || v == kVarReg2Pf)) v = kVarReg4;
    if (is_tma(v)) {
        const int grid = ctx->grid_override > 0 ? ctx->grid_override : (int)ctx->tma_grid[v];
        CK(launch_collide_stream_tma(ctx->cfg.storage, v, &ctx->tmap[cur][tmap_index(v)],
                                     ctx->g[cur], ctx->g[1 - cur], p, grid, pdl, st));
    } else {
        // Register variants.  Default grid: one row segment per warp.  SMs
        // stream at different rates (per-SM busy time spreads by +-20% at
        // equal work), and a grid the block scheduler hands out as SMs free
        // up balances them; measured 0.39 ms against 0.53 ms per step of the
        // persistent grid on an 8192 x 4096 lattice.  The software-pipelined
        // variants are persistent by design.
        const bool pf = (v == kVarReg4Pf || v == kVarReg2Pf) && pull;
        const int grid = ctx->grid_override > 0 ? ctx->grid_override
                         : pf                   ? (int)ctx->pf_grid[v == kVarReg2Pf ? 1 : 0]
                                                : kFullGrid;
        LatticeParams q = p;
        if (v == kVarReg2OccPf || v == kVarReg4L2Pf)
            q.pf_ahead = (int)ctx->pf_units[v == kVarReg4L2Pf ? 1 : 0][pull ? 1 : 0];
        CK(launch_collide_stream(ctx->cfg.storage, pull, v, ctx->g[cur], ctx->g[1 - cur], q, grid, pdl, st));
    }
    if (prof) CK(cudaEventRecord(e2, st));
    return BTDF_OK;
}

int ensure_graph(btdf_ctx* ctx, int cur) {
    if (ctx->gexec[cur]) return BTDF_OK;
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
    int rc = BTDF_OK;
    int c = cur;
    for (int i = 0; i < kGraphSteps && rc == BTDF_OK; i++) {
        rc = enqueue_step(ctx, ctx->cap, true, c, false);
        c = 1 - c;
    }
    cudaError_t e = cudaStreamEndCapture(ctx->cap, &graph);
    if (rc != BTDF_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&ctx->gexec[cur], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
    return BTDF_OK;
}

// 3-D tensor maps (x, y, population) of both population buffers for the
// TMA-tiled LBM kernel.  Failure leaves the register-pipelined kernels in use.
bool encode_tensor_maps(btdf_ctx* ctx) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || fn == nullptr) {
        cudaGetLastError();
        return false;
    }
    auto encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    const CUtensorMapDataType dt = ctx->cfg.storage == kStoreF32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : ctx->cfg.storage == kStoreF16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                                   : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint64_t dims[3] = {(cuuint64_t)ctx->nxp, (cuuint64_t)ctx->cfg.ny, 9};
    const bool interleaved = ctx->cfg.layout == BTDF_LAYOUT_ROWS;
    const cuuint64_t strides[2] = {(cuuint64_t)ctx->nxp * ctx->elem * (interleaved ? 9 : 1),
                                   (cuuint64_t)(interleaved ? ctx->nxp : ctx->plane) * ctx->elem};
    const cuuint32_t estr[3] = {1, 1, 1};
    const int rows[3] = {tma_box_rows(kVarTma8x2), tma_box_rows(kVarTma16x2), tma_box_rows(kVarTmaWs7x3)};
    for (int b = 0; b < 2; b++)
        for (int r = 0; r < 3; r++) {
            const cuuint32_t box[3] = {(cuuint32_t)(kSeg + 2 * tma_halo(ctx->cfg.storage)),
                                       (cuuint32_t)rows[r], 9};
            if (encode(&ctx->tmap[b][r], dt, 3, ctx->g[b], dims, strides, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
                CUDA_SUCCESS)
                return false;
        }
    return true;
}

int read_status(btdf_ctx* ctx) {
    CK(cudaMemcpyAsync(ctx->status_pin, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const int st = *ctx->status_pin;
    if (st & kStatusTimeout) return fail(ctx, BTDF_ETIMEOUT, "a bounded device wait gave up");
    if (st & kStatusUnstable)
        return fail(ctx, BTDF_EUNSTABLE, "non-positive or non-finite density or force at a marker");
    return BTDF_OK;
}

// Static marker data and the node-centric spreading table (Eqs. 14, 15).
int rebuild_markers(btdf_ctx* ctx) {
    drop_graphs(ctx);
    ctx->marker_gen++;
    ctx->tape.pending = false;
    ctx->band_keys.clear();
    free_markers(ctx);
    const int nx = ctx->cfg.nx, ny = ctx->cfg.ny;
    const bool px = ctx->cfg.bc_x == kBcxPeriodic, py = ctx->cfg.bc_y == kBcyPeriodic;
    const int nm = ctx->nmark, nb = (int)ctx->bodies.size();
    (void)nx;
    if (nm == 0) return BTDF_OK;
    std::vector<BodyDesc> descs;
    std::vector<int> body_ptr(nb + 1);
    std::vector<double> scale(nb);
    for (int b = 0; b < nb; b++) {
        const Body& B = ctx->bodies[b];
        descs.push_back(BodyDesc{B.n, B.ds, B.drs, B.X.data(), B.Y.data(), B.Ubx.data(),
                                 B.Uby.data(), b});
        body_ptr[b] = B.first;
        body_ptr[b + 1] = B.first + B.n;
        scale[b] = B.ds * B.drs;
    }
    HostTables t;
    build_marker_tables(ctx->cfg.nx, ctx->cfg.ny, ctx->nseg, ctx->cfg.delta, ctx->width, px, py,
                        ctx->u_ref, descs, 0, t);
    ctx->band_keys.assign(t.seg_keys.begin(), t.seg_keys.end());
    for (int b = 0; b < nb; b++) {
        Body& B = ctx->bodies[b];
        B.wsum.assign(t.wsum.begin() + B.first, t.wsum.begin() + B.first + B.n);
    }
    ctx->aux_host = t.aux;
    CK(cudaMallocHost((void**)&ctx->aux_pin, sizeof(MarkerAux) * nm * kStageSlots));
    ctx->nband = (int)t.seg_keys.size();
    const std::vector<Marker>& mk = t.mk;
    const std::vector<int>& seg_index = t.seg_index;
    const std::vector<int>& seg_ptr = t.seg_ptr;
    const std::vector<CsrEntry>& csr = t.csr;
    const size_t nseg_all = (size_t)ny * ctx->nseg;
    const size_t bytes_before = ctx->dev_bytes;
    // One allocation: the tables every IB launch and the body-force
    // reduction touch come first, so a step's small reads and writes fall
    // in one or two pages (one address translation each) instead of a
    // dozen separate allocations; the spreading table and the history follow.
    Arena A;
    const size_t o_mk = A.take<Marker>(sizeof(Marker) * nm);
    const size_t o_aux = A.take<MarkerAux>(sizeof(MarkerAux) * nm);
    const size_t o_F0 = A.take<float2>(sizeof(float2) * nm);
    const size_t o_F1 = A.take<float2>(sizeof(float2) * nm);
    const size_t o_Us = A.take<float2>(sizeof(float2) * nm);
    const size_t o_rhol = A.take<float>(sizeof(float) * nm);
    const size_t o_bptr = A.take<int>(sizeof(int) * (nb + 1));
    const size_t o_bsc = A.take<double>(sizeof(double) * nb);
    const size_t o_segi = A.take<int>(sizeof(int) * nseg_all);
    const size_t o_segp = A.take<int>(sizeof(int) * std::max<size_t>(seg_ptr.size(), 1));
    const size_t o_csr = A.take<CsrEntry>(sizeof(CsrEntry) * std::max<size_t>(csr.size(), 1));
    const size_t o_hist = A.take<double2>(sizeof(double2) * (size_t)ctx->cfg.history_len * nb);
    CK(dalloc(ctx, &ctx->d_arena, A.size));
    char* base = (char*)ctx->d_arena;
    ctx->d_mk = (Marker*)(base + o_mk);
    ctx->d_aux = (MarkerAux*)(base + o_aux);
    ctx->d_F[0] = (float2*)(base + o_F0);
    ctx->d_F[1] = (float2*)(base + o_F1);
    ctx->d_Us = (float2*)(base + o_Us);
    ctx->d_rhol = (float*)(base + o_rhol);
    ctx->d_body_ptr = (int*)(base + o_bptr);
    ctx->d_body_scale = (double*)(base + o_bsc);
    ctx->d_seg_index = (int*)(base + o_segi);
    ctx->d_seg_ptr = (int*)(base + o_segp);
    ctx->d_csr = (CsrEntry*)(base + o_csr);
    ctx->d_hist = (double2*)(base + o_hist);
    cudaStream_t st = ctx->stream;
    CK(cudaMemcpyAsync(ctx->d_mk, mk.data(), sizeof(Marker) * nm, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ctx->d_aux, ctx->aux_host.data(), sizeof(MarkerAux) * nm,
                       cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(ctx->d_F[0], 0, sizeof(float2) * nm, st));
    CK(cudaMemsetAsync(ctx->d_F[1], 0, sizeof(float2) * nm, st));
    CK(cudaMemsetAsync(ctx->d_Us, 0, sizeof(float2) * nm, st));
    CK(cudaMemsetAsync(ctx->d_rhol, 0, sizeof(float) * nm, st));
    CK(cudaMemcpyAsync(ctx->d_seg_index, seg_index.data(), sizeof(int) * nseg_all,
                       cudaMemcpyHostToDevice, st));
    if (!seg_ptr.empty())
        CK(cudaMemcpyAsync(ctx->d_seg_ptr, seg_ptr.data(), sizeof(int) * seg_ptr.size(),
                           cudaMemcpyHostToDevice, st));
    if (!csr.empty())
        CK(cudaMemcpyAsync(ctx->d_csr, csr.data(), sizeof(CsrEntry) * csr.size(),
                           cudaMemcpyHostToDevice, st));

    CK(cudaMemcpyAsync(ctx->d_body_ptr, body_ptr.data(), sizeof(int) * (nb + 1),
                       cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ctx->d_body_scale, scale.data(), sizeof(double) * nb,
                       cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(ctx->d_hist, 0, sizeof(double2) * (size_t)ctx->cfg.history_len * nb, st));
    CK(cudaStreamSynchronize(st));
    ctx->marker_bytes = ctx->dev_bytes - bytes_before;
    ctx->hist_from = ctx->steps;
    return BTDF_OK;
}

// Bytes of the convective outlet's column buffer (0 for other boundaries).
size_t outlet_bytes(const btdf_ctx* ctx) { return ctx->d_outlet ? sizeof(float) * 9 * ctx->cfg.ny : 0; }

// Marker positions must be finite and their support must touch the lattice.
// Under the convective outlet no support may reach the outlet column: the IB
// kernel would read the outlet column buffer while the overlapping LBM kernel
// rewrites it.  Every path that places markers (add, move) goes through here.
int check_positions(btdf_ctx* ctx, int n, const double* X, const double* Y) {
    const int nx = ctx->cfg.nx, ny = ctx->cfg.ny;
    const double half = 0.5 * ctx->width;
    for (int l = 0; l < n; l++) {
        if (!std::isfinite(X[l]) || !std::isfinite(Y[l]))
            return fail(ctx, BTDF_EINVAL, "marker position not finite");
        const bool inx = ctx->cfg.bc_x == kBcxPeriodic || (X[l] > -half && X[l] < nx - 1 + half);
        const bool iny = ctx->cfg.bc_y == kBcyPeriodic || (Y[l] > -half && Y[l] < ny - 1 + half);
        if (!inx || !iny) return fail(ctx, BTDF_EINVAL, "marker support lies outside the lattice");
        if ((ctx->cfg.bc_x == kBcxPeriodic && std::fabs(X[l]) > 1e9) ||
            (ctx->cfg.bc_y == kBcyPeriodic && std::fabs(Y[l]) > 1e9))
            return fail(ctx, BTDF_EINVAL, "marker position out of range");
        // last support column: floor(X - w/2) + w
        if (ctx->cfg.bc_x == BTDF_BCX_CONVECTIVE &&
            (int)std::floor(X[l] - half) + ctx->width > nx - 2)
            return fail(ctx, BTDF_EINVAL, "a marker support reaches the convective outlet column");
    }
    return BTDF_OK;
}

// ---- adjoint window ----

// State n of the window as held by the tape while segment j is processed:
// the checkpoint at the segment's start, the next checkpoint at its end,
// the segment buffer in between.
float* tape_state(const AdjointTape& T, int j, int64_t n) {
    const int64_t s = (int64_t)j * T.every;
    if (n == s) return T.ck + (size_t)j * T.state_elems;
    if (j + 1 < T.nck && n == s + T.every) return T.ck + (size_t)(j + 1) * T.state_elems;
    return T.seg + (size_t)(n - s - 1) * T.state_elems;
}

bool tape_pull(const AdjointTape& T, int64_t n) { return !(n == 0 && T.post0); }

// One forward step of the window: the IB kernel writes F^n into the tape,
// the LBM kernel spreads it and advances gin -> gout.  No body-force history
// and no step counter: the context's own state is not touched.
int tape_step(btdf_ctx* ctx, int64_t n, const float* gin, float* gout, cudaStream_t st) {
    AdjointTape& T = ctx->tape;
    const bool pull = tape_pull(T, n);
    float2* F = T.Fall + (size_t)n * ctx->nmark;
    LatticeParams p = lattice_params(ctx);
    p.F = F;
    p.nbody = 0;
    p.step = nullptr;
    p.hist = nullptr;
    IbParams q{};
    q.nmark = ctx->nmark;
    q.mk = ctx->d_mk;
    q.aux = ctx->d_aux;
    q.F_prev = nullptr;
    q.F_out = F;
    q.Us = T.Us;
    q.rhol = T.rhol;
    q.first_pass = 1;
    q.status = ctx->d_status;
    CK(launch_ib_force(kStoreF32, pull, ctx->width, gin, p, q, false, st));
    CK(launch_collide_stream(kStoreF32, pull, kVarReg4, gin, gout, p, kFullGrid, true, st));
    return BTDF_OK;
}

// Steps first .. last-1 of segment j.
int tape_run(btdf_ctx* ctx, int j, int64_t first, int64_t last, cudaStream_t st) {
    const AdjointTape& T = ctx->tape;
    for (int64_t n = first; n < last; n++) {
        const int rc = tape_step(ctx, n, tape_state(T, j, n), tape_state(T, j, n + 1), st);
        if (rc != BTDF_OK) return rc;
    }
    return BTDF_OK;
}

// The forward window after its start state: every segment, checkpoints
// at the segment ends.
int tape_forward_enqueue(btdf_ctx* ctx, cudaStream_t st) {
    const AdjointTape& T = ctx->tape;
    for (int j = 0; j < T.nck; j++) {
        const int64_t s = (int64_t)j * T.every, e = std::min<int64_t>(s + T.every, T.nsteps);
        const int rc = tape_run(ctx, j, s, e, st);
        if (rc != BTDF_OK) return rc;
    }
    return BTDF_OK;
}

// The reverse sweep: segments from the last, each recomputed from its
// checkpoint, then reversed step by step.
int tape_backward_enqueue(btdf_ctx* ctx, cudaStream_t st) {
    AdjointTape& T = ctx->tape;
    const int nm = ctx->nmark;
    const size_t sb = sizeof(float) * T.state_elems;
    CK(cudaMemsetAsync(T.acc, 0, sizeof(double) * (2 * (size_t)nm + 1), st));
    CK(cudaMemsetAsync(T.lam[0], 0, sb, st));   // dJ/dg^N = 0
    AdjParams q{};
    q.nmark = nm;
    q.nband = (int)ctx->band_keys.size();
    q.mk = ctx->d_mk;
    q.aux = ctx->d_aux;
    q.am = T.am;
    q.cscale = T.cscale;
    q.band_keys = T.band_keys;
    q.fbar_band = T.fbar_band;
    q.Fbar_band = T.Fbar_band;
    q.mbar = T.mbar;
    q.objw = T.objw;
    q.dJdX = T.acc;
    q.dJdY = T.acc + nm;
    q.dU = T.acc + 2 * nm;
    int c = 0;
    for (int j = T.nck - 1; j >= 0; j--) {
        const int64_t s = (int64_t)j * T.every, e = std::min<int64_t>(s + T.every, T.nsteps);
        // states g^{s+1} .. g^{e-1}; F^{e-1} is already on the tape
        const int rc = tape_run(ctx, j, s, e - 1, st);
        if (rc != BTDF_OK) return rc;
        for (int64_t n = e - 1; n >= s; n--) {
            LatticeParams p = lattice_params(ctx);
            p.F = T.Fall + (size_t)n * nm;
            CK(cudaMemsetAsync(T.lam[1 - c], 0, sb, st));
            CK(launch_adjoint_step(tape_state(T, j, n), T.lam[c], T.lam[1 - c], p, q, ctx->width,
                                   tape_pull(T, n), st));
            c = 1 - c;
        }
    }
    return BTDF_OK;
}

// Launches one pass of the window through its CUDA graph on the context
// stream, capturing it first when the window, the buffers, the markers or
// the inflow changed since the graph was made.
int tape_graph_launch(btdf_ctx* ctx, bool backward) {
    AdjointTape& T = ctx->tape;
    const std::vector<double> key = {(double)T.nsteps, (double)T.every, T.post0 ? 1.0 : 0.0, (double)T.gen,
                                     (double)ctx->marker_gen, ctx->cfg.u_in};
    cudaGraphExec_t& exec = backward ? T.bwd : T.fwd;
    std::vector<double>& have = backward ? T.bwd_key : T.fwd_key;
    if (!exec || have != key) {
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
        const int rc = backward ? tape_backward_enqueue(ctx, ctx->cap) : tape_forward_enqueue(ctx, ctx->cap);
        const cudaError_t e = cudaStreamEndCapture(ctx->cap, &graph);
        if (rc != BTDF_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
        // Same window shape, new arguments (moved markers, another inflow):
        // update the instantiated graph in place, which is far cheaper than
        // instantiating it again.
        bool updated = false;
        if (exec) {
            cudaGraphExecUpdateResultInfo info;
            updated = cudaGraphExecUpdate(exec, graph, &info) == cudaSuccess;
            if (!updated) {
                cudaGetLastError();
                cudaGraphExecDestroy(exec);
                exec = nullptr;
            }
        }
        cudaError_t ei = cudaSuccess;
        if (!updated) ei = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            exec = nullptr;
            return cuda_fail(ctx, ei, "cudaGraphInstantiate");
        }
        have = key;
    }
    CK(cudaGraphLaunch(exec, ctx->stream));
    return BTDF_OK;
}

int tape_alloc(btdf_ctx* ctx, int nck, int every, int64_t nsteps) {
    AdjointTape& T = ctx->tape;
    const int nm = ctx->nmark, nb = (int)ctx->band_keys.size();
    const size_t E = (size_t)9 * ctx->plane;
    if (T.ck && T.state_elems == E && T.cap_ck >= nck && T.cap_every >= every && T.cap_F >= nsteps &&
        T.cap_mark == nm && T.cap_band == nb)
        return BTDF_OK;
    free_tape(ctx);
    T.state_elems = E;
    const size_t before = ctx->dev_bytes;
    auto bail = [&](cudaError_t e) {
        const size_t got = ctx->dev_bytes - before;
        T.bytes = got;
        free_tape(ctx);
        return e == cudaErrorMemoryAllocation ? fail(ctx, BTDF_ENOMEM, "adjoint tape does not fit")
                                              : cuda_fail(ctx, e, "cudaMalloc");
    };
#define TA(ptr, count)                                                  \
    do {                                                                \
        cudaError_t e_ = dalloc(ctx, &(ptr), sizeof(*(ptr)) * (count)); \
        if (e_ != cudaSuccess) return bail(e_);                         \
    } while (0)
    TA(T.ck, E * nck);
    TA(T.seg, E * every);
    TA(T.lam[0], E);
    TA(T.lam[1], E);
    TA(T.Fall, (size_t)nsteps * nm);
    TA(T.Us, (size_t)nm);
    TA(T.rhol, (size_t)nm);
    TA(T.am, (size_t)nm);
    TA(T.cscale, (size_t)nm);
    TA(T.objw, (size_t)nm);
    TA(T.band_keys, (size_t)std::max(nb, 1));
    TA(T.fbar_band, (size_t)std::max(nb, 1) * kSeg * 9);
    TA(T.Fbar_band, (size_t)std::max(nb, 1) * kSeg);
    TA(T.mbar, (size_t)nm);
    TA(T.acc, (size_t)2 * nm + 1);
#undef TA
    T.bytes = ctx->dev_bytes - before;
    T.cap_ck = nck;
    T.cap_every = every;
    T.cap_F = nsteps;
    T.cap_mark = nm;
    T.cap_band = nb;
    return BTDF_OK;
}

// Copies steps first .. first+n-1 of the force history into dst: one
// double2 per step for one body, or, with body -1, nbody double2 per step
// (step-major); ring wraps split the copy.
int copy_history(btdf_ctx* ctx, int32_t body, int64_t first, int64_t n, double2* dst) {
    const int64_t H = ctx->cfg.history_len;
    const int nb = (int)ctx->bodies.size();
    int64_t done = 0;
    while (done < n) {
        const int64_t slot = (first + done) % H;
        const int64_t cnt = std::min<int64_t>(n - done, H - slot);
        if (body < 0)
            CK(cudaMemcpyAsync(dst + done * nb, ctx->d_hist + slot * nb, sizeof(double2) * nb * cnt,
                               cudaMemcpyDeviceToHost, ctx->stream));
        else
            CK(cudaMemcpy2DAsync(dst + done, sizeof(double2), ctx->d_hist + slot * nb + body,
                                 sizeof(double2) * nb, sizeof(double2), (size_t)cnt,
                                 cudaMemcpyDeviceToHost, ctx->stream));
        done += cnt;
    }
    return BTDF_OK;
}

}  // namespace

extern "C" {

int btdf_version(void) { return 1; }

const char* btdf_status_string(int s) {
    switch (s) {
    case BTDF_OK: return "ok";
    case BTDF_EINVAL: return "invalid argument";
    case BTDF_ENOMEM: return "out of memory";
    case BTDF_ECUDA: return "CUDA error";
    case BTDF_EUNSTABLE: return "unstable (density or force at a marker)";
    case BTDF_ETIMEOUT: return "device wait timed out";
    case BTDF_ESTATE: return "invalid state for this call";
    default: return "unknown status";
    }
}

const char* btdf_last_error(const btdf_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int btdf_config_default(btdf_config* cfg) {
    if (!cfg) return BTDF_EINVAL;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->nx = 64;
    cfg->ny = 64;
    cfg->tau = 0.6;
    cfg->u_in = 0.0;
    cfg->delta = BTDF_DELTA3;
    cfg->nf = 1;
    cfg->storage = BTDF_F32;
    cfg->bc_x = BTDF_BCX_PERIODIC;
    cfg->bc_y = BTDF_BCY_PERIODIC;
    cfg->history_len = 4096;
    cfg->layout = BTDF_LAYOUT_ROWS;
    return BTDF_OK;
}

int btdf_create(const btdf_config* cfg, void* stream, btdf_ctx** out) {
    if (!cfg || !out) return BTDF_EINVAL;
    *out = nullptr;
    const btdf_config& c = *cfg;
    // element offsets inside the kernels are 32-bit: 9 planes of the padded lattice
    if (c.nx < 4 || c.ny < 4) return BTDF_EINVAL;
    if (9ll * (((long long)c.nx + 31) / 32 * 32) * c.ny >= (1ll << 32)) return BTDF_EINVAL;
    if (!(c.tau > 0.5) || !std::isfinite(c.tau)) return BTDF_EINVAL;
    if (support_width(c.delta) == 0) return BTDF_EINVAL;
    if (c.nf < 1 || c.nf > 64) return BTDF_EINVAL;
    if (c.storage < 0 || c.storage > 2) return BTDF_EINVAL;
    if (c.bc_x < 0 || c.bc_x > 3 || c.bc_y < 0 || c.bc_y > 2) return BTDF_EINVAL;
    if (c.history_len < 1) return BTDF_EINVAL;
    if (c.layout != BTDF_LAYOUT_PLANES && c.layout != BTDF_LAYOUT_ROWS) return BTDF_EINVAL;
    if (!std::isfinite(c.u_in) || std::fabs(c.u_in) >= 0.5) return BTDF_EINVAL;
    if (!std::isfinite(c.gx) || !std::isfinite(c.gy)) return BTDF_EINVAL;

    btdf_ctx* ctx = new (std::nothrow) btdf_ctx();
    if (!ctx) return BTDF_ENOMEM;
    ctx->cfg = c;
    ctx->u_ref = c.u_in;
    ctx->stream = (cudaStream_t)stream;
    ctx->width = support_width(c.delta);
    ctx->nxp = (c.nx + 31) / 32 * 32;
    ctx->nseg = (ctx->nxp + kSeg - 1) / kSeg;
    ctx->plane = (long long)ctx->nxp * c.ny;
    ctx->elem = elem_bytes(c.storage);
    auto bail = [&](int code) {
        btdf_destroy(ctx);
        return code;
    };
    cudaError_t e = cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(BTDF_ECUDA);
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return bail(BTDF_ECUDA);
        for (int v = 0; v < kVarCount; v++)
            if (is_tma(v)) ctx->tma_grid[v] = (long long)sms * collide_stream_tma_blocks_per_sm(c.storage, v);
        ctx->pf_grid[0] = (long long)sms * collide_stream_blocks_per_sm(c.storage, true, kVarReg4Pf);
        ctx->pf_grid[1] = (long long)sms * collide_stream_blocks_per_sm(c.storage, true, kVarReg2Pf);
        // half a wave of resident warps (measured: 5% faster on 8192 x 4096,
        // no gain on 1600 x 800, where the autotuner keeps variant 9)
        const int pfv[2] = {kVarReg2OccPf, kVarReg4L2Pf};
        for (int k = 0; k < 2; k++)
            for (int pull = 0; pull < 2; pull++)
                ctx->pf_units[k][pull] =
                    (long long)sms * collide_stream_blocks_per_sm(c.storage, pull != 0, pfv[k]) *
                    (collide_stream_block_threads(c.storage, pfv[k]) / 32) / 2;
    }
    const size_t bytes = (size_t)9 * ctx->plane * ctx->elem;
    for (int i = 0; i < 2; i++) {
        e = dalloc(ctx, &ctx->g[i], bytes);
        if (e == cudaErrorMemoryAllocation) return bail(BTDF_ENOMEM);
        if (e != cudaSuccess) return bail(BTDF_ECUDA);
        if (cudaMemsetAsync(ctx->g[i], 0, bytes, ctx->stream) != cudaSuccess) return bail(BTDF_ECUDA);
    }
    ctx->tma_ok = encode_tensor_maps(ctx);
    for (int v = 0; v < kVarCount; v++)
        if (is_tma(v) && ctx->tma_grid[v] <= 0) ctx->tma_ok = false;
    if (cudaMallocHost((void**)&ctx->status_pin, sizeof(int)) != cudaSuccess) return bail(BTDF_ECUDA);
    for (cudaEvent_t& e : ctx->aux_ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return bail(BTDF_ECUDA);
    *ctx->status_pin = 0;
    if (dalloc(ctx, &ctx->d_step, sizeof(unsigned long long)) != cudaSuccess ||
        dalloc(ctx, &ctx->d_status, sizeof(int)) != cudaSuccess ||
        dalloc(ctx, &ctx->d_sched, 2 * sizeof(unsigned)) != cudaSuccess ||
        (c.bc_x == BTDF_BCX_CONVECTIVE && dalloc(ctx, &ctx->d_outlet, sizeof(float) * 9 * c.ny) != cudaSuccess) ||
        (c.bc_x == BTDF_BCX_BOX && dalloc(ctx, &ctx->d_box, sizeof(float2) * (2 * c.nx + 2 * (c.ny - 2))) != cudaSuccess))
        return bail(BTDF_ECUDA);
    if (ctx->d_box && cudaMemsetAsync(ctx->d_box, 0, sizeof(float2) * (2 * c.nx + 2 * (c.ny - 2)), ctx->stream) != cudaSuccess)
        return bail(BTDF_ECUDA);
    if (cudaMemsetAsync(ctx->d_step, 0, sizeof(unsigned long long), ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->d_sched, 0, 2 * sizeof(unsigned), ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess)
        return bail(BTDF_ECUDA);
    *out = ctx;
    return BTDF_OK;
}

int btdf_destroy(btdf_ctx* ctx) {
    if (!ctx) return BTDF_EINVAL;
    if (ctx->stream || ctx->g[0]) cudaStreamSynchronize(ctx->stream);
    drop_graphs(ctx);
    free_markers(ctx);
    free_tape(ctx);
    dfree(ctx, ctx->g[0]);
    dfree(ctx, ctx->g[1]);
    dfree(ctx, ctx->d_step);
    dfree(ctx, ctx->d_status);
    dfree(ctx, ctx->d_sched);
    dfree(ctx, ctx->d_outlet);
    dfree(ctx, ctx->d_box);
    for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->aux_ev)
        if (e) cudaEventDestroy(e);
    if (ctx->status_pin) cudaFreeHost(ctx->status_pin);
    if (ctx->pin) cudaFreeHost(ctx->pin);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    delete ctx;
    return BTDF_OK;
}

int btdf_init_fields(btdf_ctx* ctx, const double* rho, const double* ux, const double* uy) {
    if (!ctx || !rho || !ux || !uy) return fail(ctx, BTDF_EINVAL, "null argument");
    const size_t nn = (size_t)ctx->cfg.nx * ctx->cfg.ny;
    for (size_t i = 0; i < nn; i++)
        if (!(rho[i] > 0.0) || !std::isfinite(rho[i]) || !std::isfinite(ux[i]) || !std::isfinite(uy[i]))
            return fail(ctx, BTDF_EINVAL, "initial fields must be finite with rho > 0");
    double* d = nullptr;
    CK(cudaMalloc((void**)&d, sizeof(double) * 3 * nn));
    cudaStream_t st = ctx->stream;
    int rc = BTDF_OK;
    auto run = [&]() -> int {
        CK(cudaMemcpyAsync(d, rho, sizeof(double) * nn, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(d + nn, ux, sizeof(double) * nn, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(d + 2 * nn, uy, sizeof(double) * nn, cudaMemcpyHostToDevice, st));
        const size_t bytes = (size_t)9 * ctx->plane * ctx->elem;
        CK(cudaMemsetAsync(ctx->g[0], 0, bytes, st));
        CK(cudaMemsetAsync(ctx->g[1], 0, bytes, st));
        if (ctx->d_outlet) CK(cudaMemsetAsync(ctx->d_outlet, 0, sizeof(float) * 9 * ctx->cfg.ny, st));
        const LatticeParams p = lattice_params(ctx);
        CK(launch_init_equilibrium(ctx->cfg.storage, ctx->g[0], p, d, d + nn, d + 2 * nn, st));
        CK(cudaMemsetAsync(ctx->d_step, 0, sizeof(unsigned long long), st));
        CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));
        CK(cudaMemsetAsync(ctx->d_sched, 0, 2 * sizeof(unsigned), st));
        CK(cudaStreamSynchronize(st));
        return BTDF_OK;
    };
    rc = run();
    cudaFree(d);
    if (rc != BTDF_OK) return rc;
    ctx->cur = 0;
    ctx->poststream = true;
    ctx->has_fields = true;
    ctx->steps = 0;
    ctx->hist_from = 0;
    return BTDF_OK;
}

int btdf_add_markers(btdf_ctx* ctx, int32_t n, const double* X, const double* Y, const double* Ubx,
                     const double* Uby, double ds, double drs, int32_t* body_id) {
    if (!ctx) return BTDF_EINVAL;
    if (n < 1 || !X || !Y || !(ds > 0.0) || !std::isfinite(ds) || !std::isfinite(drs))
        return fail(ctx, BTDF_EINVAL, "need n >= 1 markers, positions and ds > 0");
    if ((long long)ctx->nmark + n > (1ll << 30)) return fail(ctx, BTDF_EINVAL, "too many markers");
    for (int l = 0; l < n; l++)
        if ((Ubx && !std::isfinite(Ubx[l])) || (Uby && !std::isfinite(Uby[l])))
            return fail(ctx, BTDF_EINVAL, "marker velocity not finite");
    const int rcp = check_positions(ctx, n, X, Y);
    if (rcp != BTDF_OK) return rcp;
    Body B;
    B.first = ctx->nmark;
    B.n = n;
    B.ds = ds;
    B.drs = drs > 0.0 ? drs : paper_drs(ctx->cfg.delta);
    B.X.assign(X, X + n);
    B.Y.assign(Y, Y + n);
    B.Ubx.assign(n, 0.0);
    B.Uby.assign(n, 0.0);
    if (Ubx) B.Ubx.assign(Ubx, Ubx + n);
    if (Uby) B.Uby.assign(Uby, Uby + n);
    const int id = (int)ctx->bodies.size();
    ctx->bodies.push_back(std::move(B));
    ctx->nmark += n;
    const int rc = rebuild_markers(ctx);
    if (rc != BTDF_OK) return rc;
    if (body_id) *body_id = id;
    return BTDF_OK;
}

int btdf_add_cylinder(btdf_ctx* ctx, double cx, double cy, double D, int32_t n, double drs,
                      int32_t* body_id) {
    if (!ctx) return BTDF_EINVAL;
    if (n < 1 || !(D > 0.0) || !std::isfinite(D) || !std::isfinite(cx) || !std::isfinite(cy))
        return fail(ctx, BTDF_EINVAL, "need n >= 1, D > 0 and a finite centre");
    std::vector<double> X(n), Y(n);
    for (int l = 0; l < n; l++) {
        const double th = 2.0 * M_PI * (double)l / (double)n;
        X[l] = cx + 0.5 * D * std::cos(th);
        Y[l] = cy + 0.5 * D * std::sin(th);
    }
    return btdf_add_markers(ctx, n, X.data(), Y.data(), nullptr, nullptr, M_PI * D / (double)n, drs, body_id);
}

int btdf_set_boundary_velocity(btdf_ctx* ctx, const double* ubx, const double* uby) {
    if (!ctx) return BTDF_EINVAL;
    if (!ctx->d_box) return fail(ctx, BTDF_ESTATE, "the lattice has no prescribed-velocity box");
    if (!ubx || !uby) return fail(ctx, BTDF_EINVAL, "null boundary velocity");
    const int np = 2 * ctx->cfg.nx + 2 * (ctx->cfg.ny - 2);
    std::vector<float2> v(np);
    for (int k = 0; k < np; k++) {
        if (!std::isfinite(ubx[k]) || !std::isfinite(uby[k]) || std::fabs(ubx[k]) >= 0.5 || std::fabs(uby[k]) >= 0.5)
            return fail(ctx, BTDF_EINVAL, "boundary velocity not finite or not below 0.5");
        v[k] = make_float2((float)ubx[k], (float)uby[k]);
    }
    // pageable source: the call returns once the runtime has staged it
    CK(cudaMemcpyAsync(ctx->d_box, v.data(), sizeof(float2) * np, cudaMemcpyHostToDevice, ctx->stream));
    return BTDF_OK;
}

int btdf_set_marker_velocity(btdf_ctx* ctx, int32_t body, const double* Ubx, const double* Uby) {
    if (!ctx) return BTDF_EINVAL;
    if (body < -1 || body >= (int)ctx->bodies.size() || !Ubx || !Uby || ctx->nmark == 0)
        return fail(ctx, BTDF_EINVAL, "bad body index or null velocity");
    // body -1: every body, markers in the order they were added
    const int b0 = body < 0 ? 0 : body, b1 = body < 0 ? (int)ctx->bodies.size() : body + 1;
    const int first = ctx->bodies[b0].first;
    const int count = ctx->bodies[b1 - 1].first + ctx->bodies[b1 - 1].n - first;
    for (int l = 0; l < count; l++)
        if (!std::isfinite(Ubx[l]) || !std::isfinite(Uby[l]))
            return fail(ctx, BTDF_EINVAL, "marker velocity not finite");
    // this staging slot may still feed an upload kStageSlots calls back
    const int k = ctx->aux_slot;
    ctx->aux_slot = (k + 1) % kStageSlots;
    CK(cudaEventSynchronize(ctx->aux_ev[k]));
    MarkerAux* stage = ctx->aux_pin + (size_t)k * ctx->nmark;
    for (int b = b0; b < b1; b++) {
        Body& B = ctx->bodies[b];
        const double* ux = Ubx + (B.first - first);
        const double* uy = Uby + (B.first - first);
        for (int l = 0; l < B.n; l++) {
            B.Ubx[l] = ux[l];
            B.Uby[l] = uy[l];
            MarkerAux& A = ctx->aux_host[B.first + l];
            A.ubx_rel = (float)(ux[l] - ctx->u_ref * B.wsum[l]);
            A.uby_rel = (float)uy[l];
            stage[B.first + l] = A;
        }
    }
    ctx->tape.pending = false;
    CK(cudaMemcpyAsync(ctx->d_aux + first, stage + first, sizeof(MarkerAux) * count,
                       cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaEventRecord(ctx->aux_ev[k], ctx->stream));
    return BTDF_OK;
}

int btdf_step(btdf_ctx* ctx, int64_t nsteps) {
    if (!ctx) return BTDF_EINVAL;
    if (nsteps < 0) return fail(ctx, BTDF_EINVAL, "nsteps < 0");
    if (!ctx->has_fields) return fail(ctx, BTDF_ESTATE, "call btdf_init_fields or btdf_load_state first");
    int64_t i = 0;
    if (nsteps > 0 && ctx->poststream) {
        const int rc = enqueue_step(ctx, ctx->stream, false, ctx->cur, ctx->prof);
        if (rc != BTDF_OK) return rc;
        ctx->cur = 1 - ctx->cur;
        ctx->poststream = false;
        i = 1;
    }
    if (!ctx->prof) {
        while (nsteps - i >= kGraphSteps) {
            const int rc = ensure_graph(ctx, ctx->cur);
            if (rc != BTDF_OK) return rc;
            CK(cudaGraphLaunch(ctx->gexec[ctx->cur], ctx->stream));
            i += kGraphSteps;
        }
    }
    for (; i < nsteps; i++) {
        const int rc = enqueue_step(ctx, ctx->stream, true, ctx->cur, ctx->prof);
        if (rc != BTDF_OK) return rc;
        ctx->cur = 1 - ctx->cur;
    }
    ctx->steps += nsteps;
    return BTDF_OK;
}

int btdf_sync(btdf_ctx* ctx) {
    if (!ctx) return BTDF_EINVAL;
    CK(cudaStreamSynchronize(ctx->stream));
    return read_status(ctx);
}

int64_t btdf_step_count(const btdf_ctx* ctx) { return ctx ? ctx->steps : -1; }

int btdf_read_forces(btdf_ctx* ctx, int32_t body, int64_t first, int64_t n, double* Fx, double* Fy) {
    if (!ctx) return BTDF_EINVAL;
    if (body < -1 || body >= (int)ctx->bodies.size() || ctx->bodies.empty() || n < 0 ||
        (n > 0 && (!Fx || !Fy)))
        return fail(ctx, BTDF_EINVAL, "bad body index, count or null output");
    const int64_t H = ctx->cfg.history_len;
    if (first < ctx->hist_from || first < ctx->steps - H || first + n > ctx->steps)
        return fail(ctx, BTDF_EINVAL, "requested steps are not in the force history");
    const int64_t nval = n * (body < 0 ? (int64_t)ctx->bodies.size() : 1);
    const size_t need = sizeof(double2) * (size_t)std::max<int64_t>(nval, 1);
    if (ctx->pin_cap < need) {
        CK(cudaStreamSynchronize(ctx->stream));
        if (ctx->pin) cudaFreeHost(ctx->pin);
        ctx->pin = nullptr;
        ctx->pin_cap = 0;
        CK(cudaMallocHost(&ctx->pin, need));
        ctx->pin_cap = need;
    }
    double2* tmp = (double2*)ctx->pin;
    const int rcc = copy_history(ctx, body, first, n, tmp);
    if (rcc != BTDF_OK) return rcc;
    const int rc = read_status(ctx);   // one synchronization for both copies
    for (int64_t i = 0; i < nval; i++) {
        Fx[i] = tmp[i].x;
        Fy[i] = tmp[i].y;
    }
    return rc;
}

int btdf_read_forces_async(btdf_ctx* ctx, int32_t body, int64_t first, int64_t n, double* F) {
    if (!ctx) return BTDF_EINVAL;
    if (body < -1 || body >= (int)ctx->bodies.size() || ctx->bodies.empty() || n < 0 ||
        (n > 0 && !F))
        return fail(ctx, BTDF_EINVAL, "bad body index, count or null output");
    const int64_t H = ctx->cfg.history_len;
    if (first < ctx->hist_from || first < ctx->steps - H || first + n > ctx->steps)
        return fail(ctx, BTDF_EINVAL, "requested steps are not in the force history");
    return copy_history(ctx, body, first, n, (double2*)F);
}

int btdf_read_markers(btdf_ctx* ctx, int32_t body, float* Usx, float* Usy, float* Fbx, float* Fby) {
    if (!ctx) return BTDF_EINVAL;
    if (body < 0 || body >= (int)ctx->bodies.size()) return fail(ctx, BTDF_EINVAL, "bad body index");
    const Body& B = ctx->bodies[body];
    std::vector<float2> us(B.n), F(B.n);
    CK(cudaMemcpyAsync(us.data(), ctx->d_Us + B.first, sizeof(float2) * B.n, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaMemcpyAsync(F.data(), ctx->d_F[(ctx->cfg.nf - 1) % 2] + B.first, sizeof(float2) * B.n,
                       cudaMemcpyDeviceToHost, ctx->stream));
    const int rc = read_status(ctx);
    for (int l = 0; l < B.n; l++) {
        if (Usx) Usx[l] = us[l].x;
        if (Usy) Usy[l] = us[l].y;
        if (Fbx) Fbx[l] = F[l].x;
        if (Fby) Fby[l] = F[l].y;
    }
    return rc;
}

int btdf_read_field(btdf_ctx* ctx, int32_t kind, float* dst, int32_t dst_is_device) {
    if (!ctx) return BTDF_EINVAL;
    if (kind < 0 || kind > 5 || !dst) return fail(ctx, BTDF_EINVAL, "bad field kind or null output");
    if (!ctx->has_fields) return fail(ctx, BTDF_ESTATE, "no fields");
    const size_t nn = (size_t)ctx->cfg.nx * ctx->cfg.ny * (kind == 3 ? 9 : 1);
    float* d = dst;
    if (!dst_is_device) CK(cudaMalloc((void**)&d, sizeof(float) * nn));
    int rc = BTDF_OK;
    auto run = [&]() -> int {
        const LatticeParams p = lattice_params(ctx);
        if (kind >= 4) CK(launch_force_field(p, kind - 4, d, ctx->stream));
        else
            CK(launch_read_field(ctx->cfg.storage, !ctx->poststream, ctx->g[ctx->cur], p, kind, d,
                                 ctx->stream));
        if (!dst_is_device)
            CK(cudaMemcpyAsync(dst, d, sizeof(float) * nn, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        return BTDF_OK;
    };
    rc = run();
    if (!dst_is_device) cudaFree(d);
    if (rc != BTDF_OK) return rc;
    return read_status(ctx);
}

int btdf_state_size(btdf_ctx* ctx, size_t* bytes) {
    if (!ctx || !bytes) return BTDF_EINVAL;
    *bytes = sizeof(StateHeader) + (size_t)9 * ctx->plane * ctx->elem + outlet_bytes(ctx);
    return BTDF_OK;
}

int btdf_save_state(btdf_ctx* ctx, void* dst, size_t cap, size_t* used) {
    if (!ctx || !dst) return BTDF_EINVAL;
    if (!ctx->has_fields) return fail(ctx, BTDF_ESTATE, "no fields");
    size_t need = 0;
    btdf_state_size(ctx, &need);
    if (cap < need) return fail(ctx, BTDF_EINVAL, "destination buffer too small");
    StateHeader h{kStateMagic, ctx->cfg.nx, ctx->cfg.ny, ctx->nxp, ctx->cfg.storage,
                  ctx->poststream ? 1 : 0, ctx->cfg.layout, ctx->steps, ctx->u_ref};
    std::memcpy(dst, &h, sizeof(h));
    const size_t ob = outlet_bytes(ctx);
    CK(cudaMemcpyAsync((char*)dst + sizeof(h), ctx->g[ctx->cur], need - sizeof(h) - ob,
                       cudaMemcpyDeviceToHost, ctx->stream));
    if (ob) CK(cudaMemcpyAsync((char*)dst + need - ob, ctx->d_outlet, ob, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (used) *used = need;
    return read_status(ctx);
}

int btdf_load_state(btdf_ctx* ctx, const void* src, size_t len) {
    if (!ctx || !src) return BTDF_EINVAL;
    size_t need = 0;
    btdf_state_size(ctx, &need);
    if (len < need) return fail(ctx, BTDF_EINVAL, "checkpoint too short");
    StateHeader h;
    std::memcpy(&h, src, sizeof(h));
    if (h.magic != kStateMagic || h.nx != ctx->cfg.nx || h.ny != ctx->cfg.ny || h.nxp != ctx->nxp ||
        h.storage != ctx->cfg.storage || h.layout != ctx->cfg.layout || h.steps < 0)
        return fail(ctx, BTDF_EINVAL, "checkpoint does not match this context");
    // the deviations are relative to the writer's reference velocity
    if (h.u_ref != ctx->u_ref)
        return fail(ctx, BTDF_EINVAL, "checkpoint was written with another reference velocity");
    const size_t ob = outlet_bytes(ctx);
    CK(cudaMemcpyAsync(ctx->g[ctx->cur], (const char*)src + sizeof(h), need - sizeof(h) - ob,
                       cudaMemcpyHostToDevice, ctx->stream));
    if (ob) CK(cudaMemcpyAsync(ctx->d_outlet, (const char*)src + need - ob, ob, cudaMemcpyHostToDevice, ctx->stream));
    unsigned long long s = (unsigned long long)h.steps;
    CK(cudaMemcpyAsync(ctx->d_step, &s, sizeof(s), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->poststream = h.poststream != 0;
    ctx->has_fields = true;
    ctx->steps = h.steps;
    ctx->hist_from = h.steps;
    return BTDF_OK;
}

int btdf_profile_enable(btdf_ctx* ctx, int32_t on) {
    if (!ctx) return BTDF_EINVAL;
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->prof = on != 0;
    ctx->ev_used = 0;
    return BTDF_OK;
}

int btdf_profile_read(btdf_ctx* ctx, double* ms_ib, double* ms_lbm, int64_t* launches_ib,
                      int64_t* launches_lbm) {
    if (!ctx) return BTDF_EINVAL;
    CK(cudaStreamSynchronize(ctx->stream));
    double a = 0.0, b = 0.0;
    const int64_t nst = (int64_t)(ctx->ev_used / 3);
    for (int64_t i = 0; i < nst; i++) {
        float t1 = 0.f, t2 = 0.f;
        CK(cudaEventElapsedTime(&t1, ctx->ev[3 * i], ctx->ev[3 * i + 1]));
        CK(cudaEventElapsedTime(&t2, ctx->ev[3 * i + 1], ctx->ev[3 * i + 2]));
        a += t1;
        b += t2;
    }
    if (ms_ib) *ms_ib = a;
    if (ms_lbm) *ms_lbm = b;
    if (launches_ib) *launches_ib = ctx->nmark > 0 ? nst * ctx->cfg.nf : 0;
    if (launches_lbm) *launches_lbm = nst;
    return BTDF_OK;
}

int btdf_tune(btdf_ctx* ctx, int32_t variant, int32_t grid_blocks) {
    if (!ctx) return BTDF_EINVAL;
    if (variant < 0 || variant >= kVarCount) return fail(ctx, BTDF_EINVAL, "unknown kernel variant");
    if (is_tma(variant) && !ctx->tma_ok)
        return fail(ctx, BTDF_EINVAL, "TMA variants unavailable (tensor maps not encoded)");
    if (grid_blocks < 0) return fail(ctx, BTDF_EINVAL, "grid_blocks < 0");
    CK(cudaStreamSynchronize(ctx->stream));
    drop_graphs(ctx);
    ctx->variant = variant;
    ctx->grid_override = grid_blocks;
    return BTDF_OK;
}

int btdf_set_wait_limit(btdf_ctx* ctx, int32_t polls) {
    if (!ctx) return BTDF_EINVAL;
    CK(cudaStreamSynchronize(ctx->stream));
    drop_graphs(ctx);   // the graphs hold the old limit in their kernel arguments
    ctx->wait_polls = polls < 0 ? -1 : polls;
    return BTDF_OK;
}

int btdf_set_inflow(btdf_ctx* ctx, double u_in) {
    if (!ctx) return BTDF_EINVAL;
    if (!std::isfinite(u_in) || std::fabs(u_in) >= 0.5) return fail(ctx, BTDF_EINVAL, "need |u_in| < 0.5");
    CK(cudaStreamSynchronize(ctx->stream));
    drop_graphs(ctx);   // the graphs hold the old value in their kernel arguments
    ctx->cfg.u_in = u_in;
    ctx->tape.pending = false;
    return BTDF_OK;
}

int btdf_move_markers(btdf_ctx* ctx, int32_t body, const double* X, const double* Y) {
    if (!ctx) return BTDF_EINVAL;
    if (body < 0 || body >= (int)ctx->bodies.size() || !X || !Y)
        return fail(ctx, BTDF_EINVAL, "bad body index or null positions");
    Body& B = ctx->bodies[body];
    const int rc = check_positions(ctx, B.n, X, Y);
    if (rc != BTDF_OK) return rc;
    CK(cudaStreamSynchronize(ctx->stream));
    B.X.assign(X, X + B.n);
    B.Y.assign(Y, Y + B.n);
    return rebuild_markers(ctx);
}

int btdf_adjoint_forward(btdf_ctx* ctx, int64_t nsteps, int32_t every, int32_t body, double dref,
                         double* J) {
    if (!ctx) return BTDF_EINVAL;
    if (!ctx->has_fields) return fail(ctx, BTDF_ESTATE, "call btdf_init_fields or btdf_load_state first");
    if (ctx->nmark == 0) return fail(ctx, BTDF_ESTATE, "the objective needs at least one body");
    if (ctx->cfg.nf != 1 || ctx->cfg.storage != BTDF_F32)
        return fail(ctx, BTDF_EINVAL, "the adjoint supports nf = 1 with FP32 storage");
    if (ctx->cfg.bc_x == BTDF_BCX_CONVECTIVE || ctx->cfg.bc_x == BTDF_BCX_BOX)
        return fail(ctx, BTDF_EINVAL, "the adjoint supports periodic and in/out (zero-gradient) x boundaries only");
    if (nsteps < 1 || every < 1 || nsteps > (1ll << 30))
        return fail(ctx, BTDF_EINVAL, "need nsteps >= 1 and every >= 1");
    if (!(dref > 0.0) || !std::isfinite(dref)) return fail(ctx, BTDF_EINVAL, "need dref > 0");
    if (!(std::fabs(ctx->cfg.u_in) > 0.0)) return fail(ctx, BTDF_EINVAL, "Cd needs u_in != 0");
    if (body < -1 || body >= (int)ctx->bodies.size()) return fail(ctx, BTDF_EINVAL, "bad body index");
    if (ctx->cfg.bc_x == kBcxInout) {
        const int S = ctx->width;
        for (const Body& B : ctx->bodies)
            for (int l = 0; l < B.n; l++) {
                const int i0 = (int)std::floor(B.X[l] - 0.5 * S) + 1;
                if (i0 < 1 || i0 + S - 1 > ctx->cfg.nx - 2)
                    return fail(ctx, BTDF_EINVAL, "a marker support reaches the inlet or outlet column");
            }
    }
    if (every > nsteps) every = (int32_t)nsteps;
    const int nck = (int)((nsteps + every - 1) / every);
    int rc = tape_alloc(ctx, nck, every, nsteps);
    if (rc != BTDF_OK) return rc;
    AdjointTape& T = ctx->tape;
    T.pending = false;
    T.nsteps = nsteps;
    T.every = every;
    T.nck = nck;
    T.body = body;
    T.dref = dref;
    T.post0 = ctx->poststream;

    // per-marker tables of the objective and of the position derivatives
    const int nm = ctx->nmark;
    std::vector<BodyDesc> descs;
    std::vector<float> cscale(nm);
    std::vector<float2> objw(nm, make_float2(0.f, 0.f));
    const double q = 0.5 * ctx->cfg.u_in * ctx->cfg.u_in * dref;
    for (int b = 0; b < (int)ctx->bodies.size(); b++) {
        const Body& B = ctx->bodies[b];
        descs.push_back(BodyDesc{B.n, B.ds, B.drs, B.X.data(), B.Y.data(), B.Ubx.data(), B.Uby.data(), b});
        for (int l = 0; l < B.n; l++) {
            cscale[B.first + l] = (float)(B.ds * B.drs);
            if (body < 0 || body == b)   // Cd = -c sum F_x / (U^2 D / 2), averaged over the window
                objw[B.first + l].x = (float)(-B.ds * B.drs / (q * (double)nsteps));
        }
    }
    std::vector<AdjMarker> am;
    build_adjoint_markers(ctx->cfg.nx, ctx->cfg.ny, ctx->cfg.delta, ctx->width,
                          ctx->cfg.bc_x == kBcxPeriodic, ctx->cfg.bc_y == kBcyPeriodic, descs, am);
    cudaStream_t st = ctx->stream;
    CK(cudaMemcpyAsync(T.am, am.data(), sizeof(AdjMarker) * nm, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(T.cscale, cscale.data(), sizeof(float) * nm, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(T.objw, objw.data(), sizeof(float2) * nm, cudaMemcpyHostToDevice, st));
    if (!ctx->band_keys.empty())
        CK(cudaMemcpyAsync(T.band_keys, ctx->band_keys.data(), sizeof(int) * ctx->band_keys.size(),
                           cudaMemcpyHostToDevice, st));

    // forward window from the context's state, checkpoints every `every` steps
    CK(cudaMemcpyAsync(T.ck, ctx->g[ctx->cur], sizeof(float) * T.state_elems, cudaMemcpyDeviceToDevice, st));
    rc = tape_graph_launch(ctx, false);
    if (rc != BTDF_OK) return rc;
    std::vector<float2> F((size_t)nsteps * nm);
    CK(cudaMemcpyAsync(F.data(), T.Fall, sizeof(float2) * F.size(), cudaMemcpyDeviceToHost, st));
    rc = read_status(ctx);
    if (rc != BTDF_OK) return rc;
    double acc = 0.0;
    for (int64_t n = 0; n < nsteps; n++)
        for (int b = 0; b < (int)ctx->bodies.size(); b++) {
            if (body >= 0 && body != b) continue;
            const Body& B = ctx->bodies[b];
            double sx = 0.0;
            for (int l = 0; l < B.n; l++) sx += (double)F[(size_t)n * nm + B.first + l].x;
            acc += -sx * B.ds * B.drs;
        }
    T.J = acc / (q * (double)nsteps);
    T.pending = true;
    if (J) *J = T.J;
    return BTDF_OK;
}

int btdf_adjoint_backward(btdf_ctx* ctx, double* dJdU, double* dJdX, double* dJdY) {
    if (!ctx) return BTDF_EINVAL;
    AdjointTape& T = ctx->tape;
    if (!T.pending) return fail(ctx, BTDF_ESTATE, "no forward window to reverse");
    cudaStream_t st = ctx->stream;
    const int nm = ctx->nmark;
    const int rg = tape_graph_launch(ctx, true);
    if (rg != BTDF_OK) return rg;
    std::vector<double> acc(2 * (size_t)nm + 1);
    CK(cudaMemcpyAsync(acc.data(), T.acc, sizeof(double) * acc.size(), cudaMemcpyDeviceToHost, st));
    const int rc = read_status(ctx);
    if (rc != BTDF_OK) return rc;
    if (dJdU) *dJdU = acc[2 * (size_t)nm] - 2.0 * T.J / ctx->cfg.u_in;   // inlet + 1 / (U^2 D / 2)
    for (int l = 0; l < nm; l++) {
        if (dJdX) dJdX[l] = acc[l];
        if (dJdY) dJdY[l] = acc[(size_t)nm + l];
    }
    return BTDF_OK;
}

int btdf_adjoint_release(btdf_ctx* ctx) {
    if (!ctx) return BTDF_EINVAL;
    CK(cudaStreamSynchronize(ctx->stream));
    free_tape(ctx);
    return BTDF_OK;
}

int btdf_autotune(btdf_ctx* ctx, int32_t steps, int32_t flush_l2, int32_t* chosen, float* ms) {
    if (!ctx) return BTDF_EINVAL;
    if (!ctx->has_fields) return fail(ctx, BTDF_ESTATE, "call btdf_init_fields or btdf_load_state first");
    if (steps < 1 || steps > 100000) return fail(ctx, BTDF_EINVAL, "need 1 <= steps <= 100000");
    cudaStream_t st = ctx->stream;
    CK(cudaStreamSynchronize(st));
    const int rc0 = read_status(ctx);
    if (rc0 != BTDF_OK) return rc0;
    // save what the timing steps change
    const int cur0 = ctx->cur, var0 = ctx->variant;
    const bool post0 = ctx->poststream;
    const int64_t steps0 = ctx->steps;
    unsigned long long counter0 = 0;
    const size_t pbytes = (size_t)9 * ctx->plane * ctx->elem;
    const size_t fbytes = sizeof(float2) * (size_t)ctx->nmark;
    void* save = nullptr;
    void* flush = nullptr;
    double2* th = nullptr;
    float2* fsave = nullptr;
    const size_t nb = std::max<size_t>(ctx->bodies.size(), 1);
    std::vector<cudaEvent_t> ev;
    float res[kVarCount];
    for (int v = 0; v < kVarCount; v++) res[v] = -1.0f;
    int best = kVarReg4;
    auto run = [&]() -> int {
        CK(cudaMalloc(&save, pbytes));
        CK(cudaMalloc((void**)&th, sizeof(double2) * nb));
        if (fbytes) CK(cudaMalloc((void**)&fsave, 4 * fbytes));
        if (flush_l2) CK(cudaMalloc(&flush, l2_flush_bytes()));
        CK(cudaMemcpyAsync(&counter0, ctx->d_step, sizeof(counter0), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(save, ctx->g[cur0], pbytes, cudaMemcpyDeviceToDevice, st));
        if (fbytes) {
            CK(cudaMemcpyAsync(fsave, ctx->d_F[0], fbytes, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(fsave + ctx->nmark, ctx->d_F[1], fbytes, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(fsave + 2 * ctx->nmark, ctx->d_Us, fbytes, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(fsave + 3 * ctx->nmark, ctx->d_rhol, sizeof(float) * ctx->nmark,
                               cudaMemcpyDeviceToDevice, st));
        }
        ctx->tune_hist = th;
        ev.resize(2 * (size_t)steps);
        for (auto& e : ev) CK(cudaEventCreate(&e));
        if (ctx->poststream) {   // time pull steps only
            int rc = enqueue_step(ctx, st, false, ctx->cur, false);
            if (rc != BTDF_OK) return rc;
            ctx->cur = 1 - ctx->cur;
            ctx->poststream = false;
        }
        float best_ms = 0.f;
        for (int v = 1; v < kVarCount; v++) {
            if (is_tma(v) && !ctx->tma_ok) continue;
            ctx->variant = v;
            for (int i = 0; i < 3; i++) {
                int rc = enqueue_step(ctx, st, true, ctx->cur, false);
                if (rc != BTDF_OK) return rc;
                ctx->cur = 1 - ctx->cur;
            }
            for (int i = 0; i < steps; i++) {
                if (flush) CK(launch_l2_flush(flush, l2_flush_bytes(), st));
                CK(cudaEventRecord(ev[2 * i], st));
                int rc = enqueue_step(ctx, st, true, ctx->cur, false);
                if (rc != BTDF_OK) return rc;
                CK(cudaEventRecord(ev[2 * i + 1], st));
                ctx->cur = 1 - ctx->cur;
            }
            CK(cudaStreamSynchronize(st));
            std::vector<float> t(steps);
            for (int i = 0; i < steps; i++) CK(cudaEventElapsedTime(&t[i], ev[2 * i], ev[2 * i + 1]));
            res[v] = interquartile_mean(t);
            if (v == 1 || res[v] < best_ms) {
                best_ms = res[v];
                best = v;
            }
        }
        return BTDF_OK;
    };
    int rc = run();
    // restore the state, the counter and the last step's marker results
    ctx->tune_hist = nullptr;
    ctx->variant = rc == BTDF_OK ? best : var0;
    ctx->cur = cur0;
    ctx->poststream = post0;
    ctx->steps = steps0;
    cudaError_t e = cudaSuccess;
    if (save) {
        e = cudaMemcpyAsync(ctx->g[cur0], save, pbytes, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->d_step, &counter0, sizeof(counter0), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && fsave) {
            cudaMemcpyAsync(ctx->d_F[0], fsave, fbytes, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(ctx->d_F[1], fsave + ctx->nmark, fbytes, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(ctx->d_Us, fsave + 2 * ctx->nmark, fbytes, cudaMemcpyDeviceToDevice, st);
            e = cudaMemcpyAsync(ctx->d_rhol, fsave + 3 * ctx->nmark, sizeof(float) * ctx->nmark,
                                cudaMemcpyDeviceToDevice, st);
        }
    }
    cudaStreamSynchronize(st);
    for (auto& ev1 : ev)
        if (ev1) cudaEventDestroy(ev1);
    if (save) cudaFree(save);
    if (flush) cudaFree(flush);
    if (th) cudaFree(th);
    if (fsave) cudaFree(fsave);
    drop_graphs(ctx);
    if (rc != BTDF_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "restoring the state after tuning");
    if (chosen) *chosen = best;
    if (ms)
        for (int v = 0; v < kVarCount; v++) ms[v] = res[v];
    return read_status(ctx);
}

int btdf_device_bytes(const btdf_ctx* ctx, size_t* bytes) {
    if (!ctx || !bytes) return BTDF_EINVAL;
    *bytes = ctx->dev_bytes;
    return BTDF_OK;
}

}  // extern "C"
