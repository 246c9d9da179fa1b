// btdf_batch.cu - host side of the batched form: many independent lattices
// (each with its own size, relaxation time, inflow and bodies) advanced
// together, one IB launch and one persistent LBM launch per time step,
// replayed through CUDA graphs.  Same arithmetic as a single context.
#include "btdf.h"
#include "btdf_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

using namespace btdf;

namespace {

constexpr int kBatchGraphSteps = 32;

struct BBody {
    int first = 0, n = 0, lattice = 0;
    double ds = 0.0, drs = 0.0;
    std::vector<double> X, Y, Ubx, Uby;
};

}  // namespace

struct btdf_batch {
    int n = 0;
    std::vector<btdf_config> cfg;
    std::vector<int> nxp, nseg;
    std::vector<long long> plane;
    std::vector<unsigned long long> off;   // element offset of each lattice
    unsigned long long total = 0;          // elements per population buffer
    int storage = 0, layout = 0, delta = 3, width = 3, history_len = 1;
    size_t elem = 4;
    cudaStream_t stream = nullptr, cap = nullptr;
    void* g[2] = {nullptr, nullptr};
    int cur = 0;
    bool poststream = true;
    std::vector<char> has_fields;
    int64_t steps = 0, hist_from = 0;
    // launch shape: 1 / 2 = 4 / 2 nodes per lane on a persistent grid of
    // balanced unit ranges; 3 / 4 = the same with one unit per CTA
    int variant = 1;
    int grid[2] = {1, 1};
    int sms = 1;

    std::vector<BBody> bodies;
    int nmark = 0;
    LatticeParams* d_descs = nullptr;
    unsigned long long* d_off = nullptr;
    int2* d_units[4] = {nullptr, nullptr, nullptr, nullptr};   // per launch shape
    int* d_cta[4] = {nullptr, nullptr, nullptr, nullptr};
    int grid_used[4] = {1, 1, 1, 1};
    Marker* d_mk = nullptr;
    MarkerAux* d_aux = nullptr;
    float2* d_F = nullptr;
    float2* d_Us = nullptr;
    float* d_rhol = nullptr;
    int* d_seg_index = nullptr;
    int* d_seg_ptr = nullptr;
    CsrEntry* d_csr = nullptr;
    int* d_body_ptr = nullptr;
    double* d_body_scale = nullptr;
    double2* d_hist = nullptr;
    unsigned long long* d_step = nullptr;
    unsigned int* d_done = nullptr;
    int* d_status = nullptr;
    std::vector<LatticeParams> descs;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    std::string err;
    double2* tune_hist = nullptr;          // one-slot force ring while btdf_batch_autotune times steps
};

namespace {

int bfail(btdf_batch* b, int code, const std::string& msg) {
    if (b) b->err = msg;
    return code;
}

#define BCK(call)                                                                      \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return bfail(bt, BTDF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename P>
void bfree(P*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

void drop_graphs(btdf_batch* bt) {
    for (auto& ge : bt->gexec)
        if (ge) {
            cudaGraphExecDestroy(ge);
            ge = nullptr;
        }
}

void free_marker_data(btdf_batch* bt) {
    bfree(bt->d_mk);
    bfree(bt->d_aux);
    bfree(bt->d_F);
    bfree(bt->d_Us);
    bfree(bt->d_rhol);
    bfree(bt->d_seg_index);
    bfree(bt->d_seg_ptr);
    bfree(bt->d_csr);
    bfree(bt->d_body_ptr);
    bfree(bt->d_body_scale);
    bfree(bt->d_hist);
}

// Lattice description of lattice c (the same fields a single context uses).
LatticeParams base_params(const btdf_batch* bt, int c) {
    const btdf_config& k = bt->cfg[c];
    LatticeParams p{};
    p.wait_polls = -1;   // default bound of the bounded waits
    p.nx = k.nx;
    p.ny = k.ny;
    p.nxp = bt->nxp[c];
    p.nseg = bt->nseg[c];
    p.plane = bt->plane[c];
    p.rs = bt->layout == BTDF_LAYOUT_ROWS ? 9u * (unsigned)bt->nxp[c] : (unsigned)bt->nxp[c];
    for (int a = 0; a < 9; a++)
        p.poff[a] = bt->layout == BTDF_LAYOUT_ROWS ? (unsigned)(a * bt->nxp[c])
                                                   : (unsigned)(a * bt->plane[c]);
    p.bcx = k.bc_x;
    p.bcy = k.bc_y;
    p.omega = (float)(1.0 / k.tau);
    p.guo = (float)(1.0 - 0.5 / k.tau);
    p.u_in = (float)k.u_in;
    p.urx = (float)k.u_in;
    p.ury = 0.0f;
    const double Ux = k.u_in, Uy = 0.0;
    p.one_m_omega = (float)(1.0 - 1.0 / k.tau);
    for (int a = 0; a < 9; a++) {
        const double w = a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
        const double eU = ex(a) * Ux + ey(a) * Uy;
        p.eur[a] = (float)eU;
        p.c1[a] = (float)(3.0 + 9.0 * eU);
        p.kr[a] = (float)(1.0 + 3.0 * eU + 4.5 * eU * eU - 1.5 * (Ux * Ux + Uy * Uy));
        p.wom[a] = (float)(w / k.tau * store_scale(bt->storage));
        p.wg[a] = (float)(w * (1.0 - 0.5 / k.tau) * store_scale(bt->storage));
    }
    for (int a = 0; a < 9; a++) {
        p.c1p[a] = make_float2(p.c1[a], p.c1[a]);
        p.krp[a] = make_float2(p.kr[a], p.kr[a]);
        p.womp[a] = make_float2(p.wom[a], p.wom[a]);
    }
    p.omop = make_float2(p.one_m_omega, p.one_m_omega);
    p.gx = (float)k.gx;
    p.gy = (float)k.gy;
    p.nwork = (long long)k.ny * bt->nseg[c];
    return p;
}

// Work units (lattice, first row) of 8 rows, and a split into `grid`
// contiguous CTA ranges of nearly equal segment counts.
int shape_npl(int v) { return (v == 2 || v == 4) ? 2 : 4; }

int build_units(btdf_batch* bt, int v) {
    const int npl = shape_npl(v), sw = 32 * npl;
    std::vector<int2> units;
    std::vector<long long> work;
    for (int c = 0; c < bt->n; c++) {
        const int nsegw = (bt->nxp[c] + sw - 1) / sw;
        for (int y = 0; y < bt->cfg[c].ny; y += 8) {
            units.push_back(make_int2(c, y));
            work.push_back((long long)std::min(8, bt->cfg[c].ny - y) * nsegw);
        }
    }
    long long total = 0;
    for (long long w : work) total += w;
    const long long cap = v >= 3 ? (long long)units.size() : (long long)bt->grid[npl == 2 ? 1 : 0];
    const int grid = (int)std::max<long long>(1, std::min<long long>(cap, (long long)units.size()));
    std::vector<int> cta(grid + 1, (int)units.size());
    cta[0] = 0;
    long long acc = 0;
    int b = 1;
    for (size_t u = 0; u < units.size() && b < grid; u++) {
        acc += work[u];
        while (b < grid && acc * grid >= total * b) cta[b++] = (int)u + 1;
    }
    for (; b < grid; b++) cta[b] = (int)units.size();
    const int s = v - 1;
    bfree(bt->d_units[s]);
    bfree(bt->d_cta[s]);
    BCK(cudaMalloc((void**)&bt->d_units[s], sizeof(int2) * std::max<size_t>(units.size(), 1)));
    BCK(cudaMalloc((void**)&bt->d_cta[s], sizeof(int) * (grid + 1)));
    BCK(cudaMemcpy(bt->d_units[s], units.data(), sizeof(int2) * units.size(), cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(bt->d_cta[s], cta.data(), sizeof(int) * (grid + 1), cudaMemcpyHostToDevice));
    bt->grid_used[s] = grid;
    return BTDF_OK;
}

int upload_descs(btdf_batch* bt) {
    BCK(cudaMemcpyAsync(bt->d_descs, bt->descs.data(), sizeof(LatticeParams) * bt->n,
                        cudaMemcpyHostToDevice, bt->stream));
    BCK(cudaStreamSynchronize(bt->stream));
    return BTDF_OK;
}

// Marker tables of every lattice, flattened (marker indices are global).
int rebuild(btdf_batch* bt) {
    drop_graphs(bt);
    free_marker_data(bt);
    for (int c = 0; c < bt->n; c++) {
        LatticeParams& p = bt->descs[c];
        p.seg_index = nullptr;
        p.seg_ptr = nullptr;
        p.csr = nullptr;
        p.F = nullptr;
    }
    const int nm = bt->nmark, nb = (int)bt->bodies.size();
    if (nm == 0) return upload_descs(bt);
    // Flat marker order: by lattice, then by insertion; body ids stay the
    // insertion order.
    std::vector<int> order(nb);
    for (int b = 0; b < nb; b++) order[b] = b;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return bt->bodies[a].lattice < bt->bodies[b].lattice; });
    {
        int first = 0;
        for (int b : order) {
            bt->bodies[b].first = first;
            first += bt->bodies[b].n;
        }
    }
    std::vector<Marker> mk;
    std::vector<MarkerAux> aux;
    std::vector<int> seg_index, seg_ptr;
    std::vector<CsrEntry> csr;
    std::vector<size_t> si_off(bt->n, 0), sp_off(bt->n, 0), cs_off(bt->n, 0);
    std::vector<char> has_band(bt->n, 0);
    for (int c = 0; c < bt->n; c++) {
        std::vector<BodyDesc> bd;
        int base = -1;
        for (int b : order) {
            const BBody& B = bt->bodies[b];
            if (B.lattice != c) continue;
            if (base < 0) base = B.first;
            bd.push_back(BodyDesc{B.n, B.ds, B.drs, B.X.data(), B.Y.data(), B.Ubx.data(),
                                  B.Uby.data(), c});
        }
        if (bd.empty()) continue;
        const btdf_config& k = bt->cfg[c];
        HostTables t;
        build_marker_tables(k.nx, k.ny, bt->nseg[c], bt->delta, bt->width, k.bc_x == kBcxPeriodic,
                            k.bc_y == kBcyPeriodic, k.u_in, bd, base, t);
        mk.insert(mk.end(), t.mk.begin(), t.mk.end());
        aux.insert(aux.end(), t.aux.begin(), t.aux.end());
        si_off[c] = seg_index.size();
        sp_off[c] = seg_ptr.size();
        cs_off[c] = csr.size();
        seg_index.insert(seg_index.end(), t.seg_index.begin(), t.seg_index.end());
        seg_ptr.insert(seg_ptr.end(), t.seg_ptr.begin(), t.seg_ptr.end());
        csr.insert(csr.end(), t.csr.begin(), t.csr.end());
        has_band[c] = 1;
    }
    std::vector<int> body_rng(2 * nb);
    std::vector<double> scale(nb);
    for (int b = 0; b < nb; b++) {
        body_rng[2 * b] = bt->bodies[b].first;
        body_rng[2 * b + 1] = bt->bodies[b].first + bt->bodies[b].n;
        scale[b] = bt->bodies[b].ds * bt->bodies[b].drs;
    }
    BCK(cudaMalloc((void**)&bt->d_mk, sizeof(Marker) * nm));
    BCK(cudaMalloc((void**)&bt->d_aux, sizeof(MarkerAux) * nm));
    BCK(cudaMalloc((void**)&bt->d_F, sizeof(float2) * nm));
    BCK(cudaMalloc((void**)&bt->d_Us, sizeof(float2) * nm));
    BCK(cudaMalloc((void**)&bt->d_rhol, sizeof(float) * nm));
    BCK(cudaMalloc((void**)&bt->d_seg_index, sizeof(int) * std::max<size_t>(seg_index.size(), 1)));
    BCK(cudaMalloc((void**)&bt->d_seg_ptr, sizeof(int) * std::max<size_t>(seg_ptr.size(), 1)));
    BCK(cudaMalloc((void**)&bt->d_csr, sizeof(CsrEntry) * std::max<size_t>(csr.size(), 1)));
    BCK(cudaMalloc((void**)&bt->d_body_ptr, sizeof(int) * 2 * nb));
    BCK(cudaMalloc((void**)&bt->d_body_scale, sizeof(double) * nb));
    BCK(cudaMalloc((void**)&bt->d_hist, sizeof(double2) * (size_t)bt->history_len * nb));
    cudaStream_t st = bt->stream;
    BCK(cudaMemcpyAsync(bt->d_mk, mk.data(), sizeof(Marker) * nm, cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync(bt->d_aux, aux.data(), sizeof(MarkerAux) * nm, cudaMemcpyHostToDevice, st));
    BCK(cudaMemsetAsync(bt->d_F, 0, sizeof(float2) * nm, st));
    BCK(cudaMemsetAsync(bt->d_Us, 0, sizeof(float2) * nm, st));
    BCK(cudaMemsetAsync(bt->d_rhol, 0, sizeof(float) * nm, st));
    if (!seg_index.empty())
        BCK(cudaMemcpyAsync(bt->d_seg_index, seg_index.data(), sizeof(int) * seg_index.size(),
                            cudaMemcpyHostToDevice, st));
    if (!seg_ptr.empty())
        BCK(cudaMemcpyAsync(bt->d_seg_ptr, seg_ptr.data(), sizeof(int) * seg_ptr.size(),
                            cudaMemcpyHostToDevice, st));
    if (!csr.empty())
        BCK(cudaMemcpyAsync(bt->d_csr, csr.data(), sizeof(CsrEntry) * csr.size(),
                            cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync(bt->d_body_ptr, body_rng.data(), sizeof(int) * 2 * nb, cudaMemcpyHostToDevice,
                        st));
    BCK(cudaMemcpyAsync(bt->d_body_scale, scale.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, st));
    BCK(cudaMemsetAsync(bt->d_hist, 0, sizeof(double2) * (size_t)bt->history_len * nb, st));
    for (int c = 0; c < bt->n; c++) {
        if (!has_band[c]) continue;
        LatticeParams& p = bt->descs[c];
        p.seg_index = bt->d_seg_index + si_off[c];
        p.seg_ptr = bt->d_seg_ptr + sp_off[c];
        p.csr = bt->d_csr + cs_off[c];
        p.F = bt->d_F;
    }
    bt->hist_from = bt->steps;
    return upload_descs(bt);
}

BatchLbm lbm_params(const btdf_batch* bt, int s) {
    BatchLbm b{};
    b.descs = bt->d_descs;
    b.case_off = bt->d_off;
    b.units = bt->d_units[s];
    b.cta_units = bt->d_cta[s];
    b.nbody = bt->nmark > 0 ? (int)bt->bodies.size() : 0;
    b.hist_len = bt->history_len;
    b.body_rng = bt->d_body_ptr;
    b.body_scale = bt->d_body_scale;
    b.hist = bt->d_hist;
    if (bt->tune_hist) {   // timing steps must not overwrite the force history
        b.hist_len = 1;
        b.hist = bt->tune_hist;
    }
    b.F = bt->d_F;
    b.step = bt->d_step;
    b.done = bt->d_done;
    return b;
}

int enqueue(btdf_batch* bt, cudaStream_t st, bool pull, int cur) {
    if (bt->nmark > 0) {
        IbParams q{};
        q.nmark = bt->nmark;
        q.mk = bt->d_mk;
        q.aux = bt->d_aux;
        q.F_prev = nullptr;
        q.F_out = bt->d_F;
        q.Us = bt->d_Us;
        q.rhol = bt->d_rhol;
        q.first_pass = 1;
        q.status = bt->d_status;
        BCK(launch_ib_force_batch(bt->storage, pull, bt->width, bt->g[cur], bt->d_descs, bt->d_off, q, st));
    }
    const int s = bt->variant - 1;
    BCK(launch_collide_stream_batch(bt->storage, pull, shape_npl(bt->variant), bt->g[cur],
                                    bt->g[1 - cur], lbm_params(bt, s), bt->grid_used[s],
                                    bt->nmark > 0, st));
    return BTDF_OK;
}

int ensure_graph(btdf_batch* bt, int cur) {
    if (bt->gexec[cur]) return BTDF_OK;
    cudaGraph_t graph = nullptr;
    BCK(cudaStreamBeginCapture(bt->cap, cudaStreamCaptureModeThreadLocal));
    int rc = BTDF_OK;
    int c = cur;
    for (int i = 0; i < kBatchGraphSteps && rc == BTDF_OK; i++) {
        rc = enqueue(bt, bt->cap, true, c);
        c = 1 - c;
    }
    cudaError_t e = cudaStreamEndCapture(bt->cap, &graph);
    if (rc != BTDF_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return bfail(bt, BTDF_ECUDA, "cudaStreamEndCapture failed");
    e = cudaGraphInstantiate(&bt->gexec[cur], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bfail(bt, BTDF_ECUDA, "cudaGraphInstantiate failed");
    return BTDF_OK;
}

int bstatus(btdf_batch* bt) {
    int st = 0;
    BCK(cudaMemcpyAsync(&st, bt->d_status, sizeof(int), cudaMemcpyDeviceToHost, bt->stream));
    BCK(cudaStreamSynchronize(bt->stream));
    if (st & kStatusUnstable)
        return bfail(bt, BTDF_EUNSTABLE, "non-positive or non-finite density or force at a marker");
    return BTDF_OK;
}

}  // namespace

extern "C" {

int btdf_batch_create(const btdf_config* cfgs, int32_t n, void* stream, btdf_batch** out) {
    if (!cfgs || !out || n < 1) return BTDF_EINVAL;
    *out = nullptr;
    const btdf_config& c0 = cfgs[0];
    unsigned long long total = 0;
    for (int c = 0; c < n; c++) {
        const btdf_config& k = cfgs[c];
        const int w = k.delta == 2 ? 2 : k.delta == 3 ? 3 : (k.delta == 4 || k.delta == 5) ? 4 : 0;
        if (k.nx < 4 || k.ny < 4 || !(k.tau > 0.5) || !std::isfinite(k.tau) || w == 0 ||
            k.storage < 0 || k.storage > 2 || k.bc_x < 0 || k.bc_x > 1 || k.bc_y < 0 || k.bc_y > 2 ||
            k.history_len < 1 || !std::isfinite(k.u_in) || std::fabs(k.u_in) >= 0.5 ||
            !std::isfinite(k.gx) || !std::isfinite(k.gy) ||
            (k.layout != BTDF_LAYOUT_PLANES && k.layout != BTDF_LAYOUT_ROWS))
            return BTDF_EINVAL;
        // one storage, layout, delta function and forcing scheme for the whole batch
        if (k.storage != c0.storage || k.layout != c0.layout || k.delta != c0.delta || k.nf != 1 ||
            k.history_len != c0.history_len)
            return BTDF_EINVAL;
        const long long nxp = ((long long)k.nx + 31) / 32 * 32;
        if (9ll * nxp * k.ny >= (1ll << 32)) return BTDF_EINVAL;
        total += 9ull * nxp * k.ny;
    }
    btdf_batch* bt = new (std::nothrow) btdf_batch();
    if (!bt) return BTDF_ENOMEM;
    bt->n = n;
    bt->cfg.assign(cfgs, cfgs + n);
    bt->storage = c0.storage;
    bt->layout = c0.layout;
    bt->delta = c0.delta;
    bt->width = c0.delta == 2 ? 2 : c0.delta == 3 ? 3 : 4;
    bt->history_len = c0.history_len;
    bt->elem = c0.storage == kStoreF32 ? 4 : 2;
    bt->stream = (cudaStream_t)stream;
    bt->has_fields.assign(n, 0);
    unsigned long long acc = 0;
    for (int c = 0; c < n; c++) {
        const int nxp = (cfgs[c].nx + 31) / 32 * 32;
        bt->nxp.push_back(nxp);
        bt->nseg.push_back((nxp + kSeg - 1) / kSeg);
        bt->plane.push_back((long long)nxp * cfgs[c].ny);
        bt->off.push_back(acc);
        acc += 9ull * nxp * cfgs[c].ny;
        // lattices start on 128-element boundaries so every vector access stays aligned
        acc = (acc + 127) / 128 * 128;
    }
    bt->total = acc;
    auto bail = [&](int code) {
        btdf_batch_destroy(bt);
        return code;
    };
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&bt->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bail(BTDF_ECUDA);
    bt->grid[0] = bt->sms * collide_stream_batch_blocks_per_sm(bt->storage, 4);
    bt->grid[1] = bt->sms * collide_stream_batch_blocks_per_sm(bt->storage, 2);
    if (cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking) != cudaSuccess) return bail(BTDF_ECUDA);
    for (int i = 0; i < 2; i++) {
        cudaError_t e = cudaMalloc(&bt->g[i], bt->total * bt->elem);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return bail(e == cudaErrorMemoryAllocation ? BTDF_ENOMEM : BTDF_ECUDA);
        }
        if (cudaMemsetAsync(bt->g[i], 0, bt->total * bt->elem, bt->stream) != cudaSuccess)
            return bail(BTDF_ECUDA);
    }
    if (cudaMalloc((void**)&bt->d_descs, sizeof(LatticeParams) * n) != cudaSuccess ||
        cudaMalloc((void**)&bt->d_off, sizeof(unsigned long long) * n) != cudaSuccess ||
        cudaMalloc((void**)&bt->d_step, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc((void**)&bt->d_done, sizeof(unsigned int)) != cudaSuccess ||
        cudaMalloc((void**)&bt->d_status, sizeof(int)) != cudaSuccess)
        return bail(BTDF_ECUDA);
    if (cudaMemcpy(bt->d_off, bt->off.data(), sizeof(unsigned long long) * n, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemset(bt->d_step, 0, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(bt->d_done, 0, sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(bt->d_status, 0, sizeof(int)) != cudaSuccess)
        return bail(BTDF_ECUDA);
    bt->descs.resize(n);
    for (int c = 0; c < n; c++) bt->descs[c] = base_params(bt, c);
    if (build_units(bt, 1) != BTDF_OK || build_units(bt, 2) != BTDF_OK || build_units(bt, 3) != BTDF_OK ||
        build_units(bt, 4) != BTDF_OK || rebuild(bt) != BTDF_OK)
        return bail(BTDF_ECUDA);
    *out = bt;
    return BTDF_OK;
}

int btdf_batch_destroy(btdf_batch* bt) {
    if (!bt) return BTDF_EINVAL;
    cudaStreamSynchronize(bt->stream);
    drop_graphs(bt);
    free_marker_data(bt);
    bfree(bt->g[0]);
    bfree(bt->g[1]);
    bfree(bt->d_descs);
    bfree(bt->d_off);
    for (int s = 0; s < 4; s++) {
        bfree(bt->d_units[s]);
        bfree(bt->d_cta[s]);
    }
    bfree(bt->d_step);
    bfree(bt->d_done);
    bfree(bt->d_status);
    if (bt->cap) cudaStreamDestroy(bt->cap);
    delete bt;
    return BTDF_OK;
}

int btdf_batch_init_fields(btdf_batch* bt, int32_t c, const double* rho, const double* ux,
                           const double* uy) {
    if (!bt) return BTDF_EINVAL;
    if (c < 0 || c >= bt->n || !rho || !ux || !uy) return bfail(bt, BTDF_EINVAL, "bad lattice or null field");
    if (bt->steps > 0 || !bt->poststream)
        return bfail(bt, BTDF_ESTATE, "fields are set before the first step");
    const size_t nn = (size_t)bt->cfg[c].nx * bt->cfg[c].ny;
    for (size_t i = 0; i < nn; i++)
        if (!(rho[i] > 0.0) || !std::isfinite(rho[i]) || !std::isfinite(ux[i]) || !std::isfinite(uy[i]))
            return bfail(bt, BTDF_EINVAL, "initial fields must be finite with rho > 0");
    double* d = nullptr;
    BCK(cudaMalloc((void**)&d, sizeof(double) * 3 * nn));
    cudaStream_t st = bt->stream;
    cudaError_t e = cudaMemcpyAsync(d, rho, sizeof(double) * nn, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + nn, ux, sizeof(double) * nn, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + 2 * nn, uy, sizeof(double) * nn, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_init_equilibrium(bt->storage, (char*)bt->g[0] + bt->off[c] * bt->elem, bt->descs[c], d,
                                    d + nn, d + 2 * nn, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    if (e != cudaSuccess) return bfail(bt, BTDF_ECUDA, std::string("init: ") + cudaGetErrorString(e));
    bt->has_fields[c] = 1;
    return BTDF_OK;
}

int btdf_batch_add_markers(btdf_batch* bt, int32_t c, int32_t n, const double* X, const double* Y,
                           const double* Ubx, const double* Uby, double ds, double drs, int32_t* body_id) {
    if (!bt) return BTDF_EINVAL;
    if (c < 0 || c >= bt->n || n < 1 || !X || !Y || !(ds > 0.0) || !std::isfinite(drs))
        return bfail(bt, BTDF_EINVAL, "bad lattice, marker count, positions or ds");
    if (bt->steps > 0) return bfail(bt, BTDF_ESTATE, "markers are added before the first step");
    const btdf_config& k = bt->cfg[c];
    const double half = 0.5 * bt->width;
    for (int l = 0; l < n; l++) {
        if (!std::isfinite(X[l]) || !std::isfinite(Y[l]) || (Ubx && !std::isfinite(Ubx[l])) ||
            (Uby && !std::isfinite(Uby[l])))
            return bfail(bt, BTDF_EINVAL, "marker data not finite");
        const bool inx = k.bc_x == kBcxPeriodic ? std::fabs(X[l]) <= 1e9 : (X[l] > -half && X[l] < k.nx - 1 + half);
        const bool iny = k.bc_y == kBcyPeriodic ? std::fabs(Y[l]) <= 1e9 : (Y[l] > -half && Y[l] < k.ny - 1 + half);
        if (!inx || !iny) return bfail(bt, BTDF_EINVAL, "marker support lies outside the lattice");
    }
    BBody B;
    B.lattice = c;
    B.n = n;
    B.ds = ds;
    B.drs = drs > 0.0 ? drs : (bt->delta == 2 ? 1.4 : bt->delta == 3 ? 1.9 : 2.6);
    B.X.assign(X, X + n);
    B.Y.assign(Y, Y + n);
    B.Ubx.assign(n, 0.0);
    B.Uby.assign(n, 0.0);
    if (Ubx) B.Ubx.assign(Ubx, Ubx + n);
    if (Uby) B.Uby.assign(Uby, Uby + n);
    bt->bodies.push_back(std::move(B));
    bt->nmark += n;
    const int rc = rebuild(bt);
    if (rc != BTDF_OK) return rc;
    if (body_id) *body_id = (int)bt->bodies.size() - 1;
    return BTDF_OK;
}

int btdf_batch_body_count(const btdf_batch* bt, int32_t* n) {
    if (!bt || !n) return BTDF_EINVAL;
    *n = (int)bt->bodies.size();
    return BTDF_OK;
}

int btdf_batch_body_lattice(const btdf_batch* bt, int32_t body, int32_t* lattice) {
    if (!bt || !lattice || body < 0 || body >= (int)bt->bodies.size()) return BTDF_EINVAL;
    *lattice = bt->bodies[body].lattice;
    return BTDF_OK;
}

int btdf_batch_tune(btdf_batch* bt, int32_t variant) {
    if (!bt) return BTDF_EINVAL;
    if (variant < 0 || variant > 4) return bfail(bt, BTDF_EINVAL, "variant must be 0 .. 4");
    BCK(cudaStreamSynchronize(bt->stream));
    drop_graphs(bt);
    bt->variant = variant == 0 ? 1 : variant;
    return BTDF_OK;
}

int btdf_batch_autotune(btdf_batch* bt, int32_t steps, int32_t flush_l2, int32_t* chosen, float* ms) {
    if (!bt) return BTDF_EINVAL;
    if (steps < 1 || steps > 100000) return bfail(bt, BTDF_EINVAL, "need 1 <= steps <= 100000");
    for (int c = 0; c < bt->n; c++)
        if (!bt->has_fields[c]) return bfail(bt, BTDF_ESTATE, "every lattice needs btdf_batch_init_fields");
    cudaStream_t st = bt->stream;
    BCK(cudaStreamSynchronize(st));
    const int rc0 = bstatus(bt);
    if (rc0 != BTDF_OK) return rc0;
    const int cur0 = bt->cur, var0 = bt->variant;
    const bool post0 = bt->poststream;
    unsigned long long counter0 = 0;
    const size_t pbytes = (size_t)bt->total * bt->elem;   // total counts all nine planes
    const size_t fbytes = sizeof(float2) * (size_t)bt->nmark;
    void* save = nullptr;
    void* flush = nullptr;
    double2* th = nullptr;
    float2* fsave = nullptr;
    std::vector<cudaEvent_t> ev;
    float res[5] = {-1.0f, -1.0f, -1.0f, -1.0f, -1.0f};
    int best = 1;
    auto run = [&]() -> int {
        BCK(cudaMalloc(&save, pbytes));
        BCK(cudaMalloc((void**)&th, sizeof(double2) * std::max<size_t>(bt->bodies.size(), 1)));
        if (fbytes) BCK(cudaMalloc((void**)&fsave, fbytes));
        if (flush_l2) BCK(cudaMalloc(&flush, l2_flush_bytes()));
        BCK(cudaMemcpyAsync(&counter0, bt->d_step, sizeof(counter0), cudaMemcpyDeviceToHost, st));
        BCK(cudaMemcpyAsync(save, bt->g[cur0], pbytes, cudaMemcpyDeviceToDevice, st));
        if (fbytes) BCK(cudaMemcpyAsync(fsave, bt->d_F, fbytes, cudaMemcpyDeviceToDevice, st));
        bt->tune_hist = th;
        ev.resize(2 * (size_t)steps);
        for (auto& e : ev) BCK(cudaEventCreate(&e));
        if (bt->poststream) {   // time pull steps only
            const int rc = enqueue(bt, st, false, bt->cur);
            if (rc != BTDF_OK) return rc;
            bt->cur = 1 - bt->cur;
            bt->poststream = false;
        }
        for (int v = 1; v <= 4; v++) {
            bt->variant = v;
            for (int i = 0; i < 3; i++) {
                const int rc = enqueue(bt, st, true, bt->cur);
                if (rc != BTDF_OK) return rc;
                bt->cur = 1 - bt->cur;
            }
            for (int i = 0; i < steps; i++) {
                if (flush) BCK(launch_l2_flush(flush, l2_flush_bytes(), st));
                BCK(cudaEventRecord(ev[2 * i], st));
                const int rc = enqueue(bt, st, true, bt->cur);
                if (rc != BTDF_OK) return rc;
                BCK(cudaEventRecord(ev[2 * i + 1], st));
                bt->cur = 1 - bt->cur;
            }
            BCK(cudaStreamSynchronize(st));
            std::vector<float> t(steps);
            for (int i = 0; i < steps; i++) BCK(cudaEventElapsedTime(&t[i], ev[2 * i], ev[2 * i + 1]));
            res[v] = interquartile_mean(t);
            if (v == 1 || res[v] < res[best]) best = v;
        }
        return BTDF_OK;
    };
    const int rc = run();
    bt->tune_hist = nullptr;
    bt->variant = rc == BTDF_OK ? best : var0;
    bt->cur = cur0;
    bt->poststream = post0;
    cudaError_t e = cudaSuccess;
    if (save) {
        e = cudaMemcpyAsync(bt->g[cur0], save, pbytes, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(bt->d_step, &counter0, sizeof(counter0), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && fsave) e = cudaMemcpyAsync(bt->d_F, fsave, fbytes, cudaMemcpyDeviceToDevice, st);
    }
    cudaStreamSynchronize(st);
    for (auto& ev1 : ev)
        if (ev1) cudaEventDestroy(ev1);
    if (save) cudaFree(save);
    if (flush) cudaFree(flush);
    if (th) cudaFree(th);
    if (fsave) cudaFree(fsave);
    drop_graphs(bt);
    if (rc != BTDF_OK) return rc;
    if (e != cudaSuccess) return bfail(bt, BTDF_ECUDA, "restoring the state after tuning");
    if (chosen) *chosen = best;
    if (ms)
        for (int v = 0; v < 5; v++) ms[v] = res[v];
    return bstatus(bt);
}

int btdf_batch_step(btdf_batch* bt, int64_t nsteps) {
    if (!bt) return BTDF_EINVAL;
    if (nsteps < 0) return bfail(bt, BTDF_EINVAL, "nsteps < 0");
    for (int c = 0; c < bt->n; c++)
        if (!bt->has_fields[c]) return bfail(bt, BTDF_ESTATE, "every lattice needs btdf_batch_init_fields");
    int64_t i = 0;
    if (nsteps > 0 && bt->poststream) {
        const int rc = enqueue(bt, bt->stream, false, bt->cur);
        if (rc != BTDF_OK) return rc;
        bt->cur = 1 - bt->cur;
        bt->poststream = false;
        i = 1;
    }
    while (nsteps - i >= kBatchGraphSteps) {
        const int rc = ensure_graph(bt, bt->cur);
        if (rc != BTDF_OK) return rc;
        BCK(cudaGraphLaunch(bt->gexec[bt->cur], bt->stream));
        i += kBatchGraphSteps;
    }
    for (; i < nsteps; i++) {
        const int rc = enqueue(bt, bt->stream, true, bt->cur);
        if (rc != BTDF_OK) return rc;
        bt->cur = 1 - bt->cur;
    }
    bt->steps += nsteps;
    return BTDF_OK;
}

int btdf_batch_sync(btdf_batch* bt) {
    if (!bt) return BTDF_EINVAL;
    BCK(cudaStreamSynchronize(bt->stream));
    return bstatus(bt);
}

int64_t btdf_batch_step_count(const btdf_batch* bt) { return bt ? bt->steps : -1; }

int btdf_batch_read_forces(btdf_batch* bt, int32_t body, int64_t first, int64_t n, double* Fx, double* Fy) {
    if (!bt) return BTDF_EINVAL;
    const int nb = (int)bt->bodies.size();
    if (body < 0 || body >= nb || n < 0 || (n > 0 && (!Fx || !Fy)))
        return bfail(bt, BTDF_EINVAL, "bad body, count or null output");
    const int64_t H = bt->history_len;
    if (first < bt->hist_from || first < bt->steps - H || first + n > bt->steps)
        return bfail(bt, BTDF_EINVAL, "requested steps are not in the force history");
    std::vector<double2> tmp((size_t)n);
    int64_t done = 0;
    while (done < n) {
        const int64_t s = first + done, slot = s % H;
        const int64_t cnt = std::min<int64_t>(n - done, H - slot);
        BCK(cudaMemcpy2DAsync(tmp.data() + done, sizeof(double2), bt->d_hist + slot * nb + body,
                              sizeof(double2) * nb, sizeof(double2), (size_t)cnt, cudaMemcpyDeviceToHost,
                              bt->stream));
        done += cnt;
    }
    const int rc = bstatus(bt);
    for (int64_t i = 0; i < n; i++) {
        Fx[i] = tmp[i].x;
        Fy[i] = tmp[i].y;
    }
    return rc;
}

int btdf_batch_read_field(btdf_batch* bt, int32_t c, int32_t kind, float* dst, int32_t dst_is_device) {
    if (!bt) return BTDF_EINVAL;
    if (c < 0 || c >= bt->n || kind < 0 || kind > 3 || !dst) return bfail(bt, BTDF_EINVAL, "bad arguments");
    if (!bt->has_fields[c]) return bfail(bt, BTDF_ESTATE, "no fields");
    const size_t nn = (size_t)bt->cfg[c].nx * bt->cfg[c].ny * (kind == 3 ? 9 : 1);
    float* d = dst;
    if (!dst_is_device) BCK(cudaMalloc((void**)&d, sizeof(float) * nn));
    cudaError_t e = launch_read_field(bt->storage, !bt->poststream,
                                      (const char*)bt->g[bt->cur] + bt->off[c] * bt->elem, bt->descs[c],
                                      kind, d, bt->stream);
    if (e == cudaSuccess && !dst_is_device)
        e = cudaMemcpyAsync(dst, d, sizeof(float) * nn, cudaMemcpyDeviceToHost, bt->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(bt->stream);
    if (!dst_is_device) cudaFree(d);
    if (e != cudaSuccess) return bfail(bt, BTDF_ECUDA, std::string("read: ") + cudaGetErrorString(e));
    return bstatus(bt);
}

const char* btdf_batch_last_error(const btdf_batch* bt) { return bt ? bt->err.c_str() : "null batch"; }

}  // extern "C"
