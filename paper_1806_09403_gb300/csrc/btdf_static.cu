// btdf_static.cu - the IB force stage for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: code running inside another
// framework's memory budget (a caching allocator that owns every byte of the
// device), or real-time loops that must not enter the driver's allocator.
// They bring their own population buffer and output arrays; the per-marker
// tables and the reduction scratch this stage needs live in one fixed,
// file-scope device array instead of being allocated.  The call copies its
// host inputs from pageable memory and synchronizes its stream before it
// returns.  The arithmetic is the library's own IB kernel.
#include "btdf.h"
#include "btdf_internal.cuh"

#include <cuda.h>

#include <cmath>
#include <cstdint>
#include <mutex>

using namespace btdf;

namespace {

constexpr int kStaticMaxMarkers = BTDF_STATIC_MAX_MARKERS;
constexpr int kMaxDevices = 64;

// Scratch layout (bytes): the caller's marker positions and velocities as
// copied in (FP64), the marker tables built from them, D_I u*, D_I rho, the
// FP64 force sum and the status word.
constexpr size_t kOffIn = 0;
constexpr size_t kOffMk = kOffIn + 4 * sizeof(double) * kStaticMaxMarkers;
constexpr size_t kOffAux = kOffMk + sizeof(Marker) * kStaticMaxMarkers;
constexpr size_t kOffUs = kOffAux + sizeof(MarkerAux) * kStaticMaxMarkers;
constexpr size_t kOffRho = kOffUs + sizeof(float2) * kStaticMaxMarkers;
constexpr size_t kOffSum = (kOffRho + sizeof(float) * kStaticMaxMarkers + 255) / 256 * 256;
constexpr size_t kOffStatus = kOffSum + sizeof(double2);
constexpr size_t kScratchBytes = (kOffStatus + sizeof(int) + 255) / 256 * 256;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

// Device address of the scratch array, looked up once per device and CUDA
// context with that device current (host code must not use the symbol itself
// as an address).  The cache is keyed on the context's unique id, so a
// context created after cudaDeviceReset (which reloads the module) gets a
// fresh lookup instead of a dangling address.
std::mutex g_mu;
struct ScratchSlot {
    unsigned long long ctx_id;
    void* addr;
};
ScratchSlot g_scratch[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Unique id of the current context (0 if none is current yet).
bool current_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) !=
                cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) !=
                cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
            cudaGetLastError();
            return false;
        }
        get_current = (CtxGetCurrentFn)f1;
        get_id = (CtxGetIdFn)f2;
    }
    CUcontext c = nullptr;
    if (get_current(&c) != CUDA_SUCCESS) return false;
    *id = 0;
    return c == nullptr || get_id(c, id) == CUDA_SUCCESS;
}

int scratch_address(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BTDF_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    unsigned long long id = 0;
    if (!current_context_id(&id)) return BTDF_ECUDA;
    if (id == 0 || g_scratch[dev].addr == nullptr || g_scratch[dev].ctx_id != id) {
        // cudaGetSymbolAddress makes the device's primary context current
        // if none is; the id is read again afterwards
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || ptr == nullptr)
            return BTDF_ECUDA;
        if (!current_context_id(&id) || id == 0) return BTDF_ECUDA;
        g_scratch[dev].ctx_id = id;
        g_scratch[dev].addr = ptr;
    }
    *out = (unsigned char*)g_scratch[dev].addr;
    return BTDF_OK;
}

// Regularized delta functions of Sec. 4.3 (Eqs. 37-39 and the cosine
// kernel), evaluated in FP64 with the same expressions as the context path.
__device__ double delta_eval(int kind, double r) {
    const double a = fabs(r);
    switch (kind) {
    case 2: return a <= 1.0 ? 1.0 - a : 0.0;
    case 3:
        if (a > 1.5) return 0.0;
        if (a > 0.5) return (5.0 - 3.0 * a - sqrt(1.0 - 3.0 * (1.0 - a) * (1.0 - a))) / 6.0;
        return (1.0 + sqrt(1.0 - 3.0 * a * a)) / 3.0;
    case 4:
        if (a >= 2.0) return 0.0;
        if (a >= 1.0) return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
        return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
    case 5: return a < 2.0 ? 0.25 * (1.0 + cos(M_PI * a * 0.5)) : 0.0;
    default: return 0.0;
    }
}

// Marker tables (Eq. 14 weights in FP64, stored as FP32), one thread per
// marker, built in the scratch array from the positions copied there.
__global__ void static_tables(const double* in, int n, int kind, int width, int nx, int ny, int px,
                              int py, double u_ref, Marker* mk, MarkerAux* aux) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const double X = in[l], Y = in[kStaticMaxMarkers + l];
    const double ubx = in[2 * kStaticMaxMarkers + l], uby = in[3 * kStaticMaxMarkers + l];
    const int i0 = (int)floor(X - 0.5 * width) + 1;
    const int j0 = (int)floor(Y - 0.5 * width) + 1;
    double wx[4] = {0, 0, 0, 0}, wy[4] = {0, 0, 0, 0};
    bool okx[4] = {false, false, false, false}, oky[4] = {false, false, false, false};
    Marker M;
    for (int i = 0; i < 4; i++) {
        M.xs[i] = 0;
        M.ys[i] = 0;
    }
    for (int k = 0; k < 16; k++) M.w[k] = 0.0f;
    for (int i = 0; i < width; i++) {
        int x = i0 + i, y = j0 + i;
        wx[i] = delta_eval(kind, (double)x - X);
        wy[i] = delta_eval(kind, (double)y - Y);
        if (px) x = ((x % nx) + nx) % nx;
        if (py) y = ((y % ny) + ny) % ny;
        okx[i] = x >= 0 && x < nx;
        oky[i] = y >= 0 && y < ny;
        M.xs[i] = x < 0 ? 0 : (x > nx - 1 ? nx - 1 : x);
        M.ys[i] = y < 0 ? 0 : (y > ny - 1 ? ny - 1 : y);
    }
    double wsum = 0.0;
    for (int j = 0; j < width; j++)
        for (int i = 0; i < width; i++) {
            if (!okx[i] || !oky[j]) continue;
            const double w = wx[i] * wy[j];
            M.w[j * width + i] = (float)w;
            wsum += w;
        }
    mk[l] = M;
    MarkerAux A;
    A.wsum = (float)wsum;
    A.ubx_rel = (float)(ubx - u_ref * wsum);
    A.uby_rel = (float)uby;
    A.body = 0;
    aux[l] = A;
}

// FP64 sum of the Lagrangian forces (Eq. 27 before the ds*drs factor).
__global__ void static_force_sum(const float2* F, int n, double2* out) {
    __shared__ double sx[256], sy[256];
    double ax = 0.0, ay = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        ax += (double)F[k].x;
        ay += (double)F[k].y;
    }
    sx[threadIdx.x] = ax;
    sy[threadIdx.x] = ay;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            sx[threadIdx.x] += sx[threadIdx.x + s];
            sy[threadIdx.x] += sy[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = make_double2(sx[0], sy[0]);
}

}  // namespace

extern "C" int btdf_ib_forces_static(const btdf_config* cfg, const void* pops, int32_t pull,
                                     double u_ref, int32_t n, const double* X, const double* Y,
                                     const double* Ubx, const double* Uby, double ds, double drs,
                                     float* Fb, double* Fp, void* stream) {
    if (!cfg || !pops || !X || !Y || !Fb || !Fp) return BTDF_EINVAL;
    const btdf_config& c = *cfg;
    const int width = c.delta == 2 ? 2 : c.delta == 3 ? 3 : (c.delta == 4 || c.delta == 5) ? 4 : 0;
    if (n < 1 || n > kStaticMaxMarkers) return BTDF_EINVAL;
    if (width == 0 || c.nx < 4 || c.ny < 4 || c.storage < 0 || c.storage > 2 || c.bc_x < 0 ||
        c.bc_x > 1 || c.bc_y < 0 || c.bc_y > 2 ||
        (c.layout != BTDF_LAYOUT_PLANES && c.layout != BTDF_LAYOUT_ROWS) || !(ds > 0.0) ||
        !std::isfinite(c.u_in) || std::fabs(c.u_in) >= 0.5 || !std::isfinite(u_ref) ||
        std::fabs(u_ref) >= 0.5 || !std::isfinite(drs))
        return BTDF_EINVAL;
    // F_b is written and read as 8-byte pairs; populations are read as
    // elements of the storage type
    const uintptr_t elem = c.storage == 0 ? 4 : 2;
    if ((uintptr_t)Fb % 8 != 0 || (uintptr_t)pops % elem != 0) return BTDF_EINVAL;
    const long long nxp = ((long long)c.nx + 31) / 32 * 32;
    if (9ll * nxp * c.ny >= (1ll << 32)) return BTDF_EINVAL;
    const double half = 0.5 * width;
    for (int l = 0; l < n; l++) {
        if (!std::isfinite(X[l]) || !std::isfinite(Y[l]) || (Ubx && !std::isfinite(Ubx[l])) ||
            (Uby && !std::isfinite(Uby[l])))
            return BTDF_EINVAL;
        const bool inx = c.bc_x == BTDF_BCX_PERIODIC ? std::fabs(X[l]) <= 1e9
                                                     : (X[l] > -half && X[l] < c.nx - 1 + half);
        const bool iny = c.bc_y == BTDF_BCY_PERIODIC ? std::fabs(Y[l]) <= 1e9
                                                     : (Y[l] > -half && Y[l] < c.ny - 1 + half);
        if (!inx || !iny) return BTDF_EINVAL;
    }

    unsigned char* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != BTDF_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;

    const bool px = c.bc_x == BTDF_BCX_PERIODIC, py = c.bc_y == BTDF_BCY_PERIODIC;
    const double thick = drs > 0.0 ? drs : (c.delta == 2 ? 1.4 : c.delta == 3 ? 1.9 : 2.6);

    LatticeParams p{};
    p.wait_polls = -1;   // default bound of the bounded waits
    p.nx = c.nx;
    p.ny = c.ny;
    p.nxp = (int)nxp;
    p.nseg = (int)((nxp + kSeg - 1) / kSeg);
    p.plane = nxp * c.ny;
    p.rs = c.layout == BTDF_LAYOUT_ROWS ? 9u * (unsigned)nxp : (unsigned)nxp;
    for (int a = 0; a < 9; a++)
        p.poff[a] = c.layout == BTDF_LAYOUT_ROWS ? (unsigned)(a * nxp) : (unsigned)(a * p.plane);
    p.bcx = c.bc_x;
    p.bcy = c.bc_y;
    p.u_in = (float)c.u_in;       // inlet target of the pull
    p.urx = (float)u_ref;         // reference velocity of the stored deviations
    p.ury = 0.0f;

    IbParams q{};
    q.nmark = n;
    q.mk = (const Marker*)(scratch + kOffMk);
    q.aux = (const MarkerAux*)(scratch + kOffAux);
    q.F_prev = nullptr;
    q.F_out = (float2*)Fb;
    q.Us = (float2*)(scratch + kOffUs);
    q.rhol = (float*)(scratch + kOffRho);
    q.first_pass = 1;
    q.status = (int*)(scratch + kOffStatus);

    double2 sum = make_double2(0.0, 0.0);
    int status = 0;
    // The caller's positions and velocities go into the scratch array; the
    // tables are built there on the device.  Absent velocities are zero.
    double* in = (double*)(scratch + kOffIn);
    const size_t nb = sizeof(double) * (size_t)n;
    cudaError_t e = cudaMemcpyAsync(in, X, nb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(in + kStaticMaxMarkers, Y, nb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = Ubx ? cudaMemcpyAsync(in + 2 * kStaticMaxMarkers, Ubx, nb, cudaMemcpyHostToDevice, st)
                : cudaMemsetAsync(in + 2 * kStaticMaxMarkers, 0, nb, st);
    if (e == cudaSuccess)
        e = Uby ? cudaMemcpyAsync(in + 3 * kStaticMaxMarkers, Uby, nb, cudaMemcpyHostToDevice, st)
                : cudaMemsetAsync(in + 3 * kStaticMaxMarkers, 0, nb, st);
    if (e == cudaSuccess) {
        static_tables<<<(n + 127) / 128, 128, 0, st>>>(in, n, c.delta, width, c.nx, c.ny, px ? 1 : 0,
                                                       py ? 1 : 0, u_ref, (Marker*)(scratch + kOffMk),
                                                       (MarkerAux*)(scratch + kOffAux));
        e = cudaGetLastError();
    }
    // the status word keeps the previous call's value: clear it
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch + kOffStatus, 0, sizeof(int), st);
    if (e == cudaSuccess) e = launch_ib_force(c.storage, pull != 0, width, pops, p, q, false, st);
    if (e == cudaSuccess) {
        static_force_sum<<<1, 256, 0, st>>>((const float2*)Fb, n, (double2*)(scratch + kOffSum));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&sum, scratch + kOffSum, sizeof(double2), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&status, scratch + kOffStatus, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return BTDF_ECUDA;
    const double sc = ds * thick;   // Eq. 27, force on the body
    Fp[0] = -sum.x * sc;
    Fp[1] = -sum.y * sc;
    return (status & kStatusUnstable) ? BTDF_EUNSTABLE : BTDF_OK;
}
