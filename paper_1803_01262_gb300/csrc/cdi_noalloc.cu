// cdi_step_noalloc: the fused forward step for callers that cannot allocate
// device memory (no cudaMalloc / cudaFree, no allocating library call).
//
// Who needs this: code that runs where allocation is forbidden or unsafe --
// inside a host callback or a custom allocator's hook, in a process whose
// memory pool is fixed up front by its framework, or in a latency-critical
// loop that must never hit the driver's allocator.  The regular API keeps
// its reduction scratch in a grid object created by cdi_create_grid, which
// allocates; this entry point takes no grid and instead uses the fixed
// reduction scratch below, a file-scope device array that every GPU which
// loads the library holds until the process exits.
//
// The scratch is shared by every call: calls that overlap on the GPU (for
// example on two streams at once) race on it and must be avoided.  Each call
// clears the block counter before its launch, so a call never depends on
// what an earlier call left behind.  The host looks the array's device
// address up once per device context (cudaGetSymbolAddress, which allocates
// nothing) and looks it up again when the context has changed, as after a
// cudaDeviceReset.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "cdi.h"
#include "cdi_internal.cuh"

namespace {

// Reduction scratch: one partial per block of a launch, and the counter of
// finished blocks.  CDI_NOALLOC_MAX_BLOCKS bounds the number of blocks.
constexpr int kMaxBlocks = CDI_NOALLOC_MAX_BLOCKS;

struct NoAllocScratch {
    cdi::Partial partials[kMaxBlocks];
    unsigned int counter;
};

static __device__ __align__(256) NoAllocScratch g_scratch;

// Device address of g_scratch and the SM count, per device, resolved on the
// first call made with that device current.  In host code g_scratch names a
// host-side stand-in, so the kernel is given this address instead.  Each entry
// remembers the unique id of the context it was resolved in: after a
// cudaDeviceReset the device gets a new context, whose module (and array) may
// sit elsewhere, and the next call resolves the address again.  The mutex
// keeps concurrent first calls from different host threads from seeing a
// half-written entry.
constexpr int kMaxDevices = 64;
struct DevEntry {
    unsigned long long ctx_id;  // 0: not resolved
    NoAllocScratch *addr;
    int sms;
};
static DevEntry g_dev[kMaxDevices];
static std::mutex g_dev_mutex;

static PFN_cuCtxGetCurrent_v4000 g_ctx_current = nullptr;
static PFN_cuCtxGetId_v12000 g_ctx_id = nullptr;

// Unique id of the calling thread's current context (0 if none or unavailable).
static unsigned long long current_ctx_id()
{
    if (!g_ctx_current || !g_ctx_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return 0;
        g_ctx_current = (PFN_cuCtxGetCurrent_v4000)f1;
        g_ctx_id = (PFN_cuCtxGetId_v12000)f2;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx || g_ctx_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

}  // namespace

// Errors go to the same thread-local message as every other entry point.
static int na_fail(int code, const char *msg, cudaError_t e = cudaSuccess)
{
    if (e != cudaSuccess) return cdi::set_error(code, "%s: %s", msg, cudaGetErrorString(e));
    return cdi::set_error(code, "%s", msg);
}

template <typename T>
static int noalloc_t(int nx, int ny, int nz, double dx, const void *in, void *out, const void *u,
                     const void *v, const void *w, double dt, double eps, double gamma, double vs,
                     void *stats_dev, NoAllocScratch *scr, int sms, cudaStream_t s)
{
    const int es = (int)sizeof(T);
    const int vx = 16 / es;
    int tile;
    if (nx % vx == 0 && nx >= 48) tile = ny >= 12 ? 4 : 5;
    else tile = (nx >= 32 && ny >= 16) ? 1 : 3;
    int resident = 0;
    cudaError_t e = cdi::fwd_occupancy<T>(tile, false, &resident);
    if (e != cudaSuccess) return na_fail(CDI_ERR_CUDA, "occupancy query", e);
    const long long tiles = cdi::fwd_tiles_xy(tile, es, nx, ny);
    long long nb = (long long)resident * sms;
    // one z chunk per tile column when that fills the GPU, else split the columns
    int nchunks = 1;
    while (tiles * nchunks < nb && nchunks < nz) ++nchunks;
    const int zc = (nz + nchunks - 1) / nchunks;
    const long long units = tiles * ((nz + zc - 1) / zc);
    if (nb > units) nb = units;
    if (nb > kMaxBlocks)
        return na_fail(CDI_ERR_DIM, "launch needs more blocks than the fixed scratch holds");

    cdi::FwdArgs<T> a;
    a.phi = (const T *)in;
    a.out = (T *)out;
    a.u = (const T *)u;
    a.v = (const T *)(v ? v : u);
    a.w = (const T *)(w ? w : u);
    a.nx = nx; a.ny = ny; a.nz = nz;
    a.c.c_adv = (T)(0.5 * vs);
    a.c.c_dif = (T)(gamma * eps / dx);
    a.c.c_shp = (T)(0.5 * gamma);
    a.c.c_upd = (T)(dt / dx);
    a.c.tol = es == 8 ? (T)DBL_EPSILON : (T)FLT_EPSILON;
    a.red.partials = scr->partials;
    a.red.counter = &scr->counter;
    a.red.rec = (cdi::StatsRec *)stats_dev;
    a.red.capacity = kMaxBlocks;
    a.red.dV = pow(dx, (double)((nx > 1) + (ny > 1) + (nz > 1)));
    a.red.update_run = 0;
    a.red.status = nullptr;  // bounded waits still end; a time-out is not reported here
    // The counter must start at zero; clear it on the stream (no allocation).
    if ((e = cudaMemsetAsync(&scr->counter, 0, sizeof(unsigned int), s)) != cudaSuccess)
        return na_fail(CDI_ERR_CUDA, "clearing the block counter", e);
    a.rk_base = nullptr;
    a.rk_q = nullptr;
    a.rk_qout = nullptr;
    a.rk_alpha = a.rk_delta = a.rk_mu = a.rk_beta = T(0);
    if ((e = cdi::launch_fwd<T>(a, tile, (int)nb, nchunks, false, s)) != cudaSuccess)
        return na_fail(CDI_ERR_CUDA, "forward step launch", e);
    return CDI_OK;
}

extern "C" int cdi_step_noalloc(int nx, int ny, int nz, double dx, int dtype, const void *phi_in,
                                void *phi_out, const void *u, const void *v, const void *w,
                                double dt, double eps, double gamma, double vel_scale,
                                void *stats_dev, void *stream)
{
    if (nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny >= (1LL << 31))
        return na_fail(CDI_ERR_DIM, "extents must be >= 1 with nx*ny < 2^31");
    if (!(dx > 0) || !(eps > 0) || !(gamma >= 0) || !(dt >= 0) || !isfinite(vel_scale))
        return na_fail(CDI_ERR_ARG, "bad dx, dt, eps, gamma or vel_scale");
    if (dtype != CDI_F32 && dtype != CDI_F64) return na_fail(CDI_ERR_ARG, "dtype must be CDI_F32 or CDI_F64");
    if (!phi_in || !phi_out || !u || !stats_dev) return na_fail(CDI_ERR_ARG, "NULL pointer");
    if (!v && !(ny == 1 && nz == 1)) return na_fail(CDI_ERR_ARG, "v may be NULL only when ny == nz == 1");
    if (!w && nz != 1) return na_fail(CDI_ERR_ARG, "w may be NULL only when nz == 1");
    const void *ptrs[] = {phi_in, phi_out, u, v, w};
    for (const void *p : ptrs)
        if (p && ((uintptr_t)p & 15u)) return na_fail(CDI_ERR_ARG, "arrays must be 16-byte aligned");
    if ((uintptr_t)stats_dev & 7u) return na_fail(CDI_ERR_ARG, "stats_dev must be 8-byte aligned");
    const size_t bytes = (size_t)nx * ny * nz * (dtype == CDI_F64 ? 8 : 4);
    const char *pa = (const char *)phi_in, *pb = (const char *)phi_out;
    if (pa < pb + bytes && pb < pa + bytes) return na_fail(CDI_ERR_ARG, "phi_in and phi_out overlap");

    const size_t nb_stats = sizeof(cdi_stats);
    const char *ps = (const char *)stats_dev;
    // phi_out, u, v, w, stats_dev: the kernel writes phi_out and the record while
    // it reads the others, so no written buffer may overlap a read one.
    const char *rd[] = {(const char *)phi_in, (const char *)u, (const char *)v, (const char *)w};
    for (const char *r : rd)
        if (r && r != pa && pb < r + bytes && r < pb + bytes)
            return na_fail(CDI_ERR_ARG, "phi_out overlaps a velocity array");
    for (const char *r : rd)
        if (r && ps < r + bytes && r < ps + nb_stats)
            return na_fail(CDI_ERR_ARG, "stats_dev overlaps phi_in or a velocity array");
    if (ps < pb + bytes && pb < ps + nb_stats) return na_fail(CDI_ERR_ARG, "stats_dev overlaps phi_out");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(CDI_ERR_CUDA, "cudaGetDevice", e);
    if (dev < 0 || dev >= kMaxDevices) return na_fail(CDI_ERR_STATE, "device ordinal out of range");
    DevEntry ent;
    {
        std::lock_guard<std::mutex> lock(g_dev_mutex);
        unsigned long long id = current_ctx_id();
        if (id == 0 || g_dev[dev].ctx_id != id) {
            // First call on this device (or in a new context of it): resolve the
            // scratch address (this also makes the device's primary context
            // current) and the SM count.  Neither allocates.
            void *ptr = nullptr;
            if ((e = cudaGetSymbolAddress(&ptr, g_scratch)) != cudaSuccess)
                return na_fail(CDI_ERR_CUDA, "cudaGetSymbolAddress", e);
            int sms = 0;
            if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
                return na_fail(CDI_ERR_CUDA, "cudaDeviceGetAttribute", e);
            id = current_ctx_id();
            if (id == 0) return na_fail(CDI_ERR_CUDA, "no current CUDA context after cudaGetSymbolAddress");
            g_dev[dev].addr = (NoAllocScratch *)ptr;
            g_dev[dev].sms = sms;
            g_dev[dev].ctx_id = id;
        }
        ent = g_dev[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    return dtype == CDI_F64
        ? noalloc_t<double>(nx, ny, nz, dx, phi_in, phi_out, u, v, w, dt, eps, gamma, vel_scale,
                            stats_dev, ent.addr, ent.sms, s)
        : noalloc_t<float>(nx, ny, nz, dx, phi_in, phi_out, u, v, w, dt, eps, gamma, vel_scale,
                           stats_dev, ent.addr, ent.sms, s);
}
