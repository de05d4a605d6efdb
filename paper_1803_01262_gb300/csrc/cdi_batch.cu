// Batched CDI step: many independent periodic boxes of uneven sizes, each
// with its own face velocities, spacing, eps, gamma and dt, advanced by ONE
// launch per step.  The launch is a persistent grid of resident blocks that
// takes work units round-robin from one list covering every box: a unit is a
// 32 x 8 tile of one box and a chunk of its planes, processed by the same
// per-unit body as the single-box kernel (cdi_fwd_scalar.cuh).  Units of a box
// are contiguous in the list, so blocks resident together share halo planes
// through L2.  Each unit's outputs are reduced to one partial slot; the last
// block to finish folds each box's slots, in order, into that box's
// statistics record.  Multi-step runs are captured once into a CUDA graph and
// replayed.
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <string.h>

#include <map>
#include <utility>
#include <vector>

#include "cdi.h"
#include "cdi_fwd_scalar.cuh"
#include "cdi_internal.cuh"
#include "cdi_reduce.cuh"

namespace cdi {

template <typename T>
struct BoxDev {
    FwdArgs<T> a;     // phi = phi_a, out = phi_b; coefficients for vel_scale = 1
    double dV;        // cell measure dx^D_f
    int tiles_x, ntiles, zc, unit0, nunits;
};

constexpr int BBX = 32, BBY = 8;

template <typename T>
__global__ void __launch_bounds__(BBX * BBY)
batch_kernel(const BoxDev<T> *__restrict__ boxes, const int nbox, const int *__restrict__ unit_box,
             const int total_units, const int parity, const T vs, Partial *partials,
             unsigned int *counter, StatsRec *recs)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x + BBX * threadIdx.y;
    for (int u = blockIdx.x; u < total_units; u += gridDim.x) {
        const int bi = unit_box[u];
        FwdArgs<T> a = boxes[bi].a;
        if (parity) {
            T *t = a.out;
            a.out = const_cast<T *>(a.phi);
            a.phi = t;
        }
        a.c.c_adv *= vs;
        const int lu = u - boxes[bi].unit0;
        const Unit un = unit_of(lu, boxes[bi].ntiles, boxes[bi].tiles_x, BBX, BBY, boxes[bi].zc, a.nz);
        Acc<T> acc;
        acc.init();
        scalar_unit<T, BBX, BBY>(a, un, acc, smem_raw);
        const Partial p = block_reduce(acc.partial());
        if (tid == 0) partials[u] = p;
    }
    // The last block to arrive folds each box's unit partials (in unit order).
    __shared__ int is_last;
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(counter, 1u);
        is_last = prev == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    for (int bi = 0; bi < nbox; ++bi) {
        const int u0 = boxes[bi].unit0, nu = boxes[bi].nunits;
        Partial acc = pidentity();
        for (int i = tid; i < nu; i += BBX * BBY) acc = pcombine(acc, load_partial_cg(partials + u0 + i));
        acc = block_reduce(acc);
        if (tid == 0) {
            StatsRec *r = recs + bi;
            r->mass = boxes[bi].dV * acc.sum;
            r->sum = acc.sum;
            r->mn = acc.mn;
            r->mx = acc.mx;
            r->ns = acc.ns;
            r->nt = acc.nt;
            r->mn_run = fmin(r->mn_run, acc.mn);
            r->mx_run = fmax(r->mx_run, acc.mx);
            r->ns_run += acc.ns;
            r->nt_run += acc.nt;
            r->steps_run += 1;
        }
    }
    if (tid == 0) {
        __threadfence();
        *counter = 0u;
    }
}

}  // namespace cdi

using cdi::BoxDev;
using cdi::StatsRec;

struct cdi_batch {
    int nbox, dtype, total_units, nblocks, parity;
    void *boxes_dev;           // BoxDev<T>[nbox]
    int *unit_box;             // [total_units]
    cdi::Partial *partials;    // [total_units]
    unsigned int *counter;
    StatsRec *recs;            // [nbox]
    long long cells;
    cudaStream_t cap;          // capture stream for graphs
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;  // (nsteps, parity) -> exec
};

static size_t batch_smem(int dtype)
{
    return dtype == CDI_F64 ? cdi::FwdSmem<double, cdi::BBX, cdi::BBY>::bytes
                            : cdi::FwdSmem<float, cdi::BBX, cdi::BBY>::bytes;
}

static int batch_free(cdi_batch *b)
{
    if (!b) return CDI_OK;
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaFree(b->boxes_dev);
    cudaFree(b->unit_box);
    cudaFree(b->partials);
    cudaFree(b->counter);
    cudaFree(b->recs);
    delete b;
    return CDI_OK;
}

template <typename T>
static int build_table(cdi_batch *b, const cdi_box_desc *d, int nbox, std::vector<BoxDev<T>> &tab,
                       std::vector<int> &ub)
{
    int unit = 0;
    for (int i = 0; i < nbox; ++i) {
        const cdi_box_desc &x = d[i];
        if (x.nx < 1 || x.ny < 1 || x.nz < 1 || (long long)x.nx * x.ny >= (1LL << 31))
            return cdi::set_error(CDI_ERR_DIM, "box %d: bad extents", i);
        if (!(x.dx > 0) || !(x.dt >= 0) || !(x.eps > 0) || !(x.gamma >= 0))
            return cdi::set_error(CDI_ERR_ARG, "box %d: bad dx, dt, eps or gamma", i);
        if (!x.phi_a || !x.phi_b || !x.u || (!x.v && !(x.ny == 1 && x.nz == 1)) || (!x.w && x.nz != 1))
            return cdi::set_error(CDI_ERR_ARG, "box %d: NULL array", i);
        BoxDev<T> e;
        memset(&e, 0, sizeof(e));
        e.a.phi = (const T *)x.phi_a;
        e.a.out = (T *)x.phi_b;
        e.a.u = (const T *)x.u;
        e.a.v = (const T *)(x.v ? x.v : x.u);
        e.a.w = (const T *)(x.w ? x.w : x.u);
        e.a.nx = x.nx; e.a.ny = x.ny; e.a.nz = x.nz;
        e.a.c.c_adv = (T)0.5;
        e.a.c.c_dif = (T)(x.gamma * x.eps / x.dx);
        e.a.c.c_shp = (T)(0.5 * x.gamma);
        e.a.c.c_upd = (T)(x.dt / x.dx);
        e.a.c.tol = sizeof(T) == 8 ? (T)DBL_EPSILON : (T)FLT_EPSILON;
        const int Df = (x.nx > 1) + (x.ny > 1) + (x.nz > 1);
        e.dV = pow(x.dx, (double)Df);
        e.tiles_x = (x.nx + cdi::BBX - 1) / cdi::BBX;
        e.ntiles = e.tiles_x * ((x.ny + cdi::BBY - 1) / cdi::BBY);
        int nch = (x.nz + 16) / 32;  // about 32 planes per unit
        if (nch < 1) nch = 1;
        e.zc = (x.nz + nch - 1) / nch;
        e.unit0 = unit;
        e.nunits = e.ntiles * ((x.nz + e.zc - 1) / e.zc);
        for (int k = 0; k < e.nunits; ++k) ub.push_back(i);
        unit += e.nunits;
        b->cells += (long long)x.nx * x.ny * x.nz;
        tab.push_back(e);
    }
    b->total_units = unit;
    return CDI_OK;
}

template <typename T>
static int batch_launch(cdi_batch *b, int parity, double vs, cudaStream_t s)
{
    cdi::batch_kernel<T><<<b->nblocks, dim3(cdi::BBX, cdi::BBY), batch_smem(b->dtype), s>>>(
        (const BoxDev<T> *)b->boxes_dev, b->nbox, b->unit_box, b->total_units, parity, (T)vs,
        b->partials, b->counter, b->recs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cdi::set_error(CDI_ERR_CUDA, "batch launch: %s", cudaGetErrorString(e));
    return CDI_OK;
}

static void reset_recs(std::vector<StatsRec> &h)
{
    for (auto &r : h) {
        memset(&r, 0, sizeof(r));
        r.mn = INFINITY; r.mx = -INFINITY; r.mn_run = INFINITY; r.mx_run = -INFINITY;
    }
}

int cdi_batch_create(cdi_batch **out, const cdi_box_desc *boxes, int nbox, int dtype)
{
    if (!out || !boxes || nbox < 1) return cdi::set_error(CDI_ERR_ARG, "bad batch arguments");
    *out = nullptr;
    if (dtype != CDI_F32 && dtype != CDI_F64) return cdi::set_error(CDI_ERR_ARG, "bad dtype");
    cdi_batch *b = new cdi_batch();
    b->nbox = nbox;
    b->dtype = dtype;
    std::vector<int> ub;
    std::vector<unsigned char> tab_bytes;
    int rc;
    size_t tab_size;
    if (dtype == CDI_F64) {
        std::vector<BoxDev<double>> tab;
        rc = build_table<double>(b, boxes, nbox, tab, ub);
        tab_size = tab.size() * sizeof(BoxDev<double>);
        tab_bytes.assign((unsigned char *)tab.data(), (unsigned char *)tab.data() + tab_size);
    } else {
        std::vector<BoxDev<float>> tab;
        rc = build_table<float>(b, boxes, nbox, tab, ub);
        tab_size = tab.size() * sizeof(BoxDev<float>);
        tab_bytes.assign((unsigned char *)tab.data(), (unsigned char *)tab.data() + tab_size);
    }
    if (rc) {
        batch_free(b);
        return rc;
    }
    cudaError_t e;
    int dev = 0, sms = 0, resident = 0;
    const size_t smem = batch_smem(dtype);
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = dtype == CDI_F64
                 ? cudaFuncSetAttribute(cdi::batch_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                 : cudaFuncSetAttribute(cdi::batch_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess ||
        (e = dtype == CDI_F64
                 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, cdi::batch_kernel<double>, cdi::BBX * cdi::BBY, smem)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, cdi::batch_kernel<float>, cdi::BBX * cdi::BBY, smem)) != cudaSuccess) {
        batch_free(b);
        return cdi::set_error(CDI_ERR_CUDA, "batch setup: %s", cudaGetErrorString(e));
    }
    long long nb = (long long)resident * sms;
    if (nb > b->total_units) nb = b->total_units;
    if (nb < 1) nb = 1;
    b->nblocks = (int)nb;
    std::vector<StatsRec> hrec(nbox);
    reset_recs(hrec);
    if ((e = cudaMalloc(&b->boxes_dev, tab_size)) != cudaSuccess ||
        (e = cudaMalloc(&b->unit_box, sizeof(int) * ub.size())) != cudaSuccess ||
        (e = cudaMalloc(&b->partials, sizeof(cdi::Partial) * ub.size())) != cudaSuccess ||
        (e = cudaMalloc(&b->counter, sizeof(unsigned int))) != cudaSuccess ||
        (e = cudaMalloc(&b->recs, sizeof(StatsRec) * nbox)) != cudaSuccess ||
        (e = cudaMemcpy(b->boxes_dev, tab_bytes.data(), tab_size, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->unit_box, ub.data(), sizeof(int) * ub.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->recs, hrec.data(), sizeof(StatsRec) * nbox, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(b->counter, 0, sizeof(unsigned int))) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess) {
        batch_free(b);
        return cdi::set_error(CDI_ERR_CUDA, "batch allocation: %s", cudaGetErrorString(e));
    }
    *out = b;
    return CDI_OK;
}

int cdi_batch_destroy(cdi_batch *b) { return batch_free(b); }

int cdi_batch_info(const cdi_batch *b, int *parity, int *total_units, int *nblocks, long long *cells)
{
    if (!b) return cdi::set_error(CDI_ERR_ARG, "batch is NULL");
    if (parity) *parity = b->parity;
    if (total_units) *total_units = b->total_units;
    if (nblocks) *nblocks = b->nblocks;
    if (cells) *cells = b->cells;
    return CDI_OK;
}

int cdi_batch_step(cdi_batch *b, double vel_scale, void *stream)
{
    if (!b) return cdi::set_error(CDI_ERR_ARG, "batch is NULL");
    if (!isfinite(vel_scale)) return cdi::set_error(CDI_ERR_ARG, "vel_scale must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = b->dtype == CDI_F64 ? batch_launch<double>(b, b->parity, vel_scale, s)
                                 : batch_launch<float>(b, b->parity, vel_scale, s);
    if (rc == CDI_OK) b->parity ^= 1;
    return rc;
}

int cdi_batch_run(cdi_batch *b, int nsteps, void *stream)
{
    if (!b) return cdi::set_error(CDI_ERR_ARG, "batch is NULL");
    if (nsteps < 1) return cdi::set_error(CDI_ERR_ARG, "nsteps must be >= 1");
    const std::pair<int, int> key(nsteps, b->parity);
    auto it = b->graphs.find(key);
    cudaError_t e;
    if (it == b->graphs.end()) {
        // Capture nsteps launches (parity alternating) once on the private stream.
        cudaGraph_t graph;
        if ((e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return cdi::set_error(CDI_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
        int rc = CDI_OK;
        for (int i = 0; i < nsteps && rc == CDI_OK; ++i) {
            const int p = b->parity ^ (i & 1);
            rc = b->dtype == CDI_F64 ? batch_launch<double>(b, p, 1.0, b->cap)
                                     : batch_launch<float>(b, p, 1.0, b->cap);
        }
        e = cudaStreamEndCapture(b->cap, &graph);
        if (rc) return rc;
        if (e != cudaSuccess) return cdi::set_error(CDI_ERR_CUDA, "end capture: %s", cudaGetErrorString(e));
        cudaGraphExec_t exec;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cdi::set_error(CDI_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
        it = b->graphs.emplace(key, exec).first;
    }
    if ((e = cudaGraphLaunch(it->second, (cudaStream_t)stream)) != cudaSuccess)
        return cdi::set_error(CDI_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
    b->parity ^= (nsteps & 1);
    return CDI_OK;
}

int cdi_batch_stats(cdi_batch *b, cdi_stats *out, void *stream)
{
    if (!b || !out) return cdi::set_error(CDI_ERR_ARG, "NULL argument");
    static_assert(sizeof(StatsRec) == sizeof(cdi_stats), "record layout");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(out, b->recs, sizeof(StatsRec) * b->nbox, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cdi::set_error(CDI_ERR_CUDA, "batch statistics: %s", cudaGetErrorString(e));
    for (int i = 0; i < b->nbox; ++i)
        if (!isfinite(out[i].sum)) return cdi::set_error(CDI_ERR_NAN, "box %d: non-finite phi", i);
    return CDI_OK;
}

int cdi_batch_reset_run_stats(cdi_batch *b, void *stream)
{
    if (!b) return cdi::set_error(CDI_ERR_ARG, "batch is NULL");
    std::vector<StatsRec> h(b->nbox);
    reset_recs(h);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(b->recs, h.data(), sizeof(StatsRec) * b->nbox, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cdi::set_error(CDI_ERR_CUDA, "reset batch statistics: %s", cudaGetErrorString(e));
    return CDI_OK;
}
