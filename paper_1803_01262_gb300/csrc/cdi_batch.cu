// Batched CDI step: many independent periodic boxes of uneven sizes, each
// with its own face velocities, spacing, eps, gamma and dt, advanced by ONE
// launch per step.  The launch is a persistent grid of resident blocks that
// takes work units, in order, from one list covering every box (a counter hands
// the next unit to the next block that is done with one): a unit is a
// BX x BY tile of one box and a chunk of its planes, processed by the same
// per-unit body as the single-box kernel (cdi_fwd_scalar.cuh).  Units of a box
// are contiguous in the list (chunk-major), so blocks resident together share
// halo planes through L2; the boxes come in order of decreasing unit size, so
// the launch ends on the smallest units.  Each unit's outputs are reduced to one partial
// slot; the block that completes a box's last unit folds that box's slots, in
// unit order, into the box's statistics record (reproducible, and spread over
// the launch instead of serialised at its end).  The tile shape and the number
// of planes per unit are a launch configuration (cdi_batch_set_launch), which
// cdi_batch_autotune picks by timing.  A batch of 2D boxes small enough to
// hold a whole plane in shared memory can also take one unit per box (the
// whole-plane body below).  Multi-step runs are captured once into a CUDA
// graph and replayed.
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <utility>
#include <vector>

#include "cdi.h"
#include "cdi_band.cuh"
#include "cdi_vband.cuh"
#include "cdi_fwd_scalar.cuh"
#include "cdi_internal.cuh"
#include "cdi_nvtx.h"
#include "cdi_reduce.cuh"

namespace cdi {

template <typename T>
struct BoxDev {
    FwdArgs<T> a;     // phi = phi_a, out = phi_b; coefficients for vel_scale = 1
    double dV;        // cell measure dx^D_f
    int tiles_x, ntiles, zc, unit0, nunits;
    int bh;           // row-band bodies: rows per band
    // vector row-band body: the batch's padded copies (pitch P, cdi_vband.cuh):
    // the state by parity, and the face velocities
    T *pad[2];
    const T *pu, *pv, *pw;
    int pitch;
};

// Whole-plane unit body: the unit is a whole 2D box (nz == 1) whose phi and
// both sharpening components fit in shared memory (3 nx ny values).  Cells
// are visited by their linear index l = y nx + x and the periodic neighbours
// found by index arithmetic, so every lane holds a cell of the box (no tile
// overhang) and each sharpening value is evaluated once (no ring around a
// tile).  The arithmetic is flat_unit's, expression by expression, so the
// result is the same bit for bit (FACE: the face-product sharpening, the s
// arrays holding the normals).
template <typename T, int NT, bool FACE = false>
__device__ __forceinline__ void plane_unit(const FwdArgs<T> &a, Acc<T> &acc, unsigned char *smem_raw)
{
    const int nx = a.nx, ny = a.ny, P = nx * ny;
    T *const sp = reinterpret_cast<T *>(smem_raw);  // phi [P]
    T *const ssx = sp + P;                          // s_x [P]
    T *const ssy = ssx + P;                         // s_y [P]
    const int tid = threadIdx.x;
    const T c_adv = a.c.c_adv, c_dif = a.c.c_dif, c_shp = a.c.c_shp, c_upd = a.c.c_upd;

    // periodic neighbours of cell l (a neighbour is l itself along an axis of extent 1)
    auto nbr = [&](int l, int &xm, int &xp, int &ym, int &yp) {
        const int y = l / nx, x = l - y * nx;
        xm = x == 0 ? l + nx - 1 : l - 1;
        xp = x == nx - 1 ? l - nx + 1 : l + 1;
        ym = y == 0 ? l + P - nx : l - nx;
        yp = y == ny - 1 ? l - P + nx : l + nx;
    };

    __syncthreads();  // the previous unit's readers are done with the buffers
    for (int l = tid; l < P; l += NT) cp_async<sizeof(T)>(sp + l, a.phi + l);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    for (int l = tid; l < P; l += NT) {
        int xm, xp, ym, yp;
        nbr(l, xm, xp, ym, yp);
        const T p = sp[l];
        const T g0 = sp[xp] - sp[xm];
        const T g1 = sp[yp] - sp[ym];
        const T g2 = T(0);
        const T q = fma(g2, g2, fma(g1, g1, fma(g0, g0, NumLim<T>::tiny())));
        const T inv = rsqrt_t(q);
        const T wgt = FACE ? inv : p * (T(1) - p) * inv;
        ssx[l] = wgt * g0;
        ssy[l] = wgt * g1;
    }
    __syncthreads();
    for (int l = tid; l < P; l += NT) {
        int xm, xp, ym, yp;
        nbr(l, xm, xp, ym, yp);
        const T pc = sp[l];
        const T pxm = sp[xm], pxp = sp[xp];
        const T pym = sp[ym], pyp = sp[yp];
        const T sxm = ssx[xm], sxp = ssx[xp];
        const T sym = ssy[ym], syp = ssy[yp];
        const T uc = __ldg(a.u + l), um = __ldg(a.u + xm);
        const T vc = __ldg(a.v + l), vm = __ldg(a.v + ym);
        T adv = uc * (pc + pxp);
        adv = fma(-um, pxm + pc, adv);
        adv = fma(vc, pc + pyp, adv);
        adv = fma(-vm, pym + pc, adv);
        const T dif = fma(T(-4), pc, (pxm + pxp) + (pym + pyp));
        T shp;
        if constexpr (FACE) {
            const T nxc = ssx[l], nyc = ssy[l];
            const T fxp = T(0.5) * (pc + pxp), fxm = T(0.5) * (pxm + pc);
            const T fyp = T(0.5) * (pc + pyp), fym = T(0.5) * (pym + pc);
            shp = (fxp * (T(1) - fxp) * (nxc + sxp) - fxm * (T(1) - fxm) * (sxm + nxc)) +
                  (fyp * (T(1) - fyp) * (nyc + syp) - fym * (T(1) - fym) * (sym + nyc));
        } else {
            shp = (sxp - sxm) + (syp - sym);
        }
        const T div = fma(c_adv, adv, fma(-c_dif, dif, fma(c_shp, shp, T(0))));  // z faces: Fzp - Fzm = 0
        const T o = fma(-c_upd, div, pc);
        a.out[l] = o;
        acc.add(o, a.c.tol);
    }
}

// Work hand-out and ordering of one batch launch.  The steps of a run overlap:
// launch i + 1 starts on the SMs that launch i leaves, and each of its units
// waits only until its own box has completed step i (boxes are independent, so
// the large boxes of the next step fill the tail of the current one).
struct BatchSync {
    unsigned int *queue;  // [2]: units handed out beyond the first grid's worth, blocks finished
    unsigned int *epoch;  // [nbox]: steps of the current run each box has completed
    int step;             // index of this launch in a run; its units wait for epoch >= step
    int reset;            // the last block to finish zeroes queue (launches outside a run)
    unsigned long long wait_ns;  // limit of one unit's wait
};

// Wait until *epoch >= target (acquire: the box's previous step is then visible),
// for at most limit_ns; gives up at once if another wait has already given up
// (status bit 0), else records that bit.  Returns whether the box is ready.
__device__ __forceinline__ bool wait_epoch(const unsigned int *epoch, unsigned target, unsigned int *status,
                                           unsigned long long limit_ns)
{
    const unsigned long long t0 = global_ns();
    for (;;) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(epoch) : "memory");
        if ((int)(v - target) >= 0) return true;
        unsigned st;
        asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(st) : "l"(status) : "memory");
        if (st & 1u) return false;
        if (global_ns() - t0 > limit_ns) break;
        __nanosleep(256);
    }
    atomicOr(status, 1u);
    return false;
}

// BODY 0: the 3D unit body (scalar_unit).  BODY 1: every box has nz == 1
// (e.g. a phase-diagram sweep of 2D boxes): the single-plane unit body, which
// stages the plane once (flat_unit).  BODY 2: every box has nz == 1 and fits
// in shared memory: one unit per box, the whole-plane body (plane_unit).
// BODY 3: bands of whole rows (band_unit, cdi_band.cuh), slots of sizes bs.
// BODY 4: bands of whole rows of the padded copies (vband_unit, cdi_vband.cuh),
// slots of sizes vbs; final_write: the step also writes the caller's arrays.
// FACE: the face-product sharpening (bodies 0, 1 and 2).  sync: the launch's
// hand-out counters and its place in a run (BatchSync).
template <typename T, int BX, int BY, int BODY = 0, bool FACE = false>
__global__ void __launch_bounds__(BX * BY, BODY >= 3 ? 2 : 1)
batch_kernel(const BoxDev<T> *__restrict__ boxes, const int *__restrict__ unit_box,
             const int total_units, const int parity, const T vs, Partial *partials,
             unsigned int *box_done, StatsRec *recs, const BandSlots bs, const VbandSlots vbs,
             const int final_write, const BatchSync sync)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int fold, next_u, ready;
    const int tid = threadIdx.x + BX * threadIdx.y;
    unsigned int *const status = boxes[0].a.red.status;
    // The next launch of a run may start once every block of this one has
    // started; it takes the SMs as this launch's blocks finish.
    grid_dep_launch();
    // Units are handed out in list order from a counter (queue[0]; every block
    // starts with unit blockIdx.x): a block takes the next unit when it is done
    // with one, so blocks that run faster take more.  The fields do not depend
    // on which block steps a unit, and the statistics are folded per box in
    // unit order, so the result does not either.
    int u = blockIdx.x;
    while (u < total_units) {
        const int bi = unit_box[u];
        if (sync.step > 0) {  // the box's previous step: complete and visible
            if (tid == 0) {
                ready = wait_epoch(sync.epoch + bi, (unsigned)sync.step, status, sync.wait_ns);
                __threadfence();
            }
            __syncthreads();
            if (!ready) break;  // a wait gave up (reported); the remaining units are skipped
        }
        FwdArgs<T> a = boxes[bi].a;
        if (parity) {
            T *t = a.out;
            a.out = const_cast<T *>(a.phi);
            a.phi = t;
        }
        a.c.c_adv *= vs;
        Acc<T> acc;
        acc.init();
        if constexpr (BODY == 2) {
            plane_unit<T, BX * BY, FACE>(a, acc, smem_raw);
        } else if constexpr (BODY == 3) {
            const int lu = u - boxes[bi].unit0, nb = boxes[bi].ntiles, zc = boxes[bi].zc;
            const int chunk = lu / nb, band = lu - chunk * nb;
            const int y0 = band * boxes[bi].bh;
            const int hb = min(boxes[bi].bh, a.ny - y0);
            const int z0 = chunk * zc;
            band_unit<T>(a, y0, hb, z0, min(a.nz, z0 + zc), bs, acc, smem_raw);
        } else if constexpr (BODY == 4) {
            const BoxDev<T> &bx = boxes[bi];
            const int lu = u - bx.unit0, nb = bx.ntiles, zc = bx.zc;
            const int chunk = lu / nb, band = lu - chunk * nb;
            const int z0 = chunk * zc;
            vband_unit<T>(a, bx.pad[parity], bx.pad[parity ^ 1], bx.pu, bx.pv, bx.pw, bx.pitch, final_write != 0,
                          band * bx.bh, bx.bh, z0, min(a.nz, z0 + zc), vbs, acc, smem_raw);
        } else {
            const int lu = u - boxes[bi].unit0;
            const Unit un = unit_of(lu, boxes[bi].ntiles, boxes[bi].tiles_x, BX, BY, boxes[bi].zc, a.nz);
            if constexpr (BODY == 1)
                flat_unit<T, BX, BY, FACE>(a, un, acc, smem_raw);
            else
                scalar_unit<T, BX, BY, false, SCALAR_PF, FACE>(a, un, acc, smem_raw);
        }
        int claim = 0;  // the next unit, requested before this one's reduction
        if (tid == 0) claim = (int)atomicAdd(sync.queue, 1u) + (int)gridDim.x;
        const Partial p = block_partial(acc);
        if (tid == 0) {
            next_u = claim;
            partials[u] = p;
            __threadfence();
            const unsigned done = atomicAdd(box_done + bi, 1u) + 1u;
            fold = done == (unsigned)boxes[bi].nunits ? bi : -1;
        }
        __syncthreads();
        const int fb = fold;
        if (fb >= 0) {  // this block completed box fb: fold its slots in unit order
            __threadfence();
            const int u0 = boxes[fb].unit0, nu = boxes[fb].nunits;
            const Partial q = combine_partials<IsF32<Acc<T>>::value>(partials + u0, nu);
            if (tid == 0) {
                StatsRec *r = recs + fb;
                r->mass = boxes[fb].dV * q.sum;
                r->sum = q.sum;
                r->mn = q.mn;
                r->mx = q.mx;
                r->ns = q.ns;
                r->nt = q.nt;
                r->mn_run = fmin(r->mn_run, q.mn);
                r->mx_run = fmax(r->mx_run, q.mx);
                r->ns_run += q.ns;
                r->nt_run += q.nt;
                r->steps_run += 1;
                box_done[fb] = 0u;  // every unit of the box has counted in this launch
                __threadfence();
                atomicAdd(sync.epoch + fb, 1u);  // release: the box's next step may start
            }
        }
        __syncthreads();  // every thread has read `fold` before it is written again
        u = next_u;
    }
    // outside a run, the last block to run out of units resets the counters for
    // the next launch (a run's launches each have counters of their own, zeroed
    // before the run: an overlapping launch must not see a reset)
    if (tid == 0 && sync.reset) {
        __threadfence();
        if (atomicAdd(sync.queue + 1, 1u) == gridDim.x - 1) {
            atomicExch(sync.queue, 0u);
            atomicExch(sync.queue + 1, 0u);
        }
    }
}

// Fill a box's padded copy (cdi_vband.cuh) from a caller's array: position p of
// a padded row holds the row's cell (p - VX) mod nx.  blockIdx.y: the box.
// which: 0, 1 the state of that parity (from phi_a / phi_b), 2, 3, 4 u, v, w.
template <typename T>
__global__ void __launch_bounds__(256) vband_pack(const BoxDev<T> *__restrict__ boxes, int which)
{
    constexpr int VX = 16 / sizeof(T);
    const BoxDev<T> &bx = boxes[blockIdx.y];
    const FwdArgs<T> &a = bx.a;
    const T *src = which == 0 ? a.phi : which == 1 ? a.out : which == 2 ? a.u : which == 3 ? a.v : a.w;
    T *dst = which <= 1 ? bx.pad[which] : const_cast<T *>(which == 2 ? bx.pu : which == 3 ? bx.pv : bx.pw);
    const int nx = a.nx, P = bx.pitch;
    const long long rows = (long long)a.ny * a.nz;
    for (long long row = blockIdx.x; row < rows; row += gridDim.x)
        for (int p = threadIdx.x; p < P; p += 256) dst[row * P + p] = src[row * nx + wrapi(p - VX, nx)];
}

// Batch tiles 0..3: the scalar tiles of the single-box kernel; tile 4: one
// unit per whole 2D box (plane_unit, PLANE_NT threads); tile 5: bands of whole
// rows (band_unit, BAND_NT threads).
constexpr int BATCH_TILES = 7;
constexpr int BATCH_TILE_PLANE = 4;
constexpr int BATCH_TILE_BAND = 5;
constexpr int BATCH_TILE_VBAND = 6;
constexpr int PLANE_NT = 256;
static const int batch_tile_dims[4][2] = {{32, 8}, {32, 16}, {64, 8}, {32, 4}};

}  // namespace cdi

using cdi::BandSlots;
using cdi::BoxDev;
using cdi::StatsRec;

struct cdi_batch {
    int nbox, dtype, total_units, nblocks, parity;
    int tile, zdepth;          // launch configuration: batch tile, planes per unit (0: whole box)
    bool flat;                 // every box has nz == 1: the single-plane kernel
    size_t plane_bytes;        // shared memory of the whole-plane body: 3 nx ny values of the largest box
    int sharpen;               // CDI_SHARPEN_CENTRE or CDI_SHARPEN_FACE (tiles 0 and 4 only)
    BandSlots band;            // row-band body: slot sizes for the largest box
    size_t band_bytes;         // its shared memory (0: the band body does not apply)
    cdi::VbandSlots vband;     // vector row-band body (tile 6): slot sizes for the largest box
    size_t vband_bytes;        // its shared memory (0: it does not apply)
    void *padbuf;              // tile 6: the padded copies of every box (allocated on first use)
    bool vel_packed;           // the padded face velocities are filled
    std::vector<cdi_box_desc> desc;
    void *boxes_dev;           // BoxDev<T>[nbox]
    int *unit_box;             // [unit_cap]
    cdi::Partial *partials;    // [unit_cap]
    size_t unit_cap;
    unsigned int *box_done;    // [nbox] units completed in the current launch
    unsigned int *queue;       // [2] next unit to hand out, blocks finished (self-resetting)
    unsigned int *epoch;       // [nbox] steps of the current run each box has completed
    unsigned int *run_queue;   // [2 run_cap] the counters of a run's launches, zeroed before the run
    int run_cap;
    StatsRec *recs;            // [nbox]
    unsigned int *status;      // status words (checked builds record out-of-range indices)
    long long cells;
    int sms;
    cudaStream_t cap;          // capture stream for graphs
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;  // (nsteps, parity) -> exec
};

template <typename T, int BX, int BY, int BODY, bool FACE = false>
static cudaError_t batch_occ_one(int *resident, size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute(cdi::batch_kernel<T, BX, BY, BODY, FACE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(resident, cdi::batch_kernel<T, BX, BY, BODY, FACE>,
                                                         BX * BY, smem);
}

template <typename T, int BODY>
static cudaError_t batch_occ_t(int tile, int *resident)
{
    switch (tile) {
    case 0: return batch_occ_one<T, 32, 8, BODY>(resident, cdi::FwdSmem<T, 32, 8>::bytes);
    case 1: return batch_occ_one<T, 32, 16, BODY>(resident, cdi::FwdSmem<T, 32, 16>::bytes);
    case 2: return batch_occ_one<T, 64, 8, BODY>(resident, cdi::FwdSmem<T, 64, 8>::bytes);
    case 3: return batch_occ_one<T, 32, 4, BODY>(resident, cdi::FwdSmem<T, 32, 4>::bytes);
    default: return cudaErrorInvalidValue;
    }
}

// Largest dynamic shared memory the whole-plane kernel can launch with (the
// opt-in maximum less its static shared memory); 0 if it cannot be queried.
template <typename T>
static size_t plane_limit()
{
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, cdi::batch_kernel<T, cdi::PLANE_NT, 1, 2>) != cudaSuccess ||
        (size_t)optin <= fa.sharedSizeBytes)
        return 0;
    return ((size_t)optin - fa.sharedSizeBytes) & ~(size_t)15;
}

// Largest dynamic shared memory the band kernel can launch with.
template <typename T>
static size_t band_limit()
{
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, cdi::batch_kernel<T, cdi::BAND_NT, 1, 3>) != cudaSuccess ||
        (size_t)optin <= fa.sharedSizeBytes)
        return 0;
    return ((size_t)optin - fa.sharedSizeBytes) & ~(size_t)15;
}

// Largest dynamic shared memory the vector band kernel can launch with.
template <typename T>
static size_t vband_limit()
{
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, cdi::batch_kernel<T, cdi::VBAND_NT, 1, 4>) != cudaSuccess ||
        (size_t)optin <= fa.sharedSizeBytes)
        return 0;
    return ((size_t)optin - fa.sharedSizeBytes) & ~(size_t)15;
}

template <typename T>
static cudaError_t batch_occ(const cdi_batch *b, int tile, int *resident)
{
    if (b->sharpen == CDI_SHARPEN_FACE) {  // face-product sharpening: tiles 0 and 4
        if (tile == 0)
            return b->flat ? batch_occ_one<T, 32, 8, 1, true>(resident, cdi::FwdSmem<T, 32, 8>::bytes)
                           : batch_occ_one<T, 32, 8, 0, true>(resident, cdi::FwdSmem<T, 32, 8>::bytes);
        if (tile != cdi::BATCH_TILE_PLANE) return cudaErrorInvalidValue;
        const size_t lim = plane_limit<T>();
        if (lim == 0 || b->plane_bytes > lim) return cudaErrorInvalidValue;
        cudaError_t e = cudaFuncSetAttribute(cdi::batch_kernel<T, cdi::PLANE_NT, 1, 2, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(resident, cdi::batch_kernel<T, cdi::PLANE_NT, 1, 2, true>,
                                                             cdi::PLANE_NT, b->plane_bytes);
    }
    if (tile == cdi::BATCH_TILE_VBAND) {
        const size_t lim = vband_limit<T>();
        if (lim == 0 || b->vband_bytes == 0 || b->vband_bytes > lim) return cudaErrorInvalidValue;
        cudaError_t e = cudaFuncSetAttribute(cdi::batch_kernel<T, cdi::VBAND_NT, 1, 4>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(resident, cdi::batch_kernel<T, cdi::VBAND_NT, 1, 4>,
                                                             cdi::VBAND_NT, b->vband_bytes);
    }
    if (tile == cdi::BATCH_TILE_BAND) {
        const size_t lim = band_limit<T>();
        if (lim == 0 || b->band_bytes == 0 || b->band_bytes > lim) return cudaErrorInvalidValue;
        cudaError_t e = cudaFuncSetAttribute(cdi::batch_kernel<T, cdi::BAND_NT, 1, 3>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(resident, cdi::batch_kernel<T, cdi::BAND_NT, 1, 3>,
                                                             cdi::BAND_NT, b->band_bytes);
    }
    if (tile == cdi::BATCH_TILE_PLANE) {
        // The attribute belongs to the kernel, shared by every batch: it is set
        // to the largest size any batch launches with, the occupancy taken at
        // this batch's size.
        const size_t lim = plane_limit<T>();
        if (lim == 0 || b->plane_bytes > lim) return cudaErrorInvalidValue;
        cudaError_t e = cudaFuncSetAttribute(cdi::batch_kernel<T, cdi::PLANE_NT, 1, 2>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(resident, cdi::batch_kernel<T, cdi::PLANE_NT, 1, 2>,
                                                             cdi::PLANE_NT, b->plane_bytes);
    }
    return b->flat ? batch_occ_t<T, 1>(tile, resident) : batch_occ_t<T, 0>(tile, resident);
}

// Shared memory the whole-plane body needs for this batch (3 nx ny values of
// its largest box), 0 if some box is 3D or does not fit.
template <typename T>
static size_t plane_bytes_t(const cdi_batch *b)
{
    if (!b->flat) return 0;
    size_t need = 0;
    for (const cdi_box_desc &x : b->desc) {
        const size_t bytes = 3 * sizeof(T) * (size_t)x.nx * (size_t)x.ny;
        if (bytes > need) need = bytes;
    }
    need = (need + 15) & ~(size_t)15;
    return need <= plane_limit<T>() ? need : 0;
}

static size_t plane_bytes(const cdi_batch *b)
{
    return b->dtype == CDI_F64 ? plane_bytes_t<double>(b) : plane_bytes_t<float>(b);
}

// Slot sizes of the row-band body for this batch (the largest region of each kind
// over its boxes) and their shared memory; 0 bytes if the band body does not apply:
// a batch of 2D boxes only (which has its own bodies), a row wider than a band, or
// slots beyond the shared memory of one block.
template <typename T>
static size_t band_bytes_t(cdi_batch *b)
{
    if (b->flat) return 0;
    const int vx = 16 / (int)sizeof(T);
    int phi = 0, ur = 0, vr = 0, sx = 0, sy = 0;
    for (const cdi_box_desc &x : b->desc) {
        if (x.nx > cdi::BAND_CELLS) return 0;
        const int hb = cdi::band_rows(x.nx, x.ny);
        phi = std::max(phi, cdi::round_up((hb + 4) * x.nx + vx, vx));
        ur = std::max(ur, cdi::round_up(hb * x.nx + vx, vx));
        vr = std::max(vr, cdi::round_up((hb + 1) * x.nx + vx, vx));
        sx = std::max(sx, cdi::round_up(hb * x.nx, vx));
        sy = std::max(sy, cdi::round_up((hb + 2) * x.nx, vx));
    }
    BandSlots s;
    s.phi = phi;
    s.uo = 0;
    s.vo = ur;
    s.wo = ur + vr;
    s.vel = 2 * ur + vr;
    s.sx = sx;
    s.sy = sy;
    const size_t need = cdi::band_smem_bytes(s, sizeof(T));
    if (need > band_limit<T>()) return 0;
    b->band = s;
    return need;
}

static size_t band_bytes(cdi_batch *b)
{
    return b->dtype == CDI_F64 ? band_bytes_t<double>(b) : band_bytes_t<float>(b);
}

// Slot sizes of the vector band body for this batch (each slot field the largest
// over its boxes, the velocity regions laid out one after another) and their
// shared memory; 0 if they exceed the shared memory of one block.
template <typename T>
static size_t vband_bytes_t(cdi_batch *b)
{
    const int vx = 16 / (int)sizeof(T);
    if (b->nbox > 65535) return 0;  // the copy kernels take the box from blockIdx.y
    int phi = 0, ur = 0, vr = 0, sx = 0, sy = 0;
    for (const cdi_box_desc &x : b->desc) {
        if ((x.nx + vx - 1) / vx > cdi::VBAND_NT) return 0;  // a row has more groups than the block threads
        const int P = cdi::vband_pitch(x.nx, vx), hb = cdi::vband_rows(x.nx, x.ny, vx);
        if (hb < 1) return 0;  // a padded row too wide for the staging plan
        const cdi::VbandSlots t = cdi::vband_slots(P, hb);
        phi = std::max(phi, t.phi);
        ur = std::max(ur, hb * P);
        vr = std::max(vr, (hb + 1) * P);
        sx = std::max(sx, t.sx);
        sy = std::max(sy, t.sy);
    }
    cdi::VbandSlots s;
    s.phi = phi;
    s.vo = ur;
    s.wo = ur + vr;
    s.vel = 2 * ur + vr;
    s.sx = sx;
    s.sy = sy;
    const size_t need = cdi::vband_smem_bytes(s, sizeof(T));
    if (need > vband_limit<T>()) return 0;
    b->vband = s;
    return need;
}

static size_t vband_bytes(cdi_batch *b)
{
    return b->dtype == CDI_F64 ? vband_bytes_t<double>(b) : vband_bytes_t<float>(b);
}

static int batch_free(cdi_batch *b)
{
    if (!b) return CDI_OK;
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaFree(b->boxes_dev);
    cudaFree(b->unit_box);
    cudaFree(b->partials);
    cudaFree(b->box_done);
    cudaFree(b->queue);
    cudaFree(b->epoch);
    cudaFree(b->run_queue);
    cudaFree(b->recs);
    cudaFree(b->status);
    cudaFree(b->padbuf);
    delete b;
    return CDI_OK;
}

static void drop_graphs(cdi_batch *b)
{
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

// Box table and work list for a tile and a z depth, uploaded to the device
// (synchronous; the device arrays grow when needed).
template <typename T>
static int build_units(cdi_batch *b, int tile, int zdepth)
{
    const bool plane = tile == cdi::BATCH_TILE_PLANE, band = tile == cdi::BATCH_TILE_BAND;
    const bool vband = tile == cdi::BATCH_TILE_VBAND;
    constexpr int VX = 16 / sizeof(T);
    if (plane && b->plane_bytes == 0)
        return cdi::set_error(CDI_ERR_ARG, "batch tile 4 needs 2D boxes (nz = 1) whose planes fit in shared memory");
    if (band && b->band_bytes == 0)
        return cdi::set_error(CDI_ERR_ARG, "batch tile 5 needs a batch with 3D boxes whose rows fit in a band "
                                           "(nx <= %d) and whose band slots fit in shared memory", cdi::BAND_CELLS);
    if (vband && b->vband_bytes == 0)
        return cdi::set_error(CDI_ERR_ARG, "batch tile 6 needs padded rows of at most %d vectors and band "
                                           "slots that fit in the shared memory of a block",
                                           cdi::VBAND_CPY * cdi::VBAND_NT / 5);
    cudaError_t e;
    if (vband && !b->padbuf) {  // the padded copies: state x 2, u, v, w per box
        size_t n = 0;
        for (const cdi_box_desc &x : b->desc) n += 5 * (size_t)cdi::vband_pitch(x.nx, VX) * x.ny * x.nz;
        if ((e = cudaMalloc(&b->padbuf, n * sizeof(T))) != cudaSuccess) {
            b->padbuf = nullptr;
            return cdi::set_error(CDI_ERR_CUDA, "batch padded copies (%zu bytes): %s", n * sizeof(T),
                                  cudaGetErrorString(e));
        }
        b->vel_packed = false;
    }
    const int bw = plane || band || vband ? 1 : cdi::batch_tile_dims[tile][0];
    const int bh = plane || band || vband ? 1 : cdi::batch_tile_dims[tile][1];
    T *pad = (T *)b->padbuf;
    std::vector<BoxDev<T>> tab;
    std::vector<int> ub;
    int unit = 0;
    long long cells = 0;
    for (int i = 0; i < b->nbox; ++i) {
        const cdi_box_desc &x = b->desc[i];
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
        e.a.red.status = b->status;
        const int Df = (x.nx > 1) + (x.ny > 1) + (x.nz > 1);
        e.dV = pow(x.dx, (double)Df);
        e.tiles_x = plane || band || vband ? 1 : (x.nx + bw - 1) / bw;
        e.ntiles = plane ? 1 : e.tiles_x * ((x.ny + bh - 1) / bh);  // whole-plane body: one unit per box
        if (band) {  // bands of whole rows
            e.bh = cdi::band_rows(x.nx, x.ny);
            e.ntiles = (x.ny + e.bh - 1) / e.bh;
        }
        if (vband) {  // bands of whole padded rows
            e.bh = cdi::vband_rows(x.nx, x.ny, VX);
            e.ntiles = (x.ny + e.bh - 1) / e.bh;
        }
        if (pad) {  // the padded copies (laid out box after box)
            e.pitch = cdi::vband_pitch(x.nx, VX);
            const size_t n = (size_t)e.pitch * x.ny * x.nz;
            e.pad[0] = pad;
            e.pad[1] = pad + n;
            e.pu = pad + 2 * n;
            e.pv = pad + 3 * n;
            e.pw = pad + 4 * n;
            pad += 5 * n;
        }
        int nch = zdepth > 0 && !plane ? (x.nz + zdepth / 2) / zdepth : 1;  // about zdepth planes per unit
        if (nch < 1) nch = 1;
        e.zc = (x.nz + nch - 1) / nch;
        e.nunits = e.ntiles * ((x.nz + e.zc - 1) / e.zc);
        if ((long long)unit + e.nunits >= (1LL << 31)) return cdi::set_error(CDI_ERR_DIM, "too many work units");
        unit += e.nunits;
        cells += (long long)x.nx * x.ny * x.nz;
        tab.push_back(e);
    }
    // The boxes' unit ranges in the list by decreasing unit size (cells of a unit's
    // plane times its planes plus a prologue of about four), so that the blocks
    // taking units from the list end on the smallest ones.
    std::vector<int> order(b->nbox);
    std::vector<double> ucost(b->nbox);
    for (int i = 0; i < b->nbox; ++i) {
        const cdi_box_desc &x = b->desc[i];
        order[i] = i;
        ucost[i] = (double)x.nx * x.ny / tab[i].ntiles * (tab[i].zc + 4.0);
    }
    std::stable_sort(order.begin(), order.end(), [&](int p, int q) { return ucost[p] > ucost[q]; });
    unit = 0;
    for (int i : order) {
        tab[i].unit0 = unit;
        for (int k = 0; k < tab[i].nunits; ++k) ub.push_back(i);
        unit += tab[i].nunits;
    }
    int resident = 0;
    e = batch_occ<T>(b, tile, &resident);
    if (e != cudaSuccess) return cdi::set_error(CDI_ERR_CUDA, "batch occupancy: %s", cudaGetErrorString(e));
    if (resident < 1) return cdi::set_error(CDI_ERR_CUDA, "batch kernel does not fit on an SM");
    if (ub.size() > b->unit_cap) {
        cudaFree(b->unit_box);
        cudaFree(b->partials);
        b->unit_box = nullptr;
        b->partials = nullptr;
        b->unit_cap = 0;
        if ((e = cudaMalloc(&b->unit_box, sizeof(int) * ub.size())) != cudaSuccess ||
            (e = cudaMalloc(&b->partials, sizeof(cdi::Partial) * ub.size())) != cudaSuccess)
            return cdi::set_error(CDI_ERR_CUDA, "batch allocation: %s", cudaGetErrorString(e));
        b->unit_cap = ub.size();
    }
    if (!b->boxes_dev && (e = cudaMalloc(&b->boxes_dev, sizeof(BoxDev<T>) * b->nbox)) != cudaSuccess)
        return cdi::set_error(CDI_ERR_CUDA, "batch allocation: %s", cudaGetErrorString(e));
    // The previous configuration's launches may still read the old tables.
    if ((e = cudaDeviceSynchronize()) != cudaSuccess ||
        (e = cudaMemcpy(b->boxes_dev, tab.data(), sizeof(BoxDev<T>) * b->nbox, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->unit_box, ub.data(), sizeof(int) * ub.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cdi::set_error(CDI_ERR_CUDA, "batch tables: %s", cudaGetErrorString(e));
    if (vband && !b->vel_packed) {  // the face velocities do not change: padded once
        for (int which = 2; which <= 4; ++which)
            cdi::vband_pack<T><<<dim3(256, b->nbox), 256>>>((const BoxDev<T> *)b->boxes_dev, which);
        if ((e = cudaDeviceSynchronize()) != cudaSuccess)
            return cdi::set_error(CDI_ERR_CUDA, "batch padded velocities: %s", cudaGetErrorString(e));
        b->vel_packed = true;
    }
    long long nb = (long long)resident * b->sms;
    if (nb > unit) nb = unit;
    if (nb < 1) nb = 1;
    drop_graphs(b);
    b->tile = tile;
    b->zdepth = zdepth;
    b->total_units = unit;
    b->nblocks = (int)nb;
    b->cells = cells;
    return CDI_OK;
}

static int rebuild(cdi_batch *b, int tile, int zdepth)
{
    return b->dtype == CDI_F64 ? build_units<double>(b, tile, zdepth) : build_units<float>(b, tile, zdepth);
}

// One launch of a batch kernel instantiation.  Launches after the first of a
// run are made with programmatic stream serialisation: they start while the
// launch before is finishing, ordered per box by the epochs (BatchSync).
template <typename T, int BX, int BY, int BODY, bool FACE = false>
static cudaError_t launch_batch_kernel(cdi_batch *b, size_t smem, int parity, double vs, cudaStream_t s,
                                       int final_write, const cdi::BatchSync &y)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)b->nblocks);
    cfg.blockDim = dim3(BX, BY);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = y.step > 0 && !y.reset ? 1 : 0;  // a run's launches after its first
    return cudaLaunchKernelEx(&cfg, cdi::batch_kernel<T, BX, BY, BODY, FACE>, (const BoxDev<T> *)b->boxes_dev,
                              (const int *)b->unit_box, b->total_units, parity, (T)vs, b->partials, b->box_done,
                              b->recs, b->band, b->vband, final_write, y);
}

template <typename T, int BX, int BY>
static cudaError_t batch_launch_one(cdi_batch *b, int parity, double vs, cudaStream_t s, const cdi::BatchSync &y)
{
    const size_t smem = cdi::FwdSmem<T, BX, BY>::bytes;
    if (BX == 32 && BY == 8 && b->sharpen == CDI_SHARPEN_FACE)
        return b->flat ? launch_batch_kernel<T, 32, 8, 1, true>(b, smem, parity, vs, s, 0, y)
                       : launch_batch_kernel<T, 32, 8, 0, true>(b, smem, parity, vs, s, 0, y);
    return b->flat ? launch_batch_kernel<T, BX, BY, 1>(b, smem, parity, vs, s, 0, y)
                   : launch_batch_kernel<T, BX, BY, 0>(b, smem, parity, vs, s, 0, y);
}

template <typename T>
static cudaError_t batch_launch_plane(cdi_batch *b, int parity, double vs, cudaStream_t s, const cdi::BatchSync &y)
{
    if (b->sharpen == CDI_SHARPEN_FACE)
        return launch_batch_kernel<T, cdi::PLANE_NT, 1, 2, true>(b, b->plane_bytes, parity, vs, s, 0, y);
    return launch_batch_kernel<T, cdi::PLANE_NT, 1, 2>(b, b->plane_bytes, parity, vs, s, 0, y);
}

// Tile 6: copy the current state (the caller's array of this parity) into the
// padded copy of that parity; the steps of a call then read and write the padded
// copies, the last of them the caller's array too.
static int vband_pack_state(cdi_batch *b, int parity, cudaStream_t s)
{
    if (b->dtype == CDI_F64)
        cdi::vband_pack<double><<<dim3(256, b->nbox), 256, 0, s>>>((const BoxDev<double> *)b->boxes_dev, parity);
    else
        cdi::vband_pack<float><<<dim3(256, b->nbox), 256, 0, s>>>((const BoxDev<float> *)b->boxes_dev, parity);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cdi::set_error(CDI_ERR_CUDA, "batch pack: %s", cudaGetErrorString(e));
    return CDI_OK;
}

template <typename T>
static int batch_launch(cdi_batch *b, int parity, double vs, cudaStream_t s, int final_write,
                        const cdi::BatchSync &y)
{
    cudaError_t e;
    switch (b->tile) {
    case 0: e = batch_launch_one<T, 32, 8>(b, parity, vs, s, y); break;
    case 1: e = batch_launch_one<T, 32, 16>(b, parity, vs, s, y); break;
    case 2: e = batch_launch_one<T, 64, 8>(b, parity, vs, s, y); break;
    case 3: e = batch_launch_one<T, 32, 4>(b, parity, vs, s, y); break;
    case cdi::BATCH_TILE_PLANE: e = batch_launch_plane<T>(b, parity, vs, s, y); break;
    case cdi::BATCH_TILE_BAND:
        e = launch_batch_kernel<T, cdi::BAND_NT, 1, 3>(b, b->band_bytes, parity, vs, s, 0, y);
        break;
    case cdi::BATCH_TILE_VBAND:
        e = launch_batch_kernel<T, cdi::VBAND_NT, 1, 4>(b, b->vband_bytes, parity, vs, s, final_write, y);
        break;
    default: return cdi::set_error(CDI_ERR_STATE, "bad batch tile");
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cdi::set_error(CDI_ERR_CUDA, "batch launch: %s", cudaGetErrorString(e));
    return CDI_OK;
}

// One step of every box; final_write (tile 6): the step also writes the caller's
// arrays (the last step of a call).  y: the step's place in a run (nullptr: a
// launch on its own, after everything before it on the stream).
static int launch_any(cdi_batch *b, int parity, double vs, cudaStream_t s, int final_write = 1,
                      const cdi::BatchSync *y = nullptr)
{
    const cdi::BatchSync single = {b->queue, b->epoch, 0, 1, 0ull};
    const cdi::BatchSync &sy = y ? *y : single;
    return b->dtype == CDI_F64 ? batch_launch<double>(b, parity, vs, s, final_write, sy)
                               : batch_launch<float>(b, parity, vs, s, final_write, sy);
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
    for (int i = 0; i < nbox; ++i) {
        const cdi_box_desc &x = boxes[i];
        if (x.nx < 1 || x.ny < 1 || x.nz < 1 || (long long)x.nx * x.ny >= (1LL << 31))
            return cdi::set_error(CDI_ERR_DIM, "box %d: bad extents", i);
        if (!(x.dx > 0) || !(x.dt >= 0) || !(x.eps > 0) || !(x.gamma >= 0))
            return cdi::set_error(CDI_ERR_ARG, "box %d: bad dx, dt, eps or gamma", i);
        if (!x.phi_a || !x.phi_b || !x.u || (!x.v && !(x.ny == 1 && x.nz == 1)) || (!x.w && x.nz != 1))
            return cdi::set_error(CDI_ERR_ARG, "box %d: NULL array", i);
    }
    cdi_batch *b = new cdi_batch();
    b->nbox = nbox;
    b->dtype = dtype;
    b->desc.assign(boxes, boxes + nbox);
    b->flat = true;
    for (int i = 0; i < nbox; ++i) b->flat = b->flat && boxes[i].nz == 1;
    b->plane_bytes = plane_bytes(b);
    b->band_bytes = band_bytes(b);
    b->vband_bytes = vband_bytes(b);
    cudaError_t e;
    int dev = 0;
    std::vector<StatsRec> hrec(nbox);
    reset_recs(hrec);
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaMalloc(&b->box_done, sizeof(unsigned int) * nbox)) != cudaSuccess ||
        (e = cudaMalloc(&b->queue, sizeof(unsigned int) * 2)) != cudaSuccess ||
        (e = cudaMemset(b->queue, 0, sizeof(unsigned int) * 2)) != cudaSuccess ||
        (e = cudaMalloc(&b->epoch, sizeof(unsigned int) * nbox)) != cudaSuccess ||
        (e = cudaMemset(b->epoch, 0, sizeof(unsigned int) * nbox)) != cudaSuccess ||
        (e = cudaMalloc(&b->recs, sizeof(StatsRec) * nbox)) != cudaSuccess ||
        (e = cudaMalloc(&b->status, sizeof(unsigned int) * cdi::kStatusWords)) != cudaSuccess ||
        (e = cudaMemset(b->status, 0, sizeof(unsigned int) * cdi::kStatusWords)) != cudaSuccess ||
        (e = cudaMemset(b->box_done, 0, sizeof(unsigned int) * nbox)) != cudaSuccess ||
        (e = cudaMemcpy(b->recs, hrec.data(), sizeof(StatsRec) * nbox, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess) {
        batch_free(b);
        return cdi::set_error(CDI_ERR_CUDA, "batch setup: %s", cudaGetErrorString(e));
    }
    if (int rc = rebuild(b, 0, CDI_BATCH_DEFAULT_ZDEPTH)) {
        batch_free(b);
        return rc;
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
    cdi::NvtxRange nvtx_("cdi_batch_step");
    if (!b) return cdi::set_error(CDI_ERR_ARG, "batch is NULL");
    if (!isfinite(vel_scale)) return cdi::set_error(CDI_ERR_ARG, "vel_scale must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = b->tile == cdi::BATCH_TILE_VBAND ? vband_pack_state(b, b->parity, s) : CDI_OK;
    if (rc == CDI_OK) rc = launch_any(b, b->parity, vel_scale, s);
    if (rc == CDI_OK) b->parity ^= 1;
    return rc;
}

int cdi_batch_run(cdi_batch *b, int nsteps, void *stream)
{
    cdi::NvtxRange nvtx_("cdi_batch_run");
    if (!b) return cdi::set_error(CDI_ERR_ARG, "batch is NULL");
    if (nsteps < 1) return cdi::set_error(CDI_ERR_ARG, "nsteps must be >= 1");
    const std::pair<int, int> key(nsteps, b->parity);
    auto it = b->graphs.find(key);
    cudaError_t e;
    if (it == b->graphs.end()) {
        if (nsteps > b->run_cap) {  // one counter pair per launch of the run
            if ((e = cudaDeviceSynchronize()) != cudaSuccess)  // no graph in flight uses the old counters
                return cdi::set_error(CDI_ERR_CUDA, "batch run: %s", cudaGetErrorString(e));
            drop_graphs(b);
            cudaFree(b->run_queue);
            b->run_queue = nullptr;
            b->run_cap = 0;
            if ((e = cudaMalloc(&b->run_queue, sizeof(unsigned int) * 2 * (size_t)nsteps)) != cudaSuccess) {
                b->run_queue = nullptr;
                return cdi::set_error(CDI_ERR_CUDA, "batch run counters: %s", cudaGetErrorString(e));
            }
            b->run_cap = nsteps;
        }
        // Capture nsteps launches (parity alternating) once on the private stream:
        // the run's counters and box epochs zeroed, then the steps, each after the
        // first overlapping the one before (BatchSync).
        cudaGraph_t graph;
        if ((e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return cdi::set_error(CDI_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
        int rc = CDI_OK;
        if ((e = cudaMemsetAsync(b->run_queue, 0, sizeof(unsigned int) * 2 * (size_t)nsteps, b->cap)) != cudaSuccess ||
            (e = cudaMemsetAsync(b->epoch, 0, sizeof(unsigned int) * b->nbox, b->cap)) != cudaSuccess ||
            (e = cudaMemsetAsync(b->box_done, 0, sizeof(unsigned int) * b->nbox, b->cap)) != cudaSuccess)
            rc = cdi::set_error(CDI_ERR_CUDA, "batch run counters: %s", cudaGetErrorString(e));
        if (rc == CDI_OK && b->tile == cdi::BATCH_TILE_VBAND) rc = vband_pack_state(b, b->parity, b->cap);
        // a unit waits at most about one step: one second plus 2 ns per cell (a step
        // of the slowest tile takes well under 1 ns per cell)
        const unsigned long long wait_ns = 1000000000ull + 2ull * (unsigned long long)b->cells;
        for (int i = 0; i < nsteps && rc == CDI_OK; ++i) {
            const cdi::BatchSync y = {b->run_queue + 2 * i, b->epoch, i, 0, wait_ns};
            rc = launch_any(b, b->parity ^ (i & 1), 1.0, b->cap, i == nsteps - 1, &y);
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
    unsigned int st[cdi::kStatusWords] = {0, 0, 0, 0};
    if ((e = cudaMemcpyAsync(out, b->recs, sizeof(StatsRec) * b->nbox, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(st, b->status, sizeof(st), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cdi::set_error(CDI_ERR_CUDA, "batch statistics: %s", cudaGetErrorString(e));
    if (st[0]) {
        cudaMemsetAsync(b->status, 0, sizeof(st), s);
        if (st[0] & 2u)
            return cdi::set_error(CDI_ERR_BOUNDS,
                                  "checked build: %u index(es) out of range, the last %u against a limit of %u",
                                  st[1], st[2], st[3]);
        return cdi::set_error(CDI_ERR_TIMEOUT, "a bounded wait for a box's previous step gave up; "
                                               "results are unreliable");
    }
    for (int i = 0; i < b->nbox; ++i)
        if (!isfinite(out[i].sum)) return cdi::set_error(CDI_ERR_NAN, "box %d: non-finite phi", i);
    return CDI_OK;
}

// One launch whose units wait for a step their boxes never reach: the first wait
// runs out after limit_s, the others give up on seeing its status bit, and no
// unit is stepped (fields, records and counters are left as they were).
int cdi_batch_probe_box_wait(cdi_batch *b, double limit_s, void *stream)
{
    if (!b) return cdi::set_error(CDI_ERR_ARG, "batch is NULL");
    if (!(limit_s > 0.0 && limit_s <= 2.0)) return cdi::set_error(CDI_ERR_ARG, "limit_s must be in (0, 2]");
    cudaStream_t s = (cudaStream_t)stream;
    const cdi::BatchSync y = {b->queue, b->epoch, 1 << 30, 1, (unsigned long long)(limit_s * 1e9)};
    if (int rc = launch_any(b, b->parity, 1.0, s, 0, &y)) return rc;
    unsigned int st = 0;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(&st, b->status, sizeof(st), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cdi::set_error(CDI_ERR_CUDA, "probe status readback: %s", cudaGetErrorString(e));
    if (!(st & 1u)) return CDI_OK;  // the waits did not run out: the time-out path is broken
    if ((e = cudaMemsetAsync(b->status, 0, sizeof(unsigned int) * cdi::kStatusWords, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cdi::set_error(CDI_ERR_CUDA, "probe status reset: %s", cudaGetErrorString(e));
    return cdi::set_error(CDI_ERR_TIMEOUT, "bounded wait for a box's previous step ran out (probe)");
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

int cdi_batch_set_launch(cdi_batch *b, int tile, int zdepth)
{
    if (!b) return cdi::set_error(CDI_ERR_ARG, "batch is NULL");
    if (tile < -1 || tile >= cdi::BATCH_TILES) return cdi::set_error(CDI_ERR_ARG, "batch tile %d out of range", tile);
    if (zdepth < -1) return cdi::set_error(CDI_ERR_ARG, "zdepth must be >= -1");
    if (b->sharpen == CDI_SHARPEN_FACE && tile != 0 && tile != cdi::BATCH_TILE_PLANE && tile != -1)
        return cdi::set_error(CDI_ERR_ARG, "face-product sharpening runs on batch tiles 0 and 4 only");
    return rebuild(b, tile < 0 ? 0 : tile, zdepth < 0 ? CDI_BATCH_DEFAULT_ZDEPTH : zdepth);
}

int cdi_batch_set_sharpening(cdi_batch *b, int mode)
{
    if (!b) return cdi::set_error(CDI_ERR_ARG, "batch is NULL");
    if (mode != CDI_SHARPEN_CENTRE && mode != CDI_SHARPEN_FACE)
        return cdi::set_error(CDI_ERR_ARG, "sharpening mode %d", mode);
    const int old = b->sharpen;
    b->sharpen = mode;
    if (int rc = rebuild(b, 0, b->zdepth)) {
        b->sharpen = old;
        return rc;
    }
    return CDI_OK;
}

int cdi_batch_get_sharpening(const cdi_batch *b, int *mode)
{
    if (!b || !mode) return cdi::set_error(CDI_ERR_ARG, "NULL argument");
    *mode = b->sharpen;
    return CDI_OK;
}

int cdi_batch_get_launch(const cdi_batch *b, int *tile, int *zdepth, int *nblocks, int *total_units)
{
    if (!b) return cdi::set_error(CDI_ERR_ARG, "batch is NULL");
    if (tile) *tile = b->tile;
    if (zdepth) *zdepth = b->zdepth;
    if (nblocks) *nblocks = b->nblocks;
    if (total_units) *total_units = b->total_units;
    return CDI_OK;
}

int cdi_batch_autotune(cdi_batch *b, int reps, float *best_ms, void *stream)
{
    cdi::NvtxRange nvtx_("cdi_batch_autotune");
    if (!b) return cdi::set_error(CDI_ERR_ARG, "batch is NULL");
    if (reps < 1) return cdi::set_error(CDI_ERR_ARG, "reps must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    // Trial launches all read the current state and write the other buffer (the
    // next step overwrites it anyway); they do update the statistics records,
    // which are saved here and put back afterwards.
    std::vector<StatsRec> saved(b->nbox);
    cudaError_t e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess ||
        (e = cudaMemcpy(saved.data(), b->recs, sizeof(StatsRec) * b->nbox, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cdi::set_error(CDI_ERR_CUDA, "batch autotune: %s", cudaGetErrorString(e));
    cudaEvent_t e0, e1;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return cdi::set_error(CDI_ERR_CUDA, "cudaEventCreate");
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cdi::set_error(CDI_ERR_CUDA, "cudaEventCreate");
    }
    // (2D batches: the z depth changes nothing, one trial per tile; the
    // whole-plane tile where the planes fit)
    const int zopts[] = {8, 16, 32, 64, 0};
    const int nz_opts = b->flat ? 1 : (int)(sizeof(zopts) / sizeof(int));
    int best_tile = b->tile, best_z = b->zdepth, rc = CDI_OK;
    float best_t = 1e30f;
    for (int tile = 0; tile < cdi::BATCH_TILES && rc == CDI_OK; ++tile) {
        if (tile == cdi::BATCH_TILE_PLANE && b->plane_bytes == 0) continue;
        if (tile == cdi::BATCH_TILE_BAND && b->band_bytes == 0) continue;
        if (tile == cdi::BATCH_TILE_VBAND && b->vband_bytes == 0) continue;
        if (b->sharpen == CDI_SHARPEN_FACE && tile != 0 && tile != cdi::BATCH_TILE_PLANE) continue;
        for (int zi = 0; zi < nz_opts && rc == CDI_OK; ++zi) {
            if ((rc = rebuild(b, tile, zopts[zi])) != CDI_OK) break;
            // tile 6: the state packed once, then steps between the padded copies as in a run
            if (tile == cdi::BATCH_TILE_VBAND && (rc = vband_pack_state(b, b->parity, s)) != CDI_OK) break;
            if ((rc = launch_any(b, b->parity, 1.0, s, 0)) != CDI_OK) break;  // warm-up
            if ((e = cudaEventRecord(e0, s)) != cudaSuccess) {
                rc = cdi::set_error(CDI_ERR_CUDA, "event: %s", cudaGetErrorString(e));
                break;
            }
            for (int i = 0; i < reps && rc == CDI_OK; ++i) rc = launch_any(b, b->parity, 1.0, s, 0);
            if (rc != CDI_OK) break;
            if ((e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) {
                rc = cdi::set_error(CDI_ERR_CUDA, "event: %s", cudaGetErrorString(e));
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= reps;
            if (ms < best_t) {
                best_t = ms;
                best_tile = tile;
                best_z = zopts[zi];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != CDI_OK) return rc;
    if ((rc = rebuild(b, best_tile, best_z)) != CDI_OK) return rc;
    if ((e = cudaMemcpy(b->recs, saved.data(), sizeof(StatsRec) * b->nbox, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cdi::set_error(CDI_ERR_CUDA, "batch autotune: %s", cudaGetErrorString(e));
    if (best_ms) *best_ms = best_t;
    return CDI_OK;
}
