// Fused CDI step with tile staging by the Tensor Memory Accelerator (TMA).
//
// Same arithmetic and structure as fwd_vec_kernel (cdi_fwd.cu): a block owns a
// 64 x 16 (FP32; 32 x 16 FP64) x-y tile, each of its 256 "own" threads a
// 16-byte vector of x-cells, two extra warps compute the sharpening ring, and
// the block marches along z over a chunk of planes, one barrier per plane.
// What differs is how planes reach shared memory: per plane, one elected
// thread issues seven 2-D tensor copies (cp.async.bulk.tensor) --
//   phi: the tile core (W x H) and the two 2-row halos above and below,
//   u, w: the tile core; v: the core and the row below --
// completing on an mbarrier, and 56 threads copy the 16-byte x-halo columns
// (phi on both sides, u on the left) with cp.async.  Tensor copies write
// dense rows, so the slot layout keeps the x-halos in separate side arrays.
// Requires nx % W == 0 and ny % H == 0 (no tile overhangs the grid and no box
// crosses the periodic edge); the host checks this.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "cdi_async.cuh"
#include "cdi_fwd_common.cuh"
#include "cdi_internal.cuh"
#include "cdi_reduce.cuh"

namespace cdi {

template <typename T>
struct TmaCfg {
    static constexpr int VX = 16 / sizeof(T);
    static constexpr int TX = 16, TY = 16;
    static constexpr int W = TX * VX, H = TY;
    static constexpr int NOWN = TX * TY;
    static constexpr int NT = NOWN + 64;
    static constexpr int PR = H + 4;                     // phi rows y0-2 .. y0+H+1
    static constexpr int SIDE = PR * 2 * VX;             // x-halos: [PR][left VX | right VX]
    static constexpr int PHI = PR * W + SIDE;
    static constexpr int UC = H * W, UH = H * VX;        // u core, u left halo
    static constexpr int VV = (H + 1) * W, WW = H * W;   // v rows y0-1 .. y0+H-1; w core
    static constexpr int VEL = UC + UH + VV + WW;
    static constexpr int SXP = W + 2 * VX, SXS = H * SXP, SYS = (H + 2) * W;
    static constexpr int NSP = 5, NSV = 3;
    static constexpr size_t data_bytes = sizeof(T) * (size_t)(NSP * PHI + NSV * VEL + 2 * SXS + 2 * SYS);
    static constexpr size_t bytes = data_bytes + 4 * 8 + 128;  // + barriers + alignment slack
    static_assert((sizeof(T) * PHI) % 128 == 0 && (sizeof(T) * VEL) % 128 == 0, "slot alignment");
    static_assert((sizeof(T) * 2 * W) % 128 == 0, "tensor-copy destinations on 128-byte boundaries");
    static_assert((sizeof(T) * (UC + UH)) % 128 == 0, "v destination alignment");
};

struct TmaMaps {
    CUtensorMap phi2;  // phi, box W x 2
    CUtensorMap phiH;  // phi, box W x H
    CUtensorMap u;     // box W x H
    CUtensorMap vH;    // box W x H
    CUtensorMap v1;    // box W x 1
    CUtensorMap w;     // box W x H
};

__device__ __forceinline__ void tma_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                       unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

template <typename T>
__global__ void __launch_bounds__(TmaCfg<T>::NT, 2)
fwd_tma_kernel(const FwdArgs<T> a, const __grid_constant__ TmaMaps maps, const int nchunks)
{
    using C = TmaCfg<T>;
    using VV = V16<T>;
    constexpr int VX = C::VX, W = C::W, H = C::H, TX = C::TX, SXP = C::SXP, PR = C::PR;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((128 - (smem_addr(smem_raw) & 127)) & 127);
    T *const sphi = reinterpret_cast<T *>(base);
    T *const svel = sphi + C::NSP * C::PHI;
    T *const ssx = svel + C::NSV * C::VEL;
    T *const ssy = ssx + 2 * C::SXS;
    unsigned long long *const bars = reinterpret_cast<unsigned long long *>(ssy + 2 * C::SYS);

    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long plane = (long long)nx * ny;
    const int tiles_x = nx / W;
    const int ntiles = tiles_x * (ny / H);
    const T c_adv = a.c.c_adv, c_dif = a.c.c_dif, c_shp = a.c.c_shp, c_upd = a.c.c_upd;

    const bool is_own = tid < C::NOWN;
    const int tx = tid % TX, ty = tid / TX;
    const int rr = tid - C::NOWN;  // 0..63 for the ring threads
    const bool is_yring = !is_own && rr < 32;
    const bool is_xring = !is_own && rr >= 32;
    const int ry_row = (rr < TX) ? -1 : H, ry_col = rr % TX;
    const int rx_row = (rr - 32) % C::TY;
    const bool rx_left = (rr - 32) < C::TY;
    const bool tma_thread = tid == C::NOWN + 32;  // lane 0 of the x-ring warp

    auto core = [&](int slot) { return sphi + slot * C::PHI; };
    auto side = [&](int slot) { return sphi + slot * C::PHI + PR * W; };

    // Normals and sharpening of the VX cells of group gc in local row ly.
    auto sharp_group = [&](int m, int mm, int mp, int gc, int ly, T *s0, T *s1, T *s2) {
        const int r = ly + 2;
        const int off = r * W + gc * VX;
        T c[VX], yn[VX], yp[VX], zn[VX], zp[VX];
        VV::ld(c, core(m) + off);
        VV::ld(yn, core(m) + off - W);
        VV::ld(yp, core(m) + off + W);
        VV::ld(zn, core(mm) + off);
        VV::ld(zp, core(mp) + off);
        const T L = gc > 0 ? core(m)[off - 1] : side(m)[r * 2 * VX + VX - 1];
        const T R = gc < TX - 1 ? core(m)[off + VX] : side(m)[r * 2 * VX + VX];
#pragma unroll
        for (int i = 0; i < VX; ++i) {
            const T g0 = (i + 1 < VX ? c[i + 1] : R) - (i > 0 ? c[i - 1] : L);
            const T g1 = yp[i] - yn[i];
            const T g2 = zp[i] - zn[i];
            const T q = fma(g2, g2, fma(g1, g1, fma(g0, g0, NumLim<T>::tiny())));
            const T inv = rsqrt_t(q);
            const T wgt = c[i] * (T(1) - c[i]) * inv;
            s0[i] = wgt * g0;
            s1[i] = wgt * g1;
            s2[i] = wgt * g2;
        }
    };
    // s_x of the x-ring cell just left (x0 - 1) or right (x0 + W) of row ly.
    auto sharp_cell = [&](int m, int mm, int mp, bool left, int ly) {
        const int r = ly + 2;
        const int si = r * 2 * VX + (left ? VX - 1 : VX);  // the cell in the side array
        const T p = side(m)[si];
        const T xm = left ? side(m)[si - 1] : core(m)[r * W + W - 1];
        const T xp = left ? core(m)[r * W] : side(m)[si + 1];
        const T g0 = xp - xm;
        const T g1 = side(m)[si + 2 * VX] - side(m)[si - 2 * VX];
        const T g2 = side(mp)[si] - side(mm)[si];
        const T q = fma(g2, g2, fma(g1, g1, fma(g0, g0, NumLim<T>::tiny())));
        return p * (T(1) - p) * rsqrt_t(q) * g0;
    };

    if (tid == 0) {
        for (int i = 0; i < 4; ++i) mbar_init(bars + i, 1);
        fence_barrier_init();
    }
    __syncthreads();
    int sc = 0;  // next stage id: barrier sc & 3, parity (sc >> 2) & 1
    // Copy thread: after a bounded wait has run out it issues no further tensor
    // copies, and before the kernel returns it waits (bounded) for every stage
    // it issued beyond the last one it saw complete, so that no copy is still
    // writing into this block's shared memory when the block exits.
    bool timed_out = false;
    int issued_hi = 0, waited_hi = 0;  // stage ids [waited_hi, issued_hi) may be in flight

    Acc<T> acc;
    acc.init();

    UnitIter<W, H> units(ntiles, nz, nchunks);
    Unit un;
    while (units.next(un, ntiles, tiles_x, nz, nchunks)) {
        const int x0 = un.x0, y0 = un.y0, z0 = un.z0, z1 = un.z1;
        const int ym2 = wrapi(y0 - 2, ny), yph = wrapi(y0 + H, ny), ym1 = wrapi(y0 - 1, ny);
        const int xl = wrapi(x0 - VX, nx), xr = wrapi(x0 + W, nx);

        // Halo chunk of this ring thread: ct < 40 a phi side chunk (row ct/2,
        // left/right), 40 <= ct < 56 a u left-halo chunk.
        const int ct = rr;
        int hoff = 0, hdst = 0;
        if (!is_own && ct < 40) {
            const int r = ct >> 1, sd = ct & 1;
            hoff = (int)CDI_CHK(wrapi(y0 - 2 + r, ny) * nx + (sd ? xr : xl), plane - VX + 1, a.red.status);
            hdst = r * 2 * VX + sd * VX;
        } else if (!is_own && ct < 56) {
            const int r = ct - 40;
            hoff = (int)CDI_CHK((y0 + r) * nx + xl, plane - VX + 1, a.red.status);
            hdst = r * VX;
        }
        // Issue one stage: phi planes zp0 .. zp0+np-1 into slots ps0.. (mod 5)
        // and, if zv >= 0, the velocity plane zv into velocity slot vs.
        auto issue_stage = [&](int zp0, int np, int ps0, int zv, int vs) {
            unsigned long long *bar = bars + (sc & 3);
            if (!is_own) fence_proxy_async();
            if (tma_thread && !timed_out) {
                issued_hi = sc + 1;
                for (int d = 0; d < np; ++d) {
                    int s = ps0 + d;
                    if (s >= 5) s -= 5;
                    const int z = wrapi(zp0 + d, nz);
                    tma_3d(core(s), &maps.phi2, x0, ym2, z, bar);
                    tma_3d(core(s) + 2 * W, &maps.phiH, x0, y0, z, bar);
                    tma_3d(core(s) + (H + 2) * W, &maps.phi2, x0, yph, z, bar);
                }
                if (zv >= 0) {
                    T *vb = svel + vs * C::VEL;
                    tma_3d(vb, &maps.u, x0, y0, zv, bar);
                    tma_3d(vb + C::UC + C::UH, &maps.v1, x0, ym1, zv, bar);
                    tma_3d(vb + C::UC + C::UH + W, &maps.vH, x0, y0, zv, bar);
                    tma_3d(vb + C::UC + C::UH + C::VV, &maps.w, x0, y0, zv, bar);
                }
                const unsigned bytes = (unsigned)(sizeof(T) * ((size_t)np * PR * W + (zv >= 0 ? (size_t)(C::UC + C::VV + C::WW) : 0)));
                mbar_arrive_expect_tx(bar, bytes);
            }
            if (!is_own) {
                if (ct < 40) {
                    for (int d = 0; d < np; ++d) {
                        int s = ps0 + d;
                        if (s >= 5) s -= 5;
                        cp_async<16>(side(s) + hdst, a.phi + (long long)wrapi(zp0 + d, nz) * plane + hoff);
                    }
                } else if (ct < 56 && zv >= 0) {
                    cp_async<16>(svel + vs * C::VEL + C::UC + hdst, a.u + (long long)zv * plane + hoff);
                }
                cp_async_commit();
            }
            ++sc;
        };
        // Stage s has landed: the ring threads wait for their halo copies, one
        // thread for the tensor copies; the barrier that follows publishes both.
        auto wait_stage = [&](int id, int pending) {
            if (!is_own) {
                if (pending) cp_async_wait<1>();
                else cp_async_wait<0>();
            }
            if (tma_thread && !timed_out) {
                timed_out = !mbar_wait_bounded(bars + (id & 3), (unsigned)((id >> 2) & 1), a.red.status);
                if (!timed_out && id + 1 > waited_hi) waited_hi = id + 1;
            }
        };

        __syncthreads();  // the previous unit's readers are done with every slot
        const int s0 = sc;
        issue_stage(z0 - 2, 5, 0, z0, 0);

        const int own_x = x0 + tx * VX, own_y = y0 + ty;
        const long long own_off = (long long)own_y * nx + own_x;
        T wlo[VX];
        if (is_own) {
            const T *src = a.w + (long long)wrapi(z0 - 1, nz) * plane + own_off;
#pragma unroll
            for (int i = 0; i < VX; ++i) wlo[i] = __ldg(src + i);
        }
        wait_stage(s0, 0);
        __syncthreads();

        // Prologue: s_z at plane z0-1 (own), s at plane z0 (own + ring), flux at z0-1/2.
        T szc[VX], Fzm[VX];
        if (is_own) {
            T a0[VX], a1[VX], szm[VX], s0v[VX], s1v[VX];
            sharp_group(1, 0, 2, tx, ty, a0, a1, szm);
            sharp_group(2, 1, 3, tx, ty, s0v, s1v, szc);
            VV::st(ssx + (z0 & 1) * C::SXS + ty * SXP + VX + tx * VX, s0v);
            VV::st(ssy + (z0 & 1) * C::SYS + (ty + 1) * W + tx * VX, s1v);
            T pm[VX], pc[VX];
            VV::ld(pm, core(1) + (ty + 2) * W + tx * VX);
            VV::ld(pc, core(2) + (ty + 2) * W + tx * VX);
#pragma unroll
            for (int i = 0; i < VX; ++i)
                Fzm[i] = flux(c_adv * wlo[i], c_dif, c_shp, pm[i], pc[i], szm[i], szc[i]);
        } else if (is_yring) {
            T r0[VX], r1[VX], r2[VX];
            sharp_group(2, 1, 3, ry_col, ry_row, r0, r1, r2);
            VV::st(ssy + (z0 & 1) * C::SYS + (ry_row + 1) * W + ry_col * VX, r1);
        } else if (is_xring) {
            ssx[(z0 & 1) * C::SXS + rx_row * SXP + (rx_left ? VX - 1 : VX + W)] = sharp_cell(2, 1, 3, rx_left, rx_row);
        }
        // Plane z0+3 reuses the slot of plane z0-2, which the prologue just read.
        __syncthreads();
        issue_stage(z0 + 3, z0 + 3 <= z1 + 1 ? 1 : 0, 0, z0 + 1 < z1 ? z0 + 1 : -1, 1);

        int pk = 2, vk = 0;
        for (int k = z0; k < z1; ++k) {
            const int pk1 = pk == 4 ? 0 : pk + 1;
            const int pk2 = pk1 == 4 ? 0 : pk1 + 1;
            const int pkm = pk == 0 ? 4 : pk - 1;
            const int vk2 = vk == 0 ? 2 : vk - 1;
            wait_stage(s0 + (k - z0), 1);
            __syncthreads();  // S1
            issue_stage(k + 4, k + 4 <= z1 + 1 ? 1 : 0, pkm, k + 2 < z1 ? k + 2 : -1, vk2);

            // B: sharpening at plane k+1.
            const int b1 = (k + 1) & 1;
            T szn[VX];
            if (is_own) {
                T s0v[VX], s1v[VX];
                sharp_group(pk1, pk, pk2, tx, ty, s0v, s1v, szn);
                VV::st(ssx + b1 * C::SXS + ty * SXP + VX + tx * VX, s0v);
                VV::st(ssy + b1 * C::SYS + (ty + 1) * W + tx * VX, s1v);
            } else if (is_yring) {
                T r0[VX], r1[VX], r2[VX];
                sharp_group(pk1, pk, pk2, ry_col, ry_row, r0, r1, r2);
                VV::st(ssy + b1 * C::SYS + (ry_row + 1) * W + ry_col * VX, r1);
            } else if (is_xring) {
                ssx[b1 * C::SXS + rx_row * SXP + (rx_left ? VX - 1 : VX + W)] =
                    sharp_cell(pk1, pk, pk2, rx_left, rx_row);
            }
            // C: fluxes and update at plane k (telescoped x/y faces, carried z face).
            if (is_own) {
                const int b = k & 1;
                const int r = ty + 2;
                const int po = r * W + tx * VX;
                const T *P = core(pk);
                T c[VX], yn[VX], yp[VX], zp[VX];
                VV::ld(c, P + po);
                VV::ld(yn, P + po - W);
                VV::ld(yp, P + po + W);
                VV::ld(zp, core(pk1) + po);
                const T L = tx > 0 ? P[po - 1] : side(pk)[r * 2 * VX + VX - 1];
                const T R = tx < TX - 1 ? P[po + VX] : side(pk)[r * 2 * VX + VX];
                const T *sxr = ssx + b * C::SXS + ty * SXP + VX + tx * VX;
                const T *syr = ssy + b * C::SYS + (ty + 1) * W + tx * VX;
                T sxc[VX], syn[VX], syp[VX];
                VV::ld(sxc, sxr);
                VV::ld(syn, syr - W);
                VV::ld(syp, syr + W);
                const T sxL = sxr[-1], sxR = sxr[VX];
                const T *vb = svel + vk * C::VEL;
                const T *ur = vb + ty * W + tx * VX;
                const T *vr = vb + C::UC + C::UH + (ty + 1) * W + tx * VX;
                const T *wr = vb + C::UC + C::UH + C::VV + ty * W + tx * VX;
                T uc[VX], vc[VX], vn[VX], wc[VX];
                VV::ld(uc, ur);
                VV::ld(vc, vr);
                VV::ld(vn, vr - W);
                VV::ld(wc, wr);
                const T uL = tx > 0 ? ur[-1] : vb[C::UC + ty * VX + VX - 1];
                T o[VX];
#pragma unroll
                for (int i = 0; i < VX; ++i) {
                    const T xlv = i > 0 ? c[i - 1] : L, xrv = i + 1 < VX ? c[i + 1] : R;
                    const T ul = i > 0 ? uc[i - 1] : uL;
                    const T sl = i > 0 ? sxc[i - 1] : sxL, sr = i + 1 < VX ? sxc[i + 1] : sxR;
                    T adv = uc[i] * (c[i] + xrv);
                    adv = fma(-ul, xlv + c[i], adv);
                    adv = fma(vc[i], c[i] + yp[i], adv);
                    adv = fma(-vn[i], yn[i] + c[i], adv);
                    const T dif = fma(T(-4), c[i], (xlv + xrv) + (yn[i] + yp[i]));
                    const T shp = (sr - sl) + (syp[i] - syn[i]);
                    const T Fzp = flux(c_adv * wc[i], c_dif, c_shp, c[i], zp[i], szc[i], szn[i]);
                    const T div = fma(c_adv, adv, fma(-c_dif, dif, fma(c_shp, shp, Fzp - Fzm[i])));
                    o[i] = fma(-c_upd, div, c[i]);
                    Fzm[i] = Fzp;
                    szc[i] = szn[i];
                }
                VV::st(a.out + (long long)k * plane + own_off, o);
                acc.template add_group<VX>(o, a.c.tol);
            }
            pk = pk1;
            vk = vk == 2 ? 0 : vk + 1;
        }
        if (!is_own) cp_async_wait<0>();
    }
    if (tma_thread) {
        // Stages issued at the end of the last unit and never waited for (empty
        // stages in a normal run; after a time-out, whatever was in flight).
        for (int id = waited_hi; id < issued_hi; ++id)
            if (!mbar_wait_bounded(bars + (id & 3), (unsigned)((id >> 2) & 1), a.red.status)) break;
    }
    reduce_and_finish(acc, a.red);
}

// ---------------------------------------------------------------------------
// Host side: eligibility, tensor maps, launch.

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static cudaError_t get_encode()
{
    if (g_encode) return cudaSuccess;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return cudaSuccess;
}

template <typename T>
static cudaError_t encode(CUtensorMap *m, const void *ptr, int nx, int ny, int nz, int bw, int bh)
{
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(T), (cuuint64_t)nx * ny * sizeof(T)};
    const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = g_encode(m, sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                          3, const_cast<void *>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

bool tma_eligible(int esize, int nx, int ny, int nz)
{
    const int W = 16 * (16 / esize), H = 16;
    return nz >= 1 && nx >= W && ny >= H && nx % W == 0 && ny % H == 0 && (long long)nx * ny * nz < (1LL << 32);
}

template <typename T>
cudaError_t tma_occupancy(int *resident)
{
    cudaError_t e = cudaFuncSetAttribute(fwd_tma_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)TmaCfg<T>::bytes);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(resident, fwd_tma_kernel<T>, TmaCfg<T>::NT,
                                                         TmaCfg<T>::bytes);
}

template <typename T>
cudaError_t launch_fwd_tma(const FwdArgs<T> &a, int nblocks, int nchunks, cudaStream_t s)
{
    using C = TmaCfg<T>;
    if (cudaError_t e = get_encode()) return e;
    TmaMaps m;
    cudaError_t e;
    if ((e = encode<T>(&m.phi2, a.phi, a.nx, a.ny, a.nz, C::W, 2)) ||
        (e = encode<T>(&m.phiH, a.phi, a.nx, a.ny, a.nz, C::W, C::H)) ||
        (e = encode<T>(&m.u, a.u, a.nx, a.ny, a.nz, C::W, C::H)) ||
        (e = encode<T>(&m.vH, a.v, a.nx, a.ny, a.nz, C::W, C::H)) ||
        (e = encode<T>(&m.v1, a.v, a.nx, a.ny, a.nz, C::W, 1)) ||
        (e = encode<T>(&m.w, a.w, a.nx, a.ny, a.nz, C::W, C::H)))
        return e;
    fwd_tma_kernel<T><<<nblocks, C::NT, C::bytes, s>>>(a, m, nchunks);
    return cudaGetLastError();
}

template cudaError_t tma_occupancy<float>(int *);
template cudaError_t tma_occupancy<double>(int *);
template cudaError_t launch_fwd_tma<float>(const FwdArgs<float> &, int, int, cudaStream_t);
template cudaError_t launch_fwd_tma<double>(const FwdArgs<double> &, int, int, cudaStream_t);

}  // namespace cdi
