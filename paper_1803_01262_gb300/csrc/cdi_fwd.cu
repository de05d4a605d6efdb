// Fused explicit CDI step (Eq. 1 discretised as in Section 2.2; Eq. 11 in 1D,
// Eq. 18-22 in coefficient form) for sm_103a, plus the stand-alone
// reductions.  No tensor cores: the step is a memory-bound stencil.
//
// Kernel structure (one block = a BX x BY column of cells marching along z):
//   * phi planes are staged with a halo of 2 in x and y by cp.async into an
//     8-slot shared-memory ring, PF_DIST planes ahead of use, so every phi
//     value is read from global memory about once per block and the loads
//     overlap the arithmetic; face velocities are prefetched into registers
//     one plane ahead;
//   * blocks split the (tile, plane) index space into equal contiguous
//     ranges (one launch = one wave of resident blocks, balanced to a plane);
//   * at plane k+1 the block computes the cell-centre normals
//     n = g/|g| (g = central differences, n = 0 where g = 0) and the
//     sharpening vector s = phi (1 - phi) n for its cells and for a one-cell
//     ring (the x-ring only needs s_x, the y-ring only s_y); s_x and s_y go to
//     a 2-slot shared buffer, s_z stays in a register;
//   * at plane k every thread evaluates the six face fluxes of its cell,
//       F = c_adv u_f (phi_L + phi_R) - c_dif (phi_R - phi_L) + c_shp (s_L + s_R),
//     (the z face below is carried in a register from the previous plane),
//     writes phi' = phi - c_upd sum_d (F_+ - F_-) and folds phi' into the
//     per-thread mass / min / max / violation accumulators;
//   * the block partials are finished by the last block (cdi_reduce.cuh).
// All indices wrap periodically; tiles may overhang the grid (ragged edges),
// overhanging threads compute on wrapped data but never write.
#include "cdi_internal.cuh"
#include "cdi_reduce.cuh"
#include "cdi_async.cuh"

namespace cdi {

__device__ __forceinline__ float rsqrt_t(float q) { return rsqrtf(q); }
__device__ __forceinline__ double rsqrt_t(double q) { return rsqrt(q); }

// Pipeline depth: phi plane k+2+PF_DIST is in flight while plane k is updated.
constexpr int PF_DIST = 2;
constexpr int NSLOT = 8;  // power of two >= PF_DIST + 3 live planes

template <typename T, int BX, int BY>
struct FwdSmem {
    static constexpr int PX = BX + 4, PY = BY + 4;
    static constexpr size_t bytes =
        sizeof(T) * (NSLOT * PY * PX + 2 * BY * (BX + 2) + 2 * (BY + 2) * BX);
};

template <typename T, int BX, int BY>
__global__ void __launch_bounds__(BX * BY)
fwd_kernel(const FwdArgs<T> a)
{
    constexpr int PX = BX + 4, PY = BY + 4, PLANE = PX * PY;
    constexpr int NT = BX * BY;
    constexpr int NLOAD = (PLANE + NT - 1) / NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T(*sp)[PY][PX] = reinterpret_cast<T(*)[PY][PX]>(smem_raw);           // phi ring [NSLOT]
    T(*sx)[BY][BX + 2] = reinterpret_cast<T(*)[BY][BX + 2]>(sp + NSLOT);  // s_x, x = -1..BX [2]
    T(*sy)[BY + 2][BX] = reinterpret_cast<T(*)[BY + 2][BX]>(sx + 2);      // s_y, y = -1..BY [2]

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long plane = (long long)nx * ny;
    const int tiles_x = (nx + BX - 1) / BX;

    // Ring cells: threads [0, 2BX) the y-ring, [2BX, 2BX + 2BY) the x-ring.
    int rkind = 0, rx = 0, ry = 0;
    if (tid < 2 * BX) {
        rkind = 1;
        rx = tid % BX;
        ry = tid < BX ? -1 : BY;
    } else if (tid < 2 * BX + 2 * BY) {
        rkind = 2;
        const int r = tid - 2 * BX;
        ry = r % BY;
        rx = r < BY ? -1 : BX;
    }
    const T c_adv = a.c.c_adv, c_dif = a.c.c_dif, c_shp = a.c.c_shp, c_upd = a.c.c_upd;

    // Sharpening vector s = phi (1 - phi) g/|g| at local cell (lx, ly) of plane z.
    auto sharp = [&](int z, int lx, int ly, T &s0, T &s1, T &s2) {
        const int X = lx + 2, Y = ly + 2;
        const int m = z & (NSLOT - 1), mm = (z - 1) & (NSLOT - 1), mp = (z + 1) & (NSLOT - 1);
        const T p = sp[m][Y][X];
        const T g0 = sp[m][Y][X + 1] - sp[m][Y][X - 1];
        const T g1 = sp[m][Y + 1][X] - sp[m][Y - 1][X];
        const T g2 = sp[mp][Y][X] - sp[mm][Y][X];
        const T q = g0 * g0 + g1 * g1 + g2 * g2;
        const T inv = q > T(0) ? rsqrt_t(q) : T(0);
        const T wgt = p * (T(1) - p) * inv;
        s0 = wgt * g0;
        s1 = wgt * g1;
        s2 = wgt * g2;
    };
    auto sharp_plane = [&](int z, T &szc) {
        T q0, q1;
        sharp(z, tx, ty, q0, q1, szc);
        sx[z & 1][ty][tx + 1] = q0;
        sy[z & 1][ty + 1][tx] = q1;
        if (rkind) {
            T r0, r1, r2;
            sharp(z, rx, ry, r0, r1, r2);
            if (rkind == 1) sy[z & 1][ry + 1][rx] = r1;
            else sx[z & 1][ry][rx + 1] = r0;
        }
    };

    Acc<T> acc;
    acc.init();

    // Balanced work split: the (tile, plane) index space, plane fastest, is cut
    // into equal contiguous ranges, one per block; a range may cover the end of
    // one tile column and the start of the next (each piece is a "segment").
    const long long total = (long long)tiles_x * ((ny + BY - 1) / BY) * nz;
    const long long per = (total + gridDim.x - 1) / gridDim.x;
    long long s = (long long)blockIdx.x * per;
    const long long s_end = min(total, s + per);

    while (s < s_end) {
        const int tile = (int)(s / nz);
        const int z0 = (int)(s - (long long)tile * nz);
        const int z1 = (int)min((long long)nz, z0 + (s_end - s));
        s += z1 - z0;
        const int x0 = (tile % tiles_x) * BX, y0 = (tile / tiles_x) * BY;

        int loff[NLOAD];
#pragma unroll
        for (int r = 0; r < NLOAD; ++r) {
            const int e = tid + r * NT;
            const int ey = e / PX, ex = e - ey * PX;
            loff[r] = (e < PLANE) ? wrapi(y0 + ey - 2, ny) * nx + wrapi(x0 + ex - 2, nx) : 0;
        }
        const int gx = wrapi(x0 + tx, nx), gy = wrapi(y0 + ty, ny);
        const bool own = (x0 + tx < nx) && (y0 + ty < ny);
        const int oc = gy * nx + gx;
        const int oxm = gy * nx + wrapi(gx - 1, nx);
        const int oym = wrapi(gy - 1, ny) * nx + gx;

        auto issue_plane = [&](int z) {
            const T *src = a.phi + (long long)wrapi(z, nz) * plane;
            T *dst = &sp[z & (NSLOT - 1)][0][0];
#pragma unroll
            for (int r = 0; r < NLOAD; ++r) {
                const int e = tid + r * NT;
                if (e < PLANE) cp_async<sizeof(T)>(dst + e, src + loff[r]);
            }
        };

        // Prologue: planes z0-2 .. z0+1 (one group), then PF_DIST more groups.
        __syncthreads();  // previous segment's readers are done with the ring
        issue_plane(z0 - 2);
        issue_plane(z0 - 1);
        issue_plane(z0);
        issue_plane(z0 + 1);
        cp_async_commit();
#pragma unroll
        for (int d = 0; d < PF_DIST; ++d) {
            if (z0 + 2 + d <= z1 + 1) issue_plane(z0 + 2 + d);
            cp_async_commit();
        }
        T uc, um, vc, vm, wc;
        {
            const long long zb = (long long)z0 * plane;
            uc = __ldg(a.u + zb + oc); um = __ldg(a.u + zb + oxm);
            vc = __ldg(a.v + zb + oc); vm = __ldg(a.v + zb + oym);
            wc = __ldg(a.w + zb + oc);
        }
        const T wlo = __ldg(a.w + (long long)wrapi(z0 - 1, nz) * plane + oc);
        cp_async_wait<PF_DIST>();
        __syncthreads();
        T szm, szc;
        {
            T d0, d1;
            sharp(z0 - 1, tx, ty, d0, d1, szm);
        }
        sharp_plane(z0, szc);
        T Fzm;
        {
            const T pm = sp[(z0 - 1) & (NSLOT - 1)][ty + 2][tx + 2];
            const T pc = sp[z0 & (NSLOT - 1)][ty + 2][tx + 2];
            Fzm = c_adv * wlo * (pm + pc) - c_dif * (pc - pm) + c_shp * (szm + szc);
        }

        for (int k = z0; k < z1; ++k) {
            // S1: plane k+2 has landed (and every thread left iteration k-1).
            cp_async_wait<PF_DIST - 1>();
            __syncthreads();
            if (k + 2 + PF_DIST <= z1 + 1) issue_plane(k + 2 + PF_DIST);
            cp_async_commit();
            // Next plane's face velocities, consumed one iteration later.
            T un = T(0), umn = T(0), vn = T(0), vmn = T(0), wn = T(0);
            if (k + 1 < z1) {
                const long long zb = (long long)(k + 1) * plane;
                un = __ldg(a.u + zb + oc); umn = __ldg(a.u + zb + oxm);
                vn = __ldg(a.v + zb + oc); vmn = __ldg(a.v + zb + oym);
                wn = __ldg(a.w + zb + oc);
            }
            // B: sharpening at plane k+1.
            T szn;
            sharp_plane(k + 1, szn);
            __syncthreads();
            // C: fluxes and update at plane k.
            const int m = k & (NSLOT - 1), b = k & 1;
            const T pc = sp[m][ty + 2][tx + 2];
            const T pxm = sp[m][ty + 2][tx + 1], pxp = sp[m][ty + 2][tx + 3];
            const T pym = sp[m][ty + 1][tx + 2], pyp = sp[m][ty + 3][tx + 2];
            const T pzp = sp[(k + 1) & (NSLOT - 1)][ty + 2][tx + 2];
            const T sxc = sx[b][ty][tx + 1], sxm = sx[b][ty][tx], sxp = sx[b][ty][tx + 2];
            const T syc = sy[b][ty + 1][tx], sym = sy[b][ty][tx], syp = sy[b][ty + 2][tx];
            const T Fxp = c_adv * uc * (pc + pxp) - c_dif * (pxp - pc) + c_shp * (sxc + sxp);
            const T Fxm = c_adv * um * (pxm + pc) - c_dif * (pc - pxm) + c_shp * (sxm + sxc);
            const T Fyp = c_adv * vc * (pc + pyp) - c_dif * (pyp - pc) + c_shp * (syc + syp);
            const T Fym = c_adv * vm * (pym + pc) - c_dif * (pc - pym) + c_shp * (sym + syc);
            const T Fzp = c_adv * wc * (pc + pzp) - c_dif * (pzp - pc) + c_shp * (szc + szn);
            const T o = pc - c_upd * ((Fxp - Fxm) + (Fyp - Fym) + (Fzp - Fzm));
            if (own) {
                a.out[(long long)k * plane + oc] = o;
                acc.add(o, a.c.tol);
            }
            Fzm = Fzp;
            szc = szn;
            uc = un; um = umn; vc = vn; vm = vmn; wc = wn;
        }
        cp_async_wait<0>();
    }
    reduce_and_finish(acc.partial(), a.red);
}

// ---------------------------------------------------------------------------
// Tile table and launch

struct TileDim { int bx, by; };
static const TileDim kTiles[] = {{32, 8}, {32, 16}, {64, 8}, {32, 4}};
static const int kNumTiles = sizeof(kTiles) / sizeof(kTiles[0]);

int fwd_num_tiles() { return kNumTiles; }

void fwd_tile_dims(int tile, int *bx, int *by)
{
    *bx = kTiles[tile].bx;
    *by = kTiles[tile].by;
}

// Work units (tile-planes) of a grid for a tile shape.
long long fwd_units(int tile, int nx, int ny, int nz)
{
    const TileDim t = kTiles[tile];
    return (long long)((nx + t.bx - 1) / t.bx) * ((ny + t.by - 1) / t.by) * nz;
}

template <typename T, int BX, int BY>
static cudaError_t fwd_prepare(int *resident)
{
    const size_t smem = FwdSmem<T, BX, BY>::bytes;
    cudaError_t e = cudaFuncSetAttribute(fwd_kernel<T, BX, BY>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(resident, fwd_kernel<T, BX, BY>, BX * BY, smem);
}

template <typename T>
cudaError_t fwd_occupancy(int tile, int *resident)
{
    switch (tile) {
    case 0: return fwd_prepare<T, 32, 8>(resident);
    case 1: return fwd_prepare<T, 32, 16>(resident);
    case 2: return fwd_prepare<T, 64, 8>(resident);
    case 3: return fwd_prepare<T, 32, 4>(resident);
    default: return cudaErrorInvalidValue;
    }
}
template cudaError_t fwd_occupancy<float>(int, int *);
template cudaError_t fwd_occupancy<double>(int, int *);

template <typename T, int BX, int BY>
static cudaError_t launch_fwd_t(const FwdArgs<T> &a, int nblocks, cudaStream_t s)
{
    fwd_kernel<T, BX, BY><<<nblocks, dim3(BX, BY), FwdSmem<T, BX, BY>::bytes, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fwd(const FwdArgs<T> &a, int tile, int nblocks, cudaStream_t s)
{
    switch (tile) {
    case 0: return launch_fwd_t<T, 32, 8>(a, nblocks, s);
    case 1: return launch_fwd_t<T, 32, 16>(a, nblocks, s);
    case 2: return launch_fwd_t<T, 64, 8>(a, nblocks, s);
    case 3: return launch_fwd_t<T, 32, 4>(a, nblocks, s);
    default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_fwd<float>(const FwdArgs<float> &, int, int, cudaStream_t);
template cudaError_t launch_fwd<double>(const FwdArgs<double> &, int, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Stand-alone reductions: statistics of any field, and max |component| of
// the face velocities (U of Eq. 24).

template <typename T>
__global__ void __launch_bounds__(256) stats_kernel(const T *__restrict__ phi, long long n, T tol,
                                                    RedScratch red)
{
    Acc<T> acc;
    acc.init();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride)
        acc.add(phi[i], tol);
    reduce_and_finish(acc.partial(), red);
}

template <typename T>
__global__ void __launch_bounds__(256) absmax_kernel(const T *__restrict__ u, const T *__restrict__ v,
                                                     const T *__restrict__ w, long long n,
                                                     RedScratch red)
{
    Partial p = pidentity();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        double m = fabs((double)u[i]);
        if (v) m = fmax(m, fabs((double)v[i]));
        if (w) m = fmax(m, fabs((double)w[i]));
        p.mx = fmax(p.mx, m);
    }
    reduce_and_finish(p, red);
}

template <typename T>
cudaError_t launch_stats(const T *phi, long long n, T tol, RedScratch red, int nblocks,
                         cudaStream_t s)
{
    stats_kernel<T><<<nblocks, 256, 0, s>>>(phi, n, tol, red);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_absmax(const T *u, const T *v, const T *w, long long n, RedScratch red,
                          int nblocks, cudaStream_t s)
{
    absmax_kernel<T><<<nblocks, 256, 0, s>>>(u, v, w, n, red);
    return cudaGetLastError();
}

template cudaError_t launch_stats<float>(const float *, long long, float, RedScratch, int, cudaStream_t);
template cudaError_t launch_stats<double>(const double *, long long, double, RedScratch, int, cudaStream_t);
template cudaError_t launch_absmax<float>(const float *, const float *, const float *, long long,
                                          RedScratch, int, cudaStream_t);
template cudaError_t launch_absmax<double>(const double *, const double *, const double *, long long,
                                           RedScratch, int, cudaStream_t);

}  // namespace cdi
