// Fused explicit CDI step (Eq. 1 discretised as in Section 2.2; Eq. 11 in 1D,
// Eq. 18-22 in coefficient form) for sm_103a, plus the stand-alone
// reductions.  No tensor cores: the step is a memory-bound stencil.
//
// Kernel structure (one block = a BX x BY column of cells marching along z):
//   * phi planes are staged with a halo of 2 in x and y into a 4-slot
//     shared-memory ring (planes k-1 .. k+2 while plane k is updated), so
//     every phi value is read from global memory about once per block;
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

namespace cdi {

__device__ __forceinline__ float rsqrt_t(float q) { return rsqrtf(q); }
__device__ __forceinline__ double rsqrt_t(double q) { return rsqrt(q); }

template <typename T, int BX, int BY>
__global__ void __launch_bounds__(BX * BY)
fwd_kernel(const FwdArgs<T> a)
{
    constexpr int PX = BX + 4, PY = BY + 4, PLANE = PX * PY;
    constexpr int NT = BX * BY;
    constexpr int NLOAD = (PLANE + NT - 1) / NT;
    __shared__ T sp[4][PY][PX];       // phi planes, halo 2
    __shared__ T sx[2][BY][BX + 2];   // s_x on cells x = -1 .. BX
    __shared__ T sy[2][BY + 2][BX];   // s_y on cells y = -1 .. BY

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    const long long plane = (long long)nx * ny;
    const int z0 = blockIdx.z * a.zchunk;
    const int z1 = min(z0 + a.zchunk, nz);

    // In-plane offsets of this thread's halo-load slots (constant along z).
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

    auto load_plane = [&](int z) {
        const T *src = a.phi + (long long)wrapi(z, nz) * plane;
        T *dst = &sp[z & 3][0][0];
#pragma unroll
        for (int r = 0; r < NLOAD; ++r) {
            const int e = tid + r * NT;
            if (e < PLANE) dst[e] = __ldg(src + loff[r]);
        }
    };
    // Sharpening vector s = phi (1 - phi) g/|g| at local cell (lx, ly) of plane z.
    auto sharp = [&](int z, int lx, int ly, T &s0, T &s1, T &s2) {
        const int X = lx + 2, Y = ly + 2;
        const int m = z & 3, mm = (z - 1) & 3, mp = (z + 1) & 3;
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

    // Prologue: planes z0-2 .. z0+1, s at z0 (and s_z at z0-1), flux at z0-1/2.
    load_plane(z0 - 2);
    load_plane(z0 - 1);
    load_plane(z0);
    load_plane(z0 + 1);
    __syncthreads();
    T szm, szc;
    {
        T d0, d1;
        sharp(z0 - 1, tx, ty, d0, d1, szm);
    }
    sharp_plane(z0, szc);
    const T wlo = __ldg(a.w + (long long)wrapi(z0 - 1, nz) * plane + oc);
    T Fzm;
    {
        const T pm = sp[(z0 - 1) & 3][ty + 2][tx + 2], pc = sp[z0 & 3][ty + 2][tx + 2];
        Fzm = c_adv * wlo * (pm + pc) - c_dif * (pc - pm) + c_shp * (szm + szc);
    }
    __syncthreads();

    for (int k = z0; k < z1; ++k) {
        // A: stage plane k+2; fetch this plane's face velocities.
        load_plane(k + 2);
        const long long zb = (long long)k * plane;
        const T uc = __ldg(a.u + zb + oc), um = __ldg(a.u + zb + oxm);
        const T vc = __ldg(a.v + zb + oc), vm = __ldg(a.v + zb + oym);
        const T wc = __ldg(a.w + zb + oc);
        __syncthreads();
        // B: sharpening at plane k+1.
        T szn;
        sharp_plane(k + 1, szn);
        __syncthreads();
        // C: fluxes and update at plane k.
        const int m = k & 3, b = k & 1;
        const T pc = sp[m][ty + 2][tx + 2];
        const T pxm = sp[m][ty + 2][tx + 1], pxp = sp[m][ty + 2][tx + 3];
        const T pym = sp[m][ty + 1][tx + 2], pyp = sp[m][ty + 3][tx + 2];
        const T pzp = sp[(k + 1) & 3][ty + 2][tx + 2];
        const T sxc = sx[b][ty][tx + 1], sxm = sx[b][ty][tx], sxp = sx[b][ty][tx + 2];
        const T syc = sy[b][ty + 1][tx], sym = sy[b][ty][tx], syp = sy[b][ty + 2][tx];
        const T Fxp = c_adv * uc * (pc + pxp) - c_dif * (pxp - pc) + c_shp * (sxc + sxp);
        const T Fxm = c_adv * um * (pxm + pc) - c_dif * (pc - pxm) + c_shp * (sxm + sxc);
        const T Fyp = c_adv * vc * (pc + pyp) - c_dif * (pyp - pc) + c_shp * (syc + syp);
        const T Fym = c_adv * vm * (pym + pc) - c_dif * (pc - pym) + c_shp * (sym + syc);
        const T Fzp = c_adv * wc * (pc + pzp) - c_dif * (pzp - pc) + c_shp * (szc + szn);
        const T o = pc - c_upd * ((Fxp - Fxm) + (Fyp - Fym) + (Fzp - Fzm));
        if (own) {
            a.out[zb + oc] = o;
            acc.add(o, a.c.tol);
        }
        Fzm = Fzp;
        szc = szn;
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

int fwd_blocks(int tile, int zchunk, int nx, int ny, int nz)
{
    const TileDim t = kTiles[tile];
    return ((nx + t.bx - 1) / t.bx) * ((ny + t.by - 1) / t.by) * ((nz + zchunk - 1) / zchunk);
}

template <typename T, int BX, int BY>
static cudaError_t launch_fwd_t(const FwdArgs<T> &a, cudaStream_t s)
{
    dim3 grid((a.nx + BX - 1) / BX, (a.ny + BY - 1) / BY, (a.nz + a.zchunk - 1) / a.zchunk);
    dim3 block(BX, BY);
    fwd_kernel<T, BX, BY><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fwd(const FwdArgs<T> &a, int tile, cudaStream_t s)
{
    switch (tile) {
    case 0: return launch_fwd_t<T, 32, 8>(a, s);
    case 1: return launch_fwd_t<T, 32, 16>(a, s);
    case 2: return launch_fwd_t<T, 64, 8>(a, s);
    case 3: return launch_fwd_t<T, 32, 4>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_fwd<float>(const FwdArgs<float> &, int, cudaStream_t);
template cudaError_t launch_fwd<double>(const FwdArgs<double> &, int, cudaStream_t);

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
