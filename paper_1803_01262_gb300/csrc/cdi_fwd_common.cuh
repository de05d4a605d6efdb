// Device helpers shared by the CDI step kernels (forward, batched).
#pragma once

#include "cdi_internal.cuh"

namespace cdi {

__device__ __forceinline__ float rsqrt_t(float q) { return rsqrtf(q); }
__device__ __forceinline__ double rsqrt_t(double q) { return rsqrt(q); }

template <typename T> struct NumLim;
template <> struct NumLim<float> {
    __device__ __forceinline__ static float tiny() { return 1.17549435e-38f; }  // FLT_MIN
};
template <> struct NumLim<double> {
    __device__ __forceinline__ static double tiny() { return 2.2250738585072014e-308; }  // DBL_MIN
};

// Face flux F = cadv_u (pl + pr) - cdif (pr - pl) + cshp (sl + sr).  The order of
// evaluation is fixed by explicit fused multiply-adds rather than left to the
// compiler's choice of which product to fuse, which could differ between the
// kernels that share this expression.
template <typename T>
__device__ __forceinline__ T flux(T cadv_u, T cdif, T cshp, T pl, T pr, T sl, T sr)
{
    return fma(cshp, sl + sr, fma(cadv_u, pl + pr, -(cdif * (pr - pl))));
}

// 16-byte vector of T.
template <typename T> struct V16;
template <> struct V16<float> {
    static constexpr int N = 4;
    __device__ __forceinline__ static void ld(float *d, const float *s)
    {
        const float4 v = *reinterpret_cast<const float4 *>(s);
        d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
    }
    __device__ __forceinline__ static void st(float *d, const float *s)
    {
        *reinterpret_cast<float4 *>(d) = make_float4(s[0], s[1], s[2], s[3]);
    }
};
template <> struct V16<double> {
    static constexpr int N = 2;
    __device__ __forceinline__ static void ld(double *d, const double *s)
    {
        const double2 v = *reinterpret_cast<const double2 *>(s);
        d[0] = v.x; d[1] = v.y;
    }
    __device__ __forceinline__ static void st(double *d, const double *s)
    {
        *reinterpret_cast<double2 *>(d) = make_double2(s[0], s[1]);
    }
};

// Value of the lane one below / above within segments of WIDTH lanes (the
// first / last lane of a segment gets its own value back).
template <int WIDTH, typename T>
__device__ __forceinline__ T shfl_up1(T v) { return __shfl_up_sync(0xffffffffu, v, 1, WIDTH); }
template <int WIDTH, typename T>
__device__ __forceinline__ T shfl_down1(T v) { return __shfl_down_sync(0xffffffffu, v, 1, WIDTH); }

// Work unit u -> (tile origin, z range).
struct Unit {
    int x0, y0, z0, z1;
};
__device__ __forceinline__ Unit unit_of(int u, int ntiles, int tiles_x, int bw, int bh, int zc, int nz)
{
    Unit r;
    const int chunk = u / ntiles, tile = u - chunk * ntiles;
    r.x0 = (tile % tiles_x) * bw;
    r.y0 = (tile / tiles_x) * bh;
    r.z0 = chunk * zc;
    r.z1 = min(nz, r.z0 + zc);
    return r;
}

// The work units of one block of a persistent grid, tiles of BW x BH cells.
//   nchunks >= 1: units u = blockIdx.x, blockIdx.x + gridDim.x, ... of the
//     (z chunk, tile) list in chunk-major order, chunks of ceil(nz / nchunks)
//     planes: blocks resident together work on neighbouring tiles at the same
//     planes.
//   nchunks <= 0 (balanced): block b takes the contiguous share
//     [b T / B, (b + 1) T / B) of the T = ntiles * nz tile-planes in
//     tile-major order (T < 2^31, checked by the host), cut where a tile's
//     column ends: every block gets the same number of planes (+-1) in one or
//     two units (more only when a share exceeds a column).
//   nchunks == -2 (balanced, rotated, prologue-weighted): the shares are cut
//     from a cost line on which each column counts kSharePrologue (in
//     cdi_internal.cuh) planes more than its nz (its first piece's prologue), so a share that crosses
//     into a new column, and pays a second prologue there, gets that many
//     planes fewer; and each tile's column is visited rotated, starting at
//     plane nz - e_t, where e_t is the offset of the first share that begins
//     inside that column: the shares that begin inside any column then begin
//     at the same planes (0, P, 2P, ... to rounding) for every tile, so the
//     blocks on neighbouring tiles march through the same planes at the same
//     time and the halo rows they share meet in L2, as with chunk-major units.
template <int BW, int BH>
struct UnitIter {
    int p;  // next unit, or next tile-plane (the only state: the rest is recomputed
            // from the launch parameters, which keeps it out of the registers)
    __device__ __forceinline__ UnitIter(int ntiles, int nz, int nchunks)
    {
        p = nchunks >= 1 ? (int)blockIdx.x
                         : (int)((long long)ntiles * (nz + (nchunks == -2 ? kSharePrologue : 0)) *
                                 blockIdx.x / gridDim.x);
    }
    __device__ __forceinline__ bool next(Unit &r, int ntiles, int tiles_x, int nz, int nchunks)
    {
        if (nchunks >= 1) {
            const int zc = (nz + nchunks - 1) / nchunks;
            if (p >= ntiles * ((nz + zc - 1) / zc)) return false;
            r = unit_of(p, ntiles, tiles_x, BW, BH, zc, nz);
            p += gridDim.x;
            return true;
        }
        // the cost line: each column is w prologue slots, then its nz planes
        const int w = nchunks == -2 ? kSharePrologue : 0;
        const long long L = (long long)nz + w;
        const long long T = (long long)ntiles * L;
        const long long q = T * (blockIdx.x + 1) / gridDim.x;
        int tile, j, je;
        long long cs;
        for (;;) {
            if (p >= q) return false;
            tile = (int)(p / L);
            cs = (long long)tile * L;
            const long long ce = q < cs + L ? q : cs + L;
            j = (int)(p - cs - w > 0 ? p - cs - w : 0);     // position in the tile's column
            je = (int)(ce - cs - w > 0 ? ce - cs - w : 0);
            p = (int)ce;
            if (je > j) break;                               // else only prologue slots
        }
        // offset e of the first share beginning inside this column
        int e = 0;
        if (nchunks == -2) {
            const long long bs = (cs * gridDim.x + T - 1) / T;
            const long long qs = T * bs / gridDim.x;
            e = qs < cs + L && qs - cs - w > 0 ? (int)(qs - cs - w) : 0;
        }
        r.x0 = (tile % tiles_x) * BW;
        r.y0 = (tile / tiles_x) * BH;
        r.z0 = j >= e ? j - e : nz - e + j;      // the column rotated by e
        r.z1 = r.z0 + (je - j);
        return true;
    }
};

}  // namespace cdi
