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

template <typename T>
__device__ __forceinline__ T flux(T cadv_u, T cdif, T cshp, T pl, T pr, T sl, T sr)
{
    return cadv_u * (pl + pr) - cdif * (pr - pl) + cshp * (sl + sr);
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

}  // namespace cdi
