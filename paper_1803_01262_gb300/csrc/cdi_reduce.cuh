// Fused reductions of the CDI step: discrete mass (double sum), min, max and
// two violation counts, reduced per block and finished by the last block to
// arrive (fixed combination order, so results are reproducible run to run).
#pragma once

#include <math.h>
#include "cdi_internal.cuh"

namespace cdi {

__device__ __forceinline__ Partial pidentity()
{
    Partial p;
    p.sum = 0.0;
    p.mn = INFINITY;
    p.mx = -INFINITY;
    p.ns = 0;
    p.nt = 0;
    return p;
}

__device__ __forceinline__ Partial pcombine(Partial a, const Partial &b)
{
    a.sum += b.sum;
    a.mn = fmin(a.mn, b.mn);
    a.mx = fmax(a.mx, b.mx);
    a.ns += b.ns;
    a.nt += b.nt;
    return a;
}

__device__ __forceinline__ Partial warp_reduce(Partial p)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Partial q;
        q.sum = __shfl_down_sync(0xffffffffu, p.sum, o);
        q.mn = __shfl_down_sync(0xffffffffu, p.mn, o);
        q.mx = __shfl_down_sync(0xffffffffu, p.mx, o);
        q.ns = __shfl_down_sync(0xffffffffu, p.ns, o);
        q.nt = __shfl_down_sync(0xffffffffu, p.nt, o);
        p = pcombine(p, q);
    }
    return p;
}

// Per-thread accumulator.  FP32 keeps a compensated (Kahan) float sum so the
// per-thread partial is accurate before it is promoted to double; FP64 sums
// directly.  min/max are exact; NaN is ignored by min/max and not counted
// (FP64: min, max and range tests on order keys, below).
template <typename T>
struct Acc;

template <>
struct Acc<float> {
    float s, c, mn, mx;
    int ns, nt;
    __device__ __forceinline__ void init()
    {
        s = 0.f; c = 0.f; mn = INFINITY; mx = -INFINITY; ns = 0; nt = 0;
    }
    __device__ __forceinline__ void add(float p, float tol)
    {
        float y = p - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
        mn = fminf(mn, p);
        mx = fmaxf(mx, p);
        // A tolerant violation is also a strict one; both are rare, so one test
        // guards the counting (NaN fails every comparison and is not counted).
        if (p < 0.f || p > 1.f) {
            ++ns;
            nt += (p < -tol) | (p > 1.f + tol);
        }
    }
    // N values at once: their pairwise sum is added with compensation (the
    // uncompensated pairwise rounding is random and of relative size ~1e-9 on
    // a whole field), min/max of the group, and the exact violation counts only
    // when the group leaves [0, 1].
    template <int N>
    __device__ __forceinline__ void add_group(const float *o, float tol)
    {
        float gmn = o[0], gmx = o[0];
        float g = o[0];
#pragma unroll
        for (int i = 1; i < N; ++i) {
            g += o[i];
            gmn = fminf(gmn, o[i]);
            gmx = fmaxf(gmx, o[i]);
        }
        {
            const float y = g - c;
            const float t = s + y;
            c = (t - s) - y;
            s = t;
        }
        mn = fminf(mn, gmn);
        mx = fmaxf(mx, gmx);
        if (gmn < 0.f || gmx > 1.f) {
#pragma unroll
            for (int i = 0; i < N; ++i) {
                ns += (o[i] < 0.f) | (o[i] > 1.f);
                nt += (o[i] < -tol) | (o[i] > 1.f + tol);
            }
        }
    }
    __device__ __forceinline__ Partial partial() const
    {
        Partial r;
        r.sum = (double)s - (double)c;
        r.mn = (double)mn;
        r.mx = (double)mx;
        r.ns = ns;
        r.nt = nt;
        return r;
    }
};

// Order-preserving 64-bit integer key of a double: for numbers a < b exactly
// when okey(a) < okey(b) (the magnitude bits of negatives are flipped; -0
// sorts just below +0); NaNs fall outside [okey(-inf), okey(+inf)].  The FP64
// accumulator takes its min, max and range tests on these keys, on the
// integer pipes, leaving GB300's narrow FP64 pipe to the step itself.
__device__ __forceinline__ long long okey(double x)
{
    const long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double from_okey(long long k)
{
    return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}
constexpr long long KEY_PINF = 0x7ff0000000000000LL;              // okey(+inf)
constexpr long long KEY_NINF = (long long)0x800fffffffffffffULL;  // okey(-inf)
constexpr long long KEY_NZERO = -1;                                // okey(-0.0)
constexpr long long KEY_ONE = 0x3ff0000000000000LL;               // okey(1.0)

template <>
struct Acc<double> {
    double s;
    long long kmn, kmx;  // keys of the min and max so far
    int ns, nt;
    __device__ __forceinline__ void init()
    {
        s = 0.0; kmn = KEY_PINF; kmx = KEY_NINF; ns = 0; nt = 0;
    }
    // p < 0 (strictly: -0 is not below 0), p > 1, p < -tol, p > 1 + tol, for a number p
    __device__ __forceinline__ static bool num(long long k) { return k >= KEY_NINF && k <= KEY_PINF; }
    __device__ __forceinline__ void count(long long k, double tol)
    {
        ns += num(k) & ((k < KEY_NZERO) | (k > KEY_ONE));
        nt += num(k) & ((k < okey(-tol)) | (k > okey(1.0 + tol)));
    }
    __device__ __forceinline__ void add(double p, double tol)
    {
        s += p;
        const long long k = okey(p);
        if (num(k)) {
            kmn = min(kmn, k);
            kmx = max(kmx, k);
            if ((k < KEY_NZERO) | (k > KEY_ONE)) count(k, tol);
        }
    }
    template <int N>
    __device__ __forceinline__ void add_group(const double *o, double tol)
    {
        long long k[N], gmn = KEY_PINF, gmx = KEY_NINF;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            s += o[i];
            k[i] = okey(o[i]);
            if (num(k[i])) {
                gmn = min(gmn, k[i]);
                gmx = max(gmx, k[i]);
            }
        }
        kmn = min(kmn, gmn);
        kmx = max(kmx, gmx);
        if ((gmn < KEY_NZERO) | (gmx > KEY_ONE)) {
#pragma unroll
            for (int i = 0; i < N; ++i) count(k[i], tol);
        }
    }
    __device__ __forceinline__ Partial partial() const
    {
        Partial r;
        r.sum = s;
        r.mn = from_okey(kmn);
        r.mx = from_okey(kmx);
        r.ns = ns;
        r.nt = nt;
        return r;
    }
};

__device__ __forceinline__ Partial load_partial_cg(const Partial *p)
{
    Partial r;
    r.sum = __ldcg(&p->sum);
    r.mn = __ldcg(&p->mn);
    r.mx = __ldcg(&p->mx);
    r.ns = __ldcg(&p->ns);
    r.nt = __ldcg(&p->nt);
    return r;
}

// Block-reduce p (every thread of the block must call this, block size a
// multiple of 32); the result is valid in thread 0.  Ends with a barrier so
// the shared buffer may be reused at once.
__device__ __forceinline__ Partial block_reduce(Partial p)
{
    __shared__ Partial wsum_b[32];
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    const int lane = tid & 31, wid = tid >> 5, nw = nthr >> 5;
    p = warp_reduce(p);
    if (lane == 0) wsum_b[wid] = p;
    __syncthreads();
    Partial q = pidentity();
    if (wid == 0) {
        q = lane < nw ? wsum_b[lane] : pidentity();
        q = warp_reduce(q);
    }
    __syncthreads();
    return q;
}

// Block-reduce p (every thread of the block must call this), store the block
// partial, and let the last block to finish combine all partials in index
// order into red.rec.  The block size must be a multiple of 32.
// COMBINE: the launch may be a further z slab of a step (red.combine); only the
// slab kernels are built with it.
template <bool COMBINE = false>
__device__ __forceinline__ void reduce_and_finish(Partial p, const RedScratch &red)
{
    __shared__ Partial wsum[32];
    __shared__ int is_last;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    const int lane = tid & 31, wid = tid >> 5, nw = nthr >> 5;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int nb = gridDim.x * gridDim.y * gridDim.z;

    p = warp_reduce(p);
    if (lane == 0) wsum[wid] = p;
    __syncthreads();
    if (wid == 0) {
        Partial q = lane < nw ? wsum[lane] : pidentity();
        q = warp_reduce(q);
        if (lane == 0) {
            red.partials[bid] = q;
            __threadfence();
            unsigned prev = atomicAdd(red.counter, 1u);
            is_last = (prev == (unsigned)(nb - 1));
        }
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    Partial acc = pidentity();
    for (int i = tid; i < nb; i += nthr) acc = pcombine(acc, load_partial_cg(red.partials + i));
    acc = warp_reduce(acc);
    __syncthreads();
    if (lane == 0) wsum[wid] = acc;
    __syncthreads();
    if (wid == 0) {
        Partial q = lane < nw ? wsum[lane] : pidentity();
        q = warp_reduce(q);
        if (lane == 0) {
            StatsRec *r = red.rec;
            if (COMBINE && red.combine) {  // a further z slab of the same step
                r->sum += q.sum;
                r->mn = fmin(r->mn, q.mn);
                r->mx = fmax(r->mx, q.mx);
                r->ns += q.ns;
                r->nt += q.nt;
            } else {
                r->sum = q.sum;
                r->mn = q.mn;
                r->mx = q.mx;
                r->ns = q.ns;
                r->nt = q.nt;
            }
            r->mass = red.dV * r->sum;
            if (red.update_run) {
                r->mn_run = fmin(r->mn_run, r->mn);
                r->mx_run = fmax(r->mx_run, r->mx);
                r->ns_run += r->ns;
                r->nt_run += r->nt;
                r->steps_run += 1;
            }
            __threadfence();
            *red.counter = 0u;
        }
    }
}

// Two steps' partials of one launch (a temporally blocked pass): each is
// block-reduced and stored (step 1 in slots [0, nb), step 2 in [nb, 2 nb)); the
// last block to finish combines both in index order, writes the second step's
// statistics to red.rec and folds both steps into the run accumulators.
__device__ __forceinline__ void reduce_and_finish2(Partial p1, Partial p2, const RedScratch &red)
{
    __shared__ int is_last2;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    const Partial q1 = block_reduce(p1);
    const Partial q2 = block_reduce(p2);
    if (tid == 0) {
        red.partials[bid] = q1;
        red.partials[nb + bid] = q2;
        __threadfence();
        const unsigned prev = atomicAdd(red.counter, 1u);
        is_last2 = (prev == (unsigned)(nb - 1));
    }
    __syncthreads();
    if (!is_last2) return;
    __threadfence();
    Partial a1 = pidentity(), a2 = pidentity();
    for (int i = tid; i < nb; i += nthr) {
        a1 = pcombine(a1, load_partial_cg(red.partials + i));
        a2 = pcombine(a2, load_partial_cg(red.partials + nb + i));
    }
    a1 = block_reduce(a1);
    a2 = block_reduce(a2);
    if (tid == 0) {
        StatsRec *r = red.rec;
        r->sum = a2.sum;
        r->mn = a2.mn;
        r->mx = a2.mx;
        r->ns = a2.ns;
        r->nt = a2.nt;
        r->mass = red.dV * a2.sum;
        if (red.update_run) {
            r->mn_run = fmin(r->mn_run, fmin(a1.mn, a2.mn));
            r->mx_run = fmax(r->mx_run, fmax(a1.mx, a2.mx));
            r->ns_run += a1.ns + a2.ns;
            r->nt_run += a1.nt + a2.nt;
            r->steps_run += 2;
        }
        __threadfence();
        *red.counter = 0u;
    }
}

}  // namespace cdi
