// Fused reductions of the CDI step: discrete mass (double sum), min, max and
// two violation counts, reduced per block and finished by the last block to
// arrive (fixed combination order, so results are reproducible run to run).
// The FP32 kernels reduce in FP32 arithmetic (the sum as a float pair), the
// FP64 kernels in double; partials are stored in double either way.
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

// FP32 form of a partial, for the FP32 kernels' block and grid reductions: the
// sum as an unevaluated pair hi + lo of floats (|lo| <= ulp(hi) / 2), min and
// max as floats (exact: they are FP32 values), counts of type C.  Combining two
// such partials costs a handful of FP32 adds (Knuth's two-sum of the high parts,
// then renormalisation), so a block reduction stays off GB300's narrow FP64 pipe;
// the pair keeps about 48 significant bits, against the 53 of a double sum of
// the same partials.
template <typename C>
struct PartialF {
    float hi, lo, mn, mx;
    C ns, nt;
};

template <typename C>
__device__ __forceinline__ PartialF<C> pidentity_f()
{
    PartialF<C> p;
    p.hi = 0.f;
    p.lo = 0.f;
    p.mn = INFINITY;
    p.mx = -INFINITY;
    p.ns = 0;
    p.nt = 0;
    return p;
}

// hi + lo = a + b exactly (two-sum), then the pair (hi, lo) = s + e renormalised;
// a non-finite sum is carried in hi alone.
__device__ __forceinline__ void sum_pair(float a, float b, float e_in, float &hi, float &lo)
{
    const float s = a + b;
    const float bb = s - a;
    const float e = ((a - (s - bb)) + (b - bb)) + e_in;
    const float h = s + e;
    const bool fin = isfinite(s);
    hi = fin ? h : s;
    lo = fin ? e - (h - s) : 0.f;
}

template <typename C>
__device__ __forceinline__ PartialF<C> pcombine_f(PartialF<C> a, const PartialF<C> &b)
{
    sum_pair(a.hi, b.hi, a.lo + b.lo, a.hi, a.lo);
    a.mn = fminf(a.mn, b.mn);
    a.mx = fmaxf(a.mx, b.mx);
    a.ns += b.ns;
    a.nt += b.nt;
    return a;
}

template <typename C>
__device__ __forceinline__ PartialF<C> warp_reduce_f(PartialF<C> p)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        PartialF<C> q;
        q.hi = __shfl_down_sync(0xffffffffu, p.hi, o);
        q.lo = __shfl_down_sync(0xffffffffu, p.lo, o);
        q.mn = __shfl_down_sync(0xffffffffu, p.mn, o);
        q.mx = __shfl_down_sync(0xffffffffu, p.mx, o);
        q.ns = __shfl_down_sync(0xffffffffu, p.ns, o);
        q.nt = __shfl_down_sync(0xffffffffu, p.nt, o);
        p = pcombine_f(p, q);
    }
    return p;
}

template <typename C>
__device__ __forceinline__ Partial to_partial(const PartialF<C> &q)
{
    Partial r;
    r.sum = (double)q.hi + (double)q.lo;
    r.mn = (double)q.mn;
    r.mx = (double)q.mx;
    r.ns = (long long)q.ns;
    r.nt = (long long)q.nt;
    return r;
}

// A stored partial of an FP32 kernel back in FP32 form (exact for min and max,
// which came from floats; the sum to within the pair's precision).
__device__ __forceinline__ PartialF<unsigned long long> from_partial(const Partial &p)
{
    PartialF<unsigned long long> r;
    r.hi = (float)p.sum;
    r.lo = isfinite(r.hi) ? (float)(p.sum - (double)r.hi) : 0.f;
    r.mn = (float)p.mn;
    r.mx = (float)p.mx;
    r.ns = (unsigned long long)p.ns;
    r.nt = (unsigned long long)p.nt;
    return r;
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
    // the first n (1 <= n <= N) of N values (a group cut by the end of a row)
    template <int N>
    __device__ __forceinline__ void add_group_n(const float *o, int n, float tol)
    {
        if (n == N) {
            add_group<N>(o, tol);
            return;
        }
#pragma unroll
        for (int i = 0; i < N; ++i)
            if (i < n) add(o[i], tol);
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
    // the compensated sum s - c as a renormalised pair
    __device__ __forceinline__ PartialF<unsigned> partial_f() const
    {
        PartialF<unsigned> r;
        sum_pair(s, -c, 0.f, r.hi, r.lo);
        r.mn = mn;
        r.mx = mx;
        r.ns = (unsigned)ns;
        r.nt = (unsigned)nt;
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
    template <int N>
    __device__ __forceinline__ void add_group_n(const double *o, int n, double tol)
    {
        if (n == N) {
            add_group<N>(o, tol);
            return;
        }
#pragma unroll
        for (int i = 0; i < N; ++i)
            if (i < n) add(o[i], tol);
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

// The same for the FP32 form; the result, valid in thread 0, is converted to
// the stored (double) form.
template <typename C>
__device__ __forceinline__ Partial block_reduce_f(PartialF<C> p)
{
    __shared__ PartialF<C> wsum_f[32];
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    const int lane = tid & 31, wid = tid >> 5, nw = nthr >> 5;
    p = warp_reduce_f(p);
    if (lane == 0) wsum_f[wid] = p;
    __syncthreads();
    Partial r = pidentity();
    if (wid == 0) {
        PartialF<C> q = lane < nw ? wsum_f[lane] : pidentity_f<C>();
        q = warp_reduce_f(q);
        if (lane == 0) r = to_partial(q);
    }
    __syncthreads();
    return r;
}

// The block's partial of a per-thread accumulator, valid in thread 0: FP32
// kernels reduce in the FP32 form, FP64 kernels in double.
__device__ __forceinline__ Partial block_partial(const Acc<float> &acc) { return block_reduce_f(acc.partial_f()); }
__device__ __forceinline__ Partial block_partial(const Acc<double> &acc) { return block_reduce(acc.partial()); }
__device__ __forceinline__ Partial block_partial(const Partial &p) { return block_reduce(p); }

// Combine the stored partials parts[0, n) with a fixed tree (every thread of
// the block takes part; the result is valid in thread 0): in the FP32 form for
// an FP32 kernel's partials, else in double.
template <bool F32>
__device__ __forceinline__ Partial combine_partials(const Partial *parts, int n)
{
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    if constexpr (F32) {
        PartialF<unsigned long long> a = pidentity_f<unsigned long long>();
        for (int i = tid; i < n; i += nthr) a = pcombine_f(a, from_partial(load_partial_cg(parts + i)));
        return block_reduce_f(a);
    } else {
        Partial a = pidentity();
        for (int i = tid; i < n; i += nthr) a = pcombine(a, load_partial_cg(parts + i));
        return block_reduce(a);
    }
}

template <typename A> struct IsF32 { static constexpr bool value = false; };
template <> struct IsF32<Acc<float>> { static constexpr bool value = true; };

// Combine parts[0, n) (every thread of the block; fixed order) into red.rec:
// the step's fields (added to the record's with COMBINE and red.combine, a
// further z slab of the same step), and with update_run the run accumulators.
template <bool COMBINE, bool F32>
__device__ __forceinline__ void finish_record(const Partial *parts, int n, const RedScratch &red,
                                              int update_run)
{
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    // The record's fields that are read back, fetched before the combination so
    // that their latency overlaps it.  (The grid's completion publishes the
    // record to the next launch; no fence is needed.)
    StatsRec *r = red.rec;
    StatsRec o;
    if (tid == 0) {
        if (COMBINE && red.combine) {
            o.sum = __ldcg(&r->sum);
            o.mn = __ldcg(&r->mn);
            o.mx = __ldcg(&r->mx);
            o.ns = __ldcg(&r->ns);
            o.nt = __ldcg(&r->nt);
        }
        if (update_run) {
            o.mn_run = __ldcg(&r->mn_run);
            o.mx_run = __ldcg(&r->mx_run);
            o.ns_run = __ldcg(&r->ns_run);
            o.nt_run = __ldcg(&r->nt_run);
            o.steps_run = __ldcg(&r->steps_run);
        }
    }
    Partial q = combine_partials<F32>(parts, n);
    if (tid == 0) {
        if (COMBINE && red.combine) {
            q.sum += o.sum;
            q.mn = fmin(o.mn, q.mn);
            q.mx = fmax(o.mx, q.mx);
            q.ns += o.ns;
            q.nt += o.nt;
        }
        r->sum = q.sum;
        r->mn = q.mn;
        r->mx = q.mx;
        r->ns = q.ns;
        r->nt = q.nt;
        r->mass = red.dV * q.sum;
        if (update_run) {
            r->mn_run = fmin(o.mn_run, q.mn);
            r->mx_run = fmax(o.mx_run, q.mx);
            r->ns_run = o.ns_run + q.ns;
            r->nt_run = o.nt_run + q.nt;
            r->steps_run = o.steps_run + 1;
        }
    }
}

// Store the block's partial p (valid in thread 0) and let the last block to
// finish combine all partials in index order into red.rec.  Every thread of
// the block calls this; the block size must be a multiple of 32.
// COMBINE: the launch may be a further z slab of a step (red.combine); only the
// slab kernels are built with it.  With red.prev, block 0 first finishes the
// previous launch's deferred partials (whose grid has completed: every kernel
// reaches this point after its dependency wait); with red.defer the partials
// are only stored, for the next launch to finish.
template <bool COMBINE, bool F32>
__device__ __forceinline__ void finish_partial(const Partial &p, const RedScratch &red)
{
    __shared__ int is_last;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    if (red.prev && bid == 0) finish_record<false, F32>(red.prev, red.prev_nb, red, red.prev_update_run);
    if (red.defer) {
        if (tid == 0) red.partials[bid] = p;
        return;
    }
    if (tid == 0) {
        red.partials[bid] = p;
        __threadfence();  // also orders block 0's record writes above before its arrival
        const unsigned prev = atomicAdd(red.counter, 1u);
        is_last = (prev == (unsigned)(nb - 1));
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    finish_record<COMBINE, F32>(red.partials, nb, red, red.update_run);
    if (tid == 0) *red.counter = 0u;
}

// Block-reduce the accumulator (or an already formed per-thread Partial, in
// double), store the block partial, and let the last block to finish combine
// all partials into red.rec.
template <bool COMBINE = false, typename A>
__device__ __forceinline__ void reduce_and_finish(const A &acc, const RedScratch &red)
{
    finish_partial<COMBINE, IsF32<A>::value>(block_partial(acc), red);
}

// Two steps' partials of one launch (a temporally blocked pass): each is
// block-reduced and stored (step 1 in slots [0, nb), step 2 in [nb, 2 nb)); the
// last block to finish combines both in index order, writes the second step's
// statistics to red.rec and folds both steps into the run accumulators.
template <typename A>
__device__ __forceinline__ void reduce_and_finish2(const A &acc1, const A &acc2, const RedScratch &red)
{
    constexpr bool F32 = IsF32<A>::value;
    __shared__ int is_last2;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    const Partial q1 = block_partial(acc1);
    const Partial q2 = block_partial(acc2);
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
    StatsRec *r = red.rec;
    StatsRec o;
    if (tid == 0 && red.update_run) {  // fetched early, as in finish_partial
        o.mn_run = __ldcg(&r->mn_run);
        o.mx_run = __ldcg(&r->mx_run);
        o.ns_run = __ldcg(&r->ns_run);
        o.nt_run = __ldcg(&r->nt_run);
        o.steps_run = __ldcg(&r->steps_run);
    }
    const Partial a1 = combine_partials<F32>(red.partials, nb);
    const Partial a2 = combine_partials<F32>(red.partials + nb, nb);
    if (tid == 0) {
        r->sum = a2.sum;
        r->mn = a2.mn;
        r->mx = a2.mx;
        r->ns = a2.ns;
        r->nt = a2.nt;
        r->mass = red.dV * a2.sum;
        if (red.update_run) {
            r->mn_run = fmin(o.mn_run, fmin(a1.mn, a2.mn));
            r->mx_run = fmax(o.mx_run, fmax(a1.mx, a2.mx));
            r->ns_run = o.ns_run + a1.ns + a2.ns;
            r->nt_run = o.nt_run + a1.nt + a2.nt;
            r->steps_run = o.steps_run + 2;
        }
        *red.counter = 0u;
    }
}

}  // namespace cdi
