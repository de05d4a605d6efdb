// C ABI of the CDI library (declared in include/cdi.h): argument checking,
// scratch ownership, launch-configuration choice and the native launch loop.
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "cdi.h"
#include "cdi_internal.cuh"
#include "cdi_async.cuh"
#include "cdi_nvtx.h"

using cdi::LaunchCfg;
using cdi::RedScratch;
using cdi::StatsRec;

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(CDI_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

constexpr int kZMin = 8;          // smallest z chunk any adjoint launch uses
constexpr int kStatsBlocks = 1216; // 8 blocks of 256 threads per SM on 152 SMs
constexpr int kMaxBlocksPerSM = 32;

}  // namespace

int cdi::set_error(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

struct cdi_grid {
    int nx, ny, nz;
    double dx;
    int dtype;
    int Df;
    long long n;
    const void *u, *v, *w;
    double U;
    int vel_set;
    // reduction scratch (owned)
    cdi::Partial *partials;
    unsigned int *counter;
    StatsRec *rec;    // fused-step record
    StatsRec *rec2;   // stand-alone reductions
    unsigned int *status;  // bit 0: a bounded device wait gave up
    int capacity;
    // launch configuration of the forward and adjoint kernels
    LaunchCfg fwd, adj;
    LaunchCfg rk;  // Runge-Kutta stage kernels (set on first use; nblocks 0 = unset)
    LaunchCfg slab;  // z slabs of the pipelined host step (set on first use; nblocks 0 = unset)
    LaunchCfg tb;    // two steps per pass (cdi_run with depth 2; nblocks 0 = unset)
    int run_depth;   // steps per pass of cdi_run: 1, or 2 (temporal blocking)
    int sharpen;   // CDI_SHARPEN_CENTRE (Section 2.2) or CDI_SHARPEN_FACE
    // staging for cdi_step_host (owned, allocated on first use), and the copy
    // streams and events of its slab pipeline (created on first use)
    void *stage_in, *stage_out;
    bool pipe_ready;
    cudaStream_t hs_in, hs_out;
    cudaEvent_t ev_start, ev_out, ev_in[8], ev_c[8];
    int sm_count;
};

static size_t esize(const cdi_grid *g) { return g->dtype == CDI_F64 ? 8 : 4; }

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static int check_grid(const cdi_grid *g)
{
    if (!g) return fail(CDI_ERR_ARG, "grid is NULL");
    return CDI_OK;
}

static RedScratch scratch(const cdi_grid *g, StatsRec *rec, int update_run)
{
    RedScratch r;
    r.partials = g->partials;
    r.counter = g->counter;
    r.rec = rec;
    r.capacity = g->capacity;
    r.dV = pow(g->dx, (double)g->Df);
    r.update_run = update_run;
    r.status = g->status;
    return r;
}

static void reset_run_host(StatsRec *r)
{
    memset(r, 0, sizeof(*r));
    r->mn = INFINITY;
    r->mx = -INFINITY;
    r->mn_run = INFINITY;
    r->mx_run = -INFINITY;
}

// The rotated balanced split (shares cut from a cost line where each tile column
// counts kSharePrologue planes more than its nz): its critical path in planes,
// every share's cost plus its own prologue of `pro` planes, and whether its
// cost line fits the kernels' 32-bit positions.  A share longer than a column
// runs through several tiles one after another, out of step with the blocks on
// the neighbouring tiles, whose halo rows then come from memory twice: the
// model does not offer the split there (measured at 1024^3: 4.70 ms per step
// against 4.14 ms with 6 z chunks).
static double rotated_cost(long long tiles, int nz, long long G, double pro)
{
    const long long share = (tiles * (nz + cdi::kSharePrologue) + G - 1) / G;
    return share > nz ? 1e300 : (double)share + pro;
}
static bool rotated_fits(long long tiles, int nz) { return tiles * (nz + cdi::kSharePrologue) < (1LL << 31); }

// Forward launch: a tile shape, as many blocks as fit on the GPU at once, and
// the work split.  nchunks >= 1: z chunks per tile column, (chunk, tile) units
// taken round-robin; CDI_NCHUNKS_BALANCED: equal contiguous shares of the
// tile-planes per block; 0: the split minimising the per-block critical path
// in planes, 3 planes of prologue per unit:
//   chunks: max(rounds * (planes per unit + 3), units * (planes per unit + 1) / blocks)
//   rotated balanced: ceil(tiles * (nz + kSharePrologue) / blocks) + 3.
static int fwd_cfg(const cdi_grid *g, int tile, int blocks_per_sm, int nchunks, LaunchCfg *c,
                   bool rk = false, bool slab = false)
{
    if (tile < 0 || tile >= cdi::fwd_num_tiles())
        return fail(CDI_ERR_ARG, "forward tile %d out of range", tile);
    if (rk && !cdi::fwd_tile_has_rk(tile)) return fail(CDI_ERR_ARG, "no Runge-Kutta kernel for tile %d", tile);
    const bool face = g->sharpen == CDI_SHARPEN_FACE;
    if (face && (rk || tile != 0))
        return fail(CDI_ERR_ARG, "face-product sharpening runs on forward tile 0 with Euler steps only");
    const int es = (int)esize(g);
    if (cdi::fwd_tile_is_vec(tile) && g->nx % (16 / es) != 0)
        return fail(CDI_ERR_ARG, "vector tile needs nx %% %d == 0", 16 / es);
    if (tile == 6 && !cdi::tma_eligible(es, g->nx, g->ny, g->nz))
        return fail(CDI_ERR_ARG, "tile 6 needs nx %% %d == 0 and ny %% 16 == 0", 16 * (16 / es));
    int resident = 0;
    cudaError_t e = g->dtype == CDI_F64 ? cdi::fwd_occupancy<double>(tile, rk, &resident, face, slab)
                                        : cdi::fwd_occupancy<float>(tile, rk, &resident, face, slab);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (resident < 1) return fail(CDI_ERR_CUDA, "forward kernel does not fit on an SM");
    if (blocks_per_sm > 0 && blocks_per_sm < resident) resident = blocks_per_sm;
    const long long G = (long long)resident * g->sm_count;
    const long long tiles = cdi::fwd_tiles_xy(tile, es, g->nx, g->ny);
    const int nz = g->nz;
    if (nchunks < 0 && nchunks != CDI_NCHUNKS_BALANCED && nchunks != CDI_NCHUNKS_ROTATED)
        return fail(CDI_ERR_ARG, "nchunks %d", nchunks);
    if (nchunks == 0) {
        double best = 1e300;
        for (int nc = 1; nc <= nz; ++nc) {
            const int zc = (nz + nc - 1) / nc;
            if (nc > 1 && zc == (nz + nc - 2) / (nc - 1)) continue;  // same split as nc - 1
            const long long units = tiles * ((nz + zc - 1) / zc);
            const double rounds = (double)((units + G - 1) / G);
            const double cost = fmax(rounds * (zc + 3.0), (double)units * (zc + 1.0) / (double)G);
            if (cost < best * (1.0 - 1e-9)) {
                best = cost;
                nchunks = nc;
            }
        }
        // balanced shares with rotated columns where they win: neighbouring tiles then share
        // their halo rows in L2 (measured: 256^3 79.5 vs 80.6 us, 512^3 521 vs 584 us)
        if (rotated_cost(tiles, nz, G, 3.0) < best * (1.0 - 1e-9) && rotated_fits(tiles, nz))
            nchunks = CDI_NCHUNKS_ROTATED;
    }
    long long nb;
    if (nchunks == CDI_NCHUNKS_BALANCED || nchunks == CDI_NCHUNKS_ROTATED) {
        const long long T = tiles * nz;
        if (T >= (1LL << 31) || (nchunks == CDI_NCHUNKS_ROTATED && !rotated_fits(tiles, nz)))
            return fail(CDI_ERR_DIM, "balanced split needs fewer than 2^31 tile-planes");
        nb = G < T ? G : T;
    } else {
        if (nchunks > nz) nchunks = nz;
        const int zc = (nz + nchunks - 1) / nchunks;
        const long long units = tiles * ((nz + zc - 1) / zc);
        nb = G < units ? G : units;
    }
    if (nb > g->capacity) nb = g->capacity;
    c->tile = tile;
    c->zchunk = 0;
    c->nblocks = (int)nb;
    c->nchunks = nchunks;
    return CDI_OK;
}

static int fwd_cfg_rk(const cdi_grid *g, int tile, LaunchCfg *c) { return fwd_cfg(g, tile, 0, 0, c, true); }

static int default_fwd_tile(const cdi_grid *g)
{
    if (g->sharpen == CDI_SHARPEN_FACE) return 0;
    const int vx = 16 / (int)esize(g);
    if (g->nx % vx == 0 && g->nx >= 48) return g->ny >= 12 ? 4 : 5;
    return (g->nx >= 32 && g->ny >= 16) ? 1 : 3;
}

// Vector adjoint: z chunking from the forward cost model (rounds of the
// persistent grid against per-unit prologues), or -1 for the balanced split
// when that model favours it.
static int adj_vec_zchunk(const cdi_grid *g)
{
    int resident = 0;
    cudaError_t e = g->dtype == CDI_F64 ? cdi::adj_vec_resident<double>(&resident)
                                        : cdi::adj_vec_resident<float>(&resident);
    if (e != cudaSuccess || resident < 1) resident = 1;
    int bw, bh;
    cdi::adj_vec_tile_dims((int)esize(g), &bw, &bh);
    const long long G = (long long)resident * g->sm_count;
    const long long tiles = (long long)((g->nx + bw - 1) / bw) * ((g->ny + bh - 1) / bh);
    const int nz = g->nz;
    double best = 1e300;
    int nch = 1;
    for (int nc = 1; nc <= nz; ++nc) {
        const int zc = (nz + nc - 1) / nc;
        if (nc > 1 && zc == (nz + nc - 2) / (nc - 1)) continue;
        const long long units = tiles * ((nz + zc - 1) / zc);
        const double rounds = (double)((units + G - 1) / G);
        const double cost = fmax(rounds * (zc + 3.0), (double)units * (zc + 1.0) / (double)G);
        if (cost < best * (1.0 - 1e-9)) {
            best = cost;
            nch = nc;
        }
    }
    if (rotated_cost(tiles, nz, G, 3.0) < best * (1.0 - 1e-9) && rotated_fits(tiles, nz))
        return CDI_NCHUNKS_ROTATED;
    return (nz + nch - 1) / nch;
}

static bool adj_vec_eligible(const cdi_grid *g) { return g->nx % (16 / (int)esize(g)) == 0; }

// Adjoint launch: the vector kernel where nx allows it (and the box is wide enough
// for its 16-byte tiles); else a one-cell-per-thread tile with a z chunk giving
// about eight blocks per SM.
static LaunchCfg adj_default(const cdi_grid *g)
{
    LaunchCfg c;
    if (adj_vec_eligible(g) && g->nx >= 48) {
        c.tile = 3;
        c.zchunk = adj_vec_zchunk(g);
        c.nblocks = 0;
        c.nchunks = 0;
        return c;
    }
    c.tile = (g->nx >= 32 && g->ny >= 16) ? 1 : 2;
    const int bx = 32, by = c.tile == 1 ? 16 : 4;
    long long tiles = (long long)((g->nx + bx - 1) / bx) * ((g->ny + by - 1) / by);
    long long want = (long long)g->sm_count * 8;
    long long zc = (g->nz * tiles + want - 1) / want;
    if (zc < kZMin) zc = kZMin;
    if (zc > g->nz) zc = g->nz;
    c.zchunk = (int)zc;
    c.nblocks = 0;
    c.nchunks = 0;
    return c;
}

// The public functions keep C linkage from their declarations in cdi.h.

int cdi_version(void) { return CDI_VERSION; }

const char *cdi_last_error_string(void) { return g_err; }

int cdi_create_grid(cdi_grid **out, int nx, int ny, int nz, double dx, int dtype)
{
    if (!out) return fail(CDI_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return fail(CDI_ERR_DIM, "extents must be >= 1 (got %d %d %d)", nx, ny, nz);
    if ((long long)nx * ny >= (1LL << 31)) return fail(CDI_ERR_DIM, "nx*ny must be < 2^31");
    if ((long long)nx * ny * nz >= (1LL << 36)) return fail(CDI_ERR_DIM, "nx*ny*nz must be < 2^36");
    if (!(dx > 0.0) || !isfinite(dx)) return fail(CDI_ERR_ARG, "dx must be finite and > 0");
    if (dtype != CDI_F32 && dtype != CDI_F64) return fail(CDI_ERR_ARG, "dtype must be CDI_F32 or CDI_F64");
    cdi_grid *g = new cdi_grid();
    memset(g, 0, sizeof(*g));
    g->nx = nx; g->ny = ny; g->nz = nz; g->dx = dx; g->dtype = dtype;
    g->Df = (nx > 1) + (ny > 1) + (nz > 1);
    g->n = (long long)nx * ny * nz;
    g->run_depth = 1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { delete g; return cuda_fail(e, "cudaGetDevice"); }
    e = cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) { delete g; return cuda_fail(e, "cudaDeviceGetAttribute"); }
    int cap = kStatsBlocks;
    if (g->sm_count * kMaxBlocksPerSM > cap) cap = g->sm_count * kMaxBlocksPerSM;
    for (int t = 0; t < cdi::adj_num_tiles(); ++t) {
        int b = cdi::adj_blocks(t, kZMin, nx, ny, nz);
        if (b > cap) cap = b;
    }
    g->capacity = cap;
    if ((e = cudaMalloc(&g->partials, sizeof(cdi::Partial) * (size_t)cap)) != cudaSuccess ||
        (e = cudaMalloc(&g->counter, sizeof(unsigned int))) != cudaSuccess ||
        (e = cudaMalloc(&g->rec, sizeof(StatsRec))) != cudaSuccess ||
        (e = cudaMalloc(&g->rec2, sizeof(StatsRec))) != cudaSuccess ||
        (e = cudaMalloc(&g->status, sizeof(unsigned int) * cdi::kStatusWords)) != cudaSuccess) {
        cdi_destroy_grid(g);
        return cuda_fail(e, "cudaMalloc(scratch)");
    }
    StatsRec h;
    reset_run_host(&h);
    if ((e = cudaMemset(g->counter, 0, sizeof(unsigned int))) != cudaSuccess ||
        (e = cudaMemset(g->status, 0, sizeof(unsigned int) * cdi::kStatusWords)) != cudaSuccess ||
        (e = cudaMemcpy(g->rec, &h, sizeof(h), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(g->rec2, &h, sizeof(h), cudaMemcpyHostToDevice)) != cudaSuccess) {
        cdi_destroy_grid(g);
        return cuda_fail(e, "scratch init");
    }
    if (int rc = fwd_cfg(g, default_fwd_tile(g), 0, 0, &g->fwd)) {
        cdi_destroy_grid(g);
        return rc;
    }
    g->adj = adj_default(g);
    *out = g;
    return CDI_OK;
}

int cdi_destroy_grid(cdi_grid *g)
{
    if (!g) return CDI_OK;
    if (g->pipe_ready) {
        cudaStreamDestroy(g->hs_in);
        cudaStreamDestroy(g->hs_out);
        cudaEventDestroy(g->ev_start);
        cudaEventDestroy(g->ev_out);
        for (int j = 0; j < 8; ++j) {
            cudaEventDestroy(g->ev_in[j]);
            cudaEventDestroy(g->ev_c[j]);
        }
    }
    cudaFree(g->partials);
    cudaFree(g->counter);
    cudaFree(g->rec);
    cudaFree(g->rec2);
    cudaFree(g->status);
    cudaFree(g->stage_in);
    cudaFree(g->stage_out);
    delete g;
    return CDI_OK;
}

int cdi_grid_info(const cdi_grid *g, int *nx, int *ny, int *nz, double *dx, int *dtype)
{
    if (int rc = check_grid(g)) return rc;
    if (nx) *nx = g->nx;
    if (ny) *ny = g->ny;
    if (nz) *nz = g->nz;
    if (dx) *dx = g->dx;
    if (dtype) *dtype = g->dtype;
    return CDI_OK;
}

int cdi_set_velocity(cdi_grid *g, const void *u, const void *v, const void *w, double umax,
                     void *stream)
{
    if (int rc = check_grid(g)) return rc;
    if (!u) return fail(CDI_ERR_ARG, "u is NULL");
    if (!v && !(g->ny == 1 && g->nz == 1)) return fail(CDI_ERR_ARG, "v may be NULL only when ny == nz == 1");
    if (!w && g->nz != 1) return fail(CDI_ERR_ARG, "w may be NULL only when nz == 1");
    if (!aligned16(u) || (v && !aligned16(v)) || (w && !aligned16(w)))
        return fail(CDI_ERR_ARG, "velocity arrays must be 16-byte aligned");
    if (!isfinite(umax) && umax > 0) return fail(CDI_ERR_ARG, "umax must be finite");
    g->u = u;
    g->v = v;
    g->w = w;
    g->vel_set = 1;
    if (umax >= 0.0) {
        g->U = umax;
        return CDI_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int nb = kStatsBlocks;
    RedScratch r = scratch(g, g->rec2, 0);
    cudaError_t e = g->dtype == CDI_F64
        ? cdi::launch_absmax<double>((const double *)u, (const double *)v, (const double *)w, g->n, r, nb, s)
        : cdi::launch_absmax<float>((const float *)u, (const float *)v, (const float *)w, g->n, r, nb, s);
    if (e != cudaSuccess) return cuda_fail(e, "absmax launch");
    StatsRec h;
    if ((e = cudaMemcpyAsync(&h, g->rec2, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(e, "absmax readback");
    if (!isfinite(h.mx)) return fail(CDI_ERR_NAN, "velocity contains non-finite values");
    g->U = h.mx;
    return CDI_OK;
}

int cdi_get_umax(const cdi_grid *g, double *U)
{
    if (int rc = check_grid(g)) return rc;
    if (!U) return fail(CDI_ERR_ARG, "U is NULL");
    if (!g->vel_set) return fail(CDI_ERR_STATE, "no velocity set");
    *U = g->U;
    return CDI_OK;
}

// Eq. 17 / 24: eps/dx >= (g + 1) / (2 g), g = gamma / U (g -> inf gives 1/2), and
// Eq. 25: A = dt gamma eps / dx^2 <= 1 / (2 D_f); both with relative slack rel.
// ascale widens the diffusive limit for RK3 (2.51/2, Eq. 27) and RK4 (2.79/2, Eq. 28).
static int condition_holds(double eps_over_dx, double gamma_over_U, double A, int Df, double rel,
                           double ascale = 1.0)
{
    if (!(eps_over_dx > 0) || !(gamma_over_U > 0) || !(A >= 0) || Df < 0 || Df > 3)
        return fail(CDI_ERR_ARG, "bad condition arguments");
    const double rhs = isinf(gamma_over_U) ? 0.5 : (gamma_over_U + 1.0) / (2.0 * gamma_over_U);
    const bool line_ok = eps_over_dx >= rhs * (1.0 - rel);
    const int d = Df > 0 ? Df : 1;
    const bool a_ok = A <= (ascale / (2.0 * d)) * (1.0 + rel);
    return (line_ok && a_ok) ? 1 : 0;
}

int cdi_check_condition(double eps_over_dx, double gamma_over_U, double A, int Df)
{
    return condition_holds(eps_over_dx, gamma_over_U, A, Df, 1e-12);
}

int cdi_max_dt(double dx, double eps, double gamma, int Df, int scheme, double *dt)
{
    if (!dt) return fail(CDI_ERR_ARG, "dt is NULL");
    if (!(dx > 0) || !(eps > 0) || !(gamma > 0) || Df < 1 || Df > 3)
        return fail(CDI_ERR_ARG, "bad arguments to cdi_max_dt");
    const double base = dx * dx / (gamma * eps * Df);
    switch (scheme) {
    case CDI_EULER:
    case CDI_RK2: *dt = base / 2.0; break;          // Eq. 25, 26
    case CDI_RK3: *dt = 2.51 * base / 4.0; break;   // Eq. 27
    case CDI_RK4: *dt = 2.79 * base / 4.0; break;   // Eq. 28
    default: return fail(CDI_ERR_ARG, "unknown scheme %d", scheme);
    }
    return CDI_OK;
}

int cdi_max_dt_mixed(double dx, double eps, double gamma, const double *umax, int Df, int scheme,
                     double *dt)
{
    if (!dt || !umax) return fail(CDI_ERR_ARG, "NULL argument to cdi_max_dt_mixed");
    double c;
    switch (scheme) {
    case CDI_EULER: c = 1.0; break;   // Eq. 10 at the crossover line, summed over axes
    case CDI_RK4: c = 2.83; break;    // Eq. 32
    default: return fail(CDI_ERR_ARG, "no mixed advective-diffusive criterion for scheme %d", scheme);
    }
    double dif;
    if (int rc = cdi_max_dt(dx, eps, gamma, Df, scheme, &dif)) return rc;
    double den = Df * gamma;
    for (int d = 0; d < Df; ++d) {
        if (!(umax[d] >= 0) || !isfinite(umax[d])) return fail(CDI_ERR_ARG, "umax[%d] must be finite and >= 0", d);
        den += umax[d];
    }
    const double adv = c * dx / den;
    *dt = adv < dif ? adv : dif;
    return CDI_OK;
}

static int check_step_args(const cdi_grid *g, const void *a, void *b, double dt, double eps,
                           double gamma, double vel_scale)
{
    if (int rc = check_grid(g)) return rc;
    if (!g->vel_set) return fail(CDI_ERR_STATE, "cdi_set_velocity has not been called");
    if (!a || !b) return fail(CDI_ERR_ARG, "phi pointer is NULL");
    if (!aligned16(a) || !aligned16(b)) return fail(CDI_ERR_ARG, "phi arrays must be 16-byte aligned");
    const size_t bytes = (size_t)g->n * esize(g);
    const char *pa = (const char *)a, *pb = (const char *)b;
    if (pa < pb + bytes && pb < pa + bytes) return fail(CDI_ERR_ARG, "phi_in and phi_out overlap");
    if (!(dt >= 0) || !isfinite(dt)) return fail(CDI_ERR_ARG, "dt must be finite and >= 0");
    if (!(eps > 0) || !isfinite(eps)) return fail(CDI_ERR_ARG, "eps must be finite and > 0");
    if (!(gamma >= 0) || !isfinite(gamma)) return fail(CDI_ERR_ARG, "gamma must be finite and >= 0");
    if (!isfinite(vel_scale)) return fail(CDI_ERR_ARG, "vel_scale must be finite");
    return CDI_OK;
}

static int check_condition_flag_scaled(const cdi_grid *g, double dt, double eps, double gamma,
                                       double vel_scale, double ascale);

static int check_condition_flag(const cdi_grid *g, double dt, double eps, double gamma,
                                double vel_scale)
{
    return check_condition_flag_scaled(g, dt, eps, gamma, vel_scale, 1.0);
}

static int check_condition_flag_scaled(const cdi_grid *g, double dt, double eps, double gamma,
                                       double vel_scale, double ascale)
{
    const double Ueff = fabs(vel_scale) * g->U;
    const double gU = Ueff > 0 ? gamma / Ueff : INFINITY;
    const double A = dt * gamma * eps / (g->dx * g->dx);
    if (!(gamma > 0)) return fail(CDI_ERR_CONDITION, "gamma must be > 0 for the boundedness condition");
    // U is measured on the stored (possibly FP32-rounded) velocity, so a
    // configuration placed on the line with a double gamma may sit a rounding
    // error below it: allow a slack of four units of the storage precision.
    const double rel = g->dtype == CDI_F32 ? 4.0 * FLT_EPSILON : 1e-12;
    int ok = condition_holds(eps / g->dx, gU, A, g->Df, rel, ascale);
    if (ok < 0) return ok;
    if (!ok)
        return fail(CDI_ERR_CONDITION,
                    "boundedness condition fails: eps/dx=%.6g gamma/U=%.6g A=%.6g Df=%d "
                    "(need eps/dx >= (g+1)/(2g) and A <= %.4g/(2 Df))",
                    eps / g->dx, gU, A, g->Df, ascale);
    return CDI_OK;
}

template <typename T>
static cdi::StepCoef<T> coefs(const cdi_grid *g, double dt, double eps, double gamma, double vs)
{
    cdi::StepCoef<T> c;
    c.c_adv = (T)(0.5 * vs);
    c.c_dif = (T)(gamma * eps / g->dx);
    c.c_shp = (T)(0.5 * gamma);
    c.c_upd = (T)(dt / g->dx);
    c.tol = sizeof(T) == 8 ? (T)DBL_EPSILON : (T)FLT_EPSILON;
    return c;
}

// Deferred finish of consecutive steps of a run: the step's block partials go to
// scratch slot `slot` (two slots of nblocks partials); with `defer` they are
// left for the next step, whose block 0 finishes them (`finish_prev`: the other
// slot's partials, of the previous step) while the next step's blocks work.
struct DeferCfg {
    int slot;
    bool defer;
    bool finish_prev;
};

// One forward step, or (z_hi > 0) its planes [z_lo, z_hi) folded into the record:
// combine adds to the record's per-step fields, update_run closes the step.
template <typename T>
static int step_t(cdi_grid *g, const void *in, void *out, double dt, double eps, double gamma,
                  double vs, cudaStream_t s, int z_lo = 0, int z_hi = 0, int combine = 0,
                  int update_run = 1, const DeferCfg *dfr = nullptr)
{
    cdi::FwdArgs<T> a;
    a.phi = (const T *)in;
    a.out = (T *)out;
    a.u = (const T *)g->u;
    a.v = (const T *)(g->v ? g->v : g->u);  // ny == nz == 1: v is inert
    a.w = (const T *)(g->w ? g->w : g->u);  // nz == 1: w is inert
    a.nx = g->nx; a.ny = g->ny; a.nz = g->nz;
    a.z_lo = z_lo;
    a.z_hi = z_hi;
    a.c = coefs<T>(g, dt, eps, gamma, vs);
    a.red = scratch(g, g->rec, update_run);
    a.red.combine = combine;
    a.rk_base = nullptr;
    a.rk_q = nullptr;
    a.rk_qout = nullptr;
    a.rk_alpha = a.rk_delta = a.rk_mu = a.rk_beta = T(0);
    const LaunchCfg &c = z_hi > 0 ? g->slab : g->fwd;
    if (c.nblocks > g->capacity)
        return fail(CDI_ERR_STATE, "launch configuration exceeds the reduction scratch");
    if (dfr) {
        if (2 * c.nblocks > g->capacity)
            return fail(CDI_ERR_STATE, "deferred finish needs two partial slots per block");
        a.red.partials = g->partials + (size_t)dfr->slot * c.nblocks;
        a.red.defer = dfr->defer;
        if (dfr->finish_prev) {
            a.red.prev = g->partials + (size_t)(1 - dfr->slot) * c.nblocks;
            a.red.prev_nb = c.nblocks;
            a.red.prev_update_run = update_run;
        }
    }
    cudaError_t e = cdi::launch_fwd<T>(a, c.tile, c.nblocks, c.nchunks, false, s,
                                       g->sharpen == CDI_SHARPEN_FACE);
    if (e != cudaSuccess) return cuda_fail(e, "forward step launch");
    return CDI_OK;
}

// Launch configuration of the two-steps-per-pass kernel: one block per SM (or as
// many as fit), tiles of W x 16 cells, the work split as for the forward kernel
// (nchunks >= 1 z chunks, CDI_NCHUNKS_BALANCED equal shares, 0 the cost model with
// the kernel's longer prologue: five planes of the first step per unit).
static int tb_cfg(const cdi_grid *g, int nchunks, LaunchCfg *c)
{
    const int es = (int)esize(g);
    if (g->nx % (16 / es) != 0) return fail(CDI_ERR_ARG, "two steps per pass need nx %% %d == 0", 16 / es);
    if (g->sharpen != CDI_SHARPEN_CENTRE)
        return fail(CDI_ERR_ARG, "two steps per pass take the centre-product sharpening only");
    int resident = 0;
    cudaError_t e = g->dtype == CDI_F64 ? cdi::tb2_occupancy<double>(&resident) : cdi::tb2_occupancy<float>(&resident);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query (two steps per pass)");
    if (resident < 1) return fail(CDI_ERR_CUDA, "the two-steps-per-pass kernel does not fit on an SM");
    const long long G = (long long)resident * g->sm_count;
    int bw, bh;
    cdi::tb2_tile_dims(es, &bw, &bh);
    const long long tiles = (long long)((g->nx + bw - 1) / bw) * ((g->ny + bh - 1) / bh);
    const int nz = g->nz;
    if (nchunks < 0 && nchunks != CDI_NCHUNKS_BALANCED && nchunks != CDI_NCHUNKS_ROTATED)
        return fail(CDI_ERR_ARG, "nchunks %d", nchunks);
    if (nchunks == 0) {
        double best = 1e300;
        for (int nc = 1; nc <= nz; ++nc) {
            const int zc = (nz + nc - 1) / nc;
            if (nc > 1 && zc == (nz + nc - 2) / (nc - 1)) continue;
            const long long units = tiles * ((nz + zc - 1) / zc);
            const double rounds = (double)((units + G - 1) / G);
            const double cost = fmax(rounds * (zc + 6.0), (double)units * (zc + 5.0) / (double)G);
            if (cost < best * (1.0 - 1e-9)) {
                best = cost;
                nchunks = nc;
            }
        }
        if (rotated_cost(tiles, nz, G, 6.0) < best * (1.0 - 1e-9) && rotated_fits(tiles, nz))
            nchunks = CDI_NCHUNKS_ROTATED;
    }
    long long nb;
    if (nchunks == CDI_NCHUNKS_BALANCED || nchunks == CDI_NCHUNKS_ROTATED) {
        const long long T = tiles * nz;
        if (T >= (1LL << 31) || (nchunks == CDI_NCHUNKS_ROTATED && !rotated_fits(tiles, nz)))
            return fail(CDI_ERR_DIM, "balanced split needs fewer than 2^31 tile-planes");
        nb = G < T ? G : T;
    } else {
        if (nchunks > nz) nchunks = nz;
        const int zc = (nz + nchunks - 1) / nchunks;
        const long long units = tiles * ((nz + zc - 1) / zc);
        nb = G < units ? G : units;
    }
    if (2 * nb > g->capacity) nb = g->capacity / 2;  // two partial slots per block
    c->tile = 0;
    c->zchunk = 0;
    c->nblocks = (int)nb;
    c->nchunks = nchunks;
    return CDI_OK;
}

// Two Euler steps in one pass: vel_scale vs1 for the first, vs2 for the second.
template <typename T>
static int step2_t(cdi_grid *g, const void *in, void *out, double dt, double eps, double gamma, double vs1,
                   double vs2, cudaStream_t s)
{
    if (g->tb.nblocks == 0)
        if (int rc = tb_cfg(g, 0, &g->tb)) return rc;
    cdi::FwdArgs<T> a;
    a.phi = (const T *)in;
    a.out = (T *)out;
    a.u = (const T *)g->u;
    a.v = (const T *)(g->v ? g->v : g->u);
    a.w = (const T *)(g->w ? g->w : g->u);
    a.nx = g->nx; a.ny = g->ny; a.nz = g->nz;
    a.c = coefs<T>(g, dt, eps, gamma, vs1);
    a.red = scratch(g, g->rec, 1);
    a.rk_base = nullptr;
    a.rk_q = nullptr;
    a.rk_qout = nullptr;
    a.rk_alpha = a.rk_delta = a.rk_mu = a.rk_beta = T(0);
    if (2 * g->tb.nblocks > g->capacity) return fail(CDI_ERR_STATE, "launch configuration exceeds the reduction scratch");
    cudaError_t e = cdi::launch_fwd_tb2<T>(a, (T)(0.5 * vs2), g->tb.nblocks, g->tb.nchunks, s);
    if (e != cudaSuccess) return cuda_fail(e, "two-steps-per-pass launch");
    return CDI_OK;
}

// One Runge-Kutta stage: evaluates r = dt * RHS(in) and writes
//   out = (base ? base : in) + alpha r + (q ? delta q : 0),  qout = mu (q ? q : in) + beta r.
// Uses the RK variant of the configured tile's kernel family (vector 16x16, or
// the scalar 32x16 / 32x4 tile).
struct RkStage {
    const void *in, *base, *q;
    void *out, *qout;
    double alpha, delta, mu, beta, vs;
    int last;  // fold the result into the run statistics
};

template <typename T>
static int rk_stage_t(cdi_grid *g, const RkStage &st, double dt, double eps, double gamma, cudaStream_t s)
{
    if (g->rk.nblocks == 0) {  // first use: RK launch configuration for this grid
        int tile = cdi::fwd_tile_is_vec(g->fwd.tile) ? 4 : ((g->nx >= 32 && g->ny >= 16) ? 1 : 3);
        if (int rc = fwd_cfg_rk(g, tile, &g->rk)) return rc;
    }
    cdi::FwdArgs<T> a;
    a.phi = (const T *)st.in;
    a.out = (T *)st.out;
    a.u = (const T *)g->u;
    a.v = (const T *)(g->v ? g->v : g->u);
    a.w = (const T *)(g->w ? g->w : g->u);
    a.nx = g->nx; a.ny = g->ny; a.nz = g->nz;
    a.c = coefs<T>(g, dt, eps, gamma, st.vs);
    a.red = scratch(g, g->rec, st.last);
    a.rk_base = (const T *)st.base;
    a.rk_q = (const T *)st.q;
    a.rk_qout = (T *)st.qout;
    a.rk_alpha = (T)st.alpha;
    a.rk_delta = (T)st.delta;
    a.rk_mu = (T)st.mu;
    a.rk_beta = (T)st.beta;
    cudaError_t e = cdi::launch_fwd<T>(a, g->rk.tile, g->rk.nblocks, g->rk.nchunks, true, s);
    if (e != cudaSuccess) return cuda_fail(e, "Runge-Kutta stage launch");
    return CDI_OK;
}

static int rk_stage(cdi_grid *g, const RkStage &st, double dt, double eps, double gamma, cudaStream_t s)
{
    return g->dtype == CDI_F64 ? rk_stage_t<double>(g, st, dt, eps, gamma, s)
                               : rk_stage_t<float>(g, st, dt, eps, gamma, s);
}

static double vscale(double t, double period) { return period > 0 ? cos(M_PI * t / period) : 1.0; }

// One step of the scheme from phi_in (kept) to phi_out, with work arrays w1, w2.
static int rk_step_impl(cdi_grid *g, const void *pin, void *pout, void *w1, void *w2, double dt,
                        double eps, double gamma, double t, double period, int scheme, cudaStream_t s)
{
    auto S = [&](const void *in, void *out, const void *base, const void *q, void *qout, double al,
                 double de, double mu, double be, double tt, int last) {
        RkStage st{in, base, q, out, qout, al, de, mu, be, vscale(tt, period), last};
        return rk_stage(g, st, dt, eps, gamma, s);
    };
    int rc = CDI_OK;
    switch (scheme) {
    case CDI_EULER:
        rc = S(pin, pout, nullptr, nullptr, nullptr, 1.0, 0.0, 0.0, 0.0, t, 1);
        break;
    case CDI_RK2:  // explicit midpoint
        if (!(rc = S(pin, w1, nullptr, nullptr, nullptr, 0.5, 0.0, 0.0, 0.0, t, 0)))
            rc = S(w1, pout, pin, nullptr, nullptr, 1.0, 0.0, 0.0, 0.0, t + 0.5 * dt, 1);
        break;
    case CDI_RK3: {  // Wray's low-storage scheme; w2 carries the previous stage's r
        const double g1 = 8.0 / 15.0, g2 = 5.0 / 12.0, g3 = 3.0 / 4.0, z2 = -17.0 / 60.0, z3 = -5.0 / 12.0;
        if (!(rc = S(pin, pout, nullptr, nullptr, w2, g1, 0.0, 0.0, 1.0, t, 0)) &&
            !(rc = S(pout, w1, nullptr, w2, w2, g2, z2, 0.0, 1.0, t + g1 * dt, 0)))
            rc = S(w1, pout, nullptr, w2, nullptr, g3, z3, 0.0, 0.0, t + (g1 + g2 + z2) * dt, 1);
        break;
    }
    case CDI_RK4:  // classic; w2 accumulates phi + dt/6 (k1 + 2 k2 + 2 k3)
        if (!(rc = S(pin, w1, nullptr, nullptr, w2, 0.5, 0.0, 1.0, 1.0 / 6.0, t, 0)) &&
            !(rc = S(w1, pout, pin, w2, w2, 0.5, 0.0, 1.0, 1.0 / 3.0, t + 0.5 * dt, 0)) &&
            !(rc = S(pout, w1, pin, w2, w2, 1.0, 0.0, 1.0, 1.0 / 3.0, t + 0.5 * dt, 0)))
            rc = S(w1, pout, w2, nullptr, nullptr, 1.0 / 6.0, 0.0, 0.0, 0.0, t + dt, 1);
        break;
    default:
        rc = fail(CDI_ERR_ARG, "unknown scheme %d", scheme);
    }
    return rc;
}

static int check_rk_args(cdi_grid *g, const void *a, void *b, void *w1, void *w2, double dt, double eps,
                         double gamma, int scheme, int flags)
{
    if (int rc = check_step_args(g, a, b, dt, eps, gamma, 1.0)) return rc;
    if (scheme < CDI_EULER || scheme > CDI_RK4) return fail(CDI_ERR_ARG, "unknown scheme %d", scheme);
    if (scheme != CDI_EULER) {
        if (!w1 || !w2) return fail(CDI_ERR_ARG, "work arrays are required for RK schemes");
        if (!aligned16(w1) || !aligned16(w2)) return fail(CDI_ERR_ARG, "work arrays must be 16-byte aligned");
        const size_t bytes = (size_t)g->n * esize(g);
        const char *p[4] = {(const char *)a, (const char *)b, (const char *)w1, (const char *)w2};
        for (int i = 0; i < 4; ++i)
            for (int j = i + 1; j < 4; ++j)
                if (p[i] < p[j] + bytes && p[j] < p[i] + bytes)
                    return fail(CDI_ERR_ARG, "phi_in, phi_out and the work arrays must not overlap");
    }
    if (flags & CDI_CHECK_CONDITION) {
        const double scale = scheme == CDI_RK3 ? 2.51 / 2.0 : scheme == CDI_RK4 ? 2.79 / 2.0 : 1.0;
        if (int rc = check_condition_flag_scaled(g, dt, eps, gamma, 1.0, scale)) return rc;
    }
    return CDI_OK;
}

int cdi_step_rk(cdi_grid *g, const void *phi_in, void *phi_out, void *work1, void *work2, double dt,
                double eps, double gamma, double t, double period, int scheme, int flags, void *stream)
{
    cdi::NvtxRange nvtx_("cdi_step_rk");
    if (g && g->sharpen == CDI_SHARPEN_FACE) return fail(CDI_ERR_ARG, "Runge-Kutta stages use the centre-product sharpening");
    if (int rc = check_rk_args(g, phi_in, phi_out, work1, work2, dt, eps, gamma, scheme, flags)) return rc;
    return rk_step_impl(g, phi_in, phi_out, work1, work2, dt, eps, gamma, t, period, scheme,
                        (cudaStream_t)stream);
}

int cdi_run_rk(cdi_grid *g, void *buf_a, void *buf_b, void *work1, void *work2, int nsteps, double t0,
               double dt, double eps, double gamma, double period, int scheme, int flags, int *final_in_b,
               void *stream)
{
    cdi::NvtxRange nvtx_("cdi_run_rk");
    if (nsteps < 0) return fail(CDI_ERR_ARG, "nsteps must be >= 0");
    if (g && g->sharpen == CDI_SHARPEN_FACE) return fail(CDI_ERR_ARG, "Runge-Kutta stages use the centre-product sharpening");
    if (int rc = check_rk_args(g, buf_a, buf_b, work1, work2, dt, eps, gamma, scheme, flags)) return rc;
    void *src = buf_a, *dst = buf_b;
    for (int i = 0; i < nsteps; ++i) {
        if (int rc = rk_step_impl(g, src, dst, work1, work2, dt, eps, gamma, t0 + i * dt, period, scheme,
                                  (cudaStream_t)stream))
            return rc;
        void *tmp = src;
        src = dst;
        dst = tmp;
    }
    if (final_in_b) *final_in_b = (src == buf_b);
    return CDI_OK;
}

int cdi_step(cdi_grid *g, const void *phi_in, void *phi_out, double dt, double eps, double gamma,
             double vel_scale, int flags, void *stream)
{
    cdi::NvtxRange nvtx_("cdi_step");
    if (int rc = check_step_args(g, phi_in, phi_out, dt, eps, gamma, vel_scale)) return rc;
    if (flags & CDI_CHECK_CONDITION)
        if (int rc = check_condition_flag(g, dt, eps, gamma, vel_scale)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    return g->dtype == CDI_F64 ? step_t<double>(g, phi_in, phi_out, dt, eps, gamma, vel_scale, s)
                               : step_t<float>(g, phi_in, phi_out, dt, eps, gamma, vel_scale, s);
}

int cdi_run(cdi_grid *g, void *buf_a, void *buf_b, int nsteps, double t0, double dt, double eps,
            double gamma, double period, int flags, int *final_in_b, void *stream)
{
    cdi::NvtxRange nvtx_("cdi_run");
    if (nsteps < 0) return fail(CDI_ERR_ARG, "nsteps must be >= 0");
    if (int rc = check_step_args(g, buf_a, buf_b, dt, eps, gamma, 1.0)) return rc;
    if (flags & CDI_CHECK_CONDITION)
        if (int rc = check_condition_flag(g, dt, eps, gamma, 1.0)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    void *src = buf_a, *dst = buf_b;
    const bool two = g->run_depth == 2 && g->sharpen == CDI_SHARPEN_CENTRE;
    // one step per launch: each step's statistics are finished by the next step's
    // block 0 (the last step finishes its own), taking the combination of the block
    // partials off the end of every step but the last
    const bool defer = !two && nsteps > 1 && 2 * g->fwd.nblocks <= g->capacity;
    for (int i = 0; i < nsteps;) {
        const double t = t0 + i * dt;
        const double vs = period > 0 ? cos(M_PI * t / period) : 1.0;
        int rc;
        if (two && i + 1 < nsteps) {  // steps i and i+1 in one pass
            const double vs2 = period > 0 ? cos(M_PI * (t0 + (i + 1) * dt) / period) : 1.0;
            rc = g->dtype == CDI_F64 ? step2_t<double>(g, src, dst, dt, eps, gamma, vs, vs2, s)
                                     : step2_t<float>(g, src, dst, dt, eps, gamma, vs, vs2, s);
            i += 2;
        } else {
            const DeferCfg d = {i & 1, i + 1 < nsteps, i > 0};
            const DeferCfg *dp = defer ? &d : nullptr;
            rc = g->dtype == CDI_F64 ? step_t<double>(g, src, dst, dt, eps, gamma, vs, s, 0, 0, 0, 1, dp)
                                     : step_t<float>(g, src, dst, dt, eps, gamma, vs, s, 0, 0, 0, 1, dp);
            i += 1;
        }
        if (rc) return rc;
        void *tmp = src;
        src = dst;
        dst = tmp;
    }
    if (final_in_b) *final_in_b = (src == buf_b);
    return CDI_OK;
}

// Read and clear the status words: CDI_ERR_TIMEOUT / CDI_ERR_BOUNDS if a kernel
// recorded a failure since the last read, else CDI_OK.  st (4 words) is the
// host copy, already transferred and synchronised.
static int status_code(const cdi_grid *g, const unsigned *st, cudaStream_t s)
{
    if (!st[0]) return CDI_OK;
    cudaMemsetAsync(g->status, 0, sizeof(unsigned int) * cdi::kStatusWords, s);
    if (st[0] & 2u)
        return fail(CDI_ERR_BOUNDS, "checked build: %u index(es) out of range, the last %u against a limit of %u",
                    st[1], st[2], st[3]);
    return fail(CDI_ERR_TIMEOUT, "a bounded device-side wait gave up; results are unreliable");
}

static int read_rec(const cdi_grid *g, const StatsRec *dev, cdi_stats *out, cudaStream_t s)
{
    StatsRec h;
    unsigned int st[cdi::kStatusWords] = {0, 0, 0, 0};
    cudaError_t e;
    if ((e = cudaMemcpyAsync(&h, dev, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(st, g->status, sizeof(st), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(e, "statistics readback");
    static_assert(sizeof(StatsRec) == sizeof(cdi_stats), "record layout");
    memcpy(out, &h, sizeof(h));
    if (int rc = status_code(g, st, s)) return rc;
    if (!isfinite(h.sum)) return fail(CDI_ERR_NAN, "non-finite phi (sum = %g)", h.sum);
    return CDI_OK;
}

int cdi_step_stats(cdi_grid *g, cdi_stats *out, void *stream)
{
    if (int rc = check_grid(g)) return rc;
    if (!out) return fail(CDI_ERR_ARG, "out is NULL");
    return read_rec(g, g->rec, out, (cudaStream_t)stream);
}

int cdi_reset_run_stats(cdi_grid *g, void *stream)
{
    if (int rc = check_grid(g)) return rc;
    StatsRec h;
    reset_run_host(&h);
    cudaStream_t s = (cudaStream_t)stream;
    // The host record must outlive the async copy: synchronise before returning.
    cudaError_t e;
    if ((e = cudaMemcpyAsync(g->rec, &h, sizeof(h), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(e, "reset run statistics");
    return CDI_OK;
}

int cdi_mass_and_bounds(cdi_grid *g, const void *phi, cdi_stats *out, void *stream)
{
    cdi::NvtxRange nvtx_("cdi_mass_and_bounds");
    if (int rc = check_grid(g)) return rc;
    if (!phi || !out) return fail(CDI_ERR_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    RedScratch r = scratch(g, g->rec2, 0);
    int nb = kStatsBlocks;
    if ((long long)nb * 256 > g->n) nb = (int)((g->n + 255) / 256);
    cudaError_t e = g->dtype == CDI_F64
        ? cdi::launch_stats<double>((const double *)phi, g->n, DBL_EPSILON, r, nb, s)
        : cdi::launch_stats<float>((const float *)phi, g->n, FLT_EPSILON, r, nb, s);
    if (e != cudaSuccess) return cuda_fail(e, "stats launch");
    return read_rec(g, g->rec2, out, s);
}

// Launch configuration of the z-range kernels (the slabs of the pipelined host
// step, cdi_step_planes): tile 4 where nx allows, else 0; balanced shares.
static int ensure_slab_cfg(cdi_grid *g)
{
    if (g->slab.nblocks != 0) return CDI_OK;
    const int tile = g->nx % (16 / (int)esize(g)) == 0 ? 4 : 0;
    return fwd_cfg(g, tile, 0, CDI_NCHUNKS_BALANCED, &g->slab, false, true);
}

int cdi_step_planes(cdi_grid *g, const void *phi_in, void *phi_out, int z_lo, int z_hi, double dt,
                    double eps, double gamma, double vel_scale, int flags, void *stream)
{
    cdi::NvtxRange nvtx_("cdi_step_planes");
    if (int rc = check_step_args(g, phi_in, phi_out, dt, eps, gamma, vel_scale)) return rc;
    if (!(0 <= z_lo && z_lo < z_hi && z_hi <= g->nz))
        return fail(CDI_ERR_ARG, "need 0 <= z_lo < z_hi <= nz (got %d, %d, nz %d)", z_lo, z_hi, g->nz);
    if (g->sharpen != CDI_SHARPEN_CENTRE)
        return fail(CDI_ERR_ARG, "cdi_step_planes takes the centre-product sharpening only");
    if (flags & CDI_CHECK_CONDITION)
        if (int rc = check_condition_flag(g, dt, eps, gamma, vel_scale)) return rc;
    if (int rc = ensure_slab_cfg(g)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    return g->dtype == CDI_F64
        ? step_t<double>(g, phi_in, phi_out, dt, eps, gamma, vel_scale, s, z_lo, z_hi, 0, 1)
        : step_t<float>(g, phi_in, phi_out, dt, eps, gamma, vel_scale, s, z_lo, z_hi, 0, 1);
}

// The host-buffer step's slab plan for nz >= 16 planes: slab j is planes
// [b[j], b[j+1]) (8 equal slabs); after the two seam planes nz-2, nz-1, copy-in
// piece j is planes [c0[j], c1[j]) = [b[j] + 2, b[j+1] + 2) (piece 0 from plane 0,
// the last up to nz - 2), so piece j ends with the two halo planes above slab j
// and slab j is stepped once piece j has landed (the halo below it came with
// piece j-1; the last slab's wrapped halo with the seam planes and piece 0).  For
// the smallest nz a piece may repeat seam planes.
constexpr int kHostSlabs = 8;
static_assert(kHostSlabs == sizeof(cdi_grid::ev_in) / sizeof(cudaEvent_t), "one copy-in event per slab");
static void host_slab_plan(int nz, int *b, int *c0, int *c1)
{
    constexpr int S = kHostSlabs;
    for (int j = 0; j <= S; ++j) b[j] = (int)((long long)j * nz / S);
    for (int j = 0; j < S; ++j) {
        c0[j] = j == 0 ? 0 : b[j] + 2;
        c1[j] = j == S - 1 ? nz - 2 : b[j + 1] + 2;
    }
}

int cdi_host_slab_plan(int nz, int *bounds, int *copy_lo, int *copy_hi)
{
    if (nz < 16) return fail(CDI_ERR_DIM, "the slab pipeline needs nz >= 16");
    if (!bounds || !copy_lo || !copy_hi) return fail(CDI_ERR_ARG, "NULL argument");
    host_slab_plan(nz, bounds, copy_lo, copy_hi);
    return CDI_OK;
}

// cdi_step_host in S = 8 equal z slabs (host_slab_plan): the two planes of the
// periodic seam (nz-2, nz-1) are copied in first, then the pieces in order on
// hs_in; slab j is stepped on the caller's stream as soon as piece j (which ends
// with its upper halo planes) has landed, and copied out on hs_out once stepped,
// so both copy directions and the kernel overlap.  The record is built by folding
// the slabs' partial results (combine) and closed by the last slab.  (256^3 FP32:
// 0.566 ms per step; with pieces ending at the slab bounds, each slab waiting for
// the next piece, 2 slabs 0.78 ms, 4: 0.65, 8: 0.58, 16: 0.61, 32: 0.88 -- per-slab
// copy and launch costs against overlap; the unpipelined step 0.80.)
static int step_host_pipelined(cdi_grid *g, const void *hin, void *hout, double dt, double eps,
                               double gamma, double vs, cudaStream_t s)
{
    cudaError_t e;
    if (!g->pipe_ready) {
        if ((e = cudaStreamCreateWithFlags(&g->hs_in, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamCreate");
        if ((e = cudaStreamCreateWithFlags(&g->hs_out, cudaStreamNonBlocking)) != cudaSuccess) {
            cudaStreamDestroy(g->hs_in);
            return cuda_fail(e, "cudaStreamCreate");
        }
        e = cudaEventCreateWithFlags(&g->ev_start, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_out, cudaEventDisableTiming);
        for (int j = 0; j < 8 && e == cudaSuccess; ++j) {
            e = cudaEventCreateWithFlags(&g->ev_in[j], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_c[j], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");  // (process-lifetime leak only)
        g->pipe_ready = true;
    }
    if (int rc = ensure_slab_cfg(g)) return rc;
    constexpr int S = kHostSlabs;
    const int nz = g->nz;  // nz >= 16: every slab holds the two halo planes
    int b[S + 1], c0[S], c1[S];
    host_slab_plan(nz, b, c0, c1);
    const size_t pb = (size_t)g->nx * g->ny * esize(g);
    const char *src = (const char *)hin;
    char *dst = (char *)hout;
    char *si = (char *)g->stage_in, *so = (char *)g->stage_out;
    // the copies start after the work already queued on the caller's stream
    if ((e = cudaEventRecord(g->ev_start, s)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(g->hs_in, g->ev_start, 0)) != cudaSuccess)
        return cuda_fail(e, "pipeline start");
    auto h2d = [&](int z0, int z1) {
        if (z1 <= z0) return cudaSuccess;
        return cudaMemcpyAsync(si + (size_t)z0 * pb, src + (size_t)z0 * pb, (size_t)(z1 - z0) * pb,
                               cudaMemcpyHostToDevice, g->hs_in);
    };
    // copy-in order: the two seam planes, then the pieces of host_slab_plan
    if ((e = h2d(nz - 2, nz)) != cudaSuccess) return cuda_fail(e, "host-to-device copy");
    for (int j = 0; j < S; ++j) {
        if ((e = h2d(c0[j], c1[j])) != cudaSuccess || (e = cudaEventRecord(g->ev_in[j], g->hs_in)) != cudaSuccess)
            return cuda_fail(e, "host-to-device copy");
    }
    for (int j = 0; j < S; ++j) {
        if ((e = cudaStreamWaitEvent(s, g->ev_in[j], 0)) != cudaSuccess) return cuda_fail(e, "wait");
        int rc = g->dtype == CDI_F64
                     ? step_t<double>(g, si, so, dt, eps, gamma, vs, s, b[j], b[j + 1], j > 0, j == S - 1)
                     : step_t<float>(g, si, so, dt, eps, gamma, vs, s, b[j], b[j + 1], j > 0, j == S - 1);
        if (rc) return rc;
        const size_t off = (size_t)b[j] * pb, len = (size_t)(b[j + 1] - b[j]) * pb;
        if ((e = cudaEventRecord(g->ev_c[j], s)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(g->hs_out, g->ev_c[j], 0)) != cudaSuccess ||
            (e = cudaMemcpyAsync(dst + off, so + off, len, cudaMemcpyDeviceToHost, g->hs_out)) != cudaSuccess)
            return cuda_fail(e, "device-to-host copy");
    }
    if ((e = cudaEventRecord(g->ev_out, g->hs_out)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(s, g->ev_out, 0)) != cudaSuccess)
        return cuda_fail(e, "pipeline end");
    return CDI_OK;
}

int cdi_step_host(cdi_grid *g, const void *phi_in_host, void *phi_out_host, double dt, double eps,
                  double gamma, double vel_scale, int flags, cdi_stats *stats_out, void *stream)
{
    cdi::NvtxRange nvtx_("cdi_step_host");
    if (int rc = check_grid(g)) return rc;
    if (!phi_in_host || !phi_out_host) return fail(CDI_ERR_ARG, "host pointer is NULL");
    const size_t bytes = (size_t)g->n * esize(g);
    cudaError_t e;
    if (!g->stage_in) {
        if ((e = cudaMalloc(&g->stage_in, bytes)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(stage)");
        if ((e = cudaMalloc(&g->stage_out, bytes)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(stage)");
    }
    cudaStream_t s = (cudaStream_t)stream;
    // slab pipeline when every slab holds at least the two halo planes (the
    // default sharpening form only)
    if (g->nz >= 16 && g->sharpen == CDI_SHARPEN_CENTRE) {
        if (int rc = check_step_args(g, g->stage_in, g->stage_out, dt, eps, gamma, vel_scale)) return rc;
        if (flags & CDI_CHECK_CONDITION)
            if (int rc = check_condition_flag(g, dt, eps, gamma, vel_scale)) return rc;
        if (int rc = step_host_pipelined(g, phi_in_host, phi_out_host, dt, eps, gamma, vel_scale, s))
            return rc;
        if (stats_out) return read_rec(g, g->rec, stats_out, s);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "synchronise");
        return CDI_OK;
    }
    if ((e = cudaMemcpyAsync(g->stage_in, phi_in_host, bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(e, "host-to-device copy");
    if (int rc = cdi_step(g, g->stage_in, g->stage_out, dt, eps, gamma, vel_scale, flags, stream)) return rc;
    if ((e = cudaMemcpyAsync(phi_out_host, g->stage_out, bytes, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(e, "device-to-host copy");
    if (stats_out) return read_rec(g, g->rec, stats_out, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "synchronise");
    return CDI_OK;
}

template <typename T>
static int adjoint_t(cdi_grid *g, const void *phi, const void *lam, void *out, void *gu, void *gv,
                     void *gw, double dt, double eps, double gamma, double vs, cudaStream_t s)
{
    cdi::AdjArgs<T> a;
    a.phi = (const T *)phi;
    a.lam = (const T *)lam;
    a.out = (T *)out;
    a.u = (const T *)g->u;
    a.v = (const T *)(g->v ? g->v : g->u);
    a.w = (const T *)(g->w ? g->w : g->u);
    a.gu = (T *)gu;
    a.gv = (T *)gv;
    a.gw = (T *)gw;
    a.nx = g->nx; a.ny = g->ny; a.nz = g->nz;
    a.zchunk = g->adj.zchunk;
    a.c = coefs<T>(g, dt, eps, gamma, vs);
    a.c_shp_adj = (T)(gamma * dt / (2.0 * g->dx));
    a.c_vel = (T)(0.5 * vs);
    a.status = g->status;
    if (cdi::adj_blocks(g->adj.tile, a.zchunk, g->nx, g->ny, g->nz) > g->capacity)
        return fail(CDI_ERR_STATE, "adjoint launch configuration out of range");
    cudaError_t e = cdi::launch_adj<T>(a, g->adj.tile, s);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint step launch");
    return CDI_OK;
}

int cdi_step_adjoint(cdi_grid *g, const void *phi_k, const void *lam_next, void *lam_k, void *gu,
                     void *gv, void *gw, double dt, double eps, double gamma, double vel_scale,
                     void *stream)
{
    cdi::NvtxRange nvtx_("cdi_step_adjoint");
    if (int rc = check_step_args(g, phi_k, lam_k, dt, eps, gamma, vel_scale)) return rc;
    if (g->sharpen == CDI_SHARPEN_FACE)
        return fail(CDI_ERR_ARG, "the adjoint is of the centre-product step (Section 2.2)");
    if (!lam_next || !aligned16(lam_next)) return fail(CDI_ERR_ARG, "lam_next NULL or misaligned");
    const size_t bytes = (size_t)g->n * esize(g);
    const char *pa = (const char *)lam_next, *pb = (const char *)lam_k;
    if (pa < pb + bytes && pb < pa + bytes) return fail(CDI_ERR_ARG, "lam_k overlaps lam_next");
    const int ng = (gu != nullptr) + (gv != nullptr) + (gw != nullptr);
    if (ng != 0 && ng != 3) return fail(CDI_ERR_ARG, "gu, gv, gw must be all NULL or all set");
    if (ng == 3 && (!aligned16(gu) || !aligned16(gv) || !aligned16(gw)))
        return fail(CDI_ERR_ARG, "velocity gradients must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    return g->dtype == CDI_F64
        ? adjoint_t<double>(g, phi_k, lam_next, lam_k, gu, gv, gw, dt, eps, gamma, vel_scale, s)
        : adjoint_t<float>(g, phi_k, lam_next, lam_k, gu, gv, gw, dt, eps, gamma, vel_scale, s);
}


int cdi_set_launch(cdi_grid *g, int which, int tile, int blocks_per_sm, int nchunks)
{
    if (int rc = check_grid(g)) return rc;
    if (which == CDI_KERNEL_FORWARD) {
        if (tile < 0) tile = default_fwd_tile(g);
        LaunchCfg c;
        if (int rc = fwd_cfg(g, tile, blocks_per_sm, nchunks, &c)) return rc;
        g->fwd = c;
        g->rk.nblocks = 0;  // the Runge-Kutta configuration follows on next use
        return CDI_OK;
    }
    if (which == CDI_KERNEL_ADJOINT) {
        if (tile < 0) {
            g->adj = adj_default(g);
            return CDI_OK;
        }
        if (tile >= cdi::adj_num_tiles()) return fail(CDI_ERR_ARG, "adjoint tile %d out of range", tile);
        if (cdi::adj_tile_is_vec(tile) && !adj_vec_eligible(g))
            return fail(CDI_ERR_ARG, "vector adjoint tile needs nx %% %d == 0", 16 / (int)esize(g));
        LaunchCfg c = adj_default(g);
        if (cdi::adj_tile_is_vec(tile) && !cdi::adj_tile_is_vec(c.tile)) c.zchunk = adj_vec_zchunk(g);
        c.tile = tile;
        if (nchunks > 0) c.zchunk = (g->nz + nchunks - 1) / nchunks;
        if (nchunks == CDI_NCHUNKS_BALANCED || nchunks == CDI_NCHUNKS_ROTATED) {
            if (!cdi::adj_tile_is_vec(tile)) return fail(CDI_ERR_ARG, "balanced split: vector adjoint tile only");
            int bw, bh;
            cdi::adj_vec_tile_dims((int)esize(g), &bw, &bh);
            const long long tiles = (long long)((g->nx + bw - 1) / bw) * ((g->ny + bh - 1) / bh);
            if (tiles * g->nz >= (1LL << 31) || (nchunks == CDI_NCHUNKS_ROTATED && !rotated_fits(tiles, g->nz)))
                return fail(CDI_ERR_DIM, "balanced split needs fewer than 2^31 tile-planes");
            c.zchunk = nchunks;
        } else if (nchunks < 0) {
            return fail(CDI_ERR_ARG, "nchunks %d", nchunks);
        }
        if (c.zchunk < 0 && !cdi::adj_tile_is_vec(c.tile)) c.zchunk = adj_default(g).zchunk;
        if (c.zchunk > 0 && cdi::adj_blocks(c.tile, c.zchunk, g->nx, g->ny, g->nz) > g->capacity)
            return fail(CDI_ERR_ARG, "adjoint configuration needs more blocks than the scratch holds");
        g->adj = c;
        return CDI_OK;
    }
    return fail(CDI_ERR_ARG, "unknown kernel %d", which);
}

// One block whose thread 0 waits on an mbarrier that nothing ever completes:
// the bounded wait must run out, set the status bit and let the kernel end.
__global__ void probe_wait_kernel(unsigned int *status, unsigned long long limit_ns)
{
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        cdi::mbar_init(&bar, 1);
        cdi::fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) cdi::mbar_wait_bounded(&bar, 0u, status, limit_ns);
    __syncthreads();
}

int cdi_probe_bounded_wait(cdi_grid *g, double limit_s, void *stream)
{
    if (int rc = check_grid(g)) return rc;
    if (!(limit_s > 0.0 && limit_s <= 2.0)) return fail(CDI_ERR_ARG, "limit_s must be in (0, 2]");
    cudaStream_t s = (cudaStream_t)stream;
    probe_wait_kernel<<<1, 32, 0, s>>>(g->status, (unsigned long long)(limit_s * 1e9));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "probe launch");
    unsigned int st = 0;
    if ((e = cudaMemcpyAsync(&st, g->status, sizeof(st), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(e, "probe status readback");
    if (!st) return CDI_OK;  // the wait did not run out: the time-out path is broken
    cudaMemsetAsync(g->status, 0, sizeof(unsigned int) * cdi::kStatusWords, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "probe status reset");
    return fail(CDI_ERR_TIMEOUT, "bounded device wait ran out (probe)");
}

// FP64 FMA throughput: every thread runs CHAINS independent fused multiply-add
// chains of ITERS steps (no memory traffic inside the loop); the result is
// stored only if it is negative, which it never is, so the work is kept.
constexpr int kFp64Chains = 8;
__global__ void __launch_bounds__(256) fp64_rate_kernel(int iters, double *sink)
{
    double a[kFp64Chains];
#pragma unroll
    for (int c = 0; c < kFp64Chains; ++c) a[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    const double m = 0.999999, k = 1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kFp64Chains; ++c) a[c] = fma(a[c], m, k);
    }
    double t = 0.0;
#pragma unroll
    for (int c = 0; c < kFp64Chains; ++c) t += a[c];
    if (t < 0.0) sink[blockIdx.x] = t;
}

int cdi_probe_fp64_rate(double *fma_per_s, void *stream)
{
    if (!fma_per_s) return fail(CDI_ERR_ARG, "fma_per_s is NULL");
    int dev = 0, sms = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return cuda_fail(e, "device query");
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = sms * 8, threads = 256, iters = 4096;
    cudaEvent_t e0, e1;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(e, "cudaEventCreate");
    }
    float best = 1e30f;
    int rc = CDI_OK;
    for (int rep = 0; rep < 4 && rc == CDI_OK; ++rep) {  // the first launch is a warm-up
        cudaEventRecord(e0, s);
        fp64_rate_kernel<<<blocks, threads, 0, s>>>(iters, nullptr);
        cudaEventRecord(e1, s);
        if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) {
            rc = cuda_fail(e, "fp64 rate kernel");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    *fma_per_s = (double)blocks * threads * iters * kFp64Chains / (best * 1e-3);
    return CDI_OK;
}

// One thread tests an index one past the limit with the checked-build test.
__global__ void probe_bounds_kernel(unsigned int *status, long long limit)
{
    if (threadIdx.x == 0) {
        const long long i = CDI_CHK(limit, limit, status);
        (void)i;
    }
}

int cdi_is_checked_build(void)
{
#ifdef CDI_CHECKED
    return 1;
#else
    return 0;
#endif
}

int cdi_probe_bounds_check(cdi_grid *g, void *stream)
{
    if (int rc = check_grid(g)) return rc;
    if (!cdi_is_checked_build()) return fail(CDI_ERR_STATE, "not a checked build (CDI_CHECKED)");
    cudaStream_t s = (cudaStream_t)stream;
    probe_bounds_kernel<<<1, 32, 0, s>>>(g->status, 12345);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "probe launch");
    unsigned int st[cdi::kStatusWords] = {0, 0, 0, 0};
    if ((e = cudaMemcpyAsync(st, g->status, sizeof(st), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(e, "probe status readback");
    return status_code(g, st, s);
}

int cdi_set_sharpening(cdi_grid *g, int mode)
{
    if (int rc = check_grid(g)) return rc;
    if (mode != CDI_SHARPEN_CENTRE && mode != CDI_SHARPEN_FACE) return fail(CDI_ERR_ARG, "sharpening mode %d", mode);
    const int old = g->sharpen;
    g->sharpen = mode;
    LaunchCfg c;
    if (int rc = fwd_cfg(g, default_fwd_tile(g), 0, 0, &c)) {
        g->sharpen = old;
        return rc;
    }
    g->fwd = c;
    g->rk.nblocks = 0;
    if (mode != CDI_SHARPEN_CENTRE) g->run_depth = 1;  // two steps per pass: centre form only
    return CDI_OK;
}

int cdi_get_sharpening(const cdi_grid *g, int *mode)
{
    if (int rc = check_grid(g)) return rc;
    if (!mode) return fail(CDI_ERR_ARG, "mode is NULL");
    *mode = g->sharpen;
    return CDI_OK;
}

int cdi_set_run_depth(cdi_grid *g, int depth, int nchunks)
{
    if (int rc = check_grid(g)) return rc;
    if (depth != 1 && depth != 2) return fail(CDI_ERR_ARG, "run depth must be 1 or 2 (got %d)", depth);
    if (depth == 2) {
        LaunchCfg c;
        if (int rc = tb_cfg(g, nchunks, &c)) return rc;
        g->tb = c;
    }
    g->run_depth = depth;
    return CDI_OK;
}

int cdi_get_run_depth(const cdi_grid *g, int *depth, int *nblocks, int *nchunks)
{
    if (int rc = check_grid(g)) return rc;
    if (depth) *depth = g->run_depth;
    if (nblocks) *nblocks = g->tb.nblocks;
    if (nchunks) *nchunks = g->tb.nchunks;
    return CDI_OK;
}

int cdi_get_launch(const cdi_grid *g, int which, int *tile, int *nblocks, int *nchunks)
{
    if (int rc = check_grid(g)) return rc;
    const LaunchCfg *c = which == CDI_KERNEL_FORWARD ? &g->fwd : which == CDI_KERNEL_ADJOINT ? &g->adj : nullptr;
    if (!c) return fail(CDI_ERR_ARG, "unknown kernel %d", which);
    if (tile) *tile = c->tile;
    if (nblocks) *nblocks = c->nblocks;
    if (nchunks)
        *nchunks = which == CDI_KERNEL_FORWARD ? c->nchunks
                   : c->zchunk < 0           ? c->zchunk
                                             : (g->nz + c->zchunk - 1) / c->zchunk;
    return CDI_OK;
}

int cdi_autotune(cdi_grid *g, void *phi_a, void *phi_b, double dt, double eps, double gamma, int reps,
                 double *best_ms, void *stream)
{
    cdi::NvtxRange nvtx_("cdi_autotune");
    if (int rc = check_step_args(g, phi_a, phi_b, dt, eps, gamma, 1.0)) return rc;
    if (reps < 1) return fail(CDI_ERR_ARG, "reps must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    cudaError_t e;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(e, "cudaEventCreate");
    }
    const LaunchCfg saved = g->fwd;
    LaunchCfg best = saved;
    float best_t = 1e30f;
    int rc = CDI_OK;
    const int chunk_opts[] = {CDI_NCHUNKS_BALANCED, CDI_NCHUNKS_ROTATED, 0, 1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 14,
                              16, 20, 24, 32};
    for (int tile = 0; tile < cdi::fwd_num_tiles() && rc == CDI_OK; ++tile) {
        if (cdi::fwd_tile_is_vec(tile) && g->nx % (16 / (int)esize(g)) != 0) continue;
        if (g->sharpen == CDI_SHARPEN_FACE && tile != 0) continue;
        for (int oi = 0; oi < (int)(sizeof(chunk_opts) / sizeof(int)); ++oi) {
            if (chunk_opts[oi] > g->nz) continue;
            LaunchCfg c;
            if (fwd_cfg(g, tile, 0, chunk_opts[oi], &c) != CDI_OK) continue;
            g->fwd = c;
            void *src = phi_a, *dst = phi_b;
            // warm-up launch, then reps timed launches (ping-pong)
            for (int i = 0; i <= reps && rc == CDI_OK; ++i) {
                if (i == 1 && (e = cudaEventRecord(e0, s)) != cudaSuccess) rc = cuda_fail(e, "event");
                if (rc == CDI_OK)
                    rc = g->dtype == CDI_F64 ? step_t<double>(g, src, dst, dt, eps, gamma, 1.0, s)
                                             : step_t<float>(g, src, dst, dt, eps, gamma, 1.0, s);
                void *t = src; src = dst; dst = t;
            }
            if (rc != CDI_OK) break;
            if ((e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) {
                rc = cuda_fail(e, "event");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= reps;
            if (ms < best_t) {
                best_t = ms;
                best = c;
            }
        }
    }
    // Depth of cdi_run: two steps per pass where that kernel applies and is faster
    // per step than the best single-step configuration.
    float best2 = 1e30f;
    LaunchCfg best_tb = g->tb;
    const bool tb_ok = rc == CDI_OK && g->sharpen == CDI_SHARPEN_CENTRE && g->nx % (16 / (int)esize(g)) == 0;
    const int tb_opts[] = {CDI_NCHUNKS_BALANCED, CDI_NCHUNKS_ROTATED, 0, 1, 2, 4, 8};
    for (int oi = 0; tb_ok && rc == CDI_OK && oi < (int)(sizeof(tb_opts) / sizeof(int)); ++oi) {
        if (tb_opts[oi] > g->nz) continue;
        LaunchCfg c;
        if (tb_cfg(g, tb_opts[oi], &c) != CDI_OK) continue;
        g->tb = c;
        void *src = phi_a, *dst = phi_b;
        for (int i = 0; i <= reps && rc == CDI_OK; ++i) {  // warm-up pass, then reps passes
            if (i == 1 && (e = cudaEventRecord(e0, s)) != cudaSuccess) rc = cuda_fail(e, "event");
            if (rc == CDI_OK)
                rc = g->dtype == CDI_F64 ? step2_t<double>(g, src, dst, dt, eps, gamma, 1.0, 1.0, s)
                                         : step2_t<float>(g, src, dst, dt, eps, gamma, 1.0, 1.0, s);
            void *t = src; src = dst; dst = t;
        }
        if (rc != CDI_OK) break;
        if ((e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) {
            rc = cuda_fail(e, "event");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= 2 * reps;  // per step
        if (ms < best2) {
            best2 = ms;
            best_tb = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g->fwd = rc == CDI_OK ? best : saved;
    g->rk.nblocks = 0;
    if (rc == CDI_OK) {
        g->tb = best_tb;
        g->run_depth = best2 < best_t ? 2 : 1;
        if (best_ms) *best_ms = best2 < best_t ? best2 : best_t;
    }
    return rc;
}
