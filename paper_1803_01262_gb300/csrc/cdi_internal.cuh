// Internal declarations shared by the CDI CUDA translation units.
// Not part of the public ABI (include/cdi.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cdi {

// Prologue weight, in planes, of a tile column in the rotated balanced work
// split (CDI_NCHUNKS_ROTATED): a share that starts a new column is that many
// planes shorter (best of 0..8 measured at 256^2 x 64, 256, 512 planes).
constexpr int kSharePrologue = 4;

// Per-block partial of the fused reductions (mass, min, max, violation counts).
struct Partial {
    double sum;
    double mn;
    double mx;
    long long ns;  // #(phi < 0 or phi > 1)
    long long nt;  // #(phi < -tol or phi > 1 + tol)
};

// Device-side statistics record; same layout as the public cdi_stats.
struct StatsRec {
    double mass, sum, mn, mx;
    long long ns, nt;
    double mn_run, mx_run;
    long long ns_run, nt_run, steps_run;
};

// Library-owned reduction scratch of one grid.
struct RedScratch {
    Partial *partials;      // one slot per block of the largest launch
    unsigned int *counter;  // blocks finished in the current launch (self-resetting)
    StatsRec *rec;          // result record
    int capacity;           // number of partial slots
    double dV;              // cell measure dx^D_f
    int update_run;         // 1: fold this result into the *_run accumulators
    unsigned int *status;   // nullable: the status words (kStatusWords, below)
    int combine = 0;        // 1: add this launch's result to the record's per-step fields
                            //    (a step done in several launches over z slabs)
    // Deferred finish (consecutive steps of a run): a launch with defer = 1 only
    // stores its block partials; the next launch's block 0 combines them into the
    // record (prev, prev_nb, prev_update_run), off the critical path of both.
    int defer = 0;
    const Partial *prev = nullptr;
    int prev_nb = 0;
    int prev_update_run = 0;
};

// Coefficients of one step, precomputed on the host in double and cast.
template <typename T>
struct StepCoef {
    T c_adv;  // vel_scale / 2      (advective flux u_f (phi_L + phi_R)/2)
    T c_dif;  // gamma * eps / dx   (diffusive flux)
    T c_shp;  // gamma / 2          (sharpening flux, face average of s)
    T c_upd;  // dt / dx            (flux divergence)
    T tol;    // machine epsilon of T (tolerant bound count)
};

template <typename T>
struct FwdArgs {
    const T *__restrict__ phi;
    T *__restrict__ out;
    const T *__restrict__ u;
    const T *__restrict__ v;
    const T *__restrict__ w;
    int nx, ny, nz;
    StepCoef<T> c;
    RedScratch red;
    // Runge-Kutta stage epilogue (kernels instantiated with RK), per cell with
    // r = dt * RHS(phi) = -c_upd * (flux divergence) and c = phi at the cell:
    //   out  = (rk_base ? rk_base : c) + rk_alpha r + (rk_q ? rk_delta rk_q : 0)
    //   qout = rk_mu (rk_q ? rk_q : c) + rk_beta r          (if rk_qout)
    // rk_q and rk_qout may be the same array (each cell reads before it writes).
    const T *rk_base;
    const T *rk_q;
    T *rk_qout;
    T rk_alpha, rk_delta, rk_mu, rk_beta;
    int z_lo = 0, z_hi = 0;  // z_hi > 0: only planes [z_lo, z_hi) are updated (forward
                             // tiles 0 and 4, the slabs of a pipelined host step)
};

template <typename T>
struct AdjArgs {
    const T *__restrict__ phi;
    const T *__restrict__ lam;   // lambda^{k+1}
    T *__restrict__ out;         // lambda^k
    const T *__restrict__ u;
    const T *__restrict__ v;
    const T *__restrict__ w;
    T *gu, *gv, *gw;             // nullable, accumulated
    int nx, ny, nz;
    int zchunk;
    StepCoef<T> c;
    T c_shp_adj;                 // gamma dt / (2 dx)
    T c_vel;                     // vel_scale / 2 (velocity gradient factor)
    unsigned int *status;        // nullable: status words (checked builds record here)
};

// Launch configuration of a kernel: tile shape, z chunk (adjoint), block count.
struct LaunchCfg {
    int tile;     // index into the kernel's tile table
    int zchunk;   // planes per block along z (adjoint kernel)
    int nblocks;  // blocks per launch (forward: resident blocks, units round-robin)
    int nchunks;  // z chunks per tile column (forward)
};

int fwd_num_tiles();
bool fwd_tile_is_vec(int tile);
void fwd_tile_dims(int tile, int esize, int *bw, int *bh);
long long fwd_tiles_xy(int tile, int esize, int nx, int ny);

// Blocks of the forward kernel with this tile that fit on one SM (sets the smem attribute).
template <typename T>
cudaError_t fwd_occupancy(int tile, bool rk, int *resident, bool face = false, bool slab = false);

// Two steps per pass (cdi_fwd_tb.cu): W x 16 tiles (W = 16 * 16/sizeof(T)), one
// block per SM; needs nx % (16/sizeof(T)) == 0.  c_adv2: the advective
// coefficient of the second step (a.c.c_adv that of the first).
template <typename T>
cudaError_t tb2_occupancy(int *resident);
template <typename T>
cudaError_t launch_fwd_tb2(const FwdArgs<T> &a, T c_adv2, int nblocks, int nchunks, cudaStream_t s);
void tb2_tile_dims(int esize, int *bw, int *bh);

// Tile 6: tensor-memory-accelerator staging (cdi_fwd_tma.cu); needs
// nx % W == 0 and ny % 16 == 0 with W = 16 * 16 / sizeof(T).
bool tma_eligible(int esize, int nx, int ny, int nz);
template <typename T>
cudaError_t tma_occupancy(int *resident);
template <typename T>
cudaError_t launch_fwd_tma(const FwdArgs<T> &a, int nblocks, int nchunks, cudaStream_t s);

// rk selects the Runge-Kutta stage variant (tiles with fwd_tile_has_rk only);
// face the face-product sharpening (tile 0, Euler only).
bool fwd_tile_has_rk(int tile);

template <typename T>
cudaError_t launch_fwd(const FwdArgs<T> &a, int tile, int nblocks, int nchunks, bool rk, cudaStream_t s,
                       bool face = false);

template <typename T>
cudaError_t launch_stats(const T *phi, long long n, T tol, RedScratch red, int nblocks,
                         cudaStream_t s);

template <typename T>
cudaError_t launch_absmax(const T *u, const T *v, const T *w, long long n, RedScratch red,
                          int nblocks, cudaStream_t s);

template <typename T>
cudaError_t launch_adj(const AdjArgs<T> &a, int tile, cudaStream_t s);

int adj_num_tiles();
int adj_blocks(int tile, int zchunk, int nx, int ny, int nz);
// Tile 3: vector adjoint (nx % (16/sizeof(T)) == 0), tile W x H cells, persistent grid.
bool adj_tile_is_vec(int tile);
void adj_vec_tile_dims(int esize, int *bw, int *bh);
template <typename T>
cudaError_t adj_vec_resident(int *resident);

// Record a message for cdi_last_error_string() and return code (cdi_api.cu).
int set_error(int code, const char *fmt, ...);

__host__ __device__ inline int wrapi(int a, int n)
{
    int r = a % n;
    return r < 0 ? r + n : r;
}

// Device status words of a grid or batch (4 x 32 bits, cleared when read):
//   [0] flags: bit 0 a bounded device wait gave up; bit 1 a checked build found
//       an index out of range;
//   [1] number of out-of-range indices found (checked builds);
//   [2] the last such index (low 32 bits), [3] the limit it was checked against.
constexpr int kStatusWords = 4;

// Checked builds (-DCDI_CHECKED): CDI_CHK(i, n, status) tests an index a kernel
// derived for a global access -- an in-plane offset against the plane, a plane
// index against the box -- and, if it lies outside [0, n), records it in the
// status words and returns 0 so that the access stays inside the array.  In
// other builds it is the index itself.
#ifdef CDI_CHECKED
__device__ __forceinline__ long long chk_index(long long i, long long n, unsigned *status)
{
    if (i >= 0 && i < n) return i;
    if (status) {
        atomicOr(status, 2u);
        atomicAdd(status + 1, 1u);
        atomicExch(status + 2, (unsigned)i);
        atomicExch(status + 3, (unsigned)n);
    }
    return 0;
}
#define CDI_CHK(i, n, status) ::cdi::chk_index((i), (n), (status))
#else
#define CDI_CHK(i, n, status) (i)
#endif

}  // namespace cdi
