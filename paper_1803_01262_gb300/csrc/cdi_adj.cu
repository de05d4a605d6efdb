// Discrete adjoint of one explicit CDI step (reverse mode through the five
// steps of Section 2.2), lam_k = (d phi^{k+1}/d phi^k)^T lam_{k+1}, for sm_103a.
//
// In gather form, for cell c with faces f = c +- 1/2 e_d:
//   Fbar_f      = (dt/dx) (lam'_R - lam'_L)
//   sbar_d(c)   = (gamma dt / 2dx) (lam'_{c+e_d} - lam'_{c-e_d})
//   nbar(c)     = sbar(c) phi_c (1 - phi_c)
//   gbar(c)     = (nbar - n (n . nbar)) / |g|         (0 where g = 0)
//   phibar_c    = sum_d [ Fbar_{c+1/2}(vs u_{c+1/2}/2 + gamma eps/dx)
//                       + Fbar_{c-1/2}(vs u_{c-1/2}/2 - gamma eps/dx) ]
//               + (1 - 2 phi_c) (sbar(c) . n_c)
//               + sum_d ( gbar_d(c - e_d) - gbar_d(c + e_d) )
//   lam_c       = lam'_c + phibar_c
//   ubar_{c+1/2} += Fbar_{c+1/2} vs (phi_c + phi_{c+e_d}) / 2     (optional)
// The structure mirrors the scalar forward body: phi and lam' planes (halo 2)
// and the face velocities (u from x0-1, v from y0-1, w) are staged by
// element-wise cp.async into shared rings PF_A planes ahead of use (phi and
// lam' plane j+2 travel with velocity plane j in one commit group); gbar_x /
// gbar_y of a plane go to a double-buffered shared array (written one plane
// ahead), gbar_z and the z-face term are carried in registers; one barrier
// per plane.
#include "cdi_internal.cuh"
#include "cdi_async.cuh"

namespace cdi {

__device__ __forceinline__ float rsqrt_a(float q) { return rsqrtf(q); }
__device__ __forceinline__ double rsqrt_a(double q) { return rsqrt(q); }

constexpr int PF_A = 3;    // prefetch distance (planes)
constexpr int NSLOT_A = 8; // phi / lam' ring: power of two >= PF_A + 3 live planes
constexpr int NVS_A = 4;   // velocity ring: power of two >= PF_A + 1

template <typename T, int BX, int BY>
struct AdjSmem {
    static constexpr int PX = BX + 4, PY = BY + 4;
    static constexpr int NU = BY * (BX + 1), NV = (BY + 1) * BX, NW = BY * BX;
    static constexpr int VPL = NU + NV + NW;
    static constexpr size_t bytes = sizeof(T) * (2 * NSLOT_A * PY * PX + 2 * BY * (BX + 2) +
                                                 2 * (BY + 2) * BX + NVS_A * VPL);
};

template <typename T, int BX, int BY>
__global__ void __launch_bounds__(BX * BY)
adj_kernel(const AdjArgs<T> a)
{
    using S = AdjSmem<T, BX, BY>;
    constexpr int PX = BX + 4, PY = BY + 4, PLANE = PX * PY;
    constexpr int NT = BX * BY;
    constexpr int NLOAD = (PLANE + NT - 1) / NT;
    constexpr int NU = S::NU, NV = S::NV, NW = S::NW;
    constexpr int RU = (NU + NT - 1) / NT, RV = (NV + NT - 1) / NT, RW = (NW + NT - 1) / NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T(*sp)[PY][PX] = reinterpret_cast<T(*)[PY][PX]>(smem_raw);          // phi ring [NSLOT_A]
    T(*sl)[PY][PX] = sp + NSLOT_A;                                      // lam' ring [NSLOT_A]
    T(*gxs)[BY][BX + 2] = reinterpret_cast<T(*)[BY][BX + 2]>(sl + NSLOT_A);  // gbar_x [2]
    T(*gys)[BY + 2][BX] = reinterpret_cast<T(*)[BY + 2][BX]>(gxs + 2);       // gbar_y [2]
    T *const sv = reinterpret_cast<T *>(gys + 2);                            // velocities [NVS_A][VPL]

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
    // The block is BX x BY: lets the compiler drop the bound checks of full copy rounds.
    __builtin_assume(tx >= 0 && tx < BX && ty >= 0 && ty < BY);
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    const long long plane = (long long)nx * ny;
    const int z0 = blockIdx.z * a.zchunk;
    const int z1 = min(z0 + a.zchunk, nz);

    int loff[NLOAD];
#pragma unroll
    for (int r = 0; r < NLOAD; ++r) {
        const int e = tid + r * NT;
        const int ey = e / PX, ex = e - ey * PX;
        loff[r] = (e < PLANE) ? wrapi(y0 + ey - 2, ny) * nx + wrapi(x0 + ex - 2, nx) : 0;
    }
    int uoff[RU], voff[RV], woff[RW];
#pragma unroll
    for (int r = 0; r < RU; ++r) {
        const int e = tid + r * NT, ey = e / (BX + 1), ex = e - ey * (BX + 1);
        uoff[r] = (e < NU) ? wrapi(y0 + ey, ny) * nx + wrapi(x0 - 1 + ex, nx) : 0;
    }
#pragma unroll
    for (int r = 0; r < RV; ++r) {
        const int e = tid + r * NT, ey = e / BX, ex = e - ey * BX;
        voff[r] = (e < NV) ? wrapi(y0 - 1 + ey, ny) * nx + wrapi(x0 + ex, nx) : 0;
    }
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        const int e = tid + r * NT, ey = e / BX, ex = e - ey * BX;
        woff[r] = (e < NW) ? wrapi(y0 + ey, ny) * nx + wrapi(x0 + ex, nx) : 0;
    }
    const int gx = wrapi(x0 + tx, nx), gy = wrapi(y0 + ty, ny);
    const bool own = (x0 + tx < nx) && (y0 + ty < ny);
    const int oc = gy * nx + gx;

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

    const T c_adv = a.c.c_adv, c_dif = a.c.c_dif, c_upd = a.c.c_upd, c_sb = a.c_shp_adj;
    const T c_vel = a.c_vel;
    const bool want_vel = a.gu != nullptr;

    // Stage phi and lam' plane z (ring slot z & (NSLOT_A-1)) from wrapped plane offset zo.
    auto issue_plane_at = [&](int z, long long zo) {
        T *dp = &sp[z & (NSLOT_A - 1)][0][0];
        T *dl = &sl[z & (NSLOT_A - 1)][0][0];
#pragma unroll
        for (int r = 0; r < NLOAD; ++r) {
            const int e = tid + r * NT;
            if (e < PLANE) {
                cp_async<sizeof(T)>(dp + e, a.phi + zo + loff[r]);
                cp_async<sizeof(T)>(dl + e, a.lam + zo + loff[r]);
            }
        }
    };
    auto issue_plane = [&](int z) { issue_plane_at(z, (long long)wrapi(z, nz) * plane); };
    // Stage velocity plane z (0 <= z < nz) from plane offset zo = z * plane.
    auto issue_vel_at = [&](int z, long long zo) {
        T *dst = sv + (z & (NVS_A - 1)) * S::VPL;
#pragma unroll
        for (int r = 0; r < RU; ++r) {
            const int e = tid + r * NT;
            if (e < NU) cp_async<sizeof(T)>(dst + e, a.u + zo + uoff[r]);
        }
#pragma unroll
        for (int r = 0; r < RV; ++r) {
            const int e = tid + r * NT;
            if (e < NV) cp_async<sizeof(T)>(dst + NU + e, a.v + zo + voff[r]);
        }
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            const int e = tid + r * NT;
            if (e < NW) cp_async<sizeof(T)>(dst + NU + NV + e, a.w + zo + woff[r]);
        }
    };
    auto issue_vel = [&](int z) { issue_vel_at(z, (long long)z * plane); };

    // gbar (3-vector) and the local term (1 - 2 phi)(sbar . n) at cell (lx, ly) of plane z.
    // The projection (I - n n^T) sbar is formed as n x (sbar x n), which is
    // exactly zero when sbar and n lie along one axis (the 1D case) and avoids
    // the cancellation of sbar - n (n . sbar) when |n| is off 1 by rounding.
    auto gbar = [&](int z, int lx, int ly, T &b0, T &b1, T &b2, T &tloc) {
        const int X = lx + 2, Y = ly + 2;
        const int m = z & (NSLOT_A - 1), mm = (z - 1) & (NSLOT_A - 1), mp = (z + 1) & (NSLOT_A - 1);
        const T p = sp[m][Y][X];
        const T g0 = sp[m][Y][X + 1] - sp[m][Y][X - 1];
        const T g1 = sp[m][Y + 1][X] - sp[m][Y - 1][X];
        const T g2 = sp[mp][Y][X] - sp[mm][Y][X];
        const T q = g0 * g0 + g1 * g1 + g2 * g2;
        const T inv = q > T(0) ? rsqrt_a(q) : T(0);
        const T sb0 = c_sb * (sl[m][Y][X + 1] - sl[m][Y][X - 1]);
        const T sb1 = c_sb * (sl[m][Y + 1][X] - sl[m][Y - 1][X]);
        const T sb2 = c_sb * (sl[mp][Y][X] - sl[mm][Y][X]);
        const T n0 = g0 * inv, n1 = g1 * inv, n2 = g2 * inv;
        tloc = (T(1) - T(2) * p) * (sb0 * n0 + sb1 * n1 + sb2 * n2);
        // c = sbar x n ; d = n x c = sbar - n (n . sbar) for a unit n
        const T c0 = sb1 * n2 - sb2 * n1;
        const T c1 = sb2 * n0 - sb0 * n2;
        const T c2 = sb0 * n1 - sb1 * n0;
        const T d0 = n1 * c2 - n2 * c1;
        const T d1 = n2 * c0 - n0 * c2;
        const T d2 = n0 * c1 - n1 * c0;
        // nbar = sbar p (1 - p);  gbar = (nbar - n (n . nbar)) / |g| = p (1 - p) d / |g|
        const T wgt = p * (T(1) - p) * inv;
        b0 = wgt * d0;
        b1 = wgt * d1;
        b2 = wgt * d2;
    };
    auto gbar_plane = [&](int z, T &gzc, T &tc) {
        T b0, b1;
        gbar(z, tx, ty, b0, b1, gzc, tc);
        gxs[z & 1][ty][tx + 1] = b0;
        gys[z & 1][ty + 1][tx] = b1;
        if (rkind) {
            T r0, r1, r2, rt;
            gbar(z, rx, ry, r0, r1, r2, rt);
            if (rkind == 1) gys[z & 1][ry + 1][rx] = r1;
            else gxs[z & 1][ry][rx + 1] = r0;
        }
    };

    // Commit groups: planes z0-2 .. z0+1; then PF_A prologue groups, the d-th
    // with planes z0+2+d and velocity plane z0+d; then one group per iteration j
    // with plane j+2+PF_A and velocity plane j+PF_A.  Waiting at iteration k
    // until at most PF_A-1 groups are pending lands plane k+2 and velocity k.
    issue_plane(z0 - 2);
    issue_plane(z0 - 1);
    issue_plane(z0);
    issue_plane(z0 + 1);
    cp_async_commit();
#pragma unroll
    for (int d = 0; d < PF_A; ++d) {
        if (z0 + 2 + d <= z1 + 1) issue_plane(z0 + 2 + d);
        if (z0 + d < z1) issue_vel(z0 + d);
        cp_async_commit();
    }
    const T wlo = __ldg(a.w + (long long)wrapi(z0 - 1, nz) * plane + oc);
    cp_async_wait<PF_A>();
    __syncthreads();
    T gz_m, gz_c, t_c;
    {
        T d0, d1, dt_;
        gbar(z0 - 1, tx, ty, d0, d1, gz_m, dt_);
    }
    gbar_plane(z0, gz_c, t_c);
    T Tzm;
    {
        const T Fb = c_upd * (sl[z0 & (NSLOT_A - 1)][ty + 2][tx + 2] - sl[(z0 - 1) & (NSLOT_A - 1)][ty + 2][tx + 2]);
        Tzm = Fb * (c_adv * wlo - c_dif);
    }

    // Wrapped offset of the plane issued next (k+2+PF_A) and of the next
    // velocity plane (k+PF_A), advanced by one plane per iteration.
    int zq = wrapi(z0 + 2 + PF_A, nz);
    long long oq = (long long)zq * plane, ov = (long long)(z0 + PF_A) * plane;
    for (int k = z0; k < z1; ++k) {
        // S1: plane k+2 and velocity plane k have landed; every thread has left
        // iteration k-1 (its reads of the slots written below, and of the gbar
        // buffer gbar_plane(k+1) writes).
        cp_async_wait<PF_A - 1>();
        __syncthreads();
        if (k + 2 + PF_A <= z1 + 1) issue_plane_at(k + 2 + PF_A, oq);
        if (k + PF_A < z1) issue_vel_at(k + PF_A, ov);
        cp_async_commit();
        if (++zq == nz) {
            zq = 0;
            oq = 0;
        } else {
            oq += plane;
        }
        ov += plane;

        T gz_p, t_p;
        gbar_plane(k + 1, gz_p, t_p);  // buffer (k+1)&1; phase C reads buffer k&1
        const long long zb = (long long)k * plane;
        const int m = k & (NSLOT_A - 1), b = k & 1, mp = (k + 1) & (NSLOT_A - 1);
        const T *vel = sv + (k & (NVS_A - 1)) * S::VPL;
        const T uc = vel[ty * (BX + 1) + tx + 1], um = vel[ty * (BX + 1) + tx];
        const T vc = vel[NU + (ty + 1) * BX + tx], vm = vel[NU + ty * BX + tx];
        const T wc = vel[NU + NV + ty * BX + tx];
        const T lc = sl[m][ty + 2][tx + 2];
        const T Fxp = c_upd * (sl[m][ty + 2][tx + 3] - lc);
        const T Fxm = c_upd * (lc - sl[m][ty + 2][tx + 1]);
        const T Fyp = c_upd * (sl[m][ty + 3][tx + 2] - lc);
        const T Fym = c_upd * (lc - sl[m][ty + 1][tx + 2]);
        const T Fzp = c_upd * (sl[mp][ty + 2][tx + 2] - lc);
        T pb = Fxp * (c_adv * uc + c_dif) + Fxm * (c_adv * um - c_dif);
        pb += Fyp * (c_adv * vc + c_dif) + Fym * (c_adv * vm - c_dif);
        pb += Fzp * (c_adv * wc + c_dif) + Tzm;
        pb += t_c;
        pb += (gxs[b][ty][tx] - gxs[b][ty][tx + 2]) + (gys[b][ty][tx] - gys[b][ty + 2][tx]) +
              (gz_m - gz_p);
        if (own) {
            a.out[zb + oc] = lc + pb;
            if (want_vel) {
                const T pc = sp[m][ty + 2][tx + 2];
                a.gu[zb + oc] += Fxp * c_vel * (pc + sp[m][ty + 2][tx + 3]);
                a.gv[zb + oc] += Fyp * c_vel * (pc + sp[m][ty + 3][tx + 2]);
                a.gw[zb + oc] += Fzp * c_vel * (pc + sp[mp][ty + 2][tx + 2]);
            }
        }
        Tzm = Fzp * (c_adv * wc - c_dif);
        gz_m = gz_c;
        gz_c = gz_p;
        t_c = t_p;
    }
    cp_async_wait<0>();
}

struct TileDimA { int bx, by; };
static const TileDimA kATiles[] = {{32, 8}, {32, 16}, {32, 4}};
static const int kNumATiles = sizeof(kATiles) / sizeof(kATiles[0]);

int adj_num_tiles() { return kNumATiles; }

int adj_blocks(int tile, int zchunk, int nx, int ny, int nz)
{
    const TileDimA t = kATiles[tile];
    return ((nx + t.bx - 1) / t.bx) * ((ny + t.by - 1) / t.by) * ((nz + zchunk - 1) / zchunk);
}

template <typename T, int BX, int BY>
static cudaError_t launch_adj_t(const AdjArgs<T> &a, cudaStream_t s)
{
    const size_t smem = AdjSmem<T, BX, BY>::bytes;
    static bool attr_set = false;  // per instantiation; idempotent if raced
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(adj_kernel<T, BX, BY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid((a.nx + BX - 1) / BX, (a.ny + BY - 1) / BY, (a.nz + a.zchunk - 1) / a.zchunk);
    dim3 block(BX, BY);
    adj_kernel<T, BX, BY><<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj(const AdjArgs<T> &a, int tile, cudaStream_t s)
{
    switch (tile) {
    case 0: return launch_adj_t<T, 32, 8>(a, s);
    case 1: return launch_adj_t<T, 32, 16>(a, s);
    case 2: return launch_adj_t<T, 32, 4>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_adj<float>(const AdjArgs<float> &, int, cudaStream_t);
template cudaError_t launch_adj<double>(const AdjArgs<double> &, int, cudaStream_t);

}  // namespace cdi
