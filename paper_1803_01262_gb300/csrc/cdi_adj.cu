// Discrete adjoint of one explicit CDI step (reverse mode through the five
// steps of Section 2.2), lam_k = (d phi^{k+1}/d phi^k)^T lam_{k+1}, for sm_103a.
//
// In gather form, for cell c with faces f = c +- 1/2 e_d:
//   Fbar_f      = (dt/dx) (lam'_R - lam'_L)
//   sbar_d(c)   = (gamma dt / 2dx) (lam'_{c+e_d} - lam'_{c-e_d})
//   nbar(c)     = sbar(c) phi_c (1 - phi_c)
//   gbar(c)     = (nbar - n (n . nbar)) / m           (0 where g = 0)
// with the normal n = g / m, m = sqrt(|g|^2 + delta^2), delta = 8 machine
// epsilons of T.  In every interface cell |g| >> delta and this is the
// derivative of the forward step.  In the flat bulk next to phi = 1 (or 0)
// neighbours differ by a unit or two in the last place, the unit normal is
// rounding noise, and its derivative p (1 - p)/|g| (a few, there) makes the
// linearised sharpening anti-diffusive: over a 200-step backward recursion
// that noise grows by many orders of magnitude.  The floor caps the
// derivative at p (1 - p)/delta.
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
#include "cdi_fwd_common.cuh"

namespace cdi {

__device__ __forceinline__ float rsqrt_a(float q) { return rsqrtf(q); }
__device__ __forceinline__ double rsqrt_a(double q) { return rsqrt(q); }

// delta^2 = (8 machine epsilons)^2: (2^-20)^2 in FP32, (2^-49)^2 in FP64.
template <typename T> struct AdjFloor;
template <> struct AdjFloor<float> {
    __device__ __forceinline__ static float sq() { return 9.094947017729282e-13f; }
};
template <> struct AdjFloor<double> {
    __device__ __forceinline__ static double sq() { return 3.1554436208840472e-30; }
};

// 1/m, m = sqrt(|g|^2 + delta^2), or 0 where g = 0 (no normal there, so no
// derivative either).
template <typename T>
__device__ __forceinline__ T inv_norm(T g0, T g1, T g2)
{
    const T q = fma(g2, g2, fma(g1, g1, fma(g0, g0, AdjFloor<T>::sq())));
    const bool nz = (g0 != T(0)) | (g1 != T(0)) | (g2 != T(0));
    return nz ? rsqrt_a(q) : T(0);
}

// 1 - |n|^2 = delta^2 / m^2 for n = g / m: the part of sbar that the
// projection sbar - n (n . sbar) keeps along n when n is shorter than a unit
// vector.
template <typename T>
__device__ __forceinline__ T floor_part(T inv) { return AdjFloor<T>::sq() * inv * inv; }

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
        loff[r] = (e < PLANE) ? (int)CDI_CHK(wrapi(y0 + ey - 2, ny) * nx + wrapi(x0 + ex - 2, nx), plane, a.status) : 0;
    }
    int uoff[RU], voff[RV], woff[RW];
#pragma unroll
    for (int r = 0; r < RU; ++r) {
        const int e = tid + r * NT, ey = e / (BX + 1), ex = e - ey * (BX + 1);
        uoff[r] = (e < NU) ? (int)CDI_CHK(wrapi(y0 + ey, ny) * nx + wrapi(x0 - 1 + ex, nx), plane, a.status) : 0;
    }
#pragma unroll
    for (int r = 0; r < RV; ++r) {
        const int e = tid + r * NT, ey = e / BX, ex = e - ey * BX;
        voff[r] = (e < NV) ? (int)CDI_CHK(wrapi(y0 - 1 + ey, ny) * nx + wrapi(x0 + ex, nx), plane, a.status) : 0;
    }
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        const int e = tid + r * NT, ey = e / BX, ex = e - ey * BX;
        woff[r] = (e < NW) ? (int)CDI_CHK(wrapi(y0 + ey, ny) * nx + wrapi(x0 + ex, nx), plane, a.status) : 0;
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
        const T inv = inv_norm(g0, g1, g2);
        const T sb0 = c_sb * (sl[m][Y][X + 1] - sl[m][Y][X - 1]);
        const T sb1 = c_sb * (sl[m][Y + 1][X] - sl[m][Y - 1][X]);
        const T sb2 = c_sb * (sl[mp][Y][X] - sl[mm][Y][X]);
        const T n0 = g0 * inv, n1 = g1 * inv, n2 = g2 * inv;
        tloc = (T(1) - T(2) * p) * (sb0 * n0 + sb1 * n1 + sb2 * n2);
        // c = sbar x n ; d = n x c + sbar (1 - |n|^2) = sbar - n (n . sbar).  The
        // cross-product form keeps d exactly 0 for sbar parallel to n (1D).
        const T c0 = sb1 * n2 - sb2 * n1;
        const T c1 = sb2 * n0 - sb0 * n2;
        const T c2 = sb0 * n1 - sb1 * n0;
        const T fl = floor_part(inv);
        const T d0 = fma(sb0, fl, n1 * c2 - n2 * c1);
        const T d1 = fma(sb1, fl, n2 * c0 - n0 * c2);
        const T d2 = fma(sb2, fl, n0 * c1 - n1 * c0);
        // nbar = sbar p (1 - p);  gbar = (nbar - n (n . nbar)) / m = p (1 - p) d / m
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
        const long long zb = (long long)CDI_CHK(k, nz, a.status) * plane;
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

// ===========================================================================
// Vector adjoint (nx a multiple of 16 / sizeof(T), 16-byte aligned arrays):
// the structure of the vector forward kernel.  Each of the TX x TY own threads
// holds a 16-byte vector of VX x-cells; two extra warps compute gbar on the
// one-cell ring (gbar_y for the rows y0-1 and y0+H, gbar_x for the columns
// x0-1 and x0+W) and issue every 16-byte copy of phi, lam' (5-slot rings, halo
// 2 in y, one vector in x) and u, v, w (3-slot ring) two planes ahead of use.
// Units are (z chunk, tile) pairs taken round-robin in chunk-major order by a
// persistent grid; one barrier per plane (gbar_x / gbar_y double-buffered,
// written one plane ahead; gbar_z, the local term and the z-face term carried).

template <typename T, int TX, int TY>
struct AdjVecCfg {
    static constexpr int VX = 16 / sizeof(T);
    static constexpr int W = TX * VX, H = TY;
    static constexpr int NOWN = TX * TY;
    static constexpr int NT = NOWN + 64;     // + one y-ring warp + one x-ring warp
    static constexpr int PP = W + 2 * VX;    // row pitch of phi / lam': x0-VX .. x0+W+VX-1
    static constexpr int PR = H + 4;         // rows y0-2 .. y0+H+1
    static constexpr int PHI = PR * PP;
    static constexpr int UP = W + VX;        // u row pitch: x0-VX .. x0+W-1
    static constexpr int USZ = H * UP;
    static constexpr int VSZ = (H + 1) * W;  // v rows: y0-1 .. y0+H-1
    static constexpr int WSZ = H * W;
    static constexpr int VEL = USZ + VSZ + WSZ;
    static constexpr int SXP = W + 2 * VX;   // gbar_x pitch: x0-1 at VX-1, x0+W at VX+W
    static constexpr int SXS = H * SXP;
    static constexpr int SYS = (H + 2) * W;  // gbar_y rows: y0-1 .. y0+H
    static constexpr int NSP = 5, NSV = 3;
    static constexpr int CPHI = PHI / VX, CU = USZ / VX, CV = VSZ / VX, CW = WSZ / VX;
    static constexpr size_t bytes =
        sizeof(T) * (size_t)(2 * NSP * PHI + NSV * VEL + 2 * SXS + 2 * SYS);
    static_assert(2 * TX <= 32 && 2 * TY <= 32, "ring warps hold 2*TX groups and 2*TY cells");
};

// Three FP32 blocks per SM (113 registers) measured 8% faster than two; FP64
// keeps two (it would spill at three).
// VEL: the velocity gradients are accumulated (a.gu, a.gv, a.gw not null); the
// instantiation without them keeps no face differences live for them.
template <typename T, int TX, int TY, bool VEL>
__global__ void __launch_bounds__(AdjVecCfg<T, TX, TY>::NT, sizeof(T) == 4 ? 3 : 2)
adj_vec_kernel(const AdjArgs<T> a, const int nchunks)
{
    using C = AdjVecCfg<T, TX, TY>;
    using VV = V16<T>;
    constexpr int VX = C::VX, W = C::W, H = C::H, PP = C::PP, UP = C::UP, SXP = C::SXP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *const sphi = reinterpret_cast<T *>(smem_raw);      // [NSP][PHI]
    T *const slam = sphi + C::NSP * C::PHI;                // [NSP][PHI]
    T *const svel = slam + C::NSP * C::PHI;                // [NSV][VEL] = u | v | w
    T *const sgx = svel + C::NSV * C::VEL;                 // [2][SXS]
    T *const sgy = sgx + 2 * C::SXS;                       // [2][SYS]

    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long plane = (long long)nx * ny;
    const int tiles_x = (nx + W - 1) / W;
    const int ntiles = tiles_x * ((ny + H - 1) / H);
    const T c_adv = a.c.c_adv, c_dif = a.c.c_dif, c_upd = a.c.c_upd, c_sb = a.c_shp_adj;
    const T c_vel = a.c_vel;
    constexpr bool want_vel = VEL;

    const bool is_own = tid < C::NOWN;
    const int tx = tid % TX, ty = tid / TX;
    const int rr = tid - C::NOWN;  // 0..63 for ring threads
    const bool is_yring = !is_own && rr < 32 && rr < 2 * TX;
    const bool is_xring = !is_own && rr >= 32 && rr - 32 < 2 * TY;
    const int ry_row = (rr < TX) ? -1 : H, ry_col = rr % TX;  // y-ring group
    const int rx_row = (rr - 32) % TY;                         // x-ring cell
    const int rx_col = ((rr - 32) < TY) ? -1 : W;

    // gbar and the local term (1 - 2 phi)(sbar . n) of the VX cells of group
    // (gc, ly) at the plane of slot Pm (Pmm / Pmp: planes below / above; the
    // same slots of the lam' ring).  n = g / m (0 where g = 0).  The projection
    // is evaluated as sbar - n (n . sbar), which equals the per-cell kernel's
    // n x (sbar x n) + sbar delta^2/m^2 since |n|^2 + delta^2/m^2 = 1: three FMAs
    // on the already formed n . sbar instead of two cross products (112.0 ->
    // 105.6 us per FP32 step at 256^3).  It rounds differently: where sbar is
    // parallel to n (1D) the result is delta^2/m^2 sbar plus rounding of order
    // eps |sbar|, where the cross form gives that term alone.
    // lzn_in (nullable): lam' of the group at the plane below, already loaded; lc_out
    // (nullable): receives lam' of the group at this plane (an own thread's update
    // reads both again)
    auto gbar_group = [&](int sm, int smm, int smp, int gc, int ly, T *b0, T *b1, T *b2, T *tl,
                          const T *lzn_in = nullptr, T *lc_out = nullptr) {
        const int off = (ly + 2) * PP + VX + gc * VX;
        const T *Pm = sphi + sm * C::PHI, *Pmm = sphi + smm * C::PHI, *Pmp = sphi + smp * C::PHI;
        const T *Lm = slam + sm * C::PHI, *Lmm = slam + smm * C::PHI, *Lmp = slam + smp * C::PHI;
        T c[VX], yn[VX], yp[VX], zn[VX], zp[VX];
        VV::ld(c, Pm + off);
        VV::ld(yn, Pm + off - PP);
        VV::ld(yp, Pm + off + PP);
        VV::ld(zn, Pmm + off);
        VV::ld(zp, Pmp + off);
        const T L = Pm[off - 1], R = Pm[off + VX];
        T lc[VX], lyn[VX], lyp[VX], lzn[VX], lzp[VX];
        VV::ld(lc, Lm + off);
        VV::ld(lyn, Lm + off - PP);
        VV::ld(lyp, Lm + off + PP);
        if (lzn_in) {
#pragma unroll
            for (int i = 0; i < VX; ++i) lzn[i] = lzn_in[i];
        } else {
            VV::ld(lzn, Lmm + off);
        }
        VV::ld(lzp, Lmp + off);
        const T lL = Lm[off - 1], lR = Lm[off + VX];
        if (lc_out) {
#pragma unroll
            for (int i = 0; i < VX; ++i) lc_out[i] = lc[i];
        }
#pragma unroll
        for (int i = 0; i < VX; ++i) {
            const T g0 = (i + 1 < VX ? c[i + 1] : R) - (i > 0 ? c[i - 1] : L);
            const T g1 = yp[i] - yn[i];
            const T g2 = zp[i] - zn[i];
            const T inv = inv_norm(g0, g1, g2);
            const T sb0 = c_sb * ((i + 1 < VX ? lc[i + 1] : lR) - (i > 0 ? lc[i - 1] : lL));
            const T sb1 = c_sb * (lyp[i] - lyn[i]);
            const T sb2 = c_sb * (lzp[i] - lzn[i]);
            const T n0 = g0 * inv, n1 = g1 * inv, n2 = g2 * inv;
            const T p = c[i];
            const T ns = sb0 * n0 + sb1 * n1 + sb2 * n2;
            tl[i] = (T(1) - T(2) * p) * ns;
            // the projection sbar - n (n . sbar) (|n|^2 + delta^2 / m^2 = 1), in three FMAs
            const T wgt = p * (T(1) - p) * inv;
            b0[i] = wgt * fma(-n0, ns, sb0);
            b1[i] = wgt * fma(-n1, ns, sb1);
            b2[i] = wgt * fma(-n2, ns, sb2);
        }
    };
    // gbar_x only, of cell (lx, ly) (the x-ring).
    auto gbar_x_cell = [&](int sm, int smm, int smp, int lx, int ly) {
        const int off = (ly + 2) * PP + VX + lx;
        const T *Pm = sphi + sm * C::PHI, *Pmm = sphi + smm * C::PHI, *Pmp = sphi + smp * C::PHI;
        const T *Lm = slam + sm * C::PHI, *Lmm = slam + smm * C::PHI, *Lmp = slam + smp * C::PHI;
        const T p = Pm[off];
        const T g0 = Pm[off + 1] - Pm[off - 1];
        const T g1 = Pm[off + PP] - Pm[off - PP];
        const T g2 = Pmp[off] - Pmm[off];
        const T inv = inv_norm(g0, g1, g2);
        const T sb0 = c_sb * (Lm[off + 1] - Lm[off - 1]);
        const T sb1 = c_sb * (Lm[off + PP] - Lm[off - PP]);
        const T sb2 = c_sb * (Lmp[off] - Lmm[off]);
        const T n0 = g0 * inv, n1 = g1 * inv, n2 = g2 * inv;
        const T ns = sb0 * n0 + sb1 * n1 + sb2 * n2;
        return p * (T(1) - p) * inv * fma(-n0, ns, sb0);
    };

    bool dep_waited = false;  // the previous grid on the stream has completed
    UnitIter<W, H> units(ntiles, nz, nchunks);
    Unit un;
    while (units.next(un, ntiles, tiles_x, nz, nchunks)) {
        const int x0 = un.x0, y0 = un.y0, z0 = un.z0, z1 = un.z1;

        // The 64 ring threads issue every 16-byte copy; global in-plane
        // offsets of their chunks (phi and lam' share one layout):
        constexpr int NC = 64;
        constexpr int RPHI = (C::CPHI + NC - 1) / NC, RU = (C::CU + NC - 1) / NC;
        constexpr int RV = (C::CV + NC - 1) / NC, RW = (C::CW + NC - 1) / NC;
        const int ct = tid - C::NOWN;
        int gphi[RPHI], gu_[RU], gv_[RV], gw_[RW];
        if (!is_own) {
#pragma unroll
            for (int r = 0; r < RPHI; ++r) {
                const int e = ct + r * NC, row = e / (PP / VX), col = e - row * (PP / VX);
                gphi[r] = (int)CDI_CHK(wrapi(y0 - 2 + row, ny) * nx + wrapi(x0 - VX + col * VX, nx), plane - VX + 1, a.status);
            }
#pragma unroll
            for (int r = 0; r < RU; ++r) {
                const int e = ct + r * NC, row = e / (UP / VX), col = e - row * (UP / VX);
                gu_[r] = (int)CDI_CHK(wrapi(y0 + row, ny) * nx + wrapi(x0 - VX + col * VX, nx), plane - VX + 1, a.status);
            }
#pragma unroll
            for (int r = 0; r < RV; ++r) {
                const int e = ct + r * NC, row = e / (W / VX), col = e - row * (W / VX);
                gv_[r] = (int)CDI_CHK(wrapi(y0 - 1 + row, ny) * nx + wrapi(x0 + col * VX, nx), plane - VX + 1, a.status);
            }
#pragma unroll
            for (int r = 0; r < RW; ++r) {
                const int e = ct + r * NC, row = e / (W / VX), col = e - row * (W / VX);
                gw_[r] = (int)CDI_CHK(wrapi(y0 + row, ny) * nx + wrapi(x0 + col * VX, nx), plane - VX + 1, a.status);
            }
        }
        auto issue_pl = [&](int z, int slot) {
            if (is_own) return;
            const long long zo = (long long)wrapi(z, nz) * plane;
            T *dp = sphi + slot * C::PHI;
            T *dl = slam + slot * C::PHI;
#pragma unroll
            for (int r = 0; r < RPHI; ++r) {
                const int e = ct + r * NC;
                if (e < C::CPHI) {
                    cp_async<16>(dp + e * VX, a.phi + zo + gphi[r]);
                    cp_async<16>(dl + e * VX, a.lam + zo + gphi[r]);
                }
            }
        };
        auto issue_vel = [&](int z, int slot) {
            if (is_own) return;
            const long long zo = (long long)z * plane;
            T *dst = svel + slot * C::VEL;
#pragma unroll
            for (int r = 0; r < RU; ++r) {
                const int e = ct + r * NC;
                if (e < C::CU) cp_async<16>(dst + e * VX, a.u + zo + gu_[r]);
            }
#pragma unroll
            for (int r = 0; r < RV; ++r) {
                const int e = ct + r * NC;
                if (e < C::CV) cp_async<16>(dst + C::USZ + e * VX, a.v + zo + gv_[r]);
            }
#pragma unroll
            for (int r = 0; r < RW; ++r) {
                const int e = ct + r * NC;
                if (e < C::CW) cp_async<16>(dst + C::USZ + C::VSZ + e * VX, a.w + zo + gw_[r]);
            }
        };

        // Ring slot of plane z: (z - z0 + 2) mod 5; velocity slot: (z - z0) mod 3.
        // The face velocities are staged (and w below plane z0 loaded) before
        // waiting for the previous grid on the stream; phi, lam' and the
        // accumulated velocity gradients, which it may write, only after.
        __syncthreads();  // the previous unit's readers are done with every slot
        issue_vel(z0, 0);
        const int own_x = x0 + tx * VX, own_y = y0 + ty;
        const bool writes = is_own && own_x < nx && own_y < ny;
        const long long own_off = (long long)wrapi(own_y, ny) * nx + wrapi(own_x, nx);
        T wlo[VX];  // w on the face below plane z0 (own cells)
        if (is_own) {
            const T *src = a.w + (long long)wrapi(z0 - 1, nz) * plane + own_off;
#pragma unroll
            for (int i = 0; i < VX; ++i) wlo[i] = __ldg(src + i);
        }
        if (!dep_waited) {
            grid_dep_wait();
            dep_waited = true;
        }
        for (int d = 0; d < 5; ++d) issue_pl(z0 - 2 + d, d);  // planes z0-2 .. z0+2
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();

        // Prologue: gbar_z at plane z0-1 (own); gbar, local term at z0 (own + ring);
        // z-face term at z0-1/2.
        T gzm[VX], gzc[VX], tc[VX], Tzm[VX];
        if (is_own) {
            T d0[VX], d1[VX], dt[VX], b0[VX], b1[VX];
            gbar_group(1, 0, 2, tx, ty, d0, d1, gzm, dt);
            gbar_group(2, 1, 3, tx, ty, b0, b1, gzc, tc);
            VV::st(sgx + (z0 & 1) * C::SXS + ty * SXP + VX + tx * VX, b0);
            VV::st(sgy + (z0 & 1) * C::SYS + (ty + 1) * W + tx * VX, b1);
            T lm[VX], lcv[VX];
            const int po = (ty + 2) * PP + VX + tx * VX;
            VV::ld(lm, slam + 1 * C::PHI + po);
            VV::ld(lcv, slam + 2 * C::PHI + po);
#pragma unroll
            for (int i = 0; i < VX; ++i) Tzm[i] = c_upd * (lcv[i] - lm[i]) * (c_adv * wlo[i] - c_dif);
        } else if (is_yring) {
            T b0[VX], b1[VX], b2[VX], t_[VX];
            gbar_group(2, 1, 3, ry_col, ry_row, b0, b1, b2, t_);
            VV::st(sgy + (z0 & 1) * C::SYS + (ry_row + 1) * W + ry_col * VX, b1);
        } else if (is_xring) {
            sgx[(z0 & 1) * C::SXS + rx_row * SXP + VX + rx_col] = gbar_x_cell(2, 1, 3, rx_col, rx_row);
        }
        // Plane z0+3 reuses the slot of plane z0-2, which the prologue just read.
        __syncthreads();
        if (z0 + 3 <= z1 + 1) issue_pl(z0 + 3, 0);
        if (z0 + 1 < z1) issue_vel(z0 + 1, 1);
        cp_async_commit();

        int pk = 2;  // ring slot of plane k
        int vk = 0;  // velocity slot of plane k
        for (int k = z0; k < z1; ++k) {
            const int pk1 = pk == 4 ? 0 : pk + 1;
            const int pk2 = pk1 == 4 ? 0 : pk1 + 1;
            const int pkm = pk == 0 ? 4 : pk - 1;   // also the slot of plane k+4
            const int vk2 = vk == 0 ? 2 : vk - 1;   // slot of plane k+2
            // S1: planes k+2 and the velocities of plane k have landed, and
            // every thread has left iteration k-1.
            cp_async_wait<1>();
            __syncthreads();
            if (k + 4 <= z1 + 1) issue_pl(k + 4, pkm);
            if (k + 2 < z1) issue_vel(k + 2, vk2);
            cp_async_commit();

            // B: gbar at plane k+1 (buffer (k+1)&1; phase C reads buffer k&1).  An own
            // thread runs B and C in one block, so that the compiler may overlap them.
            const int b1 = (k + 1) & 1;
            if (is_yring) {
                T b0[VX], bb1[VX], b2[VX], t_[VX];
                gbar_group(pk1, pk, pk2, ry_col, ry_row, b0, bb1, b2, t_);
                VV::st(sgy + b1 * C::SYS + (ry_row + 1) * W + ry_col * VX, bb1);
            } else if (is_xring) {
                sgx[b1 * C::SXS + rx_row * SXP + VX + rx_col] = gbar_x_cell(pk1, pk, pk2, rx_col, rx_row);
            }
            if (is_own) {
                const int po = (ty + 2) * PP + VX + tx * VX;
                T gzp[VX], tp[VX], lc[VX], lzp[VX];  // lam' of the own group at planes k, k+1
                VV::ld(lc, slam + pk * C::PHI + po);
                {
                    T b0[VX], bb1[VX];
                    gbar_group(pk1, pk, pk2, tx, ty, b0, bb1, gzp, tp, lc, lzp);
                    VV::st(sgx + b1 * C::SXS + ty * SXP + VX + tx * VX, b0);
                    VV::st(sgy + b1 * C::SYS + (ty + 1) * W + tx * VX, bb1);
                }

                // C: lam at plane k.
                const int b = k & 1;
                const T *Lk = slam + pk * C::PHI;
                T lyn[VX], lyp[VX];
                VV::ld(lyn, Lk + po - PP);
                VV::ld(lyp, Lk + po + PP);
                const T lL = Lk[po - 1], lR = Lk[po + VX];
                const T *gxr = sgx + b * C::SXS + ty * SXP + VX + tx * VX;
                const T *gyr = sgy + b * C::SYS + (ty + 1) * W + tx * VX;
                T gx[VX], gyn[VX], gyp[VX];
                VV::ld(gx, gxr);
                VV::ld(gyn, gyr - W);
                VV::ld(gyp, gyr + W);
                const T gxL = gxr[-1], gxR = gxr[VX];
                const T *vel = svel + vk * C::VEL;
                const T *ur = vel + ty * UP + VX + tx * VX;
                const T *vr = vel + C::USZ + (ty + 1) * W + tx * VX;
                const T *wr = vel + C::USZ + C::VSZ + ty * W + tx * VX;
                T uc[VX], vc[VX], vn[VX], wc[VX];
                VV::ld(uc, ur);
                VV::ld(vc, vr);
                VV::ld(vn, vr - W);
                VV::ld(wc, wr);
                const T uL = ur[-1];
                T o[VX], fxp[VX], fyp[VX], fzp[VX];
#pragma unroll
                for (int i = 0; i < VX; ++i) {
                    const T xl = i > 0 ? lc[i - 1] : lL, xr = i + 1 < VX ? lc[i + 1] : lR;
                    const T ul = i > 0 ? uc[i - 1] : uL;
                    const T Fxp = c_upd * (xr - lc[i]);
                    const T Fxm = c_upd * (lc[i] - xl);
                    const T Fyp = c_upd * (lyp[i] - lc[i]);
                    const T Fym = c_upd * (lc[i] - lyn[i]);
                    const T Fzp = c_upd * (lzp[i] - lc[i]);
                    T pb = Fxp * (c_adv * uc[i] + c_dif) + Fxm * (c_adv * ul - c_dif);
                    pb += Fyp * (c_adv * vc[i] + c_dif) + Fym * (c_adv * vn[i] - c_dif);
                    pb += Fzp * (c_adv * wc[i] + c_dif) + Tzm[i];
                    pb += tc[i];
                    const T gl = i > 0 ? gx[i - 1] : gxL, gr = i + 1 < VX ? gx[i + 1] : gxR;
                    pb += (gl - gr) + (gyn[i] - gyp[i]) + (gzm[i] - gzp[i]);
                    o[i] = lc[i] + pb;
                    fxp[i] = Fxp;
                    fyp[i] = Fyp;
                    fzp[i] = Fzp;
                    Tzm[i] = Fzp * (c_adv * wc[i] - c_dif);
                    gzm[i] = gzc[i];
                    gzc[i] = gzp[i];
                    tc[i] = tp[i];
                }
                if (writes) {
                    const long long ko = (long long)CDI_CHK(k, nz, a.status) * plane +
                                         CDI_CHK(own_off, plane - VX + 1, a.status);
                    VV::st(a.out + ko, o);
                    if (want_vel) {
                        const T *Pk = sphi + pk * C::PHI, *Pk1 = sphi + pk1 * C::PHI;
                        T pc[VX], pyp[VX], pzp[VX], gu0[VX], gv0[VX], gw0[VX];
                        VV::ld(pc, Pk + po);
                        VV::ld(pyp, Pk + po + PP);
                        VV::ld(pzp, Pk1 + po);
                        const T pR = Pk[po + VX];
                        VV::ld(gu0, a.gu + ko);
                        VV::ld(gv0, a.gv + ko);
                        VV::ld(gw0, a.gw + ko);
#pragma unroll
                        for (int i = 0; i < VX; ++i) {
                            const T pxr = i + 1 < VX ? pc[i + 1] : pR;
                            gu0[i] += fxp[i] * c_vel * (pc[i] + pxr);
                            gv0[i] += fyp[i] * c_vel * (pc[i] + pyp[i]);
                            gw0[i] += fzp[i] * c_vel * (pc[i] + pzp[i]);
                        }
                        VV::st(a.gu + ko, gu0);
                        VV::st(a.gv + ko, gv0);
                        VV::st(a.gw + ko, gw0);
                    }
                }
            }
            pk = pk1;
            vk = vk == 2 ? 0 : vk + 1;
        }
        cp_async_wait<0>();
    }
    if (!dep_waited) grid_dep_wait();
    grid_dep_launch();
}

// Adjoint tiles: 0..2 one cell per thread (32x8, 32x16, 32x4 cells, one block per tile
// and z chunk); 3 the vector kernel (16x8 threads, persistent grid).
struct TileDimA { int bx, by; };
static const TileDimA kATiles[] = {{32, 8}, {32, 16}, {32, 4}};
static const int kNumATiles = 4;

int adj_num_tiles() { return kNumATiles; }

bool adj_tile_is_vec(int tile) { return tile == 3; }

int adj_blocks(int tile, int zchunk, int nx, int ny, int nz)
{
    if (adj_tile_is_vec(tile)) return 0;  // persistent grid, no scratch
    const TileDimA t = kATiles[tile];
    return ((nx + t.bx - 1) / t.bx) * ((ny + t.by - 1) / t.by) * ((nz + zchunk - 1) / zchunk);
}

void adj_vec_tile_dims(int esize, int *bw, int *bh)
{
    *bw = 16 * (16 / esize);
    *bh = 8;
}

template <typename T>
cudaError_t adj_vec_resident(int *resident)
{
    using C = AdjVecCfg<T, 16, 8>;
    cudaError_t e = cudaFuncSetAttribute(adj_vec_kernel<T, 16, 8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(adj_vec_kernel<T, 16, 8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::bytes);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(resident, adj_vec_kernel<T, 16, 8, false>, C::NT, C::bytes);
}
template cudaError_t adj_vec_resident<float>(int *);
template cudaError_t adj_vec_resident<double>(int *);

// Persistent grid of the vector adjoint: every resident block, at most one per unit.
template <typename T>
static cudaError_t launch_adj_vec(const AdjArgs<T> &a, cudaStream_t s)
{
    using C = AdjVecCfg<T, 16, 8>;
    int resident = 0, dev = 0, sms = 0;
    cudaError_t e;
    if ((e = adj_vec_resident<T>(&resident)) != cudaSuccess) return e;
    if (resident < 1) return cudaErrorInvalidConfiguration;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    // zchunk < 0: balanced shares of the tile-planes (UnitIter; -2 rotated); else z chunks
    const long long tiles = (long long)((a.nx + C::W - 1) / C::W) * ((a.ny + C::H - 1) / C::H);
    int nchunks;
    long long units;
    if (a.zchunk < 0) {
        nchunks = a.zchunk == -2 ? -2 : -1;
        units = tiles * a.nz;
    } else {
        nchunks = (a.nz + a.zchunk - 1) / a.zchunk;
        const int zc = (a.nz + nchunks - 1) / nchunks;
        units = tiles * ((a.nz + zc - 1) / zc);
    }
    long long nb = (long long)resident * sms;
    if (nb > units) nb = units;
    // programmatic stream serialisation: the launch may overlap the previous grid's
    // end (the kernel waits for it before touching anything it may write)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nb);
    cfg.blockDim = dim3(C::NT);
    cfg.dynamicSmemBytes = C::bytes;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (a.gu) return cudaLaunchKernelEx(&cfg, adj_vec_kernel<T, 16, 8, true>, a, nchunks);
    return cudaLaunchKernelEx(&cfg, adj_vec_kernel<T, 16, 8, false>, a, nchunks);
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
    case 3: return launch_adj_vec<T>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_adj<float>(const AdjArgs<float> &, int, cudaStream_t);
template cudaError_t launch_adj<double>(const AdjArgs<double> &, int, cudaStream_t);

}  // namespace cdi
