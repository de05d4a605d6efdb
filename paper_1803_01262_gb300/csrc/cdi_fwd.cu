// Fused explicit CDI step (Eq. 1 discretised as in Section 2.2; Eq. 11 in 1D,
// Eq. 18-22 in coefficient form) for sm_103a, plus the stand-alone
// reductions.  No tensor cores: the step is a memory-bound stencil.
//
// Per face between cells L and R along axis d:
//   F = c_adv u_f (phi_L + phi_R) - c_dif (phi_R - phi_L) + c_shp (s_L + s_R),
//   s = phi (1 - phi) g/|g|,  g_d = phi_{c+e_d} - phi_{c-e_d}  (s = 0 where g = 0),
//   phi'_c = phi_c - c_upd sum_d (F_{c+1/2} - F_{c-1/2}).
//
// Two kernels share one structure (a block owns an x-y tile and marches along
// z over a chunk of planes):
//   fwd_vec_kernel  -- each thread owns a 16-byte vector of x-cells (4 float
//                      or 2 double); phi and the three face-velocity planes
//                      are staged by 16-byte cp.async two planes ahead of use;
//                      two extra warps compute the sharpening ring (one cell
//                      beyond the tile in x and in y) so the normal phase stays
//                      balanced.  Needs nx % (16/sizeof(T)) == 0.
//   fwd_kernel      -- one cell per thread, element-wise cp.async for phi,
//                      register-prefetched velocities; any extents.
// Work units are (z chunk, tile) pairs taken round-robin in chunk-major
// order, so blocks resident together work on neighbouring tiles at the same
// planes and the halo rows they share are served from L2; or (balanced) each
// block takes an equal contiguous share of the tile-planes (UnitIter).
// Every block folds its outputs into mass / min / max / violation partials,
// finished by the last block (cdi_reduce.cuh).
// All indices wrap periodically; tiles may overhang the grid (ragged edges):
// overhanging cells are computed on wrapped data but never written.
#include "cdi_internal.cuh"
#include "cdi_reduce.cuh"
#include "cdi_async.cuh"
#include "cdi_fwd_common.cuh"
#include "cdi_fwd_scalar.cuh"

namespace cdi {

// ===========================================================================
// Vector kernel

template <typename T, int TX, int TY>
struct VecCfg {
    static constexpr int VX = 16 / sizeof(T);
    static constexpr int W = TX * VX, H = TY;
    static constexpr int NOWN = TX * TY;
    static constexpr int NT = NOWN + 64;     // + one y-ring warp + one x-ring warp
    static constexpr int PP = W + 2 * VX;    // phi row pitch: x0-VX .. x0+W+VX-1
    static constexpr int PR = H + 4;         // phi rows: y0-2 .. y0+H+1
    static constexpr int PHI = PR * PP;
    static constexpr int UP = W + VX;        // u row pitch: x0-VX .. x0+W-1
    static constexpr int USZ = H * UP;
    static constexpr int VSZ = (H + 1) * W;  // v rows: y0-1 .. y0+H-1
    static constexpr int WSZ = H * W;
    static constexpr int VEL = USZ + VSZ + WSZ;
    static constexpr int SXP = W + 2 * VX;   // s_x pitch: x0-1 at VX-1, x0+W at VX+W
    static constexpr int SXS = H * SXP;
    static constexpr int SYS = (H + 2) * W;  // s_y rows: y0-1 .. y0+H
    static constexpr int NSP = 5, NSV = 3;   // ring slots (phi, velocity)
    static constexpr int CPHI = PHI / VX, CU = USZ / VX, CV = VSZ / VX, CW = WSZ / VX;
    static constexpr int RPHI = (CPHI + NT - 1) / NT;
    static constexpr int RU = (CU + NT - 1) / NT, RV = (CV + NT - 1) / NT, RW = (CW + NT - 1) / NT;
    static constexpr size_t bytes = sizeof(T) * (size_t)(NSP * PHI + NSV * VEL + 2 * SXS + 2 * SYS);
    static_assert(2 * TX <= 32 && 2 * TY <= 32, "ring warps hold 2*TX groups and 2*TY cells");
};

// ZR: update only planes [a.z_lo, a.z_hi) (the z slabs of a pipelined host
// step); the full-box instantiations keep no range.
template <typename T, int TX, int TY, bool RK, bool ZR = false>
__global__ void __launch_bounds__(VecCfg<T, TX, TY>::NT, 2)
fwd_vec_kernel(const FwdArgs<T> a, const int nchunks)
{
    using C = VecCfg<T, TX, TY>;
    using VV = V16<T>;
    constexpr int VX = C::VX, W = C::W, H = C::H, PP = C::PP, UP = C::UP, SXP = C::SXP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *const sphi = reinterpret_cast<T *>(smem_raw);      // [NSP][PHI]
    T *const svel = sphi + C::NSP * C::PHI;                // [NSV][VEL] = u | v | w
    T *const ssx = svel + C::NSV * C::VEL;                 // [2][SXS]
    T *const ssy = ssx + 2 * C::SXS;                       // [2][SYS]

    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long plane = (long long)nx * ny;
    const int tiles_x = (nx + W - 1) / W;
    const int ntiles = tiles_x * ((ny + H - 1) / H);
    const T c_adv = a.c.c_adv, c_dif = a.c.c_dif, c_shp = a.c.c_shp, c_upd = a.c.c_upd;

    // Role: own vector of cells (tx, ty), a y-ring group, or an x-ring cell.
    const bool is_own = tid < C::NOWN;
    const int tx = tid % TX, ty = tid / TX;
    const int rr = tid - C::NOWN;  // 0..63 for ring threads
    const bool is_yring = !is_own && rr < 32 && rr < 2 * TX;
    const bool is_xring = !is_own && rr >= 32 && rr - 32 < 2 * TY;
    const int ry_row = (rr < TX) ? -1 : H, ry_col = rr % TX;  // y-ring group
    const int rx_row = (rr - 32) % TY;                         // x-ring cell
    const int rx_col = ((rr - 32) < TY) ? -1 : W;

    // Normals and sharpening of the VX cells of group (gc, ly) of plane Pm
    // (Pmm, Pmp: the planes below and above).
    auto sharp_group = [&](const T *Pm, const T *Pmm, const T *Pmp, int gc, int ly, T *s0, T *s1,
                           T *s2) {
        const int off = (ly + 2) * PP + VX + gc * VX;
        T c[VX], yn[VX], yp[VX], zn[VX], zp[VX];
        VV::ld(c, Pm + off);
        VV::ld(yn, Pm + off - PP);
        VV::ld(yp, Pm + off + PP);
        VV::ld(zn, Pmm + off);
        VV::ld(zp, Pmp + off);
        const T L = Pm[off - 1], R = Pm[off + VX];
#pragma unroll
        for (int i = 0; i < VX; ++i) {
            const T g0 = (i + 1 < VX ? c[i + 1] : R) - (i > 0 ? c[i - 1] : L);
            const T g1 = yp[i] - yn[i];
            const T g2 = zp[i] - zn[i];
            // rsqrt of q + the smallest normal number: finite at g = 0, where
            // s = wgt * g = 0 exactly; only cells with |g| below ~1e-18 (float)
            // or ~1e-154 (double), whose s is negligible, see a perturbation.
            const T q = fma(g2, g2, fma(g1, g1, fma(g0, g0, NumLim<T>::tiny())));
            const T inv = rsqrt_t(q);
            const T wgt = c[i] * (T(1) - c[i]) * inv;
            s0[i] = wgt * g0;
            s1[i] = wgt * g1;
            s2[i] = wgt * g2;
        }
    };
    auto sharp_cell = [&](const T *Pm, const T *Pmm, const T *Pmp, int lx, int ly) {
        const int off = (ly + 2) * PP + VX + lx;
        const T p = Pm[off];
        const T g0 = Pm[off + 1] - Pm[off - 1];
        const T g1 = Pm[off + PP] - Pm[off - PP];
        const T g2 = Pmp[off] - Pmm[off];
        const T q = fma(g2, g2, fma(g1, g1, fma(g0, g0, NumLim<T>::tiny())));
        const T inv = rsqrt_t(q);
        return p * (T(1) - p) * inv * g0;  // s_x only
    };

    Acc<T> acc;
    acc.init();
    bool dep_waited = false;  // the previous grid on the stream has completed

    // planes [z_lo, z_hi) with ZR, else all of them
    const int zlo = ZR ? a.z_lo : 0, zr = ZR ? a.z_hi - a.z_lo : nz;
    UnitIter<W, H> units(ntiles, zr, nchunks);
    Unit un;
    while (units.next(un, ntiles, tiles_x, zr, nchunks)) {
        const int x0 = un.x0, y0 = un.y0, z0 = un.z0 + zlo, z1 = un.z1 + zlo;

        // The 64 ring threads issue every 16-byte copy (they are idle while the
        // own warps evaluate fluxes).  Global in-plane offsets of their chunks:
        constexpr int NC = 64;
        constexpr int RPHI = (C::CPHI + NC - 1) / NC, RU = (C::CU + NC - 1) / NC;
        constexpr int RV = (C::CV + NC - 1) / NC, RW = (C::CW + NC - 1) / NC;
        const int ct = tid - C::NOWN;
        int gphi[RPHI], gu[RU], gv[RV], gw[RW];
        unsigned *const st = a.red.status;
        (void)st;
        const long long lastv = plane - VX + 1;  // a 16-byte chunk must end inside the plane
        (void)lastv;
        if (!is_own) {
#pragma unroll
            for (int r = 0; r < RPHI; ++r) {
                const int e = ct + r * NC, row = e / (PP / VX), col = e - row * (PP / VX);
                gphi[r] = (int)CDI_CHK(wrapi(y0 - 2 + row, ny) * nx + wrapi(x0 - VX + col * VX, nx), lastv, st);
            }
#pragma unroll
            for (int r = 0; r < RU; ++r) {
                const int e = ct + r * NC, row = e / (UP / VX), col = e - row * (UP / VX);
                gu[r] = (int)CDI_CHK(wrapi(y0 + row, ny) * nx + wrapi(x0 - VX + col * VX, nx), lastv, st);
            }
#pragma unroll
            for (int r = 0; r < RV; ++r) {
                const int e = ct + r * NC, row = e / (W / VX), col = e - row * (W / VX);
                gv[r] = (int)CDI_CHK(wrapi(y0 - 1 + row, ny) * nx + wrapi(x0 + col * VX, nx), lastv, st);
            }
#pragma unroll
            for (int r = 0; r < RW; ++r) {
                const int e = ct + r * NC, row = e / (W / VX), col = e - row * (W / VX);
                gw[r] = (int)CDI_CHK(wrapi(y0 + row, ny) * nx + wrapi(x0 + col * VX, nx), lastv, st);
            }
        }
        auto issue_phi = [&](int z, int slot) {
            if (is_own) return;
            const T *src = a.phi + (long long)wrapi(z, nz) * plane;
            T *dst = sphi + slot * C::PHI;
#pragma unroll
            for (int r = 0; r < RPHI; ++r) {
                const int e = ct + r * NC;
                if (e < C::CPHI) cp_async<16>(dst + e * VX, src + gphi[r]);
            }
        };
        auto issue_vel = [&](int z, int slot) {
            if (is_own) return;
            const long long zo = (long long)CDI_CHK(z, nz, st) * plane;
            T *dst = svel + slot * C::VEL;
#pragma unroll
            for (int r = 0; r < RU; ++r) {
                const int e = ct + r * NC;
                if (e < C::CU) cp_async<16>(dst + e * VX, a.u + zo + gu[r]);
            }
#pragma unroll
            for (int r = 0; r < RV; ++r) {
                const int e = ct + r * NC;
                if (e < C::CV) cp_async<16>(dst + C::USZ + e * VX, a.v + zo + gv[r]);
            }
#pragma unroll
            for (int r = 0; r < RW; ++r) {
                const int e = ct + r * NC;
                if (e < C::CW) cp_async<16>(dst + C::USZ + C::VSZ + e * VX, a.w + zo + gw[r]);
            }
        };

        // phi slot of plane z: (z - z0 + 2) mod 5; velocity slot: (z - z0) mod 3.
        __syncthreads();  // the previous unit's readers are done with every slot
        // The face velocities are never written by a step: staged (and the w below
        // plane z0 loaded) before waiting for the previous grid on the stream,
        // whose outputs -- phi, the Runge-Kutta operands, the reduction scratch --
        // are touched only after it.
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
        for (int d = 0; d < 5; ++d) issue_phi(z0 - 2 + d, d);  // planes z0-2 .. z0+2
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();

        // Prologue: s_z at plane z0-1 (own), s at plane z0 (own + ring), flux at z0-1/2.
        T szc[VX], Fzm[VX];
        {
            const T *P0 = sphi + 2 * C::PHI, *Pm1 = sphi + 1 * C::PHI, *Pm2 = sphi;
            const T *P1 = sphi + 3 * C::PHI;
            if (is_own) {
                T a0[VX], a1[VX], szm[VX], s0[VX], s1[VX];
                sharp_group(Pm1, Pm2, P0, tx, ty, a0, a1, szm);
                sharp_group(P0, Pm1, P1, tx, ty, s0, s1, szc);
                VV::st(ssx + (z0 & 1) * C::SXS + ty * SXP + VX + tx * VX, s0);
                VV::st(ssy + (z0 & 1) * C::SYS + (ty + 1) * W + tx * VX, s1);
                T pm[VX], pc[VX];
                VV::ld(pm, Pm1 + (ty + 2) * PP + VX + tx * VX);
                VV::ld(pc, P0 + (ty + 2) * PP + VX + tx * VX);
#pragma unroll
                for (int i = 0; i < VX; ++i)
                    Fzm[i] = flux(c_adv * wlo[i], c_dif, c_shp, pm[i], pc[i], szm[i], szc[i]);
            } else if (is_yring) {
                T s0[VX], s1[VX], s2[VX];
                sharp_group(P0, Pm1, P1, ry_col, ry_row, s0, s1, s2);
                VV::st(ssy + (z0 & 1) * C::SYS + (ry_row + 1) * W + ry_col * VX, s1);
            } else if (is_xring) {
                ssx[(z0 & 1) * C::SXS + rx_row * SXP + VX + rx_col] = sharp_cell(P0, Pm1, P1, rx_col, rx_row);
            }
        }
        // Plane z0+3 reuses the slot of plane z0-2, which the prologue just read.
        __syncthreads();
        if (z0 + 3 <= z1 + 1) issue_phi(z0 + 3, 0);
        if (z0 + 1 < z1) issue_vel(z0 + 1, 1);
        cp_async_commit();

        int pk = 2;  // phi slot of plane k
        int vk = 0;  // velocity slot of plane k
        for (int k = z0; k < z1; ++k) {
            const int pk1 = pk == 4 ? 0 : pk + 1;
            const int pk2 = pk1 == 4 ? 0 : pk1 + 1;
            const int pkm = pk == 0 ? 4 : pk - 1;   // also the slot of plane k+4
            const int vk2 = vk == 0 ? 2 : vk - 1;   // slot of plane k+2
            // S1: phi plane k+2 and the velocities of plane k have landed, and
            // every thread has left iteration k-1.
            cp_async_wait<1>();
            __syncthreads();
            if (k + 4 <= z1 + 1) issue_phi(k + 4, pkm);
            if (k + 2 < z1) issue_vel(k + 2, vk2);
            cp_async_commit();

            // Runge-Kutta stage operands of plane k, fetched now to overlap phase B.
            T rb[VX], rq[VX];
            if constexpr (RK) {
                if (writes) {
                    const long long o = (long long)k * plane + own_off;
                    if (a.rk_base) VV::ld(rb, a.rk_base + o);
                    if (a.rk_q) VV::ld(rq, a.rk_q + o);
                }
            }

            // B: sharpening at plane k+1.
            const T *Pk = sphi + pk * C::PHI, *Pk1 = sphi + pk1 * C::PHI, *Pk2 = sphi + pk2 * C::PHI;
            const int b1 = (k + 1) & 1;
            T szn[VX];
            if (is_own) {
                T s0[VX], s1[VX];
                sharp_group(Pk1, Pk, Pk2, tx, ty, s0, s1, szn);
                VV::st(ssx + b1 * C::SXS + ty * SXP + VX + tx * VX, s0);
                VV::st(ssy + b1 * C::SYS + (ty + 1) * W + tx * VX, s1);
            } else if (is_yring) {
                T s0[VX], s1[VX], s2[VX];
                sharp_group(Pk1, Pk, Pk2, ry_col, ry_row, s0, s1, s2);
                VV::st(ssy + b1 * C::SYS + (ry_row + 1) * W + ry_col * VX, s1);
            } else if (is_xring) {
                ssx[b1 * C::SXS + rx_row * SXP + VX + rx_col] = sharp_cell(Pk1, Pk, Pk2, rx_col, rx_row);
            }
            // No barrier here: phase C reads only the s_x / s_y of plane k, which
            // were written before S1, and the s_z of plane k+1 from registers.
            // The next write of slot k&1 happens after the next S1.

            // C: fluxes and update at plane k.  Along x and y the four faces of a
            // cell telescope to
            //   c_adv [u_+(c + R) - u_-(L + c)] - c_dif (L + R - 2c) + c_shp (s_R - s_L)
            // (the cell's own s_x, s_y cancel); the z face below is carried.
            if (is_own) {
                const int b = k & 1;
                const int po = (ty + 2) * PP + VX + tx * VX;
                T c[VX], yn[VX], yp[VX], zp[VX];
                VV::ld(c, Pk + po);
                VV::ld(yn, Pk + po - PP);
                VV::ld(yp, Pk + po + PP);
                VV::ld(zp, Pk1 + po);
                const T L = Pk[po - 1], R = Pk[po + VX];
                const T *sxr = ssx + b * C::SXS + ty * SXP + VX + tx * VX;
                const T *syr = ssy + b * C::SYS + (ty + 1) * W + tx * VX;
                T sxc[VX], syn[VX], syp[VX];
                VV::ld(sxc, sxr);
                VV::ld(syn, syr - W);
                VV::ld(syp, syr + W);
                const T sxL = sxr[-1], sxR = sxr[VX];
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
                T o[VX];
#pragma unroll
                for (int i = 0; i < VX; ++i) {
                    const T xl = i > 0 ? c[i - 1] : L, xr = i + 1 < VX ? c[i + 1] : R;
                    const T ul = i > 0 ? uc[i - 1] : uL;
                    const T sl = i > 0 ? sxc[i - 1] : sxL, sr = i + 1 < VX ? sxc[i + 1] : sxR;
                    T adv = uc[i] * (c[i] + xr);
                    adv = fma(-ul, xl + c[i], adv);
                    adv = fma(vc[i], c[i] + yp[i], adv);
                    adv = fma(-vn[i], yn[i] + c[i], adv);
                    const T dif = fma(T(-4), c[i], (xl + xr) + (yn[i] + yp[i]));
                    const T shp = (sr - sl) + (syp[i] - syn[i]);
                    const T Fzp = flux(c_adv * wc[i], c_dif, c_shp, c[i], zp[i], szc[i], szn[i]);
                    const T div = fma(c_adv, adv, fma(-c_dif, dif, fma(c_shp, shp, Fzp - Fzm[i])));
                    if constexpr (RK) o[i] = -c_upd * div;  // r = dt * RHS, combined below
                    else o[i] = fma(-c_upd, div, c[i]);
                    Fzm[i] = Fzp;
                    szc[i] = szn[i];
                }
                if (writes) {
                    const long long ko = (long long)CDI_CHK(k, nz, st) * plane + CDI_CHK(own_off, lastv, st);
                    if constexpr (RK) {
                        T qo[VX];
#pragma unroll
                        for (int i = 0; i < VX; ++i) {
                            const T r = o[i];
                            const T base = a.rk_base ? rb[i] : c[i];
                            const T q = a.rk_q ? rq[i] : T(0);
                            o[i] = fma(a.rk_delta, q, fma(a.rk_alpha, r, base));
                            qo[i] = fma(a.rk_beta, r, a.rk_mu * (a.rk_q ? q : c[i]));
                        }
                        if (a.rk_qout) VV::st(a.rk_qout + ko, qo);
                    }
                    VV::st(a.out + ko, o);
                    acc.template add_group<VX>(o, a.c.tol);
                }
            }
            pk = pk1;
            vk = vk == 2 ? 0 : vk + 1;
        }
        cp_async_wait<0>();
    }
    if (!dep_waited) grid_dep_wait();
    grid_dep_launch();  // the next step may start staging its velocities
    reduce_and_finish<ZR>(acc, a.red);
}

// ===========================================================================
// Scalar kernel (any extents): the per-unit body is in cdi_fwd_scalar.cuh.

template <typename T, int BX, int BY, bool RK, bool FACE = false, bool ZR = false>
__global__ void __launch_bounds__(BX * BY)
fwd_kernel(const FwdArgs<T> a, const int nchunks)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tiles_x = (a.nx + BX - 1) / BX;
    const int ntiles = tiles_x * ((a.ny + BY - 1) / BY);
    Acc<T> acc;
    acc.init();
    const int zlo = ZR ? a.z_lo : 0, zr = ZR ? a.z_hi - a.z_lo : a.nz;
    UnitIter<BX, BY> units(ntiles, zr, nchunks);
    Unit un;
    while (units.next(un, ntiles, tiles_x, zr, nchunks)) {
        un.z0 += zlo;
        un.z1 += zlo;
        if (!RK && !FACE && a.nz == 1)
            flat_unit<T, BX, BY>(a, un, acc, smem_raw);
        else
            scalar_unit<T, BX, BY, RK, SCALAR_PF, FACE>(a, un, acc, smem_raw);
    }
    reduce_and_finish<ZR>(acc, a.red);
}

// ===========================================================================
// Kernel table and launch
//
// Forward tiles: 0..3 scalar BX x BY = 32x8, 32x16, 64x8, 32x4;
//                4, 5 vector TX x TY = 16x16, 16x8 (x width 16 * 16/sizeof(T));
//                6 vector 16x16 with tensor-memory-accelerator staging (cdi_fwd_tma.cu).

int fwd_num_tiles() { return 7; }

bool fwd_tile_is_vec(int tile) { return tile >= 4; }

void fwd_tile_dims(int tile, int esize, int *bw, int *bh)
{
    static const int sdim[4][2] = {{32, 8}, {32, 16}, {64, 8}, {32, 4}};
    if (tile < 4) {
        *bw = sdim[tile][0];
        *bh = sdim[tile][1];
    } else {
        *bw = 16 * (16 / esize);
        *bh = tile == 5 ? 8 : 16;
    }
}

long long fwd_tiles_xy(int tile, int esize, int nx, int ny)
{
    int bw, bh;
    fwd_tile_dims(tile, esize, &bw, &bh);
    return (long long)((nx + bw - 1) / bw) * ((ny + bh - 1) / bh);
}

template <typename K>
static cudaError_t occ(K kernel, int threads, size_t smem, int *resident)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(resident, kernel, threads, smem);
}

// Runge-Kutta stage kernels exist for tiles 1, 3 (scalar) and 4 (vector) only.
bool fwd_tile_has_rk(int tile) { return tile == 1 || tile == 3 || tile == 4; }

template <typename T>
cudaError_t fwd_occupancy(int tile, bool rk, int *resident, bool face, bool slab)
{
    if (slab) {  // the z-slab kernels of the pipelined host step
        if (rk || face) return cudaErrorInvalidValue;
        if (tile == 4)
            return occ(fwd_vec_kernel<T, 16, 16, false, true>, VecCfg<T, 16, 16>::NT, VecCfg<T, 16, 16>::bytes,
                       resident);
        if (tile == 0) return occ(fwd_kernel<T, 32, 8, false, false, true>, 256, FwdSmem<T, 32, 8>::bytes, resident);
        return cudaErrorInvalidValue;
    }
    if (face) {
        if (rk || tile != 0) return cudaErrorInvalidValue;
        return occ(fwd_kernel<T, 32, 8, false, true>, 256, FwdSmem<T, 32, 8>::bytes, resident);
    }
    if (rk) {
        switch (tile) {
        case 1: return occ(fwd_kernel<T, 32, 16, true>, 512, FwdSmem<T, 32, 16>::bytes, resident);
        case 3: return occ(fwd_kernel<T, 32, 4, true>, 128, FwdSmem<T, 32, 4>::bytes, resident);
        case 4: return occ(fwd_vec_kernel<T, 16, 16, true>, VecCfg<T, 16, 16>::NT, VecCfg<T, 16, 16>::bytes, resident);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (tile) {
    case 0: return occ(fwd_kernel<T, 32, 8, false>, 256, FwdSmem<T, 32, 8>::bytes, resident);
    case 1: return occ(fwd_kernel<T, 32, 16, false>, 512, FwdSmem<T, 32, 16>::bytes, resident);
    case 2: return occ(fwd_kernel<T, 64, 8, false>, 512, FwdSmem<T, 64, 8>::bytes, resident);
    case 3: return occ(fwd_kernel<T, 32, 4, false>, 128, FwdSmem<T, 32, 4>::bytes, resident);
    case 4: return occ(fwd_vec_kernel<T, 16, 16, false>, VecCfg<T, 16, 16>::NT, VecCfg<T, 16, 16>::bytes, resident);
    case 5: return occ(fwd_vec_kernel<T, 16, 8, false>, VecCfg<T, 16, 8>::NT, VecCfg<T, 16, 8>::bytes, resident);
    case 6: return tma_occupancy<T>(resident);
    default: return cudaErrorInvalidValue;
    }
}
template cudaError_t fwd_occupancy<float>(int, bool, int *, bool, bool);
template cudaError_t fwd_occupancy<double>(int, bool, int *, bool, bool);

// Launch with programmatic stream serialisation: the kernel may start while
// the previous grid on the stream finishes (it waits in grid_dep_wait before
// touching anything that grid may write).
template <typename K, typename... Args>
static cudaError_t launch_dependent(K kernel, int nblocks, int threads, size_t smem, cudaStream_t s, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblocks);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename T>
cudaError_t launch_fwd(const FwdArgs<T> &a, int tile, int nblocks, int nchunks, bool rk, cudaStream_t s,
                       bool face)
{
    if (a.z_hi > 0) {  // a z slab: tile 4 (vector) or 0 (any extents), centre form, Euler
        if (rk || face) return cudaErrorInvalidValue;
        if (tile == 4)
            fwd_vec_kernel<T, 16, 16, false, true>
                <<<nblocks, VecCfg<T, 16, 16>::NT, VecCfg<T, 16, 16>::bytes, s>>>(a, nchunks);
        else if (tile == 0)
            fwd_kernel<T, 32, 8, false, false, true><<<nblocks, dim3(32, 8), FwdSmem<T, 32, 8>::bytes, s>>>(a, nchunks);
        else
            return cudaErrorInvalidValue;
        return cudaGetLastError();
    }
    if (face) {  // face-product sharpening: tile 0 only, Euler only
        if (rk || tile != 0) return cudaErrorInvalidValue;
        fwd_kernel<T, 32, 8, false, true><<<nblocks, dim3(32, 8), FwdSmem<T, 32, 8>::bytes, s>>>(a, nchunks);
        return cudaGetLastError();
    }
    if (rk) {
        switch (tile) {
        case 1: fwd_kernel<T, 32, 16, true><<<nblocks, dim3(32, 16), FwdSmem<T, 32, 16>::bytes, s>>>(a, nchunks); break;
        case 3: fwd_kernel<T, 32, 4, true><<<nblocks, dim3(32, 4), FwdSmem<T, 32, 4>::bytes, s>>>(a, nchunks); break;
        case 4:
            fwd_vec_kernel<T, 16, 16, true><<<nblocks, VecCfg<T, 16, 16>::NT, VecCfg<T, 16, 16>::bytes, s>>>(a, nchunks);
            break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    switch (tile) {
    case 0: fwd_kernel<T, 32, 8, false><<<nblocks, dim3(32, 8), FwdSmem<T, 32, 8>::bytes, s>>>(a, nchunks); break;
    case 1: fwd_kernel<T, 32, 16, false><<<nblocks, dim3(32, 16), FwdSmem<T, 32, 16>::bytes, s>>>(a, nchunks); break;
    case 2: fwd_kernel<T, 64, 8, false><<<nblocks, dim3(64, 8), FwdSmem<T, 64, 8>::bytes, s>>>(a, nchunks); break;
    case 3: fwd_kernel<T, 32, 4, false><<<nblocks, dim3(32, 4), FwdSmem<T, 32, 4>::bytes, s>>>(a, nchunks); break;
    case 4:
        return launch_dependent(fwd_vec_kernel<T, 16, 16, false>, nblocks, VecCfg<T, 16, 16>::NT,
                                VecCfg<T, 16, 16>::bytes, s, a, nchunks);
    case 5:
        return launch_dependent(fwd_vec_kernel<T, 16, 8, false>, nblocks, VecCfg<T, 16, 8>::NT,
                                VecCfg<T, 16, 8>::bytes, s, a, nchunks);
    case 6: return launch_fwd_tma<T>(a, nblocks, nchunks, s);
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template cudaError_t launch_fwd<float>(const FwdArgs<float> &, int, int, int, bool, cudaStream_t, bool);
template cudaError_t launch_fwd<double>(const FwdArgs<double> &, int, int, int, bool, cudaStream_t, bool);

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
    reduce_and_finish(acc, red);
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
