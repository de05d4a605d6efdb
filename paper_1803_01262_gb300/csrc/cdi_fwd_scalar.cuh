// Per-unit body of the one-cell-per-thread CDI step (any extents), shared by
// the single-box forward kernel and the batched kernel.
//
// A unit is a BX x BY tile of one box and a range of planes [z0, z1).  The
// block stages phi planes with a halo of 2 in x and y, and the face-velocity
// planes u (x from x0-1), v (y from y0-1) and w, by element-wise cp.async into
// shared rings, PF planes ahead of use (phi plane j+2 and velocity plane j
// travel in one commit group); computes the sharpening vector
// s = phi (1 - phi) g/|g| of plane k+1 for its cells and a one-cell ring (s_x
// on the x-ring, s_y on the y-ring); and updates plane k from its six face
// fluxes
//   F = c_adv u_f (phi_L + phi_R) - c_dif (phi_R - phi_L) + c_shp (s_L + s_R)
// with the face below carried in a register.  Outputs go to the caller's
// accumulator.
#pragma once

#include "cdi_async.cuh"
#include "cdi_fwd_common.cuh"
#include "cdi_reduce.cuh"

namespace cdi {

constexpr int SCALAR_PF = 3;  // default prefetch distance (planes) of the scalar body
constexpr int NSLOT = 8;      // phi ring: power of two >= PF + 3 live planes (PF <= 5)

__host__ __device__ constexpr int vel_slots(int pf) { return pf + 1 <= 4 ? 4 : 8; }

template <typename T, int BX, int BY, int PF = SCALAR_PF>
struct FwdSmem {
    static_assert(PF >= 1 && PF + 3 <= NSLOT, "prefetch distance out of range");
    static constexpr int PX = BX + 4, PY = BY + 4;
    static constexpr int NU = BY * (BX + 1), NV = (BY + 1) * BX, NW = BY * BX;
    static constexpr int VPL = NU + NV + NW;  // one velocity plane: u | v | w
    static constexpr int NVS = vel_slots(PF);
    static constexpr size_t bytes =
        sizeof(T) * (NSLOT * PY * PX + 2 * BY * (BX + 2) + 2 * (BY + 2) * BX + NVS * VPL);
};

// FACE: the non-default face-product sharpening, gamma phi_f (1 - phi_f) n_f with
// phi_f and n_f the averages of the two cells (the smem s arrays then hold n).
template <typename T, int BX, int BY, bool RK = false, int PF = SCALAR_PF, bool FACE = false>
__device__ __forceinline__ void scalar_unit(const FwdArgs<T> &a, const Unit &un, Acc<T> &acc,
                                            unsigned char *smem_raw)
{
    using S = FwdSmem<T, BX, BY, PF>;
    constexpr int PX = BX + 4, PY = BY + 4, PLANE = PX * PY;
    constexpr int NT = BX * BY;
    constexpr int NLOAD = (PLANE + NT - 1) / NT;
    constexpr int NU = S::NU, NV = S::NV, NW = S::NW, NVS = S::NVS;
    constexpr int RU = (NU + NT - 1) / NT, RV = (NV + NT - 1) / NT, RW = (NW + NT - 1) / NT;
    T(*sp)[PY][PX] = reinterpret_cast<T(*)[PY][PX]>(smem_raw);           // phi ring [NSLOT]
    T(*sx)[BY][BX + 2] = reinterpret_cast<T(*)[BY][BX + 2]>(sp + NSLOT);  // s_x, x = -1..BX [2]
    T(*sy)[BY + 2][BX] = reinterpret_cast<T(*)[BY + 2][BX]>(sx + 2);      // s_y, y = -1..BY [2]
    T *const sv = reinterpret_cast<T *>(sy + 2);                          // velocity ring [NVS][VPL]

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
    // The block is BX x BY: lets the compiler drop the bound checks of full copy rounds.
    __builtin_assume(tx >= 0 && tx < BX && ty >= 0 && ty < BY);
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long plane = (long long)nx * ny;
    const int x0 = un.x0, y0 = un.y0, z0 = un.z0, z1 = un.z1;

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

    auto sharp = [&](int z, int lx, int ly, T &s0, T &s1, T &s2) {
        const int X = lx + 2, Y = ly + 2;
        const int m = z & (NSLOT - 1), mm = (z - 1) & (NSLOT - 1), mp = (z + 1) & (NSLOT - 1);
        const T p = sp[m][Y][X];
        const T g0 = sp[m][Y][X + 1] - sp[m][Y][X - 1];
        const T g1 = sp[m][Y + 1][X] - sp[m][Y - 1][X];
        const T g2 = sp[mp][Y][X] - sp[mm][Y][X];
        const T q = fma(g2, g2, fma(g1, g1, fma(g0, g0, NumLim<T>::tiny())));
        const T inv = rsqrt_t(q);
        const T wgt = FACE ? inv : p * (T(1) - p) * inv;
        s0 = wgt * g0;
        s1 = wgt * g1;
        s2 = wgt * g2;
    };
    // Face flux with the sharpening in the configured form (sl, sr: the two cells'
    // s, or their normals for FACE).
    auto face_flux = [&](T cadv_u, T pl, T pr, T sl, T sr) {
        if constexpr (FACE) {
            const T pf = T(0.5) * (pl + pr);
            return cadv_u * (pl + pr) - c_dif * (pr - pl) + c_shp * (pf * (T(1) - pf) * (sl + sr));
        } else {
            return flux(cadv_u, c_dif, c_shp, pl, pr, sl, sr);
        }
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

    unsigned *const st = a.red.status;
    (void)st;
    int loff[NLOAD];
#pragma unroll
    for (int r = 0; r < NLOAD; ++r) {
        const int e = tid + r * NT;
        const int ey = e / PX, ex = e - ey * PX;
        loff[r] = (e < PLANE) ? (int)CDI_CHK(wrapi(y0 + ey - 2, ny) * nx + wrapi(x0 + ex - 2, nx), plane, st) : 0;
    }
    const int gx = wrapi(x0 + tx, nx), gy = wrapi(y0 + ty, ny);
    const bool own = (x0 + tx < nx) && (y0 + ty < ny);
    const int oc = gy * nx + gx;

    // Stage phi plane z (ring slot z & (NSLOT-1)) from wrapped plane offset zo.
    auto issue_plane_at = [&](int z, long long zo) {
        const T *src = a.phi + zo;
        T *dst = &sp[z & (NSLOT - 1)][0][0];
#pragma unroll
        for (int r = 0; r < NLOAD; ++r) {
            const int e = tid + r * NT;
            if (e < PLANE) cp_async<sizeof(T)>(dst + e, src + loff[r]);
        }
    };
    // Velocity plane offsets: u rows y0.., columns x0-1..; v rows y0-1.., columns
    // x0..; w rows y0.., columns x0.. (periodic wrap of overhanging tiles).
    int uoff[RU], voff[RV], woff[RW];
#pragma unroll
    for (int r = 0; r < RU; ++r) {
        const int e = tid + r * NT, ey = e / (BX + 1), ex = e - ey * (BX + 1);
        uoff[r] = (e < NU) ? (int)CDI_CHK(wrapi(y0 + ey, ny) * nx + wrapi(x0 - 1 + ex, nx), plane, st) : 0;
    }
#pragma unroll
    for (int r = 0; r < RV; ++r) {
        const int e = tid + r * NT, ey = e / BX, ex = e - ey * BX;
        voff[r] = (e < NV) ? (int)CDI_CHK(wrapi(y0 - 1 + ey, ny) * nx + wrapi(x0 + ex, nx), plane, st) : 0;
    }
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        const int e = tid + r * NT, ey = e / BX, ex = e - ey * BX;
        woff[r] = (e < NW) ? (int)CDI_CHK(wrapi(y0 + ey, ny) * nx + wrapi(x0 + ex, nx), plane, st) : 0;
    }
    auto issue_plane = [&](int z) { issue_plane_at(z, (long long)wrapi(z, nz) * plane); };
    // Stage velocity plane z (0 <= z < nz) from plane offset zo = z * plane.
    auto issue_vel_at = [&](int z, long long zo) {
        T *dst = sv + (z & (NVS - 1)) * S::VPL;
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
    auto issue_vel = [&](int z) { issue_vel_at(z, (long long)CDI_CHK(z, nz, st) * plane); };

    // Commit groups: first phi planes z0-2 .. z0+1; then PF prologue groups,
    // the d-th holding phi plane z0+2+d and velocity plane z0+d; then one group
    // per iteration j holding phi plane j+2+PF and velocity plane j+PF.  At
    // iteration k, waiting until at most PF-1 groups are pending therefore
    // lands phi plane k+2 and velocity plane k.
    __syncthreads();  // the previous unit's readers are done with the rings
    issue_plane(z0 - 2);
    issue_plane(z0 - 1);
    issue_plane(z0);
    issue_plane(z0 + 1);
    cp_async_commit();
#pragma unroll
    for (int d = 0; d < PF; ++d) {
        if (z0 + 2 + d <= z1 + 1) issue_plane(z0 + 2 + d);
        if (z0 + d < z1) issue_vel(z0 + d);
        cp_async_commit();
    }
    const T wlo = __ldg(a.w + (long long)wrapi(z0 - 1, nz) * plane + oc);
    cp_async_wait<PF>();
    __syncthreads();
    T szm, szc;
    {
        T d0, d1;
        sharp(z0 - 1, tx, ty, d0, d1, szm);
    }
    sharp_plane(z0, szc);
    T Fzm;
    {
        const T pm = sp[(z0 - 1) & (NSLOT - 1)][ty + 2][tx + 2];
        const T pc = sp[z0 & (NSLOT - 1)][ty + 2][tx + 2];
        Fzm = face_flux(c_adv * wlo, pm, pc, szm, szc);
    }

    // Wrapped offset of the phi plane issued next (k+2+PF) and of the next
    // velocity plane (k+PF), advanced by one plane per iteration.
    int zq = wrapi(z0 + 2 + PF, nz);
    long long oq = (long long)zq * plane, ov = (long long)(z0 + PF) * plane;
    for (int k = z0; k < z1; ++k) {
        // S1: phi plane k+2 and velocity plane k have landed, and every thread
        // has left iteration k-1 (so the slots written below are free).
        cp_async_wait<PF - 1>();
        __syncthreads();
        if (k + 2 + PF <= z1 + 1) issue_plane_at(k + 2 + PF, oq);
        if (k + PF < z1) issue_vel_at(k + PF, ov);
        cp_async_commit();
        if (++zq == nz) {
            zq = 0;
            oq = 0;
        } else {
            oq += plane;
        }
        ov += plane;
        T rb = T(0), rq = T(0);
        if constexpr (RK) {
            if (own) {
                const long long o = (long long)k * plane + oc;
                if (a.rk_base) rb = __ldg(a.rk_base + o);
                if (a.rk_q) rq = a.rk_q[o];
            }
        }
        // B: sharpening at plane k+1 (slot (k+1)&1; phase C reads slot k&1, which
        // was written before S1, so no barrier separates B from C).
        T szn;
        sharp_plane(k + 1, szn);
        // C: fluxes and update at plane k.
        const int m = k & (NSLOT - 1), b = k & 1;
        const T pc = sp[m][ty + 2][tx + 2];
        const T pxm = sp[m][ty + 2][tx + 1], pxp = sp[m][ty + 2][tx + 3];
        const T pym = sp[m][ty + 1][tx + 2], pyp = sp[m][ty + 3][tx + 2];
        const T pzp = sp[(k + 1) & (NSLOT - 1)][ty + 2][tx + 2];
        const T sxm = sx[b][ty][tx], sxp = sx[b][ty][tx + 2];
        const T sym = sy[b][ty][tx], syp = sy[b][ty + 2][tx];
        const T *vel = sv + (k & (NVS - 1)) * S::VPL;
        const T uc = vel[ty * (BX + 1) + tx + 1], um = vel[ty * (BX + 1) + tx];
        const T vc = vel[NU + (ty + 1) * BX + tx], vm = vel[NU + ty * BX + tx];
        const T wc = vel[NU + NV + ty * BX + tx];
        // x and y faces telescoped; the cell's own s_x, s_y cancel.
        T adv = uc * (pc + pxp);
        adv = fma(-um, pxm + pc, adv);
        adv = fma(vc, pc + pyp, adv);
        adv = fma(-vm, pym + pc, adv);
        const T dif = fma(T(-4), pc, (pxm + pxp) + (pym + pyp));
        T shp;
        if constexpr (FACE) {
            // each face: phi_f (1 - phi_f) (n_L + n_R); the cell's own normal does not cancel
            const T nxc = sx[b][ty][tx + 1], nyc = sy[b][ty + 1][tx];
            const T fxp = T(0.5) * (pc + pxp), fxm = T(0.5) * (pxm + pc);
            const T fyp = T(0.5) * (pc + pyp), fym = T(0.5) * (pym + pc);
            shp = (fxp * (T(1) - fxp) * (nxc + sxp) - fxm * (T(1) - fxm) * (sxm + nxc)) +
                  (fyp * (T(1) - fyp) * (nyc + syp) - fym * (T(1) - fym) * (sym + nyc));
        } else {
            shp = (sxp - sxm) + (syp - sym);
        }
        const T Fzp = face_flux(c_adv * wc, pc, pzp, szc, szn);
        const T div = fma(c_adv, adv, fma(-c_dif, dif, fma(c_shp, shp, Fzp - Fzm)));
        T o = fma(-c_upd, div, pc);
        if (own) {
            const long long ko = (long long)CDI_CHK(k, nz, st) * plane + CDI_CHK(oc, plane, st);
            if constexpr (RK) {
                const T r = -c_upd * div;  // dt * RHS
                const T base = a.rk_base ? rb : pc;
                const T q = a.rk_q ? rq : T(0);
                o = fma(a.rk_delta, q, fma(a.rk_alpha, r, base));
                if (a.rk_qout) a.rk_qout[ko] = fma(a.rk_beta, r, a.rk_mu * (a.rk_q ? q : pc));
            }
            a.out[ko] = o;
            acc.add(o, a.c.tol);
        }
        Fzm = Fzp;
        szc = szn;
    }
    cp_async_wait<0>();
}

// Per-unit body for a box with nz == 1 (2D, or 1D with ny == 1).  The single
// plane is its own periodic neighbour in z, so g_z = 0, s_z = 0 and the two z-face
// fluxes are equal (identical inputs) and cancel exactly; the plane and its u, v
// velocities are staged once and the sharpening is evaluated once, where the
// 3D body stages five copies of the plane and evaluates three planes of
// sharpening.  The arithmetic of the remaining terms is the 3D body's
// expression by expression, so the result is the same bit for bit.  FACE: the
// face-product sharpening (the s arrays then hold the normals), as in scalar_unit.
template <typename T, int BX, int BY, bool FACE = false>
__device__ __forceinline__ void flat_unit(const FwdArgs<T> &a, const Unit &un, Acc<T> &acc,
                                          unsigned char *smem_raw)
{
    using S = FwdSmem<T, BX, BY>;
    constexpr int PX = BX + 4, PY = BY + 4, PLANE = PX * PY;
    constexpr int NT = BX * BY;
    constexpr int NU = S::NU, NV = S::NV;
    T(*sp)[PY][PX] = reinterpret_cast<T(*)[PY][PX]>(smem_raw);           // phi (slot 0)
    T(*sx)[BY][BX + 2] = reinterpret_cast<T(*)[BY][BX + 2]>(sp + NSLOT);  // s_x [0]
    T(*sy)[BY + 2][BX] = reinterpret_cast<T(*)[BY + 2][BX]>(sx + 2);      // s_y [0]
    T *const sv = reinterpret_cast<T *>(sy + 2);                          // u | v (slot 0)

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
    __builtin_assume(tx >= 0 && tx < BX && ty >= 0 && ty < BY);
    const int nx = a.nx, ny = a.ny;
    const int x0 = un.x0, y0 = un.y0;
    const T c_adv = a.c.c_adv, c_dif = a.c.c_dif, c_shp = a.c.c_shp, c_upd = a.c.c_upd;

    __syncthreads();  // the previous unit's readers are done with the buffers
    for (int e = tid; e < PLANE; e += NT) {
        const int ey = e / PX, ex = e - ey * PX;
        cp_async<sizeof(T)>(&sp[0][0][0] + e, a.phi + wrapi(y0 + ey - 2, ny) * nx + wrapi(x0 + ex - 2, nx));
    }
    for (int e = tid; e < NU; e += NT) {
        const int ey = e / (BX + 1), ex = e - ey * (BX + 1);
        cp_async<sizeof(T)>(sv + e, a.u + wrapi(y0 + ey, ny) * nx + wrapi(x0 - 1 + ex, nx));
    }
    for (int e = tid; e < NV; e += NT) {
        const int ey = e / BX, ex = e - ey * BX;
        cp_async<sizeof(T)>(sv + NU + e, a.v + wrapi(y0 - 1 + ey, ny) * nx + wrapi(x0 + ex, nx));
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();

    auto sharp = [&](int lx, int ly, T &s0, T &s1) {
        const int X = lx + 2, Y = ly + 2;
        const T p = sp[0][Y][X];
        const T g0 = sp[0][Y][X + 1] - sp[0][Y][X - 1];
        const T g1 = sp[0][Y + 1][X] - sp[0][Y - 1][X];
        const T g2 = T(0);
        const T q = fma(g2, g2, fma(g1, g1, fma(g0, g0, NumLim<T>::tiny())));
        const T inv = rsqrt_t(q);
        const T wgt = FACE ? inv : p * (T(1) - p) * inv;
        s0 = wgt * g0;
        s1 = wgt * g1;
    };
    {
        T q0, q1;
        sharp(tx, ty, q0, q1);
        sx[0][ty][tx + 1] = q0;
        sy[0][ty + 1][tx] = q1;
        // the one-cell ring: s_y of rows -1 and BY, s_x of columns -1 and BX
        if (tid < 2 * BX) {
            const int rx = tid % BX, ry = tid < BX ? -1 : BY;
            T r0, r1;
            sharp(rx, ry, r0, r1);
            sy[0][ry + 1][rx] = r1;
        } else if (tid < 2 * BX + 2 * BY) {
            const int r = tid - 2 * BX, ry = r % BY, rx = r < BY ? -1 : BX;
            T r0, r1;
            sharp(rx, ry, r0, r1);
            sx[0][ry][rx + 1] = r0;
        }
    }
    __syncthreads();
    if ((x0 + tx < nx) && (y0 + ty < ny)) {
        const T pc = sp[0][ty + 2][tx + 2];
        const T pxm = sp[0][ty + 2][tx + 1], pxp = sp[0][ty + 2][tx + 3];
        const T pym = sp[0][ty + 1][tx + 2], pyp = sp[0][ty + 3][tx + 2];
        const T sxm = sx[0][ty][tx], sxp = sx[0][ty][tx + 2];
        const T sym = sy[0][ty][tx], syp = sy[0][ty + 2][tx];
        const T uc = sv[ty * (BX + 1) + tx + 1], um = sv[ty * (BX + 1) + tx];
        const T vc = sv[NU + (ty + 1) * BX + tx], vm = sv[NU + ty * BX + tx];
        T adv = uc * (pc + pxp);
        adv = fma(-um, pxm + pc, adv);
        adv = fma(vc, pc + pyp, adv);
        adv = fma(-vm, pym + pc, adv);
        const T dif = fma(T(-4), pc, (pxm + pxp) + (pym + pyp));
        T shp;
        if constexpr (FACE) {
            const T nxc = sx[0][ty][tx + 1], nyc = sy[0][ty + 1][tx];
            const T fxp = T(0.5) * (pc + pxp), fxm = T(0.5) * (pxm + pc);
            const T fyp = T(0.5) * (pc + pyp), fym = T(0.5) * (pym + pc);
            shp = (fxp * (T(1) - fxp) * (nxc + sxp) - fxm * (T(1) - fxm) * (sxm + nxc)) +
                  (fyp * (T(1) - fyp) * (nyc + syp) - fym * (T(1) - fym) * (sym + nyc));
        } else {
            shp = (sxp - sxm) + (syp - sym);
        }
        const T div = fma(c_adv, adv, fma(-c_dif, dif, fma(c_shp, shp, T(0))));  // z faces: Fzp - Fzm = 0
        const T o = fma(-c_upd, div, pc);
        a.out[wrapi(y0 + ty, ny) * nx + wrapi(x0 + tx, nx)] = o;
        acc.add(o, a.c.tol);
    }
}

}  // namespace cdi
