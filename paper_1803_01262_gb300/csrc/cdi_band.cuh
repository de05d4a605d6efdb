// Row-band unit body of the batched CDI step (any nx up to BAND_CELLS).
//
// A unit is a band of whole rows of one box -- rows [y0, y0 + hb), all nx
// columns -- and a range of planes [z0, z1).  Whole rows make the x direction
// periodic inside the staged rows (no x halo, no tile overhanging the box),
// and every staged region of a plane is one contiguous run of the array
// (plus, for bands touching the periodic y edge, the few wrapped halo rows):
//   phi: rows y0-2 .. y0+hb+1      u, w: rows y0 .. y0+hb-1      v: rows y0-1 .. y0+hb-1
// A region is kept in shared memory as dense rows of nx values starting at an
// element shift sh in [0, VX) chosen so that shared and global addresses agree
// modulo 16 bytes: the run is then copied with 16-byte cp.async by every
// thread of the block, and only its first and last few elements and the
// wrapped rows go element by element.  (The arrays are caller-owned and nx is
// arbitrary, so rows start at any 4-byte (8-byte) boundary; the shift absorbs
// that without a per-row layout.)
//
// Each thread owns up to BAND_CPT cells of the band, visited by linear index
// (consecutive threads on consecutive x: conflict-free shared loads, coalesced
// stores); the x neighbours of a cell are found by a per-cell offset that
// wraps at the row ends.  Per plane k (one barrier): phi plane k+4 and the
// velocities of plane k+2 are issued; the sharpening s = phi (1 - phi) g/|g| of
// plane k+1 is evaluated for the band and its two ring rows (s_y only); and
// plane k is updated from its face fluxes,
//   F = c_adv u_f (phi_L + phi_R) - c_dif (phi_R - phi_L) + c_shp (s_L + s_R),
// with the x and y faces telescoped and the z face below carried in a
// register -- the expressions of the one-cell-per-thread body (scalar_unit),
// so the result is that body's bit for bit.
#pragma once

#include "cdi_async.cuh"
#include "cdi_fwd_common.cuh"
#include "cdi_reduce.cuh"

namespace cdi {

constexpr int BAND_NT = 256;   // threads of a band block
constexpr int BAND_CPT = 4;    // cells per thread
constexpr int BAND_CELLS = BAND_NT * BAND_CPT;  // largest band (hb * nx)

// Element counts of one ring slot of each staged region (the largest box of the
// batch sets them; every slot starts on a 16-byte boundary).
struct BandSlots {
    int phi;  // (hb + 4) nx + VX, rounded up to VX
    int vel;  // u | v | w regions, each hb nx (v: (hb + 1) nx) + VX, rounded up
    int uo, vo, wo;  // offsets of the u, v and w regions inside a velocity slot
    int sx, sy;  // s_x: hb nx; s_y: (hb + 2) nx
};

__host__ __device__ inline int band_rows(int nx, int ny)
{
    int hb = BAND_CELLS / nx;
    if (hb < 1) hb = 1;
    return hb < ny ? hb : ny;
}

__host__ __device__ inline int round_up(int a, int m) { return (a + m - 1) / m * m; }

// Shared slot sizes for a box of nx x ny (band height hb) in elements of VX per 16 bytes.
__host__ __device__ inline BandSlots band_slots(int nx, int hb, int vx)
{
    BandSlots s;
    s.phi = round_up((hb + 4) * nx + vx, vx);
    s.uo = 0;
    s.vo = round_up(hb * nx + vx, vx);
    s.wo = s.vo + round_up((hb + 1) * nx + vx, vx);
    s.vel = s.wo + round_up(hb * nx + vx, vx);
    s.sx = round_up(hb * nx, vx);
    s.sy = round_up((hb + 2) * nx, vx);
    return s;
}

__host__ __device__ inline size_t band_smem_bytes(const BandSlots &s, size_t esize)
{
    return esize * (size_t)(5 * s.phi + 3 * s.vel + 2 * s.sx + 2 * s.sy);
}

// Staging plan of one region of a unit: `rows` rows of nx values starting at
// row yb (wrapped in y), of which rows [rlo, rhi) do not wrap and form one
// contiguous run of the plane.  Element (r, x) of the region lands in its slot
// at sh + r nx + x, sh = (plane offset + yb nx) mod VX, so that shared and
// global addresses of the run agree modulo 16 bytes.  Everything that does not
// depend on the plane is fixed here once per unit.
struct BandRegion {
    long long run;  // in-plane offset of the run's first element: (yb + rlo) nx
    int dro;        // rlo nx: the run's first element relative to sh
    int len;        // (rhi - rlo) nx
    int a0, sh0;    // run mod VX, yb nx mod VX
    int yb, rows, rlo, rhi;
};

template <int VX>
__device__ __forceinline__ BandRegion band_region(int yb, int rows, int nx, int ny)
{
    BandRegion g;
    g.yb = yb;
    g.rows = rows;
    g.rlo = yb < 0 ? min(-yb, rows) : 0;
    g.rhi = min(ny - yb, rows);
    if (g.rhi < g.rlo) g.rhi = g.rlo;
    g.run = (long long)(yb + g.rlo) * nx;
    g.dro = g.rlo * nx;
    g.len = (g.rhi - g.rlo) * nx;
    g.a0 = (int)(g.run & (VX - 1));
    g.sh0 = (int)(((long long)yb * nx) & (VX - 1));
    return g;
}

// Stage one region of the plane at element offset zoff (am = zoff mod VX) of up
// to two arrays with the same layout (b2 may be NULL) into their slots d1, d2:
// the run by 16-byte chunks and its unaligned ends element-wise, wrapped rows
// element-wise.  Every thread of the block calls it.
template <typename T>
__device__ __forceinline__ void band_stage(const BandRegion &g, T *d1, const T *__restrict__ b1, T *d2,
                                           const T *__restrict__ b2, long long zoff, int am, int nx, int ny,
                                           int tid, unsigned *st)
{
    constexpr int VX = 16 / sizeof(T);
    (void)st;
    const int sh = (am + g.sh0) & (VX - 1);
    const int head = (VX - ((am + g.a0) & (VX - 1))) & (VX - 1);  // elements before a 16-byte boundary
    const long long gA = zoff + g.run;
    T *const r1 = d1 + sh + g.dro;
    T *const r2 = d2 + sh + g.dro;
    const T *const s1 = b1 + gA;
    const T *const s2 = b2 + gA;
    if (g.len > head) {
        const int nch = (g.len - head) / VX, tail = g.len - head - nch * VX;
        for (int c = tid; c < nch; c += BAND_NT) {
            const int o = head + c * VX;
            cp_async<16>(r1 + o, s1 + o);
            if (b2) cp_async<16>(r2 + o, s2 + o);
        }
        int e = -1;
        if (tid < head) e = tid;
        else if (tid >= VX && tid < VX + tail) e = head + nch * VX + (tid - VX);
        if (e >= 0) {
            cp_async<sizeof(T)>(r1 + e, s1 + e);
            if (b2) cp_async<sizeof(T)>(r2 + e, s2 + e);
        }
    } else if (tid < g.len) {
        cp_async<sizeof(T)>(r1 + tid, s1 + tid);
        if (b2) cp_async<sizeof(T)>(r2 + tid, s2 + tid);
    }
    // wrapped rows [0, rlo) and [rhi, rows): element by element
    const int nw = (g.rlo + g.rows - g.rhi) * nx;
    for (int e = tid; e < nw; e += BAND_NT) {
        const int q = e / nx, x = e - q * nx;
        const int r = q < g.rlo ? q : g.rhi + (q - g.rlo);
        const long long go = zoff + CDI_CHK((long long)wrapi(g.yb + r, ny) * nx + x, (long long)nx * ny, st);
        cp_async<sizeof(T)>(d1 + sh + r * nx + x, b1 + go);
        if (b2) cp_async<sizeof(T)>(d2 + sh + r * nx + x, b2 + go);
    }
}

// z index of plane z wrapped into [0, nz) (z within one period of the box in
// the common case, a full modulo otherwise).
__device__ __forceinline__ int band_wrapz(int z, int nz)
{
    if (z >= 0 && z < nz) return z;
    if (z < 0 && z + nz >= 0) return z + nz;
    if (z >= nz && z - nz < nz) return z - nz;
    return wrapi(z, nz);
}

template <typename T>
__device__ __forceinline__ void band_unit(const FwdArgs<T> &a, int y0, int hb, int z0, int z1, const BandSlots &S,
                                          Acc<T> &acc, unsigned char *smem_raw)
{
    constexpr int VX = 16 / sizeof(T);
    constexpr int NT = BAND_NT, CPT = BAND_CPT;
    T *const sphi = reinterpret_cast<T *>(smem_raw);  // [5][S.phi]
    T *const svel = sphi + 5 * S.phi;                  // [3][S.vel]
    T *const ssx = svel + 3 * S.vel;                   // [2][S.sx]
    T *const ssy = ssx + 2 * S.sx;                     // [2][S.sy]

    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long plane = (long long)nx * ny;
    unsigned *const st = a.red.status;
    (void)st;
    const T c_adv = a.c.c_adv, c_dif = a.c.c_dif, c_shp = a.c.c_shp, c_upd = a.c.c_upd;
    const int ncell = hb * nx;

    // Own cells: ci = yl nx + x; bit 2i of xw: x == 0 (x - 1 wraps to nx - 1), bit 2i+1:
    // x == nx - 1 (x + 1 wraps to 0); bit i of own: the cell exists.
    int ci[CPT];
    unsigned xw = 0u, own = 0u;
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
        const int l = tid + i * NT;
        const int yl = l / nx, x = l - yl * nx;
        ci[i] = l < ncell ? l : 0;
        own |= (l < ncell ? 1u : 0u) << i;
        xw |= ((x == 0 ? 1u : 0u) | (x == nx - 1 ? 2u : 0u)) << (2 * i);
    }
    auto dmi = [&](int i) { return (xw >> (2 * i)) & 1u ? nx - 1 : -1; };
    auto dpi = [&](int i) { return (xw >> (2 * i)) & 2u ? 1 - nx : 1; };
    auto owns = [&](int i) { return (own >> i) & 1u; };
    const long long obase = (long long)y0 * nx;  // output offset of band cell 0 in a plane

    const BandRegion gphi = band_region<VX>(y0 - 2, hb + 4, nx, ny);
    const BandRegion guw = band_region<VX>(y0, hb, nx, ny);
    const BandRegion gv = band_region<VX>(y0 - 1, hb + 1, nx, ny);
    const int pm = (int)(plane & (VX - 1));  // plane offset mod VX per plane index

    // shifted slot pointer of the phi plane of wrapped index zw in ring slot `slot`
    auto phi_ptr = [&](int slot, int zw) -> const T * {
        return sphi + slot * S.phi + ((zw * pm + gphi.sh0) & (VX - 1));
    };
    auto issue_phi = [&](int z, int slot) {
        const int zw = band_wrapz(z, nz);
        const long long zo = (long long)zw * plane;
        band_stage<T>(gphi, sphi + slot * S.phi, a.phi, nullptr, nullptr, zo, (zw * pm) & (VX - 1), nx, ny, tid,
                      st);
    };
    auto issue_vel = [&](int z, int slot) {
        T *const d = svel + slot * S.vel;
        const long long zo = (long long)CDI_CHK(z, nz, st) * plane;
        const int am = (z * pm) & (VX - 1);
        band_stage<T>(guw, d + S.uo, a.u, d + S.wo, a.w, zo, am, nx, ny, tid, st);
        band_stage<T>(gv, d + S.vo, a.v, nullptr, nullptr, zo, am, nx, ny, tid, st);
    };

    // sharpening of band row yl (-1 .. hb), column x at plane z: P, Pm, Pp its plane and
    // the planes below and above (shifted slot pointers); i = (yl + 2) nx + x
    auto sharp = [&](const T *P, const T *Pm, const T *Pp, int i, int im, int ip, T &s0, T &s1, T &s2) {
        const T p = P[i];
        const T g0 = P[i + ip] - P[i + im];
        const T g1 = P[i + nx] - P[i - nx];
        const T g2 = Pp[i] - Pm[i];
        const T q = fma(g2, g2, fma(g1, g1, fma(g0, g0, NumLim<T>::tiny())));
        const T inv = rsqrt_t(q);
        const T wgt = p * (T(1) - p) * inv;
        s0 = wgt * g0;
        s1 = wgt * g1;
        s2 = wgt * g2;
    };
    // s_x of the band and s_y of the band and its ring rows at plane z (buffer z & 1),
    // from the plane P and its neighbours Pm, Pp; s_z of the own cells to szo
    auto sharp_plane = [&](int z, const T *P, const T *Pm, const T *Pp, T *szo) {
        T *const sx = ssx + (z & 1) * S.sx;
        T *const sy = ssy + (z & 1) * S.sy;
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
            if (owns(i)) {
                T s0, s1, s2;
                sharp(P, Pm, Pp, ci[i] + 2 * nx, dmi(i), dpi(i), s0, s1, s2);
                sx[ci[i]] = s0;
                sy[ci[i] + nx] = s1;
                szo[i] = s2;
            } else {
                szo[i] = T(0);
            }
        }
        for (int l = tid; l < 2 * nx; l += NT) {  // ring rows -1 and hb: s_y only
            const int top = l >= nx;
            const int x = l - top * nx;
            const int yl = top ? hb : -1;
            T s0, s1, s2;
            sharp(P, Pm, Pp, (yl + 2) * nx + x, x == 0 ? nx - 1 : -1, x == nx - 1 ? 1 - nx : 1, s0, s1, s2);
            sy[(yl + 1) * nx + x] = s1;
        }
    };

    // phi slot of plane z: (z - z0 + 2) mod 5; velocity slot: (z - z0) mod 3.
    __syncthreads();  // the previous unit's readers are done with every slot
    for (int d = 0; d < 5; ++d) issue_phi(z0 - 2 + d, d);  // planes z0-2 .. z0+2
    issue_vel(z0, 0);
    cp_async_commit();
    T wlo[CPT];  // w on the face below plane z0 (own cells)
    {
        const T *src = a.w + (long long)band_wrapz(z0 - 1, nz) * plane + obase;
#pragma unroll
        for (int i = 0; i < CPT; ++i) wlo[i] = owns(i) ? __ldg(src + ci[i]) : T(0);
    }
    // wrapped indices of planes k-1 .. k+2 (k = z0 here), advanced one plane per iteration
    int zm1 = band_wrapz(z0 - 1, nz), zk = band_wrapz(z0, nz), zk1 = band_wrapz(z0 + 1, nz);
    int zk2 = band_wrapz(z0 + 2, nz);
    cp_async_wait<0>();
    __syncthreads();

    // Prologue: s_z at plane z0-1 (own cells), s at plane z0, flux at z0-1/2.
    T szc[CPT], Fzm[CPT];
    {
        const T *Pm2 = phi_ptr(0, band_wrapz(z0 - 2, nz)), *Pm1 = phi_ptr(1, zm1), *P0 = phi_ptr(2, zk);
        T szm[CPT];
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
            T d0, d1;
            szm[i] = T(0);
            if (owns(i)) sharp(Pm1, Pm2, P0, ci[i] + 2 * nx, dmi(i), dpi(i), d0, d1, szm[i]);
        }
        sharp_plane(z0, P0, Pm1, phi_ptr(3, zk1), szc);
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
            const T pm_ = Pm1[ci[i] + 2 * nx], pc = P0[ci[i] + 2 * nx];
            Fzm[i] = flux(c_adv * wlo[i], c_dif, c_shp, pm_, pc, szm[i], szc[i]);
        }
    }
    // plane z0+3 reuses the slot of plane z0-2, which the prologue just read
    __syncthreads();
    if (z0 + 3 <= z1 + 1) issue_phi(z0 + 3, 0);
    if (z0 + 1 < z1) issue_vel(z0 + 1, 1);
    cp_async_commit();

    int pk = 2, vk = 0;  // ring slots of phi plane k and of the velocities of plane k
    for (int k = z0; k < z1; ++k) {
        const int pk1 = pk == 4 ? 0 : pk + 1, pk2 = pk1 == 4 ? 0 : pk1 + 1;
        const int pkm = pk == 0 ? 4 : pk - 1;  // also the slot of plane k+4
        const int vkm = vk == 0 ? 2 : vk - 1;  // also the slot of plane k+2
        // phi plane k+2 and the velocities of plane k have landed, and every thread
        // has left iteration k-1 (its slots and s buffer are free)
        cp_async_wait<1>();
        __syncthreads();
        if (k + 4 <= z1 + 1) issue_phi(k + 4, pkm);
        if (k + 2 < z1) issue_vel(k + 2, vkm);
        cp_async_commit();

        // sharpening at plane k+1 (buffer (k+1)&1; the fluxes below read buffer k&1):
        // the ring rows first, then cell by cell together with the cell's update at
        // plane k, so that the chains of a thread's cells overlap
        const T *Pk = phi_ptr(pk, zk), *Pk1 = phi_ptr(pk1, zk1), *Pk2 = phi_ptr(pk2, zk2);
        T *const sxw = ssx + ((k + 1) & 1) * S.sx;
        T *const syw = ssy + ((k + 1) & 1) * S.sy;
        for (int l = tid; l < 2 * nx; l += NT) {  // ring rows -1 and hb: s_y only
            const int top = l >= nx;
            const int x = l - top * nx;
            const int yl = top ? hb : -1;
            T s0, s1, s2;
            sharp(Pk1, Pk, Pk2, (yl + 2) * nx + x, x == 0 ? nx - 1 : -1, x == nx - 1 ? 1 - nx : 1, s0, s1, s2);
            syw[(yl + 1) * nx + x] = s1;
        }

        // fluxes and update at plane k
        const T *sx = ssx + (k & 1) * S.sx, *sy = ssy + (k & 1) * S.sy;
        const T *vel = svel + vk * S.vel;
        const int am = (k * pm) & (VX - 1);
        const T *U = vel + S.uo + ((am + guw.sh0) & (VX - 1));
        const T *V = vel + S.vo + ((am + gv.sh0) & (VX - 1));
        const T *W = vel + S.wo + ((am + guw.sh0) & (VX - 1));
        T *const outp = a.out + (long long)CDI_CHK(k, nz, st) * plane + obase;
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
            if (!owns(i)) continue;
            const int c = ci[i], p = c + 2 * nx, dm = dmi(i), dp = dpi(i);
            T szn;
            {
                T s0, s1;
                sharp(Pk1, Pk, Pk2, p, dm, dp, s0, s1, szn);
                sxw[c] = s0;
                syw[c + nx] = s1;
            }
            const T pc = Pk[p];
            const T pxm = Pk[p + dm], pxp = Pk[p + dp];
            const T pym = Pk[p - nx], pyp = Pk[p + nx];
            const T pzp = Pk1[p];
            const T sxm = sx[c + dm], sxp = sx[c + dp];
            const T sym = sy[c], syp = sy[c + 2 * nx];
            const T uc = U[c], um = U[c + dm];
            const T vc = V[c + nx], vm = V[c];
            const T wc = W[c];
            T adv = uc * (pc + pxp);
            adv = fma(-um, pxm + pc, adv);
            adv = fma(vc, pc + pyp, adv);
            adv = fma(-vm, pym + pc, adv);
            const T dif = fma(T(-4), pc, (pxm + pxp) + (pym + pyp));
            const T shp = (sxp - sxm) + (syp - sym);
            const T Fzp = flux(c_adv * wc, c_dif, c_shp, pc, pzp, szc[i], szn);
            const T div = fma(c_adv, adv, fma(-c_dif, dif, fma(c_shp, shp, Fzp - Fzm[i])));
            const T o = fma(-c_upd, div, pc);
            outp[CDI_CHK(c, plane - obase, st)] = o;
            acc.add(o, a.c.tol);
            Fzm[i] = Fzp;
            szc[i] = szn;
        }
        pk = pk1;
        vk = vk == 2 ? 0 : vk + 1;
        zk = zk1;
        zk1 = zk2;
        zk2 = zk2 + 1 == nz ? 0 : zk2 + 1;
    }
    cp_async_wait<0>();
}

}  // namespace cdi
