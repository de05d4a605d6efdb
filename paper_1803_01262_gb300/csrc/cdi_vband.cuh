// Vector row-band unit body of the batched CDI step, on the batch's padded copy
// of each box.
//
// The batch keeps its own copy of every box in a padded layout: each row of nx
// cells sits at offset GH = VX (one 16-byte vector) inside a row of pitch
// P = round_up(nx + 2 VX, VX) elements, and the VX positions on either side of
// the row hold its periodic continuation (ghost cells: position GH + x holds
// phi at x mod nx for x in [-VX, nx + VX)).  Rows and planes then start on
// 16-byte boundaries whatever nx is, so a unit -- a band of whole rows
// [y0, y0 + hb) and a range of planes [z0, z1) -- is staged by 16-byte copies
// only (each thread's few vectors of a region planned once per unit, rows
// outside [0, ny) wrapped in y), and
// each thread owns one group of VX consecutive cells of the band, read with
// 16-byte shared loads like the single-box vector kernel (fwd_vec_kernel): the
// x neighbours of a group are its first and last neighbours in the padded row,
// the ghosts at the row ends.  s_x at x = -1 and x = nx is s_x at nx - 1 and 0
// (s is periodic with phi); a partial last group (nx % VX != 0) evaluates s at
// its ghost cells from their ghost neighbours, the periodic values.
//
// Per plane k (one barrier): phi plane k+4 and the velocities of plane k+2 are
// issued; the sharpening s = phi (1 - phi) g/|g| of plane k+1 is evaluated for
// the band's groups and (s_y only) its two ring rows; plane k is updated from
// its face fluxes, the x and y faces telescoped and the z face below carried --
// fwd_vec_kernel's expressions in its order, so the field is the other
// kernels' bit for bit.  The output goes to the padded copy of the next state
// (interior and ghost cells) and, on the last step of a call (final), also to
// the caller's array.
#pragma once

#include "cdi_async.cuh"
#include "cdi_fwd_common.cuh"
#include "cdi_reduce.cuh"

namespace cdi {

constexpr int VBAND_NT = 256;  // threads of a vector band block (one cell group each)

// Padded layout of a box: row pitch in elements (VX = 16 / sizeof(T)).
__host__ __device__ inline int vband_pitch(int nx, int vx) { return (nx + 2 * vx + vx - 1) / vx * vx; }

// Rows per band: as many whole rows as there are thread groups for, and few
// enough that each thread copies at most VBAND_CPY 16-byte vectors of a staged
// region per plane (the phi region is hb + 4 padded rows).  0: a padded row is
// too wide for that (then the body does not apply).
constexpr int VBAND_CPY = 2;
__host__ __device__ inline int vband_rows(int nx, int ny, int vx)
{
    const int g = (nx + vx - 1) / vx;
    const int nv = vband_pitch(nx, vx) / vx;
    int hb = VBAND_NT / g;
    const int cap = VBAND_CPY * VBAND_NT / nv - 4;
    if (hb > cap) hb = cap;
    if (hb < 1) return 0;
    return hb < ny ? hb : ny;
}

// Ring-slot sizes (elements; multiples of VX) for the largest box of a batch.
struct VbandSlots {
    int phi;          // (hb + 4) P
    int vel;          // u | v | w: hb P, (hb + 1) P, hb P
    int vo, wo;       // offsets of v and w in a velocity slot (u at 0)
    int sx, sy;       // hb P and (hb + 2) P
};

__host__ __device__ inline VbandSlots vband_slots(int P, int hb)
{
    VbandSlots s;
    s.phi = (hb + 4) * P;
    s.vo = hb * P;
    s.wo = s.vo + (hb + 1) * P;
    s.vel = s.wo + hb * P;
    s.sx = hb * P;
    s.sy = (hb + 2) * P;
    return s;
}

__host__ __device__ inline size_t vband_smem_bytes(const VbandSlots &s, size_t esize)
{
    return esize * (size_t)(5 * s.phi + 3 * s.vel + 2 * s.sx + 2 * s.sy);
}

// phi around a thread's group at one plane: the group, the groups above and below
// it in y, and its x neighbours (carried from the sharpening at plane k+1 to the
// update at plane k+1 in the next iteration).
template <typename T, int VX>
struct PhiNb {
    T c[VX], yn[VX], yp[VX];
    T L, R;
};

// Staging plan of one region -- `rows` padded rows from row yb (wrapped in y)
// -- for this thread: the in-plane offsets of its (at most VBAND_CPY) 16-byte
// vectors, chunk c = tid + i VBAND_NT of the region landing at c VX in the
// slot; -1 where the thread has no such chunk.  Fixed per unit; a plane adds
// only its base pointer.
template <int VX>
__device__ __forceinline__ void vband_plan(int *g, int yb, int rows, int P, int ny, int tid, unsigned *st)
{
    (void)st;
    const int nv = P / VX;
#pragma unroll
    for (int i = 0; i < VBAND_CPY; ++i) {
        const int c = tid + i * VBAND_NT;
        if (c < rows * nv) {
            const int row = c / nv;
            g[i] = CDI_CHK(wrapi(yb + row, ny), ny, st) * P + (c - row * nv) * VX;
        } else {
            g[i] = -1;
        }
    }
}

template <typename T>
__device__ __forceinline__ void vband_unit(const FwdArgs<T> &a, const T *__restrict__ pin, T *__restrict__ pout,
                                           const T *__restrict__ pu, const T *__restrict__ pv,
                                           const T *__restrict__ pw, int P, bool final_write, int y0, int hb,
                                           int z0, int z1, const VbandSlots &S, Acc<T> &acc,
                                           unsigned char *smem_raw)
{
    constexpr int VX = 16 / sizeof(T), GH = VX, NT = VBAND_NT;
    using VV = V16<T>;
    T *const sphi = reinterpret_cast<T *>(smem_raw);  // [5][S.phi]
    T *const svel = sphi + 5 * S.phi;                  // [3][S.vel]
    T *const ssx = svel + 3 * S.vel;                   // [2][S.sx]
    T *const ssy = ssx + 2 * S.sx;                     // [2][S.sy]

    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long planeP = (long long)P * ny;        // padded plane
    const long long plane = (long long)nx * ny;        // the caller's plane
    unsigned *const st = a.red.status;
    (void)st;
    const T c_adv = a.c.c_adv, c_dif = a.c.c_dif, c_shp = a.c.c_shp, c_upd = a.c.c_upd;

    const int G = (nx + VX - 1) / VX;    // groups per row
    const int hbe = min(hb, ny - y0);    // rows of this band
    const int r = tid / G, j = tid - r * G;
    const bool act = r < hbe;            // this thread owns group j of band row r
    const int x0 = j * VX;
    const int nown = act ? min(VX, nx - x0) : 0;  // cells of the group inside the row
    const int pos = (r + 2) * P + GH + x0;  // the group in a phi slot
    const int sxo = r * P + GH + x0;        // ... in s_x
    const int syo = (r + 1) * P + GH + x0;  // ... in s_y (row 0: the ring row below)
    const int dL = x0 == 0 ? nx : 0;                   // s_x left of x = 0 is s_x(nx - 1)
    const int dR = x0 + VX == nx ? -nx : 0;            // right of x = nx - 1 (full last group): s_x(0)
    // ghost copies of the group's cells: bit 2i, cell i feeds the left ghost at x - nx;
    // bit 2i+1, the right ghost at x + nx (nx >= GH; smaller rows take every copy)
    unsigned gmask = 0u;
#pragma unroll
    for (int i = 0; i < VX; ++i) {
        const int x = x0 + i;
        if (i < nown) gmask |= ((x >= nx - GH ? 1u : 0u) | (x < GH ? 2u : 0u)) << (2 * i);
    }

    // sharpening of the group at phi-slot offset off of plane Pm (below Pmm, above Pmp);
    // zn_in (nullable): the group at the plane below, already loaded; nb_out (nullable):
    // receives phi around the group at this plane (the own group's next update reads it)
    auto sharp_group = [&](const T *Pm, const T *Pmm, const T *Pmp, int off, T *s0, T *s1, T *s2,
                           const T *zn_in = nullptr, PhiNb<T, VX> *nb_out = nullptr) {
        T c[VX], yn[VX], yp[VX], zn[VX], zp[VX];
        VV::ld(c, Pm + off);
        VV::ld(yn, Pm + off - P);
        VV::ld(yp, Pm + off + P);
        if (zn_in) {
#pragma unroll
            for (int i = 0; i < VX; ++i) zn[i] = zn_in[i];
        } else {
            VV::ld(zn, Pmm + off);
        }
        VV::ld(zp, Pmp + off);
        const T L = Pm[off - 1], R = Pm[off + VX];
        if (nb_out) {
#pragma unroll
            for (int i = 0; i < VX; ++i) {
                nb_out->c[i] = c[i];
                nb_out->yn[i] = yn[i];
                nb_out->yp[i] = yp[i];
            }
            nb_out->L = L;
            nb_out->R = R;
        }
#pragma unroll
        for (int i = 0; i < VX; ++i) {
            const T g0 = (i + 1 < VX ? c[i + 1] : R) - (i > 0 ? c[i - 1] : L);
            const T g1 = yp[i] - yn[i];
            const T g2 = zp[i] - zn[i];
            const T q = fma(g2, g2, fma(g1, g1, fma(g0, g0, NumLim<T>::tiny())));
            const T inv = rsqrt_t(q);
            const T wgt = c[i] * (T(1) - c[i]) * inv;
            s0[i] = wgt * g0;
            s1[i] = wgt * g1;
            s2[i] = wgt * g2;
        }
    };
    // s_y of the ring rows (below and above the band) at a plane
    auto sharp_ring = [&](const T *Pm, const T *Pmm, const T *Pmp, T *sy) {
        for (int l = NT - 1 - tid; l < 2 * G; l += NT) {  // the threads without a group first
            const int top = l >= G;
            const int jj = l - top * G;
            const int row = top ? hbe : -1;
            T s0[VX], s1[VX], s2[VX];
            sharp_group(Pm, Pmm, Pmp, (row + 2) * P + GH + jj * VX, s0, s1, s2);
            VV::st(sy + (row + 1) * P + GH + jj * VX, s1);
        }
    };

    // this thread's chunks of the staged regions: phi, u and w (same rows), v
    int gphi[VBAND_CPY], guw[VBAND_CPY], gv[VBAND_CPY];
    vband_plan<VX>(gphi, y0 - 2, hbe + 4, P, ny, tid, st);
    vband_plan<VX>(guw, y0, hbe, P, ny, tid, st);
    vband_plan<VX>(gv, y0 - 1, hbe + 1, P, ny, tid, st);
    // phi plane of wrapped index zw into ring slot `slot`
    auto issue_phi = [&](int zw, int slot) {
        const T *const src = pin + (long long)zw * planeP;
        T *const d = sphi + slot * S.phi + tid * VX;
#pragma unroll
        for (int i = 0; i < VBAND_CPY; ++i)
            if (gphi[i] >= 0) cp_async<16>(d + i * VBAND_NT * VX, src + gphi[i]);
    };
    auto issue_vel = [&](int z, int slot) {
        const long long zo = (long long)CDI_CHK(z, nz, st) * planeP;
        T *const d = svel + slot * S.vel + tid * VX;
#pragma unroll
        for (int i = 0; i < VBAND_CPY; ++i) {
            if (guw[i] >= 0) {
                cp_async<16>(d + i * VBAND_NT * VX, pu + zo + guw[i]);
                cp_async<16>(d + S.wo + i * VBAND_NT * VX, pw + zo + guw[i]);
            }
            if (gv[i] >= 0) cp_async<16>(d + S.vo + i * VBAND_NT * VX, pv + zo + gv[i]);
        }
    };

    // phi slot of plane z: (z - z0 + 2) mod 5; velocity slot: (z - z0) mod 3.
    __syncthreads();  // the previous unit's readers are done with every slot
    for (int d = 0; d < 5; ++d) issue_phi(wrapi(z0 - 2 + d, nz), d);  // planes z0-2 .. z0+2
    issue_vel(z0, 0);
    cp_async_commit();
    T wlo[VX];  // w on the face below plane z0 (own cells)
    if (act) VV::ld(wlo, pw + (long long)wrapi(z0 - 1, nz) * planeP + (long long)(y0 + r) * P + GH + x0);
    cp_async_wait<0>();
    __syncthreads();

    // Prologue: s_z at plane z0-1 (own), s at plane z0 (own + ring), flux at z0-1/2.
    T szc[VX], Fzm[VX], sxk[VX];  // sxk: the own group's s_x at plane k
    {
        const T *Pm2 = sphi, *Pm1 = sphi + S.phi, *P0 = sphi + 2 * S.phi, *P1 = sphi + 3 * S.phi;
        T *const sx = ssx + (z0 & 1) * S.sx;
        T *const sy = ssy + (z0 & 1) * S.sy;
        if (act) {
            T a0[VX], a1[VX], szm[VX], s0[VX], s1[VX];
            sharp_group(Pm1, Pm2, P0, pos, a0, a1, szm);
            sharp_group(P0, Pm1, P1, pos, s0, s1, szc);
            VV::st(sx + sxo, s0);
#pragma unroll
            for (int i = 0; i < VX; ++i) sxk[i] = s0[i];
            VV::st(sy + syo, s1);
            T pm[VX], pc[VX];
            VV::ld(pm, Pm1 + pos);
            VV::ld(pc, P0 + pos);
#pragma unroll
            for (int i = 0; i < VX; ++i) Fzm[i] = flux(c_adv * wlo[i], c_dif, c_shp, pm[i], pc[i], szm[i], szc[i]);
        }
        sharp_ring(P0, Pm1, P1, sy);
    }
    // plane z0+3 reuses the slot of plane z0-2, which the prologue just read
    __syncthreads();
    int zq = wrapi(z0 + 3, nz);  // wrapped index of the next phi plane to stage
    if (z0 + 3 <= z1 + 1) issue_phi(zq, 0);
    if (z0 + 1 < z1) issue_vel(z0 + 1, 1);
    cp_async_commit();

    PhiNb<T, VX> cur;  // phi around the own group at plane z0 (slot 2)
    if (act) {
        const T *const P0 = sphi + 2 * S.phi + pos;
        VV::ld(cur.c, P0);
        VV::ld(cur.yn, P0 - P);
        VV::ld(cur.yp, P0 + P);
        cur.L = P0[-1];
        cur.R = P0[VX];
    }
    int pk = 2, vk = 0;  // ring slots of phi plane k and of the velocities of plane k
    // two planes per pass: the carried values (cur / nxt, s_x, s_z, the z flux)
    // alternate between two register sets instead of being copied
#pragma unroll 2
    for (int k = z0; k < z1; ++k) {
        const int pk1 = pk == 4 ? 0 : pk + 1, pk2 = pk1 == 4 ? 0 : pk1 + 1;
        const int pkm = pk == 0 ? 4 : pk - 1;  // also the slot of plane k+4
        const int vk2 = vk == 0 ? 2 : vk - 1;  // also the slot of plane k+2
        // phi plane k+2 and the velocities of plane k have landed, and every thread
        // has left iteration k-1
        cp_async_wait<1>();
        __syncthreads();
        zq = zq + 1 == nz ? 0 : zq + 1;  // plane k+4
        if (k + 4 <= z1 + 1) issue_phi(zq, pkm);
        if (k + 2 < z1) issue_vel(k + 2, vk2);
        cp_async_commit();

        const T *Pk = sphi + pk * S.phi, *Pk1 = sphi + pk1 * S.phi, *Pk2 = sphi + pk2 * S.phi;
        T *const sxw = ssx + ((k + 1) & 1) * S.sx;
        T *const syw = ssy + ((k + 1) & 1) * S.sy;
        // sharpening at plane k+1: the ring rows, then the own group (s_z kept)
        sharp_ring(Pk1, Pk, Pk2, syw);
        if (act) {
            T szn[VX];
            PhiNb<T, VX> nxt;  // phi around the group at plane k+1
            T sxn[VX];  // s_x of the group at plane k+1
            {
                T s1[VX];
                sharp_group(Pk1, Pk, Pk2, pos, sxn, s1, szn, cur.c, &nxt);
                VV::st(sxw + sxo, sxn);
                VV::st(syw + syo, s1);
            }
            // fluxes and update at plane k (s of plane k: buffer k & 1, written before the barrier)
            const T *sx = ssx + (k & 1) * S.sx, *sy = ssy + (k & 1) * S.sy;
            const T *vel = svel + vk * S.vel;
            // phi around the group at plane k, carried from the previous iteration
            const T *const c = cur.c, *const yn = cur.yn, *const yp = cur.yp, *const zp = nxt.c;
            const T L = cur.L, R = cur.R;
            const T *const sxc = sxk;
            T syn[VX], syp[VX];
            VV::ld(syn, sy + syo - P);
            VV::ld(syp, sy + syo + P);
            const T sxL = sx[sxo - 1 + dL], sxR = sx[sxo + VX + dR];
            const T *ur = vel + r * P + GH + x0;
            const T *vr = vel + S.vo + (r + 1) * P + GH + x0;
            const T *wr = vel + S.wo + r * P + GH + x0;
            T uc[VX], vc[VX], vn[VX], wc[VX];
            VV::ld(uc, ur);
            VV::ld(vc, vr);
            VV::ld(vn, vr - P);
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
                o[i] = fma(-c_upd, div, c[i]);
                Fzm[i] = Fzp;
                szc[i] = szn[i];
            }
            // the padded copy of the next state: the group, and the ghost cells it feeds
            T *const orow = pout + (long long)CDI_CHK(k, nz, st) * planeP + (long long)(y0 + r) * P + GH;
            if (nown == VX) {
                VV::st(orow + x0, o);
            } else {
#pragma unroll
                for (int i = 0; i < VX; ++i)
                    if (i < nown) orow[x0 + i] = o[i];
            }
            acc.template add_group_n<VX>(o, nown, a.c.tol);
            if (gmask) {  // cells within GH of a row end: their ghost copies
                if (nx >= GH) {
#pragma unroll
                    for (int i = 0; i < VX; ++i) {
                        if ((gmask >> (2 * i)) & 1u) orow[x0 + i - nx] = o[i];
                        if ((gmask >> (2 * i)) & 2u) orow[x0 + i + nx] = o[i];
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < VX; ++i) {
                        if (i >= nown) continue;
                        const int x = x0 + i;
                        for (int g = x - nx; g >= -GH; g -= nx) orow[g] = o[i];
                        for (int g = x + nx; g < nx + GH; g += nx) orow[g] = o[i];
                    }
                }
            }
            if (final_write) {  // the caller's array (rows at any 4-byte boundary: element stores)
                T *const urow = a.out + (long long)k * plane + (long long)(y0 + r) * nx + x0;
#pragma unroll
                for (int i = 0; i < VX; ++i)
                    if (i < nown) urow[i] = o[i];
            }
            cur = nxt;
#pragma unroll
            for (int i = 0; i < VX; ++i) sxk[i] = sxn[i];
        }
        pk = pk1;
        vk = vk == 2 ? 0 : vk + 1;
    }
    cp_async_wait<0>();
}

}  // namespace cdi
