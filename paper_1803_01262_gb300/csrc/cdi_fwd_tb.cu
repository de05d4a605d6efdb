// Two explicit CDI steps per pass (temporal blocking of depth 2).
//
// The Euler step of Section 2.2 (per face between L and R along d:
//   F = c_adv u_f (phi_L + phi_R) - c_dif (phi_R - phi_L) + c_shp (s_L + s_R),
//   s = phi (1 - phi) g/|g|,  phi'_c = phi_c - c_upd sum_d (F_{c+1/2} - F_{c-1/2}))
// is applied twice in one pass over the box: a block owns an x-y tile of
// W x H cells and marches along z; at plane j it
//   step 1: evaluates s at plane j+1 and phi^1 at plane j on the tile grown by
//           two cells on each side (the halo the second step's stencil reads),
//           from phi^0 staged with a halo of four, into a shared ring of phi^1
//           planes -- phi^1 never goes to memory;
//   step 2: evaluates s^1 at plane j-2 and phi^2 at plane j-3 on the tile from
//           that ring, and writes phi^2.
// So phi is read and written once per two steps, and the face velocities --
// 12 of the 20 bytes a single step moves per cell in FP32 -- are read once:
// step 1 stages them with its tile, step 2 takes its own tile's faces again
// from L2 (they were read from memory three planes earlier).  The price is the
// grown tile of step 1 (72 x 20 cells for a 64 x 16 tile in FP32, 1.41 x the
// work of the tile) and one block per SM (165 KB of shared memory).
//
// Threads own 16-byte vectors of x-cells as in fwd_vec_kernel: threads
// [0, TX1 TY1) the vectors of step 1's grown tile, [0, TX TY) those of step 2's
// tile; the sharpening rings (one cell beyond each tile along x and y) go to
// threads left idle by the other step; every thread issues a share of the
// 16-byte cp.async copies.  One barrier per plane: every phase reads only data
// written before it.  Each step's outputs on the tile (planes of the unit) are
// folded into its own statistics partial; the last block writes the second
// step's record and folds both steps into the run accumulators.
#include "cdi_async.cuh"
#include "cdi_fwd_common.cuh"
#include "cdi_internal.cuh"
#include "cdi_reduce.cuh"

namespace cdi {

template <typename T>
struct TbCfg {
    static constexpr int VX = 16 / sizeof(T);
    static constexpr int TX = 16, TY = 16;          // step-2 vectors (the tile)
    static constexpr int W = TX * VX, H = TY;
    static constexpr int TX1 = TX + 2, TY1 = H + 4; // step-1 vectors: x0-VX .. x0+W+VX, y0-2 .. y0+H+1
    static constexpr int W1 = W + 2 * VX;
    static constexpr int N1 = TX1 * TY1, N2 = TX * TY;
    static constexpr int NT = 448;                   // 14 warps
    static_assert(N1 <= NT && N2 <= NT, "threads");
    // phi^0 ring: rows y0-4 .. y0+H+3, columns x0-2VX .. x0+W+2VX-1
    static constexpr int PP0 = W + 4 * VX, PR0 = H + 8, PHI0 = PR0 * PP0;
    // phi^1 ring: rows y0-2 .. y0+H+1, columns x0-VX .. x0+W+VX-1
    static constexpr int PP1 = W1, PR1 = H + 4, PHI1 = PR1 * PP1;
    // step-1 sharpening: s_x rows y0-2 .. y0+H+1, columns x0-VX-1 .. x0+W+VX (at VX-1 .. VX+W1);
    // s_y rows y0-3 .. y0+H+2, columns x0-VX .. x0+W+VX-1
    static constexpr int SXP0 = W1 + 2 * VX, SXS0 = TY1 * SXP0, SYS0 = (TY1 + 2) * W1;
    // step-2 sharpening: s_x rows y0 .. y0+H-1, columns x0-1 .. x0+W (at VX-1 .. VX+W);
    // s_y rows y0-1 .. y0+H
    static constexpr int SXP1 = W + 2 * VX, SXS1 = H * SXP1, SYS1 = (H + 2) * W;
    // step-1 velocities: u rows y0-2 .. y0+H+1, columns x0-2VX .. x0+W+VX-1;
    // v rows y0-3 .. y0+H+1, w rows y0-2 .. y0+H+1, columns x0-VX .. x0+W+VX-1
    static constexpr int UP = W + 3 * VX, USZ = TY1 * UP, VSZ = (TY1 + 1) * W1, WSZ = TY1 * W1;
    static constexpr int VEL = USZ + VSZ + WSZ;
    static constexpr int NSP0 = 5, NSP1 = 5, NSV = 3;
    static constexpr int CPHI = PHI0 / VX, CU = USZ / VX, CV = VSZ / VX, CW = WSZ / VX;
    static constexpr int CVEL = CU + CV + CW;
    static constexpr int RPHI = (CPHI + NT - 1) / NT, RVEL = (CVEL + NT - 1) / NT;
    static constexpr size_t bytes =
        sizeof(T) * (size_t)(NSP0 * PHI0 + NSP1 * PHI1 + NSV * VEL + 2 * SXS0 + 2 * SYS0 + 2 * SXS1 + 2 * SYS1);
};

template <typename T>
__global__ void __launch_bounds__(TbCfg<T>::NT, 1)
fwd_tb2_kernel(const FwdArgs<T> a, const T c_adv2, const int nchunks)
{
    using C = TbCfg<T>;
    using VV = V16<T>;
    constexpr int VX = C::VX, W = C::W, H = C::H, TX = C::TX, TX1 = C::TX1, TY1 = C::TY1;
    constexpr int PP0 = C::PP0, PP1 = C::PP1, SXP0 = C::SXP0, SXP1 = C::SXP1, W1 = C::W1, UP = C::UP;
    constexpr int NT = C::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *const sphi0 = reinterpret_cast<T *>(smem_raw);  // [NSP0][PHI0]
    T *const sphi1 = sphi0 + C::NSP0 * C::PHI0;         // [NSP1][PHI1]
    T *const svel = sphi1 + C::NSP1 * C::PHI1;          // [NSV][VEL] = u | v | w
    T *const ssx0 = svel + C::NSV * C::VEL;             // [2][SXS0]
    T *const ssy0 = ssx0 + 2 * C::SXS0;                 // [2][SYS0]
    T *const ssx1 = ssy0 + 2 * C::SYS0;                 // [2][SXS1]
    T *const ssy1 = ssx1 + 2 * C::SXS1;                 // [2][SYS1]

    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long plane = (long long)nx * ny;
    const int tiles_x = (nx + W - 1) / W;
    const int ntiles = tiles_x * ((ny + H - 1) / H);
    const T c_dif = a.c.c_dif, c_shp = a.c.c_shp, c_upd = a.c.c_upd;
    const T c_adv1 = a.c.c_adv;
    unsigned *const st = a.red.status;
    (void)st;

    // step 1: vector (g1x, g1y) of the grown tile; step 2: vector (g2x, g2y) of the tile
    const bool is1 = tid < C::N1, is2 = tid < C::N2;
    const int g1x = tid % TX1, g1y = tid / TX1;
    const int g2x = tid % TX, g2y = tid / TX;
    // ring items: step 1 (threads N1 ..): s_y of rows -1, TY1 (TX1 vectors each), then s_x
    // of columns -1, TX1 VX (TY1 cells each); step 2 (threads N2 ..): s_y of rows -1, H, then
    // s_x of columns -1, W
    const int r1 = tid - C::N1, r2 = tid - C::N2;
    const bool ring1y = r1 >= 0 && r1 < 2 * TX1;
    const bool ring1x = r1 >= 2 * TX1 && r1 < 2 * TX1 + 2 * TY1;
    const bool ring2y = r2 >= 0 && r2 < 2 * TX;
    const bool ring2x = r2 >= 2 * TX && r2 < 2 * TX + 2 * H;

    // Normals and sharpening of the VX cells at offset off of a plane with pitch PP
    // (Pm, Pmm, Pmp: the plane and the ones below and above).
    auto sharp_vec = [&](const T *Pm, const T *Pmm, const T *Pmp, int off, int pitch, T *s0, T *s1, T *s2) {
        T c[VX], yn[VX], yp[VX], zn[VX], zp[VX];
        VV::ld(c, Pm + off);
        VV::ld(yn, Pm + off - pitch);
        VV::ld(yp, Pm + off + pitch);
        VV::ld(zn, Pmm + off);
        VV::ld(zp, Pmp + off);
        const T L = Pm[off - 1], R = Pm[off + VX];
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
    auto sharp_x = [&](const T *Pm, const T *Pmm, const T *Pmp, int off, int pitch) {
        const T p = Pm[off];
        const T g0 = Pm[off + 1] - Pm[off - 1];
        const T g1 = Pm[off + pitch] - Pm[off - pitch];
        const T g2 = Pmp[off] - Pmm[off];
        const T q = fma(g2, g2, fma(g1, g1, fma(g0, g0, NumLim<T>::tiny())));
        return p * (T(1) - p) * rsqrt_t(q) * g0;  // s_x only
    };
    // The update of the VX cells at offset po of plane P (pitch pp; Pp the plane above),
    // s_x at sxr (row of the vector, pitch-aligned, with the x-ring cells at sxr[-1] and
    // sxr[VX]), s_y rows syn / syp, velocities uc (+ uL left of it), vc, vn, wc; carried
    // Fzm and szc, szn the s_z of this plane and the next.
    auto update = [&](const T *P, const T *Pp, int po, int pp, const T *sxr, const T *syn_r, const T *syp_r,
                      const T *uc, T uL, const T *vc, const T *vn, const T *wc, T cadv, T *szc, const T *szn,
                      T *Fzm, T *o) {
        T c[VX], yn[VX], yp[VX], zp[VX], sxc[VX], syn[VX], syp[VX];
        VV::ld(c, P + po);
        VV::ld(yn, P + po - pp);
        VV::ld(yp, P + po + pp);
        VV::ld(zp, Pp + po);
        const T L = P[po - 1], R = P[po + VX];
        VV::ld(sxc, sxr);
        VV::ld(syn, syn_r);
        VV::ld(syp, syp_r);
        const T sxL = sxr[-1], sxR = sxr[VX];
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
            const T Fzp = flux(cadv * wc[i], c_dif, c_shp, c[i], zp[i], szc[i], szn[i]);
            const T div = fma(cadv, adv, fma(-c_dif, dif, fma(c_shp, shp, Fzp - Fzm[i])));
            o[i] = fma(-c_upd, div, c[i]);
            Fzm[i] = Fzp;
            szc[i] = szn[i];
        }
    };

    Acc<T> acc1, acc2;
    acc1.init();
    acc2.init();

    UnitIter<W, H> units(ntiles, nz, nchunks);
    Unit un;
    while (units.next(un, ntiles, tiles_x, nz, nchunks)) {
        const int x0 = un.x0, y0 = un.y0, z0 = un.z0, z1 = un.z1;
        const int j0 = z0 - 2, j1 = z1 + 2;  // step 1 produces phi^1 planes [j0, j1)

        // In-plane offsets of this thread's copy chunks (each thread a share of
        // every plane): phi^0 chunks e = tid + r NT; velocity chunks likewise over
        // u | v | w (the region in the top two bits).
        int gphi[C::RPHI], gvel[C::RVEL];
#pragma unroll
        for (int r = 0; r < C::RPHI; ++r) {
            const int e = tid + r * NT, row = e / (PP0 / VX), col = e - row * (PP0 / VX);
            gphi[r] = e < C::CPHI
                ? (int)CDI_CHK(wrapi(y0 - 4 + row, ny) * nx + wrapi(x0 - 2 * VX + col * VX, nx), plane - VX + 1, st)
                : 0;
        }
#pragma unroll
        for (int r = 0; r < C::RVEL; ++r) {
            const int e = tid + r * NT;
            int off = 0;
            if (e < C::CU) {
                const int row = e / (UP / VX), col = e - row * (UP / VX);
                off = wrapi(y0 - 2 + row, ny) * nx + wrapi(x0 - 2 * VX + col * VX, nx);
            } else if (e < C::CU + C::CV) {
                const int q = e - C::CU, row = q / (W1 / VX), col = q - row * (W1 / VX);
                off = wrapi(y0 - 3 + row, ny) * nx + wrapi(x0 - VX + col * VX, nx);
            } else if (e < C::CVEL) {
                const int q = e - C::CU - C::CV, row = q / (W1 / VX), col = q - row * (W1 / VX);
                off = wrapi(y0 - 2 + row, ny) * nx + wrapi(x0 - VX + col * VX, nx);
            }
            gvel[r] = (int)CDI_CHK(off, plane - VX + 1, st);
        }
        auto issue_phi = [&](int z, int slot) {
            const T *src = a.phi + (long long)wrapi(z, nz) * plane;
            T *dst = sphi0 + slot * C::PHI0;
#pragma unroll
            for (int r = 0; r < C::RPHI; ++r) {
                const int e = tid + r * NT;
                if (e < C::CPHI) cp_async<16>(dst + e * VX, src + gphi[r]);
            }
        };
        auto issue_vel = [&](int z, int slot) {
            const long long zo = (long long)wrapi(z, nz) * plane;
            T *dst = svel + slot * C::VEL;
#pragma unroll
            for (int r = 0; r < C::RVEL; ++r) {
                const int e = tid + r * NT;
                if (e < C::CVEL) {
                    const T *src = e < C::CU ? a.u : e < C::CU + C::CV ? a.v : a.w;
                    cp_async<16>(dst + e * VX, src + zo + gvel[r]);
                }
            }
        };
        // phi^0 slot of plane z: (z - j0 + 2) mod 5; velocity slot (z - j0) mod 3;
        // phi^1 slot of plane z: (z - j0) mod 5
        auto p0 = [&](int z) { return sphi0 + ((z - j0 + 2) % C::NSP0) * C::PHI0; };
        auto p1 = [&](int z) { return sphi1 + ((z - j0) % C::NSP1) * C::PHI1; };

        __syncthreads();  // the previous unit's readers are done with every slot
        for (int d = 0; d < 5; ++d) issue_phi(j0 - 2 + d, d);  // planes j0-2 .. j0+2
        issue_vel(j0, 0);
        cp_async_commit();

        // step-1 own vector: phi^0 offset (row g1y+2, column g1x VX + VX); w below plane j0
        const int o1 = (g1y + 2) * PP0 + VX + g1x * VX;
        const long long own1 = (long long)wrapi(y0 - 2 + g1y, ny) * nx + wrapi(x0 - VX + g1x * VX, nx);
        // step-2 own vector: global offset; written if inside the box
        const int own_x = x0 + g2x * VX, own_y = y0 + g2y;
        const bool writes = is2 && own_x < nx && own_y < ny;
        const long long own2 = (long long)wrapi(own_y, ny) * nx + wrapi(own_x, nx);
        // step 1 counts its outputs on the tile's own cells in the unit's planes
        const bool in_tile1 = is1 && g1x >= 1 && g1x <= TX && g1y >= 2 && g1y < H + 2 &&
                              x0 + (g1x - 1) * VX < nx && y0 + g1y - 2 < ny;
        T wlo1[VX];
        if (is1) {
            const T *src = a.w + (long long)wrapi(j0 - 1, nz) * plane + own1;
#pragma unroll
            for (int i = 0; i < VX; ++i) wlo1[i] = __ldg(src + i);
        }
        cp_async_wait<0>();
        __syncthreads();

        // Step-1 prologue: s_z at plane j0-1 (own), s at plane j0 (own + ring), flux at j0-1/2.
        T szc1[VX], Fzm1[VX];
        {
            const T *Pj = p0(j0), *Pm1 = p0(j0 - 1), *Pm2 = p0(j0 - 2), *Pp1 = p0(j0 + 1);
            T *sx = ssx0 + (j0 & 1) * C::SXS0, *sy = ssy0 + (j0 & 1) * C::SYS0;
            if (is1) {
                T a0[VX], a1[VX], szm[VX], s0v[VX], s1v[VX];
                sharp_vec(Pm1, Pm2, Pj, o1, PP0, a0, a1, szm);
                sharp_vec(Pj, Pm1, Pp1, o1, PP0, s0v, s1v, szc1);
                VV::st(sx + g1y * SXP0 + VX + g1x * VX, s0v);
                VV::st(sy + (g1y + 1) * W1 + g1x * VX, s1v);
                T pm[VX], pc[VX];
                VV::ld(pm, Pm1 + o1);
                VV::ld(pc, Pj + o1);
#pragma unroll
                for (int i = 0; i < VX; ++i) Fzm1[i] = flux(c_adv1 * wlo1[i], c_dif, c_shp, pm[i], pc[i], szm[i], szc1[i]);
            } else if (ring1y) {
                const int row = r1 < TX1 ? -1 : TY1, col = r1 % TX1;
                T s0v[VX], s1v[VX], s2v[VX];
                sharp_vec(Pj, Pm1, Pp1, (row + 2) * PP0 + VX + col * VX, PP0, s0v, s1v, s2v);
                VV::st(sy + (row + 1) * W1 + col * VX, s1v);
            } else if (ring1x) {
                const int q = r1 - 2 * TX1, row = q % TY1, left = q < TY1;
                const int c = left ? VX - 1 : VX + W1;  // column in phi^0 / s_x coordinates
                sx[row * SXP0 + c] = sharp_x(Pj, Pm1, Pp1, (row + 2) * PP0 + c, PP0);
            }
        }
        // plane j0+3 reuses the slot of plane j0-2, which the prologue just read
        __syncthreads();
        if (j0 + 3 <= j1 + 1) issue_phi(j0 + 3, 0);
        if (j0 + 1 < j1) issue_vel(j0 + 1, 1);
        cp_async_commit();

        T szc2[VX], Fzm2[VX];
        for (int j = j0; j < j1 + 1; ++j) {
            // phi^0 plane j+2 and the velocities of plane j have landed; every thread
            // has left iteration j-1 (phi^1 plane j-1, s^0 of plane j and s^1 of plane
            // j-3 are published)
            cp_async_wait<1>();
            __syncthreads();
            if (j + 4 <= j1 + 1) issue_phi(j + 4, (j - j0 + 1) % C::NSP0);
            if (j + 2 < j1) issue_vel(j + 2, (j + 2 - j0) % C::NSV);
            cp_async_commit();

            if (j < j1) {
                // ---- step 1 at plane j: s^0 at j+1 (B1), phi^1 at j (C1) ----
                const T *Pj = p0(j), *Pj1 = p0(j + 1), *Pj2 = p0(j + 2);
                const int b1 = (j + 1) & 1;
                T *sxw = ssx0 + b1 * C::SXS0, *syw = ssy0 + b1 * C::SYS0;
                T szn1[VX];
                if (is1) {
                    T s0v[VX], s1v[VX];
                    sharp_vec(Pj1, Pj, Pj2, o1, PP0, s0v, s1v, szn1);
                    VV::st(sxw + g1y * SXP0 + VX + g1x * VX, s0v);
                    VV::st(syw + (g1y + 1) * W1 + g1x * VX, s1v);
                } else if (ring1y) {
                    const int row = r1 < TX1 ? -1 : TY1, col = r1 % TX1;
                    T s0v[VX], s1v[VX], s2v[VX];
                    sharp_vec(Pj1, Pj, Pj2, (row + 2) * PP0 + VX + col * VX, PP0, s0v, s1v, s2v);
                    VV::st(syw + (row + 1) * W1 + col * VX, s1v);
                } else if (ring1x) {
                    const int q = r1 - 2 * TX1, row = q % TY1, left = q < TY1;
                    const int c = left ? VX - 1 : VX + W1;
                    sxw[row * SXP0 + c] = sharp_x(Pj1, Pj, Pj2, (row + 2) * PP0 + c, PP0);
                }
                if (is1) {
                    const int b = j & 1;
                    const T *vel = svel + ((j - j0) % C::NSV) * C::VEL;
                    const T *ur = vel + (g1y * UP) + VX + g1x * VX;
                    const T *vr = vel + C::USZ + (g1y + 1) * W1 + g1x * VX;
                    const T *wr = vel + C::USZ + C::VSZ + g1y * W1 + g1x * VX;
                    T uc[VX], vc[VX], vn[VX], wc[VX];
                    VV::ld(uc, ur);
                    VV::ld(vc, vr);
                    VV::ld(vn, vr - W1);
                    VV::ld(wc, wr);
                    const T *sxr = ssx0 + b * C::SXS0 + g1y * SXP0 + VX + g1x * VX;
                    const T *syr = ssy0 + b * C::SYS0 + (g1y + 1) * W1 + g1x * VX;
                    T o[VX];
                    update(Pj, Pj1, o1, PP0, sxr, syr - W1, syr + W1, uc, ur[-1], vc, vn, wc, c_adv1, szc1, szn1,
                           Fzm1, o);
                    VV::st(p1(j) + g1y * PP1 + g1x * VX, o);
                    if (in_tile1 && j >= z0 && j < z1) acc1.template add_group<VX>(o, a.c.tol);
                }
            }

            // ---- step 2: prologue at j = z0+2, then s^1 at j-2 (B2) and phi^2 at j-3 (C2) ----
            if (j == z0 + 2) {
                // s_z at plane z0-1 (own), s^1 at plane z0 (own + ring), flux at z0-1/2
                const T *Q0 = p1(z0), *Qm1 = p1(z0 - 1), *Qm2 = p1(z0 - 2), *Qp1 = p1(z0 + 1);
                T *sx = ssx1 + (z0 & 1) * C::SXS1, *sy = ssy1 + (z0 & 1) * C::SYS1;
                const int o2 = (g2y + 2) * PP1 + VX + g2x * VX;
                if (is2) {
                    T a0[VX], a1[VX], szm[VX], s0v[VX], s1v[VX];
                    sharp_vec(Qm1, Qm2, Q0, o2, PP1, a0, a1, szm);
                    sharp_vec(Q0, Qm1, Qp1, o2, PP1, s0v, s1v, szc2);
                    VV::st(sx + g2y * SXP1 + VX + g2x * VX, s0v);
                    VV::st(sy + (g2y + 1) * W + g2x * VX, s1v);
                    T wl[VX], pm[VX], pc[VX];
                    const T *src = a.w + (long long)wrapi(z0 - 1, nz) * plane + own2;
#pragma unroll
                    for (int i = 0; i < VX; ++i) wl[i] = __ldg(src + i);
                    VV::ld(pm, Qm1 + o2);
                    VV::ld(pc, Q0 + o2);
#pragma unroll
                    for (int i = 0; i < VX; ++i) Fzm2[i] = flux(c_adv2 * wl[i], c_dif, c_shp, pm[i], pc[i], szm[i], szc2[i]);
                } else if (ring2y) {
                    const int row = r2 < TX ? -1 : H, col = r2 % TX;
                    T s0v[VX], s1v[VX], s2v[VX];
                    sharp_vec(Q0, Qm1, Qp1, (row + 2) * PP1 + VX + col * VX, PP1, s0v, s1v, s2v);
                    VV::st(sy + (row + 1) * W + col * VX, s1v);
                } else if (ring2x) {
                    const int q = r2 - 2 * TX, row = q % H, left = q < H;
                    const int c = left ? VX - 1 : VX + W;  // column in phi^1 / s^1_x coordinates
                    sx[row * SXP1 + c] = sharp_x(Q0, Qm1, Qp1, (row + 2) * PP1 + c, PP1);
                }
            } else if (j >= z0 + 3) {
                const int m = j - 3;  // the plane step 2 updates
                const T *Qm = p1(m), *Qm1 = p1(m + 1), *Qm2 = p1(m + 2);
                const int b1 = (m + 1) & 1;
                T *sxw = ssx1 + b1 * C::SXS1, *syw = ssy1 + b1 * C::SYS1;
                T szn2[VX];
                const int o2 = (g2y + 2) * PP1 + VX + g2x * VX;
                if (is2) {
                    // step 2 takes its faces of plane m from L2 (step 1 staged them three
                    // planes ago); issued first to overlap the sharpening below
                    const long long zo = (long long)m * plane + own2;
                    T uc[VX], vc[VX], vn[VX], wc[VX];
                    VV::ld(uc, a.u + zo);
                    VV::ld(vc, a.v + zo);
                    VV::ld(wc, a.w + zo);
                    VV::ld(vn, a.v + (long long)m * plane + (long long)wrapi(own_y - 1, ny) * nx + wrapi(own_x, nx));
                    const T uL = __ldg(a.u + (long long)m * plane + (long long)wrapi(own_y, ny) * nx + wrapi(own_x - 1, nx));
                    T s0v[VX], s1v[VX];
                    sharp_vec(Qm1, Qm, Qm2, o2, PP1, s0v, s1v, szn2);
                    VV::st(sxw + g2y * SXP1 + VX + g2x * VX, s0v);
                    VV::st(syw + (g2y + 1) * W + g2x * VX, s1v);
                    const int b = m & 1;
                    const T *sxr = ssx1 + b * C::SXS1 + g2y * SXP1 + VX + g2x * VX;
                    const T *syr = ssy1 + b * C::SYS1 + (g2y + 1) * W + g2x * VX;
                    T o[VX];
                    update(Qm, Qm1, o2, PP1, sxr, syr - W, syr + W, uc, uL, vc, vn, wc, c_adv2, szc2, szn2, Fzm2, o);
                    if (writes) {
                        VV::st(a.out + (long long)CDI_CHK(m, nz, st) * plane + own2, o);
                        acc2.template add_group<VX>(o, a.c.tol);
                    }
                } else if (ring2y) {
                    const int row = r2 < TX ? -1 : H, col = r2 % TX;
                    T s0v[VX], s1v[VX], s2v[VX];
                    sharp_vec(Qm1, Qm, Qm2, (row + 2) * PP1 + VX + col * VX, PP1, s0v, s1v, s2v);
                    VV::st(syw + (row + 1) * W + col * VX, s1v);
                } else if (ring2x) {
                    const int q = r2 - 2 * TX, row = q % H, left = q < H;
                    const int c = left ? VX - 1 : VX + W;
                    sxw[row * SXP1 + c] = sharp_x(Qm1, Qm, Qm2, (row + 2) * PP1 + c, PP1);
                }
            }
        }
        cp_async_wait<0>();
    }
    reduce_and_finish2(acc1, acc2, a.red);
}

template <typename T>
cudaError_t tb2_occupancy(int *resident)
{
    cudaError_t e = cudaFuncSetAttribute(fwd_tb2_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)TbCfg<T>::bytes);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(resident, fwd_tb2_kernel<T>, TbCfg<T>::NT,
                                                         TbCfg<T>::bytes);
}

template <typename T>
cudaError_t launch_fwd_tb2(const FwdArgs<T> &a, T c_adv2, int nblocks, int nchunks, cudaStream_t s)
{
    fwd_tb2_kernel<T><<<nblocks, TbCfg<T>::NT, TbCfg<T>::bytes, s>>>(a, c_adv2, nchunks);
    return cudaGetLastError();
}

void tb2_tile_dims(int esize, int *bw, int *bh)
{
    *bw = 16 * (16 / esize);
    *bh = 16;
}

template cudaError_t tb2_occupancy<float>(int *);
template cudaError_t tb2_occupancy<double>(int *);
template cudaError_t launch_fwd_tb2<float>(const FwdArgs<float> &, float, int, int, cudaStream_t);
template cudaError_t launch_fwd_tb2<double>(const FwdArgs<double> &, double, int, int, cudaStream_t);

}  // namespace cdi
