// Column-march collide-stream pass for D3Q27 (second pass of the 3-D step,
// after k_zmacro): the pulled populations are staged in shared memory by
// asynchronous copies and the next-step moments are gathered, not scattered.
//
// A CTA of 512 threads owns an xy tile of 30 x 14 cells and a range of ZL
// planes; thread (cx, cy) = (lane, warp) keeps the same column of the
// collided 32 x 16 region (the tile plus a one-cell rim) for every plane, so
// the three moment planes it is summing (z - 1, z, z + 1) stay in its
// registers.  One plane is processed as six layers (f then g, one value of
// c_z at a time, nine populations each):
//   1. the layer's nine pulled source boxes (16 rows x 34 cells, shifted by
//      -c_y and -c_z; x rounded out to 16-byte chunks) were copied into a
//      ring buffer by cp.async several layers earlier -- the copies are in
//      flight without holding registers;
//   2. each thread relaxes its cell's nine populations (Eqs. LBM_f, LBM_g),
//      stores those of owned cells, and writes all nine to a gather buffer;
//   3. after one barrier each owned thread reads, for the plane z + c_z, the
//      nine values that stream into its own cell (from (cx - c_x, cy - c_y)):
//      rho, j and G of the next step accumulate in registers, no atomics.
//      Populations leaving through a z wall return into the cell they left,
//      reversed (half-way bounce-back).
// The plane below the current one is then complete and its moments are
// written.  Rim collisions are the repeated work, as in the scatter march:
// (32 x 16)/(30 x 14) in xy and (ZL + 2)/ZL in z.
//
// Requirements (checked by the host before selecting it): 32- or 16-bit
// storage, nx a multiple of the elements per 16-byte chunk, no
// extrapolated faces, no per-cell force or heat fields, one equation of
// state per launch.
#pragma once

#include "lbm_async.cuh"
#include "lbm_device.cuh"
#include "lbm_fused.cuh"
#include "lbm_split.cuh"

#include <type_traits>

namespace lbm {

constexpr int kZgThreads = 512;        // one thread per column of the collided region
constexpr int kZgCX = 32, kZgCY = 16;  // collided region: the owned tile plus a one-cell rim
constexpr int kZgTX = kZgCX - 2, kZgTY = kZgCY - 2;

template <typename S> struct ZgStage {
    static constexpr int C = 16 / (int)sizeof(S);                  // elements per 16-byte copy
    static constexpr int NCH = (kZgCX + 2 + 2 * (C - 1)) / C;       // copies per row: 34 cells + alignment
    static constexpr int NCOL = NCH * C;                            // staged elements per row
    static constexpr int SLOT = kZgCY * NCOL;                       // one population's box
    static constexpr int LAYER = 9 * SLOT;                          // the nine populations of a c_z layer
    static constexpr int CHUNKS = 9 * kZgCY * NCH;                  // 16-byte copies per layer
    static constexpr int RING = sizeof(S) == 4 ? 4 : 6;             // layers in the ring (in flight: RING - 1)
    static constexpr int PER_THREAD = (CHUNKS + kZgThreads - 1) / kZgThreads;  // copies per thread per layer
    static constexpr size_t stage_bytes = (size_t)RING * LAYER * sizeof(S);
    static constexpr size_t gather_bytes = (size_t)2 * 9 * kZgCY * kZgCX * sizeof(float);  // two layers
    static constexpr size_t desc_bytes = (size_t)PER_THREAD * kZgThreads * sizeof(uint4);
    static constexpr size_t smem_bytes = stage_bytes + gather_bytes + desc_bytes;
};

// opp(j) within one c_z layer of nine directions (j = d0 + 3 d1; digits 0, 1, 2
// mean c = 0, +1, -1): 4 bits per entry
constexpr unsigned long long kOpp9 = 0x453786120ULL;
__device__ __forceinline__ int opp9(int j) { return (int)((kOpp9 >> (4 * j)) & 15u); }
constexpr bool opp9_table_ok(int j = 0)
{
    return j == 9 || ((int)((kOpp9 >> (4 * j)) & 15u) == opp(j) && opp9_table_ok(j + 1));
}
static_assert(opp9_table_ok(), "kOpp9 must list opp(j) for j = 0..8");

// Macroscopic state of a cell and its stencils (div u, grad h, grad T, Phi;
// Eq. correction) from the first pass's fields: periodic x, y; z periodic or
// mirrored beyond half-way bounce-back walls (velocity and X_z odd).
template <typename R, int EK>
__device__ __forceinline__ void zg_state(const SimK<R, EK>& s, const R* __restrict__ Wc, long long Ntot, int x, int y,
                                         int z, Macro<R>& m, R& divu, R* gh, R* gT, R* Phi)
{
    const int nx = s.nx, ny = s.ny, nz = s.nz;
    const bool walls = s.zwalls != 0;
    auto cell = [&](int xx, int yy, int zz) { return (unsigned)xx + (unsigned)nx * ((unsigned)yy + (unsigned)ny * (unsigned)zz); };
    auto Wf = [&](int f, unsigned c) { return Wc[(size_t)f * Ntot + c]; };
    int zn[5];
    bool zf[5];
#pragma unroll
    for (int o = -2; o <= 2; ++o) {
        if (walls) zn[o + 2] = mirror_z(z + o, nz, zf[o + 2]);
        else {
            zn[o + 2] = wrapc(z + o, nz);
            zf[o + 2] = false;
        }
    }
    const int xm1 = x == 0 ? nx - 1 : x - 1, xp1 = x == nx - 1 ? 0 : x + 1;
    const int ym1 = y == 0 ? ny - 1 : y - 1, yp1 = y == ny - 1 ? 0 : y + 1;
    const unsigned gk = cell(x, y, z);
    m.rho = Wf(W_RHO, gk);
    m.ir = R(1) / m.rho;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        m.u[a] = Wf(W_U + a, gk);
        m.F[a] = Wf(W_F + a, gk);
    }
    m.Q = heat_q<R>(s, z);
    m.T = Wf(W_T, gk);
    m.P = Wf(W_P, gk);
    m.theta = Wf(W_TH, gk);
    m.h = Wf(W_H, gk);
    m.cv = Wf(W_CV, gk);
    m.icv = EK == EOS_PR ? R(1) / m.cv : s.inv_cv;
    m.gam = Wf(W_GAM, gk);
    m.athe = Wf(W_ATHE, gk);
    m.e = Wf(W_E, gk);
    const unsigned cxm = cell(xm1, y, z), cxp = cell(xp1, y, z);
    const unsigned cym = cell(x, ym1, z), cyp = cell(x, yp1, z);
    const unsigned czm = cell(x, y, zn[1]), czp = cell(x, y, zn[3]);
    const R szm = zf[1] ? R(-1) : R(1), szp = zf[3] ? R(-1) : R(1);
    divu = R(0.5) * ((Wf(W_U, cxp) - Wf(W_U, cxm)) + (Wf(W_U + 1, cyp) - Wf(W_U + 1, cym)) +
                     (szp * Wf(W_U + 2, czp) - szm * Wf(W_U + 2, czm)));
    gh[0] = R(0.5) * (Wf(W_H, cxp) - Wf(W_H, cxm));
    gh[1] = R(0.5) * (Wf(W_H, cyp) - Wf(W_H, cym));
    gh[2] = R(0.5) * (Wf(W_H, czp) - Wf(W_H, czm));
    gT[0] = R(0.5) * (Wf(W_T, cxp) - Wf(W_T, cxm));
    gT[1] = R(0.5) * (Wf(W_T, cyp) - Wf(W_T, cym));
    gT[2] = R(0.5) * (Wf(W_T, czp) - Wf(W_T, czm));
    R dX[3];
    if (s.phi_central) {
        dX[0] = R(0.5) * (Wf(W_X, cxp) - Wf(W_X, cxm));
        dX[1] = R(0.5) * (Wf(W_X + 1, cyp) - Wf(W_X + 1, cym));
        dX[2] = R(0.5) * (szp * Wf(W_X + 2, czp) - szm * Wf(W_X + 2, czm));
    } else {
        // upwind-biased by the sign of u_alpha (X_z odd beyond a wall)
        const R X0x = Wf(W_X, gk), X0y = Wf(W_X + 1, gk), X0z = Wf(W_X + 2, gk);
        const bool px = m.u[0] >= R(0), py = m.u[1] >= R(0), pz = m.u[2] >= R(0);
        dX[0] = upwind_biased<R>(m.u[0], Wf(W_X, cell(wrapc(x + (px ? -2 : 2), nx), y, z)), Wf(W_X, cxm), X0x,
                                 Wf(W_X, cxp));
        dX[1] = upwind_biased<R>(m.u[1], Wf(W_X + 1, cell(x, wrapc(y + (py ? -2 : 2), ny), z)), Wf(W_X + 1, cym), X0y,
                                 Wf(W_X + 1, cyp));
        const int o2 = pz ? 0 : 4;
        const R s2 = zf[o2] ? R(-1) : R(1);
        dX[2] = upwind_biased<R>(m.u[2], s2 * Wf(W_X + 2, cell(x, y, zn[o2])), szm * Wf(W_X + 2, czm), X0z,
                                 szp * Wf(W_X + 2, czp));
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) Phi[a] = -dX[a] * m.ir;
}

template <typename S, int EK>
__global__ void __launch_bounds__(kZgThreads, 1)
    k_zgather(const SimDev* __restrict__ sims, const TileEntry* __restrict__ tiles, int ntiles, int ZL,
              const S* __restrict__ src, S* __restrict__ dst, const float* __restrict__ W, float* __restrict__ Mout,
              long long Ntot)
{
    using R = float;
    using G = ZgStage<S>;
    constexpr int C = G::C, NCH = G::NCH, NCOL = G::NCOL, K = G::RING;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* stage = reinterpret_cast<S*>(smem_raw);                      // [K][9][kZgCY][NCOL]
    R* gbuf = reinterpret_cast<R*>(smem_raw + G::stage_bytes);     // [2][9][kZgCY][kZgCX]
    // per thread and copy: (staged element offset | slot << 16, source offset in a
    // plane for a shifted pull, the same without the shift for a pull across a wall)
    uint4* desc = reinterpret_cast<uint4*>(smem_raw + G::stage_bytes + G::gather_bytes);  // [PER_THREAD][threads]
    __shared__ SimK<R, EK> s;
    __shared__ int cur_sim;
    const int tid = threadIdx.x, cx = tid & 31, cy = tid >> 5;
    if (tid == 0) cur_sim = -1;
    __syncthreads();

    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const TileEntry te = tiles[t];
        if (te.sim != cur_sim) {
            __syncthreads();
            if (tid == 0) {
                simc_from<R>(static_cast<SimC<R>&>(s), sims[te.sim]);
                cur_sim = te.sim;
            }
            __syncthreads();
        }
        const int nx = s.nx, ny = s.ny, nz = s.nz;
        const bool walls = s.zwalls != 0;
        const unsigned Ncell = (unsigned)s.N;
        const unsigned plane_cells = (unsigned)nx * (unsigned)ny;
        const R* Wc = W + s.cell_off;
        const S* fb = src + s.pop_off;
        const S* gb = fb + (size_t)27 * s.N;
        S* fo = dst + s.pop_off;
        S* go = fo + (size_t)27 * s.N;
        R* Mo = Mout + s.cell_off;
        const int zend = min(te.z0 + ZL, nz);
        // collided planes: the owned range plus one rim plane each side (none beyond a wall)
        const int pfirst = (walls && te.z0 == 0) ? 0 : te.z0 - 1;
        const int plast = (walls && zend == nz) ? nz - 1 : zend;
        const int LPP = s.iso ? 3 : 6;  // isothermal: g is not evolved
        const int nstages = (plast - pfirst + 1) * LPP;
        const int vx = min(kZgTX, nx - te.x0), vy = min(kZgTY, ny - te.y0);
        const bool own_xy = cx >= 1 && cx <= vx && cy >= 1 && cy <= vy;
        const int xa = floor_div(te.x0 - 2, C) * C;  // first staged x (unwrapped, chunk-aligned)
        const int x = wrapc(te.x0 - 1 + cx, nx), y = wrapc(te.y0 - 1 + cy, ny);
        const int base_col = te.x0 - 1 + cx - xa;  // staged column of this thread's own x

        // this thread's copies of a layer: fixed per tile except for the plane and population
#pragma unroll
        for (int k = 0; k < G::PER_THREAD; ++k) {
            const int c = tid + k * kZgThreads;
            uint4 d = make_uint4(0xffffffffu, 0u, 0u, 0u);
            if (c < G::CHUNKS) {
                const int j = c / (kZgCY * NCH), r = (c / NCH) % kZgCY, q = c % NCH;
                const unsigned xg = (unsigned)wrapc(xa + q * C, nx);
                const unsigned yn = (unsigned)wrapc(te.y0 - 1 + r - cval(j / 3), ny);
                const unsigned yb = (unsigned)wrapc(te.y0 - 1 + r, ny);
                d = make_uint4((unsigned)((j * kZgCY + r) * NCOL + q * C) | ((unsigned)j << 16),
                               yn * (unsigned)nx + xg, yb * (unsigned)nx + xg, 0u);
            }
            desc[k * kZgThreads + tid] = d;
        }
        // stages in issue order: plane index ipl, layer il (0-2: f with c_z = -1, 0, +1; 3-5: g), ring slot ib
        int ipl = 0, il = 0, ib = 0, issued = 0;
        auto issue = [&]() {
            if (issued < nstages) {
                const int zc = pfirst + ipl;
                const int l3 = il < 3 ? il : il - 3;
                const int d2 = l3 == 0 ? 2 : l3 - 1;  // c_z = -1, 0, +1
                int zs = zc - cval(d2);
                const bool bounce = walls && (zs < 0 || zs >= nz);  // pulled across a wall: opp(i) of the cell itself
                zs = bounce ? zc : wrapc(zs, nz);
                const S* base = (il < 3 ? fb : gb) + (size_t)zs * plane_cells;
                S* sb = stage + (size_t)ib * G::LAYER;
                const int po = bounce ? 9 * odig(d2) : 9 * d2;
#pragma unroll
                for (int k = 0; k < G::PER_THREAD; ++k) {
                    const uint4 d = desc[k * kZgThreads + tid];
                    if (k + 1 < G::PER_THREAD || d.x != 0xffffffffu) {
                        const int j = (int)(d.x >> 16);
                        const unsigned ip = (unsigned)(po + (bounce ? opp9(j) : j));
                        cp_async16(sb + (d.x & 0xffffu), base + (ip * Ncell + (bounce ? d.z : d.y)));
                    }
                }
            }
            cp_async_commit();  // one group per stage, empty past the end
            ++issued;
            if (++il == LPP) { il = 0; ++ipl; }
            if (++ib == K) ib = 0;
        };
#pragma unroll 1
        for (int st = 0; st < K - 1; ++st) issue();

        // next-step moments (rho, j, G) of the planes zc - 1, zc, zc + 1 around the current plane zc
        R acc[3][5];
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 5; ++q) acc[p][q] = R(0);
        auto finalize = [&](int slot, int zf) {  // the moments of plane zf are complete
            if (own_xy && zf >= te.z0 && zf < zend) {
                const unsigned kk = (unsigned)x + (unsigned)nx * ((unsigned)y + (unsigned)ny * (unsigned)zf);
                Mo[M_RHO * Ntot + kk] = acc[slot][0];
                Mo[(M_J + 0) * Ntot + kk] = acc[slot][1];
                Mo[(M_J + 1) * Ntot + kk] = acc[slot][2];
                Mo[(M_J + 2) * Ntot + kk] = acc[slot][3];
                Mo[M_G * Ntot + kk] = acc[slot][4];
            }
        };
        // add (rho, j, G) contributions to the accumulator of plane zc + idx - 1
        auto add = [&](int idx, bool isg, R sr, R sx, R sy, R sz) {
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                if (p != idx) continue;
                if (isg) acc[p][4] += sr;
                else {
                    acc[p][0] += sr;
                    acc[p][1] += sx;
                    acc[p][2] += sy;
                    acc[p][3] += sz;
                }
            }
        };
        // The gather of a layer runs after the next layer's barrier (one barrier per
        // layer, two gather buffers): pending layer's buffer, c_z, distribution, plane.
        bool pend = false, pend_g = false;
        int pend_slot = 0, pend_cz = 0, pend_zc = 0, wslot = 0;
        auto gather_pending = [&](int zc) {
            if (!pend || !own_xy) return;
            const R* g0 = gbuf + pend_slot * (9 * kZgCY * kZgCX) + cy * kZgCX + cx;
            R sr = 0, sx = 0, sy = 0;
            static_for<0, 9>([&](auto J) {
                constexpr int j = decltype(J)::value;
                constexpr int cxj = cval(j % 3), cyj = cval(j / 3);
                const R w = g0[j * kZgCY * kZgCX - cyj * kZgCX - cxj];  // from (cx - c_x, cy - c_y)
                sr += w;
                if (cxj != 0) sx += R(cxj) * w;
                if (cyj != 0) sy += R(cyj) * w;
            });
            add(pend_zc + pend_cz - zc + 1, pend_g, sr, sx, sy, R(pend_cz) * sr);
        };

        int rb = 0;  // ring slot of the layer being relaxed
#pragma unroll 1
        for (int zc = pfirst; zc <= plast; ++zc) {
            const int z = wrapc(zc, nz);
            Macro<R> m;
            R divu, gh[3], gT[3], Phi[3];
            zg_state<R, EK>(s, Wc, Ntot, x, y, z, m, divu, gh, gT, Phi);
            Coll<3, R> cl = Coll<3, R>::template make<true>(s, m, divu, gh, gT, Phi);
            const bool own = own_xy && zc >= te.z0 && zc < zend;
            const unsigned gk = (unsigned)x + (unsigned)nx * ((unsigned)y + (unsigned)ny * (unsigned)z);

            // The relaxation folded per axis (Eqs. LBM_f, LBM_g with the equilibria in
            // product form): rho and the weights of f^eq, f*, g^eq, g* ride on the x factors.
            R fx1[3], fx2[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                fx1[d] = cl.cf1 * cl.rho * cl.A0[0][d];
                fx2[d] = cl.cf2 * cl.rho * cl.As[0][d];
            }
            R gx1[3] = {}, gx2[3] = {}, gx3[3] = {}, gx4[3] = {}, hq[3] = {};  // g factors, set before the g layers

            // one layer: relax the nine populations with c_z digit d2 of f (isg false) or g
            auto layer = [&](auto D2c, auto Gc, auto POSc) {
                constexpr int d2 = decltype(D2c)::value;
                constexpr bool isg = decltype(Gc)::value;
                constexpr int pos = decltype(POSc)::value;
                constexpr int cz = cval(d2);
                cp_async_wait<K - 2>();
                __syncthreads();  // this layer's copies landed everywhere; the previous layer's gather buffer is complete
                gather_pending(zc);
                pend = false;
                // after the gather of the last c_z = -1 layer of plane zc, plane zc - 1 is complete
                if (pos == (s.iso ? 1 : 4)) finalize(0, zc - 1);
                const bool bin = walls && (zc - cz < 0 || zc - cz >= nz);    // pulled across a wall
                const bool bout = walls && (zc + cz < 0 || zc + cz >= nz);   // streams across a wall
                // this thread's staged row: pulls from x - c_x (c_x = 0, +1, -1), no shift across a wall
                const S* r0 = stage + (size_t)rb * G::LAYER + cy * NCOL + base_col;
                const S* rm = bin ? r0 : r0 - 1;
                const S* rp = bin ? r0 : r0 + 1;
                R* gw = gbuf + wslot * (9 * kZgCY * kZgCX) + cy * kZgCX + cx;
                static_for<0, 9>([&](auto J) {
                    constexpr int j = decltype(J)::value;
                    constexpr int i = 9 * d2 + j;
                    constexpr int d0 = dig(i, 0), d1 = dig(i, 1);
                    constexpr int cxj = cc(i, 0), cyj = cc(i, 1);
                    const S* rowp = cxj == 0 ? r0 : (cxj > 0 ? rm : rp);
                    const R* ref = isg ? s.gref : s.fref;
                    R p = stored_to_f<S>(rowp[j * G::SLOT]);
                    if constexpr (Codec<S, R>::offset) p += bin ? ref[opp(i)] : ref[i];
                    R w;
                    if constexpr (isg) {
                        w = cl.cg0 * p;
                        w = fma(fma(gx1[d0], cl.A0[1][d1], gx2[d0] * cl.H0[1][d1]), cl.A0[2][d2], w);
                        w = fma(gx2[d0] * cl.A0[1][d1], cl.H0[2][d2], w);
                        w = fma(fma(gx3[d0], cl.B0[1][d1], gx4[d0] * cl.Hs[1][d1]), cl.B0[2][d2], w);
                        w = fma(gx4[d0] * cl.B0[1][d1], cl.Hs[2][d2], w);
                        if constexpr (cnorm2(i) == 1) w += cxj != 0 ? R(cxj) * hq[0] : (cyj != 0 ? R(cyj) * hq[1] : R(cz) * hq[2]);
                    } else {
                        w = cl.cf0 * p;
                        w = fma(fx1[d0] * cl.A0[1][d1], cl.A0[2][d2], w);
                        w = fma(fx2[d0] * cl.As[1][d1], cl.As[2][d2], w);
                    }
                    if (own) {
                        S* o = isg ? go : fo;
                        Codec<S, R>::st(o + (unsigned)i * Ncell + gk, w - (Codec<S, R>::offset ? ref[i] : R(0)));
                    }
                    gw[j * kZgCY * kZgCX] = w;
                });
                issue();  // into the buffer read one layer ago
                if (++rb == K) rb = 0;
                if (bout) {
                    // half-way bounce-back: f'_i returns to this cell as opp(i) (own values, reversed c)
                    if (own_xy) {
                        R sr = 0, sx = 0, sy = 0;
                        static_for<0, 9>([&](auto J) {
                            constexpr int j = decltype(J)::value;
                            constexpr int cxj = cval(j % 3), cyj = cval(j / 3);
                            const R w = gw[j * kZgCY * kZgCX];
                            sr += w;
                            if (cxj != 0) sx -= R(cxj) * w;
                            if (cyj != 0) sy -= R(cyj) * w;
                        });
                        add(1, isg, sr, sx, sy, -R(cz) * sr);
                    }
                } else {
                    pend = true;
                    pend_g = isg;
                    pend_slot = wslot;
                    pend_cz = cz;
                    pend_zc = zc;
                    wslot ^= 1;
                }
            };
            using IsF = std::false_type;
            using IsG = std::true_type;
            using I0 = std::integral_constant<int, 0>;
            using I1 = std::integral_constant<int, 1>;
            using I2 = std::integral_constant<int, 2>;
            // c_z = -1, 0, +1 (digits 2, 0, 1) for f, then for g
            layer(I2{}, IsF{}, std::integral_constant<int, 0>{});
            layer(I0{}, IsF{}, std::integral_constant<int, 1>{});
            layer(I1{}, IsF{}, std::integral_constant<int, 2>{});
            if (!s.iso) {
                cl.prepare_g();
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    gx1[d] = cl.cg1 * cl.rho * (cl.e * cl.A0[0][d] + cl.H0[0][d]);
                    gx2[d] = cl.cg1 * cl.rho * cl.A0[0][d];
                    gx3[d] = cl.cg2 * cl.rho * (cl.es * cl.B0[0][d] + cl.Hs[0][d]);
                    gx4[d] = cl.cg2 * cl.rho * cl.B0[0][d];
                    hq[d] = cl.cg2 * R(0.5) * cl.qc[d];
                }
                layer(I2{}, IsG{}, std::integral_constant<int, 3>{});
                layer(I0{}, IsG{}, std::integral_constant<int, 4>{});
                layer(I1{}, IsG{}, std::integral_constant<int, 5>{});
            }
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                acc[0][q] = acc[1][q];
                acc[1][q] = acc[2][q];
                acc[2][q] = R(0);
            }
        }
        // the top plane when a wall ends the march there (its last layers bounce back: nothing pending)
        finalize(0, plast);
        cp_async_wait<0>();
        __syncthreads();  // the ring is reused by the next tile
    }
}

template <typename S, int EK>
cudaError_t zgather_launch(const SimDev* sims, const TileEntry* tiles, int ntiles, int ZL, const void* src, void* dst,
                           const void* W, void* Mout, long long Ntot, cudaStream_t stream)
{
    constexpr size_t smem = ZgStage<S>::smem_bytes;
    static_assert(smem <= 227u * 1024u, "z-gather buffers do not fit in shared memory");
    static int grid_cap = 0;
    if (grid_cap == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_zgather<S, EK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0, dev = 0, nsm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_zgather<S, EK>, kZgThreads, smem);
        if (e != cudaSuccess) return e;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        grid_cap = per_sm * nsm;
    }
    const int grid = ntiles < grid_cap ? ntiles : grid_cap;
    k_zgather<S, EK><<<grid, kZgThreads, smem, stream>>>(sims, tiles, ntiles, ZL, (const S*)src, (S*)dst,
                                                         (const float*)W, (float*)Mout, Ntot);
    return cudaGetLastError();
}

template <typename S>
cudaError_t zgather_dispatch_t(int eos, int zl, const SimDev* sims, const TileEntry* tiles, int ntiles,
                               const void* src, void* dst, const void* W, void* Mout, long long Ntot,
                               cudaStream_t stream)
{
    if (eos == EOS_IDEAL) return zgather_launch<S, EOS_IDEAL>(sims, tiles, ntiles, zl, src, dst, W, Mout, Ntot, stream);
    if (eos == EOS_VDW) return zgather_launch<S, EOS_VDW>(sims, tiles, ntiles, zl, src, dst, W, Mout, Ntot, stream);
    if (eos == EOS_PR) return zgather_launch<S, EOS_PR>(sims, tiles, ntiles, zl, src, dst, W, Mout, Ntot, stream);
    return cudaErrorInvalidValue;
}

}  // namespace lbm
