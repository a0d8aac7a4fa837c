// z-marching collide-stream pass for D3Q27 (second pass of the 3-D step).
//
// The first pass (k_zmacro below) evaluates the macroscopic state of
// every cell once from the carried moments (rho, j, G) and writes the fields
// the stencils and the collision read.  This pass owns an xy tile of TX x TY
// cells and a range of ZL planes and marches along z: for each plane zc from
// z0 - 1 to z0 + ZL it collides the xy tile plus its one-cell rim (pulling
// every population once, f and then g through the registers), stores the
// post-collision populations of its own cells, and adds every post-collision
// population to the next-step moment of the cell it streams into, kept in a
// ring of three planes in shared memory; a plane's moments are complete, and
// written, once the plane above it has been collided.  The rim collisions are
// the only repeated work: (TX+2)(TY+2)/(TX TY) in xy and (ZL+2)/ZL in z.
#pragma once

#include "lbm_device.cuh"
#include "lbm_fused.cuh"
#include "lbm_mlp.cuh"
#include "lbm_split.cuh"

#include <type_traits>

namespace lbm {

constexpr int kZThreads = 256;

// NEE: z faces with non-equilibrium-extrapolation walls or duct ends
// (zwalls == 2): stencils past a face take the linear extrapolation through
// the boundary cell, 2 v(z_B) - v(2 z_B - z), instead of mirror images; the
// boundary cells themselves were rebuilt by k_nee before this pass.
template <typename R, typename S, int EK, int TX, int TY, bool NEE = false>
__global__ void __launch_bounds__(kZThreads, sizeof(R) == 4 ? 2 : 1)
    k_zmarch(const SimDev* __restrict__ sims, const TileEntry* __restrict__ tiles, int ntiles, int ZL,
             const S* __restrict__ src, S* __restrict__ dst, const R* __restrict__ W, R* __restrict__ Mout,
             long long Ntot)
{
    constexpr int Q = 27;
    constexpr int W1 = TX + 2, H1 = TY + 2, N1 = W1 * H1, N0 = TX * TY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* acc = reinterpret_cast<R*>(smem_raw);  // [3 planes][5: rho, j (3), G][N0]
    __shared__ SimK<R, EK> s;
    __shared__ int cur_sim;
    __shared__ double s_res[3];  // NEE: duct friction k, throttle K and sigma
    const int tid = threadIdx.x;
    if (tid == 0) cur_sim = -1;
    __syncthreads();

    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const TileEntry te = tiles[t];
        if (te.sim != cur_sim) {
            __syncthreads();
            if (tid == 0) {
                simc_from<R>(static_cast<SimC<R>&>(s), sims[te.sim]);
                cur_sim = te.sim;
                if constexpr (NEE) {
                    s_res[0] = sims[te.sim].friction;
                    s_res[1] = sims[te.sim].throttle_K;
                    s_res[2] = sims[te.sim].throttle_sigma;
                }
            }
            __syncthreads();
        }
        const int nx = s.nx, ny = s.ny, nz = s.nz;
        const bool walls = s.zwalls != 0;
        const unsigned Ncell = (unsigned)s.N;
        const R* Wc = W + s.cell_off;
        const S* fb = src + s.pop_off;
        const S* gb = fb + (size_t)Q * s.N;
        S* fo = dst + s.pop_off;
        S* go = fo + (size_t)Q * s.N;
        R* Mo = Mout + s.cell_off;
        const int zend = min(te.z0 + ZL, nz);
        const unsigned vx = (unsigned)min(TX, nx - te.x0), vy = (unsigned)min(TY, ny - te.y0);
        for (int k = tid; k < 15 * N0; k += kZThreads) acc[k] = R(0);
        __syncthreads();

        for (int zc = te.z0 - 1; zc <= zend; ++zc) {
            const bool ghost_plane = walls && (zc < 0 || zc >= nz);
            if (!ghost_plane) {
                const int z = wrapc(zc, nz);
                // z neighbours of the stencils: periodic, or mirrored beyond walls (flip: odd fields change sign)
                int zn[5];
                bool zf[5], zx[5];
#pragma unroll
                for (int o = -2; o <= 2; ++o) {
                    if constexpr (NEE) {
                        // past a face: the image 2 z_B - z (zx marks the extrapolated neighbours)
                        const int zz = zc + o;
                        zx[o + 2] = zz < 0 || zz >= nz;
                        zn[o + 2] = zz < 0 ? -zz : (zz >= nz ? 2 * (nz - 1) - zz : zz);
                        zf[o + 2] = false;
                    } else {
                        zx[o + 2] = false;
                        if (walls) zn[o + 2] = mirror_z(zc + o, nz, zf[o + 2]);
                        else {
                            zn[o + 2] = wrapc(zc + o, nz);
                            zf[o + 2] = false;
                        }
                    }
                }
                for (int k = tid; k < N1; k += kZThreads) {
                    const int lx = k % W1, ly = k / W1;
                    const int tx = lx - 1, ty = ly - 1;
                    const int x = wrapc(te.x0 + tx, nx), y = wrapc(te.y0 + ty, ny);
                    const int xm1 = x == 0 ? nx - 1 : x - 1, xp1 = x == nx - 1 ? 0 : x + 1;
                    const int ym1 = y == 0 ? ny - 1 : y - 1, yp1 = y == ny - 1 ? 0 : y + 1;
                    auto cell = [&](int xx, int yy, int zz) {
                        return (unsigned)xx + (unsigned)nx * ((unsigned)yy + (unsigned)ny * (unsigned)zz);
                    };
                    const unsigned gk = cell(x, y, z);
                    auto Wf = [&](int f, unsigned c) { return Wc[(size_t)f * Ntot + c]; };

                    Macro<R> m;
                    m.rho = Wf(W_RHO, gk);
                    m.ir = R(1) / m.rho;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        m.u[a] = Wf(W_U + a, gk);
                        m.F[a] = Wf(W_F + a, gk);
                    }
                    m.Q = heat_q<R>(s, z);
                    if constexpr (NEE) {
                        // heat of the duct resistance, rho (K phi + k |u|) |u|^2 (Q = -F.u of the first pass)
                        if (s_res[0] > 0.0 || s_res[1] > 0.0) {
                            R Kphi = R(0);
                            if (s_res[1] > 0.0) {
                                const double d = ((double)z - 0.5 * (double)(nz - 1)) / s_res[2];
                                Kphi = (R)(s_res[1] * exp(-d * d));
                            }
                            const R u2 = m.u[0] * m.u[0] + m.u[1] * m.u[1] + m.u[2] * m.u[2];
                            m.Q += m.rho * (Kphi + (R)s_res[0] * sqrt(u2)) * u2;
                        }
                    }
                    m.T = Wf(W_T, gk);
                    m.P = Wf(W_P, gk);
                    m.theta = Wf(W_TH, gk);
                    m.h = Wf(W_H, gk);
                    m.cv = Wf(W_CV, gk);
                    m.icv = EK == EOS_PR ? R(1) / m.cv : s.inv_cv;
                    m.gam = Wf(W_GAM, gk);
                    m.athe = Wf(W_ATHE, gk);
                    m.e = Wf(W_E, gk);

                    // stencils: div u, grad h, grad T (central) and Phi (Eq. correction)
                    R divu, gh[3], gT[3], Phi[3];
                    if constexpr (NEE) {
                        // the same stencils with extrapolated z neighbours past a face
                        auto Wz = [&](int f, int o) -> R {
                            const unsigned ci = cell(x, y, zn[o + 2]);
                            if (zx[o + 2]) return R(2) * Wf(f, cell(x, y, zc + o < 0 ? 0 : nz - 1)) - Wf(f, ci);
                            return Wf(f, ci);
                        };
                        const unsigned cxm = cell(xm1, y, z), cxp = cell(xp1, y, z);
                        const unsigned cym = cell(x, ym1, z), cyp = cell(x, yp1, z);
                        divu = R(0.5) * ((Wf(W_U, cxp) - Wf(W_U, cxm)) + (Wf(W_U + 1, cyp) - Wf(W_U + 1, cym)) +
                                         (Wz(W_U + 2, 1) - Wz(W_U + 2, -1)));
                        gh[0] = R(0.5) * (Wf(W_H, cxp) - Wf(W_H, cxm));
                        gh[1] = R(0.5) * (Wf(W_H, cyp) - Wf(W_H, cym));
                        gh[2] = R(0.5) * (Wz(W_H, 1) - Wz(W_H, -1));
                        gT[0] = R(0.5) * (Wf(W_T, cxp) - Wf(W_T, cxm));
                        gT[1] = R(0.5) * (Wf(W_T, cyp) - Wf(W_T, cym));
                        gT[2] = R(0.5) * (Wz(W_T, 1) - Wz(W_T, -1));
                        R dX[3];
                        if (s.phi_central) {
                            dX[0] = R(0.5) * (Wf(W_X, cxp) - Wf(W_X, cxm));
                            dX[1] = R(0.5) * (Wf(W_X + 1, cyp) - Wf(W_X + 1, cym));
                            dX[2] = R(0.5) * (Wz(W_X + 2, 1) - Wz(W_X + 2, -1));
                        } else {
                            const R X0x = Wf(W_X, gk), X0y = Wf(W_X + 1, gk), X0z = Wf(W_X + 2, gk);
                            const bool px = m.u[0] >= R(0), py = m.u[1] >= R(0), pz = m.u[2] >= R(0);
                            dX[0] = upwind_biased<R>(m.u[0], Wf(W_X, cell(wrapc(x + (px ? -2 : 2), nx), y, z)),
                                                     Wf(W_X, cxm), X0x, Wf(W_X, cxp));
                            dX[1] = upwind_biased<R>(m.u[1], Wf(W_X + 1, cell(x, wrapc(y + (py ? -2 : 2), ny), z)),
                                                     Wf(W_X + 1, cym), X0y, Wf(W_X + 1, cyp));
                            dX[2] = upwind_biased<R>(m.u[2], Wz(W_X + 2, pz ? -2 : 2), Wz(W_X + 2, -1), X0z,
                                                     Wz(W_X + 2, 1));
                        }
#pragma unroll
                        for (int a = 0; a < 3; ++a) Phi[a] = -dX[a] * m.ir;
                    } else {
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
                            dX[0] = upwind_biased<R>(m.u[0], Wf(W_X, cell(wrapc(x + (px ? -2 : 2), nx), y, z)),
                                                     Wf(W_X, cxm), X0x, Wf(W_X, cxp));
                            dX[1] = upwind_biased<R>(m.u[1], Wf(W_X + 1, cell(x, wrapc(y + (py ? -2 : 2), ny), z)),
                                                     Wf(W_X + 1, cym), X0y, Wf(W_X + 1, cyp));
                            const int o2 = pz ? 0 : 4;
                            const R s2 = zf[o2] ? R(-1) : R(1);
                            dX[2] = upwind_biased<R>(m.u[2], s2 * Wf(W_X + 2, cell(x, y, zn[o2])),
                                                     szm * Wf(W_X + 2, czm), X0z, szp * Wf(W_X + 2, czp));
                        }
#pragma unroll
                        for (int a = 0; a < 3; ++a) Phi[a] = -dX[a] * m.ir;
                    }
                    Coll<3, R> cl = Coll<3, R>::make(s, m, divu, gh, gT, Phi);
                    if (!s.iso) cl.prepare_g();

                    // pull sources: f_i(x) = f'_i(x - c_i), or f'_opp(i)(x) across a z wall
                    const int xs[3] = {x, xm1, xp1}, ys[3] = {y, ym1, yp1};
                    int zs[3] = {z, z == 0 ? nz - 1 : z - 1, z == nz - 1 ? 0 : z + 1};
                    bool zw[3] = {false, false, false};
                    if (walls) {
                        zw[1] = z == 0;
                        zw[2] = z == nz - 1;
                    }
                    unsigned rows[3][3];
#pragma unroll
                    for (int b = 0; b < 3; ++b)
#pragma unroll
                        for (int c = 0; c < 3; ++c) rows[b][c] = (unsigned)nx * ((unsigned)ys[b] + (unsigned)ny * (unsigned)zs[c]);
                    const bool own = tx >= 0 && ty >= 0 && tx < TX && ty < TY && (unsigned)tx < vx && (unsigned)ty < vy &&
                                     zc >= te.z0 && zc < zend;
                    const bool zlo_wall = walls && z == 0, zhi_wall = walls && z == nz - 1;
                    // destinations of f'_i: cell (tx + c, ty + c, zc + c), or (tx, ty, zc) as opp(i) across a wall
                    auto scatter = [&](auto I, int field_base, R v) {
                        constexpr int i = decltype(I)::value;
                        constexpr int c0 = cc(i, 0), c1 = cc(i, 1), c2 = cc(i, 2);
                        const bool bounce = (c2 < 0 && zlo_wall) || (c2 > 0 && zhi_wall);
                        const int dx = bounce ? tx : tx + c0, dy = bounce ? ty : ty + c1, zd = bounce ? zc : zc + c2;
                        if ((unsigned)dx < vx && (unsigned)dy < vy && zd >= te.z0 && zd < zend) {
                            R* a = acc + (zd % 3) * 5 * N0 + dx + TX * dy;
                            if (field_base == 0) {
                                atomicAdd(a, v);
                                if (c0 != 0) atomicAdd(a + 1 * N0, (c0 > 0) != bounce ? v : -v);
                                if (c1 != 0) atomicAdd(a + 2 * N0, (c1 > 0) != bounce ? v : -v);
                                if (c2 != 0) atomicAdd(a + 3 * N0, (c2 > 0) != bounce ? v : -v);
                            } else {
                                atomicAdd(a + 4 * N0, v);
                            }
                        }
                    };
                    // Pull, relax, store, scatter: f, then g, nine populations (one c_z layer)
                    // at a time.  Each layer's loads are issued together, ahead of the shared-
                    // memory atomics of the scatter, which the compiler does not move loads across.
                    auto pull = [&](auto I, const S* base, const R* ref) {
                        constexpr int i = decltype(I)::value;
                        constexpr int d0 = dig(i, 0), d1 = dig(i, 1), d2 = dig(i, 2);
                        const bool wall_src = zw[d2];
                        const int isrc = wall_src ? opp(i) : i;
                        const unsigned idx = wall_src ? (unsigned)isrc * Ncell + gk
                                                      : (unsigned)i * Ncell + (unsigned)xs[d0] + rows[d1][d2];
                        R v = Codec<S, R>::ld(base + idx);
                        if (Codec<S, R>::offset) v += ref[isrc];
                        return v;
                    };
                    static_for<0, 3>([&](auto L) {
                        constexpr int l = decltype(L)::value;
                        R v[9];
                        static_for<0, 9>([&](auto J) {
                            v[decltype(J)::value] = pull(std::integral_constant<int, 9 * l + decltype(J)::value>{}, fb, s.fref);
                        });
                        static_for<0, 9>([&](auto J) {
                            constexpr int i = 9 * l + decltype(J)::value;
                            const R w = cl.template f<i>(v[decltype(J)::value]);
                            if (own) Codec<S, R>::st(fo + (unsigned)i * Ncell + gk, w - (Codec<S, R>::offset ? s.fref[i] : R(0)));
                            scatter(std::integral_constant<int, i>{}, 0, w);
                        });
                    });
                    if (!s.iso) {  // isothermal: g is not evolved
                        static_for<0, 3>([&](auto L) {
                            constexpr int l = decltype(L)::value;
                            R v[9];
                            static_for<0, 9>([&](auto J) {
                                v[decltype(J)::value] = pull(std::integral_constant<int, 9 * l + decltype(J)::value>{}, gb, s.gref);
                            });
                            static_for<0, 9>([&](auto J) {
                                constexpr int i = 9 * l + decltype(J)::value;
                                const R w = cl.template g<i>(v[decltype(J)::value]);
                                if (own) Codec<S, R>::st(go + (unsigned)i * Ncell + gk, w - (Codec<S, R>::offset ? s.gref[i] : R(0)));
                                scatter(std::integral_constant<int, i>{}, 1, w);
                            });
                        });
                    }
                }
            }
            __syncthreads();
            // plane zc - 1 has all its contributions: write its moments and clear its slot
            const int zfin = zc - 1;
            if (zfin >= te.z0 && zfin < zend) {
                R* a = acc + (zfin % 3) * 5 * N0;
                for (int d = tid; d < N0; d += kZThreads) {
                    const int tx = d % TX, ty = d / TX;
                    const R r = a[d], j0 = a[N0 + d], j1 = a[2 * N0 + d], j2 = a[3 * N0 + d], Gv = a[4 * N0 + d];
                    a[d] = a[N0 + d] = a[2 * N0 + d] = a[3 * N0 + d] = a[4 * N0 + d] = R(0);
                    if ((unsigned)tx >= vx || (unsigned)ty >= vy) continue;
                    const unsigned kk = (unsigned)(te.x0 + tx) + (unsigned)nx * ((unsigned)(te.y0 + ty) + (unsigned)ny * (unsigned)zfin);
                    Mo[M_RHO * Ntot + kk] = r;
                    Mo[(M_J + 0) * Ntot + kk] = j0;
                    Mo[(M_J + 1) * Ntot + kk] = j1;
                    Mo[(M_J + 2) * Ntot + kk] = j2;
                    Mo[M_G * Ntot + kk] = Gv;
                }
            }
            __syncthreads();
        }
    }
}

// grad lap rho at (x, y, z) for periodic z or half-way bounce-back walls
// (mirror images beyond them), from the 25 distinct densities the six
// neighbouring Laplacians use, with 32-bit indices: the same stencil as
// grad_lap (lap rho at the images of the two neighbours along each axis).
template <typename R>
__device__ __forceinline__ void grad_lap_zm(const R* __restrict__ rho, int x, int y, int z, int nx, int ny, int nz,
                                            bool mirror, R* gl)
{
    if (nx >= 4 && y >= 2 && y < ny - 2 && z >= 2 && z < nz - 2) {
        // two or more cells from the y and z ends: the 25 densities at fixed offsets from
        // the cell (x wrapped through its four offsets), summed as in the general case below
        const int NX = nx, NP = nx * ny;
        const R* c0 = rho + ((unsigned)x + (unsigned)nx * ((unsigned)y + (unsigned)ny * (unsigned)z));
        const int xp = x + 1 < nx ? 1 : 1 - nx, xm = x > 0 ? -1 : nx - 1;
        const int xpp = x + 2 < nx ? 2 : 2 - nx, xmm = x > 1 ? -2 : nx - 2;
        auto lap7 = [&](int o, int oxp, int oxm, int oyp, int oym, int ozp, int ozm) {
            const R c = c0[o];
            R L = c0[oxp] - R(2) * c + c0[oxm];
            L += c0[oyp] - R(2) * c + c0[oym];
            L += c0[ozp] - R(2) * c + c0[ozm];
            return L;
        };
        const R Lxp = lap7(xp, xpp, 0, xp + NX, xp - NX, xp + NP, xp - NP);
        const R Lxm = lap7(xm, 0, xmm, xm + NX, xm - NX, xm + NP, xm - NP);
        const R Lyp = lap7(NX, NX + xp, NX + xm, 2 * NX, 0, NX + NP, NX - NP);
        const R Lym = lap7(-NX, -NX + xp, -NX + xm, 0, -2 * NX, -NX + NP, -NX - NP);
        const R Lzp = lap7(NP, NP + xp, NP + xm, NP + NX, NP - NX, 2 * NP, 0);
        const R Lzm = lap7(-NP, -NP + xp, -NP + xm, -NP + NX, -NP - NX, 0, -2 * NP);
        gl[0] = R(0.5) * (Lxp - Lxm);
        gl[1] = R(0.5) * (Lyp - Lym);
        gl[2] = R(0.5) * (Lzp - Lzm);
        return;
    }
    auto at = [&](int xx, int yy, int zz) {
        return rho[(unsigned)xx + (unsigned)nx * ((unsigned)yy + (unsigned)ny * (unsigned)zz)];
    };
    const int xp = nb_coord(x, 1, nx, false), xm = nb_coord(x, -1, nx, false);
    const int yp = nb_coord(y, 1, ny, false), ym = nb_coord(y, -1, ny, false);
    const int zp = nb_coord(z, 1, nz, mirror), zm = nb_coord(z, -1, nz, mirror);
    // Laplacian at an in-domain cell whose axis neighbours are given
    auto lap = [&](int cx, int cy, int cz, int cxp, int cxm, int cyp, int cym, int czp, int czm) {
        const R c = at(cx, cy, cz);
        R L = at(cxp, cy, cz) - R(2) * c + at(cxm, cy, cz);
        L += at(cx, cyp, cz) - R(2) * c + at(cx, cym, cz);
        L += at(cx, cy, czp) - R(2) * c + at(cx, cy, czm);
        return L;
    };
    const R Lxp = lap(xp, y, z, nb_coord(xp, 1, nx, false), x, yp, ym, zp, zm);
    const R Lxm = lap(xm, y, z, x, nb_coord(xm, -1, nx, false), yp, ym, zp, zm);
    const R Lyp = lap(x, yp, z, xp, xm, nb_coord(yp, 1, ny, false), y, zp, zm);
    const R Lym = lap(x, ym, z, xp, xm, y, nb_coord(ym, -1, ny, false), zp, zm);
    const R Lzp = lap(x, y, zp, xp, xm, yp, ym, nb_coord(zp, 1, nz, mirror), nb_coord(zp, -1, nz, mirror));
    const R Lzm = lap(x, y, zm, xp, xm, yp, ym, nb_coord(zm, 1, nz, mirror), nb_coord(zm, -1, nz, mirror));
    gl[0] = R(0.5) * (Lxp - Lxm);
    gl[1] = R(0.5) * (Lyp - Lym);
    gl[2] = R(0.5) * (Lzp - Lzm);
}

// First pass of the z-march step: the macroscopic state of every cell
// (Eqs. def_u, def_E, the EoS and its closure scalars, the flux X of
// Eq. correction) from the carried moments rho, j, G, with last step's T as
// the Newton start (or the learned start, ML), written to the field buffer W.
// One thread per cell, constants of the simulation typed and with the EoS
// fixed at compile time.  The pass waits mostly on its global loads: the
// float32 Peng-Robinson pass is bounded to six blocks of 256 threads per SM
// (40 registers, a small spill), which ran 1 % faster per 384^3 step than
// four blocks at 64 registers; five lost half of that, seven and eight lost it all.
// The other forms keep the blocks per SM their register use gives them.
template <typename R, int EK, bool ML> constexpr int zmacro_min_blocks()
{
    return sizeof(R) == 4 && !ML && EK == EOS_PR ? 6 : (ML || (sizeof(R) == 8 && EK == EOS_PR) ? 3 : 4);
}
template <typename R, int EK, bool ML>
__global__ void __launch_bounds__(kBlockCells, zmacro_min_blocks<R, EK, ML>()) k_zmacro(const SimDev* __restrict__ sims,
                                                        const BlockEntry* __restrict__ table, const R* __restrict__ M,
                                                        R* __restrict__ W, long long Ntot, unsigned long long* diag)
{
    __shared__ SimK<R, EK> s;
    __shared__ SimDev s_dev;
    __shared__ std::conditional_t<ML, MlpSmem, int> mlp_s;
    const BlockEntry be = table[blockIdx.x];
    load_sim(s_dev, sims, be.sim);
    simc_from_coop<R>(static_cast<SimC<R>&>(s), s_dev, threadIdx.x);
    __syncthreads();
    if constexpr (ML) {
        if (s.mlp != nullptr) {
            mlp_load(mlp_s, s.mlp);
            __syncthreads();
        }
    }
    const long long k = (long long)be.start + threadIdx.x;
    const bool valid = k < s.N;
    const long long gk = s.cell_off + k;
    int x = 0, y = 0, z = 0;
    R r = R(1), F[3] = {0, 0, 0}, j[3] = {0, 0, 0}, Gm = R(0), Tg = R(0), Qh = R(0);
    if (valid) {
        {  // Q N < 2^32 per simulation: 32-bit coordinates
            const unsigned ku = (unsigned)k, rr = ku / (unsigned)s.nx;
            x = (int)(ku - rr * (unsigned)s.nx);
            z = (int)(rr / (unsigned)s.ny);
            y = (int)(rr - (unsigned)z * (unsigned)s.ny);
        }
        const R* rho = M + M_RHO * Ntot + s.cell_off;
        r = rho[k];
        R gl[3];
        if (s.zwalls == 2) grad_lap<3, R>(rho, x, y, z, s.nx, s.ny, s.nz, s.zwalls, gl);
        else grad_lap_zm<R>(rho, x, y, z, s.nx, s.ny, s.nz, s.zwalls == 1, gl);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            F[a] = r * s.acc[a] + s.kappa * r * gl[a];  // Eqs. force_decomposition, korteweg_force
            j[a] = M[(M_J + a) * Ntot + gk];
        }
        Gm = M[M_G * Ntot + gk];
        Tg = W[W_T * Ntot + gk];
        Qh = heat_q<R>(s, z);
        apply_friction<3, R>(s_dev, z, r, j, F, Qh);  // duct friction and throttle (zero otherwise)
    }
    if constexpr (ML) {
        if (s.mlp != nullptr) {  // block-uniform: whole warps evaluate the network
            const float Tm = mlp_T_warp(mlp_s, valid ? (float)r : 1.f,
                                        valid ? (float)macro_energy<3, R>(r, j, Gm, F, Qh) : 0.f);
            if (valid) Tg = (R)Tm;
        }
    }
    unsigned flags = 0;
    if (valid) {
        const Macro<R> m = macro_cell<3, R>(s, r, j, Gm, F, Qh, Tg, flags);
        W[W_RHO * Ntot + gk] = r;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            W[(W_U + a) * Ntot + gk] = m.u[a];
            W[(W_F + a) * Ntot + gk] = m.F[a];
            W[(W_X + a) * Ntot + gk] = xflux<R>(r, m.u[a], m.theta);
        }
        W[W_T * Ntot + gk] = m.T;
        W[W_H * Ntot + gk] = m.h;
        W[W_P * Ntot + gk] = m.P;
        W[W_TH * Ntot + gk] = m.theta;
        W[W_CV * Ntot + gk] = m.cv;
        W[W_GAM * Ntot + gk] = m.gam;
        W[W_ATHE * Ntot + gk] = m.athe;
        W[W_E * Ntot + gk] = m.e;
    }
    if (diag) count_flags(flags, diag);
}

template <typename R, int EK, bool ML>
cudaError_t zmacro_launch(const SimDev* sims, const BlockEntry* table, int nblocks, const void* M, void* W,
                          long long Ntot, unsigned long long* diag, cudaStream_t stream)
{
    k_zmacro<R, EK, ML><<<nblocks, kBlockCells, 0, stream>>>(sims, table, (const R*)M, (R*)W, Ntot, diag);
    return cudaGetLastError();
}

// the first pass for one arithmetic type, by equation of state (ML: learned
// temperature start, Peng-Robinson only)
template <typename R, bool WITH_ML>
cudaError_t zmacro_dispatch_t(int eos, int mlp, const SimDev* sims, const BlockEntry* table, int nblocks,
                              const void* M, void* W, long long Ntot, unsigned long long* diag, cudaStream_t stream)
{
    if (mlp) {
        if constexpr (WITH_ML) {
            if (eos == EOS_PR) return zmacro_launch<R, EOS_PR, true>(sims, table, nblocks, M, W, Ntot, diag, stream);
        }
        return cudaErrorInvalidValue;
    }
    if (eos == EOS_IDEAL) return zmacro_launch<R, EOS_IDEAL, false>(sims, table, nblocks, M, W, Ntot, diag, stream);
    if (eos == EOS_VDW) return zmacro_launch<R, EOS_VDW, false>(sims, table, nblocks, M, W, Ntot, diag, stream);
    if (eos == EOS_PR) return zmacro_launch<R, EOS_PR, false>(sims, table, nblocks, M, W, Ntot, diag, stream);
    return cudaErrorInvalidValue;
}

template <typename R, typename S, int EK, int TX, int TY, bool NEE = false>
cudaError_t zmarch_launch_shape(const SimDev* sims, const TileEntry* tiles, int ntiles, int ZL, const void* src,
                                void* dst, const void* W, void* Mout, long long Ntot, cudaStream_t stream)
{
    constexpr size_t smem = (size_t)15 * TX * TY * sizeof(R);
    static int grid_cap = 0;
    if (grid_cap == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_zmarch<R, S, EK, TX, TY, NEE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0, dev = 0, nsm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_zmarch<R, S, EK, TX, TY, NEE>, kZThreads, smem);
        if (e != cudaSuccess) return e;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        grid_cap = per_sm * nsm;
    }
    const int grid = ntiles < grid_cap ? ntiles : grid_cap;
    k_zmarch<R, S, EK, TX, TY, NEE><<<grid, kZThreads, smem, stream>>>(sims, tiles, ntiles, ZL, (const S*)src, (S*)dst,
                                                                  (const R*)W, (R*)Mout, Ntot);
    return cudaGetLastError();
}

}  // namespace lbm
