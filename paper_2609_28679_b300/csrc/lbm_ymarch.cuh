// Row-march one-pass time step for D2Q9: the 2-D counterpart of the fused
// step without its y halos.
//
// A CTA of 128 threads owns an x strip of TX columns and YL rows and marches
// up the strip one row per step.  Thread k keeps the same column x for the
// whole march; the columns x0 - 1 - RM ... are the strip, its one-cell rim
// (collided for the moments streaming into the strip) and the RM further
// columns the stencils of the macroscopic state reach (RM = 1 with the
// central Phi, 2 with the upwind-biased one).  In y nothing is recomputed:
// every row's rho, lap rho and macroscopic state are formed once and kept in
// small shared-memory rings for as long as the stencils need them.  One step,
// with the collided row C:
//   A. (after the step's copies have landed) gather the next-step moments of
//      the row collided one step earlier from the gather buffer (rho, j, G
//      of the cell each population streams into; a row is complete two
//      steps after it was first collided into) and write the finished row;
//      lap rho of row C + RM + 2 and the macroscopic state (Eqs. def_u,
//      def_E, the equation of state; force rho a + kappa rho grad lap rho) of
//      row C + RM, from the carried moments of the previous step;
//   B. collide row C (Eqs. sh_vel_1 ... LBM_f, LBM_g) from its pulled
//      populations, store the owned cells, and write all post-collision
//      populations to the gather buffer.
// The pulled populations of a row (each population from the row it is pulled
// from), the rho row and the (j, G, T) row a step needs are staged by 16-byte
// cp.async copies K - 1 steps ahead, so two barriers per row suffice and
// nothing waits for memory in registers.
//
// Requirements (checked by the host): 32- or 16-bit storage, nx a multiple of
// the elements per 16-byte copy, one equation of state per launch, no learned
// temperature (that form keeps the fused kernel).
#pragma once

#include "lbm_async.cuh"
#include "lbm_device.cuh"
#include "lbm_fused.cuh"
#include "lbm_fused_api.h"
#include "lbm_split.cuh"

namespace lbm {

constexpr int kYmThreads = 128;

template <typename S, bool PC> struct YmShape {
    static constexpr int NT = kYmThreads;
    static constexpr int RM = PC ? 1 : 2;                        // reach of the macroscopic stencils
    static constexpr int NC = NT - 2 * RM;                       // collided columns: the strip and its rim
    static constexpr int TX = NC - 2;                            // owned columns
    static constexpr int K = PC ? 3 : 4;                         // staged steps in the ring (in flight: K - 1)
    static constexpr int C = 16 / (int)sizeof(S);                // populations per 16-byte copy
    static constexpr int PWP = (NC + 2 + C - 1 + C - 1) / C * C;  // staged columns of a population row
    static constexpr int NCHP = PWP / C;
    static constexpr int PWR = (NT + 4 + 3 + 3) / 4 * 4;         // staged columns of a rho row
    static constexpr int NCHR = PWR / 4;
    static constexpr int PWM = (NT + 3 + 3) / 4 * 4;             // staged columns of a (j, G, T) row
    static constexpr int NCHM = PWM / 4;
    static constexpr int PCH = 18 * NCHP;                        // population copies per step
    static constexpr int MCH = NCHR + 4 * NCHM;                  // moment copies per step
    static constexpr int KP = (PCH + NT - 1) / NT, KM = (MCH + NT - 1) / NT;  // copies per thread
    static constexpr int NSF = 6;  // stencil fields: u_x, u_y, T, h, X_x, X_y
    static constexpr int NLF = 9;  // local fields of a collided cell: rho, F_x, F_y, P, theta, c_v, gamma, alpha theta, e
    static constexpr int NSR = 2 * RM + 1, NLR = RM + 1;         // rows kept of each
    static constexpr int LW = NT + 2;                            // lap rho columns
    static constexpr size_t pop_bytes = (size_t)K * 18 * PWP * sizeof(S);
    static constexpr size_t rho_bytes = (size_t)(K + 3) * PWR * 4;
    static constexpr size_t jgt_bytes = (size_t)K * 4 * PWM * 4;
    static constexpr size_t lap_bytes = (size_t)4 * LW * 4;
    static constexpr size_t sten_bytes = (size_t)NSR * NSF * NT * 4;
    static constexpr size_t loc_bytes = (size_t)NLR * NLF * NT * 4;
    static constexpr size_t gb_bytes = (size_t)18 * NT * 4;
    static constexpr size_t o_rho = pop_bytes, o_jgt = o_rho + rho_bytes, o_lap = o_jgt + jgt_bytes,
                            o_sten = o_lap + lap_bytes, o_loc = o_sten + sten_bytes, o_gb = o_loc + loc_bytes;
    static constexpr size_t smem_bytes = o_gb + gb_bytes;
    static_assert(pop_bytes % 16 == 0 && rho_bytes % 16 == 0 && jgt_bytes % 16 == 0 && lap_bytes % 16 == 0 &&
                      sten_bytes % 16 == 0 && loc_bytes % 16 == 0,
                  "every ring must start on a 16-byte boundary");
};

// CTAs per SM the rings leave room for (at most 3): the register budget follows from it
template <typename S, bool PC> constexpr int ymarch_min_blocks()
{
    constexpr int n = (int)((size_t)232448 / (YmShape<S, PC>::smem_bytes + 1024));
    return n < 1 ? 1 : (n > 3 ? 3 : n);
}

template <typename S, int EK, bool PC>
__global__ void __launch_bounds__(kYmThreads, (ymarch_min_blocks<S, PC>()))
    k_ymarch(const SimDev* __restrict__ sims, const TileEntry* __restrict__ tiles, int ntiles, int YL,
             const S* __restrict__ src, S* __restrict__ dst, const float* __restrict__ Min, float* __restrict__ Mout,
             long long Ntot, unsigned long long* __restrict__ diag)
{
    using R = float;
    using G = YmShape<S, PC>;
    constexpr int NT = G::NT, RM = G::RM, TX = G::TX, K = G::K, C = G::C;
    constexpr int PWP = G::PWP, PWR = G::PWR, PWM = G::PWM, LW = G::LW, NSR = G::NSR, NLR = G::NLR;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* popr = reinterpret_cast<S*>(smem_raw);              // [K][18][PWP] pulled populations of a collided row
    R* rhor = reinterpret_cast<R*>(smem_raw + G::o_rho);   // [K + 3][PWR] rho rows
    R* jgtr = reinterpret_cast<R*>(smem_raw + G::o_jgt);   // [K][4][PWM] j_x, j_y, G, T rows
    R* lapr = reinterpret_cast<R*>(smem_raw + G::o_lap);   // [4][LW] lap rho rows
    R* sten = reinterpret_cast<R*>(smem_raw + G::o_sten);  // [NSR][NSF][NT] stencil fields
    R* loc = reinterpret_cast<R*>(smem_raw + G::o_loc);    // [NLR][NLF][NT] local fields
    R* gbuf = reinterpret_cast<R*>(smem_raw + G::o_gb);    // [18][NT] post-collision populations of a row
    __shared__ SimK<R, EK> s;
    __shared__ int cur_sim;
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
            }
            __syncthreads();
        }
        const int nx = s.nx, ny = s.ny;
        const unsigned Ncell = (unsigned)s.N;
        const S* fb = src + s.pop_off;  // f, then g at + 9 N
        S* fo = dst + s.pop_off;
        const R* Mi = Min + s.cell_off;
        R* Mo = Mout + s.cell_off;
        const int x0 = te.x0, y0 = te.y0;
        const int vx = min(TX, nx - x0), vy = min(YL, ny - y0);
        const int yc0 = y0 - 1, yc1 = y0 + vy;  // collided rows: the owned ones and a rim row each side
        const int r0 = yc0 - RM - 3;            // origin of the pipeline's rows (every row used is above it)
        const int nsteps = vy + 2 * RM + 8;
        // staging origins (unwrapped, aligned to the copies)
        const int xap = floor_div(x0 - 2, C) * C;       // populations: the collided columns +- 1
        const int xar = floor_div(x0 - 3 - RM, 4) * 4;  // rho: the lap rho columns +- 1
        const int xam = floor_div(x0 - 1 - RM, 4) * 4;  // j, G, T: the macroscopic columns
        const int xm = x0 - 1 - RM + tid;               // this thread's column
        const bool coll = tid >= RM && tid < NT - RM;    // collided
        const bool own_x = tid >= RM + 1 && tid <= RM + vx;

        // this thread's copies of a step, fixed per tile but for the row: staged
        // offset, source offset without the row, and which row
        unsigned p_so[G::KP];
        size_t p_go[G::KP];
        int p_row[G::KP];  // -1: none; else the c_y digit (pulled from C - c_y)
#pragma unroll
        for (int k = 0; k < G::KP; ++k) {
            const int c = tid + k * NT;
            p_row[k] = -1;
            p_so[k] = 0;
            p_go[k] = 0;
            if (c < G::PCH) {
                const int p = c / G::NCHP, q = c % G::NCHP;
                p_so[k] = (unsigned)(p * PWP + q * C);
                p_go[k] = (size_t)p * Ncell + (unsigned)wrapc(xap + q * C, nx);
                p_row[k] = dig(p % 9, 1);
            }
        }
        unsigned m_so[G::KM];
        size_t m_go[G::KM];
        int m_kind[G::KM];  // -1: none, 0: rho row, 1: (j, G, T) row
#pragma unroll
        for (int k = 0; k < G::KM; ++k) {
            const int c = tid + k * NT;
            m_kind[k] = -1;
            m_so[k] = 0;
            m_go[k] = 0;
            if (c < G::NCHR) {
                m_kind[k] = 0;
                m_so[k] = (unsigned)(c * 4);
                m_go[k] = (size_t)M_RHO * Ntot + (unsigned)wrapc(xar + c * 4, nx);
            } else if (c < G::MCH) {
                const int f = (c - G::NCHR) / G::NCHM, q = (c - G::NCHR) % G::NCHM;
                const int fld = f == 0 ? M_J : (f == 1 ? M_J + 1 : (f == 2 ? M_G : M_T));
                m_kind[k] = 1;
                m_so[k] = (unsigned)(f * PWM + q * 4);
                m_go[k] = (size_t)fld * Ntot + (unsigned)wrapc(xam + q * 4, nx);
            }
        }
        // Step s consumes the rho row r0 + s + 1, the (j, G, T) row and the pulled
        // populations of its macroscopic row r0 + s - 2 and collided row r0 + s - 2 - RM.
        auto issue = [&](int st) {
            if (st < nsteps) {
                const int rr = r0 + st + 1, mr = r0 + st - 2, cr = mr - RM;
                if (cr >= yc0 && cr <= yc1) {
                    S* slot = popr + (size_t)(st % K) * 18 * PWP;
                    const unsigned o0 = (unsigned)wrapc(cr, ny) * (unsigned)nx;
                    const unsigned o1 = (unsigned)wrapc(cr - 1, ny) * (unsigned)nx;  // c_y = +1
                    const unsigned o2 = (unsigned)wrapc(cr + 1, ny) * (unsigned)nx;  // c_y = -1
#pragma unroll
                    for (int k = 0; k < G::KP; ++k)
                        if (p_row[k] >= 0)
                            cp_async16(slot + p_so[k], fb + p_go[k] + (p_row[k] == 0 ? o0 : (p_row[k] == 1 ? o1 : o2)));
                }
                const bool a_rho = rr <= yc1 + RM + 2, a_m = mr >= yc0 - RM && mr <= yc1 + RM;
                R* rs = rhor + (size_t)(st % (K + 3)) * PWR;
                R* js = jgtr + (size_t)(st % K) * 4 * PWM;
                const unsigned ro = (unsigned)wrapc(rr, ny) * (unsigned)nx;
                const unsigned mo = (unsigned)wrapc(mr, ny) * (unsigned)nx;
#pragma unroll
                for (int k = 0; k < G::KM; ++k) {
                    if (m_kind[k] == 0 && a_rho) cp_async16(rs + m_so[k], Mi + m_go[k] + ro);
                    else if (m_kind[k] == 1 && a_m) cp_async16(js + m_so[k], Mi + m_go[k] + mo);
                }
            }
            cp_async_commit();  // one group per step, empty past the end
        };
#pragma unroll 1
        for (int st = 0; st < K - 1; ++st) issue(st);

        R acc[3][4];  // next-step rho, j_x, j_y, G of the rows C' - 1, C', C' + 1 around the last gathered row C'
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = R(0);
        R Tq1 = 0, Tq2 = 0;  // T of this column in the rows collided one and two steps ago

#pragma unroll 1
        for (int st = 0; st < nsteps; ++st) {
            cp_async_wait<K - 2>();
            __syncthreads();  // step st's copies landed; the previous step's rows are complete
            issue(st + K - 1);

            // ---- A1. moments streaming out of the row collided in the previous step
            const int cq = r0 + st - 3 - RM;
            if (cq >= yc0 && cq <= yc1) {
                if (own_x) {
                    static_for<0, 18>([&](auto P) {
                        constexpr int p = decltype(P)::value;
                        constexpr int i = p % 9, cx = cc(i, 0), cy = cc(i, 1);
                        const R w = gbuf[p * NT + tid - cx];  // from the column x - c_x
                        if constexpr (p < 9) {
                            acc[1 + cy][0] += w;
                            if (cx != 0) acc[1 + cy][1] += R(cx) * w;
                            if (cy != 0) acc[1 + cy][2] += R(cy) * w;
                        } else {
                            acc[1 + cy][3] += w;
                        }
                    });
                }
                // the row below it has received everything: its moments and the Newton guess
                const int fr = cq - 1;
                if (own_x && fr >= y0 && fr < y0 + vy) {
                    // the carried fields rho, j (3), G, T in order, Ntot apart
                    static_assert(M_RHO == 0 && M_J == 1 && M_G == 4 && M_T == 5, "carried field order");
                    R* pm = Mo + ((unsigned)xm + (unsigned)nx * (unsigned)fr);
                    *pm = acc[0][0];
                    *(pm += Ntot) = acc[0][1];
                    *(pm += Ntot) = acc[0][2];
                    *(pm += Ntot) = R(0);
                    *(pm += Ntot) = acc[0][3];
                    *(pm += Ntot) = Tq2;
                }
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    acc[0][b] = acc[1][b];
                    acc[1][b] = acc[2][b];
                    acc[2][b] = R(0);
                }
            }

            // ---- A2. lap rho of row r0 + st from the rho rows staged at steps st - 2 ... st
            const int Lr = r0 + st;
            if (Lr >= yc0 - RM - 1 && Lr <= yc1 + RM + 1) {
                const R* rp = rhor + (size_t)(st % (K + 3)) * PWR;
                const R* r_ = rhor + (size_t)((st + K + 2) % (K + 3)) * PWR;
                const R* rm = rhor + (size_t)((st + K + 1) % (K + 3)) * PWR;
                R* lo = lapr + (size_t)((Lr - r0) & 3) * LW;
                for (int lc = tid; lc < LW; lc += NT) {
                    const int ci = x0 - 2 - RM + lc - xar;
                    lo[lc] = r_[ci + 1] + r_[ci - 1] + rp[ci] + rm[ci] - R(4) * r_[ci];
                }
            }

            // ---- A3. macroscopic state of row r0 + st - 2 (lap rho rows of steps st - 3 ... st - 1)
            const int Mr = r0 + st - 2;
            unsigned flags = 0;
            bool own_m = false;
            if (Mr >= yc0 - RM && Mr <= yc1 + RM) {
                const R* rrow = rhor + (size_t)((st + K) % (K + 3)) * PWR;  // staged at step st - 3
                const R* js = jgtr + (size_t)(st % K) * 4 * PWM;
                const int ci = xm - xar, cm = xm - xam, lc = tid + 1;
                const R* l0 = lapr + (size_t)((Mr - r0) & 3) * LW;
                const R* lm = lapr + (size_t)((Mr - 1 - r0) & 3) * LW;
                const R* lp = lapr + (size_t)((Mr + 1 - r0) & 3) * LW;
                const R r = rrow[ci];
                R F[2], j[2];
                F[0] = r * (s.acc[0] + s.kappa * R(0.5) * (l0[lc + 1] - l0[lc - 1]));
                F[1] = r * (s.acc[1] + s.kappa * R(0.5) * (lp[lc] - lm[lc]));
                j[0] = js[cm];
                j[1] = js[PWM + cm];
                const Macro<R> m = macro_cell<2, R>(s, r, j, js[2 * PWM + cm], F, heat_q<R>(s, 0), js[3 * PWM + cm], flags);
                R* so = sten + (size_t)((Mr - r0) % NSR) * G::NSF * NT + tid;
                so[0 * NT] = m.u[0];
                so[1 * NT] = m.u[1];
                so[2 * NT] = m.T;
                so[3 * NT] = m.h;
                so[4 * NT] = xflux<R>(r, m.u[0], m.theta);
                so[5 * NT] = xflux<R>(r, m.u[1], m.theta);
                R* lo = loc + (size_t)((Mr - r0) % NLR) * G::NLF * NT + tid;
                lo[0 * NT] = r;
                lo[1 * NT] = F[0];
                lo[2 * NT] = F[1];
                lo[3 * NT] = m.P;
                lo[4 * NT] = m.theta;
                lo[5 * NT] = m.cv;
                lo[6 * NT] = m.gam;
                lo[7 * NT] = m.athe;
                lo[8 * NT] = m.e;
                own_m = own_x && Mr >= y0 && Mr < y0 + vy;
            }
            if (diag) count_flags(own_m ? flags : 0u, diag);
            __syncthreads();  // the macroscopic row is complete

            // ---- B. collide row r0 + st - 2 - RM
            const int Cr = Mr - RM;
            R Tc = R(0);
            if (coll && Cr >= yc0 && Cr <= yc1) {
                const int cr = Cr - r0;  // >= RM + 3: every stencil row index below stays non-negative
                auto SF = [&](int f, int dy, int dx) {
                    return sten[((size_t)((cr + dy) % NSR) * G::NSF + f) * NT + tid + dx];
                };
                const R* lo = loc + (size_t)(cr % NLR) * G::NLF * NT + tid;
                Macro<R> m;
                m.rho = lo[0];
                m.ir = R(1) / m.rho;
                m.F[0] = lo[1 * NT];
                m.F[1] = lo[2 * NT];
                m.F[2] = R(0);
                m.P = lo[3 * NT];
                m.theta = lo[4 * NT];
                m.cv = lo[5 * NT];
                m.gam = lo[6 * NT];
                m.athe = lo[7 * NT];
                m.e = lo[8 * NT];
                m.icv = EK == EOS_PR ? R(1) / m.cv : s.inv_cv;
                m.Q = heat_q<R>(s, 0);
                m.u[0] = SF(0, 0, 0);
                m.u[1] = SF(1, 0, 0);
                m.u[2] = R(0);
                m.T = SF(2, 0, 0);
                m.h = SF(3, 0, 0);
                const R divu = R(0.5) * (SF(0, 0, 1) - SF(0, 0, -1)) + R(0.5) * (SF(1, 1, 0) - SF(1, -1, 0));
                const R gh[3] = {R(0.5) * (SF(3, 0, 1) - SF(3, 0, -1)), R(0.5) * (SF(3, 1, 0) - SF(3, -1, 0)), R(0)};
                const R gT[3] = {R(0.5) * (SF(2, 0, 1) - SF(2, 0, -1)), R(0.5) * (SF(2, 1, 0) - SF(2, -1, 0)), R(0)};
                R dX[2];
                if (PC || s.phi_central) {
                    dX[0] = R(0.5) * (SF(4, 0, 1) - SF(4, 0, -1));
                    dX[1] = R(0.5) * (SF(5, 1, 0) - SF(5, -1, 0));
                } else {
                    // upwind-biased by the sign of u_alpha; RM = 2 here, so +-2 is in range
                    const bool px = m.u[0] >= R(0), py = m.u[1] >= R(0);
                    dX[0] = upwind_biased<R>(m.u[0], SF(4, 0, px ? -2 : 2), SF(4, 0, -1), SF(4, 0, 0), SF(4, 0, 1));
                    dX[1] = upwind_biased<R>(m.u[1], SF(5, py ? -2 : 2, 0), SF(5, -1, 0), SF(5, 0, 0), SF(5, 1, 0));
                }
                const R Phi[3] = {-dX[0] * m.ir, -dX[1] * m.ir, R(0)};
                // pre-collision populations: f_i(x) = f'_i(x - c_i), staged row by row
                const S* ps = popr + (size_t)(st % K) * 18 * PWP + (xm - xap);
                R f[9], g[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    f[i] = stored_to_f<S>(ps[i * PWP - cc(i, 0)]);
                    g[i] = stored_to_f<S>(ps[(9 + i) * PWP - cc(i, 0)]);
                    if (Codec<S, R>::offset) {
                        f[i] += s.fref[i];
                        g[i] += s.gref[i];
                    }
                }
                collide_cell<2, R>(s, m, divu, gh, gT, Phi, f, g);
                if (own_x && Cr >= y0 && Cr < y0 + vy) {
                    // one pointer per cell, advanced by N from population to population
                    S* po = fo + ((unsigned)xm + (unsigned)nx * (unsigned)Cr);
#pragma unroll
                    for (int i = 0; i < 9; ++i, po += Ncell)
                        Codec<S, R>::st(po, f[i] - (Codec<S, R>::offset ? s.fref[i] : R(0)));
#pragma unroll
                    for (int i = 0; i < 9; ++i, po += Ncell)
                        Codec<S, R>::st(po, g[i] - (Codec<S, R>::offset ? s.gref[i] : R(0)));
                }
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    gbuf[i * NT + tid] = f[i];
                    gbuf[(9 + i) * NT + tid] = g[i];
                }
                Tc = m.T;
            }
            Tq2 = Tq1;
            Tq1 = Tc;
        }
        cp_async_wait<0>();
        __syncthreads();  // the rings are reused by the next tile
    }
}

// CTAs of the row march resident on the whole device: the persistent grid
template <typename S, int EK, bool PC>
cudaError_t ymarch_grid_cap(int& cap)
{
    constexpr size_t smem = YmShape<S, PC>::smem_bytes;
    static_assert(smem <= 227u * 1024u, "row-march rings do not fit in shared memory");
    static int grid_cap = 0;
    if (grid_cap == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_ymarch<S, EK, PC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0, dev = 0, nsm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ymarch<S, EK, PC>, kYmThreads, smem);
        if (e != cudaSuccess) return e;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        grid_cap = per_sm * nsm;
    }
    cap = grid_cap;
    return cudaSuccess;
}

template <typename S, int EK, bool PC>
cudaError_t ymarch_launch(const SimDev* sims, const TileEntry* tiles, int ntiles, int YL, const void* src, void* dst,
                          const void* Min, void* Mout, long long Ntot, unsigned long long* diag, cudaStream_t stream)
{
    constexpr size_t smem = YmShape<S, PC>::smem_bytes;
    int grid_cap = 0;
    cudaError_t e = ymarch_grid_cap<S, EK, PC>(grid_cap);
    if (e != cudaSuccess) return e;
    const int grid = ntiles < grid_cap ? ntiles : grid_cap;
    k_ymarch<S, EK, PC><<<grid, kYmThreads, smem, stream>>>(sims, tiles, ntiles, YL, (const S*)src, (S*)dst,
                                                           (const float*)Min, (float*)Mout, Ntot, diag);
    return cudaGetLastError();
}

template <typename S>
cudaError_t ymarch_dispatch_t(int eos, int pc, int yl, const SimDev* sims, const TileEntry* tiles, int ntiles,
                              const void* src, void* dst, const void* Min, void* Mout, long long Ntot,
                              unsigned long long* diag, cudaStream_t stream)
{
#define LBM_YM(EK, P) return ymarch_launch<S, EK, P>(sims, tiles, ntiles, yl, src, dst, Min, Mout, Ntot, diag, stream)
    if (pc) {
        if (eos == EOS_IDEAL) LBM_YM(EOS_IDEAL, true);
        if (eos == EOS_VDW) LBM_YM(EOS_VDW, true);
        if (eos == EOS_PR) LBM_YM(EOS_PR, true);
    } else {
        if (eos == EOS_IDEAL) LBM_YM(EOS_IDEAL, false);
        if (eos == EOS_VDW) LBM_YM(EOS_VDW, false);
        if (eos == EOS_PR) LBM_YM(EOS_PR, false);
    }
#undef LBM_YM
    return cudaErrorInvalidValue;
}

template <typename S>
cudaError_t ymarch_slots_t(int eos, int pc, int* slots)
{
#define LBM_YS(EK, P) return ymarch_grid_cap<S, EK, P>(*slots)
    if (pc) {
        if (eos == EOS_IDEAL) LBM_YS(EOS_IDEAL, true);
        if (eos == EOS_VDW) LBM_YS(EOS_VDW, true);
        if (eos == EOS_PR) LBM_YS(EOS_PR, true);
    } else {
        if (eos == EOS_IDEAL) LBM_YS(EOS_IDEAL, false);
        if (eos == EOS_VDW) LBM_YS(EOS_VDW, false);
        if (eos == EOS_PR) LBM_YS(EOS_PR, false);
    }
#undef LBM_YS
    return cudaErrorInvalidValue;
}

static_assert(YmShape<float, true>::TX == kYmStripCentral && YmShape<float, false>::TX == kYmStripUpwind &&
                  YmShape<__half, true>::TX == kYmStripCentral && YmShape<__half, false>::TX == kYmStripUpwind,
              "the host tiles strips of the kernel's width");

}  // namespace lbm
