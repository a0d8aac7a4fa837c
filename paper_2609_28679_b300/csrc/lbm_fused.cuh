// One-pass ("fused") time step on shared-memory tiles.
//
// The step needs the moments of every cell within 5 cells of the cells it
// updates (rho for grad lap rho at radius 2 of the radius-3 macroscopic state
// that the radius-2 stencils of Phi and the radius-1 gradients consume, plus
// one ring of neighbours for the next moments).  Instead of a separate pass
// that re-reads all populations to form those moments, every step carries
// them: a CTA owning tile T
//   1. loads rho on T+5 from the moment buffer of the current state,
//   2. computes lap rho on T+4,
//   3. computes u, e, T, P, theta, ... on T+3 (cells beyond a z wall are
//      mirror copies of their images, velocity and X negated),
//   4. pulls the populations of T+1 once, collides them, stores those of T,
//      and adds each post-collision population of T+1 to the next-step moment
//      (rho, j, G) of the cell it streams into, if that cell is in T,
//   5. writes the next-step moments (and T as the next Newton guess) of T.
// Populations are thus read and written once per step; the moment buffers
// (6 values per cell) are double-buffered like the populations.  Tile shapes
// are compile-time so that every region index is a constant-divisor
// computation.
#pragma once

#include "lbm_device.cuh"
#include "lbm_split.cuh"

namespace lbm {

struct TileEntry {
    int sim, x0, y0, z0;
};


// RB: radius of the rho halo (5; 4 when Phi takes the central derivative and
// the macroscopic state is needed on T+2 only); lap rho on T+(RB-1) and the
// macroscopic state on T+(RB-2).
template <int D, int TX, int TY, int TZ, int RB = 5> struct TileShape {
    static constexpr int HZ = D == 3 ? 1 : 0;
    static constexpr int tz = D == 3 ? TZ : 1;
    __host__ __device__ static constexpr int w(int r) { return TX + 2 * r; }
    __host__ __device__ static constexpr int h(int r) { return TY + 2 * r; }
    __host__ __device__ static constexpr int d(int r) { return D == 3 ? TZ + 2 * r : 1; }
    __host__ __device__ static constexpr int n(int r) { return w(r) * h(r) * d(r); }
    // stencil fields on T+3: u (D), T, h, X (D); local fields on T+1: P, theta, cv, gamma, alpha theta, e
    static constexpr int NS = 2 * D + 2, NL = 6;
    static constexpr int U = 0, TT = D, H = D + 1, X = D + 2;
    static constexpr int LP = 0, LTH = 1, LCV = 2, LGAM = 3, LATHE = 4, LE = 5;
    __host__ __device__ static constexpr size_t elems()
    {
        return (size_t)n(RB) + n(RB - 1) + (size_t)NS * n(RB - 2) + (size_t)NL * n(1) + (size_t)(D + 2) * n(0);
    }
};

// periodic wrap of a coordinate at most one period outside [0, n), with a
// general fallback for periods shorter than the halo
__device__ __forceinline__ int wrapc(int v, int n)
{
    if (v < 0) v += n;
    else if (v >= n) v -= n;
    if ((unsigned)v >= (unsigned)n) v = ((v % n) + n) % n;
    return v;
}

// coordinate of a stencil neighbour in z: periodic, or mirrored beyond walls
template <typename C>
__device__ __forceinline__ int zcoord(const C& s, int z, bool& flip)
{
    flip = false;
    if (!s.zwalls) return wrapc(z, s.nz);
    return mirror_z(z, s.nz, flip);
}

// Constants with the equation of state fixed at compile time: every
// `s.eos == ...` test in the shared helpers folds away.
template <typename R, int EK> struct SimK : SimC<R> {
    static constexpr int eos = EK;
};

// Threads of the fused kernel (one place to change it per tile shape; 288
// threads for 64x14, which would spare the collide phase its nearly empty
// fifth pass, measured slower: the register cap of 96 made the kernel spill).
template <int D, int TX, int TY, int TZ> constexpr int fused_threads()
{
    return 256;
}

// CTAs per SM that the tile's shared memory leaves room for (float32 2-D
// tiles; at most 3): the register budget the compiler may use follows from it.
template <int D, typename R, int TX, int TY, int TZ, bool PC> constexpr int fused_min_blocks()
{
    if (!(D == 2 && sizeof(R) == 4)) return 1;
    constexpr size_t bytes = TileShape<D, TX, TY, TZ, PC ? 4 : 5>::elems() * sizeof(R) + 1024;
    constexpr int n = (int)((size_t)232448 / bytes);
    return n < 1 ? 1 : (n > 3 ? 3 : n);
}

// PC: Phi from the central derivative of X for every simulation of the
// launch, so the halos shrink by one cell (see TileShape)
template <int D, typename R, typename S, int EK, bool ML, int TX, int TY, int TZ, bool PC>
__global__ void __launch_bounds__((fused_threads<D, TX, TY, TZ>()), (fused_min_blocks<D, R, TX, TY, TZ, PC>()))
    k_fused(const SimDev* __restrict__ sims, const TileEntry* __restrict__ tiles, int ntiles,
            const S* __restrict__ src, S* __restrict__ dst, const R* __restrict__ Min, R* __restrict__ Mout,
            long long Ntot, unsigned long long* diag)
{
    constexpr int RB = PC ? 4 : 5, RLP = RB - 1, RM = RB - 2;  // halo radii of rho, lap rho, the macroscopic state
    using G = TileShape<D, TX, TY, TZ, RB>;
    constexpr int NT = fused_threads<D, TX, TY, TZ>();
    constexpr int Q = Lat<D>::Q;
    constexpr int HZ = G::HZ;
    constexpr int n5 = G::n(RB), n4 = G::n(RLP), n3 = G::n(RM), n1 = G::n(1), n0 = G::n(0);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ SimK<R, EK> s;
    __shared__ SimDev s_dev;  // raw constants of simulation dev_sim, converted into s when a tile needs them
    __shared__ int cur_sim;
    R* s_rho = reinterpret_cast<R*>(smem_raw);
    R* s_L = s_rho + n5;
    R* s_st = s_L + n4;            // [NS][n3]
    R* s_lo = s_st + G::NS * n3;   // [NL][n1]
    R* s_acc = s_lo + G::NL * n1;  // [D+2][n0]
    MlpSmem& mlp_s = *reinterpret_cast<MlpSmem*>(s_acc + (D + 2) * n0);  // only with ML
    const int tid = threadIdx.x;
    if (tid == 0) cur_sim = -1;
    // the constants of simulation 0 are fetched by all threads at once, in
    // parallel with the first tile entry (other simulations on demand)
    auto fetch_sim = [&](int sim) {
        const int* src = reinterpret_cast<const int*>(sims + sim);
        int* d = reinterpret_cast<int*>(&s_dev);
        for (int w = tid; w < (int)(sizeof(SimDev) / sizeof(int)); w += NT) d[w] = src[w];
    };
    int dev_sim = 0;
    fetch_sim(0);
    __syncthreads();

    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const TileEntry te = tiles[t];
        if (te.sim != cur_sim) {
            __syncthreads();
            if (te.sim != dev_sim) {  // block-uniform
                fetch_sim(te.sim);
                dev_sim = te.sim;
                __syncthreads();
            }
            simc_from_coop<R>(static_cast<SimC<R>&>(s), s_dev, tid);
            if (tid == 0) cur_sim = te.sim;
            __syncthreads();
            if (ML && s.mlp != nullptr) {
                mlp_load(mlp_s, s.mlp);
                __syncthreads();
            }
        }
        const int nx = s.nx, ny = s.ny, nz = s.nz;
        const bool walls = D == 3 && s.zwalls;
        const long long off = s.cell_off;
        const unsigned Ncell = (unsigned)s.N;
        // owned extent of the tile (ragged at the domain's far edges)
        const unsigned vx = (unsigned)min(TX, nx - te.x0), vy = (unsigned)min(TY, ny - te.y0);
        const unsigned vz = (unsigned)min(G::tz, nz - te.z0);
        const R* Mrho = Min + M_RHO * Ntot + off;
        const R* Mj = Min + M_J * Ntot + off;
        const R* MG = Min + M_G * Ntot + off;
        const R* MT = Min + M_T * Ntot + off;

        // global inputs of the macroscopic state of cell k of T+3, fetched one
        // iteration ahead so that their latency overlaps the work before use
        struct In3 {
            R j[3], Gm, T;
        };
        auto fetch3 = [&](int k) {
            In3 v;
            v.j[0] = v.j[1] = v.j[2] = v.Gm = v.T = R(0);
            if (k < n3) {
                const int lx = k % G::w(RM), ly = (k / G::w(RM)) % G::h(RM), lz = k / (G::w(RM) * G::h(RM));
                const int zr = te.z0 - RM * HZ + lz;
                if (!(walls && (zr < 0 || zr >= nz))) {
                    const int x = wrapc(te.x0 - RM + lx, nx), y = wrapc(te.y0 - RM + ly, ny);
                    const int z = D == 3 ? wrapc(zr, nz) : 0;
                    const unsigned gk = (unsigned)x + (unsigned)nx * ((unsigned)y + (unsigned)ny * (unsigned)z);
#pragma unroll
                    for (int a = 0; a < D; ++a) v.j[a] = Mj[(size_t)a * Ntot + gk];
                    v.Gm = MG[gk];
                    v.T = MT[gk];
                }
            }
            return v;
        };
        In3 nxt3 = fetch3(tid);

        // ---- 1. rho on T+5 (ghosts beyond walls: the image's value); zero the accumulators.
        // All of a thread's loads are issued before the first store, so the
        // phase waits for one memory round trip rather than one per element.
        {
            constexpr int nb5 = (n5 + NT - 1) / NT;
            R rv[nb5];
#pragma unroll
            for (int it = 0; it < nb5; ++it) {
                const int k = it * NT + tid;
                rv[it] = R(0);
                if (k < n5) {
                    const int lx = k % G::w(RB), ly = (k / G::w(RB)) % G::h(RB), lz = k / (G::w(RB) * G::h(RB));
                    bool fl;
                    const int x = wrapc(te.x0 - RB + lx, nx), y = wrapc(te.y0 - RB + ly, ny);
                    const int z = D == 3 ? zcoord(s, te.z0 - RB + lz, fl) : 0;
                    rv[it] = Mrho[(unsigned)x + (unsigned)nx * ((unsigned)y + (unsigned)ny * (unsigned)z)];
                }
            }
#pragma unroll
            for (int it = 0; it < nb5; ++it) {
                const int k = it * NT + tid;
                if (k < n5) s_rho[k] = rv[it];
            }
        }
        for (int k = tid; k < (D + 2) * n0; k += NT) s_acc[k] = R(0);
        __syncthreads();

        // ---- 2. lap rho on T+4 (non-ghost cells; ghosts copied from images after)
        for (int k = tid; k < n4; k += NT) {
            const int lx = k % G::w(RLP), ly = (k / G::w(RLP)) % G::h(RLP), lz = k / (G::w(RLP) * G::h(RLP));
            const int z = te.z0 - RLP * HZ + lz;
            if (walls && (z < 0 || z >= nz)) continue;
            const int c = (lx + 1) + G::w(RB) * ((ly + 1) + G::h(RB) * (lz + HZ));
            constexpr int sy = G::w(RB), sz = G::w(RB) * G::h(RB);
            R L = s_rho[c + 1] + s_rho[c - 1] + s_rho[c + sy] + s_rho[c - sy] - R(2 * D) * s_rho[c];
            if (D == 3) L += s_rho[c + sz] + s_rho[c - sz];
            s_L[k] = L;
        }
        __syncthreads();
        if (walls && (te.z0 < RLP || te.z0 + G::tz + RLP > nz)) {
            for (int k = tid; k < n4; k += NT) {
                const int lx = k % G::w(RLP), ly = (k / G::w(RLP)) % G::h(RLP), lz = k / (G::w(RLP) * G::h(RLP));
                const int z = te.z0 - RLP * HZ + lz;
                if (z >= 0 && z < nz) continue;
                bool fl;
                const int li = mirror_z(z, nz, fl) - (te.z0 - RLP * HZ);
                s_L[k] = (li >= 0 && li < G::d(RLP)) ? s_L[lx + G::w(RLP) * (ly + G::h(RLP) * li)] : R(0);
            }
            __syncthreads();
        }

        const S* fb = src + s.pop_off;
        const S* gb = fb + (size_t)Q * s.N;
        S* fo = dst + s.pop_off;
        S* go = fo + (size_t)Q * s.N;
        // pre-collision populations of cell k of T+1: f_i(x) = f'_i(x - c_i),
        // or f'_opp(i)(x) across a z wall (16-bit storage: offsets added back)
        auto fetch4 = [&](int k, R* f, R* gp) {
            if (k >= n1) return;
            const int lx = k % G::w(1), ly = (k / G::w(1)) % G::h(1), lz = k / (G::w(1) * G::h(1));
            const int zr = te.z0 - HZ + lz;
            if (walls && (zr < 0 || zr >= nz)) return;
            const int x = wrapc(te.x0 - 1 + lx, nx), y = wrapc(te.y0 - 1 + ly, ny);
            const int z = D == 3 ? wrapc(zr, nz) : 0;
            // pull: f_i(x) = f'_i(x - c_i), or f'_opp(i)(x) across a z wall
            const int xs[3] = {x, x == 0 ? nx - 1 : x - 1, x == nx - 1 ? 0 : x + 1};  // x - c for digit 0,1,2
            const int ys[3] = {y, y == 0 ? ny - 1 : y - 1, y == ny - 1 ? 0 : y + 1};
            int zs[3] = {z, 0, 0};
            bool zwall[3] = {false, false, false};
            if (D == 3) {
                zs[1] = z - 1;
                zs[2] = z + 1;
                if (walls) {
                    zwall[1] = zs[1] < 0;
                    zwall[2] = zs[2] >= nz;
                } else {
                    zs[1] = z == 0 ? nz - 1 : z - 1;
                    zs[2] = z == nz - 1 ? 0 : z + 1;
                }
            }
            const unsigned self = (unsigned)x + (unsigned)nx * ((unsigned)y + (unsigned)ny * (unsigned)z);
            unsigned rows[3][3];  // row offsets (y, z) of the pull sources
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int c = 0; c < (D == 3 ? 3 : 1); ++c)
                    rows[b][c] = (unsigned)nx * ((unsigned)ys[b] + (unsigned)ny * (unsigned)zs[c]);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int d0 = dig(i, 0), d1 = dig(i, 1), d2 = D == 3 ? dig(i, 2) : 0;
                unsigned idx;
                int isrc = i;
                if (D == 3 && zwall[d2]) {
                    isrc = opp(i);
                    idx = (unsigned)isrc * Ncell + self;
                } else {
                    idx = (unsigned)i * Ncell + (unsigned)xs[d0] + rows[d1][d2];
                }
                f[i] = Codec<S, R>::ld(fb + idx);
                gp[i] = Codec<S, R>::ld(gb + idx);
                if (Codec<S, R>::offset) {
                    f[i] += s.fref[isrc];
                    gp[i] += s.gref[isrc];
                }
            }
        };
        // 2-D: the populations of the next cell are fetched while this one collides
        constexpr bool kAhead = D == 2;
        R fn[Q], gn[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) fn[i] = gn[i] = R(0);
        if (kAhead) fetch4(tid, fn, gn);  // first cell of phase 4, in flight during phase 3

        // ---- 3. macroscopic state on T+3
        constexpr int nb3 = (n3 + NT - 1) / NT;
#pragma unroll 2
        for (int it = 0; it < nb3; ++it) {
            const int k = it * NT + tid;
            const In3 in3 = nxt3;
            if (it + 1 < nb3) nxt3 = fetch3(k + NT);
            unsigned flags = 0;
            bool owned = false, act = false;
            int lx = 0, ly = 0, lz = 0, zr = 0, z = 0;
            R r = R(1), G_ = R(0), Qh = R(0), Tg = R(0), Fv[3] = {0, 0, 0}, j[3] = {0, 0, 0};
            if (k < n3) {
                lx = k % G::w(RM);
                ly = (k / G::w(RM)) % G::h(RM);
                lz = k / (G::w(RM) * G::h(RM));
                zr = te.z0 - RM * HZ + lz;
                act = !(walls && (zr < 0 || zr >= nz));
                if (act) {
                    z = D == 3 ? wrapc(zr, nz) : 0;
                    const int c4 = (lx + 1) + G::w(RLP) * ((ly + 1) + G::h(RLP) * (lz + HZ));
                    r = s_rho[(lx + 2) + G::w(RB) * ((ly + 2) + G::h(RB) * (lz + 2 * HZ))];
                    constexpr int st4[3] = {1, G::w(RLP), G::w(RLP) * G::h(RLP)};
#pragma unroll
                    for (int a = 0; a < D; ++a) {
                        Fv[a] = r * (s.acc[a] + s.kappa * R(0.5) * (s_L[c4 + st4[a]] - s_L[c4 - st4[a]]));
                        j[a] = in3.j[a];
                    }
                    G_ = in3.Gm;
                    Qh = heat_q<R>(s, z);
                    Tg = in3.T;
                }
            }
            if constexpr (ML) {
                if (s.mlp != nullptr) {  // block-uniform: the whole warp evaluates the network
                    const float rr = act ? (float)r : 1.f;
                    const float ee = act ? (float)macro_energy<D, R>(r, j, G_, Fv, Qh) : 0.f;
                    const float Tm = mlp_T_warp(mlp_s, rr, ee);
                    if (act) Tg = (R)Tm;
                }
            }
            if (act) {
                const Macro<R> m = macro_cell<D, R>(s, r, j, G_, Fv, Qh, Tg, flags);
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    s_st[(G::U + a) * n3 + k] = m.u[a];
                    s_st[(G::X + a) * n3 + k] = xflux<R>(r, m.u[a], m.theta);
                }
                s_st[G::TT * n3 + k] = m.T;
                s_st[G::H * n3 + k] = m.h;
                // local fields for the cells of T+1
                const int l1x = lx - (RM - 1), l1y = ly - (RM - 1), l1z = lz - (RM - 1) * HZ;
                if (l1x >= 0 && l1y >= 0 && l1z >= 0 && l1x < G::w(1) && l1y < G::h(1) && l1z < G::d(1)) {
                    const int k1 = l1x + G::w(1) * (l1y + G::h(1) * l1z);
                    s_lo[G::LP * n1 + k1] = m.P;
                    s_lo[G::LTH * n1 + k1] = m.theta;
                    s_lo[G::LCV * n1 + k1] = m.cv;
                    s_lo[G::LGAM * n1 + k1] = m.gam;
                    s_lo[G::LATHE * n1 + k1] = m.athe;
                    s_lo[G::LE * n1 + k1] = m.e;
                }
                owned = lx >= RM && ly >= RM && lz >= RM * HZ && lx < RM + TX && ly < RM + TY && lz < RM * HZ + G::tz &&
                        te.x0 - RM + lx < nx && te.y0 - RM + ly < ny && zr < nz;
            }
            if (diag) count_flags(owned ? flags : 0u, diag);
        }
        __syncthreads();
        if (walls && (te.z0 < RM || te.z0 + G::tz + RM > nz)) {
            for (int k = tid; k < n3; k += NT) {
                const int lx = k % G::w(RM), ly = (k / G::w(RM)) % G::h(RM), lz = k / (G::w(RM) * G::h(RM));
                const int z = te.z0 - RM * HZ + lz;
                if (z >= 0 && z < nz) continue;
                bool fl;
                const int li = mirror_z(z, nz, fl) - (te.z0 - RM * HZ);
                if (li < 0 || li >= G::d(RM)) continue;  // image outside the tile's region: never read
                const int ki = lx + G::w(RM) * (ly + G::h(RM) * li);
#pragma unroll
                for (int f = 0; f < G::NS; ++f) {
                    const R v = s_st[f * n3 + ki];
                    const bool odd = (f >= G::U && f < G::U + D) || (f >= G::X && f < G::X + D);
                    s_st[f * n3 + k] = (odd && fl) ? -v : v;
                }
            }
            __syncthreads();
        }

        // ---- 4. collide T+1, store T, accumulate the next moments of T
        for (int k = tid; k < n1; k += NT) {
            R f[Q], gp[Q];
            if (kAhead) {
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    f[i] = fn[i];
                    gp[i] = gn[i];
                }
                fetch4(k + NT, fn, gn);
            }
            const int lx = k % G::w(1), ly = (k / G::w(1)) % G::h(1), lz = k / (G::w(1) * G::h(1));
            const int zr = te.z0 - HZ + lz;
            if (walls && (zr < 0 || zr >= nz)) continue;
            const int x = wrapc(te.x0 - 1 + lx, nx), y = wrapc(te.y0 - 1 + ly, ny);
            const int z = D == 3 ? wrapc(zr, nz) : 0;
            const int c3 = (lx + RM - 1) + G::w(RM) * ((ly + RM - 1) + G::h(RM) * (lz + (RM - 1) * HZ));
            const int c4 = (lx + RLP - 1) + G::w(RLP) * ((ly + RLP - 1) + G::h(RLP) * (lz + (RLP - 1) * HZ));
            constexpr int st3[3] = {1, G::w(RM), G::w(RM) * G::h(RM)};
            constexpr int st4[3] = {1, G::w(RLP), G::w(RLP) * G::h(RLP)};
            Macro<R> m;
            m.rho = s_rho[(lx + RB - 1) + G::w(RB) * ((ly + RB - 1) + G::h(RB) * (lz + (RB - 1) * HZ))];
            m.ir = R(1) / m.rho;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                m.u[a] = a < D ? s_st[(G::U + a) * n3 + c3] : R(0);
                m.F[a] = a < D ? m.rho * (s.acc[a] + s.kappa * R(0.5) * (s_L[c4 + st4[a]] - s_L[c4 - st4[a]]))
                               : R(0);
            }
            m.Q = heat_q<R>(s, z);
            m.T = s_st[G::TT * n3 + c3];
            m.h = s_st[G::H * n3 + c3];
            m.P = s_lo[G::LP * n1 + k];
            m.theta = s_lo[G::LTH * n1 + k];
            m.cv = s_lo[G::LCV * n1 + k];
            m.icv = s.eos == EOS_PR ? R(1) / m.cv : s.inv_cv;
            m.gam = s_lo[G::LGAM * n1 + k];
            m.athe = s_lo[G::LATHE * n1 + k];
            m.e = s_lo[G::LE * n1 + k];
            R divu = 0, gh[3] = {0, 0, 0}, gT[3] = {0, 0, 0}, Phi[3] = {0, 0, 0};
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const int sa = st3[a];
                const R* ua = s_st + (G::U + a) * n3;
                const R* Xa = s_st + (G::X + a) * n3;
                divu += R(0.5) * (ua[c3 + sa] - ua[c3 - sa]);
                gh[a] = R(0.5) * (s_st[G::H * n3 + c3 + sa] - s_st[G::H * n3 + c3 - sa]);
                gT[a] = R(0.5) * (s_st[G::TT * n3 + c3 + sa] - s_st[G::TT * n3 + c3 - sa]);
                R dX;
                if (PC || s.phi_central) {
                    dX = R(0.5) * (Xa[c3 + sa] - Xa[c3 - sa]);
                } else {
                    dX = upwind_biased<R>(m.u[a], Xa[c3 + (m.u[a] >= R(0) ? -2 : 2) * sa], Xa[c3 - sa], Xa[c3],
                                          Xa[c3 + sa]);
                }
                Phi[a] = -dX * m.ir;
            }

            if (!kAhead) fetch4(k, f, gp);
            const unsigned self = (unsigned)x + (unsigned)nx * ((unsigned)y + (unsigned)ny * (unsigned)z);
            collide_cell<D, R>(s, m, divu, gh, gT, Phi, f, gp);

            const int tx = lx - 1, ty = ly - 1, tz = lz - HZ;
            const bool inT = tx >= 0 && ty >= 0 && tz >= 0 && tx < TX && ty < TY && tz < G::tz;
            const int gx = te.x0 + tx, gy = te.y0 + ty, gz = te.z0 + tz;
            if (inT && gx < nx && gy < ny && gz < nz) {
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const R fr = Codec<S, R>::offset ? s.fref[i] : R(0);
                    const R gr = Codec<S, R>::offset ? s.gref[i] : R(0);
                    Codec<S, R>::st(fo + (unsigned)i * Ncell + self, f[i] - fr);
                    Codec<S, R>::st(go + (unsigned)i * Ncell + self, gp[i] - gr);
                }
            }
            // next-step moments: f'_i(x) becomes f_i(x + c_i), or f_opp(i)(x) across a z wall.
            // Branch-free: a destination counts if it lies in the owned part of T.
            if constexpr (D == 2) {
                // per axis, whether the neighbour at c = 0, +1, -1 is owned
                bool okx[3], oky[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    okx[d] = (unsigned)(tx + cval(d)) < vx;
                    oky[d] = (unsigned)(ty + cval(d)) < vy;
                }
                const int dbase = tx + TX * ty;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const int ci0 = cc(i, 0), ci1 = cc(i, 1);
                    if (okx[dig(i, 0)] && oky[dig(i, 1)]) {
                        const int dd = dbase + ci0 + TX * ci1;
                        atomicAdd(&s_acc[dd], f[i]);
                        if (ci0 != 0) atomicAdd(&s_acc[n0 + dd], ci0 > 0 ? f[i] : -f[i]);
                        if (ci1 != 0) atomicAdd(&s_acc[2 * n0 + dd], ci1 > 0 ? f[i] : -f[i]);
                        atomicAdd(&s_acc[3 * n0 + dd], gp[i]);
                    }
                }
            } else {
                const bool zlo_wall = walls && z == 0, zhi_wall = walls && z == nz - 1;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const int ci0 = cc(i, 0), ci1 = cc(i, 1), ci2 = cc(i, 2);
                    const bool bounce = (ci2 < 0 && zlo_wall) || (ci2 > 0 && zhi_wall);
                    const int dx = bounce ? tx : tx + ci0, dy = bounce ? ty : ty + ci1, dz = bounce ? tz : tz + ci2;
                    const bool ok = (unsigned)dx < vx && (unsigned)dy < vy && (unsigned)dz < vz;
                    if (ok) {
                        const int dd = dx + TX * (dy + TY * dz);
                        atomicAdd(&s_acc[dd], f[i]);
#pragma unroll
                        for (int a = 0; a < D; ++a) {
                            const int ca = cc(i, a);
                            if (ca != 0) atomicAdd(&s_acc[(1 + a) * n0 + dd], (ca > 0) != bounce ? f[i] : -f[i]);
                        }
                        atomicAdd(&s_acc[(1 + D) * n0 + dd], gp[i]);
                    }
                }
            }
        }
        __syncthreads();

        // ---- 5. next-step moments and Newton guess of T
        for (int d = tid; d < n0; d += NT) {
            const int tx = d % TX, ty = (d / TX) % TY, tz = d / (TX * TY);
            const int x = te.x0 + tx, y = te.y0 + ty, z = te.z0 + tz;
            if (x >= nx || y >= ny || z >= nz) continue;
            const unsigned kk = (unsigned)x + (unsigned)nx * ((unsigned)y + (unsigned)ny * (unsigned)z);
            R* Mo = Mout + off;
            Mo[M_RHO * Ntot + kk] = s_acc[d];
#pragma unroll
            for (int a = 0; a < 3; ++a) Mo[(M_J + a) * Ntot + kk] = a < D ? s_acc[(1 + a) * n0 + d] : R(0);
            Mo[M_G * Ntot + kk] = s_acc[(1 + D) * n0 + d];
            Mo[M_T * Ntot + kk] = s_st[G::TT * n3 + (tx + RM) + G::w(RM) * ((ty + RM) + G::h(RM) * (tz + RM * HZ))];
        }
        __syncthreads();
    }
}

// Moments (and the Newton guess from the split path's T) of the current state,
// before the first fused step after lbm_init or a split step.
template <int D, typename R, typename S>
__global__ void __launch_bounds__(kBlockCells) k_fused_prep(const SimDev* __restrict__ sims,
                                                            const BlockEntry* __restrict__ table,
                                                            const S* __restrict__ pop, const R* __restrict__ W,
                                                            R* __restrict__ M, long long Ntot)
{
    constexpr int Q = Lat<D>::Q;
    __shared__ SimDev s;
    const BlockEntry be = table[blockIdx.x];
    load_sim(s, sims, be.sim);
    const long long k = (long long)be.start + threadIdx.x;
    if (k >= s.N) return;
    int x, y, z;
    cell_xyz(s, k, x, y, z);
    R f[Q], g[Q];
    pull_cell<D, R, S>(s, pop, x, y, z, f, g);
    R rho = 0, j[3] = {0, 0, 0}, G = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        rho += f[i];
#pragma unroll
        for (int a = 0; a < D; ++a) j[a] += R(cc(i, a)) * f[i];
        G += g[i];
    }
    const long long gk = s.cell_off + k;
    M[M_RHO * Ntot + gk] = rho;
#pragma unroll
    for (int a = 0; a < 3; ++a) M[(M_J + a) * Ntot + gk] = j[a];
    M[M_G * Ntot + gk] = G;
    M[M_T * Ntot + gk] = W[W_T * Ntot + gk];
}

template <int D, typename R, typename S>
void fused_moments_launch(const SimDev* sims, const BlockEntry* table, int nblocks, const S* pop, const R* W, R* M,
                          long long Ntot, cudaStream_t stream)
{
    k_fused_prep<D, R, S><<<nblocks, kBlockCells, 0, stream>>>(sims, table, pop, W, M, Ntot);
}

// ---------------------------------------------------------------------------
// Launch of one instantiated shape (persistent grid: resident CTAs x SMs).
// ---------------------------------------------------------------------------
template <int D, typename R, int TX, int TY, int TZ, bool PC> constexpr size_t fused_smem()
{
    return TileShape<D, TX, TY, TZ, PC ? 4 : 5>::elems() * sizeof(R);
}

template <int D, typename R, typename S, int EK, bool ML, int TX, int TY, int TZ, bool PC>
cudaError_t fused_launch_pc(const SimDev* sims, const TileEntry* tiles, int ntiles, const void* src, void* dst,
                            const void* Min, void* Mout, long long Ntot, unsigned long long* diag, cudaStream_t stream)
{
    constexpr size_t smem = fused_smem<D, R, TX, TY, TZ, PC>() + (ML ? sizeof(MlpSmem) : 0);
    constexpr int nt = fused_threads<D, TX, TY, TZ>();
    static_assert(smem <= 227u * 1024u, "tile does not fit in shared memory");
    static int grid_cap = 0;
    if (grid_cap == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_fused<D, R, S, EK, ML, TX, TY, TZ, PC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0, dev = 0, nsm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused<D, R, S, EK, ML, TX, TY, TZ, PC>, nt, smem);
        if (e != cudaSuccess) return e;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        grid_cap = per_sm * nsm;
    }
    const int grid = ntiles < grid_cap ? ntiles : grid_cap;
    k_fused<D, R, S, EK, ML, TX, TY, TZ, PC><<<grid, nt, smem, stream>>>(sims, tiles, ntiles, (const S*)src, (S*)dst,
                                                                        (const R*)Min, (R*)Mout, Ntot, diag);
    return cudaGetLastError();
}

// pc: every simulation of the launch takes the central Phi (2-D tiles then
// use the narrower halos)
template <int D, typename R, typename S, int EK, bool ML, int TX, int TY, int TZ>
cudaError_t fused_launch_shape(int pc, const SimDev* sims, const TileEntry* tiles, int ntiles, const void* src,
                               void* dst, const void* Min, void* Mout, long long Ntot, unsigned long long* diag,
                               cudaStream_t stream)
{
    if constexpr (D == 2) {
        if (pc)
            return fused_launch_pc<D, R, S, EK, ML, TX, TY, TZ, true>(sims, tiles, ntiles, src, dst, Min, Mout, Ntot,
                                                                     diag, stream);
    }
    return fused_launch_pc<D, R, S, EK, ML, TX, TY, TZ, false>(sims, tiles, ntiles, src, dst, Min, Mout, Ntot, diag,
                                                              stream);
}

}  // namespace lbm
