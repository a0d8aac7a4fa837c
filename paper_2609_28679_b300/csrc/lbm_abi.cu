// Host side of the C ABI declared in include/lbm.h: argument checking,
// device buffers (through PyTorch's caching allocator), simulation tables and
// kernel launches on the handle's stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_fused.cuh"
#include "lbm_fused_api.h"
#include "lbm_split.cuh"

extern "C" void* lbm_glue_alloc(size_t nbytes, void* stream);
extern "C" void lbm_glue_free(void* ptr);
extern "C" void* lbm_glue_current_stream(int device);

using namespace lbm;

struct lbm_ctx;

namespace {

thread_local std::string g_create_error;

struct Ops {
    // blocks [b0, b0 + nb) of the block table; nb < 0: all of them
    int (*init)(lbm_ctx*, const void*, const void*, const void*, int single, int b0, int nb);  // single: float32 fields
    int (*step)(lbm_ctx*, int);
    int (*macro)(lbm_ctx*);
    int (*export_moments)(lbm_ctx*, void*, void*, void*, int single, int b0, int nb);
    int (*export_pops)(lbm_ctx*, double*, double*);
    int (*invariants)(lbm_ctx*, double*);
    int (*fused_ok)(lbm_ctx*, int, int, int);
    int (*prepare)(lbm_ctx*);  // carried moments of the current state (fused and z-march variants)
    int (*prepare_part)(lbm_ctx*, int b0, int nb);  // the same for blocks [b0, b0 + nb), M left marked as it was
    int (*state_fields)(lbm_ctx*);  // rho, u, T of the current state into W (for the export)
    // the same for blocks [b0, b0 + nb) alone where the variant allows it (the z-march's first
    // pass); returns LBM_E_UNSUPPORTED, having done nothing, where it does not
    int (*state_part)(lbm_ctx*, int b0, int nb);
};

}  // namespace

struct lbm_ctx {
    int nsim = 0, dim = 0, Q = 0, storage = 0;
    size_t rbytes = 0, sbytes = 0;
    std::vector<SimDev> sims;
    SimDev* d_sims = nullptr;
    std::vector<BlockEntry> table;
    BlockEntry* d_table = nullptr;
    std::vector<BlockEntry> face_table;  // blocks of boundary cells of extrapolated faces (k_nee)
    BlockEntry* d_face_table = nullptr;
    std::vector<int> sim_block_start;
    int* d_sim_block_start = nullptr;
    std::vector<TileEntry> tiles;
    TileEntry* d_tiles = nullptr;
    long long Ntot = 0, pop_elems = 0;
    void* pop[2] = {nullptr, nullptr};
    int cur = 0;
    void* W = nullptr;            // split-path work arrays [W_NF][Ntot]
    void* M = nullptr;            // fused-path moments 2 x [M_NF][Ntot]
    unsigned long long* d_diag = nullptr;
    double* d_partials = nullptr;
    cudaStream_t stream = nullptr;
    int device = 0;
    bool initialized = false;
    bool moments_valid = false;   // fused path: M holds the moments of the current state
    int variant = LBM_KERNEL_SPLIT, tx = 0, ty = 0, tz = 0;
    int smem_bytes = 0;
    int graph_steps = 0;               // steps per captured CUDA graph (0: launch eagerly)
    float* d_mlp = nullptr;            // learned temperature parameters (lbm_mlp_load)
    cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};  // per starting buffer parity
    std::vector<cudaEvent_t> pass_ev;  // lbm_step_timed: 4 events per step (start, after passes 1, 2, 3)
    cudaStream_t xfer = nullptr;       // host-link copies of lbm_init / lbm_moments, beside the kernels
    std::vector<cudaEvent_t> xfer_ev;
    int pass_step = -1;                // step of lbm_step_timed being recorded (-1: none)
    std::string err;
    Ops ops{};
};

namespace {

int fail(lbm_ctx* h, int code, const std::string& msg)
{
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

int cuda_fail(lbm_ctx* h, cudaError_t e, const char* where)
{
    return fail(h, LBM_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define LBM_CUDA_CHECK(h, call)                                  \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
    } while (0)

#define LBM_LAUNCH_CHECK(h, what)                                 \
    do {                                                          \
        cudaError_t e_ = cudaGetLastError();                      \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, (what)); \
    } while (0)

void* dev_alloc(lbm_ctx* h, size_t n) { return lbm_glue_alloc(n, (void*)h->stream); }

// lbm_step_timed: mark the boundary k (0 start, 1-3 after each pass) of the step being recorded
void pass_mark(lbm_ctx* h, int k)
{
    if (h->pass_step >= 0) cudaEventRecord(h->pass_ev[4 * (size_t)h->pass_step + k], h->stream);
}

// some simulation of h has non-equilibrium-extrapolation walls
bool has_nee(const lbm_ctx* h)
{
    for (const SimDev& d : h->sims)
        if (d.zwalls == 2) return true;
    return false;
}

// the fused kernels run none of: extrapolated faces, duct friction, throttle, per-cell force or heat
bool split_only(const lbm_ctx* h)
{
    for (const SimDev& d : h->sims)
        if (d.zwalls == 2 || d.friction > 0.0 || d.throttle_K > 0.0 || d.ffield || d.qfield) return true;
    return false;
}

// per-cell force or heat fields: split kernels only
bool has_fields(const lbm_ctx* h)
{
    for (const SimDev& d : h->sims)
        if (d.ffield || d.qfield) return true;
    return false;
}

// duct friction or a throttle: split kernels only
bool has_resistance(const lbm_ctx* h)
{
    for (const SimDev& d : h->sims)
        if (d.friction > 0.0 || d.throttle_K > 0.0) return true;
    return false;
}

bool zmarch_shape(int storage, int tx, int ty);

// The tiled kernels address a population as (population index) * N + cell in
// 32-bit arithmetic; per: how many populations' worth of cells their largest
// offset spans (Q for the fused step, 27 for the z-marches, 18 for the row
// march, which indexes f and g from one base).  Larger simulations run on the
// split kernels, whose indices are 64-bit.
bool offsets32(const lbm_ctx* h, unsigned long long per)
{
    for (const SimDev& d : h->sims)
        if (per * (unsigned long long)d.N > 0xffffffffULL) return false;
    return true;
}

// the z-march kernel can run h with this xy tile (extrapolated faces: tiles
// 30 x 14 and 30 x 6 with 32- or 64-bit storage)
bool zmarch_ok(const lbm_ctx* h, int tx, int ty)
{
    if (h->dim != 3 || has_fields(h) || (has_resistance(h) && !has_nee(h)) || !offsets32(h, 27))
        return false;  // resistance: extrapolated variant only
    for (const SimDev& d : h->sims)
        if (d.eos != h->sims[0].eos) return false;
    if (has_nee(h))
        return (h->storage == LBM_F32 || h->storage == LBM_F64) && tx == 30 && (ty == 14 || ty == 6);
    return zmarch_shape(h->storage, tx, ty);
}

// the column-march kernel (staged pulls, gathered moments) can run h: D3Q27,
// 32- or 16-bit storage, one equation of state, no extrapolated faces,
// resistance or per-cell fields, nx a multiple of the elements per 16-byte copy
bool zgather_ok(const lbm_ctx* h)
{
    if (h->dim != 3 || h->storage == LBM_F64 || has_fields(h) || has_resistance(h) || has_nee(h) || !offsets32(h, 27))
        return false;
    const int chunk = h->storage == LBM_F32 ? 4 : 8;
    for (const SimDev& d : h->sims)
        if (d.eos != h->sims[0].eos || d.nx % chunk != 0) return false;
    return true;
}

// the row-march kernel can run h: D2Q9, 32- or 16-bit storage, one equation
// of state, no learned temperature, per-cell fields or resistance, nx a
// multiple of the elements per 16-byte copy
bool ymarch_ok(const lbm_ctx* h)
{
    if (h->dim != 2 || h->storage == LBM_F64 || has_fields(h) || has_resistance(h) || !offsets32(h, 18)) return false;
    const int chunk = h->storage == LBM_F32 ? 4 : 8;
    for (const SimDev& d : h->sims)
        if (d.eos != h->sims[0].eos || d.nx % chunk != 0 || d.t_solver == LBM_T_MLP) return false;
    return true;
}

// owned columns of a row-march strip (narrower when some simulation takes the upwind-biased Phi)
int ymarch_strip_width(const lbm_ctx* h)
{
    bool central = true;
    for (const SimDev& d : h->sims) central = central && d.phi_central;
    return central ? kYmStripCentral : kYmStripUpwind;
}

// every face of a simulation with zwalls == 2 has its data
bool faces_ready(const lbm_ctx* h)
{
    for (const SimDev& d : h->sims)
        if (d.zwalls == 2 && !(d.face_set[0] && d.face_set[1])) return false;
    return true;
}

cudaError_t fused_dispatch(int storage, int dim, int eos, int mlp, int pc, int tx, int ty, int tz, const SimDev* sims,
                           const TileEntry* tiles, int ntiles, const void* src, void* dst, const void* Min, void* Mout,
                           long long Ntot, unsigned long long* diag, cudaStream_t stream);
bool fused_shape(int storage, int dim, int tx, int ty, int tz);
cudaError_t zmarch_dispatch(int storage, int eos, int tx, int ty, int zl, const SimDev* sims, const TileEntry* tiles,
                            int ntiles, const void* src, void* dst, const void* W, void* Mout, long long Ntot,
                            cudaStream_t stream);
bool zmarch_shape(int storage, int tx, int ty);
cudaError_t zmarch_nee_dispatch(int storage, int eos, int tx, int ty, int zl, const SimDev* sims,
                                const TileEntry* tiles, int ntiles, const void* src, void* dst, const void* W,
                                void* Mout, long long Ntot, cudaStream_t stream);
cudaError_t zmacro_dispatch(int storage, int eos, int mlp, const SimDev* sims, const BlockEntry* table, int nblocks,
                            const void* M, void* W, long long Ntot, unsigned long long* diag, cudaStream_t stream);
cudaError_t zgather_dispatch(int storage, int eos, int zl, const SimDev* sims, const TileEntry* tiles, int ntiles,
                             const void* src, void* dst, const void* W, void* Mout, long long Ntot,
                             cudaStream_t stream);
cudaError_t ymarch_dispatch(int storage, int eos, int pc, int yl, const SimDev* sims, const TileEntry* tiles,
                            int ntiles, const void* src, void* dst, const void* Min, void* Mout, long long Ntot,
                            unsigned long long* diag, cudaStream_t stream);
int ymarch_rows(const lbm_ctx* h);

// ---------------------------------------------------------------------------
// Typed implementation of every operation for one (D, arithmetic, storage).
// ---------------------------------------------------------------------------
template <int D, typename R, typename S> struct Impl {
    // carried moments of the fused path, double-buffered with the populations
    static R* mbuf(lbm_ctx* h, int which) { return (R*)h->M + (size_t)which * M_NF * h->Ntot; }

    static int nblocks(lbm_ctx* h) { return (int)h->table.size(); }

    static int init(lbm_ctx* h, const void* rho, const void* u, const void* T, int single, int b0, int nb)
    {
        if (nb < 0) { b0 = 0; nb = nblocks(h); }
        if (nb == 0) return LBM_OK;
        if (single)
            k_init<D, R, S, float><<<nb, kBlockCells, 0, h->stream>>>(
                h->d_sims, h->d_table + b0, (const float*)rho, (const float*)u, (const float*)T, (S*)h->pop[0],
                (R*)h->W, h->Ntot, h->d_diag + kDiagInitBad);
        else
            k_init<D, R, S, double><<<nb, kBlockCells, 0, h->stream>>>(
                h->d_sims, h->d_table + b0, (const double*)rho, (const double*)u, (const double*)T, (S*)h->pop[0],
                (R*)h->W, h->Ntot, h->d_diag + kDiagInitBad);
        LBM_LAUNCH_CHECK(h, "k_init");
        h->cur = 0;
        h->moments_valid = false;
        return LBM_OK;
    }

    static int split_step(lbm_ctx* h)
    {
        const int nb = nblocks(h);
        S* src = (S*)h->pop[h->cur];
        S* dst = (S*)h->pop[h->cur ^ 1];
        pass_mark(h, 0);
        k_moments<D, R, S><<<nb, kBlockCells, 0, h->stream>>>(h->d_sims, h->d_table, src, (R*)h->W, h->Ntot);
        pass_mark(h, 1);
        k_macro<D, R><<<nb, kBlockCells, 0, h->stream>>>(h->d_sims, h->d_table, (R*)h->W, h->Ntot, h->d_diag);
        if (D == 3 && has_nee(h))
            k_nee<D, R, S><<<(int)h->face_table.size(), kBlockCells, 0, h->stream>>>(h->d_sims, h->d_face_table, src,
                                                                                     (R*)h->W, h->Ntot, 1);
        pass_mark(h, 2);
        k_collide<D, R, S><<<nb, kBlockCells, 0, h->stream>>>(h->d_sims, h->d_table, src, dst, (const R*)h->W, h->Ntot);
        pass_mark(h, 3);
        LBM_LAUNCH_CHECK(h, "split step");
        h->cur ^= 1;
        h->moments_valid = false;
        return LBM_OK;
    }

    static int fused_prepare(lbm_ctx* h)
    {
        // moments of the current state into M (one pull pass), before the first fused step
        fused_moments_launch<D, R, S>(h->d_sims, h->d_table, nblocks(h), (const S*)h->pop[h->cur], (const R*)h->W,
                                      mbuf(h, h->cur), h->Ntot, h->stream);
        LBM_LAUNCH_CHECK(h, "fused moments");
        h->moments_valid = true;
        return LBM_OK;
    }

    static int prepare_part(lbm_ctx* h, int b0, int nb)
    {
        if (nb <= 0) return LBM_OK;
        fused_moments_launch<D, R, S>(h->d_sims, h->d_table + b0, nb, (const S*)h->pop[h->cur], (const R*)h->W,
                                      mbuf(h, h->cur), h->Ntot, h->stream);
        LBM_LAUNCH_CHECK(h, "fused moments");
        return LBM_OK;
    }

    static int fused_step(lbm_ctx* h)
    {
        if (!h->moments_valid) {
            int rc = fused_prepare(h);
            if (rc) return rc;
        }
        pass_mark(h, 0);
        pass_mark(h, 1);
        pass_mark(h, 2);
        cudaError_t e = fused_dispatch(h->storage, D, h->sims[0].eos, uses_mlp(h), all_central(h), h->tx, h->ty, h->tz,
                                       h->d_sims,
                                       h->d_tiles,
                                       (int)h->tiles.size(), h->pop[h->cur], h->pop[h->cur ^ 1], mbuf(h, h->cur),
                                       mbuf(h, h->cur ^ 1), h->Ntot, h->d_diag, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "fused step");
        pass_mark(h, 3);
        h->cur ^= 1;
        return LBM_OK;
    }

    // D2Q9: the row-march one-pass step
    static int ymarch_step(lbm_ctx* h)
    {
        if (!h->moments_valid) {
            int rc = fused_prepare(h);
            if (rc) return rc;
        }
        pass_mark(h, 0);
        pass_mark(h, 1);
        pass_mark(h, 2);
        cudaError_t e = ymarch_dispatch(h->storage, h->sims[0].eos, all_central(h), h->ty, h->d_sims, h->d_tiles,
                                        (int)h->tiles.size(), h->pop[h->cur], h->pop[h->cur ^ 1], mbuf(h, h->cur),
                                        mbuf(h, h->cur ^ 1), h->Ntot, h->d_diag, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "row-march step");
        pass_mark(h, 3);
        h->cur ^= 1;
        return LBM_OK;
    }

    // the z-march's first pass: the macroscopic state of every cell from the carried moments into W
    static int zfirst_pass(lbm_ctx* h, unsigned long long* diag)
    {
        if (uses_mlp(h) && h->storage != LBM_F32) {  // learned start with 16-bit or float64 storage: generic pass
            k_macro<D, R, true><<<nblocks(h), kBlockCells, 0, h->stream>>>(h->d_sims, h->d_table, (R*)h->W, h->Ntot,
                                                                           diag, mbuf(h, h->cur));
            LBM_LAUNCH_CHECK(h, "z-march macroscopic pass");
        } else {
            cudaError_t e = zmacro_dispatch(h->storage, h->sims[0].eos, uses_mlp(h), h->d_sims, h->d_table,
                                            nblocks(h), mbuf(h, h->cur), h->W, h->Ntot, diag, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "z-march macroscopic pass");
        }
        return LBM_OK;
    }

    // rho, u, T of the current state into W for the export: on the z-march paths the
    // carried moments are those of the current state and their first pass forms the
    // fields (no population pass); otherwise the populations' moments (`macro`)
    static int state_fields(lbm_ctx* h)
    {
        if (D == 3 && h->moments_valid && !has_nee(h) &&
            (h->variant == LBM_KERNEL_ZMARCH || h->variant == LBM_KERNEL_ZGATHER)) {
            if (!faces_ready(h)) return fail(h, LBM_E_STATE, "lbm_set_walls / lbm_set_face has not set every face");
            return zfirst_pass(h, nullptr);
        }
        return macro(h);
    }

    static int state_part(lbm_ctx* h, int b0, int nb)
    {
        if (!(D == 3 && h->moments_valid && !has_nee(h) &&
              (h->variant == LBM_KERNEL_ZMARCH || h->variant == LBM_KERNEL_ZGATHER)) ||
            (uses_mlp(h) && h->storage != LBM_F32))
            return LBM_E_UNSUPPORTED;
        if (!faces_ready(h)) return fail(h, LBM_E_STATE, "lbm_set_walls / lbm_set_face has not set every face");
        if (nb == 0) return LBM_OK;
        cudaError_t e = zmacro_dispatch(h->storage, h->sims[0].eos, uses_mlp(h), h->d_sims, h->d_table + b0, nb,
                                        mbuf(h, h->cur), h->W, h->Ntot, nullptr, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "z-march macroscopic pass");
        return LBM_OK;
    }

    // D3Q27: macroscopic pass from the carried moments, then the z-marching collide-stream pass
    static int zmarch_step(lbm_ctx* h)
    {
        if (D != 3) return fail(h, LBM_E_UNSUPPORTED, "the z-march kernel is built for D3Q27");
        if (!h->moments_valid) {
            int rc = fused_prepare(h);
            if (rc) return rc;
        }
        pass_mark(h, 0);
        const int rc = zfirst_pass(h, h->d_diag);
        if (rc) return rc;
        pass_mark(h, 1);
        const bool nee = has_nee(h);
        if (nee) {  // rebuild the boundary cells (slots of their pulls, fields) before the collide-stream pass
            k_nee<D, R, S><<<(int)h->face_table.size(), kBlockCells, 0, h->stream>>>(
                h->d_sims, h->d_face_table, (S*)h->pop[h->cur], (R*)h->W, h->Ntot, 1);
            LBM_LAUNCH_CHECK(h, "boundary cells");
        }
        pass_mark(h, 2);
        cudaError_t e;
        if (h->variant == LBM_KERNEL_ZGATHER)
            e = zgather_dispatch(h->storage, h->sims[0].eos, h->tz, h->d_sims, h->d_tiles, (int)h->tiles.size(),
                                 h->pop[h->cur], h->pop[h->cur ^ 1], h->W, mbuf(h, h->cur ^ 1), h->Ntot, h->stream);
        else
            e = (nee ? zmarch_nee_dispatch : zmarch_dispatch)(
                h->storage, h->sims[0].eos, h->tx, h->ty, h->tz, h->d_sims, h->d_tiles, (int)h->tiles.size(),
                h->pop[h->cur], h->pop[h->cur ^ 1], h->W, mbuf(h, h->cur ^ 1), h->Ntot, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "z-march step");
        pass_mark(h, 3);
        h->cur ^= 1;
        return LBM_OK;
    }

    static int step(lbm_ctx* h, int n)
    {
        if (!faces_ready(h)) return fail(h, LBM_E_STATE, "lbm_set_walls / lbm_set_face has not set every face");
        for (int it = 0; it < n; ++it) {
            int rc = h->variant == LBM_KERNEL_FUSED    ? fused_step(h)
                     : h->variant == LBM_KERNEL_YMARCH ? ymarch_step(h)
                     : (h->variant == LBM_KERNEL_ZMARCH || h->variant == LBM_KERNEL_ZGATHER) ? zmarch_step(h)
                                                                                              : split_step(h);
            if (rc) return rc;
        }
        return LBM_OK;
    }

    // moments and macroscopic fields of the current state into W (no counters)
    static int macro(lbm_ctx* h)
    {
        if (!faces_ready(h)) return fail(h, LBM_E_STATE, "lbm_set_walls / lbm_set_face has not set every face");
        const int nb = nblocks(h);
        k_moments<D, R, S><<<nb, kBlockCells, 0, h->stream>>>(h->d_sims, h->d_table, (const S*)h->pop[h->cur],
                                                              (R*)h->W, h->Ntot);
        k_macro<D, R><<<nb, kBlockCells, 0, h->stream>>>(h->d_sims, h->d_table, (R*)h->W, h->Ntot, nullptr);
        if (D == 3 && has_nee(h))
            k_nee<D, R, S><<<(int)h->face_table.size(), kBlockCells, 0, h->stream>>>(
                h->d_sims, h->d_face_table, (S*)h->pop[h->cur], (R*)h->W, h->Ntot, 0);
        LBM_LAUNCH_CHECK(h, "macro");
        return LBM_OK;
    }

    static int export_moments(lbm_ctx* h, void* rho, void* u, void* T, int single, int b0, int nb)
    {
        if (nb < 0) { b0 = 0; nb = nblocks(h); }
        if (nb == 0) return LBM_OK;
        if (single)
            k_export_moments<D, R, float><<<nb, kBlockCells, 0, h->stream>>>(
                h->d_sims, h->d_table + b0, (const R*)h->W, h->Ntot, (float*)rho, (float*)u, (float*)T);
        else
            k_export_moments<D, R, double><<<nb, kBlockCells, 0, h->stream>>>(
                h->d_sims, h->d_table + b0, (const R*)h->W, h->Ntot, (double*)rho, (double*)u, (double*)T);
        LBM_LAUNCH_CHECK(h, "export moments");
        return LBM_OK;
    }

    static int export_pops(lbm_ctx* h, double* f, double* g)
    {
        k_export_pops<D, R, S><<<nblocks(h), kBlockCells, 0, h->stream>>>(h->d_sims, h->d_table,
                                                                          (const S*)h->pop[h->cur], f, g);
        LBM_LAUNCH_CHECK(h, "export populations");
        return LBM_OK;
    }

    static int invariants(lbm_ctx* h, double* d_out)
    {
        const int nv = 2 * D + 3;
        k_invariants<D, R><<<nblocks(h), kBlockCells, 0, h->stream>>>(h->d_sims, h->d_table, (const R*)h->W, h->Ntot,
                                                                      h->d_partials);
        int nt = h->nsim * nv;
        k_invariants_final<<<(nt + 127) / 128, 128, 0, h->stream>>>(h->d_partials, h->d_sim_block_start, h->nsim, nv,
                                                                    d_out);
        LBM_LAUNCH_CHECK(h, "invariants");
        return LBM_OK;
    }

    // every simulation takes the central derivative in Phi (narrower halos)
    static int all_central(lbm_ctx* h)
    {
        for (const SimDev& d : h->sims)
            if (!d.phi_central) return 0;
        return 1;
    }

    static int uses_mlp(lbm_ctx* h)
    {
        for (const SimDev& d : h->sims)
            if (d.eos == EOS_PR && d.t_solver == LBM_T_MLP && d.mlp != nullptr) return 1;
        return 0;
    }

    static int fused_ok(lbm_ctx* h, int tx, int ty, int tz)
    {
        if (split_only(h) || !offsets32(h, Lat<D>::Q)) return 0;  // extrapolated faces, duct friction, size: split kernels
        for (const SimDev& d : h->sims)
            if (d.eos != h->sims[0].eos) return 0;  // one equation of state per fused launch
        if (uses_mlp(h) && h->storage != LBM_F32) return 0;  // learned start built for float32 storage
        return fused_shape(h->storage, D, tx, ty, tz) ? 1 : 0;
    }

    static Ops ops()
    {
        return Ops{init,     step,     macro,         export_moments, export_pops, invariants,
                   fused_ok, fused_prepare, prepare_part, state_fields,   state_part};
    }
};

cudaError_t fused_dispatch(int storage, int dim, int eos, int mlp, int pc, int tx, int ty, int tz, const SimDev* sims,
                           const TileEntry* tiles, int ntiles, const void* src, void* dst, const void* Min, void* Mout,
                           long long Ntot, unsigned long long* diag, cudaStream_t stream)
{
    switch (storage) {
    case LBM_F64: return fused_dispatch_f64(dim, eos, mlp, pc, tx, ty, tz, sims, tiles, ntiles, src, dst, Min, Mout, Ntot, diag, stream);
    case LBM_F32: return fused_dispatch_f32(dim, eos, mlp, pc, tx, ty, tz, sims, tiles, ntiles, src, dst, Min, Mout, Ntot, diag, stream);
    case LBM_BF16: return fused_dispatch_bf16(dim, eos, mlp, pc, tx, ty, tz, sims, tiles, ntiles, src, dst, Min, Mout, Ntot, diag, stream);
    case LBM_F16: return fused_dispatch_f16(dim, eos, mlp, pc, tx, ty, tz, sims, tiles, ntiles, src, dst, Min, Mout, Ntot, diag, stream);
    }
    return cudaErrorInvalidValue;
}

bool fused_shape(int storage, int dim, int tx, int ty, int tz)
{
    switch (storage) {
    case LBM_F64: return fused_shape_f64(dim, tx, ty, tz);
    case LBM_F32: return fused_shape_f32(dim, tx, ty, tz);
    case LBM_BF16: return fused_shape_bf16(dim, tx, ty, tz);
    case LBM_F16: return fused_shape_f16(dim, tx, ty, tz);
    }
    return false;
}

cudaError_t zmarch_dispatch(int storage, int eos, int tx, int ty, int zl, const SimDev* sims, const TileEntry* tiles,
                            int ntiles, const void* src, void* dst, const void* W, void* Mout, long long Ntot,
                            cudaStream_t stream)
{
    switch (storage) {
    case LBM_F64: return zmarch_dispatch_f64(eos, tx, ty, zl, sims, tiles, ntiles, src, dst, W, Mout, Ntot, stream);
    case LBM_F32: return zmarch_dispatch_f32(eos, tx, ty, zl, sims, tiles, ntiles, src, dst, W, Mout, Ntot, stream);
    case LBM_BF16: return zmarch_dispatch_bf16(eos, tx, ty, zl, sims, tiles, ntiles, src, dst, W, Mout, Ntot, stream);
    case LBM_F16: return zmarch_dispatch_f16(eos, tx, ty, zl, sims, tiles, ntiles, src, dst, W, Mout, Ntot, stream);
    }
    return cudaErrorInvalidValue;
}

cudaError_t zmacro_dispatch(int storage, int eos, int mlp, const SimDev* sims, const BlockEntry* table, int nblocks,
                            const void* M, void* W, long long Ntot, unsigned long long* diag, cudaStream_t stream)
{
    switch (storage) {
    case LBM_F64: return zmacro_dispatch_f64(eos, mlp, sims, table, nblocks, M, W, Ntot, diag, stream);
    case LBM_F32: return zmacro_dispatch_f32(eos, mlp, sims, table, nblocks, M, W, Ntot, diag, stream);
    case LBM_BF16: return zmacro_dispatch_bf16(eos, mlp, sims, table, nblocks, M, W, Ntot, diag, stream);
    case LBM_F16: return zmacro_dispatch_f16(eos, mlp, sims, table, nblocks, M, W, Ntot, diag, stream);
    }
    return cudaErrorInvalidValue;
}

cudaError_t zmarch_nee_dispatch(int storage, int eos, int tx, int ty, int zl, const SimDev* sims,
                                const TileEntry* tiles, int ntiles, const void* src, void* dst, const void* W,
                                void* Mout, long long Ntot, cudaStream_t stream)
{
    switch (storage) {
    case LBM_F64: return zmarch_nee_dispatch_f64(eos, tx, ty, zl, sims, tiles, ntiles, src, dst, W, Mout, Ntot, stream);
    case LBM_F32: return zmarch_nee_dispatch_f32(eos, tx, ty, zl, sims, tiles, ntiles, src, dst, W, Mout, Ntot, stream);
    }
    return cudaErrorInvalidValue;
}

cudaError_t ymarch_dispatch(int storage, int eos, int pc, int yl, const SimDev* sims, const TileEntry* tiles,
                            int ntiles, const void* src, void* dst, const void* Min, void* Mout, long long Ntot,
                            unsigned long long* diag, cudaStream_t stream)
{
    switch (storage) {
    case LBM_F32: return ymarch_dispatch_f32(eos, pc, yl, sims, tiles, ntiles, src, dst, Min, Mout, Ntot, diag, stream);
    case LBM_BF16: return ymarch_dispatch_bf16(eos, pc, yl, sims, tiles, ntiles, src, dst, Min, Mout, Ntot, diag, stream);
    case LBM_F16: return ymarch_dispatch_f16(eos, pc, yl, sims, tiles, ntiles, src, dst, Min, Mout, Ntot, diag, stream);
    }
    return cudaErrorInvalidValue;
}

cudaError_t ymarch_slots(int storage, int eos, int pc, int* slots)
{
    switch (storage) {
    case LBM_F32: return ymarch_slots_f32(eos, pc, slots);
    case LBM_BF16: return ymarch_slots_bf16(eos, pc, slots);
    case LBM_F16: return ymarch_slots_f16(eos, pc, slots);
    }
    return cudaErrorInvalidValue;
}

// Rows per range of the row march.  A range of YL rows takes YL + 2 RM + 8
// steps (the pipeline fills and drains over the rim and stencil rows; RM = 1
// for the central Phi, 2 upwind-biased).  The tile table lists the ranges
// longest first and the resident CTAs take them round-robin, one per CTA per
// round, so the first CTA carries the longest range of every round and the
// step lasts the sum of those.  The row count YL = ceil(ny / n) that
// minimises this sum is taken, no shorter than 32 rows and with at most 16
// rounds (shorter ranges re-read their halo rows for a growing share of the
// bytes and add fill steps); ties go to the longer ranges.
int ymarch_rows(const lbm_ctx* h)
{
    const int strip = ymarch_strip_width(h);
    const int pc = strip == kYmStripCentral;
    int slots = 0;
    if (ymarch_slots(h->storage, h->sims[0].eos, pc, &slots) != cudaSuccess || slots < 1) return 64;
    const int ovh = pc ? 10 : 12;
    int ny_max = 1;
    for (const SimDev& d : h->sims) ny_max = d.ny > ny_max ? d.ny : ny_max;
    long long best = -1;
    int pick = 64, prev = 0;
    std::vector<int> cost;
    for (int n = 1; n <= ny_max; ++n) {
        const int yl = (ny_max + n - 1) / n;
        if (n > 1 && yl < 32) break;
        if (yl == prev) continue;  // the same row count as fewer ranges
        prev = yl;
        cost.clear();
        for (const SimDev& d : h->sims) {
            const int nstrip = (d.nx + strip - 1) / strip;
            for (int y0 = 0; y0 < d.ny; y0 += yl) cost.insert(cost.end(), nstrip, std::min(yl, d.ny - y0) + ovh);
        }
        if (n > 1 && cost.size() > (size_t)16 * slots) break;
        std::sort(cost.begin(), cost.end(), [](int a, int b) { return a > b; });
        const size_t G = std::min(cost.size(), (size_t)slots);
        long long t = 0;
        for (size_t k = 0; k < cost.size(); k += G) t += cost[k];
        if (best < 0 || t < best) { best = t; pick = yl; }
    }
    return pick;
}

cudaError_t zgather_dispatch(int storage, int eos, int zl, const SimDev* sims, const TileEntry* tiles, int ntiles,
                             const void* src, void* dst, const void* W, void* Mout, long long Ntot,
                             cudaStream_t stream)
{
    switch (storage) {
    case LBM_F32: return zgather_dispatch_f32(eos, zl, sims, tiles, ntiles, src, dst, W, Mout, Ntot, stream);
    case LBM_BF16: return zgather_dispatch_bf16(eos, zl, sims, tiles, ntiles, src, dst, W, Mout, Ntot, stream);
    case LBM_F16: return zgather_dispatch_f16(eos, zl, sims, tiles, ntiles, src, dst, W, Mout, Ntot, stream);
    }
    return cudaErrorInvalidValue;
}

bool zmarch_shape(int storage, int tx, int ty)
{
    switch (storage) {
    case LBM_F64: return zmarch_shape_f64(tx, ty);
    case LBM_F32: return zmarch_shape_f32(tx, ty);
    case LBM_BF16: return zmarch_shape_bf16(tx, ty);
    case LBM_F16: return zmarch_shape_f16(tx, ty);
    }
    return false;
}

// default tile of the fused kernel per lattice and storage
void fused_default_tile(int dim, int storage, int& tx, int& ty, int& tz)
{
    if (dim == 2) {
        tx = 32;
        ty = storage == LBM_F64 ? 8 : 16;
        tz = 1;
    } else {
        tx = 8;
        ty = 8;
        tz = 4;
    }
}

bool pick_ops(int dim, int storage, Ops& ops, size_t& rbytes, size_t& sbytes)
{
#define LBM_PICK(D, R, S)              \
    do {                               \
        ops = Impl<D, R, S>::ops();    \
        rbytes = sizeof(R);            \
        sbytes = sizeof(S);            \
        return true;                   \
    } while (0)
    if (dim == 2) {
        if (storage == LBM_F64) LBM_PICK(2, double, double);
        if (storage == LBM_F32) LBM_PICK(2, float, float);
        if (storage == LBM_BF16) LBM_PICK(2, float, __nv_bfloat16);
        if (storage == LBM_F16) LBM_PICK(2, float, __half);
    } else if (dim == 3) {
        if (storage == LBM_F64) LBM_PICK(3, double, double);
        if (storage == LBM_F32) LBM_PICK(3, float, float);
        if (storage == LBM_BF16) LBM_PICK(3, float, __nv_bfloat16);
        if (storage == LBM_F16) LBM_PICK(3, float, __half);
    }
#undef LBM_PICK
    return false;
}

int check_lattice(const lbm_lattice* L, std::string& why)
{
    if (!L) { why = "lattice is NULL"; return LBM_E_INVALID; }
    if (L->dim != 2 && L->dim != 3) { why = "dim must be 2 or 3"; return LBM_E_INVALID; }
    if (L->nx < 1 || L->ny < 1 || L->nz < 1) { why = "nx, ny, nz must be >= 1"; return LBM_E_INVALID; }
    if (L->dim == 2 && (L->nz != 1 || L->zwalls)) { why = "2-D lattices need nz = 1 and no z walls"; return LBM_E_INVALID; }
    if ((long long)L->nx * L->ny * L->nz * (L->dim == 2 ? 9 : 27) > 0xFFFFFFFFLL) {
        why = "too many cells: Q * cells must stay below 2^32 per simulation";
        return LBM_E_INVALID;
    }
    if (L->zwalls < 0 || L->zwalls > 2) { why = "zwalls must be 0, 1 or 2"; return LBM_E_INVALID; }
    if (L->zwalls == 2 && L->nz < 4) { why = "non-equilibrium-extrapolation walls need nz >= 4"; return LBM_E_INVALID; }
    if (L->storage < LBM_F64 || L->storage > LBM_F16) { why = "unknown storage"; return LBM_E_INVALID; }
    if (L->phi_scheme != LBM_PHI_UPWIND && L->phi_scheme != LBM_PHI_CENTRAL) { why = "unknown phi_scheme"; return LBM_E_INVALID; }
    return LBM_OK;
}

int fill_sim(SimDev& s, const lbm_lattice* L, const lbm_eos* E, double tau_f, double tau_g, const lbm_force* F,
             const lbm_heat* H, std::string& why)
{
    std::memset(&s, 0, sizeof(s));
    if (!E) { why = "eos is NULL"; return LBM_E_INVALID; }
    if (E->kind < LBM_IDEAL || E->kind > LBM_PR) { why = "unknown eos kind"; return LBM_E_INVALID; }
    if (!(E->R > 0) || !(E->cv > 0)) { why = "R and cv must be > 0"; return LBM_E_INVALID; }
    if (!(tau_f > 0) || !(tau_g > 0)) { why = "tau_f and tau_g must be > 0"; return LBM_E_INVALID; }
    if (E->t_solver != LBM_T_NEWTON && E->t_solver != LBM_T_MLP) { why = "unknown t_solver"; return LBM_E_INVALID; }
    if (!(E->mu >= 0) || !std::isfinite(E->mu)) { why = "mu must be finite and >= 0"; return LBM_E_INVALID; }
    if (E->isothermal != 0 && E->isothermal != 1) { why = "isothermal must be 0 or 1"; return LBM_E_INVALID; }
    if (E->isothermal && E->t_solver == LBM_T_MLP) { why = "isothermal runs invert no temperature"; return LBM_E_INVALID; }
    if (E->isothermal && H && H->q != 0.0) { why = "isothermal runs take no heat source"; return LBM_E_INVALID; }
    if (E->isothermal && L->zwalls == 2) { why = "non-equilibrium-extrapolation walls set a temperature: not isothermal"; return LBM_E_INVALID; }
    if (F && (!(F->friction >= 0) || !std::isfinite(F->friction))) { why = "friction must be finite and >= 0"; return LBM_E_INVALID; }
    if (F && F->friction > 0 && E->isothermal) { why = "friction heat needs the energy equation: not isothermal"; return LBM_E_INVALID; }
    if (F && (!(F->throttle_K >= 0) || !std::isfinite(F->throttle_K))) { why = "throttle_K must be finite and >= 0"; return LBM_E_INVALID; }
    if (F && F->throttle_K > 0 && (L->dim != 3 || !(F->throttle_sigma > 0) || !std::isfinite(F->throttle_sigma) || E->isothermal)) {
        why = "a throttle needs dim 3, throttle_sigma > 0 and the energy equation";
        return LBM_E_INVALID;
    }
    s.nx = L->nx; s.ny = L->ny; s.nz = L->nz; s.zwalls = L->zwalls;
    s.N = (long long)L->nx * L->ny * L->nz;
    s.eos = E->kind;
    s.phi_central = L->phi_scheme == LBM_PHI_CENTRAL;
    s.t_solver = E->t_solver;
    s.R = E->R; s.cv = E->cv; s.a = E->a; s.b = E->b; s.Tc = E->Tc;
    if (E->kind == LBM_PR) {
        if (!(E->Tc > 0)) { why = "Peng-Robinson needs Tc > 0"; return LBM_E_INVALID; }
        if (E->a == 0.0) {
            if (!(E->Pc > 0)) { why = "Peng-Robinson needs a, b or Pc > 0"; return LBM_E_INVALID; }
            s.a = 0.45724 * E->R * E->R * E->Tc * E->Tc / E->Pc;
            s.b = 0.07780 * E->R * E->Tc / E->Pc;
        }
        s.kw = 0.37464 + 1.54226 * E->omega - 0.26992 * E->omega * E->omega;
        if (!(s.b > 0)) { why = "Peng-Robinson needs b > 0"; return LBM_E_INVALID; }
    }
    if (E->kind == LBM_VDW && (E->a < 0 || E->b < 0)) { why = "van der Waals needs a, b >= 0"; return LBM_E_INVALID; }
    s.kappa = E->kappa; s.eta_mu = E->eta_over_mu; s.k_mu = E->k_over_mu;
    s.mu = E->mu;
    s.iso = E->isothermal;
    s.beta_f = 1.0 / (2.0 * tau_f + 1.0);
    s.beta_g = 1.0 / (2.0 * tau_g + 1.0);
    if (F) { s.acc[0] = F->accel[0]; s.acc[1] = F->accel[1]; s.acc[2] = L->dim == 3 ? F->accel[2] : 0.0; }
    if (F) { s.friction = F->friction; s.throttle_K = F->throttle_K; s.throttle_sigma = F->throttle_sigma; }
    if (F) s.ffield = F->field;
    if (H) s.qfield = H->field;
    if (s.qfield && E->isothermal) { why = "a heat field needs the energy equation: not isothermal"; return LBM_E_INVALID; }
    s.inv_cv = 1.0 / s.cv;
    s.inv_Tc = s.Tc > 0 ? 1.0 / s.Tc : 0.0;
    s.lam_c = s.b > 0 ? 1.0 / (2.0 * std::sqrt(2.0) * s.b) : 0.0;
    s.athe_c = (double)(L->dim + 2) / (double)L->dim - s.eta_mu;
    if (H) { s.q = H->q; s.zlo = H->zmask_lo; s.zhi = H->zmask_hi; }
    return LBM_OK;
}

void drop_graph(lbm_ctx* h)
{
    for (int p = 0; p < 2; ++p) {
        if (h->graph_exec[p]) cudaGraphExecDestroy(h->graph_exec[p]);
        h->graph_exec[p] = nullptr;
    }
}

void free_all(lbm_ctx* h)
{
    drop_graph(h);
    for (cudaEvent_t ev : h->pass_ev) cudaEventDestroy(ev);
    h->pass_ev.clear();
    for (cudaEvent_t ev : h->xfer_ev) cudaEventDestroy(ev);
    h->xfer_ev.clear();
    if (h->xfer) cudaStreamDestroy(h->xfer);
    h->xfer = nullptr;
    void* ptrs[] = {h->d_sims, h->d_table, h->d_sim_block_start, h->d_tiles, h->pop[0], h->pop[1],
                    h->W, h->M, h->d_diag, h->d_partials, h->d_mlp, h->d_face_table};
    for (void* p : ptrs) lbm_glue_free(p);
    h->d_face_table = nullptr;
    h->d_sims = nullptr; h->d_table = nullptr; h->d_sim_block_start = nullptr; h->d_tiles = nullptr;
    h->pop[0] = h->pop[1] = nullptr; h->W = nullptr; h->M = nullptr; h->d_diag = nullptr; h->d_partials = nullptr;
    h->d_mlp = nullptr;
}

int upload_sims(lbm_ctx* h)
{
    LBM_CUDA_CHECK(h, cudaMemcpyAsync(h->d_sims, h->sims.data(), h->sims.size() * sizeof(SimDev),
                                      cudaMemcpyHostToDevice, h->stream));
    LBM_CUDA_CHECK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

// rows_first: the row march's order, ranges with the most rows first (its
// tiles are independent within a step, so only the schedule changes)
int build_tiles(lbm_ctx* h, int tx, int ty, int tz, bool rows_first = false)
{
    h->tiles.clear();
    for (int s = 0; s < h->nsim; ++s) {
        const SimDev& d = h->sims[s];
        int zt = h->dim == 3 ? tz : 1;
        for (int z0 = 0; z0 < d.nz; z0 += zt)
            for (int y0 = 0; y0 < d.ny; y0 += ty)
                for (int x0 = 0; x0 < d.nx; x0 += tx) h->tiles.push_back(TileEntry{s, x0, y0, z0});
    }
    if (rows_first) {
        auto rows = [&](const TileEntry& t) { return std::min(ty, h->sims[t.sim].ny - t.y0); };
        std::stable_sort(h->tiles.begin(), h->tiles.end(),
                         [&](const TileEntry& a, const TileEntry& b) { return rows(a) > rows(b); });
    }
    lbm_glue_free(h->d_tiles);
    h->d_tiles = (TileEntry*)dev_alloc(h, h->tiles.size() * sizeof(TileEntry));
    if (!h->d_tiles) return fail(h, LBM_E_NOMEM, "tile table allocation failed");
    LBM_CUDA_CHECK(h, cudaMemcpyAsync(h->d_tiles, h->tiles.data(), h->tiles.size() * sizeof(TileEntry),
                                      cudaMemcpyHostToDevice, h->stream));
    LBM_CUDA_CHECK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int create_impl(int nsim, const lbm_lattice* L, const lbm_eos* E, const double* tau_f, const double* tau_g,
                const lbm_force* F, const lbm_heat* H, lbm_handle* out)
{
    if (!out) return fail(nullptr, LBM_E_INVALID, "out is NULL");
    *out = nullptr;
    if (nsim < 1) return fail(nullptr, LBM_E_INVALID, "nsim must be >= 1");
    if (!L || !E || !tau_f || !tau_g) return fail(nullptr, LBM_E_INVALID, "NULL argument");
    std::string why;
    for (int s = 0; s < nsim; ++s) {
        int rc = check_lattice(&L[s], why);
        if (rc) return fail(nullptr, rc, "simulation " + std::to_string(s) + ": " + why);
        if (L[s].dim != L[0].dim || L[s].storage != L[0].storage)
            return fail(nullptr, LBM_E_INVALID, "all simulations of a batch must share dim and storage");
    }
    lbm_ctx* h = new lbm_ctx();
    h->nsim = nsim;
    h->dim = L[0].dim;
    h->Q = h->dim == 2 ? 9 : 27;
    h->storage = L[0].storage;
    if (!pick_ops(h->dim, h->storage, h->ops, h->rbytes, h->sbytes)) {
        delete h;
        return fail(nullptr, LBM_E_UNSUPPORTED, "lattice/storage combination not built");
    }
    h->sims.resize(nsim);
    long long cells = 0, pops = 0;
    for (int s = 0; s < nsim; ++s) {
        int rc = fill_sim(h->sims[s], &L[s], &E[s], tau_f[s], tau_g[s], F ? &F[s] : nullptr, H ? &H[s] : nullptr, why);
        if (rc) {
            delete h;
            return fail(nullptr, rc, "simulation " + std::to_string(s) + ": " + why);
        }
        h->sims[s].cell_off = cells;
        h->sims[s].pop_off = pops;
        cells += h->sims[s].N;
        pops += 2LL * h->Q * h->sims[s].N;
    }
    h->Ntot = cells;
    h->pop_elems = pops;
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) {
        delete h;
        return fail(nullptr, LBM_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(ce));
    }
    h->device = dev;
    h->stream = (cudaStream_t)lbm_glue_current_stream(dev);

    // block table of the per-cell kernels
    for (int s = 0; s < nsim; ++s) {
        h->sim_block_start.push_back((int)h->table.size());
        for (long long k = 0; k < h->sims[s].N; k += kBlockCells) h->table.push_back(BlockEntry{s, (int)k});
    }
    h->sim_block_start.push_back((int)h->table.size());
    // the boundary cells of extrapolated faces: the layers z = 0 and z = nz - 1 of each such simulation
    for (int s = 0; s < nsim; ++s) {
        if (h->sims[s].zwalls != 2) continue;
        const long long faces = 2LL * h->sims[s].nx * h->sims[s].ny;
        for (long long k = 0; k < faces; k += kBlockCells) h->face_table.push_back(BlockEntry{s, (int)k});
    }
    const int nv = 2 * h->dim + 3;

    h->d_sims = (SimDev*)dev_alloc(h, nsim * sizeof(SimDev));
    h->d_table = (BlockEntry*)dev_alloc(h, h->table.size() * sizeof(BlockEntry));
    h->d_sim_block_start = (int*)dev_alloc(h, h->sim_block_start.size() * sizeof(int));
    h->pop[0] = dev_alloc(h, (size_t)pops * h->sbytes);
    h->pop[1] = dev_alloc(h, (size_t)pops * h->sbytes);
    h->W = dev_alloc(h, (size_t)W_NF * cells * h->rbytes);
    h->M = dev_alloc(h, (size_t)2 * M_NF * cells * h->rbytes);
    h->d_diag = (unsigned long long*)dev_alloc(h, kDiagSlots * sizeof(unsigned long long));
    h->d_partials = (double*)dev_alloc(h, h->table.size() * nv * sizeof(double));
    if (!h->face_table.empty()) h->d_face_table = (BlockEntry*)dev_alloc(h, h->face_table.size() * sizeof(BlockEntry));
    if (!h->d_sims || !h->d_table || !h->d_sim_block_start || !h->pop[0] || !h->pop[1] || !h->W || !h->M ||
        !h->d_diag || !h->d_partials || (!h->face_table.empty() && !h->d_face_table)) {
        free_all(h);
        delete h;
        return fail(nullptr, LBM_E_NOMEM,
                    "device allocation failed (torch.cuda must be initialised; populations need " +
                        std::to_string(2.0 * (double)pops * (double)h->sbytes * 1e-9) + " GB)");
    }
    int rc = LBM_OK;
    auto chk = [&](cudaError_t e, const char* w) {
        if (e != cudaSuccess && rc == LBM_OK) rc = cuda_fail(h, e, w);
    };
    chk(cudaMemcpyAsync(h->d_table, h->table.data(), h->table.size() * sizeof(BlockEntry), cudaMemcpyHostToDevice,
                        h->stream), "table upload");
    chk(cudaMemcpyAsync(h->d_sim_block_start, h->sim_block_start.data(), h->sim_block_start.size() * sizeof(int),
                        cudaMemcpyHostToDevice, h->stream), "table upload");
    if (!h->face_table.empty())
        chk(cudaMemcpyAsync(h->d_face_table, h->face_table.data(), h->face_table.size() * sizeof(BlockEntry),
                            cudaMemcpyHostToDevice, h->stream), "face table upload");
    chk(cudaMemsetAsync(h->d_diag, 0, kDiagSlots * sizeof(unsigned long long), h->stream), "diag reset");
    chk(cudaMemsetAsync(h->W, 0, (size_t)W_NF * cells * h->rbytes, h->stream), "work reset");
    if (rc == LBM_OK) rc = upload_sims(h);
    if (rc == LBM_OK) {
        // default kernel: the fused one-pass step with its default tile when it runs this lattice
        int dtx, dty, dtz;
        fused_default_tile(h->dim, h->storage, dtx, dty, dtz);
        bool same_eos = true;
        for (const SimDev& d : h->sims) same_eos = same_eos && d.eos == h->sims[0].eos;
        if (zgather_ok(h)) {
            h->variant = LBM_KERNEL_ZGATHER;
            h->tx = 30; h->ty = 14; h->tz = 32;
            rc = build_tiles(h, 30, 14, 32);
        } else if (ymarch_ok(h) && cells >= (1LL << 22)) {
            // large 2-D lattices: the row march, ranges sized to the resident CTAs
            h->variant = LBM_KERNEL_YMARCH;
            h->tx = ymarch_strip_width(h); h->ty = ymarch_rows(h); h->tz = 1;
            rc = build_tiles(h, h->tx, h->ty, 1, true);
        } else if (h->dim == 3 && same_eos && zmarch_ok(h, 30, 14)) {
            h->variant = LBM_KERNEL_ZMARCH;
            h->tx = 30; h->ty = 14; h->tz = 32;
            rc = build_tiles(h, 30, 14, 32);
        } else if (h->ops.fused_ok(h, dtx, dty, dtz)) {
            h->variant = LBM_KERNEL_FUSED;
            h->tx = dtx; h->ty = dty; h->tz = dtz;
            rc = build_tiles(h, dtx, dty, dtz);
        } else {
            h->variant = LBM_KERNEL_SPLIT;
        }
    }
    if (rc != LBM_OK) {
        g_create_error = h->err;
        free_all(h);
        delete h;
        return rc;
    }
    *out = h;
    return LBM_OK;
}

}  // namespace

// message of a failing call that has no handle (lbm_create*, lbm_step_static)
void lbm_set_global_error(const std::string& msg) { g_create_error = msg; }

// the lattice and constant checks of lbm_create, for entry points without a handle
int lbm_check_and_fill_sim(SimDev& s, const lbm_lattice* L, const lbm_eos* E, double tau_f, double tau_g,
                           const lbm_force* F, const lbm_heat* H, std::string& why)
{
    int rc = check_lattice(L, why);
    if (rc) return rc;
    return fill_sim(s, L, E, tau_f, tau_g, F, H, why);
}

extern "C" {

int lbm_create(const lbm_lattice* lattice, const lbm_eos* eos, double tau_f, double tau_g, const lbm_force* force,
               const lbm_heat* heat, lbm_handle* out)
{
    return create_impl(1, lattice, eos, &tau_f, &tau_g, force, heat, out);
}

int lbm_create_batch(int nsim, const lbm_lattice* lattices, const lbm_eos* eos, const double* tau_f,
                     const double* tau_g, const lbm_force* force, const lbm_heat* heat, lbm_handle* out)
{
    return create_impl(nsim, lattices, eos, tau_f, tau_g, force, heat, out);
}

void lbm_destroy(lbm_handle h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

int lbm_set_stream(lbm_handle h, void* stream)
{
    if (!h) return fail(nullptr, LBM_E_INVALID, "handle is NULL");
    LBM_CUDA_CHECK(h, cudaStreamSynchronize(h->stream));
    drop_graph(h);
    h->graph_steps = 0;
    h->stream = (cudaStream_t)stream;
    return LBM_OK;
}

int lbm_set_force(lbm_handle h, const double* accel)
{
    if (!h) return fail(nullptr, LBM_E_INVALID, "handle is NULL");
    if (!accel) return fail(h, LBM_E_INVALID, "accel is NULL");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(accel[a])) return fail(h, LBM_E_INVALID, "accel must be finite");
    for (SimDev& d : h->sims) {
        d.acc[0] = accel[0];
        d.acc[1] = accel[1];
        d.acc[2] = h->dim == 3 ? accel[2] : 0.0;
    }
    // every kernel reads the constants from d_sims at run time (graphs included);
    // the host copy stays alive, so the stream-ordered copy needs no staging
    LBM_CUDA_CHECK(h, cudaMemcpyAsync(h->d_sims, h->sims.data(), h->sims.size() * sizeof(SimDev),
                                      cudaMemcpyHostToDevice, h->stream));
    return LBM_OK;
}

int lbm_set_walls(lbm_handle h, const double* u_lo, double T_lo, const double* u_hi, double T_hi, int wall_rho)
{
    if (!h) return fail(nullptr, LBM_E_INVALID, "handle is NULL");
    if (!u_lo || !u_hi) return fail(h, LBM_E_INVALID, "wall velocities are NULL");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(u_lo[a]) || !std::isfinite(u_hi[a])) return fail(h, LBM_E_INVALID, "wall velocities must be finite");
    if (!(T_lo > 0) || !(T_hi > 0) || !std::isfinite(T_lo) || !std::isfinite(T_hi))
        return fail(h, LBM_E_INVALID, "wall temperatures must be finite and > 0");
    if (wall_rho < 0 || wall_rho > 2) return fail(h, LBM_E_INVALID, "wall_rho must be 0, 1 or 2");
    if (!has_nee(h)) return fail(h, LBM_E_STATE, "no simulation of the handle has non-equilibrium-extrapolation walls");
    for (SimDev& d : h->sims) {
        if (d.zwalls != 2) continue;
        for (int a = 0; a < 3; ++a) { d.uw[0][a] = u_lo[a]; d.uw[1][a] = u_hi[a]; }
        d.Tw[0] = T_lo;
        d.Tw[1] = T_hi;
        d.wall_rho = wall_rho;
        d.face_kind[0] = d.face_kind[1] = 0;
        d.face_set[0] = d.face_set[1] = 1;
    }
    LBM_CUDA_CHECK(h, cudaMemcpyAsync(h->d_sims, h->sims.data(), h->sims.size() * sizeof(SimDev),
                                      cudaMemcpyHostToDevice, h->stream));
    return LBM_OK;
}

int lbm_set_face(lbm_handle h, int face, int kind, const double* u, double T, double P)
{
    if (!h) return fail(nullptr, LBM_E_INVALID, "handle is NULL");
    if (face != 0 && face != 1) return fail(h, LBM_E_INVALID, "face must be 0 (z = 0) or 1 (z = nz - 1)");
    if (kind < LBM_FACE_INLET_TOTAL || kind > LBM_FACE_INLET_PT) return fail(h, LBM_E_INVALID, "unknown face kind");
    const bool inlet = kind == LBM_FACE_INLET_TOTAL || kind == LBM_FACE_INLET_STATIC || kind == LBM_FACE_INLET_PT;
    if (kind == LBM_FACE_INLET_STATIC) {
        if (!u) return fail(h, LBM_E_INVALID, "a static inlet needs its velocity");
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(u[a])) return fail(h, LBM_E_INVALID, "velocity must be finite");
    }
    if (inlet && (!(T > 0) || !std::isfinite(T))) return fail(h, LBM_E_INVALID, "inlet temperature must be finite and > 0");
    if (kind != LBM_FACE_OUTLET_EXTRAP && (!(P > 0) || !std::isfinite(P)))
        return fail(h, LBM_E_INVALID, "face pressure must be finite and > 0");
    if (!has_nee(h)) return fail(h, LBM_E_STATE, "no simulation of the handle has non-equilibrium-extrapolation walls");
    for (const SimDev& d : h->sims)
        if (d.zwalls == 2 && kind == LBM_FACE_INLET_TOTAL && d.eos != EOS_IDEAL)
            return fail(h, LBM_E_UNSUPPORTED, "a total-state inlet needs the ideal gas");
    for (SimDev& d : h->sims) {
        if (d.zwalls != 2) continue;
        for (int a = 0; a < 3; ++a) d.uw[face][a] = (kind == LBM_FACE_INLET_STATIC) ? u[a] : 0.0;
        if (h->dim == 2) d.uw[face][2] = 0.0;
        d.Tw[face] = inlet ? T : 1.0;
        d.face_P[face] = P;
        d.face_kind[face] = kind;
        d.face_set[face] = 1;
    }
    LBM_CUDA_CHECK(h, cudaMemcpyAsync(h->d_sims, h->sims.data(), h->sims.size() * sizeof(SimDev),
                                      cudaMemcpyHostToDevice, h->stream));
    return LBM_OK;
}

extern "C++" {
// Host-field transfers in parts: the block table is cut into up to kXferParts
// runs of blocks, part c's cells cross the host link on h->xfer while the
// kernels work on part c - 1 (or part c's copy waits for its kernels, on the
// way out).  Lattices under 2 M cells go in one part.
constexpr int kXferParts = 8;

int xfer_parts(const lbm_ctx* h)
{
    const long long p = h->Ntot >> 20;
    const int nb = (int)h->table.size();
    int n = p < 2 ? 1 : (p > kXferParts ? kXferParts : (int)p);
    return n > nb ? (nb > 0 ? nb : 1) : n;
}

// the copy stream and n + 1 events (created once per handle)
int xfer_setup(lbm_ctx* h, int n)
{
    if (!h->xfer) LBM_CUDA_CHECK(h, cudaStreamCreateWithFlags(&h->xfer, cudaStreamNonBlocking));
    while ((int)h->xfer_ev.size() < n + 1) {
        cudaEvent_t ev = nullptr;
        LBM_CUDA_CHECK(h, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        h->xfer_ev.push_back(ev);
    }
    return LBM_OK;
}

// blocks and cells of part c of n: blocks [b0, b1), global cells [lo, hi)
void xfer_part(const lbm_ctx* h, int c, int n, int& b0, int& b1, long long& lo, long long& hi)
{
    const long long nb = (long long)h->table.size();
    b0 = (int)(nb * c / n);
    b1 = (int)(nb * (c + 1) / n);
    lo = hi = 0;
    if (b1 <= b0) return;
    const BlockEntry& f = h->table[b0];
    const BlockEntry& l = h->table[b1 - 1];
    const SimDev& sl = h->sims[l.sim];
    lo = h->sims[f.sim].cell_off + f.start;
    hi = sl.cell_off + std::min<long long>((long long)l.start + kBlockCells, sl.N);
}

// The pulls of run c (k_fused_prep) read only cells initialised once k_init
// has run on runs 0 .. c + 1: the run lies in one simulation, holds none of
// its first wrap layer (plane in 3-D, row in 2-D: those pull from the last
// one), and run c + 1 covers the pulls' forward reach (a layer, a row and a
// cell); everything before run c is initialised first.
bool run_pulls_ready(const lbm_ctx* h, int c, int n)
{
    if (c + 1 >= n) return false;
    int b0, b1, n0, n1;
    long long lo, hi, nlo, nhi;
    xfer_part(h, c, n, b0, b1, lo, hi);
    xfer_part(h, c + 1, n, n0, n1, nlo, nhi);
    if (b1 <= b0 || h->table[b0].sim != h->table[b1 - 1].sim) return false;
    const SimDev& d = h->sims[h->table[b0].sim];
    const long long layer = h->dim == 3 ? (long long)d.nx * d.ny : (long long)d.nx;
    const long long reach = layer + d.nx + 1;
    return lo - d.cell_off >= layer && hi + reach <= nhi;
}

// rho and T of the global cells [lo, hi) (offset lo in both arrays) and u (per
// simulation, component-major: D cell_off + a N + k), any of them null to skip
template <typename H>
cudaError_t xfer_cells(const lbm_ctx* h, H* dr, H* du, H* dT, const H* sr, const H* su, const H* sT, long long lo,
                       long long hi, cudaMemcpyKind kind, cudaStream_t st)
{
    const size_t n = (size_t)(hi - lo) * sizeof(H);
    cudaError_t e = cudaSuccess;
    if (n == 0) return e;
    if (dr && sr) e = cudaMemcpyAsync(dr + lo, sr + lo, n, kind, st);
    if (e == cudaSuccess && dT && sT) e = cudaMemcpyAsync(dT + lo, sT + lo, n, kind, st);
    if (e != cudaSuccess || !du || !su) return e;
    for (const SimDev& d : h->sims) {
        const long long a0 = std::max<long long>(lo, d.cell_off), a1 = std::min<long long>(hi, d.cell_off + d.N);
        for (int a = 0; a < h->dim && a0 < a1 && e == cudaSuccess; ++a) {
            const long long o = (long long)h->dim * d.cell_off + (long long)a * d.N + (a0 - d.cell_off);
            e = cudaMemcpyAsync(du + o, su + o, (size_t)(a1 - a0) * sizeof(H), kind, st);
        }
    }
    return e;
}

template <typename H> int init_impl(lbm_handle h, const H* rho, const H* u, const H* T, int on_device)
{
    if (!h) return fail(nullptr, LBM_E_INVALID, "handle is NULL");
    if (!rho || !u || !T) return fail(h, LBM_E_INVALID, "rho, u and T are required");
    h->initialized = false;  // whatever follows, the old state is gone or suspect
    const long long N = h->Ntot;
    const size_t nb_s = (size_t)N * sizeof(H), nb_v = (size_t)N * h->dim * sizeof(H);
    const bool offsets = h->storage == LBM_BF16 || h->storage == LBM_F16;
    if (offsets) {
        // the 16-bit storage offsets are the rest equilibria at the mean rho
        // and T: those two fields are read on the host, and checked there
        std::vector<H> hr, hT;
        const H *pr = rho, *pT = T;
        if (on_device) {
            hr.resize(N); hT.resize(N);
            LBM_CUDA_CHECK(h, cudaMemcpyAsync(hr.data(), rho, nb_s, cudaMemcpyDeviceToHost, h->stream));
            LBM_CUDA_CHECK(h, cudaMemcpyAsync(hT.data(), T, nb_s, cudaMemcpyDeviceToHost, h->stream));
            LBM_CUDA_CHECK(h, cudaStreamSynchronize(h->stream));
            pr = hr.data(); pT = hT.data();
        }
        for (long long k = 0; k < N; ++k)
            if (!(pr[k] > 0) || !(pT[k] > 0)) return fail(h, LBM_E_INVALID, "rho and T must be > 0 everywhere");
        for (int s = 0; s < h->nsim; ++s) {
            SimDev& d = h->sims[s];
            double mr = 0, mT = 0;
            for (long long k = 0; k < d.N; ++k) { mr += (double)pr[d.cell_off + k]; mT += (double)pT[d.cell_off + k]; }
            mr /= (double)d.N;
            mT /= (double)d.N;
            RhoPart<double> p = rho_part<double>(d, mr);
            double th = eos_P<double>(d, p, mT) / mr, e = eos_e<double>(d, p, mT), u0[3] = {0, 0, 0};
            double f[27], g[27];
            if (h->dim == 2) equilibria<2, double>(mr, u0, th, e, f, g);
            else equilibria<3, double>(mr, u0, th, e, f, g);
            for (int i = 0; i < h->Q; ++i) { d.fref[i] = (float)f[i]; d.gref[i] = (float)g[i]; }
        }
        int rc = upload_sims(h);
        if (rc) return rc;
    }
    // Host inputs go straight to a device staging buffer (a DMA when the
    // caller's memory is pinned), in parts: k_init of part c runs while part
    // c + 1 crosses the link.  k_init counts the cells with rho <= 0 or T <= 0
    // (or NaN) into diagnostic slot kDiagInitBad, read back below.
    const int single = sizeof(H) == sizeof(float);
    const H *dr = rho, *du = u, *dT = T;
    void* tmp = nullptr;
    int parts = 1;
    if (!on_device) {
        parts = xfer_parts(h);
        int rc = xfer_setup(h, parts);
        if (rc) return rc;
        tmp = dev_alloc(h, 2 * nb_s + nb_v);
        if (!tmp) return fail(h, LBM_E_NOMEM, "staging allocation failed");
        H* t = (H*)tmp;
        dr = t; dT = t + N; du = t + 2 * N;
    }
    unsigned long long bad = 0;
    cudaError_t e = cudaMemsetAsync(h->d_diag, 0, kDiagSlots * sizeof(unsigned long long), h->stream);
    int rc = e == cudaSuccess ? LBM_OK : cuda_fail(h, e, "diag reset");
    if (rc == LBM_OK && on_device) {
        rc = h->ops.init(h, dr, du, dT, single, 0, -1);
    } else if (rc == LBM_OK) {
        // the copies start after the work queued so far (the staging buffer may reuse its memory)
        e = cudaEventRecord(h->xfer_ev[parts], h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->xfer, h->xfer_ev[parts], 0);
        // the variants that carry moments between steps get them here, run by run
        // where the pulls allow (beside the upload), the rest after the last run
        const bool carried = parts > 1 && (h->variant == LBM_KERNEL_FUSED || h->variant == LBM_KERNEL_YMARCH ||
                                           h->variant == LBM_KERNEL_ZMARCH || h->variant == LBM_KERNEL_ZGATHER);
        std::vector<char> prepared(parts, 0);
        auto prepare_run = [&](int c) {
            int b0, b1;
            long long lo, hi;
            xfer_part(h, c, parts, b0, b1, lo, hi);
            prepared[c] = 1;
            return h->ops.prepare_part(h, b0, b1 - b0);
        };
        for (int c = 0; c < parts && e == cudaSuccess && rc == LBM_OK; ++c) {
            int b0, b1;
            long long lo, hi;
            xfer_part(h, c, parts, b0, b1, lo, hi);
            e = xfer_cells<H>(h, (H*)dr, (H*)du, (H*)dT, rho, u, T, lo, hi, cudaMemcpyHostToDevice, h->xfer);
            if (e == cudaSuccess) e = cudaEventRecord(h->xfer_ev[c], h->xfer);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->xfer_ev[c], 0);
            if (e == cudaSuccess) rc = h->ops.init(h, dr, du, dT, single, b0, b1 - b0);
            if (e == cudaSuccess && rc == LBM_OK && carried && c >= 1 && run_pulls_ready(h, c - 1, parts))
                rc = prepare_run(c - 1);
        }
        if (e != cudaSuccess && rc == LBM_OK) rc = cuda_fail(h, e, "lbm_init upload");
        for (int c = 0; c < parts && carried && rc == LBM_OK; ++c)
            if (!prepared[c]) rc = prepare_run(c);
        if (carried && rc == LBM_OK) h->moments_valid = true;
    }
    if (rc == LBM_OK) {
        e = cudaMemcpyAsync(&bad, h->d_diag + kDiagInitBad, sizeof(bad), cudaMemcpyDeviceToHost, h->stream);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "lbm_init check");
    }
    if (h->xfer) cudaStreamSynchronize(h->xfer);  // after an error copies may still be in flight
    cudaError_t se = cudaStreamSynchronize(h->stream);
    lbm_glue_free(tmp);
    if (rc) return rc;
    if (se != cudaSuccess) return cuda_fail(h, se, "lbm_init");
    if (bad) return fail(h, LBM_E_INVALID, "rho and T must be > 0 everywhere");
    h->initialized = true;
    return LBM_OK;
}
}  // extern "C++"

int lbm_init(lbm_handle h, const double* rho, const double* u, const double* T, int on_device)
{
    return init_impl<double>(h, rho, u, T, on_device);
}

int lbm_init_f32(lbm_handle h, const float* rho, const float* u, const float* T, int on_device)
{
    return init_impl<float>(h, rho, u, T, on_device);
}

// Capture graph_steps steps (an even number, so the buffers return to the
// same parity) into an executable graph on the handle's stream.
static int capture_graph(lbm_ctx* h)
{
    cudaGraph_t g = nullptr;
    LBM_CUDA_CHECK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    const int cur0 = h->cur;
    int rc = h->ops.step(h, h->graph_steps);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    h->cur = cur0;  // nothing ran yet: the steps run when the graph is launched
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->graph_exec[cur0], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->graph_exec[cur0] = nullptr;
        return cuda_fail(h, e, "cudaGraphInstantiate");
    }
    return LBM_OK;
}

int lbm_step(lbm_handle h, int n)
{
    if (!h) return fail(nullptr, LBM_E_INVALID, "handle is NULL");
    if (n < 0) return fail(h, LBM_E_INVALID, "n must be >= 0");
    if (!h->initialized) return fail(h, LBM_E_STATE, "lbm_init has not been called");
    if (h->graph_steps < 2 || n < h->graph_steps) return h->ops.step(h, n);
    // one eager step first: it prepares the carried moments and the kernels'
    // launch attributes, which must not happen inside a capture
    int rc = h->ops.step(h, 1);
    if (rc) return rc;
    int left = n - 1;
    if ((h->variant == LBM_KERNEL_FUSED || h->variant == LBM_KERNEL_YMARCH) && !h->moments_valid)
        return fail(h, LBM_E_STATE, "moments not prepared");
    if (!h->graph_exec[h->cur]) {
        rc = capture_graph(h);
        if (rc) return rc;
    }
    for (; left >= h->graph_steps; left -= h->graph_steps) {
        LBM_CUDA_CHECK(h, cudaGraphLaunch(h->graph_exec[h->cur], h->stream));
    }
    return left ? h->ops.step(h, left) : LBM_OK;
}

int lbm_step_timed(lbm_handle h, int n, double ms_per_pass[4])
{
    if (!h) return fail(nullptr, LBM_E_INVALID, "handle is NULL");
    if (n < 1 || !ms_per_pass) return fail(h, LBM_E_INVALID, "n must be >= 1 and ms_per_pass non-NULL");
    if (!h->initialized) return fail(h, LBM_E_STATE, "lbm_init has not been called");
    // the carried moments are prepared outside the recorded passes
    if ((h->variant == LBM_KERNEL_FUSED || h->variant == LBM_KERNEL_YMARCH || h->variant == LBM_KERNEL_ZMARCH ||
         h->variant == LBM_KERNEL_ZGATHER) &&
        !h->moments_valid) {
        int rc = h->ops.prepare(h);
        if (rc) return rc;
    }
    const size_t need = 4 * (size_t)n;
    while (h->pass_ev.size() < need) {
        cudaEvent_t ev;
        LBM_CUDA_CHECK(h, cudaEventCreate(&ev));
        h->pass_ev.push_back(ev);
    }
    int rc = LBM_OK;
    for (int k = 0; k < n && rc == LBM_OK; ++k) {
        h->pass_step = k;
        rc = h->ops.step(h, 1);
    }
    h->pass_step = -1;
    if (rc) return rc;
    LBM_CUDA_CHECK(h, cudaEventSynchronize(h->pass_ev[need - 1]));
    double acc[4] = {0, 0, 0, 0};
    for (int k = 0; k < n; ++k) {
        for (int p = 0; p < 3; ++p) {
            float ms = 0.f;
            LBM_CUDA_CHECK(h, cudaEventElapsedTime(&ms, h->pass_ev[4 * (size_t)k + p], h->pass_ev[4 * (size_t)k + p + 1]));
            acc[p] += ms;
        }
        float tot = 0.f;
        LBM_CUDA_CHECK(h, cudaEventElapsedTime(&tot, h->pass_ev[4 * (size_t)k], h->pass_ev[4 * (size_t)k + 3]));
        acc[3] += tot;
    }
    for (int p = 0; p < 4; ++p) ms_per_pass[p] = acc[p] / n;
    return LBM_OK;
}

int lbm_set_graph(lbm_handle h, int steps_per_graph)
{
    if (!h) return fail(nullptr, LBM_E_INVALID, "handle is NULL");
    if (steps_per_graph != 0 && (steps_per_graph < 2 || steps_per_graph % 2))
        return fail(h, LBM_E_INVALID, "steps_per_graph must be 0 or an even number >= 2");
    if (steps_per_graph && (h->stream == nullptr || h->stream == cudaStreamLegacy || h->stream == cudaStreamPerThread))
        return fail(h, LBM_E_STATE, "CUDA graphs need a created stream: call lbm_set_stream first");
    drop_graph(h);
    h->graph_steps = steps_per_graph;
    return LBM_OK;
}

extern "C++" {
template <typename H> int moments_impl(lbm_handle h, H* rho, H* u, H* T, int on_device)
{
    if (!h) return fail(nullptr, LBM_E_INVALID, "handle is NULL");
    if (!h->initialized) return fail(h, LBM_E_STATE, "lbm_init has not been called");
    const long long N = h->Ntot;
    const int single = sizeof(H) == sizeof(float);
    if (on_device) {
        int rc = h->ops.state_fields(h);
        if (rc == LBM_OK) rc = h->ops.export_moments(h, rho, u, T, single, 0, -1);
        if (rc) return rc;
        LBM_CUDA_CHECK(h, cudaStreamSynchronize(h->stream));
        return LBM_OK;
    }
    // to the host in parts: part c's fields cross the link while the kernels
    // work on part c + 1 (the z-march's first pass too, where it runs by parts)
    const int parts = xfer_parts(h);
    int rc = xfer_setup(h, parts);
    if (rc) return rc;
    const bool by_parts = parts > 1 && h->ops.state_part(h, 0, 0) == LBM_OK;
    if (!by_parts) {
        rc = h->ops.state_fields(h);
        if (rc) return rc;
    }
    const size_t nb_s = (size_t)N * sizeof(H), nb_v = (size_t)N * h->dim * sizeof(H);
    H* t = (H*)dev_alloc(h, 2 * nb_s + nb_v);
    if (!t) return fail(h, LBM_E_NOMEM, "staging allocation failed");
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < parts && rc == LBM_OK && e == cudaSuccess; ++c) {
        int b0, b1;
        long long lo, hi;
        xfer_part(h, c, parts, b0, b1, lo, hi);
        if (by_parts) rc = h->ops.state_part(h, b0, b1 - b0);
        if (rc == LBM_OK) rc = h->ops.export_moments(h, t, t + 2 * N, t + N, single, b0, b1 - b0);
        if (rc == LBM_OK) e = cudaEventRecord(h->xfer_ev[c], h->stream);
        if (rc == LBM_OK && e == cudaSuccess) e = cudaStreamWaitEvent(h->xfer, h->xfer_ev[c], 0);
        if (rc == LBM_OK && e == cudaSuccess)
            e = xfer_cells<H>(h, rho, u, T, t, t + 2 * N, t + N, lo, hi, cudaMemcpyDeviceToHost, h->xfer);
    }
    const cudaError_t sx = cudaStreamSynchronize(h->xfer);
    const cudaError_t ss = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) e = sx != cudaSuccess ? sx : ss;
    if (rc == LBM_OK && e != cudaSuccess) rc = cuda_fail(h, e, "lbm_moments copy");
    lbm_glue_free(t);
    return rc;
}
}  // extern "C++"

int lbm_moments(lbm_handle h, double* rho, double* u, double* T, int on_device)
{
    return moments_impl<double>(h, rho, u, T, on_device);
}

int lbm_moments_f32(lbm_handle h, float* rho, float* u, float* T, int on_device)
{
    return moments_impl<float>(h, rho, u, T, on_device);
}

int lbm_populations(lbm_handle h, double* f, double* g, int on_device)
{
    if (!h) return fail(nullptr, LBM_E_INVALID, "handle is NULL");
    if (!h->initialized) return fail(h, LBM_E_STATE, "lbm_init has not been called");
    const size_t nb = (size_t)h->Ntot * h->Q * sizeof(double);
    if (on_device) {
        int rc = h->ops.export_pops(h, f, g);
        if (rc) return rc;
        LBM_CUDA_CHECK(h, cudaStreamSynchronize(h->stream));
        return LBM_OK;
    }
    double* t = (double*)dev_alloc(h, 2 * nb);
    if (!t) return fail(h, LBM_E_NOMEM, "staging allocation failed");
    int rc = h->ops.export_pops(h, t, t + h->Ntot * h->Q);
    if (rc == LBM_OK) {
        cudaError_t e = cudaSuccess;
        if (f) e = cudaMemcpyAsync(f, t, nb, cudaMemcpyDeviceToHost, h->stream);
        if (g && e == cudaSuccess) e = cudaMemcpyAsync(g, t + h->Ntot * h->Q, nb, cudaMemcpyDeviceToHost, h->stream);
        cudaError_t se = cudaStreamSynchronize(h->stream);
        if (e == cudaSuccess) e = se;
        if (e != cudaSuccess) rc = cuda_fail(h, e, "lbm_populations copy");
    }
    lbm_glue_free(t);
    return rc;
}

int lbm_invariants(lbm_handle h, double* out)
{
    if (!h) return fail(nullptr, LBM_E_INVALID, "handle is NULL");
    if (!out) return fail(h, LBM_E_INVALID, "out is NULL");
    if (!h->initialized) return fail(h, LBM_E_STATE, "lbm_init has not been called");
    int rc = h->ops.macro(h);
    if (rc) return rc;
    const int nv = 2 * h->dim + 3;
    double* t = (double*)dev_alloc(h, (size_t)h->nsim * nv * sizeof(double));
    if (!t) return fail(h, LBM_E_NOMEM, "staging allocation failed");
    rc = h->ops.invariants(h, t);
    if (rc == LBM_OK) {
        cudaError_t e = cudaMemcpyAsync(out, t, (size_t)h->nsim * nv * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
        cudaError_t se = cudaStreamSynchronize(h->stream);
        if (e == cudaSuccess) e = se;
        if (e != cudaSuccess) rc = cuda_fail(h, e, "lbm_invariants copy");
    }
    lbm_glue_free(t);
    return rc;
}

int lbm_diagnostics(lbm_handle h, long long out[4])
{
    if (!h) return fail(nullptr, LBM_E_INVALID, "handle is NULL");
    if (!out) return fail(h, LBM_E_INVALID, "out is NULL");
    unsigned long long v[4];
    LBM_CUDA_CHECK(h, cudaMemcpyAsync(v, h->d_diag, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA_CHECK(h, cudaStreamSynchronize(h->stream));
    for (int i = 0; i < 4; ++i) out[i] = (long long)v[i];
    return LBM_OK;
}

int lbm_set_kernel(lbm_handle h, int variant, int tx, int ty, int tz)
{
    if (!h) return fail(nullptr, LBM_E_INVALID, "handle is NULL");
    drop_graph(h);
    h->moments_valid = false;  // the carried moments depend on the kernel and its tile
    if (variant == LBM_KERNEL_SPLIT) {
        h->variant = LBM_KERNEL_SPLIT;
        return LBM_OK;
    }
    if (variant == LBM_KERNEL_FUSED && split_only(h))
        return fail(h, LBM_E_UNSUPPORTED, "extrapolated faces, duct friction and throttles run on the split or z-march kernels");
    if (variant == LBM_KERNEL_ZMARCH && has_resistance(h) && !has_nee(h))
        return fail(h, LBM_E_UNSUPPORTED, "duct friction and throttles run on the split kernels without extrapolated faces");
    if (variant == LBM_KERNEL_ZMARCH && has_fields(h))
        return fail(h, LBM_E_UNSUPPORTED, "per-cell force and heat fields run on the split kernels");
    if (variant == LBM_KERNEL_ZGATHER) {
        if (h->dim != 3) return fail(h, LBM_E_INVALID, "the z-march kernels run D3Q27 lattices");
        if (!zgather_ok(h))
            return fail(h, LBM_E_UNSUPPORTED,
                        "the gathering z-march needs 32- or 16-bit storage, nx a multiple of 4 (float32) or 8 (16-bit), "
                        "at most 159 M cells per simulation, one equation of state and no extrapolated faces, "
                        "resistance or per-cell fields");
        if ((tx > 0 && tx != 30) || (ty > 0 && ty != 14))
            return fail(h, LBM_E_INVALID, "the gathering z-march has the fixed xy tile 30 x 14");
        if (tz <= 0) tz = 32;
        LBM_CUDA_CHECK(h, cudaStreamSynchronize(h->stream));
        int rc = build_tiles(h, 30, 14, tz);
        if (rc) return rc;
        h->variant = LBM_KERNEL_ZGATHER;
        h->tx = 30; h->ty = 14; h->tz = tz;
        return LBM_OK;
    }
    if (variant == LBM_KERNEL_YMARCH) {
        if (h->dim != 2) return fail(h, LBM_E_INVALID, "the row-march kernel runs D2Q9 lattices");
        if (!ymarch_ok(h))
            return fail(h, LBM_E_UNSUPPORTED,
                        "the row-march kernel needs 32- or 16-bit storage, nx a multiple of 4 (float32) or 8 "
                        "(16-bit), at most 238 M cells per simulation, one equation of state and no learned "
                        "temperature or per-cell fields");
        const int strip = ymarch_strip_width(h);
        if (tx > 0 && tx != strip) return fail(h, LBM_E_INVALID, "the row-march kernel has a fixed strip width");
        if (ty <= 0) ty = ymarch_rows(h);
        LBM_CUDA_CHECK(h, cudaStreamSynchronize(h->stream));
        int rc = build_tiles(h, strip, ty, 1, true);
        if (rc) return rc;
        h->variant = LBM_KERNEL_YMARCH;
        h->tx = strip; h->ty = ty; h->tz = 1;
        return LBM_OK;
    }
    if (variant == LBM_KERNEL_ZMARCH) {
        if (h->dim != 3) return fail(h, LBM_E_INVALID, "the z-march kernel runs D3Q27 lattices");
        if (tx <= 0 || ty <= 0) { tx = 30; ty = 14; }
        if (tz <= 0) tz = 32;
        for (const SimDev& d : h->sims)
            if (d.eos != h->sims[0].eos) return fail(h, LBM_E_INVALID, "one equation of state per z-march launch");
        if (!zmarch_shape(h->storage, tx, ty)) return fail(h, LBM_E_INVALID, "z-march tile not built");
        if (!zmarch_ok(h, tx, ty))
            return fail(h, LBM_E_UNSUPPORTED,
                        "the z-march needs at most 159 M cells per simulation; extrapolated faces on the z-march: tiles "
                        "30x14 or 30x6, 32- or 64-bit storage");
        LBM_CUDA_CHECK(h, cudaStreamSynchronize(h->stream));
        int rc = build_tiles(h, tx, ty, tz);
        if (rc) return rc;
        h->variant = LBM_KERNEL_ZMARCH;
        h->tx = tx; h->ty = ty; h->tz = tz;
        return LBM_OK;
    }
    if (variant != LBM_KERNEL_FUSED && variant != LBM_KERNEL_AUTO) return fail(h, LBM_E_INVALID, "unknown variant");
    int dtx, dty, dtz;
    fused_default_tile(h->dim, h->storage, dtx, dty, dtz);
    if (tx <= 0) tx = dtx;
    if (ty <= 0) ty = dty;
    if (tz <= 0) tz = h->dim == 3 ? dtz : 1;
    if (h->dim == 2) tz = 1;
    if (!h->ops.fused_ok(h, tx, ty, tz)) {
        if (variant == LBM_KERNEL_AUTO) {
            h->variant = LBM_KERNEL_SPLIT;
            return LBM_OK;
        }
        return fail(h, LBM_E_INVALID, "the fused kernel cannot run this tile (shared memory or shape)");
    }
    LBM_CUDA_CHECK(h, cudaStreamSynchronize(h->stream));
    int rc = build_tiles(h, tx, ty, tz);
    if (rc) return rc;
    h->variant = LBM_KERNEL_FUSED;
    h->tx = tx; h->ty = ty; h->tz = tz;
    return LBM_OK;
}

int lbm_autotune(lbm_handle h, int trial_steps, int* variant, int* tx, int* ty, int* tz, double* ms_per_step)
{
    if (!h) return fail(nullptr, LBM_E_INVALID, "handle is NULL");
    if (!h->initialized) return fail(h, LBM_E_STATE, "lbm_init has not been called");
    if (trial_steps < 1) trial_steps = 4;
    // snapshot of the state (populations of the current buffer, T guess) to restore afterwards
    const size_t pbytes = (size_t)h->pop_elems * h->sbytes, wbytes = (size_t)h->Ntot * h->rbytes;
    void* snap = dev_alloc(h, pbytes + wbytes);
    if (!snap) return fail(h, LBM_E_NOMEM, "autotune snapshot allocation failed");
    void* wT = (unsigned char*)h->W + (size_t)W_T * h->Ntot * h->rbytes;
    int rc = LBM_OK;
    const int cur0 = h->cur, var0 = h->variant, tx0 = h->tx, ty0 = h->ty, tz0 = h->tz, g0 = h->graph_steps;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto restore = [&]() {
        cudaMemcpyAsync(h->pop[cur0], snap, pbytes, cudaMemcpyDeviceToDevice, h->stream);
        cudaMemcpyAsync(wT, (unsigned char*)snap + pbytes, wbytes, cudaMemcpyDeviceToDevice, h->stream);
        h->cur = cur0;
        h->moments_valid = false;
    };
    if (cudaMemcpyAsync(snap, h->pop[cur0], pbytes, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess ||
        cudaMemcpyAsync((unsigned char*)snap + pbytes, wT, wbytes, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = fail(h, LBM_E_CUDA, "autotune setup failed");
    }
    // candidates: the split path and every built fused tile of this lattice and storage
    struct Cand { int v, x, y, z; };
    std::vector<Cand> cands{{LBM_KERNEL_SPLIT, 0, 0, 0}};
    const int shapes2[][3] = {{32, 8, 1}, {32, 16, 1}, {32, 32, 1}, {64, 16, 1}, {64, 14, 1}};
    const int shapes3[][3] = {{8, 8, 4}, {16, 8, 4}, {8, 8, 8}};
    if (h->dim == 2) {
        for (auto& t : shapes2)
            if (h->ops.fused_ok(h, t[0], t[1], t[2])) cands.push_back({LBM_KERNEL_FUSED, t[0], t[1], t[2]});
        if (ymarch_ok(h)) {
            const int ym = ymarch_rows(h);
            for (int yl : {32, 64, 128}) cands.push_back({LBM_KERNEL_YMARCH, 0, yl, 1});
            if (ym != 32 && ym != 64 && ym != 128) cands.push_back({LBM_KERNEL_YMARCH, 0, ym, 1});
        }
    } else {
        for (auto& t : shapes3)
            if (h->ops.fused_ok(h, t[0], t[1], t[2])) cands.push_back({LBM_KERNEL_FUSED, t[0], t[1], t[2]});
        const int zshapes[][3] = {{30, 14, 32}, {62, 14, 32}, {32, 16, 32}, {30, 6, 32}, {30, 14, 64}, {30, 14, 16}};
        bool same_eos = true;
        for (const SimDev& d : h->sims) same_eos = same_eos && d.eos == h->sims[0].eos;
        for (auto& t : zshapes)
            if (same_eos && zmarch_ok(h, t[0], t[1]))
                cands.push_back({LBM_KERNEL_ZMARCH, t[0], t[1], t[2]});
        if (zgather_ok(h))
            for (int zl : {16, 32, 64}) cands.push_back({LBM_KERNEL_ZGATHER, 30, 14, zl});
    }
    h->graph_steps = 0;
    drop_graph(h);
    double best = 1e300;
    Cand pick{var0, tx0, ty0, tz0};
    unsigned long long diag_save[4];
    cudaMemcpyAsync(diag_save, h->d_diag, sizeof(diag_save), cudaMemcpyDeviceToHost, h->stream);
    for (size_t c = 0; c < cands.size() && rc == LBM_OK; ++c) {
        rc = lbm_set_kernel(h, cands[c].v, cands[c].x, cands[c].y, cands[c].z);
        if (rc) break;
        restore();
        rc = h->ops.step(h, 2);  // warm-up (and launch set-up)
        if (rc) break;
        cudaEventRecord(e0, h->stream);
        rc = h->ops.step(h, trial_steps);
        cudaEventRecord(e1, h->stream);
        if (rc) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = fail(h, LBM_E_CUDA, "autotune timing failed"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = ms / trial_steps;
        if (per < best) { best = per; pick = cands[c]; }
    }
    restore();
    cudaMemcpyAsync(h->d_diag, diag_save, sizeof(diag_save), cudaMemcpyHostToDevice, h->stream);
    cudaStreamSynchronize(h->stream);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    lbm_glue_free(snap);
    if (rc == LBM_OK) rc = lbm_set_kernel(h, pick.v, pick.x, pick.y, pick.z);
    else lbm_set_kernel(h, var0, tx0, ty0, tz0);
    h->graph_steps = g0;
    if (rc) return rc;
    if (variant) *variant = pick.v;
    if (tx) *tx = pick.x;
    if (ty) *ty = pick.y;
    if (tz) *tz = pick.z;
    if (ms_per_step) *ms_per_step = best;
    return LBM_OK;
}

int lbm_mlp_load(lbm_handle h, const float* params)
{
    if (!h) return fail(nullptr, LBM_E_INVALID, "handle is NULL");
    if (!params) return fail(h, LBM_E_INVALID, "params is NULL");
    const int np = lbm_mlp_nparams();
    if (!h->d_mlp) {
        h->d_mlp = (float*)dev_alloc(h, (size_t)np * sizeof(float));
        if (!h->d_mlp) return fail(h, LBM_E_NOMEM, "parameter allocation failed");
    }
    LBM_CUDA_CHECK(h, cudaMemcpyAsync(h->d_mlp, params, (size_t)np * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    for (SimDev& d : h->sims)
        if (d.eos == EOS_PR && d.t_solver == LBM_T_MLP) d.mlp = h->d_mlp;
    drop_graph(h);
    int rc = upload_sims(h);
    if (rc) return rc;
    if (h->variant == LBM_KERNEL_FUSED && !h->ops.fused_ok(h, h->tx, h->ty, h->tz)) h->variant = LBM_KERNEL_SPLIT;
    return LBM_OK;
}

int lbm_get_kernel(lbm_handle h, int* variant, int* tx, int* ty, int* tz)
{
    if (!h) return fail(nullptr, LBM_E_INVALID, "handle is NULL");
    if (variant) *variant = h->variant;
    if (tx) *tx = h->tx;
    if (ty) *ty = h->ty;
    if (tz) *tz = h->tz;
    return LBM_OK;
}

const char* lbm_last_error(lbm_handle h)
{
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

}  // extern "C"
