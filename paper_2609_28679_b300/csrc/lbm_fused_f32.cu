// Fused-step kernels for float32 population storage: every tile shape below,
// for D2Q9 and D3Q27 and each equation of state.
#include "lbm_fused.cuh"
#include "lbm_fused_api.h"
#include "lbm_ymarch.cuh"
#include "lbm_zgather.cuh"
#include "lbm_zmarch.cuh"

namespace lbm {

#define TILES_2D(X) X(32, 8, 1) X(32, 16, 1) X(32, 32, 1) X(64, 16, 1) X(64, 14, 1)
#define TILES_3D(X) X(8, 8, 4) X(16, 8, 4) X(8, 8, 8)

namespace {

template <int D, int EK, bool ML>
cudaError_t go(int pc, int tx, int ty, int tz, const SimDev* sims, const TileEntry* tiles, int ntiles, const void* src,
               void* dst, const void* Min, void* Mout, long long Ntot, unsigned long long* diag, cudaStream_t stream)
{
#define CASE(A, B, C)                                                                                           \
    if (tx == A && ty == B && tz == C)                                                                          \
        return fused_launch_shape<D, float, float, EK, ML, A, B, C>(pc, sims, tiles, ntiles, src, dst, Min, Mout, Ntot, diag,  \
                                                         stream);
    if constexpr (D == 2) {
        TILES_2D(CASE)
    } else {
        TILES_3D(CASE)
    }
#undef CASE
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t fused_dispatch_f32(int dim, int eos, int mlp, int pc, int tx, int ty, int tz, const SimDev* sims, const TileEntry* tiles,
                               int ntiles, const void* src, void* dst, const void* Min, void* Mout, long long Ntot,
                               unsigned long long* diag, cudaStream_t stream)
{
#define ARGS pc, tx, ty, tz, sims, tiles, ntiles, src, dst, Min, Mout, Ntot, diag, stream
    if (mlp) {  // learned temperature start: Peng-Robinson, float32 storage
        if (eos != EOS_PR) return cudaErrorInvalidValue;
        if (dim == 2) return go<2, EOS_PR, true>(ARGS);
        if (dim == 3) return go<3, EOS_PR, true>(ARGS);
        return cudaErrorInvalidValue;
    }
    if (dim == 2) {
        if (eos == EOS_IDEAL) return go<2, EOS_IDEAL, false>(ARGS);
        if (eos == EOS_VDW) return go<2, EOS_VDW, false>(ARGS);
        if (eos == EOS_PR) return go<2, EOS_PR, false>(ARGS);
    } else if (dim == 3) {
        if (eos == EOS_IDEAL) return go<3, EOS_IDEAL, false>(ARGS);
        if (eos == EOS_VDW) return go<3, EOS_VDW, false>(ARGS);
        if (eos == EOS_PR) return go<3, EOS_PR, false>(ARGS);
    }
#undef ARGS
    return cudaErrorInvalidValue;
}

bool fused_shape_f32(int dim, int tx, int ty, int tz)
{
#define HAS(A, B, C) if (tx == A && ty == B && tz == C) return true;
    if (dim == 2) {
        TILES_2D(HAS)
    } else if (dim == 3) {
        TILES_3D(HAS)
    }
#undef HAS
    return false;
}

// z-march shapes (xy tile; the z range is a launch parameter)
#define ZTILES(X) X(30, 14) X(62, 14) X(32, 16) X(30, 6)

namespace {
template <int EK>
cudaError_t zgo(int tx, int ty, int zl, const SimDev* sims, const TileEntry* tiles, int ntiles, const void* src,
                void* dst, const void* W, void* Mout, long long Ntot, cudaStream_t stream)
{
#define ZCASE(A, B) \
    if (tx == A && ty == B) return zmarch_launch_shape<float, float, EK, A, B>(sims, tiles, ntiles, zl, src, dst, W, Mout, Ntot, stream);
    ZTILES(ZCASE)
#undef ZCASE
    return cudaErrorInvalidValue;
}
}  // namespace

// z-march with extrapolated z faces (walls and duct ends), on the default and the narrow tile
namespace {
template <int EK>
cudaError_t zgo_nee(int tx, int ty, int zl, const SimDev* sims, const TileEntry* tiles, int ntiles, const void* src,
                    void* dst, const void* W, void* Mout, long long Ntot, cudaStream_t stream)
{
    if (tx == 30 && ty == 14)
        return zmarch_launch_shape<float, float, EK, 30, 14, true>(sims, tiles, ntiles, zl, src, dst, W, Mout, Ntot, stream);
    if (tx == 30 && ty == 6)
        return zmarch_launch_shape<float, float, EK, 30, 6, true>(sims, tiles, ntiles, zl, src, dst, W, Mout, Ntot, stream);
    return cudaErrorInvalidValue;
}
}  // namespace

cudaError_t zmarch_nee_dispatch_f32(int eos, int tx, int ty, int zl, const SimDev* sims, const TileEntry* tiles,
                                    int ntiles, const void* src, void* dst, const void* W, void* Mout, long long Ntot,
                                    cudaStream_t stream)
{
    if (eos == EOS_IDEAL) return zgo_nee<EOS_IDEAL>(tx, ty, zl, sims, tiles, ntiles, src, dst, W, Mout, Ntot, stream);
    if (eos == EOS_VDW) return zgo_nee<EOS_VDW>(tx, ty, zl, sims, tiles, ntiles, src, dst, W, Mout, Ntot, stream);
    if (eos == EOS_PR) return zgo_nee<EOS_PR>(tx, ty, zl, sims, tiles, ntiles, src, dst, W, Mout, Ntot, stream);
    return cudaErrorInvalidValue;
}

cudaError_t zmarch_dispatch_f32(int eos, int tx, int ty, int zl, const SimDev* sims, const TileEntry* tiles,
                                int ntiles, const void* src, void* dst, const void* W, void* Mout, long long Ntot,
                                cudaStream_t stream)
{
    if (eos == EOS_IDEAL) return zgo<EOS_IDEAL>(tx, ty, zl, sims, tiles, ntiles, src, dst, W, Mout, Ntot, stream);
    if (eos == EOS_VDW) return zgo<EOS_VDW>(tx, ty, zl, sims, tiles, ntiles, src, dst, W, Mout, Ntot, stream);
    if (eos == EOS_PR) return zgo<EOS_PR>(tx, ty, zl, sims, tiles, ntiles, src, dst, W, Mout, Ntot, stream);
    return cudaErrorInvalidValue;
}

cudaError_t zmacro_dispatch_f32(int eos, int mlp, const SimDev* sims, const BlockEntry* table, int nblocks,
                                  const void* M, void* W, long long Ntot, unsigned long long* diag, cudaStream_t stream)
{
    return zmacro_dispatch_t<float, true>(eos, mlp, sims, table, nblocks, M, W, Ntot, diag, stream);
}

bool zmarch_shape_f32(int tx, int ty)
{
#define ZHAS(A, B) if (tx == A && ty == B) return true;
    ZTILES(ZHAS)
#undef ZHAS
    return false;
}

cudaError_t zgather_dispatch_f32(int eos, int zl, const SimDev* sims, const TileEntry* tiles, int ntiles,
                                 const void* src, void* dst, const void* W, void* Mout, long long Ntot,
                                 cudaStream_t stream)
{
    return zgather_dispatch_t<float>(eos, zl, sims, tiles, ntiles, src, dst, W, Mout, Ntot, stream);
}


cudaError_t ymarch_dispatch_f32(int eos, int pc, int yl, const SimDev* sims, const TileEntry* tiles, int ntiles,
                              const void* src, void* dst, const void* Min, void* Mout, long long Ntot,
                              unsigned long long* diag, cudaStream_t stream)
{
    return ymarch_dispatch_t<float>(eos, pc, yl, sims, tiles, ntiles, src, dst, Min, Mout, Ntot, diag, stream);
}
cudaError_t ymarch_slots_f32(int eos, int pc, int* slots)
{
    return ymarch_slots_t<float>(eos, pc, slots);
}
}  // namespace lbm
