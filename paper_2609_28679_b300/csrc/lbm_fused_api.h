// Entry points of the fused-step instantiations.  Each storage type lives in
// its own translation unit (lbm_fused_<storage>.cu) so that the kernels,
// specialised per lattice, equation of state and tile shape, compile in
// parallel.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

struct SimDev;
struct TileEntry;
struct BlockEntry;

#define LBM_FUSED_DECL(NAME)                                                                                     \
    cudaError_t fused_dispatch_##NAME(int dim, int eos, int mlp, int pc, int tx, int ty, int tz, const SimDev* sims,              \
                                      const TileEntry* tiles, int ntiles, const void* src, void* dst,            \
                                      const void* Min, void* Mout, long long Ntot, unsigned long long* diag,     \
                                      cudaStream_t stream);                                                      \
    bool fused_shape_##NAME(int dim, int tx, int ty, int tz);                                                   \
    cudaError_t zmarch_dispatch_##NAME(int eos, int tx, int ty, int zl, const SimDev* sims, const TileEntry* tiles, \
                                       int ntiles, const void* src, void* dst, const void* W, void* Mout,          \
                                       long long Ntot, cudaStream_t stream);                                      \
    bool zmarch_shape_##NAME(int tx, int ty);                                                                   \
    cudaError_t zmacro_dispatch_##NAME(int eos, int mlp, const SimDev* sims, const BlockEntry* table, int nblocks, \
                                       const void* M, void* W, long long Ntot, unsigned long long* diag,          \
                                       cudaStream_t stream);

LBM_FUSED_DECL(f64)
LBM_FUSED_DECL(f32)

// z-march with extrapolated z faces (tiles 30 x 14 and 30 x 6; 32- and 64-bit storage)
cudaError_t zmarch_nee_dispatch_f64(int eos, int tx, int ty, int zl, const SimDev* sims, const TileEntry* tiles,
                                    int ntiles, const void* src, void* dst, const void* W, void* Mout, long long Ntot,
                                    cudaStream_t stream);
cudaError_t zmarch_nee_dispatch_f32(int eos, int tx, int ty, int zl, const SimDev* sims, const TileEntry* tiles,
                                    int ntiles, const void* src, void* dst, const void* W, void* Mout, long long Ntot,
                                    cudaStream_t stream);
LBM_FUSED_DECL(bf16)
LBM_FUSED_DECL(f16)
#undef LBM_FUSED_DECL

// column-march collide-stream pass (staged pulls, gathered moments): 32- and 16-bit storage
cudaError_t zgather_dispatch_f32(int eos, int zl, const SimDev* sims, const TileEntry* tiles, int ntiles,
                                 const void* src, void* dst, const void* W, void* Mout, long long Ntot,
                                 cudaStream_t stream);
cudaError_t zgather_dispatch_bf16(int eos, int zl, const SimDev* sims, const TileEntry* tiles, int ntiles,
                                  const void* src, void* dst, const void* W, void* Mout, long long Ntot,
                                  cudaStream_t stream);
cudaError_t zgather_dispatch_f16(int eos, int zl, const SimDev* sims, const TileEntry* tiles, int ntiles,
                                 const void* src, void* dst, const void* W, void* Mout, long long Ntot,
                                 cudaStream_t stream);

// row-march one-pass step for D2Q9 (32- and 16-bit storage); pc: every simulation takes the central Phi.
// Owned columns of a strip: 128 threads less the rim and the stencils' reach (1 central, 2 upwind-biased).
constexpr int kYmStripCentral = 124, kYmStripUpwind = 122;
#define LBM_YMARCH_DECL(SUF)                                                                                          \
    cudaError_t ymarch_dispatch_##SUF(int eos, int pc, int yl, const SimDev* sims, const TileEntry* tiles, int ntiles, \
                                      const void* src, void* dst, const void* Min, void* Mout, long long Ntot,         \
                                      unsigned long long* diag, cudaStream_t stream);                         \
    cudaError_t ymarch_slots_##SUF(int eos, int pc, int* slots);
LBM_YMARCH_DECL(f32)
LBM_YMARCH_DECL(bf16)
LBM_YMARCH_DECL(f16)
#undef LBM_YMARCH_DECL

}  // namespace lbm
