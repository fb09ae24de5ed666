// Shared-memory-staged sparse x block-of-vectors product for the block-CG solves (see spmm.cu).
#pragma once

#include "internal.cuh"

namespace sbha {

constexpr int kTileRows = 128;     // matrix rows per tile
constexpr int kHaloCap = 288;      // rows a tile stages (its rows and their neighbours)
constexpr int kTileThreads = 256;  // 8 warps

// Row tiles of an m x m CSR matrix whose rows are numbered in locality order: tile t holds
// rows [t kTileRows, (t+1) kTileRows), with the sorted list of rows its entries reference (its
// halo) and, per entry, the entry's index in that list.
struct TiledPattern {
  int64_t m = 0, nnz = 0;
  int ntiles = 0;
  int rows = kTileRows;  // rows per tile
  int cap = kHaloCap;    // halo capacity per tile (halo lists are padded to multiples of 4 rows)
  const int32_t* rowptr = nullptr;  // the matrix's CSR (not owned)
  const int32_t* col = nullptr;
  int32_t* lcol = nullptr;    // [nnz] staged-row index of each entry
  uint16_t* lself = nullptr;  // [ntiles rows] staged-row index of each row itself (the halo holds the tile's rows)
  int32_t* halo = nullptr;   // [ntiles][kHaloCap] rows staged by each tile
  int32_t* nh = nullptr;     // [ntiles] halo size; above kHaloCap the tile reads global memory
  int staged_tiles = 0;      // tiles whose halo fits
  int64_t halo_rows = 0;     // sum of the staged tiles' halo sizes
};

// perm[i] = the i-th of the m items (positions xyz[3 vert[i] ..], vert nullable: identity) along
// a Morton curve through their bounding box (ties: smaller i); xyz = nullptr: perm[i] = i.
void locality_order(Ctx& c, int64_t m, const int32_t* vert, const double* xyz, int32_t* perm);

// Tiles of the m x m CSR (rowptr, col): kTileRows rows and kHaloCap halo rows per tile (the
// staged product), or, with rows = kGatherRows, the tiles of the TMA gather product.  Device
// memory from the context.
TiledPattern build_tiles(Ctx& c, int64_t m, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                         int rows = kTileRows);

// Tiles of the TMA gather product (spmm_tma.cu).
constexpr int kGatherRows = 64;
constexpr int kGatherCap = 192;

// y = alpha A x as spmm_tiled, FP32, over the tiles of build_tiles(..., kGatherRows): each tile's
// halo rows are brought into shared memory by TMA four-row gathers, a column group of four blocks
// at a time, double-buffered under a producer warp while sixteen warps compute.  Every row is summed
// in the order of its CSR entries, like the gather products of the solver, so y is bit-identical
// to theirs.  Returns false (nothing launched) where it does not apply: x not 16-byte aligned, or
// more than 2^31 block rows.
bool spmm_tma(Ctx& c, const TiledPattern& tp, int nb, const float* val, const float* x, float* y, float alpha,
              double* acc, const int32_t* blk_act, bool self_dot);

// y = alpha A x over the nb column blocks of the block layout (column c of row u at
// ((c/32) m + u) 32 + c%32); blocks with blk_act[b] == 0 are skipped (nullable).  With acc,
// also acc[c] += sum_u x_uc y_uc (or sum_u y_uc^2 with self_dot).  val: A's values (CSR order).
template <class T>
void spmm_tiled(Ctx& c, cudaStream_t s, const TiledPattern& tp, int nb, const T* val, const T* x, T* y, T alpha,
                double* acc, const int32_t* blk_act, bool self_dot);

}  // namespace sbha
