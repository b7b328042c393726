// Mixed-precision chi0 assembly on tcgen05 tensor cores (declarations).
#pragma once
#include <vector>

#include "internal.cuh"

namespace qsgw {

// Device scratch owned by a context for the mixed path, grown on demand and reused by every
// accumulate call: digit planes of the row operand, FP32 copy of Z for the column operand,
// FP32 weights, per-chunk maxima / exponents, and cached device lists of upper-triangle tiles.
struct TileList {
  int n_pb, tj, rows_i, col0, count;
  int2* tiles;
};
// Tile plan of the tensor-core launch: J columns per output tile (0: the widest the frequency count
// allows) and the chunk-range pieces each tile of a partial last wave is cut into (0: enough to fill
// the SMs, capped by the chunk count; 1: not cut).
struct TilePlan {
  int tj = 0, pieces = 0;
};
// A tuned plan for one size class: frequency count, log2 of the 64 x 64 output-tile area of all
// blocks, log2 of the largest chunk count.
struct PlanEntry {
  int L, ca, cc;
  TilePlan plan;
};
struct MixedScratch {
  void* planes = nullptr;
  size_t planes_cap = 0;
  std::vector<TileList> tile_lists;
  bool attr_set = false;
  int n_sm = 0;
  int* counter = nullptr;  // work-queue counter of the tensor-core launch
  std::vector<PlanEntry> plans;  // tuned plans (qsgw_chi0_autotune or the plan file)
  bool use_forced = false;       // qsgw_chi0_set_tile_plan: this plan for every unrestricted launch
  TilePlan forced;
};

// One block of transition columns for one q-point. acc: the q-point's accumulator, a double-float
// buffer (float2 (hi, lo) planes [L][2 (re, im)][n_pad (J)][n_pad (I)]) followed by an FP64 buffer
// of the same layout for split tiles; chi0 is their sum.
struct MixedBlock {
  const void* Z;  // complex128 (double2), or complex64 (float2) when z32
  long long ldz;
  int n_pb, n_pad, n_occ, n_unocc;
  const double* eo;
  const double* eu;
  float4* acc;
  bool z32;  // Z holds complex64: the mixed path rounds every element to FP32 first anyway
  // Given weights (L = 1) instead of the weights from Delta: w_r = wv[r mod n_unocc], wv > 0.
  const double* wv;
  // rows_i > 0: only the off-diagonal block of rows I < rows_i and columns J >= col0 (a multiple
  // of mixed_tile_cols(L), >= rows_i) is computed: the product of two row sets of Z.
  int rows_i = 0, col0 = 0;
};

// Columns per output tile of the tensor-core kernel for L frequencies (rows per tile: 64).
int mixed_tile_cols(int L);

// Prep of every block, then one persistent tensor-core launch over all (block, tile, chunk)
// items. Blocks must belong to distinct q-points (distinct accumulators); at most 32 blocks.
qsgw_status mixed_accumulate_batch(MixedScratch& s, int nb, const MixedBlock* blocks, const OmegaGrid& g, int* d_err,
                                   cudaStream_t stream);
qsgw_status mixed_accumulate(MixedScratch& s, const void* Z, bool z32, long long ldz, int n_pb, int n_pad, int n_occ,
                             int n_unocc, const double* eo, const double* eu, const double* wv, const OmegaGrid& g,
                             float4* acc, int* d_err, cudaStream_t stream);
void mixed_free(MixedScratch& s);
// Candidate plans for L frequencies (at most max_out), the tuner's search space: the three widest
// valid tile widths, each with the default tail cut and with no cut.
int mixed_plan_candidates(int L, TilePlan* out, int max_out);
bool mixed_plan_valid(int L, const TilePlan& p);
void mixed_plan_class(int nb, const MixedBlock* in, int* ca, int* cc);
// Times every candidate on these blocks (into scratch accumulators of the same sizes, so the
// blocks' own accumulators are untouched), keeps the fastest for the blocks' class in s.plans.
qsgw_status mixed_autotune(MixedScratch& s, int nb, const MixedBlock* in, const OmegaGrid& g, int* d_err,
                           cudaStream_t stream, int reps, TilePlan* best, float* best_ms);
// chi0 of one block of columns into `chi0` using only a fixed file-scope device array (no allocation).
qsgw_status mixed_chi0_noalloc(const double2* Z, long long ldz, int n_pb, int n_occ, int n_unocc, const double* eo,
                               const double* eu, const OmegaGrid& g, double spin, double2* chi0, cudaStream_t stream);

}  // namespace qsgw
