// Host-side interface between the C-ABI layer (gpp_api.cu) and the kernel files.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "gpp.h"

namespace gpp {

struct BandEntry;
struct BandEntry32;

// Layout of the caller's workspace for one forward call. Every segment starts on a
// 256-byte boundary.
struct FwdPlan {
  int threads = 128;      // threads per CTA of the main kernel
  int grid = 0;           // CTAs of the main kernel (a persistent, statically scheduled grid)
  int nw = 0;
  int64_t n_ig_tiles = 0; // ig tiles of `threads` G-vectors per column
  int64_t ntiles = 0;     // ngpown * n_ig_tiles
  size_t off_flags = 0;   // int32[4]: [0] any wx < 0, [1] bad index count, [2] any |wx| >= 1e4
  size_t off_colvalid = 0;// int32[P]
  size_t off_bt = 0;      // band table double4[B][W] = {x, x^2, 4x, 0}
  size_t off_am = 0;      // gathered weights c128[P][B] = conj(aqsmtemp[b][g(p)]) vcoul[g(p)]
  size_t off_partials = 0;// double[grid][4 W]
  size_t off_bt32 = 0;    // FP32-bulk only: BandEntry32[B][W]
  size_t off_am32 = 0;    // FP32-bulk only: gathered weights c64[P][B]
  size_t total = 0;
};

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Main-kernel CTAs that fit on one SM (occupancy query; 0 on error).
int fwd_f64_blocks_per_sm(int threads, int nw);
int fwd_f32_blocks_per_sm(int threads, int nw);
bool fwd_f32_available();

// Column gather, band table and index checks (one kernel).
cudaError_t launch_prep(const gpp_problem& p, const FwdPlan& plan, char* ws, bool fp32,
                        cudaStream_t s);
// Main sum in FP64 (writes per-CTA partials).
cudaError_t launch_fwd_f64(const gpp_problem& p, int occ_mode, const FwdPlan& plan, char* ws,
                           cudaStream_t s);
// Main sum with FP32 bulk arithmetic (writes per-CTA partials in FP64).
cudaError_t launch_fwd_f32(const gpp_problem& p, int occ_mode, const FwdPlan& plan, char* ws,
                           cudaStream_t s);
// Workspace of the adjoint: the forward's gather segments plus the batch partials.
struct BwdPlan {
  FwdPlan fwd;             // flags, colvalid, band table, gathered weights
  int batch_groups = 1;    // column groups (8 columns each) per main-kernel launch
  int max_grid = 1;        // persistent grid of the main kernel
  size_t off_bwd_bt = 0;   // BwdBand[B][W]
  size_t off_part_n = 0;   // c128[batch_groups][B][G]
  size_t off_part_r = 0;   // c128[ceil(G/32)][B][batch_groups * 8]
  size_t off_rtot = 0;     // c128[B][P]
  size_t total = 0;
};

int bwd_blocks_per_sm(int nw);
int64_t bwd_groups(int64_t P);
int bwd_tile_ig();
int bwd_tile_cols();
cudaError_t launch_bwd(const gpp_problem& p, int occ_mode, const BwdPlan& plan, char* ws,
                       const gpp_c128* g_ach, const gpp_c128* g_asx, const gpp_grads& out,
                       cudaStream_t s);

// One instance of a batched launch (device-resident descriptor; see gpp_batched.cu).
struct BatchInst {
  int B = 0, nocc = 0;
  int index = 0;  // position of the instance in the caller's array
  int pad = 0;
  int64_t G = 0, P = 0, n_ig_tiles = 0, tile0 = 0, tile_end = 0;
  const double2* aqsn = nullptr;
  const float2* aqsn32 = nullptr;
  const double2* eps = nullptr;
  const double2* wt = nullptr;
  const double2* am = nullptr;
  const float2* am32 = nullptr;
  const BandEntry* bt = nullptr;
  const BandEntry32* bt32 = nullptr;
  const int* colg = nullptr;
  const int* flags = nullptr;
  gpp_c128* ach = nullptr;
  gpp_c128* asx = nullptr;
};

int batched_blocks_per_sm(int threads, int nw, bool f32);
// Resets the tile counter, runs the persistent kernel and the per-instance reduction.
cudaError_t launch_batched(const BatchInst* inst, int ninst, int64_t ntiles, int nw, bool f32,
                           int grid, int threads, int igpt, unsigned long long* counter,
                           double* partials, cudaStream_t s);

// Sets the thread-local message returned by gpp_last_error(); returns `code`.
int report_error(int code, const char* msg);
void clear_error();

// Fixed-order reduction of the partials into achtemp / asxtemp.
cudaError_t launch_reduce_final(const FwdPlan& plan, char* ws, gpp_c128* ach, gpp_c128* asx,
                                cudaStream_t s);

}  // namespace gpp
