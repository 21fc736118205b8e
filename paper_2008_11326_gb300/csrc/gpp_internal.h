// Host-side interface between the C-ABI layer (gpp_api.cu) and the kernel files.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "gpp.h"

namespace gpp {

struct BandEntry;

// Layout of the caller's workspace for one forward call. Every segment starts on a
// 256-byte boundary. With `gather_only` (instances of a batched plan, the adjoint) the
// descriptor, counter and partial segments are empty.
struct FwdPlan {
  int threads = 128;      // threads per CTA of the main kernel
  int igpt = 4;           // G-vectors per thread per tile
  int grid = 0;           // CTAs of the persistent main kernel
  int nw = 0;
  int64_t n_ig_tiles = 0; // tiles per column: ceil(G / (threads * igpt))
  int64_t ntiles = 0;     // ngpown * n_ig_tiles
  size_t off_flags = 0;   // int32[4]: [0] any wx < 0, [1] bad index count, [2] any |wx| >= 1e4;
                          // then uint64: the bits of max |wx| (kFlagXmax)
  size_t off_colvalid = 0;// int32[P]: global column of each local column, or -1
  size_t off_bt = 0;      // band table BandEntry[B][W] = {x, x^2, 0, -x/2}
  size_t off_am = 0;      // gathered weights c128[P][B] = conj(aqsmtemp[b][g(p)]) vcoul[g(p)]
  size_t off_bt32 = 0;    // FP32-bulk only: float4[B][f32_band_quads(W)]
  size_t off_am32 = 0;    // FP32-bulk only: gathered weights c64[P][B]
  size_t off_aqsn32 = 0;  // FP32-bulk without a caller's copy: complex64 aqsntemp [B][G]
  bool convert_c64 = false;  // the gather launch writes that copy first
  size_t gather_total = 0;
  size_t off_desc = 0;    // the instance descriptor (BatchInst)
  size_t off_counter = 0; // tile counter
  size_t off_partials = 0;// 8 bytes x [ntiles][4 W]: double (FP64) or float2 (FP32-bulk)
  size_t total = 0;
};

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct BatchInst;

// Column gather, band tables and index checks (one kernel); with `desc` it also writes the
// single-instance descriptor to plan.off_desc. With plan.convert_c64 the complex64 copy of
// aqsntemp is written to plan.off_aqsn32 first.
cudaError_t launch_prep(const gpp_problem& p, const FwdPlan& plan, char* ws, bool fp32,
                        const BatchInst* desc, cudaStream_t s);
// dst[r][c] = complex64(src[r][c]) (round to nearest) for rows [0, rows) and columns
// [c0, c1); leading dimensions in elements.
cudaError_t launch_convert_c64(const gpp_c128* src, int64_t ld_src, gpp_c64* dst, int64_t ld_dst,
                               int64_t rows, int64_t c0, int64_t c1, cudaStream_t s);
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
cudaError_t launch_bwd(const gpp_problem& p, int occ_mode, double ach_scale, double sx2,
                       const BwdPlan& plan, char* ws, const gpp_c128* g_ach,
                       const gpp_c128* g_asx, const gpp_grads& out, cudaStream_t s);

// One instance of a batched launch (device-resident descriptor; see gpp_batched.cu).
struct BatchInst {
  int B = 0, nocc = 0;
  int index = 0;     // position of the instance in the caller's array
  int occ_mode = 0;  // host-side bookkeeping while a batch is laid out
  int64_t G = 0, P = 0, n_ig_tiles = 0, tile0 = 0, tile_end = 0;
  const double2* aqsn = nullptr;
  const float2* aqsn32 = nullptr;
  const double2* eps = nullptr;
  const double2* wt = nullptr;
  const double2* am = nullptr;
  const float2* am32 = nullptr;
  const BandEntry* bt = nullptr;
  const float4* bt32 = nullptr;
  const int* colg = nullptr;
  const int* flags = nullptr;
  gpp_c128* ach = nullptr;
  gpp_c128* asx = nullptr;
  double ach_scale = 1.0;  // 1/2 with GPP_PHYS_CH_HALF
  double sx2 = 0.0;        // sexcut^2 with GPP_PHYS_SX_CUTOFF, else 0
};

// Lets the main kernel take the shared memory the launch shape needs; before occupancy
// queries and launches.
cudaError_t batched_prepare(int threads, int nw, bool f32, int igpt);
int batched_blocks_per_sm(int threads, int nw, bool f32, int igpt);
// Resets the tile counter and runs the persistent main kernel over tiles [t_begin, ntiles).
cudaError_t launch_batched_main(const BatchInst* inst, int ninst, int64_t ntiles, int nw,
                                bool f32, int grid, int threads, int igpt,
                                unsigned long long* counter, double* partials, cudaStream_t s,
                                int64_t t_begin = 0);
// Per-instance fixed-order sum of the tile partials into the outputs.
cudaError_t launch_batched_reduce(const BatchInst* inst, int ninst, int nw, bool f32,
                                  const double* partials, cudaStream_t s);

// gpp_sigma's workspace bytes for this problem and these options, with the status of the
// validation (GPP_OK, or the code gpp_sigma would return for these arguments).
int sigma_workspace_query(const gpp_problem* prob, const gpp_options* opt, size_t* bytes);

// Every CUDA call whose status the entry points check passes through here: returns e, or
// a simulated failure when gpp_diag_inject_cuda_failure's countdown on this host thread
// reaches this call (the call itself has been made).
cudaError_t checked(cudaError_t e);

// Sets the thread-local message returned by gpp_last_error(); returns `code`.
int report_error(int code, const char* msg);
void clear_error();


}  // namespace gpp
