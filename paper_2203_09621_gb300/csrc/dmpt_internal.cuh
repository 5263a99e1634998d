// Internal declarations shared by the translation units of libdmpt.so.
//
// Device-resident control: the whole layer loop of Algorithms 1-3 runs on the
// GPU.  After each layer product, a one-block "decide" kernel reduces the
// per-tile FP64 partial sums written by the product's epilogue, applies the
// Alg. 2 / Alg. 3 tests and plans the next layer (branch sigma_n, whether the
// square is computed and stored, which directions still run, operand scale
// exponents).  The product kernels read that plan from State at launch.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dmpt.h"

namespace dmpt {

constexpr int kMaxK = DMPT_MAX_K;
constexpr int kMaxL = DMPT_MAX_LAYERS;
constexpr int kPad = 256;   // internal matrices are zero-padded to a multiple of this
constexpr int kNQ = 4;      // partial sums per (job, tile): see Partial* below

// Partial-sum slots per (job, tile).  Job 0 is the square (S0), job 1+k the
// response of direction k.
enum : int {
  kQTrace = 0,    // job 0: sum of the new diagonal          (Tr S_n)
  kQFroNew = 1,   // ||S_new||_F^2 over the tile (both triangles)
  kQFroDiff = 2,  // ||S_old - X||_F^2  (FroErr^(0) / FroErr^(1)_n of Alg. 2 / 3)
  kQBad = 3       // count of non-finite values seen
};

// Device state block (lives at the start of the workspace).
struct State {
  int n_layer;          // layer the next product computes (1-based)
  int done;             // 1: converged, failed or capped; later launches are no-ops
  int status;           // dmpt_status
  int timeout_flag;     // set by a kernel whose bounded wait expired
  int d0_conv;          // Alg. 2 has fired
  int d0_layer;         // layer at which it fired
  int cur0;             // ping-pong buffer holding the current S0
  int sigma_cur;        // sigma of the planned layer
  int plan_square;      // planned layer computes X = S0^2
  int plan_write0;      // ... and stores S0_n = sigma X + (1 - sigma) S0_{n-1}
  int s0_exp;           // power-of-two exponent of the 16-bit S0 copies
  int k;                // directions
  int max_layers;
  int precision;
  int layers_run;       // layers whose product finished
  int tape;             // 1: each S0 state's 16-bit copies are kept (adjoint)
  int z0_cur;           // operand slice (hi; lo = +1) of the current S0
  int z0_next;          // slice the next stored S0 copies go to
  int tape_base;        // first tape slice
  int tape_states;      // tape capacity (states)
  int d0_updates;       // S0 updates so far (tape states = d0_updates + 1)
  int layout_k;         // response slots in the workspace layout
  int k_fwd;            // directions of the forward run
  int adj_m;            // adjoint: layer whose adjoint runs next
  int rp_lmax;          // replay: last layer whose sigma the forward recorded
  int rp_layers;        // replay: layers run
  int order;            // highest response order (1: first order only)
  int k1;               // first-order directions (job 1 + (o - 1) k1 + d: order o)
  unsigned round_ctr;   // pair kernel: rounds started by its CTAs (soft alignment);
                        // every decide step resets it before the next launch
  int hole;             // 1: the recursion runs on I - P (complement form)
  int ckpt_k;           // >= 2: FP32 checkpoint of every ckpt_k-th S0 state
  int ckpt_slots;       // checkpoint capacity (states)
  int ckpt_pending;     // the last decide step made a state that is checkpointed
  int adj_seg_a;        // adjoint with checkpoints: first state held in the tape
  int64_t item_base;    // pair kernel: virtual index of its first item (0 except
                        // when a square is recomputed alone)
  int fwd_chunk, fwd_cta_pair, fwd_k_snake, fwd_band;   // the forward's product
                        // options, reused when the backward recomputes states
  int64_t n;
  int cur1[kMaxK];
  int d1_conv[kMaxK];
  int d1_layer[kMaxK];
  int plan_resp[kMaxK];
  int s1_exp_cur[kMaxK];   // exponent of the current 16-bit S1 copies
  int s1_exp_next[kMaxK];  // exponent the planned layer's epilogue writes with
  double n_occ, c_pt, c_d0;
  double eps1, epsN;
  double NS, NX;           // Tr S0 and ||S0||_F^2 of the current S0
  double froerr0;
  double s1_fro2[kMaxK];   // ||S1_k||_F^2 of the current S1_k
  double iderr[kMaxL + 2];
  double ns_hist[kMaxL + 2];   // N_S of each D0 layer (Alg. 2)
  double nx_hist[kMaxL + 2];   // N_X of each D0 layer
  double froerr1[kMaxK][kMaxL + 2];
  signed char sigma[kMaxL + 2];
};

// Product options of a forward run, kept in its control block so that the
// backward pass recomputes checkpointed states with the same launches.
struct FwdOpts {
  int ckpt_k, ckpt_slots, chunk, cta_pair, k_snake, band;
};

// Fields of a fresh control block (the block is zeroed first).
__device__ inline void state_init_fields(State* st, int k, int max_layers, int precision,
                                         double n_occ, double c_pt, double c_d0, int tape,
                                         int tape_base, int tape_states, int layout_k, int64_t n,
                                         int order, int k1, FwdOpts fo, int hole) {
  // complement form: the recursion converges to I - P, whose occupied levels
  // are the n - n_occ highest ones
  st->hole = hole;
  if (hole) n_occ = (double)n - n_occ;
  st->ckpt_k = fo.ckpt_k;
  st->ckpt_slots = fo.ckpt_slots;
  st->ckpt_pending = 0;
  st->adj_seg_a = 0;
  st->fwd_chunk = fo.chunk;
  st->fwd_cta_pair = fo.cta_pair;
  st->fwd_k_snake = fo.k_snake;
  st->fwd_band = fo.band;
  st->order = order;
  st->k1 = order >= 2 ? k1 : k;
  st->tape = tape;
  st->tape_base = tape_base;
  st->tape_states = tape_states;
  st->layout_k = layout_k;
  st->k_fwd = k;
  st->n = n;
  st->n_layer = 0;
  st->round_ctr = 0u;
  st->done = 0;
  st->status = DMPT_OK;
  st->timeout_flag = 0;
  st->k = k;
  st->max_layers = max_layers;
  st->precision = precision;
  st->n_occ = n_occ;
  st->c_pt = c_pt;
  st->c_d0 = c_d0;
  st->plan_square = 0;
  st->plan_write0 = 0;
  for (int j = 0; j < kMaxK; ++j) st->plan_resp[j] = 0;
}

// Workspace layout (byte offsets from the workspace base, 256-aligned).
struct Layout {
  int64_t n, Np;          // logical and padded size
  int k;                  // response slots (>= 1 when a tape is kept)
  int precision;
  int tape_states;        // 16-bit S0 copies kept for the adjoint (0: none)
  size_t elem;            // bytes per master element (8 or 4)
  size_t off_state, off_partials, off_master, off_ops16, off_vec, off_ckpt, total;
  int64_t partial_tiles;  // entries per job in the partials array
  int ckpt_slots;         // FP32 S0 checkpoints (Np x Np each; 0: none)
};

// pad: the internal size Np is n rounded up to a multiple of pad (256; 128
// for the batch path on 256 x 128 tiles).
Layout make_layout(int64_t n, int k, int precision, int tape_states = 0, int ckpt_slots = 0,
                   int pad = kPad);

// 16-bit operand slice of matrix m (0 = S0, 1 + j = S1_j) in ping-pong buffer
// `buf`, part 0 = hi, 1 = lo.  Tape slices follow the 4 (1 + k) ping-pong ones.
__host__ __device__ inline int zslice(int buf, int m, int part, int k) {
  return (buf * (1 + k) + m) * 2 + part;
}

// Upper-triangular tile count for block size bt.
inline int64_t upper_tiles(int64_t Np, int bt) {
  int64_t t = Np / bt;
  return t * (t + 1) / 2;
}

// ---- launchers (kernels_simt.cu) ----
cudaError_t launch_bounds(const double* H, int64_t n, int64_t ld, double* eps_out,
                          cudaStream_t s);
// first_m = 0: S0 and S1_1..k; first_m = 1: S1 only (response replay), each
// S1_j = -(H1_j + diag(shift_j)) / (eps_N - eps_1) (shift: k x n or NULL).
cudaError_t launch_init(const Layout& L, void* ws, const double* H, const double* H1,
                        int64_t ld, int k, int blocks, cudaStream_t s, int first_m = 0,
                        const double* shift = nullptr, int k_zero = 0);
// self-consistent response: v_j = gamma q_j;  q_j <- (1 - alpha) q_j + alpha diag(P1_j)
// with red[j] = {||diag(P1_j) - q_j||^2, ||diag(P1_j)||^2}
cudaError_t launch_scc_potential(const double* gamma, int64_t n, int64_t ld, const double* q,
                                 double* v, int k, cudaStream_t s);
cudaError_t launch_scc_mix(const double* P1, int64_t n, int64_t ld, double* q, int k,
                           double alpha, double* red, cudaStream_t s);
cudaError_t launch_decide(const Layout& L, void* ws, int mode, int64_t entries,
                          cudaStream_t s);
// Layer-product launchers.  *entries: partial-sum entries per job (tiles);
// *pass_flops: flops of one full-K, single-term pass over all tiles.
cudaError_t launch_layer_simt(const Layout& L, void* ws, cudaStream_t s, int64_t* entries,
                              double* pass_flops);
// 16-bit copies of the current masters of jobs first_job .. first_job + jobs - 1
// (jobs < 0: every job from first_job on)
cudaError_t launch_split(const Layout& L, void* ws, int first_job, cudaStream_t s, int jobs = -1);
// Checkpoints (ckpt_every >= 2): copy the current S0 master into its
// checkpoint slot when the last decide step asked for it (State::ckpt_pending).
cudaError_t launch_ckpt_store(const Layout& L, void* ws, cudaStream_t s);
// Backward with checkpoints: load checkpoint `c` (state a = c * ckpt_k) as the
// current S0 master (buffer 0) and the first tape state, and plan / finish
// the recompute of state m from state m - 1 (its 16-bit copies into tape slot
// m - a) with the forward's sigma_m.
cudaError_t launch_seg_load(const Layout& L, void* ws, int c, int a, cudaStream_t s);
// item_base: the forward launch's response items that preceded the square's
// (pair kernel), so that the square's tiles keep their rounds.
cudaError_t launch_recompute_plan(const Layout& L, void* ws, int m, int a, int64_t item_base,
                                  cudaStream_t s);
cudaError_t launch_recompute_done(const Layout& L, void* ws, cudaStream_t s);
// adjoint: Gbar = sym(G) into response slot 1 (upper triangle mirrored)
cudaError_t launch_adj_init(const Layout& L, void* ws, const double* G, int64_t ld, int blocks,
                            cudaStream_t s);
// dL/dH = -Gbar / (eps_N - eps_1)
cudaError_t launch_adj_finalize(const Layout& L, void* ws, double* dLdH, int64_t ld,
                                cudaStream_t s);
// P (if not NULL) and k_out response blocks from slots slot0 .. slot0 + k_out - 1
cudaError_t launch_finalize(const Layout& L, void* ws, double* P, double* P1,
                            int64_t ld, int k_out, cudaStream_t s, int slot0 = 1);
// The lower triangle of `count` n x n float64 matrices (row stride ld, one
// after another at n * ld) from their upper triangles.
cudaError_t launch_mirror_upper(double* M, int64_t n, int64_t ld, int count, cudaStream_t s);
cudaError_t launch_trivial(int64_t n, int k, int64_t ld, int full, double* P,
                           double* P1, cudaStream_t s);
int simt_tile(int precision);

// ---- tensor-core path (kernels_tc.cu) ----
// round_align: the pair kernel's producers keep their rounds in step (a
// bounded wait, never an error); off where several instances' layer kernels
// run at the same time, whose CTAs need not all be resident (dmpt_options::
// round_align; always off on the per-instance batch path).
cudaError_t launch_layer_tc(const Layout& L, void* ws, cudaStream_t s, double timeout_s,
                            int accum_chunk_k, int cta_pair, int k_snake, int band,
                            int64_t* entries, double* pass_flops, int inject_stall = 0,
                            int round_align = 1);
int tc_tile();

// ---- grouped layer products of a batch (kernels_tc.cu) ----
// One instance of a grouped launch: everything the pair kernel takes as
// arguments for a single instance, in device memory (the tensor map first;
// the struct takes the map's alignment).
struct GroupInst {
  CUtensorMap map;     // 3-D map over the instance's 16-bit operand slices
  CUtensorMap map64;   // the same slices in 64-row boxes (256 x 128 tiles)
  State* st;
  float* master;
  uint16_t* ops;
  double* partials;
  int64_t Np;
  int64_t ptiles;      // partial-sum entries per job
  int k;
  int npairs;          // CTA pairs a single-instance launch would use (K-snake rounds)
};
// Per-instance inputs of the batched decide kernel.
struct GroupDecide {
  State* st;
  const double* partials;
  int64_t ptiles;
  int64_t entries;
};
constexpr int kGroupMax = 1024;   // instances per grouped launch
// Dynamic item queue of a grouped launch: the leader CTA of each pair claims
// its next item from `counter` and publishes it in its ring of `slot`s, where
// the pair's other roles (MMA issuer, the peer CTA's producer, both CTAs'
// epilogues) read it.  A slot holds (epoch + 1) << 40 | (claim index / ring
// & 0xFF) << 32 | item (0xFFFFFFFF: no more items), so a stale value from an
// earlier launch or lap never matches.  The decide step after each grouped
// launch resets `counter` and advances `epoch`.
constexpr int kQueueRing = 64;     // claims a pair keeps in flight (>> its pipeline depth)
constexpr int kQueuePairs = 128;   // CTA pairs per grouped launch (<= 256 SMs)
struct GroupQueue {
  unsigned counter;
  unsigned epoch;
  unsigned pad[62];
  unsigned long long slot[kQueuePairs][kQueueRing];
};
// Fills `gi` for the instance whose workspace is `ws` (false: no tensor map);
// n128: also the 64-row map of the 256 x 128 tile kernel.
bool make_group_inst(const Layout& L, void* ws, int sm_count, GroupInst* gi, bool n128 = false);
// Partial-sum entries per job and the flops of one single-term pass of the
// pair kernel for layout L (n128: of the grouped 256 x 128 tile kernel).
void pair_tile_info(const Layout& L, int64_t* entries, double* pass_flops, bool n128 = false);
// One layer of every instance in `inst` (device array of `count`) in one
// launch; a bounded wait that expires sets *group_timeout.
// n128: 256 x 128 tiles (four 128-column accumulators; instances padded to a
// multiple of 128) instead of 256 x 256.
cudaError_t launch_layer_tc_group(const GroupInst* inst, int count, bool bf16, int* group_timeout,
                                  GroupQueue* queue, double timeout_s, int accum_chunk_k,
                                  int k_snake, int band, int sm_count, cudaStream_t s,
                                  bool n128 = false);
// Decide step of every instance (device array of `count`), one block each; a
// set *group_timeout marks every instance timed out.
cudaError_t launch_decide_group(const GroupDecide* args, int count, const int* group_timeout,
                                GroupQueue* queue, cudaStream_t s);

enum DecideMode {
  kDecideInit = 0,
  kDecideLayer = 1,
  kDecideAdjInit = 2,
  kDecideAdjLayer = 3,
  kDecideReplayInit = 4,
  kDecideReplayLayer = 5,
  kDecideAdjResume = 6    // adjoint: plan the pending layer after a segment reload
};

// batched solves: *flag = 1 when every instance's control block is done
cudaError_t launch_batch_all_done(const void* base, const long long* offs, int count, int* flag,
                                  cudaStream_t s);
// out[b] = the control block at base + offs[b], b < count (device arrays)
cudaError_t launch_gather_states(const void* base, const long long* offs, int count, State* out,
                                 cudaStream_t s);

// Batched set-up and outputs of the batch path: one launch per step of the
// initial layer (Alg. 1: bounds, S_0 and S_1 of Sec. III A, the first decide)
// and one for the outputs serve every active instance.  Each step splits its
// work into units (groups of kBatchRows rows for the bounds, the initial
// layer's blocks, chunks of kBatchChunk elements for the 16-bit split, 64 x 64
// tiles of one output matrix); first[s * (count + 1) + i] is the first unit
// of instance i in step s (exclusive prefix sums), so unit u belongs to the
// instance i with first[i] <= u < first[i + 1].  Every instance's values are those of
// its single-instance launches: the bounds are exact minima and maxima, the
// initial layer keeps its kInitBlocks virtual blocks (the ones without tile
// pairs only hold zero partial sums, which the set-up writes), and the split
// and the outputs are elementwise (the outputs through the same 64 x 64 tiles).
constexpr int kInitBlocks = 1024;   // blocks (partial-sum entries) of the initial layer
constexpr int kInitTile = 64;       // tile edge of the initial layer (Np is a multiple of 128)
constexpr int kBatchRows = 8;       // rows per warp of the batched bounds
constexpr int kBatchChunk = 4096;   // elements per block of the batched split
enum BatchStep { kBsRows = 0, kBsInit = 1, kBsSplit = 2, kBsOut = 3, kBsSteps = 4 };
struct BatchInst {
  State* st;
  void* master;        // FP32 (FP64 form: FP64) masters
  uint16_t* ops;       // 16-bit operand slices (dual forms)
  double* partials;
  const double* H;     // inputs, row stride ld
  const double* H1;
  double* P;           // outputs, row stride ld (P may be null when k > 0)
  double* P1;
  int64_t n, Np, ld, ptiles;
  double n_occ;
  int k, layout_k, hole;
  int init_blocks;     // initial-layer blocks that hold tile pairs (<= kInitBlocks)
};
// Per-batch fields of the fresh control blocks.
struct BatchCommon {
  int max_layers, precision;
  double c_pt, c_d0;
  FwdOpts fo;
};
// Units of each step for one instance (host and device agree on them).
__host__ __device__ inline int64_t batch_units(int step, int64_t n, int64_t Np, int k) {
  const int64_t tb = Np / kInitTile, pairs = tb * (tb + 1) / 2;
  switch (step) {
    case kBsRows: return (n + kBatchRows - 1) / kBatchRows;
    case kBsInit: return pairs < kInitBlocks ? pairs : kInitBlocks;
    case kBsSplit: return (int64_t)(1 + k) * ((Np * Np + kBatchChunk - 1) / kBatchChunk);
    default: return (int64_t)(1 + k) * ((n + 63) / 64) * ((n + 63) / 64);   // output tiles
  }
}
// Fresh control blocks, bounds keys and the zero partial sums of the
// initial layer's empty blocks; then the bounds, the initial layer, its
// decide step and (dual forms) the 16-bit split, each one launch over all
// `count` instances (device tables `bi`, `first`).
cudaError_t launch_batch_setup(const BatchInst* bi, const int64_t* first, int count,
                               const BatchCommon& c, const int64_t* units, bool dual, bool bf16,
                               cudaStream_t s);
// P, P1 of every instance (one launch).
cudaError_t launch_batch_finalize(const BatchInst* bi, const int64_t* first, int count,
                                  int64_t units, bool fp64, cudaStream_t s);

// CUDA device of a handle (-1 for NULL).
int handle_device(dmpt_handle h);
// Store `msg` as the handle's last error text (dmpt_last_error) and return s.
dmpt_status report(dmpt_handle h, dmpt_status s, const char* msg);

// State-dependent exponent for the 16-bit copies of S1: chosen so that a
// bound of the largest element maps to <= 2^14 (FP16 max is 65504).
constexpr int kFp16TargetExp = 14;

}  // namespace dmpt
