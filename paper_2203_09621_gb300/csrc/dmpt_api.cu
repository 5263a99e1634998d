// C ABI of libdmpt.so (declared in include/dmpt.h): argument checking,
// workspace carving and the host side of the layer loop of Algorithm 1.
//
// The host only issues launches.  Each layer is one product kernel (SIMT for
// FP64 / FP32, tcgen05 for the dual forms) followed by the one-block decide
// kernel that applies Algorithms 2 and 3 on the device.  Every
// `sync_every` layers the host reads the device "done" flag; launches that
// follow a finished run exit at once.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "dmpt_internal.cuh"

struct dmpt_ctx {
  int device = 0;
  int sm_count = 0;
  char err[512] = {0};
  std::vector<cudaEvent_t> events;   // timing pairs, created on first use
  std::vector<cudaStream_t> streams; // per-instance streams of batched solves
  std::vector<cudaEvent_t> joins;    // per-instance join events
  cudaStream_t origin = nullptr;     // capture / issue stream of batched solves
  cudaEvent_t fork = nullptr;
  // host-buffer pipeline: copy-in / copy-out streams and their events
  cudaStream_t copy_in = nullptr, copy_out = nullptr;
  cudaEvent_t ev_start = nullptr, ev_in[2] = {nullptr, nullptr}, ev_solved[2] = {nullptr, nullptr},
              ev_out[2] = {nullptr, nullptr}, ev_end[2] = {nullptr, nullptr};
  // autotuning: the winning layer-product configuration per (padded n, k,
  // precision), and the winning path per batch signature
  struct TuneEntry {
    int64_t Np;
    int k, precision;
    int cta_pair, tile_band, k_snake;
    double ms;
  };
  std::vector<TuneEntry> tune;
  struct BatchTune {
    std::vector<int64_t> Np;   // sorted padded sizes
    int k, precision;
    int path;                  // 0 grouped, 1 per-instance CTA pairs, 2 per-instance single
                               // CTAs, 3 grouped on 256 x 128 tiles
  };
  std::vector<BatchTune> batch_tune;
};

namespace {

using namespace dmpt;

dmpt_status fail(dmpt_handle h, dmpt_status s, const char* fmt, const char* what = "") {
  if (h) snprintf(h->err, sizeof(h->err), fmt, what);
  return s;
}

dmpt_status cuda_fail(dmpt_handle h, cudaError_t e, const char* where) {
  if (h) snprintf(h->err, sizeof(h->err), "%s: %s", where, cudaGetErrorString(e));
  return DMPT_ECUDA;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Per-layer histories of the stopping quantities of a finished run (entry
// n - 1 holds layer n): N_S, N_X and IdErr of Alg. 2 up to the D0 layer, and
// FroErr^(1) of Alg. 3 for each of `slots` response slots up to the layer
// whose test fired (`last_layer` for a slot that did not converge).
void fill_history(dmpt_info* info, const State& S, int slots, int last_layer) {
  const int d0 = S.d0_layer > 0 ? S.d0_layer : last_layer;
  for (int m = 1; m <= d0 && m <= DMPT_MAX_LAYERS; ++m) {
    info->n_s[m - 1] = S.ns_hist[m];
    info->n_x[m - 1] = S.nx_hist[m];
    info->iderr[m - 1] = S.iderr[m];
  }
  for (int j = 0; j < slots && j < DMPT_MAX_K; ++j) {
    const int last = S.d1_conv[j] ? S.d1_layer[j] : last_layer;
    for (int m = 1; m <= last && m <= DMPT_MAX_LAYERS; ++m)
      info->froerr1_hist[j][m - 1] = S.froerr1[j][m];
  }
}

// The complement form (dmpt_options::hole_form) for more occupied than empty levels.
int use_hole_form(const dmpt_options* o, int64_t n, int64_t n_occ) {
  return (o->hole_form == 1 && 2 * n_occ > n) ? 1 : 0;
}

bool valid_options(const dmpt_options* o) {
  if (o->precision < DMPT_FP64 || o->precision > DMPT_DUAL_BF16) return false;
  if (o->max_layers < 1 || o->max_layers > DMPT_MAX_LAYERS) return false;
  if (!(o->c_pt > 0.0) || !(o->c_d0 > 0.0)) return false;
  if (o->sync_every < 1) return false;
  // finite and capped: the device waits convert it to nanoseconds in 64 bits
  if (!(o->timeout_s > 0.0) || !(o->timeout_s <= DMPT_MAX_TIMEOUT_S)) return false;
  if (o->ckpt_every < 0 || o->ckpt_every > DMPT_MAX_LAYERS) return false;
  if (o->accum_chunk < 0) return false;
  if (o->cta_pair < 0 || o->cta_pair > 1) return false;
  if (o->k_snake < 0 || o->k_snake > 1) return false;
  if (o->order < 1 || o->order > DMPT_MAX_ORDER) return false;
  if (o->tile_band < 0 || o->tile_band > 1024) return false;
  if (o->inject_stall < 0 || o->inject_stall > 1) return false;
  if (o->autotune < 0 || o->autotune > 1) return false;
  if (o->round_align < 0 || o->round_align > 1) return false;
  if (o->hole_form < 0 || o->hole_form > 1) return false;
  if (o->group_tile_n != 128 && o->group_tile_n != 256) return false;
  return true;
}

// Workspace geometry for (n, k) under options o: response slots (at least
// one when S0 states are kept, for the adjoint) and tape capacity.
Layout layout_for(int64_t n, int k, const dmpt_options* o, int pad = kPad) {
  const int ck = o->ckpt_every;
  const int slots = o->order >= 2 ? o->order * k : ((ck >= 1 && k == 0) ? 1 : k);
  // ck = 1: every S0 state's 16-bit copies; ck >= 2: FP32 checkpoints of every
  // ck-th state plus a ck-state tape for the segment the backward recomputes
  const int tape_states = ck == 1 ? o->max_layers + 2 : (ck >= 2 ? ck : 0);
  const int ckpt_slots = ck >= 2 ? o->max_layers / ck + 1 : 0;
  return make_layout(n, slots, o->precision, tape_states, ckpt_slots, pad);
}

// The forward's product options, kept for the states the backward recomputes.
__global__ void state_init_kernel(State* st, int k, int max_layers, int precision, double n_occ,
                                  double c_pt, double c_d0, int tape, int tape_base,
                                  int tape_states, int layout_k, int64_t n, int order = 1,
                                  int k1 = 0, FwdOpts fo = FwdOpts{0, 0, 0, 1, 1, 8},
                                  int hole = 0) {
  state_init_fields(st, k, max_layers, precision, n_occ, c_pt, c_d0, tape, tape_base,
                    tape_states, layout_k, n, order, k1, fo, hole);
}

// Re-open a finished forward state for the adjoint run (keeps sigma, the
// bounds, the tape geometry and the number of S0 updates).
__global__ void adj_state_reset_kernel(State* st) {
  st->adj_seg_a = 0;
  st->item_base = 0;
  st->done = 0;
  st->status = DMPT_OK;
  st->timeout_flag = 0;
}

__global__ void replay_reset_kernel(State* st, int k) {
  st->item_base = 0;
  st->done = 0;
  st->status = DMPT_OK;
  st->timeout_flag = 0;
  st->k = k;
}

// Read the control block a forward run left in `workspace` and check that it
// holds an S0 tape of a converged dual-precision run of size n.
dmpt_status read_forward_state(dmpt_handle h, void* workspace, size_t ws_bytes, int64_t n,
                               cudaStream_t s, State* out, const char* who) {
  if (!workspace || ((uintptr_t)workspace) % 256 || ws_bytes < sizeof(State))
    return fail(h, DMPT_EWORKSPACE, "%s: workspace missing or misaligned", who);
  cudaError_t e = cudaMemcpyAsync(out, workspace, sizeof(State), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, who);
  if (out->tape != 1 || out->n != n || !out->done || out->d0_updates < 0 ||
      out->d0_updates + 1 > out->tape_states ||
      (out->precision != DMPT_DUAL_FP16 && out->precision != DMPT_DUAL_BF16))
    return fail(h, DMPT_EINVAL,
                "%s: the workspace holds no S0 tape of a dual-precision forward run of this n "
                "(run dmpt_sp2_response with ckpt_every = 1 first)", who);
  if (out->d0_layer < 1) return fail(h, DMPT_EINVAL, "%s: the forward run did not converge", who);
  const Layout L = make_layout(n, out->layout_k, out->precision, out->tape_states, out->ckpt_slots);
  if (ws_bytes < L.total) return fail(h, DMPT_EWORKSPACE, "%s: workspace too small", who);
  return DMPT_OK;
}

// The response recursion replayed over the stored S0 states for new
// perturbations H1_j (+ diag(shift_j)); writes P1 and fills info.
dmpt_status replay_run(dmpt_handle h, const Layout& L, const double* H1, const double* shift,
                       int k, int64_t ld, const dmpt_options* o, double* P1, dmpt_info* info,
                       void* workspace, cudaStream_t s) {
  State* st = (State*)workspace;
  cudaError_t e;
  const int blocks = kInitBlocks;
  replay_reset_kernel<<<1, 1, 0, s>>>(st, k);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "replay reset");
  if ((e = launch_init(L, workspace, nullptr, H1, ld, k, blocks, s, 1, shift)) != cudaSuccess)
    return cuda_fail(h, e, "replay init");
  if ((e = launch_decide(L, workspace, kDecideReplayInit, blocks, s)) != cudaSuccess)
    return cuda_fail(h, e, "replay decide");
  if ((e = launch_split(L, workspace, 1, s)) != cudaSuccess) return cuda_fail(h, e, "replay split");
  int launched = 0, done = 0;
  int64_t entries = 0;
  double pass_flops = 0.0;
  while (launched < o->max_layers && !done) {
    for (int j = 0; j < o->sync_every && launched < o->max_layers; ++j) {
      if ((e = launch_layer_tc(L, workspace, s, o->timeout_s, o->accum_chunk, o->cta_pair,
                               o->k_snake, o->tile_band, &entries, &pass_flops, 0,
                               o->round_align)) != cudaSuccess)
        return cuda_fail(h, e, "replay layer");
      if ((e = launch_decide(L, workspace, kDecideReplayLayer, entries, s)) != cudaSuccess)
        return cuda_fail(h, e, "replay decide");
      ++launched;
    }
    if ((e = cudaMemcpyAsync(&done, &st->done, sizeof(int), cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
      return cuda_fail(h, e, "replay poll");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(h, e, "replay loop");
  }
  if ((e = launch_finalize(L, workspace, nullptr, P1, ld, k, s)) != cudaSuccess)
    return cuda_fail(h, e, "replay finalize");
  State* hs = new State;
  e = cudaMemcpyAsync(hs, st, sizeof(State), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    delete hs;
    return cuda_fail(h, e, "replay state");
  }
  dmpt_status status = hs->done ? (dmpt_status)hs->status : DMPT_ENOTCONV;
  if (info) {
    memset(info, 0, sizeof(*info));
    info->status = status;
    info->layers = hs->rp_layers;
    info->d0_layer = hs->d0_layer;
    bool all1 = true;
    double alg = 0.0;
    for (int j = 0; j < k; ++j) {
      info->d1_layer[j] = hs->d1_layer[j];
      all1 = all1 && hs->d1_conv[j];
      const int last = hs->d1_conv[j] ? hs->d1_layer[j] : hs->rp_layers;
      info->froerr1[j] = (last >= 1 && last <= DMPT_MAX_LAYERS) ? hs->froerr1[j][last] : 0.0;
    }
    for (int m = 1; m <= hs->rp_layers; ++m) {
      int active = 0;
      for (int j = 0; j < k; ++j) active += (hs->d1_conv[j] ? m <= hs->d1_layer[j] : true) ? 1 : 0;
      alg += 3.0 * active * 2.0 * (double)L.n * L.n * L.n;
      info->mma_flops += active * 6.0 * pass_flops;
    }
    info->alg_flops = alg;
    info->converged = (status == DMPT_OK && all1) ? 1 : 0;
    info->eps_min = hs->eps1;
    info->eps_max = hs->epsN;
    info->froerr0 = hs->froerr0;
    info->product_launches = launched;
    for (int m = 1; m <= hs->rp_layers && m <= DMPT_MAX_LAYERS; ++m) info->sigma[m - 1] = hs->sigma[m];
    fill_history(info, *hs, k, hs->rp_layers);
    info->hole = hs->hole;
  }
  delete hs;
  if (status != DMPT_OK) return fail(h, status, "response replay: device status %s", "");
  return DMPT_OK;
}

// Algorithmic products of an order-o term, S0 S_o + S_o S0 + sum_{a=1}^{o-1}
// S_a S_{o-a}: S0 S_o (its transpose free), floor((o - 1) / 2) pairs
// S_a S_{o-a} + (S_a S_{o-a})^T, and for even o the square S_{o/2}^2.  In
// dual arithmetic a general product is 3 (A + B + C) and a square 2
// (A + B + B^T); in a plain form 1 each.
double term_products(int o, bool dual) {
  const double gen = dual ? 3.0 : 1.0, sq = dual ? 2.0 : 1.0;
  return gen * (1 + (o - 1) / 2) + (o % 2 == 0 ? sq : 0.0);
}

// active[o]: running terms of order o = 1 .. order
double layer_alg_flops(double n, int prec, bool square, const int* active, int order) {
  const bool dual = prec >= DMPT_DUAL_FP16;
  double p = square ? (dual ? 2.0 : 1.0) : 0.0;
  for (int od = 1; od <= order; ++od) p += term_products(od, dual) * active[od];
  return p * 2.0 * n * n * n;
}

// executed: an order-o term runs o + 1 full-K passes (3 MMAs each in dual)
double layer_mma_flops(const Layout& L, double per /* one full-K single-term pass */,
                       bool square, const int* active, int order) {
  const bool dual = L.precision >= DMPT_DUAL_FP16;
  double passes = square ? (dual ? 3.0 : 1.0) : 0.0;
  for (int od = 1; od <= order; ++od) passes += (od + 1) * (dual ? 3.0 : 1.0) * active[od];
  return passes * per;
}

}  // namespace

namespace dmpt {
int handle_device(dmpt_handle h) { return h ? h->device : -1; }

dmpt_status report(dmpt_handle h, dmpt_status s, const char* msg) {
  if (h) snprintf(h->err, sizeof(h->err), "%s", msg);
  return s;
}
}  // namespace dmpt

extern "C" {

void dmpt_default_options(dmpt_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = DMPT_DUAL_FP16;
  o->max_layers = 100;
  o->c_pt = 9.0;
  o->c_d0 = 4.5;
  o->operand_scaling = 1;
  o->sync_every = 4;
  o->timing = 0;
  o->timeout_s = 2.0;
  o->ckpt_every = 0;
  o->accum_chunk = 0;
  o->cta_pair = 1;
  o->k_snake = 1;
  o->order = 1;
  o->tile_band = 8;
  o->round_align = 1;
  o->hole_form = 1;
  o->group_tile_n = 256;
}

const char* dmpt_status_string(dmpt_status s) {
  switch (s) {
    case DMPT_OK: return "DMPT_OK";
    case DMPT_EINVAL: return "DMPT_EINVAL: invalid argument";
    case DMPT_EWORKSPACE: return "DMPT_EWORKSPACE: workspace missing, too small or misaligned";
    case DMPT_ENOTCONV: return "DMPT_ENOTCONV: layer cap reached before convergence";
    case DMPT_ENUMERIC: return "DMPT_ENUMERIC: non-finite value or empty spectral interval";
    case DMPT_ETIMEOUT: return "DMPT_ETIMEOUT: a device-side wait timed out";
    case DMPT_ECUDA: return "DMPT_ECUDA: CUDA error";
    case DMPT_EUNSUPPORTED: return "DMPT_EUNSUPPORTED: unsupported device or option";
  }
  return "unknown dmpt_status";
}

const char* dmpt_last_error(dmpt_handle h) { return h ? h->err : ""; }

dmpt_status dmpt_create(dmpt_handle* h, int device) {
  if (!h) return DMPT_EINVAL;
  *h = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
    return DMPT_EINVAL;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return DMPT_ECUDA;
  if (!(prop.major == 10 && prop.minor == 3)) return DMPT_EUNSUPPORTED;
  dmpt_ctx* c = new dmpt_ctx();
  c->device = device;
  c->sm_count = prop.multiProcessorCount;
  *h = c;
  return DMPT_OK;
}

dmpt_status dmpt_destroy(dmpt_handle h) {
  if (!h) return DMPT_EINVAL;
  {
    DeviceGuard g(h->device);
    for (cudaEvent_t e : h->events) cudaEventDestroy(e);
    for (cudaEvent_t e : h->joins) cudaEventDestroy(e);
    for (cudaStream_t st : h->streams) cudaStreamDestroy(st);
    if (h->origin) cudaStreamDestroy(h->origin);
    if (h->fork) cudaEventDestroy(h->fork);
    if (h->copy_in) cudaStreamDestroy(h->copy_in);
    if (h->copy_out) cudaStreamDestroy(h->copy_out);
    for (cudaEvent_t e : {h->ev_start, h->ev_in[0], h->ev_in[1], h->ev_solved[0], h->ev_solved[1],
                          h->ev_out[0], h->ev_out[1], h->ev_end[0], h->ev_end[1]})
      if (e) cudaEventDestroy(e);
  }
  delete h;
  return DMPT_OK;
}

size_t dmpt_workspace_size(int64_t n, int k, const dmpt_options* o) {
  dmpt_options d;
  dmpt_default_options(&d);
  if (!o) o = &d;
  if (n < 1 || k < 0 || k > DMPT_MAX_K || !valid_options(o)) return 0;
  if (o->order >= 2 && (o->order * k > DMPT_MAX_K || k < 1)) return 0;
  return layout_for(n, k, o).total;
}

dmpt_status dmpt_bounds(dmpt_handle h, const double* H, int64_t n, int64_t ld, double* eps,
                        void* stream) {
  if (!h) return DMPT_EINVAL;
  if (!H || !eps) return fail(h, DMPT_EINVAL, "dmpt_bounds: null pointer%s");
  if (n < 1 || ld < n) return fail(h, DMPT_EINVAL, "dmpt_bounds: need n >= 1 and ld >= n%s");
  if (((uintptr_t)eps) % 8) return fail(h, DMPT_EINVAL, "dmpt_bounds: eps not 8-byte aligned%s");
  DeviceGuard g(h->device);
  cudaError_t e = launch_bounds(H, n, ld, eps, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "dmpt_bounds");
  return DMPT_OK;
}

// Pk (order >= 2): the terms of orders 2 .. order, (order - 1) k blocks of n
// x n (ld), order o's block j at Pk + ((o - 2) k + j) n ld.
static dmpt_status forward_impl(dmpt_handle h, const double* H, const double* H1, int k,
                                int64_t n, int64_t ld, int64_t n_occ, const dmpt_options* o,
                                double* P, double* P1, double* Pk, dmpt_info* info,
                                void* workspace, size_t ws_bytes, void* stream) {
  const int order = o->order;
  if (info) memset(info, 0, sizeof(*info));
  if (k < 0 || k > DMPT_MAX_K) return fail(h, DMPT_EINVAL, "dmpt_sp2_response: k out of range%s");
  if (!H || (k > 0 && (!H1 || !P1)) || (k == 0 && !P))
    return fail(h, DMPT_EINVAL, "dmpt_sp2_response: null %s", "H/H1/P1/P");
  if (n < 1 || ld < n) return fail(h, DMPT_EINVAL, "dmpt_sp2_response: need n >= 1, ld >= n%s");
  if (n_occ < 0 || n_occ > n) return fail(h, DMPT_EINVAL, "dmpt_sp2_response: n_occ out of [0, n]%s");
  if (!valid_options(o)) return fail(h, DMPT_EINVAL, "dmpt_sp2_response: invalid options%s");
  if (order >= 2) {
    if (k < 1 || order * k > DMPT_MAX_K || !Pk)
      return fail(h, DMPT_EINVAL,
                  "dmpt_sp2_response_m: need k >= 1, order * k <= DMPT_MAX_K and Pk%s");
    if (o->ckpt_every != 0)
      return fail(h, DMPT_EUNSUPPORTED, "dmpt_sp2_response_m: orders >= 2 keep no tape%s");
  }
  if (o->ckpt_every != 0 && o->precision < DMPT_DUAL_FP16)
    return fail(h, DMPT_EUNSUPPORTED,
                "dmpt_sp2_response: the S0 tape / checkpoints (ckpt_every >= 1) need a dual "
                "precision%s");
  cudaStream_t s = (cudaStream_t)stream;
  DeviceGuard g(h->device);

  if (n_occ == 0 || n_occ == n) {
    cudaError_t e = launch_trivial(n, k, ld, n_occ == n, P, P1, s);
    if (e == cudaSuccess && order >= 2)
      e = launch_trivial(n, (order - 1) * k, ld, 0, nullptr, Pk, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "dmpt_sp2_response (trivial)");
    if (info) {
      info->status = DMPT_OK;
      info->converged = 1;
    }
    return DMPT_OK;
  }

  const Layout L = layout_for(n, k, o);
  if (!workspace) return fail(h, DMPT_EWORKSPACE, "dmpt_sp2_response: null workspace%s");
  if (((uintptr_t)workspace) % 256)
    return fail(h, DMPT_EWORKSPACE, "dmpt_sp2_response: workspace not 256-byte aligned%s");
  if (ws_bytes < L.total)
    return fail(h, DMPT_EWORKSPACE, "dmpt_sp2_response: workspace too small%s");
  const bool dual = o->precision >= DMPT_DUAL_FP16;

  char* base = (char*)workspace;
  State* st = (State*)(base + L.off_state);
  cudaError_t e = cudaMemsetAsync(st, 0, sizeof(State), s);
  if (e != cudaSuccess) return cuda_fail(h, e, "state reset");
  const FwdOpts fo{o->ckpt_every >= 2 ? o->ckpt_every : 0, L.ckpt_slots, o->accum_chunk,
                   o->cta_pair, o->k_snake, o->tile_band};
  state_init_kernel<<<1, 1, 0, s>>>(st, order >= 2 ? order * k : k, o->max_layers, o->precision,
                                    (double)n_occ, o->c_pt, o->c_d0, o->ckpt_every == 1 ? 1 : 0,
                                    4 * (1 + L.k), L.tape_states, L.k, n, order, k, fo,
                                    use_hole_form(o, n, n_occ));
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "state init");
  if ((e = launch_bounds(H, n, ld, &st->eps1, s)) != cudaSuccess) return cuda_fail(h, e, "bounds");
  const int init_blocks = kInitBlocks;
  if ((e = launch_init(L, workspace, H, H1, ld, k, init_blocks, s, 0, nullptr,
                       (order - 1) * k)) != cudaSuccess)
    return cuda_fail(h, e, "init");
  if ((e = launch_decide(L, workspace, kDecideInit, init_blocks, s)) != cudaSuccess)
    return cuda_fail(h, e, "decide(init)");
  const bool ckpt = o->ckpt_every >= 2;
  if (ckpt && (e = launch_ckpt_store(L, workspace, s)) != cudaSuccess)
    return cuda_fail(h, e, "checkpoint");
  if (dual && (e = launch_split(L, workspace, 0, s)) != cudaSuccess) return cuda_fail(h, e, "split");

  // events for per-launch timing of the layer products
  const int max_layers = o->max_layers;
  if (o->timing && (int)h->events.size() < 2 * max_layers) {
    while ((int)h->events.size() < 2 * max_layers) {
      cudaEvent_t ev;
      if ((e = cudaEventCreate(&ev)) != cudaSuccess) return cuda_fail(h, e, "event create");
      h->events.push_back(ev);
    }
  }

  int launched = 0;
  int64_t entries = 0;
  double pass_flops = 0.0;
  int done = 0;
  while (launched < max_layers && !done) {
    for (int j = 0; j < o->sync_every && launched < max_layers; ++j) {
      if (o->timing) cudaEventRecord(h->events[2 * launched], s);
      e = dual ? launch_layer_tc(L, workspace, s, o->timeout_s, o->accum_chunk, o->cta_pair,
                                 o->k_snake, o->tile_band, &entries, &pass_flops,
                                 o->inject_stall, o->round_align)
               : launch_layer_simt(L, workspace, s, &entries, &pass_flops);
      if (e != cudaSuccess) return cuda_fail(h, e, "layer product");
      if (o->timing) cudaEventRecord(h->events[2 * launched + 1], s);
      if ((e = launch_decide(L, workspace, kDecideLayer, entries, s)) != cudaSuccess)
        return cuda_fail(h, e, "decide(layer)");
      if (ckpt && (e = launch_ckpt_store(L, workspace, s)) != cudaSuccess)
        return cuda_fail(h, e, "checkpoint");
      ++launched;
    }
    if ((e = cudaMemcpyAsync(&done, &st->done, sizeof(int), cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
      return cuda_fail(h, e, "poll");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(h, e, "layer loop");
  }
  if ((e = launch_finalize(L, workspace, P, P1, ld, k, s)) != cudaSuccess)
    return cuda_fail(h, e, "finalize");
  for (int od = 2; od <= order; ++od)
    if ((e = launch_finalize(L, workspace, nullptr, Pk + (size_t)(od - 2) * k * n * ld, ld, k, s,
                             1 + (od - 1) * k)) != cudaSuccess)
      return cuda_fail(h, e, "finalize (higher orders)");

  State* host_state = new State;
  e = cudaMemcpyAsync(host_state, st, sizeof(State), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    delete host_state;
    return cuda_fail(h, e, "state readback");
  }
  dmpt_status status = (dmpt_status)host_state->status;
  if (!host_state->done) status = DMPT_ENOTCONV;
  if (info) {
    const State& S = *host_state;
    info->status = status;
    info->layers = S.layers_run;
    info->d0_layer = S.d0_layer;
    bool all1 = S.d0_conv != 0;
    const int kj = order >= 2 ? order * k : k;   // entries (o - 1) k .. o k - 1: order o
    for (int j = 0; j < kj; ++j) {
      info->d1_layer[j] = S.d1_layer[j];
      all1 = all1 && S.d1_conv[j];
      // last FroErr^(1) recorded for direction j
      const int last = S.d1_conv[j] ? S.d1_layer[j] : S.layers_run;
      info->froerr1[j] = (last >= 1 && last <= DMPT_MAX_LAYERS) ? S.froerr1[j][last] : 0.0;
    }
    info->converged = (status == DMPT_OK && all1) ? 1 : 0;
    info->eps_min = S.eps1;
    info->eps_max = S.epsN;
    info->froerr0 = S.froerr0;
    for (int m = 1; m <= S.layers_run && m <= DMPT_MAX_LAYERS; ++m) info->sigma[m - 1] = S.sigma[m];
    fill_history(info, S, kj, S.layers_run);
    info->hole = S.hole;
    info->product_launches = launched;
    double mma = 0.0, alg = 0.0;
    for (int m = 1; m <= S.layers_run; ++m) {
      const bool sq = S.d0_layer == 0 || m <= S.d0_layer;
      int active[DMPT_MAX_ORDER + 1] = {0};   // running terms per order
      for (int j = 0; j < kj; ++j)
        active[1 + j / (k > 0 ? k : 1)] += (S.d1_conv[j] ? m <= S.d1_layer[j] : true) ? 1 : 0;
      mma += layer_mma_flops(L, pass_flops, sq, active, order);
      alg += layer_alg_flops((double)n, o->precision, sq, active, order);
    }
    info->mma_flops = mma;
    info->alg_flops = alg;
    if (o->timing) {
      double total = 0.0;
      int timed = 0;
      for (int m = 0; m < S.layers_run && m < launched; ++m) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->events[2 * m], h->events[2 * m + 1]) == cudaSuccess) {
          total += ms;
          ++timed;
        }
      }
      info->ms_layers = total;
      info->timed_launches = timed;
    }
  }
  delete host_state;
  if (status == DMPT_ETIMEOUT) fail(h, status, "a device-side wait timed out%s");
  if (status == DMPT_ENUMERIC) fail(h, status, "non-finite values or eps_N <= eps_1%s");
  if (status == DMPT_ENOTCONV) fail(h, status, "max_layers reached%s");
  return status;
}

static const dmpt_ctx::TuneEntry* find_tune(dmpt_handle h, int64_t Np, int k, int precision) {
  for (const auto& x : h->tune)
    if (x.Np == Np && x.k == k && x.precision == precision) return &x;
  return nullptr;
}

dmpt_status dmpt_sp2_response(dmpt_handle h, const double* H, const double* H1, int k,
                              int64_t n, int64_t ld, int64_t n_occ, const dmpt_options* o,
                              double* P, double* P1, dmpt_info* info, void* workspace,
                              size_t ws_bytes, void* stream) {
  if (!h) return DMPT_EINVAL;
  h->err[0] = 0;
  dmpt_options defaults;
  dmpt_default_options(&defaults);
  if (!o) o = &defaults;
  if (info) memset(info, 0, sizeof(*info));
  if (o->order != 1)
    return fail(h, DMPT_EINVAL, "dmpt_sp2_response: o->order must be 1 (use dmpt_sp2_response2)%s");
  if (o->autotune && valid_options(o) && o->precision >= DMPT_DUAL_FP16 && n >= 1 &&
      n_occ > 0 && n_occ < n && k >= 0 && k <= DMPT_MAX_K) {
    const int64_t Np = layout_for(n, k, o).Np;
    const dmpt_ctx::TuneEntry* e = find_tune(h, Np, k, o->precision);
    if (!e) {
      const dmpt_status st = dmpt_autotune(h, H, H1, k, n, ld, n_occ, o, 0, P, P1, nullptr,
                                           nullptr, workspace, ws_bytes, stream);
      if (st != DMPT_OK) return st;
      e = find_tune(h, Np, k, o->precision);
      if (!e) return fail(h, DMPT_EINVAL, "dmpt_sp2_response: autotuning stored no entry%s");
    }
    dmpt_options t = *o;
    t.autotune = 0;
    t.cta_pair = e->cta_pair;
    t.tile_band = e->tile_band;
    t.k_snake = e->k_snake;
    return forward_impl(h, H, H1, k, n, ld, n_occ, &t, P, P1, nullptr, info, workspace, ws_bytes,
                        stream);
  }
  return forward_impl(h, H, H1, k, n, ld, n_occ, o, P, P1, nullptr, info, workspace, ws_bytes,
                      stream);
}

dmpt_status dmpt_autotune(dmpt_handle h, const double* H, const double* H1, int k, int64_t n,
                          int64_t ld, int64_t n_occ, const dmpt_options* o, int probe_layers,
                          double* P, double* P1, dmpt_options* best, double* best_layer_ms,
                          void* workspace, size_t ws_bytes, void* stream) {
  if (!h) return DMPT_EINVAL;
  h->err[0] = 0;
  dmpt_options defaults;
  dmpt_default_options(&defaults);
  if (!o) o = &defaults;
  if (!valid_options(o) || o->order != 1 || n < 1 || k < 0 || k > DMPT_MAX_K)
    return fail(h, DMPT_EINVAL, "dmpt_autotune: invalid arguments (first order only)%s");
  dmpt_options b = *o;
  b.autotune = 0;
  if (best) *best = b;
  if (best_layer_ms) *best_layer_ms = 0.0;
  if (o->precision < DMPT_DUAL_FP16 || n_occ <= 0 || n_occ >= n) return DMPT_OK;  // no candidates
  struct Cand {
    int pair, band;
  };
  static const Cand cands[] = {{1, 8}, {1, 0}, {1, 4}, {1, 16}, {0, 8}};
  dmpt_options t = b;
  t.max_layers = probe_layers > 0 ? probe_layers : 3;
  t.timing = 1;
  t.ckpt_every = 0;
  dmpt_info info;
  // warm-up: first launches of the kernels and tensor maps on this device
  dmpt_status st = forward_impl(h, H, H1, k, n, ld, n_occ, &t, P, P1, nullptr, &info, workspace,
                                ws_bytes, stream);
  if (st != DMPT_OK && st != DMPT_ENOTCONV) return st;
  double best_t = 1e300;
  Cand win = cands[0];
  for (const Cand& c : cands) {
    t.cta_pair = c.pair;
    t.tile_band = c.band;
    st = forward_impl(h, H, H1, k, n, ld, n_occ, &t, P, P1, nullptr, &info, workspace, ws_bytes,
                      stream);
    if (st != DMPT_OK && st != DMPT_ENOTCONV) return st;
    const double per = info.timed_launches > 0 ? info.ms_layers / info.timed_launches : 1e300;
    if (per < best_t) {
      best_t = per;
      win = c;
    }
  }
  h->err[0] = 0;   // the probes end at their layer cap by design
  const int64_t Np = layout_for(n, k, &b).Np;
  dmpt_ctx::TuneEntry e{Np, k, b.precision, win.pair, win.band, b.k_snake, best_t};
  bool stored = false;
  for (auto& x : h->tune)
    if (x.Np == Np && x.k == k && x.precision == b.precision) {
      x = e;
      stored = true;
    }
  if (!stored) h->tune.push_back(e);
  if (best) {
    best->cta_pair = win.pair;
    best->tile_band = win.band;
  }
  if (best_layer_ms) *best_layer_ms = best_t;
  return DMPT_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Bytes one instance's copy-in moves: the upper triangle of each matrix, in
// row blocks of DMPT_HOST_ROW_BLOCK rows from the block's diagonal onwards.
size_t dmpt_host_copy_in_bytes(int64_t n, int k) {
  if (n < 1 || k < 0 || k > DMPT_MAX_K) return 0;
  size_t per = 0;
  for (int64_t r0 = 0; r0 < n; r0 += DMPT_HOST_ROW_BLOCK) {
    const int64_t rows = n - r0 < DMPT_HOST_ROW_BLOCK ? n - r0 : DMPT_HOST_ROW_BLOCK;
    per += (size_t)rows * (size_t)(n - r0) * sizeof(double);
  }
  return per * (size_t)(1 + k);
}

size_t dmpt_workspace_size_host(int64_t n, int k, const dmpt_options* o) {
  const size_t ws = dmpt_workspace_size(n, k, o);
  if (!ws) return 0;
  const size_t io = align256((size_t)n * n * sizeof(double) * (1 + k));
  return align256(ws) + 4 * io;   // two input and two output buffer sets
}

dmpt_status dmpt_sp2_response_host(dmpt_handle h, int count, const double* const* H_host,
                                   const double* const* H1_host, int k, int64_t n,
                                   int64_t n_occ, const dmpt_options* o,
                                   double* const* P_host, double* const* P1_host,
                                   dmpt_info* info, void* workspace, size_t ws_bytes,
                                   void* stream) {
  if (!h) return DMPT_EINVAL;
  h->err[0] = 0;
  dmpt_options defaults;
  dmpt_default_options(&defaults);
  if (!o) o = &defaults;
  if (info)
    for (int i = 0; i < count; ++i) memset(&info[i], 0, sizeof(info[i]));
  if (count < 0 || k < 0 || k > DMPT_MAX_K || n < 1)
    return fail(h, DMPT_EINVAL, "dmpt_sp2_response_host: need count >= 0, 0 <= k <= DMPT_MAX_K, n >= 1%s");
  if (o->order != 1)
    return fail(h, DMPT_EINVAL, "dmpt_sp2_response_host: o->order must be 1%s");
  if (count == 0) return DMPT_OK;
  if (!H_host || (k > 0 && (!H1_host || !P1_host)) || (k == 0 && !P_host))
    return fail(h, DMPT_EINVAL, "dmpt_sp2_response_host: null %s", "pointer array");
  for (int i = 0; i < count; ++i)
    if (!H_host[i] || (k > 0 && (!H1_host[i] || !P1_host[i])) || (k == 0 && !P_host[i]))
      return fail(h, DMPT_EINVAL, "dmpt_sp2_response_host: null %s", "host buffer");
  const size_t ws = dmpt_workspace_size(n, k, o);
  if (!ws) return fail(h, DMPT_EINVAL, "dmpt_sp2_response_host: invalid options%s");
  if (!workspace || ((uintptr_t)workspace) % 256 || ws_bytes < dmpt_workspace_size_host(n, k, o))
    return fail(h, DMPT_EWORKSPACE, "dmpt_sp2_response_host: workspace too small or misaligned%s");
  DeviceGuard g(h->device);
  cudaError_t e = cudaSuccess;
  if (!h->copy_in) {
    if ((e = cudaStreamCreateWithFlags(&h->copy_in, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&h->copy_out, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(h, e, "copy stream create");
    for (cudaEvent_t* ev : {&h->ev_start, &h->ev_in[0], &h->ev_in[1], &h->ev_solved[0],
                            &h->ev_solved[1], &h->ev_out[0], &h->ev_out[1], &h->ev_end[0],
                            &h->ev_end[1]})
      if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(h, e, "copy event create");
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nn = (size_t)n * n;
  const size_t mat = nn * sizeof(double);
  const size_t io = align256(mat * (1 + k));
  char* bufs = (char*)workspace + align256(ws);
  double* in[2] = {(double*)bufs, (double*)(bufs + io)};
  double* out[2] = {(double*)(bufs + 2 * io), (double*)(bufs + 3 * io)};

  // the copies start after the caller's earlier work on `stream`
  if ((e = cudaEventRecord(h->ev_start, s)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(h->copy_in, h->ev_start, 0)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(h->copy_out, h->ev_start, 0)) != cudaSuccess)
    return cuda_fail(h, e, "copy ordering");
  // Instance i uses buffer set i % 2.  The copy-in of i + 1 is issued after
  // the solve of i - 1 has returned (forward_impl synchronises `stream`), so
  // the set it overwrites is no longer read.
  // Only the upper triangle (j >= i) of each matrix is copied: row blocks of
  // DMPT_HOST_ROW_BLOCK rows from the block's diagonal to the end of the row;
  // the solve's stream then fills the lower triangle from the upper one.
  auto copy_in = [&](int i) -> cudaError_t {
    double* d = in[i & 1];
    cudaError_t r = cudaSuccess;
    for (int m = 0; m <= k && r == cudaSuccess; ++m) {
      const double* src = m == 0 ? H_host[i] : H1_host[i] + (size_t)(m - 1) * nn;
      double* dst = d + (size_t)m * nn;
      for (int64_t r0 = 0; r0 < n && r == cudaSuccess; r0 += DMPT_HOST_ROW_BLOCK) {
        const int64_t rows = n - r0 < DMPT_HOST_ROW_BLOCK ? n - r0 : DMPT_HOST_ROW_BLOCK;
        const size_t off = (size_t)r0 * n + r0;
        r = cudaMemcpy2DAsync(dst + off, n * sizeof(double), src + off, n * sizeof(double),
                              (size_t)(n - r0) * sizeof(double), (size_t)rows,
                              cudaMemcpyHostToDevice, h->copy_in);
      }
    }
    if (r == cudaSuccess) r = cudaEventRecord(h->ev_in[i & 1], h->copy_in);
    return r;
  };
  dmpt_status status = DMPT_OK;
  if ((e = copy_in(0)) != cudaSuccess) status = cuda_fail(h, e, "copy in");
  for (int i = 0; i < count && status == DMPT_OK; ++i) {
    const int b = i & 1;
    if (i + 1 < count && (e = copy_in(i + 1)) != cudaSuccess) {
      status = cuda_fail(h, e, "copy in");
      break;
    }
    // inputs of i are on the device; the copy-out of i - 2 has left set b
    if ((e = cudaStreamWaitEvent(s, h->ev_in[b], 0)) != cudaSuccess ||
        (i >= 2 && (e = cudaStreamWaitEvent(s, h->ev_out[b], 0)) != cudaSuccess)) {
      status = cuda_fail(h, e, "copy ordering");
      break;
    }
    if ((e = launch_mirror_upper(in[b], n, n, 1 + k, s)) != cudaSuccess) {
      status = cuda_fail(h, e, "input mirror");
      break;
    }
    double* Pd = out[b];
    double* P1d = out[b] + nn;
    status = forward_impl(h, in[b], k > 0 ? in[b] + nn : nullptr, k, n, n, n_occ, o, Pd,
                          k > 0 ? P1d : nullptr, nullptr, info ? &info[i] : nullptr, workspace,
                          ws, s);
    if (status != DMPT_OK) break;
    if ((e = cudaEventRecord(h->ev_solved[b], s)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(h->copy_out, h->ev_solved[b], 0)) != cudaSuccess ||
        (P_host && P_host[i] &&
         (e = cudaMemcpyAsync(P_host[i], Pd, mat, cudaMemcpyDeviceToHost, h->copy_out)) !=
             cudaSuccess) ||
        (k > 0 && (e = cudaMemcpyAsync(P1_host[i], P1d, mat * k, cudaMemcpyDeviceToHost,
                                       h->copy_out)) != cudaSuccess) ||
        (e = cudaEventRecord(h->ev_out[b], h->copy_out)) != cudaSuccess) {
      status = cuda_fail(h, e, "copy out");
      break;
    }
  }
  // every copy has finished before the call returns; `stream` is ordered after them
  cudaError_t e1 = cudaEventRecord(h->ev_end[0], h->copy_in);
  cudaError_t e2 = cudaEventRecord(h->ev_end[1], h->copy_out);
  if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(s, h->ev_end[0], 0);
  if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s, h->ev_end[1], 0);
  cudaError_t e3 = cudaStreamSynchronize(s);
  if (status == DMPT_OK) {
    if (e1 != cudaSuccess) return cuda_fail(h, e1, "copy join");
    if (e2 != cudaSuccess) return cuda_fail(h, e2, "copy join");
    if (e3 != cudaSuccess) return cuda_fail(h, e3, "copy join");
  }
  return status;
}

dmpt_status dmpt_sp2_response_m(dmpt_handle h, const double* H, const double* H1, int k,
                                int64_t n, int64_t ld, int64_t n_occ, int order,
                                const dmpt_options* o, double* P, double* P1, double* Pk,
                                dmpt_info* info, void* workspace, size_t ws_bytes,
                                void* stream) {
  if (!h) return DMPT_EINVAL;
  h->err[0] = 0;
  if (info) memset(info, 0, sizeof(*info));
  if (order < 1 || order > DMPT_MAX_ORDER)
    return fail(h, DMPT_EINVAL, "dmpt_sp2_response_m: order out of [1, DMPT_MAX_ORDER]%s");
  dmpt_options opts;
  dmpt_default_options(&opts);
  if (o) opts = *o;
  opts.order = order;
  return forward_impl(h, H, H1, k, n, ld, n_occ, &opts, P, P1, Pk, info, workspace, ws_bytes,
                      stream);
}

dmpt_status dmpt_sp2_response2(dmpt_handle h, const double* H, const double* H1, int k,
                               int64_t n, int64_t ld, int64_t n_occ, const dmpt_options* o,
                               double* P, double* P1, double* P2, dmpt_info* info,
                               void* workspace, size_t ws_bytes, void* stream) {
  return dmpt_sp2_response_m(h, H, H1, k, n, ld, n_occ, 2, o, P, P1, P2, info, workspace,
                             ws_bytes, stream);
}

dmpt_status dmpt_sp2_backward(dmpt_handle h, const double* G, int64_t n, int64_t ld,
                              const dmpt_options* o, double* dLdH, void* workspace,
                              size_t ws_bytes, void* stream) {
  if (!h) return DMPT_EINVAL;
  h->err[0] = 0;
  dmpt_options defaults;
  dmpt_default_options(&defaults);
  if (!o) o = &defaults;
  if (!G || !dLdH) return fail(h, DMPT_EINVAL, "dmpt_sp2_backward: null %s", "G/dLdH");
  if (n < 1 || ld < n) return fail(h, DMPT_EINVAL, "dmpt_sp2_backward: need n >= 1, ld >= n%s");
  if (!valid_options(o)) return fail(h, DMPT_EINVAL, "dmpt_sp2_backward: invalid options%s");
  if (!workspace || ((uintptr_t)workspace) % 256 || ws_bytes < sizeof(State))
    return fail(h, DMPT_EWORKSPACE, "dmpt_sp2_backward: workspace missing or misaligned%s");
  cudaStream_t s = (cudaStream_t)stream;
  DeviceGuard g(h->device);
  cudaError_t e;
  State* st = (State*)workspace;
  State* hs = new State;
  e = cudaMemcpyAsync(hs, st, sizeof(State), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    delete hs;
    return cuda_fail(h, e, "dmpt_sp2_backward: state read");
  }
  const State fs = *hs;
  delete hs;
  const bool ckpt = fs.tape != 1 && fs.ckpt_k >= 2;
  const bool states_ok =
      fs.tape == 1 ? fs.d0_updates + 1 <= fs.tape_states
                   : (ckpt && fs.tape_states >= fs.ckpt_k && fs.d0_updates / fs.ckpt_k < fs.ckpt_slots);
  if (!states_ok || fs.n != n || !fs.done || fs.d0_updates < 0 ||
      (fs.precision != DMPT_DUAL_FP16 && fs.precision != DMPT_DUAL_BF16))
    return fail(h, DMPT_EINVAL,
                "dmpt_sp2_backward: the workspace holds no S0 tape or checkpoints of a "
                "dual-precision forward run of this n (run dmpt_sp2_response with ckpt_every >= 1 "
                "first)%s");
  if (fs.status != DMPT_OK)
    return fail(h, DMPT_EINVAL, "dmpt_sp2_backward: the forward run did not converge%s");
  const Layout L = make_layout(n, fs.layout_k, fs.precision, fs.tape_states, fs.ckpt_slots);
  if (ws_bytes < L.total) return fail(h, DMPT_EWORKSPACE, "dmpt_sp2_backward: workspace too small%s");

  const int blocks = 1024;
  adj_state_reset_kernel<<<1, 1, 0, s>>>(st);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "adjoint reset");
  if ((e = launch_adj_init(L, workspace, G, ld, blocks, s)) != cudaSuccess)
    return cuda_fail(h, e, "adjoint init");
  if ((e = launch_decide(L, workspace, kDecideAdjInit, blocks, s)) != cudaSuccess)
    return cuda_fail(h, e, "adjoint decide");
  if ((e = launch_split(L, workspace, 1, s)) != cudaSuccess) return cuda_fail(h, e, "adjoint split");
  int64_t entries = 0;
  double pass_flops = 0.0;
  const int U = fs.d0_updates;
  // without checkpoints the whole tape is one segment starting at state 0
  const int K = ckpt ? fs.ckpt_k : U + 1;
  int64_t rec_item_base = 0;
  if (ckpt && fs.fwd_cta_pair) {
    int64_t pt = 0;
    pair_tile_info(L, &pt, nullptr);   // 2 entries per pair tile
    rec_item_base = (int64_t)fs.k_fwd * (pt / 2);
  }
  for (int c = ckpt ? (U > 0 ? (U - 1) / K : 0) : 0; c >= 0; --c) {
    const int a = c * K;                       // first state of the segment
    const int b = U < a + K ? U : a + K;       // adjoint layers b .. a + 1 use states a .. b - 1
    if (ckpt) {
      // S_a from its checkpoint, then S_{a+1} .. S_{b-1} by the forward's own
      // square products (its sigma_m, 16-bit copies and product options)
      if ((e = launch_seg_load(L, workspace, c, a, s)) != cudaSuccess)
        return cuda_fail(h, e, "segment load");
      if ((e = launch_split(L, workspace, 0, s, 1)) != cudaSuccess)
        return cuda_fail(h, e, "segment split");
      for (int m = a + 1; m < b; ++m) {
        // in the forward's D0 layers all k_fwd response jobs ran, and their
        // items came before the square's in each launch
        if ((e = launch_recompute_plan(L, workspace, m, a, rec_item_base, s)) != cudaSuccess)
          return cuda_fail(h, e, "recompute plan");
        // no round alignment: the skipped leading items are never counted in
        if ((e = launch_layer_tc(L, workspace, s, o->timeout_s, fs.fwd_chunk, fs.fwd_cta_pair,
                                 fs.fwd_k_snake, fs.fwd_band, &entries, &pass_flops, 0,
                                 0)) != cudaSuccess)
          return cuda_fail(h, e, "recompute layer");
        if ((e = launch_recompute_done(L, workspace, s)) != cudaSuccess)
          return cuda_fail(h, e, "recompute done");
      }
      if ((e = launch_decide(L, workspace, kDecideAdjResume, 0, s)) != cudaSuccess)
        return cuda_fail(h, e, "adjoint decide");
    }
    for (int m = b; m >= a + 1; --m) {
      if ((e = launch_layer_tc(L, workspace, s, o->timeout_s, o->accum_chunk, o->cta_pair,
                               o->k_snake, o->tile_band, &entries, &pass_flops, 0,
                               o->round_align)) != cudaSuccess)
        return cuda_fail(h, e, "adjoint layer");
      if ((e = launch_decide(L, workspace, kDecideAdjLayer, entries, s)) != cudaSuccess)
        return cuda_fail(h, e, "adjoint decide");
    }
  }
  if ((e = launch_adj_finalize(L, workspace, dLdH, ld, s)) != cudaSuccess)
    return cuda_fail(h, e, "adjoint finalize");
  int status = 0;
  e = cudaMemcpyAsync(&status, &st->status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, "dmpt_sp2_backward");
  if (status != DMPT_OK) return fail(h, (dmpt_status)status, "dmpt_sp2_backward: device status%s");
  return DMPT_OK;
}

// Batch scratch: [state offsets, all-done flag] [GroupInst table]
// [GroupDecide table] [group timeout flag] [grouped item queue] [gathered
// control blocks], each 256-byte aligned.
static size_t batch_poll_bytes(int count) {
  return ((size_t)count * sizeof(long long) + 2 * sizeof(int) + 255) & ~size_t(255);
}
static size_t batch_ginst_bytes(int count) {
  return ((size_t)count * sizeof(GroupInst) + 255) & ~size_t(255);
}
static size_t batch_gdec_bytes(int count) {
  return ((size_t)count * sizeof(GroupDecide) + 255) & ~size_t(255);
}
static size_t batch_queue_bytes() { return (sizeof(GroupQueue) + 255) & ~size_t(255); }
static size_t batch_states_bytes(int count) {
  return ((size_t)count * sizeof(State) + 255) & ~size_t(255);
}
static size_t batch_binst_bytes(int count) {
  return ((size_t)count * sizeof(BatchInst) + 255) & ~size_t(255);
}
static size_t batch_first_bytes(int count) {
  return ((size_t)kBsSteps * (count + 1) * sizeof(int64_t) + 255) & ~size_t(255);
}
static size_t batch_scratch_bytes(int count) {
  return batch_poll_bytes(count) + batch_ginst_bytes(count) + batch_gdec_bytes(count) + 256 +
         batch_queue_bytes() + batch_states_bytes(count) + batch_binst_bytes(count) +
         batch_first_bytes(count);
}

size_t dmpt_workspace_size_batch(int count, const int64_t* n, int k, const dmpt_options* o) {
  dmpt_options d;
  dmpt_default_options(&d);
  if (!o) o = &d;
  if (count < 1 || !n || k < 0 || k > DMPT_MAX_K || !valid_options(o) || o->ckpt_every != 0)
    return 0;
  size_t total = batch_scratch_bytes(count);
  for (int i = 0; i < count; ++i) {
    if (n[i] < 1) return 0;
    total += (layout_for(n[i], k, o).total + 255) & ~size_t(255);
  }
  return total;
}

// path: -1 = the default rule (grouped launch for dual forms on CTA pairs),
// 0 = grouped, 1 = one launch per instance on its own stream, 3 = grouped on
// 256 x 128 tiles with the instances padded to a multiple of 128.
static dmpt_status batch_impl(dmpt_handle h, int count, const double* const* H,
                              const double* const* H1, int k, const int64_t* n,
                              const int64_t* ld, const int64_t* n_occ, const dmpt_options* o,
                              double* const* P, double* const* P1, dmpt_info* info,
                              void* workspace, size_t ws_bytes, void* stream, int path) {
  if (count < 1 || !H || !n || !ld || !n_occ || (k > 0 && (!H1 || !P1)) || (k == 0 && !P))
    return fail(h, DMPT_EINVAL, "dmpt_sp2_response_batch: bad arguments%s");
  if (k < 0 || k > DMPT_MAX_K || !valid_options(o) || o->ckpt_every != 0 || o->timing)
    return fail(h, DMPT_EINVAL, "dmpt_sp2_response_batch: bad k or options (no tape, no timing)%s");
  for (int i = 0; i < count; ++i) {
    if (!H[i] || n[i] < 1 || ld[i] < n[i] || n_occ[i] < 0 || n_occ[i] > n[i] ||
        (k > 0 && (!H1[i] || !P1[i])) || (k == 0 && !P[i]))
      return fail(h, DMPT_EINVAL, "dmpt_sp2_response_batch: bad instance%s");
  }
  const size_t need = dmpt_workspace_size_batch(count, n, k, o);
  if (!workspace || ((uintptr_t)workspace) % 256 || ws_bytes < need)
    return fail(h, DMPT_EWORKSPACE, "dmpt_sp2_response_batch: workspace missing or too small%s");
  if (info) memset(info, 0, sizeof(dmpt_info) * (size_t)count);
  DeviceGuard g(h->device);
  cudaError_t e;
  cudaStream_t caller = (cudaStream_t)stream;
  // streams and events (created once per handle, reused)
  while ((int)h->streams.size() < count) {
    cudaStream_t st;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(h, e, "batch stream");
    h->streams.push_back(st);
    cudaEvent_t ev;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(h, e, "batch event");
    h->joins.push_back(ev);
  }
  if (!h->origin && (e = cudaStreamCreateWithFlags(&h->origin, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(h, e, "batch origin stream");
  if (!h->fork && (e = cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(h, e, "batch fork event");
  const bool dual = o->precision >= DMPT_DUAL_FP16;

  // carve the workspace: [scratch: state offsets, all-done flag][instance 0][instance 1]...
  char* base = (char*)workspace;
  long long* d_offs = (long long*)base;
  int* d_flag = (int*)(base + (size_t)count * sizeof(long long));
  std::vector<Layout> L(count);
  std::vector<long long> offs(count);
  std::vector<int> active(count, 0);
  int n_act = 0;
  for (int i = 0; i < count; ++i) {
    active[i] = (n_occ[i] > 0 && n_occ[i] < n[i]) ? 1 : 0;
    n_act += active[i];
  }
  // dual precision on CTA pairs: one grouped launch per layer step for all
  // instances (GroupInst table, batched decide); otherwise one launch per
  // instance on its own stream
  const bool can_group = dual && o->cta_pair && o->order == 1 && n_act > 0 && n_act <= kGroupMax;
  // 256 x 128 tiles, padding to 128
  const bool n128 = (path == 3 || (path == -1 && o->group_tile_n == 128)) && can_group;
  size_t off = batch_scratch_bytes(count);
  for (int i = 0; i < count; ++i) {
    L[i] = layout_for(n[i], k, o, n128 ? 128 : kPad);
    offs[i] = (long long)off;
    off += (L[i].total + 255) & ~size_t(255);
  }
  // fork: the origin stream and every instance stream follow the caller's stream
  if ((e = cudaEventRecord(h->fork, caller)) != cudaSuccess) return cuda_fail(h, e, "batch fork");
  if ((e = cudaStreamWaitEvent(h->origin, h->fork, 0)) != cudaSuccess) return cuda_fail(h, e, "fork");
  // control blocks polled for completion: active (non-trivial) instances only
  std::vector<long long> act_offs;
  for (int i = 0; i < count; ++i)
    if (active[i]) act_offs.push_back(offs[i]);
  const int n_active = (int)act_offs.size();
  const bool grouped = path != 1 && can_group;
  GroupInst* d_ginst = (GroupInst*)(base + batch_poll_bytes(count));
  GroupDecide* d_gdec = (GroupDecide*)((char*)d_ginst + batch_ginst_bytes(count));
  int* d_gtimeout = (int*)((char*)d_gdec + batch_gdec_bytes(count));
  GroupQueue* d_gqueue = (GroupQueue*)((char*)d_gtimeout + 256);
  State* d_states = (State*)((char*)d_gqueue + batch_queue_bytes());
  BatchInst* d_binst = (BatchInst*)((char*)d_states + batch_states_bytes(count));
  int64_t* d_bfirst = (int64_t*)((char*)d_binst + batch_binst_bytes(count));
  // tables of the batched set-up and output launches (active instances, in
  // the order of d_offs)
  std::vector<BatchInst> bt(n_active > 0 ? n_active : 1);
  std::vector<int64_t> bfirst((size_t)kBsSteps * (n_active + 1), 0);
  int64_t units[kBsSteps] = {0, 0, 0, 0};
  for (int i = 0, a = 0; i < count; ++i) {
    if (!active[i]) continue;
    char* ws = base + offs[i];
    BatchInst& b = bt[a];
    b.st = (State*)(ws + L[i].off_state);
    b.master = ws + L[i].off_master;
    b.ops = (uint16_t*)(ws + L[i].off_ops16);
    b.partials = (double*)(ws + L[i].off_partials);
    b.H = H[i];
    b.H1 = k ? H1[i] : nullptr;
    b.P = P ? P[i] : nullptr;
    b.P1 = k ? P1[i] : nullptr;
    b.n = n[i];
    b.Np = L[i].Np;
    b.ld = ld[i];
    b.ptiles = L[i].partial_tiles;
    b.n_occ = (double)n_occ[i];
    b.k = k;
    b.layout_k = L[i].k;
    b.hole = use_hole_form(o, n[i], n_occ[i]);
    b.init_blocks = (int)batch_units(kBsInit, n[i], L[i].Np, k);
    for (int st = 0; st < kBsSteps; ++st) {
      const int64_t u = batch_units(st, n[i], L[i].Np, st == kBsSplit ? L[i].k : k);
      bfirst[(size_t)st * (n_active + 1) + a + 1] = bfirst[(size_t)st * (n_active + 1) + a] + u;
      units[st] += u;
    }
    ++a;
  }
  if (n_active > 0 &&
      ((e = cudaMemcpyAsync(d_offs, act_offs.data(), sizeof(long long) * n_active,
                            cudaMemcpyHostToDevice, h->origin)) != cudaSuccess ||
       (e = cudaMemcpyAsync(d_binst, bt.data(), sizeof(BatchInst) * n_active,
                            cudaMemcpyHostToDevice, h->origin)) != cudaSuccess ||
       (e = cudaMemcpyAsync(d_bfirst, bfirst.data(), sizeof(int64_t) * bfirst.size(),
                            cudaMemcpyHostToDevice, h->origin)) != cudaSuccess))
    return cuda_fail(h, e, "batch tables");
  std::vector<int64_t> entries(count, 0);
  std::vector<double> pass_flops(count, 0.0);
  auto issue_step = [&](int i) -> cudaError_t {
    cudaStream_t si = h->streams[i];
    void* ws = base + offs[i];
    // the instances' layer kernels run side by side: no round alignment
    cudaError_t r = dual ? launch_layer_tc(L[i], ws, si, o->timeout_s, o->accum_chunk,
                                           o->cta_pair, o->k_snake, o->tile_band, &entries[i],
                                           &pass_flops[i], 0, /*round_align=*/0)
                         : launch_layer_simt(L[i], ws, si, &entries[i], &pass_flops[i]);
    if (r != cudaSuccess) return r;
    return launch_decide(L[i], ws, kDecideLayer, entries[i], si);
  };
  int n_group = 0;
  if (grouped) {
    // instances by decreasing size, so the item pool starts with the longest tiles
    std::vector<int> order;
    for (int i = 0; i < count; ++i)
      if (active[i]) order.push_back(i);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return L[a].Np > L[b].Np; });
    std::vector<GroupInst> gi(order.size());
    std::vector<GroupDecide> gd(order.size());
    for (size_t j = 0; j < order.size(); ++j) {
      const int i = order[j];
      void* ws = base + offs[i];
      if (!make_group_inst(L[i], ws, h->sm_count, &gi[j], n128))
        return fail(h, DMPT_ECUDA, "dmpt_sp2_response_batch: %s", "tensor map encoding failed");
      pair_tile_info(L[i], &entries[i], &pass_flops[i], n128);
      gd[j].st = gi[j].st;
      gd[j].partials = gi[j].partials;
      gd[j].ptiles = gi[j].ptiles;
      gd[j].entries = entries[i];
    }
    n_group = (int)order.size();
    // copies from pageable memory return once the source is staged
    if ((e = cudaMemcpyAsync(d_ginst, gi.data(), sizeof(GroupInst) * gi.size(),
                             cudaMemcpyHostToDevice, h->origin)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_gdec, gd.data(), sizeof(GroupDecide) * gd.size(),
                             cudaMemcpyHostToDevice, h->origin)) != cudaSuccess ||
        (e = cudaMemsetAsync(d_gtimeout, 0, sizeof(int), h->origin)) != cudaSuccess ||
        (e = cudaMemsetAsync(d_gqueue, 0, sizeof(GroupQueue), h->origin)) != cudaSuccess)
      return cuda_fail(h, e, "batch group tables");
  }
  // instances with nothing to compute, then the initial layer of all others:
  // one launch per step for the whole batch
  for (int i = 0; i < count; ++i) {
    if (active[i]) continue;
    if ((e = launch_trivial(n[i], k, ld[i], n_occ[i] == n[i], P ? P[i] : nullptr,
                            k ? P1[i] : nullptr, h->origin)) != cudaSuccess)
      return cuda_fail(h, e, "batch trivial");
  }
  const BatchCommon common{o->max_layers, o->precision, o->c_pt, o->c_d0,
                           FwdOpts{0, 0, o->accum_chunk, o->cta_pair, o->k_snake, o->tile_band}};
  if ((e = launch_batch_setup(d_binst, d_bfirst, n_active, common, units, dual,
                              o->precision == DMPT_DUAL_BF16, h->origin)) != cudaSuccess)
    return cuda_fail(h, e, "batch initial layer");
  if (!grouped) {
    // the first layer of each instance on its own stream, joined into the origin stream
    if ((e = cudaEventRecord(h->fork, h->origin)) != cudaSuccess) return cuda_fail(h, e, "fork");
    for (int i = 0; i < count; ++i) {
      if (!active[i]) continue;
      if ((e = cudaStreamWaitEvent(h->streams[i], h->fork, 0)) != cudaSuccess)
        return cuda_fail(h, e, "fork");
      if ((e = issue_step(i)) != cudaSuccess) return cuda_fail(h, e, "batch first layer");
      if ((e = cudaEventRecord(h->joins[i], h->streams[i])) != cudaSuccess ||
          (e = cudaStreamWaitEvent(h->origin, h->joins[i], 0)) != cudaSuccess)
        return cuda_fail(h, e, "join");
    }
  }
  // one CUDA graph = one layer of every active instance, each on its own stream
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if ((e = cudaStreamBeginCapture(h->origin, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    return cuda_fail(h, e, "batch capture");
  cudaError_t ce = cudaEventRecord(h->fork, h->origin);
  if (grouped) {
    ce = launch_layer_tc_group(d_ginst, n_group, o->precision == DMPT_DUAL_BF16, d_gtimeout,
                               d_gqueue, o->timeout_s, o->accum_chunk, o->k_snake, o->tile_band,
                               h->sm_count, h->origin, n128);
    if (ce == cudaSuccess)
      ce = launch_decide_group(d_gdec, n_group, d_gtimeout, d_gqueue, h->origin);
  }
  for (int i = 0; i < count && ce == cudaSuccess && !grouped; ++i) {
    if (!active[i]) continue;
    ce = cudaStreamWaitEvent(h->streams[i], h->fork, 0);
    if (ce == cudaSuccess) ce = issue_step(i);
    if (ce == cudaSuccess) ce = cudaEventRecord(h->joins[i], h->streams[i]);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(h->origin, h->joins[i], 0);
  }
  e = cudaStreamEndCapture(h->origin, &graph);
  if (ce != cudaSuccess || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(h, ce != cudaSuccess ? ce : e, "batch capture");
  }
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(h, e, "batch instantiate");
  int steps = grouped ? 0 : 1, all_done = n_active == 0 ? 1 : 0;
  while (steps < o->max_layers && !all_done) {
    for (int j = 0; j < o->sync_every && steps < o->max_layers; ++j, ++steps) {
      if ((e = cudaGraphLaunch(exec, h->origin)) != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        return cuda_fail(h, e, "batch graph launch");
      }
    }
    if ((e = launch_batch_all_done(base, d_offs, n_active, d_flag, h->origin)) == cudaSuccess)
      e = cudaMemcpyAsync(&all_done, d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->origin);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->origin);
    if (e != cudaSuccess) {
      cudaGraphExecDestroy(exec);
      return cuda_fail(h, e, "batch poll");
    }
  }
  cudaGraphExecDestroy(exec);
  // every instance's outputs, then every control block in one copy and one
  // synchronisation
  if ((e = launch_batch_finalize(d_binst, d_bfirst, n_active, units[kBsOut],
                                 o->precision == DMPT_FP64, h->origin)) != cudaSuccess)
    return cuda_fail(h, e, "batch finalize");
  std::vector<State> hs(n_active > 0 ? n_active : 1);
  if (n_active > 0) {
    e = launch_gather_states(base, d_offs, n_active, d_states, h->origin);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hs.data(), d_states, sizeof(State) * n_active, cudaMemcpyDeviceToHost,
                          h->origin);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->origin);
    if (e != cudaSuccess) return cuda_fail(h, e, "batch state");
  }
  dmpt_status worst = DMPT_OK;
  int ia = 0;   // index among the active instances (the order of d_offs)
  for (int i = 0; i < count; ++i) {
    if (!active[i]) {
      if (info) {
        info[i].status = DMPT_OK;
        info[i].converged = 1;
      }
      continue;
    }
    const State& S = hs[ia++];
    const dmpt_status si = S.done ? (dmpt_status)S.status : DMPT_ENOTCONV;
    if (si != DMPT_OK && worst == DMPT_OK) worst = si;
    if (info) {
      dmpt_info& I = info[i];
      I.status = si;
      I.layers = S.layers_run;
      I.d0_layer = S.d0_layer;
      bool all1 = S.d0_conv != 0;
      for (int j = 0; j < k; ++j) {
        I.d1_layer[j] = S.d1_layer[j];
        all1 = all1 && S.d1_conv[j];
      }
      I.converged = (si == DMPT_OK && all1) ? 1 : 0;
      I.eps_min = S.eps1;
      I.eps_max = S.epsN;
      I.froerr0 = S.froerr0;
      I.product_launches = steps;
      double alg = 0.0;
      for (int m = 1; m <= S.layers_run; ++m) {
        const bool sq = S.d0_layer == 0 || m <= S.d0_layer;
        int act[2] = {0, 0};   // first-order terms only
        for (int j = 0; j < k; ++j) act[1] += (S.d1_conv[j] ? m <= S.d1_layer[j] : true) ? 1 : 0;
        alg += layer_alg_flops((double)n[i], o->precision, sq, act, 1);
        I.mma_flops += layer_mma_flops(L[i], pass_flops[i], sq, act, 1);
      }
      I.alg_flops = alg;
      for (int m = 1; m <= S.layers_run && m <= DMPT_MAX_LAYERS; ++m) I.sigma[m - 1] = S.sigma[m];
      fill_history(&I, S, k, S.layers_run);
      I.hole = S.hole;
    }
  }
  // the caller's stream continues after the batch
  if ((e = cudaEventRecord(h->fork, h->origin)) == cudaSuccess)
    e = cudaStreamWaitEvent(caller, h->fork, 0);
  if (e != cudaSuccess) return cuda_fail(h, e, "batch join");
  if (worst != DMPT_OK) return fail(h, worst, "dmpt_sp2_response_batch: an instance failed%s");
  return DMPT_OK;
}

dmpt_status dmpt_sp2_response_batch(dmpt_handle h, int count, const double* const* H,
                                    const double* const* H1, int k, const int64_t* n,
                                    const int64_t* ld, const int64_t* n_occ,
                                    const dmpt_options* o, double* const* P, double* const* P1,
                                    dmpt_info* info, void* workspace, size_t ws_bytes,
                                    void* stream) {
  if (!h) return DMPT_EINVAL;
  h->err[0] = 0;
  dmpt_options defaults;
  dmpt_default_options(&defaults);
  if (!o) o = &defaults;
  if (!(o->autotune && valid_options(o) && o->precision >= DMPT_DUAL_FP16 && o->order == 1 &&
        count >= 1 && n != nullptr))
    return batch_impl(h, count, H, H1, k, n, ld, n_occ, o, P, P1, info, workspace, ws_bytes,
                      stream, -1);
  // autotuned batch: the grouped launch on CTA pairs with 256 x 256 or
  // 256 x 128 tiles, or one launch per instance with 256 x 256 (CTA-pair) or
  // 128 x 256 (single-CTA) tiles; chosen once per batch signature by timing a
  // short probe of each
  std::vector<int64_t> sig(count);
  for (int i = 0; i < count; ++i) sig[i] = n[i] >= 1 ? make_layout(n[i], k, o->precision).Np : 0;
  std::sort(sig.begin(), sig.end());
  int path = -1;
  for (const auto& b : h->batch_tune)
    if (b.k == k && b.precision == o->precision && b.Np == sig) path = b.path;
  dmpt_options t = *o;
  t.autotune = 0;
  if (path < 0) {
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
      return cuda_fail(h, cudaGetLastError(), "batch autotune events");
    dmpt_options p = t;
    p.max_layers = 3;
    double best_ms = 1e300;
    for (int rep = 0; rep < 2; ++rep) {   // the first round warms every path up
      for (int cand = 0; cand < 4; ++cand) {
        p.cta_pair = cand == 2 ? 0 : 1;
        cudaEventRecord(e0, s);
        const dmpt_status st = batch_impl(h, count, H, H1, k, n, ld, n_occ, &p, P, P1, info,
                                          workspace, ws_bytes, stream,
                                          cand == 0 ? 0 : (cand == 3 ? 3 : 1));
        cudaEventRecord(e1, s);
        if (st != DMPT_OK && st != DMPT_ENOTCONV) {
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          return st;
        }
        float ms = 0.f;
        if (cudaEventSynchronize(e1) == cudaSuccess &&
            cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && rep == 1 && ms < best_ms) {
          best_ms = ms;
          path = cand;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (path < 0) path = 0;
    h->batch_tune.push_back({sig, k, o->precision, path});
    h->err[0] = 0;
  }
  t.cta_pair = path == 2 ? 0 : 1;
  return batch_impl(h, count, H, H1, k, n, ld, n_occ, &t, P, P1, info, workspace, ws_bytes, stream,
                    path == 0 ? 0 : (path == 3 ? 3 : 1));
}

dmpt_status dmpt_response_replay(dmpt_handle h, const double* H1, int k, int64_t n,
                                 int64_t ld, const dmpt_options* o, double* P1, dmpt_info* info,
                                 void* workspace, size_t ws_bytes, void* stream) {
  if (!h) return DMPT_EINVAL;
  h->err[0] = 0;
  dmpt_options defaults;
  dmpt_default_options(&defaults);
  if (!o) o = &defaults;
  if (info) memset(info, 0, sizeof(*info));
  if (!H1 || !P1) return fail(h, DMPT_EINVAL, "dmpt_response_replay: null %s", "H1/P1");
  if (n < 1 || ld < n || k < 1 || k > DMPT_MAX_K)
    return fail(h, DMPT_EINVAL, "dmpt_response_replay: bad n, ld or k%s");
  if (!valid_options(o)) return fail(h, DMPT_EINVAL, "dmpt_response_replay: invalid options%s");
  cudaStream_t s = (cudaStream_t)stream;
  DeviceGuard g(h->device);
  State fs;
  dmpt_status st = read_forward_state(h, workspace, ws_bytes, n, s, &fs, "dmpt_response_replay");
  if (st != DMPT_OK) return st;
  if (k > fs.layout_k)
    return fail(h, DMPT_EINVAL, "dmpt_response_replay: k exceeds the forward's response slots%s");
  const Layout L = make_layout(n, fs.layout_k, fs.precision, fs.tape_states, fs.ckpt_slots);
  return replay_run(h, L, H1, nullptr, k, ld, o, P1, info, workspace, s);
}

dmpt_status dmpt_scc_response(dmpt_handle h, const double* H1_ext, const double* gamma, int k,
                              int64_t n, int64_t ld, const dmpt_options* o, double tol,
                              int max_iter, double mixing, double* P1, dmpt_info* info,
                              int* iterations, double* residual, void* workspace,
                              size_t ws_bytes, void* stream) {
  if (!h) return DMPT_EINVAL;
  h->err[0] = 0;
  dmpt_options defaults;
  dmpt_default_options(&defaults);
  if (!o) o = &defaults;
  if (!H1_ext || !gamma || !P1) return fail(h, DMPT_EINVAL, "dmpt_scc_response: null %s", "input");
  if (n < 1 || ld < n || k < 1 || k > DMPT_MAX_K || max_iter < 1 || !(tol > 0.0) ||
      !(mixing > 0.0 && mixing <= 1.0))
    return fail(h, DMPT_EINVAL, "dmpt_scc_response: bad n, ld, k, tol, max_iter or mixing%s");
  if (!valid_options(o)) return fail(h, DMPT_EINVAL, "dmpt_scc_response: invalid options%s");
  cudaStream_t s = (cudaStream_t)stream;
  DeviceGuard g(h->device);
  State fs;
  dmpt_status st = read_forward_state(h, workspace, ws_bytes, n, s, &fs, "dmpt_scc_response");
  if (st != DMPT_OK) return st;
  if (k > fs.layout_k)
    return fail(h, DMPT_EINVAL, "dmpt_scc_response: k exceeds the forward's response slots%s");
  const Layout L = make_layout(n, fs.layout_k, fs.precision, fs.tape_states, fs.ckpt_slots);
  double* q = (double*)((char*)workspace + L.off_vec);
  double* v = q + (size_t)k * n;
  double* red = v + (size_t)k * n;
  cudaError_t e = cudaMemsetAsync(q, 0, (size_t)k * n * sizeof(double), s);
  if (e != cudaSuccess) return cuda_fail(h, e, "scc reset");
  double res = INFINITY;
  int it = 0;
  std::vector<double> hred(4 * (size_t)k);
  dmpt_info acc;
  memset(&acc, 0, sizeof(acc));
  for (it = 1; it <= max_iter; ++it) {
    // H1_eff = H1_ext + diag(gamma q_in)
    if (it > 1 && (e = launch_scc_potential(gamma, n, ld, q, v, k, s)) != cudaSuccess)
      return cuda_fail(h, e, "scc potential");
    dmpt_info ri;
    st = replay_run(h, L, H1_ext, it > 1 ? v : nullptr, k, ld, o, P1, &ri, workspace, s);
    if (st != DMPT_OK) return st;
    acc.alg_flops += ri.alg_flops;
    acc.mma_flops += ri.mma_flops;
    acc.product_launches += ri.product_launches;
    acc.layers = ri.layers;
    acc.d0_layer = ri.d0_layer;
    for (int j = 0; j < k; ++j) {
      acc.d1_layer[j] = ri.d1_layer[j];
      acc.froerr1[j] = ri.froerr1[j];
    }
    acc.eps_min = ri.eps_min;
    acc.eps_max = ri.eps_max;
    acc.froerr0 = ri.froerr0;
    // q_out = diag(P1); residual; q_in <- (1 - mixing) q_in + mixing q_out
    if ((e = launch_scc_mix(P1, n, ld, q, k, mixing, red, s)) != cudaSuccess)
      return cuda_fail(h, e, "scc mix");
    e = cudaMemcpyAsync(hred.data(), red, 4 * (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "scc residual");
    res = 0.0;
    for (int j = 0; j < k; ++j) {
      const double r = sqrt(hred[4 * j] / (hred[4 * j + 1] > 0.0 ? hred[4 * j + 1] : 1e-300));
      res = r > res ? r : res;
    }
    if (!(res == res)) return fail(h, DMPT_ENUMERIC, "dmpt_scc_response: non-finite residual%s");
    if (res < tol) break;
  }
  if (it > max_iter) it = max_iter;
  if (iterations) *iterations = it;
  if (residual) *residual = res;
  acc.status = res < tol ? DMPT_OK : DMPT_ENOTCONV;
  acc.converged = res < tol ? 1 : 0;
  if (info) *info = acc;
  if (res >= tol) return fail(h, DMPT_ENOTCONV, "dmpt_scc_response: max_iter reached%s");
  return DMPT_OK;
}

}  // extern "C"
