/*
 * dmpt.h -- C ABI of the GB300 (sm_103a) DNN-SP2-PT density-matrix response
 * library (libdmpt.so).
 *
 * Given a symmetric Hamiltonian H (orthogonal basis), K symmetric first-order
 * perturbations H1_k and an occupation count n_occ, the library computes the
 * zero-temperature density matrix P = theta(mu I - H) (Sec. II B,
 * Eq. (eq:theta)) and its first-order responses P1_k = dP(H + lambda H1_k)/
 * dlambda at lambda = 0 (Sec. III A, Eq. (eq:D_k) with k = 1) with the SP2
 * recursive Fermi-operator expansion in its deep-neural-network form
 * (Sec. II B, Eq. (LinTransf); Sec. III A, Eq. (S_n detailed), Eq. (dB)),
 * stopped by the parameter-free criteria of Algorithms 2 and 3
 * (Sec. IV A, Eq. (ConvCrit)).
 *
 * Conventions shared by every call:
 *  - Matrix arguments are DEVICE pointers owned by the caller, row-major,
 *    n x n with leading dimension ld >= n (elements), float64.  Inputs are
 *    assumed symmetric (not checked).  Stacks of K matrices are consecutive
 *    blocks with stride n * ld elements.
 *  - No call allocates device memory.  Scratch space is the caller's
 *    workspace (device pointer, at least dmpt_workspace_size() bytes,
 *    256-byte aligned); the library never frees it.
 *  - Work is issued on the caller's `stream` (a cudaStream_t passed as
 *    void*; NULL means the legacy default stream).
 *  - Every call returns a dmpt_status and never aborts the process.
 *    Argument errors are detected before any launch.  CUDA errors return
 *    DMPT_ECUDA; the text is available from dmpt_last_error().
 *  - The library only runs on an sm_103 device (GB300); other devices give
 *    DMPT_EUNSUPPORTED from dmpt_create().
 *  - Threads: a handle (its error text, events and internal streams) is
 *    used by one host thread at a time; separate handles, also on separate
 *    devices of one process, may be used from separate threads.  One-time
 *    per-device setup inside the library is thread-safe.
 */
#ifndef DMPT_H
#define DMPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DMPT_MAX_K 8        /* response slots per call: directions x order */
#define DMPT_MAX_ORDER 8    /* highest response order (k = 1)             */
#define DMPT_MAX_LAYERS 256 /* upper bound of dmpt_options.max_layers      */
#define DMPT_HOST_ROW_BLOCK 512 /* rows per copy of dmpt_sp2_response_host  */
#define DMPT_MAX_TIMEOUT_S 600.0 /* upper bound of dmpt_options.timeout_s  */

typedef enum {
  DMPT_OK = 0,
  DMPT_EINVAL = 1,        /* bad argument (null pointer, n < 1, ld < n, ...)  */
  DMPT_EWORKSPACE = 2,    /* workspace null, too small or misaligned          */
  DMPT_ENOTCONV = 3,      /* max_layers reached; last iterate written         */
  DMPT_ENUMERIC = 4,      /* non-finite value or empty spectral interval      */
  DMPT_ETIMEOUT = 5,      /* a device-side wait hit its time limit            */
  DMPT_ECUDA = 6,         /* CUDA runtime / driver error                      */
  DMPT_EUNSUPPORTED = 7   /* device or option not supported                   */
} dmpt_status;

/* Arithmetic of the layer products (Sec. II C, Eq. (DualMat2),
 * Eq. (S0 tensor core); Sec. III D, Eq. (S0S1 tensor core)).
 *  DMPT_FP64:      FP64 masters, FP64 SIMT products.
 *  DMPT_FP32:      FP32 masters, FP32 SIMT products ("GPU-only" form).
 *  DMPT_DUAL_FP16: FP32 masters split into FP16 hi + lo, products
 *                  hi*hi + hi*lo + lo*hi on tcgen05 tensor cores with FP32
 *                  accumulation (lo*lo dropped).
 *  DMPT_DUAL_BF16: same with BF16 halves. */
typedef enum {
  DMPT_FP64 = 0,
  DMPT_FP32 = 1,
  DMPT_DUAL_FP16 = 2,
  DMPT_DUAL_BF16 = 3
} dmpt_precision;

typedef struct {
  int precision;        /* dmpt_precision                                     */
  int max_layers;       /* layer cap, 1..DMPT_MAX_LAYERS (default 100)        */
  double c_pt;          /* C_pt of Eq. (ConvCrit) / Alg. 3 (default 9.0)     */
  double c_d0;          /* factor of the Alg. 2 test (default 4.5)            */
  int operand_scaling;  /* 1: exact power-of-two scaling of the 16-bit halves
                           (FP16 range); 0: none (default 1)                  */
  int sync_every;       /* layers issued between host polls of the device
                           state (default 4)                                  */
  int timing;           /* 1: time every layer-product launch with CUDA events
                           on `stream` and report it in dmpt_info             */
  double timeout_s;     /* limit of any device-side spin wait, in seconds,
                           0 < timeout_s <= DMPT_MAX_TIMEOUT_S (default 2.0)  */
  int ckpt_every;       /* S0 states kept in the workspace for the adjoint
                           (dual forms; dmpt_sp2_backward):
                           0: none (default);
                           1: the 16-bit copies of every S0 layer state (the
                              full tape; also what dmpt_response_replay and
                              dmpt_scc_response read);
                           k >= 2 (<= DMPT_MAX_LAYERS): the FP32 master of
                              every k-th S0 state (a checkpoint) plus the
                              branch sequence; the backward recomputes each
                              segment of k states from its checkpoint with
                              the forward's own layer products before running
                              its adjoint layers (bit-identical states)       */
  int accum_chunk;      /* dual forms: K elements summed per tensor-memory
                           accumulator before the running sum is carried in
                           FP32 on the CUDA cores (0: default 256)             */
  int cta_pair;         /* dual forms: 1 = products on CTA pairs (cta_group::2,
                           256 x 256 tiles, default), 0 = one CTA per
                           128 x 256 tile                                      */
  int k_snake;          /* CTA-pair form: 1 = alternate the K-sweep direction
                           between scheduling rounds for L2 reuse (default 1) */
  int order;            /* response order the workspace is sized for: 1
                           (default); m for dmpt_sp2_response_m (2 for
                           dmpt_sp2_response2)                                */
  int tile_band;        /* CTA-pair form: tile order in bands of this many
                           256-column blocks, row-major inside a band (L2 reuse
                           of operand panels); 0 = column-major (default 8)   */
  int inject_stall;     /* test hook for the failure path (dual forms): 1 makes
                           the layer product wait on a barrier nothing arrives
                           on, so its bounded waits expire and the call returns
                           DMPT_ETIMEOUT after about timeout_s; 0 (default)    */
  int autotune;         /* dual forms: 1 = take cta_pair, tile_band and k_snake
                           from the handle's tuning table (see dmpt_autotune),
                           tuning on first use of a (padded n, k, precision)
                           with the call's own inputs; in a batch, choose the
                           grouped or per-instance path the same way.  0
                           (default) = use the fields as given              */
  int round_align;      /* CTA-pair form: 1 (default) = the CTAs' operand
                           loads keep their scheduling rounds in step (a
                           bounded wait of at most 300 us, never an error), so
                           the tiles of a round share their operand panels in
                           L2; 0 = off, for several solves running at once on
                           one GPU (their CTAs need not all be resident)      */
  int hole_form;        /* 1 (default): when n_occ > n / 2, run the recursion
                           on the complement Q = I - P (the n - n_occ highest
                           levels: S_0 = (H - eps_1 I) / (eps_N - eps_1),
                           S1_0 = +H1 / (eps_N - eps_1)) and return P = I - Q,
                           P_o = -Q_o; in exact arithmetic the same layers
                           with every sigma negated (barring exact ties), but
                           the 16-bit operands then carry ||I - P||_F =
                           sqrt(n - n_occ) instead of sqrt(n_occ), which keeps
                           the rounding of the products small next to the
                           response when few levels are empty; 0: always the
                           recursion on P as printed                         */
  int group_tile_n;     /* batches on the grouped kernel: tile width 256
                           (default: 256 x 256 pair tiles, instances padded to
                           a multiple of 256) or 128 (256 x 128 tiles, four
                           tensor-memory accumulators, instances padded to a
                           multiple of 128)                                   */
} dmpt_options;

/* Filled on the host by dmpt_sp2_response (when info != NULL). */
typedef struct {
  int status;                        /* same as the return value             */
  int layers;                        /* last layer n run                     */
  int d0_layer;                      /* layer at which Alg. 2 fired          */
  int converged;                     /* 1 if Alg. 2 and every Alg. 3 fired   */
  int d1_layer[DMPT_MAX_K];          /* layer at which Alg. 3 fired, per k   */
  double eps_min, eps_max;           /* Gershgorin bounds used (Alg. 1)      */
  double froerr0;                    /* FroErr^(0) of Alg. 2                 */
  double froerr1[DMPT_MAX_K];        /* last FroErr^(1)_n of Alg. 3, per k   */
  double ms_layers;                  /* summed device time of the layer
                                        products (timing = 1), else 0        */
  int product_launches;              /* layer-product kernel launches        */
  int timed_launches;                /* launches covered by ms_layers        */
  double mma_flops;                  /* flops issued by the layer products   */
  double alg_flops;                  /* algorithmic flops: (2 + 3K) 2n^3 per
                                        D0 layer, 3K 2n^3 per D1-only layer
                                        (Eq. (flop rate formula), 2/FMA)     */
  signed char sigma[DMPT_MAX_LAYERS];/* sigma_1..sigma_layers                */
  /* Per-layer histories of the quantities the stopping rules test (entry
   * n - 1 holds layer n; 0 where a quantity was not formed at that layer),
   * so that a caller can re-check every decision against Alg. 1-3:
   *   n_s, n_x, iderr  layers 1 .. d0_layer: N_S = Tr S_{n-1}, N_X =
   *                    Tr S_{n-1}^2 (as ||S_{n-1}||_F^2) and IdErr_n =
   *                    N_S - N_X of Alg. 2, in FP64, as the device used them;
   *   froerr1_hist     per response slot, the FroErr^(1)_n of Alg. 3 at each
   *                    layer 1 .. d1_layer[j] (1 .. layers when the slot did
   *                    not converge) at which the response ran; the test of
   *                    Alg. 3 reads it from d0_layer on. */
  double n_s[DMPT_MAX_LAYERS];
  double n_x[DMPT_MAX_LAYERS];
  double iderr[DMPT_MAX_LAYERS];
  double froerr1_hist[DMPT_MAX_K][DMPT_MAX_LAYERS];
  int hole;                          /* 1: the run used the complement form
                                        (hole_form); sigma, N_S and N_X are
                                        then those of the recursion on I - P */
} dmpt_info;

typedef struct dmpt_ctx* dmpt_handle;

/* Create a context on CUDA device `device` (made current for the call).
 * Checks that the device is sm_103.  *h receives the handle. */
dmpt_status dmpt_create(dmpt_handle* h, int device);
dmpt_status dmpt_destroy(dmpt_handle h);

/* Fill `o` with the defaults listed in dmpt_options. */
void dmpt_default_options(dmpt_options* o);

const char* dmpt_status_string(dmpt_status s);
/* Last error text of this handle (never NULL; "" when none). */
const char* dmpt_last_error(dmpt_handle h);

/* Bytes of workspace dmpt_sp2_response needs for (n, k, o->precision);
 * 0 for invalid arguments. */
size_t dmpt_workspace_size(int64_t n, int k, const dmpt_options* o);

/* Gershgorin spectral bounds of H (Sec. II B; Alg. 1 inputs eps_1, eps_N):
 *   eps[0] = min_i (H_ii - sum_{j != i} |H_ij|),
 *   eps[1] = max_i (H_ii + sum_{j != i} |H_ij|),
 * computed in FP64 on the device.  `eps` is a device pointer to 2 doubles.
 * Asynchronous on `stream`. */
dmpt_status dmpt_bounds(dmpt_handle h, const double* H, int64_t n, int64_t ld,
                        double* eps, void* stream);

/* Density matrix and first-order responses by DNN-SP2-PT (Algorithms 1-3).
 *   H      device, n x n (ld), float64, symmetric.
 *   H1     device, k blocks of n x n (ld), float64, each symmetric.
 *   k      0..DMPT_MAX_K directions sharing one S_0 recursion (each has its
 *          own Alg. 3 test and stops independently); k = 0 computes P only
 *          (H1 and P1 may then be NULL, P must not).
 *   n_occ  0..n.  n_occ = 0 or n gives P = 0 or I and P1 = 0 at once.
 *   o      options (NULL: defaults).
 *   P      device n x n (ld) output, may be NULL.
 *   P1     device, k blocks n x n (ld) outputs.
 *   info   host pointer, may be NULL.
 *   workspace / ws_bytes: caller scratch of dmpt_workspace_size() bytes.
 * The call issues all work on `stream` and synchronises that stream every
 * o->sync_every layers to read the convergence flag; it returns when the
 * outputs are written.  Returns DMPT_ENOTCONV (outputs = last iterate) when
 * max_layers is reached, DMPT_ENUMERIC on non-finite values or
 * eps_N <= eps_1 for 0 < n_occ < n.  With o->ckpt_every = 1 the workspace
 * (sized by dmpt_workspace_size with the same options) also keeps every S0
 * layer state for dmpt_sp2_backward. */
dmpt_status dmpt_sp2_response(dmpt_handle h, const double* H, const double* H1,
                              int k, int64_t n, int64_t ld, int64_t n_occ,
                              const dmpt_options* o, double* P, double* P1,
                              dmpt_info* info, void* workspace, size_t ws_bytes,
                              void* stream);

/* Second-order response as well (Sec. III A, Eq. (S_n detailed) with k = 2;
 * Eq. (eq:D_k): D^(2) = (1/2) d^2 P / dlambda^2 for H(lambda) = H + lambda H1):
 *   S2_0 = 0,  S2_n = sigma_n (S0 S2 + S1 S1 + S2 S0) + (1 - sigma_n) S2,
 * each dual product on the tensor cores (passes S0 S2, S2 S0, S1 S1 into one
 * accumulator).  The paper states stopping criteria for orders 0 and 1 only;
 * each S2_j stops by the test of Alg. 3 applied to its own idempotency error
 * ||S2 - (S0 S2 + S1 S1 + S2 S0)||_F (same C_pt and FroErr^(0)).
 *   Same arguments as dmpt_sp2_response plus P2 (device, k blocks n x n,
 *   ld); 1 <= k <= DMPT_MAX_K / 2; any precision, no tape.  The workspace
 *   is dmpt_workspace_size(n, k, o) with o->order = 2.  In info, entries
 *   k .. 2k-1 of d1_layer / froerr1 are those of the second-order terms. */
dmpt_status dmpt_sp2_response2(dmpt_handle h, const double* H, const double* H1, int k,
                               int64_t n, int64_t ld, int64_t n_occ, const dmpt_options* o,
                               double* P, double* P1, double* P2, dmpt_info* info,
                               void* workspace, size_t ws_bytes, void* stream);

/* Responses of every order up to m (Sec. III A, Eq. (S_n detailed); Sec.
 * III B: P_o = D^(o), the lambda^o Taylor coefficient of theta(mu - H -
 * lambda H1), i.e. (1/o!) d^o P / dlambda^o).  With S_o,0 = 0 for o >= 2
 * (a linear perturbation):
 *   S_o,n = sigma_n (S0 S_o + S_o S0 + sum_{a=1}^{o-1} S_a S_{o-a})
 *           + (1 - sigma_n) S_o,
 * all terms from the states at the start of the layer, each term's
 * products accumulated on the tensor cores in o + 1 K passes.  Each S_o
 * stops by the test of Alg. 3 applied to its own idempotency error (the
 * reading dmpt_sp2_response2 takes for order 2).
 *   order  1 .. DMPT_MAX_ORDER, with order * k <= DMPT_MAX_K; order 1 is
 *          dmpt_sp2_response (Pk unused), order 2 is dmpt_sp2_response2.
 *   Pk     device, the terms of orders 2 .. order: (order - 1) k blocks of
 *          n x n (ld), order o's direction j at Pk + ((o - 2) k + j) n ld.
 *   Other arguments as dmpt_sp2_response; every precision, no tape for
 *   order >= 2 (the FP32 / FP64 forms run the same passes on the CUDA cores).  The workspace is dmpt_workspace_size(n, k, o) with
 *   o->order = order.  In info, entries (o - 1) k .. o k - 1 of d1_layer /
 *   froerr1 are those of order o.  Errors: DMPT_EINVAL for an order outside
 *   [1, DMPT_MAX_ORDER], order * k > DMPT_MAX_K or a null Pk;
 *   DMPT_EUNSUPPORTED for order >= 2 with a tape (o->ckpt_every). */
dmpt_status dmpt_sp2_response_m(dmpt_handle h, const double* H, const double* H1, int k,
                                int64_t n, int64_t ld, int64_t n_occ, int order,
                                const dmpt_options* o, double* P, double* P1, double* Pk,
                                dmpt_info* info, void* workspace, size_t ws_bytes,
                                void* stream);

/* Adjoint of the S0 recursion: the gradient of L = Tr[G P] with respect to H
 * for the P of the preceding dmpt_sp2_response call that used `workspace`
 * with o->ckpt_every >= 1 and a dual precision.  The paper has no backward
 * pass; this is the reverse mode of its layer map (Sec. II B, Eq. (eq:Sn)):
 *   Gbar_U = (G + G^T)/2,
 *   Gbar_{m-1} = sigma_m (S_{m-1} Gbar_m + Gbar_m S_{m-1}) + (1 - sigma_m) Gbar_m
 * over the U layers that updated S0 (newest first), each a response-type
 * layer product on the tensor cores with the stored S_{m-1}, and
 *   dL/dH = -Gbar_0 / (eps_N - eps_1),
 * with the branch choices and the Gershgorin bounds held fixed (piecewise
 * constant in H).  At convergence this equals the first-order response to
 * the perturbation G (the Daleckii-Krein derivative is self-adjoint).
 *   G      device n x n (ld), float64 (need not be symmetric).
 *   o      options for the products (precision is taken from the forward).
 *   dLdH   device n x n (ld) output, float64, symmetric.
 * With checkpoints (ckpt_every = k >= 2) the states S_{ck} .. S_{ck+k-1} of
 * each segment, newest segment first, are recomputed from the stored S_{ck}
 * by the forward's square products (its branch choices, its 16-bit copies,
 * its product options) into a k-state buffer, and the segment's adjoint
 * layers run on them: about U extra squares for a tape of U / k + k states
 * instead of U + 1.
 * The forward's response slots are reused as scratch; the S0 tape (or the
 * checkpoints) is left intact, so several backward calls may follow one
 * forward call.  Returns
 * DMPT_EINVAL when the workspace holds no tape of a converged forward run of
 * this n.  Synchronises `stream` once at entry (to read the forward state)
 * and once at exit. */
dmpt_status dmpt_sp2_backward(dmpt_handle h, const double* G, int64_t n, int64_t ld,
                              const dmpt_options* o, double* dLdH, void* workspace,
                              size_t ws_bytes, void* stream);

/* Many independent instances of dmpt_sp2_response in one call (uneven
 * sizes), e.g. a batch of molecules; each instance keeps its own control
 * block and takes its own decisions (Algorithms 1-3).  The initial layer
 * (bounds, S_0 and S_1 of Sec. III A, its decide step, the 16-bit split)
 * and the outputs of all instances take one launch per step.  In the dual
 * forms on CTA pairs (first order, up to 1024 non-trivial instances) one
 * grouped tensor-core launch per layer step serves every instance from one
 * pool of tiles, claimed through a device-side queue, followed by one
 * batched decide launch; otherwise every instance's layer kernels run on an
 * internal stream of its own.  One CUDA graph holds a layer step and is
 * replayed until all instances have converged (finished instances add no
 * work).  Each instance's results equal those of its own dmpt_sp2_response
 * call bit for bit, except on 256 x 128 tiles (o->group_tile_n = 128).
 *   count       instances; H, H1, P, P1: host arrays of `count` device
 *               pointers (H1/P1 entries: k blocks of n_i x n_i (ld_i)).
 *   n, ld, n_occ: host arrays of `count` values.
 *   k           directions per instance (same for all), 0..DMPT_MAX_K.
 *   info        host array of `count` entries (may be NULL).
 *   workspace   dmpt_workspace_size_batch() bytes, 256-byte aligned.
 * Options: no tape (ckpt_every = 0) and no per-launch timing.  Synchronises
 * the issuing stream every o->sync_every layers; the caller's `stream` is
 * ordered before and after the batch.  Returns the first failing instance's
 * status (all instances are still written). */
size_t dmpt_workspace_size_batch(int count, const int64_t* n, int k, const dmpt_options* o);
dmpt_status dmpt_sp2_response_batch(dmpt_handle h, int count, const double* const* H,
                                    const double* const* H1, int k, const int64_t* n,
                                    const int64_t* ld, const int64_t* n_occ,
                                    const dmpt_options* o, double* const* P, double* const* P1,
                                    dmpt_info* info, void* workspace, size_t ws_bytes,
                                    void* stream);

/* First-order responses to new perturbations, reusing the S0 states that a
 * preceding dmpt_sp2_response call with o->ckpt_every = 1 (dual precision)
 * kept in `workspace`: only the response recursion of Sec. III A,
 * Eq. (S_n detailed) with Eq. (dB), runs -- one response-type layer product
 * per layer, no squares -- with the forward's branch sequence (continued by
 * the sigma flip of Alg. 1 past the forward's last layer) and the Alg. 3
 * test (C_pt, FroErr^(0) of the forward).  The forward's own H1 gives the
 * forward's P1 bit for bit.
 *   H1  device, k blocks of n x n (ld); k <= the forward's k (>= 1).
 *   P1  device, k blocks of n x n (ld) outputs.
 * The forward's response slots are overwritten; the tape is kept. */
dmpt_status dmpt_response_replay(dmpt_handle h, const double* H1, int k, int64_t n,
                                 int64_t ld, const dmpt_options* o, double* P1, dmpt_info* info,
                                 void* workspace, size_t ws_bytes, void* stream);

/* Self-consistent first-order response (self-consistent-charge coupling,
 * Sec. III A; the paper skips this step for its DFTB examples, Sec. IV B):
 * the fixed point of
 *   H1_eff = H1_ext + diag(gamma q),  q = diag(P1),  P1 = R(H1_eff),
 * with R the response of the forward run whose S0 tape is in `workspace`
 * (as for dmpt_response_replay) and gamma an SPD coupling (device n x n,
 * ld).  Linear mixing of the induced charges: q <- (1 - mixing) q +
 * mixing diag(P1), until max_j ||diag(P1_j) - q_j|| / ||diag(P1_j)|| < tol
 * (mixing in (0, 1]); each iteration is one response replay.
 *   iterations, residual: host outputs (may be NULL).
 * Returns DMPT_ENOTCONV when max_iter iterations do not reach tol (P1 holds
 * the last iterate).  Synchronises `stream` once per iteration. */
dmpt_status dmpt_scc_response(dmpt_handle h, const double* H1_ext, const double* gamma, int k,
                              int64_t n, int64_t ld, const dmpt_options* o, double tol,
                              int max_iter, double mixing, double* P1, dmpt_info* info,
                              int* iterations, double* residual, void* workspace,
                              size_t ws_bytes, void* stream);

/* A sequence of problems held in host memory, solved one after another
 * (Algorithms 1-3 for each, as dmpt_sp2_response with ld = n).  Inputs are
 * copied in and results copied out on two copy streams of the handle, with
 * two device buffer sets, so that the copy-in of instance i+1 and the
 * copy-out of instance i-1 run while instance i is being solved.  Only the
 * upper triangle (j >= i) of each input matrix is read: rows are copied in
 * blocks of DMPT_HOST_ROW_BLOCK rows, from the block's diagonal to the end of
 * the row (dmpt_host_copy_in_bytes() bytes per instance, about half of the
 * matrices), and the device fills the lower triangle from the upper one.
 *   count      instances (>= 0).
 *   H_host     host array of `count` pointers to n x n row-major float64
 *              matrices in host memory.
 *   H1_host    host array of `count` pointers, each to k contiguous n x n
 *              blocks (NULL allowed when k = 0).
 *   P_host     host array of `count` output pointers (n x n), or NULL to
 *              skip copying P out; entries may be NULL.
 *   P1_host    host array of `count` output pointers (k blocks each).
 *   info       host array of `count` entries (may be NULL).
 *   workspace  dmpt_workspace_size_host() bytes of device memory, 256-byte
 *              aligned: the solver's workspace plus the two buffer sets.
 * Host buffers should be page-locked (cudaHostAlloc or cudaHostRegister) for
 * the copies to overlap the solves; pageable buffers give the same results
 * without the overlap.  First order only (o->order = 1).  `stream` is
 * ordered before the first copy and after the last; the call returns when
 * every result is in host memory.  Returns the first instance's non-OK
 * status; the instances after it are not run. */
size_t dmpt_workspace_size_host(int64_t n, int k, const dmpt_options* o);
/* Bytes dmpt_sp2_response_host copies to the device per instance of size n
 * with k directions (0 on invalid n or k). */
size_t dmpt_host_copy_in_bytes(int64_t n, int k);
dmpt_status dmpt_sp2_response_host(dmpt_handle h, int count, const double* const* H_host,
                                   const double* const* H1_host, int k, int64_t n,
                                   int64_t n_occ, const dmpt_options* o,
                                   double* const* P_host, double* const* P1_host,
                                   dmpt_info* info, void* workspace, size_t ws_bytes,
                                   void* stream);

/* Autotuning of the layer products (dual forms; the paper has no
 * counterpart -- a library feature).  Times short probe solves of
 * (H, H1) -- the first `probe_layers` layers (default 3 when <= 0), all
 * full D0 layers -- under each candidate configuration:
 *   tile shape    256 x 256 on CTA pairs (cta_pair = 1) or 128 x 256 on
 *                 single CTAs (cta_pair = 0),
 *   rasterisation tile_band in {0, 4, 8, 16} for CTA pairs,
 * with the other options of `o` (K-snake as given), and keeps the
 * configuration with the least layer-product time per layer.  The winner is
 * stored in the handle's table under (padded n, k, precision) and, when
 * `best` is not NULL, returned as a copy of *o with those fields set
 * (best->autotune = 0); *best_layer_ms receives its time per layer.  The
 * candidates differ in tile order and shape only, so any of them gives the
 * method's results within its accuracy (tile order alone: bit-identical).
 *   P, P1  device outputs of the probe solves (overwritten; as for
 *          dmpt_sp2_response), workspace as for dmpt_sp2_response.
 * FP32/FP64 forms have no candidates: *best = *o.  Synchronises `stream`. */
dmpt_status dmpt_autotune(dmpt_handle h, const double* H, const double* H1, int k, int64_t n,
                          int64_t ld, int64_t n_occ, const dmpt_options* o, int probe_layers,
                          double* P, double* P1, dmpt_options* best, double* best_layer_ms,
                          void* workspace, size_t ws_bytes, void* stream);

/* Static-scratch variant of dmpt_sp2_response for callers that cannot
 * allocate device memory (a host framework that owns every allocation, code
 * that must not allocate after start-up, plug-ins that only get input and
 * output pointers).  The paper has no counterpart; this is a library
 * convenience.
 *   Same arguments and results as dmpt_sp2_response, without the workspace:
 *   scratch comes from one fixed device array of DMPT_STATIC_SCRATCH_BYTES
 *   inside the library, resident on every GPU that loads it until exit.
 *   Limits: n <= DMPT_STATIC_MAX_N, k <= DMPT_STATIC_MAX_K; larger sizes
 *   return DMPT_EINVAL.  o->timing = 1 and o->autotune = 1 return
 *   DMPT_EUNSUPPORTED (both create CUDA events; tuning also runs probe
 *   solves), and so does o->ckpt_every = 1: this call keeps no S0 tape, so
 *   dmpt_sp2_backward and dmpt_response_replay cannot follow it.  Every
 *   refusal sets info->status (info is cleared on entry), the handle's
 *   dmpt_last_error text and a line on stderr.
 *   The first call on a device looks up the array's device address (with
 *   that device current), and looks it up again when the device's context
 *   has been replaced (e.g. after cudaDeviceReset); make that first call
 *   before any stream capture.
 *   All calls share the array and it keeps the last call's contents; calls
 *   that overlap on the GPU race on it and must be serialised by the caller.
 *   Allocates nothing: no cudaMalloc, cudaFree or allocating library call. */
#define DMPT_STATIC_MAX_N 512
#define DMPT_STATIC_MAX_K 1
#define DMPT_STATIC_SCRATCH_BYTES (8912896) /* 8.5 MiB */
dmpt_status dmpt_sp2_response_static(dmpt_handle h, const double* H, const double* H1,
                                     int k, int64_t n, int64_t ld, int64_t n_occ,
                                     const dmpt_options* o, double* P, double* P1,
                                     dmpt_info* info, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DMPT_H */
