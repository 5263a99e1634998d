// Element-wise kernels, device-side control of Algorithms 1-3, and the SIMT
// (FP64 / FP32) layer product with its fused epilogue.
//
// Matrices inside the workspace are n x n zero-padded to Np x Np (Np a
// multiple of 256).  Zero padding is invariant under the SP2 layers
// (0^2 = 0, 2*0 - 0^2 = 0) and adds nothing to traces or norms, so the
// product kernels need no bounds checks.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <mutex>

#include "dmpt_internal.cuh"

namespace dmpt {

static inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

Layout make_layout(int64_t n, int k, int precision, int tape_states, int ckpt_slots, int pad) {
  Layout L{};
  L.n = n;
  L.Np = ((n + pad - 1) / pad) * pad;
  L.k = k;
  L.precision = precision;
  L.tape_states = tape_states;
  L.elem = (precision == DMPT_FP64) ? 8 : 4;
  size_t off = 0;
  L.off_state = off;
  off = align256(off + sizeof(State));
  // one partial entry per upper tile of the smallest product tile (64) or
  // per block of the init kernel, whichever is larger
  int64_t tiles = upper_tiles(L.Np, 64);
  L.partial_tiles = tiles > 1024 ? tiles : 1024;
  L.off_partials = off;
  off = align256(off + (size_t)(1 + k) * (size_t)L.partial_tiles * kNQ * sizeof(double));
  const size_t mat = (size_t)L.Np * (size_t)L.Np;
  L.off_master = off;
  off = align256(off + 2 * (size_t)(1 + k) * mat * L.elem);
  if (precision == DMPT_DUAL_FP16 || precision == DMPT_DUAL_BF16) {
    L.off_ops16 = off;
    off = align256(off + (2 * (size_t)(1 + k) * 2 + 2 * (size_t)tape_states) * mat * 2);
  } else {
    L.off_ops16 = 0;
  }
  // small vectors of the self-consistent response: q[k][n], v[k][n], red[k][4]
  L.off_vec = off;
  off = align256(off + ((size_t)(k > 0 ? k : 1) * (2 * (size_t)n + 4)) * sizeof(double));
  // FP32 checkpoints of every ckpt_k-th S0 state (adjoint with recompute)
  L.ckpt_slots = ckpt_slots;
  L.off_ckpt = off;
  off = align256(off + (size_t)ckpt_slots * mat * 4);
  L.total = off;
  return L;
}

// ---------------------------------------------------------------------------
// Deterministic block reduction of NV doubles (fixed tree, fixed order).
template <int NV, int NT>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* smem /* NT*NV */) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int i = 0; i < NV; ++i) smem[i * NT + tid] = v[i];
  __syncthreads();
  for (int s = NT / 2; s > 0; s >>= 1) {
    if (tid < s) {
#pragma unroll
      for (int i = 0; i < NV; ++i) smem[i * NT + tid] += smem[i * NT + tid + s];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = smem[i * NT];
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Gershgorin bounds (Sec. II B; Alg. 1 inputs).  Min / max are taken with
// 64-bit integer atomics on an order-preserving encoding of the doubles, so
// the result is independent of the order in which rows finish and the call
// needs no scratch memory beyond its 2-double output.

__device__ __forceinline__ long long dkey(double x) {
  long long b = __double_as_longlong(x);
  return b >= 0 ? b : (b ^ 0x7FFFFFFFFFFFFFFFLL);
}
__device__ __forceinline__ double dkey_inv(long long k) {
  long long b = k >= 0 ? k : (k ^ 0x7FFFFFFFFFFFFFFFLL);
  return __longlong_as_double(b);
}

__global__ void bounds_init_kernel(long long* key) {
  key[0] = dkey(INFINITY);
  key[1] = dkey(-INFINITY);
}

// one warp per row; row r: centre H_rr, radius sum_{j != r} |H_rj|
__global__ void bounds_rows_kernel(const double* __restrict__ H, int64_t n, int64_t ld,
                                   long long* key) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double lo = INFINITY, hi = -INFINITY;
  for (int64_t r = warp; r < n; r += nwarps) {
    const double* row = H + r * ld;
    double s = 0.0;
    for (int64_t j = lane; j < n; j += 32) s += fabs(row[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const double d = row[r];
    const double rad = s - fabs(d);
    lo = fmin(lo, d - rad);
    hi = fmax(hi, d + rad);
  }
  if (lane == 0 && warp < n) {
    atomicMin(&key[0], dkey(lo));
    atomicMax(&key[1], dkey(hi));
  }
}

__global__ void bounds_fin_kernel(long long* key) {
  double lo = dkey_inv(key[0]);
  double hi = dkey_inv(key[1]);
  double* out = reinterpret_cast<double*>(key);
  out[0] = lo;
  out[1] = hi;
}

cudaError_t launch_bounds(const double* H, int64_t n, int64_t ld, double* eps_out,
                          cudaStream_t s) {
  long long* key = reinterpret_cast<long long*>(eps_out);
  bounds_init_kernel<<<1, 1, 0, s>>>(key);
  int64_t warps = n < 152 * 64 ? n : 152 * 64;
  int blocks = (int)((warps * 32 + 255) / 256);
  bounds_rows_kernel<<<blocks, 256, 0, s>>>(H, n, ld, key);
  bounds_fin_kernel<<<1, 1, 0, s>>>(key);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Initial normalisation layer (Alg. 1; Sec. III A, S_0(lambda)):
//   S0 = (eps_N I - H) / (eps_N - eps_1),  S1_k = -H1_k / (eps_N - eps_1).
// Only the upper triangle (j >= i) of H and H1 is read, so the stored
// matrices are exactly symmetric.  Partial sums per block: Tr S0, ||S0||_F^2,
// ||S1_k||_F^2 and a count of non-finite values.

// Block vb of a grid of vgrid blocks (256 threads): tile pairs vb, vb + vgrid,
// ... of each matrix in turn (S0, then S1_1 .. S1_k).
template <typename T>
__device__ __forceinline__ void init_body(State* st, T* master, const double* __restrict__ H,
                                          const double* __restrict__ H1, int64_t n, int64_t Np,
                                          int64_t ld, int k, int first_m,
                                          const double* __restrict__ shift, int k_zero,
                                          double* partials, int64_t ptiles, int64_t vb,
                                          int64_t vgrid) {
  // 64 x 64 tile pairs (bi <= bj): the upper tile is read row-wise (coalesced,
  // every load of the tile in flight at once), written in place and, through
  // shared memory, transposed into the mirror tile, so both triangles of S
  // come from the upper triangle of the input.  Each value is formed in FP64
  // and rounded once to T (for T = float, the off-diagonal values are formed
  // in FP32).  The squared norms are summed in FP64 for the FP64 form; for
  // T = float, as exact FP32 products with TwoSum compensation (the FP64 rate
  // of the part is low).
  constexpr bool F32 = sizeof(T) == 4;
  constexpr int TS = kInitTile;
  constexpr int RPT = TS * TS / 256;   // rows of the tile per thread
  constexpr int RS = TS / RPT;         // row step between them
  __shared__ T tile[TS][TS + 1];
  __shared__ double red[2 * 256];
  const double e1 = st->eps1, eN = st->epsN;
  __shared__ double w_sh;   // one FP64 division per block
  if (threadIdx.x == 0) w_sh = 1.0 / (eN - e1);
  __syncthreads();
  const double w = w_sh;
  const float wf = (float)w;
  const bool hole = st->hole != 0;   // complement form: S_0 = I - (eps_N I - H) w
  const size_t mat = (size_t)Np * Np;
  const int tx = threadIdx.x % TS, ty = threadIdx.x / TS;   // 64 x 4 threads
  const int64_t TB = Np / TS;
  const int64_t pairs = TB * (TB + 1) / 2;
  int nbad = 0;
  for (int m = first_m; m <= k; ++m) {
    const double* src = m == 0 ? H : H1 + (size_t)(m - 1) * n * ld;
    T* dst = master + (size_t)m * mat;   // buffer 0 (slots 0 .. layout k)
    double tr = 0.0, fd = 0.0;
    float fs = 0.0f, fc = 0.0f;
    for (int64_t tp = vb; tp < pairs; tp += vgrid) {
      // tile pair index -> (bi, bj), bj-major: tp = bj (bj + 1) / 2 + bi (an
      // FP32 estimate of bj, corrected in integers)
      int64_t bj = (int64_t)((sqrtf(8.0f * (float)tp + 1.0f) - 1.0f) * 0.5f);
      while ((bj + 1) * (bj + 2) / 2 <= tp) ++bj;
      while (bj * (bj + 1) / 2 > tp) --bj;
      const int64_t bi = tp - bj * (bj + 1) / 2;
      double hv[RPT];
      {
        const int64_t r0 = bi * TS + ty, c = bj * TS + tx;
        const double* sp = src + r0 * ld + c;
        // row r0 + RS i lies in the matrix when RS i < lim
        const int lim = c < n ? (int)min((int64_t)TS, n - r0) : 0;
#pragma unroll
        for (int i = 0; i < RPT; ++i) hv[i] = RS * i < lim ? sp[(int64_t)(RS * i) * ld] : 0.0;
      }
      if constexpr (F32) {
        // off the diagonal in FP32 arithmetic (the FP64 rate of the part is
        // low): v = -+ fl32(h) w32, within 1.5 units in the last place; zero
        // outside the matrix (h = 0 there)
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          const float hw = (float)hv[i] * wf;
          tile[ty + RS * i][tx] = hole ? hw : -hw;
        }
        // the diagonal element of column tx, formed in FP64 and rounded once
        if (bi == bj && tx % RS == ty) {
          const int64_t r = bi * TS + tx;
          if (r < n) {
            double h = src[r * ld + r];
            if (m > 0 && shift != nullptr) h += shift[(size_t)(m - 1) * n + r];
            const double x = hole ? (m == 0 ? (h - e1) * w : h * w)
                                  : (m == 0 ? (eN - h) * w : -h * w);
            const float xv = (float)x;
            tile[tx][tx] = xv;
            if (m == 0) tr += (double)xv;
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          const int rl = ty + RS * i;
          const int64_t r = bi * TS + rl, c = bj * TS + tx;
          double x = 0.0;
          if (r < n && c < n) {
            double h = hv[i];
            if (m > 0 && shift != nullptr && r == c) h += shift[(size_t)(m - 1) * n + r];
            if (hole)
              x = m == 0 ? (h - (r == c ? e1 : 0.0)) * w : h * w;
            else
              x = m == 0 ? ((r == c ? eN : 0.0) - h) * w : -h * w;
          }
          tile[rl][tx] = (T)x;
          if (m == 0 && r == c) tr += x;
        }
      }
      __syncthreads();
#pragma unroll 4
      for (int i = 0; i < RPT; ++i) {
        const int rl = ty + RS * i;
        const int64_t r = bi * TS + rl, c = bj * TS + tx;
        // diagonal tile: the lower half mirrors the upper half
        const T v = (bi < bj || rl <= tx) ? tile[rl][tx] : tile[tx][rl];
        dst[(size_t)r * Np + c] = v;
        if constexpr (F32) {
          const float wgt = bi < bj ? 2.0f : 1.0f;   // the mirror tile holds the same values
          const float p = wgt * v * v;
          const float e = wgt * fmaf(v, v, -v * v);
          const float tt = fs + p;
          const float bp = tt - fs;
          fc += (fs - (tt - bp)) + (p - bp) + e;
          fs = tt;
        } else {
          const double wgt = bi < bj ? 2.0 : 1.0;
          fd += wgt * v * v;
        }
        nbad += isfinite(v) ? 0 : 1;
        if (bi < bj) dst[(size_t)(bj * TS + rl) * Np + bi * TS + tx] = tile[tx][rl];
      }
      __syncthreads();
    }
    // partial sums of job m: Tr S0 (job 0) and ||S_m||_F^2
    double v[2] = {tr, F32 ? (double)fs + (double)fc : fd};
    block_sum<2, 256>(v, red);
    if (threadIdx.x == 0) {
      double* p = partials + ((size_t)m * ptiles + vb) * kNQ;
      p[kQTrace] = m == 0 ? v[0] : 0.0;
      p[kQFroNew] = v[1];
      p[kQFroDiff] = 0.0;
      p[kQBad] = 0.0;
    }
  }
  // higher-order slots start at zero (a linear perturbation: H^(o) = 0, o >= 2)
  for (int m = k + 1; m <= k + k_zero; ++m) {
    T* dst = master + (size_t)m * mat;
    for (int64_t idx = vb * blockDim.x + threadIdx.x; idx < (int64_t)mat;
         idx += vgrid * blockDim.x)
      dst[idx] = (T)0;
    if (threadIdx.x == 0) {
      double* p = partials + ((size_t)m * ptiles + vb) * kNQ;
      p[kQTrace] = 0.0;
      p[kQFroNew] = 0.0;
      p[kQFroDiff] = 0.0;
      p[kQBad] = 0.0;
    }
  }
  // the count of non-finite values goes with job 0 (job 1 in a replay, which
  // starts at S1_1)
  double vb_bad[1] = {(double)nbad};
  block_sum<1, 256>(vb_bad, red);
  if (threadIdx.x == 0 && (first_m == 0 || k > 0))
    partials[((size_t)first_m * ptiles + vb) * kNQ + kQBad] = vb_bad[0];
}

template <typename T>
__global__ void __launch_bounds__(256) init_kernel(State* st, T* master, const double* __restrict__ H,
                                                   const double* __restrict__ H1, int64_t n,
                                                   int64_t Np, int64_t ld, int k, int first_m,
                                                   const double* __restrict__ shift, int k_zero,
                                                   double* partials, int64_t ptiles) {
  init_body<T>(st, master, H, H1, n, Np, ld, k, first_m, shift, k_zero, partials, ptiles,
               blockIdx.x, gridDim.x);
}

cudaError_t launch_init(const Layout& L, void* ws, const double* H, const double* H1,
                        int64_t ld, int k, int blocks, cudaStream_t s, int first_m,
                        const double* shift, int k_zero) {
  char* base = (char*)ws;
  State* st = (State*)(base + L.off_state);
  double* partials = (double*)(base + L.off_partials);
  if (L.precision == DMPT_FP64)
    init_kernel<double><<<blocks, 256, 0, s>>>(st, (double*)(base + L.off_master), H, H1, L.n,
                                               L.Np, ld, k, first_m, shift, k_zero, partials,
                                               L.partial_tiles);
  else
    init_kernel<float><<<blocks, 256, 0, s>>>(st, (float*)(base + L.off_master), H, H1, L.n,
                                              L.Np, ld, k, first_m, shift, k_zero, partials,
                                              L.partial_tiles);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Self-consistent response: charge potential and linear mixing of the
// induced charges q = diag(P1).

// v_j[r] = sum_c gamma[r][c] q_j[c]; one warp per row, FP64
__global__ void scc_potential_kernel(const double* __restrict__ gamma, int64_t n, int64_t ld,
                                     const double* __restrict__ q, double* v, int k) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < n; r += nw) {
    const double* g = gamma + r * ld;
    for (int j = 0; j < k; ++j) {
      const double* qj = q + (size_t)j * n;
      double acc = 0.0;
      for (int64_t c = lane; c < n; c += 32) acc = fma(g[c], qj[c], acc);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) v[(size_t)j * n + r] = acc;
    }
  }
}

cudaError_t launch_scc_potential(const double* gamma, int64_t n, int64_t ld, const double* q,
                                 double* v, int k, cudaStream_t s) {
  int64_t warps = n < 152 * 32 ? n : 152 * 32;
  scc_potential_kernel<<<(int)((warps * 32 + 255) / 256), 256, 0, s>>>(gamma, n, ld, q, v, k);
  return cudaGetLastError();
}

// one block per direction: red[j] = {||diag(P1_j) - q_j||^2, ||diag(P1_j)||^2}, then mix
__global__ void __launch_bounds__(256) scc_mix_kernel(const double* __restrict__ P1, int64_t n,
                                                      int64_t ld, double* q, double alpha,
                                                      double* red) {
  __shared__ double sm[2 * 256];
  const int j = blockIdx.x;
  const double* p = P1 + (size_t)j * n * ld;
  double* qj = q + (size_t)j * n;
  double d2 = 0.0, o2 = 0.0;
  for (int64_t r = threadIdx.x; r < n; r += 256) {
    const double qo = p[r * ld + r];
    const double d = qo - qj[r];
    d2 += d * d;
    o2 += qo * qo;
    qj[r] = (1.0 - alpha) * qj[r] + alpha * qo;
  }
  double v[2] = {d2, o2};
  block_sum<2, 256>(v, sm);
  if (threadIdx.x == 0) {
    red[4 * j + 0] = v[0];
    red[4 * j + 1] = v[1];
  }
}

cudaError_t launch_scc_mix(const double* P1, int64_t n, int64_t ld, double* q, int k,
                           double alpha, double* red, cudaStream_t s) {
  scc_mix_kernel<<<k, 256, 0, s>>>(P1, n, ld, q, alpha, red);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Device-side control (Alg. 1 branch rule, Alg. 2, Alg. 3).

__device__ int fp16_exponent_for(double bound) {
  // exponent e with bound * 2^e < 2^kFp16TargetExp
  if (!(bound > 0.0) || !isfinite(bound)) return 0;
  int e = kFp16TargetExp - (ilogb(bound) + 1);
  return e < -100 ? -100 : (e > 100 ? 100 : e);
}

// Plan layer n (Alg. 1: branch choice; Alg. 2: D0 stopping tests).
__device__ void plan_layer(State* st, int n) {
  int sigma;
  if (!st->d0_conv) {
    const double NS = st->NS, NX = st->NX, no = st->n_occ;
    const double iderr = NS - NX;
    // sigma_n = sign(|2 N_S - N_X - N_occ| - |N_X - N_occ|); sign(0) -> -1
    const double arg = fabs(2.0 * NS - NX - no) - fabs(NX - no);
    sigma = arg > 0.0 ? 1 : -1;
    st->iderr[n] = iderr;
    st->ns_hist[n] = NS;
    st->nx_hist[n] = NX;
    st->sigma[n] = (signed char)sigma;
    bool stop = iderr <= 0.0;
    if (!stop && n > 2 && st->sigma[n - 1] != st->sigma[n - 2] &&
        iderr > st->c_d0 * st->iderr[n - 2] * st->iderr[n - 2])
      stop = true;
    st->plan_square = 1;
    if (stop) {
      st->d0_conv = 1;
      st->d0_layer = n;
      st->plan_write0 = 0;  // this layer's square only measures FroErr^(0)
    } else {
      st->plan_write0 = 1;
    }
  } else {
    sigma = -(int)st->sigma[n - 1];  // the sigma flip of Alg. 1
    st->sigma[n] = (signed char)sigma;
    st->plan_square = 0;
    st->plan_write0 = 0;
  }
  st->sigma_cur = sigma;
  for (int j = 0; j < st->k; ++j) {
    st->plan_resp[j] = !st->d1_conv[j];
    // |S1_n|_max <= ||S1_n||_2 <= (2 ||S0||_2 + |1 - sigma|) ||S1_{n-1}||_2
    //            <= 4.5 ||S1_{n-1}||_F   (spectrum of S0 within [-0.25, 1.25]);
    // an order-o slot (o >= 2) adds sum_{a=1}^{o-1} ||S_a S_{o-a}||_2
    // <= sum ||S_a||_F ||S_{o-a}||_F (twice, for 2 S - S^2)
    double bound = 4.5 * sqrt(st->s1_fro2[j]);
    if (st->order >= 2 && j >= st->k1) {
      const int o = 1 + j / st->k1, d = j % st->k1;
      double cross = 0.0;
      for (int a = 1; a < o; ++a)
        cross += sqrt(st->s1_fro2[(a - 1) * st->k1 + d] * st->s1_fro2[(o - a - 1) * st->k1 + d]);
      bound += 2.0 * cross;
    }
    st->s1_exp_next[j] = st->precision == DMPT_DUAL_FP16 ? fp16_exponent_for(bound) : 0;
  }
  st->n_layer = n;
}

// Plan layer m of a response replay: S0 operand = stored state
// min(m - 1, U), the forward's sigma_m (continued by flips past the forward's
// last layer), responses of the directions still running.
__device__ void plan_replay(State* st, int m) {
  const int U = st->d0_updates;
  st->z0_cur = st->tape_base + 2 * (m - 1 < U ? m - 1 : U);
  if (m > st->rp_lmax) st->sigma[m] = (signed char)(-st->sigma[m - 1]);
  st->sigma_cur = st->sigma[m];
  st->plan_square = 0;
  st->plan_write0 = 0;
  for (int j = 0; j < st->k; ++j) {
    st->plan_resp[j] = !st->d1_conv[j];
    st->s1_exp_next[j] = st->precision == DMPT_DUAL_FP16
                             ? fp16_exponent_for(4.5 * sqrt(st->s1_fro2[j]))
                             : 0;
  }
  st->n_layer = m;
}

// The decide step of one instance, run by one 256-thread block (red: kNQ x
// 256 doubles, sums: (kMaxK + 1) x kNQ doubles of shared memory).
__device__ void decide_body(State* st, const double* __restrict__ partials, int64_t ptiles,
                            int64_t entries, int mode, double* red, double (*sums)[kNQ]) {
  if (threadIdx.x == 0) {
    st->round_ctr = 0u;    // for the next pair-kernel launch
    st->ckpt_pending = 0;  // set again below when this step makes a checkpointed state
  }
  if (st->done) return;
  const bool adj = mode == kDecideAdjInit || mode == kDecideAdjLayer || mode == kDecideAdjResume;
  const bool rp = mode == kDecideReplayInit || mode == kDecideReplayLayer;
  const int k = adj ? 1 : st->k;
  for (int job = 0; job <= k; ++job) {
    bool ran;
    if (adj)
      ran = job == 1 && mode != kDecideAdjResume;
    else if (mode == kDecideInit)
      ran = true;
    else if (mode == kDecideReplayInit)
      ran = job >= 1;
    else
      ran = job == 0 ? st->plan_square != 0 : st->plan_resp[job - 1] != 0;
    (void)rp;
    if (!ran) continue;  // uniform across the block
    double v[kNQ] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t e = threadIdx.x; e < entries; e += 256) {
      const double* p = partials + ((size_t)job * ptiles + e) * kNQ;
#pragma unroll
      for (int q = 0; q < kNQ; ++q) v[q] += p[q];
    }
    block_sum<kNQ, 256>(v, red);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int q = 0; q < kNQ; ++q) sums[job][q] = v[q];
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;

  if (mode == kDecideReplayInit || mode == kDecideReplayLayer) {
    // ---- response recursion replayed over the stored S0 states
    if (st->timeout_flag) {
      st->status = DMPT_ETIMEOUT;
      st->done = 1;
      return;
    }
    double bad = 0.0;
    for (int j = 0; j < k; ++j)
      if (mode == kDecideReplayInit || st->plan_resp[j]) bad += sums[1 + j][kQBad];
    if (bad > 0.0) {
      st->status = DMPT_ENUMERIC;
      st->done = 1;
      return;
    }
    if (mode == kDecideReplayInit) {
      for (int j = 0; j < k; ++j) {
        st->cur1[j] = 0;
        st->d1_conv[j] = 0;
        st->d1_layer[j] = 0;
        st->s1_fro2[j] = sums[1 + j][kQFroNew];
        st->s1_exp_cur[j] = st->precision == DMPT_DUAL_FP16
                                ? fp16_exponent_for(sqrt(st->s1_fro2[j]))
                                : 0;
      }
      st->rp_lmax = st->layers_run;
      st->rp_layers = 0;
      plan_replay(st, 1);
      return;
    }
    const int n = st->n_layer;
    for (int j = 0; j < k; ++j) {
      if (!st->plan_resp[j]) continue;
      const double fe = sqrt(sums[1 + j][kQFroDiff]);
      st->froerr1[j][n] = fe;
      const bool fired = n - 2 >= st->d0_layer &&
                         fe >= st->c_pt * st->froerr0 * st->froerr1[j][n - 2];
      if (fired) {
        st->d1_conv[j] = 1;
        st->d1_layer[j] = n;
      } else {
        st->cur1[j] ^= 1;
        st->s1_fro2[j] = sums[1 + j][kQFroNew];
        st->s1_exp_cur[j] = st->s1_exp_next[j];
      }
    }
    st->rp_layers = n;
    bool all1 = true;
    for (int j = 0; j < k; ++j) all1 = all1 && st->d1_conv[j];
    if (all1) {
      st->status = DMPT_OK;
      st->done = 1;
      return;
    }
    if (n + 1 > st->max_layers) {
      st->status = DMPT_ENOTCONV;
      st->done = 1;
      return;
    }
    plan_replay(st, n + 1);
    return;
  }

  if (adj) {
    // ---- adjoint of the S0 recursion, run backwards over the stored states
    if (st->timeout_flag) {
      st->status = DMPT_ETIMEOUT;
      st->done = 1;
      return;
    }
    if (mode != kDecideAdjResume && sums[1][kQBad] > 0.0) {
      st->status = DMPT_ENUMERIC;
      st->done = 1;
      return;
    }
    int m;
    if (mode == kDecideAdjInit) {
      st->k = 1;
      st->cur1[0] = 0;
      st->plan_square = 0;
      st->plan_write0 = 0;
      for (int j = 0; j < kMaxK; ++j) st->plan_resp[j] = 0;
      st->s1_fro2[0] = sums[1][kQFroNew];
      st->s1_exp_cur[0] = st->precision == DMPT_DUAL_FP16
                              ? fp16_exponent_for(sqrt(st->s1_fro2[0]))
                              : 0;
      m = st->d0_updates;
    } else if (mode == kDecideAdjLayer) {
      st->cur1[0] ^= 1;
      st->s1_fro2[0] = sums[1][kQFroNew];
      st->s1_exp_cur[0] = st->s1_exp_next[0];
      m = st->adj_m - 1;
    } else {
      m = st->adj_m;   // resume after the host reloaded the tape with an earlier segment
    }
    st->adj_m = m;
    if (m <= 0) {
      st->plan_resp[0] = 0;
      st->status = DMPT_OK;
      st->done = 1;
      return;
    }
    if (m <= st->adj_seg_a) {
      // S_{m-1} lies before the states in the tape (checkpointed run): the
      // host recomputes the previous segment and resumes with layer m
      st->plan_resp[0] = 0;
      return;
    }
    // adjoint of layer m: Gbar <- sigma_m (S_{m-1} Gbar + Gbar S_{m-1}) + (1 - sigma_m) Gbar
    // (the tape holds states adj_seg_a, adj_seg_a + 1, ...; 0 without checkpoints)
    st->z0_cur = st->tape_base + 2 * (m - 1 - st->adj_seg_a);
    st->sigma_cur = st->sigma[m];
    st->plan_resp[0] = 1;
    st->s1_exp_next[0] = st->precision == DMPT_DUAL_FP16
                             ? fp16_exponent_for(4.5 * sqrt(st->s1_fro2[0]))
                             : 0;
    return;
  }

  if (mode == kDecideInit) {
    if (!(st->epsN > st->eps1) || !isfinite(st->epsN) || !isfinite(st->eps1) ||
        sums[0][kQBad] > 0.0) {
      st->status = DMPT_ENUMERIC;
      st->done = 1;
      return;
    }
    st->NS = sums[0][kQTrace];
    st->NX = sums[0][kQFroNew];
    st->s0_exp = st->precision == DMPT_DUAL_FP16 ? kFp16TargetExp - 1 : 0;
    st->cur0 = 0;
    st->d0_updates = 0;
    st->ckpt_pending = st->ckpt_k >= 2 ? 1 : 0;   // S_0 is checkpoint 0
    st->z0_cur = st->tape ? st->tape_base : zslice(0, 0, 0, st->layout_k);
    st->z0_next = st->tape ? st->tape_base + 2 : zslice(1, 0, 0, st->layout_k);
    st->d0_conv = 0;
    st->d0_layer = 0;
    st->layers_run = 0;
    st->froerr0 = 0.0;
    for (int j = 0; j < k; ++j) {
      st->cur1[j] = 0;
      st->d1_conv[j] = 0;
      st->d1_layer[j] = 0;
      st->s1_fro2[j] = sums[1 + j][kQFroNew];
      st->s1_exp_cur[j] = st->precision == DMPT_DUAL_FP16
                              ? fp16_exponent_for(sqrt(st->s1_fro2[j]))
                              : 0;
    }
    plan_layer(st, 1);
    return;
  }

  // ---- a layer product has finished: apply its results
  const int n = st->n_layer;
  if (st->timeout_flag) {
    st->status = DMPT_ETIMEOUT;
    st->done = 1;
    return;
  }
  double bad = 0.0;
  if (st->plan_square) bad += sums[0][kQBad];
  for (int j = 0; j < k; ++j)
    if (st->plan_resp[j]) bad += sums[1 + j][kQBad];
  if (bad > 0.0) {
    st->status = DMPT_ENUMERIC;
    st->done = 1;
    return;
  }
  if (st->plan_square) {
    if (st->plan_write0) {
      st->NS = sums[0][kQTrace];    // Tr S_n      (N_S of Alg. 2)
      st->NX = sums[0][kQFroNew];   // ||S_n||_F^2 = Tr S_n^2 (N_X of the next layer)
      st->cur0 ^= 1;
      st->d0_updates += 1;
      if (st->ckpt_k >= 2 && st->d0_updates % st->ckpt_k == 0) st->ckpt_pending = 1;
      if (st->tape) {
        st->z0_cur = st->z0_next;
        st->z0_next += 2;
      } else {
        st->z0_cur = zslice(st->cur0, 0, 0, st->layout_k);
        st->z0_next = zslice(st->cur0 ^ 1, 0, 0, st->layout_k);
      }
    } else {
      st->froerr0 = sqrt(sums[0][kQFroDiff]);  // FroErr^(0) of Alg. 2
    }
  }
  for (int j = 0; j < k; ++j) {
    if (!st->plan_resp[j]) continue;
    const double fe = sqrt(sums[1 + j][kQFroDiff]);  // FroErr^(1)_n of Alg. 3
    st->froerr1[j][n] = fe;
    bool fired = false;
    if (st->d0_conv && n - 2 >= st->d0_layer)
      fired = fe >= st->c_pt * st->froerr0 * st->froerr1[j][n - 2];
    if (fired) {
      st->d1_conv[j] = 1;  // keep S1_{n-1}: the buffer written by this layer is dropped
      st->d1_layer[j] = n;
    } else {
      st->cur1[j] ^= 1;
      st->s1_fro2[j] = sums[1 + j][kQFroNew];
      st->s1_exp_cur[j] = st->s1_exp_next[j];
    }
  }
  st->layers_run = n;
  bool all1 = true;
  for (int j = 0; j < k; ++j) all1 = all1 && st->d1_conv[j];
  if (st->d0_conv && all1) {
    st->status = DMPT_OK;
    st->done = 1;
    st->n_layer = n + 1;
    return;
  }
  if (n + 1 > st->max_layers) {
    st->status = DMPT_ENOTCONV;
    st->done = 1;
    st->n_layer = n + 1;
    return;
  }
  plan_layer(st, n + 1);
}

__global__ void __launch_bounds__(256) decide_kernel(State* st, const double* __restrict__ partials,
                                                     int64_t ptiles, int64_t entries, int mode) {
  __shared__ double red[kNQ * 256];
  __shared__ double sums[kMaxK + 1][kNQ];
  decide_body(st, partials, ptiles, entries, mode, red, sums);
}

// Layer decide of every instance of a grouped launch, one block each.
__global__ void __launch_bounds__(256) decide_group_kernel(const GroupDecide* __restrict__ args,
                                                           const int* __restrict__ group_timeout,
                                                           GroupQueue* queue) {
  __shared__ double red[kNQ * 256];
  __shared__ double sums[kMaxK + 1][kNQ];
  if (blockIdx.x == 0 && threadIdx.x == 0) {   // the next grouped launch starts a new queue
    queue->counter = 0u;
    queue->epoch += 1u;
  }
  const GroupDecide a = args[blockIdx.x];
  if (threadIdx.x == 0 && *group_timeout && !a.st->done) a.st->timeout_flag = 1;
  __syncthreads();
  decide_body(a.st, a.partials, a.ptiles, a.entries, kDecideLayer, red, sums);
}

cudaError_t launch_decide_group(const GroupDecide* args, int count, const int* group_timeout,
                                GroupQueue* queue, cudaStream_t s) {
  if (count < 1) return cudaSuccess;
  decide_group_kernel<<<count, 256, 0, s>>>(args, group_timeout, queue);
  return cudaGetLastError();
}

cudaError_t launch_decide(const Layout& L, void* ws, int mode, int64_t entries, cudaStream_t s) {
  char* base = (char*)ws;
  decide_kernel<<<1, 256, 0, s>>>((State*)(base + L.off_state),
                                  (const double*)(base + L.off_partials), L.partial_tiles,
                                  entries, mode);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// SIMT layer product with fused epilogue (FP64 and FP32 forms).
//
// Grid: (upper tiles, 1 + slots).  Job 0 computes X = S0 S0 (Sec. II B,
// Eq. (DNN-SP2_act)) for tile (I, J), I <= J; job 1+k computes
// X1 = S0 S1_k + S1_k S0 (activation f^(1), Eq. (eq:activation-function))
// as one accumulation over two K-passes; a higher-order term (Sec. III A,
// Eq. (S_n detailed)) adds its cross products S_a S_{o-a} as further passes.  Both operands are read as row
// panels: for symmetric B, B[k][j] = B[j][k].  The epilogue applies
// S_n = sigma X + (1 - sigma) S_{n-1} (Eq. (eq:Sn); Alg. 2 / Alg. 3 updates)
// to the elements with row <= col, stores them at (r, c) and (c, r) in the
// other ping-pong buffer, and reduces the Alg. 2 / 3 norms in FP64.

template <typename T>
struct Vec;
template <>
struct Vec<float> {
  using type = float4;
  static constexpr int width = 4;
};
template <>
struct Vec<double> {
  using type = double2;
  static constexpr int width = 2;
};

template <typename T, int TM>
__device__ __forceinline__ int frag_index(int t, int m) {
  // the TM rows (cols) of a thread: two runs of TM/2 contiguous elements,
  // the second BT/2 after the first
  constexpr int H = TM / 2;
  constexpr int BT = 16 * TM;
  return m < H ? t * H + m : BT / 2 + t * H + (m - H);
}

// Two blocks per SM for the FP32 form (registers <= 128), one for FP64.
template <typename T>
struct SimtBlocks {
  static constexpr int value = 2;
};
template <>
struct SimtBlocks<double> {
  static constexpr int value = 1;
};

// Jobs of a layer (as in the tensor-core kernels): 0 = square of S0; job
// 1 + (o - 1) k1 + d = the order-o term of direction d, in o + 1 K passes
// (pass 0 = S0 S_o, pass 1 = S_o S0, pass p >= 2 = S_{p-1} S_{o-p+1}).
__device__ __forceinline__ int simt_job_order(int job, int k1) { return 1 + (job - 1) / k1; }
__device__ __forceinline__ int simt_job_passes(int job, int k1) {
  return job == 0 ? 1 : (job <= k1 ? 2 : 1 + simt_job_order(job, k1));
}
__device__ __forceinline__ int simt_job_slot(int job, int a, int k1) {
  return 1 + (a - 1) * k1 + (job - 1) % k1;
}
__device__ __forceinline__ void simt_job_operands(int job, int pass, int k1, int* mA, int* mB) {
  if (job == 0) {
    *mA = 0;
    *mB = 0;
  } else if (pass == 0) {
    *mA = 0;
    *mB = job;
  } else if (pass == 1) {
    *mA = job;
    *mB = 0;
  } else {
    *mA = simt_job_slot(job, pass - 1, k1);
    *mB = simt_job_slot(job, simt_job_order(job, k1) - pass + 1, k1);
  }
}

// 16-byte asynchronous copy global -> shared (L2 only), and its group waits
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Shared memory of the SIMT layer kernel: SIMT_STAGES stages of the two
// operand slabs (BK x BT, rows padded by one 16-byte chunk), then the
// block's reduction array.
constexpr int SIMT_STAGES = 3;
template <typename T, int TM, int BK>
constexpr int simt_smem_bytes() {
  return SIMT_STAGES * 2 * BK * (16 * TM + 16 / (int)sizeof(T)) * (int)sizeof(T) + 4 * 256 * 8;
}

template <typename T, int TM, int BK>
__global__ void __launch_bounds__(256, SimtBlocks<T>::value)
    layer_simt_kernel(State* st, T* __restrict__ master, int64_t Np, int k,
                      double* __restrict__ partials, int64_t ptiles) {
  constexpr int BT = 16 * TM;
  constexpr int VW = 16 / (int)sizeof(T);      // elements per 16-byte copy
  constexpr int LD = BT + VW;                  // padded row of a slab
  constexpr int CPR = BT / VW;                 // copies per slab row
  constexpr int NCP = BK * CPR / 256;          // copies per thread per slab
  static_assert(NCP >= 1 && (BK * CPR) % 256 == 0, "slab copies divide over the block");

  // stage s: As = slab of the A operand, Bs = slab of the B operand, each
  // BK rows (K index) x BT columns (output rows / columns of the tile)
  extern __shared__ __align__(16) uint8_t simt_smem[];
  T* slabs = reinterpret_cast<T*>(simt_smem);
  double* red = reinterpret_cast<double*>(simt_smem + SIMT_STAGES * 2 * BK * LD * sizeof(T));

  if (st->done) return;
  const int job = blockIdx.y;
  const int run = job == 0 ? st->plan_square : st->plan_resp[job - 1];
  if (!run) return;

  // upper tile (I, J), I <= J, row-major over the upper triangle
  const int T_ = (int)(Np / BT);
  int64_t t = blockIdx.x;
  int I = 0;
  while (t >= T_ - I) {
    t -= T_ - I;
    ++I;
  }
  const int J = I + (int)t;

  const size_t mat = (size_t)Np * Np;
  const int cur0 = st->cur0;
  const int cur = job == 0 ? cur0 : st->cur1[job - 1];
  const T* Sj = master + (size_t)(cur * (1 + k) + job) * mat;   // the job's own slot
  T* out = master + (size_t)((cur ^ 1) * (1 + k) + job) * mat;

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  T acc[TM][TM];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TM; ++j) acc[i][j] = T(0);

  const int k1 = st->order >= 2 ? st->k1 : k;   // first-order directions
  const int passes = simt_job_passes(job, k1);
  const int nkb = (int)(Np / BK);
  for (int pass = 0; pass < passes; ++pass) {
    // pass p of the job: A = slot mA rows I, B = slot mB rows J (square:
    // S0 S0; order-o term: S0 S_o, S_o S0, then S_{p-1} S_{o-p+1}).  The
    // masters are exactly symmetric (both halves are always written with the
    // same value), so the K x BT slab A[I rows][kb ..] is read as rows
    // kb .. kb + BK - 1, columns I BT .. I BT + BT - 1: contiguous 16-byte
    // copies that land in shared memory already K-major.
    int mA, mB;
    simt_job_operands(job, pass, k1, &mA, &mB);
    const T* A = master + (size_t)((mA == 0 ? cur0 : st->cur1[mA - 1]) * (1 + k) + mA) * mat +
                 (size_t)I * BT;
    const T* B = master + (size_t)((mB == 0 ? cur0 : st->cur1[mB - 1]) * (1 + k) + mB) * mat +
                 (size_t)J * BT;
    auto load = [&](int stage, int kb) {
      T* as = slabs + (size_t)stage * 2 * BK * LD;
      T* bs = as + BK * LD;
#pragma unroll
      for (int v = 0; v < NCP; ++v) {
        const int idx = tid + 256 * v;
        const int row = idx / CPR, cq = idx % CPR;
        const size_t g = (size_t)(kb + row) * Np + cq * VW;
        cp_async16(as + row * LD + cq * VW, A + g);
        cp_async16(bs + row * LD + cq * VW, B + g);
      }
    };
    __syncthreads();   // every stage of the previous pass has been read
    // prologue: stages 0 .. SIMT_STAGES - 2 in flight (one group each)
#pragma unroll
    for (int sidx = 0; sidx < SIMT_STAGES - 1; ++sidx) {
      if (sidx < nkb) load(sidx, sidx * BK);
      cp_async_commit();
    }
    for (int it = 0; it < nkb; ++it) {
      cp_async_wait<SIMT_STAGES - 2>();   // stage it has landed (this thread's copies)
      __syncthreads();                    // ... and every thread's; stage it - 1 is free
      {
        const int nx = it + SIMT_STAGES - 1;
        if (nx < nkb) load(nx % SIMT_STAGES, nx * BK);
        cp_async_commit();
      }
      const T* as = slabs + (size_t)(it % SIMT_STAGES) * 2 * BK * LD;
      const T* bs = as + BK * LD;
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T a[TM], b[TM];
#pragma unroll
        for (int m = 0; m < TM; ++m) a[m] = as[kk * LD + frag_index<T, TM>(ty, m)];
#pragma unroll
        for (int m = 0; m < TM; ++m) b[m] = bs[kk * LD + frag_index<T, TM>(tx, m)];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TM; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
    }
    cp_async_wait<0>();   // no copy of this pass left in flight
  }

  // ---- fused epilogue
  const T sg = (T)st->sigma_cur;
  const T om = (T)1 - sg;
  const bool write = job == 0 ? st->plan_write0 != 0 : true;
  double tr = 0.0, bad = 0.0;
  // ||S_new||_F^2 and ||S_old - X||_F^2: in FP64 for the FP64 form; for the
  // FP32 form as exact FP32 products summed with TwoSum compensation (the
  // FP64 rate of the part is low), converted to FP64 once per thread
  double fnew = 0.0, fdiff = 0.0;
  float fn_s = 0.0f, fn_c = 0.0f, fd_s = 0.0f, fd_c = 0.0f;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t r = (int64_t)I * BT + frag_index<T, TM>(ty, i);
#pragma unroll
    for (int j = 0; j < TM; ++j) {
      const int64_t c = (int64_t)J * BT + frag_index<T, TM>(tx, j);
      if (r > c) continue;  // owned by the mirrored element
      const T x = acc[i][j];
      const T old = Sj[(size_t)r * Np + c];
      if (!isfinite((double)x)) bad += 1.0;
      const T nw = sg * x + om * old;
      if constexpr (sizeof(T) == 8) {
        const double w = (r == c) ? 1.0 : 2.0;
        const double dd = (double)old - (double)x;
        fdiff += w * dd * dd;
        if (write) {
          const double dn = (double)nw;
          fnew += w * dn * dn;
        }
      } else {
        const float w = (r == c) ? 1.0f : 2.0f;
        const float dd = (float)old - (float)x;
        {
          const float p = w * dd * dd;
          const float e = w * fmaf(dd, dd, -dd * dd);
          const float tt = fd_s + p;
          const float bp = tt - fd_s;
          fd_c += (fd_s - (tt - bp)) + (p - bp) + e;
          fd_s = tt;
        }
        if (write) {
          const float n1 = (float)nw;
          const float p = w * n1 * n1;
          const float e = w * fmaf(n1, n1, -n1 * n1);
          const float tt = fn_s + p;
          const float bp = tt - fn_s;
          fn_c += (fn_s - (tt - bp)) + (p - bp) + e;
          fn_s = tt;
        }
      }
      if (write) {
        out[(size_t)r * Np + c] = nw;
        if (r != c) out[(size_t)c * Np + r] = nw;
        if (r == c) tr += (double)nw;
      }
    }
  }
  if constexpr (sizeof(T) != 8) {
    fnew = (double)fn_s + (double)fn_c;
    fdiff = (double)fd_s + (double)fd_c;
  }
  double v[4] = {tr, fnew, fdiff, bad};
  block_sum<4, 256>(v, red);
  if (tid == 0) {
    double* p = partials + ((size_t)job * ptiles + blockIdx.x) * kNQ;
#pragma unroll
    for (int q = 0; q < 4; ++q) p[q] = v[q];
  }
}

int simt_tile(int precision) { return precision == DMPT_FP64 ? 64 : 128; }

// Per-device one-time setup: the SIMT layer kernels' dynamic shared memory
// exceeds the default 48 KB limit; thread-safe.
static void simt_setup() {
  constexpr int kDevices = 64;
  static std::once_flag once[kDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevices) return;
  std::call_once(once[dev], [] {
    cudaFuncSetAttribute(layer_simt_kernel<double, 4, 8>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         simt_smem_bytes<double, 4, 8>());
    cudaFuncSetAttribute(layer_simt_kernel<float, 8, 16>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         simt_smem_bytes<float, 8, 16>());
  });
}

cudaError_t launch_layer_simt(const Layout& L, void* ws, cudaStream_t s, int64_t* entries,
                              double* pass_flops) {
  char* base = (char*)ws;
  State* st = (State*)(base + L.off_state);
  double* partials = (double*)(base + L.off_partials);
  const int bt = simt_tile(L.precision);
  dim3 grid((unsigned)upper_tiles(L.Np, bt), 1 + L.k);
  constexpr int smem64 = simt_smem_bytes<double, 4, 8>();
  constexpr int smem32 = simt_smem_bytes<float, 8, 16>();
  static_assert(2 * smem32 <= 227 * 1024, "two FP32 blocks per SM");
  simt_setup();
  if (L.precision == DMPT_FP64)
    layer_simt_kernel<double, 4, 8><<<grid, 256, smem64, s>>>(
        st, (double*)(base + L.off_master), L.Np, L.k, partials, L.partial_tiles);
  else
    layer_simt_kernel<float, 8, 16><<<grid, 256, smem32, s>>>(
        st, (float*)(base + L.off_master), L.Np, L.k, partials, L.partial_tiles);
  if (entries) *entries = upper_tiles(L.Np, bt);
  if (pass_flops) *pass_flops = (double)upper_tiles(L.Np, bt) * bt * bt * (double)L.Np * 2.0;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Dual split of the initial layer (Sec. II C, Eq. (DualMat2)):
//   hi = R16[2^e X],  lo = R16[2^e X - hi]   (round to nearest even),
// with e = s0_exp for S0 and s1_exp_cur[k] for S1_k (exact power-of-two
// scaling keeps FP16 values in range; BF16 uses e = 0).

template <typename H16>
__device__ __forceinline__ H16 to16(float x);
template <>
__device__ __forceinline__ __half to16<__half>(float x) { return __float2half_rn(x); }
template <>
__device__ __forceinline__ __nv_bfloat16 to16<__nv_bfloat16>(float x) {
  return __float2bfloat16_rn(x);
}
__device__ __forceinline__ float from16(__half x) { return __half2float(x); }
__device__ __forceinline__ float from16(__nv_bfloat16 x) { return __bfloat162float(x); }

__device__ __forceinline__ unsigned short bits16(__half x) { return __half_as_ushort(x); }
__device__ __forceinline__ unsigned short bits16(__nv_bfloat16 x) {
  return __bfloat16_as_ushort(x);
}

// Elements idx .. idx + 3 (idx a multiple of 4) of a master: x = src 2^e,
// hi = x rounded to 16 bits, lo = (x - hi) rounded to 16 bits.
template <typename H16>
__device__ __forceinline__ void split4(const float* __restrict__ src, unsigned short* hi,
                                       unsigned short* lo, size_t idx, int e) {
  const float4 v = *reinterpret_cast<const float4*>(src + idx);
  const float x[4] = {ldexpf(v.x, e), ldexpf(v.y, e), ldexpf(v.z, e), ldexpf(v.w, e)};
  unsigned short hb[4], lb[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const H16 h = to16<H16>(x[t]);
    hb[t] = bits16(h);
    lb[t] = bits16(to16<H16>(x[t] - from16(h)));
  }
  *reinterpret_cast<uint2*>(hi + idx) =
      make_uint2(hb[0] | ((unsigned)hb[1] << 16), hb[2] | ((unsigned)hb[3] << 16));
  *reinterpret_cast<uint2*>(lo + idx) =
      make_uint2(lb[0] | ((unsigned)lb[1] << 16), lb[2] | ((unsigned)lb[3] << 16));
}

template <typename H16>
__global__ void split_kernel(const State* st, const float* __restrict__ master,
                             unsigned short* ops, int64_t Np, int k, int first_job) {
  const size_t mat = (size_t)Np * Np;   // a multiple of 4
  const int m = first_job + blockIdx.y;  // matrix: 0 = S0, 1 + j = S1_j
  const int cur = m == 0 ? st->cur0 : st->cur1[m - 1];
  const int e = m == 0 ? st->s0_exp : st->s1_exp_cur[m - 1];
  const float* src = master + (size_t)(cur * (1 + k) + m) * mat;
  const int zh = m == 0 ? st->z0_cur : zslice(cur, m, 0, k);
  unsigned short* hi = ops + (size_t)zh * mat;
  unsigned short* lo = ops + (size_t)(zh + 1) * mat;
  for (size_t i = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; i < mat;
       i += (size_t)gridDim.x * blockDim.x * 4)
    split4<H16>(src, hi, lo, i, e);
}

cudaError_t launch_split(const Layout& L, void* ws, int first_job, cudaStream_t s, int jobs) {
  char* base = (char*)ws;
  const State* st = (const State*)(base + L.off_state);
  dim3 grid(152 * 4, jobs < 0 ? 1 + L.k - first_job : jobs);
  if (L.precision == DMPT_DUAL_FP16)
    split_kernel<__half><<<grid, 256, 0, s>>>(st, (const float*)(base + L.off_master),
                                              (unsigned short*)(base + L.off_ops16), L.Np, L.k,
                                              first_job);
  else
    split_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(st, (const float*)(base + L.off_master),
                                                     (unsigned short*)(base + L.off_ops16),
                                                     L.Np, L.k, first_job);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Whole-matrix readers of the masters.  The tensor-core layer epilogue keeps
// an FP32 master in one orientation only (element (r, c) at (max, min): the
// lower triangle with the diagonal); the other kernels write both.  So a
// reader takes output tile (bi, bj) (kSymTile x kSymTile, 256 threads) from
// the lower tile (max(bi, bj), min(bi, bj)): loaded row by row (coalesced,
// every load of the tile in flight at once) into shared memory, written row
// by row, transposed where the output tile lies above the diagonal.
// `put(r, c, v)` writes the value of element (r, c), r, c < n.
constexpr int kSymTile = 64;
template <typename T, class Put>
__device__ __forceinline__ void sym_tile(const T* __restrict__ src, int64_t Np, int64_t n,
                                         int64_t bi, int64_t bj, T (*t)[kSymTile + 1], Put put) {
  constexpr int TS = kSymTile, RS = 256 / TS, RPT = TS / RS;   // 64 x 4 threads, 16 rows each
  const int tx = threadIdx.x % TS, ty = threadIdx.x / TS;
  const int64_t lr = TS * (bi > bj ? bi : bj), lc = TS * (bi > bj ? bj : bi);
  T v[RPT];
#pragma unroll
  for (int j = 0; j < RPT; ++j) v[j] = src[(lr + ty + RS * j) * Np + lc + tx];
#pragma unroll
  for (int j = 0; j < RPT; ++j) t[ty + RS * j][tx] = v[j];
  __syncthreads();
#pragma unroll
  for (int j = 0; j < RPT; ++j) {
    const int i = ty + RS * j;
    const int64_t r = TS * bi + i, c = TS * bj + tx;
    if (r < n && c < n) {
      const T x = bi > bj ? t[i][tx] : (bi < bj ? t[tx][i] : (tx <= i ? t[i][tx] : t[tx][i]));
      put(r, c, x);
    }
  }
  __syncthreads();   // the block's next tile reuses t
}

// ---------------------------------------------------------------------------
// Checkpoints of the S0 recursion (ckpt_every = k >= 2) and the recompute of a
// segment of states from its checkpoint in the backward pass.

__global__ void ckpt_store_kernel(const State* st, const float4* __restrict__ master,
                                  float4* ckpt, int64_t Np, int lk) {
  if (!st->ckpt_pending) return;
  const int slot = st->d0_updates / st->ckpt_k;
  if (slot >= st->ckpt_slots) return;   // cannot happen: slots cover max_layers / k + 1
  const size_t n4 = (size_t)Np * Np / 4;
  const float4* src = master + (size_t)st->cur0 * (1 + lk) * n4;
  float4* dst = ckpt + (size_t)slot * n4;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

cudaError_t launch_ckpt_store(const Layout& L, void* ws, cudaStream_t s) {
  char* base = (char*)ws;
  ckpt_store_kernel<<<152 * 4, 256, 0, s>>>((const State*)(base + L.off_state),
                                            (const float4*)(base + L.off_master),
                                            (float4*)(base + L.off_ckpt), L.Np, L.k);
  return cudaGetLastError();
}

// Checkpoint c (state a) into S0 master buffer 0; it becomes the current S0
// and its 16-bit copies go to the first tape slot (split afterwards).
__global__ void seg_load_kernel(State* st, float4* master, const float4* __restrict__ ckpt,
                                int64_t Np, int c, int a) {
  const size_t n4 = (size_t)Np * Np / 4;
  const float4* src = ckpt + (size_t)c * n4;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (size_t)gridDim.x * blockDim.x)
    master[i] = src[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->cur0 = 0;
    st->z0_cur = st->tape_base;
    st->adj_seg_a = a;
  }
}

// The upper triangle of an Np x Np master from its lower triangle (a
// checkpoint of a state that a tensor-core layer wrote holds only the lower
// one; the hi/lo split that follows a reload reads the whole matrix).
__global__ void __launch_bounds__(256) mirror_lower_kernel(float* M, int64_t Np) {
  __shared__ float t[kSymTile][kSymTile + 1];
  const int64_t tb = Np / kSymTile;
  for (int64_t tile = blockIdx.x; tile < tb * tb; tile += gridDim.x) {
    const int64_t bi = tile / tb, bj = tile % tb;
    if (bi > bj) continue;   // uniform across the block: lower tiles are only read
    sym_tile<float>(M, Np, Np, bi, bj, t, [&](int64_t r, int64_t c, float v) { M[r * Np + c] = v; });
  }
}

// M[r][c] = M[c][r] for r > c, count matrices: lower output tile (bi, bj)
// from upper tile (bj, bi), loaded row by row and transposed through shared
// memory; a diagonal tile mirrors its own upper half.
__global__ void __launch_bounds__(256) mirror_upper_kernel(double* M, int64_t n, int64_t ld) {
  constexpr int TS = kSymTile, RS = 256 / TS, RPT = TS / RS;
  __shared__ double t[TS][TS + 1];
  double* A = M + (size_t)blockIdx.y * n * ld;
  const int tx = threadIdx.x % TS, ty = threadIdx.x / TS;
  const int64_t tb = (n + TS - 1) / TS;
  for (int64_t tile = blockIdx.x; tile < tb * tb; tile += gridDim.x) {
    const int64_t bi = tile / tb, bj = tile % tb;
    if (bi < bj) continue;   // uniform across the block: upper tiles are only read
    double v[RPT];
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
      const int64_t r = TS * bj + ty + RS * j, c = TS * bi + tx;   // upper tile (bj, bi)
      v[j] = (r < n && c < n) ? A[r * ld + c] : 0.0;
    }
#pragma unroll
    for (int j = 0; j < RPT; ++j) t[ty + RS * j][tx] = v[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
      const int i = ty + RS * j;
      const int64_t r = TS * bi + i, c = TS * bj + tx;
      if (r < n && c < n && r > c) A[r * ld + c] = t[tx][i];
    }
    __syncthreads();
  }
}

cudaError_t launch_mirror_upper(double* M, int64_t n, int64_t ld, int count, cudaStream_t s) {
  if (count < 1 || n < 1) return cudaSuccess;
  mirror_upper_kernel<<<dim3(152 * 8, count), 256, 0, s>>>(M, n, ld);
  return cudaGetLastError();
}

cudaError_t launch_seg_load(const Layout& L, void* ws, int c, int a, cudaStream_t s) {
  if (c < 0 || c >= L.ckpt_slots) return cudaErrorInvalidValue;
  char* base = (char*)ws;
  seg_load_kernel<<<152 * 4, 256, 0, s>>>((State*)(base + L.off_state),
                                          (float4*)(base + L.off_master),
                                          (const float4*)(base + L.off_ckpt), L.Np, c, a);
  mirror_lower_kernel<<<152 * 16, 256, 0, s>>>((float*)(base + L.off_master), L.Np);
  return cudaGetLastError();
}

// Plan the recompute of S_m = sigma_m S_{m-1}^2 + (1 - sigma_m) S_{m-1}: the
// square job only, S0 update stored, 16-bit copies into tape slot m - a.
__global__ void recompute_plan_kernel(State* st, int m, int a, int64_t item_base) {
  st->round_ctr = 0u;
  st->item_base = item_base;
  st->plan_square = 1;
  st->plan_write0 = 1;
  st->sigma_cur = st->sigma[m];
  for (int j = 0; j < kMaxK; ++j) st->plan_resp[j] = 0;
  st->z0_next = st->tape_base + 2 * (m - a);
}

// After a recompute layer: the new state is the current S0.
__global__ void recompute_done_kernel(State* st) {
  st->round_ctr = 0u;
  st->item_base = 0;
  st->cur0 ^= 1;
  st->z0_cur = st->z0_next;
  st->plan_square = 0;
  st->plan_write0 = 0;
  if (st->timeout_flag) {
    st->status = DMPT_ETIMEOUT;
    st->done = 1;
  }
}

cudaError_t launch_recompute_plan(const Layout& L, void* ws, int m, int a, int64_t item_base,
                                  cudaStream_t s) {
  recompute_plan_kernel<<<1, 1, 0, s>>>((State*)((char*)ws + L.off_state), m, a, item_base);
  return cudaGetLastError();
}

cudaError_t launch_recompute_done(const Layout& L, void* ws, cudaStream_t s) {
  recompute_done_kernel<<<1, 1, 0, s>>>((State*)((char*)ws + L.off_state));
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Adjoint of the S0 recursion (backward pass of L = Tr[G P]).
//   Gbar = (G + G^T) / 2 into response slot 1, buffer 0 (FP32 master), with
//   ||Gbar||_F^2 partial sums; and at the end dL/dH = -Gbar / (eps_N - eps_1)
//   (S0 = (eps_N I - H) / (eps_N - eps_1), bounds held fixed).

__global__ void __launch_bounds__(256) adj_init_kernel(const double* __restrict__ G, float* master,
                                                       int64_t n, int64_t Np, int64_t ld, int lk,
                                                       double* partials, int64_t ptiles) {
  __shared__ double up[32][33];
  __shared__ double dn[32][33];
  __shared__ double red[2 * 256];
  const size_t mat = (size_t)Np * Np;
  float* dst = master + (size_t)1 * mat;   // buffer 0, slot 1
  (void)lk;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t TB = Np / 32;
  const int64_t pairs = TB * (TB + 1) / 2;
  double f = 0.0, bad = 0.0;
  for (int64_t tp = blockIdx.x; tp < pairs; tp += gridDim.x) {
    int64_t bj = (int64_t)((sqrt(8.0 * (double)tp + 1.0) - 1.0) * 0.5);
    while ((bj + 1) * (bj + 2) / 2 <= tp) ++bj;
    while (bj * (bj + 1) / 2 > tp) --bj;
    const int64_t bi = tp - bj * (bj + 1) / 2;
    for (int i = 0; i < 4; ++i) {
      const int rl = ty + 8 * i;
      const int64_t r = bi * 32 + rl, c = bj * 32 + tx;
      const int64_t r2 = bj * 32 + rl, c2 = bi * 32 + tx;
      up[rl][tx] = (r < n && c < n) ? G[r * ld + c] : 0.0;
      dn[rl][tx] = (r2 < n && c2 < n) ? G[r2 * ld + c2] : 0.0;
    }
    __syncthreads();
    for (int i = 0; i < 4; ++i) {
      const int rl = ty + 8 * i;
      const int64_t r = bi * 32 + rl, c = bj * 32 + tx;
      // (G + G^T)/2 at (r, c): up[rl][tx] and the transposed element dn[tx][rl]
      const float v = (float)(0.5 * (up[rl][tx] + dn[tx][rl]));
      dst[(size_t)r * Np + c] = v;
      const double wgt = bi < bj ? 2.0 : 1.0;
      f += wgt * (double)v * (double)v;
      if (!isfinite(v)) bad += 1.0;
      if (bi < bj) {
        const float vt = (float)(0.5 * (up[tx][rl] + dn[rl][tx]));
        dst[(size_t)(bj * 32 + rl) * Np + bi * 32 + tx] = vt;
      }
    }
    __syncthreads();
  }
  double v[2] = {f, bad};
  block_sum<2, 256>(v, red);
  if (threadIdx.x == 0) {
    double* p = partials + ((size_t)1 * ptiles + blockIdx.x) * kNQ;
    p[kQTrace] = 0.0;
    p[kQFroNew] = v[0];
    p[kQFroDiff] = 0.0;
    p[kQBad] = v[1];
  }
}

cudaError_t launch_adj_init(const Layout& L, void* ws, const double* G, int64_t ld, int blocks,
                            cudaStream_t s) {
  char* base = (char*)ws;
  adj_init_kernel<<<blocks, 256, 0, s>>>(G, (float*)(base + L.off_master), L.n, L.Np, ld, L.k,
                                         (double*)(base + L.off_partials), L.partial_tiles);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) adj_finalize_kernel(const State* st,
                                                           const float* __restrict__ master,
                                                           double* dLdH, int64_t n, int64_t Np,
                                                           int64_t ld, int lk) {
  __shared__ float t[kSymTile][kSymTile + 1];
  const size_t mat = (size_t)Np * Np;
  const float* src = master + (size_t)(st->cur1[0] * (1 + lk) + 1) * mat;
  const double scale = -1.0 / (st->epsN - st->eps1);
  const int64_t tb = (n + kSymTile - 1) / kSymTile;
  for (int64_t tile = blockIdx.x; tile < tb * tb; tile += gridDim.x)
    sym_tile<float>(src, Np, n, tile / tb, tile % tb, t, [&](int64_t r, int64_t c, float v) {
      dLdH[r * ld + c] = scale * (double)v;
    });
}

cudaError_t launch_adj_finalize(const Layout& L, void* ws, double* dLdH, int64_t ld,
                                cudaStream_t s) {
  char* base = (char*)ws;
  adj_finalize_kernel<<<152 * 16, 256, 0, s>>>((const State*)(base + L.off_state),
                                              (const float*)(base + L.off_master), dLdH, L.n,
                                              L.Np, ld, L.k);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Outputs: P = S0, P1_k = S1_k (orthogonal basis, Z = I), as float64.

// Output element (r, c) of matrix y (0 = P, 1 + j = P1_j) from master value v;
// the complement form (the recursion ran on I - P) gives P = I - S0,
// P_o = -S_o.
__device__ __forceinline__ double out_value(double v, int64_t r, int64_t c, int y, bool hole) {
  return !hole ? v : (y == 0 ? (r == c ? 1.0 : 0.0) - v : -v);
}

template <typename T>
__global__ void __launch_bounds__(256) finalize_kernel(const State* st,
                                                       const T* __restrict__ master, double* P,
                                                       double* P1, int64_t n, int64_t Np,
                                                       int64_t ld, int k, int slot0) {
  // k: layout slots; grid.y = 1 + the number of blocks written to P1, which
  // come from slots slot0, slot0 + 1, ...; kSymTile x kSymTile output tiles
  __shared__ T t[kSymTile][kSymTile + 1];
  const size_t mat = (size_t)Np * Np;
  const int y = blockIdx.y;
  if (y == 0 && P == nullptr) return;
  const int m = y == 0 ? 0 : slot0 + y - 1;
  const int cur = m == 0 ? st->cur0 : st->cur1[m - 1];
  const T* src = master + (size_t)(cur * (1 + k) + m) * mat;
  double* dst = y == 0 ? P : P1 + (size_t)(y - 1) * n * ld;
  const bool hole = st->hole != 0;
  const int64_t tb = (n + kSymTile - 1) / kSymTile;
  for (int64_t tile = blockIdx.x; tile < tb * tb; tile += gridDim.x)
    sym_tile<T>(src, Np, n, tile / tb, tile % tb, t, [&](int64_t r, int64_t c, T v) {
      dst[r * ld + c] = out_value((double)v, r, c, y, hole);
    });
}

cudaError_t launch_finalize(const Layout& L, void* ws, double* P, double* P1, int64_t ld,
                            int k_out, cudaStream_t s, int slot0) {
  char* base = (char*)ws;
  const State* st = (const State*)(base + L.off_state);
  dim3 grid(152 * 16, 1 + k_out);
  if (L.precision == DMPT_FP64)
    finalize_kernel<double><<<grid, 256, 0, s>>>(st, (const double*)(base + L.off_master), P,
                                                 P1, L.n, L.Np, ld, L.k, slot0);
  else
    finalize_kernel<float><<<grid, 256, 0, s>>>(st, (const float*)(base + L.off_master), P, P1,
                                                L.n, L.Np, ld, L.k, slot0);
  return cudaGetLastError();
}

// n_occ = 0 (full = 0) or n_occ = n (full = 1): P = 0 or I, P1 = 0.
__global__ void trivial_kernel(int64_t n, int k, int64_t ld, int full, double* P, double* P1) {
  const int m = blockIdx.y;
  if (m == 0 && P == nullptr) return;
  double* dst = m == 0 ? P : P1 + (size_t)(m - 1) * n * ld;
  const int64_t total = n * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / n, c = i - r * n;
    dst[r * ld + c] = (m == 0 && full && r == c) ? 1.0 : 0.0;
  }
}

cudaError_t launch_trivial(int64_t n, int k, int64_t ld, int full, double* P, double* P1,
                           cudaStream_t s) {
  dim3 grid(152, 1 + k);
  trivial_kernel<<<grid, 256, 0, s>>>(n, k, ld, full, P, P1);
  return cudaGetLastError();
}

}  // namespace dmpt

namespace dmpt {
// *flag = 1 when every instance's control block (at base + offs[i]) says done
__global__ void batch_all_done_kernel(const char* base, const long long* offs, int count,
                                      int* flag) {
  int all = 1;
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    const State* st = (const State*)(base + offs[i]);
    if (!st->done) all = 0;
  }
  all = __syncthreads_and(all);
  if (threadIdx.x == 0) *flag = all;
}

cudaError_t launch_batch_all_done(const void* base, const long long* offs, int count, int* flag,
                                  cudaStream_t s) {
  batch_all_done_kernel<<<1, 256, 0, s>>>((const char*)base, offs, count, flag);
  return cudaGetLastError();
}

// out[b] = the control block at base + offs[b] (one block per instance), so
// that the host reads every instance's state with one copy.
__global__ void gather_states_kernel(const char* base, const long long* offs, State* out) {
  static_assert(sizeof(State) % 4 == 0, "State copied as words");
  const unsigned* src = (const unsigned*)(base + offs[blockIdx.x]);
  unsigned* dst = (unsigned*)(out + blockIdx.x);
  for (int i = threadIdx.x; i < (int)(sizeof(State) / 4); i += blockDim.x) dst[i] = src[i];
}

cudaError_t launch_gather_states(const void* base, const long long* offs, int count, State* out,
                                 cudaStream_t s) {
  if (count < 1) return cudaSuccess;
  gather_states_kernel<<<count, 256, 0, s>>>((const char*)base, offs, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batched set-up and outputs of the batch path (one launch per step for every
// instance; the values are those of the single-instance kernels above).

// The instance that owns unit u: the largest i with first[i] <= u
// (first[0] = 0 <= u < first[count]).
__device__ __forceinline__ int batch_find(const int64_t* __restrict__ first, int count,
                                          int64_t u) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= u)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// One block per instance: a zeroed control block with its fields, the bounds
// keys, and zero partial sums for the initial layer's blocks that hold no
// tile pair.
__global__ void __launch_bounds__(256) batch_setup_kernel(const BatchInst* __restrict__ bi,
                                                          BatchCommon c) {
  const BatchInst& b = bi[blockIdx.x];
  static_assert(sizeof(State) % 4 == 0, "State zeroed as words");
  unsigned* w = reinterpret_cast<unsigned*>(b.st);
  for (int i = threadIdx.x; i < (int)(sizeof(State) / 4); i += blockDim.x) w[i] = 0u;
  const int64_t empty = (int64_t)(kInitBlocks - b.init_blocks) * kNQ;
  for (int j = 0; j <= b.k; ++j) {
    double* p = b.partials + ((size_t)j * b.ptiles + b.init_blocks) * kNQ;
    for (int64_t e = threadIdx.x; e < empty; e += blockDim.x) p[e] = 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    state_init_fields(b.st, b.k, c.max_layers, c.precision, b.n_occ, c.c_pt, c.c_d0, 0,
                      4 * (1 + b.layout_k), 0, b.layout_k, b.n, 1, 0, c.fo, b.hole);
    long long* key = reinterpret_cast<long long*>(&b.st->eps1);
    key[0] = dkey(INFINITY);
    key[1] = dkey(-INFINITY);
  }
}

// Gershgorin discs (as bounds_rows_kernel): one warp per kBatchRows rows of
// one instance, each row's radius summed in the same lane order.
__global__ void batch_bounds_rows_kernel(const BatchInst* __restrict__ bi,
                                         const int64_t* __restrict__ first, int count) {
  const int lane = threadIdx.x & 31;
  const int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (u >= first[count]) return;   // uniform across the warp
  const int i = batch_find(first, count, u);
  const BatchInst& b = bi[i];
  const int64_t r0 = (u - first[i]) * kBatchRows;
  double lo = INFINITY, hi = -INFINITY;
  for (int64_t r = r0; r < r0 + kBatchRows && r < b.n; ++r) {
    const double* row = b.H + r * b.ld;
    double s = 0.0;
    for (int64_t j = lane; j < b.n; j += 32) s += fabs(row[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const double d = row[r];
    const double rad = s - fabs(d);
    lo = fmin(lo, d - rad);
    hi = fmax(hi, d + rad);
  }
  if (lane == 0) {
    long long* key = reinterpret_cast<long long*>(&b.st->eps1);
    atomicMin(&key[0], dkey(lo));
    atomicMax(&key[1], dkey(hi));
  }
}

__global__ void batch_bounds_fin_kernel(const BatchInst* __restrict__ bi, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  long long* key = reinterpret_cast<long long*>(&bi[i].st->eps1);
  const double lo = dkey_inv(key[0]);
  const double hi = dkey_inv(key[1]);
  bi[i].st->eps1 = lo;
  bi[i].st->epsN = hi;
}

// Initial layer: unit u is virtual block u - first[i] of instance i's grid of
// kInitBlocks blocks.
template <typename T>
__global__ void __launch_bounds__(256) batch_init_kernel(const BatchInst* __restrict__ bi,
                                                         const int64_t* __restrict__ first,
                                                         int count) {
  const int64_t u = blockIdx.x;
  const int i = batch_find(first, count, u);
  const BatchInst& b = bi[i];
  init_body<T>(b.st, static_cast<T*>(b.master), b.H, b.H1, b.n, b.Np, b.ld, b.k, 0, nullptr, 0,
               b.partials, b.ptiles, u - first[i], kInitBlocks);
}

__global__ void __launch_bounds__(256) batch_decide_init_kernel(const BatchInst* __restrict__ bi) {
  __shared__ double red[kNQ * 256];
  __shared__ double sums[kMaxK + 1][kNQ];
  const BatchInst& b = bi[blockIdx.x];
  decide_body(b.st, b.partials, b.ptiles, kInitBlocks, kDecideInit, red, sums);
}

// 16-bit split of matrices 0 .. layout k (as split_kernel), kBatchChunk
// elements per block, four per thread and step.
template <typename H16>
__global__ void __launch_bounds__(256) batch_split_kernel(const BatchInst* __restrict__ bi,
                                                          const int64_t* __restrict__ first,
                                                          int count) {
  const int64_t u = blockIdx.x;
  const int i = batch_find(first, count, u);
  const BatchInst& b = bi[i];
  const State* st = b.st;
  const int lk = b.layout_k;
  const size_t mat = (size_t)b.Np * b.Np;   // a multiple of 4
  const int64_t cpm = (int64_t)((mat + kBatchChunk - 1) / kBatchChunk);
  const int64_t c = u - first[i];
  const int m = (int)(c / cpm);
  const size_t e0 = (size_t)(c - (int64_t)m * cpm) * kBatchChunk;
  const int cur = m == 0 ? st->cur0 : st->cur1[m - 1];
  const int e = m == 0 ? st->s0_exp : st->s1_exp_cur[m - 1];
  const float* src = static_cast<const float*>(b.master) + (size_t)(cur * (1 + lk) + m) * mat;
  const int zh = m == 0 ? st->z0_cur : zslice(cur, m, 0, lk);
  unsigned short* hi = b.ops + (size_t)zh * mat;
  unsigned short* lo = b.ops + (size_t)(zh + 1) * mat;
#pragma unroll
  for (int q = 0; q < kBatchChunk / (4 * 256); ++q) {
    const size_t idx = e0 + (size_t)(q * 256 + threadIdx.x) * 4;
    if (idx >= mat) break;
    split4<H16>(src, hi, lo, idx, e);
  }
}

// Outputs (as finalize_kernel with slot0 = 1): unit c of matrix y (0 = P,
// 1 + j = P1_j) is output tile c of that matrix (kSymTile x kSymTile tiles,
// row-major).
template <typename T>
__global__ void __launch_bounds__(256) batch_finalize_kernel(const BatchInst* __restrict__ bi,
                                                             const int64_t* __restrict__ first,
                                                             int count) {
  __shared__ T t[kSymTile][kSymTile + 1];
  const int64_t u = blockIdx.x;
  const int i = batch_find(first, count, u);
  const BatchInst& b = bi[i];
  const int64_t n = b.n;
  const int64_t tb = (n + kSymTile - 1) / kSymTile;
  const int64_t c = u - first[i];
  const int y = (int)(c / (tb * tb));
  if (y == 0 && b.P == nullptr) return;
  const int64_t tile = c - (int64_t)y * tb * tb;
  const State* st = b.st;
  const size_t mat = (size_t)b.Np * b.Np;
  const int cur = y == 0 ? st->cur0 : st->cur1[y - 1];
  const T* src = static_cast<const T*>(b.master) + (size_t)(cur * (1 + b.layout_k) + y) * mat;
  double* dst = y == 0 ? b.P : b.P1 + (size_t)(y - 1) * n * b.ld;
  const bool hole = st->hole != 0;
  const int64_t ld = b.ld;
  sym_tile<T>(src, b.Np, n, tile / tb, tile % tb, t, [&](int64_t r, int64_t cc, T v) {
    dst[r * ld + cc] = out_value((double)v, r, cc, y, hole);
  });
}

cudaError_t launch_batch_setup(const BatchInst* bi, const int64_t* first, int count,
                               const BatchCommon& c, const int64_t* units, bool dual, bool bf16,
                               cudaStream_t s) {
  if (count < 1) return cudaSuccess;
  const int64_t* f_rows = first + kBsRows * (count + 1);
  const int64_t* f_init = first + kBsInit * (count + 1);
  const int64_t* f_split = first + kBsSplit * (count + 1);
  batch_setup_kernel<<<count, 256, 0, s>>>(bi, c);
  batch_bounds_rows_kernel<<<(unsigned)((units[kBsRows] * 32 + 255) / 256), 256, 0, s>>>(
      bi, f_rows, count);
  batch_bounds_fin_kernel<<<(count + 255) / 256, 256, 0, s>>>(bi, count);
  if (c.precision == DMPT_FP64)
    batch_init_kernel<double><<<(unsigned)units[kBsInit], 256, 0, s>>>(bi, f_init, count);
  else
    batch_init_kernel<float><<<(unsigned)units[kBsInit], 256, 0, s>>>(bi, f_init, count);
  batch_decide_init_kernel<<<count, 256, 0, s>>>(bi);
  if (dual && units[kBsSplit] > 0) {
    if (bf16)
      batch_split_kernel<__nv_bfloat16><<<(unsigned)units[kBsSplit], 256, 0, s>>>(bi, f_split,
                                                                                  count);
    else
      batch_split_kernel<__half><<<(unsigned)units[kBsSplit], 256, 0, s>>>(bi, f_split, count);
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_finalize(const BatchInst* bi, const int64_t* first, int count,
                                  int64_t units, bool fp64, cudaStream_t s) {
  if (count < 1 || units < 1) return cudaSuccess;
  const int64_t* f_out = first + kBsOut * (count + 1);
  if (fp64)
    batch_finalize_kernel<double><<<(unsigned)units, 256, 0, s>>>(bi, f_out, count);
  else
    batch_finalize_kernel<float><<<(unsigned)units, 256, 0, s>>>(bi, f_out, count);
  return cudaGetLastError();
}
}  // namespace dmpt
