// Shared definitions of the streaming ST-HOSVD library (device control block, helpers).
//
// Design: every data-dependent decision of the streaming update (Alg. 4's ||E_k|| <= eps test,
// the rank cut of Alg. 1, Alg. 3's q <= eps test and the resulting ranks) is taken on the
// device and recorded in the control block `Ctl`, which every kernel reads. Kernels are launched
// with grids sized from capacities and loop over the live extent read from `Ctl`, so one update
// is a fixed sequence of launches with no host synchronization (and can be captured in a graph).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define TK_MAXD 8
#define TK_STREAM_CAP_MAX 512   // streaming-rank capacity limit (secular solver sizing)
#define TK_N_MAX 512            // spatial mode size limit (eigensolver sizing)

// Latched device status codes (same values as tucker_status).
#define TK_OK 0
#define TK_ECAPACITY 3
#define TK_ENUMERIC 4
#define TK_ETIMEOUT 5

struct Ctl {
  // ---- configuration (written at creation) ----
  int d;                    // number of modes
  int n[TK_MAXD];           // spatial mode sizes n_1..n_{d-1} (index 0..d-2)
  int cap[TK_MAXD];         // rank capacities (index d-1 = streaming mode)
  long long core_cap;       // capacity of prod_{k<d} r_k
  int steps_cap;            // capacity of n_d
  int ldc;                  // leading dimension (row stride) of C and V rows (= cap[d-1])
  double tau;
  double eps_m;
  int tx, tw;               // bytes of the slice type and of the work type
  long long N;              // elements of one slice
  // ---- state ----
  int r[TK_MAXD];           // current ranks
  int nd;                   // n_d: rows of U_d
  int cbuf;                 // which C/V ping-pong buffer holds the state
  int ubuf;                 // which U_d ping-pong buffer holds the state
  int status;               // latched error (0 = ok)
  int xbuf;                 // D*-buffer holding the input of the current spatial mode (-1: slice)
  int init_nt;              // > 0 only during the batch ST-HOSVD: number of initial slices
  int tcmask;               // bit k: tensor-core projection maps exist for spatial mode k
  int etmask;               // bit k: tensor-core residual-Gram maps exist for spatial mode k
  // ---- per-update record ----
  int rold[TK_MAXD];        // ranks when the update started
  double y2;                // ||Y||^2
  double eps;               // tau ||Y|| / sqrt(d)
  double e2[TK_MAXD];       // ||E_k||^2
  int grew[TK_MAXD];        // ||E_k|| > eps
  int radd[TK_MAXD];        // r'_k
  double disc[TK_MAXD];     // discarded energy of mode k
  double q2;                // ||e||^2 after re-orthogonalisation against V
  double q;                 // ||e||
  int aug;                  // q > eps
  int rnew_d;               // streaming rank after the update
  double dropped;           // energy removed by the numerical-rank cut of the compact SVD
  // ---- accumulators (Prop. 1, Prop. 2, App. D) ----
  double err2;              // running squared error bound
  double data2;             // ||X||^2 of all data seen
  long long nupdates;
  // ---- algorithmic bytes per phase, accumulated by every update (see k_end_update) ----
  double acc_bytes[8];
  // ---- completion tickets of the cross-block reductions (zero between launches) ----
  unsigned ticket[4];
  // ---- Alg. 1's tails of the grown modes: tail at r'_k - 1 (the tail at r'_k is disc[k]) ----
  double tail_prev[TK_MAXD];
  // ---- growth eigensolver of the mixed form (k_eig_sub / k_eig_refine): eig_m[k] candidate
  // eigenvectors in W, eig_it[k] subspace iterations, eig_fb[k] = 1 when the full tridiagonal
  // solver must decide instead ----
  int eig_m[TK_MAXD];
  int eig_it[TK_MAXD];
  int eig_fb[TK_MAXD];
  // ---- decision replay (a test hook): branches and cuts forced on the next update, written
  // by the host before the update and cleared by k_end_update. rp_grow[k] < 0 keeps mode k's
  // own decision, 0 forces ||E_k|| <= eps, r > 0 forces growth by r'_k = r; rp_aug < 0 keeps
  // Alg. 3's own branch, 0 forces q <= eps, 1 forces q > eps ----
  int rp_on;
  int rp_grow[TK_MAXD];
  int rp_aug;
  // ---- per-update log (device array of StepRec, one per update since the initial ST-HOSVD;
  // written by k_end_update while nupdates < log_cap) ----
  struct StepRec* log;
  long long log_cap;
  // ---- slice of the current update when the update runs as a CUDA graph (written by one
  // host-to-device copy before each launch): TMA descriptor of the slice as a row-major
  // (N / n_1) x n_1 FP32 matrix (only with the tensor-core mode-1 pass) and its address ----
  alignas(128) unsigned char ymap[128];
  const void* yptr;
  // ---- FP16-split tensor-core passes: x16e[k] is the exponent sigma of the power of two that
  // scales mode k's input before its FP16 split; xmax[k] the largest |x| of that input seen by
  // the update's pass A (float bits, atomicMax; reset by k_begin_update) ----
  int x16e[TK_MAXD];
  unsigned xmax[TK_MAXD];
  // ---- test hook: nonzero makes the next mode-1 tensor-core pass A withhold its loads, so that
  // every wait of its consumers runs out (the bounded-wait path; see tucker_test_stall_next) ----
  int test_stall;
  // ---- block update: blk slices in the current update (1 for a single slice; the spatial modes
  // take them as one tensor with a trailing mode of size blk), and the row of the block whose
  // incremental-SVD step runs ----
  int blk;
  int row;
};

// FP16 scale window: a pass's input scaled by 2^sigma must have its largest |x| in
// [2^1, 2^15) (FP16's largest finite value is 65504). sigma for a largest |x| of exponent e puts
// it at 2^8.
__host__ __device__ __forceinline__ int x16_sigma_for(int e) {
  const int s = 8 - e;
  return s < -100 ? -100 : (s > 100 ? 100 : s);
}
__host__ __device__ __forceinline__ bool x16_in_window(int e, int sigma) {
  const int s = e + sigma;
  return s >= 1 && s <= 14;
}
// Exponent floor(log2 x) of a positive float given by its bits (subnormals count as -127).
__host__ __device__ __forceinline__ int x16_exp_of_bits(unsigned b) { return (int)((b >> 23) & 255u) - 127; }

// One update's decisions as the host reads them back (same layout as tucker_step_record).
struct StepRec {
  long long nd;
  int r[TK_MAXD];
  int grew[TK_MAXD];
  int radd[TK_MAXD];
  int eig_path[TK_MAXD];
  int eig_it[TK_MAXD];
  int aug;
  int replayed;
  double eps;
  double y2;
  double e2[TK_MAXD];
  double tail_cut[TK_MAXD];
  double tail_prev[TK_MAXD];
  double q;
  double discarded;
};

// Forced decisions of the replay hook (a test hook; see Ctl::rp_on).
__device__ __forceinline__ int rp_grow_of(const Ctl* c, int k) { return c->rp_on ? c->rp_grow[k] : -1; }
__device__ __forceinline__ int rp_aug_of(const Ctl* c) { return c->rp_on ? c->rp_aug : -1; }

// Phases of one update (profiling and byte accounting).
#define TK_PH_PROJ1 0    // mode-1 projection + residual norm (the pass over the slice)
#define TK_PH_PROJN 1    // modes 2..d-1 projection + residual norm
#define TK_PH_GROW 2     // residual Gram, eigensolve, augmentation, re-projection (when grown)
#define TK_PH_ISVD 3     // p = V^T d, e = d - V p, secular SVD of S'
#define TK_PH_FACT 4     // U~_d and M
#define TK_PH_CV 5       // core and V updates
#define TK_PH_SLICE 6    // the mode-1 pass kernel alone (inside phase 0; timed, no bytes)
#define TK_NPH 6

// Mode-k view (A, n, B) of the operand of mode k, column-major: element (a, j, b) at
// a + A (j + n b).
//
// Batch ST-HOSVD (init_nt > 0): the standard view, A = product of the truncated ranks of modes
// < k, n = n_k (or the number of initial slices for the streaming mode), B = product of the
// sizes of the later modes (times the initial slices).
//
// Streaming update (init_nt == 0), rotating layout: the input of spatial mode k is a row-major
// (F_k x n_k) matrix (A = 1, B = F_k) whose rows are the mode-k fibers, with
// F_k = prod_{i>k} n_i * prod_{i<k} r~_i; mode k writes its output column-major (F_k x r_k).
// That output, read as row-major (F_{k+1} x n_{k+1}), is the next mode's input (its fibers are
// again contiguous), and after the last spatial mode the order is the natural column-major order
// of the core (i_1 fastest).
__device__ __forceinline__ int view_n(const Ctl* c, int k) {
  return (k == c->d - 1) ? c->init_nt : c->n[k];
}
__device__ __forceinline__ long long view_A(const Ctl* c, int k) {
  if (c->init_nt == 0) return 1;
  long long a = 1;
  for (int i = 0; i < k; ++i) a *= c->r[i];
  return a;
}
__device__ __forceinline__ long long view_B(const Ctl* c, int k) {
  long long b = 1;
  for (int i = k + 1; i < c->d - 1; ++i) b *= c->n[i];
  if (c->init_nt == 0) {
    for (int i = 0; i < k; ++i) b *= c->r[i];
    if (k < c->d - 1 && c->blk > 1) b *= c->blk;   // the block's trailing mode
  } else if (k < c->d - 1) {
    b *= c->init_nt;
  }
  return b;
}
// Address of output element (fiber f = a + A b, row i): standard (a + A (i + r b)) or rotating
// (f + F i) layout.
__device__ __forceinline__ long long out_base(const Ctl* c, long long f, long long A, int r) {
  if (c->init_nt == 0) return f;
  const long long a = f % A, b = f / A;
  return a + A * (long long)r * b;
}
__device__ __forceinline__ long long out_stride(const Ctl* c, long long A, long long F) {
  return (c->init_nt == 0) ? F : A;
}

__host__ __device__ inline long long tk_prod(const int* v, int a, int b) {
  long long p = 1;
  for (int i = a; i < b; ++i) p *= v[i];
  return p;
}

// ---------------------------------------------------------------------------------------------
// warp / block reductions
// ---------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v);

// Cross-block reduction in a fixed order. Every block has written its partial vector
// part[blockIdx.x * stride + c] (c < len); the last block to finish (completion ticket) sums the
// partials of all blocks into out[c], warps taking blocks w, w + W, ... in increasing order and
// the warp sums added in warp order, so the result does not depend on which block finished last.
// Returns true in that block (all its threads), after out[] is written; resets the ticket.
// true in every thread of the last block of the grid to arrive (completion ticket, reset by
// that block); the writes of the other blocks before their arrival are visible to it.
__device__ __forceinline__ bool tk_block_ticket(unsigned* ticket) {
  __shared__ int s_lastb;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_lastb = (atomicAdd(ticket, 1u) == gridDim.x - 1) ? 1 : 0;
  __syncthreads();
  if (!s_lastb) return false;
  __threadfence();
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

__device__ __forceinline__ bool tk_last_block_reduce(const double* part, long long stride, int len,
                                                     double* out, unsigned* ticket) {
  __shared__ int s_last;
  __shared__ double s_red[32][33];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1) ? 1 : 0;
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nb = gridDim.x;
  for (int c0 = 0; c0 < len; c0 += 32) {
    const int c = c0 + lane;
    double acc = 0.0;
    if (c < len) {
      // L2 loads (.cg: the partials come from other blocks), eight independent sums so that
      // the loads overlap instead of waiting on one another
      double a[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      int b = wid;
      for (; b + 7 * nw < nb; b += 8 * nw) {
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] += __ldcg(part + (long long)(b + u * nw) * stride + c);
      }
      for (; b < nb; b += nw) a[0] += __ldcg(part + (long long)b * stride + c);
      acc = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    }
    s_red[wid][lane] = acc;
    __syncthreads();
    if (wid == 0 && c < len) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += s_red[w][lane];
      out[c] = t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *ticket = 0u;
  __threadfence();
  __syncthreads();
  return true;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; every thread receives the result. `sh` needs 32 slots.
template <typename T>
__device__ T block_sum(T v, T* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T t = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  T r = sh[0];
  __syncthreads();
  return r;
}

// Compensated (Neumaier) accumulation of squares in the element type, flushed into FP64.
struct KahanF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    float t = s + x;
    if (fabsf(s) >= fabsf(x)) c += (s - t) + x; else c += (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

template <typename T> struct AccOf;
template <> struct AccOf<float> { typedef KahanF type; };
struct KahanD {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct AccOf<double> { typedef KahanD type; };

// 32-bit version of tk_map_new_to_old (core sizes stay below 2^31).
__device__ __forceinline__ int map_new_to_old32(int j, const int* rn, const int* ro, int m) {
  int jo = 0, stride = 1;
  for (int k = 0; k < m; ++k) {
    const int ik = j % rn[k];
    j /= rn[k];
    if (ik >= ro[k]) return -1;
    jo += ik * stride;
    stride *= ro[k];
  }
  return jo;
}

// Register-resident form for per-lane row passes: the loops are unrolled over TK_MAXD so that
// the rank arrays stay in registers.
__device__ __forceinline__ int map_new_to_old_reg(int j, const int (&rn)[TK_MAXD],
                                                  const int (&ro)[TK_MAXD], int m) {
  int jo = 0, stride = 1;
#pragma unroll
  for (int k = 0; k < TK_MAXD; ++k) {
    if (k < m) {
      const int ik = j % rn[k];
      j /= rn[k];
      if (ik >= ro[k]) return -1;
      jo += ik * stride;
      stride *= ro[k];
    }
  }
  return jo;
}

// Map a row index of a compact spatial tensor with dims `rn` (new) to the row index in the
// compact layout with dims `ro` (old); returns -1 if the row is a zero-padded one (some i_k >=
// ro[k]). Implements PadWithZeros (Eqs. pad_core_with_zeros, pad_singular_vectors_with_zeros).
__device__ __forceinline__ long long tk_map_new_to_old(long long j, const int* rn, const int* ro,
                                                       int m) {
  long long jo = 0, stride = 1;
  for (int k = 0; k < m; ++k) {
    const int ik = (int)(j % rn[k]);
    j /= rn[k];
    if (ik >= ro[k]) return -1;
    jo += ik * stride;
    stride *= ro[k];
  }
  return jo;
}

// ---- tensor-core path of the core / V update (mixed form) ----
#define TC_KC 32                        // FP32 elements of K per stage (128 bytes)
#define TC_BRES_BYTES (160 * 1024)      // resident B^T (TF32 hi + lo) in shared memory

// Whether the core/V update of this step runs on the tensor cores: mixed form, B^T (N x K split
// into TF32 hi/lo) fits in shared memory, N <= 256. A pure function of the control block and the
// kept streaming rank, evaluated identically by every kernel of the update.
// Row passes with one row of C / V per lane (streaming rank up to 32 before and after the
// update): the state is read once, in row-contiguous pieces, by every lane independently.
#define ROWS_RMAX 32
__device__ __forceinline__ bool rows_isvd_ok(const Ctl* ctl) {
  const int r = ctl->r[ctl->d - 1];
  return r >= 1 && r <= ROWS_RMAX;
}
__device__ __forceinline__ bool rows_cv_ok(const Ctl* ctl, int keep) {
  return rows_isvd_ok(ctl) && keep >= 1 && keep <= ROWS_RMAX;
}

// Row stride of the C and V state rows at streaming rank r: compact (r rounded up to 16 bytes)
// while the per-lane row passes handle the rank, the capacity ldc above it (the stride the
// tensor-core path's TMA maps describe). Every reader and writer of C and V derives the stride
// from the rank the rows hold, so a buffer is always read with the stride it was written with.
__host__ __device__ __forceinline__ int tk_cv_stride(int r, int ldc, int tw) {
  const int a = 16 / tw;
  if (r > ROWS_RMAX) return ldc;
  const int s = (r + a - 1) / a * a;
  return s < ldc ? s : ldc;
}

// The tensor-core core/V update keeps both strides at ldc: streaming rank above ROWS_RMAX before
// and after the update (an update that crosses ROWS_RMAX runs on the SIMT kernel).
__device__ __forceinline__ bool tc_cv_ok(const Ctl* ctl, int keep) {
  if (rows_cv_ok(ctl, keep)) return false;
  if (ctl->tw != 4) return false;
  const int r = ctl->r[ctl->d - 1];
  if (r <= ROWS_RMAX || keep <= ROWS_RMAX) return false;
  const int kc = (r + TC_KC - 1) / TC_KC;
  const int np = (keep + 15) / 16 * 16;
  if (np > 256) return false;
  return (long long)kc * np * TC_KC * 4 * 2 <= TC_BRES_BYTES;
}

__device__ __forceinline__ bool spatial_grew(const Ctl* ctl) {
  for (int k = 0; k < ctl->d - 1; ++k)
    if (ctl->r[k] != ctl->rold[k]) return true;
  return false;
}

// ---- tensor-core path of the spatial-mode projections (mixed form) ----
#define TK_H16_NMAX 384                 // largest n_k of the FP16 tensor-core pass (input tile in TMEM)
#define TP_RMAX 64                      // largest padded r_k handled on the tensor cores

// Spatial mode k on the tensor cores: mixed form, streaming update (rotating layout), the host
// built the tensor maps for this mode (bit k of tcmask), FP32 input (the slice for k = 0),
// n_k a multiple of 4 (TMA row stride) and <= 512 (above 256 the residual product runs in
// column blocks), padded rank <= 64.
__device__ __forceinline__ bool tc_proj_ok(const Ctl* c, int k, int r) {
  if (c->tw != 4 || c->init_nt != 0) return false;
  if (!((c->tcmask >> k) & 1)) return false;
  if (k == 0 && c->tx != 4) return false;
  const int nk = c->n[k];
  if (nk % 4 != 0 || nk > 512 || r < 1) return false;
  return (r + 15) / 16 * 16 <= TP_RMAX;
}
// Residual Gram of mode k on the tensor cores (needs the E^T maps, bit k of etmask, which the
// host sets only for n_k <= 384).
__device__ __forceinline__ bool tc_gram_ok(const Ctl* c, int k) {
  return c->grew[k] && ((c->etmask >> k) & 1) && c->n[k] <= 384 && tc_proj_ok(c, k, c->rold[k]);
}
