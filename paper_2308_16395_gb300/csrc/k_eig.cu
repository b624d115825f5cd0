// Symmetric eigensolver for the Gram matrices of Alg. 1 (TruncatedSVD), one CTA per problem.
//
//   eig(G):  Householder tridiagonalization (Golub & Van Loan, Matrix Computations, Sec. 8.3.1),
//            all eigenvalues by Sturm-sequence bisection (Sec. 8.4.1), the needed eigenvectors
//            by inverse iteration on the tridiagonal matrix with block Gram-Schmidt between
//            iterations (Sec. 8.2.2), back-transformed by the Householder reflectors.
//   rank:    Alg. 1's cut r = min{l : lambda_{l+1} + ... + lambda_m <= eps^2} on the
//            eigenvalues sorted descending.
//   augment: Alg. 4's U~_k = [U_k W_k] with W_k re-orthogonalised against U_k in FP64 (two
//            classical Gram-Schmidt passes, then among its own columns).
//
// TE is the arithmetic of the solve (FP64, or FP32 for the residual Grams of the mixed form,
// whose spectrum spans only the eps^2 neighbourhood); rank decisions and factors are FP64.
#include "common.cuh"
#include "kernels.cuh"

namespace tk {

constexpr int EIG_NT = 1024;
// FP32 solves run 512 threads (16 warps), so the warp-per-vector path has 128 registers a thread
constexpr int EIG_NT_F32 = 512;

template <typename TE> struct Eps;
template <> struct Eps<double> { static __device__ double u() { return 1.1102230246251565e-16; } static __device__ double tiny() { return 1e-290; } };
template <> struct Eps<float> { static __device__ float u() { return 5.9604645e-08f; } static __device__ float tiny() { return 1e-35f; } };

// Sturm counts at NS shifts in one sweep (NS independent recurrences per step). The quotient
// b_i^2 / q uses the fast hardware reciprocal in FP32: the count only needs the sign of q, and a
// relative error of a few ulp in one term moves it no more than the rounding of the subtraction.
// Each step is a dependent chain (reciprocal, FMA, pivot guard), so a lane runs NS recurrences
// interleaved: the second costs little extra time per sweep.
template <typename TE> __device__ __forceinline__ TE sturm_recip(TE q) { return TE(1) / q; }
template <> __device__ __forceinline__ float sturm_recip<float>(float q) { return __fdividef(1.f, q); }

template <typename TE, int NS>
__device__ void sturm_countN(const TE* __restrict__ a, const TE* __restrict__ b2, int n,
                             const TE (&x)[NS], TE pivmin, int (&cnt)[NS]) {
  TE q[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    q[s] = a[0] - x[s];
    if (fabs(q[s]) < pivmin) q[s] = -pivmin;
    cnt[s] = q[s] < TE(0);
  }
#pragma unroll 4
  for (int i = 1; i < n; ++i) {
    const TE ai = a[i], bi = b2[i - 1];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      q[s] = fma(-bi, sturm_recip(q[s]), ai - x[s]);
      if (fabs(q[s]) < pivmin) q[s] = -pivmin;
      cnt[s] += q[s] < TE(0);
    }
  }
}

// Householder tridiagonalization of an FP32 Gram matrix held in registers (n <= 192), one CTA of
// NW = 12 warps run before the eigensolver (24 warps measured slower: every warp repeats the
// reflector and w computations). Thread (warp w, lane l) owns A(w + NW a, l + 32b) for a < RA,
// b < CB. LAPACK convention: reflector c is H = I - tau v v^T with v_{c+1} = 1, p = tau A22 v,
// w = p - (tau/2)(p^T v) v, A22 -= v w^T + w v^T (Golub & Van Loan, Sec. 8.3.1).
// Look-ahead order, one barrier per step: the rank-2 update of step c-1 is applied in step c,
// fused with the matrix-vector product of step c (update an entry, then multiply it by v_c).
// Column c of A after step c-1 is rebuilt by every warp from the published column c of A after
// step c-2 and the vectors of step c-1 (A(:,c) - v w_c - w v_c, v_c = 1), so the column never
// waits for the update: after the barrier of step c-1 a warp reads p_{c-1}, forms w_{c-1} at
// its columns, then column c, reflector c, and runs the fused loop. p of one step, v of one step
// and the published columns alternate between two buffers. p = tau A22 v is reduced across a
// warp's lanes by a butterfly that halves the rows a lane carries at each level (RA rows cost
// RA shuffles rather than 5 RA). The step body is instantiated per column block CB0 = c / 32, so
// blocks of rows and columns left of the trailing matrix drop out at compile time; entries
// outside it are masked by selects.
// Output: reflector c in V[c n + c + 1 ...] (zeros elsewhere in the n x n block); tri = [diagonal
// (n), off-diagonal (n), tau (n)].
constexpr int TRI_NMAX = 192;   // largest n of the register kernel (12 warps x 16 rows)

// p ? x : y through PTX selp. Picking register areg[a][b] for a run-time b with a plain
// comparison lets the compiler turn the unrolled choice into an indexed access, which moves the
// whole register array to local memory; the opaque select keeps it in registers.
__device__ __forceinline__ float sel_f32(bool p, float x, float y) {
  float r;
  asm("{.reg .pred q; setp.ne.u32 q, %1, 0; selp.f32 %0, %2, %3, q;}"
      : "=f"(r) : "r"((unsigned)p), "f"(x), "f"(y));
  return r;
}

// Two buffers of SZ floats each, buffer c & 1 for step c (base + (c & 1) SZ: a run-time index
// into an array of pointers would put the array in local memory).
struct TriSmem {
  float* scol;   // column c of A after step c-2, row-permuted (see tri_perm)
  float* svp;    // v of step c, row-permuted (see tri_perm)
  float* swp;    // p = tau A22 v of step c, row-permuted
  float* sa;
  float* sb;
  float* stau;
};

// Row i of the register block (warp i % NW, block i / NW) stored at (i % NW) RS + i / NW, so a
// warp's RA rows are contiguous (row pairs load as float2, quads store as float4). RS pads the
// stride between warps: a warp reading 32 consecutive rows then touches at most 2 rows per shared-
// memory bank (6 with RS = RA = 16, 3 with RS = RA = 8).
template <int RA> constexpr int tri_rs() { return RA == 16 ? 20 : RA == 8 ? 12 : RA; }
template <int NW, int RA>
__device__ __forceinline__ int tri_perm(int i) { return (i % NW) * tri_rs<RA>() + i / NW; }

// Packed FP32 pairs: rows 2h and 2h+1 of a thread's register block share one 64-bit register
// pair, so the matrix-vector product and the rank-2 update issue one paired FMA (__ffma2_rn,
// round-to-nearest in each half) per two entries.
__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }

// Loop-carried vectors of the previous step at the thread's columns, and the shared-memory
// offsets of those columns in the row-permuted vectors (tri_perm, -1 past n), fixed per lane.
template <int CB> struct TriPrev {
  float v[CB];   // v_{c-1}
  float tau;     // tau_{c-1}
  int po[CB];
};

// w_{c-1} = p_{c-1} - (tau_{c-1}/2)(p_{c-1}^T v_{c-1}) v_{c-1} at the thread's columns (blocks
// >= B0); returns the scalar -(tau/2) p^T v. p and v vanish outside the trailing matrix of step
// c-1 (rows >= n included), so no mask is needed.
template <int NW, int RA, int CB, int B0>
__device__ __forceinline__ float tri_w(const TriPrev<CB>& pr, const float* pp, int n, int lane,
                                       float (&wc)[CB]) {
  float pc[CB];
  float pv = 0.f;
#pragma unroll
  for (int b = B0; b < CB; ++b) {
    const int j = lane + 32 * b;
    pc[b] = pr.po[b] >= 0 ? pp[pr.po[b]] : 0.f;
    pv = fmaf(pc[b], pr.v[b], pv);
  }
  const float K = -0.5f * pr.tau * warp_sum(pv);
#pragma unroll
  for (int b = B0; b < CB; ++b) wc[b] = fmaf(K, pr.v[b], pc[b]);
  return K;
}

template <int NW, int RA, int CB, int CB0>
__device__ __forceinline__ void tri_step(float2 (&a2)[RA / 2][CB], TriPrev<CB>& pr, int c, int n,
                                         int lane, int wid, float* V, const TriSmem& sm) {
  constexpr int LOGRA = RA == 16 ? 4 : RA == 8 ? 3 : RA == 4 ? 2 : RA == 2 ? 1 : 0;
  // rows <= c are not needed after step c and c >= 32 CB0: row blocks a whose rows w + NW a are
  // all <= 32 CB0 are dead; pairs start at an even row block (a dead row in a live pair is
  // updated and multiplied harmlessly, and its p entry is stored as zero)
  constexpr int A0 = 32 * CB0 >= NW - 1 ? (32 * CB0 - NW + 1) / NW + 1 : 0;
  constexpr int H0 = A0 / 2;
  constexpr int RS = tri_rs<RA>();
  constexpr int SZ = NW * RS + 32;
  const int par = (c & 1) * SZ, prv = SZ - par;
  // w_{c-1} at the thread's columns (the barrier of step c-1 published p_{c-1})
  float wc[CB];
  const float K = tri_w<NW, RA, CB, CB0>(pr, sm.swp + prv, n, lane, wc);
  const float wcc = __shfl_sync(0xffffffffu, wc[CB0], c & 31);   // w_{c-1}(c); column c in CB0
  // column c of A after step c-1: A(:,c) - v w(c) - w v(c), v(c) = 1
  const float* col = sm.scol + par;
  float xc[CB];
  float part = 0.f;
#pragma unroll
  for (int b = CB0; b < CB; ++b) {
    const int j = lane + 32 * b;
    xc[b] = fmaf(-pr.v[b], wcc, pr.po[b] >= 0 ? col[pr.po[b]] : 0.f) - wc[b];
    part += sel_f32(j >= c + 2 && j < n, xc[b] * xc[b], 0.f);
  }
  const float xn2 = warp_sum(part);
  float asrc = xc[CB0];
  if constexpr (CB0 + 1 < CB) asrc = sel_f32(((c + 1) >> 5) != CB0, xc[CB0 + 1], asrc);
  const float alpha = __shfl_sync(0xffffffffu, asrc, (c + 1) & 31);
  float tau = 0.f, scal = 0.f, beta = alpha;
  if (xn2 != 0.f) {
    beta = -copysignf(sqrtf(alpha * alpha + xn2), alpha);
    tau = __fdividef(beta - alpha, beta);
    scal = __fdividef(1.f, alpha - beta);
  }
  // tau = 0 leaves v = e_{c+1} and p = w = 0: step c is an exact no-op
  float vc[CB];
#pragma unroll
  for (int b = CB0; b < CB; ++b) {
    const int j = lane + 32 * b;
    vc[b] = sel_f32(j == c + 1, 1.f, sel_f32(j > c + 1 && j < n, xc[b] * scal, 0.f));
  }
  if (wid == 0 && lane == 0) {
    sm.stau[c] = tau;
    sm.sb[c] = beta;
    sm.sa[c] = col[tri_perm<NW, RA>(c)] - 2.f * wcc;
  }
  // reflector c to V and to the shared row vector: column block b by warp b and warp CB + b
  // (one store per lane per warp instead of all of them in one warp)
  static_assert(2 * CB <= NW, "a warp per column block for V and for the row vector");
#pragma unroll
  for (int b = 0; b < CB; ++b) {
    const int j = lane + 32 * b;
    if (wid == b && b >= CB0 && j > c && j < n) V[(long long)c * n + j] = vc[b];
    if (wid == CB + b && pr.po[b] >= 0) sm.svp[par + pr.po[b]] = b >= CB0 ? vc[b] : 0.f;
  }
  // fused: A22 -= v_{c-1} w_{c-1}^T + w_{c-1} v_{c-1}^T, then p = A22 v_c
  float wn[CB], vn[CB], vv[CB];
#pragma unroll
  for (int b = CB0; b < CB; ++b) { wn[b] = -wc[b]; vn[b] = -pr.v[b]; vv[b] = vc[b]; }
  const float2* v2p = reinterpret_cast<const float2*>(sm.svp + prv + wid * RS);
  const float2* p2p = reinterpret_cast<const float2*>(sm.swp + prv + wid * RS);
  const float2 K2 = f2(K, K);
  float acc[RA];
#pragma unroll
  for (int h = 0; h < RA / 2; ++h) {
    float2 s2 = f2(0.f, 0.f);
    if (h >= H0) {
      const float2 vi = v2p[h];
      const float2 wi = __ffma2_rn(K2, vi, p2p[h]);
#pragma unroll
      for (int b = CB0; b < CB; ++b) {
        const float2 a = __ffma2_rn(vi, f2(wn[b], wn[b]), __ffma2_rn(wi, f2(vn[b], vn[b]), a2[h][b]));
        a2[h][b] = a;
        s2 = __ffma2_rn(a, f2(vv[b], vv[b]), s2);
      }
    }
    acc[2 * h] = s2.x;
    acc[2 * h + 1] = s2.y;
  }
  // butterfly reduce-scatter: at level M the lanes with bit M set keep the upper half
#pragma unroll
  for (int lev = 0; lev < LOGRA; ++lev) {
    const int M = 16 >> lev;
    const int H = RA >> (lev + 1);
    const bool up = (lane & M) != 0;
#pragma unroll
    for (int t = 0; t < H; ++t) {
      const float keep = up ? acc[H + t] : acc[t];
      const float send = up ? acc[t] : acc[H + t];
      acc[t] = keep + __shfl_xor_sync(0xffffffffu, send, M);
    }
  }
#pragma unroll
  for (int M = 16 >> LOGRA; M > 0; M >>= 1) acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], M);
  {
    const int my_a = lane >> (5 - LOGRA);
    const bool writer = (lane & ((1 << (5 - LOGRA)) - 1)) == 0;
    const int i = wid + NW * my_a;
    if (writer && i < n) sm.swp[par + wid * RS + my_a] = (i > c) ? tau * acc[0] : 0.f;
  }
  // publish column c+1 of A after step c-1, row-permuted, so the warp's rows are contiguous and
  // go out as 16-byte stores (rows >= c+1 all lie in live pairs; the other rows of the buffer,
  // including a dead pair stored with its live neighbour, are never read)
  if (lane == ((c + 1) & 31)) {
    float* nc = sm.scol + prv + wid * RS;
    const bool hi = ((c + 1) >> 5) != CB0;
    auto colv = [&](int h) -> float2 {
      float2 val = a2[h][CB0];
      if constexpr (CB0 + 1 < CB)
        val = f2(sel_f32(hi, a2[h][CB0 + 1].x, val.x), sel_f32(hi, a2[h][CB0 + 1].y, val.y));
      return val;
    };
    if constexpr (RA % 4 == 0) {
#pragma unroll
      for (int h = H0 & ~1; h < RA / 2; h += 2) {
        const float2 v0 = colv(h), v1 = colv(h + 1);
        *reinterpret_cast<float4*>(nc + 2 * h) = make_float4(v0.x, v0.y, v1.x, v1.y);
      }
    } else {
#pragma unroll
      for (int h = H0; h < RA / 2; ++h) *reinterpret_cast<float2*>(nc + 2 * h) = colv(h);
    }
  }
#pragma unroll
  for (int b = CB0; b < CB; ++b) pr.v[b] = vc[b];
  pr.tau = tau;
  __syncthreads();
}

template <int NW, int RA, int CB, int CB0>
__device__ __forceinline__ void tri_steps(float2 (&a2)[RA / 2][CB], TriPrev<CB>& pr, int n,
                                          int lane, int wid, float* V, const TriSmem& sm) {
  // steps c = 32 CB0 .. 32 CB0 + 31 (reflectors exist for c <= n - 3)
  const int c_hi = min(32 * CB0 + 31, n - 3);
  for (int c = 32 * CB0; c <= c_hi; ++c) tri_step<NW, RA, CB, CB0>(a2, pr, c, n, lane, wid, V, sm);
  if constexpr (CB0 + 1 < CB) tri_steps<NW, RA, CB, CB0 + 1>(a2, pr, n, lane, wid, V, sm);
}

template <int NW, int RA, int CB>
__global__ void __launch_bounds__(NW * 32, 1) k_tridiag_reg(Ctl* ctl, int k, int mode,
                                                          const double* __restrict__ G, float* V,
                                                          float* tri) {
  static_assert(RA % 2 == 0, "register rows are paired");
  if (ctl->status) return;
  // mode 2: residual Gram handed over by the subspace solver (k_eig_sub.cu) only when it set
  // eig_fb[k]; otherwise as mode 0
  if (mode == 2) {
    if (!ctl->eig_fb[k]) return;
    mode = 0;
  }
  if (mode == 0 && !ctl->grew[k]) return;
  const int d = ctl->d;
  const int n = (k == d - 1) ? ctl->init_nt : ctl->n[k];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr int RS = tri_rs<RA>();
  constexpr int SZ = NW * RS + 32;
  static_assert(SZ > 32 * CB, "shared vectors must cover every column index");
  static_assert(RS % 2 == 0 && (RA % 4 != 0 || RS % 4 == 0) && SZ % 4 == 0, "vector alignment");
  __shared__ __align__(16) float scol[2][SZ];
  __shared__ __align__(16) float svp[2][SZ];
  __shared__ __align__(16) float swp[2][SZ];
  __shared__ float sa[SZ], sb[SZ], stau[SZ];
  for (int i = tid; i < SZ; i += blockDim.x) {
    scol[0][i] = 0.f; scol[1][i] = 0.f;
    svp[0][i] = 0.f; svp[1][i] = 0.f;
    swp[0][i] = 0.f; swp[1][i] = 0.f;
  }
  // the reflector block starts as zeros: entries above each reflector's leading 1 and the
  // columns n-2, n-1 (no reflector) then read as zero (the steps write rows c+1.. of column c)
  for (int L = tid; L < n * n; L += blockDim.x) V[L] = 0.f;
  float2 a2[RA / 2][CB];
#pragma unroll
  for (int h = 0; h < RA / 2; ++h)
#pragma unroll
    for (int b = 0; b < CB; ++b) {
      const int i0 = wid + NW * (2 * h), i1 = i0 + NW, j = lane + 32 * b;
      a2[h][b] = f2((i0 < n && j < n) ? (float)G[(long long)i0 * n + j] : 0.f,
                    (i1 < n && j < n) ? (float)G[(long long)i1 * n + j] : 0.f);
    }
  __syncthreads();
  // column 0 (step -1 is empty: v, p, tau start at zero)
  if (lane == 0) {
#pragma unroll
    for (int h = 0; h < RA / 2; ++h) {
      scol[0][wid * RS + 2 * h] = a2[h][0].x;
      scol[0][wid * RS + 2 * h + 1] = a2[h][0].y;
    }
  }
  __syncthreads();
  const TriSmem sm{&scol[0][0], &svp[0][0], &swp[0][0], sa, sb, stau};
  TriPrev<CB> pr;
#pragma unroll
  for (int b = 0; b < CB; ++b) {
    const int j = lane + 32 * b;
    pr.v[b] = 0.f;
    pr.po[b] = j < n ? tri_perm<NW, RA>(j) : -1;
  }
  pr.tau = 0.f;
  tri_steps<NW, RA, CB, 0>(a2, pr, n, lane, wid, V, sm);
  // trailing 2 x 2 block after step n-3, whose update was deferred: registers hold A after step
  // n-4, scol[(n-2) & 1] column n-2 of it. A(n-1, n-1) goes through shared memory first.
  if (lane == ((n - 1) & 31) && wid == (n - 1) % NW) {
    const int a0 = (n - 1) / NW, b0 = (n - 1) >> 5;
    float v = 0.f;
#pragma unroll
    for (int h = 0; h < RA / 2; ++h)
#pragma unroll
      for (int b = 0; b < CB; ++b) {
        v = sel_f32(2 * h == a0 && b == b0, a2[h][b].x, v);
        v = sel_f32(2 * h + 1 == a0 && b == b0, a2[h][b].y, v);
      }
    sa[n - 1] = v;
  }
  __syncthreads();
  if (wid == 0 && n >= 2) {
    const int c = n - 2;
    float wc[CB];
    tri_w<NW, RA, CB, 0>(pr, swp[(c + 1) & 1], n, lane, wc);
    // w_{n-3} and v_{n-3} at rows n-2 and n-1, by run-time block selection and shuffles
    float w0 = 0.f, w1 = 0.f, v1 = 0.f;
#pragma unroll
    for (int b = 0; b < CB; ++b) {
      w0 = sel_f32(b == (c >> 5), wc[b], w0);
      w1 = sel_f32(b == ((c + 1) >> 5), wc[b], w1);
      v1 = sel_f32(b == ((c + 1) >> 5), pr.v[b], v1);
    }
    w0 = __shfl_sync(0xffffffffu, w0, c & 31);
    w1 = __shfl_sync(0xffffffffu, w1, (c + 1) & 31);
    v1 = __shfl_sync(0xffffffffu, v1, (c + 1) & 31);
    if (lane == 0) {
      const float* col = scol[c & 1];
      sa[c] = col[tri_perm<NW, RA>(c)] - 2.f * w0;
      sb[c] = col[tri_perm<NW, RA>(c + 1)] - v1 * w0 - w1;
      stau[c] = 0.f;
      sa[c + 1] -= 2.f * v1 * w1;
      stau[c + 1] = 0.f;
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += blockDim.x) {
    tri[i] = sa[i];
    tri[n + i] = sb[i];
    tri[2 * n + i] = stau[i];
  }
}

struct EigArgs {
  const double* G;   // n x n FP64 input (column-major)
  void* Aw;          // n x n TE scratch
  void* Z;           // n x mcap TE scratch (eigenvectors of T, then of G)
  void* LD;          // mcap x 2n TE scratch (LDL^T factors per vector)
  double* W;         // n x mcap FP64 output (top eigenvectors)
  double* lam_out;   // n FP64 eigenvalues (descending), may be null
  int mcap;          // max vectors
};

// mode 0: residual Gram of spatial mode k (Alg. 4), predicated on ctl->grew[k].
// mode 1: data Gram of mode k in the batch ST-HOSVD (Alg. 2): r >= 1.
// use_smem: the n x n working matrix lives in (dynamic) shared memory instead of global memory.
constexpr int EIG_SMEM_VECS = 16;
constexpr int EIG_FIRST_BATCH = 8;   // top eigenvalues computed before the first cut test
constexpr int EIG_FIRST_BATCH_FV = 4;
constexpr int EIG_WY = 8;            // reflectors per compact-WY group of the back-transform

// Warp-per-vector eigenvector path for FP32 Grams tridiagonalized by k_tridiag_reg (n <= 192,
// up to EIG_SMEM_VECS vectors). Inverse iteration solves the bidiagonal systems of the LDL^T
// factors as first-order linear recurrences, which compose as affine maps: each lane runs the
// recurrence over EIG_FV_SEG consecutive rows, a warp scan composes the lanes' maps, and one more
// pass evaluates every row. The back-transform applies the reflectors in compact-WY groups of
// EIG_FV_GW whose triangular factors T are formed beforehand by the warps that do not bisect.
constexpr int EIG_FV_NMAX = 192;
constexpr int EIG_FV_SEG = EIG_FV_NMAX / 32;
constexpr int EIG_FV_GW = 16;
constexpr int EIG_FV_GMAX = (EIG_FV_NMAX - 2 + EIG_FV_GW - 1) / EIG_FV_GW;

// Butterfly reduce-scatter of 16 per-lane partial sums: returns the warp total of p[lane >> 1]
// (lanes 2a and 2a + 1 both hold the sum for a).
__device__ __forceinline__ float warp_rs16(float (&p)[16], int lane) {
#pragma unroll
  for (int lev = 0; lev < 4; ++lev) {
    const int M = 16 >> lev;
    const int H = 16 >> (lev + 1);
    const bool up = (lane & M) != 0;
#pragma unroll
    for (int t = 0; t < H; ++t) {
      const float keep = up ? p[H + t] : p[t];
      const float send = up ? p[t] : p[H + t];
      p[t] = keep + __shfl_xor_sync(0xffffffffu, send, M);
    }
  }
  return p[0] + __shfl_xor_sync(0xffffffffu, p[0], 1);
}

// T - sig I = L D L^T of the symmetric tridiagonal T (diagonal a, off-diagonal b) for inverse
// iteration: L (n, L[n-1] = 0) and the reciprocal pivots 1/D (n); pivots smaller than pivt in
// magnitude are replaced by +-pivt so the factorization is always defined. One thread.
__device__ __forceinline__ void fv_ldl(const float* __restrict__ a, const float* __restrict__ b,
                                       int n, float sig, float pivt, float* __restrict__ L,
                                       float* __restrict__ Dinv) {
  float dcur = a[0] - sig;
  if (fabsf(dcur) < pivt) dcur = copysignf(pivt, dcur == 0.f ? 1.f : dcur);
  float dinv = __fdividef(1.f, dcur);
  Dinv[0] = dinv;
#pragma unroll 4
  for (int i = 0; i < n - 1; ++i) {
    const float bi = b[i];
    const float l = bi * dinv;
    L[i] = l;
    dcur = fmaf(-l, bi, a[i + 1] - sig);
    if (fabsf(dcur) < pivt) dcur = copysignf(pivt, dcur == 0.f ? 1.f : dcur);
    dinv = __fdividef(1.f, dcur);
    Dinv[i + 1] = dinv;
  }
  L[n - 1] = 0.f;
}

// T factor of reflector group g (reflectors 16g .. 16g+gl-1; reflector c is column c of V, zero
// at rows <= c, 1 at row c + 1; the columns n-2, n-1 hold zeros): H_{16g} ... H_{16g+gl-1} =
// I - V T V^T, T upper triangular with T(j, j) = tau_j and T(0:j, j) = -tau_j T(0:j, 0:j)
// V(:, 0:j)^T v_j (Schreiber & Van Loan). One warp. Reflector indices past the last column are
// clamped to column n-1 (zeros), rows past n are clamped to row n-1 and masked, so the loops carry
// no branches. The products v_a^T v_b go through the 16 x 16 scratch sc; T outside gl x gl is 0.
__device__ void fv_wy_factor(const float* V, const float* tau, int n, int g,
                             float (*wt)[EIG_FV_GW], float* sc, int lane) {
  const int g0 = EIG_FV_GW * g;
  const int gl = min(EIG_FV_GW, n - 2 - g0);
#pragma unroll 1
  for (int b = 1; b < 16; ++b) {
    const float* vb = V + min(g0 + b, n - 1) * n;
    float xb[EIG_FV_SEG];
#pragma unroll
    for (int t = 0; t < EIG_FV_SEG; ++t) {
      const int i = lane + 32 * t;
      xb[t] = i < n ? vb[i] : 0.f;
    }
    float p[16];
#pragma unroll
    for (int a = 0; a < 16; ++a) {
      const float* va = V + min(g0 + a, n - 1) * n;
      float acc = 0.f;
#pragma unroll
      for (int t = 0; t < EIG_FV_SEG; ++t) acc = fmaf(va[min(lane + 32 * t, n - 1)], xb[t], acc);
      p[a] = acc;
    }
    const float s = warp_rs16(p, lane);
    const int a = lane >> 1;
    if ((lane & 1) == 0 && a < b) sc[a * 16 + b] = s;
  }
  __syncwarp();
  float trow[EIG_FV_GW];   // row `lane` of T (lanes 0..15)
#pragma unroll
  for (int j = 0; j < EIG_FV_GW; ++j) {
    float sacc = 0.f;
#pragma unroll
    for (int kk = 0; kk < j; ++kk)
      if (kk >= lane) sacc = fmaf(trow[kk], sc[kk * 16 + j], sacc);
    const float tj = (j < gl) ? tau[g0 + j] : 0.f;
    trow[j] = (lane < j) ? -tj * sacc : (lane == j ? tj : 0.f);
  }
  if (lane < EIG_FV_GW) {
#pragma unroll
    for (int j = 0; j < EIG_FV_GW; ++j) wt[lane][j] = trow[j];
  }
  __syncwarp();
}

// use_smem: dynamic shared memory holds the eigenvector workspaces (up to EIG_SMEM_VECS vectors)
// after the n x n working matrix when use_amat, else at its start.
template <typename TE>
__global__ void __launch_bounds__(sizeof(TE) == 4 ? EIG_NT_F32 : EIG_NT) k_eig_topk(Ctl* ctl, int k, int mode, EigArgs ea,
                                                    int use_smem, int use_amat, int pre) {
  extern __shared__ __align__(16) unsigned char eig_dyn[];
  if (ctl->status) return;
  if (mode == 2) {   // fallback of the subspace solver (see k_tridiag_reg)
    if (!ctl->eig_fb[k]) return;
    mode = 0;
  }
  if (mode == 0 && !ctl->grew[k]) return;
  const int d = ctl->d;
  const int n = (k == d - 1) ? ctl->init_nt : ctl->n[k];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nwarp = nt >> 5;
  // decision replay (test hook): a cut forced for this update
  const int want = (mode == 0) ? max(rp_grow_of(ctl, k), 0) : 0;
  // FP32 residual Grams: one eigenvector past the cut is formed as well, for the FP64
  // Rayleigh-Ritz cut that follows (k_eig_refine)
  const bool xtra = mode == 0 && sizeof(TE) == 4;
  TE* A = use_amat ? reinterpret_cast<TE*>(eig_dyn) : reinterpret_cast<TE*>(ea.Aw);
  __shared__ TE sa[TK_N_MAX], sb[TK_N_MAX], sb2[TK_N_MAX], stau[TK_N_MAX], slam[TK_N_MAX];
  __shared__ TE sv[TK_N_MAX], sp[TK_N_MAX];
  __shared__ TE tred[32];
  __shared__ int s_m;
  __shared__ double s_disc;

  __shared__ TE svb[2][TK_N_MAX];
  __shared__ int s_skip[2];
  // FP32 warp-per-vector path (the reflector copy and the WY factors are prepared by the warps
  // that do not bisect in the first batch)
  const bool fastv = sizeof(TE) == 4 && pre && use_amat && use_smem && n >= 8 && n <= EIG_FV_NMAX;
  // the WY scratch (256 floats per group) fits in the eigenvector area, so the first batch's
  // vector workspaces after it are free while the bisection runs
  const bool fv_spec = fastv && ((n - 2 + EIG_FV_GW - 1) / EIG_FV_GW) * 256 <= EIG_SMEM_VECS * n;
  // first bisection batch: fewer eigenvalues on the FP32 path, so more warps prepare the WY
  // factors meanwhile (one group each at n = 192)
  const int bs0 = fastv ? EIG_FIRST_BATCH_FV : EIG_FIRST_BATCH;
  __shared__ float wy_t[EIG_FV_GMAX][EIG_FV_GW][EIG_FV_GW];
  static_assert(EIG_SMEM_VECS <= EIG_NT_F32 / 32, "one warp per vector");
  if (pre) {
    // tridiagonal form and reflectors from k_tridiag_reg: tri follows the n x n reflector block
    const TE* V = reinterpret_cast<const TE*>(ea.Aw);
    const TE* tri = V + (long long)n * n;
    for (int i = tid; i < n; i += nt) { sa[i] = tri[i]; sb[i] = tri[n + i]; stau[i] = tri[2 * n + i]; }
    if (use_amat && !fastv)
      for (long long L = tid; L < (long long)n * n; L += nt) A[L] = V[L];
    __syncthreads();
  } else {
  for (long long L = tid; L < (long long)n * n; L += nt) A[L] = (TE)ea.G[L];
  __syncthreads();

  // ---- Householder tridiagonalization: A = Q T Q^T, reflectors stored below the diagonal ----
  // Reflector c (LAPACK convention H = I - tau v v^T, v_0 = 1) from column c below the
  // diagonal; warp 0 forms it (warp reduction) as soon as that column is final, into one of two
  // buffers, while the other warps finish the rank-2 update of the previous step.
  auto make_reflector = [&](int c, int buf) {
    // warp 0 only
    const int m = n - c - 1;
    TE* x = A + (long long)c * n + c + 1;
    TE part = TE(0);
    for (int i = 1 + lane; i < m; i += 32) part += x[i] * x[i];
    const TE xn2 = warp_sum(part);
    const TE alpha = x[0];
    if (xn2 == TE(0)) {
      if (lane == 0) { stau[c] = TE(0); sb[c] = alpha; s_skip[buf] = 1; }
      return;
    }
    const TE beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
    const TE tau = (beta - alpha) / beta;
    const TE scal = TE(1) / (alpha - beta);
    for (int i = lane; i < m; i += 32) svb[buf][i] = (i == 0) ? TE(1) : x[i] * scal;
    if (lane == 0) { stau[c] = tau; sb[c] = beta; s_skip[buf] = 0; }
  };
  if (n > 2 && wid == 0) make_reflector(0, 0);
  __syncthreads();
  for (int c = 0; c < n - 2; ++c) {
    const int m = n - c - 1;
    const int cur = c & 1;
    const TE* sv = svb[cur];
    TE* x = A + (long long)c * n + c + 1;
    if (s_skip[cur]) {
      __syncthreads();
      if (wid == 0 && c + 1 < n - 2) make_reflector(c + 1, cur ^ 1);
      __syncthreads();
      continue;
    }
    const TE tau = stau[c];
    // p = tau * A22 v  (A22 symmetric: p_i = sum_j A22(j, i) v_j, column i contiguous)
    for (int i = wid; i < m; i += nwarp) {
      const TE* col = A + (long long)(c + 1 + i) * n + (c + 1);
      TE s = TE(0);
      for (int j = lane; j < m; j += 32) s += col[j] * sv[j];
      s = warp_sum(s);
      if (lane == 0) sp[i] = tau * s;
    }
    __syncthreads();
    if (wid == 0) {
      // w = p - (tau/2)(p^T v) v
      TE pv = TE(0);
      for (int i = lane; i < m; i += 32) pv += sp[i] * sv[i];
      pv = warp_sum(pv);
      const TE K = -TE(0.5) * tau * pv;
      for (int i = lane; i < m; i += 32) sp[i] += K * sv[i];
    }
    __syncthreads();
    // A22 -= v w^T + w v^T; warp 0 owns column 0 of A22 (the next reflector's column) and forms
    // the next reflector right after updating it.
    for (int j = wid; j < m; j += nwarp) {
      TE* colj = A + (long long)(c + 1 + j) * n + (c + 1);
      const TE svj = sv[j], spj = sp[j];
      for (int i = lane; i < m; i += 32) colj[i] -= sv[i] * spj + sp[i] * svj;
      if (j == 0 && c + 1 < n - 2) {
        __syncwarp();
        make_reflector(c + 1, cur ^ 1);
      }
    }
    for (int i = tid; i < m; i += nt) x[i] = sv[i];
    __syncthreads();
  }
  for (int i = tid; i < n; i += nt) sa[i] = A[(long long)i * n + i];
  if (tid == 0) {
    if (n >= 2) { sb[n - 2] = A[(long long)(n - 2) * n + (n - 1)]; stau[n - 2] = TE(0); }
    if (n >= 1) stau[n - 1] = TE(0);
  }
  __syncthreads();
  }  // !pre
  for (int i = tid; i < n - 1; i += nt) sb2[i] = sb[i] * sb[i];
  __syncthreads();

  // ---- Alg. 1's cut from the top eigenvalues ----
  // tails[l] = lam_l + ... + lam_{n-1} = trace(G) - (lam_0 + ... + lam_{l-1}), with the trace
  // summed in FP64 from G's diagonal, so only the eigenvalues above the cut are computed: largest
  // first, one warp per eigenvalue, each by multisection of the Sturm count at 64 shifts per
  // sweep (two per lane, 65 sub-intervals, six bits per sweep); batches of one eigenvalue per
  // warp until the cut is found. The error of a tail is then that of a few eigenvalues (a few u ||G||), not of
  // the sum of all the small ones.
  __shared__ double stails[TK_N_MAX + 1];   // stails[l] = trace - (lam_0 + ... + lam_{l-1})
  __shared__ int s_cnt, s_cut;
  __shared__ double s_trace;
  if (wid == 0) {
    double t = 0.0;
    for (int i = lane; i < n; i += 32) t += ea.G[(long long)i * n + i];
    t = warp_sum(t);
    if (lane == 0) { s_trace = t; stails[0] = t; s_cnt = 0; s_cut = -1; }
  }
  // Gershgorin interval, largest b_i^2 and |T|_inf of the tridiagonal matrix (one warp)
  __shared__ TE s_gl, s_gu, s_bmax2, s_tnorm;
  if (wid == 0) {
    TE gl = sa[0], gu = sa[0], bmax2 = TE(0), tn = TE(0);
    for (int i = lane; i < n; i += 32) {
      const TE rad = (i > 0 ? fabs(sb[i - 1]) : TE(0)) + (i < n - 1 ? fabs(sb[i]) : TE(0));
      gl = min(gl, sa[i] - rad);
      gu = max(gu, sa[i] + rad);
      tn = max(tn, fabs(sa[i]) + rad);
      if (i < n - 1) bmax2 = max(bmax2, sb2[i]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      gl = min(gl, __shfl_xor_sync(0xffffffffu, gl, o));
      gu = max(gu, __shfl_xor_sync(0xffffffffu, gu, o));
      tn = max(tn, __shfl_xor_sync(0xffffffffu, tn, o));
      bmax2 = max(bmax2, __shfl_xor_sync(0xffffffffu, bmax2, o));
    }
    if (lane == 0) { s_gl = gl; s_gu = gu; s_bmax2 = bmax2; s_tnorm = tn; }
  }
  __syncthreads();
  {
    TE gl = s_gl, gu = s_gu;
    const TE bmax2 = s_bmax2;
    const TE scale = max(fabs(gl), fabs(gu));
    const TE u = Eps<TE>::u();
    gl -= TE(2) * u * scale * n + Eps<TE>::tiny();
    gu += TE(2) * u * scale * n + Eps<TE>::tiny();
    const TE pivmin = max(Eps<TE>::tiny(), u * u * bmax2);
    // absolute floor u |T|: the reduction to tridiagonal form already moves every eigenvalue by
    // that much
    const TE atol = max(pivmin, u * scale);
    const double eps2 = ctl->eps * ctl->eps;
    __syncthreads();
    if (tid == 0 && s_trace <= eps2) s_cut = 0;
    __syncthreads();
    // the first batch always runs (the initial ST-HOSVD keeps at least one eigenpair); it is
    // small because the cut of a residual Gram usually keeps a few eigenpairs. The initial
    // ST-HOSVD (mode 1) computes every eigenvalue: its discarded energy is a tiny fraction of the
    // trace, so it is summed from the bottom of the spectrum below instead.
    for (int j0 = 0; j0 < n && (j0 == 0 || s_cut < 0 || mode == 1 || s_cnt < want || (xtra && s_cnt <= s_cut)); j0 += (j0 == 0 ? bs0 : nwarp)) {
      const int bs = (j0 == 0) ? bs0 : nwarp;
      const int j = j0 + wid;            // descending index of this warp's eigenvalue
      if (wid < bs && j < n) {
        const int i = n - 1 - j;         // ascending index
        TE lo = gl, hi = gu;
        for (int it = 0; it < 40; ++it) {
          const TE w = hi - lo;
          if (w <= TE(2) * u * max(fabs(lo), fabs(hi)) + atol) break;
          // 64 shifts per sweep, two independent recurrences per lane (65 sub-intervals)
          const TE step = w / TE(65);
          TE x[2] = {lo + TE(lane + 1) * step, lo + TE(lane + 33) * step};
          if (!(lo + step > lo && lo + TE(64) * step < hi)) break;
          int cnt[2];
          sturm_countN<TE, 2>(sa, sb2, n, x, pivmin, cnt);
          // the eigenvalue lies in the first sub-interval whose right end counts more than i
          // eigenvalues below it
          const unsigned above0 = __ballot_sync(0xffffffffu, cnt[0] > i);
          const unsigned above1 = __ballot_sync(0xffffffffu, cnt[1] > i);
          const int l = above0 ? __ffs(above0) - 1 : (above1 ? 32 + __ffs(above1) - 1 : 64);
          const TE nlo = (l == 0) ? lo : lo + TE(l) * step;
          const TE nhi = (l == 64) ? hi : lo + TE(l + 1) * step;
          lo = nlo;
          hi = nhi;
        }
        if (lane == 0) slam[j] = TE(0.5) * (lo + hi);
        if (fv_spec && j0 == 0 && lane == 0) {
          // inverse-iteration factors for this eigenvalue while the other warps still bisect
          const float uf = 5.9604645e-08f, tnf = (float)s_tnorm;
          float* LDj = reinterpret_cast<float*>(eig_dyn) + (size_t)n * n + (size_t)EIG_SMEM_VECS * n + (size_t)j * 2 * n;
          fv_ldl(reinterpret_cast<const float*>(sa), reinterpret_cast<const float*>(sb), n,
                 (float)slam[j] + 4.f * uf * tnf, fmaxf(uf * tnf, 1e-35f), LDj, LDj + n);
        }
      } else if (fastv && j0 == 0 && wid >= bs) {
        // reflectors into shared memory, WY factors of every group
        // reflectors into shared memory (k_tridiag_reg wrote them with their zeros), four
        // 16-byte loads in flight per thread, then the WY factors of every group; the T scratch
        // of group g is 256 floats of the (still unused) eigenvector workspace
        const float* Vg = reinterpret_cast<const float*>(ea.Aw);
        float* Af = reinterpret_cast<float*>(eig_dyn);   // == A (use_amat): shared, not generic
        const int pw = wid - bs, np = nwarp - bs;
        const int nn = n * n, n4 = nn / 4, pt = pw * 32 + lane, ps = np * 32;
        const float4* V4 = reinterpret_cast<const float4*>(Vg);
        float4* A4 = reinterpret_cast<float4*>(Af);
        for (int q = pt; q < n4; q += 4 * ps) {
          float4 r[4];
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (q + u * ps < n4) r[u] = V4[q + u * ps];
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (q + u * ps < n4) A4[q + u * ps] = r[u];
        }
        for (int L = 4 * n4 + pt; L < nn; L += ps) Af[L] = Vg[L];
        // the copy is complete among these warps (named barrier 1; the bisecting warps do not
        // take part)
        asm volatile("bar.sync 1, %0;" ::"r"(np * 32) : "memory");
        const int ng = (n - 2 + EIG_FV_GW - 1) / EIG_FV_GW;
        float* scr = Af + (size_t)n * n;
        for (int g = pw; g < ng; g += np)
          fv_wy_factor(Af, reinterpret_cast<const float*>(stau), n, g, wy_t[g], scr + (size_t)g * 256, lane);
      }
      __syncthreads();
      if (tid == 0) {
        const int jend = min(n, j0 + bs);
        for (int jj = j0; jj < jend; ++jj) {
          stails[jj + 1] = stails[jj] - (double)slam[jj];
          if (s_cut < 0 && stails[jj + 1] <= eps2) s_cut = jj + 1;
        }
        s_cnt = jend;
        if (s_cut < 0 && jend == n) s_cut = n;   // every eigenvalue is kept
      }
      __syncthreads();
    }
  }

  // ---- rank decision (Alg. 1) in FP64: the first l with tails[l] <= eps^2 ----
  if (tid == 0 && mode == 1) {
    // all eigenvalues are known: tails summed from the smallest eigenvalue up
    const double eps2 = ctl->eps * ctl->eps;
    stails[n] = 0.0;
    for (int l = n - 1; l >= 0; --l) stails[l] = stails[l + 1] + (double)slam[l];
    int cut = n;
    for (int l = 0; l <= n; ++l)
      if (stails[l] <= eps2) { cut = l; break; }
    s_cut = cut;
    s_cnt = n;
  }
  __shared__ double s_tprev;
  __shared__ int s_mv;
  if (tid == 0) {
    int m = s_cut;
    if (want > 0) m = min(want, s_cnt);
    int status = 0;
    if (mode == 0) {
      const int rk = ctl->r[k];
      if (m > n - rk) m = n - rk;
      if (rk + m > ctl->cap[k]) status = TK_ECAPACITY;
    } else {
      if (m < 1) m = 1;
      if (m > ctl->cap[k] || m > ea.mcap) status = TK_ECAPACITY;
    }
    if (m > ea.mcap) status = TK_ECAPACITY;
    if (status) ctl->status = status;
    s_m = status ? 0 : m;
    // (a top-down tail below the eigenvalues' resolution is rounding noise of either sign; a
    // discarded energy is not negative)
    s_disc = (m <= s_cnt) ? fmax(stails[m], 0.0) : 0.0;
    s_tprev = (m >= 1 && m - 1 <= s_cnt) ? fmax(stails[m - 1], 0.0) : 0.0;
    int mv = s_m;
    if (xtra && s_m > 0) mv = min(min(s_m + 1, s_cnt), min(n - ctl->r[k], ea.mcap));
    s_mv = mv;
  }
  __syncthreads();
  const int mcut = s_m;   // the cut (Alg. 1)
  const int m = s_mv;     // eigenvectors formed
  if (ea.lam_out)
    for (int i = tid; i < s_cnt; i += nt) ea.lam_out[i] = (double)slam[i];
  if (m == 0) {
    if (tid == 0) {
      if (mode == 0) { ctl->radd[k] = 0; ctl->disc[k] = s_disc; ctl->tail_prev[k] = s_tprev; }
      else { ctl->r[k] = 0; ctl->disc[k] = s_disc; }
    }
    return;
  }

  if (fastv && m <= EIG_SMEM_VECS) {
    // ---- eigenvectors of the top m eigenvalues, one warp per vector ----
    // inverse iteration (Golub & Van Loan, Sec. 8.2.2) on T - sig I = L D L^T, sig slightly
    // above the computed eigenvalue; 3 iterations with modified Gram-Schmidt across vectors
    float* Af = reinterpret_cast<float*>(eig_dyn);   // == A (use_amat): shared, not generic
    float* Zs = Af + (size_t)n * n;                      // vector v: Zs[v n + row]
    float* LDs = Zs + (size_t)EIG_SMEM_VECS * n;         // vector v: L (n), 1/D (n)
    const float* saf = reinterpret_cast<const float*>(sa);
    const float* sbf = reinterpret_cast<const float*>(sb);
    const float uf = 5.9604645e-08f;
    const float tnf = (float)s_tnorm;
    const float pivt = fmaxf(uf * tnf, 1e-35f);
    const bool mine = wid < m;
    const int v = wid;
    float* Lv = LDs + (size_t)(mine ? v : 0) * 2 * n;
    float* Dv = Lv + n;
    constexpr int SEG = EIG_FV_SEG;
    const int r0 = SEG * lane;
    const unsigned FULL = 0xffffffffu;
    // factors of the first batch's vectors were formed by their bisection warps
    if (mine && lane == 0 && !(fv_spec && v < bs0))
      fv_ldl(saf, sbf, n, (float)slam[v] + 4.f * uf * tnf, pivt, Lv, Dv);
    __syncwarp();
    float z[SEG];
#pragma unroll
    for (int q = 0; q < SEG; ++q) {
      const int r = r0 + q;
      // deterministic start vector with entries in [1, 1.5]
      unsigned h = (unsigned)(r * 2654435761u) ^ (unsigned)((v + 1) * 40503u);
      h ^= h >> 13; h *= 0x5bd1e995u; h ^= h >> 15;
      z[q] = (r < n) ? 1.f + (0.5f / 65535.f) * (float)(h & 0xffffu) : 0.f;
    }
    for (int iter = 0; iter < 3; ++iter) {
      if (mine) {
        // L y = z: y_r = z_r - L_{r-1} y_{r-1}; per lane y_r = al_r y_in + be_r
        float al[SEG], be[SEG];
#pragma unroll
        for (int q = 0; q < SEG; ++q) {
          const int r = r0 + q;
          const float lm = (r >= 1 && r < n) ? Lv[r - 1] : 0.f;
          al[q] = (q == 0) ? -lm : -lm * al[q - 1];
          be[q] = (q == 0) ? z[0] : fmaf(-lm, be[q - 1], z[q]);
        }
        float Am = al[SEG - 1], Bm = be[SEG - 1];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const float A2 = __shfl_up_sync(FULL, Am, off), B2 = __shfl_up_sync(FULL, Bm, off);
          if (lane >= off) { Bm = fmaf(Am, B2, Bm); Am *= A2; }
        }
        float yin = __shfl_up_sync(FULL, Bm, 1);
        if (lane == 0) yin = 0.f;
#pragma unroll
        for (int q = 0; q < SEG; ++q) z[q] = fmaf(al[q], yin, be[q]);
        // D L^T x = y: x_r = y_r / d_r - L_r x_{r+1}; per lane x_r = ga_r x_in + de_r
        float ga[SEG], de[SEG];
#pragma unroll
        for (int q = SEG - 1; q >= 0; --q) {
          const int r = r0 + q;
          const float lr = (r < n) ? Lv[r] : 0.f;
          const float dr = (r < n) ? Dv[r] : 0.f;
          ga[q] = (q == SEG - 1) ? -lr : -lr * ga[q + 1];
          de[q] = (q == SEG - 1) ? z[q] * dr : fmaf(-lr, de[q + 1], z[q] * dr);
        }
        float Cm = ga[0], Em = de[0];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const float C2 = __shfl_down_sync(FULL, Cm, off), E2 = __shfl_down_sync(FULL, Em, off);
          if (lane + off < 32) { Em = fmaf(Cm, E2, Em); Cm *= C2; }
        }
        float xin = __shfl_down_sync(FULL, Em, 1);
        if (lane == 31) xin = 0.f;
        float amax = 0.f;
#pragma unroll
        for (int q = 0; q < SEG; ++q) {
          z[q] = fmaf(ga[q], xin, de[q]);
          amax = fmaxf(amax, fabsf(z[q]));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(FULL, amax, o));
        // the solve amplifies by up to 1/(4 u |T|): back to unit max-norm
        const float sc = amax > 0.f ? 1.f / amax : 0.f;
#pragma unroll
        for (int q = 0; q < SEG; ++q) z[q] *= sc;
      }
      if (m > 1) {
        // modified Gram-Schmidt in vector order through shared memory
        if (mine) {
#pragma unroll
          for (int q = 0; q < SEG; ++q)
            if (r0 + q < n) Zs[(size_t)v * n + r0 + q] = z[q];
        }
        __syncthreads();
        for (int vv = 0; vv + 1 < m; ++vv) {
          if (mine && v > vv) {
            float sdot = 0.f, zz = 0.f, zv[SEG];
#pragma unroll
            for (int q = 0; q < SEG; ++q) {
              zv[q] = (r0 + q < n) ? Zs[(size_t)vv * n + r0 + q] : 0.f;
              sdot = fmaf(zv[q], z[q], sdot);
              zz = fmaf(zv[q], zv[q], zz);
            }
            sdot = warp_sum(sdot);
            zz = warp_sum(zz);
            const float coef = zz > 0.f ? sdot / zz : 0.f;
#pragma unroll
            for (int q = 0; q < SEG; ++q) {
              z[q] = fmaf(-coef, zv[q], z[q]);
              if (r0 + q < n) Zs[(size_t)v * n + r0 + q] = z[q];
            }
          }
          __syncthreads();
        }
      }
      if (mine) {
        float part = 0.f;
#pragma unroll
        for (int q = 0; q < SEG; ++q) part = fmaf(z[q], z[q], part);
        const float nrm = sqrtf(warp_sum(part));
        const float inv = nrm > 0.f ? 1.f / nrm : 0.f;
#pragma unroll
        for (int q = 0; q < SEG; ++q) z[q] *= inv;
      }
    }
    // ---- back-transform x = H_0 H_1 ... H_{n-3} z, last WY group first ----
    if (mine) {
#pragma unroll
      for (int q = 0; q < SEG; ++q)
        if (r0 + q < n) Zs[(size_t)v * n + r0 + q] = z[q];
      __syncwarp();
      float zr[SEG];   // rows lane + 32 t
#pragma unroll
      for (int t = 0; t < SEG; ++t) {
        const int i = lane + 32 * t;
        zr[t] = (i < n) ? Zs[(size_t)v * n + i] : 0.f;
      }
      const int ng = (n - 2 + EIG_FV_GW - 1) / EIG_FV_GW;
      // branch-free group loop: reflector columns past n-1 clamp to column n-1 (zeros), rows
      // past n clamp to row n-1 and are masked out of the update (zr stays 0 there)
      const int am = lane >> 1;
#pragma unroll 1
      for (int g = ng - 1; g >= 0; --g) {
        const int g0 = EIG_FV_GW * g;
        // s = V^T z
        float p[16];
#pragma unroll
        for (int a = 0; a < 16; ++a) {
          const float* va = Af + min(g0 + a, n - 1) * n;
          float x[SEG];
#pragma unroll
          for (int t = 0; t < SEG; ++t) x[t] = va[min(lane + 32 * t, n - 1)];
          float acc = 0.f;
#pragma unroll
          for (int t = 0; t < SEG; ++t) acc = fmaf(x[t], zr[t], acc);
          p[a] = acc;
        }
        const float s_mine = warp_rs16(p, lane);          // s_{lane >> 1}
        // u = T s (T upper triangular, zero below the diagonal): lanes 2a, 2a + 1 form u_a
        float u_mine = 0.f;
#pragma unroll
        for (int j = 0; j < 16; ++j)
          u_mine = fmaf(wy_t[g][am][j], __shfl_sync(FULL, s_mine, 2 * j), u_mine);
        // z -= V u
#pragma unroll
        for (int a = 0; a < 16; ++a) {
          const float ua = __shfl_sync(FULL, u_mine, 2 * a);
          const float* va = Af + min(g0 + a, n - 1) * n;
#pragma unroll
          for (int t = 0; t < SEG; ++t) {
            const int i = lane + 32 * t;
            const float dz = va[min(i, n - 1)] * ua;
            zr[t] = i < n ? zr[t] - dz : zr[t];
          }
        }
      }
#pragma unroll
      for (int t = 0; t < SEG; ++t) {
        const int i = lane + 32 * t;
        if (i < n) ea.W[(long long)v * n + i] = (double)zr[t];
      }
    }
    if (tid == 0) {
      if (mode == 0) { ctl->radd[k] = mcut; ctl->disc[k] = s_disc; ctl->tail_prev[k] = s_tprev; ctl->eig_m[k] = m; }
      else { ctl->r[k] = mcut; ctl->disc[k] = s_disc; }
    }
    return;
  }

  // ---- inverse iteration for the top m eigenvalues ----
  // eigenvector workspaces in shared memory when up to EIG_SMEM_VECS vectors are needed
  const bool zsm = use_smem && m <= EIG_SMEM_VECS;
  TE* zbase = reinterpret_cast<TE*>(eig_dyn) + (size_t)n * n * use_amat;
  TE* Z = zsm ? zbase : reinterpret_cast<TE*>(ea.Z);                       // n x m
  TE* LD = zsm ? zbase + (size_t)EIG_SMEM_VECS * n : reinterpret_cast<TE*>(ea.LD);  // L, D
  const TE tnorm = s_tnorm;
  const TE u = Eps<TE>::u();
  const TE pivt = max(u * tnorm, Eps<TE>::tiny());
  for (int v = tid; v < m; v += nt) {
    // shift slightly away from the computed eigenvalue so the factorization is nonsingular;
    // LD holds L (n) and the reciprocal pivots 1/D (n) of T - sig I = L D L^T
    const TE sig = slam[v] + TE(4) * u * tnorm;
    TE* Lv = LD + (long long)v * 2 * n;
    TE* Dv = Lv + n;
    TE dcur = sa[0] - sig;
    if (fabs(dcur) < pivt) dcur = copysign(pivt, dcur == TE(0) ? TE(1) : dcur);
    TE dinv = TE(1) / dcur;
    Dv[0] = dinv;
    for (int i = 0; i < n - 1; ++i) {
      const TE l = sb[i] * dinv;
      Lv[i] = l;
      dcur = (sa[i + 1] - sig) - l * sb[i];
      if (fabs(dcur) < pivt) dcur = copysign(pivt, dcur == TE(0) ? TE(1) : dcur);
      dinv = TE(1) / dcur;
      Dv[i + 1] = dinv;
    }
    // deterministic start vector with entries in [1, 1.5]
#pragma unroll 4
    for (int i = 0; i < n; ++i) {
      unsigned h = (unsigned)(i * 2654435761u) ^ (unsigned)((v + 1) * 40503u);
      h ^= h >> 13; h *= 0x5bd1e995u; h ^= h >> 15;
      Z[(long long)v * n + i] = TE(1) + TE(0.5 / 65535.0) * (TE)(h & 0xffffu);
    }
  }
  __syncthreads();
  for (int iter = 0; iter < 3; ++iter) {
    for (int v = tid; v < m; v += nt) {
      const TE* Lv = LD + (long long)v * 2 * n;
      const TE* Dv = Lv + n;
      TE* z = Z + (long long)v * n;
      // L y = z, then D L^T x = y with the pivot scaling folded into the backward sweep
      TE prev = z[0];
#pragma unroll 8
      for (int i = 1; i < n; ++i) { prev = z[i] - Lv[i - 1] * prev; z[i] = prev; }
      prev = prev * Dv[n - 1];
      z[n - 1] = prev;
      TE amax = fabs(prev);
#pragma unroll 8
      for (int i = n - 2; i >= 0; --i) {
        prev = z[i] * Dv[i] - Lv[i] * prev;
        z[i] = prev;
        amax = max(amax, fabs(prev));
      }
      // the solve amplifies by up to 1/(4 u |T|): rescale to unit max-norm so the sums of
      // squares below cannot overflow whatever the scale of the Gram matrix
      const TE sc = amax > TE(0) ? TE(1) / amax : TE(0);
#pragma unroll 8
      for (int i = 0; i < n; ++i) z[i] *= sc;
    }
    __syncthreads();
    // modified Gram-Schmidt across the m vectors (separates clusters): at step v, every later
    // vector loses its component along z_v (one warp per later vector, z_v's norm recomputed
    // by each warp), one barrier per step; all vectors are normalised together at the end
    for (int v = 0; v + 1 < m; ++v) {
      const TE* z = Z + (long long)v * n;
      for (int w = v + 1 + wid; w < m; w += nwarp) {
        TE* y = Z + (long long)w * n;
        TE s = TE(0), zz = TE(0);
        for (int i = lane; i < n; i += 32) { s += z[i] * y[i]; zz += z[i] * z[i]; }
        s = warp_sum(s);
        zz = warp_sum(zz);
        const TE coef = zz > TE(0) ? s / zz : TE(0);
        for (int i = lane; i < n; i += 32) y[i] -= coef * z[i];
      }
      __syncthreads();
    }
    for (int v = wid; v < m; v += nwarp) {
      TE* z = Z + (long long)v * n;
      TE part = TE(0);
      for (int i = lane; i < n; i += 32) part += z[i] * z[i];
      const TE nrm = sqrt(warp_sum(part));
      const TE inv = nrm > TE(0) ? TE(1) / nrm : TE(0);
      for (int i = lane; i < n; i += 32) z[i] *= inv;
    }
    __syncthreads();
  }
  // ---- back-transform: x = H_0 H_1 ... H_{n-3} z ----
  // Groups of EIG_WY consecutive reflectors in compact WY form, H_a ... H_b = I - V T V^T with T
  // upper triangular (Schreiber & Van Loan, SIAM J. Sci. Stat. Comput. 10, 1989), applied last
  // group first: one round of dot products (V^T V and V^T Z) over all warps, T and T (V^T Z) on
  // one warp, then Z -= V (T V^T Z) over all threads. Reflector c is column c of A below the
  // diagonal, with its leading 1 stored at row c + 1.
  if (m <= EIG_SMEM_VECS) {
    __shared__ TE wy_s[EIG_WY][EIG_WY];            // v_a^T v_b, a < b
    __shared__ TE wy_w[EIG_WY][EIG_SMEM_VECS];     // V^T Z, then T V^T Z
    const int nref = n - 2;
    for (int g0 = nref > 0 ? ((nref - 1) / EIG_WY) * EIG_WY : -1; g0 >= 0; g0 -= EIG_WY) {
      const int gl = min(EIG_WY, nref - g0);
      const int npair = gl * (gl - 1) / 2;
      for (int t = wid; t < npair + gl * m; t += nwarp) {
        TE s = TE(0);
        if (t < npair) {
          int b = 1;
          while (b * (b + 1) / 2 <= t) ++b;
          const int a = t - b * (b - 1) / 2;
          const TE* va = A + (long long)(g0 + a) * n;
          const TE* vb = A + (long long)(g0 + b) * n;
          for (int i = g0 + b + 1 + lane; i < n; i += 32) s += va[i] * vb[i];
          s = warp_sum(s);
          if (lane == 0) wy_s[a][b] = s;
        } else {
          const int a = (t - npair) % gl, v = (t - npair) / gl;
          const TE* va = A + (long long)(g0 + a) * n;
          const TE* z = Z + (long long)v * n;
          for (int i = g0 + a + 1 + lane; i < n; i += 32) s += va[i] * z[i];
          s = warp_sum(s);
          if (lane == 0) wy_w[a][v] = s;
        }
      }
      __syncthreads();
      if (wid == 0) {
        // lane i holds row i of T in registers: column j is T(i, j) = -tau_j sum_{i<=k<j}
        // T(i, k) v_k^T v_j for i < j, tau_j on the diagonal
        TE trow[EIG_WY];
#pragma unroll
        for (int j = 0; j < EIG_WY; ++j) {
          TE acc = TE(0);
#pragma unroll
          for (int k = 0; k < EIG_WY; ++k)
            if (k < j && k >= lane) acc += trow[k] * wy_s[k][j];
          const TE tj = (j < gl) ? stau[g0 + j] : TE(0);
          trow[j] = (lane < j) ? -tj * acc : (lane == j ? tj : TE(0));
        }
        // (T V^T Z)(i, v) for the lane's row i, every vector
        TE outv[EIG_SMEM_VECS];
#pragma unroll
        for (int v = 0; v < EIG_SMEM_VECS; ++v) {
          TE acc = TE(0);
          if (v < m) {
#pragma unroll
            for (int k = 0; k < EIG_WY; ++k)
              if (k < gl) acc += trow[k] * wy_w[k][v];
          }
          outv[v] = acc;
        }
        __syncwarp();
        if (lane < gl) {
#pragma unroll
          for (int v = 0; v < EIG_SMEM_VECS; ++v)
            if (v < m) wy_w[lane][v] = outv[v];
        }
      }
      __syncthreads();
      for (long long L = tid; L < (long long)m * n; L += nt) {
        const int v = (int)(L / n), i = (int)(L % n);
        if (i <= g0) continue;
        TE acc = TE(0);
        for (int a = 0; a < gl && g0 + a + 1 <= i; ++a) acc += A[(long long)(g0 + a) * n + i] * wy_w[a][v];
        Z[(long long)v * n + i] -= acc;
      }
      __syncthreads();
    }
  } else {
    // one warp per vector, reflectors applied one at a time
    for (int v = wid; v < m; v += nwarp) {
      TE* z = Z + (long long)v * n;
      for (int c = n - 3; c >= 0; --c) {
        const TE tau = stau[c];
        if (tau == TE(0)) continue;
        const TE* hv = A + (long long)c * n + c + 1;
        const int len = n - c - 1;
        TE s = TE(0);
        for (int i = lane; i < len; i += 32) s += hv[i] * z[c + 1 + i];
        s = warp_sum(s) * tau;
        for (int i = lane; i < len; i += 32) z[c + 1 + i] -= s * hv[i];
        __syncwarp();
      }
    }
  }
  __syncthreads();
  for (long long L = tid; L < (long long)m * n; L += nt) ea.W[L] = (double)Z[L];
  if (tid == 0) {
    if (mode == 0) { ctl->radd[k] = mcut; ctl->disc[k] = s_disc; ctl->tail_prev[k] = s_tprev; ctl->eig_m[k] = m; }
    else { ctl->r[k] = mcut; ctl->disc[k] = s_disc; }
  }
}

// Alg. 4, U~_k = [U_k W_k]: re-orthogonalise W (n x radd) against U_k[:, 0:r) (two CGS passes
// in FP64) and among its own columns, then append it to the FP64 factor and its work copy.
// mode 0: growth (predicated), mode 1: init (r = 0, copy the r_k vectors).
template <typename TW>
__global__ void __launch_bounds__(1024) k_append_factor(Ctl* ctl, int k, int mode, const double* W,
                                                       double* U, TW* Uw, int ldu) {
  if (ctl->status) return;
  if (mode == 0 && !ctl->grew[k]) return;
  const int d = ctl->d;
  const int n = (k == d - 1) ? ctl->init_nt : ctl->n[k];
  const int r0 = (mode == 0) ? ctl->r[k] : 0;
  const int m = (mode == 0) ? ctl->radd[k] : ctl->r[k];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nwarp = nt >> 5;
  __shared__ double red[32];
  __shared__ double coef[TK_N_MAX];
  extern __shared__ double wcol[];   // n
  for (int v = 0; v < m; ++v) {
    for (int i = tid; i < n; i += nt) wcol[i] = W[(long long)v * n + i];
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      const int ncols = r0 + v;  // against existing columns and the already appended ones
      for (int c = wid; c < ncols; c += nwarp) {
        const double* uc = U + (long long)c * ldu;
        double s = 0.0;
        for (int i = lane; i < n; i += 32) s += uc[i] * wcol[i];
        s = warp_sum(s);
        if (lane == 0) coef[c] = s;
      }
      __syncthreads();
      for (int i = tid; i < n; i += nt) {
        double s = 0.0;
        for (int c = 0; c < ncols; ++c) s += U[(long long)c * ldu + i] * coef[c];
        wcol[i] -= s;
      }
      __syncthreads();
    }
    double part = 0.0;
    for (int i = tid; i < n; i += nt) part += wcol[i] * wcol[i];
    const double nrm = sqrt(block_sum(part, red));
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (int i = tid; i < n; i += nt) {
      const double val = wcol[i] * inv;
      U[(long long)(r0 + v) * ldu + i] = val;
      if (Uw) Uw[(long long)(r0 + v) * ldu + i] = (TW)val;
    }
    __syncthreads();
  }
  if (tid == 0 && mode == 0) ctl->r[k] = r0 + m;
}

constexpr size_t EIG_SMEM_MAX = 200 * 1024;

template <typename TE>
cudaError_t launch_eig(Ctl* ctl, int k, int mode, const double* G, void* Aw, void* Z, void* LD,
                       double* W, double* lam, int mcap, int n, cudaStream_t st) {
  EigArgs ea{G, Aw, Z, LD, W, lam, mcap};
  // dynamic shared memory may use what the kernel's static arrays leave of the opt-in maximum
  static size_t dyn_max[2] = {0, 0};
  size_t& lim = dyn_max[sizeof(TE) == 8 ? 1 : 0];
  if (lim == 0) {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_eig_topk<TE>);
    if (e != cudaSuccess) return e;
    lim = (size_t)optin > fa.sharedSizeBytes + 1024 ? (size_t)optin - fa.sharedSizeBytes - 1024 : 0;
    lim = std::min(lim, EIG_SMEM_MAX);
  }
  const size_t mat = (size_t)n * n * sizeof(TE);
  const size_t vec = (size_t)EIG_SMEM_VECS * 3 * n * sizeof(TE);
  const int use_vec = (vec <= std::min<size_t>(150 * 1024, lim)) ? 1 : 0;
  const int use_amat = (use_vec && mat + vec <= lim) ? 1 : 0;
  const size_t sm = (use_amat ? mat : 0) + (use_vec ? vec : 0);
  // raised to the largest size seen so far, never lowered (see launch_eig_sub)
  static size_t attr_set[2] = {0, 0};
  size_t& aset = attr_set[sizeof(TE) == 8 ? 1 : 0];
  if (sm > aset) {
    cudaFuncSetAttribute(k_eig_topk<TE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    aset = sm;
  }
  // FP32 Grams up to 192 x 192 are tridiagonalized by the register kernel first; the reflectors
  // (n x n floats) and the tridiagonal (3n floats) fit in Aw, which holds n x n doubles
  int pre = 0;
  if (sizeof(TE) == 4 && n >= 3 && n <= TRI_NMAX) {
    float* V = reinterpret_cast<float*>(Aw);
    float* tri = V + (size_t)n * n;
    if (n <= 24) k_tridiag_reg<12, 2, 1><<<1, 12 * 32, 0, st>>>(ctl, k, mode, G, V, tri);
    else if (n <= 48) k_tridiag_reg<12, 4, 2><<<1, 12 * 32, 0, st>>>(ctl, k, mode, G, V, tri);
    else if (n <= 96) k_tridiag_reg<12, 8, 3><<<1, 12 * 32, 0, st>>>(ctl, k, mode, G, V, tri);
    else k_tridiag_reg<12, 16, 6><<<1, 12 * 32, 0, st>>>(ctl, k, mode, G, V, tri);
    pre = 1;
  }
  k_eig_topk<TE><<<1, sizeof(TE) == 4 ? EIG_NT_F32 : EIG_NT, sm, st>>>(ctl, k, mode, ea, use_vec, use_amat, pre);
  return cudaGetLastError();
}

template <typename TW>
cudaError_t launch_append(Ctl* ctl, int k, int mode, const double* W, double* U, void* Uw, int ldu,
                          int n, cudaStream_t st) {
  k_append_factor<TW><<<1, 1024, sizeof(double) * n, st>>>(ctl, k, mode, W, U, (TW*)Uw, ldu);
  return cudaGetLastError();
}

template cudaError_t launch_eig<double>(Ctl*, int, int, const double*, void*, void*, void*, double*,
                                        double*, int, int, cudaStream_t);
template cudaError_t launch_eig<float>(Ctl*, int, int, const double*, void*, void*, void*, double*,
                                       double*, int, int, cudaStream_t);
template cudaError_t launch_append<double>(Ctl*, int, int, const double*, double*, void*, int, int,
                                           cudaStream_t);
template cudaError_t launch_append<float>(Ctl*, int, int, const double*, double*, void*, int, int,
                                          cudaStream_t);

}  // namespace tk
