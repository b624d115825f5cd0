// Growth eigensolver of the mixed form: the top eigenpairs of a residual Gram G = E_(k) E_(k)^T
// and Alg. 1's rank cut (inside Alg. 4), without the O(n^3) tridiagonalization.
//
// Alg. 1 keeps the smallest l with lambda_{l+1} + ... + lambda_n <= eps^2. For a residual Gram
// the cut sits at the top of the spectrum (||E_k||^2 = trace(G) exceeds eps^2 by a little), so
// only the few eigenpairs above the cut are needed:
//
//   k_eig_sub     one CTA, FP32: block subspace iteration Z = G Q on SB vectors with a
//                 Rayleigh-Ritz step every iteration (Golub & Van Loan, Matrix Computations,
//                 Sec. 8.2.4 "orthogonal iteration" and Sec. 8.1.2 Rayleigh-Ritz; rotating the
//                 basis to the Ritz vectors every iteration keeps the next G Q well conditioned
//                 for the Cholesky QR), one-sided Jacobi for the SB x SB projected matrix
//                 (Sec. 8.6.3, round-robin ordering), column-scaled Cholesky QR applied twice for
//                 the orthonormalization. It stops when the
//                 residuals ||G q_c - theta_c q_c|| of the Ritz pairs up to one past the FP32 cut
//                 are below SUB_TOL theta_1, and hands those m Ritz vectors on.
//   k_eig_refine  all SMs, FP64: P = W^T G W and M = W^T W for the m vectors, then the cut in
//                 FP64 from the nested Rayleigh-Ritz sums: the energy of G captured by
//                 span(w_1..w_l) is trace(M_l^-1 P_l) (leading l x l blocks), evaluated to first
//                 order in Delta = M - I (|Delta| is at FP32 rounding level, so the neglected
//                 terms are ~|Delta|^2 |P|); tail(l) = trace(G) - that energy, with trace(G)
//                 summed in FP64 from G's diagonal. tail(l) is the exact discarded energy of the
//                 subspace that the augmentation appends.
//
// When the subspace step cannot certify the cut (no convergence within SUB_MAXIT iterations, the
// cut deeper than SB - 2 vectors, a Cholesky breakdown, small problems) it sets ctl->eig_fb[k]
// and the full tridiagonal solver of k_eig.cu (predicated on that flag) decides instead.
#include "common.cuh"
#include "kernels.cuh"

namespace tk {

constexpr int SB = 16;                   // block size of the subspace iteration
constexpr int SUB_NT = 512;              // one thread per row of Q and Z (n <= 512)
constexpr int SUB_NW = SUB_NT / 32;
constexpr int SUB_MAXIT = 40;

constexpr float SUB_TOL = 4e-6f;         // Ritz residual / theta_1 accepted as converged
constexpr int SUB_GS_NMAX = 192;         // G held in shared memory (FP32) up to this n
constexpr int SUB_NMIN = 48;             // smaller Grams go to the full solver (cheap there)
constexpr int REF_NT = 128;
constexpr int REF_MAXB = 96;             // CTAs of k_eig_refine

// Floats of the shared-memory copy of G, rounded up to a multiple of 4 so that the region after
// it starts on a 16-byte boundary (n odd gives an odd n^2).
__host__ __device__ __forceinline__ size_t sub_gs_floats(int n) {
  return ((size_t)n * n + 3) / 4 * 4;
}

// Counter-based start vectors (a hash of row and column): deterministic, entries in [-1, 1).
__device__ __forceinline__ float sub_hash(int i, int c) {
  unsigned h = (unsigned)i * 0x9E3779B1u ^ ((unsigned)(c + 1) * 0x85EBCA77u);
  h ^= h >> 16; h *= 0x7FEB352Du; h ^= h >> 15; h *= 0x846CA68Bu; h ^= h >> 16;
  return (float)(h >> 8) * (2.0f / 16777216.0f) - 1.0f;
}

// Sum over the block of the SB x SB outer products a_i b_i^T of every thread's row vectors,
// into out[SB * SB] (shared). Four rounds of 64 values (rows 4g .. 4g + 3 of the product): a
// butterfly reduce-scatter leaves lane l with the warp sums of values 2l and 2l + 1, the warps'
// sums are then added in warp order (a fixed order: deterministic).
__device__ void sub_outer_sum(const float (&a)[SB], const float (&b)[SB], float* red, float* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll 1
  for (int g = 0; g < SB / 4; ++g) {
    float p[64];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 16; ++c) p[r * 16 + c] = a[4 * g + r] * b[c];
#pragma unroll
    for (int lev = 0; lev < 5; ++lev) {
      const int M = 16 >> lev;          // lane bit exchanged at this level
      const int H = 32 >> lev;          // half of the values still held
      const bool up = (lane & M) != 0;
#pragma unroll
      for (int t = 0; t < H; ++t) {
        const float keep = up ? p[H + t] : p[t];
        const float send = up ? p[t] : p[H + t];
        p[t] = keep + __shfl_xor_sync(0xffffffffu, send, M);
      }
    }
    red[wid * 64 + 2 * lane] = p[0];
    red[wid * 64 + 2 * lane + 1] = p[1];
    __syncthreads();
    if (threadIdx.x < 64) {
      float s = 0.f;
      for (int w = 0; w < SUB_NW; ++w) s += red[w * 64 + threadIdx.x];
      out[64 * g + threadIdx.x] = s;
    }
    __syncthreads();
  }
}

// Block sums of SB per-thread values into out[SB] (shared): reduce-scatter to lanes 2c, 2c + 1
// holding value c, then warp order.
__device__ void sub_vec_sum(const float (&v)[SB], float* red, float* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float p[SB];
#pragma unroll
  for (int c = 0; c < SB; ++c) p[c] = v[c];
#pragma unroll
  for (int lev = 0; lev < 4; ++lev) {
    const int M = 16 >> lev;
    const int H = 8 >> lev;
    const bool up = (lane & M) != 0;
#pragma unroll
    for (int t = 0; t < H; ++t) {
      const float keep = up ? p[H + t] : p[t];
      const float send = up ? p[t] : p[H + t];
      p[t] = keep + __shfl_xor_sync(0xffffffffu, send, M);
    }
  }
  const float tot = p[0] + __shfl_xor_sync(0xffffffffu, p[0], 1);   // value lane >> 1
  if ((lane & 1) == 0) red[wid * SB + (lane >> 1)] = tot;
  __syncthreads();
  if (threadIdx.x < SB) {
    float s = 0.f;
    for (int w = 0; w < SUB_NW; ++w) s += red[w * SB + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// Eigenpairs of the symmetric positive semidefinite SB x SB matrix H (shared, row stride SB + 1)
// by one-sided (Hestenes) Jacobi, one warp in registers: lane i (and its mirror i + 16) holds
// column i of W (initially H) and of V (initially I); each round of the round-robin ordering
// pairs every column with one partner, whose columns come by shuffle, and rotates the pair so
// that the two columns of W V become orthogonal (Golub & Van Loan, Matrix Computations,
// Sec. 8.6.3, one-sided Jacobi). At convergence H V = W has orthogonal columns, so V holds the
// eigenvectors and the column norms of W are the eigenvalues (for H positive semidefinite its
// singular values). A pair counts as orthogonal once |w_p . w_q| <= 4e-6 |w_p| |w_q| (the FP32
// rounding of a 16-term dot product is ~1e-6 of that bound's scale, so tighter tests only stir
// noise; the cut and the captured energy are recomputed in FP64 afterwards). Stops after a
// sweep that rotated nothing, or after max_sweeps. Writes the
// eigenvectors as the columns of Y (stride SB + 1) and the eigenvalues over the diagonal of H.
__device__ void sub_jacobi(float* H, float* Y, int lane, int max_sweeps) {
  constexpr int L = SB + 1;
  const int i = lane & (SB - 1);
  const int half = lane & SB;   // lanes 16..31 repeat the work of lanes 0..15
  float w[SB], v[SB];
#pragma unroll
  for (int x = 0; x < SB; ++x) {
    w[x] = H[x * L + i];
    v[x] = x == i ? 1.f : 0.f;
  }
  __syncwarp();
#pragma unroll 1
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    int rotated = 0;
#pragma unroll 1
    for (int rnd = 0; rnd < SB - 1; ++rnd) {
      // position of column i in this round, and its partner (positions x and SB - 1 - x pair up)
      const int xi = i == 0 ? 0 : 1 + (i - 1 - rnd + 2 * (SB - 1)) % (SB - 1);
      const int xp = SB - 1 - xi;
      const int j = xp == 0 ? 0 : 1 + (xp - 1 + rnd) % (SB - 1);
      const int src = half | j;
      float wo[SB], vo[SB];
#pragma unroll
      for (int x = 0; x < SB; ++x) {
        wo[x] = __shfl_sync(0xffffffffu, w[x], src);
        vo[x] = __shfl_sync(0xffffffffu, v[x], src);
      }
      // the same sums on both lanes of the pair (products commute, same order)
      float nown = 0.f, noth = 0.f, dot = 0.f;
#pragma unroll
      for (int x = 0; x < SB; ++x) {
        nown = fmaf(w[x], w[x], nown);
        noth = fmaf(wo[x], wo[x], noth);
        dot = fmaf(w[x], wo[x], dot);
      }
      const bool isp = i < j;
      const float al = isp ? nown : noth, be = isp ? noth : nown;
      if (fabsf(dot) > 4e-6f * sqrtf(al * be) && fabsf(dot) > 1e-30f) {
        const float ze = (be - al) / (2.f * dot);
        const float t = copysignf(1.f, ze) / (fabsf(ze) + sqrtf(fmaf(ze, ze, 1.f)));
        const float c = rsqrtf(fmaf(t, t, 1.f));
        const float sn = c * t;
        // p <- c p - s q, q <- s p + c q
#pragma unroll
        for (int x = 0; x < SB; ++x) {
          w[x] = isp ? fmaf(c, w[x], -sn * wo[x]) : fmaf(sn, wo[x], c * w[x]);
          v[x] = isp ? fmaf(c, v[x], -sn * vo[x]) : fmaf(sn, vo[x], c * v[x]);
        }
        rotated = 1;
      }
    }
    if (!__any_sync(0xffffffffu, rotated)) break;
  }
  float nn = 0.f;
#pragma unroll
  for (int x = 0; x < SB; ++x) nn = fmaf(w[x], w[x], nn);
  if (lane < SB) {
#pragma unroll
    for (int x = 0; x < SB; ++x) Y[x * L + i] = v[x];
    H[i * L + i] = sqrtf(nn);
  }
  __syncwarp();
}

// Cholesky R^T R = M of the SB x SB matrix M (shared, stride SB + 1; read only), one warp in
// registers: lane j (< SB) holds column j of the shrinking Schur complement, the pivot row of
// each step is shuffled from its owner. R upper triangular into R (stride SB + 1),
// rinv[c] = 1 / R(c, c). Returns false on a non-positive pivot.
__device__ bool sub_cholesky(const float* M, float* R, float* rinv, int lane) {
  constexpr int L = SB + 1;
  const int j = lane < SB ? lane : SB - 1;
  float col[SB];
#pragma unroll
  for (int x = 0; x < SB; ++x) col[x] = M[x * L + j];
  bool ok = true;
  float rrow[SB];   // rrow[c] = R(c, j)
#pragma unroll
  for (int c = 0; c < SB; ++c) {
    const float dcc = __shfl_sync(0xffffffffu, col[c], c);
    if (!(dcc > 0.f)) ok = false;
    const float rcc = ok ? sqrtf(dcc) : 1.f;
    const float ri = 1.f / rcc;
    const float rcj = j < c ? 0.f : (j == c ? rcc : col[c] * ri);
    rrow[c] = rcj;
    if (lane == 0) rinv[c] = ri;
    // Schur complement: col[x] -= R(c, x) R(c, j) for x > c (R(c, x) from lane x)
#pragma unroll
    for (int x = c + 1; x < SB; ++x) {
      const float rcx = __shfl_sync(0xffffffffu, rcj, x);
      col[x] = fmaf(-rcx, rcj, col[x]);
    }
  }
  if (lane < SB) {
#pragma unroll
    for (int c = 0; c < SB; ++c) R[c * L + lane] = rrow[c];
  }
  __syncwarp();
  return __all_sync(0xffffffffu, ok);
}

struct SubArgs {
  const double* G;   // n x n residual Gram (FP64, column-major, symmetric)
  float* Gf;         // n x n FP32 scratch (global) when G does not fit in shared memory
  double* W;         // n x mcap: the m Ritz vectors (FP64 copies)
  int mcap;
};

__global__ void __launch_bounds__(SUB_NT, 1) k_eig_sub(Ctl* ctl, int k, SubArgs a) {
  extern __shared__ __align__(16) float sub_dyn[];
  if (ctl->status || !ctl->grew[k]) return;
  const int n = ctl->n[k];
  const int r0 = ctl->r[k];
  const int nfree = n - r0;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int want = max(rp_grow_of(ctl, k), 0);
  // small or nearly full problems, or a forced cut deeper than the block: the full solver
  if (n < SUB_NMIN || nfree < SB + 2 || want + 1 > SB - 2 || n > SUB_NT) {
    if (tid == 0) ctl->eig_fb[k] = 1;
    return;
  }
  const bool gsm = n <= SUB_GS_NMAX;
  float* Gs = sub_dyn;                                   // n x n (if gsm)
  // Q's rows are read and written as float4: its offset is rounded up to 4 floats (16 bytes)
  float* Qs = sub_dyn + (gsm ? sub_gs_floats(n) : 0);   // [n][SB], row j's SB values contiguous
  float* red = Qs + (size_t)n * SB;                      // [SUB_NW][64]
  float* H = red + SUB_NW * 64;                          // SB x (SB + 1)
  float* Y = H + SB * (SB + 1);                          // SB x (SB + 1)
  float* R = Y + SB * (SB + 1);                          // SB x (SB + 1)
  float* vs = R + SB * (SB + 1);                         // [4][SB]: theta, residual^2, scale, rinv
  __shared__ int s_flag[4];
  __shared__ double s_tr[SUB_NW];
  const float* Gcol = gsm ? Gs : a.Gf;

  // G in FP32 (k_gram_f32 wrote it to the global scratch; small ones are copied into shared
  // memory), trace(G) in FP64 from its diagonal
  const int nn = n * n;
  if (gsm) {
    const float4* g4 = reinterpret_cast<const float4*>(a.Gf);
    for (int L = tid; L < nn / 4; L += SUB_NT) reinterpret_cast<float4*>(Gs)[L] = g4[L];
    for (int L = nn / 4 * 4 + tid; L < nn; L += SUB_NT) Gs[L] = a.Gf[L];
  }
  double trp = tid < n ? a.G[(size_t)tid * (n + 1)] : 0.0;
  trp = warp_sum(trp);
  if (lane == 0) s_tr[wid] = trp;
  if (tid == 0) { s_flag[0] = 0; s_flag[1] = 0; s_flag[2] = -1; s_flag[3] = 0; }
  __syncthreads();
  double trace = 0.0;
  for (int w = 0; w < SUB_NW; ++w) trace += s_tr[w];
  const double eps2 = ctl->eps * ctl->eps;

  const bool live = tid < n;
  float q[SB], z[SB];
#pragma unroll
  for (int c = 0; c < SB; ++c) q[c] = live ? sub_hash(tid, c) : 0.f;

  // column-scaled Cholesky QR of the rows x[] (every thread's row), twice; false on breakdown
  auto orthonormalize = [&](float (&x)[SB]) -> bool {
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
      float sq[SB];
#pragma unroll
      for (int c = 0; c < SB; ++c) sq[c] = x[c] * x[c];
      sub_vec_sum(sq, red, vs + 2 * SB);
      // scale columns to unit norm; a vanished column restarts from a hash vector
#pragma unroll
      for (int c = 0; c < SB; ++c) {
        const float nn = vs[2 * SB + c];
        if (nn > 1e-30f) x[c] *= rsqrtf(nn);
        else x[c] = live ? sub_hash(tid + 7919 * (pass + 1), c) * rsqrtf((float)n) : 0.f;
      }
      sub_outer_sum(x, x, red, Y);   // M = X^T X into Y (scratch, row stride SB)
      if (wid == 0) {
        // M to row stride SB + 1 (in H) for the factorization
        for (int it = lane; it < SB * SB; it += 32) H[(it / SB) * (SB + 1) + it % SB] = Y[it];
        __syncwarp();
        const bool ok = sub_cholesky(H, R, vs + 3 * SB, lane);
        if (lane == 0 && !ok) s_flag[1] = 1;
      }
      __syncthreads();
      if (s_flag[1]) return false;
      // x <- x R^-1 (row times the inverse of the upper triangular factor)
#pragma unroll
      for (int c = 0; c < SB; ++c) {
        float v = x[c];
#pragma unroll
        for (int b = 0; b < SB; ++b)
          if (b < c) v = fmaf(-x[b], R[b * (SB + 1) + c], v);
        x[c] = v * vs[3 * SB + c];
      }
      __syncthreads();
    }
    return true;
  };

  bool ok = orthonormalize(q);
  int it = 0, m = 0;
  bool conv = false;
#pragma unroll 1
  for (; ok && it < SUB_MAXIT; ++it) {
    // Q into shared memory, then Z = G Q (thread i: row i, G(j, i) = G(i, j) read down column i)
    if (live) {
#pragma unroll
      for (int c4 = 0; c4 < SB / 4; ++c4)
        reinterpret_cast<float4*>(Qs + (size_t)tid * SB)[c4] = make_float4(q[4 * c4], q[4 * c4 + 1], q[4 * c4 + 2], q[4 * c4 + 3]);
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < SB; ++c) z[c] = 0.f;
    if (live) {
      // G's column tid in groups of 16 entries, all loaded before their FMAs (G comes from L2
      // when it does not fit in shared memory: its latency is hidden by the loads in flight)
      const float* gc = Gcol + tid;
      int j = 0;
#pragma unroll 1
      for (; j + 16 <= n; j += 16) {
        float g[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) g[u] = gc[(size_t)(j + u) * n];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const float4* qj = reinterpret_cast<const float4*>(Qs + (size_t)(j + u) * SB);
#pragma unroll
          for (int c4 = 0; c4 < SB / 4; ++c4) {
            const float4 v = qj[c4];
            z[4 * c4] = fmaf(g[u], v.x, z[4 * c4]);
            z[4 * c4 + 1] = fmaf(g[u], v.y, z[4 * c4 + 1]);
            z[4 * c4 + 2] = fmaf(g[u], v.z, z[4 * c4 + 2]);
            z[4 * c4 + 3] = fmaf(g[u], v.w, z[4 * c4 + 3]);
          }
        }
      }
      for (; j < n; ++j) {
        const float g = gc[(size_t)j * n];
        const float4* qj = reinterpret_cast<const float4*>(Qs + (size_t)j * SB);
#pragma unroll
        for (int c4 = 0; c4 < SB / 4; ++c4) {
          const float4 v = qj[c4];
          z[4 * c4] = fmaf(g, v.x, z[4 * c4]);
          z[4 * c4 + 1] = fmaf(g, v.y, z[4 * c4 + 1]);
          z[4 * c4 + 2] = fmaf(g, v.z, z[4 * c4 + 2]);
          z[4 * c4 + 3] = fmaf(g, v.w, z[4 * c4 + 3]);
        }
      }
    }
    // Rayleigh-Ritz: H = Q^T Z, H = Y Theta Y^T
    sub_outer_sum(q, z, red, Y);
    if (wid == 0) {
      for (int it2 = lane; it2 < SB * SB; it2 += 32) {
        const int x = it2 / SB, y = it2 % SB;
        H[x * (SB + 1) + y] = 0.5f * (Y[x * SB + y] + Y[y * SB + x]);
      }
      __syncwarp();
      // (from the second iteration on the basis holds the previous Ritz vectors: H is nearly
      // diagonal and the sweeps stop early)
      sub_jacobi(H, R, lane, 10);
      // sort the Ritz values descending (rank of each, ties by index); Y = eigenvectors sorted
      float th = lane < SB ? H[lane * (SB + 1) + lane] : 0.f;
      int rk = 0;
      for (int j = 0; j < SB; ++j) {
        const float tj = __shfl_sync(0xffffffffu, th, j);
        if (lane < SB && (tj > th || (tj == th && j < lane))) ++rk;
      }
      if (lane < SB) {
        vs[rk] = th;
        for (int x = 0; x < SB; ++x) Y[x * (SB + 1) + rk] = R[x * (SB + 1) + lane];
      }
    }
    __syncthreads();
    // rotate Q and Z to the Ritz basis: q <- q Y, z <- z Y
    {
      float q2[SB], z2[SB];
#pragma unroll
      for (int c = 0; c < SB; ++c) {
        float aq = 0.f, az = 0.f;
#pragma unroll
        for (int b = 0; b < SB; ++b) {
          const float y = Y[b * (SB + 1) + c];
          aq = fmaf(q[b], y, aq);
          az = fmaf(z[b], y, az);
        }
        q2[c] = aq;
        z2[c] = az;
      }
#pragma unroll
      for (int c = 0; c < SB; ++c) { q[c] = q2[c]; z[c] = z2[c]; }
    }
    // residual norms of the Ritz pairs
    {
      float rr[SB];
#pragma unroll
      for (int c = 0; c < SB; ++c) {
        const float e = fmaf(-vs[c], q[c], z[c]);
        rr[c] = e * e;
      }
      sub_vec_sum(rr, red, vs + SB);
    }
    // FP32 cut estimate and convergence of the Ritz pairs up to one past it
    if (tid == 0) {
      double tail = trace;
      int l = -1;
      for (int c = 0; c < SB - 2; ++c) {
        tail -= (double)vs[c];
        if (tail <= eps2) { l = c + 1; break; }
      }
      int mm = (want > 0) ? want + 1 : (l > 0 ? l + 1 : 0);
      if (mm > nfree) mm = nfree;
      bool cv = mm > 0 && vs[0] > 0.f;
      const float tol = SUB_TOL * vs[0];
      for (int c = 0; c < mm && cv; ++c) cv = sqrtf(vs[SB + c]) <= tol;
      s_flag[0] = cv ? 1 : 0;
      s_flag[2] = mm;
    }
    __syncthreads();
    if (s_flag[0]) { conv = true; m = s_flag[2]; break; }
    // next basis: the columns of Z, orthonormalized
#pragma unroll
    for (int c = 0; c < SB; ++c) q[c] = z[c];
    ok = orthonormalize(q);
  }
  if (!conv) {
    if (tid == 0) { ctl->eig_fb[k] = 1; ctl->eig_it[k] = it; }
    return;
  }
  if (live)
    for (int c = 0; c < m; ++c) a.W[(long long)c * n + tid] = (double)q[c];
  if (tid == 0) {
    ctl->eig_m[k] = m;
    ctl->eig_it[k] = it + 1;
    ctl->eig_fb[k] = 0;
  }
}

// FP64 Rayleigh-Ritz over the m Ritz vectors and Alg. 1's cut (see the file comment).
// Grid: up to REF_MAXB CTAs, one warp per row of G W at a time. post = 0: the vectors of
// k_eig_sub (skipped when it handed the mode to the full solver); post = 1: after the full FP32
// solver (only then), over the eigenvectors it formed (its cut and one more): the cut and its
// tails in FP64 again, the FP32 cut kept if the FP64 one lies past those vectors.
__global__ void __launch_bounds__(REF_NT) k_eig_refine(Ctl* ctl, int k, const double* __restrict__ G,
                                                      const double* __restrict__ W, double* part, int mcap,
                                                      int post) {
  if (ctl->status || !ctl->grew[k]) return;
  if (post ? !ctl->eig_fb[k] : ctl->eig_fb[k]) return;
  const int n = ctl->n[k];
  const int m = ctl->eig_m[k];
  // (after the full solver the vectors may exceed the block: its FP32 cut then stands)
  if (m < 1 || m > SB) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int NWR = REF_NT / 32;
  constexpr int E = SB * SB / 32;   // entries of an m x m matrix per lane (m <= SB)
  // per-warp partials of P = W^T G W and M = W^T W, entry e = lane + 32 u (row e / SB, col e % SB)
  double pp[E], pm[E];
#pragma unroll
  for (int u = 0; u < E; ++u) { pp[u] = 0.0; pm[u] = 0.0; }
  for (int i = blockIdx.x * NWR + wid; i < n; i += gridDim.x * NWR) {
    // (G W)(i, c) = sum_j G(j, i) W(j, c), lanes over j
    double gw[SB];
#pragma unroll
    for (int c = 0; c < SB; ++c) gw[c] = 0.0;
    for (int j = lane; j < n; j += 32) {
      const double g = G[(long long)i * n + j];
#pragma unroll
      for (int c = 0; c < SB; ++c)
        if (c < m) gw[c] = fma(g, W[(long long)c * n + j], gw[c]);
    }
#pragma unroll
    for (int c = 0; c < SB; ++c) if (c < m) gw[c] = warp_sum(gw[c]);
#pragma unroll
    for (int u = 0; u < E; ++u) {
      const int e = lane + 32 * u, x = e / SB, y = e % SB;
      if (x < m && y < m) {
        const double wx = W[(long long)x * n + i];
        double gy = 0.0, wy = W[(long long)y * n + i];
#pragma unroll
        for (int c = 0; c < SB; ++c) if (c == y) gy = gw[c];
        pp[u] = fma(wx, gy, pp[u]);
        pm[u] = fma(wx, wy, pm[u]);
      }
    }
  }
  __shared__ double sp[NWR][2 * SB * SB];
#pragma unroll
  for (int u = 0; u < E; ++u) {
    sp[wid][lane + 32 * u] = pp[u];
    sp[wid][SB * SB + lane + 32 * u] = pm[u];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 2 * SB * SB; e += REF_NT) {
    double s = 0.0;
    for (int w = 0; w < NWR; ++w) s += sp[w][e];
    part[(long long)blockIdx.x * 2 * SB * SB + e] = s;
  }
  if (!tk_block_ticket(&ctl->ticket[3])) return;
  // last block: sum the partials in block order, then the nested traces and the cut
  __shared__ double Pm[2 * SB * SB];
  for (int e = threadIdx.x; e < 2 * SB * SB; e += REF_NT) {
    double s = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(part + (long long)b * 2 * SB * SB + e);
    Pm[e] = s;
  }
  __syncthreads();
  const double* P = Pm;
  const double* M = Pm + SB * SB;
  // energy captured by span(w_1..w_{l+1}) minus that of span(w_1..w_l), to first order in
  // Delta = M - I: trace(M_l^-1 P_l) = trace(P_l) - trace(Delta_l P_l) + O(|Delta|^2 |P|), so
  // inc(l) = P_ll - Delta_ll P_ll - 2 sum_{x<l} Delta_lx P_xl (P and Delta symmetric)
  __shared__ double inc[SB];
  if (threadIdx.x < SB) {
    const int l = threadIdx.x;
    double v = 0.0;
    if (l < m) {
      double d1 = (M[l * SB + l] - 1.0) * P[l * SB + l];
      for (int x = 0; x < l; ++x) d1 = fma(2.0 * M[l * SB + x], P[x * SB + l], d1);
      v = P[l * SB + l] - d1;
    }
    inc[l] = v;
  }
  // trace(G) in FP64, one warp over the diagonal
  __shared__ double s_trace;
  if (threadIdx.x < 32) {
    double tr = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) tr += G[(long long)i * n + i];
    tr = warp_sum(tr);
    if (threadIdx.x == 0) s_trace = tr;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double eps2 = ctl->eps * ctl->eps;
    const double trace = s_trace;
    const int want = max(rp_grow_of(ctl, k), 0);
    const int r0 = ctl->r[k];
    double tail = trace, prev = trace;
    int l = -1;
    for (int c = 0; c < m; ++c) {
      prev = tail;
      tail -= inc[c];
      if ((want > 0 && c + 1 == want) || (want == 0 && tail <= eps2)) { l = c + 1; break; }
    }
    if (l < 0 && post) {
      // past the vectors formed: the full solver's cut stands, its tails recomputed in FP64
      l = min(ctl->radd[k], m);
      if (l >= 1) {
        double tt = trace;
        for (int c = 0; c < l; ++c) { prev = tt; tt -= inc[c]; }
        tail = tt;
      } else {
        l = -2;   // nothing to refine
      }
    }
    if (l == -1) {
      ctl->eig_fb[k] = 1;   // the cut lies beyond the certified vectors: full solver
    } else if (l >= 1) {
      if (l > n - r0) l = n - r0;
      if (r0 + l > ctl->cap[k] || l > mcap) { ctl->status = TK_ECAPACITY; return; }
      // a discarded energy is not negative: below the Gram's own resolution (its FP32
      // accumulation, ~u_fp32 trace(G)) the computed tail is rounding noise of either sign
      ctl->radd[k] = l;
      ctl->disc[k] = fmax(tail, 0.0);
      ctl->tail_prev[k] = fmax(prev, 0.0);
    }
  }
}

size_t eig_sub_smem(int n) {
  const bool gsm = n <= SUB_GS_NMAX;
  return sizeof(float) * ((gsm ? sub_gs_floats(n) : 0) + (size_t)n * SB + SUB_NW * 64 + 3 * SB * (SB + 1) + 4 * SB + 2 * SB);
}

// G (FP64) -> Gf (FP32) over all SMs for the subspace iteration (only when mode k grew).
__global__ void k_gram_f32(const Ctl* ctl, int k, const double* __restrict__ G, float* __restrict__ Gf) {
  if (ctl->status || !ctl->grew[k]) return;
  const int n = ctl->n[k];
  const int nn = n * n;
  for (int L = blockIdx.x * blockDim.x + threadIdx.x; L < nn; L += gridDim.x * blockDim.x)
    Gf[L] = (float)G[L];
}

cudaError_t launch_eig_sub(Ctl* ctl, int k, const double* G, void* Gf, double* W, int mcap,
                           double* part, int n, cudaStream_t st) {
  // the attribute is raised to the largest size any n needs (n = SUB_GS_NMAX, G in shared
  // memory) once, and never lowered: launches captured into a graph for one n must stay valid
  // after launches for another
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_eig_sub, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)eig_sub_smem(SUB_GS_NMAX));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const size_t sm = eig_sub_smem(n);
  SubArgs a{G, reinterpret_cast<float*>(Gf), W, mcap};
  k_gram_f32<<<std::min(152, std::max(1, (n * n + 1023) / 1024)), 256, 0, st>>>(ctl, k, G, a.Gf);
  k_eig_sub<<<1, SUB_NT, sm, st>>>(ctl, k, a);
  const int nb = std::min(REF_MAXB, std::max(1, (n + 3) / 4));
  k_eig_refine<<<nb, REF_NT, 0, st>>>(ctl, k, G, W, part, mcap, 0);
  return cudaGetLastError();
}

cudaError_t launch_eig_refine_post(Ctl* ctl, int k, const double* G, double* W, int mcap,
                                   double* part, int n, cudaStream_t st) {
  const int nb = std::min(REF_MAXB, std::max(1, (n + 3) / 4));
  k_eig_refine<<<nb, REF_NT, 0, st>>>(ctl, k, G, W, part, mcap, 1);
  return cudaGetLastError();
}

}  // namespace tk
