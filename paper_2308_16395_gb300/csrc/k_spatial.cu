// Spatial-mode kernels of the streaming update (Alg. 4) and of the batch ST-HOSVD (Alg. 2).
//
// A mode-k operand is viewed as a column-major (A, n, B) array: A = product of the (already
// updated) ranks of modes < k, n = n_k, B = product of the sizes of the spatial modes > k.
// Its mode-k fibers (the columns of the unfolding X_(k), Sec. 2.1) are indexed by f = a + A b.
//
//   k_ttm_proj   P = X x_k U^T (the TTM of Alg. 4, first step) and, fused, the residual
//                E = X - P x_k U with its squared norm (Alg. 4, second step) and ||Y||^2.
//   k_resid_gram partial Gram tiles of the residual unfolding E_(k) E_(k)^T (Alg. 1 on E_(k)).
//   k_ttm_expand out = X x_k U (reconstruction, Eq. tucker_def).
//   k_gram_data  partial Gram tiles of a data unfolding X_(k) X_(k)^T (Alg. 2's TruncatedSVD).
#include "common.cuh"
#include "kernels.cuh"

namespace tk {

constexpr int FT = 64;   // fibers per tile
constexpr int JC = 32;   // rows of the mode-k index per chunk
constexpr int RC = 128;  // output rows per register pass
constexpr int NT = 256;  // threads

struct SpatialView {
  long long A, B;
  int n;
};

template <typename TX, typename TW>
__device__ __forceinline__ void load_x_chunk(const TX* __restrict__ X, long long A, int n,
                                             long long F, long long f0, int j0, TW* Xs,
                                             const long long* fbase, typename AccOf<TW>::type* yacc) {
  // Xs[jj * FT + ff] = X(f0+ff, j0+jj)
  for (int L = threadIdx.x; L < JC * FT; L += NT) {
    int jj, ff;
    if (A == 1) { jj = L % JC; ff = L / JC; } else { jj = L / FT; ff = L % FT; }
    const long long f = f0 + ff;
    const int j = j0 + jj;
    TW v = TW(0);
    if (f < F && j < n) v = (TW)X[fbase[ff] + (long long)A * j];
    Xs[jj * FT + ff] = v;
    if (yacc) yacc->add(v * v);
  }
}

// P = X x_k U^T for every fiber; with RESID, also the squared norm of E = X - P x_k U.
// U: n x r (column-major, ld = ldu). P: (A, r, B) column-major. Partials per block.
// out_off: the output goes to D-buffer (xbuf + out_off) mod 3 (1: P_k of pass A, 2: D*_k of
// pass C). pred: run only if mode k grew (Alg. 4's else-branch).
template <typename TX, typename TW, bool RESID>
__global__ void __launch_bounds__(NT) k_ttm_proj(const Ctl* __restrict__ ctl, int k, int out_off,
                                                int pred, const TX* __restrict__ Xext,
                                                TW* const* dbufs, const TW* __restrict__ U,
                                                int ldu, double* __restrict__ part_e2,
                                                double* __restrict__ part_y2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (ctl->status) return;
  if (pred && !ctl->grew[k]) return;
  const int n = view_n(ctl, k);
  const long long A = view_A(ctl, k);
  const long long B = view_B(ctl, k);
  const int r = ctl->r[k];
  if (tc_proj_ok(ctl, k, r)) return;   // the tensor-core kernel does this pass
  const long long F = A * B;
  const long long pstr = out_stride(ctl, A, F);
  const int xb = ctl->xbuf;
  // the slice: the launch argument, or the graph update's slot in the control block
  const TX* X = (xb < 0) ? (Xext ? Xext : reinterpret_cast<const TX*>(ctl->yptr))
                         : reinterpret_cast<const TX*>(dbufs[xb]);
  TW* P = dbufs[(xb + out_off + 3) % 3];

  TW* Xs = reinterpret_cast<TW*>(smem_raw);                 // JC * FT
  TW* Us = Xs + JC * FT;                                    // JC * max(RC, r)
  const int ucols = r > RC ? r : RC;
  TW* Ps = Us + JC * ucols;                                 // r * FT (RESID only)
  __shared__ long long fbase[FT], pbase[FT];
  __shared__ double red[32];

  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  typename AccOf<TW>::type eacc, yacc;
  const bool want_y = (part_y2 != nullptr);
  const long long ntiles = (F + FT - 1) / FT;

  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long f0 = tile * FT;
    __syncthreads();
    if (tid < FT) {
      long long f = f0 + tid;
      if (f >= F) f = F - 1;
      const long long a = f % A, b = f / A;
      fbase[tid] = a + A * (long long)n * b;
      pbase[tid] = out_base(ctl, f, A, r);
    }
    __syncthreads();
    for (int rc0 = 0; rc0 < r; rc0 += RC) {
      const int rcn = min(RC, r - rc0);
      TW acc[RC / 16][FT / 16];
#pragma unroll
      for (int i = 0; i < RC / 16; ++i)
#pragma unroll
        for (int f = 0; f < FT / 16; ++f) acc[i][f] = TW(0);
      for (int j0 = 0; j0 < n; j0 += JC) {
        __syncthreads();
        load_x_chunk<TX, TW>(X, A, n, F, f0, j0, Xs, fbase,
                             (want_y && rc0 == 0) ? &yacc : nullptr);
        for (int L = tid; L < JC * RC; L += NT) {
          const int jj = L % JC, c = L / JC;
          const int j = j0 + jj;
          Us[jj * RC + c] = (c < rcn && j < n) ? U[(long long)(rc0 + c) * ldu + j] : TW(0);
        }
        __syncthreads();
#pragma unroll 4
        for (int jj = 0; jj < JC; ++jj) {
          TW xv[FT / 16];
#pragma unroll
          for (int f = 0; f < FT / 16; ++f) xv[f] = Xs[jj * FT + tx + 16 * f];
#pragma unroll
          for (int i = 0; i < RC / 16; ++i) {
            if (16 * i < rcn) {
              const TW u = Us[jj * RC + ty + 16 * i];
#pragma unroll
              for (int f = 0; f < FT / 16; ++f) acc[i][f] += u * xv[f];
            }
          }
        }
      }
      // write the P rows of this chunk
#pragma unroll
      for (int i = 0; i < RC / 16; ++i) {
        const int row = rc0 + ty + 16 * i;
        if (row >= rc0 + rcn) continue;
#pragma unroll
        for (int f = 0; f < FT / 16; ++f) {
          const int ff = tx + 16 * f;
          const long long fg = f0 + ff;
          if (fg < F) P[pbase[ff] + pstr * (long long)row] = acc[i][f];
          if (RESID) Ps[(long long)row * FT + ff] = acc[i][f];
        }
      }
    }
    if (RESID) {
      // E = X - U P, chunk by chunk over the mode-k index; squared norm accumulated.
      for (int j0 = 0; j0 < n; j0 += JC) {
        __syncthreads();
        load_x_chunk<TX, TW>(X, A, n, F, f0, j0, Xs, fbase, nullptr);
        for (int L = tid; L < JC * ucols; L += NT) {
          const int jj = L % JC, c = L / JC;
          const int j = j0 + jj;
          Us[jj * ucols + c] = (c < r && j < n) ? U[(long long)c * ldu + j] : TW(0);
        }
        __syncthreads();
        const int ff = tid % FT;
        const int jb = tid / FT;  // 0..3
        TW e[JC / 4];
#pragma unroll
        for (int i = 0; i < JC / 4; ++i) e[i] = Xs[(jb + 4 * i) * FT + ff];
        for (int c = 0; c < r; ++c) {
          const TW pv = Ps[(long long)c * FT + ff];
#pragma unroll
          for (int i = 0; i < JC / 4; ++i) e[i] -= Us[(jb + 4 * i) * ucols + c] * pv;
        }
        const bool fok = (f0 + ff) < F;
#pragma unroll
        for (int i = 0; i < JC / 4; ++i) {
          const int j = j0 + jb + 4 * i;
          if (fok && j < n) eacc.add(e[i] * e[i]);
        }
      }
    }
  }
  if (RESID) {
    const double s = block_sum(eacc.value(), red);
    if (tid == 0) part_e2[blockIdx.x] = s;
  }
  if (want_y) {
    const double s = block_sum(yacc.value(), red);
    if (tid == 0) part_y2[blockIdx.x] = s;
  }
}

// Reduce the per-block partials of mode k and take Alg. 4's branch: grew = ||E_k|| > eps.
// For k = 0 also ||Y||^2 and eps = tau ||Y|| / sqrt(d) (Alg. 5, first step).
// hcond (graph form): the conditional handle of mode k's growth body, set to grew[k].
__global__ void k_decide(Ctl* ctl, int k, const double* part_e2, const double* part_y2, int nparts,
                         cudaGraphConditionalHandle hcond) {
  if (ctl->status) {
    if (hcond && threadIdx.x == 0) cudaGraphSetConditional(hcond, 0u);
    return;
  }
  __shared__ double red[32];
  double se = 0.0, sy = 0.0;
  // fixed-order reduction (deterministic)
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    se += part_e2[i];
    if (k == 0) sy += part_y2[i];
  }
  se = block_sum(se, red);
  sy = block_sum(sy, red);
  if (threadIdx.x == 0) {
    // Alg. 4: skip if ||E_k|| <= eps, taken as ||E_k||^2 <= eps^2 (eps^2 = tau^2 ||Y||^2 / d) so
    // that the branch does not wait on square roots and a division (FP64 is long-latency here)
    double eps2;
    if (k == 0) {
      if (!isfinite(sy)) {
        ctl->y2 = sy;
        ctl->status = TK_ENUMERIC;
        if (hcond) cudaGraphSetConditional(hcond, 0u);
        return;
      }
      const double tau = ctl->tau;
      eps2 = tau * tau * sy * (1.0 / (double)ctl->d);
    } else {
      const double e = ctl->eps;
      eps2 = e * e;
    }
    int g = se > eps2 ? 1 : 0;
    // decision replay (test hook): the branch forced for this update
    const int fg = rp_grow_of(ctl, k);
    if (fg >= 0) g = fg > 0 ? 1 : 0;
    if (hcond) cudaGraphSetConditional(hcond, g ? 1u : 0u);
    ctl->e2[k] = se;
    ctl->grew[k] = g;
    // no growth: D*_k is P_k, the next buffer in the rotation (the growth chain, which would have
    // moved it two ahead, does not run; its kernels return before reading xbuf)
    if (!g) ctl->xbuf = (ctl->xbuf + 1) % 3;
    ctl->radd[k] = 0;
    ctl->disc[k] = g ? 0.0 : se;
    if (k == 0) {
      ctl->y2 = sy;
      ctl->eps = ctl->tau * sqrt(sy) / sqrt((double)ctl->d);
    }
    // FP16 scale of mode k's input for this update's later passes and the next update's pass A,
    // from the largest |x| of this input
    const unsigned mb = ctl->xmax[k];
    if (mb != 0u && mb < 0x7f800000u) ctl->x16e[k] = x16_sigma_for(x16_exp_of_bits(mb));
  }
}

// After mode k: the buffer holding D*_k becomes the input of mode k+1.
// grown_only (updates): the last kernel of mode k's growth chain, a no-op when mode k did not
// grow (k_decide advanced the buffer then). A growth changes the spatial core size, which must
// still fit the C/V capacity; without growth the size is the one checked when it last changed.
// Otherwise (initial ST-HOSVD): advance by one, as no mode grows there.
__global__ void k_mode_end(Ctl* ctl, int k, int grown_only) {
  if (ctl->status) return;
  if (grown_only && !ctl->grew[k]) return;
  const int xb = ctl->xbuf;
  ctl->xbuf = ctl->grew[k] ? (xb + 2 + 3) % 3 : (xb + 1 + 3) % 3;
  if (grown_only) {
    long long R = 1;
    for (int i = 0; i < ctl->d - 1; ++i) R *= ctl->r[i];
    if (R > ctl->core_cap) ctl->status = TK_ECAPACITY;
  }
}

// ---------------------------------------------------------------------------------------------
// Residual Gram: G = E_(k) E_(k)^T, E = X - P x_k U, tiles of 64 x 64 over (i, j), partial over
// fiber chunks. Grid: x = tile pair index (ti <= tj), y = fiber chunk.
// ---------------------------------------------------------------------------------------------
constexpr int GT = 64;   // Gram tile
constexpr int GF = 32;   // fibers per sub-step
constexpr int GC = 32;   // rank chunk

template <typename TX, typename TW>
__global__ void __launch_bounds__(NT) k_resid_gram(const Ctl* __restrict__ ctl, int k,
                                                  const TX* __restrict__ Xext, TW* const* dbufs,
                                                  const TW* __restrict__ U, int ldu,
                                                  double* __restrict__ gpart, int data_only) {
  if (ctl->status) return;
  if (!data_only && !ctl->grew[k]) return;
  if (!data_only && tc_gram_ok(ctl, k)) return;   // tensor-core Gram
  const int n = view_n(ctl, k);
  const long long A = view_A(ctl, k);
  const long long B = view_B(ctl, k);
  const int r = data_only ? 0 : ctl->rold[k];
  const long long F = A * B;
  const long long pstr = out_stride(ctl, A, F);
  const int xb = ctl->xbuf;
  // the slice: the launch argument, or the graph update's slot in the control block
  const TX* X = (xb < 0) ? (Xext ? Xext : reinterpret_cast<const TX*>(ctl->yptr))
                         : reinterpret_cast<const TX*>(dbufs[xb]);
  const TW* P = data_only ? nullptr : dbufs[(xb + 1 + 3) % 3];

  const int T = (n + GT - 1) / GT;
  // decode tile pair
  int pair = blockIdx.x, ti = 0;
  while (pair >= T - ti) { pair -= T - ti; ++ti; }
  const int tj = ti + pair;
  const int chunks = gridDim.y;
  const long long per = (F + chunks - 1) / chunks;
  const long long fb = (long long)blockIdx.y * per;
  const long long fe = min(F, fb + per);

  extern __shared__ __align__(16) unsigned char gsm_raw[];
  typedef TW RowF[GF + 1];
  typedef TW RowC[GC + 1];
  RowF* Ei = reinterpret_cast<RowF*>(gsm_raw);            // [GT][GF+1]
  RowF* Ej = Ei + GT;                                      // [GT][GF+1]
  RowC* Uci = reinterpret_cast<RowC*>(Ej + GT);            // [GT][GC+1]
  RowC* Ucj = Uci + GT;                                    // [GT][GC+1]
  RowF* Pc = reinterpret_cast<RowF*>(Ucj + GT);            // [GC][GF+1]
  __shared__ long long fbase[GF], pbase[GF];
  const int tid = threadIdx.x;
  const int gy = tid / 16, gx = tid % 16;   // 4 x 4 micro tile of G
  TW g[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) g[a][b] = TW(0);

  for (long long f0 = fb; f0 < fe; f0 += GF) {
    __syncthreads();
    if (tid < GF) {
      long long f = f0 + tid;
      if (f >= fe) f = fe - 1;
      const long long a = f % A, b = f / A;
      fbase[tid] = a + A * (long long)n * b;
      pbase[tid] = out_base(ctl, f, A, r);
    }
    __syncthreads();
    // x rows of both tiles
    for (int L = tid; L < 2 * GT * GF; L += NT) {
      const int which = L / (GT * GF);
      const int rem = L % (GT * GF);
      int row, ff;
      if (A == 1) { row = rem % GT; ff = rem / GT; } else { row = rem / GF; ff = rem % GF; }
      const int j = (which ? tj : ti) * GT + row;
      const bool ok = (f0 + ff < fe) && j < n;
      const TW v = ok ? (TW)X[fbase[ff] + A * (long long)j] : TW(0);
      if (which) Ej[row][ff] = v; else Ei[row][ff] = v;
    }
    for (int c0 = 0; c0 < r; c0 += GC) {
      __syncthreads();
      for (int L = tid; L < GC * GF; L += NT) {
        const int c = L / GF, ff = L % GF;
        const bool ok = (f0 + ff < fe) && (c0 + c < r);
        Pc[c][ff] = ok ? P[pbase[ff] + pstr * (long long)(c0 + c)] : TW(0);
      }
      for (int L = tid; L < 2 * GT * GC; L += NT) {
        const int which = L / (GT * GC);
        const int rem = L % (GT * GC);
        const int row = rem % GT, c = rem / GT;
        const int j = (which ? tj : ti) * GT + row;
        const TW v = (j < n && c0 + c < r) ? U[(long long)(c0 + c) * ldu + j] : TW(0);
        if (which) Ucj[row][c] = v; else Uci[row][c] = v;
      }
      __syncthreads();
      // E -= U_chunk * P_chunk for the 2 x 64 x 32 elements (16 per thread)
      for (int L = tid; L < 2 * GT * GF; L += NT) {
        const int which = L / (GT * GF);
        const int rem = L % (GT * GF);
        const int row = rem / GF, ff = rem % GF;
        TW s = TW(0);
#pragma unroll 8
        for (int c = 0; c < GC; ++c) s += (which ? Ucj[row][c] : Uci[row][c]) * Pc[c][ff];
        if (which) Ej[row][ff] -= s; else Ei[row][ff] -= s;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int ff = 0; ff < GF; ++ff) {
      TW a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = Ei[gy + 16 * q][ff]; b[q] = Ej[gx + 16 * q][ff]; }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) g[p][q] += a[p] * b[q];
    }
  }
  double* out = gpart + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * (GT * GT);
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) out[(gy + 16 * p) * GT + (gx + 16 * q)] = (double)g[p][q];
}

// Sum the Gram partials in fixed order into the symmetric n x n FP64 matrix G (column-major).
__global__ void k_gram_reduce(const Ctl* ctl, int k, const double* gpart, int pairs, int chunks,
                              double* G, int data_only) {
  if (ctl->status) return;
  if (!data_only && !ctl->grew[k]) return;
  if (!data_only && tc_gram_ok(ctl, k)) return;   // tensor-core Gram
  const int n = view_n(ctl, k);
  const int T = (n + GT - 1) / GT;
  const long long total = (long long)pairs * GT * GT;
  for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < total;
       L += (long long)gridDim.x * blockDim.x) {
    const int pr = (int)(L / (GT * GT));
    const int rem = (int)(L % (GT * GT));
    const int ii = rem / GT, jj = rem % GT;
    int pair = pr, ti = 0;
    while (pair >= T - ti) { pair -= T - ti; ++ti; }
    const int tj = ti + pair;
    const int i = ti * GT + ii, j = tj * GT + jj;
    if (i >= n || j >= n) continue;
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += gpart[((long long)c * pairs + pr) * (GT * GT) + rem];
    G[(long long)j * n + i] = s;
    G[(long long)i * n + j] = s;
  }
}

// out = X x_k U : out(a, j, b) = sum_i U(j, i) X(a, i, b); X is (A, r, B), out is (A, n, B).
template <typename TI, typename TW, typename TO>
__global__ void k_ttm_expand(const TI* __restrict__ X, long long A, int r, long long B,
                             const TW* __restrict__ U, int ldu, int n, TO* __restrict__ out) {
  const long long F = A * B;
  const long long total = F * n;
  for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < total;
       L += (long long)gridDim.x * blockDim.x) {
    const long long a = L % A;
    const long long rest = L / A;
    const int j = (int)(rest % n);
    const long long b = rest / n;
    TW s = TW(0);
    const TI* x = X + a + A * (long long)r * b;
    for (int i = 0; i < r; ++i) s += U[(long long)i * ldu + j] * (TW)x[A * (long long)i];
    out[L] = (TO)s;
  }
}

// ---------------------------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------------------------
size_t proj_smem_bytes(int r, int tw_size) {
  const int ucols = r > RC ? r : RC;
  return (size_t)tw_size * ((size_t)JC * FT + (size_t)JC * ucols + (size_t)r * FT);
}

// Raise a kernel's dynamic shared-memory limit to at least `bytes`, never lowering it: launches
// of one kernel with different sizes are captured into the same update graph, and each must stay
// within the limit in force when the graph runs. `seen` is the kernel's own high-water mark.
static inline void raise_smem_limit(const void* kern, size_t bytes, size_t* seen) {
  if (bytes > *seen) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    *seen = bytes;
  }
}

template <typename TX, typename TW>
cudaError_t launch_proj(const Ctl* ctl, int k, int out_off, int pred, const void* Xext,
                        void* const* dbufs, const void* U, int ldu, int rmax, double* part_e2,
                        double* part_y2, int grid, cudaStream_t st) {
  const size_t sm = proj_smem_bytes(rmax, sizeof(TW));
  static size_t seen[2] = {0, 0};
  if (part_e2) {
    auto kern = k_ttm_proj<TX, TW, true>;
    raise_smem_limit((const void*)kern, sm, &seen[0]);
    kern<<<grid, NT, sm, st>>>(ctl, k, out_off, pred, (const TX*)Xext, (TW* const*)dbufs,
                               (const TW*)U, ldu, part_e2, part_y2);
  } else {
    auto kern = k_ttm_proj<TX, TW, false>;
    raise_smem_limit((const void*)kern, sm, &seen[1]);
    kern<<<grid, NT, sm, st>>>(ctl, k, out_off, pred, (const TX*)Xext, (TW* const*)dbufs,
                               (const TW*)U, ldu, nullptr, part_y2);
  }
  return cudaGetLastError();
}

// ||X||^2 of a dense array (compensated per thread, FP64 per block; partials per block).
template <typename TX>
__global__ void k_norm2(const TX* __restrict__ X, long long N, double* part) {
  __shared__ double red[32];
  typename AccOf<TX>::type acc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const TX v = X[i];
    acc.add(v * v);
  }
  const double s = block_sum(acc.value(), red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <typename TX>
cudaError_t launch_norm2(const void* X, long long N, double* part, int grid, cudaStream_t st) {
  k_norm2<TX><<<grid, 256, 0, st>>>((const TX*)X, N, part);
  return cudaGetLastError();
}
template cudaError_t launch_norm2<float>(const void*, long long, double*, int, cudaStream_t);
template cudaError_t launch_norm2<double>(const void*, long long, double*, int, cudaStream_t);

template <typename TX, typename TW>
cudaError_t launch_resid_gram(const Ctl* ctl, int k, int n, const void* Xext, void* const* dbufs,
                              const void* U, int ldu, double* gpart, int pairs, int chunks,
                              int data_only, cudaStream_t st) {
  dim3 grid(pairs, chunks);
  const size_t sm = sizeof(TW) * ((size_t)2 * GT * (GF + 1) + (size_t)2 * GT * (GC + 1) +
                                  (size_t)GC * (GF + 1));
  auto kern = k_resid_gram<TX, TW>;
  static size_t seen = 0;
  raise_smem_limit((const void*)kern, sm, &seen);
  kern<<<grid, NT, sm, st>>>(ctl, k, (const TX*)Xext, (TW* const*)dbufs, (const TW*)U, ldu, gpart,
                             data_only);
  return cudaGetLastError();
}

cudaError_t launch_decide(Ctl* ctl, int k, const double* pe, const double* py, int nparts,
                          cudaGraphConditionalHandle hcond, cudaStream_t st) {
  k_decide<<<1, 256, 0, st>>>(ctl, k, pe, py, nparts, hcond);
  return cudaGetLastError();
}

cudaError_t launch_mode_end(Ctl* ctl, int k, int grown_only, cudaStream_t st) {
  k_mode_end<<<1, 1, 0, st>>>(ctl, k, grown_only);
  return cudaGetLastError();
}

cudaError_t launch_gram_reduce(const Ctl* ctl, int k, const double* gpart, int pairs, int chunks,
                               double* G, int data_only, cudaStream_t st) {
  k_gram_reduce<<<64, 256, 0, st>>>(ctl, k, gpart, pairs, chunks, G, data_only);
  return cudaGetLastError();
}

template <typename TI, typename TW, typename TO>
cudaError_t launch_expand(const void* X, long long A, int r, long long B, const void* U, int ldu,
                          int n, void* out, cudaStream_t st) {
  const long long total = A * B * n;
  int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
  if (grid < 1) grid = 1;
  k_ttm_expand<TI, TW, TO><<<grid, 256, 0, st>>>((const TI*)X, A, r, B, (const TW*)U, ldu, n,
                                                 (TO*)out);
  return cudaGetLastError();
}

#define INST_PROJ(TX, TW)                                                                          \
  template cudaError_t launch_proj<TX, TW>(const Ctl*, int, int, int, const void*, void* const*,   \
                                           const void*, int, int, double*, double*, int,           \
                                           cudaStream_t);                                          \
  template cudaError_t launch_resid_gram<TX, TW>(const Ctl*, int, int, const void*, void* const*,  \
                                                 const void*, int, double*, int, int, int,         \
                                                 cudaStream_t);
INST_PROJ(float, float)
INST_PROJ(double, double)
INST_PROJ(float, double)
INST_PROJ(double, float)

template cudaError_t launch_expand<float, float, float>(const void*, long long, int, long long,
                                                        const void*, int, int, void*, cudaStream_t);
template cudaError_t launch_expand<double, double, double>(const void*, long long, int, long long,
                                                           const void*, int, int, void*,
                                                           cudaStream_t);
template cudaError_t launch_expand<double, double, float>(const void*, long long, int, long long,
                                                          const void*, int, int, void*,
                                                          cudaStream_t);
template cudaError_t launch_expand<float, double, double>(const void*, long long, int, long long,
                                                          const void*, int, int, void*,
                                                          cudaStream_t);
template cudaError_t launch_expand<float, float, double>(const void*, long long, int, long long,
                                                         const void*, int, int, void*,
                                                         cudaStream_t);

}  // namespace tk
