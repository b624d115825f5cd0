// Streaming-mode kernels of the update (Alg. 3 inside Alg. 5) and the core update (Alg. 5, last
// step).
//
// State layout (device): C and V are stored "row per spatial index": row j (the column-major
// linear index of (i_1..i_{d-1}) over the current spatial ranks) holds the r_d streaming-mode
// coefficients contiguously, row stride tk_cv_stride(r_d) (compact up to r_d = 32, the
// streaming-rank capacity ldc above). So C_(d) = C^T and the
// matrix V of Alg. 3 (V = V_(d)^T) is exactly the stored R x r_d array. U_d is row-major
// (steps_cap x ldc). Zero padding of C and V in spatial modes (Alg. 4, PadWithZeros) is never
// materialised: kernels read old rows through the new->old index map (missing rows are zero).
//
//   k_isvd_p       p = V^T d                                    (Alg. 3, first step)
//   k_isvd_e       e = d - V p, ||e||^2, s = V^T e              (Alg. 3, second step + one
//                  classical Gram-Schmidt re-orthogonalisation of e against V, the QR of Alg. 3
//                  specialised to orthonormal V)
//   isvd_small_body q, the q <= eps branch, the compact SVD of S' through the secular equation
//                  of S'^T S' = diag(S^2[,0]) + z z^T (O(r^2) instead of O(r^3))
//   k_ud_update    U~_d = [U_d U''(1:r,:); U''(r+1,:)]          (Alg. 3)
//   k_core_m       M = U~_d(1:n_d,:)^T U_d                      (Alg. 5, last step)
//   k_cv_update    C~ = C M^T + d u^T and V~ = V' V''           (Alg. 5 / Alg. 3)
#include "common.cuh"
#include "kernels.cuh"

namespace tk {

// ---------------------------------------------------------------------------------------------
// Row passes over V (Alg. 3's projections). A warp streams batches of RB rows; lanes cover 32
// columns per column group, so every row read is coalesced and each lane keeps RB independent
// loads in flight. FP32 products are accumulated in FP32 over 32 rows, then flushed to FP64.
// ---------------------------------------------------------------------------------------------
constexpr int RB = 8;   // rows per warp batch

// p = V_pad^T d over the old rows; partials per block (TK_STREAM_CAP_MAX doubles each).
template <typename TW>
__global__ void __launch_bounds__(256) k_isvd_p(Ctl* __restrict__ ctl, TW* const* dbufs,
                                               TW* const* vbufs, double* __restrict__ part,
                                               double* __restrict__ pout) {
  if (ctl->status) return;
  if (rows_isvd_ok(ctl)) return;   // k_isvd_p_rows does this pass
  const int d = ctl->d, m = d - 1;
  const int r = ctl->r[d - 1];
  const int ldc = tk_cv_stride(r, ctl->ldc, (int)sizeof(TW));
  const TW* V = vbufs[ctl->cbuf];
  const TW* dv = dbufs[ctl->xbuf];
  long long Ro = 1;
  for (int i = 0; i < m; ++i) Ro *= ctl->rold[i];
  const bool same = !spatial_grew(ctl);
  int ro[TK_MAXD], rn[TK_MAXD];
  for (int i = 0; i < TK_MAXD; ++i) { ro[i] = ctl->rold[i]; rn[i] = ctl->r[i]; }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int CPL = TK_STREAM_CAP_MAX / 32;   // column groups
  const int CG = (r + 31) / 32;
  double acc[CPL];
  TW accf[CPL];
#pragma unroll
  for (int i = 0; i < CPL; ++i) { acc[i] = 0.0; accf[i] = TW(0); }
  const long long gw = (long long)blockIdx.x * 8 + wid;
  const long long nw = (long long)gridDim.x * 8;
  int batches = 0;
  for (long long j0 = gw * RB; j0 < Ro; j0 += nw * RB) {
    TW dj[RB];
    long long jo[RB];
#pragma unroll
    for (int i = 0; i < RB; ++i) {
      jo[i] = j0 + i;
      if (jo[i] < Ro) {
        int jn = (int)jo[i];
        if (!same) {
          int t = (int)jo[i], stride = 1;
          jn = 0;
          for (int k = 0; k < m; ++k) {
            const int ik = t % ro[k];
            t /= ro[k];
            jn += ik * stride;
            stride *= rn[k];
          }
        }
        dj[i] = dv[jn];
      } else {
        dj[i] = TW(0);
        jo[i] = -1;
      }
    }
#pragma unroll
    for (int g = 0; g < CPL; ++g) {
      if (g >= CG) break;
      const int c = g * 32 + lane;
      TW v[RB];
#pragma unroll
      for (int i = 0; i < RB; ++i) v[i] = (jo[i] >= 0 && c < r) ? V[jo[i] * ldc + c] : TW(0);
#pragma unroll
      for (int i = 0; i < RB; ++i) accf[g] += v[i] * dj[i];
    }
    if (++batches == 4) {
#pragma unroll
      for (int g = 0; g < CPL; ++g) { acc[g] += (double)accf[g]; accf[g] = TW(0); }
      batches = 0;
    }
  }
  __shared__ double sh[8][TK_STREAM_CAP_MAX];
#pragma unroll
  for (int g = 0; g < CPL; ++g) sh[wid][g * 32 + lane] = acc[g] + (double)accf[g];
  __syncthreads();
  for (int c = threadIdx.x; c < r; c += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += sh[w][c];
    part[(long long)blockIdx.x * TK_STREAM_CAP_MAX + c] = s;
  }
  tk_last_block_reduce(part, TK_STREAM_CAP_MAX, r, pout, &ctl->ticket[0]);
}

// q, the q <= eps branch of Alg. 3 and the deflated secular problem of S'^T S' (one thread of
// the e-pass's last block, once the cross-block sums p and [s; ||e||^2] are complete).
__device__ void isvd_small_body(Ctl* ctl, const double* p, const double* es, const double* S,
                                const SecWork& w) {
  const int d = ctl->d;
  const int r = ctl->r[d - 1];
  // CGS-corrected projection: p' = p + s, q'^2 = ||e||^2 - ||s||^2
  double s2 = 0.0;
  for (int c = 0; c < r; ++c) s2 += es[c] * es[c];
  double q2 = es[r] - s2;
  if (q2 < 0.0) q2 = 0.0;
  const double q = sqrt(q2);
  for (int c = 0; c < r; ++c) w.pq[c] = p[c] + es[c];
  w.pq[r] = q;
  ctl->q2 = q2;
  ctl->q = q;
  const int aug = q > ctl->eps ? 1 : 0;   // Alg. 3: ignore e if q <= eps
  ctl->aug = aug;
  if (aug && r + 1 > ctl->cap[d - 1]) { ctl->status = TK_ECAPACITY; return; }
  long long Rn = 1;
  for (int i = 0; i < d - 1; ++i) Rn *= ctl->r[i];
  if (Rn > ctl->core_cap) { ctl->status = TK_ECAPACITY; return; }
  const int m = r + aug;
  // poles (descending since S is descending) and weights
  double zn2 = 0.0;
  for (int i = 0; i < m; ++i) {
    const double zi = (i < r) ? w.pq[i] : q;
    zn2 += zi * zi;
  }
  const double u = 1.1102230246251565e-16;
  const double d1 = (r > 0) ? S[0] * S[0] : 0.0;
  const double scale = fmax(d1, zn2) > 0.0 ? fmax(d1, zn2) : 1.0;
  const double tol = 8.0 * u * scale;
  const double zn = sqrt(zn2);
  int mk = 0, nl = 0, nr = 0;
  // deflation of tiny weights, merge of (nearly) equal poles by a Givens rotation
  double pz = 0.0, pd = 0.0;
  int pidx = -1;
  for (int i = 0; i < m; ++i) {
    const double di = (i < r) ? S[i] * S[i] : 0.0;
    double zi = (i < r) ? w.pq[i] : q;
    if (fabs(zi) * zn <= tol) {   // deflate: eigenpair (di, e_i)
      w.lam[nl] = di;
      w.lsrc[nl] = -(i + 1);
      ++nl;
      continue;
    }
    if (pidx >= 0 && fabs(pd - di) <= tol) {
      // rotate (pz at pidx, zi at i) so that the weight of pole i vanishes
      const double h = hypot(pz, zi);
      const double c = pz / h, s = zi / h;
      w.rot[4 * nr + 0] = pidx; w.rot[4 * nr + 1] = i; w.rot[4 * nr + 2] = c; w.rot[4 * nr + 3] = s;
      ++nr;
      pz = h;
      w.z[mk - 1] = h;
      w.lam[nl] = di;
      w.lsrc[nl] = -(i + 1);
      ++nl;
      continue;
    }
    w.delta[mk] = di;
    w.z[mk] = zi;
    w.idx[mk] = i;
    pz = zi; pd = di; pidx = i;
    ++mk;
  }
  w.nrot[0] = nr;
  w.meta[0] = m;
  w.meta[1] = mk;
  w.meta[3] = nl;
}

// ---------------------------------------------------------------------------------------------
// e = d - V_pad p over the new rows (stored), ||e||^2 and s = V_pad^T e; partials (r + 1).
// ---------------------------------------------------------------------------------------------
template <typename TW>
__global__ void __launch_bounds__(256) k_isvd_e(Ctl* __restrict__ ctl, TW* const* dbufs,
                                               TW* const* vbufs, const double* __restrict__ p,
                                               TW* __restrict__ evec, double* __restrict__ part,
                                               double* __restrict__ es, const double* __restrict__ S,
                                               SecWork w) {
  if (ctl->status) return;
  if (rows_isvd_ok(ctl)) return;   // k_isvd_e_rows does this pass
  const int d = ctl->d, m = d - 1;
  const int r = ctl->r[d - 1];
  const int ldc = tk_cv_stride(r, ctl->ldc, (int)sizeof(TW));
  const TW* V = vbufs[ctl->cbuf];
  const TW* dv = dbufs[ctl->xbuf];
  long long Rn = 1;
  for (int i = 0; i < m; ++i) Rn *= ctl->r[i];
  const bool same = !spatial_grew(ctl);
  int ro[TK_MAXD], rn[TK_MAXD];
  for (int i = 0; i < TK_MAXD; ++i) { ro[i] = ctl->rold[i]; rn[i] = ctl->r[i]; }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int CPL = TK_STREAM_CAP_MAX / 32;
  const int CG = (r + 31) / 32;
  TW pl[CPL];
#pragma unroll
  for (int g = 0; g < CPL; ++g) {
    const int c = lane + 32 * g;
    pl[g] = (c < r) ? (TW)p[c] : TW(0);
  }
  double acc[CPL];
  TW accf[CPL];
#pragma unroll
  for (int g = 0; g < CPL; ++g) { acc[g] = 0.0; accf[g] = TW(0); }
  typename AccOf<TW>::type eacc;
  const long long gw = (long long)blockIdx.x * 8 + wid;
  const long long nw = (long long)gridDim.x * 8;
  int batches = 0;
  for (long long j0 = gw * RB; j0 < Rn; j0 += nw * RB) {
    long long jo[RB];
    TW dj[RB], dot[RB];
#pragma unroll
    for (int i = 0; i < RB; ++i) {
      const long long jn = j0 + i;
      jo[i] = (jn < Rn) ? (same ? jn : (long long)map_new_to_old32((int)jn, rn, ro, m)) : -1;
      dj[i] = (jn < Rn) ? dv[jn] : TW(0);
      dot[i] = TW(0);
    }
#pragma unroll
    for (int g = 0; g < CPL; ++g) {
      if (g >= CG) break;
      const int c = g * 32 + lane;
      TW v[RB];
#pragma unroll
      for (int i = 0; i < RB; ++i) v[i] = (jo[i] >= 0 && c < r) ? V[jo[i] * ldc + c] : TW(0);
#pragma unroll
      for (int i = 0; i < RB; ++i) dot[i] += v[i] * pl[g];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int i = 0; i < RB; ++i) dot[i] += __shfl_xor_sync(0xffffffffu, dot[i], o);
    TW e[RB];
#pragma unroll
    for (int i = 0; i < RB; ++i) {
      e[i] = dj[i] - dot[i];
      if (j0 + i >= Rn) e[i] = TW(0);
    }
    if (lane < RB) {
      TW mine = e[0];
#pragma unroll
      for (int i = 1; i < RB; ++i) if (lane == i) mine = e[i];
      if (j0 + lane < Rn) evec[j0 + lane] = mine;
    }
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < RB; ++i) eacc.add(e[i] * e[i]);
    }
#pragma unroll
    for (int g = 0; g < CPL; ++g) {
      if (g >= CG) break;
      const int c = g * 32 + lane;
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        const TW v = (jo[i] >= 0 && c < r) ? V[jo[i] * ldc + c] : TW(0);
        accf[g] += v * e[i];
      }
    }
    if (++batches == 4) {
#pragma unroll
      for (int g = 0; g < CPL; ++g) { acc[g] += (double)accf[g]; accf[g] = TW(0); }
      batches = 0;
    }
  }
  __shared__ double sh[8][TK_STREAM_CAP_MAX + 1];
#pragma unroll
  for (int g = 0; g < CPL; ++g) sh[wid][lane + 32 * g] = acc[g] + (double)accf[g];
  if (lane == 0) sh[wid][TK_STREAM_CAP_MAX] = eacc.value();
  __syncthreads();
  for (int c = threadIdx.x; c <= r; c += blockDim.x) {
    const int src = (c == r) ? TK_STREAM_CAP_MAX : c;
    double s = 0.0;
    for (int ww = 0; ww < 8; ++ww) s += sh[ww][src];
    part[(long long)blockIdx.x * (TK_STREAM_CAP_MAX + 2) + c] = s;
  }
  if (tk_last_block_reduce(part, TK_STREAM_CAP_MAX + 2, r + 1, es, &ctl->ticket[1]) &&
      threadIdx.x == 0)
    isvd_small_body(ctl, p, es, S, w);
}

// ---------------------------------------------------------------------------------------------
// Secular-equation SVD of S'. Problem: S'^T S' = diag(delta) + z z^T with delta = S^2 (and a
// trailing 0 when q > eps), z = [p'; q'] (or p'). Eigenvalues lambda = singular values^2 of S',
// eigenvectors = right singular vectors V''; U'' = S' V'' S~^-1.
// Roots by bisection refined with safeguarded Newton steps; eigenvectors by the Loewner-formula
// weights of Gu & Eisenstat (SIAM J. Matrix Anal. Appl. 15, 1994), which keep them orthogonal.
// ---------------------------------------------------------------------------------------------


__device__ double sec_f(const double* delta, const double* z, int mk, double dorg, double tau,
                        double* fp, int lane) {
  double f = 0.0, g = 0.0;
  for (int i = lane; i < mk; i += 32) {
    const double den = (delta[i] - dorg) - tau;
    const double t = z[i] / den;
    f += z[i] * t;
    g += t * t;
  }
  f = warp_sum(f);
  g = warp_sum(g);
  *fp = g;
  return 1.0 + f;
}

// FP32 form of sec_f on scaled, origin-shifted data: df[i] = (delta_i - delta_o) / scale,
// zf2[i] = z_i^2 / scale, t = tau / scale.
__device__ __forceinline__ float sec_f32(const float* df, const float* zf2, int mk, float t,
                                         float* fp, int lane) {
  float f = 0.f, g = 0.f;
  for (int i = lane; i < mk; i += 32) {
    const float den = df[i] - t;
    const float q = zf2[i] / den;
    f += q;
    g += q / den;
  }
  f = warp_sum(f);
  g = warp_sum(g);
  *fp = g;
  return 1.f + f;
}

constexpr int SEC_WARPS = 4;       // roots per block of k_secular_roots
constexpr int SEC_PAIR_MAX = 48;   // pair-parallel Loewner weights up to this many poles

// One warp per root of 1 + sum z_i^2 / (delta_i - lambda) = 0. The root is first located in FP32
// (bisection with Newton steps on the origin-shifted, scaled equation, about 24 bits), then
// polished in FP64 by safeguarded Newton steps inside a bracket checked in FP64: FP64 runs at a
// small fraction of the FP32 rate here, and from a 24-bit start Newton needs two or three steps.
__global__ void __launch_bounds__(32 * SEC_WARPS) k_secular_roots(const Ctl* ctl, SecWork w) {
  if (ctl->status) return;
  const int mk = w.meta[1];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int root = blockIdx.x * SEC_WARPS + wl;
  if (root >= mk) return;
  __shared__ float s_df[SEC_WARPS][TK_STREAM_CAP_MAX + 1];
  __shared__ float s_z2[SEC_WARPS][TK_STREAM_CAP_MAX + 1];
  double zn2 = 0.0;
  for (int i = lane; i < mk; i += 32) zn2 += w.z[i] * w.z[i];
  zn2 = warp_sum(zn2);
  double fp;
  // interval of lambda_root: (delta_root, delta_{root-1}) or (delta_0, delta_0 + ||z||^2]; the
  // origin is the nearer pole (sign of f at the midpoint)
  int o;
  double lo, hi;   // offsets relative to delta[o]
  if (root == 0) {
    o = 0; lo = 0.0; hi = zn2;
  } else {
    const double a = w.delta[root], b = w.delta[root - 1];
    const double mid = 0.5 * (b - a);
    const double fm = sec_f(w.delta, w.z, mk, a, mid, &fp, lane);
    if (fm >= 0.0) { o = root; lo = 0.0; hi = mid; }
    else { o = root - 1; lo = a - b + mid; hi = 0.0; }   // lo = -(b - a)/2 relative to b
  }
  const double dorg = w.delta[o];
  // ---- FP32 search ----
  const double scale = fmax(fmax(fabs(w.delta[0]), zn2), 1e-300);
  const double inv = 1.0 / scale;
  for (int i = lane; i < mk; i += 32) {
    s_df[wl][i] = (float)((w.delta[i] - dorg) * inv);
    s_z2[wl][i] = (float)(w.z[i] * w.z[i] * inv);
  }
  __syncwarp();
  float lf = (float)(lo * inv), hf = (float)(hi * inv);
  float t = 0.5f * (lf + hf);
  for (int it = 0; it < 80; ++it) {
    float gp;
    const float f = sec_f32(s_df[wl], s_z2[wl], mk, t, &gp, lane);
    if (f == 0.f) break;
    if (f > 0.f) hf = t; else lf = t;
    float tn = t - f / gp;
    if (!(tn > lf && tn < hf)) tn = 0.5f * (lf + hf);
    if (hf - lf <= 4.f * 5.9604645e-08f * fmaxf(fabsf(lf), fabsf(hf)) ||
        fabsf(tn - t) <= 2.f * 5.9604645e-08f * fabsf(t)) { t = tn; break; }
    t = tn;
  }
  // ---- FP64 polish ----
  double tau = (double)t * scale;
  if (!(tau > lo && tau < hi)) tau = 0.5 * (lo + hi);
  for (int it = 0; it < 100; ++it) {
    const double f = sec_f(w.delta, w.z, mk, dorg, tau, &fp, lane);
    if (f == 0.0) break;
    if (f > 0.0) hi = tau; else lo = tau;
    double tn = tau - f / fp;
    if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
    const double width = hi - lo;
    if (width <= 4.0 * 1.1102230246251565e-16 * fmax(fabs(lo), fabs(hi)) ||
        fabs(tn - tau) <= 2.0 * 1.1102230246251565e-16 * fabs(tau))
    { tau = tn; break; }
    tau = tn;
  }
  if (lane == 0) { w.tau[root] = tau; w.org[root] = o; }
}

// Eigenvalues merged and sorted, Loewner weights, eigenvectors V'' and U'' = S' V'' / sigma.
__global__ void __launch_bounds__(1024) k_secular_vectors(Ctl* ctl, const double* S, SecWork w,
                                                         double* Sout) {
  if (ctl->status) return;
  const int d = ctl->d;
  const int r = ctl->r[d - 1];
  const int aug = ctl->aug;
  const int m = w.meta[0], mk = w.meta[1], nl = w.meta[3];
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ double zhat[TK_STREAM_CAP_MAX + 1];
  __shared__ double lam_all[TK_STREAM_CAP_MAX + 1];
  __shared__ int src_all[TK_STREAM_CAP_MAX + 1];
  __shared__ int order[TK_STREAM_CAP_MAX + 1];
  __shared__ int s_keep;
  __shared__ double s_fac[SEC_PAIR_MAX][SEC_PAIR_MAX];
  // roots first (index k -> lambda = delta[org] + tau), then deflated
  for (int k = tid; k < mk; k += nt) {
    lam_all[k] = w.delta[w.org[k]] + w.tau[k];
    src_all[k] = k;
  }
  for (int k = tid; k < nl; k += nt) {
    lam_all[mk + k] = w.lam[k];
    src_all[mk + k] = w.lsrc[k];
  }
  __syncthreads();
  // Loewner weights of the non-deflated problem:
  // zhat_i^2 = (lambda_i - delta_i) prod_{j != i} (lambda_j - delta_i) / (delta_j - delta_i)
  if (mk <= SEC_PAIR_MAX) {
    // every factor in parallel (one FP64 division each), then one warp per product
    for (int L = tid; L < mk * mk; L += nt) {
      const int i = L / mk, j = L - i * mk;
      double f;
      if (j == i) f = (w.delta[w.org[i]] - w.delta[i]) + w.tau[i];
      else f = ((w.delta[w.org[j]] - w.delta[i]) + w.tau[j]) / (w.delta[j] - w.delta[i]);
      s_fac[i][j] = f;
    }
    __syncthreads();
    const int lane = tid & 31, nwarp = nt >> 5;
    for (int i = tid >> 5; i < mk; i += nwarp) {
      double prod = 1.0;
      for (int j = lane; j < mk; j += 32) prod *= s_fac[i][j];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) prod *= __shfl_xor_sync(0xffffffffu, prod, off);
      if (lane == 0) zhat[i] = copysign(sqrt(fabs(prod)), w.z[i]);
    }
  } else {
    for (int i = tid; i < mk; i += nt) {
      double prod = (w.delta[w.org[i]] - w.delta[i]) + w.tau[i];
      for (int j = 0; j < mk; ++j) {
        if (j == i) continue;
        const double num = (w.delta[w.org[j]] - w.delta[i]) + w.tau[j];
        prod *= num / (w.delta[j] - w.delta[i]);
      }
      zhat[i] = copysign(sqrt(fabs(prod)), w.z[i]);
    }
  }
  // descending order of all m eigenvalues (rank sort; ties by position)
  for (int a = tid; a < m; a += nt) {
    int rank = 0;
    const double la = lam_all[a];
    for (int b = 0; b < m; ++b) {
      const double lb = lam_all[b];
      if (lb > la || (lb == la && b < a)) ++rank;
    }
    order[rank] = a;
  }
  __syncthreads();
  if (tid == 0) {
    // numerical rank of the compact SVD: keep lambda > (r+1) u lambda_max, at most #columns
    const double lmax = m > 0 ? lam_all[order[0]] : 0.0;
    const double thr = (double)(r + 1) * 1.1102230246251565e-16 * lmax;
    int keep = 0;
    double drop = 0.0;
    for (int k = 0; k < m; ++k) {
      const double l = lam_all[order[k]];
      if (keep < m && l > thr && lmax > 0.0) ++keep; else drop += fmax(l, 0.0);
    }
    s_keep = keep;
    w.meta[2] = keep;
    ctl->rnew_d = keep;
    ctl->dropped = drop;
  }
  __syncthreads();
  const int keep = s_keep;
  // V'' columns: for kept sorted eigenvalue k
  for (long long L = tid; L < (long long)m * keep; L += nt) {
    const int k = (int)(L / m), i = (int)(L % m);   // column k, original row i
    w.V2[(long long)k * m + i] = 0.0;
  }
  __syncthreads();
  // eigenvector entries of the non-deflated columns, one division per (column, row) pair
  for (long long L = tid; L < (long long)keep * mk; L += nt) {
    const int k = (int)(L / mk), i = (int)(L % mk);
    const int src = src_all[order[k]];
    if (src < 0) continue;
    const double den = (w.delta[i] - w.delta[w.org[src]]) - w.tau[src];
    w.V2[(long long)k * m + w.idx[i]] = zhat[i] / den;
  }
  __syncthreads();
  // one warp per column: normalise (or the unit vector of a deflated pair), undo the Givens
  // merges (in reverse order), singular value
  {
    const int lane = tid & 31, nwarp = nt >> 5;
    for (int k = tid >> 5; k < keep; k += nwarp) {
      const int a = order[k];
      const int src = src_all[a];
      double* col = w.V2 + (long long)k * m;
      if (src >= 0) {
        double nrm = 0.0;
        for (int i = lane; i < mk; i += 32) {
          const double v = col[w.idx[i]];
          nrm += v * v;
        }
        nrm = sqrt(warp_sum(nrm));
        for (int i = lane; i < mk; i += 32) col[w.idx[i]] /= nrm;
      } else if (lane == 0) {
        col[-src - 1] = 1.0;
      }
      __syncwarp();
      if (lane == 0) {
        for (int t = w.nrot[0] - 1; t >= 0; --t) {
          const int i = (int)w.rot[4 * t + 0], j = (int)w.rot[4 * t + 1];
          const double c = w.rot[4 * t + 2], sn = w.rot[4 * t + 3];
          const double xi = col[i], xj = col[j];
          // merged weight lives on i: original (z_i, z_j) = h (c, s); x_orig = G^T x_rot
          col[i] = c * xi - sn * xj;
          col[j] = sn * xi + c * xj;
        }
        const double sig = sqrt(fmax(lam_all[a], 0.0));
        w.sv[k] = sig;
        Sout[k] = sig;
      }
    }
  }
  __syncthreads();
  // U'' = S' V'' / sigma: rows 0..r-1: S_i V''(i,k); row r: p'^T V''(0:r,k) + q' V''(r,k)
  for (long long L = tid; L < (long long)(r + 1) * keep; L += nt) {
    const int k = (int)(L / (r + 1)), i = (int)(L % (r + 1));
    const double* col = w.V2 + (long long)k * m;
    double val;
    if (i < r) {
      val = S[i] * col[i];
    } else {
      val = 0.0;
      for (int c = 0; c < r; ++c) val += w.pq[c] * col[c];
      if (aug) val += w.pq[r] * col[r];
    }
    const double sig = w.sv[k];
    w.U2[(long long)k * (r + 1) + i] = sig > 0.0 ? val / sig : 0.0;
  }
}

// ---------------------------------------------------------------------------------------------
// U~_d = [U_d U''(1:r,:); U''(r+1,:)] into the other buffer (row-major, ld = ldc).
// ---------------------------------------------------------------------------------------------
__global__ void k_ud_update(const Ctl* ctl, double* const* udbufs, SecWork w) {
  if (ctl->status) return;
  const int d = ctl->d;
  const int r = ctl->r[d - 1];
  const int nd = ctl->nd;
  const int ldc = ctl->ldc;
  const int keep = w.meta[2];
  const double* Ud = udbufs[ctl->ubuf];
  double* Un = udbufs[ctl->ubuf ^ 1];
  const long long total = (long long)(nd + 1) * keep;
  for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < total;
       L += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(L / keep), c = (int)(L % keep);
    const double* u2 = w.U2 + (long long)c * (r + 1);
    double s;
    if (t < nd) {
      s = 0.0;
      const double* row = Ud + (long long)t * ldc;
      for (int i = 0; i < r; ++i) s += row[i] * u2[i];
    } else {
      s = u2[r];
    }
    Un[(long long)t * ldc + c] = s;
  }
}

// M = U~_d(1:n_d,:)^T U_d (keep x r), plus the small matrices of the C and V updates:
//   Bc = M^T (r x keep), cu = U''(r+1,:) (keep)
//   Bv = V''(1:r,:) - s w^T (r x keep), wv = V''(r+1,:) / q' (keep)   [q > eps]
//   Bv = V''                                                         [q <= eps]
// bsplit (mixed form only): B^T of both updates split into TF32 hi/lo, row stride 512, zero padded
// to K = ceil32(r), N = ceil16(keep): [0] Mhi, [1] Mlo (= (M^T)^T), [2] Bv^T hi, [3] Bv^T lo.
template <typename TW>
__global__ void k_core_m(const Ctl* ctl, double* const* udbufs, SecWork w, const double* es,
                         TW* Bc, TW* cu, TW* Bv, TW* wv, int ldb, float* const* bsplit) {
  if (ctl->status) return;
  const int d = ctl->d;
  const int r = ctl->r[d - 1];
  const int nd = ctl->nd;
  const int ldc = ctl->ldc;
  const int keep = w.meta[2];
  const int m = w.meta[0];
  const int aug = ctl->aug;
  const double* Ud = udbufs[ctl->ubuf];
  const double* Un = udbufs[ctl->ubuf ^ 1];
  const long long total = (long long)keep * r;
  for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < total;
       L += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(L / r), b = (int)(L % r);   // M(a, b)
    double s = 0.0;
    for (int t = 0; t < nd; ++t) s += Un[(long long)t * ldc + a] * Ud[(long long)t * ldc + b];
    Bc[(long long)b * ldb + a] = (TW)s;              // Bc(b, a) = M(a, b), row-major r x keep
    const double* col = w.V2 + (long long)a * m;
    double bv = col[b];
    if (aug) bv -= es[b] * (col[r] / w.pq[r]);
    Bv[(long long)b * ldb + a] = (TW)bv;
    if (bsplit) {
      // B^T(n = a, k = b) split for the tensor-core update
      const float fs = (float)s, fb = (float)bv;
      const float hs = __uint_as_float((__float_as_uint(fs) + 0x1000u) & 0xFFFFE000u);
      const float hb = __uint_as_float((__float_as_uint(fb) + 0x1000u) & 0xFFFFE000u);
      const long long o = (long long)a * 512 + b;
      bsplit[0][o] = hs;
      bsplit[1][o] = fs - hs;
      bsplit[2][o] = hb;
      bsplit[3][o] = fb - hb;
    }
  }
  if (bsplit) {
    // zero the padding read by the tensor cores: k in [r, ceil32(r)) for n < ceil16(keep), and
    // rows n in [keep, ceil16(keep))
    const int kp = (r + 31) / 32 * 32, np = (keep + 15) / 16 * 16;
    const long long tot = (long long)np * kp;
    for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < tot;
         L += (long long)gridDim.x * blockDim.x) {
      const int n = (int)(L / kp), k = (int)(L % kp);
      if (n < keep && k < r) continue;
      const long long o = (long long)n * 512 + k;
      bsplit[0][o] = 0.f;
      bsplit[1][o] = 0.f;
      bsplit[2][o] = 0.f;
      bsplit[3][o] = 0.f;
    }
  }
  for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < keep;
       L += (long long)gridDim.x * blockDim.x) {
    const int a = (int)L;
    cu[a] = (TW)w.U2[(long long)a * (r + 1) + r];
    const double* col = w.V2 + (long long)a * m;
    wv[a] = aug ? (TW)(col[r] / w.pq[r]) : TW(0);
  }
}

// ---------------------------------------------------------------------------------------------
// Out[j, :] = In_pad[j, 0:r] B + x[j] c  for every new row j (SIMT tiled GEMM).
// In rows come from the old layout through the new->old row map (zero rows for padding).
// ---------------------------------------------------------------------------------------------
constexpr int CV_TM = 64, CV_TN = 64, CV_TK = 32;

template <typename TW>
__global__ void __launch_bounds__(256) k_cv_update(const Ctl* __restrict__ ctl, TW* const* ibufs,
                                                  TW* const* obufs, const TW* __restrict__ Bm,
                                                  int ldb, const TW* __restrict__ cvec,
                                                  const TW* __restrict__ xvec, TW* const* xbufs,
                                                  const SecWork w) {
  if (ctl->status) return;
  if (tc_cv_ok(ctl, w.meta[2])) return;   // the tensor-core kernel does this update
  if (rows_cv_ok(ctl, w.meta[2])) return;  // k_cv_rows does this update
  const int d = ctl->d, mm = d - 1;
  const int r = ctl->r[d - 1];
  const int keep = w.meta[2];
  const int ldi = tk_cv_stride(r, ctl->ldc, (int)sizeof(TW));      // rows read (rank r)
  const int ldo = tk_cv_stride(keep, ctl->ldc, (int)sizeof(TW));   // rows written (rank keep)
  long long Rn = 1;
  for (int i = 0; i < mm; ++i) Rn *= ctl->r[i];
  const TW* In = ibufs[ctl->cbuf];
  TW* Out = obufs[ctl->cbuf ^ 1];
  const TW* X = xvec ? xvec : xbufs[ctl->xbuf];
  __shared__ TW As[CV_TK][CV_TM + 1];
  __shared__ TW Bs[CV_TK][CV_TN];
  __shared__ long long rowsrc[CV_TM];
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  const long long ntm = (Rn + CV_TM - 1) / CV_TM;
  const int ntn = (keep + CV_TN - 1) / CV_TN;
  for (long long tile = blockIdx.x; tile < ntm * ntn; tile += gridDim.x) {
    const long long tm = tile / ntn;
    const int tn = (int)(tile % ntn);
    const long long j0 = tm * CV_TM;
    const int n0 = tn * CV_TN;
    __syncthreads();
    if (tid < CV_TM) {
      const long long j = j0 + tid;
      rowsrc[tid] = (j < Rn) ? tk_map_new_to_old(j, ctl->r, ctl->rold, mm) : -1;
    }
    TW acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = TW(0);
    for (int k0 = 0; k0 < r; k0 += CV_TK) {
      __syncthreads();
      for (int L = tid; L < CV_TM * CV_TK; L += 256) {
        const int row = L / CV_TK, kk = L % CV_TK;
        const long long src = rowsrc[row];
        As[kk][row] = (src >= 0 && k0 + kk < r) ? In[src * ldi + k0 + kk] : TW(0);
      }
      for (int L = tid; L < CV_TK * CV_TN; L += 256) {
        const int kk = L / CV_TN, cc = L % CV_TN;
        Bs[kk][cc] = (k0 + kk < r && n0 + cc < keep) ? Bm[(long long)(k0 + kk) * ldb + n0 + cc] : TW(0);
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < CV_TK; ++kk) {
        TW a[4], b[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) { a[q] = As[kk][ty + 16 * q]; b[q] = Bs[kk][tx + 16 * q]; }
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[p][q] += a[p] * b[q];
      }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const long long j = j0 + ty + 16 * p;
      if (j >= Rn) continue;
      const TW xj = X[j];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = n0 + tx + 16 * q;
        if (c < keep) Out[j * ldo + c] = acc[p][q] + xj * cvec[c];
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Row passes with one row per lane (r_d <= 32). Each lane owns rows jn = g, g + G, ... of the new
// spatial layout, maps each to its old row (zero padding has none), reads that row's r_d
// coefficients as 16-byte pieces (the row start is aligned when the stride is a multiple of 4 floats /
// 2 doubles) and keeps them in registers. Nothing is recomputed across lanes, so the index map
// costs one mixed-radix decomposition per row. FP32 partial sums cover at most ROWS_FLUSH rows
// before they are added into FP64 shared-memory slots.
// ---------------------------------------------------------------------------------------------
constexpr int ROWS_NT = 256;
constexpr int ROWS_FLUSH = 32;

template <typename TW>
__device__ __forceinline__ void load_row(const TW* __restrict__ row, int r, bool vec, TW (&v)[ROWS_RMAX]) {
  if (sizeof(TW) == 4 && vec) {
    const float4* r4 = reinterpret_cast<const float4*>(row);
#pragma unroll
    for (int q = 0; q < ROWS_RMAX / 4; ++q) {
      if (4 * q < r) {
        const float4 t = __ldg(r4 + q);
        v[4 * q] = (TW)t.x; v[4 * q + 1] = (TW)t.y; v[4 * q + 2] = (TW)t.z; v[4 * q + 3] = (TW)t.w;
      } else {
        v[4 * q] = v[4 * q + 1] = v[4 * q + 2] = v[4 * q + 3] = TW(0);
      }
    }
  } else if (sizeof(TW) == 8 && vec) {
    const double2* r2 = reinterpret_cast<const double2*>(row);
#pragma unroll
    for (int q = 0; q < ROWS_RMAX / 2; ++q) {
      if (2 * q < r) {
        const double2 t = __ldg(r2 + q);
        v[2 * q] = (TW)t.x; v[2 * q + 1] = (TW)t.y;
      } else {
        v[2 * q] = v[2 * q + 1] = TW(0);
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < ROWS_RMAX; ++c) v[c] = (c < r) ? row[c] : TW(0);
  }
  // columns r.. of the last piece are not part of the state (possibly never written)
#pragma unroll
  for (int c = 0; c < ROWS_RMAX; ++c) v[c] = (c < r) ? v[c] : TW(0);
}

// Adds the warp's partial sums acc[c] (live columns c < r) into the FP64 slots sw[c] (lane 0).
// The sum across lanes runs in the work type (FP32 in the mixed form: the FP64 pipe is a small
// fraction of the FP32 rate, and a 32-term FP32 sum of 32-row FP32 partials keeps the 1e-7
// relative accuracy of the products); only the per-warp totals are added in FP64.
template <typename TW>
__device__ __forceinline__ void rows_flush(TW (&acc)[ROWS_RMAX], double* sw, int lane, int r) {
#pragma unroll
  for (int c = 0; c < ROWS_RMAX; ++c) {
    if (c < r) {
      const TW t = warp_sum(acc[c]);
      if (lane == 0) sw[c] += (double)t;
    }
    acc[c] = TW(0);
  }
}

// part[blockIdx.x * stride + c] = sum over the block's warps of sw[w][c], c < ncol.
__device__ __forceinline__ void rows_block_sum(double (*sw)[ROWS_RMAX + 1], int ncol,
                                               double* __restrict__ part, long long stride) {
  __syncthreads();
  for (int c = threadIdx.x; c < ncol; c += ROWS_NT) {
    double s = 0.0;
    for (int w = 0; w < ROWS_NT / 32; ++w) s += sw[w][c];
    part[(long long)blockIdx.x * stride + c] = s;
  }
}

// p = V_pad^T d: partials per block in the layout of k_isvd_p. Warps walk 32 consecutive new
// rows at a time (a warp-uniform loop, so the periodic FP64 flush is a warp reduction).
template <typename TW>
__global__ void __launch_bounds__(ROWS_NT) k_isvd_p_rows(Ctl* __restrict__ ctl,
                                                        TW* const* dbufs, TW* const* vbufs,
                                                        double* __restrict__ part,
                                                        double* __restrict__ pout) {
  if (ctl->status) return;
  if (!rows_isvd_ok(ctl)) return;
  const int d = ctl->d, m = d - 1;
  const int r = ctl->r[d - 1];
  const int ldc = tk_cv_stride(r, ctl->ldc, (int)sizeof(TW));
  const bool vec = (ldc % (16 / (int)sizeof(TW))) == 0;
  const TW* V = vbufs[ctl->cbuf];
  const TW* dv = dbufs[ctl->xbuf];
  int ro[TK_MAXD], rn[TK_MAXD];
  long long Rn = 1;
#pragma unroll
  for (int i = 0; i < TK_MAXD; ++i) {
    ro[i] = (i < m) ? ctl->rold[i] : 1;
    rn[i] = (i < m) ? ctl->r[i] : 1;
    Rn *= rn[i];
  }
  const bool same = !spatial_grew(ctl);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __shared__ double sw[ROWS_NT / 32][ROWS_RMAX + 1];
  for (int c = lane; c <= ROWS_RMAX; c += 32) sw[wid][c] = 0.0;
  TW acc[ROWS_RMAX];
#pragma unroll
  for (int c = 0; c < ROWS_RMAX; ++c) acc[c] = TW(0);
  int it = 0;
  const long long G = (long long)gridDim.x * ROWS_NT;
  for (long long jb = (long long)blockIdx.x * ROWS_NT + wid * 32; jb < Rn; jb += G) {
    const long long jn = jb + lane;
    const int jo = (jn >= Rn) ? -1 : (same ? (int)jn : map_new_to_old_reg((int)jn, rn, ro, m));
    if (jo >= 0) {
      const TW dj = dv[jn];
      TW v[ROWS_RMAX];
      load_row<TW>(V + (long long)jo * ldc, r, vec, v);
#pragma unroll
      for (int c = 0; c < ROWS_RMAX; ++c) acc[c] += v[c] * dj;
    }
    if (++it == ROWS_FLUSH) { rows_flush<TW>(acc, sw[wid], lane, r); it = 0; }
  }
  rows_flush<TW>(acc, sw[wid], lane, r);
  rows_block_sum(sw, r, part, TK_STREAM_CAP_MAX);
  tk_last_block_reduce(part, TK_STREAM_CAP_MAX, r, pout, &ctl->ticket[0]);
}

// e = d - V_pad p (stored), ||e||^2 and s = V_pad^T e: partials in the layout of k_isvd_e
// (s in columns 0..r-1, ||e||^2 in column r).
template <typename TW>
__global__ void __launch_bounds__(ROWS_NT) k_isvd_e_rows(Ctl* __restrict__ ctl,
                                                        TW* const* dbufs, TW* const* vbufs,
                                                        const double* __restrict__ p,
                                                        TW* __restrict__ evec,
                                                        double* __restrict__ part,
                                                        double* __restrict__ es,
                                                        const double* __restrict__ S,
                                                        SecWork w) {
  if (ctl->status) return;
  if (!rows_isvd_ok(ctl)) return;
  const int d = ctl->d, m = d - 1;
  const int r = ctl->r[d - 1];
  const int ldc = tk_cv_stride(r, ctl->ldc, (int)sizeof(TW));
  const bool vec = (ldc % (16 / (int)sizeof(TW))) == 0;
  const TW* V = vbufs[ctl->cbuf];
  const TW* dv = dbufs[ctl->xbuf];
  int ro[TK_MAXD], rn[TK_MAXD];
  long long Rn = 1;
#pragma unroll
  for (int i = 0; i < TK_MAXD; ++i) {
    ro[i] = (i < m) ? ctl->rold[i] : 1;
    rn[i] = (i < m) ? ctl->r[i] : 1;
    Rn *= rn[i];
  }
  const bool same = !spatial_grew(ctl);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __shared__ double sw[ROWS_NT / 32][ROWS_RMAX + 1];
  __shared__ TW pl[ROWS_RMAX];
  for (int c = lane; c <= ROWS_RMAX; c += 32) sw[wid][c] = 0.0;
  if (threadIdx.x < ROWS_RMAX) pl[threadIdx.x] = (threadIdx.x < r) ? (TW)p[threadIdx.x] : TW(0);
  __syncthreads();
  TW acc[ROWS_RMAX];
#pragma unroll
  for (int c = 0; c < ROWS_RMAX; ++c) acc[c] = TW(0);
  typename AccOf<TW>::type eacc;
  int it = 0;
  const long long G = (long long)gridDim.x * ROWS_NT;
  for (long long jb = (long long)blockIdx.x * ROWS_NT + wid * 32; jb < Rn; jb += G) {
    const long long jn = jb + lane;
    if (jn < Rn) {
      const int jo = same ? (int)jn : map_new_to_old_reg((int)jn, rn, ro, m);
      const TW dj = dv[jn];
      TW e = dj;
      if (jo >= 0) {
        TW v[ROWS_RMAX];
        load_row<TW>(V + (long long)jo * ldc, r, vec, v);
        TW dot = TW(0);
#pragma unroll
        for (int c = 0; c < ROWS_RMAX; ++c) dot += v[c] * pl[c];
        e = dj - dot;
#pragma unroll
        for (int c = 0; c < ROWS_RMAX; ++c) acc[c] += v[c] * e;
      }
      evec[jn] = e;
      eacc.add(e * e);
    }
    if (++it == ROWS_FLUSH) { rows_flush<TW>(acc, sw[wid], lane, r); it = 0; }
  }
  rows_flush<TW>(acc, sw[wid], lane, r);
  const double e2 = warp_sum(eacc.value());
  if (lane == 0) sw[wid][ROWS_RMAX] = e2;
  __syncthreads();
  // ||e||^2 moves to column r (columns r.. of the slots hold zeros)
  if (threadIdx.x < ROWS_NT / 32 && r < ROWS_RMAX) {
    sw[threadIdx.x][r] = sw[threadIdx.x][ROWS_RMAX];
  }
  rows_block_sum(sw, r + 1, part, TK_STREAM_CAP_MAX + 2);
  if (tk_last_block_reduce(part, TK_STREAM_CAP_MAX + 2, r + 1, es, &ctl->ticket[1]) &&
      threadIdx.x == 0)
    isvd_small_body(ctl, p, es, S, w);
}

// C~ = C_pad B_c + d c_c^T (blockIdx.y = 0) and V~ = V_pad B_v + e w_v^T (blockIdx.y = 1), one
// new row per lane, into the other buffer. B is r x keep row-major (ld ldb), staged in shared
// memory and read as 4-wide broadcasts.
template <typename TW>
__global__ void __launch_bounds__(ROWS_NT) k_cv_rows(const Ctl* __restrict__ ctl,
                                                    TW* const* cbufs, TW* const* vbufs,
                                                    const TW* __restrict__ Bc,
                                                    const TW* __restrict__ Bv, int ldb,
                                                    const TW* __restrict__ cu,
                                                    const TW* __restrict__ wv,
                                                    const TW* __restrict__ evec,
                                                    TW* const* dbufs, const SecWork w) {
  if (ctl->status) return;
  const int keep = w.meta[2];
  if (!rows_cv_ok(ctl, keep)) return;
  const int d = ctl->d, m = d - 1;
  const int r = ctl->r[d - 1];
  const int ldi = tk_cv_stride(r, ctl->ldc, (int)sizeof(TW));      // rows read (rank r)
  const int ldo = tk_cv_stride(keep, ctl->ldc, (int)sizeof(TW));   // rows written (rank keep)
  const bool vec = (ldi % (16 / (int)sizeof(TW))) == 0 && (ldo % (16 / (int)sizeof(TW))) == 0;
  const bool isV = blockIdx.y == 1;
  const TW* In = (isV ? vbufs : cbufs)[ctl->cbuf];
  TW* Out = (isV ? vbufs : cbufs)[ctl->cbuf ^ 1];
  const TW* B = isV ? Bv : Bc;
  const TW* cvec = isV ? wv : cu;
  const TW* X = isV ? evec : dbufs[ctl->xbuf];
  __shared__ __align__(16) TW Bs[ROWS_RMAX][ROWS_RMAX];
  __shared__ __align__(16) TW cs[ROWS_RMAX];
  for (int L = threadIdx.x; L < ROWS_RMAX * ROWS_RMAX; L += ROWS_NT) {
    const int k = L / ROWS_RMAX, c = L % ROWS_RMAX;
    Bs[k][c] = (k < r && c < keep) ? B[(long long)k * ldb + c] : TW(0);
  }
  if (threadIdx.x < ROWS_RMAX) cs[threadIdx.x] = (threadIdx.x < keep) ? cvec[threadIdx.x] : TW(0);
  int ro[TK_MAXD], rn[TK_MAXD];
  long long Rn = 1;
#pragma unroll
  for (int i = 0; i < TK_MAXD; ++i) {
    ro[i] = (i < m) ? ctl->rold[i] : 1;
    rn[i] = (i < m) ? ctl->r[i] : 1;
    Rn *= rn[i];
  }
  const bool same = !spatial_grew(ctl);
  __syncthreads();
  const long long G = (long long)gridDim.x * ROWS_NT;
  for (long long jn = (long long)blockIdx.x * ROWS_NT + threadIdx.x; jn < Rn; jn += G) {
    const int jo = same ? (int)jn : map_new_to_old_reg((int)jn, rn, ro, m);
    TW v[ROWS_RMAX];
    if (jo >= 0) load_row<TW>(In + (long long)jo * ldi, r, vec, v);
    else {
#pragma unroll
      for (int c = 0; c < ROWS_RMAX; ++c) v[c] = TW(0);
    }
    const TW xj = X[jn];
    TW* orow = Out + jn * ldo;
#pragma unroll
    for (int c4 = 0; c4 < ROWS_RMAX / 4; ++c4) {
      if (4 * c4 >= keep) break;
      TW o[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) o[t] = xj * cs[4 * c4 + t];
#pragma unroll
      for (int k = 0; k < ROWS_RMAX; ++k) {
        if (k >= r) break;
#pragma unroll
        for (int t = 0; t < 4; ++t) o[t] += v[k] * Bs[k][4 * c4 + t];
      }
      if (vec && sizeof(TW) == 4) {
        // columns keep.. of the last piece are zero (B and c are zero-padded); ldo % 4 == 0
        // keeps the piece inside the row
        *reinterpret_cast<float4*>(orow + 4 * c4) = make_float4((float)o[0], (float)o[1], (float)o[2], (float)o[3]);
      } else {
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (4 * c4 + t < keep) orow[4 * c4 + t] = o[t];
      }
    }
  }
}

// End of the update: S <- S~, ranks, n_d, buffers, error bookkeeping (Prop. 1, Prop. 2).
__global__ void k_end_update(Ctl* ctl, const double* Snew, double* S) {
  if (ctl->status) return;
  const int d = ctl->d;
  const int keep = ctl->rnew_d;
  for (int i = threadIdx.x; i < keep; i += blockDim.x) S[i] = Snew[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    // algorithmic bytes of this update (each operand read or written once per pass)
    const double tw = ctl->tw, tx = ctl->tx;
    const int r = ctl->r[d - 1];
    double Ro = 1.0, Rn = 1.0;
    for (int k = 0; k < d - 1; ++k) { Ro *= ctl->rold[k]; Rn *= ctl->r[k]; }
    double A = 1.0;
    for (int k = 0; k < d - 1; ++k) {
      double B = 1.0;
      for (int i = k + 1; i < d - 1; ++i) B *= ctl->n[i];
      const double in_el = A * ctl->n[k] * B;
      const double in_b = (k == 0 ? tx : tw) * in_el;
      const double p_b = tw * A * ctl->rold[k] * B;
      ctl->acc_bytes[k == 0 ? TK_PH_PROJ1 : TK_PH_PROJN] += in_b + p_b;
      if (ctl->grew[k]) ctl->acc_bytes[TK_PH_GROW] += 2.0 * in_b + p_b + tw * A * ctl->r[k] * B;
      A *= ctl->r[k];
    }
    ctl->acc_bytes[TK_PH_ISVD] += tw * (2.0 * Ro * r + 3.0 * Rn);
    ctl->acc_bytes[TK_PH_FACT] += 8.0 * 2.0 * ((double)ctl->nd * r + (double)(ctl->nd + 1) * keep);
    ctl->acc_bytes[TK_PH_CV] += tw * (2.0 * Ro * r + 2.0 * Rn * keep + 2.0 * Rn);
    double disc = 0.0;
    for (int k = 0; k < d - 1; ++k) disc += ctl->disc[k];
    disc += ctl->aug ? 0.0 : ctl->q2;
    disc += ctl->dropped;
    ctl->err2 += disc;
    ctl->data2 += ctl->y2;
    // the tensor-core path after spatial growth expands into the other buffer and writes back
    // into this one; every other path writes the other buffer
    const bool stay = tc_cv_ok(ctl, keep) && spatial_grew(ctl);
    ctl->r[d - 1] = keep;
    ctl->nd += 1;
    if (!stay) ctl->cbuf ^= 1;
    ctl->ubuf ^= 1;
    ctl->nupdates += 1;
  }
}

__global__ void k_begin_update(Ctl* ctl) {
  if (ctl->status) return;
  for (int k = 0; k < TK_MAXD; ++k) {
    ctl->rold[k] = ctl->r[k];
    ctl->grew[k] = 0;
    ctl->radd[k] = 0;
    ctl->e2[k] = 0.0;
    ctl->disc[k] = 0.0;
  }
  ctl->xbuf = -1;
  ctl->aug = 0;
  ctl->q = 0.0;
  ctl->q2 = 0.0;
  ctl->dropped = 0.0;
  if (ctl->nd + 1 > ctl->steps_cap) ctl->status = TK_ECAPACITY;
}

// ---------------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------------
template <typename TW>
cudaError_t launch_isvd(Ctl* ctl, void* const* dbufs, void* const* vbufs, double* part_p,
                        double* part_e, double* p, double* es, void* evec, const double* S,
                        SecWork w, int grid, cudaStream_t st) {
  // p = V^T d, then e = d - V p with [s; ||e||^2] and the small ISVD bookkeeping; each pass
  // finishes its cross-block sum in its last block
  k_isvd_p_rows<TW><<<grid, ROWS_NT, 0, st>>>(ctl, (TW* const*)dbufs, (TW* const*)vbufs, part_p, p);
  k_isvd_p<TW><<<grid, 256, 0, st>>>(ctl, (TW* const*)dbufs, (TW* const*)vbufs, part_p, p);
  k_isvd_e_rows<TW><<<grid, ROWS_NT, 0, st>>>(ctl, (TW* const*)dbufs, (TW* const*)vbufs, p,
                                               (TW*)evec, part_e, es, S, w);
  k_isvd_e<TW><<<grid, 256, 0, st>>>(ctl, (TW* const*)dbufs, (TW* const*)vbufs, p, (TW*)evec,
                                     part_e, es, S, w);
  k_secular_roots<<<(TK_STREAM_CAP_MAX + 1 + SEC_WARPS - 1) / SEC_WARPS, 32 * SEC_WARPS, 0, st>>>(ctl, w);
  return cudaGetLastError();
}

cudaError_t launch_secular_vectors(Ctl* ctl, const double* S, SecWork w, double* Snew,
                                   cudaStream_t st) {
  k_secular_vectors<<<1, 1024, 0, st>>>(ctl, S, w, Snew);
  return cudaGetLastError();
}

template <typename TW>
cudaError_t launch_factor(Ctl* ctl, double* const* udbufs, SecWork w, const double* es, void* Bc,
                          void* cu, void* Bv, void* wv, int ldb, float* const* bsplit,
                          int grid_small, cudaStream_t st) {
  k_ud_update<<<grid_small, 256, 0, st>>>(ctl, udbufs, w);
  k_core_m<TW><<<grid_small, 256, 0, st>>>(ctl, udbufs, w, es, (TW*)Bc, (TW*)cu, (TW*)Bv, (TW*)wv,
                                           ldb, bsplit);
  return cudaGetLastError();
}

template <typename TW>
cudaError_t launch_cv(Ctl* ctl, void* const* dbufs, void* const* cbufs, void* const* vbufs,
                      SecWork w, const void* Bc, const void* cu, const void* Bv, const void* wv,
                      int ldb, const void* evec, int grid_cv, cudaStream_t st) {
  k_cv_rows<TW><<<dim3(grid_cv, 2), ROWS_NT, 0, st>>>(ctl, (TW* const*)cbufs, (TW* const*)vbufs,
                                                      (const TW*)Bc, (const TW*)Bv, ldb,
                                                      (const TW*)cu, (const TW*)wv,
                                                      (const TW*)evec, (TW* const*)dbufs, w);
  k_cv_update<TW><<<grid_cv, 256, 0, st>>>(ctl, (TW* const*)cbufs, (TW* const*)cbufs,
                                           (const TW*)Bc, ldb, (const TW*)cu, nullptr,
                                           (TW* const*)dbufs, w);
  k_cv_update<TW><<<grid_cv, 256, 0, st>>>(ctl, (TW* const*)vbufs, (TW* const*)vbufs,
                                           (const TW*)Bv, ldb, (const TW*)wv, (const TW*)evec,
                                           (TW* const*)dbufs, w);
  return cudaGetLastError();
}

cudaError_t launch_begin(Ctl* ctl, cudaStream_t st) {
  k_begin_update<<<1, 1, 0, st>>>(ctl);
  return cudaGetLastError();
}

cudaError_t launch_end(Ctl* ctl, const double* Snew, double* S, cudaStream_t st) {
  k_end_update<<<1, 256, 0, st>>>(ctl, Snew, S);
  return cudaGetLastError();
}

template cudaError_t launch_isvd<float>(Ctl*, void* const*, void* const*, double*, double*, double*,
                                        double*, void*, const double*, SecWork, int, cudaStream_t);
template cudaError_t launch_isvd<double>(Ctl*, void* const*, void* const*, double*, double*,
                                         double*, double*, void*, const double*, SecWork, int,
                                         cudaStream_t);
template cudaError_t launch_factor<float>(Ctl*, double* const*, SecWork, const double*, void*,
                                          void*, void*, void*, int, float* const*, int,
                                          cudaStream_t);
template cudaError_t launch_factor<double>(Ctl*, double* const*, SecWork, const double*, void*,
                                           void*, void*, void*, int, float* const*, int,
                                           cudaStream_t);
template cudaError_t launch_cv<float>(Ctl*, void* const*, void* const*, void* const*, SecWork,
                                      const void*, const void*, const void*, const void*, int,
                                      const void*, int, cudaStream_t);
template cudaError_t launch_cv<double>(Ctl*, void* const*, void* const*, void* const*, SecWork,
                                       const void*, const void*, const void*, const void*, int,
                                       const void*, int, cudaStream_t);

}  // namespace tk
