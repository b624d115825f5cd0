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
#include "tc_common.cuh"

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
  if (rows_isvd_ok(ctl)) return;   // k_isvd_p_all does this pass (bulk tiles or a lane per row)
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
// The part of the small ISVD step after its sums: the q <= eps decision of Alg. 3, the poles
// S_i^2 and weights z = [p'; q] of S'^T S' = diag(S^2[, 0]) + z z^T, deflation of tiny weights
// and merges of (nearly) equal poles (one thread). pq = [p'; q] (may be shared memory); zr2 =
// sum_{i<r} pq_i^2; Rn the new spatial core size; eps and capd ctl->eps and ctl->cap[d - 1].
__device__ void isvd_small_tail(Ctl* ctl, const double* S, const SecWork& w, const double* pq,
                                int r, double q2, double q, double zr2, long long Rn, double eps,
                                int capd) {
  ctl->q2 = q2;
  ctl->q = q;
  int aug = q > eps ? 1 : 0;   // Alg. 3: ignore e if q <= eps
  // decision replay (test hook): the branch forced for this update (never a new direction
  // from e = 0)
  const int fa = rp_aug_of(ctl);
  if (fa >= 0) aug = (fa > 0 && q > 0.0) ? 1 : 0;
  ctl->aug = aug;
  if (aug && r + 1 > capd) { ctl->status = TK_ECAPACITY; return; }
  if (Rn > ctl->core_cap) { ctl->status = TK_ECAPACITY; return; }
  const int m = r + aug;
  // poles (descending since S is descending) and weights
  const double zn2 = zr2 + (aug ? q * q : 0.0);
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
    double zi = (i < r) ? pq[i] : q;
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

// The small ISVD step on one thread (the SIMT passes, streaming rank above ROWS_RMAX):
// CGS-corrected projection p' = p + s, q'^2 = ||e||^2 - ||s||^2, then isvd_small_tail.
__device__ void isvd_small_body(Ctl* ctl, const double* p, const double* es, const double* S,
                                const SecWork& w, int r, long long Rn, double eps, int capd) {
  double s2 = 0.0;
  for (int c = 0; c < r; ++c) s2 += es[c] * es[c];
  double q2 = es[r] - s2;
  if (q2 < 0.0) q2 = 0.0;
  const double q = sqrt(q2);
  double zr2 = 0.0;
  for (int c = 0; c < r; ++c) {
    const double v = p[c] + es[c];
    w.pq[c] = v;
    zr2 += v * v;
  }
  w.pq[r] = q;
  isvd_small_tail(ctl, S, w, w.pq, r, q2, q, zr2, Rn, eps, capd);
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
  if (rows_isvd_ok(ctl)) return;   // k_isvd_e_all does this pass (bulk tiles or a lane per row)
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
      threadIdx.x == 0) {
    long long Rn = 1;
    for (int i = 0; i < d - 1; ++i) Rn *= ctl->r[i];
    isvd_small_body(ctl, p, es, S, w, r, Rn, ctl->eps, ctl->cap[d - 1]);
  }
}

// ---------------------------------------------------------------------------------------------
// Secular-equation SVD of S'. Problem: S'^T S' = diag(delta) + z z^T with delta = S^2 (and a
// trailing 0 when q > eps), z = [p'; q'] (or p'). Eigenvalues lambda = singular values^2 of S',
// eigenvectors = right singular vectors V''; U'' = S' V'' S~^-1.
// Roots by bisection refined with safeguarded Newton steps; eigenvectors by the Loewner-formula
// weights of Gu & Eisenstat (SIAM J. Matrix Anal. Appl. 15, 1994), which keep them orthogonal.
// ---------------------------------------------------------------------------------------------


// 1/x in FP64 from the FP32 reciprocal refined by two Newton steps r <- r + r (1 - x r) (each
// doubles the correct bits: ~2^-24 -> 2^-48 -> below FP64 rounding); about half the latency of an
// FP64 division on this GPU. Outside the normal FP32 range it divides.
__device__ __forceinline__ double drcp(double x) {
  const float xf = (float)x;
  const float ax = fabsf(xf);
  if (!(ax > 1e-36f && ax < 1e36f)) return 1.0 / x;
  double r = (double)__frcp_rn(xf);
  r = fma(r, fma(-x, r, 1.0), r);
  r = fma(r, fma(-x, r, 1.0), r);
  return r;
}

__device__ double sec_f(const double* delta, const double* z, int mk, double dorg, double tau,
                        double* fp, int lane) {
  double f = 0.0, g = 0.0;
  for (int i = lane; i < mk; i += 32) {
    const double den = (delta[i] - dorg) - tau;
    const double t = z[i] * drcp(den);
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
    // fast reciprocal: the FP32 search only seeds the FP64 polish (scaled data, |den| <= ~1)
    const float rd = __fdividef(1.f, df[i] - t);
    const float q = zf2[i] * rd;
    f += q;
    g += q * rd;
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
    float tn = t - __fdividef(f, gp);
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
    double tn = tau - f * drcp(fp);
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
  {
    // numerical rank of the compact SVD: keep lambda > (r+1) u lambda_max (a count over the
    // sorted eigenvalues, which are descending, so the kept ones come first), the rest dropped;
    // count and dropped energy by block reductions in a fixed order (FP64 is long-latency: no
    // serial loop on one thread)
    const double lmax = m > 0 ? lam_all[order[0]] : 0.0;
    const double thr = (double)(r + 1) * 1.1102230246251565e-16 * lmax;
    double drop = 0.0;
    int kept = 0;
    if (tid < m) {
      const double l = lam_all[order[tid]];
      if (l > thr && lmax > 0.0) kept = 1; else drop = fmax(l, 0.0);
    }
    const int keep = __syncthreads_count(kept);
    __shared__ double s_drop[32];
    const int lane = tid & 31, wid = tid >> 5;
    drop = warp_sum(drop);
    if (lane == 0) s_drop[wid] = drop;
    __syncthreads();
    if (tid == 0) {
      double dsum = 0.0;
      for (int i = 0; i < (nt >> 5); ++i) dsum += s_drop[i];
      s_keep = keep;
      w.meta[2] = keep;
      ctl->rnew_d = keep;
      ctl->dropped = dsum;
    }
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
        const double inv = drcp(sqrt(warp_sum(nrm)));
        for (int i = lane; i < mk; i += 32) col[w.idx[i]] *= inv;
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
  // U'' = S' V'' / sigma: rows 0..r-1: S_i V''(i,k); row r: p'^T V''(0:r,k) + q' V''(r,k) (one
  // warp per column k, lanes over the r terms)
  for (long long L = tid; L < (long long)r * keep; L += nt) {
    const int k = (int)(L / r), i = (int)(L % r);
    const double* col = w.V2 + (long long)k * m;
    const double sig = w.sv[k];
    w.U2[(long long)k * (r + 1) + i] = sig > 0.0 ? S[i] * col[i] * drcp(sig) : 0.0;
  }
  {
    const int lane = tid & 31, nwarp = nt >> 5;
    for (int k = tid >> 5; k < keep; k += nwarp) {
      const double* col = w.V2 + (long long)k * m;
      double val = 0.0;
      for (int c = lane; c < r; c += 32) val += w.pq[c] * col[c];
      val = warp_sum(val);
      if (lane == 0) {
        if (aug) val += w.pq[r] * col[r];
        const double sig = w.sv[k];
        w.U2[(long long)k * (r + 1) + r] = sig > 0.0 ? val * drcp(sig) : 0.0;
      }
    }
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
  const long long nthr = (long long)gridDim.x * blockDim.x;
  if (total * 32 <= nthr) {
    // few entries (short streams): one warp per entry, lanes over the r terms (see k_core_m)
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    for (long long L = gw; L < total; L += nthr >> 5) {
      const int t = (int)(L / keep), c = (int)(L % keep);
      const double* u2 = w.U2 + (long long)c * (r + 1);
      double s;
      if (t < nd) {
        s = 0.0;
        const double* row = Ud + (long long)t * ldc;
        for (int i = lane; i < r; i += 32) s += row[i] * u2[i];
        s = warp_sum(s);
      } else {
        s = u2[r];
      }
      if (lane == 0) Un[(long long)t * ldc + c] = s;
    }
    return;
  }
  // many entries (long streams, n_d large): one thread per entry
  for (long long L = (long long)blockIdx.x * blockDim.x + threadIdx.x; L < total; L += nthr) {
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
  // one warp per entry of M: lanes split the sum over the n_d rows (FP64 is long-latency: a
  // 32-way split and a tree replace a chain of n_d dependent FMAs)
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwt = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long L = gw; L < total; L += nwt) {
    const int a = (int)(L / r), b = (int)(L % r);   // M(a, b)
    double s = 0.0;
    for (int t = lane; t < nd; t += 32) s += Un[(long long)t * ldc + a] * Ud[(long long)t * ldc + b];
    s = warp_sum(s);
    if (lane != 0) continue;
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

// The small ISVD step run by the last block of the e pass (r <= ROWS_RMAX): the block loads p,
// [s; ||e||^2], S and the ranks in parallel into shared memory (one round of loads instead of a
// chain of dependent ones on one thread), warp 0 forms p' and the sums as warp reductions, then
// thread 0 runs isvd_small_tail.
__device__ void isvd_small_block(Ctl* ctl, const double* p, const double* es, const double* S,
                                 const SecWork& w) {
  __shared__ double sp_[ROWS_RMAX + 1], ses_[ROWS_RMAX + 2], sS_[ROWS_RMAX + 1], spq_[ROWS_RMAX + 2];
  __shared__ int srk_[TK_MAXD];
  __shared__ double seps_, sq2_, sq_, szr2_;
  __shared__ int scap_;
  const int d = ctl->d;
  const int r = ctl->r[d - 1];
  for (int i = threadIdx.x; i <= r; i += blockDim.x) {
    ses_[i] = __ldcg(es + i);   // written by other blocks of the calling kernel
    if (i < r) { sp_[i] = p[i]; sS_[i] = S[i]; }
  }
  if (threadIdx.x < d - 1) srk_[threadIdx.x] = ctl->r[threadIdx.x];
  if (threadIdx.x == 32) { seps_ = ctl->eps; scap_ = ctl->cap[d - 1]; }
  __syncthreads();
  // warp 0: p' = p + s, ||s||^2, q'^2 and ||p'||^2 as warp sums (r <= 32: one entry per lane)
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const double sc = lane < r ? ses_[lane] : 0.0;
    const double pc = lane < r ? sp_[lane] + sc : 0.0;
    if (lane < r) { spq_[lane] = pc; w.pq[lane] = pc; }
    const double s2 = warp_sum(sc * sc);
    const double zr2 = warp_sum(pc * pc);
    if (lane == 0) {
      double q2 = ses_[r] - s2;
      if (q2 < 0.0) q2 = 0.0;
      const double q = sqrt(q2);
      spq_[r] = q;
      w.pq[r] = q;
      sq2_ = q2;
      sq_ = q;
      szr2_ = zr2;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long Rn = 1;
    for (int i = 0; i < d - 1; ++i) Rn *= srk_[i];
    isvd_small_tail(ctl, sS_, w, spq_, r, sq2_, sq_, szr2_, Rn, seps_, scap_);
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

// The bulk-tile passes (below) take the update when the slice rows are FP32 work rows and no
// spatial rank grew (old row j is new row j).
__device__ __forceinline__ bool bulk_rows_ok(const Ctl* ctl) {
  return ctl->tw == 4 && rows_isvd_ok(ctl) && !spatial_grew(ctl);
}


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
__device__ __forceinline__ void isvd_p_rows(Ctl* __restrict__ ctl,
                                                        TW* const* dbufs, TW* const* vbufs,
                                                        double* __restrict__ part,
                                                        double* __restrict__ pout) {
  if (ctl->status) return;
  if (!rows_isvd_ok(ctl)) return;
  if (sizeof(TW) == 4 && bulk_rows_ok(ctl)) return;   // the bulk-tile pass ran
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
  rows_block_sum(sw, r, part, TK_STREAM_CAP_MAX);   // k_col_reduce finishes p
  (void)pout;
}

// e = d - V_pad p (stored), ||e||^2 and s = V_pad^T e: partials in the layout of k_isvd_e
// (s in columns 0..r-1, ||e||^2 in column r).
template <typename TW>
__device__ __forceinline__ void isvd_e_rows(Ctl* __restrict__ ctl,
                                                        TW* const* dbufs, TW* const* vbufs,
                                                        const double* __restrict__ p,
                                                        TW* __restrict__ evec,
                                                        double* __restrict__ part,
                                                        double* __restrict__ es,
                                                        const double* __restrict__ S,
                                                        SecWork w) {
  if (ctl->status) return;
  if (!rows_isvd_ok(ctl)) return;
  if (sizeof(TW) == 4 && bulk_rows_ok(ctl)) return;   // the bulk-tile pass ran
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
  rows_block_sum(sw, r + 1, part, TK_STREAM_CAP_MAX + 2);   // k_col_reduce finishes [s; ||e||^2]
  (void)es; (void)S; (void)w;
}

// ---------------------------------------------------------------------------------------------
// Bulk-tile row passes: mixed form, streaming rank <= ROWS_RMAX, no spatial growth in this update
// (old row j is new row j, so the rows of a tile are one contiguous range of V). Tiles of BR_NT
// rows, one per thread, move into shared memory by 1D TMA bulk copies, BR_S stages deep (BR_S - 1
// tiles in flight per block), and each thread reads its row there: V streams from global memory
// at full sector efficiency whatever the row stride. The arithmetic and the FP32 -> FP64 flush
// schedule are those of the lane-per-row passes above.
// ---------------------------------------------------------------------------------------------
constexpr int BR_NT = ROWS_NT;
constexpr int BR_S = 3;
constexpr int BR_TILE = BR_NT * ROWS_RMAX * 4;        // bytes of a tile at the largest row stride
constexpr size_t BR_SMEM = (size_t)BR_S * BR_TILE + 128;

struct BulkTiles {
  const unsigned char* src;   // first row of V
  unsigned char* sm;          // BR_S stages of BR_TILE bytes
  uint64_t* full;             // BR_S mbarriers
  long long R;                // rows
  int rowbytes;               // row stride in bytes (a multiple of 16)
  long long nmine;            // tiles of this block: blockIdx.x, blockIdx.x + gridDim.x, ...
  __device__ void issue(long long i) const {
    const long long row0 = (blockIdx.x + i * (long long)gridDim.x) * BR_NT;
    const long long rows = R - row0 < BR_NT ? R - row0 : BR_NT;
    const uint32_t bytes = (uint32_t)(rows * rowbytes);
    const int st = (int)(i % BR_S);
    tc::mbar_arrive_expect_tx(&full[st], bytes);
    tc::bulk_load(sm + (size_t)st * BR_TILE, src + row0 * rowbytes, bytes, &full[st]);
  }
};

// Set-up common to the bulk passes: barriers, tile counts, the first BR_S - 1 copies.
__device__ __forceinline__ BulkTiles bulk_begin(const float* V, long long R, int s,
                                                unsigned char* dyn, volatile int* abort) {
  BulkTiles bt;
  bt.sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dyn) + 127) & ~uintptr_t(127));
  bt.full = reinterpret_cast<uint64_t*>(bt.sm + (size_t)BR_S * BR_TILE);
  bt.src = reinterpret_cast<const unsigned char*>(V);
  bt.R = R;
  bt.rowbytes = s * 4;
  const long long ntiles = (R + BR_NT - 1) / BR_NT;
  bt.nmine = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  if (threadIdx.x == 0) {
    for (int st = 0; st < BR_S; ++st) tc::mbar_init(&bt.full[st], 1);
    *abort = 0;
    tc::fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (long long i = 0; i < BR_S - 1 && i < bt.nmine; ++i) bt.issue(i);
  return bt;
}

// After an aborted wait: thread 0 waits (bounded) for the copies still in flight, tiles
// consumed .. issued - 1, so none lands after the block has exited.
__device__ __forceinline__ void bulk_drain(const BulkTiles& bt, long long consumed) {
  if (threadIdx.x != 0) return;
  const long long issued = consumed + BR_S - 1 < bt.nmine ? consumed + BR_S - 1 : bt.nmine;
  for (long long i = consumed; i < issued; ++i)
    for (long long k = 0; k < tc::kWaitLimit; ++k)
      if (tc::mbar_try_wait(&bt.full[i % BR_S], (uint32_t)((i / BR_S) & 1))) break;
}

// Adds the per-thread FP32 partials acc[c] (c < r) into the FP64 slots of the warp.
template <int C>
__device__ __forceinline__ void bulk_flush(float (&acc)[C], double* sw, int lane, int r) {
#pragma unroll
  for (int c = 0; c < C; ++c) {
    if (c < r) {
      const float t = warp_sum(acc[c]);
      if (lane == 0) sw[c] += (double)t;
    }
    acc[c] = 0.f;
  }
}

// p = V^T d, S4 = row stride / 4.
template <int S4>
__device__ __forceinline__ long long isvd_p_tiles(const BulkTiles& bt, const float* __restrict__ dv,
                                                  int r, double* sw, volatile int* abort) {
  constexpr int C = 4 * S4;
  float acc[C];
#pragma unroll
  for (int c = 0; c < C; ++c) acc[c] = 0.f;
  const int tid = threadIdx.x, lane = tid & 31;
  int it = 0;
  long long i = 0;
  for (; i < bt.nmine; ++i) {
    if (tid == 0 && i + BR_S - 1 < bt.nmine) bt.issue(i + BR_S - 1);
    const long long row = (blockIdx.x + i * (long long)gridDim.x) * BR_NT + tid;
    const float dj = row < bt.R ? dv[row] : 0.f;
    const int st = (int)(i % BR_S);
    const bool ok = tc::mbar_wait(&bt.full[st], (uint32_t)((i / BR_S) & 1), abort);
    if (ok && row < bt.R) {
      const float4* rp = reinterpret_cast<const float4*>(bt.sm + (size_t)st * BR_TILE) + tid * S4;
#pragma unroll
      for (int q = 0; q < S4; ++q) {
        const float4 v = rp[q];
        acc[4 * q] = fmaf(v.x, dj, acc[4 * q]);
        acc[4 * q + 1] = fmaf(v.y, dj, acc[4 * q + 1]);
        acc[4 * q + 2] = fmaf(v.z, dj, acc[4 * q + 2]);
        acc[4 * q + 3] = fmaf(v.w, dj, acc[4 * q + 3]);
      }
    }
    if (++it == ROWS_FLUSH) { bulk_flush<C>(acc, sw, lane, r); it = 0; }
    if (!__syncthreads_and(ok)) { ++i; break; }
  }
  bulk_flush<C>(acc, sw, lane, r);
  return i;
}

template <typename TW>
__device__ __forceinline__ void isvd_p_bulk(Ctl* __restrict__ ctl, TW* const* dbufs,
                                                      TW* const* vbufs, double* __restrict__ part,
                                                      double* __restrict__ pout) {
  if (ctl->status) return;
  if (sizeof(TW) != 4 || !bulk_rows_ok(ctl)) return;
  extern __shared__ __align__(128) unsigned char br_dyn[];
  __shared__ double sw[ROWS_NT / 32][ROWS_RMAX + 1];
  __shared__ int s_abort;
  const int d = ctl->d, m = d - 1;
  const int r = ctl->r[d - 1];
  const int s = tk_cv_stride(r, ctl->ldc, 4);
  long long R = 1;
  for (int i = 0; i < m; ++i) R *= ctl->r[i];
  const float* V = reinterpret_cast<const float*>(vbufs[ctl->cbuf]);
  const float* dv = reinterpret_cast<const float*>(dbufs[ctl->xbuf]);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int c = lane; c <= ROWS_RMAX; c += 32) sw[wid][c] = 0.0;
  volatile int* abort = &s_abort;
  const BulkTiles bt = bulk_begin(V, R, s, br_dyn, abort);
  long long done = 0;
  switch (s >> 2) {
    case 1: done = isvd_p_tiles<1>(bt, dv, r, sw[wid], abort); break;
    case 2: done = isvd_p_tiles<2>(bt, dv, r, sw[wid], abort); break;
    case 3: done = isvd_p_tiles<3>(bt, dv, r, sw[wid], abort); break;
    case 4: done = isvd_p_tiles<4>(bt, dv, r, sw[wid], abort); break;
    case 5: done = isvd_p_tiles<5>(bt, dv, r, sw[wid], abort); break;
    case 6: done = isvd_p_tiles<6>(bt, dv, r, sw[wid], abort); break;
    case 7: done = isvd_p_tiles<7>(bt, dv, r, sw[wid], abort); break;
    default: done = isvd_p_tiles<8>(bt, dv, r, sw[wid], abort); break;
  }
  if (*abort) {
    bulk_drain(bt, done);
    if (threadIdx.x == 0) ctl->status = TK_ETIMEOUT;
  }
  rows_block_sum(sw, r, part, TK_STREAM_CAP_MAX);   // k_col_reduce finishes p
  (void)pout;
}

// e = d - V p (stored), ||e||^2 (compensated) and s = V^T e as per-block partials; k_col_reduce
// sums them and its last block runs the small ISVD step (as for the lane-per-row body).
template <int S4>
__device__ __forceinline__ long long isvd_e_tiles(const BulkTiles& bt, const float* __restrict__ dv,
                                                  const float* pl, float* __restrict__ evec, int r,
                                                  double* sw, KahanF& eacc, volatile int* abort) {
  constexpr int C = 4 * S4;
  float acc[C], pr[C];
#pragma unroll
  for (int c = 0; c < C; ++c) { acc[c] = 0.f; pr[c] = pl[c]; }
  const int tid = threadIdx.x, lane = tid & 31;
  int it = 0;
  long long i = 0;
  for (; i < bt.nmine; ++i) {
    if (tid == 0 && i + BR_S - 1 < bt.nmine) bt.issue(i + BR_S - 1);
    const long long row = (blockIdx.x + i * (long long)gridDim.x) * BR_NT + tid;
    const float dj = row < bt.R ? dv[row] : 0.f;
    const int st = (int)(i % BR_S);
    const bool ok = tc::mbar_wait(&bt.full[st], (uint32_t)((i / BR_S) & 1), abort);
    if (ok && row < bt.R) {
      const float4* rp = reinterpret_cast<const float4*>(bt.sm + (size_t)st * BR_TILE) + tid * S4;
      float v[C];
#pragma unroll
      for (int q = 0; q < S4; ++q) {
        const float4 t = rp[q];
        v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
      }
      // columns r.. of the last piece are not part of the state (possibly never written)
#pragma unroll
      for (int c = 0; c < C; ++c) v[c] = c < r ? v[c] : 0.f;
      float dot = 0.f;
#pragma unroll
      for (int c = 0; c < C; ++c) dot = fmaf(v[c], pr[c], dot);
      const float e = dj - dot;
#pragma unroll
      for (int c = 0; c < C; ++c) acc[c] = fmaf(v[c], e, acc[c]);
      evec[row] = e;
      eacc.add(e * e);
    }
    if (++it == ROWS_FLUSH) { bulk_flush<C>(acc, sw, lane, r); it = 0; }
    if (!__syncthreads_and(ok)) { ++i; break; }
  }
  bulk_flush<C>(acc, sw, lane, r);
  return i;
}

template <typename TW>
__device__ __forceinline__ void isvd_e_bulk(Ctl* __restrict__ ctl, TW* const* dbufs,
                                                      TW* const* vbufs, const double* __restrict__ p,
                                                      TW* __restrict__ evec, double* __restrict__ part,
                                                      double* __restrict__ es,
                                                      const double* __restrict__ S, SecWork w) {
  if (ctl->status) return;
  if (sizeof(TW) != 4 || !bulk_rows_ok(ctl)) return;
  extern __shared__ __align__(128) unsigned char br_dyn[];
  __shared__ double sw[ROWS_NT / 32][ROWS_RMAX + 1];
  __shared__ float pl[ROWS_RMAX];
  __shared__ int s_abort;
  const int d = ctl->d, m = d - 1;
  const int r = ctl->r[d - 1];
  const int s = tk_cv_stride(r, ctl->ldc, 4);
  long long R = 1;
  for (int i = 0; i < m; ++i) R *= ctl->r[i];
  const float* V = reinterpret_cast<const float*>(vbufs[ctl->cbuf]);
  const float* dv = reinterpret_cast<const float*>(dbufs[ctl->xbuf]);
  float* ev = reinterpret_cast<float*>(evec);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int c = lane; c <= ROWS_RMAX; c += 32) sw[wid][c] = 0.0;
  if (threadIdx.x < ROWS_RMAX) pl[threadIdx.x] = threadIdx.x < r ? (float)p[threadIdx.x] : 0.f;
  volatile int* abort = &s_abort;
  const BulkTiles bt = bulk_begin(V, R, s, br_dyn, abort);   // barrier inside: pl is visible
  KahanF eacc;
  long long done = 0;
  switch (s >> 2) {
    case 1: done = isvd_e_tiles<1>(bt, dv, pl, ev, r, sw[wid], eacc, abort); break;
    case 2: done = isvd_e_tiles<2>(bt, dv, pl, ev, r, sw[wid], eacc, abort); break;
    case 3: done = isvd_e_tiles<3>(bt, dv, pl, ev, r, sw[wid], eacc, abort); break;
    case 4: done = isvd_e_tiles<4>(bt, dv, pl, ev, r, sw[wid], eacc, abort); break;
    case 5: done = isvd_e_tiles<5>(bt, dv, pl, ev, r, sw[wid], eacc, abort); break;
    case 6: done = isvd_e_tiles<6>(bt, dv, pl, ev, r, sw[wid], eacc, abort); break;
    case 7: done = isvd_e_tiles<7>(bt, dv, pl, ev, r, sw[wid], eacc, abort); break;
    default: done = isvd_e_tiles<8>(bt, dv, pl, ev, r, sw[wid], eacc, abort); break;
  }
  if (*abort) {
    bulk_drain(bt, done);
    if (threadIdx.x == 0) ctl->status = TK_ETIMEOUT;
  }
  const double e2 = warp_sum(eacc.value());
  if (lane == 0) sw[wid][ROWS_RMAX] = e2;
  __syncthreads();
  // ||e||^2 moves to column r (columns r.. of the slots hold zeros)
  if (threadIdx.x < ROWS_NT / 32 && r < ROWS_RMAX) sw[threadIdx.x][r] = sw[threadIdx.x][ROWS_RMAX];
  rows_block_sum(sw, r + 1, part, TK_STREAM_CAP_MAX + 2);   // k_col_reduce finishes [s; ||e||^2]
  (void)es; (void)S; (void)w;
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
  // the whole control block is copied to shared memory in one round of loads by all threads;
  // thread 0 then reads it there (its updates go to global memory) instead of waiting on a
  // chain of dependent global loads
  __shared__ __align__(128) unsigned char cbuf_[sizeof(Ctl)];
  static_assert(sizeof(Ctl) % 16 == 0, "control block copied in 16-byte words");
  for (int i = threadIdx.x; i < (int)(sizeof(Ctl) / 16); i += blockDim.x)
    reinterpret_cast<uint4*>(cbuf_)[i] = __ldcg(reinterpret_cast<const uint4*>(ctl) + i);
  __syncthreads();
  const Ctl& c = *reinterpret_cast<const Ctl*>(cbuf_);
  const int d = c.d;
  const int keep = c.rnew_d;
  for (int i = threadIdx.x; i < keep; i += blockDim.x) S[i] = Snew[i];
  if (threadIdx.x == 0) {
    // algorithmic bytes of this update (each operand read or written once per pass), in integer
    // arithmetic (FP64 operations are long-latency on this part and this is one thread)
    const long long tw = c.tw, tx = c.tx;
    const long long r = c.r[d - 1];
    long long Ro = 1, Rn = 1;
    for (int k = 0; k < d - 1; ++k) { Ro *= c.rold[k]; Rn *= c.r[k]; }
    long long A = 1;
    long long bp1 = 0, bpn = 0, bgr = 0;
    for (int k = 0; k < d - 1; ++k) {
      long long B = 1;
      for (int i = k + 1; i < d - 1; ++i) B *= c.n[i];
      const long long in_b = (k == 0 ? tx : tw) * A * c.n[k] * B;
      const long long p_b = tw * A * c.rold[k] * B;
      if (k == 0) bp1 += in_b + p_b; else bpn += in_b + p_b;
      if (c.grew[k]) bgr += 2 * in_b + p_b + tw * A * c.r[k] * B;
      A *= c.r[k];
    }
    const long long nd = c.nd;
    // a block update's spatial passes covered blk slices, once (its row 0)
    const long long bm = c.row == 0 ? (c.blk > 1 ? c.blk : 1) : 0;
    ctl->acc_bytes[TK_PH_PROJ1] = c.acc_bytes[TK_PH_PROJ1] + (double)(bm * bp1);
    ctl->acc_bytes[TK_PH_PROJN] = c.acc_bytes[TK_PH_PROJN] + (double)(bm * bpn);
    ctl->acc_bytes[TK_PH_GROW] = c.acc_bytes[TK_PH_GROW] + (double)(bm * bgr);
    ctl->acc_bytes[TK_PH_ISVD] = c.acc_bytes[TK_PH_ISVD] + (double)(tw * (2 * Ro * r + 3 * Rn));
    ctl->acc_bytes[TK_PH_FACT] = c.acc_bytes[TK_PH_FACT] + (double)(16 * (nd * r + (nd + 1) * keep));
    ctl->acc_bytes[TK_PH_CV] = c.acc_bytes[TK_PH_CV] + (double)(tw * (2 * Ro * r + 2 * Rn * keep + 2 * Rn));
    // error bookkeeping (Prop. 1, Prop. 2, App. D): discarded energies of this update
    double disc = 0.0;
    for (int k = 0; k < d - 1; ++k) disc += c.disc[k];
    disc += c.aug ? 0.0 : c.q2;
    disc += c.dropped;
    ctl->err2 = c.err2 + disc;
    ctl->data2 = c.data2 + c.y2;
    // the tensor-core path after spatial growth expands into the other buffer and writes back
    // into this one; every other path writes the other buffer
    const bool stay = tc_cv_ok(&c, keep) && spatial_grew(&c);
    ctl->r[d - 1] = keep;
    ctl->nd = c.nd + 1;
    if (!stay) ctl->cbuf = c.cbuf ^ 1;
    ctl->ubuf = c.ubuf ^ 1;
    ctl->nupdates = c.nupdates + 1;
    // the update's decisions into the log, and the replay hook is spent
    if (c.log && c.nupdates < c.log_cap) {
      StepRec& o = c.log[c.nupdates];
      o.nd = c.nd + 1;
      for (int k = 0; k < TK_MAXD; ++k) {
        const bool sp = k < d - 1;
        o.r[k] = (k < d - 1) ? c.r[k] : (k == d - 1 ? keep : 0);
        o.grew[k] = sp ? c.grew[k] : 0;
        o.radd[k] = sp ? c.radd[k] : 0;
        o.eig_path[k] = (sp && c.grew[k]) ? (c.eig_fb[k] ? 2 : 1) : 0;
        o.eig_it[k] = (sp && c.grew[k]) ? c.eig_it[k] : 0;
        o.e2[k] = sp ? c.e2[k] : 0.0;
        o.tail_cut[k] = (sp && c.grew[k]) ? c.disc[k] : 0.0;
        o.tail_prev[k] = (sp && c.grew[k]) ? c.tail_prev[k] : 0.0;
      }
      o.aug = c.aug;
      o.replayed = c.rp_on;
      o.eps = c.eps;
      o.y2 = c.y2;
      o.q = c.q;
      o.discarded = disc;
    }
    ctl->rp_on = 0;
  }
}

__global__ void k_begin_update(Ctl* ctl, int blk) {
  if (ctl->status) return;
  ctl->blk = blk;
  ctl->row = 0;
  for (int k = 0; k < TK_MAXD; ++k) {
    ctl->rold[k] = ctl->r[k];
    ctl->grew[k] = 0;
    ctl->radd[k] = 0;
    ctl->e2[k] = 0.0;
    ctl->disc[k] = 0.0;
    ctl->tail_prev[k] = 0.0;
    ctl->eig_m[k] = 0;
    ctl->eig_it[k] = 0;
    ctl->eig_fb[k] = 0;
    ctl->xmax[k] = 0u;
  }
  ctl->xbuf = -1;
  ctl->aug = 0;
  ctl->q = 0.0;
  ctl->q2 = 0.0;
  ctl->dropped = 0.0;
  if (ctl->nd + blk > ctl->steps_cap) ctl->status = TK_ECAPACITY;
}

// Block update, after the spatial modes: D*_{d-1} holds the blk projected slices with the slice
// index fastest (blk x R, the rotating layout's order); Dt gets them as blk contiguous vectors of
// R entries (R x blk), and the streaming mode's tolerance becomes eps / sqrt(blk) per row (the
// block's streaming share split evenly; see tucker_stream_update_block).
template <typename TW>
__global__ void k_block_rows(Ctl* ctl, TW* const* dbufs, TW* __restrict__ Dt) {
  if (ctl->status) return;
  const int d = ctl->d, B = ctl->blk;
  long long R = 1;
  for (int k = 0; k < d - 1; ++k) R *= ctl->r[k];
  const TW* D = dbufs[ctl->xbuf];
  for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < R * B;
       L += (long long)gridDim.x * blockDim.x) {
    const long long j = L % R, b = L / R;
    Dt[L] = D[b + B * j];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->eps = ctl->eps / sqrt((double)B);
}

// Row b of a block update: its projected slice into the D*_{d-1} buffer (the input of the
// incremental-SVD and core kernels); for b > 0 the per-update record is reset, as the spatial
// modes' decisions, discards and the block's norm belong to row 0 only.
template <typename TW>
__global__ void k_row_begin(Ctl* ctl, int b, TW* const* dbufs, const TW* __restrict__ Dt) {
  if (ctl->status) return;
  const int d = ctl->d;
  long long R = 1;
  for (int k = 0; k < d - 1; ++k) R *= ctl->r[k];
  TW* D = dbufs[ctl->xbuf];
  const TW* src = Dt + (long long)b * R;
  for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < R;
       L += (long long)gridDim.x * blockDim.x)
    D[L] = src[L];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->row = b;
    if (b > 0) {
      for (int k = 0; k < TK_MAXD; ++k) {
        ctl->rold[k] = ctl->r[k];
        ctl->grew[k] = 0;
        ctl->radd[k] = 0;
        ctl->e2[k] = 0.0;
        ctl->disc[k] = 0.0;
        ctl->tail_prev[k] = 0.0;
        ctl->eig_m[k] = 0;
        ctl->eig_it[k] = 0;
        ctl->eig_fb[k] = 0;
      }
      ctl->y2 = 0.0;
      ctl->aug = 0;
      ctl->q = 0.0;
      ctl->q2 = 0.0;
      ctl->dropped = 0.0;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------------
// One launch for the bulk-tile and lane-per-row bodies of each pass, chosen on the device (one
// kernel node instead of two in the update graph); both take 256 threads and the pass's grid.
// The SIMT pass (streaming rank above ROWS_RMAX) stays a kernel of its own: its shared tiles
// would leave this launch one block per SM.
template <typename TW>
__global__ void __launch_bounds__(256) k_isvd_p_all(Ctl* __restrict__ ctl, TW* const* dbufs,
                                                   TW* const* vbufs, double* __restrict__ part,
                                                   double* __restrict__ pout) {
  if (ctl->status) return;
  if (sizeof(TW) == 4 && bulk_rows_ok(ctl)) isvd_p_bulk<TW>(ctl, dbufs, vbufs, part, pout);
  else if (rows_isvd_ok(ctl)) isvd_p_rows<TW>(ctl, dbufs, vbufs, part, pout);
}

template <typename TW>
__global__ void __launch_bounds__(256) k_isvd_e_all(Ctl* __restrict__ ctl, TW* const* dbufs,
                                                   TW* const* vbufs, const double* __restrict__ p,
                                                   TW* __restrict__ evec, double* __restrict__ part,
                                                   double* __restrict__ es,
                                                   const double* __restrict__ S, SecWork w) {
  if (ctl->status) return;
  if (sizeof(TW) == 4 && bulk_rows_ok(ctl)) isvd_e_bulk<TW>(ctl, dbufs, vbufs, p, evec, part, es, S, w);
  else if (rows_isvd_ok(ctl)) isvd_e_rows<TW>(ctl, dbufs, vbufs, p, evec, part, es, S, w);
}

// Cross-block sums of the lane-per-row and bulk-tile passes (streaming rank <= ROWS_RMAX; the
// SIMT passes sum in their own last block): out[c] = sum over blocks b < nb of part[b stride + c]
// for c < len, one block per column, every partial loaded in one round, added in a fixed order
// (per-thread, then warp, then block). which = 1 (the e pass, len = r + 1): the last block to
// finish then runs the small ISVD step.
constexpr int CR_NT = 256;
__global__ void __launch_bounds__(CR_NT) k_col_reduce(Ctl* __restrict__ ctl, const double* __restrict__ part,
                                                     long long stride, int nb, double* __restrict__ out,
                                                     int which, const double* __restrict__ p,
                                                     const double* __restrict__ S, SecWork w) {
  if (ctl->status) return;
  if (!rows_isvd_ok(ctl)) return;
  const int r = ctl->r[ctl->d - 1];
  const int len = which ? r + 1 : r;
  const int c = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __shared__ double red[CR_NT / 32];
  if (c < len) {
    double a0 = 0.0, a1 = 0.0;
    int b = threadIdx.x;
    for (; b + CR_NT < nb; b += 2 * CR_NT) {
      a0 += __ldcg(part + (long long)b * stride + c);
      a1 += __ldcg(part + (long long)(b + CR_NT) * stride + c);
    }
    if (b < nb) a0 += __ldcg(part + (long long)b * stride + c);
    const double t = warp_sum(a0 + a1);
    if (lane == 0) red[wid] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double u = 0.0;
#pragma unroll
      for (int i = 0; i < CR_NT / 32; ++i) u += red[i];
      out[c] = u;
    }
  }
  if (which && tk_block_ticket(&ctl->ticket[2])) isvd_small_block(ctl, p, out, S, w);
}

template <typename TW>
cudaError_t launch_isvd(Ctl* ctl, void* const* dbufs, void* const* vbufs, double* part_p,
                        double* part_e, double* p, double* es, void* evec, const double* S,
                        SecWork w, int grid, cudaStream_t st) {
  // p = V^T d, then e = d - V p with [s; ||e||^2] and the small ISVD bookkeeping; each pass
  // finishes its cross-block sum in its last block. Exactly one of the bulk-tile, lane-per-row
  // and SIMT kernels of each pass does the work (device-side conditions).
  // dynamic shared memory: the bulk-tile stages (FP32 work type only)
  const size_t dyn = sizeof(TW) == 4 ? BR_SMEM : 0;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_isvd_p_all<TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BR_SMEM);
    cudaFuncSetAttribute(k_isvd_e_all<TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BR_SMEM);
    attr = true;
  }
  k_isvd_p_all<TW><<<grid, 256, dyn, st>>>(ctl, (TW* const*)dbufs, (TW* const*)vbufs, part_p, p);
  k_isvd_p<TW><<<grid, 256, 0, st>>>(ctl, (TW* const*)dbufs, (TW* const*)vbufs, part_p, p);
  k_col_reduce<<<ROWS_RMAX + 1, CR_NT, 0, st>>>(ctl, part_p, TK_STREAM_CAP_MAX, grid, p, 0, nullptr, nullptr, w);
  k_isvd_e_all<TW><<<grid, 256, dyn, st>>>(ctl, (TW* const*)dbufs, (TW* const*)vbufs, p,
                                           (TW*)evec, part_e, es, S, w);
  k_isvd_e<TW><<<grid, 256, 0, st>>>(ctl, (TW* const*)dbufs, (TW* const*)vbufs, p, (TW*)evec,
                                     part_e, es, S, w);
  k_col_reduce<<<ROWS_RMAX + 1, CR_NT, 0, st>>>(ctl, part_e, TK_STREAM_CAP_MAX + 2, grid, es, 1, p, S, w);
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

template <typename TW>
cudaError_t launch_block_rows(Ctl* ctl, void* const* dbufs, void* Dt, cudaStream_t st) {
  k_block_rows<TW><<<152 * 2, 256, 0, st>>>(ctl, (TW* const*)dbufs, (TW*)Dt);
  return cudaGetLastError();
}
template <typename TW>
cudaError_t launch_row_begin(Ctl* ctl, int b, void* const* dbufs, const void* Dt, cudaStream_t st) {
  k_row_begin<TW><<<152 * 2, 256, 0, st>>>(ctl, b, (TW* const*)dbufs, (const TW*)Dt);
  return cudaGetLastError();
}
template cudaError_t launch_block_rows<float>(Ctl*, void* const*, void*, cudaStream_t);
template cudaError_t launch_block_rows<double>(Ctl*, void* const*, void*, cudaStream_t);
template cudaError_t launch_row_begin<float>(Ctl*, int, void* const*, const void*, cudaStream_t);
template cudaError_t launch_row_begin<double>(Ctl*, int, void* const*, const void*, cudaStream_t);

cudaError_t launch_begin(Ctl* ctl, cudaStream_t st, int blk) {
  k_begin_update<<<1, 1, 0, st>>>(ctl, blk);
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
