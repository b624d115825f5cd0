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

template <typename TE> struct Eps;
template <> struct Eps<double> { static __device__ double u() { return 1.1102230246251565e-16; } static __device__ double tiny() { return 1e-290; } };
template <> struct Eps<float> { static __device__ float u() { return 5.9604645e-08f; } static __device__ float tiny() { return 1e-35f; } };

// Sturm count: number of eigenvalues of the tridiagonal (a, b) strictly below x.
template <typename TE>
__device__ __forceinline__ TE sturm_div(TE a, TE b) { return a / b; }
template <>
__device__ __forceinline__ float sturm_div<float>(float a, float b) { return __fdividef(a, b); }

template <typename TE>
__device__ int sturm_count(const TE* a, const TE* b2, int n, TE x, TE pivmin) {
  int cnt = 0;
  TE q = a[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < TE(0)) ++cnt;
  for (int i = 1; i < n; ++i) {
    q = (a[i] - x) - sturm_div(b2[i - 1], q);
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < TE(0)) ++cnt;
  }
  return cnt;
}

// Sturm counts at three shifts in one sweep (three independent recurrences per step).
template <typename TE>
__device__ void sturm_count3(const TE* a, const TE* b2, int n, TE x0, TE x1, TE x2, TE pivmin,
                             int& c0, int& c1, int& c2) {
  c0 = c1 = c2 = 0;
  TE q0 = a[0] - x0, q1 = a[0] - x1, q2 = a[0] - x2;
  if (fabs(q0) < pivmin) q0 = -pivmin;
  if (fabs(q1) < pivmin) q1 = -pivmin;
  if (fabs(q2) < pivmin) q2 = -pivmin;
  c0 += q0 < TE(0); c1 += q1 < TE(0); c2 += q2 < TE(0);
  for (int i = 1; i < n; ++i) {
    const TE ai = a[i], bi = b2[i - 1];
    q0 = (ai - x0) - sturm_div(bi, q0);
    q1 = (ai - x1) - sturm_div(bi, q1);
    q2 = (ai - x2) - sturm_div(bi, q2);
    if (fabs(q0) < pivmin) q0 = -pivmin;
    if (fabs(q1) < pivmin) q1 = -pivmin;
    if (fabs(q2) < pivmin) q2 = -pivmin;
    c0 += q0 < TE(0); c1 += q1 < TE(0); c2 += q2 < TE(0);
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

// use_smem: dynamic shared memory holds the eigenvector workspaces (up to EIG_SMEM_VECS vectors)
// after the n x n working matrix when use_amat, else at its start.
template <typename TE>
__global__ void __launch_bounds__(EIG_NT) k_eig_topk(Ctl* ctl, int k, int mode, EigArgs ea,
                                                    int use_smem, int use_amat) {
  extern __shared__ __align__(16) unsigned char eig_dyn[];
  if (ctl->status) return;
  if (mode == 0 && !ctl->grew[k]) return;
  const int d = ctl->d;
  const int n = (k == d - 1) ? ctl->init_nt : ctl->n[k];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nwarp = nt >> 5;
  TE* A = use_amat ? reinterpret_cast<TE*>(eig_dyn) : reinterpret_cast<TE*>(ea.Aw);
  __shared__ TE sa[TK_N_MAX], sb[TK_N_MAX], sb2[TK_N_MAX], stau[TK_N_MAX], slam[TK_N_MAX];
  __shared__ TE sv[TK_N_MAX], sp[TK_N_MAX];
  __shared__ TE tred[32];
  __shared__ int s_m;
  __shared__ double s_disc;

  for (long long L = tid; L < (long long)n * n; L += nt) A[L] = (TE)ea.G[L];
  __syncthreads();

  // ---- Householder tridiagonalization: A = Q T Q^T, reflectors stored below the diagonal ----
  // Reflector c (LAPACK convention H = I - tau v v^T, v_0 = 1) from column c below the
  // diagonal; warp 0 forms it (warp reduction) as soon as that column is final, into one of two
  // buffers, while the other warps finish the rank-2 update of the previous step.
  __shared__ TE svb[2][TK_N_MAX];
  __shared__ int s_skip[2];
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
  for (int i = tid; i < n - 1; i += nt) sb2[i] = sb[i] * sb[i];
  __syncthreads();

  // ---- eigenvalues by bisection (one thread per eigenvalue, ascending index) ----
  {
    TE gl = sa[0], gu = sa[0], bmax2 = TE(0);
    for (int i = 0; i < n; ++i) {
      const TE rad = (i > 0 ? fabs(sb[i - 1]) : TE(0)) + (i < n - 1 ? fabs(sb[i]) : TE(0));
      gl = min(gl, sa[i] - rad);
      gu = max(gu, sa[i] + rad);
      if (i < n - 1) bmax2 = max(bmax2, sb2[i]);
    }
    const TE scale = max(fabs(gl), fabs(gu));
    const TE u = Eps<TE>::u();
    gl -= TE(2) * u * scale * n + Eps<TE>::tiny();
    gu += TE(2) * u * scale * n + Eps<TE>::tiny();
    const TE pivmin = max(Eps<TE>::tiny(), u * u * bmax2);
    for (int i = tid; i < n; i += nt) {
      TE lo = gl, hi = gu;
      for (int it = 0; it < 100; ++it) {
        const TE w = hi - lo;
        if (w <= TE(2) * u * max(fabs(lo), fabs(hi)) + pivmin) break;
        const TE x0 = lo + TE(0.25) * w, x1 = lo + TE(0.5) * w, x2 = lo + TE(0.75) * w;
        if (!(x0 > lo && x2 < hi)) break;
        int c0, c1, c2;
        sturm_count3(sa, sb2, n, x0, x1, x2, pivmin, c0, c1, c2);
        if (c0 > i) hi = x0;
        else if (c1 > i) { lo = x0; hi = x1; }
        else if (c2 > i) { lo = x1; hi = x2; }
        else lo = x2;
      }
      slam[n - 1 - i] = TE(0.5) * (lo + hi);   // store descending
    }
  }
  __syncthreads();

  // ---- rank decision (Alg. 1) in FP64: tails[l] = lam_l + ... + lam_{n-1}, first l with
  // tails[l] <= eps^2 ----
  __shared__ double stails[TK_N_MAX + 1];
  if (tid == 0) {
    const double eps2 = ctl->eps * ctl->eps;
    stails[n] = 0.0;
    for (int l = n - 1; l >= 0; --l) stails[l] = stails[l + 1] + (double)slam[l];
    int m = n;
    for (int l = 0; l <= n; ++l) {
      if (stails[l] <= eps2) { m = l; break; }
    }
    double disc = 0.0;
    for (int i = m; i < n; ++i) disc += (double)slam[i];
    int status = 0;
    if (mode == 0) {
      const int rk = ctl->r[k];
      if (m > n - rk) m = n - rk;
      disc = 0.0;
      for (int i = m; i < n; ++i) disc += (double)slam[i];
      if (rk + m > ctl->cap[k]) status = TK_ECAPACITY;
    } else {
      if (m < 1) m = 1;
      disc = 0.0;
      for (int i = m; i < n; ++i) disc += (double)slam[i];
      if (m > ctl->cap[k] || m > ea.mcap) status = TK_ECAPACITY;
    }
    if (m > ea.mcap) status = TK_ECAPACITY;
    if (status) ctl->status = status;
    s_m = status ? 0 : m;
    s_disc = disc;
  }
  __syncthreads();
  const int m = s_m;
  if (ea.lam_out)
    for (int i = tid; i < n; i += nt) ea.lam_out[i] = (double)slam[i];
  if (m == 0) {
    if (tid == 0) {
      if (mode == 0) { ctl->radd[k] = 0; ctl->disc[k] = s_disc; }
      else { ctl->r[k] = 0; ctl->disc[k] = s_disc; }
    }
    return;
  }

  // ---- inverse iteration for the top m eigenvalues ----
  // eigenvector workspaces in shared memory when up to EIG_SMEM_VECS vectors are needed
  const bool zsm = use_smem && m <= EIG_SMEM_VECS;
  TE* zbase = reinterpret_cast<TE*>(eig_dyn) + (size_t)n * n * use_amat;
  TE* Z = zsm ? zbase : reinterpret_cast<TE*>(ea.Z);                       // n x m
  TE* LD = zsm ? zbase + (size_t)EIG_SMEM_VECS * n : reinterpret_cast<TE*>(ea.LD);  // L, D
  TE tnorm = TE(0);
  for (int i = 0; i < n; ++i) tnorm = max(tnorm, fabs(sa[i]) + (i < n - 1 ? fabs(sb[i]) : TE(0)) + (i > 0 ? fabs(sb[i - 1]) : TE(0)));
  const TE u = Eps<TE>::u();
  const TE pivt = max(u * tnorm, Eps<TE>::tiny());
  for (int v = tid; v < m; v += nt) {
    // shift slightly away from the computed eigenvalue so the factorization is nonsingular
    const TE sig = slam[v] + TE(4) * u * tnorm;
    TE* Lv = LD + (long long)v * 2 * n;
    TE* Dv = Lv + n;
    TE dcur = sa[0] - sig;
    if (fabs(dcur) < pivt) dcur = copysign(pivt, dcur == TE(0) ? TE(1) : dcur);
    Dv[0] = dcur;
    for (int i = 0; i < n - 1; ++i) {
      const TE l = sb[i] / dcur;
      Lv[i] = l;
      dcur = (sa[i + 1] - sig) - l * sb[i];
      if (fabs(dcur) < pivt) dcur = copysign(pivt, dcur == TE(0) ? TE(1) : dcur);
      Dv[i + 1] = dcur;
    }
    // deterministic start vector
    for (int i = 0; i < n; ++i) {
      unsigned h = (unsigned)(i * 2654435761u) ^ (unsigned)((v + 1) * 40503u);
      h ^= h >> 13; h *= 0x5bd1e995u; h ^= h >> 15;
      Z[(long long)v * n + i] = TE(1) + TE(0.5) * (TE)((h & 0xffff) / 65535.0);
    }
  }
  __syncthreads();
  for (int iter = 0; iter < 3; ++iter) {
    for (int v = tid; v < m; v += nt) {
      const TE* Lv = LD + (long long)v * 2 * n;
      const TE* Dv = Lv + n;
      TE* z = Z + (long long)v * n;
      for (int i = 1; i < n; ++i) z[i] -= Lv[i - 1] * z[i - 1];
      for (int i = 0; i < n; ++i) z[i] /= Dv[i];
      for (int i = n - 2; i >= 0; --i) z[i] -= Lv[i] * z[i + 1];
    }
    __syncthreads();
    // modified Gram-Schmidt across the m vectors (separates clusters), block-wide
    for (int v = 0; v < m; ++v) {
      TE* z = Z + (long long)v * n;
      TE part = TE(0);
      for (int i = tid; i < n; i += nt) part += z[i] * z[i];
      const TE nrm = sqrt(block_sum(part, tred));
      const TE inv = nrm > TE(0) ? TE(1) / nrm : TE(0);
      for (int i = tid; i < n; i += nt) z[i] *= inv;
      __syncthreads();
      // project out of later vectors: one warp per later vector
      for (int w = v + 1 + wid; w < m; w += nwarp) {
        TE* y = Z + (long long)w * n;
        TE s = TE(0);
        for (int i = lane; i < n; i += 32) s += z[i] * y[i];
        s = warp_sum(s);
        for (int i = lane; i < n; i += 32) y[i] -= s * z[i];
      }
      __syncthreads();
    }
  }
  // ---- back-transform: x = H_0 H_1 ... H_{n-3} z (one warp per vector) ----
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
  __syncthreads();
  for (long long L = tid; L < (long long)m * n; L += nt) ea.W[L] = (double)Z[L];
  if (tid == 0) {
    if (mode == 0) { ctl->radd[k] = m; ctl->disc[k] = s_disc; }
    else { ctl->r[k] = m; ctl->disc[k] = s_disc; }
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
  const size_t mat = (size_t)n * n * sizeof(TE);
  const size_t vec = (size_t)EIG_SMEM_VECS * 3 * n * sizeof(TE);
  const int use_vec = (vec <= 150 * 1024) ? 1 : 0;
  const int use_amat = (use_vec && mat + vec <= EIG_SMEM_MAX) ? 1 : 0;
  const size_t sm = (use_amat ? mat : 0) + (use_vec ? vec : 0);
  if (sm) cudaFuncSetAttribute(k_eig_topk<TE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_eig_topk<TE><<<1, EIG_NT, sm, st>>>(ctl, k, mode, ea, use_vec, use_amat);
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
