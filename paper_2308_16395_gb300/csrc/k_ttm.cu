// Tucker projection / reconstruction chains and their adjoints (C ABI in include/tucker_ttm.h).
//
// Every step is one of two kernels:
//   k_ttm_mode : one mode product out = X x_k W for a column-major tensor viewed as (A, I, B)
//                (A = product of the sizes before mode k, B = after it): out(a, j, b) =
//                sum_i W(j, i) X(a, i, b) (Sec. 2.1), with W = U_k^T (projection) or U_k
//                (reconstruction) read through strides, never transposed in memory;
//   k_ttm_gram : the factor gradient dL/dU_n(i, j) = sum_{a,b} Z(a, i, b) H(a, j, b), i.e.
//                Z_(n) H_(n)^T with Z = X x_{k!=n} U_k^T and H the core-shaped tensor (Gbar or G).
// The adjoints recompute X x_{k!=n} U_k^T from their inputs: a prefix X x_1 U_1^T .. x_{n-1}
// U_{n-1}^T is carried from mode to mode and each mode's chain continues from it.
// At the sizes this serves (slices of a few million elements, ranks of tens) every launch is
// short and the data stays in L2: the chain is latency-bound, so the kernels are plain FP32 / FP64
// FMA loops with coalesced loads along the fastest index and no tensor-core staging.
#include <stdio.h>

#include <algorithm>

#include "../../include/tucker_ttm.h"
#include "common.cuh"

namespace {

constexpr int kJT = 8;            // outputs per thread along the produced mode
constexpr int kThreads = 256;
constexpr int kWsmemMax = 32768;  // bytes of W staged in shared memory

// out(a, j, b) = sum_i W(j, i) X(a, i, b);  W(j, i) = W[j * wj + i * wi].
// Thread index L = a + A (jb + nJB b): a warp covers consecutive a (coalesced when A >= 32) or,
// for A = 1, the j-blocks of consecutive columns b.
template <typename T, bool kSmemW>
__global__ void __launch_bounds__(kThreads) k_ttm_mode(const T* __restrict__ X, long long A, int I,
                                                       long long B, const T* __restrict__ W,
                                                       long long wj, long long wi, int J,
                                                       T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ws = reinterpret_cast<T*>(smem_raw);  // Ws[i * J + j]
  if (kSmemW) {
    for (int e = threadIdx.x; e < I * J; e += blockDim.x) {
      const int i = e / J, j = e - i * J;
      Ws[e] = W[(long long)j * wj + (long long)i * wi];
    }
    __syncthreads();
  }
  const int nJB = (J + kJT - 1) / kJT;
  const long long total = A * B * nJB;
  for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < total;
       L += (long long)gridDim.x * blockDim.x) {
    const long long a = L % A;
    const long long q = L / A;
    const int jb = (int)(q % nJB);
    const long long b = q / nJB;
    const int j0 = jb * kJT;
    const T* x = X + a + A * (long long)I * b;
    T acc[kJT];
#pragma unroll
    for (int t = 0; t < kJT; ++t) acc[t] = T(0);
    if (j0 + kJT <= J) {
      for (int i = 0; i < I; ++i) {
        const T xv = x[A * (long long)i];
#pragma unroll
        for (int t = 0; t < kJT; ++t) {
          const T w = kSmemW ? Ws[i * J + j0 + t] : __ldg(W + (long long)(j0 + t) * wj + (long long)i * wi);
          acc[t] = fma(w, xv, acc[t]);
        }
      }
    } else {
      const int jn = J - j0;
      for (int i = 0; i < I; ++i) {
        const T xv = x[A * (long long)i];
#pragma unroll
        for (int t = 0; t < kJT; ++t) {
          if (t < jn) {
            const T w = kSmemW ? Ws[i * J + j0 + t] : __ldg(W + (long long)(j0 + t) * wj + (long long)i * wi);
            acc[t] = fma(w, xv, acc[t]);
          }
        }
      }
    }
    T* o = out + a + A * ((long long)j0 + (long long)J * b);
    const int jn = min(kJT, J - j0);
#pragma unroll
    for (int t = 0; t < kJT; ++t)
      if (t < jn) o[A * (long long)t] = acc[t];
  }
}

// out(i, j) = sum_{a, b} Z(a, i, b) H(a, j, b); Z is (A, I, B), H is (A, J, B), out is I x J
// column-major. One warp per output; lanes stride over the (a, b) pairs (coalesced along a).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_ttm_gram(const T* __restrict__ Z,
                                                       const T* __restrict__ H, long long A, int I,
                                                       int J, long long B, T* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const long long AB = A * B;
  for (long long o = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
       o < (long long)I * J; o += warps) {
    const int i = (int)(o % I), j = (int)(o / I);
    T s = T(0);
    for (long long L = lane; L < AB; L += 32) {
      const long long a = L % A, b = L / A;
      s = fma(Z[a + A * (i + (long long)I * b)], H[a + A * (j + (long long)J * b)], s);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) out[i + (long long)I * j] = s;
  }
}

struct Shape {
  int m = 0;
  long long dim[TUCKER_MAX_MODES]{};
  long long numel() const {
    long long p = 1;
    for (int k = 0; k < m; ++k) p *= dim[k];
    return p;
  }
  long long before(int k) const {
    long long p = 1;
    for (int i = 0; i < k; ++i) p *= dim[i];
    return p;
  }
  long long after(int k) const {
    long long p = 1;
    for (int i = k + 1; i < m; ++i) p *= dim[i];
    return p;
  }
};

int g_nsm = 0;

int grid_for(long long work) {
  if (g_nsm == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      g_nsm = 152;
  }
  long long g = (work + kThreads - 1) / kThreads;
  g = std::min<long long>(g, (long long)g_nsm * 16);
  return (int)std::max<long long>(g, 1);
}

// X (shape s, s.dim[k] == I) x_k W -> out (shape s with dim[k] = J).
template <typename T>
cudaError_t mode_product(const T* X, const Shape& s, int k, const T* W, long long wj, long long wi,
                         int J, T* out, cudaStream_t st) {
  const long long A = s.before(k), B = s.after(k);
  const int I = (int)s.dim[k];
  const long long work = A * B * ((J + kJT - 1) / kJT);
  const size_t wbytes = (size_t)I * J * sizeof(T);
  if (wbytes <= (size_t)kWsmemMax) {
    k_ttm_mode<T, true><<<grid_for(work), kThreads, wbytes, st>>>(X, A, I, B, W, wj, wi, J, out);
  } else {
    k_ttm_mode<T, false><<<grid_for(work), kThreads, 0, st>>>(X, A, I, B, W, wj, wi, J, out);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t gram(const T* Z, const T* H, const Shape& zs, int n, int J, T* out, cudaStream_t st) {
  const long long A = zs.before(n), B = zs.after(n);
  const int I = (int)zs.dim[n];
  const long long warps = (long long)I * J;
  k_ttm_gram<T><<<grid_for(warps * 32), kThreads, 0, st>>>(Z, H, A, I, J, B, out);
  return cudaGetLastError();
}

struct Ctx {
  Shape full, core;
  int m = 0;
  long long M = 0;  // elements of each workspace buffer
};

bool make_ctx(const tucker_ttm_desc* d, Ctx* c) {
  if (!d || d->ndim < 1 || d->ndim > TUCKER_MAX_MODES) return false;
  if (d->dtype != TUCKER_F32 && d->dtype != TUCKER_F64) return false;
  c->m = d->ndim;
  c->full.m = c->core.m = d->ndim;
  long long N = 1;
  for (int k = 0; k < d->ndim; ++k) {
    if (d->n[k] < 1 || d->r[k] < 1 || d->r[k] > d->n[k] || d->n[k] > (1LL << 30)) return false;
    c->full.dim[k] = d->n[k];
    c->core.dim[k] = d->r[k];
    N *= d->n[k];
    if (N > (1LL << 40)) return false;
  }
  // every intermediate of the chains has at least one mode at its rank: at most N r_k / n_k
  long long M = 1;
  for (int k = 0; k < d->ndim; ++k) M = std::max(M, N / d->n[k] * d->r[k]);
  c->M = M;
  return true;
}

size_t buf_bytes(const Ctx& c, int tsize) { return ((size_t)c.M * tsize + 255) / 256 * 256; }

int64_t workspace(const Ctx& c, int tsize) { return (int64_t)(4 * buf_bytes(c, tsize)); }

template <typename T>
T* buf(void* work, const Ctx& c, int i) {
  return reinterpret_cast<T*>(static_cast<unsigned char*>(work) + (size_t)i * buf_bytes(c, sizeof(T)));
}

// projection of mode k: W = U_k^T (r_k x n_k) read from the column-major n_k x r_k factor
template <typename T>
cudaError_t proj_mode(const T* X, const Shape& s, int k, const T* U, long long nk, int rk, T* out,
                      cudaStream_t st) {
  return mode_product<T>(X, s, k, U, nk, 1, rk, out, st);
}
// reconstruction of mode k: W = U_k (n_k x r_k)
template <typename T>
cudaError_t expand_mode(const T* X, const Shape& s, int k, const T* U, long long nk, T* out,
                        cudaStream_t st) {
  return mode_product<T>(X, s, k, U, 1, nk, (int)nk, out, st);
}

// X (full shape) x_1 U_1^T ... x_m U_m^T -> out, through workspace buffers b0, b1.
template <typename T>
cudaError_t run_project(const Ctx& c, const T* const* U, const T* X, T* out, T* b0, T* b1,
                        cudaStream_t st) {
  Shape s = c.full;
  const T* cur = X;
  T* pp[2] = {b0, b1};
  for (int k = 0; k < c.m; ++k) {
    T* dst = (k == c.m - 1) ? out : pp[k & 1];
    cudaError_t e = proj_mode<T>(cur, s, k, U[k], c.full.dim[k], (int)c.core.dim[k], dst, st);
    if (e != cudaSuccess) return e;
    s.dim[k] = c.core.dim[k];
    cur = dst;
  }
  return cudaSuccess;
}

// G (core shape) x_1 U_1 ... x_m U_m -> out.
template <typename T>
cudaError_t run_reconstruct(const Ctx& c, const T* const* U, const T* G, T* out, T* b0, T* b1,
                            cudaStream_t st) {
  Shape s = c.core;
  const T* cur = G;
  T* pp[2] = {b0, b1};
  for (int k = 0; k < c.m; ++k) {
    T* dst = (k == c.m - 1) ? out : pp[k & 1];
    cudaError_t e = expand_mode<T>(cur, s, k, U[k], c.full.dim[k], dst, st);
    if (e != cudaSuccess) return e;
    s.dim[k] = c.full.dim[k];
    cur = dst;
  }
  return cudaSuccess;
}

// Factor gradients Ubar[n] = [X x_{k!=n} U_k^T]_(n) H_(n)^T for every requested n, and, if
// full_out is not NULL, the full projection X x_1 U_1^T ... x_m U_m^T into full_out.
template <typename T>
cudaError_t run_factor_grads(const Ctx& c, const T* const* U, const T* X, const T* H,
                             T* const* Ubar, T* full_out, void* work, cudaStream_t st) {
  T* P[2] = {buf<T>(work, c, 0), buf<T>(work, c, 1)};
  T* Cb[2] = {buf<T>(work, c, 2), buf<T>(work, c, 3)};
  int last_needed = -1;  // the prefix must advance through this mode
  for (int n = 0; n < c.m; ++n)
    if (Ubar && Ubar[n]) last_needed = n;
  const int prefix_end = full_out ? c.m : last_needed;  // modes applied to the prefix: [0, prefix_end)
  Shape ps = c.full;                                    // shape of the prefix
  const T* pref = X;
  for (int n = 0; n < c.m; ++n) {
    if (Ubar && Ubar[n]) {
      // Z = prefix x_{k>n} U_k^T
      Shape zs = ps;
      const T* z = pref;
      int pc = 0;
      for (int k = n + 1; k < c.m; ++k) {
        T* dst = Cb[pc];
        cudaError_t e = proj_mode<T>(z, zs, k, U[k], c.full.dim[k], (int)c.core.dim[k], dst, st);
        if (e != cudaSuccess) return e;
        zs.dim[k] = c.core.dim[k];
        z = dst;
        pc ^= 1;
      }
      cudaError_t e = gram<T>(z, H, zs, n, (int)c.core.dim[n], Ubar[n], st);
      if (e != cudaSuccess) return e;
    }
    if (n < prefix_end) {
      T* dst = (n == c.m - 1) ? full_out : P[n & 1];
      cudaError_t e = proj_mode<T>(pref, ps, n, U[n], c.full.dim[n], (int)c.core.dim[n], dst, st);
      if (e != cudaSuccess) return e;
      ps.dim[n] = c.core.dim[n];
      pref = dst;
    }
  }
  return cudaSuccess;
}

tucker_status check_common(const tucker_ttm_desc* d, const void* const* U, int64_t work_bytes,
                           const void* work, Ctx* c) {
  if (!make_ctx(d, c) || !U || !work) return TUCKER_EINVAL;
  for (int k = 0; k < c->m; ++k)
    if (!U[k]) return TUCKER_EINVAL;
  const int ts = d->dtype == TUCKER_F32 ? 4 : 8;
  if (work_bytes < workspace(*c, ts)) return TUCKER_EINVAL;
  if ((reinterpret_cast<uintptr_t>(work) & 255) != 0) return TUCKER_EINVAL;
  return TUCKER_OK;
}

tucker_status status_of(cudaError_t e) {
  if (e == cudaSuccess) return TUCKER_OK;
  fprintf(stderr, "tucker_ttm: %s\n", cudaGetErrorString(e));
  return TUCKER_ECUDA;
}

template <typename T>
const T* const* as_t(const void* const* p) {
  return reinterpret_cast<const T* const*>(p);
}

}  // namespace

extern "C" {

int64_t tucker_ttm_workspace_bytes(const tucker_ttm_desc* desc) {
  Ctx c;
  if (!make_ctx(desc, &c)) return -1;
  return workspace(c, desc->dtype == TUCKER_F32 ? 4 : 8);
}

tucker_status tucker_ttm_project(const tucker_ttm_desc* desc, const void* const* U_dev,
                                 const void* Y_dev, void* G_dev, void* work_dev,
                                 int64_t work_bytes, void* stream) {
  Ctx c;
  tucker_status rc = check_common(desc, U_dev, work_bytes, work_dev, &c);
  if (rc != TUCKER_OK || !Y_dev || !G_dev) return rc != TUCKER_OK ? rc : TUCKER_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (desc->dtype == TUCKER_F32)
    return status_of(run_project<float>(c, as_t<float>(U_dev), (const float*)Y_dev, (float*)G_dev,
                                        buf<float>(work_dev, c, 0), buf<float>(work_dev, c, 1), st));
  return status_of(run_project<double>(c, as_t<double>(U_dev), (const double*)Y_dev, (double*)G_dev,
                                       buf<double>(work_dev, c, 0), buf<double>(work_dev, c, 1), st));
}

tucker_status tucker_ttm_reconstruct(const tucker_ttm_desc* desc, const void* const* U_dev,
                                     const void* G_dev, void* Yhat_dev, void* work_dev,
                                     int64_t work_bytes, void* stream) {
  Ctx c;
  tucker_status rc = check_common(desc, U_dev, work_bytes, work_dev, &c);
  if (rc != TUCKER_OK || !G_dev || !Yhat_dev) return rc != TUCKER_OK ? rc : TUCKER_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (desc->dtype == TUCKER_F32)
    return status_of(run_reconstruct<float>(c, as_t<float>(U_dev), (const float*)G_dev, (float*)Yhat_dev,
                                            buf<float>(work_dev, c, 0), buf<float>(work_dev, c, 1), st));
  return status_of(run_reconstruct<double>(c, as_t<double>(U_dev), (const double*)G_dev,
                                           (double*)Yhat_dev, buf<double>(work_dev, c, 0),
                                           buf<double>(work_dev, c, 1), st));
}

tucker_status tucker_ttm_project_adjoint(const tucker_ttm_desc* desc, const void* const* U_dev,
                                         const void* Y_dev, const void* Gbar_dev, void* Ybar_dev,
                                         void* const* Ubar_dev, void* work_dev,
                                         int64_t work_bytes, void* stream) {
  Ctx c;
  tucker_status rc = check_common(desc, U_dev, work_bytes, work_dev, &c);
  if (rc != TUCKER_OK) return rc;
  if (!Y_dev || !Gbar_dev) return TUCKER_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (desc->dtype == TUCKER_F32) {
    if (Ybar_dev)
      e = run_reconstruct<float>(c, as_t<float>(U_dev), (const float*)Gbar_dev, (float*)Ybar_dev,
                                 buf<float>(work_dev, c, 0), buf<float>(work_dev, c, 1), st);
    if (e == cudaSuccess && Ubar_dev)
      e = run_factor_grads<float>(c, as_t<float>(U_dev), (const float*)Y_dev, (const float*)Gbar_dev,
                                  reinterpret_cast<float* const*>(Ubar_dev), nullptr, work_dev, st);
  } else {
    if (Ybar_dev)
      e = run_reconstruct<double>(c, as_t<double>(U_dev), (const double*)Gbar_dev, (double*)Ybar_dev,
                                  buf<double>(work_dev, c, 0), buf<double>(work_dev, c, 1), st);
    if (e == cudaSuccess && Ubar_dev)
      e = run_factor_grads<double>(c, as_t<double>(U_dev), (const double*)Y_dev,
                                   (const double*)Gbar_dev, reinterpret_cast<double* const*>(Ubar_dev),
                                   nullptr, work_dev, st);
  }
  return status_of(e);
}

tucker_status tucker_ttm_reconstruct_adjoint(const tucker_ttm_desc* desc,
                                             const void* const* U_dev, const void* G_dev,
                                             const void* Yhbar_dev, void* Gbar_dev,
                                             void* const* Ubar_dev, void* work_dev,
                                             int64_t work_bytes, void* stream) {
  Ctx c;
  tucker_status rc = check_common(desc, U_dev, work_bytes, work_dev, &c);
  if (rc != TUCKER_OK) return rc;
  if (!G_dev || !Yhbar_dev) return TUCKER_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (desc->dtype == TUCKER_F32)
    e = run_factor_grads<float>(c, as_t<float>(U_dev), (const float*)Yhbar_dev, (const float*)G_dev,
                                reinterpret_cast<float* const*>(Ubar_dev), (float*)Gbar_dev, work_dev, st);
  else
    e = run_factor_grads<double>(c, as_t<double>(U_dev), (const double*)Yhbar_dev, (const double*)G_dev,
                                 reinterpret_cast<double* const*>(Ubar_dev), (double*)Gbar_dev,
                                 work_dev, st);
  return status_of(e);
}

}  // extern "C"
