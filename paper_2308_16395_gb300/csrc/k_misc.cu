// Layout conversions between the paper's column-major tensors and the device state layout, and
// the streaming-mode contraction of the reconstruction.
#include "common.cuh"
#include "kernels.cuh"

namespace tk {

// After the batch ST-HOSVD: Ccol is the core as a column-major (R x r_d) array (C_(d)^T).
// State: C[j*ls + i] = C(j, i), V[j*ls + i] = C(j, i) / S_i (V_(d) = S^-1 C_(d), Assumption
// 1(c)), ls = tk_cv_stride(r_d); S_i = sqrt(lambda_i) of the streaming-mode Gram; U_d row-major
// (ld ldc) from Utmp (nt x r_d, column-major).
template <typename TW>
__global__ void k_init_finish(const TW* Ccol, long long R, int rd, const double* lam,
                              const double* Utmp, int nt, TW* C, TW* V, double* Ud, double* S,
                              int ldc) {
  const int ls = tk_cv_stride(rd, ldc, (int)sizeof(TW));
  const long long total = R * rd;
  for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < total;
       L += (long long)gridDim.x * blockDim.x) {
    const long long j = L % R;
    const int i = (int)(L / R);
    const TW c = Ccol[L];
    const double s = sqrt(fmax(lam[i], 0.0));
    C[j * ls + i] = c;
    V[j * ls + i] = (TW)((double)c / s);
  }
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < rd; i += blockDim.x) S[i] = sqrt(fmax(lam[i], 0.0));
    for (int L = threadIdx.x; L < nt * rd; L += blockDim.x) {
      const int t = L % nt, c = L / nt;
      Ud[(long long)t * ldc + c] = Utmp[L];
    }
  }
}

// Mixed form: C and V of the initial state from C_(d)^T = C*_{d-1} U_d computed in FP64 (C64,
// column-major R x rd). V = C_(d)^T U S^-1 is then orthonormal to FP64 accuracy before it is
// stored in FP32; from an FP32 product its weak columns (small S) would carry errors of about
// u_fp32 S_1 / S_c, and the incremental SVD needs V orthonormal well below q / ||d||.
template <typename TW>
__global__ void k_init_cv64(const double* C64, long long R, int rd, const double* lam, TW* C, TW* V,
                            int ldc) {
  const int ls = tk_cv_stride(rd, ldc, (int)sizeof(TW));
  const long long total = R * rd;
  for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < total;
       L += (long long)gridDim.x * blockDim.x) {
    const long long j = L % R;
    const int i = (int)(L / R);
    const double c = C64[L];
    const double s = sqrt(fmax(lam[i], 0.0));
    C[j * ls + i] = (TW)c;
    V[j * ls + i] = (TW)(c / s);
  }
}

template <typename TW>
cudaError_t launch_init_cv64(const double* C64, long long R, int rd, const double* lam, void* C,
                             void* V, int ldc, cudaStream_t st) {
  const long long total = R * rd;
  int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 8);
  if (grid < 1) grid = 1;
  k_init_cv64<TW><<<grid, 256, 0, st>>>(C64, R, rd, lam, (TW*)C, (TW*)V, ldc);
  return cudaGetLastError();
}
template cudaError_t launch_init_cv64<float>(const double*, long long, int, const double*, void*,
                                             void*, int, cudaStream_t);

template <typename TW>
cudaError_t launch_init_finish(Ctl* ctl, const void* Ccol, long long R, int rd, const double* lam,
                               const double* Utmp, int nt, void* C, void* V, double* Ud, double* S,
                               int ldc, cudaStream_t st) {
  (void)ctl;
  const long long total = R * rd;
  int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 8);
  if (grid < 1) grid = 1;
  k_init_finish<TW><<<grid, 256, 0, st>>>((const TW*)Ccol, R, rd, lam, Utmp, nt, (TW*)C, (TW*)V,
                                          Ud, S, ldc);
  return cudaGetLastError();
}

// out(j, t) = sum_i C(j, i) U_d(t0 + t, i): the core contracted with rows of U_d, as a
// column-major (R x T) array (the first step of X^ = C x_d U_d x_{d-1} ... x_1 U_1). C rows have
// stride tk_cv_stride(r_d), U_d rows stride ldc.
template <typename TW>
__global__ void k_core_times_ud(const TW* C, long long R, int rd, int ldc, const double* Ud,
                                long long t0, long long T, TW* out) {
  const int ls = tk_cv_stride(rd, ldc, (int)sizeof(TW));
  const long long total = R * T;
  for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < total;
       L += (long long)gridDim.x * blockDim.x) {
    const long long j = L % R, t = L / R;
    const TW* row = C + j * ls;
    const double* u = Ud + (t0 + t) * ldc;
    double s = 0.0;
    for (int i = 0; i < rd; ++i) s += (double)row[i] * u[i];
    out[L] = (TW)s;
  }
}

template <typename TW>
cudaError_t launch_core_times_ud(const void* C, long long R, int rd, int ldc, const double* Ud,
                                 long long t0, long long T, void* out, cudaStream_t st) {
  const long long total = R * T;
  int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 8);
  if (grid < 1) grid = 1;
  k_core_times_ud<TW><<<grid, 256, 0, st>>>((const TW*)C, R, rd, ldc, Ud, t0, T, (TW*)out);
  return cudaGetLastError();
}

// Rows (R x rd, row stride ldc, type TW) -> FP64 column-major (R x rd). For the C and V state the
// caller passes tk_cv_stride(r_d) as the stride.
template <typename TW>
__global__ void k_state_to_col(const TW* Src, long long R, int rd, int ldc, double* dst) {
  const long long total = R * rd;
  for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < total;
       L += (long long)gridDim.x * blockDim.x) {
    const long long j = L % R;
    const int i = (int)(L / R);
    dst[L] = (double)Src[j * ldc + i];
  }
}

template <typename TW>
cudaError_t launch_state_to_colmajor(const void* Src, long long R, int rd, int ldc, double* dst,
                                     cudaStream_t st) {
  const long long total = R * rd;
  int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 8);
  if (grid < 1) grid = 1;
  k_state_to_col<TW><<<grid, 256, 0, st>>>((const TW*)Src, R, rd, ldc, dst);
  return cudaGetLastError();
}

cudaError_t launch_ud_to_colmajor(const double* Ud, int nd, int rd, int ldc, double* dst,
                                  cudaStream_t st) {
  return launch_state_to_colmajor<double>(Ud, nd, rd, ldc, dst, st);
}

// Graph form of the update: the slice's TMA descriptor and address, passed as kernel parameters,
// written into the control block's slot (a kernel rather than a host-to-device copy, so that the
// write never queues behind a large slice transfer on a copy engine).
__global__ void k_set_slot(Ctl* ctl, const __grid_constant__ SlotArgs a) {
  const int t = threadIdx.x;
  if (t < 32) reinterpret_cast<unsigned*>(ctl->ymap)[t] = a.map[t];
  if (t == 32) ctl->yptr = a.y;
  // the descriptor is read by the tensor-map proxy of later kernels (which acquire it)
  asm volatile("fence.proxy.tensormap::generic.release.gpu;" ::: "memory");
}

cudaError_t launch_set_slot(Ctl* ctl, const SlotArgs& a, cudaStream_t st) {
  k_set_slot<<<1, 64, 0, st>>>(ctl, a);
  return cudaGetLastError();
}

__global__ void k_read_err(const Ctl* ctl, double* out2) {
  if (threadIdx.x == 0) {
    out2[0] = ctl->err2;
    out2[1] = ctl->data2;
    __threadfence_system();
  }
}

cudaError_t launch_read_err(const Ctl* ctl, double* out2, cudaStream_t st) {
  k_read_err<<<1, 32, 0, st>>>(ctl, out2);
  return cudaGetLastError();
}

template cudaError_t launch_init_finish<float>(Ctl*, const void*, long long, int, const double*,
                                               const double*, int, void*, void*, double*, double*,
                                               int, cudaStream_t);
template cudaError_t launch_init_finish<double>(Ctl*, const void*, long long, int, const double*,
                                                const double*, int, void*, void*, double*, double*,
                                                int, cudaStream_t);
template cudaError_t launch_core_times_ud<float>(const void*, long long, int, int, const double*,
                                                 long long, long long, void*, cudaStream_t);
template cudaError_t launch_core_times_ud<double>(const void*, long long, int, int, const double*,
                                                  long long, long long, void*, cudaStream_t);
template cudaError_t launch_state_to_colmajor<float>(const void*, long long, int, int, double*,
                                                     cudaStream_t);
template cudaError_t launch_state_to_colmajor<double>(const void*, long long, int, int, double*,
                                                      cudaStream_t);

}  // namespace tk

namespace tk {

// out(i, c) = sum_j A(i, j) B(j, c) in FP64 for the small products of the re-compression
// (U_k Q_k and U_d Q_d): A(i, j) at A[i * as_i + j * as_j], B column-major (ldb), out(i, c) at
// out[i * os_i + c * os_c]; outw (may be NULL) receives the same values in FP32. One thread per
// entry (rows x cols is at most n_k x r_k).
__global__ void k_small_gemm(const double* __restrict__ A, long long as_i, long long as_j,
                             int rows, int inner, const double* __restrict__ B, long long bs_j,
                             long long bs_c, int cols, double* __restrict__ out, long long os_i,
                             long long os_c, float* __restrict__ outw) {
  const long long total = (long long)rows * cols;
  for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < total;
       L += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(L % rows), c = (int)(L / rows);
    double s = 0.0;
    for (int j = 0; j < inner; ++j) s = fma(A[i * as_i + j * as_j], B[c * bs_c + j * bs_j], s);
    out[i * os_i + c * os_c] = s;
    if (outw) outw[i * os_i + c * os_c] = (float)s;
  }
}

cudaError_t launch_small_gemm(const double* A, long long as_i, long long as_j, int rows, int inner,
                              const double* B, int ldb, int cols, double* out, long long os_i,
                              long long os_c, float* outw, cudaStream_t st) {
  return launch_gemm64(A, as_i, as_j, rows, inner, B, 1, ldb, cols, out, os_i, os_c, outw, st);
}

cudaError_t launch_gemm64(const double* A, long long as_i, long long as_j, int rows, int inner,
                          const double* B, long long bs_j, long long bs_c, int cols, double* out,
                          long long os_i, long long os_c, float* outw, cudaStream_t st) {
  const long long total = (long long)rows * cols;
  int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 4);
  if (grid < 1) grid = 1;
  k_small_gemm<<<grid, 256, 0, st>>>(A, as_i, as_j, rows, inner, B, bs_j, bs_c, cols, out, os_i,
                                     os_c, outw);
  return cudaGetLastError();
}

// T = (3 I - G) / 2 (r x r, column-major): one Newton-Schulz step towards the polar factor.
__global__ void k_ns_matrix(const double* __restrict__ G, int r, double* __restrict__ T) {
  for (int L = blockIdx.x * blockDim.x + threadIdx.x; L < r * r; L += gridDim.x * blockDim.x)
    T[L] = (L % (r + 1) == 0 ? 1.5 : 0.0) - 0.5 * G[L];
}

// part[b]: block b's share of ||G - I||_F^2 (G r x r column-major).
__global__ void k_frob_minus_i(const double* __restrict__ G, int r, double* __restrict__ part) {
  __shared__ double red[32];
  double a = 0.0;
  for (int L = blockIdx.x * blockDim.x + threadIdx.x; L < r * r; L += gridDim.x * blockDim.x) {
    const double v = G[L] - (L % (r + 1) == 0 ? 1.0 : 0.0);
    a = fma(v, v, a);
  }
  a = block_sum(a, red);
  if (threadIdx.x == 0) part[blockIdx.x] = a;
}

// part[b]: block b's share of sum_t sum_c ((U1 - U0)(t, c) S(c))^2, U row-major rows x ld.
__global__ void k_change_norm(const double* __restrict__ U1, const double* __restrict__ U0,
                              int rows, int r, int ld, const double* __restrict__ S,
                              double* __restrict__ part) {
  __shared__ double red[32];
  double a = 0.0;
  const long long total = (long long)rows * r;
  for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < total;
       L += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(L / r), c = (int)(L % r);
    const double v = (U1[(long long)t * ld + c] - U0[(long long)t * ld + c]) * S[c];
    a = fma(v, v, a);
  }
  a = block_sum(a, red);
  if (threadIdx.x == 0) part[blockIdx.x] = a;
}

cudaError_t launch_ns_matrix(const double* G, int r, double* T, cudaStream_t st) {
  k_ns_matrix<<<std::max(1, std::min(256, (r * r + 255) / 256)), 256, 0, st>>>(G, r, T);
  return cudaGetLastError();
}
cudaError_t launch_frob_minus_i(const double* G, int r, double* part, int nparts, cudaStream_t st) {
  k_frob_minus_i<<<nparts, 256, 0, st>>>(G, r, part);
  return cudaGetLastError();
}
cudaError_t launch_change_norm(const double* U1, const double* U0, int rows, int r, int ld,
                               const double* S, double* part, int nparts, cudaStream_t st) {
  k_change_norm<<<nparts, 256, 0, st>>>(U1, U0, rows, r, ld, S, part);
  return cudaGetLastError();
}

// C and V state rows (stride ld, type TW) from FP64 column-major R x rd arrays.
template <typename TW>
__global__ void k_set_cv(const double* C64, const double* V64, long long R, int rd, TW* C, TW* V,
                         int ld) {
  const long long total = R * rd;
  for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < total;
       L += (long long)gridDim.x * blockDim.x) {
    const long long j = L % R;
    const int i = (int)(L / R);
    C[j * ld + i] = (TW)C64[L];
    V[j * ld + i] = (TW)V64[L];
  }
}

template <typename TW>
cudaError_t launch_set_cv(const double* C64, const double* V64, long long R, int rd, void* C,
                          void* V, int ld, cudaStream_t st) {
  const long long total = R * rd;
  int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 8);
  if (grid < 1) grid = 1;
  k_set_cv<TW><<<grid, 256, 0, st>>>(C64, V64, R, rd, (TW*)C, (TW*)V, ld);
  return cudaGetLastError();
}
template cudaError_t launch_set_cv<float>(const double*, const double*, long long, int, void*,
                                          void*, int, cudaStream_t);
template cudaError_t launch_set_cv<double>(const double*, const double*, long long, int, void*,
                                           void*, int, cudaStream_t);

}  // namespace tk
