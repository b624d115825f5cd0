// Host-side launchers of the device kernels (one declaration per translation unit export).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"

namespace tk {

// ---- k_spatial.cu ----
size_t proj_smem_bytes(int r, int tw_size);
template <typename TX, typename TW>
cudaError_t launch_proj(const Ctl* ctl, int k, int out_off, int pred, const void* Xext,
                        void* const* dbufs, const void* U, int ldu, int rmax, double* part_e2,
                        double* part_y2, int grid, cudaStream_t st);
template <typename TX, typename TW>
cudaError_t launch_resid_gram(const Ctl* ctl, int k, int n, const void* Xext, void* const* dbufs,
                              const void* U, int ldu, double* gpart, int pairs, int chunks,
                              int data_only, cudaStream_t st);
cudaError_t launch_decide(Ctl* ctl, int k, const double* pe, const double* py, int nparts,
                          cudaGraphConditionalHandle hcond, cudaStream_t st);
cudaError_t launch_mode_end(Ctl* ctl, int k, int grown_only, cudaStream_t st);
cudaError_t launch_gram_reduce(const Ctl* ctl, int k, const double* gpart, int pairs, int chunks,
                               double* G, int data_only, cudaStream_t st);
template <typename TI, typename TW, typename TO>
cudaError_t launch_expand(const void* X, long long A, int r, long long B, const void* U, int ldu,
                          int n, void* out, cudaStream_t st);
template <typename TX>
cudaError_t launch_norm2(const void* X, long long N, double* part, int grid, cudaStream_t st);

// ---- k_eig.cu ----
template <typename TE>
cudaError_t launch_eig(Ctl* ctl, int k, int mode, const double* G, void* Aw, void* Z, void* LD,
                       double* W, double* lam, int mcap, int n, cudaStream_t st);
template <typename TW>
cudaError_t launch_append(Ctl* ctl, int k, int mode, const double* W, double* U, void* Uw, int ldu,
                          int n, cudaStream_t st);

// ---- k_eig_sub.cu ----
// Residual-Gram eigensolve of the mixed form (subspace iteration + FP64 Rayleigh-Ritz cut); sets
// ctl->eig_fb[k] when the full solver (launch_eig with mode 2) must decide instead.
cudaError_t launch_eig_sub(Ctl* ctl, int k, const double* G, void* Gf, double* W, int mcap,
                           double* part, int n, cudaStream_t st);
// FP64 Rayleigh-Ritz cut over the eigenvectors of the full FP32 solver (runs when it ran).
cudaError_t launch_eig_refine_post(Ctl* ctl, int k, const double* G, double* W, int mcap,
                                   double* part, int n, cudaStream_t st);

// ---- k_stream.cu ----
struct SecWork {
  double* delta;
  double* z;
  int* idx;
  double* tau;
  int* org;
  double* lam;
  int* lsrc;
  double* rot;
  int* nrot;
  double* V2;
  double* U2;
  double* sv;
  double* pq;
  int* meta;
};
template <typename TW>
cudaError_t launch_isvd(Ctl* ctl, void* const* dbufs, void* const* vbufs, double* part_p,
                        double* part_e, double* p, double* es, void* evec, const double* S,
                        SecWork w, int grid, cudaStream_t st);
cudaError_t launch_secular_vectors(Ctl* ctl, const double* S, SecWork w, double* Snew,
                                   cudaStream_t st);
template <typename TW>
cudaError_t launch_factor(Ctl* ctl, double* const* udbufs, SecWork w, const double* es, void* Bc,
                          void* cu, void* Bv, void* wv, int ldb, float* const* bsplit,
                          int grid_small, cudaStream_t st);
template <typename TW>
cudaError_t launch_cv(Ctl* ctl, void* const* dbufs, void* const* cbufs, void* const* vbufs,
                      SecWork w, const void* Bc, const void* cu, const void* Bv, const void* wv,
                      int ldb, const void* evec, int grid_cv, cudaStream_t st);
cudaError_t launch_begin(Ctl* ctl, cudaStream_t st, int blk = 1);
// block update (blk > 1): the projected slices as contiguous rows, then each row's turn
template <typename TW>
cudaError_t launch_block_rows(Ctl* ctl, void* const* dbufs, void* Dt, cudaStream_t st);
template <typename TW>
cudaError_t launch_row_begin(Ctl* ctl, int b, void* const* dbufs, const void* Dt, cudaStream_t st);
cudaError_t launch_end(Ctl* ctl, const double* Snew, double* S, cudaStream_t st);

// ---- k_tc.cu ----
struct TcMaps {
  CUtensorMap c0, c1, v0, v1;           // state buffers: rows x ldc FP32, box 32 x 128
  CUtensorMap bc_hi, bc_lo, bv_hi, bv_lo;  // B^T (N x K) TF32 splits, row stride 512, box 32 x 16
};
bool make_map_2d_f32(CUtensorMap* map, const void* base, long long rows, long long cols,
                     long long ld, int box_cols, int box_rows);
size_t tc_rowgemm_smem();
cudaError_t launch_tc_cv(Ctl* ctl, SecWork w, const TcMaps& maps, void* const* cbufs_host,
                         void* const* vbufs_host, void* const* d_cbufs, void* const* d_vbufs,
                         const void* cu, const void* wv, const void* evec, void* const* dbufs,
                         int ldc, int grid, cudaStream_t st);
struct TcProjMaps {
  CUtensorMap uhi, ulo;     // U_k TF32 splits, column-major n_k x cap (rows of B1 = columns of U)
  CUtensorMap urhi, urlo;   // U_k TF32 splits, row-major n_k x 64
  CUtensorMap d[3];         // the D* buffers viewed as row-major (rows x n_k), box 32 x 128
  CUtensorMap eta;          // E^T (n_k x Fs), box 32 x 128
  CUtensorMap h1hi, h1lo;   // FP16 parts of 2^14 U_k, 64 x n_k (row i = column i of U_k), box 64 x 16
  CUtensorMap h2hi, h2lo;   // FP16 parts of 2^14 U_k, n_k x 64 (row-major), box 64 x 64
};
cudaError_t launch_split_u(const Ctl* ctl, int k, int pred, const double* U, int ldu,
                           float* const* sp, cudaStream_t st);
// mode 0: projection only (pass C), 1: projection + residual norms (pass A),
// 2: residual E^T written to Et (pre-pass of the Gram, only when mode k grew).
cudaError_t launch_tc_proj(const Ctl* ctl, int k, int mode, int pred, const float* Y,
                           long long F0, int n0, const TcProjMaps& m, void* const* dbufs,
                           int out_off, double* part_e2, double* part_y2, int nparts, float* Et,
                           long long et_stride, int grid, cudaStream_t st);
// FP16-split pass of mode k (n_k <= TK_H16_NMAX), same modes and outputs as launch_tc_proj;
// rerun = 1: the second launch of pass A, which runs only when the first one's input fell outside
// the FP16 scale window.
cudaError_t launch_tc_pass16(Ctl* ctl, int k, int mode, int pred, int rerun, const float* Y,
                             long long F0, int n0, const TcProjMaps& m, void* const* dbufs,
                             int out_off, double* part_e2, double* part_y2, int nparts, float* Et,
                             long long et_stride, int grid, cudaStream_t st);
cudaError_t launch_split_u16(const Ctl* ctl, int k, int pred, const double* U, int ldu, int ld1,
                             void* const* u16, cudaStream_t st);
bool make_map_2d_f16(CUtensorMap* map, const void* base, long long rows, long long cols,
                     long long ld, int box_cols, int box_rows);
cudaError_t launch_tc_gram(const Ctl* ctl, int k, const TcProjMaps& m, int n1, double* gpart,
                           double* G, int nsm, cudaStream_t st);

// ---- k_misc.cu ----
struct SlotArgs {
  unsigned map[32];        // TMA descriptor of the slice (128 bytes)
  const void* y;           // slice address
};
cudaError_t launch_set_slot(Ctl* ctl, const SlotArgs& a, cudaStream_t st);
// (err^2, ||X||^2) of the control block stored by one GPU thread into memory the GPU can address
// (mapped pinned host memory, managed or device memory): no copy engine involved.
cudaError_t launch_read_err(const Ctl* ctl, double* out2, cudaStream_t st);
template <typename TW>
cudaError_t launch_init_finish(Ctl* ctl, const void* Ccol, long long R, int rd, const double* lam,
                               const double* Utmp, int nt, void* C, void* V, double* Ud, double* S,
                               int ldc, cudaStream_t st);
template <typename TW>
cudaError_t launch_init_cv64(const double* C64, long long R, int rd, const double* lam, void* C,
                             void* V, int ldc, cudaStream_t st);
// out(i, c) = sum_j A[i as_i + j as_j] B[j bs_j + c bs_c] (FP64), written at i os_i + c os_c, and
// in FP32 to outw at the same offsets when outw is not NULL.
cudaError_t launch_gemm64(const double* A, long long as_i, long long as_j, int rows, int inner,
                          const double* B, long long bs_j, long long bs_c, int cols, double* out,
                          long long os_i, long long os_c, float* outw, cudaStream_t st);
cudaError_t launch_ns_matrix(const double* G, int r, double* T, cudaStream_t st);
cudaError_t launch_frob_minus_i(const double* G, int r, double* part, int nparts, cudaStream_t st);
cudaError_t launch_change_norm(const double* U1, const double* U0, int rows, int r, int ld,
                               const double* S, double* part, int nparts, cudaStream_t st);
cudaError_t launch_small_gemm(const double* A, long long as_i, long long as_j, int rows, int inner,
                              const double* B, int ldb, int cols, double* out, long long os_i,
                              long long os_c, float* outw, cudaStream_t st);
template <typename TW>
cudaError_t launch_set_cv(const double* C64, const double* V64, long long R, int rd, void* C,
                          void* V, int ld, cudaStream_t st);
template <typename TW>
cudaError_t launch_core_times_ud(const void* C, long long R, int rd, int ldc, const double* Ud,
                                 long long t0, long long T, void* out, cudaStream_t st);
template <typename TW>
cudaError_t launch_state_to_colmajor(const void* Src, long long R, int rd, int ldc, double* dst,
                                     cudaStream_t st);
cudaError_t launch_ud_to_colmajor(const double* Ud, int nd, int rd, int ldc, double* dst,
                                  cudaStream_t st);

}  // namespace tk
