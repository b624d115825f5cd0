/*
 * tucker_ttm.h -- C ABI of the Tucker projection and reconstruction chains and of their adjoints.
 *
 * Definitions (Sec. 2.1: the mode-k product X x_k A with (X x_k A)_(k) = A X_(k); Sec. 2.2: the
 * Tucker model and its Kronecker form X_(k) = U_k C_(k) (U_m (x) ... (x) U_{k+1} (x) U_{k-1}
 * (x) ... (x) U_1)^T):
 *
 *   projection      G  = Y x_1 U_1^T x_2 U_2^T ... x_m U_m^T     (r_1 x ... x r_m)
 *   reconstruction  Y^ = G x_1 U_1 x_2 U_2 ... x_m U_m           (n_1 x ... x n_m)
 *
 * and, for a scalar loss L with upstream gradients Gbar = dL/dG or Yhbar = dL/dY^, the adjoints
 *
 *   projection:      dL/dY = Gbar x_1 U_1 ... x_m U_m,   dL/dU_n = [Y x_{k!=n} U_k^T]_(n) Gbar_(n)^T
 *   reconstruction:  dL/dG = Yhbar x_1 U_1^T ... x_m U_m^T,
 *                    dL/dU_n = [Yhbar x_{k!=n} U_k^T]_(n) G_(n)^T
 *
 * The factors are unconstrained matrices here (Euclidean gradients). The adjoints recompute the
 * partial products Y x_{k!=n} U_k^T from their inputs (sharing the prefix x_1 .. x_{n-1} between
 * modes) instead of keeping the forward chain's intermediates.
 *
 * Layouts: every tensor is dense column-major (mode 1 fastest, Sec. 2.1); U_k is column-major
 * n_k x r_k (leading dimension n_k); dL/dU_k is written in the same layout. All tensors and
 * factors of one call have the element type desc->dtype. Pointers named *_dev are device
 * pointers on the current device; `U_dev` and `Ubar_dev` are HOST arrays of desc->ndim device
 * pointers. `stream` is a cudaStream_t (NULL = legacy default stream).
 *
 * Workspace: each call takes a caller-owned device buffer `work_dev` of at least
 * tucker_ttm_workspace_bytes(desc) bytes (256-byte aligned); the calls allocate nothing. Calls on
 * different streams need different workspaces.
 *
 * Ownership and errors: the caller owns every buffer; inputs are only read. A bad descriptor, a
 * NULL required pointer or a short workspace returns TUCKER_EINVAL before any device work; a
 * failed launch returns TUCKER_ECUDA. The calls are asynchronous on `stream` (no host
 * synchronization) and may be captured in a CUDA graph.
 */
#ifndef TUCKER_TTM_H
#define TUCKER_TTM_H

#include <stdint.h>

#include "tucker_stream.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t ndim;                      /* m, number of modes, 1..8 */
  int32_t dtype;                     /* TUCKER_F32 or TUCKER_F64 */
  int64_t n[TUCKER_MAX_MODES];       /* full sizes n_1..n_m, each >= 1 */
  int64_t r[TUCKER_MAX_MODES];       /* ranks r_1..r_m, 1 <= r_k <= n_k */
} tucker_ttm_desc;

/* Workspace bytes every call below needs for this descriptor, or -1 if the descriptor is
 * invalid. */
int64_t tucker_ttm_workspace_bytes(const tucker_ttm_desc* desc);

/* G = Y x_1 U_1^T ... x_m U_m^T. Y_dev: n_1 x ... x n_m; G_dev: r_1 x ... x r_m. */
tucker_status tucker_ttm_project(const tucker_ttm_desc* desc, const void* const* U_dev,
                                 const void* Y_dev, void* G_dev, void* work_dev,
                                 int64_t work_bytes, void* stream);

/* Y^ = G x_1 U_1 ... x_m U_m. G_dev: r_1 x ... x r_m; Yhat_dev: n_1 x ... x n_m. */
tucker_status tucker_ttm_reconstruct(const tucker_ttm_desc* desc, const void* const* U_dev,
                                     const void* G_dev, void* Yhat_dev, void* work_dev,
                                     int64_t work_bytes, void* stream);

/* Adjoint of the projection at (Y, U) for the upstream gradient Gbar (r_1 x ... x r_m):
 * Ybar_dev (n_1 x ... x n_m) = dL/dY and Ubar_dev[k] (n_k x r_k) = dL/dU_k. Ybar_dev may be
 * NULL, Ubar_dev may be NULL, and entries of Ubar_dev may be NULL: those outputs are skipped.
 * Outputs are overwritten, not accumulated. */
tucker_status tucker_ttm_project_adjoint(const tucker_ttm_desc* desc, const void* const* U_dev,
                                         const void* Y_dev, const void* Gbar_dev, void* Ybar_dev,
                                         void* const* Ubar_dev, void* work_dev,
                                         int64_t work_bytes, void* stream);

/* Adjoint of the reconstruction at (G, U) for the upstream gradient Yhbar (n_1 x ... x n_m):
 * Gbar_dev (r_1 x ... x r_m) = dL/dG and Ubar_dev[k] (n_k x r_k) = dL/dU_k. NULL outputs are
 * skipped as above; outputs are overwritten. */
tucker_status tucker_ttm_reconstruct_adjoint(const tucker_ttm_desc* desc,
                                             const void* const* U_dev, const void* G_dev,
                                             const void* Yhbar_dev, void* Gbar_dev,
                                             void* const* Ubar_dev, void* work_dev,
                                             int64_t work_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TUCKER_TTM_H */
