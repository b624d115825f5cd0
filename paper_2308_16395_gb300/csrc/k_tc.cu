// Tensor-core (tcgen05 + TMA) kernels of the mixed form.
//
// k_tc_rowgemm: Out[j, 0:N] = In[j, 0:K] B + x[j] c for every row j of the state (the core
// update C~ = C M^T + d u^T of Alg. 5 and V~ = V' V'' of Alg. 3, Sec. 3.4). In rows stream through
// shared memory by TMA (128 rows x 32 FP32 per stage, 128-byte swizzle); B^T (N x K) is split
// once per update into TF32 high/low parts and kept resident in shared memory; each 32-wide K chunk
// issues 3 MMAs per K step of 8 (hi*hi + hi*lo + lo*hi, "3xTF32"), accumulating in FP32 in tensor
// memory. The A low part is produced on chip by converter warps. The kernel is persistent: one CTA
// per SM loops over 128-row tiles with two TMEM accumulators, so the epilogue of one tile overlaps
// the loads and MMAs of the next.
//
// Warp roles (256 threads): warp 0 TMA producer, warp 1 TMEM owner + MMA issuer, warps 2-3 A
// splitters, warps 4-7 epilogue (TMEM lanes 0-127 = the tile's rows).
#include "common.cuh"
#include "kernels.cuh"
#include "tc_common.cuh"

namespace tk {

using namespace tc;

constexpr int TC_M = 128;        // rows per tile
constexpr int TC_S = 2;          // pipeline stages
constexpr int TC_BROWS = 16;     // rows of B^T per TMA box
constexpr int TC_STAGE_BYTES = 2 * TC_M * TC_KC * 4;  // hi + lo of one A stage
constexpr size_t TC_SMEM = (size_t)TC_S * TC_STAGE_BYTES + TC_BRES_BYTES + 1024 + 256;

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait (1 s of wall time), sets *abort on timeout.
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  for (long long i = 0;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63) == 63) {
      if (*abort) return false;
      if (gtimer() - t0 > 1000000000ull) { *abort = 1; return false; }
    }
  }
}

// Zero-padded expansion of the old C and V rows into the new spatial layout (PadWithZeros of
// Alg. 4), written into the other buffer, only when a spatial rank grew and the tensor-core path
// runs (the tensor-core kernel reads contiguous rows through TMA).
__global__ void __launch_bounds__(256) k_cv_expand(const Ctl* __restrict__ ctl, const SecWork w,
                                                  float* const* cbufs, float* const* vbufs) {
  if (ctl->status) return;
  if (!tc_cv_ok(ctl, w.meta[2]) || !spatial_grew(ctl)) return;
  const int d = ctl->d, m = d - 1;
  const int r = ctl->r[d - 1];
  const int ldc = ctl->ldc;
  long long Rn = 1;
  for (int i = 0; i < m; ++i) Rn *= ctl->r[i];
  const float* Ci = cbufs[ctl->cbuf];
  const float* Vi = vbufs[ctl->cbuf];
  float* Co = cbufs[ctl->cbuf ^ 1];
  float* Vo = vbufs[ctl->cbuf ^ 1];
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long j = gw; j < Rn; j += nw) {
    const long long jo = tk_map_new_to_old(j, ctl->r, ctl->rold, m);
    for (int c = lane; c < r; c += 32) {
      Co[j * ldc + c] = jo >= 0 ? Ci[jo * ldc + c] : 0.f;
      Vo[j * ldc + c] = jo >= 0 ? Vi[jo * ldc + c] : 0.f;
    }
  }
}

struct TcRowGemmArgs {
  float* buf0;          // the two state buffers (also the A tensor maps' bases)
  float* buf1;
  const float* cvec;    // rank-1 column vector (N)
  const float* xvec;    // rank-1 row vector (rows); nullptr: D*_{d-1} in dbufs[xbuf]
  float* const* dbufs;
  int ldc;
};

__global__ void __launch_bounds__(256, 1) k_tc_rowgemm(Ctl* ctl, const SecWork w,
                                                      const __grid_constant__ CUtensorMap mA0,
                                                      const __grid_constant__ CUtensorMap mA1,
                                                      const __grid_constant__ CUtensorMap mBhi,
                                                      const __grid_constant__ CUtensorMap mBlo,
                                                      TcRowGemmArgs a) {
  if (ctl->status) return;
  const int keep = w.meta[2];
  if (!tc_cv_ok(ctl, keep)) return;
  const int d = ctl->d;
  const int K = ctl->r[d - 1];
  const int Kc = (K + TC_KC - 1) / TC_KC;
  const int Np = (keep + 15) / 16 * 16;
  long long Rn = 1;
  for (int i = 0; i < d - 1; ++i) Rn *= ctl->r[i];
  const bool grown = spatial_grew(ctl);
  const int inb = grown ? (ctl->cbuf ^ 1) : ctl->cbuf;
  const CUtensorMap* mA = inb ? &mA1 : &mA0;
  float* out = (inb ? a.buf0 : a.buf1);
  const float* X = a.xvec ? a.xvec : a.dbufs[ctl->xbuf];
  const long long ntiles = (Rn + TC_M - 1) / TC_M;

  extern __shared__ __align__(1024) unsigned char tsm_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(tsm_raw) + 1023) & ~uintptr_t(1023));
  float* Ast = reinterpret_cast<float*>(base);                              // [S][2][M*KC]
  float* Bhi = reinterpret_cast<float*>(base + TC_S * TC_STAGE_BYTES);      // [Kc][Np*KC]
  float* Blo = Bhi + (size_t)Kc * Np * TC_KC;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + TC_S * TC_STAGE_BYTES + TC_BRES_BYTES);
  uint64_t* full = bars;
  uint64_t* conv = bars + TC_S;
  uint64_t* empty = bars + 2 * TC_S;
  uint64_t* accfull = bars + 3 * TC_S;
  uint64_t* accempty = accfull + 2;
  uint64_t* bload = accempty + 2;
  uint64_t* done = bload + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], 64);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accfull[b], 1);
      mbar_init(&accempty[b], 128);
    }
    mbar_init(bload, 1);
    mbar_init(done, 1);
    *abort = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
    // ---------------- TMA producer (one thread; lanes 1-31 idle) ----------------
    tma_prefetch(mA);
    tma_prefetch(&mBhi);
    tma_prefetch(&mBlo);
    const uint32_t bbytes = (uint32_t)Kc * Np * TC_KC * 4 * 2;
    mbar_arrive_expect_tx(bload, bbytes);
    for (int kc = 0; kc < Kc; ++kc)
      for (int n0 = 0; n0 < Np; n0 += TC_BROWS) {
        tma_load_2d(&mBhi, bload, Bhi + ((size_t)kc * Np + n0) * TC_KC, kc * TC_KC, n0);
        tma_load_2d(&mBlo, bload, Blo + ((size_t)kc * Np + n0) * TC_KC, kc * TC_KC, n0);
      }
    long long q = 0;
    for (long long t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
      for (int kc = 0; kc < Kc; ++kc, ++q) {
        const int s = (int)(q % TC_S);
        const uint32_t ph = (uint32_t)((q / TC_S) & 1);
        if (!wait_bar(&empty[s], ph ^ 1, abort)) break;
        mbar_arrive_expect_tx(&full[s], TC_M * TC_KC * 4);
        tma_load_2d(mA, &full[s], Ast + (size_t)s * 2 * TC_M * TC_KC, kc * TC_KC, (int)(t * TC_M));
      }
    }
    // drain: wait until the last issued stages were consumed before leaving
    for (long long j = (q > TC_S ? q - TC_S : 0); j < q; ++j) {
      const int s = (int)(j % TC_S);
      wait_bar(&empty[s], (uint32_t)((j / TC_S) & 1), abort);
    }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(TC_M, Np);
      bool ok = wait_bar(bload, 0, abort);
      long long q = 0;
      int it = 0;
      for (long long t = blockIdx.x; ok && t < ntiles; t += gridDim.x, ++it) {
        const int b = it & 1;
        if (!wait_bar(&accempty[b], (uint32_t)(((it >> 1) & 1) ^ 1), abort)) break;
        tc_fence_after();
        const uint32_t dt = tmem + (uint32_t)(b * 256);
        for (int kc = 0; kc < Kc; ++kc, ++q) {
          const int s = (int)(q % TC_S);
          if (!wait_bar(&conv[s], (uint32_t)((q / TC_S) & 1), abort)) { ok = false; break; }
          tc_fence_after();
          const uint64_t ahi = desc_sw128(Ast + (size_t)s * 2 * TC_M * TC_KC);
          const uint64_t alo = desc_sw128(Ast + (size_t)s * 2 * TC_M * TC_KC + TC_M * TC_KC);
          const uint64_t bhi = desc_sw128(Bhi + (size_t)kc * Np * TC_KC);
          const uint64_t blo = desc_sw128(Blo + (size_t)kc * Np * TC_KC);
#pragma unroll
          for (int k4 = 0; k4 < TC_KC / 8; ++k4) {
            const uint64_t o = (uint64_t)(k4 * 32) >> 4;   // 8 TF32 = 32 bytes per K step
            mma_tf32(dt, ahi + o, bhi + o, idesc, (kc | k4) ? 1u : 0u);
            mma_tf32(dt, ahi + o, blo + o, idesc, 1u);
            mma_tf32(dt, alo + o, bhi + o, idesc, 1u);
          }
          tc_commit(&empty[s]);
        }
        if (!ok) break;
        tc_commit(&accfull[b]);
      }
      tc_commit(done);
      wait_bar(done, 0, abort);
    }
    __syncwarp();
  } else if (warp == 2 || warp == 3) {
    // ---------------- A splitters: hi = tf32(a) in place, lo = a - hi ----------------
    const int ct = threadIdx.x - 64;   // 0..63
    long long q = 0;
    for (long long t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
      for (int kc = 0; kc < Kc; ++kc, ++q) {
        const int s = (int)(q % TC_S);
        if (!wait_bar(&full[s], (uint32_t)((q / TC_S) & 1), abort)) break;
        float4* hi = reinterpret_cast<float4*>(Ast + (size_t)s * 2 * TC_M * TC_KC);
        float4* lo = hi + TC_M * TC_KC / 4;
#pragma unroll 4
        for (int i = ct; i < TC_M * TC_KC / 4; i += 64) {
          float4 v = hi[i], h, l;
          tf32_split(v.x, h.x, l.x);
          tf32_split(v.y, h.y, l.y);
          tf32_split(v.z, h.z, l.z);
          tf32_split(v.w, h.w, l.w);
          hi[i] = h;
          lo[i] = l;
        }
        fence_proxy_async_smem();
        mbar_arrive(&conv[s]);
      }
      if (*abort) break;
    }
  } else if (warp >= 4 && warp < 8) {
    // ---------------- epilogue: TMEM -> registers -> + x_j c -> global (full warps only) ----
    const int wq = warp - 4;   // TMEM lane quarter
    int it = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      const int b = it & 1;
      bool okw = wait_bar(&accfull[b], (uint32_t)((it >> 1) & 1), abort);
      okw = __all_sync(0xffffffffu, okw);
      if (!okw) break;
      tc_fence_after();
      const long long row = t * TC_M + wq * 32 + lane;
      const bool live = row < Rn;
      const float xj = live ? X[row] : 0.f;
      float* orow = out + row * a.ldc;
      for (int c0 = 0; c0 < Np; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)(b * 256 + c0), v);
        if (live) {
          if (c0 + 32 <= keep) {
#pragma unroll
            for (int i = 0; i < 32; i += 4) {
              float4 o;
              o.x = v[i] + xj * a.cvec[c0 + i];
              o.y = v[i + 1] + xj * a.cvec[c0 + i + 1];
              o.z = v[i + 2] + xj * a.cvec[c0 + i + 2];
              o.w = v[i + 3] + xj * a.cvec[c0 + i + 3];
              *reinterpret_cast<float4*>(orow + c0 + i) = o;
            }
          } else {
            for (int i = 0; i < 32 && c0 + i < keep; ++i) orow[c0 + i] = v[i] + xj * a.cvec[c0 + i];
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&accempty[b]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, 512);
  if (threadIdx.x == 0 && *abort) ctl->status = 5;   // TUCKER_ETIMEOUT
}

// ---------------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2D FP32 row-major matrix (rows x cols, row stride ld elements), box (box_cols x box_rows),
// 128-byte swizzle, out-of-range elements read as zero.
bool make_map_2d_f32(CUtensorMap* map, const void* base, long long rows, long long cols,
                     long long ld, int box_cols, int box_rows) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// 2D FP16 row-major matrix (rows x cols, row stride ld elements, a multiple of 8), box
// (box_cols x box_rows), 128-byte swizzle, out-of-range elements read as zero.
bool make_map_2d_f16(CUtensorMap* map, const void* base, long long rows, long long cols,
                     long long ld, int box_cols, int box_rows) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

size_t tc_rowgemm_smem() { return TC_SMEM; }

cudaError_t launch_tc_cv(Ctl* ctl, SecWork w, const TcMaps& maps, void* const* cbufs_host,
                         void* const* vbufs_host, void* const* d_cbufs, void* const* d_vbufs,
                         const void* cu, const void* wv, const void* evec, void* const* dbufs,
                         int ldc, int grid, cudaStream_t st) {
  k_cv_expand<<<152 * 4, 256, 0, st>>>(ctl, w, (float* const*)d_cbufs, (float* const*)d_vbufs);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tc_rowgemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
    attr = true;
  }
  TcRowGemmArgs ac{(float*)cbufs_host[0], (float*)cbufs_host[1], (const float*)cu, nullptr,
                   (float* const*)dbufs, ldc};
  k_tc_rowgemm<<<grid, 256, TC_SMEM, st>>>(ctl, w, maps.c0, maps.c1, maps.bc_hi, maps.bc_lo, ac);
  TcRowGemmArgs av{(float*)vbufs_host[0], (float*)vbufs_host[1], (const float*)wv,
                   (const float*)evec, (float* const*)dbufs, ldc};
  k_tc_rowgemm<<<grid, 256, TC_SMEM, st>>>(ctl, w, maps.v0, maps.v1, maps.bv_hi, maps.bv_lo, av);
  return cudaGetLastError();
}

}  // namespace tk

namespace tk {

// =============================================================================================
// k_tc_proj: the pass of Alg. 4 for spatial mode k on the tensor cores, fused. The input X is
// the row-major (F x n_k) matrix of mode-k fibers (the slice for k = 0, else the previous mode's
// output in the rotating layout).
//   MMA1  P[f, :] = X[f, :] U_k (K = n_k), 3xTF32, X tiles by TMA, U_k chunks (TF32 hi/lo)
//         streamed with them; P accumulates in TMEM.
//   epi-1 P = (hi x hi part, TMEM cols 0..63 of its buffer) + (correction part, cols 64..127)
//         -> global, column-major (F x r_k) (the next mode's input); P split in place into
//         TF32 hi (TMEM cols 0..63 of its buffer) and lo (cols 64..127).
//   MMA2  (RESID) Rec = P U_k^T with A = P read from tensor memory, B = U_k rows resident in
//         shared memory, 3xTF32; Rec in TMEM cols 256..256+n_k.
// P has two TMEM buffers (tile t in buffer t & 1, cols 128 (t & 1) ..): MMA1 of tile t+1 runs
// while the epilogue reads P of tile t, and MMA2 of tile t is issued between the chunk MMAs of
// tile t+1 as soon as the epilogue has stored P's split (the tensor pipe runs MMAs in issue
// order). Barriers that complete once per tile and are waited for across a tile boundary
// (d1full, pready, mma2done) have one instance per buffer, so a phase is never two ahead.
//   epi-2 (RESID) E = X - Rec with X re-read (L2-resident), ||E||^2 (and ||Y||^2 for k = 0) as
//         per-block partials; WRITE_ET: E^T (n_k x Fs, row stride Fs) for the residual Gram.
// Blocked form (n_k > 256: Rec no longer fits 256 TMEM columns, nor U_k's rows in shared memory):
// MMA2 runs in column blocks of TP_NB = 128. Block g of the CTA's sequence (tile g / NB, columns
// TP_NB (g % NB) ..) accumulates into D2 buffer g & 1 (TMEM cols 256 + 128 (g & 1)), with B =
// rows TP_NB (g % NB) .. of U_k (TF32 hi/lo) in one shared buffer. The residual epilogue's
// leader loads B2 block g + 1 as soon as block g's MMA2 has completed (its d2full), and the MMA
// issuer issues block g once the tile's P split is stored, B2 block g has landed and D2 buffer
// g & 1 has been read (d2free, block g - 2), between the chunk MMAs of the next tile.
// =============================================================================================
constexpr int TP_STAGE = 48 * 1024;                // X hi | X lo | U chunk hi | U chunk lo
// stages: 2 when the residual runs (the resident U rows for MMA2 and the Y buffers take 128 KB),
// 4 for the re-projection (pass C), which needs neither
template <bool RESID> struct TpCfg {
  static constexpr int S = RESID ? 2 : 4;
  static constexpr size_t B2 = RESID ? 128 * 1024 : 0;
  static constexpr size_t SMEM = (size_t)S * TP_STAGE + B2 + 1024 + 512;
};
constexpr int TP_NB = 128;                          // columns of an MMA2 block (blocked form)
constexpr int TP_PF = 12;                           // X chunks prefetched into L2 ahead
// warps: 0 TMA producer, 1 MMA issuer, 2 .. 2+TP_SPLIT_WARPS-1 TF32 splitters of the X chunks,
// then 4 warps for epilogue 1 (P) and 4 for epilogue 2 (the residual), so that epilogue 1 of
// tile t+1 runs while epilogue 2 of tile t waits for its reloaded X (TMEM lane quarter =
// warp % 4, so each group starts at a multiple of 4)
constexpr int TP_SPLIT_WARPS = 6;
constexpr int TP_EPI_W0 = 2 + TP_SPLIT_WARPS;
constexpr int TP_NT = 32 * (TP_EPI_W0 + 8);
static_assert(TP_EPI_W0 % 4 == 0, "epilogue warps must start at a TMEM lane quarter boundary");

struct TcProjArgs {
  const CUtensorMap* mYg;   // slice descriptor in the control block (graph form), else NULL
  float* const* dbufs;
  int out_off;
  double* part_e2;
  double* part_y2;
  int nparts;
  const float* Y;
  float* Et;
  long long et_stride;
  int k;
};

template <bool RESID, bool WRITE_ET>
__global__ void __launch_bounds__(TP_NT, 1) k_tc_proj(const Ctl* __restrict__ ctl, int pred,
                                                   const __grid_constant__ CUtensorMap mY,
                                                   const __grid_constant__ CUtensorMap mD0,
                                                   const __grid_constant__ CUtensorMap mD1,
                                                   const __grid_constant__ CUtensorMap mD2,
                                                   const __grid_constant__ CUtensorMap mUhi,
                                                   const __grid_constant__ CUtensorMap mUlo,
                                                   const __grid_constant__ CUtensorMap mUrhi,
                                                   const __grid_constant__ CUtensorMap mUrlo,
                                                   TcProjArgs a) {
  if (ctl->status) return;
  const int k = a.k;
  if (pred && !ctl->grew[k]) return;
  const int r = ctl->r[k];
  if (!tc_proj_ok(ctl, k, r)) return;
  const int n1 = ctl->n[k];
  const long long F = view_B(ctl, k);
  const int Rp = (r + 15) / 16 * 16;
  const int n1p = (n1 + 15) / 16 * 16;
  const int Kc1 = (n1 + TC_KC - 1) / TC_KC;
  const int Kc2 = (Rp + TC_KC - 1) / TC_KC;
  const long long ntiles = (F + TC_M - 1) / TC_M;
  // blocked MMA2 (n_k > 256): NB column blocks per tile
  const bool blocked = RESID && n1p > 256;
  const int NB = blocked ? (n1p + TP_NB - 1) / TP_NB : 1;
  const int xb = ctl->xbuf;
  const CUtensorMap* mX = xb < 0 ? (a.mYg ? a.mYg : &mY) : (xb == 0 ? &mD0 : (xb == 1 ? &mD1 : &mD2));
  const float* Xg = xb < 0 ? (a.Y ? a.Y : reinterpret_cast<const float*>(ctl->yptr)) : a.dbufs[xb];
  float* P = a.dbufs[(xb + a.out_off + 3) % 3];

  extern __shared__ __align__(1024) unsigned char psm_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(psm_raw) + 1023) & ~uintptr_t(1023));
  constexpr int TP_S = TpCfg<RESID>::S;
  // RESID: U_k rows for MMA2, [Kc2][n1p][32] hi then lo (resident), or [Kc2][TP_NB][32] hi then
  // lo (one column block, blocked form)
  const int b2rows = blocked ? TP_NB : n1p;
  float* B2hi = reinterpret_cast<float*>(base + TP_S * TP_STAGE);
  float* B2lo = B2hi + (size_t)Kc2 * b2rows * TC_KC;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + TP_S * TP_STAGE + TpCfg<RESID>::B2);
  uint64_t* full = bars;
  uint64_t* conv = bars + TP_S;
  uint64_t* empty = bars + 2 * TP_S;
  uint64_t* d1full = bars + 3 * TP_S;              // [2] per P buffer
  uint64_t* pready = d1full + 2;                   // [2]
  uint64_t* d2full = pready + 2;                   // [2] per D2 buffer (blocked form; else [0])
  uint64_t* d2free = d2full + 2;                   // [2]
  uint64_t* mma2done = d2free + 2;                 // [2]
  uint64_t* bload = mma2done + 2;                  // resident B2 (one load) or B2 block g (phase g)
  uint64_t* done = bload + 1;
  uint64_t* ybar = done + 1;                       // [2] Y chunk loaded (residual epilogue)
  uint64_t* yfree = ybar + 2;                      // [2] Y chunk consumed by the 4 epilogue warps
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(yfree + 2);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  double* red = reinterpret_cast<double*>(tmem_slot + 4);   // [8] doubles

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TP_S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], 32 * TP_SPLIT_WARPS);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&d1full[b], 1);
      mbar_init(&pready[b], 128);
      mbar_init(&mma2done[b], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&d2full[b], 1);
      mbar_init(&d2free[b], 128);
    }
    mbar_init(bload, 1);
    mbar_init(done, 1);
    mbar_init(&ybar[0], 1);
    mbar_init(&ybar[1], 1);
    mbar_init(&yfree[0], 4);
    mbar_init(&yfree[1], 4);
    *abort = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t tD2 = tmem + 256;   // P buffers at tmem + 128 b (hi) and + 64 (lo)

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      if (xb < 0 && a.mYg) tensormap_acquire(a.mYg);   // written by a copy before the launch
      tma_prefetch(mX);
      tma_prefetch(&mUhi);
      tma_prefetch(&mUlo);
      if (RESID) {
        tma_prefetch(&mUrhi);
        tma_prefetch(&mUrlo);
      }
      if (RESID && !blocked) {
        mbar_arrive_expect_tx(bload, (uint32_t)Kc2 * n1p * TC_KC * 4 * 2);
        for (int kc = 0; kc < Kc2; ++kc)
          for (int n0 = 0; n0 < n1p; n0 += 16) {
            tma_load_2d(&mUrhi, bload, B2hi + ((size_t)kc * n1p + n0) * TC_KC, kc * TC_KC, n0);
            tma_load_2d(&mUrlo, bload, B2lo + ((size_t)kc * n1p + n0) * TC_KC, kc * TC_KC, n0);
          }
      }
      // the X chunk TP_PF chunks ahead of the one loaded is prefetched into L2, so the two
      // stages wait on L2 rather than on DRAM latency
      const long long nq = (long long)((ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x) * Kc1;
      auto prefetch_chunk = [&](long long qq) {
        if (qq >= nq) return;
        const long long tt = blockIdx.x + (qq / Kc1) * (long long)gridDim.x;
        tma_prefetch_l2_2d(mX, (int)(qq % Kc1) * TC_KC, (int)(tt * TC_M));
      };
      for (long long qq = 0; qq < TP_PF; ++qq) prefetch_chunk(qq);
      long long q = 0;
      for (long long t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
        for (int kc = 0; kc < Kc1; ++kc, ++q) {
          const int s = (int)(q % TP_S);
          prefetch_chunk(q + TP_PF);
          if (!wait_bar(&empty[s], (uint32_t)(((q / TP_S) & 1) ^ 1), abort)) break;
          unsigned char* st = base + (size_t)s * TP_STAGE;
          mbar_arrive_expect_tx(&full[s], (uint32_t)(TC_M * TC_KC * 4 + Rp * TC_KC * 4 * 2));
          tma_load_2d(mX, &full[s], st, kc * TC_KC, (int)(t * TC_M));
          for (int n0 = 0; n0 < Rp; n0 += 16) {
            tma_load_2d(&mUhi, &full[s], st + 32 * 1024 + n0 * 128, kc * TC_KC, n0);
            tma_load_2d(&mUlo, &full[s], st + 40 * 1024 + n0 * 128, kc * TC_KC, n0);
          }
        }
      }
      for (long long j = (q > TP_S ? q - TP_S : 0); j < q; ++j)
        wait_bar(&empty[j % TP_S], (uint32_t)((j / TP_S) & 1), abort);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t id1 = idesc_tf32(TC_M, Rp);
      const uint32_t id2 = idesc_tf32(TC_M, blocked ? TP_NB : n1p);
      bool ok = (RESID && !blocked) ? wait_bar(bload, 0, abort) : true;
      // MMA2 of tile jt: Rec = P U_k^T into D2 once the epilogue has stored P's split and has
      // read D2 of tile jt - 1 (it did so before it stored P of tile jt)
      auto mma2 = [&](int jt) -> bool {
        const uint32_t pb = (uint32_t)((jt >> 1) & 1);
        if (!wait_bar(&pready[jt & 1], pb, abort)) return false;
        if (!wait_bar(&d2free[0], (uint32_t)((jt & 1) ^ 1), abort)) return false;
        tc_fence_after();
        const uint32_t tA = tmem + 128u * (uint32_t)(jt & 1);
        for (int k8 = 0; k8 < Rp / 8; ++k8) {
          const int kc = k8 >> 2;
          const uint64_t o = (uint64_t)((k8 & 3) * 32) >> 4;
          const uint64_t bhi = desc_sw128(B2hi + (size_t)kc * n1p * TC_KC) + o;
          const uint64_t blo = desc_sw128(B2lo + (size_t)kc * n1p * TC_KC) + o;
          mma_tf32_ts(tD2, tA + 8 * k8, bhi, id2, k8 ? 1u : 0u);
          mma_tf32_ts(tD2, tA + 8 * k8, blo, id2, 1u);
          mma_tf32_ts(tD2, tA + 64 + 8 * k8, bhi, id2, 1u);
        }
        tc_commit(&d2full[0]);
        tc_commit(&mma2done[jt & 1]);
        return true;
      };
      // blocked form: the next MMA2 block to issue is block b_nb of tile b_tile (-1: none), the
      // CTA's g2-th block; returns 1 once issued, 0 if not ready (non-blocking), -1 on abort
      long long g2 = 0;
      int b_tile = -1, b_nb = 0;
      auto mma2_block = [&](bool blocking) -> int {
        const uint32_t pb = (uint32_t)((b_tile >> 1) & 1);
        const int bb = (int)(g2 & 1);
        const uint32_t lpar = (uint32_t)(g2 & 1), fpar2 = (uint32_t)(((g2 >> 1) & 1) ^ 1);
        if (blocking) {
          if (b_nb == 0 && !wait_bar(&pready[b_tile & 1], pb, abort)) return -1;
          if (!wait_bar(bload, lpar, abort)) return -1;
          if (!wait_bar(&d2free[bb], fpar2, abort)) return -1;
        } else {
          if (b_nb == 0 && !mbar_try_wait(&pready[b_tile & 1], pb)) return 0;
          if (!mbar_try_wait(bload, lpar)) return 0;
          if (!mbar_try_wait(&d2free[bb], fpar2)) return 0;
        }
        tc_fence_after();
        const int ncol = min(TP_NB, n1p - TP_NB * b_nb);
        const uint32_t idb = idesc_tf32(TC_M, ncol);
        const uint32_t tA = tmem + 128u * (uint32_t)(b_tile & 1);
        const uint32_t tDb = tD2 + 128u * (uint32_t)bb;
        for (int k8 = 0; k8 < Rp / 8; ++k8) {
          const int kc = k8 >> 2;
          const uint64_t o = (uint64_t)((k8 & 3) * 32) >> 4;
          const uint64_t bhi = desc_sw128(B2hi + (size_t)kc * TP_NB * TC_KC) + o;
          const uint64_t blo = desc_sw128(B2lo + (size_t)kc * TP_NB * TC_KC) + o;
          mma_tf32_ts(tDb, tA + 8 * k8, bhi, idb, k8 ? 1u : 0u);
          mma_tf32_ts(tDb, tA + 8 * k8, blo, idb, 1u);
          mma_tf32_ts(tDb, tA + 64 + 8 * k8, bhi, idb, 1u);
        }
        tc_commit(&d2full[bb]);
        ++g2;
        if (++b_nb == NB) {
          tc_commit(&mma2done[b_tile & 1]);
          b_tile = -1;
          b_nb = 0;
        }
        return 1;
      };
      long long q = 0;
      int it = 0;
      int pend = -1;   // tile whose MMA2 is not issued yet (RESID)
      for (long long t = blockIdx.x; ok && t < ntiles; t += gridDim.x, ++it) {
        const int b = it & 1;
        const uint32_t tD1 = tmem + 128u * (uint32_t)b;
        // P buffer b is free once tile it - 2 is done with it: its MMA2 completed (RESID,
        // issued by the end of tile it - 1), else its epi-1 read it. First uses pass at once.
        const uint32_t fpar = (uint32_t)(((it >> 1) & 1) ^ 1);
        if (RESID) ok = wait_bar(&mma2done[b], fpar, abort);
        else ok = wait_bar(&pready[b], fpar, abort);
        if (!ok) break;
        tc_fence_after();
        for (int kc = 0; kc < Kc1; ++kc, ++q) {
          const int s = (int)(q % TP_S);
          if (!wait_bar(&conv[s], (uint32_t)((q / TP_S) & 1), abort)) { ok = false; break; }
          tc_fence_after();
          unsigned char* st = base + (size_t)s * TP_STAGE;
          const uint64_t ahi = desc_sw128(st), alo = desc_sw128(st + 16 * 1024);
          const uint64_t bhi = desc_sw128(st + 32 * 1024), blo = desc_sw128(st + 40 * 1024);
          // hi x hi into the accumulator at cols 0.. of the P buffer, the two correction
          // products into a second one at cols 64..: the FP32 accumulation error of a chain grows
          // with its number of steps and is mostly toward zero, so P's large part is summed over
          // n_k / 8 steps rather than 3 n_k / 8 (an error of P lies in span(U_k) and adds its
          // square to ||E_k||^2); epilogue 1 adds the two
#pragma unroll
          for (int k4 = 0; k4 < TC_KC / 8; ++k4) {
            const uint64_t o = (uint64_t)(k4 * 32) >> 4;
            mma_tf32(tD1, ahi + o, bhi + o, id1, (kc | k4) ? 1u : 0u);
            mma_tf32(tD1 + 64, ahi + o, blo + o, id1, (kc | k4) ? 1u : 0u);
            mma_tf32(tD1 + 64, alo + o, bhi + o, id1, 1u);
          }
          tc_commit(&empty[s]);
          if (blocked) {
            // pending MMA2 blocks of the previous tile go in as soon as they are ready
            int rc = 1;
            while (b_tile >= 0 && (rc = mma2_block(false)) > 0) {}
            if (rc < 0) { ok = false; break; }
          } else if (RESID && pend >= 0 && mbar_try_wait(&pready[pend & 1], (uint32_t)((pend >> 1) & 1))) {
            // the pending MMA2 goes in as soon as its P split is stored
            if (!mma2(pend)) { ok = false; break; }
            pend = -1;
          }
        }
        if (!ok) break;
        tc_commit(&d1full[b]);
        if (blocked) {
          while (ok && b_tile >= 0) ok = mma2_block(true) > 0;
          if (!ok) break;
          b_tile = it;
          b_nb = 0;
        } else if (RESID) {
          if (pend >= 0 && !mma2(pend)) break;
          pend = it;
        }
      }
      if (blocked) {
        while (ok && b_tile >= 0) ok = mma2_block(true) > 0;
      } else if (RESID && ok && pend >= 0) {
        mma2(pend);
      }
      tc_commit(done);
      wait_bar(done, 0, abort);
    }
    __syncwarp();
  } else if (warp >= 2 && warp < 2 + TP_SPLIT_WARPS) {
    // ---------------- X splitters ----------------
    const int ct = threadIdx.x - 64;
    long long q = 0;
    for (long long t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
      for (int kc = 0; kc < Kc1; ++kc, ++q) {
        const int s = (int)(q % TP_S);
        if (!wait_bar(&full[s], (uint32_t)((q / TP_S) & 1), abort)) break;
        float4* hi = reinterpret_cast<float4*>(base + (size_t)s * TP_STAGE);
        float4* lo = hi + TC_M * TC_KC / 4;
#pragma unroll 4
        for (int i = ct; i < TC_M * TC_KC / 4; i += 32 * TP_SPLIT_WARPS) {
          float4 v = hi[i], h, l;
          tf32_split(v.x, h.x, l.x);
          tf32_split(v.y, h.y, l.y);
          tf32_split(v.z, h.z, l.z);
          tf32_split(v.w, h.w, l.w);
          hi[i] = h;
          lo[i] = l;
        }
        fence_proxy_async_smem();
        mbar_arrive(&conv[s]);
      }
    }
  } else if (warp >= TP_EPI_W0 && warp < TP_EPI_W0 + 4) {
    // ---------------- epilogue 1: P ----------------
    const int wq = warp - TP_EPI_W0;   // TMEM lane quarter (warp % 4)
    const uint32_t lq = (uint32_t)(wq * 32) << 16;
    int it = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      const uint32_t tD1 = tmem + 128u * (uint32_t)(it & 1), tDlo = tD1 + 64;
      bool okw = wait_bar(&d1full[it & 1], (uint32_t)((it >> 1) & 1), abort);
      okw = __all_sync(0xffffffffu, okw);
      if (!okw) break;
      tc_fence_after();
      const long long f = t * TC_M + wq * 32 + lane;
      const bool live = f < F;
      for (int c0 = 0; c0 < Rp; c0 += 32) {
        float v[32], w[32];
        tmem_ld32(tD1 + lq + c0, v);
        tmem_ld32(tDlo + lq + c0, w);
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] += w[i];
        if (live && !WRITE_ET) {
          // column-major (F x r): consecutive threads write consecutive addresses
#pragma unroll
          for (int i = 0; i < 32; ++i)
            if (c0 + i < r) P[f + F * (c0 + i)] = v[i];
        }
        if (RESID) {
          float l[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) tf32_split(v[i], v[i], l[i]);
          tmem_st32(tD1 + lq + c0, v);
          tmem_st32(tDlo + lq + c0, l);
        }
      }
      tc_fence_before();
      mbar_arrive(&pready[it & 1]);
    }
  } else if (RESID && warp >= TP_EPI_W0 + 4) {
    // ---------------- epilogue 2: E = X - Rec, norms ----------------
    const int wq = warp - TP_EPI_W0 - 4;   // TMEM lane quarter (warp % 4)
    const uint32_t lq = (uint32_t)(wq * 32) << 16;
    double eacc = 0.0, yacc = 0.0;
    // The residual needs the tile's Y again: when the resident U copy leaves 32 KB, these warps
    // reload Y by 32-column chunks (TMA, an L2 hit: the tile was streamed moments before) into
    // two swizzled buffers, instead of 128 strided row reads per chunk from global memory.
    const int nck = (n1 + TC_KC - 1) / TC_KC;
    const bool ysm = blocked || (size_t)2 * Kc2 * n1p * TC_KC * 4 + 2 * TC_M * TC_KC * 4 <= 128 * 1024;
    float* ybuf = B2lo + (size_t)Kc2 * b2rows * TC_KC;   // [2][TC_M][TC_KC], 1024-byte aligned
    const bool yleader = (wq == 0 && lane == 0);
    if (ysm && yleader && xb < 0 && a.mYg) tensormap_acquire(a.mYg);
    long long yq = 0;                                 // Y chunks consumed so far
    // chunk seq goes to buffer seq & 1 once the 4 warps have consumed chunk seq - 2 (bounded
    // wait of the issuing thread); returns false if that wait gave up
    auto issue_y = [&](long long t_, int ci, long long seq) -> bool {
      if (seq >= 2 && !wait_bar(&yfree[seq & 1], (uint32_t)(((seq - 2) >> 1) & 1), abort)) return false;
      mbar_arrive_expect_tx(&ybar[seq & 1], (uint32_t)(TC_M * TC_KC * 4));
      tma_load_2d(mX, &ybar[seq & 1], ybuf + (size_t)(seq & 1) * TC_M * TC_KC, ci * TC_KC, (int)(t_ * TC_M));
      return true;
    };
    // blocked form: B2 block gg (rows TP_NB (gg % NB) .. of U_k) into the B2 buffer, issued by
    // the leader once block gg - 1's MMA2 has completed
    const long long myt = ntiles > blockIdx.x ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const long long nblk = myt * NB;
    auto issue_b2 = [&](long long gg) {
      const int nb = (int)(gg % NB);
      mbar_arrive_expect_tx(bload, (uint32_t)Kc2 * TP_NB * TC_KC * 4 * 2);
      for (int kc = 0; kc < Kc2; ++kc)
        for (int n0 = 0; n0 < TP_NB; n0 += 16) {
          tma_load_2d(&mUrhi, bload, B2hi + ((size_t)kc * TP_NB + n0) * TC_KC, kc * TC_KC, TP_NB * nb + n0);
          tma_load_2d(&mUrlo, bload, B2lo + ((size_t)kc * TP_NB + n0) * TC_KC, kc * TC_KC, TP_NB * nb + n0);
        }
    };
    if (blocked && yleader && nblk > 0) issue_b2(0);
    long long g = 0;    // MMA2 blocks consumed (blocked form)
    bool okall = true;
    int it = 0;
    for (long long t = blockIdx.x; okall && t < ntiles; t += gridDim.x, ++it) {
      if (ysm && yleader) {
        if (issue_y(t, 0, yq) && nck > 1) issue_y(t, 1, yq + 1);
      }
      __syncwarp();
      bool okw = true;
      if (!blocked) {
        okw = wait_bar(&d2full[0], (uint32_t)(it & 1), abort);
        okw = __all_sync(0xffffffffu, okw);
        if (!okw) break;
        tc_fence_after();
      }
      const long long f = t * TC_M + wq * 32 + lane;
      const bool live = f < F;
      const float* xrow = Xg + f * n1;
      const int row = wq * 32 + lane;
      for (int c0 = 0, ci = 0; c0 < n1p; c0 += 32, ++ci) {
        if (blocked && c0 % TP_NB == 0) {
          // start of column block g: wait for its MMA2, then refill the B2 buffer with block g + 1
          okw = wait_bar(&d2full[g & 1], (uint32_t)((g >> 1) & 1), abort);
          okw = __all_sync(0xffffffffu, okw);
          if (!okw) { okall = false; break; }
          tc_fence_after();
          if (yleader && g + 1 < nblk) issue_b2(g + 1);
          __syncwarp();
        }
        const uint32_t tcol = blocked ? tD2 + 128u * (uint32_t)(g & 1) + (uint32_t)(c0 % TP_NB) : tD2 + (uint32_t)c0;
        float v[32];
        tmem_ld32(tcol + lq, v);
        const float4* ych = reinterpret_cast<const float4*>(ybuf + (size_t)(yq & 1) * TC_M * TC_KC) + row * 8;
        if (ysm) {
          okw = wait_bar(&ybar[yq & 1], (uint32_t)((yq >> 1) & 1), abort);
          okw = __all_sync(0xffffffffu, okw);
        }
        if (live && okw) {
          // FP32 partial sums over 32 elements, flushed to FP64 per chunk
          float es = 0.f, ys = 0.f;
#pragma unroll
          for (int i = 0; i < 32; i += 4) {
            if (c0 + i < n1) {
              // SWIZZLE_128B: 16-byte piece j of row `row` sits at piece j ^ (row & 7)
              const float4 y = ysm ? ych[(i >> 2) ^ (row & 7)]
                                   : *reinterpret_cast<const float4*>(xrow + c0 + i);
              const float e0 = y.x - v[i], e1 = y.y - v[i + 1], e2 = y.z - v[i + 2], e3 = y.w - v[i + 3];
              es = fmaf(e0, e0, es); es = fmaf(e1, e1, es); es = fmaf(e2, e2, es); es = fmaf(e3, e3, es);
              ys = fmaf(y.x, y.x, ys); ys = fmaf(y.y, y.y, ys); ys = fmaf(y.z, y.z, ys); ys = fmaf(y.w, y.w, ys);
              if (WRITE_ET) {
                float* et = a.Et + f;
                et[(long long)(c0 + i) * a.et_stride] = e0;
                et[(long long)(c0 + i + 1) * a.et_stride] = e1;
                et[(long long)(c0 + i + 2) * a.et_stride] = e2;
                et[(long long)(c0 + i + 3) * a.et_stride] = e3;
              }
            }
          }
          eacc += (double)es;
          yacc += (double)ys;
        } else if (WRITE_ET && f < a.et_stride) {
          // zero the padding fibers the Gram's last K chunk reads
          for (int i = 0; i < 32; ++i)
            if (c0 + i < n1) a.Et[(long long)(c0 + i) * a.et_stride + f] = 0.f;
        }
        if (ysm) {
          // this warp is done with the buffer; it is refilled with chunk ci + 2 once all four
          // warps of this group are
          __syncwarp();
          if (lane == 0) mbar_arrive(&yfree[yq & 1]);
          if (yleader && ci + 2 < nck) issue_y(t, ci + 2, yq + 2);
          __syncwarp();   // the next tcgen05.ld is warp-collective: lane 0 may have waited
          ++yq;
        }
        if (blocked && ((c0 + 32) % TP_NB == 0 || c0 + 32 >= n1p)) {
          // end of column block g: its D2 buffer may be reused by block g + 2
          tc_fence_before();
          mbar_arrive(&d2free[g & 1]);
          ++g;
        }
      }
      if (!okall) break;
      if (!blocked) {
        tc_fence_before();
        mbar_arrive(&d2free[0]);
      }
    }
    if (!WRITE_ET) {
      double se = warp_sum(eacc), sy = warp_sum(yacc);
      if (lane == 0) { red[wq] = se; red[4 + wq] = sy; }
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (wq == 0 && lane == 0) {
        const double te = red[0] + red[1] + red[2] + red[3];
        const double ty = red[4] + red[5] + red[6] + red[7];
        for (int j = blockIdx.x; j < a.nparts; j += gridDim.x) {
          a.part_e2[j] = (j == (int)blockIdx.x) ? te : 0.0;
          if (a.part_y2) a.part_y2[j] = (j == (int)blockIdx.x) ? ty : 0.0;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, 512);
  if (threadIdx.x == 0 && *abort) const_cast<Ctl*>(ctl)->status = 5;
}

// Split copies of U_k for the tensor-core passes (after the initial ST-HOSVD and after growth):
// column-major (n_k x cap, as the FP32 work copy) and row-major (n_k x 64) TF32 hi/lo parts.
__global__ void k_split_u(const Ctl* ctl, int k, int pred, const double* U, int ldu, float* uhi,
                          float* ulo, float* urhi, float* urlo) {
  if (ctl->status) return;
  if (pred && !ctl->grew[k]) return;
  const int n1 = ctl->n[k];
  const int r = ctl->r[k];
  const int cap = ctl->cap[k];
  for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < (long long)n1 * cap;
       L += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(L % n1), i = (int)(L / n1);
    const float v = (i < r) ? (float)U[(long long)i * ldu + j] : 0.f;
    float h, l;
    tf32_split(v, h, l);
    uhi[L] = h;
    ulo[L] = l;
    if (i < TP_RMAX) {
      urhi[(long long)j * TP_RMAX + i] = h;
      urlo[(long long)j * TP_RMAX + i] = l;
    }
  }
}

cudaError_t launch_split_u(const Ctl* ctl, int k, int pred, const double* U, int ldu,
                           float* const* sp, cudaStream_t st) {
  k_split_u<<<64, 256, 0, st>>>(ctl, k, pred, U, ldu, sp[0], sp[1], sp[2], sp[3]);
  return cudaGetLastError();
}

cudaError_t launch_tc_proj(const Ctl* ctl, int k, int mode, int pred, const float* Y,
                           long long F0, int n0, const TcProjMaps& m, void* const* dbufs,
                           int out_off, double* part_e2, double* part_y2, int nparts, float* Et,
                           long long et_stride, int grid, cudaStream_t st) {
  CUtensorMap mY;
  const CUtensorMap* mYg = nullptr;
  if (k == 0 && Y) {
    if (!make_map_2d_f32(&mY, Y, F0, n0, n0, 32, 128)) return cudaErrorInvalidValue;
  } else {
    mY = m.d[0];   // unused for k >= 1 (the input is a D buffer)
    // graph form (Y == NULL): the slice descriptor is read from the control block
    if (k == 0) mYg = reinterpret_cast<const CUtensorMap*>(reinterpret_cast<const unsigned char*>(ctl) + offsetof(Ctl, ymap));
  }
  TcProjArgs a{mYg, (float* const*)dbufs, out_off, part_e2, part_y2, nparts, Y, Et, et_stride, k};
  static bool attr[3] = {false, false, false};
  if (mode == 0) {
    if (!attr[0]) { cudaFuncSetAttribute(k_tc_proj<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TpCfg<false>::SMEM); attr[0] = true; }
    k_tc_proj<false, false><<<grid, TP_NT, TpCfg<false>::SMEM, st>>>(ctl, pred, mY, m.d[0], m.d[1], m.d[2], m.uhi, m.ulo, m.urhi, m.urlo, a);
  } else if (mode == 1) {
    if (!attr[1]) { cudaFuncSetAttribute(k_tc_proj<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TpCfg<true>::SMEM); attr[1] = true; }
    k_tc_proj<true, false><<<grid, TP_NT, TpCfg<true>::SMEM, st>>>(ctl, pred, mY, m.d[0], m.d[1], m.d[2], m.uhi, m.ulo, m.urhi, m.urlo, a);
  } else {
    if (!attr[2]) { cudaFuncSetAttribute(k_tc_proj<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TpCfg<true>::SMEM); attr[2] = true; }
    k_tc_proj<true, true><<<grid, TP_NT, TpCfg<true>::SMEM, st>>>(ctl, pred, mY, m.d[0], m.d[1], m.d[2], m.uhi, m.ulo, m.urhi, m.urlo, a);
  }
  return cudaGetLastError();
}

// =============================================================================================
// k_tc_syrk: partial Gram G = E^T E of the mode-k residual unfolding (Alg. 1's Gram of E_(k)),
// split over the fibers (K). A chunk is the n_k rows x 32 fibers of E^T (TMA, 128-row boxes,
// rows past n_k zero-filled), split on chip into TF32 hi/lo (3xTF32); the MMA operands are row
// ranges of that one buffer. Only the blocks on and right of the diagonal of 128-row blocks are
// formed (the rest of G is their transpose): row block a covers rows 128a .. 128a + 127 and
// columns 128a .. n_k. Up to 256 rows (ROWS = 256) one CTA per K split forms both row blocks
// (TMEM cols 0.. and 256..); up to 384 rows (ROWS = 384) the three row blocks do not fit 512
// TMEM columns together, so the splits run twice (blockIdx.y): group 0 forms row block 0 (two
// MMAs, columns 0..255 and 256..), group 1 row blocks 1 and 2, each group streaming the same
// chunks. FP32 partial blocks per split are summed in FP64 by k_syrk_reduce, in a fixed order.
// Warps: 0 TMA producer, 1 MMA issuer, 2..11 splitters; 4..7 also read the accumulators out.
// =============================================================================================
constexpr int TS_SPLIT_W = 10;
constexpr int TS_NT = 32 * (2 + TS_SPLIT_W);
template <int ROWS> struct TsCfg {
  static constexpr int STAGE = 2 * ROWS * TC_KC * 4;     // hi | lo: 64 KB (256 rows), 96 KB (384)
  static constexpr int S = ROWS <= 256 ? 3 : 2;
  static constexpr size_t SMEM = (size_t)S * STAGE + 1024 + 256;
};
constexpr int TS_NMAX = 384;                          // largest n_k of the tensor-core Gram

// One MMA target of a CTA: D (TMEM cols tm ..) += rows [128 a, 128 a + 128) x rows [cs, cs + N)
// of the chunk.
struct TsTarget { int a, cs, N, tm; };
__device__ __forceinline__ int ts_targets(int n1p, int group, TsTarget (&t)[2]) {
  if (n1p <= 256) {
    t[0] = {0, 0, n1p, 0};
    if (n1p <= TC_M) return 1;
    t[1] = {1, TC_M, n1p - TC_M, 256};
    return 2;
  }
  if (group == 0) {
    t[0] = {0, 0, 256, 0};
    t[1] = {0, 256, n1p - 256, 256};
  } else {
    t[0] = {1, TC_M, n1p - TC_M, 0};
    t[1] = {2, 256, n1p - 256, 256};
  }
  return 2;
}

template <int ROWS>
__global__ void __launch_bounds__(TS_NT, 1) k_tc_syrk(const Ctl* __restrict__ ctl, int k,
                                                     const __grid_constant__ CUtensorMap mEa,
                                                     float* __restrict__ gpart) {
  constexpr int TS_S = TsCfg<ROWS>::S;
  constexpr int TS_STAGE = TsCfg<ROWS>::STAGE;
  if (ctl->status) return;
  if (!tc_gram_ok(ctl, k)) return;
  const int n1 = ctl->n[k];
  const long long F = view_B(ctl, k);
  const int n1p = (n1 + 15) / 16 * 16;
  if (n1p > ROWS || (ROWS > 256 && n1p <= 256)) return;   // the other instance takes this size
  const int MT = (n1p + TC_M - 1) / TC_M;             // row blocks loaded per chunk
  TsTarget tg[2];
  const int ntg = ts_targets(n1p, blockIdx.y, tg);
  const int S = gridDim.x, sp = blockIdx.x;
  const long long KC = (F + TC_KC - 1) / TC_KC;
  const long long per = (KC + S - 1) / S;
  const long long c_beg = sp * per;
  const long long c_end = c_beg + per < KC ? c_beg + per : KC;
  const int nchunks = c_end > c_beg ? (int)(c_end - c_beg) : 0;
  extern __shared__ __align__(1024) unsigned char ssm_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(ssm_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + TS_S * TS_STAGE);
  uint64_t* full = bars;
  uint64_t* conv = bars + TS_S;
  uint64_t* empty = bars + 2 * TS_S;
  uint64_t* accfull = bars + 3 * TS_S;
  uint64_t* done = accfull + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TS_S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], 32 * TS_SPLIT_W);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accfull, 1);
    mbar_init(done, 1);
    *abort = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // stage layout: hi rows [0, ROWS) x 128 B, then lo rows [0, ROWS) x 128 B
  if (warp == 0) {
    if (lane == 0) {
      tma_prefetch(&mEa);
      for (int c = 0; c < nchunks && !*abort; ++c) {
        const int s = c % TS_S;
        if (!wait_bar(&empty[s], (uint32_t)(((c / TS_S) & 1) ^ 1), abort)) break;
        unsigned char* st = base + (size_t)s * TS_STAGE;
        const int x = (int)((c_beg + c) * TC_KC);
        mbar_arrive_expect_tx(&full[s], (uint32_t)(MT * TC_M * TC_KC * 4));
        for (int mt = 0; mt < MT; ++mt)
          tma_load_2d(&mEa, &full[s], st + (size_t)mt * TC_M * 128, x, mt * TC_M);
      }
      for (int j = (nchunks > TS_S ? nchunks - TS_S : 0); j < nchunks; ++j)
        wait_bar(&empty[j % TS_S], (uint32_t)((j / TS_S) & 1), abort);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t id[2];
      for (int g = 0; g < ntg; ++g) id[g] = idesc_tf32(TC_M, tg[g].N);
      bool ok = true;
      for (int c = 0; c < nchunks; ++c) {
        const int s = c % TS_S;
        if (!wait_bar(&conv[s], (uint32_t)((c / TS_S) & 1), abort)) { ok = false; break; }
        tc_fence_after();
        unsigned char* st = base + (size_t)s * TS_STAGE;
        for (int g = 0; g < ntg; ++g) {
          const uint64_t ha = desc_sw128(st + (size_t)tg[g].a * TC_M * 128);
          const uint64_t la = desc_sw128(st + (size_t)ROWS * 128 + (size_t)tg[g].a * TC_M * 128);
          const uint64_t hb = desc_sw128(st + (size_t)tg[g].cs * 128);
          const uint64_t lb = desc_sw128(st + (size_t)ROWS * 128 + (size_t)tg[g].cs * 128);
          const uint32_t td = tmem + (uint32_t)tg[g].tm;
#pragma unroll
          for (int k4 = 0; k4 < TC_KC / 8; ++k4) {
            const uint64_t o = (uint64_t)(k4 * 32) >> 4;
            const uint32_t acc = (c | k4) ? 1u : 0u;
            mma_tf32(td, ha + o, hb + o, id[g], acc);
            mma_tf32(td, ha + o, lb + o, id[g], 1u);
            mma_tf32(td, la + o, hb + o, id[g], 1u);
          }
        }
        tc_commit(&empty[s]);
      }
      if (ok) tc_commit(accfull);
      tc_commit(done);
      wait_bar(done, 0, abort);
    }
    __syncwarp();
  } else {
    // splitters: rows [0, n1p) of the chunk (rows n1p.. are only read into accumulator rows
    // that are never stored)
    const int ct = threadIdx.x - 64;
    const int nv4 = n1p * TC_KC / 4;
    for (int c = 0; c < nchunks && !*abort; ++c) {
      const int s = c % TS_S;
      if (!wait_bar(&full[s], (uint32_t)((c / TS_S) & 1), abort)) break;
      unsigned char* st = base + (size_t)s * TS_STAGE;
      float4* hi = reinterpret_cast<float4*>(st);
      float4* lo = reinterpret_cast<float4*>(st + (size_t)ROWS * 128);
      for (int i = ct; i < nv4; i += 32 * TS_SPLIT_W) {
        float4 v = hi[i], h, l;
        tf32_split(v.x, h.x, l.x); tf32_split(v.y, h.y, l.y);
        tf32_split(v.z, h.z, l.z); tf32_split(v.w, h.w, l.w);
        hi[i] = h; lo[i] = l;
      }
      fence_proxy_async_smem();
      mbar_arrive(&conv[s]);
    }
    if (warp >= 4 && warp < 8) {
      // partial blocks out: gpart[sp][row][col] (row-major, n1p x n1p FP32); row block a holds
      // columns 128 a ..
      const int wq = warp - 4;
      bool okw = nchunks > 0 ? wait_bar(accfull, 0, abort) : false;
      okw = __all_sync(0xffffffffu, okw);
      float* outp = gpart + (long long)sp * n1p * n1p;
      for (int g = 0; g < ntg; ++g) {
        const int row = tg[g].a * TC_M + wq * 32 + lane;
        const int cb = tg[g].cs;                     // first column of the target
        const uint32_t tb = tmem + (uint32_t)tg[g].tm + ((uint32_t)(wq * 32) << 16);
        for (int c0 = 0; c0 < tg[g].N; c0 += 32) {
          float v[32];
          if (okw) {
            tc_fence_after();
            tmem_ld32(tb + (uint32_t)c0, v);
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = 0.f;
          }
          if (row < n1p) {
            float* o = outp + (long long)row * n1p + cb + c0;
#pragma unroll
            for (int i = 0; i < 32; ++i)
              if (c0 + i < tg[g].N && cb + c0 + i < n1p) o[i] = v[i];
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, 512);
  if (threadIdx.x == 0 && *abort) const_cast<Ctl*>(ctl)->status = 5;
}

// G (n_k x n_k, FP64, column-major) = sum over the K splits of the partial blocks. Block: 32
// consecutive entries of G (lanes) x 8 warps; warp w sums the splits w, w + 8, ... in FP64 and
// the 8 warp sums are added in warp order (a fixed summation order). Entry (i, j) is read as
// partial (j, i) (consecutive lanes, consecutive i: contiguous) when the 128-row block of i is
// not left of that of j, else as partial (i, j) (the mirror, held by the row block of i).
constexpr int SR_W = 8;
constexpr int SR_SMAX = 160;   // K splits (grid of k_tc_syrk) at most
__global__ void __launch_bounds__(32 * SR_W) k_syrk_reduce(const Ctl* ctl, int k, const float* gpart,
                                                          int S, double* G) {
  if (ctl->status) return;
  if (!tc_gram_ok(ctl, k)) return;
  const int n1 = ctl->n[k];
  const int n1p = (n1 + 15) / 16 * 16;
  const long long plane = (long long)n1p * n1p;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __shared__ double red[SR_W][33];
  const long long L = (long long)blockIdx.x * 32 + lane;
  const bool live = L < (long long)n1 * n1;
  double acc = 0.0;
  long long off = 0;
  if (live) {
    const int i = (int)(L % n1), j = (int)(L / n1);
    const bool direct = (i / TC_M) >= (j / TC_M);
    off = direct ? (long long)j * n1p + i : (long long)i * n1p + j;
    // every partial of this warp's splits is loaded before the first add (one round of L2
    // latency rather than one per split)
    constexpr int PER = (SR_SMAX + SR_W - 1) / SR_W;
    float v[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int sp = wid + u * SR_W;
      v[u] = sp < S ? gpart[sp * plane + off] : 0.f;
    }
    double a0 = 0.0, a1 = 0.0;
#pragma unroll
    for (int u = 0; u + 1 < PER; u += 2) { a0 += (double)v[u]; a1 += (double)v[u + 1]; }
    if (PER & 1) a0 += (double)v[PER - 1];
    acc = a0 + a1;
  }
  red[wid][lane] = acc;
  __syncthreads();
  if (wid == 0 && live) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < SR_W; ++w) t += red[w][lane];
    G[L] = t;   // L = j n1 + i: column-major
  }
}

cudaError_t launch_tc_gram(const Ctl* ctl, int k, const TcProjMaps& m, int n1, double* gpart,
                           double* G, int nsm, cudaStream_t st) {
  const int S = nsm > 0 ? (nsm < SR_SMAX ? nsm : SR_SMAX) : 1;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tc_syrk<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TsCfg<256>::SMEM);
    cudaFuncSetAttribute(k_tc_syrk<TS_NMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TsCfg<TS_NMAX>::SMEM);
    attr = true;
  }
  float* gp = reinterpret_cast<float*>(gpart);
  const int n1p = (n1 + 15) / 16 * 16;
  if (n1p <= 256) k_tc_syrk<256><<<S, TS_NT, TsCfg<256>::SMEM, st>>>(ctl, k, m.eta, gp);
  else k_tc_syrk<TS_NMAX><<<dim3(S, 2), TS_NT, TsCfg<TS_NMAX>::SMEM, st>>>(ctl, k, m.eta, gp);
  k_syrk_reduce<<<(n1 * n1 + 31) / 32, 32 * SR_W, 0, st>>>(ctl, k, gp, S, G);
  return cudaGetLastError();
}

}  // namespace tk
